/*
 * tc.h -- C ABI of the GB300 Stokeslet + stresslet treecode.
 *
 * The library evaluates the velocity of eq. (1.3) of Wang, Tlupova and
 * Krasny, "A treecode algorithm for 3D Stokeslets and stresslets"
 * (arXiv:1811.12498):
 *
 *   u_i(x^m) = sum_{n != m} S_ij(x^m, x^n) f_j^n + T_ijl(x^m, x^n) h_j^n nu_l^n
 *
 * with S_ij = delta_ij/r + d_i d_j/r^3 and T_ijl = d_i d_j d_l/r^5
 * (eqs. 1.2a,b, prefactor 1, d = x - y, r = |d|), by the treecode of
 * Section 5 (Algorithm 1): an octree of particle clusters, the MAC
 * r/R <= theta (eq. 5.1), an order-p Cartesian Taylor far field built from
 * the Coulomb-coefficient recurrence (3.2) and contracted as in
 * eqs. (4.4) and (4.9), and a direct near field (Section 4.1).
 *
 * Conventions for every call:
 *  - Arrays of 3-vectors are FP64 structure-of-arrays in DEVICE memory:
 *    component a of item n is at ptr[a * count + n].  The caller owns every
 *    array it passes; the library only reads inputs and writes outputs.
 *  - The library owns everything reachable from a tc_ctx (tree, moments,
 *    interaction lists, scratch) and frees it in tc_destroy.
 *  - Work is enqueued on the context's CUDA stream (tc_config.stream,
 *    NULL = legacy default stream).  Calls that must size buffers
 *    (tc_build, tc_eval) synchronise that stream internally.  Inside a
 *    context some work also runs on a second, library-owned stream (the
 *    moment passes, the contraction tables and the far field), forked from
 *    and joined back to the context's stream by events: everything a call
 *    reads from the caller's arrays is read on the context's stream, and
 *    every result a call writes to them (u, the gradients) is complete in
 *    the context's stream order.
 *  - No call aborts or prints.  Every failure returns a status; the message
 *    is available from tc_last_error.  Kernels report through a device flag
 *    word that the next synchronising call (or tc_sync) reads (TC_EDEVICE).
 *    The one check that writes it, the MAC traversal's stack bound (176
 *    entries), is a guard only: a walk of a tree of depth <= 21 holds at
 *    most 7 * 21 + 8 = 155 entries, so no input reaches it.
 *  - Pairs with |x - y| == 0 contribute nothing.  When targets are the
 *    sources this is the n != m exclusion of eq. (1.3).
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_ctx tc_ctx;

typedef enum {
    TC_OK = 0,
    TC_EINVAL = 1,   /* an argument is out of range or a pointer is NULL       */
    TC_ENOMEM = 2,   /* a device or host allocation failed                      */
    TC_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
    TC_ESTATE = 4,   /* calls out of order, e.g. tc_eval before tc_moments      */
    TC_ETIMEOUT = 5, /* reserved for a bounded device-side wait; no kernel here
                      * waits on another block or a flag (work queues take
                      * items by atomics only), so it is never returned      */
    TC_EDEVICE = 6   /* a device-side check failed (message says which)        */
} tc_status;

typedef enum {
    /* every stage in FP64 */
    TC_FP64 = 0,
    /* near field, far-field Coulomb-coefficient recurrence and contraction
     * in FP32 (positions split into FP32 hi + lo parts; the FP32 partial
     * sums per source tile and per cluster accumulated by compensated FP32
     * summation and widened to FP64 per leaf and per target); cluster
     * moments and contraction tables always built in FP64.  With
     * tc_config.rec64 the recurrence runs in FP64 for p >= 8. */
    TC_MIXED = 1
} tc_precision;

typedef struct {
    int32_t precision; /* tc_precision                                         */
    int32_t shrink;    /* 1: cluster centre = centre of the tight bounding box
                        *    of its particles (test case 1 of Section 6);
                        * 0: centre of the octree cell                         */
    void* stream;      /* cudaStream_t the context enqueues on; NULL = default */
    int32_t rec64;     /* TC_MIXED only: 1 = far-field recurrence in FP64 for
                        * p >= 8 (the contraction stays FP32); 0 = FP32, the
                        * default, as accurate on the folded tables          */
    int32_t reserved1; /* must be 0                                            */
    double reg_eps;    /* 0: the kernels of eqs. (1.2a,b).  > 0: regularized
                        * Stokeslet and stresslet with this eps (the blob of
                        * Cortez, Fauci and Medovikov, Phys. Fluids 17, 2005;
                        * the paper names regularized kernels as future work):
                        * with s = r^2 + eps^2,
                        *   S^eps_ij = (delta_ij (r^2 + 2 eps^2) + d_i d_j) / s^(3/2),
                        *   T^eps_ijl = (d_i d_j d_l + (eps^2/2)(delta_ij d_l
                        *               + delta_jl d_i + delta_il d_j)) / s^(5/2),
                        * the same tree, MAC, moments and lists; far and near
                        * fields as the precision mode says, the far field on
                        * the full (unfolded) tables, since the harmonic
                        * folding does not hold for eps > 0 (TC_MIXED with
                        * rec64 at p >= 8: far field in FP64).
                        * Not available for tc_adjoint, tc_tune and batches.  */
} tc_config;

/* Create a context.  cfg may be NULL (TC_MIXED, shrink = 1, default stream).
 * *out receives the handle, or NULL on failure.  The CUDA device current on
 * the calling thread is the context's device. */
tc_status tc_create(tc_ctx** out, const tc_config* cfg);

/* Free a context and every device buffer it owns.  NULL is accepted. */
tc_status tc_destroy(tc_ctx* ctx);

/* Message of the last failure on ctx (or of the last context-free call on
 * this thread when ctx is NULL).  Never NULL; valid until the next call. */
const char* tc_last_error(const tc_ctx* ctx);

/* Wait for the context's stream and report any device-side failure. */
tc_status tc_sync(tc_ctx* ctx);

/*
 * Build the octree of Section 5 over N source positions.
 *  x  : device, 3*N FP64, SoA.  Read during the call only (positions are
 *       copied into Morton order).
 *  N  : 1 <= N < 2^31.
 *  N0 : maximum number of particles in a leaf, >= 1 (Section 6 uses 2000).
 * Root: the cube with the per-axis minimum corner and side equal to the
 * largest axis extent.  Cells follow 21-bit quantised coordinates; a cell
 * is split into its non-empty octants while it holds more than N0 particles
 * and is above depth 21.  Cluster centres and radii (r = max distance from
 * the centre to the cluster's particles, Section 2) are computed here.
 * Invalidates moments and interaction lists.  Synchronises the stream.
 */
tc_status tc_build(tc_ctx* ctx, const double* x, int64_t N, int32_t N0);

/*
 * Cluster moments (Section 2) for every cluster:
 *   M_j^k = sum_{n in C} (y^n - y_c)^k f_j^n,
 *   M~_jl^k = sum_{n in C} (y^n - y_c)^k h_j^n nu_l^n,   ||k|| <= p,
 * computed in FP64 and held in a flattened graded order (Section 6.1.1).
 *  f, h, nu : device, 3*N FP64 SoA each, in the caller's particle order.
 *  p        : 0 <= p <= 12.
 * Requires tc_build.  Enqueued only (no synchronisation).
 */
tc_status tc_moments(tc_ctx* ctx, const double* f, const double* h, const double* nu, int32_t p);

/*
 * Treecode velocity (Algorithm 1) at M targets.
 *  targets : device, 3*M FP64 SoA, or NULL to evaluate at the sources
 *            themselves (then M must equal N and u is in the source order).
 *  theta   : MAC parameter, 0 < theta < 1 (eq. 5.1).
 *  p       : Taylor order, 0 <= p <= the order given to tc_moments.
 *  u       : device, 3*M FP64 SoA, written.
 * Every target makes exactly the far/near decisions of Algorithm 1: the MAC
 * is tested per target in FP64.  Synchronises the stream once to size the
 * interaction lists.
 */
tc_status tc_eval(tc_ctx* ctx, const double* targets, int64_t M, double theta, int32_t p, double* u);

/*
 * tc_build + tc_moments + tc_eval (targets = the particles) from HOST
 * arrays, for callers without device memory of their own.
 *  x, f, h, nu : host, 3*N FP64 SoA each, in the caller's particle order;
 *                pinned (page-locked) memory gives asynchronous copies,
 *                pageable memory works too.  Read during the call only.
 *  N, N0, theta, p : as for tc_build, tc_moments and tc_eval; all checked
 *                before anything is copied or enqueued.
 *  u           : host, 3*N FP64 SoA, written.
 * The inputs are copied into library-owned device buffers on the context's
 * stream, the three calls run on them, u is copied back, and the stream is
 * synchronised (u is complete on return; a device-side failure is reported
 * as by tc_sync).  Afterwards the context holds the tree, moments and lists
 * as after the three calls, so tc_adjoint (with device arrays) may follow.
 */
tc_status tc_velocity_host(tc_ctx* ctx, const double* x, const double* f, const double* h, const double* nu,
                           int64_t N, int32_t N0, double theta, int32_t p, double* u);

/*
 * Adjoint of the last tc_eval with its structure frozen.  For
 *   L = sum_m g^m . u(x^m)
 * it returns dL/df, dL/dh, dL/dnu, dL/dx and dL/dt while the tree (cluster
 * membership, centres y_c and radii), every target's far/near decisions and
 * the Taylor order p of that tc_eval are held fixed; this is the exact
 * derivative of the discrete map that tc_eval computes, up to rounding.
 * (The paper does not differentiate the method; the formulas follow from
 * eqs. (1.3), (2.9), (3.2) and Section 4.1 by the chain rule.)
 *  g       : device 3*M FP64 SoA in the target order of the last tc_eval.
 *  grad_f, grad_h, grad_nu : device 3*N FP64 SoA (caller's source order),
 *            written; any may be NULL.
 *  grad_x  : device 3*N FP64 or NULL.  Derivative with respect to the
 *            source positions; when the last tc_eval had targets = NULL it is
 *            the total derivative with respect to the particle positions.
 *  grad_t  : device 3*M FP64 or NULL: derivative with respect to the target
 *            positions of a tc_eval with disjoint targets; must be NULL when
 *            the targets were the sources.
 * The source-side far-field term is accumulated per cluster with FP64
 * atomics, so repeated calls agree to FP64 rounding, not bit for bit.
 * Requires tc_eval.  Synchronises the stream the first time after a tc_eval
 * (its interaction lists are sorted by cluster).
 */
tc_status tc_adjoint(tc_ctx* ctx, const double* g, double* grad_f, double* grad_h, double* grad_nu, double* grad_x,
                     double* grad_t);

/*
 * Frozen-structure re-evaluation (for finite differences of the adjoint, or
 * any caller that moves the particles slightly and wants the map tc_adjoint
 * differentiates).  The paper has no counterpart.
 * tc_update_positions: replace the particle positions (device, 3*N FP64
 * SoA, caller's order) after a tc_eval with targets = NULL, keeping the
 * tree's cells, cluster centres and radii and that tc_eval's interaction
 * lists (its far/near decisions); the moments about the unchanged centres
 * and the contraction tables are recomputed.  Enqueued only.
 * tc_eval_frozen: the velocity at the (moved) particles with those lists,
 * written to u (device, 3*N FP64 SoA, caller's order).  Coincident pairs are
 * skipped by r = 0, as for disjoint targets.  The result equals Algorithm 1
 * when no position moved.  A later tc_eval makes new decisions at the moved
 * positions but keeps the old centres and radii (a moved particle may lie
 * outside its cluster's radius, which weakens the MAC's error bound);
 * tc_build starts afresh.
 */
tc_status tc_update_positions(tc_ctx* ctx, const double* x);
tc_status tc_eval_frozen(tc_ctx* ctx, double* u);

/*
 * Direct O(N*M) sum of eq. (1.3) (with the contraction of Section 4.1).
 *  x, f, h, nu : device, 3*N FP64 SoA.  targets: device 3*M SoA or NULL
 *  (targets = sources, M must equal N).  u: device 3*M FP64 SoA, written.
 *  precision   : TC_FP64 or TC_MIXED (FP32 pair terms on hi/lo positions).
 *  stream      : cudaStream_t or NULL.
 * Allocates its scratch with stream-ordered cudaMallocAsync and frees it
 * before returning; enqueued only.
 */
tc_status tc_direct(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                    const double* targets, int64_t M, int32_t precision, void* stream, double* u);

/*
 * tc_direct with the regularized kernels of tc_config.reg_eps (eps > 0,
 * finite): the reference sum for the regularized treecode.  Pairs with
 * |x - y| == 0 are skipped as in tc_direct.  Same arrays, precision modes,
 * scratch and stream behaviour as tc_direct.
 */
tc_status tc_direct_reg(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                        const double* targets, int64_t M, double eps, int32_t precision, void* stream, double* u);

/*
 * tc_direct without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * on their own, for example a host application whose device memory is owned
 * by a framework pool that forbids allocations from third-party libraries,
 * or a latency-sensitive caller that cannot pay for an allocator call (an
 * allocation may wait for the device or grow a memory pool) on its path.
 *
 * Same arguments, layouts, results and precision modes as tc_direct.  The
 * scratch (the FP32 source pack of TC_MIXED, 64 B per source, and the
 * per-split partial sums, 24 B per target per split) lives in one fixed
 * array of TC_DIRECT_NOALLOC_SCRATCH_BYTES of device memory that is part of
 * the library image: every device that loads the library holds it until
 * the process exits.  A problem whose scratch does not fit even unsplit
 * (64 B * N, rounded up to 256 B, in TC_MIXED, plus 24 B * M) is rejected
 * with TC_EINVAL and a message that says so, before anything is enqueued;
 * otherwise the source range is split into as many chunks as fit.
 *
 * No cudaMalloc, cudaFree or other allocating routine is called.  The first
 * call on a device looks up the array's device address once for that device
 * (with that device current); make that first call before any stream
 * capture.  The address is kept for the life of the process: a
 * cudaDeviceReset (or any other destruction of the device's primary context)
 * unloads the library's device image and makes it stale, so do not call
 * tc_direct_noalloc on a device after resetting it in the same process.  All calls on a device share the one array and it keeps the last
 * call's contents; every scratch word a call reads is first written by the
 * same call, so nothing needs clearing, but calls whose kernels overlap on
 * the GPU (different streams, no ordering between them) race on the array
 * and give wrong results.  Enqueued only.
 */
#define TC_DIRECT_NOALLOC_SCRATCH_BYTES (64ull << 20)
tc_status tc_direct_noalloc(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                            const double* targets, int64_t M, int32_t precision, void* stream, double* u);

/*
 * Interaction counts of the last tc_eval (host outputs, any may be NULL):
 *  near_pairs       : sum over targets of the sizes of the leaves summed directly
 *  far_interactions : number of (target, cluster) far-field evaluations
 *  clusters         : number of clusters in the tree
 */
tc_status tc_stats(tc_ctx* ctx, int64_t* near_pairs, int64_t* far_interactions, int64_t* clusters);

/*
 * Interaction-list sizes of the last tc_eval (host outputs, any may be NULL):
 *  far_entries         : (batch, cluster) far-field list entries; a batch is 32
 *                        targets, so far_interactions / (32 far_entries) is the
 *                        fraction of far-kernel lanes doing useful work
 *  near_entries        : (batch, leaf) near-field list entries
 *  near_entry_sources  : sum over near entries of the leaf size; near_pairs /
 *                        (32 near_entry_sources) is the near-kernel lane use
 */
tc_status tc_list_stats(tc_ctx* ctx, int64_t* far_entries, int64_t* near_entries, int64_t* near_entry_sources);

/*
 * Per-target counts of the last tc_eval, in the target order of that call
 * (device int64 arrays of M entries, any may be NULL): number of far
 * clusters and number of near-field source particles examined.
 */
tc_status tc_eval_counts(tc_ctx* ctx, int64_t* nfar, int64_t* nnear_pairs);

/* ---------------------------------------------------------------------- */
/* Parameters for a target accuracy.                                      */
/* ---------------------------------------------------------------------- */
/*
 * The fastest (theta, p, N0) of a grid whose error reaches target_E on the
 * caller's own system.  Section 6 of the paper closes with the remark that
 * choosing these three for the accuracy wanted would make the method more
 * efficient, and its Table 1 shows the best theta moving with the accuracy
 * regime (0.8 for low, 0.5 for medium, 0.2 for high accuracy).
 *
 *  x, f, h, nu        : the system, FP64 SoA device arrays of N particles;
 *                       the targets are the particles themselves
 *  thetas, n_theta    : candidate MAC parameters, each in (0, 1)   (host)
 *  orders, n_order    : candidate orders p, each in [0, 12]        (host)
 *  leaf_sizes, n_leaf : candidate leaf sizes N0 >= 1                (host)
 *  sample, n_sample   : indices in [0, N) of the particles at which
 *                       the error is measured, 1 <= n_sample <= N   (host)
 *  target_E           : the accuracy wanted, > 0
 *  seconds, errors    : host outputs, one entry per candidate
 *                       k = (i_leaf * n_order + i_order) * n_theta + i_theta:
 *                       device time of tc_build + tc_moments + tc_eval (the
 *                       second of two full runs, CUDA events on the context's
 *                       stream), and E, the relative L2 error of Section 6
 *                       over the sample, against the FP64 direct sum
 *  best               : host output, the candidate of smallest time among
 *                       those with E <= target_E, or -1 if there is none
 *
 * Runs in the context's precision mode; afterwards the context holds the tree,
 * moments and lists of the last candidate.  Synchronises.  TC_EINVAL for a
 * NULL pointer, an empty grid or a value out of range, before anything runs.
 */
tc_status tc_tune(tc_ctx* ctx, const double* x, const double* f, const double* h, const double* nu, int64_t N,
                  const double* thetas, int32_t n_theta, const int32_t* orders, int32_t n_order,
                  const int32_t* leaf_sizes, int32_t n_leaf, const int64_t* sample, int64_t n_sample,
                  double target_E, double* seconds, double* errors, int32_t* best);

/* ---------------------------------------------------------------------- */
/* Batches of independent systems.                                        */
/* ---------------------------------------------------------------------- */
/*
 * A batch evaluates many independent particle systems (each its own eq. (1.3)
 * with targets = sources) together.  Arrays are segmented FP64 SoA in device
 * memory: with ntot = offsets[nsys], component a of particle i of system s
 * is at ptr[a * ntot + offsets[s] + i].  offsets is a HOST array of nsys + 1
 * entries, offsets[0] = 0, strictly increasing.  Every system uses the
 * batch's tc_config; the batch owns one context per system.
 *
 * tc_batch_eval runs, after preparing every system's interaction lists, the
 * far field, the near field and the final sum of all systems as one
 * persistent far kernel, one persistent near kernel and one finalize: warps
 * take (system, batch of 32 targets) items from a device counter until the
 * queue is empty.  That phase is captured into a CUDA graph on the first call
 * and replayed while the output pointer, the order p, the launch shapes and
 * the systems' buffers are unchanged.  Launch shapes come from an autotuner
 * that times candidate shapes on the first evaluation at each order.
 */
typedef struct tc_batch tc_batch;

tc_status tc_batch_create(tc_batch** out, const tc_config* cfg);
tc_status tc_batch_destroy(tc_batch* b);
const char* tc_batch_last_error(const tc_batch* b);
/* autotune (default 1) and CUDA-graph replay (default 1) switches */
tc_status tc_batch_set(tc_batch* b, int32_t autotune, int32_t use_graph);
/* tc_build of every system (x segmented, see above); synchronises */
tc_status tc_batch_build(tc_batch* b, const double* x, int32_t nsys, const int64_t* offsets, int32_t N0);
/* tc_moments of every system (f, h, nu segmented) */
tc_status tc_batch_moments(tc_batch* b, const double* f, const double* h, const double* nu, int32_t p);
/* velocity of every system at its own particles into u (segmented 3 x ntot) */
tc_status tc_batch_eval(tc_batch* b, double theta, int32_t p, double* u);
/* the same result by one ordinary tc_eval per system (u_sys: host array of
 * nsys device pointers, system s writes a 3 x n_s SoA array); for comparison */
tc_status tc_batch_eval_separate(tc_batch* b, double theta, int32_t p, double* const* u_sys);
/* chosen launch shapes {far warps/block, far blocks, near warps/block, near
 * blocks} (0 blocks = occupancy limit) and the tuned kernels' times in ms */
tc_status tc_batch_info(tc_batch* b, int32_t* shape, float* tune_ms);
/* context of system s (owned by the batch), e.g. for tc_stats; NULL if out of range */
tc_ctx* tc_batch_system(tc_batch* b, int32_t s);

/* ---------------------------------------------------------------------- */
/* Tracing.                                                               */
/* ---------------------------------------------------------------------- */

/* Phases timed with CUDA events on the context's stream. */
typedef enum {
    TC_PH_BUILD = 0,    /* tc_build: keys, sort, topology, geometry          */
    TC_PH_MOMENTS = 1,  /* tc_moments: weight gather, leaf moments, upward pass */
    TC_PH_TABLES = 2,   /* contraction tables (first tc_eval at an order)    */
    TC_PH_TARGETS = 3,  /* tc_eval: keys and sort of disjoint targets        */
    TC_PH_LISTS = 4,    /* tc_eval: MAC traversal, both passes and scans     */
    TC_PH_FAR = 5,      /* tc_eval: far-field kernel                         */
    TC_PH_NEAR = 6,     /* tc_eval: near-field kernel                        */
    TC_PH_FINAL = 7,    /* tc_eval: sum and scatter to the caller's order    */
    TC_PH_ADJ_FAR_T = 8,   /* tc_adjoint: far field, target side (dL/dx of targets)  */
    TC_PH_ADJ_FAR_S = 9,   /* tc_adjoint: far field, source side (adjoint tables)    */
    TC_PH_ADJ_NEAR_T = 10, /* tc_adjoint: near field, target side                    */
    TC_PH_ADJ_NEAR_S = 11, /* tc_adjoint: near field, source side                    */
    TC_PH_ADJ_REST = 12,   /* tc_adjoint: adjoint moments, downward pass and
                            * per-particle evaluation (second stream)            */
    TC_NPHASES = 13
} tc_phase;

/* Enable (1) or disable (0) per-phase event timing on ctx.  Enabling resets
 * the recorded phases.  Costs two event records per phase.  Some phases run
 * on the context's second stream beside others: the moment passes of
 * tc_moments and the far field of tc_eval beside the near field, and the
 * adjoint's moments, downward pass and per-particle evaluation
 * (TC_PH_ADJ_REST) beside its near-field phases; their phase times then
 * overlap.  enable = 2 runs everything on one stream, one phase after the
 * other, so that each phase time is that work's own duration (the result is
 * the same). */
tc_status tc_profile(tc_ctx* ctx, int32_t enable);

/* Durations in ms of the most recent run of each phase (host array of
 * TC_NPHASES; -1 for a phase not run since profiling was enabled).
 * Synchronises the stream. */
tc_status tc_phase_times(tc_ctx* ctx, double* ms);

/* Number of kernels this library has launched in this process so far. */
int64_t tc_kernel_launches(void);

/*
 * Measured arithmetic peak of the current device in TFLOP/s (an FMA counts
 * as two flops), the denominator of a roofline fraction: every thread of a
 * grid of 8 blocks of 256 threads per SM runs 8 independent FMA chains, timed
 * with CUDA events on `stream` (cudaStream_t or NULL), best of 5 launches of
 * about 1 ms after a warm-up, at whatever clock the device runs.
 *  precision : TC_MIXED measures FP32 (the faster of scalar and packed
 *              FP32x2 FMAs), TC_FP64 measures FP64.
 *  tflops    : host output.
 * Synchronises the stream.  The paper has no counterpart (it reports CPU
 * seconds only).
 */
tc_status tc_fma_peak(int32_t precision, void* stream, double* tflops);

/*
 * Host-side fault injection for tests of the out-of-memory path: after
 * `after` further device allocations by this library (across all contexts
 * and threads), every allocation it attempts fails as if the device were out
 * of memory, so the call that needed it returns TC_ENOMEM, until this is
 * called again; after < 0 switches the injection off (the default).  Nothing
 * is done on the device.
 */
void tc_fail_allocations(int64_t after);

/* ---------------------------------------------------------------------- */
/* Inspection of the tree (host outputs; for tests and tools).            */
/* ---------------------------------------------------------------------- */

/* Number of clusters and maximum depth of the last tc_build; root corner
 * lo[3] and side (host pointers, any may be NULL). */
tc_status tc_tree_info(tc_ctx* ctx, int64_t* nnodes, int32_t* depth, double* lo, double* side);

/*
 * Copy per-cluster records to host arrays of nnodes entries (any may be
 * NULL).  Clusters are numbered level by level, children of one parent
 * consecutively in octant order (x bit most significant).
 *  begin, count : particle range in Morton order
 *  level        : depth (root 0); cell: 3*nnodes integer cell coordinates
 *  parent       : parent index (-1 for the root)
 *  first_child, nchild : children are first_child .. first_child+nchild-1
 *  yc           : 3*nnodes cluster centres (x,y,z interleaved per cluster)
 *  rc2          : squared cluster radius
 */
tc_status tc_tree_export(tc_ctx* ctx, int32_t* begin, int32_t* count, int32_t* level, int32_t* cell,
                         int32_t* parent, int32_t* first_child, int32_t* nchild, double* yc, double* rc2);

/* Morton order of the sources (host int32 array of N): entry i is the
 * caller's index of the i-th particle in Morton order. */
tc_status tc_tree_order(tc_ctx* ctx, int32_t* order);

/*
 * Moments of one cluster as host FP64 cubes of order q = p of tc_moments:
 * Mf[(j*(q+1) + k1)*(q+1)^2 + k2*(q+1) + k3] = M_j^k (3 cubes) and
 * Mt[((3j+l)*(q+1) + k1)*(q+1)^2 + ...] = M~_jl^k (9 cubes); entries with
 * ||k|| > q are 0.
 */
tc_status tc_moments_export(tc_ctx* ctx, int64_t node, double* Mf, double* Mt);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
