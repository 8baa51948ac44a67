// Internal declarations shared by the translation units of libtc.
// Not part of the C ABI (see include/tc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/tc.h"

namespace tc {

constexpr int kMaxDepth = 21;   // 21-bit quantised coordinates, 63-bit Morton keys
constexpr int kPMax = 12;       // largest Taylor order accepted
constexpr int kQMax = kPMax + 2;  // far field needs Coulomb coefficients to p+2
constexpr int kBatch = 32;      // targets per interaction list (one warp)
// traversal stack: a preorder walk keeps at most 7 siblings per level plus
// the children of the deepest node, 7 * kMaxDepth + 8 = 155 entries, so the
// kernels' bound check on this size is a guard that no tree of this library
// reaches
constexpr int kStack = 8 * (kMaxDepth + 1);

// number of multi-indices with ||k|| == n, and with ||k|| <= n
__host__ __device__ constexpr int level_size(int n) { return (n + 1) * (n + 2) / 2; }
__host__ __device__ constexpr int ncoef(int n) { return (n + 1) * (n + 2) * (n + 3) / 6; }

// Flattened graded order: level by level; inside a level k1 descending, then
// k2 descending.  With a = k2 + k3 the position inside level n is
// a(a+1)/2 + k3, and the flat index is ncoef(n-1) + that.
__host__ __device__ inline int flat_index(int k1, int k2, int k3)
{
    int n = k1 + k2 + k3, a = k2 + k3;
    return (n > 0 ? ncoef(n - 1) : 0) + a * (a + 1) / 2 + k3;
}

// Compensated (Kahan) FP32 summation: s accumulates, c carries the rounding
// error of the last addition (s - c is the better estimate of the sum).
// Written out so that no reassociation can cancel the compensation (the
// library is built without fast-math).
// 1/sqrt(x) by the special-function unit with subnormal inputs and results
// flushed to zero: the plain rsqrtf adds scaling steps for subnormals on the
// FP32 pipe (12 % of the near field's FP32 instructions).  Pair distances
// whose square is subnormal in FP32 (|d| < 1.1e-19) are out of range of the
// FP32 pair terms anyway (their powers overflow).
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float b)
{
    const float y = b - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Error flags raised by kernels (bit mask in device memory).
enum DevFlag : int {
    kFlagStack = 1,     // traversal stack bound exceeded
};

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

// Cluster centre y_c and squared radius r^2 (32-byte aligned record).
struct __align__(32) Geo {
    double x, y, z, w;
};

// 8-byte list entry: cluster id and the mask of batch lanes it applies to.
struct ListEntry {
    int32_t node;
    uint32_t mask;
};

// Device-side description of one system for the batched (persistent) far,
// near and finalize kernels: the buffers of its context after eval_prepare.
struct SysDesc {
    const double* ts;          // 3*M sorted targets
    int64_t M;
    const Geo* geo;
    const double* invrho;
    const void* ab;            // folded contraction tables (double or float)
    const float4* geo32;       // FP32 cluster geometry of the mixed far kernel
    const int64_t* far_off;
    const ListEntry* far_list;
    double* u_far;
    const int4* topo;
    const float4* spack;
    const double* xs;
    const double* ws;
    int64_t N;
    const int64_t* near_off;
    const ListEntry* near_list;
    double* u_near;
    const int32_t* tperm;      // sorted target -> caller's target index
    int64_t out_off;           // first column of this system in the batched output
    // leaf-major near-field schedule (mixed precision; NearSched)
    const int2* units;
    const int32_t* nunits;
    const int64_t* node_inc0;
    const int32_t* node_A;
    const int32_t* inc_m;
    const int32_t* inc_e;
    double* slots;
    int64_t near_entries;      // sizes the schedule's work was enqueued for
    int64_t nnodes;
};

}  // namespace tc

struct tc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t stream2 = nullptr;     // moment passes and far field, concurrent with the first stream
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_mom = nullptr;
    int mom_pending = 0;                // moment passes enqueued on stream2, not yet joined
    int precision = TC_MIXED;
    int rec64 = 0;  // mixed: FP64 far-field recurrence for p >= 8
    int shrink = 1;
    std::string err;

    // ---- tree (tc_build)
    int built = 0;
    int64_t N = 0;
    int N0 = 0;
    int depth = 0;
    int64_t nnodes = 0;
    std::vector<int64_t> level_begin;  // node index where each level starts (+ end)
    double lo[3] = {0, 0, 0}, side = 0;
    tc::DevBuf root;                    // double[8]: lo[3], side, scale
    tc::DevBuf bbox_part;               // per-block min/max partials
    tc::DevBuf keys, keys_alt;          // uint64 Morton keys
    tc::DevBuf perm, perm_alt;          // int32 permutation (Morton -> caller)
    tc::DevBuf hist;                    // radix histograms
    tc::DevBuf xs;                      // 3*N FP64 sorted positions
    tc::DevBuf node_topo;               // int4 {begin, count, first_child, nchild}
    tc::DevBuf node_info;               // int4 {level, parent, 0, 0}
    tc::DevBuf node_key;                // uint64 Morton prefix
    tc::DevBuf node_geo;                // Geo {yc, rc2}
    tc::DevBuf node_invrho;             // double 1/rho (rho = r, or 1 if r == 0)
    tc::DevBuf node_geof;               // float4 x2: (y_c hi, fl32(rc2)), (y_c lo, 0) for the MAC screen
    tc::DevBuf geo_tmp;                 // geometry scratch (per-cluster accumulators, item map)
    tc::DevBuf split_cnt, split_off;    // per-level scan buffers
    tc::DevBuf scan_tmp;                // device scalar(s)

    // ---- moments (tc_moments)
    int have_moments = 0;
    int p_mom = -1;
    tc::DevBuf ws;                      // 9*N FP64 sorted weights: f(3) h(3) nu(3)
    tc::DevBuf spack;                   // MIXED source pack: 4 float4 per source
    tc::DevBuf mom;                     // FP64 [node][12][ncoef(p)]
    tc::DevBuf mom_tmp;                 // leaf-pass scratch: item map and per-item partial moments
    tc::DevBuf m2m_tmp;                 // upward-pass scratch: shifted moments per child of one level
    int ab_p = -1;                      // order the contraction tables were built for
    tc::DevBuf ab64;                    // FP64 [node][ncoef(p+2)][12]
    tc::DevBuf ab32;                    // FP32 [node][ncoef(p+2)][12]
    tc::DevBuf abf64, abf32;            // folded tables [node][(p+3)^2][12], level n times lambda_n
    tc::DevBuf geo32;                   // mixed: per node (y_c hi, 1/rho), (y_c lo, 0) as float4
    tc::DevBuf reg_et;                  // regularized kernels: FP64 [node][ncoef(p+1)][3] eps^2 table
    tc::DevBuf reg_et32;                // its FP32 copy (mixed precision)
    double reg_eps = 0.0;               // > 0: regularized kernels (tc_config.reg_eps)
    int64_t* host_words = nullptr;      // pinned: far and near list totals, device flags
    int counted = 0;                    // eval_prepare_count done, finish pending
    double pending_theta = 0.0;
    int pending_p = 0;
    const double* pending_ts = nullptr;
    int64_t pending_M = 0;

    // ---- evaluation (tc_eval)
    int64_t M = 0;
    int eval_self = 1;
    int moved = 0;                      // positions replaced by tc_update_positions since tc_build
    tc::DevBuf tkeys, tkeys_alt, tperm, tperm_alt;  // disjoint targets
    tc::DevBuf ts;                      // 3*M FP64 sorted targets
    tc::DevBuf host_in, host_u;         // tc_velocity_host: device copies of x, f, h, nu (12*N) and of u (3*N)
    tc::DevBuf nfar_e, nnear_e;         // per batch entry counts (int32)
    tc::DevBuf far_off, near_off;       // per batch exclusive offsets (int64)
    tc::DevBuf far_list, near_list;     // ListEntry
    tc::DevBuf cnt_far, cnt_near;       // per sorted target counts (int64)
    tc::DevBuf u_far, u_near;           // 3*M FP64 sorted order
    // near entries sorted by leaf (keys, entry index, batch of each entry;
    // the adjoint's source side), and the leaf-major near-field schedule
    // (near_schedule): per node its incidence count, sort key and order, the
    // counts and first incidences in that order, its first incidence and fill
    // cursor, units per node and their offsets, the units, per incidence target
    // and entry, and the slots of the leaf sums
    tc::DevBuf nl_keys, nl_keys_alt, nl_idx, nl_idx_alt, nl_eb, nl_hist;
    tc::DevBuf nl_nA, nl_nkey, nl_nkey_alt, nl_nord, nl_nord_alt, nl_sA, nl_inc0s, nl_ninc0, nl_cur;
    tc::DevBuf nl_ucnt, nl_uoff, nl_units, nl_inc_m, nl_inc_e, nl_slots;
    int near_sched_ready = 0;  // bit 1: entries sorted, bit 2: schedule built (for the lists of the last tc_eval)
    tc::DevBuf flags;                   // int32 device error flags at byte 0; work-queue counters
                                        // of the far field (byte 128) and its adjoint's target side (192)
    int64_t far_entries = 0, near_entries = 0;  // list sizes of the last tc_eval
    int p_eval = -1;                            // order of the last tc_eval
    int prepared = 0;                           // lists ready for the far/near kernels
    int have_eval = 0;

    // ---- adjoint (tc_adjoint)
    tc::DevBuf adj_fkeys, adj_fkeys_alt, adj_fidx, adj_fidx_alt, adj_febatch;  // far entries sorted by cluster
    tc::DevBuf adj_hist;
    tc::DevBuf adj_scnt, adj_soff;        // near source side: units per leaf and their offsets
    tc::DevBuf adj_gs, adj_gt;            // 3*M sorted g and target-position gradient
    tc::DevBuf adj_abar;                  // FP64 [node][ncoef(p+2)][12] adjoint of the tables
    tc::DevBuf adj_fbar;                  // FP64 [node][(p+3)^2][12] adjoint of the folded tables (mixed)
    tc::DevBuf adj_lam, adj_lamacc;       // FP64 [node][12][ncoef(p)] adjoint moments, accumulated down
    tc::DevBuf adj_gfar, adj_gnear;       // 12*N FP64 sorted: d/df, d/dh, d/dnu, d/dx
    int adj_lists_ready = 0;              // sorted lists match the last tc_eval

    // ---- phase timing (tc_profile / tc_phase_times)
    int profile = 0;
    cudaEvent_t ev[2 * TC_NPHASES] = {};
    int ev_recorded[TC_NPHASES] = {};
};
namespace tc {
// The second stream and its events, created on first use.
inline cudaError_t second_stream(tc_ctx* ctx)
{
    if (ctx->stream2) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->stream2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_mom, cudaEventDisableTiming);
    return e;
}
// Order the first stream after the moment passes that tc_moments left
// running on the second stream (before anything reads the moments or
// rewrites what those passes read).
inline cudaError_t join_moments(tc_ctx* ctx)
{
    if (!ctx->mom_pending) return cudaSuccess;
    ctx->mom_pending = 0;
    return cudaStreamWaitEvent(ctx->stream, ctx->ev_mom, 0);
}
}  // namespace tc


namespace tc {

// count one kernel launch (process-wide counter read by tc_kernel_launches)
// phase timing: events around a phase when profiling is on (tc_profile)
inline void ph_begin(tc_ctx* ctx, int ph, cudaStream_t s = nullptr)
{
    if (ctx->profile) cudaEventRecord(ctx->ev[2 * ph], s ? s : ctx->stream);
}
inline void ph_end(tc_ctx* ctx, int ph, cudaStream_t s = nullptr)
{
    if (ctx->profile) {
        cudaEventRecord(ctx->ev[2 * ph + 1], s ? s : ctx->stream);
        ctx->ev_recorded[ph] = 1;
    }
}
void note_launch();
// host-side allocation-failure injection (tc_fail_allocations): true when the
// next device allocation must fail as out of memory
bool alloc_should_fail();
cudaError_t run_probe(int kind, cudaStream_t s, double* tflops, double* ms_best);

// tc_eval in two halves (tc_api.cu): lists, then far/near/finalize
tc_status eval_prepare(tc_ctx* ctx, const double* targets, int64_t M, double theta, int p);
// eval_prepare in two halves around the one synchronisation it needs (a batch
// counts every system's lists, synchronises once, then finishes them all)
tc_status eval_prepare_count(tc_ctx* ctx, const double* targets, int64_t M, double theta, int p);
tc_status eval_prepare_finish(tc_ctx* ctx);
tc_status eval_compute(tc_ctx* ctx, double* u);

// Exclusive scan of n values with one block of 1024 threads (in and out may
// be the same array).  A tile is 32 warps x kScanRows rows of 32 values; each
// warp reads its rows with coalesced loads (all of a tile's loads are
// independent, so its latency is paid once per tile), scans each row by
// shuffles with a running carry, the 32 warp sums are scanned by warp 0, and
// the tiles are chained by a running carry.  total (may be NULL) receives the
// sum of all n values.
constexpr int kScanRows = 8;
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(1024) k_scan_tiles(const Tin* in, Tout* out, int64_t n, Tout* total)
{
    constexpr int64_t kTile = 1024 * kScanRows;
    __shared__ Tout wex[32];
    __shared__ Tout ttot;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    Tout carry = 0;
    for (int64_t base = 0; base < n; base += kTile) {
        const int64_t wb = base + (int64_t)w * (32 * kScanRows);
        Tin v[kScanRows];
#pragma unroll
        for (int r = 0; r < kScanRows; r++) {
            const int64_t i = wb + r * 32 + lane;
            v[r] = i < n ? in[i] : (Tin)0;
        }
        Tout ex[kScanRows];  // exclusive prefix inside the warp's rows
        Tout run = 0;
#pragma unroll
        for (int r = 0; r < kScanRows; r++) {
            Tout x = (Tout)v[r];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Tout y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            ex[r] = run + x - (Tout)v[r];
            run += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) wex[w] = run;
        __syncthreads();
        if (w == 0) {
            const Tout t0 = wex[lane];
            Tout y = t0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const Tout z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            wex[lane] = y - t0;
            if (lane == 31) ttot = y;
        }
        __syncthreads();
        const Tout off = carry + wex[w];
#pragma unroll
        for (int r = 0; r < kScanRows; r++) {
            const int64_t i = wb + r * 32 + lane;
            if (i < n) out[i] = off + ex[r];
        }
        carry += ttot;
        __syncthreads();  // wex and ttot are rewritten by the next tile
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// error helpers (tc_api.cu)
tc_status fail(tc_ctx* ctx, tc_status st, const char* fmt, ...);
tc_status cuda_fail(tc_ctx* ctx, cudaError_t e, const char* where);

// grow a device buffer to hold at least `bytes`; contents are not preserved
cudaError_t ensure(DevBuf& b, size_t bytes);
void release(DevBuf& b);

template <typename T>
inline T* ptr(DevBuf& b) { return reinterpret_cast<T*>(b.p); }

// ---- launchers (each returns cudaGetLastError() after enqueueing)
// tc_build.cu
cudaError_t launch_bbox(const double* x, int64_t N, double* part, int nblk, double* root, cudaStream_t s);
cudaError_t launch_keys(const double* x, int64_t N, const double* root, uint64_t* keys, int32_t* idx,
                        int clamp_outside, cudaStream_t s);
int radix_blocks(int64_t N);
cudaError_t radix_sort(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, uint32_t* hist,
                       int64_t N, cudaStream_t s);
cudaError_t radix_sort_bits(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, uint32_t* hist,
                            int64_t N, int bits, cudaStream_t s);
cudaError_t launch_gather3(const double* src, const int32_t* perm, int64_t N, double* dst, cudaStream_t s);
cudaError_t launch_init_root(int4* topo, int4* info, uint64_t* nkey, int64_t N, cudaStream_t s);
cudaError_t launch_split_count(const int4* topo, const int4* info, const uint64_t* keys, int64_t lb, int64_t le,
                               int N0, int32_t* cnt, cudaStream_t s);
cudaError_t launch_scan_i32(const int32_t* in, int32_t* out_excl, int64_t n, int32_t* total, cudaStream_t s);
cudaError_t launch_split_write(int4* topo, int4* info, uint64_t* nkey, const uint64_t* keys, int64_t lb, int64_t le,
                               int N0, const int32_t* off, cudaStream_t s);
cudaError_t launch_geometry(const int4* topo, const int4* info, const uint64_t* nkey, const double* xs, int64_t N,
                            int64_t nnodes, const double* root, int shrink, Geo* geo, double* invrho, float4* geof,
                            void* scratch, cudaStream_t s);
size_t geometry_scratch_bytes(int64_t nnodes);

// tc_moments.cu
cudaError_t launch_gather_weights(const double* f, const double* h, const double* nu, const int32_t* perm,
                                  int64_t N, double* ws, cudaStream_t s);
cudaError_t launch_source_pack(const double* xs, const double* ws, int64_t N, float4* pack, cudaStream_t s);
// scratch bytes of launch_moments (item map and per-item partial moments)
size_t moments_scratch_bytes(int64_t N, int64_t nnodes, int p);
// leaf moments of every leaf; blocks_per_sm sizes the leaf pass's resident
// grid (0: one block per item)
cudaError_t launch_moments(const int4* topo, const Geo* geo, const double* xs, const double* ws, int64_t N,
                           int64_t nnodes, int p, double* mom, void* scratch, int blocks_per_sm, cudaStream_t s);
// upward pass of one level [lb, le) whose children start at cb; shifted:
// scratch of m2m_scratch_bytes (one slot of moments per child of the level)
cudaError_t launch_m2m(const int4* topo, const Geo* geo, int64_t lb, int64_t le, int64_t cb, int p, double* mom,
                       double* shifted, cudaStream_t s);
cudaError_t launch_ab_tables(const double* mom, const double* invrho, int64_t nnodes, int pm, int p, double* ab64,
                             float* ab32, cudaStream_t s);
cudaError_t launch_eps_table(const double* mom, const double* invrho, int64_t nnodes, int pm, int p, double eps,
                             double* et, cudaStream_t s);
cudaError_t launch_fold_tables(const double* ab64, int64_t nnodes, int p, double* abf64, float* abf32,
                               const Geo* geo, const double* invrho, float4* geo32, cudaStream_t s);

// Subset of multi-indices with k1 <= 1 ("harmonic basis"): level n has 2n+1
// of them, level n starts at n^2; inside a level, (0, n-k3, k3) is at k3 and
// (1, n-1-k3, k3) at n+1+k3.
__host__ __device__ constexpr int hsize(int P) { return (P + 1) * (P + 1); }

// tc_lists.cu
cudaError_t launch_lists(const double* ts, int64_t M, const int4* topo, const Geo* geo, const float4* geof,
                         float scale2, double theta, int write, int32_t* nfar_e, int32_t* nnear_e,
                         const int64_t* far_off, const int64_t* near_off, ListEntry* far_list, ListEntry* near_list,
                         int64_t* cnt_far, int64_t* cnt_near, int32_t* flags, cudaStream_t s);
cudaError_t launch_scan_i32_to_i64(const int32_t* in, int64_t* out_excl, int64_t n, int64_t* total,
                                   cudaStream_t s);
cudaError_t launch_sum_i64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t s);
cudaError_t launch_sum_entry_sizes(const ListEntry* list, int64_t n, const int4* topo, int64_t* out, cudaStream_t s);
// Sort the n entries of a list by cluster (stable): keys = cluster, idx =
// entry index, in sorted order; eb = batch of each entry, by entry index.
cudaError_t sort_list_entries(const ListEntry* list, int64_t n, const int64_t* off, int64_t nbatch, int64_t nnodes,
                              DevBuf& keys, DevBuf& keys_alt, DevBuf& idx, DevBuf& idx_alt, DevBuf& eb,
                              DevBuf& hist, cudaStream_t s);

// tc_far.cu
cudaError_t launch_far(int precision, int rec64, const double* ts, int64_t M, const int4* topo, const Geo* geo,
                       const double* invrho, const float4* geo32, const double* ab64, const float* ab32, int p,
                       const int64_t* far_off,
                       const ListEntry* far_list, double* u_far, unsigned* queue,
                       cudaStream_t s);

cudaError_t launch_far_batched(int precision, int rec64, const SysDesc* sys, int nsys, const int64_t* item_off, int64_t nitems,
                               int p, unsigned long long* counter, int warps_per_block, int blocks, cudaStream_t s);

// tc_near.cu
// The leaf-major schedule of the one-system near field, built once per set
// of near lists by near_schedule: the near entries sorted by leaf, the
// targets of each leaf's entries (its incidences) in that order, and the units
// of work, (leaf, pair of 32-target streams), in order of decreasing leaf size.
struct NearSched {
    const int64_t* node_inc0;  // per node: its first incidence
    const int32_t* node_A;     // per node: its incidences (0 for a node in no near list)
    const int2* units;         // per unit: (node, stream pair)
    const int32_t* nunits;     // device word: the number of units
    const int32_t* inc_m;      // per incidence: sorted target index
    const int32_t* inc_e;      // per incidence: its near-list entry
    double* slots;             // 96 per near entry: leaf sums per (entry, component, lane)
    int64_t E;                 // near entries
    int64_t max_units;         // bound on the number of units
    unsigned* queue;           // device word: the work-queue counter (the caller's)
};
// Build the schedule for the lists of the last tc_eval, unless built already;
// full = 0: sort the near entries by leaf instead (nl_keys, nl_idx, nl_eb).
cudaError_t near_schedule(tc_ctx* ctx, int full, NearSched& sc, cudaStream_t s);
// Its two halves, for a caller that captures the work in a graph: the
// buffers (host side, nothing enqueued), then the work (no allocation).
cudaError_t near_schedule_alloc(tc_ctx* ctx, int full);
cudaError_t near_schedule_build(tc_ctx* ctx, int full, cudaStream_t s);
NearSched near_schedule_desc(tc_ctx* ctx);
// Near field of many systems: FP64, one persistent kernel over the (system,
// batch) items; mixed, the systems' first units (unit_off, nsys + 1, written
// here), one persistent kernel over all units of their schedules (built
// beforehand), and the sums per target of every system.  batch_off: nsys + 1
// offsets of the systems' batches, nbatches in all.
cudaError_t launch_near_batched(int precision, const SysDesc* sys, int nsys, const int64_t* batch_off,
                                int64_t nbatches, int64_t* unit_off, unsigned long long* counter, int warps_per_block,
                                int blocks, cudaStream_t s);
cudaError_t launch_finalize_batched(const SysDesc* sys, int nsys, const int64_t* moff, int64_t mtotal, double* u,
                                    int64_t ntot, cudaStream_t s);
cudaError_t launch_near(int precision, const double* ts, int64_t M, const int4* topo,
                        const double* xs, const double* ws, const float4* spack, int64_t N,
                        const int64_t* near_off, const ListEntry* near_list, double* u_near, int self,
                        const NearSched& sched, double eps, cudaStream_t s);
// tc_reg.cu: far field of the regularized kernels (eps > 0), FP64, on the
// FP64 contraction tables ab64 and the eps^2 table et of launch_eps_table
cudaError_t launch_far_reg(const double* ts, int64_t M, const Geo* geo, const double* invrho, const double* ab64,
                           const double* et, int p, double eps, const int64_t* far_off, const ListEntry* far_list,
                           double* u_far, cudaStream_t s);
// the same in FP32 (mixed precision) on the FP32 tables ab32 and et32
cudaError_t launch_far_reg32(const double* ts, int64_t M, const float4* geo32, const float* ab32, const float* et32,
                             int p, double eps, const int64_t* far_off, const ListEntry* far_list, double* u_far,
                             cudaStream_t s);
// dst = the FP32 rounding of the n FP64 values src (as the FP32 contraction tables are rounded)
cudaError_t launch_narrow_table(const double* src, int64_t n, float* dst, cudaStream_t s);
cudaError_t launch_finalize(const double* u_far, const double* u_near, const int32_t* perm, int64_t M, double* u,
                            cudaStream_t s);
cudaError_t launch_scatter_counts(const int64_t* cs, const int32_t* perm, int64_t M, int64_t* out,
                                  cudaStream_t s);

// tc_direct.cu
// eps > 0: the regularized kernels
cudaError_t launch_direct(int precision, const double* x, const double* f, const double* h, const double* nu,
                          int64_t N, const double* t, int64_t M, double* u, void* scratch, size_t scratch_bytes,
                          double eps, cudaStream_t s);
size_t direct_scratch_bytes(int precision, int64_t N, int64_t M);

}  // namespace tc
