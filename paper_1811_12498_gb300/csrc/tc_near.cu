// Near field: direct summation over the leaves that fail the MAC, in the
// contracted form of Section 4.1:
//   u_i += f_i / r + d_i (s + t),  s = (d.f) / r^3,  t = (d.h)(d.nu) / r^5,
// d = x - y, skipping pairs with r == 0 (the n != m exclusion of eq. 1.3).
//
// Sources are streamed through a per-warp shared-memory tile of 32 records
// (one coalesced load per lane, then broadcast reads).
//
// Mixed precision: positions are split as x = hi + lo (both FP32) and
// d = (x_hi - y_hi) + (x_lo - y_lo), so d keeps FP32 relative accuracy even
// for close pairs; pair terms are FP32; the 32-source tiles' partial sums of
// a leaf are accumulated by compensated (Kahan) FP32 summation and each
// leaf's sum is added to an FP64 per-target accumulator (an FP64 addition per
// tile stalled every tile's end on the slow FP64 pipe).  Work is scheduled
// leaf by leaf (tc_nearpair.cuh): the near entries are sorted by leaf, the
// targets that need a leaf are packed densely into 32-lane streams, and two
// streams share every staged tile, so every broadcast source value feeds two
// targets.  The tile holds the sources in pairs, field by field
// ((y_2q.f, y_2q+1.f) adjacent), and the pair terms run on packed FP32x2
// arithmetic, two sources per instruction.  Each leaf's sums go to a slot
// per (near entry, lane), added per target in list order by a second kernel.
//
// FP64 mode computes everything in FP64, one batch per warp.
#include <algorithm>

#include "tc_nearpair.cuh"

namespace tc {

namespace {

constexpr int kNearWarps = 4;
constexpr int kNearMaxWarps = 8;  // largest block the batched kernel accepts

// ---------------------------------------------------------------------------
// mixed precision: packed FP32x2 arithmetic (tile staging and the group walk
// in tc_nearpair.cuh)

using nearpair::sub2;
using nearpair::kPairStride;
using nearpair::kTileFloat4;

// one target, replicated into both halves of each pair
struct Tgt2 {
    float2 h0, h1, h2, l0, l1, l2;
};

__device__ inline Tgt2 load_target(const double* __restrict__ ts, int64_t M, int64_t m, bool valid)
{
    float h[3] = {0, 0, 0}, l[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            const double v = ts[a * M + m];
            h[a] = __double2float_rn(v);
            l[a] = __double2float_rn(v - (double)h[a]);
        }
    Tgt2 t;
    t.h0 = make_float2(h[0], h[0]), t.h1 = make_float2(h[1], h[1]), t.h2 = make_float2(h[2], h[2]);
    t.l0 = make_float2(l[0], l[0]), t.l1 = make_float2(l[1], l[1]), t.l2 = make_float2(l[2], l[2]);
    return t;
}

// Stokeslet + stresslet terms of one target against source pair tp, both
// sources at once.  kGuard: a source may coincide with the target (r^2 = 0,
// the pair is skipped); without it 1/r comes straight from rsqrt.
template <bool kGuard>
__device__ __forceinline__ void pair_terms(const Tgt2& t, const float4* tp, float2& ax, float2& ay, float2& az)
{
    const float4 A = tp[0], B = tp[1], C = tp[2], D = tp[3], E = tp[4], F = tp[5], G = tp[6], Q = tp[7];
    const float2 dx = __fadd2_rn(sub2(t.h0, make_float2(A.x, A.y)), sub2(t.l0, make_float2(C.x, C.y)));
    const float2 dy = __fadd2_rn(sub2(t.h1, make_float2(A.z, A.w)), sub2(t.l1, make_float2(C.z, C.w)));
    const float2 dz = __fadd2_rn(sub2(t.h2, make_float2(B.x, B.y)), sub2(t.l2, make_float2(D.x, D.y)));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 ri;
    if (kGuard) {
        ri.x = r2.x > 0.f ? rsqrt_ftz(r2.x) : 0.f;
        ri.y = r2.y > 0.f ? rsqrt_ftz(r2.y) : 0.f;
    } else {
        ri.x = rsqrt_ftz(r2.x);
        ri.y = rsqrt_ftz(r2.y);
    }
    const float2 ri2 = __fmul2_rn(ri, ri);
    const float2 f0 = make_float2(B.z, B.w), f1 = make_float2(D.z, D.w), f2 = make_float2(E.x, E.y);
    const float2 df = __ffma2_rn(dx, f0, __ffma2_rn(dy, f1, __fmul2_rn(dz, f2)));
    const float2 dh = __ffma2_rn(dx, make_float2(E.z, E.w),
                                 __ffma2_rn(dy, make_float2(F.x, F.y), __fmul2_rn(dz, make_float2(F.z, F.w))));
    const float2 dn = __ffma2_rn(dx, make_float2(G.x, G.y),
                                 __ffma2_rn(dy, make_float2(G.z, G.w), __fmul2_rn(dz, make_float2(Q.x, Q.y))));
    // u += (1/r) (f + d s),  s = (d.f + (d.h)(d.nu) / r^2) / r^2
    const float2 st = __fmul2_rn(ri2, __ffma2_rn(__fmul2_rn(dh, dn), ri2, df));
    ax = __ffma2_rn(ri, __ffma2_rn(dx, st, f0), ax);
    ay = __ffma2_rn(ri, __ffma2_rn(dy, st, f1), ay);
    az = __ffma2_rn(ri, __ffma2_rn(dz, st, f2), az);
}

// forward near field: u = sum of the pair terms, stored
struct NearOpU {
    using Tgt = Tgt2;
    static constexpr bool kAdd = false;
    static constexpr bool kUnguarded = true;
    __device__ static Tgt load(const double* ts, const double*, int64_t M, int64_t m, bool valid, float)
    {
        return load_target(ts, M, m, valid);
    }
    template <bool kGuard>
    __device__ static void terms(const Tgt& t, const float4* tp, float2& ax, float2& ay, float2& az)
    {
        pair_terms<kGuard>(t, tp, ax, ay, az);
    }
};

// Regularized kernels (the blob of Cortez, Fauci and Medovikov), s = r^2 +
// eps^2, q = s^-1/2:
//   u_i += f_i q (1 + eps^2 q^2) + d_i q^3 ((d.f) + q^2 ((d.h)(d.nu) + (eps^2/2)(h.nu)))
//          + (eps^2/2) q^5 (h_i (d.nu) + nu_i (d.h)),
// h.nu from the last field of the source record; coincident pairs skipped as
// for the paper's kernels.
struct TgtReg {
    Tgt2 p;
    float2 e2, e2h;
};

template <bool kGuard>
__device__ __forceinline__ void pair_terms_reg(const TgtReg& T, const float4* tp, float2& ax, float2& ay, float2& az)
{
    const Tgt2& t = T.p;
    const float4 A = tp[0], B = tp[1], C = tp[2], D = tp[3], E = tp[4], F = tp[5], G = tp[6], Q = tp[7];
    const float2 dx = __fadd2_rn(sub2(t.h0, make_float2(A.x, A.y)), sub2(t.l0, make_float2(C.x, C.y)));
    const float2 dy = __fadd2_rn(sub2(t.h1, make_float2(A.z, A.w)), sub2(t.l1, make_float2(C.z, C.w)));
    const float2 dz = __fadd2_rn(sub2(t.h2, make_float2(B.x, B.y)), sub2(t.l2, make_float2(D.x, D.y)));
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    const float2 sr = __fadd2_rn(r2, T.e2);
    float2 q;
    if (kGuard) {
        q.x = r2.x > 0.f ? rsqrt_ftz(sr.x) : 0.f;
        q.y = r2.y > 0.f ? rsqrt_ftz(sr.y) : 0.f;
    } else {
        q.x = rsqrt_ftz(sr.x);
        q.y = rsqrt_ftz(sr.y);
    }
    const float2 q2 = __fmul2_rn(q, q);
    const float2 f0 = make_float2(B.z, B.w), f1 = make_float2(D.z, D.w), f2 = make_float2(E.x, E.y);
    const float2 h0 = make_float2(E.z, E.w), h1 = make_float2(F.x, F.y), h2 = make_float2(F.z, F.w);
    const float2 n0 = make_float2(G.x, G.y), n1 = make_float2(G.z, G.w), n2 = make_float2(Q.x, Q.y);
    const float2 df = __ffma2_rn(dx, f0, __ffma2_rn(dy, f1, __fmul2_rn(dz, f2)));
    const float2 dh = __ffma2_rn(dx, h0, __ffma2_rn(dy, h1, __fmul2_rn(dz, h2)));
    const float2 dn = __ffma2_rn(dx, n0, __ffma2_rn(dy, n1, __fmul2_rn(dz, n2)));
    const float2 one = make_float2(1.f, 1.f);
    const float2 a1 = __fmul2_rn(q, __ffma2_rn(T.e2, q2, one));
    const float2 t1 = __ffma2_rn(dh, dn, __fmul2_rn(T.e2h, make_float2(Q.z, Q.w)));
    const float2 qs = __fmul2_rn(__fmul2_rn(q, q2), __ffma2_rn(q2, t1, df));
    const float2 w = __fmul2_rn(__fmul2_rn(T.e2h, q), __fmul2_rn(q2, q2));
    const float2 wn = __fmul2_rn(w, dn), wh = __fmul2_rn(w, dh);
    ax = __ffma2_rn(f0, a1, __ffma2_rn(dx, qs, __ffma2_rn(h0, wn, __ffma2_rn(n0, wh, ax))));
    ay = __ffma2_rn(f1, a1, __ffma2_rn(dy, qs, __ffma2_rn(h1, wn, __ffma2_rn(n1, wh, ay))));
    az = __ffma2_rn(f2, a1, __ffma2_rn(dz, qs, __ffma2_rn(h2, wn, __ffma2_rn(n2, wh, az))));
}

struct NearOpReg {
    using Tgt = TgtReg;
    static constexpr bool kAdd = false;
    static constexpr bool kUnguarded = true;
    __device__ static Tgt load(const double* ts, const double*, int64_t M, int64_t m, bool valid, float e2)
    {
        TgtReg t;
        t.p = load_target(ts, M, m, valid);
        t.e2 = make_float2(e2, e2);
        t.e2h = make_float2(0.5f * e2, 0.5f * e2);
        return t;
    }
    template <bool kGuard>
    __device__ static void terms(const Tgt& t, const float4* tp, float2& ax, float2& ay, float2& az)
    {
        pair_terms_reg<kGuard>(t, tp, ax, ay, az);
    }
};

// ---------------------------------------------------------------------------
// FP64

// FP64 near field of batch b on one warp; tw is the warp's tile [12][32].
// kReg: the regularized kernels with e2 = eps^2 (formula at NearOpReg).
template <bool kReg = false>
__device__ inline void near_batch_fp64(const double* __restrict__ ts, int64_t M, const int4* __restrict__ topo,
                                       const double* __restrict__ xs, const double* __restrict__ ws, int64_t N,
                                       const int64_t* __restrict__ near_off, const ListEntry* __restrict__ near_list,
                                       double* __restrict__ u_near, int64_t b, double* tw, int lane, double e2 = 0.0)
{
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    double tx[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) tx[a] = ts[a * M + m];
    double ux = 0.0, uy = 0.0, uz = 0.0;
    const int64_t e0 = near_off[b], e1 = near_off[b + 1];
    for (int64_t e = e0; e < e1; e++) {
        const ListEntry le = near_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const int4 t = topo[le.node];
        for (int base = t.x; base < t.x + t.y; base += 32) {
            const int cnt = min(32, t.x + t.y - base);
            __syncwarp();
            if (lane < cnt) {
                const int64_t i = base + lane;
                for (int a = 0; a < 3; a++) tw[a * 32 + lane] = xs[a * N + i];
                for (int c = 0; c < 9; c++) tw[(3 + c) * 32 + lane] = ws[c * N + i];
            }
            __syncwarp();
            if (!in) continue;
            for (int j = 0; j < cnt && kReg; j++) {
                const double dx = tx[0] - tw[j], dy = tx[1] - tw[32 + j], dz = tx[2] - tw[64 + j];
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 > 0.0)) continue;
                const double f0 = tw[96 + j], f1 = tw[128 + j], f2 = tw[160 + j];
                const double h0 = tw[192 + j], h1 = tw[224 + j], h2 = tw[256 + j];
                const double n0 = tw[288 + j], n1 = tw[320 + j], n2 = tw[352 + j];
                const double df = dx * f0 + dy * f1 + dz * f2;
                const double dh = dx * h0 + dy * h1 + dz * h2;
                const double dn = dx * n0 + dy * n1 + dz * n2;
                const double q = rsqrt(r2 + e2), q2 = q * q;
                const double a1 = q * (1.0 + e2 * q2);
                const double qs = q * q2 * (df + q2 * (dh * dn + 0.5 * e2 * (h0 * n0 + h1 * n1 + h2 * n2)));
                const double w = 0.5 * e2 * q * q2 * q2;
                ux += f0 * a1 + dx * qs + w * (h0 * dn + n0 * dh);
                uy += f1 * a1 + dy * qs + w * (h1 * dn + n1 * dh);
                uz += f2 * a1 + dz * qs + w * (h2 * dn + n2 * dh);
            }
            for (int j = 0; j < cnt && !kReg; j++) {
                const double dx = tx[0] - tw[j], dy = tx[1] - tw[32 + j], dz = tx[2] - tw[64 + j];
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double ri = r2 > 0.0 ? rsqrt(r2) : 0.0;
                const double ri2 = ri * ri, ri3 = ri2 * ri;
                const double f0 = tw[96 + j], f1 = tw[128 + j], f2 = tw[160 + j];
                const double df = dx * f0 + dy * f1 + dz * f2;
                const double dh = dx * tw[192 + j] + dy * tw[224 + j] + dz * tw[256 + j];
                const double dn = dx * tw[288 + j] + dy * tw[320 + j] + dz * tw[352 + j];
                const double st = ri3 * (df + dh * dn * ri2);
                ux += f0 * ri + dx * st;
                uy += f1 * ri + dy * st;
                uz += f2 * ri + dz * st;
            }
        }
    }
    if (valid) {
        u_near[m] = ux;
        u_near[M + m] = uy;
        u_near[2 * M + m] = uz;
    }
}

template <bool kReg>
__global__ void __launch_bounds__(kNearWarps * 32)
    k_near_fp64(const double* __restrict__ ts, int64_t M, const int4* __restrict__ topo,
                const double* __restrict__ xs, const double* __restrict__ ws, int64_t N,
                const int64_t* __restrict__ near_off, const ListEntry* __restrict__ near_list,
                double* __restrict__ u_near, double e2)
{
    __shared__ double tile[kNearWarps][12 * 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b = blockIdx.x * (int64_t)kNearWarps + w;
    if (b >= nbatch) return;
    near_batch_fp64<kReg>(ts, M, topo, xs, ws, N, near_off, near_list, u_near, b, tile[w], lane, e2);
}

// system of a global item: the largest s with off[s] <= item (off: the
// systems' nsys + 1 first items; systems without items are passed over)
__device__ __forceinline__ int find_system(const int64_t* __restrict__ off, int nsys, int64_t item)
{
    int lo = 0, hi = nsys;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Persistent FP64 near-field kernel over many systems (see k_far32_batched):
// an item is a (system, batch).
__global__ void __launch_bounds__(kNearMaxWarps * 32)
    k_near_batched_fp64(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ item_off,
                        int64_t nitems, unsigned long long* __restrict__ counter)
{
    __shared__ __align__(16) double tile[kNearMaxWarps][12 * 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= nitems) break;
        const int s = find_system(item_off, nsys, (int64_t)item);
        const SysDesc& d = sys[s];
        near_batch_fp64(d.ts, d.M, d.topo, d.xs, d.ws, d.N, d.near_off, d.near_list, d.u_near,
                        (int64_t)item - item_off[s], tile[w], lane);
    }
}

// first unit of each system's schedule (one thread; nsys + 1 offsets)
__global__ void k_unit_offsets(const SysDesc* __restrict__ sys, int nsys, int64_t* __restrict__ uoff)
{
    int64_t run = 0;
    for (int s = 0; s < nsys; s++) {
        uoff[s] = run;
        run += *sys[s].nunits;
    }
    uoff[nsys] = run;
}

// Persistent leaf-major near field over the units of many systems' schedules
// (mixed precision; targets = sources in every system).
__global__ void __launch_bounds__(kNearMaxWarps * 32)
    k_near_leaf_batched(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ uoff,
                        unsigned long long* __restrict__ counter)
{
    __shared__ float4 tile[kNearMaxWarps][kTileFloat4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nitems = uoff[nsys];
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= nitems) break;
        const int s = find_system(uoff, nsys, (int64_t)item);
        const SysDesc& d = sys[s];
        nearpair::leaf_unit<NearOpU>(d.ts, nullptr, d.M, d.topo, d.spack, d.units, d.node_inc0, d.node_A, d.inc_m,
                                     d.inc_e, d.slots, 1, 0.0f, (int64_t)item - uoff[s], tile[w], lane);
    }
}

// the sums per target of every system: one warp per (system, batch)
__global__ void k_near_reduce_batched(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ boff,
                                      int64_t nbatches)
{
    const int64_t item = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (item >= nbatches) return;
    const int s = find_system(boff, nsys, item);
    const SysDesc& d = sys[s];
    nearpair::reduce_batch<false>(d.near_off, d.near_list, d.M, d.slots, d.u_near, item - boff[s], threadIdx.x & 31);
}

__global__ void k_finalize(const double* __restrict__ uf, const double* __restrict__ un,
                           const int32_t* __restrict__ perm, int64_t M, double* __restrict__ u)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    int64_t d = perm[i];
    for (int a = 0; a < 3; a++) u[a * M + d] = uf[a * M + i] + un[a * M + i];
}

// Batched finalize: system s writes columns [out_off, out_off + M_s) of the
// (3, ntot) output.  moff: nsys + 1 offsets of the systems' targets.
__global__ void k_finalize_batched(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ moff,
                                   int64_t mtotal, double* __restrict__ u, int64_t ntot)
{
    const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gi >= mtotal) return;
    int lo = 0, hi = nsys;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (moff[mid] <= gi)
            lo = mid;
        else
            hi = mid;
    }
    const SysDesc& d = sys[lo];
    const int64_t i = gi - moff[lo];
    const int64_t c = d.out_off + d.tperm[i];
    for (int a = 0; a < 3; a++) u[a * ntot + c] = d.u_far[a * d.M + i] + d.u_near[a * d.M + i];
}

__global__ void k_scatter_counts(const int64_t* __restrict__ cs, const int32_t* __restrict__ perm, int64_t M,
                                 int64_t* __restrict__ out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    out[perm[i]] = cs[i];
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

// ---------------------------------------------------------------------------
// leaf-major schedule (near_schedule)

// incidences per leaf (nA zeroed before)
__global__ void k_leaf_count(const ListEntry* __restrict__ list, int64_t E, int32_t* __restrict__ nA)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < E) {
        const ListEntry le = list[e];
        atomicAdd(nA + le.node, __popc(le.mask));
    }
}

// sort key of a node in no near list; the others' keys, below it, put the
// largest leaves first
constexpr uint64_t kLeafKeyNone = 0xffff;
constexpr int kLeafKeyBits = 16;

// per node its sort key; ord = identity
__global__ void k_leaf_keys(const int4* __restrict__ topo, int64_t nnodes, const int32_t* __restrict__ nA,
                            uint64_t* __restrict__ key, int32_t* __restrict__ ord)
{
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= nnodes) return;
    const uint64_t size = (uint64_t)topo[n].y;
    key[n] = nA[n] > 0 ? kLeafKeyNone - 1 - (size < kLeafKeyNone - 1 ? size : kLeafKeyNone - 1) : kLeafKeyNone;
    ord[n] = (int32_t)n;
}

// the node at sorted position j: its incidences and its units (pairs of
// 32-target streams)
__global__ void k_unit_count(const int32_t* __restrict__ ord, const int32_t* __restrict__ nA, int64_t nnodes,
                             int32_t* __restrict__ sA, int32_t* __restrict__ ucnt)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nnodes) return;
    const int32_t A = nA[ord[j]];
    sA[j] = A;
    ucnt[j] = (A + 63) / 64;
}

// per node its first incidence (incidences numbered in the sorted node
// order) and the cursor of the fill; the unit list
__global__ void k_unit_fill(const int32_t* __restrict__ ord, const int32_t* __restrict__ ucnt,
                            const int32_t* __restrict__ uoff, const int64_t* __restrict__ inc0s, int64_t nnodes,
                            int64_t* __restrict__ node_inc0, unsigned long long* __restrict__ cur,
                            int2* __restrict__ units)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= nnodes) return;
    const int node = ord[j], c = ucnt[j];
    node_inc0[node] = inc0s[j];
    cur[node] = (unsigned long long)inc0s[j];
    int2* u = units + uoff[j];
    for (int q = 0; q < c; q++) u[q] = make_int2(node, q);
}

// Incidences of every entry at its leaf's cursor: one warp per batch, its
// entries 32 at a time (lane j reserves entry j's places), then entry by
// entry the lanes of its mask write their target and the entry.  The order of
// the incidences inside a leaf depends on the order of the atomics, which
// changes nothing: a target's sums do not depend on its stream.
__global__ void k_inc_fill(const int64_t* __restrict__ near_off, const ListEntry* __restrict__ list, int64_t nbatch,
                           unsigned long long* __restrict__ cur, int32_t* __restrict__ inc_m,
                           int32_t* __restrict__ inc_e)
{
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (b >= nbatch) return;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t e0 = near_off[b], e1 = near_off[b + 1];
    for (int64_t base = e0; base < e1; base += 32) {
        const int64_t e = base + lane;
        ListEntry le{0, 0};
        unsigned long long pos = 0;
        if (e < e1) {
            le = list[e];
            pos = atomicAdd(cur + le.node, (unsigned long long)__popc(le.mask));
        }
        const int cnt = (int)min((int64_t)32, e1 - base);
        for (int j = 0; j < cnt; j++) {
            const unsigned mj = __shfl_sync(0xffffffffu, le.mask, j);
            const unsigned long long pj = __shfl_sync(0xffffffffu, pos, j);
            if ((mj >> lane) & 1u) {
                const unsigned long long q = pj + __popc(mj & lt);
                inc_m[q] = (int32_t)(b * kBatch + lane);
                inc_e[q] = (int32_t)(base + j);
            }
        }
    }
}

}  // namespace

// bound on the units of a schedule: sum over leaves of ceil(A / 64) <= 32 E / 64 + the leaves
static int64_t schedule_max_units(const tc_ctx* ctx) { return ctx->near_entries / 2 + ctx->nnodes + 1; }

cudaError_t near_schedule_alloc(tc_ctx* ctx, int full)
{
    const int64_t E = ctx->near_entries, nnodes = ctx->nnodes;
    cudaError_t e;
    // one histogram buffer for both sorts (entries, nodes)
    if ((e = ensure(ctx->nl_hist, (size_t)256 * radix_blocks(std::max(E, nnodes)) * 4)) != cudaSuccess) return e;
    if (!full) {
        if ((e = ensure(ctx->nl_keys, (size_t)E * 8)) != cudaSuccess) return e;
        if ((e = ensure(ctx->nl_keys_alt, (size_t)E * 8)) != cudaSuccess) return e;
        if ((e = ensure(ctx->nl_idx, (size_t)E * 4)) != cudaSuccess) return e;
        if ((e = ensure(ctx->nl_idx_alt, (size_t)E * 4)) != cudaSuccess) return e;
        return ensure(ctx->nl_eb, (size_t)E * 4);
    }
    if ((e = ensure(ctx->nl_nA, (size_t)nnodes * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_sA, (size_t)nnodes * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_inc0s, (size_t)(nnodes + 1) * 8)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_ninc0, (size_t)nnodes * 8)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_cur, (size_t)nnodes * 8)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_nkey, (size_t)nnodes * 8)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_nkey_alt, (size_t)nnodes * 8)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_nord, (size_t)nnodes * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_nord_alt, (size_t)nnodes * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_ucnt, (size_t)nnodes * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_uoff, (size_t)(nnodes + 1) * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_units, (size_t)schedule_max_units(ctx) * 8)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_inc_m, (size_t)E * 32 * 4)) != cudaSuccess) return e;
    if ((e = ensure(ctx->nl_inc_e, (size_t)E * 32 * 4)) != cudaSuccess) return e;
    return ensure(ctx->nl_slots, (size_t)E * 96 * 8);
}

cudaError_t near_schedule_build(tc_ctx* ctx, int full, cudaStream_t s)
{
    const int64_t E = ctx->near_entries, nnodes = ctx->nnodes;
    const int64_t nbatch = (ctx->M + kBatch - 1) / kBatch;
    const ListEntry* list = ptr<ListEntry>(ctx->near_list);
    cudaError_t e;
    if (!full)  // the entries sorted by leaf
        return sort_list_entries(list, E, ptr<int64_t>(ctx->near_off), nbatch, nnodes, ctx->nl_keys, ctx->nl_keys_alt,
                                 ctx->nl_idx, ctx->nl_idx_alt, ctx->nl_eb, ctx->nl_hist, s);
    int32_t* uoff = ptr<int32_t>(ctx->nl_uoff);
    if (E == 0) return cudaMemsetAsync(uoff + nnodes, 0, 4, s);
    int32_t* nA = ptr<int32_t>(ctx->nl_nA);
    int64_t* inc0s = ptr<int64_t>(ctx->nl_inc0s);
    if ((e = cudaMemsetAsync(nA, 0, (size_t)nnodes * 4, s)) != cudaSuccess) return e;
    k_leaf_count<<<grid_for(E, 256), 256, 0, s>>>(list, E, nA);
    note_launch();
    k_leaf_keys<<<grid_for(nnodes, 256), 256, 0, s>>>(ptr<int4>(ctx->node_topo), nnodes, nA,
                                                      ptr<uint64_t>(ctx->nl_nkey), ptr<int32_t>(ctx->nl_nord));
    note_launch();
    if ((e = radix_sort_bits(ptr<uint64_t>(ctx->nl_nkey), ptr<int32_t>(ctx->nl_nord), ptr<uint64_t>(ctx->nl_nkey_alt),
                             ptr<int32_t>(ctx->nl_nord_alt), ptr<uint32_t>(ctx->nl_hist), nnodes, kLeafKeyBits, s)) !=
        cudaSuccess)
        return e;
    k_unit_count<<<grid_for(nnodes, 256), 256, 0, s>>>(ptr<int32_t>(ctx->nl_nord), nA, nnodes,
                                                       ptr<int32_t>(ctx->nl_sA), ptr<int32_t>(ctx->nl_ucnt));
    note_launch();
    if ((e = launch_scan_i32_to_i64(ptr<int32_t>(ctx->nl_sA), inc0s, nnodes, inc0s + nnodes, s)) != cudaSuccess)
        return e;
    if ((e = launch_scan_i32(ptr<int32_t>(ctx->nl_ucnt), uoff, nnodes, uoff + nnodes, s)) != cudaSuccess) return e;
    k_unit_fill<<<grid_for(nnodes, 256), 256, 0, s>>>(ptr<int32_t>(ctx->nl_nord), ptr<int32_t>(ctx->nl_ucnt), uoff,
                                                      inc0s, nnodes, ptr<int64_t>(ctx->nl_ninc0),
                                                      ptr<unsigned long long>(ctx->nl_cur), ptr<int2>(ctx->nl_units));
    note_launch();
    k_inc_fill<<<grid_for(nbatch * 32, 256), 256, 0, s>>>(ptr<int64_t>(ctx->near_off), list, nbatch,
                                                          ptr<unsigned long long>(ctx->nl_cur),
                                                          ptr<int32_t>(ctx->nl_inc_m), ptr<int32_t>(ctx->nl_inc_e));
    note_launch();
    return cudaGetLastError();
}

NearSched near_schedule_desc(tc_ctx* ctx)
{
    NearSched sc;
    sc.node_inc0 = ptr<int64_t>(ctx->nl_ninc0);
    sc.node_A = ptr<int32_t>(ctx->nl_nA);
    sc.units = ptr<int2>(ctx->nl_units);
    sc.nunits = ptr<int32_t>(ctx->nl_uoff) + ctx->nnodes;
    sc.inc_m = ptr<int32_t>(ctx->nl_inc_m);
    sc.inc_e = ptr<int32_t>(ctx->nl_inc_e);
    sc.slots = ptr<double>(ctx->nl_slots);
    sc.E = ctx->near_entries;
    sc.max_units = schedule_max_units(ctx);
    sc.queue = nullptr;
    return sc;
}

cudaError_t near_schedule(tc_ctx* ctx, int full, NearSched& sc, cudaStream_t s)
{
    const int want = full ? 2 : 1;  // bit 1: entries sorted, bit 2: schedule built
    if (!(ctx->near_sched_ready & want)) {
        cudaError_t e = near_schedule_alloc(ctx, full);
        if (e == cudaSuccess) e = near_schedule_build(ctx, full, s);
        if (e != cudaSuccess) return e;
        ctx->near_sched_ready |= want;
    }
    sc = near_schedule_desc(ctx);
    return cudaSuccess;
}

cudaError_t launch_near(int precision, const double* ts, int64_t M, const int4* topo,
                        const double* xs, const double* ws, const float4* spack, int64_t N,
                        const int64_t* near_off, const ListEntry* near_list, double* u_near, int self,
                        const NearSched& sched, double eps, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const double e2 = eps * eps;
    if (precision == TC_FP64) {
        const unsigned grid = (unsigned)((nbatch + kNearWarps - 1) / kNearWarps);
        if (eps > 0.0)
            k_near_fp64<true><<<grid, kNearWarps * 32, 0, s>>>(ts, M, topo, xs, ws, N, near_off, near_list, u_near, e2);
        else
            k_near_fp64<false><<<grid, kNearWarps * 32, 0, s>>>(ts, M, topo, xs, ws, N, near_off, near_list, u_near,
                                                                0.0);
    } else if (eps > 0.0) {
        return nearpair::run_near_leaf<NearOpReg>(ts, nullptr, M, topo, spack, near_off, near_list, u_near, self,
                                                  (float)e2, sched, s);
    } else {
        return nearpair::run_near_leaf<NearOpU>(ts, nullptr, M, topo, spack, near_off, near_list, u_near, self,
                                                0.0f, sched, s);
    }
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_near_batched(int precision, const SysDesc* sys, int nsys, const int64_t* batch_off,
                                int64_t nbatches, int64_t* unit_off, unsigned long long* counter, int warps_per_block,
                                int blocks, cudaStream_t s)
{
    if (warps_per_block < 1 || warps_per_block > kNearMaxWarps) return cudaErrorInvalidValue;
    const void* fn = precision == TC_FP64 ? (const void*)k_near_batched_fp64 : (const void*)k_near_leaf_batched;
    cudaError_t e;
    if (blocks <= 0) {
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, warps_per_block * 32, 0);
        if (e != cudaSuccess) return e;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = (per_sm > 0 ? per_sm : 1) * sms;
    }
    if (precision == TC_FP64) {
        k_near_batched_fp64<<<blocks, warps_per_block * 32, 0, s>>>(sys, nsys, batch_off, nbatches, counter);
        note_launch();
        return cudaGetLastError();
    }
    k_unit_offsets<<<1, 1, 0, s>>>(sys, nsys, unit_off);
    note_launch();
    k_near_leaf_batched<<<blocks, warps_per_block * 32, 0, s>>>(sys, nsys, unit_off, counter);
    note_launch();
    k_near_reduce_batched<<<grid_for(nbatches * 32, 256), 256, 0, s>>>(sys, nsys, batch_off, nbatches);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize(const double* u_far, const double* u_near, const int32_t* perm, int64_t M, double* u,
                            cudaStream_t s)
{
    k_finalize<<<grid_for(M, 256), 256, 0, s>>>(u_far, u_near, perm, M, u);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_finalize_batched(const SysDesc* sys, int nsys, const int64_t* moff, int64_t mtotal, double* u,
                                    int64_t ntot, cudaStream_t s)
{
    k_finalize_batched<<<grid_for(mtotal, 256), 256, 0, s>>>(sys, nsys, moff, mtotal, u, ntot);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter_counts(const int64_t* cs, const int32_t* perm, int64_t M, int64_t* out, cudaStream_t s)
{
    k_scatter_counts<<<grid_for(M, 256), 256, 0, s>>>(cs, perm, M, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc
