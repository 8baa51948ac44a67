// Adjoint of the treecode velocity with the structure frozen.
//
// For L = sum_m g^m . u(x^m), with the tree (membership, centres y_c, radii),
// every target's MAC decisions and the order p of the last tc_eval held
// fixed, this computes dL/df, dL/dh, dL/dnu and dL/dx (source and target
// positions).  The paper does not differentiate its method; the derivation
// below is the chain rule applied to its formulas.
//
// Near field (Section 4.1 kernel K_i(d) = f_i/r + d_i (s + t), d = x_m - y_n):
//   g.K = (g.f)/r + (g.d)(s + t),  s = (d.f)/r^3,  t = (d.h)(d.nu)/r^5,
//   d(g.K)/df_j  = g_j/r + d_j (g.d)/r^3,
//   d(g.K)/dh_j  = d_j (g.d)(d.nu)/r^5,   d(g.K)/dnu_l = d_l (g.d)(d.h)/r^5,
//   d(g.K)/dd_a  = d_a c1 + g_a (s + t) + f_a c3 + h_a c4 + nu_a c5,
//   c1 = -((g.f)/r^3 + (g.d)(3 (d.f)/r^5 + 5 (d.h)(d.nu)/r^7)),
//   c3 = (g.d)/r^3,  c4 = (g.d)(d.nu)/r^5,  c5 = (g.d)(d.h)/r^5;
// the target gets +d(g.K)/dd, the source -d(g.K)/dd.
//
// Far field, target side: with u_i = sum_k b^k(d') (Â_i^k + d'_q B̂_iq^k),
// d' = (x - y_c)/rho, and d b^k/d d'_l = -(k_l + 1) b^{k+e_l} (b^k is a
// Taylor coefficient in y of a function of x - y):
//   sum_i g_i du_i/dx_l = (1/rho) sum_k [ b^k beta_l^k - (k_l + 1) b^{k+e_l} alpha^k ],
//   alpha^k = g.(Â^k + d'_q B̂_.q^k),  beta_l^k = sum_i g_i B̂_il^k,
// so the recurrence runs one level further, to p + 3.
//
// Far field, source side: the tables are linear in the moments, so
//   Ā_i^k = sum_m g_i^m b^k(d'_m),  B̄_iq^k = sum_m g_i^m d'_q b^k(d'_m)
// summed over the targets m that accept the cluster, give the adjoint moments
// Lambda_c^k = dL/dM_c^k by the transpose of the table map (k_lambda).  A
// particle y in clusters C then has dL/dw_c = sum_C sum_k Lambda_c^k(C) (y - y_C)^k;
// the ancestors' polynomials are re-expanded about the leaf centre by the
// binomial theorem (k_l2l) and evaluated once per particle (k_leaf_eval),
// with dL/dy = sum_c w_c grad_y of the same polynomial.  Weights:
// w = (f_0..2, h_j nu_l), so dL/dh_j = sum_l nu_l dL/dw_{3+3j+l} and
// dL/dnu_l = sum_j h_j dL/dw_{3+3j+l}.
//
// Work decomposition: the target-side kernels are batch-major like the
// forward ones; the source-side kernels are cluster-major or leaf-major over
// the forward lists sorted by cluster (stable radix sort, so entries keep
// their batch order).  The cluster-major far kernel accumulates per warp in
// shared memory and flushes with FP64 atomics when the cluster changes, so
// the source-side far gradient is reproducible only up to FP64 rounding.
#include <algorithm>

#include "tc_nearpair.cuh"
#include "tc_recurrence.cuh"

namespace tc {

namespace {

__constant__ LevelConst c_lev = make_level_const();
__constant__ LevelConst32 c_lev32 = make_level_const32();

inline int sm_count_adj()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

__device__ inline void unflatten(int idx, int& k1, int& k2, int& k3)
{
    int n = 0;
    while (ncoef(n) <= idx) n++;
    int pos = idx - (n > 0 ? ncoef(n - 1) : 0);
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= pos) a++;
    k3 = pos - a * (a + 1) / 2;
    k2 = a - k3;
    k1 = n - a;
}

__global__ void k_gather_g(const double* __restrict__ g, const int32_t* __restrict__ perm, int64_t M,
                           double* __restrict__ gs)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    int64_t j = perm[i];
    gs[i] = g[j];
    gs[M + i] = g[M + j];
    gs[2 * M + i] = g[2 * M + j];
}

// first index in sorted keys[0, n) that is >= v
__device__ inline int64_t lower_key(const uint64_t* keys, int64_t n, uint64_t v)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// ------------------------------------------------------- near, pair terms
// Writes the five scalar factors of d(g.K)/dd and of the weight gradients.
template <typename T>
struct NearTerms {
    T ri, st, c1, c3, c4, c5;
};

template <typename T>
__device__ inline NearTerms<T> near_terms(T dx, T dy, T dz, const T* f, const T* h, const T* nu, const T* g,
                                          T ri)
{
    NearTerms<T> o;
    const T ri2 = ri * ri, ri3 = ri2 * ri, ri5 = ri3 * ri2, ri7 = ri5 * ri2;
    const T df = dx * f[0] + dy * f[1] + dz * f[2];
    const T dh = dx * h[0] + dy * h[1] + dz * h[2];
    const T dn = dx * nu[0] + dy * nu[1] + dz * nu[2];
    const T gd = dx * g[0] + dy * g[1] + dz * g[2];
    const T gf = g[0] * f[0] + g[1] * f[1] + g[2] * f[2];
    o.ri = ri;
    o.st = df * ri3 + dh * dn * ri5;
    o.c1 = -(gf * ri3 + gd * (3 * df * ri5 + 5 * dh * dn * ri7));
    o.c3 = gd * ri3;
    o.c4 = gd * dn * ri5;
    o.c5 = gd * dh * ri5;
    return o;
}

constexpr int kNearAdjWarps = 4;

// Target side of the near field, batch-major (one warp per 32 targets).
template <typename T>
__global__ void __launch_bounds__(kNearAdjWarps * 32)
    k_near_adj_target(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                      const int4* __restrict__ topo, const double* __restrict__ xs, const double* __restrict__ ws,
                      int64_t N, const int64_t* __restrict__ near_off, const ListEntry* __restrict__ near_list,
                      double* __restrict__ gt)
{
    // source tile: x_hi(3) x_lo(3) f(3) h(3) nu(3) per source
    __shared__ T tile[kNearAdjWarps][15][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b = blockIdx.x * (int64_t)kNearAdjWarps + w;
    if (b >= nbatch) return;
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    T th[3] = {0, 0, 0}, tl[3] = {0, 0, 0}, g[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            const double v = ts[a * M + m];
            th[a] = (T)v;
            tl[a] = (T)(v - (double)th[a]);
            g[a] = (T)gs[a * M + m];
        }
    double acc[3] = {0, 0, 0};
    for (int64_t e = near_off[b]; e < near_off[b + 1]; e++) {
        const ListEntry le = near_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const int4 t = topo[le.node];
        for (int base = t.x; base < t.x + t.y; base += 32) {
            const int cnt = min(32, t.x + t.y - base);
            __syncwarp();
            if (lane < cnt) {
                const int64_t i = base + lane;
                for (int a = 0; a < 3; a++) {
                    const double v = xs[a * N + i];
                    const T hi = (T)v;
                    tile[w][a][lane] = hi;
                    tile[w][3 + a][lane] = (T)(v - (double)hi);
                }
                for (int c = 0; c < 9; c++) tile[w][6 + c][lane] = (T)ws[c * N + i];
            }
            __syncwarp();
            if (!in) continue;
            T a0 = 0, a1 = 0, a2 = 0;
            for (int j = 0; j < cnt; j++) {
                const T dx = (th[0] - tile[w][0][j]) + (tl[0] - tile[w][3][j]);
                const T dy = (th[1] - tile[w][1][j]) + (tl[1] - tile[w][4][j]);
                const T dz = (th[2] - tile[w][2][j]) + (tl[2] - tile[w][5][j]);
                const T r2 = dx * dx + dy * dy + dz * dz;
                const T ri = r2 > (T)0 ? (T)1 / sqrt(r2) : (T)0;
                const T f[3] = {tile[w][6][j], tile[w][7][j], tile[w][8][j]};
                const T h[3] = {tile[w][9][j], tile[w][10][j], tile[w][11][j]};
                const T nu[3] = {tile[w][12][j], tile[w][13][j], tile[w][14][j]};
                const NearTerms<T> q = near_terms<T>(dx, dy, dz, f, h, nu, g, ri);
                a0 += dx * q.c1 + g[0] * q.st + f[0] * q.c3 + h[0] * q.c4 + nu[0] * q.c5;
                a1 += dy * q.c1 + g[1] * q.st + f[1] * q.c3 + h[1] * q.c4 + nu[1] * q.c5;
                a2 += dz * q.c1 + g[2] * q.st + f[2] * q.c3 + h[2] * q.c4 + nu[2] * q.c5;
            }
            acc[0] += (double)a0;
            acc[1] += (double)a1;
            acc[2] += (double)a2;
        }
    }
    if (valid)
        for (int a = 0; a < 3; a++) gt[a * M + m] += acc[a];
}

// Source side of the near field, leaf-major: a block per leaf, a warp per 32
// of its sources, looping over the near entries (batch, lane mask) that name
// the leaf; targets of an entry are staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(kNearAdjWarps * 32)
    k_near_adj_source(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                      const int4* __restrict__ topo, const double* __restrict__ xs, const double* __restrict__ ws,
                      int64_t N, const uint64_t* __restrict__ skeys, const int32_t* __restrict__ sidx,
                      const ListEntry* __restrict__ near_list, const int32_t* __restrict__ ebatch, int64_t nent,
                      double* __restrict__ gnear)
{
    __shared__ T tile[kNearAdjWarps][9][32];  // target x_hi(3) x_lo(3) g(3)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t node = blockIdx.x;
    const int4 t = topo[node];
    if (t.w != 0) return;
    const int64_t j0 = lower_key(skeys, nent, (uint64_t)node), j1 = lower_key(skeys, nent, (uint64_t)node + 1);
    for (int tile0 = w * 32; tile0 < t.y; tile0 += kNearAdjWarps * 32) {
        const int64_t si = t.x + tile0 + lane;
        const bool valid = tile0 + lane < t.y;
        T sh[3] = {0, 0, 0}, sl[3] = {0, 0, 0}, f[3] = {0, 0, 0}, h[3] = {0, 0, 0}, nu[3] = {0, 0, 0};
        if (valid)
            for (int a = 0; a < 3; a++) {
                const double v = xs[a * N + si];
                sh[a] = (T)v;
                sl[a] = (T)(v - (double)sh[a]);
                f[a] = (T)ws[a * N + si];
                h[a] = (T)ws[(3 + a) * N + si];
                nu[a] = (T)ws[(6 + a) * N + si];
            }
        double acc[12];
        for (int c = 0; c < 12; c++) acc[c] = 0.0;
        for (int64_t j = j0; j < j1; j++) {
            const int32_t e = sidx[j];
            const unsigned mask = near_list[e].mask;
            const int64_t m = (int64_t)ebatch[e] * kBatch + lane;
            __syncwarp();
            if ((mask >> lane) & 1u)
                for (int a = 0; a < 3; a++) {
                    const double v = ts[a * M + m];
                    const T hi = (T)v;
                    tile[w][a][lane] = hi;
                    tile[w][3 + a][lane] = (T)(v - (double)hi);
                    tile[w][6 + a][lane] = (T)gs[a * M + m];
                }
            __syncwarp();
            T a[12];
            for (int c = 0; c < 12; c++) a[c] = 0;
            unsigned mm = mask;
            while (mm) {
                const int q = __ffs(mm) - 1;
                mm &= mm - 1;
                const T dx = (tile[w][0][q] - sh[0]) + (tile[w][3][q] - sl[0]);
                const T dy = (tile[w][1][q] - sh[1]) + (tile[w][4][q] - sl[1]);
                const T dz = (tile[w][2][q] - sh[2]) + (tile[w][5][q] - sl[2]);
                const T g[3] = {tile[w][6][q], tile[w][7][q], tile[w][8][q]};
                const T r2 = dx * dx + dy * dy + dz * dz;
                const T ri = r2 > (T)0 ? (T)1 / sqrt(r2) : (T)0;
                const NearTerms<T> z = near_terms<T>(dx, dy, dz, f, h, nu, g, ri);
                const T d[3] = {dx, dy, dz};
                for (int c = 0; c < 3; c++) {
                    a[c] += g[c] * z.ri + d[c] * z.c3;
                    a[3 + c] += d[c] * z.c4;
                    a[6 + c] += d[c] * z.c5;
                    a[9 + c] -= d[c] * z.c1 + g[c] * z.st + f[c] * z.c3 + h[c] * z.c4 + nu[c] * z.c5;
                }
            }
            for (int c = 0; c < 12; c++) acc[c] += (double)a[c];
        }
        if (valid)
            for (int c = 0; c < 12; c++) gnear[c * N + si] = acc[c];
    }
}

// ------------------------------------------ near, mixed precision (FP32)
// The same pair terms in FP32 on hi/lo positions (as the forward near field),
// 1/r from rsqrt_ftz, packed FP32x2 arithmetic.

// target side: the forward near field's group walk (tc_nearpair.cuh: four
// batches per warp, the targets of each leaf packed into 32-lane streams, two
// sources per packed FP32x2 instruction) with the gradient's pair terms;
// the result is added to the far part already in gt.
struct NearOpG {
    struct Tgt {
        float2 h0, h1, h2, l0, l1, l2, g0, g1, g2;
    };
    static constexpr bool kAdd = true;
    // the guard-free variant measured slower here (more registers)
    static constexpr bool kUnguarded = false;
    __device__ static Tgt load(const double* ts, const double* gs, int64_t M, int64_t m, bool valid, float)
    {
        float h[3] = {0, 0, 0}, l[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        if (valid)
            for (int a = 0; a < 3; a++) {
                const double v = ts[a * M + m];
                h[a] = __double2float_rn(v);
                l[a] = __double2float_rn(v - (double)h[a]);
                g[a] = __double2float_rn(gs[a * M + m]);
            }
        Tgt t;
        t.h0 = make_float2(h[0], h[0]), t.h1 = make_float2(h[1], h[1]), t.h2 = make_float2(h[2], h[2]);
        t.l0 = make_float2(l[0], l[0]), t.l1 = make_float2(l[1], l[1]), t.l2 = make_float2(l[2], l[2]);
        t.g0 = make_float2(g[0], g[0]), t.g1 = make_float2(g[1], g[1]), t.g2 = make_float2(g[2], g[2]);
        return t;
    }
    // d(g.K)/dd_a = d_a c1 + g_a st + f_a c3 + h_a c4 + nu_a c5 for two sources
    template <bool kGuard>
    __device__ static void terms(const Tgt& t, const float4* tp, float2& ax, float2& ay, float2& az)
    {
        using nearpair::sub2;
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
        const float2 ri2 = __fmul2_rn(ri, ri), ri3 = __fmul2_rn(ri2, ri), ri5 = __fmul2_rn(ri3, ri2);
        const float2 f0 = make_float2(B.z, B.w), f1 = make_float2(D.z, D.w), f2 = make_float2(E.x, E.y);
        const float2 h0 = make_float2(E.z, E.w), h1 = make_float2(F.x, F.y), h2 = make_float2(F.z, F.w);
        const float2 n0 = make_float2(G.x, G.y), n1 = make_float2(G.z, G.w), n2 = make_float2(Q.x, Q.y);
        const float2 df = __ffma2_rn(dx, f0, __ffma2_rn(dy, f1, __fmul2_rn(dz, f2)));
        const float2 dh = __ffma2_rn(dx, h0, __ffma2_rn(dy, h1, __fmul2_rn(dz, h2)));
        const float2 dn = __ffma2_rn(dx, n0, __ffma2_rn(dy, n1, __fmul2_rn(dz, n2)));
        const float2 gd = __ffma2_rn(dx, t.g0, __ffma2_rn(dy, t.g1, __fmul2_rn(dz, t.g2)));
        const float2 gf = __ffma2_rn(t.g0, f0, __ffma2_rn(t.g1, f1, __fmul2_rn(t.g2, f2)));
        const float2 t5 = __fmul2_rn(__fmul2_rn(dh, dn), ri5);
        const float2 st = __ffma2_rn(df, ri3, t5);
        const float2 c3 = __fmul2_rn(gd, ri3);
        const float2 inner = __ffma2_rn(__fmul2_rn(make_float2(3.f, 3.f), df), ri3, __fmul2_rn(make_float2(5.f, 5.f), t5));
        const float2 c1n = __ffma2_rn(gf, ri3, __fmul2_rn(__fmul2_rn(gd, ri2), inner));  // -c1
        const float2 c4 = __fmul2_rn(__fmul2_rn(c3, dn), ri2);
        const float2 c5 = __fmul2_rn(__fmul2_rn(c3, dh), ri2);
        ax = __ffma2_rn(t.g0, st, __ffma2_rn(f0, c3, __ffma2_rn(h0, c4, __ffma2_rn(n0, c5, nearpair::sub2(ax, __fmul2_rn(dx, c1n))))));
        ay = __ffma2_rn(t.g1, st, __ffma2_rn(f1, c3, __ffma2_rn(h1, c4, __ffma2_rn(n1, c5, nearpair::sub2(ay, __fmul2_rn(dy, c1n))))));
        az = __ffma2_rn(t.g2, st, __ffma2_rn(f2, c3, __ffma2_rn(h2, c4, __ffma2_rn(n2, c5, nearpair::sub2(az, __fmul2_rn(dz, c1n))))));
    }
};


// Source side, on the leaf-major schedule of the forward near field: a unit
// is (leaf, tile of 32 of its sources, segment of kAdjSeg of its incidences);
// a warp holds one source per lane and runs over the segment's targets in
// chunks of 32, staged in shared memory (positions as FP32 hi/lo, g), two
// targets per packed instruction; a chunk's terms are summed by compensated
// FP32 summation and a unit's sums added to the FP64 source gradients with
// atomics (gnear is zeroed first).  The units of a leaf are numbered from
// its first unit soff[leaf] (k_adj_src_count + scan), tile-minor.
constexpr int kAdjSeg = 1024;
constexpr int kAdjSrcWarps = 4;

// units of each node: tiles of 32 sources x segments of its incidences
__global__ void k_adj_src_count(const int4* __restrict__ topo, const int32_t* __restrict__ node_A, int64_t nnodes,
                                int32_t* __restrict__ cnt)
{
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= nnodes) return;
    const int A = node_A[n];
    cnt[n] = A > 0 ? ((topo[n].y + 31) / 32) * ((A + kAdjSeg - 1) / kAdjSeg) : 0;
}

// The source-side terms of the lane's source (sh/sl: position hi/lo; f, h,
// nu) against staged targets q, q+1 (T: their 9 fields as pairs), added to
// a[12]: dL/df (3), dL/dh (3), dL/dnu (3), dL/dy (3).
__device__ __forceinline__ void adj_src_pair(const float2 (&T)[9], const float2 (&sh)[3], const float2 (&sl)[3],
                                             const float2 (&f)[3], const float2 (&h)[3], const float2 (&n)[3],
                                             float2 (&a)[12])
{
    using nearpair::sub2;
    const float2 dx = __fadd2_rn(sub2(T[0], sh[0]), sub2(T[3], sl[0]));
    const float2 dy = __fadd2_rn(sub2(T[1], sh[1]), sub2(T[4], sl[1]));
    const float2 dz = __fadd2_rn(sub2(T[2], sh[2]), sub2(T[5], sl[2]));
    const float2 g0 = T[6], g1 = T[7], g2 = T[8];
    const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
    float2 ri;
    ri.x = r2.x > 0.f ? rsqrt_ftz(r2.x) : 0.f;
    ri.y = r2.y > 0.f ? rsqrt_ftz(r2.y) : 0.f;
    const float2 ri2 = __fmul2_rn(ri, ri), ri3 = __fmul2_rn(ri2, ri), ri5 = __fmul2_rn(ri3, ri2);
    const float2 df = __ffma2_rn(dx, f[0], __ffma2_rn(dy, f[1], __fmul2_rn(dz, f[2])));
    const float2 dh = __ffma2_rn(dx, h[0], __ffma2_rn(dy, h[1], __fmul2_rn(dz, h[2])));
    const float2 dn = __ffma2_rn(dx, n[0], __ffma2_rn(dy, n[1], __fmul2_rn(dz, n[2])));
    const float2 gd = __ffma2_rn(dx, g0, __ffma2_rn(dy, g1, __fmul2_rn(dz, g2)));
    const float2 gf = __ffma2_rn(g0, f[0], __ffma2_rn(g1, f[1], __fmul2_rn(g2, f[2])));
    const float2 t5 = __fmul2_rn(__fmul2_rn(dh, dn), ri5);
    const float2 st = __ffma2_rn(df, ri3, t5);
    const float2 c3 = __fmul2_rn(gd, ri3);
    const float2 inner =
        __ffma2_rn(__fmul2_rn(make_float2(3.f, 3.f), df), ri3, __fmul2_rn(make_float2(5.f, 5.f), t5));
    const float2 c1n = __ffma2_rn(gf, ri3, __fmul2_rn(__fmul2_rn(gd, ri2), inner));  // -c1
    const float2 c4 = __fmul2_rn(__fmul2_rn(c3, dn), ri2);
    const float2 c5 = __fmul2_rn(__fmul2_rn(c3, dh), ri2);
    a[0] = __ffma2_rn(g0, ri, __ffma2_rn(dx, c3, a[0]));
    a[1] = __ffma2_rn(g1, ri, __ffma2_rn(dy, c3, a[1]));
    a[2] = __ffma2_rn(g2, ri, __ffma2_rn(dz, c3, a[2]));
    a[3] = __ffma2_rn(dx, c4, a[3]);
    a[4] = __ffma2_rn(dy, c4, a[4]);
    a[5] = __ffma2_rn(dz, c4, a[5]);
    a[6] = __ffma2_rn(dx, c5, a[6]);
    a[7] = __ffma2_rn(dy, c5, a[7]);
    a[8] = __ffma2_rn(dz, c5, a[8]);
    // dL/dy = -d(g.K)/dd = -(d c1 + g st + f c3 + h c4 + nu c5)
    a[9] = __ffma2_rn(dx, c1n, sub2(a[9], __ffma2_rn(g0, st, __ffma2_rn(f[0], c3,
                                       __ffma2_rn(h[0], c4, __fmul2_rn(n[0], c5))))));
    a[10] = __ffma2_rn(dy, c1n, sub2(a[10], __ffma2_rn(g1, st, __ffma2_rn(f[1], c3,
                                        __ffma2_rn(h[1], c4, __fmul2_rn(n[1], c5))))));
    a[11] = __ffma2_rn(dz, c1n, sub2(a[11], __ffma2_rn(g2, st, __ffma2_rn(f[2], c3,
                                        __ffma2_rn(h[2], c4, __fmul2_rn(n[2], c5))))));
}

__global__ void __launch_bounds__(kAdjSrcWarps * 32)
    k_near_adj_source_units(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                            const int4* __restrict__ topo, const float4* __restrict__ spack, int64_t N,
                            int64_t nnodes, const int64_t* __restrict__ soff, const int64_t* __restrict__ node_inc0,
                            const int32_t* __restrict__ node_A, const int32_t* __restrict__ inc_m,
                            double* __restrict__ gnear, unsigned long long* __restrict__ queue)
{
    // staged targets, field-major: x_hi (3), x_lo (3), g (3); targets q, q+1
    // are read together as one float2 per field
    __shared__ __align__(8) float tile[kAdjSrcWarps][9][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nunits = soff[nnodes];
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(queue, 1ull);
        u = __shfl_sync(0xffffffffu, u, 0);
        if ((int64_t)u >= nunits) break;
        int64_t lo = 0, hi = nnodes;  // soff[lo] <= u < soff[hi]; nodes without units share offsets
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (soff[mid] <= (int64_t)u)
                lo = mid;
            else
                hi = mid;
        }
        const int4 t = topo[lo];
        const int S = (t.y + 31) / 32;
        const int64_t r = (int64_t)u - soff[lo];
        const int tile_s = (int)(r % S), seg = (int)(r / S);
        const int64_t I0 = node_inc0[lo];
        const int k0 = seg * kAdjSeg, k1 = min(node_A[lo], k0 + kAdjSeg);
        const int64_t si = t.x + 32 * tile_s + lane;
        const bool valid = 32 * tile_s + lane < t.y;
        float4 A = make_float4(0, 0, 0, 0), B = A, C = A, D = A;
        if (valid) {
            const float4* src = spack + 4 * si;
            A = src[0], B = src[1], C = src[2], D = src[3];
        }
        // this lane's source, replicated into both halves of each pair
        const float2 sh[3] = {make_float2(A.x, A.x), make_float2(A.y, A.y), make_float2(A.z, A.z)};
        const float2 sl[3] = {make_float2(B.x, B.x), make_float2(B.y, B.y), make_float2(B.z, B.z)};
        const float2 f[3] = {make_float2(A.w, A.w), make_float2(B.w, B.w), make_float2(C.x, C.x)};
        const float2 h[3] = {make_float2(C.y, C.y), make_float2(C.z, C.z), make_float2(C.w, C.w)};
        const float2 n[3] = {make_float2(D.x, D.x), make_float2(D.y, D.y), make_float2(D.z, D.z)};
        float acc[12], cmp[12];
#pragma unroll
        for (int c = 0; c < 12; c++) acc[c] = cmp[c] = 0.f;
        for (int kc = k0; kc < k1; kc += 32) {
            const int cnt = min(32, k1 - kc);
            __syncwarp();
            {
                float v[9];
#pragma unroll
                for (int k = 0; k < 9; k++) v[k] = 0.f;  // past cnt: a zero-weight target, zero terms
                if (lane < cnt) {
                    const int64_t m = inc_m[I0 + kc + lane];
                    for (int a = 0; a < 3; a++) {
                        const double x = ts[a * M + m];
                        v[a] = __double2float_rn(x);
                        v[3 + a] = __double2float_rn(x - (double)v[a]);
                        v[6 + a] = __double2float_rn(gs[a * M + m]);
                    }
                }
#pragma unroll
                for (int k = 0; k < 9; k++) tile[w][k][lane] = v[k];
            }
            __syncwarp();
            float2 a[12];
#pragma unroll
            for (int c = 0; c < 12; c++) a[c] = make_float2(0.f, 0.f);
            for (int q = 0; q < cnt; q += 2) {
                float2 T[9];
#pragma unroll
                for (int k = 0; k < 9; k++) T[k] = *reinterpret_cast<const float2*>(&tile[w][k][q]);
                adj_src_pair(T, sh, sl, f, h, n, a);
            }
#pragma unroll
            for (int c = 0; c < 12; c++) kahan_add(acc[c], cmp[c], a[c].x + a[c].y);
        }
        if (valid)
            for (int c = 0; c < 12; c++) atomicAdd(&gnear[c * N + si], (double)acc[c] - (double)cmp[c]);
    }
}

// --------------------------------------------------- far, target side
// Batch-major like k_far; the recurrence runs to P + 1 = p + 3 and the
// level-(n-1) values alpha^k are kept in a second two-slot store.
template <typename TR, typename TC>
__global__ void __launch_bounds__(32)
    k_far_adj_target(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                     const Geo* __restrict__ geo, const double* __restrict__ invrho, const TC* __restrict__ ab, int p,
                     const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list,
                     double* __restrict__ gt)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b = blockIdx.x;
    if (b >= nbatch) return;
    const int P = p + 2, Q = P + 1;
    const int C2 = ncoef(P);
    TR* cs_q = reinterpret_cast<TR*>(smraw);  // parity of Q: levels Q, Q-2, ...
    TR* cs_o = cs_q + (size_t)level_size(Q) * 32;
    TC* as_p = reinterpret_cast<TC*>(cs_o + (size_t)level_size(P) * 32);  // parity of P
    TC* as_o = as_p + (size_t)level_size(P) * 32;
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    double x[3] = {0, 0, 0};
    TC g[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            x[a] = ts[a * M + m];
            g[a] = (TC)gs[a * M + m];
        }
    double G[3] = {0, 0, 0};
    for (int64_t e = far_off[b]; e < far_off[b + 1]; e++) {
        const ListEntry le = far_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const Geo gc = geo[le.node];
        const double ir = invrho[le.node];
        const double d0 = (x[0] - gc.x) * ir, d1 = (x[1] - gc.y) * ir, d2 = (x[2] - gc.z) * ir;
        double R2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (!in) R2 = 1.0;
        const double iR = rsqrt(R2);
        const TR w0 = (TR)(d0 * iR), w1 = (TR)(d1 * iR), w2 = (TR)(d2 * iR);
        const TC dd[3] = {(TC)d0, (TC)d1, (TC)d2};
        const TC* __restrict__ tab = ab + (int64_t)le.node * C2 * 12;
        TC scale = (TC)iR;
        TC Gl[3];
        {  // level 0: c^0 = 1
            const TC* t = tab;
            TC v[3], beta[3];
            for (int i = 0; i < 3; i++) v[i] = t[i] + dd[0] * t[3 + 3 * i] + dd[1] * t[4 + 3 * i] + dd[2] * t[5 + 3 * i];
            for (int l = 0; l < 3; l++) beta[l] = g[0] * t[3 + l] + g[1] * t[6 + l] + g[2] * t[9 + l];
            (((0 ^ P) & 1) ? as_o : as_p)[lane] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
            (((0 ^ Q) & 1) ? cs_o : cs_q)[lane] = (TR)1;
            for (int l = 0; l < 3; l++) Gl[l] = scale * beta[l];
        }
        for (int n = 1; n <= Q; n++) {
            const TR kap = (TR)c_lev.kappa[n];
            scale *= (TC)(c_lev.ratio[n] * iR);
            TR* Rn = ((n ^ Q) & 1) ? cs_o : cs_q;
            const TR* R1 = ((n ^ Q) & 1) ? cs_q : cs_o;
            TC* An = ((n ^ P) & 1) ? as_o : as_p;
            const TC* A1 = ((n ^ P) & 1) ? as_p : as_o;
            const TC* tl = tab + (int64_t)ncoef(n - 1) * 12;
            TC acc1[3] = {0, 0, 0}, acc2[3] = {0, 0, 0};
            for (int a = n; a >= 0; a--) {
                const int k1 = n - a;
                const int base = a * (a + 1) / 2;
                for (int k3 = a; k3 >= 0; k3--) {
                    const int k2 = a - k3;
                    const int pos = base + k3;
                    const TR ck = coef<TR>(R1, Rn, pos, a, k1, k2, k3, w0, w1, w2, kap, lane);
                    Rn[pos * 32 + lane] = ck;
                    const TC cc = to_tc<TR, TC>(ck);
                    if (k1 >= 1) acc2[0] += cc * (TC)k1 * A1[pos * 32 + lane];
                    if (k2 >= 1) acc2[1] += cc * (TC)k2 * A1[(pos - a) * 32 + lane];
                    if (k3 >= 1) acc2[2] += cc * (TC)k3 * A1[(pos - a - 1) * 32 + lane];
                    if (n <= P) {
                        const TC* t = tl + pos * 12;
                        TC v[3];
                        for (int i = 0; i < 3; i++)
                            v[i] = t[i] + dd[0] * t[3 + 3 * i] + dd[1] * t[4 + 3 * i] + dd[2] * t[5 + 3 * i];
                        An[pos * 32 + lane] = g[0] * v[0] + g[1] * v[1] + g[2] * v[2];
                        for (int l = 0; l < 3; l++) acc1[l] += cc * (g[0] * t[3 + l] + g[1] * t[6 + l] + g[2] * t[9 + l]);
                    }
                }
            }
            for (int l = 0; l < 3; l++) Gl[l] += scale * (acc1[l] - acc2[l]);
        }
        if (in)
            for (int l = 0; l < 3; l++) G[l] += ir * (double)Gl[l];
    }
    if (valid)
        for (int l = 0; l < 3; l++) gt[l * M + m] = G[l];
}

// --------------------------------------------------- far, source side
// Cluster-major over the far entries sorted by cluster; a warp takes `chunk`
// consecutive sorted entries.  Per entry the lanes are the batch's targets
// (g = 0 on lanes outside the mask, so they add nothing).  After each level
// the scaled coefficients s_n c^k of all lanes sit in a padded buffer and
// each lane sums, for its own positions, over the 32 targets into the
// warp's accumulators [coefficient][12]; the accumulators are flushed to the
// cluster's FP64 adjoint tables with atomics when the cluster changes.
template <typename TR, typename TC>
__global__ void __launch_bounds__(32)
    k_far_adj_source(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                     const Geo* __restrict__ geo, const double* __restrict__ invrho, int p,
                     const uint64_t* __restrict__ skeys, const int32_t* __restrict__ sidx,
                     const ListEntry* __restrict__ far_list, const int32_t* __restrict__ ebatch, int64_t nent,
                     int chunk, double* __restrict__ abar)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)blockIdx.x * chunk;
    if (j0 >= nent) return;
    const int64_t j1 = min(nent, j0 + chunk);
    const int P = p + 2;
    const int C2 = ncoef(P);
    const int LSP = level_size(P);
    TR* cs_p = reinterpret_cast<TR*>(smraw);  // parity of P
    TR* cs_o = cs_p + (size_t)LSP * 32;
    TC* sc = reinterpret_cast<TC*>(cs_o + (size_t)level_size(P - 1) * 32);  // [LSP][33]
    TC* gb = sc + (size_t)LSP * 33;                                           // [32][12]
    TC* acc = gb + 32 * 12;                                                   // [C2][12]
    int64_t cur = -1;
    for (int q = lane; q < C2 * 12; q += 32) acc[q] = (TC)0;
    for (int64_t j = j0; j < j1; j++) {
        const int64_t node = (int64_t)skeys[j];
        if (node != cur) {
            __syncwarp();
            if (cur >= 0)
                for (int q = lane; q < C2 * 12; q += 32) {
                    atomicAdd(&abar[cur * C2 * 12 + q], (double)acc[q]);
                    acc[q] = (TC)0;
                }
            cur = node;
            __syncwarp();
        }
        const int32_t e = sidx[j];
        const unsigned mask = far_list[e].mask;
        const int64_t m = (int64_t)ebatch[e] * kBatch + lane;
        const bool in = (mask >> lane) & 1u;
        double x[3] = {0, 0, 0};
        TC g[3] = {0, 0, 0};
        if (in)
            for (int a = 0; a < 3; a++) {
                x[a] = ts[a * M + m];
                g[a] = (TC)gs[a * M + m];
            }
        const Geo gc = geo[node];
        const double ir = invrho[node];
        const double d0 = (x[0] - gc.x) * ir, d1 = (x[1] - gc.y) * ir, d2 = (x[2] - gc.z) * ir;
        double R2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (!in) R2 = 1.0;
        const double iR = rsqrt(R2);
        const TR w0 = (TR)(d0 * iR), w1 = (TR)(d1 * iR), w2 = (TR)(d2 * iR);
        const TC dd[3] = {(TC)d0, (TC)d1, (TC)d2};
        TC scale = (TC)iR;
        for (int i = 0; i < 3; i++) {
            gb[lane * 12 + i] = g[i];
            for (int l = 0; l < 3; l++) gb[lane * 12 + 3 + 3 * i + l] = g[i] * dd[l];
        }
        (((0 ^ P) & 1) ? cs_o : cs_p)[lane] = (TR)1;
        sc[lane] = scale;  // position 0, column lane
        for (int n = 0; n <= P; n++) {
            if (n > 0) {
                const TR kap = (TR)c_lev.kappa[n];
                scale *= (TC)(c_lev.ratio[n] * iR);
                TR* Rn = ((n ^ P) & 1) ? cs_o : cs_p;
                const TR* R1 = ((n ^ P) & 1) ? cs_p : cs_o;
                for (int a = n; a >= 0; a--) {
                    const int k1 = n - a;
                    const int base = a * (a + 1) / 2;
                    for (int k3 = a; k3 >= 0; k3--) {
                        const int pos = base + k3;
                        const TR ck = coef<TR>(R1, Rn, pos, a, k1, a - k3, k3, w0, w1, w2, kap, lane);
                        Rn[pos * 32 + lane] = ck;
                        sc[pos * 33 + lane] = scale * to_tc<TR, TC>(ck);
                    }
                }
            }
            __syncwarp();
            const int ls = level_size(n);
            TC* accl = acc + (size_t)(n > 0 ? ncoef(n - 1) : 0) * 12;
            for (int pos = lane; pos < ls; pos += 32) {
                TC r[12];
                for (int c = 0; c < 12; c++) r[c] = (TC)0;
                for (int t = 0; t < 32; t++) {
                    const TC v = sc[pos * 33 + t];
                    for (int c = 0; c < 12; c++) r[c] += v * gb[t * 12 + c];
                }
                for (int c = 0; c < 12; c++) accl[pos * 12 + c] += r[c];
            }
            __syncwarp();
        }
    }
    __syncwarp();
    if (cur >= 0)
        for (int q = lane; q < C2 * 12; q += 32) atomicAdd(&abar[cur * C2 * 12 + q], (double)acc[q]);
}

// ------------------------------------- far, mixed precision, folded tables
// The forward far field in mixed precision is u_i = (1/R') sum_h c^h(v)
// (T_i^h + d'_q T_{3+3i+q}^h) over the harmonic subset h (k1 <= 1) with the
// folded, lambda-scaled FP32 tables T (tc_far.cu).  The folded sum equals the
// unfolded one for every d', so it is differentiated as it stands.

// Target side.  With b^k = lambda_n c^k / R' and d b^k/d d'_m =
// -(k_m + 1) b^{k+e_m}:
//   d(g.u)/dd'_m = (1/R') sum_h [ c^h gB_m^h - (k_m + 1) r_n c^{k+e_m} alpha^h ],
//   alpha^h = g_i (T_i^h + d'_q T_{3+3i+q}^h),  gB_m^h = g_i T_{3+3i+m}^h,
//   r_n = lambda_{n+1} / lambda_n = (2n+1)/(n+1),
// so the recurrence runs to level P + 1.  k + e_1 leaves the subset when
// k1 = 1; Laplace's identity on level n+1 gives
//   c^{(2,a,b)} = -[(a+2)(a+1) c^{(0,a+2,b)} + (b+2)(b+1) c^{(0,a,b+2)}] / 2.
// One warp per batch, one target per lane, three levels in registers; the
// grid is resident and its warps take batches from a work queue (queue: a
// counter zeroed before the launch), as in the forward far field.
template <int P>
__device__ __noinline__ void far_adj_target32_batch(const double* __restrict__ ts, const double* __restrict__ gs,
                                                    int64_t M, const float4* __restrict__ geo32,
                                                    const float* __restrict__ ab, const int64_t* __restrict__ far_off,
                                                    const ListEntry* __restrict__ far_list, double* __restrict__ gt,
                                                    int64_t b, int lane)
{
    constexpr int H = (P + 1) * (P + 1);
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    float xh[3] = {0, 0, 0}, xl[3] = {0, 0, 0}, g[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            const double v = ts[a * M + m];
            xh[a] = __double2float_rn(v);
            xl[a] = __double2float_rn(v - (double)xh[a]);
            g[a] = __double2float_rn(gs[a * M + m]);
        }
    // per-entry contributions summed by compensated FP32 summation
    float G[3] = {0.f, 0.f, 0.f}, K[3] = {0.f, 0.f, 0.f};
    for (int64_t e = far_off[b]; e < far_off[b + 1]; e++) {
        const ListEntry le = far_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const float4 gh = __ldg(geo32 + 2 * (int64_t)le.node), gl = __ldg(geo32 + 2 * (int64_t)le.node + 1);
        const float d0 = ((xh[0] - gh.x) + (xl[0] - gl.x)) * gh.w;
        const float d1 = ((xh[1] - gh.y) + (xl[1] - gl.y)) * gh.w;
        const float d2 = ((xh[2] - gh.z) + (xl[2] - gl.z)) * gh.w;
        float R2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        if (!in) R2 = 1.0f;
        const float iR = rsqrtf(R2), iR2 = iR * iR;
        const float v0 = d0 * iR2, v1 = d1 * iR2, v2 = d2 * iR2;
        const float4* __restrict__ tab = reinterpret_cast<const float4*>(ab + (int64_t)le.node * H * 12);
        float cs[3][2 * P + 3];  // levels n-1, n, n+1 (slot = level mod 3)
        cs[0][0] = 1.0f;
        cs[1][0] = v1, cs[1][1] = v2, cs[1][2] = v0;  // level 1: (0,1,0), (0,0,1), (1,0,0)
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int n = 0; n <= P; n++) {
            if (n >= 1) {  // level n + 1 from levels n and n - 1
                const float kap = c_lev32.kappa[n + 1] * iR2;
#pragma unroll
                for (int h = 2 * n + 2; h >= 0; h--)
                    cs[(n + 1) % 3][h] = hcoef_r(cs[n % 3], cs[(n + 2) % 3], n + 1, h, v0, v1, v2, kap);
            }
            const float rn = (float)(2 * n + 1) / (float)(n + 1);
            const float* C1 = cs[(n + 1) % 3];
#pragma unroll
            for (int h = 0; h <= 2 * n; h++) {
                const float4 ta = __ldg(tab + 3 * (n * n + h)), tb = __ldg(tab + 3 * (n * n + h) + 1),
                             tc = __ldg(tab + 3 * (n * n + h) + 2);
                // T_0..2 = ta.xyz; T_3+3i+q: i = 0 -> ta.w tb.x tb.y, i = 1 -> tb.z tb.w tc.x,
                // i = 2 -> tc.y tc.z tc.w
                const float gB0 = fmaf(g[0], ta.w, fmaf(g[1], tb.z, g[2] * tc.y));
                const float gB1 = fmaf(g[0], tb.x, fmaf(g[1], tb.w, g[2] * tc.z));
                const float gB2 = fmaf(g[0], tb.y, fmaf(g[1], tc.x, g[2] * tc.w));
                // alpha^k = g.T_0..2 + sum_q d'_q gB_q  (sum_iq g_i d'_q T_{3+3i+q} regrouped)
                float al = fmaf(g[0], ta.x, fmaf(g[1], ta.y, g[2] * ta.z));
                al = fmaf(d0, gB0, fmaf(d1, gB1, fmaf(d2, gB2, al)));
                const float c = cs[n % 3][h];
                a0 = fmaf(c, gB0, a0);
                a1 = fmaf(c, gB1, a1);
                a2 = fmaf(c, gB2, a2);
                float e0, e1, e2;  // (k_m + 1) r_n c^{k+e_m}
                if (h <= n) {      // k = (0, n-h, h)
                    const int k2 = n - h, k3 = h;
                    e0 = rn * C1[n + 2 + h];
                    e1 = (float)(k2 + 1) * rn * C1[h];
                    e2 = (float)(k3 + 1) * rn * C1[h + 1];
                } else {  // k = (1, a, b)
                    const int bq = h - n - 1, aq = n - 1 - bq;
                    e0 = -rn * fmaf((float)((aq + 2) * (aq + 1)), C1[bq], (float)((bq + 2) * (bq + 1)) * C1[bq + 2]);
                    e1 = (float)(aq + 1) * rn * C1[h + 1];
                    e2 = (float)(bq + 1) * rn * C1[h + 2];
                }
                a0 = fmaf(-e0, al, a0);
                a1 = fmaf(-e1, al, a1);
                a2 = fmaf(-e2, al, a2);
            }
        }
        if (in) {
            const float s = iR * gh.w;  // 1/R' and d'/dx = 1/rho
            kahan_add(G[0], K[0], a0 * s);
            kahan_add(G[1], K[1], a1 * s);
            kahan_add(G[2], K[2], a2 * s);
        }
    }
    if (valid) {
        gt[m] = (double)G[0] - (double)K[0];
        gt[M + m] = (double)G[1] - (double)K[1];
        gt[2 * M + m] = (double)G[2] - (double)K[2];
    }
}

// c^k of hcoef_r for the two targets of a lane at once (target a, target b
// in the two halves of each FP32x2 register pair); nkap = -kappa_n / R'^2.
__device__ __forceinline__ float2 hcoef_pair(const float2* R1, const float2* R2, int n, int h, float2 v0, float2 v1,
                                             float2 v2, float2 nkap)
{
    float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
    bool any1 = false, any2 = false;
    if (h <= n) {
        const int k3 = h, k2 = n - h;
        if (k2 >= 1) s1 = __fmul2_rn(v1, R1[k3]), any1 = true;
        if (k3 >= 1) s1 = any1 ? __ffma2_rn(v2, R1[k3 - 1], s1) : __fmul2_rn(v2, R1[k3 - 1]);
        if (k2 >= 2) s2 = R2[k3], any2 = true;
        if (k3 >= 2) s2 = any2 ? __fadd2_rn(s2, R2[k3 - 2]) : R2[k3 - 2], any2 = true;
    } else {
        const int k3 = h - n - 1, k2 = n - 1 - k3;
        s1 = __fmul2_rn(v0, R1[k3]);
        if (k2 >= 1) s1 = __ffma2_rn(v1, R1[n + k3], s1);
        if (k3 >= 1) s1 = __ffma2_rn(v2, R1[n + k3 - 1], s1);
        if (k2 >= 2) s2 = R2[n - 1 + k3], any2 = true;
        if (k3 >= 2) s2 = any2 ? __fadd2_rn(s2, R2[n - 3 + k3]) : R2[n - 3 + k3], any2 = true;
    }
    return any2 ? __ffma2_rn(nkap, s2, s1) : s1;
}

__device__ __forceinline__ float2 f2(float x) { return make_float2(x, x); }

constexpr int kFarAdjPairMaxP = 10;  // largest P of the two-target form (register budget)

// The target side for batches 2B and 2B+1 (the second may not exist) on one
// warp, two targets per lane, over the merge of their far lists (tree
// preorder; a cluster in both lists is evaluated once for both): the
// arithmetic of far_adj_target32_batch on packed FP32x2 operations, every
// table value loaded once for both targets.  Levels n - 1 and n + 1 share a
// slot (level n + 1 overwrites level n - 1 in place, positions running
// downward: a coefficient reads level n - 1 only at positions <= its own).
template <int P>
__device__ __noinline__ void far_adj_target32_pair(const double* __restrict__ ts, const double* __restrict__ gs,
                                                   int64_t M, const int4* __restrict__ topo,
                                                   const float4* __restrict__ geo32, const float* __restrict__ ab,
                                                   const int64_t* __restrict__ far_off,
                                                   const ListEntry* __restrict__ far_list, double* __restrict__ gt,
                                                   int64_t B, int lane)
{
    constexpr int H = (P + 1) * (P + 1);
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t ba = 2 * B, bb = 2 * B + 1;
    const int64_t ma = ba * kBatch + lane, mb = bb * kBatch + lane;
    const bool va = ma < M, vb = mb < M;
    float2 xh[3], xl[3], g[3];
    for (int a = 0; a < 3; a++) {
        const double xa = va ? ts[a * M + ma] : 0.0, xb = vb ? ts[a * M + mb] : 0.0;
        const float ha = __double2float_rn(xa), hb = __double2float_rn(xb);
        xh[a] = make_float2(ha, hb);
        xl[a] = make_float2(__double2float_rn(xa - (double)ha), __double2float_rn(xb - (double)hb));
        g[a] = make_float2(va ? __double2float_rn(gs[a * M + ma]) : 0.f, vb ? __double2float_rn(gs[a * M + mb]) : 0.f);
    }
    // per-entry contributions summed by compensated FP32 summation
    float Ga[3] = {0.f, 0.f, 0.f}, Ka[3] = {0.f, 0.f, 0.f}, Gb[3] = {0.f, 0.f, 0.f}, Kb[3] = {0.f, 0.f, 0.f};
    int64_t ia = far_off[ba], ea = far_off[ba + 1], ib = 0, eb = 0;
    if (bb < nbatch) {
        ib = far_off[bb];
        eb = far_off[bb + 1];
    }
    ListEntry la{0, 0}, lb{0, 0};
    int4 qa = make_int4(0, 0, 0, 0), qb = make_int4(0, 0, 0, 0);
    if (ia < ea) {
        la = far_list[ia];
        qa = topo[la.node];
    }
    if (ib < eb) {
        lb = far_list[ib];
        qb = topo[lb.node];
    }
    while (ia < ea || ib < eb) {
        bool takeA, takeB;
        if (ia >= ea) {
            takeA = false, takeB = true;
        } else if (ib >= eb) {
            takeA = true, takeB = false;
        } else if (la.node == lb.node) {
            takeA = takeB = true;
        } else {
            takeA = qa.x < qb.x || (qa.x == qb.x && (qa.y > qb.y || (qa.y == qb.y && la.node < lb.node)));
            takeB = !takeA;
        }
        const int node = takeA ? la.node : lb.node;
        const bool inA = takeA && ((la.mask >> lane) & 1u), inB = takeB && ((lb.mask >> lane) & 1u);
        const float4 gh = __ldg(geo32 + 2 * (int64_t)node), gl = __ldg(geo32 + 2 * (int64_t)node + 1);
        using nearpair::sub2;
        const float2 d0 = __fmul2_rn(__fadd2_rn(sub2(xh[0], f2(gh.x)), sub2(xl[0], f2(gl.x))), f2(gh.w));
        const float2 d1 = __fmul2_rn(__fadd2_rn(sub2(xh[1], f2(gh.y)), sub2(xl[1], f2(gl.y))), f2(gh.w));
        const float2 d2 = __fmul2_rn(__fadd2_rn(sub2(xh[2], f2(gh.z)), sub2(xl[2], f2(gl.z))), f2(gh.w));
        float2 R2 = __ffma2_rn(d0, d0, __ffma2_rn(d1, d1, __fmul2_rn(d2, d2)));
        if (!inA) R2.x = 1.0f;
        if (!inB) R2.y = 1.0f;
        const float2 iR = make_float2(rsqrtf(R2.x), rsqrtf(R2.y)), iR2 = __fmul2_rn(iR, iR);
        const float2 v0 = __fmul2_rn(d0, iR2), v1 = __fmul2_rn(d1, iR2), v2 = __fmul2_rn(d2, iR2);
        const float4* __restrict__ tab = reinterpret_cast<const float4*>(ab + (int64_t)node * H * 12);
        float2 cs[2][2 * P + 3];  // level n in slot n & 1
        cs[0][0] = f2(1.0f);
        cs[1][0] = v1, cs[1][1] = v2, cs[1][2] = v0;  // level 1: (0,1,0), (0,0,1), (1,0,0)
        float2 a0 = f2(0.f), a1 = f2(0.f), a2 = f2(0.f);
#pragma unroll
        for (int n = 0; n <= P; n++) {
            if (n >= 1) {  // level n + 1 from levels n and n - 1, over level n - 1
                const float2 nkap = make_float2(-c_lev32.kappa[n + 1] * iR2.x, -c_lev32.kappa[n + 1] * iR2.y);
#pragma unroll
                for (int h = 2 * n + 2; h >= 0; h--)
                    cs[(n + 1) & 1][h] = hcoef_pair(cs[n & 1], cs[(n + 1) & 1], n + 1, h, v0, v1, v2, nkap);
            }
            const float rn = (float)(2 * n + 1) / (float)(n + 1);
            const float2* C1 = cs[(n + 1) & 1];
#pragma unroll
            for (int h = 0; h <= 2 * n; h++) {
                const float4 ta = __ldg(tab + 3 * (n * n + h)), tb = __ldg(tab + 3 * (n * n + h) + 1),
                             tc = __ldg(tab + 3 * (n * n + h) + 2);
                const float2 gB0 = __ffma2_rn(g[0], f2(ta.w), __ffma2_rn(g[1], f2(tb.z), __fmul2_rn(g[2], f2(tc.y))));
                const float2 gB1 = __ffma2_rn(g[0], f2(tb.x), __ffma2_rn(g[1], f2(tb.w), __fmul2_rn(g[2], f2(tc.z))));
                const float2 gB2 = __ffma2_rn(g[0], f2(tb.y), __ffma2_rn(g[1], f2(tc.x), __fmul2_rn(g[2], f2(tc.w))));
                // alpha^k = g.T_0..2 + sum_q d'_q gB_q  (sum_iq g_i d'_q T_{3+3i+q} regrouped)
                float2 al = __ffma2_rn(g[0], f2(ta.x), __ffma2_rn(g[1], f2(ta.y), __fmul2_rn(g[2], f2(ta.z))));
                al = __ffma2_rn(d0, gB0, __ffma2_rn(d1, gB1, __ffma2_rn(d2, gB2, al)));
                const float2 c = cs[n & 1][h];
                a0 = __ffma2_rn(c, gB0, a0);
                a1 = __ffma2_rn(c, gB1, a1);
                a2 = __ffma2_rn(c, gB2, a2);
                float2 e0, e1, e2;  // (k_m + 1) r_n c^{k+e_m}
                if (h <= n) {       // k = (0, n-h, h)
                    const int k2 = n - h, k3 = h;
                    e0 = __fmul2_rn(f2(rn), C1[n + 2 + h]);
                    e1 = __fmul2_rn(f2((float)(k2 + 1) * rn), C1[h]);
                    e2 = __fmul2_rn(f2((float)(k3 + 1) * rn), C1[h + 1]);
                } else {  // k = (1, a, b)
                    const int bq = h - n - 1, aq = n - 1 - bq;
                    e0 = __fmul2_rn(f2(-rn), __ffma2_rn(f2((float)((aq + 2) * (aq + 1))), C1[bq],
                                                       __fmul2_rn(f2((float)((bq + 2) * (bq + 1))), C1[bq + 2])));
                    e1 = __fmul2_rn(f2((float)(aq + 1) * rn), C1[h + 1]);
                    e2 = __fmul2_rn(f2((float)(bq + 1) * rn), C1[h + 2]);
                }
                a0 = __ffma2_rn(make_float2(-e0.x, -e0.y), al, a0);
                a1 = __ffma2_rn(make_float2(-e1.x, -e1.y), al, a1);
                a2 = __ffma2_rn(make_float2(-e2.x, -e2.y), al, a2);
                // keep the table loads of later coefficients from being
                // hoisted here: that would exhaust the registers
                asm volatile("" ::: "memory");
            }
        }
        const float2 sc = __fmul2_rn(iR, f2(gh.w));  // 1/R' and d'/dx = 1/rho
        if (inA) {
            kahan_add(Ga[0], Ka[0], a0.x * sc.x);
            kahan_add(Ga[1], Ka[1], a1.x * sc.x);
            kahan_add(Ga[2], Ka[2], a2.x * sc.x);
        }
        if (inB) {
            kahan_add(Gb[0], Kb[0], a0.y * sc.y);
            kahan_add(Gb[1], Kb[1], a1.y * sc.y);
            kahan_add(Gb[2], Kb[2], a2.y * sc.y);
        }
        if (takeA && ++ia < ea) {
            la = far_list[ia];
            qa = topo[la.node];
        }
        if (takeB && ++ib < eb) {
            lb = far_list[ib];
            qb = topo[lb.node];
        }
    }
    if (va) {
        gt[ma] = (double)Ga[0] - (double)Ka[0];
        gt[M + ma] = (double)Ga[1] - (double)Ka[1];
        gt[2 * M + ma] = (double)Ga[2] - (double)Ka[2];
    }
    if (vb) {
        gt[mb] = (double)Gb[0] - (double)Kb[0];
        gt[M + mb] = (double)Gb[1] - (double)Kb[1];
        gt[2 * M + mb] = (double)Gb[2] - (double)Kb[2];
    }
}

// One resident grid of single-warp blocks taking batch pairs from a queue.
template <int P>
__global__ void __launch_bounds__(32)
    k_far_adj_target32p(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                        const int4* __restrict__ topo, const float4* __restrict__ geo32, const float* __restrict__ ab,
                        const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list,
                        double* __restrict__ gt, unsigned* __restrict__ queue)
{
    const int lane = threadIdx.x & 31;
    const int64_t nsuper = ((M + kBatch - 1) / kBatch + 1) / 2;
    for (;;) {
        unsigned B = 0;
        if (lane == 0) B = atomicAdd(queue, 1u);
        B = __shfl_sync(0xffffffffu, B, 0);
        if ((int64_t)B >= nsuper) break;
        far_adj_target32_pair<P>(ts, gs, M, topo, geo32, ab, far_off, far_list, gt, (int64_t)B, lane);
    }
}

template <int P>
__global__ void __launch_bounds__(32)
    k_far_adj_target32(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                       const float4* __restrict__ geo32, const float* __restrict__ ab,
                       const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list,
                       double* __restrict__ gt, unsigned* __restrict__ queue)
{
    const int lane = threadIdx.x & 31;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    for (;;) {
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(queue, 1u);
        b = __shfl_sync(0xffffffffu, b, 0);
        if ((int64_t)b >= nbatch) break;
        far_adj_target32_batch<P>(ts, gs, M, geo32, ab, far_off, far_list, gt, (int64_t)b, lane);
    }
}

// Source side.  The forward map is linear in the folded tables:
//   dL/dT_i^h = sum_m g_i^m c^h(v_m)/R'_m,  dL/dT_{3+3i+q}^h = sum_m g_i^m d'_qm c^h(v_m)/R'_m,
// over the targets m that accept the cluster.  Cluster-major over the far
// entries sorted by cluster; per entry every lane (target) computes its
// coefficients into shared memory, then each lane sums, for the coefficients
// it owns, over the 32 targets (a 32 x (P+1)^2 by 32 x 12 product); the
// accumulators go to the cluster's FP64 folded adjoint tables with atomics
// when the cluster changes.  Lanes outside the mask carry g = 0.
template <int P>
__global__ void __launch_bounds__(32)
    k_far_adj_source32(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                       const float4* __restrict__ geo32, const uint64_t* __restrict__ skeys,
                       const int32_t* __restrict__ sidx, const ListEntry* __restrict__ far_list,
                       const int32_t* __restrict__ ebatch, int64_t nent, int chunk, double* __restrict__ fbar)
{
    constexpr int H = (P + 1) * (P + 1);
    constexpr int NPL = (H + 31) / 32;
    __shared__ float sc[H][33];
    __shared__ __align__(16) float wt[32][12];
    const int lane = threadIdx.x & 31;
    const int64_t j0 = (int64_t)blockIdx.x * chunk;
    if (j0 >= nent) return;
    const int64_t j1 = min(nent, j0 + chunk);
    float2 acc[NPL][6];  // components (2c, 2c+1) packed
#pragma unroll
    for (int q = 0; q < NPL; q++)
#pragma unroll
        for (int c = 0; c < 6; c++) acc[q][c] = make_float2(0.f, 0.f);
    int64_t cur = -1;
    for (int64_t j = j0; j <= j1; j++) {
        const int64_t node = j < j1 ? (int64_t)skeys[j] : -2;
        if (node != cur) {
            if (cur >= 0) {
#pragma unroll
                for (int q = 0; q < NPL; q++) {
                    const int h = lane + 32 * q;
                    if (h < H)
                        for (int c = 0; c < 6; c++) {
                            atomicAdd(&fbar[(cur * H + h) * 12 + 2 * c], (double)acc[q][c].x);
                            atomicAdd(&fbar[(cur * H + h) * 12 + 2 * c + 1], (double)acc[q][c].y);
                        }
                }
            }
#pragma unroll
            for (int q = 0; q < NPL; q++)
#pragma unroll
                for (int c = 0; c < 6; c++) acc[q][c] = make_float2(0.f, 0.f);
            cur = node;
        }
        if (j == j1) break;
        const int32_t e = sidx[j];
        const unsigned mask = far_list[e].mask;
        const int64_t m = (int64_t)ebatch[e] * kBatch + lane;
        const bool in = (mask >> lane) & 1u;
        float xh[3] = {0, 0, 0}, xl[3] = {0, 0, 0}, g[3] = {0, 0, 0};
        if (in)
            for (int a = 0; a < 3; a++) {
                const double v = ts[a * M + m];
                xh[a] = __double2float_rn(v);
                xl[a] = __double2float_rn(v - (double)xh[a]);
                g[a] = __double2float_rn(gs[a * M + m]);
            }
        const float4 gh = __ldg(geo32 + 2 * node), gl = __ldg(geo32 + 2 * node + 1);
        const float d0 = ((xh[0] - gh.x) + (xl[0] - gl.x)) * gh.w;
        const float d1 = ((xh[1] - gh.y) + (xl[1] - gl.y)) * gh.w;
        const float d2 = ((xh[2] - gh.z) + (xl[2] - gl.z)) * gh.w;
        float R2 = fmaf(d0, d0, fmaf(d1, d1, d2 * d2));
        if (!in) R2 = 1.0f;
        const float iR = rsqrtf(R2), iR2 = iR * iR;
        const float v0 = d0 * iR2, v1 = d1 * iR2, v2 = d2 * iR2;
        __syncwarp();
        {
            float* w = wt[lane];
            w[0] = g[0], w[1] = g[1], w[2] = g[2];
            w[3] = g[0] * d0, w[4] = g[0] * d1, w[5] = g[0] * d2;
            w[6] = g[1] * d0, w[7] = g[1] * d1, w[8] = g[1] * d2;
            w[9] = g[2] * d0, w[10] = g[2] * d1, w[11] = g[2] * d2;
        }
        float cs[2][2 * P + 1];
        cs[0][0] = 1.0f;
        sc[0][lane] = iR;
#pragma unroll
        for (int n = 1; n <= P; n++) {
            const float kap = c_lev32.kappa[n] * iR2;
#pragma unroll
            for (int h = 2 * n; h >= 0; h--) {
                const float cf = hcoef_r(cs[(n - 1) & 1], cs[n & 1], n, h, v0, v1, v2, kap);
                cs[n & 1][h] = cf;
                sc[n * n + h][lane] = cf * iR;
            }
        }
        __syncwarp();
        for (int t = 0; t < 32; t++) {
            const float4* w4 = reinterpret_cast<const float4*>(wt[t]);
            const float4 wa = w4[0], wb = w4[1], wc = w4[2];
            const float2 w01 = make_float2(wa.x, wa.y), w23 = make_float2(wa.z, wa.w), w45 = make_float2(wb.x, wb.y),
                         w67 = make_float2(wb.z, wb.w), w89 = make_float2(wc.x, wc.y), wab = make_float2(wc.z, wc.w);
#pragma unroll
            for (int q = 0; q < NPL; q++) {
                const int h = lane + 32 * q;
                const float sv = h < H ? sc[h < H ? h : 0][t] : 0.f;
                const float2 s2 = make_float2(sv, sv);
                acc[q][0] = __ffma2_rn(s2, w01, acc[q][0]);
                acc[q][1] = __ffma2_rn(s2, w23, acc[q][1]);
                acc[q][2] = __ffma2_rn(s2, w45, acc[q][2]);
                acc[q][3] = __ffma2_rn(s2, w67, acc[q][3]);
                acc[q][4] = __ffma2_rn(s2, w89, acc[q][4]);
                acc[q][5] = __ffma2_rn(s2, wab, acc[q][5]);
            }
        }
    }
}

// Adjoint of the folding (k_fold_tables): from the adjoint of the folded,
// lambda-scaled tables (fbar, [node][(P+1)^2][12]) to the adjoint of the full
// tables (abar, [node][C(P+3,3)][12]).  The folding pushes row k1 of a level
// onto rows k1-2 (k1 from n down to 2) and keeps k1 in {0, 1}, scaled by
// lambda_n; its transpose seeds k1 in {0, 1} with lambda_n fbar and pulls
// row k1 from rows k1-2, k1 from 2 up to n.  FP64, one block per cluster.
__global__ void k_unfold_adj(const double* __restrict__ fbar, int64_t nnodes, int p, double* __restrict__ abar)
{
    extern __shared__ double lvb[];  // one level: [position][12]
    const int64_t node = blockIdx.x;
    const int P = p + 2;
    const int C2 = ncoef(P), H = hsize(P);
    double lambda = 1.0;
    for (int n = 0; n <= P; n++) {
        if (n > 0) lambda *= (double)(2 * n - 1) / (double)n;
        const int L = level_size(n);
        for (int q = threadIdx.x; q < L * 12; q += blockDim.x) lvb[q] = 0.0;
        __syncthreads();
        for (int q = threadIdx.x; q < (2 * n + 1) * 12; q += blockDim.x) {
            const int h = q / 12, c = q % 12;
            const int pos = h <= n ? n * (n + 1) / 2 + h : (n - 1) * n / 2 + (h - n - 1);
            lvb[pos * 12 + c] = lambda * fbar[((int64_t)node * H + n * n + h) * 12 + c];
        }
        __syncthreads();
        for (int k1 = 2; k1 <= n; k1++) {
            const int a = n - k1, a2 = a + 2;
            const double inv = 1.0 / ((double)k1 * (k1 - 1));
            for (int q = threadIdx.x; q < (a + 1) * 12; q += blockDim.x) {
                const int k3 = q / 12, c = q % 12, k2 = a - k3;
                const int src = a * (a + 1) / 2 + k3;
                const int dst2 = a2 * (a2 + 1) / 2 + k3, dst3 = dst2 + 2;
                const double f2 = -(double)((k2 + 2) * (k2 + 1)) * inv, f3 = -(double)((k3 + 2) * (k3 + 1)) * inv;
                lvb[src * 12 + c] += f2 * lvb[dst2 * 12 + c] + f3 * lvb[dst3 * 12 + c];
            }
            __syncthreads();
        }
        const int base = n > 0 ? ncoef(n - 1) : 0;
        for (int q = threadIdx.x; q < L * 12; q += blockDim.x)
            abar[((int64_t)node * C2 + base) * 12 + q] = lvb[q];
        __syncthreads();
    }
}

// ------------------------------------------- adjoint moments (table transpose)
// One block per cluster; its threads scatter the transpose of the table map of
// tc_moments.cu (k_ab_tables) into shared memory (shared-memory FP64 atomics,
// so the order of the additions varies), so each moment gathers
//   Lambda_c^k = sum over the table entries that read M_c^k of (entry
//   coefficient) x (scaled adjoint table entry).
__global__ void k_lambda(const double* __restrict__ abar, const double* __restrict__ invrho, int p,
                         double* __restrict__ lam)
{
    extern __shared__ double ls[];
    const int64_t node = blockIdx.x;
    const int C = ncoef(p), C2 = ncoef(p + 2);
    for (int q = threadIdx.x; q < 12 * C; q += blockDim.x) ls[q] = 0.0;
    __syncthreads();
    {
        const double ir = invrho[node];
        const double third = 1.0 / 3.0;
        auto add = [&](int c, int k1, int k2, int k3, double v) {
            if (k1 < 0 || k2 < 0 || k3 < 0 || k1 + k2 + k3 > p) return;
            atomicAdd(&ls[c * C + flat_index(k1, k2, k3)], v);
        };
        for (int kidx = threadIdx.x; kidx < C2; kidx += blockDim.x) {
            int kp[3];
            unflatten(kidx, kp[0], kp[1], kp[2]);
            const int n = kp[0] + kp[1] + kp[2];
            double sB = 1.0;
            for (int q = 0; q < n; q++) sB *= ir;
            const double sA = sB * ir;
            const double* ab = abar + (node * C2 + kidx) * 12;
            for (int i = 0; i < 3; i++) {
                const int ei[3] = {i == 0, i == 1, i == 2};
                const double Ab = ab[i] * sA;
                if (Ab != 0.0) {
                    add(i, kp[0], kp[1], kp[2], Ab);
                    for (int j = 0; j < 3; j++) {
                        const int ej[3] = {j == 0, j == 1, j == 2};
                        add(j, kp[0] - ei[0] + ej[0], kp[1] - ei[1] + ej[1], kp[2] - ei[2] + ej[2], -kp[i] * Ab);
                    }
                    for (int l = 0; l < 3; l++) {
                        const int el[3] = {l == 0, l == 1, l == 2};
                        add(3 + 3 * i + l, kp[0] - el[0], kp[1] - el[1], kp[2] - el[2], third * kp[l] * Ab);
                    }
                    for (int j = 0; j < 3; j++) {
                        const int ej[3] = {j == 0, j == 1, j == 2};
                        const double cj = (double)(kp[i] - (i == j)) * kp[j];
                        if (cj == 0.0) continue;
                        for (int l = 0; l < 3; l++) {
                            const int el[3] = {l == 0, l == 1, l == 2};
                            add(3 + 3 * j + l, kp[0] - ei[0] - ej[0] + el[0], kp[1] - ei[1] - ej[1] + el[1],
                                kp[2] - ei[2] - ej[2] + el[2], -third * cj * Ab);
                        }
                    }
                }
                for (int l = 0; l < 3; l++) {
                    const double Bb = ab[3 + 3 * i + l] * sB;
                    if (Bb == 0.0) continue;
                    add(l, kp[0] - ei[0], kp[1] - ei[1], kp[2] - ei[2], kp[i] * Bb);
                    for (int j = 0; j < 3; j++) {
                        const int ej[3] = {j == 0, j == 1, j == 2};
                        const double cj = (double)kp[i] * (kp[j] - (i == j));
                        if (cj == 0.0) continue;
                        add(3 + 3 * j + l, kp[0] - ei[0] - ej[0], kp[1] - ei[1] - ej[1], kp[2] - ei[2] - ej[2],
                            third * cj * Bb);
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 12 * C; q += blockDim.x) lam[node * 12 * C + q] = ls[q];
}

// Pascal's triangle up to row kPMax.
struct Binom {
    double v[kPMax + 1][kPMax + 1];
};
__host__ __device__ constexpr Binom make_binom()
{
    Binom b{};
    for (int n = 0; n <= kPMax; n++) {
        b.v[n][0] = 1.0;
        for (int k = 1; k <= n; k++) b.v[n][k] = b.v[n - 1][k - 1] + (k <= n - 1 ? b.v[n - 1][k] : 0.0);
    }
    return b;
}
__constant__ Binom c_binom = make_binom();

// Downward pass: the adjoint polynomial of the parent, sum_k L^k (y - y_P)^k,
// re-expanded about the child centre (y - y_P = (y - y_C) + s, s = y_C - y_P):
//   L'^j = sum_{k >= j} binom(k, j) s^(k-j) L^k,  added to the child's own.
// Grid (nodes of one level, 3): each block takes 4 of the 12 components, so
// that the upper levels, with few nodes, still spread over the GPU.
__global__ void k_l2l(const int4* __restrict__ info, const Geo* __restrict__ geo, int64_t lb, int64_t le, int p,
                      const double* __restrict__ lam, double* __restrict__ lamacc)
{
    __shared__ double sp[3][kPMax + 1];
    const int64_t node = lb + blockIdx.x;
    if (node >= le) return;
    const int C = ncoef(p);
    const int64_t parent = info[node].y;
    const int c0 = 4 * blockIdx.y;  // this block's components c0 .. c0 + 3
    if (parent < 0) {
        for (int q = threadIdx.x; q < 4 * C; q += blockDim.x)
            lamacc[node * 12 * C + c0 * C + q] = lam[node * 12 * C + c0 * C + q];
        return;
    }
    const Geo gc = geo[node], gp = geo[parent];
    if (threadIdx.x < 3) {
        const double s = threadIdx.x == 0 ? gc.x - gp.x : (threadIdx.x == 1 ? gc.y - gp.y : gc.z - gp.z);
        double v = 1.0;
        sp[threadIdx.x][0] = 1.0;
        for (int k = 1; k <= p; k++) {
            v *= s;
            sp[threadIdx.x][k] = v;
        }
    }
    __syncthreads();
    const double* lp = lamacc + parent * 12 * C;
    for (int jdx = threadIdx.x; jdx < C; jdx += blockDim.x) {
        int j1, j2, j3;
        unflatten(jdx, j1, j2, j3);
        double acc[4];
        for (int c = 0; c < 4; c++) acc[c] = lam[(node * 12 + c0 + c) * C + jdx];
        for (int k1 = j1; k1 <= p; k1++) {
            const double w1 = c_binom.v[k1][j1] * sp[0][k1 - j1];
            for (int k2 = j2; k1 + k2 <= p; k2++) {
                const double w12 = w1 * c_binom.v[k2][j2] * sp[1][k2 - j2];
                for (int k3 = j3; k1 + k2 + k3 <= p; k3++) {
                    const double wk = w12 * c_binom.v[k3][j3] * sp[2][k3 - j3];
                    const int kidx = flat_index(k1, k2, k3);
                    for (int c = 0; c < 4; c++) acc[c] = fma(wk, lp[(c0 + c) * C + kidx], acc[c]);
                }
            }
        }
        for (int c = 0; c < 4; c++) lamacc[(node * 12 + c0 + c) * C + jdx] = acc[c];
    }
}

// Per particle of a leaf: Q_c(y) = sum_k L_c^k (y - y_L)^k and
// grad_y sum_c w_c Q_c(y); writes dL/df, dL/dh, dL/dnu, dL/dx (far, source side).
// Grid (clusters, kLeafEvalSplit): the particles of a leaf are shared by
// kLeafEvalSplit blocks.
constexpr int kLeafEvalSplit = 8;

__global__ void k_leaf_eval(const int4* __restrict__ topo, const Geo* __restrict__ geo, const double* __restrict__ xs,
                            const double* __restrict__ ws, int64_t N, int p, const double* __restrict__ lamacc,
                            double* __restrict__ gfar)
{
    extern __shared__ double ll[];
    const int64_t node = blockIdx.x;
    const int4 t = topo[node];
    if (t.w != 0) return;
    const int C = ncoef(p);
    for (int q = threadIdx.x; q < 12 * C; q += blockDim.x) ll[q] = lamacc[node * 12 * C + q];
    __syncthreads();
    const Geo gc = geo[node];
    for (int i = t.x + blockIdx.y * blockDim.x + threadIdx.x; i < t.x + t.y; i += gridDim.y * blockDim.x) {
        const double dl[3] = {xs[i] - gc.x, xs[N + i] - gc.y, xs[2 * N + i] - gc.z};
        double w[12];
        for (int c = 0; c < 3; c++) w[c] = ws[c * N + i];
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++) w[3 + 3 * j + l] = ws[(3 + j) * N + i] * ws[(6 + l) * N + i];
        double Qv[12], gx[3] = {0, 0, 0};
        for (int c = 0; c < 12; c++) Qv[c] = 0.0;
        double p1 = 1.0, p1m = 0.0;
        for (int k1 = 0; k1 <= p; k1++) {
            double p2 = 1.0, p2m = 0.0;
            for (int k2 = 0; k1 + k2 <= p; k2++) {
                double p3 = 1.0, p3m = 0.0;
                for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                    const int kidx = flat_index(k1, k2, k3);
                    const double mono = p1 * p2 * p3;
                    double R = 0.0;
                    for (int c = 0; c < 12; c++) {
                        const double L = ll[c * C + kidx];
                        Qv[c] = fma(L, mono, Qv[c]);
                        R = fma(w[c], L, R);
                    }
                    gx[0] = fma(R, k1 * p1m * p2 * p3, gx[0]);
                    gx[1] = fma(R, k2 * p1 * p2m * p3, gx[1]);
                    gx[2] = fma(R, k3 * p1 * p2 * p3m, gx[2]);
                    p3m = p3;
                    p3 *= dl[2];
                }
                p2m = p2;
                p2 *= dl[1];
            }
            p1m = p1;
            p1 *= dl[0];
        }
        for (int a = 0; a < 3; a++) {
            gfar[a * N + i] = Qv[a];
            double gh = 0.0, gn = 0.0;
            for (int l = 0; l < 3; l++) gh += ws[(6 + l) * N + i] * Qv[3 + 3 * a + l];
            for (int j = 0; j < 3; j++) gn += ws[(3 + j) * N + i] * Qv[3 + 3 * j + a];
            gfar[(3 + a) * N + i] = gh;
            gfar[(6 + a) * N + i] = gn;
            gfar[(9 + a) * N + i] = gx[a];
        }
    }
}

// Mixed precision: the same evaluation in FP32 (the polynomial is the far
// field's adjoint expanded about the leaf centre, a convergent Taylor sum
// led by its low orders, so FP32 terms leave about 1e-7 relative error), the
// leaf's coefficients rounded to FP32 in shared memory.
__global__ void k_leaf_eval32(const int4* __restrict__ topo, const Geo* __restrict__ geo,
                              const double* __restrict__ xs, const double* __restrict__ ws, int64_t N, int p,
                              const double* __restrict__ lamacc, double* __restrict__ gfar)
{
    extern __shared__ float llf[];
    const int64_t node = blockIdx.x;
    const int4 t = topo[node];
    if (t.w != 0) return;
    const int C = ncoef(p);
    for (int q = threadIdx.x; q < 12 * C; q += blockDim.x) llf[q] = (float)lamacc[node * 12 * C + q];
    __syncthreads();
    const Geo gc = geo[node];
    for (int i = t.x + blockIdx.y * blockDim.x + threadIdx.x; i < t.x + t.y; i += gridDim.y * blockDim.x) {
        const float dl[3] = {(float)(xs[i] - gc.x), (float)(xs[N + i] - gc.y), (float)(xs[2 * N + i] - gc.z)};
        float w[12];
        for (int c = 0; c < 3; c++) w[c] = (float)ws[c * N + i];
        for (int j = 0; j < 3; j++)
            for (int l = 0; l < 3; l++) w[3 + 3 * j + l] = (float)(ws[(3 + j) * N + i] * ws[(6 + l) * N + i]);
        float Qv[12], gx[3] = {0.f, 0.f, 0.f};
        for (int c = 0; c < 12; c++) Qv[c] = 0.f;
        float p1 = 1.f, p1m = 0.f;
        for (int k1 = 0; k1 <= p; k1++) {
            float p2 = 1.f, p2m = 0.f;
            for (int k2 = 0; k1 + k2 <= p; k2++) {
                float p3 = 1.f, p3m = 0.f;
                for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                    const int kidx = flat_index(k1, k2, k3);
                    const float mono = p1 * p2 * p3;
                    float R = 0.f;
#pragma unroll
                    for (int c = 0; c < 12; c++) {
                        const float L = llf[c * C + kidx];
                        Qv[c] = fmaf(L, mono, Qv[c]);
                        R = fmaf(w[c], L, R);
                    }
                    gx[0] = fmaf(R, (float)k1 * p1m * p2 * p3, gx[0]);
                    gx[1] = fmaf(R, (float)k2 * p1 * p2m * p3, gx[1]);
                    gx[2] = fmaf(R, (float)k3 * p1 * p2 * p3m, gx[2]);
                    p3m = p3;
                    p3 *= dl[2];
                }
                p2m = p2;
                p2 *= dl[1];
            }
            p1m = p1;
            p1 *= dl[0];
        }
        for (int a = 0; a < 3; a++) {
            gfar[a * N + i] = Qv[a];
            double gh = 0.0, gn = 0.0;
            for (int l = 0; l < 3; l++) gh += ws[(6 + l) * N + i] * (double)Qv[3 + 3 * a + l];
            for (int j = 0; j < 3; j++) gn += ws[(3 + j) * N + i] * (double)Qv[3 + 3 * j + a];
            gfar[(3 + a) * N + i] = gh;
            gfar[(6 + a) * N + i] = gn;
            gfar[(9 + a) * N + i] = gx[a];
        }
    }
}

// Sum the parts and scatter from Morton order to the caller's order.
__global__ void k_adj_final(const double* __restrict__ gfar, const double* __restrict__ gnear,
                            const double* __restrict__ gt, const int32_t* __restrict__ perm, int64_t N, int self,
                            double* __restrict__ gf, double* __restrict__ gh, double* __restrict__ gnu,
                            double* __restrict__ gx)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int64_t d = perm[i];
    for (int a = 0; a < 3; a++) {
        if (gf) gf[a * N + d] = gfar[a * N + i] + gnear[a * N + i];
        if (gh) gh[a * N + d] = gfar[(3 + a) * N + i] + gnear[(3 + a) * N + i];
        if (gnu) gnu[a * N + d] = gfar[(6 + a) * N + i] + gnear[(6 + a) * N + i];
        if (gx) gx[a * N + d] = gfar[(9 + a) * N + i] + gnear[(9 + a) * N + i] + (self ? gt[a * N + i] : 0.0);
    }
}

__global__ void k_scatter3(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t M,
                           double* __restrict__ dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= M) return;
    const int64_t d = perm[i];
    for (int a = 0; a < 3; a++) dst[a * M + d] = src[a * M + i];
}

constexpr int kFarAdjChunk = 48;  // sorted far entries per warp in the cluster-major pass

template <typename TR, typename TC>
cudaError_t run_far_adj(tc_ctx* ctx, const double* ts, int64_t M, int p, cudaStream_t s)
{
    const int P = p + 2, Q = P + 1;
    const TC* ab = (const TC*)(ctx->precision == TC_FP64 ? ctx->ab64.p : ctx->ab32.p);
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    size_t sm1 = (size_t)(level_size(Q) + level_size(P)) * 32 * sizeof(TR) +
                 (size_t)(level_size(P) + level_size(P - 1)) * 32 * sizeof(TC);
    cudaError_t e =
        cudaFuncSetAttribute(k_far_adj_target<TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    ph_begin(ctx, TC_PH_ADJ_FAR_T);
    k_far_adj_target<TR, TC><<<(unsigned)nbatch, 32, sm1, s>>>(
        ts, ptr<double>(ctx->adj_gs), M, ptr<Geo>(ctx->node_geo), ptr<double>(ctx->node_invrho), ab, p,
        ptr<int64_t>(ctx->far_off), ptr<ListEntry>(ctx->far_list), ptr<double>(ctx->adj_gt));
    note_launch();
    ph_end(ctx, TC_PH_ADJ_FAR_T);
    const int64_t nent = ctx->far_entries;
    ph_begin(ctx, TC_PH_ADJ_FAR_S);
    if (nent > 0) {
        size_t sm2 = (size_t)(level_size(P) + level_size(P - 1)) * 32 * sizeof(TR) +
                     ((size_t)level_size(P) * 33 + 32 * 12 + (size_t)ncoef(P) * 12) * sizeof(TC);
        e = cudaFuncSetAttribute(k_far_adj_source<TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        if (e != cudaSuccess) return e;
        k_far_adj_source<TR, TC><<<grid_for(nent, kFarAdjChunk), 32, sm2, s>>>(
            ts, ptr<double>(ctx->adj_gs), M, ptr<Geo>(ctx->node_geo), ptr<double>(ctx->node_invrho), p,
            ptr<uint64_t>(ctx->adj_fkeys), ptr<int32_t>(ctx->adj_fidx), ptr<ListEntry>(ctx->far_list),
            ptr<int32_t>(ctx->adj_febatch), nent, kFarAdjChunk, ptr<double>(ctx->adj_abar));
        note_launch();
    }
    ph_end(ctx, TC_PH_ADJ_FAR_S);
    return cudaGetLastError();
}

// Mixed precision: the folded-table adjoint (target side, source side into
// the folded adjoint tables, then their unfolding into adj_abar).
template <int P>
cudaError_t run_far_adj32(tc_ctx* ctx, const double* ts, int64_t M, cudaStream_t s)
{
    const int p = P - 2;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t nnodes = ctx->nnodes;
    const int H = hsize(P);
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned* queue = reinterpret_cast<unsigned*>(ptr<char>(ctx->flags) + 192);
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    ph_begin(ctx, TC_PH_ADJ_FAR_T);
    // two targets per lane up to P = 10 (p = 8); above, the packed form runs
    // out of registers and the one-target form is used
    if constexpr (P <= kFarAdjPairMaxP) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_far_adj_target32p<P>, 32, 0);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::min<int64_t>((nbatch + 1) / 2, (int64_t)std::max(per_sm, 1) * sms);
        k_far_adj_target32p<P><<<(unsigned)grid, 32, 0, s>>>(ts, ptr<double>(ctx->adj_gs), M,
                                                             ptr<int4>(ctx->node_topo), ptr<float4>(ctx->geo32),
                                                             ptr<float>(ctx->abf32), ptr<int64_t>(ctx->far_off),
                                                             ptr<ListEntry>(ctx->far_list), ptr<double>(ctx->adj_gt),
                                                             queue);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_far_adj_target32<P>, 32, 0);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::min<int64_t>(nbatch, (int64_t)std::max(per_sm, 1) * sms);
        k_far_adj_target32<P><<<(unsigned)grid, 32, 0, s>>>(ts, ptr<double>(ctx->adj_gs), M,
                                                            ptr<float4>(ctx->geo32), ptr<float>(ctx->abf32),
                                                            ptr<int64_t>(ctx->far_off), ptr<ListEntry>(ctx->far_list),
                                                            ptr<double>(ctx->adj_gt), queue);
    }
    note_launch();
    ph_end(ctx, TC_PH_ADJ_FAR_T);
    e = ensure(ctx->adj_fbar, (size_t)nnodes * H * 12 * 8);
    if (e != cudaSuccess) return e;
    ph_begin(ctx, TC_PH_ADJ_FAR_S);
    e = cudaMemsetAsync(ctx->adj_fbar.p, 0, (size_t)nnodes * H * 12 * 8, s);
    if (e != cudaSuccess) return e;
    const int64_t nent = ctx->far_entries;
    if (nent > 0) {
        k_far_adj_source32<P><<<grid_for(nent, kFarAdjChunk), 32, 0, s>>>(
            ts, ptr<double>(ctx->adj_gs), M, ptr<float4>(ctx->geo32), ptr<uint64_t>(ctx->adj_fkeys),
            ptr<int32_t>(ctx->adj_fidx), ptr<ListEntry>(ctx->far_list), ptr<int32_t>(ctx->adj_febatch), nent,
            kFarAdjChunk, ptr<double>(ctx->adj_fbar));
        note_launch();
    }
    const size_t smem = (size_t)level_size(P) * 12 * sizeof(double);
    e = cudaFuncSetAttribute(k_unfold_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_unfold_adj<<<(unsigned)nnodes, 128, smem, s>>>(ptr<double>(ctx->adj_fbar), nnodes, p, ptr<double>(ctx->adj_abar));
    note_launch();
    ph_end(ctx, TC_PH_ADJ_FAR_S);
    return cudaGetLastError();
}

cudaError_t launch_far_adj32(tc_ctx* ctx, const double* ts, int64_t M, int p, cudaStream_t s)
{
    switch (p + 2) {
#define TC_FARADJ_CASE(P) \
    case P: return run_far_adj32<P>(ctx, ts, M, s);
        TC_FARADJ_CASE(2) TC_FARADJ_CASE(3) TC_FARADJ_CASE(4) TC_FARADJ_CASE(5) TC_FARADJ_CASE(6)
        TC_FARADJ_CASE(7) TC_FARADJ_CASE(8) TC_FARADJ_CASE(9) TC_FARADJ_CASE(10) TC_FARADJ_CASE(11)
        TC_FARADJ_CASE(12) TC_FARADJ_CASE(13) TC_FARADJ_CASE(14)
#undef TC_FARADJ_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace tc

using namespace tc;

#define TC_CK(call, where)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

extern "C" tc_status tc_adjoint(tc_ctx* ctx, const double* g, double* grad_f, double* grad_h, double* grad_nu,
                                double* grad_x, double* grad_t)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_adjoint: ctx is NULL");
    if (!ctx->have_eval) return fail(ctx, TC_ESTATE, "tc_adjoint: call tc_eval first");
    if (ctx->reg_eps > 0.0) return fail(ctx, TC_EINVAL, "tc_adjoint: not available for the regularized kernels");
    if (!g) return fail(ctx, TC_EINVAL, "tc_adjoint: g is NULL");
    if (ctx->eval_self && grad_t)
        return fail(ctx, TC_EINVAL, "tc_adjoint: grad_t must be NULL when targets are the sources (use grad_x)");
    TC_CK(join_moments(ctx), "adjoint");
    cudaStream_t s = ctx->stream;
    const int64_t N = ctx->N, M = ctx->M, nnodes = ctx->nnodes;
    const int p = ctx->ab_p;
    const int C = ncoef(p), C2 = ncoef(p + 2);
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int32_t* tperm = ctx->eval_self ? ptr<int32_t>(ctx->perm) : ptr<int32_t>(ctx->tperm);
    const double* ts = ctx->eval_self ? ptr<double>(ctx->xs) : ptr<double>(ctx->ts);

    TC_CK(ensure(ctx->adj_gs, (size_t)3 * M * 8), "alloc adjoint");
    TC_CK(ensure(ctx->adj_gt, (size_t)3 * M * 8), "alloc adjoint");
    TC_CK(ensure(ctx->adj_abar, (size_t)nnodes * C2 * 12 * 8), "alloc adjoint");
    TC_CK(ensure(ctx->adj_lam, (size_t)nnodes * 12 * C * 8), "alloc adjoint");
    TC_CK(ensure(ctx->adj_lamacc, (size_t)nnodes * 12 * C * 8), "alloc adjoint");
    TC_CK(ensure(ctx->adj_gfar, (size_t)12 * N * 8), "alloc adjoint");
    TC_CK(ensure(ctx->adj_gnear, (size_t)12 * N * 8), "alloc adjoint");

    if (!ctx->adj_lists_ready) {
        TC_CK(sort_list_entries(ptr<ListEntry>(ctx->far_list), ctx->far_entries, ptr<int64_t>(ctx->far_off), nbatch,
                                nnodes, ctx->adj_fkeys, ctx->adj_fkeys_alt, ctx->adj_fidx, ctx->adj_fidx_alt,
                                ctx->adj_febatch, ctx->adj_hist, s),
              "sort far entries");
        ctx->adj_lists_ready = 1;
    }
    // the near entries sorted by leaf (source side); in mixed precision the
    // leaf-major schedule too (target side), shared with the forward field
    NearSched sched;
    TC_CK(near_schedule(ctx, 0, sched, s), "near schedule");
    if (ctx->precision != TC_FP64) TC_CK(near_schedule(ctx, 1, sched, s), "near schedule");
    sched.queue = reinterpret_cast<unsigned*>(ptr<char>(ctx->flags) + 224);
    k_gather_g<<<grid_for(M, 256), 256, 0, s>>>(g, tperm, M, ptr<double>(ctx->adj_gs));
    note_launch();
    TC_CK(cudaMemsetAsync(ctx->adj_abar.p, 0, (size_t)nnodes * C2 * 12 * 8, s), "zero adjoint tables");

    // far field: target side (writes adj_gt) and source side (adjoint tables)
    cudaError_t e;
    if (ctx->precision == TC_FP64)
        e = run_far_adj<double, double>(ctx, ts, M, p, s);
    else
        e = launch_far_adj32(ctx, ts, M, p, s);
    TC_CK(e, "far adjoint");

    // Adjoint moments, downward pass (FP64) and per-particle evaluation:
    // they read only the far field's adjoint tables and write only the far
    // gradients, so they run on the second stream beside the near field
    // (FP32 pipe), which reads and writes none of that, and join before the
    // final sums.  Profile mode 2 keeps them on the first stream.
    TC_CK(second_stream(ctx), "second stream");
    cudaStream_t sr = ctx->profile == 2 ? s : ctx->stream2;
    if (sr != s) {
        TC_CK(cudaEventRecord(ctx->ev_fork, s), "fork");
        TC_CK(cudaStreamWaitEvent(sr, ctx->ev_fork, 0), "fork");
    }
    ph_begin(ctx, TC_PH_ADJ_REST, sr);
    size_t lsm = (size_t)12 * C * 8;
    TC_CK(cudaFuncSetAttribute(k_lambda, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm), "lambda attr");
    k_lambda<<<(unsigned)nnodes, 128, lsm, sr>>>(ptr<double>(ctx->adj_abar), ptr<double>(ctx->node_invrho), p,
                                               ptr<double>(ctx->adj_lam));
    note_launch();
    for (size_t L = 0; L + 1 < ctx->level_begin.size(); L++) {
        const int64_t lb = ctx->level_begin[L], le = ctx->level_begin[L + 1];
        if (le <= lb) continue;
        k_l2l<<<dim3((unsigned)(le - lb), 3), 128, 0, sr>>>(ptr<int4>(ctx->node_info), ptr<Geo>(ctx->node_geo), lb,
                                                            le, p, ptr<double>(ctx->adj_lam),
                                                            ptr<double>(ctx->adj_lamacc));
        note_launch();
    }
    if (ctx->precision == TC_FP64) {
        TC_CK(cudaFuncSetAttribute(k_leaf_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm), "leaf attr");
        k_leaf_eval<<<dim3((unsigned)nnodes, kLeafEvalSplit), 128, lsm, sr>>>(
            ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo), ptr<double>(ctx->xs), ptr<double>(ctx->ws), N, p,
            ptr<double>(ctx->adj_lamacc), ptr<double>(ctx->adj_gfar));
    } else {
        const size_t lsm32 = (size_t)12 * C * 4;
        TC_CK(cudaFuncSetAttribute(k_leaf_eval32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm32),
              "leaf attr");
        k_leaf_eval32<<<dim3((unsigned)nnodes, kLeafEvalSplit), 128, lsm32, sr>>>(
            ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo), ptr<double>(ctx->xs), ptr<double>(ctx->ws), N, p,
            ptr<double>(ctx->adj_lamacc), ptr<double>(ctx->adj_gfar));
    }
    note_launch();
    ph_end(ctx, TC_PH_ADJ_REST, sr);
    if (sr != s) TC_CK(cudaEventRecord(ctx->ev_join, sr), "join");

    // near field: target side adds to adj_gt; source side writes adj_gnear
    const unsigned ngrid = (unsigned)((nbatch + kNearAdjWarps - 1) / kNearAdjWarps);
    ph_begin(ctx, TC_PH_ADJ_NEAR_T);
    if (ctx->precision == TC_FP64) {
        k_near_adj_target<double><<<ngrid, kNearAdjWarps * 32, 0, s>>>(
            ts, ptr<double>(ctx->adj_gs), M, ptr<int4>(ctx->node_topo), ptr<double>(ctx->xs), ptr<double>(ctx->ws), N,
            ptr<int64_t>(ctx->near_off), ptr<ListEntry>(ctx->near_list), ptr<double>(ctx->adj_gt));
        note_launch();
        ph_end(ctx, TC_PH_ADJ_NEAR_T);
        ph_begin(ctx, TC_PH_ADJ_NEAR_S);
        k_near_adj_source<double><<<(unsigned)nnodes, kNearAdjWarps * 32, 0, s>>>(
            ts, ptr<double>(ctx->adj_gs), M, ptr<int4>(ctx->node_topo), ptr<double>(ctx->xs), ptr<double>(ctx->ws), N,
            ptr<uint64_t>(ctx->nl_keys), ptr<int32_t>(ctx->nl_idx), ptr<ListEntry>(ctx->near_list),
            ptr<int32_t>(ctx->nl_eb), ctx->near_entries, ptr<double>(ctx->adj_gnear));
        note_launch();
    } else {
        TC_CK((nearpair::run_near_leaf<NearOpG>(ts, ptr<double>(ctx->adj_gs), M, ptr<int4>(ctx->node_topo),
                                                ptr<float4>(ctx->spack), ptr<int64_t>(ctx->near_off),
                                                ptr<ListEntry>(ctx->near_list), ptr<double>(ctx->adj_gt),
                                                ctx->eval_self, 0.0f, sched, s)),
              "near adjoint target side");
        ph_end(ctx, TC_PH_ADJ_NEAR_T);
        ph_begin(ctx, TC_PH_ADJ_NEAR_S);
        TC_CK(cudaMemsetAsync(ctx->adj_gnear.p, 0, (size_t)12 * N * 8, s), "zero near gradients");
        TC_CK(ensure(ctx->adj_scnt, (size_t)nnodes * 4), "alloc adjoint");
        TC_CK(ensure(ctx->adj_soff, (size_t)(nnodes + 1) * 8), "alloc adjoint");
        int64_t* soff = ptr<int64_t>(ctx->adj_soff);
        k_adj_src_count<<<grid_for(nnodes, 256), 256, 0, s>>>(ptr<int4>(ctx->node_topo), sched.node_A, nnodes,
                                                              ptr<int32_t>(ctx->adj_scnt));
        note_launch();
        TC_CK(launch_scan_i32_to_i64(ptr<int32_t>(ctx->adj_scnt), soff, nnodes, soff + nnodes, s), "source units");
        unsigned long long* squeue = reinterpret_cast<unsigned long long*>(ptr<char>(ctx->flags) + 240);
        TC_CK(cudaMemsetAsync(squeue, 0, sizeof(unsigned long long), s), "source queue");
        static int src_blocks = 0;
        if (src_blocks == 0) {
            int per_sm = 0;
            TC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_near_adj_source_units, kAdjSrcWarps * 32, 0),
                  "source grid");
            src_blocks = (per_sm > 0 ? per_sm : 1) * sm_count_adj();
        }
        k_near_adj_source_units<<<(unsigned)src_blocks, kAdjSrcWarps * 32, 0, s>>>(
            ts, ptr<double>(ctx->adj_gs), M, ptr<int4>(ctx->node_topo), ptr<float4>(ctx->spack), N, nnodes, soff,
            sched.node_inc0, sched.node_A, sched.inc_m, ptr<double>(ctx->adj_gnear), squeue);
        note_launch();
    }
    ph_end(ctx, TC_PH_ADJ_NEAR_S);
    TC_CK(cudaGetLastError(), "near adjoint");

    if (sr != s) TC_CK(cudaStreamWaitEvent(s, ctx->ev_join, 0), "join");
    k_adj_final<<<grid_for(N, 256), 256, 0, s>>>(ptr<double>(ctx->adj_gfar), ptr<double>(ctx->adj_gnear),
                                                 ptr<double>(ctx->adj_gt), ptr<int32_t>(ctx->perm), N, ctx->eval_self,
                                                 grad_f, grad_h, grad_nu, grad_x);
    note_launch();
    if (!ctx->eval_self && grad_t) {
        k_scatter3<<<grid_for(M, 256), 256, 0, s>>>(ptr<double>(ctx->adj_gt), tperm, M, grad_t);
        note_launch();
    }
    TC_CK(cudaGetLastError(), "adjoint");
    return TC_OK;
}
