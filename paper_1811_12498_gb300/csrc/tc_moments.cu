// Cluster moments (Section 2) and the per-cluster contraction tables of the
// far field.
//
// Moments, for every cluster C and ||k|| <= p, in FP64:
//   M_j^k   = sum_{n in C} (y^n - y_c)^k f_j^n                 (comp j = 0..2)
//   M~_jl^k = sum_{n in C} (y^n - y_c)^k h_j^n nu_l^n          (comp 3 + 3j + l)
// stored as mom[node][comp][flat(k)] in the graded order of tc_internal.cuh.
//
// Contraction tables.  Substituting eq. (3.4) into sum_k a^k_ij M_j^k and
// eq. (3.7) into sum_k a~^k_ijl M~_jl^k and collecting by the index k' of the
// Coulomb coefficient b^{k'} gives, for ||k'|| <= p + 2,
//   u_i = sum_{k'} b^{k'} ( A_i^{k'} + sum_l d_l B_il^{k'} ),   d = x - y_c,
// with (terms whose moment index is negative or above p vanish)
//   A_i^{k'}  = M_i^{k'} - k'_i sum_j M_j^{k'-e_i+e_j}
//             + 1/3 sum_l k'_l M~_il^{k'-e_l}
//             - 1/3 sum_{j,l} (k'_i - delta_ij) k'_j M~_jl^{k'-e_i-e_j+e_l}
//   B_il^{k'} = k'_i M_l^{k'-e_i} + 1/3 sum_j k'_i (k'_j - delta_ij) M~_jl^{k'-e_i-e_j}.
// This is the same sum as eqs. (4.4) + (4.9) regrouped: every term there is
// b^{k'} times a cluster constant or times one component of d (sigma^k and
// tau_j are linear in d), so the per-target work becomes one pass over b.
//
// Scaling.  b^{k'} is homogeneous of degree -(||k'||+1) in d, so with
// rho = cluster radius, d' = d / rho:
//   u_i = sum_{k'} b^{k'}(d') ( Â_i^{k'} + sum_l d'_l B̂_il^{k'} ),
//   Â = A rho^-(n+1),  B̂ = B rho^-n,  n = ||k'||.
// Under the MAC |d'| >= 1/theta, so every b^{k'}(d') is at most about
// theta^n and the tables stay well inside FP32 range for deep trees.
#include "tc_internal.cuh"

namespace tc {

namespace {

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

__global__ void k_gather_weights(const double* __restrict__ f, const double* __restrict__ h,
                                 const double* __restrict__ nu, const int32_t* __restrict__ perm, int64_t N,
                                 double* __restrict__ ws)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t j = perm[i];
    for (int a = 0; a < 3; a++) {
        ws[a * N + i] = f[a * N + j];
        ws[(3 + a) * N + i] = h[a * N + j];
        ws[(6 + a) * N + i] = nu[a * N + j];
    }
}

// FP32 source record for the mixed near field: position split as hi + lo
// (hi = fl32(x), lo = fl32(x - hi)), then f, h, nu.
__global__ void k_source_pack(const double* __restrict__ xs, const double* __restrict__ ws, int64_t N,
                              float4* __restrict__ pack)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float hi[3], lo[3];
    for (int a = 0; a < 3; a++) {
        double v = xs[a * N + i];
        hi[a] = (float)v;
        lo[a] = (float)(v - (double)hi[a]);
    }
    float w[9];
    for (int c = 0; c < 9; c++) w[c] = (float)ws[c * N + i];
    pack[4 * i + 0] = make_float4(hi[0], hi[1], hi[2], w[0]);
    pack[4 * i + 1] = make_float4(lo[0], lo[1], lo[2], w[1]);
    pack[4 * i + 2] = make_float4(w[2], w[3], w[4], w[5]);
    // the last slot holds h.nu, which only the regularized pair terms read
    const double hn = ws[3 * N + i] * ws[6 * N + i] + ws[4 * N + i] * ws[7 * N + i] + ws[5 * N + i] * ws[8 * N + i];
    pack[4 * i + 3] = make_float4(w[6], w[7], w[8], (float)hn);
}

constexpr int kMomThreads = 128;
constexpr int kMomChunk = 32;
constexpr int kLeafMomThreads = 192;  // threads of a leaf-pass block
constexpr int kLeafMomSlots = (ncoef(kPMax) + kLeafMomThreads - 1) / kLeafMomThreads;

constexpr int kMomItem = 256;       // particles of a leaf per item of the leaf pass

// Leaf pass (P2M, from the definition), balanced: every leaf is cut into
// items of at most kMomItem particles, each writing its partial moments to
// part[item]; k_moments_sum adds a leaf's partials in item order (so the
// result does not depend on scheduling).  One block per leaf left the GPU
// waiting on its largest leaves (N = 262144 in Gaussian clusters: leaves of
// very different sizes).  Particles are staged in chunks: their powers of
// (y - y_c) per axis and their 12 weights; each thread owns S = C / 192
// (rounded up) of the k, so the accumulators take 24 S registers.  The
// blocks walk the items.  Beside the near field (launched while the moments
// are still in flight) the grid is one resident block per SM: the pass is
// bound by the FP64 pipe, which the near field's FP32 work leaves free, and
// at S = 1 (p <= 8) a block takes 192 x 64 registers, which fits in what
// the near field's resident blocks leave.  Otherwise it is one block per
// item, whose blocks come and go, so kernels launched after it on other
// streams start as soon as blocks retire.  Internal clusters are assembled
// from their children by k_m2m.
__global__ void k_mom_items(const int4* __restrict__ topo, int64_t nnodes, int32_t* __restrict__ cnt)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nnodes) return;
    const int4 t = topo[id];
    cnt[id] = t.w == 0 ? (t.y + kMomItem - 1) / kMomItem : 0;
}

template <int S>
__global__ void __launch_bounds__(kLeafMomThreads, S * kLeafMomThreads <= 256 ? 5 : 1)
    k_moments(const int4* __restrict__ topo, const Geo* __restrict__ geo, const double* __restrict__ xs,
              const double* __restrict__ ws, int64_t N, int p, const int32_t* __restrict__ item_off,
              const int32_t* __restrict__ nitems, int64_t nnodes, double* __restrict__ part)
{
    __shared__ double pw[3][kMomChunk][kPMax + 1];
    __shared__ double wt[kMomChunk][12];
    const int C = ncoef(p);
    int kk[S][3];
    for (int s = 0; s < S; s++) {
        const int idx = threadIdx.x + s * kLeafMomThreads;
        if (idx < C)
            unflatten(idx, kk[s][0], kk[s][1], kk[s][2]);
        else
            kk[s][0] = kk[s][1] = kk[s][2] = 0;
    }
    const int items = *nitems;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        int64_t lo = 0, hi = nnodes;  // item_off[lo] <= item < item_off[hi]
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (item_off[mid] <= item)
                lo = mid;
            else
                hi = mid;
        }
        // lo is the last node with item_off <= item; nodes without items
        // (cnt 0) share their successor's offset and come before it, so lo
        // owns the item
        const int64_t node = lo;
        const int4 t0 = topo[node];
        const int first = t0.x + (item - item_off[node]) * kMomItem;
        const int end = first + min(kMomItem, t0.x + t0.y - first);
        const Geo g = geo[node];
        double acc[S][12];
        for (int s = 0; s < S; s++)
            for (int c = 0; c < 12; c++) acc[s][c] = 0.0;
        for (int base = first; base < end; base += kMomChunk) {
            const int nq = min(kMomChunk, end - base);
            __syncthreads();
            if (threadIdx.x < nq) {
                const int i = base + threadIdx.x;
                const double d[3] = {xs[i] - g.x, xs[N + i] - g.y, xs[2 * N + i] - g.z};
                for (int a = 0; a < 3; a++) {
                    double v = 1.0;
                    pw[a][threadIdx.x][0] = 1.0;
                    for (int k = 1; k <= p; k++) {
                        v *= d[a];
                        pw[a][threadIdx.x][k] = v;
                    }
                }
                const double h[3] = {ws[3 * N + i], ws[4 * N + i], ws[5 * N + i]};
                const double nu[3] = {ws[6 * N + i], ws[7 * N + i], ws[8 * N + i]};
                wt[threadIdx.x][0] = ws[i];
                wt[threadIdx.x][1] = ws[N + i];
                wt[threadIdx.x][2] = ws[2 * N + i];
                for (int j = 0; j < 3; j++)
                    for (int l = 0; l < 3; l++) wt[threadIdx.x][3 + 3 * j + l] = h[j] * nu[l];
            }
            __syncthreads();
            for (int s = 0; s < S; s++) {
                if (threadIdx.x + s * kLeafMomThreads >= C) break;
                for (int q = 0; q < nq; q++) {
                    const double mono = pw[0][q][kk[s][0]] * pw[1][q][kk[s][1]] * pw[2][q][kk[s][2]];
                    for (int c = 0; c < 12; c++) acc[s][c] = fma(mono, wt[q][c], acc[s][c]);
                }
            }
        }
        for (int s = 0; s < S; s++) {
            const int idx = threadIdx.x + s * kLeafMomThreads;
            if (idx >= C) break;
            for (int c = 0; c < 12; c++) part[((int64_t)item * 12 + c) * C + idx] = acc[s][c];
        }
    }
}

// mom[leaf] = sum of the leaf's item partials, in item order
__global__ void k_moments_sum(const int4* __restrict__ topo, const int32_t* __restrict__ cnt,
                              const int32_t* __restrict__ item_off, int64_t nnodes, int p,
                              const double* __restrict__ part, double* __restrict__ mom)
{
    const int64_t node = blockIdx.x;
    if (node >= nnodes || topo[node].w != 0) return;
    const int C = ncoef(p);
    const int i0 = item_off[node], ni = cnt[node];
    for (int q = threadIdx.x; q < 12 * C; q += blockDim.x) {
        double v = 0.0;
        for (int k = 0; k < ni; k++) v += part[(int64_t)(i0 + k) * 12 * C + q];
        mom[node * 12 * C + q] = v;
    }
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

// M2M: moments of an internal cluster P from those of its children C by the
// binomial theorem, (y - c_P)^k = sum_{m <= k} binom(k, m) (y - c_C)^m (c_C - c_P)^(k-m):
//   M^k(P) = sum_C sum_{m <= k} binom(k, m) (c_C - c_P)^(k-m) M^m(C),
// the same for all 12 components.  The shift factorises over the axes, so
// each child's moments are shifted along x, then y, then z: three passes of
// at most p+1 terms per coefficient instead of one of prod_a (k_a + 1).  One
// block per (internal cluster of one level, child), the two working arrays
// [C][12] in shared memory, the shifted moments to a scratch slot per child;
// then k_m2m_sum adds each cluster's children in order.  Levels are
// processed from the deepest up.
__global__ void __launch_bounds__(kMomThreads) k_m2m_shift(const int4* __restrict__ topo, const Geo* __restrict__ geo,
                                                           int64_t lb, int64_t le, int64_t cb, int p,
                                                           const double* __restrict__ mom,
                                                           double* __restrict__ shifted)
{
    extern __shared__ double m2m_sh[];
    __shared__ double sp[3][kPMax + 1];
    __shared__ unsigned char kidx[ncoef(kPMax)][3];
    const int64_t node = lb + blockIdx.x;
    if (node >= le) return;
    const int4 t = topo[node];
    const int ci = blockIdx.y;
    if (ci >= t.w) return;
    const Geo gp = geo[node];
    const int C = ncoef(p), W = C * 12;
    for (int k = threadIdx.x; k < C; k += blockDim.x) {
        int k1, k2, k3;
        unflatten(k, k1, k2, k3);
        kidx[k][0] = (unsigned char)k1, kidx[k][1] = (unsigned char)k2, kidx[k][2] = (unsigned char)k3;
    }
    double* A = m2m_sh;
    double* B = A + W;
    const int64_t child = t.z + ci;
    const Geo gc = geo[child];
    const double* mc = mom + child * 12 * C;
    double* out = shifted + (child - cb) * (int64_t)W;
    if (threadIdx.x < 3) {
        const double sh = threadIdx.x == 0 ? gc.x - gp.x : (threadIdx.x == 1 ? gc.y - gp.y : gc.z - gp.z);
        double v = 1.0;
        sp[threadIdx.x][0] = 1.0;
        for (int k = 1; k <= p; k++) {
            v *= sh;
            sp[threadIdx.x][k] = v;
        }
    }
    for (int i = threadIdx.x; i < W; i += blockDim.x) A[i] = mc[(i % 12) * C + i / 12];
    __syncthreads();
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
        const double* src = ax == 1 ? B : A;
        double* dst = ax == 0 ? B : (ax == 1 ? A : out);
        for (int i = threadIdx.x; i < W; i += blockDim.x) {
            const int k = i / 12, c = i % 12;
            int kk[3] = {kidx[k][0], kidx[k][1], kidx[k][2]};
            const int ka = kk[ax];
            double v = 0.0;
            for (int m = 0; m <= ka; m++) {
                kk[ax] = m;
                v = fma(c_binom.v[ka][m] * sp[ax][ka - m], src[flat_index(kk[0], kk[1], kk[2]) * 12 + c], v);
            }
            dst[i] = v;
        }
        __syncthreads();
    }
}

// mom[cluster] = sum of its children's shifted moments, in child order
__global__ void k_m2m_sum(const int4* __restrict__ topo, int64_t lb, int64_t le, int64_t cb, int p,
                          const double* __restrict__ shifted, double* __restrict__ mom)
{
    const int64_t node = lb + blockIdx.x;
    if (node >= le) return;
    const int4 t = topo[node];
    if (t.w == 0) return;
    const int C = ncoef(p), W = C * 12;
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        double acc = 0.0;
        for (int ci = 0; ci < t.w; ci++) acc += shifted[(t.z + ci - cb) * (int64_t)W + i];
        mom[(node * 12 + i % 12) * C + i / 12] = acc;
    }
}

// moment of component c at multi-index (k1,k2,k3); 0 outside 0 <= k, ||k|| <= p
__device__ inline double mget(const double* m, int C, int p, int c, int k1, int k2, int k3)
{
    if (k1 < 0 || k2 < 0 || k3 < 0 || k1 + k2 + k3 > p) return 0.0;
    return m[c * C + flat_index(k1, k2, k3)];
}

// One thread per (cluster, k'), ||k'|| <= p + 2.  Output layout
// [node][flat(k')][12]: A_0..A_2, then B_il at 3 + 3i + l.
// Moments are stored at order pm >= p; only ||k|| <= p enter the tables.
__global__ void k_ab_tables(const double* __restrict__ mom, const double* __restrict__ invrho, int64_t nnodes,
                            int pm, int p, double* __restrict__ ab64, float* __restrict__ ab32)
{
    const int C = ncoef(pm), C2 = ncoef(p + 2);
    int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= nnodes * C2) return;
    int64_t node = gid / C2;
    int kidx = (int)(gid - node * C2);
    int kp[3];
    unflatten(kidx, kp[0], kp[1], kp[2]);
    const int n = kp[0] + kp[1] + kp[2];
    const double* m = mom + node * 12 * C;
    double A[3] = {0, 0, 0}, B[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    const double third = 1.0 / 3.0;
    for (int i = 0; i < 3; i++) {
        int ei[3] = {i == 0, i == 1, i == 2};
        // Stokeslet part
        double a = mget(m, C, p, i, kp[0], kp[1], kp[2]);
        double s = 0.0;
        for (int j = 0; j < 3; j++) {
            int ej[3] = {j == 0, j == 1, j == 2};
            s += mget(m, C, p, j, kp[0] - ei[0] + ej[0], kp[1] - ei[1] + ej[1], kp[2] - ei[2] + ej[2]);
        }
        a -= kp[i] * s;
        // stresslet part
        double t3 = 0.0, t2 = 0.0;
        for (int l = 0; l < 3; l++) {
            int el[3] = {l == 0, l == 1, l == 2};
            t3 += kp[l] * mget(m, C, p, 3 + 3 * i + l, kp[0] - el[0], kp[1] - el[1], kp[2] - el[2]);
        }
        for (int j = 0; j < 3; j++) {
            int ej[3] = {j == 0, j == 1, j == 2};
            double cj = (double)(kp[i] - (i == j)) * kp[j];
            if (cj == 0.0) continue;
            for (int l = 0; l < 3; l++) {
                int el[3] = {l == 0, l == 1, l == 2};
                t2 += cj * mget(m, C, p, 3 + 3 * j + l, kp[0] - ei[0] - ej[0] + el[0], kp[1] - ei[1] - ej[1] + el[1],
                                kp[2] - ei[2] - ej[2] + el[2]);
            }
        }
        A[i] = a + third * (t3 - t2);
        for (int l = 0; l < 3; l++) {
            double bv = kp[i] * mget(m, C, p, l, kp[0] - ei[0], kp[1] - ei[1], kp[2] - ei[2]);
            double tb = 0.0;
            for (int j = 0; j < 3; j++) {
                int ej[3] = {j == 0, j == 1, j == 2};
                double cj = (double)kp[i] * (kp[j] - (i == j));
                if (cj == 0.0) continue;
                tb += cj * mget(m, C, p, 3 + 3 * j + l, kp[0] - ei[0] - ej[0], kp[1] - ei[1] - ej[1],
                                kp[2] - ei[2] - ej[2]);
            }
            B[i][l] = bv + third * tb;
        }
    }
    double ir = invrho[node];
    double sB = 1.0;
    for (int q = 0; q < n; q++) sB *= ir;  // rho^-n
    double sA = sB * ir;                    // rho^-(n+1)
    double out[12];
    for (int i = 0; i < 3; i++) out[i] = A[i] * sA;
    for (int i = 0; i < 3; i++)
        for (int l = 0; l < 3; l++) out[3 + 3 * i + l] = B[i][l] * sB;
    int64_t o = gid * 12;
    if (ab64)
        for (int c = 0; c < 12; c++) ab64[o + c] = out[c];
    if (ab32)
        for (int c = 0; c < 12; c++) ab32[o + c] = (float)out[c];
}

// Regularized kernels.  With G_m = (|x - y|^2 + eps^2)^(-m/2) the
// regularized Stokeslet is delta_ij G_1 + (x_j - y_j) D_{y_i} G_1 + eps^2
// delta_ij G_3 and the regularized stresslet is
// (1/3)[(x_l - y_l) D_{y_i} D_{y_j} G_1 + delta_ij D_{y_l} G_1]
// + (eps^2/6)(delta_ij D_{y_l} G_3 + delta_jl D_{y_i} G_3 + delta_il D_{y_j} G_3):
// the G_1 parts have the structure of eqs. (4.4)/(4.9), so the tables above
// apply with the Coulomb coefficients replaced by those of G_1; the eps^2
// parts contract the Taylor coefficients c^k of G_3 against
//   E_i^k = eps^2 M_i^k + (eps^2/6)[sum_l k_l M~_il^{k-e_l}
//           + k_i sum_j M~_jj^{k-e_i} + sum_j k_j M~_ji^{k-e_j}],  ||k|| <= p + 1,
// stored scaled by rho^-(n+3) (n = ||k||; the coefficients are then taken at
// d' = (x - y_c)/rho and eps' = eps/rho).  One thread per (cluster, k),
// layout [node][flat(k)][3].
__global__ void k_eps_table(const double* __restrict__ mom, const double* __restrict__ invrho, int64_t nnodes,
                            int pm, int p, double eps, double* __restrict__ et)
{
    const int C = ncoef(pm), C1 = ncoef(p + 1);
    const int64_t gid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gid >= nnodes * C1) return;
    const int64_t node = gid / C1;
    int k[3];
    unflatten((int)(gid - node * C1), k[0], k[1], k[2]);
    const int n = k[0] + k[1] + k[2];
    const double* m = mom + node * 12 * C;
    const double e2 = eps * eps;
    double tr = 0.0;  // sum_j M~_jj shifted per i below
    double sc = invrho[node] * invrho[node] * invrho[node];
    for (int q = 0; q < n; q++) sc *= invrho[node];
    for (int i = 0; i < 3; i++) {
        int ei[3] = {i == 0, i == 1, i == 2};
        double v = e2 * mget(m, C, p, i, k[0], k[1], k[2]);
        double t = 0.0;
        for (int l = 0; l < 3; l++) {
            int el[3] = {l == 0, l == 1, l == 2};
            t += k[l] * mget(m, C, p, 3 + 3 * i + l, k[0] - el[0], k[1] - el[1], k[2] - el[2]);
            t += k[l] * mget(m, C, p, 3 + 3 * l + i, k[0] - el[0], k[1] - el[1], k[2] - el[2]);
        }
        tr = 0.0;
        for (int j = 0; j < 3; j++) tr += mget(m, C, p, 3 + 4 * j, k[0] - ei[0], k[1] - ei[1], k[2] - ei[2]);
        t += k[i] * tr;
        et[gid * 3 + i] = (v + e2 / 6.0 * t) * sc;
    }
}

// Harmonic folding of the tables.  The b^k are the Taylor coefficients of
// 1/|d - t| in t, a harmonic function, so (Laplace's equation)
//   sum_i (k_i + 2)(k_i + 1) b^{k + 2 e_i} = 0,
// i.e. within a level every b^k with k1 >= 2 is
//   b^k = -[(k2+2)(k2+1) b^{k-2e1+2e2} + (k3+2)(k3+1) b^{k-2e1+2e3}] / (k1 (k1-1)).
// Substituting this row by row, from k1 = n down to 2, into sum_k b^k T^k
// moves each table entry with k1 >= 2 onto two entries with k1 smaller by 2;
// at the end only k1 in {0, 1} carry weight, and
//   sum_{|k| <= P} b^k T^k = sum_{|k| <= P, k1 <= 1} b^k T'^k
// exactly, for every d.  The far field then needs the (P+1)^2 coefficients
// with k1 <= 1 only (2n+1 per level instead of (n+1)(n+2)/2), and those obey
// recurrence (3.2) among themselves (it never raises k1).  One block per
// cluster; the folding is done in FP64 and then stored in the working type,
// level n multiplied by lambda_n = prod_{j<=n} (2j-1)/j, the factor that the
// far kernels' scale-free recurrence leaves out (tc_far.cu).  In mixed
// precision the block also writes the cluster's FP32 geometry for the far
// kernel: (y_c hi, 1/rho) and (y_c lo, 0), hi = fl32(y_c), lo = fl32(y_c - hi).
__global__ void k_fold_tables(const double* __restrict__ ab64, int64_t nnodes, int p, double* __restrict__ abf64,
                              float* __restrict__ abf32, const Geo* __restrict__ geo,
                              const double* __restrict__ invrho, float4* __restrict__ geo32)
{
    extern __shared__ double lv[];  // one level: [position][12]
    const int64_t node = blockIdx.x;
    const int P = p + 2;
    const int C2 = ncoef(P), H = hsize(P);
    if (geo32 && threadIdx.x == 0) {
        const Geo g = geo[node];
        const float hx = __double2float_rn(g.x), hy = __double2float_rn(g.y), hz = __double2float_rn(g.z);
        geo32[2 * node] = make_float4(hx, hy, hz, __double2float_rn(invrho[node]));
        geo32[2 * node + 1] = make_float4(__double2float_rn(g.x - (double)hx), __double2float_rn(g.y - (double)hy),
                                          __double2float_rn(g.z - (double)hz), 0.0f);
    }
    double lambda = 1.0;  // lambda_n
    for (int n = 0; n <= P; n++) {
        if (n > 0) lambda *= (double)(2 * n - 1) / (double)n;
        const int L = level_size(n);
        const int base = n > 0 ? ncoef(n - 1) : 0;
        for (int q = threadIdx.x; q < L * 12; q += blockDim.x) lv[q] = ab64[((int64_t)node * C2 + base) * 12 + q];
        __syncthreads();
        for (int k1 = n; k1 >= 2; k1--) {
            const int a = n - k1;  // row k1 holds positions a(a+1)/2 + k3, k3 = 0..a
            const double inv = 1.0 / ((double)k1 * (k1 - 1));
            // pushes along e2, then along e3 (each phase writes distinct entries)
            for (int ph = 0; ph < 2; ph++) {
                for (int q = threadIdx.x; q < (a + 1) * 12; q += blockDim.x) {
                    const int k3 = q / 12, c = q % 12, k2 = a - k3;
                    const int src = a * (a + 1) / 2 + k3;
                    const int a2 = a + 2;
                    int dst;
                    double fct;
                    if (ph == 0) {
                        dst = a2 * (a2 + 1) / 2 + k3;  // (k1-2, k2+2, k3)
                        fct = -(double)((k2 + 2) * (k2 + 1)) * inv;
                    } else {
                        dst = a2 * (a2 + 1) / 2 + k3 + 2;  // (k1-2, k2, k3+2)
                        fct = -(double)((k3 + 2) * (k3 + 1)) * inv;
                    }
                    lv[dst * 12 + c] += fct * lv[src * 12 + c];
                }
                __syncthreads();
            }
        }
        // keep k1 = 0 (positions n(n+1)/2 + k3) and k1 = 1 ((n-1)n/2 + k3)
        for (int q = threadIdx.x; q < (2 * n + 1) * 12; q += blockDim.x) {
            const int h = q / 12, c = q % 12;
            const int src = h <= n ? n * (n + 1) / 2 + h : (n - 1) * n / 2 + (h - n - 1);
            const int64_t o = ((int64_t)node * H + n * n + h) * 12 + c;
            const double v = lambda * lv[src * 12 + c];
            if (abf64) abf64[o] = v;
            if (abf32) abf32[o] = (float)v;
        }
        __syncthreads();
    }
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_gather_weights(const double* f, const double* h, const double* nu, const int32_t* perm,
                                  int64_t N, double* ws, cudaStream_t s)
{
    k_gather_weights<<<grid_for(N, 256), 256, 0, s>>>(f, h, nu, perm, N, ws);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_source_pack(const double* xs, const double* ws, int64_t N, float4* pack, cudaStream_t s)
{
    k_source_pack<<<grid_for(N, 256), 256, 0, s>>>(xs, ws, N, pack);
    note_launch();
    return cudaGetLastError();
}

int64_t moments_item_bound(int64_t N, int64_t nnodes) { return nnodes + (N + kMomItem - 1) / kMomItem; }

size_t moments_scratch_bytes(int64_t N, int64_t nnodes, int p)
{
    return (size_t)(2 * nnodes + 1) * 4 + 16 + (size_t)moments_item_bound(N, nnodes) * 12 * ncoef(p) * 8;
}

// One block per item, or a resident grid of blocks_per_sm blocks per SM
static unsigned moments_grid(int blocks_per_sm, int64_t bound)
{
    if (blocks_per_sm <= 0) return (unsigned)bound;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (int64_t)blocks_per_sm * (sms > 0 ? sms : 1);
    return (unsigned)(bound < want ? bound : want);
}

cudaError_t launch_moments(const int4* topo, const Geo* geo, const double* xs, const double* ws, int64_t N,
                           int64_t nnodes, int p, double* mom, void* scratch, int blocks_per_sm, cudaStream_t s)
{
    // scratch: cnt [nnodes] i32, item_off [nnodes] i32, nitems i32, then (16-byte aligned) the partials
    int32_t* cnt = reinterpret_cast<int32_t*>(scratch);
    int32_t* item_off = cnt + nnodes;
    int32_t* nitems = item_off + nnodes;
    const size_t head = ((size_t)(2 * nnodes + 1) * 4 + 15) & ~(size_t)15;
    double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) + head);
    k_mom_items<<<(unsigned)((nnodes + 255) / 256), 256, 0, s>>>(topo, nnodes, cnt);
    note_launch();
    cudaError_t e = launch_scan_i32(cnt, item_off, nnodes, nitems, s);
    if (e != cudaSuccess) return e;
    // the item count stays on the device: the grid walks the items up to it
    const unsigned grid = moments_grid(blocks_per_sm, moments_item_bound(N, nnodes));
    const int S = (ncoef(p) + kLeafMomThreads - 1) / kLeafMomThreads;
    if (S == 1)
        k_moments<1><<<grid, kLeafMomThreads, 0, s>>>(topo, geo, xs, ws, N, p, item_off, nitems, nnodes, part);
    else if (S == 2)
        k_moments<2><<<grid, kLeafMomThreads, 0, s>>>(topo, geo, xs, ws, N, p, item_off, nitems, nnodes, part);
    else
        k_moments<kLeafMomSlots><<<grid, kLeafMomThreads, 0, s>>>(topo, geo, xs, ws, N, p, item_off, nitems, nnodes,
                                                                   part);
    note_launch();
    k_moments_sum<<<(unsigned)nnodes, 128, 0, s>>>(topo, cnt, item_off, nnodes, p, part, mom);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_m2m(const int4* topo, const Geo* geo, int64_t lb, int64_t le, int64_t cb, int p, double* mom,
                       double* shifted, cudaStream_t s)
{
    if (le <= lb) return cudaSuccess;
    const size_t smem = (size_t)2 * ncoef(p) * 12 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_m2m_shift, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_m2m_shift<<<dim3((unsigned)(le - lb), 8), kMomThreads, smem, s>>>(topo, geo, lb, le, cb, p, mom, shifted);
    note_launch();
    k_m2m_sum<<<(unsigned)(le - lb), 256, 0, s>>>(topo, lb, le, cb, p, shifted, mom);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_fold_tables(const double* ab64, int64_t nnodes, int p, double* abf64, float* abf32,
                               const Geo* geo, const double* invrho, float4* geo32, cudaStream_t s)
{
    const size_t smem = (size_t)level_size(p + 2) * 12 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_fold_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fold_tables<<<(unsigned)nnodes, 128, smem, s>>>(ab64, nnodes, p, abf64, abf32, geo, invrho, geo32);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_eps_table(const double* mom, const double* invrho, int64_t nnodes, int pm, int p, double eps,
                             double* et, cudaStream_t s)
{
    const int64_t total = nnodes * ncoef(p + 1);
    k_eps_table<<<grid_for(total, 128), 128, 0, s>>>(mom, invrho, nnodes, pm, p, eps, et);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_ab_tables(const double* mom, const double* invrho, int64_t nnodes, int pm, int p, double* ab64,
                             float* ab32, cudaStream_t s)
{
    int64_t total = nnodes * ncoef(p + 2);
    k_ab_tables<<<grid_for(total, 128), 128, 0, s>>>(mom, invrho, nnodes, pm, p, ab64, ab32);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc
