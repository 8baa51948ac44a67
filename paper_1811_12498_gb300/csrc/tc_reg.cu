// Far field of the regularized Stokeslet and stresslet (the blob of Cortez,
// Fauci and Medovikov; the paper lists regularized kernels as future work).
//
// With G_nu = (|x - y|^2 + eps^2)^(-nu), the regularized kernels are the
// structure of eqs. (4.4)/(4.9) built on G_1/2 plus eps^2 terms in G_3/2
// (tc_moments.cu, k_eps_table), so per (target, cluster):
//   u_i = sum_{||k|| <= p+2} c_{1/2}^k (Â_i^k + d'_l B̂_il^k)
//       + sum_{||k|| <= p+1} c_{3/2}^k Ê_i^k,
// d' = (x - y_c)/rho, with the contraction tables of the paper's kernels
// (k_ab_tables) and the eps^2 table Ê.  The Taylor coefficients c_nu^k of
// G_nu at (d', eps' = eps/rho) follow the recurrence that generalizes (3.2):
// from s D_y G_nu = 2 nu (x - y) G_nu (s = |x - y|^2 + eps^2),
//   n s' c^k = (2n + 2nu - 2) sum_i d'_i c^{k-e_i} - (n + 2nu - 2) sum_i c^{k-2e_i},
//   c^0 = s'^-nu,  s' = |d'|^2 + eps'^2,  n = ||k||.
// G_1/2 is not harmonic when eps > 0, so the harmonic folding of the
// paper's kernels does not apply: the full index set is formed.  One batch of
// 32 targets per warp; the coefficients of two levels live in a per-warp
// shared-memory store [slot][position][lane] (level n overwrites level n-2 in
// place, positions running downward).  FP64 mode (and mixed precision with
// tc_config.rec64 at p >= 8) runs it in FP64 on the FP64 tables; mixed
// precision runs the same recurrence and contraction in FP32 on the FP32
// tables (the full tables and an FP32 copy of the eps^2 table), d' from FP32
// hi/lo splits of the target and the centre, the per-entry velocities summed
// by compensated FP32 summation and widened to FP64 once per target, as in
// the mixed far field of the paper's kernels.
#include "tc_recurrence.cuh"

namespace tc {

namespace {

// one coefficient pass: the recurrence for G_nu (two_nu = 2 nu) up to order
// P, each coefficient contracted against W table values at once
template <int W>
__device__ inline void reg_pass(double* slot0, double* slot1, int P, double two_nu, double sp, double d0, double d1,
                                double d2, const double* __restrict__ tab, double* tot, int lane)
{
    double c0 = rsqrt(sp);
    if (two_nu > 1.5) c0 = c0 * c0 * c0;  // nu = 3/2
    slot0[lane] = c0;
#pragma unroll
    for (int q = 0; q < W; q++) tot[q] = fma(c0, tab[q], tot[q]);
    const double isp = 1.0 / sp;
    for (int n = 1; n <= P; n++) {
        double* Rn = (n & 1) ? slot1 : slot0;  // also holds level n-2
        const double* R1 = (n & 1) ? slot0 : slot1;
        const double al = (2.0 * n + two_nu - 2.0) * isp / n, be = (n + two_nu - 2.0) * isp / n;
        const double w0 = al * d0, w1 = al * d1, w2 = al * d2;
        const double* tl = tab + (int64_t)ncoef(n - 1) * W;
        __syncwarp();
        for (int a = n; a >= 0; a--) {
            const int k1 = n - a, base = a * (a + 1) / 2;
            for (int k3 = a; k3 >= 0; k3--) {
                const int pos = base + k3;
                const double ck = coef<double>(R1, Rn, pos, a, k1, a - k3, k3, w0, w1, w2, be, lane);
                Rn[pos * 32 + lane] = ck;
                const double* t = tl + pos * W;
#pragma unroll
                for (int q = 0; q < W; q++) tot[q] = fma(ck, t[q], tot[q]);
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32)
    k_far_reg(const double* __restrict__ ts, int64_t M, const Geo* __restrict__ geo, const double* __restrict__ invrho,
              const double* __restrict__ ab64, const double* __restrict__ et, int p, double eps,
              const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list, double* __restrict__ u_far)
{
    extern __shared__ double store[];
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    if (b >= nbatch) return;
    const int L = (p + 3) * (p + 4) / 2;  // largest level, order p + 2
    double* slot0 = store;
    double* slot1 = store + (size_t)L * 32;
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    double x0 = 0, x1 = 0, x2 = 0;
    if (valid) {
        x0 = ts[m];
        x1 = ts[M + m];
        x2 = ts[2 * M + m];
    }
    const int C2 = ncoef(p + 2), C1 = ncoef(p + 1);
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int64_t e = far_off[b]; e < far_off[b + 1]; e++) {
        const ListEntry le = far_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const Geo g = geo[le.node];
        const double ir = invrho[le.node];
        double d0 = (x0 - g.x) * ir, d1 = (x1 - g.y) * ir, d2 = (x2 - g.z) * ir;
        if (!in) d0 = 2.0, d1 = 0.0, d2 = 0.0;  // keep idle lanes finite
        const double ep = eps * ir;
        const double sp = d0 * d0 + d1 * d1 + d2 * d2 + ep * ep;
        double t12[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, t3[3] = {0, 0, 0};
        reg_pass<12>(slot0, slot1, p + 2, 1.0, sp, d0, d1, d2, ab64 + (int64_t)le.node * C2 * 12, t12, lane);
        reg_pass<3>(slot0, slot1, p + 1, 3.0, sp, d0, d1, d2, et + (int64_t)le.node * C1 * 3, t3, lane);
        if (in) {
            ux += t12[0] + d0 * t12[3] + d1 * t12[4] + d2 * t12[5] + t3[0];
            uy += t12[1] + d0 * t12[6] + d1 * t12[7] + d2 * t12[8] + t3[1];
            uz += t12[2] + d0 * t12[9] + d1 * t12[10] + d2 * t12[11] + t3[2];
        }
    }
    if (valid) {
        u_far[m] = ux;
        u_far[M + m] = uy;
        u_far[2 * M + m] = uz;
    }
}

// FP32 form of reg_pass
template <int W>
__device__ inline void reg_pass32(float* slot0, float* slot1, int P, float two_nu, float sp, float d0, float d1,
                                  float d2, const float* __restrict__ tab, float* tot, int lane)
{
    float c0 = rsqrtf(sp);
    if (two_nu > 1.5f) c0 = c0 * c0 * c0;  // nu = 3/2
    slot0[lane] = c0;
#pragma unroll
    for (int q = 0; q < W; q++) tot[q] = fmaf(c0, __ldg(tab + q), tot[q]);
    const float isp = 1.0f / sp;
    for (int n = 1; n <= P; n++) {
        float* Rn = (n & 1) ? slot1 : slot0;  // also holds level n-2
        const float* R1 = (n & 1) ? slot0 : slot1;
        const float al = (2.0f * n + two_nu - 2.0f) * isp / (float)n, be = ((float)n + two_nu - 2.0f) * isp / (float)n;
        const float w0 = al * d0, w1 = al * d1, w2 = al * d2;
        const float* tl = tab + (int64_t)ncoef(n - 1) * W;
        __syncwarp();
        for (int a = n; a >= 0; a--) {
            const int k1 = n - a, base = a * (a + 1) / 2;
            for (int k3 = a; k3 >= 0; k3--) {
                const int pos = base + k3;
                const float ck = coef<float>(R1, Rn, pos, a, k1, a - k3, k3, w0, w1, w2, be, lane);
                Rn[pos * 32 + lane] = ck;
                const float* t = tl + pos * W;
#pragma unroll
                for (int q = 0; q < W; q++) tot[q] = fmaf(ck, __ldg(t + q), tot[q]);
            }
        }
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32)
    k_far_reg32(const double* __restrict__ ts, int64_t M, const float4* __restrict__ geo32,
                const float* __restrict__ ab32, const float* __restrict__ et32, int p, float eps,
                const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list, double* __restrict__ u_far)
{
    extern __shared__ float store32[];
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    if (b >= nbatch) return;
    const int L = (p + 3) * (p + 4) / 2;  // largest level, order p + 2
    float* slot0 = store32;
    float* slot1 = store32 + (size_t)L * 32;
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    float xh[3] = {0, 0, 0}, xl[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            const double v = ts[a * M + m];
            xh[a] = __double2float_rn(v);
            xl[a] = __double2float_rn(v - (double)xh[a]);
        }
    const int C2 = ncoef(p + 2), C1 = ncoef(p + 1);
    float su[3] = {0.f, 0.f, 0.f}, ku[3] = {0.f, 0.f, 0.f};
    for (int64_t e = far_off[b]; e < far_off[b + 1]; e++) {
        const ListEntry le = far_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const float4 gh = __ldg(geo32 + 2 * (int64_t)le.node), gl = __ldg(geo32 + 2 * (int64_t)le.node + 1);
        float d0 = ((xh[0] - gh.x) + (xl[0] - gl.x)) * gh.w;
        float d1 = ((xh[1] - gh.y) + (xl[1] - gl.y)) * gh.w;
        float d2 = ((xh[2] - gh.z) + (xl[2] - gl.z)) * gh.w;
        if (!in) d0 = 2.0f, d1 = 0.0f, d2 = 0.0f;  // keep idle lanes finite
        const float ep = eps * gh.w;
        const float sp = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, ep * ep)));
        float t12[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, t3[3] = {0, 0, 0};
        reg_pass32<12>(slot0, slot1, p + 2, 1.0f, sp, d0, d1, d2, ab32 + (int64_t)le.node * C2 * 12, t12, lane);
        reg_pass32<3>(slot0, slot1, p + 1, 3.0f, sp, d0, d1, d2, et32 + (int64_t)le.node * C1 * 3, t3, lane);
        if (in) {
            kahan_add(su[0], ku[0], t12[0] + d0 * t12[3] + d1 * t12[4] + d2 * t12[5] + t3[0]);
            kahan_add(su[1], ku[1], t12[1] + d0 * t12[6] + d1 * t12[7] + d2 * t12[8] + t3[1]);
            kahan_add(su[2], ku[2], t12[2] + d0 * t12[9] + d1 * t12[10] + d2 * t12[11] + t3[2]);
        }
    }
    if (valid) {
        u_far[m] = (double)su[0] - (double)ku[0];
        u_far[M + m] = (double)su[1] - (double)ku[1];
        u_far[2 * M + m] = (double)su[2] - (double)ku[2];
    }
}

// FP32, compile-time order P (p + 2 <= 10; above, the shared-memory store
// of k_far_reg32): both live levels of the coefficients in registers (the
// recurrence fully unrolled, level n overwriting level n-2 in place,
// positions running downward), the tables read as float4 when W = 12.
// NU2 = 2 nu.

template <int P, int W, int NU2>
__device__ __forceinline__ void reg_pass_r(float sp, float d0, float d1, float d2, const float* __restrict__ tab,
                                           float (&tot)[W])
{
    constexpr int L = (P + 1) * (P + 2) / 2;  // level P, the largest
    float cs[2][L];
    float c0 = rsqrtf(sp);
    if (NU2 == 3) c0 = c0 * c0 * c0;
    cs[0][0] = c0;
    if (W == 12) {
        const float4* t4 = reinterpret_cast<const float4*>(tab);
        const float4 a = __ldg(t4), b = __ldg(t4 + 1), c = __ldg(t4 + 2);
        const float t[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < W; q++) tot[q] = fmaf(c0, t[q % 12], tot[q]);
    } else {
#pragma unroll
        for (int q = 0; q < W; q++) tot[q] = fmaf(c0, __ldg(tab + q), tot[q]);
    }
    const float isp = 1.0f / sp;
#pragma unroll
    for (int n = 1; n <= P; n++) {
        const float al = ((float)(2 * n + NU2 - 2) / (float)n) * isp, be = ((float)(n + NU2 - 2) / (float)n) * isp;
        const float w0 = al * d0, w1 = al * d1, w2 = al * d2;
        float* Rn = cs[n & 1];  // also holds level n-2
        const float* R1 = cs[(n - 1) & 1];
#pragma unroll
        for (int a = n; a >= 0; a--) {
            const int k1 = n - a, base = a * (a + 1) / 2;
#pragma unroll
            for (int k3 = a; k3 >= 0; k3--) {
                const int k2 = a - k3, pos = base + k3;
                float s1 = 0.f, s2 = 0.f;
                if (k1 >= 1) s1 = w0 * R1[pos];
                if (k2 >= 1) s1 = fmaf(w1, R1[pos - a], s1);
                if (k3 >= 1) s1 = fmaf(w2, R1[pos - a - 1], s1);
                if (k1 >= 2) s2 = Rn[pos];
                if (k2 >= 2) s2 += Rn[pos - 2 * a + 1];
                if (k3 >= 2) s2 += Rn[pos - 2 * a - 1];
                const float ck = fmaf(-be, s2, s1);
                Rn[pos] = ck;
                const float* t = tab + (int64_t)(ncoef(n - 1) + pos) * W;
                if (W == 12) {
                    const float4* t4 = reinterpret_cast<const float4*>(t);
                    const float4 x = __ldg(t4), y = __ldg(t4 + 1), z = __ldg(t4 + 2);
                    const float tv[12] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, z.x, z.y, z.z, z.w};
#pragma unroll
                    for (int q = 0; q < W; q++) tot[q] = fmaf(ck, tv[q % 12], tot[q]);
                } else {
#pragma unroll
                    for (int q = 0; q < W; q++) tot[q] = fmaf(ck, __ldg(t + q), tot[q]);
                }
                // keep the table loads of later coefficients from being
                // hoisted here: that would exhaust the registers
                asm volatile("" ::: "memory");
            }
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32)
    k_far_reg32r(const double* __restrict__ ts, int64_t M, const float4* __restrict__ geo32,
                 const float* __restrict__ ab32, const float* __restrict__ et32, float eps,
                 const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list,
                 double* __restrict__ u_far)
{
    const int lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    if (b >= nbatch) return;
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    float xh[3] = {0, 0, 0}, xl[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            const double v = ts[a * M + m];
            xh[a] = __double2float_rn(v);
            xl[a] = __double2float_rn(v - (double)xh[a]);
        }
    constexpr int C2 = (P + 1) * (P + 2) * (P + 3) / 6, C1 = P * (P + 1) * (P + 2) / 6;
    float su[3] = {0.f, 0.f, 0.f}, ku[3] = {0.f, 0.f, 0.f};
    for (int64_t e = far_off[b]; e < far_off[b + 1]; e++) {
        const ListEntry le = far_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const float4 gh = __ldg(geo32 + 2 * (int64_t)le.node), gl = __ldg(geo32 + 2 * (int64_t)le.node + 1);
        float d0 = ((xh[0] - gh.x) + (xl[0] - gl.x)) * gh.w;
        float d1 = ((xh[1] - gh.y) + (xl[1] - gl.y)) * gh.w;
        float d2 = ((xh[2] - gh.z) + (xl[2] - gl.z)) * gh.w;
        if (!in) d0 = 2.0f, d1 = 0.0f, d2 = 0.0f;  // keep idle lanes finite
        const float ep = eps * gh.w;
        const float sp = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, ep * ep)));
        float t12[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, t3[3] = {0, 0, 0};
        reg_pass_r<P, 12, 1>(sp, d0, d1, d2, ab32 + (int64_t)le.node * C2 * 12, t12);
        reg_pass_r<P - 1, 3, 3>(sp, d0, d1, d2, et32 + (int64_t)le.node * C1 * 3, t3);
        if (in) {
            kahan_add(su[0], ku[0], t12[0] + d0 * t12[3] + d1 * t12[4] + d2 * t12[5] + t3[0]);
            kahan_add(su[1], ku[1], t12[1] + d0 * t12[6] + d1 * t12[7] + d2 * t12[8] + t3[1]);
            kahan_add(su[2], ku[2], t12[2] + d0 * t12[9] + d1 * t12[10] + d2 * t12[11] + t3[2]);
        }
    }
    if (valid) {
        u_far[m] = (double)su[0] - (double)ku[0];
        u_far[M + m] = (double)su[1] - (double)ku[1];
        u_far[2 * M + m] = (double)su[2] - (double)ku[2];
    }
}

// FP32 copy of an FP64 table, rounded as the contraction tables are (narrow)
__global__ void k_narrow_table(const double* __restrict__ src, int64_t n, float* __restrict__ dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = narrow(src[i]);
}

}  // namespace

cudaError_t launch_far_reg(const double* ts, int64_t M, const Geo* geo, const double* invrho, const double* ab64,
                           const double* et, int p, double eps, const int64_t* far_off, const ListEntry* far_list,
                           double* u_far, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const size_t smem = (size_t)2 * ((p + 3) * (p + 4) / 2) * 32 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_far_reg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_far_reg<<<(unsigned)nbatch, 32, smem, s>>>(ts, M, geo, invrho, ab64, et, p, eps, far_off, far_list, u_far);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_far_reg32(const double* ts, int64_t M, const float4* geo32, const float* ab32, const float* et32,
                             int p, double eps, const int64_t* far_off, const ListEntry* far_list, double* u_far,
                             cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    switch (p + 2) {
#define TC_REG32R_CASE(P)                                                                                          \
    case P:                                                                                                        \
        k_far_reg32r<P><<<(unsigned)nbatch, 32, 0, s>>>(ts, M, geo32, ab32, et32, (float)eps, far_off, far_list, \
                                                        u_far);                                                   \
        note_launch();                                                                                             \
        return cudaGetLastError();
        TC_REG32R_CASE(2) TC_REG32R_CASE(3) TC_REG32R_CASE(4) TC_REG32R_CASE(5) TC_REG32R_CASE(6)
        TC_REG32R_CASE(7) TC_REG32R_CASE(8) TC_REG32R_CASE(9) TC_REG32R_CASE(10)
#undef TC_REG32R_CASE
    default: break;  // higher orders: the shared-memory store
    }
    const size_t smem = (size_t)2 * ((p + 3) * (p + 4) / 2) * 32 * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_far_reg32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_far_reg32<<<(unsigned)nbatch, 32, smem, s>>>(ts, M, geo32, ab32, et32, p, (float)eps, far_off, far_list,
                                                   u_far);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_narrow_table(const double* src, int64_t n, float* dst, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_narrow_table<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, n, dst);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc
