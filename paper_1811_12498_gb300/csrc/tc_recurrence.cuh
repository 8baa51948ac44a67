// Device helpers shared by the far-field kernels (tc_far.cu) and the adjoint
// (tc_adjoint.cu): the Coulomb-coefficient recurrence (3.2) on a unit
// direction (full index set, FP64 or FP32), its scale-free FP32 form on the
// harmonic subset, the level constants, and the FP64 -> FP32 narrowing.
//
// With w = d'/|d'| and b^k(w) = lambda_n c^k, lambda_n = prod_{j<=n} (2j-1)/j,
// recurrence (3.2) becomes
//   c^k = sum_i w_i c^{k-e_i} - kappa_n sum_i c^{k-2e_i},
//   kappa_n = (n-1)^2 / ((2n-1)(2n-3)),  c^0 = 1,
// and b^k(d') = lambda_n |d'|^-(n+1) c^k.
#pragma once

#include "tc_internal.cuh"

namespace tc {

struct LevelConst {
    double kappa[kQMax + 2];  // kappa_n (one level beyond p+2 for the adjoint)
    double ratio[kQMax + 2];  // (2n-1)/n = lambda_n / lambda_{n-1}
};
__host__ __device__ constexpr LevelConst make_level_const()
{
    LevelConst c{};
    for (int n = 0; n <= kQMax + 1; n++) {
        c.kappa[n] = n >= 2 ? (double)((n - 1) * (n - 1)) / (double)((2 * n - 1) * (2 * n - 3)) : 0.0;
        c.ratio[n] = n >= 1 ? (double)(2 * n - 1) / (double)n : 1.0;
    }
    return c;
}

// kappa_n in FP32 for the register kernels
struct LevelConst32 {
    float kappa[kQMax + 2];
};
__host__ __device__ constexpr LevelConst32 make_level_const32()
{
    LevelConst32 c{};
    for (int n = 0; n <= kQMax + 1; n++)
        c.kappa[n] = n >= 2 ? (float)((double)((n - 1) * (n - 1)) / (double)((2 * n - 1) * (2 * n - 3))) : 0.0f;
    return c;
}

// The harmonic subset (k1 <= 1) of level n, 2n+1 coefficients, is stored by
// position h: k = (0, n-h, h) for h <= n, k = (1, n-1-k3, k3) with
// k3 = h-n-1 above.  hcoef_r: c^k of level n at position h of the
// subset from R1 = level n-1 and R2 = level n-2 (scale-free recurrence,
// tc_far.cu); n and h are compile-time constants after unrolling, so every
// branch folds away.
__device__ __forceinline__ float hcoef_r(const float* R1, const float* R2, int n, int h, float v0, float v1, float v2,
                                         float kap)
{
    float s1 = 0.0f, s2 = 0.0f;
    bool any2 = false;
    if (h <= n) {
        const int k3 = h, k2 = n - h;
        if (k2 >= 1) s1 = v1 * R1[k3];
        if (k3 >= 1) s1 = k2 >= 1 ? fmaf(v2, R1[k3 - 1], s1) : v2 * R1[k3 - 1];
        if (k2 >= 2) {
            s2 = R2[k3];
            any2 = true;
        }
        if (k3 >= 2) {
            s2 = any2 ? s2 + R2[k3 - 2] : R2[k3 - 2];
            any2 = true;
        }
    } else {
        const int k3 = h - n - 1, k2 = n - 1 - k3;
        s1 = v0 * R1[k3];
        if (k2 >= 1) s1 = fmaf(v1, R1[n + k3], s1);
        if (k3 >= 1) s1 = fmaf(v2, R1[n + k3 - 1], s1);
        if (k2 >= 2) {
            s2 = R2[n - 1 + k3];
            any2 = true;
        }
        if (k3 >= 2) {
            s2 = any2 ? s2 + R2[n - 3 + k3] : R2[n - 3 + k3];
            any2 = true;
        }
    }
    return any2 ? fmaf(-kap, s2, s1) : s1;
}

// FP64 -> FP32 by bit manipulation: round the magnitude to 23 mantissa bits
// (adding half a unit of the last kept bit, ties away from zero; a carry
// into the exponent is the correct result), re-bias the exponent, keep the
// sign; values below the FP32 normal range give 0.  The inputs here are the
// O(1) coefficients c^k, far from FP32 overflow.
__device__ inline float narrow(double v)
{
    const unsigned long long r = (unsigned long long)__double_as_longlong(v) + 0x10000000ull;
    const unsigned hi = (unsigned)(r >> 32);
    const unsigned lo = (unsigned)r;
    const unsigned e = (hi >> 20) & 0x7ffu;
    const unsigned m = __funnelshift_l(lo, hi, 3);  // top 23 mantissa bits in m & 0x7fffff
    const unsigned bits = (hi & 0x80000000u) | ((e - 896u) << 23) | (m & 0x7fffffu);
    return e > 896u ? __uint_as_float(bits) : 0.0f;
}

template <typename TR, typename TC>
__device__ inline TC to_tc(TR v)
{
    return (TC)v;
}
template <>
__device__ inline float to_tc<double, float>(double v)
{
    return narrow(v);
}

// One coefficient c^k, |k| = n, k = (k1, k2, k3), a = k2 + k3, at position
// pos = a(a+1)/2 + k3 of its level; R1 holds level n-1 and R2 level n-2,
// both laid out [position][lane].
template <typename TR>
__device__ inline TR coef(const TR* R1, const TR* R2, int pos, int a, int k1, int k2, int k3, TR w0, TR w1, TR w2,
                          TR kap, int lane)
{
    TR s1 = 0, s2 = 0;
    if (k1 >= 1) s1 = w0 * R1[pos * 32 + lane];
    if (k2 >= 1) s1 = fma(w1, R1[(pos - a) * 32 + lane], s1);
    if (k3 >= 1) s1 = fma(w2, R1[(pos - a - 1) * 32 + lane], s1);
    if (k1 >= 2) s2 = R2[pos * 32 + lane];
    if (k2 >= 2) s2 += R2[(pos - 2 * a + 1) * 32 + lane];
    if (k3 >= 2) s2 += R2[(pos - 2 * a - 1) * 32 + lane];
    return fma(-kap, s2, s1);
}

}  // namespace tc
