// Far field: particle-cluster Taylor approximation, eq. (2.9), evaluated in
// the contracted form of the contraction tables (tc_moments.cu):
//   u_i += sum_{||k'|| <= p+2} b^{k'}(d') ( Â_i^{k'} + sum_l d'_l B̂_il^{k'} ),
// with d' = (x - y_c) / rho and the Coulomb coefficients b^k of the
// recurrence (3.2):
//   n R^2 b^k = (2n-1) sum_i d_i b^{k-e_i} - (n-1) sum_i b^{k-2e_i},  n = ||k||.
//
// Scale-free form.  With lambda_n = prod_{j<=n} (2j-1)/j and b^k = lambda_n
// c^k / R', the recurrence becomes
//   c^k = sum_i v_i c^{k-e_i} - (kappa_n / R'^2) sum_i c^{k-2e_i},
//   v = d' / R'^2,  kappa_n = (n-1)^2 / ((2n-1)(2n-3)),  c^0 = 1,
// (divide (3.2) by n lambda_n R'^2 and use n lambda_n = (2n-1) lambda_{n-1}).
// The factors lambda_n are folded into the tables once per cluster
// (k_fold_tables), and 1/R' multiplies the finished sum, so the inner loop
// has no per-level scaling at all; |c^k| <= R'^-n with R' >= 1/theta, so
// nothing grows.  Because the tables are also folded onto the harmonic subset
// k1 <= 1 (Laplace's equation expresses every b^k with k1 >= 2 through
// coefficients of smaller k1 on the same level), only the (P+1)^2
// coefficients with k1 <= 1 are formed, 2n+1 per level, at most five
// operations each, and the recurrence never needs any other.
//
// A batch is 32 targets (one per lane) with one far list; a lane outside an
// entry's mask idles for that entry.  Each coefficient is contracted against
// the cluster's 12 folded table entries as soon as it exists (12 FMA into the
// per-lane totals).
//
// Two implementations:
//  * FP32 (mixed precision), order known at compile time (P = p + 2 is a
//    template parameter, one instantiation per order 0..12): every loop is
//    unrolled, the two live levels of coefficients are registers, the tables
//    are read as float4.  One warp takes two consecutive batches (two targets
//    per lane) and walks the merge of their far lists, so every table value
//    the warp loads serves both targets of a lane wherever the lists share a
//    cluster: the broadcast table loads, not the arithmetic, bound this
//    kernel (4 B of L1 bandwidth per FMA at one target per lane).  The grid
//    is resident (one single-warp block per free slot) and its warps take
//    batch pairs from a work queue, so a warp whose pairs have short lists
//    takes more instead of idling while the last blocks run.  The
//    contraction runs on packed FP32x2 FMAs over pairs of table columns and
//    the two targets' recurrences on packed FP32x2 arithmetic side by side,
//    which shrinks the fully unrolled body (its size, not only its
//    arithmetic, limits the kernel: instruction fetch stalls).  d' is
//    formed from FP32 hi/lo splits of the target and the cluster centre
//    (x_hi - y_hi is computed with one rounding, so d' carries FP32 relative
//    accuracy however close x and y_c are in absolute terms), with no FP64
//    operation per entry: the per-entry velocities are summed by compensated
//    (Kahan) FP32 summation, widened to FP64 once per target (an FP64
//    accumulation stalled every entry's end on the slow FP64 pipe).  On the
//    folded tables an FP32 recurrence is as accurate as an FP64 one (at
//    p = 6, 8, 10 on a uniform cube the mixed result differs from FP64 by the
//    same 1.8e-7, set by the FP32 near field).
//  * FP64, any order at run time, one batch per warp: the coefficients live
//    in a per-warp shared memory store of two slots laid out
//    [slot][position][lane] (no bank conflicts); level n overwrites level n-2
//    in place, positions running downward, which is safe because a
//    coefficient reads level n-2 only at positions <= its own.  Two
//    coefficients per step for instruction-level parallelism.
#include "tc_recurrence.cuh"

namespace tc {

namespace {

__constant__ LevelConst c_lev = make_level_const();

__constant__ LevelConst32 c_lev32 = make_level_const32();

// ---------------------------------------------------------------------------
// FP64, run-time order

// One coefficient c^k of the harmonic subset (k1 <= 1) at level n, subset
// position h (0..2n): k1 = 0 for h <= n (k3 = h), else k1 = 1 (k3 = h-n-1).
// R1 holds level n-1 and R2 level n-2 of the subset, [position][lane].
__device__ inline double hcoef(const double* R1, const double* R2, int n, int h, double v0, double v1, double v2,
                               double kap, int lane)
{
    double s1, s2 = 0;
    if (h <= n) {  // k = (0, n - h, h)
        const int k3 = h, k2 = n - h;
        s1 = 0;
        if (k2 >= 1) s1 = v1 * R1[k3 * 32 + lane];
        if (k3 >= 1) s1 = fma(v2, R1[(k3 - 1) * 32 + lane], s1);
        if (k2 >= 2) s2 = R2[k3 * 32 + lane];
        if (k3 >= 2) s2 += R2[(k3 - 2) * 32 + lane];
    } else {  // k = (1, n - 1 - k3, k3)
        const int k3 = h - n - 1, k2 = n - 1 - k3;
        s1 = v0 * R1[k3 * 32 + lane];
        if (k2 >= 1) s1 = fma(v1, R1[(n + k3) * 32 + lane], s1);
        if (k3 >= 1) s1 = fma(v2, R1[(n + k3 - 1) * 32 + lane], s1);
        if (k2 >= 2) s2 = R2[(n - 1 + k3) * 32 + lane];
        if (k3 >= 2) s2 += R2[(n - 3 + k3) * 32 + lane];
    }
    return fma(-kap, s2, s1);
}

__device__ inline void contract12(double c, const double* __restrict__ t, double* tot)
{
    const double2* t2 = reinterpret_cast<const double2*>(t);
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const double2 a = t2[q];
        tot[2 * q] = fma(c, a.x, tot[2 * q]);
        tot[2 * q + 1] = fma(c, a.y, tot[2 * q + 1]);
    }
}

// FP64 coefficient against FP32 tables: the coefficient is narrowed with
// integer operations (tc_recurrence.cuh), the 12 products are FP32
__device__ inline void contract12(double c, const float* __restrict__ t, float* tot)
{
    const float cf = narrow(c);
    const float4* t4 = reinterpret_cast<const float4*>(t);
#pragma unroll
    for (int q = 0; q < 3; q++) {
        const float4 a = t4[q];
        tot[4 * q] = fmaf(cf, a.x, tot[4 * q]);
        tot[4 * q + 1] = fmaf(cf, a.y, tot[4 * q + 1]);
        tot[4 * q + 2] = fmaf(cf, a.z, tot[4 * q + 2]);
        tot[4 * q + 3] = fmaf(cf, a.w, tot[4 * q + 3]);
    }
}

// TC = double: the FP64 mode.  TC = float: mixed precision with the FP64
// recurrence (tc_config.rec64), the FP32 folded tables and FP32 contraction.
template <typename TC>
__device__ inline void far_batch64(const double* __restrict__ ts, int64_t M, const Geo* __restrict__ geo,
                                   const double* __restrict__ invrho, const TC* __restrict__ ab, int p,
                                   const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list,
                                   double* __restrict__ u_far, int64_t b, double* slot_p, double* slot_q, int lane)
{
    const int P = p + 2;
    const int H = hsize(P);
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    double x0 = 0, x1 = 0, x2 = 0;
    if (valid) {
        x0 = ts[m];
        x1 = ts[M + m];
        x2 = ts[2 * M + m];
    }
    double ux = 0.0, uy = 0.0, uz = 0.0;
    const int64_t e0 = far_off[b], e1 = far_off[b + 1];
    for (int64_t e = e0; e < e1; e++) {
        const ListEntry le = far_list[e];
        const bool in = (le.mask >> lane) & 1u;
        const Geo g = geo[le.node];
        const double ir = invrho[le.node];
        const double d0 = (x0 - g.x) * ir, d1 = (x1 - g.y) * ir, d2 = (x2 - g.z) * ir;
        double R2 = d0 * d0 + d1 * d1 + d2 * d2;
        if (!in) R2 = 1.0;  // keep idle lanes finite
        const double iR = rsqrt(R2);
        const double iR2 = iR * iR;
        const double v0 = d0 * iR2, v1 = d1 * iR2, v2 = d2 * iR2;
        const TC* __restrict__ tab = ab + (int64_t)le.node * H * 12;
        TC tot[12];
#pragma unroll
        for (int q = 0; q < 12; q++) tot[q] = tab[q];  // level 0: c^0 = 1
        ((P & 1) ? slot_q : slot_p)[lane] = 1.0;      // level 0 has parity 0
        __syncwarp();
        for (int n = 1; n <= P; n++) {
            const double kap = c_lev.kappa[n] * iR2;
            double* Rn = ((n ^ P) & 1) ? slot_q : slot_p;  // also holds level n-2
            const double* R1 = ((n ^ P) & 1) ? slot_p : slot_q;
            const TC* tl = tab + (int64_t)n * n * 12;
            int h = 2 * n;
            for (; h >= 1; h -= 2) {
                const double ca = hcoef(R1, Rn, n, h, v0, v1, v2, kap, lane);
                const double cb = hcoef(R1, Rn, n, h - 1, v0, v1, v2, kap, lane);
                Rn[h * 32 + lane] = ca;
                Rn[(h - 1) * 32 + lane] = cb;
                contract12(ca, tl + h * 12, tot);
                contract12(cb, tl + (h - 1) * 12, tot);
            }
            if (h == 0) {
                const double ca = hcoef(R1, Rn, n, 0, v0, v1, v2, kap, lane);
                Rn[lane] = ca;
                contract12(ca, tl, tot);
            }
            __syncwarp();
        }
        if (in) {
            double T[12];
#pragma unroll
            for (int q = 0; q < 12; q++) T[q] = (double)tot[q];
            ux += (T[0] + d0 * T[3] + d1 * T[4] + d2 * T[5]) * iR;
            uy += (T[1] + d0 * T[6] + d1 * T[7] + d2 * T[8]) * iR;
            uz += (T[2] + d0 * T[9] + d1 * T[10] + d2 * T[11]) * iR;
        }
    }
    if (valid) {
        u_far[m] = ux;
        u_far[M + m] = uy;
        u_far[2 * M + m] = uz;
    }
}

// per-warp coefficient store of the FP64 kernel: 2P+1 and 2P-1 entries
// (P = p + 2) of 32 lanes
__host__ __device__ inline size_t far_store_entries(int p) { return (size_t)4 * (p + 2); }

__device__ inline void far_slots(unsigned char* smraw, int p, int w, double*& slot_p, double*& slot_q)
{
    const int P = p + 2;
    slot_p = reinterpret_cast<double*>(smraw) + (size_t)w * far_store_entries(p) * 32;
    slot_q = slot_p + (size_t)(2 * P + 1) * 32;
}

// ---------------------------------------------------------------------------
// FP32, compile-time order: coefficients in registers

// A target as FP32 hi/lo splits of its FP64 coordinates.
struct Tgt32 {
    float h0, h1, h2, l0, l1, l2;
};

__device__ inline Tgt32 load_tgt32(const double* __restrict__ ts, int64_t M, int64_t m, bool valid)
{
    Tgt32 t{0, 0, 0, 0, 0, 0};
    if (valid) {
        const double x0 = ts[m], x1 = ts[M + m], x2 = ts[2 * M + m];
        t.h0 = __double2float_rn(x0);
        t.h1 = __double2float_rn(x1);
        t.h2 = __double2float_rn(x2);
        t.l0 = __double2float_rn(x0 - (double)t.h0);
        t.l1 = __double2float_rn(x1 - (double)t.h1);
        t.l2 = __double2float_rn(x2 - (double)t.h2);
    }
    return t;
}

// c^k of hcoef_r for the two targets of a lane at once, (target 0, target 1)
// in the two halves of each FP32x2 register pair; nkap = -kappa_n / R'^2.
__device__ __forceinline__ float2 hcoef_r2(const float2* R1, const float2* R2, int n, int h, float2 v0, float2 v1,
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

// Far-field contribution of one cluster (folded FP32 tables tab, geometry
// gh = (y_c hi, 1/rho), gl = (y_c lo, 0)) to the two targets held by this
// lane.  Their recurrences run side by side on packed FP32x2 arithmetic and
// share every table load, so a table value broadcast to the warp feeds
// 2 x 32 products.  Lanes for which in[t] is false get finite garbage,
// discarded by the caller.
template <int P>
__device__ __forceinline__ void far_entry32(const Tgt32 (&tg)[2], const bool (&in)[2], const float4 gh,
                                            const float4 gl, const float4* __restrict__ tab, float (&res)[2][3])
{
    float d0[2], d1[2], d2[2], iR[2], iR2[2], v0[2], v1[2], v2[2];
#pragma unroll
    for (int t = 0; t < 2; t++) {
        d0[t] = ((tg[t].h0 - gh.x) + (tg[t].l0 - gl.x)) * gh.w;
        d1[t] = ((tg[t].h1 - gh.y) + (tg[t].l1 - gl.y)) * gh.w;
        d2[t] = ((tg[t].h2 - gh.z) + (tg[t].l2 - gl.z)) * gh.w;
        float R2 = fmaf(d0[t], d0[t], fmaf(d1[t], d1[t], d2[t] * d2[t]));
        if (!in[t]) R2 = 1.0f;
        iR[t] = rsqrtf(R2);
        iR2[t] = iR[t] * iR[t];
        v0[t] = d0[t] * iR2[t];
        v1[t] = d1[t] * iR2[t];
        v2[t] = d2[t] * iR2[t];
    }
    const float2 w0 = make_float2(v0[0], v0[1]), w1 = make_float2(v1[0], v1[1]), w2 = make_float2(v2[0], v2[1]);
    float2 tot[2][6];
    {
        const float4 a = __ldg(tab), b = __ldg(tab + 1), c = __ldg(tab + 2);
#pragma unroll
        for (int t = 0; t < 2; t++) {
            tot[t][0] = make_float2(a.x, a.y), tot[t][1] = make_float2(a.z, a.w);
            tot[t][2] = make_float2(b.x, b.y), tot[t][3] = make_float2(b.z, b.w);
            tot[t][4] = make_float2(c.x, c.y), tot[t][5] = make_float2(c.z, c.w);
        }
    }
    float2 cs[2][2 * P + 1];
    cs[0][0] = make_float2(1.0f, 1.0f);
#pragma unroll
    for (int n = 1; n <= P; n++) {
        const float2 nkap = make_float2(-c_lev32.kappa[n] * iR2[0], -c_lev32.kappa[n] * iR2[1]);
#pragma unroll
        for (int h = 2 * n; h >= 0; h--) {
            const float4* tl = tab + 3 * (n * n + h);
            const float4 a = __ldg(tl), b = __ldg(tl + 1), c = __ldg(tl + 2);
            const float2 cf = hcoef_r2(cs[(n - 1) & 1], cs[n & 1], n, h, w0, w1, w2, nkap);
            cs[n & 1][h] = cf;  // level n overwrites level n-2
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const float x = t == 0 ? cf.x : cf.y;
                const float2 c2 = make_float2(x, x);
                tot[t][0] = __ffma2_rn(c2, make_float2(a.x, a.y), tot[t][0]);
                tot[t][1] = __ffma2_rn(c2, make_float2(a.z, a.w), tot[t][1]);
                tot[t][2] = __ffma2_rn(c2, make_float2(b.x, b.y), tot[t][2]);
                tot[t][3] = __ffma2_rn(c2, make_float2(b.z, b.w), tot[t][3]);
                tot[t][4] = __ffma2_rn(c2, make_float2(c.x, c.y), tot[t][4]);
                tot[t][5] = __ffma2_rn(c2, make_float2(c.z, c.w), tot[t][5]);
            }
            // keep the table loads of later coefficients from being hoisted
            // here: that would exhaust the registers
            asm volatile("" ::: "memory");
        }
    }
#pragma unroll
    for (int t = 0; t < 2; t++) {
        const float T0 = tot[t][0].x, T1 = tot[t][0].y, T2 = tot[t][1].x, T3 = tot[t][1].y, T4 = tot[t][2].x,
                    T5 = tot[t][2].y, T6 = tot[t][3].x, T7 = tot[t][3].y, T8 = tot[t][4].x, T9 = tot[t][4].y,
                    T10 = tot[t][5].x, T11 = tot[t][5].y;
        res[t][0] = fmaf(d0[t], T3, fmaf(d1[t], T4, fmaf(d2[t], T5, T0))) * iR[t];
        res[t][1] = fmaf(d0[t], T6, fmaf(d1[t], T7, fmaf(d2[t], T8, T1))) * iR[t];
        res[t][2] = fmaf(d0[t], T9, fmaf(d1[t], T10, fmaf(d2[t], T11, T2))) * iR[t];
    }
}

// Far field of batches 2B and 2B+1 (the second may not exist) on one warp,
// two targets per lane, over the merge of the two far lists.  Both lists are
// in tree preorder, which orders clusters by (first source ascending, size
// descending, index ascending: a parent is numbered before its children);
// equal entries are the same cluster and are evaluated once for both batches.
template <int P>
__device__ __forceinline__ void far_pair32(const double* __restrict__ ts, int64_t M, const int4* __restrict__ topo,
                                           const float4* __restrict__ geo32, const float* __restrict__ ab,
                                           const int64_t* __restrict__ far_off,
                                           const ListEntry* __restrict__ far_list, double* __restrict__ u_far,
                                           int64_t B, int lane)
{
    constexpr int H = (P + 1) * (P + 1);
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t ba = 2 * B, bb = 2 * B + 1;
    const int64_t ma = ba * kBatch + lane, mb = bb * kBatch + lane;
    const bool va = ma < M, vb = mb < M;
    const Tgt32 ta = load_tgt32(ts, M, ma, va), tb = load_tgt32(ts, M, mb, vb);
    // per-entry contributions summed by compensated FP32 summation
    float sa[3] = {0.f, 0.f, 0.f}, ka[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f}, kb[3] = {0.f, 0.f, 0.f};
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
        const unsigned mA = takeA ? la.mask : 0u, mB = takeB ? lb.mask : 0u;
        const float4 gh = __ldg(geo32 + 2 * (int64_t)node), gl = __ldg(geo32 + 2 * (int64_t)node + 1);
        const float4* tab = reinterpret_cast<const float4*>(ab + (int64_t)node * H * 12);
        const bool inA = (mA >> lane) & 1u, inB = (mB >> lane) & 1u;
        {
            // both targets of the lane in one pass (a lane whose target is not
            // in the entry computes finite garbage for it, discarded here)
            const Tgt32 tg[2] = {ta, tb};
            const bool in[2] = {inA, inB};
            float r[2][3];
            far_entry32<P>(tg, in, gh, gl, tab, r);
            if (inA) {
                kahan_add(sa[0], ka[0], r[0][0]);
                kahan_add(sa[1], ka[1], r[0][1]);
                kahan_add(sa[2], ka[2], r[0][2]);
            }
            if (inB) {
                kahan_add(sb[0], kb[0], r[1][0]);
                kahan_add(sb[1], kb[1], r[1][1]);
                kahan_add(sb[2], kb[2], r[1][2]);
            }
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
        u_far[ma] = (double)sa[0] - (double)ka[0];
        u_far[M + ma] = (double)sa[1] - (double)ka[1];
        u_far[2 * M + ma] = (double)sa[2] - (double)ka[2];
    }
    if (vb) {
        u_far[mb] = (double)sb[0] - (double)kb[0];
        u_far[M + mb] = (double)sb[1] - (double)kb[1];
        u_far[2 * M + mb] = (double)sb[2] - (double)kb[2];
    }
}

// ---------------------------------------------------------------------------
// kernels

template <typename TC>
__global__ void __launch_bounds__(32)
    k_far64(const double* __restrict__ ts, int64_t M, const Geo* __restrict__ geo, const double* __restrict__ invrho,
            const TC* __restrict__ ab, int p, const int64_t* __restrict__ far_off,
            const ListEntry* __restrict__ far_list, double* __restrict__ u_far)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b = blockIdx.x;
    if (b >= nbatch) return;
    double *slot_p, *slot_q;
    far_slots(smraw, p, 0, slot_p, slot_q);
    far_batch64<TC>(ts, M, geo, invrho, ab, p, far_off, far_list, u_far, b, slot_p, slot_q, lane);
}

template <int P>
__device__ __noinline__ void far_pair32_at(const double* ts, int64_t M, const int4* topo, const float4* geo32,
                                           const float* ab, const int64_t* far_off, const ListEntry* far_list,
                                           double* u_far, int64_t B, int lane)
{
    far_pair32<P>(ts, M, topo, geo32, ab, far_off, far_list, u_far, B, lane);
}

// One resident grid of single-warp blocks taking batch pairs from a work
// queue (queue: a counter zeroed before the launch) until none is left.
template <int P>
__global__ void __launch_bounds__(32)
    k_far32(const double* __restrict__ ts, int64_t M, const int4* __restrict__ topo,
            const float4* __restrict__ geo32, const float* __restrict__ ab, const int64_t* __restrict__ far_off,
            const ListEntry* __restrict__ far_list, double* __restrict__ u_far, unsigned* __restrict__ queue)
{
    const int lane = threadIdx.x & 31;
    const int64_t nsuper = ((M + kBatch - 1) / kBatch + 1) / 2;
    for (;;) {
        unsigned B = 0;
        if (lane == 0) B = atomicAdd(queue, 1u);
        B = __shfl_sync(0xffffffffu, B, 0);
        if ((int64_t)B >= nsuper) break;
        far_pair32_at<P>(ts, M, topo, geo32, ab, far_off, far_list, u_far, (int64_t)B, lane);
    }
}

// Persistent far-field kernels over many systems: every warp repeatedly takes
// the next (system, item) from a device counter until the queue is empty.
// Items are numbered system by system (item_off: nsys + 1 offsets); an item
// is a batch in FP64 mode and a pair of batches in mixed precision.
__device__ inline int64_t next_item(const int64_t* __restrict__ item_off, int nsys, int64_t nitems,
                                    unsigned long long* counter, int lane, int& sys)
{
    unsigned long long item = 0;
    if (lane == 0) item = atomicAdd(counter, 1ull);
    item = __shfl_sync(0xffffffffu, item, 0);
    if ((int64_t)item >= nitems) return -1;
    int lo = 0, hi = nsys;  // item_off[lo] <= item < item_off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (item_off[mid] <= (int64_t)item)
            lo = mid;
        else
            hi = mid;
    }
    sys = lo;
    return (int64_t)item - item_off[lo];
}

// The batch bodies sit behind a call boundary in the persistent kernels:
// inlined into the work-queue loop they compiled to a body that issued about
// 1.6x the instructions of the one-batch kernel (measured: 108 ms against
// 40 ms for the same eight systems); as called functions they match it.
template <typename TC>
__device__ __noinline__ void far_batch64_call(const SysDesc* d, int p, int64_t b, double* slot_p, double* slot_q,
                                              int lane)
{
    far_batch64<TC>(d->ts, d->M, d->geo, d->invrho, (const TC*)d->ab, p, d->far_off, d->far_list, d->u_far, b,
                    slot_p, slot_q, lane);
}

template <int P>
__device__ __noinline__ void far_pair32_call(const SysDesc* d, int64_t B, int lane)
{
    far_pair32<P>(d->ts, d->M, d->topo, d->geo32, (const float*)d->ab, d->far_off, d->far_list, d->u_far, B, lane);
}

template <typename TC>
__global__ void k_far64_batched(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ item_off,
                                int64_t nitems, int p, unsigned long long* __restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *slot_p, *slot_q;
    far_slots(smraw, p, w, slot_p, slot_q);
    for (;;) {
        int s = 0;
        const int64_t b = next_item(item_off, nsys, nitems, counter, lane, s);
        if (b < 0) break;
        if (sizeof(TC) == 8) {
            far_batch64_call<TC>(sys + s, p, b, slot_p, slot_q, lane);
        } else {  // mixed precision: the item is the batch pair 2b, 2b+1
            const int64_t nb = (sys[s].M + kBatch - 1) / kBatch;
            far_batch64_call<TC>(sys + s, p, 2 * b, slot_p, slot_q, lane);
            if (2 * b + 1 < nb) far_batch64_call<TC>(sys + s, p, 2 * b + 1, slot_p, slot_q, lane);
        }
    }
}

template <int P>
__global__ void k_far32_batched(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ item_off,
                                int64_t nitems, unsigned long long* __restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        int s = 0;
        const int64_t b = next_item(item_off, nsys, nitems, counter, lane, s);
        if (b < 0) break;
        far_pair32_call<P>(sys + s, b, lane);
    }
}

// ---------------------------------------------------------------------------
// launchers

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename K>
cudaError_t persistent_grid(K kernel, int warps_per_block, size_t smem, int& blocks)
{
    if (blocks > 0) return cudaSuccess;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, warps_per_block * 32, smem);
    if (e != cudaSuccess) return e;
    blocks = (per_sm > 0 ? per_sm : 1) * sm_count();
    return cudaSuccess;
}

template <int P>
cudaError_t run_far32(const double* ts, int64_t M, const int4* topo, const float4* geo32, const float* ab,
                      const int64_t* far_off, const ListEntry* far_list, double* u_far, unsigned* queue,
                      cudaStream_t s)
{
    const int64_t nsuper = ((M + kBatch - 1) / kBatch + 1) / 2;
    int blocks = 0;
    cudaError_t e = persistent_grid(k_far32<P>, 1, 0, blocks);
    if (e != cudaSuccess) return e;
    if ((int64_t)blocks > nsuper) blocks = (int)nsuper;
    e = cudaMemsetAsync(queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_far32<P><<<(unsigned)blocks, 32, 0, s>>>(ts, M, topo, geo32, ab, far_off, far_list, u_far, queue);
    note_launch();
    return cudaGetLastError();
}

template <int P>
cudaError_t run_far32_batched(const SysDesc* sys, int nsys, const int64_t* item_off, int64_t nitems,
                              unsigned long long* counter, int warps_per_block, int blocks, cudaStream_t s)
{
    cudaError_t e = persistent_grid(k_far32_batched<P>, warps_per_block, 0, blocks);
    if (e != cudaSuccess) return e;
    k_far32_batched<P><<<blocks, warps_per_block * 32, 0, s>>>(sys, nsys, item_off, nitems, counter);
    note_launch();
    return cudaGetLastError();
}

template <typename TC>
cudaError_t run_far64(const double* ts, int64_t M, const Geo* geo, const double* invrho, const TC* ab, int p,
                      const int64_t* far_off, const ListEntry* far_list, double* u_far, cudaStream_t s)
{
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const size_t smem = far_store_entries(p) * 32 * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_far64<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_far64<TC><<<(unsigned)nbatch, 32, smem, s>>>(ts, M, geo, invrho, ab, p, far_off, far_list, u_far);
    note_launch();
    return cudaGetLastError();
}

template <typename TC>
cudaError_t run_far64_batched(const SysDesc* sys, int nsys, const int64_t* item_off, int64_t nitems, int p,
                              unsigned long long* counter, int warps_per_block, int blocks, cudaStream_t s)
{
    const size_t smem = (size_t)warps_per_block * far_store_entries(p) * 32 * sizeof(double);
    cudaError_t e =
        cudaFuncSetAttribute(k_far64_batched<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = persistent_grid(k_far64_batched<TC>, warps_per_block, smem, blocks);
    if (e != cudaSuccess) return e;
    k_far64_batched<TC><<<blocks, warps_per_block * 32, smem, s>>>(sys, nsys, item_off, nitems, p, counter);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_far(int precision, int rec64, const double* ts, int64_t M, const int4* topo, const Geo* geo,
                       const double* invrho, const float4* geo32, const double* ab64, const float* ab32, int p,
                       const int64_t* far_off, const ListEntry* far_list, double* u_far, unsigned* queue,
                       cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    if (precision == TC_FP64) return run_far64<double>(ts, M, geo, invrho, ab64, p, far_off, far_list, u_far, s);
    if (rec64 && p >= 8) return run_far64<float>(ts, M, geo, invrho, ab32, p, far_off, far_list, u_far, s);
    switch (p + 2) {
#define TC_FAR32_CASE(P) \
    case P: return run_far32<P>(ts, M, topo, geo32, ab32, far_off, far_list, u_far, queue, s);
        TC_FAR32_CASE(2) TC_FAR32_CASE(3) TC_FAR32_CASE(4) TC_FAR32_CASE(5) TC_FAR32_CASE(6)
        TC_FAR32_CASE(7) TC_FAR32_CASE(8) TC_FAR32_CASE(9) TC_FAR32_CASE(10) TC_FAR32_CASE(11)
        TC_FAR32_CASE(12) TC_FAR32_CASE(13) TC_FAR32_CASE(14)
#undef TC_FAR32_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_far_batched(int precision, int rec64, const SysDesc* sys, int nsys, const int64_t* item_off,
                               int64_t nitems, int p, unsigned long long* counter, int warps_per_block, int blocks,
                               cudaStream_t s)
{
    if (precision == TC_FP64)
        return run_far64_batched<double>(sys, nsys, item_off, nitems, p, counter, warps_per_block, blocks, s);
    if (rec64 && p >= 8)
        return run_far64_batched<float>(sys, nsys, item_off, nitems, p, counter, warps_per_block, blocks, s);
    switch (p + 2) {
#define TC_FAR32B_CASE(P) \
    case P: return run_far32_batched<P>(sys, nsys, item_off, nitems, counter, warps_per_block, blocks, s);
        TC_FAR32B_CASE(2) TC_FAR32B_CASE(3) TC_FAR32B_CASE(4) TC_FAR32B_CASE(5) TC_FAR32B_CASE(6)
        TC_FAR32B_CASE(7) TC_FAR32B_CASE(8) TC_FAR32B_CASE(9) TC_FAR32B_CASE(10) TC_FAR32B_CASE(11)
        TC_FAR32B_CASE(12) TC_FAR32B_CASE(13) TC_FAR32B_CASE(14)
#undef TC_FAR32B_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace tc
