// Far field: particle-cluster Taylor approximation, eq. (2.9), evaluated in
// the contracted form of the contraction tables (tc_moments.cu):
//   u_i += sum_{||k'|| <= p+2} b^{k'}(d') ( Â_i^{k'} + sum_l d'_l B̂_il^{k'} ),
// with d' = (x - y_c) / rho and the Coulomb coefficients b^k of the
// recurrence (3.2):
//   n R^2 b^k = (2n-1) sum_i d_i b^{k-e_i} - (n-1) sum_i b^{k-2e_i},  n = ||k||.
//
// The recurrence is run on the unit vector w = d'/R' (R' = |d'|): b^k is
// homogeneous of degree -(n+1), so b^k(d') = R'^-(n+1) b^k(w), and with
// |w| = 1 the coefficients (2n-1)/n and (n-1)/n no longer depend on the
// target.  Writing b^k(w) = lambda_n c^k with lambda_n = prod_{j<=n} (2j-1)/j
// turns the recurrence into
//   c^k = sum_i w_i c^{k-e_i} - kappa_n sum_i c^{k-2e_i},
//   kappa_n = (n-1)^2 / ((2n-1)(2n-3)),  c^0 = 1,
// all O(1) in magnitude.  The level factor lambda_n R'^-(n+1) multiplies the
// level's 12 partial contractions.  Because the tables are folded onto the
// harmonic subset k1 <= 1 (k_fold_tables: Laplace's equation expresses every
// b^k with k1 >= 2 through coefficients of smaller k1 on the same level), only
// the (P+1)^2 coefficients with k1 <= 1 are formed, at most five FP64
// operations each, and the recurrence never needs any other.
//
// One warp handles a batch of 32 targets (one per lane) and walks the batch's
// far list; a lane outside an entry's mask idles for that entry.  The
// coefficients live in a per-warp shared-memory store of two slots laid out
// [slot][position][lane] (no bank conflicts): level n overwrites level n-2 in
// place, positions running downward, which is safe because a coefficient
// reads level n-2 only at positions <= its own.  Two coefficients are formed
// per step for instruction-level parallelism.  Each coefficient is contracted
// against the cluster's 12 folded table entries as soon as it exists.
//
// Precision: TR is the recurrence type, TC the table/contraction type.
// FP64 mode: TR = TC = double.  Mixed: TC = float, TR = double for p >= 8 and
// float below; the FP64 -> FP32 narrowing of each coefficient is done with
// integer operations (round to nearest, ties away from zero; magnitudes below
// 2^-126 flushed to zero) so that it does not occupy the FP64 pipe.  Each
// cluster's contribution is added to an FP64 per-target accumulator.
#include "tc_recurrence.cuh"

namespace tc {

namespace {

constexpr int kFarWarps = 1;

__constant__ LevelConst c_lev = make_level_const();

template <typename TC>
__device__ inline void contract(TC c, const TC* __restrict__ t, TC* acc)
{
#pragma unroll
    for (int q = 0; q < 12; q++) acc[q] = fma(c, t[q], acc[q]);
}

// One coefficient c^k of the harmonic subset (k1 <= 1) at level n, subset
// position h (0..2n): k1 = 0 for h <= n (k3 = h), else k1 = 1 (k3 = h-n-1).
// R1 holds level n-1 and R2 level n-2 of the subset, [position][lane].
template <typename TR>
__device__ inline TR hcoef(const TR* R1, const TR* R2, int n, int h, TR w0, TR w1, TR w2, TR kap, int lane)
{
    TR s1, s2 = 0;
    if (h <= n) {  // k = (0, n - h, h)
        const int k3 = h, k2 = n - h;
        s1 = 0;
        if (k2 >= 1) s1 = w1 * R1[k3 * 32 + lane];
        if (k3 >= 1) s1 = fma(w2, R1[(k3 - 1) * 32 + lane], s1);
        if (k2 >= 2) s2 = R2[k3 * 32 + lane];
        if (k3 >= 2) s2 += R2[(k3 - 2) * 32 + lane];
    } else {  // k = (1, n - 1 - k3, k3)
        const int k3 = h - n - 1, k2 = n - 1 - k3;
        s1 = w0 * R1[k3 * 32 + lane];
        if (k2 >= 1) s1 = fma(w1, R1[(n + k3) * 32 + lane], s1);
        if (k3 >= 1) s1 = fma(w2, R1[(n + k3 - 1) * 32 + lane], s1);
        if (k2 >= 2) s2 = R2[(n - 1 + k3) * 32 + lane];
        if (k3 >= 2) s2 += R2[(n - 3 + k3) * 32 + lane];
    }
    return fma(-kap, s2, s1);
}

// The far field of batch b (32 targets, one per lane) on one warp, with the
// folded tables of the harmonic subset (tc_moments.cu, k_fold_tables): only
// the (P+1)^2 coefficients with k1 <= 1 are formed, 2n+1 per level.  slot_p
// holds the levels of the parity of P = p + 2 (2P+1 entries x 32 lanes) and
// slot_q the others (2P-1 x 32); level n overwrites level n-2 in place,
// positions running downward (a coefficient reads level n-2 only at
// positions <= its own).
template <typename TR, typename TC>
__device__ inline void far_batch(const double* __restrict__ ts, int64_t M, const Geo* __restrict__ geo,
                                 const double* __restrict__ invrho, const TC* __restrict__ ab, int p,
                                 const int64_t* __restrict__ far_off, const ListEntry* __restrict__ far_list,
                                 double* __restrict__ u_far, int64_t b, TR* slot_p, TR* slot_q, int lane)
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
        const TR w0 = (TR)(d0 * iR), w1 = (TR)(d1 * iR), w2 = (TR)(d2 * iR);
        const TC* __restrict__ tab = ab + (int64_t)le.node * H * 12;
        TC tot[12];
        TC scale = (TC)iR;  // lambda_0 R'^-1; level 0: c^0 = 1
#pragma unroll
        for (int q = 0; q < 12; q++) tot[q] = scale * tab[q];
        ((P & 1) ? slot_q : slot_p)[lane] = (TR)1;  // level 0 has parity 0
        __syncwarp();
        for (int n = 1; n <= P; n++) {
            const TR kap = (TR)c_lev.kappa[n];
            scale *= (TC)(c_lev.ratio[n] * iR);
            TR* Rn = ((n ^ P) & 1) ? slot_q : slot_p;  // also holds level n-2
            const TR* R1 = ((n ^ P) & 1) ? slot_p : slot_q;
            const TC* tl = tab + (int64_t)n * n * 12;
            TC acc[12];
#pragma unroll
            for (int q = 0; q < 12; q++) acc[q] = (TC)0;
            int h = 2 * n;
            for (; h >= 1; h -= 2) {
                const TR ca = hcoef<TR>(R1, Rn, n, h, w0, w1, w2, kap, lane);
                const TR cb = hcoef<TR>(R1, Rn, n, h - 1, w0, w1, w2, kap, lane);
                Rn[h * 32 + lane] = ca;
                Rn[(h - 1) * 32 + lane] = cb;
                contract<TC>(to_tc<TR, TC>(ca), tl + h * 12, acc);
                contract<TC>(to_tc<TR, TC>(cb), tl + (h - 1) * 12, acc);
            }
            if (h == 0) {
                const TR ca = hcoef<TR>(R1, Rn, n, 0, w0, w1, w2, kap, lane);
                Rn[lane] = ca;
                contract<TC>(to_tc<TR, TC>(ca), tl, acc);
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < 12; q++) tot[q] = fma(scale, acc[q], tot[q]);
        }
        if (in) {
            const TC e0c = (TC)d0, e1c = (TC)d1, e2c = (TC)d2;
            const TC v0 = tot[0] + e0c * tot[3] + e1c * tot[4] + e2c * tot[5];
            const TC v1 = tot[1] + e0c * tot[6] + e1c * tot[7] + e2c * tot[8];
            const TC v2 = tot[2] + e0c * tot[9] + e1c * tot[10] + e2c * tot[11];
            ux += (double)v0;
            uy += (double)v1;
            uz += (double)v2;
        }
    }
    if (valid) {
        u_far[m] = ux;
        u_far[M + m] = uy;
        u_far[2 * M + m] = uz;
    }
}

// per-warp coefficient store: 2P+1 and 2P-1 entries (P = p + 2) of 32 lanes
__host__ __device__ inline size_t far_store_entries(int p) { return (size_t)4 * (p + 2); }

template <typename TR>
__device__ inline void far_slots(unsigned char* smraw, int p, int w, TR*& slot_p, TR*& slot_q)
{
    const int P = p + 2;
    slot_p = reinterpret_cast<TR*>(smraw) + (size_t)w * far_store_entries(p) * 32;
    slot_q = slot_p + (size_t)(2 * P + 1) * 32;
}

template <typename TR, typename TC>
__global__ void __launch_bounds__(kFarWarps * 32)
    k_far(const double* __restrict__ ts, int64_t M, const Geo* __restrict__ geo,
          const double* __restrict__ invrho, const TC* __restrict__ ab, int p, const int64_t* __restrict__ far_off,
          const ListEntry* __restrict__ far_list, double* __restrict__ u_far)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b = blockIdx.x * (int64_t)kFarWarps + w;
    if (b >= nbatch) return;
    TR *slot_p, *slot_q;
    far_slots<TR>(smraw, p, w, slot_p, slot_q);
    far_batch<TR, TC>(ts, M, geo, invrho, ab, p, far_off, far_list, u_far, b, slot_p, slot_q, lane);
}

// Persistent far-field kernel over many systems: every warp repeatedly takes
// the next (system, batch) item from a device counter until the queue is
// empty.  Items are numbered system by system (item_off: nsys + 1 offsets).
template <typename TR, typename TC>
__global__ void k_far_batched(const SysDesc* __restrict__ sys, int nsys, const int64_t* __restrict__ item_off,
                              int64_t nitems, int p, unsigned long long* __restrict__ counter)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    TR *slot_p, *slot_q;
    far_slots<TR>(smraw, p, w, slot_p, slot_q);
    for (;;) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(counter, 1ull);
        item = __shfl_sync(0xffffffffu, item, 0);
        if ((int64_t)item >= nitems) break;
        int lo = 0, hi = nsys;  // item_off[lo] <= item < item_off[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (item_off[mid] <= (int64_t)item)
                lo = mid;
            else
                hi = mid;
        }
        const SysDesc& d = sys[lo];
        far_batch<TR, TC>(d.ts, d.M, d.geo, d.invrho, (const TC*)d.ab, p, d.far_off, d.far_list, d.u_far,
                          (int64_t)item - item_off[lo], slot_p, slot_q, lane);
    }
}

template <typename TR, typename TC>
cudaError_t run_far_batched(const SysDesc* sys, int nsys, const int64_t* item_off, int64_t nitems, int p,
                            unsigned long long* counter, int warps_per_block, int blocks, cudaStream_t s)
{
    size_t smem = (size_t)warps_per_block * far_store_entries(p) * 32 * sizeof(TR);
    cudaError_t e =
        cudaFuncSetAttribute(k_far_batched<TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks <= 0) {
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_far_batched<TR, TC>, warps_per_block * 32, smem);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        blocks = (per_sm > 0 ? per_sm : 1) * sms;
    }
    k_far_batched<TR, TC><<<blocks, warps_per_block * 32, smem, s>>>(sys, nsys, item_off, nitems, p, counter);
    note_launch();
    return cudaGetLastError();
}

template <typename TR, typename TC>
cudaError_t run_far(const double* ts, int64_t M, const Geo* geo, const double* invrho, const TC* ab, int p,
                    const int64_t* far_off, const ListEntry* far_list, double* u_far, cudaStream_t s)
{
    int64_t nbatch = (M + kBatch - 1) / kBatch;
    unsigned grid = (unsigned)((nbatch + kFarWarps - 1) / kFarWarps);
    size_t smem = (size_t)kFarWarps * far_store_entries(p) * 32 * sizeof(TR);
    cudaError_t e = cudaFuncSetAttribute(k_far<TR, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_far<TR, TC><<<grid, kFarWarps * 32, smem, s>>>(ts, M, geo, invrho, ab, p, far_off, far_list, u_far);
    note_launch();
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_far(int precision, const double* ts, int64_t M, const Geo* geo, const double* invrho,
                       const double* ab64, const float* ab32, int p, const int64_t* far_off,
                       const ListEntry* far_list, double* u_far, cudaStream_t s)
{
    if (precision == TC_FP64) return run_far<double, double>(ts, M, geo, invrho, ab64, p, far_off, far_list, u_far, s);
    if (p >= 8) return run_far<double, float>(ts, M, geo, invrho, ab32, p, far_off, far_list, u_far, s);
    return run_far<float, float>(ts, M, geo, invrho, ab32, p, far_off, far_list, u_far, s);
}

cudaError_t launch_far_batched(int precision, const SysDesc* sys, int nsys, const int64_t* item_off, int64_t nitems,
                               int p, unsigned long long* counter, int warps_per_block, int blocks, cudaStream_t s)
{
    if (precision == TC_FP64)
        return run_far_batched<double, double>(sys, nsys, item_off, nitems, p, counter, warps_per_block, blocks, s);
    if (p >= 8)
        return run_far_batched<double, float>(sys, nsys, item_off, nitems, p, counter, warps_per_block, blocks, s);
    return run_far_batched<float, float>(sys, nsys, item_off, nitems, p, counter, warps_per_block, blocks, s);
}

}  // namespace tc
