// Packed FP32x2 near-field machinery shared by the forward near field
// (tc_near.cu) and the target side of its adjoint (tc_adjoint.cu): the
// staging of 32-source tiles as source pairs, the sums of one leaf at one or
// two 32-target streams, and the leaf-major schedule that packs the targets
// of each leaf into full streams.  See tc_near.cu for the design.
#pragma once

#include "tc_internal.cuh"

namespace tc {
namespace nearpair {

// ---------------------------------------------------------------------------
// mixed precision: packed FP32x2 arithmetic

__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 r;
    asm("{\n\t.reg .b64 ta, tb, td;\n\tmov.b64 ta, {%2, %3};\n\tmov.b64 tb, {%4, %5};\n\t"
        "sub.rn.f32x2 td, ta, tb;\n\tmov.b64 {%0, %1}, td;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// A source record is 16 FP32 fields: x_hi (3), f0, x_lo (3), f1, f2, h (3),
// nu (3), pad.  The tile stores source pair q (sources 2q, 2q+1) as 8 float4,
// float4 k = (y_2q.f_2k, y_2q+1.f_2k, y_2q.f_2k+1, y_2q+1.f_2k+1), with a
// stride of 9 float4 per pair so that the staging stores are free of bank
// conflicts.
constexpr int kPairStride = 9;
constexpr int kTileFloat4 = 16 * kPairStride;

// Stage sources [base, base + cnt), cnt <= 32, into the tile.  Lanes past cnt
// contribute a source at 1e30 with zero weights (its terms are exactly 0:
// r^2 overflows to inf, 1/r = 0, and every weight is 0).
__device__ inline void stage_pairs(const float4* __restrict__ spack, int64_t base, int cnt, float4* tw, int lane)
{
    float f[16];
    if (lane < cnt) {
        const float4* src = spack + 4 * (base + lane);
        const float4 a = src[0], b = src[1], c = src[2], d = src[3];
        f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w;
        f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
        f[8] = c.x, f[9] = c.y, f[10] = c.z, f[11] = c.w;
        f[12] = d.x, f[13] = d.y, f[14] = d.z, f[15] = d.w;
    } else {
#pragma unroll
        for (int k = 0; k < 16; k++) f[k] = k < 3 ? 1e30f : 0.0f;
    }
    const int par = lane & 1;
    float recv[8];
#pragma unroll
    for (int k = 0; k < 8; k++) recv[k] = __shfl_xor_sync(0xffffffffu, par ? f[k] : f[8 + k], 1);
    float4* dst = tw + (lane >> 1) * kPairStride;
    if (!par) {
#pragma unroll
        for (int j = 0; j < 4; j++) dst[j] = make_float4(f[2 * j], recv[2 * j], f[2 * j + 1], recv[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < 4; j++)
            dst[4 + j] = make_float4(recv[2 * j], f[8 + 2 * j], recv[2 * j + 1], f[9 + 2 * j]);
    }
}

// The near field of one leaf (sources first .. first + count - 1) at the
// targets of one or two streams (ta, and tb when two), on the warp's tile:
// per 32-source tile the packed pair sums of each target, accumulated over
// the leaf's tiles by compensated FP32 summation (sum, compensation per
// component) and returned in FP64 as sum less compensation (ra for ta, rb for
// tb).  guard: a source of the leaf may coincide with a target.  Every
// schedule of the near field computes a leaf's sums here, so a target's sums
// do not depend on the schedule.
template <typename Op>
__device__ __forceinline__ void leaf_sums(const typename Op::Tgt& ta, const typename Op::Tgt& tb, bool two,
                                          bool guard, int first, int count, const float4* __restrict__ spack,
                                          float4* tile, int lane, double (&ra)[3], double (&rb)[3])
{
    float sa[3] = {0.f, 0.f, 0.f}, ka[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f}, kb[3] = {0.f, 0.f, 0.f};
    for (int base = first; base < first + count; base += 32) {
        const int cnt = min(32, first + count - base);
        __syncwarp();
        stage_pairs(spack, base, cnt, tile, lane);
        __syncwarp();
        const int npairs = (cnt + 1) >> 1;
        float2 axa = make_float2(0.f, 0.f), aya = axa, aza = axa, axb = axa, ayb = axa, azb = axa;
        if (two && guard) {
            for (int q = 0; q < npairs; q++) {
                const float4* tp = tile + q * kPairStride;
                Op::template terms<true>(ta, tp, axa, aya, aza);
                Op::template terms<true>(tb, tp, axb, ayb, azb);
            }
        } else if (two) {
            for (int q = 0; q < npairs; q++) {
                const float4* tp = tile + q * kPairStride;
                Op::template terms<false>(ta, tp, axa, aya, aza);
                Op::template terms<false>(tb, tp, axb, ayb, azb);
            }
        } else if (guard) {
            for (int q = 0; q < npairs; q++) Op::template terms<true>(ta, tile + q * kPairStride, axa, aya, aza);
        } else {
            for (int q = 0; q < npairs; q++) Op::template terms<false>(ta, tile + q * kPairStride, axa, aya, aza);
        }
        kahan_add(sa[0], ka[0], axa.x + axa.y);
        kahan_add(sa[1], ka[1], aya.x + aya.y);
        kahan_add(sa[2], ka[2], aza.x + aza.y);
        kahan_add(sb[0], kb[0], axb.x + axb.y);
        kahan_add(sb[1], kb[1], ayb.x + ayb.y);
        kahan_add(sb[2], kb[2], azb.x + azb.y);
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        ra[k] = (double)sa[k] - (double)ka[k];
        rb[k] = (double)sb[k] - (double)kb[k];
    }
}

// ---------------------------------------------------------------------------
// Leaf-major schedule of the near field and of the target side of its
// adjoint.  The near entries are sorted by leaf (near_schedule); the targets
// of all entries of a leaf, its incidences, are packed densely into 32-lane
// streams, so that only a leaf's last stream is partial, and the units of
// work, (leaf, pair of streams), are drained by a resident grid in order of
// decreasing leaf size.  A unit writes each of its targets' leaf sums to the
// slot of its (entry, lane); k_near_reduce then adds each target's slots in
// list order (tree order), starting from zero.  A target's sums do not depend
// on which stream or lane it is packed into, nor on the order of the units,
// so the result is the same whatever the packing, the grid or the number of
// systems in a batch.
constexpr int kLeafWarps = 4;       // warps per block of k_near_leaf
constexpr int kLeafFreeBlocks = 1;  // block slots per SM left free (for the far field on the second stream)

// Unit i of a schedule on one warp (tile: the warp's source tile).
template <typename Op>
__device__ __forceinline__ void leaf_unit(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                                          const int4* __restrict__ topo, const float4* __restrict__ spack,
                                          const int2* __restrict__ units, const int64_t* __restrict__ node_inc0,
                                          const int32_t* __restrict__ node_A, const int32_t* __restrict__ inc_m,
                                          const int32_t* __restrict__ inc_e, double* __restrict__ slots, int self,
                                          float prm, int64_t i, float4* tile, int lane)
{
    const int2 un = units[i];
    const int node = un.x;
    const int64_t I0 = node_inc0[node];
    const int A = node_A[node];
    const int k1 = 64 * un.y + lane, k2 = k1 + 32;
    const bool two = 64 * un.y + 32 < A;
    const bool v1 = k1 < A, v2 = k2 < A;
    const int m1 = v1 ? inc_m[I0 + k1] : 0, m2 = v2 ? inc_m[I0 + k2] : 0;
    const typename Op::Tgt ta = Op::load(ts, gs, M, m1, v1, prm);
    const typename Op::Tgt tb = Op::load(ts, gs, M, m2, v2, prm);
    const int4 t = topo[node];
    // r = 0 needs the target to coincide with a source of this leaf.  With
    // targets = sources (self) that is only possible for a target inside the
    // leaf's own range (coincident points have one Morton key, so they share
    // a leaf); otherwise (disjoint targets) every pair keeps the guard.
    const bool guard = !Op::kUnguarded || !self ||
                       __any_sync(0xffffffffu, (v1 && m1 >= t.x && m1 < t.x + t.y) ||
                                                   (v2 && m2 >= t.x && m2 < t.x + t.y));
    double a[3], c[3];
    leaf_sums<Op>(ta, tb, two, guard, t.x, t.y, spack, tile, lane, a, c);
    // slot of (entry e, component k, lane l): 96 e + 32 k + l
    if (v1) {
        double* q = slots + (int64_t)inc_e[I0 + k1] * 96 + (m1 & 31);
        q[0] = a[0], q[32] = a[1], q[64] = a[2];
    }
    if (v2) {
        double* q = slots + (int64_t)inc_e[I0 + k2] * 96 + (m2 & 31);
        q[0] = c[0], q[32] = c[1], q[64] = c[2];
    }
}

template <typename Op>
__global__ void __launch_bounds__(kLeafWarps * 32)
    k_near_leaf(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                const int4* __restrict__ topo, const float4* __restrict__ spack, const int2* __restrict__ units,
                const int32_t* __restrict__ nunits, const int64_t* __restrict__ node_inc0,
                const int32_t* __restrict__ node_A, const int32_t* __restrict__ inc_m,
                const int32_t* __restrict__ inc_e, double* __restrict__ slots, int self, float prm,
                unsigned* __restrict__ queue)
{
    __shared__ float4 tile[kLeafWarps][kTileFloat4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned nu = (unsigned)*nunits;
    for (;;) {
        unsigned i = 0;
        if (lane == 0) i = atomicAdd(queue, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if (i >= nu) break;
        leaf_unit<Op>(ts, gs, M, topo, spack, units, node_inc0, node_A, inc_m, inc_e, slots, self, prm, i, tile[w],
                      lane);
    }
}

// One warp per batch: each lane adds its target's slots over the batch's near
// entries, in list order, starting from zero, and stores (or, kAdd, adds) the
// sum.
template <bool kAdd>
__device__ __forceinline__ void reduce_batch(const int64_t* __restrict__ near_off,
                                             const ListEntry* __restrict__ near_list, int64_t M,
                                             const double* __restrict__ slots, double* __restrict__ out, int64_t b,
                                             int lane)
{
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    const int64_t e1 = near_off[b + 1];
    for (int64_t e = near_off[b]; e < e1; e++)
        if ((near_list[e].mask >> lane) & 1u) {
            const double* q = slots + e * 96 + lane;
            a0 += q[0];
            a1 += q[32];
            a2 += q[64];
        }
    const int64_t m = b * kBatch + lane;
    if (m < M) {
        if (kAdd) {
            out[m] += a0;
            out[M + m] += a1;
            out[2 * M + m] += a2;
        } else {
            out[m] = a0;
            out[M + m] = a1;
            out[2 * M + m] = a2;
        }
    }
}

template <bool kAdd>
__global__ void k_near_reduce(const int64_t* __restrict__ near_off, const ListEntry* __restrict__ near_list,
                              int64_t M, const double* __restrict__ slots, double* __restrict__ out)
{
    const int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= (M + kBatch - 1) / kBatch) return;
    reduce_batch<kAdd>(near_off, near_list, M, slots, out, b, threadIdx.x & 31);
}

// blocks of k_near_leaf<Op> the grid takes: the occupancy limit less
// kLeafFreeBlocks per SM, times the SMs
template <typename Op>
int64_t leaf_resident_blocks()
{
    static int ps = 0, sms = 0;
    if (ps == 0) {
        int dev = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_near_leaf<Op>, kLeafWarps * 32, 0) != cudaSuccess ||
            ps < 1)
            ps = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return (int64_t)(ps > kLeafFreeBlocks ? ps - kLeafFreeBlocks : 1) * (sms > 0 ? sms : 1);
}

// The near field of Op over the schedule sc (near_schedule): the units, then
// the sums per target into out.
template <typename Op>
cudaError_t run_near_leaf(const double* ts, const double* gs, int64_t M, const int4* topo, const float4* spack,
                          const int64_t* near_off, const ListEntry* near_list, double* out, int self, float prm,
                          const NearSched& sc, cudaStream_t s)
{
    if (sc.E > 0) {
        // at most one unit per warp of the grid when every entry had its own unit
        const int64_t resident = leaf_resident_blocks<Op>();
        const int64_t need = (sc.max_units + kLeafWarps - 1) / kLeafWarps;
        const unsigned grid = (unsigned)(need < resident ? (need > 0 ? need : 1) : resident);
        cudaError_t e = cudaMemsetAsync(sc.queue, 0, sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        k_near_leaf<Op><<<grid, kLeafWarps * 32, 0, s>>>(ts, gs, M, topo, spack, sc.units, sc.nunits, sc.node_inc0,
                                                         sc.node_A, sc.inc_m, sc.inc_e, sc.slots, self, prm, sc.queue);
        note_launch();
    }
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    k_near_reduce<Op::kAdd><<<(unsigned)((nbatch + 7) / 8), 256, 0, s>>>(near_off, near_list, M, sc.slots, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace nearpair
}  // namespace tc
