// Packed FP32x2 near-field machinery shared by the forward near field
// (tc_near.cu) and the target side of its adjoint (tc_adjoint.cu): the
// staging of 32-source tiles as source pairs, and the walk of a group of
// batches over the merge of their near lists with the targets of each leaf
// packed into 32-lane streams.  See tc_near.cu for the design.
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

// Per-warp scratch of the compacted near kernel: the source tile, the
// accumulators of the warp's G x 32 targets and the stream slot map.
template <int G>
struct NearScratch {
    float4 tile[kTileFloat4];
    double acc[G][3][32];
    int slot[G * 32];
};

// Near field of batches G*B .. G*B+G-1 (the last ones may not exist) on one
// warp, over the merge of their G near lists (all in tree order, so by the
// leaf's first source); lane g < G holds the cursor of list g, so the merge
// state costs a few registers whatever G.  For each leaf, the targets of the
// G batches that need it (the union of the entries' lane masks, A of them)
// are packed densely into ceil(A/32) streams of 32 lanes, so lanes whose
// target does not need the leaf are not computed (lane use of single-batch
// lists at N = 1M: 0.74); streams are evaluated two at a time, each sharing
// the staged tile, and each result is added to its target's accumulator in
// shared memory.  A target's arithmetic does not depend on which stream or
// lane it is packed into, so any group size gives the same bits.  self: the targets are the sources (sorted index = source
// index), which lets leaves that cannot hold a stream's own target skip the
// r = 0 guard.
//
// Op supplies the per-target record (Op::Tgt, Op::load), the pair terms of one
// target against a staged source pair (Op::terms<kGuard>, three FP32x2
// accumulators), whether the result is stored or added (Op::kAdd), and
// whether its terms are also compiled without the r = 0 guard (Op::kUnguarded);
// gs and prm are passed through to Op::load (the adjoint's target weights g,
// unused by the forward field; prm: eps^2 of the regularized kernels).
template <int G, typename Op>
__device__ inline void near_group(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                                  const int4* __restrict__ topo, const float4* __restrict__ spack,
                                  const int64_t* __restrict__ near_off, const ListEntry* __restrict__ near_list,
                                  double* __restrict__ out, int64_t B, int self, float prm, NearScratch<G>& sc,
                                  int lane)
{
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b0 = (int64_t)G * B;
    constexpr int kEnd = 0x7fffffff;
    constexpr unsigned kAll = 0xffffffffu;
    // lane g < G holds the cursor of list g
    int64_t cur = 0, end = 0;
    if (lane < G && b0 + lane < nbatch) {
        cur = near_off[b0 + lane];
        end = near_off[b0 + lane + 1];
    }
    ListEntry le{0, 0};
    int key = kEnd;
    if (cur < end) {
        le = near_list[cur];
        key = topo[le.node].x;
    }
#pragma unroll
    for (int g = 0; g < G; g++)
#pragma unroll
        for (int c = 0; c < 3; c++) sc.acc[g][c][lane] = 0.0;
    const unsigned lt = (1u << lane) - 1u;
    for (;;) {
        int kmin = key;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) kmin = min(kmin, __shfl_xor_sync(kAll, kmin, o));
        kmin = __shfl_sync(kAll, kmin, 0);
        if (kmin == kEnd) break;
        // leaves are disjoint ranges, so equal first sources name one leaf
        const bool match = lane < G && key == kmin;
        const unsigned mine = match ? le.mask : 0u;
        const int node = __shfl_sync(kAll, le.node, __ffs(__ballot_sync(kAll, match)) - 1);
        unsigned m[G];
        int A = 0, P[G];
#pragma unroll
        for (int g = 0; g < G; g++) {
            m[g] = __shfl_sync(kAll, mine, g);
            P[g] = A;
            A += __popc(m[g]);
        }
        __syncwarp();
#pragma unroll
        for (int g = 0; g < G; g++)
            if ((m[g] >> lane) & 1u) sc.slot[P[g] + __popc(m[g] & lt)] = g * 32 + lane;
        __syncwarp();
        const int4 t = topo[node];
        const int S = (A + 31) >> 5;
        for (int s = 0; s < S; s += 2) {
            const bool two = s + 1 < S;
            const int k1 = 32 * s + lane, k2 = k1 + 32;
            const bool v1 = k1 < A, v2 = two && k2 < A;
            const int id1 = v1 ? sc.slot[k1] : 0, id2 = v2 ? sc.slot[k2] : 0;
            const int64_t m1 = (b0 + (id1 >> 5)) * kBatch + (id1 & 31), m2 = (b0 + (id2 >> 5)) * kBatch + (id2 & 31);
            const typename Op::Tgt ta = Op::load(ts, gs, M, m1, v1, prm);
            const typename Op::Tgt tb = Op::load(ts, gs, M, m2, v2, prm);
            // r = 0 needs the target to coincide with a source of this leaf.
            // With targets = sources (self) that is only possible for a
            // target inside the leaf's own range (coincident points have
            // one Morton key, so they share a leaf); otherwise (disjoint
            // targets) every pair keeps the guard.
            const bool guard = !Op::kUnguarded || !self ||
                               __any_sync(0xffffffffu, (v1 && m1 >= t.x && m1 < (int64_t)t.x + t.y) ||
                                                           (v2 && m2 >= t.x && m2 < (int64_t)t.x + t.y));
            // per-tile partial sums, accumulated over the leaf's tiles by
            // compensated FP32 summation (sum, compensation per component)
            float sa[3] = {0.f, 0.f, 0.f}, ka[3] = {0.f, 0.f, 0.f}, sb[3] = {0.f, 0.f, 0.f},
                  kb[3] = {0.f, 0.f, 0.f};
            for (int base = t.x; base < t.x + t.y; base += 32) {
                const int cnt = min(32, t.x + t.y - base);
                __syncwarp();
                stage_pairs(spack, base, cnt, sc.tile, lane);
                __syncwarp();
                const int npairs = (cnt + 1) >> 1;
                float2 axa = make_float2(0.f, 0.f), aya = axa, aza = axa, axb = axa, ayb = axa, azb = axa;
                if (two && guard) {
                    for (int q = 0; q < npairs; q++) {
                        const float4* tp = sc.tile + q * kPairStride;
                        Op::template terms<true>(ta, tp, axa, aya, aza);
                        Op::template terms<true>(tb, tp, axb, ayb, azb);
                    }
                } else if (two) {
                    for (int q = 0; q < npairs; q++) {
                        const float4* tp = sc.tile + q * kPairStride;
                        Op::template terms<false>(ta, tp, axa, aya, aza);
                        Op::template terms<false>(tb, tp, axb, ayb, azb);
                    }
                } else if (guard) {
                    for (int q = 0; q < npairs; q++)
                        Op::template terms<true>(ta, sc.tile + q * kPairStride, axa, aya, aza);
                } else {
                    for (int q = 0; q < npairs; q++)
                        Op::template terms<false>(ta, sc.tile + q * kPairStride, axa, aya, aza);
                }
                kahan_add(sa[0], ka[0], axa.x + axa.y);
                kahan_add(sa[1], ka[1], aya.x + aya.y);
                kahan_add(sa[2], ka[2], aza.x + aza.y);
                kahan_add(sb[0], kb[0], axb.x + axb.y);
                kahan_add(sb[1], kb[1], ayb.x + ayb.y);
                kahan_add(sb[2], kb[2], azb.x + azb.y);
            }
            const double a0 = (double)sa[0] - (double)ka[0], a1 = (double)sa[1] - (double)ka[1],
                         a2 = (double)sa[2] - (double)ka[2], c0 = (double)sb[0] - (double)kb[0],
                         c1 = (double)sb[1] - (double)kb[1], c2 = (double)sb[2] - (double)kb[2];
            // each (batch, lane) target holds one slot per leaf: no two lanes
            // add to the same accumulator here
            if (v1) {
                sc.acc[id1 >> 5][0][id1 & 31] += a0;
                sc.acc[id1 >> 5][1][id1 & 31] += a1;
                sc.acc[id1 >> 5][2][id1 & 31] += a2;
            }
            if (v2) {
                sc.acc[id2 >> 5][0][id2 & 31] += c0;
                sc.acc[id2 >> 5][1][id2 & 31] += c1;
                sc.acc[id2 >> 5][2][id2 & 31] += c2;
            }
        }
        if (match) {
            if (++cur < end) {
                le = near_list[cur];
                key = topo[le.node].x;
            } else {
                key = kEnd;
            }
        }
    }
    __syncwarp();
#pragma unroll
    for (int g = 0; g < G; g++) {
        const int64_t mm = (b0 + g) * kBatch + lane;
        if (mm < M)
            for (int c = 0; c < 3; c++) {
                if (Op::kAdd)
                    out[c * M + mm] += sc.acc[g][c][lane];
                else
                    out[c * M + mm] = sc.acc[g][c][lane];
            }
    }
}

// ---------------------------------------------------------------------------
// Scheduling of the groups over a resident grid (the one-system near field and
// the target side of its adjoint).  A grid one block per SM short of the
// occupancy limit drains a queue of groups; when the groups outnumber its
// warps, they are taken in order of decreasing work (k_group_work + radix
// sort), so each warp drains several and the end of the kernel is made of the
// smallest ones.  Measured at N = 10^6 (near kernel alone / step): groups of
// eight at full occupancy 37.4 / 53.0 ms, eight one block short 35.7 / 53.1,
// four at full occupancy 34.2 / 54.3, four one block short 33.3 / 54.1, four
// two blocks short 34.4 / 54.4.

constexpr int kQueueWarps = 4;       // warps per block of the queued kernels
constexpr int kQueueFreeBlocks = 1;  // block slots per SM left free

// Work of each group of G batches, its pair count (over its near entries, the
// active targets times the leaf size), as a sort key that puts the groups
// with the most work first; order receives the identity.
template <int G>
__global__ void k_group_work(const int64_t* __restrict__ near_off, const ListEntry* __restrict__ near_list,
                             const int4* __restrict__ topo, int64_t nbatch, int64_t ngroup, uint64_t* __restrict__ keys,
                             int32_t* __restrict__ order)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= ngroup) return;
    const int64_t b0 = g * G, b1 = min(nbatch, b0 + G);
    uint64_t w = 0;
    for (int64_t e = near_off[b0]; e < near_off[b1]; e++) {
        const ListEntry le = near_list[e];
        w += (uint64_t)__popc(le.mask) * (uint64_t)topo[le.node].y;
    }
    keys[g] = 0xffffffffull - (w < 0xffffffffull ? w : 0xffffffffull);
    order[g] = (int32_t)g;
}

// Each warp takes the next group from the queue: order[i], or i when order is
// NULL (the grid holds every group at once).
template <int G, typename Op>
__global__ void __launch_bounds__(kQueueWarps * 32)
    k_near_queue(const double* __restrict__ ts, const double* __restrict__ gs, int64_t M,
                 const int4* __restrict__ topo, const float4* __restrict__ spack, const int64_t* __restrict__ near_off,
                 const ListEntry* __restrict__ near_list, double* __restrict__ out, int self, float prm,
                 const int32_t* __restrict__ order, int64_t ngroup, unsigned* __restrict__ queue)
{
    __shared__ NearScratch<G> sc[kQueueWarps];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        unsigned i = 0;
        if (lane == 0) i = atomicAdd(queue, 1u);
        i = __shfl_sync(0xffffffffu, i, 0);
        if ((int64_t)i >= ngroup) break;
        near_group<G, Op>(ts, gs, M, topo, spack, near_off, near_list, out, order ? order[i] : i, self, prm, sc[w],
                          lane);
    }
}

// blocks of k_near_queue<G, Op> the grid takes: the occupancy limit less
// kQueueFreeBlocks per SM, times the SMs
template <int G, typename Op>
int64_t queue_resident_blocks()
{
    static int ps = 0, sms = 0;
    if (ps == 0) {
        int dev = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_near_queue<G, Op>, kQueueWarps * 32, 0) !=
                cudaSuccess ||
            ps < 1)
            ps = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return (int64_t)(ps > kQueueFreeBlocks ? ps - kQueueFreeBlocks : 1) * (sms > 0 ? sms : 1);
}

template <int G, typename Op>
cudaError_t run_near_queue(const double* ts, const double* gs, int64_t M, const int4* topo, const float4* spack,
                           const int64_t* near_off, const ListEntry* near_list, double* out, int self, float prm,
                           const NearSched& sc, cudaStream_t s)
{
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t ngroup = (nbatch + G - 1) / G;
    const int64_t need = (ngroup + kQueueWarps - 1) / kQueueWarps;
    const int64_t resident = queue_resident_blocks<G, Op>();
    const unsigned grid = (unsigned)(need < resident ? need : resident);
    // the order matters only when some warps take more than one group
    const int32_t* order = nullptr;
    if (need > resident) {
        k_group_work<G><<<(unsigned)((ngroup + 255) / 256), 256, 0, s>>>(near_off, near_list, topo, nbatch, ngroup,
                                                                        sc.keys, sc.order);
        note_launch();
        cudaError_t e = radix_sort_bits(sc.keys, sc.order, sc.keys_alt, sc.order_alt, sc.hist, ngroup, 32, s);
        if (e != cudaSuccess) return e;
        order = sc.order;
    }
    cudaError_t e = cudaMemsetAsync(sc.queue, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    k_near_queue<G, Op><<<grid, kQueueWarps * 32, 0, s>>>(ts, gs, M, topo, spack, near_off, near_list, out, self, prm,
                                                           order, ngroup, sc.queue);
    note_launch();
    return cudaGetLastError();
}

// Groups of four batches when there are at least kQueueMinGroups of them per
// warp of the grid, else groups of two (more, smaller groups, so that the
// queue can still balance the warps of a smaller or more uneven problem).
constexpr int kQueueMinGroups = 2;

template <typename Op>
cudaError_t run_near_auto(const double* ts, const double* gs, int64_t M, const int4* topo, const float4* spack,
                          const int64_t* near_off, const ListEntry* near_list, double* out, int self, float prm,
                          const NearSched& sc, cudaStream_t s)
{
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    if ((nbatch + 3) / 4 >= kQueueMinGroups * kQueueWarps * queue_resident_blocks<4, Op>())
        return run_near_queue<4, Op>(ts, gs, M, topo, spack, near_off, near_list, out, self, prm, sc, s);
    return run_near_queue<2, Op>(ts, gs, M, topo, spack, near_off, near_list, out, self, prm, sc, s);
}

}  // namespace nearpair
}  // namespace tc
