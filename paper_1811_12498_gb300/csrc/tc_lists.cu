// MAC traversal (Algorithm 1, eq. 5.1) producing per-batch interaction lists.
//
// A batch is 32 consecutive Morton-ordered targets, one per lane of a warp.
// The warp walks the tree with an explicit stack of (cluster, lane mask)
// entries.  At a cluster every lane still in the mask tests its own MAC in
// FP64; the lanes that pass get a far-field entry, the lanes that fail
// descend (or get a near-field entry at a leaf).  Each target therefore meets
// exactly the clusters, and makes exactly the decisions, of Algorithm 1 run on
// its own.  Children are pushed so that they are visited in octant order.
//
// The MAC R^2 > 0 && r_c^2 <= theta^2 R^2 is decided in FP64 exactly as the
// definition reads (every operation rounded to nearest), but most decisions
// are settled by an FP32 screen first: R^2 from FP32 hi/lo splits of the
// target and the centre has a relative error below 2e-6 whenever
// |x - y_c| >= 1e-7 S (S bounds the coordinates' magnitude), so a screened
// ratio theta^2 R^2 / r_c^2 farther than 2^-12 from 1 gives the FP64 answer;
// the rest (near-ties, and centres within 1e-7 S of the target) are decided
// in FP64.  The decisions, and so the lists, are those of the FP64 test.
//
// The kernel runs twice: once to count entries per batch, once (after an
// exclusive scan of the counts) to write them.
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kListWarps = 4;

__global__ void __launch_bounds__(kListWarps * 32, 12)
    k_lists(const double* __restrict__ ts, int64_t M, const int4* __restrict__ topo,
            const Geo* __restrict__ geo, const float4* __restrict__ geof, float tiny2, float th2f, double theta2,
            int write, int32_t* __restrict__ nfar_e,
            int32_t* __restrict__ nnear_e, const int64_t* __restrict__ far_off, const int64_t* __restrict__ near_off,
            ListEntry* __restrict__ far_list, ListEntry* __restrict__ near_list, int64_t* __restrict__ cnt_far,
            int64_t* __restrict__ cnt_near, int32_t* __restrict__ flags)
{
    __shared__ ListEntry stack[kListWarps][kStack];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    const int64_t b = blockIdx.x * (int64_t)kListWarps + w;
    if (b >= nbatch) return;
    const int64_t m = b * kBatch + lane;
    const bool valid = m < M;
    float xh0, xh1, xh2, xl0, xl1, xl2;
    {
        double x0 = 0, x1 = 0, x2 = 0;
        if (valid) {
            x0 = ts[m];
            x1 = ts[M + m];
            x2 = ts[2 * M + m];
        }
        xh0 = __double2float_rn(x0), xh1 = __double2float_rn(x1), xh2 = __double2float_rn(x2);
        xl0 = __double2float_rn(x0 - (double)xh0), xl1 = __double2float_rn(x1 - (double)xh1),
        xl2 = __double2float_rn(x2 - (double)xh2);
    }
    ListEntry* st = stack[w];
    int sp = 0;
    const unsigned active = __ballot_sync(0xffffffffu, valid);
    if (lane == 0) st[0] = ListEntry{0, active};
    sp = 1;
    __syncwarp();
    // 32-bit counters: entries per batch and interactions per target are all
    // below N < 2^31 (64-bit ones made this kernel measurably slower)
    int nf = 0, nn = 0, my_far = 0, my_near = 0;
    const int64_t fo = write ? far_off[b] : 0, no = write ? near_off[b] : 0;
    bool overflow = false;
    while (sp > 0) {
        ListEntry e = st[--sp];
        __syncwarp();
        int4 t = topo[e.node];
        bool in = (e.mask >> lane) & 1u;
        const float4 gh = geof[2 * (int64_t)e.node], gl = geof[2 * (int64_t)e.node + 1];
        const float fx = (xh0 - gh.x) + (xl0 - gl.x), fy = (xh1 - gh.y) + (xl1 - gl.y),
                    fz = (xh2 - gh.z) + (xl2 - gl.z);
        const float R2f = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
        const float q = th2f * R2f;
        const bool screened = R2f > tiny2 && q < 1e37f && gh.w < 1e37f;  // far from FP32 under/overflow
        bool pass = screened && q >= gh.w * (1.0f + 0x1p-12f);
        const bool sure = screened && (pass || q <= gh.w * (1.0f - 0x1p-12f));
        // warp-uniform guard: the FP64 test is rare, and issued predicated for
        // the whole warp it would keep the FP64 pipe busy on every visit
        if (__any_sync(0xffffffffu, in && !sure) && in && !sure) {
            // the FP64 coordinates are reloaded here rather than kept live
            // through the walk: with them live the pass took 1.1 ms at
            // N = 10^6, reloaded (and 12 blocks per SM) 0.6 ms
            const Geo g = geo[e.node];
            const double x0 = ts[m], x1 = ts[M + m], x2 = ts[2 * M + m];
            double dx = __dsub_rn(x0, g.x), dy = __dsub_rn(x1, g.y), dz = __dsub_rn(x2, g.z);
            double R2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            pass = (R2 > 0.0) && (g.w <= __dmul_rn(theta2, R2));
        }
        pass = pass && in;
        unsigned pm = __ballot_sync(0xffffffffu, pass);
        unsigned fm = e.mask & ~pm;
        if (pm) {
            if (write && lane == 0) far_list[fo + nf] = ListEntry{e.node, pm};
            nf++;
            my_far += pass;
        }
        if (fm) {
            if (t.w == 0) {
                if (write && lane == 0) near_list[no + nn] = ListEntry{e.node, fm};
                nn++;
                if (in && !pass) my_near += t.y;
            } else {
                if (sp + t.w > kStack) {
                    overflow = true;
                    break;
                }
                if (lane == 0)
                    for (int c = t.w - 1; c >= 0; c--) st[sp + (t.w - 1 - c)] = ListEntry{t.z + c, fm};
                sp += t.w;
            }
        }
        __syncwarp();
    }
    if (overflow && lane == 0) atomicOr(flags, kFlagStack);
    if (!write && lane == 0) {
        nfar_e[b] = (int32_t)nf;
        nnear_e[b] = (int32_t)nn;
    }
    if (valid && cnt_far) {
        cnt_far[m] = my_far;
        cnt_near[m] = my_near;
    }
}


__global__ void k_sum_i64(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out)
{
    __shared__ int64_t part[1024];
    int64_t s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += in[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// sum over list entries of the entry's cluster size
__global__ void k_sum_entry_sizes(const ListEntry* __restrict__ list, int64_t n, const int4* __restrict__ topo,
                                  int64_t* __restrict__ out)
{
    __shared__ int64_t part[1024];
    int64_t s = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += topo[list[i].node].y;
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0];
}

// cluster of each list entry as its sort key, and the identity
__global__ void k_entry_keys(const ListEntry* __restrict__ list, int64_t n, uint64_t* __restrict__ keys,
                             int32_t* __restrict__ idx)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    keys[i] = (uint64_t)(uint32_t)list[i].node;
    idx[i] = (int32_t)i;
}

// batch of each list entry: largest b with off[b] <= e
__global__ void k_entry_batch(const int64_t* __restrict__ off, int64_t nbatch, int64_t n, int32_t* __restrict__ eb)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    int64_t lo = 0, hi = nbatch;  // off[lo] <= e < off[hi]
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    eb[e] = (int32_t)lo;
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t sort_list_entries(const ListEntry* list, int64_t n, const int64_t* off, int64_t nbatch, int64_t nnodes,
                              DevBuf& keys, DevBuf& keys_alt, DevBuf& idx, DevBuf& idx_alt, DevBuf& eb,
                              DevBuf& hist, cudaStream_t s)
{
    cudaError_t e;
    if ((e = ensure(keys, (size_t)n * 8)) != cudaSuccess) return e;
    if ((e = ensure(keys_alt, (size_t)n * 8)) != cudaSuccess) return e;
    if ((e = ensure(idx, (size_t)n * 4)) != cudaSuccess) return e;
    if ((e = ensure(idx_alt, (size_t)n * 4)) != cudaSuccess) return e;
    if ((e = ensure(eb, (size_t)n * 4)) != cudaSuccess) return e;
    if ((e = ensure(hist, (size_t)256 * radix_blocks(n) * 4)) != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    k_entry_keys<<<grid_for(n, 256), 256, 0, s>>>(list, n, ptr<uint64_t>(keys), ptr<int32_t>(idx));
    note_launch();
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) < nnodes) bits++;
    e = radix_sort_bits(ptr<uint64_t>(keys), ptr<int32_t>(idx), ptr<uint64_t>(keys_alt), ptr<int32_t>(idx_alt),
                        ptr<uint32_t>(hist), n, bits, s);
    if (e != cudaSuccess) return e;
    k_entry_batch<<<grid_for(n, 256), 256, 0, s>>>(off, nbatch, n, ptr<int32_t>(eb));
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_entry_sizes(const ListEntry* list, int64_t n, const int4* topo, int64_t* out, cudaStream_t s)
{
    k_sum_entry_sizes<<<1, 1024, 0, s>>>(list, n, topo, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_lists(const double* ts, int64_t M, const int4* topo, const Geo* geo, const float4* geof,
                         float scale2, double theta, int write, int32_t* nfar_e, int32_t* nnear_e,
                         const int64_t* far_off, const int64_t* near_off, ListEntry* far_list, ListEntry* near_list,
                         int64_t* cnt_far, int64_t* cnt_near, int32_t* flags, cudaStream_t s)
{
    int64_t nbatch = (M + kBatch - 1) / kBatch;
    unsigned grid = (unsigned)((nbatch + kListWarps - 1) / kListWarps);
    double theta2 = theta * theta;
    // screen only where |x - y_c|^2 > 1e-14 S^2 (and R^2 is a normal FP32 number)
    const float tiny2 = fmaxf(1e-14f * scale2, 1e-30f);
    k_lists<<<grid, kListWarps * 32, 0, s>>>(ts, M, topo, geo, geof, tiny2, (float)theta2, theta2, write, nfar_e,
                                             nnear_e, far_off, near_off, far_list, near_list, cnt_far, cnt_near,
                                             flags);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scan_i32_to_i64(const int32_t* in, int64_t* out_excl, int64_t n, int64_t* total,
                                   cudaStream_t s)
{
    k_scan_tiles<int32_t, int64_t><<<1, 1024, 0, s>>>(in, out_excl, n, total);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum_i64(const int64_t* in, int64_t n, int64_t* out, cudaStream_t s)
{
    k_sum_i64<<<1, 1024, 0, s>>>(in, n, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc
