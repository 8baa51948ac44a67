// Tree construction (Section 5): root cube, 21-bit quantisation, Morton keys,
// a hand-written stable LSD radix sort, level-synchronous octree topology and
// cluster geometry (centre y_c and squared radius r^2, Section 2).
//
// Every floating-point step that decides tree membership or a MAC outcome is
// written with explicit round-to-nearest intrinsics (__dsub_rn, __dmul_rn,
// __dadd_rn) so that no multiply-add is contracted and the tree is
// reproducible bit for bit.
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kBboxThreads = 256;

__device__ inline double warp_min(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Per-block min/max of each axis; non-finite inputs poison the block result
// with NaN so that the host can reject them.
__global__ void k_bbox_partial(const double* __restrict__ x, int64_t N, double* __restrict__ part)
{
    __shared__ double sm[6][kBboxThreads / 32];
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; a++) {
            double v = x[a * N + i];
            bad |= !isfinite(v);
            mn[a] = fmin(mn[a], v);
            mx[a] = fmax(mx[a], v);
        }
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    bad = __any_sync(0xffffffffu, bad);
    for (int a = 0; a < 3; a++) {
        double a0 = warp_min(mn[a]), a1 = warp_max(mx[a]);
        if (lane == 0) {
            sm[a][w] = bad ? NAN : a0;
            sm[3 + a][w] = bad ? NAN : a1;
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        int c = threadIdx.x;
        double v = sm[c][0];
        bool nan = isnan(v);
        for (int k = 1; k < kBboxThreads / 32; k++) {
            nan |= isnan(sm[c][k]);
            v = c < 3 ? fmin(v, sm[c][k]) : fmax(v, sm[c][k]);
        }
        part[blockIdx.x * 6 + c] = nan ? NAN : v;
    }
}

// root[0..2] = per-axis minimum, root[3] = side (largest extent),
// root[4] = 2^21 / side (0 if side == 0), root[5] = 1 if an input was not finite.
// One block of kBboxThreads: strided partial min/max, then a block reduction.
__global__ void __launch_bounds__(kBboxThreads) k_bbox_final(const double* __restrict__ part, int nblk,
                                                              double* __restrict__ root)
{
    __shared__ double sm[6][kBboxThreads / 32];
    __shared__ int sbad;
    double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x)
        for (int a = 0; a < 3; a++) {
            double v0 = part[b * 6 + a], v1 = part[b * 6 + 3 + a];
            bad |= isnan(v0) || isnan(v1);
            mn[a] = fmin(mn[a], v0);
            mx[a] = fmax(mx[a], v1);
        }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (__any_sync(0xffffffffu, bad) && lane == 0) sbad = 1;
    for (int a = 0; a < 3; a++) {
        double a0 = warp_min(mn[a]), a1 = warp_max(mx[a]);
        if (lane == 0) {
            sm[a][w] = a0;
            sm[3 + a][w] = a1;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int k = 1; k < kBboxThreads / 32; k++)
        for (int a = 0; a < 3; a++) {
            sm[a][0] = fmin(sm[a][0], sm[a][k]);
            sm[3 + a][0] = fmax(sm[3 + a][0], sm[3 + a][k]);
        }
    double side = 0.0;
    for (int a = 0; a < 3; a++) {
        double e = __dsub_rn(sm[3 + a][0], sm[a][0]);
        if (e > side) side = e;
    }
    root[0] = sm[0][0];
    root[1] = sm[1][0];
    root[2] = sm[2][0];
    root[3] = side;
    root[4] = side > 0.0 ? 2097152.0 / side : 0.0;
    root[5] = sbad ? 1.0 : 0.0;
}

// 21-bit spread: bit j of v goes to bit 3j.
__device__ inline uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ inline uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffffull;
    return (uint32_t)x;
}

// q_a = min(2^21 - 1, floor((x_a - lo_a) * 2^21 / side)); key interleaves the
// bits of q with x most significant inside each 3-bit octant digit.
__global__ void k_keys(const double* __restrict__ x, int64_t N, const double* __restrict__ root,
                       uint64_t* __restrict__ keys, int32_t* __restrict__ idx, int clamp_outside)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double scale = root[4];
    uint32_t q[3];
    for (int a = 0; a < 3; a++) {
        double v = floor(__dmul_rn(__dsub_rn(x[a * N + i], root[a]), scale));
        if (v > 2097151.0) v = 2097151.0;
        if (clamp_outside && !(v >= 0.0)) v = 0.0;
        q[a] = (uint32_t)v;
    }
    keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    idx[i] = (int32_t)i;
}

// ---------------------------------------------------------------- radix sort
// Stable LSD sort of 64-bit keys carrying int32 values, 8 passes of 8 bits.
// A block owns a tile of 2048 keys; warp w owns items w*256 + i*32 + lane
// (i = 0..7), so (warp, i, lane) order equals index order and the ranking
// below is stable.
constexpr int kRadixThreads = 256;
constexpr int kRadixItems = 8;
constexpr int kRadixTile = kRadixThreads * kRadixItems;

__global__ void k_radix_hist(const uint64_t* __restrict__ keys, int64_t N, int shift, uint32_t* __restrict__ hist)
{
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = 0; i < kRadixItems; i++) {
        int64_t g = base + w * 256 + i * 32 + lane;
        if (g < N) atomicAdd(&cnt[(keys[g] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = cnt[threadIdx.x];
}


__global__ void k_radix_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                uint64_t* __restrict__ kout, int32_t* __restrict__ vout, int64_t N, int shift,
                                const uint32_t* __restrict__ hist)
{
    __shared__ uint32_t wcnt[kRadixThreads / 32][256];
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int d = lane; d < 256; d += 32) wcnt[w][d] = 0;
    __syncwarp();
    int64_t base = (int64_t)blockIdx.x * kRadixTile;
    uint32_t rank[kRadixItems];
    int digit[kRadixItems];
    uint64_t key[kRadixItems];
    int32_t val[kRadixItems];
    const unsigned lt = (1u << lane) - 1u;
    for (int i = 0; i < kRadixItems; i++) {
        int64_t g = base + w * 256 + i * 32 + lane;
        bool valid = g < N;
        key[i] = valid ? kin[g] : 0;
        val[i] = valid ? vin[g] : 0;
        int dg = valid ? (int)((key[i] >> shift) & 255u) : 256;
        unsigned peers = __match_any_sync(0xffffffffu, dg);
        uint32_t before = valid ? wcnt[w][dg] : 0;
        __syncwarp();
        int leader = __ffs(peers) - 1;
        if (valid && lane == leader) wcnt[w][dg] = before + __popc(peers);
        __syncwarp();
        rank[i] = before + __popc(peers & lt);
        digit[i] = dg;
    }
    __syncthreads();
    {
        int d = threadIdx.x;  // one digit per thread
        uint32_t run = 0;
        for (int ww = 0; ww < kRadixThreads / 32; ww++) {
            uint32_t c = wcnt[ww][d];
            wcnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int i = 0; i < kRadixItems; i++) {
        if (digit[i] == 256) continue;
        int64_t pos = (int64_t)hist[(int64_t)digit[i] * gridDim.x + blockIdx.x] + wcnt[w][digit[i]] + rank[i];
        kout[pos] = key[i];
        vout[pos] = val[i];
    }
}

__global__ void k_gather3(const double* __restrict__ src, const int32_t* __restrict__ perm, int64_t N,
                          double* __restrict__ dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    int64_t j = perm[i];
    dst[i] = src[j];
    dst[N + i] = src[N + j];
    dst[2 * N + i] = src[2 * N + j];
}

// ---------------------------------------------------------------- topology
__global__ void k_init_root(int4* topo, int4* info, uint64_t* nkey, int64_t N)
{
    topo[0] = make_int4(0, (int)N, -1, 0);
    info[0] = make_int4(0, -1, 0, 0);
    nkey[0] = 0;
}

__device__ inline int octant_at(uint64_t key, int shift) { return (int)((key >> shift) & 7u); }

// first index in [lo, hi) whose octant digit is >= o (digits are sorted)
__device__ inline int lower_digit(const uint64_t* keys, int lo, int hi, int shift, int o)
{
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        if (octant_at(keys[mid], shift) < o)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_split_count(const int4* __restrict__ topo, const int4* __restrict__ info,
                              const uint64_t* __restrict__ keys, int64_t lb, int64_t le, int N0,
                              int32_t* __restrict__ cnt)
{
    int64_t id = lb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= le) return;
    int4 t = topo[id];
    int lvl = info[id].x;
    int c = 0;
    if (t.y > N0 && lvl < kMaxDepth) {
        int shift = 63 - 3 * (lvl + 1);
        int b = t.x, e = t.x + t.y;
        int prev = b;
        for (int o = 1; o <= 8; o++) {
            int s = o < 8 ? lower_digit(keys, b, e, shift, o) : e;
            c += s > prev;
            prev = s;
        }
    }
    cnt[id - lb] = c;
}

__global__ void k_split_write(int4* __restrict__ topo, int4* __restrict__ info, uint64_t* __restrict__ nkey,
                              const uint64_t* __restrict__ keys, int64_t lb, int64_t le, int N0,
                              const int32_t* __restrict__ off)
{
    int64_t id = lb + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= le) return;
    int4 t = topo[id];
    int lvl = info[id].x;
    if (!(t.y > N0 && lvl < kMaxDepth)) return;
    int shift = 63 - 3 * (lvl + 1);
    int b = t.x, e = t.x + t.y;
    int64_t fc = le + off[id - lb];
    int j = 0, prev = b;
    for (int o = 1; o <= 8; o++) {
        int s = o < 8 ? lower_digit(keys, b, e, shift, o) : e;
        if (s > prev) {
            int64_t c = fc + j++;
            topo[c] = make_int4(prev, s - prev, -1, 0);
            info[c] = make_int4(lvl + 1, (int)id, 0, 0);
            nkey[c] = nkey[id] | ((uint64_t)(o - 1) << shift);
        }
        prev = s;
    }
    topo[id].z = (int)fc;
    topo[id].w = j;
}

// ---------------------------------------------------------------- geometry
constexpr int kGeoThreads = 256;

__device__ inline double block_reduce(double v, bool is_max, double* sm)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = is_max ? warp_max(v) : warp_min(v);
    __syncthreads();
    if (lane == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < kGeoThreads / 32 ? sm[lane] : (is_max ? -INFINITY : INFINITY);
        v = is_max ? warp_max(v) : warp_min(v);
        if (lane == 0) sm[0] = v;
    }
    __syncthreads();
    return sm[0];
}

// Cluster geometry: centre (tight box or cell centre) and r^2 = max |y - y_c|^2.
// The work is split into items of at most kGeoChunk particles of one cluster,
// so that the large clusters near the root are spread over the whole GPU;
// per-item partial results are combined with atomic min/max, which are exact
// (the result does not depend on the order), on order-preserving integer
// images of the doubles.
constexpr int kGeoChunk = 2048;

// double -> uint64 with the same order (a negative value's bits inverted, a
// non-negative value's sign bit set)
__device__ inline unsigned long long dorder(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ inline double dunorder(unsigned long long k)
{
    return __longlong_as_double((long long)((k >> 63) ? (k ^ 0x8000000000000000ull) : ~k));
}

// items per cluster; reset of the per-cluster accumulators
__global__ void k_geo_items(const int4* __restrict__ topo, int64_t nnodes, int32_t* __restrict__ cnt,
                            unsigned long long* __restrict__ acc)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nnodes) return;
    cnt[id] = (topo[id].y + kGeoChunk - 1) / kGeoChunk;
    unsigned long long* a = acc + id * 7;
    for (int c = 0; c < 3; c++) {
        a[c] = dorder(INFINITY);       // min
        a[3 + c] = dorder(-INFINITY);  // max
    }
    a[6] = 0ull;  // r^2 >= 0: its bits order like the value
}

// item -> (cluster, particle range)
__device__ inline int64_t geo_item(const int4* __restrict__ topo, const int32_t* __restrict__ item_off,
                                   int64_t nnodes, int item, int& b, int& e)
{
    int64_t lo = 0, hi = nnodes;  // item_off[lo] <= item < item_off[hi]
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (item_off[mid] <= item)
            lo = mid;
        else
            hi = mid;
    }
    const int4 t = topo[lo];
    b = t.x + (item - item_off[lo]) * kGeoChunk;
    e = min(b + kGeoChunk, t.x + t.y);
    return lo;
}

__global__ void __launch_bounds__(kGeoThreads)
    k_geo_box(const int4* __restrict__ topo, const int32_t* __restrict__ item_off, const int32_t* __restrict__ nitems,
              int64_t nnodes, const double* __restrict__ xs, int64_t N, unsigned long long* __restrict__ acc)
{
    __shared__ double sm[kGeoThreads / 32];
    const int total = *nitems;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int b, e;
        const int64_t id = geo_item(topo, item_off, nnodes, item, b, e);
        for (int a = 0; a < 3; a++) {
            double mn = INFINITY, mx = -INFINITY;
            for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
                const double v = xs[a * N + i];
                mn = fmin(mn, v);
                mx = fmax(mx, v);
            }
            mn = block_reduce(mn, false, sm);
            mx = block_reduce(mx, true, sm);
            if (threadIdx.x == 0) {
                atomicMin(acc + id * 7 + a, dorder(mn));
                atomicMax(acc + id * 7 + 3 + a, dorder(mx));
            }
        }
    }
}

// centre of each cluster (tight box or cell centre)
__global__ void k_geo_centre(const int4* __restrict__ info, const uint64_t* __restrict__ nkey, int64_t nnodes,
                             const double* __restrict__ root, int shrink, const unsigned long long* __restrict__ acc,
                             Geo* __restrict__ geo)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nnodes) return;
    double yc[3];
    if (shrink) {
        for (int a = 0; a < 3; a++)
            yc[a] = __dmul_rn(__dadd_rn(dunorder(acc[id * 7 + a]), dunorder(acc[id * 7 + 3 + a])), 0.5);
    } else {
        const int L = info[id].x;
        const uint64_t k = nkey[id];
        const uint32_t c[3] = {compact3(k >> 2) >> (kMaxDepth - L), compact3(k >> 1) >> (kMaxDepth - L),
                               compact3(k) >> (kMaxDepth - L)};
        const double cs = ldexp(root[3], -L);
        for (int a = 0; a < 3; a++) yc[a] = __dadd_rn(root[a], __dmul_rn((double)c[a] + 0.5, cs));
    }
    geo[id] = Geo{yc[0], yc[1], yc[2], 0.0};
}

__global__ void __launch_bounds__(kGeoThreads)
    k_geo_r2(const int4* __restrict__ topo, const int32_t* __restrict__ item_off, const int32_t* __restrict__ nitems,
             int64_t nnodes, const double* __restrict__ xs, int64_t N, const Geo* __restrict__ geo,
             unsigned long long* __restrict__ acc)
{
    __shared__ double sm[kGeoThreads / 32];
    const int total = *nitems;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int b, e;
        const int64_t id = geo_item(topo, item_off, nnodes, item, b, e);
        const Geo g = geo[id];
        double r2 = 0.0;
        for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
            const double dx = __dsub_rn(xs[i], g.x), dy = __dsub_rn(xs[N + i], g.y), dz = __dsub_rn(xs[2 * N + i], g.z);
            const double s = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            r2 = fmax(r2, s);
        }
        r2 = block_reduce(r2, true, sm);
        if (threadIdx.x == 0) atomicMax(acc + id * 7 + 6, (unsigned long long)__double_as_longlong(r2));
    }
}

// r^2, 1/rho, and the FP32 copy of the geometry used by the MAC screen of
// the list traversal: (fl32(y_c), fl32(r^2)) and (fl32(y_c - fl32(y_c)), 0)
__global__ void k_geo_final(int64_t nnodes, const unsigned long long* __restrict__ acc, Geo* __restrict__ geo,
                            double* __restrict__ invrho, float4* __restrict__ geof)
{
    const int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (id >= nnodes) return;
    const double r2 = __longlong_as_double((long long)acc[id * 7 + 6]);
    Geo g = geo[id];
    g.w = r2;
    geo[id] = g;
    invrho[id] = r2 > 0.0 ? 1.0 / sqrt(r2) : 1.0;
    const float hx = __double2float_rn(g.x), hy = __double2float_rn(g.y), hz = __double2float_rn(g.z);
    geof[2 * id] = make_float4(hx, hy, hz, __double2float_rn(r2));
    geof[2 * id + 1] = make_float4(__double2float_rn(g.x - (double)hx), __double2float_rn(g.y - (double)hy),
                                   __double2float_rn(g.z - (double)hz), 0.0f);
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_bbox(const double* x, int64_t N, double* part, int nblk, double* root, cudaStream_t s)
{
    k_bbox_partial<<<nblk, kBboxThreads, 0, s>>>(x, N, part);
    note_launch();
    k_bbox_final<<<1, kBboxThreads, 0, s>>>(part, nblk, root);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_keys(const double* x, int64_t N, const double* root, uint64_t* keys, int32_t* idx,
                        int clamp_outside, cudaStream_t s)
{
    k_keys<<<grid_for(N, 256), 256, 0, s>>>(x, N, root, keys, idx, clamp_outside);
    note_launch();
    return cudaGetLastError();
}

int radix_blocks(int64_t N) { return (int)((N + kRadixTile - 1) / kRadixTile); }

cudaError_t radix_sort(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, uint32_t* hist,
                       int64_t N, cudaStream_t s)
{
    return radix_sort_bits(keys, vals, keys_alt, vals_alt, hist, N, 64, s);
}

// Sort on the low `bits` key bits only (an even number of 8-bit passes, so
// the result always ends in keys/vals).
cudaError_t radix_sort_bits(uint64_t* keys, int32_t* vals, uint64_t* keys_alt, int32_t* vals_alt, uint32_t* hist,
                            int64_t N, int bits, cudaStream_t s)
{
    int nblk = radix_blocks(N);
    if (nblk < 1) return cudaSuccess;
    int passes = (bits + 7) / 8;
    passes += passes & 1;
    if (passes > 8) passes = 8;
    uint64_t *ki = keys, *ko = keys_alt;
    int32_t *vi = vals, *vo = vals_alt;
    for (int pass = 0; pass < passes; pass++) {
        int shift = 8 * pass;
        k_radix_hist<<<nblk, kRadixThreads, 0, s>>>(ki, N, shift, hist);
        note_launch();
        k_scan_tiles<uint32_t, uint32_t><<<1, 1024, 0, s>>>(hist, hist, (int64_t)256 * nblk, nullptr);
        note_launch();
        k_radix_scatter<<<nblk, kRadixThreads, 0, s>>>(ki, vi, ko, vo, N, shift, hist);
        note_launch();
        uint64_t* tk = ki;
        ki = ko;
        ko = tk;
        int32_t* tv = vi;
        vi = vo;
        vo = tv;
    }
    return cudaGetLastError();  // even number of passes: result is back in keys/vals
}

cudaError_t launch_gather3(const double* src, const int32_t* perm, int64_t N, double* dst, cudaStream_t s)
{
    k_gather3<<<grid_for(N, 256), 256, 0, s>>>(src, perm, N, dst);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_init_root(int4* topo, int4* info, uint64_t* nkey, int64_t N, cudaStream_t s)
{
    k_init_root<<<1, 1, 0, s>>>(topo, info, nkey, N);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_split_count(const int4* topo, const int4* info, const uint64_t* keys, int64_t lb, int64_t le,
                               int N0, int32_t* cnt, cudaStream_t s)
{
    k_split_count<<<grid_for(le - lb, 128), 128, 0, s>>>(topo, info, keys, lb, le, N0, cnt);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_scan_i32(const int32_t* in, int32_t* out_excl, int64_t n, int32_t* total, cudaStream_t s)
{
    k_scan_tiles<int32_t, int32_t><<<1, 1024, 0, s>>>(in, out_excl, n, total);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_split_write(int4* topo, int4* info, uint64_t* nkey, const uint64_t* keys, int64_t lb, int64_t le,
                               int N0, const int32_t* off, cudaStream_t s)
{
    k_split_write<<<grid_for(le - lb, 128), 128, 0, s>>>(topo, info, nkey, keys, lb, le, N0, off);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_geometry(const int4* topo, const int4* info, const uint64_t* nkey, const double* xs, int64_t N,
                            int64_t nnodes, const double* root, int shrink, Geo* geo, double* invrho, float4* geof,
                            void* scratch, cudaStream_t s)
{
    // scratch: acc [nnodes][7] u64, cnt [nnodes] i32, item_off [nnodes] i32, nitems i32
    unsigned long long* acc = static_cast<unsigned long long*>(scratch);
    int32_t* cnt = reinterpret_cast<int32_t*>(acc + nnodes * 7);
    int32_t* item_off = cnt + nnodes;
    int32_t* nitems = item_off + nnodes;
    k_geo_items<<<grid_for(nnodes, 256), 256, 0, s>>>(topo, nnodes, cnt, acc);
    note_launch();
    cudaError_t e = launch_scan_i32(cnt, item_off, nnodes, nitems, s);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)(sms > 0 ? sms : 1) * 4;
    k_geo_box<<<grid, kGeoThreads, 0, s>>>(topo, item_off, nitems, nnodes, xs, N, acc);
    note_launch();
    k_geo_centre<<<grid_for(nnodes, 256), 256, 0, s>>>(info, nkey, nnodes, root, shrink, acc, geo);
    note_launch();
    k_geo_r2<<<grid, kGeoThreads, 0, s>>>(topo, item_off, nitems, nnodes, xs, N, geo, acc);
    note_launch();
    k_geo_final<<<grid_for(nnodes, 256), 256, 0, s>>>(nnodes, acc, geo, invrho, geof);
    note_launch();
    return cudaGetLastError();
}

size_t geometry_scratch_bytes(int64_t nnodes) { return (size_t)nnodes * 7 * 8 + (size_t)(2 * nnodes + 1) * 4; }

}  // namespace tc
