// Direct O(N*M) evaluation of eq. (1.3) in the contracted form of
// Section 4.1 (the reference u^d of eq. 6.1 for the error E), and of the same
// sum with the regularized kernels (kReg; the blob of Cortez, Fauci and
// Medovikov, s = r^2 + eps^2, q = s^-1/2):
//   u_i += f_i q (1 + eps^2 q^2) + d_i q^3 ((d.f) + q^2 ((d.h)(d.nu) + (eps^2/2)(h.nu)))
//          + (eps^2/2) q^5 (h_i (d.nu) + nu_i (d.h)).
//
// Warps own 32 targets; the source range is split into `nsplit` chunks along
// gridDim.y so that few targets (e.g. 10^4 sampled targets against 10^6
// sources) still fill the GPU.  Each split writes a partial sum to scratch;
// a second kernel adds the partials in split order (deterministic).
#include "tc_internal.cuh"

namespace tc {

namespace {

constexpr int kDirWarps = 4;
constexpr int kDirTargetWarps = 152 * 32;  // aim for about this many warps in flight

__global__ void k_direct_pack(const double* __restrict__ x, const double* __restrict__ f,
                              const double* __restrict__ h, const double* __restrict__ nu, int64_t N,
                              float4* __restrict__ pack)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    float hi[3], lo[3];
    for (int a = 0; a < 3; a++) {
        double v = x[a * N + i];
        hi[a] = (float)v;
        lo[a] = (float)(v - (double)hi[a]);
    }
    pack[4 * i + 0] = make_float4(hi[0], hi[1], hi[2], (float)f[i]);
    pack[4 * i + 1] = make_float4(lo[0], lo[1], lo[2], (float)f[N + i]);
    pack[4 * i + 2] = make_float4((float)f[2 * N + i], (float)h[i], (float)h[N + i], (float)h[2 * N + i]);
    // the fourth slot holds h.nu, which only the regularized pair terms read
    const double hn = h[i] * nu[i] + h[N + i] * nu[N + i] + h[2 * N + i] * nu[2 * N + i];
    pack[4 * i + 3] = make_float4((float)nu[i], (float)nu[N + i], (float)nu[2 * N + i], (float)hn);
}

template <bool kReg>
__global__ void __launch_bounds__(kDirWarps * 32)
    k_direct_mixed(const double* __restrict__ t, int64_t M, const float4* __restrict__ pack, int64_t N, int64_t chunk,
                   double* __restrict__ part, float e2)
{
    const float e2h = 0.5f * e2;
    __shared__ float4 tile[kDirWarps][32][4];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nbatch = (M + 31) / 32;
    const int64_t b = blockIdx.x * (int64_t)kDirWarps + w;
    if (b >= nbatch) return;
    const int64_t m = b * 32 + lane;
    const bool valid = m < M;
    float th[3] = {0, 0, 0}, tl[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) {
            double v = t[a * M + m];
            th[a] = (float)v;
            tl[a] = (float)(v - (double)th[a]);
        }
    const int64_t s0 = blockIdx.y * chunk, s1 = min(N, s0 + chunk);
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int64_t base = s0; base < s1; base += 32) {
        const int cnt = (int)min((int64_t)32, s1 - base);
        __syncwarp();
        if (lane < cnt) {
            const float4* src = pack + 4 * (base + lane);
            tile[w][lane][0] = src[0];
            tile[w][lane][1] = src[1];
            tile[w][lane][2] = src[2];
            tile[w][lane][3] = src[3];
        }
        __syncwarp();
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int j = 0; j < cnt; j++) {
            const float4 p0 = tile[w][j][0], p1 = tile[w][j][1], p2 = tile[w][j][2], p3 = tile[w][j][3];
            const float dx = (th[0] - p0.x) + (tl[0] - p1.x);
            const float dy = (th[1] - p0.y) + (tl[1] - p1.y);
            const float dz = (th[2] - p0.z) + (tl[2] - p1.z);
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float df = fmaf(dx, p0.w, fmaf(dy, p1.w, dz * p2.x));
            const float dh = fmaf(dx, p2.y, fmaf(dy, p2.z, dz * p2.w));
            const float dn = fmaf(dx, p3.x, fmaf(dy, p3.y, dz * p3.z));
            if (kReg) {
                const float q = r2 > 0.f ? rsqrt_ftz(r2 + e2) : 0.f;
                const float q2 = q * q;
                const float a1 = q * fmaf(e2, q2, 1.0f);
                const float qs = q * q2 * fmaf(q2, fmaf(dh, dn, e2h * p3.w), df);
                const float w = e2h * q * q2 * q2;
                const float wn = w * dn, wh = w * dh;
                ax = fmaf(p0.w, a1, fmaf(dx, qs, fmaf(p2.y, wn, fmaf(p3.x, wh, ax))));
                ay = fmaf(p1.w, a1, fmaf(dy, qs, fmaf(p2.z, wn, fmaf(p3.y, wh, ay))));
                az = fmaf(p2.x, a1, fmaf(dz, qs, fmaf(p2.w, wn, fmaf(p3.z, wh, az))));
            } else {
                const float ri = r2 > 0.f ? rsqrt_ftz(r2) : 0.f;
                const float ri2 = ri * ri;
                const float ri3 = ri2 * ri;
                const float st = ri3 * fmaf(dh * dn, ri2, df);
                ax = fmaf(p0.w, ri, fmaf(dx, st, ax));
                ay = fmaf(p1.w, ri, fmaf(dy, st, ay));
                az = fmaf(p2.x, ri, fmaf(dz, st, az));
            }
        }
        ux += (double)ax;
        uy += (double)ay;
        uz += (double)az;
    }
    if (valid) {
        double* o = part + (int64_t)blockIdx.y * 3 * M;
        o[m] = ux;
        o[M + m] = uy;
        o[2 * M + m] = uz;
    }
}

template <bool kReg>
__global__ void __launch_bounds__(kDirWarps * 32)
    k_direct_fp64(const double* __restrict__ t, int64_t M, const double* __restrict__ x, const double* __restrict__ f,
                  const double* __restrict__ h, const double* __restrict__ nu, int64_t N, int64_t chunk,
                  double* __restrict__ part, double e2)
{
    const double e2h = 0.5 * e2;
    __shared__ double tile[kDirWarps][12][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t nbatch = (M + 31) / 32;
    const int64_t b = blockIdx.x * (int64_t)kDirWarps + w;
    if (b >= nbatch) return;
    const int64_t m = b * 32 + lane;
    const bool valid = m < M;
    double tx[3] = {0, 0, 0};
    if (valid)
        for (int a = 0; a < 3; a++) tx[a] = t[a * M + m];
    const int64_t s0 = blockIdx.y * chunk, s1 = min(N, s0 + chunk);
    double ux = 0.0, uy = 0.0, uz = 0.0;
    for (int64_t base = s0; base < s1; base += 32) {
        const int cnt = (int)min((int64_t)32, s1 - base);
        __syncwarp();
        if (lane < cnt) {
            const int64_t i = base + lane;
            for (int a = 0; a < 3; a++) {
                tile[w][a][lane] = x[a * N + i];
                tile[w][3 + a][lane] = f[a * N + i];
                tile[w][6 + a][lane] = h[a * N + i];
                tile[w][9 + a][lane] = nu[a * N + i];
            }
        }
        __syncwarp();
        for (int j = 0; j < cnt; j++) {
            const double dx = tx[0] - tile[w][0][j], dy = tx[1] - tile[w][1][j], dz = tx[2] - tile[w][2][j];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double f0 = tile[w][3][j], f1 = tile[w][4][j], f2 = tile[w][5][j];
            const double df = dx * f0 + dy * f1 + dz * f2;
            const double dh = dx * tile[w][6][j] + dy * tile[w][7][j] + dz * tile[w][8][j];
            const double dn = dx * tile[w][9][j] + dy * tile[w][10][j] + dz * tile[w][11][j];
            if (kReg) {
                if (!(r2 > 0.0)) continue;
                const double hn = tile[w][6][j] * tile[w][9][j] + tile[w][7][j] * tile[w][10][j] +
                                  tile[w][8][j] * tile[w][11][j];
                const double q = rsqrt(r2 + e2), q2 = q * q;
                const double a1 = q * (1.0 + e2 * q2);
                const double qs = q * q2 * (df + q2 * (dh * dn + e2h * hn));
                const double wq = e2h * q * q2 * q2;
                ux += f0 * a1 + dx * qs + wq * (tile[w][6][j] * dn + tile[w][9][j] * dh);
                uy += f1 * a1 + dy * qs + wq * (tile[w][7][j] * dn + tile[w][10][j] * dh);
                uz += f2 * a1 + dz * qs + wq * (tile[w][8][j] * dn + tile[w][11][j] * dh);
            } else {
                const double ri = r2 > 0.0 ? rsqrt(r2) : 0.0;
                const double ri2 = ri * ri, ri3 = ri2 * ri;
                const double st = ri3 * (df + dh * dn * ri2);
                ux += f0 * ri + dx * st;
                uy += f1 * ri + dy * st;
                uz += f2 * ri + dz * st;
            }
        }
    }
    if (valid) {
        double* o = part + (int64_t)blockIdx.y * 3 * M;
        o[m] = ux;
        o[M + m] = uy;
        o[2 * M + m] = uz;
    }
}

__global__ void k_direct_reduce(const double* __restrict__ part, int nsplit, int64_t M, double* __restrict__ u)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 3 * M) return;
    double s = 0.0;
    for (int k = 0; k < nsplit; k++) s += part[(int64_t)k * 3 * M + i];
    u[i] = s;
}

struct DirectPlan {
    int nsplit;
    int64_t chunk;
    size_t pack_bytes, part_bytes;
};

DirectPlan plan_direct(int precision, int64_t N, int64_t M)
{
    DirectPlan pl;
    int64_t nwarps = (M + 31) / 32;
    int64_t want = (kDirTargetWarps + nwarps - 1) / nwarps;
    int64_t maxsplit = N / 512 > 1 ? N / 512 : 1;
    if (want > maxsplit) want = maxsplit;
    if (want > 65535) want = 65535;
    if (want < 1) want = 1;
    pl.chunk = (N + want - 1) / want;
    pl.chunk = (pl.chunk + 31) / 32 * 32;
    pl.nsplit = (int)((N + pl.chunk - 1) / pl.chunk);
    if (pl.nsplit < 1) pl.nsplit = 1;
    pl.pack_bytes = precision == TC_FP64 ? 0 : (size_t)N * 64;
    pl.part_bytes = (size_t)pl.nsplit * 3 * (size_t)M * sizeof(double);
    return pl;
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

size_t direct_scratch_bytes(int precision, int64_t N, int64_t M)
{
    DirectPlan pl = plan_direct(precision, N, M);
    return ((pl.pack_bytes + 255) / 256) * 256 + pl.part_bytes;
}

cudaError_t launch_direct(int precision, const double* x, const double* f, const double* h, const double* nu,
                          int64_t N, const double* t, int64_t M, double* u, void* scratch, size_t scratch_bytes,
                          double eps, cudaStream_t s)
{
    DirectPlan pl = plan_direct(precision, N, M);
    size_t pack_off = ((pl.pack_bytes + 255) / 256) * 256;
    if (scratch_bytes < pack_off + pl.part_bytes) return cudaErrorInvalidValue;
    float4* pack = reinterpret_cast<float4*>(scratch);
    double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(scratch) + pack_off);
    int64_t nbatch = (M + 31) / 32;
    dim3 grid((unsigned)((nbatch + kDirWarps - 1) / kDirWarps), (unsigned)pl.nsplit);
    const double e2 = eps * eps;
    if (precision == TC_FP64) {
        if (eps > 0.0)
            k_direct_fp64<true><<<grid, kDirWarps * 32, 0, s>>>(t, M, x, f, h, nu, N, pl.chunk, part, e2);
        else
            k_direct_fp64<false><<<grid, kDirWarps * 32, 0, s>>>(t, M, x, f, h, nu, N, pl.chunk, part, 0.0);
        note_launch();
    } else {
        k_direct_pack<<<grid_for(N, 256), 256, 0, s>>>(x, f, h, nu, N, pack);
        note_launch();
        if (eps > 0.0)
            k_direct_mixed<true><<<grid, kDirWarps * 32, 0, s>>>(t, M, pack, N, pl.chunk, part, (float)e2);
        else
            k_direct_mixed<false><<<grid, kDirWarps * 32, 0, s>>>(t, M, pack, N, pl.chunk, part, 0.0f);
        note_launch();
    }
    k_direct_reduce<<<grid_for(3 * M, 256), 256, 0, s>>>(part, pl.nsplit, M, u);
    note_launch();
    return cudaGetLastError();
}

}  // namespace tc

// ---------------------------------------------------------------------------
// tc_direct_noalloc: the same direct sum, with its scratch (the FP32 source
// pack of the mixed path and the per-split partial sums) in one fixed array
// of device memory that is part of the library image, for callers that may
// not allocate device memory themselves.  See include/tc.h for the contract.
// ---------------------------------------------------------------------------
#include <mutex>

namespace tc {
namespace {

constexpr size_t kNoAllocBytes = (size_t)TC_DIRECT_NOALLOC_SCRATCH_BYTES;
constexpr int kNoAllocMaxDevices = 64;

// Device-side scratch shared by every tc_direct_noalloc call on a device.
// Host code must not use this name as an address: it is a host-side stand-in.
static __device__ __align__(256) unsigned char g_direct_scratch[kNoAllocBytes];

// Device address of g_direct_scratch per device, looked up once per device.
void* g_noalloc_addr[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mu;

cudaError_t noalloc_scratch(int dev, void** out)
{
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_direct_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace tc

extern "C" tc_status tc_direct_noalloc(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                                       const double* targets, int64_t M, int32_t precision, void* stream, double* u)
{
    using namespace tc;
    if (!x || !f || !h || !nu || !u) return fail(nullptr, TC_EINVAL, "tc_direct_noalloc: a pointer is NULL");
    if (N < 1 || N >= ((int64_t)1 << 31)) return fail(nullptr, TC_EINVAL, "tc_direct_noalloc: N out of range");
    if (!targets && M != N) return fail(nullptr, TC_EINVAL, "tc_direct_noalloc: targets = NULL requires M = N");
    if (M < 1 || M >= ((int64_t)1 << 31)) return fail(nullptr, TC_EINVAL, "tc_direct_noalloc: M out of range");
    if (precision != TC_FP64 && precision != TC_MIXED)
        return fail(nullptr, TC_EINVAL, "tc_direct_noalloc: unknown precision");
    // size check first: nothing is launched for a problem that does not fit
    DirectPlan pl = plan_direct(precision, N, M);
    const size_t pack_off = ((pl.pack_bytes + 255) / 256) * 256;
    const size_t per_split = (size_t)3 * (size_t)M * sizeof(double);
    if (pack_off + per_split > kNoAllocBytes)
        return fail(nullptr, TC_EINVAL,
                    "tc_direct_noalloc: needs %zu bytes of scratch (64 B per source in mixed precision + 24 B per "
                    "target), the fixed array holds %zu bytes; use tc_direct for this size",
                    pack_off + per_split, kNoAllocBytes);
    const int64_t max_split = (int64_t)((kNoAllocBytes - pack_off) / per_split);
    if (pl.nsplit > max_split) {
        pl.chunk = (N + max_split - 1) / max_split;
        pl.chunk = (pl.chunk + 31) / 32 * 32;
        pl.nsplit = (int)((N + pl.chunk - 1) / pl.chunk);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tc_direct_noalloc device");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(nullptr, TC_EINVAL, "tc_direct_noalloc: device %d", dev);
    void* base = nullptr;
    e = noalloc_scratch(dev, &base);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tc_direct_noalloc scratch address");
    cudaStream_t s = (cudaStream_t)stream;
    const double* t = targets ? targets : x;
    float4* pack = reinterpret_cast<float4*>(base);
    double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(base) + pack_off);
    const int64_t nbatch = (M + 31) / 32;
    dim3 grid((unsigned)((nbatch + kDirWarps - 1) / kDirWarps), (unsigned)pl.nsplit);
    // every scratch word read below is first written by this call: the pack by
    // k_direct_pack, each split's partial block by its own k_direct_* launch
    if (precision == TC_FP64) {
        k_direct_fp64<false><<<grid, kDirWarps * 32, 0, s>>>(t, M, x, f, h, nu, N, pl.chunk, part, 0.0);
        note_launch();
    } else {
        k_direct_pack<<<grid_for(N, 256), 256, 0, s>>>(x, f, h, nu, N, pack);
        note_launch();
        k_direct_mixed<false><<<grid, kDirWarps * 32, 0, s>>>(t, M, pack, N, pl.chunk, part, 0.0f);
        note_launch();
    }
    k_direct_reduce<<<grid_for(3 * M, 256), 256, 0, s>>>(part, pl.nsplit, M, u);
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "tc_direct_noalloc launch");
    return TC_OK;
}
