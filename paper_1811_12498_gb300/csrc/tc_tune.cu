// Choice of (theta, p, N0) for a target accuracy.
//
// Section 6 of the paper ends on the remark that tuning the MAC parameter
// theta, the order p and the leaf size N0 to the accuracy wanted would make
// the treecode more efficient; its Table 1 shows why: at low accuracy
// theta = 0.8 is the fastest way to a given error E, at medium accuracy 0.5,
// at high accuracy 0.2.  tc_tune measures that trade-off on the caller's own
// system: every candidate of a (theta, p, N0) grid is run in full (tc_build,
// tc_moments, tc_eval with targets = sources) and timed on the device, its
// error E (the relative L2 error of Section 6) is taken against the FP64
// direct sum at a sample of the particles, and the fastest candidate whose E
// reaches the target is returned.
#include <cmath>
#include <vector>

#include "tc_internal.cuh"

namespace tc {
namespace {

// dst (3 x m) = rows idx of src (3 x n)
__global__ void k_gather_rows(const double* __restrict__ src, int64_t n, const int64_t* __restrict__ idx, int64_t m,
                              double* __restrict__ dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t j = idx[i];
    dst[i] = src[j];
    dst[m + i] = src[n + j];
    dst[2 * m + i] = src[2 * n + j];
}

cudaError_t gather_rows(const double* src, int64_t n, const int64_t* idx, int64_t m, double* dst, cudaStream_t s)
{
    k_gather_rows<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(src, n, idx, m, dst);
    note_launch();
    return cudaGetLastError();
}

// scratch owned by one tc_tune call
struct TuneBufs {
    DevBuf idx, xs, ud, ut, u;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TuneBufs()
    {
        release(idx), release(xs), release(ud), release(ut), release(u);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

double rel_l2(const std::vector<double>& a, const std::vector<double>& ref)
{
    double num = 0.0, den = 0.0;
    for (size_t i = 0; i < a.size(); i++) {
        const double d = a[i] - ref[i];
        num += d * d;
        den += ref[i] * ref[i];
    }
    return den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
}

}  // namespace
}  // namespace tc

using namespace tc;

#define TT_CK(call, where)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

#define TT_ST(call)                          \
    do {                                     \
        tc_status s_ = (call);               \
        if (s_ != TC_OK) return s_;          \
    } while (0)

extern "C" tc_status tc_tune(tc_ctx* ctx, const double* x, const double* f, const double* h, const double* nu,
                             int64_t N, const double* thetas, int32_t n_theta, const int32_t* orders, int32_t n_order,
                             const int32_t* leaf_sizes, int32_t n_leaf, const int64_t* sample, int64_t n_sample,
                             double target_E, double* seconds, double* errors, int32_t* best)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_tune: ctx is NULL");
    if (ctx->reg_eps > 0.0) return fail(ctx, TC_EINVAL, "tc_tune: not available for the regularized kernels");
    if (!x || !f || !h || !nu) return fail(ctx, TC_EINVAL, "tc_tune: a particle array is NULL");
    if (!thetas || !orders || !leaf_sizes || !sample || !seconds || !errors || !best)
        return fail(ctx, TC_EINVAL, "tc_tune: a host array is NULL");
    if (N < 1 || N >= ((int64_t)1 << 31)) return fail(ctx, TC_EINVAL, "tc_tune: N = %lld out of range", (long long)N);
    if (n_theta < 1 || n_order < 1 || n_leaf < 1) return fail(ctx, TC_EINVAL, "tc_tune: an empty parameter grid");
    if (n_sample < 1 || n_sample > N)
        return fail(ctx, TC_EINVAL, "tc_tune: n_sample = %lld out of [1, N]", (long long)n_sample);
    if (!(target_E > 0.0) || !std::isfinite(target_E)) return fail(ctx, TC_EINVAL, "tc_tune: target_E must be > 0");
    for (int i = 0; i < n_theta; i++)
        if (!(thetas[i] > 0.0 && thetas[i] < 1.0))
            return fail(ctx, TC_EINVAL, "tc_tune: theta = %g out of (0, 1)", thetas[i]);
    for (int i = 0; i < n_order; i++)
        if (orders[i] < 0 || orders[i] > kPMax)
            return fail(ctx, TC_EINVAL, "tc_tune: p = %d out of [0, %d]", orders[i], kPMax);
    for (int i = 0; i < n_leaf; i++)
        if (leaf_sizes[i] < 1) return fail(ctx, TC_EINVAL, "tc_tune: N0 = %d < 1", leaf_sizes[i]);
    for (int64_t i = 0; i < n_sample; i++)
        if (sample[i] < 0 || sample[i] >= N)
            return fail(ctx, TC_EINVAL, "tc_tune: sample[%lld] = %lld out of [0, N)", (long long)i,
                        (long long)sample[i]);
    cudaStream_t s = ctx->stream;
    TuneBufs b;
    const int64_t m = n_sample;
    TT_CK(ensure(b.idx, (size_t)m * 8), "tc_tune: alloc");
    TT_CK(ensure(b.xs, (size_t)3 * m * 8), "tc_tune: alloc");
    TT_CK(ensure(b.ud, (size_t)3 * m * 8), "tc_tune: alloc");
    TT_CK(ensure(b.ut, (size_t)3 * m * 8), "tc_tune: alloc");
    TT_CK(ensure(b.u, (size_t)3 * N * 8), "tc_tune: alloc");
    TT_CK(cudaEventCreate(&b.e0), "tc_tune: event");
    TT_CK(cudaEventCreate(&b.e1), "tc_tune: event");
    TT_CK(cudaMemcpyAsync(b.idx.p, sample, (size_t)m * 8, cudaMemcpyHostToDevice, s), "tc_tune: sample");
    // the reference: FP64 direct sum at the sampled particles (coincident
    // pairs, i.e. the particle itself, contribute nothing)
    TT_CK(gather_rows(x, N, ptr<int64_t>(b.idx), m, ptr<double>(b.xs), s), "tc_tune: gather");
    {
        tc_status st = tc_direct(x, f, h, nu, N, ptr<double>(b.xs), m, TC_FP64, (void*)s, ptr<double>(b.ud));
        if (st != TC_OK) return fail(ctx, st, "tc_tune: direct sum: %s", tc_last_error(nullptr));
    }
    std::vector<double> ud(3 * m), ut(3 * m);
    TT_CK(cudaMemcpyAsync(ud.data(), b.ud.p, (size_t)3 * m * 8, cudaMemcpyDeviceToHost, s), "tc_tune: copy");
    TT_CK(cudaStreamSynchronize(s), "tc_tune: sync");
    *best = -1;
    double best_s = 0.0;
    int32_t k = 0;
    for (int il = 0; il < n_leaf; il++)
        for (int ip = 0; ip < n_order; ip++)
            for (int it = 0; it < n_theta; it++, k++) {
                // two full runs; the second is timed (the first loads the
                // kernels of this order and sizes the buffers)
                for (int rep = 0; rep < 2; rep++) {
                    TT_CK(cudaEventRecord(b.e0, s), "tc_tune: event");
                    TT_ST(tc_build(ctx, x, N, leaf_sizes[il]));
                    TT_ST(tc_moments(ctx, f, h, nu, orders[ip]));
                    TT_ST(tc_eval(ctx, nullptr, N, thetas[it], orders[ip], ptr<double>(b.u)));
                    TT_CK(cudaEventRecord(b.e1, s), "tc_tune: event");
                }
                TT_CK(gather_rows(ptr<double>(b.u), N, ptr<int64_t>(b.idx), m, ptr<double>(b.ut), s),
                      "tc_tune: gather");
                TT_CK(cudaMemcpyAsync(ut.data(), b.ut.p, (size_t)3 * m * 8, cudaMemcpyDeviceToHost, s),
                      "tc_tune: copy");
                TT_CK(cudaStreamSynchronize(s), "tc_tune: sync");
                TT_ST(tc_sync(ctx));
                float ms = 0.0f;
                TT_CK(cudaEventElapsedTime(&ms, b.e0, b.e1), "tc_tune: timing");
                seconds[k] = 1e-3 * ms;
                errors[k] = rel_l2(ut, ud);
                if (errors[k] <= target_E && (*best < 0 || seconds[k] < best_s)) {
                    *best = k;
                    best_s = seconds[k];
                }
            }
    return TC_OK;
}
