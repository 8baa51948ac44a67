// C ABI entry points (include/tc.h): argument checks, buffer management and
// the order of kernel launches for tree build, moments and evaluation.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <new>

#include "tc_internal.cuh"

namespace tc {

static thread_local std::string g_thread_err = "no error";

tc_status fail(tc_ctx* ctx, tc_status st, const char* fmt, ...)
{
    char buf[768];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_thread_err = buf;
    return st;
}

tc_status cuda_fail(tc_ctx* ctx, cudaError_t e, const char* where)
{
    if (e == cudaErrorMemoryAllocation)
        return fail(ctx, TC_ENOMEM, "%s: %s", where, cudaGetErrorString(e));
    return fail(ctx, TC_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

cudaError_t ensure(DevBuf& b, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (b.p && b.cap >= bytes) return cudaSuccess;
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        if (e != cudaSuccess) return e;
    }
    size_t want = (bytes + 255) / 256 * 256;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        b.p = nullptr;
        return e;
    }
    b.cap = want;
    return cudaSuccess;
}

// grow keeping the first `keep` bytes
static cudaError_t grow_keep(DevBuf& b, size_t bytes, size_t keep, cudaStream_t s)
{
    if (b.p && b.cap >= bytes) return cudaSuccess;
    size_t want = (bytes + 255) / 256 * 256;
    void* np = nullptr;
    if (alloc_should_fail()) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMalloc(&np, want);
    if (e != cudaSuccess) return e;
    if (b.p && keep) {
        e = cudaMemcpyAsync(np, b.p, keep, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(np);
            return e;
        }
    }
    if (b.p) cudaFree(b.p);
    b.p = np;
    b.cap = want;
    return cudaSuccess;
}

void release(DevBuf& b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

}  // namespace tc

using namespace tc;

static std::atomic<int64_t> g_launches{0};
void tc::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

// allocations still allowed before injected failures start; -1 = no injection
static std::atomic<int64_t> g_alloc_budget{-1};
bool tc::alloc_should_fail()
{
    int64_t b = g_alloc_budget.load(std::memory_order_relaxed);
    while (b > 0 && !g_alloc_budget.compare_exchange_weak(b, b - 1, std::memory_order_relaxed)) {
    }
    return b == 0;
}


#define TC_CK(call, where)                                  \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, where); \
    } while (0)

static void release_all(tc_ctx* c)
{
    DevBuf* bufs[] = {&c->root, &c->bbox_part, &c->keys, &c->keys_alt, &c->perm, &c->perm_alt, &c->hist, &c->xs,
                      &c->node_topo, &c->node_info, &c->node_key, &c->node_geo, &c->node_invrho, &c->node_geof, &c->geo_tmp,
                      &c->split_cnt,
                      &c->split_off, &c->scan_tmp, &c->ws, &c->spack, &c->mom, &c->mom_tmp, &c->m2m_tmp, &c->ab64, &c->ab32,
                      &c->abf64,
                      &c->abf32, &c->geo32, &c->reg_et, &c->reg_et32, &c->tkeys,
                      &c->tkeys_alt, &c->tperm, &c->tperm_alt, &c->ts, &c->nfar_e, &c->nnear_e,
                      &c->far_off, &c->near_off, &c->far_list, &c->near_list, &c->cnt_far, &c->cnt_near, &c->u_far,
                      &c->u_near, &c->nl_keys, &c->nl_keys_alt, &c->nl_idx, &c->nl_idx_alt, &c->nl_eb, &c->nl_hist,
                      &c->nl_nA, &c->nl_nkey, &c->nl_nkey_alt, &c->nl_nord, &c->nl_nord_alt, &c->nl_sA,
                      &c->nl_inc0s, &c->nl_ninc0, &c->nl_cur, &c->nl_ucnt, &c->nl_uoff, &c->nl_units,
                      &c->nl_inc_m, &c->nl_inc_e, &c->nl_slots, &c->flags, &c->adj_fkeys, &c->adj_fkeys_alt,
                      &c->adj_fidx, &c->adj_fidx_alt, &c->adj_febatch, &c->adj_hist, &c->adj_scnt, &c->adj_soff, &c->adj_gs, &c->adj_gt, &c->adj_abar, &c->adj_fbar, &c->adj_lam,
                      &c->adj_lamacc, &c->adj_gfar, &c->adj_gnear, &c->host_in, &c->host_u};
    for (DevBuf* b : bufs) release(*b);
}

extern "C" {

tc_status tc_create(tc_ctx** out, const tc_config* cfg)
{
    tc_ctx* ctx = nullptr;
    if (!out) return fail(nullptr, TC_EINVAL, "tc_create: out is NULL");
    *out = nullptr;
    tc_config c = {TC_MIXED, 1, nullptr, 0, 0, 0.0};
    if (cfg) c = *cfg;
    if (!(c.reg_eps >= 0.0) || !std::isfinite(c.reg_eps))
        return fail(nullptr, TC_EINVAL, "tc_create: reg_eps = %g must be >= 0 and finite", c.reg_eps);
    if (c.precision != TC_FP64 && c.precision != TC_MIXED)
        return fail(nullptr, TC_EINVAL, "tc_create: unknown precision %d", c.precision);
    if (c.shrink != 0 && c.shrink != 1) return fail(nullptr, TC_EINVAL, "tc_create: shrink must be 0 or 1");
    if (c.reserved1 != 0) return fail(nullptr, TC_EINVAL, "tc_create: reserved1 must be 0");
    if (c.rec64 != 0 && c.rec64 != 1) return fail(nullptr, TC_EINVAL, "tc_create: rec64 must be 0 or 1");
    ctx = new (std::nothrow) tc_ctx();
    if (!ctx) return fail(nullptr, TC_ENOMEM, "tc_create: out of host memory");
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = ensure(ctx->flags, 256);
    if (e == cudaSuccess) e = ensure(ctx->scan_tmp, 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->flags.p, 0, 256, (cudaStream_t)c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)c.stream);
    if (e != cudaSuccess) {
        tc_status st = cuda_fail(nullptr, e, "tc_create");
        release_all(ctx);
        delete ctx;
        return st;
    }
    ctx->precision = c.precision;
    ctx->rec64 = c.precision == TC_MIXED ? c.rec64 : 0;
    ctx->shrink = c.shrink;
    ctx->reg_eps = c.reg_eps;
    ctx->stream = (cudaStream_t)c.stream;
    ctx->err = "no error";
    *out = ctx;
    return TC_OK;
}

tc_status tc_destroy(tc_ctx* ctx)
{
    if (!ctx) return TC_OK;
    cudaStreamSynchronize(ctx->stream);
    if (ctx->stream2) cudaStreamSynchronize(ctx->stream2);
    release_all(ctx);
    for (cudaEvent_t& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_mom) cudaEventDestroy(ctx->ev_mom);
    if (ctx->stream2) cudaStreamDestroy(ctx->stream2);
    if (ctx->host_words) cudaFreeHost(ctx->host_words);
    delete ctx;
    return TC_OK;
}

tc_status tc_profile(tc_ctx* ctx, int32_t enable)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_profile: ctx is NULL");
    if (enable && !ctx->ev[0])
        for (cudaEvent_t& e : ctx->ev) TC_CK(cudaEventCreate(&e), "tc_profile event");
    if (enable < 0 || enable > 2) return fail(ctx, TC_EINVAL, "tc_profile: enable must be 0, 1 or 2");
    for (int& r : ctx->ev_recorded) r = 0;
    ctx->profile = enable;
    return TC_OK;
}

tc_status tc_phase_times(tc_ctx* ctx, double* ms)
{
    if (!ctx || !ms) return fail(ctx, TC_EINVAL, "tc_phase_times: NULL argument");
    TC_CK(cudaStreamSynchronize(ctx->stream), "tc_phase_times sync");
    for (int ph = 0; ph < TC_NPHASES; ph++) {
        ms[ph] = -1.0;
        if (!ctx->ev_recorded[ph]) continue;
        float t = 0.f;
        TC_CK(cudaEventElapsedTime(&t, ctx->ev[2 * ph], ctx->ev[2 * ph + 1]), "tc_phase_times");
        ms[ph] = t;
    }
    return TC_OK;
}

int64_t tc_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

void tc_fail_allocations(int64_t after)
{
    g_alloc_budget.store(after < 0 ? -1 : after, std::memory_order_relaxed);
}

tc_status tc_fma_peak(int32_t precision, void* stream, double* tflops)
{
    if (!tflops) return fail(nullptr, TC_EINVAL, "tc_fma_peak: tflops is NULL");
    if (precision != TC_FP64 && precision != TC_MIXED)
        return fail(nullptr, TC_EINVAL, "tc_fma_peak: unknown precision %d", precision);
    cudaStream_t s = (cudaStream_t)stream;
    double r = 0.0, ms = 0.0;
    tc_ctx* ctx = nullptr;
    if (precision == TC_FP64) {
        TC_CK(run_probe(2, s, &r, &ms), "tc_fma_peak");
    } else {
        double r2 = 0.0;
        TC_CK(run_probe(0, s, &r, &ms), "tc_fma_peak");
        TC_CK(run_probe(1, s, &r2, &ms), "tc_fma_peak");
        r = r2 > r ? r2 : r;
    }
    *tflops = r;
    return TC_OK;
}

const char* tc_last_error(const tc_ctx* ctx)
{
    if (ctx) return ctx->err.c_str();
    return g_thread_err.c_str();
}

static tc_status check_flags(tc_ctx* ctx)
{
    int32_t f = 0;
    TC_CK(cudaMemcpyAsync(&f, ctx->flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream), "flags");
    TC_CK(cudaStreamSynchronize(ctx->stream), "flags sync");
    if (f & kFlagStack) return fail(ctx, TC_EDEVICE, "device check: traversal stack bound exceeded");
    if (f) return fail(ctx, TC_EDEVICE, "device check: flags 0x%x", f);
    return TC_OK;
}

tc_status tc_sync(tc_ctx* ctx)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_sync: ctx is NULL");
    TC_CK(join_moments(ctx), "tc_sync");
    TC_CK(cudaStreamSynchronize(ctx->stream), "tc_sync");
    return check_flags(ctx);
}

tc_status tc_build(tc_ctx* ctx, const double* x, int64_t N, int32_t N0)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_build: ctx is NULL");
    if (!x) return fail(ctx, TC_EINVAL, "tc_build: x is NULL");
    if (N < 1 || N >= ((int64_t)1 << 31)) return fail(ctx, TC_EINVAL, "tc_build: N = %lld out of [1, 2^31)", (long long)N);
    if (N0 < 1) return fail(ctx, TC_EINVAL, "tc_build: N0 = %d must be >= 1", N0);
    TC_CK(join_moments(ctx), "tc_build");
    cudaStream_t s = ctx->stream;
    ctx->built = ctx->have_moments = ctx->have_eval = 0;
    ctx->ab_p = -1;
    ctx->N = N;
    ctx->N0 = N0;
    int nblk = (int)((N + 255) / 256);
    if (nblk > 152 * 4) nblk = 152 * 4;
    int nrad = radix_blocks(N);
    TC_CK(ensure(ctx->root, 64), "alloc root");
    TC_CK(ensure(ctx->bbox_part, (size_t)nblk * 6 * sizeof(double)), "alloc bbox");
    TC_CK(ensure(ctx->keys, (size_t)N * 8), "alloc keys");
    TC_CK(ensure(ctx->keys_alt, (size_t)N * 8), "alloc keys");
    TC_CK(ensure(ctx->perm, (size_t)N * 4), "alloc perm");
    TC_CK(ensure(ctx->perm_alt, (size_t)N * 4), "alloc perm");
    TC_CK(ensure(ctx->hist, (size_t)256 * nrad * 4), "alloc hist");
    TC_CK(ensure(ctx->xs, (size_t)3 * N * 8), "alloc xs");

    ph_begin(ctx, TC_PH_BUILD);
    TC_CK(launch_bbox(x, N, ptr<double>(ctx->bbox_part), nblk, ptr<double>(ctx->root), s), "bbox");
    TC_CK(launch_keys(x, N, ptr<double>(ctx->root), ptr<uint64_t>(ctx->keys), ptr<int32_t>(ctx->perm), 0, s), "keys");
    TC_CK(radix_sort(ptr<uint64_t>(ctx->keys), ptr<int32_t>(ctx->perm), ptr<uint64_t>(ctx->keys_alt),
                     ptr<int32_t>(ctx->perm_alt), ptr<uint32_t>(ctx->hist), N, s),
          "sort");
    TC_CK(launch_gather3(x, ptr<int32_t>(ctx->perm), N, ptr<double>(ctx->xs), s), "gather x");
    double root[6];
    TC_CK(cudaMemcpyAsync(root, ctx->root.p, sizeof(root), cudaMemcpyDeviceToHost, s), "root copy");
    TC_CK(cudaStreamSynchronize(s), "root sync");
    if (root[5] != 0.0) return fail(ctx, TC_EINVAL, "tc_build: x holds a NaN or an infinity");
    for (int a = 0; a < 3; a++) ctx->lo[a] = root[a];
    ctx->side = root[3];

    // level-synchronous topology
    size_t cap = 1024;
    TC_CK(grow_keep(ctx->node_topo, cap * sizeof(int4), 0, s), "alloc nodes");
    TC_CK(grow_keep(ctx->node_info, cap * sizeof(int4), 0, s), "alloc nodes");
    TC_CK(grow_keep(ctx->node_key, cap * sizeof(uint64_t), 0, s), "alloc nodes");
    TC_CK(launch_init_root(ptr<int4>(ctx->node_topo), ptr<int4>(ctx->node_info), ptr<uint64_t>(ctx->node_key), N, s),
          "root node");
    ctx->level_begin.assign(1, 0);
    int64_t lb = 0, le = 1;
    for (int level = 0; level < kMaxDepth; level++) {
        int64_t n = le - lb;
        TC_CK(ensure(ctx->split_cnt, (size_t)n * 4), "alloc split");
        TC_CK(ensure(ctx->split_off, (size_t)n * 4), "alloc split");
        TC_CK(launch_split_count(ptr<int4>(ctx->node_topo), ptr<int4>(ctx->node_info), ptr<uint64_t>(ctx->keys), lb, le,
                                 N0, ptr<int32_t>(ctx->split_cnt), s),
              "split count");
        TC_CK(launch_scan_i32(ptr<int32_t>(ctx->split_cnt), ptr<int32_t>(ctx->split_off), n,
                              ptr<int32_t>(ctx->scan_tmp), s),
              "split scan");
        int32_t total = 0;
        TC_CK(cudaMemcpyAsync(&total, ctx->scan_tmp.p, 4, cudaMemcpyDeviceToHost, s), "split total");
        TC_CK(cudaStreamSynchronize(s), "split sync");
        if (total == 0) break;
        if ((size_t)(le + total) > cap) {
            size_t ncap = cap;
            while (ncap < (size_t)(le + total)) ncap *= 2;
            TC_CK(grow_keep(ctx->node_topo, ncap * sizeof(int4), (size_t)le * sizeof(int4), s), "grow nodes");
            TC_CK(grow_keep(ctx->node_info, ncap * sizeof(int4), (size_t)le * sizeof(int4), s), "grow nodes");
            TC_CK(grow_keep(ctx->node_key, ncap * sizeof(uint64_t), (size_t)le * sizeof(uint64_t), s), "grow nodes");
            cap = ncap;
        }
        TC_CK(launch_split_write(ptr<int4>(ctx->node_topo), ptr<int4>(ctx->node_info), ptr<uint64_t>(ctx->node_key),
                                 ptr<uint64_t>(ctx->keys), lb, le, N0, ptr<int32_t>(ctx->split_off), s),
              "split write");
        ctx->level_begin.push_back(le);
        lb = le;
        le += total;
    }
    ctx->level_begin.push_back(le);
    ctx->nnodes = le;
    ctx->depth = (int)ctx->level_begin.size() - 2;
    TC_CK(ensure(ctx->node_geo, (size_t)le * sizeof(Geo)), "alloc geo");
    TC_CK(ensure(ctx->node_invrho, (size_t)le * sizeof(double)), "alloc geo");
    TC_CK(ensure(ctx->geo_tmp, geometry_scratch_bytes(le)), "alloc geo");
    TC_CK(ensure(ctx->node_geof, (size_t)le * 2 * sizeof(float4)), "alloc geo");
    TC_CK(launch_geometry(ptr<int4>(ctx->node_topo), ptr<int4>(ctx->node_info), ptr<uint64_t>(ctx->node_key),
                          ptr<double>(ctx->xs), N, le, ptr<double>(ctx->root), ctx->shrink, ptr<Geo>(ctx->node_geo),
                          ptr<double>(ctx->node_invrho), ptr<float4>(ctx->node_geof), ctx->geo_tmp.p, s),
          "geometry");
    ph_end(ctx, TC_PH_BUILD);
    ctx->built = 1;
    ctx->moved = 0;
    return TC_OK;
}

tc_status tc_moments(tc_ctx* ctx, const double* f, const double* h, const double* nu, int32_t p)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_moments: ctx is NULL");
    if (!ctx->built) return fail(ctx, TC_ESTATE, "tc_moments: call tc_build first");
    if (!f || !h || !nu) return fail(ctx, TC_EINVAL, "tc_moments: a weight pointer is NULL");
    if (p < 0 || p > kPMax) return fail(ctx, TC_EINVAL, "tc_moments: p = %d out of [0, %d]", p, kPMax);
    TC_CK(join_moments(ctx), "tc_moments");
    TC_CK(second_stream(ctx), "second stream");
    cudaStream_t s = ctx->stream;
    const int64_t N = ctx->N;
    ctx->have_moments = ctx->have_eval = 0;
    ctx->ab_p = -1;
    TC_CK(ensure(ctx->ws, (size_t)9 * N * 8), "alloc weights");
    TC_CK(ensure(ctx->mom, (size_t)ctx->nnodes * 12 * ncoef(p) * 8), "alloc moments");
    TC_CK(ensure(ctx->mom_tmp, moments_scratch_bytes(N, ctx->nnodes, p)), "alloc moments");
    {
        // upward-pass scratch: one slot of moments per node of the widest level
        int64_t widest = 1;
        for (size_t L = 0; L + 1 < ctx->level_begin.size(); L++)
            widest = std::max<int64_t>(widest, ctx->level_begin[L + 1] - ctx->level_begin[L]);
        TC_CK(ensure(ctx->m2m_tmp, (size_t)widest * 12 * ncoef(p) * 8), "alloc moments");
    }
    if (ctx->precision == TC_MIXED) TC_CK(ensure(ctx->spack, (size_t)N * 64), "alloc pack");
    ph_begin(ctx, TC_PH_MOMENTS);
    TC_CK(launch_gather_weights(f, h, nu, ptr<int32_t>(ctx->perm), N, ptr<double>(ctx->ws), s), "gather weights");
    if (ctx->precision == TC_MIXED) {
        TC_CK(launch_source_pack(ptr<double>(ctx->xs), ptr<double>(ctx->ws), N, ptr<float4>(ctx->spack), s), "pack");
    }
    // The caller's weights are consumed above; the moment passes read only the
    // library's sorted copies, so they run on the second stream, overlapping
    // the list traversal and the near field of the next tc_eval (FP64 pipe
    // against FP32 and memory latency), and are joined before anything reads
    // the moments.
    // Profile mode 2 keeps them on the first stream.
    const bool async = ctx->profile != 2;
    cudaStream_t sm = async ? ctx->stream2 : s;
    if (async) {
        TC_CK(cudaEventRecord(ctx->ev_fork, s), "fork");
        TC_CK(cudaStreamWaitEvent(sm, ctx->ev_fork, 0), "fork");
    }
    // In mixed precision the near field of the Stokeslet + stresslet kernel
    // takes most of the step and needs no moments: the leaf pass then runs
    // one block per SM beside it, and the far field follows.  Where the far
    // field, which waits for the moments, takes most of the step (the
    // regularized kernels: there it gains from sharing the SMs with the near
    // field) or the near field runs on the FP64 pipe too, the leaf pass runs
    // one block per item and ends first.
    const int mom_blocks = ctx->precision == TC_MIXED && ctx->reg_eps == 0.0 ? 1 : 0;
    TC_CK(launch_moments(ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo), ptr<double>(ctx->xs),
                         ptr<double>(ctx->ws), N, ctx->nnodes, p, ptr<double>(ctx->mom), ctx->mom_tmp.p, mom_blocks,
                         sm),
          "moments");
    // upward pass: level_begin holds the first node of each level and the end
    for (int L = (int)ctx->level_begin.size() - 3; L >= 0; L--)
        TC_CK(launch_m2m(ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo), ctx->level_begin[L],
                         ctx->level_begin[L + 1], ctx->level_begin[L + 1], p, ptr<double>(ctx->mom),
                         ptr<double>(ctx->m2m_tmp), sm),
              "m2m");
    ph_end(ctx, TC_PH_MOMENTS, sm);
    if (async) {
        TC_CK(cudaEventRecord(ctx->ev_mom, sm), "moments done");
        ctx->mom_pending = 1;
    }
    ctx->p_mom = p;
    ctx->have_moments = 1;
    return TC_OK;
}

static tc_status ensure_tables(tc_ctx* ctx, int p, cudaStream_t s)
{
    if (ctx->ab_p == p) return TC_OK;
    const int64_t n = ctx->nnodes * ncoef(p + 2) * 12;
    const int64_t nf = ctx->nnodes * (int64_t)(p + 3) * (p + 3) * 12;
    // FP64 full tables (always: they are the input of the folding), FP32 full
    // tables in mixed precision (the adjoint reads them), folded tables in the
    // working precision (the forward far field reads them)
    TC_CK(ensure(ctx->ab64, (size_t)n * 8), "alloc tables");
    float* ab32 = nullptr;
    if (ctx->precision != TC_FP64) {
        TC_CK(ensure(ctx->ab32, (size_t)n * 4), "alloc tables");
        ab32 = ptr<float>(ctx->ab32);
        TC_CK(ensure(ctx->abf32, (size_t)nf * 4), "alloc tables");
        TC_CK(ensure(ctx->geo32, (size_t)ctx->nnodes * 2 * sizeof(float4)), "alloc tables");
    } else {
        TC_CK(ensure(ctx->abf64, (size_t)nf * 8), "alloc tables");
    }
    ph_begin(ctx, TC_PH_TABLES, s);
    TC_CK(launch_ab_tables(ptr<double>(ctx->mom), ptr<double>(ctx->node_invrho), ctx->nnodes, ctx->p_mom, p,
                           ptr<double>(ctx->ab64), ab32, s),
          "tables");
    TC_CK(launch_fold_tables(ptr<double>(ctx->ab64), ctx->nnodes, p,
                             ctx->precision == TC_FP64 ? ptr<double>(ctx->abf64) : nullptr,
                             ctx->precision == TC_FP64 ? nullptr : ptr<float>(ctx->abf32),
                             ptr<Geo>(ctx->node_geo), ptr<double>(ctx->node_invrho),
                             ctx->precision == TC_FP64 ? nullptr : ptr<float4>(ctx->geo32), s),
          "fold tables");
    if (ctx->reg_eps > 0.0) {
        TC_CK(ensure(ctx->reg_et, (size_t)ctx->nnodes * ncoef(p + 1) * 3 * 8), "alloc tables");
        TC_CK(launch_eps_table(ptr<double>(ctx->mom), ptr<double>(ctx->node_invrho), ctx->nnodes, ctx->p_mom, p,
                               ctx->reg_eps, ptr<double>(ctx->reg_et), s),
              "eps table");
        if (ctx->precision == TC_MIXED) {
            const int64_t ne = ctx->nnodes * ncoef(p + 1) * 3;
            TC_CK(ensure(ctx->reg_et32, (size_t)ne * 4), "alloc tables");
            TC_CK(launch_narrow_table(ptr<double>(ctx->reg_et), ne, ptr<float>(ctx->reg_et32), s), "eps table");
        }
    }
    ph_end(ctx, TC_PH_TABLES, s);
    ctx->ab_p = p;
    return TC_OK;
}

}  // extern "C"

// First half of tc_eval: contraction tables, target ordering and the
// interaction lists (synchronises once to size the lists).
tc_status tc::eval_prepare(tc_ctx* ctx, const double* targets, int64_t M, double theta, int p)
{
    tc_status st = eval_prepare_count(ctx, targets, M, theta, p);
    if (st != TC_OK) return st;
    TC_CK(cudaStreamSynchronize(ctx->stream), "list totals");
    return eval_prepare_finish(ctx);
}

// The part of eval_prepare before the host needs the list sizes: target
// ordering, the counting pass of the traversal and its scans, and the copy of
// the two totals and the device flags into the context's pinned host words.
// Nothing here waits for the device; eval_prepare_finish must follow after
// the context's stream has been synchronised.
tc_status tc::eval_prepare_count(tc_ctx* ctx, const double* targets, int64_t M, double theta, int p)
{
    if (!ctx->have_moments) return fail(ctx, TC_ESTATE, "tc_eval: call tc_build and tc_moments first");
    if (!(theta > 0.0 && theta < 1.0)) return fail(ctx, TC_EINVAL, "tc_eval: theta = %g out of (0, 1)", theta);
    if (p < 0 || p > ctx->p_mom)
        return fail(ctx, TC_EINVAL, "tc_eval: p = %d out of [0, %d] (order of tc_moments)", p, ctx->p_mom);
    if (!targets && M != ctx->N)
        return fail(ctx, TC_EINVAL, "tc_eval: targets = NULL requires M = N (%lld)", (long long)ctx->N);
    if (M < 1 || M >= ((int64_t)1 << 31)) return fail(ctx, TC_EINVAL, "tc_eval: M = %lld out of range", (long long)M);
    cudaStream_t s = ctx->stream;
    ctx->have_eval = 0;
    ctx->prepared = 0;
    ctx->adj_lists_ready = 0;
    ctx->near_sched_ready = 0;
    const double* ts;
    if (!targets) {
        ts = ptr<double>(ctx->xs);
        ctx->eval_self = 1;
    } else {
        int nrad = radix_blocks(M);
        TC_CK(ensure(ctx->tkeys, (size_t)M * 8), "alloc tkeys");
        TC_CK(ensure(ctx->tkeys_alt, (size_t)M * 8), "alloc tkeys");
        TC_CK(ensure(ctx->tperm, (size_t)M * 4), "alloc tperm");
        TC_CK(ensure(ctx->tperm_alt, (size_t)M * 4), "alloc tperm");
        TC_CK(ensure(ctx->hist, (size_t)256 * nrad * 4), "alloc hist");
        TC_CK(ensure(ctx->ts, (size_t)3 * M * 8), "alloc ts");
        ph_begin(ctx, TC_PH_TARGETS);
        TC_CK(launch_keys(targets, M, ptr<double>(ctx->root), ptr<uint64_t>(ctx->tkeys), ptr<int32_t>(ctx->tperm), 1, s),
              "target keys");
        TC_CK(radix_sort(ptr<uint64_t>(ctx->tkeys), ptr<int32_t>(ctx->tperm), ptr<uint64_t>(ctx->tkeys_alt),
                         ptr<int32_t>(ctx->tperm_alt), ptr<uint32_t>(ctx->hist), M, s),
              "target sort");
        TC_CK(launch_gather3(targets, ptr<int32_t>(ctx->tperm), M, ptr<double>(ctx->ts), s), "gather targets");
        ph_end(ctx, TC_PH_TARGETS);
        ts = ptr<double>(ctx->ts);
        ctx->eval_self = 0;
    }
    const int64_t nbatch = (M + kBatch - 1) / kBatch;
    TC_CK(ensure(ctx->nfar_e, (size_t)nbatch * 4), "alloc lists");
    TC_CK(ensure(ctx->nnear_e, (size_t)nbatch * 4), "alloc lists");
    TC_CK(ensure(ctx->far_off, (size_t)(nbatch + 1) * 8), "alloc lists");
    TC_CK(ensure(ctx->near_off, (size_t)(nbatch + 1) * 8), "alloc lists");
    TC_CK(ensure(ctx->cnt_far, (size_t)M * 8), "alloc counts");
    TC_CK(ensure(ctx->cnt_near, (size_t)M * 8), "alloc counts");
    TC_CK(ensure(ctx->u_far, (size_t)3 * M * 8), "alloc u");
    TC_CK(ensure(ctx->u_near, (size_t)3 * M * 8), "alloc u");
    TC_CK(cudaMemsetAsync(ctx->flags.p, 0, 4, s), "flags");
    const int4* topo = ptr<int4>(ctx->node_topo);
    const Geo* geo = ptr<Geo>(ctx->node_geo);
    const float4* geof = ptr<float4>(ctx->node_geof);
    // squared magnitude bound of the cluster centres (all inside the root box)
    double S = 0.0;
    for (int a = 0; a < 3; a++) S = std::max(S, std::max(std::fabs(ctx->lo[a]), std::fabs(ctx->lo[a] + ctx->side)));
    const float scale2 = (float)(S * S);
    ph_begin(ctx, TC_PH_LISTS);
    TC_CK(launch_lists(ts, M, topo, geo, geof, scale2, theta, 0, ptr<int32_t>(ctx->nfar_e),
                       ptr<int32_t>(ctx->nnear_e), nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                       ptr<int32_t>(ctx->flags), s),
          "list count");
    int64_t* far_off = ptr<int64_t>(ctx->far_off);
    int64_t* near_off = ptr<int64_t>(ctx->near_off);
    TC_CK(launch_scan_i32_to_i64(ptr<int32_t>(ctx->nfar_e), far_off, nbatch, far_off + nbatch, s), "far scan");
    TC_CK(launch_scan_i32_to_i64(ptr<int32_t>(ctx->nnear_e), near_off, nbatch, near_off + nbatch, s), "near scan");
    if (!ctx->host_words) TC_CK(cudaMallocHost((void**)&ctx->host_words, 4 * sizeof(int64_t)), "host words");
    TC_CK(cudaMemcpyAsync(&ctx->host_words[0], far_off + nbatch, 8, cudaMemcpyDeviceToHost, s), "list totals");
    TC_CK(cudaMemcpyAsync(&ctx->host_words[1], near_off + nbatch, 8, cudaMemcpyDeviceToHost, s), "list totals");
    ctx->host_words[2] = 0;
    TC_CK(cudaMemcpyAsync(&ctx->host_words[2], ctx->flags.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "flags");
    ctx->pending_theta = theta;
    ctx->pending_p = p;
    ctx->pending_ts = ts;
    ctx->pending_M = M;
    ctx->counted = 1;
    return TC_OK;
}

// The rest of eval_prepare once the totals are on the host: the write pass of
// the traversal and the contraction tables.
tc_status tc::eval_prepare_finish(tc_ctx* ctx)
{
    if (!ctx->counted) return fail(ctx, TC_ESTATE, "tc_eval: lists were not counted");
    ctx->counted = 0;
    tc_status st = TC_OK;
    cudaStream_t s = ctx->stream;
    const int64_t M = ctx->pending_M;
    const int p = ctx->pending_p;
    const double theta = ctx->pending_theta;
    const double* ts = ctx->pending_ts;
    const int32_t f = (int32_t)ctx->host_words[2];
    if (f & kFlagStack) return fail(ctx, TC_EDEVICE, "device check: traversal stack bound exceeded");
    if (f) return fail(ctx, TC_EDEVICE, "device check: flags 0x%x", f);
    const int64_t tot[2] = {ctx->host_words[0], ctx->host_words[1]};
    const int4* topo = ptr<int4>(ctx->node_topo);
    const Geo* geo = ptr<Geo>(ctx->node_geo);
    const float4* geof = ptr<float4>(ctx->node_geof);
    double S = 0.0;
    for (int a = 0; a < 3; a++) S = std::max(S, std::max(std::fabs(ctx->lo[a]), std::fabs(ctx->lo[a] + ctx->side)));
    const float scale2 = (float)(S * S);
    int64_t* far_off = ptr<int64_t>(ctx->far_off);
    int64_t* near_off = ptr<int64_t>(ctx->near_off);
    TC_CK(ensure(ctx->far_list, (size_t)(tot[0] > 0 ? tot[0] : 1) * sizeof(ListEntry)), "alloc far list");
    TC_CK(ensure(ctx->near_list, (size_t)(tot[1] > 0 ? tot[1] : 1) * sizeof(ListEntry)), "alloc near list");
    TC_CK(launch_lists(ts, M, topo, geo, geof, scale2, theta, 1, nullptr, nullptr, far_off, near_off,
                       ptr<ListEntry>(ctx->far_list), ptr<ListEntry>(ctx->near_list), ptr<int64_t>(ctx->cnt_far),
                       ptr<int64_t>(ctx->cnt_near), ptr<int32_t>(ctx->flags), s),
          "list write");
    ph_end(ctx, TC_PH_LISTS);
    // The tables read the moments.  While the moment passes are still in
    // flight on the second stream, the tables follow them there: the far
    // field, which reads them, runs on that stream too, and the near field,
    // which needs neither, starts on the first stream right after the lists.
    // The moment event then marks the end of the tables.
    if (ctx->mom_pending) {
        st = ensure_tables(ctx, p, ctx->stream2);
        if (st != TC_OK) return st;
        TC_CK(cudaEventRecord(ctx->ev_mom, ctx->stream2), "tables done");
    } else {
        st = ensure_tables(ctx, p, s);
        if (st != TC_OK) return st;
    }
    ctx->M = M;
    ctx->far_entries = tot[0];
    ctx->near_entries = tot[1];
    ctx->p_eval = p;
    ctx->prepared = 1;
    return TC_OK;
}

// Second half of tc_eval: far field, near field, sum and scatter to u.
tc_status tc::eval_compute(tc_ctx* ctx, double* u)
{
    if (!ctx->prepared) return fail(ctx, TC_ESTATE, "tc_eval: lists are not prepared");
    cudaStream_t s = ctx->stream;
    const int64_t M = ctx->M;
    const int p = ctx->p_eval;
    const double* ts = ctx->eval_self ? ptr<double>(ctx->xs) : ptr<double>(ctx->ts);
    const int32_t* tperm = ctx->eval_self ? ptr<int32_t>(ctx->perm) : ptr<int32_t>(ctx->tperm);
    // the far and near fields are independent: the far field runs on the
    // context's second stream (after the moments and tables, when those are
    // still in flight there), forked from and joined back to the first
    TC_CK(second_stream(ctx), "second stream");
    // profile mode 2: serialised, so that each phase time is one kernel's own
    if (ctx->profile == 2) TC_CK(join_moments(ctx), "join moments");
    cudaStream_t s2 = ctx->profile == 2 ? s : ctx->stream2;
    TC_CK(cudaEventRecord(ctx->ev_fork, s), "fork");
    TC_CK(cudaStreamWaitEvent(s2, ctx->ev_fork, 0), "fork");
    ph_begin(ctx, TC_PH_FAR, s2);
    if (ctx->reg_eps > 0.0 && ctx->precision == TC_MIXED && !(ctx->rec64 && p >= 8))
        TC_CK(launch_far_reg32(ts, M, ptr<float4>(ctx->geo32), ptr<float>(ctx->ab32), ptr<float>(ctx->reg_et32), p,
                               ctx->reg_eps, ptr<int64_t>(ctx->far_off), ptr<ListEntry>(ctx->far_list),
                               ptr<double>(ctx->u_far), s2),
              "far field");
    else if (ctx->reg_eps > 0.0)
        TC_CK(launch_far_reg(ts, M, ptr<Geo>(ctx->node_geo), ptr<double>(ctx->node_invrho), ptr<double>(ctx->ab64),
                             ptr<double>(ctx->reg_et), p, ctx->reg_eps, ptr<int64_t>(ctx->far_off),
                             ptr<ListEntry>(ctx->far_list), ptr<double>(ctx->u_far), s2),
              "far field");
    else
        TC_CK(launch_far(ctx->precision, ctx->rec64, ts, M, ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo),
                         ptr<double>(ctx->node_invrho),
                         ptr<float4>(ctx->geo32), ptr<double>(ctx->abf64), ptr<float>(ctx->abf32), p,
                         ptr<int64_t>(ctx->far_off),
                         ptr<ListEntry>(ctx->far_list), ptr<double>(ctx->u_far),
                         reinterpret_cast<unsigned*>(ptr<char>(ctx->flags) + 128), s2),
              "far field");
    ph_end(ctx, TC_PH_FAR, s2);
    TC_CK(cudaEventRecord(ctx->ev_join, s2), "join");
    ph_begin(ctx, TC_PH_NEAR);
    NearSched sched{};
    if (ctx->precision == TC_MIXED) TC_CK(near_schedule(ctx, 1, sched, s), "near schedule");
    sched.queue = reinterpret_cast<unsigned*>(ptr<char>(ctx->flags) + 160);
    TC_CK(launch_near(ctx->precision, ts, M, ptr<int4>(ctx->node_topo), ptr<double>(ctx->xs), ptr<double>(ctx->ws),
                      ptr<float4>(ctx->spack), ctx->N, ptr<int64_t>(ctx->near_off), ptr<ListEntry>(ctx->near_list),
                      ptr<double>(ctx->u_near), ctx->eval_self && !ctx->moved, sched, ctx->reg_eps, s),
          "near field");
    ph_end(ctx, TC_PH_NEAR);
    TC_CK(cudaStreamWaitEvent(s, ctx->ev_join, 0), "join");
    // the join covers everything enqueued on the second stream, the moment
    // passes and tables included
    if (s2 == ctx->stream2) ctx->mom_pending = 0;
    ph_begin(ctx, TC_PH_FINAL);
    TC_CK(launch_finalize(ptr<double>(ctx->u_far), ptr<double>(ctx->u_near), tperm, M, u, s), "finalize");
    ph_end(ctx, TC_PH_FINAL);
    ctx->have_eval = 1;
    return TC_OK;
}

extern "C" {

tc_status tc_update_positions(tc_ctx* ctx, const double* x)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_update_positions: ctx is NULL");
    if (!x) return fail(ctx, TC_EINVAL, "tc_update_positions: x is NULL");
    if (!ctx->prepared || !ctx->have_moments)
        return fail(ctx, TC_ESTATE, "tc_update_positions: call tc_eval (targets = NULL) first");
    if (!ctx->eval_self)
        return fail(ctx, TC_ESTATE, "tc_update_positions: the last tc_eval must have had targets = NULL");
    TC_CK(join_moments(ctx), "tc_update_positions");
    cudaStream_t s = ctx->stream;
    const int64_t N = ctx->N;
    // the new positions in the tree's order; cells, centres, radii and the
    // interaction lists of the last tc_eval stay as they are
    TC_CK(launch_gather3(x, ptr<int32_t>(ctx->perm), N, ptr<double>(ctx->xs), s), "gather x");
    if (ctx->precision == TC_MIXED)
        TC_CK(launch_source_pack(ptr<double>(ctx->xs), ptr<double>(ctx->ws), N, ptr<float4>(ctx->spack), s), "pack");
    // moments of the moved particles about the unchanged centres, then the tables
    TC_CK(launch_moments(ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo), ptr<double>(ctx->xs),
                         ptr<double>(ctx->ws), N, ctx->nnodes, ctx->p_mom, ptr<double>(ctx->mom), ctx->mom_tmp.p, 0, s),
          "moments");
    for (int L = (int)ctx->level_begin.size() - 3; L >= 0; L--)
        TC_CK(launch_m2m(ptr<int4>(ctx->node_topo), ptr<Geo>(ctx->node_geo), ctx->level_begin[L],
                         ctx->level_begin[L + 1], ctx->level_begin[L + 1], ctx->p_mom, ptr<double>(ctx->mom),
                         ptr<double>(ctx->m2m_tmp), s),
              "m2m");
    ctx->ab_p = -1;
    tc_status st = ensure_tables(ctx, ctx->p_eval, s);
    if (st != TC_OK) return st;
    ctx->moved = 1;
    ctx->have_eval = 0;
    return TC_OK;
}

tc_status tc_eval_frozen(tc_ctx* ctx, double* u)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_eval_frozen: ctx is NULL");
    if (!u) return fail(ctx, TC_EINVAL, "tc_eval_frozen: u is NULL");
    if (!ctx->prepared) return fail(ctx, TC_ESTATE, "tc_eval_frozen: call tc_eval first");
    return eval_compute(ctx, u);
}

tc_status tc_velocity_host(tc_ctx* ctx, const double* x, const double* f, const double* h, const double* nu,
                           int64_t N, int32_t N0, double theta, int32_t p, double* u)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_velocity_host: ctx is NULL");
    if (!x || !f || !h || !nu || !u) return fail(ctx, TC_EINVAL, "tc_velocity_host: a host pointer is NULL");
    if (N < 1 || N >= ((int64_t)1 << 31))
        return fail(ctx, TC_EINVAL, "tc_velocity_host: N = %lld out of [1, 2^31)", (long long)N);
    if (N0 < 1) return fail(ctx, TC_EINVAL, "tc_velocity_host: N0 = %d must be >= 1", N0);
    if (!(theta > 0.0 && theta < 1.0)) return fail(ctx, TC_EINVAL, "tc_velocity_host: theta = %g out of (0, 1)", theta);
    if (p < 0 || p > kPMax) return fail(ctx, TC_EINVAL, "tc_velocity_host: p = %d out of [0, %d]", p, kPMax);
    // the staging buffers may still be read by moment passes of an earlier call
    TC_CK(join_moments(ctx), "tc_velocity_host");
    cudaStream_t s = ctx->stream;
    const size_t b3 = (size_t)3 * N * sizeof(double);
    TC_CK(ensure(ctx->host_in, 4 * b3), "alloc staging");
    TC_CK(ensure(ctx->host_u, b3), "alloc staging");
    double* d_in = ptr<double>(ctx->host_in);
    const double* src[4] = {x, f, h, nu};
    for (int a = 0; a < 4; a++)
        TC_CK(cudaMemcpyAsync(d_in + (size_t)a * 3 * N, src[a], b3, cudaMemcpyHostToDevice, s), "copy in");
    tc_status st = tc_build(ctx, d_in, N, N0);
    if (st == TC_OK) st = tc_moments(ctx, d_in + 3 * N, d_in + 6 * N, d_in + 9 * N, p);
    if (st == TC_OK) st = tc_eval(ctx, nullptr, N, theta, p, ptr<double>(ctx->host_u));
    if (st != TC_OK) return st;
    TC_CK(cudaMemcpyAsync(u, ctx->host_u.p, b3, cudaMemcpyDeviceToHost, s), "copy out");
    return tc_sync(ctx);
}

tc_status tc_eval(tc_ctx* ctx, const double* targets, int64_t M, double theta, int32_t p, double* u)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_eval: ctx is NULL");
    if (!ctx->have_moments) return fail(ctx, TC_ESTATE, "tc_eval: call tc_build and tc_moments first");
    if (!u) return fail(ctx, TC_EINVAL, "tc_eval: u is NULL");
    tc_status st = eval_prepare(ctx, targets, M, theta, p);
    if (st != TC_OK) return st;
    return eval_compute(ctx, u);
}

static tc_status direct_impl(const char* name, const double* x, const double* f, const double* h, const double* nu,
                             int64_t N, const double* targets, int64_t M, double eps, int32_t precision, void* stream,
                             double* u)
{
    tc_ctx* ctx = nullptr;
    if (!x || !f || !h || !nu || !u) return fail(nullptr, TC_EINVAL, "%s: a pointer is NULL", name);
    if (N < 1 || N >= ((int64_t)1 << 31)) return fail(nullptr, TC_EINVAL, "%s: N out of range", name);
    if (!targets && M != N) return fail(nullptr, TC_EINVAL, "%s: targets = NULL requires M = N", name);
    if (M < 1 || M >= ((int64_t)1 << 31)) return fail(nullptr, TC_EINVAL, "%s: M out of range", name);
    if (precision != TC_FP64 && precision != TC_MIXED) return fail(nullptr, TC_EINVAL, "%s: unknown precision", name);
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = direct_scratch_bytes(precision, N, M);
    void* scratch = nullptr;
    TC_CK(alloc_should_fail() ? cudaErrorMemoryAllocation : cudaMallocAsync(&scratch, bytes, s), "direct scratch");
    cudaError_t e = launch_direct(precision, x, f, h, nu, N, targets ? targets : x, M, u, scratch, bytes, eps, s);
    cudaError_t e2 = cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, name);
    if (e2 != cudaSuccess) return cuda_fail(nullptr, e2, "direct free");
    return TC_OK;
}

tc_status tc_direct(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                    const double* targets, int64_t M, int32_t precision, void* stream, double* u)
{
    return direct_impl("tc_direct", x, f, h, nu, N, targets, M, 0.0, precision, stream, u);
}

tc_status tc_direct_reg(const double* x, const double* f, const double* h, const double* nu, int64_t N,
                        const double* targets, int64_t M, double eps, int32_t precision, void* stream, double* u)
{
    if (!(eps > 0.0) || !std::isfinite(eps))
        return fail(nullptr, TC_EINVAL, "tc_direct_reg: eps = %g must be positive and finite", eps);
    return direct_impl("tc_direct_reg", x, f, h, nu, N, targets, M, eps, precision, stream, u);
}

tc_status tc_stats(tc_ctx* ctx, int64_t* near_pairs, int64_t* far_interactions, int64_t* clusters)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_stats: ctx is NULL");
    if (clusters) *clusters = ctx->built ? ctx->nnodes : 0;
    if (!near_pairs && !far_interactions) return TC_OK;
    if (!ctx->have_eval) return fail(ctx, TC_ESTATE, "tc_stats: no evaluation yet");
    cudaStream_t s = ctx->stream;
    int64_t* tmp = ptr<int64_t>(ctx->scan_tmp);
    TC_CK(launch_sum_i64(ptr<int64_t>(ctx->cnt_near), ctx->M, tmp, s), "stats");
    TC_CK(launch_sum_i64(ptr<int64_t>(ctx->cnt_far), ctx->M, tmp + 1, s), "stats");
    int64_t h[2];
    TC_CK(cudaMemcpyAsync(h, tmp, 16, cudaMemcpyDeviceToHost, s), "stats copy");
    TC_CK(cudaStreamSynchronize(s), "stats sync");
    if (near_pairs) *near_pairs = h[0];
    if (far_interactions) *far_interactions = h[1];
    return TC_OK;
}

tc_status tc_list_stats(tc_ctx* ctx, int64_t* far_entries, int64_t* near_entries, int64_t* near_entry_sources)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_list_stats: ctx is NULL");
    if (!ctx->have_eval) return fail(ctx, TC_ESTATE, "tc_list_stats: no evaluation yet");
    if (far_entries) *far_entries = ctx->far_entries;
    if (near_entries) *near_entries = ctx->near_entries;
    if (near_entry_sources) {
        int64_t* tmp = ptr<int64_t>(ctx->scan_tmp) + 2;
        TC_CK(launch_sum_entry_sizes(ptr<ListEntry>(ctx->near_list), ctx->near_entries, ptr<int4>(ctx->node_topo), tmp,
                                     ctx->stream),
              "list stats");
        TC_CK(cudaMemcpyAsync(near_entry_sources, tmp, 8, cudaMemcpyDeviceToHost, ctx->stream), "list stats copy");
        TC_CK(cudaStreamSynchronize(ctx->stream), "list stats sync");
    }
    return TC_OK;
}

tc_status tc_eval_counts(tc_ctx* ctx, int64_t* nfar, int64_t* nnear_pairs)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_eval_counts: ctx is NULL");
    if (!ctx->have_eval) return fail(ctx, TC_ESTATE, "tc_eval_counts: no evaluation yet");
    const int32_t* perm = ctx->eval_self ? ptr<int32_t>(ctx->perm) : ptr<int32_t>(ctx->tperm);
    if (nfar) TC_CK(launch_scatter_counts(ptr<int64_t>(ctx->cnt_far), perm, ctx->M, nfar, ctx->stream), "counts");
    if (nnear_pairs)
        TC_CK(launch_scatter_counts(ptr<int64_t>(ctx->cnt_near), perm, ctx->M, nnear_pairs, ctx->stream), "counts");
    return TC_OK;
}

tc_status tc_tree_info(tc_ctx* ctx, int64_t* nnodes, int32_t* depth, double* lo, double* side)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_tree_info: ctx is NULL");
    if (!ctx->built) return fail(ctx, TC_ESTATE, "tc_tree_info: no tree");
    if (nnodes) *nnodes = ctx->nnodes;
    if (depth) *depth = ctx->depth;
    if (lo)
        for (int a = 0; a < 3; a++) lo[a] = ctx->lo[a];
    if (side) *side = ctx->side;
    return TC_OK;
}

static uint32_t host_compact3(uint64_t x)
{
    uint32_t v = 0;
    for (int j = 0; j < 21; j++) v |= (uint32_t)((x >> (3 * j)) & 1u) << j;
    return v;
}

tc_status tc_tree_export(tc_ctx* ctx, int32_t* begin, int32_t* count, int32_t* level, int32_t* cell, int32_t* parent,
                         int32_t* first_child, int32_t* nchild, double* yc, double* rc2)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_tree_export: ctx is NULL");
    if (!ctx->built) return fail(ctx, TC_ESTATE, "tc_tree_export: no tree");
    const int64_t n = ctx->nnodes;
    std::vector<int4> topo(n), info(n);
    std::vector<uint64_t> key(n);
    std::vector<Geo> geo(n);
    cudaStream_t s = ctx->stream;
    TC_CK(cudaMemcpyAsync(topo.data(), ctx->node_topo.p, n * sizeof(int4), cudaMemcpyDeviceToHost, s), "export");
    TC_CK(cudaMemcpyAsync(info.data(), ctx->node_info.p, n * sizeof(int4), cudaMemcpyDeviceToHost, s), "export");
    TC_CK(cudaMemcpyAsync(key.data(), ctx->node_key.p, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, s), "export");
    TC_CK(cudaMemcpyAsync(geo.data(), ctx->node_geo.p, n * sizeof(Geo), cudaMemcpyDeviceToHost, s), "export");
    TC_CK(cudaStreamSynchronize(s), "export sync");
    for (int64_t i = 0; i < n; i++) {
        if (begin) begin[i] = topo[i].x;
        if (count) count[i] = topo[i].y;
        if (first_child) first_child[i] = topo[i].z;
        if (nchild) nchild[i] = topo[i].w;
        if (level) level[i] = info[i].x;
        if (parent) parent[i] = info[i].y;
        if (cell) {
            int L = info[i].x;
            cell[3 * i + 0] = (int32_t)(host_compact3(key[i] >> 2) >> (kMaxDepth - L));
            cell[3 * i + 1] = (int32_t)(host_compact3(key[i] >> 1) >> (kMaxDepth - L));
            cell[3 * i + 2] = (int32_t)(host_compact3(key[i]) >> (kMaxDepth - L));
        }
        if (yc) {
            yc[3 * i + 0] = geo[i].x;
            yc[3 * i + 1] = geo[i].y;
            yc[3 * i + 2] = geo[i].z;
        }
        if (rc2) rc2[i] = geo[i].w;
    }
    return TC_OK;
}

tc_status tc_tree_order(tc_ctx* ctx, int32_t* order)
{
    if (!ctx || !order) return fail(ctx, TC_EINVAL, "tc_tree_order: NULL argument");
    if (!ctx->built) return fail(ctx, TC_ESTATE, "tc_tree_order: no tree");
    TC_CK(cudaMemcpyAsync(order, ctx->perm.p, ctx->N * 4, cudaMemcpyDeviceToHost, ctx->stream), "order");
    TC_CK(cudaStreamSynchronize(ctx->stream), "order sync");
    return TC_OK;
}

tc_status tc_moments_export(tc_ctx* ctx, int64_t node, double* Mf, double* Mt)
{
    if (!ctx) return fail(nullptr, TC_EINVAL, "tc_moments_export: ctx is NULL");
    if (!ctx->have_moments) return fail(ctx, TC_ESTATE, "tc_moments_export: no moments");
    if (node < 0 || node >= ctx->nnodes) return fail(ctx, TC_EINVAL, "tc_moments_export: node out of range");
    TC_CK(join_moments(ctx), "moments export");
    const int p = ctx->p_mom, C = ncoef(p), q1 = p + 1;
    std::vector<double> m((size_t)12 * C);
    TC_CK(cudaMemcpyAsync(m.data(), ptr<double>(ctx->mom) + node * 12 * C, m.size() * 8, cudaMemcpyDeviceToHost,
                          ctx->stream),
          "moments export");
    TC_CK(cudaStreamSynchronize(ctx->stream), "moments export sync");
    const size_t cube = (size_t)q1 * q1 * q1;
    if (Mf) memset(Mf, 0, 3 * cube * 8);
    if (Mt) memset(Mt, 0, 9 * cube * 8);
    for (int k1 = 0; k1 <= p; k1++)
        for (int k2 = 0; k1 + k2 <= p; k2++)
            for (int k3 = 0; k1 + k2 + k3 <= p; k3++) {
                int idx = flat_index(k1, k2, k3);
                size_t o = ((size_t)k1 * q1 + k2) * q1 + k3;
                for (int c = 0; c < 3; c++)
                    if (Mf) Mf[c * cube + o] = m[(size_t)c * C + idx];
                for (int c = 0; c < 9; c++)
                    if (Mt) Mt[c * cube + o] = m[(size_t)(3 + c) * C + idx];
            }
    return TC_OK;
}

}  // extern "C"
