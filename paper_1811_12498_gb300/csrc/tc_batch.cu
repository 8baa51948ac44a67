// Batched evaluation of many independent particle systems.
//
// A batch holds one context per system.  tc_batch_build / tc_batch_moments
// split the caller's segmented arrays into per-system ones and run the
// ordinary build and moments.  tc_batch_eval prepares every system's
// interaction lists, then runs the far field, near field and the final sum of
// ALL systems as one far and one near persistent kernel (each warp takes
// items from a device counter until the queue is empty: (system, batch) items
// in the far field, the units of the systems' leaf-major schedules in the
// near field, whose builds run beside the far field on a second stream) plus
// the batched sums and finalize, captured once into a CUDA graph and
// replayed.  The launch shapes of the two persistent kernels come from a
// small autotuner that times candidate shapes on the first evaluation of each
// (order, precision) and keeps the fastest.
#include <algorithm>
#include <new>

#include "tc_internal.cuh"

namespace tc {
namespace {

// segmented (3, ntot) -> per-system blocks [s][3][n_s] back to back
__global__ void k_split_segments(const double* __restrict__ src, const int64_t* __restrict__ off, int nsys,
                                 int64_t ntot, double* __restrict__ dst)
{
    const int64_t gi = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gi >= ntot) return;
    int lo = 0, hi = nsys;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= gi)
            lo = mid;
        else
            hi = mid;
    }
    const int64_t n = off[lo + 1] - off[lo], i = gi - off[lo];
    double* d = dst + 3 * off[lo];
    for (int a = 0; a < 3; a++) d[a * n + i] = src[a * ntot + gi];
}

inline unsigned grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    return (unsigned)(g > 0 ? g : 1);
}

struct Shape {
    int far_warps = 1, far_blocks = 0, near_warps = 4, near_blocks = 0;
};

}  // namespace
}  // namespace tc

using namespace tc;

struct tc_batch {
    tc_config cfg{};
    int autotune = 1;
    std::string err = "no error";
    int nsys = 0;
    int64_t ntot = 0;
    std::vector<int64_t> off;          // nsys + 1 host offsets
    std::vector<tc_ctx*> ctx;
    // each system's context works on a stream of its own, forked from and
    // joined back to the batch's stream, so that the small launches of many
    // systems' preparation run side by side
    std::vector<cudaStream_t> sys_stream;
    std::vector<cudaEvent_t> sys_ev;
    DevBuf d_off;                      // device copy of off
    DevBuf xseg, fseg, hseg, nuseg;    // per-system copies
    DevBuf desc;                       // SysDesc[nsys]
    DevBuf item_off;                   // far item offsets (nsys + 1), then batch offsets (nsys + 1)
    DevBuf unit_off;                   // the systems' first near-field units (nsys + 1)
    DevBuf counters;                   // two queue counters
    std::vector<SysDesc> hdesc;
    std::vector<int64_t> hitem;
    // tuned shapes keyed by (p, precision)
    int tuned_p = -1;
    Shape shape;
    float tune_ms[2] = {0, 0};
    // captured graph of the compute phase
    cudaGraphExec_t exec = nullptr;
    double* graph_u = nullptr;
    int graph_p = -1;
    int64_t graph_items = -1;
    Shape graph_shape;
    std::vector<SysDesc> graph_desc;
    int use_graph = 1;
    // graphs cannot be captured on the legacy default stream, so the compute
    // phase is captured and replayed on a private stream, ordered after the
    // caller's stream by events
    cudaStream_t cap = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // second stream of the compute phase: the near-field schedules' builds
    cudaStream_t cap2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

static tc_status bfail(tc_batch* b, tc_status st, const char* msg, cudaError_t e = cudaSuccess)
{
    char buf[512];
    if (e != cudaSuccess)
        snprintf(buf, sizeof(buf), "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof(buf), "%s", msg);
    b->err = buf;
    if (e == cudaErrorMemoryAllocation) return TC_ENOMEM;
    return st;
}

#define TB_CK(call, where)                                               \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return bfail(b, TC_ECUDA, where, e_);     \
    } while (0)

static tc_status from_ctx(tc_batch* b, tc_ctx* c, tc_status st, int s)
{
    char buf[640];
    snprintf(buf, sizeof(buf), "system %d: %s", s, tc_last_error(c));
    b->err = buf;
    return st;
}

static void drop_graph(tc_batch* b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->graph_u = nullptr;
}

static void free_systems(tc_batch* b)
{
    for (tc_ctx* c : b->ctx) tc_destroy(c);
    b->ctx.clear();
    for (cudaStream_t q : b->sys_stream) cudaStreamDestroy(q);
    for (cudaEvent_t e : b->sys_ev) cudaEventDestroy(e);
    b->sys_stream.clear();
    b->sys_ev.clear();
}

// order systems [s0, s1)'s streams after the work enqueued so far on st
static cudaError_t fork_systems(tc_batch* b, cudaStream_t st, int s0, int s1)
{
    cudaError_t e = cudaEventRecord(b->ev_in, st);
    for (int s = s0; s < s1 && e == cudaSuccess; s++) e = cudaStreamWaitEvent(b->sys_stream[s], b->ev_in, 0);
    return e;
}

// order st after everything enqueued on systems [s0, s1)'s streams (their
// moment passes included)
static cudaError_t join_systems(tc_batch* b, cudaStream_t st, int s0, int s1)
{
    cudaError_t e = cudaSuccess;
    for (int s = s0; s < s1 && e == cudaSuccess; s++) {
        e = join_moments(b->ctx[s]);
        if (e == cudaSuccess) e = cudaEventRecord(b->sys_ev[s], b->sys_stream[s]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->sys_ev[s], 0);
    }
    return e;
}

// the near-field schedules of all systems (mixed precision; no allocation)
static tc_status build_schedules(tc_batch* b, cudaStream_t s)
{
    for (int i = 0; i < b->nsys; i++) TB_CK(near_schedule_build(b->ctx[i], 1, s), "near schedule");
    return TC_OK;
}

// far + near + finalize of all systems (stream-ordered; capturable).  In
// mixed precision the near field runs on the second stream, after its
// schedules' builds and beside the far field, as in tc_eval.
static tc_status launch_compute(tc_batch* b, const Shape& sh, int p, int64_t nitems, int64_t nnear, double* u,
                                cudaStream_t s)
{
    unsigned long long* cnt = ptr<unsigned long long>(b->counters);
    TB_CK(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), s), "reset queue");
    const SysDesc* d = ptr<SysDesc>(b->desc);
    const int64_t* io = ptr<int64_t>(b->item_off);
    const bool mixed = b->cfg.precision == TC_MIXED;
    cudaStream_t sn = s;
    if (mixed) {
        sn = b->cap2;
        TB_CK(cudaEventRecord(b->ev_fork, s), "fork");
        TB_CK(cudaStreamWaitEvent(sn, b->ev_fork, 0), "fork");
        tc_status r = build_schedules(b, sn);
        if (r != TC_OK) return r;
    }
    TB_CK(launch_far_batched(b->cfg.precision, b->cfg.rec64, d, b->nsys, io, nitems, p, cnt, sh.far_warps,
                             sh.far_blocks, s),
          "batched far field");
    TB_CK(launch_near_batched(b->cfg.precision, d, b->nsys, io + b->nsys + 1, nnear, ptr<int64_t>(b->unit_off),
                              cnt + 1, sh.near_warps, sh.near_blocks, sn),
          "batched near field");
    if (mixed) {
        TB_CK(cudaEventRecord(b->ev_join, sn), "join");
        TB_CK(cudaStreamWaitEvent(s, b->ev_join, 0), "join");
    }
    TB_CK(launch_finalize_batched(d, b->nsys, ptr<int64_t>(b->d_off), b->ntot, u, b->ntot, s), "batched finalize");
    return TC_OK;
}

static int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

// Time each candidate shape of one kernel on the real work and keep the best.
static tc_status tune(tc_batch* b, int p, int64_t nitems, int64_t nnear, double* u)
{
    cudaStream_t s = (cudaStream_t)b->cfg.stream;
    const int sms = sm_count();
    cudaEvent_t e0, e1;
    TB_CK(cudaEventCreate(&e0), "tune event");
    TB_CK(cudaEventCreate(&e1), "tune event");
    unsigned long long* cnt = ptr<unsigned long long>(b->counters);
    const SysDesc* d = ptr<SysDesc>(b->desc);
    const int64_t* io = ptr<int64_t>(b->item_off);
    Shape best;
    float best_far = 1e30f, best_near = 1e30f;
    // far: warps per block x blocks per SM (0 = occupancy limit)
    const int far_w[] = {1, 2};
    const int far_b[] = {0, 2, 4};
    for (int fw : far_w)
        for (int fb : far_b) {
            const int blocks = fb ? fb * sms : 0;
            cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
            cudaEventRecord(e0, s);
            cudaError_t e =
                launch_far_batched(b->cfg.precision, b->cfg.rec64, d, b->nsys, io, nitems, p, cnt, fw, blocks, s);
            cudaEventRecord(e1, s);
            if (e != cudaSuccess) {
                cudaGetLastError();  // a shape that does not fit is skipped
                continue;
            }
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_far) {
                best_far = ms;
                best.far_warps = fw;
                best.far_blocks = blocks;
            }
        }
    const int near_w[] = {2, 4, 8};
    const int near_b[] = {0, 4, 8};
    for (int nw : near_w)
        for (int nb : near_b) {
            const int blocks = nb ? nb * sms : 0;
            cudaMemsetAsync(cnt + 1, 0, sizeof(unsigned long long), s);
            cudaEventRecord(e0, s);
            cudaError_t e = launch_near_batched(b->cfg.precision, d, b->nsys, io + b->nsys + 1, nnear,
                                                ptr<int64_t>(b->unit_off), cnt + 1, nw, blocks, s);
            cudaEventRecord(e1, s);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_near) {
                best_near = ms;
                best.near_warps = nw;
                best.near_blocks = blocks;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_far >= 1e30f || best_near >= 1e30f) return bfail(b, TC_ECUDA, "autotune: no launch shape ran");
    b->shape = best;
    b->tune_ms[0] = best_far;
    b->tune_ms[1] = best_near;
    b->tuned_p = p;
    (void)u;
    return TC_OK;
}

static bool same_desc(const std::vector<SysDesc>& a, const std::vector<SysDesc>& c)
{
    if (a.size() != c.size()) return false;
    return std::equal(a.begin(), a.end(), c.begin(), [](const SysDesc& x, const SysDesc& y) {
        return memcmp(&x, &y, sizeof(SysDesc)) == 0;
    });
}

extern "C" {

tc_status tc_batch_create(tc_batch** out, const tc_config* cfg)
{
    if (!out) return fail(nullptr, TC_EINVAL, "tc_batch_create: out is NULL");
    *out = nullptr;
    tc_config c = {TC_MIXED, 1, nullptr, 0, 0, 0.0};
    if (cfg) c = *cfg;
    if (c.precision != TC_FP64 && c.precision != TC_MIXED)
        return fail(nullptr, TC_EINVAL, "tc_batch_create: unknown precision %d", c.precision);
    if (c.reg_eps != 0.0) return fail(nullptr, TC_EINVAL, "tc_batch_create: batches use the kernels of eqs. (1.2a,b)");
    if (c.shrink != 0 && c.shrink != 1) return fail(nullptr, TC_EINVAL, "tc_batch_create: shrink must be 0 or 1");
    if (c.rec64 != 0 && c.rec64 != 1) return fail(nullptr, TC_EINVAL, "tc_batch_create: rec64 must be 0 or 1");
    tc_batch* b = new (std::nothrow) tc_batch();
    if (!b) return fail(nullptr, TC_ENOMEM, "tc_batch_create: out of host memory");
    b->cfg = c;
    b->cfg.reserved1 = 0;
    if (b->cfg.precision != TC_MIXED) b->cfg.rec64 = 0;
    cudaError_t e = ensure(b->counters, 256);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        tc_batch_destroy(b);
        return fail(nullptr, TC_ECUDA, "tc_batch_create: %s", cudaGetErrorString(e));
    }
    *out = b;
    return TC_OK;
}

tc_status tc_batch_destroy(tc_batch* b)
{
    if (!b) return TC_OK;
    cudaStreamSynchronize((cudaStream_t)b->cfg.stream);
    drop_graph(b);
    free_systems(b);
    DevBuf* bufs[] = {&b->d_off, &b->xseg,     &b->fseg,     &b->hseg,    &b->nuseg,
                      &b->desc,  &b->item_off, &b->unit_off, &b->counters};
    for (DevBuf* d : bufs) release(*d);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->cap2) cudaStreamDestroy(b->cap2);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
    return TC_OK;
}

const char* tc_batch_last_error(const tc_batch* b) { return b ? b->err.c_str() : tc_last_error(nullptr); }

tc_status tc_batch_set(tc_batch* b, int32_t autotune, int32_t use_graph)
{
    if (!b) return fail(nullptr, TC_EINVAL, "tc_batch_set: batch is NULL");
    b->autotune = autotune ? 1 : 0;
    b->use_graph = use_graph ? 1 : 0;
    if (!b->use_graph) drop_graph(b);
    return TC_OK;
}

tc_status tc_batch_build(tc_batch* b, const double* x, int32_t nsys, const int64_t* offsets, int32_t N0)
{
    if (!b) return fail(nullptr, TC_EINVAL, "tc_batch_build: batch is NULL");
    if (!x || !offsets) return bfail(b, TC_EINVAL, "tc_batch_build: NULL argument");
    if (nsys < 1) return bfail(b, TC_EINVAL, "tc_batch_build: nsys must be >= 1");
    if (offsets[0] != 0) return bfail(b, TC_EINVAL, "tc_batch_build: offsets[0] must be 0");
    for (int s = 0; s < nsys; s++)
        if (offsets[s + 1] <= offsets[s]) return bfail(b, TC_EINVAL, "tc_batch_build: every system needs >= 1 particle");
    cudaStream_t st = (cudaStream_t)b->cfg.stream;
    drop_graph(b);
    if ((int)b->ctx.size() != nsys) {
        free_systems(b);
        for (int s = 0; s < nsys; s++) {
            cudaStream_t q = nullptr;
            cudaEvent_t ev = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->sys_stream.push_back(q);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->sys_ev.push_back(ev);
            if (e != cudaSuccess) {
                free_systems(b);
                return bfail(b, TC_ECUDA, "system stream", e);
            }
            tc_config cs = b->cfg;
            cs.stream = q;
            tc_ctx* c = nullptr;
            tc_status r = tc_create(&c, &cs);
            if (r != TC_OK) {
                free_systems(b);
                return bfail(b, r, tc_last_error(nullptr));
            }
            b->ctx.push_back(c);
        }
    }
    b->nsys = nsys;
    b->off.assign(offsets, offsets + nsys + 1);
    b->ntot = offsets[nsys];
    TB_CK(ensure(b->d_off, (size_t)(nsys + 1) * 8), "alloc offsets");
    TB_CK(cudaMemcpyAsync(b->d_off.p, offsets, (size_t)(nsys + 1) * 8, cudaMemcpyHostToDevice, st), "copy offsets");
    TB_CK(ensure(b->xseg, (size_t)3 * b->ntot * 8), "alloc positions");
    k_split_segments<<<grid_for(b->ntot, 256), 256, 0, st>>>(x, ptr<int64_t>(b->d_off), nsys, b->ntot,
                                                              ptr<double>(b->xseg));
    note_launch();
    TB_CK(cudaGetLastError(), "split positions");
    TB_CK(fork_systems(b, st, 0, nsys), "fork systems");
    for (int s = 0; s < nsys; s++) {
        tc_status r = tc_build(b->ctx[s], ptr<double>(b->xseg) + 3 * offsets[s], offsets[s + 1] - offsets[s], N0);
        if (r != TC_OK) return from_ctx(b, b->ctx[s], r, s);
    }
    TB_CK(join_systems(b, st, 0, nsys), "join systems");
    b->tuned_p = -1;
    return TC_OK;
}

tc_status tc_batch_moments(tc_batch* b, const double* f, const double* h, const double* nu, int32_t p)
{
    if (!b) return fail(nullptr, TC_EINVAL, "tc_batch_moments: batch is NULL");
    if (b->nsys < 1) return bfail(b, TC_ESTATE, "tc_batch_moments: call tc_batch_build first");
    if (!f || !h || !nu) return bfail(b, TC_EINVAL, "tc_batch_moments: NULL argument");
    cudaStream_t st = (cudaStream_t)b->cfg.stream;
    DevBuf* segs[3] = {&b->fseg, &b->hseg, &b->nuseg};
    const double* srcs[3] = {f, h, nu};
    for (int k = 0; k < 3; k++) {
        TB_CK(ensure(*segs[k], (size_t)3 * b->ntot * 8), "alloc weights");
        k_split_segments<<<grid_for(b->ntot, 256), 256, 0, st>>>(srcs[k], ptr<int64_t>(b->d_off), b->nsys, b->ntot,
                                                                  ptr<double>(*segs[k]));
        note_launch();
    }
    TB_CK(cudaGetLastError(), "split weights");
    TB_CK(fork_systems(b, st, 0, b->nsys), "fork systems");
    for (int s = 0; s < b->nsys; s++) {
        const int64_t o = 3 * b->off[s];
        tc_status r = tc_moments(b->ctx[s], ptr<double>(b->fseg) + o, ptr<double>(b->hseg) + o,
                                 ptr<double>(b->nuseg) + o, p);
        if (r != TC_OK) return from_ctx(b, b->ctx[s], r, s);
    }
    TB_CK(join_systems(b, st, 0, b->nsys), "join systems");
    return TC_OK;
}

tc_status tc_batch_eval(tc_batch* b, double theta, int32_t p, double* u)
{
    if (!b) return fail(nullptr, TC_EINVAL, "tc_batch_eval: batch is NULL");
    if (b->nsys < 1) return bfail(b, TC_ESTATE, "tc_batch_eval: call tc_batch_build first");
    if (!u) return bfail(b, TC_EINVAL, "tc_batch_eval: u is NULL");
    cudaStream_t st = (cudaStream_t)b->cfg.stream;
    // 1. every system's tables and interaction lists, each on its system's
    // stream: the counting passes of all systems, one wait for all their
    // list sizes, then the write passes and tables
    TB_CK(fork_systems(b, st, 0, b->nsys), "fork systems");
    for (int s = 0; s < b->nsys; s++) {
        tc_status r = eval_prepare_count(b->ctx[s], nullptr, b->off[s + 1] - b->off[s], theta, p);
        if (r != TC_OK) return from_ctx(b, b->ctx[s], r, s);
    }
    for (int s = 0; s < b->nsys; s++) TB_CK(cudaStreamSynchronize(b->sys_stream[s]), "list sizes");
    for (int s = 0; s < b->nsys; s++) {
        tc_status r = eval_prepare_finish(b->ctx[s]);
        if (r != TC_OK) return from_ctx(b, b->ctx[s], r, s);
        // the buffers of its near-field schedule (built in the compute phase)
        if (b->cfg.precision == TC_MIXED) {
            cudaError_t e = near_schedule_alloc(b->ctx[s], 1);
            if (e != cudaSuccess) return bfail(b, TC_ECUDA, "near schedule", e);
            b->ctx[s]->near_sched_ready = 0;  // its work is enqueued by the batch
        }
    }
    // the persistent kernels read every system's lists and tables
    TB_CK(join_systems(b, st, 0, b->nsys), "join systems");
    // 2. descriptors and the item numbering
    b->hdesc.resize(b->nsys);
    b->hitem.assign(2 * (b->nsys + 1), 0);
    int64_t* hnear = b->hitem.data() + b->nsys + 1;
    for (int s = 0; s < b->nsys; s++) {
        tc_ctx* c = b->ctx[s];
        SysDesc& d = b->hdesc[s];
        d.ts = ptr<double>(c->xs);
        d.M = c->M;
        d.geo = ptr<Geo>(c->node_geo);
        d.invrho = ptr<double>(c->node_invrho);
        d.ab = c->precision == TC_FP64 ? c->abf64.p : c->abf32.p;  // folded tables
        d.geo32 = ptr<float4>(c->geo32);
        d.far_off = ptr<int64_t>(c->far_off);
        d.far_list = ptr<ListEntry>(c->far_list);
        d.u_far = ptr<double>(c->u_far);
        d.topo = ptr<int4>(c->node_topo);
        d.spack = ptr<float4>(c->spack);
        d.xs = ptr<double>(c->xs);
        d.ws = ptr<double>(c->ws);
        d.N = c->N;
        d.near_off = ptr<int64_t>(c->near_off);
        d.near_list = ptr<ListEntry>(c->near_list);
        d.u_near = ptr<double>(c->u_near);
        d.tperm = ptr<int32_t>(c->perm);
        d.out_off = b->off[s];
        const NearSched sc = near_schedule_desc(c);
        d.units = sc.units;
        d.nunits = sc.nunits;
        d.node_inc0 = sc.node_inc0;
        d.node_A = sc.node_A;
        d.inc_m = sc.inc_m;
        d.inc_e = sc.inc_e;
        d.slots = sc.slots;
        d.near_entries = c->near_entries;
        d.nnodes = c->nnodes;
        const int64_t nb = (c->M + kBatch - 1) / kBatch;
        b->hitem[s + 1] = b->hitem[s] + (b->cfg.precision == TC_FP64 ? nb : (nb + 1) / 2);
        hnear[s + 1] = hnear[s] + nb;
    }
    const int64_t nitems = b->hitem[b->nsys], nnear = hnear[b->nsys];
    TB_CK(ensure(b->desc, sizeof(SysDesc) * b->nsys), "alloc descriptors");
    TB_CK(ensure(b->item_off, (size_t)(b->nsys + 1) * 16), "alloc items");
    TB_CK(ensure(b->unit_off, (size_t)(b->nsys + 1) * 8), "alloc units");
    TB_CK(cudaMemcpyAsync(b->desc.p, b->hdesc.data(), sizeof(SysDesc) * b->nsys, cudaMemcpyHostToDevice, st),
          "copy descriptors");
    TB_CK(cudaMemcpyAsync(b->item_off.p, b->hitem.data(), (size_t)(b->nsys + 1) * 16, cudaMemcpyHostToDevice, st),
          "copy items");
    TB_CK(cudaStreamSynchronize(st), "descriptor sync");  // host arrays are reused next call
    // 3. launch shapes
    if (b->autotune && b->tuned_p != p) {
        // the near kernel reads the schedules: build them for the timing runs
        if (b->cfg.precision == TC_MIXED) {
            tc_status r = build_schedules(b, st);
            if (r != TC_OK) return r;
        }
        tc_status r = tune(b, p, nitems, nnear, u);
        if (r != TC_OK) return r;
    }
    // 4. compute phase: replay the captured graph, capturing it when stale
    if (!b->use_graph) return launch_compute(b, b->shape, p, nitems, nnear, u, st);
    const bool stale = !b->exec || b->graph_u != u || b->graph_p != p || b->graph_items != nitems ||
                       memcmp(&b->graph_shape, &b->shape, sizeof(Shape)) != 0 || !same_desc(b->graph_desc, b->hdesc);
    if (stale) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        TB_CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
        tc_status r = launch_compute(b, b->shape, p, nitems, nnear, u, b->cap);
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (r != TC_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return bfail(b, TC_ECUDA, "end capture", e);
        e = cudaGraphInstantiate(&b->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->exec = nullptr;
            return bfail(b, TC_ECUDA, "instantiate graph", e);
        }
        b->graph_u = u;
        b->graph_p = p;
        b->graph_items = nitems;
        b->graph_shape = b->shape;
        b->graph_desc = b->hdesc;
    }
    TB_CK(cudaEventRecord(b->ev_in, st), "order graph");
    TB_CK(cudaStreamWaitEvent(b->cap, b->ev_in, 0), "order graph");
    TB_CK(cudaGraphLaunch(b->exec, b->cap), "graph launch");
    TB_CK(cudaEventRecord(b->ev_out, b->cap), "order graph");
    TB_CK(cudaStreamWaitEvent(st, b->ev_out, 0), "order graph");
    return TC_OK;
}

tc_status tc_batch_eval_separate(tc_batch* b, double theta, int32_t p, double* const* u_sys)
{
    if (!b) return fail(nullptr, TC_EINVAL, "tc_batch_eval_separate: batch is NULL");
    if (b->nsys < 1) return bfail(b, TC_ESTATE, "tc_batch_eval_separate: call tc_batch_build first");
    if (!u_sys) return bfail(b, TC_EINVAL, "tc_batch_eval_separate: u is NULL");
    // one system after the other, each ordered after the last on the batch's stream
    cudaStream_t st = (cudaStream_t)b->cfg.stream;
    for (int s = 0; s < b->nsys; s++) {
        TB_CK(fork_systems(b, st, s, s + 1), "fork system");
        tc_status r = tc_eval(b->ctx[s], nullptr, b->off[s + 1] - b->off[s], theta, p, u_sys[s]);
        if (r != TC_OK) return from_ctx(b, b->ctx[s], r, s);
        TB_CK(join_systems(b, st, s, s + 1), "join system");
    }
    return TC_OK;
}

tc_status tc_batch_info(tc_batch* b, int32_t* shape, float* tune_ms)
{
    if (!b) return fail(nullptr, TC_EINVAL, "tc_batch_info: batch is NULL");
    if (shape) {
        shape[0] = b->shape.far_warps;
        shape[1] = b->shape.far_blocks;
        shape[2] = b->shape.near_warps;
        shape[3] = b->shape.near_blocks;
    }
    if (tune_ms) {
        tune_ms[0] = b->tune_ms[0];
        tune_ms[1] = b->tune_ms[1];
    }
    return TC_OK;
}

tc_ctx* tc_batch_system(tc_batch* b, int32_t s)
{
    if (!b || s < 0 || s >= b->nsys) return nullptr;
    return b->ctx[s];
}

}  // extern "C"
