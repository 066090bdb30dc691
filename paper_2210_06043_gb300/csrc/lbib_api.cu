// lbib_api.cu -- host runtime behind include/lbib.h: contexts, device memory,
// streams, CUDA graphs of the time step and the C ABI.
//
// Time-step pipeline.  Lattice step m (bulk + near kernels) must follow the
// Lagrangian step m - 1 only on near tiles, and the bulk and near updates of
// one step write disjoint tiles from the same input, so the bulk lattice
// update of step m runs on a forked stream alongside the chain
//
//     Lagrangian(m-1) -> near lattice(m)      ||      bulk lattice(m)
//
// one captured graph per m % 6 (buffer parity and near-flag slot).  A context
// keeps the last Lagrangian step pending after lbib_advance (so back-to-back
// calls overlap it with the next lattice step); every call that reads
// Lagrangian state completes it.
//
// A context holds a batch of one or more capillary instances side by side in
// one lattice (instance i at node columns [x0_i, x0_i + nx_i), x0_i a multiple
// of the tile width), stepped by the same three launches.  Membranes, bonds and
// observables are per instance and in the instance's own coordinates; the
// bodies are stored grouped by instance.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "lbib_internal.cuh"
#include "lbib_trace.h"

using namespace lbib;

namespace {

struct HostBody {
    int inst = 0;  // capillary instance the body lives in
    int kind = 0, motion = 0, nv = 0;
    std::vector<double> xy, xy_ref;
    double ca = 0, beta = 0, ka = 0, dens = 1;
    bool adhesive = false;
    lbib_adhesion_params adh{};
};

thread_local std::string g_create_error;

// polygon measures of a closed chain: area, perimeter, area centroid, polar
// moment about the centroid
struct Poly {
    double A, P, cx, cy, Jc;
};

Poly polygon(const std::vector<double>& xy)
{
    const size_t nv = xy.size() / 2;
    double a2 = 0, per = 0, sx = 0, sy = 0, j = 0;
    for (size_t v = 0; v < nv; ++v) {
        size_t w = (v + 1) % nv;
        double x0 = xy[2 * v], y0 = xy[2 * v + 1], x1 = xy[2 * w], y1 = xy[2 * w + 1];
        double c = x0 * y1 - x1 * y0;
        a2 += c;
        per += std::sqrt((x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0));
        sx += (x0 + x1) * c;
        sy += (y0 + y1) * c;
        j += c * (x0 * x0 + x0 * x1 + x1 * x1 + y0 * y0 + y0 * y1 + y1 * y1);
    }
    Poly p;
    p.A = 0.5 * a2;
    p.P = per;
    p.cx = sx / (3.0 * a2);
    p.cy = sy / (3.0 * a2);
    p.Jc = j / 12.0 - p.A * (p.cx * p.cx + p.cy * p.cy);
    return p;
}

template <typename T>
cudaError_t dalloc(std::vector<void*>& reg, T** p, size_t n)
{
    void* q = nullptr;
    cudaError_t e = device_malloc(&q, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) {
        reg.push_back(q);
        *p = static_cast<T*>(q);
    }
    return e;
}

// The arrays of one phase (creation, set-up) carved out of one device
// allocation, each on a 256-byte boundary: one cudaMalloc and one cudaFree
// instead of one per array (about 45 of each per context).
struct Arena {
    std::vector<std::pair<void**, size_t>> parts;  // where each pointer goes, byte offset
    size_t bytes = 0;
    template <typename T>
    void add(T** p, size_t n)
    {
        parts.push_back({reinterpret_cast<void**>(p), bytes});
        bytes += (std::max<size_t>(n, 1) * sizeof(T) + 255) & ~size_t(255);
    }
    // stream-ordered: allocated, and at lbib_destroy freed, in the order of
    // the context stream's work, so neither waits for the device
    cudaError_t commit(std::vector<void*>& reg, cudaStream_t stream)
    {
        void* base = nullptr;
        cudaError_t e = device_malloc_async(&base, std::max<size_t>(bytes, 256), stream);
        if (e != cudaSuccess) return e;
        reg.push_back(base);
        for (auto& pr : parts) *pr.first = static_cast<char*>(base) + pr.second;
        return cudaSuccess;
    }
};

}  // namespace

void lbib::set_global_error(const char* msg) { g_create_error = msg; }

namespace lbib {
__global__ void k_raise_status(uint32_t* status, uint32_t bits) { atomicOr(status, bits); }
}  // namespace lbib

// allocations left before the injected failure (-1: none injected)
static std::atomic<long long> g_alloc_countdown{-1};

static bool injected_failure()
{
    long long c = g_alloc_countdown.load();
    while (c >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(c, c - 1)) return c == 0;  // the injected failure (once)
    }
    return false;
}

cudaError_t lbib::device_malloc(void** p, size_t bytes)
{
    if (injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

// The library's memory pool of each device: contexts' arenas come from it in
// stream order and go back to it at lbib_destroy, and it keeps up to
// kPoolKeep bytes of them for the next context (mapping and unmapping a
// sweep's 1.6 GB cost about 2 ms per context otherwise);
// lbib_release_cached_memory gives them back to the device.
static constexpr uint64_t kPoolKeep = uint64_t(8) << 30;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaError_t device_pool(cudaMemPool_t* out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = kPoolKeep;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

cudaError_t lbib::device_malloc_async(void** p, size_t bytes, cudaStream_t s)
{
    if (injected_failure()) return cudaErrorMemoryAllocation;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = device_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

struct lbib_ctx {
    std::string err;
    lbib_fluid_params P{};
    int prec = PREC_F64;
    size_t rsz = 8;  // bytes of one compute value
    size_t ssz = 8;  // bytes of one stored population
    Dev d{};
    std::vector<HostBody> bodies;
    bool finalized = false;
    int64_t s_f = 0, s_l = 0;  // lattice and Lagrangian steps done
    cudaStream_t stream = nullptr, side = nullptr, cap = nullptr, obs = nullptr;
    bool own_stream = false;
    cudaGraphExec_t unit[2][6] = {};  // [profiling][lattice step % 6]: buffer parity and flag slot
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_lag = nullptr, ev_obs = nullptr;
    int obs_branch = 0;  // observables record: 0 after the near update, 1 on its own branch
    int chain_pdl = 0;   // chain kernels as programmatic dependents of the kernel before them
    // copies of lbib_read_latest_observables_async run on `copy` after ev_step;
    // ev_copy marks the newest; copy_first is the oldest step whose copy may
    // still be in flight (its ring slot is written again ring_cap steps later)
    cudaStream_t copy = nullptr;
    cudaEvent_t ev_step = nullptr, ev_copy = nullptr;
    // activation of the step after next: a branch of the step graph
    cudaStream_t act = nullptr;
    cudaEvent_t ev_act = nullptr;
    bool copy_pending = false;
    int64_t copy_first = 0;
    cudaEvent_t pe[6] = {};
    bool profiling = false, profiled_last = false;
    alignas(64) unsigned char fmaps[256];  // tensor maps of the population buffers (two CUtensorMap)
    int near_grid = 0;         // force gather blocks; 0: default, set at finalize
    int near_update_grid = 0;  // near lattice update blocks; 0: default, set at finalize
    std::vector<void*> allocs;
    std::vector<void*> stream_allocs;  // stream-ordered allocations (the arenas), freed on `stream`
    double* macro_buf = nullptr;
    int device = 0;
    // batch of instances
    int ninst = 1;
    std::vector<int> inst_x0, inst_nx;
    std::vector<uint64_t> inst_seed;
    std::vector<int64_t> obs_consumed;     // [ninst] last observables step handed out
    std::vector<int> inst_nbodies;         // [ninst]
    std::vector<int> slot;                 // body id -> stored index (grouped by instance)
    std::vector<int> mark_off, lig_off;    // body id -> first marker / first ligand site
    int4* colinfo = nullptr;
    InstConst* inst = nullptr;
    // a fault after which the state cannot be trusted (a bounded device wait
    // gave up, so some nodes or markers were not updated): lbib_advance refuses
    // until lbib_load_state restores a saved state
    lbib_status fault = LBIB_OK;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

lbib_status fail(lbib_ctx* c, lbib_status s, const std::string& msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

lbib_status cuda_fail(lbib_ctx* c, cudaError_t e, const char* what)
{
    cudaGetLastError();
    return fail(c, e == cudaErrorMemoryAllocation ? LBIB_ERR_OOM : LBIB_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);     \
    } while (0)

lbib_status check_status(lbib_ctx* ctx)
{
    uint32_t st = 0;
    CK(cudaMemcpy(&st, ctx->d.status, sizeof(st), cudaMemcpyDeviceToHost));
    if (st & ST_DIVERGED) return fail(ctx, LBIB_ERR_DIVERGED, "non-finite or non-positive state on the device");
    if (st & ST_LIST_OVERFLOW) return fail(ctx, LBIB_ERR_STATE, "near-tile list overflow");
    if (st & ST_READ_MISS)
        return fail(ctx, LBIB_ERR_STATE, "an interpolation stencil left the tiles updated as near-membrane");
    if (st & ST_SPREAD_MISS)
        return fail(ctx, LBIB_ERR_STATE, "a spreading stencil left the tiles scheduled as near-membrane");
    if (st & ST_BOUNDS) return fail(ctx, LBIB_ERR_STATE, "an index left its array (bounds-checked build)");
    if (st & ST_TMA_TIMEOUT) {
        ctx->fault = LBIB_ERR_TIMEOUT;
        return fail(ctx, LBIB_ERR_TIMEOUT, "a bulk-update block gave up waiting for a tensor copy");
    }
    return LBIB_OK;
}

bool valid_instance(const lbib_ctx* ctx, int32_t i) { return i >= 0 && i < ctx->ninst; }

// Before the stream gets the membrane update of step `step` (which writes the
// ring slot step % ring_cap): wait for the observables copies in flight if one
// of them may read that slot.
lbib_status guard_ring(lbib_ctx* ctx, int64_t step)
{
    if (ctx->copy_pending && step >= ctx->copy_first + ctx->d.ring_cap) {
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_copy, 0));
        ctx->copy_pending = false;
    }
    return LBIB_OK;
}

lbib_status finish_pending(lbib_ctx* ctx)
{
    if (ctx->d.nbodies > 0 && ctx->s_l < ctx->s_f) {
        lbib_status s = guard_ring(ctx, ctx->s_l + 1);
        if (s != LBIB_OK) return s;
        CK(launch_lagrangian(ctx->d, ctx->prec, (int)((ctx->s_l + 1) & 1), ctx->stream));
        CK(launch_activate_next(ctx->d, ctx->stream));
        CK(launch_observables(ctx->d, ctx->stream, true, ctx->chain_pdl != 0));  // after the membrane kernel
        ctx->s_l += 1;
    }
    return LBIB_OK;
}

// Graph of lattice step m (v = m % 6): the membrane update of step m - 1 then
// the near lattice update of step m on one branch, the bulk lattice update of
// step m on the other (they write disjoint tiles and read only step m's
// populations).
lbib_status capture_unit(lbib_ctx* ctx, int prof, int v)
{
    Dev& d = ctx->d;
    const int p = v & 1, slot = v % 3;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    auto rec = [&](int i, cudaStream_t s) {
        if (prof && e == cudaSuccess) e = cudaEventRecordWithFlags(ctx->pe[i], s, cudaEventRecordExternal);
    };
    // the membrane kernel is enqueued first so that its blocks are resident
    // before the bulk lattice blocks fill the SMs
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_fork, ctx->cap);
    rec(2, ctx->cap);
    if (e == cudaSuccess) e = launch_lagrangian(d, ctx->prec, p, ctx->cap);
    rec(3, ctx->cap);
    // near tiles of lattice step m + 1 on a branch of their own (first needed
    // by the next graph)
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_lag, ctx->cap);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->act, ctx->ev_lag, 0);
    if (e == cudaSuccess) e = launch_activate_next(d, ctx->act);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_act, ctx->act);
    // observables record on a branch of its own (the near update does not wait
    // for it; best when the chain sets the step) or after the near update
    // (best when the bulk update does: a lone block queued at normal priority
    // would wait behind the bulk blocks and end the step late)
    if (ctx->obs_branch) {
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->obs, ctx->ev_lag, 0);
        if (e == cudaSuccess) e = launch_observables(d, ctx->obs, false, false);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_obs, ctx->obs);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->side, ctx->ev_fork, 0);
    rec(0, ctx->side);
    if (e == cudaSuccess) e = launch_lbm_bulk(d, ctx->prec, p, slot, ctx->side);
    rec(1, ctx->side);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_join, ctx->side);
    rec(4, ctx->cap);
    // optionally programmatic dependents of the kernel before them on the
    // chain (launch latency hidden behind its tail), never in the profiling
    // graphs, whose timing events sit between the kernels
    const bool pdl = ctx->chain_pdl && !prof;
    if (e == cudaSuccess) e = launch_lbm_near(d, ctx->prec, p, ctx->near_grid, ctx->near_update_grid, ctx->cap, pdl);
    rec(5, ctx->cap);
    if (!ctx->obs_branch && e == cudaSuccess) e = launch_observables(d, ctx->cap, true, pdl);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap, ctx->ev_join, 0);
    if (ctx->obs_branch && e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap, ctx->ev_obs, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->cap, ctx->ev_act, 0);
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(ctx, e, "capturing the step graph");
    }
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
    // per-node priorities: the membrane -> near chain ahead of the bulk blocks
    e = cudaGraphInstantiate(&ctx->unit[prof][v], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    return LBIB_OK;
}

lbib_status ensure_graphs(lbib_ctx* ctx)
{
    int prof = ctx->profiling ? 1 : 0;
    for (int v = 0; v < 6; ++v)
        if (!ctx->unit[prof][v]) {
            lbib_status s = capture_unit(ctx, prof, v);
            if (s != LBIB_OK) return s;
        }
    return LBIB_OK;
}

// Positions of buffer k as float-float pairs (hi, lo) of the compute type,
// from the host copy of the positions (x block then y block) just uploaded.
lbib_status upload_posf(lbib_ctx* ctx, int k, const std::vector<double>& pos)
{
    Dev& d = ctx->d;
    const size_t nm = std::max(d.nmark, 1);
    if (ctx->prec == PREC_F64) {
        std::vector<double> f(4 * nm, 0.0);
        for (size_t i = 0; i < nm; ++i) {
            f[i] = pos[i];
            f[2 * nm + i] = pos[nm + i];
        }
        CK(cudaMemcpyAsync(d.posf[k], f.data(), f.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        std::vector<float> f(4 * nm, 0.f);
        for (size_t i = 0; i < nm; ++i) {
            float hx = (float)pos[i], hy = (float)pos[nm + i];
            f[i] = hx;
            f[nm + i] = (float)(pos[i] - (double)hx);
            f[2 * nm + i] = hy;
            f[3 * nm + i] = (float)(pos[nm + i] - (double)hy);
        }
        CK(cudaMemcpyAsync(d.posf[k], f.data(), f.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    return LBIB_OK;
}

// Builds the device Lagrangian arrays from the host bodies (first advance).
lbib_status finalize(lbib_ctx* ctx)
{
    LBIB_TRACE("lbib set-up (first advance)");
    if (ctx->finalized) return LBIB_OK;
    Dev& d = ctx->d;
    const Lattice& L = d.L;
    const int nb = (int)ctx->bodies.size();
    const int ni = ctx->ninst;
    d.nbodies = nb;
    // stored order: grouped by instance, in order of addition within one
    std::vector<int> order(nb);
    for (int b = 0; b < nb; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return ctx->bodies[a].inst < ctx->bodies[b].inst; });
    ctx->slot.assign(nb, 0);
    ctx->mark_off.assign(nb, 0);
    ctx->lig_off.assign(nb, 0);
    for (int k = 0; k < nb; ++k) ctx->slot[order[k]] = k;
    std::vector<BodyConst> bc(nb);
    std::vector<InstConst> ic(ni);
    int nmark = 0, nlig = 0, nv_max = 0, mw = 1;
    for (int i = 0; i < ni; ++i) {
        InstConst& I = ic[i];
        std::memset(&I, 0, sizeof(I));
        I.x0 = ctx->inst_x0[i];
        I.nx = ctx->inst_nx[i];
        I.seed = ctx->inst_seed[i];
        I.first_cell = I.first_particle = -1;
        I.moff = nmark;
        I.lig0 = nlig;
        I.body0 = 0;
        for (int k = 0; k < nb; ++k)
            if (ctx->bodies[order[k]].inst < i) I.body0 = k + 1;
        for (int k = I.body0; k < nb && ctx->bodies[order[k]].inst == i; ++k) {
            const HostBody& h = ctx->bodies[order[k]];
            I.nbodies += 1;
            I.nmark += h.nv;
            if (h.adhesive) I.nlig += h.adh.n_ligands;
            if (h.kind == LBIB_CELL && I.first_cell < 0) I.first_cell = k;
            if (h.kind == LBIB_PARTICLE && I.first_particle < 0) I.first_particle = k;
            nv_max = std::max(nv_max, h.nv);
        }
        nmark += I.nmark;
        nlig += I.nlig;
        mw = std::max(mw, (I.nmark + 31) / 32);
    }
    d.nmark = nmark;
    d.nlig = nlig;
    d.nv_max = std::max(nv_max, 1);
    d.mw = mw;
    ctx->inst_nbodies.assign(ni, 0);
    for (int i = 0; i < ni; ++i) ctx->inst_nbodies[i] = ic[i].nbodies;
    std::vector<double> pos(2 * (size_t)std::max(nmark, 1)), rref(2 * (size_t)std::max(nmark, 1));
    std::vector<double> l0(std::max(nmark, 1)), th0(std::max(nmark, 1));
    std::vector<double> rig((size_t)std::max(nb, 1) * RG_N, 0.0), bobs((size_t)std::max(nb, 1) * BO_N, 0.0);
    std::vector<int32_t> lig_el(std::max(nlig, 1)), bound(std::max(nlig, 1), 0), site_off(nmark + 1, 0);
    std::vector<double> lig_t(std::max(nlig, 1)), anchor(2 * (size_t)std::max(nlig, 1), 0.0);
    const double nu = L.nu, umax = L.umax;
    int off = 0, loff = 0;
    for (int b = 0; b < nb; ++b) {
        const HostBody& h = ctx->bodies[order[b]];
        const InstConst& I = ic[h.inst];
        BodyConst& B = bc[b];
        std::memset(&B, 0, sizeof(B));
        B.kind = h.kind;
        B.motion = h.motion;
        B.nv = h.nv;
        B.off = off;
        B.inst = h.inst;
        B.x0 = I.x0;
        B.nxi = I.nx;
        B.moff = I.moff;
        B.lig0 = I.lig0;
        B.b0 = I.body0;
        B.nbi = I.nbodies;
        ctx->mark_off[order[b]] = off;
        ctx->lig_off[order[b]] = loff;
        const std::vector<double>& ref = h.xy_ref.empty() ? h.xy : h.xy_ref;
        const int nv = h.nv;
        // stress-free lengths and turning angles (the angles only where Eq. 10
        // acts: a deformable membrane with k_b > 0; elsewhere they stay 0)
        const bool bends = h.motion == LBIB_DEFORMABLE && h.beta != 0.0;
        for (int l = 0; l < nv; ++l) {
            int w = (l + 1) % nv, lm = (l + nv - 1) % nv;
            double dx = ref[2 * w] - ref[2 * l], dy = ref[2 * w + 1] - ref[2 * l + 1];
            l0[off + l] = std::sqrt(dx * dx + dy * dy);
            double ax = ref[2 * l] - ref[2 * lm], ay = ref[2 * l + 1] - ref[2 * lm + 1];
            th0[off + l] = bends ? std::atan2(ax * dy - ay * dx, ax * dx + ay * dy) : 0.0;
        }
        Poly pr = polygon(ref), pc = polygon(h.xy);
        B.A0 = pr.A;
        B.P0 = pr.P;
        B.inv_A0 = 1.0 / pr.A;
        B.inv_P0 = 1.0 / pr.P;
        B.ks = (h.motion == LBIB_DEFORMABLE) ? 1.0 * nu * umax / h.ca : 0.0;  // Ca = rho nu u_max / k_s
        B.kb = h.beta * B.ks;
        B.ka = h.ka;
        B.mv = h.dens * pr.A / nv;
        B.mass = h.dens * pc.A;
        B.inertia = h.dens * pc.Jc;
        double* rs = &rig[(size_t)b * RG_N];
        rs[RG_XC] = pc.cx;
        rs[RG_YC] = pc.cy;
        for (int v = 0; v < nv; ++v) {
            pos[off + v] = h.xy[2 * v];
            pos[nmark + off + v] = h.xy[2 * v + 1];
            rref[off + v] = h.xy[2 * v] - pc.cx;
            rref[nmark + off + v] = h.xy[2 * v + 1] - pc.cy;
        }
        double* bo = &bobs[(size_t)b * BO_N];
        bo[BO_AREA] = pc.A;
        bo[BO_DPERIM] = pc.P - pr.P;
        bo[BO_CX] = pc.cx;
        bo[BO_CY] = pc.cy;
        bo[BO_XMIN] = bo[BO_YMIN] = 1e300;
        bo[BO_XMAX] = bo[BO_YMAX] = -1e300;
        for (int v = 0; v < nv; ++v) {
            bo[BO_XMIN] = std::min(bo[BO_XMIN], h.xy[2 * v]);
            bo[BO_XMAX] = std::max(bo[BO_XMAX], h.xy[2 * v]);
            bo[BO_YMIN] = std::min(bo[BO_YMIN], h.xy[2 * v + 1]);
            bo[BO_YMAX] = std::max(bo[BO_YMAX], h.xy[2 * v + 1]);
        }
        if (h.adhesive) {
            const lbib_adhesion_params& a = h.adh;
            B.adhesive = 1;
            B.nlig = a.n_ligands;
            B.lig_off = loff;
            B.sigma_inf = std::isinf(a.sigma) ? 1 : 0;
            B.sigma = B.sigma_inf ? 0.0 : a.sigma * 1.0 * nu * nu / L.ny;  // units rho nu^2 / H
            B.ycr = a.y_cr;
            B.yeq = a.y_eq;
            B.Pf = 1.0 - std::exp(-a.kf_dt);
            B.kr0_dt = a.kr0_dt;
            B.xi = a.xi;
            // sites at arc lengths (k + 1/2) P / n along the current chain
            std::vector<double> cum(nv + 1, 0.0);
            for (int l = 0; l < nv; ++l) {
                int w = (l + 1) % nv;
                double dx = h.xy[2 * w] - h.xy[2 * l], dy = h.xy[2 * w + 1] - h.xy[2 * l + 1];
                cum[l + 1] = cum[l] + std::sqrt(dx * dx + dy * dy);
            }
            int l = 0;
            for (int k = 0; k < a.n_ligands; ++k) {
                double s = (k + 0.5) * cum[nv] / a.n_ligands;
                while (l < nv - 1 && s > cum[l + 1]) ++l;
                double t = (s - cum[l]) / (cum[l + 1] - cum[l]);
                t = std::min(1.0, std::max(0.0, t));
                int w = (l + 1) % nv;
                double px = h.xy[2 * l] + t * (h.xy[2 * w] - h.xy[2 * l]);
                double py = h.xy[2 * l + 1] + t * (h.xy[2 * w + 1] - h.xy[2 * l + 1]);
                lig_el[loff + k] = off + l;
                lig_t[loff + k] = t;
                site_off[off + l + 1] += 1;
                if (std::min(py, (double)L.ny - py) < a.y_cr) {
                    bound[loff + k] = 1;
                    anchor[loff + k] = px;
                    anchor[nlig + loff + k] = (py < (double)L.ny - py) ? 0.0 : (double)L.ny;
                    B.nl0 += 1;
                }
            }
            bo[BO_NBOUND] = B.nl0;
            loff += a.n_ligands;
        }
        off += nv;
    }
    for (int e = 0; e < nmark; ++e) site_off[e + 1] += site_off[e];
    d.ring_cap = ctx->P.obs_capacity > 0 ? ctx->P.obs_capacity : 4096;

    // device arrays
    auto& reg = ctx->allocs;
    const size_t rs = ctx->rsz;
    const size_t nm1 = std::max(nmark, 1), nl1 = std::max(nlig, 1);
    BodyConst* dbody = nullptr;
    void *dl0 = nullptr, *dth0 = nullptr, *dligt = nullptr;
    double* drref = nullptr;
    int32_t *dligel = nullptr, *dsite = nullptr;
    Arena ar;
    ar.add(&d.pos[0], 2 * nm1);
    ar.add(&d.pos[1], 2 * nm1);
    ar.add(reinterpret_cast<char**>(&d.posf[0]), 4 * nm1 * rs);
    ar.add(reinterpret_cast<char**>(&d.posf[1]), 4 * nm1 * rs);
    ar.add(&dbody, std::max(nb, 1));
    ar.add(&d.rigid, (size_t)std::max(nb, 1) * RG_N);
    ar.add(reinterpret_cast<char**>(&dl0), nm1 * rs);
    ar.add(reinterpret_cast<char**>(&dth0), nm1 * rs);
    ar.add(&drref, 2 * nm1);
    ar.add(&dligel, nl1);
    ar.add(reinterpret_cast<char**>(&dligt), nl1 * rs);
    ar.add(&d.bound, nl1);
    ar.add(&d.anchor, 2 * nl1);
    ar.add(reinterpret_cast<char**>(&d.margin), nl1 * rs);
    ar.add(&dsite, (size_t)nmark + 1);
    ar.add(reinterpret_cast<char**>(&d.diag), (size_t)NDIAG * nm1 * rs);
    ar.add(&d.body_obs[0], (size_t)std::max(nb, 1) * BO_N);
    ar.add(&d.body_obs[1], (size_t)std::max(nb, 1) * BO_N);
    ar.add(&d.ring, (size_t)ni * d.ring_cap);
    for (int k = 0; k < 2; ++k) {
        ar.add(&d.mki[k], 2 * nm1);
        ar.add(reinterpret_cast<char**>(&d.mkf[k]), 4 * nm1 * rs);
    }
    ar.add(&d.mask[0], (size_t)L.ntiles * d.mw);
    ar.add(&d.mask[1], (size_t)L.ntiles * d.mw);
    CK(ar.commit(ctx->stream_allocs, ctx->stream));
    d.body = dbody;
    d.l0 = dl0;
    d.th0 = dth0;
    d.rref = drref;
    d.lig_el = dligel;
    d.lig_t = dligt;
    d.site_off = dsite;

    auto up_real = [&](void* dst, const std::vector<double>& src) -> cudaError_t {
        if (ctx->prec == PREC_F64)
            return cudaMemcpyAsync(dst, src.data(), src.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
        std::vector<float> t(src.begin(), src.end());
        return cudaMemcpyAsync(dst, t.data(), t.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
    };
    CK(cudaMemcpyAsync(d.pos[0], pos.data(), pos.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d.pos[1], pos.data(), pos.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    for (int k = 0; k < 2; ++k) {
        lbib_status st = upload_posf(ctx, k, pos);
        if (st != LBIB_OK) return st;
    }
    if (nb) CK(cudaMemcpyAsync(dbody, bc.data(), bc.size() * sizeof(BodyConst), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->inst, ic.data(), ic.size() * sizeof(InstConst), cudaMemcpyHostToDevice, ctx->stream));
    {
        // tile-column table with the instances' first markers, now known
        std::vector<int4> cols;
        for (int i = 0; i < ni; ++i)
            for (int c = 0; c < (ic[i].nx + TX - 1) / TX; ++c)
                cols.push_back(make_int4(ic[i].x0, ic[i].nx, ic[i].moff, i));
        CK(cudaMemcpyAsync(ctx->colinfo, cols.data(), cols.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaMemcpyAsync(d.rigid, rig.data(), rig.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(up_real(dl0, l0));
    CK(up_real(dth0, th0));
    CK(cudaMemcpyAsync(drref, rref.data(), rref.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dligel, lig_el.data(), lig_el.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(up_real(dligt, lig_t));
    CK(cudaMemcpyAsync(d.bound, bound.data(), bound.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d.anchor, anchor.data(), anchor.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(d.margin, 0, nl1 * rs, ctx->stream));
    CK(cudaMemcpyAsync(dsite, site_off.data(), site_off.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(d.diag, 0, (size_t)NDIAG * nm1 * rs, ctx->stream));
    CK(cudaMemcpyAsync(d.body_obs[0], bobs.data(), bobs.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d.body_obs[1], bobs.data(), bobs.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemsetAsync(d.ring, 0, (size_t)ni * d.ring_cap * sizeof(lbib_obs), ctx->stream));
    for (int k = 0; k < 2; ++k) {
        CK(cudaMemsetAsync(d.mki[k], 0, 2 * nm1 * 4, ctx->stream));
        CK(cudaMemsetAsync(d.mkf[k], 0, 4 * nm1 * rs, ctx->stream));
    }
    CK(cudaMemsetAsync(d.mask[0], 0, (size_t)L.ntiles * d.mw * 4, ctx->stream));
    CK(cudaMemsetAsync(d.mask[1], 0, (size_t)L.ntiles * d.mw * 4, ctx->stream));
    if (nb) {
        if (lagrangian_smem_bytes(ctx->prec, d.nv_max) > 227 * 1024)
            return fail(ctx, LBIB_ERR_UNSUPPORTED, "membrane too large for one block's shared memory");
        CK(configure_kernels(ctx->prec, d.nv_max));
        CK(launch_activate(d, ctx->prec, ctx->s_f, 3, ctx->stream));
    }
    int nsm = 152;
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    // default launch shapes (lbib_set_launch_config / lbib_autotune may change them):
    // membrane blocks of 256 threads once the bodies outnumber half the SMs, so that
    // they share SMs with the bulk lattice update; near kernel 4 blocks per SM
    if (!d.lag_threads) d.lag_threads = (nb > nsm / 2) ? 256 : 512;
    {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        d.chain_priority = greatest;  // numerically lowest = most urgent
    }
    if (!ctx->near_grid) ctx->near_grid = std::max(1, std::min(L.ntiles, 4 * nsm));
    if (!ctx->near_update_grid) ctx->near_update_grid = std::max(1, std::min(L.ntiles, 16 * nsm));
    ctx->finalized = true;  // the step graphs are captured at the first step (after any launch configuration)
    CK(cudaStreamSynchronize(ctx->stream));
    return LBIB_OK;
}

lbib_status pre_read(lbib_ctx* ctx)
{
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    s = finish_pending(ctx);
    if (s != LBIB_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaStreamSynchronize(ctx->copy));
    ctx->copy_pending = false;
    return check_status(ctx);
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

const char* lbib_last_error(lbib_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"

namespace {

lbib_status create_impl(const lbib_fluid_params* P, int32_t ninst, const int32_t* nxs, const uint64_t* seeds,
                        lbib_ctx** out)
{
    lbib_ctx* ctx = nullptr;
    if (!P || !out || !nxs) return fail(nullptr, LBIB_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (ninst < 1) return fail(nullptr, LBIB_ERR_INVALID_ARG, "need at least one instance");
    for (int i = 0; i < ninst; ++i)
        if (nxs[i] < 3) return fail(nullptr, LBIB_ERR_INVALID_ARG, "need nx >= 3 for every instance");
    if (P->ny < 2) return fail(nullptr, LBIB_ERR_INVALID_ARG, "need nx >= 3 and ny >= 2");
    if (!(P->tau > 0.5)) return fail(nullptr, LBIB_ERR_INVALID_ARG, "tau must exceed 1/2");
    if (!(P->re >= 0.0) || !(P->rho_out > 0.0)) return fail(nullptr, LBIB_ERR_INVALID_ARG, "re >= 0 and rho_out > 0");
    if (P->bc_mode != LBIB_BC_INLET_OUTLET && P->bc_mode != LBIB_BC_PERIODIC_FORCE)
        return fail(nullptr, LBIB_ERR_INVALID_ARG, "unknown bc_mode");
    if (P->transfer != LBIB_TRANSFER_PESKIN && P->transfer != LBIB_TRANSFER_MLS)
        return fail(nullptr, LBIB_ERR_INVALID_ARG, "unknown transfer kernel");
    if (P->storage != LBIB_STORE_FP64 && P->storage != LBIB_STORE_FP32 && P->storage != LBIB_STORE_BF16 &&
        P->storage != LBIB_STORE_FP16)
        return fail(nullptr, LBIB_ERR_INVALID_ARG, "unknown storage");
    if (P->obs_capacity < 0) return fail(nullptr, LBIB_ERR_INVALID_ARG, "obs_capacity < 0");
    // instances side by side, each starting on a tile column
    long long ntx = 0;
    for (int i = 0; i < ninst; ++i) ntx += (nxs[i] + TX - 1) / TX;
    long long qs = ntx * TX * (long long)P->ny;
    if (qs * 9 >= (1LL << 31)) return fail(nullptr, LBIB_ERR_UNSUPPORTED, "lattice too large for 32-bit indexing");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || P->device < 0 || P->device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, LBIB_ERR_CUDA, "no CUDA device with that ordinal");
    }
    ctx = new (std::nothrow) lbib_ctx();
    if (!ctx) return fail(nullptr, LBIB_ERR_OOM, "host allocation failed");
    ctx->P = *P;
    ctx->device = P->device;
    DeviceGuard guard(ctx->device);
    ctx->prec = (P->storage == LBIB_STORE_FP64) ? PREC_F64 : PREC_F32;
    ctx->rsz = (ctx->prec == PREC_F64) ? 8 : 4;
    ctx->ssz = (P->storage == LBIB_STORE_FP64) ? 8 : (P->storage == LBIB_STORE_FP32 ? 4 : 2);
    ctx->d.store = (P->storage == LBIB_STORE_FP64)   ? STORE_F64
                   : (P->storage == LBIB_STORE_FP32) ? STORE_F32
                   : (P->storage == LBIB_STORE_BF16) ? STORE_BF16
                                                     : STORE_F16;
    ctx->ninst = ninst;
    std::vector<int4> cols;
    for (int i = 0, x0 = 0; i < ninst; ++i) {
        ctx->inst_x0.push_back(x0);
        ctx->inst_nx.push_back(nxs[i]);
        ctx->inst_seed.push_back(seeds ? seeds[i] : P->seed + (uint64_t)i);
        const int w = (nxs[i] + TX - 1) / TX;
        for (int c = 0; c < w; ++c) cols.push_back(make_int4(x0, nxs[i], 0, i));  // moff set once bodies are known
        x0 += w * TX;
    }
    ctx->obs_consumed.assign(ninst, 0);
    ctx->inst_nbodies.assign(ninst, 0);
    Lattice& L = ctx->d.L;
    L.nx = ctx->inst_x0.back() + nxs[ninst - 1];
    L.ny = P->ny;
    L.ntx = (int)ntx;
    L.nty = (P->ny + TY - 1) / TY;
    L.nxp = L.ntx * TX;
    L.ntiles = L.ntx * L.nty;
    L.bc = P->bc_mode;
    L.transfer = P->transfer;
    L.qstride = (int)qs;
    L.tau = P->tau;
    L.omega = 1.0 / P->tau;
    L.nu = (P->tau - 0.5) / 3.0;
    L.umax = P->re * L.nu / P->ny;  // Re = u_max H / nu
    L.rho_out = P->rho_out;
    L.gx = P->gx;
    L.gy = P->gy;
    set_float_params(L);
    Dev& d = ctx->d;
    d.list_cap = L.ntiles;
    d.dcut = 2.0;
    d.probe = 1.2;
    d.uscale = L.umax / P->ny;
    d.ring_cap = 1;
    d.ninst = ninst;
    d.lag_threads = 0;  // 0: default, set at finalize
    d.bulk_tiles_y = 1;
    d.bulk_nodes_per_thread = 1;
    d.act_stride = ACT_STRIDE;
    auto bail = [&](lbib_status s) {
        std::string m = ctx->err;
        lbib_destroy(ctx);
        g_create_error = m;
        return s;
    };
#define CKC(call)                                                           \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return bail(cuda_fail(ctx, e_, #call));      \
    } while (0)
    auto& reg = ctx->allocs;
    size_t nq = (size_t)9 * qs, nn = (size_t)qs;
    // streams first: every set-up copy and fill below is ordered on the
    // context stream (a fill on the legacy default stream is not ordered with
    // this non-blocking stream, and with other contexts' work in flight the
    // initial populations were overwritten by their own zero fill)
    if (P->cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(P->cuda_stream);
    } else {
        CKC(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
        ctx->own_stream = true;
    }
    CKC(cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&ctx->obs, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&ctx->copy, cudaStreamNonBlocking));
    CKC(cudaStreamCreateWithFlags(&ctx->act, cudaStreamNonBlocking));
    CKC(cudaEventCreateWithFlags(&ctx->ev_act, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&ctx->ev_step, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&ctx->ev_copy, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&ctx->ev_lag, cudaEventDisableTiming));
    CKC(cudaEventCreateWithFlags(&ctx->ev_obs, cudaEventDisableTiming));
    Arena ar;
    ar.add(reinterpret_cast<char**>(&d.f[0]), nq * ctx->ssz);
    ar.add(reinterpret_cast<char**>(&d.f[1]), nq * ctx->ssz);
    ar.add(reinterpret_cast<char**>(&d.drho), nn * ctx->rsz);
    ar.add(reinterpret_cast<char**>(&d.ux), nn * ctx->rsz);
    ar.add(reinterpret_cast<char**>(&d.uy), nn * ctx->rsz);
    ar.add(reinterpret_cast<char**>(&d.fx), nn * ctx->rsz);
    ar.add(reinterpret_cast<char**>(&d.fy), nn * ctx->rsz);
    ar.add(&d.fresh, L.ntiles);
    for (int i = 0; i < 3; ++i) ar.add(&d.nearflag[i], L.ntiles);
    for (int i = 0; i < 3; ++i) ar.add(&d.list[i], d.list_cap);
    ar.add(&d.count, 3);
    ar.add(&d.step, 1);
    ar.add(&d.status, 1);
    ar.add(&d.ticket, 1);
    ar.add(&ctx->colinfo, cols.size());
    ar.add(&ctx->inst, (size_t)ninst);
    CKC(ar.commit(ctx->stream_allocs, ctx->stream));
#ifdef LBIB_CHECKED
    L.chk_status = d.status;
#endif
    d.colinfo = ctx->colinfo;
    d.inst = ctx->inst;
    CKC(cudaMemcpyAsync(ctx->colinfo, cols.data(), cols.size() * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    // populations: the initial state is written whole (padding included) by
    // the init kernel below; the second buffer needs no fill either: the first
    // lattice step writes every node of it, and the row padding past an
    // instance's end is never read as data by any kernel
    // tensor maps for the TMA-staged bulk update (left out where the driver
    // has no encoder: the direct-load kernel then runs whatever the option)
    d.bulk_tma = 0;
    d.fmaps = nullptr;
    if (make_population_maps(d, ctx->fmaps) == cudaSuccess && configure_bulk_tma(d.store) == cudaSuccess)
        d.fmaps = ctx->fmaps;
    cudaGetLastError();
    CKC(cudaMemsetAsync(d.drho, 0, nn * ctx->rsz, ctx->stream));
    CKC(cudaMemsetAsync(d.ux, 0, nn * ctx->rsz, ctx->stream));
    CKC(cudaMemsetAsync(d.uy, 0, nn * ctx->rsz, ctx->stream));
    CKC(cudaMemsetAsync(d.fx, 0, nn * ctx->rsz, ctx->stream));
    CKC(cudaMemsetAsync(d.fy, 0, nn * ctx->rsz, ctx->stream));
    CKC(cudaMemsetAsync(d.fresh, 0x80, L.ntiles * 4, ctx->stream));  // matches no step
    for (int i = 0; i < 3; ++i) CKC(cudaMemsetAsync(d.nearflag[i], 0, L.ntiles * 4, ctx->stream));
    CKC(cudaMemsetAsync(d.count, 0, 12, ctx->stream));
    CKC(cudaMemsetAsync(d.step, 0, 8, ctx->stream));
    CKC(cudaMemsetAsync(d.status, 0, 4, ctx->stream));
    CKC(cudaMemsetAsync(d.ticket, 0, 4, ctx->stream));
    CKC(launch_init_populations(d, ctx->prec, 0, ctx->stream));  // the stream orders it before any use
#undef CKC
    *out = ctx;
    return LBIB_OK;
}

}  // namespace

extern "C" {

lbib_status lbib_create(const lbib_fluid_params* P, lbib_ctx** out)
{
    LBIB_TRACE("lbib_create");
    if (!P || !out) return fail(nullptr, LBIB_ERR_INVALID_ARG, "null argument");
    const uint64_t seed = P->seed;
    return create_impl(P, 1, &P->nx, &seed, out);
}

lbib_status lbib_create_batch(const lbib_fluid_params* P, int32_t n_instances, const int32_t* nx,
                              const uint64_t* seeds, lbib_ctx** out)
{
    LBIB_TRACE("lbib_create_batch");
    return create_impl(P, n_instances, nx, seeds, out);
}

lbib_status lbib_add_membrane_to(lbib_ctx* ctx, int32_t instance, const lbib_membrane_desc* m, int32_t* id_out)
{
    LBIB_TRACE("lbib_add_membrane_to");
    if (!ctx || !m) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (!valid_instance(ctx, instance)) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such instance");
    if (ctx->finalized) return fail(ctx, LBIB_ERR_STATE, "membranes must be added before the first advance");
    if (ctx->inst_nbodies[instance] >= MAX_BODIES)
        return fail(ctx, LBIB_ERR_UNSUPPORTED, "too many bodies in one instance");
    if (m->nv < 3 || m->nv > MAX_NV || !m->xy) return fail(ctx, LBIB_ERR_INVALID_ARG, "need 3 <= nv <= 1024 and xy");
    if (m->kind != LBIB_CELL && m->kind != LBIB_PARTICLE) return fail(ctx, LBIB_ERR_INVALID_ARG, "unknown kind");
    if (m->motion < LBIB_DEFORMABLE || m->motion > LBIB_FIXED) return fail(ctx, LBIB_ERR_INVALID_ARG, "unknown motion");
    if (m->motion == LBIB_DEFORMABLE && !(m->ca > 0.0))
        return fail(ctx, LBIB_ERR_INVALID_ARG, "a deformable membrane needs Ca > 0");
    if (!(m->density_ratio > 0.0)) return fail(ctx, LBIB_ERR_INVALID_ARG, "density_ratio must be > 0");
    HostBody h;
    h.inst = instance;
    h.kind = m->kind;
    h.motion = m->motion;
    h.nv = m->nv;
    h.xy.assign(m->xy, m->xy + 2 * (size_t)m->nv);
    if (m->xy_ref) h.xy_ref.assign(m->xy_ref, m->xy_ref + 2 * (size_t)m->nv);
    for (double v : h.xy)
        if (!std::isfinite(v)) return fail(ctx, LBIB_ERR_INVALID_ARG, "non-finite vertex");
    if (polygon(h.xy).A <= 0.0 || (!h.xy_ref.empty() && polygon(h.xy_ref).A <= 0.0))
        return fail(ctx, LBIB_ERR_INVALID_ARG, "chains must be counter-clockwise with positive area");
    h.ca = m->ca;
    h.beta = m->beta;
    h.ka = m->ka;
    h.dens = m->density_ratio;
    ctx->bodies.push_back(h);
    ctx->inst_nbodies[instance] += 1;
    if (id_out) *id_out = (int32_t)ctx->bodies.size() - 1;
    return LBIB_OK;
}

lbib_status lbib_add_membrane(lbib_ctx* ctx, const lbib_membrane_desc* m, int32_t* id_out)
{
    return lbib_add_membrane_to(ctx, 0, m, id_out);
}

lbib_status lbib_add_membranes(lbib_ctx* ctx, int32_t n, const int32_t* instance, const lbib_membrane_desc* descs,
                               const lbib_adhesion_params* const* adhesion, int32_t* ids_out)
{
    LBIB_TRACE("lbib_add_membranes");
    if (!ctx || n < 0 || (n > 0 && (!instance || !descs))) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    for (int32_t k = 0; k < n; ++k) {
        int32_t id = -1;
        lbib_status s = lbib_add_membrane_to(ctx, instance[k], &descs[k], &id);
        if (s == LBIB_OK && adhesion && adhesion[k]) s = lbib_set_adhesion(ctx, id, adhesion[k]);
        if (s != LBIB_OK) return s;  // bodies before k stay added
        if (ids_out) ids_out[k] = id;
    }
    return LBIB_OK;
}

lbib_status lbib_set_adhesion(lbib_ctx* ctx, int32_t body, const lbib_adhesion_params* a)
{
    LBIB_TRACE("lbib_set_adhesion");
    if (!ctx || !a) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (ctx->finalized) return fail(ctx, LBIB_ERR_STATE, "adhesion must be set before the first advance");
    if (body < 0 || body >= (int)ctx->bodies.size()) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such body");
    if (a->n_ligands <= 0 || !(a->y_cr >= 0) || !(a->kf_dt >= 0) || !(a->kr0_dt >= 0) || std::isnan(a->sigma))
        return fail(ctx, LBIB_ERR_INVALID_ARG, "invalid adhesion parameters");
    if (std::isinf(a->sigma) && ctx->bodies[body].motion != LBIB_FIXED)
        return fail(ctx, LBIB_ERR_INVALID_ARG, "sigma = inf requires a FIXED particle");
    ctx->bodies[body].adhesive = true;
    ctx->bodies[body].adh = *a;
    return LBIB_OK;
}

lbib_status lbib_advance(lbib_ctx* ctx, int64_t nsteps)
{
    LBIB_TRACE("lbib_advance");
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    if (nsteps < 0) return fail(ctx, LBIB_ERR_INVALID_ARG, "nsteps < 0");
    if (ctx->fault != LBIB_OK)
        return fail(ctx, ctx->fault, "a bounded device wait gave up earlier: restore a saved state (lbib_load_state)");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    Dev& d = ctx->d;
    if (d.nbodies == 0) {
        for (int64_t k = 0; k < nsteps; ++k) {
            CK(launch_lbm_bulk(d, ctx->prec, (int)(ctx->s_f & 1), (int)(ctx->s_f % 3), ctx->stream));
            ctx->s_f += 1;
        }
        ctx->s_l = ctx->s_f;
        return LBIB_OK;
    }
    if (nsteps == 0) return LBIB_OK;
    s = ensure_graphs(ctx);
    if (s != LBIB_OK) return s;
    if (ctx->s_l == ctx->s_f) {  // open the pipeline: lattice step s_f alone
        int p = (int)(ctx->s_f & 1);
        CK(launch_lbm_bulk(d, ctx->prec, p, (int)(ctx->s_f % 3), ctx->stream));
        CK(launch_lbm_near(d, ctx->prec, p, ctx->near_grid, ctx->near_update_grid, ctx->stream, false));
        ctx->s_f += 1;
        nsteps -= 1;
        ctx->profiled_last = false;
    }
    const int prof = ctx->profiling ? 1 : 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        s = guard_ring(ctx, ctx->s_l + 1);
        if (s != LBIB_OK) return s;
        CK(cudaGraphLaunch(ctx->unit[prof][ctx->s_f % 6], ctx->stream));
        ctx->s_f += 1;
        ctx->s_l += 1;
        ctx->profiled_last = (prof != 0);
    }
    return LBIB_OK;
}

lbib_status lbib_sync(lbib_ctx* ctx)
{
    LBIB_TRACE("lbib_sync");
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    DeviceGuard guard(ctx->device);
    return pre_read(ctx);
}

lbib_status lbib_step_count(lbib_ctx* ctx, int64_t* steps)
{
    if (!ctx || !steps) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    *steps = ctx->s_f;
    return s;
}

static lbib_status read_macro(lbib_ctx* ctx, int32_t inst, double* rho, double* ux, double* uy, size_t n)
{
    if (!valid_instance(ctx, inst)) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such instance");
    const Lattice& L = ctx->d.L;
    const int inx = ctx->inst_nx[inst];
    size_t nn = (size_t)inx * L.ny;
    if (n < nn) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than nx * ny");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK) return s;
    int max_nx = 0;
    for (int v : ctx->inst_nx) max_nx = std::max(max_nx, v);
    const size_t cap = (size_t)max_nx * L.ny;
    if (!ctx->macro_buf) {
        Arena ar;
        ar.add(&ctx->macro_buf, 3 * cap);
        CK(ar.commit(ctx->stream_allocs, ctx->stream));
    }
    int64_t m = ctx->s_f - 1;
    CK(launch_macro(ctx->d, ctx->prec, (int)(ctx->s_f & 1), m, ctx->inst_x0[inst], inx, ctx->macro_buf,
                    ctx->macro_buf + cap, ctx->macro_buf + 2 * cap, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (rho) CK(cudaMemcpy(rho, ctx->macro_buf, nn * 8, cudaMemcpyDeviceToHost));
    if (ux) CK(cudaMemcpy(ux, ctx->macro_buf + cap, nn * 8, cudaMemcpyDeviceToHost));
    if (uy) CK(cudaMemcpy(uy, ctx->macro_buf + 2 * cap, nn * 8, cudaMemcpyDeviceToHost));
    return LBIB_OK;
}

lbib_status lbib_read_instance_velocity(lbib_ctx* ctx, int32_t instance, double* ux, double* uy, size_t n)
{
    LBIB_TRACE("lbib_read_instance_velocity");
    if (!ctx || !ux || !uy) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    return read_macro(ctx, instance, nullptr, ux, uy, n);
}

lbib_status lbib_read_velocity(lbib_ctx* ctx, double* ux, double* uy, size_t n)
{
    return lbib_read_instance_velocity(ctx, 0, ux, uy, n);
}

lbib_status lbib_read_density(lbib_ctx* ctx, double* rho, size_t n)
{
    LBIB_TRACE("lbib_read_density");
    if (!ctx || !rho) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    return read_macro(ctx, 0, rho, nullptr, nullptr, n);
}

lbib_status lbib_read_velocity_device(lbib_ctx* ctx, void* dux, void* duy, size_t n, int32_t dtype)
{
    LBIB_TRACE("lbib_read_velocity_device");
    if (!ctx || !dux || !duy) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (dtype != 0 && dtype != 1) return fail(ctx, LBIB_ERR_INVALID_ARG, "dtype must be 0 (float) or 1 (double)");
    const Lattice& L = ctx->d.L;
    if (n < (size_t)ctx->inst_nx[0] * L.ny) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than nx * ny");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    s = finish_pending(ctx);
    if (s != LBIB_OK) return s;
    CK(launch_macro_typed(ctx->d, ctx->prec, (int)(ctx->s_f & 1), ctx->s_f - 1, ctx->inst_x0[0], ctx->inst_nx[0], dux,
                          duy, dtype, ctx->stream));
    return LBIB_OK;
}

static double wrest(int q) { return q == 0 ? 4.0 / 9.0 : (q < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

// stored deviation element k of a host copy <-> double (the storage rules of
// the device's ld / st: FP16 carries the HALF_SCALE factor)
static double stored_to_double(const lbib_ctx* ctx, const char* raw, size_t k)
{
    switch (ctx->d.store) {
    case STORE_F64: return reinterpret_cast<const double*>(raw)[k];
    case STORE_F32: return (double)reinterpret_cast<const float*>(raw)[k];
    case STORE_BF16: return (double)__bfloat162float(reinterpret_cast<const __nv_bfloat16*>(raw)[k]);
    default: return (double)(__half2float(reinterpret_cast<const __half*>(raw)[k]) * (1.0f / HALF_SCALE));
    }
}

static void double_to_stored(const lbib_ctx* ctx, char* raw, size_t k, double v)
{
    switch (ctx->d.store) {
    case STORE_F64: reinterpret_cast<double*>(raw)[k] = v; break;
    case STORE_F32: reinterpret_cast<float*>(raw)[k] = (float)v; break;
    case STORE_BF16: reinterpret_cast<__nv_bfloat16*>(raw)[k] = __float2bfloat16_rn((float)v); break;
    default: reinterpret_cast<__half*>(raw)[k] = __float2half_rn((float)v * HALF_SCALE); break;
    }
}

lbib_status lbib_read_instance_populations(lbib_ctx* ctx, int32_t instance, double* f, size_t n)
{
    LBIB_TRACE("lbib_read_instance_populations");
    if (!ctx || !f) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (!valid_instance(ctx, instance)) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such instance");
    const Lattice& L = ctx->d.L;
    const int inx = ctx->inst_nx[instance], x0 = ctx->inst_x0[instance];
    size_t nn = (size_t)inx * L.ny;
    if (n < 9 * nn) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than 9 nx ny");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK) return s;
    // one strided copy per direction: rows of the instance's columns
    const size_t es = ctx->ssz;
    std::vector<char> raw((size_t)9 * nn * es);
    const char* src = static_cast<const char*>(ctx->d.f[ctx->s_f & 1]);
    for (int q = 0; q < 9; ++q)
        CK(cudaMemcpy2D(raw.data() + (size_t)q * nn * es, (size_t)inx * es, src + ((size_t)q * L.qstride + x0) * es,
                        (size_t)L.nxp * es, (size_t)inx * es, L.ny, cudaMemcpyDeviceToHost));
    for (int q = 0; q < 9; ++q)
        for (size_t i = 0; i < nn; ++i) {
            const size_t k = (size_t)q * nn + i;
            f[k] = stored_to_double(ctx, raw.data(), k) + wrest(q);
        }
    return LBIB_OK;
}

lbib_status lbib_read_populations(lbib_ctx* ctx, double* f, size_t n)
{
    return lbib_read_instance_populations(ctx, 0, f, n);
}

lbib_status lbib_write_instance_populations(lbib_ctx* ctx, int32_t instance, const double* f, size_t n)
{
    LBIB_TRACE("lbib_write_instance_populations");
    if (!ctx || !f) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (!valid_instance(ctx, instance)) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such instance");
    const Lattice& L = ctx->d.L;
    const int inx = ctx->inst_nx[instance], x0 = ctx->inst_x0[instance];
    size_t nn = (size_t)inx * L.ny;
    if (n < 9 * nn) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than 9 nx ny");
    if (ctx->s_f != 0) return fail(ctx, LBIB_ERR_STATE, "populations can only be written before the first step");
    DeviceGuard guard(ctx->device);
    const size_t es = ctx->ssz;
    std::vector<char> raw((size_t)9 * nn * es);
    for (int q = 0; q < 9; ++q)
        for (size_t i = 0; i < nn; ++i) {
            const size_t k = (size_t)q * nn + i;
            double_to_stored(ctx, raw.data(), k, f[k] - wrest(q));
        }
    CK(cudaStreamSynchronize(ctx->stream));
    char* dst = static_cast<char*>(ctx->d.f[0]);
    for (int q = 0; q < 9; ++q)
        CK(cudaMemcpy2DAsync(dst + ((size_t)q * L.qstride + x0) * es, (size_t)L.nxp * es,
                             raw.data() + (size_t)q * nn * es, (size_t)inx * es, (size_t)inx * es, L.ny,
                             cudaMemcpyHostToDevice, ctx->stream));
    return LBIB_OK;
}

lbib_status lbib_write_populations(lbib_ctx* ctx, const double* f, size_t n)
{
    return lbib_write_instance_populations(ctx, 0, f, n);
}

lbib_status lbib_read_instance_observables(lbib_ctx* ctx, int32_t instance, lbib_obs* out, size_t cap,
                                           size_t* n_out)
{
    LBIB_TRACE("lbib_read_instance_observables");
    if (!ctx || !n_out || (cap && !out)) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (!valid_instance(ctx, instance)) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such instance");
    *n_out = 0;
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (ctx->inst_nbodies[instance] == 0) return s;
    const int64_t last = ctx->s_l, rc = ctx->d.ring_cap;
    int64_t& consumed = ctx->obs_consumed[instance];
    int64_t first = std::max<int64_t>(consumed + 1, last - rc + 1);
    int64_t cnt = std::min<int64_t>((int64_t)cap, last - first + 1);
    const lbib_obs* ring = ctx->d.ring + (size_t)instance * rc;
    // the requested steps occupy at most two contiguous runs of the ring
    int64_t k = 0;
    while (k < cnt) {
        const int64_t slot = (first + k) % rc;
        const int64_t run = std::min<int64_t>(cnt - k, rc - slot);
        CK(cudaMemcpy(out + k, ring + slot, (size_t)run * sizeof(lbib_obs), cudaMemcpyDeviceToHost));
        k += run;
    }
    if (cnt > 0) consumed = first + cnt - 1;
    *n_out = (size_t)std::max<int64_t>(cnt, 0);
    return s;
}

lbib_status lbib_read_latest_observables(lbib_ctx* ctx, lbib_obs* out, size_t n)
{
    LBIB_TRACE("lbib_read_latest_observables");
    if (!ctx || !out) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (n < (size_t)ctx->ninst) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than n_instances");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK && s != LBIB_ERR_DIVERGED) return s;
    const int64_t rc = ctx->d.ring_cap, last = ctx->s_l;
    if (ctx->d.nbodies > 0 && last > 0) {
        // one strided copy: slot last % rc of every instance's ring
        CK(cudaMemcpy2D(out, sizeof(lbib_obs), ctx->d.ring + last % rc, (size_t)rc * sizeof(lbib_obs),
                        sizeof(lbib_obs), (size_t)ctx->ninst, cudaMemcpyDeviceToHost));
    }
    for (int i = 0; i < ctx->ninst; ++i)
        if (ctx->inst_nbodies[i] == 0 || last == 0) {
            std::memset(&out[i], 0, sizeof(lbib_obs));
            out[i].step = -1;
        }
    return s;
}

lbib_status lbib_read_latest_observables_async(lbib_ctx* ctx, lbib_obs* out, size_t n)
{
    LBIB_TRACE("lbib_read_latest_observables_async");
    if (!ctx || !out) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (n < (size_t)ctx->ninst) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than n_instances");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    const int64_t rc = ctx->d.ring_cap, last = ctx->s_l;
    for (int i = 0; i < ctx->ninst; ++i)
        if (ctx->inst_nbodies[i] == 0 || last == 0) {
            std::memset(&out[i], 0, sizeof(lbib_obs));
            out[i].step = -1;
        }
    if (ctx->d.nbodies > 0 && last > 0) {
        // every instance's ring slot last % rc, copied on the copy stream after
        // the steps enqueued so far, so the next step need not wait for it;
        // instances without membranes have no ring entries and keep the record
        // set above
        CK(cudaEventRecord(ctx->ev_step, ctx->stream));
        CK(cudaStreamWaitEvent(ctx->copy, ctx->ev_step, 0));
        for (int i = 0; i < ctx->ninst;) {
            if (ctx->inst_nbodies[i] == 0) {
                ++i;
                continue;
            }
            int j = i;
            while (j < ctx->ninst && ctx->inst_nbodies[j] != 0) ++j;  // a run of instances with membranes
            CK(cudaMemcpy2DAsync(out + i, sizeof(lbib_obs), ctx->d.ring + (size_t)i * rc + last % rc,
                                 (size_t)rc * sizeof(lbib_obs), sizeof(lbib_obs), (size_t)(j - i),
                                 cudaMemcpyDeviceToHost, ctx->copy));
            i = j;
        }
        CK(cudaEventRecord(ctx->ev_copy, ctx->copy));
        if (!ctx->copy_pending) {
            ctx->copy_pending = true;
            ctx->copy_first = last;
        }
    }
    return LBIB_OK;
}

lbib_status lbib_read_observables(lbib_ctx* ctx, lbib_obs* out, size_t cap, size_t* n_out)
{
    return lbib_read_instance_observables(ctx, 0, out, cap, n_out);
}

lbib_status lbib_read_markers(lbib_ctx* ctx, int32_t id, double* xy, size_t n)
{
    LBIB_TRACE("lbib_read_markers");
    if (!ctx || !xy) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (id < 0 || id >= (int)ctx->bodies.size()) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such body");
    const int nv = ctx->bodies[id].nv;
    if (n < 2 * (size_t)nv) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than 2 nv");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK && s != LBIB_ERR_DIVERGED) return s;
    const Dev& d = ctx->d;
    const int off = ctx->mark_off[id];
    std::vector<double> x(nv), y(nv);
    const double* P = d.pos[ctx->s_l & 1];
    CK(cudaMemcpy(x.data(), P + off, nv * 8, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(y.data(), P + d.nmark + off, nv * 8, cudaMemcpyDeviceToHost));
    for (int v = 0; v < nv; ++v) {
        xy[2 * v] = x[v];
        xy[2 * v + 1] = y[v];
    }
    return s;
}

lbib_status lbib_read_body_field(lbib_ctx* ctx, int32_t id, int32_t field, double* out, size_t n)
{
    LBIB_TRACE("lbib_read_body_field");
    if (!ctx || !out) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (id < 0 || id >= (int)ctx->bodies.size()) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such body");
    if (field < 0 || field >= LBIB_FIELD_COUNT) return fail(ctx, LBIB_ERR_INVALID_ARG, "unknown field");
    const int nv = ctx->bodies[id].nv;
    if (n < (size_t)nv) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than nv");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK && s != LBIB_ERR_DIVERGED) return s;
    const Dev& d = ctx->d;
    const int off = ctx->mark_off[id];
    if (field <= LBIB_FIELD_YPREV) {
        int64_t k = (field <= LBIB_FIELD_Y) ? ctx->s_l : ctx->s_l - 1;
        const double* P = d.pos[k & 1];
        size_t o = (field == LBIB_FIELD_X || field == LBIB_FIELD_XPREV) ? off : (size_t)d.nmark + off;
        CK(cudaMemcpy(out, P + o, nv * 8, cudaMemcpyDeviceToHost));
        return s;
    }
    size_t o = (size_t)field * d.nmark + off;
    if (ctx->prec == PREC_F64) {
        CK(cudaMemcpy(out, static_cast<double*>(d.diag) + o, nv * 8, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> t(nv);
        CK(cudaMemcpy(t.data(), static_cast<float*>(d.diag) + o, nv * 4, cudaMemcpyDeviceToHost));
        for (int v = 0; v < nv; ++v) out[v] = t[v];
    }
    return s;
}

lbib_status lbib_read_bonds(lbib_ctx* ctx, int32_t id, int32_t* bound, double* ax, double* ay, double* margin,
                            size_t n)
{
    LBIB_TRACE("lbib_read_bonds");
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    if (id < 0 || id >= (int)ctx->bodies.size()) return fail(ctx, LBIB_ERR_INVALID_ARG, "no such body");
    const HostBody& h = ctx->bodies[id];
    if (!h.adhesive) return fail(ctx, LBIB_ERR_INVALID_ARG, "body has no ligands");
    const int nl = h.adh.n_ligands;
    if (n < (size_t)nl) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than n_ligands");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK && s != LBIB_ERR_DIVERGED) return s;
    const Dev& d = ctx->d;
    const int loff = ctx->lig_off[id];
    if (bound) CK(cudaMemcpy(bound, d.bound + loff, nl * 4, cudaMemcpyDeviceToHost));
    if (ax) CK(cudaMemcpy(ax, d.anchor + loff, nl * 8, cudaMemcpyDeviceToHost));
    if (ay) CK(cudaMemcpy(ay, d.anchor + d.nlig + loff, nl * 8, cudaMemcpyDeviceToHost));
    if (margin) {
        if (ctx->prec == PREC_F64) {
            CK(cudaMemcpy(margin, static_cast<double*>(d.margin) + loff, nl * 8, cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> t(nl);
            CK(cudaMemcpy(t.data(), static_cast<float*>(d.margin) + loff, nl * 4, cudaMemcpyDeviceToHost));
            for (int k = 0; k < nl; ++k) margin[k] = t[k];
        }
    }
    return s;
}

// ------------------------------------------------------------- checkpoints
// layout: header | populations f*^{s-1} | force density of the near tiles and
//         their step stamps | X^s | X^{s-1} | X^s as compute-type pairs |
//         rigid | bonds | anchors | markers for lattice step s | extents of
//         X^s | per-vertex diagnostics and bond margins of the last step
namespace {
struct CkHeader {
    uint64_t magic;
    int32_t nx, ny, nbodies, nmark, nlig, prec;
    int64_t steps;
    int32_t ninst, pad;
};
constexpr uint64_t kMagic = 0x334b4350424942ULL;  // "BIBPCK3"

size_t state_bytes(const lbib_ctx* ctx)
{
    const Dev& d = ctx->d;
    size_t nq = (size_t)9 * d.L.qstride;
    size_t nm = std::max(d.nmark, 1), nl = std::max(d.nlig, 1), nb = std::max(d.nbodies, 1);
    size_t nn = (size_t)d.L.qstride;
    return sizeof(CkHeader) + nq * ctx->ssz + 2 * nn * ctx->rsz + (size_t)d.L.ntiles * 4 + 4 * nm * 8 +
           4 * nm * ctx->rsz + nb * RG_N * 8 + nl * 4 + 2 * nl * 8 + 2 * nm * 4 + 4 * nm * ctx->rsz + nb * BO_N * 8 +
           (size_t)NDIAG * nm * ctx->rsz + nl * ctx->rsz;
}
}  // namespace

lbib_status lbib_state_size(lbib_ctx* ctx, size_t* bytes)
{
    if (!ctx || !bytes) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    *bytes = state_bytes(ctx);
    return LBIB_OK;
}

}  // extern "C"

namespace {

// Copies the context state into buf (host or device memory, `kind` the
// direction of every copy) in the layout above.  Everything a later step or
// read uses is saved exactly, so a restored context continues bit for bit.
lbib_status save_into(lbib_ctx* ctx, char* p, cudaMemcpyKind kind)
{
    const Dev& d = ctx->d;
    const int64_t st = ctx->s_f;
    CkHeader h{kMagic, d.L.nx, d.L.ny, d.nbodies, d.nmark, d.nlig, ctx->prec, st, ctx->ninst, 0};
    if (kind == cudaMemcpyDeviceToHost) std::memcpy(p, &h, sizeof(h));
    else CK(cudaMemcpyAsync(p, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->stream));
    p += sizeof(h);
    size_t nq = (size_t)9 * d.L.qstride;
    size_t nm = std::max(d.nmark, 1), nl = std::max(d.nlig, 1), nb = std::max(d.nbodies, 1);
    auto put = [&](const void* src, size_t n) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(p, src, n, kind, ctx->stream);
        p += n;
        return e;
    };
    const size_t nn = (size_t)d.L.qstride;
    CK(put(d.f[st & 1], nq * ctx->ssz));
    CK(put(d.fx, nn * ctx->rsz));
    CK(put(d.fy, nn * ctx->rsz));
    CK(put(d.fresh, (size_t)d.L.ntiles * 4));
    CK(put(d.pos[st & 1], 2 * nm * 8));
    CK(put(d.pos[(st + 1) & 1], 2 * nm * 8));
    CK(put(d.posf[st & 1], 4 * nm * ctx->rsz));
    CK(put(d.rigid, nb * RG_N * 8));
    CK(put(d.bound, nl * 4));
    CK(put(d.anchor, 2 * nl * 8));
    CK(put(d.mki[st & 1], 2 * nm * 4));
    CK(put(d.mkf[st & 1], 4 * nm * ctx->rsz));
    CK(put(d.body_obs[st & 1], nb * BO_N * 8));
    CK(put(d.diag, (size_t)NDIAG * nm * ctx->rsz));
    CK(put(d.margin, nl * ctx->rsz));
    return LBIB_OK;
}

// Restores a state written by save_into (kind: direction of the copies).
lbib_status load_from(lbib_ctx* ctx, const char* p, cudaMemcpyKind kind)
{
    Dev& d = ctx->d;
    CkHeader h;
    if (kind == cudaMemcpyHostToDevice) std::memcpy(&h, p, sizeof(h));
    else {
        CK(cudaMemcpyAsync(&h, p, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    p += sizeof(h);
    if (h.magic != kMagic || h.nx != d.L.nx || h.ny != d.L.ny || h.nbodies != d.nbodies || h.nmark != d.nmark ||
        h.nlig != d.nlig || h.prec != ctx->prec || h.steps < 0 || h.ninst != ctx->ninst)
        return fail(ctx, LBIB_ERR_INVALID_ARG, "checkpoint does not match this context");
    const int64_t st = h.steps;
    size_t nq = (size_t)9 * d.L.qstride;
    size_t nm = std::max(d.nmark, 1), nl = std::max(d.nlig, 1), nb = std::max(d.nbodies, 1);
    auto get = [&](void* dst, size_t n) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(dst, p, n, kind, ctx->stream);
        p += n;
        return e;
    };
    const size_t nn = (size_t)d.L.qstride;
    CK(get(d.f[st & 1], nq * ctx->ssz));
    CK(get(d.fx, nn * ctx->rsz));
    CK(get(d.fy, nn * ctx->rsz));
    CK(get(d.fresh, (size_t)d.L.ntiles * 4));
    CK(get(d.pos[st & 1], 2 * nm * 8));
    CK(get(d.pos[(st + 1) & 1], 2 * nm * 8));
    CK(get(d.posf[st & 1], 4 * nm * ctx->rsz));  // the next membrane update reads these pairs
    CK(get(d.rigid, nb * RG_N * 8));
    CK(get(d.bound, nl * 4));
    CK(get(d.anchor, 2 * nl * 8));
    CK(get(d.mki[st & 1], 2 * nm * 4));
    CK(get(d.mkf[st & 1], 4 * nm * ctx->rsz));
    CK(get(d.body_obs[st & 1], nb * BO_N * 8));
    CK(get(d.diag, (size_t)NDIAG * nm * ctx->rsz));
    CK(get(d.margin, nl * ctx->rsz));
    // scheduling state is rebuilt from the restored positions and markers
    const Lattice& L = d.L;
    for (int i = 0; i < 3; ++i) CK(cudaMemsetAsync(d.nearflag[i], 0, L.ntiles * 4, ctx->stream));
    CK(cudaMemsetAsync(d.mask[0], 0, (size_t)L.ntiles * d.mw * 4, ctx->stream));
    CK(cudaMemsetAsync(d.mask[1], 0, (size_t)L.ntiles * d.mw * 4, ctx->stream));
    CK(cudaMemsetAsync(d.count, 0, 12, ctx->stream));
    CK(cudaMemsetAsync(d.status, 0, 4, ctx->stream));
    CK(cudaMemsetAsync(d.ticket, 0, 4, ctx->stream));
    CK(cudaMemcpyAsync(d.step, &st, 8, cudaMemcpyHostToDevice, ctx->stream));
    ctx->s_f = ctx->s_l = st;
    ctx->obs_consumed.assign(ctx->ninst, st);
    if (d.nbodies) {
        CK(launch_activate(d, ctx->prec, st, 3, ctx->stream));
        CK(launch_rebuild_mask(d, ctx->prec, st, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return check_status(ctx);
}

bool valid_config(const lbib_launch_config& c)
{
    return (c.lagrangian_threads == 256 || c.lagrangian_threads == 512) && c.near_blocks >= 1 &&
           (c.bulk_tiles_y == 1 || c.bulk_tiles_y == 2 || c.bulk_tiles_y == 4) &&
           (c.activation_stride == 1 || c.activation_stride == 2 || c.activation_stride == 4) &&
           (c.bulk_nodes_per_thread == 1 || c.bulk_nodes_per_thread == 2 || c.bulk_nodes_per_thread == 4) &&
           (c.observables_branch == 0 || c.observables_branch == 1) &&
           (c.chain_programmatic == 0 || c.chain_programmatic == 1) && c.near_update_blocks >= 1 &&
           (c.bulk_tma == 0 || c.bulk_tma == 1);
}

lbib_launch_config current_config(const lbib_ctx* ctx)
{
    lbib_launch_config c{};
    c.lagrangian_threads = ctx->d.lag_threads;
    c.near_blocks = ctx->near_grid;
    c.bulk_tiles_y = ctx->d.bulk_tiles_y;
    c.activation_stride = ctx->d.act_stride;
    c.bulk_nodes_per_thread = ctx->d.bulk_nodes_per_thread;
    c.observables_branch = ctx->obs_branch;
    c.chain_programmatic = ctx->chain_pdl;
    c.near_update_blocks = ctx->near_update_grid;
    c.bulk_tma = ctx->d.bulk_tma;
    return c;
}

void destroy_graphs(lbib_ctx* ctx)
{
    for (auto& row : ctx->unit)
        for (auto& g : row)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
}

void apply_config(lbib_ctx* ctx, const lbib_launch_config& c)
{
    destroy_graphs(ctx);
    ctx->d.lag_threads = c.lagrangian_threads;
    ctx->near_grid = c.near_blocks;
    ctx->d.bulk_tiles_y = c.bulk_tiles_y;
    ctx->d.act_stride = c.activation_stride;
    ctx->d.bulk_nodes_per_thread = c.bulk_nodes_per_thread;
    ctx->obs_branch = c.observables_branch;
    ctx->chain_pdl = c.chain_programmatic;
    ctx->near_update_grid = c.near_update_blocks;
    ctx->d.bulk_tma = c.bulk_tma;
}

}  // namespace

extern "C" {

lbib_status lbib_save_state(lbib_ctx* ctx, void* buf, size_t bytes)
{
    LBIB_TRACE("lbib_save_state");
    if (!ctx || !buf) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK) return s;
    if (bytes < state_bytes(ctx)) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than lbib_state_size");
    return save_into(ctx, static_cast<char*>(buf), cudaMemcpyDeviceToHost);
}

lbib_status lbib_load_state(lbib_ctx* ctx, const void* buf, size_t bytes)
{
    LBIB_TRACE("lbib_load_state");
    if (!ctx || !buf) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK && s != LBIB_ERR_DIVERGED && s != LBIB_ERR_STATE && s != LBIB_ERR_TIMEOUT) return s;
    if (bytes < state_bytes(ctx)) return fail(ctx, LBIB_ERR_INVALID_ARG, "buffer smaller than lbib_state_size");
    s = load_from(ctx, static_cast<const char*>(buf), cudaMemcpyHostToDevice);
    if (s == LBIB_OK) ctx->fault = LBIB_OK;  // a trusted state again
    return s;
}

lbib_status lbib_inject_fault(lbib_ctx* ctx, int32_t kind)
{
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    if (kind != LBIB_FAULT_WAIT_TIMEOUT) return fail(ctx, LBIB_ERR_INVALID_ARG, "unknown fault kind");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    // the status bit a bulk-update block sets when its bounded wait for a
    // tensor copy gives up, raised in stream order after the work enqueued so far
    k_raise_status<<<1, 1, 0, ctx->stream>>>(ctx->d.status, ST_TMA_TIMEOUT);
    CK(cudaGetLastError());
    return LBIB_OK;
}

void lbib_inject_alloc_failure(int64_t after) { g_alloc_countdown.store(after < 0 ? -1 : (long long)after); }

lbib_status lbib_release_cached_memory(int32_t device)
{
    if (device < 0 || device >= 64) return fail(nullptr, LBIB_ERR_INVALID_ARG, "device ordinal");
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        pool = g_pool[device];
    }
    if (!pool) return LBIB_OK;  // nothing cached on that device
    DeviceGuard guard(device);
    cudaError_t e = cudaDeviceSynchronize();  // frees still in flight reach the pool first
    if (e == cudaSuccess) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "lbib_release_cached_memory");
    return LBIB_OK;
}

lbib_status lbib_get_launch_config(lbib_ctx* ctx, lbib_launch_config* out)
{
    if (!ctx || !out) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    *out = current_config(ctx);
    return LBIB_OK;
}

lbib_status lbib_set_launch_config(lbib_ctx* ctx, const lbib_launch_config* cfg)
{
    if (!ctx || !cfg) return fail(ctx, LBIB_ERR_INVALID_ARG, "null argument");
    if (!valid_config(*cfg)) return fail(ctx, LBIB_ERR_INVALID_ARG, "launch configuration out of range");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    s = finish_pending(ctx);
    if (s != LBIB_OK) return s;
    // no wait: launches already enqueued keep the parameters they were given,
    // and a step graph still in flight is freed when it completes
    apply_config(ctx, *cfg);
    return LBIB_OK;
}

lbib_status lbib_autotune(lbib_ctx* ctx, int32_t steps_per_trial, lbib_launch_config* chosen)
{
    LBIB_TRACE("lbib_autotune");
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    if (steps_per_trial < 1) return fail(ctx, LBIB_ERR_INVALID_ARG, "steps_per_trial < 1");
    DeviceGuard guard(ctx->device);
    lbib_status s = pre_read(ctx);
    if (s != LBIB_OK) return s;
    Dev& d = ctx->d;
    // device snapshot of the state, the observables rings and the cursors
    const size_t sb = state_bytes(ctx);
    const size_t rb = (size_t)ctx->ninst * d.ring_cap * sizeof(lbib_obs);
    char* snap = nullptr;
    lbib_obs* ring = nullptr;
    CK(device_malloc(reinterpret_cast<void**>(&snap), sb));
    cudaError_t e = device_malloc(reinterpret_cast<void**>(&ring), std::max<size_t>(rb, 1));
    if (e != cudaSuccess) {
        cudaFree(snap);
        return cuda_fail(ctx, e, "cudaMalloc");
    }
    const std::vector<int64_t> cursors = ctx->obs_consumed;
    const lbib_launch_config entry = current_config(ctx);
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    cudaEvent_t a = nullptr, b = nullptr;
    auto cleanup = [&]() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
        cudaFree(snap);
        cudaFree(ring);
    };
    s = save_into(ctx, snap, cudaMemcpyDeviceToDevice);
    if (s == LBIB_OK && rb) {
        e = cudaMemcpyAsync(ring, d.ring, rb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "ring snapshot");
    }
    if (s == LBIB_OK && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
        s = cuda_fail(ctx, cudaErrorUnknown, "cudaEventCreate");
    // one trial: restore, two warm-up steps, then the faster of two timed runs
    // of steps_per_trial steps
    auto trial = [&](const lbib_launch_config& c, float* ms) -> lbib_status {
        apply_config(ctx, c);
        lbib_status t = load_from(ctx, snap, cudaMemcpyDeviceToDevice);
        if (t != LBIB_OK) return t;
        t = lbib_advance(ctx, 2);
        if (t != LBIB_OK) return t;
        *ms = 3.4e38f;
        for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(a, ctx->stream));
            t = lbib_advance(ctx, steps_per_trial);
            if (t != LBIB_OK) return t;
            CK(cudaEventRecord(b, ctx->stream));
            CK(cudaEventSynchronize(b));
            float r = 0.f;
            CK(cudaEventElapsedTime(&r, a, b));
            *ms = std::min(*ms, r);
        }
        t = finish_pending(ctx);
        if (t != LBIB_OK) return t;
        CK(cudaStreamSynchronize(ctx->stream));
        return check_status(ctx);
    };
    lbib_launch_config best = entry;
    float best_ms = 0.f;
    if (s == LBIB_OK) s = trial(best, &best_ms);
    auto consider = [&](lbib_launch_config c) {
        if (s != LBIB_OK || !valid_config(c)) return;
        if (c.lagrangian_threads == best.lagrangian_threads && c.near_blocks == best.near_blocks &&
            c.bulk_tiles_y == best.bulk_tiles_y && c.activation_stride == best.activation_stride &&
            c.bulk_nodes_per_thread == best.bulk_nodes_per_thread && c.observables_branch == best.observables_branch &&
            c.chain_programmatic == best.chain_programmatic && c.near_update_blocks == best.near_update_blocks &&
            c.bulk_tma == best.bulk_tma)
            return;
        float ms = 0.f;
        s = trial(c, &ms);
        if (s == LBIB_OK && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    // coordinate descent, two rounds: the bulk shape and the near grid interact
    // (the near blocks take SMs from the bulk blocks), so the second round
    // revisits each coordinate from the first round's optimum
    for (int round = 0; round < 2; ++round) {
        const lbib_launch_config start = best;
        for (int npt : {1, 2, 4})
            for (int rt : {1, 2, 4}) {
                lbib_launch_config c = start;
                c.bulk_tiles_y = rt;
                c.bulk_nodes_per_thread = npt;
                c.bulk_tma = 0;
                consider(c);
            }
        if (d.fmaps) {
            lbib_launch_config c = start;
            c.bulk_tma = 1;
            consider(c);
        }
        if (d.nbodies) {
            const lbib_launch_config after_bulk = best;
            for (int lt : {256, 512}) {
                lbib_launch_config c = after_bulk;
                c.lagrangian_threads = lt;
                consider(c);
            }
            const lbib_launch_config after_lag = best;
            for (int stride : {1, 2, 4}) {
                lbib_launch_config c = after_lag;
                c.activation_stride = stride;
                consider(c);
            }
            const lbib_launch_config after_stride = best;
            for (int per_sm : {2, 4, 6, 8, 12}) {
                lbib_launch_config c = after_stride;
                c.near_blocks = per_sm * nsm;
                consider(c);
            }
            const lbib_launch_config after_gather = best;
            for (int per_sm : {4, 8, 16}) {
                lbib_launch_config c = after_gather;
                c.near_update_blocks = per_sm * nsm;
                consider(c);
            }
            const lbib_launch_config after_near = best;
            for (int ob : {0, 1}) {
                lbib_launch_config c = after_near;
                c.observables_branch = ob;
                consider(c);
            }
            const lbib_launch_config after_obs = best;
            for (int pdl : {0, 1}) {
                lbib_launch_config c = after_obs;
                c.chain_programmatic = pdl;
                consider(c);
            }
        }
    }
    // back to the entry state with the chosen configuration
    if (s == LBIB_OK) {
        apply_config(ctx, best);
        s = load_from(ctx, snap, cudaMemcpyDeviceToDevice);
    }
    if (s == LBIB_OK && rb) {
        e = cudaMemcpyAsync(d.ring, ring, rb, cudaMemcpyDeviceToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) s = cuda_fail(ctx, e, "ring restore");
    }
    ctx->obs_consumed = cursors;
    cleanup();
    if (s == LBIB_OK && chosen) *chosen = best;
    return s;
}

lbib_status lbib_set_profiling(lbib_ctx* ctx, int32_t enable)
{
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    if (enable && !ctx->pe[0]) {  // timing events only for contexts that profile
        DeviceGuard guard(ctx->device);
        for (int i = 0; i < 6; ++i) CK(cudaEventCreate(&ctx->pe[i]));
    }
    ctx->profiling = enable != 0;
    return LBIB_OK;
}

lbib_status lbib_read_kernel_times(lbib_ctx* ctx, float* bulk_ms, float* lagr_ms, float* near_ms)
{
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    DeviceGuard guard(ctx->device);
    float t[3] = {0, 0, 0};
    if (ctx->profiled_last) {
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaEventElapsedTime(&t[0], ctx->pe[0], ctx->pe[1]));
        CK(cudaEventElapsedTime(&t[1], ctx->pe[2], ctx->pe[3]));
        CK(cudaEventElapsedTime(&t[2], ctx->pe[4], ctx->pe[5]));
    }
    if (bulk_ms) *bulk_ms = t[0];
    if (lagr_ms) *lagr_ms = t[1];
    if (near_ms) *near_ms = t[2];
    return LBIB_OK;
}

lbib_status lbib_describe(lbib_ctx* ctx, int32_t* kernels_per_step, int32_t* near_tiles, int32_t* tiles)
{
    if (!ctx) return fail(ctx, LBIB_ERR_INVALID_ARG, "null context");
    DeviceGuard guard(ctx->device);
    lbib_status s = finalize(ctx);
    if (s != LBIB_OK) return s;
    if (kernels_per_step) *kernels_per_step = ctx->d.nbodies ? 6 : 1;
    if (tiles) *tiles = ctx->d.L.ntiles;
    if (near_tiles) {
        int32_t c[3] = {0, 0, 0};
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMemcpy(c, ctx->d.count, 12, cudaMemcpyDeviceToHost));
        *near_tiles = c[ctx->s_f % 3];
    }
    return LBIB_OK;
}

void lbib_destroy(lbib_ctx* ctx)
{
    LBIB_TRACE("lbib_destroy");
    if (!ctx) return;
    DeviceGuard guard(ctx->device);
    // no wait for the device: graphs still in flight are freed when they
    // complete, and the arenas are freed in the stream's order after them and
    // after the last observables copy (which reads the ring)
    if (ctx->stream && ctx->ev_copy) cudaStreamWaitEvent(ctx->stream, ctx->ev_copy, 0);
    destroy_graphs(ctx);
    for (void* p : ctx->stream_allocs) cudaFreeAsync(p, ctx->stream);
    if (!ctx->allocs.empty() && ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (void* p : ctx->allocs) cudaFree(p);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_lag) cudaEventDestroy(ctx->ev_lag);
    if (ctx->ev_obs) cudaEventDestroy(ctx->ev_obs);
    if (ctx->obs) cudaStreamDestroy(ctx->obs);
    if (ctx->copy) cudaStreamDestroy(ctx->copy);
    if (ctx->act) cudaStreamDestroy(ctx->act);
    if (ctx->ev_act) cudaEventDestroy(ctx->ev_act);
    if (ctx->ev_step) cudaEventDestroy(ctx->ev_step);
    if (ctx->ev_copy) cudaEventDestroy(ctx->ev_copy);
    for (auto& e : ctx->pe)
        if (e) cudaEventDestroy(e);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    cudaGetLastError();
    delete ctx;
}

}  // extern "C"
