// hrc_runtime.cu -- host runtime behind the C ABI of include/hrc.h:
// contexts, buffer plans, ray-shape tables, arc tables and launch sequencing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "hrc.h"
#include "hrc_internal.cuh"
#include "launch.h"

using namespace hrc;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace hrc {

void set_global_error(const char *msg) { g_create_error = msg; }

// Kernel attributes are per device: set them once for each device used.
cudaError_t prepare_device_once() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return cudaSuccess;
    e = prepare_forward_kernels();
    if (e == cudaSuccess) e = prepare_backward_kernels();
    if (e == cudaSuccess) done[dev] = true;
    return e;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int levels_for(int U, int cascades) {
    int N = 0;
    while ((1 << N) < U) ++N;
    if (cascades > 0 && cascades < N) N = cascades;
    return N;
}

size_t sl_bytes(int prec) { return prec == P_FP32 ? 4 : (prec == P_FP64 ? 8 : 2); }
size_t st_bytes(int prec) { return prec == P_FP64 ? 8 : 4; }

// Ray shapes of the directly traced levels 0..2 (Sec. 4.2): from a pixel
// centre (1/2, 1/2) along v_n(k) = (2^n, 2k - 2^n).  The segment is clipped
// against the integer grid lines in exact integer arithmetic: with
// a = 2^n and b = 2k - 2^n, the crossings of u = g are at t = (2g-1)/(2a)
// and those of v at t = (2m-1)/(2|b|); over the common denominator 2a|b|
// all crossing parameters are integers.  Zero-length pieces (the ray
// passing exactly through a grid corner) are dropped.
RayTable make_ray_table() {
    RayTable rt;
    std::memset(&rt, 0, sizeof(rt));
    int np = 0;
    for (int n = 0; n <= 2; ++n) {
        const int a = 1 << n;
        for (int k = 0; k <= a; ++k) {
            const int r = ray_id(n, k);
            rt.start[r] = np;
            const int b = 2 * k - a, ab = b < 0 ? -b : b;
            const long long D = 2LL * a * (ab > 0 ? ab : 1);
            std::vector<long long> ts = {0, D};
            for (int g = 1; g <= a; ++g) ts.push_back((2LL * g - 1) * (D / (2LL * a)));
            for (int m = 1; m <= ab; ++m) ts.push_back((2LL * m - 1) * (D / (2LL * ab)));
            std::sort(ts.begin(), ts.end());
            ts.erase(std::unique(ts.begin(), ts.end()), ts.end());
            const double len = std::sqrt(double(a) * a + double(b) * b);
            for (size_t i = 0; i + 1 < ts.size(); ++i) {
                const double tm = 0.5 * double(ts[i] + ts[i + 1]) / double(D);
                const int du = (int)std::floor(0.5 + a * tm);
                const int dv = (int)std::floor(0.5 + b * tm);
                const double l = double(ts[i + 1] - ts[i]) / double(D) * len;
                rt.p[np].du = (int8_t)du;
                rt.p[np].dv = (int8_t)dv;
                rt.p[np].len = (float)l;
                rt.lenD[np] = l;
                ++np;
            }
        }
    }
    rt.start[HRC_MAXRAY] = np;
    return rt;
}

// Lays out T_0..T_N and R_0..R_{N-1} of all four frames from byte `off`
// (and, with `adjoint`, the dL/dT_n and dL/dR_n buffers of the backward
// pass); returns the end offset.
size_t build_plan(int W, int H, int C, int cascades, int prec, size_t off, Plan &pl, bool adjoint) {
    std::memset(&pl, 0, sizeof(pl));
    pl.W = W; pl.H = H; pl.C = C; pl.prec = prec;
    pl.sched = 0;
    pl.mgroups = 1;
    pl.mthreads = 128;
    pl.vmajor = 0;
    pl.mdown = 0;
    pl.bulk_limit_ns = 2000000000LL;   // 2 s
    pl.bulk_extra_tx = 0;
    const size_t SLb = sl_bytes(prec), STb = st_bytes(prec);
    int Nmax = 0;
    for (int q = 0; q < 4; ++q) {
        QuadGeom &g = pl.q[q];
        g.U = q < 2 ? W : H;
        g.V = q < 2 ? H : W;
        g.Vs = (int)align_up((size_t)g.V, 32);
        g.N = levels_for(g.U, cascades);
        Nmax = std::max(Nmax, g.N);
        for (int n = 0; n <= g.N; ++n) {
            g.Un[n] = (g.U + (1 << n) - 1) >> n;
            const size_t G = (size_t)g.Vs * (C * SLb + STb);
            g.Toff[n] = (long long)off;
            off = align_up(off + (size_t)g.Un[n] * ((1u << n) + 1) * G, 256);
        }
        for (int n = 0; n < g.N; ++n) {
            g.Roff[n] = (long long)off;
            off = align_up(off + (size_t)g.Un[n] * (1u << n) * C * g.Vs * SLb, 256);
        }
    }
    // adjoint buffers (arithmetic type: fp64 for the fp64 precision, else fp32)
    const size_t Ab = prec == P_FP64 ? 8 : 4;
    for (int q = 0; q < 4 && adjoint; ++q) {
        QuadGeom &g = pl.q[q];
        for (int n = 0; n <= g.N; ++n) {
            g.gToff[n] = (long long)off;
            off = align_up(off + (size_t)g.Un[n] * ((1u << n) + 1) * g.Vs * (C + 1) * Ab, 256);
        }
        for (int n = 0; n < g.N; ++n) {
            g.gRoff[n] = (long long)off;
            off = align_up(off + (size_t)g.Un[n] * (1u << n) * C * g.Vs * Ab, 256);
        }
    }
    pl.arcs_off = (long long)off;
    off = align_up(off + sizeof(float) * (size_t(2) << Nmax), 256);
    pl.arcs_off_d = (long long)off;
    off = align_up(off + sizeof(double) * (size_t(2) << Nmax), 256);
    return off;
}

int plan_nmax(const Plan &pl) {
    int N = 0;
    for (int q = 0; q < 4; ++q) N = std::max(N, pl.q[q].N);
    return N;
}

// Eq. 13: A_n(j + 1/2) = angle(v_n(j + 1)) - angle(v_n(j)), angle = atan(y/x).
void fill_arcs(int Nmax, std::vector<float> &af, std::vector<double> &ad) {
    af.assign(size_t(2) << Nmax, 0.f);
    ad.assign(size_t(2) << Nmax, 0.0);
    for (int n = 0; n <= Nmax; ++n) {
        const double s = double(1 << n);
        for (int j = 0; j < (1 << n); ++j) {
            const double a = std::atan2(2.0 * (j + 1) - s, s) - std::atan2(2.0 * j - s, s);
            ad[(size_t(1) << n) + j] = a;
            af[(size_t(1) << n) + j] = (float)a;
        }
    }
}

}  // namespace hrc

struct hrc_ctx {
    int W = 0, H = 0, C = 0, cascades = 0;
    int prec = P_FP32;
    int sched = 0;
    int mgroups = 1;
    int mthreads = 128;
    int vmajor = 0;
    int mdown = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    RayTable rt;
    Plan plan;                   // layout of the current (non-fp64) precision
    Plan plan64;                 // fp64 layout (arena64)
    char *arena = nullptr;
    size_t arena_bytes = 0;
    char *arena64 = nullptr;
    size_t arena64_bytes = 0;
    char *pctl = nullptr;        // control block of the persistent merge down (ticket, status, counters)
    size_t pctl_bytes = 0;
    float *dev_e = nullptr, *dev_s = nullptr, *dev_F = nullptr;   // hrc_fluence_host staging
    const void *last_e = nullptr, *last_s = nullptr;
    bool have_fwd = false;
    bool bwd_recompute = false;  // backward recomputes the levels instead of reading the forward's
    Branches br{};               // the forward's four frame branches (launch schedule 2)
    bool br_ok = false;
    bool blur = false;           // cross blur (Eq. 21) after the fluence sum
    float blur_thr = 0.5f;       // its opacity threshold
    void *blur_buf = nullptr;    // W * H * C doubles: unblurred F, or dL/d(unblurred F)
    // multiple bounces: e_1..e_cap and F_0..F_{cap-1} of the last bounce
    // forward, then the backward's dL/de_k, dL/dF_{k-1} and dL/dsigma_k
    int bounce_cap = 0;
    char *bounce_buf = nullptr;
    size_t bounce_plane = 0;        // bytes of one [C][H][W] set of doubles
    bool have_bounce = false;       // a bounce forward ran (its inputs below)
    const void *last_a = nullptr;
    int last_K = 0;
    bool bounce_levels_ok = false;  // the level buffers hold those of bounce last_K
    // environment map: per-frame, per-level cone values (kernels_env.cu), and
    // a copy of the map with 16-byte-aligned rows (for per-channel contexts)
    char *env_tab = nullptr;
    bool env_on = false;
    float *env_map = nullptr;
    int env_M = 0, env_pitch = 0;
    // or the top-level radiance supplied by the caller: [C][4 K] per channel
    // (channel c's [4][K] table, for per-channel contexts)
    bool env_top = false;
    float *top_map = nullptr;
    int top_K = 0;
    size_t top_cap = 0;
    // per-channel extinction: one single-channel context per channel (the
    // method separates exactly by channel once the extinction does), on this
    // context's stream; channel planes whose address is not 16-byte aligned
    // (W * H not a multiple of 4) pass through kStagePlanes aligned buffers
    bool per_channel = false;
    std::vector<hrc_ctx *> chan;
    char *chan_stage = nullptr;
    size_t chan_plane = 0;
    static constexpr int kStagePlanes = 7;   // e, sigma, albedo, F / dL/dF, dL/de, dL/dsigma, dL/dalbedo
    int launches = 0;
    Recorder rec;
    int timing_mode = 0;         // 0 off, 1 direct launches with events, 2 / 3 events inside the graphs
    std::string err;
    // CUDA graphs of whole passes, keyed by pass kind, precision, schedule
    // and the caller's pointers; captured on a context-owned stream and
    // replayed on the caller's stream.
    struct GraphEntry {
        int kind = -1, prec = -1, sched = -1, mgroups = -1, tune = -1;
        int timed = 0;                       // captured with event-record nodes: the timing mode (2 or 3)
        std::vector<Recorder::Rec> recs;     // those nodes' events
        const void *p[8] = {};
        cudaGraphExec_t exec = nullptr;
        int launches = 0;
        long long replays = 0;
    };
    GraphEntry graphs[8];
    int graph_next = 0;
    bool use_graphs = true;
    long long graph_captures = 0;   // graphs captured and instantiated so far
    // Passes whose pointer set is new while the cache thrashes (most cached
    // graphs never replayed: the caller's tensors move every call) launch
    // directly; the keys of those passes are remembered, and one that comes
    // back is captured after all.
    unsigned long long seen[16] = {};
    int seen_next = 0;
    cudaStream_t cap_stream = nullptr;
    // batched contexts
    bool batched = false;
    int nscenes = 0;
    std::vector<int> Ws, Hs;
    std::vector<Plan> bplans;
    std::vector<long long> eoff, soff;
    Plan *d_plans = nullptr;
    long long *d_eoff = nullptr, *d_soff = nullptr;
    StageBlock *d_blocks[3] = {nullptr, nullptr, nullptr};
    int *d_chunk[3] = {nullptr, nullptr, nullptr};   // ticket -> block index per mode
    // tile steps of every scene as ordinary launches around the persistent one
    struct TileLaunch {
        int kind = 0, pair = 0, total = 0;
        bool before = true;              // before the persistent launch (trace) or after (adjoint trace)
        int *d_off = nullptr, *d_nx = nullptr;
        double bytes = 0;
    };
    std::vector<TileLaunch> tiles[3];
    // schedule 2: level-major multi-scene launches of each mode
    struct MultiLaunch {
        int kind = 0, level = 0, blocks = 0, nent = 0;
        MultiEnt *d_ents = nullptr;
        double bytes = 0;
    };
    std::vector<MultiLaunch> multi[3];
    int nblocks[3] = {0, 0, 0};
    long long total[3] = {0, 0, 0};
    double bbytes[3] = {0, 0, 0};
    int *d_counters = nullptr;
    int ncounters[3] = {0, 0, 0};
    unsigned long long *d_ticket = nullptr;
    int *d_status = nullptr;
    int withhold = -1;
    long long spin_limit = 1LL << 24;   // ~2 s of 128 ns polls
    int blocks_per_sm = 0;              // 0: as many as fit
    int order = 0;                      // 0: scenes in input order per stage, 1: largest first
    // schedule 1: one graph whose branches are the scenes' per-level launch
    // chains, spread over kAux streams (forked from and joined to the pass)
    int bsched = 0;
    static constexpr int kAux = 8;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kAux] = {};
    std::vector<int> by_size;           // scene indices, largest first
};

namespace {

hrc_status fail(hrc_ctx *ctx, hrc_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_error = msg;
    return st;
}

hrc_status cuda_fail(hrc_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, HRC_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

namespace hrc {

cudaError_t read_plan_status(const Plan &pl, int *status) {
    *status = 0;
    if (!pl.status) return cudaSuccess;
    cudaError_t e = cudaMemcpy(status, pl.status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && *status != 0) e = cudaMemset(pl.status, 0, sizeof(int));
    return e;
}

}  // namespace hrc

namespace {

// Upload the arc tables of a plan into its arena.
cudaError_t upload_arcs(const Plan &pl, char *arena) {
    std::vector<float> af;
    std::vector<double> ad;
    fill_arcs(plan_nmax(pl), af, ad);
    cudaError_t e = cudaMemcpy(arena + pl.arcs_off, af.data(), af.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    return cudaMemcpy(arena + pl.arcs_off_d, ad.data(), ad.size() * sizeof(double), cudaMemcpyHostToDevice);
}

// Enqueue one pass (forward or backward) on the context's stream: replay its
// CUDA graph when one exists for these pointers, capture one otherwise.
// With per-launch timing on, the kernels are launched directly.
struct PassKey {
    const void *p[8];
};

template <class ENQ>
hrc_status run_pass(hrc_ctx *ctx, int kind, const void *p0, const void *p1, const void *p2, const void *p3,
                    const void *p4, ENQ &&enqueue, const char *where);

// Same, keyed by up to eight pointers (or counts cast to pointers).
template <class ENQ>
hrc_status run_pass_key(hrc_ctx *ctx, int kind, const PassKey &pk, ENQ &&enqueue, const char *where) {
    ctx->launches = 0;
    if ((ctx->rec.on && ctx->timing_mode == 1) || !ctx->use_graphs) {
        ctx->rec.ext = false;
        ctx->rec.coarse = false;
        ctx->rec.reset(ctx->stream);
        cudaError_t e = enqueue(ctx->stream, &ctx->launches, &ctx->rec);
        ctx->rec.finish();
        if (e != cudaSuccess) return cuda_fail(ctx, e, where);
        return HRC_OK;
    }
    const bool timed = ctx->rec.on;
    const void *const *key = pk.p;
    for (auto &g : ctx->graphs) {
        if (g.exec && g.kind == kind && g.prec == ctx->prec && g.sched == ctx->sched && g.mgroups == ctx->mgroups &&
            g.tune == ctx->mthreads * 8 + ctx->vmajor * 4 + ctx->mdown && g.timed == (timed ? ctx->timing_mode : 0) &&
            std::memcmp(g.p, key, sizeof(pk.p)) == 0) {
            cudaError_t e = cudaGraphLaunch(g.exec, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, where);
            ++g.replays;
            ctx->launches = g.launches;
            if (timed) ctx->rec.recs = g.recs;
            return HRC_OK;
        }
    }
    if (!timed) {
        // the key of this pass (FNV-1a over the pass kind, the configuration and the pointers)
        unsigned long long hk = 1469598103934665603ULL;
        auto mix = [&hk](unsigned long long v) {
            for (int b = 0; b < 8; ++b) {
                hk ^= (v >> (8 * b)) & 0xffULL;
                hk *= 1099511628211ULL;
            }
        };
        mix((unsigned long long)kind);
        mix((unsigned long long)ctx->prec);
        mix((unsigned long long)ctx->sched);
        mix((unsigned long long)ctx->mgroups);
        mix((unsigned long long)(ctx->mthreads * 8 + ctx->vmajor * 4 + ctx->mdown));
        for (int i = 0; i < 8; ++i) mix((unsigned long long)(uintptr_t)key[i]);
        int unreplayed = 0;
        for (const auto &g : ctx->graphs) unreplayed += (g.exec && g.replays == 0) ? 1 : 0;
        bool seen = false;
        for (unsigned long long h : ctx->seen) seen = seen || h == hk;
        if (unreplayed >= 6 && !seen) {
            ctx->seen[ctx->seen_next] = hk;
            ctx->seen_next = (ctx->seen_next + 1) % 16;
            ctx->rec.ext = false;
            ctx->rec.coarse = false;
            ctx->rec.reset(ctx->stream);
            cudaError_t e = enqueue(ctx->stream, &ctx->launches, &ctx->rec);
            ctx->rec.finish();
            if (e != cudaSuccess) return cuda_fail(ctx, e, where);
            return HRC_OK;
        }
    }
    Recorder off;
    Recorder *rr = &off;
    if (timed) {   // fresh events from the pool for this graph's record nodes
        ctx->rec.ext = true;
        ctx->rec.coarse = ctx->timing_mode == 3;
        ctx->rec.open = false;
        ctx->rec.st = ctx->cap_stream;
        ctx->rec.recs.clear();
        rr = &ctx->rec;
    }
    int n = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    cudaError_t e1 = enqueue(ctx->cap_stream, &n, rr);
    rr->finish();
    cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
    ctx->rec.ext = false;
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(ctx, e1 != cudaSuccess ? e1 : e2, where);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    ++ctx->graph_captures;
    auto &slot = ctx->graphs[ctx->graph_next];
    ctx->graph_next = (ctx->graph_next + 1) % 8;
    if (slot.exec) cudaGraphExecDestroy(slot.exec);
    slot.exec = exec;
    slot.kind = kind;
    slot.prec = ctx->prec;
    slot.sched = ctx->sched;
    slot.mgroups = ctx->mgroups;
    slot.tune = ctx->mthreads * 8 + ctx->vmajor * 4 + ctx->mdown;
    slot.timed = timed ? ctx->timing_mode : 0;
    slot.recs = timed ? ctx->rec.recs : std::vector<Recorder::Rec>();
    std::memcpy(slot.p, key, sizeof(pk.p));
    slot.launches = n;
    slot.replays = 0;
    e = cudaGraphLaunch(exec, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    ctx->launches = n;
    return HRC_OK;
}

template <class ENQ>
hrc_status run_pass(hrc_ctx *ctx, int kind, const void *p0, const void *p1, const void *p2, const void *p3,
                    const void *p4, ENQ &&enqueue, const char *where) {
    const PassKey pk{{p0, p1, p2, p3, p4, nullptr, nullptr, nullptr}};
    return run_pass_key(ctx, kind, pk, enqueue, where);
}

void clear_graphs(hrc_ctx *ctx) {
    for (auto &g : ctx->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = hrc_ctx::GraphEntry();
    }
}

// Point the plans at the environment table (or at none).
void apply_env(hrc_ctx *ctx) {
    for (Plan *p : {&ctx->plan, &ctx->plan64}) {
        if (ctx->env_on) {
            const long long stride = env_table_stride(ctx->plan);
            p->envd = reinterpret_cast<const double *>(ctx->env_tab);
            p->envf = reinterpret_cast<const float *>(p->envd + 4 * stride);
            p->env_stride = stride;
        } else {
            p->envd = nullptr;
            p->envf = nullptr;
            p->env_stride = 0;
        }
    }
}

// One Lighting pass (Algorithm 1, then the Eq. 21 blur when enabled) and
// its adjoint, as enqueued by every single-scene entry point.
cudaError_t enqueue_lighting(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                             void *blur_buf, double thr, cudaStream_t st, int *n, Recorder *r, const Branches *br) {
    if (!blur_buf) return launch_forward(pl, rt, e, s, F, st, n, r, br);
    cudaError_t err = launch_forward(pl, rt, e, s, blur_buf, st, n, r, br);
    if (err != cudaSuccess) return err;
    return launch_cross_blur(pl, blur_buf, s, F, thr, st, n, r);
}

cudaError_t enqueue_lighting_adj(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                                 void *ge, void *gs, bool recompute, void *blur_buf, double thr, cudaStream_t st,
                                 int *n, Recorder *r) {
    if (!blur_buf) return launch_backward(pl, rt, e, s, gF, ge, gs, recompute, st, n, r);
    cudaError_t err = launch_cross_blur_adj(pl, gF, s, blur_buf, thr, st, n, r);
    if (err != cudaSuccess) return err;
    return launch_backward(pl, rt, e, s, blur_buf, ge, gs, recompute, st, n, r);
}

hrc_status check_ctx(hrc_ctx *ctx) {
    if (!ctx) return HRC_EINVAL;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pending CUDA error");
    return HRC_OK;
}

}  // namespace

namespace {
hrc_status build_batched_plans(hrc_ctx *ctx, int prec);
}

extern "C" {

const char *hrc_version(void) { return "hrc-gb300 0.1 (sm_103a)"; }

const char *hrc_last_error(const hrc_ctx *ctx) {
    static thread_local std::string copy;
    copy = ctx ? ctx->err : g_create_error;
    return copy.c_str();
}

int hrc_last_launch_count(const hrc_ctx *ctx) { return ctx ? ctx->launches : 0; }

hrc_status hrc_set_graphs(hrc_ctx *ctx, int enable) {
    if (!ctx) return HRC_EINVAL;
    if (enable != 0 && enable != 1) return fail(ctx, HRC_EINVAL, "hrc_set_graphs: 0 or 1");
    ctx->use_graphs = enable != 0;
    for (hrc_ctx *k : ctx->chan) hrc_set_graphs(k, enable);
    return HRC_OK;
}

long long hrc_graph_captures(const hrc_ctx *ctx) {
    if (!ctx) return -1;
    long long n = ctx->graph_captures;
    for (const hrc_ctx *k : ctx->chan) n += k->graph_captures;
    return n;
}

hrc_status hrc_set_timing(hrc_ctx *ctx, int enable) {
    if (!ctx) return HRC_EINVAL;
    if (enable < 0 || enable > 3) return fail(ctx, HRC_EINVAL, "hrc_set_timing: 0, 1, 2 or 3");
    ctx->rec.on = enable != 0;
    ctx->timing_mode = enable;
    for (hrc_ctx *k : ctx->chan) hrc_set_timing(k, enable);
    return HRC_OK;
}

int hrc_get_timing(hrc_ctx *ctx, hrc_kernel_time *out, int cap) {
    if (!ctx) return -1;
    if (ctx->per_channel) {   // the channels' records, channel after channel
        int n = 0;
        for (hrc_ctx *k : ctx->chan) {
            const int m = hrc_get_timing(k, out ? out + n : nullptr, cap - n);
            if (m < 0) return -1;
            n += m;
        }
        return n;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return -1;
    int n = 0;
    for (const auto &r : ctx->rec.recs) {
        if (n >= cap) break;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return -1;
        if (out) out[n] = hrc_kernel_time{r.kind, r.level, ms, r.bytes, r.launches};
        ++n;
    }
    return n;
}

hrc_status hrc_create(int W, int H, int channels, int cascades, hrc_ctx **out) {
    if (!out) return fail(nullptr, HRC_EINVAL, "hrc_create: out is NULL");
    *out = nullptr;
    if (W < 1 || H < 1 || W > 16384 || H > 16384)
        return fail(nullptr, HRC_EINVAL, "hrc_create: W and H must be in [1, 16384]");
    if (channels < 1 || channels > 4) return fail(nullptr, HRC_EINVAL, "hrc_create: channels must be in [1, 4]");
    hrc_ctx *ctx = new (std::nothrow) hrc_ctx();
    if (!ctx) return fail(nullptr, HRC_ENOMEM, "hrc_create: host allocation failed");
    ctx->W = W; ctx->H = H; ctx->C = channels; ctx->cascades = cascades;
    ctx->rt = make_ray_table();
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = prepare_device_once();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&ctx->br.s[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->br.fork, cudaEventDisableTiming);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ctx->br.join[i], cudaEventDisableTiming);
    if (e == cudaSuccess) ctx->br_ok = true;
    if (e != cudaSuccess) {
        for (int i = 0; i < 4; ++i) {
            if (ctx->br.s[i]) cudaStreamDestroy(ctx->br.s[i]);
            if (ctx->br.join[i]) cudaEventDestroy(ctx->br.join[i]);
        }
        if (ctx->br.fork) cudaEventDestroy(ctx->br.fork);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        delete ctx;
        return fail(nullptr, HRC_ECUDA, std::string("hrc_create: ") + cudaGetErrorString(e));
    }
    // The fp32 layout is the largest of the fp32 / fp16 / bf16 layouts.
    Plan p32;
    size_t bytes = build_plan(W, H, channels, cascades, P_FP32, 0, p32, true);
    ctx->arena_bytes = bytes;
    e = cudaMalloc(&ctx->arena, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return fail(nullptr, HRC_ENOMEM, "hrc_create: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    const size_t img = (size_t)W * H;
    e = cudaMalloc(&ctx->dev_e, img * channels * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dev_s, img * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->dev_F, img * channels * sizeof(float));
    if (e != cudaSuccess) {
        cudaGetLastError();
        hrc_destroy(ctx);
        return fail(nullptr, HRC_ENOMEM, "hrc_create: staging allocation failed");
    }
    ctx->pctl_bytes = persist_ctl_bytes(p32);
    e = cudaMalloc(&ctx->pctl, ctx->pctl_bytes);
    if (e == cudaSuccess) e = cudaMemset(ctx->pctl, 0, ctx->pctl_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->pctl = nullptr;
        hrc_destroy(ctx);
        return fail(nullptr, HRC_ENOMEM, "hrc_create: control block allocation failed");
    }
    p32.pctl = ctx->pctl;
    p32.pctl_bytes = (long long)ctx->pctl_bytes;
    p32.status = reinterpret_cast<int *>(ctx->pctl + 8);
    ctx->plan = p32;
    ctx->plan.arena = ctx->arena;
    ctx->plan.sched = ctx->sched;
    ctx->plan.mgroups = ctx->mgroups;
    ctx->plan.mthreads = ctx->mthreads;
    ctx->plan.vmajor = ctx->vmajor;
    ctx->plan.mdown = ctx->mdown;
    e = upload_arcs(ctx->plan, ctx->arena);
    if (e != cudaSuccess) { hrc_destroy(ctx); return fail(nullptr, HRC_ECUDA, "hrc_create: arc upload failed"); }
    *out = ctx;
    return HRC_OK;
}

hrc_status hrc_destroy(hrc_ctx *ctx) {
    if (!ctx) return HRC_EINVAL;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    cudaFree(ctx->arena);
    cudaFree(ctx->arena64);
    cudaFree(ctx->pctl);
    cudaFree(ctx->dev_e);
    cudaFree(ctx->dev_s);
    cudaFree(ctx->dev_F);
    cudaFree(ctx->blur_buf);
    cudaFree(ctx->bounce_buf);
    cudaFree(ctx->env_tab);
    cudaFree(ctx->env_map);
    cudaFree(ctx->top_map);
    cudaFree(ctx->chan_stage);
    for (hrc_ctx *k : ctx->chan) hrc_destroy(k);
    for (auto &g : ctx->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    cudaFree(ctx->d_plans);
    cudaFree(ctx->d_eoff);
    cudaFree(ctx->d_soff);
    for (int k = 0; k < hrc_ctx::kAux; ++k) {
        if (ctx->aux[k]) cudaStreamDestroy(ctx->aux[k]);
        if (ctx->ev_join[k]) cudaEventDestroy(ctx->ev_join[k]);
    }
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    for (int m = 0; m < 3; ++m) {
        for (auto &ml : ctx->multi[m]) cudaFree(ml.d_ents);
        cudaFree(ctx->d_blocks[m]);
        cudaFree(ctx->d_chunk[m]);
        for (auto &t : ctx->tiles[m]) {
            cudaFree(t.d_off);
            cudaFree(t.d_nx);
        }
    }
    cudaFree(ctx->d_counters);
    cudaFree(ctx->d_ticket);
    cudaFree(ctx->d_status);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (int i = 0; i < 4; ++i) {
        if (ctx->br.s[i]) cudaStreamDestroy(ctx->br.s[i]);
        if (ctx->br.join[i]) cudaEventDestroy(ctx->br.join[i]);
    }
    if (ctx->br.fork) cudaEventDestroy(ctx->br.fork);
    delete ctx;
    return HRC_OK;
}

hrc_status hrc_set_schedule(hrc_ctx *ctx, int schedule) {
    if (!ctx) return HRC_EINVAL;
    if (schedule < 0 || schedule > 2) return fail(ctx, HRC_EINVAL, "hrc_set_schedule: 0, 1 or 2");
    ctx->sched = schedule;
    ctx->plan.sched = schedule;
    ctx->plan64.sched = schedule;
    for (hrc_ctx *k : ctx->chan) hrc_set_schedule(k, schedule);
    return HRC_OK;
}

}  // extern "C"

namespace {
bool config_valid(const hrc_ctx *ctx, const hrc_launch_config &c) {
    return (c.schedule >= 0 && c.schedule <= 2) && (c.groups == 1 || c.groups == 2 || c.groups == 4) &&
           (c.threads == 64 || c.threads == 128 || c.threads == 256 || c.threads == 512) &&
           (c.vmajor == 0 || c.vmajor == 1) && (c.mdown >= 0 && c.mdown <= 2) &&
           !(c.mdown == 2 && c.schedule == 2) &&
           !(c.vmajor && 4LL * (ctx->W + ctx->H) > 65535);
}

void apply_config(hrc_ctx *ctx, const hrc_launch_config &c) {
    hrc_set_schedule(ctx, c.schedule);
    ctx->mgroups = ctx->plan.mgroups = ctx->plan64.mgroups = c.groups;
    ctx->mthreads = ctx->plan.mthreads = ctx->plan64.mthreads = c.threads;
    ctx->vmajor = ctx->plan.vmajor = ctx->plan64.vmajor = c.vmajor;
    ctx->mdown = ctx->plan.mdown = ctx->plan64.mdown = c.mdown;
}
}  // namespace

extern "C" {

hrc_status hrc_debug_bulk_wait(hrc_ctx *ctx, int extra_bytes, long long limit_ns) {
    if (!ctx || ctx->batched || extra_bytes < 0 || extra_bytes > 4096) return HRC_EINVAL;
    const long long lim = limit_ns > 0 ? limit_ns : 2000000000LL;
    ctx->plan.bulk_extra_tx = ctx->plan64.bulk_extra_tx = extra_bytes;
    ctx->plan.bulk_limit_ns = ctx->plan64.bulk_limit_ns = lim;
    clear_graphs(ctx);   // the graphs hold the plan by value
    ctx->have_fwd = false;
    return HRC_OK;
}

hrc_status hrc_sync(hrc_ctx *ctx) {
    if (!ctx) return HRC_EINVAL;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    int status = 0;
    if (e == cudaSuccess) e = read_plan_status(ctx->plan, &status);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_sync");
    for (hrc_ctx *k : ctx->chan) {   // per-channel contexts keep status words of their own
        const hrc_status st = hrc_sync(k);
        if (st != HRC_OK) return fail(ctx, st, k->err);
    }
    if (status == kWaitLost)
        return fail(ctx, HRC_ETIMEOUT, "a copy wait gave up and its copies did not land within the drain bound: "
                                       "results of later launches on this device are suspect");
    if (status != 0) return fail(ctx, HRC_ETIMEOUT, "a bounded copy or dependency wait gave up (its launch ended early)");
    return HRC_OK;
}

hrc_status hrc_set_backward_recompute(hrc_ctx *ctx, int on) {
    if (!ctx) return HRC_EINVAL;
    if (on != 0 && on != 1) return fail(ctx, HRC_EINVAL, "hrc_set_backward_recompute: 0 or 1");
    ctx->bwd_recompute = on != 0;
    for (hrc_ctx *k : ctx->chan) hrc_set_backward_recompute(k, on);
    return HRC_OK;
}

hrc_status hrc_set_cross_blur(hrc_ctx *ctx, int enable, float threshold) {
    if (!ctx) return HRC_EINVAL;
    if (ctx->batched) return fail(ctx, HRC_EINVAL, "hrc_set_cross_blur: single-scene contexts only");
    if ((enable != 0 && enable != 1) || !(threshold >= 0.f && threshold <= 1.f))
        return fail(ctx, HRC_EINVAL, "hrc_set_cross_blur: enable 0 or 1, threshold in [0, 1]");
    if (enable && !ctx->blur_buf) {
        const size_t bytes = (size_t)ctx->W * ctx->H * ctx->C * sizeof(double);
        cudaError_t e = cudaMalloc(&ctx->blur_buf, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->blur_buf = nullptr;
            return fail(ctx, HRC_ENOMEM, "hrc_set_cross_blur: buffer of " + std::to_string(bytes) + " bytes does not fit");
        }
    }
    ctx->blur = enable != 0;
    ctx->blur_thr = threshold;
    clear_graphs(ctx);   // the graphs hold the pass as it was captured
    for (hrc_ctx *k : ctx->chan) {
        hrc_status st = hrc_set_cross_blur(k, enable, threshold);
        if (st != HRC_OK) return fail(ctx, st, k->err);
    }
    return HRC_OK;
}

hrc_status hrc_get_cross_blur(const hrc_ctx *ctx, int *enable, float *threshold) {
    if (!ctx || !enable || !threshold) return HRC_EINVAL;
    *enable = ctx->blur ? 1 : 0;
    *threshold = ctx->blur_thr;
    return HRC_OK;
}

hrc_status hrc_get_launch_config(const hrc_ctx *ctx, hrc_launch_config *cfg) {
    if (!ctx || !cfg) return HRC_EINVAL;
    cfg->schedule = ctx->sched;
    cfg->groups = ctx->mgroups;
    cfg->threads = ctx->mthreads;
    cfg->vmajor = ctx->vmajor;
    cfg->mdown = ctx->mdown;
    return HRC_OK;
}

hrc_status hrc_set_launch_config(hrc_ctx *ctx, const hrc_launch_config *cfg) {
    if (!ctx || !cfg) return HRC_EINVAL;
    if (ctx->batched) return fail(ctx, HRC_EINVAL, "hrc_set_launch_config: single-scene contexts only");
    if (!config_valid(ctx, *cfg)) return fail(ctx, HRC_EINVAL, "hrc_set_launch_config: value out of range");
    apply_config(ctx, *cfg);
    ctx->have_fwd = false;
    for (hrc_ctx *k : ctx->chan) hrc_set_launch_config(k, cfg);
    return HRC_OK;
}

hrc_status hrc_autotune(hrc_ctx *ctx, float *best_ms) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->per_channel) {   // tune one channel's context, apply its pick to all
        st = hrc_autotune(ctx->chan[0], best_ms);
        if (st != HRC_OK) return fail(ctx, st, ctx->chan[0]->err);
        hrc_launch_config c;
        hrc_get_launch_config(ctx->chan[0], &c);
        return hrc_set_launch_config(ctx, &c);
    }
    if (ctx->batched || ctx->prec == P_FP64) return fail(ctx, HRC_EINVAL, "hrc_autotune: single-scene fp32/fp16/bf16 contexts");
    // the timing does not depend on the data: time on the context's own buffers
    const size_t img = (size_t)ctx->W * ctx->H;
    cudaError_t e = cudaMemsetAsync(ctx->dev_e, 0, img * ctx->C * sizeof(float), ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->dev_s, 0, img * sizeof(float), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_autotune");
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    hrc_launch_config best_c;
    hrc_get_launch_config(ctx, &best_c);
    const bool timing = ctx->rec.on;
    ctx->rec.on = false;
    static const int kThreads[4] = {64, 128, 256, 512};
    static const int kGroups[3] = {1, 2, 4};
    for (int cand = 0; cand < 3 * 3 * 4 * 2 * 3 && st == HRC_OK; ++cand) {
        const hrc_launch_config c{cand % 3, kGroups[(cand / 3) % 3], kThreads[(cand / 9) & 3], (cand / 36) & 1,
                                  (cand / 72) % 3};
        if (c.mdown == 2 && !persist_down_usable(ctx->plan)) continue;
        if (!config_valid(ctx, c)) continue;
        apply_config(ctx, c);
        for (int r = 0; r < 2 && st == HRC_OK; ++r) st = hrc_fluence(ctx, ctx->dev_e, ctx->dev_s, ctx->dev_F);
        cudaEventRecord(a, ctx->stream);
        for (int r = 0; r < 5 && st == HRC_OK; ++r) st = hrc_fluence(ctx, ctx->dev_e, ctx->dev_s, ctx->dev_F);
        cudaEventRecord(b, ctx->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        ms /= 5.f;
        if (ms < best) { best = ms; best_c = c; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->rec.on = timing;
    apply_config(ctx, best_c);
    ctx->have_fwd = false;
    if (st != HRC_OK) return st;
    if (best_ms) *best_ms = best;
    return HRC_OK;
}

hrc_status hrc_set_stream(hrc_ctx *ctx, void *stream) {
    if (!ctx) return HRC_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    for (hrc_ctx *k : ctx->chan) hrc_set_stream(k, stream);
    return HRC_OK;
}

hrc_status hrc_set_precision(hrc_ctx *ctx, hrc_precision prec) {
    if (!ctx) return HRC_EINVAL;
    if (prec < HRC_FP32 || prec > HRC_FP64_TEST) return fail(ctx, HRC_EINVAL, "hrc_set_precision: unknown precision");
    clear_graphs(ctx);
    if (ctx->batched) {
        if (prec == HRC_FP64_TEST) return fail(ctx, HRC_EINVAL, "hrc_set_precision: fp64 is not available on batched contexts");
        size_t bytes = 0;
        for (int i = 0; i < ctx->nscenes; ++i) {
            Plan p;
            bytes = build_plan(ctx->Ws[i], ctx->Hs[i], ctx->C, ctx->cascades, (int)prec, bytes, p, true);
        }
        if (bytes > ctx->arena_bytes) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->arena);
            ctx->arena = nullptr;
            ctx->arena_bytes = 0;
            cudaError_t e = cudaMalloc(&ctx->arena, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->arena = nullptr;
                return fail(ctx, HRC_ENOMEM, "hrc_set_precision: batched buffers do not fit");
            }
            ctx->arena_bytes = bytes;
        }
        ctx->prec = (int)prec;
        ctx->have_fwd = false;
        return build_batched_plans(ctx, (int)prec);
    }
    if (prec == HRC_FP64_TEST) {
        if (!ctx->arena64) {
            Plan p64;
            size_t bytes = build_plan(ctx->W, ctx->H, ctx->C, ctx->cascades, P_FP64, 0, p64, true);
            cudaError_t e = cudaMalloc(&ctx->arena64, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->arena64 = nullptr;
                return fail(ctx, HRC_ENOMEM, "hrc_set_precision: fp64 buffers do not fit");
            }
            ctx->arena64_bytes = bytes;
            p64.arena = ctx->arena64;
            p64.sched = ctx->sched;
            p64.mgroups = ctx->mgroups;
            p64.mthreads = ctx->mthreads;
            p64.vmajor = ctx->vmajor;
            p64.mdown = ctx->mdown;
            p64.status = reinterpret_cast<int *>(ctx->pctl + 8);
            ctx->plan64 = p64;
            e = upload_arcs(ctx->plan64, ctx->arena64);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_set_precision");
        }
    } else {
        Plan p;
        build_plan(ctx->W, ctx->H, ctx->C, ctx->cascades, (int)prec, 0, p, true);
        p.arena = ctx->arena;
        p.sched = ctx->sched;
        p.mgroups = ctx->mgroups;
        p.mthreads = ctx->mthreads;
        p.vmajor = ctx->vmajor;
        p.mdown = ctx->mdown;
        p.pctl = ctx->pctl;
        p.pctl_bytes = (long long)ctx->pctl_bytes;
        p.status = reinterpret_cast<int *>(ctx->pctl + 8);
        ctx->plan = p;
        cudaError_t e = upload_arcs(ctx->plan, ctx->arena);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_set_precision");
    }
    ctx->prec = (int)prec;
    ctx->have_fwd = false;
    ctx->have_bounce = false;
    apply_env(ctx);
    for (hrc_ctx *k : ctx->chan) {
        hrc_status st = hrc_set_precision(k, prec);
        if (st != HRC_OK) return fail(ctx, st, k->err);
    }
    return HRC_OK;
}

}  // extern "C"

namespace {

// Channel c's plane of a [C][H][W] argument: p + c W H elements, read
// directly when 16-byte aligned, else copied into aligned staging buffer
// `slot` of that channel first (inputs) or written there and copied out
// afterwards (outputs).
struct ChanArgs {
    hrc_ctx *ctx;
    size_t esz, plane;
    cudaError_t err = cudaSuccess;
    char *stage(int c, int slot) const {
        return ctx->chan_stage + ((size_t)c * hrc_ctx::kStagePlanes + slot) * ctx->chan_plane;
    }
    const void *in(int c, int slot, const void *p) {
        const char *q = static_cast<const char *>(p) + (size_t)c * plane;
        if (aligned16(q)) return q;
        if (err == cudaSuccess) err = cudaMemcpyAsync(stage(c, slot), q, plane, cudaMemcpyDeviceToDevice, ctx->stream);
        return stage(c, slot);
    }
    void *out(int c, int slot, void *p) const {
        char *q = static_cast<char *>(p) + (size_t)c * plane;
        return aligned16(q) ? static_cast<void *>(q) : static_cast<void *>(stage(c, slot));
    }
    void done(int c, int slot, void *p) {
        char *q = static_cast<char *>(p) + (size_t)c * plane;
        if (!aligned16(q) && err == cudaSuccess)
            err = cudaMemcpyAsync(q, stage(c, slot), plane, cudaMemcpyDeviceToDevice, ctx->stream);
    }
};

ChanArgs chan_args(hrc_ctx *ctx, bool f64) {
    ChanArgs a{ctx, f64 ? sizeof(double) : sizeof(float), 0};
    a.plane = (size_t)ctx->W * ctx->H * a.esz;
    return a;
}

// Sum of the channels' launch counts into the parent's.
void chan_launches(hrc_ctx *ctx) {
    int n = 0;
    for (hrc_ctx *k : ctx->chan) n += k->launches;
    ctx->launches = n;
}

hrc_status chan_status(hrc_ctx *ctx, hrc_status st, hrc_ctx *k) { return st == HRC_OK ? st : fail(ctx, st, k->err); }

hrc_status chan_forward(hrc_ctx *ctx, const void *e, const void *s, void *F, bool f64) {
    if (!e || !s || !F) return fail(ctx, HRC_EINVAL, "hrc_fluence: NULL pointer");
    ChanArgs a = chan_args(ctx, f64);
    for (int c = 0; c < ctx->C; ++c) {
        hrc_ctx *k = ctx->chan[c];
        const void *ec = a.in(c, 0, e), *sc = a.in(c, 1, s);
        void *Fc = a.out(c, 3, F);
        if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence (per-channel staging)");
        hrc_status st = f64 ? hrc_fluence_f64(k, (const double *)ec, (const double *)sc, (double *)Fc)
                            : hrc_fluence(k, (const float *)ec, (const float *)sc, (float *)Fc);
        if (st != HRC_OK) return chan_status(ctx, st, k);
        a.done(c, 3, F);
    }
    if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence (per-channel staging)");
    chan_launches(ctx);
    ctx->have_fwd = true;
    return HRC_OK;
}

hrc_status chan_backward(hrc_ctx *ctx, const void *gF, void *ge, void *gs, bool f64) {
    if (!gF || !ge || !gs) return fail(ctx, HRC_EINVAL, "hrc_fluence_backward: NULL pointer");
    ChanArgs a = chan_args(ctx, f64);
    for (int c = 0; c < ctx->C; ++c) {
        hrc_ctx *k = ctx->chan[c];
        const void *gc = a.in(c, 3, gF);
        void *ec = a.out(c, 4, ge), *sc = a.out(c, 5, gs);
        if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence_backward (per-channel staging)");
        hrc_status st = f64 ? hrc_fluence_backward_f64(k, (const double *)gc, (double *)ec, (double *)sc)
                            : hrc_fluence_backward(k, (const float *)gc, (float *)ec, (float *)sc);
        if (st != HRC_OK) return chan_status(ctx, st, k);
        a.done(c, 4, ge);
        a.done(c, 5, gs);
    }
    if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence_backward (per-channel staging)");
    chan_launches(ctx);
    return HRC_OK;
}

hrc_status chan_bounces(hrc_ctx *ctx, const void *e, const void *s, const void *al, int K, void *F, bool f64) {
    if (!e || !s || !al || !F) return fail(ctx, HRC_EINVAL, "hrc_fluence_bounces: NULL pointer");
    ChanArgs a = chan_args(ctx, f64);
    for (int c = 0; c < ctx->C; ++c) {
        hrc_ctx *k = ctx->chan[c];
        const void *ec = a.in(c, 0, e), *sc = a.in(c, 1, s), *ac = a.in(c, 2, al);
        void *Fc = a.out(c, 3, F);
        if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence_bounces (per-channel staging)");
        hrc_status st =
            f64 ? hrc_fluence_bounces_f64(k, (const double *)ec, (const double *)sc, (const double *)ac, K, (double *)Fc)
                : hrc_fluence_bounces(k, (const float *)ec, (const float *)sc, (const float *)ac, K, (float *)Fc);
        if (st != HRC_OK) return chan_status(ctx, st, k);
        a.done(c, 3, F);
    }
    if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence_bounces (per-channel staging)");
    chan_launches(ctx);
    ctx->have_bounce = true;
    return HRC_OK;
}

hrc_status chan_bounces_backward(hrc_ctx *ctx, const void *gF, void *ge, void *gs, void *ga, bool f64) {
    if (!gF || !ge || !gs || !ga) return fail(ctx, HRC_EINVAL, "hrc_fluence_bounces_backward: NULL pointer");
    ChanArgs a = chan_args(ctx, f64);
    for (int c = 0; c < ctx->C; ++c) {
        hrc_ctx *k = ctx->chan[c];
        const void *gc = a.in(c, 3, gF);
        void *ec = a.out(c, 4, ge), *sc = a.out(c, 5, gs), *ac = a.out(c, 6, ga);
        if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence_bounces_backward (per-channel staging)");
        hrc_status st = f64 ? hrc_fluence_bounces_backward_f64(k, (const double *)gc, (double *)ec, (double *)sc, (double *)ac)
                            : hrc_fluence_bounces_backward(k, (const float *)gc, (float *)ec, (float *)sc, (float *)ac);
        if (st != HRC_OK) return chan_status(ctx, st, k);
        a.done(c, 4, ge);
        a.done(c, 5, gs);
        a.done(c, 6, ga);
    }
    if (a.err != cudaSuccess) return cuda_fail(ctx, a.err, "hrc_fluence_bounces_backward (per-channel staging)");
    chan_launches(ctx);
    return HRC_OK;
}

}  // namespace

extern "C" {

hrc_status hrc_set_channel_extinction(hrc_ctx *ctx, int per_channel) {
    if (!ctx) return HRC_EINVAL;
    if (ctx->batched) return fail(ctx, HRC_EINVAL, "hrc_set_channel_extinction: single-scene contexts only");
    if (per_channel != 0 && per_channel != 1) return fail(ctx, HRC_EINVAL, "hrc_set_channel_extinction: 0 or 1");
    if (per_channel && ctx->chan.empty()) {
        const size_t img = (size_t)ctx->W * ctx->H;
        if (img % 4 != 0) {   // some channel planes are not 16-byte aligned: staging buffers
            ctx->chan_plane = align_up(img * sizeof(double), 256);
            cudaError_t e = cudaMalloc(&ctx->chan_stage, ctx->chan_plane * hrc_ctx::kStagePlanes * ctx->C);
            if (e != cudaSuccess) {
                cudaGetLastError();
                ctx->chan_stage = nullptr;
                return fail(ctx, HRC_ENOMEM, "hrc_set_channel_extinction: staging buffers do not fit");
            }
        }
        hrc_launch_config cfg;
        hrc_get_launch_config(ctx, &cfg);
        for (int c = 0; c < ctx->C; ++c) {
            hrc_ctx *k = nullptr;
            hrc_status st = hrc_create(ctx->W, ctx->H, 1, ctx->cascades, &k);
            if (st == HRC_OK) ctx->chan.push_back(k);
            if (st == HRC_OK) st = hrc_set_stream(k, ctx->stream);
            if (st == HRC_OK) st = hrc_set_precision(k, (hrc_precision)ctx->prec);
            if (st == HRC_OK) st = hrc_set_launch_config(k, &cfg);
            if (st == HRC_OK) st = hrc_set_backward_recompute(k, ctx->bwd_recompute ? 1 : 0);
            if (st == HRC_OK && ctx->blur_buf) st = hrc_set_cross_blur(k, ctx->blur ? 1 : 0, ctx->blur_thr);
            if (st == HRC_OK && ctx->bounce_buf) st = hrc_reserve_bounces(k, ctx->bounce_cap);
            if (st == HRC_OK) st = hrc_set_timing(k, ctx->timing_mode);
            if (st == HRC_OK && ctx->env_on && ctx->env_top)
                st = hrc_set_top_radiance(k, ctx->top_map + (size_t)c * 4 * ctx->top_K, ctx->top_K);
            else if (st == HRC_OK && ctx->env_on)
                st = hrc_set_environment(k, ctx->env_map + (size_t)c * ctx->env_pitch, ctx->env_M);
            if (st != HRC_OK) {
                std::string msg = k ? k->err : g_create_error;
                for (hrc_ctx *x : ctx->chan) hrc_destroy(x);
                ctx->chan.clear();
                cudaFree(ctx->chan_stage);
                ctx->chan_stage = nullptr;
                return fail(ctx, st, "hrc_set_channel_extinction: " + msg);
            }
        }
    }
    ctx->per_channel = per_channel != 0;
    ctx->have_fwd = false;
    ctx->have_bounce = false;
    return HRC_OK;
}

hrc_status hrc_set_environment(hrc_ctx *ctx, const float *env, int M) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->batched) return fail(ctx, HRC_EINVAL, "hrc_set_environment: single-scene contexts only");
    if (env && (M < 1 || M > (1 << 20)))
        return fail(ctx, HRC_EINVAL, "hrc_set_environment: M must be in [1, 2^20]");
    if (env && !aligned16(env)) return fail(ctx, HRC_EINVAL, "hrc_set_environment: env must be 16-byte aligned");
    if (env && !ctx->env_tab) {
        const size_t bytes = env_table_bytes(ctx->plan);
        cudaError_t e = cudaMalloc(&ctx->env_tab, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->env_tab = nullptr;
            return fail(ctx, HRC_ENOMEM, "hrc_set_environment: table does not fit");
        }
    }
    if (env) {
        cudaError_t e = launch_env_table(ctx->plan, env, M, ctx->env_tab, ctx->stream);
        const int pitch = (M + 3) / 4 * 4;   // a row per channel, 16-byte aligned
        if (e == cudaSuccess && pitch * ctx->C > ctx->env_pitch * ctx->C) {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->env_map);
            ctx->env_map = nullptr;
            ctx->env_pitch = 0;
            e = cudaMalloc(&ctx->env_map, sizeof(float) * pitch * ctx->C);
        }
        if (e == cudaSuccess) {
            ctx->env_pitch = ctx->env_pitch > pitch ? ctx->env_pitch : pitch;
            ctx->env_M = M;
            e = cudaMemcpy2DAsync(ctx->env_map, sizeof(float) * ctx->env_pitch, env, sizeof(float) * M,
                                  sizeof(float) * M, ctx->C, cudaMemcpyDeviceToDevice, ctx->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_set_environment");
    }
    for (int c = 0; c < (int)ctx->chan.size(); ++c) {   // channel c sees row c
        hrc_status st2 = hrc_set_environment(ctx->chan[c], env ? ctx->env_map + (size_t)c * ctx->env_pitch : nullptr, M);
        if (st2 != HRC_OK) return fail(ctx, st2, ctx->chan[c]->err);
    }
    ctx->env_on = env != nullptr;
    ctx->env_top = false;
    apply_env(ctx);
    clear_graphs(ctx);     // the graphs hold the plans by value
    ctx->have_fwd = false; // levels and fluence of an earlier forward saw the old map
    ctx->have_bounce = false;
    return HRC_OK;
}

hrc_status hrc_set_top_radiance(hrc_ctx *ctx, const float *top, int K) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->batched) return fail(ctx, HRC_EINVAL, "hrc_set_top_radiance: single-scene contexts only");
    if (!top) return hrc_set_environment(ctx, nullptr, 0);
    const int need = 1 << plan_nmax(ctx->plan);
    if (K < need || K > (1 << 20))
        return fail(ctx, HRC_EINVAL, "hrc_set_top_radiance: K must be in [2^N, 2^20] with N = " +
                                         std::to_string(plan_nmax(ctx->plan)));
    if (!ctx->env_tab) {
        const size_t bytes = env_table_bytes(ctx->plan);
        cudaError_t e = cudaMalloc(&ctx->env_tab, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->env_tab = nullptr;
            return fail(ctx, HRC_ENOMEM, "hrc_set_top_radiance: table does not fit");
        }
    }
    cudaError_t e = launch_env_top(ctx->plan, top, K, ctx->env_tab, ctx->stream);
    // keep a channel-major copy [C][4 K] for the per-channel contexts
    const size_t cap = (size_t)ctx->C * 4 * K;
    if (e == cudaSuccess && cap > ctx->top_cap) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(ctx->top_map);
        ctx->top_map = nullptr;
        ctx->top_cap = 0;
        e = cudaMalloc(&ctx->top_map, sizeof(float) * cap);
        if (e == cudaSuccess) ctx->top_cap = cap;
    }
    for (int c = 0; c < ctx->C && e == cudaSuccess; ++c)
        e = cudaMemcpy2DAsync(ctx->top_map + (size_t)c * 4 * K, sizeof(float), top + c, sizeof(float) * ctx->C,
                              sizeof(float), (size_t)4 * K, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_set_top_radiance");
    ctx->top_K = K;
    for (int c = 0; c < (int)ctx->chan.size(); ++c) {   // channel c sees its own table
        hrc_status st2 = hrc_set_top_radiance(ctx->chan[c], ctx->top_map + (size_t)c * 4 * K, K);
        if (st2 != HRC_OK) return fail(ctx, st2, ctx->chan[c]->err);
    }
    ctx->env_on = true;
    ctx->env_top = true;
    apply_env(ctx);
    clear_graphs(ctx);     // the graphs hold the plans by value
    ctx->have_fwd = false;
    ctx->have_bounce = false;
    return HRC_OK;
}

hrc_status hrc_fluence(hrc_ctx *ctx, const float *emission, const float *sigma_t, float *out) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->per_channel && ctx->prec != P_FP64) return chan_forward(ctx, emission, sigma_t, out, false);
    if (ctx->prec == P_FP64) return fail(ctx, HRC_ESTATE, "hrc_fluence: context is in HRC_FP64_TEST; use hrc_fluence_f64");
    if (ctx->batched) return fail(ctx, HRC_ESTATE, "hrc_fluence: batched context; use hrc_fluence_batched");
    if (!emission || !sigma_t || !out) return fail(ctx, HRC_EINVAL, "hrc_fluence: NULL pointer");
    if (!aligned16(emission) || !aligned16(sigma_t) || !aligned16(out))
        return fail(ctx, HRC_EINVAL, "hrc_fluence: pointers must be 16-byte aligned");
    const Plan pl = ctx->plan;
    const RayTable *rt = &ctx->rt;
    void *Fr = ctx->blur ? ctx->blur_buf : nullptr;
    const double thr = ctx->blur_thr;
    const Branches *br = ctx->br_ok ? &ctx->br : nullptr;
    st = run_pass(ctx, 0, emission, sigma_t, out, nullptr, nullptr,
                  [&](cudaStream_t s, int *n, Recorder *r) {
                      return enqueue_lighting(pl, *rt, emission, sigma_t, out, Fr, thr, s, n, r, br);
                  },
                  "hrc_fluence");
    if (st != HRC_OK) return st;
    ctx->last_e = emission;
    ctx->last_s = sigma_t;
    ctx->have_fwd = true;
    ctx->have_bounce = false;
    return HRC_OK;
}

hrc_status hrc_fluence_host(hrc_ctx *ctx, const float *emission, const float *sigma_t, float *out) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->per_channel) {   // channel c: its planes of the host arrays through its own staging
        if (!emission || !sigma_t || !out) return fail(ctx, HRC_EINVAL, "hrc_fluence_host: NULL pointer");
        const size_t img = (size_t)ctx->W * ctx->H;
        for (int c = 0; c < ctx->C; ++c) {
            st = hrc_fluence_host(ctx->chan[c], emission + c * img, sigma_t + c * img, out + c * img);
            if (st != HRC_OK) return chan_status(ctx, st, ctx->chan[c]);
        }
        chan_launches(ctx);
        ctx->have_fwd = true;
        return HRC_OK;
    }
    if (!emission || !sigma_t || !out) return fail(ctx, HRC_EINVAL, "hrc_fluence_host: NULL pointer");
    const size_t img = (size_t)ctx->W * ctx->H;
    cudaError_t e = cudaMemcpyAsync(ctx->dev_e, emission, img * ctx->C * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->dev_s, sigma_t, img * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_fluence_host: upload");
    st = hrc_fluence(ctx, ctx->dev_e, ctx->dev_s, ctx->dev_F);
    if (st != HRC_OK) return st;
    e = cudaMemcpyAsync(out, ctx->dev_F, img * ctx->C * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_fluence_host: download");
    return HRC_OK;
}

hrc_status hrc_fluence_f64(hrc_ctx *ctx, const double *emission, const double *sigma_t, double *out) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->per_channel && ctx->prec == P_FP64) return chan_forward(ctx, emission, sigma_t, out, true);
    if (ctx->prec != P_FP64) return fail(ctx, HRC_ESTATE, "hrc_fluence_f64: set HRC_FP64_TEST first");
    if (!emission || !sigma_t || !out) return fail(ctx, HRC_EINVAL, "hrc_fluence_f64: NULL pointer");
    if (!aligned16(emission) || !aligned16(sigma_t) || !aligned16(out))
        return fail(ctx, HRC_EINVAL, "hrc_fluence_f64: pointers must be 16-byte aligned");
    const Plan pl = ctx->plan64;
    const RayTable *rt = &ctx->rt;
    void *Fr = ctx->blur ? ctx->blur_buf : nullptr;
    const double thr = ctx->blur_thr;
    const Branches *br = ctx->br_ok ? &ctx->br : nullptr;
    st = run_pass(ctx, 2, emission, sigma_t, out, nullptr, nullptr,
                  [&](cudaStream_t s, int *n, Recorder *r) {
                      return enqueue_lighting(pl, *rt, emission, sigma_t, out, Fr, thr, s, n, r, br);
                  },
                  "hrc_fluence_f64");
    if (st != HRC_OK) return st;
    ctx->last_e = emission;
    ctx->last_s = sigma_t;
    ctx->have_fwd = true;
    ctx->have_bounce = false;
    return HRC_OK;
}

hrc_status hrc_fluence_backward(hrc_ctx *ctx, const float *grad_F, float *grad_emission, float *grad_sigma_t) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->per_channel && ctx->prec != P_FP64) return chan_backward(ctx, grad_F, grad_emission, grad_sigma_t, false);
    if (ctx->prec == P_FP64) return fail(ctx, HRC_ESTATE, "hrc_fluence_backward: context is in HRC_FP64_TEST");
    if (!ctx->have_fwd) return fail(ctx, HRC_ESTATE, "hrc_fluence_backward: no forward pass on this context");
    if (!grad_F || !grad_emission || !grad_sigma_t) return fail(ctx, HRC_EINVAL, "hrc_fluence_backward: NULL pointer");
    if (!aligned16(grad_F) || !aligned16(grad_emission) || !aligned16(grad_sigma_t))
        return fail(ctx, HRC_EINVAL, "hrc_fluence_backward: pointers must be 16-byte aligned");
    const Plan pl = ctx->plan;
    const RayTable *rt = &ctx->rt;
    const void *le = ctx->last_e, *ls = ctx->last_s;
    const bool rc = ctx->bwd_recompute;
    void *gFr = ctx->blur ? ctx->blur_buf : nullptr;
    const double thr = ctx->blur_thr;
    return run_pass(ctx, rc ? 4 : 1, le, ls, grad_F, grad_emission, grad_sigma_t,
                    [&](cudaStream_t s, int *n, Recorder *r) {
                        return enqueue_lighting_adj(pl, *rt, le, ls, grad_F, grad_emission, grad_sigma_t, rc, gFr,
                                                    thr, s, n, r);
                    },
                    "hrc_fluence_backward");
}

hrc_status hrc_fluence_backward_f64(hrc_ctx *ctx, const double *grad_F, double *grad_emission, double *grad_sigma_t) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->per_channel && ctx->prec == P_FP64) return chan_backward(ctx, grad_F, grad_emission, grad_sigma_t, true);
    if (ctx->prec != P_FP64) return fail(ctx, HRC_ESTATE, "hrc_fluence_backward_f64: set HRC_FP64_TEST first");
    if (!ctx->have_fwd) return fail(ctx, HRC_ESTATE, "hrc_fluence_backward_f64: no forward pass on this context");
    if (!grad_F || !grad_emission || !grad_sigma_t) return fail(ctx, HRC_EINVAL, "hrc_fluence_backward_f64: NULL pointer");
    if (!aligned16(grad_F) || !aligned16(grad_emission) || !aligned16(grad_sigma_t))
        return fail(ctx, HRC_EINVAL, "hrc_fluence_backward_f64: pointers must be 16-byte aligned");
    const Plan pl = ctx->plan64;
    const RayTable *rt = &ctx->rt;
    const void *le = ctx->last_e, *ls = ctx->last_s;
    const bool rc = ctx->bwd_recompute;
    void *gFr = ctx->blur ? ctx->blur_buf : nullptr;
    const double thr = ctx->blur_thr;
    return run_pass(ctx, rc ? 5 : 3, le, ls, grad_F, grad_emission, grad_sigma_t,
                    [&](cudaStream_t s, int *n, Recorder *r) {
                        return enqueue_lighting_adj(pl, *rt, le, ls, grad_F, grad_emission, grad_sigma_t, rc, gFr,
                                                    thr, s, n, r);
                    },
                    "hrc_fluence_backward_f64");
}


// ---------------------------------------------------------------------------
// Multiple bounces
// ---------------------------------------------------------------------------
hrc_status hrc_reserve_bounces(hrc_ctx *ctx, int max_bounces) {
    if (!ctx) return HRC_EINVAL;
    if (ctx->batched) return fail(ctx, HRC_EINVAL, "hrc_reserve_bounces: single-scene contexts only");
    if (max_bounces < 0 || max_bounces > 64) return fail(ctx, HRC_EINVAL, "hrc_reserve_bounces: 0 .. 64 bounces");
    if (ctx->bounce_buf && max_bounces <= ctx->bounce_cap) return HRC_OK;
    const size_t img = (size_t)ctx->W * ctx->H;
    const size_t plane = align_up(img * ctx->C * sizeof(double), 256);
    const size_t bytes = (2 * (size_t)max_bounces + 2) * plane + img * sizeof(double);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    clear_graphs(ctx);   // graphs may hold the old buffers
    cudaFree(ctx->bounce_buf);
    cudaFree(ctx->env_tab);
    ctx->bounce_buf = nullptr;
    ctx->bounce_cap = 0;
    ctx->have_bounce = false;
    cudaError_t e = cudaMalloc(&ctx->bounce_buf, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->bounce_buf = nullptr;
        return fail(ctx, HRC_ENOMEM, "hrc_reserve_bounces: " + std::to_string(bytes) + " bytes do not fit");
    }
    ctx->bounce_cap = max_bounces;
    ctx->bounce_plane = plane;
    for (hrc_ctx *k : ctx->chan) {
        hrc_status st = hrc_reserve_bounces(k, max_bounces);
        if (st != HRC_OK) return fail(ctx, st, k->err);
    }
    return HRC_OK;
}

}  // extern "C"

namespace {

// Buffers of the bounce arena: e_k (k = 1 .. cap), F_k (k = 0 .. cap - 1),
// then the backward's dL/de_k, dL/dF_{k-1} (both [C][H][W]) and dL/dsigma_k.
char *bounce_e(hrc_ctx *ctx, int k) { return ctx->bounce_buf + (size_t)(k - 1) * ctx->bounce_plane; }
char *bounce_F(hrc_ctx *ctx, int k) { return ctx->bounce_buf + (size_t)(ctx->bounce_cap + k) * ctx->bounce_plane; }
char *bounce_scratch(hrc_ctx *ctx, int j) {
    return ctx->bounce_buf + (size_t)(2 * ctx->bounce_cap + j) * ctx->bounce_plane;
}

hrc_status bounces_forward(hrc_ctx *ctx, const void *e, const void *s, const void *a, int K, void *out, bool f64,
                           const char *where) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->batched) return fail(ctx, HRC_ESTATE, std::string(where) + ": batched context");
    if (f64 != (ctx->prec == P_FP64))
        return fail(ctx, HRC_ESTATE, std::string(where) + (f64 ? ": set HRC_FP64_TEST first" : ": context is in HRC_FP64_TEST"));
    if (!e || !s || !a || !out) return fail(ctx, HRC_EINVAL, std::string(where) + ": NULL pointer");
    if (!aligned16(e) || !aligned16(s) || !aligned16(a) || !aligned16(out))
        return fail(ctx, HRC_EINVAL, std::string(where) + ": pointers must be 16-byte aligned");
    if (!ctx->bounce_buf) return fail(ctx, HRC_ESTATE, std::string(where) + ": call hrc_reserve_bounces first");
    if (K < 0 || K > ctx->bounce_cap)
        return fail(ctx, HRC_EINVAL, std::string(where) + ": bounces must be in [0, the count reserved by hrc_reserve_bounces]");
    const Plan pl = f64 ? ctx->plan64 : ctx->plan;
    const RayTable *rt = &ctx->rt;
    void *blur = ctx->blur ? ctx->blur_buf : nullptr;
    const double thr = ctx->blur_thr;
    const Branches *br = ctx->br_ok ? &ctx->br : nullptr;
    const PassKey key{{e, s, a, out, (const void *)(intptr_t)K, nullptr, nullptr, nullptr}};
    st = run_pass_key(ctx, f64 ? 13 : 12, key,
                      [&](cudaStream_t sm, int *n, Recorder *r) {
                          for (int k = 0; k <= K; ++k) {
                              const void *ek = k == 0 ? e : (const void *)bounce_e(ctx, k);
                              void *Fk = k == K ? out : (void *)bounce_F(ctx, k);
                              cudaError_t err = enqueue_lighting(pl, *rt, ek, s, Fk, blur, thr, sm, n, r, br);
                              if (err == cudaSuccess && k < K)
                                  err = launch_bounce_source(pl, e, s, a, Fk, bounce_e(ctx, k + 1), sm, n, r);
                              if (err != cudaSuccess) return err;
                          }
                          return cudaSuccess;
                      },
                      where);
    if (st != HRC_OK) return st;
    ctx->have_fwd = false;   // the levels are those of bounce K, not of (e, s)
    ctx->have_bounce = true;
    ctx->last_e = e;
    ctx->last_s = s;
    ctx->last_a = a;
    ctx->last_K = K;
    ctx->bounce_levels_ok = true;
    return HRC_OK;
}

hrc_status bounces_backward(hrc_ctx *ctx, const void *gF, void *ge, void *gs, void *ga, bool f64, const char *where) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (f64 != (ctx->prec == P_FP64))
        return fail(ctx, HRC_ESTATE, std::string(where) + (f64 ? ": set HRC_FP64_TEST first" : ": context is in HRC_FP64_TEST"));
    if (!ctx->have_bounce) return fail(ctx, HRC_ESTATE, std::string(where) + ": no bounce forward on this context");
    if (!gF || !ge || !gs || !ga) return fail(ctx, HRC_EINVAL, std::string(where) + ": NULL pointer");
    if (!aligned16(gF) || !aligned16(ge) || !aligned16(gs) || !aligned16(ga))
        return fail(ctx, HRC_EINVAL, std::string(where) + ": pointers must be 16-byte aligned");
    const Plan pl = f64 ? ctx->plan64 : ctx->plan;
    const RayTable *rt = &ctx->rt;
    void *blur = ctx->blur ? ctx->blur_buf : nullptr;
    const double thr = ctx->blur_thr;
    const void *le = ctx->last_e, *ls = ctx->last_s, *la = ctx->last_a;
    const int K = ctx->last_K;
    // the last bounce may read the levels its forward left, unless a
    // backward since recomputed earlier bounces over them
    const bool rcK = ctx->bwd_recompute || !ctx->bounce_levels_ok;
    void *gek = bounce_scratch(ctx, 0), *gFp = bounce_scratch(ctx, 1), *gsk = bounce_scratch(ctx, 2);
    const PassKey key{{le, ls, la, gF, ge, gs, ga, (const void *)(intptr_t)(2 * K + (rcK ? 1 : 0))}};
    st = run_pass_key(ctx, f64 ? 15 : 14, key,
                      [&](cudaStream_t sm, int *n, Recorder *r) {
                          const void *gin = gF;
                          for (int k = K; k >= 0; --k) {
                              const void *ek = k == 0 ? le : (const void *)bounce_e(ctx, k);
                              cudaError_t err = enqueue_lighting_adj(pl, *rt, ek, ls, gin, gek, gsk, k == K ? rcK : true,
                                                                     blur, thr, sm, n, r);
                              if (err == cudaSuccess)
                                  err = launch_bounce_adj(pl, k == K, k > 0, gek, gsk, k > 0 ? bounce_F(ctx, k - 1) : nullptr,
                                                          la, ls, ge, gs, ga, gFp, sm, n, r);
                              if (err != cudaSuccess) return err;
                              gin = gFp;
                          }
                          return cudaSuccess;
                      },
                      where);
    if (st != HRC_OK) return st;
    if (K > 0) ctx->bounce_levels_ok = false;   // bounce 0's levels are in the buffers now
    return HRC_OK;
}

}  // namespace

extern "C" {

hrc_status hrc_fluence_bounces(hrc_ctx *ctx, const float *emission, const float *sigma_t, const float *albedo,
                               int bounces, float *out) {
    if (ctx && ctx->per_channel && ctx->prec != P_FP64 && check_ctx(ctx) == HRC_OK)
        return chan_bounces(ctx, emission, sigma_t, albedo, bounces, out, false);
    return bounces_forward(ctx, emission, sigma_t, albedo, bounces, out, false, "hrc_fluence_bounces");
}

hrc_status hrc_fluence_bounces_f64(hrc_ctx *ctx, const double *emission, const double *sigma_t,
                                   const double *albedo, int bounces, double *out) {
    if (ctx && ctx->per_channel && ctx->prec == P_FP64 && check_ctx(ctx) == HRC_OK)
        return chan_bounces(ctx, emission, sigma_t, albedo, bounces, out, true);
    return bounces_forward(ctx, emission, sigma_t, albedo, bounces, out, true, "hrc_fluence_bounces_f64");
}

hrc_status hrc_fluence_bounces_backward(hrc_ctx *ctx, const float *grad_F, float *grad_emission,
                                        float *grad_sigma_t, float *grad_albedo) {
    if (ctx && ctx->per_channel && ctx->prec != P_FP64 && check_ctx(ctx) == HRC_OK)
        return chan_bounces_backward(ctx, grad_F, grad_emission, grad_sigma_t, grad_albedo, false);
    return bounces_backward(ctx, grad_F, grad_emission, grad_sigma_t, grad_albedo, false,
                            "hrc_fluence_bounces_backward");
}

hrc_status hrc_fluence_bounces_backward_f64(hrc_ctx *ctx, const double *grad_F, double *grad_emission,
                                            double *grad_sigma_t, double *grad_albedo) {
    if (ctx && ctx->per_channel && ctx->prec == P_FP64 && check_ctx(ctx) == HRC_OK)
        return chan_bounces_backward(ctx, grad_F, grad_emission, grad_sigma_t, grad_albedo, true);
    return bounces_backward(ctx, grad_F, grad_emission, grad_sigma_t, grad_albedo, true,
                            "hrc_fluence_bounces_backward_f64");
}

hrc_status hrc_bounce_source(hrc_ctx *ctx, const float *emission, const float *sigma_t, const float *albedo,
                             const float *fluence, float *out) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (ctx->batched || ctx->prec == P_FP64)
        return fail(ctx, HRC_ESTATE, "hrc_bounce_source: single-scene fp32 / fp16 / bf16 contexts");
    if (!emission || !sigma_t || !albedo || !fluence || !out) return fail(ctx, HRC_EINVAL, "hrc_bounce_source: NULL pointer");
    if (!aligned16(emission) || !aligned16(sigma_t) || !aligned16(albedo) || !aligned16(fluence) || !aligned16(out))
        return fail(ctx, HRC_EINVAL, "hrc_bounce_source: pointers must be 16-byte aligned");
    Recorder off;
    int n = 0;
    cudaError_t e = launch_bounce_source(ctx->plan, emission, sigma_t, albedo, fluence, out, ctx->stream, &n, &off,
                                         ctx->per_channel);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_bounce_source");
    ctx->launches = n;
    return HRC_OK;
}


// ---------------------------------------------------------------------------
// Batched contexts
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// Build and upload the ticket tables of the three modes (forward, backward,
// backward with recomputed levels).
hrc_status build_batched_tables(hrc_ctx *ctx) {
    std::vector<int> order(ctx->nscenes);
    for (int i = 0; i < ctx->nscenes; ++i) order[i] = i;
    if (ctx->order == 1)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (long long)ctx->Ws[a] * ctx->Hs[a] > (long long)ctx->Ws[b] * ctx->Hs[b];
        });
    for (int mode = 0; mode < 3; ++mode) {
        std::vector<std::vector<StageDesc>> st(ctx->nscenes);
        size_t maxs = 0;
        // the tile steps (trace, adjoint trace) leave the persistent stage
        // lists and become one multi-scene launch each, in list order
        for (auto &t : ctx->tiles[mode]) {
            cudaFree(t.d_off);
            cudaFree(t.d_nx);
        }
        ctx->tiles[mode].clear();
        std::vector<std::vector<int>> toff, tnx;
        for (int i = 0; i < ctx->nscenes; ++i) {
            std::vector<StageDesc> all;
            batched_stages(ctx->bplans[i], mode, all);
            int ti = 0;
            for (const StageDesc &d : all) {
                if (d.kind != BK_TRACE && d.kind != BK_ADJ_TRACE) {
                    st[i].push_back(d);
                    continue;
                }
                if (i == 0) {
                    hrc_ctx::TileLaunch t;
                    t.kind = d.kind;
                    t.pair = d.level;
                    t.before = d.kind == BK_TRACE;
                    ctx->tiles[mode].push_back(t);
                    toff.push_back(std::vector<int>(1, 0));
                    tnx.push_back(std::vector<int>());
                }
                auto &t = ctx->tiles[mode][ti];
                toff[ti].push_back(toff[ti].back() + d.count);
                tnx[ti].push_back(d.nvb);
                t.total += d.count;
                t.bytes += d.bytes;
                ++ti;
            }
            maxs = std::max(maxs, st[i].size());
        }
        for (size_t k = 0; k < ctx->tiles[mode].size(); ++k) {
            auto &t = ctx->tiles[mode][k];
            cudaError_t e = cudaMalloc(&t.d_off, sizeof(int) * toff[k].size());
            if (e == cudaSuccess) e = cudaMalloc(&t.d_nx, sizeof(int) * tnx[k].size());
            if (e == cudaSuccess)
                e = cudaMemcpy(t.d_off, toff[k].data(), sizeof(int) * toff[k].size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(t.d_nx, tnx[k].data(), sizeof(int) * tnx[k].size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batched tile tables");
        }
        std::vector<int> cbase(ctx->nscenes);
        int nc = 0;
        for (int i = 0; i < ctx->nscenes; ++i) { cbase[i] = nc; nc += (int)st[i].size(); }
        std::vector<StageBlock> blocks;
        long long tick = 0;
        double bytes = 0;
        for (size_t k = 0; k < maxs; ++k)
            for (int i : order) {
                if (k >= st[i].size()) continue;
                const StageDesc &d = st[i][k];
                StageBlock b;
                b.first = tick;
                b.count = d.count;
                b.scene = i;
                b.kind = d.kind;
                b.level = d.level;
                b.nvb = d.nvb;
                b.rpi = d.rpi;
                b.rows = d.rows;
                b.dep = k == 0 ? -1 : cbase[i] + (int)k - 1;
                b.dep_target = k == 0 ? 0 : st[i][k - 1].count;
                b.own = cbase[i] + (int)k;
                b.rs = d.rs;
                blocks.push_back(b);
                tick += d.count;
                bytes += d.bytes;
            }
        // chunk[c] = the block holding ticket c << shift (c = 0 .. last chunk
        // + 1, the extra entry bounding the search of the last chunk)
        const long long nchunk = ((tick + (1LL << kTicketChunkShift) - 1) >> kTicketChunkShift) + 1;
        std::vector<int> chunk((size_t)nchunk);
        {
            size_t b = 0;
            for (long long c = 0; c < nchunk; ++c) {
                const long long t = std::min(c << kTicketChunkShift, tick > 0 ? tick - 1 : 0);
                while (b + 1 < blocks.size() && blocks[b + 1].first <= t) ++b;
                chunk[(size_t)c] = (int)b;
            }
        }
        if (ctx->d_blocks[mode]) cudaFree(ctx->d_blocks[mode]);
        if (ctx->d_chunk[mode]) cudaFree(ctx->d_chunk[mode]);
        ctx->d_blocks[mode] = nullptr;
        ctx->d_chunk[mode] = nullptr;
        cudaError_t e = cudaMalloc(&ctx->d_blocks[mode], sizeof(StageBlock) * blocks.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->d_blocks[mode], blocks.data(), sizeof(StageBlock) * blocks.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMalloc(&ctx->d_chunk[mode], sizeof(int) * chunk.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->d_chunk[mode], chunk.data(), sizeof(int) * chunk.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batched tables");
        ctx->nblocks[mode] = (int)blocks.size();
        ctx->total[mode] = tick;
        ctx->ncounters[mode] = nc;
        ctx->bbytes[mode] = bytes;
        // schedule 2: the same stages as level-major multi-scene launches
        for (auto &ml : ctx->multi[mode]) cudaFree(ml.d_ents);
        ctx->multi[mode].clear();
        std::vector<MultiDesc> md;
        multi_stages(ctx->bplans, mode, md);
        for (const MultiDesc &d : md) {
            hrc_ctx::MultiLaunch ml;
            ml.kind = d.kind;
            ml.level = d.level;
            ml.blocks = d.blocks;
            ml.nent = (int)d.ents.size();
            ml.bytes = d.bytes;
            e = cudaMalloc(&ml.d_ents, sizeof(MultiEnt) * d.ents.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(ml.d_ents, d.ents.data(), sizeof(MultiEnt) * d.ents.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(ml.d_ents);
                return cuda_fail(ctx, e, "batched multi-scene tables");
            }
            ctx->multi[mode].push_back(ml);
        }
    }
    return HRC_OK;
}

// Lay out every scene's levels (fp32 layout = the largest) in the arena and
// upload plans, offsets and arc tables for the current precision.
hrc_status build_batched_plans(hrc_ctx *ctx, int prec) {
    size_t off = 0;
    ctx->bplans.assign(ctx->nscenes, Plan());
    for (int i = 0; i < ctx->nscenes; ++i) {
        off = build_plan(ctx->Ws[i], ctx->Hs[i], ctx->C, ctx->cascades, prec, off, ctx->bplans[i], true);
        ctx->bplans[i].arena = ctx->arena;
        ctx->bplans[i].sched = 0;
        ctx->bplans[i].mgroups = 1;
        ctx->bplans[i].mthreads = 128;
        ctx->bplans[i].vmajor = 0;
        // per-scene chains (schedule 1): the launch configuration the
        // single-scene autotuner picks at most sizes: four v per thread in the
        // merge up, and bulk-copy staging of the merge down in the 16-bit
        // precisions
        ctx->bplans[i].mgroups = 4;
        ctx->bplans[i].mdown = (prec == P_FP16 || prec == P_BF16) ? 1 : 0;
        ctx->bplans[i].status = ctx->d_status;
    }
    if (off > ctx->arena_bytes) return fail(ctx, HRC_ENOMEM, "batched layout exceeds the arena");
    for (int i = 0; i < ctx->nscenes; ++i) {
        cudaError_t e = upload_arcs(ctx->bplans[i], ctx->arena);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batched arcs");
    }
    cudaError_t e = cudaMemcpy(ctx->d_plans, ctx->bplans.data(), sizeof(Plan) * ctx->nscenes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batched plans");
    return build_batched_tables(ctx);
}

// Schedule 1: every scene's own launch sequence (as a single-scene pass),
// scenes largest first, round-robin over the auxiliary streams forked from
// and joined back to the pass's stream; captured, the graph has one
// independent branch per stream, so kernels of different scenes overlap.
hrc_status run_batched_chains(hrc_ctx *ctx, int mode, const void *e, const void *s, void *F, const void *gF,
                              void *ge, void *gs, const char *where) {
    auto enqueue = [&](cudaStream_t st, int *n, Recorder *) {
        Recorder off;   // per-launch timing is not recorded across streams
        cudaError_t err = cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st);
        if (err == cudaSuccess) err = cudaEventRecord(ctx->ev_fork, st);
        for (int k = 0; k < hrc_ctx::kAux && err == cudaSuccess; ++k) err = cudaStreamWaitEvent(ctx->aux[k], ctx->ev_fork, 0);
        for (int idx = 0; idx < ctx->nscenes && err == cudaSuccess; ++idx) {
            const int i = ctx->by_size[idx];
            cudaStream_t as = ctx->aux[idx % hrc_ctx::kAux];
            const Plan &pl = ctx->bplans[i];
            const float *ei = (const float *)e + ctx->eoff[i], *si = (const float *)s + ctx->soff[i];
            if (mode == 0)
                err = launch_forward(pl, ctx->rt, ei, si, (float *)F + ctx->eoff[i], as, n, &off);
            else
                err = launch_backward(pl, ctx->rt, ei, si, (const float *)gF + ctx->eoff[i], (float *)ge + ctx->eoff[i],
                                      (float *)gs + ctx->soff[i], mode == 2, as, n, &off);
        }
        for (int k = 0; k < hrc_ctx::kAux && err == cudaSuccess; ++k) {
            err = cudaEventRecord(ctx->ev_join[k], ctx->aux[k]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(st, ctx->ev_join[k], 0);
        }
        return err;
    };
    const void *k3 = (const void *)(intptr_t)(1 << 20);
    return run_pass(ctx, 8 + mode, mode == 0 ? e : gF, mode == 0 ? s : ge, mode == 0 ? F : gs, k3, nullptr, enqueue,
                    where);
}

// Schedule 2: the tile steps of every scene as multi-scene tile launches and
// every other stage as one level-major multi-scene launch, in dependency
// order (kernels_batched.cu, multi_stages).
hrc_status run_batched_levels(hrc_ctx *ctx, int mode, const void *e, const void *s, void *F, const void *gF,
                              void *ge, void *gs, const char *where) {
    BatchArgs a;
    std::memset(&a, 0, sizeof(a));
    a.plans = ctx->d_plans;
    a.eoff = ctx->d_eoff;
    a.soff = ctx->d_soff;
    a.status = ctx->d_status;
    a.e = e;
    a.s = s;
    a.F = F;
    a.gF = gF;
    a.ge = ge;
    a.gs = gs;
    const int prec = ctx->prec, C = ctx->C, nsc = ctx->nscenes;
    const std::vector<hrc_ctx::TileLaunch> &tl = ctx->tiles[mode];
    const std::vector<hrc_ctx::MultiLaunch> &ml = ctx->multi[mode];
    auto enqueue = [&](cudaStream_t st, int *n, Recorder *r) {
        cudaError_t err = cudaMemsetAsync(a.status, 0, sizeof(int), st);
        auto tiles = [&](bool before) {
            for (const auto &t : tl) {
                if (t.before != before || err != cudaSuccess) continue;
                r->begin(t.kind == BK_TRACE ? K_TRACE012 : K_ADJ_TRACE, t.pair, t.bytes);
                err = launch_batched_tiles(a, prec, C, t.kind, t.d_off, t.d_nx, nsc, t.pair, t.total, st);
                r->end();
                ++*n;
            }
        };
        tiles(true);
        for (const auto &m : ml) {
            if (err != cudaSuccess) break;
            const int kk = m.kind == MK_MERGE_UP4 ? K_MERGE_UP
                           : (m.kind == MK_MERGE_DOWN4 || m.kind == MK_MERGE_DOWN_BULK) ? K_MERGE_DOWN
                           : m.kind == MK_SUM ? K_FLUENCE_SUM
                           : m.kind == MK_ADJ_SUM ? K_ADJ_SUM
                           : m.kind == MK_ADJ_MU ? K_ADJ_MERGE_UP : K_ADJ_MERGE_DOWN;
            void *io = m.kind == MK_SUM ? F : (m.kind == MK_ADJ_SUM ? const_cast<void *>(gF) : nullptr);
            r->begin(kk, m.level, m.bytes);
            err = launch_multi(prec, C, m.kind, ctx->d_plans, m.d_ents, m.nent, m.level, m.blocks, ctx->d_eoff, io, st);
            r->end();
            ++*n;
        }
        if (err == cudaSuccess) tiles(false);
        return err;
    };
    const void *k3 = (const void *)(intptr_t)(2 << 20);
    return run_pass(ctx, 8 + mode, mode == 0 ? e : gF, mode == 0 ? s : ge, mode == 0 ? F : gs, k3, nullptr, enqueue,
                    where);
}

hrc_status run_batched(hrc_ctx *ctx, int mode, const void *e, const void *s, void *F, const void *gF, void *ge,
                       void *gs, const char *where) {
    if (ctx->bsched == 1) return run_batched_chains(ctx, mode, e, s, F, gF, ge, gs, where);
    if (ctx->bsched == 2) return run_batched_levels(ctx, mode, e, s, F, gF, ge, gs, where);
    BatchArgs a;
    a.plans = ctx->d_plans;
    a.eoff = ctx->d_eoff;
    a.soff = ctx->d_soff;
    a.blocks = ctx->d_blocks[mode];
    a.chunk = ctx->d_chunk[mode];
    a.nblocks = ctx->nblocks[mode];
    a.total = ctx->total[mode];
    a.ticket = ctx->d_ticket;
    a.counters = ctx->d_counters;
    a.status = ctx->d_status;
    a.withhold = ctx->withhold;
    a.spin_limit = ctx->spin_limit;
    a.e = e;
    a.s = s;
    a.F = F;
    a.gF = gF;
    a.ge = ge;
    a.gs = gs;
    const int prec = ctx->prec, C = ctx->C, bpsm = ctx->blocks_per_sm, nc = ctx->ncounters[mode];
    const double bytes = ctx->bbytes[mode];
    const int nsc = ctx->nscenes;
    const std::vector<hrc_ctx::TileLaunch> &tl = ctx->tiles[mode];
    auto enqueue = [&](cudaStream_t st, int *n, Recorder *r) {
        cudaError_t err = cudaMemsetAsync(a.counters, 0, sizeof(int) * nc, st);
        if (err == cudaSuccess) err = cudaMemsetAsync(a.ticket, 0, sizeof(unsigned long long), st);
        if (err == cudaSuccess) err = cudaMemsetAsync(a.status, 0, sizeof(int), st);
        auto tiles = [&](bool before) {
            for (const auto &t : tl) {
                if (t.before != before || err != cudaSuccess) continue;
                r->begin(t.kind == BK_TRACE ? K_TRACE012 : K_ADJ_TRACE, t.pair, t.bytes);
                err = launch_batched_tiles(a, prec, C, t.kind, t.d_off, t.d_nx, nsc, t.pair, t.total, st);
                r->end();
                ++*n;
            }
        };
        tiles(true);
        if (err != cudaSuccess) return err;
        r->begin(K_BATCHED, mode, bytes);
        err = launch_batched(a, prec, C, bpsm, mode == 0 ? 0 : 1, st);
        r->end();
        ++*n;
        if (err != cudaSuccess) return err;
        tiles(false);
        return err;
    };
    // the graph key includes the tuning state (blocks per SM, order, test hooks)
    const void *k3 = (const void *)(intptr_t)((ctx->blocks_per_sm << 8) | (ctx->order << 4) | (ctx->withhold >= 0 ? 1 : 0));
    const void *k4 = (const void *)(intptr_t)ctx->spin_limit;
    return run_pass(ctx, 8 + mode, mode == 0 ? e : gF, mode == 0 ? s : ge, mode == 0 ? F : gs, k3, k4, enqueue, where);
}

}  // namespace

extern "C" {

hrc_status hrc_create_batched(int n, const int *W, const int *H, int channels, int cascades, hrc_ctx **out) {
    return hrc_create_batched_prec(n, W, H, channels, cascades, HRC_FP32, out);
}

hrc_status hrc_create_batched_prec(int n, const int *W, const int *H, int channels, int cascades, hrc_precision prec,
                                   hrc_ctx **out) {
    if (!out) return fail(nullptr, HRC_EINVAL, "hrc_create_batched: out is NULL");
    if (prec < HRC_FP32 || prec > HRC_BF16_LOGT)
        return fail(nullptr, HRC_EINVAL, "hrc_create_batched: precision must be fp32, fp16 or bf16");
    *out = nullptr;
    if (n < 1 || !W || !H) return fail(nullptr, HRC_EINVAL, "hrc_create_batched: need n >= 1 scenes");
    if (channels < 1 || channels > 4) return fail(nullptr, HRC_EINVAL, "hrc_create_batched: channels must be in [1, 4]");
    for (int i = 0; i < n; ++i)
        if (W[i] < 1 || H[i] < 1 || W[i] > 16384 || H[i] > 16384)
            return fail(nullptr, HRC_EINVAL, "hrc_create_batched: W and H must be in [1, 16384]");
    hrc_ctx *ctx = new (std::nothrow) hrc_ctx();
    if (!ctx) return fail(nullptr, HRC_ENOMEM, "hrc_create_batched: host allocation failed");
    ctx->batched = true;
    ctx->nscenes = n;
    ctx->Ws.assign(W, W + n);
    ctx->Hs.assign(H, H + n);
    ctx->C = channels;
    ctx->cascades = cascades;
    ctx->rt = make_ray_table();
    ctx->by_size.resize(n);
    for (int i = 0; i < n; ++i) ctx->by_size[i] = i;
    std::stable_sort(ctx->by_size.begin(), ctx->by_size.end(),
                     [&](int a, int b) { return (long long)W[a] * H[a] > (long long)W[b] * H[b]; });
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = prepare_device_once();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    for (int k = 0; k < hrc_ctx::kAux && e == cudaSuccess; ++k) {
        e = cudaStreamCreateWithFlags(&ctx->aux[k], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) { delete ctx; return fail(nullptr, HRC_ECUDA, std::string("hrc_create_batched: ") + cudaGetErrorString(e)); }
    size_t bytes = 0;
    ctx->eoff.assign(n + 1, 0);
    ctx->soff.assign(n + 1, 0);
    ctx->prec = (int)prec;
    for (int i = 0; i < n; ++i) {
        Plan p;
        bytes = build_plan(W[i], H[i], channels, cascades, (int)prec, bytes, p, true);
        ctx->eoff[i + 1] = ctx->eoff[i] + (long long)channels * W[i] * H[i];
        ctx->soff[i + 1] = ctx->soff[i] + (long long)W[i] * H[i];
    }
    ctx->arena_bytes = bytes;
    int maxstages = 0;
    for (int i = 0; i < n; ++i) maxstages += 4 * (levels_for(std::max(W[i], H[i]), cascades) + 3) + 8;
    e = cudaMalloc(&ctx->arena, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_plans, sizeof(Plan) * n);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_eoff, sizeof(long long) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_soff, sizeof(long long) * (n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_counters, sizeof(int) * maxstages);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_ticket, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        hrc_destroy(ctx);
        return fail(nullptr, HRC_ENOMEM, "hrc_create_batched: cudaMalloc of " + std::to_string(bytes) + " bytes failed");
    }
    e = cudaMemcpy(ctx->d_eoff, ctx->eoff.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx->d_soff, ctx->soff.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e != cudaSuccess) { hrc_destroy(ctx); return fail(nullptr, HRC_ECUDA, "hrc_create_batched: upload failed"); }
    hrc_status st = build_batched_plans(ctx, (int)prec);
    if (st != HRC_OK) {
        std::string msg = ctx->err;
        hrc_destroy(ctx);
        return fail(nullptr, st, msg);
    }
    for (int mode = 0; mode < 3; ++mode)
        if (ctx->ncounters[mode] > maxstages) {
            hrc_destroy(ctx);
            return fail(nullptr, HRC_EINVAL, "hrc_create_batched: stage count exceeds the counter buffer");
        }
    *out = ctx;
    return HRC_OK;
}

hrc_status hrc_scene_offsets(const hrc_ctx *ctx, long long *emis_off, long long *sigma_off) {
    if (!ctx || !ctx->batched) return HRC_EINVAL;
    for (int i = 0; i <= ctx->nscenes; ++i) {
        if (emis_off) emis_off[i] = ctx->eoff[i];
        if (sigma_off) sigma_off[i] = ctx->soff[i];
    }
    return HRC_OK;
}

hrc_status hrc_fluence_batched(hrc_ctx *ctx, const float *emission, const float *sigma_t, float *out) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (!ctx->batched) return fail(ctx, HRC_ESTATE, "hrc_fluence_batched: not a batched context");
    if (!emission || !sigma_t || !out) return fail(ctx, HRC_EINVAL, "hrc_fluence_batched: NULL pointer");
    if (!aligned16(emission) || !aligned16(sigma_t) || !aligned16(out))
        return fail(ctx, HRC_EINVAL, "hrc_fluence_batched: pointers must be 16-byte aligned");
    st = run_batched(ctx, 0, emission, sigma_t, out, nullptr, nullptr, nullptr, "hrc_fluence_batched");
    if (st != HRC_OK) return st;
    ctx->last_e = emission;
    ctx->last_s = sigma_t;
    ctx->have_fwd = true;
    return HRC_OK;
}

hrc_status hrc_fluence_backward_batched(hrc_ctx *ctx, const float *grad_F, float *grad_emission, float *grad_sigma_t) {
    hrc_status st = check_ctx(ctx);
    if (st != HRC_OK) return st;
    if (!ctx->batched) return fail(ctx, HRC_ESTATE, "hrc_fluence_backward_batched: not a batched context");
    if (!ctx->have_fwd) return fail(ctx, HRC_ESTATE, "hrc_fluence_backward_batched: no forward pass on this context");
    if (!grad_F || !grad_emission || !grad_sigma_t) return fail(ctx, HRC_EINVAL, "hrc_fluence_backward_batched: NULL pointer");
    if (!aligned16(grad_F) || !aligned16(grad_emission) || !aligned16(grad_sigma_t))
        return fail(ctx, HRC_EINVAL, "hrc_fluence_backward_batched: pointers must be 16-byte aligned");
    return run_batched(ctx, ctx->bwd_recompute ? 2 : 1, ctx->last_e, ctx->last_s, nullptr, grad_F, grad_emission, grad_sigma_t,
                       "hrc_fluence_backward_batched");
}

hrc_status hrc_batched_sync(hrc_ctx *ctx) {
    if (!ctx || !ctx->batched) return HRC_EINVAL;
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_batched_sync");
    if (status == HRC_ETIMEOUT) return fail(ctx, HRC_ETIMEOUT, "batched launch: a dependency wait gave up");
    return status == 0 ? HRC_OK : (hrc_status)status;
}

hrc_status hrc_batched_debug(hrc_ctx *ctx, int withhold_counter, long long spin_limit) {
    if (!ctx || !ctx->batched) return HRC_EINVAL;
    ctx->withhold = withhold_counter;
    ctx->spin_limit = spin_limit > 0 ? spin_limit : (1LL << 24);
    return HRC_OK;
}

hrc_status hrc_batched_schedule(hrc_ctx *ctx, int schedule) {
    if (!ctx || !ctx->batched) return HRC_EINVAL;
    if (schedule < 0 || schedule > 2) return fail(ctx, HRC_EINVAL, "hrc_batched_schedule: 0, 1 or 2");
    ctx->bsched = schedule;
    return HRC_OK;
}

hrc_status hrc_batched_tune(hrc_ctx *ctx, int blocks_per_sm, int order) {
    if (!ctx || !ctx->batched || blocks_per_sm < 0 || order < 0 || order > 1) return HRC_EINVAL;
    ctx->blocks_per_sm = blocks_per_sm;
    if (order != ctx->order) {
        ctx->order = order;
        return build_batched_tables(ctx);
    }
    return HRC_OK;
}

hrc_status hrc_copy_level(hrc_ctx *ctx, int q, int which, int n, float *dst, long long *count) {
    if (!ctx) return HRC_EINVAL;
    if (ctx->per_channel) return fail(ctx, HRC_ESTATE, "hrc_copy_level: per-channel extinction (levels live per channel)");
    const Plan &pl = ctx->prec == P_FP64 ? ctx->plan64 : ctx->plan;
    if (q < 0 || q > 3 || (which != 0 && which != 1)) return fail(ctx, HRC_EINVAL, "hrc_copy_level: bad q / which");
    const QuadGeom &g = pl.q[q];
    if (n < 0 || (which == 0 && n > g.N) || (which == 1 && n >= g.N))
        return fail(ctx, HRC_EINVAL, "hrc_copy_level: level does not exist");
    const long long cnt = which == 0 ? (long long)g.Un[n] * ((1 << n) + 1) * g.V * (ctx->C + 1)
                                     : (long long)g.Un[n] * (1 << n) * g.V * ctx->C;
    if (count) *count = cnt;
    if (!dst) return HRC_OK;
    cudaError_t e = cudaSuccess;
    if (which == 1 && n == 0) e = launch_r0(pl, ctx->stream);   // the forward does not store R_0
    if (e == cudaSuccess) e = launch_copy_level(pl, q, which, n, dst, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hrc_copy_level");
    return HRC_OK;
}

}  // extern "C"
