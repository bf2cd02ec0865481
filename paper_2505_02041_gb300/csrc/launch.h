// launch.h -- host-side entry points of the kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "hrc_internal.cuh"

namespace hrc {

// Kernel kinds, for per-launch timing records.
enum KernelKind {
    K_TRACE012 = 0, K_MERGE_UP = 1, K_MERGE_DOWN = 2, K_FLUENCE_SUM = 3,
    K_ADJ_SUM = 4, K_ADJ_MERGE_DOWN = 5, K_ADJ_MERGE_UP = 6, K_ADJ_TRACE = 7,
    K_BATCHED = 8, K_OTHER = 9, K_CROSS_BLUR = 10, K_ADJ_CROSS_BLUR = 11, K_BOUNCE = 12, K_ADJ_BOUNCE = 13
};

// Optional per-launch CUDA-event timing (off by default).  Events come from
// a pool created when timing is enabled; recording is stream-ordered.  With
// `ext` the records are made while a graph is being captured: they become
// event-record nodes of the graph (cudaEventRecordExternal), so every replay
// times the kernels as the graph runs them.
// With `coarse`, consecutive launches of one kind form one record (a phase:
// one event before its first launch, one after its last), so that no event
// sits between the launches of a phase.
struct Recorder {
    struct Rec { int kind, level; double bytes; cudaEvent_t a, b; int launches; };
    bool on = false;
    bool ext = false;
    bool coarse = false;
    bool open = false;
    cudaStream_t st = nullptr;
    std::vector<cudaEvent_t> pool;
    std::vector<Rec> recs;
    size_t used = 0;
    void reset(cudaStream_t s) { st = s; recs.clear(); used = 0; open = false; }
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void record(cudaEvent_t e) {
        if (ext) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    }
    void begin(int kind, int level, double bytes) {
        if (!on) return;
        if (coarse && open) {
            if (recs.back().kind == kind) {   // the phase continues
                recs.back().bytes += bytes;
                ++recs.back().launches;
                return;
            }
            finish();
        }
        Rec r{kind, level, bytes, next(), next(), 1};
        record(r.a);
        recs.push_back(r);
        open = coarse;
    }
    void end() {
        if (!on || recs.empty() || coarse) return;
        record(recs.back().b);
    }
    // closes the open phase (coarse records); called at the end of a pass
    void finish() {
        if (!on || !open || recs.empty()) return;
        record(recs.back().b);
        open = false;
    }
    ~Recorder() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// Parallel branches of a pass (launch schedule 2): the pass forks from its
// stream onto s[0..3] through `fork` and joins back through join[0..3];
// inside graph capture the branches become parallel paths of the graph.
struct Branches {
    cudaStream_t s[4];
    cudaEvent_t fork, join[4];
};

// Forward pass of Algorithm 1 (all four quadrant frames), enqueued on `st`.
// e, s, F are fp32 device pointers (fp64 for P_FP64).  With schedule 2 and
// `br`, each frame's chain (trace, merge up, merge down) runs on its own
// branch and the fluence sum after the join; without `br` (or with per-launch
// timing on) schedule 2 runs level-major like schedule 0.
cudaError_t launch_forward(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                           cudaStream_t st, int *launches, Recorder *rec, const Branches *br = nullptr);

// ---------------------------------------------------------------------------
// Batched persistent launch (kernels_batched.cu)
// ---------------------------------------------------------------------------
enum BatchKind {
    BK_TRACE = 0, BK_MERGE_UP, BK_MERGE_DOWN2, BK_SUM, BK_ADJ_SUM, BK_ADJ_R2, BK_ADJ_R1,
    BK_ADJ_T2, BK_ADJ_T1, BK_ADJ_MU, BK_ADJ_TRACE
};

// One stage of one scene: tickets first .. first+count-1.  Row kinds decode
// an item j as (row j / nvb, v-block j % nvb); tile kinds as (x-block
// j % nvb, y-block j / nvb).
struct StageBlock {
    long long first;
    int count, scene, kind, level, nvb;
    int rpi;               // rows per item (row kinds); item j covers rows (j / nvb) * rpi ..
    long long rows;        // rows of the stage (row kinds)
    int dep, dep_target;   // counter waited on (-1: none) and its final value
    int own;               // counter published to
    RowSplit rs;
};

constexpr int kTicketChunkShift = 6;   // tickets per entry of the ticket -> block index: 64

struct BatchArgs {
    const Plan *plans;
    const long long *eoff, *soff;     // per-scene element offsets of [C][H][W] / [H][W] blocks
    const StageBlock *blocks;
    int nblocks;
    long long total;                  // tickets
    const int *chunk;                 // chunk[c]: the block holding ticket c << kTicketChunkShift
    int pad_;
    unsigned long long *ticket;
    int *counters;
    int *status;
    int withhold;                     // test hook: a counter never published (-1: none)
    long long spin_limit;             // polls before a wait gives up
    const void *e, *s;
    void *F;
    const void *gF;
    void *ge, *gs;
};

// Stage list of one scene: mode 0 = forward (with the fluence sum),
// mode 1 = backward (every adjoint step over the levels of the last forward);
// mode 2 = backward recomputing the levels first (forward stages without the
// fluence sum, then the adjoint stages; run by the mode-1 kernel).
struct StageDesc {
    int kind, level, count, nvb, rpi;
    long long rows;
    RowSplit rs;
    double bytes;
};
void batched_stages(const Plan &pl, int mode, std::vector<StageDesc> &out);
cudaError_t launch_batched(const BatchArgs &a, int prec, int C, int blocks_per_sm, int mode, cudaStream_t st);
// The tile steps of every scene (kind BK_TRACE, or BK_ADJ_TRACE of quadrant
// pair `pair`) in one launch of `total` blocks (off / nx: per-scene prefix
// sums of tile counts and tiles along x, device arrays).
cudaError_t launch_batched_tiles(const BatchArgs &a, int prec, int C, int kind, const int *off, const int *nx,
                                 int nscenes, int pair, int total, cudaStream_t st);

// Level-major multi-scene launches (batched schedule 2): one launch runs one
// stage (a merge-up level, a merge-down level, an adjoint level, the fluence
// sum or its reverse) of every scene that has it.  Block b of the launch is
// block b - first of the entry (scene) with the largest first <= b.
enum MultiKind { MK_MERGE_UP4 = 0, MK_MERGE_DOWN4, MK_SUM, MK_ADJ_SUM, MK_ADJ_R2, MK_ADJ_R1, MK_ADJ_T2, MK_ADJ_T1,
                 MK_ADJ_MU, MK_MERGE_DOWN_BULK };
struct MultiEnt {
    int first;       // first block of this scene
    int scene;
    int nvb;         // v-blocks per row (row kinds), tiles along x (tile kinds)
    int pad;
    RowSplit rs;     // the stage's rows (row kinds)
};
// Threads per block of a kind, and the v covered by one block of a row kind.
int multi_threads(int kind);
int multi_vblock(int kind);
cudaError_t launch_multi(int prec, int C, int kind, const Plan *plans, const MultiEnt *ents, int nent, int n,
                         int blocks, const long long *eoff, void *io, cudaStream_t st);
// The multi-scene launches of a pass (mode as batched_stages), level-major:
// forward merge up n ascending, merge down n descending, the sum; backward
// reverse of the sum, dL/dR n ascending, dL/dT n ascending, merge-up reverse
// n descending.  The tile steps (trace, adjoint trace) are not included.
struct MultiDesc {
    int kind, level, blocks;
    double bytes;
    std::vector<MultiEnt> ents;
};
void multi_stages(const std::vector<Plan> &plans, int mode, std::vector<MultiDesc> &out);

// Host-side plan and table builders (hrc_runtime.cu).
size_t align_up(size_t x, size_t a);
int levels_for(int U, int cascades);
RayTable make_ray_table();
size_t build_plan(int W, int H, int C, int cascades, int prec, size_t off, Plan &pl, bool adjoint);
int plan_nmax(const Plan &pl);
// Message returned by hrc_last_error(NULL) on this thread.
void set_global_error(const char *msg);

// Backward pass: the adjoint of every step over the levels T_n / R_n,
// either recomputed from (e, s) first (recompute) or as the last forward left
// them in the plan's buffers; writes dL/de (ge) and dL/dsigma (gs) from dL/dF
// (gF), re-tracing (e, s).
cudaError_t launch_backward(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, bool recompute, cudaStream_t st, int *launches, Recorder *rec);

// One-time per-device kernel set-up (dynamic shared-memory limits); must run
// with the device current before the kernels are launched or captured.
cudaError_t prepare_forward_kernels();
cudaError_t prepare_backward_kernels();
cudaError_t prepare_device_once();

// Cross blur of Eq. 21 with opacity rejection (kernels_blur.cu): F = B Fr,
// and its transpose gFr = B^T g for fixed sigma; arrays [C][H][W] (fp64 for
// P_FP64, else fp32), s = sigma_t [H][W].
cudaError_t launch_cross_blur(const Plan &pl, const void *Fr, const void *s, void *F, double thr, cudaStream_t st,
                              int *launches, Recorder *rec);
cudaError_t launch_cross_blur_adj(const Plan &pl, const void *g, const void *s, void *gFr, double thr,
                                  cudaStream_t st, int *launches, Recorder *rec);
double bytes_cross_blur(const Plan &pl);

// Multi-bounce source update (kernels_bounce.cu): eo = e + a * s * F / (2 pi)
// over [C][H][W] planes (s: [H][W]); and its reverse for bounce k (first: k
// is the last bounce, the accumulators ge / gs / ga are overwritten; has_prev:
// k >= 1, so F_{k-1} = Fp exists and dL/dF_{k-1} is written to gFp).
cudaError_t launch_bounce_source(const Plan &pl, const void *e, const void *s, const void *a, const void *F,
                                 void *eo, cudaStream_t st, int *launches, Recorder *rec,
                                 bool per_channel_sigma = false);
cudaError_t launch_bounce_adj(const Plan &pl, bool first, bool has_prev, const void *gek, const void *gsk,
                              const void *Fp, const void *a, const void *s, void *ge, void *gs, void *ga, void *gFp,
                              cudaStream_t st, int *launches, Recorder *rec);

// Environment table of a map env[C][M] (kernels_env.cu): 4 * stride doubles
// then the same values as floats, stride = 2^(Nmax + 1) * C elements per
// frame, entry (2^n + j) * C + c; see Plan::envf / envd.
long long env_table_stride(const Plan &pl);
size_t env_table_bytes(const Plan &pl);
cudaError_t launch_env_table(const Plan &pl, const float *env, int M, void *table, cudaStream_t st);
// The same table from caller-supplied level-N values top[4][K][C].
cudaError_t launch_env_top(const Plan &pl, const float *top, int K, void *table, cudaStream_t st);

// Dense fp32 copy of level n of frame q (which = 0: T_n, 1: R_n).
cudaError_t launch_copy_level(const Plan &pl, int q, int which, int n, float *dst, cudaStream_t st);

// Algorithmic bytes of one launch (each array read once per consuming
// phase, each written once): T entries of C radiances + 1 transmittance,
// R entries of C values.
// R_0 of every frame into the plan's buffer (the forward does not store it).
cudaError_t launch_r0(const Plan &pl, cudaStream_t st);

// Persistent merge down (kernels_persist.cu): R_{n_hi} .. R_{n_lo} of the
// frames in qm in one launch, after resetting the plan's control block
// (pl.pctl, persist_ctl_bytes(pl) bytes).  `bytes`: the algorithmic bytes
// recorded for the launch.
bool persist_down_usable(const Plan &pl);
size_t persist_ctl_bytes(const Plan &pl);
cudaError_t launch_merge_down_persist(const Plan &pl, int qm, int n_hi, int n_lo, cudaStream_t st, int *launches,
                                      Recorder *rec, double bytes);

// Reads and clears a plan's status word (after its stream has been
// synchronised): 0, kWaitTimeout or kWaitLost.
cudaError_t read_plan_status(const Plan &pl, int *status);

// Tensor maps of fp32 emission / extinction for TMA tile staging (false when
// the layout does not allow them).
bool encode_image_maps(const Plan &pl, const void *e, const void *s, int box_x, int box_y, CUtensorMap &me,
                       CUtensorMap &ms);

double bytes_T(const Plan &pl, int q, int n);
double bytes_T_odd(const Plan &pl, int q, int n);
double bytes_T_even_dirs(const Plan &pl, int q, int n);
double bytes_R(const Plan &pl, int q, int n);

}  // namespace hrc
