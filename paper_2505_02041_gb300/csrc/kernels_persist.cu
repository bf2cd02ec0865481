// kernels_persist.cu -- the merge down (Eqs. 13-17, Sec. 4.1) over every
// level n = N-1 .. 1 of the four quadrant frames in ONE persistent launch.
//
// A per-level launch sequence pays, at every level boundary, a launch, a
// ramp (the first loads of an empty GPU) and a tail (the last, partly empty
// wave): a few microseconds per level, which dominate once the levels are
// small (a 512^2 frame's levels move 20-50 MB each).  Here persistent CTAs
// of 128 threads, as many as fit on every SM, run the whole cascade:
//
//   * Work items are row segments (q, n, x, ip, 512 v) of R_n, numbered
//     level-major (n descending), then frame, column x, cone ip, v-block.
//     Thread 0 of a CTA takes tickets from a global counter, one item
//     ahead, decodes the item and checks its dependencies: the columns of
//     R_{n+1} the item reads (Eq. 14: column (x+1)/2; Eqs. 15-17: x/2 and
//     x/2 + 1) must be complete.  A column of R_n is complete when its
//     counter reaches 2^n x v-blocks; thread 0 remembers the last columns it
//     found complete.
//   * Every thread then loads its operands for four consecutive v with
//     16-byte loads, evaluates Eq. 14 (odd x) or Eqs. 15-17 (even x) --
//     the arithmetic of the per-level kernel, entry for entry -- and stores.
//   * Thread 0 publishes each finished item: a fence, then an increment of
//     the item's column counter (publishing several items per fence was
//     measured slower: their dependents wait longer).  It never waits on a
//     dependency while holding an unpublished item.
//
// Deadlock freedom: tickets are taken in increasing order by running CTAs
// only, and an item waits only on items of the level above, whose tickets
// are smaller.  A CTA that waits holds no unpublished item, so by induction
// the smallest unfinished ticket always proceeds.  Every wait is bounded by
// the global timer (Plan::bulk_limit_ns); one that gives up records
// kWaitTimeout in the plan's status word (read by hrc_sync) and the CTA
// returns.
//
// Memory ordering: the stores of an item -> __syncthreads -> thread 0's
// __threadfence -> counter increment; a reading CTA's thread 0 acquires the
// counter (ld.acquire.gpu), then __syncthreads orders every thread's loads
// after it.
#include <climits>
#include <cstring>

#include "fwd_bodies.cuh"
#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

constexpr int kPV = 512;          // v per item: 128 threads x 4
constexpr int kPTThreads = 128;
constexpr int kPTPub = 1;         // items published per fence (more delays the dependents)

struct PSched {
    int nlev, n_hi;               // levels n_hi, n_hi - 1, .., n_hi - nlev + 1
    int deps;                     // wait on the level above (more than one level per launch)
    int total;                    // items
    int nvb[4];                   // v-blocks of kPV per row, per frame
    int lstart[HRC_MAXL + 1];     // first ticket of level index l; lstart[nlev] = total
    int qstart[HRC_MAXL][4];      // first ticket of frame q within level index l
    int cbase[4][HRC_MAXL + 1];   // counter of column x of level n, frame q: cbase[q][n] + x
    int *tick;                    // ticket counter
    int *cnt;                     // column counters
};

struct MDItem {
    int q, n, x, ip, v0;
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ MDItem md_decode(const PSched &ps, int t) {
    int l = 0;
    while (l + 1 < ps.nlev && t >= ps.lstart[l + 1]) ++l;
    int q = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (t >= ps.qstart[l][j]) q = j;
    MDItem it;
    it.q = q;
    it.n = ps.n_hi - l;
    const int local = t - ps.qstart[l][q];
    const int nvb = ps.nvb[q];
    const int row = local / nvb;
    it.v0 = (local - row * nvb) * kPV;
    it.x = 1 + (row >> it.n);
    it.ip = row & ((1 << it.n) - 1);
    return it;
}

template <int P, int C, bool ENV>
__global__ void __launch_bounds__(kPTThreads, 8) k_merge_down_persist(Plan pl, PSched ps) {
    using A = typename Prec<P>::A;
    __shared__ MDItem s_it;
    __shared__ int s_go;
    __shared__ int cache[4];           // columns thread 0 found complete
    const int tid = threadIdx.x;
    int t_cur = 0, t_next = 0, cpos = 0;
    int pend[kPTPub], npend = 0;       // thread 0: finished items not yet published
    auto publish = [&]() {
        if (npend == 0) return;
        __threadfence();
        if (pl.bulk_extra_tx == 0)   // the wait test hook withholds every publication
            for (int i = 0; i < npend; ++i) atomicAdd(ps.cnt + pend[i], 1);
        npend = 0;
    };
    if (tid == 0) {
        t_cur = atomicAdd(ps.tick, 1);
        t_next = atomicAdd(ps.tick, 1);
        cache[0] = cache[1] = cache[2] = cache[3] = -1;
    }
    for (;;) {
        if (tid == 0) {
            int go = t_cur < ps.total;
            MDItem m{0, 0, 0, 0, 0};
            if (go) {
                m = md_decode(ps, t_cur);
                const QuadGeom &g = pl.q[m.q];
                if (ps.deps && m.n < ps.n_hi && m.n + 1 < g.N) {
                    const int need = (1 << (m.n + 1)) * ps.nvb[m.q];
                    const int cb = ps.cbase[m.q][m.n + 1];
                    int cols[2] = {-1, -1};
                    if (m.x & 1) {
                        if (((m.x + 1) >> 1) < g.Un[m.n + 1]) cols[0] = cb + ((m.x + 1) >> 1);
                    } else {
                        cols[0] = cb + (m.x >> 1);
                        if ((m.x >> 1) + 1 < g.Un[m.n + 1]) cols[1] = cb + (m.x >> 1) + 1;
                    }
                    for (int d = 0; d < 2 && go; ++d) {
                        const int ci = cols[d];
                        if (ci < 0 || cache[0] == ci || cache[1] == ci || cache[2] == ci || cache[3] == ci) continue;
                        if (ld_acquire_gpu(ps.cnt + ci) < need) {
                            publish();   // hold nothing while waiting
                            const unsigned long long t0 = global_ns();
                            while (ld_acquire_gpu(ps.cnt + ci) < need) {
                                if ((long long)(global_ns() - t0) > pl.bulk_limit_ns) {
                                    atomicMax(pl.status, kWaitTimeout);
                                    go = 0;
                                    break;
                                }
                                __nanosleep(64);
                            }
                        }
                        cache[cpos] = ci;
                        cpos = (cpos + 1) & 3;
                    }
                }
            }
            s_it = m;
            s_go = go;
            t_cur = t_next;
            if (go && t_next < ps.total) t_next = atomicAdd(ps.tick, 1);   // used by the next item
        }
        __syncthreads();
        if (!s_go) break;
        const MDItem m = s_it;
        const QuadGeom &g = pl.q[m.q];
        const int v = m.v0 + 4 * tid;
        if (v < g.V) {
            A acc[4][C];
            merge_down_entry<P, C, 4, ENV>(pl, m.q, m.n, m.x, m.ip, v, acc);
            const RLevel<P, C> Rn(pl, m.q, m.n);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A o[4] = {acc[0][c], acc[1][c], acc[2][c], acc[3][c]};
                Rn.store4(m.x, m.ip, c, v, o);
            }
        }
        __syncthreads();   // the item's stores are issued; s_it may be rewritten
        if (tid == 0 && ps.deps) {
            pend[npend++] = ps.cbase[m.q][m.n] + m.x;
            if (npend == kPTPub) publish();
        }
    }
    if (tid == 0) publish();
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int sm_count() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        cached[dev] = n;
    }
    return cached[dev];
}

// Control block: ticket (bytes 0 .. 3), the context's status word (bytes
// 8 .. 11), then one counter per column of R_1 .. R_{N-1} of every frame.
size_t persist_ctl_bytes(const Plan &pl) {
    long long n = 0;
    for (int q = 0; q < 4; ++q)
        for (int lv = 1; lv < pl.q[q].N; ++lv) n += pl.q[q].Un[lv];
    return 16 + 4 * (size_t)n;
}

template <int P, int C, bool ENV>
static cudaError_t launch_pd(const Plan &pl, const PSched &ps, cudaStream_t st) {
    const int sms = sm_count();
    if (sms <= 0) return cudaErrorInvalidDevice;
    static int per_sm = 0;   // resident CTAs per SM (the same on every device of this architecture)
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_merge_down_persist<P, C, ENV>,
                                                                      kPTThreads, 0);
        if (e != cudaSuccess || per_sm <= 0) per_sm = 1;
    }
    k_merge_down_persist<P, C, ENV><<<sms * per_sm, kPTThreads, 0, st>>>(pl, ps);
    return cudaGetLastError();
}

template <int P, int C>
static cudaError_t pd_dispatch(const Plan &pl, const PSched &ps, cudaStream_t st) {
    if (plan_has_env(pl)) return launch_pd<P, C, true>(pl, ps, st);
    return launch_pd<P, C, false>(pl, ps, st);
}

template <int P>
static cudaError_t pd_prec(const Plan &pl, const PSched &ps, cudaStream_t st) {
    switch (pl.C) {
    case 1: return pd_dispatch<P, 1>(pl, ps, st);
    case 2: return pd_dispatch<P, 2>(pl, ps, st);
    case 3: return pd_dispatch<P, 3>(pl, ps, st);
    default: return pd_dispatch<P, 4>(pl, ps, st);
    }
}

bool persist_down_usable(const Plan &pl) { return pl.pctl != nullptr && pl.prec != P_FP64 && sm_count() > 0; }

// Merge down R_{n_hi} .. R_{n_lo} of the frames in qm in one launch, after
// resetting the ticket and the column counters; n_hi > n_lo makes the launch
// wait on its own counters between levels.
cudaError_t launch_merge_down_persist(const Plan &pl, int qm, int n_hi, int n_lo, cudaStream_t st, int *launches,
                                      Recorder *rec, double bytes) {
    if (n_hi < n_lo || n_lo < 1) return cudaSuccess;
    PSched ps;
    std::memset(&ps, 0, sizeof(ps));
    ps.nlev = n_hi - n_lo + 1;
    ps.n_hi = n_hi;
    ps.deps = ps.nlev > 1 ? 1 : 0;
    for (int q = 0; q < 4; ++q) ps.nvb[q] = (pl.q[q].V + kPV - 1) / kPV;
    long long acc = 0;
    for (int l = 0; l < ps.nlev; ++l) {
        const int n = n_hi - l;
        ps.lstart[l] = (int)acc;
        for (int q = 0; q < 4; ++q) {
            ps.qstart[l][q] = (int)acc;
            const QuadGeom &g = pl.q[q];
            if (((qm >> q) & 1) && n < g.N) acc += (long long)(g.Un[n] - 1) * (1LL << n) * ps.nvb[q];
        }
    }
    if (acc >= (1LL << 30)) return cudaErrorInvalidValue;   // tickets are 32-bit
    ps.lstart[ps.nlev] = (int)acc;
    ps.total = (int)acc;
    if (acc == 0) return cudaSuccess;
    int ci = 0;
    for (int q = 0; q < 4; ++q)
        for (int n = 1; n < pl.q[q].N; ++n) {
            ps.cbase[q][n] = ci;
            ci += pl.q[q].Un[n];
        }
    if ((size_t)pl.pctl_bytes < 16 + 4 * (size_t)ci) return cudaErrorInvalidValue;
    ps.tick = reinterpret_cast<int *>(pl.pctl);
    ps.cnt = reinterpret_cast<int *>(pl.pctl + 16);
    // reset the ticket and the counters (bytes 8 .. 11 hold the context's
    // status word, which hrc_sync reads and clears)
    cudaError_t e = cudaMemsetAsync(pl.pctl, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl.pctl + 16, 0, 4 * (size_t)ci, st);
    if (e != cudaSuccess) return e;
    rec->begin(K_MERGE_DOWN, n_hi, bytes);
    switch (pl.prec) {
    case P_FP32: e = pd_prec<P_FP32>(pl, ps, st); break;
    case P_FP16: e = pd_prec<P_FP16>(pl, ps, st); break;
    case P_BF16: e = pd_prec<P_BF16>(pl, ps, st); break;
    default: e = cudaErrorInvalidValue;
    }
    rec->end();
    ++*launches;
    return e;
}

}  // namespace hrc
