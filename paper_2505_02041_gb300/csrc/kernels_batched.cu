// kernels_batched.cu -- many scenes of uneven size in one persistent launch.
//
// Every step of every scene (trace, each merge-up level, each merge-down
// level, the fluence sum, and for the backward pass every adjoint step) is
// cut into work items of the same shape the standalone kernels use.  Items
// are numbered by tickets in a topological order: stage-major across scenes
// (stage 0 of every scene, then stage 1, ...), so a CTA only ever waits for
// items handed out before its own.  A CTA pops a ticket (one atomicAdd),
// waits until the previous stage of that scene has published all its items
// (a bounded spin on a per-(scene, stage) counter), runs the body and
// publishes.  The wait is bounded: after `spin_limit` polls the CTA records
// HRC_ETIMEOUT in the status word and returns; every CTA checks the status
// before taking a ticket, so a withheld dependency ends the launch with an
// error instead of a hang.
//
// Tickets are taken at run time by resident CTAs only, so a waiting CTA
// waits only for items held by running CTAs: the smallest outstanding
// ticket always has its dependencies satisfied, and the launch cannot
// deadlock whatever the number of resident CTAs.
//
// Memory ordering: a producer's stores are made visible by __threadfence()
// before thread 0 publishes with atomicAdd; a consumer's thread 0 polls with
// an acquire load, fences, and the CTA synchronises before reading.  No SM
// reads a buffer region before its producing stage completed (every stage
// reads only levels of earlier stages), so no stale L1 line can be hit.
#include <algorithm>
#include <cstring>
#include <type_traits>
#include <vector>

#include "bwd_bodies.cuh"
#include "fwd_bodies.cuh"
#include "launch.h"

namespace hrc {

__device__ __forceinline__ int load_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// One work item of a row stage: rows r0 .. r1-1 of v-block vb.  Not inlined,
// so that each stage kind gets its own register allocation and the
// persistent kernel needs only the largest of them.
template <int P, int C, int KIND>
__device__ __noinline__ void item_rows(const Plan *pl, const StageBlock *sb, long long j) {
    const int vb = (int)(j % sb->nvb);
    const long long r0 = (j / sb->nvb) * sb->rpi;
    const long long r1 = r0 + sb->rpi < sb->rows ? r0 + sb->rpi : sb->rows;
    const int n = sb->level;
#pragma unroll 1
    for (long long r = r0; r < r1; ++r) {
        if constexpr (KIND == BK_MERGE_UP) body_merge_up<P, C>(*pl, sb->rs, n, r, vb);
        else if constexpr (KIND == BK_MERGE_DOWN2) body_merge_down<P, C, true>(*pl, sb->rs, n, r, vb);
        else if constexpr (KIND == BK_ADJ_R2) body_adj_R<P, C, 2>(*pl, sb->rs, n, r, vb);
        else if constexpr (KIND == BK_ADJ_R1) body_adj_R<P, C, 1>(*pl, sb->rs, n, r, vb);
        else if constexpr (KIND == BK_ADJ_T2) body_adj_T<P, C, 2>(*pl, sb->rs, n, r, vb);
        else if constexpr (KIND == BK_ADJ_T1) body_adj_T<P, C, 1>(*pl, sb->rs, n, r, vb);
        else body_adj_merge_up<P, C>(*pl, sb->rs, n, r, vb);
    }
}

// One tile item: the fluence (forward) or the reverse of the sum (backward).
template <int P, int C, int KIND, class IN>
__device__ __noinline__ void item_tile(const Plan *pl, const StageBlock *sb, long long j, IN *io, unsigned char *smem) {
    const int bx = (int)(j % sb->nvb), by = (int)(j / sb->nvb);
    if constexpr (KIND == BK_SUM) body_fluence<P, C, IN>(*pl, io, bx, by, smem);
    else body_adj_sum<P, C, IN>(*pl, (const IN *)io, bx, by, smem);
}

// The tile steps (direct trace of T_0..T_2, its adjoint) of every scene in
// one ordinary launch: block b is tile b - off[i] of scene i (off = prefix
// sums of the scenes' tile counts, nx = tiles along x).  KIND 0: trace;
// KIND 1: adjoint trace of quadrant pair `pair`.
template <int P, int C, int KIND>
__global__ void __launch_bounds__(256, KIND == 1 ? 3 : 2) k_batched_tiles(BatchArgs a, const int *__restrict__ off,
                                                       const int *__restrict__ nx, int nscenes, int pair) {
    using IN = typename std::conditional<P == P_FP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int scene_sh;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nscenes - 1;                 // last scene with off <= block
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        scene_sh = lo;
    }
    __syncthreads();
    const int i = scene_sh;
    const int local = (int)blockIdx.x - off[i];
    const int bx = local % nx[i], by = local / nx[i];
    const Plan &pl = a.plans[i];
    const long long eo = a.eoff[i], so = a.soff[i];
    const IN *e = (const IN *)a.e + eo;
    const IN *s = (const IN *)a.s + so;
    if constexpr (KIND == 0)
        body_trace012<P, C>(pl, (const float *)e, (const float *)s, (const double *)e, (const double *)s, 15, bx, by,
                            smem);
    else
        body_adj_trace<P, C, IN>(pl, e, s, (IN *)a.ge + eo, (IN *)a.gs + so, pair, bx, by, smem);
}

// The merge cascade of every scene.  MODE 0: the forward's merge and
// fluence stages; MODE 1: the backward's (the adjoint merges, preceded by the
// forward's merge stages when the levels are recomputed).  The tile steps run
// in k_batched_tiles launches before / after it.
template <int P, int C, int MODE>
__global__ void __launch_bounds__(256, 5) k_batched(BatchArgs a) {
    using IN = typename std::conditional<P == P_FP64, double, float>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long t_sh;
    __shared__ int b_sh, stop_sh;
    for (;;) {
        if (threadIdx.x == 0) {
            stop_sh = *((volatile int *)a.status) != 0;
            t_sh = stop_sh ? a.total : (long long)atomicAdd(a.ticket, 1ULL);
            int b = -1;
            if (t_sh < a.total) {
                // last block with first <= t, between the index entries
                // around t (usually one or two blocks apart)
                const long long c = t_sh >> kTicketChunkShift;
                int lo = a.chunk[c], hi = a.chunk[c + 1];
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (a.blocks[mid].first <= t_sh) lo = mid;
                    else hi = mid - 1;
                }
                b = lo;
                const StageBlock &sb = a.blocks[b];
                if (sb.dep >= 0) {
                    long long polls = 0;
                    while (load_acquire(a.counters + sb.dep) < sb.dep_target) {
                        if (*((volatile int *)a.status) != 0) { stop_sh = 1; break; }
                        if (++polls > a.spin_limit) {
                            atomicExch(a.status, (int)5 /* HRC_ETIMEOUT */);
                            stop_sh = 1;
                            break;
                        }
                        __nanosleep(128);
                    }
                }
                __threadfence();
            }
            b_sh = b;
        }
        __syncthreads();
        const long long t = t_sh;
        if (t >= a.total || stop_sh) break;
        const StageBlock &sb = a.blocks[b_sh];
        const long long j = t - sb.first;
        const Plan *pl = a.plans + sb.scene;
        const long long eo = a.eoff[sb.scene];
        switch (sb.kind) {
        case BK_MERGE_UP: item_rows<P, C, BK_MERGE_UP>(pl, &sb, j); break;
        case BK_MERGE_DOWN2: item_rows<P, C, BK_MERGE_DOWN2>(pl, &sb, j); break;
        default:
            if constexpr (MODE == 0) {       // BK_SUM (with the level-0 merge down)
                item_tile<P, C, BK_SUM, IN>(pl, &sb, j, (IN *)a.F + eo, smem);
            } else {
                switch (sb.kind) {
                case BK_ADJ_SUM: item_tile<P, C, BK_ADJ_SUM, IN>(pl, &sb, j, (IN *)a.gF + eo, smem); break;
                case BK_ADJ_R2: item_rows<P, C, BK_ADJ_R2>(pl, &sb, j); break;
                case BK_ADJ_R1: item_rows<P, C, BK_ADJ_R1>(pl, &sb, j); break;
                case BK_ADJ_T2: item_rows<P, C, BK_ADJ_T2>(pl, &sb, j); break;
                case BK_ADJ_T1: item_rows<P, C, BK_ADJ_T1>(pl, &sb, j); break;
                default: item_rows<P, C, BK_ADJ_MU>(pl, &sb, j); break;
                }
            }
            break;
        }
        __syncthreads();
        if (threadIdx.x == 0 && sb.own != a.withhold) {
            __threadfence();
            atomicAdd(a.counters + sb.own, 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Level-major multi-scene launches: one stage of every scene per launch, so a
// batch of many small scenes becomes a few large launches instead of a long
// chain of small ones per scene.  Every block runs the standalone kernel's
// body on its scene's plan (read from global memory).
// ---------------------------------------------------------------------------
int multi_threads(int kind) {
    switch (kind) {
    case MK_SUM: return 128;
    case MK_ADJ_SUM: return 256;
    case MK_ADJ_R1:
    case MK_ADJ_T1: return 256;
    default: return 128;
    }
}

int multi_vblock(int kind) {
    switch (kind) {
    case MK_MERGE_UP4:
    case MK_MERGE_DOWN4:
    case MK_MERGE_DOWN_BULK: return 4 * 128;   // four v per thread
    case MK_ADJ_R1:
    case MK_ADJ_T1: return 256;            // one v per thread
    default: return 2 * 128;               // a pair of v per thread
    }
}

// The block's entry (binary search) and its scene's plan, copied into
// shared memory: the bodies read the plan's fields in every address
// computation, which then cost a shared-memory load instead of a global one.
__device__ __forceinline__ const MultiEnt &multi_entry(const Plan *__restrict__ plans,
                                                       const MultiEnt *__restrict__ ents, int nent, Plan &spl) {
    __shared__ int ent_sh;
    if (threadIdx.x == 0) {
        int lo = 0, hi = nent - 1;                    // last entry with first <= block
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (ents[mid].first <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        ent_sh = lo;
    }
    __syncthreads();
    const MultiEnt &m = ents[ent_sh];
    static_assert(sizeof(Plan) % 4 == 0, "plan copied as 32-bit words");
    const unsigned *src = reinterpret_cast<const unsigned *>(plans + m.scene);
    unsigned *dst = reinterpret_cast<unsigned *>(&spl);
    for (int i = threadIdx.x; i < (int)(sizeof(Plan) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    return m;
}

template <int P, int C, int KIND>
__global__ void __launch_bounds__(256) k_multi(const Plan *__restrict__ plans, const MultiEnt *__restrict__ ents,
                                               int nent, int n, const long long *__restrict__ eoff, void *io) {
    using IN = typename std::conditional<P == P_FP64, double, float>::type;
    __shared__ __align__(16) unsigned char smem[sizeof(typename Prec<P>::A) * C * 32 * 33];
    __shared__ __align__(16) Plan spl;
    const MultiEnt &m = multi_entry(plans, ents, nent, spl);
    const Plan &pl = spl;
    const int local = (int)blockIdx.x - m.first;
    const int row = local / m.nvb, vb = local - row * m.nvb;
    if constexpr (KIND == MK_MERGE_UP4) body_merge_up4<P, C>(pl, m.rs, n, row, vb);
    else if constexpr (KIND == MK_MERGE_DOWN4) body_merge_down4<P, C, false>(pl, m.rs, n, row, vb);
    else if constexpr (KIND == MK_SUM) body_fluence<P, C, IN, false>(pl, (IN *)io + eoff[m.scene], vb, row, smem);
    else if constexpr (KIND == MK_ADJ_SUM) body_adj_sum<P, C, IN>(pl, (const IN *)io + eoff[m.scene], vb, row, smem);
    else if constexpr (KIND == MK_ADJ_R2) body_adj_R<P, C, 2>(pl, m.rs, n, row, vb);
    else if constexpr (KIND == MK_ADJ_R1) body_adj_R<P, C, 1>(pl, m.rs, n, row, vb);
    else if constexpr (KIND == MK_ADJ_T2) body_adj_T<P, C, 2, false>(pl, m.rs, n, row, vb);
    else if constexpr (KIND == MK_ADJ_T1) body_adj_T<P, C, 1, false>(pl, m.rs, n, row, vb);
    else body_adj_merge_up<P, C, false>(pl, m.rs, n, row, vb);
}

// The merge down with the block's rows staged by bulk copies (the 16-bit
// precisions' faster form).
template <int P, int C>
__global__ void __launch_bounds__(128) k_multi_bulk(const Plan *__restrict__ plans, const MultiEnt *__restrict__ ents,
                                                    int nent, int n) {
    extern __shared__ __align__(128) unsigned char dsmem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) Plan spl;
    const MultiEnt &m = multi_entry(plans, ents, nent, spl);
    const int local = (int)blockIdx.x - m.first;
    const int row = local / m.nvb, vb = local - row * m.nvb;
    body_merge_down_bulk<P, C, false>(spl, m.rs, n, row, vb, dsmem, bar);
}

template <int P, int C>
static cudaError_t multi_impl(int kind, const Plan *plans, const MultiEnt *ents, int nent, int n, int blocks,
                              const long long *eoff, void *io, cudaStream_t st) {
    const int t = multi_threads(kind);
    if (kind == MK_MERGE_DOWN_BULK) {
        if constexpr (P == P_FP64) {
            return cudaErrorInvalidValue;
        } else {
            const size_t smem = BulkMD<P, C>::bytes();
            cudaError_t e = cudaFuncSetAttribute(k_multi_bulk<P, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            k_multi_bulk<P, C><<<blocks, 128, smem, st>>>(plans, ents, nent, n);
            return cudaGetLastError();
        }
    }
    switch (kind) {
    case MK_MERGE_UP4: k_multi<P, C, MK_MERGE_UP4><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_MERGE_DOWN4: k_multi<P, C, MK_MERGE_DOWN4><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_SUM: k_multi<P, C, MK_SUM><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_ADJ_SUM: k_multi<P, C, MK_ADJ_SUM><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_ADJ_R2: k_multi<P, C, MK_ADJ_R2><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_ADJ_R1: k_multi<P, C, MK_ADJ_R1><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_ADJ_T2: k_multi<P, C, MK_ADJ_T2><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    case MK_ADJ_T1: k_multi<P, C, MK_ADJ_T1><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    default: k_multi<P, C, MK_ADJ_MU><<<blocks, t, 0, st>>>(plans, ents, nent, n, eoff, io); break;
    }
    return cudaGetLastError();
}

template <int P>
static cudaError_t multi_prec(int C, int kind, const Plan *plans, const MultiEnt *ents, int nent, int n, int blocks,
                              const long long *eoff, void *io, cudaStream_t st) {
    switch (C) {
    case 1: return multi_impl<P, 1>(kind, plans, ents, nent, n, blocks, eoff, io, st);
    case 2: return multi_impl<P, 2>(kind, plans, ents, nent, n, blocks, eoff, io, st);
    case 3: return multi_impl<P, 3>(kind, plans, ents, nent, n, blocks, eoff, io, st);
    default: return multi_impl<P, 4>(kind, plans, ents, nent, n, blocks, eoff, io, st);
    }
}

cudaError_t launch_multi(int prec, int C, int kind, const Plan *plans, const MultiEnt *ents, int nent, int n,
                         int blocks, const long long *eoff, void *io, cudaStream_t st) {
    if (blocks <= 0 || nent <= 0) return cudaSuccess;
    switch (prec) {
    case P_FP32: return multi_prec<P_FP32>(C, kind, plans, ents, nent, n, blocks, eoff, io, st);
    case P_FP16: return multi_prec<P_FP16>(C, kind, plans, ents, nent, n, blocks, eoff, io, st);
    case P_BF16: return multi_prec<P_BF16>(C, kind, plans, ents, nent, n, blocks, eoff, io, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------
// Host: the stage list of one scene (same work decomposition as the
// standalone launch sequences, with 256-thread blocks: paired-v bodies cover
// 512 v per block, single-v bodies 256).
// ---------------------------------------------------------------------------
namespace {

RowSplit rows_for(const Plan &pl, int kind, int n) {
    RowSplit rs;
    long long acc = 0;
    for (int q = 0; q < 4; ++q) {
        rs.start[q] = acc;
        const QuadGeom &g = pl.q[q];
        long long rows = 0;
        switch (kind) {
        case BK_MERGE_UP: rows = (n >= 3 && n <= g.N) ? (long long)(g.Un[n] - 1) * ((1 << n) + 1) : 0; break;
        case BK_MERGE_DOWN2: rows = n < g.N ? (long long)(g.Un[n] - 1) * (1 << n) : 0; break;
        case BK_ADJ_R2:
        case BK_ADJ_R1: rows = (n + 1 < g.N) ? (long long)(g.Un[n + 1] - 1) * (2 << n) : 0; break;
        case BK_ADJ_T2:
        case BK_ADJ_T1:   // level 0: odd columns only
            rows = (g.N >= 1 && n <= g.N && !adj_T_fused(n, g.N))
                       ? (n == 0 ? (long long)(g.Un[0] / 2) * 2 : (long long)(g.Un[n] - 1) * ((1 << n) + 1)) : 0;
            break;
        case BK_ADJ_MU: rows = (n >= 3 && n <= g.N) ? (long long)(g.Un[n - 1] - 1) * ((1 << (n - 1)) + 1) : 0; break;
        default: break;
        }
        acc += rows;
    }
    rs.start[4] = acc;
    return rs;
}

}  // namespace

void batched_stages(const Plan &pl, int mode, std::vector<StageDesc> &out) {
    out.clear();
    int Nmax = 0, Vmax = 0;
    for (int q = 0; q < 4; ++q) {
        Nmax = pl.q[q].N > Nmax ? pl.q[q].N : Nmax;
        Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    }
    const int tx = (pl.W + 31) / 32, ty = (pl.H + 31) / 32;
    const int vb2 = (Vmax + 511) / 512, vb1 = (Vmax + 255) / 256;
    const double esz = pl.prec == P_FP64 ? 8.0 : 4.0, img = double(pl.W) * pl.H;
    // rows per item: about 4096 entries of work per item, so that the
    // ticket, dependency poll and publish of an item are amortised
    auto rowstage = [&](int kind, int n, int nvb, double bytes) {
        StageDesc d;
        d.kind = kind;
        d.level = n;
        d.rs = rows_for(pl, kind, n);
        d.nvb = nvb;
        d.rows = d.rs.start[4];
        const int per_row = (kind == BK_ADJ_R1 || kind == BK_ADJ_T1) ? 256 : 512;
        d.rpi = 4096 / per_row;
        d.count = (int)((d.rows + d.rpi - 1) / d.rpi * nvb);
        d.bytes = bytes;
        if (d.count > 0) out.push_back(d);
    };
    auto tilestage = [&](int kind, int nx, int ny, double bytes, int level = 0) {
        StageDesc d;
        d.kind = kind;
        d.level = level;
        std::memset(&d.rs, 0, sizeof(d.rs));
        d.nvb = nx;
        d.rows = ny;
        d.rpi = 1;
        d.count = nx * ny;
        d.bytes = bytes;
        out.push_back(d);
    };
    double by = 0;
    if (mode != 1) {   // mode 1 reads the levels the forward left in the buffers
        by = img * (pl.C + 1) * esz;
        for (int q = 0; q < 4; ++q)
            for (int n = 0; n <= 2; ++n) by += bytes_T(pl, q, n);
        tilestage(BK_TRACE, tx, ty, by);
        for (int n = 3; n <= Nmax; ++n) {
            by = 0;
            for (int q = 0; q < 4; ++q)
                if (n <= pl.q[q].N) by += bytes_T(pl, q, n - 1) + bytes_T(pl, q, n);
            rowstage(BK_MERGE_UP, n, vb2, by);
        }
        for (int n = Nmax - 1; n >= 1; --n) {   // level 0 inside the fluence stage
            by = 0;
            for (int q = 0; q < 4; ++q) {
                const QuadGeom &g = pl.q[q];
                if (n >= g.N) continue;
                by += bytes_T_odd(pl, q, n);
                by += bytes_T_even_dirs(pl, q, n + 1);
                by += bytes_R(pl, q, n + 1) + bytes_R(pl, q, n);
            }
            rowstage(BK_MERGE_DOWN2, n, vb2, by);
        }
        if (mode == 0) {
            by = img * pl.C * esz;
            for (int q = 0; q < 4; ++q) {
                if (pl.q[q].N < 1) continue;
                by += bytes_T_odd(pl, q, 0) + bytes_R(pl, q, 1) + bytes_T_even_dirs(pl, q, 1);
            }
            tilestage(BK_SUM, tx, ty, by);   // 32 x 32 tiles, as the standalone kernel
            return;
        }
    }
    const double ab = 4.0;   // adjoint buffers are fp32 in the batched precisions
    auto gT = [&](int q, int n) {
        const QuadGeom &g = pl.q[q];
        return (n < 0 || n > g.N) ? 0.0 : double(t_live_rows(n, g.Un[n])) * g.V * (pl.C + 1) * ab;
    };
    auto gR = [&](int q, int n) {
        const QuadGeom &g = pl.q[q];
        return (n < 0 || n >= g.N) ? 0.0 : double(g.Un[n] - 1) * (1 << n) * g.V * pl.C * ab;
    };
    by = img * pl.C * esz;
    for (int q = 0; q < 4; ++q) by += gR(q, 0);
    tilestage(BK_ADJ_SUM, tx, ty, by);
    for (int n = 0; n + 1 < Nmax; ++n) {
        by = 0;
        for (int q = 0; q < 4; ++q)
            if (n + 1 < pl.q[q].N) by += gR(q, n) + gR(q, n + 1);
        rowstage(n >= 1 ? BK_ADJ_R2 : BK_ADJ_R1, n, n >= 1 ? vb2 : vb1, by);
    }
    for (int n = 0; n <= Nmax; ++n) {
        by = 0;
        for (int q = 0; q < 4; ++q)
            if (pl.q[q].N >= 1 && n <= pl.q[q].N && !adj_T_fused(n, pl.q[q].N))
                by += gT(q, n) + gR(q, n) + gR(q, n - 1) + bytes_R(pl, q, n) + bytes_R(pl, q, n + 1);
        rowstage(n >= 1 ? BK_ADJ_T2 : BK_ADJ_T1, n, n >= 1 ? vb2 : vb1, by);
    }
    for (int n = Nmax; n >= 3; --n) {
        by = 0;
        for (int q = 0; q < 4; ++q)
            if (n <= pl.q[q].N)
                by += gT(q, n - 1) + gT(q, n) + bytes_T(pl, q, n - 1) + gR(q, n - 1) + gR(q, n - 2) +
                      bytes_R(pl, q, n - 1) + bytes_R(pl, q, n);
        rowstage(BK_ADJ_MU, n, vb2, by);
    }
    for (int pair = 0; pair < 2; ++pair) {
        double bt = img * (pl.C + 1) * esz * (pair == 0 ? 1.0 : 2.0);
        for (int q = 2 * pair; q < 2 * pair + 2; ++q)
            for (int n = 0; n <= 2; ++n) bt += gT(q, n);
        tilestage(BK_ADJ_TRACE, pair_tiles_x(pair, pl.W), pair_tiles_y(pair, pl.H), bt, pair);
    }
}

void multi_stages(const std::vector<Plan> &plans, int mode, std::vector<MultiDesc> &out) {
    out.clear();
    const int ns = (int)plans.size();
    const bool bulk = ns > 0 && (plans[0].prec == P_FP16 || plans[0].prec == P_BF16);
    std::vector<std::vector<StageDesc>> st(ns);
    int Nmax = 0;
    for (int i = 0; i < ns; ++i) {
        batched_stages(plans[i], mode, st[i]);
        Nmax = std::max(Nmax, plan_nmax(plans[i]));
    }
    auto mk = [](int bk) {
        switch (bk) {
        case BK_MERGE_UP: return (int)MK_MERGE_UP4;
        case BK_MERGE_DOWN2: return (int)MK_MERGE_DOWN4;   // bulk form chosen below
        case BK_SUM: return (int)MK_SUM;
        case BK_ADJ_SUM: return (int)MK_ADJ_SUM;
        case BK_ADJ_R2: return (int)MK_ADJ_R2;
        case BK_ADJ_R1: return (int)MK_ADJ_R1;
        case BK_ADJ_T2: return (int)MK_ADJ_T2;
        case BK_ADJ_T1: return (int)MK_ADJ_T1;
        case BK_ADJ_MU: return (int)MK_ADJ_MU;
        default: return -1;
        }
    };
    // the launches in dependency order: (multi kind, level)
    std::vector<std::pair<int, int>> keys;
    if (mode != 1) {
        for (int n = 3; n <= Nmax; ++n) keys.push_back({MK_MERGE_UP4, n});
        for (int n = Nmax - 1; n >= 1; --n) keys.push_back({MK_MERGE_DOWN4, n});   // (bulk in 16-bit)
        if (mode == 0) keys.push_back({MK_SUM, 0});
    }
    if (mode != 0) {
        keys.push_back({MK_ADJ_SUM, 0});
        keys.push_back({MK_ADJ_R1, 0});
        for (int n = 1; n + 1 < Nmax; ++n) keys.push_back({MK_ADJ_R2, n});
        keys.push_back({MK_ADJ_T1, 0});
        for (int n = 1; n <= Nmax; ++n) keys.push_back({MK_ADJ_T2, n});
        for (int n = Nmax; n >= 3; --n) keys.push_back({MK_ADJ_MU, n});
    }
    for (const auto &key : keys) {
        MultiDesc d;
        d.kind = key.first;
        d.level = key.second;
        d.blocks = 0;
        d.bytes = 0;
        for (int i = 0; i < ns; ++i)
            for (const StageDesc &sd : st[i]) {
                if (mk(sd.kind) != d.kind || sd.level != d.level) continue;
                MultiEnt m;
                std::memset(&m, 0, sizeof(m));
                m.first = d.blocks;
                m.scene = i;
                m.rs = sd.rs;
                long long rows;
                if (d.kind == MK_SUM || d.kind == MK_ADJ_SUM) {
                    m.nvb = sd.nvb;           // tiles along x
                    rows = sd.rows;           // tiles along y
                } else {
                    int Vmax = 0;
                    for (int q = 0; q < 4; ++q) Vmax = std::max(Vmax, plans[i].q[q].V);
                    m.nvb = (Vmax + multi_vblock(d.kind) - 1) / multi_vblock(d.kind);
                    rows = sd.rs.start[4];
                }
                if (rows <= 0) continue;
                d.ents.push_back(m);
                d.blocks += (int)(rows * m.nvb);
                d.bytes += sd.bytes;
            }
        if (d.kind == MK_MERGE_DOWN4 && bulk) d.kind = MK_MERGE_DOWN_BULK;
        if (d.blocks > 0) out.push_back(d);
    }
}

// Dynamic shared memory of the persistent launch: the fluence tile (forward)
// or the transposed dL/dF tile (backward), both C x 32 x 33 words.
template <int P, int C> size_t batched_smem(int) { return fluence_smem<P, C>(); }

template <int P, int C, int MODE>
static cudaError_t batched_launch(const BatchArgs &a, int blocks_per_sm, cudaStream_t st) {
    const size_t smem = batched_smem<P, C>(MODE);
    cudaError_t e = cudaFuncSetAttribute(k_batched<P, C, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched<P, C, MODE>, 256, smem);
    if (e != cudaSuccess) return e;
    if (occ < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = blocks_per_sm > 0 && blocks_per_sm < occ ? blocks_per_sm : occ;
    long long grid = (long long)sms * per_sm;
    if (grid > a.total) grid = a.total;
    if (grid < 1) grid = 1;
    k_batched<P, C, MODE><<<(unsigned)grid, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <int P, int C>
static cudaError_t batched_impl(const BatchArgs &a, int blocks_per_sm, int mode, cudaStream_t st) {
    return mode == 0 ? batched_launch<P, C, 0>(a, blocks_per_sm, st) : batched_launch<P, C, 1>(a, blocks_per_sm, st);
}

template <int P>
static cudaError_t batched_prec(const BatchArgs &a, int C, int bpsm, int mode, cudaStream_t st) {
    switch (C) {
    case 1: return batched_impl<P, 1>(a, bpsm, mode, st);
    case 2: return batched_impl<P, 2>(a, bpsm, mode, st);
    case 3: return batched_impl<P, 3>(a, bpsm, mode, st);
    default: return batched_impl<P, 4>(a, bpsm, mode, st);
    }
}

cudaError_t launch_batched(const BatchArgs &a, int prec, int C, int blocks_per_sm, int mode, cudaStream_t st) {
    switch (prec) {
    case P_FP32: return batched_prec<P_FP32>(a, C, blocks_per_sm, mode, st);
    case P_FP16: return batched_prec<P_FP16>(a, C, blocks_per_sm, mode, st);
    case P_BF16: return batched_prec<P_BF16>(a, C, blocks_per_sm, mode, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int P, int C, int KIND>
static cudaError_t tiles_launch(const BatchArgs &a, const int *off, const int *nx, int nscenes, int pair, int total,
                                cudaStream_t st) {
    using A = typename Prec<P>::A;
    const size_t smem = KIND == 0 ? TraceTile<A, C>::bytes() : adj_trace_smem<A, C>();
    cudaError_t e = cudaFuncSetAttribute(k_batched_tiles<P, C, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_batched_tiles<P, C, KIND><<<(unsigned)total, 256, smem, st>>>(a, off, nx, nscenes, pair);
    return cudaGetLastError();
}

template <int P, int C>
static cudaError_t tiles_impl(const BatchArgs &a, int kind, const int *off, const int *nx, int nscenes, int pair,
                              int total, cudaStream_t st) {
    return kind == BK_TRACE ? tiles_launch<P, C, 0>(a, off, nx, nscenes, pair, total, st)
                            : tiles_launch<P, C, 1>(a, off, nx, nscenes, pair, total, st);
}

template <int P>
static cudaError_t tiles_prec(const BatchArgs &a, int C, int kind, const int *off, const int *nx, int nscenes,
                              int pair, int total, cudaStream_t st) {
    switch (C) {
    case 1: return tiles_impl<P, 1>(a, kind, off, nx, nscenes, pair, total, st);
    case 2: return tiles_impl<P, 2>(a, kind, off, nx, nscenes, pair, total, st);
    case 3: return tiles_impl<P, 3>(a, kind, off, nx, nscenes, pair, total, st);
    default: return tiles_impl<P, 4>(a, kind, off, nx, nscenes, pair, total, st);
    }
}

cudaError_t launch_batched_tiles(const BatchArgs &a, int prec, int C, int kind, const int *off, const int *nx,
                                 int nscenes, int pair, int total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    switch (prec) {
    case P_FP32: return tiles_prec<P_FP32>(a, C, kind, off, nx, nscenes, pair, total, st);
    case P_FP16: return tiles_prec<P_FP16>(a, C, kind, off, nx, nscenes, pair, total, st);
    case P_BF16: return tiles_prec<P_BF16>(a, C, kind, off, nx, nscenes, pair, total, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hrc
