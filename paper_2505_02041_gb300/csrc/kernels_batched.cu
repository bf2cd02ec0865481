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

// One item of an adjoint stage (backward launches only).
template <int P, int C, class IN>
__device__ __forceinline__ void batched_adjoint_item(const BatchArgs &a, const StageBlock &sb, const Plan &pl,
                                                     long long j, int vb, long long r0, long long r1, long long eo,
                                                     long long so, const IN *e, const IN *s, unsigned char *smem) {
    switch (sb.kind) {
    case BK_ADJ_SUM:
        body_adj_sum<P, C, IN>(pl, (const IN *)a.gF + eo, vb, (int)(j / sb.nvb), smem);
        break;
    case BK_ADJ_R2:
        for (long long r = r0; r < r1; ++r) body_adj_R<P, C, 2>(pl, sb.rs, sb.level, r, vb);
        break;
    case BK_ADJ_R1:
        for (long long r = r0; r < r1; ++r) body_adj_R<P, C, 1>(pl, sb.rs, sb.level, r, vb);
        break;
    case BK_ADJ_T2:
        for (long long r = r0; r < r1; ++r) body_adj_T<P, C, 2>(pl, sb.rs, sb.level, r, vb);
        break;
    case BK_ADJ_T1:
        for (long long r = r0; r < r1; ++r) body_adj_T<P, C, 1>(pl, sb.rs, sb.level, r, vb);
        break;
    case BK_ADJ_MU:
        for (long long r = r0; r < r1; ++r) body_adj_merge_up<P, C>(pl, sb.rs, sb.level, r, vb);
        break;
    default:   // BK_ADJ_TRACE
        body_adj_trace<P, C, IN>(pl, e, s, (IN *)a.ge + eo, (IN *)a.gs + so, sb.level, vb, (int)(j / sb.nvb), smem);
        break;
    }
}

// MODE 0: the forward stages; MODE 1: the stages of the backward (the
// adjoint, preceded by the forward's level stages when they are recomputed).
template <int P, int C, int MODE>
__global__ void __launch_bounds__(256, 3) k_batched(BatchArgs a) {
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
                int lo = 0, hi = a.nblocks - 1;          // last block with first <= t
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
        const Plan &pl = a.plans[sb.scene];
        const long long eo = a.eoff[sb.scene], so = a.soff[sb.scene];
        const IN *e = (const IN *)a.e + eo;
        const IN *s = (const IN *)a.s + so;
        // row kinds: rows r0 .. r1-1 of v-block vb; tile kinds: one tile
        const int vb = (int)(j % sb.nvb);
        const long long r0 = (j / sb.nvb) * sb.rpi;
        const long long r1 = r0 + sb.rpi < sb.rows ? r0 + sb.rpi : sb.rows;
        if (MODE == 0 || sb.kind <= BK_MERGE_DOWN2) {   // forward stages (mode 2 recomputes them)
            switch (sb.kind) {
            case BK_TRACE:
                body_trace012<P, C>(pl, (const float *)e, (const float *)s, (const double *)e, (const double *)s, 15,
                                    vb, (int)(j / sb.nvb), smem);
                break;
            case BK_MERGE_UP:
                for (long long r = r0; r < r1; ++r) body_merge_up<P, C>(pl, sb.rs, sb.level, r, vb);
                break;
            case BK_MERGE_DOWN2:
                for (long long r = r0; r < r1; ++r) body_merge_down<P, C, true>(pl, sb.rs, sb.level, r, vb);
                break;
            default:   // BK_SUM (with the level-0 merge down); forward launches only
                if constexpr (MODE == 0) body_fluence<P, C, IN>(pl, (IN *)a.F + eo, vb, (int)(j / sb.nvb), smem);
                break;
            }
        } else if constexpr (MODE == 1) {
            batched_adjoint_item<P, C, IN>(a, sb, pl, j, vb, r0, r1, eo, so, e, s, smem);
        }
        __syncthreads();
        if (threadIdx.x == 0 && sb.own != a.withhold) {
            __threadfence();
            atomicAdd(a.counters + sb.own, 1);
        }
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

// Dynamic shared memory of a launch: the forward needs the trace tile, the
// backward the adjoint-trace tile and the transposed dL/dF tile.
template <int P, int C> size_t batched_smem(int mode) {
    using A = typename Prec<P>::A;
    const size_t tr = TraceTile<A, C>::bytes();
    if (mode == 0) return tr > fluence_smem<P, C>() ? tr : fluence_smem<P, C>();
    size_t m = adj_trace_smem<A, C>();
    const size_t sum_tile = sizeof(A) * C * 32 * 33;
    m = m > sum_tile ? m : sum_tile;
    return m > tr ? m : tr;   // the recomputing backward runs the trace stage too
}

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

}  // namespace hrc
