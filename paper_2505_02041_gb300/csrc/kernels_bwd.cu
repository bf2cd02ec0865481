// kernels_bwd.cu -- adjoint HRC kernels for sm_103a (standalone launches of
// the bodies in bwd_bodies.cuh) and the backward launch sequence.
#include <type_traits>

#include <cstring>

#include "bwd_bodies.cuh"
#include "launch.h"

namespace hrc {

template <int P, int C, class GIN>
__global__ void __launch_bounds__(256) k_adj_sum(Plan pl, const GIN *__restrict__ gF) {
    __shared__ __align__(16) unsigned char smem[sizeof(typename Prec<P>::A) * C * 32 * 33];
    body_adj_sum<P, C, GIN>(pl, gF, blockIdx.x, blockIdx.y, smem);
}

// Row and v-block of this block (see the forward merge kernels).
__device__ __forceinline__ void row_block_b(const Plan &pl, long long &row, int &vb) {
    if (pl.vmajor) { row = blockIdx.y; vb = blockIdx.x; }
    else { row = blockIdx.x; vb = blockIdx.y; }
}

template <int P, int C, int E>
__global__ void __launch_bounds__(512) k_adj_R(Plan pl, RowSplitB rs, int n) {
    long long row;
    int vb;
    row_block_b(pl, row, vb);
    body_adj_R<P, C, E>(pl, rs, n, row, vb);
}

template <int P, int C, int E, bool ENV>
__global__ void __launch_bounds__(512) k_adj_T(Plan pl, RowSplitB rs, int n) {
    long long row;
    int vb;
    row_block_b(pl, row, vb);
    body_adj_T<P, C, E, ENV>(pl, rs, n, row, vb);
}

template <int P, int C, bool ENV>
__global__ void __launch_bounds__(512) k_adj_merge_up(Plan pl, RowSplitB rs, int n) {
    long long row;
    int vb;
    row_block_b(pl, row, vb);
    body_adj_merge_up<P, C, ENV>(pl, rs, n, row, vb);
}

template <int P, int C, class IN>
__global__ void __launch_bounds__(ADJ_THREADS, 3) k_adj_trace(Plan pl, const IN *__restrict__ e, const IN *__restrict__ s,
                                                   IN *__restrict__ ge, IN *__restrict__ gs, int pair,
                                                   const __grid_constant__ CUtensorMap tme,
                                                   const __grid_constant__ CUtensorMap tms, int use_tma) {
    extern __shared__ __align__(128) unsigned char tb_smem[];
    body_adj_trace<P, C, IN>(pl, e, s, ge, gs, pair, blockIdx.x, blockIdx.y, tb_smem, use_tma ? &tme : nullptr,
                             use_tma ? &tms : nullptr);
}

// ---------------------------------------------------------------------------
// Host-side launcher of the whole backward pass.
// ---------------------------------------------------------------------------
namespace {

RowSplitB split_rows(const Plan &pl, int kind, int n) {
    // kind 0: R_0 rows (q, x); 1: rows of gR_{n+1} (q, x', j); 2: rows of gT_n (q, x, k);
    // 3: rows of gT_{n-1} for the level-n merge-up reverse
    RowSplitB rs;
    long long acc = 0;
    for (int q = 0; q < 4; ++q) {
        rs.start[q] = acc;
        const QuadGeom &g = pl.q[q];
        long long rows = 0;
        if (kind == 0) rows = g.N >= 1 ? g.Un[0] : 0;
        else if (kind == 1) rows = (n + 1 < g.N) ? (long long)(g.Un[n + 1] - 1) * (2 << n) : 0;
        else if (kind == 2)   // level 0: odd columns only
            rows = (g.N >= 1 && n <= g.N && !adj_T_fused(n, g.N))
                       ? (n == 0 ? (long long)(g.Un[0] / 2) * 2 : (long long)(g.Un[n] - 1) * ((1 << n) + 1)) : 0;
        else rows = (n >= 3 && n <= g.N) ? (long long)(g.Un[n - 1] - 1) * ((1 << (n - 1)) + 1) : 0;
        acc += rows;
    }
    rs.start[4] = acc;
    return rs;
}

dim3 row_grid_b(const Plan &pl, long long rows, int per_block) {
    int Vmax = 0;
    for (int q = 0; q < 4; ++q) Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    const unsigned vb = (unsigned)((Vmax + per_block - 1) / per_block);
    return pl.vmajor ? dim3(vb, (unsigned)rows) : dim3((unsigned)rows, vb);
}

int vblocks_b(const Plan &pl, int bs) {
    int Vmax = 0;
    for (int q = 0; q < 4; ++q) Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    return (Vmax + bs - 1) / bs;
}

}  // namespace

template <int P, int C>
static cudaError_t bwd_impl(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, bool recompute, cudaStream_t st, int *launches, Recorder *rec) {
    using IN = typename std::conditional<P == P_FP64, double, float>::type;
    const int mt = pl.mthreads, ts = 2 * mt > 512 ? 512 : 2 * mt;   // paired-v / single-v block sizes
    const bool env = plan_has_env(pl);   // kernels compiled for an environment map
    int Nmax = 0;
    for (int q = 0; q < 4; ++q) Nmax = pl.q[q].N > Nmax ? pl.q[q].N : Nmax;
    const double ab = P == P_FP64 ? 8.0 : 4.0;
    const double img = double(pl.W) * pl.H;
    // live columns x >= 1 only (column 0 is dead)
    auto gTbytes = [&](int q, int n) {
        const QuadGeom &g = pl.q[q];
        return (n < 0 || n > g.N) ? 0.0 : double(t_live_rows(n, g.Un[n])) * g.V * (pl.C + 1) * ab;
    };
    auto gRbytes = [&](int q, int n) {
        const QuadGeom &g = pl.q[q];
        return (n < 0 || n >= g.N) ? 0.0 : double(g.Un[n] - 1) * (1 << n) * g.V * pl.C * ab;
    };
    // T_0..T_N and R_1..R_{N-1}: recomputed from (e, s), or the ones the last
    // forward left in the plan's buffers (the inputs unchanged since, by
    // contract).
    if (recompute) {
        cudaError_t err = launch_forward(pl, rt, e, s, nullptr, st, launches, rec);
        if (err != cudaSuccess) return err;
    }
    {
        double by = img * pl.C * ab;
        for (int q = 0; q < 4; ++q) by += gRbytes(q, 0);
        rec->begin(K_ADJ_SUM, 0, by);
        k_adj_sum<P, C, IN><<<dim3((pl.W + 31) / 32, (pl.H + 31) / 32), 256, 0, st>>>(pl, (const IN *)gF);
        rec->end();
        ++*launches;
    }
    for (int n = 0; n + 1 < Nmax; ++n) {
        RowSplitB rs = split_rows(pl, 1, n);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q)
            if (n + 1 < pl.q[q].N)
                by += gRbytes(q, n) + gRbytes(q, n + 1) + bytes_T(pl, q, n) / (pl.C + 1) / 2 +
                      bytes_T(pl, q, n + 1) / (pl.C + 1) / 2;
        rec->begin(K_ADJ_MERGE_DOWN, n, by);
        if (n >= 1) k_adj_R<P, C, 2><<<row_grid_b(pl, rs.start[4], 2 * mt), mt, 0, st>>>(pl, rs, n);
        else k_adj_R<P, C, 1><<<row_grid_b(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    for (int n = 0; n <= Nmax; ++n) {
        RowSplitB rs = split_rows(pl, 2, n);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q)
            if (pl.q[q].N >= 1 && n <= pl.q[q].N && !adj_T_fused(n, pl.q[q].N))
                by += gTbytes(q, n) + gRbytes(q, n) + gRbytes(q, n - 1) + bytes_R(pl, q, n) + bytes_R(pl, q, n + 1);
        rec->begin(K_ADJ_MERGE_DOWN, n, by);
        if (n >= 1) {
            if (env) k_adj_T<P, C, 2, true><<<row_grid_b(pl, rs.start[4], 2 * mt), mt, 0, st>>>(pl, rs, n);
            else k_adj_T<P, C, 2, false><<<row_grid_b(pl, rs.start[4], 2 * mt), mt, 0, st>>>(pl, rs, n);
        } else {
            if (env) k_adj_T<P, C, 1, true><<<row_grid_b(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, n);
            else k_adj_T<P, C, 1, false><<<row_grid_b(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, n);
        }
        rec->end();
        ++*launches;
    }
    for (int n = Nmax; n >= 3; --n) {
        RowSplitB rs = split_rows(pl, 3, n);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q)
            if (n <= pl.q[q].N)   // merge-up reverse + the fused merge-down part of level n-1
                by += gTbytes(q, n - 1) + gTbytes(q, n) + bytes_T(pl, q, n - 1) + gRbytes(q, n - 1) +
                      gRbytes(q, n - 2) + bytes_R(pl, q, n - 1) + bytes_R(pl, q, n);
        rec->begin(K_ADJ_MERGE_UP, n, by);
        if (env) k_adj_merge_up<P, C, true><<<row_grid_b(pl, rs.start[4], 2 * mt), mt, 0, st>>>(pl, rs, n);
        else k_adj_merge_up<P, C, false><<<row_grid_b(pl, rs.start[4], 2 * mt), mt, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    {
        using A = typename Prec<P>::A;
        const size_t smem = adj_trace_smem<A, C>();
        for (int pair = 0; pair < 2; ++pair) {
            double by = img * (pl.C + 1) * ab * (pair == 0 ? 1.0 : 2.0);   // pair 1 adds to the gradients
            for (int q = 2 * pair; q < 2 * pair + 2; ++q)
                for (int n = 0; n <= 2; ++n) by += gTbytes(q, n);
            dim3 grid(pair_tiles_x(pair, pl.W), pair_tiles_y(pair, pl.H));
            rec->begin(K_ADJ_TRACE, pair, by);
            CUtensorMap me, ms;
            std::memset(&me, 0, sizeof(me));
            std::memset(&ms, 0, sizeof(ms));
            const int use_tma = (P != P_FP64 && encode_image_maps(pl, e, s, pair == 0 ? PT_RU : PT_RV,
                                                                  pair == 0 ? PT_RV : PT_RU, me, ms))
                                    ? 1 : 0;
            k_adj_trace<P, C, IN><<<grid, ADJ_THREADS, smem, st>>>(pl, (const IN *)e, (const IN *)s, (IN *)ge, (IN *)gs,
                                                                   pair, me, ms, use_tma);
            rec->end();
            ++*launches;
        }
    }
    return cudaGetLastError();
}

template <int P>
static cudaError_t bwd_prec(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, bool rc, cudaStream_t st, int *launches, Recorder *rec) {
    switch (pl.C) {
    case 1: return bwd_impl<P, 1>(pl, rt, e, s, gF, ge, gs, rc, st, launches, rec);
    case 2: return bwd_impl<P, 2>(pl, rt, e, s, gF, ge, gs, rc, st, launches, rec);
    case 3: return bwd_impl<P, 3>(pl, rt, e, s, gF, ge, gs, rc, st, launches, rec);
    default: return bwd_impl<P, 4>(pl, rt, e, s, gF, ge, gs, rc, st, launches, rec);
    }
}

template <int P>
static cudaError_t prepare_bwd_prec() {
    using IN = typename std::conditional<P == P_FP64, double, float>::type;
    using A = typename Prec<P>::A;
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_adj_trace<P, 1, IN>, adj_trace_smem<A, 1>());
    set((const void *)k_adj_trace<P, 2, IN>, adj_trace_smem<A, 2>());
    set((const void *)k_adj_trace<P, 3, IN>, adj_trace_smem<A, 3>());
    set((const void *)k_adj_trace<P, 4, IN>, adj_trace_smem<A, 4>());
    return e;
}

cudaError_t prepare_backward_kernels() {
    cudaError_t e = prepare_bwd_prec<P_FP32>();
    if (e == cudaSuccess) e = prepare_bwd_prec<P_FP16>();
    if (e == cudaSuccess) e = prepare_bwd_prec<P_BF16>();
    if (e == cudaSuccess) e = prepare_bwd_prec<P_FP64>();
    return e;
}

cudaError_t launch_backward(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, bool recompute, cudaStream_t st, int *launches, Recorder *rec) {
    switch (pl.prec) {
    case P_FP32: return bwd_prec<P_FP32>(pl, rt, e, s, gF, ge, gs, recompute, st, launches, rec);
    case P_FP16: return bwd_prec<P_FP16>(pl, rt, e, s, gF, ge, gs, recompute, st, launches, rec);
    case P_BF16: return bwd_prec<P_BF16>(pl, rt, e, s, gF, ge, gs, recompute, st, launches, rec);
    default: return bwd_prec<P_FP64>(pl, rt, e, s, gF, ge, gs, recompute, st, launches, rec);
    }
}

}  // namespace hrc
