// kernels_fwd.cu -- forward HRC kernels for sm_103a (standalone launches of
// the bodies in fwd_bodies.cuh) and the forward launch sequence.
#include "fwd_bodies.cuh"
#include "launch.h"

namespace hrc {

template <int P, int C>
__global__ void __launch_bounds__(256) k_trace012(Plan pl, const float *__restrict__ e, const float *__restrict__ s,
                                                  const double *__restrict__ ed, const double *__restrict__ sd,
                                                  int qmask) {
    extern __shared__ __align__(16) unsigned char tr_smem[];
    body_trace012<P, C>(pl, e, s, ed, sd, qmask, blockIdx.x, blockIdx.y, tr_smem);
}

// Row and v-block of this block: the launch grid is (rows, v-blocks), or
// (v-blocks, rows) when the plan puts the v-blocks of a row side by side.
__device__ __forceinline__ void row_block(const Plan &pl, long long &row, int &vb) {
    if (pl.vmajor) { row = blockIdx.y; vb = blockIdx.x; }
    else { row = blockIdx.x; vb = blockIdx.y; }
}

template <int P, int C, int G>
__global__ void __launch_bounds__(512) k_merge_up(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_up<P, C, G>(pl, rs, n, row, vb);
}

template <int P, int C, bool PAIR>
__global__ void __launch_bounds__(512) k_merge_down(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_down<P, C, PAIR>(pl, rs, n, row, vb);
}

template <int P, int C>
__global__ void __launch_bounds__(512) k_merge_up4(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_up4<P, C>(pl, rs, n, row, vb);
}

template <int P, int C>
__global__ void __launch_bounds__(512) k_merge_down4(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_down4<P, C>(pl, rs, n, row, vb);
}

template <int P, int C, class OUT>
__global__ void __launch_bounds__(128) k_fluence(Plan pl, OUT *__restrict__ F) {
    __shared__ __align__(16) unsigned char smem[fluence_smem<P, C>()];
    body_fluence<P, C, OUT>(pl, F, blockIdx.x, blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
static RowSplit make_split(const Plan &pl, int n, int kind, int qsel) {
    // kind 0: trace rows (q, u); 1: merge-up rows (q, x, k) at level n;
    // 2: merge-down rows (q, x, ip) at level n.  qsel >= 0 keeps one frame.
    RowSplit rs;
    long long acc = 0;
    for (int q = 0; q < 4; ++q) {
        rs.start[q] = acc;
        const QuadGeom &g = pl.q[q];
        long long rows = 0;
        if (qsel >= 0 && q != qsel) continue;
        if (kind == 0) rows = g.U;
        else if (kind == 1) rows = (n <= g.N && n >= 3) ? (long long)(g.Un[n] - 1) * ((1 << n) + 1) : 0;
        else rows = (n < g.N) ? (long long)(g.Un[n] - 1) * (1 << n) : 0;
        acc += rows;
    }
    rs.start[4] = acc;
    return rs;
}

// Grid of a row kernel: `rows` rows of blocks covering `per_block` v each.
static dim3 row_grid(const Plan &pl, long long rows, int per_block) {
    int Vmax = 0;
    for (int q = 0; q < 4; ++q) Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    const unsigned vb = (unsigned)((Vmax + per_block - 1) / per_block);
    return pl.vmajor ? dim3(vb, (unsigned)rows) : dim3((unsigned)rows, vb);
}

static int vblocks(const Plan &pl, int bs) {
    int Vmax = 0;
    for (int q = 0; q < 4; ++q) Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    return (Vmax + bs - 1) / bs;
}

// Algorithmic bytes of T_n / R_n of frame q: the live entries only (column 0
// of every level and the dead entries of T_0 / T_1 are never touched).
static double t_entry_bytes(const Plan &pl) {
    return pl.C * (pl.prec == P_FP32 ? 4.0 : (pl.prec == P_FP64 ? 8.0 : 2.0)) + (pl.prec == P_FP64 ? 8.0 : 4.0);
}

double bytes_T(const Plan &pl, int q, int n) {
    const QuadGeom &g = pl.q[q];
    if (n < 0 || n > g.N) return 0.0;
    return double(t_live_rows(n, g.Un[n])) * g.V * t_entry_bytes(pl);
}

// The odd live columns of T_n (read by the level-n merge down, Eq. 14).
double bytes_T_odd(const Plan &pl, int q, int n) {
    const QuadGeom &g = pl.q[q];
    if (n < 0 || n > g.N) return 0.0;
    return double(g.Un[n] / 2) * ((1 << n) + 1) * g.V * t_entry_bytes(pl);
}

// The even directions of the live columns of T_n (read by the level n-1
// merge down at even columns, Eqs. 15-17).
double bytes_T_even_dirs(const Plan &pl, int q, int n) {
    const QuadGeom &g = pl.q[q];
    if (n < 1 || n > g.N) return 0.0;
    return double(g.Un[n] - 1) * ((1 << (n - 1)) + 1) * g.V * t_entry_bytes(pl);
}

double bytes_R(const Plan &pl, int q, int n) {
    const QuadGeom &g = pl.q[q];
    if (n < 0 || n >= g.N) return 0.0;
    const double vr = pl.C * (pl.prec == P_FP32 ? 4.0 : (pl.prec == P_FP64 ? 8.0 : 2.0));
    return double(g.Un[n] - 1) * (1 << n) * g.V * vr;
}

template <int P, int C>
static cudaError_t fwd_impl(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                            cudaStream_t st, int *launches, Recorder *rec, bool with_sum) {
    const int bs = 256;
    int Nmax = 0;
    for (int q = 0; q < 4; ++q) Nmax = pl.q[q].N > Nmax ? pl.q[q].N : Nmax;
    const float *ef = (const float *)e, *sf = (const float *)s;
    const double *ed = (const double *)e, *sd = (const double *)s;
    const double esz = P == P_FP64 ? 8.0 : 4.0;
    const double img = double(pl.W) * pl.H;
    const size_t smem = TraceTile<typename Prec<P>::A, C>::bytes();
    // sched 0: every launch covers the four frames (level-major);
    // sched 1: frame by frame, so that each level's producer and consumer
    //          (tens of MB per frame) meet in L2.
    const int passes = pl.sched == 1 ? 4 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        const int qsel = pl.sched == 1 ? pass : -1;
        {
            double by = img * (pl.C + 1) * esz / (pl.sched == 1 ? 4 : 1);
            for (int q = 0; q < 4; ++q)
                if (qsel < 0 || q == qsel)
                    for (int n = 0; n <= 2; ++n) by += bytes_T(pl, q, n);
            dim3 grid((pl.W + TR_TILE - 1) / TR_TILE, (pl.H + TR_TILE - 1) / TR_TILE);
            rec->begin(K_TRACE012, 0, by);
            k_trace012<P, C><<<grid, 256, smem, st>>>(pl, ef, sf, ed, sd, qsel < 0 ? 15 : (1 << qsel));
            rec->end();
            ++*launches;
        }
        for (int n = 3; n <= Nmax; ++n) {
            RowSplit rs = make_split(pl, n, 1, qsel);
            if (rs.start[4] == 0) continue;
            double by = 0;
            for (int q = 0; q < 4; ++q)
                if ((qsel < 0 || q == qsel) && n <= pl.q[q].N) by += bytes_T(pl, q, n - 1) + bytes_T(pl, q, n);
            const int mt = pl.mthreads;
            rec->begin(K_MERGE_UP, n, by);
            // groups: 1 = a pair of v per thread, 2 = two pairs blockDim apart,
            // 4 = four consecutive v
            if (pl.mgroups == 4) k_merge_up4<P, C><<<row_grid(pl, rs.start[4], 4 * mt), mt, 0, st>>>(pl, rs, n);
            else if (pl.mgroups == 2) k_merge_up<P, C, 2><<<row_grid(pl, rs.start[4], 4 * mt), mt, 0, st>>>(pl, rs, n);
            else k_merge_up<P, C, 1><<<row_grid(pl, rs.start[4], 2 * mt), mt, 0, st>>>(pl, rs, n);
            rec->end();
            ++*launches;
        }
        // R_0 feeds only the fluence sum, which computes it in place
        for (int n = Nmax - 1; n >= 1; --n) {
            RowSplit rs = make_split(pl, n, 2, qsel);
            if (rs.start[4] == 0) continue;
            double by = 0;
            for (int q = 0; q < 4; ++q) {
                const QuadGeom &g = pl.q[q];
                if ((qsel >= 0 && q != qsel) || n >= g.N) continue;
                // odd columns of T_n, even directions of T_{n+1}, R_{n+1} once, R_n written
                by += bytes_T_odd(pl, q, n);
                by += bytes_T_even_dirs(pl, q, n + 1);
                by += bytes_R(pl, q, n + 1) + bytes_R(pl, q, n);
            }
            const int mt = pl.mthreads;
            rec->begin(K_MERGE_DOWN, n, by);
            if (n >= 1) k_merge_down4<P, C><<<row_grid(pl, rs.start[4], 4 * mt), mt, 0, st>>>(pl, rs, n);
            else {
                const int ts = 2 * mt > 512 ? 512 : 2 * mt;   // single v per thread at level 0
                k_merge_down<P, C, false><<<row_grid(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, n);
            }
            rec->end();
            ++*launches;
        }
    }
    if (with_sum) {
        // level-0 merge-down reads (odd columns of T_0, even directions of
        // T_1, R_1) and the fluence written
        double by = img * pl.C * esz;
        for (int q = 0; q < 4; ++q) {
            if (pl.q[q].N < 1) continue;
            by += bytes_T_odd(pl, q, 0) + bytes_R(pl, q, 1) + bytes_T_even_dirs(pl, q, 1);
        }
        dim3 grid((pl.W + 31) / 32, (pl.H + 31) / 32);
        rec->begin(K_FLUENCE_SUM, 0, by);
        // 128 threads: every tile of a 1024^2 image is resident at once
        if (P == P_FP64) k_fluence<P, C, double><<<grid, 128, 0, st>>>(pl, (double *)F);
        else k_fluence<P, C, float><<<grid, 128, 0, st>>>(pl, (float *)F);
        rec->end();
        ++*launches;
    }
    return cudaGetLastError();
}

// R_0 of every frame into its buffer (the forward with the fluence sum never
// stores it); for introspection.
template <int P, int C>
static cudaError_t r0_impl(const Plan &pl, cudaStream_t st) {
    RowSplit rs = make_split(pl, 0, 2, -1);
    if (rs.start[4] == 0) return cudaSuccess;
    const int ts = 2 * pl.mthreads > 512 ? 512 : 2 * pl.mthreads;
    k_merge_down<P, C, false><<<row_grid(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, 0);
    return cudaGetLastError();
}

template <int P>
static cudaError_t r0_prec(const Plan &pl, cudaStream_t st) {
    switch (pl.C) {
    case 1: return r0_impl<P, 1>(pl, st);
    case 2: return r0_impl<P, 2>(pl, st);
    case 3: return r0_impl<P, 3>(pl, st);
    default: return r0_impl<P, 4>(pl, st);
    }
}

cudaError_t launch_r0(const Plan &pl, cudaStream_t st) {
    switch (pl.prec) {
    case P_FP32: return r0_prec<P_FP32>(pl, st);
    case P_FP16: return r0_prec<P_FP16>(pl, st);
    case P_BF16: return r0_prec<P_BF16>(pl, st);
    default: return r0_prec<P_FP64>(pl, st);
    }
}

template <int P>
static cudaError_t fwd_prec(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                            cudaStream_t st, int *launches, Recorder *rec) {
    switch (pl.C) {
    case 1: return fwd_impl<P, 1>(pl, rt, e, s, F, st, launches, rec, F != nullptr);
    case 2: return fwd_impl<P, 2>(pl, rt, e, s, F, st, launches, rec, F != nullptr);
    case 3: return fwd_impl<P, 3>(pl, rt, e, s, F, st, launches, rec, F != nullptr);
    default: return fwd_impl<P, 4>(pl, rt, e, s, F, st, launches, rec, F != nullptr);
    }
}

template <int P>
static cudaError_t prepare_prec() {
    cudaError_t e = cudaSuccess;
    auto set = [&](const void *fn, size_t bytes) {
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    };
    set((const void *)k_trace012<P, 1>, TraceTile<typename Prec<P>::A, 1>::bytes());
    set((const void *)k_trace012<P, 2>, TraceTile<typename Prec<P>::A, 2>::bytes());
    set((const void *)k_trace012<P, 3>, TraceTile<typename Prec<P>::A, 3>::bytes());
    set((const void *)k_trace012<P, 4>, TraceTile<typename Prec<P>::A, 4>::bytes());
    return e;
}

cudaError_t prepare_forward_kernels() {
    cudaError_t e = prepare_prec<P_FP32>();
    if (e == cudaSuccess) e = prepare_prec<P_FP16>();
    if (e == cudaSuccess) e = prepare_prec<P_BF16>();
    if (e == cudaSuccess) e = prepare_prec<P_FP64>();
    return e;
}

cudaError_t launch_forward(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                           cudaStream_t st, int *launches, Recorder *rec) {
    switch (pl.prec) {
    case P_FP32: return fwd_prec<P_FP32>(pl, rt, e, s, F, st, launches, rec);
    case P_FP16: return fwd_prec<P_FP16>(pl, rt, e, s, F, st, launches, rec);
    case P_BF16: return fwd_prec<P_BF16>(pl, rt, e, s, F, st, launches, rec);
    default: return fwd_prec<P_FP64>(pl, rt, e, s, F, st, launches, rec);
    }
}

}  // namespace hrc
