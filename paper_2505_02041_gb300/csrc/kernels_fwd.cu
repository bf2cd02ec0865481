// kernels_fwd.cu -- forward HRC kernels for sm_103a (standalone launches of
// the bodies in fwd_bodies.cuh) and the forward launch sequence.
#include <cudaTypedefs.h>
#include <cstring>

#include "bulk_copy.cuh"
#include "fwd_bodies.cuh"
#include "launch.h"

namespace hrc {

template <int P, int C>
__global__ void __launch_bounds__(256) k_trace012(Plan pl, const float *__restrict__ e, const float *__restrict__ s,
                                                  const double *__restrict__ ed, const double *__restrict__ sd,
                                                  int qmask, const __grid_constant__ CUtensorMap tme,
                                                  const __grid_constant__ CUtensorMap tms, int use_tma) {
    extern __shared__ __align__(128) unsigned char tr_smem[];
    body_trace012<P, C>(pl, e, s, ed, sd, qmask, blockIdx.x, blockIdx.y, tr_smem, use_tma ? &tme : nullptr,
                        use_tma ? &tms : nullptr);
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

template <int P, int C, bool PAIR, bool ENV>
__global__ void __launch_bounds__(512) k_merge_down(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_down<P, C, PAIR, ENV>(pl, rs, n, row, vb);
}

template <int P, int C>
__global__ void __launch_bounds__(512) k_merge_up4(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_up4<P, C>(pl, rs, n, row, vb);
}

template <int P, int C, bool ENV>
__global__ void __launch_bounds__(512) k_merge_down4(Plan pl, RowSplit rs, int n) {
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_down4<P, C, ENV>(pl, rs, n, row, vb);
}

template <int P, int C, bool ENV>
__global__ void __launch_bounds__(128) k_merge_down_bulk(Plan pl, RowSplit rs, int n) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    long long row;
    int vb;
    row_block(pl, row, vb);
    body_merge_down_bulk<P, C, ENV>(pl, rs, n, row, vb, smem, bar);
}

template <int P, int C, class OUT, bool ENV>
__global__ void __launch_bounds__(512) k_fluence(Plan pl, OUT *__restrict__ F) {
    __shared__ __align__(16) unsigned char smem[fluence_smem<P, C>()];
    body_fluence<P, C, OUT, ENV>(pl, F, blockIdx.x, blockIdx.y, smem);
}

// Four pixels per thread, 128 threads, 7 blocks per SM (at most 73
// registers): without a cap the quad body takes 80-100 registers and 5
// blocks per SM and is slower than the pair body; with 8 blocks (64
// registers) it spills more and gains less (bf16, 1024^2: 49 us with pairs,
// 42 us at 8 blocks, 39 us at 7, 59 us at 6).
template <int P, int C, class OUT, bool ENV>
__global__ void __launch_bounds__(128, 7) k_fluence4(Plan pl, OUT *__restrict__ F) {
    __shared__ __align__(16) unsigned char smem[fluence_smem<P, C>()];
    body_fluence4<P, C, OUT, ENV>(pl, F, blockIdx.x, blockIdx.y, smem);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
static RowSplit make_split(const Plan &pl, int n, int kind, int qm) {
    // kind 0: trace rows (q, u); 1: merge-up rows (q, x, k) at level n;
    // 2: merge-down rows (q, x, ip) at level n.  qm: mask of the frames kept.
    RowSplit rs;
    long long acc = 0;
    for (int q = 0; q < 4; ++q) {
        rs.start[q] = acc;
        const QuadGeom &g = pl.q[q];
        long long rows = 0;
        if (!((qm >> q) & 1)) continue;
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

// Tensor maps of the fp32 inputs for the TMA staging of the trace kernels:
// emission [C][H][W] (3D) and extinction [H][W] (2D), box_x x box_y boxes,
// zero fill outside.  Needs 16-byte row strides (W a multiple of 4) and
// 16-byte aligned bases; false otherwise (the kernels then stage with plain
// loads).
bool encode_image_maps(const Plan &pl, const void *e, const void *s, int box_x, int box_y, CUtensorMap &me,
                       CUtensorMap &ms) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode || pl.W % 4 != 0 || (reinterpret_cast<uintptr_t>(e) & 15) || (reinterpret_cast<uintptr_t>(s) & 15))
        return false;
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1}, estr[3] = {1, 1, 1};
    const cuuint64_t de[3] = {(cuuint64_t)pl.W, (cuuint64_t)pl.H, (cuuint64_t)pl.C};
    const cuuint64_t se[2] = {(cuuint64_t)pl.W * 4, (cuuint64_t)pl.W * pl.H * 4};
    if (encode(&me, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(e), de, se, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (encode(&ms, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(s), de, se, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return true;
}

template <int P, int C>
static cudaError_t fwd_impl(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                            cudaStream_t st0, int *launches, Recorder *rec, bool with_sum, const Branches *br) {
    const int bs = 256;
    const bool env = plan_has_env(pl);   // kernels compiled for an environment map
    int Nmax = 0;
    for (int q = 0; q < 4; ++q) Nmax = pl.q[q].N > Nmax ? pl.q[q].N : Nmax;
    const float *ef = (const float *)e, *sf = (const float *)s;
    const double *ed = (const double *)e, *sd = (const double *)s;
    const double esz = P == P_FP64 ? 8.0 : 4.0;
    const double img = double(pl.W) * pl.H;
    const size_t smem = TraceTile<typename Prec<P>::A, C>::bytes();
    // sched 0: every launch covers the four frames (level-major);
    // sched 1: frame by frame, so that each level's producer and consumer
    //          (tens of MB per frame) meet in L2;
    // sched 2: frames {0, 1} and {2, 3} (equal extents) on two parallel
    //          branches, so that one branch's launch fills the SMs while the
    //          other's drains.
    const bool par = pl.sched == 2 && br != nullptr && !rec->on;
    const int sched = (pl.sched == 2 && !par) ? 0 : pl.sched;
    const int passes = sched == 1 ? 4 : (sched == 2 ? 2 : 1);
    const int nbr = passes;
    if (par) {
        cudaError_t err = cudaEventRecord(br->fork, st0);
        for (int i = 0; i < nbr && err == cudaSuccess; ++i) err = cudaStreamWaitEvent(br->s[i], br->fork, 0);
        if (err != cudaSuccess) return err;
    }
    for (int pass = 0; pass < passes; ++pass) {
        const int qm = sched == 1 ? 1 << pass : (sched == 2 ? 3 << (2 * pass) : 15);
        const int nq = __builtin_popcount(qm);
        const cudaStream_t st = par ? br->s[pass] : st0;
        {
            double by = img * (pl.C + 1) * esz * nq / 4;
            for (int q = 0; q < 4; ++q)
                if ((qm >> q) & 1)
                    for (int n = 0; n <= 2; ++n) by += bytes_T(pl, q, n);
            dim3 grid((pl.W + TR_TILE - 1) / TR_TILE, (pl.H + TR_TILE - 1) / TR_TILE);
            rec->begin(K_TRACE012, 0, by);
            CUtensorMap me, ms;
            std::memset(&me, 0, sizeof(me));
            std::memset(&ms, 0, sizeof(ms));
            const int use_tma = (P != P_FP64 && encode_image_maps(pl, e, s, TR_REG, TR_REG, me, ms)) ? 1 : 0;
            k_trace012<P, C><<<grid, 256, smem, st>>>(pl, ef, sf, ed, sd, qm, me, ms, use_tma);
            rec->end();
            ++*launches;
        }
        for (int n = 3; n <= Nmax; ++n) {
            RowSplit rs = make_split(pl, n, 1, qm);
            if (rs.start[4] == 0) continue;
            double by = 0;
            for (int q = 0; q < 4; ++q)
                if (((qm >> q) & 1) && n <= pl.q[q].N) by += bytes_T(pl, q, n - 1) + bytes_T(pl, q, n);
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
        // R_0 feeds only the fluence sum, which computes it in place.
        // mdown 2: every level in one persistent launch (kernels_persist.cu)
        if (pl.mdown == 2 && P != P_FP64 && persist_down_usable(pl)) {
            auto level_bytes = [&](int n) {
                double by = 0;
                for (int q = 0; q < 4; ++q) {
                    const QuadGeom &g = pl.q[q];
                    if (!((qm >> q) & 1) || n >= g.N) continue;
                    by += bytes_T_odd(pl, q, n) + bytes_T_even_dirs(pl, q, n + 1);
                    by += bytes_R(pl, q, n + 1) + bytes_R(pl, q, n);
                }
                return by;
            };
            double by = 0;
            for (int n = Nmax - 1; n >= 1; --n) by += level_bytes(n);
            const cudaError_t err = launch_merge_down_persist(pl, qm, Nmax - 1, 1, st, launches, rec, by);
            if (err != cudaSuccess) return err;
            continue;
        }
        for (int n = Nmax - 1; n >= 1; --n) {
            RowSplit rs = make_split(pl, n, 2, qm);
            if (rs.start[4] == 0) continue;
            double by = 0;
            for (int q = 0; q < 4; ++q) {
                const QuadGeom &g = pl.q[q];
                if (!((qm >> q) & 1) || n >= g.N) continue;
                // odd columns of T_n, even directions of T_{n+1}, R_{n+1} once, R_n written
                by += bytes_T_odd(pl, q, n);
                by += bytes_T_even_dirs(pl, q, n + 1);
                by += bytes_R(pl, q, n + 1) + bytes_R(pl, q, n);
            }
            const int mt = pl.mthreads;
            rec->begin(K_MERGE_DOWN, n, by);
            if (n >= 1 && pl.mdown == 1 && P != P_FP64) {
                if (env)
                    k_merge_down_bulk<P, C, true><<<row_grid(pl, rs.start[4], kBV), 128, BulkMD<P, C>::bytes(), st>>>(pl, rs, n);
                else
                    k_merge_down_bulk<P, C, false><<<row_grid(pl, rs.start[4], kBV), 128, BulkMD<P, C>::bytes(), st>>>(pl, rs, n);
            } else if (n >= 1) {
                if (env) k_merge_down4<P, C, true><<<row_grid(pl, rs.start[4], 4 * mt), mt, 0, st>>>(pl, rs, n);
                else k_merge_down4<P, C, false><<<row_grid(pl, rs.start[4], 4 * mt), mt, 0, st>>>(pl, rs, n);
            } else {
                const int ts = 2 * mt > 512 ? 512 : 2 * mt;   // single v per thread at level 0
                if (env) k_merge_down<P, C, false, true><<<row_grid(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, n);
                else k_merge_down<P, C, false, false><<<row_grid(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, n);
            }
            rec->end();
            ++*launches;
        }
    }
    if (par) {
        cudaError_t err = cudaSuccess;
        for (int i = 0; i < nbr && err == cudaSuccess; ++i) {
            err = cudaEventRecord(br->join[i], br->s[i]);
            if (err == cudaSuccess) err = cudaStreamWaitEvent(st0, br->join[i], 0);
        }
        if (err != cudaSuccess) return err;
    }
    const cudaStream_t st = st0;
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
        // Pairs of pixels per thread, 256 threads on large grids; grids of
        // fewer than 600 tiles (about 4 per SM; 512^2 and below) take 512, so
        // that the GPU still holds enough loads in flight.  The 16-bit modes
        // on large grids take four pixels per thread (k_fluence4): a pair of
        // 16-bit radiances is only a 4-byte access.
        const long long tiles = (long long)grid.x * grid.y;
        const int ft = tiles < 600 ? 512 : 256;
        if constexpr (P == P_FP64) {
            if (env) k_fluence<P, C, double, true><<<grid, ft, 0, st>>>(pl, (double *)F);
            else k_fluence<P, C, double, false><<<grid, ft, 0, st>>>(pl, (double *)F);
        } else if constexpr (P == P_FP16 || P == P_BF16) {
            if (tiles >= 600) {
                if (env) k_fluence4<P, C, float, true><<<grid, 128, 0, st>>>(pl, (float *)F);
                else k_fluence4<P, C, float, false><<<grid, 128, 0, st>>>(pl, (float *)F);
            } else {
                if (env) k_fluence<P, C, float, true><<<grid, ft, 0, st>>>(pl, (float *)F);
                else k_fluence<P, C, float, false><<<grid, ft, 0, st>>>(pl, (float *)F);
            }
        } else {
            if (env) k_fluence<P, C, float, true><<<grid, ft, 0, st>>>(pl, (float *)F);
            else k_fluence<P, C, float, false><<<grid, ft, 0, st>>>(pl, (float *)F);
        }
        rec->end();
        ++*launches;
    }
    return cudaGetLastError();
}

// R_0 of every frame into its buffer (the forward with the fluence sum never
// stores it); for introspection.
template <int P, int C>
static cudaError_t r0_impl(const Plan &pl, cudaStream_t st) {
    RowSplit rs = make_split(pl, 0, 2, 15);
    if (rs.start[4] == 0) return cudaSuccess;
    const int ts = 2 * pl.mthreads > 512 ? 512 : 2 * pl.mthreads;
    if (plan_has_env(pl)) k_merge_down<P, C, false, true><<<row_grid(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, 0);
    else k_merge_down<P, C, false, false><<<row_grid(pl, rs.start[4], ts), ts, 0, st>>>(pl, rs, 0);
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
                            cudaStream_t st, int *launches, Recorder *rec, const Branches *br) {
    switch (pl.C) {
    case 1: return fwd_impl<P, 1>(pl, rt, e, s, F, st, launches, rec, F != nullptr, br);
    case 2: return fwd_impl<P, 2>(pl, rt, e, s, F, st, launches, rec, F != nullptr, br);
    case 3: return fwd_impl<P, 3>(pl, rt, e, s, F, st, launches, rec, F != nullptr, br);
    default: return fwd_impl<P, 4>(pl, rt, e, s, F, st, launches, rec, F != nullptr, br);
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
    if constexpr (P != P_FP64) {
        set((const void *)k_merge_down_bulk<P, 1, false>, BulkMD<P, 1>::bytes());
        set((const void *)k_merge_down_bulk<P, 1, true>, BulkMD<P, 1>::bytes());
        set((const void *)k_merge_down_bulk<P, 2, false>, BulkMD<P, 2>::bytes());
        set((const void *)k_merge_down_bulk<P, 2, true>, BulkMD<P, 2>::bytes());
        set((const void *)k_merge_down_bulk<P, 3, false>, BulkMD<P, 3>::bytes());
        set((const void *)k_merge_down_bulk<P, 3, true>, BulkMD<P, 3>::bytes());
        set((const void *)k_merge_down_bulk<P, 4, false>, BulkMD<P, 4>::bytes());
        set((const void *)k_merge_down_bulk<P, 4, true>, BulkMD<P, 4>::bytes());
    }
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
                           cudaStream_t st, int *launches, Recorder *rec, const Branches *br) {
    switch (pl.prec) {
    case P_FP32: return fwd_prec<P_FP32>(pl, rt, e, s, F, st, launches, rec, br);
    case P_FP16: return fwd_prec<P_FP16>(pl, rt, e, s, F, st, launches, rec, br);
    case P_BF16: return fwd_prec<P_BF16>(pl, rt, e, s, F, st, launches, rec, br);
    default: return fwd_prec<P_FP64>(pl, rt, e, s, F, st, launches, rec, br);
    }
}

}  // namespace hrc
