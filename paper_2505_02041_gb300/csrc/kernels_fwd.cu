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

// ---------------------------------------------------------------------------
// Merge down (level n >= 1) with the block's rows staged in shared memory by
// bulk copies.  One block of 128 threads = one row (q, x, ip) x kBV v (four
// consecutive v per thread).  Thread 0 copies, for both edges of the cone
// (Eq. 14 at odd x, Eqs. 15-17 at even x), the T planes of the edge's row,
// the far R window (its start rounded down to 16 bytes, clipped to the
// row) and, at even x, the near R row; every thread then reads only shared
// memory.  Out-of-range far values (and R_N) are the environment's values
// (0 without a map), chosen by a select; they are never read from the rows.
// ---------------------------------------------------------------------------
constexpr int kBV = 512;

template <int P, int C> struct BulkMD {
    using SL = typename Prec<P>::SL;
    using ST = typename Prec<P>::ST;
    static constexpr int AL = 16 / (int)sizeof(SL);   // elements per 16 bytes
    static constexpr int FW = kBV + 16;                  // far window length
    static constexpr size_t bytes() {
        return sizeof(SL) * 2 * C * kBV + sizeof(ST) * 2 * kBV + sizeof(SL) * 2 * C * FW + sizeof(SL) * 2 * C * kBV;
    }
};

template <int P, int C, bool ENV>
__global__ void __launch_bounds__(128) k_merge_down_bulk(Plan pl, RowSplit rs, int n) {
    using SL = typename Prec<P>::SL;
    using ST = typename Prec<P>::ST;
    using A = typename Prec<P>::A;
    using B = BulkMD<P, C>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    long long row;
    int vb;
    row_block(pl, row, vb);
    int local;
    const int q = find_quadrant(rs, row, local);
    const QuadGeom &g = pl.q[q];
    const int v0 = vb * kBV;
    if (v0 >= g.V) return;                                   // uniform over the block
    const int I = 1 << n;
    local += I;
    const int x = local >> n, ip = local & (I - 1);
    const bool top = n + 1 >= g.N;                           // R_N: 0, or the environment map
    const int s = 1 << n;
    const bool odd = (x & 1) != 0;
    const int x2 = x >> 1;
    const int xt = odd ? x : x2;                             // T row: T_n(x, .) or T_{n+1}(x/2, .)
    const int xq = odd ? (x + 1) >> 1 : x2 + 1;              // far column at level n+1
    const bool far_ok = !top && xq < g.Un[n + 1];
    const bool near_ok = !odd && !top;
    int kk[2], j[2], off[2], fa[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        kk[e] = odd ? (e == 0 ? ip + 1 : ip) : (e == 0 ? 2 * ip + 2 : 2 * ip);
        j[e] = e == 0 ? 2 * ip + 1 : 2 * ip;
        off[e] = 2 * kk[e] - (odd ? s : 2 * s);
        const int a = v0 + off[e];
        fa[e] = a >= 0 ? a / B::AL * B::AL : -((-a + B::AL - 1) / B::AL) * B::AL;   // round down
    }
    SL *tl = reinterpret_cast<SL *>(smem);                   // [2][C][kBV]
    ST *tt = reinterpret_cast<ST *>(tl + 2 * C * kBV);       // [2][kBV]
    SL *rf = reinterpret_cast<SL *>(tt + 2 * kBV);           // [2][C][FW]
    SL *rn = rf + 2 * C * B::FW;                             // [2][C][kBV]
    const int vend = v0 + kBV < g.Vs ? v0 + kBV : g.Vs;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const TLevel<P, C> Tt(pl, q, odd ? n : n + 1);
        const RLevel<P, C> R1(pl, q, top ? n : n + 1);
        const unsigned tb = (unsigned)(vend - v0);
        unsigned total = 2u * tb * (unsigned)(C * sizeof(SL) + sizeof(ST));
        int fs[2], fe[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            fs[e] = fa[e] > 0 ? fa[e] : 0;
            fe[e] = fa[e] + B::FW < g.Vs ? fa[e] + B::FW : g.Vs;
            if (far_ok && fe[e] > fs[e]) total += (unsigned)(C * (fe[e] - fs[e]) * sizeof(SL));
        }
        if (near_ok) total += 2u * (unsigned)(C * tb * sizeof(SL));
        mbar_arrive_expect(&bar, total + (unsigned)pl.bulk_extra_tx);
        const uint64_t pol = l2_evict_first();               // T rows: read once from HBM
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const char *gr = Tt.row(xt, kk[e]);
#pragma unroll
            for (int c = 0; c < C; ++c)
                bulk_load_hint(tl + (e * C + c) * kBV, reinterpret_cast<const SL *>(gr) + (long long)c * g.Vs + v0,
                               tb * sizeof(SL), &bar, pol);
            bulk_load_hint(tt + e * kBV, reinterpret_cast<const ST *>(gr + (long long)C * g.Vs * sizeof(SL)) + v0,
                           tb * sizeof(ST), &bar, pol);
            if (far_ok && fe[e] > fs[e])
#pragma unroll
                for (int c = 0; c < C; ++c)
                    bulk_load(rf + (e * C + c) * B::FW + (fs[e] - fa[e]), R1.base + R1.idx(xq, j[e], c, fs[e]),
                              (unsigned)((fe[e] - fs[e]) * sizeof(SL)), &bar);
            if (near_ok)
#pragma unroll
                for (int c = 0; c < C; ++c)
                    bulk_load(rn + (e * C + c) * kBV, R1.base + R1.idx(x2, j[e], c, v0), tb * sizeof(SL), &bar);
        }
    }
    if (!mbar_wait(&bar, 0, pl.bulk_limit_ns)) {              // gave up: let the copies land, report, leave
        const int code = mbar_wait(&bar, 0, drain_limit_ns(pl.bulk_limit_ns)) ? kWaitTimeout : kWaitLost;
        if (threadIdx.x == 0) atomicMax(pl.status, code);
        return;
    }
    const int v = v0 + 4 * (int)threadIdx.x;
    if (v >= g.V) return;
    const int ti = v - v0;
    const A Ap = arc<P>(pl, n + 1, 2 * ip + 1), Am = arc<P>(pl, n + 1, 2 * ip);
    A acc[4][C];
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[l][c] = A(0);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const A Aj = e == 0 ? Ap : Am;
        A tr[4];
        ld4(tt + e * kBV + ti, tr);
#pragma unroll
        for (int l = 0; l < 4; ++l) tr[l] = Prec<P>::LOG ? fexp(-tr[l]) : tr[l];
        const int fi = ti + (v0 + off[e] - fa[e]);           // far window index of v (even)
#pragma unroll
        for (int c = 0; c < C; ++c) {
            A L[4], r[4], r0[4];
            const A ev = renv<P, C, ENV>(pl, q, n + 1, j[e], c);   // out of range: the environment
            ld4(tl + (e * C + c) * kBV + ti, L);
            ld2(rf + (e * C + c) * B::FW + fi, r[0], r[1]);
            ld2(rf + (e * C + c) * B::FW + fi + 2, r[2], r[3]);
            if (near_ok) ld4(rn + (e * C + c) * kBV + ti, r0);
#pragma unroll
            for (int l = 0; l < 4; ++l) {
                const int vf = v + l + off[e];
                const A rr = (far_ok && vf >= 0 && vf < g.V) ? r[l] : ev;
                const A f = fma(Aj, L[l], tr[l] * rr);
                if (odd) acc[l][c] += f;                                         // Eq. 14
                else acc[l][c] += A(0.5) * ((near_ok ? r0[l] : ev) + f);         // Eqs. 15-17
            }
        }
    }
    const RLevel<P, C> Rn(pl, q, n);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const A o[4] = {acc[0][c], acc[1][c], acc[2][c], acc[3][c]};
        Rn.store4(x, ip, c, v, o);
    }
}

template <int P, int C, class OUT, bool ENV>
__global__ void __launch_bounds__(128) k_fluence(Plan pl, OUT *__restrict__ F) {
    __shared__ __align__(16) unsigned char smem[fluence_smem<P, C>()];
    body_fluence<P, C, OUT, ENV>(pl, F, blockIdx.x, blockIdx.y, smem);
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
        // 128 threads: every tile of a 1024^2 image is resident at once
        if (P == P_FP64) {
            if (env) k_fluence<P, C, double, true><<<grid, 128, 0, st>>>(pl, (double *)F);
            else k_fluence<P, C, double, false><<<grid, 128, 0, st>>>(pl, (double *)F);
        } else {
            if (env) k_fluence<P, C, float, true><<<grid, 128, 0, st>>>(pl, (float *)F);
            else k_fluence<P, C, float, false><<<grid, 128, 0, st>>>(pl, (float *)F);
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
