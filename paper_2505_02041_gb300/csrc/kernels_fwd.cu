// kernels_fwd.cu -- forward HRC kernels for sm_103a.
//
//   k_trace012    : T_0..T_min(2,N) by direct tracing (Sec. 4.2, Eq. 9)
//   k_merge_up    : T_n from T_{n-1} (Eq. 18 even k, Eqs. 19-20 odd k)
//   k_merge_down  : R_n from R_{n+1}, T_n, T_{n+1} (Eq. 14 odd x, Eqs. 15-17 even x)
//   k_fluence_sum : F = sum over quadrants of R_0([u+1, v], 1/2) (Algorithm 1, Lighting)
//
// All four quadrant frames run in one launch.  The work is memory-bound
// (about one FMA per byte), so the kernels are organised around coalesced,
// v-contiguous rows: one CTA handles one (x, k) or (x, i) row segment of
// BLOCK consecutive v, every neighbour access being a shifted run of the
// same length.  Out-of-range lookups read as vacuum (T = <0, 1>, R = 0),
// which is exact for this method: paths are monotone in v, so a path that
// leaves the grid never re-enters, and nothing outside the grid emits.
#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

// Row-to-quadrant lookup for flattened (q, row) grids.
struct RowSplit {
    long long start[5];   // first global row of each quadrant; start[4] = total
};

__device__ __forceinline__ int find_quadrant(const RowSplit &rs, long long r, int &local) {
    int q = 0;
    long long base = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (r >= rs.start[j]) { q = j; base = rs.start[j]; }
    local = (int)(r - base);
    return q;
}

// Piece weights of a uniform pixel crossed over length len (Eq. 4 over one
// piece): returns w = len * phi(sigma len) and sets tp = exp(-sigma len).
__device__ __forceinline__ float piece(float sg, float len, float &tp) {
    const float tau = sg * len;
    tp = __expf(-tau);
    // len * phi(tau): (1 - e^-tau) / sigma away from 0, a short Taylor series near 0
    const float series = len * (1.f - tau * (0.5f - tau * (1.f / 6.f - tau * (1.f / 24.f))));
    return fabsf(tau) < 0.03f ? series : (1.f - tp) / sg;
}
__device__ __forceinline__ double piece(double sg, double len, double &tp) {
    const double tau = sg * len;
    const double m = expm1(-tau);
    tp = 1.0 + m;
    return sg != 0.0 ? -m / sg : len;
}

// T_0..T_min(2,N) of all four quadrant frames for one 32 x 32 image tile.
// The tile's extinction and emission plus a 4-pixel halo (the longest
// directly traced ray, v_2(k), reaches 4 pixels along and across) are
// staged once in shared memory, zero outside the image (= vacuum, exact).
// Work rows are (column c of the tile along the frame's u axis, ray r):
// each warp traces one row for 32 consecutive v, so its T stores are
// 128-byte coalesced row segments in every frame.
constexpr int TR_TILE = 32, TR_HALO = 4, TR_REG = TR_TILE + 2 * TR_HALO, TR_PITCH = TR_REG + 1;

template <int P, int C>
__global__ void __launch_bounds__(256) k_trace012(Plan pl, RayTable rt, const float *__restrict__ e,
                                                  const float *__restrict__ s, const double *__restrict__ ed,
                                                  const double *__restrict__ sd) {
    using A = typename Prec<P>::A;
    extern __shared__ __align__(16) unsigned char tr_smem[];
    A *sm_s = reinterpret_cast<A *>(tr_smem);                 // [TR_REG][TR_PITCH]
    A *sm_e = sm_s + TR_REG * TR_PITCH;                        // [C][TR_REG][TR_PITCH]
    const int W = pl.W, H = pl.H;
    const int x0 = blockIdx.x * TR_TILE, y0 = blockIdx.y * TR_TILE;
    const long long HW = (long long)W * H;
    for (int i = threadIdx.x; i < TR_REG * TR_REG; i += blockDim.x) {
        const int ry = i / TR_REG, rx = i - ry * TR_REG;
        const int x = x0 - TR_HALO + rx, y = y0 - TR_HALO + ry;
        const bool in = x >= 0 && x < W && y >= 0 && y < H;
        const long long pix = (long long)y * W + x;
        sm_s[ry * TR_PITCH + rx] = in ? ((P == P_FP64) ? A(sd[pix]) : A(s[pix])) : A(0);
#pragma unroll
        for (int c = 0; c < C; ++c)
            sm_e[(c * TR_REG + ry) * TR_PITCH + rx] = in ? ((P == P_FP64) ? A(ed[c * HW + pix]) : A(e[c * HW + pix])) : A(0);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int q = 0; q < 4; ++q) {
        const QuadGeom &g = pl.q[q];
        const int nmax = g.N < 2 ? g.N : 2;
        const bool xu = q < 2;                              // frame u runs along image x
        const int tu = xu ? x0 : y0, tv = xu ? y0 : x0;     // tile origin along u / v axes
        const int ext_u = xu ? W : H;
        const int v = tv + lane;
        for (int row = warp; row < TR_TILE * HRC_MAXRAY; row += nwarp) {
            const int c = row / HRC_MAXRAY, r = row - c * HRC_MAXRAY;
            const int n = r < 2 ? 0 : (r < 5 ? 1 : 2);
            const int k = r - (n == 0 ? 0 : (n == 1 ? 2 : 5));
            if (n > nmax || tu + c >= ext_u) continue;
            const int u = (q == 0 || q == 2) ? tu + c : ext_u - 1 - (tu + c);
            if (u & ((1 << n) - 1)) continue;
            if (v >= g.V) continue;
            A L[C];
#pragma unroll
            for (int cc = 0; cc < C; ++cc) L[cc] = A(0);
            A Tacc = A(1), tau = A(0);
            const int sgn = (q == 0 || q == 2) ? 1 : -1;     // image step along u
            for (int j = rt.start[r]; j < rt.start[r + 1]; ++j) {
                const int du = rt.p[j].du, dv = rt.p[j].dv;
                const int a = TR_HALO + c + sgn * du, b = TR_HALO + lane + dv;   // tile coords (u axis, v axis)
                const int sx = xu ? a : b, sy = xu ? b : a;
                const int o = sy * TR_PITCH + sx;
                const A len = (P == P_FP64) ? A(rt.lenD[j]) : A(rt.p[j].len);
                const A sg = sm_s[o];
                A tp;
                const A w = piece(sg, len, tp);
                const A wt = Tacc * w;
#pragma unroll
                for (int cc = 0; cc < C; ++cc) L[cc] = fma(wt, sm_e[cc * TR_REG * TR_PITCH + o], L[cc]);
                Tacc *= tp;
                tau += sg * len;
            }
            Iv<P, C> iv;
#pragma unroll
            for (int cc = 0; cc < C; ++cc) iv.L[cc] = L[cc];
            iv.t = Prec<P>::LOG ? tau : Tacc;
            TLevel<P, C>(pl, q, n).store(u >> n, k, v, iv);
        }
    }
}

// T_n(p, k) from T_{n-1}; p = (x 2^n, v).  Near operand at column 2x, far
// operand at column 2x + 1 shifted by 2k' - 2^{n-1} along v.
template <int P, int C>
__global__ void __launch_bounds__(256) k_merge_up(Plan pl, RowSplit rs, int n) {
    int local;
    const int q = find_quadrant(rs, blockIdx.x, local);   // row = (q, x, k)
    const QuadGeom &g = pl.q[q];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    if (v >= g.V) return;
    const int K = (1 << n) + 1;
    const int x = local / K, k = local - x * K;
    const int m = n - 1, sm = 1 << m;
    TLevel<P, C> Tm(pl, q, m), Tn(pl, q, n);
    const int xn = 2 * x, xf = 2 * x + 1;
    const bool far_ok = xf < g.Un[m];
    auto far = [&](int kk, int vv) {
        return (far_ok && vv >= 0 && vv < g.V) ? Tm.load(xf, kk, vv) : Iv<P, C>::vacuum();
    };
    Iv<P, C> out;
    if ((k & 1) == 0) {                             // Eq. 18
        const int kk = k >> 1;
        out = merge<P, C>(Tm.load(xn, kk, v), far(kk, v + 2 * kk - sm));
    } else {                                        // Eqs. 19-20
        const int kp = (k + 1) >> 1, km = (k - 1) >> 1;
        Iv<P, C> Fp = merge<P, C>(Tm.load(xn, kp, v), far(km, v + 2 * kp - sm));
        Iv<P, C> Fm = merge<P, C>(Tm.load(xn, km, v), far(kp, v + 2 * km - sm));
        out = blend<P, C>(Fm, Fp);
    }
    Tn.store(x, k, v, out);
}

// R_n(p, i) = F_+ + F_-, p = (x 2^n, v), i = ip + 1/2, j_+ = 2ip+1, j_- = 2ip.
template <int P, int C>
__global__ void __launch_bounds__(256) k_merge_down(Plan pl, RowSplit rs, int n) {
    using A = typename Prec<P>::A;
    int local;
    const int q = find_quadrant(rs, blockIdx.x, local);   // row = (q, x, ip)
    const QuadGeom &g = pl.q[q];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    if (v >= g.V) return;
    const int I = 1 << n;
    const int x = local >> n, ip = local & (I - 1);
    const bool top = (n + 1 >= g.N);               // R_N = 0
    const int s = 1 << n;
    A acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = A(0);
    const A Ap = arc<P>(pl, n + 1, 2 * ip + 1), Am = arc<P>(pl, n + 1, 2 * ip);
    RLevel<P, C> Rn(pl, q, n);
    if (x & 1) {
        // Eq. 14: F_+- = A_{n+1}(j) T_n(p, i +- 1/2).L + T_n(p, i +- 1/2).T R_{n+1}(p + v_n(i +- 1/2), j)
        TLevel<P, C> Tn(pl, q, n);
        const int xq = (x + 1) >> 1;
        const bool rq_ok = !top && xq < g.Un[n + 1];
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const int kk = sg == 0 ? ip + 1 : ip;
            const int j = sg == 0 ? 2 * ip + 1 : 2 * ip;
            const A Aj = sg == 0 ? Ap : Am;
            const Iv<P, C> t = Tn.load(x, kk, v);
            const A tr = t.trans();
            const int vq = v + 2 * kk - s;
            if (rq_ok && vq >= 0 && vq < g.V) {
                RLevel<P, C> R1(pl, q, n + 1);
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += fma(Aj, t.L[c], tr * R1.load(xq, j, c, vq));
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) acc[c] += Aj * t.L[c];
            }
        }
    } else {
        // Eqs. 15-17 with Sec. 4.1: F_+- = (R_{n+1}(p, j) + A T_{n+1}(p, 2i +- 1).L
        //                                    + T_{n+1}(p, 2i +- 1).T R_{n+1}(p + v_{n+1}(2i +- 1), j)) / 2
        TLevel<P, C> T1(pl, q, n + 1);
        const int x2 = x >> 1;
        const int s1 = 2 * s;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const int kk = sg == 0 ? 2 * ip + 2 : 2 * ip;
            const int j = sg == 0 ? 2 * ip + 1 : 2 * ip;
            const A Aj = sg == 0 ? Ap : Am;
            const Iv<P, C> t = T1.load(x2, kk, v);
            const A tr = t.trans();
            const int vq = v + 2 * kk - s1;
            A r0[C], r1[C];
#pragma unroll
            for (int c = 0; c < C; ++c) { r0[c] = A(0); r1[c] = A(0); }
            if (!top) {
                RLevel<P, C> R1(pl, q, n + 1);
#pragma unroll
                for (int c = 0; c < C; ++c) r0[c] = R1.load(x2, j, c, v);
                if (x2 + 1 < g.Un[n + 1] && vq >= 0 && vq < g.V) {
#pragma unroll
                    for (int c = 0; c < C; ++c) r1[c] = R1.load(x2 + 1, j, c, vq);
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] += A(0.5) * (r0[c] + fma(Aj, t.L[c], tr * r1[c]));
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) Rn.store(x, ip, c, v, acc[c]);
}

// F[c][y][x] = sum_q R_0^q(u_q + 1, v_q)   (Algorithm 1, Lighting, +1 offset).
template <int P, int C, class OUT>
__global__ void __launch_bounds__(256) k_fluence_sum(Plan pl, OUT *__restrict__ F) {
    using A = typename Prec<P>::A;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= pl.W) return;
    A acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = A(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const QuadGeom &g = pl.q[q];
        int u, v;
        image_to_frame(q, pl.W, pl.H, x, y, u, v);
        if (g.N >= 1 && u + 1 < g.U) {
            RLevel<P, C> R0(pl, q, 0);
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] += R0.load(u + 1, 0, c, v);
        }
    }
    const long long HW = (long long)pl.W * pl.H;
#pragma unroll
    for (int c = 0; c < C; ++c) F[c * HW + (long long)y * pl.W + x] = (OUT)acc[c];
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
static RowSplit make_split(const Plan &pl, int n, int kind) {
    // kind 0: trace rows (q, u); 1: merge-up rows (q, x, k) at level n;
    // 2: merge-down rows (q, x, ip) at level n
    RowSplit rs;
    long long acc = 0;
    for (int q = 0; q < 4; ++q) {
        rs.start[q] = acc;
        const QuadGeom &g = pl.q[q];
        long long rows = 0;
        if (kind == 0) rows = g.U;
        else if (kind == 1) rows = (n <= g.N && n >= 3) ? (long long)g.Un[n] * ((1 << n) + 1) : 0;
        else rows = (n < g.N) ? (long long)g.Un[n] * (1 << n) : 0;
        acc += rows;
    }
    rs.start[4] = acc;
    return rs;
}

static int vblocks(const Plan &pl, int bs) {
    int Vmax = 0;
    for (int q = 0; q < 4; ++q) Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    return (Vmax + bs - 1) / bs;
}

double bytes_T(const Plan &pl, int q, int n) {
    const QuadGeom &g = pl.q[q];
    if (n < 0 || n > g.N) return 0.0;
    const double vt = pl.C * (pl.prec == P_FP32 ? 4.0 : (pl.prec == P_FP64 ? 8.0 : 2.0)) + (pl.prec == P_FP64 ? 8.0 : 4.0);
    return double(g.Un[n]) * ((1 << n) + 1) * g.V * vt;
}

double bytes_R(const Plan &pl, int q, int n) {
    const QuadGeom &g = pl.q[q];
    if (n < 0 || n >= g.N) return 0.0;
    const double vr = pl.C * (pl.prec == P_FP32 ? 4.0 : (pl.prec == P_FP64 ? 8.0 : 2.0));
    return double(g.Un[n]) * (1 << n) * g.V * vr;
}

template <int P, int C>
static cudaError_t fwd_impl(const Plan &pl, const RayTable &rt, const void *e, const void *s, void *F,
                            cudaStream_t st, int *launches, Recorder *rec, bool with_sum) {
    const int bs = 256;
    const int vb = vblocks(pl, bs);
    int Nmax = 0;
    for (int q = 0; q < 4; ++q) Nmax = pl.q[q].N > Nmax ? pl.q[q].N : Nmax;
    const float *ef = (const float *)e, *sf = (const float *)s;
    const double *ed = (const double *)e, *sd = (const double *)s;
    const double esz = P == P_FP64 ? 8.0 : 4.0;
    const double img = double(pl.W) * pl.H;
    {
        double by = img * (pl.C + 1) * esz;
        for (int q = 0; q < 4; ++q)
            for (int n = 0; n <= 2; ++n) by += bytes_T(pl, q, n);
        const size_t smem = sizeof(typename Prec<P>::A) * (C + 1) * TR_REG * TR_PITCH;
        static bool attr_set = false;   // per template instance
        if (!attr_set) {
            cudaFuncSetAttribute(k_trace012<P, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr_set = true;
        }
        dim3 grid((pl.W + TR_TILE - 1) / TR_TILE, (pl.H + TR_TILE - 1) / TR_TILE);
        rec->begin(K_TRACE012, 0, by);
        k_trace012<P, C><<<grid, 256, smem, st>>>(pl, rt, ef, sf, ed, sd);
        rec->end();
        ++*launches;
    }
    for (int n = 3; n <= Nmax; ++n) {
        RowSplit rs = make_split(pl, n, 1);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q)
            if (n <= pl.q[q].N) by += bytes_T(pl, q, n - 1) + bytes_T(pl, q, n);
        dim3 grid((unsigned)rs.start[4], vb);
        rec->begin(K_MERGE_UP, n, by);
        k_merge_up<P, C><<<grid, bs, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    for (int n = Nmax - 1; n >= 0; --n) {
        RowSplit rs = make_split(pl, n, 2);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q) {
            const QuadGeom &g = pl.q[q];
            if (n >= g.N) continue;
            // odd columns of T_n, even directions of T_{n+1}, R_{n+1} once, R_n written
            by += bytes_T(pl, q, n) * (double(g.Un[n] / 2) / g.Un[n]);
            by += bytes_T(pl, q, n + 1) * (double((1 << n) + 1) / ((1 << (n + 1)) + 1));
            by += bytes_R(pl, q, n + 1) + bytes_R(pl, q, n);
        }
        dim3 grid((unsigned)rs.start[4], vb);
        rec->begin(K_MERGE_DOWN, n, by);
        k_merge_down<P, C><<<grid, bs, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    if (with_sum) {
        double by = img * pl.C * esz;
        for (int q = 0; q < 4; ++q) by += bytes_R(pl, q, 0);
        dim3 grid((pl.W + bs - 1) / bs, pl.H);
        rec->begin(K_FLUENCE_SUM, 0, by);
        if (P == P_FP64) k_fluence_sum<P, C, double><<<grid, bs, 0, st>>>(pl, (double *)F);
        else k_fluence_sum<P, C, float><<<grid, bs, 0, st>>>(pl, (float *)F);
        rec->end();
        ++*launches;
    }
    return cudaGetLastError();
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

cudaError_t launch_forward_levels(const Plan &pl, const RayTable &rt, const void *e, const void *s,
                                  cudaStream_t st, int *launches, Recorder *rec) {
    return launch_forward(pl, rt, e, s, nullptr, st, launches, rec);
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
