// kernels_bwd.cu -- adjoint (reverse-mode) HRC kernels for sm_103a.
//
// The backward pass recomputes T_0..T_N and R_0..R_{N-1} from the inputs
// (forward kernels), then runs the exact reverse of every forward step in
// gather form: each adjoint entry is written by exactly one thread that
// collects every term feeding it, so there are no atomics and the result is
// deterministic.
//
//   k_adj_sum      : dL/dR_0(x, v) = dL/dF at the pixel of frame (x-1, v)
//   k_adj_R        : dL/dR_{n+1} from dL/dR_n (reverse of Eqs. 14-17; three
//                    terms: odd parent x = 2x'-1, even parents 2x' and 2x'-2)
//   k_adj_T        : the merge-down part of dL/dT_n: odd columns from the
//                    level-n cones (Eq. 14), even directions from the level
//                    n-1 cones at even columns (Eqs. 15-17 with Sec. 4.1)
//   k_adj_merge_up : dL/dT_{n-1} += reverse of Eq. 18 / Eqs. 19-20 (<= 3
//                    terms per entry: near operand or far operand)
//   k_adj_trace    : dL/de, dL/dsigma from dL/dT_0..T_2 (reverse of Trace,
//                    Eq. 9): each pixel gathers every directly traced ray
//                    crossing it, re-tracing the ray from shared memory.
//
// For Merge <r_n + t_n r_f, t_n t_f> with output gradient g:
//   d/dr_n = g.L;  d/dt_n = g.L . r_f + g.T t_f;  d/dr_f = t_n g.L;  d/dt_f = t_n g.T.
// Gradients are taken with respect to the LINEAR transmittance in every
// precision (the log-T forms compute the same function of T).
#include <type_traits>

#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

namespace {

struct RowSplitB {
    long long start[5];
};

__device__ __forceinline__ int quadrant_of(const RowSplitB &rs, long long r, int &local) {
    int q = 0;
    long long base = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (r >= rs.start[j]) { q = j; base = rs.start[j]; }
    local = (int)(r - base);
    return q;
}

}  // namespace

// ---------------------------------------------------------------------------
// Reverse of the fluence sum (Algorithm 1, Lighting): F(x,y) += R_0^q(u+1, v)
// ---------------------------------------------------------------------------
template <int P, int C, class GIN>
__global__ void __launch_bounds__(256) k_adj_sum(Plan pl, RowSplitB rs, const GIN *__restrict__ gF) {
    using A = typename Prec<P>::A;
    int x;
    const int q = quadrant_of(rs, blockIdx.x, x);   // row = (q, x) of R_0
    const QuadGeom &g = pl.q[q];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    if (v >= g.V) return;
    GRLevel<P, C> gR0(pl, q, 0);
    const long long HW = (long long)pl.W * pl.H;
    int px = 0, py = 0;
    if (x >= 1) frame_to_image(q, pl.W, pl.H, x - 1, v, px, py);
#pragma unroll
    for (int c = 0; c < C; ++c)
        gR0.store(x, 0, c, v, x >= 1 ? A(gF[c * HW + (long long)py * pl.W + px]) : A(0));
}

// ---------------------------------------------------------------------------
// dL/dR_{n+1}(x', j, w).  For cone index j (j + 1/2 at level n+1) the parent
// cone at level n is ip = j >> 1 and its edge direction kk = (j + 1) >> 1
// (sign + for odd j, - for even j), with offset d = 2 kk - 2^n:
//   odd parent x = 2x'-1 (Eq. 14):      T_n(x, kk, w-d).T   * gR_n(x, ip, w-d)
//   even parent x = 2x' (Eq. 16):       1/2                 * gR_n(x, ip, w)
//   even parent x = 2x'-2 (Eq. 17):     T_{n+1}(x'-1, 2kk, w-2d).T / 2 * gR_n(x, ip, w-2d)
// ---------------------------------------------------------------------------
template <int P, int C>
__global__ void __launch_bounds__(256) k_adj_R(Plan pl, RowSplitB rs, int n) {
    using A = typename Prec<P>::A;
    int local;
    const int q = quadrant_of(rs, blockIdx.x, local);   // row = (q, x', j) at level n+1
    const QuadGeom &g = pl.q[q];
    const int w = blockIdx.y * blockDim.x + threadIdx.x;
    if (w >= g.V) return;
    const int x1 = local >> (n + 1), j = local & ((2 << n) - 1);
    const int ip = j >> 1, kk = (j + 1) >> 1;
    const int d = 2 * kk - (1 << n);
    GRLevel<P, C> gRn(pl, q, n), gR1(pl, q, n + 1);
    A acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = A(0);
    const int xo = 2 * x1 - 1;
    if (x1 >= 1 && xo < g.Un[n]) {
        const int v = w - d;
        if (v >= 0 && v < g.V) {
            const A t = TLevel<P, C>(pl, q, n).load(xo, kk, v).trans();
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fma(t, gRn.load(xo, ip, c, v), acc[c]);
        }
    }
    if (2 * x1 < g.Un[n]) {
#pragma unroll
        for (int c = 0; c < C; ++c) acc[c] = fma(A(0.5), gRn.load(2 * x1, ip, c, w), acc[c]);
    }
    const int xe = 2 * x1 - 2;
    if (x1 >= 1 && xe < g.Un[n]) {
        const int v = w - 2 * d;
        if (v >= 0 && v < g.V) {
            const A t = A(0.5) * TLevel<P, C>(pl, q, n + 1).load(x1 - 1, 2 * kk, v).trans();
#pragma unroll
            for (int c = 0; c < C; ++c) acc[c] = fma(t, gRn.load(xe, ip, c, v), acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) gR1.store(x1, j, c, w, acc[c]);
}

// ---------------------------------------------------------------------------
// Merge-down part of dL/dT_n(x, k, v); every entry is written (zeros where no
// cone reads it).
//   odd x (Eq. 14 at level n): cone k-1 uses edge k as F_+ (arc j = 2k-1),
//     cone k uses it as F_- (arc j = 2k); far fluence R_{n+1}((x+1)/2, j, v+d).
//   even k (Eqs. 15-17 at level n-1, even column 2x): cone k/2-1 uses
//     T_n(x, k) as F_+ (arc A_n(k-1)), cone k/2 as F_- (arc A_n(k)), each
//     with weight 1/2; far fluence R_n(x+1, j, v+d), d = 2k - 2^n.
// ---------------------------------------------------------------------------
template <int P, int C>
__global__ void __launch_bounds__(256) k_adj_T(Plan pl, RowSplitB rs, int n) {
    using A = typename Prec<P>::A;
    int local;
    const int q = quadrant_of(rs, blockIdx.x, local);   // row = (q, x, k) at level n
    const QuadGeom &g = pl.q[q];
    const int v = blockIdx.y * blockDim.x + threadIdx.x;
    if (v >= g.V) return;
    const int K = (1 << n) + 1;
    const int x = local / K, k = local - x * K;
    const int s = 1 << n;
    const int d = 2 * k - s;
    A gL[C];
#pragma unroll
    for (int c = 0; c < C; ++c) gL[c] = A(0);
    A gT = A(0);
    if ((x & 1) && n < g.N) {
        GRLevel<P, C> gRn(pl, q, n);
        const int xq = (x + 1) >> 1;
        const bool rq = (n + 1 < g.N) && xq < g.Un[n + 1] && v + d >= 0 && v + d < g.V;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const int ip = sg == 0 ? k - 1 : k;          // F_+ of cone k-1, F_- of cone k
            if (ip < 0 || ip >= s) continue;
            const int j = sg == 0 ? 2 * k - 1 : 2 * k;
            const A Aj = arc<P>(pl, n + 1, j);
            A dot = A(0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A gr = gRn.load(x, ip, c, v);
                gL[c] = fma(Aj, gr, gL[c]);
                if (rq) dot = fma(gr, RLevel<P, C>(pl, q, n + 1).load(xq, j, c, v + d), dot);
            }
            gT += dot;
        }
    }
    if (!(k & 1) && n >= 1) {
        const int m = n - 1;
        GRLevel<P, C> gRm(pl, q, m);
        const int xe = 2 * x;                              // even column of level n-1
        const bool rq = (n < g.N) && x + 1 < g.Un[n] && v + d >= 0 && v + d < g.V;
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const int ip = sg == 0 ? (k >> 1) - 1 : (k >> 1);
            if (ip < 0 || ip >= (1 << m)) continue;
            const int j = sg == 0 ? k - 1 : k;
            const A Aj = A(0.5) * arc<P>(pl, n, j);
            A dot = A(0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A gr = gRm.load(xe, ip, c, v);
                gL[c] = fma(Aj, gr, gL[c]);
                if (rq) dot = fma(gr, RLevel<P, C>(pl, q, n).load(x + 1, j, c, v + d), dot);
            }
            gT = fma(A(0.5), dot, gT);
        }
    }
    GTLevel<P, C>(pl, q, n).store(x, k, v, gL, gT);
}

// ---------------------------------------------------------------------------
// dL/dT_{n-1}(x', kap, w) += reverse of the level-n merge up.  h = 2^{n-1}.
//  even x' (near operand of column x = x'/2, far column x'+1, far offset
//  w + 2 kap - h, shared by the three outputs):
//    k = 2 kap (weight 1, far dir kap), k = 2 kap + 1 (F_-, weight 1/2, far
//    dir kap + 1), k = 2 kap - 1 (F_+, weight 1/2, far dir kap - 1)
//  odd x' (far operand of column x = (x'-1)/2, near column x'-1):
//    k = 2 kap at v = w - (2 kap - h) (near dir kap, weight 1),
//    k = 2 kap + 1 at v = w - (2 kap + 2 - h) (F_+, near dir kap + 1, 1/2),
//    k = 2 kap - 1 at v = w - (2 kap - 2 - h) (F_-, near dir kap - 1, 1/2)
// ---------------------------------------------------------------------------
template <int P, int C>
__global__ void __launch_bounds__(256) k_adj_merge_up(Plan pl, RowSplitB rs, int n) {
    using A = typename Prec<P>::A;
    int local;
    const int q = quadrant_of(rs, blockIdx.x, local);   // row = (q, x', kap) at level n-1
    const QuadGeom &g = pl.q[q];
    const int w = blockIdx.y * blockDim.x + threadIdx.x;
    if (w >= g.V) return;
    const int m = n - 1, h = 1 << m;
    const int Km = h + 1;
    const int x1 = local / Km, kap = local - x1 * Km;
    TLevel<P, C> Tm(pl, q, m);
    GTLevel<P, C> gTm(pl, q, m), gTn(pl, q, n);
    A aL[C], aT;
    gTm.load(x1, kap, w, aL, aT);
    if (!(x1 & 1)) {
        const int x = x1 >> 1, xf = x1 + 1;
        const int vf = w + 2 * kap - h;
        const bool fok = xf < g.Un[m] && vf >= 0 && vf < g.V;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int kout = t == 0 ? 2 * kap : (t == 1 ? 2 * kap + 1 : 2 * kap - 1);
            const int fdir = t == 0 ? kap : (t == 1 ? kap + 1 : kap - 1);
            if (kout < 0 || kout > 2 * h) continue;
            const A wgt = t == 0 ? A(1) : A(0.5);
            A gL[C], gT;
            gTn.load(x, kout, w, gL, gT);
            const Iv<P, C> fr = fok ? Tm.load(xf, fdir, vf) : Iv<P, C>::vacuum();
            A dT = gT * fr.trans();
#pragma unroll
            for (int c = 0; c < C; ++c) {
                aL[c] = fma(wgt, gL[c], aL[c]);
                dT = fma(gL[c], fr.L[c], dT);
            }
            aT = fma(wgt, dT, aT);
        }
    } else {
        const int x = (x1 - 1) >> 1, xn = x1 - 1;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int kout = t == 0 ? 2 * kap : (t == 1 ? 2 * kap + 1 : 2 * kap - 1);
            const int ndir = t == 0 ? kap : (t == 1 ? kap + 1 : kap - 1);
            if (kout < 0 || kout > 2 * h) continue;
            const int v = w - (2 * ndir - h);
            if (v < 0 || v >= g.V) continue;
            const A wgt = t == 0 ? A(1) : A(0.5);
            A gL[C], gT;
            gTn.load(x, kout, v, gL, gT);
            const A tn = wgt * Tm.load(xn, ndir, v).trans();
#pragma unroll
            for (int c = 0; c < C; ++c) aL[c] = fma(tn, gL[c], aL[c]);
            aT = fma(tn, gT, aT);
        }
    }
    gTm.store(x1, kap, w, aL, aT);
}

// ---------------------------------------------------------------------------
// Reverse of Trace for T_0..T_2.  A ray with pieces m (pixel sigma_m, e_m,
// length l_m, transmittance t_m, weight w_m = l_m phi(sigma_m l_m)) has
//   L = sum_m P_m e_m w_m,  P_m = prod_{m'<m} t_m',  T = prod_m t_m.
// For upstream (gL, gT):
//   dL/de_j     = gL P_j w_j
//   dL/dsigma_j = sum_c gL_c (P_j e_jc l_j^2 phi'(sigma_j l_j) - l_j S_jc) - gT l_j T,
//   S_j = sum_{m>j} P_m e_m w_m.
// Each tile pixel gathers, for every quadrant, ray shape and piece index j,
// the one ray that crosses it as its piece j (probe = pixel - offset_j).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dphi_l2(float sg, float len, float tp) {
    // l^2 phi'(sigma l), phi'(t) = (e^-t (1 + t) - 1) / t^2
    const float tau = sg * len;
    const float series = len * len * (-0.5f + tau * (1.f / 3.f + tau * (-1.f / 8.f + tau * (1.f / 30.f))));
    return fabsf(tau) < 0.05f ? series : (tp * (1.f + tau) - 1.f) / (sg * sg);
}
__device__ __forceinline__ double dphi_l2(double sg, double len, double tp) {
    const double tau = sg * len;
    if (fabs(tau) < 1e-2)
        return len * len * (-0.5 + tau * (1.0 / 3.0 + tau * (-1.0 / 8.0 + tau * (1.0 / 30.0 + tau * (-1.0 / 144.0 + tau * (1.0 / 840.0))))));
    return (tp * (1.0 + tau) - 1.0) / (sg * sg);
}

__device__ __forceinline__ float piece_b(float sg, float len, float &tp) {
    const float tau = sg * len;
    tp = __expf(-tau);
    const float series = len * (1.f - tau * (0.5f - tau * (1.f / 6.f - tau * (1.f / 24.f))));
    return fabsf(tau) < 0.03f ? series : (1.f - tp) / sg;
}
__device__ __forceinline__ double piece_b(double sg, double len, double &tp) {
    const double tau = sg * len;
    const double m = expm1(-tau);
    tp = 1.0 + m;
    return sg != 0.0 ? -m / sg : len;
}

constexpr int TB_TILE = 32, TB_HALO = 4, TB_REG = TB_TILE + 2 * TB_HALO, TB_PITCH = TB_REG + 1;

template <int P, int C, class IN>
__global__ void __launch_bounds__(256) k_adj_trace(Plan pl, RayTable rt, const IN *__restrict__ e,
                                                   const IN *__restrict__ s, IN *__restrict__ ge,
                                                   IN *__restrict__ gs) {
    using A = typename Prec<P>::A;
    extern __shared__ __align__(16) unsigned char tb_smem[];
    A *sm_s = reinterpret_cast<A *>(tb_smem);                 // [TB_REG][TB_PITCH]
    A *sm_e = sm_s + TB_REG * TB_PITCH;                        // [C][TB_REG][TB_PITCH]
    A *acc = sm_e + C * TB_REG * TB_PITCH;                     // [C+1][TB_TILE][TB_TILE + 1]
    constexpr int AP = TB_TILE + 1;
    const int W = pl.W, H = pl.H;
    const int x0 = blockIdx.x * TB_TILE, y0 = blockIdx.y * TB_TILE;
    const long long HW = (long long)W * H;
    for (int i = threadIdx.x; i < TB_REG * TB_REG; i += blockDim.x) {
        const int ry = i / TB_REG, rx = i - ry * TB_REG;
        const int x = x0 - TB_HALO + rx, y = y0 - TB_HALO + ry;
        const bool in = x >= 0 && x < W && y >= 0 && y < H;
        const long long pix = (long long)y * W + x;
        sm_s[ry * TB_PITCH + rx] = in ? A(s[pix]) : A(0);
#pragma unroll
        for (int c = 0; c < C; ++c) sm_e[(c * TB_REG + ry) * TB_PITCH + rx] = in ? A(e[c * HW + pix]) : A(0);
    }
    for (int i = threadIdx.x; i < (C + 1) * TB_TILE * AP; i += blockDim.x) acc[i] = A(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int q = 0; q < 4; ++q) {
        const QuadGeom &g = pl.q[q];
        const int nmax = g.N < 2 ? g.N : 2;
        const bool xu = q < 2;
        const int tu = xu ? x0 : y0, tv = xu ? y0 : x0;
        const int ext_u = xu ? W : H;
        const int sgn = (q == 0 || q == 2) ? 1 : -1;
        const int vs = tv + lane;
        for (int c = warp; c < TB_TILE; c += nwarp) {
            if (tu + c >= ext_u || vs >= g.V) continue;
            const int us = (q == 0 || q == 2) ? tu + c : ext_u - 1 - (tu + c);
            A dE[C], dS = A(0);
#pragma unroll
            for (int cc = 0; cc < C; ++cc) dE[cc] = A(0);
            for (int r = 0; r < HRC_MAXRAY; ++r) {
                const int n = r < 2 ? 0 : (r < 5 ? 1 : 2);
                if (n > nmax) break;
                const int k = r - (n == 0 ? 0 : (n == 1 ? 2 : 5));
                const int j0 = rt.start[r], j1 = rt.start[r + 1];
                GTLevel<P, C> gT(pl, q, n);
                for (int j = j0; j < j1; ++j) {
                    const int up = us - rt.p[j].du, vp = vs - rt.p[j].dv;
                    if (up < 0 || (up & ((1 << n) - 1)) || vp < 0 || vp >= g.V) continue;
                    A gL[C], gTT;
                    gT.load(up >> n, k, vp, gL, gTT);
                    // re-trace the ray from probe (up, vp): tile coords of piece m are
                    // (c - du_j + du_m, lane - dv_j + dv_m) along the (u, v) axes
                    A Pp = A(1), Pj = A(0), wj = A(0), tj = A(1), sgj = A(0), lenj = A(0);
                    A Ltot[C], Lle[C], ej[C];
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) { Ltot[cc] = A(0); Lle[cc] = A(0); ej[cc] = A(0); }
                    for (int mm = j0; mm < j1; ++mm) {
                        const int a = TB_HALO + c + sgn * (rt.p[mm].du - rt.p[j].du);
                        const int b = TB_HALO + lane + (rt.p[mm].dv - rt.p[j].dv);
                        const int o = (xu ? b : a) * TB_PITCH + (xu ? a : b);
                        const A len = (P == P_FP64) ? A(rt.lenD[mm]) : A(rt.p[mm].len);
                        const A sg = sm_s[o];
                        A tp;
                        const A wgt = piece_b(sg, len, tp);
                        const A pw = Pp * wgt;
#pragma unroll
                        for (int cc = 0; cc < C; ++cc) {
                            const A em = sm_e[cc * TB_REG * TB_PITCH + o];
                            Ltot[cc] = fma(pw, em, Ltot[cc]);
                            if (mm <= j) Lle[cc] = fma(pw, em, Lle[cc]);
                            if (mm == j) ej[cc] = em;
                        }
                        if (mm == j) { Pj = Pp; wj = wgt; tj = tp; sgj = sg; lenj = len; }
                        Pp *= tp;
                    }
                    const A Ttot = Pp;
                    const A dd = dphi_l2(sgj, lenj, tj);
                    A gsig = -gTT * lenj * Ttot;
#pragma unroll
                    for (int cc = 0; cc < C; ++cc) {
                        dE[cc] = fma(gL[cc], Pj * wj, dE[cc]);
                        gsig = fma(gL[cc], Pj * ej[cc] * dd - lenj * (Ltot[cc] - Lle[cc]), gsig);
                    }
                    dS += gsig;
                }
            }
            // image pixel of this frame pixel, relative to the tile
            const int ix = xu ? c : lane, iy = xu ? lane : c;
#pragma unroll
            for (int cc = 0; cc < C; ++cc) acc[(cc * TB_TILE + iy) * AP + ix] += dE[cc];
            acc[(C * TB_TILE + iy) * AP + ix] += dS;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < TB_TILE * TB_TILE; i += blockDim.x) {
        const int iy = i / TB_TILE, ix = i - iy * TB_TILE;
        const int x = x0 + ix, y = y0 + iy;
        if (x >= W || y >= H) continue;
        const long long pix = (long long)y * W + x;
#pragma unroll
        for (int cc = 0; cc < C; ++cc) ge[cc * HW + pix] = IN(acc[(cc * TB_TILE + iy) * AP + ix]);
        gs[pix] = IN(acc[(C * TB_TILE + iy) * AP + ix]);
    }
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
        else if (kind == 1) rows = (n + 1 < g.N) ? (long long)g.Un[n + 1] * (2 << n) : 0;
        else if (kind == 2) rows = (g.N >= 1 && n <= g.N) ? (long long)g.Un[n] * ((1 << n) + 1) : 0;
        else rows = (n >= 3 && n <= g.N) ? (long long)g.Un[n - 1] * ((1 << (n - 1)) + 1) : 0;
        acc += rows;
    }
    rs.start[4] = acc;
    return rs;
}

int vblocks_b(const Plan &pl, int bs) {
    int Vmax = 0;
    for (int q = 0; q < 4; ++q) Vmax = pl.q[q].V > Vmax ? pl.q[q].V : Vmax;
    return (Vmax + bs - 1) / bs;
}

}  // namespace

template <int P, int C>
static cudaError_t bwd_impl(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, cudaStream_t st, int *launches, Recorder *rec) {
    using IN = typename std::conditional<P == P_FP64, double, float>::type;
    const int bs = 256, vb = vblocks_b(pl, bs);
    int Nmax = 0;
    for (int q = 0; q < 4; ++q) Nmax = pl.q[q].N > Nmax ? pl.q[q].N : Nmax;
    const double ab = P == P_FP64 ? 8.0 : 4.0;
    const double img = double(pl.W) * pl.H;
    auto gTbytes = [&](int q, int n) {
        const QuadGeom &g = pl.q[q];
        return (n < 0 || n > g.N) ? 0.0 : double(g.Un[n]) * ((1 << n) + 1) * g.V * (pl.C + 1) * ab;
    };
    auto gRbytes = [&](int q, int n) {
        const QuadGeom &g = pl.q[q];
        return (n < 0 || n >= g.N) ? 0.0 : double(g.Un[n]) * (1 << n) * g.V * pl.C * ab;
    };
    // forward recompute of every T and R level (no fluence sum)
    cudaError_t err = launch_forward_levels(pl, rt, e, s, st, launches, rec);
    if (err != cudaSuccess) return err;
    {
        RowSplitB rs = split_rows(pl, 0, 0);
        if (rs.start[4] > 0) {
            double by = img * pl.C * ab;
            for (int q = 0; q < 4; ++q) by += gRbytes(q, 0);
            rec->begin(K_ADJ_SUM, 0, by);
            k_adj_sum<P, C, IN><<<dim3((unsigned)rs.start[4], vb), bs, 0, st>>>(pl, rs, (const IN *)gF);
            rec->end();
            ++*launches;
        }
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
        k_adj_R<P, C><<<dim3((unsigned)rs.start[4], vb), bs, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    for (int n = 0; n <= Nmax; ++n) {
        RowSplitB rs = split_rows(pl, 2, n);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q)
            if (pl.q[q].N >= 1 && n <= pl.q[q].N)
                by += gTbytes(q, n) + gRbytes(q, n) + gRbytes(q, n - 1) + bytes_R(pl, q, n) + bytes_R(pl, q, n + 1);
        rec->begin(K_ADJ_MERGE_DOWN, n, by);
        k_adj_T<P, C><<<dim3((unsigned)rs.start[4], vb), bs, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    for (int n = Nmax; n >= 3; --n) {
        RowSplitB rs = split_rows(pl, 3, n);
        if (rs.start[4] == 0) continue;
        double by = 0;
        for (int q = 0; q < 4; ++q)
            if (n <= pl.q[q].N) by += 2 * gTbytes(q, n - 1) + gTbytes(q, n) + bytes_T(pl, q, n - 1);
        rec->begin(K_ADJ_MERGE_UP, n, by);
        k_adj_merge_up<P, C><<<dim3((unsigned)rs.start[4], vb), bs, 0, st>>>(pl, rs, n);
        rec->end();
        ++*launches;
    }
    {
        using A = typename Prec<P>::A;
        const size_t smem = sizeof(A) * ((C + 1) * TB_REG * TB_PITCH + (C + 1) * TB_TILE * (TB_TILE + 1));
        static bool attr_set = false;
        if (!attr_set) {
            cudaFuncSetAttribute(k_adj_trace<P, C, IN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            attr_set = true;
        }
        double by = img * (pl.C + 1) * ab * 2;
        for (int q = 0; q < 4; ++q)
            for (int n = 0; n <= 2; ++n) by += gTbytes(q, n);
        dim3 grid((pl.W + TB_TILE - 1) / TB_TILE, (pl.H + TB_TILE - 1) / TB_TILE);
        rec->begin(K_ADJ_TRACE, 0, by);
        k_adj_trace<P, C, IN><<<grid, 256, smem, st>>>(pl, rt, (const IN *)e, (const IN *)s, (IN *)ge, (IN *)gs);
        rec->end();
        ++*launches;
    }
    return cudaGetLastError();
}

template <int P>
static cudaError_t bwd_prec(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, cudaStream_t st, int *launches, Recorder *rec) {
    switch (pl.C) {
    case 1: return bwd_impl<P, 1>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    case 2: return bwd_impl<P, 2>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    case 3: return bwd_impl<P, 3>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    default: return bwd_impl<P, 4>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    }
}

cudaError_t launch_backward(const Plan &pl, const RayTable &rt, const void *e, const void *s, const void *gF,
                            void *ge, void *gs, cudaStream_t st, int *launches, Recorder *rec) {
    switch (pl.prec) {
    case P_FP32: return bwd_prec<P_FP32>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    case P_FP16: return bwd_prec<P_FP16>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    case P_BF16: return bwd_prec<P_BF16>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    default: return bwd_prec<P_FP64>(pl, rt, e, s, gF, ge, gs, st, launches, rec);
    }
}

}  // namespace hrc
