// bwd_bodies.cuh -- device bodies of the adjoint (reverse-mode) HRC kernels.
//
// The backward pass reads T_0..T_N and R_0..R_{N-1} as the forward pass left
// them in the context's buffers and runs the exact reverse of every forward
// step in gather form: each adjoint entry is written by exactly one thread that
// collects every term feeding it, so there are no atomics and the result is
// deterministic.
//
//   body_adj_sum      : dL/dR_0(x, v) = dL/dF at the pixel of frame (x-1, v)
//   body_adj_R        : dL/dR_{n+1} from dL/dR_n (reverse of Eqs. 14-17; three
//                       terms: odd parent x = 2x'-1, even parents 2x' and 2x'-2)
//   body_adj_T        : the merge-down part of dL/dT_n: odd columns from the
//                       level-n cones (Eq. 14), even directions from the level
//                       n-1 cones at even columns (Eqs. 15-17 with Sec. 4.1)
//   body_adj_merge_up : dL/dT_{n-1} += reverse of Eq. 18 / Eqs. 19-20 (<= 3
//                       terms per entry: near operand or far operand)
//   body_adj_trace    : dL/de, dL/dsigma from dL/dT_0..T_2 (reverse of Trace,
//                       Eq. 9): each pixel gathers every directly traced ray
//                       crossing it, re-tracing the ray from shared memory.
//
// For Merge <r_n + t_n r_f, t_n t_f> with output gradient g:
//   d/dr_n = g.L;  d/dt_n = g.L . r_f + g.T t_f;  d/dr_f = t_n g.L;  d/dt_f = t_n g.T.
// Gradients are taken with respect to the LINEAR transmittance in every
// precision (the log-T forms compute the same function of T).
// Each body processes one block of work at an explicit block index (bx, by).
#pragma once

#include <type_traits>

#include "hrc_internal.cuh"
#include "pair_tile.cuh"
#include "trace_shapes.cuh"

namespace hrc {


using RowSplitB = RowSplit;

__device__ __forceinline__ int quadrant_of(const RowSplitB &rs, long long r, int &local) {
    int q = 0;
    long long base = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (r >= rs.start[j]) { q = j; base = rs.start[j]; }
    local = (int)(r - base);
    return q;
}

// ---------------------------------------------------------------------------
// Reverse of the fluence sum (Algorithm 1, Lighting): F(x,y) += R_0^q(u+1, v),
// so dL/dR_0^q(u+1, v) = dL/dF at the pixel of frame (u, v), and column 0 of
// every dL/dR_0^q is zero.  One CTA per 32 x 32 image tile: the tile of dL/dF
// is read coalesced into shared memory and written out transposed for the
// frames whose v runs along image x.
// ---------------------------------------------------------------------------
template <int P, int C, class GIN>
__device__ __forceinline__ void body_adj_sum(const Plan &pl, const GIN *__restrict__ gF, int bx, int by,
                                             unsigned char *smem) {
    using A = typename Prec<P>::A;
    A (*tile)[32][33] = reinterpret_cast<A (*)[32][33]>(smem);   // [C][32][33]
    const int W = pl.W, H = pl.H;
    const int x0 = bx * 32, y0 = by * 32;
    const long long HW = (long long)W * H;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int r = warp; r < 32; r += 8) {
        const int x = x0 + lane, y = y0 + r;
#pragma unroll
        for (int c = 0; c < C; ++c) tile[c][r][lane] = (x < W && y < H) ? A(gF[c * HW + (long long)y * W + x]) : A(0);
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const QuadGeom &g = pl.q[q];
        if (g.N < 1) continue;
        GRLevel<P, C> gR0(pl, q, 0);
        const bool xu = q < 2;
        const int tu = xu ? x0 : y0, tv = xu ? y0 : x0, ext_u = xu ? W : H;
        const int v = tv + lane;
        if (v >= g.V) continue;
        for (int cidx = warp; cidx < 32; cidx += 8) {
            if (tu + cidx >= ext_u) continue;
            const int u = (q == 0 || q == 2) ? tu + cidx : ext_u - 1 - (tu + cidx);
            const int iy = xu ? lane : cidx, ix = xu ? cidx : lane;
#pragma unroll
            for (int c = 0; c < C; ++c) gR0.store(u + 1 < g.U ? u + 1 : 0, 0, c, v, u + 1 < g.U ? tile[c][iy][ix] : A(0));
            if (u == 0) {
#pragma unroll
                for (int c = 0; c < C; ++c) gR0.store(0, 0, c, v, A(0));
            }
        }
    }
}

// Two consecutive v per thread (E = 2, all neighbour offsets even) or one.
template <class A, int E> struct Lanes {
    A x[E];
};

// ---------------------------------------------------------------------------
// dL/dR_{n+1}(x', j, w).  For cone index j (j + 1/2 at level n+1) the parent
// cone at level n is ip = j >> 1 and its edge direction kk = (j + 1) >> 1
// (sign + for odd j, - for even j), with offset d = 2 kk - 2^n:
//   odd parent x = 2x'-1 (Eq. 14):      T_n(x, kk, w-d).T   * gR_n(x, ip, w-d)
//   even parent x = 2x' (Eq. 16):       1/2                 * gR_n(x, ip, w)
//   even parent x = 2x'-2 (Eq. 17):     T_{n+1}(x'-1, 2kk, w-2d).T / 2 * gR_n(x, ip, w-2d)
// ---------------------------------------------------------------------------
template <int P, int C, int E>
__device__ __forceinline__ void body_adj_R(const Plan &pl, const RowSplitB &rs, int n, long long bx, int by) {
    using A = typename Prec<P>::A;
    int local;
    const int q = quadrant_of(rs, bx, local);   // row = (q, x', j) at level n+1, x' >= 1
    const QuadGeom &g = pl.q[q];
    const int w = E * (by * blockDim.x + threadIdx.x);
    if (w >= g.V) return;
    local += 2 << n;                              // column 0 is dead: its gradient is never read
    const int x1 = local >> (n + 1), j = local & ((2 << n) - 1);
    const int ip = j >> 1, kk = (j + 1) >> 1;
    const int d = 2 * kk - (1 << n);
    GRLevel<P, C> gRn(pl, q, n), gR1(pl, q, n + 1);
    A acc[E][C];
#pragma unroll
    for (int l = 0; l < E; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[l][c] = A(0);
    // terms at v = w - sh (sh even when E = 2): weight * T * gR_n(xp, ip, v)
    auto term = [&](int xp, int sh, A wgt, const TLevel<P, C> *T, int xt, int kt) {
        const int v = w - sh;
#pragma unroll
        for (int l = 0; l < E; ++l) {
            if (v + l < 0 || v + l >= g.V) continue;
            const A t = T ? wgt * T->load(xt, kt, v + l).trans() : wgt;
#pragma unroll
            for (int c = 0; c < C; ++c) acc[l][c] = fma(t, gRn.load(xp, ip, c, v + l), acc[l][c]);
        }
    };
    const int xo = 2 * x1 - 1;
    if (xo < g.Un[n]) {
        TLevel<P, C> Tn(pl, q, n);
        term(xo, d, A(1), &Tn, xo, kk);
    }
    if (2 * x1 < g.Un[n]) term(2 * x1, 0, A(0.5), nullptr, 0, 0);
    const int xe = 2 * x1 - 2;
    if (x1 >= 2 && xe < g.Un[n]) {                // xe = 0 is dead (its gradient is zero)
        TLevel<P, C> T1(pl, q, n + 1);
        term(xe, 2 * d, A(0.5), &T1, x1 - 1, 2 * kk);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (E == 2) gR1.store2(x1, j, c, w, acc[0][c], acc[E - 1][c]);
        else gR1.store(x1, j, c, w, acc[0][c]);
    }
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
template <int P, int C, int E>
__device__ __forceinline__ void body_adj_T(const Plan &pl, const RowSplitB &rs, int n, long long bx, int by) {
    using A = typename Prec<P>::A;
    int local;
    const int q = quadrant_of(rs, bx, local);   // row = (q, x, k) at level n, x >= 1
    const QuadGeom &g = pl.q[q];
    const int v = E * (by * blockDim.x + threadIdx.x);
    if (v >= g.V) return;
    const int K = (1 << n) + 1;
    local += K;
    const int x = local / K, k = local - x * K;
    const int s = 1 << n;
    const int d = 2 * k - s;
    A gL[E][C], gT[E];
#pragma unroll
    for (int l = 0; l < E; ++l) {
        gT[l] = A(0);
#pragma unroll
        for (int c = 0; c < C; ++c) gL[l][c] = A(0);
    }
    // one cone's contribution: arc weight Aw on gR(xg, ip), dot weight dw
    // with R(xr, j, v + d) when rq
    auto cone = [&](const GRLevel<P, C> &gR, int xg, int ip, A Aw, A dw, bool rq, const RLevel<P, C> &R, int xr, int j) {
#pragma unroll
        for (int l = 0; l < E; ++l) {
            const int vv = v + l;
            const bool rok = rq && vv + d >= 0 && vv + d < g.V;
            A dot = A(0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A gr = gR.load(xg, ip, c, vv);
                gL[l][c] = fma(Aw, gr, gL[l][c]);
                if (rok) dot = fma(gr, R.load(xr, j, c, vv + d), dot);
            }
            gT[l] = fma(dw, dot, gT[l]);
        }
    };
    if ((x & 1) && n < g.N) {
        GRLevel<P, C> gRn(pl, q, n);
        const int xq = (x + 1) >> 1;
        const bool rq = (n + 1 < g.N) && xq < g.Un[n + 1];
        RLevel<P, C> R1(pl, q, rq ? n + 1 : n);
        if (k >= 1) cone(gRn, x, k - 1, arc<P>(pl, n + 1, 2 * k - 1), A(1), rq, R1, xq, 2 * k - 1);
        if (k < s) cone(gRn, x, k, arc<P>(pl, n + 1, 2 * k), A(1), rq, R1, xq, 2 * k);
    }
    if (!(k & 1) && n >= 1) {
        const int m = n - 1;
        GRLevel<P, C> gRm(pl, q, m);
        const bool rq = (n < g.N) && x + 1 < g.Un[n];
        RLevel<P, C> Rn(pl, q, rq ? n : 0);
        if (k >= 2) cone(gRm, 2 * x, (k >> 1) - 1, A(0.5) * arc<P>(pl, n, k - 1), A(0.5), rq, Rn, x + 1, k - 1);
        if (k < s) cone(gRm, 2 * x, k >> 1, A(0.5) * arc<P>(pl, n, k), A(0.5), rq, Rn, x + 1, k);
    }
    GTLevel<P, C> gTn(pl, q, n);
#pragma unroll
    for (int l = 0; l < E; ++l)
        if (v + l < g.Vs) gTn.store(x, k, v + l, gL[l], gT[l]);
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
// Two consecutive w per thread (all offsets are even for n >= 3).
// ---------------------------------------------------------------------------
template <int P, int C>
__device__ __forceinline__ void body_adj_merge_up(const Plan &pl, const RowSplitB &rs, int n, long long bx, int by) {
    using A = typename Prec<P>::A;
    constexpr int E = 2;
    int local;
    const int q = quadrant_of(rs, bx, local);   // row = (q, x', kap) at level n-1
    const QuadGeom &g = pl.q[q];
    const int w = E * (by * blockDim.x + threadIdx.x);
    if (w >= g.V) return;
    const int m = n - 1, h = 1 << m;
    const int Km = h + 1;
    local += Km;                                  // x' >= 1: column 0 is dead
    const int x1 = local / Km, kap = local - x1 * Km;
    TLevel<P, C> Tm(pl, q, m);
    GTLevel<P, C> gTm(pl, q, m), gTn(pl, q, n);
    A aL[E][C], aT[E];
#pragma unroll
    for (int l = 0; l < E; ++l) gTm.load(x1, kap, w + l, aL[l], aT[l]);
    if (!(x1 & 1)) {
        const int x = x1 >> 1, xf = x1 + 1;
        const int vf = w + 2 * kap - h;
        const bool xok = xf < g.Un[m];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int kout = t == 0 ? 2 * kap : (t == 1 ? 2 * kap + 1 : 2 * kap - 1);
            const int fdir = t == 0 ? kap : (t == 1 ? kap + 1 : kap - 1);
            if (kout < 0 || kout > 2 * h) continue;
            const A wgt = t == 0 ? A(1) : A(0.5);
            Iv<P, C> fr[E];
            if (xok) Tm.load2_masked(xf, fdir, vf, g.V, fr[0], fr[1]);
            else fr[0] = fr[1] = Iv<P, C>::vacuum();
#pragma unroll
            for (int l = 0; l < E; ++l) {
                A gL[C], gT;
                gTn.load(x, kout, w + l, gL, gT);
                A dT = gT * fr[l].trans();
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    aL[l][c] = fma(wgt, gL[c], aL[l][c]);
                    dT = fma(gL[c], fr[l].L[c], dT);
                }
                aT[l] = fma(wgt, dT, aT[l]);
            }
        }
    } else if (x1 >= 3) {                         // x' = 1 is the far operand of the dead column 0
        const int x = (x1 - 1) >> 1, xn = x1 - 1;
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            const int kout = t == 0 ? 2 * kap : (t == 1 ? 2 * kap + 1 : 2 * kap - 1);
            const int ndir = t == 0 ? kap : (t == 1 ? kap + 1 : kap - 1);
            if (kout < 0 || kout > 2 * h) continue;
            const int v = w - (2 * ndir - h);
            const A wgt = t == 0 ? A(1) : A(0.5);
            if (v < 0 || v >= g.V) continue;          // v even: then v + 1 may still be in range
            Iv<P, C> nr[E];
            Tm.load2(xn, ndir, v, nr[0], nr[1]);
#pragma unroll
            for (int l = 0; l < E; ++l) {
                if (v + l >= g.V) continue;
                A gL[C], gT;
                gTn.load(x, kout, v + l, gL, gT);
                const A tn = wgt * nr[l].trans();
#pragma unroll
                for (int c = 0; c < C; ++c) aL[l][c] = fma(tn, gL[c], aL[l][c]);
                aT[l] = fma(tn, gT, aT[l]);
            }
        }
    }
#pragma unroll
    for (int l = 0; l < E; ++l) gTm.store(x1, kap, w + l, aL[l], aT[l]);
}

// ---------------------------------------------------------------------------
// Reverse of Trace for T_0..T_2.  A ray with pieces m (pixel sigma_m, e_m,
// length l_m, transmittance t_m, weight w_m = l_m phi(sigma_m l_m)) has
//   L = sum_m P_m e_m w_m,  P_m = prod_{m'<m} t_m',  T = prod_m t_m.
// For upstream (gL, gT):
//   dL/de_j     = gL P_j w_j
//   dL/dsigma_j = sum_c gL_c (P_j e_jc dw_j/dsigma - l_j S_jc) - gT l_j T,
//   S_j = sum_{m>j} P_m e_m w_m,   dw/dsigma = l^2 phi'(sigma l).
// Each tile pixel gathers, for every quadrant, ray shape R and piece index
// J, the one ray that crosses it as its piece J (probe = pixel - offset_J),
// and re-traces that ray from the staged tile (shapes unrolled at compile
// time, per-pixel piece factors from the tile, as in the forward trace).
// ---------------------------------------------------------------------------

// dw/dsigma of a half piece of length l with t = exp(-sigma l):
// l^2 phi'(sigma l), phi'(x) = (e^-x (1 + x) - 1) / x^2, by its Taylor
// series near 0.
__device__ __forceinline__ float dw_dsigma(float sg, float len, float t) {
    const float tau = sg * len;
    const float series = len * len * (-0.5f + tau * (1.f / 3.f + tau * (-1.f / 8.f + tau * (1.f / 30.f))));
    return fabsf(tau) < 0.05f ? series : (t * (1.f + tau) - 1.f) / (sg * sg);
}
__device__ __forceinline__ double dw_dsigma(double sg, double len, double t) {
    const double tau = sg * len;
    if (fabs(tau) < 1e-2)
        return len * len * (-0.5 + tau * (1.0 / 3.0 + tau * (-1.0 / 8.0 + tau * (1.0 / 30.0 + tau * (-1.0 / 144.0 + tau * (1.0 / 840.0))))));
    return (t * (1.0 + tau) - 1.0) / (sg * sg);
}

// Re-trace pieces M .. END-1 of a ray; piece J is the one at the gathering
// pixel.  Accumulates the attenuated radiance of all pieces (Ltot) and of
// pieces <= J (Lle), and records P_J, the half-piece factors of J, its
// extinction and emission.
template <class A, int C, int M, int END, int J>
__device__ __forceinline__ void adj_retrace(const PairTile<A, C> &tt, int base, int su, A &Pp, A (&Ltot)[C],
                                            A (&Lle)[C], A &Pj, A &tj, A &wj, A &sj, A (&ej)[C]) {
    if constexpr (M < END) {
        using pc = PieceAt<M>;
        const int o = base + pc::du * su + pc::dv;
        A t, w, em[C], sg;
        tt.piece(pc::cls, o, t, w);
        tt.emis(o, em, sg);
        if constexpr (M == J) {
            tj = t;
            wj = w;
            sj = sg;
            Pj = Pp;
#pragma unroll
            for (int c = 0; c < C; ++c) ej[c] = em[c];
        }
        if constexpr (pc::full != 0) {
            w = w * (A(1) + t);
            t = t * t;
        }
        const A pw = Pp * w;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            Ltot[c] = fma(pw, em[c], Ltot[c]);
            if constexpr (M <= J) Lle[c] = fma(pw, em[c], Lle[c]);
        }
        Pp *= t;
        adj_retrace<A, C, M + 1, END, J>(tt, base, su, Pp, Ltot, Lle, Pj, tj, wj, sj, ej);
    }
}

template <int P, int C, int R, int J>
__device__ __forceinline__ void adj_gather(const Plan &pl, const PairTile<typename Prec<P>::A, C> &tt, int q, int nmax,
                                           int V, int us, int vs, int base, int su,
                                           typename Prec<P>::A (&dE)[C], typename Prec<P>::A &dS) {
    using A = typename Prec<P>::A;
    using ray = RayAt<R>;
    if constexpr (J < ray::end) {
        using pc = PieceAt<J>;
        const int up = us - pc::du, vp = vs - pc::dv;
        if (up >= 1 && !(up & ((1 << ray::n) - 1)) && vp >= 0 && vp < V) {   // probes at u = 0 are dead
            A gL[C], gT;
            GTLevel<P, C>(pl, q, ray::n).load(up >> ray::n, ray::k, vp, gL, gT);
            const int pbase = base - pc::du * su - pc::dv;
            A Pp = A(1), Pj = A(0), tj = A(1), wj = A(0), sj = A(0);
            A Ltot[C], Lle[C], ej[C];
#pragma unroll
            for (int c = 0; c < C; ++c) { Ltot[c] = A(0); Lle[c] = A(0); ej[c] = A(0); }
            adj_retrace<A, C, ray::begin, ray::end, J>(tt, pbase, su, Pp, Ltot, Lle, Pj, tj, wj, sj, ej);
            const A lh = class_len<A>(pc::cls);
            A d = dw_dsigma(sj, lh, tj);
            A wq = wj, len = lh;
            if constexpr (pc::full != 0) {            // w2 = w (1 + t), dw2 = d (1 + t) - l t w
                d = fma(d, A(1) + tj, -lh * tj * wj);
                wq = wj * (A(1) + tj);
                len = A(2) * lh;
            }
            A g = -gT * len * Pp;                     // Pp is now the ray's total T
#pragma unroll
            for (int c = 0; c < C; ++c) {
                dE[c] = fma(gL[c], Pj * wq, dE[c]);
                g = fma(gL[c], Pj * ej[c] * d - len * (Ltot[c] - Lle[c]), g);
            }
            dS += g;
        }
        adj_gather<P, C, R, J + 1>(pl, tt, q, nmax, V, us, vs, base, su, dE, dS);
    }
}

template <int P, int C, int R>
__device__ __forceinline__ void adj_ray(const Plan &pl, const PairTile<typename Prec<P>::A, C> &tt, int q, int nmax,
                                        int V, int us, int vs, int base, int su,
                                        typename Prec<P>::A (&dE)[C], typename Prec<P>::A &dS) {
    if constexpr (R < HRC_MAXRAY) {
        if (RayAt<R>::n <= nmax) adj_gather<P, C, R, RayAt<R>::begin>(pl, tt, q, nmax, V, us, vs, base, su, dE, dS);
        adj_ray<P, C, R + 1>(pl, tt, q, nmax, V, us, vs, base, su, dE, dS);
    }
}

// Shared memory of the adjoint trace: the pair tile, then (pair 0 only) a
// transposed accumulator so that dL/de and dL/dsigma leave coalesced.
template <class A, int C> constexpr size_t adj_trace_smem() {
    return PairTile<A, C>::bytes() + sizeof(A) * (C + 1) * PT_V * (PT_U + 1);
}

// dL/de and dL/dsigma of quadrant pair `pair` for one tile.  Each thread
// owns the two pixels of its tile columns for both frames of the pair and
// accumulates in registers.  Pair 0 writes the image gradients, pair 1
// (launched after it) adds to them.
template <int P, int C, class IN>
__device__ __forceinline__ void body_adj_trace(const Plan &pl, const IN *__restrict__ e, const IN *__restrict__ s,
                                               IN *__restrict__ ge, IN *__restrict__ gs, int pair, int bx, int by,
                                               unsigned char *smem) {
    using A = typename Prec<P>::A;
    PairTile<A, C> tt(smem);
    A *acc = reinterpret_cast<A *>(smem + PairTile<A, C>::bytes());   // [C+1][PT_V][PT_U+1]
    const int W = pl.W, H = pl.H;
    const long long HW = (long long)W * H;
    const int x0 = pair == 0 ? bx * PT_U : bx * PT_V;
    const int y0 = pair == 0 ? by * PT_V : by * PT_U;
    tt.stage(pair, W, H, x0, y0, e, s);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll 1
    for (int i = 0; i < 2; ++i) {
        const int c = 8 * i + ((warp + i) & 7);
        A dE[C], dS = A(0);
#pragma unroll
        for (int cc = 0; cc < C; ++cc) dE[cc] = A(0);
#pragma unroll 1
        for (int qq = 0; qq < 2; ++qq) {
            const int q = 2 * pair + qq;
            const QuadGeom &g = pl.q[q];
            if (g.N < 1) continue;
            const int nmax = g.N < 2 ? g.N : 2;
            const PairGeom pg = pair_geom(pl, q, x0, y0, c, lane);
            if (!pg.valid) continue;
            adj_ray<P, C, 0>(pl, tt, q, nmax, g.V, pg.u, pg.v, pg.base, pg.su, dE, dS);
        }
        // image pixel: pair 0 (c along x, lane along y); pair 1 (c along y, lane along x)
        const int x = pair == 0 ? x0 + c : x0 + lane, y = pair == 0 ? y0 + lane : y0 + c;
        if (x >= W || y >= H) continue;
        const long long pix = (long long)y * W + x;
        if (pair == 0) {
#pragma unroll
            for (int cc = 0; cc < C; ++cc) acc[(cc * PT_V + lane) * (PT_U + 1) + c] = dE[cc];
            acc[(C * PT_V + lane) * (PT_U + 1) + c] = dS;
        } else {
#pragma unroll
            for (int cc = 0; cc < C; ++cc) ge[cc * HW + pix] = IN(A(ge[cc * HW + pix]) + dE[cc]);
            gs[pix] = IN(A(gs[pix]) + dS);
        }
    }
    if (pair == 0) {
        __syncthreads();
        for (int k = threadIdx.x; k < PT_U * PT_V; k += blockDim.x) {
            const int ly = k / PT_U, lx = k - ly * PT_U;
            const int x = x0 + lx, y = y0 + ly;
            if (x >= W || y >= H) continue;
            const long long pix = (long long)y * W + x;
#pragma unroll
            for (int cc = 0; cc < C; ++cc) ge[cc * HW + pix] = IN(acc[(cc * PT_V + ly) * (PT_U + 1) + lx]);
            gs[pix] = IN(acc[(C * PT_V + ly) * (PT_U + 1) + lx]);
        }
    }
}

}  // namespace hrc
