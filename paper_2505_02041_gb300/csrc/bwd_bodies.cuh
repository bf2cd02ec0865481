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
//   body_adj_merge_up : dL/dT_{n-1} = its merge-down part (as body_adj_T,
//                       fused) + reverse of Eq. 18 / Eqs. 19-20 (<= 3 terms
//                       per entry: near operand or far operand)
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < 32; r += nw) {
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
        for (int cidx = warp; cidx < 32; cidx += nw) {
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
        if (E == 2 && v >= 0 && v + 1 < g.V) {   // both inside: 2-wide loads
            A t0 = wgt, t1 = wgt;
            if (T) {
                T->load_t2(xt, kt, v, t0, t1);
                t0 *= wgt;
                t1 *= wgt;
            }
#pragma unroll
            for (int c = 0; c < C; ++c) {
                A g0, g1;
                gRn.load2(xp, ip, c, v, g0, g1);
                acc[0][c] = fma(t0, g0, acc[0][c]);
                acc[E - 1][c] = fma(t1, g1, acc[E - 1][c]);
            }
            return;
        }
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
template <int P, int C, int E, bool ENV = false>
__device__ __forceinline__ void adj_T_part(const Plan &pl, int q, int n, int x, int k, int v,
                                           typename Prec<P>::A (&gL)[E][C], typename Prec<P>::A (&gT)[E]) {
    using A = typename Prec<P>::A;
    const QuadGeom &g = pl.q[q];
    const int s = 1 << n;
    const int d = 2 * k - s;
#pragma unroll
    for (int l = 0; l < E; ++l) {
        gT[l] = A(0);
#pragma unroll
        for (int c = 0; c < C; ++c) gL[l][c] = A(0);
    }
    // one cone's contribution: arc weight Aw on gR(xg, ip), dot weight dw
    // with R(xr, j, v + d) when rq
    // (R of level rl; out of range, the environment's value, 0 without a map)
    auto cone = [&](const GRLevel<P, C> &gR, int xg, int ip, A Aw, A dw, bool rq, const RLevel<P, C> &R, int xr, int j,
                    int rl) {
        if (E == 2 && v + 1 < g.V) {             // 2-wide loads (v, d even)
            const bool r0 = rq && v + d >= 0 && v + d < g.V, r1 = rq && v + d + 1 >= 0 && v + d + 1 < g.V;
            A dot0 = A(0), dot1 = A(0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                A g0, g1, q0, q1;
                gR.load2(xg, ip, c, v, g0, g1);
                const A ev = renv<P, C, ENV>(pl, q, rl, j, c);
                q0 = q1 = ev;
                if (r0) {
                    R.load2(xr, j, c, v + d, q0, q1);
                    if (!r1) q1 = ev;
                }
                gL[0][c] = fma(Aw, g0, gL[0][c]);
                gL[E - 1][c] = fma(Aw, g1, gL[E - 1][c]);
                dot0 = fma(g0, q0, dot0);
                dot1 = fma(g1, q1, dot1);
            }
            gT[0] = fma(dw, dot0, gT[0]);
            gT[E - 1] = fma(dw, dot1, gT[E - 1]);
            return;
        }
#pragma unroll
        for (int l = 0; l < E; ++l) {
            const int vv = v + l;
            const bool rok = rq && vv + d >= 0 && vv + d < g.V;
            A dot = A(0);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A gr = gR.load(xg, ip, c, vv);
                gL[l][c] = fma(Aw, gr, gL[l][c]);
                dot = fma(gr, rok ? R.load(xr, j, c, vv + d) : renv<P, C, ENV>(pl, q, rl, j, c), dot);
            }
            gT[l] = fma(dw, dot, gT[l]);
        }
    };
    if ((x & 1) && n < g.N) {
        GRLevel<P, C> gRn(pl, q, n);
        const int xq = (x + 1) >> 1;
        const bool rq = (n + 1 < g.N) && xq < g.Un[n + 1];
        RLevel<P, C> R1(pl, q, rq ? n + 1 : n);
        if (k >= 1) cone(gRn, x, k - 1, arc<P>(pl, n + 1, 2 * k - 1), A(1), rq, R1, xq, 2 * k - 1, n + 1);
        if (k < s) cone(gRn, x, k, arc<P>(pl, n + 1, 2 * k), A(1), rq, R1, xq, 2 * k, n + 1);
    }
    if (!(k & 1) && n >= 1) {
        const int m = n - 1;
        GRLevel<P, C> gRm(pl, q, m);
        const bool rq = (n < g.N) && x + 1 < g.Un[n];
        RLevel<P, C> Rn(pl, q, rq ? n : 0);
        if (k >= 2) cone(gRm, 2 * x, (k >> 1) - 1, A(0.5) * arc<P>(pl, n, k - 1), A(0.5), rq, Rn, x + 1, k - 1, n);
        if (k < s) cone(gRm, 2 * x, k >> 1, A(0.5) * arc<P>(pl, n, k), A(0.5), rq, Rn, x + 1, k, n);
    }
}

// Levels whose merge-down part is computed inside the merge-up reverse of
// the level above (n = 2 .. N-1); adj_T covers the others.
__host__ __device__ inline bool adj_T_fused(int n, int N) { return n >= 2 && n <= N - 1; }

template <int P, int C, int E, bool ENV = false>
__device__ __forceinline__ void body_adj_T(const Plan &pl, const RowSplitB &rs, int n, long long bx, int by) {
    using A = typename Prec<P>::A;
    int local;
    const int q = quadrant_of(rs, bx, local);   // row = (q, x, k) at level n, live x only
    const QuadGeom &g = pl.q[q];
    const int v = E * (by * blockDim.x + threadIdx.x);
    if (v >= g.V) return;
    int x, k;
    if (n == 0) {                                 // odd columns only (t_live)
        x = 2 * (local >> 1) + 1;
        k = local & 1;
    } else {
        const int K = (1 << n) + 1;
        local += K;
        x = local / K;
        k = local - x * K;
    }
    A gL[E][C], gT[E];
    adj_T_part<P, C, E, ENV>(pl, q, n, x, k, v, gL, gT);
    GTLevel<P, C> gTn(pl, q, n);
#pragma unroll
    for (int l = 0; l < E; ++l)
        if (v + l < g.Vs) gTn.store(x, k, v + l, gL[l], gT[l]);
}

// ---------------------------------------------------------------------------
// dL/dT_{n-1}(x', kap, w) = its merge-down part (adj_T_part, fused here) +
// the reverse of the level-n merge up.  h = 2^{n-1}.
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
template <int P, int C, bool ENV = false>
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
    adj_T_part<P, C, E, ENV>(pl, q, m, x1, kap, w, aL, aT);   // the merge-down part of dL/dT_{n-1}
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
            A gL[E][C], gT[E];
            gTn.load2(x, kout, w, gL, gT);      // w even, w + 1 < Vs
#pragma unroll
            for (int l = 0; l < E; ++l) {
                A dT = gT[l] * fr[l].trans();
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    aL[l][c] = fma(wgt, gL[l][c], aL[l][c]);
                    dT = fma(gL[l][c], fr[l].L[c], dT);
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
            A gL[E][C], gT[E];
            if (v + 1 < g.V) {
                gTn.load2(x, kout, v, gL, gT);
            } else {                            // v + 1 outside: its term is dropped below
                gTn.load(x, kout, v, gL[0], gT[0]);
            }
#pragma unroll
            for (int l = 0; l < E; ++l) {
                if (v + l >= g.V) continue;
                const A tn = wgt * nr[l].trans();
#pragma unroll
                for (int c = 0; c < C; ++c) aL[l][c] = fma(tn, gL[l][c], aL[l][c]);
                aT[l] = fma(tn, gT[l], aT[l]);
            }
        }
    }
    gTm.store2(x1, kap, w, aL, aT);           // w even, w + 1 < Vs
}

// ---------------------------------------------------------------------------
// Reverse of Trace for T_0..T_2.  A ray with pieces m (pixel sigma_m, e_m,
// length l_m, transmittance t_m, weight w_m = l_m phi(sigma_m l_m)) has
//   L = sum_m P_m e_m w_m,  P_m = prod_{m'<m} t_m',  T = prod_m t_m.
// For upstream (gL, gT):
//   dL/de_j     = gL P_j w_j
//   dL/dsigma_j = sum_c gL_c (P_j e_jc dw_j/dsigma - l_j S_jc) - gT l_j T,
//   S_j = sum_{m>j} P_m e_m w_m,   dw/dsigma = l^2 phi'(sigma l).
// Writing G_j = sum_{m<=j} P_m w_m (gL . e_m) (so that sum_c gL_c S_jc =
// G_tot - G_j), the sigma term is
//   dL/dsigma_j = [P_j dw_j (gL . e_j) + l_j G_j] - l_j (G_tot + gT T),
// where the bracket is known at piece j and the last factor once per ray.
//
// Ray-centric and deterministic, one pair tile per block, per quadrant and
// ray shape R (shapes unrolled at compile time):
//   phase A: one thread per probe whose ray reaches the tile traces the ray
//            once from the staged tile and writes each piece's
//            (dL/de_j, dL/dsigma_j) to a shared-memory slot [j][probe];
//   phase B: each tile pixel adds, piece index by piece index, the slot of
//            the one probe whose ray crosses it as piece j
//            (probe = pixel - offset_j), so the summation order is fixed.
// ---------------------------------------------------------------------------

// Probe box of ray shape R for a tile of PT_U x PT_V frame pixels: the probes
// (spacing S = 2^n along u) whose ray reaches the tile lie in
// u in [u0 - S, u0 + PT_U) (PT_U / S + 1 aligned columns) and
// v in [v0 - dvhi, v0 + PT_V - dvlo), dv of the shape in [dvlo, dvhi] (one
// sign: a ray is monotone in v).
constexpr int shape_dv_min(int R) {
    int m = 0;
    for (int j = kShapes.start[R]; j < kShapes.start[R + 1]; ++j) m = kShapes.p[j].dv < m ? kShapes.p[j].dv : m;
    return m;
}
constexpr int shape_dv_max(int R) {
    int m = 0;
    for (int j = kShapes.start[R]; j < kShapes.start[R + 1]; ++j) m = kShapes.p[j].dv > m ? kShapes.p[j].dv : m;
    return m;
}
constexpr int shape_slots(int R) {
    const int n = R < 2 ? 0 : (R < 5 ? 1 : 2);
    return (kShapes.start[R + 1] - kShapes.start[R]) * (PT_U / (1 << n) + 1) *
           (PT_V + shape_dv_max(R) - shape_dv_min(R));
}
constexpr int adj_max_slots() {
    int m = 0;
    for (int R = 0; R < HRC_MAXRAY; ++R) m = shape_slots(R) > m ? shape_slots(R) : m;
    return m;
}
constexpr int ADJ_SLOTS = adj_max_slots();

constexpr int ADJ_THREADS = 256;   // block size of the adjoint trace
constexpr int ADJ_ROUNDS = 3;      // probes per thread and shape, at most

template <int R> struct RayBox {
    static constexpr int n = RayAt<R>::n, k = RayAt<R>::k, S = 1 << n;
    static constexpr int NP = RayAt<R>::end - RayAt<R>::begin;
    static constexpr int dvlo = shape_dv_min(R), dvhi = shape_dv_max(R);
    static constexpr int NVB = PT_V + dvhi - dvlo;
    static constexpr int NPROBE = (PT_U / S + 1) * NVB;
    static constexpr int ROUNDS = (NPROBE + ADJ_THREADS - 1) / ADJ_THREADS;
    static_assert(dvlo == 0 || dvhi == 0, "a ray is monotone in v");
    static_assert(S <= PT_HALO && dvhi - dvlo <= PT_HALO, "the halo covers every probe of the box");
    static_assert(ROUNDS <= ADJ_ROUNDS, "prefetch registers");
};

// dL/dT of the rays of one shape for the thread's probes (round r = probe
// threadIdx.x + r * ADJ_THREADS), loaded ahead of their use.
template <class A, int C> struct AdjPre {
    A gL[ADJ_ROUNDS][C], gT[ADJ_ROUNDS];
};

// Per-(piece, probe) slots: fp32 with C <= 3 as float4 {dE_0..dE_{C-1}, dS};
// otherwise C + 1 planes.
template <class A, int C> struct AdjSlots {
    static constexpr bool packed = PackES<A, C>::packed;
    A *p;
    static constexpr size_t bytes() { return packed ? sizeof(float4) * ADJ_SLOTS : sizeof(A) * (C + 1) * ADJ_SLOTS; }
    __device__ __forceinline__ void put(int i, const A (&dE)[C], A dS) const {
        if constexpr (packed) {
            float4 v = make_float4(dE[0], 0.f, 0.f, dS);
            if constexpr (C > 1) v.y = dE[1];
            if constexpr (C > 2) v.z = dE[2];
            reinterpret_cast<float4 *>(p)[i] = v;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) p[c * ADJ_SLOTS + i] = dE[c];
            p[C * ADJ_SLOTS + i] = dS;
        }
    }
    __device__ __forceinline__ void add_to(int i, A (&dE)[C], A &dS) const {
        if constexpr (packed) {
            const float4 v = reinterpret_cast<const float4 *>(p)[i];
            dE[0] += v.x;
            if constexpr (C > 1) dE[1] += v.y;
            if constexpr (C > 2) dE[2] += v.z;
            dS += v.w;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) dE[c] += p[c * ADJ_SLOTS + i];
            dS += p[C * ADJ_SLOTS + i];
        }
    }
};

// Phase A, pieces J .. end-1 of shape R for the ray at region offset `base`.
// Pp: transmittance before piece J; G: sum over earlier pieces of
// P_m w_m (gL . e_m).  Writes dE[j] and the known part of dS[j].
template <class A, int C, int R, int J>
__device__ __forceinline__ void adj_pieces(const PairTile<A, C> &tt, int base, int su, const A (&gL)[C], A &Pp, A &G,
                                           A (&dE)[RayBox<R>::NP][C], A (&dS)[RayBox<R>::NP]) {
    if constexpr (J < RayAt<R>::end) {
        using pc = PieceAt<J>;
        constexpr int L = J - RayAt<R>::begin;
        const int o = base + pc::du * su + pc::dv;
        A t, w, d, em[C], sg;
        tt.piece(pc::cls, o, t, w, d);
        tt.emis(o, em, sg);
        const A lh = class_len<A>(pc::cls);
        A wq = w;
        if constexpr (pc::full != 0) {                // w2 = w (1 + t), dw2 = d (1 + t) - l t w, t2 = t^2
            d = fma(d, A(1) + t, -lh * t * w);
            wq = w * (A(1) + t);
            t = t * t;
        }
        const A len = pc::full != 0 ? A(2) * lh : lh;
        A ge = A(0);
#pragma unroll
        for (int c = 0; c < C; ++c) ge = fma(gL[c], em[c], ge);
        const A pw = Pp * wq;
#pragma unroll
        for (int c = 0; c < C; ++c) dE[L][c] = gL[c] * pw;
        G = fma(pw, ge, G);
        dS[L] = fma(Pp * d, ge, len * G);
        Pp *= t;
        adj_pieces<A, C, R, J + 1>(tt, base, su, gL, Pp, G, dE, dS);
    }
}

template <class A, int R, int J>
__device__ __forceinline__ void adj_finish(A K, A (&dS)[RayBox<R>::NP]) {
    if constexpr (J < RayAt<R>::end) {
        using pc = PieceAt<J>;
        const A len = pc::full != 0 ? A(2) * class_len<A>(pc::cls) : class_len<A>(pc::cls);
        dS[J - RayAt<R>::begin] = fma(-len, K, dS[J - RayAt<R>::begin]);
        adj_finish<A, R, J + 1>(K, dS);
    }
}

// Geometry of one quadrant frame of the tile: u0 / v0 = the tile's first
// frame column / row (u0 may be negative at the image edge for the reversed
// frames), tu = the tile's image origin along u, fwd = frame u runs with the
// image axis.
struct AdjFrame {
    int q, U, V, u0, v0, tu;
    bool fwd;
};

// Probe of round r of shape R: frame position and whether it is a live
// probe inside the frame.
template <int R>
__device__ __forceinline__ bool adj_probe(const AdjFrame &f, int ua, int i, int &up, int &vp) {
    using B = RayBox<R>;
    const int col = i / B::NVB, vb = i - col * B::NVB;
    up = ua + col * B::S;
    vp = f.v0 - B::dvhi + vb;
    return i < B::NPROBE && up >= 1 && up < f.U && vp >= 0 && vp < f.V && t_live(B::n, up >> B::n, B::k);
}

template <int P, int C, int R>
__device__ __forceinline__ void adj_prefetch(const Plan &pl, const AdjFrame &f, AdjPre<typename Prec<P>::A, C> &pre) {
    using B = RayBox<R>;
    const int ua = (f.u0 - 1) & ~(B::S - 1);      // first aligned column >= u0 - S
    const GTLevel<P, C> gTl(pl, f.q, B::n);
#pragma unroll
    for (int r = 0; r < B::ROUNDS; ++r) {
        int up, vp;
        if (adj_probe<R>(f, ua, threadIdx.x + r * ADJ_THREADS, up, vp)) gTl.load(up >> B::n, B::k, vp, pre.gL[r], pre.gT[r]);
    }
}

template <int P, int C, int R>
__device__ __forceinline__ void adj_phase_a(const PairTile<typename Prec<P>::A, C> &tt,
                                            const AdjSlots<typename Prec<P>::A, C> &sl, const AdjFrame &f,
                                            const AdjPre<typename Prec<P>::A, C> &pre) {
    using A = typename Prec<P>::A;
    using B = RayBox<R>;
    const int ua = (f.u0 - 1) & ~(B::S - 1);
    const int su = f.fwd ? PT_PITCH : -PT_PITCH;
#pragma unroll
    for (int r = 0; r < B::ROUNDS; ++r) {
        const int i = threadIdx.x + r * ADJ_THREADS;
        if (i >= B::NPROBE) break;
        int up, vp;
        A dE[B::NP][C], dS[B::NP];
        if (adj_probe<R>(f, ua, i, up, vp)) {
            const int ap = (f.fwd ? up - f.tu : f.U - 1 - up - f.tu) + PT_HALO;
            const int base = ap * PT_PITCH + (vp - f.v0 + PT_HALO);
            A Pp = A(1), G = A(0);
            adj_pieces<A, C, R, RayAt<R>::begin>(tt, base, su, pre.gL[r], Pp, G, dE, dS);
            adj_finish<A, R, RayAt<R>::begin>(fma(pre.gT[r], Pp, G), dS);   // Pp is now the ray's T
        } else {
#pragma unroll
            for (int l = 0; l < B::NP; ++l) {
                dS[l] = A(0);
#pragma unroll
                for (int c = 0; c < C; ++c) dE[l][c] = A(0);
            }
        }
#pragma unroll
        for (int l = 0; l < B::NP; ++l) sl.put(l * B::NPROBE + i, dE[l], dS[l]);
    }
}

// Phase B for the pieces J .. end-1 of shape R that can reach a pixel whose
// frame column u has u mod S == RHO (piece J crosses it for the probe at
// u - du_J only when that column is a probe column, i.e. du_J mod S == RHO):
// the selection is made at compile time, so no piece is tested at run time.
template <class A, int C, int R, int RHO, int J>
__device__ __forceinline__ void adj_phase_b_res(const AdjSlots<A, C> &sl, int u, int v, int ua, int v0, A (&dE)[C],
                                                A &dS) {
    if constexpr (J < RayAt<R>::end) {
        using B = RayBox<R>;
        using pc = PieceAt<J>;
        if constexpr ((pc::du & (B::S - 1)) == RHO)
            sl.add_to((J - RayAt<R>::begin) * B::NPROBE + ((u - pc::du - ua) >> B::n) * B::NVB +
                          (v - pc::dv - v0 + B::dvhi),
                      dE, dS);
        adj_phase_b_res<A, C, R, RHO, J + 1>(sl, u, v, ua, v0, dE, dS);
    }
}

// Dispatch on the pixel column's residue (uniform over a warp).
template <class A, int C, int R, int RHO = 0>
__device__ __forceinline__ void adj_phase_b(const AdjSlots<A, C> &sl, int u, int v, int ua, int v0, A (&dE)[C],
                                            A &dS) {
    if constexpr (RHO < RayBox<R>::S) {
        if ((u & (RayBox<R>::S - 1)) == RHO)
            adj_phase_b_res<A, C, R, RHO, RayAt<R>::begin>(sl, u, v, ua, v0, dE, dS);
        else
            adj_phase_b<A, C, R, RHO + 1>(sl, u, v, ua, v0, dE, dS);
    }
}

// Every shape R <= HRC_MAXRAY - 1 with level <= nmax (shapes are ordered by
// level): phase A from the prefetched dL/dT, prefetch of the next shape's,
// barrier, phase B for the thread's two pixels (frame columns uc[i],
// valid[i]), barrier.  nmax is uniform over the block, so are the barriers.
template <int P, int C, int R>
__device__ __forceinline__ void adj_shapes(const Plan &pl, const PairTile<typename Prec<P>::A, C> &tt,
                                           const AdjSlots<typename Prec<P>::A, C> &sl, const AdjFrame &f, int nmax,
                                           const int (&uc)[2], const bool (&valid)[2], int v,
                                           AdjPre<typename Prec<P>::A, C> &pre,
                                           typename Prec<P>::A (&dE)[2][C], typename Prec<P>::A (&dS)[2]) {
    using A = typename Prec<P>::A;
    if constexpr (R < HRC_MAXRAY) {
        if (RayAt<R>::n <= nmax) {
            adj_phase_a<P, C, R>(tt, sl, f, pre);
            if constexpr (R + 1 < HRC_MAXRAY)
                if (RayAt<R + 1>::n <= nmax) adj_prefetch<P, C, R + 1>(pl, f, pre);
            __syncthreads();
            const int ua = (f.u0 - 1) & ~(RayBox<R>::S - 1);
#pragma unroll
            for (int i = 0; i < 2; ++i)
                if (valid[i]) adj_phase_b<A, C, R>(sl, uc[i], v, ua, f.v0, dE[i], dS[i]);
            __syncthreads();
        }
        adj_shapes<P, C, R + 1>(pl, tt, sl, f, nmax, uc, valid, v, pre, dE, dS);
    }
}

// Shared memory of the adjoint trace: the pair tile, then the slots (reused
// at the end, pair 0, as a transposed accumulator so that dL/de and
// dL/dsigma leave coalesced).
template <class A, int C> constexpr size_t adj_trace_smem() {
    const size_t acc = sizeof(A) * (C + 1) * PT_V * (PT_U + 1);
    const size_t sl = AdjSlots<A, C>::bytes();
    return PairTile<A, C>::bytes() + (sl > acc ? sl : acc);
}

// dL/de and dL/dsigma of quadrant pair `pair` for one tile.  Each thread
// owns two pixels of the tile (columns c[i] along u, its lane along v) and
// accumulates them in registers over both frames of the pair.  Pair 0
// writes the image gradients, pair 1 (launched after it) adds to them.
// With tme / tms (fp32 inputs) the tile region is fetched by TMA tensor
// copies; a copy wait that gives up records its code in the plan's status
// word and leaves the tile's gradients unwritten.
template <int P, int C, class IN>
__device__ __forceinline__ void body_adj_trace(const Plan &pl, const IN *__restrict__ e, const IN *__restrict__ s,
                                               IN *__restrict__ ge, IN *__restrict__ gs, int pair, int bx, int by,
                                               unsigned char *smem, const CUtensorMap *tme = nullptr,
                                               const CUtensorMap *tms = nullptr) {
    using A = typename Prec<P>::A;
    PairTile<A, C> tt(smem);
    const AdjSlots<A, C> sl{reinterpret_cast<A *>(smem + PairTile<A, C>::bytes())};
    A *acc = sl.p;                                     // [C+1][PT_V][PT_U+1], after the last phase
    const int W = pl.W, H = pl.H;
    const long long HW = (long long)W * H;
    const int x0 = pair == 0 ? bx * PT_U : bx * PT_V;
    const int y0 = pair == 0 ? by * PT_V : by * PT_U;
    if constexpr (sizeof(A) == 4) {
        if (tme) {
            __shared__ __align__(8) uint64_t bar;
            const int code = tt.stage_tma(pair, x0, y0, tme, tms, &bar, pl.bulk_limit_ns);
            if (code != 0) {
                if (threadIdx.x == 0) atomicMax(pl.status, code);
                return;
            }
        } else {
            tt.stage(pair, W, H, x0, y0, e, s);
        }
    } else {
        tt.stage(pair, W, H, x0, y0, e, s);
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cc[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) cc[i] = 8 * i + ((warp + i) & 7);
    A dE[2][C], dS[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        dS[i] = A(0);
#pragma unroll
        for (int c = 0; c < C; ++c) dE[i][c] = A(0);
    }
#pragma unroll 1
    for (int qq = 0; qq < 2; ++qq) {
        const int q = 2 * pair + qq;
        const QuadGeom &g = pl.q[q];
        if (g.N < 1) continue;
        AdjFrame f;
        f.q = q;
        f.U = g.U;
        f.V = g.V;
        f.fwd = (q == 0 || q == 2);
        f.tu = pair == 0 ? x0 : y0;
        f.v0 = pair == 0 ? y0 : x0;
        f.u0 = f.fwd ? f.tu : f.U - PT_U - f.tu;
        int uc[2];
        bool valid[2];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int iu = f.tu + cc[i];               // image coordinate along u
            valid[i] = iu < f.U && f.v0 + lane < f.V;
            uc[i] = f.fwd ? iu : f.U - 1 - iu;
        }
        AdjPre<A, C> pre;
        adj_prefetch<P, C, 0>(pl, f, pre);
        adj_shapes<P, C, 0>(pl, tt, sl, f, g.N < 2 ? g.N : 2, uc, valid, f.v0 + lane, pre, dE, dS);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int c = cc[i];
        // image pixel: pair 0 (c along x, lane along y); pair 1 (c along y, lane along x)
        const int x = pair == 0 ? x0 + c : x0 + lane, y = pair == 0 ? y0 + lane : y0 + c;
        if (x >= W || y >= H) continue;
        const long long pix = (long long)y * W + x;
        if (pair == 0) {
#pragma unroll
            for (int k = 0; k < C; ++k) acc[(k * PT_V + lane) * (PT_U + 1) + c] = dE[i][k];
            acc[(C * PT_V + lane) * (PT_U + 1) + c] = dS[i];
        } else {
#pragma unroll
            for (int k = 0; k < C; ++k) ge[k * HW + pix] = IN(A(ge[k * HW + pix]) + dE[i][k]);
            gs[pix] = IN(A(gs[pix]) + dS[i]);
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
            for (int c = 0; c < C; ++c) ge[c * HW + pix] = IN(acc[(c * PT_V + ly) * (PT_U + 1) + lx]);
            gs[pix] = IN(acc[(C * PT_V + ly) * (PT_U + 1) + lx]);
        }
    }
}

}  // namespace hrc
