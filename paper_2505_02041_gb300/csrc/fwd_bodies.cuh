// fwd_bodies.cuh -- device bodies of the forward HRC kernels.
//
//   body_trace012    : T_0..T_min(2,N) by direct tracing (Sec. 4.2, Eq. 9)
//   body_merge_up    : T_n from T_{n-1} (Eq. 18 even k, Eqs. 19-20 odd k)
//   body_merge_down  : R_n from R_{n+1}, T_n, T_{n+1} (Eq. 14 odd x, Eqs. 15-17 even x)
//   body_fluence     : F = sum over quadrants of R_0([u+1, v], 1/2) (Algorithm 1,
//                      Lighting), with the level-0 merge down computed in place
//
// Each body processes one block of work given by an explicit block index
// (bx, by), so the same code runs as a standalone kernel (one launch per
// step, bx = blockIdx.x) and inside the batched persistent kernel (work
// items popped from a queue).  The work is memory-bound (about one FMA per
// byte), so the bodies are organised around coalesced, v-contiguous rows:
// a block handles one (x, k) or (x, i) row segment of consecutive v, every
// neighbour access being a shifted run of the same length.  Out-of-range
// lookups read as vacuum (T = <0, 1>, R = 0), which is exact for this
// method: paths are monotone in v, so a path that leaves the grid never
// re-enters, and nothing outside the grid emits.
//
// Column x = 0 of every level is dead: the fluence sum reads R_0 at u + 1,
// R_n(0) feeds only R_{n-1}(0), and T_n(0) only T_{n+1}(0) and R_n(0).  No
// body computes or reads it (T_N, a single column when U <= 2^N, is then
// skipped entirely).  The even columns of T_0 and the odd directions of T_1
// at even columns are dead too (t_live) and are not traced.
#pragma once

#include <type_traits>

#include "bulk_copy.cuh"
#include "hrc_internal.cuh"
#include "trace_shapes.cuh"

namespace hrc {


__device__ __forceinline__ int find_quadrant(const RowSplit &rs, long long r, int &local) {
    int q = 0;
    long long base = 0;
#pragma unroll
    for (int j = 1; j < 4; ++j)
        if (r >= rs.start[j]) { q = j; base = rs.start[j]; }
    local = (int)(r - base);
    return q;
}

// Per-pixel piece factors of the three ray classes (trace_shapes.cuh): for
// the half length l of class c, t = exp(-sigma l) and w = l phi(sigma l) =
// (1 - e^{-sigma l}) / sigma, the radiance weight of Eq. 4 over a uniform
// piece.  Full pieces use t^2 and w (1 + t).
template <class A> __device__ __forceinline__ void piece_factors(A sg, A len, A &t, A &w) {
    const A m = fexpm1(-sg * len);
    t = A(1) + m;
    w = sg != A(0) ? -m / sg : len;
}

// Shared-memory tile of a 32 x 32 image block with a 4-pixel halo (the
// longest directly traced ray, v_2(k), reaches 4 pixels along and across):
// the piece factors {t, w} of the three ray classes as 2-vectors, and the
// emission with the extinction (one float4 per pixel in fp32 with C <= 3,
// else planes), so a ray piece costs two shared loads.  Outside the image
// every field is vacuum (sigma = e = 0, t = 1, w = l).
constexpr int TR_TILE = 32, TR_HALO = 4, TR_REG = TR_TILE + 2 * TR_HALO, TR_PITCH = TR_REG + 1;
constexpr int TR_PLANE = TR_REG * TR_PITCH;

template <class A, int C> struct TraceTile {
    using V2 = typename Vec2<A>::T;
    static constexpr bool packed = PackES<A, C>::packed;
    V2 *tw;        // [3][PLANE]
    float4 *es4;   // [PLANE] when packed
    A *e;          // [C][PLANE] otherwise
    A *s;          // [PLANE] otherwise
    __device__ __forceinline__ explicit TraceTile(unsigned char *smem) {
        tw = reinterpret_cast<V2 *>(smem);
        es4 = reinterpret_cast<float4 *>(tw + 3 * TR_PLANE);
        e = reinterpret_cast<A *>(tw + 3 * TR_PLANE);
        s = e + C * TR_PLANE;
    }
    static constexpr size_t bytes() {
        return sizeof(V2) * 3 * TR_PLANE + (packed ? sizeof(float4) * TR_PLANE : sizeof(A) * (C + 1) * TR_PLANE);
    }
    __device__ __forceinline__ void emis(int o, A (&em)[C], A &sg) const {
        if constexpr (packed) {
            const float4 v = es4[o];
            em[0] = v.x;
            if constexpr (C > 1) em[1] = v.y;
            if constexpr (C > 2) em[2] = v.z;
            sg = v.w;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) em[c] = e[c * TR_PLANE + o];
            sg = s[o];
        }
    }
    // the fields of region pixel o from its extinction and emission
    __device__ __forceinline__ void put(int o, A sg, const A (&ev)[C]) const {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A tc, wc;
            piece_factors<A>(sg, class_len<A>(c), tc, wc);
            V2 p;
            p.x = tc;
            p.y = wc;
            tw[c * TR_PLANE + o] = p;
        }
        if constexpr (packed) {
            float4 v = make_float4(ev[0], 0.f, 0.f, sg);
            if constexpr (C > 1) v.y = ev[1];
            if constexpr (C > 2) v.z = ev[2];
            es4[o] = v;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) e[c * TR_PLANE + o] = ev[c];
            s[o] = sg;
        }
    }
    template <class IN>
    __device__ __forceinline__ void stage(int W, int H, int x0, int y0, const IN *__restrict__ ein,
                                          const IN *__restrict__ sin) {
        const long long HW = (long long)W * H;
        for (int i = threadIdx.x; i < TR_REG * TR_REG; i += blockDim.x) {
            const int ry = i / TR_REG, rx = i - ry * TR_REG;
            const int x = x0 - TR_HALO + rx, y = y0 - TR_HALO + ry;
            const bool in = x >= 0 && x < W && y >= 0 && y < H;
            const long long pix = (long long)y * W + x;
            A ev[C];
#pragma unroll
            for (int c = 0; c < C; ++c) ev[c] = in ? A(ein[c * HW + pix]) : A(0);
            put(ry * TR_PITCH + rx, in ? A(sin[pix]) : A(0), ev);
        }
    }
    // The same staging with the region of e and sigma fetched by TMA tensor
    // copies (fp32 inputs; the out-of-grid part of the box reads as zero,
    // which is vacuum).  The boxes land in a staging area that overlaps the
    // {t, w} planes: every thread first takes its pixels into registers,
    // then the planes are written.  Returns 0, or kWaitTimeout / kWaitLost
    // when the copy wait gave up.
    __device__ __forceinline__ int stage_tma(int x0, int y0, const CUtensorMap *tme, const CUtensorMap *tms,
                                             uint64_t *bar, long long limit_ns, unsigned extra_tx) {
        static_assert(sizeof(A) == 4, "fp32 staging");
        constexpr int BOX = TR_REG * TR_REG;                        // 40 x 40
        constexpr int PER = (BOX + 255) / 256;                      // pixels per thread (256 threads)
        static_assert((C + 1) * BOX * sizeof(float) <= 3 * TR_PLANE * sizeof(V2), "staging fits the {t, w} planes");
        float *stg = reinterpret_cast<float *>(tw);                 // [C + 1][BOX]
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect(bar, (unsigned)((C + 1) * BOX * sizeof(float)) + extra_tx);
#pragma unroll
            for (int c = 0; c < C; ++c) tma_load_3d(stg + c * BOX, tme, x0 - TR_HALO, y0 - TR_HALO, c, bar);
            tma_load_2d(stg + C * BOX, tms, x0 - TR_HALO, y0 - TR_HALO, bar);
        }
        if (!mbar_wait(bar, 0, limit_ns))                           // gave up: let the copies land
            return mbar_wait(bar, 0, drain_limit_ns(limit_ns)) ? kWaitTimeout : kWaitLost;
        float sv[PER], ev[PER][C];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + 256 * k;
            if (i >= BOX) break;
            sv[k] = stg[C * BOX + i];
#pragma unroll
            for (int c = 0; c < C; ++c) ev[k][c] = stg[c * BOX + i];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + 256 * k;
            if (i >= BOX) break;
            const int ry = i / TR_REG, rx = i - ry * TR_REG;
            put(ry * TR_PITCH + rx, sv[k], ev[k]);
        }
        return 0;
    }
};

// Trace of ray shape R from the probe whose tile offset is `base`; su / sv
// are the tile strides along the frame's u and v axes.  Pieces J .. END-1
// are unrolled at compile time.
template <int P, int C, int J, int END>
__device__ __forceinline__ void trace_pieces(const TraceTile<typename Prec<P>::A, C> &tt, int base, int su, int sv,
                                             typename Prec<P>::A (&L)[C], typename Prec<P>::A &Tacc,
                                             typename Prec<P>::A &tau) {
    using A = typename Prec<P>::A;
    if constexpr (J < END) {
        using pc = PieceAt<J>;
        const int o = base + pc::du * su + pc::dv * sv;
        const typename TraceTile<A, C>::V2 p = tt.tw[pc::cls * TR_PLANE + o];
        A t = p.x, w = p.y, em[C], sg;
        tt.emis(o, em, sg);
        if constexpr (pc::full != 0) {
            w = w * (A(1) + t);
            t = t * t;
        }
        const A wt = Tacc * w;
#pragma unroll
        for (int c = 0; c < C; ++c) L[c] = fma(wt, em[c], L[c]);
        Tacc *= t;
        if constexpr (Prec<P>::LOG) tau = fma(sg, A(pc::full ? 2 : 1) * class_len<A>(pc::cls), tau);
        trace_pieces<P, C, J + 1, END>(tt, base, su, sv, L, Tacc, tau);
    }
}

template <int P, int C, int R>
__device__ __forceinline__ void trace_store(const Plan &pl, const TraceTile<typename Prec<P>::A, C> &tt, int q,
                                            int nmax, int u, int v, int base, int su, int sv) {
    using A = typename Prec<P>::A;
    using ray = RayAt<R>;
    if (ray::n > nmax || (u & ((1 << ray::n) - 1)) || !t_live(ray::n, u >> ray::n, ray::k)) return;
    Iv<P, C> iv;
#pragma unroll
    for (int c = 0; c < C; ++c) iv.L[c] = A(0);
    A Tacc = A(1), tau = A(0);
    trace_pieces<P, C, ray::begin, ray::end>(tt, base, su, sv, iv.L, Tacc, tau);
    iv.t = Prec<P>::LOG ? tau : Tacc;
    TLevel<P, C>(pl, q, ray::n).store(u >> ray::n, ray::k, v, iv);
}

// T_0..T_min(2,N) of the selected quadrant frames for one 32 x 32 image
// tile.  Warp w handles tile columns c = 8i + ((w + i) mod 8) along the
// frame's u axis (one column of every residue mod 4, so the warps get equal
// shares of the level-1 and level-2 probes); its lanes run along v, so every
// T store is a 128-byte coalesced row segment in every frame.
// With tme / tms (fp32 inputs), the region is fetched by TMA tensor copies;
// a copy wait that gives up records its code in the plan's status word and
// leaves the tile's T entries unwritten.
template <int P, int C>
__device__ __forceinline__ void body_trace012(const Plan &pl, const float *__restrict__ e, const float *__restrict__ s,
                                              const double *__restrict__ ed, const double *__restrict__ sd, int qmask,
                                              int bx, int by, unsigned char *tr_smem,
                                              const CUtensorMap *tme = nullptr, const CUtensorMap *tms = nullptr) {
    using A = typename Prec<P>::A;
    TraceTile<A, C> tt(tr_smem);
    const int W = pl.W, H = pl.H;
    const int x0 = bx * TR_TILE, y0 = by * TR_TILE;
    if constexpr (P == P_FP64) {
        tt.stage(W, H, x0, y0, ed, sd);
    } else {
        if (tme) {
            __shared__ __align__(8) uint64_t bar;
            const int code = tt.stage_tma(x0, y0, tme, tms, &bar, pl.bulk_limit_ns, (unsigned)pl.bulk_extra_tx);
            if (code != 0) {
                if (threadIdx.x == 0) atomicMax(pl.status, code);
                return;
            }
        } else {
            tt.stage(W, H, x0, y0, e, s);
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = 0; q < 4; ++q) {
        if (!((qmask >> q) & 1)) continue;
        const QuadGeom &g = pl.q[q];
        const int nmax = g.N < 2 ? g.N : 2;
        const bool xu = q < 2;                              // frame u runs along image x
        const int tu = xu ? x0 : y0, tv = xu ? y0 : x0;     // tile origin along u / v axes
        const int ext_u = xu ? W : H;
        const int v = tv + lane;
        const int sgn = (q == 0 || q == 2) ? 1 : -1;        // image step along u
        const int su = sgn * (xu ? 1 : TR_PITCH), sv = xu ? TR_PITCH : 1;
        for (int i = 0; i < TR_TILE / 8; ++i) {
            const int c = 8 * i + ((warp + i) & 7);
            if (tu + c >= ext_u || v >= g.V) continue;
            const int u = (q == 0 || q == 2) ? tu + c : ext_u - 1 - (tu + c);
            const int base = xu ? (TR_HALO + lane) * TR_PITCH + TR_HALO + c
                                : (TR_HALO + c) * TR_PITCH + TR_HALO + lane;
            trace_store<P, C, 0>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 1>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 2>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 3>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 4>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 5>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 6>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 7>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 8>(pl, tt, q, nmax, u, v, base, su, sv);
            trace_store<P, C, 9>(pl, tt, q, nmax, u, v, base, su, sv);
        }
    }
}

// T_n(p, k) from T_{n-1}; p = (x 2^n, v).  Near operand at column 2x, far
// operand at column 2x + 1 shifted by 2k' - 2^{n-1} along v (even for n >= 3,
// so every thread handles aligned pairs v, v+1 with 2-wide accesses).  A
// thread handles G such pairs, blockDim.x pairs apart, and issues all their
// loads before any arithmetic.
template <int P, int C, int G = 1>
__device__ __forceinline__ void body_merge_up(const Plan &pl, const RowSplit &rs, int n, long long bx, int by) {
    int local;
    const int q = find_quadrant(rs, bx, local);   // row = (q, x, k), x >= 1 (column 0 is dead)
    const QuadGeom &g = pl.q[q];
    const int K = (1 << n) + 1;
    local += K;
    const int x = local / K, k = local - x * K;
    const int m = n - 1, sm = 1 << m;
    TLevel<P, C> Tm(pl, q, m), Tn(pl, q, n);
    const int xn = 2 * x, xf = 2 * x + 1;
    const bool far_ok = xf < g.Un[m];
    int v[G];
#pragma unroll
    for (int gi = 0; gi < G; ++gi) v[gi] = 2 * ((by * G + gi) * blockDim.x + threadIdx.x);
    if ((k & 1) == 0) {                             // Eq. 18
        const int kk = k >> 1;
        Iv<P, C> n0[G], n1[G], f0[G], f1[G];
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
            if (v[gi] >= g.V) continue;
            Tm.load2(xn, kk, v[gi], n0[gi], n1[gi]);
            if (far_ok) Tm.load2_masked(xf, kk, v[gi] + 2 * kk - sm, g.V, f0[gi], f1[gi]);
            else f0[gi] = f1[gi] = Iv<P, C>::vacuum();
        }
#pragma unroll
        for (int gi = 0; gi < G; ++gi)
            if (v[gi] < g.V) Tn.store2(x, k, v[gi], merge<P, C>(n0[gi], f0[gi]), merge<P, C>(n1[gi], f1[gi]));
    } else {                                        // Eqs. 19-20
        const int kp = (k + 1) >> 1, km = (k - 1) >> 1;
        Iv<P, C> np0[G], np1[G], nm0[G], nm1[G], fp0[G], fp1[G], fm0[G], fm1[G];
#pragma unroll
        for (int gi = 0; gi < G; ++gi) {
            if (v[gi] >= g.V) continue;
            Tm.load2(xn, kp, v[gi], np0[gi], np1[gi]);
            Tm.load2(xn, km, v[gi], nm0[gi], nm1[gi]);
            if (far_ok) {
                Tm.load2_masked(xf, km, v[gi] + 2 * kp - sm, g.V, fp0[gi], fp1[gi]);
                Tm.load2_masked(xf, kp, v[gi] + 2 * km - sm, g.V, fm0[gi], fm1[gi]);
            } else {
                fp0[gi] = fp1[gi] = fm0[gi] = fm1[gi] = Iv<P, C>::vacuum();
            }
        }
#pragma unroll
        for (int gi = 0; gi < G; ++gi)
            if (v[gi] < g.V)
                Tn.store2(x, k, v[gi], blend<P, C>(merge<P, C>(nm0[gi], fm0[gi]), merge<P, C>(np0[gi], fp0[gi])),
                          blend<P, C>(merge<P, C>(nm1[gi], fm1[gi]), merge<P, C>(np1[gi], fp1[gi])));
    }
}

// As body_merge_up with four consecutive v per thread (v a multiple of 4):
// one 4-wide access per plane; a far run whose offset is not a multiple of
// 4, or that crosses the grid edge, is read as two pairs.
template <int P, int C>
__device__ __forceinline__ void body_merge_up4(const Plan &pl, const RowSplit &rs, int n, long long bx, int by) {
    int local;
    const int q = find_quadrant(rs, bx, local);
    const QuadGeom &g = pl.q[q];
    const int v = 4 * (by * blockDim.x + threadIdx.x);
    if (v >= g.V) return;
    const int K = (1 << n) + 1;
    local += K;
    const int x = local / K, k = local - x * K;
    const int m = n - 1, sm = 1 << m;
    TLevel<P, C> Tm(pl, q, m), Tn(pl, q, n);
    const int xn = 2 * x, xf = 2 * x + 1;
    const bool far_ok = xf < g.Un[m];
    Iv<P, C> out[4];
    if ((k & 1) == 0) {                             // Eq. 18
        const int kk = k >> 1;
        Iv<P, C> nr[4], fr[4];
        Tm.load4(xn, kk, v, nr);
        if (far_ok) Tm.load4_masked(xf, kk, v + 2 * kk - sm, g.V, fr);
        else
#pragma unroll
            for (int l = 0; l < 4; ++l) fr[l] = Iv<P, C>::vacuum();
#pragma unroll
        for (int l = 0; l < 4; ++l) out[l] = merge<P, C>(nr[l], fr[l]);
    } else {                                        // Eqs. 19-20
        // the two merges one after the other: half the operands live at a
        // time (the four-operand form needed ~95 registers, 5 blocks per SM)
        const int kp = (k + 1) >> 1, km = (k - 1) >> 1;
        Iv<P, C> mm[4];
        {
            Iv<P, C> nm[4], fm[4];
            Tm.load4(xn, km, v, nm);
            if (far_ok) Tm.load4_masked(xf, kp, v + 2 * km - sm, g.V, fm);
            else
#pragma unroll
                for (int l = 0; l < 4; ++l) fm[l] = Iv<P, C>::vacuum();
#pragma unroll
            for (int l = 0; l < 4; ++l) mm[l] = merge<P, C>(nm[l], fm[l]);
        }
        {
            Iv<P, C> np[4], fp[4];
            Tm.load4(xn, kp, v, np);
            if (far_ok) Tm.load4_masked(xf, km, v + 2 * kp - sm, g.V, fp);
            else
#pragma unroll
                for (int l = 0; l < 4; ++l) fp[l] = Iv<P, C>::vacuum();
#pragma unroll
            for (int l = 0; l < 4; ++l) out[l] = blend<P, C>(mm[l], merge<P, C>(np[l], fp[l]));
        }
    }
    Tn.store4(x, k, v, out);
}

// R_n(p, i) = F_+ + F_-, p = (x 2^n, v), i = ip + 1/2, j_+ = 2ip+1, j_- = 2ip,
// for v .. v+E-1 of column x >= 1 of frame q (E = 2: all neighbour offsets
// even, n >= 1).
template <int P, int C, int E, bool ENV = false>
__device__ __forceinline__ void merge_down_entry(const Plan &pl, int q, int n, int x, int ip, int v,
                                                 typename Prec<P>::A (&acc)[E][C]) {
    using A = typename Prec<P>::A;
    constexpr bool PAIR = E == 2;
    const QuadGeom &g = pl.q[q];
    const bool top = (n + 1 >= g.N);               // R_N: 0, or the environment map
    const int s = 1 << n;
#pragma unroll
    for (int l = 0; l < E; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[l][c] = A(0);
    const A Ap = arc<P>(pl, n + 1, 2 * ip + 1), Am = arc<P>(pl, n + 1, 2 * ip);
    if constexpr (E == 4) {
        // four consecutive v (v a multiple of 4, n >= 1): one 4-wide access
        // per plane and row; a far run whose even offset is not a multiple
        // of 4, or that crosses the grid edge, is read as two pairs
        auto loadR4 = [&](const RLevel<P, C> &R1, int xr, int j, int c, int vq, A (&r)[4]) {
            if ((vq & 3) == 0 && vq >= 0 && vq + 3 < g.V) {
                R1.load4(xr, j, c, vq, r);
                return;
            }
            const A ev = renv<P, C, ENV>(pl, q, n + 1, j, c);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int vp = vq + 2 * h;
                if (vp >= 0 && vp < g.V) {
                    R1.load2(xr, j, c, vp, r[2 * h], r[2 * h + 1]);
                    if (vp + 1 >= g.V) r[2 * h + 1] = ev;
                } else {
                    r[2 * h] = r[2 * h + 1] = ev;
                }
            }
        };
        if (x & 1) {   // Eq. 14
            TLevel<P, C> Tn(pl, q, n);
            const int xq = (x + 1) >> 1;
            const bool rq_ok = !top && xq < g.Un[n + 1];
            RLevel<P, C> R1(pl, q, rq_ok ? n + 1 : n);
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
                const int kk = sg == 0 ? ip + 1 : ip;
                const int j = sg == 0 ? 2 * ip + 1 : 2 * ip;
                const A Aj = sg == 0 ? Ap : Am;
                Iv<P, C> t[4];
                Tn.load4(x, kk, v, t);
                const int vq = v + 2 * kk - s;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    A r[4];
                    if (rq_ok) loadR4(R1, xq, j, c, vq, r);
                    else r[0] = r[1] = r[2] = r[3] = renv<P, C, ENV>(pl, q, n + 1, j, c);
#pragma unroll
                    for (int l = 0; l < 4; ++l) acc[l][c] += fma(Aj, t[l].L[c], t[l].trans() * r[l]);
                }
            }
        } else {       // Eqs. 15-17
            TLevel<P, C> T1(pl, q, n + 1);
            const int x2 = x >> 1;
            const bool r1_ok = !top && x2 + 1 < g.Un[n + 1];
            RLevel<P, C> R1(pl, q, top ? n : n + 1);
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
                const int kk = sg == 0 ? 2 * ip + 2 : 2 * ip;
                const int j = sg == 0 ? 2 * ip + 1 : 2 * ip;
                const A Aj = sg == 0 ? Ap : Am;
                Iv<P, C> t[4];
                T1.load4(x2, kk, v, t);
                const int vq = v + 2 * kk - 2 * s;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    A r0[4], r1[4];
                    const A ev = renv<P, C, ENV>(pl, q, n + 1, j, c);
                    if (!top) R1.load4(x2, j, c, v, r0);
                    else r0[0] = r0[1] = r0[2] = r0[3] = ev;
                    if (r1_ok) loadR4(R1, x2 + 1, j, c, vq, r1);
                    else r1[0] = r1[1] = r1[2] = r1[3] = ev;
#pragma unroll
                    for (int l = 0; l < 4; ++l)
                        acc[l][c] += A(0.5) * (r0[l] + fma(Aj, t[l].L[c], t[l].trans() * r1[l]));
                }
            }
        }
        return;
    }
    // R_{n+1}(xr, j, vq .. vq+E-1); outside [0, V) the environment's value
    auto loadR = [&](const RLevel<P, C> &R1, int xr, int j, int c, int vq, A (&r)[E]) {
        if (PAIR) {
            if (vq >= 0 && vq < g.V) {
                R1.load2(xr, j, c, vq, r[0], r[E - 1]);
                if (vq + 1 >= g.V) r[E - 1] = renv<P, C, ENV>(pl, q, n + 1, j, c);
            } else {
                r[0] = r[E - 1] = renv<P, C, ENV>(pl, q, n + 1, j, c);
            }
        } else {
            r[0] = (vq >= 0 && vq < g.V) ? R1.load(xr, j, c, vq) : renv<P, C, ENV>(pl, q, n + 1, j, c);
        }
    };
    auto loadT = [&](const TLevel<P, C> &T, int xx, int kk, Iv<P, C> (&t)[E]) {
        if (PAIR) T.load2(xx, kk, v, t[0], t[E - 1]);
        else t[0] = T.load_ef(xx, kk, v, l2_evict_first());   // level 0: T rows read once from HBM
    };
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
            Iv<P, C> t[E];
            loadT(Tn, x, kk, t);
            const int vq = v + 2 * kk - s;
            RLevel<P, C> R1(pl, q, rq_ok ? n + 1 : n);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                A r[E];
                if (rq_ok) loadR(R1, xq, j, c, vq, r);
                else
#pragma unroll
                    for (int l = 0; l < E; ++l) r[l] = renv<P, C, ENV>(pl, q, n + 1, j, c);
#pragma unroll
                for (int l = 0; l < E; ++l) acc[l][c] += fma(Aj, t[l].L[c], t[l].trans() * r[l]);
            }
        }
    } else {
        // Eqs. 15-17 with Sec. 4.1: F_+- = (R_{n+1}(p, j) + A T_{n+1}(p, 2i +- 1).L
        //                                    + T_{n+1}(p, 2i +- 1).T R_{n+1}(p + v_{n+1}(2i +- 1), j)) / 2
        TLevel<P, C> T1(pl, q, n + 1);
        const int x2 = x >> 1;
        const int s1 = 2 * s;
        const bool r1_ok = !top && x2 + 1 < g.Un[n + 1];
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
            const int kk = sg == 0 ? 2 * ip + 2 : 2 * ip;
            const int j = sg == 0 ? 2 * ip + 1 : 2 * ip;
            const A Aj = sg == 0 ? Ap : Am;
            Iv<P, C> t[E];
            loadT(T1, x2, kk, t);
            const int vq = v + 2 * kk - s1;
            RLevel<P, C> R1(pl, q, top ? n : n + 1);
#pragma unroll
            for (int c = 0; c < C; ++c) {
                A r0[E], r1[E];
                const A ev = renv<P, C, ENV>(pl, q, n + 1, j, c);
#pragma unroll
                for (int l = 0; l < E; ++l) { r0[l] = ev; r1[l] = ev; }
                if (!top) {
                    if (PAIR) R1.load2(x2, j, c, v, r0[0], r0[E - 1]);
                    else r0[0] = R1.load(x2, j, c, v);
                }
                if (r1_ok) loadR(R1, x2 + 1, j, c, vq, r1);
#pragma unroll
                for (int l = 0; l < E; ++l)
                    acc[l][c] += A(0.5) * (r0[l] + fma(Aj, t[l].L[c], t[l].trans() * r1[l]));
            }
        }
    }
}

// One row segment of R_n with four consecutive v per thread (n >= 1).
template <int P, int C, bool ENV = false>
__device__ __forceinline__ void body_merge_down4(const Plan &pl, const RowSplit &rs, int n, long long bx, int by) {
    using A = typename Prec<P>::A;
    int local;
    const int q = find_quadrant(rs, bx, local);
    const QuadGeom &g = pl.q[q];
    const int v = 4 * (by * blockDim.x + threadIdx.x);
    if (v >= g.V) return;
    const int I = 1 << n;
    local += I;
    const int x = local >> n, ip = local & (I - 1);
    A acc[4][C];
    merge_down_entry<P, C, 4, ENV>(pl, q, n, x, ip, v, acc);
    RLevel<P, C> Rn(pl, q, n);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        A o[4] = {acc[0][c], acc[1][c], acc[2][c], acc[3][c]};
        Rn.store4(x, ip, c, v, o);
    }
}

// One row segment of R_n: row = (q, x, ip), x >= 1 (column 0 is dead).
template <int P, int C, bool PAIR, bool ENV = false>
__device__ __forceinline__ void body_merge_down(const Plan &pl, const RowSplit &rs, int n, long long bx, int by) {
    using A = typename Prec<P>::A;
    constexpr int E = PAIR ? 2 : 1;
    int local;
    const int q = find_quadrant(rs, bx, local);
    const QuadGeom &g = pl.q[q];
    const int v = E * (by * blockDim.x + threadIdx.x);
    if (v >= g.V) return;
    const int I = 1 << n;
    local += I;
    const int x = local >> n, ip = local & (I - 1);
    A acc[E][C];
    merge_down_entry<P, C, E, ENV>(pl, q, n, x, ip, v, acc);
    RLevel<P, C> Rn(pl, q, n);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        if (PAIR) Rn.store2(x, ip, c, v, acc[0][c], acc[E - 1][c]);
        else Rn.store(x, ip, c, v, acc[0][c]);
    }
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
__device__ __forceinline__ void body_merge_down_bulk(const Plan &pl, const RowSplit &rs, int n, long long row, int vb,
                                                     unsigned char *smem, uint64_t &bar) {
    using SL = typename Prec<P>::SL;
    using ST = typename Prec<P>::ST;
    using A = typename Prec<P>::A;
    using B = BulkMD<P, C>;
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


// R_0^q(x, 0, v) and R_0^q(x, 0, v + 1) (v even) added to a[0] / a[1]: the
// n = 0 case of merge_down_entry for a pair of v, with the same arithmetic
// per entry.  At odd x the far run starts at the odd offset v -+ 1 and is
// read as the aligned pairs on either side of it; v + 1 may lie past V
// (inside the padded row): that entry is computed and never used.
template <int P, int C, bool ENV>
__device__ __forceinline__ void r0_pair_add(const Plan &pl, int q, int x, int v, typename Prec<P>::A (&a)[2][C]) {
    using A = typename Prec<P>::A;
    const QuadGeom &g = pl.q[q];
    if (g.N < 1 || x >= g.U) {                 // the probe at u + 1 is outside: the environment
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const A ev = renv<P, C, ENV>(pl, q, 0, 0, c);
            a[0][c] += ev;
            a[1][c] += ev;
        }
        return;
    }
    const bool top = g.N <= 1;                  // R_1 is R_N: 0, or the environment map
    const A Ap = arc<P>(pl, 1, 1), Am = arc<P>(pl, 1, 0);
    const uint64_t pol = l2_evict_first();      // T rows: read once from HBM
    A acc[2][C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[0][c] = acc[1][c] = A(0);
    if (x & 1) {                                // Eq. 14 at n = 0: k = j = 1, 0
        const TLevel<P, C> T0(pl, q, 0);
        const int xq = (x + 1) >> 1;
        const bool rq_ok = !top && xq < g.Un[1];
        const RLevel<P, C> R1(pl, q, rq_ok ? 1 : 0);
#pragma unroll
        for (int j = 1; j >= 0; --j) {
            const A Aj = j ? Ap : Am;
            Iv<P, C> t0, t1;
            T0.load2_ef(x, j, v, pol, t0, t1);
            const A tr0 = t0.trans(), tr1 = t1.trans();
            const int vq = v + 2 * j - 1;       // odd
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A ev = renv<P, C, ENV>(pl, q, 1, j, c);
                A r0 = ev, r1 = ev, lo, hi;
                if (rq_ok) {
                    if (vq >= 0 && vq < g.V) {
                        R1.load2(xq, j, c, vq - 1, lo, hi);
                        r0 = hi;
                    }
                    if (vq + 1 < g.V) {
                        R1.load2(xq, j, c, vq + 1, lo, hi);
                        r1 = lo;
                    }
                }
                acc[0][c] += fma(Aj, t0.L[c], tr0 * r0);
                acc[1][c] += fma(Aj, t1.L[c], tr1 * r1);
            }
        }
    } else {                                    // Eqs. 15-17 at n = 0: k = 2, 0 and j = 1, 0
        const TLevel<P, C> T1(pl, q, 1);
        const int x2 = x >> 1;
        const bool r1_ok = !top && x2 + 1 < g.Un[1];
        const RLevel<P, C> R1(pl, q, top ? 0 : 1);
#pragma unroll
        for (int j = 1; j >= 0; --j) {
            const A Aj = j ? Ap : Am;
            Iv<P, C> t0, t1;
            T1.load2_ef(x2, 2 * j, v, pol, t0, t1);
            const A tr0 = t0.trans(), tr1 = t1.trans();
            const int vq = v + 4 * j - 2;       // even
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A ev = renv<P, C, ENV>(pl, q, 1, j, c);
                A n0 = ev, n1 = ev, f0 = ev, f1 = ev;
                if (!top) R1.load2(x2, j, c, v, n0, n1);
                if (r1_ok && vq >= 0 && vq < g.V) {
                    R1.load2(x2 + 1, j, c, vq, f0, f1);
                    if (vq + 1 >= g.V) f1 = ev;
                }
                acc[0][c] += A(0.5) * (n0 + fma(Aj, t0.L[c], tr0 * f0));
                acc[1][c] += A(0.5) * (n1 + fma(Aj, t1.L[c], tr1 * f1));
            }
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
        a[0][c] += acc[0][c];
        a[1][c] += acc[1][c];
    }
}

// F[c][y][x] = sum_q R_0^q(u_q + 1, v_q)   (Algorithm 1, Lighting, +1 offset),
// with R_0 computed in place (r0_pair_add): R_0 feeds only this sum, so it
// is never stored.  One block per 32 x 32 image tile (any multiple of 32
// threads).  Frames q0, q1 run v along image y and q2, q3 along image x, so
// the first pair is computed with v along y, parked in shared memory, and the
// second pair with v along x adds to it and writes F; the sum runs in frame
// order q0 + q1 + q2 + q3.  A thread takes two consecutive pixels along v
// (one 2-wide access per plane and row), a half-warp one tile line; the two
// half-warps take lines 2 apart, so the warp's x = u + 1 share one parity and
// it runs one branch of the merge.
template <int P, int C>
constexpr size_t fluence_smem() { return sizeof(typename Prec<P>::A) * C * 32 * 33; }

template <int P, int C, class OUT, bool ENV = false>
__device__ __forceinline__ void body_fluence(const Plan &pl, OUT *__restrict__ F, int bx, int by, unsigned char *smem) {
    using A = typename Prec<P>::A;
    A (*tile)[32][33] = reinterpret_cast<A (*)[32][33]>(smem);   // [C][y][x] of the tile
    const int W = pl.W, H = pl.H;
    const int x0 = bx * 32, y0 = by * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int hl = lane & 15, half = lane >> 4;
    // line pair p = 0 .. 15 -> tile lines 4 (p >> 1) + (p & 1) + {0, 2}
    auto line = [&](int p) { return 4 * (p >> 1) + (p & 1) + 2 * half; };
    auto add_frame = [&](int q, int x, int y, A (&a)[2][C]) {
        int u, v;
        image_to_frame(q, W, H, x, y, u, v);
        r0_pair_add<P, C, ENV>(pl, q, u + 1, v, a);
    };
    for (int p = warp; p < 16; p += nw) {       // q0, q1: pixels (x, y), (x, y + 1)
        const int ca = line(p), y = y0 + 2 * hl;
        A a[2][C];
#pragma unroll
        for (int c = 0; c < C; ++c) a[0][c] = a[1][c] = A(0);
        if (y < H && x0 + ca < W) {
            add_frame(0, x0 + ca, y, a);
            add_frame(1, x0 + ca, y, a);
        }
#pragma unroll
        for (int c = 0; c < C; ++c) {
            tile[c][2 * hl][ca] = a[0][c];
            tile[c][2 * hl + 1][ca] = a[1][c];
        }
    }
    __syncthreads();
    const long long HW = (long long)W * H;
    // F rows of even width from an aligned base take 2-wide stores
    const bool wide = (W & 1) == 0 && (reinterpret_cast<uintptr_t>(F) & (2 * sizeof(OUT) - 1)) == 0;
    auto put = [&](int y, int x, const A (&a)[2][C]) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            OUT *o = F + c * HW + (long long)y * W + x;
            if (wide) {
                st2(o, a[0][c], a[1][c]);
            } else {
                o[0] = (OUT)a[0][c];
                if (x + 1 < W) o[1] = (OUT)a[1][c];
            }
        }
    };
    for (int p = warp; p < 16; p += nw) {       // q2, q3: pixels (x, y), (x + 1, y)
        const int ra = line(p), x = x0 + 2 * hl;
        if (x >= W || y0 + ra >= H) continue;
        A a[2][C];
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int e = 0; e < 2; ++e) a[e][c] = tile[c][ra][2 * hl + e];
        add_frame(2, x, y0 + ra, a);
        add_frame(3, x, y0 + ra, a);
        put(y0 + ra, x, a);
    }
}


// R_0^q(x, 0, v .. v + 3) (v a multiple of 4) added to a[0 .. 3]: the n = 0
// case of merge_down_entry for four consecutive v, with the same arithmetic
// per entry.  T rows and the near R row are read as aligned quads; a far
// run starts off the quad boundary (at v -+ 1 at odd x, v -+ 2 at even x)
// and is read as the aligned quad at v plus the one or two entries beyond
// it.  Entries v + l past V (inside the padded row) are computed and never
// used.
template <int P, int C, bool ENV>
__device__ __forceinline__ void r0_quad_add(const Plan &pl, int q, int x, int v, typename Prec<P>::A (&a)[4][C]) {
    using A = typename Prec<P>::A;
    const QuadGeom &g = pl.q[q];
    if (g.N < 1 || x >= g.U) {                 // the probe at u + 1 is outside: the environment
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const A ev = renv<P, C, ENV>(pl, q, 0, 0, c);
#pragma unroll
            for (int l = 0; l < 4; ++l) a[l][c] += ev;
        }
        return;
    }
    const bool top = g.N <= 1;                  // R_1 is R_N: 0, or the environment map
    const A Ap = arc<P>(pl, 1, 1), Am = arc<P>(pl, 1, 0);
    const uint64_t pol = l2_evict_first();      // T rows: read once from HBM
    const int V = g.V;
    A acc[4][C];
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) acc[l][c] = A(0);
    if (x & 1) {                                // Eq. 14 at n = 0: k = j = 1, 0
        const TLevel<P, C> T0(pl, q, 0);
        const int xq = (x + 1) >> 1;
        const bool rq_ok = !top && xq < g.Un[1];
        const RLevel<P, C> R1(pl, q, rq_ok ? 1 : 0);
#pragma unroll
        for (int j = 1; j >= 0; --j) {
            const A Aj = j ? Ap : Am;
            Iv<P, C> t[4];
            T0.load4_ef(x, j, v, pol, t);
            A tr[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) tr[l] = t[l].trans();
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A ev = renv<P, C, ENV>(pl, q, 1, j, c);
                A r[4] = {ev, ev, ev, ev}, w[4];
                if (rq_ok) {
                    // far run v + 2j - 1 .. v + 2j + 2: the quad at v and the entry before or after it
                    R1.load4(xq, j, c, v, w);
                    if (j) {
#pragma unroll
                        for (int l = 0; l < 3; ++l)
                            if (v + 1 + l < V) r[l] = w[l + 1];
                        if (v + 4 < V) r[3] = R1.load(xq, j, c, v + 4);
                    } else {
                        if (v >= 1) r[0] = R1.load(xq, j, c, v - 1);
#pragma unroll
                        for (int l = 1; l < 4; ++l)
                            if (v + l - 1 < V) r[l] = w[l - 1];
                    }
                }
#pragma unroll
                for (int l = 0; l < 4; ++l) acc[l][c] += fma(Aj, t[l].L[c], tr[l] * r[l]);
            }
        }
    } else {                                    // Eqs. 15-17 at n = 0: k = 2, 0 and j = 1, 0
        const TLevel<P, C> T1(pl, q, 1);
        const int x2 = x >> 1;
        const bool r1_ok = !top && x2 + 1 < g.Un[1];
        const RLevel<P, C> R1(pl, q, top ? 0 : 1);
#pragma unroll
        for (int j = 1; j >= 0; --j) {
            const A Aj = j ? Ap : Am;
            Iv<P, C> t[4];
            T1.load4_ef(x2, 2 * j, v, pol, t);
            A tr[4];
#pragma unroll
            for (int l = 0; l < 4; ++l) tr[l] = t[l].trans();
#pragma unroll
            for (int c = 0; c < C; ++c) {
                const A ev = renv<P, C, ENV>(pl, q, 1, j, c);
                A n0[4] = {ev, ev, ev, ev}, f[4] = {ev, ev, ev, ev}, w[4];
                if (!top) R1.load4(x2, j, c, v, n0);
                if (r1_ok) {
                    // far run v + 4j - 2 .. v + 4j + 1: the quad at v and the pair after or before it
                    R1.load4(x2 + 1, j, c, v, w);
                    if (j) {
                        if (v + 2 < V) f[0] = w[2];
                        if (v + 3 < V) f[1] = w[3];
                        if (v + 4 < V) {
                            A p0, p1;
                            R1.load2(x2 + 1, j, c, v + 4, p0, p1);
                            f[2] = p0;
                            if (v + 5 < V) f[3] = p1;
                        }
                    } else {
                        if (v >= 2) R1.load2(x2 + 1, j, c, v - 2, f[0], f[1]);
                        if (v < V) f[2] = w[0];
                        if (v + 1 < V) f[3] = w[1];
                    }
                }
#pragma unroll
                for (int l = 0; l < 4; ++l) acc[l][c] += A(0.5) * (n0[l] + fma(Aj, t[l].L[c], tr[l] * f[l]));
            }
        }
    }
#pragma unroll
    for (int l = 0; l < 4; ++l)
#pragma unroll
        for (int c = 0; c < C; ++c) a[l][c] += acc[l][c];
}

// body_fluence with four consecutive pixels along v per thread (one 4-wide
// access per plane and row; r0_quad_add), eight lanes one tile line; a
// warp's four line groups are lines two apart, so its x = u + 1 share one
// parity and it runs one branch of the merge.  Same sum, same order, same
// shared tile.  Used for the 16-bit storage modes on large grids, where a
// 2-wide access moves only 4 bytes of radiance (any multiple of 32 threads;
// 8 warps keep every line group busy).
template <int P, int C, class OUT, bool ENV = false>
__device__ __forceinline__ void body_fluence4(const Plan &pl, OUT *__restrict__ F, int bx, int by, unsigned char *smem) {
    using A = typename Prec<P>::A;
    A (*tile)[32][33] = reinterpret_cast<A (*)[32][33]>(smem);   // [C][y][x] of the tile
    const int W = pl.W, H = pl.H;
    const int x0 = bx * 32, y0 = by * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int ql = lane & 7, grp = lane >> 3;
    // line group p = 0 .. 7 -> tile lines 8 (p >> 1) + (p & 1) + 2 grp
    auto line = [&](int p) { return 8 * (p >> 1) + (p & 1) + 2 * grp; };
    auto add_frame = [&](int q, int x, int y, A (&a)[4][C]) {
        int u, v;
        image_to_frame(q, W, H, x, y, u, v);
        r0_quad_add<P, C, ENV>(pl, q, u + 1, v, a);
    };
    for (int p = warp; p < 8; p += nw) {        // q0, q1: pixels (x, y .. y + 3)
        const int ca = line(p), y = y0 + 4 * ql;
        A a[4][C];
#pragma unroll
        for (int l = 0; l < 4; ++l)
#pragma unroll
            for (int c = 0; c < C; ++c) a[l][c] = A(0);
        if (y < H && x0 + ca < W) {
            add_frame(0, x0 + ca, y, a);
            add_frame(1, x0 + ca, y, a);
        }
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int l = 0; l < 4; ++l) tile[c][4 * ql + l][ca] = a[l][c];
    }
    __syncthreads();
    const long long HW = (long long)W * H;
    // F rows whose width is a multiple of 4, from an aligned base, take 4-wide stores
    const bool wide = (W & 3) == 0 && (reinterpret_cast<uintptr_t>(F) & (4 * sizeof(OUT) - 1)) == 0;
    for (int p = warp; p < 8; p += nw) {        // q2, q3: pixels (x .. x + 3, y)
        const int ra = line(p), x = x0 + 4 * ql;
        if (x >= W || y0 + ra >= H) continue;
        A a[4][C];
#pragma unroll
        for (int c = 0; c < C; ++c)
#pragma unroll
            for (int l = 0; l < 4; ++l) a[l][c] = tile[c][ra][4 * ql + l];
        add_frame(2, x, y0 + ra, a);
        add_frame(3, x, y0 + ra, a);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            OUT *o = F + c * HW + (long long)(y0 + ra) * W + x;
            if (wide) {
                const OUT t[4] = {(OUT)a[0][c], (OUT)a[1][c], (OUT)a[2][c], (OUT)a[3][c]};
                st4(o, t);
            } else {
#pragma unroll
                for (int l = 0; l < 4; ++l)
                    if (x + l < W) o[l] = (OUT)a[l][c];
            }
        }
    }
}

}  // namespace hrc
