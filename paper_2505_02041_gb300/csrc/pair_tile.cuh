// pair_tile.cuh -- the staged image tile of the adjoint trace.
//
// The adjoint of the directly traced levels (Sec. 4.2) is gathered one
// quadrant pair at a time: pair 0 = frames q0, q1 (u along image x), pair 1 =
// frames q2, q3 (u along image y).  A block covers a tile
// of PT_U pixels along u by PT_V pixels along v; the region staged in shared
// memory adds a PT_HALO-pixel halo on every side (the longest directly
// traced ray, v_2(k), reaches 4 pixels along and across).  The region is
// stored as [a][b] with a along u and b along v, so a warp's lanes (32
// consecutive v) read consecutive words in every frame.
//
// Per region pixel it holds, for the three ray classes c of trace_shapes.cuh
// (half length l_c), the half-piece factors {t, w} = {exp(-sigma l_c),
// l_c phi(sigma l_c)} (Eq. 4 over a uniform piece) and dw/dsigma, and the
// emission with the extinction.  Outside the image every field is vacuum
// (sigma = e = 0, t = 1, w = l_c, dw/dsigma = -l_c^2 / 2), which is exact.
#pragma once

#include <type_traits>

#include "bulk_copy.cuh"
#include "hrc_internal.cuh"
#include "trace_shapes.cuh"

namespace hrc {

constexpr int PT_U = 16, PT_V = 32, PT_HALO = 4;
constexpr int PT_RU = PT_U + 2 * PT_HALO, PT_RV = PT_V + 2 * PT_HALO, PT_PITCH = PT_RV + 1;
constexpr int PT_PLANE = PT_RU * PT_PITCH;

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

template <class A, int C> struct PairTile {
    using V2 = typename Vec2<A>::T;
    V2 *tw;        // [3][PLANE]
    A *dw;         // [3][PLANE]
    float4 *es4;   // [PLANE] when packed
    A *e;          // [C][PLANE] otherwise
    A *s;          // [PLANE] otherwise
    __device__ __forceinline__ explicit PairTile(unsigned char *smem) {
        tw = reinterpret_cast<V2 *>(smem);
        dw = reinterpret_cast<A *>(tw + 3 * PT_PLANE);
        es4 = reinterpret_cast<float4 *>(dw + 3 * PT_PLANE);
        e = dw + 3 * PT_PLANE;
        s = e + C * PT_PLANE;
    }
    static_assert((sizeof(A) * 3 * PT_PLANE) % 16 == 0, "16-byte aligned planes");
    static constexpr size_t bytes() {
        return (sizeof(V2) + sizeof(A)) * 3 * PT_PLANE +
               (PackES<A, C>::packed ? sizeof(float4) * PT_PLANE : sizeof(A) * (C + 1) * PT_PLANE);
    }
    __device__ __forceinline__ void piece(int cls, int o, A &t, A &w, A &d) const {
        const V2 p = tw[cls * PT_PLANE + o];
        t = p.x;
        w = p.y;
        d = dw[cls * PT_PLANE + o];
    }
    __device__ __forceinline__ void emis(int o, A (&em)[C], A &sg) const {
        if constexpr (PackES<A, C>::packed) {
            const float4 v = es4[o];
            em[0] = v.x;
            if constexpr (C > 1) em[1] = v.y;
            if constexpr (C > 2) em[2] = v.z;
            sg = v.w;
        } else {
#pragma unroll
            for (int c = 0; c < C; ++c) em[c] = e[c * PT_PLANE + o];
            sg = s[o];
        }
    }
    __device__ __forceinline__ A sigma(int o) const {
        if constexpr (PackES<A, C>::packed) return es4[o].w;
        else return s[o];
    }
    // Stage the region of the tile whose origin (along u, along v) in the
    // frames of `pair` is the image tile (x0, y0).  Threads walk the region
    // along image x so the global reads are coalesced.
    template <class IN>
    __device__ __forceinline__ void stage(int pair, int W, int H, int x0, int y0, const IN *__restrict__ ein,
                                          const IN *__restrict__ sin) {
        const long long HW = (long long)W * H;
        const int nx = pair == 0 ? PT_RU : PT_RV;     // region extent along image x
        for (int i = threadIdx.x; i < PT_RU * PT_RV; i += blockDim.x) {
            const int ix = i % nx, iy = i / nx;
            const int x = x0 - PT_HALO + ix, y = y0 - PT_HALO + iy;
            const int a = pair == 0 ? ix : iy, b = pair == 0 ? iy : ix;
            const int o = a * PT_PITCH + b;
            const bool in = x >= 0 && x < W && y >= 0 && y < H;
            const long long pix = (long long)y * W + x;
            const A sg = in ? A(sin[pix]) : A(0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const A len = class_len<A>(c);
                const A m = fexpm1(-sg * len);
                V2 p;
                p.x = A(1) + m;
                p.y = sg != A(0) ? -m / sg : len;
                tw[c * PT_PLANE + o] = p;
                dw[c * PT_PLANE + o] = dw_dsigma(sg, len, p.x);
            }
            if constexpr (PackES<A, C>::packed) {
                float4 v = make_float4(0.f, 0.f, 0.f, (float)sg);
                if (in) {
                    v.x = float(ein[pix]);
                    if constexpr (C > 1) v.y = float(ein[HW + pix]);
                    if constexpr (C > 2) v.z = float(ein[2 * HW + pix]);
                }
                es4[o] = v;
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) e[c * PT_PLANE + o] = in ? A(ein[c * HW + pix]) : A(0);
                s[o] = sg;
            }
        }
    }
    // The same staging with the region of e and sigma fetched by TMA tensor
    // copies (fp32; box PT_RU x PT_RV along image x, y for pair 0, PT_RV x
    // PT_RU for pair 1; zero outside the grid = vacuum).  The boxes land in a
    // staging area overlapping the tw planes: every thread takes its pixels
    // into registers first, then the planes are written.  Returns 0, or
    // kWaitTimeout / kWaitLost when the copy wait gave up.
    __device__ __forceinline__ int stage_tma(int pair, int x0, int y0, const CUtensorMap *tme, const CUtensorMap *tms,
                                             uint64_t *bar, long long limit_ns) {
        static_assert(sizeof(A) == 4, "fp32 staging");
        constexpr int BOX = PT_RU * PT_RV;
        constexpr int PER = (BOX + 255) / 256;
        static_assert((C + 1) * BOX * 4 <= 3 * PT_PLANE * 8, "staging fits the tw planes");
        float *stg = reinterpret_cast<float *>(tw);   // [C + 1][BOX]
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_arrive_expect(bar, (unsigned)((C + 1) * BOX * sizeof(float)));
#pragma unroll
            for (int c = 0; c < C; ++c) tma_load_3d(stg + c * BOX, tme, x0 - PT_HALO, y0 - PT_HALO, c, bar);
            tma_load_2d(stg + C * BOX, tms, x0 - PT_HALO, y0 - PT_HALO, bar);
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
        const int nx = pair == 0 ? PT_RU : PT_RV;     // box extent along image x
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int i = threadIdx.x + 256 * k;
            if (i >= BOX) break;
            const int ix = i % nx, iy = i / nx;
            const int a = pair == 0 ? ix : iy, b = pair == 0 ? iy : ix;
            const int o = a * PT_PITCH + b;
            const A sg = sv[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const A len = class_len<A>(c);
                const A m = fexpm1(-sg * len);
                V2 p;
                p.x = A(1) + m;
                p.y = sg != A(0) ? -m / sg : len;
                tw[c * PT_PLANE + o] = p;
                dw[c * PT_PLANE + o] = dw_dsigma(sg, len, p.x);
            }
            if constexpr (PackES<A, C>::packed) {
                float4 v = make_float4(ev[k][0], 0.f, 0.f, sg);
                if constexpr (C > 1) v.y = ev[k][1];
                if constexpr (C > 2) v.z = ev[k][2];
                es4[o] = v;
            } else {
#pragma unroll
                for (int c = 0; c < C; ++c) e[c * PT_PLANE + o] = ev[k][c];
                s[o] = sg;
            }
        }
        return 0;
    }
};

// Frame geometry of a tile column: quadrant q of pair p, tile origin (x0,
// y0); column c (along u) and lane (along v).
struct PairGeom {
    int u, v;          // frame coordinates of the pixel
    int base;          // region offset of the pixel
    int su;            // region step for +1 along u (+-PT_PITCH); +1 along v is +1
    bool valid;        // pixel inside the image
};

__device__ __forceinline__ PairGeom pair_geom(const Plan &pl, int q, int x0, int y0, int c, int lane) {
    PairGeom g;
    const bool xu = q < 2;
    const int tu = xu ? x0 : y0, tv = xu ? y0 : x0;
    const int ext_u = xu ? pl.W : pl.H, ext_v = xu ? pl.H : pl.W;
    const bool fwd = (q == 0 || q == 2);
    g.valid = tu + c < ext_u && tv + lane < ext_v;
    g.u = fwd ? tu + c : ext_u - 1 - (tu + c);
    g.v = tv + lane;
    g.base = (PT_HALO + c) * PT_PITCH + PT_HALO + lane;
    g.su = fwd ? PT_PITCH : -PT_PITCH;
    return g;
}

// Tile grid of a quadrant pair.
__host__ __device__ inline int pair_tiles_x(int pair, int W) { return pair == 0 ? (W + PT_U - 1) / PT_U : (W + PT_V - 1) / PT_V; }
__host__ __device__ inline int pair_tiles_y(int pair, int H) { return pair == 0 ? (H + PT_V - 1) / PT_V : (H + PT_U - 1) / PT_U; }

}  // namespace hrc
