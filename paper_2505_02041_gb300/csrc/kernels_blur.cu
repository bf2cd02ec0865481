// kernels_blur.cu -- the cross blur of Sec. 4.2 (Eq. 21) after the fluence
// sum, and its adjoint.
//
// Each pixel becomes the weighted mean of itself (weight 4) and those of its
// four edge neighbours (weight 1 each) that lie inside the grid and whose
// opacity a = 1 - exp(-sigma) is within the threshold of its own; the kept
// weights are renormalised, so with every neighbour kept this is the
// 1/8 [0 1 0; 1 4 1; 0 1 0] stencil of Eq. 21.  The test
// |a_m - a_c| <= thr is written |exp(-sigma_c) - exp(-sigma_m)| <= thr.
//
// The blur is a 5-point stencil over C + 1 planes.  A block owns a 32 x TY
// output tile (TY = 32 for fp32, 16 for fp64) and stages its region with
// a 1-pixel halo in shared memory: t = exp(-sigma), computed once per
// staged pixel, and the C planes of the unblurred fluence; each output is
// then formed from shared memory and written as a coalesced row.  DRAM sees
// each plane about once ((2C + 1) element sizes per pixel); the halo rows
// (1/16 of a tile) come from L2.
//
// The adjoint is the transpose for fixed sigma (the kept set is piecewise
// constant in sigma, so it adds nothing to dL/dsigma), in gather form:
// pixel m collects 4 h_m + sum over its kept neighbours c of h_c, with
// h_c = g_c / w_c and w_c = 4 + (kept neighbours of c); keeping is
// symmetric, so m's own kept mask selects the terms.  A block stages t over
// its tile with a 2-pixel halo, then h and the kept masks over a 1-pixel
// halo, then gathers.
#include <cuda_runtime.h>

#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

namespace {

template <class T> __device__ __forceinline__ T neg_exp(T s);
template <> __device__ __forceinline__ float neg_exp<float>(float s) { return expf(-s); }
template <> __device__ __forceinline__ double neg_exp<double>(double s) { return exp(-s); }

// t of a pixel outside the grid: no pixel keeps it (|t_c - 1e30| > 1)
template <class T> __device__ __forceinline__ T t_outside() { return T(1e30); }

template <class T> __device__ __forceinline__ bool kept(T tc, T tm, T thr) { return fabs(tc - tm) <= thr; }

constexpr int kBX = 32, kBY = 8;
template <class T> constexpr int tile_y() { return sizeof(T) == 8 ? 16 : 32; }

template <class T, int C> constexpr size_t blur_smem() {
    return sizeof(T) * (size_t)(tile_y<T>() + 2) * (kBX + 2) * (1 + C);
}
template <class T, int C> constexpr size_t blur_adj_smem() {
    return sizeof(T) * ((size_t)(tile_y<T>() + 4) * (kBX + 4) + (size_t)C * (tile_y<T>() + 2) * (kBX + 2)) +
           (size_t)(tile_y<T>() + 2) * (kBX + 2);
}

template <class T, int C>
__global__ void __launch_bounds__(kBX * kBY, sizeof(T) == 4 ? 6 : 1) k_cross_blur(int W, int H, const T *__restrict__ Fr,
                                                          const T *__restrict__ s, T *__restrict__ F, T thr) {
    constexpr int TY = tile_y<T>(), RX = kBX + 2, RY = TY + 2, RP = RX * RY;
    __shared__ __align__(16) unsigned char smem[blur_smem<T, C>()];
    T *t = reinterpret_cast<T *>(smem);   // [RY][RX]
    T *f = t + RP;                        // [C][RY][RX]
    const int x0 = blockIdx.x * kBX - 1, y0 = blockIdx.y * TY - 1;
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const long long HW = (long long)W * H;
    // every global load of the staging first (one memory round trip), then
    // the exponentials and the shared-memory stores
    constexpr int NT = kBX * kBY, NIT = (RP + NT - 1) / NT;
    T sv[NIT], fv[NIT][C];
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int i = tid + k * NT, ry = i / RX, rx = i - ry * RX, gx = x0 + rx, gy = y0 + ry;
        const bool in = i < RP && gx >= 0 && gx < W && gy >= 0 && gy < H;
        const long long pix = (long long)gy * W + gx;
        sv[k] = in ? __ldg(s + pix) : T(0);
#pragma unroll
        for (int c = 0; c < C; ++c) fv[k][c] = in ? __ldg(Fr + c * HW + pix) : T(0);
    }
#pragma unroll
    for (int k = 0; k < NIT; ++k) {
        const int i = tid + k * NT, ry = i / RX, rx = i - ry * RX, gx = x0 + rx, gy = y0 + ry;
        if (i >= RP) break;
        const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
        t[i] = in ? neg_exp<T>(sv[k]) : t_outside<T>();
#pragma unroll
        for (int c = 0; c < C; ++c) f[c * RP + i] = fv[k][c];
    }
    __syncthreads();
    const int x = blockIdx.x * kBX + threadIdx.x;
    if (x >= W) return;
    for (int r = threadIdx.y; r < TY; r += kBY) {
        const int y = blockIdx.y * TY + r;
        if (y >= H) break;
        const int i = (r + 1) * RX + threadIdx.x + 1;
        const T tc = t[i];
        const bool k0 = kept(tc, t[i + 1], thr), k1 = kept(tc, t[i - 1], thr);
        const bool k2 = kept(tc, t[i + RX], thr), k3 = kept(tc, t[i - RX], thr);
        const T inv = T(1) / T(4 + (int)k0 + (int)k1 + (int)k2 + (int)k3);
        const long long pix = (long long)y * W + x;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const T *fc = f + c * RP;
            T a = T(4) * fc[i];
            if (k0) a += fc[i + 1];
            if (k1) a += fc[i - 1];
            if (k2) a += fc[i + RX];
            if (k3) a += fc[i - RX];
            F[c * HW + pix] = a * inv;
        }
    }
}

template <class T, int C>
__global__ void __launch_bounds__(kBX * kBY, sizeof(T) == 4 ? 6 : 1) k_cross_blur_adj(int W, int H, const T *__restrict__ g,
                                                              const T *__restrict__ s, T *__restrict__ gFr, T thr) {
    constexpr int TY = tile_y<T>();
    constexpr int RX2 = kBX + 4, RY2 = TY + 4, RP2 = RX2 * RY2;   // t: 2-pixel halo
    constexpr int RX = kBX + 2, RY = TY + 2, RP = RX * RY;        // h, masks: 1-pixel halo
    __shared__ __align__(16) unsigned char smem[blur_adj_smem<T, C>()];
    T *t = reinterpret_cast<T *>(smem);   // [RY2][RX2]
    T *h = t + RP2;                       // [C][RY][RX]
    unsigned char *mk = reinterpret_cast<unsigned char *>(h + C * RP);   // [RY][RX]
    const int tid = threadIdx.y * kBX + threadIdx.x;
    const long long HW = (long long)W * H;
    constexpr int NT = kBX * kBY, NIT2 = (RP2 + NT - 1) / NT, NIT = (RP + NT - 1) / NT;
    // every global load first: sigma over the 2-pixel halo, g over the
    // 1-pixel halo (one memory round trip)
    T sv[NIT2], gv[NIT][C];
    {
        const int x0 = blockIdx.x * kBX - 2, y0 = blockIdx.y * TY - 2;
#pragma unroll
        for (int k = 0; k < NIT2; ++k) {
            const int i = tid + k * NT, ry = i / RX2, rx = i - ry * RX2, gx = x0 + rx, gy = y0 + ry;
            const bool in = i < RP2 && gx >= 0 && gx < W && gy >= 0 && gy < H;
            sv[k] = in ? __ldg(s + (long long)gy * W + gx) : T(0);
        }
    }
    {
        const int x0 = blockIdx.x * kBX - 1, y0 = blockIdx.y * TY - 1;
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
            const int i = tid + k * NT, ry = i / RX, rx = i - ry * RX, gx = x0 + rx, gy = y0 + ry;
            const bool in = i < RP && gx >= 0 && gx < W && gy >= 0 && gy < H;
            const long long pix = (long long)gy * W + gx;
#pragma unroll
            for (int c = 0; c < C; ++c) gv[k][c] = in ? __ldg(g + c * HW + pix) : T(0);
        }
    }
    {
        const int x0 = blockIdx.x * kBX - 2, y0 = blockIdx.y * TY - 2;
#pragma unroll
        for (int k = 0; k < NIT2; ++k) {
            const int i = tid + k * NT, ry = i / RX2, rx = i - ry * RX2, gx = x0 + rx, gy = y0 + ry;
            if (i >= RP2) break;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            t[i] = in ? neg_exp<T>(sv[k]) : t_outside<T>();
        }
    }
    __syncthreads();
    {
        const int x0 = blockIdx.x * kBX - 1, y0 = blockIdx.y * TY - 1;
#pragma unroll
        for (int k = 0; k < NIT; ++k) {
            const int i = tid + k * NT, ry = i / RX, rx = i - ry * RX, gx = x0 + rx, gy = y0 + ry;
            if (i >= RP) break;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            unsigned m = 0;
            T inv = T(0);
            if (in) {
                const int j = (ry + 1) * RX2 + rx + 1;   // the same pixel in t
                const T tc = t[j];
                m = (unsigned)kept(tc, t[j + 1], thr) | (unsigned)kept(tc, t[j - 1], thr) << 1 |
                    (unsigned)kept(tc, t[j + RX2], thr) << 2 | (unsigned)kept(tc, t[j - RX2], thr) << 3;
                inv = T(1) / T(4 + __popc(m));
            }
            mk[i] = (unsigned char)m;
#pragma unroll
            for (int c = 0; c < C; ++c) h[c * RP + i] = gv[k][c] * inv;
        }
    }
    __syncthreads();
    const int x = blockIdx.x * kBX + threadIdx.x;
    if (x >= W) return;
    for (int r = threadIdx.y; r < TY; r += kBY) {
        const int y = blockIdx.y * TY + r;
        if (y >= H) break;
        const int i = (r + 1) * RX + threadIdx.x + 1;
        const unsigned m = mk[i];
        const long long pix = (long long)y * W + x;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const T *hc = h + c * RP;
            T a = T(4) * hc[i];
            if (m & 1u) a += hc[i + 1];
            if (m & 2u) a += hc[i - 1];
            if (m & 4u) a += hc[i + RX];
            if (m & 8u) a += hc[i - RX];
            gFr[c * HW + pix] = a;
        }
    }
}

}  // namespace

double bytes_cross_blur(const Plan &pl) {
    const double img = (double)pl.W * pl.H;
    const double esz = pl.prec == P_FP64 ? 8.0 : 4.0;
    return img * (2 * pl.C + 1) * esz;
}

cudaError_t launch_cross_blur(const Plan &pl, const void *Fr, const void *s, void *F, double thr, cudaStream_t st,
                              int *launches, Recorder *rec) {
    const dim3 block(kBX, kBY);
    const int ty = pl.prec == P_FP64 ? tile_y<double>() : tile_y<float>();
    const dim3 grid((pl.W + kBX - 1) / kBX, (pl.H + ty - 1) / ty);
    rec->begin(K_CROSS_BLUR, 0, bytes_cross_blur(pl));
    switch (pl.C) {
#define HRC_BLUR_CASE(CC)                                                                                         \
    case CC:                                                                                                      \
        if (pl.prec == P_FP64)                                                                                    \
            k_cross_blur<double, CC><<<grid, block, 0, st>>>(pl.W, pl.H, (const double *)Fr, (const double *)s,   \
                                                             (double *)F, thr);                                   \
        else                                                                                                      \
            k_cross_blur<float, CC><<<grid, block, 0, st>>>(pl.W, pl.H, (const float *)Fr, (const float *)s,      \
                                                            (float *)F, (float)thr);                              \
        break;
        HRC_BLUR_CASE(1) HRC_BLUR_CASE(2) HRC_BLUR_CASE(3) HRC_BLUR_CASE(4)
#undef HRC_BLUR_CASE
    default: return cudaErrorInvalidValue;
    }
    rec->end();
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_cross_blur_adj(const Plan &pl, const void *g, const void *s, void *gFr, double thr,
                                  cudaStream_t st, int *launches, Recorder *rec) {
    const dim3 block(kBX, kBY);
    const int ty = pl.prec == P_FP64 ? tile_y<double>() : tile_y<float>();
    const dim3 grid((pl.W + kBX - 1) / kBX, (pl.H + ty - 1) / ty);
    rec->begin(K_ADJ_CROSS_BLUR, 0, bytes_cross_blur(pl));
    switch (pl.C) {
#define HRC_BLUR_CASE(CC)                                                                                         \
    case CC:                                                                                                      \
        if (pl.prec == P_FP64)                                                                                    \
            k_cross_blur_adj<double, CC><<<grid, block, 0, st>>>(pl.W, pl.H, (const double *)g,                   \
                                                                 (const double *)s, (double *)gFr, thr);          \
        else                                                                                                      \
            k_cross_blur_adj<float, CC><<<grid, block, 0, st>>>(pl.W, pl.H, (const float *)g, (const float *)s,   \
                                                                (float *)gFr, (float)thr);                        \
        break;
        HRC_BLUR_CASE(1) HRC_BLUR_CASE(2) HRC_BLUR_CASE(3) HRC_BLUR_CASE(4)
#undef HRC_BLUR_CASE
    default: return cudaErrorInvalidValue;
    }
    rec->end();
    ++*launches;
    return cudaGetLastError();
}

}  // namespace hrc
