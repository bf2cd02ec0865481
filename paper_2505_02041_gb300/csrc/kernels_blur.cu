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
// The blur is a 5-point stencil over C + 1 planes: one thread per pixel,
// 32-wide rows of a 32 x 8 block so that every plane access is a coalesced
// row and the neighbour rows come from L1 / L2; DRAM sees each plane about
// once (read F_raw and sigma, write F: (2C + 1) * 4 bytes per pixel).
//
// The adjoint is the transpose for fixed sigma (the kept set is piecewise
// constant in sigma, so it adds nothing to dL/dsigma), in gather form: pixel
// m collects 4 g_m / w_m + sum over kept neighbours c of g_c / w_c, where
// w_c = 4 + (kept neighbours of c), read from a 2-pixel diamond of sigma.
#include <cuda_runtime.h>

#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

namespace {

template <class T> __device__ __forceinline__ T neg_exp(T s);
template <> __device__ __forceinline__ float neg_exp<float>(float s) { return expf(-s); }
template <> __device__ __forceinline__ double neg_exp<double>(double s) { return exp(-s); }

// exp(-sigma) at (x, y), or a value that no pixel can keep (outside)
template <class T> __device__ __forceinline__ T trans_at(const T *__restrict__ s, int W, int H, int x, int y) {
    if (x < 0 || x >= W || y < 0 || y >= H) return T(1e30);
    return neg_exp<T>(__ldg(s + (long long)y * W + x));
}

template <class T> __device__ __forceinline__ bool kept(T tc, T tm, T thr) {
    return fabs(tc - tm) <= thr;   // tm = 1e30 outside the grid: never kept
}

template <class T>
__global__ void __launch_bounds__(256) k_cross_blur(int W, int H, int C, const T *__restrict__ Fr,
                                                    const T *__restrict__ s, T *__restrict__ F, T thr) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    const T tc = trans_at(s, W, H, x, y);
    const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
    bool k[4];
    T w = T(4);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        k[d] = kept(tc, trans_at(s, W, H, x + dx[d], y + dy[d]), thr);
        w += k[d] ? T(1) : T(0);
    }
    const T inv = T(1) / w;
    const long long HW = (long long)W * H, pix = (long long)y * W + x;
    for (int c = 0; c < C; ++c) {
        const T *p = Fr + c * HW;
        T a = T(4) * __ldg(p + pix);
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (k[d]) a += __ldg(p + pix + (long long)dy[d] * W + dx[d]);
        F[c * HW + pix] = a * inv;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_cross_blur_adj(int W, int H, int C, const T *__restrict__ g,
                                                        const T *__restrict__ s, T *__restrict__ gFr, T thr) {
    const int x = blockIdx.x * 32 + threadIdx.x, y = blockIdx.y * 8 + threadIdx.y;
    if (x >= W || y >= H) return;
    const int dx[4] = {1, -1, 0, 0}, dy[4] = {0, 0, 1, -1};
    const T tm = trans_at(s, W, H, x, y);
    // kept neighbours c of m, and the weight sum w_c of each
    bool k[4];
    T inv_c[4];
    T wm = T(4);
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int cx = x + dx[d], cy = y + dy[d];
        const T tcn = trans_at(s, W, H, cx, cy);
        k[d] = kept(tm, tcn, thr);
        wm += k[d] ? T(1) : T(0);
        T wc = T(4);
        if (k[d]) {
#pragma unroll
            for (int e = 0; e < 4; ++e)
                wc += kept(tcn, trans_at(s, W, H, cx + dx[e], cy + dy[e]), thr) ? T(1) : T(0);
        }
        inv_c[d] = T(1) / wc;
    }
    const T inv_m = T(1) / wm;
    const long long HW = (long long)W * H, pix = (long long)y * W + x;
    for (int c = 0; c < C; ++c) {
        const T *p = g + c * HW;
        T a = T(4) * __ldg(p + pix) * inv_m;
#pragma unroll
        for (int d = 0; d < 4; ++d)
            if (k[d]) a += __ldg(p + pix + (long long)dy[d] * W + dx[d]) * inv_c[d];
        gFr[c * HW + pix] = a;
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
    const dim3 block(32, 8), grid((pl.W + 31) / 32, (pl.H + 7) / 8);
    rec->begin(K_CROSS_BLUR, 0, bytes_cross_blur(pl));
    if (pl.prec == P_FP64)
        k_cross_blur<double><<<grid, block, 0, st>>>(pl.W, pl.H, pl.C, (const double *)Fr, (const double *)s,
                                                     (double *)F, thr);
    else
        k_cross_blur<float><<<grid, block, 0, st>>>(pl.W, pl.H, pl.C, (const float *)Fr, (const float *)s,
                                                    (float *)F, (float)thr);
    rec->end();
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_cross_blur_adj(const Plan &pl, const void *g, const void *s, void *gFr, double thr,
                                  cudaStream_t st, int *launches, Recorder *rec) {
    const dim3 block(32, 8), grid((pl.W + 31) / 32, (pl.H + 7) / 8);
    rec->begin(K_ADJ_CROSS_BLUR, 0, bytes_cross_blur(pl));
    if (pl.prec == P_FP64)
        k_cross_blur_adj<double><<<grid, block, 0, st>>>(pl.W, pl.H, pl.C, (const double *)g, (const double *)s,
                                                         (double *)gFr, thr);
    else
        k_cross_blur_adj<float><<<grid, block, 0, st>>>(pl.W, pl.H, pl.C, (const float *)g, (const float *)s,
                                                        (float *)gFr, (float)thr);
    rec->end();
    ++*launches;
    return cudaGetLastError();
}

}  // namespace hrc
