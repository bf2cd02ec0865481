// kernels_bounce.cu -- multiple diffuse bounces (Sec. 4.2: the output
// fluence fed into another iteration of the method), and their adjoint.
//
// Bounce k + 1 runs the whole forward on the emission
//     e_{k+1} = e + albedo * sigma * F_k / (2 pi)
// (isotropic single scattering in 2D: a pixel scatters albedo * sigma of
// the fluence F, the radiance integrated over the full turn, evenly over
// 2 pi).  The source update and its reverse are elementwise over C + 1
// planes: one thread per pixel, grid-stride, coalesced rows; 4-wide fp32
// accesses when the plane length is a multiple of 4.
//
// Reverse of one bounce k >= 1, given dL/de_k (ge_k) and dL/dsigma from the
// forward at e_k (gs_k):
//     dL/de      += ge_k
//     dL/dsigma  += gs_k + sum_c ge_k albedo F_{k-1} / (2 pi)
//     dL/dalbedo += ge_k sigma F_{k-1} / (2 pi)
//     dL/dF_{k-1} = ge_k albedo sigma / (2 pi)
// and of bounce 0: dL/de += ge_0, dL/dsigma += gs_0.  The first reverse step
// (k = K) overwrites the accumulators instead of adding.
#include <cuda_runtime.h>

#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

namespace {

template <class T> __device__ __forceinline__ T inv_two_pi() { return T(0.15915494309189533576888376337251436); }

// ss: stride between the channels' extinction planes (0: one plane shared
// by all channels; n: per-channel extinction)
template <class T, int C>
__global__ void __launch_bounds__(256) k_bounce_source(long long n, long long ss, const T *__restrict__ e,
                                                       const T *__restrict__ s, const T *__restrict__ a,
                                                       const T *__restrict__ F, T *__restrict__ eo) {
    const T k = inv_two_pi<T>();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const long long j = c * n + i;
            eo[j] = __ldg(e + j) + __ldg(a + j) * (__ldg(s + c * ss + i) * k) * __ldg(F + j);
        }
    }
}

// fp32, n % 4 == 0: 4-wide accesses (every plane starts 16-byte aligned)
template <int C>
__global__ void __launch_bounds__(256) k_bounce_source4(long long n4, long long ss4, const float4 *__restrict__ e,
                                                        const float4 *__restrict__ s, const float4 *__restrict__ a,
                                                        const float4 *__restrict__ F, float4 *__restrict__ eo) {
    const float k = inv_two_pi<float>();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < C; ++c) {
            float4 sg = __ldg(s + c * ss4 + i);
            sg.x *= k; sg.y *= k; sg.z *= k; sg.w *= k;
            const long long j = c * n4 + i;
            const float4 ev = __ldg(e + j), av = __ldg(a + j), fv = __ldg(F + j);
            eo[j] = make_float4(ev.x + av.x * sg.x * fv.x, ev.y + av.y * sg.y * fv.y, ev.z + av.z * sg.z * fv.z,
                                ev.w + av.w * sg.w * fv.w);
        }
    }
}

template <class T, int C>
__global__ void __launch_bounds__(256) k_bounce_adj(long long n, int first, int has_prev, const T *__restrict__ gek,
                                                    const T *__restrict__ gsk, const T *__restrict__ Fp,
                                                    const T *__restrict__ a, const T *__restrict__ s,
                                                    T *__restrict__ ge, T *__restrict__ gs, T *__restrict__ ga,
                                                    T *__restrict__ gFp) {
    const T k = inv_two_pi<T>();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const T sg = __ldg(s + i);
        T gsum = (first ? T(0) : gs[i]) + __ldg(gsk + i);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const long long j = c * n + i;
            const T g = __ldg(gek + j);
            ge[j] = (first ? T(0) : ge[j]) + g;
            if (has_prev) {
                const T f = __ldg(Fp + j), ac = __ldg(a + j), gk = g * k;
                gsum += gk * ac * f;
                ga[j] = (first ? T(0) : ga[j]) + gk * sg * f;
                gFp[j] = gk * ac * sg;
            } else if (first) {
                ga[j] = T(0);
            }
        }
        gs[i] = gsum;
    }
}

int stride_grid(long long n, int threads) {
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long blocks = (n + threads - 1) / threads;
    const long long cap = (long long)sms * 8;
    return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

double bytes_bounce_source(const Plan &pl) {
    const double img = (double)pl.W * pl.H, esz = pl.prec == P_FP64 ? 8.0 : 4.0;
    return img * (4 * pl.C + 1) * esz;
}

double bytes_bounce_adj(const Plan &pl, bool first, bool has_prev) {
    const double img = (double)pl.W * pl.H, esz = pl.prec == P_FP64 ? 8.0 : 4.0;
    // ge_k, gs_k, s read; ge, gs written (and read unless first); with a
    // previous bounce also F_{k-1}, albedo read, ga written (read unless
    // first), dL/dF_{k-1} written
    double planes = pl.C + 1 + 1 + (pl.C + 1) * (first ? 1 : 2);
    if (has_prev) planes += 2 * pl.C + pl.C * (first ? 1 : 2) + pl.C;
    else if (first) planes += pl.C;
    return img * planes * esz;
}

cudaError_t launch_bounce_source(const Plan &pl, const void *e, const void *s, const void *a, const void *F,
                                 void *eo, cudaStream_t st, int *launches, Recorder *rec, bool per_channel_sigma) {
    const long long n = (long long)pl.W * pl.H, ss = per_channel_sigma ? n : 0;
    rec->begin(K_BOUNCE, 0, bytes_bounce_source(pl));
    const bool v4 = pl.prec != P_FP64 && n % 4 == 0;
    const int grid = stride_grid(v4 ? n / 4 : n, 256);
    switch (pl.C) {
#define HRC_BOUNCE_CASE(CC)                                                                                       \
    case CC:                                                                                                      \
        if (pl.prec == P_FP64)                                                                                    \
            k_bounce_source<double, CC><<<grid, 256, 0, st>>>(n, ss, (const double *)e, (const double *)s,        \
                                                              (const double *)a, (const double *)F, (double *)eo); \
        else if (v4)                                                                                              \
            k_bounce_source4<CC><<<grid, 256, 0, st>>>(n / 4, ss / 4, (const float4 *)e, (const float4 *)s,      \
                                                       (const float4 *)a, (const float4 *)F, (float4 *)eo);       \
        else                                                                                                      \
            k_bounce_source<float, CC><<<grid, 256, 0, st>>>(n, ss, (const float *)e, (const float *)s,           \
                                                             (const float *)a, (const float *)F, (float *)eo);    \
        break;
        HRC_BOUNCE_CASE(1) HRC_BOUNCE_CASE(2) HRC_BOUNCE_CASE(3) HRC_BOUNCE_CASE(4)
#undef HRC_BOUNCE_CASE
    default: return cudaErrorInvalidValue;
    }
    rec->end();
    ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_bounce_adj(const Plan &pl, bool first, bool has_prev, const void *gek, const void *gsk,
                              const void *Fp, const void *a, const void *s, void *ge, void *gs, void *ga, void *gFp,
                              cudaStream_t st, int *launches, Recorder *rec) {
    const long long n = (long long)pl.W * pl.H;
    rec->begin(K_ADJ_BOUNCE, 0, bytes_bounce_adj(pl, first, has_prev));
    const int grid = stride_grid(n, 256);
    const int f = first ? 1 : 0, h = has_prev ? 1 : 0;
    switch (pl.C) {
#define HRC_BOUNCE_CASE(CC)                                                                                       \
    case CC:                                                                                                      \
        if (pl.prec == P_FP64)                                                                                    \
            k_bounce_adj<double, CC><<<grid, 256, 0, st>>>(n, f, h, (const double *)gek, (const double *)gsk,     \
                                                           (const double *)Fp, (const double *)a,                 \
                                                           (const double *)s, (double *)ge, (double *)gs,         \
                                                           (double *)ga, (double *)gFp);                          \
        else                                                                                                      \
            k_bounce_adj<float, CC><<<grid, 256, 0, st>>>(n, f, h, (const float *)gek, (const float *)gsk,        \
                                                          (const float *)Fp, (const float *)a, (const float *)s,  \
                                                          (float *)ge, (float *)gs, (float *)ga, (float *)gFp);   \
        break;
        HRC_BOUNCE_CASE(1) HRC_BOUNCE_CASE(2) HRC_BOUNCE_CASE(3) HRC_BOUNCE_CASE(4)
#undef HRC_BOUNCE_CASE
    default: return cudaErrorInvalidValue;
    }
    rec->end();
    ++*launches;
    return cudaGetLastError();
}

}  // namespace hrc
