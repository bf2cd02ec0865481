// kernels_util.cu -- introspection kernels (dense fp32 export of T_n / R_n).
#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

// T_n of frame q -> dst[x][k][v][C+1] (C radiances, then linear T).  Entries
// that no fluence depends on (t_live) are never computed and are exported as
// NaN.
template <int P, int C>
__global__ void k_export_T(Plan pl, int q, int n, float *__restrict__ dst) {
    const QuadGeom &g = pl.q[q];
    const int K = (1 << n) + 1;
    const long long total = (long long)g.Un[n] * K * g.V;
    TLevel<P, C> T(pl, q, n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % g.V);
        const long long r = i / g.V;
        const int k = (int)(r % K), x = (int)(r / K);
        float *o = dst + i * (C + 1);
        if (!t_live(n, x, k)) {
#pragma unroll
            for (int c = 0; c <= C; ++c) o[c] = __int_as_float(0x7fc00000);
            continue;
        }
        Iv<P, C> iv = T.load(x, k, v);
#pragma unroll
        for (int c = 0; c < C; ++c) o[c] = (float)iv.L[c];
        o[C] = (float)iv.trans();
    }
}

// R_n of frame q -> dst[x][i][v][C]; column 0 exported as NaN.
template <int P, int C>
__global__ void k_export_R(Plan pl, int q, int n, float *__restrict__ dst) {
    const QuadGeom &g = pl.q[q];
    const int I = 1 << n;
    const long long total = (long long)g.Un[n] * I * g.V;
    RLevel<P, C> R(pl, q, n);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i % g.V);
        const long long r = i / g.V;
        const int ip = (int)(r % I), x = (int)(r / I);
#pragma unroll
        for (int c = 0; c < C; ++c) dst[i * C + c] = x == 0 ? __int_as_float(0x7fc00000) : (float)R.load(x, ip, c, v);
    }
}

template <int P, int C>
static cudaError_t copy_impl(const Plan &pl, int q, int which, int n, float *dst, cudaStream_t st) {
    if (which == 0) k_export_T<P, C><<<1024, 256, 0, st>>>(pl, q, n, dst);
    else k_export_R<P, C><<<1024, 256, 0, st>>>(pl, q, n, dst);
    return cudaGetLastError();
}

template <int P>
static cudaError_t copy_prec(const Plan &pl, int q, int which, int n, float *dst, cudaStream_t st) {
    switch (pl.C) {
    case 1: return copy_impl<P, 1>(pl, q, which, n, dst, st);
    case 2: return copy_impl<P, 2>(pl, q, which, n, dst, st);
    case 3: return copy_impl<P, 3>(pl, q, which, n, dst, st);
    default: return copy_impl<P, 4>(pl, q, which, n, dst, st);
    }
}

cudaError_t launch_copy_level(const Plan &pl, int q, int which, int n, float *dst, cudaStream_t st) {
    switch (pl.prec) {
    case P_FP32: return copy_prec<P_FP32>(pl, q, which, n, dst, st);
    case P_FP16: return copy_prec<P_FP16>(pl, q, which, n, dst, st);
    case P_BF16: return copy_prec<P_BF16>(pl, q, which, n, dst, st);
    default: return copy_prec<P_FP64>(pl, q, which, n, dst, st);
    }
}

}  // namespace hrc
