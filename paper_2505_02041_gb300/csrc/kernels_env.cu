// kernels_env.cu -- environment map (footnote 1 of Sec. 4.2: with no
// occluders outside the grid, R_N is the map looked up along v_N(i)), or
// the top-level radiance R_N itself supplied by the caller.
//
// The map env[c][m] holds the radiance seen along the image-space look
// angle theta_m = 2 pi (m + 1/2) / M, theta measured from +x towards +y
// (down the rows), linearly interpolated between samples and periodic.
// Frame q looks along +u; its direction (du, dv) is the image direction
// (du, dv), (-du, dv), (dv, du) or (dv, -du) for q = 0 .. 3 (the inverse of
// the quadrant maps).
//
// Table: for every frame q and level n <= N_q, cone j gets
//     sum over its level-N descendants m of A_N(m) env(direction of v_N(m)),
// the value of R_N(., m) = A_N(m) env(...) summed the way Eqs. 14 / 15 sum
// two cones when every interval is vacuum <0, 1>: an R_n lookup outside the
// grid sees exactly this (nothing outside absorbs or emits, and a path that
// has left the grid never re-enters).  Computed once per map, in double,
// with a float copy for the fp32 / fp16 / bf16 kernels: one thread per
// level-N cone evaluates the map, then one thread per (q, 2^n + j, c) sums
// its descendants in increasing order.
#include <cuda_runtime.h>

#include "hrc_internal.cuh"
#include "launch.h"

namespace hrc {

namespace {

__device__ double env_at(const float *__restrict__ env, int M, int c, double dx, double dy) {
    const double two_pi = 6.283185307179586476925286766559;
    double th = atan2(dy, dx);
    if (th < 0.0) th += two_pi;
    const double t = th * M / two_pi - 0.5;
    const double m0 = floor(t), f = t - m0;
    long long i0 = (long long)m0 % M;
    if (i0 < 0) i0 += M;
    const long long i1 = i0 + 1 == M ? 0 : i0 + 1;
    return (1.0 - f) * (double)env[(long long)c * M + i0] + f * (double)env[(long long)c * M + i1];
}

// Level-N entries: A_N(m) env(direction of v_N(m)), one thread each.
__global__ void __launch_bounds__(128) k_env_leaves(Plan pl, const float *__restrict__ env, int M, int C, int S,
                                                    double *__restrict__ td) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int q = (int)(idx / ((long long)S * C));
    if (q >= 4) return;
    const int rem = (int)(idx - (long long)q * S * C);
    const int m = rem / C, c = rem - m * C;
    const int N = pl.q[q].N;
    if (m >= (1 << N)) return;
    const double sN = (double)(1 << N);
    const double du = sN, dv = 2.0 * m + 1.0 - sN;        // v_N(m + 1/2)
    const double dx = q == 0 ? du : (q == 1 ? -du : dv);
    const double dy = q == 0 ? dv : (q == 1 ? dv : (q == 2 ? du : -du));
    const double a = atan((2.0 * (m + 1) - sN) / sN) - atan((2.0 * m - sN) / sN);   // Eq. 13
    td[(long long)q * S * C + ((long long)(1 << N) + m) * C + c] = a * env_at(env, M, c, dx, dy);
}

// Level-N entries supplied by the caller (footnote 1 of Sec. 4.2: R_N from
// another method): top[(q K + m) C + c] for cone m < 2^N of frame q.
__global__ void __launch_bounds__(128) k_env_top(Plan pl, const float *__restrict__ top, int K, int C, int S,
                                                 double *__restrict__ td) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int q = (int)(idx / ((long long)S * C));
    if (q >= 4) return;
    const int rem = (int)(idx - (long long)q * S * C);
    const int m = rem / C, c = rem - m * C;
    const int N = pl.q[q].N;
    if (m >= (1 << N)) return;
    td[(long long)q * S * C + ((long long)(1 << N) + m) * C + c] = (double)top[((long long)q * K + m) * C + c];
}

// Every entry: the sum of its level-N descendants (in increasing order),
// read from the leaves; the float copy beside it.
__global__ void __launch_bounds__(128) k_env_table(Plan pl, int C, int S, double *__restrict__ td,
                                                   float *__restrict__ tf) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long total = 4LL * S * C;
    if (idx >= total) return;
    const int q = (int)(idx / ((long long)S * C));
    const int rem = (int)(idx - (long long)q * S * C);
    const int lv = rem / C, c = rem - lv * C;
    const int N = pl.q[q].N;
    const int n = lv > 0 ? 31 - __clz(lv) : -1;
    double acc = 0.0;
    if (n >= 0 && n <= N) {
        const int j = lv - (1 << n);
        const double *leaf = td + (long long)q * S * C + (long long)(1 << N) * C + c;
        for (int m = j << (N - n); m < (j + 1) << (N - n); ++m) acc += leaf[(long long)m * C];
    }
    if (n != N) td[idx] = acc;   // (level N keeps its leaves; unused entries become 0)
    tf[idx] = (float)acc;
}

}  // namespace

long long env_table_stride(const Plan &pl) { return (2LL << plan_nmax(pl)) * pl.C; }

size_t env_table_bytes(const Plan &pl) {
    return (size_t)(4 * env_table_stride(pl)) * (sizeof(double) + sizeof(float));
}

cudaError_t launch_env_table(const Plan &pl, const float *env, int M, void *table, cudaStream_t st) {
    const long long stride = env_table_stride(pl);
    const long long total = 4 * stride;
    double *td = reinterpret_cast<double *>(table);
    float *tf = reinterpret_cast<float *>(td + total);
    const int S = (int)(stride / pl.C);
    const unsigned grid = (unsigned)((total + 127) / 128);
    k_env_leaves<<<grid, 128, 0, st>>>(pl, env, M, pl.C, S, td);
    k_env_table<<<grid, 128, 0, st>>>(pl, pl.C, S, td, tf);
    return cudaGetLastError();
}

cudaError_t launch_env_top(const Plan &pl, const float *top, int K, void *table, cudaStream_t st) {
    const long long stride = env_table_stride(pl);
    const long long total = 4 * stride;
    double *td = reinterpret_cast<double *>(table);
    float *tf = reinterpret_cast<float *>(td + total);
    const int S = (int)(stride / pl.C);
    const unsigned grid = (unsigned)((total + 127) / 128);
    k_env_top<<<grid, 128, 0, st>>>(pl, top, K, pl.C, S, td);
    k_env_table<<<grid, 128, 0, st>>>(pl, pl.C, S, td, tf);
    return cudaGetLastError();
}

}  // namespace hrc
