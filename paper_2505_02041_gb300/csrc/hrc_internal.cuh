// hrc_internal.cuh -- device-side building blocks shared by the HRC kernels.
//
// Frame geometry (Algorithm 1, procedure Lighting).  Instead of rotating the
// world four times, each quadrant q is computed in its own frame (u, v), the
// gathering direction being +u; the per-quadrant recursion is symmetric under
// v -> V-1-v (Eqs. 13-20), so reflections give the same result as rotations:
//   q0: (u,v) = (x, y)     q1: (u,v) = (W-1-x, y)
//   q2: (u,v) = (y, x)     q3: (u,v) = (H-1-y, x)
//
// Probe layout (Sec. 4): level n has probes p = (x 2^n, v) for x < U_n =
// ceil(U / 2^n); direction k in [0, 2^n] has offset v_n(k) = (2^n, 2k - 2^n);
// cone i = i' + 1/2 spans directions i' .. i'+1.
//
// HBM layout (per quadrant, per level; v is contiguous, rows padded to Vs):
//   T_n: row group (x, k) holds C radiance rows of SL then one transmittance
//        row of ST (T, or tau = -ln T in the log-T precisions):
//        byte offset of component c of (x, k, v) =
//            Toff + (x*K_n + k) * G_n + c * Vs * sizeof(SL) + v * sizeof(elem),
//        G_n = Vs * (C * sizeof(SL) + sizeof(ST)), K_n = 2^n + 1.
//   R_n: planar per channel: element (x, i, c, v) at ((x*2^n + i)*C + c)*Vs + v.
// Every Eq. 18/19 and Eq. 14/15 access is then a contiguous run along v,
// shifted by an even offset for n >= 1: coalesced, sector-aligned loads.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define HRC_MAXL 15
#define HRC_MAXRAY 10      // ray shapes of levels 0..2: 2 + 3 + 5
#define HRC_MAXPIECE 48    // their pixel pieces: 4 + 9 + 29 = 42

namespace hrc {

struct QuadGeom {
    int U, V, Vs, N;                 // frame extent, padded row stride, cascade count
    int Un[HRC_MAXL + 1];            // probe columns per level
    long long Toff[HRC_MAXL + 1];    // byte offset of T_n in the arena
    long long Roff[HRC_MAXL + 1];    // byte offset of R_n (n < N)
    long long gToff[HRC_MAXL + 1];   // adjoint buffers: dLoss/dT_n (C radiances + linear T) ...
    long long gRoff[HRC_MAXL + 1];   // ... and dLoss/dR_n, in the arithmetic type
};

struct Plan {
    int W, H, C, prec;
    int sched;                       // 0: each launch covers all four frames; 1: frame by frame
    int mgroups;                     // merge up: 1 = a pair of v per thread, 2 = two pairs, 4 = four consecutive v
    int mthreads;                    // merge kernels: threads per block for paired-v bodies
    int vmajor;                      // merge kernels: 1 = v-blocks of a row are adjacent in launch order
    int mdown;                       // merge down: 0 = per-thread loads, 1 = rows staged by bulk copies,
                                     // 2 = every level in one persistent launch
    long long bulk_limit_ns;         // bound of a bulk-copy barrier wait
    int bulk_extra_tx;               // test hook: bytes expected but never copied (0 in use)
    long long arcs_off;              // byte offset: float A[2^n + j] for level n (n >= 1)
    long long arcs_off_d;            // same table in double
    char *arena;
    // environment map (footnote 1 of Sec. 4.2): value of cone j at level n of
    // frame q at [q * env_stride + (2^n + j) * C + c] (fp32 / fp64 copies);
    // null without a map (out-of-grid R lookups are then 0)
    const float *envf;
    const double *envd;
    long long env_stride;
    // control block of the persistent merge-down launch (kernels_persist.cu):
    // ticket counter, status word and per-column completion counters; null
    // where the context has none (the persistent launch is then not used)
    char *pctl;
    long long pctl_bytes;
    // status word of this plan's kernels: 0, or a code set by a bounded wait
    // that gave up (kWaitTimeout; kWaitLost when a copy may still have been
    // in flight as the block left); read and cleared by the host after a
    // synchronisation.  Never null for a plan that is launched.
    int *status;
    QuadGeom q[4];
};

// Codes of the status word (Plan::status).  A wait on a copy barrier that
// gives up after its bound is kWaitTimeout; the block then waits once more,
// with the longer drain bound, for the copies already issued to land, and
// records kWaitLost if even that runs out (shared memory of a later block on
// the same SM could then still be written by them).
constexpr int kWaitTimeout = 5;
constexpr int kWaitLost = 7;
__host__ __device__ inline long long drain_limit_ns(long long limit_ns) { return 4 * limit_ns + 100000000LL; }

// Pieces of the directly traced rays (levels 0..2) from a pixel centre:
// pixel offset (du, dv) and length.  Ray r of level n, direction k:
// r = 0,1 (n=0), 2..4 (n=1), 5..9 (n=2).
struct RayPiece { int8_t du, dv; int8_t pad0, pad1; float len; };
struct RayTable {
    int start[HRC_MAXRAY + 1];
    RayPiece p[HRC_MAXPIECE];
    double lenD[HRC_MAXPIECE];
};

// Row-to-quadrant lookup for flattened (q, row) grids: the first global row
// of each quadrant frame; start[4] = total rows.
struct RowSplit {
    long long start[5];
};

__host__ __device__ inline int ray_id(int n, int k) { return n == 0 ? k : (n == 1 ? 2 + k : 5 + k); }

// Entries T_n(x, k) that some fluence depends on.  Column 0 of every level
// is dead (the fluence sum reads R_0 at u + 1).  T_0 is read only at odd
// columns (Eq. 14 at level 0; the even columns of level 0 take T_1), and T_1
// at even columns only in its even directions (Eqs. 15-17 at level 0), as
// the merge up starts from T_2.  Dead entries are neither traced, merged,
// nor differentiated.
__host__ __device__ inline bool t_live(int n, int x, int k) {
    if (x <= 0) return false;
    if (n == 0) return (x & 1) != 0;
    if (n == 1) return (x & 1) != 0 || (k & 1) == 0;
    return true;
}

// Number of live (x, k) rows of T_n over the columns 0 .. Un-1.
__host__ __device__ inline long long t_live_rows(int n, int Un) {
    const long long odd = Un / 2, even = Un - 1 - odd;     // live columns 1 .. Un-1
    if (n == 0) return odd * 2;
    if (n == 1) return odd * 3 + even * 2;
    return (long long)(Un - 1) * ((1 << n) + 1);
}

// frame (u, v) of quadrant q -> image pixel (x, y)
__host__ __device__ inline void frame_to_image(int q, int W, int H, int u, int v, int &x, int &y) {
    x = q == 0 ? u : (q == 1 ? W - 1 - u : v);
    y = q < 2 ? v : (q == 2 ? u : H - 1 - u);
}
// image pixel (x, y) -> frame (u, v) of quadrant q
__host__ __device__ inline void image_to_frame(int q, int W, int H, int x, int y, int &u, int &v) {
    u = q == 0 ? x : (q == 1 ? W - 1 - x : (q == 2 ? y : H - 1 - y));
    v = q < 2 ? y : x;
}

// ---------------------------------------------------------------------------
// Precision traits.  SL: radiance / fluence storage, ST: transmittance
// storage, A: arithmetic type, LOG: ST holds tau = -ln T.
// ---------------------------------------------------------------------------
enum { P_FP32 = 0, P_FP16 = 1, P_BF16 = 2, P_FP64 = 3 };

template <int P> struct Prec;
template <> struct Prec<P_FP32> { using SL = float;          using ST = float;  using A = float;  static constexpr bool LOG = false; };
template <> struct Prec<P_FP16> { using SL = __half;         using ST = float;  using A = float;  static constexpr bool LOG = true;  };
template <> struct Prec<P_BF16> { using SL = __nv_bfloat16;  using ST = float;  using A = float;  static constexpr bool LOG = true;  };
template <> struct Prec<P_FP64> { using SL = double;         using ST = double; using A = double; static constexpr bool LOG = false; };

// Shared-memory tiles of the two trace kernels: a pixel's {t, w} of one ray
// class as one 2-vector, and {e0, e1, e2, sigma} as one float4 in fp32 with
// C <= 3 (one shared load each); otherwise e and sigma as separate planes.
template <class A> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };
template <class A, int C> struct PackES {
    static constexpr bool packed = sizeof(A) == 4 && C <= 3;
};

__device__ __forceinline__ float to_acc(float x) { return x; }
__device__ __forceinline__ double to_acc(double x) { return x; }
__device__ __forceinline__ float to_acc(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_acc(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class S> __device__ __forceinline__ S from_acc(float x);
template <> __device__ __forceinline__ float from_acc<float>(float x) { return x; }
template <> __device__ __forceinline__ __half from_acc<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <class S> __device__ __forceinline__ S from_acc(double x);
template <> __device__ __forceinline__ double from_acc<double>(double x) { return x; }

__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float fexpm1(float x) { return expm1f(x); }
__device__ __forceinline__ double fexpm1(double x) { return expm1(x); }
__device__ __forceinline__ float flog(float x) { return __logf(x); }
__device__ __forceinline__ double flog(double x) { return log(x); }

// ---------------------------------------------------------------------------
// An interval <L, T> in registers (Eq. 9).  For LOG precisions `t` holds
// tau = -ln T so that Merge adds and long opaque paths never underflow.
// ---------------------------------------------------------------------------
template <int P, int C> struct Iv {
    using A = typename Prec<P>::A;
    A L[C];
    A t;
    __device__ __forceinline__ static Iv vacuum() {
        Iv r;
#pragma unroll
        for (int c = 0; c < C; ++c) r.L[c] = A(0);
        r.t = Prec<P>::LOG ? A(0) : A(1);
        return r;
    }
    __device__ __forceinline__ A trans() const { return Prec<P>::LOG ? fexp(-t) : t; }
};

// A product the compiler may not contract into a later addition: the blend
// (Eq. 20) adds two merged transmittances, and an FMA formed there in one
// kernel and not in another would round the same entry differently.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Merge (Eq. 7): <r_n + t_n r_f, t_n t_f>
template <int P, int C>
__device__ __forceinline__ Iv<P, C> merge(const Iv<P, C> &n, const Iv<P, C> &f) {
    Iv<P, C> r;
    typename Prec<P>::A tn = n.trans();
#pragma unroll
    for (int c = 0; c < C; ++c) r.L[c] = fma(tn, f.L[c], n.L[c]);
    r.t = Prec<P>::LOG ? n.t + f.t : mul_rn(n.t, f.t);
    return r;
}

// Eq. 20: the average of two intervals (radiance and transmittance).
template <int P, int C>
__device__ __forceinline__ Iv<P, C> blend(const Iv<P, C> &a, const Iv<P, C> &b) {
    using A = typename Prec<P>::A;
    Iv<P, C> r;
#pragma unroll
    for (int c = 0; c < C; ++c) r.L[c] = A(0.5) * (a.L[c] + b.L[c]);
    if (Prec<P>::LOG) {
        // -ln((e^-a + e^-b)/2) = min + ln 2 - ln(1 + e^-|a-b|); the argument of
        // the last log is in [1, 2], where the fast log is accurate to ~1e-7
        A lo = fmin(a.t, b.t), d = fabs(a.t - b.t);
        r.t = lo + A(0.69314718055994530942) - flog(A(1) + fexp(-d));
    } else {
        r.t = A(0.5) * (a.t + b.t);
    }
    return r;
}

// 2-wide loads / stores of two consecutive v (the first v even, so every
// pair is 2-element aligned).
__device__ __forceinline__ void ld2(const float *p, float &x, float &y) {
    const float2 t = *reinterpret_cast<const float2 *>(p); x = t.x; y = t.y;
}
__device__ __forceinline__ void ld2(const double *p, double &x, double &y) {
    const double2 t = *reinterpret_cast<const double2 *>(p); x = t.x; y = t.y;
}
__device__ __forceinline__ void ld2(const __half *p, float &x, float &y) {
    const __half2 t = *reinterpret_cast<const __half2 *>(p); x = __low2float(t); y = __high2float(t);
}
__device__ __forceinline__ void ld2(const __nv_bfloat16 *p, float &x, float &y) {
    const __nv_bfloat162 t = *reinterpret_cast<const __nv_bfloat162 *>(p); x = __low2float(t); y = __high2float(t);
}
__device__ __forceinline__ void st2(float *p, float x, float y) { *reinterpret_cast<float2 *>(p) = make_float2(x, y); }
__device__ __forceinline__ void st2(double *p, double x, double y) { *reinterpret_cast<double2 *>(p) = make_double2(x, y); }
__device__ __forceinline__ void st2(__half *p, float x, float y) { *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(x, y); }
__device__ __forceinline__ void st2(__nv_bfloat16 *p, float x, float y) {
    *reinterpret_cast<__nv_bfloat162 *>(p) = __floats2bfloat162_rn(x, y);
}

// 4-wide loads / stores of four consecutive v (the first a multiple of 4,
// so every quadruple is 4-element aligned).
__device__ __forceinline__ void ld4(const float *p, float (&r)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p); r[0] = t.x; r[1] = t.y; r[2] = t.z; r[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&r)[4]) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
}
__device__ __forceinline__ void ld4(const __half *p, float (&r)[4]) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const __half2 a = *reinterpret_cast<const __half2 *>(&u.x), b = *reinterpret_cast<const __half2 *>(&u.y);
    r[0] = __low2float(a); r[1] = __high2float(a); r[2] = __low2float(b); r[3] = __high2float(b);
}
__device__ __forceinline__ void ld4(const __nv_bfloat16 *p, float (&r)[4]) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x),
                         b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
    r[0] = __low2float(a); r[1] = __high2float(a); r[2] = __low2float(b); r[3] = __high2float(b);
}
__device__ __forceinline__ void st4(float *p, const float (&r)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
__device__ __forceinline__ void st4(double *p, const double (&r)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(r[0], r[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(r[2], r[3]);
}
__device__ __forceinline__ void st4(__half *p, const float (&r)[4]) {
    const __half2 a = __floats2half2_rn(r[0], r[1]), b = __floats2half2_rn(r[2], r[3]);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned *>(&a);
    u.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}
__device__ __forceinline__ void st4(__nv_bfloat16 *p, const float (&r)[4]) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(r[0], r[1]), b = __floats2bfloat162_rn(r[2], r[3]);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned *>(&a);
    u.y = *reinterpret_cast<const unsigned *>(&b);
    *reinterpret_cast<uint2 *>(p) = u;
}

// ---------------------------------------------------------------------------
// L2 residency.  The merge down reads each T row from HBM (the merge up
// wrote it long before), while R_{n+1} -- written by the previous launch --
// is read three times (near at even x, far from both neighbours).  Loading
// the T rows with the evict-first policy lets them stream through the L2
// without displacing the R levels.  Used where it measured faster: the
// bulk-staged merge down and the level-0 merge down inside the fluence sum
// (the per-thread merge down at 2048^2 was slower with it: a T row is read
// by two neighbouring blocks, and the second read then misses).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float ld1_ef(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld1_ef(const double *p, uint64_t) { return *p; }
template <class H> __device__ __forceinline__ float ld1_ef_16(const H *p, uint64_t pol) {
    unsigned short u;
    asm volatile("ld.global.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(u) : "l"(p), "l"(pol));
    return to_acc(*reinterpret_cast<const H *>(&u));
}
__device__ __forceinline__ float ld1_ef(const __half *p, uint64_t pol) { return ld1_ef_16(p, pol); }
__device__ __forceinline__ float ld1_ef(const __nv_bfloat16 *p, uint64_t pol) { return ld1_ef_16(p, pol); }
// entries p[0], p[1] (p 2-element aligned) with an L2 policy
__device__ __forceinline__ void ld2_ef(const float *p, uint64_t pol, float &x, float &y) {
    asm volatile("ld.global.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(x), "=f"(y) : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld2_ef(const double *p, uint64_t, double &x, double &y) { ld2(p, x, y); }
template <class H2> __device__ __forceinline__ void ld2_ef_16(const void *p, uint64_t pol, float &x, float &y) {
    unsigned u;
    asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(u) : "l"(p), "l"(pol));
    const H2 t = *reinterpret_cast<const H2 *>(&u);
    x = __low2float(t);
    y = __high2float(t);
}
__device__ __forceinline__ void ld2_ef(const __half *p, uint64_t pol, float &x, float &y) {
    ld2_ef_16<__half2>(p, pol, x, y);
}
__device__ __forceinline__ void ld2_ef(const __nv_bfloat16 *p, uint64_t pol, float &x, float &y) {
    ld2_ef_16<__nv_bfloat162>(p, pol, x, y);
}
// entries p[0 .. 3] (p 4-element aligned) with an L2 policy
__device__ __forceinline__ void ld4_ef(const float *p, uint64_t pol, float (&r)[4]) {
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(r[0]), "=f"(r[1]), "=f"(r[2]), "=f"(r[3])
                 : "l"(p), "l"(pol));
}
__device__ __forceinline__ void ld4_ef(const double *p, uint64_t, double (&r)[4]) { ld4(p, r); }
template <class H2> __device__ __forceinline__ void ld4_ef_16(const void *p, uint64_t pol, float (&r)[4]) {
    unsigned u0, u1;
    asm volatile("ld.global.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;" : "=r"(u0), "=r"(u1) : "l"(p), "l"(pol));
    const H2 a = *reinterpret_cast<const H2 *>(&u0), b = *reinterpret_cast<const H2 *>(&u1);
    r[0] = __low2float(a);
    r[1] = __high2float(a);
    r[2] = __low2float(b);
    r[3] = __high2float(b);
}
__device__ __forceinline__ void ld4_ef(const __half *p, uint64_t pol, float (&r)[4]) { ld4_ef_16<__half2>(p, pol, r); }
__device__ __forceinline__ void ld4_ef(const __nv_bfloat16 *p, uint64_t pol, float (&r)[4]) {
    ld4_ef_16<__nv_bfloat162>(p, pol, r);
}

// ---------------------------------------------------------------------------
// Level addressing
// ---------------------------------------------------------------------------
template <int P, int C> struct TLevel {
    using SL = typename Prec<P>::SL;
    using ST = typename Prec<P>::ST;
    char *base;
    int K, Vs;
    long long G;   // bytes per (x, k) row group
    __device__ __forceinline__ TLevel(const Plan &pl, int q, int n) {
        base = pl.arena + pl.q[q].Toff[n];
        K = (1 << n) + 1;
        Vs = pl.q[q].Vs;
        G = (long long)Vs * (C * (long long)sizeof(SL) + (long long)sizeof(ST));
    }
    __device__ __forceinline__ char *row(int x, int k) const { return base + ((long long)x * K + k) * G; }
    __device__ __forceinline__ Iv<P, C> load(int x, int k, int v) const {
        const char *g = row(x, k);
        Iv<P, C> r;
#pragma unroll
        for (int c = 0; c < C; ++c) r.L[c] = to_acc(reinterpret_cast<const SL *>(g)[(long long)c * Vs + v]);
        r.t = to_acc(reinterpret_cast<const ST *>(g + (long long)C * Vs * sizeof(SL))[v]);
        return r;
    }
    __device__ __forceinline__ void store(int x, int k, int v, const Iv<P, C> &r) const {
        char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) reinterpret_cast<SL *>(g)[(long long)c * Vs + v] = from_acc<SL>(r.L[c]);
        reinterpret_cast<ST *>(g + (long long)C * Vs * sizeof(SL))[v] = from_acc<ST>(r.t);
    }
    // entries v and v+1 (v even)
    __device__ __forceinline__ void load2(int x, int k, int v, Iv<P, C> &a, Iv<P, C> &b) const {
        const char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) ld2(reinterpret_cast<const SL *>(g) + (long long)c * Vs + v, a.L[c], b.L[c]);
        ld2(reinterpret_cast<const ST *>(g + (long long)C * Vs * sizeof(SL)) + v, a.t, b.t);
    }
    // entries v, v+1 with vacuum outside [0, V) (v even, so v < 0 means both out)
    __device__ __forceinline__ void load2_masked(int x, int k, int v, int V, Iv<P, C> &a, Iv<P, C> &b) const {
        if (v >= 0 && v < V) {
            load2(x, k, v, a, b);
            if (v + 1 >= V) b = Iv<P, C>::vacuum();
        } else {
            a = Iv<P, C>::vacuum();
            b = a;
        }
    }
    __device__ __forceinline__ void store2(int x, int k, int v, const Iv<P, C> &a, const Iv<P, C> &b) const {
        char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) st2(reinterpret_cast<SL *>(g) + (long long)c * Vs + v, a.L[c], b.L[c]);
        st2(reinterpret_cast<ST *>(g + (long long)C * Vs * sizeof(SL)) + v, a.t, b.t);
    }    // linear transmittance of entries v and v+1 (v even)
    __device__ __forceinline__ void load_t2(int x, int k, int v, typename Prec<P>::A &a,
                                            typename Prec<P>::A &b) const {
        ld2(reinterpret_cast<const ST *>(row(x, k) + (long long)C * Vs * sizeof(SL)) + v, a, b);
        if (Prec<P>::LOG) {
            a = fexp(-a);
            b = fexp(-b);
        }
    }
    __device__ __forceinline__ void store4(int x, int k, int v, const Iv<P, C> (&r)[4]) const {
        using A = typename Prec<P>::A;
        char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const A t[4] = {r[0].L[c], r[1].L[c], r[2].L[c], r[3].L[c]};
            st4(reinterpret_cast<SL *>(g) + (long long)c * Vs + v, t);
        }
        const A t[4] = {r[0].t, r[1].t, r[2].t, r[3].t};
        st4(reinterpret_cast<ST *>(g + (long long)C * Vs * sizeof(SL)) + v, t);
    }
    // entries v .. v+3 with vacuum outside [0, V) (v even): one 4-wide load
    // when v is a multiple of 4 and the run is inside, else two pairs
    __device__ __forceinline__ void load4_masked(int x, int k, int v, int V, Iv<P, C> (&r)[4]) const {
        if ((v & 3) == 0 && v >= 0 && v + 3 < V) {
            load4(x, k, v, r);
            return;
        }
        load2_masked(x, k, v, V, r[0], r[1]);
        load2_masked(x, k, v + 2, V, r[2], r[3]);
    }
    // entry v, loaded with an L2 policy
    __device__ __forceinline__ Iv<P, C> load_ef(int x, int k, int v, uint64_t pol) const {
        const char *g = row(x, k);
        Iv<P, C> r;
#pragma unroll
        for (int c = 0; c < C; ++c) r.L[c] = ld1_ef(reinterpret_cast<const SL *>(g) + (long long)c * Vs + v, pol);
        r.t = ld1_ef(reinterpret_cast<const ST *>(g + (long long)C * Vs * sizeof(SL)) + v, pol);
        return r;
    }
    // entries v and v+1 (v even), loaded with an L2 policy
    // entries v .. v+3 (v a multiple of 4; v + 3 < Vs), loaded with an L2 policy
    __device__ __forceinline__ void load4_ef(int x, int k, int v, uint64_t pol, Iv<P, C> (&r)[4]) const {
        using A = typename Prec<P>::A;
        const char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            A t[4];
            ld4_ef(reinterpret_cast<const SL *>(g) + (long long)c * Vs + v, pol, t);
#pragma unroll
            for (int l = 0; l < 4; ++l) r[l].L[c] = t[l];
        }
        A t[4];
        ld4_ef(reinterpret_cast<const ST *>(g + (long long)C * Vs * sizeof(SL)) + v, pol, t);
#pragma unroll
        for (int l = 0; l < 4; ++l) r[l].t = t[l];
    }
    __device__ __forceinline__ void load2_ef(int x, int k, int v, uint64_t pol, Iv<P, C> &a, Iv<P, C> &b) const {
        const char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) ld2_ef(reinterpret_cast<const SL *>(g) + (long long)c * Vs + v, pol, a.L[c], b.L[c]);
        ld2_ef(reinterpret_cast<const ST *>(g + (long long)C * Vs * sizeof(SL)) + v, pol, a.t, b.t);
    }
    // entries v .. v+3 (v a multiple of 4; v + 3 < Vs)
    __device__ __forceinline__ void load4(int x, int k, int v, Iv<P, C> (&r)[4]) const {
        using A = typename Prec<P>::A;
        const char *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            A t[4];
            ld4(reinterpret_cast<const SL *>(g) + (long long)c * Vs + v, t);
#pragma unroll
            for (int l = 0; l < 4; ++l) r[l].L[c] = t[l];
        }
        A t[4];
        ld4(reinterpret_cast<const ST *>(g + (long long)C * Vs * sizeof(SL)) + v, t);
#pragma unroll
        for (int l = 0; l < 4; ++l) r[l].t = t[l];
    }
};

// Value of an R_n lookup outside the stored ranges (and of any R_N lookup):
// the environment's value of cone j (the sum of its level-N descendants,
// i.e. the recursion continued outside the grid through vacuum) in kernels
// compiled for a map (ENV), else 0 -- a compile-time choice, so that the
// map-free kernels carry none of its code or registers.
template <int P, int C, bool ENV>
__device__ __forceinline__ typename Prec<P>::A renv(const Plan &pl, int q, int n, int j, int c) {
    using A = typename Prec<P>::A;
    if constexpr (!ENV) {
        return A(0);
    } else {
        const long long i = q * pl.env_stride + ((long long)(1 << n) + j) * C + c;
        if constexpr (P == P_FP64) return pl.envd[i];
        else return pl.envf[i];
    }
}

// Whether a plan carries an environment map (kernels dispatch on it).
inline bool plan_has_env(const Plan &pl) { return pl.envf != nullptr || pl.envd != nullptr; }

template <int P, int C> struct RLevel {
    using SL = typename Prec<P>::SL;
    using A = typename Prec<P>::A;
    SL *base;
    int I, Vs;
    __device__ __forceinline__ RLevel(const Plan &pl, int q, int n) {
        base = reinterpret_cast<SL *>(pl.arena + pl.q[q].Roff[n]);
        I = 1 << n;
        Vs = pl.q[q].Vs;
    }
    __device__ __forceinline__ long long idx(int x, int i, int c, int v) const {
        return (((long long)x * I + i) * C + c) * Vs + v;
    }
    __device__ __forceinline__ A load(int x, int i, int c, int v) const { return to_acc(base[idx(x, i, c, v)]); }
    __device__ __forceinline__ void store(int x, int i, int c, int v, A val) const { base[idx(x, i, c, v)] = from_acc<SL>(val); }
    __device__ __forceinline__ void load2(int x, int i, int c, int v, A &a, A &b) const { ld2(base + idx(x, i, c, v), a, b); }
    __device__ __forceinline__ void store2(int x, int i, int c, int v, A a, A b) const { st2(base + idx(x, i, c, v), a, b); }
    __device__ __forceinline__ void load4(int x, int i, int c, int v, A (&r)[4]) const { ld4(base + idx(x, i, c, v), r); }
    __device__ __forceinline__ void store4(int x, int i, int c, int v, const A (&r)[4]) const {
        st4(base + idx(x, i, c, v), r);
    }
};

// Adjoint levels: dLoss/dT_n entries (C radiance components, then the
// derivative with respect to the LINEAR transmittance, in every precision)
// and dLoss/dR_n, both stored in the arithmetic type with the T/R layouts.
template <int P, int C> struct GTLevel {
    using A = typename Prec<P>::A;
    char *base;
    int K, Vs;
    long long G;
    __device__ __forceinline__ GTLevel(const Plan &pl, int q, int n) {
        base = pl.arena + pl.q[q].gToff[n];
        K = (1 << n) + 1;
        Vs = pl.q[q].Vs;
        G = (long long)Vs * (C + 1) * (long long)sizeof(A);
    }
    __device__ __forceinline__ A *row(int x, int k) const { return reinterpret_cast<A *>(base + ((long long)x * K + k) * G); }
    __device__ __forceinline__ void load(int x, int k, int v, A (&L)[C], A &T) const {
        const A *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) L[c] = g[(long long)c * Vs + v];
        T = g[(long long)C * Vs + v];
    }
    __device__ __forceinline__ void store(int x, int k, int v, const A (&L)[C], A T) const {
        A *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) g[(long long)c * Vs + v] = L[c];
        g[(long long)C * Vs + v] = T;
    }
    // entries v and v+1 (v even)
    __device__ __forceinline__ void load2(int x, int k, int v, A (&L)[2][C], A (&T)[2]) const {
        const A *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) ld2(g + (long long)c * Vs + v, L[0][c], L[1][c]);
        ld2(g + (long long)C * Vs + v, T[0], T[1]);
    }
    __device__ __forceinline__ void store2(int x, int k, int v, const A (&L)[2][C], const A (&T)[2]) const {
        A *g = row(x, k);
#pragma unroll
        for (int c = 0; c < C; ++c) st2(g + (long long)c * Vs + v, L[0][c], L[1][c]);
        st2(g + (long long)C * Vs + v, T[0], T[1]);
    }
};

template <int P, int C> struct GRLevel {
    using A = typename Prec<P>::A;
    A *base;
    int I, Vs;
    __device__ __forceinline__ GRLevel(const Plan &pl, int q, int n) {
        base = reinterpret_cast<A *>(pl.arena + pl.q[q].gRoff[n]);
        I = 1 << n;
        Vs = pl.q[q].Vs;
    }
    __device__ __forceinline__ long long idx(int x, int i, int c, int v) const {
        return (((long long)x * I + i) * C + c) * Vs + v;
    }
    __device__ __forceinline__ A load(int x, int i, int c, int v) const { return base[idx(x, i, c, v)]; }
    __device__ __forceinline__ void load2(int x, int i, int c, int v, A &a, A &b) const { ld2(base + idx(x, i, c, v), a, b); }
    __device__ __forceinline__ void store(int x, int i, int c, int v, A val) const { base[idx(x, i, c, v)] = val; }
    __device__ __forceinline__ void store2(int x, int i, int c, int v, A a, A b) const { st2(base + idx(x, i, c, v), a, b); }
};

template <int P> __device__ __forceinline__ typename Prec<P>::A arc(const Plan &pl, int n, int j) {
    if (P == P_FP64) return reinterpret_cast<const double *>(pl.arena + pl.arcs_off_d)[(1 << n) + j];
    return reinterpret_cast<const float *>(pl.arena + pl.arcs_off)[(1 << n) + j];
}

}  // namespace hrc
