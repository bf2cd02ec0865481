// trace_shapes.cuh -- compile-time shapes of the directly traced rays.
//
// Levels 0..2 are traced directly (Sec. 4.2) from the probe at a pixel
// centre along v_n(k) = (2^n, 2k - 2^n) (Sec. 4), so the pixels a ray
// crosses and the lengths inside them do not depend on the probe: ten fixed
// shapes.  They are derived here at compile time by clipping the segment
// against the integer grid lines in exact integer arithmetic (crossings of
// u = g at t = (2g-1)/(2a), of v at t = (2m-1)/(2|b|), over the common
// denominator D = 2a|b|).  Every piece then has one of three directions
// classes and is either a "half" piece (t-length 1/(2a): from a pixel centre
// to an edge, or the short pieces of the slope-1/2 rays) or a "full" piece
// (twice that length):
//   class 0: along the axis,  half length 1/2
//   class 1: diagonal,        half length sqrt(2)/2
//   class 2: slope 1/2,       half length sqrt(5)/4
// so a pixel's per-piece transmittance and weight for a full piece follow
// from the half piece's: t2 = t^2, w2 = w (1 + t).
#pragma once

#include "hrc_internal.cuh"

namespace hrc {

struct ShapePiece {
    int du, dv, cls, full;
};
struct Shapes {
    int start[HRC_MAXRAY + 1];
    ShapePiece p[HRC_MAXPIECE];
};

constexpr long long floor_div(long long a, long long b) {   // b > 0
    return a >= 0 ? a / b : -((-a + b - 1) / b);
}

constexpr Shapes make_shapes() {
    Shapes S{};
    int np = 0;
    for (int n = 0; n <= 2; ++n) {
        const int a = 1 << n;
        for (int k = 0; k <= a; ++k) {
            const int r = n == 0 ? k : (n == 1 ? 2 + k : 5 + k);
            S.start[r] = np;
            const int b = 2 * k - a;
            const int ab = b < 0 ? -b : b;
            const long long D = 2LL * a * (ab > 0 ? ab : 1);
            long long ts[16] = {};
            int nt = 0;
            ts[nt++] = 0;
            ts[nt++] = D;
            for (int g = 1; g <= a; ++g) ts[nt++] = (2LL * g - 1) * (D / (2LL * a));
            for (int m = 1; m <= ab; ++m) ts[nt++] = (2LL * m - 1) * (D / (2LL * ab));
            for (int i = 1; i < nt; ++i)                 // insertion sort
                for (int j = i; j > 0 && ts[j - 1] > ts[j]; --j) {
                    const long long t = ts[j]; ts[j] = ts[j - 1]; ts[j - 1] = t;
                }
            const int cls = b == 0 ? 0 : (ab == a ? 1 : 2);
            for (int i = 0; i + 1 < nt; ++i) {
                if (ts[i + 1] == ts[i]) continue;         // corner crossing: zero length
                const long long tsum = ts[i] + ts[i + 1];  // 2 D t_mid
                S.p[np].du = (int)floor_div(D + a * tsum, 2 * D);
                S.p[np].dv = (int)floor_div(D + b * tsum, 2 * D);
                S.p[np].cls = cls;
                S.p[np].full = (ts[i + 1] - ts[i]) == D / a ? 1 : 0;
                ++np;
            }
        }
    }
    S.start[HRC_MAXRAY] = np;
    return S;
}

constexpr Shapes kShapes = make_shapes();
static_assert(kShapes.start[HRC_MAXRAY] == 42, "4 + 9 + 29 pieces");
static_assert(kShapes.start[2] == 4 && kShapes.start[5] == 13, "ray boundaries");

// Compile-time access for device code (template constants).
template <int J> struct PieceAt {
    static constexpr int du = kShapes.p[J].du;
    static constexpr int dv = kShapes.p[J].dv;
    static constexpr int cls = kShapes.p[J].cls;
    static constexpr int full = kShapes.p[J].full;
};
template <int R> struct RayAt {
    static constexpr int begin = kShapes.start[R];
    static constexpr int end = kShapes.start[R + 1];
    static constexpr int n = R < 2 ? 0 : (R < 5 ? 1 : 2);
    static constexpr int k = R - (n == 0 ? 0 : (n == 1 ? 2 : 5));
};

// half-piece lengths of the three classes
template <class A> __host__ __device__ constexpr A class_len(int cls) {
    return cls == 0 ? A(0.5) : (cls == 1 ? A(0.70710678118654752440) : A(0.55901699437494742410));
}

}  // namespace hrc
