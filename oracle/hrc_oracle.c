/*
 * hrc_oracle.c -- plain, slow FP64 CPU oracle of Holographic Radiance
 * Cascades (HRC), written from the paper's equations and Algorithm 1.
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA path.  Only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the product never links, imports or calls it, and the two share no
 * code, header, table or helper.
 *
 * Conventions (the readings of passages the paper leaves open):
 *   - Pixel (u, v) is the unit square [u, u+1] x [v, v+1]; the probe of
 *     pixel (u, v) sits at its centre (u + 1/2, v + 1/2)  (Sec. 4, Sec. 5).
 *   - Input e is the per-unit-length source term integrated in Eq. 4, so a
 *     uniform piece of length l gives L = e * l * phi(sigma*l) with
 *     phi(t) = (1 - exp(-t)) / t, T = exp(-sigma*l)  (Eqs. 2, 4; Fig. 2).
 *   - Quadrant frames replace the world rotation of Algorithm 1 (Lighting):
 *       q0: (u,v) = (x, y)      q1: (u,v) = (W-1-x, y)
 *       q2: (u,v) = (y, x)      q3: (u,v) = (H-1-y, x)
 *     Each frame gathers the quadrant of directions within pi/4 of +u.
 *   - N = ceil(log2 U) per frame (Sec. 4.2); a positive `cascades` caps it.
 *   - Arrays cover exactly Algorithm 1's ranges; T lookups outside them are
 *     vacuum <0, 1>, R lookups outside them and R_N are 0 (Sec. 4.2,
 *     footnote 1).
 *   - Eq. 20 averages both radiance and transmittance; Eq. 15 averages
 *     angular fluence.
 *
 * Every function cites the passage it follows.  Parity of the whole method
 * against Eq. 1 (brute force) is an approximation bound, not an identity.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 16

/* ---------------------------------------------------------------------------
 * Frame fields (Algorithm 1, Lighting: one orientation per quadrant).
 * ------------------------------------------------------------------------ */
typedef struct {
    int C, U, V;
    double *e;   /* [C][U][V] */
    double *s;   /* [U][V]    */
} Frame;

/* frame (u, v) -> original pixel (x, y) for quadrant q */
static void frame_to_image(int q, int W, int H, long u, long v, long *x, long *y)
{
    switch (q) {
    case 0: *x = u;         *y = v;         break;
    case 1: *x = W - 1 - u; *y = v;         break;
    case 2: *x = v;         *y = u;         break;
    default: *x = v;        *y = H - 1 - u; break;
    }
}

static void frame_dims(int q, int W, int H, int *U, int *V)
{
    if (q < 2) { *U = W; *V = H; } else { *U = H; *V = W; }
}

static Frame frame_build(int q, const double *e, const double *s, int C, int W, int H)
{
    Frame f;
    frame_dims(q, W, H, &f.U, &f.V);
    f.C = C;
    f.e = (double *)malloc(sizeof(double) * (size_t)C * f.U * f.V);
    f.s = (double *)malloc(sizeof(double) * (size_t)f.U * f.V);
    for (long u = 0; u < f.U; ++u)
        for (long v = 0; v < f.V; ++v) {
            long x, y;
            frame_to_image(q, W, H, u, v, &x, &y);
            f.s[u * f.V + v] = s[y * W + x];
            for (int c = 0; c < C; ++c)
                f.e[((size_t)c * f.U + u) * f.V + v] = e[((size_t)c * H + y) * W + x];
        }
    return f;
}

static void frame_free(Frame *f) { free(f->e); free(f->s); }

/* ---------------------------------------------------------------------------
 * Trace (Eq. 9): <L_r(p <- q), T_r(p <- q)> of Eqs. 2 and 4, by exact
 * clipping of the segment p->q against the pixel squares (Sec. 5: each
 * pixel is a square of uniform extinction and emission).  Pieces are folded
 * front to back with Merge (Eq. 7).
 * ------------------------------------------------------------------------ */
typedef struct { long u, v; double len; } Piece;

static int cmp_double(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Pieces of segment p->q, front to back.  Uses the caller's buffers when
 * they are large enough (cap entries), else allocates; *owned tells the
 * caller to free *out. */
static int segment_pieces(double pu, double pv, double qu, double qv,
                          Piece *buf, double *tbuf, int cap, Piece **out, int *owned)
{
    double du = qu - pu, dv = qv - pv;
    double d = sqrt(du * du + dv * dv);
    long nu = (long)fabs(floor(qu) - floor(pu)) + 2;
    long nv = (long)fabs(floor(qv) - floor(pv)) + 2;
    long need = nu + nv + 2;
    double *t = need <= cap ? tbuf : (double *)malloc(sizeof(double) * (size_t)need);
    Piece *pc = need <= cap ? buf : (Piece *)malloc(sizeof(Piece) * (size_t)need);
    int nt = 0;
    t[nt++] = 0.0;
    t[nt++] = 1.0;
    if (du != 0.0) {
        double lo = fmin(pu, qu), hi = fmax(pu, qu);
        for (double g = floor(lo) + 1.0; g < hi; g += 1.0) t[nt++] = (g - pu) / du;
    }
    if (dv != 0.0) {
        double lo = fmin(pv, qv), hi = fmax(pv, qv);
        for (double g = floor(lo) + 1.0; g < hi; g += 1.0) t[nt++] = (g - pv) / dv;
    }
    qsort(t, (size_t)nt, sizeof(double), cmp_double);
    int np = 0;
    for (int a = 0; a + 1 < nt; ++a) {
        double ta = t[a], tb = t[a + 1];
        if (!(tb > ta)) continue;
        double tm = 0.5 * (ta + tb);
        pc[np].u = (long)floor(pu + tm * du);
        pc[np].v = (long)floor(pv + tm * dv);
        pc[np].len = (tb - ta) * d;
        ++np;
    }
    if (t != tbuf) free(t);
    *owned = pc != buf;
    *out = pc;
    return np;
}

#define PIECE_CAP 64

static double frame_sigma(const Frame *f, long u, long v)
{
    if (u < 0 || v < 0 || u >= f->U || v >= f->V) return 0.0;
    return f->s[u * f->V + v];
}

static double frame_emis(const Frame *f, int c, long u, long v)
{
    if (u < 0 || v < 0 || u >= f->U || v >= f->V) return 0.0;
    return f->e[((size_t)c * f->U + u) * f->V + v];
}

/* phi(t) = (1 - exp(-t)) / t, phi(0) = 1: radiance of a uniform piece is
 * e * l * phi(sigma * l)  (Eq. 4 integrated over a piece). */
static double phi(double t) { return t != 0.0 ? -expm1(-t) / t : 1.0; }

/* d phi / d t, evaluated without cancellation near 0 (Taylor series of
 * phi'(t) = (exp(-t)(1+t) - 1)/t^2). */
static double dphi(double t)
{
    if (fabs(t) < 1e-2)
        return -0.5 + t * (1.0 / 3.0 + t * (-1.0 / 8.0 + t * (1.0 / 30.0 + t * (-1.0 / 144.0 + t * (1.0 / 840.0)))));
    return (exp(-t) * (1.0 + t) - 1.0) / (t * t);
}

/* Trace(p, q), Eq. 9, in frame coordinates. L has C entries. */
static void trace(const Frame *f, double pu, double pv, double qu, double qv, double *L, double *T)
{
    Piece buf[PIECE_CAP], *pc;
    double tbuf[PIECE_CAP];
    int owned;
    int np = segment_pieces(pu, pv, qu, qv, buf, tbuf, PIECE_CAP, &pc, &owned);
    for (int c = 0; c < f->C; ++c) L[c] = 0.0;
    double Tacc = 1.0;
    for (int m = 0; m < np; ++m) {
        double sg = frame_sigma(f, pc[m].u, pc[m].v);
        double l = pc[m].len;
        double tau = sg * l;
        double w = l * phi(tau);
        for (int c = 0; c < f->C; ++c) L[c] += Tacc * frame_emis(f, c, pc[m].u, pc[m].v) * w;
        Tacc *= exp(-tau);
    }
    *T = Tacc;
    if (owned) free(pc);
}

/* Adjoint of trace: accumulates d/d e and d/d sigma of
 * sum_c gL[c] * L[c] + gT * T into ge (frame [C][U][V]) and gs ([U][V]). */
static void trace_adjoint(const Frame *f, double pu, double pv, double qu, double qv,
                          const double *gL, double gT, double *ge, double *gs)
{
    Piece buf[PIECE_CAP], *pc;
    double tbuf[PIECE_CAP];
    int owned;
    int np = segment_pieces(pu, pv, qu, qv, buf, tbuf, PIECE_CAP, &pc, &owned);
    int C = f->C;
    double *P = (double *)malloc(sizeof(double) * (size_t)(np + 1));   /* prefix T */
    double *a = (double *)malloc(sizeof(double) * (size_t)(np * C + 1)); /* P_m * a_m */
    double *S = (double *)malloc(sizeof(double) * (size_t)(np * C + 1)); /* sum_{m'>m} */
    P[0] = 1.0;
    for (int m = 0; m < np; ++m) {
        double sg = frame_sigma(f, pc[m].u, pc[m].v);
        double l = pc[m].len;
        for (int c = 0; c < C; ++c)
            a[m * C + c] = P[m] * frame_emis(f, c, pc[m].u, pc[m].v) * l * phi(sg * l);
        P[m + 1] = P[m] * exp(-sg * l);
    }
    double Ttot = P[np];
    for (int c = 0; c < C; ++c) {
        double acc = 0.0;
        for (int m = np - 1; m >= 0; --m) {
            S[m * C + c] = acc;
            acc += a[m * C + c];
        }
    }
    for (int m = 0; m < np; ++m) {
        long u = pc[m].u, v = pc[m].v;
        if (u < 0 || v < 0 || u >= f->U || v >= f->V) continue;
        double sg = f->s[u * f->V + v];
        double l = pc[m].len;
        double g = 0.0;
        for (int c = 0; c < C; ++c) {
            double em = f->e[((size_t)c * f->U + u) * f->V + v];
            ge[((size_t)c * f->U + u) * f->V + v] += gL[c] * P[m] * l * phi(sg * l);
            g += gL[c] * (P[m] * em * l * l * dphi(sg * l) - l * S[m * C + c]);
        }
        g -= gT * l * Ttot;
        gs[u * f->V + v] += g;
    }
    free(P); free(a); free(S);
    if (owned) free(pc);
}

/* ---------------------------------------------------------------------------
 * Probe layout (Sec. 4): level n has probes p = (x 2^n, y); direction
 * k in [0, 2^n] has offset v_n(k) = (2^n, 2k - 2^n).  Cone i (half-integer,
 * stored as i' = i - 1/2) spans v_n(i - 1/2) .. v_n(i + 1/2).
 * ------------------------------------------------------------------------ */
static long level_cols(long U, int n) { return (U + (1L << n) - 1) >> n; }

/* Eq. 13: A_n(i) = angle(v_n(i + 1/2)) - angle(v_n(i - 1/2)),
 * angle([x, y]) = atan(y / x); ip = i - 1/2. */
double orc_arc(int n, int ip)
{
    double s = (double)(1L << n);
    double hi = atan((2.0 * (ip + 1) - s) / s);
    double lo = atan((2.0 * ip - s) / s);
    return hi - lo;
}

int orc_levels(int U, int cascades)
{
    int N = 0;
    while ((1L << N) < U) ++N;
    if (cascades > 0 && cascades < N) N = cascades;
    return N;
}

typedef struct {
    int C, U, V, N;
    long Un[ORC_MAXL + 1];
    double *T[ORC_MAXL + 1];   /* [x][k][v][C+1]: C radiances then T */
    double *R[ORC_MAXL + 1];   /* [x][i][v][C]; R[N] unused (== 0)   */
    double *Renv[ORC_MAXL + 1];/* [i][C] environment values, or NULL */
} Cascades;

static size_t T_index(const Cascades *cs, int n, long x, long k, long v)
{
    long K = (1L << n) + 1;
    return (((size_t)x * K + k) * cs->V + v) * (cs->C + 1);
}

static size_t R_index(const Cascades *cs, int n, long x, long i, long v)
{
    long I = 1L << n;
    return (((size_t)x * I + i) * cs->V + v) * cs->C;
}

/* T_n(p, k) at position p = (pu, pv) with pu a multiple of 2^n; outside
 * the stored ranges the interval is vacuum <0, 1> (handled by caller via
 * the returned flag). */
static const double *T_get(const Cascades *cs, int n, long pu, long pv, long k)
{
    long x = pu >> n;
    if (pu < 0 || x >= cs->Un[n] || pv < 0 || pv >= cs->V) return NULL;
    return cs->T[n] + T_index(cs, n, x, k, pv);
}

/* R_n(p, i) (i' index), zero outside the stored ranges and for n >= N. */
static const double *R_get(const Cascades *cs, int n, long pu, long pv, long ip)
{
    if (n >= cs->N) return NULL;
    long x = pu >> n;
    if (pu < 0 || x >= cs->Un[n] || pv < 0 || pv >= cs->V) return NULL;
    return cs->R[n] + R_index(cs, n, x, ip, pv);
}

/* The value of R_n(p, i) wherever it is looked up: the stored entry, else
 * (outside the stored ranges, or n = N) the environment's value of cone i
 * at level n, or NULL (= 0) without an environment (footnote 1 of
 * Sec. 4.2: R_N from an environment map looked up along v_N(i)). */
static const double *R_val(const Cascades *cs, int n, long pu, long pv, long ip)
{
    const double *r = R_get(cs, n, pu, pv, ip);
    if (r) return r;
    return cs->Renv[n] ? cs->Renv[n] + (size_t)ip * cs->C : NULL;
}

/* Environment radiance seen along the image direction (dx, dy), y down the
 * rows: env[c][m] samples the look angle theta_m = 2 pi (m + 1/2) / M with
 * theta = atan2(dy, dx) in [0, 2 pi); linear interpolation, periodic. */
static double env_lookup(const double *env, int M, int c, double dx, double dy)
{
    double th = atan2(dy, dx);
    if (th < 0) th += 2.0 * M_PI;
    double t = th * M / (2.0 * M_PI) - 0.5;
    double m0 = floor(t), fr = t - m0;
    long i0 = ((long)m0 % M + M) % M, i1 = (i0 + 1) % M;
    return (1.0 - fr) * env[(size_t)c * M + i0] + fr * env[(size_t)c * M + i1];
}

/* frame direction (du, dv) -> image direction (dx, dy), inverse of the
 * quadrant maps of frame_to_image */
static void frame_dir_to_image(int q, double du, double dv, double *dx, double *dy)
{
    switch (q) {
    case 0: *dx = du;  *dy = dv;  break;
    case 1: *dx = -du; *dy = dv;  break;
    case 2: *dx = dv;  *dy = du;  break;
    default: *dx = dv; *dy = -du; break;
    }
}

/* Environment values of frame q: at level N, cone j' = j + 1/2 sees
 * A_N(j') E(direction of v_N(j')) -- or, when the caller supplies the
 * top-level radiance itself (footnote 1 of Sec. 4.2: R_N computed by some
 * other method), top[q][j][c] (K entries per frame); an out-of-range lookup
 * at level n < N sees, through vacuum (nothing outside the grid absorbs or
 * emits), the sum of its two cones at level n + 1 (Eq. 14 / Eq. 15 with
 * T = <0, 1>), i.e. of its level-N descendants. */
static void env_tables(Cascades *cs, int q, const double *env, int M, const double *top, int K)
{
    int C = cs->C, N = cs->N;
    for (int n = 0; n <= N; ++n) cs->Renv[n] = NULL;
    if (!env && !top) return;
    for (int n = N; n >= 0; --n) {
        long I = 1L << n;
        cs->Renv[n] = (double *)calloc((size_t)I * C, sizeof(double));
        for (long j = 0; j < I; ++j)
            for (int c = 0; c < C; ++c) {
                double v;
                if (n == N && top) {
                    v = top[((size_t)q * K + j) * C + c];
                } else if (n == N) {
                    double dx, dy, s2 = (double)(1L << n);
                    frame_dir_to_image(q, s2, 2.0 * j + 1.0 - s2, &dx, &dy);
                    v = orc_arc(n, (int)j) * env_lookup(env, M, c, dx, dy);
                } else {
                    v = cs->Renv[n + 1][(size_t)(2 * j) * C + c] + cs->Renv[n + 1][(size_t)(2 * j + 1) * C + c];
                }
                cs->Renv[n][(size_t)j * C + c] = v;
            }
    }
}

/* Merge (Eq. 7) of near a and far b, each C radiances + T; NULL = vacuum. */
static void merge(int C, const double *a, const double *b, double *out)
{
    double Ta = a ? a[C] : 1.0, Tb = b ? b[C] : 1.0;
    for (int c = 0; c < C; ++c) {
        double La = a ? a[c] : 0.0, Lb = b ? b[c] : 0.0;
        out[c] = La + Ta * Lb;
    }
    out[C] = Ta * Tb;
}

/* Algorithm 1, procedure HRC, for one frame.  Keeps every T and R level. */
static void hrc_frame(const Frame *f, int cascades, int q, const double *env, int M, const double *top, int K,
                      Cascades *cs)
{
    int C = f->C;
    cs->C = C; cs->U = f->U; cs->V = f->V;
    cs->N = orc_levels(f->U, cascades);
    int N = cs->N;
    env_tables(cs, q, env, M, top, K);
    for (int n = 0; n <= N; ++n) {
        cs->Un[n] = level_cols(f->U, n);
        long K = (1L << n) + 1;
        cs->T[n] = (double *)calloc((size_t)cs->Un[n] * K * f->V * (C + 1), sizeof(double));
        cs->R[n] = NULL;
        if (n < N)
            cs->R[n] = (double *)calloc((size_t)cs->Un[n] * (1L << n) * f->V * C, sizeof(double));
    }

    /* T_0 .. T_2 by direct tracing (Algorithm 1; Sec. 4.2: levels 0-2 are
     * traced to reduce error).  Levels above 2 but <= N are merged. */
    int ntrace = N < 2 ? N : 2;
    for (int n = 0; n <= ntrace; ++n) {
        long s = 1L << n, K = s + 1;
#pragma omp parallel for schedule(static)
        for (long y = 0; y < f->V; ++y)
            for (long x = 0; x < cs->Un[n]; ++x)
                for (long k = 0; k < K; ++k) {
                    double pu = x * s + 0.5, pv = y + 0.5;
                    double *o = cs->T[n] + T_index(cs, n, x, k, y);
                    trace(f, pu, pv, pu + s, pv + (2.0 * k - s), o, o + C);
                }
    }

    /* T_3 .. T_N from T_{n-1}: Eq. 18 (even k), Eqs. 19-20 (odd k). */
    for (int n = 3; n <= N; ++n) {
        int m = n - 1;                 /* the level merged from */
        long sm = 1L << m, K = (1L << n) + 1;
#pragma omp parallel for schedule(static)
        for (long y = 0; y < f->V; ++y) {
            double Fp[8], Fm[8];
            for (long x = 0; x < cs->Un[n]; ++x)
                for (long k = 0; k < K; ++k) {
                    long pu = x << n, pv = y;
                    double *o = cs->T[n] + T_index(cs, n, x, k, y);
                    if ((k & 1) == 0) {
                        long kk = k / 2;   /* T_n(p, 2kk) = Merge(T_m(p,kk), T_m(p+v_m(kk),kk)) */
                        merge(C, T_get(cs, m, pu, pv, kk),
                              T_get(cs, m, pu + sm, pv + 2 * kk - sm, kk), o);
                    } else {
                        long kp = (k + 1) / 2, km = (k - 1) / 2;   /* kappa +- 1/2 */
                        /* F_+ = Merge(T_m(p, kappa+1/2), T_m(p + v_m(kappa+1/2), kappa-1/2)) */
                        merge(C, T_get(cs, m, pu, pv, kp),
                              T_get(cs, m, pu + sm, pv + 2 * kp - sm, km), Fp);
                        /* F_- = Merge(T_m(p, kappa-1/2), T_m(p + v_m(kappa-1/2), kappa+1/2)) */
                        merge(C, T_get(cs, m, pu, pv, km),
                              T_get(cs, m, pu + sm, pv + 2 * km - sm, kp), Fm);
                        for (int c = 0; c <= C; ++c) o[c] = 0.5 * (Fm[c] + Fp[c]);   /* Eq. 20 */
                    }
                }
        }
    }

    /* R_{N-1} .. R_0 (Eqs. 14-17 with T from Sec. 4.1), R_N = 0. */
    for (int n = N - 1; n >= 0; --n) {
        long s = 1L << n, I = s;
#pragma omp parallel for schedule(static)
        for (long y = 0; y < f->V; ++y)
            for (long x = 0; x < cs->Un[n]; ++x)
                for (long ip = 0; ip < I; ++ip) {
                    long pu = x * s, pv = y;
                    double *o = cs->R[n] + R_index(cs, n, x, ip, y);
                    /* j_+ = 2i + 1/2 -> index 2ip+1; j_- = 2i - 1/2 -> 2ip */
                    long jp = 2 * ip + 1, jm = 2 * ip;
                    double Ap = orc_arc(n + 1, (int)jp);
                    double Am = orc_arc(n + 1, (int)jm);
                    for (int c = 0; c < C; ++c) o[c] = 0.0;
                    if (x & 1) {
                        /* Eq. 14: F_+- = Merge_r(A x T_n(p, i +- 1/2), R_{n+1}(q_+-, j_+-)),
                         * q_+- = p + v_n(i +- 1/2); i + 1/2 = ip + 1, i - 1/2 = ip. */
                        for (int sgn = 0; sgn < 2; ++sgn) {
                            long kk = sgn == 0 ? ip + 1 : ip;
                            long j = sgn == 0 ? jp : jm;
                            double A = sgn == 0 ? Ap : Am;
                            const double *t = T_get(cs, n, pu, pv, kk);
                            const double *r = R_val(cs, n + 1, pu + s, pv + 2 * kk - s, j);
                            double Tt = t ? t[C] : 1.0;
                            for (int c = 0; c < C; ++c)
                                o[c] += A * (t ? t[c] : 0.0) + Tt * (r ? r[c] : 0.0);
                        }
                    } else {
                        /* Eqs. 15-17: F_+- = (R_{n+1}(p, j) + Merge_r(A x T_{n+1}(p, 2i +- 1),
                         * R_{n+1}(p + v_{n+1}(2i +- 1), j))) / 2; 2i+1 = 2ip+2, 2i-1 = 2ip. */
                        long s1 = 2 * s;
                        for (int sgn = 0; sgn < 2; ++sgn) {
                            long kk = sgn == 0 ? 2 * ip + 2 : 2 * ip;
                            long j = sgn == 0 ? jp : jm;
                            double A = sgn == 0 ? Ap : Am;
                            const double *r0 = R_val(cs, n + 1, pu, pv, j);
                            const double *t = T_get(cs, n + 1, pu, pv, kk);
                            const double *r1 = R_val(cs, n + 1, pu + s1, pv + 2 * kk - s1, j);
                            double Tt = t ? t[C] : 1.0;
                            for (int c = 0; c < C; ++c)
                                o[c] += 0.5 * ((r0 ? r0[c] : 0.0) + A * (t ? t[c] : 0.0) +
                                               Tt * (r1 ? r1[c] : 0.0));
                        }
                    }
                }
    }
}

static void cascades_free(Cascades *cs)
{
    for (int n = 0; n <= cs->N; ++n) { free(cs->T[n]); free(cs->R[n]); free(cs->Renv[n]); }
}

/* ---------------------------------------------------------------------------
 * Exported entry points.  Images are row-major: e[C][H][W], s[H][W].
 * ------------------------------------------------------------------------ */

/* Trace (Eq. 9) in image coordinates (frame q0). */
void orc_trace(const double *e, const double *s, int C, int W, int H,
               double px, double py, double qx, double qy, double *L, double *T)
{
    Frame f = frame_build(0, e, s, C, W, H);
    trace(&f, px, py, qx, qy, L, T);
    frame_free(&f);
}

/* Algorithm 1, Lighting: F(x, y) = sum over quadrants of R_0([x+1, y], 0);
 * with an environment map env[C][M] (NULL: none), footnote 1 of Sec. 4.2. */
static void fluence_outside(const double *e, const double *s, int C, int W, int H, int cascades, const double *env,
                            int M, const double *top, int K, double *F)
{
    memset(F, 0, sizeof(double) * (size_t)C * W * H);
    for (int q = 0; q < 4; ++q) {
        Frame f = frame_build(q, e, s, C, W, H);
        Cascades cs;
        hrc_frame(&f, cascades, q, env, M, top, K, &cs);
        for (long u = 0; u < f.U; ++u)
            for (long v = 0; v < f.V; ++v) {
                long x, y;
                frame_to_image(q, W, H, u, v, &x, &y);
                const double *r = R_val(&cs, 0, u + 1, v, 0);
                if (!r) continue;
                for (int c = 0; c < C; ++c) F[((size_t)c * H + y) * W + x] += r[c];
            }
        cascades_free(&cs);
        frame_free(&f);
    }
}

void orc_fluence_env(const double *e, const double *s, int C, int W, int H, int cascades, const double *env, int M,
                     double *F)
{
    fluence_outside(e, s, C, W, H, cascades, env, M, NULL, 0, F);
}

/* The same with the top-level radiance top[4][K][C] given (cone j < 2^N of
 * frame q at level N at top[(q K + j) C + c]). */
void orc_fluence_top(const double *e, const double *s, int C, int W, int H, int cascades, const double *top, int K,
                     double *F)
{
    fluence_outside(e, s, C, W, H, cascades, NULL, 0, top, K, F);
}

void orc_fluence(const double *e, const double *s, int C, int W, int H, int cascades, double *F)
{
    fluence_outside(e, s, C, W, H, cascades, NULL, 0, NULL, 0, F);
}

/* One level of one frame, for level-by-level tests.  which = 0: T_n
 * ([x][k][v][C+1]); which = 1: R_n ([x][i][v][C]).  Returns the number of
 * doubles written, or -1 when the level does not exist. */
long orc_frame_level(const double *e, const double *s, int C, int W, int H, int q,
                     int cascades, int which, int n, double *out)
{
    Frame f = frame_build(q, e, s, C, W, H);
    Cascades cs;
    hrc_frame(&f, cascades, q, NULL, 0, NULL, 0, &cs);
    long cnt = -1;
    if (which == 0 && n >= 0 && n <= cs.N) {
        cnt = cs.Un[n] * ((1L << n) + 1) * f.V * (C + 1);
        if (out) memcpy(out, cs.T[n], sizeof(double) * (size_t)cnt);
    } else if (which == 1 && n >= 0 && n < cs.N) {
        cnt = cs.Un[n] * (1L << n) * f.V * C;
        if (out) memcpy(out, cs.R[n], sizeof(double) * (size_t)cnt);
    }
    cascades_free(&cs);
    frame_free(&f);
    return cnt;
}

/* Gradient of sum(gF * F) with respect to e and s (the FP64 reverse of
 * orc_fluence: reverse fluence sum, reverse merge down, reverse merge up,
 * reverse trace).  ge, gs are overwritten. */
static void adjoint_outside(const double *e, const double *s, const double *gF, int C, int W, int H, int cascades,
                            const double *env, int M, const double *top, int K, double *ge, double *gs)
{
    memset(ge, 0, sizeof(double) * (size_t)C * W * H);
    memset(gs, 0, sizeof(double) * (size_t)W * H);
    for (int q = 0; q < 4; ++q) {
        Frame f = frame_build(q, e, s, C, W, H);
        Cascades cs;
        hrc_frame(&f, cascades, q, env, M, top, K, &cs);
        int N = cs.N;
        if (N < 1) { cascades_free(&cs); frame_free(&f); continue; }
        double *gT[ORC_MAXL + 1], *gR[ORC_MAXL + 1];
        for (int n = 0; n <= N; ++n) {
            size_t nt = (size_t)cs.Un[n] * ((1L << n) + 1) * f.V * (C + 1);
            gT[n] = (double *)calloc(nt, sizeof(double));
            gR[n] = NULL;
            if (n < N) gR[n] = (double *)calloc((size_t)cs.Un[n] * (1L << n) * f.V * C, sizeof(double));
        }
        /* reverse of the fluence sum */
        for (long u = 0; u < f.U; ++u)
            for (long v = 0; v < f.V; ++v) {
                long x, y;
                frame_to_image(q, W, H, u, v, &x, &y);
                if (u + 1 >= cs.Un[0]) continue;
                double *g = gR[0] + R_index(&cs, 0, u + 1, 0, v);
                for (int c = 0; c < C; ++c) g[c] += gF[((size_t)c * H + y) * W + x];
            }
        /* reverse merge down: n = 0 .. N-1 */
        for (int n = 0; n < N; ++n) {
            long sn = 1L << n;
            for (long x = 0; x < cs.Un[n]; ++x)
                for (long ip = 0; ip < sn; ++ip)
                    for (long y = 0; y < f.V; ++y) {
                        const double *g = gR[n] + R_index(&cs, n, x, ip, y);
                        long pu = x * sn, pv = y;
                        long jp = 2 * ip + 1, jm = 2 * ip;
                        for (int sgn = 0; sgn < 2; ++sgn) {
                            long j = sgn == 0 ? jp : jm;
                            double A = orc_arc(n + 1, (int)j);
                            if (x & 1) {
                                long kk = sgn == 0 ? ip + 1 : ip;
                                long qu = pu + sn, qv = pv + 2 * kk - sn;
                                const double *t = T_get(&cs, n, pu, pv, kk);
                                const double *r = R_get(&cs, n + 1, qu, qv, j);
                                const double *rv = R_val(&cs, n + 1, qu, qv, j);
                                double Tt = t ? t[C] : 1.0;
                                if (t) {
                                    double *gt = gT[n] + T_index(&cs, n, x, kk, y);
                                    for (int c = 0; c < C; ++c) {
                                        gt[c] += A * g[c];
                                        gt[C] += g[c] * (rv ? rv[c] : 0.0);
                                    }
                                }
                                if (r) {
                                    double *gr = gR[n + 1] + R_index(&cs, n + 1, qu >> (n + 1), j, qv);
                                    for (int c = 0; c < C; ++c) gr[c] += Tt * g[c];
                                }
                            } else {
                                long s1 = 2 * sn;
                                long kk = sgn == 0 ? 2 * ip + 2 : 2 * ip;
                                long qu = pu + s1, qv = pv + 2 * kk - s1;
                                const double *r0 = R_get(&cs, n + 1, pu, pv, j);
                                const double *t = T_get(&cs, n + 1, pu, pv, kk);
                                const double *r1 = R_get(&cs, n + 1, qu, qv, j);
                                const double *r1v = R_val(&cs, n + 1, qu, qv, j);
                                double Tt = t ? t[C] : 1.0;
                                if (r0) {
                                    double *gr = gR[n + 1] + R_index(&cs, n + 1, pu >> (n + 1), j, pv);
                                    for (int c = 0; c < C; ++c) gr[c] += 0.5 * g[c];
                                }
                                if (t) {
                                    double *gt = gT[n + 1] + T_index(&cs, n + 1, pu >> (n + 1), kk, pv);
                                    for (int c = 0; c < C; ++c) {
                                        gt[c] += 0.5 * A * g[c];
                                        gt[C] += 0.5 * g[c] * (r1v ? r1v[c] : 0.0);
                                    }
                                }
                                if (r1) {
                                    double *gr = gR[n + 1] + R_index(&cs, n + 1, qu >> (n + 1), j, qv);
                                    for (int c = 0; c < C; ++c) gr[c] += 0.5 * Tt * g[c];
                                }
                            }
                        }
                    }
        }
        /* reverse merge up: n = N .. 3 */
        for (int n = N; n >= 3; --n) {
            int m = n - 1;
            long sm = 1L << m, K = (1L << n) + 1;
            for (long x = 0; x < cs.Un[n]; ++x)
                for (long k = 0; k < K; ++k)
                    for (long y = 0; y < f.V; ++y) {
                        const double *g = gT[n] + T_index(&cs, n, x, k, y);
                        long pu = x << n, pv = y;
                        /* list of (weight, near, far) pairs */
                        long nk[2], fk[2], fv[2];
                        double wgt;
                        int npair;
                        if ((k & 1) == 0) {
                            npair = 1; wgt = 1.0;
                            nk[0] = k / 2; fk[0] = k / 2; fv[0] = pv + 2 * (k / 2) - sm;
                        } else {
                            long kp = (k + 1) / 2, km = (k - 1) / 2;
                            npair = 2; wgt = 0.5;
                            nk[0] = kp; fk[0] = km; fv[0] = pv + 2 * kp - sm;
                            nk[1] = km; fk[1] = kp; fv[1] = pv + 2 * km - sm;
                        }
                        for (int a = 0; a < npair; ++a) {
                            const double *nr = T_get(&cs, m, pu, pv, nk[a]);
                            const double *fr = T_get(&cs, m, pu + sm, fv[a], fk[a]);
                            double Tn = nr ? nr[C] : 1.0, Tf = fr ? fr[C] : 1.0;
                            if (nr) {
                                double *gn = gT[m] + T_index(&cs, m, pu >> m, nk[a], pv);
                                double gTn = g[C] * Tf;
                                for (int c = 0; c < C; ++c) {
                                    gn[c] += wgt * g[c];
                                    gTn += g[c] * (fr ? fr[c] : 0.0);
                                }
                                gn[C] += wgt * gTn;
                            }
                            if (fr) {
                                double *gf = gT[m] + T_index(&cs, m, (pu + sm) >> m, fk[a], fv[a]);
                                for (int c = 0; c < C; ++c) gf[c] += wgt * Tn * g[c];
                                gf[C] += wgt * Tn * g[C];
                            }
                        }
                    }
        }
        /* reverse trace of T_0 .. T_min(2,N) */
        double *gef = (double *)calloc((size_t)C * f.U * f.V, sizeof(double));
        double *gsf = (double *)calloc((size_t)f.U * f.V, sizeof(double));
        int ntrace = N < 2 ? N : 2;
        for (int n = 0; n <= ntrace; ++n) {
            long sn = 1L << n, K = sn + 1;
            for (long x = 0; x < cs.Un[n]; ++x)
                for (long k = 0; k < K; ++k)
                    for (long y = 0; y < f.V; ++y) {
                        const double *g = gT[n] + T_index(&cs, n, x, k, y);
                        double pu = x * sn + 0.5, pv = y + 0.5;
                        trace_adjoint(&f, pu, pv, pu + sn, pv + (2.0 * k - sn), g, g[C], gef, gsf);
                    }
        }
        for (long u = 0; u < f.U; ++u)
            for (long v = 0; v < f.V; ++v) {
                long x, y;
                frame_to_image(q, W, H, u, v, &x, &y);
                gs[y * W + x] += gsf[u * f.V + v];
                for (int c = 0; c < C; ++c)
                    ge[((size_t)c * H + y) * W + x] += gef[((size_t)c * f.U + u) * f.V + v];
            }
        free(gef); free(gsf);
        for (int n = 0; n <= N; ++n) { free(gT[n]); free(gR[n]); }
        cascades_free(&cs);
        frame_free(&f);
    }
}

void orc_fluence_adjoint(const double *e, const double *s, const double *gF, int C, int W, int H,
                         int cascades, double *ge, double *gs)
{
    adjoint_outside(e, s, gF, C, W, H, cascades, NULL, 0, NULL, 0, ge, gs);
}

void orc_fluence_adjoint_env(const double *e, const double *s, const double *gF, int C, int W, int H,
                             int cascades, const double *env, int M, double *ge, double *gs)
{
    adjoint_outside(e, s, gF, C, W, H, cascades, env, M, NULL, 0, ge, gs);
}

void orc_fluence_adjoint_top(const double *e, const double *s, const double *gF, int C, int W, int H,
                             int cascades, const double *top, int K, double *ge, double *gs)
{
    adjoint_outside(e, s, gF, C, W, H, cascades, NULL, 0, top, K, ge, gs);
}

/* Eq. 1 by brute force: F(p) = sum_m (2 pi / M) L_r(p <- p + D w(theta_m)),
 * theta_m = 2 pi (m + 1/2) / M, at every pixel centre, D past the grid.
 * The segment is clipped to the grid box first (outside is vacuum). */
void orc_bruteforce(const double *e, const double *s, int C, int W, int H, int M, double *F)
{
    Frame f = frame_build(0, e, s, C, W, H);
    double D = 2.0 * (W + H) + 4.0;
#pragma omp parallel for schedule(dynamic, 4)
    for (long y = 0; y < H; ++y) {
        double L[8], T;
        for (long x = 0; x < W; ++x) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            double pu = x + 0.5, pv = y + 0.5;
            for (int m = 0; m < M; ++m) {
                double th = 2.0 * M_PI * (m + 0.5) / M;
                double du = cos(th), dv = sin(th);
                /* exit parameter of the ray from the box [0,W] x [0,H] */
                double tmax = D;
                if (du > 0) tmax = fmin(tmax, (W - pu) / du);
                if (du < 0) tmax = fmin(tmax, (0 - pu) / du);
                if (dv > 0) tmax = fmin(tmax, (H - pv) / dv);
                if (dv < 0) tmax = fmin(tmax, (0 - pv) / dv);
                trace(&f, pu, pv, pu + tmax * du, pv + tmax * dv, L, &T);
                for (int c = 0; c < C; ++c) acc[c] += L[c];
            }
            for (int c = 0; c < C; ++c) F[((size_t)c * H + y) * W + x] = acc[c] * 2.0 * M_PI / M;
        }
    }
    frame_free(&f);
}

/* ---------------------------------------------------------------------------
 * Cross blur (Sec. 4.2, Eq. 21).  After the four quadrants are summed, each
 * pixel becomes the weighted mean of itself (weight 4) and its four edge
 * neighbours (weight 1 each), the 1/8 of Eq. 21, leaving out the neighbours
 * whose opacity differs significantly from the pixel's.  The paper gives no
 * measure or threshold; the reading used here: opacity is the absorptance of
 * one pixel length, alpha = 1 - exp(-sigma); a neighbour is kept iff it lies
 * inside the grid and |alpha_m - alpha_c| <= thr; the kept weights are
 * renormalised to sum to 1 (so the interior with every neighbour kept is
 * exactly Eq. 21).
 * ------------------------------------------------------------------------ */
static const int blur_dx[4] = {1, -1, 0, 0}, blur_dy[4] = {0, 0, 1, -1};

static int blur_keep(const double *s, int W, int H, long x, long y, long xm, long ym, double thr)
{
    if (xm < 0 || xm >= W || ym < 0 || ym >= H) return 0;
    double ac = 1.0 - exp(-s[y * W + x]);
    double am = 1.0 - exp(-s[ym * W + xm]);
    return fabs(am - ac) <= thr;
}

/* out = B F: the blurred image (F, out: [C][H][W]; s: [H][W]). */
void orc_cross_blur(const double *F, const double *s, int C, int W, int H, double thr, double *out)
{
    const double wc = 4.0;
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double wsum = wc;
            double acc[8];
            for (int c = 0; c < C; ++c) acc[c] = wc * F[((size_t)c * H + y) * W + x];
            for (int d = 0; d < 4; ++d) {
                long xm = x + blur_dx[d], ym = y + blur_dy[d];
                if (!blur_keep(s, W, H, x, y, xm, ym, thr)) continue;
                wsum += 1.0;
                for (int c = 0; c < C; ++c) acc[c] += F[((size_t)c * H + ym) * W + xm];
            }
            for (int c = 0; c < C; ++c) out[((size_t)c * H + y) * W + x] = acc[c] / wsum;
        }
}

/* gF = B^T g, the adjoint of the blur for fixed s, by scattering each
 * output pixel's weights back onto the pixels it read.  The kept set depends
 * on s only through the threshold test, which is piecewise constant, so the
 * blur contributes nothing to dL/dsigma (away from the measure-zero set where
 * a pair sits exactly at the threshold). */
void orc_cross_blur_adjoint(const double *g, const double *s, int C, int W, int H, double thr, double *gF)
{
    memset(gF, 0, sizeof(double) * (size_t)C * W * H);
    for (long y = 0; y < H; ++y)
        for (long x = 0; x < W; ++x) {
            double wsum = 4.0;
            for (int d = 0; d < 4; ++d)
                wsum += blur_keep(s, W, H, x, y, x + blur_dx[d], y + blur_dy[d], thr) ? 1.0 : 0.0;
            for (int c = 0; c < C; ++c) {
                const double gc = g[((size_t)c * H + y) * W + x] / wsum;
                gF[((size_t)c * H + y) * W + x] += 4.0 * gc;
                for (int d = 0; d < 4; ++d) {
                    long xm = x + blur_dx[d], ym = y + blur_dy[d];
                    if (!blur_keep(s, W, H, x, y, xm, ym, thr)) continue;
                    gF[((size_t)c * H + ym) * W + xm] += gc;
                }
            }
        }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
