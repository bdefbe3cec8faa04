/*
 * Plain CPU oracle for Refined Random Search (RRS) projection depths.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header or constant table with
 * the CUDA sources: both implement the same written direction-stream formula
 * independently.
 *
 * What it computes (paper: "Massive parallelization of projection-based
 * depths", arXiv 2506.08262):
 *   - univariate depths of Sec. 2: halfspace D_H, projection D_P and
 *     asymmetric projection D_AP, in FP64 (halfspace signs exactly);
 *   - the refined random search of Alg. 1 / Alg. S3: r rounds of
 *     m = ceil(k/r) directions, round minimum and its direction, strict-<
 *     update of the running minimum and of the pole, cap shrink by alpha;
 *   - directions: Alg. S1 (normalised Gaussian vector) for round 1 and
 *     Alg. S4 (angle in the cap, Gaussian remainder, reflection of e1 onto
 *     the pole) for later rounds, in FP32 with a fixed operation order, drawn
 *     from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
 *
 * Readings of the paper (each also listed in the design notes):
 *   R1 round 1 is uniform on the whole sphere (Alg. S1), not the hemisphere
 *      of Alg. S3: the symmetry used for the hemisphere (Supp. A) fails for
 *      D_AP.  Later rounds use the cap angle (pi/2) * alpha^(l-1).
 *   R2 the garbled reflection of Alg. S4 is read as the Householder map
 *      H = I - 2 v v^T / (v^T v), v = e1 - p, which sends e1 to p; the paper's
 *      lambda equals -2 v^T u / (v^T v) when |p| = 1.  v^T v is formed as a
 *      sum of squares.  If v = 0 the map is the identity.
 *   R3 the remaining coordinates of a cap direction are sin(theta) * g/|g|
 *      (Alg. S4 writes sqrt(1 - u1^2), equal in exact arithmetic).
 *   R4 median of an even count is the mean of the two middle order
 *      statistics; MAD is unscaled; MAD_+ is the median of y_i - med over
 *      y_i > med (strict); a zero MAD (or MAD_+) gives depth 1 when the
 *      numerator is 0 and 0 otherwise; an empty positive set gives MAD_+ = 0.
 *   R5 if no direction ever beats the initial minimum (1, i.e. count n), the
 *      pole stays e1 and the best index is -1.
 *   R6 m = ceil(k/r) (Alg. S5 prints k/m).
 *
 * Direction stream (the written formula both sides implement):
 *   key = (seed mod 2^32, seed >> 32); counter = (b, j, l-1, q) with b the
 *   4-word block index, j the direction in the round, l the round (1-based)
 *   and q the query index within the call.
 *   unif(w) = float(2*(w >> 9) + 1) * 2^-24, in (0, 1).
 *   Gaussian i: block i/4, word pair (2p, 2p+1) with p = (i/2) mod 2;
 *     U = unif(w_2p), V = unif(w_2p+1), R = sqrt(-2 ln U),
 *     g = R cos(2 pi V) if i even, R sin(2 pi V) if i odd.
 *   ln and sin/cos are the polynomials below (atanh series; Taylor series
 *   on [-pi/4, pi/4] after an exact quarter-turn reduction), evaluated in
 *   FP32 with round-to-nearest, one rounding per written operation (no
 *   fused multiply-add), so that every direction is bit-identical on any
 *   IEEE-754 machine.
 *   Round 1: u = g / sqrt(sum g_i^2) over i = 0..d-1.
 *   Round l >= 2: a = alpha^(l-1) by repeated FP32 products, theta in
 *     quarter turns t = unif(w_0 of block 0xFFFFFFFF) * a;
 *     u~ = (cos, sin * g'/|g'|) with g' the first d-1 Gaussians; u = H u~.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { KIND_HALFSPACE = 0, KIND_PROJECTION = 1, KIND_ASYM = 2 };

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

void rrs_oracle_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static float unif01(uint32_t w)
{
    uint32_t odd = 2u * (w >> 9) + 1u; /* < 2^24: exact in float */
    return (float)odd * 0x1p-24f;
}

/* ln(a) for a in (0, 1]: a = 2^e f with f in [sqrt(1/2), sqrt(2)],
 * ln f = 2 atanh(s), s = (f-1)/(f+1), series up to s^13. */
float rrs_oracle_logf(float a)
{
    uint32_t bits;
    memcpy(&bits, &a, 4);
    int e = (int)((bits >> 23) & 0xFFu) - 127;
    uint32_t fbits = (bits & 0x007FFFFFu) | 0x3F800000u;
    float f;
    memcpy(&f, &fbits, 4);
    if (f > 1.41421356f) {
        f = f * 0.5f;
        e = e + 1;
    }
    float s = (f - 1.0f) / (f + 1.0f);
    float z = s * s;
    float p = 1.0f / 13.0f;
    p = p * z + 1.0f / 11.0f;
    p = p * z + 1.0f / 9.0f;
    p = p * z + 1.0f / 7.0f;
    p = p * z + 1.0f / 5.0f;
    p = p * z + 1.0f / 3.0f;
    float t = 2.0f * s;
    float w = z * p;
    w = t * w;
    float lnf = t + w;
    float ef = (float)e;
    float hi = ef * 0.693145751953125f;   /* ln 2, leading 16 bits */
    float lo = ef * 1.42860682e-06f;      /* ln 2 - leading part */
    return hi + (lo + lnf);
}

/* sin and cos of (pi/2) * a, for a in [0, 4) quarter turns. */
void rrs_oracle_sincos_qturn(float a, float* s_out, float* c_out)
{
    int q = (int)a;
    float r = a - (float)q;
    if (r > 0.5f) {
        r = r - 1.0f;
        q = q + 1;
    }
    float x = r * 1.57079637f;
    float z = x * x;
    float ps = 1.0f / 362880.0f;
    ps = ps * z + -(1.0f / 5040.0f);
    ps = ps * z + 1.0f / 120.0f;
    ps = ps * z + -(1.0f / 6.0f);
    float ws = z * ps;
    ws = x * ws;
    float sx = x + ws;
    float pc = -(1.0f / 3628800.0f);
    pc = pc * z + 1.0f / 40320.0f;
    pc = pc * z + -(1.0f / 720.0f);
    pc = pc * z + 1.0f / 24.0f;
    pc = pc * z + -0.5f;
    float wc = z * pc;
    float cx = 1.0f + wc;
    switch (q & 3) {
    case 0: *s_out = sx;  *c_out = cx;  break;
    case 1: *s_out = cx;  *c_out = -sx; break;
    case 2: *s_out = -sx; *c_out = -cx; break;
    default: *s_out = -cx; *c_out = sx; break;
    }
}

typedef struct {
    uint32_t key[2];
    uint32_t j, round0, q;
    uint32_t cached_block;
    uint32_t words[4];
    int have;
} gauss_stream;

static void gs_init(gauss_stream* g, uint64_t seed, uint32_t q, uint32_t round0, uint32_t j)
{
    g->key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
    g->key[1] = (uint32_t)(seed >> 32);
    g->j = j; g->round0 = round0; g->q = q;
    g->have = 0;
}

static void gs_block(gauss_stream* g, uint32_t b, uint32_t out[4])
{
    if (g->have && g->cached_block == b) {
        memcpy(out, g->words, sizeof g->words);
        return;
    }
    uint32_t ctr[4] = { b, g->j, g->round0, g->q };
    rrs_oracle_philox(ctr, g->key, g->words);
    g->cached_block = b;
    g->have = 1;
    memcpy(out, g->words, sizeof g->words);
}

static float gs_gaussian(gauss_stream* g, uint32_t i)
{
    uint32_t w[4];
    gs_block(g, i >> 2, w);
    uint32_t p = (i >> 1) & 1u;
    float U = unif01(w[2 * p]);
    float V = unif01(w[2 * p + 1]);
    float R = sqrtf(-2.0f * rrs_oracle_logf(U));
    float s, c;
    rrs_oracle_sincos_qturn(4.0f * V, &s, &c);
    return (i & 1u) ? R * s : R * c;
}

/* One direction (Alg. S1 for round 1, Alg. S4 with readings R2/R3 after). */
static void direction(uint64_t seed, uint32_t q, uint32_t round0, uint32_t j, int d,
                      float alpha, const float* pole, float* u)
{
    gauss_stream gs;
    gs_init(&gs, seed, q, round0, j);
    if (round0 == 0) {
        float s2 = 0.0f;
        for (int i = 0; i < d; ++i) {
            u[i] = gs_gaussian(&gs, (uint32_t)i);
            s2 = s2 + u[i] * u[i];
        }
        float nrm = sqrtf(s2);
        for (int i = 0; i < d; ++i) u[i] = u[i] / nrm;
        return;
    }
    float a = 1.0f;
    for (uint32_t t = 0; t < round0; ++t) a = a * alpha;
    uint32_t wcap[4];
    gs_block(&gs, 0xFFFFFFFFu, wcap);
    float t = unif01(wcap[0]) * a;
    float st, ct;
    rrs_oracle_sincos_qturn(t, &st, &ct);
    u[0] = ct;
    if (d > 1) {
        float s2 = 0.0f;
        for (int i = 0; i < d - 1; ++i) {
            u[i + 1] = gs_gaussian(&gs, (uint32_t)i);
            s2 = s2 + u[i + 1] * u[i + 1];
        }
        float nrm = sqrtf(s2);
        for (int i = 1; i < d; ++i) {
            float h = u[i] / nrm;
            u[i] = st * h;
        }
    }
    /* Householder reflection sending e1 to the pole. */
    float vv = 0.0f, vu = 0.0f;
    for (int i = 0; i < d; ++i) {
        float v = (i == 0) ? (1.0f - pole[0]) : -pole[i];
        vv = vv + v * v;
    }
    if (vv == 0.0f) return;
    for (int i = 0; i < d; ++i) {
        float v = (i == 0) ? (1.0f - pole[0]) : -pole[i];
        vu = vu + v * u[i];
    }
    float lam = (2.0f * vu) / vv;
    for (int i = 0; i < d; ++i) {
        float v = (i == 0) ? (1.0f - pole[0]) : -pole[i];
        u[i] = u[i] - lam * v;
    }
}

/* m directions of round `round0` (0-based) for query q into U (m x d). */
int rrs_oracle_directions(uint64_t seed, int32_t q, int32_t round0, int32_t m, int32_t d,
                          float alpha, const float* pole, float* U)
{
    if (m < 0 || d < 1 || q < 0 || round0 < 0) return -1;
    for (int j = 0; j < m; ++j)
        direction(seed, (uint32_t)q, (uint32_t)round0, (uint32_t)j, d, alpha, pole, U + (size_t)j * d);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact sign of u^T (x - z)  (halfspace counts, Sec. 2)                     */
/* ------------------------------------------------------------------------ */

static void two_sum(double a, double b, double* s, double* e)
{
    double x = a + b;
    double bv = x - a;
    double av = x - bv;
    *s = x;
    *e = (a - av) + (b - bv);
}

/* Shewchuk's grow-expansion: add b to the nonoverlapping expansion h. */
static int grow_expansion(double* h, int hlen, double b)
{
    double q = b;
    for (int i = 0; i < hlen; ++i) {
        double s, e;
        two_sum(q, h[i], &s, &e);
        h[i] = e;
        q = s;
    }
    h[hlen] = q;
    return hlen + 1;
}

/* Returns -1, 0 or +1.  scratch must hold 4*d+1 doubles. */
static int exact_sign(const float* u, const double* x, const double* z, int d, double* scratch)
{
    double a = 0.0, b = 0.0, mag = 0.0;
    for (int l = 0; l < d; ++l) {
        double ul = (double)u[l];
        a = a + ul * x[l];
        b = b + ul * z[l];
        mag = mag + fabs(ul) * (fabs(x[l]) + fabs(z[l]));
    }
    double t = a - b;
    /* forward bound for two FP64 dot products and one subtraction, with slack */
    double bound = (double)(2 * d + 8) * 0x1p-53 * mag * (1.0 + 0x1p-40);
    if (t > bound) return 1;
    if (t < -bound) return -1;
    /* exact: each product u*x is p + e exactly (fma), summed without error */
    int len = 0;
    for (int l = 0; l < d; ++l) {
        double ul = (double)u[l];
        double p = ul * x[l];
        double e = fma(ul, x[l], -p);
        len = grow_expansion(scratch, len, p);
        len = grow_expansion(scratch, len, e);
        p = ul * z[l];
        e = fma(ul, z[l], -p);
        len = grow_expansion(scratch, len, -p);
        len = grow_expansion(scratch, len, -e);
    }
    for (int i = len - 1; i >= 0; --i) {
        if (scratch[i] > 0.0) return 1;
        if (scratch[i] < 0.0) return -1;
    }
    return 0;
}

int rrs_oracle_sign(const float* u, const double* x, const double* z, int32_t d)
{
    double* scratch = (double*)malloc(sizeof(double) * (size_t)(4 * d + 1));
    if (!scratch) return -2;
    int s = exact_sign(u, x, z, d, scratch);
    free(scratch);
    return s;
}

/* ------------------------------------------------------------------------ */
/* Univariate depths (Sec. 2)                                                */
/* ------------------------------------------------------------------------ */

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

static double median_sorted(const double* v, int64_t len)
{
    if (len % 2 == 1) return v[(len - 1) / 2];
    return (v[len / 2 - 1] + v[len / 2]) / 2.0;
}

typedef struct {
    double* y;        /* n */
    double* dev;      /* n */
    double* scratch;  /* 4d+1 */
} workspace;

/* Depth of z along u.  For the halfspace kind *count_out receives
 * min(#{u'x <= u'z}, #{u'x >= u'z}). */
static double univariate(int kind, const double* X, int64_t n, int d, const double* z,
                         const float* u, workspace* ws, int64_t* count_out)
{
    if (kind == KIND_HALFSPACE) {
        int64_t lt = 0, gt = 0;
        for (int64_t i = 0; i < n; ++i) {
            int s = exact_sign(u, X + (size_t)i * d, z, d, ws->scratch);
            if (s < 0) ++lt;
            else if (s > 0) ++gt;
        }
        int64_t le = n - gt, ge = n - lt;
        int64_t c = le < ge ? le : ge;
        if (count_out) *count_out = c;
        return (double)c / (double)n;
    }
    double yz = 0.0;
    for (int l = 0; l < d; ++l) yz = yz + (double)u[l] * z[l];
    for (int64_t i = 0; i < n; ++i) {
        const double* x = X + (size_t)i * d;
        double acc = 0.0;
        for (int l = 0; l < d; ++l) acc = acc + (double)u[l] * x[l];
        ws->y[i] = acc;
    }
    qsort(ws->y, (size_t)n, sizeof(double), cmp_double);
    double med = median_sorted(ws->y, n);
    if (count_out) *count_out = -1;
    if (kind == KIND_PROJECTION) {
        for (int64_t i = 0; i < n; ++i) ws->dev[i] = fabs(ws->y[i] - med);
        qsort(ws->dev, (size_t)n, sizeof(double), cmp_double);
        double mad = median_sorted(ws->dev, n);
        double num = fabs(yz - med);
        if (mad == 0.0) return num == 0.0 ? 1.0 : 0.0;
        return 1.0 / (1.0 + num / mad);
    }
    /* asymmetric: y is sorted, so the positive deviations are a suffix */
    int64_t first = 0;
    while (first < n && !(ws->y[first] > med)) ++first;
    int64_t npos = n - first;
    double madp = 0.0;
    if (npos > 0) {
        for (int64_t i = 0; i < npos; ++i) ws->dev[i] = ws->y[first + i] - med;
        madp = median_sorted(ws->dev, npos);
    }
    double num = yz - med > 0.0 ? yz - med : 0.0;
    if (madp == 0.0) return num == 0.0 ? 1.0 : 0.0;
    return 1.0 / (1.0 + num / madp);
}

static int ws_alloc(workspace* ws, int64_t n, int d)
{
    ws->y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ws->dev = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ws->scratch = (double*)malloc(sizeof(double) * (size_t)(4 * d + 1));
    return (ws->y && ws->dev && ws->scratch) ? 0 : -2;
}

static void ws_free(workspace* ws)
{
    free(ws->y); free(ws->dev); free(ws->scratch);
}

int rrs_oracle_univariate(int32_t kind, const double* X, int64_t n, int32_t d, const double* z,
                          const float* u, double* depth_out, int64_t* count_out)
{
    if (n < 1 || d < 1 || kind < 0 || kind > 2) return -1;
    workspace ws;
    if (ws_alloc(&ws, n, d)) { ws_free(&ws); return -2; }
    *depth_out = univariate(kind, X, n, d, z, u, &ws, count_out);
    ws_free(&ws);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Refined random search (Alg. 1 / Alg. S3)                                  */
/* ------------------------------------------------------------------------ */

/*
 * For each query: D_min = 1 (count n), pole e1; for round l = 1..r draw m
 * directions, take their depths, the round minimum and its lowest index
 * j*, and if it is strictly below D_min update D_min, the pole and the best
 * flat index (l-1)*m + j*.
 *
 * follow (optional, nq*r): replay another implementation's pole updates.
 * Entry >= 0 is the direction that implementation took as the new pole in
 * that round, -1 means it kept the pole.  The depths are still the
 * oracle's own.  round_min/round_arg (optional, nq*r) receive the oracle's
 * round minimum and argmin; round_at_follow (optional) the oracle's depth at
 * the followed index (NaN where follow is -1).
 * qidx (optional, nq) gives the query counter index of each row (default:
 * the row number).
 */
int rrs_oracle_rrs(const double* X, int64_t n, int32_t d, const double* Z, int64_t nq,
                   const int64_t* qidx, int32_t kind, int32_t k, int32_t r, double alpha,
                   uint64_t seed, const int32_t* follow, double* depth_out, int64_t* count_out,
                   int32_t* best_out, double* round_min, int32_t* round_arg,
                   double* round_at_follow, int32_t nthreads)
{
    if (n < 1 || d < 1 || nq < 0 || kind < 0 || kind > 2 || r < 1 || k < r || !(alpha > 0.0) ||
        alpha > 1.0)
        return -1;
    const int32_t m = (k + r - 1) / r;
    const float alpha_f = (float)alpha;
    int err = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(| : err)
#endif
    for (int64_t qi = 0; qi < nq; ++qi) {
        workspace ws;
        float* U = (float*)malloc(sizeof(float) * (size_t)m * d);
        float* pole = (float*)malloc(sizeof(float) * (size_t)d);
        double* Dj = (double*)malloc(sizeof(double) * (size_t)m);
        int64_t* Cj = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
        if (ws_alloc(&ws, n, d) || !U || !pole || !Dj || !Cj) {
            err |= 1;
        } else {
            const double* z = Z + (size_t)qi * d;
            uint32_t qc = (uint32_t)(qidx ? qidx[qi] : qi);
            for (int i = 0; i < d; ++i) pole[i] = 0.0f;
            pole[0] = 1.0f;
            double dmin = 1.0;
            int64_t cmin = n;
            int32_t best = -1;
            for (int32_t l = 0; l < r; ++l) {
                for (int32_t j = 0; j < m; ++j) {
                    direction(seed, qc, (uint32_t)l, (uint32_t)j, d, alpha_f, pole, U + (size_t)j * d);
                    Dj[j] = univariate(kind, X, n, d, z, U + (size_t)j * d, &ws, &Cj[j]);
                }
                int32_t ja = 0;
                for (int32_t j = 1; j < m; ++j) {
                    int better = (kind == KIND_HALFSPACE) ? (Cj[j] < Cj[ja]) : (Dj[j] < Dj[ja]);
                    if (better) ja = j;
                }
                size_t slot = (size_t)qi * r + l;
                if (round_min) round_min[slot] = Dj[ja];
                if (round_arg) round_arg[slot] = ja;
                int32_t take = -1;
                if (follow) {
                    take = follow[slot];
                    if (round_at_follow) round_at_follow[slot] = take >= 0 && take < m ? Dj[take] : NAN;
                    if (take >= m) take = -1;
                } else {
                    int improves = (kind == KIND_HALFSPACE) ? (Cj[ja] < cmin) : (Dj[ja] < dmin);
                    if (improves) take = ja;
                }
                if (take >= 0) {
                    dmin = Dj[take];
                    cmin = Cj[take];
                    best = l * m + take;
                    memcpy(pole, U + (size_t)take * d, sizeof(float) * (size_t)d);
                }
            }
            depth_out[qi] = dmin;
            if (count_out) count_out[qi] = (kind == KIND_HALFSPACE) ? cmin : -1;
            if (best_out) best_out[qi] = best;
        }
        ws_free(&ws);
        free(U); free(pole); free(Dj); free(Cj);
    }
    return err ? -2 : 0;
}

int rrs_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
