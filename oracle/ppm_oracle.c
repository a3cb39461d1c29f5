/*
 * ppm_oracle.c -- CPU oracle for hypothesis-tested progressive kernel
 * estimation (FPPM / VCM+ merge path).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU path computes.  Only tests/, the smoke check in
 * __graft_entry__ and the cpu_baseline / reference arm of bench.py may load
 * it.  The product library never links or calls it, and it shares no code,
 * header, table or constant generator with the CUDA sources.
 *
 * Precision: every statistic is FP64 (two-pass ANOVA over all m samples of a
 * group, zeros included).  The per-pair geometric decisions (disk test,
 * annulus, sector) are taken in a fixed FP32 operation sequence, because a
 * floating-point comparison decides an integer there and both sides must
 * take it in the same precision.  Compile with -ffp-contract=off: the only
 * fused multiply-adds are the explicit fmaf() calls below.
 *
 * Paper: "Hypothesis Testing for Progressive Kernel Estimation and VCM
 * Framework" (Lin, Hu, Jia, Li).  Each function cites the section or
 * equation it restates.
 *
 * Parity pins (tests/test_oracle_pins.py): F critical values against closed
 * forms (F(1,d)=t^2, F(2,d), F(d,2)), the chi-square limit 24.725/11 printed
 * in Sec. 6.1.1 and scipy; the ANOVA F against scipy.stats.f_oneway on full
 * sample tables and against the exact value F=1 for a single nonzero sample;
 * classification against FP64 atan2 geometry and brute-force area fractions;
 * the estimate against the analytic constant-irradiance plane; the rejection
 * rate against alpha_F; the radius update against Eq. (radiusupdate).  The
 * chi-square test of CPPM: its critical value against the closed form
 * -2 ln(alpha) of two degrees of freedom, the 24.724 printed in Sec. 6.1.1
 * and scipy; the statistic against scipy.stats.chisquare; its rejection rate
 * against alpha; its blindness to a zero-flux shadow edge (Sec. 3.2.3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NA 2            /* equi-areal annuli, Sec. 6.1.1 */
#define OR_NS 6            /* equi-areal sectors per annulus, Sec. 6.1.1 */
#define OR_NG (OR_NA * OR_NS)

/* ------------------------------------------------------------------------
 * 1. F distribution (Sec. 3.2.2): the critical value F_c is the (1-alpha_F)
 *    quantile of F(d1, d2) with d1 = n-1 and d2 = n(m-1).
 *
 *    CDF_F(f; d1, d2) = I_x(d1/2, d2/2), x = d1 f / (d1 f + d2), where I is
 *    the regularized incomplete beta function.  I is evaluated from its
 *    hypergeometric series (DLMF Sec. 8.17(ii)):
 *        I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * 2F1(a+b, 1; a+1; x)
 *                 = x^a (1-x)^b / (a B(a,b)) * sum_{j>=0} (a+b)_j / (a+1)_j x^j,
 *    ((q)_j the rising factorial), whose terms are all positive: no
 *    cancellation.  The sum is taken on the side of the symmetry
 *    I_x(a,b) = 1 - I_{1-x}(b,a) where its terms fall off fastest: the
 *    direct side below x = (a+1)/(a+b+2), and always when b >> a (there x is
 *    tiny, the direct terms behave like (b x)^j / j!, and the other side's
 *    ratio tends to 1 - x ~ 1).  The series and the log-Beta prefactor are
 *    taken in quadruple precision (binary128: long double on aarch64,
 *    __float128 on x86-64) because lgamma(b) and lgamma(a+b) are ~1e11 at
 *    the sample sizes of this method.  The quantile is found by plain
 *    bisection on the CDF.
 * ---------------------------------------------------------------------- */
#if defined(__x86_64__)
#include <quadmath.h>
typedef __float128 or_quad;
#define OR_LGAMMA lgammaq
#define OR_LOG logq
#define OR_LOG1P log1pq
#define OR_EXP expq
#else
typedef long double or_quad;
#define OR_LGAMMA lgammal
#define OR_LOG logl
#define OR_LOG1P log1pl
#define OR_EXP expl
#endif

/* I_x(a,b) by the series above, on the side the caller chose (0 < x < 1) */
static double or_beta_series(double a, double b, double x)
{
    const or_quad qa = a, qb = b, qx = x;
    or_quad term = 1, sum = 1;
    for (int j = 0; j < 10000000; ++j) {
        term *= (qa + qb + j) / (qa + 1 + j) * qx;
        sum += term;
        if (term < sum * (or_quad)1e-34) break;
    }
    const or_quad lnB = OR_LGAMMA(qa) + OR_LGAMMA(qb) - OR_LGAMMA(qa + qb);
    const or_quad ln = qa * OR_LOG(qx) + qb * OR_LOG1P(-qx) - lnB - OR_LOG(qa) + OR_LOG(sum);
    return (double)OR_EXP(ln);
}

double oracle_betainc(double a, double b, double x)
{
    if (x <= 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    if (x < (a + 1.0) / (a + b + 2.0) || b > 50.0 * a)
        return or_beta_series(a, b, x);
    return 1.0 - or_beta_series(b, a, 1.0 - x);
}

double oracle_f_cdf(double d1, double d2, double f)
{
    if (f <= 0.0) return 0.0;
    double x = d1 * f / (d1 * f + d2);
    return oracle_betainc(0.5 * d1, 0.5 * d2, x);
}

double oracle_f_crit(double d1, double d2, double alpha)
{
    double target = 1.0 - alpha, lo = 0.0, hi = 1.0;
    while (oracle_f_cdf(d1, d2, hi) < target) { lo = hi; hi *= 2.0; }
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (oracle_f_cdf(d1, d2, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------
 * 1b. The chi-square test that CPPM uses (Sec. 3.2.3; settings in Sec.
 *     6.1.1): are the in-disk photons spread evenly over the n equi-areal
 *     groups?  It looks at the counts c_g only, not at what the photons
 *     carry.  Statistic: Pearson's X^2 = sum_g (c_g - E)^2 / E with
 *     E = C / n and C = sum_g c_g; a disk without photons gives X^2 = 0 (no
 *     evidence against uniformity).  Critical value chi_c: the (1 - alpha)
 *     quantile of chi^2(n - 1), whose CDF is P(k/2, x/2) with P the
 *     regularized lower incomplete gamma function.  P comes from its power
 *     series
 *         P(a, z) = z^a e^-z / Gamma(a + 1) * sum_{j >= 0} z^j / ((a+1)...(a+j)),
 *     whose terms are all positive (no cancellation), summed in binary128.
 *     The quantile is found by plain bisection on the CDF.
 * ---------------------------------------------------------------------- */
double oracle_chi2_cdf(double k, double x)
{
    if (x <= 0.0) return 0.0;
    const or_quad a = (or_quad)k / 2, z = (or_quad)x / 2;
    or_quad term = 1, sum = 1;
    for (int j = 1; j < 100000; ++j) {
        term *= z / (a + j);
        sum += term;
        if (term < sum * (or_quad)1e-33) break;
    }
    const or_quad lp = a * OR_LOG(z) - z - OR_LGAMMA(a + 1) + OR_LOG(sum);
    return (double)OR_EXP(lp);
}

double oracle_chi2_crit(double k, double alpha)
{
    double target = 1.0 - alpha, lo = 0.0, hi = 1.0;
    while (oracle_chi2_cdf(k, hi) < target) { lo = hi; hi *= 2.0; }
    for (int it = 0; it < 2000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (oracle_chi2_cdf(k, mid) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

double oracle_chi2_counts(int n, const int64_t* counts)
{
    int64_t C = 0;
    for (int g = 0; g < n; ++g) C += counts[g];
    if (C == 0) return 0.0;
    const double E = (double)C / n;
    double x2 = 0.0;
    for (int g = 0; g < n; ++g) {
        const double d = (double)counts[g] - E;
        x2 += d * d / E;
    }
    return x2;
}

/* ------------------------------------------------------------------------
 * 2. One-way ANOVA F statistic, Eq. (f-statistic), two passes, FP64.
 *    Group g holds m samples: the c_g stored values vals[off_g .. off_g+c_g)
 *    plus m - c_g implicit zeros (Sec. 3.2.1: one light sub-path gives one
 *    sample to every sector; the sectors it does not reach get a zero).
 *    Returns F; *ssw_out receives the within-group sum of squares.
 * ---------------------------------------------------------------------- */
double oracle_anova_f(int n, double m, const int64_t* counts,
                      const double* vals, double* ssw_out)
{
    double total = 0.0, mean_g[64], ssb = 0.0, ssw = 0.0;
    int64_t off = 0;
    if (n > 64) return -1.0;
    /* pass 1: group means and grand mean over all n*m samples */
    for (int g = 0; g < n; ++g) {
        double s = 0.0;
        for (int64_t j = 0; j < counts[g]; ++j) s += vals[off + j];
        mean_g[g] = s / m;
        total += s;
        off += counts[g];
    }
    double grand = total / (n * m);
    /* pass 2: deviations */
    off = 0;
    for (int g = 0; g < n; ++g) {
        double dev = mean_g[g] - grand;
        ssb += m * dev * dev;
        for (int64_t j = 0; j < counts[g]; ++j) {
            double e = vals[off + j] - mean_g[g];
            ssw += e * e;
        }
        ssw += (m - (double)counts[g]) * mean_g[g] * mean_g[g];
        off += counts[g];
    }
    if (ssw_out) *ssw_out = ssw;
    if (ssw <= 0.0) return 0.0;
    return (ssb / (n - 1)) / (ssw / (n * (m - 1.0)));
}

/* ------------------------------------------------------------------------
 * 3. Per-pair classification in the unified 2D space.
 *    - same-surface filter (the paper is silent; standard photon-mapping
 *      normal check): integer dot of the two snorm8-packed normals > 8064,
 *      i.e. cosine > ~1/2; skipped when either side has no normals;
 *    - disk test (kernel support, Eq. kaplanyan-integral): closed disk,
 *      d2 = fma(dz,dz, fma(dy,dy, dx*dx)) <= r*r, dx = x_h - x_p;
 *    - map to the unified space, Eq. (map-function):
 *      y_u = <x_h - x_p, u>, y_v = <x_h - x_p, v>;
 *    - two equi-areal annuli (Sec. 3.2.1 / 6.1.1): inner iff 2 rho^2 < r^2;
 *    - six equi-areal 60-degree sectors by exact sign logic against
 *      sqrt(3) = 1.7320508f (tan 60 degrees).
 *    Returns the group 0..11 (annulus * 6 + sector) or -1 if not gathered.
 * ---------------------------------------------------------------------- */
static int or_s8(uint32_t q, int byte)
{
    int v = (int)((q >> (8 * byte)) & 0xffu);
    return v >= 128 ? v - 256 : v;
}

int oracle_normal_dot(uint32_t a, uint32_t b)
{
    return or_s8(a, 0) * or_s8(b, 0) + or_s8(a, 1) * or_s8(b, 1)
         + or_s8(a, 2) * or_s8(b, 2) + or_s8(a, 3) * or_s8(b, 3);
}

int oracle_classify(const float* xh, const float* u, const float* v,
                    float r, const float* xp,
                    int use_normals, uint32_t nq_h, uint32_t nq_p)
{
    if (use_normals && oracle_normal_dot(nq_h, nq_p) <= 8064) return -1;
    float dx = xh[0] - xp[0], dy = xh[1] - xp[1], dz = xh[2] - xp[2];
    float r2 = r * r;
    float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if (!(d2 <= r2)) return -1;
    float yu = fmaf(dz, u[2], fmaf(dy, u[1], dx * u[0]));
    float yv = fmaf(dz, v[2], fmaf(dy, v[1], dx * v[0]));
    float rho2 = fmaf(yv, yv, yu * yu);
    int ring = ((rho2 + rho2) < r2) ? 0 : 1;
    float ax = fabsf(yu), ay = fabsf(yv);
    float tx = 1.7320508f * ax;
    int up = (yv > 0.0f) || (yv == 0.0f && yu >= 0.0f);
    int sector;
    if (ay >= tx) sector = up ? 1 : 4;
    else if (up)  sector = (yu > 0.0f) ? 0 : 2;
    else          sector = (yu < 0.0f) ? 3 : 5;
    return ring * OR_NS + sector;
}

/* ------------------------------------------------------------------------
 * 4. Radius update, Eq. (radiusupdate): after iteration i, a rejected radius
 *    becomes max(k r_i, r_min sqrt((i+1)^(alpha-1))).  The bound is a
 *    per-iteration scalar, evaluated in FP64 and rounded to FP32; the radius
 *    itself is FP32 state.
 * ---------------------------------------------------------------------- */
float oracle_radius_bound(float r_min, float alpha, int i)
{
    return (float)((double)r_min * sqrt(pow((double)i + 1.0, (double)alpha - 1.0)));
}

float oracle_shrink(float r, float k, float bound)
{
    float kr = k * r;
    return kr > bound ? kr : bound;
}

/* ------------------------------------------------------------------------
 * 5. VCM+ merge weight, balance heuristic (beta = 1), Eq. (mis-weight):
 *    dividing numerator and denominator by n_VM p_VM of the technique that
 *    produced the pair gives w = 1 / (1 + R_VM + R_VC / eta) with
 *    eta = n_VM pi r^2 (p_VM is proportional to r^2, p_VC independent of r).
 *    R_VM = rho_vm_h cos_l / pi + rho_vm_l (other merge techniques),
 *    R_VC = rho_vc_h + rho_vc_l (connection techniques), cos_l = max(0,
 *    n_h . w_l) from the snorm8-packed incoming direction of the light
 *    vertex.  The rho are synthetic r-independent pdf ratios given as input.
 * ---------------------------------------------------------------------- */
double oracle_mis_weight(double rho_vm_h, double rho_vc_h, double rho_vm_l,
                         double rho_vc_l, int cos_dot, double n_vm, double r)
{
    double cosl = cos_dot > 0 ? (double)cos_dot / (127.0 * 127.0) : 0.0;
    double r_vm = rho_vm_h * cosl / M_PI + rho_vm_l;
    double r_vc = rho_vc_h + rho_vc_l;
    double eta = n_vm * M_PI * r * r;
    return 1.0 / (1.0 + r_vm + r_vc / eta);
}

/* Luminance of an RGB flux (Rec. 709 weights; the paper tests luminance by
 * default, Sec. 5.1, without stating the weights). */
static double or_lum(double R, double G, double B)
{
    return 0.2126 * R + 0.7152 * G + 0.0722 * B;
}

double oracle_lum(double R, double G, double B)
{
    return or_lum(R, G, B);
}

/* ------------------------------------------------------------------------
 * 6. The full method, brute force over all pairs (Sec. 5.1, steps 1-5, with
 *    the estimate of Eq. progressive-VCM-estimator).  For every iteration
 *    i = i0 .. i0+iters-1 and every hit point h:
 *      a. classify every photon of the iteration (section 3 above);
 *      b. append (group, psi) of each gathered photon to the window of h;
 *         psi = luminance (or one RGB channel) of w * Phi;
 *      c. tau_h += sum(w * Phi) / (pi r^2) with the radius of this iteration;
 *      d. m = t' J with t' = t+1 iterations in the window; two-pass ANOVA F
 *         per tested channel; F_c from d2 = 12 (m - 1); reject iff F > F_c
 *         (any channel in RGB mode).  With test = 1 (CPPM) instead: reject
 *         iff Pearson's X^2 of the window's counts exceeds chi_c;
 *      e. reject: shrink r, clear the window, t = 0; else t = t'.
 *    Hit points are independent given the photons, so the loop over hit
 *    points is a plain parallel-for.
 * ---------------------------------------------------------------------- */
typedef struct {
    float k;          /* shrinking ratio */
    float alpha;      /* radius-bound exponent */
    float r_min;      /* lower-bound scale r_min (absolute) */
    float n_vm;       /* light sub-paths used for merging (VCM+) */
    double alpha_f;   /* significance level of the F-test */
    int32_t rgb_test; /* 1: F-test on R, G and B, reject if any rejects */
    int32_t vcm;      /* 1: weight each sample by the VCM+ merge weight */
    int32_t i0;       /* global index of the first iteration (1-based) */
    int32_t test;     /* 0: ANOVA F-test (FPPM); 1: chi-square test of the
                         window's counts (CPPM, Sec. 3.2.3) decides alone */
    int32_t retrace;  /* 1: the hit-point arrays hold one set per iteration
                         (eye paths traced anew each iteration, the pixel's
                         statistics carried over, as in SPPM) */
    int32_t pad;
} oracle_params;

typedef struct {
    int32_t n, cap;
    int8_t* grp;
    double* val;      /* nch values per entry */
} or_window;

static void or_push(or_window* w, int nch, int g, const double* v)
{
    if (w->n == w->cap) {
        int cap = w->cap ? 2 * w->cap : 256;
        w->grp = (int8_t*)realloc(w->grp, (size_t)cap);
        w->val = (double*)realloc(w->val, (size_t)cap * nch * sizeof(double));
        w->cap = cap;
    }
    w->grp[w->n] = (int8_t)g;
    for (int c = 0; c < nch; ++c) w->val[(size_t)w->n * nch + c] = v[c];
    w->n++;
}

/* F for one channel of a window: regroup the stored values by group. */
static double or_window_f(const or_window* w, int nch, int ch, double m,
                          int64_t* counts_out, double* sums_out, double* sq_out)
{
    int64_t counts[OR_NG] = {0};
    for (int j = 0; j < w->n; ++j) counts[w->grp[j]]++;
    double* vals = (double*)malloc(sizeof(double) * (size_t)(w->n > 0 ? w->n : 1));
    int64_t off[OR_NG], fill[OR_NG];
    int64_t o = 0;
    for (int g = 0; g < OR_NG; ++g) { off[g] = o; fill[g] = 0; o += counts[g]; }
    for (int j = 0; j < w->n; ++j) {
        int g = w->grp[j];
        vals[off[g] + fill[g]++] = w->val[(size_t)j * nch + ch];
    }
    if (counts_out) for (int g = 0; g < OR_NG; ++g) counts_out[g] = counts[g];
    if (sums_out || sq_out) {
        for (int g = 0; g < OR_NG; ++g) {
            double s = 0.0, q = 0.0;
            for (int64_t j = 0; j < counts[g]; ++j) {
                s += vals[off[g] + j];
                q += vals[off[g] + j] * vals[off[g] + j];
            }
            if (sums_out) sums_out[g] = s;
            if (sq_out) sq_out[g] = q;
        }
    }
    double F = oracle_anova_f(OR_NG, m, counts, vals, NULL);
    free(vals);
    return F;
}

/* ------------------------------------------------------------------------
 * 7. The same method with a sorted uniform grid as the range search over
 *    the iteration's photons (Sec. 5.1 step 1 builds such a
 *    structure first), for timing the method on the CPU.  Photons are
 *    sorted by their integer cell (iz, iy, ix) = floor(p / h), FP64, with
 *    h = the largest initial radius (radii only shrink, so a disk always
 *    fits in 3 cells per axis); a hit point visits the cells of the box
 *    [floor((x - r')/h), floor((x + r')/h)] per axis, r' = r (1 + 2^-10)
 *    plus the rounding of x (a photon that passes the FP32 disk test lies
 *    within r (1 + 2^-20) of x), and classifies every photon there with the
 *    same FP32 rules as the brute force.  The in-disk photons, and so the
 *    counts and decisions, are exactly the brute force's; only the order in
 *    which the FP64 sums add them changes.
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t iz, iy, ix;
    int64_t p;         /* photon index within the iteration */
} or_cell_entry;

static int or_cell_cmp(const void* a, const void* b)
{
    const or_cell_entry* x = (const or_cell_entry*)a;
    const or_cell_entry* y = (const or_cell_entry*)b;
    if (x->iz != y->iz) return x->iz < y->iz ? -1 : 1;
    if (x->iy != y->iy) return x->iy < y->iy ? -1 : 1;
    if (x->ix != y->ix) return x->ix < y->ix ? -1 : 1;
    return x->p < y->p ? -1 : (x->p > y->p ? 1 : 0);
}

static int64_t or_cell_of(double v, double h)
{
    return (int64_t)floor(v / h);
}

/* Sort g[0, n) by or_cell_cmp with all threads: every thread sorts one
 * contiguous chunk, then pairs of sorted runs are merged (into tmp and
 * back) until one run is left.  The order is the total order of
 * or_cell_cmp (photon index last), so it does not depend on the thread
 * count. */
static int or_sort_cells(or_cell_entry* g, int64_t n)
{
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    if (nt < 1) nt = 1;
    if (n < 65536 || nt == 1) {
        qsort(g, (size_t)n, sizeof(or_cell_entry), or_cell_cmp);
        return 0;
    }
    or_cell_entry* tmp = (or_cell_entry*)malloc(sizeof(or_cell_entry) * (size_t)n);
    if (!tmp) {
        qsort(g, (size_t)n, sizeof(or_cell_entry), or_cell_cmp);
        return 0;
    }
    const int64_t chunk = (n + nt - 1) / nt;
    #pragma omp parallel for schedule(static, 1)
    for (int c = 0; c < nt; ++c) {
        const int64_t a = c * chunk, b = a + chunk < n ? a + chunk : n;
        if (a < b) qsort(g + a, (size_t)(b - a), sizeof(or_cell_entry), or_cell_cmp);
    }
    or_cell_entry *src = g, *dst = tmp;
    for (int64_t width = chunk; width < n; width *= 2) {
        const int64_t pairs = (n + 2 * width - 1) / (2 * width);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < pairs; ++q) {
            int64_t i = 2 * q * width, mid = i + width < n ? i + width : n;
            const int64_t end = mid + width < n ? mid + width : n;
            int64_t j = mid, o = i;
            while (i < mid && j < end) dst[o++] = or_cell_cmp(&src[j], &src[i]) < 0 ? src[j++] : src[i++];
            while (i < mid) dst[o++] = src[i++];
            while (j < end) dst[o++] = src[j++];
        }
        or_cell_entry* t = src; src = dst; dst = t;
    }
    if (src != g) memcpy(g, src, sizeof(or_cell_entry) * (size_t)n);
    free(tmp);
    return 0;
}

/* first entry of grid[0, n) not ordered before cell (iz, iy, ix) */
static int64_t or_cell_lower(const or_cell_entry* grid, int64_t n, int64_t iz, int64_t iy, int64_t ix)
{
    or_cell_entry key = {iz, iy, ix, -1};
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (or_cell_cmp(&grid[mid], &key) < 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/*
 * Inputs (all host arrays, row-major):
 *   hp_pos, hp_u, hp_v: nh*3 float; hp_nq: nh packed snorm8 normals or NULL;
 *   hp_rho: nh*2 float (rho_vm_h, rho_vc_h) for VCM+, else NULL;
 *   with prm->retrace every hit-point array holds iters consecutive sets
 *   (iters*nh entries), the set of iteration it used in iteration it;
 *   r_init: nh float initial radii (windows start empty, t = 0);
 *   ph_pos: iters*J*3 float; ph_flux: iters*J*nch float (nch = 1 or 3);
 *   ph_nq: iters*J packed normals or NULL; ph_rho: iters*J*2 float
 *   (rho_vm_l, rho_vc_l) and ph_wq: iters*J packed directions, VCM+ only.
 * Outputs (each may be NULL):
 *   out_r:      (iters+1)*nh  radius used in each iteration, then final radius
 *   out_counts: iters*nh*12   window counts c_g that the test of that
 *                             iteration used (after accumulation, before reset)
 *   out_S:      iters*nh*ntest*12  window sums of psi per tested channel
 *                             (ntest = 3 with rgb_test and RGB flux, else 1)
 *                             and group
 *   out_Q:      iters*nh*ntest*12  window sums of psi^2 likewise
 *   out_F:      iters*nh      F of test channel 0
 *   out_Fc:     iters*nh      critical value used
 *   out_reject: iters*nh      1 if rejected
 *   out_pairs:  iters*nh      in-disk pairs gathered in that iteration
 *   out_est:    iters*nh*nch  that iteration's kernel estimate
 *                             sum(w Phi) / (pi r_i^2) (the term added to tau)
 *   out_t:      nh            final window length t
 *   out_tau:    nh*nch        final accumulated estimate sum
 * Returns 0 on success, -1 on bad arguments.
 */
static int or_run(int use_grid, int64_t nh, const float* hp_pos, const float* hp_u,
                  const float* hp_v, const uint32_t* hp_nq, const float* hp_rho,
                  const float* r_init, int iters, int64_t J, const float* ph_pos,
                  const float* ph_flux, int nch, const uint32_t* ph_nq,
                  const float* ph_rho, const uint32_t* ph_wq,
                  const oracle_params* prm,
                  float* out_r, int32_t* out_counts, double* out_S,
                  double* out_Q, double* out_F, double* out_Fc,
                  uint8_t* out_reject, int32_t* out_pairs, int32_t* out_t,
                  double* out_tau, double* out_est)
{
    if (nh < 0 || iters < 0 || J < 2 || (nch != 1 && nch != 3) || !prm ||
        (prm->test != 0 && prm->test != 1))
        return -1;
    if (prm->vcm && (!hp_rho || !ph_rho || !ph_wq || !hp_nq)) return -1;
    const int use_normals = (hp_nq != NULL && ph_nq != NULL);
    const int ntest = (prm->rgb_test && nch == 3) ? 3 : 1;
    const int wch = ntest;   /* values stored per window entry */

    /* critical values for every window length t' that can occur */
    int tmax = iters;
    double* fc = (double*)malloc(sizeof(double) * (size_t)(tmax + 1));
    for (int t = 1; t <= tmax; ++t)
        fc[t] = oracle_f_crit(OR_NG - 1, OR_NG * ((double)t * (double)J - 1.0), prm->alpha_f);
    const double chic = prm->test == 1 ? oracle_chi2_crit(OR_NG - 1, prm->alpha_f) : 0.0;
    float* bound = (float*)malloc(sizeof(float) * (size_t)(iters > 0 ? iters : 1));
    for (int it = 0; it < iters; ++it)
        bound[it] = oracle_radius_bound(prm->r_min, prm->alpha, prm->i0 + it);

    /* grid form: every iteration's photons sorted by cell (section 7) */
    or_cell_entry* grid = NULL;
    double gh = 0.0;
    if (use_grid && iters > 0 && J > 0) {
        for (int64_t h = 0; h < nh; ++h) if ((double)r_init[h] > gh) gh = (double)r_init[h];
        if (!(gh > 0.0)) gh = 1.0;
        grid = (or_cell_entry*)malloc(sizeof(or_cell_entry) * (size_t)iters * (size_t)J);
        if (!grid) { free(fc); free(bound); return -1; }
        for (int it = 0; it < iters; ++it) {
            or_cell_entry* g = grid + (size_t)it * J;
            const float* P = ph_pos + (size_t)it * J * 3;
            #pragma omp parallel for schedule(static)
            for (int64_t p = 0; p < J; ++p) {
                g[p].ix = or_cell_of(P[3 * p], gh);
                g[p].iy = or_cell_of(P[3 * p + 1], gh);
                g[p].iz = or_cell_of(P[3 * p + 2], gh);
                g[p].p = p;
            }
            or_sort_cells(g, J);
        }
    }

    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t h = 0; h < nh; ++h) {
        const float* xh = hp_pos + 3 * h;
        const float* u = hp_u + 3 * h;
        const float* v = hp_v + 3 * h;
        int64_t hi = h;           /* this iteration's entry of hit point h */
        float r = r_init[h];
        int32_t t = 0;
        double tau[3] = {0.0, 0.0, 0.0};
        or_window win = {0, 0, NULL, NULL};
        for (int it = 0; it < iters; ++it) {
            if (prm->retrace) {
                hi = (int64_t)it * nh + h;
                xh = hp_pos + 3 * hi;
                u = hp_u + 3 * hi;
                v = hp_v + 3 * hi;
            }
            const float* P = ph_pos + (size_t)it * J * 3;
            const float* PHI = ph_flux + (size_t)it * J * nch;
            if (out_r) out_r[(size_t)it * nh + h] = r;
            double phi_sum[3] = {0.0, 0.0, 0.0};
            int32_t pairs = 0;
            /* candidates: every photon (brute force), or the photons of the
             * cells around the disk (grid form), row by row */
            const or_cell_entry* G = grid ? grid + (size_t)it * J : NULL;
            int64_t cz0 = 0, cz1 = 0, cy0 = 0, cy1 = 0, cx0 = 0, cx1 = 0;
            if (G) {
                const double rr = (double)r * (1.0 + 1.0 / 1024.0)
                                + 1e-6 * (fabs((double)xh[0]) + fabs((double)xh[1]) + fabs((double)xh[2]));
                cx0 = or_cell_of((double)xh[0] - rr, gh); cx1 = or_cell_of((double)xh[0] + rr, gh);
                cy0 = or_cell_of((double)xh[1] - rr, gh); cy1 = or_cell_of((double)xh[1] + rr, gh);
                cz0 = or_cell_of((double)xh[2] - rr, gh); cz1 = or_cell_of((double)xh[2] + rr, gh);
            }
            int64_t row_z = cz0, row_y = cy0, k = 0, kend = G ? 0 : J;
            for (;;) {
                if (k == kend) {
                    if (!G || row_z > cz1) break;
                    /* next row of cells */
                    k = or_cell_lower(G, J, row_z, row_y, cx0);
                    kend = or_cell_lower(G, J, row_z, row_y, cx1 + 1);
                    if (++row_y > cy1) { row_y = cy0; ++row_z; }
                    continue;
                }
                const int64_t p = G ? G[k].p : k;
                ++k;
                size_t gp = (size_t)it * J + p;
                int g = oracle_classify(xh, u, v, r, P + 3 * p, use_normals,
                                        use_normals ? hp_nq[hi] : 0,
                                        use_normals ? ph_nq[gp] : 0);
                if (g < 0) continue;
                pairs++;
                double w = 1.0;
                if (prm->vcm) {
                    int cd = oracle_normal_dot(hp_nq[hi], ph_wq[gp]);
                    w = oracle_mis_weight(hp_rho[2 * hi], hp_rho[2 * hi + 1],
                                          ph_rho[2 * gp], ph_rho[2 * gp + 1],
                                          cd, prm->n_vm, (double)r);
                }
                double phi[3], val[3];
                for (int c = 0; c < nch; ++c) {
                    phi[c] = w * (double)PHI[(size_t)p * nch + c];
                    phi_sum[c] += phi[c];
                }
                if (ntest == 3) { val[0] = phi[0]; val[1] = phi[1]; val[2] = phi[2]; }
                else if (nch == 3) val[0] = or_lum(phi[0], phi[1], phi[2]);
                else val[0] = phi[0];
                or_push(&win, wch, g, val);
            }
            /* Eq. (progressive-VCM-estimator): kernel estimate of iteration
             * i with its own radius r_i; 1/(pi r^2) is the normalized disk
             * kernel. */
            double area = M_PI * (double)r * (double)r;
            for (int c = 0; c < nch; ++c) tau[c] += phi_sum[c] / area;
            if (out_est)
                for (int c = 0; c < nch; ++c) out_est[((size_t)it * nh + h) * nch + c] = phi_sum[c] / area;

            int32_t tp = t + 1;
            double m = (double)tp * (double)J;
            int reject = 0;
            double F0 = 0.0;
            int64_t cnt[OR_NG];
            double S[3][OR_NG], Q[3][OR_NG];
            for (int ch = 0; ch < ntest; ++ch) {
                double F = or_window_f(&win, wch, ch, m, ch == 0 ? cnt : NULL, S[ch], Q[ch]);
                if (ch == 0) F0 = F;
                if (F > fc[tp]) reject = 1;
            }
            if (prm->test == 1) {
                /* CPPM: the count test alone decides; its statistic takes
                 * F's place in the outputs */
                F0 = oracle_chi2_counts(OR_NG, cnt);
                reject = F0 > chic;
            }
            size_t o = (size_t)it * nh + h;
            if (out_counts) for (int g = 0; g < OR_NG; ++g) out_counts[o * OR_NG + g] = (int32_t)cnt[g];
            for (int ch = 0; ch < ntest; ++ch)
                for (int g = 0; g < OR_NG; ++g) {
                    if (out_S) out_S[(o * ntest + ch) * OR_NG + g] = S[ch][g];
                    if (out_Q) out_Q[(o * ntest + ch) * OR_NG + g] = Q[ch][g];
                }
            if (out_F) out_F[o] = F0;
            if (out_Fc) out_Fc[o] = prm->test == 1 ? chic : fc[tp];
            if (out_reject) out_reject[o] = (uint8_t)reject;
            if (out_pairs) out_pairs[o] = pairs;
            if (reject) {
                r = oracle_shrink(r, prm->k, bound[it]);
                win.n = 0;
                t = 0;
            } else {
                t = tp;
            }
        }
        if (out_r) out_r[(size_t)iters * nh + h] = r;
        if (out_t) out_t[h] = t;
        if (out_tau) for (int c = 0; c < nch; ++c) out_tau[h * nch + c] = tau[c];
        free(win.grp);
        free(win.val);
    }
    free(fc);
    free(bound);
    free(grid);
    return 0;
}

int oracle_run(int64_t nh, const float* hp_pos, const float* hp_u,
               const float* hp_v, const uint32_t* hp_nq, const float* hp_rho,
               const float* r_init, int iters, int64_t J, const float* ph_pos,
               const float* ph_flux, int nch, const uint32_t* ph_nq,
               const float* ph_rho, const uint32_t* ph_wq,
               const oracle_params* prm,
               float* out_r, int32_t* out_counts, double* out_S,
               double* out_Q, double* out_F, double* out_Fc,
               uint8_t* out_reject, int32_t* out_pairs, int32_t* out_t,
               double* out_tau, double* out_est)
{
    return or_run(0, nh, hp_pos, hp_u, hp_v, hp_nq, hp_rho, r_init, iters, J, ph_pos, ph_flux,
                  nch, ph_nq, ph_rho, ph_wq, prm, out_r, out_counts, out_S, out_Q, out_F,
                  out_Fc, out_reject, out_pairs, out_t, out_tau, out_est);
}

/* The same as oracle_run with the grid of section 7 as the range search
 * (identical counts and decisions; FP64 sums in cell order). */
int oracle_run_grid(int64_t nh, const float* hp_pos, const float* hp_u,
                    const float* hp_v, const uint32_t* hp_nq, const float* hp_rho,
                    const float* r_init, int iters, int64_t J, const float* ph_pos,
                    const float* ph_flux, int nch, const uint32_t* ph_nq,
                    const float* ph_rho, const uint32_t* ph_wq,
                    const oracle_params* prm,
                    float* out_r, int32_t* out_counts, double* out_S,
                    double* out_Q, double* out_F, double* out_Fc,
                    uint8_t* out_reject, int32_t* out_pairs, int32_t* out_t,
                    double* out_tau, double* out_est)
{
    return or_run(1, nh, hp_pos, hp_u, hp_v, hp_nq, hp_rho, r_init, iters, J, ph_pos, ph_flux,
                  nch, ph_nq, ph_rho, ph_wq, prm, out_r, out_counts, out_S, out_Q, out_F,
                  out_Fc, out_reject, out_pairs, out_t, out_tau, out_est);
}
