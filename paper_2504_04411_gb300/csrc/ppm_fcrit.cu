// ppm_fcrit.cu -- table of F-test critical values, FP64 on the GPU (and
// the chi-square critical value of CPPM's count test, Sec. 3.2.3).
//
// Sec. 3.2.2: reject the null hypothesis iff F > F_c, where F_c is the
// (1 - alpha_F) quantile of the F distribution with d1 = n - 1 = 11 and
// d2 = n (m - 1) degrees of freedom; Sec. 6.1.1 updates F_c at run time with
// the sample count.  With m = t J samples per group (t iterations in the
// window, J light paths per iteration) the table is indexed by t.
//
// CDF_F(f) = I_x(d1/2, d2/2) with x = d1 f / (d1 f + d2) (regularized
// incomplete beta).  I is evaluated from its continued fraction (DLMF
// Sec. 8.17(v)), whose convergents are built by the three-term forward
// recurrences of their numerators and denominators (Wallis), rescaled at
// every step.  The fraction is taken on the side of the symmetry
// I_x(a,b) = 1 - I_{1-x}(b,a) where it converges quickly, except for b >> a
// (d2 >> d1, always the case here), where the other side's odd terms are
// close to -1 and every step cancels most digits: there the direct side is
// well conditioned and converges in a few dozen terms.  The quantile is
// found by Newton's method on the CDF (derivative = the F density) kept
// inside a bisection bracket.  d2 reaches ~1e11, where lgamma(b) -
// lgamma(a+b) loses ~1e-6 to cancellation in FP64, so for b >= 64 that
// difference is taken from the Stirling series of log Gamma written as a
// difference (no cancellation; the first omitted term, 1/(1680 b^7), is
// below 1e-15 there).
#include "ppm_internal.cuh"

namespace {

__device__ double lbeta_fp64(double a, double b)
{
    if (b < 64.0) return lgamma(a) + lgamma(b) - lgamma(a + b);
    // log G(b) - log G(a+b) from log G(z) = (z-1/2) log z - z + log(2 pi)/2
    //   + 1/(12 z) - 1/(360 z^3) + 1/(1260 z^5) - ...
    const double ab = a + b;
    double d = -(b - 0.5) * log1p(a / b) - a * log(ab) + a;
    const double ib = 1.0 / b, iab = 1.0 / ab;
    const double ib3 = ib * ib * ib, iab3 = iab * iab * iab;
    d += (ib - iab) / 12.0 - (ib3 - iab3) / 360.0 + (ib3 * ib * ib - iab3 * iab * iab) / 1260.0;
    return lgamma(a) + d;
}

// Value of the continued fraction 1 / (1 + e_1 / (1 + e_2 / (1 + ...))) of
// DLMF Sec. 8.17(v), so that I_x(a,b) = x^a (1-x)^b / (a B(a,b)) times it, with
//   e_{2j}   =  j (b - j) x / ((a + 2j - 1)(a + 2j)),
//   e_{2j+1} = -(a + j)(a + b + j) x / ((a + 2j)(a + 2j + 1)).
// Convergent n is num_n / den_n with num_n = num_{n-1} + e_{n-1} num_{n-2}
// (den likewise) from num = (1, 1), den = (1, 1 + e_1); the pair of the
// last two convergents is divided by den_n every step so nothing overflows.
__device__ double beta_fraction_fp64(double a, double b, double x)
{
    double num_prev = 1.0, den_prev = 1.0;            // convergent 1: 1 / 1
    double num = 1.0, den = 1.0 - (a + b) * x / (a + 1.0);   // convergent 2: 1 / (1 + e_1)
    double value = num / den;
    for (int n = 2; n <= 8000; ++n) {
        const int j = n >> 1;
        const double e = (n & 1) ? -(a + j) * (a + b + j) * x / ((a + 2.0 * j) * (a + 2.0 * j + 1.0))
                                 : j * (b - j) * x / ((a + 2.0 * j - 1.0) * (a + 2.0 * j));
        const double num_next = num + e * num_prev;
        double den_next = den + e * den_prev;
        if (den_next == 0.0) den_next = 1e-300;       // a zero denominator: step over it
        const double s = 1.0 / den_next;
        num_prev = num * s;
        den_prev = den * s;
        num = num_next * s;
        den = 1.0;
        const double v = num;
        const bool done = fabs(v - value) <= 4e-16 * fabs(v);
        value = v;
        if (done && (n & 1)) break;                   // stop after an odd term
    }
    return value;
}

// CDF and density of F(d1, d2) at f > 0
__device__ void f_cdf_pdf(double d1, double d2, double f, double* cdf, double* pdf)
{
    const double a = 0.5 * d1, b = 0.5 * d2;
    const double s = d1 * f;
    const double x = s / (s + d2);
    const double lx = log(x);
    const double l1x = -log1p(s / d2);          // log(1 - x) without cancellation
    const double lb = lbeta_fp64(a, b);
    const double front = exp(a * lx + b * l1x - lb);
    if (x < (a + 1.0) / (a + b + 2.0) || b > 50.0 * a) *cdf = front * beta_fraction_fp64(a, b, x) / a;
    else *cdf = 1.0 - front * beta_fraction_fp64(b, a, d2 / (s + d2)) / b;
    // d/df I_x = x^(a-1) (1-x)^(b-1) / B(a,b) * dx/df, dx/df = d1 d2 / (s + d2)^2
    *pdf = exp((a - 1.0) * lx + (b - 1.0) * l1x - lb) * d1 * d2 / ((s + d2) * (s + d2));
}

__device__ double f_quantile(double d1, double d2, double q)
{
    double lo = 0.0, hi = 4.0, c, p;
    for (int i = 0; i < 200; ++i) {             // bracket the root
        f_cdf_pdf(d1, d2, hi, &c, &p);
        if (c >= q) break;
        lo = hi;
        hi *= 2.0;
    }
    double f = 0.5 * (lo + hi);
    for (int it = 0; it < 100; ++it) {
        f_cdf_pdf(d1, d2, f, &c, &p);
        const double g = c - q;
        if (g < 0.0) lo = f; else hi = f;
        double fn = (p > 0.0) ? f - g / p : 0.5 * (lo + hi);
        if (!(fn > lo && fn < hi)) fn = 0.5 * (lo + hi);   // keep Newton in the bracket
        if (fabs(fn - f) <= 1e-15 * f || hi - lo <= 1e-15 * hi) { f = fn; break; }
        f = fn;
    }
    return f;
}

__global__ void k_fcrit_table(double* __restrict__ table, int t_from, int t_to,
                              double J, double alpha)
{
    const int t = t_from + blockIdx.x * blockDim.x + threadIdx.x;
    if (t > t_to) return;
    const double m = (double)t * J;                  // samples per group
    const double d1 = PPM_NG - 1, d2 = PPM_NG * (m - 1.0);
    table[t] = f_quantile(d1, d2, 1.0 - alpha);
}

// The F statistic's dependence on the window length t: with m = t J samples
// per group (an integer, taken in FP64, never FP32),
//   SSW = sum_g Q_g - (1/m) sum_g S_g^2,
//   F = (SSB / (n-1)) / (SSW / (n (m-1))) = (dev2 / SSW) * n (m-1) / ((n-1) m),
// dev2 = sum_g (S_g - S/n)^2.  mtab[t] = (1/m, n (m-1) / ((n-1) m)), each
// computed in FP64 and rounded once to FP32 for the gather's epilogue.
__global__ void k_window_m(float2* __restrict__ mtab, int t_from, int t_to, double J)
{
    const int t = t_from + blockIdx.x * blockDim.x + threadIdx.x;
    if (t > t_to) return;
    const double m = (double)t * J;
    mtab[t] = make_float2((float)(1.0 / m),
                          (float)((double)PPM_NG * (m - 1.0) / ((double)(PPM_NG - 1) * m)));
}

// CPPM's count test (Sec. 3.2.3): chi_c = the (1 - alpha) quantile of
// chi^2(k) with k = n - 1 = 11, whose CDF is P(k/2, x/2), P the regularized
// lower incomplete gamma function.  Below z = a + 1, P comes from its power
// series (DLMF Sec. 8.7)
//   P(a, z) = z^a e^-z / Gamma(a + 1) * sum_{j >= 0} z^j / ((a+1)...(a+j));
// above, 1 - Q with Q from the continued fraction of Gamma(a, z) (DLMF Sec. 8.9)
//   Gamma(a, z) = e^-z z^a / (z + (1-a) / (1 + 1 / (z + (2-a) / (1 + 2 / (z + ...))))),
// whose convergents come from the forward recurrences, as for the beta.
__device__ double gamma_p_fp64(double a, double z)
{
    if (z <= 0.0) return 0.0;
    if (z < a + 1.0) {
        double term = 1.0, sum = 1.0;
        for (int j = 1; j < 8000; ++j) {
            term *= z / (a + j);
            sum += term;
            if (term <= 1e-17 * sum) break;
        }
        return exp(a * log(z) - z - lgamma(a + 1.0)) * sum;
    }
    // partial numerators / denominators: 1 / z first, then for k = 1, 2, ...
    // (k - a) / 1 (even n = 2k) and k / z (odd n = 2k + 1)
    double num_prev = 0.0, den_prev = 1.0;            // convergent 0: 0 / 1
    double num = 1.0, den = z;                        // convergent 1: 1 / z
    double value = num / den;
    for (int n = 2; n <= 16000; ++n) {
        const int k = n >> 1;
        const double an = (n & 1) ? (double)k : (double)k - a;   // partial numerator
        const double bn = (n & 1) ? z : 1.0;                      // partial denominator
        const double num_next = bn * num + an * num_prev;
        double den_next = bn * den + an * den_prev;
        if (den_next == 0.0) den_next = 1e-300;
        const double s = 1.0 / den_next;
        num_prev = num * s;
        den_prev = den * s;
        num = num_next * s;
        den = 1.0;
        const bool done = fabs(num - value) <= 4e-16 * fabs(num);
        value = num;
        if (done && (n & 1)) break;
    }
    return 1.0 - exp(a * log(z) - z - lgamma(a)) * value;
}

// quantile of chi^2(k) at q: Newton on the CDF (derivative = the density
// x^(a-1) e^(-x/2) / (2^a Gamma(a)), a = k/2) inside a bisection bracket
__device__ double chi2_quantile(double k, double q)
{
    const double a = 0.5 * k;
    double lo = 0.0, hi = k + 16.0;
    for (int i = 0; i < 2000 && gamma_p_fp64(a, 0.5 * hi) < q; ++i) {
        lo = hi;
        hi *= 2.0;
    }
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double g = gamma_p_fp64(a, 0.5 * x) - q;
        if (g < 0.0) lo = x; else hi = x;
        const double pdf = exp((a - 1.0) * log(x) - 0.5 * x - a * 0.6931471805599453 - lgamma(a));
        double xn = pdf > 0.0 ? x - g / pdf : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-15 * x || hi - lo <= 1e-15 * hi) { x = xn; break; }
        x = xn;
    }
    return x;
}

// every entry t_from .. t_to of the table gets chi_c: the count test's
// critical value does not depend on the window length
__global__ void k_chi2_table(double* __restrict__ table, int t_from, int t_to, double k, double alpha)
{
    const int t = t_from + blockIdx.x * blockDim.x + threadIdx.x;
    if (t > t_to) return;
    table[t] = chi2_quantile(k, 1.0 - alpha);
}

}  // namespace

int ppm_chi2_fill(double* table, int t_from, int t_to, double k, double alpha, cudaStream_t st)
{
    if (t_to < t_from) return PPM_OK;
    const int n = t_to - t_from + 1;
    k_chi2_table<<<(n + 63) / 64, 64, 0, st>>>(table, t_from, t_to, k, alpha);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_window_m_fill(float2* mtab, int t_from, int t_to, double J, cudaStream_t st)
{
    if (t_to < t_from) return PPM_OK;
    const int n = t_to - t_from + 1;
    k_window_m<<<(n + 127) / 128, 128, 0, st>>>(mtab, t_from, t_to, J);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}

int ppm_fcrit_fill(double* table, int t_from, int t_to, double J, double alpha, cudaStream_t st)
{
    if (t_to < t_from) return PPM_OK;
    const int n = t_to - t_from + 1;
    k_fcrit_table<<<(n + 63) / 64, 64, 0, st>>>(table, t_from, t_to, J, alpha);
    PPM_LAUNCH_CHECK();
    return PPM_OK;
}
