/*
 * oracle.c -- plain, slow, FP64 CPU reference for the fast aperture-mass
 * pipeline of Leonard, Pires & Starck, "Fast Calculation of the Weak Lensing
 * Aperture Mass Statistic" (MNRAS 2012).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Every function follows the passage it cites and is written for a reader to
 * check by eye: no blocking, no fusion, FP64 throughout.  Where the paper is
 * silent the reading taken is stated at the function.
 *
 * Conventions (the same everywhere in this file):
 *   maps are n x n, row-major, element (y, x) at [y*n + x];
 *   x is the column index and pairs with k1, y pairs with k2;
 *   integer frequency of index i is k = i for i < n/2, else i - n
 *   (so index n/2 is -n/2);
 *   FFT: forward exp(-2 pi i k x / n) unnormalised, inverse exp(+...) / n.
 *
 * Parity pins: every function here is checked in tests/ against something
 * other than itself (closed forms, brute force on tiny inputs, numpy.fft,
 * invariants of the transform, the analytic noise variance).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Filter functions (Sec. 4)                                                */
/* ------------------------------------------------------------------------ */

/* B3-spline scaling function phi(x) of the starlet (Sec. 4.2, equation after
 * eq. splinewl). Zero for |x| > 2. */
double oracle_phi_b3(double x)
{
    double a = fabs(x - 2.0), b = fabs(x - 1.0), c = fabs(x);
    double d = fabs(x + 1.0), e = fabs(x + 2.0);
    return (a * a * a - 4.0 * b * b * b + 6.0 * c * c * c - 4.0 * d * d * d + e * e * e) / 12.0;
}

/* The discrete a-trous filter.  The paper does not print it; the B3 two-scale
 * relation phi(x/2)/2 = sum_k h_k phi(x - k) fixes h = [1, 4, 6, 4, 1] / 16
 * (checked against oracle_phi_b3 in the tests). */
static const double H_B3[5] = {1.0 / 16.0, 4.0 / 16.0, 6.0 / 16.0, 4.0 / 16.0, 1.0 / 16.0};

void oracle_starlet_taps(double *h5)
{
    for (int k = 0; k < 5; ++k) h5[k] = H_B3[k];
}

static double cube(double v) { return v * v * v; }

/* Starlet aperture filter U(eta), eta = vartheta / theta (Sec. 4.2, closed
 * form printed after eq. splinewl). */
double oracle_u_starlet(double eta)
{
    double e = fabs(eta);
    return (93.0 * cube(e) - 64.0 * (cube(fabs(0.5 - eta)) + cube(fabs(0.5 + eta))) +
            18.0 * (cube(fabs(1.0 - eta)) + cube(fabs(1.0 + eta))) -
            0.5 * (cube(fabs(2.0 - eta)) + cube(fabs(2.0 + eta)))) / 9.0;
}

/* Starlet shear filter Q(eta) (Sec. 4.2, closed form printed with U).  The
 * 1/eta^2 prefactor makes eta = 0 undefined; the direct sum never evaluates
 * it (the d = 0 offset is dropped) and the limit there is 0. */
double oracle_q_starlet(double eta)
{
    if (eta == 0.0) return 0.0;
    double e2 = eta * eta;
    double s = -279.0 * e2 * cube(fabs(eta));
    s += 8.0 * (1.0 + 6.0 * eta + 24.0 * e2) * cube(fabs(0.5 - eta));
    s -= 9.0 * (1.0 + 3.0 * eta + 6.0 * e2) * cube(fabs(1.0 - eta));
    s -= 9.0 * (1.0 - 3.0 * eta + 6.0 * e2) * cube(fabs(1.0 + eta));
    s += (1.0 + 1.5 * eta + 1.5 * e2) * cube(fabs(2.0 - eta));
    s += (1.0 - 1.5 * eta + 1.5 * e2) * cube(fabs(2.0 + eta));
    s += 8.0 * (1.0 - 6.0 * eta + 24.0 * e2) * cube(fabs(0.5 + eta));
    return s / (45.0 * e2);
}

/* Polynomial filter family of Schneider et al. 1998, eq. sch (Sec. 4.1).
 * Both carry the 1/theta^2 of the paper and the Heaviside cut at theta. */
double oracle_u_s98(double vartheta, double theta, int ell)
{
    if (vartheta > theta) return 0.0;
    double x2 = vartheta * vartheta / (theta * theta);
    double l = (double)ell;
    return (l + 2.0) * (l + 2.0) / (M_PI * theta * theta) * pow(1.0 - x2, l) * (1.0 / (l + 2.0) - x2);
}

double oracle_q_s98(double vartheta, double theta, int ell)
{
    if (vartheta > theta) return 0.0;
    double x2 = vartheta * vartheta / (theta * theta);
    double l = (double)ell;
    return (1.0 + l) * (2.0 + l) / (M_PI * theta * theta) * x2 * pow(1.0 - x2, l);
}

/* Gaussian filter of eq. mexhat (Sec. 4.1), normalisation A = 1 (the paper
 * leaves A free).  b = 1/2 for JBJ04, b = 4 for vW98. */
double oracle_q_gauss(double vartheta, double theta, double b)
{
    double x = b * vartheta * vartheta / (theta * theta);
    return x * exp(-x) / (theta * theta);
}

double oracle_u_gauss(double vartheta, double theta, double b)
{
    double x = b * vartheta * vartheta / (theta * theta);
    return (1.0 - x) * exp(-x) / (theta * theta);
}

/* ------------------------------------------------------------------------ */
/* FFT: textbook iterative radix-2 Cooley-Tukey (bit reversal, then stages). */
/* ------------------------------------------------------------------------ */

static void fft1d(double complex *a, int n, int inverse)
{
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double complex t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; ++k) {
            double ang = (inverse ? 2.0 : -2.0) * M_PI * (double)k / (double)len;
            double complex w = cos(ang) + I * sin(ang);
            for (int i = 0; i < n; i += len) {
                double complex u = a[i + k];
                double complex v = a[i + k + half] * w;
                a[i + k] = u + v;
                a[i + k + half] = u - v;
            }
        }
    }
    if (inverse)
        for (int i = 0; i < n; ++i) a[i] /= (double)n;
}

/* 2-D transform: every row, then every column. */
static void fft2d(double complex *a, int n, int inverse)
{
    double complex *col = (double complex *)malloc(sizeof(double complex) * (size_t)n);
    for (int y = 0; y < n; ++y) fft1d(a + (size_t)y * n, n, inverse);
    for (int x = 0; x < n; ++x) {
        for (int y = 0; y < n; ++y) col[y] = a[(size_t)y * n + x];
        fft1d(col, n, inverse);
        for (int y = 0; y < n; ++y) a[(size_t)y * n + x] = col[y];
    }
    free(col);
}

/* Exposed for the tests: in-place 2-D FFT of an interleaved (re, im) array. */
void oracle_fft2(double *re_im, int n, int inverse)
{
    fft2d((double complex *)re_im, n, inverse);
}

static int freq_of(int i, int n) { return i < n / 2 ? i : i - n; }

/* ------------------------------------------------------------------------ */
/* Kaiser-Squires in Fourier space (Sec. 4.5).                              */
/* The paper states only that shear and convergence are related by a 2-D    */
/* convolution inverted in Fourier space; the multiplier used is the        */
/* standard D(k) = (k1 + i k2)^2 / |k|^2 with D(0) = 0, forward             */
/* gamma = IFFT(D FFT kappa) and inverse kappa = IFFT(conj(D) FFT gamma).   */
/* ------------------------------------------------------------------------ */

static double complex ks_multiplier(int k1, int k2)
{
    double kk = (double)k1 * k1 + (double)k2 * k2;
    if (kk == 0.0) return 0.0;
    double complex num = ((double)k1 + I * (double)k2) * ((double)k1 + I * (double)k2);
    return num / kk;
}

void oracle_ks_forward(const double *kappa, double *g1, double *g2, int n)
{
    size_t nn = (size_t)n * n;
    double complex *a = (double complex *)malloc(sizeof(double complex) * nn);
    for (size_t i = 0; i < nn; ++i) a[i] = kappa[i];
    fft2d(a, n, 0);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            a[(size_t)y * n + x] *= ks_multiplier(freq_of(x, n), freq_of(y, n));
    fft2d(a, n, 1);
    for (size_t i = 0; i < nn; ++i) {
        g1[i] = creal(a[i]);
        g2[i] = cimag(a[i]);
    }
    free(a);
}

/* kappa_E = Re, kappa_B = Im of IFFT(conj(D) FFT(gamma1 + i gamma2)).
 * kappa_B may be NULL. */
void oracle_ks_invert(const double *g1, const double *g2, double *kE, double *kB, int n)
{
    size_t nn = (size_t)n * n;
    double complex *a = (double complex *)malloc(sizeof(double complex) * nn);
    for (size_t i = 0; i < nn; ++i) a[i] = g1[i] + I * g2[i];
    fft2d(a, n, 0);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x)
            a[(size_t)y * n + x] *= conj(ks_multiplier(freq_of(x, n), freq_of(y, n)));
    fft2d(a, n, 1);
    for (size_t i = 0; i < nn; ++i) {
        kE[i] = creal(a[i]);
        if (kB) kB[i] = cimag(a[i]);
    }
    free(a);
}

/* ------------------------------------------------------------------------ */
/* Starlet (isotropic undecimated, a trous) transform (Sec. 3, Sec. 4.2).   */
/* ------------------------------------------------------------------------ */

/* Boundary index fold.  The paper does not state a boundary rule.  Mirror
 * (boundary 0) is whole-sample symmetric: -i for i < 0 and 2(n-1) - i for
 * i >= n, repeated while out of range (equivalently, period 2(n-1)).
 * Periodic (boundary 1) is i mod n. */
static int fold_index(int i, int n, int boundary)
{
    if (boundary == 1) {
        int m = i % n;
        return m < 0 ? m + n : m;
    }
    if (n == 1) return 0;
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}

/* pyr receives J arrays of n*n: w_1 .. w_{J-1}, then the smooth array left
 * after J-1 bands (the paper's c_J) in slot J-1.  Scale j uses the filter h
 * with holes: taps at offsets 0, +-2^(j-1), +-2^j; rows first, then columns;
 * w_j = c_{j-1} - c_j.  c_0 = kappa. */
void oracle_starlet(const double *kappa, double *pyr, int n, int J, int boundary)
{
    size_t nn = (size_t)n * n;
    double *c = (double *)malloc(sizeof(double) * nn);
    double *t = (double *)malloc(sizeof(double) * nn);
    double *cn = (double *)malloc(sizeof(double) * nn);
    memcpy(c, kappa, sizeof(double) * nn);
    for (int j = 1; j <= J - 1; ++j) {
        int s = 1 << (j - 1);
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double acc = 0.0;
                for (int k = 0; k < 5; ++k)
                    acc += H_B3[k] * c[(size_t)y * n + fold_index(x + (k - 2) * s, n, boundary)];
                t[(size_t)y * n + x] = acc;
            }
        for (int y = 0; y < n; ++y)
            for (int x = 0; x < n; ++x) {
                double acc = 0.0;
                for (int k = 0; k < 5; ++k)
                    acc += H_B3[k] * t[(size_t)fold_index(y + (k - 2) * s, n, boundary) * n + x];
                cn[(size_t)y * n + x] = acc;
            }
        double *w = pyr + (size_t)(j - 1) * nn;
        for (size_t i = 0; i < nn; ++i) w[i] = c[i] - cn[i];
        double *sw = c;
        c = cn;
        cn = sw;
    }
    memcpy(pyr + (size_t)(J - 1) * nn, c, sizeof(double) * nn);
    free(c);
    free(t);
    free(cn);
}

/* KS inversion followed by the starlet of kappa_E: the fast aperture-mass
 * maps of Sec. 3 computed from shear (Sec. 4.5). */
void oracle_map_starlet(const double *g1, const double *g2, double *pyr, int n, int J, int boundary)
{
    size_t nn = (size_t)n * n;
    double *kE = (double *)malloc(sizeof(double) * nn);
    oracle_ks_invert(g1, g2, kE, NULL, n);
    oracle_starlet(kE, pyr, n, J, boundary);
    free(kE);
}

/* ------------------------------------------------------------------------ */
/* Direct aperture mass from tangential shear, eq. shearmap (Sec. 2.1),     */
/* brute force as in Sec. 5.1.                                              */
/* ------------------------------------------------------------------------ */

/* Filter ids: 0 = starlet Q(eta)/theta^2 (support eta <= 2, default cut 2
 * theta); 1 = S98 with order ell (default cut theta); 2 = Gaussian with
 * b = 1/2 (JBJ04), 3 = Gaussian with b = 4 (vW98), both with A = 1 and a
 * default cut of 5 theta.  cut_over_theta > 0 overrides the default. */
double oracle_q_filter(int filter, double vartheta, double theta, int ell)
{
    switch (filter) {
    case 0: return oracle_q_starlet(vartheta / theta) / (theta * theta);
    case 1: return oracle_q_s98(vartheta, theta, ell);
    case 2: return oracle_q_gauss(vartheta, theta, 0.5);
    case 3: return oracle_q_gauss(vartheta, theta, 4.0);
    default: return 0.0;
    }
}

double oracle_default_cut(int filter)
{
    switch (filter) {
    case 0: return 2.0;
    case 1: return 1.0;
    default: return 5.0;
    }
}

/* M(x) = sum over integer offsets d, 0 < |d| <= R, of Q(|d|) gamma_t(x + d),
 * gamma_t = -[gamma1 cos 2 phi_d + gamma2 sin 2 phi_d], phi_d = atan2(dy, dx),
 * pixel area 1.  Pixels outside the field carry no data and add nothing. */
void oracle_map_direct(const double *g1, const double *g2, double *map, int n, int filter, double theta,
                       int ell, double cut_over_theta)
{
    double cut = cut_over_theta > 0.0 ? cut_over_theta : oracle_default_cut(filter);
    double R = cut * theta;
    int ri = (int)floor(R);
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            double acc = 0.0;
            for (int dy = -ri; dy <= ri; ++dy)
                for (int dx = -ri; dx <= ri; ++dx) {
                    double r2 = (double)dx * dx + (double)dy * dy;
                    if (r2 == 0.0 || r2 > R * R) continue;
                    int xx = x + dx, yy = y + dy;
                    if (xx < 0 || xx >= n || yy < 0 || yy >= n) continue;
                    double phi = atan2((double)dy, (double)dx);
                    double q = oracle_q_filter(filter, sqrt(r2), theta, ell);
                    double gt = -(g1[(size_t)yy * n + xx] * cos(2.0 * phi) + g2[(size_t)yy * n + xx] * sin(2.0 * phi));
                    acc += q * gt;
                }
            map[(size_t)y * n + x] = acc;
        }
}

/* Same sum at a list of pixels only (for spot checks of large maps). */
void oracle_map_direct_at(const double *g1, const double *g2, const int *ys, const int *xs, int npts, double *out,
                          int n, int filter, double theta, int ell, double cut_over_theta)
{
    double cut = cut_over_theta > 0.0 ? cut_over_theta : oracle_default_cut(filter);
    double R = cut * theta;
    int ri = (int)floor(R);
    for (int p = 0; p < npts; ++p) {
        int y = ys[p], x = xs[p];
        double acc = 0.0;
        for (int dy = -ri; dy <= ri; ++dy)
            for (int dx = -ri; dx <= ri; ++dx) {
                double r2 = (double)dx * dx + (double)dy * dy;
                if (r2 == 0.0 || r2 > R * R) continue;
                int xx = x + dx, yy = y + dy;
                if (xx < 0 || xx >= n || yy < 0 || yy >= n) continue;
                double phi = atan2((double)dy, (double)dx);
                double q = oracle_q_filter(filter, sqrt(r2), theta, ell);
                acc += q * -(g1[(size_t)yy * n + xx] * cos(2.0 * phi) + g2[(size_t)yy * n + xx] * sin(2.0 * phi));
            }
        out[p] = acc;
    }
}

/* Direct M_ap on a field with missing data (Sec. 4.3: edges and missing
 * data; Sec. 4.5: masked stars and bad pixels).  Pixel y carries a weight
 * w(y) >= 0, 0 where it is masked.  Over the lattice offsets 0 < |d| <= R
 * that stay inside the field,
 *   S(x) = sum w(x+d) Q(|d|) gamma_t(x+d; x),   D(x) = sum w(x+d),
 * and with N_R the number of lattice offsets 0 < |d| <= R (the aperture's
 * area in pixels) the weighted estimate of eq. shearmap is
 *   M(x) = N_R S(x) / D(x)   (0 where D(x) <= 0),   coverage(x) = D(x) / N_R.
 * With all weights 1 and the aperture inside the field, D = N_R and M is
 * the plain sum of oracle_map_direct.  Evaluated at a list of pixels. */
void oracle_map_direct_masked_at(const double *g1, const double *g2, const double *w, const int *ys, const int *xs,
                                 int npts, double *out_map, double *out_cov, int n, int filter, double theta, int ell,
                                 double cut_over_theta)
{
    double cut = cut_over_theta > 0.0 ? cut_over_theta : oracle_default_cut(filter);
    double R = cut * theta;
    int ri = (int)floor(R);
    double n_r = 0.0;
    for (int dy = -ri; dy <= ri; ++dy)
        for (int dx = -ri; dx <= ri; ++dx) {
            double r2 = (double)dx * dx + (double)dy * dy;
            if (r2 > 0.0 && r2 <= R * R) n_r += 1.0;
        }
    for (int p = 0; p < npts; ++p) {
        int y = ys[p], x = xs[p];
        double num = 0.0, den = 0.0;
        for (int dy = -ri; dy <= ri; ++dy)
            for (int dx = -ri; dx <= ri; ++dx) {
                double r2 = (double)dx * dx + (double)dy * dy;
                if (r2 == 0.0 || r2 > R * R) continue;
                int xx = x + dx, yy = y + dy;
                if (xx < 0 || xx >= n || yy < 0 || yy >= n) continue;
                size_t i = (size_t)yy * n + xx;
                double phi = atan2((double)dy, (double)dx);
                double q = oracle_q_filter(filter, sqrt(r2), theta, ell);
                double gt = -(g1[i] * cos(2.0 * phi) + g2[i] * sin(2.0 * phi));
                num += w[i] * q * gt;
                den += w[i];
            }
        out_map[p] = den > 0.0 ? n_r * num / den : 0.0;
        out_cov[p] = n_r > 0.0 ? den / n_r : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Noise by randomising the data (Sec. 1, Sec. 5.1).                        */
/* ------------------------------------------------------------------------ */

/* Counter-based generator: the (index+1)-th output of SplitMix64 (Steele,
 * Lea & Flood 2014) started from state `seed`: state advances by the golden
 * gamma 0x9E3779B97F4A7C15, output = the published 64-bit finaliser. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t index)
{
    uint64_t z = seed + (index + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Rotation angle of pixel (y, x) in realisation r: alpha = pi u, u the top
 * 24 bits of the generator output at counter (r n + y) n + x, times 2^-24,
 * so alpha is uniform on [0, pi). Returns u. */
double oracle_noise_u(uint64_t seed, int r, int y, int x, int n)
{
    uint64_t idx = ((uint64_t)r * (uint64_t)n + (uint64_t)y) * (uint64_t)n + (uint64_t)x;
    return (double)(oracle_splitmix64(seed, idx) >> 40) * (1.0 / 16777216.0);
}

/* gamma rotated by 2 alpha: (g1 + i g2) exp(2 i alpha). */
void oracle_rotate_shear(const double *g1, const double *g2, double *o1, double *o2, int n, int r, uint64_t seed)
{
    for (int y = 0; y < n; ++y)
        for (int x = 0; x < n; ++x) {
            size_t i = (size_t)y * n + x;
            double two_alpha = 2.0 * M_PI * oracle_noise_u(seed, r, y, x, n);
            double c = cos(two_alpha), s = sin(two_alpha);
            o1[i] = g1[i] * c - g2[i] * s;
            o2[i] = g1[i] * s + g2[i] * c;
        }
}

/* sigma^2 of each band over R randomised realisations, by the textbook
 * two-pass unbiased sample variance (mean first, then squared deviations,
 * divided by R - 1); snr = w_j(data) / sigma_j (Sec. 1).  var_out and
 * snr_out are (J-1) n^2; snr_out may be NULL.  Holds all R realisations. */
void oracle_map_noise(const double *g1, const double *g2, double *var_out, double *snr_out, int n, int J, int R,
                      uint64_t seed, int boundary)
{
    size_t nn = (size_t)n * n;
    size_t nb = (size_t)(J - 1) * nn;
    double *pyr = (double *)malloc(sizeof(double) * (size_t)J * nn);
    double *all = (double *)malloc(sizeof(double) * nb * (size_t)R);
    double *r1 = (double *)malloc(sizeof(double) * nn);
    double *r2 = (double *)malloc(sizeof(double) * nn);
    for (int r = 0; r < R; ++r) {
        oracle_rotate_shear(g1, g2, r1, r2, n, r, seed);
        oracle_map_starlet(r1, r2, pyr, n, J, boundary);
        memcpy(all + (size_t)r * nb, pyr, sizeof(double) * nb);
    }
    for (size_t i = 0; i < nb; ++i) {
        double mean = 0.0;
        for (int r = 0; r < R; ++r) mean += all[(size_t)r * nb + i];
        mean /= (double)R;
        double ss = 0.0;
        for (int r = 0; r < R; ++r) {
            double d = all[(size_t)r * nb + i] - mean;
            ss += d * d;
        }
        var_out[i] = ss / (double)(R - 1);
    }
    if (snr_out) {
        oracle_map_starlet(g1, g2, pyr, n, J, boundary);
        for (size_t i = 0; i < nb; ++i) snr_out[i] = pyr[i] / sqrt(var_out[i]);
    }
    free(pyr);
    free(all);
    free(r1);
    free(r2);
}

/* Exact expectation of the noise variance (Sec. 1): with a uniform phase per
 * pixel, KS followed by starlet band j is (periodic boundary) the convolution
 * w_j(x) = sum_y Re[K_j(x - y) gamma(y)] with a complex kernel K_j, and
 *   Var[w_j(x)] = 1/2 sum_y |K_j(x - y)|^2 |gamma(y)|^2
 * because E[Re(z e^{i phi})^2] = |z|^2 / 2 and distinct pixels are
 * independent.  K_j is read off the pipeline's response to a unit shear at
 * pixel 0: Re K_j from gamma = (delta, 0), -Im K_j from gamma = (0, delta).
 * Evaluated at listed pixels; out[(j-1) * npts + p], j = 1..J-1.  Periodic
 * boundary only (the convolution form needs shift invariance). */
void oracle_map_noise_expected_at(const double *g1, const double *g2, const int *ys, const int *xs, int npts,
                                  double *out, int n, int J)
{
    size_t nn = (size_t)n * n;
    double *d = (double *)calloc(nn, sizeof(double));
    double *z = (double *)calloc(nn, sizeof(double));
    double *pa = (double *)malloc(sizeof(double) * (size_t)J * nn);
    double *pb = (double *)malloc(sizeof(double) * (size_t)J * nn);
    d[0] = 1.0;
    oracle_map_starlet(d, z, pa, n, J, 1);
    oracle_map_starlet(z, d, pb, n, J, 1);
    for (int j = 0; j < J - 1; ++j)
        for (int p = 0; p < npts; ++p) {
            int y = ys[p], x = xs[p];
            double acc = 0.0;
            for (int yy = 0; yy < n; ++yy)
                for (int xx = 0; xx < n; ++xx) {
                    /* offset x - y, wrapped onto the periodic grid */
                    int dy = ((y - yy) % n + n) % n, dx = ((x - xx) % n + n) % n;
                    size_t ki = (size_t)j * nn + (size_t)dy * n + dx;
                    double k2 = pa[ki] * pa[ki] + pb[ki] * pb[ki];
                    size_t gi = (size_t)yy * n + xx;
                    acc += k2 * (g1[gi] * g1[gi] + g2[gi] * g2[gi]);
                }
            out[(size_t)j * npts + p] = 0.5 * acc;
        }
    free(d);
    free(z);
    free(pa);
    free(pb);
}
