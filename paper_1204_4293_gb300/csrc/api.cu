// api.cu -- the compute entry points of libfastmap's C ABI (declared in
// include/fastmap.h): argument validation, scratch sizing and dispatch to
// the kernels and to the batched pipeline.
#include <math.h>
#include <string.h>

#include <string>

#include "common.cuh"

namespace fm {

static fm_config cfg_or_default(const fm_config *c)
{
    fm_config d;
    memset(&d, 0, sizeof(d));
    if (c) d = *c;
    return d;
}

int check_config(const fm_config &c)
{
    if (c.precision != FM_F32 && c.precision != FM_F64) return einval("precision must be FM_F32 or FM_F64");
    if (c.boundary != FM_MIRROR && c.boundary != FM_PERIODIC) return einval("boundary must be FM_MIRROR or FM_PERIODIC");
    if (c.accum != 0 && c.accum != 1) return einval("accum must be 0 (FP64 sums) or 1 (Kahan fp32 sums)");
    if (c.accum == 1 && c.precision != FM_F32) return einval("accum = 1 (Kahan fp32 sums) needs FM_F32 maps");
    if (c.fuse_depth < -1 || c.fuse_depth > 8) return einval("fuse_depth out of range [-1, 8]");
    if (c.large_path < 0 || c.large_path > 4) return einval("large_path must be 0, 1, 2, 3 or 4");
    return FM_OK;
}

static size_t esize(const fm_config &c) { return c.precision == FM_F64 ? 8 : 4; }

static int check_fft_n(int n)
{
    if (n < 4 || n > 8192 || !is_pow2(n)) return einval("n must be a power of two in [4, 8192]");
    return FM_OK;
}

static int check_J(int n, int J)
{
    if (J < 2 || J > 20) return einval("J must be in [2, 20]");
    if ((long)n < (1L << J)) return einval("n must be >= 2^J (N >= 2^J)");
    return FM_OK;
}


size_t map_starlet_scratch_bytes(int n, int J, int batch, const fm_config &cfg)
{
    // the FFT work buffer (2 n^2 a map) and kappa (n^2); the starlet's
    // scratch maps live in the work buffer when they fit there (the chunk
    // plan's rule), else in their own buffer
    const size_t es = esize(cfg), nn = (size_t)n * n;
    const size_t st = starlet_scratch_elems(n, J, 1, cfg) <= 2 * nn ? 0 : starlet_scratch_elems(n, J, batch, cfg) * es;
    return (size_t)batch * nn * 3 * es + st + 3 * 256;
}

}  // namespace fm

using namespace fm;

extern "C" {

int fm_ks_invert(const void *g1, const void *g2, void *kappa_E, void *kappa_B, int n, int batch, const fm_config *cfgp,
                 void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if (batch < 1) return einval("batch must be >= 1");
    if (!g1 || !g2 || !kappa_E) return einval("null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch work;
    const size_t bytes = (size_t)batch * n * n * 2 * esize(cfg);
    if ((st = scratch_alloc(work, bytes, s))) return st;
    return launch_ks(g1, g2, (long)n * n, kappa_E, kappa_B, work.p, n, batch, cfg.precision, false, 0, 0, false, s);
}

int fm_ks_forward(const void *kappa, void *g1, void *g2, int n, int batch, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if (batch < 1) return einval("batch must be >= 1");
    if (!kappa || !g1 || !g2) return einval("null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch work;
    if ((st = scratch_alloc(work, (size_t)batch * n * n * 2 * esize(cfg), s))) return st;
    return launch_ks(kappa, nullptr, (long)n * n, g1, g2, work.p, n, batch, cfg.precision, true, 0, 0, false, s);
}

int fm_starlet_forward(const void *kappa, void *pyramid, int n, int J, int batch, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (n < 1) return einval("n must be >= 1");
    if ((st = check_J(n, J))) return st;
    if (batch < 1) return einval("batch must be >= 1");
    if (!kappa || !pyramid) return einval("null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc;
    if ((st = scratch_alloc(sc, starlet_scratch_elems(n, J, batch, cfg) * esize(cfg), s))) return st;
    return launch_starlet(kappa, pyramid, (long)J * n * n, n, J, batch, cfg, sc.p, s);
}

int fm_starlet_fuse_depth(int n, int J, const fm_config *cfgp)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (n < 1) return einval("n must be >= 1");
    if ((st = check_J(n, J))) return st;
    return starlet_fuse_depth(n, J, cfg);
}

int fm_map_starlet(const void *g1, const void *g2, void *pyramid, int n, int J, int batch, const fm_config *cfgp,
                   void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (batch < 1) return einval("batch must be >= 1");
    if (!g1 || !g2 || !pyramid) return einval("null pointer");
    return map_starlet_run(g1, g2, pyramid, n, J, batch, cfg, (cudaStream_t)stream);
}

int fm_map_starlet_host(const void *g1_host, const void *g2_host, void *pyramid_host, int n, int J, int batch,
                        const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (batch < 1) return einval("batch must be >= 1");
    if (!g1_host || !g2_host || !pyramid_host) return einval("null pointer");
    return map_starlet_host_run(static_cast<const char *>(g1_host), static_cast<const char *>(g2_host),
                                static_cast<char *>(pyramid_host), n, J, batch, cfg, (cudaStream_t)stream);
}

int fm_map_direct(const void *g1, const void *g2, void *map, int n, int filter, double theta_px, int ell,
                  double cut_over_theta, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (n < 1 || n > 65536) return einval("n must be in [1, 65536]");
    if (filter < FM_FILTER_STARLET || filter > FM_FILTER_VW98) return einval("unknown filter");
    if (!(theta_px > 0) || theta_px > 4096) return einval("theta_px must be in (0, 4096]");
    if (filter == FM_FILTER_S98 && (ell < 0 || ell > 64)) return einval("ell must be in [0, 64]");
    const double cut = cut_over_theta > 0 ? cut_over_theta : 0.0;
    const double R = (cut > 0 ? cut : (filter == FM_FILTER_STARLET ? 2.0 : filter == FM_FILTER_S98 ? 1.0 : 5.0)) *
                     theta_px;
    if (R > 2048) return einval("cut radius above 2048 px");
    if (!g1 || !g2 || !map) return einval("null pointer");
    return launch_map_direct(g1, g2, nullptr, 0, map, nullptr, n, 1, filter, theta_px, ell, cut, cfg.precision,
                             (cudaStream_t)stream);
}

int fm_map_direct_batch(const void *g1, const void *g2, void *map, int n, int batch, int filter, double theta_px,
                        int ell, double cut_over_theta, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (n < 1 || n > 65536) return einval("n must be in [1, 65536]");
    if (batch < 1 || batch > 65535) return einval("batch must be in [1, 65535]");
    if (filter < FM_FILTER_STARLET || filter > FM_FILTER_VW98) return einval("unknown filter");
    if (!(theta_px > 0) || theta_px > 4096) return einval("theta_px must be in (0, 4096]");
    if (filter == FM_FILTER_S98 && (ell < 0 || ell > 64)) return einval("ell must be in [0, 64]");
    const double cut = cut_over_theta > 0 ? cut_over_theta : 0.0;
    const double R = (cut > 0 ? cut : (filter == FM_FILTER_STARLET ? 2.0 : filter == FM_FILTER_S98 ? 1.0 : 5.0)) *
                     theta_px;
    if (R > 2048) return einval("cut radius above 2048 px");
    if (!g1 || !g2 || !map) return einval("null pointer");
    return launch_map_direct(g1, g2, nullptr, 0, map, nullptr, n, batch, filter, theta_px, ell, cut, cfg.precision,
                             (cudaStream_t)stream);
}

int fm_map_direct_masked(const void *g1, const void *g2, const void *weight, long weight_bstride, void *map,
                         void *coverage, int n, int batch, int filter, double theta_px, int ell,
                         double cut_over_theta, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (n < 1 || n > 65536) return einval("n must be in [1, 65536]");
    if (batch < 1 || batch > 65535) return einval("batch must be in [1, 65535]");
    if (weight_bstride < 0) return einval("weight_bstride must be >= 0");
    if (filter < FM_FILTER_STARLET || filter > FM_FILTER_VW98) return einval("unknown filter");
    if (!(theta_px > 0) || theta_px > 4096) return einval("theta_px must be in (0, 4096]");
    if (filter == FM_FILTER_S98 && (ell < 0 || ell > 64)) return einval("ell must be in [0, 64]");
    const double cut = cut_over_theta > 0 ? cut_over_theta : 0.0;
    const double R = (cut > 0 ? cut : (filter == FM_FILTER_STARLET ? 2.0 : filter == FM_FILTER_S98 ? 1.0 : 5.0)) *
                     theta_px;
    if (R > 2048) return einval("cut radius above 2048 px");
    if (R < 1) return einval("cut radius below one pixel: the aperture holds no pixel");
    if (!g1 || !g2 || !weight || !map) return einval("null pointer");
    return launch_map_direct(g1, g2, weight, weight_bstride, map, coverage, n, batch, filter, theta_px, ell, cut,
                             cfg.precision, (cudaStream_t)stream);
}

// Noise maps (Sec. 1): one unrotated pass for w_j(data), then R rotated
// realisations in chunks, each chunk a batch through KS and the starlet with
// the bands accumulated into FP64 S1, S2; then the finalize kernel.
int fm_map_noise(const void *g1, const void *g2, double *var_out, void *snr_out, int n, int J, int R, uint64_t seed,
                 const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (R < 2) return einval("R must be >= 2");
    if (!g1 || !g2 || !var_out) return einval("null pointer");
    return map_noise_run(g1, g2, var_out, snr_out, n, J, R, seed, cfg, (cudaStream_t)stream, true);
}

// Noise maps in parts (checkpoint and resume, or realisations split over
// GPUs): realisations r0 .. r0 + R - 1 added to the caller's FP64 sums, and
// the variance (and S/N) from sums of R_total realisations.
int fm_map_noise_accumulate(const void *g1, const void *g2, double *sums, int n, int J, int r0, int R, uint64_t seed,
                            const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (cfg.accum != 0) return einval("fm_map_noise_accumulate keeps FP64 sums (accum = 0)");
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (R < 1 || r0 < 0 || (long)r0 + R > 2147483647L) return einval("need R >= 1, r0 >= 0, r0 + R < 2^31");
    if (!g1 || !g2 || !sums) return einval("null pointer");
    return map_noise_accumulate_run(g1, g2, sums, n, J, r0, R, seed, cfg, (cudaStream_t)stream);
}

int fm_noise_finalize(const double *sums, const void *pyramid, double *var_out, void *snr_out, int n, int J,
                      int R_total, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (cfg.accum != 0) return einval("fm_noise_finalize reads FP64 sums (accum = 0)");
    if ((st = check_fft_n(n))) return st;  // the sizes fm_map_noise_accumulate produces sums for
    if ((st = check_J(n, J))) return st;
    if (R_total < 2) return einval("R_total must be >= 2");
    if (!sums || !var_out) return einval("null pointer");
    if (snr_out && !pyramid) return einval("S/N needs the data's pyramid");
    return launch_noise_finalize(sums, snr_out ? pyramid : nullptr, var_out, snr_out, (long)(J - 1) * n * n,
                                 R_total, cfg.precision, 0, (cudaStream_t)stream);
}

// Exact expected noise variance (Sec. 1), periodic boundary:
// Var_j = 1/2 |K_j|^2 (*) |gamma|^2 (circular convolution).  K_j is the
// pipeline's response to unit shears at pixel 0 (Re K_j from gamma1, -Im K_j
// from gamma2); the convolution runs through the FFT pipeline: the spectra of
// |K_j|^2, then rows FFT of |gamma|^2 (broadcast to the J - 1 bands) -> columns
// FFT -> times the band's spectrum -> inverse -> real part / 2.
int fm_map_noise_expected(const void *g1, const void *g2, void *var_out, int n, int J, const fm_config *cfgp,
                          void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (cfg.boundary != FM_PERIODIC)
        return einval("fm_map_noise_expected needs cfg->boundary = FM_PERIODIC: with mirror edges KS + starlet is "
                      "not a convolution");
    if (!g1 || !g2 || !var_out) return einval("null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    const int prec = cfg.precision;
    const size_t es = prec == FM_F64 ? 8 : 4;
    const long nn = (long)n * n;
    const int nb = J - 1;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t b_delta = up(2 * nn * es), b_pyr = up((size_t)2 * J * nn * es), b_q = up((size_t)nb * nn * es),
                 b_p = up(nn * es), b_spec = up((size_t)nb * nn * 2 * es);
    Scratch sc;
    if ((st = scratch_alloc(sc, 2 * b_delta + b_pyr + b_q + b_p + 2 * b_spec, s))) return st;
    char *base = static_cast<char *>(sc.p);
    char *g1d = base, *g2d = g1d + b_delta, *pyr = g2d + b_delta, *q = pyr + b_pyr, *p = q + b_q, *spec = p + b_p,
         *work = spec + b_spec;
    if ((st = launch_unit_shears(g1d, g2d, nn, prec, s))) return st;
    if ((st = map_starlet_run(g1d, g2d, pyr, n, J, 2, cfg, s))) return st;
    // |K_j|^2 = (Re K_j)^2 + (Im K_j)^2 from the two responses [2][J][n][n]
    if ((st = launch_modulus2(pyr, nn, pyr + (size_t)J * nn * es, nn, q, nn, nb, prec, s))) return st;
    if ((st = launch_modulus2(g1, 0, g2, 0, p, nn, 1, prec, s))) return st;
    if ((st = launch_fft_op(q, nullptr, nn, nullptr, nullptr, spec, n, nb, prec, FFT_OP_SPECTRUM, nullptr, 1.0, 0, 0,
                            false, s)))
        return st;
    return launch_fft_op(p, nullptr, 0, var_out, nullptr, work, n, nb, prec, FFT_OP_FILTER, spec, 0.5, 0, 0, false, s);
}

int fm_band_moments(const void *pyramid, double *moments, int n, int J, int batch, const fm_config *cfgp,
                    void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_config(cfg);
    if (st) return st;
    if (n < 1 || n > 65536) return einval("n must be in [1, 65536]");
    if (J < 1 || J > 20) return einval("J must be in [1, 20]");
    if (batch < 1 || batch > 65535) return einval("batch must be in [1, 65535]");
    if (!pyramid || !moments) return einval("null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Scratch sc;
    if ((st = scratch_alloc(sc, sizeof(double) * 4 * (size_t)batch * J, s))) return st;
    return launch_band_moments(pyramid, moments, n, J, batch, cfg.precision, sc.p, s);
}

}  // extern "C"
