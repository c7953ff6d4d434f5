/*
 * fastmap.h -- C ABI of libfastmap, GB300 (sm_103a) fast aperture-mass maps.
 *
 * Implements the pipeline of Leonard, Pires & Starck, "Fast Calculation of
 * the Weak Lensing Aperture Mass Statistic" (MNRAS 2012):
 *   shear (gamma1, gamma2) --Kaiser-Squires in Fourier space (Sec. 4.5)-->
 *   convergence kappa --starlet / a trous B3-spline transform (Sec. 3,
 *   Sec. 4.2)--> aperture-mass maps w_j = c_{j-1} - c_j at theta = 2^j px;
 *   the brute-force direct M_ap of eq. shearmap (Sec. 2.1, Sec. 5.1) as the
 *   comparison path; and noise maps from randomly rotated shear (Sec. 1).
 *
 * Conventions shared by every entry point
 *   - Maps are square n x n, row-major, element (y, x) at [y*n + x]; x pairs
 *     with frequency k1, y with k2; a batch of maps is contiguous (map b at
 *     offset b*n*n).  Integer frequency of index i: i for i < n/2, else i - n.
 *   - A starlet pyramid holds J arrays of n*n per map: w_1 .. w_{J-1}, then
 *     the smooth array left after J-1 bands (the paper's c_J), so a batch of
 *     pyramids is [batch][J][n][n].  J counts arrays including the smooth one
 *     (Sec. 5.1); band j has aperture radius theta = 2^j pixels (Sec. 3).
 *   - Element type: float when cfg->precision == FM_F32 (default), double when
 *     FM_F64.  Noise variances are always double.
 *   - Data pointers are DEVICE pointers owned by the caller, except where an
 *     entry point says HOST.  The library keeps no reference after a call's
 *     work completes.  It owns only its scratch (stream-ordered allocations
 *     freed on the same stream) and small per-device tables (FFT twiddles),
 *     kept until process exit.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Every compute entry point is asynchronous on that stream: it
 *     returns once the work is queued.  The first call for a given n and
 *     precision builds a table with a synchronous copy, so make it before
 *     any CUDA-graph capture.
 *   - Return value: FM_OK (0) or a negative FM_E* code; nothing aborts and no
 *     C++ exception crosses the ABI.  fm_last_error() gives a message.
 *   - Validity: n >= 2^J and J >= 2 (Sec. 5.1: N >= 2^J); FFT-based entry
 *     points also need n a power of two, 4 <= n <= 8192.
 */
#ifndef FASTMAP_H
#define FASTMAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define FM_OK 0
#define FM_PENDING 1      /* serving: request not finished yet */
#define FM_EINVAL (-1)    /* bad size, J, filter, pointer or config */
#define FM_ENOMEM (-2)    /* device scratch allocation failed */
#define FM_EBUDGET (-3)   /* serving: request larger than the memory budget */
#define FM_ETIMEOUT (-4)  /* a bounded device wait gave up */
#define FM_ECUDA (-5)     /* a CUDA runtime call or kernel launch failed */
#define FM_ENOTFOUND (-6) /* serving: unknown ticket */
#define FM_EBUSY (-7)     /* serving: queue full */

/* ---- configuration ----------------------------------------------------- */
#define FM_F32 0
#define FM_F64 1
#define FM_MIRROR 0   /* whole-sample symmetric boundary (the paper states none) */
#define FM_PERIODIC 1

/* Direct M_ap filters (Sec. 4): starlet-shaped Q(eta)/theta^2 (default cut
 * 2 theta), S98 polynomial of order ell (eq. sch, cut theta), Gaussian of
 * eq. mexhat with A = 1 and b = 1/2 (JBJ04) or b = 4 (vW98), cut 5 theta. */
#define FM_FILTER_STARLET 0
#define FM_FILTER_S98 1
#define FM_FILTER_JBJ04 2
#define FM_FILTER_VW98 3

typedef struct {
    int precision;  /* FM_F32 (0) or FM_F64 (1) */
    int boundary;   /* starlet boundary: FM_MIRROR (0) or FM_PERIODIC (1) */
    int accum;      /* noise running sums: 0 = FP64, 1 = fp32 with Kahan
                       compensation (FM_F32 maps only); same scratch size */
    int fuse_depth; /* starlet scales done by the fused 2-D tile kernel:
                       0 = automatic (the autotuned plan, else 2 for fp32
                       maps of 512^2 to 2048^2 and 3 otherwise; see
                       fm_starlet_fuse_depth, fm_autotune), k > 0 = scales
                       1..k (at most 4 in fp32, 3 in fp64, J - 1), -1 = none
                       (the plain one-scale-per-pass form) */
    int large_path; /* scales after the fused ones: 0 = automatic (the
                       autotuned plan, else 4 where it applies after at
                       least two fused scales, 3 after fused small scales
                       on maps up to 256^2, 1 otherwise),
                       1 = one row pass + one column pass per scale, 2 = all
                       large scales in one row kernel + one column-strip
                       kernel, 3 = the column pass of each scale fused with
                       the row pass of the next (one row pass, then one
                       kernel per scale; the pyramid's smooth-array slot
                       serves as scratch until its final write), 4 = one
                       pass per scale that row-filters c_{j-1} from shared
                       memory (fp32, n a multiple of 512, scales with
                       spacing 4..128 px; otherwise the form 1) */
} fm_config;

/* ---- Kaiser-Squires (Sec. 4.5) ---------------------------------------------
 * Forward: gamma = IFFT(D FFT kappa); inverse: kappa = IFFT(conj(D) FFT gamma),
 * D(k) = (k1 + i k2)^2 / |k|^2, D(0) = 0 (standard KS; the paper names the
 * Fourier-space inversion without printing D).
 * fm_ks_invert: g1, g2 in [batch][n][n]; kappa_E (real part) out, kappa_B
 * (imaginary part, the B-mode) out or NULL.  fm_ks_forward: kappa in, g1, g2
 * out.  Scratch: batch*n*n complex. */
int fm_ks_invert(const void *g1, const void *g2, void *kappa_E, void *kappa_B, int n, int batch,
                 const fm_config *cfg, void *stream);
int fm_ks_forward(const void *kappa, void *g1, void *g2, int n, int batch, const fm_config *cfg, void *stream);

/* ---- starlet transform (Sec. 3, Sec. 4.2) -----------------------------------
 * kappa [batch][n][n] in, pyramid [batch][J][n][n] out (layout above).
 * Scale j filters rows then columns with h = [1,4,6,4,1]/16 at spacing
 * 2^(j-1) (the B3 two-scale filter) and stores w_j = c_{j-1} - c_j.
 * n need not be a power of two here (n >= 2^J).  kappa and pyramid must not
 * overlap.  Scratch: up to 2*batch*n*n elements. */
int fm_starlet_forward(const void *kappa, void *pyramid, int n, int J, int batch, const fm_config *cfg,
                       void *stream);

/* Number of scales the fused tile kernel computes for fm_starlet_forward /
 * fm_map_starlet with these n, J and cfg (0 = none); the remaining
 * J - 1 - depth scales take one row and one column pass each.  Host only;
 * FM_EINVAL on a bad n, J or cfg. */
int fm_starlet_fuse_depth(int n, int J, const fm_config *cfg);

/* KS inversion then the starlet of kappa_E: the aperture-mass maps of every
 * band from shear in one call (the paper's fast method end to end). */
int fm_map_starlet(const void *g1, const void *g2, void *pyramid, int n, int J, int batch, const fm_config *cfg,
                   void *stream);

/* Same as fm_map_starlet with HOST buffers (pinned host memory is fastest):
 * the batch streams through the library's chunk slots (see fm_tune) so that
 * each chunk's copy in, compute and copy out overlap those of the others;
 * the work forks from `stream` and joins back into it, so the results are in
 * pyramid_host once `stream` reaches that point, and the host buffers must
 * stay valid until then.  Device buffers are stream-ordered scratch of the
 * chunks in flight (not the whole batch). */
int fm_map_starlet_host(const void *g1_host, const void *g2_host, void *pyramid_host, int n, int J, int batch,
                        const fm_config *cfg, void *stream);

/* ---- direct aperture mass, eq. shearmap (Sec. 2.1), brute force (Sec. 5.1)
 * map(x) = sum over integer offsets d, 0 < |d| <= R, of Q(|d|) gamma_t(x+d),
 * gamma_t = -(gamma1 cos 2phi + gamma2 sin 2phi), phi the angle of d; pixels
 * outside the field add nothing.  R = cut_over_theta * theta_px, or the
 * filter's default cut when cut_over_theta <= 0.  ell is the S98 order.
 * One n x n map (n >= 1, any size).  Cost O(n^2 R^2). */
int fm_map_direct(const void *g1, const void *g2, void *map, int n, int filter, double theta_px, int ell,
                  double cut_over_theta, const fm_config *cfg, void *stream);

/* The same for a batch of maps [batch][n][n] in one launch (the maps share
 * the filter's weight table; small radii no longer leave most of the GPU
 * idle in the grid's last wave). */
int fm_map_direct_batch(const void *g1, const void *g2, void *map, int n, int batch, int filter, double theta_px,
                        int ell, double cut_over_theta, const fm_config *cfg, void *stream);

/* ---- direct M_ap with missing data (Sec. 4.3, Sec. 4.5) -----------------------
 * The paper notes that masks (bright stars, bad pixels) and field edges
 * leave pixels without data and that the brute-force aperture sum suffers
 * more the larger the aperture.  This call weights each pixel: weight[y][x]
 * >= 0, 0 for a masked pixel (a galaxy count or inverse variance also
 * works).  Over the lattice offsets 0 < |d| <= R inside the field,
 *   S(x) = sum w(x+d) Q(|d|) gamma_t(x+d; x),   D(x) = sum w(x+d),
 *   map(x) = N_R S(x) / D(x)  (0 where D(x) <= 0),
 *   coverage(x) = D(x) / N_R  (NULL: not written),
 * N_R = number of lattice offsets 0 < |d| <= R.  With all weights 1 and the
 * aperture inside the field this is fm_map_direct's value.  g1, g2, map and
 * coverage are [batch][n][n]; weight map b starts at weight + b *
 * weight_bstride elements (0: one weight map for the whole batch).  Element
 * type per cfg precision; R as in fm_map_direct and >= 1.  Arguments are
 * checked on the host (FM_EINVAL); weights are not read on the host. */
int fm_map_direct_masked(const void *g1, const void *g2, const void *weight, long weight_bstride, void *map,
                         void *coverage, int n, int batch, int filter, double theta_px, int ell,
                         double cut_over_theta, const fm_config *cfg, void *stream);

/* ---- noise maps by randomised shear (Sec. 1, Sec. 5.1) ------------------------
 * Realisation r rotates every pixel's shear by 2 alpha, alpha = pi u with u
 * the top 24 bits (times 2^-24) of SplitMix64 at counter (r*n + y)*n + x from
 * state `seed`; then KS + starlet.  var_out [(J-1)][n][n] (double) receives
 * the unbiased variance of each band over the R realisations (R >= 2);
 * snr_out (element type, same shape, or NULL) receives w_j(data)/sigma_j.
 * One map; n a power of two.  Realisations run in batches of up to 32 (the
 * batch's pyramids within 8 GiB); each batch goes through KS and the starlet
 * (bands only) in L2-sized chunks alternating over the library's streams,
 * then one pass adds its bands to the FP64 sums (or, with cfg->accum = 1,
 * to fp32 sums with Kahan compensation) while the chunks run on into the
 * next batch (two pyramid buffers).  The whole call is recorded once into a
 * CUDA graph (keyed by pointers, sizes, R, seed, config and chunk plan) and
 * replayed as one launch.  Scratch: 16 (J-1) bytes per pixel of sums, the
 * batches' pyramids and the chunks' intermediates, kept with the graph until
 * fm_trim or eviction. */
int fm_map_noise(const void *g1, const void *g2, double *var_out, void *snr_out, int n, int J, int R, uint64_t seed,
                 const fm_config *cfg, void *stream);

/* Noise maps in parts, for checkpoint / resume or realisations split over
 * GPUs.  fm_map_noise_accumulate adds realisations r0 .. r0 + R - 1 (the
 * generator of fm_map_noise) to `sums` = [2][J-1][n][n] doubles (S1 = sum w,
 * then S2 = sum w^2; zero them before the first part): sums from disjoint
 * ranges add, on one device or after copying between devices.  Runs on the
 * caller's stream with stream-ordered scratch (the batches' pyramids and the
 * chunks' intermediates; none for the sums, which are the caller's);
 * cfg->accum must be 0.
 * fm_noise_finalize turns sums of R_total >= 2 realisations into the
 * variance var_out [(J-1)][n][n] (double) and, when snr_out is given, S/N =
 * w_j(data) / sigma_j from the data's pyramid [J][n][n] (fm_map_starlet of the
 * same map, element type).  `sums` must be exactly the [2][J-1][n][n]
 * doubles that fm_map_noise_accumulate wrote for the same n and J (n a power
 * of two in [4, 8192], FM_EINVAL otherwise: the C ABI cannot check the
 * buffer's length).  The variance equals fm_map_noise's up to the grouping
 * of the fp32 partial sums (~1e-7 relative). */
int fm_map_noise_accumulate(const void *g1, const void *g2, double *sums, int n, int J, int r0, int R, uint64_t seed,
                            const fm_config *cfg, void *stream);
int fm_noise_finalize(const double *sums, const void *pyramid, double *var_out, void *snr_out, int n, int J,
                      int R_total, const fm_config *cfg, void *stream);

/* ---- exact expected noise variance (Sec. 1) -----------------------------------
 * The expectation of fm_map_noise's variance over the random rotation: with a
 * uniform phase per pixel, Var[w_j(x)] = 1/2 sum_y |K_j(x - y)|^2 |gamma(y)|^2,
 * K_j the complex kernel of KS followed by band j.  One FFT pipeline instead
 * of R realisations; not the paper's Monte-Carlo procedure but its limit.
 * Needs the periodic boundary (cfg->boundary = FM_PERIODIC; mirror edges make
 * the pipeline position dependent, FM_EINVAL).  var_out [(J-1)][n][n] in the
 * element type of cfg->precision; one map; n a power of two.  Scratch:
 * about (2J + 6J) n^2 elements, stream-ordered. */
int fm_map_noise_expected(const void *g1, const void *g2, void *var_out, int n, int J, const fm_config *cfg,
                          void *stream);

/* ---- Kaiser-Squires inversion without device allocation --------------------
 * No counterpart in the paper: an engineering variant of fm_ks_invert for
 * callers that cannot allocate device memory where they run the inversion
 * (their device memory is reserved up front by another framework's pool, or
 * the code path must never enter the allocator).  Same arguments, layout and
 * results as fm_ks_invert, FM_F32 only (cfg NULL or a valid config with
 * precision FM_F32), n a power of two in [32, 2048], batch * n^2 <= 4194304
 * (so a batch of one 2048^2 map, four of 1024^2, ...).  The FFT work buffer
 * and twiddle tables are file-scope device arrays (32 MiB + 32 KiB per
 * device); this entry point calls no cudaMalloc, cudaFree or other
 * allocating routine.  The driver allocates the arrays when it loads their
 * module on a device: with CUDA's default lazy module loading that is the
 * first call on that device, so make the first call before another pool
 * reserves the device's memory (and before any stream capture); the arrays
 * stay allocated until the process exits.  Larger sizes return FM_EINVAL.
 * The first call on each device also sets up (looks up the arrays' device
 * addresses and copies the twiddle tables synchronously) with that device
 * current.  All calls share the one work buffer, which keeps the last
 * call's contents (every call overwrites all of the part it uses, so nothing
 * needs clearing); calls whose work overlaps on the GPU race on it and must
 * be ordered by the caller, e.g. by issuing them on one stream. */
int fm_ks_invert_noalloc(const void *g1, const void *g2, void *kappa_E, void *kappa_B, int n, int batch,
                         const fm_config *cfg, void *stream);

/* ---- statistics of the aperture-mass maps (Sec. 2.2) ----------------------------
 * For every map b and pyramid array j of pyramid [batch][J][n][n] (any n),
 * moments[(b*J + j)*4 + 0..3] = mean, variance <M_ap^2> (over the n^2
 * pixels, divided by n^2), skewness and excess kurtosis.  Two passes; fp32
 * partial sums of at most ~16 pixels per thread, FP64 across threads. */
int fm_band_moments(const void *pyramid, double *moments, int n, int J, int batch, const fm_config *cfg,
                    void *stream);

/* ---- serving: continuous batching of map requests -------------------------- */
typedef struct {
    int n, J, R;          /* R = 0: pyramid only; R >= 2: also noise variance */
    uint64_t seed;
    int precision;        /* FM_F32 or FM_F64 */
    const void *g1, *g2;  /* device input, borrowed until the request finishes */
    void *out_pyramid;    /* device [J][n][n], element type */
    double *out_var;      /* device [(J-1)][n][n] or NULL (needs R >= 2) */
} fm_request;

typedef struct {
    int status;           /* FM_PENDING, FM_OK or a negative code */
    int64_t t_submit_ns, t_admit_ns, t_done_ns; /* steady-clock times */
} fm_result;

/* A server owns a host thread, max_slots CUDA streams and the scratch of the
 * requests it runs.  A request is admitted when a slot is free and its
 * scratch fits in mem_budget_bytes minus the scratch of running requests;
 * requests run concurrently on their own streams.  A pyramid-only request
 * (R = 0) of a map up to 1024^2 at the head of the queue takes the queued
 * requests of the same n, J and precision with it (at most
 * FM_TUNE_SERVE_MERGE maps, within the budget): they run as one batched
 * call on one slot (inputs gathered and pyramids scattered by one
 * device-to-device copy per request), with results identical to running
 * alone.  Heavy requests (n^2 J (1 + R) >= 2^32 pixel-scales) run at most
 * FM_TUNE_SERVE_HEAVY at a time; light requests queued behind a waiting heavy
 * one are admitted past it.  submit copies the request descriptor (device
 * buffers are borrowed) and returns a ticket. */
int fm_serve_create(size_t mem_budget_bytes, int max_slots, void **server);
int fm_serve_submit(void *server, const fm_request *req, uint64_t *ticket);
int fm_serve_poll(void *server, uint64_t ticket, fm_result *result);
int fm_serve_wait(void *server, uint64_t ticket, fm_result *result, double timeout_s);
int fm_serve_destroy(void *server);
size_t fm_request_scratch_bytes(const fm_request *req);

/* ---- diagnostics ------------------------------------------------------------- */
const char *fm_status_string(int status);
const char *fm_last_error(void);   /* message of the calling thread's last error */
int64_t fm_launch_count(void);     /* kernels launched by this library so far */
/* Device allocations this library has made (stream-ordered scratch, graph
 * scratch, twiddle tables, the autotuner's buffers) since the last reset:
 * their number and the largest one in bytes; reset != 0 zeroes both after
 * reading.  Either pointer may be NULL. */
int fm_alloc_stats(int64_t *count, int64_t *max_bytes, int reset);
/* Memory-side rates on the current device for a working set of `bytes`
 * (two buffers of bytes / 2; 32 MiB stays in L2, a few GiB streams from
 * HBM): GB/s of a streaming float4 read of one buffer and of a copy of one
 * into the other (read + written bytes), `reps` sweeps in one launch each.
 * Allocates and frees the buffers; synchronises.  A measurement aid for the
 * rooflines, not part of the method. */
int fm_measure_bandwidth(size_t bytes, int reps, double *read_gbs, double *copy_gbs);
/* 1 if the inverse KS of n x n fp32 maps without kappa_B takes the
 * real-output path (half spectrum) under the current FM_TUNE_KS_REAL
 * setting, 0 if the complex one; batched != 0 asks for the chunks of
 * fm_map_starlet / fm_map_noise, 0 for fm_ks_invert. */
int fm_ks_real_output(int n, int batched);
/* 1 if a kernel on the current device gave up waiting for a bulk tensor copy
 * (an iteration-bounded wait that ran out; its outputs are then missing),
 * else 0; clears the flag.  Synchronises with the device.  FM_EINVAL if no
 * device is usable. */
int fm_device_error(void);

/* Tuning knobs (process-wide; value < 0 restores the default):
 *   FM_TUNE_CHUNK_BYTES  budget of one chunk's intermediates in batched
 *                        KS + starlet calls (3 n^2 values a map: the FFT
 *                        work buffer, which also holds the starlet's scratch
 *                        maps, and kappa; default 48 MiB, four 1024^2 fp32
 *                        maps, so two chunks in flight stay in L2); 0 = no
 *                        chunking
 *   FM_TUNE_GRAPHS       1 = replay batched calls from cached CUDA graphs
 *                        (default), 0 = launch every kernel each call
 *   FM_TUNE_CHUNK_STREAMS number of streams chunks alternate on (1 to 4,
 *                        default 2)
 *   FM_TUNE_PDL          1 = launch kernels as programmatic dependents of
 *                        the previous kernel in their stream (default), 0 = off
 *   FM_TUNE_TMA          mask of the loads done by bulk tensor copies (TMA)
 *                        instead of per-thread loads: 1 = the halo of the
 *                        fused small-scale starlet tiles, 2 = the input rows
 *                        of the row FFT, 4 = those of the row inverse FFT,
 *                        8 / 16 = the window rows / the c_{j-1} rows of the
 *                        large-scale column pass (fp32 maps of 4096^2 and
 *                        up), 32 = the column strips of the column FFT
 *                        (n >= 1024), 64 = their stores (n = 8192);
 *                        default 127
 *   FM_TUNE_TILE         fp32 kernel of the fused small starlet scales:
 *                        0 = row-filtered shared buffer, 1 = register
 *                        window; default: the autotuned plan's, else 1
 *   FM_TUNE_WAIT_TEST    test hook of the bounded-wait path: 1 = the fused
 *                        tile kernel's halo copy announces 16 bytes more than
 *                        it delivers, so every interior tile's wait runs out
 *                        (within about 0.1 s), the tile leaves its outputs
 *                        unwritten and fm_device_error reports 1; 0 = off
 *                        (default)
 *   FM_TUNE_DIRECT       kernel of the fp32 direct M_ap without weights:
 *                        0 = scalar FMAs with synchronous row staging,
 *                        1 = packed two-lane FMAs with asynchronous row
 *                        staging, 4 rows x 8 columns per lane, 4 warps;
 *                        2, 3, 4 = the same with 2 x 8 per lane and 4 warps,
 *                        4 x 8 and 2 warps, 2 x 8 and 8 warps; default: 2
 *                        below a 48-pixel cut radius, else 3
 *   FM_TUNE_KS_REAL      inverse KS without kappa_B: 1 = compute only the
 *                        Hermitian half of kappa_E's spectrum (real-output
 *                        column and row passes; fp32, n >= 64, kappa_E
 *                        16-byte aligned), 0 = the complex inverse and its
 *                        real part; default: the real output from
 *                        n = 512 up, in fm_ks_invert and in the batched
 *                        pipeline's chunks (where it measured faster)
 *   FM_TUNE_SERVE_MERGE  servers: most maps that one merged run of queued
 *                        pyramid-only requests (R = 0, n <= 1024) of one
 *                        shape may hold (default 16; 1 = every request runs
 *                        alone)
 *   FM_TUNE_SERVE_HEAVY  servers: heavy requests (n^2 J (1 + R) >= 2^32
 *                        pixel-scales) running at once (default 1; 0 = no
 *                        limit); light requests queued behind a waiting heavy
 *                        one are admitted past it
 * FM_TUNE_CHUNK_BYTES set this way also overrides autotuned budgets. */
#define FM_TUNE_CHUNK_BYTES 1
#define FM_TUNE_GRAPHS 2
#define FM_TUNE_CHUNK_STREAMS 3
#define FM_TUNE_PDL 4
#define FM_TUNE_TILE 5
#define FM_TUNE_TMA 6
#define FM_TUNE_WAIT_TEST 7
#define FM_TUNE_DIRECT 8
#define FM_TUNE_KS_REAL 9
#define FM_TUNE_SERVE_MERGE 10
#define FM_TUNE_SERVE_HEAVY 11
int fm_tune(int knob, int64_t value);

/* ---- autotuner ----------------------------------------------------------------
 * fm_autotune times fm_map_starlet on `batch` synthetic n x n maps (J scales,
 * cfg->precision and cfg->boundary; cfg's fuse_depth and large_path are
 * ignored) for candidate plans, by coordinate descent from the built-in rules
 * over: fused depth 1..4 (fp64 1..3, at most J - 1), large-scale path 1 or 3,
 * fp32 tile kernel form (1 = register window, 0 = shared buffer) and chunk
 * budget 40 / 60 / 80 / 120 MiB; a candidate replaces the best so far only
 * when 1 % faster.  The winner goes into a process-wide table keyed by
 * (n, J, precision), which the automatic fields (fuse_depth = 0,
 * large_path = 0) and the default tile form and chunk budget then follow
 * (knobs set by fm_tune keep precedence).  fm_autotune allocates its own
 * buffers, synchronises with the device and drops the cached graphs; do not
 * run it concurrently with other calls.  `best` (may be NULL) receives the
 * plan, its time and the built-in plan's time.
 * fm_autotune_get: FM_ENOTFOUND if the table has no entry.  fm_autotune_set
 * enters a plan by hand (validated).  fm_autotune_save writes the table as
 * JSON ({"fastmap_autotune": 1, "entries": [{"n", "J", "precision",
 * "fuse_depth", "large_path", "tile", "chunk_mb", "ms", "default_ms"}]});
 * fm_autotune_load merges such a file (nothing changes if it is malformed:
 * FM_EINVAL); fm_autotune_clear empties the table.  Host only except
 * fm_autotune. */
typedef struct {
    int fuse_depth; /* scales of the fused tile kernel */
    int large_path; /* 1, 3 or 4 (see fm_config) */
    int tile;       /* fp32 tile kernel: 1 = register window, 0 = shared buffer */
    int chunk_mb;   /* chunk budget of batched calls, MiB (0 = the default) */
    double ms;         /* fm_map_starlet with this plan, per call (tuning batch) */
    double default_ms; /* the same with the built-in rules */
} fm_plan;
int fm_autotune(int n, int J, int batch, const fm_config *cfg, fm_plan *best);
int fm_autotune_get(int n, int J, int precision, fm_plan *plan);
int fm_autotune_set(int n, int J, int precision, const fm_plan *plan);
int fm_autotune_save(const char *path);
int fm_autotune_load(const char *path);
int fm_autotune_clear(void);

/* Batched fm_map_starlet calls (when chunked) and fm_map_noise calls are
 * recorded once into CUDA graphs that keep their scratch (a few per kind,
 * least recently used dropped first).  fm_trim waits for the device and
 * frees all of them. */
int fm_trim(void);

/* Kernel ids for fm_profile_select. */
#define FM_K_FFT_ROWS_FWD 1
#define FM_K_FFT_COLS_KS 2
#define FM_K_FFT_ROWS_INV 3
#define FM_K_STARLET_TILE 4
#define FM_K_STARLET_ROW 5
#define FM_K_STARLET_COL 6
#define FM_K_MAP_DIRECT 7
#define FM_K_NOISE_FINAL 8
#define FM_K_NOISE_ACCUM 9
#define FM_K_STARLET_COLROW 10 /* a large scale's column pass + the next scale's row pass */

/* Bracket every later launch of kernel `kid` (0 = none) with CUDA events on
 * its launch stream; fm_profile_read synchronises those events and returns
 * the summed device time (ms) and the launch count since the selection. */
int fm_profile_select(int kid);
int fm_profile_read(double *total_ms, int64_t *launches);

#ifdef __cplusplus
}
#endif
#endif /* FASTMAP_H */
