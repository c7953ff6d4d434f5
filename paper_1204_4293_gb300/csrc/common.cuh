// common.cuh -- shared device/host helpers of libfastmap (CUDA, sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <utility>

#include "../../include/fastmap.h"

namespace fm {

// ---- error reporting --------------------------------------------------------
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define FM_CUDA_TRY(call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return fm::cuda_fail(e_, #call); \
    } while (0)

#define FM_CHECK_LAUNCH(name)                                        \
    do {                                                             \
        cudaError_t e_ = cudaGetLastError();                         \
        if (e_ != cudaSuccess) return fm::cuda_fail(e_, name);       \
    } while (0)

// ---- launch accounting and optional per-kernel event timing -----------------
extern std::atomic<int64_t> g_launches;
void prof_before(int kid, cudaStream_t s);
void prof_after(int kid, cudaStream_t s);

// Programmatic dependent launch: every kernel of the library starts with
// pdl_entry(), which waits until the kernel it depends on in the stream has
// finished (a no-op when launched without the attribute) and then lets the
// next kernel's CTAs be scheduled into SMs this grid leaves idle in its tail.
extern std::atomic<int> g_pdl;
// fp32 fused-scale tile kernel: 0 = shared row-filtered buffer, 1 = register
// window, -1 = automatic (the autotuned plan, else the register window)
extern std::atomic<int> g_tile_variant;
// bulk tensor copies (mask): 1 = starlet tile halo, 2 = row FFT input rows,
// 4 = row IFFT input rows, 8 = large-scale column window rows, 16 = its
// c_{j-1} rows (the last two on maps of 4096^2 and up), 32 = the column
// FFT's strips (n >= 1024), 64 = their stores (n = 8192)
constexpr int kDefaultTma = 127;
extern std::atomic<int> g_use_tma;
extern std::atomic<int> g_prof_kid;  // kernel id whose launches are being timed (0: none)
// test hook (FM_TUNE_WAIT_TEST): the fused tile kernel's bulk copy waits for
// more bytes than arrive, so its bounded wait runs out and is flagged
extern std::atomic<int> g_wait_test;
// kernel form of the unmasked fp32 direct M_ap (FM_TUNE_DIRECT)
extern std::atomic<int> g_direct_form;
// 1 if a kernel of that file gave up waiting on a bulk copy (see fm_device_error)
int starlet_wait_error(bool clear);
int fft_wait_error(bool clear);
int einval(const std::string &msg);  // records msg as the last error, returns FM_EINVAL
__device__ __forceinline__ void pdl_entry()
{
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    cudaGridDependencySynchronize();
    cudaTriggerProgrammaticLaunchCompletion();
#endif
}

template <typename... KArgs, typename... Args>
cudaError_t launch_ex(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = g_pdl.load(std::memory_order_relaxed) ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch helper: counts the launch, brackets it with profiling events when
// that kernel id is selected, and checks the launch status.
#define FM_LAUNCH(kid, kernel, grid, block, smem, stream, ...)                              \
    do {                                                                                    \
        fm::prof_before(kid, stream);                                                       \
        cudaError_t le_ = fm::launch_ex(kernel, dim3(grid), dim3(block), smem, stream, __VA_ARGS__); \
        fm::g_launches.fetch_add(1, std::memory_order_relaxed);                             \
        if (le_ != cudaSuccess) return fm::cuda_fail(le_, #kernel);                          \
        fm::prof_after(kid, stream);                                                        \
    } while (0)

// ---- complex helpers ----------------------------------------------------------
template <typename T> struct cplx;
template <> struct cplx<float> { using type = float2; };
template <> struct cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename cplx<T>::type;

template <typename V> __host__ __device__ __forceinline__ V cmake(decltype(V::x) a, decltype(V::x) b)
{
    V v;
    v.x = a;
    v.y = b;
    return v;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return cmake<V>(a.x * s, a.y * s); }
// fp32: one packed two-lane instruction each (add.rn.f32x2; a - b as
// fma.rn.f32x2(b, -1, a), exact in the product, so the same rounding as the
// scalar forms)
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// ---- index folding at the map edge ------------------------------------------------
// Mirror: whole-sample symmetric extension (period 2(n-1)); periodic: mod n.
__host__ __device__ __forceinline__ int fold_mirror(int i, int n)
{
    if (n == 1) return 0;
    // reflect about 0 and n-1 until inside; one reflection covers offsets up
    // to n - 1, which every caller's halo (<= n / 2 + tile halo) meets except
    // on the smallest maps
    while (i < 0 || i >= n) {
        if (i < 0) i = -i;
        if (i >= n) i = 2 * (n - 1) - i;
    }
    return i;
}
__host__ __device__ __forceinline__ int fold_periodic(int i, int n)
{
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}
__host__ __device__ __forceinline__ int fold_index(int i, int n, int boundary)
{
    return boundary == FM_PERIODIC ? fold_periodic(i, n) : fold_mirror(i, n);
}

__host__ __device__ __forceinline__ int ilog2(unsigned v)
{
    int r = 0;
    while ((1u << (r + 1)) <= v) ++r;
    return r;
}
__host__ __device__ __forceinline__ bool is_pow2(long v) { return v > 0 && (v & (v - 1)) == 0; }

// ---- per-device tables and scratch (api.cu) ---------------------------------------
// Twiddles exp(-2 pi i t / n), t = 0..n-1, computed on the host in FP64.
const void *twiddles(int n, int precision, cudaStream_t s, int *status);

struct Scratch {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~Scratch()
    {
        if (p) cudaFreeAsync(p, s);
    }
};
int scratch_alloc(Scratch &sc, size_t bytes, cudaStream_t s);
// cudaMalloc, counted by fm_alloc_stats (graph scratch, tables, tuner buffers)
cudaError_t dev_malloc(void **p, size_t bytes);
// the checks every entry point applies to its fm_config (api.cu)
int check_config(const fm_config &c);

// Raise a kernel's dynamic shared-memory limit once per (device, kernel,
// size); later calls with no larger size make no driver call.
cudaError_t smem_attr(const void *kernel, size_t bytes);

// ---- internal launchers (defined per .cu file) ------------------------------------
// batched: a chunk of the batched KS + starlet pipeline (the real-output
// inverse is chosen by ks_real_for(n, batched))
int launch_ks(const void *in1, const void *in2, long in_bstride, void *out1, void *out2, void *work, int n, int batch,
              int precision, bool forward, uint64_t rot_seed, int rot_r0, bool rotate, cudaStream_t s,
              bool batched = false);
// bands_only: the smooth array c_{J-1} is not written (noise realisations)
int launch_starlet(const void *kappa, void *pyr, long pyr_bstride, int n, int J, int batch, const fm_config &cfg,
                   void *scratch, cudaStream_t s, bool bands_only = false);
// tw2: the twiddle table of n/2 (the real-output inverse), or null for the
// complex inverse
int launch_ks32(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int n,
                int batch, bool forward, uint64_t seed, int r0, bool rotate, const float2 *tw, const float2 *tw2,
                cudaStream_t s);
// Spectral operation of the column pass of the 2-D FFT pipeline
// rows FFT -> columns FFT -> op -> columns IFFT -> rows IFFT (Re, Im):
//   FFT_OP_KS_INV   multiply by conj(D)  (KS inversion, Sec. 4.5)
//   FFT_OP_KS_FWD   multiply by D        (shear of a convergence map)
//   FFT_OP_FILTER   multiply by the spectrum filt[b][ky][kx] (a periodic
//                   convolution; outputs times out_scale)
//   FFT_OP_SPECTRUM stop after the columns FFT: `work` holds the spectrum
enum { FFT_OP_KS_INV = 0, FFT_OP_KS_FWD = 1, FFT_OP_FILTER = 2, FFT_OP_SPECTRUM = 3 };
int launch_fft_op(const void *in1, const void *in2, long in_bstride, void *out1, void *out2, void *work, int n,
                  int batch, int precision, int op, const void *filt, double out_scale, uint64_t rot_seed, int rot_r0,
                  bool rotate, cudaStream_t s, bool real_ok = false);
int launch_fft32(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int n,
                 int batch, int op, const float2 *filt, float out_scale, uint64_t seed, int r0, bool rotate,
                 const float2 *tw, const float2 *tw2, cudaStream_t s);
// inverse KS with a real output (kappa_E only) through the half spectrum
// (FM_TUNE_KS_REAL): -1 = by size (default), 0 = never, 1 = whenever
// possible (fp32, n >= 64)
extern std::atomic<int> g_ks_real;
bool ks_real_for(int n, bool batched);
size_t starlet_scratch_elems(int n, int J, int batch, const fm_config &cfg);
// ---- autotuned plans (tune.cu) ----------------------------------------------------
// A plan for maps of n^2, J scales, one precision: fused depth, large-scale
// path (1 or 3), fp32 tile kernel form (1 = register window, 0 = shared
// buffer), chunk budget in MiB of batched calls (0 = the default).
struct TunedPlan {
    int fuse = 0, large_path = 0, tile = 1, chunk_mb = 0;
    double ms = 0, default_ms = 0;
};
bool tune_lookup(int n, int J, int precision, TunedPlan *out);  // false if no entry
int starlet_builtin_fuse(int n, int J, const fm_config &cfg);  // automatic depth without a table entry
int starlet_builtin_large_path(int n, int J, int fuse);
int64_t chunk_budget_default();
int starlet_fuse_depth(int n, int J, const fm_config &cfg);  // scales of the fused tile kernel
int launch_map_direct(const void *g1, const void *g2, const void *weight, long w_bs, void *map, void *coverage, int n,
                      int batch, int filter, double theta, int ell, double cut, int precision, cudaStream_t s);
// batched pipeline (pipeline.cu)
// allow_graph: batches of several chunks are recorded into a CUDA graph kept
// per (pointers, sizes, config) and replayed; false launches them eagerly
// (callers whose buffers change from call to call)
int map_starlet_run(const void *g1, const void *g2, void *pyramid, int n, int J, int batch, const fm_config &cfg,
                    cudaStream_t s, bool allow_graph = true);
// serving (serve.cu): most maps one merged run of queued pyramid-only requests
// of one shape holds (FM_TUNE_SERVE_MERGE; 1 = no merging)
extern std::atomic<int> g_serve_merge;
// serving: heavy requests running at once (FM_TUNE_SERVE_HEAVY; 0 = no limit)
extern std::atomic<int> g_serve_heavy;
int map_starlet_host_run(const char *g1h, const char *g2h, char *pyrh, int n, int J, int batch, const fm_config &cfg,
                         cudaStream_t origin);
// multi_stream: the layout of map_noise_run's internal-stream forms
size_t noise_scratch_bytes(int n, int J, int R, const fm_config &cfg, bool with_snr, bool multi_stream = false);
size_t map_starlet_scratch_bytes(int n, int J, int batch, const fm_config &cfg);
// allow_graph: record the call into a cached CUDA graph and replay it;
// otherwise launch now, on `s` alone or, with multi_eager, with the chunks
// over the internal streams (the serving path's heavy requests)
int map_noise_run(const void *g1, const void *g2, double *var_out, void *snr_out, int n, int J, int R, uint64_t seed,
                  const fm_config &cfg, cudaStream_t s, bool allow_graph, bool multi_eager = false);
int map_noise_accumulate_run(const void *g1, const void *g2, double *sums, int n, int J, int r0, int R, uint64_t seed,
                             const fm_config &cfg, cudaStream_t s);
int launch_modulus2(const void *a, long a_bs, const void *b, long b_bs, void *out, long nn, int count, int precision,
                    cudaStream_t s);
int launch_unit_shears(void *g1d, void *g2d, long nn, int precision, cudaStream_t s);
int launch_band_moments(const void *pyr, double *moments, int n, int J, int batch, int precision, void *scratch,
                        cudaStream_t s);
// acc: FP64 S1, S2 (accum 0) or fp32 Kahan pairs s1, c1, s2, c2 (accum 1), bands * nn elements each
int launch_noise_accum(const void *pyr, int nb, long pyr_bs, long nn, int bands, void *acc, int precision, int accum,
                       cudaStream_t s);
int launch_noise_finalize(const void *acc, const void *wdata, double *var, void *snr, long nelem, int R,
                          int precision, int accum, cudaStream_t s);

}  // namespace fm
