// runtime.cu -- shared services of libfastmap: the calling thread's last
// error, launch counting and the per-kernel profiling hooks, per-device
// twiddle tables, stream-ordered scratch, dynamic shared-memory attributes,
// the driver's tensor-map encoder (TMA), and the diagnostic C entry points.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "tma.cuh"

namespace fm {

// ---- errors -----------------------------------------------------------------
static thread_local std::string t_last_error;

void set_error(const std::string &msg) { t_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // allocation failures are not sticky; clear them
        return FM_ENOMEM;
    }
    return FM_ECUDA;
}

int einval(const std::string &msg)
{
    set_error(msg);
    return FM_EINVAL;
}

// ---- launch accounting and profiling ------------------------------------------
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_pdl{1};
std::atomic<int> g_tile_variant{-1};
std::atomic<int> g_use_tma{kDefaultTma};
std::atomic<int> g_wait_test{0};

namespace {
struct Prof {
    std::mutex mu;
    int kid = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pairs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t pending = nullptr;
    cudaEvent_t get()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};
Prof g_prof;
}  // namespace
std::atomic<int> g_prof_kid{0};

void prof_before(int kid, cudaStream_t s)
{
    if (kid == 0 || g_prof_kid.load(std::memory_order_relaxed) != kid) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.pending = g_prof.get();
    cudaEventRecord(g_prof.pending, s);
}

void prof_after(int kid, cudaStream_t s)
{
    if (kid == 0 || g_prof_kid.load(std::memory_order_relaxed) != kid) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    if (!g_prof.pending) return;
    cudaEvent_t e = g_prof.get();
    cudaEventRecord(e, s);
    g_prof.pairs.emplace_back(g_prof.pending, e);
    g_prof.pending = nullptr;
}

// ---- twiddle tables ------------------------------------------------------------
namespace {
std::mutex g_tw_mu;
std::unordered_map<uint64_t, void *> g_tw;  // key: device, precision, n
}  // namespace

static const void *twiddles_one(int n, int precision, cudaStream_t s, int *status);

// The table of n and, for fp32 n >= 64, the one of n / 2 as well, which the
// real-output inverse transform uses: both exist once this returns, so a call
// before a stream capture leaves nothing to allocate inside it.
const void *twiddles(int n, int precision, cudaStream_t s, int *status)
{
    if (precision == FM_F32 && n >= 64 && !twiddles_one(n / 2, precision, s, status)) return nullptr;
    return twiddles_one(n, precision, s, status);
}

static const void *twiddles_one(int n, int precision, cudaStream_t s, int *status)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *status = cuda_fail(e, "cudaGetDevice");
        return nullptr;
    }
    const uint64_t key = ((uint64_t)dev << 40) | ((uint64_t)precision << 32) | (uint64_t)n;
    std::lock_guard<std::mutex> lk(g_tw_mu);
    auto it = g_tw.find(key);
    if (it != g_tw.end()) return it->second;
    // exp(-2 pi i t / n) in FP64 on the host, rounded once to the element type
    const size_t esz = precision == FM_F64 ? 16 : 8;
    std::vector<unsigned char> host((size_t)n * esz);
    for (int t = 0; t < n; ++t) {
        const double ang = -2.0 * M_PI * (double)t / (double)n;
        const double c = cos(ang), sn = sin(ang);
        if (precision == FM_F64) {
            double v[2] = {c, sn};
            memcpy(&host[(size_t)t * esz], v, esz);
        } else {
            float v[2] = {(float)c, (float)sn};
            memcpy(&host[(size_t)t * esz], v, esz);
        }
    }
    void *d = nullptr;
    e = dev_malloc(&d, host.size());
    if (e == cudaSuccess) e = cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (d) cudaFree(d);
        *status = cuda_fail(e, "twiddle table");
        return nullptr;
    }
    (void)s;
    g_tw[key] = d;
    return d;
}

// ---- kernel attributes -------------------------------------------------------------
namespace {
std::mutex g_attr_mu;
std::unordered_map<uint64_t, size_t> g_attr;  // (device, kernel) -> smem bytes set
}  // namespace

cudaError_t smem_attr(const void *kernel, size_t bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t key = ((uint64_t)(uintptr_t)kernel) ^ ((uint64_t)dev << 56);
    std::lock_guard<std::mutex> lk(g_attr_mu);
    auto it = g_attr.find(key);
    if (it != g_attr.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_attr[key] = bytes;
    return e;
}

// ---- device allocations ---------------------------------------------------------
// Every device allocation the library makes (stream-ordered scratch, graph
// scratch, tables, the autotuner's buffers) is counted here: fm_alloc_stats.
std::atomic<int64_t> g_alloc_count{0}, g_alloc_max{0};

void note_alloc(size_t bytes)
{
    g_alloc_count.fetch_add(1);
    int64_t cur = g_alloc_max.load();
    while ((int64_t)bytes > cur && !g_alloc_max.compare_exchange_weak(cur, (int64_t)bytes)) {
    }
}

cudaError_t dev_malloc(void **p, size_t bytes)
{
    note_alloc(bytes);
    return cudaMalloc(p, bytes);
}

// ---- scratch -------------------------------------------------------------------
int scratch_alloc(Scratch &sc, size_t bytes, cudaStream_t s)
{
    sc.s = s;
    if (bytes == 0) return FM_OK;
    note_alloc(bytes);
    static std::once_flag pool_once;
    std::call_once(pool_once, [] {
        // keep freed stream-ordered memory in the pool instead of returning it
        // to the driver after every call (a setting of this process only)
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
    });
    cudaError_t e = cudaMallocAsync(&sc.p, bytes, s);
    if (e != cudaSuccess) {
        sc.p = nullptr;
        return cuda_fail(e, "cudaMallocAsync (scratch)");
    }
    return FM_OK;
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            fn = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    return encode;
}

static bool encode_map_f32(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                           const uint64_t *strides, const uint32_t *box)
{
    PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode || (reinterpret_cast<uintptr_t>(base) & 15)) return false;
    cuuint64_t d[5], st[4];
    cuuint32_t bx[5], estr[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        estr[i] = 1;
        if (i + 1 < rank) {
            if (strides[i] % 16) return false;
            st[i] = strides[i];
        }
    }
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (cuuint32_t)rank, const_cast<void *>(base), d, st, bx, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_map3d_f32(CUtensorMap *map, const void *base, const uint64_t dims[3], const uint64_t strides[2],
                      const uint32_t box[3])
{
    return encode_map_f32(map, base, 3, dims, strides, box);
}

bool encode_map5d_f32(CUtensorMap *map, const void *base, const uint64_t dims[5], const uint64_t strides[4],
                      const uint32_t box[5])
{
    return encode_map_f32(map, base, 5, dims, strides, box);
}

}  // namespace fm

using namespace fm;

extern "C" {

const char *fm_status_string(int status)
{
    switch (status) {
    case FM_OK: return "ok";
    case FM_PENDING: return "pending";
    case FM_EINVAL: return "invalid argument";
    case FM_ENOMEM: return "out of device memory";
    case FM_EBUDGET: return "request exceeds the memory budget";
    case FM_ETIMEOUT: return "timed out";
    case FM_ECUDA: return "CUDA error";
    case FM_ENOTFOUND: return "unknown ticket";
    case FM_EBUSY: return "queue full";
    }
    return "unknown status";
}

const char *fm_last_error(void) { return t_last_error.c_str(); }

int64_t fm_launch_count(void) { return g_launches.load(); }

int fm_ks_real_output(int n, int batched) { return ks_real_for(n, batched != 0) ? 1 : 0; }

}  // extern "C"

namespace fm {
// streaming read (sum of float4 loads that bypass L1) and copy over n4 float4,
// `reps` sweeps inside one launch: the memory-side rates a kernel of this
// library can reach for a working set of that size (L2-resident or not)
__global__ void k_bw_read(const float4 *__restrict__ a, long n4, int reps, float *sink)
{
    float acc = 0.f;
    for (int r = 0; r < reps; ++r)
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
            const float4 v = __ldcg(a + i);
            acc += v.x + v.y + v.z + v.w;
        }
    if (acc == 1.5f) sink[0] = acc;  // keeps the loads; the inputs are zeros
}
__global__ void k_bw_copy(const float4 *__restrict__ a, float4 *__restrict__ b, long n4, int reps)
{
    for (int r = 0; r < reps; ++r)
        for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x)
            __stcg(b + i, __ldcg(a + i));
}
}  // namespace fm

extern "C" {

int fm_measure_bandwidth(size_t bytes, int reps, double *read_gbs, double *copy_gbs)
{
    if (bytes < (1u << 20) || bytes > (64ull << 30) || reps < 1 || reps > 1000)
        return einval("bytes must be in [1 MiB, 64 GiB] and reps in [1, 1000]");
    const long n4 = (long)(bytes / 32);  // two buffers of bytes / 2 each
    void *a = nullptr, *b = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = FM_OK;
    float ms = 0.f;
    cudaError_t e = dev_malloc(&a, (size_t)n4 * 16);
    if (e == cudaSuccess) e = dev_malloc(&b, (size_t)n4 * 16);
    if (e == cudaSuccess) e = dev_malloc(&sink, 16);
    if (e == cudaSuccess) e = cudaMemset(a, 0, (size_t)n4 * 16);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const unsigned grid = 152 * 16;
    if (e == cudaSuccess) {
        // two buffers of bytes / 2: the read sweeps the first, the copy moves it into the second
        k_bw_read<<<grid, 256>>>((const float4 *)a, n4, 1, (float *)sink);  // warm-up
        cudaEventRecord(e0);
        k_bw_read<<<grid, 256>>>((const float4 *)a, n4, reps, (float *)sink);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && read_gbs) *read_gbs = (double)n4 * 16 * reps / (ms * 1e-3) / 1e9;
    }
    if (e == cudaSuccess) {
        k_bw_copy<<<grid, 256>>>((const float4 *)a, (float4 *)b, n4, 1);
        cudaEventRecord(e0);
        k_bw_copy<<<grid, 256>>>((const float4 *)a, (float4 *)b, n4, reps);
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && copy_gbs) *copy_gbs = (double)n4 * 32 * reps / (ms * 1e-3) / 1e9;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "fm_measure_bandwidth");
    g_launches.fetch_add(4);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (sink) cudaFree(sink);
    return st;
}

int fm_alloc_stats(int64_t *count, int64_t *max_bytes, int reset)
{
    if (count) *count = g_alloc_count.load();
    if (max_bytes) *max_bytes = g_alloc_max.load();
    if (reset) {
        g_alloc_count.store(0);
        g_alloc_max.store(0);
    }
    return FM_OK;
}

int fm_profile_select(int kid)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    for (auto &p : g_prof.pairs) {
        g_prof.pool.push_back(p.first);
        g_prof.pool.push_back(p.second);
    }
    g_prof.pairs.clear();
    g_prof.pending = nullptr;
    g_prof_kid.store(kid);
    return FM_OK;
}

int fm_device_error(void)
{
    const int a = starlet_wait_error(true), b = fft_wait_error(true);
    if (a < 0 || b < 0) return einval("fm_device_error: no device");
    return a | b;
}

int fm_profile_read(double *total_ms, int64_t *launches)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    double tot = 0;
    for (auto &p : g_prof.pairs) {
        cudaError_t e = cudaEventSynchronize(p.second);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float ms = 0;
        e = cudaEventElapsedTime(&ms, p.first, p.second);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventElapsedTime");
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (launches) *launches = (int64_t)g_prof.pairs.size();
    return FM_OK;
}

}  // extern "C"
