// api.cu -- the C ABI of libfastmap (declared in include/fastmap.h): argument
// validation, per-device tables, stream-ordered scratch, dispatch to the
// kernels, the noise-map driver, diagnostics and profiling hooks.
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

static int einval(const std::string &msg)
{
    set_error(msg);
    return FM_EINVAL;
}

// ---- launch accounting and profiling ------------------------------------------
std::atomic<int64_t> g_launches{0};
std::atomic<int> g_pdl{1};
std::atomic<int> g_tile_variant{1};
// bulk tensor copies: 1 = starlet tile halo, 2 = row FFT input rows, 4 = row
// IFFT input rows, 8 = large-scale column window rows, 16 = its c_{j-1} rows
// (the last two on maps of 4096^2 and up)
constexpr int kDefaultTma = 31;
std::atomic<int> g_use_tma{kDefaultTma};

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
std::atomic<int> g_prof_kid{0};
}  // namespace

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

const void *twiddles(int n, int precision, cudaStream_t s, int *status)
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
    e = cudaMalloc(&d, host.size());
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

// ---- scratch -------------------------------------------------------------------
int scratch_alloc(Scratch &sc, size_t bytes, cudaStream_t s)
{
    sc.s = s;
    if (bytes == 0) return FM_OK;
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

static fm_config cfg_or_default(const fm_config *c)
{
    fm_config d;
    memset(&d, 0, sizeof(d));
    if (c) d = *c;
    return d;
}

static int check_cfg(const fm_config &c)
{
    if (c.precision != FM_F32 && c.precision != FM_F64) return einval("precision must be FM_F32 or FM_F64");
    if (c.boundary != FM_MIRROR && c.boundary != FM_PERIODIC) return einval("boundary must be FM_MIRROR or FM_PERIODIC");
    if (c.accum != 0) return einval("accum must be 0 (FP64 accumulation)");
    if (c.fuse_depth < -1 || c.fuse_depth > 8) return einval("fuse_depth out of range [-1, 8]");
    if (c.large_path < 0 || c.large_path > 2) return einval("large_path must be 0, 1 or 2");
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

// realisations per noise chunk: keep a chunk's working set (~20 B/px each
// in fp32) near 64 MB so it stays in L2
// realisations per batched pass: enough maps per launch to fill the GPU
// (~256 MB of per-realisation working set), at most 32
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

size_t map_starlet_scratch_bytes(int n, int J, int batch, const fm_config &cfg)
{
    const size_t es = esize(cfg), nn = (size_t)n * n;
    return (size_t)batch * nn * 3 * es + starlet_scratch_elems(n, J, batch, cfg) * es + 3 * 256;
}

}  // namespace fm

using namespace fm;

// ---- entry points ----------------------------------------------------------------
extern "C" {

int fm_ks_invert(const void *g1, const void *g2, void *kappa_E, void *kappa_B, int n, int batch, const fm_config *cfgp,
                 void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_cfg(cfg);
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
    int st = check_cfg(cfg);
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
    int st = check_cfg(cfg);
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

}  // extern "C"

namespace fm {

// ---- KS + starlet over a batch, in L2-sized chunks ---------------------------------
// A chunk of C maps runs KS then the starlet before the next chunk starts, so
// its intermediates (FFT work buffer, kappa, starlet scratch: ~20 B/px fp32)
// stay in L2 and only the shear and the pyramid cross HBM.  Chunks alternate
// between two internal streams (one scratch slot each) so one chunk's
// kernels overlap the next one's.  Batches of more than one chunk are
// recorded once into a CUDA graph per (pointers, sizes, config) and replayed.
namespace {

constexpr int kMaxChunkStreams = 4;
struct DevStreams {
    cudaStream_t cap = nullptr;  // origin stream for graph capture
    cudaStream_t s[kMaxChunkStreams] = {};
    cudaEvent_t fork = nullptr, join[kMaxChunkStreams] = {};
};
std::mutex g_ds_mu;  // guards g_ds and serialises multi-stream submission
std::unordered_map<int, DevStreams> g_ds;

int dev_streams(DevStreams **out)
{
    int dev = 0;
    FM_CUDA_TRY(cudaGetDevice(&dev));
    DevStreams &d = g_ds[dev];
    if (!d.cap) {
        FM_CUDA_TRY(cudaStreamCreateWithFlags(&d.cap, cudaStreamNonBlocking));
        for (int k = 0; k < kMaxChunkStreams; ++k) {
            FM_CUDA_TRY(cudaStreamCreateWithFlags(&d.s[k], cudaStreamNonBlocking));
            FM_CUDA_TRY(cudaEventCreateWithFlags(&d.join[k], cudaEventDisableTiming));
        }
        FM_CUDA_TRY(cudaEventCreateWithFlags(&d.fork, cudaEventDisableTiming));
    }
    *out = &d;
    return FM_OK;
}

struct ChunkPlan {
    int C = 1, slots = 1;
    size_t work_b = 0, kap_b = 0, st_b = 0, slot_b = 0;
};

// measured on GB300 (32 x 1024^2, J = 7): 2 streams x 80 MB chunks with graph
// replay 0.89 ms per batch, unchunked 1.05 ms, 40 MB 1.06 ms, 100 MB 0.97 ms
constexpr int64_t kDefaultChunkBytes = 80ll << 20;
std::atomic<int64_t> g_chunk_bytes{kDefaultChunkBytes};
std::atomic<int> g_chunk_streams{2};
std::atomic<int> g_use_graphs{1};

// intermediates of one slot kept near the chunk budget (two slots in flight)
ChunkPlan plan_chunks(int n, int J, int batch, const fm_config &cfg)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const size_t nn = (size_t)n * n;
    const size_t per_map = nn * 3 * es + starlet_scratch_elems(n, J, 1, cfg) * es;
    ChunkPlan p;
    const int64_t budget = g_chunk_bytes.load();
    p.C = budget <= 0 ? batch : (int)(budget / (int64_t)per_map);
    if (p.C < 1) p.C = 1;
    if (p.C > batch) p.C = batch;
    p.slots = batch > p.C ? g_chunk_streams.load() : 1;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    p.work_b = up((size_t)p.C * nn * 2 * es);
    p.kap_b = up((size_t)p.C * nn * es);
    p.st_b = up(starlet_scratch_elems(n, J, p.C, cfg) * es);
    p.slot_b = p.work_b + p.kap_b + p.st_b;
    return p;
}

// KS + starlet of maps b0 .. b0 + bc - 1 into their pyramids.  With `rotate`
// every map of the chunk is the one input map rotated as realisation
// r0 + (index in the chunk) of the noise generator (seed).
int run_chunk(const char *g1, const char *g2, char *pyr, int n, int J, int b0, int bc, const fm_config &cfg,
              const ChunkPlan &p, char *slot, cudaStream_t s, bool rotate = false, uint64_t seed = 0, int r0 = 0)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const size_t nn = (size_t)n * n;
    char *work = slot, *kap = slot + p.work_b, *st = kap + p.kap_b;
    const size_t in_off = rotate ? 0 : b0 * nn * es;
    int r = launch_ks(g1 + in_off, g2 + in_off, rotate ? 0 : (long)nn, kap, nullptr, work, n, bc, cfg.precision, false,
                      seed, r0, rotate, s);
    if (r != FM_OK) return r;
    return launch_starlet(kap, pyr + (size_t)b0 * J * nn * es, (long)J * nn, n, J, bc, cfg, st, s);
}

// All chunks, forked from `origin` onto the internal streams (round robin
// over p.slots of them) and joined back.  Caller holds g_ds_mu.
int run_chunks(const void *g1, const void *g2, void *pyr, int n, int J, int batch, const fm_config &cfg,
               const ChunkPlan &p, char *scratch, cudaStream_t origin, DevStreams &ds)
{
    FM_CUDA_TRY(cudaEventRecord(ds.fork, origin));
    for (int k = 0; k < p.slots; ++k) FM_CUDA_TRY(cudaStreamWaitEvent(ds.s[k], ds.fork, 0));
    int i = 0;
    for (int b0 = 0; b0 < batch; b0 += p.C, ++i) {
        const int k = i % p.slots;
        const int bc = batch - b0 < p.C ? batch - b0 : p.C;
        int r = run_chunk((const char *)g1, (const char *)g2, (char *)pyr, n, J, b0, bc, cfg, p,
                          scratch + (size_t)k * p.slot_b, ds.s[k]);
        if (r != FM_OK) return r;
    }
    for (int k = 0; k < p.slots; ++k) {
        FM_CUDA_TRY(cudaEventRecord(ds.join[k], ds.s[k]));
        FM_CUDA_TRY(cudaStreamWaitEvent(origin, ds.join[k], 0));
    }
    return FM_OK;
}

struct GraphKey {
    const void *g1, *g2, *pyr;
    int n, J, batch, dev;
    fm_config cfg;
    int chunk, slots, pdl;  // the plan and launch mode (PDL bit, tile variant) the graph was recorded with
    bool operator==(const GraphKey &o) const
    {
        return g1 == o.g1 && g2 == o.g2 && pyr == o.pyr && n == o.n && J == o.J && batch == o.batch &&
               dev == o.dev && memcmp(&cfg, &o.cfg, sizeof(cfg)) == 0 && chunk == o.chunk && slots == o.slots &&
               pdl == o.pdl;
    }
};
struct GraphEntry {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    void *scratch = nullptr;
    uint64_t used = 0;
    int64_t kernels = 0;  // kernel nodes per replay (counted into g_launches)
};
std::vector<GraphEntry> g_graphs;  // guarded by g_ds_mu
uint64_t g_graph_clock = 0;
constexpr size_t kMaxGraphs = 4;

void drop_graph(GraphEntry &e)
{
    cudaDeviceSynchronize();  // an evicted graph may still be running
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.scratch) cudaFree(e.scratch);
    e.exec = nullptr;
    e.scratch = nullptr;
}

}  // namespace

static int map_starlet_dev(const void *g1, const void *g2, void *pyramid, int n, int J, int batch,
                           const fm_config &cfg, cudaStream_t s, bool allow_graph = true)
{
    const ChunkPlan p = plan_chunks(n, J, batch, cfg);
    if (p.C >= batch) {  // one chunk: straight onto the caller's stream
        Scratch sc;
        int st = scratch_alloc(sc, p.slot_b, s);
        if (st) return st;
        return run_chunk((const char *)g1, (const char *)g2, (char *)pyramid, n, J, 0, batch, cfg, p, (char *)sc.p, s);
    }
    int st = FM_OK;
    if (!twiddles(n, cfg.precision, s, &st)) return st;  // build tables outside any capture
    std::lock_guard<std::mutex> lk(g_ds_mu);
    DevStreams *ds = nullptr;
    if ((st = dev_streams(&ds))) return st;
    const bool profiling = g_prof_kid.load() != 0;
    if (!allow_graph || profiling || !g_use_graphs.load()) {
        Scratch sc;
        if ((st = scratch_alloc(sc, p.slot_b * p.slots, s))) return st;
        return run_chunks(g1, g2, pyramid, n, J, batch, cfg, p, (char *)sc.p, s, *ds);
    }
    GraphKey key{g1, g2, pyramid, n, J, batch, 0, cfg, p.C, p.slots,
                 g_pdl.load() | (g_tile_variant.load() << 1) | (g_use_tma.load() << 3)};
    FM_CUDA_TRY(cudaGetDevice(&key.dev));
    GraphEntry *hit = nullptr;
    for (auto &e : g_graphs)
        if (e.key == key) hit = &e;
    if (!hit) {
        if (g_graphs.size() >= kMaxGraphs) {
            auto lru = std::min_element(g_graphs.begin(), g_graphs.end(),
                                        [](const GraphEntry &a, const GraphEntry &b) { return a.used < b.used; });
            drop_graph(*lru);
            g_graphs.erase(lru);
        }
        GraphEntry e;
        e.key = key;
        cudaError_t ce = cudaMalloc(&e.scratch, p.slot_b * p.slots);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMalloc (graph scratch)");
        cudaGraph_t graph = nullptr;
        ce = cudaStreamBeginCapture(ds->cap, cudaStreamCaptureModeRelaxed);
        if (ce != cudaSuccess) {
            cudaFree(e.scratch);
            return cuda_fail(ce, "cudaStreamBeginCapture");
        }
        const int64_t before = g_launches.load();
        st = run_chunks(g1, g2, pyramid, n, J, batch, cfg, p, (char *)e.scratch, ds->cap, *ds);
        e.kernels = g_launches.load() - before;
        g_launches.fetch_sub(e.kernels);  // recorded, not launched
        ce = cudaStreamEndCapture(ds->cap, &graph);
        if (st == FM_OK && ce != cudaSuccess) st = cuda_fail(ce, "cudaStreamEndCapture");
        if (st == FM_OK) {
            ce = cudaGraphInstantiate(&e.exec, graph, 0);
            if (ce != cudaSuccess) st = cuda_fail(ce, "cudaGraphInstantiate");
        }
        if (graph) cudaGraphDestroy(graph);
        if (st != FM_OK) {
            if (e.exec) cudaGraphExecDestroy(e.exec);
            cudaFree(e.scratch);
            return st;
        }
        g_graphs.push_back(e);
        hit = &g_graphs.back();
    }
    hit->used = ++g_graph_clock;
    FM_CUDA_TRY(cudaGraphLaunch(hit->exec, s));
    g_launches.fetch_add(hit->kernels);
    return FM_OK;
}

// ---- noise maps: R rotated realisations, batched, in one graph launch ------------
namespace {

struct NoiseLayout {
    int batch = 1;  // realisations per accumulation pass
    ChunkPlan p;    // KS + starlet of a batch, chunk by chunk
    int slots = 1;  // chunk slots in use: internal streams, or 1 on the caller's stream
    size_t acc_b = 0, pyr_b = 0, total = 0;
};

// A batch's pyramids stay within ~1 GiB (at most 32 realisations: the
// accumulation's partial sums are fp32 over at most 32 terms).
NoiseLayout noise_layout(int n, int J, int R, const fm_config &cfg, bool multi_stream)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const size_t nn = (size_t)n * n;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    NoiseLayout L;
    long batch = (1L << 30) / (long)((size_t)J * nn * es);
    batch = batch < 1 ? 1 : (batch > 32 ? 32 : batch);
    L.batch = (int)(batch > R ? R : batch);
    L.p = plan_chunks(n, J, L.batch, cfg);
    L.slots = multi_stream ? L.p.slots : 1;
    L.acc_b = up(2 * (size_t)(J - 1) * nn * sizeof(double));
    L.pyr_b = up((size_t)L.batch * J * nn * es);
    L.total = L.acc_b + L.pyr_b + (size_t)L.slots * L.p.slot_b;
    return L;
}

// Everything of one fm_map_noise call: zero the FP64 sums; every batch of
// rotated realisations through KS + starlet, chunk by chunk (over the
// internal streams when `ds` is given, else on `s`), then S1 += w, S2 += w^2
// over the batch's pyramids on `s`; the unrotated pass for S/N; the finalize
// kernel.  (A second pyramid buffer, letting the chunk streams run on into the
// next batch during an accumulation, measured no faster: 36.5 vs 35.6 ms for
// R = 1000 at 1024^2.)
int noise_submit(const void *g1, const void *g2, double *var_out, void *snr_out, int n, int J, int R, uint64_t seed,
                 const fm_config &cfg, const NoiseLayout &L, char *scr, cudaStream_t s, DevStreams *ds)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const long nn = (long)n * n;
    const long nb = (long)(J - 1) * nn;
    double *s1 = reinterpret_cast<double *>(scr);
    double *s2 = s1 + nb;
    char *pyr = scr + L.acc_b, *slots = pyr + L.pyr_b;
    const ChunkPlan &p = L.p;
    const bool multi = ds && L.slots > 1;
    const char *c1 = static_cast<const char *>(g1), *c2 = static_cast<const char *>(g2);
    int r;
    FM_CUDA_TRY(cudaMemsetAsync(s1, 0, (size_t)2 * nb * sizeof(double), s));
    for (int r0 = 0; r0 < R; r0 += L.batch) {
        const int b = R - r0 < L.batch ? R - r0 : L.batch;
        if (multi) {  // the batch's pyramid buffer is free once `s` has accumulated the last batch
            FM_CUDA_TRY(cudaEventRecord(ds->fork, s));
            for (int k = 0; k < L.slots; ++k) FM_CUDA_TRY(cudaStreamWaitEvent(ds->s[k], ds->fork, 0));
        }
        int i = 0;
        for (int c0 = 0; c0 < b; c0 += p.C, ++i) {
            const int k = multi ? i % L.slots : 0;
            const int bc = b - c0 < p.C ? b - c0 : p.C;
            if ((r = run_chunk(c1, c2, pyr + (size_t)c0 * J * nn * es, n, J, 0, bc, cfg, p, slots + k * p.slot_b,
                               multi ? ds->s[k] : s, true, seed, r0 + c0)))
                return r;
        }
        if (multi)
            for (int k = 0; k < L.slots; ++k) {
                FM_CUDA_TRY(cudaEventRecord(ds->join[k], ds->s[k]));
                FM_CUDA_TRY(cudaStreamWaitEvent(s, ds->join[k], 0));
            }
        if ((r = launch_noise_accum(pyr, b, (long)J * nn, nn, J - 1, s1, s2, cfg.precision, s))) return r;
    }
    // S/N needs the unrotated bands; finalize reads them from the first pyramid
    // (every chunk stream has joined `s` after the last batch)
    if (snr_out && (r = run_chunk(c1, c2, pyr, n, J, 0, 1, cfg, p, slots, s))) return r;
    return launch_noise_finalize(s1, s2, snr_out ? pyr : nullptr, var_out, snr_out, nb, R, cfg.precision, s);
}

struct NoiseKey {
    const void *g1, *g2, *var, *snr;
    int n, J, R, dev;
    uint64_t seed;
    fm_config cfg;
    int chunk, slots, pdl;  // the plan and launch mode the graph was recorded with
    bool operator==(const NoiseKey &o) const
    {
        return g1 == o.g1 && g2 == o.g2 && var == o.var && snr == o.snr && n == o.n && J == o.J && R == o.R &&
               dev == o.dev && seed == o.seed && memcmp(&cfg, &o.cfg, sizeof(cfg)) == 0 && chunk == o.chunk &&
               slots == o.slots && pdl == o.pdl;
    }
};
struct NoiseGraph {
    NoiseKey key;
    cudaGraphExec_t exec = nullptr;
    void *scratch = nullptr;
    uint64_t used = 0;
    int64_t kernels = 0;
};
std::vector<NoiseGraph> g_noise_graphs;  // guarded by g_ds_mu
constexpr size_t kMaxNoiseGraphs = 2;

void drop_noise_graph(NoiseGraph &e)
{
    cudaDeviceSynchronize();
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.scratch) cudaFree(e.scratch);
    e.exec = nullptr;
    e.scratch = nullptr;
}

}  // namespace

// allow_graph: record the whole call once into a CUDA graph (kept with its
// scratch, LRU of two) and replay it; otherwise launch eagerly with
// stream-ordered scratch (the serving path, whose buffers change per call).
int map_noise_run(const void *g1, const void *g2, double *var_out, void *snr_out, int n, int J, int R, uint64_t seed,
                  const fm_config &cfg, cudaStream_t s, bool allow_graph)
{
    int st = FM_OK;
    if (!twiddles(n, cfg.precision, s, &st)) return st;  // tables before any capture
    if (!allow_graph || g_prof_kid.load() != 0 || !g_use_graphs.load()) {
        const NoiseLayout L = noise_layout(n, J, R, cfg, false);
        Scratch sc;
        if ((st = scratch_alloc(sc, L.total, s))) return st;
        return noise_submit(g1, g2, var_out, snr_out, n, J, R, seed, cfg, L, (char *)sc.p, s, nullptr);
    }
    const NoiseLayout L = noise_layout(n, J, R, cfg, true);
    std::lock_guard<std::mutex> lk(g_ds_mu);
    DevStreams *ds = nullptr;
    if ((st = dev_streams(&ds))) return st;
    NoiseKey key{g1, g2, var_out, snr_out, n, J, R, 0, seed, cfg, L.p.C, L.slots,
                 g_pdl.load() | (g_tile_variant.load() << 1) | (g_use_tma.load() << 3)};
    FM_CUDA_TRY(cudaGetDevice(&key.dev));
    NoiseGraph *hit = nullptr;
    for (auto &e : g_noise_graphs)
        if (e.key == key) hit = &e;
    if (!hit) {
        if (g_noise_graphs.size() >= kMaxNoiseGraphs) {
            auto lru = std::min_element(g_noise_graphs.begin(), g_noise_graphs.end(),
                                        [](const NoiseGraph &a, const NoiseGraph &b) { return a.used < b.used; });
            drop_noise_graph(*lru);
            g_noise_graphs.erase(lru);
        }
        NoiseGraph e;
        e.key = key;
        cudaError_t ce = cudaMalloc(&e.scratch, L.total);
        if (ce != cudaSuccess) return cuda_fail(ce, "cudaMalloc (noise graph scratch)");
        cudaGraph_t graph = nullptr;
        ce = cudaStreamBeginCapture(ds->cap, cudaStreamCaptureModeRelaxed);
        if (ce != cudaSuccess) {
            cudaFree(e.scratch);
            return cuda_fail(ce, "cudaStreamBeginCapture");
        }
        const int64_t before = g_launches.load();
        st = noise_submit(g1, g2, var_out, snr_out, n, J, R, seed, cfg, L, (char *)e.scratch, ds->cap, ds);
        e.kernels = g_launches.load() - before;
        g_launches.fetch_sub(e.kernels);
        ce = cudaStreamEndCapture(ds->cap, &graph);
        if (st == FM_OK && ce != cudaSuccess) st = cuda_fail(ce, "cudaStreamEndCapture");
        if (st == FM_OK) {
            ce = cudaGraphInstantiate(&e.exec, graph, 0);
            if (ce != cudaSuccess) st = cuda_fail(ce, "cudaGraphInstantiate");
        }
        if (graph) cudaGraphDestroy(graph);
        if (st != FM_OK) {
            if (e.exec) cudaGraphExecDestroy(e.exec);
            cudaFree(e.scratch);
            return st;
        }
        g_noise_graphs.push_back(e);
        hit = &g_noise_graphs.back();
    }
    hit->used = ++g_graph_clock;
    FM_CUDA_TRY(cudaGraphLaunch(hit->exec, s));
    g_launches.fetch_add(hit->kernels);
    return FM_OK;
}

// scratch of a noise call on the caller's stream (the serving path)
size_t noise_scratch_bytes(int n, int J, int R, const fm_config &cfg, bool with_snr)
{
    (void)with_snr;
    return noise_layout(n, J, R, cfg, false).total + 256;
}

int map_starlet_run(const void *g1, const void *g2, void *pyramid, int n, int J, int batch, const fm_config &cfg,
                    cudaStream_t s)
{
    return map_starlet_dev(g1, g2, pyramid, n, J, batch, cfg, s);
}

// Host buffers: the chunks of the batch stream through the slots of the
// internal streams; each copies its shear in, runs KS + starlet and copies its
// pyramid out.  A slot's next chunk follows its previous copy out on the same
// stream, so with two or more slots the copies of one chunk overlap the
// compute of another and the two copy directions overlap each other.
static int map_starlet_host_run(const char *g1h, const char *g2h, char *pyrh, int n, int J, int batch,
                                const fm_config &cfg, cudaStream_t origin)
{
    ChunkPlan p = plan_chunks(n, J, batch, cfg);
    const size_t es = esize(cfg), nn = (size_t)n * n;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t in_b = up((size_t)p.C * nn * es), pyr_b = up((size_t)p.C * J * nn * es);
    const size_t slot_b = p.slot_b + 2 * in_b + pyr_b;
    int st = FM_OK;
    if (!twiddles(n, cfg.precision, origin, &st)) return st;
    Scratch sc;  // freed on `origin` after the join below
    if ((st = scratch_alloc(sc, slot_b * p.slots, origin))) return st;
    std::lock_guard<std::mutex> lk(g_ds_mu);
    DevStreams *ds = nullptr;
    if ((st = dev_streams(&ds))) return st;
    FM_CUDA_TRY(cudaEventRecord(ds->fork, origin));
    for (int k = 0; k < p.slots; ++k) FM_CUDA_TRY(cudaStreamWaitEvent(ds->s[k], ds->fork, 0));
    int i = 0;
    for (int b0 = 0; b0 < batch; b0 += p.C, ++i) {
        const int k = i % p.slots;
        const int bc = batch - b0 < p.C ? batch - b0 : p.C;
        cudaStream_t sk = ds->s[k];
        char *slot = static_cast<char *>(sc.p) + (size_t)k * slot_b;
        char *d1 = slot + p.slot_b, *d2 = d1 + in_b, *dp = d2 + in_b;
        const size_t map_b = (size_t)bc * nn * es;
        FM_CUDA_TRY(cudaMemcpyAsync(d1, g1h + (size_t)b0 * nn * es, map_b, cudaMemcpyHostToDevice, sk));
        FM_CUDA_TRY(cudaMemcpyAsync(d2, g2h + (size_t)b0 * nn * es, map_b, cudaMemcpyHostToDevice, sk));
        if ((st = run_chunk(d1, d2, dp, n, J, 0, bc, cfg, p, slot, sk))) return st;
        FM_CUDA_TRY(cudaMemcpyAsync(pyrh + (size_t)b0 * J * nn * es, dp, (size_t)J * map_b, cudaMemcpyDeviceToHost,
                                    sk));
    }
    for (int k = 0; k < p.slots; ++k) {
        FM_CUDA_TRY(cudaEventRecord(ds->join[k], ds->s[k]));
        FM_CUDA_TRY(cudaStreamWaitEvent(origin, ds->join[k], 0));
    }
    return FM_OK;
}

}  // namespace fm

extern "C" {

int fm_map_starlet(const void *g1, const void *g2, void *pyramid, int n, int J, int batch, const fm_config *cfgp,
                   void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_cfg(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (batch < 1) return einval("batch must be >= 1");
    if (!g1 || !g2 || !pyramid) return einval("null pointer");
    return map_starlet_dev(g1, g2, pyramid, n, J, batch, cfg, (cudaStream_t)stream);
}

int fm_map_starlet_host(const void *g1_host, const void *g2_host, void *pyramid_host, int n, int J, int batch,
                        const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_cfg(cfg);
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
    int st = check_cfg(cfg);
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

int fm_map_direct_masked(const void *g1, const void *g2, const void *weight, long weight_bstride, void *map,
                         void *coverage, int n, int batch, int filter, double theta_px, int ell,
                         double cut_over_theta, const fm_config *cfgp, void *stream)
{
    fm_config cfg = cfg_or_default(cfgp);
    int st = check_cfg(cfg);
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
    int st = check_cfg(cfg);
    if (st) return st;
    if ((st = check_fft_n(n))) return st;
    if ((st = check_J(n, J))) return st;
    if (R < 2) return einval("R must be >= 2");
    if (!g1 || !g2 || !var_out) return einval("null pointer");
    return map_noise_run(g1, g2, var_out, snr_out, n, J, R, seed, cfg, (cudaStream_t)stream, true);
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
    int st = check_cfg(cfg);
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
    int st = check_cfg(cfg);
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

int fm_trim(void)
{
    std::lock_guard<std::mutex> lk(g_ds_mu);
    for (auto &e : g_graphs) drop_graph(e);
    g_graphs.clear();
    for (auto &e : g_noise_graphs) drop_noise_graph(e);
    g_noise_graphs.clear();
    return FM_OK;
}

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

int fm_tune(int knob, int64_t value)
{
    switch (knob) {
    case FM_TUNE_CHUNK_BYTES: g_chunk_bytes.store(value < 0 ? kDefaultChunkBytes : value); return FM_OK;
    case FM_TUNE_GRAPHS: g_use_graphs.store(value < 0 ? 1 : (value != 0)); return FM_OK;
    case FM_TUNE_CHUNK_STREAMS:
        g_chunk_streams.store(value < 0 ? 2 : (int)(value < 1 ? 1 : value > kMaxChunkStreams ? kMaxChunkStreams : value));
        return FM_OK;
    case FM_TUNE_PDL: g_pdl.store(value < 0 ? 1 : (value != 0)); return FM_OK;
    case FM_TUNE_TMA:
        if (value > 31) return einval("FM_TUNE_TMA is a mask of 1, 2, 4, 8 and 16");
        g_use_tma.store(value < 0 ? kDefaultTma : (int)value);
        return FM_OK;
    case FM_TUNE_TILE:
        if (value > 1) return einval("FM_TUNE_TILE takes 0 or 1");
        g_tile_variant.store(value < 0 ? 1 : (int)value);
        return FM_OK;
    }
    return einval("unknown tuning knob");
}

int64_t fm_launch_count(void) { return g_launches.load(); }

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
