// pipeline.cu -- how batched calls run on the device: L2-sized chunks of the
// batch alternating over internal streams, CUDA-graph recording and replay,
// the host-buffer copy pipeline, the noise-map driver, and the tuning knobs
// and caches that shape them (fm_tune, fm_trim).
#include <string.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace fm {

// ---- KS + starlet over a batch, in L2-sized chunks ---------------------------------
// A chunk of C maps runs KS then the starlet before the next chunk starts, so
// its intermediates (FFT work buffer, kappa, starlet scratch: ~20 B/px fp32)
// stay in L2 and only the shear and the pyramid cross HBM.  Chunks alternate
// over the internal streams (two by default, one scratch slot each) so one
// chunk's kernels overlap the next one's.  Batches of more than one chunk are
// recorded once into a CUDA graph per (pointers, sizes, config) and replayed.
namespace {

constexpr int kMaxChunkStreams = 4;
struct DevStreams {
    cudaStream_t cap = nullptr;  // origin stream for graph capture
    cudaStream_t s[kMaxChunkStreams] = {};
    cudaEvent_t fork = nullptr, join[kMaxChunkStreams] = {};
    cudaEvent_t acc[2] = {};  // noise: accumulation of the batch in pyramid buffer 0 / 1 done
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
        for (auto &e : d.acc) FM_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    *out = &d;
    return FM_OK;
}

struct ChunkPlan {
    int C = 1, slots = 1;
    size_t work_b = 0, kap_b = 0, st_b = 0, slot_b = 0;
};

// A chunk's intermediates: the FFT work buffer (2 n^2 per map), kappa (n^2)
// and, where they do not fit in the work buffer (dead once kappa is formed),
// the starlet's scratch maps.  Measured on GB300 (32 x 1024^2, J = 7), with
// the scratch in its own buffer (20 MB a map): 2 streams x 80 MB chunks with
// graph replay 0.89 ms per batch, unchunked 1.05 ms, 40 MB 1.06 ms, 100 MB
// 0.97 ms; four maps a chunk stayed the best choice as the kernels changed.
// With the scratch in the work buffer (12 MB a map) four maps take 48 MB.
constexpr int64_t kDefaultChunkBytes = 48ll << 20;
std::atomic<int64_t> g_chunk_bytes{kDefaultChunkBytes};
std::atomic<int> g_chunk_bytes_set{0};  // set by fm_tune: overrides the autotuned budget
std::atomic<int> g_chunk_streams{2};
std::atomic<int> g_use_graphs{1};

}  // namespace

int64_t chunk_budget_default() { return kDefaultChunkBytes; }

namespace {

// intermediates of one slot kept near the chunk budget (two slots in flight)
ChunkPlan plan_chunks(int n, int J, int batch, const fm_config &cfg)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const size_t nn = (size_t)n * n;
    // the starlet's scratch maps go to the work buffer when they fit there
    const bool st_in_work = starlet_scratch_elems(n, J, 1, cfg) <= 2 * nn;
    const size_t per_map = nn * 3 * es + (st_in_work ? 0 : starlet_scratch_elems(n, J, 1, cfg) * es);
    ChunkPlan p;
    int64_t budget = g_chunk_bytes.load();
    TunedPlan tp;
    if (!g_chunk_bytes_set.load() && tune_lookup(n, J, cfg.precision, &tp) && tp.chunk_mb > 0)
        budget = (int64_t)tp.chunk_mb << 20;
    p.C = budget <= 0 ? batch : (int)(budget / (int64_t)per_map);
    if (p.C < 1) p.C = 1;
    if (p.C > batch) p.C = batch;
    p.slots = batch > p.C ? g_chunk_streams.load() : 1;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    p.work_b = up((size_t)p.C * nn * 2 * es);
    p.kap_b = up((size_t)p.C * nn * es);
    p.st_b = st_in_work ? 0 : up(starlet_scratch_elems(n, J, p.C, cfg) * es);
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
    // the starlet's scratch: its own buffer, or the work buffer, which the
    // starlet kernels (later on the same stream) find dead
    char *work = slot, *kap = slot + p.work_b, *st = p.st_b ? kap + p.kap_b : work;
    const size_t in_off = rotate ? 0 : b0 * nn * es;
    int r = launch_ks(g1 + in_off, g2 + in_off, rotate ? 0 : (long)nn, kap, nullptr, work, n, bc, cfg.precision, false,
                      seed, r0, rotate, s, true);
    if (r != FM_OK) return r;
    // a noise realisation needs its bands only (the smooth array is not accumulated)
    return launch_starlet(kap, pyr + (size_t)b0 * J * nn * es, (long)J * nn, n, J, bc, cfg, st, s, rotate);
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
                 g_pdl.load() | ((g_tile_variant.load() + 1) << 1) | (g_use_tma.load() << 3) | (g_wait_test.load() << 10) | ((g_ks_real.load() + 1) << 11)};
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
        cudaError_t ce = dev_malloc(&e.scratch, p.slot_b * p.slots);
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
    int pyr_bufs = 1;  // batch pyramid buffers: 2 lets the chunk streams run on during an accumulation
    size_t acc_b = 0, pyr_b = 0, total = 0;
};
constexpr int kNoisePyrBufs = 2;
constexpr long kNoisePyrBatchBytes = 8L << 30;  // pyramids of one accumulation batch

// A batch's pyramids stay within 8 GiB (at most 32 realisations: the
// accumulation's partial sums are fp32 over at most 32 terms).  Each batch
// re-reads and re-writes the FP64 sums (32 bytes per band pixel), so large
// maps need several realisations per batch: with 1 GiB a 4096^2 J = 10 map
// had one, and R = 100 took 273 ms; with 4 GiB (six) 116 ms, with 8 GiB
// (twelve) 102 ms; the serving trace went 3.9 -> 8.0 -> 9.0 requests/s.
// ext_sums: the running sums are the caller's (partial accumulation), so the
// layout holds no space for them.
NoiseLayout noise_layout(int n, int J, int R, const fm_config &cfg, bool multi_stream, bool ext_sums = false)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const size_t nn = (size_t)n * n;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    NoiseLayout L;
    long batch = kNoisePyrBatchBytes / (long)((size_t)J * nn * es);
    batch = batch < 1 ? 1 : (batch > 32 ? 32 : batch);
    L.batch = (int)(batch > R ? R : batch);
    L.p = plan_chunks(n, J, L.batch, cfg);
    L.slots = multi_stream ? L.p.slots : 1;
    L.pyr_bufs = L.slots > 1 && R > L.batch ? kNoisePyrBufs : 1;
    L.acc_b = ext_sums ? 0 : up(2 * (size_t)(J - 1) * nn * sizeof(double));
    L.pyr_b = up((size_t)L.batch * J * nn * es);
    L.total = L.acc_b + (size_t)L.pyr_bufs * L.pyr_b + (size_t)L.slots * L.p.slot_b;
    return L;
}

// Everything of one fm_map_noise call: zero the FP64 sums; every batch of
// rotated realisations through KS + starlet, chunk by chunk (over the
// internal streams when `ds` is given, else on `s`), then S1 += w, S2 += w^2
// over the batch's pyramids on `s`; the unrotated pass for S/N; the finalize
// kernel.  With internal streams and more than one batch, two pyramid
// buffers alternate so that the chunk streams run on into the next batch
// while `s` accumulates (R = 1000 at 1024^2: 32.2 -> 31.6 ms; the
// accumulation's pyramid loads are streaming, evict-first: 31.5 ms).
// ext_sums (partial accumulation): the caller's FP64 sums, added to without
// zeroing and without the S/N pass and finalize; realisations rbase ..
// rbase + R - 1.
int noise_submit(const void *g1, const void *g2, double *var_out, void *snr_out, int n, int J, int R, uint64_t seed,
                 const fm_config &cfg, const NoiseLayout &L, char *scr, cudaStream_t s, DevStreams *ds,
                 double *ext_sums = nullptr, int rbase = 0)
{
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const long nn = (long)n * n;
    const long nb = (long)(J - 1) * nn;
    void *acc = ext_sums ? static_cast<void *>(ext_sums) : static_cast<void *>(scr);  // FP64 S1, S2 or the fp32
                                                                                       // Kahan pairs: 16 B / band px
    char *pyr = scr + L.acc_b, *slots = pyr + (size_t)L.pyr_bufs * L.pyr_b;
    const ChunkPlan &p = L.p;
    const bool multi = ds && L.slots > 1;
    const char *c1 = static_cast<const char *>(g1), *c2 = static_cast<const char *>(g2);
    int r;
    if (!ext_sums) FM_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)2 * nb * sizeof(double), s));
    for (int r0 = 0, ib = 0; r0 < R; r0 += L.batch, ++ib) {
        const int b = R - r0 < L.batch ? R - r0 : L.batch;
        const int buf = ib % L.pyr_bufs;
        char *pb = pyr + (size_t)buf * L.pyr_b;
        if (multi && (L.pyr_bufs == 1 || ib == 0)) {
            // start after `s` (the zeroed sums; with one buffer, the last accumulation)
            FM_CUDA_TRY(cudaEventRecord(ds->fork, s));
            for (int k = 0; k < L.slots; ++k) FM_CUDA_TRY(cudaStreamWaitEvent(ds->s[k], ds->fork, 0));
        } else if (multi && ib >= L.pyr_bufs) {
            // this buffer is free once the accumulation of batch ib - 2 has read it
            for (int k = 0; k < L.slots; ++k) FM_CUDA_TRY(cudaStreamWaitEvent(ds->s[k], ds->acc[buf], 0));
        }
        int i = 0;
        for (int c0 = 0; c0 < b; c0 += p.C, ++i) {
            const int k = multi ? i % L.slots : 0;
            const int bc = b - c0 < p.C ? b - c0 : p.C;
            if ((r = run_chunk(c1, c2, pb + (size_t)c0 * J * nn * es, n, J, 0, bc, cfg, p, slots + k * p.slot_b,
                               multi ? ds->s[k] : s, true, seed, rbase + r0 + c0)))
                return r;
        }
        if (multi)
            for (int k = 0; k < L.slots; ++k) {
                FM_CUDA_TRY(cudaEventRecord(ds->join[k], ds->s[k]));
                FM_CUDA_TRY(cudaStreamWaitEvent(s, ds->join[k], 0));
            }
        if ((r = launch_noise_accum(pb, b, (long)J * nn, nn, J - 1, acc, cfg.precision, cfg.accum, s))) return r;
        if (multi && L.pyr_bufs > 1) FM_CUDA_TRY(cudaEventRecord(ds->acc[buf], s));
    }
    if (ext_sums) return FM_OK;
    // S/N needs the unrotated bands; finalize reads them from the first pyramid
    // (every chunk stream has joined `s` after the last batch)
    if (snr_out && (r = run_chunk(c1, c2, pyr, n, J, 0, 1, cfg, p, slots, s))) return r;
    return launch_noise_finalize(acc, snr_out ? pyr : nullptr, var_out, snr_out, nb, R, cfg.precision, cfg.accum, s);
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
                  const fm_config &cfg, cudaStream_t s, bool allow_graph, bool multi_eager)
{
    int st = FM_OK;
    if (!twiddles(n, cfg.precision, s, &st)) return st;  // tables before any capture
    if (multi_eager && !allow_graph) {
        // launched now, chunks over the internal streams (stream-ordered scratch on s)
        const NoiseLayout L = noise_layout(n, J, R, cfg, true);
        Scratch sc;
        if ((st = scratch_alloc(sc, L.total, s))) return st;
        std::lock_guard<std::mutex> lk(g_ds_mu);
        DevStreams *ds = nullptr;
        if ((st = dev_streams(&ds))) return st;
        return noise_submit(g1, g2, var_out, snr_out, n, J, R, seed, cfg, L, (char *)sc.p, s, ds);
    }
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
                 g_pdl.load() | ((g_tile_variant.load() + 1) << 1) | (g_use_tma.load() << 3) | (g_wait_test.load() << 10) | ((g_ks_real.load() + 1) << 11)};
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
        cudaError_t ce = dev_malloc(&e.scratch, L.total);
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

// Realisations r0 .. r0 + R - 1 added to the caller's FP64 sums, on `s`
// (one stream, stream-ordered scratch).
int map_noise_accumulate_run(const void *g1, const void *g2, double *sums, int n, int J, int r0, int R, uint64_t seed,
                             const fm_config &cfg, cudaStream_t s)
{
    int st = FM_OK;
    if (!twiddles(n, cfg.precision, s, &st)) return st;
    const NoiseLayout L = noise_layout(n, J, R, cfg, false, true);
    Scratch sc;
    if ((st = scratch_alloc(sc, L.total, s))) return st;
    return noise_submit(g1, g2, nullptr, nullptr, n, J, R, seed, cfg, L, (char *)sc.p, s, nullptr, sums, r0);
}

// scratch of a noise call on the caller's stream (the serving path)
size_t noise_scratch_bytes(int n, int J, int R, const fm_config &cfg, bool with_snr, bool multi_stream)
{
    (void)with_snr;
    return noise_layout(n, J, R, cfg, multi_stream).total + 256;
}

int map_starlet_run(const void *g1, const void *g2, void *pyramid, int n, int J, int batch, const fm_config &cfg,
                    cudaStream_t s, bool allow_graph)
{
    return map_starlet_dev(g1, g2, pyramid, n, J, batch, cfg, s, allow_graph);
}

// Host buffers: the chunks of the batch stream through the slots of the
// internal streams; each copies its shear in, runs KS + starlet and copies its
// pyramid out.  A slot's next chunk follows its previous copy out on the same
// stream, so with two or more slots the copies of one chunk overlap the
// compute of another and the two copy directions overlap each other.
int map_starlet_host_run(const char *g1h, const char *g2h, char *pyrh, int n, int J, int batch, const fm_config &cfg,
                         cudaStream_t origin)
{
    ChunkPlan p = plan_chunks(n, J, batch, cfg);
    const size_t es = cfg.precision == FM_F64 ? 8 : 4, nn = (size_t)n * n;
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

using namespace fm;

extern "C" {

int fm_trim(void)
{
    std::lock_guard<std::mutex> lk(g_ds_mu);
    for (auto &e : g_graphs) drop_graph(e);
    g_graphs.clear();
    for (auto &e : g_noise_graphs) drop_noise_graph(e);
    g_noise_graphs.clear();
    return FM_OK;
}

int fm_tune(int knob, int64_t value)
{
    switch (knob) {
    case FM_TUNE_CHUNK_BYTES:
        g_chunk_bytes.store(value < 0 ? kDefaultChunkBytes : value);
        g_chunk_bytes_set.store(value >= 0);
        return FM_OK;
    case FM_TUNE_GRAPHS: g_use_graphs.store(value < 0 ? 1 : (value != 0)); return FM_OK;
    case FM_TUNE_CHUNK_STREAMS:
        g_chunk_streams.store(value < 0 ? 2 : (int)(value < 1 ? 1 : value > kMaxChunkStreams ? kMaxChunkStreams : value));
        return FM_OK;
    case FM_TUNE_PDL: g_pdl.store(value < 0 ? 1 : (value != 0)); return FM_OK;
    case FM_TUNE_TMA:
        if (value > 127) return einval("FM_TUNE_TMA is a mask of 1, 2, 4, 8, 16, 32 and 64");
        g_use_tma.store(value < 0 ? kDefaultTma : (int)value);
        return FM_OK;
    case FM_TUNE_WAIT_TEST: g_wait_test.store(value > 0 ? 1 : 0); return FM_OK;
    case FM_TUNE_SERVE_MERGE:
        if (value > 256) return einval("FM_TUNE_SERVE_MERGE takes at most 256 maps");
        g_serve_merge.store(value < 0 ? 16 : (value < 1 ? 1 : (int)value));
        return FM_OK;
    case FM_TUNE_SERVE_HEAVY:
        if (value > 64) return einval("FM_TUNE_SERVE_HEAVY takes at most 64");
        g_serve_heavy.store(value < 0 ? 1 : (int)value);
        return FM_OK;
    case FM_TUNE_KS_REAL: g_ks_real.store(value < 0 ? -1 : (value != 0)); return FM_OK;
    case FM_TUNE_DIRECT:
        if (value > 4) return einval("FM_TUNE_DIRECT takes 0 .. 4");
        g_direct_form.store(value < 0 ? -1 : (int)value);
        return FM_OK;
    case FM_TUNE_TILE:
        if (value > 1) return einval("FM_TUNE_TILE takes 0 or 1");
        g_tile_variant.store(value < 0 ? -1 : (int)value);
        return FM_OK;
    }
    return einval("unknown tuning knob");
}

}  // extern "C"
