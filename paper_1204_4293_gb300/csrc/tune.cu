// tune.cu -- the autotuner of the batched KS + starlet path: it times
// fm_map_starlet on synthetic maps for candidate plans (fused depth,
// large-scale path 1 / 3 / 4, fp32 tile kernel form, chunk budget) and keeps the
// fastest per (n, J, precision) in a process-wide table that the automatic
// fields of fm_config follow; the table saves to and loads from JSON.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace fm {

namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TunedPlan> g_table;  // (n, J, precision) -> plan

bool valid_plan(const TunedPlan &p, int precision)
{
    const int fmax = precision == FM_F64 ? 3 : 4;
    return p.fuse >= 1 && p.fuse <= fmax && (p.large_path == 1 || p.large_path == 3 || p.large_path == 4) &&
           (p.tile == 0 || p.tile == 1) &&
           p.chunk_mb >= 0 && p.chunk_mb <= 65536;
}

void table_put(int n, int J, int precision, const TunedPlan &p)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table[std::make_tuple(n, J, precision)] = p;
}

void table_erase(int n, int J, int precision)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_table.erase(std::make_tuple(n, J, precision));
}

// synthetic shear for timing: uniform in [-0.1, 0.1) from a SplitMix64 hash
// of the element index (values do not change the kernels' work)
template <typename T> __global__ void k_tune_fill(T *p, long count, uint64_t salt)
{
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
        uint64_t z = (uint64_t)i + salt + 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        p[i] = (T)((double)(z >> 40) * (0.2 / 16777216.0) - 0.1);
    }
}

int fill(void *p, long count, int precision, uint64_t salt, cudaStream_t s)
{
    const unsigned g = (unsigned)std::min<long>((count + 255) / 256, 152L * 8);
    if (precision == FM_F64)
        k_tune_fill<double><<<g, 256, 0, s>>>((double *)p, count, salt);
    else
        k_tune_fill<float><<<g, 256, 0, s>>>((float *)p, count, salt);
    FM_CHECK_LAUNCH("k_tune_fill");
    return FM_OK;
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf()
    {
        if (p) cudaFree(p);
    }
};
struct Stream {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~Stream()
    {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

// the built-in rules, as if no table entry existed
TunedPlan builtin_plan(int n, int J, const fm_config &cfg)
{
    TunedPlan p;
    fm_config c = cfg;
    c.fuse_depth = 0;
    c.large_path = 0;
    p.fuse = starlet_builtin_fuse(n, J, c);
    p.large_path = starlet_builtin_large_path(n, J, p.fuse);
    p.tile = 1;
    p.chunk_mb = (int)(chunk_budget_default() >> 20);
    return p;
}
}  // namespace

bool tune_lookup(int n, int J, int precision, TunedPlan *out)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_table.find(std::make_tuple(n, J, precision));
    if (it == g_table.end()) return false;
    if (out) *out = it->second;
    return true;
}

}  // namespace fm

using namespace fm;

extern "C" {

int fm_autotune(int n, int J, int batch, const fm_config *cfgp, fm_plan *best)
{
    fm_config cfg;
    memset(&cfg, 0, sizeof(cfg));
    if (cfgp) cfg = *cfgp;
    if (cfg.precision != FM_F32 && cfg.precision != FM_F64) return einval("precision must be FM_F32 or FM_F64");
    if (cfg.boundary != FM_MIRROR && cfg.boundary != FM_PERIODIC) return einval("boundary must be FM_MIRROR or FM_PERIODIC");
    if (n < 4 || n > 8192 || !is_pow2(n)) return einval("n must be a power of two in [4, 8192]");
    if (J < 2 || J > 20 || (long)n < (1L << J)) return einval("J must be in [2, 20] with n >= 2^J");
    if (batch < 1) return einval("batch must be >= 1");
    cfg.fuse_depth = 0;  // the plans decide
    cfg.large_path = 0;
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const long nn = (long)n * n;
    DevBuf g1, g2, pyr;
    FM_CUDA_TRY(dev_malloc(&g1.p, (size_t)batch * nn * es));
    FM_CUDA_TRY(dev_malloc(&g2.p, (size_t)batch * nn * es));
    FM_CUDA_TRY(dev_malloc(&pyr.p, (size_t)batch * J * nn * es));
    Stream st;
    FM_CUDA_TRY(cudaStreamCreateWithFlags(&st.s, cudaStreamNonBlocking));
    FM_CUDA_TRY(cudaEventCreate(&st.e0));
    FM_CUDA_TRY(cudaEventCreate(&st.e1));
    int r;
    if ((r = fill(g1.p, batch * nn, cfg.precision, 1, st.s))) return r;
    if ((r = fill(g2.p, batch * nn, cfg.precision, 2, st.s))) return r;

    TunedPlan saved;
    const bool had = tune_lookup(n, J, cfg.precision, &saved);
    auto restore = [&]() {
        if (had)
            table_put(n, J, cfg.precision, saved);
        else
            table_erase(n, J, cfg.precision);
        fm_trim();
    };
    // time one plan: enter it in the table, drop graphs recorded with the old
    // one, run twice (the first call records the batched graph), then time
    // enough calls for ~20 ms of work
    auto time_plan = [&](const TunedPlan &p, double *ms) -> int {
        table_put(n, J, cfg.precision, p);
        fm_trim();
        for (int w = 0; w < 2; ++w)
            if ((r = map_starlet_run(g1.p, g2.p, pyr.p, n, J, batch, cfg, st.s))) return r;
        FM_CUDA_TRY(cudaEventRecord(st.e0, st.s));
        if ((r = map_starlet_run(g1.p, g2.p, pyr.p, n, J, batch, cfg, st.s))) return r;
        FM_CUDA_TRY(cudaEventRecord(st.e1, st.s));
        FM_CUDA_TRY(cudaEventSynchronize(st.e1));
        float one = 0.f;
        FM_CUDA_TRY(cudaEventElapsedTime(&one, st.e0, st.e1));
        const int reps = (int)std::min(50.0, std::max(3.0, ceil(20.0 / std::max(one, 1e-3f))));
        FM_CUDA_TRY(cudaEventRecord(st.e0, st.s));
        for (int k = 0; k < reps; ++k)
            if ((r = map_starlet_run(g1.p, g2.p, pyr.p, n, J, batch, cfg, st.s))) return r;
        FM_CUDA_TRY(cudaEventRecord(st.e1, st.s));
        FM_CUDA_TRY(cudaEventSynchronize(st.e1));
        float tot = 0.f;
        FM_CUDA_TRY(cudaEventElapsedTime(&tot, st.e0, st.e1));
        *ms = tot / reps;
        return FM_OK;
    };

    // coordinate descent from the built-in plan over fused depth, large-scale
    // path, tile form (fp32) and chunk budget, two sweeps; a candidate must
    // beat the best so far by 1 % to replace it
    const TunedPlan base = builtin_plan(n, J, cfg);
    std::vector<std::pair<TunedPlan, double>> seen;
    auto key = [](const TunedPlan &p) { return std::make_tuple(p.fuse, p.large_path, p.tile, p.chunk_mb); };
    auto measure = [&](const TunedPlan &p, double *ms) -> int {
        for (auto &e : seen)
            if (key(e.first) == key(p)) {
                *ms = e.second;
                return FM_OK;
            }
        int rr = time_plan(p, ms);
        if (rr == FM_OK) seen.push_back({p, *ms});
        return rr;
    };
    double base_ms = 0;
    if ((r = measure(base, &base_ms))) {
        restore();
        return r;
    }
    TunedPlan cur = base;
    double cur_ms = base_ms;
    const int fmax = std::min(cfg.precision == FM_F64 ? 3 : 4, J - 1);
    const int chunks[] = {24, 36, 48, 64, 96};
    for (int sweep = 0; sweep < 2; ++sweep) {
        for (int dim = 0; dim < 4; ++dim) {
            std::vector<TunedPlan> cand;
            if (dim == 0)
                for (int f = 1; f <= fmax; ++f) {
                    TunedPlan p = cur;
                    p.fuse = f;
                    cand.push_back(p);
                }
            if (dim == 1 && cur.fuse < J - 1)
                for (int lp : {1, 3, 4}) {
                    TunedPlan p = cur;
                    p.large_path = lp;
                    cand.push_back(p);
                }
            if (dim == 2 && cfg.precision == FM_F32)
                for (int t : {0, 1}) {
                    TunedPlan p = cur;
                    p.tile = t;
                    cand.push_back(p);
                }
            if (dim == 3 && batch > 1)
                for (int c : chunks) {
                    TunedPlan p = cur;
                    p.chunk_mb = c;
                    cand.push_back(p);
                }
            for (auto &p : cand) {
                double ms = 0;
                if ((r = measure(p, &ms))) {
                    restore();
                    return r;
                }
                if (ms < cur_ms * 0.99) {
                    cur = p;
                    cur_ms = ms;
                }
            }
        }
    }
    cur.ms = cur_ms;
    cur.default_ms = base_ms;
    table_put(n, J, cfg.precision, cur);
    fm_trim();
    if (best) {
        best->fuse_depth = cur.fuse;
        best->large_path = cur.large_path;
        best->tile = cur.tile;
        best->chunk_mb = cur.chunk_mb;
        best->ms = cur.ms;
        best->default_ms = cur.default_ms;
    }
    return FM_OK;
}

int fm_autotune_get(int n, int J, int precision, fm_plan *plan)
{
    TunedPlan p;
    if (!tune_lookup(n, J, precision, &p)) return FM_ENOTFOUND;
    if (plan) {
        plan->fuse_depth = p.fuse;
        plan->large_path = p.large_path;
        plan->tile = p.tile;
        plan->chunk_mb = p.chunk_mb;
        plan->ms = p.ms;
        plan->default_ms = p.default_ms;
    }
    return FM_OK;
}

int fm_autotune_set(int n, int J, int precision, const fm_plan *plan)
{
    if (!plan) return einval("null plan");
    if (precision != FM_F32 && precision != FM_F64) return einval("precision must be FM_F32 or FM_F64");
    if (n < 1 || J < 2 || J > 20 || (long)n < (1L << J)) return einval("J must be in [2, 20] with n >= 2^J");
    TunedPlan p;
    p.fuse = plan->fuse_depth;
    p.large_path = plan->large_path;
    p.tile = plan->tile;
    p.chunk_mb = plan->chunk_mb;
    p.ms = plan->ms;
    p.default_ms = plan->default_ms;
    if (!valid_plan(p, precision))
        return einval("plan: fuse_depth 1..4 (fp64 1..3), large_path 1, 3 or 4, tile 0 or 1, chunk_mb 0..65536");
    table_put(n, J, precision, p);
    return fm_trim();
}

int fm_autotune_clear(void)
{
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_table.clear();
    }
    return fm_trim();
}

// {"fastmap_autotune": 1, "entries": [{"n": .., "J": .., "precision": ..,
// "fuse_depth": .., "large_path": .., "tile": .., "chunk_mb": .., "ms": ..,
// "default_ms": ..}, ...]}, one entry per line
int fm_autotune_save(const char *path)
{
    if (!path) return einval("null path");
    std::map<std::tuple<int, int, int>, TunedPlan> copy;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        copy = g_table;
    }
    FILE *f = fopen(path, "w");
    if (!f) return einval(std::string("cannot write ") + path);
    fprintf(f, "{\"fastmap_autotune\": 1, \"entries\": [");
    bool first = true;
    for (auto &e : copy) {
        const TunedPlan &p = e.second;
        fprintf(f,
                "%s\n  {\"n\": %d, \"J\": %d, \"precision\": %d, \"fuse_depth\": %d, \"large_path\": %d, "
                "\"tile\": %d, \"chunk_mb\": %d, \"ms\": %.6f, \"default_ms\": %.6f}",
                first ? "" : ",", std::get<0>(e.first), std::get<1>(e.first), std::get<2>(e.first), p.fuse,
                p.large_path, p.tile, p.chunk_mb, p.ms, p.default_ms);
        first = false;
    }
    fprintf(f, "\n]}\n");
    const bool ok = fclose(f) == 0;
    return ok ? FM_OK : einval(std::string("cannot write ") + path);
}

namespace {
// value of "key": <number> inside one entry's text; false if absent
bool json_num(const std::string &obj, const char *key, double *v)
{
    const std::string k = std::string("\"") + key + "\"";
    size_t p = obj.find(k);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + k.size());
    if (p == std::string::npos) return false;
    const char *s = obj.c_str() + p + 1;
    char *end = nullptr;
    *v = strtod(s, &end);
    return end != s;
}
}  // namespace

// Entries are merged into the table (an entry replaces the one with the same
// key); a malformed file changes nothing and returns FM_EINVAL.
int fm_autotune_load(const char *path)
{
    if (!path) return einval("null path");
    FILE *f = fopen(path, "r");
    if (!f) return einval(std::string("cannot read ") + path);
    std::string text;
    char buf[4096];
    size_t got;
    while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
    fclose(f);
    if (text.find("\"fastmap_autotune\"") == std::string::npos) return einval("not an autotune table");
    size_t p = text.find("\"entries\"");
    if (p == std::string::npos) return einval("autotune table without entries");
    std::vector<std::pair<std::tuple<int, int, int>, TunedPlan>> add;
    while ((p = text.find('{', p)) != std::string::npos) {
        const size_t q = text.find('}', p);
        if (q == std::string::npos) return einval("unterminated autotune entry");
        const std::string obj = text.substr(p, q - p + 1);
        p = q + 1;
        double n, J, prec, fuse, lp, tile, chunk, ms = 0, dms = 0;
        if (!json_num(obj, "n", &n) || !json_num(obj, "J", &J) || !json_num(obj, "precision", &prec) ||
            !json_num(obj, "fuse_depth", &fuse) || !json_num(obj, "large_path", &lp) || !json_num(obj, "tile", &tile) ||
            !json_num(obj, "chunk_mb", &chunk))
            return einval("autotune entry misses a field: " + obj);
        json_num(obj, "ms", &ms);
        json_num(obj, "default_ms", &dms);
        TunedPlan t;
        t.fuse = (int)fuse;
        t.large_path = (int)lp;
        t.tile = (int)tile;
        t.chunk_mb = (int)chunk;
        t.ms = ms;
        t.default_ms = dms;
        const int ni = (int)n, Ji = (int)J, pi = (int)prec;
        if ((pi != FM_F32 && pi != FM_F64) || ni < 1 || Ji < 2 || Ji > 20 || (long)ni < (1L << Ji) ||
            !valid_plan(t, pi))
            return einval("invalid autotune entry: " + obj);
        add.push_back({std::make_tuple(ni, Ji, pi), t});
    }
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto &e : add) g_table[e.first] = e.second;
    }
    return fm_trim();
}

}  // extern "C"
