// noalloc.cu -- Kaiser-Squires inversion that allocates no device memory.
//
// fm_ks_invert needs a complex work buffer of batch * n^2 elements, which it
// takes from the stream-ordered allocator.  Some callers cannot allocate at
// the point where they run the inversion: for instance a program whose device
// memory is reserved up front by another framework's pool, so that a fresh
// allocation would fail, or a latency-critical loop that must never enter the
// allocator.  fm_ks_invert_noalloc serves them: its work buffer and FFT
// twiddle tables live in file-scope device arrays (32 MiB + 32 KiB per
// device).  The driver allocates them when it loads this file's module on a
// device: under CUDA's default lazy module loading that happens at the first
// call on that device (the set-up below), with eager loading when the
// library's context starts; either way they are held until the process exits.
#include <math.h>

#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace fm {
namespace {

constexpr long kNoallocWorkElems = 4l << 20;  // float2 elements: 32 MiB
// batch * n^2 <= 4194304 caps n at 2048 (a batch of one)
constexpr int kTwMinN = 32, kTwMaxN = 2048;
constexpr int kTwElems = 2 * kTwMaxN - kTwMinN;  // tables n = 32, 64, ..., 2048 back to back

static __device__ __align__(256) float2 g_noalloc_work[kNoallocWorkElems];
static __device__ __align__(256) float2 g_noalloc_tw[kTwElems];

struct DevState {
    float2 *work = nullptr;  // device addresses of the two arrays on this device
    float2 *tw = nullptr;
};
std::mutex g_mu;
std::unordered_map<int, DevState> g_state;

// Once per device, with that device current: take the arrays' device
// addresses (their host-side names are only stand-ins) and fill the twiddle
// tables exp(-2 pi i t / n), computed on the host in FP64, with a synchronous
// copy.  Nothing is allocated.
int setup(int dev, DevState **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_state.find(dev);
    if (it != g_state.end()) {
        *out = &it->second;
        return FM_OK;
    }
    DevState st;
    FM_CUDA_TRY(cudaGetSymbolAddress((void **)&st.work, g_noalloc_work));
    FM_CUDA_TRY(cudaGetSymbolAddress((void **)&st.tw, g_noalloc_tw));
    std::vector<float2> host(kTwElems);
    for (int n = kTwMinN, off = 0; n <= kTwMaxN; off += n, n *= 2)
        for (int t = 0; t < n; ++t) {
            const double ang = -2.0 * M_PI * (double)t / (double)n;
            host[off + t] = make_float2((float)cos(ang), (float)sin(ang));
        }
    FM_CUDA_TRY(cudaMemcpy(st.tw, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice));
    *out = &(g_state[dev] = st);
    return FM_OK;
}

}  // namespace
}  // namespace fm

using namespace fm;

extern "C" int fm_ks_invert_noalloc(const void *g1, const void *g2, void *kappa_E, void *kappa_B, int n, int batch,
                                    const fm_config *cfg, void *stream)
{
    if (cfg) {
        const int c = check_config(*cfg);  // the same configs fm_ks_invert accepts
        if (c != FM_OK) return c;
        if (cfg->precision != FM_F32) {
            set_error("fm_ks_invert_noalloc: only FM_F32 is supported");
            return FM_EINVAL;
        }
    }
    if (n < kTwMinN || n > kTwMaxN || !is_pow2(n)) {
        set_error("fm_ks_invert_noalloc: n must be a power of two in [32, 2048]");
        return FM_EINVAL;
    }
    if (batch < 1 || (long)batch * n * n > kNoallocWorkElems) {
        set_error("fm_ks_invert_noalloc: batch * n^2 must be in [1, 4194304] (the static work buffer)");
        return FM_EINVAL;
    }
    if (!g1 || !g2 || !kappa_E) {
        set_error("fm_ks_invert_noalloc: null pointer");
        return FM_EINVAL;
    }
    int dev = 0;
    FM_CUDA_TRY(cudaGetDevice(&dev));
    DevState *st = nullptr;
    int r = setup(dev, &st);
    if (r != FM_OK) return r;
    const float2 *tw = st->tw + (n - kTwMinN);  // sum of the smaller tables' sizes
    // the half-length table for the real-output inverse where it is the faster one
    const float2 *tw2 = n >= 2 * kTwMinN && ks_real_for(n, false) ? st->tw + (n / 2 - kTwMinN) : nullptr;
    return launch_ks32((const float *)g1, (const float *)g2, (long)n * n, (float *)kappa_E, (float *)kappa_B, st->work,
                       n, batch, false, 0, 0, false, tw, tw2, (cudaStream_t)stream);
}
