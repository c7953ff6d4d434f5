// noise.cu -- randomised-shear noise maps (Sec. 1): the FP64 accumulation of
// the bands over realisations, the per-pixel unbiased variance and S/N, and
// the elementwise helpers of the exact expected variance.
#include "common.cuh"

namespace fm {

// S1 += sum_b w, S2 += sum_b w^2 over a batch of `nb` (<= 32) realisations'
// pyramids ([nb][J][n][n], bands 0..J-2 used).  The batch's partial sums are
// formed in the element type (at most 32 terms) and added once to the FP64
// running sums: GB300's FP64 rate is a small fraction of its FP32 rate, so
// the FP64 work is two additions per band pixel per batch.  The pyramids are
// read once with streaming (evict-first) loads, so they do not push the chunk
// pipeline's intermediates out of L2.
template <typename T, typename V>
__global__ void __launch_bounds__(256) k_noise_accum(const T *__restrict__ pyr, int nb, long pyr_bs, long nn,
                                                     int bands, double *__restrict__ s1, double *__restrict__ s2)
{
    pdl_entry();
    constexpr int VW = sizeof(V) / sizeof(T);
    const long nq = bands * nn / VW;  // nn % 4 == 0 (n a power of two >= 4)
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nq; i += (long)gridDim.x * blockDim.x) {
        const long e = i * VW;  // band-major element index: band * nn + pixel
        T a[VW], q[VW];
#pragma unroll
        for (int u = 0; u < VW; ++u) a[u] = q[u] = (T)0;
        for (int b = 0; b < nb; ++b) {
            const V v = __ldcs(reinterpret_cast<const V *>(pyr + b * pyr_bs + e));
            const T *w = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                a[u] += w[u];
                q[u] = fma(w[u], w[u], q[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            s1[e + u] += (double)a[u];
            s2[e + u] += (double)q[u];
        }
    }
}

// accum = 1 (fp32 maps): the running sums are fp32 with Kahan compensation
// (Kahan 1965): per element a sum s and a compensation c, the true sum being
// s - c; a batch's partial sum a enters as y = a - c, t = s + y,
// c = (t - s) - y, s = t.  The arrays are s1, c1, s2, c2, each nb floats.
__global__ void __launch_bounds__(256) k_noise_accum_kahan(const float *__restrict__ pyr, int nb, long pyr_bs,
                                                           long nn, int bands, float *__restrict__ acc)
{
    pdl_entry();
    const long ne = bands * nn;
    const long nq = ne / 4;
    float4 *s1 = reinterpret_cast<float4 *>(acc), *c1 = s1 + nq, *s2 = c1 + nq, *c2 = s2 + nq;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nq; i += (long)gridDim.x * blockDim.x) {
        float a[4] = {0.f, 0.f, 0.f, 0.f}, q[4] = {0.f, 0.f, 0.f, 0.f};
        for (int b = 0; b < nb; ++b) {
            const float4 v = __ldcs(reinterpret_cast<const float4 *>(pyr + b * pyr_bs) + i);
            const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] += w[u];
                q[u] = fmaf(w[u], w[u], q[u]);
            }
        }
        float4 S1 = s1[i], C1 = c1[i], S2 = s2[i], C2 = c2[i];
        float *ps1 = &S1.x, *pc1 = &C1.x, *ps2 = &S2.x, *pc2 = &C2.x;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float y1 = __fsub_rn(a[u], pc1[u]);
            const float t1 = __fadd_rn(ps1[u], y1);
            pc1[u] = __fsub_rn(__fsub_rn(t1, ps1[u]), y1);
            ps1[u] = t1;
            const float y2 = __fsub_rn(q[u], pc2[u]);
            const float t2 = __fadd_rn(ps2[u], y2);
            pc2[u] = __fsub_rn(__fsub_rn(t2, ps2[u]), y2);
            ps2[u] = t2;
        }
        s1[i] = S1;
        c1[i] = C1;
        s2[i] = S2;
        c2[i] = C2;
    }
}

// acc: FP64 s1, s2 (accum 0) or fp32 s1, c1, s2, c2 (accum 1), bands * nn each
int launch_noise_accum(const void *pyr, int nb, long pyr_bs, long nn, int bands, void *acc, int precision, int accum,
                       cudaStream_t s)
{
    long g = (bands * nn / 4 + 255) / 256;
    if (g > 152L * 16) g = 152L * 16;
    double *s1 = static_cast<double *>(acc), *s2 = s1 + (long)bands * nn;
    if (accum == 1)
        FM_LAUNCH(FM_K_NOISE_ACCUM, k_noise_accum_kahan, (unsigned)g, 256, 0, s, (const float *)pyr, nb, pyr_bs, nn,
                  bands, static_cast<float *>(acc));
    else if (precision == FM_F64)
        FM_LAUNCH(FM_K_NOISE_ACCUM, (k_noise_accum<double, double2>), (unsigned)g, 256, 0, s, (const double *)pyr,
                  nb, pyr_bs, nn, bands, s1, s2);
    else
        FM_LAUNCH(FM_K_NOISE_ACCUM, (k_noise_accum<float, float4>), (unsigned)g, 256, 0, s, (const float *)pyr, nb,
                  pyr_bs, nn, bands, s1, s2);
    return FM_OK;
}

// S1 and S2 of element i in FP64: the FP64 sums, or s - c of the Kahan pairs
template <bool KAHAN>
__device__ __forceinline__ void noise_sums(const void *acc, long nelem, long i, double &a, double &q)
{
    if constexpr (KAHAN) {
        const float *f = static_cast<const float *>(acc);
        a = (double)f[i] - (double)f[nelem + i];
        q = (double)f[2 * nelem + i] - (double)f[3 * nelem + i];
    } else {
        const double *d = static_cast<const double *>(acc);
        a = d[i];
        q = d[nelem + i];
    }
}

template <typename T, bool KAHAN>
__global__ void k_noise_final(const void *__restrict__ acc, const T *__restrict__ wdata, double *__restrict__ var,
                              T *__restrict__ snr, long nelem, int R)
{
    pdl_entry();
    const double invR = 1.0 / R, invR1 = 1.0 / (R - 1);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nelem; i += (long)gridDim.x * blockDim.x) {
        double a, q;
        noise_sums<KAHAN>(acc, nelem, i, a, q);
        double v = (q - a * a * invR) * invR1;
        v = v < 0 ? 0 : v;
        var[i] = v;
        if (snr) snr[i] = (T)((double)wdata[i] / sqrt(v));
    }
}

int launch_noise_finalize(const void *acc, const void *wdata, double *var, void *snr, long nelem, int R,
                          int precision, int accum, cudaStream_t s)
{
    long g = (nelem + 255) / 256;
    if (g > 152L * 16) g = 152L * 16;
    if (precision == FM_F64)
        FM_LAUNCH(FM_K_NOISE_FINAL, (k_noise_final<double, false>), (unsigned)g, 256, 0, s, acc,
                  (const double *)wdata, var, (double *)snr, nelem, R);
    else if (accum == 1)
        FM_LAUNCH(FM_K_NOISE_FINAL, (k_noise_final<float, true>), (unsigned)g, 256, 0, s, acc, (const float *)wdata,
                  var, (float *)snr, nelem, R);
    else
        FM_LAUNCH(FM_K_NOISE_FINAL, (k_noise_final<float, false>), (unsigned)g, 256, 0, s, acc, (const float *)wdata,
                  var, (float *)snr, nelem, R);
    return FM_OK;
}

// ---- exact expected variance (periodic boundary) ----------------------------
// out[c][p] = a[c][p]^2 + b[c][p]^2, c < count, p < nn (|K_j|^2 from the two
// delta responses; |gamma|^2 from the shear)
template <typename T>
__global__ void __launch_bounds__(256) k_modulus2(const T *__restrict__ a, long a_bs, const T *__restrict__ b,
                                                  long b_bs, T *__restrict__ out, long nn, int count)
{
    pdl_entry();
    const long total = nn * count;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        const long c = i / nn, p = i - c * nn;
        const T x = a[c * a_bs + p], y = b[c * b_bs + p];
        out[i] = x * x + y * y;
    }
}

// unit shear at pixel 0: gamma1 of map 0 and gamma2 of map 1 (arrays zeroed before)
template <typename T> __global__ void k_unit_shears(T *g1d, T *g2d, long nn)
{
    pdl_entry();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        g1d[0] = (T)1;
        g2d[nn] = (T)1;
    }
}

int launch_modulus2(const void *a, long a_bs, const void *b, long b_bs, void *out, long nn, int count, int precision,
                    cudaStream_t s)
{
    long g = (nn * count + 255) / 256;
    if (g > 152L * 16) g = 152L * 16;
    if (precision == FM_F64)
        FM_LAUNCH(0, k_modulus2<double>, (unsigned)g, 256, 0, s, (const double *)a, a_bs,
                  (const double *)b, b_bs, (double *)out, nn, count);
    else
        FM_LAUNCH(0, k_modulus2<float>, (unsigned)g, 256, 0, s, (const float *)a, a_bs,
                  (const float *)b, b_bs, (float *)out, nn, count);
    return FM_OK;
}

int launch_unit_shears(void *g1d, void *g2d, long nn, int precision, cudaStream_t s)
{
    const size_t es = precision == FM_F64 ? 8 : 4;
    FM_CUDA_TRY(cudaMemsetAsync(g1d, 0, 2 * nn * es, s));
    FM_CUDA_TRY(cudaMemsetAsync(g2d, 0, 2 * nn * es, s));
    if (precision == FM_F64)
        FM_LAUNCH(0, k_unit_shears<double>, 1, 32, 0, s, (double *)g1d, (double *)g2d, nn);
    else
        FM_LAUNCH(0, k_unit_shears<float>, 1, 32, 0, s, (float *)g1d, (float *)g2d, nn);
    return FM_OK;
}

}  // namespace fm
