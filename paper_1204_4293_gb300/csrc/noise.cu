// noise.cu -- finalize step of the randomised-shear noise maps (Sec. 1):
// per-pixel, per-band unbiased variance from FP64 sums and the S/N map.
#include "common.cuh"

namespace fm {

// S1 += sum_b w, S2 += sum_b w^2 over a batch of `nb` realisations' pyramids
// ([nb][J][n][n], bands 0..J-2 used); one thread per 4 band pixels, FP64
// sums in registers, one plain read-modify-write of S1 and S2 per batch.
template <typename T>
__global__ void __launch_bounds__(256) k_noise_accum(const T *__restrict__ pyr, int nb, long pyr_bs, long nn,
                                                     int bands, double *__restrict__ s1, double *__restrict__ s2)
{
    const long nq = bands * nn / 4;  // nn % 4 == 0 (n a power of two >= 4)
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nq; i += (long)gridDim.x * blockDim.x) {
        const long e = i * 4;  // band-major element index: band * nn + pixel
        double a[4] = {0, 0, 0, 0}, q[4] = {0, 0, 0, 0};
        for (int b = 0; b < nb; ++b) {
            const T *p = pyr + b * pyr_bs + e;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const double w = (double)__ldg(p + u);
                a[u] += w;
                q[u] += w * w;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s1[e + u] += a[u];
            s2[e + u] += q[u];
        }
    }
}

int launch_noise_accum(const void *pyr, int nb, long pyr_bs, long nn, int bands, double *s1, double *s2,
                       int precision, cudaStream_t s)
{
    long g = (bands * nn / 4 + 255) / 256;
    if (g > 152L * 16) g = 152L * 16;
    if (precision == FM_F64)
        FM_LAUNCH(FM_K_NOISE_FINAL, k_noise_accum<double>, (unsigned)g, 256, 0, s, (const double *)pyr, nb, pyr_bs,
                  nn, bands, s1, s2);
    else
        FM_LAUNCH(FM_K_NOISE_FINAL, k_noise_accum<float>, (unsigned)g, 256, 0, s, (const float *)pyr, nb, pyr_bs,
                  nn, bands, s1, s2);
    return FM_OK;
}

template <typename T>
__global__ void k_noise_final(const double *__restrict__ s1, const double *__restrict__ s2,
                              const T *__restrict__ wdata, double *__restrict__ var, T *__restrict__ snr, long nelem,
                              int R)
{
    const double invR = 1.0 / R, invR1 = 1.0 / (R - 1);
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nelem; i += (long)gridDim.x * blockDim.x) {
        const double a = s1[i], q = s2[i];
        double v = (q - a * a * invR) * invR1;
        v = v < 0 ? 0 : v;
        var[i] = v;
        if (snr) snr[i] = (T)((double)wdata[i] / sqrt(v));
    }
}

int launch_noise_finalize(const double *s1, const double *s2, const void *wdata, double *var, void *snr, long nelem,
                          int R, int precision, cudaStream_t s)
{
    long g = (nelem + 255) / 256;
    if (g > 152L * 16) g = 152L * 16;
    if (precision == FM_F64)
        FM_LAUNCH(FM_K_NOISE_FINAL, k_noise_final<double>, (unsigned)g, 256, 0, s, s1, s2, (const double *)wdata, var,
                  (double *)snr, nelem, R);
    else
        FM_LAUNCH(FM_K_NOISE_FINAL, k_noise_final<float>, (unsigned)g, 256, 0, s, s1, s2, (const float *)wdata, var,
                  (float *)snr, nelem, R);
    return FM_OK;
}

}  // namespace fm
