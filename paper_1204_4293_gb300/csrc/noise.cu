// noise.cu -- finalize step of the randomised-shear noise maps (Sec. 1):
// per-pixel, per-band unbiased variance from FP64 sums and the S/N map.
#include "common.cuh"

namespace fm {

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
