// moments.cu -- statistics of the aperture-mass maps (Sec. 2.2): per map and
// per pyramid array the mean, variance <M_ap^2>, skewness and excess
// kurtosis over the pixels.
//
// Two passes over the pyramid: the first sums x per (map, array), the second
// sums (x - mean)^2, ^3, ^4.  Each thread keeps fp32 partial sums over its
// pixels, a block folds them in FP64 through warp shuffles and one FP64
// atomic per block and quantity lands in the per-array sums; a last tiny
// kernel forms the moments.
#include "common.cuh"

namespace fm {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// grid = (blocks per array, J, batch); sums[(b * J + j) * 4 + q]
template <typename T, int PASS>
__global__ void __launch_bounds__(256) k_moments(const T *__restrict__ pyr, long nn, int J, double *__restrict__ sums)
{
    pdl_entry();
    const long b = blockIdx.z;
    const int j = blockIdx.y;
    const T *x = pyr + (b * J + j) * nn;
    double *acc = sums + (b * J + j) * 4;
    const float mean = PASS == 0 ? 0.f : (float)(acc[0] / (double)nn);
    float s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nn; i += (long)gridDim.x * blockDim.x) {
        const float v = (float)x[i];
        if (PASS == 0) {
            s1 += v;
        } else {
            const float d = v - mean, d2 = d * d;
            s1 += d2;
            s2 += d2 * d;
            s3 += d2 * d2;
        }
    }
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double r0 = warp_sum((double)s1), r1 = 0, r2 = 0;
    if (PASS) {
        r1 = warp_sum((double)s2);
        r2 = warp_sum((double)s3);
    }
    if (lane == 0) {
        red[0][warp] = r0;
        red[1][warp] = r1;
        red[2][warp] = r2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t0 += red[0][w];
            t1 += red[1][w];
            t2 += red[2][w];
        }
        if (PASS == 0) {
            atomicAdd(acc + 0, t0);
        } else {
            atomicAdd(acc + 1, t0);
            atomicAdd(acc + 2, t1);
            atomicAdd(acc + 3, t2);
        }
    }
}

// moments[(b * J + j) * 4 + {0,1,2,3}] = mean, variance, skewness, excess kurtosis
__global__ void k_moments_final(const double *__restrict__ sums, double *__restrict__ out, long nn, int count)
{
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double *s = sums + 4 * (long)i;
    const double m2 = s[1] / (double)nn, m3 = s[2] / (double)nn, m4 = s[3] / (double)nn;
    double *o = out + 4 * (long)i;
    o[0] = s[0] / (double)nn;
    o[1] = m2;
    o[2] = m2 > 0 ? m3 / (m2 * sqrt(m2)) : 0.0;
    o[3] = m2 > 0 ? m4 / (m2 * m2) - 3.0 : 0.0;
}

int launch_band_moments(const void *pyr, double *moments, int n, int J, int batch, int precision, void *scratch,
                        cudaStream_t s)
{
    const long nn = (long)n * n;
    double *sums = static_cast<double *>(scratch);
    const int count = batch * J;
    FM_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(double) * 4 * (size_t)count, s));
    long per = (nn + 256 * 16 - 1) / (256 * 16);  // ~16 pixels per thread (fp32 partial sums)
    if (per > 4096) per = 4096;
    const dim3 grid((unsigned)per, J, batch);
    if (precision == FM_F64) {
        FM_LAUNCH(0, (k_moments<double, 0>), grid, 256, 0, s, (const double *)pyr, nn, J, sums);
        FM_LAUNCH(0, (k_moments<double, 1>), grid, 256, 0, s, (const double *)pyr, nn, J, sums);
    } else {
        FM_LAUNCH(0, (k_moments<float, 0>), grid, 256, 0, s, (const float *)pyr, nn, J, sums);
        FM_LAUNCH(0, (k_moments<float, 1>), grid, 256, 0, s, (const float *)pyr, nn, J, sums);
    }
    FM_LAUNCH(0, k_moments_final, (unsigned)((count + 127) / 128), 128, 0, s, sums, moments, nn, count);
    return FM_OK;
}

}  // namespace fm
