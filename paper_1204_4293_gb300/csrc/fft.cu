// fft.cu -- batched 2-D FFT staged in shared memory, with the Kaiser-Squires
// multiplier fused between the column passes (Sec. 4.5).
//
// Three kernels per transform, each one HBM read and one HBM write:
//   rows_fwd : pack (gamma1 + i gamma2) [optionally rotated by a per-pixel
//              random angle for the noise maps, Sec. 1], row FFT
//   cols_ks  : column FFT -> multiply by conj(D) (inverse KS) or D (forward)
//              -> column inverse FFT, on a strip of W columns held in smem
//   rows_inv : row inverse FFT, scale 1/n^2, split into real / imaginary maps
// The 1-D transforms are Stockham autosort passes (radix 8, then 4 or 2),
// done in place in shared memory with a barrier between the loads and the
// stores of a pass; twiddles come from an FP64-computed table.
#include "common.cuh"
#include "dft.cuh"
#include "rng.cuh"

namespace fm {

// element address inside one smem vector: padded (one slot per 8) for the
// row layout to spread the stride-R stores over the banks.
template <bool PAD> __device__ __forceinline__ int eaddr(int i, int estride)
{
    return PAD ? i + (i >> 3) : i * estride;
}

// One Stockham pass of radix R over `nvec` vectors of length n held in smem.
// Element i of vector v sits at buf[v * vstride + eaddr(i)].  Every thread
// owns E/R butterflies; n * nvec == E * nthreads.
template <int R, int E, bool INV, bool VEC_FAST, bool PAD, typename V>
__device__ __forceinline__ void stockham_pass(V *buf, int n, int logn, int Ns, int lognvec, int vstride, int estride,
                                              const V *__restrict__ tw, int tid, int nthreads)
{
    constexpr int B = E / R;
    constexpr int LOGR = R == 8 ? 3 : (R == 4 ? 2 : 1);
    const int nbf = n >> LOGR;
    const int lognbf = logn - LOGR;
    V v[B][R];
    int jj[B];
    V *base[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        const int idx = tid + b * nthreads;
        int vec, j;
        if (VEC_FAST) {
            vec = idx & ((1 << lognvec) - 1);
            j = idx >> lognvec;
        } else {
            vec = idx >> lognbf;
            j = idx & (nbf - 1);
        }
        jj[b] = j;
        base[b] = buf + (long)vec * vstride;
        const int k = j & (Ns - 1);
        const int tstep = k * (n / (Ns * R));
#pragma unroll
        for (int r = 0; r < R; ++r) {
            V x = base[b][eaddr<PAD>(j + r * nbf, estride)];
            if (r > 0 && Ns > 1) {
                V w = __ldg(&tw[r * tstep]);
                if (INV) w.y = -w.y;
                x = cmul(x, w);
            }
            v[b][r] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B; ++b) {
        Dft<R, INV, V>::run(v[b]);
        const int j = jj[b];
        const int k = j & (Ns - 1);
        const int out0 = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) base[b][eaddr<PAD>(out0 + r * Ns, estride)] = v[b][r];
    }
    __syncthreads();
}

template <int E, bool INV, bool VEC_FAST, bool PAD, typename V>
__device__ void smem_fft(V *buf, int n, int logn, int lognvec, int vstride, int estride, const V *__restrict__ tw,
                         int tid, int nthreads)
{
    int Ns = 1;
    int rem = logn;
    while (rem > 0) {
        if (rem >= 3) {
            stockham_pass<8, E, INV, VEC_FAST, PAD>(buf, n, logn, Ns, lognvec, vstride, estride, tw, tid, nthreads);
            Ns <<= 3;
            rem -= 3;
        } else if (rem == 2) {
            stockham_pass<4, E, INV, VEC_FAST, PAD>(buf, n, logn, Ns, lognvec, vstride, estride, tw, tid, nthreads);
            Ns <<= 2;
            rem -= 2;
        } else {
            stockham_pass<2, E, INV, VEC_FAST, PAD>(buf, n, logn, Ns, lognvec, vstride, estride, tw, tid, nthreads);
            Ns <<= 1;
            rem -= 1;
        }
    }
}

// ---------------------------------------------------------------------------
// rows_fwd: one CTA holds `1 << lognvec` rows.  in2 may be null (real input).
template <typename T, int E>
__global__ void __launch_bounds__(1024) k_rows_fwd(const T *__restrict__ in1, const T *__restrict__ in2,
                                                   long in_bstride, cplx_t<T> *__restrict__ work, int n, int logn,
                                                   int lognvec, long total_rows, const cplx_t<T> *__restrict__ tw,
                                                   uint64_t seed, int r0, int rotate)
{
    pdl_entry();
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *buf = reinterpret_cast<V *>(smem_raw);
    const int rows = 1 << lognvec;
    const int vstride = n + (n >> 3);
    const long row0 = (long)blockIdx.x * rows;
    for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
        const int rr = idx >> logn, x = idx & (n - 1);
        const long grow = row0 + rr;
        V val = cmake<V>((T)0, (T)0);
        if (grow < total_rows) {
            const long b = grow >> logn;
            const int y = (int)(grow & (n - 1));
            const long off = b * in_bstride + (long)y * n + x;
            T a = in1[off];
            T c = in2 ? in2[off] : (T)0;
            if (rotate) rotate_shear(a, c, seed, r0 + b, y, x, n);
            val = cmake<V>(a, c);
        }
        buf[rr * vstride + x + (x >> 3)] = val;
    }
    __syncthreads();
    smem_fft<E, false, false, true>(buf, n, logn, lognvec, vstride, 1, tw, threadIdx.x, blockDim.x);
    for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
        const int rr = idx >> logn, x = idx & (n - 1);
        const long grow = row0 + rr;
        if (grow < total_rows) work[grow * n + x] = buf[rr * vstride + x + (x >> 3)];
    }
}

// cols_ks: one CTA holds a strip of W = 1 << logw columns of one map.
template <typename T, int E>
__global__ void __launch_bounds__(1024) k_cols_ks(cplx_t<T> *__restrict__ work, int n, int logn, int logw,
                                                  const cplx_t<T> *__restrict__ tw, int op,
                                                  const cplx_t<T> *__restrict__ filt)
{
    pdl_entry();
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *buf = reinterpret_cast<V *>(smem_raw);
    const int W = 1 << logw;
    const int strips = n >> logw;
    const long b = blockIdx.x / strips;
    const int x0 = (blockIdx.x % strips) * W;
    V *base = work + b * (long)n * n + x0;
    for (int idx = threadIdx.x; idx < n * W; idx += blockDim.x) {
        const int r = idx >> logw, c = idx & (W - 1);
        buf[idx] = base[(long)r * n + c];
    }
    __syncthreads();
    smem_fft<E, false, true, false>(buf, n, logn, logw, 1, W, tw, threadIdx.x, blockDim.x);
    if (op == FFT_OP_SPECTRUM) {  // the 2-D spectrum [ky][kx] is the result
        for (int idx = threadIdx.x; idx < n * W; idx += blockDim.x) {
            const int r = idx >> logw, c = idx & (W - 1);
            base[(long)r * n + c] = buf[idx];
        }
        return;
    }
    // kappa_hat = conj(D) gamma_hat (inverse) or gamma_hat = D kappa_hat (forward),
    // D = (k1 + i k2)^2 / |k|^2 = (k1^2 - k2^2 + 2 i k1 k2) / (k1^2 + k2^2), D(0) = 0;
    // or the given spectrum filt[b][ky][kx].
    const int half = n >> 1;
    for (int idx = threadIdx.x; idx < n * W; idx += blockDim.x) {
        const int r = idx >> logw, c = idx & (W - 1);
        const int xi = x0 + c;
        V d;
        if (op == FFT_OP_FILTER) {
            d = filt[b * (long)n * n + (long)r * n + xi];
        } else {
            const int k2 = r < half ? r : r - n;
            const int k1 = xi < half ? xi : xi - n;
            const int den = k1 * k1 + k2 * k2;
            d = cmake<V>((T)0, (T)0);
            if (den != 0) {
                const T inv = (T)1 / (T)den;
                const T re = (T)(k1 * k1 - k2 * k2) * inv;
                const T im = (T)(2 * k1 * k2) * inv;
                d = cmake<V>(re, op == FFT_OP_KS_FWD ? im : -im);
            }
        }
        buf[idx] = cmul(buf[idx], d);
    }
    __syncthreads();
    smem_fft<E, true, true, false>(buf, n, logn, logw, 1, W, tw, threadIdx.x, blockDim.x);
    for (int idx = threadIdx.x; idx < n * W; idx += blockDim.x) {
        const int r = idx >> logw, c = idx & (W - 1);
        base[(long)r * n + c] = buf[idx];
    }
}

// rows_inv: inverse row FFT, times `scale`, real part -> out1, imaginary -> out2.
template <typename T, int E>
__global__ void __launch_bounds__(1024) k_rows_inv(const cplx_t<T> *__restrict__ work, T *__restrict__ out1,
                                                   T *__restrict__ out2, int n, int logn, int lognvec,
                                                   long total_rows, const cplx_t<T> *__restrict__ tw, T scale)
{
    pdl_entry();
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V *buf = reinterpret_cast<V *>(smem_raw);
    const int rows = 1 << lognvec;
    const int vstride = n + (n >> 3);
    const long row0 = (long)blockIdx.x * rows;
    for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
        const int rr = idx >> logn, x = idx & (n - 1);
        const long grow = row0 + rr;
        V val = cmake<V>((T)0, (T)0);
        if (grow < total_rows) val = work[grow * n + x];
        buf[rr * vstride + x + (x >> 3)] = val;
    }
    __syncthreads();
    smem_fft<E, true, false, true>(buf, n, logn, lognvec, vstride, 1, tw, threadIdx.x, blockDim.x);
    for (int idx = threadIdx.x; idx < rows * n; idx += blockDim.x) {
        const int rr = idx >> logn, x = idx & (n - 1);
        const long grow = row0 + rr;
        if (grow < total_rows) {
            const V v = buf[rr * vstride + x + (x >> 3)];
            out1[grow * n + x] = v.x * scale;
            if (out2) out2[grow * n + x] = v.y * scale;
        }
    }
}

// ---------------------------------------------------------------------------
template <typename T>
static int ks_impl(const T *in1, const T *in2, long in_bstride, T *out1, T *out2, cplx_t<T> *work, int n, int batch,
                   int op, const cplx_t<T> *filt, T out_scale, uint64_t seed, int r0, bool rotate, cudaStream_t s)
{
    using V = cplx_t<T>;
    int st = FM_OK;
    const V *tw = static_cast<const V *>(twiddles(n, sizeof(T) == 8 ? FM_F64 : FM_F32, s, &st));
    if (!tw) return st;
    const int logn = ilog2((unsigned)n);
    const long total_rows = (long)batch * n;

    // rows: E = 8 elements per thread, 2048 elements per CTA when n <= 2048
    constexpr int ER = 8;
    const int rows_per = n >= 2048 ? 1 : 2048 / n;
    const int lognvec = ilog2((unsigned)rows_per);
    const int row_threads = rows_per * n / ER;
    const size_t row_smem = (size_t)rows_per * (n + (n >> 3)) * sizeof(V);
    const unsigned row_grid = (unsigned)((total_rows + rows_per - 1) / rows_per);

    // columns: fp32 E = 16 with W*n = 16384; fp64 E = 8 with W*n = 8192
    constexpr int EC = sizeof(T) == 4 ? 16 : 8;
    const int cap = sizeof(T) == 4 ? 16384 : 8192;
    const int W = n * n <= cap ? n : cap / n;
    const int logw = ilog2((unsigned)W);
    const int col_threads = W * n / EC;
    const size_t col_smem = (size_t)W * n * sizeof(V);
    const unsigned col_grid = (unsigned)((long)batch * (n / W));

    auto krf = k_rows_fwd<T, ER>;
    auto kcs = k_cols_ks<T, EC>;
    auto kri = k_rows_inv<T, ER>;
    FM_CUDA_TRY(fm::smem_attr((const void *)krf, row_smem));
    FM_CUDA_TRY(fm::smem_attr((const void *)kri, row_smem));
    FM_CUDA_TRY(fm::smem_attr((const void *)kcs, col_smem));

    FM_LAUNCH(FM_K_FFT_ROWS_FWD, krf, row_grid, row_threads, row_smem, s, in1, in2, in_bstride, work, n, logn,
              lognvec, total_rows, tw, seed, r0, rotate ? 1 : 0);
    FM_LAUNCH(FM_K_FFT_COLS_KS, kcs, col_grid, col_threads, col_smem, s, work, n, logn, logw, tw, op, filt);
    if (op == FFT_OP_SPECTRUM) return FM_OK;
    const T scale = out_scale / ((T)n * (T)n);
    FM_LAUNCH(FM_K_FFT_ROWS_INV, kri, row_grid, row_threads, row_smem, s, work, out1, out2, n, logn, lognvec,
              total_rows, tw, scale);
    return FM_OK;
}

int launch_fft_op(const void *in1, const void *in2, long in_bstride, void *out1, void *out2, void *work, int n,
                  int batch, int precision, int op, const void *filt, double out_scale, uint64_t rot_seed, int rot_r0,
                  bool rotate, cudaStream_t s, bool real_ok)
{
    if (precision == FM_F64)
        return ks_impl<double>((const double *)in1, (const double *)in2, in_bstride, (double *)out1, (double *)out2,
                               (double2 *)work, n, batch, op, (const double2 *)filt, out_scale, rot_seed, rot_r0,
                               rotate, s);
    if (n >= 32) {  // register-resident radix-32 path (fft32.cu)
        int st = FM_OK;
        const float2 *tw = static_cast<const float2 *>(twiddles(n, FM_F32, s, &st));
        if (!tw) return st;
        const float2 *tw2 = nullptr;  // the half-length table of the real-output inverse
        if (real_ok && n >= 64 && op == FFT_OP_KS_INV && !out2 &&
            !(tw2 = static_cast<const float2 *>(twiddles(n / 2, FM_F32, s, &st))))
            return st;
        return launch_fft32((const float *)in1, (const float *)in2, in_bstride, (float *)out1, (float *)out2,
                            (float2 *)work, n, batch, op, (const float2 *)filt, (float)out_scale, rot_seed, rot_r0,
                            rotate, tw, tw2, s);
    }
    return ks_impl<float>((const float *)in1, (const float *)in2, in_bstride, (float *)out1, (float *)out2,
                          (float2 *)work, n, batch, op, (const float2 *)filt, (float)out_scale, rot_seed, rot_r0,
                          rotate, s);
}

int launch_ks(const void *in1, const void *in2, long in_bstride, void *out1, void *out2, void *work, int n, int batch,
              int precision, bool forward, uint64_t rot_seed, int rot_r0, bool rotate, cudaStream_t s, bool batched)
{
    return launch_fft_op(in1, in2, in_bstride, out1, out2, work, n, batch, precision,
                         forward ? FFT_OP_KS_FWD : FFT_OP_KS_INV, nullptr, 1.0, rot_seed, rot_r0, rotate, s,
                         !forward && ks_real_for(n, batched));
}

}  // namespace fm
