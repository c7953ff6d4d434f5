// fft32.cu -- fp32 Kaiser-Squires FFT (Sec. 4.5) with register-resident
// radix-32 sub-transforms, for n = 32 .. 8192.
//
// A length-n transform (n = 2^LOGN) is split into Stockham passes: radix 32,
// then radix 32 again while needed, then one last radix RL = n / 32^k.  Each
// thread owns 32 elements.  The first pass reads its inputs straight from
// global memory (x[j + r n/32], coalesced over j), the last pass writes its
// outputs straight back (X[b + r n/RL], coalesced over b), and the passes in
// between exchange through shared memory (one slot of padding per 32
// elements keeps the stride-32 stores conflict free).  Small DFTs run in
// registers with constant twiddles; inter-pass twiddles come from the FP64
// table.
//
//   rows_fwd32 : (gamma1 + i gamma2) [rotated for noise maps] -> row FFT
//   cols_ks32  : column FFT -> x conj(D) (or D, or a given spectrum) ->
//                column inverse FFT, on a strip of W columns; for n = 1024 the
//                forward output is already in the inverse's input order, so it
//                stays in registers.  The spectrum-only mode stores the 2-D
//                spectrum after the forward transform.
//   rows_inv32 : row inverse FFT -> (Re, Im) * scale / n^2
#include "common.cuh"
#include "dft.cuh"
#include "rng.cuh"
#include "tma.cuh"

namespace fm {

__device__ __forceinline__ int pad32(int a) { return a + (a >> 5); }

// threads of a row-pass CTA (RPC rows of TV threads; one row when TV is
// larger): 128-thread CTAs overlap better with the other chunk stream's
// kernels than 256-thread ones (KS + starlet, 256 -> 128: 32 x 1024^2
// 0.813 -> 0.805 ms, 16 x 2048^2 2.025 -> 1.988, 16 x 4096^2 10.95 -> 10.83,
// noise R = 1000 at 1024^2 31.1 -> 30.7)
constexpr int kRowThreads = 128;

template <int LOGN> struct Plan32 {
    static constexpr int N = 1 << LOGN;
    static constexpr int TV = N / 32;                     // threads per vector
    static constexpr int NPASS = (LOGN + 4) / 5;          // passes (all radix 32 but the last)
    static constexpr int LOGRL = LOGN - 5 * (NPASS - 1);  // log2 of the last radix
    static constexpr int RL = 1 << LOGRL;
    static constexpr int ML = 32 / RL;                    // butterflies per thread in the last pass
    static constexpr int NSL = N / RL;                    // stride of the last pass outputs
    // column strip width: 64 B row segments at n = 1024, 32 B at 2048 and
    // 4096 (one full sector; 512 threads, 136 KB of shared memory at 4096:
    // 13 % faster than 16 B strips), 16 B at 8192
    static constexpr int W = N <= 512 ? 16 : (N >= 8192 ? 2 : (N == 4096 ? 4 : 8192 / N));
};

template <bool INV> __device__ __forceinline__ float2 twid(const float2 *__restrict__ tw, int t)
{
    float2 w = __ldg(tw + t);
    if (INV) w.y = -w.y;
    return w;
}

// In: v[r] = x[j + r TV].  Out: v[m RL + r] = X[j + m TV + r NSL].
// Element i of the vector lives at sm[pad32(i W + c)] between passes.
// Every thread of the CTA must call this (it holds barriers).
template <int LOGN, int W, bool INV>
__device__ __forceinline__ void fft_vec(float2 (&v)[32], float2 *sm, int c, int j, const float2 *__restrict__ tw)
{
    using P = Plan32<LOGN>;
    Dft<32, INV, float2>::run(v);  // pass 1: Ns = 1, no twiddles; outputs at 32 j + r
    if constexpr (P::NPASS > 1) {
        __syncthreads();  // the buffer may still be read by an earlier pass
#pragma unroll
        for (int r = 0; r < 32; ++r) sm[pad32((j * 32 + r) * W + c)] = v[r];
        __syncthreads();
        if constexpr (P::NPASS > 2) {
            // pass 2: radix 32, Ns = 32
            constexpr int NS = 32;
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = sm[pad32((j + r * P::TV) * W + c)];
            const int k = j & (NS - 1);
            const int step = k * (P::N / (NS * 32));
#pragma unroll
            for (int r = 1; r < 32; ++r) v[r] = cmul(v[r], twid<INV>(tw, r * step));
            Dft<32, INV, float2>::run(v);
            __syncthreads();
            const int o = (j - k) * 32 + k;
#pragma unroll
            for (int r = 0; r < 32; ++r) sm[pad32((o + r * NS) * W + c)] = v[r];
            __syncthreads();
        }
        // last pass: radix RL, Ns = NSL, butterfly b = j + m TV (< NSL), twiddle W_n^(r b)
#pragma unroll
        for (int m = 0; m < P::ML; ++m) {
            const int b = j + m * P::TV;
#pragma unroll
            for (int r = 0; r < P::RL; ++r) {
                float2 x = sm[pad32((b + r * P::NSL) * W + c)];
                if (r > 0) x = cmul(x, twid<INV>(tw, r * b));
                v[m * P::RL + r] = x;
            }
            Dft<P::RL, INV, float2>::run(v + m * P::RL);
        }
    }
}

// With use_tma (n >= 64; in_bs = n^2, or in_bs = 0 with RPC <= n), the CTA's
// rows of gamma1 (m1) and gamma2 (m2) arrive by bulk tensor copies into the
// exchange buffer, viewed as [RPC][n] floats per array, before the first
// pass reads them.
template <int LOGN>
__global__ void __launch_bounds__(256, 2) k_rows_fwd32(const float *__restrict__ in1, const float *__restrict__ in2,
                                                       long in_bs, float2 *__restrict__ work, long total_rows,
                                                       const float2 *__restrict__ tw, uint64_t seed, int r0,
                                                       int rotate, const __grid_constant__ CUtensorMap m1,
                                                       const __grid_constant__ CUtensorMap m2, int use_tma)
{
    pdl_entry();
    using P = Plan32<LOGN>;
    constexpr int RPC = P::TV >= kRowThreads ? 1 : kRowThreads / P::TV;
    extern __shared__ __align__(16) float2 sm32[];
    __shared__ uint64_t bar;
    float2 *smb = align128<float2>(sm32);
    const int vr = threadIdx.x / P::TV, j = threadIdx.x % P::TV;
    const long row = (long)blockIdx.x * RPC + vr;
    float2 *sm = smb + vr * (P::N + P::N / 32);
    const bool live = row < total_rows;
    float2 v[32];
    bool staged = false;
    if constexpr (P::NPASS > 1) {
        if (use_tma) {
            float *st1 = reinterpret_cast<float *>(smb), *st2 = st1 + RPC * P::N;
            if (threadIdx.x == 0) mbar_init(&bar, 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                const long row0 = (long)blockIdx.x * RPC;
                const int z = (int)(in_bs == 0 ? (row0 & (P::N - 1)) : row0);
                mbar_expect_tx(&bar, (uint32_t)(RPC * P::N * sizeof(float) * (in2 ? 2 : 1)));
                tma_load_3d(st1, &m1, 0, 0, z, &bar);
                if (in2) tma_load_3d(st2, &m2, 0, 0, z, &bar);
            }
            if (!tma_wait_all(&bar, 0)) return;  // the copies never completed (flagged)
            const long b = row >> LOGN;
            const int y = (int)(row & (P::N - 1));
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int x = j + r * P::TV;
                float a = st1[vr * P::N + x];
                float cc = in2 ? st2[vr * P::N + x] : 0.f;
                if (rotate) rotate_shear(a, cc, seed, r0 + b, y, x, P::N);
                v[r] = make_float2(a, cc);
            }
            staged = true;  // fft_vec's first barrier orders these reads before the exchange writes
        }
    }
    if (!staged && live) {
        const long b = row >> LOGN;
        const int y = (int)(row & (P::N - 1));
        const float *p1 = in1 + b * in_bs + (long)y * P::N;
        const float *p2 = in2 ? in2 + b * in_bs + (long)y * P::N : nullptr;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const int x = j + r * P::TV;
            float a = __ldcs(p1 + x);  // the shear is read once
            float cc = p2 ? __ldcs(p2 + x) : 0.f;
            if (rotate) rotate_shear(a, cc, seed, r0 + b, y, x, P::N);
            v[r] = make_float2(a, cc);
        }
    } else if (!staged) {
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    }
    fft_vec<LOGN, 1, false>(v, sm, 0, j, tw);
    if (live) {
        float2 *dst = work + row * P::N;
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) dst[j + m * P::TV + r * P::NSL] = v[m * P::RL + r];
    }
}

// With use_tma (n >= 64, every CTA's RPC rows inside the batch), the CTA's
// complex rows arrive by one bulk tensor copy (mw: the work buffer as floats)
// into the exchange buffer, viewed as [RPC][n] float2.
template <int LOGN>
__global__ void __launch_bounds__(256, 2) k_rows_inv32(const float2 *__restrict__ work, float *__restrict__ out1,
                                                       float *__restrict__ out2, long total_rows,
                                                       const float2 *__restrict__ tw, float scale,
                                                       const __grid_constant__ CUtensorMap mw, int use_tma)
{
    pdl_entry();
    using P = Plan32<LOGN>;
    constexpr int RPC = P::TV >= kRowThreads ? 1 : kRowThreads / P::TV;
    extern __shared__ __align__(16) float2 sm32[];
    __shared__ uint64_t bar;
    float2 *smb = align128<float2>(sm32);
    const int vr = threadIdx.x / P::TV, j = threadIdx.x % P::TV;
    const long row = (long)blockIdx.x * RPC + vr;
    float2 *sm = smb + vr * (P::N + P::N / 32);
    const bool live = row < total_rows;
    float2 v[32];
    bool staged = false;
    if constexpr (P::NPASS > 1) {
        if (use_tma) {
            if (threadIdx.x == 0) mbar_init(&bar, 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                mbar_expect_tx(&bar, (uint32_t)(RPC * P::N * sizeof(float2)));
                tma_load_3d(smb, &mw, 0, 0, (int)((long)blockIdx.x * RPC), &bar);
            }
            if (!tma_wait_all(&bar, 0)) return;  // the copy never completed (flagged)
#pragma unroll
            for (int r = 0; r < 32; ++r) v[r] = smb[vr * P::N + j + r * P::TV];
            staged = true;  // fft_vec's first barrier orders these reads before the exchange writes
        }
    }
    if (!staged) {
        const float2 *src = work + row * P::N;
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = live ? src[j + r * P::TV] : make_float2(0.f, 0.f);
    }
    fft_vec<LOGN, 1, true>(v, sm, 0, j, tw);
    if (live) {
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) {
                const long pos = row * P::N + j + m * P::TV + r * P::NSL;
                const float2 x = v[m * P::RL + r];
                out1[pos] = x.x * scale;
                if (out2) out2[pos] = x.y * scale;
            }
    }
}

// With use_tma bit 0 (mw: the work buffer as floats {2n, n, batch}, box
// {2W, min(n, 256), 1}), the CTA's strip of W columns arrives by
// n / min(n, 256) bulk tensor copies into the exchange buffer, densely as
// [n][W] float2, instead of 32 strided loads per thread; with bit 1 the
// result leaves the same way (the spectrum-only mode stores per thread).
template <int LOGN>
__global__ void __launch_bounds__(512) k_cols_ks32(float2 *__restrict__ work, const float2 *__restrict__ tw,
                                                   int op, const float2 *__restrict__ filt,
                                                   const __grid_constant__ CUtensorMap mw, int use_tma)
{
    pdl_entry();
    using P = Plan32<LOGN>;
    constexpr int W = P::W, N = P::N;
    constexpr int STRIPS = N / W;
    extern __shared__ __align__(16) unsigned char smem_col[];
    float2 *sm32 = align128<float2>(smem_col);
    const long b = blockIdx.x / STRIPS;
    const int x0 = (blockIdx.x % STRIPS) * W;
    const int c = threadIdx.x % W, j = threadIdx.x / W;
    float2 *base = work + b * (long)N * N + x0 + c;
    float2 v[32];
    if (use_tma & 1) {
        __shared__ uint64_t bar;
        constexpr int BR = N < 256 ? N : 256;  // rows per copy
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, (uint32_t)(N * W * sizeof(float2)));
            for (int k = 0; k < N / BR; ++k) tma_load_3d(sm32 + k * BR * W, &mw, 2 * x0, k * BR, (int)b, &bar);
        }
        if (!tma_wait_all(&bar, 0)) return;  // the copies never completed (flagged)
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = sm32[(j + r * P::TV) * W + c];
    } else {
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = base[(long)(j + r * P::TV) * N];
    }
    fft_vec<LOGN, W, false>(v, sm32, c, j, tw);
    if (op == FFT_OP_SPECTRUM) {  // the 2-D spectrum [ky][kx] is the result
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) base[(long)(j + m * P::TV + r * P::NSL) * N] = v[m * P::RL + r];
        return;
    }
    // kappa_hat = conj(D) gamma_hat (inverse KS) or D kappa_hat (forward KS),
    // D = (k1^2 - k2^2 + 2 i k1 k2) / (k1^2 + k2^2), D(0) = 0; or the given
    // spectrum filt[b][ky][kx]
    const int xi = x0 + c;
    const int k1 = xi < N / 2 ? xi : xi - N;
    const float2 *fb = filt ? filt + b * (long)N * N + xi : nullptr;
#pragma unroll
    for (int m = 0; m < P::ML; ++m)
#pragma unroll
        for (int r = 0; r < P::RL; ++r) {
            const int yi = j + m * P::TV + r * P::NSL;
            float2 d;
            if (op == FFT_OP_FILTER) {
                d = fb[(long)yi * N];
            } else {
                const int k2 = yi < N / 2 ? yi : yi - N;
                const int den = k1 * k1 + k2 * k2;
                d = make_float2(0.f, 0.f);
                if (den != 0) {
                    const float inv = 1.f / (float)den;
                    const float im = (float)(2 * k1 * k2) * inv;
                    d = make_float2((float)(k1 * k1 - k2 * k2) * inv, op == FFT_OP_KS_FWD ? im : -im);
                }
            }
            v[m * P::RL + r] = cmul(v[m * P::RL + r], d);
        }
    if constexpr (!(P::RL == 32 || P::NPASS == 1)) {
        // bring the spectrum back to the inverse's input order x[j + r TV]
        __syncthreads();
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) sm32[pad32((j + m * P::TV + r * P::NSL) * W + c)] = v[m * P::RL + r];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = sm32[pad32((j + r * P::TV) * W + c)];
    }
    fft_vec<LOGN, W, true>(v, sm32, c, j, tw);
    if (use_tma & 2) {
        // the strip back through shared memory, dense [n][W], and out by bulk
        // tensor stores of the same boxes
        constexpr int BR = N < 256 ? N : 256;
        __syncthreads();  // the last pass may still read the exchange buffer
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) sm32[(j + m * P::TV + r * P::NSL) * W + c] = v[m * P::RL + r];
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 0; k < N / BR; ++k) tma_store_3d(&mw, 2 * x0, k * BR, (int)b, sm32 + k * BR * W);
            bulk_commit();
            bulk_wait_all();
        }
        return;
    }
#pragma unroll
    for (int m = 0; m < P::ML; ++m)
#pragma unroll
        for (int r = 0; r < P::RL; ++r) base[(long)(j + m * P::TV + r * P::NSL) * N] = v[m * P::RL + r];
}

// ---------------------------------------------------------------------------
template <int LOGN>
static int ks32_impl(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int batch,
                     int op, const float2 *filt, float out_scale, uint64_t seed, int r0, bool rotate,
                     const float2 *tw, cudaStream_t s)
{
    using P = Plan32<LOGN>;
    constexpr int RPC = P::TV >= kRowThreads ? 1 : kRowThreads / P::TV;
    const long total_rows = (long)batch * P::N;
    const unsigned row_grid = (unsigned)((total_rows + RPC - 1) / RPC);
    // exchange buffer (which also stages the TMA rows: RPC n floats per input
    // array or RPC n float2 <= RPC (n + n/32) float2) + 128 bytes of alignment
    const size_t row_smem = P::NPASS > 1 ? (size_t)RPC * (P::N + P::N / 32) * sizeof(float2) + 128 : 0;
    const int col_threads = P::W * P::TV;
    // exchange buffer (also the TMA strip: n W float2) + 128 bytes of alignment
    const size_t col_smem = P::NPASS > 1 ? (size_t)(P::N * P::W + P::N * P::W / 32 + 1) * sizeof(float2) + 128 : 0;
    const unsigned col_grid = (unsigned)((long)batch * (P::N / P::W));
    FM_CUDA_TRY(fm::smem_attr((const void *)k_rows_fwd32<LOGN>, row_smem));
    FM_CUDA_TRY(fm::smem_attr((const void *)k_rows_inv32<LOGN>, row_smem));
    FM_CUDA_TRY(fm::smem_attr((const void *)k_cols_ks32<LOGN>, col_smem));
    // bulk tensor copies of whole row groups (RPC consecutive rows of the
    // batch): n >= 64; the input rows either contiguous over the batch
    // (in_bs = n^2) or one broadcast map (in_bs = 0) holding a CTA's rows
    CUtensorMap m1, m2, mw;
    memset(&m1, 0, sizeof(m1));
    memset(&m2, 0, sizeof(m2));
    memset(&mw, 0, sizeof(mw));
    int tma_in = 0, tma_out = 0;
    const int tma_mode = g_use_tma.load(std::memory_order_relaxed);
    if (P::NPASS > 1 && (tma_mode & 6)) {
        const long nn = (long)P::N * P::N;
        const uint32_t d0 = P::N < 256 ? P::N : 256;
        const uint64_t rows = in_bs == 0 ? (uint64_t)P::N : (uint64_t)total_rows;
        const uint64_t dims[3] = {d0, (uint64_t)(P::N / d0), rows};
        const uint64_t strides[2] = {(uint64_t)d0 * 4, (uint64_t)P::N * 4};
        const uint32_t box[3] = {d0, (uint32_t)(P::N / d0), (uint32_t)RPC};
        // a broadcast map needs each CTA's rows inside it (RPC <= n, i.e. n >= 128)
        tma_in = (tma_mode & 2) && (in_bs == nn || (in_bs == 0 && RPC <= P::N)) &&
                 encode_map3d_f32(&m1, in1, dims, strides, box) && (!in2 || encode_map3d_f32(&m2, in2, dims, strides, box));
        const uint32_t e0 = 2 * P::N < 256 ? 2 * P::N : 256;
        const uint64_t wdims[3] = {e0, (uint64_t)(2 * P::N / e0), (uint64_t)total_rows};
        const uint64_t wstrides[2] = {(uint64_t)e0 * 4, (uint64_t)P::N * 8};
        const uint32_t wbox[3] = {e0, (uint32_t)(2 * P::N / e0), (uint32_t)RPC};
        tma_out = (tma_mode & 4) && encode_map3d_f32(&mw, work, wdims, wstrides, wbox);
    }
    // column strips by bulk tensor copies: the work buffer as floats
    // {2n, n, batch}, a box of 2W floats (16 B at n = 8192) x min(n, 256) rows.
    // Measured (KS + starlet, mask 31 -> 63): 32 x 1024^2 0.822 -> 0.815 ms,
    // 16 x 2048^2 2.055 -> 2.020, 16 x 4096^2 11.32 -> 10.93, 1 x 8192^2
    // 3.41 -> 3.17; 64 x 512^2 no change (the plain KS 0.177 -> 0.182), so
    // from n = 1024 up.
    CUtensorMap mc;
    memset(&mc, 0, sizeof(mc));
    int tma_col = 0;
    if (P::NPASS > 1 && P::N >= 1024 && (tma_mode & 32)) {
        const uint64_t cdims[3] = {(uint64_t)2 * P::N, (uint64_t)P::N, (uint64_t)batch};
        const uint64_t cstrides[2] = {(uint64_t)P::N * 8, (uint64_t)P::N * P::N * 8};
        const uint32_t cbox[3] = {(uint32_t)(2 * P::W), (uint32_t)(P::N < 256 ? P::N : 256), 1};
        // stores the same way only at n = 8192 (KS + starlet: 1 x 8192^2 3.18 ->
        // 3.15 ms; 32 x 1024^2 0.813 -> 0.828, 16 x 4096^2 10.95 -> 11.00)
        tma_col = encode_map3d_f32(&mc, work, cdims, cstrides, cbox)
                      ? (1 | ((tma_mode & 64) && P::N >= 8192 ? 2 : 0))
                      : 0;
    }
    FM_LAUNCH(FM_K_FFT_ROWS_FWD, k_rows_fwd32<LOGN>, row_grid, RPC * P::TV, row_smem, s, in1, in2, in_bs, work,
              total_rows, tw, seed, r0, rotate ? 1 : 0, m1, m2, tma_in);
    FM_LAUNCH(FM_K_FFT_COLS_KS, k_cols_ks32<LOGN>, col_grid, col_threads, col_smem, s, work, tw, op, filt, mc,
              tma_col);
    if (op == FFT_OP_SPECTRUM) return FM_OK;
    const float scale = out_scale / ((float)P::N * (float)P::N);
    FM_LAUNCH(FM_K_FFT_ROWS_INV, k_rows_inv32<LOGN>, row_grid, RPC * P::TV, row_smem, s, work, out1, out2,
              total_rows, tw, scale, mw, tma_out);
    return FM_OK;
}

// n = 32 .. 8192 (power of two); other sizes return FM_EINVAL to the caller,
// which then uses the generic shared-memory Stockham kernels.
int launch_fft32(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int n,
                 int batch, int op, const float2 *filt, float out_scale, uint64_t seed, int r0, bool rotate,
                 const float2 *tw, cudaStream_t s)
{
#define FM_KS32(L) \
    ks32_impl<L>(in1, in2, in_bs, out1, out2, work, batch, op, filt, out_scale, seed, r0, rotate, tw, s)
    switch (n) {
    case 32: return FM_KS32(5);
    case 64: return FM_KS32(6);
    case 128: return FM_KS32(7);
    case 256: return FM_KS32(8);
    case 512: return FM_KS32(9);
    case 1024: return FM_KS32(10);
    case 2048: return FM_KS32(11);
    case 4096: return FM_KS32(12);
    case 8192: return FM_KS32(13);
    }
#undef FM_KS32
    return FM_EINVAL;
}

int fft_wait_error(bool clear) { return wait_error_flag(clear); }

int launch_ks32(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int n,
                int batch, bool forward, uint64_t seed, int r0, bool rotate, const float2 *tw, cudaStream_t s)
{
    return launch_fft32(in1, in2, in_bs, out1, out2, work, n, batch, forward ? FFT_OP_KS_FWD : FFT_OP_KS_INV,
                        nullptr, 1.f, seed, r0, rotate, tw, s);
}

}  // namespace fm
