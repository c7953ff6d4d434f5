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
//
// Real-output inverse (kappa_E alone, n >= 64).  kappa_E is real, so half of
// its spectrum carries it.  With Gamma1, Gamma2 the 2-D spectra of the real
// maps gamma1 and gamma2, the Hermitian part of conj(D) gamma_hat is
//   kappa_E_hat = Re(D) Gamma1 + Im(D) Gamma2,
// except on the Nyquist row and column (one index n/2, the other neither 0
// nor n/2), where the index convention k = -n/2 makes D(-k) = conj(D(k)) and
// the Hermitian part is conj(D) Gamma1.  Three passes, 36 instead of 44 bytes
// per pixel and three quarters of the butterflies:
//   rows_fwd32<SPLIT> : the complex row FFT Z of gamma1 + i gamma2 split into
//                       the half spectra Gamma1 = (Z(kx) + conj Z(-kx)) / 2,
//                       Gamma2 = (Z(kx) - conj Z(-kx)) / 2i, kx = 0 .. n/2,
//                       each row stored as n/2 slots (Gamma1(kx), Gamma2(kx)),
//                       16 bytes each, slot 0 packing the real pairs
//                       (X(0), X(n/2));
//   cols_ks32_e       : per strip of WS slots, column FFTs of the Gamma1 and
//                       Gamma2 slots, kappa_E_hat, column inverse FFT; writes
//                       the half spectrum H [n][n/2] into kappa's buffer;
//   rows_inv32_c2r    : in place in kappa's buffer, each row's length-n
//                       complex-to-real inverse as one length-n/2 complex
//                       inverse FFT (even samples real part, odd imaginary).
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
// barrier of the threads taking part: the whole CTA (NB = 0) or the first NB
// threads (named barrier 1; NB a multiple of 32)
template <int NB> __device__ __forceinline__ void part_sync()
{
    if constexpr (NB == 0)
        __syncthreads();
    else
        asm volatile("bar.sync 1, %0;" ::"n"(NB) : "memory");
}

template <int LOGN, int W, bool INV, int NB = 0>
__device__ __forceinline__ void fft_vec(float2 (&v)[32], float2 *sm, int c, int j, const float2 *__restrict__ tw)
{
    using P = Plan32<LOGN>;
    Dft<32, INV, float2>::run(v);  // pass 1: Ns = 1, no twiddles; outputs at 32 j + r
    if constexpr (P::NPASS > 1) {
        part_sync<NB>();  // the buffer may still be read by an earlier pass
#pragma unroll
        for (int r = 0; r < 32; ++r) sm[pad32((j * 32 + r) * W + c)] = v[r];
        part_sync<NB>();
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
            part_sync<NB>();
            const int o = (j - k) * 32 + k;
#pragma unroll
            for (int r = 0; r < 32; ++r) sm[pad32((o + r * NS) * W + c)] = v[r];
            part_sync<NB>();
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
// ROT: the noise maps' rotated shear (a separate instantiation, so that the
// plain transform carries none of the generator's code)
template <int LOGN, bool SPLIT, bool ROT>
__global__ void __launch_bounds__(256, 2) k_rows_fwd32(const float *__restrict__ in1, const float *__restrict__ in2,
                                                       long in_bs, float2 *__restrict__ work, long total_rows,
                                                       const float2 *__restrict__ tw, uint64_t seed, int r0,
                                                       const __grid_constant__ CUtensorMap m1,
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
                if constexpr (ROT) rotate_shear(a, cc, seed, r0 + b, y, x, P::N);
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
            if constexpr (ROT) rotate_shear(a, cc, seed, r0 + b, y, x, P::N);
            v[r] = make_float2(a, cc);
        }
    } else if (!staged) {
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    }
    fft_vec<LOGN, 1, false>(v, sm, 0, j, tw);
    if constexpr (SPLIT && P::NPASS > 1) {
        // Z through the exchange buffer so that Z(kx) and Z(n - kx) meet
        __syncthreads();  // the last pass's reads of the buffer
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) sm[pad32(j + m * P::TV + r * P::NSL)] = v[m * P::RL + r];
        __syncthreads();
        if (live) {
            // slot kx of the row: (Gamma1(kx), Gamma2(kx)) as one 16-byte element
            float4 *d = reinterpret_cast<float4 *>(work + row * P::N);
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const int kx = j + t * P::TV;
                const float2 a = sm[pad32(kx)];
                if (kx == 0) {
                    const float2 h = sm[pad32(P::N / 2)];
                    d[0] = make_float4(a.x, h.x, a.y, h.y);
                } else {
                    const float2 bm = sm[pad32(P::N - kx)];  // Z(n - kx); B = conj of it
                    d[kx] = make_float4(0.5f * (a.x + bm.x), 0.5f * (a.y - bm.y), 0.5f * (a.y + bm.y),
                                        -0.5f * (a.x - bm.x));
                }
            }
        }
        return;
    }
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
// WITH_B: kappa_B (the imaginary part) written too, a separate instantiation
// so that the kappa_E-only store loop has no per-element branch
template <int LOGN, bool WITH_B>
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
                if constexpr (WITH_B) out2[pos] = x.y * scale;
            }
    }
}

// With use_tma bit 0 (mw: the work buffer as floats {2n, n, batch}, box
// {2W, min(n, 256), 1}), the CTA's strip of W columns arrives by
// n / min(n, 256) bulk tensor copies into the exchange buffer, densely as
// [n][W] float2, instead of 32 strided loads per thread; with bit 1 the
// result leaves the same way (the spectrum-only mode stores per thread).
// KSINV: the inverse KS multiply fixed at compile time (the pipeline's
// instantiation, no per-element branch on op); else op chooses at run time.
template <int LOGN, bool KSINV>
__global__ void __launch_bounds__(512) k_cols_ks32(float2 *__restrict__ work, const float2 *__restrict__ tw,
                                                   int op_arg, const float2 *__restrict__ filt,
                                                   const __grid_constant__ CUtensorMap mw, int use_tma)
{
    pdl_entry();
    const int op = KSINV ? FFT_OP_KS_INV : op_arg;
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
                    // the pipeline's instantiation: the fast reciprocal (2 ulp, no
                    // division subroutine in the unrolled loop)
                    const float inv = KSINV ? __fdividef(1.f, (float)den) : 1.f / (float)den;
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

// ---- real-output inverse: column and row kernels ------------------------------
// Slots per column strip (WS; a strip is WS 16-byte (Gamma1, Gamma2) pairs
// per row, one bulk tensor copy box wide).  A CTA of 2 WS n/32 threads: its
// first half transforms the strip's Gamma1 columns, the second half the
// Gamma2 columns, at the same time; the second half hands its spectra over
// through shared memory and leaves, and the first half forms kappa_E_hat and
// runs the one inverse transform per slot on its own named barrier.  The two
// halves' exchange regions overlay the staged strip.  One-slot strips at
// 4096^2 (68 KB, two 256-thread CTAs per SM) measured slower than two-slot
// ones (one 512-thread CTA): 3.09 against 2.65 ms per 16 maps.
template <int LOGN> struct PlanE {
    static constexpr int N = 1 << LOGN;
    static constexpr int WS = N <= 256 ? 16 : (N == 512 ? 8 : (N == 1024 ? 4 : (N <= 4096 ? 2 : 1)));
    static constexpr int RSZ = (N * WS + N * WS / 32 + 1 + 15) & ~15;  // float2 per region, 128-byte multiple
    // the corner strip's dense exchange (2n elements): with WS >= 2 both
    // halves go to the Gamma1 region after its transform (the Gamma2 region
    // carries the other slots' hand-over); with WS = 1 the strip is the
    // corner slot alone and the second half writes its half in row order to
    // its own region
    static_assert(WS == 1 || RSZ >= 2 * N, "corner exchange");
    static constexpr int NH = WS * N / 32;  // threads of one half
    static constexpr int NT = 2 * NH;
    // CTAs per SM the register budget must allow: at most 128 registers a thread
    static constexpr int MINB = 65536 / (NT * 128) < 1 ? 1 : (65536 / (NT * 128) > 8 ? 8 : 65536 / (NT * 128));
};

// With use_tma (mw: the work buffer as floats {2n, n, batch}, box {4 WS,
// min(n, 256), 1}) the strip's slots arrive by bulk tensor copies, else by
// per-thread loads.
template <int LOGN>
__global__ void __launch_bounds__(PlanE<LOGN>::NT, PlanE<LOGN>::MINB)
    k_cols_ks32_e(const float2 *__restrict__ work, float2 *__restrict__ half, const float2 *__restrict__ tw,
                  const __grid_constant__ CUtensorMap mw, int use_tma)
{
    pdl_entry();
    using P = Plan32<LOGN>;
    using E = PlanE<LOGN>;
    constexpr int N = P::N, WS = E::WS, NH = E::NH;
    constexpr int STRIPS = N / 2 / WS;
    extern __shared__ __align__(16) unsigned char smem_col[];
    float2 *R1 = align128<float2>(smem_col);
    float2 *R2 = R1 + E::RSZ;
    float2 *U1 = R1, *U2 = WS == 1 ? R2 : R1 + N;  // corner exchange
    const long b = blockIdx.x / STRIPS;
    const int s0 = (blockIdx.x % STRIPS) * WS;
    const int tid = threadIdx.x, hf = tid / NH, t = tid % NH, c = t % WS, j = t / WS;
    float2 *R = hf ? R2 : R1;  // this half's strip and exchange region
    float2 v[32];
    if (use_tma) {
        __shared__ uint64_t bar;
        constexpr int BR = N < 256 ? N : 256;  // rows per copy
        if (tid == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (tid == 0) {
            // the strip, [n][WS] (Gamma1, Gamma2) pairs, over both regions
            mbar_expect_tx(&bar, (uint32_t)(2 * N * WS * sizeof(float2)));
            for (int k = 0; k < N / BR; ++k) tma_load_3d(R1 + 2 * k * BR * WS, &mw, 4 * s0, k * BR, (int)b, &bar);
        }
        if (!tma_wait_all(&bar, 0)) return;  // the copies never completed (flagged)
        // fft_vec's first barrier orders every thread's reads of the strip
        // before the exchange writes that overlay it
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = R1[((j + r * P::TV) * WS + c) * 2 + hf];
    } else {
        // rows of n/2 slots (Gamma1, Gamma2)
        const float2 *src = work + b * (long)N * N + 2 * (s0 + c) + hf;
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = src[(long)(j + r * P::TV) * N];
    }
    fft_vec<LOGN, WS, false>(v, R, c, j, tw);  // Gamma1_hat (first half), Gamma2_hat (second)
    __syncthreads();                           // the last passes' reads of R1 and R2 are done
    if (hf) {
        if (WS == 1 && s0 == 0) {  // the corner slot: in row order
#pragma unroll
            for (int m = 0; m < P::ML; ++m)
#pragma unroll
                for (int r = 0; r < P::RL; ++r) U2[j + m * P::TV + r * P::NSL] = v[m * P::RL + r];
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) R2[e * NH + t] = v[e];  // for the thread t of the first half
        }
    }
    __syncthreads();
    if (hf) return;  // the rest runs on named barrier 1 of the first NH threads
    const bool corner = s0 == 0 && c == 0;  // slot 0: kx = 0 and kx = n/2 packed
    if (!corner) {
        const int k1 = s0 + c;  // 1 .. n/2 - 1
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) {
                const int e = m * P::RL + r, yi = j + m * P::TV + r * P::NSL;
                const int k2 = yi < N / 2 ? yi : yi - N;
                const float inv = __fdividef(1.f, (float)(k1 * k1 + k2 * k2));  // 2 ulp
                const float dr = (float)(k1 * k1 - k2 * k2) * inv, di = (float)(2 * k1 * k2) * inv;
                const float2 a = v[e], g = R2[e * NH + t];
                v[e] = yi == N / 2 ? make_float2(dr * a.x + di * a.y, dr * a.y - di * a.x)  // conj(D) Gamma1
                                   : make_float2(dr * a.x + di * g.x, dr * a.y + di * g.y);
            }
    }
    if (s0 == 0) {  // CTA-uniform: the corner column pair needs ky and -ky together
        if (c == 0) {
#pragma unroll
            for (int m = 0; m < P::ML; ++m)
#pragma unroll
                for (int r = 0; r < P::RL; ++r) {
                    const int e = m * P::RL + r, yi = j + m * P::TV + r * P::NSL;
                    U1[yi] = v[e];
                    if (WS > 1) U2[yi] = R2[e * NH + t];
                }
        }
        part_sync<NH>();
        if (c == 0) {
#pragma unroll
            for (int m = 0; m < P::ML; ++m)
#pragma unroll
                for (int r = 0; r < P::RL; ++r) {
                    const int e = m * P::RL + r, yi = j + m * P::TV + r * P::NSL;
                    const int yp = (N - yi) & (N - 1);
                    const float2 p1 = U1[yi], q1 = U1[yp], p2 = U2[yi], q2 = U2[yp];
                    // A = Gamma(ky, 0) = (P + conj P(-ky)) / 2, B = Gamma(ky, n/2) = (P - conj P(-ky)) / 2i
                    const float2 a1 = make_float2(0.5f * (p1.x + q1.x), 0.5f * (p1.y - q1.y));
                    const float2 b1 = make_float2(0.5f * (p1.y + q1.y), -0.5f * (p1.x - q1.x));
                    const float2 b2 = make_float2(0.5f * (p2.y + q2.y), -0.5f * (p2.x - q2.x));
                    const int k2 = yi < N / 2 ? yi : yi - N;
                    // kx = 0: D = -1 (0 at k = 0)
                    const float2 kz = yi == 0 ? make_float2(0.f, 0.f) : make_float2(-a1.x, -a1.y);
                    // kx = n/2 (k1 = -n/2)
                    const float inv = __fdividef(1.f, (float)(N / 2 * (N / 2) + k2 * k2));
                    const float dr = (float)(N / 2 * (N / 2) - k2 * k2) * inv, di = (float)(-N * k2) * inv;
                    const float2 kh = (yi == 0 || yi == N / 2)
                                          ? make_float2(dr * b1.x + di * b2.x, dr * b1.y + di * b2.y)
                                          : make_float2(dr * b1.x + di * b1.y, dr * b1.y - di * b1.x);
                    v[e] = make_float2(kz.x - kh.y, kz.y + kh.x);  // packed kz + i kh
                }
        }
    }
    if constexpr (!(P::RL == 32 || P::NPASS == 1)) {
        // bring the spectrum back to the inverse's input order x[j + r TV]
        part_sync<NH>();
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) R1[pad32((j + m * P::TV + r * P::NSL) * WS + c)] = v[m * P::RL + r];
        part_sync<NH>();
#pragma unroll
        for (int r = 0; r < 32; ++r) v[r] = R1[pad32((j + r * P::TV) * WS + c)];
    }
    fft_vec<LOGN, WS, true, NH>(v, R1, c, j, tw);
    float2 *dst = half + b * (long)N * (N / 2) + s0 + c;
#pragma unroll
    for (int m = 0; m < P::ML; ++m)
#pragma unroll
        for (int r = 0; r < P::RL; ++r) dst[(long)(j + m * P::TV + r * P::NSL) * (N / 2)] = v[m * P::RL + r];
}

// In place: row y of kap holds the half spectrum H(y, 0 .. n/2) as n/2 float2
// (slot 0 = the real pair H(0), H(n/2)) and receives kappa_E's row.  With
// use_tma (n >= 128; mk: kap as floats {d0, n/d0, rows}) the CTA's rows are
// staged by one bulk tensor copy.  Every read of the row precedes the
// transform's first barrier, and every write follows it.
template <int LOGN>
__global__ void __launch_bounds__(256, 2) k_rows_inv32_c2r(float *kap, long total_rows, const float2 *__restrict__ tw,
                                                           const float2 *__restrict__ tw2, float scale,
                                                           const __grid_constant__ CUtensorMap mk, int use_tma)
{
    pdl_entry();
    using P = Plan32<LOGN - 1>;  // the length n/2 complex transform
    constexpr int N2 = P::N;
    constexpr int RPC = P::TV >= kRowThreads ? 1 : kRowThreads / P::TV;
    extern __shared__ __align__(16) float2 sm32[];
    __shared__ uint64_t bar;
    float2 *smb = align128<float2>(sm32);
    const int vr = threadIdx.x / P::TV, j = threadIdx.x % P::TV;
    const long row = (long)blockIdx.x * RPC + vr;
    float2 *sm = smb + vr * (N2 + N2 / 32);
    const bool live = row < total_rows;
    const float2 *h = reinterpret_cast<const float2 *>(kap) + row * N2;
    if constexpr (P::NPASS > 1) {
        if (use_tma) {
            if (threadIdx.x == 0) mbar_init(&bar, 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                mbar_expect_tx(&bar, (uint32_t)(RPC * N2 * sizeof(float2)));
                tma_load_3d(smb, &mk, 0, 0, (int)((long)blockIdx.x * RPC), &bar);
            }
            if (!tma_wait_all(&bar, 0)) return;  // the copy never completed (flagged)
            h = smb + vr * N2;
        }
    }
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const int k = j + r * P::TV;
        float2 z = make_float2(0.f, 0.f);
        if (live) {
            const float2 hk = h[k];
            if (k == 0) {
                z = make_float2(hk.x + hk.y, hk.x - hk.y);
            } else {
                const float2 hm = h[N2 - k];
                const float2 ee = make_float2(hk.x + hm.x, hk.y - hm.y);  // H(k) + conj H(n/2 - k)
                float2 od = make_float2(hk.x - hm.x, hk.y + hm.y);        // H(k) - conj H(n/2 - k)
                od = cmul(od, twid<true>(tw, k));                         // times exp(+2 pi i k / n)
                z = make_float2(ee.x - od.y, ee.y + od.x);
            }
        }
        v[r] = z;
    }
    fft_vec<LOGN - 1, 1, true>(v, sm, 0, j, tw2);
    if (live) {
        float2 *out = reinterpret_cast<float2 *>(kap) + row * N2;  // (kappa(2m), kappa(2m + 1))
#pragma unroll
        for (int m = 0; m < P::ML; ++m)
#pragma unroll
            for (int r = 0; r < P::RL; ++r) {
                const float2 z = v[m * P::RL + r];
                out[j + m * P::TV + r * P::NSL] = make_float2(z.x * scale, z.y * scale);
            }
    }
}

std::atomic<int> g_ks_real{-1};

// Measured on GB300 (ms, complex / real-output inverse), KS + starlet in
// the batched chunks (two streams, one pass per large scale, packed adds and
// the fast reciprocal in the KS multiply): 32 x 1024^2 0.599 / 0.574,
// 16 x 2048^2 1.494 / 1.466, 64 x 512^2 0.303 / 0.291, 16 x 4096^2 8.03 /
// 7.53, 1 x 8192^2 2.47 / 2.41; the inverse alone 32 x 1024^2 0.296 / 0.266,
// 16 x 4096^2 3.98 / 3.49.  (Before the fast reciprocal the real column
// pass, with its per-element divisions, lost inside the 512^2-2048^2
// pipelines: 32 x 1024^2 0.652 / 0.658.)  Below 512^2 the complex inverse
// stays ahead: 128 x 256^2 J = 6 0.204 / 0.206, 256 x 128^2 J = 5 0.138 /
// 0.145 (the inverse alone 0.046 / 0.054).
bool ks_real_for(int n, bool batched)
{
    const int mode = g_ks_real.load(std::memory_order_relaxed);
    (void)batched;
    if (mode >= 0) return mode == 1 && n >= 64;
    return n >= 512;
}

// ---------------------------------------------------------------------------
// Real-output inverse KS (kappa_E only): the split row FFT into `work`, the
// column pass into kappa's buffer `out1` (the half spectrum, [rows][n/2]
// float2, 16-byte aligned), the complex-to-real row pass in place there.
template <int LOGN>
static int ks32_real_impl(const float *in1, const float *in2, long in_bs, float *out1, float2 *work, int batch,
                          float out_scale, uint64_t seed, int r0, bool rotate, const float2 *tw, const float2 *tw2,
                          cudaStream_t s)
{
    using P = Plan32<LOGN>;
    using P2 = Plan32<LOGN - 1>;
    using E = PlanE<LOGN>;
    constexpr int RPC = P::TV >= kRowThreads ? 1 : kRowThreads / P::TV;
    constexpr int RPC2 = P2::TV >= kRowThreads ? 1 : kRowThreads / P2::TV;
    const long total_rows = (long)batch * P::N;
    const unsigned row_grid = (unsigned)((total_rows + RPC - 1) / RPC);
    const unsigned row2_grid = (unsigned)((total_rows + RPC2 - 1) / RPC2);
    const size_t row_smem = (size_t)RPC * (P::N + P::N / 32) * sizeof(float2) + 128;
    const size_t row2_smem = P2::NPASS > 1 ? (size_t)RPC2 * (P2::N + P2::N / 32) * sizeof(float2) + 128 : 0;
    const size_t col_smem = (size_t)(2 * E::RSZ) * sizeof(float2) + 128;
    const int col_threads = E::NT;
    const unsigned col_grid = (unsigned)((long)batch * (P::N / 2 / E::WS));
    auto krf = rotate ? k_rows_fwd32<LOGN, true, true> : k_rows_fwd32<LOGN, true, false>;
    FM_CUDA_TRY(fm::smem_attr((const void *)krf, row_smem));
    FM_CUDA_TRY(fm::smem_attr((const void *)k_cols_ks32_e<LOGN>, col_smem));
    if (row2_smem) FM_CUDA_TRY(fm::smem_attr((const void *)k_rows_inv32_c2r<LOGN>, row2_smem));
    CUtensorMap m1, m2, mc, mk;
    memset(&m1, 0, sizeof(m1));
    memset(&m2, 0, sizeof(m2));
    memset(&mc, 0, sizeof(mc));
    memset(&mk, 0, sizeof(mk));
    int tma_in = 0, tma_col = 0, tma_out = 0;
    const int tma_mode = g_use_tma.load(std::memory_order_relaxed);
    {
        const long nn = (long)P::N * P::N;
        const uint32_t d0 = P::N < 256 ? P::N : 256;
        const uint64_t rows = in_bs == 0 ? (uint64_t)P::N : (uint64_t)total_rows;
        const uint64_t dims[3] = {d0, (uint64_t)(P::N / d0), rows};
        const uint64_t strides[2] = {(uint64_t)d0 * 4, (uint64_t)P::N * 4};
        const uint32_t box[3] = {d0, (uint32_t)(P::N / d0), (uint32_t)RPC};
        tma_in = (tma_mode & 2) && (in_bs == nn || (in_bs == 0 && RPC <= P::N)) &&
                 encode_map3d_f32(&m1, in1, dims, strides, box) && (!in2 || encode_map3d_f32(&m2, in2, dims, strides, box));
        // kappa's buffer as rows of n floats (= n/2 float2 of half spectrum)
        if (P2::NPASS > 1 && (tma_mode & 4)) {
            const uint64_t kdims[3] = {d0, (uint64_t)(P::N / d0), (uint64_t)total_rows};
            const uint32_t kbox[3] = {d0, (uint32_t)(P::N / d0), (uint32_t)RPC2};
            tma_out = encode_map3d_f32(&mk, out1, kdims, strides, kbox);
        }
    }
    if (P::N >= 1024 && (tma_mode & 32)) {
        const uint64_t cdims[3] = {(uint64_t)2 * P::N, (uint64_t)P::N, (uint64_t)batch};
        const uint64_t cstrides[2] = {(uint64_t)P::N * 8, (uint64_t)P::N * P::N * 8};
        const uint32_t cbox[3] = {(uint32_t)(4 * E::WS), (uint32_t)(P::N < 256 ? P::N : 256), 1};
        tma_col = encode_map3d_f32(&mc, work, cdims, cstrides, cbox) ? 1 : 0;
    }
    FM_LAUNCH(FM_K_FFT_ROWS_FWD, krf, row_grid, RPC * P::TV, row_smem, s, in1, in2, in_bs, work, total_rows, tw, seed,
              r0, m1, m2, tma_in);
    FM_LAUNCH(FM_K_FFT_COLS_KS, k_cols_ks32_e<LOGN>, col_grid, col_threads, col_smem, s, (const float2 *)work,
              reinterpret_cast<float2 *>(out1), tw, mc, tma_col);
    const float scale = out_scale / ((float)P::N * (float)P::N);
    FM_LAUNCH(FM_K_FFT_ROWS_INV, k_rows_inv32_c2r<LOGN>, row2_grid, RPC2 * P2::TV, row2_smem, s, out1, total_rows, tw,
              tw2, scale, mk, tma_out);
    return FM_OK;
}

template <int LOGN>
static int ks32_impl(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int batch,
                     int op, const float2 *filt, float out_scale, uint64_t seed, int r0, bool rotate,
                     const float2 *tw, const float2 *tw2, cudaStream_t s)
{
    if constexpr (LOGN >= 6) {
        if (op == FFT_OP_KS_INV && !out2 && tw2 && (reinterpret_cast<uintptr_t>(out1) & 15) == 0)
            return ks32_real_impl<LOGN>(in1, in2, in_bs, out1, work, batch, out_scale, seed, r0, rotate, tw, tw2, s);
    }
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
    auto krf = rotate ? k_rows_fwd32<LOGN, false, true> : k_rows_fwd32<LOGN, false, false>;
    FM_CUDA_TRY(fm::smem_attr((const void *)krf, row_smem));
    auto kri = out2 ? k_rows_inv32<LOGN, true> : k_rows_inv32<LOGN, false>;
    auto kcl = op == FFT_OP_KS_INV ? k_cols_ks32<LOGN, true> : k_cols_ks32<LOGN, false>;
    FM_CUDA_TRY(fm::smem_attr((const void *)kri, row_smem));
    FM_CUDA_TRY(fm::smem_attr((const void *)kcl, col_smem));
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
    FM_LAUNCH(FM_K_FFT_ROWS_FWD, krf, row_grid, RPC * P::TV, row_smem, s, in1, in2, in_bs, work, total_rows, tw, seed,
              r0, m1, m2, tma_in);
    FM_LAUNCH(FM_K_FFT_COLS_KS, kcl, col_grid, col_threads, col_smem, s, work, tw, op, filt, mc, tma_col);
    if (op == FFT_OP_SPECTRUM) return FM_OK;
    const float scale = out_scale / ((float)P::N * (float)P::N);
    FM_LAUNCH(FM_K_FFT_ROWS_INV, kri, row_grid, RPC * P::TV, row_smem, s, work, out1, out2, total_rows, tw, scale,
              mw, tma_out);
    return FM_OK;
}

// n = 32 .. 8192 (power of two); other sizes return FM_EINVAL to the caller,
// which then uses the generic shared-memory Stockham kernels.
int launch_fft32(const float *in1, const float *in2, long in_bs, float *out1, float *out2, float2 *work, int n,
                 int batch, int op, const float2 *filt, float out_scale, uint64_t seed, int r0, bool rotate,
                 const float2 *tw, const float2 *tw2, cudaStream_t s)
{
#define FM_KS32(L) \
    ks32_impl<L>(in1, in2, in_bs, out1, out2, work, batch, op, filt, out_scale, seed, r0, rotate, tw, tw2, s)
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
                int batch, bool forward, uint64_t seed, int r0, bool rotate, const float2 *tw, const float2 *tw2,
                cudaStream_t s)
{
    return launch_fft32(in1, in2, in_bs, out1, out2, work, n, batch, forward ? FFT_OP_KS_FWD : FFT_OP_KS_INV,
                        nullptr, 1.f, seed, r0, rotate, tw, tw2, s);
}

}  // namespace fm
