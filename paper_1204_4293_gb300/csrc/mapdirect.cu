// mapdirect.cu -- brute-force aperture mass from tangential shear,
// eq. shearmap (Sec. 2.1) evaluated as in Sec. 5.1: the comparison path whose
// O(n^2 R^2) cost the starlet removes.
//
// M(x) = sum_{0 < |d| <= R} Q(|d|) gamma_t(x + d; x),
// gamma_t = -(gamma1 cos 2 phi_d + gamma2 sin 2 phi_d), so with per-offset
// weights A(d) = -Q cos 2 phi = -Q (dx^2 - dy^2) / |d|^2 and
// B(d) = -Q sin 2 phi = -Q 2 dx dy / |d|^2 (built on the host in FP64) the map
// is the 2-D correlation M = A * gamma1 + B * gamma2, zero outside the field.
//
// Kernel layout: a CTA owns TY = NW*RY output rows x TX = 32*CX columns; warp
// w owns RY rows, lane l owns CX adjacent columns.  The CTA walks the input
// rows iy covering its rows +- R; each input row (both components, halo R)
// is staged once in shared memory and serves every output row within R of
// it: output row y uses it with the weight row dy = iy - y.  Within a warp
// all lanes share the output rows, so the dy tests and dx loop bounds are
// warp-uniform, and weights are warp-wide broadcast loads.  The staged row
// is stored with one pad slot per 8 so that the lanes' 8-column windows hit
// distinct banks.  FP32 cores (FFMA), no tensor cores: not a contraction the
// tensor cores can take at this precision.
//
// Missing data (Sec. 4.3, Sec. 4.5): with pixel weights w >= 0 (0 = masked)
// the same pass also forms D(x) = sum w(x+d) over the in-field offsets
// 0 < |d| <= R (a third staged component and a 0/1 disc table), stages
// w gamma1, w gamma2 instead of the shear, and writes
// M = N_R S / D (0 where D <= 0) and optionally coverage = D / N_R, N_R the
// aperture's pixel count.
#include <math.h>

#include <atomic>
#include <vector>

#include "common.cuh"

namespace fm {

// ---- filters (Sec. 4), FP64 on the host --------------------------------------
static double cube(double v) { return v * v * v; }

// starlet Q(eta) printed in Sec. 4.2; the direct sum never evaluates eta = 0.
static double q_starlet(double e)
{
    const double e2 = e * e;
    double s = -279.0 * e2 * cube(fabs(e));
    s += 8.0 * (1.0 + 6.0 * e + 24.0 * e2) * cube(fabs(0.5 - e));
    s += 8.0 * (1.0 - 6.0 * e + 24.0 * e2) * cube(fabs(0.5 + e));
    s -= 9.0 * (1.0 + 3.0 * e + 6.0 * e2) * cube(fabs(1.0 - e));
    s -= 9.0 * (1.0 - 3.0 * e + 6.0 * e2) * cube(fabs(1.0 + e));
    s += (1.0 + 1.5 * e + 1.5 * e2) * cube(fabs(2.0 - e));
    s += (1.0 - 1.5 * e + 1.5 * e2) * cube(fabs(2.0 + e));
    return s / (45.0 * e2);
}

static double q_of(int filter, double v, double theta, int ell)
{
    const double t2 = theta * theta;
    switch (filter) {
    case FM_FILTER_STARLET: return q_starlet(v / theta) / t2;  // U, Q scale as 1/theta^2
    case FM_FILTER_S98: {  // eq. sch
        if (v > theta) return 0.0;
        const double x2 = v * v / t2;
        return (1.0 + ell) * (2.0 + ell) / (M_PI * t2) * x2 * pow(1.0 - x2, (double)ell);
    }
    case FM_FILTER_JBJ04:
    case FM_FILTER_VW98: {  // eq. mexhat with A = 1
        const double b = filter == FM_FILTER_JBJ04 ? 0.5 : 4.0;
        const double x = b * v * v / t2;
        return x * exp(-x) / t2;
    }
    }
    return 0.0;
}

static double default_cut(int filter) { return filter == FM_FILTER_STARLET ? 2.0 : filter == FM_FILTER_S98 ? 1.0 : 5.0; }

// ---- kernel -------------------------------------------------------------------
__device__ __forceinline__ int padc(int c) { return c + (c >> 3); }
__device__ __forceinline__ uint32_t smem_u32_md(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <typename T, int CX, int RY, int NW, bool MASK>
__global__ void __launch_bounds__(NW * 32) k_map_direct(const T *__restrict__ g1, const T *__restrict__ g2,
                                                        const T *__restrict__ wgt, long w_bs,
                                                        const cplx_t<T> *__restrict__ taps,
                                                        const T *__restrict__ disc, int tw,
                                                        const int *__restrict__ dxmax, T *__restrict__ out,
                                                        T *__restrict__ cov, int n, int Ri, T n_r)
{
    pdl_entry();
    using V = cplx_t<T>;
    constexpr int TX = 32 * CX, TY = NW * RY;
    constexpr int NC = MASK ? 3 : 2;  // staged components
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int width = TX + 2 * Ri + 8;
    const int pw = padc(width) + 1;
    T *s1 = reinterpret_cast<T *>(smem_raw);  // [2 buffers][NC comps][pw]
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const long nn = (long)n * n;
    const long b = blockIdx.z;
    g1 += b * nn;
    g2 += b * nn;
    out += b * nn;
    if (MASK) {
        wgt += b * w_bs;
        if (cov) cov += b * nn;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int yw = y0 + warp * RY;
    const int lc = lane * CX;

    T acc[RY][CX], accw[MASK ? RY : 1][CX];
#pragma unroll
    for (int k = 0; k < RY; ++k)
#pragma unroll
        for (int o = 0; o < CX; ++o) {
            acc[k][o] = (T)0;
            if (MASK) accw[k][o] = (T)0;
        }

    const int iy_lo = y0 - Ri, iy_hi = y0 + TY - 1 + Ri;
    for (int iy = iy_lo; iy <= iy_hi; ++iy) {
        T *buf = s1 + ((iy - iy_lo) & 1) * NC * pw;
        const bool rin = iy >= 0 && iy < n;
        for (int c = threadIdx.x; c < width; c += blockDim.x) {
            const int gx = x0 - Ri + c;
            T a = (T)0, bb = (T)0, ww = (T)0;
            if (rin && gx >= 0 && gx < n) {
                a = g1[(long)iy * n + gx];
                bb = g2[(long)iy * n + gx];
                if (MASK) {
                    ww = wgt[(long)iy * n + gx];
                    a *= ww;
                    bb *= ww;
                }
            }
            buf[padc(c)] = a;
            buf[pw + padc(c)] = bb;
            if (MASK) buf[2 * pw + padc(c)] = ww;
        }
        __syncthreads();

        int dy[RY];
        bool act[RY];
        int dxm = -1;
#pragma unroll
        for (int k = 0; k < RY; ++k) {
            dy[k] = iy - (yw + k);
            act[k] = dy[k] >= -Ri && dy[k] <= Ri && (yw + k) < n;
            if (act[k]) {
                const int m = __ldg(dxmax + dy[k] + Ri);
                dxm = m > dxm ? m : dxm;
            }
        }
        if (dxm >= 0) {
            // two-level sum: this input row's taps first, then into the total
            T part[RY][CX], partw[MASK ? RY : 1][CX];
#pragma unroll
            for (int k = 0; k < RY; ++k)
#pragma unroll
                for (int o = 0; o < CX; ++o) {
                    part[k][o] = (T)0;
                    if (MASK) partw[k][o] = (T)0;
                }
            for (int dx0 = -dxm; dx0 <= dxm; dx0 += 8) {
                T w1[CX + 7], w2[CX + 7], w3[MASK ? CX + 7 : 1];
                const int base = lc + dx0 + Ri;
#pragma unroll
                for (int q = 0; q < CX + 7; ++q) {
                    w1[q] = buf[padc(base + q)];
                    w2[q] = buf[pw + padc(base + q)];
                    if (MASK) w3[q] = buf[2 * pw + padc(base + q)];
                }
#pragma unroll
                for (int k = 0; k < RY; ++k) {
                    if (!act[k]) continue;
                    const long toff = (long)(dy[k] + Ri) * tw + (dx0 + Ri);
                    const V *trow = taps + toff;
#pragma unroll
                    for (int t = 0; t < 8; ++t) {
                        const V ab = __ldg(trow + t);
#pragma unroll
                        for (int o = 0; o < CX; ++o) {
                            part[k][o] = fma(ab.x, w1[o + t], part[k][o]);
                            part[k][o] = fma(ab.y, w2[o + t], part[k][o]);
                        }
                        if (MASK) {
                            const T in_disc = __ldg(disc + toff + t);
#pragma unroll
                            for (int o = 0; o < CX; ++o) partw[k][o] = fma(in_disc, w3[o + t], partw[k][o]);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < RY; ++k)
#pragma unroll
                for (int o = 0; o < CX; ++o) {
                    acc[k][o] += part[k][o];
                    if (MASK) accw[k][o] += partw[k][o];
                }
        }
    }
#pragma unroll
    for (int k = 0; k < RY; ++k) {
        const int y = yw + k;
        if (y >= n) continue;
#pragma unroll
        for (int o = 0; o < CX; ++o) {
            const int x = x0 + lc + o;
            if (x >= n) continue;
            if (MASK) {
                const T d = accw[k][o];
                out[(long)y * n + x] = d > (T)0 ? n_r * acc[k][o] / d : (T)0;
                if (cov) cov[(long)y * n + x] = d / n_r;
            } else {
                out[(long)y * n + x] = acc[k][o];
            }
        }
    }
}

// ---- fp32 form without weights ------------------------------------------------
// The same walk over input rows with two changes: the next input row arrives
// by asynchronous 4-byte copies (cp.async, zero-filled outside the field)
// into the other buffer while the CTA works on the current one, so the
// global-memory latency of the staging is hidden; and the two components are
// staged interleaved, (gamma1, gamma2) per column, so that one packed
// two-lane FMA (fma.rn.f32x2) per tap adds A gamma1 into lane x and
// B gamma2 into lane y of a partial sum; the lanes are added when the input
// row is done.  Half the FMA instructions of the scalar form.
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32_md(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

//
// With P > 1 the input rows a tile needs (TY + 2R of them) are split into P
// consecutive parts, one CTA each (blockIdx.z = b P + p), so that a single
// map with a large radius still gives the GPU several waves of CTAs; part p
// writes its sums to part_out[p][b] and k_sum_parts adds the parts in order
// (the same order whatever the batch, so a map's result does not depend on
// the maps beside it).
template <int CX, int RY, int NW>
__global__ void __launch_bounds__(NW * 32) k_map_direct_f2(const float *__restrict__ g1, const float *__restrict__ g2,
                                                           const float2 *__restrict__ taps, int tw,
                                                           const int *__restrict__ dxmax, float *__restrict__ out,
                                                           int n, int Ri, int P, int batch)
{
    pdl_entry();
    constexpr int TX = 32 * CX, TY = NW * RY;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int width = TX + 2 * Ri + 8;
    const int pw = padc(width) + 1;
    float2 *s2 = reinterpret_cast<float2 *>(smem_raw);  // [2 buffers][pw] of (gamma1, gamma2)
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const long nn = (long)n * n;
    const long b = blockIdx.z / P;
    const int p = blockIdx.z % P;
    g1 += b * nn;
    g2 += b * nn;
    out += ((long)p * batch + b) * nn;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int yw = y0 + warp * RY;
    const int lc = lane * CX;
    const int rows = TY + 2 * Ri, chunk = (rows + P - 1) / P;
    const int iy_lo = y0 - Ri + p * chunk;
    const int iy_end = y0 + TY - 1 + Ri;
    const int iy_hi = iy_lo + chunk - 1 < iy_end ? iy_lo + chunk - 1 : iy_end;

    auto stage = [&](int iy) {  // this thread's copies of input row iy into its buffer
        float *buf = reinterpret_cast<float *>(s2 + ((iy - iy_lo) & 1) * pw);
        const bool rin = iy >= 0 && iy < n;
        for (int c = threadIdx.x; c < width; c += NW * 32) {
            const int gx = x0 - Ri + c;
            const bool in = rin && gx >= 0 && gx < n;
            const long off = in ? (long)iy * n + gx : 0;
            cp_async4(buf + 2 * padc(c), g1 + off, in ? 4 : 0);
            cp_async4(buf + 2 * padc(c) + 1, g2 + off, in ? 4 : 0);
        }
        cp_async_commit();
    };

    float acc[RY][CX];
#pragma unroll
    for (int k = 0; k < RY; ++k)
#pragma unroll
        for (int o = 0; o < CX; ++o) acc[k][o] = 0.f;

    if (iy_lo <= iy_hi) stage(iy_lo);
    for (int iy = iy_lo; iy <= iy_hi; ++iy) {
        cp_async_wait_all();  // this thread's copies of row iy have landed
        __syncthreads();      // everyone's have; the other buffer is no longer read
        if (iy < iy_hi) stage(iy + 1);
        const float2 *buf = s2 + ((iy - iy_lo) & 1) * pw;

        int dy[RY];
        bool act[RY];
        int dxm = -1;
#pragma unroll
        for (int k = 0; k < RY; ++k) {
            dy[k] = iy - (yw + k);
            act[k] = dy[k] >= -Ri && dy[k] <= Ri && (yw + k) < n;
            if (act[k]) {
                const int m = __ldg(dxmax + dy[k] + Ri);
                dxm = m > dxm ? m : dxm;
            }
        }
        if (dxm < 0) continue;
        float2 part[RY][CX];
#pragma unroll
        for (int k = 0; k < RY; ++k)
#pragma unroll
            for (int o = 0; o < CX; ++o) part[k][o] = make_float2(0.f, 0.f);
        for (int dx0 = -dxm; dx0 <= dxm; dx0 += 8) {
            float2 w[CX + 7];
            const int base = lc + dx0 + Ri;
#pragma unroll
            for (int q = 0; q < CX + 7; ++q) w[q] = buf[padc(base + q)];
#pragma unroll
            for (int k = 0; k < RY; ++k) {
                if (!act[k]) continue;
                const float2 *trow = taps + (long)(dy[k] + Ri) * tw + (dx0 + Ri);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float2 ab = __ldg(trow + t);
#pragma unroll
                    for (int o = 0; o < CX; ++o) part[k][o] = __ffma2_rn(ab, w[o + t], part[k][o]);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < RY; ++k)
#pragma unroll
            for (int o = 0; o < CX; ++o) acc[k][o] += part[k][o].x + part[k][o].y;
    }
#pragma unroll
    for (int k = 0; k < RY; ++k) {
        const int y = yw + k;
        if (y >= n) continue;
#pragma unroll
        for (int o = 0; o < CX; ++o) {
            const int x = x0 + lc + o;
            if (x < n) out[(long)y * n + x] = acc[k][o];
        }
    }
}

// out[i] = sum over p of part[p][i], p in order (float4 where the size allows)
__global__ void k_sum_parts(const float *__restrict__ part, float *__restrict__ out, long total, int P)
{
    pdl_entry();
    const long i4 = ((long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    // float4 access needs `out` 16-byte aligned and every part's start too
    // (`part` is 256-byte aligned scratch, part p starts p * total floats on)
    const bool vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0 && (total & 3) == 0;
    if (vec && i4 + 3 < total) {
        float4 a = *reinterpret_cast<const float4 *>(part + i4);
        for (int p = 1; p < P; ++p) {
            const float4 v = *reinterpret_cast<const float4 *>(part + (long)p * total + i4);
            a.x += v.x;
            a.y += v.y;
            a.z += v.z;
            a.w += v.w;
        }
        *reinterpret_cast<float4 *>(out + i4) = a;
    } else {
        for (long i = i4; i < total && i < i4 + 4; ++i) {
            float a = part[i];
            for (int p = 1; p < P; ++p) a += part[(long)p * total + i];
            out[i] = a;
        }
    }
}

// kernel form of the unmasked fp32 direct map: 0 = scalar FMAs (k_map_direct),
// 1 .. 4 = k_map_direct_f2 shapes (fm_tune FM_TUNE_DIRECT), -1 = by radius:
// measured on one 1024^2 map (ms, forms 1 / 2 / 3 / 4), S98 theta = 8:
// 0.084 / 0.062 / 0.068 / 0.070, theta = 32: 0.531 / 0.435 / 0.484 / 0.496,
// theta = 64: 1.53 / 1.48 / 1.46 / 1.52, starlet Q theta = 64 (R = 128):
// 5.01 / 5.08 / 4.99 / 5.13; the scalar form 0.091, 0.597, 1.98, 7.01
std::atomic<int> g_direct_form{-1};
static int direct_form(int Ri)
{
    const int f = g_direct_form.load();
    return f >= 0 ? f : (Ri < 48 ? 2 : 3);
}

// parts of the input-row walk: about 16 rows each, at most 16 (a function of
// the tile height and radius only, so results never depend on the batch).
// Measured on one 1024^2 map (ms), parts of ~32 rows (at most 8) / ~16 (16) /
// ~64 (4): S98 theta = 64 1.41 / 1.33 / 1.65, starlet Q theta = 64 4.83 /
// 4.71 / 5.19, JBJ04 theta = 16 (cut 5 theta) 2.01 / 1.92 / 2.46.
static int direct_parts(int TY, int Ri)
{
    const int P = (TY + 2 * Ri) / 16;
    return P < 1 ? 1 : (P > 16 ? 16 : P);
}
// maps per launch pair when the parts go through scratch: at most 256 MiB of
// partial sums (the order of the sums is per map, so the slicing of a batch
// does not change any result)
static int direct_slice(int P, int n, int batch)
{
    if (P <= 1) return batch;
    const long per_map = (long)P * n * n * (long)sizeof(float);
    long m = (256L << 20) / per_map;
    m = m < 1 ? 1 : m;
    return m < batch ? (int)m : batch;
}

template <int RY, int NW>
static int launch_direct_f2(const float *g1, const float *g2, const float2 *dtaps, int tw, const int *ddx, float *map,
                            float *parts, int n, int batch, int Ri, cudaStream_t s)
{
    constexpr int CX = 8, TX = 32 * CX, TY = NW * RY;
    const int width = TX + 2 * Ri + 8;
    const int pw = width + (width >> 3) + 1;
    const size_t smem = 2ull * pw * sizeof(float2);
    const int P = direct_parts(TY, Ri);
    const int slice = direct_slice(P, n, batch);
    auto k = k_map_direct_f2<CX, RY, NW>;
    FM_CUDA_TRY(fm::smem_attr((const void *)k, smem));
    const long nn = (long)n * n;
    for (int b0 = 0; b0 < batch; b0 += slice) {
        const int bs = batch - b0 < slice ? batch - b0 : slice;
        dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, bs * P);
        FM_LAUNCH(FM_K_MAP_DIRECT, k, grid, NW * 32, smem, s, g1 + b0 * nn, g2 + b0 * nn, dtaps, tw, ddx,
                  P > 1 ? parts : map + b0 * nn, n, Ri, P, bs);
        if (P > 1) {
            const long total = (long)bs * nn;
            const unsigned g = (unsigned)((total / 4 + 255) / 256 + 1);
            FM_LAUNCH(FM_K_MAP_DIRECT, k_sum_parts, g, 256, 0, s, (const float *)parts, map + b0 * nn, total, P);
        }
    }
    return FM_OK;
}

static size_t direct_parts_bytes(int form, int n, int batch, int Ri)
{
    const int TY = form == 2 ? 8 : form == 3 ? 8 : 16;
    const int P = direct_parts(TY, Ri);
    return P > 1 ? (size_t)P * direct_slice(P, n, batch) * n * n * sizeof(float) : 0;
}

template <typename T>
static int map_direct_impl(const T *g1, const T *g2, const T *wgt, long w_bs, T *map, T *cov, int n, int batch,
                           int filter, double theta, int ell, double cut, cudaStream_t s)
{
    using V = cplx_t<T>;
    const bool mask = wgt != nullptr;
    const double R = (cut > 0 ? cut : default_cut(filter)) * theta;
    const int Ri = (int)floor(R);
    const int tw = 2 * Ri + 8;  // weight row: dx = -Ri .. Ri + 7 (zeros beyond R)
    const size_t ntap = (size_t)(2 * Ri + 1) * tw;
    std::vector<V> htaps(ntap);
    std::vector<T> hdisc(mask ? ntap : 0);
    std::vector<int> hdx(2 * Ri + 1);
    long n_r = 0;  // lattice offsets 0 < |d| <= R
    for (int dy = -Ri; dy <= Ri; ++dy) {
        const double m2 = R * R - (double)dy * dy;
        hdx[dy + Ri] = m2 >= 0 ? (int)floor(sqrt(m2)) : -1;
        for (int c = 0; c < tw; ++c) {
            const int dx = c - Ri;
            const double r2 = (double)dx * dx + (double)dy * dy;
            V ab;
            ab.x = ab.y = 0;
            const bool in = r2 > 0 && r2 <= R * R;
            if (in) {
                const double q = q_of(filter, sqrt(r2), theta, ell);
                ab.x = (decltype(ab.x))(-q * ((double)dx * dx - (double)dy * dy) / r2);
                ab.y = (decltype(ab.y))(-q * 2.0 * dx * dy / r2);
                ++n_r;
            }
            htaps[(size_t)(dy + Ri) * tw + c] = ab;
            if (mask) hdisc[(size_t)(dy + Ri) * tw + c] = in ? (T)1 : (T)0;
        }
    }
    Scratch sc;
    auto up = [](size_t b) { return ((b + 255) / 256) * 256; };
    const size_t tap_bytes = htaps.size() * sizeof(V);
    const size_t disc_bytes = hdisc.size() * sizeof(T);
    const size_t dx_bytes = hdx.size() * sizeof(int);
    const int form = direct_form(Ri);
    const size_t part_bytes = (sizeof(T) == 4 && !mask && form > 0) ? direct_parts_bytes(form, n, batch, Ri) : 0;
    int st = scratch_alloc(sc, up(tap_bytes) + up(disc_bytes) + up(dx_bytes) + part_bytes, s);
    if (st != FM_OK) return st;
    char *base = static_cast<char *>(sc.p);
    V *dtaps = reinterpret_cast<V *>(base);
    T *ddisc = mask ? reinterpret_cast<T *>(base + up(tap_bytes)) : nullptr;
    int *ddx = reinterpret_cast<int *>(base + up(tap_bytes) + up(disc_bytes));
    float *dparts = reinterpret_cast<float *>(base + up(tap_bytes) + up(disc_bytes) + up(dx_bytes));
    FM_CUDA_TRY(cudaMemcpyAsync(dtaps, htaps.data(), tap_bytes, cudaMemcpyHostToDevice, s));
    if (mask) FM_CUDA_TRY(cudaMemcpyAsync(ddisc, hdisc.data(), disc_bytes, cudaMemcpyHostToDevice, s));
    FM_CUDA_TRY(cudaMemcpyAsync(ddx, hdx.data(), dx_bytes, cudaMemcpyHostToDevice, s));

    constexpr int CX = 8, NW = 4;
    const int width = 32 * CX + 2 * Ri + 8;
    const int pw = width + (width >> 3) + 1;
    if constexpr (sizeof(T) == 4) {
        const float2 *ft = reinterpret_cast<const float2 *>(dtaps);
        if (!mask && form == 1) return launch_direct_f2<4, 4>(g1, g2, ft, tw, ddx, map, dparts, n, batch, Ri, s);
        if (!mask && form == 2) return launch_direct_f2<2, 4>(g1, g2, ft, tw, ddx, map, dparts, n, batch, Ri, s);
        if (!mask && form == 3) return launch_direct_f2<4, 2>(g1, g2, ft, tw, ddx, map, dparts, n, batch, Ri, s);
        if (!mask && form == 4) return launch_direct_f2<2, 8>(g1, g2, ft, tw, ddx, map, dparts, n, batch, Ri, s);
    }
    if (!mask) {
        constexpr int RY = 4, TX = 32 * CX, TY = NW * RY;
        const size_t smem = 2ull * 2 * pw * sizeof(T);
        auto k = k_map_direct<T, CX, RY, NW, false>;
        FM_CUDA_TRY(fm::smem_attr((const void *)k, smem));
        dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, batch);
        FM_LAUNCH(FM_K_MAP_DIRECT, k, grid, NW * 32, smem, s, g1, g2, (const T *)nullptr, 0l, dtaps,
                  (const T *)nullptr, tw, ddx, map, (T *)nullptr, n, Ri, (T)n_r);
    } else {
        constexpr int RY = 2, TX = 32 * CX, TY = NW * RY;
        const size_t smem = 2ull * 3 * pw * sizeof(T);
        auto k = k_map_direct<T, CX, RY, NW, true>;
        FM_CUDA_TRY(fm::smem_attr((const void *)k, smem));
        dim3 grid((n + TX - 1) / TX, (n + TY - 1) / TY, batch);
        FM_LAUNCH(FM_K_MAP_DIRECT, k, grid, NW * 32, smem, s, g1, g2, wgt, w_bs, dtaps, ddisc, tw, ddx, map, cov,
                  n, Ri, (T)n_r);
    }
    return FM_OK;
}

int launch_map_direct(const void *g1, const void *g2, const void *weight, long w_bs, void *map, void *coverage, int n,
                      int batch, int filter, double theta, int ell, double cut, int precision, cudaStream_t s)
{
    if (precision == FM_F64)
        return map_direct_impl<double>((const double *)g1, (const double *)g2, (const double *)weight, w_bs,
                                       (double *)map, (double *)coverage, n, batch, filter, theta, ell, cut, s);
    return map_direct_impl<float>((const float *)g1, (const float *)g2, (const float *)weight, w_bs, (float *)map,
                                  (float *)coverage, n, batch, filter, theta, ell, cut, s);
}

}  // namespace fm
