// starlet.cu -- isotropic undecimated (a trous, B3-spline) starlet transform
// (Sec. 3, Sec. 4.2).
//
// Scale j filters c_{j-1} along rows then columns with h = [1,4,6,4,1]/16 at
// taps 0, +-2^(j-1), +-2^j (the B3 two-scale filter with holes) giving c_j,
// and stores the aperture-mass map w_j = c_{j-1} - c_j (theta = 2^j px).
//
// Kernels:
//   st_tile32v2 : (fp32, default) scales 1..F fused on a 64 x 64 tile held in
//             shared memory with a halo of sum_j 2^j pixels per side; each
//             thread row-filters the rows of its column run into a register
//             window and filters that down the column; reads kappa once,
//             writes w_1..w_F and c_F.
//   st_tile32 / st_tile : the same scales with a row-filtered shared buffer
//             (fp32 alternative behind a tuning knob / fp64 and generic).
//   st_row  : r = rows-filtered c_{j-1} for one (large) scale.
//   st_col  : c_j = columns-filtered r, w_j = c_{j-1} - c_j; c_j may overwrite
//             c_{j-1} in place (each thread reads and writes only its own
//             pixel of that array).
//   st_rows_multi / st_cols_multi : every large scale in two kernels (the
//             row and column filters commute); optional, slower here.
#include <algorithm>

#include "common.cuh"
#include "tma.cuh"

namespace fm {

template <typename T> struct B3 {
    // h = [1, 4, 6, 4, 1] / 16
    static constexpr T h0 = (T)0.0625, h1 = (T)0.25, h2 = (T)0.375;
    __device__ __forceinline__ static T apply(T m2, T m1, T c, T p1, T p2)
    {
        return h0 * (m2 + p2) + h1 * (m1 + p1) + h2 * c;
    }
};

// 16-byte vectors: 4 floats or 2 doubles
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int W = 4;
    using V = float4;
};
template <> struct Vec16<double> {
    static constexpr int W = 2;
    using V = double2;
};

template <typename T> __device__ __forceinline__ void ld16(T (&d)[16 / sizeof(T)], const T *p)
{
    using V = typename Vec16<T>::V;
    *reinterpret_cast<V *>(d) = *reinterpret_cast<const V *>(p);
}
template <typename T> __device__ __forceinline__ void st16(T *p, const T (&d)[16 / sizeof(T)])
{
    using V = typename Vec16<T>::V;
    *reinterpret_cast<V *>(p) = *reinterpret_cast<const V *>(d);
}
// streaming (evict-first) store for outputs nothing in the pipeline reads
// again, so they do not push intermediates out of L2
template <typename T> __device__ __forceinline__ void st16cs(T *p, const T (&d)[16 / sizeof(T)])
{
    using V = typename Vec16<T>::V;
    __stcs(reinterpret_cast<V *>(p), *reinterpret_cast<const V *>(d));
}

// Store VW consecutive values at global pixel (gy, gx..gx+VW-1).  Band
// values are final outputs and use streaming stores; `keep` selects plain
// stores (for arrays a later kernel reads).
template <typename T>
__device__ __forceinline__ void emit_band(const T (&w)[16 / sizeof(T)], T *dst, long px, int gy, int gx, int n,
                                          bool vec_ok, bool keep = false)
{
    constexpr int VW = 16 / sizeof(T);
    if (gy >= n) return;
    if (vec_ok && gx + VW <= n) {
        if (keep)
            st16(dst + px, w);
        else
            st16cs(dst + px, w);
    } else {
#pragma unroll
        for (int t = 0; t < VW; ++t)
            if (gx + t < n) dst[px + t] = w[t];
    }
}

// ---------------------------------------------------------------------------
// Scales 1..F fused on a TS x TS output tile.  Shared memory holds the tile
// with a halo of HP >= sum_{j<=F} 2^j pixels (rounded up to 4) per side,
// twice: A = c_{j-1} (then c_j), B = rows-filtered c_{j-1}.  Each thread
// works on VW adjacent pixels with 16-byte shared-memory accesses.
template <typename T, int F, int TS>
__global__ void __launch_bounds__(256) k_st_tile(const T *__restrict__ in, long in_bs, T *__restrict__ w_out, long w_bs,
                                                 long w_ss, T *__restrict__ c_out, long c_bs, int n, int boundary,
                                                 int tiles_x, int tiles_per_map, int vec_ok)
{
    pdl_entry();
    constexpr int VW = 16 / sizeof(T);
    constexpr int H = (1 << (F + 1)) - 2;
    constexpr int HP = ((H + 3) / 4) * 4;
    constexpr int P = TS + 2 * HP;
    constexpr int NQ = P / VW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *A = reinterpret_cast<T *>(smem_raw);
    T *Bf = A + P * P;
    const long b = blockIdx.x / tiles_per_map;
    const int t = blockIdx.x - (int)(b * tiles_per_map);
    const int ty0 = (t / tiles_x) * TS;
    const int tx0 = (t % tiles_x) * TS;
    const T *src = in + b * in_bs;
    const bool vok = vec_ok != 0;

    for (int e = threadIdx.x; e < P * NQ; e += blockDim.x) {
        const int i = e / NQ, q = e % NQ;
        const int gy = fold_index(ty0 - HP + i, n, boundary);
        const int gx0 = tx0 - HP + q * VW;
        const T *rowp = src + (long)gy * n;
        alignas(16) T v[VW];
        if (vok && gx0 >= 0 && gx0 + VW <= n) {
            ld16(v, rowp + gx0);
        } else {
#pragma unroll
            for (int u = 0; u < VW; ++u) v[u] = rowp[fold_index(gx0 + u, n, boundary)];
        }
        st16(A + i * P + q * VW, v);
    }
    __syncthreads();

#pragma unroll
    for (int j = 1; j <= F; ++j) {
        const int s = 1 << (j - 1);
        const int hb = (1 << (F + 1)) - (1 << j);        // halo still valid before scale j
        const int ha = (1 << (F + 1)) - (1 << (j + 1));  // after
        const int ncq = (TS + 2 * ha) / VW;
        // rows pass
        {
            const int nr = TS + 2 * hb;
            for (int e = threadIdx.x; e < nr * ncq; e += blockDim.x) {
                const int i = HP - hb + e / ncq;
                const int x = HP - ha + (e % ncq) * VW;
                const T *row = A + i * P;
                alignas(16) T o[VW];
                if (2 * s <= VW) {
                    alignas(16) T win[3 * VW];
                    T *wp = win;
                    ld16(*reinterpret_cast<T(*)[VW]>(wp), row + x - VW);
                    ld16(*reinterpret_cast<T(*)[VW]>(wp + VW), row + x);
                    ld16(*reinterpret_cast<T(*)[VW]>(wp + 2 * VW), row + x + VW);
#pragma unroll
                    for (int u = 0; u < VW; ++u)
                        o[u] = B3<T>::apply(win[VW + u - 2 * s], win[VW + u - s], win[VW + u], win[VW + u + s],
                                            win[VW + u + 2 * s]);
                } else {
                    alignas(16) T m2[VW]; alignas(16) T m1[VW]; alignas(16) T c0[VW]; alignas(16) T p1[VW]; alignas(16) T p2[VW];
                    ld16(m2, row + x - 2 * s);
                    ld16(m1, row + x - s);
                    ld16(c0, row + x);
                    ld16(p1, row + x + s);
                    ld16(p2, row + x + 2 * s);
#pragma unroll
                    for (int u = 0; u < VW; ++u) o[u] = B3<T>::apply(m2[u], m1[u], c0[u], p1[u], p2[u]);
                }
                st16(Bf + i * P + x, o);
            }
        }
        __syncthreads();
        // columns pass, band output, c_j over c_{j-1}
        {
            const int nr = TS + 2 * ha;
            for (int e = threadIdx.x; e < nr * ncq; e += blockDim.x) {
                const int i = HP - ha + e / ncq;
                const int x = HP - ha + (e % ncq) * VW;
                const T *bp = Bf + i * P + x;
                alignas(16) T m2[VW]; alignas(16) T m1[VW]; alignas(16) T c0[VW]; alignas(16) T p1[VW]; alignas(16) T p2[VW]; alignas(16) T cj[VW]; alignas(16) T prev[VW]; alignas(16) T w[VW];
                ld16(m2, bp - 2 * s * P);
                ld16(m1, bp - s * P);
                ld16(c0, bp);
                ld16(p1, bp + s * P);
                ld16(p2, bp + 2 * s * P);
                ld16(prev, A + i * P + x);
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    cj[u] = B3<T>::apply(m2[u], m1[u], c0[u], p1[u], p2[u]);
                    w[u] = prev[u] - cj[u];
                }
                const int oi = i - HP, ox = x - HP;
                if (oi >= 0 && oi < TS && ox >= 0 && ox < TS) {
                    const int gy = ty0 + oi, gx = tx0 + ox;
                    const long px = (long)gy * n + gx;
                    emit_band<T>(w, w_out + b * w_bs + (long)(j - 1) * w_ss, px, gy, gx, n, vok);
                    if (j == F && c_out) emit_band<T>(cj, c_out + b * c_bs, px, gy, gx, n, vok, true);
                }
                if (j < F) st16(A + i * P + x, cj);
            }
        }
        if (j < F) __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// fp32 variant of the fused tile with register reuse of the filter taps in
// the columns pass: a thread computes 4 pixels of one float4 column at rows
// i, i+s, i+2s, i+3s from 8 row loads.  Tasks of one row (or row group) start
// on an 8-lane boundary so 128-bit shared-memory accesses do not conflict.  Filter sums are kept
// unnormalised (taps 1,4,6,4,1) and scaled by 1/256 once per scale, which is
// exact (a power of two).
__device__ __forceinline__ float4 f4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sf4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float tap5(float a, float b, float c, float d, float e)
{
    // (a + e) + 4 (b + d) + 6 c
    return fmaf(6.f, c, fmaf(4.f, b + d, a + e));
}
__device__ __forceinline__ float4 tap5(float4 a, float4 b, float4 c, float4 d, float4 e)
{
    return make_float4(tap5(a.x, b.x, c.x, d.x, e.x), tap5(a.y, b.y, c.y, d.y, e.y), tap5(a.z, b.z, c.z, d.z, e.z),
                       tap5(a.w, b.w, c.w, d.w, e.w));
}
__device__ __forceinline__ float get(const float4 &v, int u) { return u == 0 ? v.x : u == 1 ? v.y : u == 2 ? v.z : v.w; }

template <int F>
__global__ void __launch_bounds__(256) k_st_tile32(const float *__restrict__ in, long in_bs, float *__restrict__ w_out,
                                                   long w_bs, long w_ss, float *__restrict__ c_out, long c_bs, int n,
                                                   int boundary, int tiles_x, int tiles_per_map,
                                                   int vec_ok)
{
    pdl_entry();
    constexpr int TS = 64;
    constexpr int H = (1 << (F + 1)) - 2;
    constexpr int HP = ((H + 3) / 4) * 4;
    constexpr int P = TS + 2 * HP;
    constexpr int NQ = P / 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *A = reinterpret_cast<float *>(smem_raw);  // c_{j-1} (true scale)
    float *Bf = A + P * P;                            // 16 x rows-filtered c_{j-1}
    const long b = blockIdx.x / tiles_per_map;
    const int t = blockIdx.x - (int)(b * tiles_per_map);
    const int ty0 = (t / tiles_x) * TS;
    const int tx0 = (t % tiles_x) * TS;
    const float *src = in + b * in_bs;
    const bool vok = vec_ok != 0;

    for (int e = threadIdx.x; e < P * NQ; e += blockDim.x) {
        const int i = e / NQ, q = e % NQ;
        const int gy = fold_index(ty0 - HP + i, n, boundary);
        const int gx0 = tx0 - HP + q * 4;
        const float *rowp = src + (long)gy * n;
        float4 v;
        if (vok && gx0 >= 0 && gx0 + 4 <= n) {
            v = f4(rowp + gx0);
        } else {
            v.x = rowp[fold_index(gx0, n, boundary)];
            v.y = rowp[fold_index(gx0 + 1, n, boundary)];
            v.z = rowp[fold_index(gx0 + 2, n, boundary)];
            v.w = rowp[fold_index(gx0 + 3, n, boundary)];
        }
        sf4(A + i * P + q * 4, v);
    }
    __syncthreads();

#pragma unroll
    for (int j = 1; j <= F; ++j) {
        const int s = 1 << (j - 1);
        const int hb = (1 << (F + 1)) - (1 << j);
        const int ha = (1 << (F + 1)) - (1 << (j + 1));
        const int ncq = (TS + 2 * ha) / 4;  // float4 columns of the region (even)
        const int c_lo = HP - ha;
        // rows pass: one float4 per task; a row's tasks start on an 8-lane
        // boundary (ncq padded to ncqp) so a quarter warp's 128-bit loads
        // stay within one row and hit distinct banks
        const int ncqp = (ncq + 7) & ~7;
        {
            const int nr = TS + 2 * hb;
            for (int e = threadIdx.x; e < nr * ncqp; e += blockDim.x) {
                const int q = e % ncqp;
                if (q >= ncq) continue;
                const int i = HP - hb + e / ncqp;
                const int x = c_lo + q * 4;
                const float *row = A + i * P + x;
                float4 o;
                if (s <= 2) {
                    const float4 a = f4(row - 4), bq = f4(row), c = f4(row + 4);
                    const float w[12] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w, c.x, c.y, c.z, c.w};
                    o = make_float4(tap5(w[4 - 2 * s], w[4 - s], w[4], w[4 + s], w[4 + 2 * s]),
                                    tap5(w[5 - 2 * s], w[5 - s], w[5], w[5 + s], w[5 + 2 * s]),
                                    tap5(w[6 - 2 * s], w[6 - s], w[6], w[6 + s], w[6 + 2 * s]),
                                    tap5(w[7 - 2 * s], w[7 - s], w[7], w[7 + s], w[7 + 2 * s]));
                } else {
                    o = tap5(f4(row - 2 * s), f4(row - s), f4(row), f4(row + s), f4(row + 2 * s));
                }
                sf4(Bf + i * P + x, o);
            }
        }
        __syncthreads();
        // columns pass: rows lo + r + s (4m + k), k = 0..3, one float4 column
        {
            const int nr = TS + 2 * ha;  // divisible by 4 s
            const int groups = nr / (4 * s);
            const int ntask = s * groups * ncqp;
            for (int e = threadIdx.x; e < ntask; e += blockDim.x) {
                const int qq = e % ncqp;
                if (qq >= ncq) continue;
                const int rg = e / ncqp;  // residue + s * group
                const int r = rg % s, m = rg / s;
                const int x = c_lo + qq * 4;
                const int i0 = HP - ha + r + s * 4 * m;
                const float *bp = Bf + i0 * P + x;
                float4 win[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) win[u] = f4(bp + (u - 2) * s * P);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * s;
                    float4 c = tap5(win[k], win[k + 1], win[k + 2], win[k + 3], win[k + 4]);
                    c.x *= (1.f / 256.f);
                    c.y *= (1.f / 256.f);
                    c.z *= (1.f / 256.f);
                    c.w *= (1.f / 256.f);
                    float *ap = A + i * P + x;
                    const float4 prev = f4(ap);
                    const int oi = i - HP, ox = x - HP;
                    if (oi >= 0 && oi < TS && ox >= 0 && ox < TS) {
                        const int gy = ty0 + oi, gx = tx0 + ox;
                        alignas(16) float w[4] = {prev.x - c.x, prev.y - c.y, prev.z - c.z, prev.w - c.w};
                        const long px = (long)gy * n + gx;
                        emit_band<float>(w, w_out + b * w_bs + (long)(j - 1) * w_ss, px, gy, gx, n, vok);
                        if (j == F && c_out) {
                            alignas(16) float cc[4] = {c.x, c.y, c.z, c.w};
                            emit_band<float>(cc, c_out + b * c_bs, px, gy, gx, n, vok, true);
                        }
                    }
                    if (j < F) sf4(ap, c);
                }
            }
        }
        if (j < F) __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Fused small scales 1..F, register-window form (fp32).  Same tile, halo and
// integer taps as k_st_tile32, but each thread owns a vertical run of K
// outputs of one float4 column at row stride s and forms the row-filtered
// values it needs itself: it walks the K + 4 rows i0 + s (t - 2), filters
// each along the row (taps +-s, +-2s from shared memory) into a five-deep
// register window and filters the window down the column.  The centre of a
// walked row is c_{j-1} at that row, so the band w_j = c_{j-1} - c_j needs no
// further read.  c_j goes to the other shared buffer: one barrier per scale,
// no row-filtered buffer.  K per scale is chosen at compile time from the
// task count (tile_k below).  Measured on 32 maps of 1024^2 (scales 1-3):
// 0.241 ms against 0.280 ms for k_st_tile32.
__host__ __device__ constexpr int tile_task_cols(int F, int j, int TS)
{
    return (TS + 2 * ((1 << (F + 1)) - (1 << (j + 1)))) / 4;
}
// K for scale j: the fewest rows walked by one thread, ceil(tasks / 256) (K + 4)
// (measured against the choice with the least shared-memory traffic among
// one-round task sets: the tile kernel is bound by latency more than by the
// shared-memory pipe, 0.241 vs 0.269 ms per 32 maps of 1024^2).
__host__ __device__ constexpr int tile_k(int F, int j, int TS)
{
    const int s = 1 << (j - 1);
    const int nr = TS + 2 * ((1 << (F + 1)) - (1 << (j + 1)));
    const int ncq = nr / 4, ncqp = (ncq + 7) & ~7;
    const int lds = s <= 2 ? 3 : 5;
    int best = 1;
    long bc = -1, bw = -1;
    for (int K = 1; K <= 16; ++K) {
        if (nr % (s * K)) continue;
        const long nt = (long)s * (nr / (s * K)) * ncqp;
        const long cost = (nt + 255) / 256 * (K + 4);
        const long work = (long)s * (nr / (s * K)) * ncq * ((K + 4) * lds + K);
        if (bc < 0 || cost < bc || (cost == bc && work < bw)) {
            best = K;
            bc = cost;
            bw = work;
        }
    }
    return best;
}

template <int F, int J>
__device__ __forceinline__ void tile2_scale(const float *__restrict__ A, float *__restrict__ C, int ty0, int tx0,
                                            float *__restrict__ w_dst, float *__restrict__ c_dst, int n, bool vok)
{
    constexpr int TS = 64;
    constexpr int H = (1 << (F + 1)) - 2;
    constexpr int HP = ((H + 3) / 4) * 4;
    constexpr int P = TS + 2 * HP;
    constexpr int s = 1 << (J - 1);
    constexpr int ha = (1 << (F + 1)) - (1 << (J + 1));
    constexpr int nr = TS + 2 * ha;
    constexpr int ncq = nr / 4;
    constexpr int ncqp = (ncq + 7) & ~7;
    constexpr int K = tile_k(F, J, TS);
    static_assert(nr % (s * K) == 0, "task rows");
    constexpr int groups = nr / (s * K);
    constexpr int ntask = s * groups * ncqp;
    constexpr int c_lo = HP - ha;
    static_assert(HP >= H + 2, "the s <= 2 row loads reach 4 columns left of the region");
    for (int e = threadIdx.x; e < ntask; e += blockDim.x) {
        const int qq = e % ncqp;
        if (qq >= ncq) continue;
        const int rg = e / ncqp;  // residue + s * group
        const int r = rg % s, m = rg / s;
        const int x = c_lo + qq * 4;
        const int i0 = HP - ha + r + s * K * m;
        float4 win[5], ctr[3];
#pragma unroll
        for (int t = 0; t < K + 4; ++t) {
            const float *row = A + (i0 + (t - 2) * s) * P + x;
            if constexpr (s <= 2) {
                const float4 a = f4(row - 4), bq = f4(row), c = f4(row + 4);
                const float w[12] = {a.x, a.y, a.z, a.w, bq.x, bq.y, bq.z, bq.w, c.x, c.y, c.z, c.w};
                win[t % 5] = make_float4(tap5(w[4 - 2 * s], w[4 - s], w[4], w[4 + s], w[4 + 2 * s]),
                                         tap5(w[5 - 2 * s], w[5 - s], w[5], w[5 + s], w[5 + 2 * s]),
                                         tap5(w[6 - 2 * s], w[6 - s], w[6], w[6 + s], w[6 + 2 * s]),
                                         tap5(w[7 - 2 * s], w[7 - s], w[7], w[7 + s], w[7 + 2 * s]));
                ctr[t % 3] = bq;
            } else {
                const float4 c0 = f4(row);
                win[t % 5] = tap5(f4(row - 2 * s), f4(row - s), c0, f4(row + s), f4(row + 2 * s));
                ctr[t % 3] = c0;
            }
            if (t >= 4) {
                const int k = t - 4;
                const int i = i0 + k * s;
                float4 c = tap5(win[k % 5], win[(k + 1) % 5], win[(k + 2) % 5], win[(k + 3) % 5], win[(k + 4) % 5]);
                c.x *= (1.f / 256.f);
                c.y *= (1.f / 256.f);
                c.z *= (1.f / 256.f);
                c.w *= (1.f / 256.f);
                const float4 prev = ctr[(k + 2) % 3];
                const int oi = i - HP, ox = x - HP;
                if (oi >= 0 && oi < TS && ox >= 0 && ox < TS) {
                    const int gy = ty0 + oi, gx = tx0 + ox;
                    alignas(16) float w[4] = {prev.x - c.x, prev.y - c.y, prev.z - c.z, prev.w - c.w};
                    const long px = (long)gy * n + gx;
                    emit_band<float>(w, w_dst, px, gy, gx, n, vok);
                    if (J == F && c_dst) {
                        alignas(16) float cc[4] = {c.x, c.y, c.z, c.w};
                        emit_band<float>(cc, c_dst, px, gy, gx, n, vok, true);
                    }
                }
                if (J < F) sf4(C + i * P + x, c);
            }
        }
    }
}

// Shared memory: 128 bytes of alignment slack, two P x P buffers, one mbarrier.
template <int F> constexpr size_t tile2_smem()
{
    constexpr int H = (1 << (F + 1)) - 2, HP = ((H + 3) / 4) * 4, P = 64 + 2 * HP;
    return 128 + 2ull * P * P * sizeof(float) + 8;
}

// tmap (when use_tma): kappa as a 3-D tensor {n, n, batch} of fp32 with a
// P x P x 1 box; every tile's box then arrives by one bulk tensor copy (edge
// tiles fold the part outside the map afterwards).  VOK (16-byte row
// accesses valid: vec_ok) is a template parameter, so that the stores of the
// usual case carry no scalar fallback.
template <int F, bool VOK>
__global__ void __launch_bounds__(256, F >= 4 ? 1 : 3)
    k_st_tile32v2(const float *__restrict__ in, long in_bs, float *__restrict__ w_out, long w_bs, long w_ss,
                  float *__restrict__ c_out, long c_bs, int n, int boundary, int tiles_x, int tiles_per_map,
                  int vec_ok, const __grid_constant__ CUtensorMap tmap, int use_tma)
{
    pdl_entry();
    constexpr int TS = 64;
    constexpr int H = (1 << (F + 1)) - 2;
    constexpr int HP = ((H + 3) / 4) * 4;
    constexpr int P = TS + 2 * HP;
    constexpr int NQ = P / 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *b0 = align128<float>(smem_raw);  // c_0, c_2, ... (a bulk copy destination)
    float *b1 = b0 + P * P;                 // c_1, c_3, ...
    uint64_t *bar = reinterpret_cast<uint64_t *>(b1 + P * P);
    const long b = blockIdx.x / tiles_per_map;
    const int t = blockIdx.x - (int)(b * tiles_per_map);
    const int ty0 = (t / tiles_x) * TS;
    const int tx0 = (t % tiles_x) * TS;
    const float *src = in + b * in_bs;
    constexpr bool vok = VOK;

    const bool interior = vok && ty0 >= HP && tx0 >= HP && ty0 + TS + HP <= n && tx0 + TS + HP <= n;
    if (use_tma & 1) {
        // one bulk tensor copy of the P x P halo box, completion on the mbarrier
        // (use_tma bit 1, a test hook: 16 bytes more are announced than the
        // copy delivers, so the bounded wait runs out and is flagged).  Box
        // columns and rows outside the map arrive as zeros.
        if (threadIdx.x == 0) mbar_init(bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(bar, (uint32_t)(P * P * sizeof(float)) + ((use_tma & 2) ? 16u : 0u));
            tma_load_3d(b0, &tmap, tx0 - HP, ty0 - HP, (int)b, bar);
        }
        if (!tma_wait_all(bar, 0)) return;  // the copy never completed (flagged)
        if (!interior) {
            // Edge tile: each box position outside the map takes the value at
            // its folded position.  Mirrored, that position lies in the box
            // for every position the scales read (the halo H is at most HP,
            // and a ragged last tile starts at most n - 1); it came with the
            // copy and is not itself rewritten here.  Periodic positions, and
            // far ones of a ragged tile, load from global memory.
            // The outside positions are enumerated directly: whole box rows
            // above or below the map, then the columns left or right of it in
            // the other rows.
            const int oy = ty0 - HP, ox = tx0 - HP;
            const int rt = oy < 0 ? -oy : 0, rb = oy + P > n ? oy + P - n : 0;
            const int cl = ox < 0 ? -ox : 0, cr = ox + P > n ? ox + P - n : 0, cw = cl + cr;
            auto fix = [&](int i, int q) {
                const int fy = fold_index(oy + i, n, boundary), fx = fold_index(ox + q, n, boundary);
                const int si = fy - oy, sq = fx - ox;
                b0[i * P + q] = boundary != FM_PERIODIC && si >= 0 && si < P && sq >= 0 && sq < P
                                    ? b0[si * P + sq]
                                    : src[(long)fy * n + fx];
            };
            for (int e = threadIdx.x; e < (rt + rb) * P; e += blockDim.x) {
                const int k = e / P, q = e - k * P;
                fix(k < rt ? k : P - rb + (k - rt), q);
            }
            if (cw > 0) {
                for (int e = threadIdx.x; e < (P - rt - rb) * cw; e += blockDim.x) {
                    const int k = e / cw, c = e - k * cw;
                    fix(rt + k, c < cl ? c : P - cr + (c - cl));
                }
            }
        }
    } else if (interior) {
        // interior tile: no folding; every thread's loads are in flight together
        constexpr int IT = (P * NQ + 255) / 256;
        const float *org = src + (long)(ty0 - HP) * n + (tx0 - HP);
        float4 v[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int e = threadIdx.x + it * 256;
            if (e < P * NQ) v[it] = f4(org + (long)(e / NQ) * n + (e % NQ) * 4);
        }
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const int e = threadIdx.x + it * 256;
            if (e < P * NQ) sf4(b0 + (e / NQ) * P + (e % NQ) * 4, v[it]);
        }
    } else {
        for (int e = threadIdx.x; e < P * NQ; e += blockDim.x) {
            const int i = e / NQ, q = e % NQ;
            const int gy = fold_index(ty0 - HP + i, n, boundary);
            const int gx0 = tx0 - HP + q * 4;
            const float *rowp = src + (long)gy * n;
            float4 v;
            if (vok && gx0 >= 0 && gx0 + 4 <= n) {
                v = f4(rowp + gx0);
            } else {
                v.x = rowp[fold_index(gx0, n, boundary)];
                v.y = rowp[fold_index(gx0 + 1, n, boundary)];
                v.z = rowp[fold_index(gx0 + 2, n, boundary)];
                v.w = rowp[fold_index(gx0 + 3, n, boundary)];
            }
            sf4(b0 + i * P + q * 4, v);
        }
    }
    __syncthreads();
    float *wb = w_out + b * w_bs;
    float *cb = c_out ? c_out + b * c_bs : nullptr;
    tile2_scale<F, 1>(b0, b1, ty0, tx0, wb, cb, n, vok);
    if constexpr (F >= 2) {
        __syncthreads();
        tile2_scale<F, (F >= 2 ? 2 : 1)>(b1, b0, ty0, tx0, wb + w_ss, cb, n, vok);
    }
    if constexpr (F >= 3) {
        __syncthreads();
        tile2_scale<F, (F >= 3 ? 3 : 1)>(b0, b1, ty0, tx0, wb + 2 * w_ss, cb, n, vok);
    }
    if constexpr (F >= 4) {
        __syncthreads();
        tile2_scale<F, (F >= 4 ? 4 : 1)>(b1, b0, ty0, tx0, wb + 3 * w_ss, cb, n, vok);
    }
}

// ---------------------------------------------------------------------------
// One large scale, rows: r = rows-filtered c (taps +-s, +-2s), VW pixels per
// thread.  grid = (ceil(n / (blockDim.x VW)), n, batch).
template <typename T>
__global__ void __launch_bounds__(256) k_st_row(const T *__restrict__ c, long c_bs, T *__restrict__ r, long r_bs,
                                                int n, int s, int boundary, int vec_ok)
{
    pdl_entry();
    constexpr int VW = 16 / sizeof(T);
    const int x = (blockIdx.x * blockDim.x + threadIdx.x) * VW;
    if (x >= n) return;
    const int y = blockIdx.y;
    const long b = blockIdx.z;
    const T *row = c + b * c_bs + (long)y * n;
    T *dst = r + b * r_bs + (long)y * n;
    alignas(16) T o[VW];
    if (vec_ok && s % VW == 0 && x - 2 * s >= 0 && x + VW + 2 * s <= n) {
        alignas(16) T m2[VW]; alignas(16) T m1[VW]; alignas(16) T c0[VW]; alignas(16) T p1[VW]; alignas(16) T p2[VW];
        ld16(m2, row + x - 2 * s);
        ld16(m1, row + x - s);
        ld16(c0, row + x);
        ld16(p1, row + x + s);
        ld16(p2, row + x + 2 * s);
#pragma unroll
        for (int u = 0; u < VW; ++u) o[u] = B3<T>::apply(m2[u], m1[u], c0[u], p1[u], p2[u]);
    } else {
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            const int xx = x + u < n ? x + u : n - 1;
            o[u] = B3<T>::apply(row[fold_index(xx - 2 * s, n, boundary)], row[fold_index(xx - s, n, boundary)],
                                row[xx], row[fold_index(xx + s, n, boundary)],
                                row[fold_index(xx + 2 * s, n, boundary)]);
        }
    }
    if (vec_ok && x + VW <= n) {
        st16(dst + x, o);
    } else {
#pragma unroll
        for (int u = 0; u < VW; ++u)
            if (x + u < n) dst[x + u] = o[u];
    }
}

// One large scale, columns: thread owns VW adjacent columns and KR rows at
// stride s (rows r0 + s (m KR + k)), so its five taps slide down a register
// window: KR + 4 row loads for KR outputs.  c_j = column-filtered r,
// w_j = c_{j-1} - c_j, c_j written over c_{j-1} when they alias.
// grid = (ceil(n / (128 VW)), s * ceil(n / (s KR)), batch).
// tma (fp32, n a multiple of 512, 512 columns per CTA): bit 0 = the KR + 4
// window rows of r arrive by one bulk tensor copy (mr: r as {256, n/256, s,
// n/s, batch}, box {256, 2, 1, KR + 4, 1}), bit 1 = the KR rows of c_{j-1}
// likewise (mp); row groups whose window leaves the map use plain loads.
template <typename T, int KR>
__global__ void __launch_bounds__(128) k_st_col(const T *__restrict__ r, long r_bs, const T *c_prev, long prev_bs,
                                                T *c_next, long next_bs, T *__restrict__ w_out, long w_bs, int n,
                                                int s, int boundary, int vec_ok,
                                                const __grid_constant__ CUtensorMap mr,
                                                const __grid_constant__ CUtensorMap mp, int tma)
{
    pdl_entry();
    constexpr int VW = 16 / sizeof(T);
    const int x = (blockIdx.x * blockDim.x + threadIdx.x) * VW;
    if (x >= n) return;
    const int r0 = blockIdx.y % s, m = blockIdx.y / s;
    const long b = blockIdx.z;
    if constexpr (sizeof(T) == 4) {
        const int mb = m * KR;
        if (tma && mb >= 2 && r0 + s * (mb + KR + 1) < n) {
            extern __shared__ __align__(16) unsigned char smem_raw[];
            __shared__ uint64_t bar;
            float *sr = align128<float>(smem_raw);  // [KR + 4][512] window rows
            float *sp = sr + (KR + 4) * 512;        // [KR][512] rows of c_{j-1}
            const int x0 = blockIdx.x * 512, xl = threadIdx.x * 4;
            if (threadIdx.x == 0) mbar_init(&bar, 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                mbar_expect_tx(&bar, ((tma & 1) ? (KR + 4) * 2048u : 0u) + ((tma & 2) ? KR * 2048u : 0u));
                if (tma & 1) tma_load_5d(sr, &mr, 0, x0 / 256, r0, mb - 2, (int)b, &bar);
                if (tma & 2) tma_load_5d(sp, &mp, 0, x0 / 256, r0, mb, (int)b, &bar);
            }
            if (!tma_wait_all(&bar, 0)) return;  // the copies never completed (flagged)
            const float *rb = reinterpret_cast<const float *>(r) + b * r_bs;
            float4 win[5];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                win[u] = (tma & 1) ? f4(sr + u * 512 + xl) : f4(rb + (long)(r0 + s * (mb + u - 2)) * n + x);
#pragma unroll
            for (int k = 0; k < KR; ++k) {
                const int y = r0 + s * (mb + k);
                win[(k + 4) % 5] = (tma & 1) ? f4(sr + (k + 4) * 512 + xl) : f4(rb + (long)(y + 2 * s) * n + x);
                const long px = (long)y * n + x;
                const float4 p4 =
                    (tma & 2) ? f4(sp + k * 512 + xl) : f4(reinterpret_cast<const float *>(c_prev) + b * prev_bs + px);
                // the same arithmetic as the plain-load path below
                const float4 &a = win[k % 5], &bq = win[(k + 1) % 5], &c = win[(k + 2) % 5],
                             &d = win[(k + 3) % 5], &e = win[(k + 4) % 5];
                alignas(16) float cj[4] = {B3<float>::apply(a.x, bq.x, c.x, d.x, e.x),
                                           B3<float>::apply(a.y, bq.y, c.y, d.y, e.y),
                                           B3<float>::apply(a.z, bq.z, c.z, d.z, e.z),
                                           B3<float>::apply(a.w, bq.w, c.w, d.w, e.w)};
                alignas(16) float w[4] = {p4.x - cj[0], p4.y - cj[1], p4.z - cj[2], p4.w - cj[3]};
                emit_band<float>(w, reinterpret_cast<float *>(w_out) + b * w_bs, px, y, x, n, true);
                if (c_next) emit_band<float>(cj, reinterpret_cast<float *>(c_next) + b * next_bs, px, y, x, n, true, true);
            }
            return;
        }
    }
    const bool vok = vec_ok && x + VW <= n;
    const T *rb = r + b * r_bs;
    auto load_row = [&](int yy, T (&d)[VW]) {
        const T *p = rb + (long)fold_index(yy, n, boundary) * n;
        if (vok) {
            ld16(d, p + x);
        } else {
#pragma unroll
            for (int u = 0; u < VW; ++u) d[u] = p[x + u < n ? x + u : n - 1];
        }
    };
    alignas(16) T win[5][VW];
    const int ybase = r0 + s * (m * KR);
#pragma unroll
    for (int u = 0; u < 4; ++u) load_row(ybase + (u - 2) * s, win[u]);
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const int y = ybase + k * s;
        if (y >= n) break;
        load_row(y + 2 * s, win[(k + 4) % 5]);
        alignas(16) T cj[VW]; alignas(16) T prev[VW]; alignas(16) T w[VW];
        const long px = (long)y * n + x;
        if (vok) {
            ld16(prev, c_prev + b * prev_bs + px);
        } else {
#pragma unroll
            for (int u = 0; u < VW; ++u) prev[u] = x + u < n ? c_prev[b * prev_bs + px + u] : (T)0;
        }
#pragma unroll
        for (int u = 0; u < VW; ++u) {
            cj[u] = B3<T>::apply(win[k % 5][u], win[(k + 1) % 5][u], win[(k + 2) % 5][u], win[(k + 3) % 5][u],
                                 win[(k + 4) % 5][u]);
            w[u] = prev[u] - cj[u];
        }
        emit_band<T>(w, w_out + b * w_bs, px, y, x, n, vok);
        if (c_next) emit_band<T>(cj, c_next + b * next_bs, px, y, x, n, vok, true);
    }
}

// ---------------------------------------------------------------------------
// One large scale in one pass (fp32, large_path 4: maps whose arrays stream
// through HBM).  A CTA owns 512 columns (128 threads x float4) and KR output
// rows y_k = r0 + s (mb + k) of one map, like k_st_col.  Its KR + 4 window
// rows of c_{j-1} (rows r0 + s (mb + t - 2), folded at the map's top and
// bottom) arrive by one bulk tensor copy each, 512 + 4s columns wide
// (x0 - 2s .. x0 + 512 + 2s; mc views c_{j-1} as {2s, n / 2s, rows}), into
// shared memory; halo columns outside the map are then loaded folded.  Each
// thread row-filters its window rows there (taps +-s, +-2s) into a five-row
// register window and filters that down the column: c_j, and w_j = c_{j-1} -
// c_j with c_{j-1} the centre of the window row.  The row-filtered map never
// goes through memory (the pair k_st_row + k_st_col moves 24 bytes per pixel,
// this pass 8 + 4 (KR + 4) / KR (512 + 4s) / 512).  c_next must not alias
// c_prev: other CTAs read its rows and halo columns.  4 <= s <= 128.
template <int KR>
__global__ void __launch_bounds__(128) k_st_scale(const float *c_prev, float *c_next, long next_bs,
                                                  float *__restrict__ w_out, long w_bs, int n, int s, int boundary,
                                                  const __grid_constant__ CUtensorMap mc)
{
    pdl_entry();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t bar;
    const int RW = (512 + 4 * s + 31) & ~31;  // floats per staged row: 512 + 4s, padded so that every row (a
                                              // bulk tensor copy destination) starts 128-byte aligned
    float *sw = align128<float>(smem_raw);    // [KR + 4][RW]
    const int x0 = blockIdx.x * 512;
    const int r0 = blockIdx.y % s, mb = (blockIdx.y / s) * KR;
    const long b = blockIdx.z;
    const float *cb = c_prev + b * (long)n * n;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    // one window row per lane of the first warp, after lane 0 announced the bytes
    static_assert(KR + 4 <= 32, "window rows per warp");
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) mbar_expect_tx(&bar, (uint32_t)((KR + 4) * (512 + 4 * s) * sizeof(float)));
        __syncwarp();
        const int t = threadIdx.x;
        if (t < KR + 4) {
            const int y = fold_index(r0 + s * (mb + t - 2), n, boundary);
            tma_load_3d(sw + t * RW, &mc, 0, x0 / (2 * s) - 1, (int)(b * n + y), &bar);
        }
    }
    if (!tma_wait_all(&bar, 0)) return;  // the copies never completed (flagged)
    if ((x0 == 0 || x0 + 512 == n) && boundary != FM_PERIODIC) {
        // halo columns outside the map (the copies filled them with zeros):
        // with 2s <= 256 < 512 only the first CTA's left halo and the last
        // one's right halo leave the map.  Mirrored, staged column 2s + x of
        // map column x (x0 = 0) gets column -x, and map column n + h
        // (x0 = n - 512) gets n - 2 - h; both lie inside the map and were
        // staged by this CTA.
        const bool lo = x0 == 0, hi = x0 + 512 == n;
        for (int h = threadIdx.x; h < 2 * s; h += blockDim.x) {
#pragma unroll
            for (int t = 0; t < KR + 4; ++t) {
                float *row = sw + t * RW;
                if (lo) row[h] = row[4 * s - h];
                if (hi) row[512 + 2 * s + h] = row[510 + 2 * s - h];
            }
        }
        __syncthreads();
    } else if (x0 - 2 * s < 0 || x0 + 512 + 2 * s > n) {
        // periodic: halo columns outside the map wrap to its other edge and
        // come from global memory
        for (int e = threadIdx.x; e < (KR + 4) * 4 * s; e += blockDim.x) {
            const int t = e / (4 * s), h = e % (4 * s);
            const int xl = h < 2 * s ? h : 512 + h;  // left halo, then right halo
            const int x = x0 - 2 * s + xl;
            if (x < 0 || x >= n) {
                const int xf = fold_index(x, n, boundary);
                if (boundary == FM_PERIODIC) {
                    const int y = fold_index(r0 + s * (mb + t - 2), n, boundary);
                    sw[t * RW + xl] = cb[(long)y * n + xf];
                } else {
                    sw[t * RW + xl] = sw[t * RW + xf - x0 + 2 * s];
                }
            }
        }
        __syncthreads();
    }
    const int xl = 2 * s + 4 * threadIdx.x, x = x0 + 4 * threadIdx.x;
    float4 win[5], ctr[3];
#pragma unroll
    for (int t = 0; t < KR + 4; ++t) {
        const float *row = sw + t * RW + xl;
        const float4 m2 = f4(row - 2 * s), m1 = f4(row - s), c0 = f4(row), p1 = f4(row + s), p2 = f4(row + 2 * s);
        // the same arithmetic as k_st_row
        win[t % 5] = make_float4(B3<float>::apply(m2.x, m1.x, c0.x, p1.x, p2.x),
                                 B3<float>::apply(m2.y, m1.y, c0.y, p1.y, p2.y),
                                 B3<float>::apply(m2.z, m1.z, c0.z, p1.z, p2.z),
                                 B3<float>::apply(m2.w, m1.w, c0.w, p1.w, p2.w));
        ctr[t % 3] = c0;
        if (t >= 4) {
            const int k = t - 4;
            const int y = r0 + s * (mb + k);
            if (y < n) {
                // the same arithmetic as k_st_col
                const float4 &a = win[k % 5], &bq = win[(k + 1) % 5], &c = win[(k + 2) % 5], &d = win[(k + 3) % 5],
                             &e = win[(k + 4) % 5];
                alignas(16) float cj[4] = {B3<float>::apply(a.x, bq.x, c.x, d.x, e.x),
                                           B3<float>::apply(a.y, bq.y, c.y, d.y, e.y),
                                           B3<float>::apply(a.z, bq.z, c.z, d.z, e.z),
                                           B3<float>::apply(a.w, bq.w, c.w, d.w, e.w)};
                const float4 p = ctr[(k + 2) % 3];
                alignas(16) float w[4] = {p.x - cj[0], p.y - cj[1], p.z - cj[2], p.w - cj[3]};
                const long px = (long)y * n + x;
                // n is a multiple of 512: the whole vector is inside
                st16cs(w_out + b * w_bs + px, w);
                if (c_next) st16(c_next + b * next_bs + px, cj);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Column pass of large scale j fused with the row pass of scale j + 1.  A CTA
// owns KR whole rows y_k = r0 + s (m KR + k) of one map (rows at the stride s
// of scale j, like k_st_col): each thread runs the column filter down CPT
// columns of VW pixels (the register window of k_st_col), writes w_j and c_j,
// and keeps its c_j in shared memory; after one barrier it filters those rows
// along x at spacing 2s (the row pass of scale j + 1) into r_next.  The row
// pass then reads c_j from shared memory instead of L2 and needs no launch of
// its own.  r_next must not alias r (other CTAs still read r's rows).
// grid = (1, s * ceil(ceil(n / s) / KR), batch), block = n / (VW CPT).
template <typename T, int KR, int CPT>
__global__ void __launch_bounds__(256) k_st_colrow(const T *__restrict__ r, long r_bs, const T *c_prev, long prev_bs,
                                                   T *c_next, long next_bs, T *__restrict__ w_out, long w_bs,
                                                   T *__restrict__ r_next, long rn_bs, int n, int s, int boundary)
{
    pdl_entry();
    constexpr int VW = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *rows = reinterpret_cast<T *>(smem_raw);  // [KR][n]: c_j of the CTA's rows
    const int r0 = blockIdx.y % s, m = blockIdx.y / s;
    const long b = blockIdx.z;
    const T *rb = r + b * r_bs;
    const int ybase = r0 + s * (m * KR);
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int x = (threadIdx.x + q * blockDim.x) * VW;
        alignas(16) T win[5][VW];
#pragma unroll
        for (int u = 0; u < 4; ++u) ld16(win[u], rb + (long)fold_index(ybase + (u - 2) * s, n, boundary) * n + x);
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int y = ybase + k * s;
            if (y >= n) break;
            ld16(win[(k + 4) % 5], rb + (long)fold_index(y + 2 * s, n, boundary) * n + x);
            const long px = (long)y * n + x;
            alignas(16) T prev[VW]; alignas(16) T cj[VW]; alignas(16) T w[VW];
            ld16(prev, c_prev + b * prev_bs + px);
#pragma unroll
            for (int u = 0; u < VW; ++u) {
                cj[u] = B3<T>::apply(win[k % 5][u], win[(k + 1) % 5][u], win[(k + 2) % 5][u], win[(k + 3) % 5][u],
                                     win[(k + 4) % 5][u]);
                w[u] = prev[u] - cj[u];
            }
            st16cs(w_out + b * w_bs + px, w);
            st16(c_next + b * next_bs + px, cj);
            st16(rows + k * n + x, cj);
        }
    }
    __syncthreads();
    const int s2 = 2 * s;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
        const int x = (threadIdx.x + q * blockDim.x) * VW;
        const bool inner = s2 % VW == 0 && x - 2 * s2 >= 0 && x + VW + 2 * s2 <= n;
#pragma unroll
        for (int k = 0; k < KR; ++k) {
            const int y = ybase + k * s;
            if (y >= n) break;
            const T *row = rows + k * n;
            alignas(16) T o[VW];
            if (inner) {
                alignas(16) T m2[VW]; alignas(16) T m1[VW]; alignas(16) T c0[VW]; alignas(16) T p1[VW];
                alignas(16) T p2[VW];
                ld16(m2, row + x - 2 * s2);
                ld16(m1, row + x - s2);
                ld16(c0, row + x);
                ld16(p1, row + x + s2);
                ld16(p2, row + x + 2 * s2);
#pragma unroll
                for (int u = 0; u < VW; ++u) o[u] = B3<T>::apply(m2[u], m1[u], c0[u], p1[u], p2[u]);
            } else {
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    const int xx = x + u;
                    o[u] = B3<T>::apply(row[fold_index(xx - 2 * s2, n, boundary)],
                                        row[fold_index(xx - s2, n, boundary)], row[xx],
                                        row[fold_index(xx + s2, n, boundary)],
                                        row[fold_index(xx + 2 * s2, n, boundary)]);
                }
            }
            st16(r_next + b * rn_bs + (long)y * n + x, o);
        }
    }
}

// ---------------------------------------------------------------------------
// Large scales a+1..b in two passes.  The row filters X_j and the column
// filters Y_j act on different axes and commute, so
//   c_{a+k} = Y_{a+k} ... Y_{a+1} u_{a+k},  u_{a+k} = X_{a+k} ... X_{a+1} c_a.
// k_st_rows_multi makes every u_{a+k} from full rows of c_a held in shared
// memory (no halo: the row edge folds inside the row); k_st_cols_multi then
// holds full-height strips of W columns, applies the column filters, and
// writes w_{a+k} = c_{a+k-1} - c_{a+k} and the smooth array.

// one CTA per row; u_out[k] = X_{a+k} ... X_{a+1} c_a (rows), k = 1..K
template <typename T>
__global__ void __launch_bounds__(256) k_st_rows_multi(const T *__restrict__ c, long c_bs, T *__restrict__ u_out,
                                                       long u_ks, int n, int a, int K, int boundary)
{
    pdl_entry();
    constexpr int VW = 16 / sizeof(T);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *buf0 = reinterpret_cast<T *>(smem_raw);
    T *buf1 = buf0 + n;
    const long b = blockIdx.y;
    const int y = blockIdx.x;
    const T *src = c + b * c_bs + (long)y * n;
    const long roff = (b * n + y) * (long)n;
    for (int x = threadIdx.x * VW; x < n; x += blockDim.x * VW) {
        alignas(16) T v[VW];
        ld16(v, src + x);
        st16(buf0 + x, v);
    }
    __syncthreads();
    T *in = buf0, *out = buf1;
    for (int k = 1; k <= K; ++k) {
        const int s = 1 << (a + k - 1);
        T *dst = u_out + (long)(k - 1) * u_ks + roff;
        for (int x = threadIdx.x * VW; x < n; x += blockDim.x * VW) {
            alignas(16) T o[VW];
            if (s % VW == 0 && x - 2 * s >= 0 && x + VW + 2 * s <= n) {  // 16-byte aligned taps only
                alignas(16) T m2[VW]; alignas(16) T m1[VW]; alignas(16) T c0[VW]; alignas(16) T p1[VW]; alignas(16) T p2[VW];
                ld16(m2, in + x - 2 * s);
                ld16(m1, in + x - s);
                ld16(c0, in + x);
                ld16(p1, in + x + s);
                ld16(p2, in + x + 2 * s);
#pragma unroll
                for (int u = 0; u < VW; ++u) o[u] = B3<T>::apply(m2[u], m1[u], c0[u], p1[u], p2[u]);
            } else {
#pragma unroll
                for (int u = 0; u < VW; ++u) {
                    const int xx = x + u;
                    o[u] = B3<T>::apply(in[fold_index(xx - 2 * s, n, boundary)], in[fold_index(xx - s, n, boundary)],
                                        in[xx], in[fold_index(xx + s, n, boundary)],
                                        in[fold_index(xx + 2 * s, n, boundary)]);
                }
            }
            st16(out + x, o);
            st16(dst + x, o);
        }
        __syncthreads();
        T *t = in;
        in = out;
        out = t;
    }
}

// one CTA per strip of W columns x n rows, n * (W / VW) / NR threads; a thread
// owns VW adjacent columns of the NR rows y = ty + m n / NR.
template <typename T, int W, int NR>
__global__ void __launch_bounds__(512) k_st_cols_multi(const T *__restrict__ c_a, long ca_bs,
                                                       const T *__restrict__ u_in, long u_ks, T *__restrict__ w_out,
                                                       long w_bs, long w_ss, T *__restrict__ c_out, long c_bs, int n,
                                                       int a, int K, int boundary)
{
    pdl_entry();
    constexpr int VW = 16 / sizeof(T);
    constexpr int QW = W / VW;  // vectors per row of the strip
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *bufA = reinterpret_cast<T *>(smem_raw);
    T *bufB = bufA + (long)n * W;
    const int strips = n / W;
    const long b = blockIdx.x / strips;
    const int x0 = (blockIdx.x % strips) * W;
    const int q = threadIdx.x % QW;
    const int ty = threadIdx.x / QW;
    const int rstep = n / NR;
    const long nn = (long)n * n;
    const int xs = x0 + q * VW;

    alignas(16) T prev[NR][VW];  // c_{a+k-1} at the thread's pixels
#pragma unroll
    for (int m = 0; m < NR; ++m) ld16(prev[m], c_a + b * ca_bs + (long)(ty + m * rstep) * n + xs);

    for (int k = 1; k <= K; ++k) {
        const T *u = u_in + (long)(k - 1) * u_ks + b * nn;
        for (int e = threadIdx.x; e < n * QW; e += blockDim.x) {
            const int yy = e / QW, qq = e % QW;
            alignas(16) T v[VW];
            ld16(v, u + (long)yy * n + x0 + qq * VW);
            st16(bufA + yy * W + qq * VW, v);
        }
        __syncthreads();
        T *in = bufA, *out = bufB;
        for (int p = 1; p <= k; ++p) {
            const int s = 1 << (a + p - 1);
            for (int e = threadIdx.x; e < n * QW; e += blockDim.x) {
                const int yy = e / QW, qq = e % QW;
                alignas(16) T m2[VW]; alignas(16) T m1[VW]; alignas(16) T c0[VW]; alignas(16) T p1[VW]; alignas(16) T p2[VW]; alignas(16) T o[VW];
                ld16(m2, in + fold_index(yy - 2 * s, n, boundary) * W + qq * VW);
                ld16(m1, in + fold_index(yy - s, n, boundary) * W + qq * VW);
                ld16(c0, in + yy * W + qq * VW);
                ld16(p1, in + fold_index(yy + s, n, boundary) * W + qq * VW);
                ld16(p2, in + fold_index(yy + 2 * s, n, boundary) * W + qq * VW);
#pragma unroll
                for (int uu = 0; uu < VW; ++uu) o[uu] = B3<T>::apply(m2[uu], m1[uu], c0[uu], p1[uu], p2[uu]);
                st16(out + yy * W + qq * VW, o);
            }
            __syncthreads();
            T *t = in;
            in = out;
            out = t;
        }
        // in = c_{a+k} on the strip
        const int band = a + k;
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            const int yy = ty + m * rstep;
            alignas(16) T cj[VW]; alignas(16) T w[VW];
            ld16(cj, in + yy * W + q * VW);
#pragma unroll
            for (int uu = 0; uu < VW; ++uu) {
                w[uu] = prev[m][uu] - cj[uu];
                prev[m][uu] = cj[uu];
            }
            const long px = (long)yy * n + xs;
            emit_band<T>(w, w_out + b * w_bs + (long)(band - 1) * w_ss, px, yy, xs, n, true);
        }
        __syncthreads();  // bufA is reloaded next
    }
    if (c_out) {
#pragma unroll
        for (int m = 0; m < NR; ++m) {
            const int yy = ty + m * rstep;
            st16(c_out + b * c_bs + (long)yy * n + xs, prev[m]);
        }
    }
}

// ---------------------------------------------------------------------------
// Scales handled by the fused tile kernel; never more than fit a tile with
// its halo (two buffers) in shared memory.  Automatic choice: see
// starlet_builtin_fuse (measured with the large scales in one pass each; with
// a row and a column pass per large scale it was 0.898 / 0.812 / 0.837 ms for
// 32 x 1024^2 fusing 1 / 2 / 3 scales and 0.489 / 0.451 / 0.446 for 64 x
// 512^2).  An autotuned plan for (n, J, precision) overrides the rule.
static int clamp_fuse(int f, int J, const fm_config &cfg)
{
    const int fmax = cfg.precision == FM_F64 ? 3 : 4;  // tile + halo must fit shared memory
    if (f > fmax) f = fmax;
    if (f > J - 1) f = J - 1;
    return f;
}

// Built-in fused depth: two scales for fp32 maps of 512^2 to 2048^2, three
// otherwise.  With one pass per large scale (KS + starlet per batch, ms,
// fusing 1 / 2 / 3 scales): 64 x 512^2 (J = 7) 0.490 / 0.366 / 0.376, 32 x
// 1024^2 (J = 7) 0.878 / 0.709 / 0.726, 16 x 2048^2 (J = 8) 2.14 / 1.77 /
// 1.80, 16 x 4096^2 (J = 9) 11.9 / 8.28 / 8.24.
int starlet_builtin_fuse(int n, int J, const fm_config &cfg)
{
    if (cfg.fuse_depth < 0) return 0;
    const int f = cfg.fuse_depth != 0 ? cfg.fuse_depth : (cfg.precision == FM_F32 && n >= 512 && n <= 2048 ? 2 : 3);
    return clamp_fuse(f, J, cfg);
}

static int auto_fuse(int n, int J, const fm_config &cfg)
{
    TunedPlan tp;
    if (cfg.fuse_depth == 0 && tune_lookup(n, J, cfg.precision, &tp)) return clamp_fuse(tp.fuse, J, cfg);
    return starlet_builtin_fuse(n, J, cfg);
}

// Large-scale path when cfg.large_path = 0: the autotuned plan's, else one
// pass per scale (k_st_scale) where it applies (n a multiple of 512, large
// scales of spacing 4..128 px; fp32 only, fp64 takes the form 1), else the
// column pass fused with the next row pass on maps up to 256^2 after fused
// small scales, else one row and one column pass per scale.  One pass per
// scale against the row + column pair (KS + starlet per batch, ms): 32 x
// 1024^2 J = 7 0.818 -> 0.715, 16 x 2048^2 J = 8 1.99 -> 1.78, 16 x 4096^2
// J = 9 10.52 -> 8.25, 1 x 8192^2 J = 9 3.16 -> 2.56.
int starlet_builtin_large_path(int n, int J, int fuse)
{
    if (fuse >= 2 && n % 512 == 0 && (1 << (J - 2)) <= 128) return 4;
    return fuse >= 1 && n <= 256 ? 3 : 1;
}

static int resolve_large_path(int n, int J, int f, const fm_config &cfg)
{
    if (cfg.large_path != 0) return cfg.large_path;
    TunedPlan tp;
    if (tune_lookup(n, J, cfg.precision, &tp)) return tp.large_path;
    return starlet_builtin_large_path(n, J, f);
}

// Strip width of the column-strip kernel: 2 n W elements must fit 128 KB.
// 0 = use the one-scale-per-pass kernels instead.
static int cols_multi_width(int n, size_t es)
{
    const int vw = (int)(16 / es);
    if (n < 64 || n % 8) return 0;
    int w = (int)((64 * 1024 / es) / n);
    if (w > 16) w = 16;
    if (w < vw || n % w) return 0;
    return w;
}

int starlet_fuse_depth(int n, int J, const fm_config &cfg) { return auto_fuse(n, J, cfg); }

size_t starlet_scratch_elems(int n, int J, int batch, const fm_config &cfg)
{
    const int f = auto_fuse(n, J, cfg);
    // an automatic depth may follow a table entry that changes before the
    // launch: it gets the two maps of the large-scale passes whenever J > 2
    if (f >= J - 1 && (cfg.fuse_depth != 0 || J == 2)) return 0;
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    const size_t per = (size_t)batch * n * n;
    if (f >= 1 && cfg.large_path == 2 && cols_multi_width(n, es)) return (size_t)(J - f) * per;  // c_f + u's
    return 2 * per;
}

template <typename T, int F, int TS>
static int tile_launch(const T *in, T *w_out, long w_bs, long w_ss, T *c_out, long c_bs, int n, int boundary,
                       int batch, bool vec_ok, cudaStream_t s)
{
    constexpr int H = (1 << (F + 1)) - 2;
    constexpr int HP = ((H + 3) / 4) * 4;
    constexpr int P = TS + 2 * HP;
    const size_t smem = 2ull * P * P * sizeof(T);
    const int tiles_x = (n + TS - 1) / TS;
    const int tiles_per_map = tiles_x * tiles_x;
    auto k = k_st_tile<T, F, TS>;
    FM_CUDA_TRY(fm::smem_attr((const void *)k, smem));
    FM_LAUNCH(FM_K_STARLET_TILE, k, (unsigned)(tiles_per_map * (long)batch), 256, smem, s, in, (long)n * n, w_out,
              w_bs, w_ss, c_out, c_bs, n, boundary, tiles_x, tiles_per_map, vec_ok ? 1 : 0);
    return FM_OK;
}

int starlet_wait_error(bool clear) { return wait_error_flag(clear); }

template <int F>
static int tile32_launch(const float *in, float *w_out, long w_bs, long w_ss, float *c_out, long c_bs, int n,
                         int boundary, int batch, bool vec_ok, int variant, cudaStream_t s)
{
    constexpr int TS = 64;
    constexpr int H = (1 << (F + 1)) - 2;
    constexpr int HP = ((H + 3) / 4) * 4;
    constexpr int P = TS + 2 * HP;
    const size_t smem = 2ull * P * P * sizeof(float);
    const int tiles_x = (n + TS - 1) / TS;
    const int tiles_per_map = tiles_x * tiles_x;
    if (variant == 1) {
        auto k = vec_ok ? k_st_tile32v2<F, true> : k_st_tile32v2<F, false>;
        const size_t smem2 = tile2_smem<F>();
        FM_CUDA_TRY(fm::smem_attr((const void *)k, smem2));
        CUtensorMap map;
        const uint64_t dims[3] = {(uint64_t)n, (uint64_t)n, (uint64_t)batch};
        const uint64_t strides[2] = {(uint64_t)n * 4, (uint64_t)n * n * 4};
        const uint32_t box[3] = {(uint32_t)P, (uint32_t)P, 1};
        int use_tma = (g_use_tma.load(std::memory_order_relaxed) & 1) && vec_ok && n >= 2 * TS + 2 * HP &&
                      encode_map3d_f32(&map, in, dims, strides, box);
        if (use_tma && g_wait_test.load(std::memory_order_relaxed)) use_tma |= 2;
        if (!use_tma) memset(&map, 0, sizeof(map));
        FM_LAUNCH(FM_K_STARLET_TILE, k, (unsigned)(tiles_per_map * (long)batch), 256, smem2, s, in, (long)n * n,
                  w_out, w_bs, w_ss, c_out, c_bs, n, boundary, tiles_x, tiles_per_map, vec_ok ? 1 : 0, map,
                  use_tma);
        return FM_OK;
    }
    FM_CUDA_TRY(fm::smem_attr((const void *)k_st_tile32<F>, smem));
    FM_LAUNCH(FM_K_STARLET_TILE, k_st_tile32<F>, (unsigned)(tiles_per_map * (long)batch), 256, smem, s, in,
              (long)n * n, w_out, w_bs, w_ss, c_out, c_bs, n, boundary, tiles_x, tiles_per_map, vec_ok ? 1 : 0);
    return FM_OK;
}

template <typename T>
static int tile_dispatch(int f, const T *in, T *w_out, long w_bs, long w_ss, T *c_out, long c_bs, int n,
                         int boundary, int batch, bool vec_ok, int variant, cudaStream_t s)
{
    constexpr int TS = sizeof(T) == 4 ? 64 : 32;
    if constexpr (sizeof(T) == 4) {
        const float *fi = (const float *)in;
        float *fw = (float *)w_out, *fc = (float *)c_out;
        switch (f) {
        case 1: return tile32_launch<1>(fi, fw, w_bs, w_ss, fc, c_bs, n, boundary, batch, vec_ok, variant, s);
        case 2: return tile32_launch<2>(fi, fw, w_bs, w_ss, fc, c_bs, n, boundary, batch, vec_ok, variant, s);
        case 3: return tile32_launch<3>(fi, fw, w_bs, w_ss, fc, c_bs, n, boundary, batch, vec_ok, variant, s);
        case 4: return tile32_launch<4>(fi, fw, w_bs, w_ss, fc, c_bs, n, boundary, batch, vec_ok, variant, s);
        }
        return FM_EINVAL;
    }
    switch (f) {
    case 1: return tile_launch<T, 1, TS>(in, w_out, w_bs, w_ss, c_out, c_bs, n, boundary, batch, vec_ok, s);
    case 2: return tile_launch<T, 2, TS>(in, w_out, w_bs, w_ss, c_out, c_bs, n, boundary, batch, vec_ok, s);
    case 3: return tile_launch<T, 3, TS>(in, w_out, w_bs, w_ss, c_out, c_bs, n, boundary, batch, vec_ok, s);
    case 4: return tile_launch<T, 4, TS>(in, w_out, w_bs, w_ss, c_out, c_bs, n, boundary, batch, vec_ok, s);
    }
    return FM_EINVAL;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

template <typename T>
static int starlet_impl(const T *kappa, T *pyr, long pyr_bs, int n, int J, int batch, const fm_config &cfg,
                        T *scratch, cudaStream_t s, bool bands_only)
{
    constexpr int VW = 16 / sizeof(T);
    constexpr int KR = 8;
    const long nn = (long)n * n;
    const int f = auto_fuse(n, J, cfg);
    const int bnd = cfg.boundary;
    T *A = scratch;
    T *Bb = scratch ? scratch + (long)batch * nn : nullptr;
    T *last = pyr + (long)(J - 1) * nn;  // slot of the smooth array
    const bool vec_ok = n % VW == 0 && aligned16(kappa) && aligned16(pyr) && (!scratch || aligned16(scratch));
    if (f >= 1) {
        T *c_out = f == J - 1 ? (bands_only ? nullptr : last) : A;
        const long c_bs = f == J - 1 ? pyr_bs : nn;
        int tvar = g_tile_variant.load(std::memory_order_relaxed);
        if (tvar < 0) {
            TunedPlan tp;
            tvar = tune_lookup(n, J, cfg.precision, &tp) ? tp.tile : 1;
        }
        int st = tile_dispatch<T>(f, kappa, pyr, pyr_bs, nn, c_out, c_bs, n, bnd, batch, vec_ok, tvar, s);
        if (st != FM_OK) return st;
    }
    const int K = J - 1 - f;  // large scales left after the tile kernel
    const int Wc = cols_multi_width(n, sizeof(T));
    const int lpath = resolve_large_path(n, J, f, cfg);
    if (K >= 1 && f >= 1 && Wc && vec_ok && lpath == 2) {
        T *U = A + (long)batch * nn;  // u_{f+1} .. u_{f+K}, each batch * nn
        const size_t rsm = 2ull * n * sizeof(T);
        FM_CUDA_TRY(fm::smem_attr((const void *)k_st_rows_multi<T>, rsm));
        FM_LAUNCH(FM_K_STARLET_ROW, k_st_rows_multi<T>, dim3(n, batch), 256, rsm, s, A, nn, U, (long)batch * nn, n,
                  f, K, bnd);
        constexpr int NR = 8;
        const size_t csm = 2ull * n * Wc * sizeof(T);
        const unsigned cgrid = (unsigned)((long)batch * (n / Wc));
        const int cthreads = n * (Wc / VW) / NR;
#define FM_COLS_MULTI(WW)                                                                                          \
    do {                                                                                                            \
        auto kc = k_st_cols_multi<T, WW, NR>;                                                                       \
        FM_CUDA_TRY(fm::smem_attr((const void *)kc, csm));               \
        FM_LAUNCH(FM_K_STARLET_COL, kc, cgrid, cthreads, csm, s, A, nn, U, (long)batch * nn, pyr, pyr_bs, nn, last,  \
                  pyr_bs, n, f, K, bnd);                                                                           \
    } while (0)
        switch (Wc) {
        case 16: FM_COLS_MULTI(16); break;
        case 8: FM_COLS_MULTI(8); break;
        case 4: FM_COLS_MULTI(4); break;
        case 2:
            if constexpr (VW <= 2) FM_COLS_MULTI(2);
            break;
        }
#undef FM_COLS_MULTI
        return FM_OK;
    }
    if constexpr (sizeof(T) == 4) {
        // large_path 4: one pass per large scale, row filter from shared memory
        const int s_lo = 1 << f, s_hi = 1 << (J - 2);  // spacing of the first and last large scale
        if (K >= 1 && lpath == 4 && vec_ok && n % 512 == 0 && s_lo >= 4 && s_hi <= 128 && Bb) {
            constexpr int KRS = 8;
            // c_j alternates between A and Bb (never in place); the last goes to
            // the smooth-array slot.  Tensor maps first: if the driver refuses
            // one, the two-pass path below runs instead.
            const T *srcs[20];
            T *dsts[20];
            CUtensorMap maps[20];
            bool ok = true;
            const T *src = f >= 1 ? A : kappa;
            for (int j = f + 1; j <= J - 1 && ok; ++j) {
                const int sp = 1 << (j - 1);
                T *dst = j == J - 1 ? (bands_only ? nullptr : last) : (src == Bb ? A : Bb);
                const uint64_t dims[3] = {(uint64_t)(2 * sp), (uint64_t)(n / (2 * sp)), (uint64_t)batch * n};
                const uint64_t str[2] = {(uint64_t)(2 * sp) * 4, (uint64_t)n * 4};
                const uint32_t box[3] = {(uint32_t)(2 * sp), (uint32_t)(256 / sp + 2), 1};
                ok = encode_map3d_f32(&maps[j], src, dims, str, box);
                srcs[j] = src;
                dsts[j] = dst;
                src = dst;
            }
            if (ok) {
                for (int j = f + 1; j <= J - 1; ++j) {
                    const int sp = 1 << (j - 1);
                    const long dst_bs = j == J - 1 ? pyr_bs : nn;
                    // wide halos (s >= 32): 16 output rows a CTA, so that the
                    // window's four extra rows are re-read less often
                    const int kr = sp >= 32 ? 16 : KRS;
                    auto ksc = kr == 16 ? k_st_scale<16> : k_st_scale<KRS>;
                    const size_t ssm = 128 + (size_t)(kr + 4) * ((512 + 4 * sp + 31) & ~31) * sizeof(float);
                    FM_CUDA_TRY(fm::smem_attr((const void *)ksc, ssm));
                    const unsigned gys = (unsigned)(sp * ((((n + sp - 1) / sp) + kr - 1) / kr));
                    FM_LAUNCH(FM_K_STARLET_COL, ksc, dim3(n / 512, gys, batch), 128, ssm, s, (const float *)srcs[j],
                              (float *)dsts[j], dst_bs, (float *)(pyr + (long)(j - 1) * nn), pyr_bs, n, sp, bnd,
                              maps[j]);
                }
                return FM_OK;
            }
        }
    }
    const unsigned gx = (unsigned)((n + 128 * VW - 1) / (128 * VW));
    // row pass: up to 256 threads (1024 fp32 pixels) of one row per CTA, so
    // the taps at +-s, +-2s mostly hit lines the CTA itself brought into L1
    // (128-thread CTAs re-read them from L2: 0.897 -> 0.834 ms per 32-map step)
    const int rt = std::min(256, std::max(32, (n / VW + 31) / 32 * 32));
    const unsigned gxr = (unsigned)((n + rt * VW - 1) / (rt * VW));
    // Column pass of scale j fused with the row pass of j + 1 (large_path 3;
    // automatic after fused small scales on maps up to 256^2): whole rows per
    // CTA, CPT vectors per thread, KRC rows per CTA.  Alone, on a 4-map chunk
    // of 1024^2 fp32, it takes 14.4-15.7 us against 16.4-18.5 us for the two
    // kernels, and the launches' summed event times per 32-map batch drop
    // 0.79 -> 0.70 ms; but in the chunked two-stream pipeline the batch is
    // slower (0.812 -> 0.855 ms; 16 x 2048^2: 2.05 -> 2.46 ms, KRC = 1: 2.27,
    // KRC = 4: 2.68; a dedicated scratch map instead of the smooth-array slot
    // does not help), while 128 x 256^2 gains (0.228 -> 0.222 ms).
    constexpr int KRC = 2;
    const int ct = std::min(256, n / VW);
    const int cpt = ct > 0 && (n / VW) % ct == 0 ? (n / VW) / ct : 0;
    const size_t rsm = (size_t)KRC * n * sizeof(T);
    const bool colrow = vec_ok && (cpt == 1 || cpt == 2 || cpt == 4 || cpt == 8) && rsm <= 64 * 1024 && lpath == 3;
    // r_j lives in Bb; with the fused kernel the row-filtered maps alternate
    // between Bb and the pyramid's smooth-array slot (unused until the last
    // column pass writes c_{J-1} there), placed so that r_{J-1} is in Bb.
    auto r_in_last = [&](int j) { return colrow && (J - 1 - j) % 2 == 1; };
    for (int j = f + 1; j <= J - 1; ++j) {
        const int sp = 1 << (j - 1);
        const T *c_prev = j == 1 ? kappa : A;
        T *c_next = j == J - 1 ? (bands_only ? nullptr : last) : A;
        const long next_bs = j == J - 1 ? pyr_bs : nn;
        T *rj = r_in_last(j) ? last : Bb;
        const long rj_bs = r_in_last(j) ? pyr_bs : nn;
        if (!colrow || j == f + 1)
            FM_LAUNCH(FM_K_STARLET_ROW, k_st_row<T>, dim3(gxr, n, batch), rt, 0, s, c_prev, nn, rj, rj_bs, n, sp, bnd,
                      vec_ok ? 1 : 0);
        if (colrow && j < J - 1) {
            T *rn = r_in_last(j + 1) ? last : Bb;
            const long rn_bs = r_in_last(j + 1) ? pyr_bs : nn;
            const unsigned gyc = (unsigned)(sp * ((((n + sp - 1) / sp) + KRC - 1) / KRC));
#define FM_COLROW(CP)                                                                                               \
    do {                                                                                                            \
        auto kc = k_st_colrow<T, KRC, CP>;                                                                          \
        FM_CUDA_TRY(fm::smem_attr((const void *)kc, rsm));                                                          \
        FM_LAUNCH(FM_K_STARLET_COLROW, kc, dim3(1, gyc, batch), ct, rsm, s, rj, rj_bs, c_prev, nn, c_next, next_bs,  \
                  pyr + (long)(j - 1) * nn, pyr_bs, rn, rn_bs, n, sp, bnd);                                         \
    } while (0)
            switch (cpt) {
            case 1: FM_COLROW(1); break;
            case 2: FM_COLROW(2); break;
            case 4: FM_COLROW(4); break;
            default: FM_COLROW(8); break;
            }
#undef FM_COLROW
            continue;
        }
        const unsigned gy = (unsigned)(sp * ((((n + sp - 1) / sp) + KR - 1) / KR));
        CUtensorMap mr, mp;
        memset(&mr, 0, sizeof(mr));
        memset(&mp, 0, sizeof(mp));
        int tma = 0;
        const int mask = g_use_tma.load(std::memory_order_relaxed);
        // only for maps of 4096^2 and up, whose arrays do not stay in L2: there
        // the copies cut 16 x 4096^2 (J = 9) from 11.75 to 11.40 ms, while on
        // the L2-resident chunks of 1024^2 maps they cost 0.835 -> 0.849 ms
        if (sizeof(T) == 4 && vec_ok && n >= 4096 && n % 512 == 0 && (mask & 24) && rj == Bb) {
            // r and c_{j-1} viewed as {256, n/256, sp, n/sp, batch}: a box picks
            // 512 columns of rows r0 + sp (m0 .. m0 + rows - 1)
            const uint64_t dims[5] = {256, (uint64_t)n / 256, (uint64_t)sp, (uint64_t)(n / sp), (uint64_t)batch};
            const uint64_t str[4] = {1024, (uint64_t)n * 4, (uint64_t)sp * n * 4, (uint64_t)nn * 4};
            const uint32_t box_r[5] = {256, 2, 1, KR + 4, 1}, box_p[5] = {256, 2, 1, KR, 1};
            if ((mask & 8) && encode_map5d_f32(&mr, Bb, dims, str, box_r)) tma |= 1;
            if ((mask & 16) && encode_map5d_f32(&mp, c_prev, dims, str, box_p)) tma |= 2;
        }
        const size_t csm = tma ? 128 + (size_t)(2 * KR + 4) * 512 * sizeof(float) : 0;
        if (tma) FM_CUDA_TRY(fm::smem_attr((const void *)k_st_col<T, KR>, csm));
        FM_LAUNCH(FM_K_STARLET_COL, (k_st_col<T, KR>), dim3(gx, gy, batch), 128, csm, s, rj, rj_bs, c_prev, nn,
                  c_next, next_bs, pyr + (long)(j - 1) * nn, pyr_bs, n, sp, bnd, vec_ok ? 1 : 0, mr, mp, tma);
    }
    return FM_OK;
}

int launch_starlet(const void *kappa, void *pyr, long pyr_bstride, int n, int J, int batch, const fm_config &cfg,
                   void *scratch, cudaStream_t s, bool bands_only)
{
    if (cfg.precision == FM_F64)
        return starlet_impl<double>((const double *)kappa, (double *)pyr, pyr_bstride, n, J, batch, cfg,
                                    (double *)scratch, s, bands_only);
    return starlet_impl<float>((const float *)kappa, (float *)pyr, pyr_bstride, n, J, batch, cfg, (float *)scratch,
                               s, bands_only);
}

}  // namespace fm
