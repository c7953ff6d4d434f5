// starlet.cu -- isotropic undecimated (a trous, B3-spline) starlet transform
// (Sec. 3, Sec. 4.2).
//
// Scale j filters c_{j-1} along rows then columns with h = [1,4,6,4,1]/16 at
// taps 0, +-2^(j-1), +-2^j (the B3 two-scale filter with holes) giving c_j,
// and stores the aperture-mass map w_j = c_{j-1} - c_j (theta = 2^j px).
//
// Kernels:
//   st_tile : scales j0..j1 fused on a 2-D tile held in shared memory with a
//             halo of sum_j 2^j pixels per side; reads c_{j0-1} once, writes
//             w_j0..w_j1 and c_j1.  Used for the small scales.
//   st_row  : r = rows-filtered c_{j-1} for one (large) scale.
//   st_col  : c_j = columns-filtered r, w_j = c_{j-1} - c_j; c_j may overwrite
//             c_{j-1} in place (each thread reads and writes only its own
//             pixel of that array).
// In noise mode the band values are not stored; each band's S1 += w and
// S2 += w^2 are accumulated in FP64 instead (Sec. 1).
#include "common.cuh"

namespace fm {

template <typename T> struct B3 {
    // h = [1, 4, 6, 4, 1] / 16
    static constexpr T h0 = (T)0.0625, h1 = (T)0.25, h2 = (T)0.375;
    __device__ __forceinline__ static T apply(T m2, T m1, T c, T p1, T p2)
    {
        return h0 * (m2 + p2) + h1 * (m1 + p1) + h2 * c;
    }
};

__device__ __forceinline__ void acc_band(double *s1, double *s2, long i, double w, bool atomic)
{
    if (atomic) {
        atomicAdd(s1 + i, w);
        atomicAdd(s2 + i, w * w);
    } else {
        s1[i] += w;
        s2[i] += w * w;
    }
}

// ---------------------------------------------------------------------------
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(256) k_st_tile(const T *__restrict__ in, long in_bs, T *__restrict__ w_out, long w_bs,
                                                 long w_ss, T *__restrict__ c_out, long c_bs, int n, int j0, int j1,
                                                 int boundary, int tiles_x, int tiles_per_map, double *__restrict__ acc1,
                                                 double *__restrict__ acc2, int acc_atomic)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *A = reinterpret_cast<T *>(smem_raw);
    const int H = (1 << (j1 + 1)) - (1 << j0);  // sum_{j=j0..j1} 2^j
    const int P = TX + 2 * H;
    const int rows = TY + 2 * H;
    T *Bf = A + rows * P;
    const long b = blockIdx.x / tiles_per_map;
    const int t = blockIdx.x % tiles_per_map;
    const int ty0 = (t / tiles_x) * TY;
    const int tx0 = (t % tiles_x) * TX;
    const T *src = in + b * in_bs;
    const long nn = (long)n * n;

    for (int idx = threadIdx.x; idx < rows * P; idx += blockDim.x) {
        const int i = idx / P, k = idx - (idx / P) * P;
        const int gy = fold_index(ty0 - H + i, n, boundary);
        const int gx = fold_index(tx0 - H + k, n, boundary);
        A[idx] = src[(long)gy * n + gx];
    }
    __syncthreads();

    int halo = H;
    for (int j = j0; j <= j1; ++j) {
        const int s = 1 << (j - 1);
        const int halo2 = halo - 2 * s;
        // rows pass on every still-valid row, narrowing the columns by 2s
        {
            const int r_lo = H - halo, nr = TY + 2 * halo;
            const int c_lo = H - halo2, nc = TX + 2 * halo2;
            for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
                const int i = r_lo + idx / nc, k = c_lo + idx % nc;
                const T *a = A + i * P + k;
                Bf[i * P + k] = B3<T>::apply(a[-2 * s], a[-s], a[0], a[s], a[2 * s]);
            }
        }
        __syncthreads();
        // columns pass, band output, and c_j written back over c_{j-1}
        {
            const int lo = H - halo2, nr = TY + 2 * halo2, nc = TX + 2 * halo2;
            const int sp = s * P;
            for (int idx = threadIdx.x; idx < nr * nc; idx += blockDim.x) {
                const int i = lo + idx / nc, k = lo + idx % nc;
                const T *bp = Bf + i * P + k;
                const T c = B3<T>::apply(bp[-2 * sp], bp[-sp], bp[0], bp[sp], bp[2 * sp]);
                const int oi = i - H, ok = k - H;
                if (oi >= 0 && oi < TY && ok >= 0 && ok < TX) {
                    const int gy = ty0 + oi, gx = tx0 + ok;
                    if (gy < n && gx < n) {
                        const T w = A[i * P + k] - c;
                        const long px = (long)gy * n + gx;
                        if (acc1)
                            acc_band(acc1, acc2, (long)(j - 1) * nn + px, (double)w, acc_atomic != 0);
                        else
                            w_out[b * w_bs + (long)(j - j0) * w_ss + px] = w;
                    }
                }
                A[i * P + k] = c;
            }
        }
        __syncthreads();
        halo = halo2;
    }
    if (c_out) {
        for (int idx = threadIdx.x; idx < TX * TY; idx += blockDim.x) {
            const int oi = idx / TX, ok = idx % TX;
            const int gy = ty0 + oi, gx = tx0 + ok;
            if (gy < n && gx < n) c_out[b * c_bs + (long)gy * n + gx] = A[(H + oi) * P + H + ok];
        }
    }
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_st_row(const T *__restrict__ c, long c_bs, T *__restrict__ r, int n, int s,
                                                int boundary, long total)
{
    const long nn = (long)n * n;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long b = g / nn;
        const long p = g - b * nn;
        const int y = (int)(p / n), x = (int)(p - (long)y * n);
        const T *row = c + b * c_bs + (long)y * n;
        const T v = B3<T>::apply(__ldg(row + fold_index(x - 2 * s, n, boundary)),
                                 __ldg(row + fold_index(x - s, n, boundary)), __ldg(row + x),
                                 __ldg(row + fold_index(x + s, n, boundary)),
                                 __ldg(row + fold_index(x + 2 * s, n, boundary)));
        r[g] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_st_col(const T *__restrict__ r, const T *c_prev, long prev_bs, T *c_next,
                                                long next_bs, T *__restrict__ w_out, long w_bs, int n, int s,
                                                int boundary, long total, int band, double *__restrict__ acc1,
                                                double *__restrict__ acc2, int acc_atomic)
{
    const long nn = (long)n * n;
    for (long g = blockIdx.x * (long)blockDim.x + threadIdx.x; g < total; g += (long)gridDim.x * blockDim.x) {
        const long b = g / nn;
        const long p = g - b * nn;
        const int y = (int)(p / n), x = (int)(p - (long)y * n);
        const T *col = r + b * nn + x;
        const T c = B3<T>::apply(__ldg(col + (long)fold_index(y - 2 * s, n, boundary) * n),
                                 __ldg(col + (long)fold_index(y - s, n, boundary) * n), __ldg(col + (long)y * n),
                                 __ldg(col + (long)fold_index(y + s, n, boundary) * n),
                                 __ldg(col + (long)fold_index(y + 2 * s, n, boundary) * n));
        const T w = c_prev[b * prev_bs + p] - c;
        if (acc1)
            acc_band(acc1, acc2, (long)(band - 1) * nn + p, (double)w, acc_atomic != 0);
        else
            w_out[b * w_bs + p] = w;
        if (c_next) c_next[b * next_bs + p] = c;
    }
}

// ---------------------------------------------------------------------------
// Scales handled by the fused tile kernel: 3 by default; never more than
// fit a 32 x 32 tile with its halo (two buffers) in 200 KB of shared memory.
static int auto_fuse(int J, const fm_config &cfg)
{
    if (cfg.fuse_depth < 0) return 0;
    int f = cfg.fuse_depth == 0 ? 3 : cfg.fuse_depth;
    if (f > J - 1) f = J - 1;
    const size_t es = cfg.precision == FM_F64 ? 8 : 4;
    while (f > 1) {
        const size_t side = 32 + 2 * ((1u << (f + 1)) - 2);
        if (2 * side * side * es <= 200 * 1024) break;
        --f;
    }
    return f;
}

size_t starlet_scratch_elems(int n, int J, int batch, const fm_config &cfg)
{
    const int f = auto_fuse(J, cfg);
    if (f >= J - 1) return 0;
    return 2ull * (size_t)batch * n * n;
}

template <typename T, int TS>
static int tile_launch(const T *in, long in_bs, T *w_out, long w_bs, long w_ss, T *c_out, long c_bs, int n, int j0,
                       int j1, int boundary, int batch, double *acc1, double *acc2, cudaStream_t s)
{
    const int H = (1 << (j1 + 1)) - (1 << j0);
    const size_t smem = 2ull * (TS + 2 * H) * (TS + 2 * H) * sizeof(T);
    const int tiles_x = (n + TS - 1) / TS;
    const int tiles_per_map = tiles_x * tiles_x;
    auto k = k_st_tile<T, TS, TS>;
    FM_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FM_LAUNCH(FM_K_STARLET_TILE, k, (unsigned)(tiles_per_map * (long)batch), 256, smem, s, in, in_bs, w_out, w_bs,
              w_ss, c_out, c_bs, n, j0, j1, boundary, tiles_x, tiles_per_map, acc1, acc2, batch > 1 ? 1 : 0);
    return FM_OK;
}

static unsigned grid_for(long total)
{
    long g = (total + 255) / 256;
    const long cap = 152L * 16;
    return (unsigned)(g < cap ? g : cap);
}

template <typename T>
static int starlet_impl(const T *kappa, T *pyr, long pyr_bs, int n, int J, int batch, const fm_config &cfg,
                        T *scratch, double *acc1, double *acc2, cudaStream_t s)
{
    const long nn = (long)n * n;
    const int f = auto_fuse(J, cfg);
    const int bnd = cfg.boundary;
    T *A = scratch;
    T *Bb = scratch ? scratch + (long)batch * nn : nullptr;
    const bool noise = acc1 != nullptr;
    T *last = noise ? nullptr : pyr + (long)(J - 1) * nn;  // slot of the smooth array
    if (f >= 1) {
        T *c_out = f == J - 1 ? last : A;
        const long c_bs = f == J - 1 ? pyr_bs : nn;
        const int H = (1 << (f + 1)) - 2;
        const size_t smem64 = 2ull * (64 + 2 * H) * (64 + 2 * H) * sizeof(T);
        int st = smem64 <= 200 * 1024
                     ? tile_launch<T, 64>(kappa, nn, pyr, pyr_bs, nn, c_out, c_bs, n, 1, f, bnd, batch, acc1, acc2, s)
                     : tile_launch<T, 32>(kappa, nn, pyr, pyr_bs, nn, c_out, c_bs, n, 1, f, bnd, batch, acc1, acc2, s);
        if (st != FM_OK) return st;
    }
    const long total = (long)batch * nn;
    for (int j = f + 1; j <= J - 1; ++j) {
        const int sp = 1 << (j - 1);
        const T *c_prev = j == 1 ? kappa : A;
        T *c_next = j == J - 1 ? last : A;
        const long next_bs = j == J - 1 ? pyr_bs : nn;
        FM_LAUNCH(FM_K_STARLET_ROW, k_st_row<T>, grid_for(total), 256, 0, s, c_prev, nn, Bb, n, sp, bnd, total);
        FM_LAUNCH(FM_K_STARLET_COL, k_st_col<T>, grid_for(total), 256, 0, s, Bb, c_prev, nn, c_next, next_bs,
                  noise ? nullptr : pyr + (long)(j - 1) * nn, pyr_bs, n, sp, bnd, total, j, acc1, acc2,
                  batch > 1 ? 1 : 0);
    }
    return FM_OK;
}

int launch_starlet(const void *kappa, void *pyr, long pyr_bstride, int n, int J, int batch, const fm_config &cfg,
                   void *scratch, double *acc_s1, double *acc_s2, cudaStream_t s)
{
    if (cfg.precision == FM_F64)
        return starlet_impl<double>((const double *)kappa, (double *)pyr, pyr_bstride, n, J, batch, cfg,
                                    (double *)scratch, acc_s1, acc_s2, s);
    return starlet_impl<float>((const float *)kappa, (float *)pyr, pyr_bstride, n, J, batch, cfg, (float *)scratch,
                               acc_s1, acc_s2, s);
}

}  // namespace fm
