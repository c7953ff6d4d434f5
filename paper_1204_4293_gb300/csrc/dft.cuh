// dft.cuh -- small DFTs held in registers (radix 2, 4, 8; 16 and 32 for
// float2 by the four-step split R = R1 * R2 with constant twiddles).
// Forward kernel exp(-2 pi i m k / R); inverse uses exp(+...).
#pragma once

#include "common.cuh"

namespace fm {

template <bool INV, typename V> __device__ __forceinline__ V mul_minus_i(V a)
{
    // forward: a * (-i); inverse: a * (+i)
    return INV ? cmake<V>(-a.y, a.x) : cmake<V>(a.y, -a.x);
}

template <int R, bool INV, typename V> struct Dft;

template <bool INV, typename V> struct Dft<2, INV, V> {
    __device__ __forceinline__ static void run(V *v)
    {
        V a = cadd(v[0], v[1]);
        V b = csub(v[0], v[1]);
        v[0] = a;
        v[1] = b;
    }
};

template <bool INV, typename V> struct Dft<4, INV, V> {
    __device__ __forceinline__ static void run(V *v)
    {
        V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        V t2 = cadd(v[1], v[3]), t3 = mul_minus_i<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

template <bool INV, typename V> struct Dft<8, INV, V> {
    __device__ __forceinline__ static void run(V *v)
    {
        using T = decltype(V::x);
        const T h = (T)0.70710678118654752440;  // sqrt(1/2)
        V e[4] = {v[0], v[2], v[4], v[6]};
        V o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, INV, V>::run(e);
        Dft<4, INV, V>::run(o);
        // o_k *= W8^k, W8 = exp(-+ i pi / 4)
        o[1] = INV ? cmake<V>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y))
                   : cmake<V>(h * (o[1].x + o[1].y), h * (o[1].y - o[1].x));
        o[2] = mul_minus_i<INV>(o[2]);
        o[3] = INV ? cmake<V>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y))
                   : cmake<V>(h * (o[3].y - o[3].x), -h * (o[3].x + o[3].y));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = cadd(e[k], o[k]);
            v[k + 4] = csub(e[k], o[k]);
        }
    }
};


// W32^m = exp(-2 pi i m / 32), m = 0..31 (cos, -sin of 2 pi m / 32).
static __constant__ float2 c_w32[32] = {
{1.000000000e+00f, -0.000000000e+00f},
{9.807852804e-01f, -1.950903220e-01f},
{9.238795325e-01f, -3.826834324e-01f},
{8.314696123e-01f, -5.555702330e-01f},
{7.071067812e-01f, -7.071067812e-01f},
{5.555702330e-01f, -8.314696123e-01f},
{3.826834324e-01f, -9.238795325e-01f},
{1.950903220e-01f, -9.807852804e-01f},
{6.123233996e-17f, -1.000000000e+00f},
{-1.950903220e-01f, -9.807852804e-01f},
{-3.826834324e-01f, -9.238795325e-01f},
{-5.555702330e-01f, -8.314696123e-01f},
{-7.071067812e-01f, -7.071067812e-01f},
{-8.314696123e-01f, -5.555702330e-01f},
{-9.238795325e-01f, -3.826834324e-01f},
{-9.807852804e-01f, -1.950903220e-01f},
{-1.000000000e+00f, -1.224646799e-16f},
{-9.807852804e-01f, 1.950903220e-01f},
{-9.238795325e-01f, 3.826834324e-01f},
{-8.314696123e-01f, 5.555702330e-01f},
{-7.071067812e-01f, 7.071067812e-01f},
{-5.555702330e-01f, 8.314696123e-01f},
{-3.826834324e-01f, 9.238795325e-01f},
{-1.950903220e-01f, 9.807852804e-01f},
{-1.836970199e-16f, 1.000000000e+00f},
{1.950903220e-01f, 9.807852804e-01f},
{3.826834324e-01f, 9.238795325e-01f},
{5.555702330e-01f, 8.314696123e-01f},
{7.071067812e-01f, 7.071067812e-01f},
{8.314696123e-01f, 5.555702330e-01f},
{9.238795325e-01f, 3.826834324e-01f},
{9.807852804e-01f, 1.950903220e-01f}

};

template <bool INV> __device__ __forceinline__ float2 mul_w32(float2 a, int m)
{
    float2 w = c_w32[m];
    if (INV) w.y = -w.y;
    return cmul(a, w);
}

// R = R1 * R2 <= 32: input index n = R2 n1 + n2, output k = k1 + R1 k2.
// Step 1: length-R1 DFTs over n1 for each n2, times W_R^(n2 k1); step 2:
// length-R2 DFTs over n2 for each k1.
template <int R1, int R2, bool INV> __device__ __forceinline__ void dft_split(float2 *v)
{
    constexpr int R = R1 * R2;
    float2 t[R];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
        float2 a[R1];
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) a[n1] = v[R2 * n1 + n2];
        Dft<R1, INV, float2>::run(a);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) {
            const int m = ((n2 * k1) % R) * (32 / R);
            t[k1 * R2 + n2] = m == 0 ? a[k1] : mul_w32<INV>(a[k1], m);
        }
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 b[R2];
#pragma unroll
        for (int n2 = 0; n2 < R2; ++n2) b[n2] = t[k1 * R2 + n2];
        Dft<R2, INV, float2>::run(b);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
    }
}

template <bool INV> struct Dft<16, INV, float2> {
    __device__ __forceinline__ static void run(float2 *v) { dft_split<4, 4, INV>(v); }
};
template <bool INV> struct Dft<32, INV, float2> {
    __device__ __forceinline__ static void run(float2 *v) { dft_split<4, 8, INV>(v); }
};

}  // namespace fm
