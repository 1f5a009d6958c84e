// Radix-16/32 FFT building blocks shared by the overlap-save kernels
// (chromatic-dispersion compensation, Kramers-Kronig Hilbert transform):
// register-resident 4-, 16- and 32-point DFTs with compile-time twiddles,
// and table twiddles exp(-/+ 2 pi i e / N).
#pragma once

#include "rx_internal.h"

namespace fftdev {

// cos / sin of 2*pi*e/32
constexpr float kC32[8] = {1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f,
                                      8.314696123e-01f, 7.071067812e-01f, 5.555702330e-01f,
                                      3.826834324e-01f, 1.950903220e-01f};

// exp(-/+ 2 pi i e / 32) * v  (INV: +)
template <int E, bool INV>
__device__ __forceinline__ float2 tw32(float2 v) {
    constexpr int e = E & 31;
    if constexpr (e == 0) return v;
    else if constexpr (e == 8) return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    else if constexpr (e == 16) return make_float2(-v.x, -v.y);
    else if constexpr (e == 24) return INV ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    else {
        // cos(2 pi e/32), sin(2 pi e/32) from the first-octant table
        constexpr int q = e / 8, r = e % 8;
        constexpr float c0 = kC32[r];
        constexpr float s0 = (r == 0) ? 0.f : kC32[8 - r];
        constexpr float c = (q == 0) ? c0 : (q == 1) ? -s0 : (q == 2) ? -c0 : s0;
        constexpr float s = (q == 0) ? s0 : (q == 1) ? c0 : (q == 2) ? -s0 : -c0;
        // forward: (c - i s) v ; inverse: (c + i s) v
        if (INV) return make_float2(c * v.x - s * v.y, c * v.y + s * v.x);
        return make_float2(c * v.x + s * v.y, c * v.y - s * v.x);
    }
}

template <bool INV>
__device__ __forceinline__ float2 mul_mj(float2 v) {   // * (-i) forward, * (+i) inverse
    return INV ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2 &a, float2 &b, float2 &c, float2 &d) {
    float2 t0 = cadd(a, c), t1 = csub(a, c), t2 = cadd(b, d), t3 = mul_mj<INV>(csub(b, d));
    a = cadd(t0, t2);
    c = csub(t0, t2);
    b = cadd(t1, t3);
    d = csub(t1, t3);
}

// 16-point DFT of in[0..15] (stride IS in the array), natural-order output
template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
    // X[k1 + 4 k2] = sum_n0 W4^{n0 k2} W16^{n0 k1} sum_n1 x[n0 + 4 n1] W4^{n1 k1}
#pragma unroll
    for (int n0 = 0; n0 < 4; ++n0) dft4<INV>(v[n0], v[n0 + 4], v[n0 + 8], v[n0 + 12]);
    // v[n0 + 4 k1] now holds the inner sum; twiddle W16^{n0 k1} = W32^{2 n0 k1}
    v[5] = tw32<2, INV>(v[5]);   v[6] = tw32<4, INV>(v[6]);   v[7] = tw32<6, INV>(v[7]);
    v[9] = tw32<4, INV>(v[9]);   v[10] = tw32<8, INV>(v[10]); v[11] = tw32<12, INV>(v[11]);
    v[13] = tw32<6, INV>(v[13]); v[14] = tw32<12, INV>(v[14]); v[15] = tw32<18, INV>(v[15]);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
    // v[k2 + 4 k1] = X[k1 + 4 k2]: transpose the 4x4 index
    float2 o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = v[k2 + 4 * k1];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
}

// 32-point DFT: two 16-point DFTs of the even and odd samples, then radix 2.
template <bool INV>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
    float2 e[16], o[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    dft16<INV>(e);
    dft16<INV>(o);
    o[1] = tw32<1, INV>(o[1]);   o[2] = tw32<2, INV>(o[2]);   o[3] = tw32<3, INV>(o[3]);
    o[4] = tw32<4, INV>(o[4]);   o[5] = tw32<5, INV>(o[5]);   o[6] = tw32<6, INV>(o[6]);
    o[7] = tw32<7, INV>(o[7]);   o[8] = tw32<8, INV>(o[8]);   o[9] = tw32<9, INV>(o[9]);
    o[10] = tw32<10, INV>(o[10]); o[11] = tw32<11, INV>(o[11]); o[12] = tw32<12, INV>(o[12]);
    o[13] = tw32<13, INV>(o[13]); o[14] = tw32<14, INV>(o[14]); o[15] = tw32<15, INV>(o[15]);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 16] = csub(e[k], o[k]);
    }
}

__device__ __forceinline__ float2 twid(const float2 *__restrict__ tw, int e, int mask, bool inv) {
    float2 w = __ldg(tw + (e & mask));   // w = exp(-2 pi i e / N)
    return inv ? make_float2(w.x, -w.y) : w;
}

}  // namespace fftdev
