// A1: overlap-save chromatic-dispersion compensation.
//
// Each CUDA block filters overlap-save frames of one polarisation of one
// stream entirely on chip: load n_fft samples, forward FFT, multiply by the
// receiver response conj(H_CD) * H_MF (pre-scaled by 1/n_fft), inverse FFT,
// store the n_fft - n_ov centre samples (Sec. 2 runs its static equaliser as
// an FFT pair in the same way).  The forward FFT leaves its output in a
// digit order that the inverse FFT consumes directly, so no reordering pass
// is needed; the spectral multiply reads H at the matching natural index.
//
//   n_fft = 4096 = 16*16*16: 256 threads, 16 points per thread in registers,
//     radix-16 passes with shared-memory exchanges (rows padded to 257).
//   n_fft = 1024 = 32*32: one warp per frame (4 frames per block), radix-32
//     passes, warp-synchronous exchanges only.
//
// Frame f reads input samples f*S - n_ov/2 .. f*S - n_ov/2 + n_fft - 1
// (S = n_fft - n_ov, zero outside the stream) and writes outputs
// f*S .. f*S + S - 1 (clipped to the stream).
#include "rx_internal.h"

namespace {

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

// ---------------------------------------------------------------------------
// 4096 points, 256 threads
// ---------------------------------------------------------------------------
template <int SK>
__global__ void __launch_bounds__(256, 2)
cdc4096_kernel(const float2 *__restrict__ in, typename Store<SK>::T *__restrict__ out, long ns, int S, int half,
               long f0, const float2 *__restrict__ H, const float2 *__restrict__ tw) {
    constexpr int RP = 257;   // padded row
    __shared__ float2 sm[16 * RP];
    const int t = threadIdx.x;
    const long f = f0 + blockIdx.x;
    const float2 *src = in + (long)blockIdx.y * ns;
    typename Store<SK>::T *dst = out + (long)blockIdx.y * ns;
    const long start = f * S - half;
    float2 v[16];

    // stage 1: thread n2 = t holds x[n2 + 256 n1], DFT over n1 -> k1
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        long idx = start + t + 256 * i;
        v[i] = (idx >= 0 && idx < ns) ? src[idx] : make_float2(0.f, 0.f);
    }
    dft16<false>(v);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) v[k1] = cmul(v[k1], twid(tw, t * k1, 4095, false));
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) sm[k1 * RP + t] = v[k1];
    __syncthreads();

    // stage 2: thread (k1, n2a), DFT over n2b -> k2a, twiddle W256^{n2a k2a}
    {
        const int k1 = t >> 4, n2a = t & 15;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[k1 * RP + n2a + 16 * i];
        dft16<false>(v);
#pragma unroll
        for (int k2a = 1; k2a < 16; ++k2a) v[k2a] = cmul(v[k2a], twid(tw, 16 * n2a * k2a, 4095, false));
        __syncthreads();
#pragma unroll
        for (int k2a = 0; k2a < 16; ++k2a) sm[k1 * RP + 16 * k2a + n2a] = v[k2a];
        __syncthreads();
    }
    // stage 3: thread (k1 = t & 15, k2a = t >> 4), DFT over n2a -> k2b
    {
        const int k1 = t & 15, k2a = t >> 4;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[k1 * RP + 16 * k2a + i];
        dft16<false>(v);
        // X[k1 + 16 k2a + 256 k2b] = X[t + 256 k2b]
#pragma unroll
        for (int k2b = 0; k2b < 16; ++k2b) v[k2b] = cmul(v[k2b], __ldg(H + t + 256 * k2b));
        // inverse of stage 3: over k2b -> n2a, twiddle W256^{-n2a k2a}
        dft16<true>(v);
#pragma unroll
        for (int n2a = 1; n2a < 16; ++n2a) v[n2a] = cmul(v[n2a], twid(tw, 16 * n2a * k2a, 4095, true));
        __syncthreads();
#pragma unroll
        for (int n2a = 0; n2a < 16; ++n2a) sm[k1 * RP + 16 * k2a + n2a] = v[n2a];
        __syncthreads();
    }
    // inverse of stage 2: thread (k1, n2a), over k2a -> n2b, twiddle W4096^{-n2 k1}
    {
        const int k1 = t >> 4, n2a = t & 15;
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = sm[k1 * RP + 16 * i + n2a];
        dft16<true>(v);
#pragma unroll
        for (int n2b = 0; n2b < 16; ++n2b) {
            const int n2 = n2a + 16 * n2b;
            if (k1 != 0) v[n2b] = cmul(v[n2b], twid(tw, n2 * k1, 4095, true));
        }
        __syncthreads();
#pragma unroll
        for (int n2b = 0; n2b < 16; ++n2b) sm[k1 * RP + n2a + 16 * n2b] = v[n2b];
        __syncthreads();
    }
    // inverse of stage 1: thread n2 = t, over k1 -> n1: y[t + 256 n1]
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = sm[i * RP + t];
    dft16<true>(v);
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) {
        const int pos = t + 256 * n1;
        if (pos >= half && pos < half + S) {
            long o = f * S + (pos - half);
            if (o < ns) Store<SK>::st(dst, o, v[n1]);
        }
    }
}

// ---------------------------------------------------------------------------
// 1024 points, one warp per frame
// ---------------------------------------------------------------------------
template <int SK>
__global__ void __launch_bounds__(128)
cdc1024_kernel(const float2 *__restrict__ in, typename Store<SK>::T *__restrict__ out, long ns, int S, int half,
               long f0, long f1, const float2 *__restrict__ H, const float2 *__restrict__ tw) {
    constexpr int RP = 33;
    __shared__ float2 smem[4][32 * RP];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const long f = f0 + (long)blockIdx.x * 4 + w;
    if (f >= f1) return;
    float2 *sm = smem[w];
    const float2 *src = in + (long)blockIdx.y * ns;
    typename Store<SK>::T *dst = out + (long)blockIdx.y * ns;
    const long start = f * S - half;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        long idx = start + l + 32 * i;
        v[i] = (idx >= 0 && idx < ns) ? src[idx] : make_float2(0.f, 0.f);
    }
    // lane n2 = l: DFT over n1 -> k1, twiddle W1024^{n2 k1}
    dft32<false>(v);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmul(v[k1], twid(tw, l * k1, 1023, false));
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) sm[k1 * RP + l] = v[k1];
    __syncwarp();
    // lane k1 = l: DFT over n2 -> k2: X[l + 32 k2]
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = sm[l * RP + i];
    dft32<false>(v);
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) v[k2] = cmul(v[k2], __ldg(H + l + 32 * k2));
    // inverse: over k2 -> n2, twiddle W1024^{-n2 k1}
    dft32<true>(v);
    if (l != 0) {
#pragma unroll
        for (int n2 = 1; n2 < 32; ++n2) v[n2] = cmul(v[n2], twid(tw, n2 * l, 1023, true));
    }
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) sm[l * RP + n2] = v[n2];
    __syncwarp();
    // lane n2 = l: over k1 -> n1: y[l + 32 n1]
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = sm[i * RP + l];
    dft32<true>(v);
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) {
        const int pos = l + 32 * n1;
        if (pos >= half && pos < half + S) {
            long o = f * S + (pos - half);
            if (o < ns) Store<SK>::st(dst, o, v[n1]);
        }
    }
}



template <int SK>
cudaError_t cdc_t(const float2 *in, void *out, long ns, int n_streams2, int n_fft, int S, int half, long f0,
                  long f1, const float2 *H, const float2 *tw, cudaStream_t st) {
    auto *o = static_cast<typename Store<SK>::T *>(out);
    if (n_fft == 4096) {
        dim3 grid((unsigned)(f1 - f0), (unsigned)n_streams2);
        cdc4096_kernel<SK><<<grid, 256, 0, st>>>(in, o, ns, S, half, f0, H, tw);
    } else if (n_fft == 1024) {
        dim3 grid((unsigned)((f1 - f0 + 3) / 4), (unsigned)n_streams2);
        cdc1024_kernel<SK><<<grid, 128, 0, st>>>(in, o, ns, S, half, f0, f1, H, tw);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_cdc(const float2 *in, void *out, long ns, int n_streams2, int n_fft,
                       int n_ov, const float2 *H, const float2 *tw, cudaStream_t st, long f0, long f1, int sk) {
    const int S = n_fft - n_ov, half = n_ov / 2;
    const long nframes = (ns + S - 1) / S;
    if (f1 < 0 || f1 > nframes) f1 = nframes;
    if (f0 < 0) f0 = 0;
    if (f1 <= f0 || n_streams2 <= 0) return cudaSuccess;
    switch (sk) {
        case SK_F32: return cdc_t<SK_F32>(in, out, ns, n_streams2, n_fft, S, half, f0, f1, H, tw, st);
        case SK_F16: return cdc_t<SK_F16>(in, out, ns, n_streams2, n_fft, S, half, f0, f1, H, tw, st);
        case SK_BF16: return cdc_t<SK_BF16>(in, out, ns, n_streams2, n_fft, S, half, f0, f1, H, tw, st);
        default: return cudaErrorInvalidValue;
    }
}
