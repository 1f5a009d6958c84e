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
//     radix-16 passes with shared-memory exchanges (rows padded to 257);
//     three blocks per SM (80 registers), so that one block's exchanges and
//     barriers overlap the others' arithmetic.
//   n_fft = 1024 = 32*32: one warp per frame (4 frames per block), radix-32
//     passes, warp-synchronous exchanges only.
//
// Frame f reads input samples f*S - n_ov/2 .. f*S - n_ov/2 + n_fft - 1
// (S = n_fft - n_ov, zero outside the stream) and writes outputs
// f*S .. f*S + S - 1 (clipped to the stream).
#include "fft_dev.h"

namespace {

using namespace fftdev;

// ---------------------------------------------------------------------------
// 4096 points, 256 threads
// ---------------------------------------------------------------------------
template <int SK>
__global__ void __launch_bounds__(256, 3)
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
