// Kramers-Kronig front-end (Sec. 2: ADC codes to floating point with the DC
// term added back, square root and logarithm, a frequency-domain Hilbert
// transform by an overlap-save FFT pair, field reconstruction and
// downconversion), one kernel.
//
// For a minimum-phase field E = A + s e^{-j 2 pi fc n} (signal below the
// carrier) ln E has only negative-frequency content, so the phase is
// phi = IFFT(G FFT(ln|E|)), G = +j on positive bins, -j on negative bins, 0
// at DC and N/2.  phi is real and G maps real sequences to real sequences,
// so one complex FFT pair carries two streams at once: z = l_a + j l_b
// (l = log2|E| = log2(I)/2, the ln 2 folded into G), and IFFT(G FFT(z)) =
// phi_a + j phi_b.  The DC bin of FFT(z) gives each stream's frame mean of
// l, whose 2^ is the carrier amplitude A removed from the field:
// s = (sqrt(I) e^{j phi} - A) e^{j 2 pi fc n}.
//
// One warp per 1024-point frame (radix 32 x 32 in registers, warp-synchronous
// exchanges through padded shared memory), four frames per block sharing one
// staged span of log2|E|, one stream pair per grid row.  Frame f reads
// samples f*step - n_ov/2 .. + 1023 (code 0, i.e. intensity = DC term,
// outside the stream) and writes outputs f*step .. f*step + step - 1.
#include "k_kk.h"

#include <atomic>

#include "fft_dev.h"

namespace {

using namespace fftdev;

// l2 = log2|E| = log2(I) / 2 (base 2: the Hilbert transform is linear, so
// phi = ln 2 * H{l2}, folded into the spectral gain)
__device__ __forceinline__ float kk_log2_amp(int code, float2 lv, float floor_) {
    return 0.5f * log2f(fmaxf(fmaf(lv.x, (float)code, lv.y), floor_));
}

// Four consecutive frames per block (one warp each).  The block first
// stages l = log2|E| of both streams over the samples its frames read,
// span = 3 step + 1024 (each sample's logarithm taken once per block, the
// codes read with 16-byte loads where aligned), then every warp runs its
// frame's FFT pair from shared memory and rebuilds the field from the staged
// l: s = (2^l e^{j phi} - A) e^{j theta}, theta = 2 pi u / 2^32.
__global__ void __launch_bounds__(128, 4)
kk1024_kernel(const int16_t *__restrict__ codes, float2 *__restrict__ out, long ns, int step, int half, long f0,
              long f1, const __grid_constant__ KKDev p, const float2 *__restrict__ tw) {
    constexpr int N = 1024, RP = 33;
    extern __shared__ __align__(16) float kk_smem[];
    const int span = 3 * step + N, span_pad = (span + 3) & ~3;
    float *la = kk_smem, *lb = kk_smem + span_pad;                      // staged l of both streams
    float2 *xch = reinterpret_cast<float2 *>(kk_smem + 2 * span_pad);   // [4][32 * RP] exchanges
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const long F0 = f0 + (long)blockIdx.x * 4;
    const int sa = 2 * blockIdx.y, sb = sa + 1;
    const bool has_b = sb < p.n_streams;
    const float2 lva = p.lv[sa], lvb = has_b ? p.lv[sb] : make_float2(0.f, 1.f);
    const int16_t *ca = codes + (long)sa * ns;
    const int16_t *cb = codes + (long)(has_b ? sb : sa) * ns;
    const long base = F0 * step - half;
    // stage: chunks of 8 samples; a 16-byte load where the chunk lies in the
    // stream and is 16-byte aligned, element loads (0 outside) otherwise
    const bool vec_ok = ((ns & 7) == 0) && ((base & 7) == 0) && ((reinterpret_cast<uintptr_t>(codes) & 15) == 0);
    for (int c = threadIdx.x; c * 8 < span; c += 128) {
        const long g = base + 8 * c;
        const bool vec = vec_ok && g >= 0 && g + 8 <= ns && 8 * c + 8 <= span;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int16_t *cq = q ? cb : ca;
            const float2 lv = q ? lvb : lva;
            float *dq = q ? lb : la;
            const bool use = q == 0 || has_b;
            int qv[8];
            if (vec) {
                const int4 x = use ? __ldg(reinterpret_cast<const int4 *>(cq + g)) : make_int4(0, 0, 0, 0);
                const int wv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    qv[2 * e] = (int)(int16_t)(wv[e] & 0xffff);
                    qv[2 * e + 1] = wv[e] >> 16;
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const long idx = g + e;
                    qv[e] = (use && idx >= 0 && idx < ns) ? (int)cq[idx] : 0;
                }
            }
            float y[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) y[e] = kk_log2_amp(qv[e], lv, p.floor);
            if (8 * c + 8 <= span) {
                // 16-byte aligned: the staged rows start at multiples of 4 floats
                float4 *d4 = reinterpret_cast<float4 *>(dq + 8 * c);
                d4[0] = make_float4(y[0], y[1], y[2], y[3]);
                d4[1] = make_float4(y[4], y[5], y[6], y[7]);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (8 * c + e < span) dq[8 * c + e] = y[e];
            }
        }
    }
    __syncthreads();
    const long f = F0 + w;
    if (f >= f1) return;
    float2 *sm = xch + w * 32 * RP;
    const int o = w * step;                     // the frame's offset in the staged span
    const long start = f * step - half;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = make_float2(la[o + l + 32 * i], lb[o + l + 32 * i]);
    // lane n2 = l: DFT over n1 -> k1, twiddle W1024^{n2 k1}
    dft32<false>(v);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) v[k1] = cmul(v[k1], twid(tw, l * k1, 1023, false));
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) sm[k1 * RP + l] = v[k1];
    __syncwarp();
    // lane k1 = l: DFT over n2 -> k2: Z[l + 32 k2]
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = sm[l * RP + i];
    dft32<false>(v);
    // frame means of l_a, l_b from Z[0] (lane 0, k2 = 0)
    const float2 z0 = make_float2(__shfl_sync(0xffffffffu, v[0].x, 0), __shfl_sync(0xffffffffu, v[0].y, 0));
    // G ln2 / N: +j for 0 < k < N/2, -j for N/2 < k < N, 0 at 0 and N/2
    constexpr float inv = 1.f / N, g = 0.693147180559945309f / N;
#pragma unroll
    for (int k2 = 0; k2 < 32; ++k2) {
        const int k = l + 32 * k2;
        const float2 z = v[k2];
        if (k == 0 || k == N / 2) v[k2] = make_float2(0.f, 0.f);
        else if (k < N / 2) v[k2] = make_float2(-z.y * g, z.x * g);
        else v[k2] = make_float2(z.y * g, -z.x * g);
    }
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
    // lane n2 = l: over k1 -> n1: (phi_a, phi_b) at frame position l + 32 n1
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = sm[i * RP + l];
    dft32<true>(v);
    // phases back to the exchange buffer by frame position, then the kept
    // positions in a rolled loop (one copy of the epilogue's code)
    __syncwarp();
#pragma unroll
    for (int n1 = 0; n1 < 32; ++n1) sm[n1 * RP + l] = v[n1];
    __syncwarp();
    const float Aa = exp2f(z0.x * inv), Ab = exp2f(z0.y * inv);
    float2 *oa = out + (long)sa * ns;
    float2 *ob = out + (long)sb * ns;
    // e^{j phi} by the hardware sine / cosine: absolute error about 5e-7 for
    // |phi| <= pi, growing in proportion to |phi| beyond (the phase leaves
    // (-pi/2, pi/2) only where the field violates the minimum-phase condition)
    // downconversion e^{j theta}, theta = 2 pi u / 2^32, u = fc_step * n mod
    // 2^32: sincospi at the lane's first kept position, then a rotation by
    // e^{j 2 pi 32 fc} per step of 32 positions (at most 31 steps)
    float sd, cd, sr, cr;
    {
        const long n0 = start + half + l;
        sincospif((float)(int32_t)((uint32_t)n0 * p.fc_step) * 4.656612873e-10f, &sd, &cd);   // 2^-31
        sincospif((float)(int32_t)(32u * p.fc_step) * 4.656612873e-10f, &sr, &cr);
    }
#pragma unroll 1
    for (int pos = half + l; pos < half + step; pos += 32) {
        const long n = start + pos;
        if (n >= ns) break;
        const float2 ph = sm[(pos >> 5) * RP + (pos & 31)];
        {
            const float a = exp2f(la[o + pos]);
            float sp, cp;
            __sincosf(ph.x, &sp, &cp);
            const float ex = a * cp - Aa, ey = a * sp;
            oa[n] = make_float2(ex * cd - ey * sd, ex * sd + ey * cd);
        }
        if (has_b) {
            const float a = exp2f(lb[o + pos]);
            float sp, cp;
            __sincosf(ph.y, &sp, &cp);
            const float ex = a * cp - Ab, ey = a * sp;
            ob[n] = make_float2(ex * cd - ey * sd, ex * sd + ey * cd);
        }
        const float c2 = cd * cr - sd * sr;
        sd = fmaf(sd, cr, cd * sr);
        cd = c2;
    }
}

}  // namespace

cudaError_t launch_kk(const int16_t *codes, float2 *out, long ns, int n_ov, const KKDev &p, const float2 *tw,
                      cudaStream_t st, long f0, long f1) {
    constexpr int N = 1024;
    if (n_ov <= 0 || n_ov >= N || (n_ov & 1)) return cudaErrorInvalidValue;
    if (p.n_streams <= 0 || p.n_streams > kKKMaxStreams) return cudaErrorInvalidValue;
    const int step = N - n_ov, half = n_ov / 2;
    const long nframes = (ns + step - 1) / step;
    if (f1 < 0 || f1 > nframes) f1 = nframes;
    if (f0 < 0) f0 = 0;
    if (f1 <= f0 || ns <= 0) return cudaSuccess;
    const size_t smem = sizeof(float) * 2 * ((3 * step + N + 3) & ~3) + sizeof(float2) * 4 * 32 * 33;
    // > 48 KB of dynamic shared memory needs the opt-in, once per device
    static std::atomic<unsigned long long> attr_done{0};   // bit d: set on device d
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 64 || !((attr_done.load(std::memory_order_relaxed) >> dev) & 1ull)) {
        e = cudaFuncSetAttribute(kk1024_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(float) * 2 * ((3 * 1022 + N + 3) & ~3) + sizeof(float2) * 4 * 32 * 33));
        if (e != cudaSuccess) return e;
        if (dev < 64) attr_done.fetch_or(1ull << dev, std::memory_order_relaxed);
    }
    dim3 grid((unsigned)((f1 - f0 + 3) / 4), (unsigned)((p.n_streams + 1) / 2));
    kk1024_kernel<<<grid, 128, smem, st>>>(codes, out, ns, step, half, f0, f1, p, tw);
    return cudaGetLastError();
}
