// Static frequency-domain equaliser (Sec. 2: 203 taps optimised offline
// from a training sequence whenever acquisition starts, applied by an FFT
// pair that also resamples from 4 to 2 samples per symbol).
//
// Training, in float64: the regularised least-squares normal equations over
// the symbol instants, their Cholesky solution in one block, and the
// equaliser's response on the output band.
//
// Application: one warp per overlap-save frame of 1024 input samples.  The
// forward 1024-point FFT is the radix 32 x 32 of the CDC kernel; of its
// output lane l holds bins l + 32 k2, and the output band (k < 256 or
// k >= 768) is k2 < 8 or k2 >= 24, i.e. the 512-point spectrum index
// k' = l + 32 k2' (k2' = k2, or k2 - 16).  The inverse is a 512-point FFT
// at the output rate, m = m1 + 16 m2:
//   y[m] = sum_l e^{j 2 pi l m2/32} e^{j 2 pi l m1/512} sum_k2' Y[l + 32 k2'] e^{j 2 pi k2' m1/16}
// the inner 16-point DFTs in registers (one per lane), then for each m1 a
// 32-point DFT over l split into even / odd l (lanes m1 and m1 + 16, 16
// points each) joined by one radix-2 step through a shuffle.
#include "k_fde.h"

#include "fft_dev.h"

namespace {

using namespace fftdev;

__device__ __forceinline__ double2 dconj_mul(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// One block per row t; threads over the columns t'.  u_{i,t} is the same
// for all threads of the block (a broadcast load), u_{i,t'} runs over
// consecutive samples.  Products of float32 values are exact in float64.
__global__ void __launch_bounds__(256)
fde_corr_kernel(const float2 *__restrict__ x, long n, const float2 *__restrict__ d, int K, int T, int sps,
                double2 *__restrict__ R, double2 *__restrict__ p) {
    const int t = blockIdx.x, D = (T - 1) / 2;
    for (int t2 = threadIdx.x; t2 <= T; t2 += blockDim.x) {
        // t2 == T: the right-hand side p[t]
        double ax = 0.0, ay = 0.0;
        for (int i = 0; i < K; ++i) {
            const long na = (long)sps * i + D - t;
            if (na < 0 || na >= n) continue;
            const float2 ua = x[na];
            float2 ub;
            if (t2 < T) {
                const long nb = (long)sps * i + D - t2;
                if (nb < 0 || nb >= n) continue;
                ub = x[nb];
            } else {
                ub = d[i];
            }
            ax = fma((double)ua.x, (double)ub.x, fma((double)ua.y, (double)ub.y, ax));
            ay = fma((double)ua.x, (double)ub.y, fma(-(double)ua.y, (double)ub.x, ay));
        }
        if (t2 < T) R[(long)t * T + t2] = make_double2(ax, ay);
        else p[t] = make_double2(ax, ay);
    }
}

// Cholesky R + lam I = L L^H in place (lower triangle, row-major), then
// L y = p and L^H h = y; one block, barriers between the column steps.
__global__ void __launch_bounds__(1024)
fde_solve_kernel(double2 *__restrict__ A, const double2 *__restrict__ p, double2 *__restrict__ y, int T,
                 double delta, double2 *__restrict__ h) {
    __shared__ double red[32];
    __shared__ double s_lam;
    const int tid = threadIdx.x, nt = blockDim.x;
    double tr = 0.0;
    for (int t = tid; t < T; t += nt) tr += A[(long)t * T + t].x;
    for (int o = 16; o > 0; o >>= 1) tr += __shfl_down_sync(0xffffffffu, tr, o);
    if ((tid & 31) == 0) red[tid >> 5] = tr;
    __syncthreads();
    if (tid == 0) {
        double s = 0.0;
        for (int w = 0; w < nt / 32; ++w) s += red[w];
        s_lam = delta * s / T;
    }
    __syncthreads();
    for (int t = tid; t < T; t += nt) {
        A[(long)t * T + t].x += s_lam;
        y[t] = p[t];
    }
    __syncthreads();
    for (int j = 0; j < T; ++j) {
        if (tid == 0) A[(long)j * T + j] = make_double2(sqrt(A[(long)j * T + j].x), 0.0);
        __syncthreads();
        const double ljj = A[(long)j * T + j].x;
        for (int i = j + 1 + tid; i < T; i += nt) {
            double2 &a = A[(long)i * T + j];
            a.x /= ljj;
            a.y /= ljj;
        }
        __syncthreads();
        // trailing update of the lower triangle: A[i][k] -= L[i][j] conj(L[k][j])
        const int m = T - j - 1;
        for (int idx = tid; idx < m * m; idx += nt) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k > i) continue;
            const double2 li = A[(long)i * T + j], lk = A[(long)k * T + j];
            double2 &a = A[(long)i * T + k];
            a.x -= li.x * lk.x + li.y * lk.y;
            a.y -= li.y * lk.x - li.x * lk.y;
        }
        __syncthreads();
    }
    // forward: L y = p (column-oriented)
    for (int j = 0; j < T; ++j) {
        if (tid == 0) {
            const double l = A[(long)j * T + j].x;
            y[j] = make_double2(y[j].x / l, y[j].y / l);
        }
        __syncthreads();
        const double2 yj = y[j];
        for (int i = j + 1 + tid; i < T; i += nt) {
            const double2 l = A[(long)i * T + j];
            y[i].x -= l.x * yj.x - l.y * yj.y;
            y[i].y -= l.x * yj.y + l.y * yj.x;
        }
        __syncthreads();
    }
    // back: L^H h = y, (L^H)[i][j] = conj(L[j][i])
    for (int j = T - 1; j >= 0; --j) {
        if (tid == 0) {
            const double l = A[(long)j * T + j].x;
            h[j] = make_double2(y[j].x / l, y[j].y / l);
        }
        __syncthreads();
        const double2 hj = h[j];
        for (int i = tid; i < j; i += nt) {
            const double2 l = A[(long)j * T + i];      // conj(l) * hj
            y[i].x -= l.x * hj.x + l.y * hj.y;
            y[i].y -= l.x * hj.y - l.y * hj.x;
        }
        __syncthreads();
    }
}

__global__ void fde_response_kernel(const double2 *__restrict__ h, int T, float2 *__restrict__ H) {
    constexpr int N = 1024;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    if (k >= N / 4 && k < 3 * N / 4) {
        H[k] = make_float2(0.f, 0.f);
        return;
    }
    const int D = (T - 1) / 2;
    double ax = 0.0, ay = 0.0;
    for (int t = 0; t < T; ++t) {
        // e^{-j 2 pi k (t - D) / N}, the exponent reduced mod N exactly
        int e = (k * (t - D)) % N;
        if (e < 0) e += N;
        double s, c;
        sincospi(-2.0 * e / N, &s, &c);
        ax += h[t].x * c - h[t].y * s;
        ay += h[t].x * s + h[t].y * c;
    }
    H[k] = make_float2((float)(ax / N), (float)(ay / N));
}

__global__ void __launch_bounds__(128)
fde1024_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, long ns, int step, int half, long f1,
               const float2 *__restrict__ H, const float2 *__restrict__ tw) {
    constexpr int RP = 33;
    __shared__ float2 smem[4][32 * RP];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const long f = (long)blockIdx.x * 4 + w;
    if (f >= f1) return;
    float2 *sm = smem[w];
    const float2 *src = in + (long)blockIdx.y * ns;
    float2 *dst = out + (long)blockIdx.y * (ns / 2);
    const long start = f * step - half;
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const long idx = start + l + 32 * i;
        v[i] = (idx >= 0 && idx < ns) ? src[idx] : make_float2(0.f, 0.f);
    }
    // forward: lane n2 = l, DFT over n1 -> k1, twiddle W1024^{n2 k1}
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
    // output band times H (1/1024 included): Y[l + 32 k2']
    float2 u[16];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        u[j] = cmul(v[j], __ldg(H + l + 32 * j));
        u[j + 8] = cmul(v[j + 24], __ldg(H + l + 32 * (j + 24)));
    }
    // inner inverse 16-point DFT over k2' -> m1, twiddle e^{j 2 pi l m1 / 512}
    dft16<true>(u);
#pragma unroll
    for (int m1 = 1; m1 < 16; ++m1) u[m1] = cmul(u[m1], twid(tw, 2 * l * m1, 1023, true));
    __syncwarp();
#pragma unroll
    for (int m1 = 0; m1 < 16; ++m1) sm[m1 * RP + l] = u[m1];
    __syncwarp();
    // lane (m1, q): 16-point inverse DFT over r of the values of l = 2r + q
    const int m1 = l & 15, q = l >> 4;
#pragma unroll
    for (int r = 0; r < 16; ++r) u[r] = sm[m1 * RP + 2 * r + q];
    dft16<true>(u);
    if (q) {
#pragma unroll
        for (int m2 = 1; m2 < 16; ++m2) u[m2] = cmul(u[m2], twid(tw, 32 * m2, 1023, true));
    }
    // radix 2 with the partner lane: q = 0 keeps E + w O (m2 < 16), q = 1 E - w O
    const int hm = half / 2, sm_out = step / 2;
    const long o0 = f * sm_out - hm;
#pragma unroll
    for (int m2 = 0; m2 < 16; ++m2) {
        const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, u[m2].x, 16),
                                         __shfl_xor_sync(0xffffffffu, u[m2].y, 16));
        const float2 y = q ? csub(other, u[m2]) : cadd(u[m2], other);
        const int m = m1 + 16 * (m2 + 16 * q);
        if (m >= hm && m < hm + sm_out) {
            const long o = o0 + m;
            if (o < ns / 2) dst[o] = y;
        }
    }
}

}  // namespace

// Overlap-save application with 4 -> 2 resampling: rows of ns input
// samples (ns even) -> rows of ns/2 outputs; n_ov a multiple of 4.
cudaError_t launch_fde_apply(const float2 *in, float2 *out, long ns, int n_rows, int n_ov, const float2 *H,
                             const float2 *tw, cudaStream_t st) {
    const int step = 1024 - n_ov, half = n_ov / 2;
    if (n_ov <= 0 || n_ov >= 1024 || (n_ov & 3) || (ns & 1)) return cudaErrorInvalidValue;
    const long nframes = (ns + step - 1) / step;
    if (nframes <= 0 || n_rows <= 0) return cudaSuccess;
    dim3 grid((unsigned)((nframes + 3) / 4), (unsigned)n_rows);
    fde1024_kernel<<<grid, 128, 0, st>>>(in, out, ns, step, half, nframes, H, tw);
    return cudaGetLastError();
}

cudaError_t launch_fde_corr(const float2 *x, long n, const float2 *d, int K, int T, int sps, double2 *R,
                            double2 *p, cudaStream_t st) {
    if (T < 1 || K < 1 || sps < 1) return cudaErrorInvalidValue;
    fde_corr_kernel<<<T, 256, 0, st>>>(x, n, d, K, T, sps, R, p);
    return cudaGetLastError();
}

cudaError_t launch_fde_solve(double2 *R, const double2 *p, double2 *y, int T, double delta, double2 *h,
                             cudaStream_t st) {
    fde_solve_kernel<<<1, 1024, 0, st>>>(R, p, y, T, delta, h);
    return cudaGetLastError();
}

cudaError_t launch_fde_response(const double2 *h, int T, float2 *H, cudaStream_t st) {
    fde_response_kernel<<<4, 256, 0, st>>>(h, T, H);
    return cudaGetLastError();
}
