// A2: 2x2 butterfly FIR, T/2-spaced input, one output per symbol:
//   y_q[k] = sum_{p in X,Y} sum_{t<T} conj(h_qp[t]) x_p[2k + D - t],  D = (T-1)/2.
//
// One block of 128 threads makes 512 consecutive outputs of one stream.  The
// 1024 + 2D input samples of each polarisation are staged in shared memory
// (one pad slot every 8 samples, so that threads 8 samples apart hit
// different banks) and the conjugated taps sit in shared memory, read as
// broadcasts.  Each thread makes 4 consecutive outputs for both q: per tap
// it needs one new sample per even/odd tap chain (the other three slide
// through registers), so the loop is 32 FMAs per shared-memory sample load.
#include "rx_internal.h"

namespace {

constexpr int kOut = 512;
constexpr int kThreads = 128;

__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }

template <int T>
__global__ void __launch_bounds__(kThreads)
fir_kernel(const float2 *__restrict__ x, long ns, const float2 *__restrict__ taps, long k0,
           long k1, float2 *__restrict__ y, long y_stride, long y_off) {
    constexpr int D = (T - 1) / 2;
    constexpr int NS = 2 * kOut + 2 * D;
    constexpr int NSP = NS + NS / 8 + 1;
    __shared__ float2 xs[2][NSP];
    __shared__ float2 hs[2][2][T];   // conj(h[q][p][t])
    const int s = blockIdx.y;
    const int tid = threadIdx.x;
    const long kb = k0 + (long)blockIdx.x * kOut;
    const long base = 2 * kb - D;   // global sample of local index 0
    const float2 *xs0 = x + (long)s * 2 * ns;
    for (int i = tid; i < 2 * NS; i += kThreads) {
        const int p = i / NS, j = i - p * NS;
        const long g = base + j;
        xs[p][pad8(j)] = (g >= 0 && g < ns) ? xs0[(long)p * ns + g] : make_float2(0.f, 0.f);
    }
    for (int i = tid; i < 4 * T; i += kThreads) {
        float2 h = taps[(long)s * 4 * T + i];
        (&hs[0][0][0])[i] = make_float2(h.x, -h.y);
    }
    __syncthreads();

    float2 acc[2][4];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] = make_float2(0.f, 0.f);

    const int lb = 8 * tid + 2 * D;   // local index of (r = 0, t = 0)
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        float2 E[4], O[4];   // even / odd tap chains: E[r] = x[lb + 2r - 2j], O[r] = x[lb + 2r - 2j - 1]
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            E[r] = xs[p][pad8(lb + 2 * r)];
            O[r] = xs[p][pad8(lb + 2 * r - 1)];
        }
#pragma unroll
        for (int j = 0; j <= D; ++j) {
            const int te = 2 * j;
            {
                const float2 h0 = hs[0][p][te], h1 = hs[1][p][te];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[0][r].x = fmaf(h0.x, E[r].x, fmaf(-h0.y, E[r].y, acc[0][r].x));
                    acc[0][r].y = fmaf(h0.x, E[r].y, fmaf(h0.y, E[r].x, acc[0][r].y));
                    acc[1][r].x = fmaf(h1.x, E[r].x, fmaf(-h1.y, E[r].y, acc[1][r].x));
                    acc[1][r].y = fmaf(h1.x, E[r].y, fmaf(h1.y, E[r].x, acc[1][r].y));
                }
            }
            if (j < D) {
                const int to = 2 * j + 1;
                const float2 h0 = hs[0][p][to], h1 = hs[1][p][to];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[0][r].x = fmaf(h0.x, O[r].x, fmaf(-h0.y, O[r].y, acc[0][r].x));
                    acc[0][r].y = fmaf(h0.x, O[r].y, fmaf(h0.y, O[r].x, acc[0][r].y));
                    acc[1][r].x = fmaf(h1.x, O[r].x, fmaf(-h1.y, O[r].y, acc[1][r].x));
                    acc[1][r].y = fmaf(h1.x, O[r].y, fmaf(h1.y, O[r].x, acc[1][r].y));
                }
                // slide the windows by one output (two samples)
#pragma unroll
                for (int r = 3; r > 0; --r) { E[r] = E[r - 1]; O[r] = O[r - 1]; }
                E[0] = xs[p][pad8(lb - 2 * (j + 1))];
                if (j + 1 < D) O[0] = xs[p][pad8(lb - 2 * (j + 1) - 1)];
            }
        }
    }
    const long kt = kb + 4 * tid;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        float2 *yq = y + ((long)s * 2 + q) * y_stride + y_off;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (kt + r < k1) yq[kt + r - k0] = acc[q][r];
    }
}

}  // namespace

cudaError_t launch_fir(const float2 *x, long ns, const float2 *taps, long k0, long k1, float2 *y,
                       long y_stride, long y_off, int n_streams, int T, cudaStream_t st) {
    if (k1 <= k0 || n_streams <= 0) return cudaSuccess;
    dim3 grid((unsigned)((k1 - k0 + kOut - 1) / kOut), (unsigned)n_streams);
    switch (T) {
        case 7: fir_kernel<7><<<grid, kThreads, 0, st>>>(x, ns, taps, k0, k1, y, y_stride, y_off); break;
        case 15: fir_kernel<15><<<grid, kThreads, 0, st>>>(x, ns, taps, k0, k1, y, y_stride, y_off); break;
        case 31: fir_kernel<31><<<grid, kThreads, 0, st>>>(x, ns, taps, k0, k1, y, y_stride, y_off); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
