// Issue-rate probe of the FP32 pipes: the measured denominator of the
// "alu" roofline of the phase search (one FP32 lane-instruction per
// candidate distance).  Not part of the receiver chain.
//
// Every thread runs kChains independent dependency chains of one
// instruction kind, unrolled kUnroll times per loop trip, so that the loop
// overhead is under 3 % and the pipes, not latency, bound the rate (two
// blocks of 1024 threads per SM: 16 warps per scheduler).  The chains' values
// are stored only when a runtime flag is set, so nothing is dead code.
#include <cuda_runtime.h>

#include "rx_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThreads = 1024;

template <int KIND>
__global__ void __launch_bounds__(kThreads, 2) issue_kernel(int iters, float x, float y, int store, float *out) {
    float s = 0.f;
    if constexpr (KIND == 1) {            // FFMA2: two multiply-adds per lane (packed pair)
        unsigned long long p[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) p[c] = pk2(x + (float)(threadIdx.x + c), y - (float)c);
        const unsigned long long q = pk2(x, y), r = pk2(y, x);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < kChains; ++c)
                    asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(q), "l"(r));
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float lo, hi;
            upk2(p[c], lo, hi);
            s += lo + hi;
        }
    } else {
        float a[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = x + (float)(threadIdx.x + c);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
                for (int c = 0; c < kChains; ++c) {
                    if constexpr (KIND == 0)      // FFMA: one multiply-add per lane
                        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[c]) : "f"(x), "f"(y));
                    else                          // FMNMX: min of two
                        asm volatile("min.f32 %0, %0, %1;" : "+f"(a[c]) : "f"(u & 1 ? x : y));
                }
            }
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += a[c];
    }
    if (store) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int rx_issue_rate(int kind, int iters, double *lane_instr_per_s, double *ms) {
    if (kind < 0 || kind > 2 || iters < 1 || !lane_instr_per_s) return RX_EINVAL;
    const int blocks = 2 * sm_count();
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return RX_ECUDA;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&](int n) {
        if (kind == 0) issue_kernel<0><<<blocks, kThreads, 0, st>>>(n, 1.0001f, -0.5f, 0, nullptr);
        else if (kind == 1) issue_kernel<1><<<blocks, kThreads, 0, st>>>(n, 1.0001f, -0.5f, 0, nullptr);
        else issue_kernel<2><<<blocks, kThreads, 0, st>>>(n, 1.0001f, -0.5f, 0, nullptr);
    };
    launch(16);                                  // warm-up
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float t = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&t, e0, e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (err != cudaSuccess || t <= 0.f) return RX_ECUDA;
    const double lanes = (double)blocks * kThreads * iters * kUnroll * kChains;
    *lane_instr_per_s = lanes / (t * 1e-3);
    if (ms) *ms = t;
    return RX_OK;
}
