// Device helpers of the learned demapper's kernels (k_mlp.cu, k_mlp_tc.cu):
// layer sizes, bfloat16 rounding and the three-term bfloat16 split of
// float32 values, GELU (exact erf form) and its derivative.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

namespace mlpd {

constexpr int H = 128;
constexpr int NOUT = 6;

// GEMM epilogues (float32 and tensor-core GEMMs):
//   EPI_BIAS_GELU: pre = C + bias[n] -> out0 = pre, out1 = gelu(pre)
//   EPI_GELU_GRAD: out0 = C * gelu'(aux[m][n])
//   EPI_STORE:     out0 = C
enum { EPI_BIAS_GELU = 0, EPI_GELU_GRAD = 1, EPI_STORE = 2 };

__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __uint_as_float((unsigned)b << 16); }

__device__ __forceinline__ uint16_t f_to_bf16(float f) {   // round to nearest, ties to even
    const unsigned u = __float_as_uint(f);
    return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float a) {
    return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * expf(-0.5f * a * a) * 0.39894228040143268f;
}

// two float32 values rounded to bfloat16 (nearest, ties to even: the same
// rounding as f_to_bf16) in one register, the first in the low half
__device__ __forceinline__ unsigned cvt_bf16x2(float first, float second) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(first, second);
    return *reinterpret_cast<const unsigned *>(&v);
}
__device__ __forceinline__ float bf16_lo(unsigned v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf16_hi(unsigned v) { return __uint_as_float(v & 0xffff0000u); }

// (hi, mid, lo) bfloat16 pairs of two float32 values
__device__ __forceinline__ void split3_bf16x2(float a, float b, unsigned &hi, unsigned &mid, unsigned &lo) {
    hi = cvt_bf16x2(a, b);
    const float ra = a - bf16_lo(hi), rb = b - bf16_hi(hi);
    mid = cvt_bf16x2(ra, rb);
    lo = cvt_bf16x2(ra - bf16_lo(mid), rb - bf16_hi(mid));
}

}  // namespace mlpd
