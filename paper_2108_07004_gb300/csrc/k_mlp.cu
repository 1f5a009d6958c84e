// Learned demapper: MLP 4 -> 128 -> 128 -> 6 with GELU, bfloat16 weights,
// float32 activations and accumulation.  Input: the de-rotated 4D symbol
// (Re z_X, Im z_X, Re z_Y, Im z_Y); output o = sigma^2 * LLR (LLR > 0 means
// bit 0), trained with the mean binary cross-entropy over the bits and Adam.
//
// Kernels (batch of n samples).  Inference: infer_umma_kernel (k_mlp_tc.cu,
// tcgen05) or infer_tc_kernel below (mma.sync).  Training: the kernels below,
// with the three 128-wide GEMMs either on the tcgen05 tensor cores
// (gemm_tc_kernel, k_mlp_tc.cu) or the float32 gemm_kernel:
//   layer1_kernel      a1 = x W1^T + b1, h1 = gelu(a1)
//   gemm_kernel        tiled float32 GEMM (64 x 64 tiles, 4 x 4 per thread)
//                      with bfloat16 weight operands and fused epilogues:
//                      a2 = h1 W2^T + b2 -> h2 = gelu(a2); dh1 = da2 W2 ->
//                      da1 = dh1 gelu'(a1); dW2 = da2^T h1 over batch slices
//   layer3_loss_kernel o = h2 W3^T + b3, LLR = o / sigma^2, BCE terms and
//                      d loss / d o per sample
//   back3_kernel       dh2 = do W3, da2 = dh2 gelu'(a2)
//   colsum kernels     the batch reductions (dW1, dW3, biases, loss) in a
//                      fixed order: per-block partials, then one pass
//   adam_kernel        Adam on the float32 master weights, then the
//                      bfloat16 copies the layers use
// Every reduction over the batch is in a fixed order, so a step gives the
// same bits on every run.
#include <algorithm>
#include <cmath>

#include <cuda_bf16.h>

#include "mlp_dev.h"
#include "rx_internal.h"

namespace {

using namespace mlpd;

__device__ __forceinline__ float softplus(float t) { return fmaxf(t, 0.f) + log1pf(expf(-fabsf(t))); }
__device__ __forceinline__ float sigmoid(float t) { return 1.f / (1.f + expf(-t)); }

// a1, h1 [n][H]
__global__ void layer1_kernel(const float *__restrict__ x, long n, const uint16_t *__restrict__ W1,
                              const float *__restrict__ b1, float *__restrict__ a1, float *__restrict__ h1) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * H) return;
    const long s = i / H;
    const int j = (int)(i - s * H);
    float a = b1[j];
#pragma unroll
    for (int c = 0; c < 4; ++c) a = fmaf(x[s * 4 + c], bf16_to_f(W1[j * 4 + c]), a);
    a1[i] = a;
    h1[i] = gelu(a);
}

// C[M][N] (+)= op(A) op(B): A float32 (row-major [M][K], or [K][M] when TA),
// B bfloat16 or float32 ([N][K] when TB, else [K][N]); epilogues EPI_*.
constexpr int TM = 64, TN = 64, TK = 16;

template <bool TA, bool TB, bool BBF, int EPI>
__global__ void __launch_bounds__(256)
gemm_kernel(int M, int N, int K, const float *__restrict__ A, int lda, const void *__restrict__ Bv, int ldb,
            const float *__restrict__ bias, const float *__restrict__ aux, int ldaux, float *__restrict__ out0,
            float *__restrict__ out1, int ldo, long k_slice, long out_slice_stride) {
    __shared__ float As[TK][TM + 4];
    __shared__ float Bs[TK][TN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    // batch slice (split K) of this block
    const long kb = (long)blockIdx.z * k_slice, ke = min((long)K, kb + k_slice);
    float acc[4][4] = {};
    for (long k0 = kb; k0 < ke; k0 += TK) {
        for (int i = tid; i < TK * TM; i += 256) {
            const int kk = i / TM, mm = i - kk * TM;
            const long k = k0 + kk;
            const int m = m0 + mm;
            float v = 0.f;
            if (k < ke && m < M) v = TA ? A[k * lda + m] : A[(long)m * lda + k];
            As[kk][mm] = v;
        }
        for (int i = tid; i < TK * TN; i += 256) {
            const int kk = i / TN, nn = i - kk * TN;
            const long k = k0 + kk;
            const int nidx = n0 + nn;
            float v = 0.f;
            if (k < ke && nidx < N) {
                const long off = TB ? (long)nidx * ldb + k : k * ldb + nidx;
                v = BBF ? bf16_to_f(static_cast<const uint16_t *>(Bv)[off]) : static_cast<const float *>(Bv)[off];
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        }
        __syncthreads();
    }
    float *o0 = out0 + (long)blockIdx.z * out_slice_stride;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int m = m0 + ty * 4 + r;
        if (m >= M) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int nidx = n0 + tx * 4 + c;
            if (nidx >= N) continue;
            const long o = (long)m * ldo + nidx;
            if (EPI == EPI_BIAS_GELU) {
                const float pre = acc[r][c] + bias[nidx];
                o0[o] = pre;
                out1[o] = gelu(pre);
            } else if (EPI == EPI_GELU_GRAD) {
                o0[o] = acc[r][c] * gelu_grad(aux[(long)m * ldaux + nidx]);
            } else {
                o0[o] = acc[r][c];
            }
        }
    }
}

// o = h2 W3^T + b3; LLR = o / sigma^2; per sample: sum of BCE terms and
// d loss / d o (mean over n x 6 bits), and (inference) the LLRs
__global__ void __launch_bounds__(128)
layer3_kernel(const float *__restrict__ h2, long n, const uint16_t *__restrict__ W3, const float *__restrict__ b3,
              const float *__restrict__ sigma2, const uint8_t *__restrict__ bits, float *__restrict__ dO,
              float *__restrict__ loss_s, float *__restrict__ llr) {
    __shared__ float w[NOUT][H];
    for (int i = threadIdx.x; i < NOUT * H; i += blockDim.x) w[i / H][i % H] = bf16_to_f(W3[i]);
    __syncthreads();
    const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float o[NOUT];
#pragma unroll
    for (int k = 0; k < NOUT; ++k) o[k] = b3[k];
    const float *hs = h2 + s * H;
    for (int j = 0; j < H; ++j) {
        const float v = hs[j];
#pragma unroll
        for (int k = 0; k < NOUT; ++k) o[k] = fmaf(v, w[k][j], o[k]);
    }
    const float inv = 1.f / sigma2[s];
    const float scale = 1.f / (float)(n * NOUT);
    float ls = 0.f;
#pragma unroll
    for (int k = 0; k < NOUT; ++k) {
        const float L = o[k] * inv;
        if (llr) llr[s * NOUT + k] = L;
        if (bits) {
            const float sg = bits[s * NOUT + k] ? -1.f : 1.f;     // +1 for bit 0
            ls += softplus(-sg * L);
            dO[s * NOUT + k] = -sg * sigmoid(-sg * L) * scale * inv;
        }
    }
    if (bits) loss_s[s] = ls * scale;
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores: one warp per 16 samples, the 128 x 128
// layer as bfloat16 mma.sync m16n8k16 with float32 accumulation.  The
// weights are bfloat16 already; each float32 activation h is split into
// three bfloat16 terms, hi = bf16(h), mid = bf16(h - hi), lo = bf16(h - hi -
// mid) (what is left is below 2^-24 |h|, float32's own rounding), and the
// layer is the three products W hi + W mid + W lo, each exact in the float32
// accumulator's inputs.  Layer 2 runs k-step by k-step: layer 1's 16
// columns of the step are computed straight into the A fragments (lane:
// rows g = lane/4 and g + 8, columns 2 (lane % 4) + {0, 1} and + 8) and
// multiplied into the accumulators of all 16 output tiles, so only one
// step's fragments are live (125 registers, 4 blocks per SM); the
// accumulators of layer 2 (rows g,
// g + 8, columns 2 (lane % 4) + {0, 1} of every 8-column tile) feed layer 3
// as per-lane partial sums reduced over the four lanes of a row.
// Persistent blocks stage W2 once (rows padded to 136 bfloat16, so that the
// B-fragment loads of a warp hit 32 banks) and loop over 64-sample tiles.
// ---------------------------------------------------------------------------
constexpr int kW2P = H + 8;   // padded row of the staged W2 (bfloat16)

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128, 4)
infer_tc_kernel(const float *__restrict__ x, const float *__restrict__ sigma2, long n,
                const uint16_t *__restrict__ W1q, const float *__restrict__ b1, const uint16_t *__restrict__ W2q,
                const float *__restrict__ b2, const uint16_t *__restrict__ W3q, const float *__restrict__ b3,
                float *__restrict__ llr) {
    __shared__ __align__(16) uint16_t w2[H * kW2P];
    __shared__ float w1[H][4], bb1[H], bb2[H], w3[NOUT][H], bb3[NOUT];
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) w2[(i / H) * kW2P + (i % H)] = W2q[i];
    for (int i = threadIdx.x; i < H * 4; i += blockDim.x) w1[i / 4][i % 4] = bf16_to_f(W1q[i]);
    for (int i = threadIdx.x; i < NOUT * H; i += blockDim.x) w3[i / H][i % H] = bf16_to_f(W3q[i]);
    for (int i = threadIdx.x; i < H; i += blockDim.x) { bb1[i] = b1[i]; bb2[i] = b2[i]; }
    if (threadIdx.x < NOUT) bb3[threadIdx.x] = b3[threadIdx.x];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, c0 = 2 * (lane & 3);
    const long n_tiles = (n + 63) / 64;
    for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const long r0 = tile * 64 + warp * 16 + g, r1 = r0 + 8;     // this lane's two samples
        float xa[4], xb[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            xa[c] = r0 < n ? x[r0 * 4 + c] : 0.f;
            xb[c] = r1 < n ? x[r1 * 4 + c] : 0.f;
        }
        // layer 2 k-step by k-step: that step's 16 columns of layer 1 are made
        // straight into the A fragments (three bfloat16 terms), then multiplied
        // into the accumulators of all 16 output tiles, so only one step's
        // fragments are live
        float acc[16][4];
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll 1
        for (int kk = 0; kk < 8; ++kk) {
            unsigned ah[4], am[4], al[4];
#pragma unroll
            for (int half = 0; half < 2; ++half) {          // columns + 0 / + 8
                const int j0 = kk * 16 + half * 8 + c0;
                float pa[2], pb[2];                          // rows g / g + 8, columns j0, j0 + 1
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    pa[e] = bb1[j0 + e];
                    pb[e] = bb1[j0 + e];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        pa[e] = fmaf(xa[c], w1[j0 + e][c], pa[e]);
                        pb[e] = fmaf(xb[c], w1[j0 + e][c], pb[e]);
                    }
                }
                split3_bf16x2(gelu(pa[0]), gelu(pa[1]), ah[2 * half], am[2 * half], al[2 * half]);
                split3_bf16x2(gelu(pb[0]), gelu(pb[1]), ah[2 * half + 1], am[2 * half + 1], al[2 * half + 1]);
            }
#pragma unroll
            for (int nt = 0; nt < 16; ++nt) {
                const uint16_t *wrow = w2 + (nt * 8 + g) * kW2P + c0 + kk * 16;
                const unsigned bq0 = *reinterpret_cast<const unsigned *>(wrow);
                const unsigned bq1 = *reinterpret_cast<const unsigned *>(wrow + 8);
                mma_bf16(acc[nt], al, bq0, bq1);      // smallest terms first
                mma_bf16(acc[nt], am, bq0, bq1);
                mma_bf16(acc[nt], ah, bq0, bq1);
            }
        }
        // GELU of layer 2 and layer 3's partial sums over this lane's columns
        float o0[NOUT], o1[NOUT];
#pragma unroll
        for (int k = 0; k < NOUT; ++k) { o0[k] = 0.f; o1[k] = 0.f; }
#pragma unroll
        for (int nt = 0; nt < 16; ++nt) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int j = nt * 8 + c0 + e;
                const float ha = gelu(acc[nt][e] + bb2[j]), hb = gelu(acc[nt][2 + e] + bb2[j]);
#pragma unroll
                for (int k = 0; k < NOUT; ++k) {
                    o0[k] = fmaf(ha, w3[k][j], o0[k]);
                    o1[k] = fmaf(hb, w3[k][j], o1[k]);
                }
            }
        }
        // the four lanes of a row hold disjoint columns: sum them
#pragma unroll
        for (int k = 0; k < NOUT; ++k) {
            o0[k] += __shfl_xor_sync(0xffffffffu, o0[k], 1);
            o0[k] += __shfl_xor_sync(0xffffffffu, o0[k], 2);
            o1[k] += __shfl_xor_sync(0xffffffffu, o1[k], 1);
            o1[k] += __shfl_xor_sync(0xffffffffu, o1[k], 2);
        }
        if ((lane & 3) == 0) {
            if (r0 < n) {
                const float inv = 1.f / sigma2[r0];
#pragma unroll
                for (int k = 0; k < NOUT; ++k) llr[r0 * NOUT + k] = (o0[k] + bb3[k]) * inv;
            }
            if (r1 < n) {
                const float inv = 1.f / sigma2[r1];
#pragma unroll
                for (int k = 0; k < NOUT; ++k) llr[r1 * NOUT + k] = (o1[k] + bb3[k]) * inv;
            }
        }
    }
}

// da2[s][j] = (sum_k dO[s][k] W3[k][j]) * gelu'(a2[s][j])
__global__ void back3_kernel(const float *__restrict__ dO, long n, const uint16_t *__restrict__ W3,
                             const float *__restrict__ a2, float *__restrict__ da2) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * H) return;
    const long s = i / H;
    const int j = (int)(i - s * H);
    float v = 0.f;
#pragma unroll
    for (int k = 0; k < NOUT; ++k) v = fmaf(dO[s * NOUT + k], bf16_to_f(W3[k * H + j]), v);
    da2[i] = v * gelu_grad(a2[i]);
}

// column sums over the batch in a fixed order: out[c] = sum_s f(s, c) for
// C columns, where f is src[s][c] (src2 == null) or src[s][c] * src2[s][c2]
// (outer product column c = (c1, c2) with c1 < C1 over src, c2 < C2 over src2).
// Block b sums rows b*rows .. (b+1)*rows - 1 into part[b][c]; a second launch
// (one block per 256 columns) adds the blocks in order.
__global__ void colsum_partial_kernel(const float *__restrict__ src, int ld, const float *__restrict__ src2,
                                      int ld2, int C1, int C2, long n, long rows, float *__restrict__ part) {
    const int C = src2 ? C1 * C2 : C1;
    const long s0 = (long)blockIdx.y * rows, s1 = min(n, s0 + rows);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const int c1 = src2 ? c / C2 : c, c2 = src2 ? c - (c / C2) * C2 : 0;
        float acc = 0.f;
        for (long s = s0; s < s1; ++s) {
            float v = src[s * ld + c1];
            if (src2) v *= src2[s * ld2 + c2];
            acc += v;
        }
        part[(long)blockIdx.y * C + c] = acc;
    }
}

__global__ void colsum_final_kernel(const float *__restrict__ part, int nb, int C, float *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float acc = 0.f;
    for (int b = 0; b < nb; ++b) acc += part[(long)b * C + c];
    out[c] = acc;
}

// Adam on the float32 masters, then the bfloat16 copies of the weights
__global__ void adam_kernel(float *__restrict__ theta, float *__restrict__ m, float *__restrict__ v,
                            const float *__restrict__ g, int np, float lr, float b1, float b2, float eps,
                            float bc1, float bc2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void quantize_kernel(const float *__restrict__ theta, int off, int cnt, uint16_t *__restrict__ q) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < cnt) q[i] = f_to_bf16(theta[off + i]);
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * 4, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + NOUT * H, NPAR = OFF_B3 + NOUT;
static_assert(NPAR == RX_MLP_PARAMS, "parameter count");
constexpr long kRows = 256;          // batch rows per partial-sum block
constexpr long kSliceTc = 256;       // batch rows per dW2 slice of the tensor-core GEMM
}  // namespace

static cudaError_t mlp_ensure(MlpDev &d, long n) {
    if (d.cap >= n) return cudaSuccess;
    float **bufs[] = {&d.a1, &d.h1, &d.a2, &d.h2, &d.da2, &d.da1};
    for (float **b : bufs) { cudaFree(*b); *b = nullptr; }
    cudaFree(d.dO); cudaFree(d.loss_s); cudaFree(d.part); cudaFree(d.wpart);
    d.dO = d.loss_s = d.part = d.wpart = nullptr;
    cudaError_t e;
    for (float **b : bufs)
        if ((e = cudaMalloc(b, sizeof(float) * (size_t)n * H)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.dO, sizeof(float) * (size_t)n * NOUT)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.loss_s, sizeof(float) * (size_t)n)) != cudaSuccess) return e;
    const long nb = (n + kRows - 1) / kRows;
    // column-sum partials: the widest is dW1 (H x 4) / biases (H) / dW3 (6 x H)
    if ((e = cudaMalloc(&d.part, sizeof(float) * (size_t)nb * H * 8)) != cudaSuccess) return e;
    // dW2 over batch slices of kRows * 8 samples (float32 GEMM) or kSliceTc
    const long ns = std::max((n + kRows * 8 - 1) / (kRows * 8), (n + kSliceTc - 1) / kSliceTc);
    if ((e = cudaMalloc(&d.wpart, sizeof(float) * (size_t)ns * H * H)) != cudaSuccess) return e;
    d.cap = n;
    return cudaSuccess;
}

cudaError_t mlp_alloc(MlpDev &d) {
    cudaError_t e;
    float **p[] = {&d.theta, &d.m, &d.v, &d.grad};
    for (float **b : p) {
        if ((e = cudaMalloc(b, sizeof(float) * NPAR)) != cudaSuccess) return e;
        if ((e = cudaMemset(*b, 0, sizeof(float) * NPAR)) != cudaSuccess) return e;
    }
    if ((e = cudaMalloc(&d.W1q, sizeof(uint16_t) * H * 4)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.W2q, sizeof(uint16_t) * H * H)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&d.W3q, sizeof(uint16_t) * NOUT * H)) != cudaSuccess) return e;
    return cudaSuccess;
}

void mlp_free(MlpDev &d) {
    float *bufs[] = {d.theta, d.m, d.v, d.grad, d.a1, d.h1, d.a2, d.h2, d.dO, d.da2, d.da1, d.loss_s, d.part, d.wpart};
    for (float *b : bufs) cudaFree(b);
    cudaFree(d.W1q); cudaFree(d.W2q); cudaFree(d.W3q);
    d = MlpDev{};
}

cudaError_t mlp_quantize(MlpDev &d, cudaStream_t st) {
    quantize_kernel<<<(H * 4 + 255) / 256, 256, 0, st>>>(d.theta, OFF_W1, H * 4, d.W1q);
    quantize_kernel<<<(H * H + 255) / 256, 256, 0, st>>>(d.theta, OFF_W2, H * H, d.W2q);
    quantize_kernel<<<(NOUT * H + 255) / 256, 256, 0, st>>>(d.theta, OFF_W3, NOUT * H, d.W3q);
    return cudaGetLastError();
}

static cudaError_t colsum(MlpDev &d, const float *src, int ld, const float *src2, int ld2, int C1, int C2,
                          long n, float *out, cudaStream_t st) {
    const int C = src2 ? C1 * C2 : C1;
    const long nb = (n + kRows - 1) / kRows;
    dim3 g((unsigned)((C + 255) / 256), (unsigned)nb);
    colsum_partial_kernel<<<g, 256, 0, st>>>(src, ld, src2, ld2, C1, C2, n, kRows, d.part);
    colsum_final_kernel<<<(C + 255) / 256, 256, 0, st>>>(d.part, (int)nb, C, out);
    return cudaGetLastError();
}

// forward (and, with bits, the loss terms and d loss / d o)
static cudaError_t mlp_forward(MlpDev &d, const float *x, const float *s2, const uint8_t *bits, long n,
                               float *llr, cudaStream_t st) {
    cudaError_t e = mlp_ensure(d, n);
    if (e != cudaSuccess) return e;
    layer1_kernel<<<(unsigned)((n * H + 255) / 256), 256, 0, st>>>(x, n, d.W1q, d.theta + OFF_B1, d.a1, d.h1);
    if (d.train_tc) {
        // a2[s][j] = sum_i h1[s][i] W2[j][i] + b2[j]
        e = launch_gemm_tc(EPI_BIAS_GELU, true, (int)n, H, H, d.h1, H, 1, d.W2q, H, 1, d.theta + OFF_B2, nullptr,
                           0, d.a2, d.h2, H, H, 0, 1, st);
        if (e != cudaSuccess) return e;
    } else {
        dim3 g2(H / TN, (unsigned)((n + TM - 1) / TM), 1);
        gemm_kernel<false, true, true, EPI_BIAS_GELU><<<g2, 256, 0, st>>>(
            (int)n, H, H, d.h1, H, d.W2q, H, d.theta + OFF_B2, nullptr, 0, d.a2, d.h2, H, H, 0);
    }
    layer3_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d.h2, n, d.W3q, d.theta + OFF_B3, s2, bits, d.dO,
                                                              d.loss_s, llr);
    return cudaGetLastError();
}

// gradient of the mean BCE into d.grad (and the loss into loss[0])
cudaError_t mlp_grad(MlpDev &d, const float *x, const float *s2, const uint8_t *bits, long n, float *loss,
                     cudaStream_t st) {
    cudaError_t e = mlp_forward(d, x, s2, bits, n, nullptr, st);
    if (e != cudaSuccess) return e;
    float *g = d.grad;
    // layer 3: dW3[k][j] = sum_s dO[s][k] h2[s][j], db3 = sum dO
    if ((e = colsum(d, d.dO, NOUT, d.h2, H, NOUT, H, n, g + OFF_W3, st)) != cudaSuccess) return e;
    if ((e = colsum(d, d.dO, NOUT, nullptr, 0, NOUT, 1, n, g + OFF_B3, st)) != cudaSuccess) return e;
    back3_kernel<<<(unsigned)((n * H + 255) / 256), 256, 0, st>>>(d.dO, n, d.W3q, d.a2, d.da2);
    // layer 2: dW2 = da2^T h1 (batch slices, then an ordered sum), db2
    const long slice = d.train_tc ? kSliceTc : kRows * 8;
    const long ns = (n + slice - 1) / slice;
    if (d.train_tc) {
        // dW2[j][i] = sum_s da2[s][j] h1[s][i]: both operands float32 (six term products)
        e = launch_gemm_tc(EPI_STORE, false, H, H, n, d.da2, 1, H, d.h1, 1, H, nullptr, nullptr, 0, d.wpart,
                           nullptr, H, slice, (long)H * H, (int)ns, st);
        if (e != cudaSuccess) return e;
    } else {
        dim3 gw(H / TN, H / TM, (unsigned)ns);
        gemm_kernel<true, false, false, EPI_STORE><<<gw, 256, 0, st>>>(
            H, H, (int)n, d.da2, H, d.h1, H, nullptr, nullptr, 0, d.wpart, nullptr, H, slice, (long)H * H);
    }
    colsum_final_kernel<<<(H * H + 255) / 256, 256, 0, st>>>(d.wpart, (int)ns, H * H, g + OFF_W2);
    if ((e = colsum(d, d.da2, H, nullptr, 0, H, 1, n, g + OFF_B2, st)) != cudaSuccess) return e;
    // layer 1: da1 = (da2 W2) gelu'(a1); dW1 = da1^T x; db1
    if (d.train_tc) {
        // dh1[s][i] = sum_j da2[s][j] W2[j][i]
        e = launch_gemm_tc(EPI_GELU_GRAD, true, (int)n, H, H, d.da2, H, 1, d.W2q, 1, H, nullptr, d.a1, H, d.da1,
                           nullptr, H, H, 0, 1, st);
        if (e != cudaSuccess) return e;
    } else {
        dim3 g1(H / TN, (unsigned)((n + TM - 1) / TM), 1);
        gemm_kernel<false, false, true, EPI_GELU_GRAD><<<g1, 256, 0, st>>>(
            (int)n, H, H, d.da2, H, d.W2q, H, nullptr, d.a1, H, d.da1, nullptr, H, H, 0);
    }
    if ((e = colsum(d, d.da1, H, x, 4, H, 4, n, g + OFF_W1, st)) != cudaSuccess) return e;
    if ((e = colsum(d, d.da1, H, nullptr, 0, H, 1, n, g + OFF_B1, st)) != cudaSuccess) return e;
    if (loss) {
        if ((e = colsum(d, d.loss_s, 1, nullptr, 0, 1, 1, n, loss, st)) != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t mlp_adam(MlpDev &d, int t, float lr, cudaStream_t st) {
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)t), bc2 = 1.f - powf(b2, (float)t);
    adam_kernel<<<(NPAR + 255) / 256, 256, 0, st>>>(d.theta, d.m, d.v, d.grad, NPAR, lr, b1, b2, 1e-8f, bc1, bc2);
    return mlp_quantize(d, st);
}

cudaError_t mlp_infer_seg(MlpDev &d, const float *x, const float *s2, long n, int n_seg, long x_stride,
                          float *llr, long llr_stride, cudaStream_t st) {
    if (d.infer == 2)
        return launch_infer_umma(x, s2, n, n_seg, x_stride, llr_stride, d.W1q, d.theta + OFF_B1, d.W2q,
                                 d.theta + OFF_B2, d.W3q, d.theta + OFF_B3, llr, st);
    for (int g = 0; g < n_seg; ++g) {
        const cudaError_t e = mlp_infer(d, x + (size_t)g * x_stride * 4, s2 + (size_t)g * x_stride, n,
                                        llr + (size_t)g * llr_stride * NOUT, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t mlp_infer(MlpDev &d, const float *x, const float *s2, long n, float *llr, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (d.infer == 2)
        return launch_infer_umma(x, s2, n, 1, n, n, d.W1q, d.theta + OFF_B1, d.W2q, d.theta + OFF_B2, d.W3q,
                                 d.theta + OFF_B3, llr, st);
    const long tiles = (n + 63) / 64;
    const int grid = (int)std::min<long>(tiles, 4L * sm_count());
    infer_tc_kernel<<<grid, 128, 0, st>>>(x, s2, n, d.W1q, d.theta + OFF_B1, d.W2q, d.theta + OFF_B2, d.W3q,
                                          d.theta + OFF_B3, llr);
    return cudaGetLastError();
}
