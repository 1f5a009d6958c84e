// Learned demapper on the tcgen05 tensor cores: the fused inference kernel
// and the GEMM kernel of the training steps.
//
// Both run the 128-wide contractions as tcgen05.mma kind::f16 with bfloat16
// operands and float32 accumulators in tensor memory (TMEM), M = N = 128,
// K = 16 per MMA.  Weights are bfloat16 by the network's definition (every
// layer computes with its weights rounded to bfloat16), so they enter the
// MMA exactly; a float32 activation or gradient v is split into three
// bfloat16 terms hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid)
// (what is left is below 2^-24 |v|), and a product of two float32 operands
// keeps the six term products down to 2^-16 of the leading one (hi hi,
// hi mid, mid hi, hi lo, lo hi, mid mid; the dropped ones are below 2^-23).
// The float32 accumulator then sees the same products as a float32 GEMM, up
// to the order of the additions (the three-way bfloat16 emulation of
// float32 products: Henry, Tang and Heinecke, "Leveraging the bfloat16
// artificial intelligence datatype for higher-precision computations",
// ARITH 2019).
//
// Operands are written by the threads into shared memory in the canonical
// K-major layout without swizzle (tc_dev.h), one 4 KB tile per 128 rows x
// 16 bfloat16 and term; one thread issues the MMAs of a K-step and commits
// them to an mbarrier, which the threads wait on (bounded: a wait that
// gives up sets a flag read by mlp_tc_status, and the block stops issuing)
// before they overwrite the tiles.  Each thread owns one row of the 128-row
// tile, which is TMEM lane (row) of the accumulator: the epilogue reads its
// row with tcgen05.ld.
#include <algorithm>
#include <atomic>

#include "mlp_dev.h"
#include "rx_internal.h"
#include "tc_dev.h"

namespace {

using namespace mlpd;

constexpr int kThr = 128;                  // one thread per accumulator row
constexpr int kKstep = 16;                 // K of one MMA (bfloat16)
constexpr uint32_t kTileB = 4096;          // one 128 x 16 bfloat16 operand tile
constexpr int kKsteps = H / kKstep;        // K-steps of the 128-wide layer

// set when a bounded wait gave up (read and cleared by mlp_tc_status)
__device__ unsigned int g_mlp_tc_err;

__device__ __forceinline__ uint4 u4(const unsigned (&v)[8], int half) {
    return make_uint4(v[4 * half], v[4 * half + 1], v[4 * half + 2], v[4 * half + 3]);
}

// row `row` of one K-step (16 values as 8 bfloat16 pairs) into a tile
__device__ __forceinline__ void put_row(unsigned char *tile, int row, const unsigned (&v)[8]) {
    *reinterpret_cast<uint4 *>(tile + tc::kstep_off_bf16(row, 0)) = u4(v, 0);
    *reinterpret_cast<uint4 *>(tile + tc::kstep_off_bf16(row, 8)) = u4(v, 1);
}

// ---------------------------------------------------------------------------
// GELU of a pair of values for the inference kernel: a Phi(a) with the
// normal distribution function from erfc by Abramowitz and Stegun's rational
// approximation 7.1.26 (Handbook of Mathematical Functions, after Hastings;
// |error| <= 1.5e-7 on erf):
//   erfc(z) ~ t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-z^2},
//   t = 1 / (1 + p z),  z = |a| / sqrt(2) >= 0,
//   Phi(a) = 1/2 + copysign(1/2 - erfc(z) / 2, a),
// with e^{-a^2/2} = 2^{-a^2 log2(e) / 2}.  The reciprocal and the power of
// two are one hardware instruction each; the rest runs on packed f32x2
// pairs.  (The training kernels keep the exact-erf GELU of mlp_dev.h; the
// two agree to a few 1e-7 of |a|.)
// ---------------------------------------------------------------------------
constexpr float kAsP = 0.3275911f * 0.70710678118654752f;     // p / sqrt(2): t from |a|
// a1 .. a5 halved (the erfc / 2 of Phi)
constexpr float kAs1 = 0.5f * 0.254829592f, kAs2 = 0.5f * -0.284496736f, kAs3 = 0.5f * 1.421413741f,
                kAs4 = 0.5f * -1.453152027f, kAs5 = 0.5f * 1.061405429f;
constexpr float kNegHalfLog2e = -0.72134752044448170f;          // -log2(e) / 2

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ f32x2 gelu2(f32x2 a2) {
    float a0, a1;
    upk2(a2, a0, a1);
    const f32x2 t = pk2(rcp_approx(fmaf(fabsf(a0), kAsP, 1.f)), rcp_approx(fmaf(fabsf(a1), kAsP, 1.f)));
    f32x2 P = fma2(t, pk2(kAs5, kAs5), pk2(kAs4, kAs4));
    P = fma2(t, P, pk2(kAs3, kAs3));
    P = fma2(t, P, pk2(kAs2, kAs2));
    P = fma2(t, P, pk2(kAs1, kAs1));
    P = mul2(t, P);                                         // erfc(z) / 2 without e^{-z^2}
    const f32x2 u = mul2(mul2(a2, a2), pk2(kNegHalfLog2e, kNegHalfLog2e));
    float u0, u1;
    upk2(u, u0, u1);
    const f32x2 q = mul2(P, pk2(ex2_approx(u0), ex2_approx(u1)));   // erfc(z) / 2
    float q0, q1;
    upk2(sub2(pk2(0.5f, 0.5f), q), q0, q1);
    const f32x2 phi = add2(pk2(copysignf(q0, a0), copysignf(q1, a1)), pk2(0.5f, 0.5f));
    return mul2(a2, phi);
}

// ---------------------------------------------------------------------------
// Inference: x [n][4] -> LLR [n][6].  A block loops over tiles of 128
// samples (thread = sample = accumulator row).  Per K-step the threads make
// 16 columns of layer 1 (bias, GELU; pairs of columns as packed f32x2) and
// write their three bfloat16 terms; one thread issues the three MMAs against
// the K-step's tile of W2 (staged once per block) while the threads make the
// next K-step's columns.  After the eighth K-step each thread reads its row
// of layer 2 from TMEM, adds the bias, applies GELU and forms layer 3 (each
// output as a packed pair of even- and odd-column partial sums) and the LLRs.
// ---------------------------------------------------------------------------
struct InferSmem {
    unsigned char w2[kKsteps][kTileB];     // B operand: W2 [n][k], one tile per K-step
    unsigned char a[3][kTileB];            // A operand of the current K-step: hi, mid, lo
    f32x2 w1p[H / 2][4];                   // (W1[2i][c], W1[2i+1][c]) (bfloat16 values)
    f32x2 b1p[H / 2], b2p[H / 2];          // bias pairs
    f32x2 w3p[H / 2][NOUT];                // (W3[k][2i], W3[k][2i+1])
    float b3[8];
    unsigned long long bar;
    uint32_t tmem_slot;
    int fail;
};

// Segments: n_seg runs of n samples each, segment g's samples at rows
// g x_stride .. of x (and sigma2) and its LLRs at rows g llr_stride .. (the
// chain's streams of one block); tiles never straddle two segments.
__global__ void __launch_bounds__(kThr, 4)
infer_umma_kernel(const float *__restrict__ x, const float *__restrict__ sigma2, long n, int n_seg, long x_stride,
                  long llr_stride, const uint16_t *__restrict__ W1q, const float *__restrict__ b1,
                  const uint16_t *__restrict__ W2q, const float *__restrict__ b2, const uint16_t *__restrict__ W3q,
                  const float *__restrict__ b3, float *__restrict__ llr) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    InferSmem &sm = *reinterpret_cast<InferSmem *>(sm_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    // W2 (row-major [n][k], 16 bytes = 8 k per item) into the K-step tiles
    for (int i = tid; i < H * H / 8; i += kThr) {
        const int row = i / (H / 8), k = 8 * (i % (H / 8));
        const uint4 v = reinterpret_cast<const uint4 *>(W2q)[i];
        *reinterpret_cast<uint4 *>(sm.w2[k / kKstep] + tc::kstep_off_bf16(row, k % kKstep)) = v;
    }
    for (int i = tid; i < H / 2; i += kThr) {
        const int j = 2 * i;
#pragma unroll
        for (int c = 0; c < 4; ++c) sm.w1p[i][c] = pk2(bf16_to_f(W1q[4 * j + c]), bf16_to_f(W1q[4 * j + 4 + c]));
        sm.b1p[i] = pk2(b1[j], b1[j + 1]);
        sm.b2p[i] = pk2(b2[j], b2[j + 1]);
#pragma unroll
        for (int k = 0; k < NOUT; ++k) sm.w3p[i][k] = pk2(bf16_to_f(W3q[k * H + j]), bf16_to_f(W3q[k * H + j + 1]));
    }
    if (tid < 8) sm.b3[tid] = tid < NOUT ? b3[tid] : 0.f;
    if (warp == 0) tc::tmem_alloc(&sm.tmem_slot, 128);
    if (tid == 0) {
        tc::mbar_init(tc::smem_u32(&sm.bar), 1);
        sm.fail = 0;
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sm.tmem_slot, bar = tc::smem_u32(&sm.bar);
    const uint32_t idesc = tc::idesc_bf16(128, 128);
    const uint32_t t_row = tmem + ((uint32_t)(32 * warp) << 16);   // this warp's 32 lanes
    uint32_t issued = 0;                                          // K-steps committed
    bool stop = false;
    const long tps = (n + 127) / 128, n_tiles = tps * n_seg;
    for (long tile = blockIdx.x; tile < n_tiles && !stop; tile += gridDim.x) {
        const long seg = tile / tps;
        const long rl = (tile - seg * tps) * 128 + tid;           // sample within the segment
        const bool ok = rl < n;
        const long rx = seg * x_stride + rl, ro = seg * llr_stride + rl;
        f32x2 X[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float v = ok ? x[rx * 4 + c] : 0.f;
            X[c] = pk2(v, v);
        }
#pragma unroll 1
        for (int kk = 0; kk < kKsteps; ++kk) {
            unsigned th[8], tm[8], tl[8];
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const int i = kk * (kKstep / 2) + p;            // column pair 2i, 2i + 1
                f32x2 A = sm.b1p[i];
#pragma unroll
                for (int c = 0; c < 4; ++c) A = fma2(X[c], sm.w1p[i][c], A);
                float g0, g1;
                upk2(gelu2(A), g0, g1);
                split3_bf16x2(g0, g1, th[p], tm[p], tl[p]);
            }
            // the A tiles are free once the previous K-step's MMAs are done
            if (issued > 0 && !tc::mbar_wait(bar, (issued - 1) & 1)) sm.fail = 1;
            put_row(sm.a[0], tid, th);
            put_row(sm.a[1], tid, tm);
            put_row(sm.a[2], tid, tl);
            tc::fence_async_smem();
            tc::fence_before();
            __syncthreads();
            tc::fence_after();
            if (sm.fail) { stop = true; break; }
            if (tid == 0) {
                const uint64_t bd = tc::sdesc(tc::smem_u32(sm.w2[kk]), 128, 256);
                // smallest terms first
                tc::mma_bf16(tmem, tc::sdesc(tc::smem_u32(sm.a[2]), 128, 256), bd, idesc, kk > 0);
                tc::mma_bf16(tmem, tc::sdesc(tc::smem_u32(sm.a[1]), 128, 256), bd, idesc, 1);
                tc::mma_bf16(tmem, tc::sdesc(tc::smem_u32(sm.a[0]), 128, 256), bd, idesc, 1);
                tc::mma_commit(bar);
            }
            ++issued;
        }
        if (stop) break;
        // layer 2 of this tile is in TMEM
        if (!tc::mbar_wait(bar, (issued - 1) & 1)) sm.fail = 1;
        tc::fence_after();
        f32x2 o[NOUT];
#pragma unroll
        for (int k = 0; k < NOUT; ++k) o[k] = pk2(0.f, 0.f);
#pragma unroll 1
        for (int q = 0; q < H / 32; ++q) {
            float v[32];
            tc::tmem_ld32(t_row + (uint32_t)(32 * q), v);
#pragma unroll
            for (int p = 0; p < 16; ++p) {
                const int i = 16 * q + p;                        // column pair 2i, 2i + 1
                const f32x2 h = gelu2(add2(pk2(v[2 * p], v[2 * p + 1]), sm.b2p[i]));
#pragma unroll
                for (int k = 0; k < NOUT; ++k) o[k] = fma2(h, sm.w3p[i][k], o[k]);
            }
        }
        tc::fence_before();     // the TMEM reads come before the next tile's first MMA
        if (ok) {
            const float inv = 1.f / sigma2[rx];
#pragma unroll
            for (int k = 0; k < NOUT; ++k) {
                float e0, e1;
                upk2(o[k], e0, e1);
                llr[ro * NOUT + k] = ((e0 + e1) + sm.b3[k]) * inv;
            }
        }
    }
    // a block that stopped early may still have MMAs in flight: wait for them
    // (bounded) before the columns are freed
    if (stop && issued > 0) tc::mbar_wait(bar, (issued - 1) & 1);
    tc::fence_before();
    __syncthreads();
    if (tid == 0 && sm.fail) atomicOr(&g_mlp_tc_err, 1u);
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tmem, 128);
    }
}

// ---------------------------------------------------------------------------
// GEMM of the training steps: C[m][n] = sum_{k in slice} A(m, k) B(n, k) for
// one 128 x 128 tile (block x: M tiles, y: N tiles, z: K slices), A float32
// at A[m sam + k sak], B float32 at B[n sbn + k sbk] (three terms) or, with
// BBF, bfloat16 weights (one term).  Two operand stages: the threads load
// K-step i + 1 from global memory while the tensor cores multiply K-step i.
// Epilogues EPI_* (mlp_dev.h); EPI_STORE writes slice z at z out_slice_stride.
// ---------------------------------------------------------------------------
constexpr int kStages = 2;

template <bool BBF>
struct GemmSmem {
    unsigned char a[kStages][3][kTileB];
    unsigned char b[kStages][BBF ? 1 : 3][kTileB];
    unsigned long long bar[kStages];
    uint32_t tmem_slot;
    int fail;
};

// 16 float32 values of row `row`, k0 .. k0 + 15 (zero outside the matrix)
__device__ __forceinline__ void load_row_f32(const float *__restrict__ p, long row, long rows, long sr, long sk,
                                             long k0, long ke, bool vec, float (&v)[16]) {
    if (row < rows && vec && k0 + 16 <= ke) {
        const float4 *q = reinterpret_cast<const float4 *>(p + row * sr + k0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float4 t = q[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
        return;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = (row < rows && k0 + i < ke) ? p[row * sr + (k0 + i) * sk] : 0.f;
}

// 16 bfloat16 values (8 pairs, first in the low half) of row `row`
__device__ __forceinline__ void load_row_bf16(const uint16_t *__restrict__ p, long row, long rows, long sr,
                                              long sk, long k0, long ke, bool vec, unsigned (&v)[8]) {
    if (row < rows && vec && k0 + 16 <= ke) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p + row * sr + k0);
        const uint4 t0 = q[0], t1 = q[1];
        v[0] = t0.x; v[1] = t0.y; v[2] = t0.z; v[3] = t0.w;
        v[4] = t1.x; v[5] = t1.y; v[6] = t1.z; v[7] = t1.w;
        return;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const unsigned lo = (row < rows && k0 + 2 * i < ke) ? p[row * sr + (k0 + 2 * i) * sk] : 0u;
        const unsigned hi = (row < rows && k0 + 2 * i + 1 < ke) ? p[row * sr + (k0 + 2 * i + 1) * sk] : 0u;
        v[i] = lo | (hi << 16);
    }
}

__device__ __forceinline__ void split_row(const float (&v)[16], unsigned (&h)[8], unsigned (&m)[8],
                                          unsigned (&l)[8]) {
#pragma unroll
    for (int p = 0; p < 8; ++p) split3_bf16x2(v[2 * p], v[2 * p + 1], h[p], m[p], l[p]);
}

template <bool BBF, int EPI>
__global__ void __launch_bounds__(kThr, 4)
gemm_tc_kernel(int M, int N, long K, const float *__restrict__ A, long sam, long sak, bool a_vec,
               const void *__restrict__ Bv, long sbn, long sbk, bool b_vec, const float *__restrict__ bias,
               const float *__restrict__ aux, int ldaux, float *__restrict__ out0, float *__restrict__ out1,
               int ldo, long k_slice, long out_slice_stride) {
    extern __shared__ __align__(128) unsigned char sm_raw[];
    GemmSmem<BBF> &sm = *reinterpret_cast<GemmSmem<BBF> *>(sm_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const long m0 = (long)blockIdx.x * 128, n0 = (long)blockIdx.y * 128;
    const long kb = (long)blockIdx.z * k_slice, ke = min(K, kb + k_slice);
    const int nk = ke > kb ? (int)((ke - kb + kKstep - 1) / kKstep) : 0;
    if (warp == 0) tc::tmem_alloc(&sm.tmem_slot, 128);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) tc::mbar_init(tc::smem_u32(&sm.bar[s]), 1);
        sm.fail = 0;
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = sm.tmem_slot;
    const uint32_t idesc = tc::idesc_bf16(128, 128);
    const float *Bf = static_cast<const float *>(Bv);
    const uint16_t *Bq = static_cast<const uint16_t *>(Bv);

    float av[16], bv[16];
    unsigned bq[8];
    if (nk > 0) {
        load_row_f32(A, m0 + tid, M, sam, sak, kb, ke, a_vec, av);
        if constexpr (BBF) load_row_bf16(Bq, n0 + tid, N, sbn, sbk, kb, ke, b_vec, bq);
        else load_row_f32(Bf, n0 + tid, N, sbn, sbk, kb, ke, b_vec, bv);
    }
    int i = 0;
    for (; i < nk; ++i) {
        const int s = i % kStages;
        unsigned ah[8], am[8], al[8], bh[8], bm[8], bl[8];
        split_row(av, ah, am, al);
        if constexpr (!BBF) split_row(bv, bh, bm, bl);
        // stage s is free once the MMAs of K-step i - kStages are done
        if (i >= kStages && !tc::mbar_wait(tc::smem_u32(&sm.bar[s]), ((i - kStages) / kStages) & 1)) sm.fail = 1;
        put_row(sm.a[s][0], tid, ah);
        put_row(sm.a[s][1], tid, am);
        put_row(sm.a[s][2], tid, al);
        if constexpr (BBF) {
            put_row(sm.b[s][0], tid, bq);
        } else {
            put_row(sm.b[s][0], tid, bh);
            put_row(sm.b[s][1], tid, bm);
            put_row(sm.b[s][2], tid, bl);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (sm.fail) break;
        if (tid == 0) {
            auto ad = [&](int t) { return tc::sdesc(tc::smem_u32(sm.a[s][t]), 128, 256); };
            auto bd = [&](int t) { return tc::sdesc(tc::smem_u32(sm.b[s][t]), 128, 256); };
            // term products, smallest first: (a, b) with 0 = hi, 1 = mid, 2 = lo
            if constexpr (BBF) {
                tc::mma_bf16(tmem, ad(2), bd(0), idesc, i > 0);
                tc::mma_bf16(tmem, ad(1), bd(0), idesc, 1);
                tc::mma_bf16(tmem, ad(0), bd(0), idesc, 1);
            } else {
                tc::mma_bf16(tmem, ad(1), bd(1), idesc, i > 0);
                tc::mma_bf16(tmem, ad(2), bd(0), idesc, 1);
                tc::mma_bf16(tmem, ad(0), bd(2), idesc, 1);
                tc::mma_bf16(tmem, ad(1), bd(0), idesc, 1);
                tc::mma_bf16(tmem, ad(0), bd(1), idesc, 1);
                tc::mma_bf16(tmem, ad(0), bd(0), idesc, 1);
            }
            tc::mma_commit(tc::smem_u32(&sm.bar[s]));
        }
        // the next K-step's operands, in flight while the tensor cores run
        if (i + 1 < nk) {
            const long k0 = kb + (long)(i + 1) * kKstep;
            load_row_f32(A, m0 + tid, M, sam, sak, k0, ke, a_vec, av);
            if constexpr (BBF) load_row_bf16(Bq, n0 + tid, N, sbn, sbk, k0, ke, b_vec, bq);
            else load_row_f32(Bf, n0 + tid, N, sbn, sbk, k0, ke, b_vec, bv);
        }
    }
    const bool ok = (i == nk);
    // the last commit covers every MMA issued
    if (i > 0 && !tc::mbar_wait(tc::smem_u32(&sm.bar[(i - 1) % kStages]), ((i - 1) / kStages) & 1)) sm.fail = 1;
    tc::fence_after();
    const long m = m0 + tid;
    if (ok) {
        // every lane of a warp takes part in its TMEM reads; rows beyond M store nothing
        float *o0 = out0 + (long)blockIdx.z * out_slice_stride + m * ldo;
        for (int q = 0; q < 4; ++q) {
            const long nb = n0 + 32 * q;
            if (nb >= N) break;
            float v[32];
            if (nk > 0) {
                tc::tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * q), v);
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c) v[c] = 0.f;
            }
            if (m >= M) continue;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const long nn = nb + c;
                if (nn >= N) break;
                if (EPI == EPI_BIAS_GELU) {
                    const float pre = v[c] + bias[nn];
                    o0[nn] = pre;
                    out1[m * ldo + nn] = gelu(pre);
                } else if (EPI == EPI_GELU_GRAD) {
                    o0[nn] = v[c] * gelu_grad(aux[m * ldaux + nn]);
                } else {
                    o0[nn] = v[c];
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
    if (tid == 0 && sm.fail) atomicOr(&g_mlp_tc_err, 1u);
    if (warp == 0) {
        tc::fence_after();
        tc::tmem_free(tmem, 128);
    }
}

// opt in to the dynamic shared memory of a kernel once per device
template <typename K>
cudaError_t smem_opt_in(K kern, int bytes, std::atomic<unsigned long long> &set_on) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev >= 64 || !((set_on.load(std::memory_order_relaxed) >> dev) & 1ull)) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (err != cudaSuccess) return err;
        if (dev < 64) set_on.fetch_or(1ull << dev, std::memory_order_relaxed);
    }
    return cudaSuccess;
}

template <bool BBF, int EPI>
cudaError_t gemm_tc_t(int M, int N, long K, const float *A, long sam, long sak, const void *B, long sbn, long sbk,
                      const float *bias, const float *aux, int ldaux, float *out0, float *out1, int ldo,
                      long k_slice, long out_slice_stride, int n_slices, cudaStream_t st) {
    static std::atomic<unsigned long long> set_on{0};
    // at least 48 KB, so that at most four blocks (4 x 128 TMEM columns) share an SM
    const int smem = (int)std::max<size_t>(sizeof(GemmSmem<BBF>), 48 * 1024);
    cudaError_t e = smem_opt_in(gemm_tc_kernel<BBF, EPI>, smem, set_on);
    if (e != cudaSuccess) return e;
    const bool a_vec = sak == 1 && sam % 4 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
    const bool b_vec = sbk == 1 && sbn % (BBF ? 8 : 4) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
    dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + 127) / 128), (unsigned)n_slices);
    gemm_tc_kernel<BBF, EPI><<<grid, kThr, smem, st>>>(M, N, K, A, sam, sak, a_vec, B, sbn, sbk, b_vec, bias, aux,
                                                      ldaux, out0, out1, ldo, k_slice, out_slice_stride);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_tc(int epi, bool b_bf16, int M, int N, long K, const float *A, long sam, long sak,
                           const void *B, long sbn, long sbk, const float *bias, const float *aux, int ldaux,
                           float *out0, float *out1, int ldo, long k_slice, long out_slice_stride, int n_slices,
                           cudaStream_t st) {
    if (M <= 0 || N <= 0 || n_slices <= 0) return cudaSuccess;
    if (k_slice <= 0 || (long)n_slices * k_slice < K || M > (1 << 30)) return cudaErrorInvalidValue;
#define RX_GEMM_TC(BB, EP) \
    return gemm_tc_t<BB, EP>(M, N, K, A, sam, sak, B, sbn, sbk, bias, aux, ldaux, out0, out1, ldo, k_slice, \
                             out_slice_stride, n_slices, st)
    if (b_bf16) {
        if (epi == EPI_BIAS_GELU) RX_GEMM_TC(true, EPI_BIAS_GELU);
        if (epi == EPI_GELU_GRAD) RX_GEMM_TC(true, EPI_GELU_GRAD);
        if (epi == EPI_STORE) RX_GEMM_TC(true, EPI_STORE);
    } else {
        if (epi == EPI_STORE) RX_GEMM_TC(false, EPI_STORE);
    }
#undef RX_GEMM_TC
    return cudaErrorInvalidValue;
}

cudaError_t launch_infer_umma(const float *x, const float *s2, long n, int n_seg, long x_stride, long llr_stride,
                              const uint16_t *W1q, const float *b1, const uint16_t *W2q, const float *b2,
                              const uint16_t *W3q, const float *b3, float *llr, cudaStream_t st) {
    if (n <= 0 || n_seg <= 0) return cudaSuccess;
    if (n_seg > 1 && (x_stride < n || llr_stride < n)) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(W2q) & 15) != 0) return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> set_on{0};
    const int smem = (int)sizeof(InferSmem);
    cudaError_t e = smem_opt_in(infer_umma_kernel, smem, set_on);
    if (e != cudaSuccess) return e;
    const long tiles = (n + 127) / 128 * n_seg;
    // four blocks per SM hold all 512 TMEM columns (128 each); the shared
    // memory request keeps a fifth off the SM
    const int grid = (int)std::min<long>(tiles, 4L * sm_count());
    infer_umma_kernel<<<grid, kThr, smem, st>>>(x, s2, n, n_seg, x_stride, llr_stride, W1q, b1, W2q, b2, W3q, b3,
                                                llr);
    return cudaGetLastError();
}

// Read and clear the flag of a bounded wait that gave up (1) in any of the
// kernels above on the current device since the last call.
cudaError_t mlp_tc_status(unsigned int *flag) {
    const unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_mlp_tc_err, sizeof(unsigned int));
    if (e == cudaSuccess && *flag) e = cudaMemcpyToSymbol(g_mlp_tc_err, &zero, sizeof(unsigned int));
    return e;
}
