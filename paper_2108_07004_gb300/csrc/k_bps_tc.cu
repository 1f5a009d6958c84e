// A4 phase search with the correlations on the tensor cores (tcgen05).
//
// For a 4D table closed under the joint rotation by pi/2 (S = 4) the phase
// search needs, per symbol y and test phase phi_b, the correlation of the
// de-rotated symbol with every orbit representative r_o:
//   P + jQ = e^{-j phi_b} c_o,   c_o = sum_p y_p conj(r_{o,p}),
// (see k_bps.cu: the orbit's best rotation is max(|P|, |Q|), and the phase
// shifted by pi/4 follows from |P| + |Q|).  P and Q are linear in the four
// real components Y = (Re y_X, Im y_X, Re y_Y, Im y_Y):
//   P = sum_c Y_c (cos phi_b a_c + sin phi_b b_c),
//   Q = sum_c Y_c (cos phi_b b_c - sin phi_b a_c),
//   a = (r0, r1, r2, r3), b = (-r1, r0, -r3, r2),
// so for a tile of 128 symbols all P and Q of the B/2 phase pairs and 16
// orbits are one product [128 x 4] . [4 x 16 B], a dense contraction with
// an inner dimension of 4.  It runs as tcgen05.mma kind::tf32 (M = 128,
// N = 256, K = 8) with the float32 operands split into TF32 high and low
// parts so that three partial products keep about 22 bits:
//   D  = [Y_hi, Y_lo] . [W_hi; W_hi]  (= Y_hi W_hi + Y_lo W_hi)
//   D += [Y_hi, Y_lo] . [W_lo; 0]     (= Y_hi W_lo),
// the two halves of K = 8 carrying the split, so no K is padding.  The
// accumulators land in tensor memory (TMEM); each warp reads the rows of its
// 32 symbols (tcgen05.ld) and the SIMT epilogue forms the orbit values, the
// minima over the orbits and the window sums exactly as the SIMT kernel
// does (same chunk ring, window and argmin code).
//
// Block: 8 warps, rounds of 8 chunks of 32 symbols (warp w: chunk 8r-1+w,
// tile w/4, TMEM lanes 32 (w%4) ..).  Per round and tile the A operand
// (128 x 8 TF32, canonical K-major layout without swizzle) is written by the
// warps; per sub-round of 8 phase pairs one thread issues the four MMAs
// (two tiles x two split terms) into 2 x 256 TMEM columns and commits them
// to an mbarrier; the warps wait (bounded), read and reduce.  The B operand
// (W, 2 x 16 B x 8 floats, host-built in the same layout) is copied into
// shared memory once per block.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "rx_internal.h"
#include "tc_dev.h"

namespace {

constexpr int kMaxChunks = 252;           // one block per SM: longer ranges than the SIMT kernel
constexpr int kThr = 256;
constexpr int kTileM = 128;
constexpr int kSubN = 256;              // MMA N: 8 phase pairs x 16 orbits x (P, Q)

__host__ __device__ __forceinline__ int range_tc(int chunks) { return 32 * chunks; }

// set when a bounded wait gave up (read and cleared by bps_tc_status)
__device__ unsigned int g_tc_err;

// ---- tcgen05 / mbarrier primitives (tc_dev.h) plus the TF32 kind ----------
using tc::fence_async_smem;
using tc::mbar_wait;
using tc::mma_commit;
using tc::sdesc;
using tc::smem_u32;
using tc::tmem_ld32;
__device__ __forceinline__ void tc_fence_before() { tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc::fence_after(); }

// instruction descriptor: kind::tf32, D float32, A and B TF32, both K-major
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                        // D format: float32
         | (2u << 7) | (2u << 10)           // A, B format: TF32
         | ((uint32_t)(N >> 3) << 17)
         | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(dtmem), "l"(a), "l"(b), "r"(idesc), "r"(acc) : "memory");
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of element (row, k) in a canonical K-major tile of K = 8 floats
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k) {
    return (uint32_t)((row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// The phase search of k_bps.cu for 4D tables of 16 orbits (S = 4), B a
// multiple of 16, with the correlations on the tensor cores.  Arguments and
// outputs as bps_kernel; W: the B operand in global memory (host-built).
__global__ void __launch_bounds__(kThr, 1)
bps_tc_kernel(const void *__restrict__ y, long y_stride, long a, long e, long n_valid, int W,
              uint8_t *__restrict__ bout, long bout_stride, int *__restrict__ dsum,
              double *__restrict__ mdsum, int n_cta, int chunks, int sk, const float4 *__restrict__ Wg,
              const __grid_constant__ FmtDev f) {
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    const int B = f.B, hb = B >> 1;
    const int NT = 16 * B;                                   // MMA outputs per symbol (all phase pairs)
    const int n_sub = NT / kSubN;                            // sub-rounds of 8 phase pairs
    const int kChunks = chunks, kR = range_tc(chunks);
    const int rounds = (kChunks + 2 + 7) / 8;
    constexpr int kRow = 33;
    // shared memory: W (hi, lo) | A tiles | ring of chunk prefixes | totals
    float *W1 = reinterpret_cast<float *>(sm_raw);
    float *W2 = W1 + NT * 8;
    float *At = W2 + NT * 8;                                  // [2 tiles][128 x 8]
    float *Eb = At + 2 * kTileM * 8;                          // [10][B][kRow]
    float *Tb = Eb + RX_NCHUNK * B * kRow;                    // [10][B]
    float *T2 = Tb + RX_NCHUNK * B;                           // [8][B]
    uint8_t *bsm = reinterpret_cast<uint8_t *>(T2 + 8 * B);  // [kR]
    __shared__ int red[8];
    __shared__ float redm[8];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int fail_sh;
    const int s = blockIdx.y, c = blockIdx.x;
    const long out0 = a + (long)c * kR;
    const long out1 = min(out0 + kR, e);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long yoff = (long)s * 2 * y_stride;
    const int hw = W >> 1;
    float md_acc = 0.f;

    // W into shared memory (already in the MMA layout), TMEM and the mbarrier
    {
        float4 *dst = reinterpret_cast<float4 *>(W1);
        for (int i = tid; i < NT * 4; i += kThr) dst[i] = Wg[i];   // W1 and W2: 2 x NT x 8 floats
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_slot)), "r"(512) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_sh = 0;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t bar = smem_u32(&mbar);
    const uint32_t idesc = idesc_tf32(kTileM, kSubN);
    const int tile = warp >> 2, quarter = warp & 3;
    // this warp's TMEM rows: lanes 32 quarter .., columns of its tile
    const uint32_t t_base = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(tile * kSubN);
    uint32_t phase = 0;
    const f32x2 CV = pk2(-2.f, -2.f), CU = pk2(-1.41421356237309515f, -1.41421356237309515f);

    for (int r = 0; r < rounds; ++r) {
        // ---- this warp's chunk: the A rows (TF32 split of Y) ----
        const int jc = 8 * r - 1 + warp;
        const bool chunk_ok = jc <= kChunks;
        const long i = out0 + 32L * jc + lane;
        const bool valid = chunk_ok && (i >= 0) && (i < n_valid);
        float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);
        if (valid) { ya = ld_sample(y, yoff + i, sk); yb = ld_sample(y, yoff + y_stride + i, sk); }
        const float yn0 = cnorm(ya) + cnorm(yb);
        {
            const float Y[4] = {ya.x, ya.y, yb.x, yb.y};
            float hi[4], lo[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                hi[k] = tf32_rna(Y[k]);
                lo[k] = tf32_rna(Y[k] - hi[k]);
            }
            const int row = 32 * quarter + lane;
            unsigned char *at = reinterpret_cast<unsigned char *>(At + tile * kTileM * 8);
            *reinterpret_cast<float4 *>(at + kmaj_off(row, 0)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<float4 *>(at + kmaj_off(row, 4)) = make_float4(lo[0], lo[1], lo[2], lo[3]);
        }
        fence_async_smem();
        const int slot = (jc + 1) % RX_NCHUNK;
        for (int sr = 0; sr < n_sub; ++sr) {
            tc_fence_before();
            __syncthreads();          // A written; the previous sub-round's TMEM reads done
            tc_fence_after();
            if (fail_sh) break;       // a wait gave up: no more work is issued
            if (tid == 0) {
                const uint32_t w1 = smem_u32(W1) + (uint32_t)(sr * (kSubN / 8) * 256);
                const uint32_t w2 = smem_u32(W2) + (uint32_t)(sr * (kSubN / 8) * 256);
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const uint64_t ad = sdesc(smem_u32(At + t * kTileM * 8), 128, 256);
                    const uint32_t dt = tmem + (uint32_t)(t * kSubN);
                    mma_tf32(dt, ad, sdesc(w1, 128, 256), idesc, 0);
                    mma_tf32(dt, ad, sdesc(w2, 128, 256), idesc, 1);
                }
                mma_commit(bar);
            }
            const bool ok = mbar_wait(bar, phase);
            phase ^= 1u;
            if (!ok) fail_sh = 1;
            tc_fence_after();
            // ---- epilogue: 8 phase pairs of this sub-round ----
#pragma unroll 1
            for (int q = 0; q < kSubN / 32; ++q) {
                float v[32];
                tmem_ld32(t_base + (uint32_t)(32 * q), v);
                const int b = sr * (kSubN / 32) + q;         // phase pair b, b + B/2
                float a0 = 3.0e38f, a1 = 3.0e38f;
#pragma unroll
                for (int o = 0; o < 16; o += 2) {
                    const float P = v[2 * o], Q = v[2 * o + 1], R = v[2 * o + 2], U = v[2 * o + 3];
                    const float v0 = fmaxf(fabsf(P), fabsf(Q)), u0 = fabsf(P) + fabsf(Q);
                    const float v1 = fmaxf(fabsf(R), fabsf(U)), u1 = fabsf(R) + fabsf(U);
                    const f32x2 EO = pk2(f.orbe[o], f.orbe[o + 1]);
                    float d0, d1, h0, h1;
                    upk2(fma2(CV, pk2(v0, v1), EO), d0, d1);
                    upk2(fma2(CU, pk2(u0, u1), EO), h0, h1);
                    a0 = fmin3(a0, d0, d1);
                    a1 = fmin3(a1, h0, h1);
                }
                if (chunk_ok) {
                    Eb[(slot * B + b) * kRow + lane] = valid ? yn0 + a0 : 0.f;
                    Eb[(slot * B + b + hb) * kRow + lane] = valid ? yn0 + a1 : 0.f;
                }
            }
        }
        __syncwarp();
        if (chunk_ok) {
            // exclusive prefix of every test phase's row over the chunk
            for (int b = lane; b < B; b += 32) {
                float *row = Eb + (slot * B + b) * kRow;
                float run = 0.f;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float x = row[j];
                    row[j] = run;
                    run += x;
                }
                Tb[slot * B + b] = run;
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- window costs and argmin for output chunk oc (as bps_kernel) ----
        const int oc = 8 * r - 2 + warp;
        float *t2 = T2 + warp * B;
        if (oc >= 0 && oc < kChunks) {
            const int sa = oc % RX_NCHUNK, sb = (oc + 1) % RX_NCHUNK;
            for (int b = lane; b < B; b += 32) t2[b] = Tb[sa * B + b] + Tb[sb * B + b];
        }
        __syncwarp();
        if (oc >= 0 && oc < kChunks) {
            const long k = out0 + 32L * oc + lane;
            if (k < out1) {
                const int i0 = 32 * oc + lane - hw, i1 = 32 * oc + lane + hw;
                const int c0 = (i0 >= 0) ? (i0 >> 5) : -1;
                const int l0 = i0 - 32 * c0;
                const int c1 = i1 >> 5, l1 = i1 - 32 * c1;
                const int s0 = (c0 + 1) % RX_NCHUNK, s1 = (c1 + 1) % RX_NCHUNK;
                const int smid = (c0 + 2) % RX_NCHUNK;
                float best = 3.0e38f;
                int bb = 0;
                const float *e0 = Eb + s0 * B * kRow + l0, *e1 = Eb + s1 * B * kRow + l1;
                if (c0 == oc - 1 && c1 == oc + 1) {
#pragma unroll 4
                    for (int b = 0; b < B; ++b) {
                        const float cst = (t2[b] - e0[b * kRow]) + e1[b * kRow];
                        if (cst < best) { best = cst; bb = b; }
                    }
                } else if (c0 == c1) {
                    for (int b = 0; b < B; ++b) {
                        const float cst = e1[b * kRow] - e0[b * kRow];
                        if (cst < best) { best = cst; bb = b; }
                    }
                } else {
                    for (int b = 0; b < B; ++b) {
                        float cst = Tb[s0 * B + b] - e0[b * kRow];
                        if (c1 - c0 == 2) cst += Tb[smid * B + b];
                        cst += e1[b * kRow];
                        if (cst < best) { best = cst; bb = b; }
                    }
                }
                bsm[k - out0] = (uint8_t)bb;
                bout[(long)s * bout_stride + (k - a)] = (uint8_t)bb;
                const int sc = (oc + 1) % RX_NCHUNK;
                const float hi = (lane < 31) ? Eb[(sc * B + bb) * kRow + lane + 1] : Tb[sc * B + bb];
                md_acc += hi - Eb[(sc * B + bb) * kRow + lane];
            }
        }
        __syncthreads();
    }
    // ---- unwrap increments inside this block's range ----
    int acc = 0;
    const int nloc = (int)(out1 - out0);
    for (int t = tid + 1; t < nloc; t += kThr) acc += unwrap_step(bsm[t - 1], bsm[t], B);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        md_acc += __shfl_xor_sync(0xffffffffu, md_acc, off);
    }
    if (lane == 0) { red[warp] = acc; redm[warp] = md_acc; }
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        double mt = 0.0;
        for (int w = 0; w < 8; ++w) { tot += red[w]; mt += (double)redm[w]; }
        dsum[s * n_cta + c] = tot;
        if (mdsum) mdsum[s * n_cta + c] = mt;
        if (fail_sh) atomicOr(&g_tc_err, 1u);
    }
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

}  // namespace

size_t bps_tc_table_floats(int B) { return (size_t)2 * 16 * B * 8; }

// Output chunks per block for about one wave of one block per SM.
int bps_chunks_tc(long len, int n_streams, int sm_avail) {
    if (sm_avail <= 0) sm_avail = sm_count();
    const long per_stream = std::max(1L, (long)sm_avail / std::max(1, n_streams));
    const long nch = std::max(1L, (len + 31) / 32);
    long c = (nch + per_stream - 1) / per_stream;
    c = std::max<long>(c, 6);
    c = std::min<long>(c, kMaxChunks);
    return (int)c;
}

// B operand of bps_tc_kernel for the table's 16 orbits and B test phases:
// W1 = [W_hi; W_hi], W2 = [W_lo; 0] (K = 8 each), outputs n = 32 p + 2 o + q
// (phase pair p, orbit o, q = 0: P, 1: Q), canonical K-major layout.
void bps_tc_table(const FmtDev &f, float *out) {
    const int B = f.B, NT = 16 * B;
    unsigned char *w1 = reinterpret_cast<unsigned char *>(out);
    unsigned char *w2 = w1 + (size_t)NT * 8 * sizeof(float);
    auto tf32 = [](double x) {
        // round to nearest with 10 explicit mantissa bits (ties away), as cvt.rna.tf32
        float v = (float)x;
        uint32_t u;
        std::memcpy(&u, &v, 4);
        if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
        float r;
        std::memcpy(&r, &u, 4);
        return r;
    };
    for (int p = 0; p < B / 2; ++p) {
        const double cs = f.cs[p][0], sn = f.cs[p][1];
        for (int o = 0; o < 16; ++o) {
            const double r0 = f.orb[o][0], r1 = f.orb[o][1], r2 = f.orb[o][2], r3 = f.orb[o][3];
            const double av[4] = {r0, r1, r2, r3}, bv[4] = {-r1, r0, -r3, r2};
            for (int q = 0; q < 2; ++q) {
                const int n = 32 * p + 2 * o + q;
                for (int k = 0; k < 4; ++k) {
                    const double w = q == 0 ? cs * av[k] + sn * bv[k] : cs * bv[k] - sn * av[k];
                    const float hi = tf32(w), lo = tf32(w - (double)hi);
                    const float vals1[2] = {hi, hi}, vals2[2] = {lo, 0.f};
                    for (int half = 0; half < 2; ++half) {
                        std::memcpy(w1 + kmaj_off(n, 4 * half + k), &vals1[half], 4);
                        std::memcpy(w2 + kmaj_off(n, 4 * half + k), &vals2[half], 4);
                    }
                }
            }
        }
    }
}

bool bps_tc_supported(const FmtDev &f) { return f.dims == 4 && f.n_orb == 16 && f.S == 4 && f.B % 16 == 0; }

cudaError_t launch_bps_tc(const void *y, long y_stride, long a, long e, long n_valid, int W, uint8_t *bout,
                          long bout_stride, long bout_off, int *dsum, double *mdsum, int chunks, int n_streams,
                          const float *Wg, const FmtDev &f, cudaStream_t st, int sk) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    if (chunks < 1 || chunks > kMaxChunks || !bps_tc_supported(f) || !Wg) return cudaErrorInvalidValue;
    const int kR = range_tc(chunks);
    const int n_cta = (int)((e - a + kR - 1) / kR);
    const int B = f.B;
    const size_t smem = sizeof(float) * (bps_tc_table_floats(B) + 2 * kTileM * 8 + RX_NCHUNK * B * 33 +
                                         RX_NCHUNK * B + 8 * B) + kR + 16;
    constexpr size_t kMax = sizeof(float) * ((size_t)2 * 16 * RX_MAXB * 8 + 2 * kTileM * 8 + RX_NCHUNK * RX_MAXB * 33 +
                                             RX_NCHUNK * RX_MAXB + 8 * RX_MAXB) + 32 * kMaxChunks + 16;
    if (smem > kMax) return cudaErrorInvalidValue;
    // at least 116 KB, so that no two blocks share an SM: each holds all 512
    // TMEM columns for its life
    const size_t smem_req = std::max<size_t>(smem, 116 * 1024);
    static std::atomic<unsigned long long> set_on{0};
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev >= 64 || !((set_on.load(std::memory_order_relaxed) >> dev) & 1ull)) {
        err = cudaFuncSetAttribute(bps_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMax);
        if (err != cudaSuccess) return err;
        if (dev < 64) set_on.fetch_or(1ull << dev, std::memory_order_relaxed);
    }
    dim3 grid((unsigned)n_cta, (unsigned)n_streams);
    bps_tc_kernel<<<grid, kThr, smem_req, st>>>(y, y_stride, a, e, n_valid, W, bout + bout_off, bout_stride, dsum,
                                            mdsum, n_cta, chunks, sk, reinterpret_cast<const float4 *>(Wg), f);
    return cudaGetLastError();
}

// Read and clear the flag of a bounded wait that gave up (1) in any
// bps_tc_kernel launch on the current device since the last call.
cudaError_t bps_tc_status(unsigned int *flag) {
    const unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_tc_err, sizeof(unsigned int));
    if (e == cudaSuccess && *flag) e = cudaMemcpyToSymbol(g_tc_err, &zero, sizeof(unsigned int));
    return e;
}
