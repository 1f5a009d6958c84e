// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "rx.h"
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#define RX_MAXM 128       // largest table (4D: 64 points; 2D: 128 points per polarisation)
// reference label of one 4D symbol (m bits, MSB first): up to 14 bits (two 2D labels of 7)
typedef uint16_t reflab_t;
#define RX_MAXB 64        // largest number of BPS test phases
#define RX_NCHUNK 10      // BPS ring of 32-symbol chunks

// Constellation and phase-search tables, passed to kernels by value
// (__grid_constant__), so that uniform reads come from the constant bank.
// 16-byte aligned so that the packed (64-bit) reads of csp are aligned.
struct __align__(16) FmtDev {
    int dims;             // 2 or 4
    int M;                // table size
    int m;                // bits per 4D symbol
    int m_pol;            // bits per table entry (dims 2) / m (dims 4)
    int S;                // rotational symmetry order used by the phase search (1, 2, 4)
    int n_orb;            // number of orbits (M / S)
    int B;                // BPS test phases
    float R2;             // CMA radius E|s|^4 / E|s|^2 (per-polarisation marginal)
    float pts[RX_MAXM][4];      // label order: (xr, xi, yr, yi) or (re, im, -, -)
    float ptsT[4][RX_MAXM];     // the same, component-major (labels j, j+1 adjacent: packed pairs)
    float pe[RX_MAXM];          // energy of each point
    float orb[RX_MAXM][4];      // orbit representatives
    float orbe[RX_MAXM];        // energy of each representative
    int orb_lab[RX_MAXM][4];    // label of representative o rotated by k quarter turns (k < S)
    float cs[RX_MAXB][2];       // cos, sin of the test phases phi_b
    float csp[RX_MAXB][4];      // (cos, cos, sin, sin) of phi_b, for packed pairs
    // the (at most 16) orbit representatives component-major (orbits o, o+1
    // adjacent: packed pairs) and their energies, +inf past n_orb
    float orbT[4][16];
    float orbeP[16];
};
static_assert(offsetof(FmtDev, csp) % 16 == 0, "packed phase table must be 16-byte aligned");
static_assert(offsetof(FmtDev, ptsT) % 8 == 0, "packed point pairs must be 8-byte aligned");
static_assert(alignof(FmtDev) == 16, "FmtDev alignment");
static_assert(offsetof(FmtDev, orbT) % 8 == 0 && offsetof(FmtDev, orbeP) % 8 == 0,
              "packed orbit pairs must be 8-byte aligned");

// Per-stream device state.
struct StreamDev {
    int32_t carry[2][2];            // unwrap carry [slot][m, b]
    unsigned long long bit_errors;
    unsigned long long n_sym;
    double gmi_sum;
    double evm_num;
    double evm_den;
    double sigma2;                  // noise variance of the current block
    unsigned int ticket_unwrap;
    unsigned int ticket_demap;
    int pad[2];
};

// ---- storage of the chain's intermediate samples -------------------------------
// The CDC output x and the FIR output y are stored as float32 pairs, or (the
// precision variant) as half or bfloat16 pairs; all arithmetic is float32.
enum { SK_F32 = 0, SK_F16 = 1, SK_BF16 = 2 };
template <int SK> struct Store;
template <> struct Store<SK_F32> {
    using T = float2;
    static __device__ __forceinline__ float2 ld(const T *p, long i) { return p[i]; }
    static __device__ __forceinline__ void st(T *p, long i, float2 v) { p[i] = v; }
};
template <> struct Store<SK_F16> {
    using T = __half2;
    static __device__ __forceinline__ float2 ld(const T *p, long i) { return __half22float2(p[i]); }
    static __device__ __forceinline__ void st(T *p, long i, float2 v) { p[i] = __float22half2_rn(v); }
};
template <> struct Store<SK_BF16> {
    using T = __nv_bfloat162;
    static __device__ __forceinline__ float2 ld(const T *p, long i) { return __bfloat1622float2(p[i]); }
    static __device__ __forceinline__ void st(T *p, long i, float2 v) { p[i] = __float22bfloat162_rn(v); }
};
inline size_t store_bytes(int sk) { return sk == SK_F32 ? sizeof(float2) : sizeof(__half2); }
// element i of a sample array of storage kind sk (a uniform branch)
__device__ __forceinline__ float2 ld_sample(const void *p, long i, int sk) {
    if (sk == SK_F16) return Store<SK_F16>::ld(static_cast<const __half2 *>(p), i);
    if (sk == SK_BF16) return Store<SK_BF16>::ld(static_cast<const __nv_bfloat162 *>(p), i);
    return static_cast<const float2 *>(p)[i];
}

// ---- complex helpers --------------------------------------------------------
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float cnorm(float2 a) { return a.x * a.x + a.y * a.y; }

// Unwrap increment between consecutive phase indices (integer form of
// phi_hat_k = phi_k + q round((phi_hat_{k-1} - phi_k) / q), round(x) = floor(x + 1/2)):
// floor((2 (b_{k-1} - b_k) + B) / (2B)).
__device__ __forceinline__ int unwrap_step(int bprev, int b, int B) {
    const int num = 2 * (bprev - b) + B;   // in [2 - B, 3B - 2]
    return num < 0 ? -1 : (num >= 2 * B ? 1 : 0);
}

// ---- packed float pairs (sm_100+ f32x2 arithmetic) ---------------------------
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {   // a * b + c, per lane
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// ---- launchers (return cudaError_t of the launch) -----------------------------
// Overlap-save frames f0 .. f1-1 (frame f writes outputs f*(n_fft-n_ov) ..
// (f+1)*(n_fft-n_ov) - 1); f1 < 0 means every frame of the ns samples.
cudaError_t launch_cdc(const float2 *in, void *out, long ns, int n_streams2, int n_fft,
                       int n_ov, const float2 *H, const float2 *tw, cudaStream_t st,
                       long f0 = 0, long f1 = -1, int sk = SK_F32);

// wl: widely-linear taps [S][2][2][2T] (T on x, then T on conj(x))
cudaError_t launch_fir(const void *x, long ns, const float2 *taps, long k0, long k1,
                       void *y, long y_stride, long y_off, int n_streams, int T,
                       cudaStream_t st, int sk = SK_F32, int sm_avail = 0, int wl = 0);

// opts of launch_lms: LMS_WL widely-linear taps; LMS_EXACT_DD the warp-wide
// nearest-point search on every DD update (no decisions taken ahead; the
// results are the same)
enum { LMS_WL = 1, LMS_EXACT_DD = 2 };
cudaError_t launch_lms(const void *x, long ns, const float2 *taps_in, float2 *taps_out,
                       long k0, int n_upd, const uint16_t *pcode, long pcode_stride,
                       int mode, int passes, unsigned long long u0, int n_cma, float mu,
                       const reflab_t *ref_lab, long ref_stride,
                       int n_streams, int T, const FmtDev &f, cudaStream_t st, int sk = SK_F32,
                       int opts = 0);

// Block LMS: groups of P (1..64) updates share the taps at the group start
// (mode 0 CMA, 1 DD, 2 CMA below n_cma updates then DD).
cudaError_t launch_lms_block(const void *x, long ns, const float2 *taps_in, float2 *taps_out, long k0,
                             int n_upd, const uint16_t *pcode, long pcode_stride, int mode,
                             unsigned long long u0, int n_cma, float mu, int P, int n_streams, int T,
                             const FmtDev &f, cudaStream_t st, int sk = SK_F32, int wl = 0);

// Training stage kernels on the equalised training span y [S][2][ystride]
// (storage kind sk): data-aided phase codes, and the output order / phase
// alignment of the taps [S][2][2][T] (in place).
cudaError_t launch_train_phase(const void *y, long ystride, const reflab_t *ref_lab, long ref_stride, int n,
                               int W, uint16_t *pcode, long pcode_stride, int32_t *carry, int carry_stride,
                               int n_streams, const FmtDev &f, cudaStream_t st, int sk = SK_F32);

cudaError_t launch_align(const void *y, long ystride, float2 *taps, const reflab_t *ref_lab,
                         long ref_stride, int n_train, int n_streams, int T, const FmtDev &f,
                         cudaStream_t st, int sk = SK_F32);

int bps_cta_range(int chunks);              // output symbols per BPS / unwrap block
int bps_chunks(long len, int n_streams, int sm_avail = 0);    // chunks per block for about one wave

// mdsum (optional, [S][n_blocks] float64): per-block sums of the minimum
// distance at the chosen phase, the decision-directed noise of the range
cudaError_t launch_bps(const void *y, long y_stride, long a, long e, long n_valid,
                       int W, uint8_t *bout, long bout_stride, long bout_off,
                       int *dsum, double *mdsum, int chunks, int n_streams, const FmtDev &f,
                       cudaStream_t st, int sk = SK_F32);

// Phase search with the correlations on the tensor cores (k_bps_tc.cu): 4D
// tables of 16 orbits with S = 4 and B a multiple of 16.  W: the B operand
// (bps_tc_table_floats(B) floats, built by bps_tc_table), device memory.
bool bps_tc_supported(const FmtDev &f);
size_t bps_tc_table_floats(int B);
void bps_tc_table(const FmtDev &f, float *out);
int bps_chunks_tc(long len, int n_streams, int sm_avail = 0);
cudaError_t launch_bps_tc(const void *y, long y_stride, long a, long e, long n_valid, int W, uint8_t *bout,
                          long bout_stride, long bout_off, int *dsum, double *mdsum, int chunks, int n_streams,
                          const float *Wg, const FmtDev &f, cudaStream_t st, int sk = SK_F32);
// 1 if a bounded wait of the tensor-core phase search gave up since the last
// call (the flag is then cleared)
cudaError_t bps_tc_status(unsigned int *flag);

cudaError_t launch_unwrap(const float2 *y, long y_stride, const uint8_t *b, long b_stride,
                          long b_off, long a, long e, const int *dsum,
                          const int32_t *carry_in, int carry_in_stride,
                          int32_t *carry_out, int carry_out_stride,
                          float2 *z, long z_stride, long z_off,
                          uint16_t *pcode, long pcode_stride, long pcode_off,
                          double *partial, double *sigma2_out, int sigma2_stride,
                          unsigned int *ticket, int ticket_stride, int chunks,
                          const double *mdsum, int n_streams, const FmtDev &f, cudaStream_t st);

cudaError_t launch_anchor(const uint8_t *b, long b_stride, const uint16_t *tcode, long t_stride,
                          int n, int32_t *carry, int carry_stride, int n_streams, int B, int S,
                          cudaStream_t st);

cudaError_t launch_dsum_from_b(const uint8_t *b, long b_stride, long a, long e, int *dsum,
                               int chunks, int n_streams, int B, cudaStream_t st);

struct DemapCount {
    const reflab_t *ref_lab;   // [S][N] labels of the reference (or null)
    long ref_stride;
    long c0, c1;              // count symbols with c0 <= k < c1 (stream index)
    StreamDev *sd;            // per-stream accumulators (or null)
    double *partial;          // [S][n_cta][3] scratch
};

// Optional symbol outputs of the chain: x4 [S][stride][4] float32 (Re, Im of
// z_X, z_Y) and s2 [S][stride] float32 (the block's sigma^2), at absolute
// symbol index k; null pointers are skipped.
struct SymOut {
    float *x4 = nullptr;
    float *s2 = nullptr;
    long stride = 0;
};

// Counting (errors, GMI, EVM) for LLRs made by the learned demapper, rows
// a .. e-1 of llr (row k - a, stride llr_stride per stream).
cudaError_t launch_count_llr(const float *llr, long llr_stride, const float *x4, long x_stride, long a, long e,
                             const double *sigma2, int s2_stride, const DemapCount &cnt, int n_streams,
                             const FmtDev &f, cudaStream_t st);

// De-rotation by the unwrapped phase fused with the LLRs and counting, for
// the chain: reads the equaliser output y and the BPS indices b (index k - a)
// with BPS's per-range increment sums dsum and minimum-distance sums mdsum
// ([S][n_cta], ranges of kR symbols), writes the phase codes and the LLRs
// (llr null: symbols only, into sym);
// sigma^2 = sum(mdsum) / (2 (e - a)) unless sigma2_fixed is given.  The
// block's sigma^2 goes to sigma2_out[s * s2_stride].  No z is written.
cudaError_t launch_derot_demap(const void *y, long y_stride, const uint8_t *b, long b_stride,
                               long a, long e, const int *dsum, const double *mdsum, int kR,
                               const int32_t *carry_in, int cin_stride, int32_t *carry_out,
                               int cout_stride, uint16_t *pcode, long pc_stride,
                               const double *sigma2_fixed, double *sigma2_out, int s2_stride,
                               float *llr, long llr_stride, const DemapCount &cnt, const SymOut &sym,
                               int n_streams, const FmtDev &f, cudaStream_t st, int sk = SK_F32,
                               int sm_avail = 0);
// number of partial-sum rows launch_derot_demap needs per stream
long derot_demap_ctas(long len, int n_streams, int sm_avail);

// SMs of the device (cached).  Launchers that size a grid to one wave take
// the number of SMs to plan for: the chain passes all of them less those the
// side-stream LMS holds (one per stream) while it runs beside them.
int sm_count();

// ---- learned demapper (k_mlp.cu) ----
// Device state of one MLP: float32 master parameters (order W1 [128][4],
// b1 [128], W2 [128][128], b2 [128], W3 [6][128], b3 [6]), Adam moments,
// the gradient, bfloat16 copies of the weights, and activation scratch.
struct MlpDev {
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    uint16_t *W1q = nullptr, *W2q = nullptr, *W3q = nullptr;
    // activations and scratch for up to cap samples
    long cap = 0;
    float *a1 = nullptr, *h1 = nullptr, *a2 = nullptr, *h2 = nullptr, *dO = nullptr, *da2 = nullptr,
          *da1 = nullptr, *loss_s = nullptr, *part = nullptr, *wpart = nullptr;
    long part_cap = 0;
    // kernel paths: training GEMMs (0: float32 SIMT, 1: tcgen05 with split
    // bfloat16 operands), inference (1: mma.sync, 2: tcgen05)
    int train_tc = 1, infer = 2;
};


cudaError_t mlp_alloc(MlpDev &d);
void mlp_free(MlpDev &d);
cudaError_t mlp_quantize(MlpDev &d, cudaStream_t st);
cudaError_t mlp_grad(MlpDev &d, const float *x, const float *s2, const uint8_t *bits, long n, float *loss,
                     cudaStream_t st);
cudaError_t mlp_adam(MlpDev &d, int t, float lr, cudaStream_t st);
cudaError_t mlp_infer(MlpDev &d, const float *x, const float *s2, long n, float *llr, cudaStream_t st);
// k_mlp_tc.cu: tcgen05 GEMM of the training steps (C = A B^T over K slices,
// strided float32 A, float32 or bfloat16 B, epilogue epi of mlp_dev.h), the
// fused tcgen05 inference, and the flag of their bounded waits
cudaError_t launch_gemm_tc(int epi, bool b_bf16, int M, int N, long K, const float *A, long sam, long sak,
                           const void *B, long sbn, long sbk, const float *bias, const float *aux, int ldaux,
                           float *out0, float *out1, int ldo, long k_slice, long out_slice_stride, int n_slices,
                           cudaStream_t st);
cudaError_t launch_infer_umma(const float *x, const float *s2, long n, int n_seg, long x_stride, long llr_stride,
                              const uint16_t *W1q, const float *b1, const uint16_t *W2q, const float *b2,
                              const uint16_t *W3q, const float *b3, float *llr, cudaStream_t st);
// inference of n_seg segments of n samples (segment g at rows g x_stride of
// x and sigma2, its LLRs at rows g llr_stride): one launch on the tcgen05
// path, one per segment on the mma.sync path
cudaError_t mlp_infer_seg(MlpDev &d, const float *x, const float *s2, long n, int n_seg, long x_stride,
                          float *llr, long llr_stride, cudaStream_t st);
cudaError_t mlp_tc_status(unsigned int *flag);

cudaError_t launch_demap(const float2 *z, long z_stride, long z_off, long a, long e,
                         const double *sigma2, int sigma2_stride, float *llr,
                         long llr_stride, const DemapCount &cnt, int n_streams,
                         const FmtDev &f, cudaStream_t st);

cudaError_t launch_ref_labels(const uint8_t *bits, reflab_t *lab, long n_sym, int n_streams,
                              int m, int dims, int m_pol, cudaStream_t st);
// rows i0 .. i1 - 1 only (bits [S][n_sym][m], labels [S][n_sym])
cudaError_t launch_ref_labels_rows(const uint8_t *bits, reflab_t *lab, long n_sym, long i0, long i1,
                                   int n_streams, int m, cudaStream_t st);
