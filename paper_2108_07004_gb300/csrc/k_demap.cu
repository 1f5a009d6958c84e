// A5: exact soft demapping to bit LLRs, A6: BER / GMI / EVM counting.
//
//   LLR_i = ln sum_{j: b_i(j)=0} exp(-||z - s_j||^2 / sigma^2)
//         - ln sum_{j: b_i(j)=1} exp(-||z - s_j||^2 / sigma^2)
//
// One thread per symbol.  The table (label order) is read from the kernel's
// parameter space: every thread walks it in the same order, so the reads
// are uniform constant-bank loads.  All exponentials share one shift, the
// minimum distance g, plus a constant 2^120 headroom:
//   e_j = 2^{(g - d_j) log2(e) / sigma^2 + 120}
// so the M terms are computed once; the per-bit subset sums are built as a
// binary tree over the label bits (bit 0 splits even/odd labels, then pairs
// are summed and bit 1 splits the pairs, ...), about 3M additions instead
// of m*M.  A subset whose terms all lie below 2^-100 of the shift is
// recomputed from z with its own minimum as shift (then |LLR| > 150).
// Counting (Sec. 3 counts errors offline; here it is fused): hard bits are
// LLR < 0, errors against the reference label, the GMI term
// log2(1 + exp(-(1 - 2b) LLR)) per bit and the EVM sums; block partials are
// reduced in a fixed order by the last block of the launch.
#include "rx_internal.h"

namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kOff = 120.f;

__device__ __forceinline__ float softplus_bits(float x) {   // log2(1 + exp(x))
    return (fmaxf(x, 0.f) + log1pf(expf(-fabsf(x)))) * kLog2e;
}

template <int DIMS>
__device__ __forceinline__ float dist_to(float2 z0, float2 z1, const FmtDev &f, int j) {
    const float a0 = z0.x - f.pts[j][0], a1 = z0.y - f.pts[j][1];
    float d = fmaf(a0, a0, a1 * a1);
    if (DIMS == 4) {
        const float a2 = z1.x - f.pts[j][2], a3 = z1.y - f.pts[j][3];
        d = fmaf(a2, a2, fmaf(a3, a3, d));
    }
    return d;
}

// Rare path, for a lookup where some bit's subset sum fell below 2^-100 of
// the common shift: every subset gets its own minimum as shift.  Rewrites
// out[] and the counting terms of this lookup.
template <int DIMS, int MT, int MB>
__device__ __noinline__ void llr_table_slow(float2 z0, float2 z1, const FmtDev &f, float c2,
                                            float *out, int ref, int *nerr, float *gs) {
    int ne = 0;
    float g2 = 0.f;
    for (int bp = 0; bp < MB; ++bp) {
        float lg[2];
        for (int v = 0; v < 2; ++v) {
            float dm = 3.0e38f;
            for (int j = 0; j < MT; ++j)
                if (((j >> bp) & 1) == v) dm = fminf(dm, dist_to<DIMS>(z0, z1, f, j));
            float acc = 0.f;
            for (int j = 0; j < MT; ++j)
                if (((j >> bp) & 1) == v) acc += exp2f((dm - dist_to<DIMS>(z0, z1, f, j)) * c2);
            lg[v] = -dm * c2 + log2f(acc);
        }
        const float L = (lg[0] - lg[1]) * kLn2;
        out[MB - 1 - bp] = L;
        if (ref >= 0) {
            const int bit = (ref >> bp) & 1;
            ne += (int)((L < 0.f) != (bit != 0));
            g2 += softplus_bits(bit ? L : -L);
        }
    }
    *nerr = ne;
    *gs = g2;
}

// LLRs of one table lookup of z (DIMS 4: joint; DIMS 2: z0 alone), MB bits,
// written to out[0..MB-1] (MSB first).  When ref >= 0 (the reference label of
// this lookup) the hard-decision errors and the GMI terms are accumulated.
template <int DIMS, int MT, int MB>
__device__ __forceinline__ void llr_table(float2 z0, float2 z1, const FmtDev &f, float c2,
                                          float *out, float &g, int &jmin, int ref, int &nerr,
                                          float &gs) {
    float cur[MT];
#pragma unroll
    for (int j = 0; j < MT; ++j) cur[j] = dist_to<DIMS>(z0, z1, f, j);
    g = cur[0];
    jmin = 0;
#pragma unroll
    for (int j = 1; j < MT; ++j)
        if (cur[j] < g) { g = cur[j]; jmin = j; }
#pragma unroll
    for (int j = 0; j < MT; ++j) cur[j] = exp2f(fmaf(g - cur[j], c2, kOff));
    bool low = false;
    int ne = 0;
    float g2 = 0.f;
#pragma unroll
    for (int bp = 0; bp < MB; ++bp) {
        const int n = MT >> bp;
        float s0 = 0.f, s1 = 0.f;
#pragma unroll
        for (int i = 0; i < MT; i += 2)
            if (i < n) { s0 += cur[i]; s1 += cur[i + 1]; }
        low |= (s0 < 7.888609052e-31f) | (s1 < 7.888609052e-31f);   // 2^-100
        const float L = (__log2f(s0) - __log2f(s1)) * kLn2;
        out[MB - 1 - bp] = L;
        if (ref >= 0) {
            const int bit = (ref >> bp) & 1;
            ne += (int)((L < 0.f) != (bit != 0));
            g2 += softplus_bits(bit ? L : -L);
        }
#pragma unroll
        for (int i = 0; i < MT / 2; ++i)
            if (2 * i < n) cur[i] = cur[2 * i] + cur[2 * i + 1];
    }
    if (low) llr_table_slow<DIMS, MT, MB>(z0, z1, f, c2, out, ref, &ne, &g2);
    nerr += ne;
    gs += g2;
}

// 4D table of MT points with MB label bits, streaming form: the shift is the
// minimum distance from the orbit form (|z|^2 + |rep|^2 - 2 max(|P|,|Q|), no
// per-point state), then every point's exact distance and exponential is
// added to the two running subset sums of each label bit (the bit pattern of
// point j is known at compile time).  Twelve accumulators instead of 64
// stored terms keep the registers low; the result is the same sum.
template <int MT, int MB>
__device__ __forceinline__ void llr_4d_stream(float2 z0, float2 z1, const FmtDev &f, float c2,
                                              float *out, float &gmin, int &jmin, int ref,
                                              int &nerr, float &gs) {
    float g = 3.0e38f;
    const float zn = cnorm(z0) + cnorm(z1);
#pragma unroll
    for (int o = 0; o < 16; ++o) {
        if (o < f.n_orb) {
            const float P = z0.x * f.orb[o][0] + z0.y * f.orb[o][1] + z1.x * f.orb[o][2] + z1.y * f.orb[o][3];
            const float Q = z0.y * f.orb[o][0] - z0.x * f.orb[o][1] + z1.y * f.orb[o][2] - z1.x * f.orb[o][3];
            const float v = (f.S == 4) ? fmaxf(fabsf(P), fabsf(Q)) : (f.S == 2 ? fabsf(P) : P);
            g = fminf(g, zn + f.orbe[o] - 2.f * v);
        }
    }
    const float sh = fmaf(g, c2, kOff);      // exponent of point j: sh - d_j c2
    float s0[MB], s1[MB];
#pragma unroll
    for (int i = 0; i < MB; ++i) { s0[i] = 0.f; s1[i] = 0.f; }
    float dmin = 3.0e38f;
    int jm = 0;
    // groups of 8 points: the low 3 label bits are fixed per point, the high
    // bits per group (the group total is added to their subset sums)
#pragma unroll 1
    for (int g8 = 0; g8 < MT; g8 += 8) {
        float tot = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int j = g8 + u;
            const float d = dist_to<4>(z0, z1, f, j);
            if (d < dmin) { dmin = d; jm = j; }
            const float ej = exp2f(fmaf(-d, c2, sh));
            tot += ej;
#pragma unroll
            for (int i = 0; i < 3 && i < MB; ++i) {
                if ((u >> i) & 1) s1[i] += ej;
                else s0[i] += ej;
            }
        }
#pragma unroll
        for (int i = 3; i < MB; ++i) {
            if ((g8 >> i) & 1) s1[i] += tot;
            else s0[i] += tot;
        }
    }
    gmin = dmin;
    jmin = jm;
    bool low = false;
    int ne = 0;
    float g2 = 0.f;
#pragma unroll
    for (int bp = 0; bp < MB; ++bp) {
        low |= (s0[bp] < 7.888609052e-31f) | (s1[bp] < 7.888609052e-31f);   // 2^-100
        const float L = (__log2f(s0[bp]) - __log2f(s1[bp])) * kLn2;
        out[MB - 1 - bp] = L;
        if (ref >= 0) {
            const int bit = (ref >> bp) & 1;
            ne += (int)((L < 0.f) != (bit != 0));
            g2 += softplus_bits(bit ? L : -L);
        }
    }
    if (low) llr_table_slow<4, MT, MB>(z0, z1, f, c2, out, ref, &ne, &g2);
    nerr += ne;
    gs += g2;
}

template <int DIMS, int MT, int MB>
__global__ void __launch_bounds__(256, (DIMS == 4 ? 4 : 2))
demap_kernel(const float2 *__restrict__ z, long z_stride, long a, long e,
             const double *__restrict__ sigma2, int s2_stride, float *__restrict__ llr,
             long llr_stride, DemapCount cnt, const __grid_constant__ FmtDev f) {
    constexpr int M_OUT = (DIMS == 4) ? MB : 2 * MB;
    __shared__ float red[8][3];
    __shared__ int redn[8][2];
    __shared__ bool last;
    const int s = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long k = a + (long)blockIdx.x * blockDim.x + tid;
    const float c2 = 1.4426950408889634f / (float)sigma2[s * s2_stride];
    const float2 *zx = z + (long)s * 2 * z_stride;
    const float2 *zy = zx + z_stride;
    // per-thread counts in 32-bit / float (one symbol each); warp sums are
    // widened to float64 before the block and grid reductions
    int nerr = 0, ncnt = 0;
    float gsum = 0.f, en = 0.f, ed = 0.f;
    if (k < e) {
        const float2 z0 = zx[k - a], z1 = zy[k - a];
        const bool counted = cnt.ref_lab && k >= cnt.c0 && k < cnt.c1;
        const int ref = counted ? (int)cnt.ref_lab[(long)s * cnt.ref_stride + k] : -1;
        float *row = llr + (long)s * llr_stride + (k - a) * M_OUT;
        int ne = 0;
        float gs = 0.f, dist_min, dmin_energy;
        if (DIMS == 4) {
            float g;
            int jm;
            llr_4d_stream<MT, MB>(z0, z1, f, c2, row, g, jm, ref, ne, gs);
            dist_min = g;
            dmin_energy = f.pe[jm];
        } else {
            dist_min = 0.f;
            dmin_energy = 0.f;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const float2 zp = p ? z1 : z0;
                const int rp = ref < 0 ? -1 : (p ? (ref & ((1 << MB) - 1)) : (ref >> MB));
                float g;
                int jm;
                llr_table<2, MT, MB>(zp, zp, f, c2, row + p * MB, g, jm, rp, ne, gs);
                dist_min += g;
                dmin_energy += f.pe[jm];
            }
        }
        if (counted) {
            nerr = ne;
            ncnt = 1;
            gsum = gs;
            en = dist_min;
            ed = dmin_energy;
        }
    }
    if (!cnt.sd) return;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        nerr += __shfl_xor_sync(0xffffffffu, nerr, off);
        ncnt += __shfl_xor_sync(0xffffffffu, ncnt, off);
        gsum += __shfl_xor_sync(0xffffffffu, gsum, off);
        en += __shfl_xor_sync(0xffffffffu, en, off);
        ed += __shfl_xor_sync(0xffffffffu, ed, off);
    }
    if (lane == 0) {
        red[warp][0] = gsum; red[warp][1] = en; red[warp][2] = ed;
        redn[warp][0] = nerr; redn[warp][1] = ncnt;
    }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        unsigned long long n0 = 0, n1 = 0;
        for (int w = 0; w < 8; ++w) {
            t0 += red[w][0]; t1 += red[w][1]; t2 += red[w][2];
            n0 += redn[w][0]; n1 += redn[w][1];
        }
        double *pp = cnt.partial + ((long)s * gridDim.x + blockIdx.x) * 5;
        pp[0] = t0; pp[1] = t1; pp[2] = t2;
        pp[3] = (double)n0; pp[4] = (double)n1;
        __threadfence();
        const unsigned prev = atomicAdd(&cnt.sd[s].ticket_demap, 1u);
        last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    // the last block of this stream adds the partials: strided per thread, then
    // a fixed-order tree, so the sum does not depend on block timing
    __threadfence();
    const volatile double *pp = cnt.partial + (long)s * gridDim.x * 5;
    __shared__ double tr[5][256];
    double v[5] = {0, 0, 0, 0, 0};
    for (unsigned c = tid; c < gridDim.x; c += blockDim.x)
        for (int i = 0; i < 5; ++i) v[i] += pp[c * 5 + i];
    for (int i = 0; i < 5; ++i) tr[i][tid] = v[i];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
            for (int i = 0; i < 5; ++i) tr[i][tid] += tr[i][tid + w];
        __syncthreads();
    }
    if (tid == 0) {
        StreamDev &sd = cnt.sd[s];
        sd.gmi_sum += tr[0][0];
        sd.evm_num += tr[1][0];
        sd.evm_den += tr[2][0];
        sd.bit_errors += (unsigned long long)tr[3][0];
        sd.n_sym += (unsigned long long)tr[4][0];
        sd.sigma2 = sigma2[s * s2_stride];
        sd.ticket_demap = 0u;
    }
}

template <int DIMS, int MT, int MB>
cudaError_t demap_t(const float2 *z, long zs, long a, long e, const double *s2, int s2s, float *llr,
                    long ls, const DemapCount &cnt, int n_streams, const FmtDev &f, cudaStream_t st) {
    dim3 grid((unsigned)((e - a + 255) / 256), (unsigned)n_streams);
    demap_kernel<DIMS, MT, MB><<<grid, 256, 0, st>>>(z, zs, a, e, s2, s2s, llr, ls, cnt, f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_demap(const float2 *z, long z_stride, long z_off, long a, long e,
                         const double *sigma2, int sigma2_stride, float *llr, long llr_stride,
                         const DemapCount &cnt, int n_streams, const FmtDev &f, cudaStream_t st) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    const float2 *zz = z + z_off;
    if (f.dims == 4 && f.M == 64)
        return demap_t<4, 64, 6>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 4)
        return demap_t<2, 4, 2>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 16)
        return demap_t<2, 16, 4>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    return cudaErrorInvalidValue;
}
