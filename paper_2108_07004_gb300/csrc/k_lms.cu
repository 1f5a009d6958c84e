// A3: block-wise adaptation of the 2x2 butterfly (CMA, then DD-LMS).
//
// The recursion is sequential, so one warp runs it per stream (Sec. 2: the
// adaptive equaliser is the hard-to-parallelise step; the paper runs it on
// its own processing stream next to the parallel kernels, as the library
// does when the tap lag is >= 2).  Lane (q, p, j) holds the taps
// h_qp[j + 8 i]; an update is
//   y_q   = sum conj(h_qp[t]) x_p[2k + D - t]       (lane MACs + 4 xor-shuffles)
//   CMA:  e_q = (R^2 - |y_q|^2) y_q
//   DD:   z = y exp(-j phi_k); d = nearest table point (orbit per lane,
//         (distance, label) min over 16 lanes, ties -> lowest label);
//         e_q = d_q exp(j phi_k) - y_q
//   h_qp[t] += mu conj(e_q) x_p[2k + D - t]
// The samples of up to 1024 updates are staged in shared memory by the whole
// block before the warp runs through them.
//
// The start-up training alignment (Sec. 2: the equaliser first converges on
// a known sequence) is align_kernel: it correlates the equalised training
// span with the known symbols and fixes the output order and phases.
#include "rx_internal.h"

namespace {

constexpr int kCH = 1024;

struct Tables {
    float4 orb[RX_MAXM];
    float orbe[RX_MAXM];
    int orblab[RX_MAXM][4];
    float4 pts[RX_MAXM];
};

__device__ __forceinline__ void load_tables(Tables &tb, const FmtDev &f) {
    for (int i = threadIdx.x; i < f.n_orb; i += blockDim.x) {
        tb.orb[i] = make_float4(f.orb[i][0], f.orb[i][1], f.orb[i][2], f.orb[i][3]);
        tb.orbe[i] = f.orbe[i];
        for (int k = 0; k < 4; ++k) tb.orblab[i][k] = f.orb_lab[i][k];
    }
    for (int i = threadIdx.x; i < f.M; i += blockDim.x)
        tb.pts[i] = make_float4(f.pts[i][0], f.pts[i][1], f.pts[i][2], f.pts[i][3]);
}

__device__ __forceinline__ unsigned long long shfl_xor_u64(unsigned long long v, int m) {
    unsigned lo = __shfl_xor_sync(0xffffffffu, (unsigned)v, m);
    unsigned hi = __shfl_xor_sync(0xffffffffu, (unsigned)(v >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

// best rotation of an orbit given P + jQ = sum_p z_p conj(rep_p):
// Re of the correlation with rep * j^k is P, Q, -P, -Q for k = 0..3.
__device__ __forceinline__ void best_rot(float P, float Q, int S, float &v, int &k) {
    if (S == 4) {
        const float aP = fabsf(P), aQ = fabsf(Q);
        if (aP >= aQ) { v = aP; k = P >= 0.f ? 0 : 2; }
        else          { v = aQ; k = Q >= 0.f ? 1 : 3; }
    } else if (S == 2) {
        v = fabsf(P); k = P >= 0.f ? 0 : 1;
    } else {
        v = P; k = 0;
    }
}

// Nearest-point label, distributed over the 16 lanes of each half warp.
// DIMS 4: both halves decide the joint point of (z0, z1).
// DIMS 2: half q decides the point of its own polarisation zq.
template <int DIMS>
__device__ __forceinline__ int decide_warp(float2 z0, float2 z1, float2 zq, const Tables &tb,
                                           const FmtDev &f, int lane) {
    const int o = lane & 15;
    unsigned long long key = ~0ull;
    if (o < f.n_orb) {
        const float4 r = tb.orb[o];
        float P, Q, zn;
        if (DIMS == 4) {
            P = z0.x * r.x + z0.y * r.y + z1.x * r.z + z1.y * r.w;
            Q = z0.y * r.x - z0.x * r.y + z1.y * r.z - z1.x * r.w;
            zn = cnorm(z0) + cnorm(z1);
        } else {
            P = zq.x * r.x + zq.y * r.y;
            Q = zq.y * r.x - zq.x * r.y;
            zn = cnorm(zq);
        }
        float v;
        int k;
        best_rot(P, Q, f.S, v, k);
        const float dist = fmaxf(zn + tb.orbe[o] - 2.f * v, 0.f);
        key = ((unsigned long long)__float_as_uint(dist) << 32) | (unsigned)tb.orblab[o][k];
    }
#pragma unroll
    for (int m = 1; m < 16; m <<= 1) {
        unsigned long long other = shfl_xor_u64(key, m);
        key = other < key ? other : key;
    }
    return (int)(key & 0xffffffffu);
}

template <int T, int DIMS>
__global__ void __launch_bounds__(256)
lms_kernel(const float2 *__restrict__ x, long ns, const float2 *__restrict__ taps_in,
           float2 *__restrict__ taps_out, long k0, int n_upd, const uint16_t *__restrict__ pcode,
           long pcode_stride, int mode, int passes, unsigned long long u0, int n_cma, float mu,
           const uint8_t *__restrict__ ref_lab, long ref_stride, const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    constexpr int NSX = 2 * kCH + 2 * D;
    constexpr int NT = (T + 7) / 8;
    __shared__ float2 xs[2][NSX];
    __shared__ uint16_t pc[kCH];
    __shared__ uint8_t rl[kCH];
    __shared__ Tables tb;
    const int s = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane >> 4, p = (lane >> 3) & 1, j = lane & 7;
    load_tables(tb, f);

    float2 h[NT];
#pragma unroll
    for (int i = 0; i < NT; ++i) {
        const int t = j + 8 * i;
        h[i] = (t < T) ? taps_in[(((long)s * 2 + q) * 2 + p) * T + t] : make_float2(0.f, 0.f);
    }
    const float2 *xsrc = x + (long)s * 2 * ns;
    unsigned long long u = u0;
    for (int pass = 0; pass < passes; ++pass) {
        for (int c0 = 0; c0 < n_upd; c0 += kCH) {
            const int n = min(kCH, n_upd - c0);
            const long kb = k0 + c0;
            const int nsx = 2 * n + 2 * D;
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * nsx; i += blockDim.x) {
                const int pp = i / nsx, jj = i - pp * nsx;
                const long g = 2 * kb - D + jj;
                xs[pp][jj] = (g >= 0 && g < ns) ? xsrc[(long)pp * ns + g] : make_float2(0.f, 0.f);
            }
            if (mode != 0)
                for (int i = threadIdx.x; i < n; i += blockDim.x)
                    pc[i] = pcode[(long)s * pcode_stride + kb + i];
            if (mode == 3)
                for (int i = threadIdx.x; i < n; i += blockDim.x)
                    rl[i] = ref_lab[(long)s * ref_stride + kb + i];
            __syncthreads();
            if (warp != 0) continue;

            float2 xv[NT], xn[NT];
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const int t = j + 8 * i;
                xn[i] = (t < T) ? xs[p][2 * D - t] : make_float2(0.f, 0.f);
            }
            for (int kk = 0; kk < n; ++kk, ++u) {
#pragma unroll
                for (int i = 0; i < NT; ++i) xv[i] = xn[i];
                if (kk + 1 < n) {
#pragma unroll
                    for (int i = 0; i < NT; ++i) {
                        const int t = j + 8 * i;
                        if (t < T) xn[i] = xs[p][2 * (kk + 1) + 2 * D - t];
                    }
                }
                float2 part = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    part.x += h[i].x * xv[i].x + h[i].y * xv[i].y;
                    part.y += h[i].x * xv[i].y - h[i].y * xv[i].x;
                }
#pragma unroll
                for (int m = 1; m < 16; m <<= 1) {
                    part.x += __shfl_xor_sync(0xffffffffu, part.x, m);
                    part.y += __shfl_xor_sync(0xffffffffu, part.y, m);
                }
                const float2 yq = part;
                const bool cma = (mode == 0) || (mode == 2 && u < (unsigned long long)n_cma);
                float2 e;
                if (cma) {
                    const float g = f.R2 - cnorm(yq);
                    e = make_float2(g * yq.x, g * yq.y);
                } else {
                    const unsigned code = pc[kk];
                    const int b = min((int)(code & 255), f.B - 1), mq = (code >> 8) & 3;
                    float2 r = make_float2(f.cs[b][0], f.cs[b][1]);   // exp(j phi_b)
                    const int qt = mq * (4 / f.S);   // quarter turns of exp(j mq 2pi/S)
                    for (int i = 0; i < qt; ++i) r = make_float2(-r.y, r.x);
                    float2 yo;
                    yo.x = __shfl_xor_sync(0xffffffffu, yq.x, 16);
                    yo.y = __shfl_xor_sync(0xffffffffu, yq.y, 16);
                    const float2 y0 = q ? yo : yq, y1 = q ? yq : yo;
                    int lab;
                    if (mode == 3) {          // data-aided: the known symbol
                        lab = rl[kk];
                        if (DIMS == 2) lab = q ? (lab & ((1 << f.m_pol) - 1)) : (lab >> f.m_pol);
                    } else {
                        const float2 z0 = cmulc(r, y0), z1 = cmulc(r, y1), zq = cmulc(r, yq);
                        lab = decide_warp<DIMS>(z0, z1, zq, tb, f, lane);
                    }
                    const float4 pt = tb.pts[lab];
                    float2 d;
                    if (DIMS == 4) d = q ? make_float2(pt.z, pt.w) : make_float2(pt.x, pt.y);
                    else d = make_float2(pt.x, pt.y);
                    e = csub(cmul(d, r), yq);
                }
                const float2 ce = make_float2(mu * e.x, -mu * e.y);   // mu conj(e)
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    h[i].x += ce.x * xv[i].x - ce.y * xv[i].y;
                    h[i].y += ce.x * xv[i].y + ce.y * xv[i].x;
                }
            }
        }
    }
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            const int t = j + 8 * i;
            if (t < T) taps_out[(((long)s * 2 + q) * 2 + p) * T + t] = h[i];
        }
    }
}

// ---------------------------------------------------------------------------
// training alignment
// ---------------------------------------------------------------------------
template <int T, int DIMS>
__global__ void __launch_bounds__(256)
align_kernel(const float2 *__restrict__ x, long ns, float2 *__restrict__ taps,
             const uint8_t *__restrict__ ref_lab, long ref_stride, int n_train,
             const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    __shared__ float2 hs[4 * T];
    __shared__ double red[8][256];
    __shared__ float2 rot[2];
    __shared__ int src[2];
    const int s = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < 4 * T; i += 256) hs[i] = taps[(long)s * 4 * T + i];
    __syncthreads();
    const float2 *xs = x + (long)s * 2 * ns;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // C[q][p] re, im
    for (int k = tid; k < n_train; k += 256) {
        float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp)
                for (int t = 0; t < T; ++t) {
                    const long g = 2L * k + D - t;
                    if (g < 0 || g >= ns) continue;
                    const float2 hv = hs[(qq * 2 + pp) * T + t];
                    const float2 xv = xs[(long)pp * ns + g];
                    y[qq] = cadd(y[qq], cmulc(hv, xv));
                }
        const int lab = ref_lab[(long)s * ref_stride + k];
        float2 sp[2];
        if (DIMS == 4) {
            sp[0] = make_float2(f.pts[lab][0], f.pts[lab][1]);
            sp[1] = make_float2(f.pts[lab][2], f.pts[lab][3]);
        } else {
            const int lx = lab >> f.m_pol, ly = lab & ((1 << f.m_pol) - 1);
            sp[0] = make_float2(f.pts[lx][0], f.pts[lx][1]);
            sp[1] = make_float2(f.pts[ly][0], f.pts[ly][1]);
        }
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp) {
                const float2 c = cmulc(sp[pp], y[qq]);   // y_q conj(s_p)
                acc[(qq * 2 + pp) * 2] += c.x;
                acc[(qq * 2 + pp) * 2 + 1] += c.y;
            }
    }
    for (int i = 0; i < 8; ++i) red[i][tid] = acc[i];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w)
            for (int i = 0; i < 8; ++i) red[i][tid] += red[i][tid + w];
        __syncthreads();
    }
    if (tid == 0) {
        double C[2][2][2];
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp) {
                C[qq][pp][0] = red[(qq * 2 + pp) * 2][0];
                C[qq][pp][1] = red[(qq * 2 + pp) * 2 + 1][0];
            }
        auto n2 = [&](int a, int b) { return C[a][b][0] * C[a][b][0] + C[a][b][1] * C[a][b][1]; };
        const bool swap = (n2(0, 1) + n2(1, 0)) > (n2(0, 0) + n2(1, 1));
        for (int pn = 0; pn < 2; ++pn) {
            const int qo = swap ? 1 - pn : pn;
            src[pn] = qo;
            const double re = C[qo][pn][0], im = C[qo][pn][1];
            const double a = sqrt(re * re + im * im);
            rot[pn] = a > 0 ? make_float2((float)(re / a), (float)(im / a)) : make_float2(1.f, 0.f);
        }
    }
    __syncthreads();
    for (int i = tid; i < 4 * T; i += 256) {
        const int pn = i / (2 * T), rest = i - pn * 2 * T;
        taps[(long)s * 4 * T + i] = cmul(hs[src[pn] * 2 * T + rest], rot[pn]);
    }
}

// Data-aided phase codes over the training span [0, n):
//   R_k = sum_{i in [k - W/2, k + W/2) within the span} sum_p y_p[i] conj(s_p[i]),
//   n_k = floor(arg(R_k) / (2 pi / (S B)) + 1/2), code = b | (m mod S) << 8 with
//   b = n_k + B/2 - m B, m = floor((n_k + B/2) / B).
template <int T, int DIMS>
__global__ void __launch_bounds__(256)
train_phase_kernel(const float2 *__restrict__ x, long ns, const float2 *__restrict__ taps,
                   const uint8_t *__restrict__ ref_lab, long ref_stride, int n, int W,
                   uint16_t *__restrict__ pcode, long pcode_stride, int32_t *__restrict__ carry,
                   int carry_stride, const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    extern __shared__ float2 rs[];      // [n] per-symbol correlations
    __shared__ float2 hs[4 * T];
    const int s = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < 4 * T; i += 256) hs[i] = taps[(long)s * 4 * T + i];
    __syncthreads();
    const float2 *xs = x + (long)s * 2 * ns;
    for (int k = tid; k < n; k += 256) {
        float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp)
                for (int t = 0; t < T; ++t) {
                    const long g = 2L * k + D - t;
                    if (g < 0 || g >= ns) continue;
                    y[qq] = cadd(y[qq], cmulc(hs[(qq * 2 + pp) * T + t], xs[(long)pp * ns + g]));
                }
        const int lab = ref_lab[(long)s * ref_stride + k];
        float2 s0, s1;
        if (DIMS == 4) {
            s0 = make_float2(f.pts[lab][0], f.pts[lab][1]);
            s1 = make_float2(f.pts[lab][2], f.pts[lab][3]);
        } else {
            const int lx = lab >> f.m_pol, ly = lab & ((1 << f.m_pol) - 1);
            s0 = make_float2(f.pts[lx][0], f.pts[lx][1]);
            s1 = make_float2(f.pts[ly][0], f.pts[ly][1]);
        }
        rs[k] = cadd(cmulc(s0, y[0]), cmulc(s1, y[1]));   // sum_p y_p conj(s_p)
    }
    __syncthreads();
    const int B = f.B, S = f.S;
    const double step = 2.0 * 3.14159265358979323846 / ((double)S * B);
    for (int k = tid; k < n; k += 256) {
        float2 R = make_float2(0.f, 0.f);
        const int i0 = max(0, k - W / 2), i1 = min(n, k + W / 2);
        for (int i = i0; i < i1; ++i) R = cadd(R, rs[i]);
        const int nk = (int)floor((double)atan2f(R.y, R.x) / step + 0.5);
        const int m = (int)floor((double)(nk + B / 2) / B);
        const int b = nk + B / 2 - m * B;
        const int mq = ((m % S) + S) % S;
        pcode[(long)s * pcode_stride + k] = (uint16_t)(b | (mq << 8));
        if (k == 0 && carry) {                 // the unwrap starts from this phase
            carry[s * carry_stride + 0] = mq;
            carry[s * carry_stride + 1] = b;
        }
    }
}

__global__ void ref_labels_kernel(const uint8_t *__restrict__ bits, uint8_t *__restrict__ lab,
                                  long n, int m) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= n) return;
    const uint8_t *b = bits + ((long)s * n + i) * m;
    int v = 0;
    for (int c = 0; c < m; ++c) v = (v << 1) | (b[c] & 1);
    lab[(long)s * n + i] = (uint8_t)v;
}

template <int T>
cudaError_t lms_dispatch_dims(const float2 *x, long ns, const float2 *ti, float2 *to, long k0,
                              int n_upd, const uint16_t *pcode, long pstride, int mode,
                              int passes, unsigned long long u0, int n_cma, float mu,
                              const uint8_t *ref, long rstride, int S, const FmtDev &f,
                              cudaStream_t st) {
    if (f.dims == 4)
        lms_kernel<T, 4><<<S, 256, 0, st>>>(x, ns, ti, to, k0, n_upd, pcode, pstride, mode, passes,
                                            u0, n_cma, mu, ref, rstride, f);
    else
        lms_kernel<T, 2><<<S, 256, 0, st>>>(x, ns, ti, to, k0, n_upd, pcode, pstride, mode, passes,
                                            u0, n_cma, mu, ref, rstride, f);
    return cudaGetLastError();
}

template <int T>
cudaError_t align_dispatch(const float2 *x, long ns, float2 *taps, const uint8_t *ref,
                           long rstride, int n_train, int S, const FmtDev &f, cudaStream_t st) {
    if (f.dims == 4)
        align_kernel<T, 4><<<S, 256, 0, st>>>(x, ns, taps, ref, rstride, n_train, f);
    else
        align_kernel<T, 2><<<S, 256, 0, st>>>(x, ns, taps, ref, rstride, n_train, f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lms(const float2 *x, long ns, const float2 *taps_in, float2 *taps_out, long k0,
                       int n_upd, const uint16_t *pcode, long pcode_stride, int mode, int passes,
                       unsigned long long u0, int n_cma, float mu, const uint8_t *ref_lab,
                       long ref_stride, int n_streams, int T, const FmtDev &f, cudaStream_t st) {
    if (n_upd <= 0 || n_streams <= 0) {
        if (taps_in != taps_out)
            return cudaMemcpyAsync(taps_out, taps_in, sizeof(float2) * 4 * T * (size_t)n_streams,
                                   cudaMemcpyDeviceToDevice, st);
        return cudaSuccess;
    }
    switch (T) {
        case 7: return lms_dispatch_dims<7>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st);
        case 15: return lms_dispatch_dims<15>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st);
        case 31: return lms_dispatch_dims<31>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_align(const float2 *x, long ns, float2 *taps, const uint8_t *ref_lab,
                         long ref_stride, int n_train, int n_streams, int T, const FmtDev &f,
                         cudaStream_t st) {
    if (n_train <= 0 || n_streams <= 0) return cudaSuccess;
    switch (T) {
        case 7: return align_dispatch<7>(x, ns, taps, ref_lab, ref_stride, n_train, n_streams, f, st);
        case 15: return align_dispatch<15>(x, ns, taps, ref_lab, ref_stride, n_train, n_streams, f, st);
        case 31: return align_dispatch<31>(x, ns, taps, ref_lab, ref_stride, n_train, n_streams, f, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_train_phase(const float2 *x, long ns, const float2 *taps, const uint8_t *ref_lab,
                               long ref_stride, int n, int W, uint16_t *pcode, long pcode_stride,
                               int32_t *carry, int carry_stride, int n_streams, int T,
                               const FmtDev &f, cudaStream_t st) {
    if (n <= 0 || n_streams <= 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)n;
    if (smem > 160 * 1024) return cudaErrorInvalidValue;
#define RX_TP(TT, DD)                                                                          \
    do {                                                                                       \
        auto k_ = train_phase_kernel<TT, DD>;                                                  \
        cudaError_t e_ = cudaFuncSetAttribute(k_, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              (int)smem);                                     \
        if (e_ != cudaSuccess) return e_;                                                      \
        k_<<<n_streams, 256, smem, st>>>(x, ns, taps, ref_lab, ref_stride, n, W, pcode,        \
                                         pcode_stride, carry, carry_stride, f);                \
    } while (0)
    const bool d4 = f.dims == 4;
    switch (T) {
        case 7: if (d4) RX_TP(7, 4); else RX_TP(7, 2); break;
        case 15: if (d4) RX_TP(15, 4); else RX_TP(15, 2); break;
        case 31: if (d4) RX_TP(31, 4); else RX_TP(31, 2); break;
        default: return cudaErrorInvalidValue;
    }
#undef RX_TP
    return cudaGetLastError();
}

cudaError_t launch_ref_labels(const uint8_t *bits, uint8_t *lab, long n_sym, int n_streams, int m,
                              int dims, int m_pol, cudaStream_t st) {
    (void)dims;
    (void)m_pol;
    if (n_sym <= 0 || n_streams <= 0) return cudaSuccess;
    dim3 grid((unsigned)((n_sym + 255) / 256), (unsigned)n_streams);
    ref_labels_kernel<<<grid, 256, 0, st>>>(bits, lab, n_sym, m);
    return cudaGetLastError();
}
