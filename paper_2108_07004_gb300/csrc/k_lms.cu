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
#include <algorithm>

#include "rx_internal.h"

namespace {

constexpr int kCH = 1024;
// dynamic shared memory: rotations, two target rows, e_k and base_k rows
constexpr int kDynBytes = 3 * kCH * sizeof(float2) + 2 * kCH * sizeof(float4);
// named barriers between the decision warp (0) and the tap warp (1), one
// pair each way; consecutive updates alternate, so a barrier never receives
// a second arrival before its waiter has passed (barrier 0 is __syncthreads)
constexpr int kBarErr0 = 1, kBarBase0 = 3;

__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

struct Tables {
    float4 orb[RX_MAXM];
    float orbe[RX_MAXM];
    int orblab[RX_MAXM][4];
    float4 pts[RX_MAXM];
    float2 cs[RX_MAXB];
};

__device__ __forceinline__ void load_tables(Tables &tb, const FmtDev &f) {
    for (int i = threadIdx.x; i < f.n_orb; i += blockDim.x) {
        tb.orb[i] = make_float4(f.orb[i][0], f.orb[i][1], f.orb[i][2], f.orb[i][3]);
        tb.orbe[i] = f.orbe[i];
        for (int k = 0; k < 4; ++k) tb.orblab[i][k] = f.orb_lab[i][k];
    }
    for (int i = threadIdx.x; i < f.M; i += blockDim.x)
        tb.pts[i] = make_float4(f.pts[i][0], f.pts[i][1], f.pts[i][2], f.pts[i][3]);
    for (int i = threadIdx.x; i < f.B; i += blockDim.x) tb.cs[i] = make_float2(f.cs[i][0], f.cs[i][1]);
}

// best rotation of an orbit given P + jQ = sum_p z_p conj(rep_p):
// Re of the correlation with rep * j^k is P, Q, -P, -Q for k = 0..3.
__device__ __forceinline__ void best_rot(float P, float Q, int S, float &v, int &k) {
    if (S == 4) {
        const float aP = fabsf(P), aQ = fabsf(Q);
        const bool pw = aP >= aQ;
        v = pw ? aP : aQ;
        k = pw ? (P >= 0.f ? 0 : 2) : (Q >= 0.f ? 1 : 3);
    } else if (S == 2) {
        v = fabsf(P); k = P >= 0.f ? 0 : 1;
    } else {
        v = P; k = 0;
    }
}

// Nearest table point of the candidates held by the lanes: lane o (o < 16)
// holds orbit o's best rotation, its squared distance and its label; the
// minimum distance over the lanes wins and exact ties go to the lowest label.
// Two warp reductions return the winning label itself.
__device__ __forceinline__ int argmin_label(float dist, bool valid, int label) {
    const unsigned bits = valid ? __float_as_uint(fmaxf(dist, 0.f)) : 0xffffffffu;
    const unsigned mn = __reduce_min_sync(0xffffffffu, bits);
    const unsigned key = (bits == mn) ? (unsigned)label : 0xffffffffu;
    return (int)__reduce_min_sync(0xffffffffu, key);
}

// (y0, y1) from per-lane partials of both outputs: xor-16 halving step, four
// xor steps within the half warp, then exchange of the halves.
__device__ __forceinline__ void reduce_pair(float2 a, float2 b, int p, float2 &y0, float2 &y1) {
    float2 send = p ? a : b, keep = p ? b : a;
    keep.x += __shfl_xor_sync(0xffffffffu, send.x, 16);
    keep.y += __shfl_xor_sync(0xffffffffu, send.y, 16);
#pragma unroll
    for (int m = 8; m > 0; m >>= 1) {
        keep.x += __shfl_xor_sync(0xffffffffu, keep.x, m);
        keep.y += __shfl_xor_sync(0xffffffffu, keep.y, m);
    }
    float2 other;
    other.x = __shfl_xor_sync(0xffffffffu, keep.x, 16);
    other.y = __shfl_xor_sync(0xffffffffu, keep.y, 16);
    y0 = p ? other : keep;
    y1 = p ? keep : other;
}

// Sequential CMA (MODE 0), DD-LMS (MODE 1) or data-aided LMS (MODE 3).
//
// Lane (p, j) = (lane >> 4, lane & 15) holds h_qp[j + 16 i] of both outputs
// q.  The recursion is written in look-ahead form: with X_k the stacked
// input window of symbol k and h_k the taps after update k,
//   y_k = h_{k-1}^H X_k = h_{k-2}^H X_k + mu e_{k-1} X_{k-1}^H X_k,
// so the 32-lane reduction of base_k = h_{k-2}^H X_k is issued two updates
// ahead and overlaps with the decision of the update in between; only the
// scalar correction with r1_k = X_{k-1}^H X_k (precomputed by the whole block
// for the staged span) is on the sequential path.
template <int T, int DIMS, int MODE>
__global__ void __launch_bounds__(256, 1)
lms_kernel(const void *__restrict__ x, long ns, const float2 *__restrict__ taps_in,
           float2 *__restrict__ taps_out, long k0, int n_upd, const uint16_t *__restrict__ pcode,
           long pcode_stride, int passes, float mu, const uint8_t *__restrict__ ref_lab,
           long ref_stride, int sk, const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    constexpr int NSX = 2 * kCH + 2 * D + 8;   // + slack read by the look-ahead past the span
    constexpr int NT = (T + 15) / 16;
    __shared__ float2 xs[2][NSX];
    __shared__ float2 r1s[kCH];
    __shared__ uint16_t pc[kCH];
    __shared__ uint8_t rl[kCH];
    __shared__ Tables tb;
    // dynamic: exp(j phi_k) of the span (MODE 1, 3) and the data-aided
    // targets d_q exp(j phi_k) (MODE 3), prepared by the whole block
    // and the exchange between the decision and tap warps: e_k and base_k
    // of both outputs as (re0, im0, re1, im1)
    extern __shared__ float2 dyn_sm[];
    float2 *rots = dyn_sm;
    float2 *tg0 = dyn_sm + kCH, *tg1 = dyn_sm + 2 * kCH;
    float4 *es = reinterpret_cast<float4 *>(dyn_sm + 3 * kCH);
    float4 *bs = es + kCH;
    const int s = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int p = lane >> 4, j = lane & 15;
    load_tables(tb, f);

    float2 h[2][NT];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int i = 0; i < NT; ++i) {
            const int t = j + 16 * i;
            h[q][i] = (t < T) ? taps_in[(((long)s * 2 + q) * 2 + p) * T + t] : make_float2(0.f, 0.f);
        }
    const long xoff = (long)s * 2 * ns;
    const int qt_step = 4 / f.S;
    for (int pass = 0; pass < passes; ++pass) {
        for (int c0 = 0; c0 < n_upd; c0 += kCH) {
            const int n = min(kCH, n_upd - c0);
            const long kb = k0 + c0;
            const int nsx = 2 * n + 2 * D + 8;
            __syncthreads();
            // local sample index of symbol kb + kk, tap t: 2 kk + 2 + 2D - t
            for (int i = threadIdx.x; i < 2 * nsx; i += blockDim.x) {
                const int pp = i / nsx, jj = i - pp * nsx;
                const long g = 2 * (kb - 1) - D + jj;
                xs[pp][jj] = (g >= 0 && g < ns) ? ld_sample(x, xoff + (long)pp * ns + g, sk) : make_float2(0.f, 0.f);
            }
            if (MODE != 0)
                for (int i = threadIdx.x; i < n; i += blockDim.x) pc[i] = pcode[(long)s * pcode_stride + kb + i];
            if (MODE == 3)
                for (int i = threadIdx.x; i < n; i += blockDim.x) rl[i] = ref_lab[(long)s * ref_stride + kb + i];
            __syncthreads();
            for (int kk = threadIdx.x; kk < n; kk += blockDim.x) {   // r1_k = X_{k-1}^H X_k
                float2 acc = make_float2(0.f, 0.f);
                for (int pp = 0; pp < 2; ++pp)
#pragma unroll 8
                    for (int t = 0; t < T; ++t)
                        acc = cadd(acc, cmulc(xs[pp][2 * kk + 2 * D - t], xs[pp][2 * kk + 2 + 2 * D - t]));
                r1s[kk] = acc;
                if (MODE != 0) {
                    // exp(j phi_k) = cs_b j^qt
                    const unsigned code = pc[kk];
                    const int b = min((int)(code & 255), f.B - 1);
                    const int qt = ((int)((code >> 8) & 3) * qt_step) & 3;
                    float2 rot = tb.cs[b];
                    if (qt & 2) rot = make_float2(-rot.x, -rot.y);
                    if (qt & 1) rot = make_float2(-rot.y, rot.x);
                    rots[kk] = rot;
                    if (MODE == 3) {
                        const int lab = rl[kk];
                        float2 d0, d1;
                        if (DIMS == 4) {
                            const float4 pt = tb.pts[lab];
                            d0 = make_float2(pt.x, pt.y);
                            d1 = make_float2(pt.z, pt.w);
                        } else {
                            const float4 px = tb.pts[lab >> f.m_pol];
                            const float4 py = tb.pts[lab & ((1 << f.m_pol) - 1)];
                            d0 = make_float2(px.x, px.y);
                            d1 = make_float2(py.x, py.y);
                        }
                        tg0[kk] = cmul(d0, rot);
                        tg1[kk] = cmul(d1, rot);
                    }
                }
            }
            __syncthreads();
            auto xval = [&](int kk, int i) -> float2 {
                const int t = j + 16 * i;
                return (t < T) ? xs[p][2 * kk + 2 + 2 * D - t] : make_float2(0.f, 0.f);
            };
            auto base = [&](int kk, float2 &b0, float2 &b1) {
                float2 a = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
#pragma unroll
                for (int i = 0; i < NT; ++i) {
                    const float2 xv = xval(kk, i);
                    a = cadd(a, cmulc(h[0][i], xv));
                    c = cadd(c, cmulc(h[1][i], xv));
                }
                reduce_pair(a, c, p, b0, b1);
            };
            if (warp == 1) {
                // tap warp: h_k = h_{k-1} + mu conj(e_k) X_k, then publishes
                // base_{k+2} = h_k^H X_{k+2} (base_0, base_1 from the
                // chunk's initial taps); only bases inside the span are
                // published, so every barrier phase is matched
                float2 b0, b1;
                base(0, b0, b1);
                bs[0] = make_float4(b0.x, b0.y, b1.x, b1.y);
                bar_arrive(kBarBase0, 64);
                if (n > 1) {
                    base(1, b0, b1);
                    bs[1] = make_float4(b0.x, b0.y, b1.x, b1.y);
                    bar_arrive(kBarBase0 + 1, 64);
                }
#pragma unroll 2
                for (int kk = 0; kk < n; ++kk) {
                    bar_sync(kBarErr0 + (kk & 1), 64);
                    const float4 e = es[kk];
                    const float2 c0v = make_float2(mu * e.x, -mu * e.y), c1v = make_float2(mu * e.z, -mu * e.w);
#pragma unroll
                    for (int i = 0; i < NT; ++i) {
                        const float2 xv = xval(kk, i);
                        h[0][i] = cadd(h[0][i], cmul(c0v, xv));
                        h[1][i] = cadd(h[1][i], cmul(c1v, xv));
                    }
                    if (kk + 2 < n) {
                        base(kk + 2, b0, b1);
                        bs[kk + 2] = make_float4(b0.x, b0.y, b1.x, b1.y);
                        bar_arrive(kBarBase0 + (kk & 1), 64);
                    }
                }
                continue;
            }
            if (warp != 0) continue;
            // decision warp: y_k = base_k + mu e_{k-1} r1_k, e_k, published
            // for the tap warp
            // this lane's orbit (DD decisions): representative, energy, and
            // the labels of its S rotations packed one per byte
            const int o = lane & 15;
            const bool valid = o < f.n_orb;
            const float4 r = tb.orb[valid ? o : 0];
            const float eo = tb.orbe[valid ? o : 0];
            unsigned lab4 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) lab4 |= (unsigned)(tb.orblab[valid ? o : 0][k] & 255) << (8 * k);
            auto label_of = [&](int k) { return (int)((lab4 >> (8 * k)) & 255u); };
            float2 ep0 = make_float2(0.f, 0.f), ep1 = make_float2(0.f, 0.f);
#pragma unroll 2
            for (int kk = 0; kk < n; ++kk) {
                const float2 r1 = r1s[kk];
                bar_sync(kBarBase0 + (kk & 1), 64);
                const float4 bb = bs[kk];
                const float2 y0 = cadd(make_float2(bb.x, bb.y), cmul(make_float2(mu * ep0.x, mu * ep0.y), r1));
                const float2 y1 = cadd(make_float2(bb.z, bb.w), cmul(make_float2(mu * ep1.x, mu * ep1.y), r1));
                float2 e0, e1;
                if (MODE == 0) {
                    const float g0 = f.R2 - cnorm(y0), g1 = f.R2 - cnorm(y1);
                    e0 = make_float2(g0 * y0.x, g0 * y0.y);
                    e1 = make_float2(g1 * y1.x, g1 * y1.y);
                } else if (MODE == 3) {
                    e0 = csub(tg0[kk], y0);
                    e1 = csub(tg1[kk], y1);
                } else {
                    const float2 rot = rots[kk];                               // exp(j phi)
                    float2 d0, d1;
                    const float2 z0 = cmulc(rot, y0), z1 = cmulc(rot, y1);   // y exp(-j phi)
                    if (DIMS == 4) {
                        const float P = (z0.x * r.x + z0.y * r.y) + (z1.x * r.z + z1.y * r.w);
                        const float Q = (z0.y * r.x - z0.x * r.y) + (z1.y * r.z - z1.x * r.w);
                        float v;
                        int k;
                        best_rot(P, Q, f.S, v, k);
                        const float dist = (cnorm(z0) + cnorm(z1)) + (eo - 2.f * v);
                        const float4 pt = tb.pts[argmin_label(dist, valid, label_of(k))];
                        d0 = make_float2(pt.x, pt.y);
                        d1 = make_float2(pt.z, pt.w);
                    } else {
                        float v0, v1;
                        int k0r, k1r;
                        best_rot(z0.x * r.x + z0.y * r.y, z0.y * r.x - z0.x * r.y, f.S, v0, k0r);
                        best_rot(z1.x * r.x + z1.y * r.y, z1.y * r.x - z1.x * r.y, f.S, v1, k1r);
                        const float4 p0 = tb.pts[argmin_label(cnorm(z0) + eo - 2.f * v0, valid, label_of(k0r))];
                        const float4 p1 = tb.pts[argmin_label(cnorm(z1) + eo - 2.f * v1, valid, label_of(k1r))];
                        d0 = make_float2(p0.x, p0.y);
                        d1 = make_float2(p1.x, p1.y);
                    }
                    e0 = csub(cmul(d0, rot), y0);
                    e1 = csub(cmul(d1, rot), y1);
                }
                es[kk] = make_float4(e0.x, e0.y, e1.x, e1.y);   // every lane: the same value
                bar_arrive(kBarErr0 + (kk & 1), 64);
                ep0 = e0; ep1 = e1;
            }
        }
    }
    if (warp == 1) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int i = 0; i < NT; ++i) {
                const int t = j + 16 * i;
                if (t < T) taps_out[(((long)s * 2 + q) * 2 + p) * T + t] = h[q][i];
            }
    }
}

// ---------------------------------------------------------------------------
// training alignment
// ---------------------------------------------------------------------------
template <int T, int DIMS>
__global__ void __launch_bounds__(256)
align_kernel(const void *__restrict__ x, long ns, float2 *__restrict__ taps,
             const uint8_t *__restrict__ ref_lab, long ref_stride, int n_train, int sk,
             const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    __shared__ float2 hs[4 * T];
    __shared__ double red[8][256];
    __shared__ float2 rot[2];
    __shared__ int src[2];
    const int s = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < 4 * T; i += 256) hs[i] = taps[(long)s * 4 * T + i];
    __syncthreads();
    const long xoff = (long)s * 2 * ns;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // C[q][p] re, im
    for (int k = tid; k < n_train; k += 256) {
        float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp)
                for (int t = 0; t < T; ++t) {
                    const long g = 2L * k + D - t;
                    if (g < 0 || g >= ns) continue;
                    const float2 hv = hs[(qq * 2 + pp) * T + t];
                    const float2 xv = ld_sample(x, xoff + (long)pp * ns + g, sk);
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
train_phase_kernel(const void *__restrict__ x, long ns, const float2 *__restrict__ taps,
                   const uint8_t *__restrict__ ref_lab, long ref_stride, int n, int W,
                   uint16_t *__restrict__ pcode, long pcode_stride, int32_t *__restrict__ carry,
                   int carry_stride, int sk, const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    extern __shared__ float2 rs[];      // [n] per-symbol correlations
    __shared__ float2 hs[4 * T];
    const int s = blockIdx.x, tid = threadIdx.x;
    for (int i = tid; i < 4 * T; i += 256) hs[i] = taps[(long)s * 4 * T + i];
    __syncthreads();
    const long xoff = (long)s * 2 * ns;
    for (int k = tid; k < n; k += 256) {
        float2 y[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp)
                for (int t = 0; t < T; ++t) {
                    const long g = 2L * k + D - t;
                    if (g < 0 || g >= ns) continue;
                    y[qq] = cadd(y[qq], cmulc(hs[(qq * 2 + pp) * T + t], ld_sample(x, xoff + (long)pp * ns + g, sk)));
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

// The recursion is latency-bound: a block asks for (nearly) all of an SM's
// shared memory so that no other kernel's blocks share its SM and its warp
// issues whenever it is ready.
template <int T, int DIMS, int MODE>
cudaError_t lms_launch_one(const void *x, long ns, const float2 *ti, float2 *to, long k0, int n_upd,
                           const uint16_t *pcode, long pstride, int passes, float mu,
                           const uint8_t *ref, long rstride, int S, const FmtDev &f, cudaStream_t st, int sk) {
    auto kern = lms_kernel<T, DIMS, MODE>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int dyn = optin - (int)fa.sharedSizeBytes;
    if (dyn < (int)(kDynBytes)) return cudaErrorInvalidValue;   // rotations, targets, exchange
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    if (e != cudaSuccess) return e;
    kern<<<S, 256, dyn, st>>>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, sk, f);
    return cudaGetLastError();
}

template <int T, int MODE>
cudaError_t lms_launch_mode(const void *x, long ns, const float2 *ti, float2 *to, long k0,
                            int n_upd, const uint16_t *pcode, long pstride, int passes, float mu,
                            const uint8_t *ref, long rstride, int S, const FmtDev &f,
                            cudaStream_t st, int sk) {
    if (f.dims == 4)
        return lms_launch_one<T, 4, MODE>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref,
                                          rstride, S, f, st, sk);
    return lms_launch_one<T, 2, MODE>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref,
                                      rstride, S, f, st, sk);
}

template <int T>
cudaError_t lms_dispatch_dims(const void *x, long ns, const float2 *ti, float2 *to, long k0,
                              int n_upd, const uint16_t *pcode, long pstride, int mode,
                              int passes, unsigned long long u0, int n_cma, float mu,
                              const uint8_t *ref, long rstride, int S, const FmtDev &f,
                              cudaStream_t st, int sk) {
    switch (mode) {
        case 0: return lms_launch_mode<T, 0>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, S, f, st, sk);
        case 1: return lms_launch_mode<T, 1>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, S, f, st, sk);
        case 3: return lms_launch_mode<T, 3>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, S, f, st, sk);
        case 2: {
            // CMA while the update count is below n_cma, DD after (one pass)
            const long ncma = (u0 >= (unsigned long long)n_cma) ? 0 : std::min<long>(n_upd, (long)(n_cma - u0));
            cudaError_t e = cudaSuccess;
            const float2 *src = ti;
            if (ncma > 0) {
                e = lms_launch_mode<T, 0>(x, ns, src, to, k0, (int)ncma, pcode, pstride, 1, mu, ref, rstride, S, f, st, sk);
                if (e != cudaSuccess) return e;
                src = to;
            }
            if (n_upd - ncma > 0)
                e = lms_launch_mode<T, 1>(x, ns, src, to, k0 + ncma, (int)(n_upd - ncma), pcode, pstride, 1, mu,
                                          ref, rstride, S, f, st, sk);
            return e;
        }
        default: return cudaErrorInvalidValue;
    }
}

template <int T>
cudaError_t align_dispatch(const void *x, long ns, float2 *taps, const uint8_t *ref,
                           long rstride, int n_train, int S, const FmtDev &f, cudaStream_t st, int sk) {
    if (f.dims == 4)
        align_kernel<T, 4><<<S, 256, 0, st>>>(x, ns, taps, ref, rstride, n_train, sk, f);
    else
        align_kernel<T, 2><<<S, 256, 0, st>>>(x, ns, taps, ref, rstride, n_train, sk, f);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lms(const void *x, long ns, const float2 *taps_in, float2 *taps_out, long k0,
                       int n_upd, const uint16_t *pcode, long pcode_stride, int mode, int passes,
                       unsigned long long u0, int n_cma, float mu, const uint8_t *ref_lab,
                       long ref_stride, int n_streams, int T, const FmtDev &f, cudaStream_t st, int sk) {
    if (n_upd <= 0 || n_streams <= 0) {
        if (taps_in != taps_out)
            return cudaMemcpyAsync(taps_out, taps_in, sizeof(float2) * 4 * T * (size_t)n_streams,
                                   cudaMemcpyDeviceToDevice, st);
        return cudaSuccess;
    }
    switch (T) {
        case 7: return lms_dispatch_dims<7>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st, sk);
        case 15: return lms_dispatch_dims<15>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st, sk);
        case 31: return lms_dispatch_dims<31>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st, sk);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_align(const void *x, long ns, float2 *taps, const uint8_t *ref_lab,
                         long ref_stride, int n_train, int n_streams, int T, const FmtDev &f,
                         cudaStream_t st, int sk) {
    if (n_train <= 0 || n_streams <= 0) return cudaSuccess;
    switch (T) {
        case 7: return align_dispatch<7>(x, ns, taps, ref_lab, ref_stride, n_train, n_streams, f, st, sk);
        case 15: return align_dispatch<15>(x, ns, taps, ref_lab, ref_stride, n_train, n_streams, f, st, sk);
        case 31: return align_dispatch<31>(x, ns, taps, ref_lab, ref_stride, n_train, n_streams, f, st, sk);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_train_phase(const void *x, long ns, const float2 *taps, const uint8_t *ref_lab,
                               long ref_stride, int n, int W, uint16_t *pcode, long pcode_stride,
                               int32_t *carry, int carry_stride, int n_streams, int T,
                               const FmtDev &f, cudaStream_t st, int sk) {
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
                                         pcode_stride, carry, carry_stride, sk, f);            \
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
