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

__device__ __forceinline__ float ex2_ftz(float x) {        // 2^x, subnormal results flushed to 0
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float softplus_bits(float x) {   // log2(1 + exp(x))
    const float t = x * kLog2e;
    return fmaxf(t, 0.f) + __log2f(1.f + ex2_ftz(-fabsf(t)));
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

// Rare path, for lookups where some bit's subset sum fell below 2^-100 of
// the common shift (|LLR| beyond ~150): every subset gets its own minimum
// as shift.  The whole warp serves the flagged lanes one after another:
// the lanes split the table (points lane, lane + 32), and the subset minima
// and sums are warp reductions in a fixed order.  Rewrites the flagged
// lanes' LLRs L[0..MB-1] and their counting terms (ne, g2) of this lookup.
template <int DIMS, int MT, int MB>
__device__ __forceinline__ void llr_fixup_warp(unsigned need, float2 z0, float2 z1, const FmtDev &f, float c2,
                                            float *L, int ref, int &ne, float &g2) {
    const int lane = threadIdx.x & 31;
    constexpr int NPL = (MT + 31) / 32;   // points per lane
    while (need) {
        const int src = __ffs(need) - 1;
        need &= need - 1;
        const float2 a0 = make_float2(__shfl_sync(0xffffffffu, z0.x, src), __shfl_sync(0xffffffffu, z0.y, src));
        const float2 a1 = make_float2(__shfl_sync(0xffffffffu, z1.x, src), __shfl_sync(0xffffffffu, z1.y, src));
        const float cc = __shfl_sync(0xffffffffu, c2, src);
        float d[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int j = lane + 32 * i;
            d[i] = j < MT ? dist_to<DIMS>(a0, a1, f, j) : 3.0e38f;
        }
        int ne_s = 0;
        float g2_s = 0.f;
        const int rs = __shfl_sync(0xffffffffu, ref, src);
#pragma unroll
        for (int bp = 0; bp < MB; ++bp) {
            float lg[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                float dm = 3.0e38f;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int j = lane + 32 * i;
                    if (j < MT && ((j >> bp) & 1) == v) dm = fminf(dm, d[i]);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) dm = fminf(dm, __shfl_xor_sync(0xffffffffu, dm, off));
                float acc = 0.f;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int j = lane + 32 * i;
                    if (j < MT && ((j >> bp) & 1) == v) acc += exp2f((dm - d[i]) * cc);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                lg[v] = -dm * cc + log2f(acc);
            }
            const float Lb = (lg[0] - lg[1]) * kLn2;
            if (lane == src) L[MB - 1 - bp] = Lb;
            if (rs >= 0) {
                const int bit = (rs >> bp) & 1;
                ne_s += (int)((Lb < 0.f) != (bit != 0));
                g2_s += softplus_bits(bit ? Lb : -Lb);
            }
        }
        if (lane == src) { ne = ne_s; g2 = g2_s; }
    }
}

// LLRs of one table lookup of z (DIMS 4: joint; DIMS 2: z0 alone), MB bits,
// written to out[0..MB-1] (MSB first).  When ref >= 0 (the reference label of
// this lookup) the hard-decision errors and the GMI terms are accumulated.
template <int DIMS, int MT, int MB>
__device__ __forceinline__ bool llr_table(float2 z0, float2 z1, const FmtDev &f, float c2,
                                          float *out, float &g, int &jmin, int ref, int &ne,
                                          float &g2) {
    float cur[MT];
#pragma unroll
    for (int j = 0; j < MT; ++j) cur[j] = dist_to<DIMS>(z0, z1, f, j);
    g = cur[0];
    jmin = 0;
#pragma unroll
    for (int j = 1; j < MT; ++j)
        if (cur[j] < g) { g = cur[j]; jmin = j; }
#pragma unroll
    for (int j = 0; j < MT; ++j) cur[j] = ex2_ftz(fmaf(g - cur[j], c2, kOff));
    bool low = false;
    ne = 0;
    g2 = 0.f;
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
    return low;
}

// Eight consecutive labels g8 .. g8+7 as packed pairs E[v] = (e_{2v}, e_{2v+1})
// (the low three label bits vary, the high ones are those of g8): packed
// running sums for the low three bits (bit 0: evens / odds of every group;
// bit 1: F = (e0+e4, e1+e5) / G = (e2+e6, e3+e7) per group, i.e. labels
// with bit 1 clear / set; bit 2: H = (e0+e2, e1+e3) / I = (e4+e6, e5+e7)),
// and the group total for the high bits, added once per group.
struct GroupSums {
    f32x2 b0 = 0ull, f = 0ull, g = 0ull, h = 0ull, i = 0ull;
};
template <int MB>
__device__ __forceinline__ void add_group8(const f32x2 (&E)[4], int g8, GroupSums &gs, float (&s0)[MB],
                                           float (&s1)[MB]) {
    const f32x2 H = add2(E[0], E[1]), I = add2(E[2], E[3]);   // (e0+e2, e1+e3), (e4+e6, e5+e7)
    const f32x2 F = add2(E[0], E[2]), G = add2(E[1], E[3]);   // (e0+e4, e1+e5), (e2+e6, e3+e7)
    const f32x2 HI = add2(H, I);                              // (evens, odds) of the group
    gs.b0 = add2(gs.b0, HI);
    gs.f = add2(gs.f, F);
    gs.g = add2(gs.g, G);
    gs.h = add2(gs.h, H);
    gs.i = add2(gs.i, I);
    if (MB > 3) {
        float hx, hy;
        upk2(HI, hx, hy);
        const float tot = hx + hy;
#pragma unroll
        for (int b = 3; b < MB; ++b) {
            if ((g8 >> b) & 1) s1[b] += tot;
            else s0[b] += tot;
        }
    }
}

// 4D table of MT points with MB label bits, streaming form: the shift is the
// minimum distance from the orbit form (|z|^2 + |rep|^2 - 2 max(|P|,|Q|)),
// two orbits at a time as packed pairs; its orbit comes with it as the low
// four bits of a signed-integer key (distance bits with the low four
// cleared, so ties and 2^-19 differences go to the lower orbit; the shift
// and the nearest point's energy need no more), and gives the nearest
// point's energy.  Then every point's exact distance |z - s_j|^2
// (differences, no cancellation) and exponential is added to the subset
// sums of its label bits, eight labels at a time.  The loop is fully
// unrolled, so every table entry is a constant-bank operand and every label
// bit is known at compile time; a few packed accumulators instead of 64
// stored terms keep the registers low.
template <int MT, int MB>
__device__ __forceinline__ bool llr_4d_stream(float2 z0, float2 z1, const FmtDev &f, const float *en, float c2,
                                              float *out, float &gmin, float &emin, int ref,
                                              int &ne, float &g2) {
    const float zn = cnorm(z0) + cnorm(z1);
    const f32x2 Z0 = pk2(z0.x, z0.x), Z1 = pk2(z0.y, z0.y), Z2 = pk2(z1.x, z1.x), Z3 = pk2(z1.y, z1.y);
    {
        // Re c and Im c of c = sum_p z_p conj(rep_p), two orbits per packed pair
        const f32x2 N0 = pk2(-z0.x, -z0.x), N2 = pk2(-z1.x, -z1.x), ZN = pk2(zn, zn), M2 = pk2(-2.f, -2.f);
        const f32x2 *R0 = reinterpret_cast<const f32x2 *>(f.orbT[0]);
        const f32x2 *R1 = reinterpret_cast<const f32x2 *>(f.orbT[1]);
        const f32x2 *R2 = reinterpret_cast<const f32x2 *>(f.orbT[2]);
        const f32x2 *R3 = reinterpret_cast<const f32x2 *>(f.orbT[3]);
        const f32x2 *EO = reinterpret_cast<const f32x2 *>(f.orbeP);
        int key = 0x7fffffff;
#pragma unroll
        for (int op = 0; op < 8; ++op) {
            if (2 * op < f.n_orb) {
                const f32x2 P = fma2(Z3, R3[op], fma2(Z2, R2[op], fma2(Z1, R1[op], mul2(Z0, R0[op]))));
                const f32x2 Q = fma2(N2, R3[op], fma2(Z3, R2[op], fma2(N0, R1[op], mul2(Z1, R0[op]))));
                float p0, p1, q0, q1, v0, v1, d0, d1;
                upk2(P, p0, p1);
                upk2(Q, q0, q1);
                v0 = (f.S == 4) ? fmaxf(fabsf(p0), fabsf(q0)) : (f.S == 2 ? fabsf(p0) : p0);
                v1 = (f.S == 4) ? fmaxf(fabsf(p1), fabsf(q1)) : (f.S == 2 ? fabsf(p1) : p1);
                upk2(fma2(M2, pk2(v0, v1), add2(ZN, EO[op])), d0, d1);   // +inf past n_orb
                key = min(key, (__float_as_int(d0) & ~15) | (2 * op));
                key = min(key, (__float_as_int(d1) & ~15) | (2 * op + 1));
            }
        }
        gmin = __int_as_float(key & ~15);
        emin = en[key & 15];       // the lanes' orbits differ: a shared-memory read
    }
    const float sh = fmaf(gmin, c2, kOff);   // exponent of point j: sh - d_j c2
    float s0[MB], s1[MB];
#pragma unroll
    for (int i = 0; i < MB; ++i) { s0[i] = 0.f; s1[i] = 0.f; }
    GroupSums gs;
    // labels j, j+1 as packed pairs: d = sum_c (z_c - s_c)^2 per lane
    const f32x2 NC = pk2(-c2, -c2), SH = pk2(sh, sh);
    const f32x2 *T0 = reinterpret_cast<const f32x2 *>(f.ptsT[0]);
    const f32x2 *T1 = reinterpret_cast<const f32x2 *>(f.ptsT[1]);
    const f32x2 *T2 = reinterpret_cast<const f32x2 *>(f.ptsT[2]);
    const f32x2 *T3 = reinterpret_cast<const f32x2 *>(f.ptsT[3]);
#pragma unroll
    for (int g8 = 0; g8 < MT; g8 += 8) {
        f32x2 E[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int jp = g8 / 2 + v;
            const f32x2 u0 = sub2(Z0, T0[jp]), u1 = sub2(Z1, T1[jp]);
            const f32x2 u2 = sub2(Z2, T2[jp]), u3 = sub2(Z3, T3[jp]);
            f32x2 d = mul2(u0, u0);
            d = fma2(u1, u1, d);
            d = fma2(u2, u2, d);
            d = fma2(u3, u3, d);
            float a0, a1;
            upk2(fma2(d, NC, SH), a0, a1);
            E[v] = pk2(ex2_ftz(a0), ex2_ftz(a1));
        }
        add_group8<MB>(E, g8, gs, s0, s1);
    }
    {
        float x, y;
        upk2(gs.b0, s0[0], s1[0]);
        upk2(gs.f, x, y);
        s0[1] = x + y;
        upk2(gs.g, x, y);
        s1[1] = x + y;
        upk2(gs.h, x, y);
        s0[2] = x + y;
        upk2(gs.i, x, y);
        s1[2] = x + y;
    }
    gmin = fmaxf(gmin, 0.f);
    bool low = false;
    ne = 0;
    g2 = 0.f;
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
    return low;
}

// 2D table of MT points (128: GS-128) with MB label bits, every bit's two
// subsets with their own shift: a first pass finds the nearest label (lowest
// on ties) and each subset's minimum distance m_{b,v}; the second
// recomputes every distance |z - s_j|^2 (differences, two labels per packed
// pair) and adds 2^{(m_{b,v} - d_j) c2} to the subset sum of each of its
// label bits, so every sum is at least 1 (its nearest point) and at most MT:
//   LLR_b = ln 2 (log2 S_{b,0} - m_{b,0} c2 - log2 S_{b,1} + m_{b,1} c2).
// (With one common shift, at high SNR most symbols of a large table have a
// subset below the float range and would take the warp-wide rare path.)
template <int MT, int MB>
__device__ __forceinline__ bool llr_2d_subsets(float2 z, const FmtDev &f, float c2, float *out, float &g,
                                               int &jmin, int ref, int &ne, float &g2) {
    const f32x2 ZX = pk2(z.x, z.x), ZY = pk2(z.y, z.y);
    const f32x2 *T0 = reinterpret_cast<const f32x2 *>(f.ptsT[0]);
    const f32x2 *T1 = reinterpret_cast<const f32x2 *>(f.ptsT[1]);
    float m0[MB], m1[MB];
#pragma unroll
    for (int b = 0; b < MB; ++b) { m0[b] = 3.0e38f; m1[b] = 3.0e38f; }
    float best = 3.0e38f;
    int bj = 0;
    // groups of eight labels: the low three label bits known at compile time
#pragma unroll 1
    for (int g8 = 0; g8 < MT; g8 += 8) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int jp = g8 / 2 + v;
            const f32x2 u0 = sub2(ZX, T0[jp]), u1 = sub2(ZY, T1[jp]);
            float d[2];
            upk2(fma2(u1, u1, mul2(u0, u0)), d[0], d[1]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jl = 2 * v + h;                 // label g8 + jl
                if (d[h] < best) { best = d[h]; bj = g8 + jl; }
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    if ((jl >> b) & 1) m1[b] = fminf(m1[b], d[h]);
                    else m0[b] = fminf(m0[b], d[h]);
                }
            }
            const float dm = fminf(d[0], d[1]);
#pragma unroll
            for (int b = 3; b < MB; ++b) {
                const bool set = (g8 >> b) & 1;
                m1[b] = set ? fminf(m1[b], dm) : m1[b];
                m0[b] = set ? m0[b] : fminf(m0[b], dm);
            }
        }
    }
    // subset sums as packed pairs: S[0] = (S_{0,0}, S_{0,1}) (bit 0 splits
    // the two labels of a pair); for b >= 1 S[b] and S1[b] the bit-clear and
    // bit-set subsets, each as even / odd label partial sums
    f32x2 S[MB], S1[MB];
#pragma unroll
    for (int b = 0; b < MB; ++b) { S[b] = 0ull; S1[b] = 0ull; }
    const f32x2 NC = pk2(-c2, -c2), O0 = pk2(m0[0] * c2, m1[0] * c2);
    float o0[MB], o1[MB];
#pragma unroll
    for (int b = 0; b < MB; ++b) { o0[b] = m0[b] * c2; o1[b] = m1[b] * c2; }
#pragma unroll 1
    for (int g8 = 0; g8 < MT; g8 += 8) {
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int jp = g8 / 2 + v;
            const f32x2 u0 = sub2(ZX, T0[jp]), u1 = sub2(ZY, T1[jp]);
            const f32x2 d = fma2(u1, u1, mul2(u0, u0));
            float a0, a1;
            // bit 0: label 2 jp in subset (0, 0), label 2 jp + 1 in subset (0, 1)
            upk2(fma2(d, NC, O0), a0, a1);
            S[0] = add2(S[0], pk2(ex2_ftz(a0), ex2_ftz(a1)));
#pragma unroll
            for (int b = 1; b < MB; ++b) {
                // both labels of the pair share bit b
                const bool set = b < 3 ? (((2 * v) >> b) & 1) : ((g8 >> b) & 1);
                const float ob = set ? o1[b] : o0[b];
                upk2(fma2(d, NC, pk2(ob, ob)), a0, a1);
                const f32x2 e2 = pk2(ex2_ftz(a0), ex2_ftz(a1));
                if (set) S1[b] = add2(S1[b], e2);
                else S[b] = add2(S[b], e2);
            }
        }
    }
    g = fmaxf(best, 0.f);
    jmin = bj;
    ne = 0;
    g2 = 0.f;
#pragma unroll
    for (int bp = 0; bp < MB; ++bp) {
        float s0, s1;
        if (bp == 0) {
            upk2(S[0], s0, s1);
        } else {
            float x, y;
            upk2(S[bp], x, y);
            s0 = x + y;
            upk2(S1[bp], x, y);
            s1 = x + y;
        }
        const float L = ((__log2f(s0) - o0[bp]) - (__log2f(s1) - o1[bp])) * kLn2;
        out[MB - 1 - bp] = L;
        if (ref >= 0) {
            const int bit = (ref >> bp) & 1;
            ne += (int)((L < 0.f) != (bit != 0));
            g2 += softplus_bits(bit ? L : -L);
        }
    }
    return false;
}

// Per-thread counting terms of the symbols one thread demapped.
struct CountAcc {
    int nerr = 0, ncnt = 0;
    float gsum = 0.f, en = 0.f, ed = 0.f;
};

// LLRs of one symbol (z0, z1) into L[M_OUT] and its counting terms.  Every
// lane of the warp calls it (inactive lanes on a valid symbol, writing
// nothing), so the warp-wide rare path sees the whole warp.
// en: shared-memory copy of the energies the nearest point is looked up in
// (4D: the orbit energies, 2D: the point energies; see load_energies)
template <int DIMS, int MT, int MB>
__device__ __forceinline__ void demap_symbol(float2 z0, float2 z1, float c2, const FmtDev &f, const float *en,
                                             bool active, int ref, bool counted, float *row, CountAcc &acc) {
    constexpr int M_OUT = (DIMS == 4) ? MB : 2 * MB;
    float L[M_OUT];
    int ne = 0;
    float gs = 0.f, dist_min, dmin_energy;
    if (DIMS == 4) {
        float g2;
        const bool low = llr_4d_stream<MT, MB>(z0, z1, f, en, c2, L, dist_min, dmin_energy, ref, ne, g2);
        const unsigned need = __ballot_sync(0xffffffffu, low && active);
        if (need) llr_fixup_warp<4, MT, MB>(need, z0, z1, f, c2, L, ref, ne, g2);
        gs = g2;
    } else {
        dist_min = 0.f;
        dmin_energy = 0.f;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float2 zp = p ? z1 : z0;
            const int rp = ref < 0 ? -1 : (p ? (ref & ((1 << MB) - 1)) : (ref >> MB));
            float g, g2;
            int jm, nep;
            bool low;
            if constexpr (MT > 64) low = llr_2d_subsets<MT, MB>(zp, f, c2, L + p * MB, g, jm, rp, nep, g2);
            else low = llr_table<2, MT, MB>(zp, zp, f, c2, L + p * MB, g, jm, rp, nep, g2);
            const unsigned need = __ballot_sync(0xffffffffu, low && active);
            if (need) llr_fixup_warp<2, MT, MB>(need, zp, zp, f, c2, L + p * MB, rp, nep, g2);
            ne += nep;
            gs += g2;
            dist_min += g;
            dmin_energy += en[jm];
        }
    }
    if (active) {
#pragma unroll
        for (int i = 0; i < M_OUT; ++i) row[i] = L[i];
    }
    if (counted) {
        acc.nerr += ne;
        acc.ncnt += 1;
        acc.gsum += gs;
        acc.en += dist_min;
        acc.ed += dmin_energy;
    }
}

// The tables a block reads with lane-dependent indices, in shared memory (a
// constant-bank read whose address differs across the warp is serialised):
// the energies of demap_symbol and, for the de-rotation, the test phases'
// (cos, -sin).  Callers synchronise before use.
template <int DIMS>
__device__ __forceinline__ void load_tables(const FmtDev &f, float *en, float2 *rot) {
    for (int i = threadIdx.x; i < RX_MAXM; i += blockDim.x) {
        if (DIMS == 4) { if (i < 16) en[i] = f.orbeP[i]; }
        else en[i] = i < f.M ? f.pe[i] : 0.f;
    }
    if (rot)
        for (int i = threadIdx.x; i < f.B; i += blockDim.x) rot[i] = make_float2(f.cs[i][0], -f.cs[i][1]);
}

// Block sums of the counting terms into this block's partial row, then the
// last block of the stream (ticket) adds the rows in a fixed order (so the
// totals do not depend on block timing) into the stream's accumulators.
__device__ __forceinline__ void count_reduce(CountAcc acc, const DemapCount &cnt, int s, int cta, int n_cta,
                                             double sigma2) {
    __shared__ float red[8][3];
    __shared__ int redn[8][2];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc.nerr += __shfl_xor_sync(0xffffffffu, acc.nerr, off);
        acc.ncnt += __shfl_xor_sync(0xffffffffu, acc.ncnt, off);
        acc.gsum += __shfl_xor_sync(0xffffffffu, acc.gsum, off);
        acc.en += __shfl_xor_sync(0xffffffffu, acc.en, off);
        acc.ed += __shfl_xor_sync(0xffffffffu, acc.ed, off);
    }
    if (lane == 0) {
        red[warp][0] = acc.gsum; red[warp][1] = acc.en; red[warp][2] = acc.ed;
        redn[warp][0] = acc.nerr; redn[warp][1] = acc.ncnt;
    }
    __syncthreads();
    if (tid == 0) {
        double t0 = 0, t1 = 0, t2 = 0;
        unsigned long long n0 = 0, n1 = 0;
        for (int w = 0; w < 8; ++w) {
            t0 += red[w][0]; t1 += red[w][1]; t2 += red[w][2];
            n0 += redn[w][0]; n1 += redn[w][1];
        }
        double *pp = cnt.partial + ((long)s * n_cta + cta) * 5;
        pp[0] = t0; pp[1] = t1; pp[2] = t2;
        pp[3] = (double)n0; pp[4] = (double)n1;
        __threadfence();
        const unsigned prev = atomicAdd(&cnt.sd[s].ticket_demap, 1u);
        last = (prev == (unsigned)n_cta - 1);
    }
    __syncthreads();
    if (!last) return;
    // strided per thread, then a fixed-order tree
    __threadfence();
    const volatile double *pp = cnt.partial + (long)s * n_cta * 5;
    __shared__ double tr[5][256];
    double v[5] = {0, 0, 0, 0, 0};
    for (int c = tid; c < n_cta; c += blockDim.x)
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
        sd.sigma2 = sigma2;
        sd.ticket_demap = 0u;
    }
}

template <int DIMS, int MT, int MB>
__global__ void __launch_bounds__(256, (DIMS == 4 ? 3 : 2))
demap_kernel(const float2 *__restrict__ z, long z_stride, long a, long e,
             const double *__restrict__ sigma2, int s2_stride, float *__restrict__ llr,
             long llr_stride, DemapCount cnt, const __grid_constant__ FmtDev f) {
    constexpr int M_OUT = (DIMS == 4) ? MB : 2 * MB;
    __shared__ float en_sh[RX_MAXM];
    load_tables<DIMS>(f, en_sh, nullptr);
    __syncthreads();
    const int s = blockIdx.y, tid = threadIdx.x;
    const long k = a + (long)blockIdx.x * blockDim.x + tid;
    const float c2 = 1.4426950408889634f / (float)sigma2[s * s2_stride];
    const float2 *zx = z + (long)s * 2 * z_stride;
    const float2 *zy = zx + z_stride;
    const bool active = k < e;
    const long kk = active ? k : e - 1;
    const bool counted = active && cnt.ref_lab && k >= cnt.c0 && k < cnt.c1;
    const int ref = counted ? (int)cnt.ref_lab[(long)s * cnt.ref_stride + k] : -1;
    CountAcc acc;
    demap_symbol<DIMS, MT, MB>(zx[kk - a], zy[kk - a], c2, f, en_sh, active, ref, counted,
                               llr + (long)s * llr_stride + (kk - a) * M_OUT, acc);
    if (!cnt.sd) return;
    count_reduce(acc, cnt, s, blockIdx.x, gridDim.x, sigma2[s * s2_stride]);
}

// ---------------------------------------------------------------------------
// De-rotation fused with demapping (the chain's path).  A block takes a tile
// of TILE consecutive symbols: the unwrap count m before the tile is the
// stream carry plus the increments of the BPS ranges before it (dsum, and
// the boundary increments) plus those of its own range up to the tile;
// inside the tile a block scan gives m per symbol; then each symbol is
// de-rotated by exp(-j (phi_b + m 2 pi / S)) and demapped in place.  Tiles
// are 1024 symbols for the 4D table (64 distances and exponentials a
// symbol) and 4096 for 2D tables, whose per-symbol work is small against
// the tile's prologue and reduction.
// ---------------------------------------------------------------------------
constexpr int kTile = 1024;                 // the 4D table's tile (the smallest)
template <int DIMS> __host__ __device__ constexpr int tile_of() { return DIMS == 4 ? 1024 : 4096; }

template <int DIMS, int MT, int MB>
__global__ void __launch_bounds__(256, (DIMS == 4 ? 4 : 2))
derot_demap_kernel(const void *__restrict__ y, long y_stride, const uint8_t *__restrict__ bsrc,
                   long b_stride, long a, long e, const int *__restrict__ dsum,
                   const double *__restrict__ mdsum, int n_rng, int kR,
                   const int32_t *__restrict__ carry_in, int cin_stride, int32_t *__restrict__ carry_out,
                   int cout_stride, uint16_t *__restrict__ pcode, long pc_stride,
                   const double *__restrict__ sigma2_fixed, double *__restrict__ sigma2_out, int s2_stride,
                   float *__restrict__ llr, long llr_stride, DemapCount cnt, SymOut sym, int sk,
                   const __grid_constant__ FmtDev f) {
    constexpr int M_OUT = (DIMS == 4) ? MB : 2 * MB;
    constexpr int TILE = tile_of<DIMS>();
    constexpr int PT = TILE / 256;
    __shared__ uint8_t bl[TILE];
    __shared__ uint8_t mql[TILE];
    __shared__ float en_sh[RX_MAXM];
    __shared__ float2 rot_sh[RX_MAXB];
    load_tables<DIMS>(f, en_sh, rot_sh);
    __shared__ int wsum[8];
    __shared__ int mstart_sh;
    __shared__ float c2_sh;
    __shared__ double s2_sh;
    const int s = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int B = f.B, S = f.S;
    const uint8_t *bs = bsrc + (long)s * b_stride;   // index k - a
    const long t0 = a + (long)blockIdx.x * TILE;
    const long t1 = min(t0 + TILE, e);
    const int nloc = (int)(t1 - t0);
    const int m_in = carry_in[s * cin_stride + 0], b_in = carry_in[s * cin_stride + 1];
    const int r0 = (int)((t0 - a) / kR);              // BPS range holding the tile start
    const long a_r0 = a + (long)r0 * kR;

    // m before the tile: whole ranges before r0 (warp 0), then the part of
    // range r0 before the tile (all threads)
    int part = 0;
    if (warp == 0) {
        for (int r = lane; r < r0; r += 32) {
            const long st0 = a + (long)r * kR;
            const int bp = (r == 0) ? b_in : bs[st0 - 1 - a];
            part += unwrap_step(bp, bs[st0 - a], B) + dsum[s * n_rng + r];
        }
    }
#pragma unroll 4
    for (long k = a_r0 + tid; k < t0; k += 256)
        part += unwrap_step(k == a ? b_in : bs[k - 1 - a], bs[k - a], B);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
    if (lane == 0) wsum[warp] = part;
    for (int t = tid; t < nloc; t += 256) bl[t] = bs[t0 - a + t];
    if (warp == 1) {
        // the block's sigma^2: warp sum of the ranges' minimum-distance sums
        // (lane-strided, then a butterfly: the same order in every block)
        double tot = 0.0;
        if (!sigma2_fixed)
            for (int r = lane; r < n_rng; r += 32) tot += mdsum[s * n_rng + r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, off);
        if (lane == 0) {
            const double s2 = sigma2_fixed ? sigma2_fixed[s * s2_stride] : tot / (2.0 * (double)(e - a));
            s2_sh = s2;
            c2_sh = 1.4426950408889634f / (float)s2;
            if (blockIdx.x == 0) sigma2_out[s * s2_stride] = s2;
        }
    }
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += wsum[w];
        mstart_sh = m_in + tot;
    }
    const int bprev0 = (t0 == a) ? b_in : (int)bs[t0 - 1 - a];
    // block scan of the tile's increments: thread t owns symbols PT t .. PT t + PT - 1
    int d[PT], run = 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        const int t = PT * tid + u;
        int inc = 0;
        if (t < nloc) inc = unwrap_step(t == 0 ? bprev0 : bl[t - 1], bl[t], B);
        run += inc;
        d[u] = run;
    }
    int incl = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    __syncthreads();
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    const int tpre = mstart_sh + wpre + incl - run;
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        const int t = PT * tid + u;
        if (t >= nloc) continue;
        const int m = tpre + d[u];
        mql[t] = (uint8_t)(((m % S) + S) % S);
        if (t0 + t == e - 1) {
            carry_out[s * cout_stride + 0] = m;
            carry_out[s * cout_stride + 1] = bl[t];
        }
    }
    __syncthreads();
    const float c2 = c2_sh;
    const long yoff = (long)s * 2 * y_stride;      // y of stream s: [2][y_stride], storage kind sk
    uint16_t *pc = pcode + (long)s * pc_stride;
    CountAcc acc;
    // the samples (and reference label) of the next symbol are loaded while
    // this one is demapped
    auto sym_k = [&](int u) { const int t = u * 256 + tid; return t0 + (t < nloc ? t : nloc - 1); };
    auto ref_of = [&](long k) {
        return (llr && cnt.ref_lab && k >= cnt.c0 && k < cnt.c1) ? (int)cnt.ref_lab[(long)s * cnt.ref_stride + k] : -1;
    };
    long k_n = sym_k(0);
    float2 ya_n = ld_sample(y, yoff + k_n, sk), yb_n = ld_sample(y, yoff + y_stride + k_n, sk);
    int ref_n = ref_of(k_n);
    for (int u = 0; u < PT; ++u) {
        const int t = u * 256 + tid;
        const bool active = t < nloc;
        const int tt = active ? t : nloc - 1;
        const long k = t0 + tt;
        const float2 ya = ya_n, yb = yb_n;
        const int ref_k = ref_n;
        if (u + 1 < PT) {
            k_n = sym_k(u + 1);
            ya_n = ld_sample(y, yoff + k_n, sk);
            yb_n = ld_sample(y, yoff + y_stride + k_n, sk);
            ref_n = ref_of(k_n);
        }
        const int b = bl[tt], mq = mql[tt];
        // exp(-j phi) = conj(cs_b) (-j)^mq
        float2 rot = rot_sh[b];
        if (S == 4) {
            if (mq & 2) rot = make_float2(-rot.x, -rot.y);
            if (mq & 1) rot = make_float2(rot.y, -rot.x);
        } else if (S == 2) {
            if (mq) rot = make_float2(-rot.x, -rot.y);
        }
        const float2 z0 = cmul(ya, rot), z1 = cmul(yb, rot);
        if (active) {
            pc[k - a] = (uint16_t)(b | (mq << 8));
            if (sym.x4)
                reinterpret_cast<float4 *>(sym.x4)[(long)s * sym.stride + k] = make_float4(z0.x, z0.y, z1.x, z1.y);
            if (sym.s2) sym.s2[(long)s * sym.stride + k] = (float)s2_sh;
        }
        if (!llr) continue;                   // symbols only (another demapper follows)
        const bool counted = active && cnt.ref_lab && k >= cnt.c0 && k < cnt.c1;
        const int ref = counted ? ref_k : -1;
        demap_symbol<DIMS, MT, MB>(z0, z1, c2, f, en_sh, active, ref, counted,
                                   llr + (long)s * llr_stride + (k - a) * M_OUT, acc);
    }
    if (!cnt.sd || !llr) return;
    count_reduce(acc, cnt, s, blockIdx.x, gridDim.x, s2_sh);
}

// Counting for LLRs made by another demapper (the learned one): hard-decision
// errors and GMI terms against the reference labels, EVM from the symbols
// x4 (nearest point by the orbit form), over symbols a .. e-1 of each
// stream; the same fixed-order reductions as the exact path.
template <int DIMS, int MB>
__global__ void __launch_bounds__(256)
count_llr_kernel(const float *__restrict__ llr, long llr_stride, const float4 *__restrict__ x4, long x_stride,
                 long a, long e, const double *__restrict__ sigma2, int s2_stride, DemapCount cnt,
                 const __grid_constant__ FmtDev f) {
    constexpr int M_OUT = (DIMS == 4) ? MB : 2 * MB;
    const int s = blockIdx.y;
    const long k = a + (long)blockIdx.x * blockDim.x + threadIdx.x;
    CountAcc acc;
    if (k < e && cnt.ref_lab && k >= cnt.c0 && k < cnt.c1) {
        const int ref = cnt.ref_lab[(long)s * cnt.ref_stride + k];
        const float *row = llr + (long)s * llr_stride + (k - a) * M_OUT;
        int ne = 0;
        float g2 = 0.f;
#pragma unroll
        for (int i = 0; i < M_OUT; ++i) {
            const int bit = (ref >> (M_OUT - 1 - i)) & 1;
            const float L = row[i];
            ne += (int)((L < 0.f) != (bit != 0));
            g2 += softplus_bits(bit ? L : -L);
        }
        const float4 v = x4[(long)s * x_stride + k];
        float dist = 0.f, en = 0.f;
        const int npol = DIMS == 4 ? 1 : 2;
        for (int pp = 0; pp < npol; ++pp) {
            const float2 z0 = DIMS == 4 ? make_float2(v.x, v.y) : (pp ? make_float2(v.z, v.w) : make_float2(v.x, v.y));
            const float2 z1 = make_float2(v.z, v.w);
            const float zn = DIMS == 4 ? cnorm(z0) + cnorm(z1) : cnorm(z0);
            float g = 3.0e38f, eg = 0.f;
            for (int o = 0; o < f.n_orb; ++o) {
                float P = z0.x * f.orb[o][0] + z0.y * f.orb[o][1];
                float Q = z0.y * f.orb[o][0] - z0.x * f.orb[o][1];
                if (DIMS == 4) {
                    P += z1.x * f.orb[o][2] + z1.y * f.orb[o][3];
                    Q += z1.y * f.orb[o][2] - z1.x * f.orb[o][3];
                }
                const float vv = (f.S == 4) ? fmaxf(fabsf(P), fabsf(Q)) : (f.S == 2 ? fabsf(P) : P);
                const float dd = zn + f.orbe[o] - 2.f * vv;
                if (dd < g) { g = dd; eg = f.orbe[o]; }
            }
            dist += fmaxf(g, 0.f);
            en += eg;
        }
        acc.nerr = ne;
        acc.ncnt = 1;
        acc.gsum = g2;
        acc.en = dist;
        acc.ed = en;
    }
    count_reduce(acc, cnt, s, blockIdx.x, gridDim.x, sigma2[s * s2_stride]);
}

template <int DIMS, int MT, int MB>
cudaError_t demap_t(const float2 *z, long zs, long a, long e, const double *s2, int s2s, float *llr,
                    long ls, const DemapCount &cnt, int n_streams, const FmtDev &f, cudaStream_t st) {
    dim3 grid((unsigned)((e - a + 255) / 256), (unsigned)n_streams);
    demap_kernel<DIMS, MT, MB><<<grid, 256, 0, st>>>(z, zs, a, e, s2, s2s, llr, ls, cnt, f);
    return cudaGetLastError();
}

template <int DIMS, int MT, int MB>
cudaError_t derot_demap_t(const void *y, long ys, const uint8_t *b, long bst, long a, long e,
                          const int *dsum, const double *mdsum, int kR, const int32_t *cin, int cis,
                          int32_t *cout, int cos, uint16_t *pc, long pcs, const double *s2f, double *s2o,
                          int s2s, float *llr, long ls, const DemapCount &cnt, const SymOut &sym, int n_streams,
                          const FmtDev &f, cudaStream_t st, int sk) {
    const int n_rng = (int)((e - a + kR - 1) / kR);
    constexpr int TILE = tile_of<DIMS>();
    dim3 grid((unsigned)((e - a + TILE - 1) / TILE), (unsigned)n_streams);
    derot_demap_kernel<DIMS, MT, MB><<<grid, 256, 0, st>>>(y, ys, b, bst, a, e, dsum, mdsum, n_rng, kR, cin, cis,
                                                           cout, cos, pc, pcs, s2f, s2o, s2s, llr, ls, cnt, sym, sk, f);
    return cudaGetLastError();
}

}  // namespace

// the most blocks any table's tiles need (the smallest tile)
long derot_demap_ctas(long len, int n_streams, int sm_avail) {
    (void)n_streams;
    (void)sm_avail;
    return (len + kTile - 1) / kTile;
}

cudaError_t launch_derot_demap(const void *y, long y_stride, const uint8_t *b, long b_stride,
                               long a, long e, const int *dsum, const double *mdsum, int kR,
                               const int32_t *carry_in, int cin_stride, int32_t *carry_out,
                               int cout_stride, uint16_t *pcode, long pc_stride,
                               const double *sigma2_fixed, double *sigma2_out, int s2_stride,
                               float *llr, long llr_stride, const DemapCount &cnt, const SymOut &sym,
                               int n_streams, const FmtDev &f, cudaStream_t st, int sk, int sm_avail) {
    (void)sm_avail;   // 1024-symbol tiles measured best whatever the SMs left by the LMS
    if (e <= a || n_streams <= 0) return cudaSuccess;
    if (!cnt.sd || !cnt.partial || !mdsum) return cudaErrorInvalidValue;
#define RX_DD(D_, M_, B_)                                                                                  \
    return derot_demap_t<D_, M_, B_>(y, y_stride, b, b_stride, a, e, dsum, mdsum, kR, carry_in, cin_stride, \
                                     carry_out, cout_stride, pcode, pc_stride, sigma2_fixed, sigma2_out,    \
                                     s2_stride, llr, llr_stride, cnt, sym, n_streams, f, st, sk)
    if (f.dims == 4 && f.M == 64) RX_DD(4, 64, 6);
    if (f.dims == 2 && f.M == 4) RX_DD(2, 4, 2);
    if (f.dims == 2 && f.M == 8) RX_DD(2, 8, 3);
    if (f.dims == 2 && f.M == 16) RX_DD(2, 16, 4);
    if (f.dims == 2 && f.M == 32) RX_DD(2, 32, 5);
    if (f.dims == 2 && f.M == 64) RX_DD(2, 64, 6);
    if (f.dims == 2 && f.M == 128) RX_DD(2, 128, 7);
#undef RX_DD
    return cudaErrorInvalidValue;
}

cudaError_t launch_count_llr(const float *llr, long llr_stride, const float *x4, long x_stride, long a, long e,
                             const double *sigma2, int s2_stride, const DemapCount &cnt, int n_streams,
                             const FmtDev &f, cudaStream_t st) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    if (!cnt.sd || !cnt.partial) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((e - a + 255) / 256), (unsigned)n_streams);
    const float4 *xv = reinterpret_cast<const float4 *>(x4);
    if (f.dims == 4 && f.m == 6)
        count_llr_kernel<4, 6><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else if (f.dims == 2 && f.m_pol == 2)
        count_llr_kernel<2, 2><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else if (f.dims == 2 && f.m_pol == 3)
        count_llr_kernel<2, 3><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else if (f.dims == 2 && f.m_pol == 4)
        count_llr_kernel<2, 4><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else if (f.dims == 2 && f.m_pol == 5)
        count_llr_kernel<2, 5><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else if (f.dims == 2 && f.m_pol == 6)
        count_llr_kernel<2, 6><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else if (f.dims == 2 && f.m_pol == 7)
        count_llr_kernel<2, 7><<<grid, 256, 0, st>>>(llr, llr_stride, xv, x_stride, a, e, sigma2, s2_stride, cnt, f);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_demap(const float2 *z, long z_stride, long z_off, long a, long e,
                         const double *sigma2, int sigma2_stride, float *llr, long llr_stride,
                         const DemapCount &cnt, int n_streams, const FmtDev &f, cudaStream_t st) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    const float2 *zz = z + z_off;
    if (f.dims == 4 && f.M == 64)
        return demap_t<4, 64, 6>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 4)
        return demap_t<2, 4, 2>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 8)
        return demap_t<2, 8, 3>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 16)
        return demap_t<2, 16, 4>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 32)
        return demap_t<2, 32, 5>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 64)
        return demap_t<2, 64, 6>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    if (f.dims == 2 && f.M == 128)
        return demap_t<2, 128, 7>(zz, z_stride, a, e, sigma2, sigma2_stride, llr, llr_stride, cnt, n_streams, f, st);
    return cudaErrorInvalidValue;
}
