// A4: blind phase search and its unwrap / de-rotation.
//
// BPS (per symbol k, test phases phi_b = (b/B - 1/2) 2 pi / S):
//   md_b(i)  = min_j || y_i exp(-j phi_b) - s_j ||^2
//   cost_b(k) = sum_{i = k - W/2}^{k + W/2 - 1} md_b(i)   (i outside [0, n_valid) adds 0)
//   b_k      = argmin_b cost_b(k)   (lowest b on ties)
// With the table closed under rotation by 2 pi / S, the minimum over the S
// members of an orbit {rep * j^k} follows from one correlation
// c = sum_p y_p conj(rep_p):  || y e^{-j phi} - rep j^k ||^2 =
// |y|^2 + |rep|^2 - 2 Re(e^{-j phi} (-j)^k c), so for S = 4 the orbit minimum
// is |y|^2 + |rep|^2 - 2 max(|P|, |Q|) with P + jQ = e^{-j phi} c.  The
// 4D 64-ary table has 16 orbits: 16 correlations per symbol, then per test
// phase 16 x (2 MUL + 2 FMA + max + FMA + min).
//
// Window sums: a warp computes md_b for 32 consecutive symbols (one per
// lane), scans them with shuffles and stores the exclusive prefix of every
// 32-symbol chunk and its total in a shared-memory ring of 10 chunks; a
// window of W <= 64 symbols then spans at most three chunks and costs three
// shared loads per test phase.  A block makes the outputs of a whole number
// of chunks in rounds of 8 chunks (one per warp), computing one extra chunk
// on each side; the launch splits each stream's range evenly.
//
// Unwrap (integer form of phi_hat_k = phi_k + q round((phi_hat_{k-1} -
// phi_k)/q), q = 2 pi/S, round(x) = floor(x + 1/2)):
//   m_k = m_{k-1} + floor((2 (b_{k-1} - b_k) + B) / (2B)),
// a prefix sum: the BPS kernel sums the increments inside its range, the
// unwrap kernel adds the block boundaries and scans its own range.
#include <algorithm>

#include <atomic>

#include "rx_internal.h"

namespace {

constexpr int kMaxChunks = 126;
constexpr int kMaxR = 32 * kMaxChunks;              // largest output range per block (4032)
constexpr int kMinChunks = 6;                       // halo (two chunks) at most a third

// Output symbols per block of `chunks` 32-symbol output chunks; the block
// computes the minimum distances of one halo chunk on each side as well,
// eight chunks per round (one per warp).
__host__ __device__ __forceinline__ int range_of(int chunks) { return 32 * chunks; }

__device__ __forceinline__ float orbit_v(float P, float Q, int S) {
    if (S == 4) return fmaxf(fabsf(P), fabsf(Q));
    if (S == 2) return fabsf(P);
    return P;
}

// |rep|^2 - 2 (orbit value at the test phase shifted by half the phase span,
// 2 pi / (2S)) from (P, Q) at the unshifted phase: the shift rotates P + jQ
// by -pi/4, -pi/2 or -pi, so max(|P'|, |Q'|) = (|P| + |Q|) / sqrt 2 (S = 4),
// |P'| = |Q| (S = 2), P' = -P (S = 1).
__device__ __forceinline__ float half_turn_d(float P, float Q, int S, float e) {
    if (S == 4) return fmaf(-1.41421356237309515f, fabsf(P) + fabsf(Q), e);
    if (S == 2) return fmaf(-2.f, fabsf(Q), e);
    return fmaf(2.f, P, e);
}

// Orbit value v and the half-turn value u of (P, Q) with their distance
// coefficients: d = e + cv * v at the test phase, d' = e + cu * u at the
// phase shifted by pi/S (see half_turn_d).
template <int SS>
__device__ __forceinline__ void orbit_vu(float P, float Q, float &v, float &u) {
    if (SS == 4) { v = fmaxf(fabsf(P), fabsf(Q)); u = fabsf(P) + fabsf(Q); }
    else if (SS == 2) { v = fabsf(P); u = fabsf(Q); }
    else { v = P; u = P; }
}
template <int SS> struct OrbitCoef {
    static constexpr float cv = -2.f;
    static constexpr float cu = SS == 4 ? -1.41421356237309515f : (SS == 2 ? -2.f : 2.f);
};

// SS: the table's rotation order S as a constant, so that the per-orbit
// value and the half-turn identity compile to their one case
template <int DIMS, int NORB, int SS>
__global__ void __launch_bounds__(256, 2)
bps_kernel(const void *__restrict__ y, long y_stride, long a, long e, long n_valid, int W,
           uint8_t *__restrict__ bout, long bout_stride, int *__restrict__ dsum,
           double *__restrict__ mdsum, int n_cta, int chunks, int sk, const __grid_constant__ FmtDev f) {
    extern __shared__ __align__(16) float smem[];
    const int B = f.B;
    const int kChunks = chunks, kR = range_of(chunks);
    const int rounds = (kChunks + 2 + 7) / 8;           // chunks -1 .. kChunks
    constexpr int kRow = 33;                              // padded row of 32 prefixes
    float *Eb = smem;                                     // [10][B][kRow] exclusive prefixes
    float *Tb = smem + RX_NCHUNK * B * kRow;              // [10][B] chunk totals
    float *T2 = Tb + RX_NCHUNK * B;                       // [8 warps][B] totals of two chunks
    uint8_t *bsm = reinterpret_cast<uint8_t *>(T2 + 8 * B);   // [kR]
    __shared__ int red[8];
    __shared__ float redm[8];
    const int s = blockIdx.y, c = blockIdx.x;
    const long out0 = a + (long)c * kR;
    float md_acc = 0.f;   // min distance at the chosen phase: the decision-directed noise
    const long out1 = min(out0 + kR, e);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long yoff = (long)s * 2 * y_stride;      // y of stream s: [2][y_stride], storage kind sk
    const int hw = W >> 1;

    for (int r = 0; r < rounds; ++r) {
        // ---- min distances of chunk jc for every test phase, scanned ----
        const int jc = 8 * r - 1 + warp;
        if (jc <= kChunks) {
            const long i = out0 + 32L * jc + lane;
            const bool valid = (i >= 0) && (i < n_valid);
            float2 ya = make_float2(0.f, 0.f), yb = make_float2(0.f, 0.f);
            if (valid) { ya = ld_sample(y, yoff + i, sk); yb = ld_sample(y, yoff + y_stride + i, sk); }
            // per orbit o (and polarisation for 2D tables): CR = (Re c, Im c) and
            // CI = (Im c, -Re c), c = sum_p y_p conj(rep_p); then for a test phase,
            // (P, Q) = cos(phi) CR + sin(phi) CI is one packed multiply and one packed FMA
            // 2D tables of more than 16 orbits (GS-128: 32) form the
            // correlations per pass over the test phases instead (registers)
            constexpr bool kBig = DIMS == 2 && NORB > 16;
            f32x2 CR[2][kBig ? 1 : NORB], CI[2][kBig ? 1 : NORB];
            float yn0, yn1;
            if (DIMS == 4) {
                yn0 = cnorm(ya) + cnorm(yb);
                yn1 = 0.f;
    #pragma unroll
                for (int o = 0; o < NORB; ++o) {
                    if (o < f.n_orb) {
                        const float r0 = f.orb[o][0], r1 = f.orb[o][1], r2 = f.orb[o][2], r3 = f.orb[o][3];
                        const float cr = ya.x * r0 + ya.y * r1 + yb.x * r2 + yb.y * r3;
                        const float ci = ya.y * r0 - ya.x * r1 + yb.y * r2 - yb.x * r3;
                        CR[0][o] = pk2(cr, ci);
                        CI[0][o] = pk2(ci, -cr);
                    }
                }
            } else if (!kBig) {
                yn0 = cnorm(ya);
                yn1 = cnorm(yb);
    #pragma unroll
                for (int o = 0; o < (kBig ? 1 : NORB); ++o) {
                    if (o < f.n_orb) {
                        const float r0 = f.orb[o][0], r1 = f.orb[o][1];
                        const float cr0 = ya.x * r0 + ya.y * r1, ci0 = ya.y * r0 - ya.x * r1;
                        const float cr1 = yb.x * r0 + yb.y * r1, ci1 = yb.y * r0 - yb.x * r1;
                        CR[0][o] = pk2(cr0, ci0);
                        CI[0][o] = pk2(ci0, -cr0);
                        CR[1][o] = pk2(cr1, ci1);
                        CI[1][o] = pk2(ci1, -cr1);
                    }
                }
            } else {
                yn0 = cnorm(ya);
                yn1 = cnorm(yb);
            }
            const int slot = (jc + 1) % RX_NCHUNK;
            const int hb = B >> 1;
            const float yq1 = (yn0 + yn1) + 2.f * f.orbe[0];      // one-orbit tables
            if constexpr (kBig) {
                // passes of eight phase pairs; per orbit pair the
                // correlations of both polarisations, then the phase pairs'
                // minima (the same roundings as the loop below; the minima
                // are exact in any order)
                constexpr int kCh = 8;
                for (int b0 = 0; b0 < hb; b0 += kCh) {
                    float x0[kCh], x1[kCh], w0[kCh], w1[kCh];
                    f32x2 Cp[kCh], Sp[kCh];          // (cos, cos), (sin, sin) of the pass's phases
#pragma unroll
                    for (int i = 0; i < kCh; ++i) {
                        x0[i] = x1[i] = w0[i] = w1[i] = 3.0e38f;
                        const f32x2 *cp1 = reinterpret_cast<const f32x2 *>(f.csp[min(b0 + i, hb - 1)]);
                        Cp[i] = cp1[0];
                        Sp[i] = cp1[1];
                    }
                    const f32x2 CV = pk2(OrbitCoef<SS>::cv, OrbitCoef<SS>::cv);
                    const f32x2 CU = pk2(OrbitCoef<SS>::cu, OrbitCoef<SS>::cu);
                    // two orbits at a time (as the 4D loop): their distances
                    // as packed FMAs, then three-input minima
#pragma unroll 1
                    for (int o = 0; o < NORB; o += 2) {
                        if (o < f.n_orb) {
                            const bool two = o + 1 < f.n_orb;
                            const float ra0 = f.orb[o][0], ra1 = f.orb[o][1];
                            const float rb0 = two ? f.orb[o + 1][0] : 0.f, rb1 = two ? f.orb[o + 1][1] : 0.f;
                            const f32x2 EO = pk2(f.orbe[o], two ? f.orbe[o + 1] : __int_as_float(0x7f800000));
                            f32x2 CRa[2], CIa[2], CRb[2], CIb[2];
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                const float2 yq = q ? yb : ya;
                                const float cra = yq.x * ra0 + yq.y * ra1, cia = yq.y * ra0 - yq.x * ra1;
                                const float crb = yq.x * rb0 + yq.y * rb1, cib = yq.y * rb0 - yq.x * rb1;
                                CRa[q] = pk2(cra, cia);
                                CIa[q] = pk2(cia, -cra);
                                CRb[q] = pk2(crb, cib);
                                CIb[q] = pk2(cib, -crb);
                            }
#pragma unroll
                            for (int i = 0; i < kCh; ++i) {
                                if (b0 + i < hb) {
                                    const f32x2 C1 = Cp[i], S1 = Sp[i];
#pragma unroll
                                    for (int q = 0; q < 2; ++q) {
                                        float P, Q, R, U, v0, u0, v1, u1, d0, d1, h0, h1;
                                        upk2(fma2(S1, CIa[q], mul2(C1, CRa[q])), P, Q);
                                        upk2(fma2(S1, CIb[q], mul2(C1, CRb[q])), R, U);
                                        orbit_vu<SS>(P, Q, v0, u0);
                                        orbit_vu<SS>(R, U, v1, u1);
                                        upk2(fma2(CV, pk2(v0, v1), EO), d0, d1);
                                        upk2(fma2(CU, pk2(u0, u1), EO), h0, h1);
                                        if (q == 0) {
                                            x0[i] = fmin3(x0[i], d0, d1);
                                            w0[i] = fmin3(w0[i], h0, h1);
                                        } else {
                                            x1[i] = fmin3(x1[i], d0, d1);
                                            w1[i] = fmin3(w1[i], h0, h1);
                                        }
                                    }
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int i = 0; i < kCh; ++i) {
                        const int b = b0 + i;
                        if (b < hb) {
                            float md = (yn0 + x0[i]) + (yn1 + x1[i]);
                            float md2 = (yn0 + w0[i]) + (yn1 + w1[i]);
                            if (!valid) { md = 0.f; md2 = 0.f; }
                            Eb[(slot * B + b) * kRow + lane] = md;
                            Eb[(slot * B + b + hb) * kRow + lane] = md2;
                        }
                    }
                }
            } else {
            // test phases b and b + B/2 together: phi_{b+B/2} = phi_b + pi/S, a
            // rotation of P + jQ that half_turn_d applies without another multiply
            // two phase pairs per trip: independent min chains for the scheduler
#pragma unroll 2
            for (int b = 0; b < hb; ++b) {
                const f32x2 *cp1 = reinterpret_cast<const f32x2 *>(f.csp[b]);
                const f32x2 C1 = cp1[0], S1 = cp1[1];
                float md, md2;
                if (DIMS == 4) {
                    // two orbits per step: (e - 2v) and (e + cu u) of both as one
                    // packed FMA each, then a three-input min
                    float a0 = 3.0e38f, a1 = 3.0e38f;
                    const f32x2 CV = pk2(OrbitCoef<SS>::cv, OrbitCoef<SS>::cv);
                    const f32x2 CU = pk2(OrbitCoef<SS>::cu, OrbitCoef<SS>::cu);
    #pragma unroll
                    for (int o = 0; o + 1 < NORB; o += 2) {
                        float P, Q, R, U, v0, u0, v1, u1, d0, d1, h0, h1;
                        upk2(fma2(S1, CI[0][o], mul2(C1, CR[0][o])), P, Q);
                        upk2(fma2(S1, CI[0][o + 1], mul2(C1, CR[0][o + 1])), R, U);
                        orbit_vu<SS>(P, Q, v0, u0);
                        orbit_vu<SS>(R, U, v1, u1);
                        const f32x2 EO = pk2(f.orbe[o], f.orbe[o + 1]);
                        upk2(fma2(CV, pk2(v0, v1), EO), d0, d1);
                        upk2(fma2(CU, pk2(u0, u1), EO), h0, h1);
                        a0 = fmin3(a0, d0, d1);
                        a1 = fmin3(a1, h0, h1);
                    }
                    if (NORB & 1) {
                        float P, Q;
                        upk2(fma2(S1, CI[0][NORB - 1], mul2(C1, CR[0][NORB - 1])), P, Q);
                        a0 = fminf(a0, fmaf(-2.f, orbit_v(P, Q, SS), f.orbe[NORB - 1]));
                        a1 = fminf(a1, half_turn_d(P, Q, SS, f.orbe[NORB - 1]));
                    }
                    md = yn0 + a0;
                    md2 = yn0 + a1;
                } else if (NORB == 1) {
                    // one orbit (QPSK): no minimum over orbits, so both
                    // polarisations' distances share one sum, |y_X|^2 +
                    // |y_Y|^2 + 2 e - 2 (v_X + v_Y)
                    float P0, Q0, P1, Q1, v0, u0, v1, u1;
                    upk2(fma2(S1, CI[0][0], mul2(C1, CR[0][0])), P0, Q0);
                    upk2(fma2(S1, CI[1][0], mul2(C1, CR[1][0])), P1, Q1);
                    orbit_vu<SS>(P0, Q0, v0, u0);
                    orbit_vu<SS>(P1, Q1, v1, u1);
                    md = fmaf(OrbitCoef<SS>::cv, v0 + v1, yq1);
                    md2 = fmaf(OrbitCoef<SS>::cu, u0 + u1, yq1);
                } else {
                    float x0 = 3.0e38f, x1 = 3.0e38f, w0 = 3.0e38f, w1 = 3.0e38f;
    #pragma unroll
                    for (int o = 0; o < (kBig ? 1 : NORB); ++o) {
                        float P0, Q0, P1, Q1;
                        upk2(fma2(S1, CI[0][o], mul2(C1, CR[0][o])), P0, Q0);
                        upk2(fma2(S1, CI[1][o], mul2(C1, CR[1][o])), P1, Q1);
                        x0 = fminf(x0, fmaf(-2.f, orbit_v(P0, Q0, SS), f.orbe[o]));
                        x1 = fminf(x1, fmaf(-2.f, orbit_v(P1, Q1, SS), f.orbe[o]));
                        w0 = fminf(w0, half_turn_d(P0, Q0, SS, f.orbe[o]));
                        w1 = fminf(w1, half_turn_d(P1, Q1, SS, f.orbe[o]));
                    }
                    md = (yn0 + x0) + (yn1 + x1);
                    md2 = (yn0 + w0) + (yn1 + w1);
                }
                if (!valid) { md = 0.f; md2 = 0.f; }
                Eb[(slot * B + b) * kRow + lane] = md;
                Eb[(slot * B + b + hb) * kRow + lane] = md2;
            }
            }
            __syncwarp();
            // exclusive prefix of every test phase's row over the chunk's 32
            // symbols, in place: lane l takes phases l and l + 32 (rows padded to
            // 33 floats, so the lanes' serial walks hit 32 different banks)
            if (B == 64) {
                // two independent rows per lane, interleaved
                float *ra = Eb + (slot * B + lane) * kRow, *rb = ra + 32 * kRow;
                float run_a = 0.f, run_b = 0.f;
    #pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float va = ra[j], vb = rb[j];
                    ra[j] = run_a;
                    rb[j] = run_b;
                    run_a += va;
                    run_b += vb;
                }
                Tb[slot * B + lane] = run_a;
                Tb[slot * B + lane + 32] = run_b;
            } else {
                for (int b = lane; b < B; b += 32) {
                    float *row = Eb + (slot * B + b) * kRow;
                    float run = 0.f;
    #pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float v = row[j];
                        row[j] = run;
                        run += v;
                    }
                    Tb[slot * B + b] = run;
                }
            }
        }
        __syncthreads();
        // ---- window costs and argmin for output chunk oc ----
        const int oc = 8 * r - 2 + warp;
        // totals of chunks oc - 1 and oc per test phase (the middle of a
        // 64-symbol window), once per warp
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
                const int c0 = (i0 >= 0) ? (i0 >> 5) : -1;   // i0 >= -32
                const int l0 = i0 - 32 * c0;
                const int c1 = i1 >> 5, l1 = i1 - 32 * c1;
                const int s0 = (c0 + 1) % RX_NCHUNK, s1 = (c1 + 1) % RX_NCHUNK;
                const int sm = (c0 + 2) % RX_NCHUNK;
                float best = 3.0e38f;
                int bb = 0;
                const float *e0 = Eb + s0 * B * kRow + l0, *e1 = Eb + s1 * B * kRow + l1;
                if (c0 == oc - 1 && c1 == oc + 1 && (B & 3) == 0) {
                    // window over chunks oc - 1 .. oc + 1: the two-chunk total
                    // minus the head of chunk oc - 1 plus the head of oc + 1.
                    // Four argmin chains (phases b = 4 q + j) keep the compare
                    // latency off a single chain; each keeps its lowest phase on
                    // ties, and the merge takes the lowest phase of equal costs
                    float bst[4] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f};
                    int bi[4] = {0, 1, 2, 3};
#pragma unroll 2
                    for (int b = 0; b < B; b += 4) {
                        const float4 t = *reinterpret_cast<const float4 *>(t2 + b);
                        const float tt[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float cst = (tt[j] - e0[(b + j) * kRow]) + e1[(b + j) * kRow];
                            if (cst < bst[j]) { bst[j] = cst; bi[j] = b + j; }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (bst[j] < best || (bst[j] == best && bi[j] < bb)) { best = bst[j]; bb = bi[j]; }
                } else if (c0 == oc - 1 && c1 == oc + 1) {
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
                        if (c1 - c0 == 2) cst += Tb[sm * B + b];
                        cst += e1[b * kRow];
                        if (cst < best) { best = cst; bb = b; }
                    }
                }
                bsm[k - out0] = (uint8_t)bb;
                bout[(long)s * bout_stride + (k - a)] = (uint8_t)bb;
                // md at (bb, k) from the chunk prefixes: |z_k - d_k|^2 of the
                // de-rotated symbol (the table is closed under the rotations)
                const int sc = (oc + 1) % RX_NCHUNK;
                const float hi = (lane < 31) ? Eb[(sc * B + bb) * kRow + lane + 1] : Tb[sc * B + bb];
                md_acc += hi - Eb[(sc * B + bb) * kRow + lane];
            }
        }
        __syncthreads();
    }
    // ---- unwrap increments inside this block's range (boundary excluded) ----
    int acc = 0;
    const int nloc = (int)(out1 - out0);
    for (int t = tid + 1; t < nloc; t += 256) acc += unwrap_step(bsm[t - 1], bsm[t], B);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        acc += __shfl_xor_sync(0xffffffffu, acc, off);
        md_acc += __shfl_xor_sync(0xffffffffu, md_acc, off);
    }
    if (lane == 0) { red[warp] = acc; redm[warp] = md_acc; }
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        double mt = 0.0;
        for (int w = 0; w < 8; ++w) { tot += red[w]; mt += (double)redm[w]; }
        dsum[s * n_cta + c] = tot;
        if (mdsum) mdsum[s * n_cta + c] = mt;
    }
}

// nearest-point squared distance of z (orbit form)
template <int DIMS, int NORB>
__device__ __forceinline__ float nearest_dist(float2 z0, float2 z1, const FmtDev &f) {
    if (DIMS == 4) {
        const float zn = cnorm(z0) + cnorm(z1);
        float best = 3.0e38f;
#pragma unroll
        for (int o = 0; o < NORB; ++o) {
            if (o < f.n_orb) {
                const float P = z0.x * f.orb[o][0] + z0.y * f.orb[o][1] + z1.x * f.orb[o][2] + z1.y * f.orb[o][3];
                const float Q = z0.y * f.orb[o][0] - z0.x * f.orb[o][1] + z1.y * f.orb[o][2] - z1.x * f.orb[o][3];
                best = fminf(best, f.orbe[o] - 2.f * orbit_v(P, Q, f.S));
            }
        }
        return fmaxf(zn + best, 0.f);
    } else {
        float tot = 0.f;
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float2 zp = p ? z1 : z0;
            float best = 3.0e38f;
#pragma unroll
            for (int o = 0; o < NORB; ++o) {
                if (o < f.n_orb) {
                    const float P = zp.x * f.orb[o][0] + zp.y * f.orb[o][1];
                    const float Q = zp.y * f.orb[o][0] - zp.x * f.orb[o][1];
                    best = fminf(best, f.orbe[o] - 2.f * orbit_v(P, Q, f.S));
                }
            }
            tot += fmaxf(cnorm(zp) + best, 0.f);
        }
        return tot;
    }
}

template <int DIMS, int NORB>
__global__ void __launch_bounds__(256)
unwrap_kernel(const float2 *__restrict__ y, long y_stride, const uint8_t *__restrict__ bsrc,
              long b_stride, long a, long e, const int *__restrict__ dsum, int n_cta,
              const int32_t *__restrict__ carry_in, int cin_stride, int32_t *__restrict__ carry_out,
              int cout_stride, float2 *__restrict__ z, long z_stride, uint16_t *__restrict__ pcode,
              long pc_stride, double *__restrict__ partial, double *__restrict__ sigma2_out,
              int s2_stride, unsigned int *__restrict__ ticket, int ticket_stride, int kR,
              const double *__restrict__ mdsum, const __grid_constant__ FmtDev f) {
    __shared__ uint8_t bl[kMaxR];
    __shared__ uint8_t mql[kMaxR];
    __shared__ int wsum[8];
    __shared__ int mstart_sh;
    __shared__ double dred[8];
    __shared__ bool last;
    const int s = blockIdx.y, c = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long out0 = a + (long)c * kR;
    const long out1 = min(out0 + kR, e);
    const int nloc = (int)(out1 - out0);
    const int B = f.B, S = f.S;
    const uint8_t *bs = bsrc + (long)s * b_stride;   // index k - a
    const int m_in = carry_in[s * cin_stride + 0], b_in = carry_in[s * cin_stride + 1];

    // m at the start of this range: carry + increments of all earlier ranges
    if (warp == 0) {
        int acc = 0;
        for (int cc = lane; cc < c; cc += 32) {
            const long st0 = a + (long)cc * kR;
            const int bp = (cc == 0) ? b_in : bs[st0 - 1 - a];
            acc += unwrap_step(bp, bs[st0 - a], B) + dsum[s * n_cta + cc];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) mstart_sh = m_in + acc;
    }
    for (int t = tid; t < nloc; t += 256) bl[t] = bs[out0 - a + t];
    __syncthreads();
    const int bprev0 = (c == 0) ? b_in : (int)bs[out0 - 1 - a];

    // block scan of the increments: thread t owns local symbols PT t .. PT t + PT - 1
    constexpr int PT = (kMaxR + 255) / 256;
    int d[PT], run = 0;
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
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int wpre = 0;
    for (int w = 0; w < warp; ++w) wpre += wsum[w];
    const int tpre = mstart_sh + wpre + incl - run;   // m before this thread's symbols

    // quadrant count m mod S of every local symbol into shared memory; the
    // de-rotation below then walks the symbols in coalesced order
#pragma unroll
    for (int u = 0; u < PT; ++u) {
        const int t = PT * tid + u;
        if (t >= nloc) continue;
        const int m = tpre + d[u];
        mql[t] = (uint8_t)(((m % S) + S) % S);
        if (out0 + t == e - 1) {
            carry_out[s * cout_stride + 0] = m;
            carry_out[s * cout_stride + 1] = bl[t];
        }
    }
    __syncthreads();
    const float2 *yx = y + (long)s * 2 * y_stride;
    const float2 *yy = yx + y_stride;
    float2 *zx = z + (long)s * 2 * z_stride;
    float2 *zy = zx + z_stride;
    uint16_t *pc = pcode + (long)s * pc_stride;
    double dsum_loc = 0.0;
#pragma unroll 4
    for (int t = tid; t < nloc; t += 256) {
        const long k = out0 + t;
        const int b = bl[t], mq = mql[t];
        // exp(-j phi) = conj(cs_b) (-j)^mq
        float2 rot = make_float2(f.cs[b][0], -f.cs[b][1]);
        if (S == 4) {
            if (mq & 2) rot = make_float2(-rot.x, -rot.y);
            if (mq & 1) rot = make_float2(rot.y, -rot.x);
        } else if (S == 2) {
            if (mq) rot = make_float2(-rot.x, -rot.y);
        }
        const float2 z0 = cmul(yx[k], rot), z1 = cmul(yy[k], rot);
        zx[k - a] = z0;
        zy[k - a] = z1;
        pc[k - a] = (uint16_t)(b | (mq << 8));
        if (!mdsum) dsum_loc += (double)nearest_dist<DIMS, NORB>(z0, z1, f);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) dsum_loc += __shfl_xor_sync(0xffffffffu, dsum_loc, off);
    if (lane == 0) dred[warp] = dsum_loc;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < 8; ++w) tot += dred[w];
        partial[(long)s * n_cta + c] = mdsum ? mdsum[(long)s * n_cta + c] : tot;
        __threadfence();
        const unsigned prev = atomicAdd(&ticket[s * ticket_stride], 1u);
        last = (prev == (unsigned)n_cta - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const volatile double *pp = partial + (long)s * n_cta;
    double v = 0.0;
    for (int cc = tid; cc < n_cta; cc += 256) v += pp[cc];
    __shared__ double tr[256];
    tr[tid] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (tid < w) tr[tid] += tr[tid + w];
        __syncthreads();
    }
    if (tid == 0) {
        sigma2_out[s * s2_stride] = tr[0] / (2.0 * (double)(e - a));
        ticket[s * ticket_stride] = 0u;
    }
}

// interior unwrap increments of each kR range, from phase indices b (index k - a)
__global__ void dsum_kernel(const uint8_t *__restrict__ b, long b_stride, long a, long e,
                            int *__restrict__ dsum, int n_cta, int B, int kR) {
    __shared__ int red[8];
    const int s = blockIdx.y, c = blockIdx.x, tid = threadIdx.x;
    const long out0 = a + (long)c * kR, out1 = min(out0 + kR, e);
    const uint8_t *bs = b + (long)s * b_stride;
    int acc = 0;
    for (long k = out0 + 1 + tid; k < out1; k += 256) acc += unwrap_step(bs[k - 1 - a], bs[k - a], B);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        int tot = 0;
        for (int w = 0; w < 8; ++w) tot += red[w];
        dsum[s * n_cta + c] = tot;
    }
}

template <int DIMS, int NORB, int SS>
cudaError_t bps_launch_t(const void *y, long ys, long a, long e, long nv, int W, uint8_t *bout,
                         long bst, int *dsum, double *mdsum, int chunks, int n_streams,
                         const FmtDev &f, cudaStream_t st, int sk) {
    const int kR = range_of(chunks);
    const int n_cta = (int)((e - a + kR - 1) / kR);
    const size_t smem = sizeof(float) * (RX_NCHUNK * f.B * 33 + RX_NCHUNK * f.B + 8 * f.B) + kR + 16;
    auto kern = bps_kernel<DIMS, NORB, SS>;
    // the dynamic shared-memory limit is set once per device, to the largest
    // any launch can ask for (RX_MAXB phases, kMaxChunks chunks), so that host
    // threads issuing concurrently never lower it under one another's launch
    constexpr size_t kMaxSmem =
        sizeof(float) * (RX_NCHUNK * RX_MAXB * 33 + RX_NCHUNK * RX_MAXB + 8 * RX_MAXB) + 32 * kMaxChunks + 16;
    if (smem > kMaxSmem) return cudaErrorInvalidValue;
    static std::atomic<unsigned long long> set_on{0};   // bit d: set on device d
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev >= 64 || !((set_on.load(std::memory_order_relaxed) >> dev) & 1ull)) {
        err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
        if (err != cudaSuccess) return err;
        if (dev < 64) set_on.fetch_or(1ull << dev, std::memory_order_relaxed);
    }
    dim3 grid((unsigned)n_cta, (unsigned)n_streams);
    kern<<<grid, 256, smem, st>>>(y, ys, a, e, nv, W, bout, bst, dsum, mdsum, n_cta, chunks, sk, f);
    return cudaGetLastError();
}

}  // namespace

int bps_cta_range(int chunks) { return range_of(chunks); }

int sm_count() {
    static std::atomic<int> cached{0};
    int n = cached.load(std::memory_order_relaxed);
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
        cached.store(n, std::memory_order_relaxed);
    }
    return n;
}

// Output chunks per block so that one launch of S streams x len outputs is
// about one wave of 2 blocks per SM: the fewest blocks per stream that fit
// in the wave, with the range split evenly among them (whole chunks), so the
// blocks carry equal work (the ring of 10 chunks takes ~88 KB per block).
int bps_chunks(long len, int n_streams, int sm_avail) {
    if (sm_avail <= 0) sm_avail = sm_count();
    const long per_stream = std::max(1L, (long)(2 * sm_avail) / std::max(1, n_streams));
    const long nch = std::max(1L, (len + 31) / 32);
    long c = (nch + per_stream - 1) / per_stream;                  // chunks per block
    c = std::max<long>(c, kMinChunks);
    c = std::min<long>(c, kMaxChunks);
    return (int)c;
}

// Start quadrant of the unwrap from the training phases (one block per
// stream): unwrap b[0..n) from phi_hat = 0 (m0), compare with the training
// phase codes in grid units, q_k = floor((2 d_k + B) / (2B)) mod S with
// d_k = (b_train - b_k) + B ((m_train - m0_k) mod S), and write the most
// common q (lowest on ties) with b = B/2 as the unwrap carry.
__global__ void __launch_bounds__(256)
anchor_kernel(const uint8_t *__restrict__ b, long b_stride, const uint16_t *__restrict__ tcode,
              long t_stride, int n, int32_t *__restrict__ carry, int carry_stride, int B, int S) {
    __shared__ int tot[256];
    __shared__ int votes[4];
    const int s = blockIdx.x, tid = threadIdx.x;
    const uint8_t *bs = b + (long)s * b_stride;
    const uint16_t *ts = tcode + (long)s * t_stride;
    if (tid < 4) votes[tid] = 0;
    const int L = (n + 255) / 256, i0 = min(n, tid * L), i1 = min(n, i0 + L);
    int run = 0;
    for (int i = i0; i < i1; ++i) run += unwrap_step(i == 0 ? B / 2 : bs[i - 1], bs[i], B);
    tot[tid] = run;
    __syncthreads();
    if (tid == 0) {                      // exclusive scan of the 256 segment totals
        int acc = 0;
        for (int t = 0; t < 256; ++t) { const int v = tot[t]; tot[t] = acc; acc += v; }
    }
    __syncthreads();
    int m0 = tot[tid];
    for (int i = i0; i < i1; ++i) {
        m0 += unwrap_step(i == 0 ? B / 2 : bs[i - 1], bs[i], B);
        const int bt = ts[i] & 255, mt = (ts[i] >> 8) & 3;
        const int dm = (((mt - m0) % S) + S) % S;
        const int d = (bt - (int)bs[i]) + B * dm;
        const int num = 2 * d + B;
        const int q = ((num >= 0 ? num / (2 * B) : -((-num + 2 * B - 1) / (2 * B))) % S + S) % S;
        atomicAdd(&votes[q], 1);
    }
    __syncthreads();
    if (tid == 0) {
        int best = 0;
        for (int q = 1; q < S; ++q)
            if (votes[q] > votes[best]) best = q;
        carry[s * carry_stride + 0] = best;
        carry[s * carry_stride + 1] = B / 2;
    }
}

cudaError_t launch_anchor(const uint8_t *b, long b_stride, const uint16_t *tcode, long t_stride,
                          int n, int32_t *carry, int carry_stride, int n_streams, int B, int S,
                          cudaStream_t st) {
    if (n <= 0 || n_streams <= 0) return cudaSuccess;
    anchor_kernel<<<n_streams, 256, 0, st>>>(b, b_stride, tcode, t_stride, n, carry, carry_stride, B, S);
    return cudaGetLastError();
}

cudaError_t launch_dsum_from_b(const uint8_t *b, long b_stride, long a, long e, int *dsum,
                               int chunks, int n_streams, int B, cudaStream_t st) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    const int kR = range_of(chunks);
    const int n_cta = (int)((e - a + kR - 1) / kR);
    dim3 grid((unsigned)n_cta, (unsigned)n_streams);
    dsum_kernel<<<grid, 256, 0, st>>>(b, b_stride, a, e, dsum, n_cta, B, kR);
    return cudaGetLastError();
}

cudaError_t launch_bps(const void *y, long y_stride, long a, long e, long n_valid, int W,
                       uint8_t *bout, long bout_stride, long bout_off, int *dsum, double *mdsum,
                       int chunks, int n_streams, const FmtDev &f, cudaStream_t st, int sk) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    if (chunks < 1 || chunks > kMaxChunks || (f.B & 1)) return cudaErrorInvalidValue;
    uint8_t *bo = bout + bout_off;
#define RX_BPS(DD, NO)                                                                                   \
    switch (f.S) {                                                                                       \
        case 4: return bps_launch_t<DD, NO, 4>(y, y_stride, a, e, n_valid, W, bo, bout_stride, dsum, mdsum, \
                                               chunks, n_streams, f, st, sk);                             \
        case 2: return bps_launch_t<DD, NO, 2>(y, y_stride, a, e, n_valid, W, bo, bout_stride, dsum, mdsum, \
                                               chunks, n_streams, f, st, sk);                             \
        case 1: return bps_launch_t<DD, NO, 1>(y, y_stride, a, e, n_valid, W, bo, bout_stride, dsum, mdsum, \
                                               chunks, n_streams, f, st, sk);                             \
        default: return cudaErrorInvalidValue;                                                           \
    }
    if (f.dims == 4) {
        switch (f.n_orb) {
            case 16: RX_BPS(4, 16);
            case 8: RX_BPS(4, 8);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (f.n_orb) {
        case 1: RX_BPS(2, 1);
        case 2: RX_BPS(2, 2);
        case 4: RX_BPS(2, 4);
        case 8: RX_BPS(2, 8);
        case 16: RX_BPS(2, 16);
        case 32: RX_BPS(2, 32);
        default: return cudaErrorInvalidValue;
    }
#undef RX_BPS
}

cudaError_t launch_unwrap(const float2 *y, long y_stride, const uint8_t *b, long b_stride,
                          long b_off, long a, long e, const int *dsum,
                          const int32_t *carry_in, int carry_in_stride,
                          int32_t *carry_out, int carry_out_stride,
                          float2 *z, long z_stride, long z_off,
                          uint16_t *pcode, long pcode_stride, long pcode_off,
                          double *partial, double *sigma2_out, int sigma2_stride,
                          unsigned int *ticket, int ticket_stride, int chunks,
                          const double *mdsum, int n_streams, const FmtDev &f, cudaStream_t st) {
    if (e <= a || n_streams <= 0) return cudaSuccess;
    if (chunks < 1 || chunks > kMaxChunks) return cudaErrorInvalidValue;
    const int kR = range_of(chunks);
    const int n_cta = (int)((e - a + kR - 1) / kR);
    dim3 grid((unsigned)n_cta, (unsigned)n_streams);
    if (f.dims == 4) {
        unwrap_kernel<4, 16><<<grid, 256, 0, st>>>(y, y_stride, b + b_off, b_stride, a, e, dsum, n_cta,
                                                    carry_in, carry_in_stride, carry_out, carry_out_stride,
                                                    z + z_off, z_stride, pcode + pcode_off, pcode_stride,
                                                    partial, sigma2_out, sigma2_stride, ticket, ticket_stride, kR, mdsum, f);
    } else {
        // NORB bounds the orbit loop (predicated on f.n_orb): 16, or 32 for larger 2D tables
        if (f.n_orb > 16)
            unwrap_kernel<2, 32><<<grid, 256, 0, st>>>(y, y_stride, b + b_off, b_stride, a, e, dsum, n_cta,
                                                        carry_in, carry_in_stride, carry_out, carry_out_stride,
                                                        z + z_off, z_stride, pcode + pcode_off, pcode_stride,
                                                        partial, sigma2_out, sigma2_stride, ticket, ticket_stride, kR,
                                                        mdsum, f);
        else
            unwrap_kernel<2, 16><<<grid, 256, 0, st>>>(y, y_stride, b + b_off, b_stride, a, e, dsum, n_cta,
                                                        carry_in, carry_in_stride, carry_out, carry_out_stride,
                                                        z + z_off, z_stride, pcode + pcode_off, pcode_stride,
                                                        partial, sigma2_out, sigma2_stride, ticket, ticket_stride, kR,
                                                        mdsum, f);
    }
    return cudaGetLastError();
}
