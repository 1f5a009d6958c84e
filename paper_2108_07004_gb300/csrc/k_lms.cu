// A3: block-wise adaptation of the 2x2 butterfly (CMA, then DD-LMS).
//
// The recursion is sequential (Sec. 2: the adaptive equaliser is the
// hard-to-parallelise step; the paper runs it on its own processing stream
// next to the parallel kernels, as the library does when the tap lag is
// >= 2).  An update is
//   y_q   = sum conj(h_qp[t]) x_p[2k + D - t]
//   CMA:  e_q = (R^2 - |y_q|^2) y_q
//   DD:   z = y exp(-j phi_k); d = nearest table point (orbit per lane,
//         (distance, label) min over 16 lanes, ties -> lowest label; taken
//         a sub-block ahead where the margin allows, see lms_kernel);
//         e_q = d_q exp(j phi_k) - y_q
//   h_qp[t] += mu conj(e_q) x_p[2k + D - t]
// Per stream one block of 12 warps (see lms_kernel), in sub-blocks of 16
// updates with a look-ahead of one sub-block: a decision warp takes the
// sequential decisions (each lane holds the partial output of one update and
// adds one correlation term per decision); a tap group of four warps applies
// the previous sub-block's updates to the taps and forms the next
// sub-block's outputs from them; a correlation group of four warps forms the
// window correlations r(j, j + d) the decision warp's corrections need.  The
// samples of up to 1024 updates are staged in shared memory by the whole
// block before the warps run through them.
//
// The start-up training alignment (Sec. 2: the equaliser first converges on
// a known sequence) is align_kernel: it correlates the equalised training
// span with the known symbols and fixes the output order and phases.
#include <algorithm>
#include <type_traits>

#include <atomic>

#include "rx_internal.h"

namespace {

constexpr int kCH = 1024;      // updates staged per chunk
constexpr int kSB = 16;        // updates per sub-block
constexpr int kLag = 2 * kSB;  // correlation lags kept per row: 0 .. 31 (lag 0 is zero)
// warp 0 decides; warps 4 and 8 share its scheduler and do no phase work;
// helper warps 1, 2, 3, 5 form the tap group, 6, 7, 9, 10 the correlation
// group, 11 stages only
constexpr int kWarps = 12;
constexpr int kThreads = 32 * kWarps;
constexpr int kBarTap = 1;     // named barrier of the tap group (128 threads)
constexpr int kBarCor = 2;     // named barrier of the correlation group (128 threads)

// shared-memory layout of lms_kernel<T> (float2 units)
__host__ __device__ constexpr int lms_nsx(int T) { return 2 * kCH + (T - 1) + 2 * (kSB + kLag) + 4; }
__host__ __device__ constexpr int lms_off_h(int T) { return 2 * lms_nsx(T); }
__host__ __device__ constexpr int lms_off_r(int T) { return lms_off_h(T) + 8 * T; }   // taps: room for 2T per branch
__host__ __device__ constexpr int lms_off_rp(int T) { return lms_off_r(T) + 2 * kSB * kLag; }
__host__ __device__ constexpr int lms_off_b(int T) { return lms_off_rp(T) + kSB * kLag * 4; }
__host__ __device__ constexpr int lms_off_e(int T) { return lms_off_b(T) + 2 * kSB * 2; }
__host__ __device__ constexpr int lms_off_rot(int T) { return lms_off_e(T) + 2 * kSB * 2; }
__host__ __device__ constexpr int lms_off_pc(int T) { return lms_off_rot(T) + 3 * kCH; }
__host__ __device__ constexpr int lms_smem_f2(int T) { return lms_off_pc(T) + kCH / 4 + kCH / 4; }

__device__ __forceinline__ void bar_sync(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

struct Tables {
    float4 orb[RX_MAXM];
    float orbe[RX_MAXM];
    int orblab[RX_MAXM][4];
    float4 pts[RX_MAXM];
    float4 rpts[RX_MAXM];   // point of orbit o turned by k (k < S) at o S + k
    float2 cs[RX_MAXB];
};

__device__ __forceinline__ void load_tables(Tables &tb, const FmtDev &f) {
    // at least 16 orbit entries: past n_orb a zero representative of energy
    // +inf, never a candidate of the orbit searches
    for (int i = threadIdx.x; i < max(f.n_orb, 16); i += blockDim.x) {
        const bool v = i < f.n_orb;
        tb.orb[i] = v ? make_float4(f.orb[i][0], f.orb[i][1], f.orb[i][2], f.orb[i][3]) : make_float4(0.f, 0.f, 0.f, 0.f);
        tb.orbe[i] = v ? f.orbe[i] : __int_as_float(0x7f800000);
        for (int k = 0; k < 4; ++k) tb.orblab[i][k] = v ? f.orb_lab[i][k] : 0;
    }
    for (int i = threadIdx.x; i < f.M; i += blockDim.x)
        tb.pts[i] = make_float4(f.pts[i][0], f.pts[i][1], f.pts[i][2], f.pts[i][3]);
    for (int i = threadIdx.x; i < f.n_orb * f.S; i += blockDim.x) {
        const int lab = f.orb_lab[i / f.S][i % f.S] & 255;
        tb.rpts[i] = make_float4(f.pts[lab][0], f.pts[lab][1], f.pts[lab][2], f.pts[lab][3]);
    }
    for (int i = threadIdx.x; i < f.B; i += blockDim.x) tb.cs[i] = make_float2(f.cs[i][0], f.cs[i][1]);
}

// Best rotation of an orbit given P + jQ = sum_p y_p conj(rep_p exp(j phi))
// (Re of the correlation with rep * j^k is P, Q, -P, -Q for k = 0..3): its
// value v and the label of that rotation (lab[k] = label of rep * j^k).
__device__ __forceinline__ void best_rot_label(float P, float Q, int S, const int (&lab)[4], float &v, int &label) {
    if (S == 4) {
        const float aP = fabsf(P), aQ = fabsf(Q);
        const bool pw = aP >= aQ;
        v = pw ? aP : aQ;
        label = pw ? (P >= 0.f ? lab[0] : lab[2]) : (Q >= 0.f ? lab[1] : lab[3]);
    } else if (S == 2) {
        v = fabsf(P);
        label = P >= 0.f ? lab[0] : lab[1];
    } else {
        v = P;
        label = lab[0];
    }
}

// Nearest table point of the candidates held by the lanes: each lane holds
// its orbit's best rotation, the squared distance and the label (lanes
// without an orbit hold +inf); the minimum distance wins and exact ties go
// to the lowest label.  Two warp reductions return the winning label.
__device__ __forceinline__ int argmin_label(float dist, int label) {
    const unsigned bits = __float_as_uint(fmaxf(dist, 0.f));
    const unsigned mn = __reduce_min_sync(0xffffffffu, bits);
    const unsigned key = (bits == mn) ? (unsigned)label : 0xffffffffu;
    return (int)__reduce_min_sync(0xffffffffu, key);
}

// a b with its rounding fixed (one product rounded, then one fused
// multiply-add), so a table point turned by a phase is the same value
// wherever it is formed; with sub_rn the decision-directed error
// d exp(j phi) - y is the same whichever path took the decision
__device__ __forceinline__ float2 cmul_fixed(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -__fmul_rn(a.y, b.y)), fmaf(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 sub_rn(float2 a, float2 b) {
    return make_float2(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y));
}

// Orbit o's two best rotations (for S = 4 the values max and min of |P|,
// |Q|): their squared distances dA <= dB and o S + k of the nearer (k quarter
// turns).
template <int DIMS>
__device__ __forceinline__ void orbit_two(float2 z0, float2 z1, float zz, float4 r, float e, int o, int S,
                                          float &dA, float &dB, int &ix) {
    float P = z0.x * r.x + z0.y * r.y, Q = z0.y * r.x - z0.x * r.y;
    if (DIMS == 4) {
        P += z1.x * r.z + z1.y * r.w;
        Q += z1.y * r.z - z1.x * r.w;
    }
    float v1, v2;
    int k1;
    if (S == 4) {
        const float aP = fabsf(P), aQ = fabsf(Q);
        v1 = fmaxf(aP, aQ);
        v2 = fminf(aP, aQ);
        k1 = aP >= aQ ? (P >= 0.f ? 0 : 2) : (Q >= 0.f ? 1 : 3);
    } else if (S == 2) {
        v1 = fabsf(P);
        v2 = -v1;
        k1 = P >= 0.f ? 0 : 1;
    } else {
        v1 = P;
        v2 = -__int_as_float(0x7f800000);
        k1 = 0;
    }
    const float base = zz + e;
    dA = fmaf(-2.f, v1, base);
    dB = fmaf(-2.f, v2, base);
    ix = o * S + k1;
}

// The two smallest of N sorted pairs (a_i <= b_i) by a merge tree (the
// second smallest of two pairs is min(max(a_1, a_2), min(b_1, b_2))), so the
// compare latency grows with log N; ix follows the smaller a.
template <int N>
__device__ __forceinline__ void two_smallest_tree(float (&a)[N], float (&b)[N], int (&ix)[N]) {
#pragma unroll
    for (int w = 1; w < N; w *= 2)
#pragma unroll
        for (int o = 0; o + w < N; o += 2 * w) {
            const bool sw = a[o + w] < a[o];
            const float m2 = fminf(fmaxf(a[o], a[o + w]), fminf(b[o], b[o + w]));
            a[o] = fminf(a[o], a[o + w]);
            b[o] = m2;
            ix[o] = sw ? ix[o + w] : ix[o];
        }
}

// The two smallest squared distances from the de-rotated z to the table
// (each orbit's two best rotations hold the nearest point and the
// second-nearest) and o S + k of the nearest.  DIMS 4: the lanes of half h
// take orbits 2 o + h (o < 8, adjacent table entries: one shared-memory
// wavefront), then every second orbit past 16; DIMS 2 reads z0 alone and
// takes every orbit.  The table holds at least 16 entries (energy +inf
// past n_orb).
template <int DIMS>
__device__ __forceinline__ void two_nearest(float2 z0, float2 z1, const Tables &tb, const FmtDev &f, int h,
                                            float &d1, float &d2, int &best) {
    const float zz = DIMS == 4 ? cnorm(z0) + cnorm(z1) : cnorm(z0);
    const int S = f.S, n = f.n_orb;
    if (DIMS == 4) {
        float a[8], b[8];
        int ix[8];
#pragma unroll
        for (int o = 0; o < 8; ++o)
            orbit_two<4>(z0, z1, zz, tb.orb[2 * o + h], tb.orbe[2 * o + h], 2 * o + h, S, a[o], b[o], ix[o]);
        two_smallest_tree<8>(a, b, ix);
        d1 = a[0];
        d2 = b[0];
        best = ix[0];
        for (int oo = 16 + h; oo < n; oo += 2) {
            float dA, dB;
            int io;
            orbit_two<4>(z0, z1, zz, tb.orb[oo], tb.orbe[oo], oo, S, dA, dB, io);
            best = dA < d1 ? io : best;
            d2 = fminf(fmaxf(d1, dA), fminf(d2, dB));
            d1 = fminf(d1, dA);
        }
    } else if (n <= 4) {
        float a[4], b[4];
        int ix[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) orbit_two<2>(z0, z0, zz, tb.orb[o], tb.orbe[o], o, S, a[o], b[o], ix[o]);
        two_smallest_tree<4>(a, b, ix);
        d1 = a[0];
        d2 = b[0];
        best = ix[0];
    } else {
        float a[16], b[16];
        int ix[16];
#pragma unroll
        for (int o = 0; o < 16; ++o) orbit_two<2>(z0, z0, zz, tb.orb[o], tb.orbe[o], o, S, a[o], b[o], ix[o]);
        two_smallest_tree<16>(a, b, ix);
        d1 = a[0];
        d2 = b[0];
        best = ix[0];
        for (int o = 16; o < n; ++o) {
            float dA, dB;
            int io;
            orbit_two<2>(z0, z0, zz, tb.orb[o], tb.orbe[o], o, S, dA, dB, io);
            best = dA < d1 ? io : best;
            d2 = fminf(fmaxf(d1, dA), fminf(d2, dB));
            d1 = fminf(d1, dA);
        }
    }
}

__device__ __forceinline__ float sqrt_approx(float x) {   // x >= 0; relative error ~1e-7
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The decision's margin T = |z - s_2| - |z - s_1| from the second-smallest
// squared distance d2 and the nearest point s_1 = p (|z - s_1| from the
// coordinate differences, free of the cancellation in |z|^2 + |s|^2 - 2 Re);
// the hold radius' slack covers the approximate square roots
template <int DIMS>
__device__ __forceinline__ float margin_of(float2 z0, float2 z1, float4 p, float d2) {
    float a = cnorm(make_float2(z0.x - p.x, z0.y - p.y));
    if (DIMS == 4) a += cnorm(make_float2(z1.x - p.z, z1.y - p.w));
    return sqrt_approx(fmaxf(d2, 0.f)) - sqrt_approx(a);
}

// Largest squared correction |y - z|^2 under which the decision taken on z
// holds for y: with margin T, every other point stays at least T - 2|y - z|
// farther from y than the nearest (triangle inequality); the slack keeps
// that gap far above the float32 rounding of the squared distances, so the
// warp-wide decision on y would pick the same point.  Negative: never.
__device__ __forceinline__ float hold_radius2(float T, float zz) {
    const float m = T - 1e-4f * (1.f + zz);
    return m > 0.f ? 0.25f * m * m : -1.f;
}

// Sequential CMA (MODE 0), DD-LMS (MODE 1) or data-aided LMS (MODE 3).
//
// With X_k the stacked input window of symbol k, h_k the taps after update
// k and r(j, k) = X_j^H X_k, the output of update k is
//   y_k = h_{k-1}^H X_k = H^H X_k + sum_{j = j0}^{k-1} mu e_j r(j, k)
// for any earlier taps H = h_{j0-1}.  Updates run in sub-blocks of kSB = 16;
// for update k of sub-block s the library takes H = the taps before
// sub-block s - 1, so the sum has at most 2 kSB - 1 terms and everything but
// the scalar corrections is computed a sub-block ahead by helper warps:
// * decision warp: lane l holds the partial y of update 16 s + l (l < 16:
//   this sub-block, l >= 16: the next); per update it takes the decision on
//   y_k, every lane adds mu e_k r(k, 16 s + l) to its own partial (one
//   complex FMA per output), and y_{k+1} is lane k+1's partial, fetched by a
//   shuffle while the decision ran, plus mu e_k r(k, k + 1).  DD decisions
//   are taken ahead: at the start of a sub-block lanes l and l + 16 decide
//   update 16 s + l on its partial p_l (which lacks only the terms of the
//   sub-block's earlier updates) and keep the margin T_l between the
//   nearest and the second-nearest point.  Update k then takes that point
//   when 2 |y_k - p_k| < T_k - slack (no other point can be nearer to y_k,
//   and the slack keeps the float32 warp-wide search on y_k from ruling
//   otherwise); else, for a few per cent of the updates, the warp-wide
//   search on y_k.  The decisions, and the errors (one fixed rounding on
//   both paths), are those of the warp-wide search on every update.
// * tap group: applies the previous sub-block's 16 updates to the taps,
//   h += sum_j mu conj(e_j) X_j, then forms H^H X_k for the next sub-block;
// * correlation group: r(j, j + d) for the next sub-block's rows j and lags
//   d < 32, by a window sliding along j (two products in, two out per row).
// One __syncthreads per sub-block hands the products over.
template <int T, int DIMS, int MODE>
__global__ void __launch_bounds__(kThreads, 1)
lms_kernel(const void *__restrict__ x, long ns, const float2 *__restrict__ taps_in,
           float2 *__restrict__ taps_out, long k0, int n_upd, const uint16_t *__restrict__ pcode,
           long pcode_stride, int passes, float mu, const reflab_t *__restrict__ ref_lab,
           long ref_stride, int sk, int opts, const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    const int wl = opts & LMS_WL;
    const bool ahead = (opts & LMS_EXACT_DD) == 0;   // DD decisions taken a sub-block ahead
    constexpr int NSX = lms_nsx(T);
    const int L = wl ? 2 * T : T;                     // taps per branch (widely linear: [h on x, g on conj x])
    __shared__ Tables tb;
    // the decision warp's decisions taken ahead on the partial outputs: per
    // update of the sub-block the partial (y_0, y_1), the chosen points
    // turned by exp(j phi_k), and the squared hold radii (DIMS 2: per output)
    __shared__ float4 sp_base[kSB], sp_dr[kSB];
    __shared__ float2 sp_hold[kSB];
    extern __shared__ float2 dyn_sm[];
    // local sample index of x_p[2 (kb + k) + D - t] is 2 k + 2 D - t
    float2 *xs0 = dyn_sm, *xs1 = dyn_sm + NSX;
    float2 *Hs = dyn_sm + lms_off_h(T);               // taps [q][p][t], t < L
    float2 *Rt = dyn_sm + lms_off_r(T);               // [2][kSB][kLag]: mu r(j, j + d)
    float2 *Rp = dyn_sm + lms_off_rp(T);              // [kSB][kLag][4]: per (p, parity) partial sums
    float2 *bsb = dyn_sm + lms_off_b(T);              // [2][kSB][q]: H^H X_k
    float4 *es = reinterpret_cast<float4 *>(dyn_sm + lms_off_e(T));   // [2][kSB]: e_k
    float2 *rots = dyn_sm + lms_off_rot(T);           // exp(j phi_k) (MODE 1, 3)
    float2 *tg0 = rots + kCH, *tg1 = rots + 2 * kCH;  // d_q exp(j phi_k) (MODE 3)
    uint16_t *pc = reinterpret_cast<uint16_t *>(dyn_sm + lms_off_pc(T));
    reflab_t *rl = reinterpret_cast<reflab_t *>(pc + kCH);
    const int s_id = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int hw = (warp & 3) ? warp - 1 - (warp >> 2) : -1;   // helper index 0 .. 8
    const bool tap_grp = hw >= 0 && hw < 4, cor_grp = hw >= 4 && hw < 8;
    const int gt = (hw & 3) * 32 + lane;                       // index within a group
    auto xsp = [&](int pp) { return pp ? xs1 : xs0; };
    load_tables(tb, f);
    for (int i = threadIdx.x; i < 4 * L; i += blockDim.x) Hs[i] = taps_in[(long)s_id * 4 * L + i];
    const long xoff = (long)s_id * 2 * ns;
    const int qt_step = 4 / f.S;

    // tap group: h += mu sum_{i < m} conj(e_{jb + i}) X_{jb + i}; thread
    // (q, p, t) owns one tap (two when widely linear: the taps on conj(x)
    // take the conjugate samples)
    auto tap_update = [&](int jb, int m, const float4 *E) {
        for (int te = gt; te < 4 * L; te += 128) {
            const int q = te / (2 * L), rem = te - q * 2 * L, pp = rem / L, tt = rem - pp * L;
            const bool cj = tt >= T;
            const int t = cj ? tt - T : tt;
            const float2 *xp = xsp(pp) + 2 * jb + 2 * D - t;
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
            auto xv = [&](int i) { const float2 v = xp[2 * i]; return cj ? make_float2(v.x, -v.y) : v; };
            if (m == kSB) {
#pragma unroll
                for (int i = 0; i < kSB; i += 2) {
                    const float4 e = E[i], f1 = E[i + 1];
                    a0 = cadd(a0, cmulc(q ? make_float2(e.z, e.w) : make_float2(e.x, e.y), xv(i)));
                    a1 = cadd(a1, cmulc(q ? make_float2(f1.z, f1.w) : make_float2(f1.x, f1.y), xv(i + 1)));
                }
            } else {
                for (int i = 0; i < m; ++i) {
                    const float4 e = E[i];
                    a0 = cadd(a0, cmulc(q ? make_float2(e.z, e.w) : make_float2(e.x, e.y), xv(i)));
                }
            }
            const float2 a = cadd(a0, a1);
            Hs[te] = cadd(Hs[te], make_float2(mu * a.x, mu * a.y));
        }
    };
    // tap group: H^H X_k for the kSB updates from kb0 into bsb row set `buf`;
    // thread (kk, q, p, half) sums half of one polarisation's taps
    auto bases = [&](int kb0, int buf) {
        const int kk = gt >> 3, q = (gt >> 2) & 1, pp = (gt >> 1) & 1, half = gt & 1;
        const int k = kb0 + kk;
        const float2 *xp = xsp(pp);
        const float2 *hq = Hs + (q * 2 + pp) * L;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        if (wl) {
            // half 0: taps on x, half 1: taps on conj(x)
            const float2 *hh = hq + half * T;
#pragma unroll
            for (int t = 0; t < T; ++t) {
                const float2 v = xp[2 * k + 2 * D - t];
                const float2 xv = half ? make_float2(v.x, -v.y) : v;
                if (t & 1) a1 = cadd(a1, cmulc(hh[t], xv));
                else a0 = cadd(a0, cmulc(hh[t], xv));
            }
        } else {
#pragma unroll
            for (int tt = 0; tt < 16; tt += 2) {
                const int t = 16 * half + tt;
                if (t < T) a0 = cadd(a0, cmulc(hq[t], xp[2 * k + 2 * D - t]));
                if (t + 1 < T) a1 = cadd(a1, cmulc(hq[t + 1], xp[2 * k + 2 * D - t - 1]));
            }
        }
        float2 acc = cadd(a0, a1);
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
        if ((gt & 3) == 0) bsb[(buf * kSB + kk) * 2 + q] = acc;
    };
    // correlation group: r(j, j + d) = sum_{u = 2j}^{2j + 2D} c[u] with
    // c[u] = sum_p conj(x_p[u]) x_p[u + 2d] (local sample index u).  Thread
    // (d, p, parity) slides its share of the window one row per step (one
    // product in, one out) and keeps its products of the last 32 samples in a
    // register ring (slot (u >> 1) mod 16, so a sub-block of 16 rows turns it
    // exactly once); the four partial sums per (row, lag) go through shared
    // memory and are added, times mu, after a group barrier
    // warps 6, 7 take the even samples, 9, 10 the odd ones (a warp-uniform
    // parity keeps the ring indices static); lane pairs are the two
    // polarisations of one lag
    const int ce = (hw >> 1) & 1, cd = ((hw & 1) * 32 + lane) >> 1, cp = lane & 1;
    float2 ring[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) ring[i] = make_float2(0.f, 0.f);
    float2 Rc = make_float2(0.f, 0.f);
    auto corr_sum = [&](int buf) {
        bar_sync(kBarCor, 128);
#pragma unroll
        for (int r4 = 0; r4 < kSB * kLag / 128; ++r4) {
            const int idx = r4 * 128 + gt;             // (row, lag)
            const float4 *pp4 = reinterpret_cast<const float4 *>(Rp + idx * 4);
            const float4 a = pp4[0], b = pp4[1];
            const float2 sum = make_float2((a.x + a.z) + (b.x + b.z), (a.y + a.w) + (b.y + b.w));
            // widely linear: the augmented windows correlate to r + conj(r)
            const float2 v = wl ? make_float2(2.f * mu * sum.x, 0.f) : make_float2(mu * sum.x, mu * sum.y);
            Rt[buf * kSB * kLag + idx] = (idx & (kLag - 1)) ? v : make_float2(0.f, 0.f);
        }
    };
    // one step of the even (E = 0) or odd (E = 1) share: row j from row j - 1
    auto corr_step = [&](auto E, int j, int jj, const float2 *xp) {
        constexpr int e = decltype(E)::value;
        const int uin = e ? 2 * j + 2 * D - 1 : 2 * j + 2 * D;
        const int s_out = (jj - 1) & 15;
        const int s_in = e ? (jj + D - 1) & 15 : (jj + D) & 15;
        const float2 old = ring[s_out];
        ring[s_in] = cmulc(xp[uin], xp[uin + 2 * cd]);
        Rc = cadd(Rc, csub(ring[s_in], old));
    };
    auto corr_first_e = [&](auto E, int buf) {   // rows 0 .. kSB - 1 of the chunk
        constexpr int e = decltype(E)::value;
        const float2 *xp = xsp(cp);
#pragma unroll
        for (int i = 0; i < 16; ++i) ring[i] = make_float2(0.f, 0.f);
        Rc = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = e; u <= 2 * D; u += 2) {
            ring[(u >> 1) & 15] = cmulc(xp[u], xp[u + 2 * cd]);
            Rc = cadd(Rc, ring[(u >> 1) & 15]);
        }
#pragma unroll
        for (int jj = 0; jj < kSB; ++jj) {
            if (jj > 0) corr_step(E, jj, jj, xp);
            Rp[(jj * kLag + cd) * 4 + cp * 2 + e] = Rc;
        }
    };
    auto corr_first = [&](int buf) {
        if (ce) corr_first_e(std::integral_constant<int, 1>(), buf);
        else corr_first_e(std::integral_constant<int, 0>(), buf);
        corr_sum(buf);
    };
    auto corr_next_e = [&](auto E, int jr0) {     // rows jr0 .. jr0 + kSB - 1, jr0 = 16 s'
        constexpr int e = decltype(E)::value;
        const float2 *xp = xsp(cp);
        // jr0 is a multiple of 16: the ring slots depend on jj only
#pragma unroll
        for (int jj = 0; jj < kSB; ++jj) {
            corr_step(E, jr0 + jj, jj, xp);
            Rp[(jj * kLag + cd) * 4 + cp * 2 + e] = Rc;
        }
    };
    auto corr_next = [&](int jr0, int buf) {
        if (ce) corr_next_e(std::integral_constant<int, 1>(), jr0);
        else corr_next_e(std::integral_constant<int, 0>(), jr0);
        corr_sum(buf);
    };

    for (int pass = 0; pass < passes; ++pass) {
        for (int c0 = 0; c0 < n_upd; c0 += kCH) {
            const int n = min(kCH, n_upd - c0);
            const long kb = k0 + c0;
            const int nsb = (n + kSB - 1) / kSB;
            const int nsx = 2 * n + 2 * D + 2 * (kSB + kLag) + 4;
            __syncthreads();
            for (int i = threadIdx.x; i < 2 * nsx; i += blockDim.x) {
                const int pp = i / nsx, jj = i - pp * nsx;
                const long g = 2 * kb - D + jj;
                xsp(pp)[jj] = (g >= 0 && g < ns) ? ld_sample(x, xoff + (long)pp * ns + g, sk) : make_float2(0.f, 0.f);
            }
            if (MODE != 0)
                for (int i = threadIdx.x; i < n; i += blockDim.x) pc[i] = pcode[(long)s_id * pcode_stride + kb + i];
            if (MODE == 3)
                for (int i = threadIdx.x; i < n; i += blockDim.x) rl[i] = ref_lab[(long)s_id * ref_stride + kb + i];
            __syncthreads();
            if (MODE != 0)
                for (int kk = threadIdx.x; kk < n; kk += blockDim.x) {
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
            if (tap_grp) bases(0, 0);
            if (cor_grp) corr_first(0);
            __syncthreads();

            // decision warp state: partial y of update 16 s + lane, both outputs
            float2 v0 = make_float2(0.f, 0.f), v1 = make_float2(0.f, 0.f);
            // lane o holds orbit o: 16 orbits twice over (4D and up to 16 2D
            // orbits), or 32 for 2D tables of more than 16 orbits
            const int o = (DIMS == 2 && f.n_orb > 16) ? lane : (lane & 15);
            const bool valid = o < f.n_orb;
            const float4 r = tb.orb[valid ? o : 0];
            const float eo = valid ? tb.orbe[o] : __int_as_float(0x7f800000);   // +inf: never the minimum
            int lab[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) lab[k] = tb.orblab[valid ? o : 0][k] & 255;
            for (int s = 0; s < nsb; ++s) {
                const int buf = s & 1;
                if (warp == 0) {
                    // lanes < 16 take this sub-block's bases plus what the
                    // previous sub-block left in lanes >= 16
                    float2 c0, c1;
                    c0.x = __shfl_down_sync(0xffffffffu, v0.x, 16);
                    c0.y = __shfl_down_sync(0xffffffffu, v0.y, 16);
                    c1.x = __shfl_down_sync(0xffffffffu, v1.x, 16);
                    c1.y = __shfl_down_sync(0xffffffffu, v1.y, 16);
                    // p: the partial of update 16 s + (lane & 15), in both
                    // lanes of the pair (lane u + 16 adds the same two values)
                    float2 p0, p1;
                    {
                        const float2 b0 = bsb[(buf * kSB + (lane & 15)) * 2];
                        const float2 b1 = bsb[(buf * kSB + (lane & 15)) * 2 + 1];
                        if (lane < kSB) {
                            v0 = cadd(c0, b0);
                            v1 = cadd(c1, b1);
                            p0 = v0;
                            p1 = v1;
                        } else {
                            p0 = cadd(v0, b0);
                            p1 = cadd(v1, b1);
                            v0 = v1 = make_float2(0.f, 0.f);
                        }
                    }
                    const float2 *Rr = Rt + buf * kSB * kLag;
                    const int ms = min(kSB, n - kSB * s);
                    if (MODE == 1 && ahead) {
                        // decisions taken ahead: update 16 s + u (u < 16) on its
                        // partial, which lacks only the terms of updates
                        // 16 s .. 16 s + u - 1; lanes u and u + 16 share it (4D
                        // tables: even / odd orbits, merged; 2D: polarisation h)
                        const int u = lane & 15, h = lane >> 4;
                        const float2 rot = rots[kSB * s + min(u, ms - 1)];
                        const float2 rm = make_float2(rot.x, -rot.y);
                        const float2 z0 = cmul(p0, rm), z1 = cmul(p1, rm);
                        float d1, d2;
                        int best;
                        if (DIMS == 4) {
                            two_nearest<4>(z0, z1, tb, f, h, d1, d2, best);
                            const float od1 = __shfl_xor_sync(0xffffffffu, d1, 16);
                            const float od2 = __shfl_xor_sync(0xffffffffu, d2, 16);
                            const int ob = __shfl_xor_sync(0xffffffffu, best, 16);
                            d2 = fminf(fmaxf(d1, od1), fminf(d2, od2));
                            best = od1 < d1 ? ob : best;   // exact ties: margin 0, never held
                            d1 = fminf(d1, od1);
                        } else {
                            two_nearest<2>(h ? z1 : z0, z1, tb, f, h, d1, d2, best);
                        }
                        const float4 pt = tb.rpts[best];
                        if (u < ms) {
                            float2 *dr2 = reinterpret_cast<float2 *>(sp_dr);
                            float *hd = reinterpret_cast<float *>(sp_hold);
                            if (DIMS == 4) {
                                if (h == 0) {
                                    const float mg = margin_of<4>(z0, z1, pt, d2);
                                    dr2[2 * u] = cmul_fixed(make_float2(pt.x, pt.y), rot);
                                    dr2[2 * u + 1] = cmul_fixed(make_float2(pt.z, pt.w), rot);
                                    hd[2 * u] = hold_radius2(mg, cnorm(z0) + cnorm(z1));
                                    sp_base[u] = make_float4(p0.x, p0.y, p1.x, p1.y);
                                }
                            } else {
                                const float2 zh = h ? z1 : z0;
                                const float mg = margin_of<2>(zh, zh, pt, d2);
                                dr2[2 * u + h] = cmul_fixed(make_float2(pt.x, pt.y), rot);
                                hd[2 * u + h] = hold_radius2(mg, cnorm(zh));
                                if (h == 0) sp_base[u] = make_float4(p0.x, p0.y, p1.x, p1.y);
                            }
                        }
                        __syncwarp();
                    }
                    float2 y0, y1;
                    y0.x = __shfl_sync(0xffffffffu, v0.x, 0);
                    y0.y = __shfl_sync(0xffffffffu, v0.y, 0);
                    y1.x = __shfl_sync(0xffffffffu, v1.x, 0);
                    y1.y = __shfl_sync(0xffffffffu, v1.y, 0);
                    const float2 *Rl = Rr + lane;
                    // the shared operands of update i are read one update ahead
                    // (program order puts those reads before the update's store,
                    // so their latency overlaps the update)
                    float2 rc_n = Rl[0], r1_n = Rr[1];
                    float4 sb_n, dr_n;
                    float2 hr_n;
                    if (MODE == 1) {
                        sb_n = sp_base[0];
                        dr_n = sp_dr[0];
                        hr_n = sp_hold[0];
                    }
#pragma unroll 2
                    for (int i = 0; i < ms; ++i) {
                        const int k = kSB * s + i;
                        // mu r(k, 16 s + lane) (lanes <= i read values they never use)
                        const float2 rc = rc_n;
                        const float2 r1 = r1_n;                                         // mu r(k, k + 1)
                        const float4 sb = sb_n, dr = dr_n;
                        const float2 hr = hr_n;
                        {
                            const int in = min(i + 1, kSB - 1);
                            rc_n = Rl[in * (kLag - 1)];
                            r1_n = Rr[in * kLag + 1];
                            if (MODE == 1) {
                                sb_n = sp_base[in];
                                dr_n = sp_dr[in];
                                hr_n = sp_hold[in];
                            }
                        }
                        // the next update's partial before this update's term:
                        // fetched while the decision runs
                        float2 w0, w1;
                        w0.x = __shfl_sync(0xffffffffu, v0.x, i + 1);
                        w0.y = __shfl_sync(0xffffffffu, v0.y, i + 1);
                        w1.x = __shfl_sync(0xffffffffu, v1.x, i + 1);
                        w1.y = __shfl_sync(0xffffffffu, v1.y, i + 1);
                        float2 e0, e1;
                        if (MODE == 0) {
                            const float g0 = f.R2 - cnorm(y0), g1 = f.R2 - cnorm(y1);
                            e0 = make_float2(g0 * y0.x, g0 * y0.y);
                            e1 = make_float2(g1 * y1.x, g1 * y1.y);
                        } else if (MODE == 3) {
                            e0 = csub(tg0[k], y0);
                            e1 = csub(tg1[k], y1);
                        } else {
                            // the decision taken ahead holds while the terms added
                            // since stay inside its hold radius (the same for every
                            // lane: y and the shared values are warp-uniform)
                            bool hold;
                            if (DIMS == 4)
                                hold = cnorm(make_float2(y0.x - sb.x, y0.y - sb.y)) +
                                       cnorm(make_float2(y1.x - sb.z, y1.y - sb.w)) < hr.x;
                            else
                                hold = cnorm(make_float2(y0.x - sb.x, y0.y - sb.y)) < hr.x &&
                                       cnorm(make_float2(y1.x - sb.z, y1.y - sb.w)) < hr.y;
                            e0 = sub_rn(make_float2(dr.x, dr.y), y0);
                            e1 = sub_rn(make_float2(dr.z, dr.w), y1);
                            if (!__all_sync(0xffffffffu, hold && ahead)) {
                                const float2 rot = rots[k];                               // exp(j phi)
                                // this lane's representative turned by phi: the
                                // correlation with y equals that of y exp(-j phi)
                                // with the representative, and |y| = |y exp(-j phi)|
                                const float2 q0 = cmul(make_float2(r.x, r.y), rot);
                                float2 d0, d1;
                                if (DIMS == 4) {
                                    const float2 q1 = cmul(make_float2(r.z, r.w), rot);
                                    const float P = (y0.x * q0.x + y0.y * q0.y) + (y1.x * q1.x + y1.y * q1.y);
                                    const float Q = (y0.y * q0.x - y0.x * q0.y) + (y1.y * q1.x - y1.x * q1.y);
                                    float v;
                                    int lb;
                                    best_rot_label(P, Q, f.S, lab, v, lb);
                                    const float dist = (cnorm(y0) + cnorm(y1)) + (eo - 2.f * v);
                                    const float4 pt = tb.pts[argmin_label(dist, lb)];
                                    d0 = make_float2(pt.x, pt.y);
                                    d1 = make_float2(pt.z, pt.w);
                                } else {
                                    float va, vb;
                                    int la, lc;
                                    best_rot_label(y0.x * q0.x + y0.y * q0.y, y0.y * q0.x - y0.x * q0.y, f.S, lab, va, la);
                                    best_rot_label(y1.x * q0.x + y1.y * q0.y, y1.y * q0.x - y1.x * q0.y, f.S, lab, vb, lc);
                                    // one orbit (e.g. QPSK): every lane holds the same candidate
                                    // (lanes past the table use orbit 0 too), so it is the decision
                                    if (f.n_orb > 1) {
                                        la = argmin_label(cnorm(y0) + (eo - 2.f * va), la);
                                        lc = argmin_label(cnorm(y1) + (eo - 2.f * vb), lc);
                                    }
                                    const float4 p0 = tb.pts[la];
                                    const float4 p1 = tb.pts[lc];
                                    d0 = make_float2(p0.x, p0.y);
                                    d1 = make_float2(p1.x, p1.y);
                                }
                                e0 = sub_rn(cmul_fixed(d0, rot), y0);
                                e1 = sub_rn(cmul_fixed(d1, rot), y1);
                            }
                        }
                        v0 = cadd(v0, cmul(e0, rc));
                        v1 = cadd(v1, cmul(e1, rc));
                        // lane i + 1's new partial, formed the same way in every lane
                        y0 = cadd(w0, cmul(e0, r1));
                        y1 = cadd(w1, cmul(e1, r1));
                        es[buf * kSB + i] = make_float4(e0.x, e0.y, e1.x, e1.y);   // every lane: the same value
                    }
                } else if (tap_grp) {
                    if (s >= 1) tap_update(kSB * (s - 1), kSB, es + (buf ^ 1) * kSB);
                    bar_sync(kBarTap, 128);
                    if (s + 1 < nsb) bases(kSB * (s + 1), buf ^ 1);
                } else if (cor_grp) {
                    if (s + 1 < nsb) corr_next(kSB * (s + 1), buf ^ 1);
                }
                __syncthreads();
            }
            // the last sub-block's updates (the next chunk, the next pass or
            // the output read the taps after the next barrier)
            if (tap_grp) tap_update(kSB * (nsb - 1), n - kSB * (nsb - 1), es + ((nsb - 1) & 1) * kSB);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * L; i += blockDim.x) taps_out[(long)s_id * 4 * L + i] = Hs[i];
}

// ---------------------------------------------------------------------------
// block LMS
// ---------------------------------------------------------------------------

// Nearest table point of (z0, z1) by one thread: every orbit's best rotation
// (P + jQ = sum_p z_p conj(rep_p)), the minimum distance, lowest label on
// exact ties (the rule of the warp-wide search in lms_kernel).
template <int DIMS>
__device__ __forceinline__ void decide_serial(float2 z0, float2 z1, const Tables &tb, const FmtDev &f,
                                              float2 &d0, float2 &d1) {
    if (DIMS == 4) {
        const float zn = cnorm(z0) + cnorm(z1);
        float best = __int_as_float(0x7f800000);
        int bl = 0x7fffffff;
        for (int o = 0; o < f.n_orb; ++o) {
            const float4 r = tb.orb[o];
            const float P = (z0.x * r.x + z0.y * r.y) + (z1.x * r.z + z1.y * r.w);
            const float Q = (z0.y * r.x - z0.x * r.y) + (z1.y * r.z - z1.x * r.w);
            const int lab[4] = {tb.orblab[o][0] & 255, tb.orblab[o][1] & 255, tb.orblab[o][2] & 255,
                                tb.orblab[o][3] & 255};
            float v;
            int lb;
            best_rot_label(P, Q, f.S, lab, v, lb);
            const float dist = fmaxf(zn + (tb.orbe[o] - 2.f * v), 0.f);
            if (dist < best || (dist == best && lb < bl)) { best = dist; bl = lb; }
        }
        const float4 pt = tb.pts[bl];
        d0 = make_float2(pt.x, pt.y);
        d1 = make_float2(pt.z, pt.w);
    } else {
#pragma unroll
        for (int pol = 0; pol < 2; ++pol) {
            const float2 z = pol ? z1 : z0;
            float best = __int_as_float(0x7f800000);
            int bl = 0x7fffffff;
            for (int o = 0; o < f.n_orb; ++o) {
                const float4 r = tb.orb[o];
                const int lab[4] = {tb.orblab[o][0] & 255, tb.orblab[o][1] & 255, tb.orblab[o][2] & 255,
                                    tb.orblab[o][3] & 255};
                float v;
                int lb;
                best_rot_label(z.x * r.x + z.y * r.y, z.y * r.x - z.x * r.y, f.S, lab, v, lb);
                const float dist = fmaxf(cnorm(z) + (tb.orbe[o] - 2.f * v), 0.f);
                if (dist < best || (dist == best && lb < bl)) { best = dist; bl = lb; }
            }
            const float4 pt = tb.pts[bl];
            (pol ? d1 : d0) = make_float2(pt.x, pt.y);
        }
    }
}

// Block LMS (Clark, Mitra and Parker): the updates run in groups of P; all
// outputs and errors of a group use the taps at its start, then the group's
// gradient terms are applied together, h_q += mu sum_k conj(e_q[k]) X_k.
// Update u0 + i is CMA while below n_cma, DD after (per update, so groups may
// straddle the switch).  One block of 256 threads per stream; per group:
// outputs (thread (k, q, p, half of the taps), shuffles over the four), one
// thread per error, one thread per tap for the update, a barrier after each.
template <int T, int DIMS>
__global__ void __launch_bounds__(256)
lms_block_kernel(const void *__restrict__ x, long ns, const float2 *__restrict__ taps_in,
                 float2 *__restrict__ taps_out, long k0, int n_upd, const uint16_t *__restrict__ pcode,
                 long pcode_stride, long u0, long n_cma, float mu, int P, int sk, int wl,
                 const __grid_constant__ FmtDev f) {
    constexpr int D = (T - 1) / 2;
    constexpr int NSX = 2 * kCH + 2 * D + 2;
    const int L = wl ? 2 * T : T;         // taps per branch
    __shared__ Tables tb;
    __shared__ float2 xs[2][NSX];         // local index of x_p[2 (kb + k) + D - t]: 2 k + 2 D - t
    __shared__ float2 Hs[4 * 2 * T];
    __shared__ float2 ys[64][2];
    __shared__ float2 es[64][2];
    __shared__ uint16_t pc[kCH];
    const int s = blockIdx.x, tid = threadIdx.x;
    load_tables(tb, f);
    for (int i = tid; i < 4 * L; i += blockDim.x) Hs[i] = taps_in[(long)s * 4 * L + i];
    const long xoff = (long)s * 2 * ns;
    const int qt_step = 4 / f.S;
    for (int c0 = 0; c0 < n_upd; c0 += kCH) {
        const int n = min(kCH, n_upd - c0);
        const long kb = k0 + c0;
        const int nsx = 2 * n + 2 * D + 2;
        __syncthreads();
        for (int i = tid; i < 2 * nsx; i += blockDim.x) {
            const int pp = i / nsx, jj = i - pp * nsx;
            const long g = 2 * kb - D + jj;
            xs[pp][jj] = (g >= 0 && g < ns) ? ld_sample(x, xoff + (long)pp * ns + g, sk) : make_float2(0.f, 0.f);
        }
        if (pcode)
            for (int i = tid; i < n; i += blockDim.x) pc[i] = pcode[(long)s * pcode_stride + kb + i];
        __syncthreads();
        for (int g0 = 0; g0 < n; g0 += P) {
            const int m = min(P, n - g0);
            // outputs of the group with its starting taps
            for (int base = 0; base < m * 8; base += blockDim.x) {
                const int it = base + tid;
                const bool act = it < m * 8;
                const int kk = it >> 3, q = (it >> 2) & 1, pp = (it >> 1) & 1, half = it & 1;
                float2 acc = make_float2(0.f, 0.f);
                if (act) {
                    const float2 *hq = Hs + (q * 2 + pp) * L;
                    const float2 *xp = xs[pp] + 2 * (g0 + kk) + 2 * D;
                    if (wl) {                        // half 0: taps on x, half 1: on conj(x)
                        for (int t = 0; t < T; ++t) {
                            const float2 v = xp[-t];
                            acc = cadd(acc, cmulc(hq[half * T + t], half ? make_float2(v.x, -v.y) : v));
                        }
                    } else {
                        const int t1 = half ? T : (T < 16 ? T : 16);
                        for (int t = half ? 16 : 0; t < t1; ++t) acc = cadd(acc, cmulc(hq[t], xp[-t]));
                    }
                }
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
                acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 2);
                acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 2);
                if (act && (it & 3) == 0) ys[kk][q] = acc;
            }
            __syncthreads();
            if (tid < m) {
                const int k = g0 + tid;
                const float2 y0 = ys[tid][0], y1 = ys[tid][1];
                float2 e0, e1;
                if (u0 + c0 + k < n_cma) {
                    const float g0c = f.R2 - cnorm(y0), g1c = f.R2 - cnorm(y1);
                    e0 = make_float2(g0c * y0.x, g0c * y0.y);
                    e1 = make_float2(g1c * y1.x, g1c * y1.y);
                } else {
                    // exp(j phi_k) = cs_b j^qt
                    const unsigned code = pc[k];
                    const int b = min((int)(code & 255), f.B - 1);
                    const int qt = ((int)((code >> 8) & 3) * qt_step) & 3;
                    float2 rot = tb.cs[b];
                    if (qt & 2) rot = make_float2(-rot.x, -rot.y);
                    if (qt & 1) rot = make_float2(-rot.y, rot.x);
                    float2 d0, d1;
                    decide_serial<DIMS>(cmulc(rot, y0), cmulc(rot, y1), tb, f, d0, d1);
                    e0 = csub(cmul(d0, rot), y0);
                    e1 = csub(cmul(d1, rot), y1);
                }
                es[tid][0] = e0;
                es[tid][1] = e1;
            }
            __syncthreads();
            if (tid < 4 * L) {
                const int q = tid / (2 * L), rem = tid - q * 2 * L, pp = rem / L, tt = rem - pp * L;
                const bool cj = tt >= T;
                const float2 *xp = xs[pp] + 2 * g0 + 2 * D - (cj ? tt - T : tt);
                float2 acc = make_float2(0.f, 0.f);
                for (int i = 0; i < m; ++i) {
                    const float2 v = xp[2 * i];
                    acc = cadd(acc, cmulc(es[i][q], cj ? make_float2(v.x, -v.y) : v));
                }
                Hs[tid] = cadd(Hs[tid], make_float2(mu * acc.x, mu * acc.y));
            }
            __syncthreads();
        }
    }
    for (int i = tid; i < 4 * L; i += blockDim.x) taps_out[(long)s * 4 * L + i] = Hs[i];
}

// ---------------------------------------------------------------------------
// training alignment
// ---------------------------------------------------------------------------
// Correlation of the equalised training span (y [S][2][ystride], storage sk,
// the FIR's output with the start-up taps) with the known symbols:
// C[q][p] = sum_k y_q[k] conj(s_p[k]); keep or swap the outputs, then turn
// each by the phase of its matched correlation (taps [S][2][2][T] in place).
template <int DIMS>
__global__ void __launch_bounds__(256)
align_kernel(const void *__restrict__ y, long ystride, float2 *__restrict__ taps, int T,
             const reflab_t *__restrict__ ref_lab, long ref_stride, int n_train, int sk,
             const __grid_constant__ FmtDev f) {
    __shared__ double red[8][256];
    __shared__ float2 rot[2];
    __shared__ int src[2];
    __shared__ float2 hs[4 * 62];
    const int s = blockIdx.x, tid = threadIdx.x;
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // C[q][p] re, im
    for (int k = tid; k < n_train; k += 256) {
        const float2 y0 = ld_sample(y, ((long)s * 2 + 0) * ystride + k, sk);
        const float2 y1 = ld_sample(y, ((long)s * 2 + 1) * ystride + k, sk);
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
        const float2 yq[2] = {y0, y1};
        for (int qq = 0; qq < 2; ++qq)
            for (int pp = 0; pp < 2; ++pp) {
                const float2 c = cmulc(sp[pp], yq[qq]);   // y_q conj(s_p)
                acc[(qq * 2 + pp) * 2] += c.x;
                acc[(qq * 2 + pp) * 2 + 1] += c.y;
            }
    }
    for (int i = 0; i < 8; ++i) red[i][tid] = acc[i];
    for (int i = tid; i < 4 * T; i += 256) hs[i] = taps[(long)s * 4 * T + i];
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

// Data-aided phase codes over the training span [0, n) from the equalised
// span y (the FIR's output with the aligned taps):
//   R_k = sum_{i in [k - W/2, k + W/2) within the span} sum_p y_p[i] conj(s_p[i]),
//   n_k = floor(arg(R_k) / (2 pi / (S B)) + 1/2), code = b | (m mod S) << 8 with
//   b = n_k + B/2 - m B, m = floor((n_k + B/2) / B).
template <int DIMS>
__global__ void __launch_bounds__(256)
train_phase_kernel(const void *__restrict__ y, long ystride, const reflab_t *__restrict__ ref_lab,
                   long ref_stride, int n, int W, uint16_t *__restrict__ pcode, long pcode_stride,
                   int32_t *__restrict__ carry, int carry_stride, int sk, const __grid_constant__ FmtDev f) {
    extern __shared__ float2 rs[];      // [n] per-symbol correlations
    const int s = blockIdx.x, tid = threadIdx.x;
    for (int k = tid; k < n; k += 256) {
        const float2 y0 = ld_sample(y, ((long)s * 2 + 0) * ystride + k, sk);
        const float2 y1 = ld_sample(y, ((long)s * 2 + 1) * ystride + k, sk);
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
        rs[k] = cadd(cmulc(s0, y0), cmulc(s1, y1));   // sum_p y_p conj(s_p)
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

// labels of rows i0 .. i1 - 1 of bits [S][n][m] into lab [S][n]
__global__ void ref_labels_kernel(const uint8_t *__restrict__ bits, reflab_t *__restrict__ lab,
                                  long n, long i0, long i1, int m) {
    const long i = i0 + (long)blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (i >= i1) return;
    const uint8_t *b = bits + ((long)s * n + i) * m;
    int v = 0;
    for (int c = 0; c < m; ++c) v = (v << 1) | (b[c] & 1);
    lab[(long)s * n + i] = (reflab_t)v;
}

// The recursion is latency-bound: a block asks for (nearly) all of an SM's
// shared memory so that no other kernel's blocks share its SM and its warp
// issues whenever it is ready.
template <int T, int DIMS, int MODE>
cudaError_t lms_launch_one(const void *x, long ns, const float2 *ti, float2 *to, long k0, int n_upd,
                           const uint16_t *pcode, long pstride, int passes, float mu,
                           const reflab_t *ref, long rstride, int S, const FmtDev &f, cudaStream_t st, int sk, int opts) {
    auto kern = lms_kernel<T, DIMS, MODE>;
    // the opt-in size is looked up and set once per device (host queries per
    // launch cost more than the launch when a handle runs one stream)
    static std::atomic<int> dyn_of[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int dyn = dev < 64 ? dyn_of[dev].load(std::memory_order_relaxed) : 0;
    if (dyn == 0) {
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
        int optin = 0;
        if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
        dyn = optin - (int)fa.sharedSizeBytes;
        if (dyn < (int)(lms_smem_f2(T) * sizeof(float2))) return cudaErrorInvalidValue;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) != cudaSuccess) return e;
        if (dev < 64) dyn_of[dev].store(dyn, std::memory_order_relaxed);
    }
    kern<<<S, kThreads, dyn, st>>>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, sk, opts, f);
    return cudaGetLastError();
}

template <int T, int MODE>
cudaError_t lms_launch_mode(const void *x, long ns, const float2 *ti, float2 *to, long k0,
                            int n_upd, const uint16_t *pcode, long pstride, int passes, float mu,
                            const reflab_t *ref, long rstride, int S, const FmtDev &f,
                            cudaStream_t st, int sk, int opts) {
    if (f.dims == 4)
        return lms_launch_one<T, 4, MODE>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref,
                                          rstride, S, f, st, sk, opts);
    return lms_launch_one<T, 2, MODE>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref,
                                      rstride, S, f, st, sk, opts);
}

template <int T>
cudaError_t lms_dispatch_dims(const void *x, long ns, const float2 *ti, float2 *to, long k0,
                              int n_upd, const uint16_t *pcode, long pstride, int mode,
                              int passes, unsigned long long u0, int n_cma, float mu,
                              const reflab_t *ref, long rstride, int S, const FmtDev &f,
                              cudaStream_t st, int sk, int opts) {
    switch (mode) {
        case 0: return lms_launch_mode<T, 0>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, S, f, st, sk, opts);
        case 1: return lms_launch_mode<T, 1>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, S, f, st, sk, opts);
        case 3: return lms_launch_mode<T, 3>(x, ns, ti, to, k0, n_upd, pcode, pstride, passes, mu, ref, rstride, S, f, st, sk, opts);
        case 2: {
            // CMA while the update count is below n_cma, DD after (one pass)
            const long ncma = (u0 >= (unsigned long long)n_cma) ? 0 : std::min<long>(n_upd, (long)(n_cma - u0));
            cudaError_t e = cudaSuccess;
            const float2 *src = ti;
            if (ncma > 0) {
                e = lms_launch_mode<T, 0>(x, ns, src, to, k0, (int)ncma, pcode, pstride, 1, mu, ref, rstride, S, f, st, sk, opts);
                if (e != cudaSuccess) return e;
                src = to;
            }
            if (n_upd - ncma > 0)
                e = lms_launch_mode<T, 1>(x, ns, src, to, k0 + ncma, (int)(n_upd - ncma), pcode, pstride, 1, mu,
                                          ref, rstride, S, f, st, sk, opts);
            return e;
        }
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_lms(const void *x, long ns, const float2 *taps_in, float2 *taps_out, long k0,
                       int n_upd, const uint16_t *pcode, long pcode_stride, int mode, int passes,
                       unsigned long long u0, int n_cma, float mu, const reflab_t *ref_lab,
                       long ref_stride, int n_streams, int T, const FmtDev &f, cudaStream_t st, int sk, int opts) {
    if (n_upd <= 0 || n_streams <= 0) {
        if (taps_in != taps_out)
            return cudaMemcpyAsync(taps_out, taps_in, sizeof(float2) * 4 * ((opts & LMS_WL) ? 2 * T : T) * (size_t)n_streams,
                                   cudaMemcpyDeviceToDevice, st);
        return cudaSuccess;
    }
    switch (T) {
        case 7: return lms_dispatch_dims<7>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st, sk, opts);
        case 15: return lms_dispatch_dims<15>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st, sk, opts);
        case 31: return lms_dispatch_dims<31>(x, ns, taps_in, taps_out, k0, n_upd, pcode, pcode_stride, mode, passes, u0, n_cma, mu, ref_lab, ref_stride, n_streams, f, st, sk, opts);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lms_block(const void *x, long ns, const float2 *taps_in, float2 *taps_out, long k0,
                             int n_upd, const uint16_t *pcode, long pcode_stride, int mode,
                             unsigned long long u0, int n_cma, float mu, int P, int n_streams, int T,
                             const FmtDev &f, cudaStream_t st, int sk, int wl) {
    if (P < 1 || P > 64) return cudaErrorInvalidValue;
    if (n_upd <= 0 || n_streams <= 0) {
        if (taps_in != taps_out)
            return cudaMemcpyAsync(taps_out, taps_in, sizeof(float2) * 4 * (wl ? 2 * T : T) * (size_t)n_streams,
                                   cudaMemcpyDeviceToDevice, st);
        return cudaSuccess;
    }
    // mode 0: CMA throughout, 1: DD throughout, 2: CMA below n_cma updates
    const long ncma = mode == 0 ? (long)(u0 + n_upd) : (mode == 1 ? 0 : (long)n_cma);
    if (mode != 0 && !pcode) return cudaErrorInvalidValue;
#define RX_LB(TT, DD)                                                                                      \
    lms_block_kernel<TT, DD><<<n_streams, 256, 0, st>>>(x, ns, taps_in, taps_out, k0, n_upd, pcode,          \
                                                       pcode_stride, (long)u0, ncma, mu, P, sk, wl, f)
    const bool d4 = f.dims == 4;
    switch (T) {
        case 7: if (d4) RX_LB(7, 4); else RX_LB(7, 2); break;
        case 15: if (d4) RX_LB(15, 4); else RX_LB(15, 2); break;
        case 31: if (d4) RX_LB(31, 4); else RX_LB(31, 2); break;
        default: return cudaErrorInvalidValue;
    }
#undef RX_LB
    return cudaGetLastError();
}

cudaError_t launch_align(const void *y, long ystride, float2 *taps, const reflab_t *ref_lab,
                         long ref_stride, int n_train, int n_streams, int T, const FmtDev &f,
                         cudaStream_t st, int sk) {
    if (n_train <= 0 || n_streams <= 0) return cudaSuccess;
    if (T < 1 || T > 62) return cudaErrorInvalidValue;      // taps per branch (2 x 31 widely linear)
    if (f.dims == 4)
        align_kernel<4><<<n_streams, 256, 0, st>>>(y, ystride, taps, T, ref_lab, ref_stride, n_train, sk, f);
    else
        align_kernel<2><<<n_streams, 256, 0, st>>>(y, ystride, taps, T, ref_lab, ref_stride, n_train, sk, f);
    return cudaGetLastError();
}

cudaError_t launch_train_phase(const void *y, long ystride, const reflab_t *ref_lab, long ref_stride, int n,
                               int W, uint16_t *pcode, long pcode_stride, int32_t *carry, int carry_stride,
                               int n_streams, const FmtDev &f, cudaStream_t st, int sk) {
    if (n <= 0 || n_streams <= 0) return cudaSuccess;
    const size_t smem = sizeof(float2) * (size_t)n;
    if (smem > 160 * 1024) return cudaErrorInvalidValue;
    if (f.dims == 4) {
        cudaError_t e = cudaFuncSetAttribute(train_phase_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        train_phase_kernel<4><<<n_streams, 256, smem, st>>>(y, ystride, ref_lab, ref_stride, n, W, pcode,
                                                             pcode_stride, carry, carry_stride, sk, f);
    } else {
        cudaError_t e = cudaFuncSetAttribute(train_phase_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        train_phase_kernel<2><<<n_streams, 256, smem, st>>>(y, ystride, ref_lab, ref_stride, n, W, pcode,
                                                             pcode_stride, carry, carry_stride, sk, f);
    }
    return cudaGetLastError();
}

cudaError_t launch_ref_labels(const uint8_t *bits, reflab_t *lab, long n_sym, int n_streams, int m,
                              int dims, int m_pol, cudaStream_t st) {
    (void)dims;
    (void)m_pol;
    return launch_ref_labels_rows(bits, lab, n_sym, 0, n_sym, n_streams, m, st);
}

cudaError_t launch_ref_labels_rows(const uint8_t *bits, reflab_t *lab, long n_sym, long i0, long i1,
                                   int n_streams, int m, cudaStream_t st) {
    if (i1 <= i0 || n_streams <= 0) return cudaSuccess;
    dim3 grid((unsigned)((i1 - i0 + 255) / 256), (unsigned)n_streams);
    ref_labels_kernel<<<grid, 256, 0, st>>>(bits, lab, n_sym, i0, i1, m);
    return cudaGetLastError();
}
