// A2: 2x2 butterfly FIR, T/2-spaced input, one output per symbol:
//   y_q[k] = sum_{p in X,Y} sum_{t<T} conj(h_qp[t]) x_p[2k + D - t],  D = (T-1)/2.
//
// A tile is 512 consecutive outputs of one stream; blocks of 128 threads
// loop over tiles (persistent grid, a few blocks per SM) and stage the next
// tile's 1024 + 2D input samples per polarisation with cp.async while they
// filter the current one (double buffer; one pad slot every 8 samples, so
// that threads 8 samples apart hit different banks).  Each thread makes 4
// consecutive outputs for both q: per tap it needs one new sample per
// even/odd tap chain (the other three slide through registers).  The
// complex multiply-accumulate conj(h) x is two packed f32x2 FMAs:
//   acc += (a, a) * (xr, xi) + (-b, b) * (xi, xr),   conj(h) = a + jb.
// Widely linear (taps h on x and g on conj(x), 2T per branch, [h, g]):
//   conj(g) conj(x) = (c, -c) * (xr, xi) + (-d, -d) * (xi, xr),  g = c + jd,
// two more packed FMAs on the same sample registers.
#include "rx_internal.h"

namespace {

constexpr int kOut = 512;
constexpr int kThreads = 128;

__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(BYTES),
                 "r"(valid ? BYTES : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N)); }

template <int T, int SK, bool WL>
struct FirSmem {
    using X = typename Store<SK>::T;
    static constexpr int D = (T - 1) / 2;
    static constexpr int L = WL ? 2 * T : T;     // taps per branch
    static constexpr int NS = 2 * kOut + 2 * D;
    static constexpr int NSP = NS + NS / 8 + 1;
    X xs[2][2][NSP];         // [buffer][p], the storage type of x
    float2 hraw[2][4 * L];   // [buffer] taps h[q][p][t] of the tile's stream
    f32x2 hA[2][2][T];       // [q][p][t] (a, a)
    f32x2 hB[2][2][T];       // [q][p][t] (-b, b), conj(h) = a + jb
    f32x2 gA[2][2][WL ? T : 1];   // (c, -c), g = c + jd (widely linear)
    f32x2 gB[2][2][WL ? T : 1];   // (-d, -d)
};

// stage tile `tile` (stream s = tile / tps) into buffer `buf`
template <int T, int SK, bool WL>
__device__ __forceinline__ void fir_stage(FirSmem<T, SK, WL> &sm, int buf, int tile, int tps,
                                          const typename Store<SK>::T *x, long ns, const float2 *taps, long k0) {
    constexpr int D = FirSmem<T, SK, WL>::D, NS = FirSmem<T, SK, WL>::NS, L = FirSmem<T, SK, WL>::L;
    constexpr int XB = sizeof(typename Store<SK>::T);
    const int s = tile / tps, tl = tile - s * tps;
    const long base = 2 * (k0 + (long)tl * kOut) - D;   // global sample of local index 0
    const typename Store<SK>::T *xs0 = x + (long)s * 2 * ns;
    for (int i = threadIdx.x; i < 2 * NS; i += kThreads) {
        const int p = i / NS, j = i - p * NS;
        const long g = base + j;
        const bool ok = g >= 0 && g < ns;
        cp_async<XB>(&sm.xs[buf][p][pad8(j)], xs0 + (long)p * ns + (ok ? g : 0), ok);
    }
    for (int i = threadIdx.x; i < 4 * L; i += kThreads)
        cp_async<8>(&sm.hraw[buf][i], taps + (long)s * 4 * L + i, true);
    cp_async_commit();
}

template <int T, int SK, bool WL>
__global__ void __launch_bounds__(kThreads)
fir_kernel(const typename Store<SK>::T *__restrict__ x, long ns, const float2 *__restrict__ taps, long k0,
           long k1, typename Store<SK>::T *__restrict__ y, long y_stride, long y_off, int tps, int n_tiles) {
    constexpr int D = (T - 1) / 2;
    constexpr int L = FirSmem<T, SK, WL>::L;
    __shared__ __align__(16) FirSmem<T, SK, WL> sm;
    const int tid = threadIdx.x;
    int tile = blockIdx.x, buf = 0;
    if (tile < n_tiles) fir_stage<T, SK, WL>(sm, 0, tile, tps, x, ns, taps, k0);
    for (; tile < n_tiles; tile += gridDim.x, buf ^= 1) {
        const int next = tile + gridDim.x;
        if (next < n_tiles) {
            fir_stage<T, SK, WL>(sm, buf ^ 1, next, tps, x, ns, taps, k0);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        for (int i = tid; i < 4 * L; i += kThreads) {
            const float2 h = sm.hraw[buf][i];
            const int q = i / (2 * L), p = (i / L) & 1, t = i % L;
            if (t < T) {
                sm.hA[q][p][t] = pk2(h.x, h.x);
                sm.hB[q][p][t] = pk2(h.y, -h.y);
            } else if (WL) {
                sm.gA[q][p][t - T] = pk2(h.x, -h.x);
                sm.gB[q][p][t - T] = pk2(-h.y, -h.y);
            }
        }
        __syncthreads();

        f32x2 acc[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[q][r] = pk2(0.f, 0.f);

        const int lb = 8 * tid + 2 * D;   // local index of (r = 0, t = 0)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const typename Store<SK>::T *xp = sm.xs[buf][p];
            // even / odd tap chains: E[r] = x[lb + 2r - 2j], O[r] = x[lb + 2r - 2j - 1],
            // each kept as (xr, xi) and swapped (xi, xr)
            f32x2 E[4], Es[4], O[4], Os[4];
            auto ld = [&](int i, f32x2 &v, f32x2 &vs) {
                const float2 a = Store<SK>::ld(xp, pad8(i));
                v = pk2(a.x, a.y);
                vs = pk2(a.y, a.x);
            };
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                ld(lb + 2 * r, E[r], Es[r]);
                ld(lb + 2 * r - 1, O[r], Os[r]);
            }
#pragma unroll
            for (int j = 0; j <= D; ++j) {
                {
                    const f32x2 a0 = sm.hA[0][p][2 * j], b0 = sm.hB[0][p][2 * j];
                    const f32x2 a1 = sm.hA[1][p][2 * j], b1 = sm.hB[1][p][2 * j];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[0][r] = fma2(b0, Es[r], fma2(a0, E[r], acc[0][r]));
                        acc[1][r] = fma2(b1, Es[r], fma2(a1, E[r], acc[1][r]));
                    }
                    if (WL) {
                        const f32x2 c0 = sm.gA[0][p][2 * j], d0 = sm.gB[0][p][2 * j];
                        const f32x2 c1 = sm.gA[1][p][2 * j], d1 = sm.gB[1][p][2 * j];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            acc[0][r] = fma2(d0, Es[r], fma2(c0, E[r], acc[0][r]));
                            acc[1][r] = fma2(d1, Es[r], fma2(c1, E[r], acc[1][r]));
                        }
                    }
                }
                if (j < D) {
                    const f32x2 a0 = sm.hA[0][p][2 * j + 1], b0 = sm.hB[0][p][2 * j + 1];
                    const f32x2 a1 = sm.hA[1][p][2 * j + 1], b1 = sm.hB[1][p][2 * j + 1];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        acc[0][r] = fma2(b0, Os[r], fma2(a0, O[r], acc[0][r]));
                        acc[1][r] = fma2(b1, Os[r], fma2(a1, O[r], acc[1][r]));
                    }
                    if (WL) {
                        const f32x2 c0 = sm.gA[0][p][2 * j + 1], d0 = sm.gB[0][p][2 * j + 1];
                        const f32x2 c1 = sm.gA[1][p][2 * j + 1], d1 = sm.gB[1][p][2 * j + 1];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            acc[0][r] = fma2(d0, Os[r], fma2(c0, O[r], acc[0][r]));
                            acc[1][r] = fma2(d1, Os[r], fma2(c1, O[r], acc[1][r]));
                        }
                    }
                    // slide the windows by one output (two samples)
#pragma unroll
                    for (int r = 3; r > 0; --r) {
                        E[r] = E[r - 1]; Es[r] = Es[r - 1];
                        O[r] = O[r - 1]; Os[r] = Os[r - 1];
                    }
                    ld(lb - 2 * (j + 1), E[0], Es[0]);
                    if (j + 1 < D) ld(lb - 2 * (j + 1) - 1, O[0], Os[0]);
                }
            }
        }
        const int s = tile / tps, tl = tile - s * tps;
        const long kt = k0 + (long)tl * kOut + 4 * tid;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            typename Store<SK>::T *yq = y + ((long)s * 2 + q) * y_stride + y_off;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                float re, im;
                upk2(acc[q][r], re, im);
                if (kt + r < k1) Store<SK>::st(yq, kt + r - k0, make_float2(re, im));
            }
        }
        __syncthreads();   // buffer `buf` is restaged two tiles later
    }
}




template <int SK, bool WL>
cudaError_t fir_t(const void *x, long ns, const float2 *taps, long k0, long k1, void *y, long y_stride,
                  long y_off, int T, int grid, long tps, long n_tiles, cudaStream_t st) {
    using X = typename Store<SK>::T;
    const X *xx = static_cast<const X *>(x);
    X *yy = static_cast<X *>(y);
    switch (T) {
        case 7: fir_kernel<7, SK, WL><<<grid, kThreads, 0, st>>>(xx, ns, taps, k0, k1, yy, y_stride, y_off, (int)tps, (int)n_tiles); break;
        case 15: fir_kernel<15, SK, WL><<<grid, kThreads, 0, st>>>(xx, ns, taps, k0, k1, yy, y_stride, y_off, (int)tps, (int)n_tiles); break;
        case 31: fir_kernel<31, SK, WL><<<grid, kThreads, 0, st>>>(xx, ns, taps, k0, k1, yy, y_stride, y_off, (int)tps, (int)n_tiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fir(const void *x, long ns, const float2 *taps, long k0, long k1, void *y,
                       long y_stride, long y_off, int n_streams, int T, cudaStream_t st, int sk, int sm_avail,
                       int wl) {
    if (k1 <= k0 || n_streams <= 0) return cudaSuccess;
    const long tps = (k1 - k0 + kOut - 1) / kOut;
    const long n_tiles = tps * n_streams;
    if (n_tiles > (1L << 30)) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long>(n_tiles, 4L * (sm_avail > 0 ? sm_avail : sm_count()));
    if (wl) {
        switch (sk) {
            case SK_F32: return fir_t<SK_F32, true>(x, ns, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
            case SK_F16: return fir_t<SK_F16, true>(x, ns, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
            case SK_BF16: return fir_t<SK_BF16, true>(x, ns, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sk) {
        case SK_F32: return fir_t<SK_F32, false>(x, ns, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
        case SK_F16: return fir_t<SK_F16, false>(x, ns, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
        case SK_BF16: return fir_t<SK_BF16, false>(x, ns, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}
