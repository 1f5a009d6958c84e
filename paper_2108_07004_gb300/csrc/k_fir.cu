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
//
// fir_tma_kernel (the default where the sample rows are 16-byte aligned
// whole 64-byte groups): the same sums, with each tile's input window of both
// polarisations staged by the tensor memory accelerator (one
// cp.async.bulk.tensor.3d box per row over x viewed as [2S][ns/R][R], R
// samples per 64-byte group; groups before sample 0 and past ns are filled
// with zeros by the copy itself) into a double buffer whose completion an
// mbarrier tracks (bounded waits).  The copy applies the 64-byte swizzle, so
// the threads (4 consecutive outputs each, 64 bytes apart) read the two
// samples of a tap pair (odd tap, even tap) as one 16-byte (8-byte for
// 16-bit storage) vector from distinct banks, one read per tap pair and
// polarisation, the chains sliding through registers as in fir_kernel.  The
// additions run in fir_kernel's order, so both kernels give the same bits.
#include <atomic>
#include <cstring>
#include <type_traits>

#include <cudaTypedefs.h>

#include "k_fir.h"
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

// ---------------------------------------------------------------------------
// TMA-staged form
// ---------------------------------------------------------------------------
// A row of x is viewed as 64-byte groups (8 float32 or 16 16-bit samples);
// the window of a tile is kG groups of one polarisation's row, copied as one
// 3D box with the 64-byte swizzle (16-byte chunk c of group g lands at chunk
// c ^ ((g >> 1) & 3)), so that the threads' 16-byte reads, 64 bytes apart,
// fall on distinct banks.
template <int SK> struct FirTmaGeom {
    static constexpr int XB = (int)sizeof(typename Store<SK>::T);
    static constexpr int R = 64 / XB;                 // samples per group
    // window: local indices up to 8*127 + 2D + delta + 6 < 1068 (D <= 15, delta < R)
    static constexpr int G = (1068 + R - 1) / R;      // groups per window: 134 / 67
    static constexpr int BYTES = 64 * G;              // one polarisation's box
    static constexpr int PITCH = (BYTES + 1023) / 1024 * 1024;   // swizzle-aligned slots
};

// set when a bounded wait gave up (read and cleared by fir_tma_status)
__device__ unsigned int g_fir_err;

template <int T, int SK, bool WL>
struct FirTmaSmem {
    static constexpr int L = WL ? 2 * T : T;
    unsigned char xs[2][2][FirTmaGeom<SK>::PITCH];   // [buffer][p] swizzled windows
    float2 hraw[2][4 * L];
    f32x2 hA[2][2][T], hB[2][2][T];
    f32x2 gA[2][2][WL ? T : 1], gB[2][2][WL ? T : 1];
    unsigned long long bar[2];
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of window index i (a 16-byte aligned pair for 32-bit reads,
// 8-byte for 16-bit) in the swizzled window
template <int SK>
__device__ __forceinline__ int swz(int i) {
    const int off = i * FirTmaGeom<SK>::XB;
    return off ^ (((off >> 7) & 3) << 4);
}

// window of tile `tile` into buffer `buf` (one thread): both polarisations'
// rows, one box each, on the buffer's mbarrier
template <int T, int SK, bool WL>
__device__ __forceinline__ void fir_tma_issue(FirTmaSmem<T, SK, WL> &sm, int buf, int tile, int tps, long k0,
                                              const CUtensorMap *tmap) {
    constexpr int D = (T - 1) / 2;
    constexpr int R = FirTmaGeom<SK>::R;
    const int s = tile / tps, tl = tile - s * tps;
    const long base = 2 * (k0 + (long)tl * kOut) - D;
    const long g0 = (base - (((base % R) + R) % R)) / R;        // first group (may be negative)
    const uint32_t bar = smem_addr(&sm.bar[buf]);
    const uint32_t bytes = 2u * FirTmaGeom<SK>::BYTES;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
#pragma unroll
    for (int p = 0; p < 2; ++p)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3, %4}], [%5];"
            ::"r"(smem_addr(sm.xs[buf][p])), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"((int)g0),
              "r"(2 * s + p), "r"(bar)
            : "memory");
}

__device__ __forceinline__ bool fir_mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

template <int T, int SK, bool WL>
__global__ void __launch_bounds__(kThreads, 4)
fir_tma_kernel(const __grid_constant__ CUtensorMap tmap, const float2 *__restrict__ taps, long k0, long k1,
               typename Store<SK>::T *__restrict__ y, long y_stride, long y_off, int tps, int n_tiles) {
    constexpr int D = (T - 1) / 2;
    constexpr int R = FirTmaGeom<SK>::R;
    constexpr int L = FirTmaSmem<T, SK, WL>::L;
    using X = typename Store<SK>::T;
    using V = typename std::conditional<sizeof(X) == 8, float4, uint2>::type;   // two samples
    __shared__ __align__(1024) FirTmaSmem<T, SK, WL> sm;
    __shared__ int fail_sh;
    const int tid = threadIdx.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fail_sh = 0;
    }
    __syncthreads();
    int tile = blockIdx.x, buf = 0;
    uint32_t phases = 0u;      // bit b: parity of buffer b's next completion
    if (tile < n_tiles) {
        if (tid == 0) fir_tma_issue<T, SK, WL>(sm, 0, tile, tps, k0, &tmap);
        const int s = tile / tps;
        for (int i = tid; i < 4 * L; i += kThreads) sm.hraw[0][i] = taps[(long)s * 4 * L + i];
    }
    for (; tile < n_tiles; tile += gridDim.x, buf ^= 1) {
        const int next = tile + gridDim.x;
        if (next < n_tiles) {
            // buffer buf ^ 1 was last read by the previous tile (the block
            // synchronised after it): order those reads before the copy
            if (tid == 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                fir_tma_issue<T, SK, WL>(sm, buf ^ 1, next, tps, k0, &tmap);
            }
            const int s = next / tps;
            for (int i = tid; i < 4 * L; i += kThreads) sm.hraw[buf ^ 1][i] = taps[(long)s * 4 * L + i];
        }
        if (!fir_mbar_wait(smem_addr(&sm.bar[buf]), (phases >> buf) & 1u)) fail_sh = 1;
        phases ^= 1u << buf;
        __syncthreads();
        if (fail_sh) break;
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

        const int s = tile / tps, tl = tile - s * tps;
        const long base = 2 * (k0 + (long)tl * kOut) - D;
        const int delta = (int)(((base % R) + R) % R);     // window index of global sample `base`
        f32x2 acc[2][4];
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[q][r] = pk2(0.f, 0.f);
        const int lb = 8 * tid + 2 * D + delta;   // window index of (output 4 tid, tap 0)
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const unsigned char *xp = sm.xs[buf][p];
            // even / odd tap chains as in fir_kernel: E[r] = x[lb + 2r - 2j],
            // O[r] = x[lb + 2r - 2j - 1], each pair (O, E) one vector read
            f32x2 E[4], Es[4], O[4], Os[4];
            auto ld = [&](int i, int r) {          // pair at window indices i, i + 1 (i even)
                const V v = *reinterpret_cast<const V *>(xp + swz<SK>(i));
                const X *pr = reinterpret_cast<const X *>(&v);
                const float2 xo = Store<SK>::ld(pr, 0), xe = Store<SK>::ld(pr, 1);
                E[r] = pk2(xe.x, xe.y);
                Es[r] = pk2(xe.y, xe.x);
                O[r] = pk2(xo.x, xo.y);
                Os[r] = pk2(xo.y, xo.x);
            };
#pragma unroll
            for (int r = 0; r < 4; ++r) ld(lb + 2 * r - 1, r);
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
                    ld(lb - 2 * (j + 1) - 1, 0);
                }
            }
        }
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
        __syncthreads();   // buffer `buf`, its taps and hA / hB are rewritten from the next tile on
    }
    // a block that stopped on a failed wait leaves no copy in flight behind
    // (bounded waits): the copy it gave up on, and the other buffer's if one
    // was issued for the next tile
    if (fail_sh) {
        fir_mbar_wait(smem_addr(&sm.bar[buf]), ((phases >> buf) & 1u) ^ 1u);
        if (tile + (int)gridDim.x < n_tiles)
            fir_mbar_wait(smem_addr(&sm.bar[buf ^ 1]), (phases >> (buf ^ 1)) & 1u);
        if (tid == 0) atomicOr(&g_fir_err, 1u);
    }
}

template <int SK, bool WL>
cudaError_t fir_tma_t(const CUtensorMap &tm, const float2 *taps, long k0, long k1, void *y, long y_stride,
                      long y_off, int T, int grid, long tps, long n_tiles, cudaStream_t st) {
    using X = typename Store<SK>::T;
    X *yy = static_cast<X *>(y);
    switch (T) {
        case 7: fir_tma_kernel<7, SK, WL><<<grid, kThreads, 0, st>>>(tm, taps, k0, k1, yy, y_stride, y_off, (int)tps, (int)n_tiles); break;
        case 15: fir_tma_kernel<15, SK, WL><<<grid, kThreads, 0, st>>>(tm, taps, k0, k1, yy, y_stride, y_off, (int)tps, (int)n_tiles); break;
        case 31: fir_tma_kernel<31, SK, WL><<<grid, kThreads, 0, st>>>(tm, taps, k0, k1, yy, y_stride, y_off, (int)tps, (int)n_tiles); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static std::atomic<PFN_cuTensorMapEncodeTiled_v12000> fn{nullptr};
    PFN_cuTensorMapEncodeTiled_v12000 f = fn.load(std::memory_order_acquire);
    if (!f) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess || q != cudaDriverEntryPointSuccess)
            return nullptr;
        f = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        fn.store(f, std::memory_order_release);
    }
    return f;
}

}  // namespace

bool fir_tma_usable(const void *x, long ns, int sk) {
    // rows of whole 64-byte groups, 16-byte aligned
    const size_t xb = store_bytes(sk);
    return (reinterpret_cast<uintptr_t>(x) & 15) == 0 && ((size_t)ns * xb) % 64 == 0 && encode_fn() != nullptr;
}

cudaError_t launch_fir_ex(const void *x, long ns, const float2 *taps, long k0, long k1, void *y, long y_stride,
                          long y_off, int n_streams, int T, cudaStream_t st, int sk, int sm_avail, int wl,
                          int tma) {
    if (!tma || !fir_tma_usable(x, ns, sk))
        return launch_fir(x, ns, taps, k0, k1, y, y_stride, y_off, n_streams, T, st, sk, sm_avail, wl);
    if (k1 <= k0 || n_streams <= 0) return cudaSuccess;
    const long tps = (k1 - k0 + kOut - 1) / kOut;
    const long n_tiles = tps * n_streams;
    if (n_tiles > (1L << 30) || 2L * n_streams > (1L << 31) || ns >= (1L << 31) - 4096) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long>(n_tiles, 4L * (sm_avail > 0 ? sm_avail : sm_count()));
    // x as [2S rows][ns / R groups][R samples] (64-byte groups); a box is
    // one window of one row, with the 64-byte swizzle; groups outside the
    // row read zeros
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof tm);
    const size_t xb = store_bytes(sk);
    const cuuint32_t R = (cuuint32_t)(64 / xb);
    const cuuint32_t G = xb == 8 ? (cuuint32_t)FirTmaGeom<SK_F32>::G : (cuuint32_t)FirTmaGeom<SK_F16>::G;
    const cuuint64_t dims[3] = {(cuuint64_t)R, (cuuint64_t)ns / R, (cuuint64_t)(2 * n_streams)};
    const cuuint64_t strides[2] = {64, (cuuint64_t)ns * xb};
    const cuuint32_t box[3] = {R, G, 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = encode_fn()(&tm, xb == 8 ? CU_TENSOR_MAP_DATA_TYPE_INT64 : CU_TENSOR_MAP_DATA_TYPE_INT32, 3,
                                   const_cast<void *>(x), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                   CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    // a map the driver refuses leaves the cp.async form (the same results)
    if (r != CUDA_SUCCESS)
        return launch_fir(x, ns, taps, k0, k1, y, y_stride, y_off, n_streams, T, st, sk, sm_avail, wl);
    if (wl) {
        switch (sk) {
            case SK_F32: return fir_tma_t<SK_F32, true>(tm, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
            case SK_F16: return fir_tma_t<SK_F16, true>(tm, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
            case SK_BF16: return fir_tma_t<SK_BF16, true>(tm, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sk) {
        case SK_F32: return fir_tma_t<SK_F32, false>(tm, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
        case SK_F16: return fir_tma_t<SK_F16, false>(tm, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
        case SK_BF16: return fir_tma_t<SK_BF16, false>(tm, taps, k0, k1, y, y_stride, y_off, T, grid, tps, n_tiles, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fir_tma_status(unsigned int *flag) {
    const unsigned int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(flag, g_fir_err, sizeof(unsigned int));
    if (e == cudaSuccess && *flag) e = cudaMemcpyToSymbol(g_fir_err, &zero, sizeof(unsigned int));
    return e;
}

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
