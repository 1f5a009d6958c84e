// Static frequency-domain equaliser kernels (host side of k_fde.cu).
#pragma once

#include <cuda_runtime.h>

// R[t][t'] = sum_i conj(u_{i,t}) u_{i,t'}, p[t] = sum_i conj(u_{i,t}) d_i,
// u_{i,t} = x[sps*i + D - t] (0 outside [0, n)), D = (T-1)/2; float64.
cudaError_t launch_fde_corr(const float2 *x, long n, const float2 *d, int K, int T, int sps, double2 *R,
                            double2 *p, cudaStream_t st);
// (R + lam I) h = p, lam = delta * trace(R) / T, by Cholesky (R overwritten).
cudaError_t launch_fde_solve(double2 *R, const double2 *p, double2 *y, int T, double delta, double2 *h,
                             cudaStream_t st);
// H[k] = B[k] / 1024 * sum_t h[t] e^{-j 2 pi k (t - D) / 1024}, B the output band.
cudaError_t launch_fde_response(const double2 *h, int T, float2 *H, cudaStream_t st);
// Overlap-save application with 4 -> 2 resampling (n_ov a multiple of 4).
cudaError_t launch_fde_apply(const float2 *in, float2 *out, long ns, int n_rows, int n_ov, const float2 *H,
                             const float2 *tw, cudaStream_t st);
