// Device-side initialisation of a stream's start-up state (host side of
// k_init.cu): written by kernels rather than uploaded from host memory, so
// that no copy from pageable memory synchronises a stream at a call's start.
#pragma once

#include "rx_internal.h"

// taps [S][4][L] (branches XX, XY, YX, YY; L taps each): 1 at index D of XX and
// YY, 0 elsewhere (the identity butterfly)
cudaError_t launch_center_spike(float2 *taps, int S, int L, int D, cudaStream_t st);
// StreamDev [S]: counters zero, unwrap carry (m, b) = (0, B/2)
cudaError_t launch_stream_init(StreamDev *sd, int S, int B, cudaStream_t st);
// The CDC's receiver response on n bins: H[k] = mag[k] exp(j ph_k) with the
// dispersion phase ph_k = -dl lambda^2 w_k^2 / (4 pi c), w_k = 2 pi f_k,
// f_k = (k < n/2 ? k : k - n) fs / n (conj of the all-pass CD response;
// dl = D L in s/m, lambda in m); mag (device, double) carries the matched
// filter and 1/n.  Double precision, in the host formula's operation order.
cudaError_t launch_cd_response(float2 *H, const double *mag, int n, double fs, double dl, double wavelength,
                               cudaStream_t st);
