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
