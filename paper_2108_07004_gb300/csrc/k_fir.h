// The FIR with its input windows staged by the tensor memory accelerator
// (k_fir.cu): launch_fir_ex takes the TMA form when tma is set and the
// sample rows allow it (16-byte aligned base, rows of whole 64-byte groups),
// else the cp.async form of launch_fir; both give the same bits.
#pragma once

#include <cuda_runtime.h>

bool fir_tma_usable(const void *x, long ns, int sk);
cudaError_t launch_fir_ex(const void *x, long ns, const float2 *taps, long k0, long k1, void *y, long y_stride,
                          long y_off, int n_streams, int T, cudaStream_t st, int sk, int sm_avail, int wl, int tma);
// Read and clear the flag of a bounded wait that gave up (1) in any TMA FIR
// launch on the current device since the last call.
cudaError_t fir_tma_status(unsigned int *flag);
