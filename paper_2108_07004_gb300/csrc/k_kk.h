// Kramers-Kronig front-end kernel interface (host side of k_kk.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

constexpr int kKKMaxStreams = 256;

// Per-call parameters, passed by value (__grid_constant__).
struct KKDev {
    float floor;                  // intensity clamp before sqrt / log
    uint32_t fc_step;             // carrier offset, cycles per sample * 2^32
    int n_streams;
    float2 lv[kKKMaxStreams];     // per stream (photocurrent per code, DC term)
};

// codes [S][ns] int16 -> field [S][ns] (float2), frames f0 .. f1-1 of
// n_fft = 1024 samples advancing by 1024 - n_ov; tw = exp(-2 pi i e / 1024).
cudaError_t launch_kk(const int16_t *codes, float2 *out, long ns, int n_ov, const KKDev &p, const float2 *tw,
                      cudaStream_t st, long f0 = 0, long f1 = -1);
