// Start-up state of the streams, written on the device (see k_init.h).
#include "k_init.h"

namespace {

__global__ void center_spike_kernel(float2 *__restrict__ taps, int S, int L, int D) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S * 4 * L) return;
    const int t = i % L, br = (i / L) % 4;
    taps[i] = ((br == 0 || br == 3) && t == D) ? make_float2(1.f, 0.f) : make_float2(0.f, 0.f);
}

__global__ void stream_init_kernel(StreamDev *__restrict__ sd, int S, int B) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    StreamDev v;
    memset(&v, 0, sizeof v);
    v.carry[0][0] = 0;
    v.carry[0][1] = B / 2;
    sd[s] = v;
}

constexpr double kPiD = 3.14159265358979323846;
constexpr double kCD = 299792458.0;

__global__ void cd_response_kernel(float2 *__restrict__ H, const double *__restrict__ mag, int n, double fs,
                                   double dl, double wl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double f = (k < n / 2 ? k : k - n) * fs / n;
    const double w = 2 * kPiD * f;
    const double ph = -dl * wl * wl * w * w / (4 * kPiD * kCD);
    double sn, cs;
    sincos(ph, &sn, &cs);
    H[k] = make_float2((float)(mag[k] * cs), (float)(mag[k] * sn));
}

}  // namespace

cudaError_t launch_cd_response(float2 *H, const double *mag, int n, double fs, double dl, double wavelength,
                               cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    cd_response_kernel<<<(n + 255) / 256, 256, 0, st>>>(H, mag, n, fs, dl, wavelength);
    return cudaGetLastError();
}

cudaError_t launch_center_spike(float2 *taps, int S, int L, int D, cudaStream_t st) {
    const int n = S * 4 * L;
    if (n <= 0) return cudaSuccess;
    center_spike_kernel<<<(n + 255) / 256, 256, 0, st>>>(taps, S, L, D);
    return cudaGetLastError();
}

cudaError_t launch_stream_init(StreamDev *sd, int S, int B, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    stream_init_kernel<<<(S + 127) / 128, 128, 0, st>>>(sd, S, B);
    return cudaGetLastError();
}
