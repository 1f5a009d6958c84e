// C ABI of the receiver: handle, parameters, tables, block schedule.
//
// The schedule follows Sec. 2 of the paper: the parallel stages (FFT
// filtering, phase search, demapping) run over whole blocks, while the
// sequential equaliser adaptation uses the first n_upd symbols of a block and
// its taps are applied to later blocks.  With a tap lag >= 2 the adaptation
// of block n runs on a second CUDA stream next to the parallel kernels of
// block n + 1 (the paper's multi-stream idea).
#include <cmath>
#include <cstdarg>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <chrono>
#include <limits>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "k_fir.h"
#include "rx_internal.h"
#include "gs4d64_table.inc"   // kGs4d64Points, kGs4d64Labels (written by build.py)
#include "k_kk.h"
#include "k_fde.h"
#include "k_init.h"

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

// A failed runtime call is reported through rx_last_error; the runtime's
// own last-error state is cleared (cudaGetLastError), so that the caller's
// next CUDA call does not see a stale error of the library's.
#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) {                                                      \
            (void)cudaGetLastError();                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? RX_ENOMEM : RX_ECUDA,       \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                             \
    } while (0)

constexpr double kPi = 3.14159265358979323846;
constexpr double kC = 299792458.0;

}  // namespace

struct rx_mlp {
    MlpDev d;
    cudaStream_t st = nullptr;
    int t = 0;                       // Adam steps taken
    long scratch_n = 0;
};

struct rx_kk {
    rx_kk_params p{};
    float2 *tw = nullptr;            // exp(-2 pi i e / 1024)
    cudaStream_t st = nullptr;
};

struct rx_fde {
    int T = 203, n_ov = 256;
    double2 *R = nullptr, *p = nullptr, *y = nullptr, *h = nullptr;   // float64 training scratch, taps
    float2 *H = nullptr;             // response on the 1024 bins (1/1024 included)
    float2 *tw = nullptr;            // exp(-2 pi i e / 1024)
    cudaStream_t st = nullptr;
    bool ready = false;              // taps set or trained
};

struct rx_handle {
    // format
    FmtDev fmt{};
    // link / receiver parameters
    double symbol_rate = 28e9;
    int sps = 2;
    double cd = 0.0;
    int T = 15;
    int B = 32;
    int n_fft = 1024, n_ov = 256;
    double mu = 1e-3;
    int W = 64;
    long block = 4096;
    int n_upd = 1024;
    int lag = 1;
    long n_pre = 2048;
    int cma_passes = 1;
    long n_cma = 0;
    int lms_block = 1;       // block-wise updates in groups of this many (1: sequential)
    double sig_fixed_up = 0; // fixed sigma^2 value on the device (0: none yet)
    int wl = 0;              // widely-linear butterfly: taps [S][2][2][2T] (x, then conj x)
    long n_train = 1024;
    int train_passes = 3;
    double sigma2_fixed = 0.0;
    long skip_head = 4096, skip_tail = 512;
    int streams = 1;
    double rolloff = 0.1;
    bool matched_filter = true;     // root-raised-cosine matched filter in the CDC multiply
    double wavelength = 1550e-9;
    // CUDA
    cudaStream_t st = nullptr;
    cudaStream_t side = nullptr;
    // the de-rotation/demap of block n runs on its own stream beside the
    // FIR and BPS of block n + 1 (ev_bps: BPS of a block done; ev_dm: its
    // demap done, by block parity)
    cudaStream_t dst = nullptr;
    // the equalised training span [S][2][n_train] (start-up scratch)
    void *ytr = nullptr;
    size_t ytr_cap = 0;
    cudaEvent_t ev_bps[2] = {nullptr, nullptr}, ev_dm[2] = {nullptr, nullptr}, ev_setup = nullptr;
    cudaEvent_t ev_unwrap = nullptr;
    cudaEvent_t ev_cdc0 = nullptr, ev_start = nullptr;   // start-up overlap with the CDC
    // host-buffer entry: input and output copies on their own streams
    cudaStream_t cp_in = nullptr, cp_out = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    // the input of the first group beyond the start-up's frames (the main
    // stream waits for it before the CDC of the remaining frames)
    cudaEvent_t ev_in_rest = nullptr;
    bool wait_rest = false;
    // host entry, groups after the first: their CDC runs on cst as soon as
    // their samples are in (ev_in), beside the previous group's kernels
    bool cdc_side = false;
    cudaStream_t cst = nullptr;
    cudaEvent_t ev_cdcg = nullptr;
    // issue mode of the device entry points (parameter "issue"): 0 the
    // stages on their own streams with events between them; 1 every stage
    // on the main stream, no event operations (handles that run beside many
    // others: the other handles fill the device); 2 as 1, and the blocks of
    // a call after the stream's first are captured as a CUDA graph and
    // launched as one, the instantiated graph updated in place per block
    int issue = 0;
    // the FIR's input windows staged by TMA where the rows allow (parameter
    // "fir_tma"; 0: the cp.async form, the same bits)
    int fir_tma = 1;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gst = nullptr;   // capture stream (the handle's own stream may be a default stream)
    bool in_host = false;     // inside rx_process_host (multi-stream always)
    // reference bits left in host memory (rx_set_reference_host): copied in
    // with the next host-entry call, group by group, into ref_bits
    const uint8_t *ref_host = nullptr;
    size_t ref_cap = 0;                       // reflab_t entries the label buffer holds
    uint8_t *ref_bits = nullptr;
    size_t ref_bits_cap = 0;
    std::vector<cudaEvent_t> ev_lms;     // one per tap-ring slot: the LMS that wrote it is done
    // lms_start = 1: the update of block n starts from W_n = U_{n-lag}, so the
    // blocks n = r (mod lag) form lag independent chains, chain r on
    // side (r = 0) or side_x[r - 1]
    int lms_start = 0;
    cudaStream_t side_x[3] = {nullptr, nullptr, nullptr};
    // device tables: the CDC response H (per dispersion, formed on the
    // device), the twiddles tw (per FFT size) and the matched filter's
    // magnitude with 1/n_fft (per FFT size, sample rate and roll-off)
    float2 *H = nullptr, *tw = nullptr;
    double *Hmag = nullptr;
    double mag_key[5] = {0, 0, 0, 0, -1};
    cudaEvent_t ev_tab = nullptr;
    // the tensor-core phase search (parameter "bps_tc", default on where the
    // format allows): its B operand, built for the table and B test phases
    int bps_tc = 0;
    // the DD-LMS's warp-wide nearest-point search on every update (parameter
    // "lms_exact"; default 0: decisions taken a sub-block ahead where the
    // margin allows, with the same results)
    int lms_exact = 0;
    // SMs left to other work on the GPU (parameter "sm_reserve"; e.g. the LMS
    // blocks of another handle's frame in flight): the grids that size
    // themselves to one wave count them out
    int sm_reserve = 0;
    float *bps_w = nullptr;
    int tab_fft = 0;
    bool tables_dirty = true;
    // device buffers
    long cap_n = 0;
    int cap_s = 0, cap_lag = 0, cap_wl = 0, cap_ring = 0;
    void *x = nullptr, *y = nullptr;                  // CDC and FIR outputs, storage kind prec
    float2 *ring = nullptr;
    uint8_t *bidx = nullptr;
    uint16_t *pcode = nullptr;
    int *dsum = nullptr;
    double *part_u = nullptr, *part_d = nullptr, *sig = nullptr, *sig_fixed = nullptr;
    double *mdsum = nullptr;
    StreamDev *sd = nullptr;
    long cap_dsum = 0, cap_pd = 0;
    // reference
    reflab_t *ref = nullptr;
    long ref_n = 0;
    int ref_s = 0;
    // stream state (host mirror of the scalars)
    bool started = false;
    bool trained = false;
    int prec = SK_F32;                                // storage of x and y (precision variant)
    int cap_prec = -1;
    // learned demapper (null: exact log-sum-exp) and symbol outputs
    rx_mlp *mlp = nullptr;
    float *user_x4 = nullptr, *user_s2 = nullptr;   // caller's [S][N][4], [S][N]
    float *x4 = nullptr, *s2sym = nullptr;          // own, for the learned demapper
    long cap_x4 = 0;
    long blocks_done = 0;
    unsigned long long u = 0;
    long cur_n = 0;
    // profiling (parameter "profile"): 1 = CUDA events around every launch
    // group and every block, 2 = around the BPS launches only
    int profile = 0;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    struct Rec { int stage; cudaEvent_t a, b; };
    std::vector<Rec> recs;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> blk;
    unsigned long long nlaunch[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // host sources of asynchronous uploads (kept alive until the next call)
    std::vector<double> h_sig;
    // streaming entry (rx_push / rx_flush): the stream is held in a window of
    // `cap` symbols whose local symbol 0 is global symbol `origin`; input and
    // LLR windows are double-buffered so that a move of the window's origin
    // is a copy between the two
    struct Push {
        bool on = false;
        long tot = 0;         // samples per polarisation pushed so far
        long origin = 0;      // global symbol of local symbol 0
        long nb = 0;          // next block to run (global)
        long emitted = 0;     // output rows handed out so far
        long delay = 0;       // fixed stream delay d in symbols
        long cap = 0;         // window length in symbols
        long step = 0;        // origin moves in multiples of this many symbols
        long piece = 0;       // largest number of samples appended at once
        float2 *in[2] = {nullptr, nullptr};
        float *llr[2] = {nullptr, nullptr};
        int cur = 0;
        void *halo = nullptr; // [S][2][W] FIR output, moved on a flush
        size_t in_bytes = 0, llr_bytes = 0, halo_bytes = 0;
    } push;
    // host staging
    void *h_in = nullptr, *h_out = nullptr;
    size_t h_in_cap = 0, h_out_cap = 0;
    float2 *d_in = nullptr;
    float *d_out = nullptr;
    size_t d_in_cap = 0, d_out_cap = 0;
};

namespace {

// ---------------------------------------------------------------------------
// tables
// ---------------------------------------------------------------------------
void gray_qam(int m_pol, std::vector<float> &pts) {
    // square Gray QAM: label = (I bits)(Q bits), per-axis Gray code, bit 0 on the positive side
    const int h = m_pol / 2, L = 1 << h;
    std::vector<double> lev(L);
    for (int pidx = 0; pidx < L; ++pidx) {
        const int g = pidx ^ (pidx >> 1);
        lev[g] = (L - 1) - 2.0 * pidx;
    }
    const int M = 1 << m_pol;
    double e = 0;
    pts.assign(M * 2, 0.f);
    std::vector<double> tmp(M * 2);
    for (int lab = 0; lab < M; ++lab) {
        tmp[2 * lab] = lev[lab >> h];
        tmp[2 * lab + 1] = lev[lab & (L - 1)];
        e += tmp[2 * lab] * tmp[2 * lab] + tmp[2 * lab + 1] * tmp[2 * lab + 1];
    }
    const double sc = 1.0 / std::sqrt(e / M);
    for (int i = 0; i < M * 2; ++i) pts[i] = (float)(tmp[i] * sc);
}

bool same4(const float *a, const float *b, int n) {
    for (int i = 0; i < n; ++i)
        if (a[i] != b[i]) return false;
    return true;
}

// rotate a point by k quarter turns (exact in float)
void rot_q(const float *p, int dims, int k, float *out) {
    for (int i = 0; i < dims; i += 2) {
        float re = p[i], im = p[i + 1];
        for (int t = 0; t < k; ++t) { const float r2 = -im; im = re; re = r2; }
        out[i] = re;
        out[i + 1] = im;
    }
}

int build_format(const rx_format *f, FmtDev &d) {
    std::vector<float> pts;
    int dims, mb, S;
    if (f->kind == RX_FMT_DP_QPSK || f->kind == RX_FMT_DP_16QAM || f->kind == RX_FMT_DP_64QAM) {
        dims = 2;
        mb = f->kind == RX_FMT_DP_QPSK ? 2 : (f->kind == RX_FMT_DP_16QAM ? 4 : 6);
        S = 4;
        gray_qam(mb, pts);
    } else if (f->kind == RX_FMT_CUSTOM || f->kind == RX_FMT_GS4D64) {
        const bool gs = f->kind == RX_FMT_GS4D64;
        dims = gs ? 4 : f->dims;
        mb = gs ? 6 : f->m_bits;
        S = gs ? 4 : f->sym_order;
        const float *fp = gs ? &kGs4d64Points[0][0] : f->points;
        const uint32_t *fl = gs ? kGs4d64Labels : f->labels;
        if (dims != 2 && dims != 4) return fail(RX_EINVAL, "format dims must be 2 or 4");
        if (!fp || !fl) return fail(RX_EINVAL, "custom format needs points and labels");
        if (mb < 1 || mb > (dims == 2 ? 7 : 6)) return fail(RX_EINVAL, "m_bits %d out of range", mb);
        const int M = 1 << mb;
        pts.assign((size_t)M * dims, 0.f);
        std::vector<int> seen(M, 0);
        for (int i = 0; i < M; ++i) {
            const uint32_t lab = fl[i];
            if (lab >= (uint32_t)M || seen[lab]) return fail(RX_EINVAL, "labels are not a permutation");
            seen[lab] = 1;
            for (int c = 0; c < dims; ++c) pts[(size_t)lab * dims + c] = fp[(size_t)i * dims + c];
        }
    } else {
        return fail(RX_EINVAL, "unknown format kind %d", f->kind);
    }
    const int M = 1 << mb;
    if (S != 1 && S != 2 && S != 4) return fail(RX_EINVAL, "sym_order must be 1, 2 or 4");
    if (dims == 2 && (M < 4 || M > 128)) return fail(RX_EINVAL, "2D tables of 4 to 128 points are supported");
    if (dims == 4 && M != 64) return fail(RX_EINVAL, "4D tables of 64 points are supported");
    std::memset(&d, 0, sizeof d);
    d.dims = dims;
    d.M = M;
    d.m_pol = mb;
    d.m = dims == 4 ? mb : 2 * mb;
    d.S = S;
    double e2 = 0, e4 = 0;
    int cnt = 0;
    for (int j = 0; j < M; ++j) {
        double pe = 0;
        for (int c = 0; c < dims; ++c) {
            d.pts[j][c] = pts[(size_t)j * dims + c];
            d.ptsT[c][j] = d.pts[j][c];
            pe += (double)d.pts[j][c] * d.pts[j][c];
        }
        d.pe[j] = (float)pe;
        for (int c = 0; c < dims; c += 2) {
            const double a2 = (double)d.pts[j][c] * d.pts[j][c] + (double)d.pts[j][c + 1] * d.pts[j][c + 1];
            e2 += a2;
            e4 += a2 * a2;
            ++cnt;
        }
    }
    d.R2 = (float)(e4 / e2);
    // orbits under rotation by 2 pi / S (verified exactly)
    const int step = 4 / S;   // quarter turns per symmetry step
    std::vector<int> orb_of(M, -1);
    int no = 0;
    for (int j = 0; j < M; ++j) {
        if (orb_of[j] >= 0) continue;
        if (no >= RX_MAXM) return fail(RX_EINVAL, "too many orbits");
        for (int c = 0; c < 4; ++c) d.orb[no][c] = c < dims ? d.pts[j][c] : 0.f;
        d.orbe[no] = d.pe[j];
        for (int k = 0; k < S; ++k) {
            float rp[4];
            rot_q(d.pts[j], dims, k * step, rp);
            int found = -1;
            for (int jj = 0; jj < M; ++jj)
                if (same4(rp, d.pts[jj], dims)) { found = jj; break; }
            if (found < 0 || (orb_of[found] >= 0 && !(k == 0 && found == j)))
                return fail(RX_EINVAL, "table is not invariant under rotation by 2pi/%d", S);
            orb_of[found] = no;
            d.orb_lab[no][k] = found;
        }
        ++no;
    }
    d.n_orb = no;
    for (int o = 0; o < 16; ++o) {
        for (int c = 0; c < 4; ++c) d.orbT[c][o] = o < no ? d.orb[o][c] : 0.f;
        d.orbeP[o] = o < no ? d.orbe[o] : std::numeric_limits<float>::infinity();
    }
    if (no > (dims == 2 ? 32 : 16))
        return fail(RX_EINVAL, "%d orbits under the rotation by 2pi/%d; at most %d are supported", no, S,
                    dims == 2 ? 32 : 16);
    return RX_OK;
}

void set_phases(FmtDev &d, int B) {
    d.B = B;
    for (int b = 0; b < B; ++b) {
        const double ph = ((double)b / B - 0.5) * 2.0 * kPi / d.S;
        d.cs[b][0] = (float)std::cos(ph);
        d.cs[b][1] = (float)std::sin(ph);
        d.csp[b][0] = d.csp[b][1] = d.cs[b][0];
        d.csp[b][2] = d.csp[b][3] = d.cs[b][1];
    }
}

double raised_cosine(double f, double rs, double beta) {
    const double af = std::fabs(f), lo = (1 - beta) * rs / 2, hi = (1 + beta) * rs / 2;
    if (af <= lo) return 1.0;
    if (af <= hi) return 0.5 * (1 + std::cos(kPi * (af - lo) / (beta * rs)));
    return 0.0;
}

// whether the chain's phase search runs on the tensor cores
bool use_bps_tc(const rx_handle *h) { return h->bps_tc && bps_tc_supported(h->fmt); }

int upload_tables(rx_handle *h) {
    if (use_bps_tc(h) && !h->bps_w) {
        std::vector<float> w(bps_tc_table_floats(h->B));
        bps_tc_table(h->fmt, w.data());
        CK(cudaMalloc(&h->bps_w, sizeof(float) * w.size()));
        CK(cudaMemcpy(h->bps_w, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice));
    }
    if (!h->tables_dirty && h->tab_fft == h->n_fft) return RX_OK;
    const int n = h->n_fft;
    const double fs = h->sps * h->symbol_rate;
    if (h->tab_fft != n) {
        cudaFree(h->H);
        cudaFree(h->tw);
        cudaFree(h->Hmag);
        h->H = h->tw = nullptr;
        h->Hmag = nullptr;
        CK(cudaMalloc(&h->H, sizeof(float2) * n));
        CK(cudaMalloc(&h->tw, sizeof(float2) * n));
        CK(cudaMalloc(&h->Hmag, sizeof(double) * n));
        std::vector<float2> tw(n);
        for (int k = 0; k < n; ++k)
            tw[k] = make_float2((float)std::cos(2 * kPi * k / n), (float)(-std::sin(2 * kPi * k / n)));
        CK(cudaMemcpy(h->tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
        h->tab_fft = n;
        h->mag_key[4] = -1;
    }
    const double key[5] = {fs, h->symbol_rate, h->rolloff, h->matched_filter ? 1.0 : 0.0, (double)n};
    if (std::memcmp(key, h->mag_key, sizeof key) != 0) {
        std::vector<double> mag(n);
        for (int k = 0; k < n; ++k) {
            const double f = (k < n / 2 ? k : k - n) * fs / n;
            mag[k] = (h->matched_filter ? std::sqrt(h->sps * raised_cosine(f, h->symbol_rate, h->rolloff)) : 1.0) / n;
        }
        CK(cudaMemcpy(h->Hmag, mag.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
        std::memcpy(h->mag_key, key, sizeof key);
    }
    // the dispersion phase on the device (a request's new link costs one
    // small kernel, not a host loop and a synchronous copy)
    CK(launch_cd_response(h->H, h->Hmag, n, fs, h->cd * 1e-3, h->wavelength, h->st));
    if (h->cst) {
        // the host entry's CDC of later groups runs on its own stream
        if (!h->ev_tab) CK(cudaEventCreateWithFlags(&h->ev_tab, cudaEventDisableTiming));
        CK(cudaEventRecord(h->ev_tab, h->st));
        CK(cudaStreamWaitEvent(h->cst, h->ev_tab, 0));
    }
    h->tables_dirty = false;
    return RX_OK;
}

void free_buffers(rx_handle *h) {
    cudaFree(h->x); cudaFree(h->y); cudaFree(h->ring);
    cudaFree(h->bidx); cudaFree(h->pcode); cudaFree(h->dsum); cudaFree(h->part_u);
    cudaFree(h->part_d); cudaFree(h->sig); cudaFree(h->sig_fixed); cudaFree(h->sd);
    cudaFree(h->mdsum);
    h->mdsum = nullptr;
    h->x = h->y = h->ring = nullptr;
    h->bidx = nullptr; h->pcode = nullptr; h->dsum = nullptr;
    h->part_u = h->part_d = h->sig = h->sig_fixed = nullptr;
    h->sd = nullptr;
    h->cap_n = 0; h->cap_s = 0; h->cap_lag = 0; h->cap_ring = 0;
}

int ensure_symbol_buffers(rx_handle *h, long N) {
    const size_t need = (size_t)h->streams * N;
    if (h->x4 && h->cap_x4 >= (long)need) return RX_OK;
    cudaFree(h->x4);
    cudaFree(h->s2sym);
    h->x4 = h->s2sym = nullptr;
    h->cap_x4 = 0;
    CK(cudaMalloc(&h->x4, sizeof(float) * 4 * need));
    CK(cudaMalloc(&h->s2sym, sizeof(float) * need));
    h->cap_x4 = (long)need;
    return RX_OK;
}

// taps per butterfly branch (widely linear: T on x, then T on conj x)
int tl(const rx_handle *h) { return h->wl ? 2 * h->T : h->T; }
int lms_opts(const rx_handle *h) { return (h->wl ? LMS_WL : 0) | (h->lms_exact ? LMS_EXACT_DD : 0); }

// Tap-ring slots.  U_n goes to slot n; it is read by the FIR of block
// n + lag and by the update that starts from it.  Sequential chain
// (lms_start 0): lag + 1 slots.  Independent chains (lms_start 1, lag >= 2):
// 2 lag slots, so that the update that overwrites slot n (that of block
// n + 2 lag) runs on the same chain stream after the reader of slot n
// (the update of block n + lag) and after the FIR of block n + lag.
int ring_size(const rx_handle *h) { return (h->lms_start && h->lag >= 2) ? 2 * h->lag : h->lag + 1; }

int ensure_buffers(rx_handle *h, long N) {
    const int S = h->streams;
    if (h->cap_n >= N && h->cap_s == S && h->cap_lag == h->lag && h->cap_prec == h->prec && h->cap_wl == h->wl &&
        h->cap_ring == ring_size(h) && h->sd)
        return RX_OK;
    free_buffers(h);
    const long ns = 2 * N;
    const long ncta = (N + bps_cta_range(1) - 1) / bps_cta_range(1) + 2;
    const long ncta_d = (h->block + 2 * h->W + 255) / 256 + 2;
    CK(cudaMalloc(&h->x, store_bytes(h->prec) * (size_t)S * 2 * ns));
    CK(cudaMalloc(&h->y, store_bytes(h->prec) * (size_t)S * 2 * N));
    CK(cudaMalloc(&h->ring, sizeof(float2) * (size_t)ring_size(h) * S * 4 * tl(h)));
    CK(cudaMalloc(&h->bidx, (size_t)S * N));
    CK(cudaMalloc(&h->pcode, sizeof(uint16_t) * (size_t)S * N));
    CK(cudaMalloc(&h->dsum, sizeof(int) * 2 * (size_t)S * ncta));        // by block parity
    CK(cudaMalloc(&h->part_u, sizeof(double) * (size_t)S * ncta));
    CK(cudaMalloc(&h->mdsum, sizeof(double) * 2 * (size_t)S * ncta));
    CK(cudaMalloc(&h->part_d, sizeof(double) * 5 * (size_t)S * ncta_d));
    CK(cudaMalloc(&h->sig, sizeof(double) * S));
    CK(cudaMalloc(&h->sig_fixed, sizeof(double) * S));
    h->sig_fixed_up = 0;
    CK(cudaMalloc(&h->sd, sizeof(StreamDev) * S));
    CK(cudaMemset(h->sd, 0, sizeof(StreamDev) * S));
    h->cap_dsum = ncta;
    h->cap_pd = ncta_d;
    h->cap_n = N;
    h->cap_wl = h->wl;
    h->cap_s = S;
    h->cap_lag = h->lag;
    h->cap_ring = ring_size(h);
    h->cap_prec = h->prec;
    return RX_OK;
}

int ensure_streams(rx_handle *h) {
    if (!h->side) {
        // the sequential adaptation (start-up, and block updates for lag >= 2)
        // runs on a high-priority stream
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        CK(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest));
        CK(cudaEventCreateWithFlags(&h->ev_unwrap, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_cdc0, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_start, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&h->dst, cudaStreamNonBlocking));
        for (int i = 0; i < 2; ++i) {
            CK(cudaEventCreateWithFlags(&h->ev_bps[i], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ev_dm[i], cudaEventDisableTiming));
        }
        CK(cudaEventCreateWithFlags(&h->ev_setup, cudaEventDisableTiming));
    }
    if (h->lms_start) {
        int least = 0, greatest = 0;
        CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        for (int r = 1; r < h->lag; ++r)
            if (!h->side_x[r - 1]) CK(cudaStreamCreateWithPriority(&h->side_x[r - 1], cudaStreamNonBlocking, greatest));
    }
    while ((int)h->ev_lms.size() < ring_size(h)) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        h->ev_lms.push_back(e);
    }
    return RX_OK;
}

int check_config(rx_handle *h) {
    if (h->sps != 2) return fail(RX_EINVAL, "sps must be 2");
    if (h->T != 7 && h->T != 15 && h->T != 31) return fail(RX_EINVAL, "taps must be 7, 15 or 31");
    if (h->B < 2 || h->B > RX_MAXB || (h->B & 1)) return fail(RX_EINVAL, "bps_phases must be even, 2..%d", RX_MAXB);
    if (h->n_fft != 1024 && h->n_fft != 4096) return fail(RX_EINVAL, "fft must be 1024 or 4096");
    if (h->n_ov < 2 || (h->n_ov & 1) || h->n_ov >= h->n_fft / 2)
        return fail(RX_EINVAL, "overlap must be even and < fft/2");
    if (h->W < 2 || h->W > 64 || (h->W & 1)) return fail(RX_EINVAL, "bps_window must be even, 2..64");
    if (h->lag < 1 || h->lag > 4) return fail(RX_EINVAL, "lag must be 1..4");
    if (h->n_upd < 0 || h->n_upd + h->W / 2 > h->block)
        return fail(RX_EINVAL, "n_upd + bps_window/2 must not exceed block");
    if (h->block < 64) return fail(RX_EINVAL, "block too small");
    if (h->streams < 1) return fail(RX_EINVAL, "streams must be >= 1");
    return RX_OK;
}

float2 *slot(rx_handle *h, long n) {
    const int L1 = ring_size(h);
    const long i = ((n % L1) + L1) % L1;
    return h->ring + (size_t)i * h->streams * 4 * tl(h);
}

enum { ST_CDC = 0, ST_FIR, ST_BPS, ST_UNWRAP, ST_DEMAP, ST_LMS, ST_STARTUP, ST_N };
const char *kStageNames[ST_N] = {"cdc", "fir", "bps", "unwrap", "demap", "lms", "startup"};

cudaEvent_t prof_event(rx_handle *h) {
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

// record the start of a launch group of `stage` on stream `s`; returns a token
cudaEvent_t prof_begin(rx_handle *h, cudaStream_t s, int stage) {
    if (!h->profile || (h->profile == 2 && stage != ST_BPS)) return nullptr;
    cudaEvent_t e = prof_event(h);
    if (e) cudaEventRecord(e, s);
    return e;
}

void prof_end(rx_handle *h, int stage, cudaEvent_t a, cudaStream_t s, int launches) {
    h->nlaunch[stage] += launches;
    if (!h->profile || !a) return;
    cudaEvent_t b = prof_event(h);
    if (!b) return;
    cudaEventRecord(b, s);
    h->recs.push_back({stage, a, b});
}

#define STAGE(stage, stream, nl, call)                  \
    do {                                               \
        cudaEvent_t ev_a_ = prof_begin(h, stream, stage); \
        CK(call);                                      \
        prof_end(h, stage, ev_a_, stream, nl);         \
    } while (0)

// A host reference that no host-entry call has taken in yet: copied and
// labelled whole on the main stream before a device entry point uses it.
int flush_ref(rx_handle *h) {
    if (!h->ref_host) return RX_OK;
    const uint8_t *rh = h->ref_host;
    h->ref_host = nullptr;
    const size_t nb = (size_t)h->ref_s * h->ref_n * h->fmt.m;
    CK(cudaMemcpyAsync(h->ref_bits, rh, nb, cudaMemcpyHostToDevice, h->st));
    CK(launch_ref_labels_rows(h->ref_bits, h->ref, h->ref_n, 0, h->ref_n, h->ref_s, h->fmt.m, h->st));
    return RX_OK;
}

// Training stage (Sec. 2: the equaliser converges on a known sequence before
// it runs blind): output order and phases from the correlation with the
// known symbols, data-aided phase codes over the span, then train_passes
// passes of data-aided LMS.  Taps are updated in place.
int train_stage(rx_handle *h, const void *x, long ns, float2 *taps, long ntr, uint16_t *pcode,
                long pcode_stride, int32_t *carry, int carry_stride, cudaStream_t st, int sk) {
    const int S = h->streams, T = h->T;
    // the training span equalised by the FIR kernel, once with the start-up
    // taps (for the alignment) and once with the aligned taps (for the phases)
    const size_t need = store_bytes(sk) * (size_t)S * 2 * ntr;
    if (h->ytr_cap < need) {
        if (h->ytr) { CK(cudaStreamSynchronize(st)); cudaFree(h->ytr); h->ytr = nullptr; }
        CK(cudaMalloc(&h->ytr, need));
        h->ytr_cap = need;
    }
    STAGE(ST_STARTUP, st, 1, launch_fir_ex(x, ns, taps, 0, ntr, h->ytr, ntr, 0, S, T, st, sk, 0, h->wl, h->fir_tma));
    STAGE(ST_STARTUP, st, 1, launch_align(h->ytr, ntr, taps, h->ref, h->ref_n, (int)ntr, S, tl(h), h->fmt, st, sk));
    STAGE(ST_STARTUP, st, 1, launch_fir_ex(x, ns, taps, 0, ntr, h->ytr, ntr, 0, S, T, st, sk, 0, h->wl, h->fir_tma));
    STAGE(ST_STARTUP, st, 1, launch_train_phase(h->ytr, ntr, h->ref, h->ref_n, (int)ntr, h->W, pcode,
                                                pcode_stride, carry, carry_stride, S, h->fmt, st, sk));
    if (h->train_passes > 0)
        STAGE(ST_STARTUP, st, 1, launch_lms(x, ns, taps, taps, 0, (int)ntr, pcode, pcode_stride, 3,
                                            h->train_passes, 0, 0, (float)h->mu, h->ref, h->ref_n,
                                            S, T, h->fmt, st, sk, lms_opts(h)));
    return RX_OK;
}

// CDC frames that blocks [b0, b1) (and, for b0 = 0, the start-up) read:
// output k of the FIR and the LMS reads samples 2k - D .. 2k + D.  [f0, fs)
// are the start-up's frames (b0 = 0), [fs, f1) the rest.
struct CdcFrames {
    long f0, fs, f1;
};
CdcFrames cdc_frames(const rx_handle *h, long N, long b0, long b1) {
    const long Nb = h->block, ns = 2 * N;
    const int D = (h->T - 1) / 2;
    const long k_hi = std::min(b1 * Nb, N);
    const long k_st = b0 == 0 ? std::min(N, std::max(h->n_pre, h->n_train)) : 0;
    const long Sk = h->n_fft - h->n_ov;
    const long s_lo = std::max(0L, 2 * b0 * Nb - D);
    CdcFrames c;
    c.f0 = s_lo / Sk;
    c.f1 = (std::min(ns, 2 * std::max(k_hi, k_st) + D) + Sk - 1) / Sk;
    c.fs = b0 == 0 ? std::min(c.f1, (std::min(ns, 2 * k_st + D) + Sk - 1) / Sk) : c.f0;
    return c;
}

// A window of a longer stream (the streaming entry points): local symbol 0
// of the buffers is global symbol `origin`, a multiple of the block length
// with 2 origin a multiple of the CDC hop, so blocks and CDC frames fall as
// in the whole stream.  Blocks keep their global numbers (bofs = origin /
// block) for the tap ring, the events and the parity-indexed buffers;
// counting covers global symbols [c0, c1) against the reference indexed
// globally.
struct Window {
    long bofs = 0, origin = 0, c0 = 0, c1 = 0;
};

// Run blocks [b0, b1) of S streams of N symbols whose samples are at `in`;
// `fresh` starts new per-call records (stage times, block latencies);
// `join` makes the main stream wait for the side stream's last LMS, so that
// the state is complete when the main stream's work is (calls that return
// to the user; the host entry's groups pass false except for the last).
// `win` (may be null): the buffers hold a window of a longer stream.
int run_blocks(rx_handle *h, const float2 *in, long N, long b0, long b1, float *llr, bool fresh = true,
               bool join = true, const Window *win = nullptr) {
    const int S = h->streams, T = h->T, L = h->lag;
    const long G = win ? win->bofs : 0;   // global number of local block 0
    const long Nb = h->block, ns = 2 * N;
    const long nblk = (N + Nb - 1) / Nb;
    const size_t tapsz = sizeof(float2) * (size_t)S * 4 * tl(h);
    cudaStream_t st = h->st;
    int rc;
    if ((rc = flush_ref(h)) != RX_OK) return rc;
    if ((rc = upload_tables(h)) != RX_OK) return rc;
    if ((rc = ensure_buffers(h, N)) != RX_OK) return rc;
    if ((rc = ensure_streams(h)) != RX_OK) return rc;
    // one-stream issue: every stage on the main stream, where stream order
    // gives every dependency the events below would (skipped)
    const bool one = h->issue != 0 && !win && !h->in_host;
    auto rec = [one](cudaEvent_t e, cudaStream_t s) { return one ? cudaSuccess : cudaEventRecord(e, s); };
    auto wt = [one](cudaStream_t s, cudaEvent_t e) { return one ? cudaSuccess : cudaStreamWaitEvent(s, e, 0); };
    const cudaStream_t side = one ? st : h->side;
    const FmtDev &f = h->fmt;
    const int D = (T - 1) / 2;

    // CDC of the frames that these blocks (and, for b0 = 0, the start-up)
    // read: output k of the FIR and the LMS reads samples 2k - D .. 2k + D.
    // For b0 = 0 the start-up's frames go first; the start-up then runs on
    // the side stream while the main stream filters the rest.
    {
        const CdcFrames cf = cdc_frames(h, N, b0, b1);
        const long f0 = cf.f0, fs = cf.fs, f1 = cf.f1;
        if (fresh) {
            h->ev_used = 0;
            h->recs.clear();
            h->blk.clear();
            for (auto &c : h->nlaunch) c = 0;
        }
        if (fs > f0) {
            STAGE(ST_CDC, st, 1, launch_cdc(in, h->x, ns, 2 * S, h->n_fft, h->n_ov, h->H, h->tw, st, f0, fs,
                                            h->prec));
            CK(rec(h->ev_cdc0, st));
            CK(wt(side, h->ev_cdc0));
        }
        if (h->wait_rest) {
            CK(cudaStreamWaitEvent(st, h->ev_in_rest, 0));
            h->wait_rest = false;
        }
        if (f1 > fs && h->cdc_side && fs == f0) {
            // frames shared with the previous group are recomputed to the
            // same values, so its readers are not disturbed
            CK(cudaStreamWaitEvent(h->cst, h->ev_in, 0));
            STAGE(ST_CDC, h->cst, 1, launch_cdc(in, h->x, ns, 2 * S, h->n_fft, h->n_ov, h->H, h->tw, h->cst, fs,
                                                f1, h->prec));
            CK(cudaEventRecord(h->ev_cdcg, h->cst));
            CK(cudaStreamWaitEvent(st, h->ev_cdcg, 0));
        } else if (f1 > fs) {
            STAGE(ST_CDC, st, 1, launch_cdc(in, h->x, ns, 2 * S, h->n_fft, h->n_ov, h->H, h->tw, st, fs, f1,
                                            h->prec));
        }
    }
    if (b0 == 0 && G == 0) {
        const cudaStream_t ss = side;        // start-up stream
        // the identity butterfly and the stream state are written by kernels:
        // a copy from pageable host memory would synchronise its stream first
        float2 *w0 = slot(h, 0);
        CK(launch_center_spike(w0, S, tl(h), (h->T - 1) / 2, ss));
        const long npre = std::min(h->n_pre, N);
        STAGE(ST_STARTUP, ss, 1, launch_lms(h->x, ns, w0, w0, 0, (int)npre, nullptr, 0, 0, h->cma_passes,
                                            0, 0, (float)h->mu, nullptr, 0, S, T, f, ss, h->prec, lms_opts(h)));
        // stream state: counters zero, unwrap carry phi_hat = 0
        CK(launch_stream_init(h->sd, S, h->B, st));
        const long ntr = std::min(h->n_train, N);
        h->trained = false;
        if (h->ref && ntr > 0 && h->ref_n >= ntr) {
            h->trained = true;
            int rc2 = train_stage(h, h->x, ns, w0, ntr, h->pcode, N, nullptr, 0, ss, h->prec);
            if (rc2 != RX_OK) return rc2;
        }
        // W_0 into the slots of U_{-lag} .. U_{-1}
        for (int i = 1; i <= L; ++i) CK(cudaMemcpyAsync(slot(h, -i), w0, tapsz, cudaMemcpyDeviceToDevice, ss));
        CK(rec(h->ev_start, ss));
        CK(wt(st, h->ev_start));
        h->u = 0;
        h->blocks_done = 0;
        h->started = true;
        h->cur_n = N;
    }
    // grids of the main stream leave room for the side-stream LMS (one SM
    // per stream) when it runs beside them
    const int chains = (h->lms_start && L >= 2) ? L : 1;
    const int sms = std::max(sm_count() / 2, sm_count() - h->sm_reserve);
    const int avail = (L >= 2 && h->lms_block == 1) ? std::max(sm_count() / 2, sms - chains * S) : sms;
    const int R = ring_size(h);
    if (h->sigma2_fixed > 0 && h->sig_fixed_up != h->sigma2_fixed) {
        // uploaded when it changes (demaps of an earlier call may still read it)
        h->h_sig.assign(S, h->sigma2_fixed);
        CK(cudaMemcpyAsync(h->sig_fixed, h->h_sig.data(), sizeof(double) * S, cudaMemcpyHostToDevice, st));
        h->sig_fixed_up = h->sigma2_fixed;
    }
    const int m = f.m;
    const long sd_stride = sizeof(StreamDev) / sizeof(int32_t);
    SymOut sym;
    if (h->user_x4 || h->user_s2) {
        sym.x4 = h->user_x4;
        sym.s2 = h->user_s2;
        sym.stride = N;
    }
    if (h->mlp && (!sym.x4 || !sym.s2)) {
        if ((rc = ensure_symbol_buffers(h, N)) != RX_OK) return rc;
        if (!sym.x4) sym.x4 = h->x4;
        if (!sym.s2) sym.s2 = h->s2sym;
        sym.stride = N;
    }
    int32_t *carry_base = reinterpret_cast<int32_t *>(h->sd);
    DemapCount cnt{};
    cnt.ref_lab = (h->ref && h->ref_n >= N) ? h->ref : nullptr;
    cnt.ref_stride = h->ref_n;
    cnt.c0 = std::min(h->skip_head, N);
    cnt.c1 = std::max(cnt.c0, N - h->skip_tail);
    if (win) {
        // global counting window, the reference indexed from the origin
        cnt.c0 = std::min(N, std::max(0L, win->c0 - win->origin));
        cnt.c1 = std::max(cnt.c0, std::min(N, std::min(win->c1, (long)h->ref_n) - win->origin));
        cnt.ref_lab = (h->ref && cnt.c1 > cnt.c0) ? h->ref + win->origin : nullptr;
    }
    cnt.sd = h->sd;
    cnt.partial = h->part_d;
    const cudaStream_t ds = one ? st : h->dst;
    // the demap stream starts after this call's set-up on the main stream
    CK(rec(h->ev_setup, st));
    CK(wt(ds, h->ev_setup));
    for (long n = b0; n < b1; ++n) {
        const long g = n + G;                 // global block number
        const long k0 = n * Nb, k1 = std::min(k0 + Nb, N);
        if (L >= 2 && g >= L) CK(wt(st, h->ev_lms[(g - L) % R]));
        // W_g = U_{g-lag}; for g < lag the slot read has not been written since start-up (W_0)
        const float2 *wn = slot(h, g - L);
        cudaEvent_t blk0 = nullptr;
        if (h->profile == 1 && (blk0 = prof_event(h))) CK(cudaEventRecord(blk0, st));
        STAGE(ST_FIR, st, 1,
              launch_fir_ex(h->x, ns, wn, k0, k1, h->y, N, k0, S, T, st, h->prec, avail, h->wl, h->fir_tma));
        const long a = std::max(0L, k0 - h->W / 2);
        const long e = (n == nblk - 1) ? N : k1 - h->W / 2;
        const bool tc = use_bps_tc(h);
        const int chunks = tc ? bps_chunks_tc(e - a, S, avail) : bps_chunks(e - a, S, avail);
        const int par = (int)(g & 1);
        int *dsum_n = h->dsum + (size_t)par * S * h->cap_dsum;
        double *mdsum_n = h->mdsum + (size_t)par * S * h->cap_dsum;
        // the partial sums of this parity were read by the demap of block n - 2
        // (possibly of an earlier call: the demap stream is not joined between
        // the host entry's groups)
        if (g >= 2) CK(wt(st, h->ev_dm[par]));
        if (tc)
            STAGE(ST_BPS, st, 1, launch_bps_tc(h->y, N, a, e, k1, h->W, h->bidx, N, a, dsum_n, mdsum_n, chunks, S,
                                               h->bps_w, f, st, h->prec));
        else
            STAGE(ST_BPS, st, 1, launch_bps(h->y, N, a, e, k1, h->W, h->bidx, N, a, dsum_n, mdsum_n, chunks, S,
                                            f, st, h->prec));
        CK(rec(h->ev_bps[par], st));
        CK(wt(ds, h->ev_bps[par]));
        const int cin = (int)(g & 1), cout = 1 - cin;
        if (g == 0 && h->trained) {
            // the training phases fix the start quadrant of the unwrap
            STAGE(ST_UNWRAP, ds, 1, launch_anchor(h->bidx, N, h->pcode, N, (int)std::min(h->n_train, e),
                                                  carry_base, (int)sd_stride, S, h->B, f.S, ds));
        }
        // unwrap, de-rotation, LLRs and counting in one pass over y (no z);
        // with the learned demapper the pass writes the symbols instead
        if (derot_demap_ctas(e - a, S, avail) > h->cap_pd || (e - a + 255) / 256 > h->cap_pd)
            return fail(RX_EINVAL, "internal: demap partials");
        STAGE(ST_DEMAP, ds, 1,
              launch_derot_demap(h->y, N, h->bidx + a, N, a, e, dsum_n, mdsum_n, bps_cta_range(chunks),
                                 carry_base + 2 * cin, (int)sd_stride, carry_base + 2 * cout, (int)sd_stride,
                                 h->pcode + a, N, h->sigma2_fixed > 0 ? h->sig_fixed : nullptr, h->sig, 1,
                                 h->mlp ? nullptr : llr + (size_t)a * m, N * m, cnt, sym, S, f, ds, h->prec,
                                 avail));
        if (h->mlp) {
            // every stream's symbols of the block in one launch (tcgen05 path)
            STAGE(ST_DEMAP, ds, h->mlp->d.infer == 2 ? 1 : S,
                  mlp_infer_seg(h->mlp->d, sym.x4 + (size_t)a * 4, sym.s2 + a, e - a, S, N, llr + (size_t)a * m, N,
                                ds));
            STAGE(ST_DEMAP, ds, 1,
                  launch_count_llr(llr + (size_t)a * m, N * m, sym.x4, N, a, e, h->sig, 1, cnt, S, f, ds));
        }
        CK(rec(h->ev_dm[par], ds));
        if (blk0) {
            cudaEvent_t blk1 = prof_event(h);
            if (blk1) { CK(cudaEventRecord(blk1, ds)); h->blk.push_back({blk0, blk1}); }
        }
        const long span = std::max(0L, std::min((long)h->n_upd, N - k0));
        // the LMS of block n reads the phase codes its demap wrote
        CK(rec(h->ev_unwrap, ds));
        cudaStream_t ls = st;
        if (L >= 2 && !one) {
            const int r = (int)(g % chains);
            ls = r == 0 ? side : h->side_x[r - 1];
            CK(wt(ls, h->ev_unwrap));
        } else {
            CK(wt(st, h->ev_unwrap));
        }
        // the update starts from U_{n-1} (one chain) or from W_n = U_{n-lag}
        const float2 *u_in = slot(h, chains > 1 ? g - L : g - 1);
        if (h->lms_block > 1)
            STAGE(ST_LMS, ls, span > 0 ? 1 : 0,
                  launch_lms_block(h->x, ns, u_in, slot(h, g), k0, (int)span, h->pcode, N, 2, h->u,
                                   (int)h->n_cma, (float)h->mu, h->lms_block, S, T, f, ls, h->prec, h->wl));
        else
            STAGE(ST_LMS, ls, span > 0 ? 1 : 0,
                  launch_lms(h->x, ns, u_in, slot(h, g), k0, (int)span, h->pcode, N, 2, 1,
                             h->u, (int)h->n_cma, (float)h->mu, nullptr, 0, S, T, f, ls, h->prec, lms_opts(h)));
        if (L >= 2) CK(rec(h->ev_lms[g % R], ls));
        h->u += span;
        h->blocks_done = g + 1;
    }
    // the caller's stream sees the demaps (LLRs, counters, carries) done
    if (join && b1 > b0) CK(wt(st, h->ev_dm[(int)((b1 - 1 + G) & 1)]));
    if (join && L >= 2)
        for (long n = std::max(b0, b1 - chains); n < b1; ++n) CK(wt(st, h->ev_lms[(n + G) % R]));
    return RX_OK;
}

int fill_stats(rx_handle *h, rx_stats *out) {
    const int S = h->streams;
    std::vector<StreamDev> sd(S);
    CK(cudaStreamSynchronize(h->st));
    if (use_bps_tc(h)) {
        unsigned int gave_up = 0;
        CK(bps_tc_status(&gave_up));
        if (gave_up) return fail(RX_ETIMEDOUT, "a bounded wait of the tensor-core phase search gave up");
    }
    if (h->fir_tma) {
        unsigned int gave_up = 0;
        CK(fir_tma_status(&gave_up));
        if (gave_up) return fail(RX_ETIMEDOUT, "a bounded wait of the TMA-staged FIR gave up");
    }
    if (h->mlp) {
        unsigned int gave_up = 0;
        CK(mlp_tc_status(&gave_up));
        if (gave_up) return fail(RX_ETIMEDOUT, "a bounded wait of the MLP's tensor-core kernels gave up");
    }
    // before the first block of a handle there are no device counters yet
    if (h->sd) CK(cudaMemcpy(sd.data(), h->sd, sizeof(StreamDev) * S, cudaMemcpyDeviceToHost));
    else std::memset(sd.data(), 0, sizeof(StreamDev) * S);
    for (int s = 0; s < S; ++s) {
        rx_stats &o = out[s];
        std::memset(&o, 0, sizeof o);
        o.n_sym = sd[s].n_sym;
        o.n_bits = sd[s].n_sym * (uint64_t)h->fmt.m;
        o.bit_errors = sd[s].bit_errors;
        o.gmi_sum = sd[s].gmi_sum;
        o.gmi = o.n_sym ? h->fmt.m - o.gmi_sum / (double)o.n_sym : 0.0;
        o.ber = o.n_bits ? (double)o.bit_errors / (double)o.n_bits : 0.0;
        o.evm_num = sd[s].evm_num;
        o.evm_den = sd[s].evm_den;
        o.sigma2_last = sd[s].sigma2;
        o.n_out = (uint64_t)h->cur_n;
        o.blocks = (uint32_t)h->blocks_done;
    }
    return RX_OK;
}

// ---------------------------------------------------------------------------
// streaming entry (rx_push / rx_flush): Sec. 2 processes the ADC's DMA
// buffers one after another, the taps learned on one buffer serving later
// ones.  The stream is held in a window of the handle's buffers; blocks run
// as soon as the samples their CDC frames read are in, and LLR rows leave
// with a fixed delay.
// ---------------------------------------------------------------------------
long cdc_hop(const rx_handle *h) { return h->n_fft - h->n_ov; }

// Input samples per polarisation that blocks 0 .. n of a stream read (their
// CDC frames and the start-up's): frame f reads samples f*hop - n_ov/2 ..
// f*hop + hop + n_ov/2 - 1, and block n's FIR / LMS outputs k < (n+1)*block
// read CDC outputs up to 2k + D.
long need_samples(const rx_handle *h, long n) {
    const long Sk = cdc_hop(h), D = (h->T - 1) / 2;
    const long k_hi = (n + 1) * h->block;
    const long k_st = std::max(h->n_pre, h->n_train);
    const long f1 = (2 * std::max(k_hi, k_st) + D + Sk - 1) / Sk;
    return f1 * Sk + h->n_ov / 2;
}

long gcd_l(long a, long b) {
    while (b) {
        const long t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Origin step, fixed delay and window length of the streaming entry.
void push_geometry(rx_handle *h) {
    auto &P = h->push;
    const long Nb = h->block, Sk = cdc_hop(h), W2 = h->W / 2, D = (h->T - 1) / 2;
    // the window's origin moves in whole blocks that are also whole CDC hops
    // (2 origin a multiple of hop), so blocks and frames fall as in the stream
    const long per = Sk / gcd_l(2 * Nb, Sk);
    P.step = per * Nb;
    // With tot samples in, blocks 0 .. n-1 have run exactly when
    // need(n-1) <= tot < need(n); their LLRs cover symbols < C(n) =
    // n*block - W/2 (C(0) = 0).  Output row r = tot/2 - 1 holds symbol
    // r - d, so every row handed out is computed when d >= (need(n) - 1)/2
    // - C(n) for all n.  The pattern repeats every `per` blocks once the
    // start-up span is passed.
    const long st_blocks = (std::max(h->n_pre, h->n_train) + Nb - 1) / Nb;
    long d = 0;
    for (long n = 0; n <= per + st_blocks + 2; ++n) {
        const long C = n == 0 ? 0 : n * Nb - W2;
        d = std::max(d, (need_samples(h, n) - 1) / 2 - C);
    }
    P.delay = d;
    // appended at most one block of symbols at a time; after each piece the
    // window keeps the symbols from min((nb-1) block, the first CDC frame of
    // block nb, the first row not yet handed out) rounded down to the step:
    // less than step + max(2 block + 2 hop + n_ov + 2 D + W, d) symbols
    P.piece = 2 * Nb;
    const long cap = std::max(std::max(P.step + 3 * Nb + 2 * Sk + h->n_ov + 2 * D + h->W + 64,
                                       (need_samples(h, 0) + 1) / 2 + Nb + 64),
                              d + P.step + Nb + 64);
    P.cap = (cap + 255) / 256 * 256;
}

int push_alloc(rx_handle *h) {
    auto &P = h->push;
    const int S = h->streams, m = h->fmt.m;
    const size_t in_b = sizeof(float2) * (size_t)S * 2 * 2 * P.cap;
    const size_t llr_b = sizeof(float) * (size_t)S * P.cap * m;
    const size_t halo_b = store_bytes(h->prec) * (size_t)S * 2 * h->W;
    if (P.in_bytes < in_b) {
        for (auto &b : P.in) { cudaFree(b); b = nullptr; }
        P.in_bytes = 0;
        for (auto &b : P.in) CK(cudaMalloc(&b, in_b));
        P.in_bytes = in_b;
    }
    if (P.llr_bytes < llr_b) {
        for (auto &b : P.llr) { cudaFree(b); b = nullptr; }
        P.llr_bytes = 0;
        for (auto &b : P.llr) CK(cudaMalloc(&b, llr_b));
        P.llr_bytes = llr_b;
    }
    if (P.halo_bytes < halo_b) {
        cudaFree(P.halo);
        P.halo = nullptr;
        P.halo_bytes = 0;
        CK(cudaMalloc(&P.halo, halo_b));
        P.halo_bytes = halo_b;
    }
    return RX_OK;
}

void push_free(rx_handle *h) {
    auto &P = h->push;
    for (auto &b : P.in) { cudaFree(b); b = nullptr; }
    for (auto &b : P.llr) { cudaFree(b); b = nullptr; }
    cudaFree(P.halo);
    P.halo = nullptr;
    P.in_bytes = P.llr_bytes = P.halo_bytes = 0;
}

Window push_window(const rx_handle *h) {
    Window w;
    w.origin = h->push.origin;
    w.bofs = h->push.origin / h->block;
    // counting over the stream's symbols skip_head .. ref_n - skip_tail - 1:
    // the reference covers the stream, whose end is not known before rx_flush
    w.c0 = h->skip_head;
    w.c1 = (long)h->ref_n - h->skip_tail;
    return w;
}

// symbols whose LLRs are computed (global): those of blocks 0 .. nb-1
long push_done(const rx_handle *h) { return h->push.nb == 0 ? 0 : h->push.nb * h->block - h->W / 2; }

// Rows [row0, row0 + cnt) of the output (row r holds symbol r - d; rows
// r < d are zeros) into out, [S][out_rows][m], from row out_off on.
int push_emit(rx_handle *h, float *out, long out_rows, long out_off, long row0, long cnt) {
    auto &P = h->push;
    const int S = h->streams, m = h->fmt.m;
    const size_t rb = sizeof(float) * m;
    const long z = std::min(cnt, std::max(0L, P.delay - row0));
    if (z > 0) CK(cudaMemset2DAsync(out + (size_t)out_off * m, rb * out_rows, 0, rb * z, S, h->st));
    const long k0 = row0 + z - P.delay, k1 = row0 + cnt - P.delay;
    if (k1 > k0) {
        if (k0 < P.origin || k1 > push_done(h))
            return fail(RX_EINVAL, "internal: rows %ld .. %ld not in the stream window", k0, k1);
        CK(cudaMemcpy2DAsync(out + (size_t)(out_off + z) * m, rb * out_rows,
                             P.llr[P.cur] + (size_t)(k0 - P.origin) * m, rb * P.cap, rb * (k1 - k0), S,
                             cudaMemcpyDeviceToDevice, h->st));
    }
    return RX_OK;
}

// Run every block whose samples are in.
int push_run(rx_handle *h, bool fresh) {
    auto &P = h->push;
    long n1 = P.nb;
    while (need_samples(h, n1) <= P.tot) ++n1;
    if (n1 == P.nb) return RX_OK;
    const Window w = push_window(h);
    int rc = run_blocks(h, P.in[P.cur], P.cap, P.nb - w.bofs, n1 - w.bofs, P.llr[P.cur], fresh, true, &w);
    if (rc != RX_OK) return rc;
    P.nb = n1;
    return RX_OK;
}

// Move the window's origin forward as far as the next blocks, their CDC
// frames and the rows not yet handed out allow (a copy into the other
// buffer of each pair, and the phase-search halo of block nb).
int push_rebase(rx_handle *h) {
    auto &P = h->push;
    if (P.nb < 1) return RX_OK;
    const long Nb = h->block, Sk = cdc_hop(h), D = (h->T - 1) / 2;
    const long f0 = (2 * P.nb * Nb - D) / Sk;           // first CDC frame of block nb
    const long e0 = P.emitted - P.delay;                // first symbol not handed out
    const long lim = std::min(std::min((P.nb - 1) * Nb, (f0 - 1) * Sk / 2), e0);
    if (lim <= P.origin) return RX_OK;
    const long o = lim / P.step * P.step;
    if (o <= P.origin) return RX_OK;
    const long dl = o - P.origin;
    const int S = h->streams, m = h->fmt.m, nx = 1 - P.cur;
    const size_t ip = sizeof(float2) * 2 * P.cap, rb = sizeof(float) * m;
    const long keep = P.tot - 2 * o;
    if (keep > 0)
        CK(cudaMemcpy2DAsync(P.in[nx], ip, P.in[P.cur] + 2 * dl, ip, sizeof(float2) * keep, (size_t)2 * S,
                             cudaMemcpyDeviceToDevice, h->st));
    const long c = push_done(h), r0 = std::max(e0, o);
    if (c > r0)
        CK(cudaMemcpy2DAsync(P.llr[nx] + (size_t)(r0 - o) * m, rb * P.cap, P.llr[P.cur] + (size_t)(r0 - P.origin) * m,
                             rb * P.cap, rb * (c - r0), S, cudaMemcpyDeviceToDevice, h->st));
    // FIR output of symbols nb*block - W .. nb*block - 1 (the window moves by
    // at least one block >= W, so source and destination do not overlap)
    const size_t eb = store_bytes(h->prec);
    char *y = static_cast<char *>(h->y);
    const long ys = P.nb * Nb - P.origin - h->W, yd = P.nb * Nb - o - h->W;
    CK(cudaMemcpy2DAsync(y + eb * yd, eb * P.cap, y + eb * ys, eb * P.cap, eb * h->W, (size_t)2 * S,
                         cudaMemcpyDeviceToDevice, h->st));
    P.origin = o;
    P.cur = nx;
    return RX_OK;
}

// Append n samples per polarisation (columns col .. col+n-1 of src,
// [S][2][src_ns]), run what they complete, hand out n/2 rows.
int push_piece(rx_handle *h, const float2 *src, long src_ns, long col, long n, float *out, long out_rows,
               long out_off, bool fresh) {
    auto &P = h->push;
    const int S = h->streams;
    if (P.tot - 2 * P.origin + n > 2 * P.cap)
        return fail(RX_EINVAL, "internal: stream window of %ld symbols overflows", P.cap);
    const size_t ip = sizeof(float2) * 2 * P.cap;
    CK(cudaMemcpy2DAsync(P.in[P.cur] + (P.tot - 2 * P.origin), ip, src + col, sizeof(float2) * src_ns,
                         sizeof(float2) * n, (size_t)2 * S, cudaMemcpyDefault, h->st));
    P.tot += n;
    int rc;
    if ((rc = push_run(h, fresh)) != RX_OK) return rc;
    if ((rc = push_emit(h, out, out_rows, out_off, P.emitted, n / 2)) != RX_OK) return rc;
    P.emitted += n / 2;
    return push_rebase(h);
}

int push_begin(rx_handle *h) {
    auto &P = h->push;
    if (P.on) return RX_OK;
    if (h->user_x4 || h->user_s2) return fail(RX_EINVAL, "symbol outputs are not available when streaming");
    P.tot = P.origin = P.nb = P.emitted = 0;
    P.cur = 0;
    push_geometry(h);
    int rc = push_alloc(h);
    if (rc != RX_OK) return rc;
    h->started = false;
    P.on = true;
    return RX_OK;
}

int push_stats(rx_handle *h, rx_stats *stats, long first_valid) {
    int rc = fill_stats(h, stats);
    if (rc != RX_OK) return rc;
    const long valid = std::max(0L, h->push.emitted - h->push.delay);
    for (int s = 0; s < h->streams; ++s) {
        stats[s].n_out = (uint64_t)valid;
        stats[s].first_valid = (uint64_t)first_valid;
    }
    return RX_OK;
}

int set_param_impl(rx_handle *h, const std::string &k, double v) {
    auto as_int = [&](long lo, long hi, long &dst) -> int {
        if (v != std::floor(v) || v < lo || v > hi) return fail(RX_EINVAL, "%s out of range", k.c_str());
        dst = (long)v;
        return RX_OK;
    };
    long t = 0;
    int rc = RX_OK;
    if (k == "fft") { rc = as_int(1024, 4096, t); h->n_fft = (int)t; h->tables_dirty = true; }
    else if (k == "overlap") { rc = as_int(2, 4094, t); h->n_ov = (int)t; }
    else if (k == "mu") { if (!(v > 0 && v < 1)) return fail(RX_EINVAL, "mu out of range"); h->mu = v; }
    else if (k == "bps_window") { rc = as_int(2, 64, t); h->W = (int)t; }
    else if (k == "block") { rc = as_int(64, 1L << 30, t); h->block = t; }
    else if (k == "n_upd") { rc = as_int(0, 1L << 30, t); h->n_upd = (int)t; }
    else if (k == "lag") { rc = as_int(1, 4, t); h->lag = (int)t; }
    else if (k == "n_pre") { rc = as_int(0, 1L << 30, t); h->n_pre = t; }
    else if (k == "cma_passes") { rc = as_int(0, 16, t); h->cma_passes = (int)t; }
    else if (k == "n_cma") { rc = as_int(0, 1L << 40, t); h->n_cma = t; }
    else if (k == "lms_block") { rc = as_int(1, 64, t); h->lms_block = (int)t; }
    else if (k == "lms_start") { rc = as_int(0, 1, t); h->lms_start = (int)t; }
    else if (k == "widely_linear") { rc = as_int(0, 1, t); h->wl = (int)t; h->started = false; }
    else if (k == "n_train") { rc = as_int(0, 20000, t); h->n_train = t; }
    else if (k == "train_passes") { rc = as_int(0, 64, t); h->train_passes = (int)t; }
    else if (k == "sigma2") { if (!(v >= 0)) return fail(RX_EINVAL, "sigma2 < 0"); h->sigma2_fixed = v; }
    else if (k == "skip_head") { rc = as_int(0, 1L << 40, t); h->skip_head = t; }
    else if (k == "skip_tail") { rc = as_int(0, 1L << 40, t); h->skip_tail = t; }
    else if (k == "streams") { rc = as_int(1, 4096, t); h->streams = (int)t; }
    else if (k == "rolloff") { if (!(v > 0 && v <= 1)) return fail(RX_EINVAL, "rolloff out of range"); h->rolloff = v; h->tables_dirty = true; }
    else if (k == "cd_ps_per_nm") { if (!std::isfinite(v)) return fail(RX_EINVAL, "cd_ps_per_nm must be finite"); h->cd = v; h->tables_dirty = true; }
    else if (k == "matched_filter") { if (v != 0 && v != 1) return fail(RX_EINVAL, "matched_filter is 0 or 1"); h->matched_filter = v != 0; h->tables_dirty = true; }
    else if (k == "wavelength_nm") { if (!(v > 100 && v < 10000)) return fail(RX_EINVAL, "wavelength out of range"); h->wavelength = v * 1e-9; h->tables_dirty = true; }
    else if (k == "profile") { rc = as_int(0, 2, t); h->profile = (int)t; }
    else if (k == "precision") { rc = as_int(0, 2, t); h->prec = (int)t; }
    else if (k == "bps_tc") { rc = as_int(0, 1, t); h->bps_tc = (int)t; }
    else if (k == "lms_exact") { rc = as_int(0, 1, t); h->lms_exact = (int)t; }
    else if (k == "sm_reserve") { rc = as_int(0, 1024, t); h->sm_reserve = (int)t; }
    else if (k == "fir_tma") { rc = as_int(0, 1, t); h->fir_tma = (int)t; }
    else if (k == "issue") {
        rc = as_int(0, 2, t);
        h->issue = (int)t;
        if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    }
    else return fail(RX_EINVAL, "unknown parameter '%s'", k.c_str());
    if (rc != RX_OK) return rc;
    if (k == "overlap") h->tables_dirty = true;
    h->started = false;
    h->push.on = false;
    return check_config(h);
}

// ---------------------------------------------------------------------------
// Scratch of rx_unwrap_static, which allocates no device memory: one static
// device array shared by every call in the process (per device).  Layout per
// call: S tickets (uint32), then S x n_blocks unwrap increments (int32), then
// S x n_blocks noise partial sums (float64), each region 256-byte aligned.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = 64 * 1024;
static __device__ __align__(256) unsigned char g_unwrap_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};   // device address of g_unwrap_scratch per device
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device.  The first call
// on a device looks it up with that device current (host code cannot use the
// array's name as a device address).
int static_scratch(void **out) {
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(RX_EINVAL, "device %d beyond the %d supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_unwrap_scratch);
        if (e != cudaSuccess || !p)
            return fail(RX_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return RX_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

static_assert(sizeof(rx_state_header) == 64 && sizeof(rx_state_counters) == 48,
              "the state layout is part of the ABI");

// Byte offsets of the parts of a state buffer (layout documented with
// rx_state_header): header, taps, carry, y halo, counters, packed.
struct StateLayout {
    size_t taps, carry, y_tail, counters, total;
};

StateLayout state_layout(const rx_handle *h) {
    const size_t S = (size_t)h->streams;
    StateLayout l{};
    l.taps = sizeof(rx_state_header);
    l.carry = l.taps + (size_t)h->lag * S * 4 * tl(h) * sizeof(float2);
    l.y_tail = l.carry + S * 2 * sizeof(int32_t);
    l.counters = l.y_tail + S * 2 * (size_t)h->W * sizeof(float2);
    l.total = l.counters + S * sizeof(rx_state_counters);
    return l;
}

}  // namespace

// ===========================================================================
// exported
// ===========================================================================
extern "C" {

const char *rx_last_error(void) { return g_err.c_str(); }

rx_handle *rx_create(const rx_format *format, double symbol_rate, int sps, double cd_ps_per_nm,
                     int taps, int bps_phases) {
    if (!format) { fail(RX_EINVAL, "format is NULL"); return nullptr; }
    if (!(symbol_rate > 0)) { fail(RX_EINVAL, "symbol_rate must be > 0"); return nullptr; }
    rx_handle *h = new rx_handle();
    if (build_format(format, h->fmt) != RX_OK) { delete h; return nullptr; }
    h->symbol_rate = symbol_rate;
    h->sps = sps;
    h->cd = cd_ps_per_nm;
    h->T = taps;
    h->B = bps_phases;
    if (check_config(h) != RX_OK) { delete h; return nullptr; }
    set_phases(h->fmt, bps_phases);
    if (h->fmt.n_orb > (h->fmt.dims == 2 ? 32 : 16)) {
        fail(RX_EINVAL, "phase search needs at most 16 (4D) / 32 (2D) orbits (use sym_order 4)");
        delete h;
        return nullptr;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        fail(RX_ECUDA, "no CUDA device");
        delete h;
        return nullptr;
    }
    return h;
}

void rx_destroy(rx_handle *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->gst) cudaStreamDestroy(h->gst);
    if (h->side) { cudaStreamSynchronize(h->side); cudaStreamDestroy(h->side); }
    for (auto &x : h->side_x)
        if (x) { cudaStreamSynchronize(x); cudaStreamDestroy(x); }
    if (h->cp_in) { cudaStreamSynchronize(h->cp_in); cudaStreamDestroy(h->cp_in); }
    if (h->cp_out) { cudaStreamSynchronize(h->cp_out); cudaStreamDestroy(h->cp_out); }
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->ev_in_rest) cudaEventDestroy(h->ev_in_rest);
    if (h->cst) { cudaStreamSynchronize(h->cst); cudaStreamDestroy(h->cst); }
    if (h->ev_cdcg) cudaEventDestroy(h->ev_cdcg);
    if (h->ev_unwrap) cudaEventDestroy(h->ev_unwrap);
    if (h->ev_cdc0) cudaEventDestroy(h->ev_cdc0);
    if (h->ev_start) cudaEventDestroy(h->ev_start);
    if (h->dst) { cudaStreamSynchronize(h->dst); cudaStreamDestroy(h->dst); }
    for (int i = 0; i < 2; ++i) {
        if (h->ev_bps[i]) cudaEventDestroy(h->ev_bps[i]);
        if (h->ev_dm[i]) cudaEventDestroy(h->ev_dm[i]);
    }
    if (h->ev_setup) cudaEventDestroy(h->ev_setup);
    for (auto e : h->ev_lms) cudaEventDestroy(e);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    free_buffers(h);
    push_free(h);
    cudaFree(h->x4);
    cudaFree(h->s2sym);
    cudaFree(h->H);
    cudaFree(h->tw);
    cudaFree(h->Hmag);
    if (h->ev_tab) cudaEventDestroy(h->ev_tab);
    cudaFree(h->bps_w);
    cudaFree(h->ref);
    cudaFree(h->d_in);
    cudaFree(h->d_out);
    cudaFree(h->ytr);
    cudaFree(h->ref_bits);
    if (h->h_in) cudaFreeHost(h->h_in);
    if (h->h_out) cudaFreeHost(h->h_out);
    delete h;
}

int rx_set_param(rx_handle *h, const char *key, double value) {
    if (!h || !key) return fail(RX_EINVAL, "NULL argument");
    return set_param_impl(h, key, value);
}

int rx_get_param(const rx_handle *h, const char *key, double *value) {
    if (!h || !key || !value) return fail(RX_EINVAL, "NULL argument");
    const std::string k = key;
    if (k == "fft") *value = h->n_fft;
    else if (k == "overlap") *value = h->n_ov;
    else if (k == "mu") *value = h->mu;
    else if (k == "bps_window") *value = h->W;
    else if (k == "block") *value = (double)h->block;
    else if (k == "n_upd") *value = h->n_upd;
    else if (k == "lag") *value = h->lag;
    else if (k == "n_pre") *value = (double)h->n_pre;
    else if (k == "cma_passes") *value = h->cma_passes;
    else if (k == "n_cma") *value = (double)h->n_cma;
    else if (k == "lms_block") *value = h->lms_block;
    else if (k == "lms_start") *value = h->lms_start;
    else if (k == "widely_linear") *value = h->wl;
    else if (k == "n_train") *value = (double)h->n_train;
    else if (k == "train_passes") *value = h->train_passes;
    else if (k == "sigma2") *value = h->sigma2_fixed;
    else if (k == "skip_head") *value = (double)h->skip_head;
    else if (k == "skip_tail") *value = (double)h->skip_tail;
    else if (k == "streams") *value = h->streams;
    else if (k == "rolloff") *value = h->rolloff;
    else if (k == "matched_filter") *value = h->matched_filter ? 1.0 : 0.0;
    else if (k == "wavelength_nm") *value = h->wavelength * 1e9;
    else if (k == "taps") *value = h->T;
    else if (k == "bps_phases") *value = h->B;
    else if (k == "bps_tc") *value = use_bps_tc(h) ? 1.0 : 0.0;
    else if (k == "lms_exact") *value = h->lms_exact;
    else if (k == "sm_reserve") *value = h->sm_reserve;
    else if (k == "issue") *value = h->issue;
    else if (k == "fir_tma") *value = h->fir_tma;
    else if (k == "cd_ps_per_nm") *value = h->cd;
    else if (k == "profile") *value = h->profile;
    else if (k == "precision") *value = h->prec;
    else return fail(RX_EINVAL, "unknown parameter '%s'", key);
    return RX_OK;
}

int rx_set_stream(rx_handle *h, void *cuda_stream) {
    if (!h) return fail(RX_EINVAL, "NULL handle");
    h->st = (cudaStream_t)cuda_stream;
    return RX_OK;
}

rx_mlp *rx_mlp_create(const float *params) {
    rx_mlp *m = new rx_mlp();
    cudaError_t e = mlp_alloc(m->d);
    if (e != cudaSuccess) {
        fail(RX_ENOMEM, "rx_mlp_create: %s", cudaGetErrorString(e));
        mlp_free(m->d);
        delete m;
        return nullptr;
    }
    if (params && rx_mlp_set_params(m, params) != RX_OK) {
        mlp_free(m->d);
        delete m;
        return nullptr;
    }
    if (!params && mlp_quantize(m->d, m->st) != cudaSuccess) {
        fail(RX_ECUDA, "rx_mlp_create: weight copies");
        mlp_free(m->d);
        delete m;
        return nullptr;
    }
    return m;
}

void rx_mlp_destroy(rx_mlp *m) {
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    else cudaDeviceSynchronize();
    mlp_free(m->d);
    delete m;
}

int rx_mlp_set_stream(rx_mlp *m, void *cuda_stream) {
    if (!m) return fail(RX_EINVAL, "NULL handle");
    m->st = (cudaStream_t)cuda_stream;
    return RX_OK;
}

int rx_mlp_get_params(rx_mlp *m, float *params) {
    if (!m || !params) return fail(RX_EINVAL, "NULL argument");
    CK(cudaStreamSynchronize(m->st));
    unsigned int gave_up = 0;
    CK(mlp_tc_status(&gave_up));
    if (gave_up) return fail(RX_ETIMEDOUT, "a bounded wait of the MLP's tensor-core kernels gave up");
    CK(cudaMemcpy(params, m->d.theta, sizeof(float) * RX_MLP_PARAMS, cudaMemcpyDeviceToHost));
    return RX_OK;
}

int rx_mlp_set_params(rx_mlp *m, const float *params) {
    if (!m || !params) return fail(RX_EINVAL, "NULL argument");
    CK(cudaStreamSynchronize(m->st));
    CK(cudaMemcpy(m->d.theta, params, sizeof(float) * RX_MLP_PARAMS, cudaMemcpyHostToDevice));
    CK(cudaMemset(m->d.m, 0, sizeof(float) * RX_MLP_PARAMS));
    CK(cudaMemset(m->d.v, 0, sizeof(float) * RX_MLP_PARAMS));
    m->t = 0;
    CK(mlp_quantize(m->d, m->st));
    CK(cudaStreamSynchronize(m->st));
    return RX_OK;
}

int rx_mlp_set_param(rx_mlp *m, const char *key, double value) {
    if (!m || !key) return fail(RX_EINVAL, "NULL argument");
    const std::string k(key);
    if (k == "train_tc") {
        if (value != 0.0 && value != 1.0) return fail(RX_EINVAL, "train_tc must be 0 or 1");
        m->d.train_tc = (int)value;
    } else if (k == "infer") {
        if (value != 1.0 && value != 2.0) return fail(RX_EINVAL, "infer must be 1 or 2");
        m->d.infer = (int)value;
    } else {
        return fail(RX_EINVAL, "unknown MLP parameter '%s'", key);
    }
    return RX_OK;
}

int rx_mlp_get_param(const rx_mlp *m, const char *key, double *value) {
    if (!m || !key || !value) return fail(RX_EINVAL, "NULL argument");
    const std::string k(key);
    if (k == "train_tc") *value = m->d.train_tc;
    else if (k == "infer") *value = m->d.infer;
    else return fail(RX_EINVAL, "unknown MLP parameter '%s'", key);
    return RX_OK;
}

int rx_mlp_grad(rx_mlp *m, const float *x, const float *sigma2, const uint8_t *bits, size_t n, float *grad,
                float *loss) {
    if (!m || !x || !sigma2 || !bits || !grad) return fail(RX_EINVAL, "NULL argument");
    if (n == 0 || n > (1u << 26)) return fail(RX_EINVAL, "batch of %zu samples (1 .. 2^26)", n);
    CK(mlp_grad(m->d, x, sigma2, bits, (long)n, loss, m->st));
    CK(cudaMemcpyAsync(grad, m->d.grad, sizeof(float) * RX_MLP_PARAMS, cudaMemcpyDeviceToDevice, m->st));
    return RX_OK;
}

int rx_mlp_train_step(rx_mlp *m, const float *x, const float *sigma2, const uint8_t *bits, size_t n, float lr,
                      float *loss) {
    if (!m || !x || !sigma2 || !bits) return fail(RX_EINVAL, "NULL argument");
    if (n == 0 || n > (1u << 26)) return fail(RX_EINVAL, "batch of %zu samples (1 .. 2^26)", n);
    if (!(lr > 0.f)) return fail(RX_EINVAL, "learning rate must be > 0");
    CK(mlp_grad(m->d, x, sigma2, bits, (long)n, loss, m->st));
    CK(mlp_adam(m->d, ++m->t, lr, m->st));
    return RX_OK;
}

int rx_mlp_infer(rx_mlp *m, const float *x, const float *sigma2, size_t n, float *llr) {
    if (!m || !x || !sigma2 || !llr) return fail(RX_EINVAL, "NULL argument");
    if (n == 0) return RX_OK;
    if (n > (1u << 26)) return fail(RX_EINVAL, "%zu samples (at most 2^26 per call)", n);
    CK(mlp_infer(m->d, x, sigma2, (long)n, llr, m->st));
    return RX_OK;
}

int rx_set_demapper(rx_handle *h, rx_mlp *m) {
    if (!h) return fail(RX_EINVAL, "NULL handle");
    if (m && !(h->fmt.dims == 4 && h->fmt.m == 6))
        return fail(RX_EINVAL, "the learned demapper maps 4D symbols to 6 bits (a 64-point 4D table)");
    h->mlp = m;
    return RX_OK;
}

int rx_set_symbol_output(rx_handle *h, float *x4, float *sigma2) {
    if (!h) return fail(RX_EINVAL, "NULL handle");
    h->user_x4 = x4;
    h->user_s2 = sigma2;
    return RX_OK;
}

int rx_format_info(const rx_handle *h, int *dims, int *m, int *M) {
    if (!h) return fail(RX_EINVAL, "NULL handle");
    if (dims) *dims = h->fmt.dims;
    if (m) *m = h->fmt.m;
    if (M) *M = h->fmt.M;
    return RX_OK;
}

int rx_set_reference(rx_handle *h, const uint8_t *bits, size_t n_sym) {
    if (!h || (!bits && n_sym)) return fail(RX_EINVAL, "NULL argument");
    const int S = h->streams;
    // the label buffer is kept while it is large enough (no free, which
    // would synchronise the device, when a handle is reused)
    if (h->ref && h->ref_cap < (size_t)S * n_sym) { cudaFree(h->ref); h->ref = nullptr; h->ref_cap = 0; }
    h->ref_n = (long)n_sym;
    h->ref_s = S;
    h->ref_host = nullptr;
    h->push.on = false;
    if (!n_sym) return RX_OK;
    if (!h->ref) { CK(cudaMalloc(&h->ref, sizeof(reflab_t) * (size_t)S * n_sym)); h->ref_cap = (size_t)S * n_sym; }
    CK(launch_ref_labels(bits, h->ref, (long)n_sym, S, h->fmt.m, h->fmt.dims, h->fmt.m_pol, h->st));
    h->started = false;
    return RX_OK;
}

int rx_set_reference_host(rx_handle *h, const uint8_t *bits, size_t n_sym) {
    if (!h || !bits || !n_sym) return fail(RX_EINVAL, "NULL argument");
    const int S = h->streams;
    if (h->ref && h->ref_cap < (size_t)S * n_sym) { cudaFree(h->ref); h->ref = nullptr; h->ref_cap = 0; }
    h->ref_n = (long)n_sym;
    h->ref_s = S;
    if (!h->ref) { CK(cudaMalloc(&h->ref, sizeof(reflab_t) * (size_t)S * n_sym)); h->ref_cap = (size_t)S * n_sym; }
    const size_t need = (size_t)S * n_sym * h->fmt.m;
    if (h->ref_bits_cap < need) {
        cudaFree(h->ref_bits);
        h->ref_bits = nullptr;
        CK(cudaMalloc(&h->ref_bits, need));
        h->ref_bits_cap = need;
    }
    h->ref_host = bits;
    h->started = false;
    h->push.on = false;
    return RX_OK;
}


int rx_reset(rx_handle *h) {
    if (!h) return fail(RX_EINVAL, "NULL handle");
    h->push.on = false;
    h->started = false;
    h->blocks_done = 0;
    h->u = 0;
    return RX_OK;
}

int rx_process(rx_handle *h, const void *samples, size_t n_samples, float *llr_out, rx_stats *stats) {
    if (!h || !samples || !llr_out) return fail(RX_EINVAL, "NULL argument");
    if (n_samples < 2 || (n_samples & 1)) return fail(RX_EINVAL, "n_samples must be a positive multiple of 2");
    const long N = (long)n_samples / 2;
    const long nblk = (N + h->block - 1) / h->block;
    h->push.on = false;
    int rc = run_blocks(h, (const float2 *)samples, N, 0, nblk, llr_out);
    if (rc != RX_OK) return rc;
    CK(cudaGetLastError());
    if (stats) return fill_stats(h, stats);
    return RX_OK;
}

int rx_stream_delay(rx_handle *h, size_t *delay) {
    if (!h || !delay) return fail(RX_EINVAL, "NULL argument");
    int rc = check_config(h);
    if (rc != RX_OK) return rc;
    if (!h->push.on) push_geometry(h);
    *delay = (size_t)h->push.delay;
    return RX_OK;
}

int rx_push(rx_handle *h, const void *samples, size_t n_samples, float *llr_out, rx_stats *stats) {
    if (!h) return fail(RX_EINVAL, "NULL handle");
    if (n_samples % 2) return fail(RX_EINVAL, "n_samples must be a multiple of 2 (sps)");
    if (n_samples && (!samples || !llr_out)) return fail(RX_EINVAL, "NULL argument");
    int rc = check_config(h);
    if (rc != RX_OK) return rc;
    if ((rc = push_begin(h)) != RX_OK) return rc;
    auto &P = h->push;
    const long n = (long)n_samples, rows = n / 2;
    const long first_valid = std::min(rows, std::max(0L, P.delay - P.emitted));
    for (long c = 0; c < n;) {
        const long piece = std::min(P.piece, n - c);
        if ((rc = push_piece(h, static_cast<const float2 *>(samples), n, c, piece, llr_out, rows, c / 2, c == 0)) !=
            RX_OK) {
            P.on = false;
            return rc;
        }
        c += piece;
    }
    CK(cudaGetLastError());
    if (stats) return push_stats(h, stats, first_valid);
    return RX_OK;
}

int rx_flush(rx_handle *h, float *llr_out, size_t *n_rows, rx_stats *stats) {
    if (!h || !n_rows) return fail(RX_EINVAL, "NULL argument");
    auto &P = h->push;
    if (!P.on) return fail(RX_ESTATE, "no stream is being pushed");
    const long N = P.tot / 2, e0 = std::max(0L, P.emitted - P.delay);
    const long rows = N - e0;
    if (rows > 0 && !llr_out) return fail(RX_EINVAL, "NULL llr_out");
    const int S = h->streams, m = h->fmt.m;
    const size_t rb = sizeof(float) * m;
    int rc;
    if (N > 0) {
        // rows computed before the flush go first
        const long c = push_done(h);
        long off = 0;
        if (c > e0) {
            CK(cudaMemcpy2DAsync(llr_out, rb * rows, P.llr[P.cur] + (size_t)(e0 - P.origin) * m, rb * P.cap,
                                 rb * (c - e0), S, cudaMemcpyDeviceToDevice, h->st));
            off = c - e0;
        }
        // the rest as the end of a stream of N - origin symbols in the
        // window (zeros after it, as in rx_process): the window's samples
        // and the phase-search halo laid out for that length
        const long Nf = N - P.origin, Nb = h->block;
        const int nx = 1 - P.cur;
        CK(cudaMemcpy2DAsync(P.in[nx], sizeof(float2) * 2 * Nf, P.in[P.cur], sizeof(float2) * 2 * P.cap,
                             sizeof(float2) * 2 * Nf, (size_t)2 * S, cudaMemcpyDeviceToDevice, h->st));
        if (P.nb > 0) {
            const size_t eb = store_bytes(h->prec);
            char *y = static_cast<char *>(h->y);
            const long col = P.nb * Nb - P.origin - h->W;
            CK(cudaMemcpy2DAsync(P.halo, eb * h->W, y + eb * col, eb * P.cap, eb * h->W, (size_t)2 * S,
                                 cudaMemcpyDeviceToDevice, h->st));
            CK(cudaMemcpy2DAsync(y + eb * col, eb * Nf, P.halo, eb * h->W, eb * h->W, (size_t)2 * S,
                                 cudaMemcpyDeviceToDevice, h->st));
        }
        const Window w = push_window(h);
        const long lb0 = P.nb - w.bofs, lb1 = (Nf + Nb - 1) / Nb;
        if ((rc = run_blocks(h, P.in[nx], Nf, lb0, lb1, P.llr[nx], true, true, &w)) != RX_OK) {
            P.on = false;
            return rc;
        }
        const long k0 = std::max(c, e0);
        if (N > k0)
            CK(cudaMemcpy2DAsync(llr_out + (size_t)off * m, rb * rows, P.llr[nx] + (size_t)(k0 - P.origin) * m,
                                 rb * Nf, rb * (N - k0), S, cudaMemcpyDeviceToDevice, h->st));
        P.nb = w.bofs + lb1;
    }
    P.emitted = N + P.delay;
    *n_rows = (size_t)std::max(0L, rows);
    CK(cudaGetLastError());
    rc = stats ? push_stats(h, stats, 0) : RX_OK;
    if (stats)
        for (int s = 0; s < S; ++s) stats[s].n_out = (uint64_t)N;
    P.on = false;
    return rc;
}

int rx_wait(rx_handle *h, double timeout_ms) {
    if (!h || !(timeout_ms >= 0)) return fail(RX_EINVAL, "NULL handle or negative timeout");
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaStreamQuery(h->st);
        if (e == cudaSuccess) return RX_OK;
        if (e != cudaErrorNotReady) return fail(RX_ECUDA, "rx_wait: %s", cudaGetErrorString(e));
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms >= timeout_ms) return fail(RX_ETIMEDOUT, "the handle's work did not finish within %.3f ms", timeout_ms);
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int rx_get_stats(rx_handle *h, rx_stats *stats) {
    if (!h || !stats) return fail(RX_EINVAL, "NULL argument");
    if (!h->sd) return fail(RX_ESTATE, "nothing processed yet");
    return fill_stats(h, stats);
}

int rx_process_host(rx_handle *h, const void *samples, size_t n_samples, float *llr_out, rx_stats *stats) {
    if (!h || !samples || !llr_out) return fail(RX_EINVAL, "NULL argument");
    if (n_samples < 2 || (n_samples & 1)) return fail(RX_EINVAL, "n_samples must be a positive multiple of 2");
    const int S = h->streams, m = h->fmt.m;
    const long N = (long)n_samples / 2, ns = (long)n_samples;
    h->push.on = false;
    const size_t in_b = sizeof(float2) * (size_t)S * 2 * n_samples;
    const size_t out_b = sizeof(float) * (size_t)S * N * m;
    if (h->d_in_cap < in_b) { cudaFree(h->d_in); h->d_in = nullptr; CK(cudaMalloc(&h->d_in, in_b)); h->d_in_cap = in_b; }
    if (h->d_out_cap < out_b) { cudaFree(h->d_out); h->d_out = nullptr; CK(cudaMalloc(&h->d_out, out_b)); h->d_out_cap = out_b; }
    if (!h->cp_in) {
        CK(cudaStreamCreateWithFlags(&h->cp_in, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->cp_out, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&h->ev_in_rest, cudaEventDisableTiming));
        CK(cudaStreamCreateWithFlags(&h->cst, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&h->ev_cdcg, cudaEventDisableTiming));
    }
    // the previous call's output copies and this call's device buffers
    CK(cudaEventRecord(h->ev_out, h->st));
    CK(cudaStreamWaitEvent(h->cp_in, h->ev_out, 0));
    // Groups of blocks: the input samples a group's CDC frames read go in on
    // one copy stream, its LLR rows come out on another, so both overlap the
    // chain of the neighbouring groups (with pinned host buffers the copies
    // are asynchronous).  Samples [S][2][n_samples] and LLRs [S][N][m] are
    // 2D regions: one row per stream and polarisation (stream).
    const long Nb = h->block, nblk = (N + Nb - 1) / Nb;
    const long Sk = h->n_fft - h->n_ov, half = h->n_ov / 2;
    const long G = 2;                         // blocks per group
    const size_t pin = sizeof(float2) * (size_t)ns, pout = sizeof(float) * (size_t)N * m;
    long copied = 0;                          // samples [0, copied) of every row are on the device
    long out_done = 0;                        // LLR rows [0, out_done) copied out
    long ref_done = 0;                        // reference rows [0, ref_done) copied in and labelled
    const uint8_t *rh = h->ref_host;
    h->ref_host = nullptr;                    // this call takes the reference in
    const size_t pref = (size_t)h->ref_n * m;
    const float2 *src = static_cast<const float2 *>(samples);
    // reference rows [ref_done, r_hi): bits in, then their labels, both on
    // the input copy stream so that the events below cover them
    auto ref_rows = [&](long r_hi) -> int {
        r_hi = std::min(r_hi, h->ref_n);
        if (!rh || r_hi <= ref_done) return RX_OK;
        CK(cudaMemcpy2DAsync(h->ref_bits + ref_done * m, pref, rh + ref_done * m, pref,
                             (size_t)((r_hi - ref_done) * m), (size_t)S, cudaMemcpyHostToDevice, h->cp_in));
        CK(launch_ref_labels_rows(h->ref_bits, h->ref, h->ref_n, ref_done, r_hi, S, m, h->cp_in));
        ref_done = r_hi;
        return RX_OK;
    };
    int rc;
    for (long g0 = 0; g0 < nblk; g0 += G) {
        const long g1 = std::min(nblk, g0 + G);
        const CdcFrames cf = cdc_frames(h, N, g0, g1);
        const long hi = std::min(ns, (cf.f1 - 1) * Sk - half + h->n_fft);
        if (g0 == 0 && cf.fs > cf.f0) {
            // the start-up's frames first: the start-up runs while the rest
            // of the first group comes in
            const long hs = std::min(hi, (cf.fs - 1) * Sk - half + h->n_fft);
            CK(cudaMemcpy2DAsync(h->d_in, pin, src, pin, sizeof(float2) * (size_t)hs, (size_t)(2 * S),
                                 cudaMemcpyHostToDevice, h->cp_in));
            if ((rc = ref_rows(std::min(N, h->n_train))) != RX_OK) return rc;
            CK(cudaEventRecord(h->ev_in, h->cp_in));
            copied = hs;
        }
        if (hi > copied) {
            CK(cudaMemcpy2DAsync(h->d_in + copied, pin, src + copied, pin, sizeof(float2) * (size_t)(hi - copied),
                                 (size_t)(2 * S), cudaMemcpyHostToDevice, h->cp_in));
            copied = hi;
        }
        // reference rows the group's blocks (and the training span) count with
        if ((rc = ref_rows(std::min(N, std::max(g1 * Nb, g0 == 0 ? h->n_train : 0L)))) != RX_OK) return rc;
        if (g0 == 0 && cf.fs > cf.f0) {
            CK(cudaEventRecord(h->ev_in_rest, h->cp_in));
            h->wait_rest = true;
        } else {
            CK(cudaEventRecord(h->ev_in, h->cp_in));
        }
        // the first group's kernels start after its input; later groups'
        // CDC waits for theirs on its own stream (run_blocks)
        if (g0 == 0) CK(cudaStreamWaitEvent(h->st, h->ev_in, 0));
        h->cdc_side = g0 > 0;
        h->in_host = true;
        rc = run_blocks(h, h->d_in, N, g0, g1, h->d_out, g0 == 0, g1 == nblk);
        h->in_host = false;
        h->cdc_side = false;
        h->wait_rest = false;
        if (rc != RX_OK) return rc;
        // block n writes rows [k0 - W/2, k1 - W/2) (the last block up to N)
        const long e = (g1 == nblk) ? N : std::min(N, g1 * Nb) - h->W / 2;
        // the group's LLR rows are final when its last demap is (demap stream)
        CK(cudaEventRecord(h->ev_out, h->dst));
        CK(cudaStreamWaitEvent(h->cp_out, h->ev_out, 0));
        if (e > out_done) {
            CK(cudaMemcpy2DAsync(llr_out + out_done * m, pout, h->d_out + out_done * m, pout,
                                 sizeof(float) * (size_t)((e - out_done) * m), (size_t)S,
                                 cudaMemcpyDeviceToHost, h->cp_out));
            out_done = e;
        }
    }
    CK(cudaEventRecord(h->ev_out, h->cp_out));
    CK(cudaStreamWaitEvent(h->st, h->ev_out, 0));
    if (stats) return fill_stats(h, stats);
    CK(cudaStreamSynchronize(h->st));
    return RX_OK;
}

int rx_get_profile(rx_handle *h, const char *stage, double *ms_total, uint64_t *launches) {
    if (!h || !stage) return fail(RX_EINVAL, "NULL argument");
    int id = -1;
    const std::string k = stage;
    if (k != "all") {
        for (int i = 0; i < ST_N; ++i)
            if (k == kStageNames[i]) id = i;
        if (id < 0) return fail(RX_EINVAL, "unknown stage '%s'", stage);
    }
    uint64_t nl = 0;
    for (int i = 0; i < ST_N; ++i)
        if (id < 0 || id == i) nl += h->nlaunch[i];
    if (launches) *launches = nl;
    if (ms_total) {
        *ms_total = 0.0;
        if (!h->recs.empty()) {
            CK(cudaDeviceSynchronize());
            for (const auto &r : h->recs) {
                if (id >= 0 && r.stage != id) continue;
                float ms = 0.f;
                CK(cudaEventElapsedTime(&ms, r.a, r.b));
                *ms_total += ms;
            }
        }
    }
    return RX_OK;
}

int rx_get_block_latency(rx_handle *h, double *ms, size_t cap, size_t *n) {
    if (!h || !n) return fail(RX_EINVAL, "NULL argument");
    *n = h->blk.size();
    if (!ms) return RX_OK;
    if (!h->blk.empty()) CK(cudaDeviceSynchronize());
    for (size_t i = 0; i < h->blk.size() && i < cap; ++i) {
        float v = 0.f;
        CK(cudaEventElapsedTime(&v, h->blk[i].first, h->blk[i].second));
        ms[i] = v;
    }
    return RX_OK;
}

int rx_process_blocks(rx_handle *h, const void *samples, size_t n_samples, size_t b0, size_t b1,
                      float *llr_out, rx_stats *stats) {
    if (!h || !samples || !llr_out) return fail(RX_EINVAL, "NULL argument");
    if (n_samples < 2 || (n_samples & 1)) return fail(RX_EINVAL, "n_samples must be a positive multiple of 2");
    const long N = (long)n_samples / 2;
    const long nblk = (N + h->block - 1) / h->block;
    if (b1 <= b0 || (long)b1 > nblk)
        return fail(RX_EINVAL, "block range [%zu, %zu) not inside the stream's %ld blocks", b0, b1, nblk);
    if (h->push.on) return fail(RX_ESTATE, "the handle is streaming (rx_push): rx_flush or rx_reset first");
    if (b0 > 0 && !(h->started && h->cur_n == N && h->blocks_done == (long)b0))
        return fail(RX_ESTATE, "block %zu does not continue the handle's stream (at block %ld of a %ld-symbol "
                    "stream%s)", b0, h->blocks_done, h->cur_n, h->started ? "" : ", not started");
    int rc;
    if (h->issue == 2 && b0 > 0 && !h->profile && !h->ref_host) {
        // the blocks as one CUDA graph: captured on a private stream (a
        // default stream cannot be captured), the instantiated graph of the
        // previous call updated in place (same topology: new kernel
        // arguments only) or instantiated anew, launched on the handle's stream
        if (!h->gst) CK(cudaStreamCreateWithFlags(&h->gst, cudaStreamNonBlocking));
        cudaGraph_t gr = nullptr;
        const cudaStream_t user = h->st;
        CK(cudaStreamBeginCapture(h->gst, cudaStreamCaptureModeThreadLocal));
        h->st = h->gst;
        rc = run_blocks(h, (const float2 *)samples, N, (long)b0, (long)b1, llr_out);
        h->st = user;
        const cudaError_t ce = cudaStreamEndCapture(h->gst, &gr);
        if (rc != RX_OK) {
            if (gr) cudaGraphDestroy(gr);
            return rc;
        }
        CK(ce);
        if (h->gexec) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(h->gexec, gr, &info) != cudaSuccess) {
                cudaGetLastError();
                cudaGraphExecDestroy(h->gexec);
                h->gexec = nullptr;
            }
        }
        const cudaError_t ie = h->gexec ? cudaSuccess : cudaGraphInstantiate(&h->gexec, gr, 0);
        cudaGraphDestroy(gr);
        CK(ie);
        CK(cudaGraphLaunch(h->gexec, h->st));
    } else {
        rc = run_blocks(h, (const float2 *)samples, N, (long)b0, (long)b1, llr_out);
        if (rc != RX_OK) return rc;
    }
    CK(cudaGetLastError());
    if (stats) return fill_stats(h, stats);
    return RX_OK;
}

int rx_get_state(rx_handle *h, void *buf, size_t *len) {
    if (!h || !len) return fail(RX_EINVAL, "NULL argument");
    if (h->push.on) return fail(RX_ESTATE, "the handle is streaming (rx_push): rx_flush or rx_reset first");
    if (h->prec != SK_F32) return fail(RX_EINVAL, "stream state is kept for float32 storage only (precision 0)");
    if (!h->started || h->blocks_done < 1) return fail(RX_ESTATE, "no block of a stream has run yet");
    const StateLayout lay = state_layout(h);
    if (!buf) { *len = lay.total; return RX_OK; }
    if (*len < lay.total) {
        *len = lay.total;
        return fail(RX_EINVAL, "state needs %zu bytes", lay.total);
    }
    const int S = h->streams, T = tl(h), L = h->lag, W = h->W;   // T: taps per branch
    const long n = h->blocks_done, N = h->cur_n, K = n * h->block;
    unsigned char *out = static_cast<unsigned char *>(buf);
    std::memset(out, 0, lay.total);
    CK(cudaStreamSynchronize(h->st));
    rx_state_header hd{};
    hd.magic = RX_STATE_MAGIC;
    hd.version = RX_STATE_VERSION;
    hd.streams = S; hd.taps = T; hd.lag = L; hd.bps_window = W; hd.bps_phases = h->B; hd.m_bits = h->fmt.m;
    hd.block = h->block; hd.n_sym = N; hd.blocks_done = n; hd.lms_updates = h->u;
    std::memcpy(out, &hd, sizeof hd);
    const size_t tapsz = sizeof(float2) * (size_t)S * 4 * T;
    for (int j = 0; j < L; ++j)
        CK(cudaMemcpy(out + lay.taps + j * tapsz, slot(h, n - L + j), tapsz, cudaMemcpyDeviceToHost));
    std::vector<StreamDev> sd(S);
    CK(cudaMemcpy(sd.data(), h->sd, sizeof(StreamDev) * S, cudaMemcpyDeviceToHost));
    int32_t *carry = reinterpret_cast<int32_t *>(out + lay.carry);
    rx_state_counters *cnt = reinterpret_cast<rx_state_counters *>(out + lay.counters);
    for (int s = 0; s < S; ++s) {
        carry[2 * s] = sd[s].carry[n & 1][0];
        carry[2 * s + 1] = sd[s].carry[n & 1][1];
        cnt[s].bit_errors = sd[s].bit_errors;
        cnt[s].n_sym = sd[s].n_sym;
        cnt[s].gmi_sum = sd[s].gmi_sum;
        cnt[s].evm_num = sd[s].evm_num;
        cnt[s].evm_den = sd[s].evm_den;
        cnt[s].sigma2 = sd[s].sigma2;
    }
    // y rows [S*2][N]; the halo is symbols K-W .. K-1 (zeros outside 0 .. N-1)
    const long lo = std::max(0L, K - W), hi = std::min(K, N), skip = lo - (K - W);
    if (hi > lo)
        CK(cudaMemcpy2D(out + lay.y_tail + sizeof(float2) * skip, sizeof(float2) * W, static_cast<float2 *>(h->y) + lo,
                        sizeof(float2) * N, sizeof(float2) * (hi - lo), (size_t)2 * S, cudaMemcpyDeviceToHost));
    *len = lay.total;
    return RX_OK;
}

int rx_set_state(rx_handle *h, const void *buf, size_t len) {
    if (!h || !buf) return fail(RX_EINVAL, "NULL argument");
    h->push.on = false;
    if (h->prec != SK_F32) return fail(RX_EINVAL, "stream state is kept for float32 storage only (precision 0)");
    if (len < sizeof(rx_state_header)) return fail(RX_EINVAL, "state of %zu bytes is shorter than its header", len);
    rx_state_header hd;
    std::memcpy(&hd, buf, sizeof hd);
    if (hd.magic != RX_STATE_MAGIC || hd.version != RX_STATE_VERSION)
        return fail(RX_EINVAL, "not a version-%u receiver state", RX_STATE_VERSION);
    if (hd.streams != h->streams || hd.taps != tl(h) || hd.lag != h->lag || hd.bps_window != h->W ||
        hd.bps_phases != h->B || hd.m_bits != h->fmt.m || hd.block != h->block)
        return fail(RX_EINVAL, "state (S %d, T %d, lag %d, W %d, B %d, m %d, block %lld) does not match the "
                    "handle (S %d, T %d, lag %d, W %d, B %d, m %d, block %ld)", hd.streams, hd.taps, hd.lag,
                    hd.bps_window, hd.bps_phases, hd.m_bits, (long long)hd.block, h->streams, tl(h), h->lag,
                    h->W, h->B, h->fmt.m, h->block);
    const long N = (long)hd.n_sym, n = (long)hd.blocks_done;
    const long nblk = N > 0 ? (N + h->block - 1) / h->block : 0;
    if (N <= 0 || n < 1 || n > nblk || hd.lms_updates < 0)
        return fail(RX_EINVAL, "state at block %lld of a %lld-symbol stream cannot be resumed",
                    (long long)n, (long long)N);
    const StateLayout lay = state_layout(h);
    if (len != lay.total) return fail(RX_EINVAL, "state has %zu bytes, expected %zu", len, lay.total);
    int rc;
    if ((rc = upload_tables(h)) != RX_OK) return rc;
    if ((rc = ensure_buffers(h, N)) != RX_OK) return rc;
    if ((rc = ensure_streams(h)) != RX_OK) return rc;
    const int S = h->streams, T = tl(h), L = h->lag, W = h->W;   // T: taps per branch
    const long K = n * h->block;
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    CK(cudaStreamSynchronize(h->st));
    if (h->side) CK(cudaStreamSynchronize(h->side));
    for (auto x : h->side_x)
        if (x) CK(cudaStreamSynchronize(x));
    const size_t tapsz = sizeof(float2) * (size_t)S * 4 * T;
    for (int j = 0; j < L; ++j)
        CK(cudaMemcpy(slot(h, n - L + j), in + lay.taps + j * tapsz, tapsz, cudaMemcpyHostToDevice));
    std::vector<StreamDev> sd(S);
    std::memset(sd.data(), 0, sizeof(StreamDev) * S);
    const int32_t *carry = reinterpret_cast<const int32_t *>(in + lay.carry);
    const rx_state_counters *cnt = reinterpret_cast<const rx_state_counters *>(in + lay.counters);
    for (int s = 0; s < S; ++s) {
        sd[s].carry[n & 1][0] = carry[2 * s];
        sd[s].carry[n & 1][1] = carry[2 * s + 1];
        sd[s].bit_errors = cnt[s].bit_errors;
        sd[s].n_sym = cnt[s].n_sym;
        sd[s].gmi_sum = cnt[s].gmi_sum;
        sd[s].evm_num = cnt[s].evm_num;
        sd[s].evm_den = cnt[s].evm_den;
        sd[s].sigma2 = cnt[s].sigma2;
    }
    CK(cudaMemcpy(h->sd, sd.data(), sizeof(StreamDev) * S, cudaMemcpyHostToDevice));
    const long lo = std::max(0L, K - W), hi = std::min(K, N), skip = lo - (K - W);
    if (hi > lo)
        CK(cudaMemcpy2D(static_cast<float2 *>(h->y) + lo, sizeof(float2) * N, in + lay.y_tail + sizeof(float2) * skip,
                        sizeof(float2) * W, sizeof(float2) * (hi - lo), (size_t)2 * S, cudaMemcpyHostToDevice));
    h->u = (long)hd.lms_updates;
    h->blocks_done = n;
    h->cur_n = N;
    h->trained = false;
    h->started = true;
    return RX_OK;
}

// ---- single stages ---------------------------------------------------------

int rx_cdc(rx_handle *h, const void *in, void *out, size_t n_samples) {
    if (!h || !in || !out) return fail(RX_EINVAL, "NULL argument");
    if (in == out) return fail(RX_EINVAL, "in and out must differ");
    int rc = upload_tables(h);
    if (rc != RX_OK) return rc;
    CK(launch_cdc((const float2 *)in, out, (long)n_samples, 2 * h->streams, h->n_fft,
                  h->n_ov, h->H, h->tw, h->st, 0, -1, h->prec));
    return RX_OK;
}

int rx_fir(rx_handle *h, const void *x, size_t n_samples, const void *taps, size_t k0, size_t k1, void *y) {
    if (!h || !x || !taps || !y) return fail(RX_EINVAL, "NULL argument");
    if (k1 < k0) return fail(RX_EINVAL, "k1 < k0");
    CK(launch_fir_ex(x, (long)n_samples, (const float2 *)taps, (long)k0, (long)k1,
                     y, (long)(k1 - k0), 0, h->streams, h->T, h->st, h->prec, 0, h->wl, h->fir_tma));
    return RX_OK;
}

int rx_lms(rx_handle *h, const void *x, size_t n_samples, void *taps, size_t k0, size_t n_upd,
           const uint16_t *pcode, int mode, int passes, uint64_t u0) {
    if (!h || !x || !taps) return fail(RX_EINVAL, "NULL argument");
    if (mode < 0 || mode > 3) return fail(RX_EINVAL, "mode must be 0, 1, 2 or 3");
    if (mode != 0 && !pcode) return fail(RX_EINVAL, "DD mode needs phase codes");
    if (mode == 3 && flush_ref(h) != RX_OK) return RX_ECUDA;
    if (mode == 3 && (!h->ref || h->ref_n < (long)(k0 + n_upd)))
        return fail(RX_ESTATE, "data-aided mode needs a reference covering the span");
    const long N = (long)n_samples / 2;
    if ((long)(k0 + n_upd) > N) return fail(RX_EINVAL, "update span beyond the stream");
    if (h->lms_block > 1 && mode != 3) {
        // block LMS (passes repeat the span)
        for (int pass = 0; pass < passes; ++pass)
            CK(launch_lms_block((const float2 *)x, (long)n_samples, (const float2 *)taps, (float2 *)taps,
                                (long)k0, (int)n_upd, pcode, N, mode, u0, (int)h->n_cma, (float)h->mu,
                                h->lms_block, h->streams, h->T, h->fmt, h->st, SK_F32, h->wl));
        return RX_OK;
    }
    CK(launch_lms((const float2 *)x, (long)n_samples, (const float2 *)taps, (float2 *)taps, (long)k0,
                  (int)n_upd, pcode, N, mode, passes, u0, (int)h->n_cma, (float)h->mu, h->ref,
                  h->ref_n, h->streams, h->T, h->fmt, h->st, SK_F32, lms_opts(h)));
    return RX_OK;
}

int rx_train(rx_handle *h, const void *x, size_t n_samples, void *taps, uint16_t *pcode) {
    if (!h || !x || !taps || !pcode) return fail(RX_EINVAL, "NULL argument");
    const long N = (long)n_samples / 2;
    const long ntr = std::min(h->n_train, N);
    if (!h->ref || h->ref_n < ntr) return fail(RX_ESTATE, "training needs a reference (rx_set_reference)");
    if (flush_ref(h) != RX_OK) return RX_ECUDA;
    return train_stage(h, x, (long)n_samples, (float2 *)taps, ntr, pcode, ntr, nullptr, 0, h->st, SK_F32);
}

int rx_bps(rx_handle *h, const void *y, size_t n_y, size_t a, size_t e, size_t n_valid, uint8_t *b_out) {
    if (!h || !y || !b_out) return fail(RX_EINVAL, "NULL argument");
    if (e < a || e > n_y || n_valid > n_y) return fail(RX_EINVAL, "bad range");
    int *dsum = nullptr;
    int rc = upload_tables(h);
    if (rc != RX_OK) return rc;
    const bool tc = use_bps_tc(h);
    const int chunks = tc ? bps_chunks_tc((long)(e - a), h->streams) : bps_chunks((long)(e - a), h->streams);
    const long ncta = ((long)(e - a) + bps_cta_range(chunks) - 1) / bps_cta_range(chunks);
    CK(cudaMallocAsync(&dsum, sizeof(int) * (size_t)h->streams * (ncta + 1), h->st));
    cudaError_t err = tc ? launch_bps_tc(y, (long)n_y, (long)a, (long)e, (long)n_valid, h->W, b_out, (long)(e - a), 0,
                                         dsum, nullptr, chunks, h->streams, h->bps_w, h->fmt, h->st)
                         : launch_bps((const float2 *)y, (long)n_y, (long)a, (long)e, (long)n_valid, h->W,
                                      b_out, (long)(e - a), 0, dsum, nullptr, chunks, h->streams, h->fmt, h->st);
    cudaFreeAsync(dsum, h->st);
    CK(err);
    return RX_OK;
}

int rx_unwrap(rx_handle *h, const void *y, size_t n_y, const uint8_t *b, size_t a, size_t e,
              const int32_t *carry_in, void *z, uint16_t *pcode, int32_t *carry_out, double *sigma2) {
    if (!h || !y || !b || !carry_in || !z || !pcode || !carry_out || !sigma2)
        return fail(RX_EINVAL, "NULL argument");
    if (e <= a || e > n_y) return fail(RX_EINVAL, "bad range");
    const int S = h->streams;
    const long K = (long)(e - a);
    const int chunks = bps_chunks(K, S);
    const long ncta = (K + bps_cta_range(chunks) - 1) / bps_cta_range(chunks);
    // interior increments come from the phase search; recompute them here
    int *dsum = nullptr;
    double *part = nullptr;
    unsigned *ticket = nullptr;
    CK(cudaMallocAsync(&dsum, sizeof(int) * (size_t)S * ncta, h->st));
    CK(cudaMallocAsync(&part, sizeof(double) * (size_t)S * ncta, h->st));
    CK(cudaMallocAsync(&ticket, sizeof(unsigned) * (size_t)S, h->st));
    CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned) * (size_t)S, h->st));
    CK(launch_dsum_from_b(b, K, a, e, dsum, chunks, S, h->fmt.B, h->st));
    cudaError_t err = launch_unwrap((const float2 *)y, (long)n_y, b, K, 0, (long)a, (long)e, dsum,
                                    carry_in, 2, carry_out, 2, (float2 *)z, K, 0, pcode, K, 0, part,
                                    sigma2, 1, ticket, 1, chunks, nullptr, S, h->fmt, h->st);
    cudaFreeAsync(dsum, h->st);
    cudaFreeAsync(part, h->st);
    cudaFreeAsync(ticket, h->st);
    CK(err);
    return RX_OK;
}

int rx_unwrap_static(rx_handle *h, const void *y, size_t n_y, const uint8_t *b, size_t a, size_t e,
                     const int32_t *carry_in, void *z, uint16_t *pcode, int32_t *carry_out,
                     double *sigma2) {
    if (!h || !y || !b || !carry_in || !z || !pcode || !carry_out || !sigma2)
        return fail(RX_EINVAL, "NULL argument");
    if (e <= a || e > n_y) return fail(RX_EINVAL, "bad range");
    const int S = h->streams;
    const long K = (long)(e - a);
    const int chunks = bps_chunks(K, S);
    const long ncta = (K + bps_cta_range(chunks) - 1) / bps_cta_range(chunks);
    const size_t off_dsum = align256(sizeof(unsigned) * (size_t)S);
    const size_t off_part = off_dsum + align256(sizeof(int) * (size_t)S * ncta);
    const size_t need = off_part + sizeof(double) * (size_t)S * ncta;
    if (need > kStaticScratchBytes)
        return fail(RX_EINVAL,
                    "rx_unwrap_static: %d stream(s) x %ld block(s) need %zu bytes of scratch, "
                    "more than the static %zu bytes; use fewer streams or a shorter range",
                    S, ncta, need, kStaticScratchBytes);
    void *base = nullptr;
    int rc = static_scratch(&base);
    if (rc != RX_OK) return rc;
    unsigned char *sc = static_cast<unsigned char *>(base);
    unsigned *ticket = reinterpret_cast<unsigned *>(sc);
    int *dsum = reinterpret_cast<int *>(sc + off_dsum);
    double *part = reinterpret_cast<double *>(sc + off_part);
    // the tickets must start at zero; the other regions are written before read
    CK(cudaMemsetAsync(ticket, 0, sizeof(unsigned) * (size_t)S, h->st));
    CK(launch_dsum_from_b(b, K, a, e, dsum, chunks, S, h->fmt.B, h->st));
    CK(launch_unwrap((const float2 *)y, (long)n_y, b, K, 0, (long)a, (long)e, dsum, carry_in, 2,
                     carry_out, 2, (float2 *)z, K, 0, pcode, K, 0, part, sigma2, 1, ticket, 1,
                     chunks, nullptr, S, h->fmt, h->st));
    return RX_OK;
}

int rx_demap(rx_handle *h, const void *z, size_t K, const double *sigma2, float *llr) {
    if (!h || !z || !sigma2 || !llr) return fail(RX_EINVAL, "NULL argument");
    DemapCount cnt{};
    CK(launch_demap((const float2 *)z, (long)K, 0, 0, (long)K, sigma2, 1, llr, (long)K * h->fmt.m, cnt,
                    h->streams, h->fmt, h->st));
    return RX_OK;
}

rx_kk *rx_kk_create(const rx_kk_params *p) {
    if (!p) { fail(RX_EINVAL, "NULL argument"); return nullptr; }
    if (p->n_ov <= 0 || p->n_ov >= 1024 || (p->n_ov & 1)) {
        fail(RX_EINVAL, "n_ov must be even, 0 < n_ov < 1024");
        return nullptr;
    }
    if (!(p->floor > 0.f)) { fail(RX_EINVAL, "floor must be > 0"); return nullptr; }
    rx_kk *k = new rx_kk();
    k->p = *p;
    std::vector<float2> tw(1024);
    for (int e = 0; e < 1024; ++e)
        tw[e] = make_float2((float)std::cos(2 * kPi * e / 1024), (float)(-std::sin(2 * kPi * e / 1024)));
    if (cudaMalloc(&k->tw, sizeof(float2) * 1024) != cudaSuccess ||
        cudaMemcpy(k->tw, tw.data(), sizeof(float2) * 1024, cudaMemcpyHostToDevice) != cudaSuccess) {
        fail(RX_ENOMEM, "rx_kk_create: twiddle table");
        cudaFree(k->tw);
        delete k;
        return nullptr;
    }
    return k;
}

void rx_kk_destroy(rx_kk *k) {
    if (!k) return;
    if (k->st) cudaStreamSynchronize(k->st);
    else cudaDeviceSynchronize();
    cudaFree(k->tw);
    delete k;
}

int rx_kk_set_stream(rx_kk *k, void *cuda_stream) {
    if (!k) return fail(RX_EINVAL, "NULL handle");
    k->st = (cudaStream_t)cuda_stream;
    return RX_OK;
}

int rx_kk_field(rx_kk *k, const int16_t *codes, size_t n_streams, size_t n, const float *levels,
                float *field_out) {
    if (!k || !codes || !levels || !field_out) return fail(RX_EINVAL, "NULL argument");
    if (n == 0) return fail(RX_EINVAL, "n must be > 0");
    if (n_streams < 1 || n_streams > (size_t)kKKMaxStreams)
        return fail(RX_EINVAL, "n_streams must be 1 .. %d", kKKMaxStreams);
    KKDev d{};
    d.floor = k->p.floor;
    d.fc_step = k->p.fc_step;
    d.n_streams = (int)n_streams;
    for (size_t s = 0; s < n_streams; ++s) d.lv[s] = make_float2(levels[2 * s], levels[2 * s + 1]);
    CK(launch_kk(codes, reinterpret_cast<float2 *>(field_out), (long)n, k->p.n_ov, d, k->tw, k->st));
    return RX_OK;
}

rx_fde *rx_fde_create(int taps, int n_ov) {
    if (n_ov <= 0 || n_ov >= 1024 || (n_ov & 3)) {
        fail(RX_EINVAL, "n_ov must be a multiple of 4, 0 < n_ov < 1024");
        return nullptr;
    }
    if (taps < 1 || !(taps & 1) || taps > n_ov + 1) { fail(RX_EINVAL, "taps must be odd, 1 .. n_ov + 1"); return nullptr; }
    rx_fde *e = new rx_fde();
    e->T = taps;
    e->n_ov = n_ov;
    std::vector<float2> tw(1024);
    for (int k = 0; k < 1024; ++k)
        tw[k] = make_float2((float)std::cos(2 * kPi * k / 1024), (float)(-std::sin(2 * kPi * k / 1024)));
    const size_t T = (size_t)taps;
    if (cudaMalloc(&e->R, sizeof(double2) * T * T) != cudaSuccess || cudaMalloc(&e->p, sizeof(double2) * T) != cudaSuccess ||
        cudaMalloc(&e->y, sizeof(double2) * T) != cudaSuccess || cudaMalloc(&e->h, sizeof(double2) * T) != cudaSuccess ||
        cudaMalloc(&e->H, sizeof(float2) * 1024) != cudaSuccess || cudaMalloc(&e->tw, sizeof(float2) * 1024) != cudaSuccess ||
        cudaMemcpy(e->tw, tw.data(), sizeof(float2) * 1024, cudaMemcpyHostToDevice) != cudaSuccess) {
        fail(RX_ENOMEM, "rx_fde_create: device buffers");
        cudaFree(e->R); cudaFree(e->p); cudaFree(e->y); cudaFree(e->h); cudaFree(e->H); cudaFree(e->tw);
        delete e;
        return nullptr;
    }
    return e;
}

void rx_fde_destroy(rx_fde *e) {
    if (!e) return;
    if (e->st) cudaStreamSynchronize(e->st);
    else cudaDeviceSynchronize();
    cudaFree(e->R); cudaFree(e->p); cudaFree(e->y); cudaFree(e->h); cudaFree(e->H); cudaFree(e->tw);
    delete e;
}

int rx_fde_set_stream(rx_fde *e, void *cuda_stream) {
    if (!e) return fail(RX_EINVAL, "NULL handle");
    e->st = (cudaStream_t)cuda_stream;
    return RX_OK;
}

int rx_fde_train(rx_fde *e, const float *x, size_t n, const float *d, size_t K, int sps, double delta) {
    if (!e || !x || !d) return fail(RX_EINVAL, "NULL argument");
    if (n == 0 || K == 0 || sps < 1 || !(delta >= 0.0)) return fail(RX_EINVAL, "n, K, sps must be > 0, delta >= 0");
    if (K > (size_t)INT32_MAX) return fail(RX_EINVAL, "K too large");
    CK(launch_fde_corr(reinterpret_cast<const float2 *>(x), (long)n, reinterpret_cast<const float2 *>(d), (int)K,
                       e->T, sps, e->R, e->p, e->st));
    CK(launch_fde_solve(e->R, e->p, e->y, e->T, delta, e->h, e->st));
    CK(launch_fde_response(e->h, e->T, e->H, e->st));
    e->ready = true;
    return RX_OK;
}

int rx_fde_set_taps(rx_fde *e, const double *taps) {
    if (!e || !taps) return fail(RX_EINVAL, "NULL argument");
    CK(cudaMemcpyAsync(e->h, taps, sizeof(double2) * e->T, cudaMemcpyHostToDevice, e->st));
    CK(launch_fde_response(e->h, e->T, e->H, e->st));
    CK(cudaStreamSynchronize(e->st));     // the host taps may go away
    e->ready = true;
    return RX_OK;
}

int rx_fde_get_taps(rx_fde *e, double *taps) {
    if (!e || !taps) return fail(RX_EINVAL, "NULL argument");
    if (!e->ready) return fail(RX_ESTATE, "no taps yet");
    CK(cudaStreamSynchronize(e->st));
    CK(cudaMemcpy(taps, e->h, sizeof(double2) * e->T, cudaMemcpyDeviceToHost));
    return RX_OK;
}

int rx_fde_apply(rx_fde *e, const float *x, size_t n_streams, size_t n, float *y) {
    if (!e || !x || !y) return fail(RX_EINVAL, "NULL argument");
    if (n == 0 || (n & 1)) return fail(RX_EINVAL, "n must be a positive even number");
    if (n_streams == 0 || n_streams > 65535) return fail(RX_EINVAL, "n_streams must be 1 .. 65535");
    if (!e->ready) return fail(RX_ESTATE, "the equaliser has no taps (rx_fde_train or rx_fde_set_taps)");
    CK(launch_fde_apply(reinterpret_cast<const float2 *>(x), reinterpret_cast<float2 *>(y), (long)n, (int)n_streams,
                        e->n_ov, e->H, e->tw, e->st));
    return RX_OK;
}

}  // extern "C"
