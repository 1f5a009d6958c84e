"""FP64 oracle of the receiver chain (test infrastructure only).

Chain: overlap-save chromatic-dispersion compensation with the matched
filter fused into the spectral multiply -> 2x2 butterfly FIR adapted
block-wise (CMA, then decision-directed LMS) -> blind phase search (BPS) ->
exact log-sum-exp bit LLRs -> BER / GMI counting.

What the paper fixes (arXiv 2108.07004, Sec. 2): overlap-save FFT
filtering; a time-domain adaptive equaliser whose taps are updated from part
of one buffer and used for later buffers; minimum-Euclidean-distance
decisions from an uploaded table of points and bit labels with no symmetry
assumed; decisions demapped to bits.  PCG64 symbols and error counting over
many buffers come from Sec. 3.  Everything else (CD transfer function, CMA,
BPS, LLRs, GMI) is the textbook definition, and each constant the paper
does not fix is a reading stated where it is used.

All arithmetic is float64 / complex128.  Python loops appear only where the
method itself is sequential (the LMS recursion).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .formats import OracleFormat

C_LIGHT = 299_792_458.0


@dataclass
class RxParams:
    symbol_rate: float = 28e9
    sps: int = 2
    cd_ps_per_nm: float = 0.0
    wavelength: float = 1550e-9
    rolloff: float = 0.1
    matched_filter: bool = True  # False: input already filtered (static equaliser after KK)
    n_fft: int = 1024          # overlap-save FFT size
    n_ov: int = 256            # overlap (discarded samples per frame)
    taps: int = 15             # FIR taps per butterfly branch (odd)
    mu: float = 1e-3
    bps_phases: int = 32       # B
    bps_window: int = 64       # W (even, centred window k-W/2 .. k+W/2-1)
    block: int = 4096          # symbols per processing block
    n_upd: int = 1024          # LMS updates per block (first symbols of it)
    lag: int = 1               # taps from block n's update apply from block n+lag
    n_pre: int = 2048          # start-up CMA span (symbols)
    cma_passes: int = 1
    n_cma: int = 0             # block-wise updates run as CMA before DD
    lms_block: int = 1         # block-wise updates in groups of this many (1: sequential)
    lms_start: int = 0         # update of block n starts from U_{n-1} (0) or from W_n = U_{n-lag} (1)
    widely_linear: bool = False  # butterfly on x and conj(x) (augmented taps, 2T per branch)
    n_train: int = 1024        # known training symbols at the stream start
    train_passes: int = 3      # data-aided LMS passes over the training span
    sigma2: float | None = None  # fixed noise variance, else per-block estimate
    skip_head: int = 4096      # symbols excluded from counting at stream start
    skip_tail: int = 512       # ... and at the stream end


# ---------------------------------------------------------------------------
# A1: chromatic-dispersion compensation (overlap-save)
# ---------------------------------------------------------------------------

def raised_cosine(f: np.ndarray, rs: float, beta: float) -> np.ndarray:
    """Raised-cosine spectrum normalised to 1 in the pass band."""
    out = np.zeros(f.shape)
    for i, fi in enumerate(np.abs(f)):
        lo, hi = (1 - beta) * rs / 2, (1 + beta) * rs / 2
        if fi <= lo:
            out[i] = 1.0
        elif fi <= hi:
            out[i] = 0.5 * (1 + np.cos(np.pi * (fi - lo) / (beta * rs)))
    return out


def cd_response(f: np.ndarray, cd_ps_per_nm: float, wavelength: float) -> np.ndarray:
    """H_CD(f) = exp(j * D*L * lambda^2 * omega^2 / (4 pi c)), omega = 2 pi f.

    D*L is given in ps/nm (1 ps/nm = 1e-3 s/m)."""
    dl = cd_ps_per_nm * 1e-3
    omega = 2 * np.pi * f
    return np.exp(1j * dl * wavelength ** 2 * omega ** 2 / (4 * np.pi * C_LIGHT))


def cdc_filter(p: RxParams) -> np.ndarray:
    """Receiver spectral multiply for one FFT frame: conj(H_CD) * H_MF.

    H_MF = sqrt(sps * raised_cosine): the root-raised-cosine matched filter
    (reading: the paper's static FD equaliser is replaced by CD inversion
    plus matched filtering in the same FFT pair)."""
    f = np.fft.fftfreq(p.n_fft, d=1.0 / (p.sps * p.symbol_rate))
    hmf = np.sqrt(p.sps * raised_cosine(f, p.symbol_rate, p.rolloff)) if p.matched_filter else 1.0
    return np.conj(cd_response(f, p.cd_ps_per_nm, p.wavelength)) * hmf


def cdc(r: np.ndarray, p: RxParams, H: np.ndarray | None = None) -> np.ndarray:
    """Overlap-save filtering of each polarisation of r [2, Ns].

    Framing is global to the stream: frame f reads input samples
    f*S - n_ov/2 .. f*S - n_ov/2 + n_fft - 1 (S = n_fft - n_ov; samples
    outside the stream are zero), multiplies its FFT by H, inverse-FFTs and
    keeps frame positions n_ov/2 .. n_ov/2 + S - 1 as outputs f*S .. f*S+S-1
    (symmetric discard, reading: the CD response is non-causal)."""
    if H is None:
        H = cdc_filter(p)
    r = np.asarray(r, dtype=np.complex128)
    ns = r.shape[1]
    S = p.n_fft - p.n_ov
    half = p.n_ov // 2
    nfr = -(-ns // S)
    out = np.zeros_like(r)
    for pol in range(2):
        padded = np.concatenate([np.zeros(half, complex), r[pol],
                                 np.zeros(nfr * S + p.n_fft, complex)])
        for fr in range(nfr):
            seg = padded[fr * S: fr * S + p.n_fft]      # starts at input fr*S - half
            y = np.fft.ifft(np.fft.fft(seg) * H)
            keep = y[half: half + S]
            lo, hi = fr * S, min(fr * S + S, ns)
            out[pol, lo:hi] = keep[: hi - lo]
    return out


# ---------------------------------------------------------------------------
# A2: 2x2 butterfly FIR, T/2-spaced in, one output per symbol
# ---------------------------------------------------------------------------

def center_spike(T: int, widely_linear: bool = False) -> np.ndarray:
    """h[q, p, t]: identity butterfly, h_XX[D] = h_YY[D] = 1, D=(T-1)/2.
    Widely linear: 2T taps per branch, the first T on x (identity), the
    last T on conj(x) (zero)."""
    h = np.zeros((2, 2, 2 * T if widely_linear else T), dtype=np.complex128)
    D = (T - 1) // 2
    h[0, 0, D] = 1.0
    h[1, 1, D] = 1.0
    return h


def window(x: np.ndarray, k: int, L: int) -> np.ndarray:
    """The input window of update k for taps of length L per branch: x_window
    for odd L (= T), and for even L = 2T the widely-linear window
    [x_window, conj(x_window)] (paper Sec. 2: a widely linear equaliser acts
    on the signal and its conjugate)."""
    if L % 2:
        return x_window(x, k, L)
    xw = x_window(x, k, L // 2)
    return np.concatenate([xw, np.conj(xw)], axis=1)


def x_window(x: np.ndarray, k: int, T: int) -> np.ndarray:
    """[2, T] with entry [p, t] = x_p[2k + D - t]; zero outside the stream."""
    D = (T - 1) // 2
    ns = x.shape[1]
    w = np.zeros((2, T), dtype=np.complex128)
    for t in range(T):
        i = 2 * k + D - t
        if 0 <= i < ns:
            w[:, t] = x[:, i]
    return w


def fir(x: np.ndarray, h: np.ndarray, k0: int, k1: int) -> np.ndarray:
    """y_q[k] = sum_p sum_t conj(h[q,p,t]) * x_p[2k + D - t] for k0 <= k < k1;
    with widely-linear taps (2T per branch) also + conj(h[q,p,T+t]) *
    conj(x_p[2k + D - t])."""
    L = h.shape[2]
    wl = L % 2 == 0
    T = L // 2 if wl else L
    D = (T - 1) // 2
    ns = x.shape[1]
    k = np.arange(k0, k1)
    y = np.zeros((2, k1 - k0), dtype=np.complex128)
    for q in range(2):
        for pol in range(2):
            for t in range(T):
                i = 2 * k + D - t
                ok = (i >= 0) & (i < ns)
                v = np.zeros(k.shape, dtype=np.complex128)
                v[ok] = x[pol, i[ok]]
                y[q] += np.conj(h[q, pol, t]) * v
                if wl:
                    y[q] += np.conj(h[q, pol, T + t]) * np.conj(v)
    return y


# ---------------------------------------------------------------------------
# decisions (Sec. 2: minimum Euclidean distance over the uploaded table)
# ---------------------------------------------------------------------------

def decide(z: np.ndarray, fmt: OracleFormat):
    """Nearest table point for z [2, K].

    4D tables: joint over both polarisations; 2D tables: per polarisation.
    Ties go to the lowest label.  Returns (d [2,K], label(s), margin [K]) with
    margin = second-smallest minus smallest squared distance (the smaller of
    the two polarisations' margins for 2D tables)."""
    if fmt.dims == 4:
        dist = (np.abs(z[0][:, None] - fmt.points[None, :, 0]) ** 2 +
                np.abs(z[1][:, None] - fmt.points[None, :, 1]) ** 2)
        j = np.argmin(dist, axis=1)
        srt = np.sort(dist, axis=1)
        return fmt.points[j].T.copy(), j, srt[:, 1] - srt[:, 0]
    d = np.empty_like(z)
    js, margins = [], []
    for pol in range(2):
        dist = np.abs(z[pol][:, None] - fmt.points[None, :]) ** 2
        j = np.argmin(dist, axis=1)
        srt = np.sort(dist, axis=1)
        d[pol] = fmt.points[j]
        js.append(j)
        margins.append(srt[:, 1] - srt[:, 0])
    return d, np.stack(js), np.minimum(margins[0], margins[1])


# ---------------------------------------------------------------------------
# A3: sequential CMA / DD-LMS
# ---------------------------------------------------------------------------

@dataclass
class LmsInfo:
    dd_margin: list = field(default_factory=list)   # (k, margin) of each DD update


def lms(x: np.ndarray, h: np.ndarray, ks, fmt: OracleFormat, p: RxParams,
        u0: int = 0, phase: dict | None = None, force_cma: bool = False,
        info: LmsInfo | None = None) -> np.ndarray:
    """Run the stochastic-gradient recursion over symbols ``ks`` in order.

    Update u (global count u0, u0+1, ...) is CMA while u < n_cma (or always
    when ``force_cma``), DD-LMS afterwards:
      CMA:  h_qp[t] += mu * (R^2 - |y_q|^2) * conj(y_q) * x_p[2k+D-t]
      DD:   e_q = d_q * exp(j phi_k) - y_q,  d = decide(y * exp(-j phi_k)),
            h_qp[t] += mu * conj(e_q) * x_p[2k+D-t]
    with y_q = sum conj(h_qp[t]) x_p[2k+D-t], R^2 = E|s|^4/E|s|^2 and phi_k
    the carrier phase estimate of symbol k (``phase[k]``)."""
    h = h.copy()
    T = h.shape[2]
    R2 = fmt.cma_radius2()
    u = u0
    for k in ks:
        xw = window(x, k, T)
        y = np.array([np.sum(np.conj(h[q]) * xw) for q in range(2)])
        if force_cma or u < p.n_cma:
            e = (R2 - np.abs(y) ** 2) * y           # conj(e) = (R^2-|y|^2) conj(y)
        else:
            ph = phase[k]
            zc = (y * np.exp(-1j * ph))[:, None]
            d, _, marg = decide(zc, fmt)
            e = d[:, 0] * np.exp(1j * ph) - y
            if info is not None:
                info.dd_margin.append((k, float(marg[0])))
        for q in range(2):
            h[q] += p.mu * np.conj(e[q]) * xw
        u += 1
    return h


def lms_block(x: np.ndarray, h: np.ndarray, ks, fmt: OracleFormat, p: RxParams, P: int,
              u0: int = 0, phase: dict | None = None, info: LmsInfo | None = None) -> np.ndarray:
    """Block LMS (Clark, Mitra and Parker, 1981) over symbols ``ks``: the
    updates run in groups of P consecutive symbols; every output y_k and
    error e_k of a group is computed with the taps at the start of the group
    (CMA or DD per update count exactly as in ``lms``), then the group's P
    gradient terms are applied together, h_q += mu * sum_k conj(e_q[k]) x[k].
    P = 1 is the sequential recursion.  Reading: the paper names the
    sequential tap update as the part of the chain that is hard to
    parallelise (Sec. 2) and prints no alternative; this is the textbook
    parallel form, a variant beside the exact chain."""
    h = h.copy()
    T = h.shape[2]
    R2 = fmt.cma_radius2()
    ks = list(ks)
    u = u0
    for g0 in range(0, len(ks), P):
        terms = []
        for k in ks[g0:g0 + P]:
            xw = window(x, k, T)
            y = np.array([np.sum(np.conj(h[q]) * xw) for q in range(2)])
            if u < p.n_cma:
                e = (R2 - np.abs(y) ** 2) * y
            else:
                ph = phase[k]
                d, _, marg = decide((y * np.exp(-1j * ph))[:, None], fmt)
                e = d[:, 0] * np.exp(1j * ph) - y
                if info is not None:
                    info.dd_margin.append((k, float(marg[0])))
            terms.append((e, xw))
            u += 1
        for e, xw in terms:
            for q in range(2):
                h[q] += p.mu * np.conj(e[q]) * xw
    return h


def align_training(x: np.ndarray, h: np.ndarray, ref_sym: np.ndarray) -> np.ndarray:
    """Fix the output permutation and per-output phase from known symbols.

    Sec. 2: the adaptive equaliser converges with a training sequence before
    running blind.  Reading: after start-up CMA, correlate the equalised
    outputs over the training span with the known symbols,
    C[q, p] = sum_k y_q[k] conj(s_p[k]); keep the output order if
    |C00|^2+|C11|^2 >= |C01|^2+|C10|^2, else swap; then rotate each output by
    -arg C[q, matched p] (h row multiplied by exp(+j arg))."""
    n = ref_sym.shape[1]
    y = fir(x, h, 0, n)
    C = y @ np.conj(ref_sym).T
    swap = (abs(C[0, 1]) ** 2 + abs(C[1, 0]) ** 2) > (abs(C[0, 0]) ** 2 + abs(C[1, 1]) ** 2)
    src = [1, 0] if swap else [0, 1]             # new output p takes old output src[p]
    out = np.empty_like(h)
    for pnew in range(2):
        q = src[pnew]
        out[pnew] = h[q] * np.exp(1j * np.angle(C[q, pnew]))
    return out


def train_phase(y: np.ndarray, ref_sym: np.ndarray, W: int, B: int, S: int):
    """Data-aided phase over the training span, on the phase-search grid.

    R_k = sum over i in [k - W/2, k + W/2) (within the span) of
    sum_p y_p[i] conj(s_p[i]); phi_k = arg R_k, rounded to the nearest
    multiple n_k of q/B (q = 2 pi/S; round(x) = floor(x + 1/2)), written as
    phi_k = phi_b + m q with b = n_k + B/2 - m B, m = floor((n_k + B/2)/B).
    Reading: the paper trains the equaliser on a known sequence before it
    runs blind (Sec. 2); the known symbols give the phase without the
    rotational ambiguity."""
    n = y.shape[1]
    r = np.sum(y * np.conj(ref_sym), axis=0)
    b = np.empty(n, dtype=np.int64)
    m = np.empty(n, dtype=np.int64)
    step = 2 * np.pi / S / B
    for k in range(n):
        R = np.sum(r[max(0, k - W // 2): min(n, k + W // 2)])
        nk = int(np.floor(np.angle(R) / step + 0.5))
        m[k] = (nk + B // 2) // B
        b[k] = nk + B // 2 - m[k] * B
    return b, m


def lms_trained(x: np.ndarray, h: np.ndarray, ks, ref_sym: np.ndarray, phase: np.ndarray,
                p: RxParams) -> np.ndarray:
    """Data-aided LMS over symbols ks: e_q = s_q[k] exp(j phi_k) - y_q,
    h_qp[t] += mu conj(e_q) x_p[2k + D - t] (the DD update with the known
    symbol in place of the decision)."""
    h = h.copy()
    T = h.shape[2]
    for k in ks:
        xw = window(x, k, T)
        y = np.array([np.sum(np.conj(h[q]) * xw) for q in range(2)])
        e = ref_sym[:, k] * np.exp(1j * phase[k]) - y
        for q in range(2):
            h[q] += p.mu * np.conj(e[q]) * xw
    return h


# ---------------------------------------------------------------------------
# A4: blind phase search
# ---------------------------------------------------------------------------

def bps_phases(B: int, S: int) -> np.ndarray:
    """Test phases phi_b = (b/B - 1/2) * 2 pi / S, b = 0..B-1."""
    return (np.arange(B) / B - 0.5) * 2 * np.pi / S


def bps_min_dist(y: np.ndarray, phis: np.ndarray, fmt: OracleFormat) -> np.ndarray:
    """[K, B]: min_j || y_k exp(-j phi_b) - s_j ||^2 (4D joint, or summed over
    polarisations of per-polarisation minima for a 2D table)."""
    K = y.shape[1]
    out = np.empty((K, len(phis)))
    for b, ph in enumerate(phis):
        r = y * np.exp(-1j * ph)
        if fmt.dims == 4:
            d = (np.abs(r[0][:, None] - fmt.points[None, :, 0]) ** 2 +
                 np.abs(r[1][:, None] - fmt.points[None, :, 1]) ** 2)
            out[:, b] = np.min(d, axis=1)
        else:
            out[:, b] = sum(np.min(np.abs(r[pol][:, None] - fmt.points[None, :]) ** 2, axis=1)
                            for pol in range(2))
    return out


def bps(y: np.ndarray, a: int, e: int, n_valid: int, p: RxParams, fmt: OracleFormat):
    """Phase index b_k for a <= k < e.

    cost_b(k) = sum over i in [k - W/2, k + W/2) intersected with
    [0, n_valid) of min-distance(i, b); b_k = argmin_b cost (lowest b on
    ties).  Returns (b [e-a], relative gap between the two smallest costs,
    min-distance [e-a] at the chosen phase)."""
    W = p.bps_window
    lo, hi = max(0, a - W // 2), min(n_valid, e + W // 2 - 1)
    phis = bps_phases(p.bps_phases, fmt.sym_order)
    md = bps_min_dist(y[:, lo:hi], phis, fmt)          # rows lo..hi-1
    # rows a-W/2 .. e+W/2-2; rows outside [lo, hi) (outside the stream) add 0
    full = np.zeros((e - a + W - 1, len(phis)))
    off = (a - W // 2)
    full[lo - off: hi - off] = md
    # window of k is rows k-W/2 .. k+W/2-1, i.e. full[k-a : k-a+W]
    cost = np.lib.stride_tricks.sliding_window_view(full, W, axis=0).sum(axis=-1)
    b = np.argmin(cost, axis=1).astype(np.int64)          # first minimum: lowest b
    srt = np.sort(cost, axis=1)
    gap = (srt[:, 1] - srt[:, 0]) / np.maximum(srt[:, 0], 1e-300)
    chosen = full[np.arange(e - a) + W // 2, b]
    return b, gap, chosen


def unwrap(b: np.ndarray, m_prev: int, b_prev: int, B: int):
    """phi_hat_k = phi_k + q * round(((phi_hat_{k-1}) - phi_k) / q), q = 2 pi/S,
    round(x) = floor(x + 1/2) (reading: ties round up).

    Since every phi_k lies on the grid, phi_hat_k = phi_{b_k} + q*m_k with an
    integer m_k, and (phi_hat_{k-1} - phi_k)/q = m_{k-1} + (b_{k-1} - b_k)/B
    exactly, so the rounding is evaluated in integers:
    m_k = m_{k-1} + floor((2 (b_{k-1} - b_k) + B) / (2B)).
    The stream starts from phi_hat = 0 (m = 0 at b = B/2)."""
    m = np.empty(len(b), dtype=np.int64)
    for i, bk in enumerate(b):
        m_prev = m_prev + (2 * (b_prev - int(bk)) + B) // (2 * B)
        b_prev = int(bk)
        m[i] = m_prev
    return m, m_prev, b_prev


def quadrant_anchor(b: np.ndarray, train_b: np.ndarray, train_m: np.ndarray, B: int,
                    S: int) -> int:
    """Resolve the rotational ambiguity of the blind phase against the
    training phases (reading: the known start of the stream fixes it once).

    Unwrap the first phase indices from phi_hat = 0, and over the training
    span compare with the training phase in grid units (n = b - B/2 + m B):
    q_k = floor((n_train_k - n_blind_k) / B + 1/2) mod S.  The most common
    q (lowest on ties) is the quadrant count the unwrap starts from."""
    n = min(len(b), len(train_b))
    m0, _, _ = unwrap(b[:n], 0, B // 2, B)
    d = (train_b[:n] - B // 2 + train_m[:n] * B) - (b[:n] - B // 2 + m0 * B)
    q = np.floor_divide(2 * d + B, 2 * B) % S
    votes = np.bincount(q, minlength=S)
    return int(np.argmax(votes))


def phase_of(b: np.ndarray, m: np.ndarray, B: int, S: int) -> np.ndarray:
    q = 2 * np.pi / S
    return (b / B - 0.5) * q + m * q


# ---------------------------------------------------------------------------
# A5: exact LLRs, A6: counting
# ---------------------------------------------------------------------------

def estimate_sigma2(z: np.ndarray, fmt: OracleFormat) -> float:
    """sigma^2 = mean over symbols and polarisations of |z - d|^2, d the
    nearest table point (reading: decision-directed block estimate of the
    complex noise variance per polarisation)."""
    d, _, _ = decide(z, fmt)
    return float(np.sum(np.abs(z - d) ** 2) / (2 * z.shape[1]))


def _lse(v: np.ndarray) -> np.ndarray:
    mx = np.max(v, axis=-1, keepdims=True)
    return mx[..., 0] + np.log(np.sum(np.exp(v - mx), axis=-1))


def llr(z: np.ndarray, sigma2: float, fmt: OracleFormat) -> np.ndarray:
    """LLR_i = ln sum_{j: b_i(j)=0} exp(-||z - s_j||^2/sigma^2)
             - ln sum_{j: b_i(j)=1} exp(-||z - s_j||^2/sigma^2)
    (max-shifted log-sum-exp).  Positive means bit 0.  4D tables: joint over
    both polarisations, m LLRs per symbol; 2D tables: per polarisation, the
    row holds the X bits then the Y bits."""
    bt = fmt.bit_table()
    if fmt.dims == 4:
        dist = (np.abs(z[0][:, None] - fmt.points[None, :, 0]) ** 2 +
                np.abs(z[1][:, None] - fmt.points[None, :, 1]) ** 2)
        lg = -dist / sigma2
        return np.stack([_lse(lg[:, bt[:, i] == 0]) - _lse(lg[:, bt[:, i] == 1])
                         for i in range(fmt.m)], axis=1)
    cols = []
    for pol in range(2):
        lg = -np.abs(z[pol][:, None] - fmt.points[None, :]) ** 2 / sigma2
        for i in range(fmt.m_pol):
            cols.append(_lse(lg[:, bt[:, i] == 0]) - _lse(lg[:, bt[:, i] == 1]))
    return np.stack(cols, axis=1)


def count(llrs: np.ndarray, bits: np.ndarray) -> dict:
    """Bit errors of the hard decisions (LLR < 0 -> 1) and the GMI sum
    sum log2(1 + exp(-(1 - 2b) * LLR)) over the given rows."""
    hard = (llrs < 0).astype(np.uint8)
    errors = int(np.sum(hard != bits))
    sgn = 1.0 - 2.0 * bits
    gsum = float(np.sum(np.logaddexp(0.0, -sgn * llrs)) / np.log(2))
    n = llrs.shape[0]
    m = llrs.shape[1]
    return dict(n_sym=n, n_bits=n * m, bit_errors=errors, gmi_sum=gsum,
                ber=errors / max(1, n * m), gmi=m - gsum / max(1, n))


# ---------------------------------------------------------------------------
# the block schedule
# ---------------------------------------------------------------------------

@dataclass
class ChainResult:
    x: np.ndarray
    w0: np.ndarray
    taps_used: list            # W_n per block
    taps_after: list           # LMS state U_n after block n
    y: np.ndarray
    b: np.ndarray
    m: np.ndarray
    phi: np.ndarray
    z: np.ndarray
    sigma2: list               # per block
    ranges: list               # (a, e) BPS/demap range per block
    llr: np.ndarray
    bps_gap: np.ndarray
    dd_margin: list
    stats: dict
    train_b: np.ndarray | None = None
    train_m: np.ndarray | None = None
    w_cma: np.ndarray | None = None


def state_at(res: ChainResult, p: RxParams, n: int) -> dict:
    """What block n (n >= 1) of the schedule in run_chain takes from the
    blocks before it: the LMS results U_{n-lag} .. U_{n-1} (U_i = W_0 for
    i < 0; block n+j equalises with entry j and the LMS of block n starts
    from the last), the unwrap carry (m, b) of the last symbol before block
    n's range, the equaliser output of the W symbols before n*block (the
    phase-search halo; zeros before symbol 0) and the number of LMS updates
    so far.  Everything else in block n is computed from the samples."""
    N = res.y.shape[1]
    L, W = p.lag, p.bps_window
    assert 1 <= n <= len(res.ranges)
    taps = [res.taps_after[i] if i >= 0 else res.w0 for i in range(n - L, n)]
    last = res.ranges[n - 1][1] - 1
    K = n * p.block
    y_tail = np.zeros((2, W), complex)
    lo = max(0, K - W)
    y_tail[:, lo - (K - W):] = res.y[:, lo:K]
    u = sum(len(range(i * p.block, min(i * p.block + p.n_upd, N))) for i in range(n))
    return {"taps": taps, "carry": (int(res.m[last]), int(res.b[last])), "y_tail": y_tail,
            "lms_updates": u}


def run_chain(r: np.ndarray, fmt: OracleFormat, p: RxParams,
              ref_bits: np.ndarray | None = None, resume: tuple | None = None) -> ChainResult:
    """Whole receiver on one stream r [2, sps*N] with the block schedule:

    start-up: CMA over the first n_pre symbols (cma_passes passes) from the
    identity butterfly; then, if known bits are given, the training stage
    over the first n_train symbols: output order and phases from the
    correlation with the known symbols, a data-aided phase estimate, and
    train_passes passes of data-aided LMS -> W_0.  Block n (symbols
    n*block .. n*block+block-1):
      1. FIR with W_n = U_{n-lag} (W_0 while n < lag);
      2. BPS, unwrap, de-rotation and LLRs over the range
         [n*block - W/2, (n+1)*block - W/2) (clipped to the stream; the last
         block runs to the stream end), which needs FIR output of block n only;
         in block 0 the unwrap's start quadrant comes from the training phases;
      3. LMS over the first n_upd symbols of block n starting from U_{n-1}
         (U_{-1} = W_0), or with lms_start = 1 from W_n, the taps that
         equalised block n -> U_n  (Sec. 2: part of a buffer updates the
         taps used for subsequent buffers).
    resume = (n, state_at(...) of block n): skip the start-up and blocks
    before n and continue from that state (outputs before block n's range
    stay zero; counting still covers skip_head .. N - skip_tail)."""
    r = np.asarray(r, dtype=np.complex128)
    N = r.shape[1] // p.sps
    W, B, L, S = p.bps_window, p.bps_phases, p.lag, fmt.sym_order
    assert p.n_upd + W // 2 <= p.block, "update span must have phases in its block"
    x = cdc(r, p)
    h = center_spike(p.taps, p.widely_linear)
    npre = 0 if resume else min(p.n_pre, N)
    for _ in range(p.cma_passes if npre else 0):
        h = lms(x, h, range(npre), fmt, p, force_cma=True)
    w_cma = h.copy()
    train_b = train_m = None
    if ref_bits is not None and p.n_train > 0 and not resume:
        ntr = min(p.n_train, N)
        ref = fmt.symbols_from_bits(ref_bits[:ntr])
        h = align_training(x, h, ref)
        train_b, train_m = train_phase(fir(x, h, 0, ntr), ref, p.bps_window, p.bps_phases, S)
        tphi = phase_of(train_b, train_m, p.bps_phases, S)
        for _ in range(p.train_passes):
            h = lms_trained(x, h, range(ntr), ref, tphi, p)
    w0 = h.copy()
    ring = [w0.copy() for _ in range(L + 1)]
    y = np.zeros((2, N), complex)
    z = np.zeros((2, N), complex)
    bb = np.zeros(N, np.int64)
    mm = np.zeros(N, np.int64)
    gap = np.zeros(N)
    out = np.zeros((N, fmt.m))
    m_prev, b_prev = 0, B // 2          # phi_hat = 0 before the first symbol
    u = 0
    nblk = -(-N // p.block)
    used, after, s2s, ranges, info = [], [], [], [], LmsInfo()
    n_first = 0
    if resume:
        n_first, stt = resume
        for j, t in enumerate(stt["taps"]):
            ring[(n_first - L + j) % (L + 1)] = np.array(t, dtype=complex)
        m_prev, b_prev = stt["carry"]
        K = n_first * p.block
        lo = max(0, K - W)
        y[:, lo:K] = stt["y_tail"][:, lo - (K - W):]
        u = stt["lms_updates"]
        used, after, s2s, ranges = [None] * n_first, [None] * n_first, [None] * n_first, [None] * n_first
    for n in range(n_first, nblk):
        k0, k1 = n * p.block, min((n + 1) * p.block, N)
        wn = ring[(n - L) % (L + 1)]
        used.append(wn.copy())
        y[:, k0:k1] = fir(x, wn, k0, k1)
        a = max(0, k0 - W // 2)
        e = N if n == nblk - 1 else k1 - W // 2
        b, g, _ = bps(y, a, e, k1, p, fmt)
        if n == 0 and train_b is not None:
            m_prev = quadrant_anchor(b, train_b, train_m, B, S)
        m, m_prev, b_prev = unwrap(b, m_prev, b_prev, B)
        bb[a:e], mm[a:e], gap[a:e] = b, m, g
        phi = phase_of(b, m, B, S)
        z[:, a:e] = y[:, a:e] * np.exp(-1j * phi)[None, :]
        s2 = p.sigma2 if p.sigma2 is not None else estimate_sigma2(z[:, a:e], fmt)
        s2s.append(s2)
        ranges.append((a, e))
        out[a:e] = llr(z[:, a:e], s2, fmt)
        span = range(k0, min(k0 + p.n_upd, N))
        phase = {k: phi[k - a] for k in span}
        h_in = wn if p.lms_start else ring[(n - 1) % (L + 1)]
        if p.lms_block > 1:
            hn = lms_block(x, h_in, span, fmt, p, p.lms_block, u0=u, phase=phase, info=info)
        else:
            hn = lms(x, h_in, span, fmt, p, u0=u, phase=phase, info=info)
        u += len(span)
        ring[n % (L + 1)] = hn
        after.append(hn.copy())
    phi_all = phase_of(bb, mm, B, S)
    stats = {}
    if ref_bits is not None:
        c0, c1 = min(p.skip_head, N), max(min(p.skip_head, N), N - p.skip_tail)
        stats = count(out[c0:c1], np.asarray(ref_bits[c0:c1], dtype=np.float64))
        d, _, _ = decide(z[:, c0:c1], fmt)
        stats["evm_num"] = float(np.sum(np.abs(z[:, c0:c1] - d) ** 2))
        stats["evm_den"] = float(np.sum(np.abs(d) ** 2))
    return ChainResult(x, w0, used, after, y, bb, mm, phi_all, z, s2s, ranges, out,
                       gap, info.dd_margin, stats, train_b, train_m, w_cma)
