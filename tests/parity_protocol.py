"""The end-to-end acceptance rule of the GPU parity tests (test
infrastructure; no torch, so that spawned oracle workers can use it).

FP32 cannot resolve a phase-search argmin whose two best window costs
differ by less than TIE relative, so at such a near-tie either phase index
is a valid result.  From the oracle alone this bounds, per block, what the
GPU may validly hold: the symbol's own de-rotated z (each candidate index,
the unwrap continued from the symbol before) and the block's
decision-directed sigma^2, which moves by the candidate's change of minimum
distance / 2K.  A near-tie inside an LMS span may change the taps of the
blocks lag later, so a run is cut there and resumed from the oracle's
state.
"""
import numpy as np

from oracle import chain

LLR_RTOL = 1e-4
TIE = 1e-4
DD_TIE = 1e-5


def segments(res, p, N):
    """Cut the block schedule into runs [n0, n1) over which the GPU and the
    oracle equalise with the same taps: a near-tie (BPS or DD decision)
    inside block nb's LMS span may change U_nb, which blocks nb+lag and
    later use, so a run ends at nb + lag and the next one resumes from the
    oracle's state there."""
    tie = res.bps_gap < TIE
    dd_ties = {k for k, mg in res.dd_margin if mg < DD_TIE}
    nblk = len(res.ranges)
    segs, n0 = [], 0
    while n0 < nblk:
        n1 = nblk
        for nb in range(n0, nblk):
            span = range(nb * p.block, min(nb * p.block + p.n_upd, N))
            if any(tie[k] or k in dd_ties for k in span):
                n1 = min(nblk, nb + p.lag)
                break
        segs.append((n0, n1))
        n0 = n1
    return segs


def inc(b_prev, b, B):
    return (2 * (int(b_prev) - int(b)) + B) // (2 * B)


def block_valid(res, p, fmt, n, N):
    """What the block-n range may validly hold.  At a BPS near-tie symbol k
    (oracle gap < TIE) every phase index whose window cost is within TIE of
    the minimum is a valid choice; it changes z at k (the unwrap continued
    from symbol k-1) and the block's decision-directed sigma^2 (the mean of
    the minimum distances at the chosen phases), which then lies in an
    interval [s2 + t_lo, s2 + t_hi] around the oracle's s2.  Returns the
    oracle's LLRs L0 at s2, their derivative dL in sigma^2, the interval
    (t_lo, t_hi), and for the near-tie rows an envelope [lo, hi] over all
    choices and the interval."""
    a, e = res.ranges[n]
    K = e - a
    B, S, W = p.bps_phases, fmt.sym_order, p.bps_window
    phis = chain.bps_phases(B, S)
    n_valid = min((n + 1) * p.block, N)
    y = res.y
    ties = [k for k in range(a, e) if res.bps_gap[k] < TIE]
    s2 = res.sigma2[n]
    d_lo = d_hi = 0.0
    alts = {}
    for k in ties:
        lo_w, hi_w = max(0, k - W // 2), min(n_valid, k + W // 2)
        md = chain.bps_min_dist(y[:, lo_w:hi_w], phis, fmt)
        cost = md.sum(axis=0)
        c0 = cost.min()
        cand = np.flatnonzero((cost - c0) / max(c0, 1e-300) < TIE)
        row = md[k - lo_w]
        dd = row[cand] - row[res.b[k]]
        d_lo += min(0.0, dd.min())
        d_hi += max(0.0, dd.max())
        if k > 0:
            m_p, b_p = res.m[k - 1], res.b[k - 1]
        else:                                  # carry into symbol 0 from the anchored start
            b_p = B // 2
            m_p = res.m[0] - inc(b_p, res.b[0], B)
        alts[k] = [(int(c), int(m_p) + inc(b_p, c, B)) for c in cand]
    fixed = p.sigma2 is not None
    t_lo, t_hi = (0.0, 0.0) if fixed else (d_lo / (2 * K), d_hi / (2 * K))
    z = res.z[:, a:e]
    L0 = chain.llr(z, s2, fmt)
    if t_hi > t_lo:
        dL = (chain.llr(z, s2 + t_hi, fmt) - chain.llr(z, s2 + t_lo, fmt)) / (t_hi - t_lo)
    else:
        dL = np.zeros_like(L0)
    sig = [s2 + t_lo, s2, s2 + t_hi]
    env = {}
    for k, cl in alts.items():
        zk = []
        for c, m in cl:
            ph = chain.phase_of(np.array([c]), np.array([m]), B, S)[0]
            zk.append(y[:, k] * np.exp(-1j * ph))
        zk = np.stack(zk, axis=1)
        Lk = np.stack([chain.llr(zk, v, fmt) for v in sig])        # [sigma, choice, bit]
        env[k] = (Lk.min(axis=(0, 1)), Lk.max(axis=(0, 1)))
    return L0, dL, (t_lo, t_hi), env


def check_block(g, L0, dL, t_range, env, a):
    """Rows of one block: the near-tie rows inside their envelopes, and one
    common sigma^2 offset t in t_range under which every other row is within
    1e-4 * max(1, |LLR|) of the oracle's LLR (linear in t over the tiny
    interval).  Returns a list of (row, message) failures."""
    fails = []
    tie_rows = np.zeros(len(L0), bool)
    for k, (lo, hi) in env.items():
        i = k - a
        tie_rows[i] = True
        tol = LLR_RTOL * np.maximum(1.0, np.maximum(np.abs(lo), np.abs(hi)))
        if np.any((g[i] < lo - tol) | (g[i] > hi + tol)):
            fails.append((k, f"near-tie row outside [{lo}, {hi}]: {g[i]}"))
    rows = np.flatnonzero(~tie_rows)
    G, L, D = g[rows], L0[rows], dL[rows]
    tol = LLR_RTOL * np.maximum(1.0, np.abs(L))
    t_lo, t_hi = t_range
    width = t_hi - t_lo
    if width <= 0:
        far = np.abs(G - L) > tol
        for i in np.unique(np.nonzero(far)[0])[:8]:
            fails.append((a + rows[i], f"llr {L[i]} gpu {G[i]}"))
        return fails
    slope = np.abs(D) * width > 1e-3 * tol          # entries for which t matters
    flat_bad = ~slope & (np.abs(G - L) > tol + np.abs(D) * max(abs(t_lo), abs(t_hi)))
    for i in np.unique(np.nonzero(flat_bad)[0])[:8]:
        fails.append((a + rows[i], f"llr {L[i]} gpu {G[i]}"))
    t_mid = 0.0
    if slope.any():
        u1 = (G - tol - L)[slope] / D[slope]
        u2 = (G + tol - L)[slope] / D[slope]
        t_lo = max(t_lo, np.max(np.minimum(u1, u2)))
        t_hi = min(t_hi, np.min(np.maximum(u1, u2)))
        t_mid = np.median(0.5 * (u1 + u2))
    if t_lo > t_hi:
        t = min(max(t_mid, t_range[0]), t_range[1])     # robust to a few wrong rows
        far = np.abs(G - (L + D * t)) > tol
        for i in np.unique(np.nonzero(far)[0])[:8]:
            fails.append((a + rows[i], f"no common sigma^2 offset in [{t_range[0]:.3g}, {t_range[1]:.3g}]: "
                                       f"llr {L[i]} gpu {G[i]}"))
        if not far.any():
            fails.append((a, "no common sigma^2 offset"))
    return fails
