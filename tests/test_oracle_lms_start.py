"""Pins of the oracle's alternative update start (lms_start = 1: the update
over block n starts from W_n = U_{n-lag}, the taps that equalised block n,
so the blocks n = r mod lag form independent chains).

At lag 1 W_n = U_{n-1}: both readings are the same schedule, output for
output.  At lag > 1 the chains interleave: every block's update starts from
the taps its own FIR used, and only the taps of block n - lag (not those of
block n - 1) reach it; and the chain keeps the error rate of the sequential
reading on a 1000 km 4D-64 stream."""
import numpy as np

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth

BASE = dict(cd_ps_per_nm=17000.0, n_fft=4096, n_ov=1024, taps=31, bps_phases=64, block=2048, n_pre=2048)


def _stream():
    st = synth.make_stream("gs4d64", 1 << 13, seed=synth.stream_seed(12, 1), esn0_db=13.0,
                           cd_ps_per_nm=17000.0, linewidth_ts=1e-5)
    return st, oracle_format("gs4d64")


def test_lag_one_readings_coincide():
    st, fmt = _stream()
    a = chain.run_chain(st.rx, fmt, chain.RxParams(**BASE, lag=1), ref_bits=st.bits)
    b = chain.run_chain(st.rx, fmt, chain.RxParams(**BASE, lag=1, lms_start=1), ref_bits=st.bits)
    assert np.array_equal(a.llr, b.llr)
    for x, y in zip(a.taps_after, b.taps_after):
        assert np.array_equal(x, y)


def test_independent_chains_wiring_and_error_rate():
    st, fmt = _stream()
    L = 3
    seq = chain.run_chain(st.rx, fmt, chain.RxParams(**BASE, lag=L), ref_bits=st.bits)
    ind = chain.run_chain(st.rx, fmt, chain.RxParams(**BASE, lag=L, lms_start=1), ref_bits=st.bits)
    nblk = len(ind.taps_used)
    for n in range(L, nblk):
        assert np.array_equal(ind.taps_used[n], ind.taps_after[n - L])     # W_n = U_{n-lag}
        assert np.array_equal(seq.taps_used[n], seq.taps_after[n - L])
    # block n's update moved the taps its FIR used (not U_{n-1}): rerun one
    # block's update from each candidate start and keep the one that matches
    p = chain.RxParams(**BASE, lag=L, lms_start=1)
    n = L                                  # the last of the stream's 4 blocks
    span = range(n * p.block, n * p.block + p.n_upd)
    phase = {k: ind.phi[k] for k in span}
    u0 = n * p.n_upd                      # updates before block n (n_upd per block)
    from_w = chain.lms(ind.x, ind.taps_used[n], span, fmt, p, u0=u0, phase=phase)
    from_prev = chain.lms(ind.x, ind.taps_after[n - 1], span, fmt, p, u0=u0, phase=phase)
    assert np.allclose(from_w, ind.taps_after[n], rtol=0, atol=1e-12)
    assert not np.allclose(from_prev, ind.taps_after[n], rtol=0, atol=1e-6)
    assert ind.stats["ber"] <= 1.5 * seq.stats["ber"] + 1e-3
