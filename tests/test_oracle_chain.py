"""End-to-end behaviour of the oracle chain (block schedule, A1-A6)."""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import chain, oracle_format
from paper_2108_07004_gb300 import synth


def test_chain_dp_qpsk_ber_near_awgn_theory():
    """Small DP-QPSK link shaped like the 80 km workload: after CD, rotation
    and phase noise the chain's BER stays within a small penalty of the
    AWGN bound, and sigma^2 estimates N0."""
    fmt = oracle_format("dp_qpsk")
    n = 1 << 15
    st = synth.make_stream("dp_qpsk", n, seed=synth.stream_seed(1), esn0_db=9.0,
                           cd_ps_per_nm=1360.0, linewidth_ts=1e-5)
    p = chain.RxParams(cd_ps_per_nm=1360.0, block=4096, n_pre=4096)
    res = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
    pb = 0.5 * erfc(math.sqrt(10 ** 0.9 / 2))
    assert pb * 0.8 < res.stats["ber"] < pb * 1.6
    # decision-directed estimate: biased low by decision errors at 9 dB
    assert all(0.8 < s / st.n0 < 1.05 for s in res.sigma2[2:])
    # no cycle slip: the unwrapped phase follows the laser phase at the symbol instants
    true = st.phase[0::2]
    off = np.mean(true[:2000] - res.phi[:2000])
    assert np.sqrt(np.mean((res.phi[4096:-512] + off - true[4096:-512]) ** 2)) < 0.1


def test_chain_schedule_lag_and_update_span():
    """The block schedule: W_n = U_{n-lag}; the first lag blocks use W_0."""
    fmt = oracle_format("dp_qpsk")
    n = 1 << 14
    st = synth.make_stream("dp_qpsk", n, seed=21, esn0_db=12.0, cd_ps_per_nm=500.0,
                           linewidth_ts=1e-5)
    for lag in (1, 2):
        p = chain.RxParams(cd_ps_per_nm=500.0, block=2048, n_pre=2048, lag=lag, n_upd=512)
        r = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
        for nb in range(len(r.taps_used)):
            ref = r.w0 if nb < lag else r.taps_after[nb - lag]
            assert np.array_equal(r.taps_used[nb], ref)
        assert r.ranges[0][0] == 0 and r.ranges[-1][1] == n
        for (a0, e0), (a1, e1) in zip(r.ranges, r.ranges[1:]):
            assert e0 == a1                      # ranges tile the stream
        assert r.stats["ber"] < 1e-3


def test_chain_gs4d64_small():
    """The 4D 64-ary format through the 1000 km chain shape (reduced length)."""
    fmt = oracle_format("gs4d64")
    n = 1 << 14
    st = synth.make_stream("gs4d64", n, seed=synth.stream_seed(2, 4), esn0_db=12.0,
                           cd_ps_per_nm=17000.0, linewidth_ts=2e-5)
    p = chain.RxParams(cd_ps_per_nm=17000.0, n_fft=4096, n_ov=1024, taps=31,
                       bps_phases=64, block=4096, n_pre=4096)
    res = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
    # AWGN-only BER of this table at 12 dB is about 7e-3 (exact LLRs, known N0)
    c = chain.count(res.llr[8192:-512], st.bits[8192:-512].astype(float))
    assert c["ber"] < 2e-2 and c["gmi"] > 5.5
    # once DD-LMS runs, the decision-directed sigma^2 estimate is close to N0
    assert abs(res.sigma2[-1] / st.n0 - 1) < 0.1


@pytest.mark.parametrize("lag", [1, 2])
def test_chain_resumes_from_block_state(lag):
    """Nothing but the block-boundary state carries from block to block: a
    run restarted at block n from state_at(n) of a continuous run gives
    that run's taps, phases and LLRs from block n on, exactly."""
    fmt = oracle_format("dp_qpsk")
    n = 10000
    st = synth.make_stream("dp_qpsk", n, seed=22, esn0_db=11.0, cd_ps_per_nm=500.0,
                           linewidth_ts=1e-5)
    p = chain.RxParams(cd_ps_per_nm=500.0, block=2048, n_pre=2048, lag=lag, n_upd=512, n_cma=600)
    full = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
    for nb in (1, 3):
        stt = chain.state_at(full, p, nb)
        part = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits, resume=(nb, stt))
        a = full.ranges[nb][0]
        assert part.ranges[nb:] == full.ranges[nb:]
        assert np.array_equal(part.llr[a:], full.llr[a:])
        assert np.array_equal(part.b[a:], full.b[a:]) and np.array_equal(part.m[a:], full.m[a:])
        for i in range(nb, len(full.taps_after)):
            assert np.array_equal(part.taps_after[i], full.taps_after[i])
        assert np.all(part.llr[:a] == 0)
