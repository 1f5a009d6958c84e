"""Oracle runs for the GPU tests, executed in spawned worker processes.

Test infrastructure only: each job generates one seeded stream with the
shared input generator and runs the FP64 oracle chain on it.  Nothing here
imports torch or the CUDA library, so the workers can be started with
``spawn`` at any point of a GPU test session.
"""
from __future__ import annotations

import os


def chain_job(job: dict):
    """One stream through the oracle: job holds the stream recipe (fmt,
    n_sym, seed, esn0_db, cd_ps_per_nm, linewidth_ts) and the oracle's
    RxParams fields under "params".  Returns (stream, result) with the
    result's CDC output dropped (the comparisons do not use it), and with
    job["valid"] also the near-tie protocol's block_valid of every block."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(k, "1")
    from oracle import chain, oracle_format
    from paper_2108_07004_gb300 import synth
    st = synth.make_stream(job["fmt"], job["n_sym"], seed=job["seed"], esn0_db=job["esn0_db"],
                           cd_ps_per_nm=job["cd_ps_per_nm"], linewidth_ts=job["linewidth_ts"])
    p = chain.RxParams(**job["params"])
    fmt = oracle_format(job["fmt"])
    res = chain.run_chain(st.rx, fmt, p, ref_bits=st.bits)
    res.x = None
    if not job.get("valid"):
        return st, res
    # per block, what the GPU may validly hold (near-tie protocol)
    from parity_protocol import block_valid
    N = res.llr.shape[0]
    return st, res, [block_valid(res, p, fmt, n, N) for n in range(len(res.ranges))]


def run_jobs(jobs: list[dict], workers: int | None = None):
    """The jobs in a spawned process pool (one thread per worker), in order."""
    import multiprocessing as mp
    n = max(1, min(len(jobs), workers or (os.cpu_count() or 1)))
    if n == 1:
        return [chain_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(chain_job, jobs, chunksize=1)
