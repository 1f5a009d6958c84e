#!/usr/bin/env python3
"""Receiver throughput benchmark: Rx line rate in Gbit/s of LLRs out.

Workload (one step): the 4D 64-ary GS format over 1000 km of SSMF
(D*L = 17000 ps/nm), 28 GBd, 2 samples per symbol, a random 2x2
polarisation rotation, laser phase noise linewidth*Ts = 2e-5, and the Es/N0
sweep 8..16 dB in 1 dB steps: 9 independent streams of 2^20 4D symbols,
processed by one handle (FFT 4096 / overlap 1024, 31 taps, BPS with 64
test phases and window 64, blocks of 2^16 symbols with 1024 LMS updates,
tap lag 3: block n is equalised with the taps the LMS made on block n - 3).
Inputs (9 x 32 MiB) are larger than L2, so no flush is used.

value: 9 * 2^20 * 6 LLR bits per step / device time per step.
e2e:   the same metric through rx_process_host (samples and reference bits
       copied in from pinned host memory group by group, LLRs copied out,
       every step).
--impl reference times the FP64 CPU oracle on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2108_07004_gb300 import synth  # noqa: E402

METRIC = "Rx line rate Gbit/s (LLRs out) per GB300 at oracle-matched BER; p99 block latency"
WL = dict(workload="gs4d64_1000km_esn0_8to16dB", fmt="gs4d64", n_sym=1 << 20,
          esn0_db=list(range(8, 17)), cd_ps_per_nm=17000.0, linewidth_ts=2e-5,
          symbol_rate=28e9, sps=2, fft=4096, overlap=1024, taps=31, bps_phases=64,
          bps_window=64, block=1 << 16, n_upd=1024, lag=3, mu=1e-3, n_pre=2048,
          cma_passes=1, n_cma=0, n_train=1024, train_passes=3, skip_head=16384, skip_tail=512)
FP32_LANES_PER_SM, N_SM, SM_MAX_MHZ = 128, 152, 2070.0
# DRAM bytes (read + write) of one bps_kernel launch at this workload's launch
# size (9 streams x one 2^16-symbol block), from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum); reported only while the
# kernel's sources hash to the captured ones.
BPS_TRAFFIC = {"bytes": 9472000, "sources": {
    "paper_2108_07004_gb300/csrc/k_bps.cu": "28310398d330b46577c37a2ba83c36d32628331dcfb0d731a1ca08e2c60e37f2",
    "paper_2108_07004_gb300/csrc/rx_internal.h": "3148d108ac307fe3e65bd256f2a72a17dbafcbfb8de0b60b6acadc0ed407ed64"}}


# DRAM bytes per launch of the KK front-end and of the static equaliser on
# 32 x 2^22 samples (ncu, dram__bytes_read.sum + dram__bytes_write.sum)
KK_TRAFFIC = {"bytes": 1322521256, "sources": {
    "paper_2108_07004_gb300/csrc/k_kk.cu": "03b389bbbbb5c1e2f051f821098ce41c31e2ee55578aa11009cdfa3a2323592a",
    "paper_2108_07004_gb300/csrc/k_kk.h": "05cdf23e99f0a71be65778a0c3732065e56779d3321528217a13afbb237b5906",
    "paper_2108_07004_gb300/csrc/fft_dev.h": "92a928291a79b5288f304fd8c6240edefe3569028d1f823498bb1d7ee0a7ac28"}}
FDE_TRAFFIC = {"bytes": 1580040768, "sources": {
    "paper_2108_07004_gb300/csrc/k_fde.cu": "cec31bdb6e1c3f106427aad676c53ded7e2f6850a3e4c18620845867a90a16dd",
    "paper_2108_07004_gb300/csrc/fft_dev.h": "92a928291a79b5288f304fd8c6240edefe3569028d1f823498bb1d7ee0a7ac28"}}


def issue_peaks(rx_mod, gpu: int) -> dict:
    """Measured FP32 issue rates (lane-instructions/s) of FFMA, FFMA2 and
    FMNMX on this GPU (rx_issue_rate: two blocks of 1024 threads per SM,
    eight independent chains per thread), with the SM clock sampled while
    the probes run; per_sm_clk = rate / (SMs x median SM clock)."""
    import torch
    n_sm = torch.cuda.get_device_properties(gpu).multi_processor_count
    clk = Clocks(gpu)
    clk.start()
    time.sleep(0.3)
    out = {}
    for kind, name in ((0, "ffma"), (1, "ffma2"), (2, "fmnmx")):
        rx_mod.issue_rate(kind, 2048)                        # ramp the clock
        best = max(rx_mod.issue_rate(kind, 8192)[0] for _ in range(5))
        out[name] = best
    clocks = clk.stop()
    mhz = clocks.get("sm_mhz")
    res = {k: {"lane_instr_per_s": v,
               "per_sm_clk": (v / (n_sm * mhz * 1e6)) if mhz else None} for k, v in out.items()}
    res["clocks"] = clocks
    res["sms"] = n_sm
    return res


def pinned_traffic(pin: dict):
    """The captured DRAM bytes while the kernel's sources hash to the captured ones, else None."""
    import hashlib
    for rel, want in pin["sources"].items():
        try:
            with open(os.path.join(ROOT, rel), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != want:
                    return None
        except OSError:
            return None
    return pin["bytes"]


def bps_traffic():
    return pinned_traffic(BPS_TRAFFIC)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


def rank_env():
    """(rank, world size, local rank) of this process under torchrun; (0, 1, 0) alone."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(v: float, device=None) -> float:
    """The largest v over the ranks of the process group (v itself with no
    group): every rank's timed region must have ended for the job's step to
    have, so the job's time per step is the slowest rank's.  The tensor sits
    on `device` (the rank's GPU under NCCL; None: the host, as gloo wants)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(v)
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(rank: int, n_sym: int, n_streams: int):
    rxs, bits = [], []
    for p in range(n_streams):
        st = synth.make_stream(WL["fmt"], n_sym, seed=synth.stream_seed(2, p) + 1000 * rank,
                               esn0_db=WL["esn0_db"][p % len(WL["esn0_db"])],
                               cd_ps_per_nm=WL["cd_ps_per_nm"], linewidth_ts=WL["linewidth_ts"])
        rxs.append(st.rx)
        bits.append(st.bits)
    return np.stack(rxs), np.stack(bits)


def rx_params(wl: dict = WL):
    keys = ["fft", "overlap", "bps_window", "block", "n_upd", "lag", "mu", "n_pre",
            "cma_passes", "n_cma", "n_train", "train_passes", "skip_head", "skip_tail"]
    out = {k: wl[k] for k in keys}
    if wl.get("lms_block", 1) > 1:
        out["lms_block"] = wl["lms_block"]
    if wl.get("widely_linear"):
        out["widely_linear"] = 1
    if wl.get("lms_start"):
        out["lms_start"] = 1
    return out


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu, self.proc, self.f = gpu, None, None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons, n = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            n += 1
            for nm, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": n}


def oracle_params(wl: dict, **over):
    from oracle import chain
    kw = dict(cd_ps_per_nm=wl["cd_ps_per_nm"], n_fft=wl["fft"], n_ov=wl["overlap"], taps=wl["taps"],
              bps_phases=wl["bps_phases"], bps_window=wl["bps_window"], block=wl["block"],
              n_upd=wl["n_upd"], lag=wl["lag"], mu=wl["mu"], n_pre=wl["n_pre"], cma_passes=wl["cma_passes"],
              n_cma=wl["n_cma"], n_train=wl["n_train"], train_passes=wl["train_passes"],
              skip_head=wl["skip_head"], skip_tail=wl["skip_tail"], lms_block=wl.get("lms_block", 1),
              widely_linear=bool(wl.get("widely_linear", 0)), lms_start=int(wl.get("lms_start", 0)))
    kw.update(over)
    return chain.RxParams(**kw)


def cpu_baseline(n_sym: int, wl: dict = WL, esn0_db: float = 12.0, seed: int | None = None):
    """The FP64 oracle as it stands, single process, on one stream of n_sym
    symbols; returns (Gbit/s, seconds, stream, oracle result)."""
    from oracle import chain, oracle_format
    st = synth.make_stream(wl["fmt"], n_sym, seed=seed if seed is not None else synth.stream_seed(2, 4),
                           esn0_db=esn0_db, cd_ps_per_nm=wl["cd_ps_per_nm"], linewidth_ts=wl["linewidth_ts"],
                           iq_imbalance=wl.get("iq"))
    fmt = oracle_format(wl["fmt"])
    t0 = time.perf_counter()
    res = chain.run_chain(st.rx, fmt, oracle_params(wl), ref_bits=st.bits)
    dt = time.perf_counter() - t0
    return n_sym * fmt.m / dt / 1e9, dt, st, res


def _oracle_warm(_):
    """Worker warm-up: import the oracle before the timed region."""
    from oracle import chain, oracle_format  # noqa: F401
    return 0


def _oracle_stream_job(job):
    """One stream through the oracle (a worker of the parallel CPU baseline)."""
    rxs, bits = job
    from oracle import chain, oracle_format
    chain.run_chain(rxs, oracle_format(WL["fmt"]), oracle_params(WL), ref_bits=bits)
    return 0


def cpu_baseline_parallel(n_sym: int):
    """The oracle on the bench's nine Es/N0 points at once, one process per
    stream (spawned, one BLAS/OpenMP thread each) on up to nine host cores:
    the oracle parallelised over streams, its LMS sequential within each.
    Returns (Gbit/s, processes, wall seconds of the timed map)."""
    import multiprocessing as mp
    procs = max(1, min(len(WL["esn0_db"]), os.cpu_count() or 1))
    jobs = []
    for i, e in enumerate(WL["esn0_db"]):
        st = synth.make_stream(WL["fmt"], n_sym, seed=synth.stream_seed(2, 10 + i), esn0_db=float(e),
                               cd_ps_per_nm=WL["cd_ps_per_nm"], linewidth_ts=WL["linewidth_ts"])
        jobs.append((st.rx, st.bits))
    keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in keep:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_oracle_warm, range(procs), chunksize=1)
            t0 = time.perf_counter()
            pool.map(_oracle_stream_job, jobs, chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for k, v in keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return len(jobs) * n_sym * 6 / wall / 1e9, procs, wall


def parity_on(rx_mod, torch, st, res, wl: dict = WL, precision: int = 0):
    """The GPU chain on the oracle's own sample stream (part of the CPU
    baseline leg): LLR error outside BPS near-ties, bit errors, and the EVM
    of the de-rotated symbols against the oracle's."""
    n = st.rx.shape[1] // 2
    r = rx_mod.Receiver(wl["fmt"], cd_ps_per_nm=wl["cd_ps_per_nm"], taps=wl["taps"],
                        bps_phases=wl["bps_phases"], **rx_params(wl), precision=precision)
    r.set_reference(torch.from_numpy(st.bits[None]).cuda())
    x4 = torch.zeros((1, n, 4), dtype=torch.float32, device="cuda")
    r.set_symbol_output(x4, None)
    llr, stats = r.process(torch.from_numpy(st.rx[None]).cuda())
    g = llr[0].cpu().numpy().astype(np.float64)
    zz = x4[0].cpu().numpy().astype(np.float64)
    z = np.stack([zz[:, 0] + 1j * zz[:, 1], zz[:, 2] + 1j * zz[:, 3]])
    ok = res.bps_gap >= 1e-4
    rel = (np.abs(g - res.llr) / np.maximum(1.0, np.abs(res.llr)))[ok]
    ref = res.z[:, ok]
    evm = float(np.sqrt(np.mean(np.abs(z[:, ok] - ref) ** 2) / np.mean(np.abs(ref) ** 2)))
    r.close()
    return {"sample": f"one stream of {n} symbols", "max_rel_llr_err": float(rel.max()),
            "frac_within_1e-4": float(np.mean(rel <= 1e-4)), "evm_vs_oracle": evm,
            "near_tie_symbols": int((~ok).sum()),
            "bit_errors_gpu": int(stats[0]["bit_errors"]), "bit_errors_oracle": int(res.stats["bit_errors"])}


def stage_errors(rx_mod, torch, st, res, wl: dict, precision: int) -> dict:
    """Per-stage error of a storage form against the oracle on its sample:
    EVM of the stored CDC output x (rx_cdc) and of the stored FIR output y
    (rx_fir reading the stored x, with the oracle's taps of block 1)."""
    from oracle import chain
    r = rx_mod.Receiver(wl["fmt"], cd_ps_per_nm=wl["cd_ps_per_nm"], taps=wl["taps"],
                        bps_phases=wl["bps_phases"], **rx_params(wl), precision=precision)
    ns = st.rx.shape[1]
    x_in = torch.from_numpy(st.rx[None]).cuda()
    if precision:
        xs = torch.zeros((1, 2, ns), dtype=torch.int32, device="cuda")
        dt = torch.float16 if precision == 1 else torch.bfloat16

        def unpack(t):
            v = t.view(dt).float().cpu().numpy().astype(np.float64)
            return v[..., 0::2] + 1j * v[..., 1::2]
    else:
        xs = torch.zeros((1, 2, ns), dtype=torch.complex64, device="cuda")

        def unpack(t):
            return t.cpu().numpy().astype(np.complex128)
    r.cdc(x_in, xs)
    x = unpack(xs)[0]
    blk = wl["block"]
    k0, k1 = blk, min(2 * blk, ns // 2)
    taps = res.taps_used[1]
    ys = torch.zeros((1, 2, k1 - k0), dtype=xs.dtype, device="cuda")
    r.fir(xs, torch.from_numpy(taps.astype(np.complex64)[None]).cuda(), k0, k1, ys)
    y = unpack(ys)[0]
    yref = chain.fir(res.x, taps.astype(np.complex64).astype(np.complex128), k0, k1)
    r.close()

    def evm(a, b):
        return float(np.sqrt(np.mean(np.abs(a - b) ** 2) / np.mean(np.abs(b) ** 2)))
    return {"cdc_x_evm": evm(x, res.x), "fir_y_evm": evm(y, yref)}


def run_reference(args):
    rank, _, _ = rank_env()
    if rank != 0:
        return
    n = args.ref_sym
    for _ in range(args.warmup):
        cpu_baseline(n)
    times = []
    for _ in range(args.steps):
        _, dt, _, _ = cpu_baseline(n)
        times.append(dt)
    tot = sum(times)
    val = args.steps * n * 6 / tot / 1e9
    line = {"metric": METRIC, "value": val, "unit": "Gbit/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WL["workload"], "sample_symbols": n, "streams": 1},
            "cpu_baseline": {"value": val, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                             "sample": f"one stream of {n} 4D symbols (12 dB) per step"},
            "e2e": {"value": val, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2108_07004_gb300 import rx as rx_mod

    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    n_sym, S = args.n_sym, args.streams
    F = max(1, args.frames_in_flight)
    rx_h, bits_h = make_inputs(rank, n_sym, S)
    samples = torch.from_numpy(rx_h).cuda()
    bits = torch.from_numpy(bits_h).cuda()
    # F handles, each on a stream of its own; consecutive steps (one complete
    # 9-stream frame each) alternate between them, so one frame's start-up
    # (the sequential CMA and training on 9 SMs) runs beside the previous
    # frame's blocks.  Every step's work is complete; the results of every
    # handle are those of a single handle.
    cur = torch.cuda.current_stream()
    hst = [torch.cuda.Stream() for _ in range(F)]
    rs = []
    for i in range(F):
        ri = rx_mod.Receiver(WL["fmt"], cd_ps_per_nm=WL["cd_ps_per_nm"], taps=WL["taps"],
                             bps_phases=WL["bps_phases"], streams=S, stream=hst[i], **rx_params())
        ri.set_reference(bits)
        rs.append(ri)
    r = rs[0]
    llrs = [torch.empty((S, n_sym, 6), dtype=torch.float32, device="cuda") for _ in range(F)]
    llr = llrs[0]

    def steps(k, handles):
        for s_ in hst[:handles]:
            s_.wait_stream(cur)
        for i in range(k):
            rs[i % handles].process(samples, llrs[i % handles], stats=False)
        for s_ in hst[:handles]:
            cur.wait_stream(s_)

    # with frames in flight each handle sizes its one-wave grids to leave SMs
    # to the other frames (their LMS blocks and their main-stream kernels)
    reserve = 2 * S * (F - 1)
    for ri in rs:
        ri.set("sm_reserve", reserve)
    # timed steps: CUDA events around the BPS launches only (the roofline's
    # live kernel time); the stage breakdown comes from profiled steps after
    for ri in rs:
        ri.set("profile", 2)
    steps(max(args.warmup, F), F)
    torch.cuda.synchronize()
    # the roofline's denominator, measured on this GPU before the timed steps
    ipk = issue_peaks(rx_mod, local) if rank == 0 else None
    steps(2 * F, F)
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(cur)
    steps(args.steps, F)
    ev1.record(cur)
    torch.cuda.synchronize()
    barrier()
    clocks = clk.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    stats = r.stats()
    bps_live = r.profile("bps")                 # last timed step of handle 0
    launches_per_step = r.launches()
    same = all(torch.equal(llrs[0], l_) for l_ in llrs[1:])
    # one frame at a time (one handle, no SMs left out), the same steps
    ms_one, bps_live_one = None, None
    if F > 1:
        r.set("sm_reserve", 0)
        r.set("profile", 2)
        steps(2, 1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(cur)
        steps(args.steps, 1)
        e1.record(cur)
        torch.cuda.synchronize()
        ms_one = e0.elapsed_time(e1) / args.steps
        bps_live_one = r.profile("bps")         # last step, one frame at a time
    r.set("profile", 1)                         # untimed: every stage and block
    for _ in range(2):
        r.process(samples, llr, stats=False)
    stage = {s: r.profile(s) for s in ("cdc", "fir", "bps", "unwrap", "demap", "lms", "startup")}
    lat = sorted(r.block_latency())
    r.set("profile", 0)
    ms = max_over_ranks(ms, device="cuda")
    bits_per_step = S * n_sym * 6 * world
    value = bits_per_step / (ms * 1e-3) / 1e9

    # ---- end to end through the host-buffer entry point ----
    e2e = None
    if not args.no_e2e:
        import threading
        s_h = torch.from_numpy(rx_h).pin_memory()
        b_h = torch.from_numpy(bits_h).pin_memory()
        l_hs = [torch.empty((S, n_sym, 6), dtype=torch.float32).pin_memory() for _ in range(F)]
        for ri in rs:
            ri.set("profile", 0)
            ri.set("sm_reserve", reserve)
        ke = max(3, args.steps // 4)

        def host_steps(i, k):
            # one host thread per handle (the entry point returns when the
            # LLRs are in host memory); the GIL is released inside the call
            torch.cuda.set_device(local)
            for _ in range(k):
                rs[i].set_reference_host(b_h)
                rs[i].process_host(s_h, l_hs[i], stats=False)

        def run_host(k):
            th = [threading.Thread(target=host_steps, args=(i, k)) for i in range(F)]
            for t_ in th:
                t_.start()
            for t_ in th:
                t_.join()

        run_host(2)
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        run_host(ke)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / (ke * F)
        l_h = l_hs[0]
        dt = max_over_ranks(dt, device="cuda")
        e2e = {"value": bits_per_step / dt / 1e9, "unit": "Gbit/s",
               "h2d_bytes_per_step": int(rx_h.nbytes + bits_h.nbytes),
               "d2h_bytes_per_step": int(l_h.numel() * 4), "ms_per_step": dt * 1e3}

    if rank != 0:
        return
    pk, pk_kind = peaks()
    bps_ms, bps_n = bps_live
    ops = S * n_sym * WL["bps_phases"] * 64            # candidate (phase, point) distances
    # peak: one candidate per FP32 lane-instruction at the measured FFMA
    # issue rate (the nominal 128 lanes x SMs x max clock if the probe fails)
    peak_ops = FP32_LANES_PER_SM * N_SM * SM_MAX_MHZ * 1e6 / 1e12
    peak_from = "nominal: 128 FP32 lanes x 152 SMs x 2070 MHz (probe unavailable)"
    if ipk and ipk["ffma"]["lane_instr_per_s"] > 0:
        peak_ops = ipk["ffma"]["lane_instr_per_s"] / 1e12
        c = ipk["clocks"]
        peak_from = (f"measured: FFMA issue probe (rx_issue_rate), "
                     f"{ipk['ffma']['per_sm_clk']:.1f} lane-instr/SM/clk at {c.get('sm_mhz')} MHz median"
                     if ipk["ffma"]["per_sm_clk"] else "measured: FFMA issue probe (rx_issue_rate)")
    achieved = ops / (bps_ms * 1e-3) / 1e12 if bps_ms > 0 else None
    # the same kernel's live rate when one frame runs at a time (its launches
    # then share the SMs only with the same frame's demap)
    ach_one = (ops / (bps_live_one[0] * 1e-3) / 1e12 if bps_live_one and bps_live_one[0] > 0 else None)
    cdc_ms = stage["cdc"][0]
    cdc_bytes = S * 2 * 2 * n_sym * 8 * (WL["fft"] / (WL["fft"] - WL["overlap"]) + 1)
    line = {
        "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WL["workload"], "streams": S, "symbols_per_stream": n_sym,
                   "format": WL["fmt"], "fft": WL["fft"], "overlap": WL["overlap"],
                   "taps": WL["taps"], "bps_phases": WL["bps_phases"], "block": WL["block"],
                   "lag": WL["lag"], "l2": "inputs 9 x 32 MiB > L2, no flush",
                   "frames_in_flight": F, "sm_reserve": 2 * S * (F - 1)},
        "one_frame_at_a_time": ({"value": bits_per_step / (ms_one * 1e-3) / 1e9, "ms_per_step": ms_one}
                                if ms_one else None),
        "frames_identical": same,
        "latency": {"block_p50_ms": lat[len(lat) // 2] if lat else None,
                    "block_p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
                    "blocks_per_step": len(lat)},
        "roofline": {"bound": "alu", "kernel": "bps", "achieved": achieved, "peak": peak_ops,
                     "unit": "Top/s", "frac": (achieved / peak_ops) if achieved else None,
                     "traffic": bps_traffic() if n_sym == WL["n_sym"] and S == 9 else None,
                     "op": "one (test phase, constellation point) candidate distance",
                     "peak_from": peak_from,
                     "frac_one_frame_at_a_time": (ach_one / peak_ops) if ach_one else None,
                     "issue_probe": ipk},
        "realtime_channels": value / (WL["symbol_rate"] * 6 / 1e9),
        "stages_ms": {k: v[0] for k, v in stage.items()},
        "stage_hbm": {"cdc": {"achieved_gbs": cdc_bytes / (cdc_ms * 1e-3) / 1e9 if cdc_ms else None,
                              "peak_gbs": pk.get("hbm_gbs"), "peak_kind": pk_kind}},
        "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clocks,
        "stats": [{"esn0_db": WL["esn0_db"][i % 9], "ber": s["ber"], "gmi": s["gmi"],
                   "sigma2": s["sigma2_last"]} for i, s in enumerate(stats)],
    }
    if e2e:
        line["e2e"] = e2e
    if not args.no_cpu_baseline and world == 1:
        # CPU baseline leg: the oracle timed on a sample, and the GPU chain
        # checked against the oracle's result on that same sample
        v, dt, st_o, res_o = cpu_baseline(args.cpu_sym)
        line["cpu_baseline"] = {"value": v, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                "sample": f"one stream of {args.cpu_sym} 4D symbols (12 dB), "
                                          f"{dt:.1f} s"}
        if not args.no_parity:
            line["parity"] = parity_on(rx_mod, torch, st_o, res_o)
        vp, procs, wall = cpu_baseline_parallel(args.cpu_sym // 4)
        line["cpu_baseline_parallel"] = {"value": vp, "unit": "Gbit/s", "cores": procs, "kind": "oracle",
                                         "sample": f"the nine Es/N0 streams of {args.cpu_sym // 4} 4D symbols, "
                                                   f"one process each, {wall:.1f} s wall"}
    print(json.dumps(line), flush=True)


# ---- precision variant (config 3): DP-QPSK, 80 km, CDC/FIR data in half / bfloat16 ----
WL3 = dict(workload="dp_qpsk_80km_12dB_2p24_symbols", fmt="dp_qpsk", n_sym=1 << 20, streams=16, esn0_db=12.0,
           cd_ps_per_nm=1360.0, linewidth_ts=1e-5, symbol_rate=28e9, sps=2, fft=1024, overlap=256, taps=15,
           bps_phases=32, bps_window=64, block=1 << 16, n_upd=1024, lag=3, mu=1e-3, n_pre=2048, cma_passes=1,
           n_cma=0, n_train=1024, train_passes=3, skip_head=16384, skip_tail=512, lms_start=1)


def chain_bytes_per_symbol(wl: dict, store: int) -> float:
    """Algorithmic HBM bytes per 4D symbol of the stage-separated chain, with
    x and y stored in `store` bytes per complex sample: CDC reads the c64
    input (overlap re-read) and writes x; FIR reads x, writes y; BPS reads y,
    writes the phase index; de-rotation/demap reads y and the index, writes
    the phase code and the float32 LLRs."""
    m = 4 if wl["fmt"] == "dp_qpsk" else (8 if wl["fmt"] == "dp_16qam" else 6)
    ovl = wl["fft"] / (wl["fft"] - wl["overlap"])
    return (32 * ovl + 4 * store) + (4 * store + 2 * store) + (2 * store + 1) + (2 * store + 1 + 2 + 4 * m)


def timed_steps(r, samples, llr, steps: int, warmup: int, r2=None, llr2=None):
    """Device ms per step (CUDA events, library events around the BPS
    launches only), then the stage breakdown of one profiled step and the
    statistics.  With a second handle r2 (on a stream of its own, as r's)
    consecutive steps alternate between the two, two frames in flight."""
    import torch
    rs, ls = ([r, r2], [llr, llr2]) if r2 is not None else ([r], [llr])
    cur = torch.cuda.current_stream()
    for ri in rs:
        ri.set("profile", 2)

    def run(k):
        for ri in rs:
            ri.stream.wait_stream(cur)
        for i in range(k):
            rs[i % len(rs)].process(samples, ls[i % len(rs)], stats=False)
        for ri in rs:
            cur.wait_stream(ri.stream)

    run(max(warmup, len(rs)))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    run(steps)
    e1.record(cur)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    for ri in rs[1:]:
        ri.set("profile", 0)
    st_ = r.stats()
    r.set("profile", 1)
    r.process(samples, llr, stats=False)
    stg = {k: r.profile(k)[0] for k in ("cdc", "fir", "bps", "demap", "lms", "startup")}
    r.set("profile", 0)
    return ms, stg, st_


# ---- block LMS (next row F2): groups of P updates share the taps at the group start ----
BLOCK_LMS = dict(P=(1, 4, 16, 64), lag=(1, 2, 3), cpu_P=16)


def run_block_lms(args):
    """The bench workload with the block-wise tap updates in groups of P
    (P = 1: the exact recursion) for tap lags 1..3: Gbit/s, the LMS stage's
    device time per block and the bit errors over the 9 streams."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n_sym, S = args.n_sym, args.streams
    rx_h, bits_h = make_inputs(0, n_sym, S)
    samples = torch.from_numpy(rx_h).cuda()
    bits = torch.from_numpy(bits_h).cuda()
    del rx_h
    m = 6
    nblk = (n_sym + WL["block"] - 1) // WL["block"]
    sweep = []
    for lag in BLOCK_LMS["lag"]:
        for P in BLOCK_LMS["P"]:
            wl = dict(WL, lag=lag, lms_block=P)
            r = rx_mod.Receiver(WL["fmt"], cd_ps_per_nm=WL["cd_ps_per_nm"], taps=WL["taps"],
                                bps_phases=WL["bps_phases"], streams=S, **rx_params(wl))
            r.set_reference(bits)
            llr = torch.empty((S, n_sym, m), dtype=torch.float32, device="cuda")
            ms, stg, st_ = timed_steps(r, samples, llr, args.steps, args.warmup)
            sweep.append({"lms_block": P, "lag": lag, "gbps": S * n_sym * m / (ms * 1e-3) / 1e9,
                          "ms_per_step": ms, "lms_ms_per_block": stg["lms"] / nblk,
                          "main_ms_per_block": (stg["fir"] + stg["bps"] + stg["demap"]) / nblk,
                          "bit_errors": int(sum(x["bit_errors"] for x in st_)),
                          "n_bits": int(sum(x["n_bits"] for x in st_)),
                          "ber_12db": st_[4]["ber"]})
            r.close()
    ex = {(e["lag"], e["lms_block"]): e for e in sweep}
    for e in sweep:
        base = ex[(e["lag"], 1)]["bit_errors"]
        e["ber_delta_rel_vs_exact"] = (e["bit_errors"] - base) / max(base, 1)
    head = ex[(1, 16)]
    line = {
        "metric": METRIC, "value": head["gbps"], "unit": "Gbit/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WL["workload"] + "_block_lms", "streams": S, "symbols_per_stream": n_sym,
                   "format": WL["fmt"], "taps": WL["taps"], "bps_phases": WL["bps_phases"],
                   "block": WL["block"], "lag": 1, "lms_block": 16},
        "sweep": sweep,
    }
    if not args.no_cpu_baseline:
        wl = dict(WL, lag=1, lms_block=BLOCK_LMS["cpu_P"])
        v, dt, st_o, res_o = cpu_baseline(args.cpu_sym, wl, 12.0)
        line["cpu_baseline"] = {"value": v, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                "sample": f"one stream of {args.cpu_sym} 4D symbols (12 dB), block LMS P = "
                                          f"{BLOCK_LMS['cpu_P']}, {dt:.1f} s"}
        if not args.no_parity:
            line["parity"] = parity_on(rx_mod, torch, st_o, res_o, wl)
    print(json.dumps(line), flush=True)


# ---- widely-linear butterfly (next row F3): DP-16QAM with a transmitter IQ imbalance ----
# no carrier phase noise: the regime of the paper's widely-linear equaliser (its KK receiver
# has none); with phase noise the conjugate term turns against the carrier before the phase
# search and a butterfly in front of it cannot hold its conjugate taps
WLIN = dict(workload="dp_16qam_80km_18dB_iq15pct_no_phase_noise", fmt="dp_16qam", n_sym=1 << 20, streams=9,
            esn0_db=18.0, cd_ps_per_nm=1360.0, linewidth_ts=0.0, iq=(0.15, 0.12), fft=1024, overlap=256,
            taps=15, bps_phases=32, bps_window=64, block=1 << 16, n_upd=1024, lag=2, mu=1e-3, n_pre=4096,
            cma_passes=1, n_cma=0, n_train=1024, train_passes=3, skip_head=65536, skip_tail=512)


def run_widely_linear(args):
    """Nine DP-16QAM streams with a transmitter IQ imbalance (15 %, 0.12 rad):
    the linear butterfly, the widely-linear one, and the linear one on the
    same streams without the imbalance; Gbit/s and bit errors of each."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl0 = WLIN
    S = wl0["streams"]
    n = args.n_sym if args.n_sym != WL["n_sym"] else wl0["n_sym"]
    m = 8
    forms = {}
    for name, iq, wlin in (("linear", wl0["iq"], 0), ("widely_linear", wl0["iq"], 1), ("linear_no_iq", None, 0)):
        rxs, bits = [], []
        for p_ in range(S):
            st = synth.make_stream(wl0["fmt"], n, seed=synth.stream_seed(14, p_), esn0_db=wl0["esn0_db"],
                                   cd_ps_per_nm=wl0["cd_ps_per_nm"], linewidth_ts=wl0["linewidth_ts"],
                                   iq_imbalance=iq)
            rxs.append(st.rx)
            bits.append(st.bits)
        samples = torch.from_numpy(np.stack(rxs)).cuda()
        bits_d = torch.from_numpy(np.stack(bits)).cuda()
        del rxs
        wcfg = dict(wl0, widely_linear=wlin)
        r = rx_mod.Receiver(wl0["fmt"], cd_ps_per_nm=wl0["cd_ps_per_nm"], taps=wl0["taps"],
                            bps_phases=wl0["bps_phases"], streams=S, **rx_params(wcfg))
        r.set_reference(bits_d)
        llr = torch.empty((S, n, m), dtype=torch.float32, device="cuda")
        ms, stg, st_ = timed_steps(r, samples, llr, args.steps, args.warmup)
        forms[name] = {"gbps": S * n * m / (ms * 1e-3) / 1e9, "ms_per_step": ms, "stages_ms": stg,
                       "bit_errors": int(sum(x["bit_errors"] for x in st_)),
                       "n_bits": int(sum(x["n_bits"] for x in st_)),
                       "ber": sum(x["bit_errors"] for x in st_) / max(1, sum(x["n_bits"] for x in st_))}
        r.close()
        del samples, bits_d, llr
    head = forms["widely_linear"]
    line = {
        "metric": METRIC, "value": head["gbps"], "unit": "Gbit/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": wl0["workload"], "streams": S, "symbols_per_stream": n, "format": wl0["fmt"],
                   "fft": wl0["fft"], "overlap": wl0["overlap"], "taps": wl0["taps"],
                   "bps_phases": wl0["bps_phases"], "block": wl0["block"], "lag": wl0["lag"],
                   "iq_imbalance": list(wl0["iq"]), "widely_linear": 1},
        "forms": forms,
    }
    if not args.no_cpu_baseline:
        wcfg = dict(wl0, widely_linear=1)
        v, dt, st_o, res_o = cpu_baseline(1 << 16, wcfg, wl0["esn0_db"], synth.stream_seed(14, 99))
        line["cpu_baseline"] = {"value": v, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                "sample": f"one stream of 65536 16QAM symbols with the IQ imbalance, widely "
                                          f"linear, {dt:.1f} s"}
        if not args.no_parity:
            line["parity"] = parity_on(rx_mod, torch, st_o, res_o, wcfg)
    print(json.dumps(line), flush=True)


# ---- GS-128 (Sec. 5's 128-point 2D format) through the chain ----
WGS128 = dict(workload="gs128_500km_24dB_9x2p20", fmt="gs128", n_sym=1 << 20, streams=9, esn0_db=24.0,
              cd_ps_per_nm=8500.0, linewidth_ts=1e-6, symbol_rate=28e9, sps=2, fft=1024, overlap=256,
              taps=15, bps_phases=64, bps_window=64, block=1 << 16, n_upd=1024, lag=3, lms_start=1,
              mu=1e-3, n_pre=2048, cma_passes=1, n_cma=0, n_train=1024, train_passes=3, skip_head=16384,
              skip_tail=512)


def run_gs128(args):
    """Nine streams of the 2D 128-point GS format at 24 dB (500 km, lag 3 with
    independent LMS chains): Gbit/s of LLRs (14 bits per 4D symbol), the
    bit-error rate, and the oracle on one stream.  At the format's 20 dB
    design point the blind phase search (64 test phases, 64-symbol window)
    slips quadrants within 2^18 symbols, in the oracle as on the GPU; at 22
    and 24 dB the oracle holds the quadrant over 2^18 symbols."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl = WGS128
    S = wl["streams"]
    n = args.n_sym if args.n_sym != WL["n_sym"] else wl["n_sym"]
    m = 14
    rxs, bits = [], []
    for p_ in range(S):
        st = synth.make_stream(wl["fmt"], n, seed=synth.stream_seed(16, p_), esn0_db=wl["esn0_db"],
                               cd_ps_per_nm=wl["cd_ps_per_nm"], linewidth_ts=wl["linewidth_ts"])
        rxs.append(st.rx)
        bits.append(st.bits)
    samples = torch.from_numpy(np.stack(rxs)).cuda()
    bits_d = torch.from_numpy(np.stack(bits)).cuda()
    del rxs
    r = rx_mod.Receiver(wl["fmt"], cd_ps_per_nm=wl["cd_ps_per_nm"], taps=wl["taps"], bps_phases=wl["bps_phases"],
                        streams=S, **rx_params(wl))
    r.set_reference(bits_d)
    llr = torch.empty((S, n, m), dtype=torch.float32, device="cuda")
    ms, stg, st_ = timed_steps(r, samples, llr, args.steps, args.warmup)
    nb = sum(x["n_bits"] for x in st_)
    line = {
        "metric": METRIC, "value": S * n * m / (ms * 1e-3) / 1e9, "unit": "Gbit/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl["workload"], "streams": S, "symbols_per_stream": n, "format": wl["fmt"],
                   "fft": wl["fft"], "overlap": wl["overlap"], "taps": wl["taps"],
                   "bps_phases": wl["bps_phases"], "block": wl["block"], "lag": wl["lag"], "lms_start": 1,
                   "esn0_db": wl["esn0_db"]},
        "stages_ms": stg,
        "ber": sum(x["bit_errors"] for x in st_) / max(1, nb),
        "gmi_per_4d_symbol": float(np.mean([x["gmi"] for x in st_])),
        "gpu_launches": None,
    }
    if not args.no_cpu_baseline:
        v, dt, st_o, res_o = cpu_baseline(1 << 14, wl, wl["esn0_db"], synth.stream_seed(16, 99))
        line["cpu_baseline"] = {"value": v, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                "sample": f"one stream of 16384 GS-128 symbols, {dt:.1f} s"}
        if not args.no_parity:
            line["parity"] = parity_on(rx_mod, torch, st_o, res_o, wl)
    r.close()
    print(json.dumps(line), flush=True)


# ---- Kramers-Kronig receiver front-end (Sec. 2): 32 streams of 2^22 ADC samples ----
KKW = dict(workload="kk_frontend_fde_32x2p22", streams=32, n=1 << 22, distinct=4, fmt="dp_16qam", cspr_db=14.0,
           esn0_db=25.0, n_ov=512, floor=1e-3, fde_taps=203, fde_ov=256, n_train=4096)


def _event_ms(fn, steps, warmup):
    import torch
    for _ in range(max(3, warmup)):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_kk(args):
    """The paper's receiver front-end as two FFT-pair kernels per step: the
    KK front-end (int16 ADC codes at 4 samples per symbol -> downconverted
    field, complex64) and the trained 203-tap static equaliser with 4 -> 2
    resampling, over 32 streams of 2^22 samples (the paper's buffer size);
    GSa/s of ADC samples in.  The equaliser is trained once beforehand
    (float64 least squares on 4096 known symbols of stream 0)."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = KKW
    S, n = w["streams"], w["n"]
    ks = [synth.make_kk_stream(w["fmt"], n // 4, seed=synth.stream_seed(15, p_), cspr_db=w["cspr_db"],
                               esn0_db=w["esn0_db"]) for p_ in range(w["distinct"])]
    codes_h = np.stack([ks[p_ % w["distinct"]].codes for p_ in range(S)])
    levels = np.array([[ks[p_ % w["distinct"]].scale, ks[p_ % w["distinct"]].dc] for p_ in range(S)],
                      dtype=np.float32)
    codes = torch.from_numpy(codes_h).cuda()
    field = torch.empty((S, n), dtype=torch.complex64, device="cuda")
    y = torch.empty((S, n // 2), dtype=torch.complex64, device="cuda")
    k = rx_mod.KK(ks[0].fc_step, n_ov=w["n_ov"], floor=w["floor"])
    e = rx_mod.FDE(w["fde_taps"], w["fde_ov"])
    k.field(codes, levels, field)
    d = torch.from_numpy(ks[0].sym[:w["n_train"]].astype(np.complex64)).cuda()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    e.train(field[0], d)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)

    ms_kk = _event_ms(lambda: k.field(codes, levels, field), args.steps, args.warmup)
    ms_fde = _event_ms(lambda: e.apply(field, y), args.steps, args.warmup)

    def step():
        k.field(codes, levels, field)
        e.apply(field, y)

    clk = Clocks(torch.cuda.current_device())
    clk.start()
    ms = _event_ms(step, args.steps, args.warmup)
    clocks = clk.stop()
    value = S * n / (ms * 1e-3) / 1e9
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    b_kk, b_fde = 2 + 8, 8 + 4                     # algorithmic bytes per ADC sample
    kern = {"kk1024": {"ms": ms_kk, "gsa_s": S * n / (ms_kk * 1e-3) / 1e9, "bytes_per_sample": b_kk,
                       "hbm_frac": S * n * b_kk / (ms_kk * 1e-3) / 1e9 / hbm, "traffic": pinned_traffic(KK_TRAFFIC)},
            "fde1024": {"ms": ms_fde, "gsa_s": S * n / (ms_fde * 1e-3) / 1e9, "bytes_per_sample": b_fde,
                        "hbm_frac": S * n * b_fde / (ms_fde * 1e-3) / 1e9 / hbm,
                        "traffic": pinned_traffic(FDE_TRAFFIC)}}
    top = max(kern, key=lambda q: kern[q]["ms"])
    alg = S * n * kern[top]["bytes_per_sample"]
    line = {
        "metric": "KK receiver front-end (KK field + trained static equaliser with 4->2 resampling) ADC samples "
                  "per second", "value": value, "unit": "GSa/s", "n_gpus": 1,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["workload"], "streams": S, "samples_per_stream": n, "sps": 4, "fft": 1024,
                   "kk_overlap": w["n_ov"], "fde_taps": w["fde_taps"], "fde_overlap": w["fde_ov"],
                   "format": w["fmt"], "cspr_db": w["cspr_db"],
                   "l2": "inputs 256 MiB, field 1 GiB, output 512 MiB > L2, no flush"},
        "realtime_1gbd_channels": value / 4.0, "fde_train_ms": train_ms, "kernels": kern,
        "roofline": {"bound": "hbm", "kernel": top, "achieved": alg / (kern[top]["ms"] * 1e-3) / 1e9, "peak": hbm,
                     "unit": "GB/s", "frac": alg / (kern[top]["ms"] * 1e-3) / 1e9 / hbm,
                     "traffic": kern[top]["traffic"], "peak_kind": pk_kind},
        "gpu_launches": 2 * args.steps, "clocks": clocks,
    }
    # end to end: pinned host codes in, equalised 2-sps output out, every step
    if not args.no_e2e:
        c_h = torch.from_numpy(codes_h).pin_memory()
        o_h = torch.empty((S, n // 2), dtype=torch.complex64).pin_memory()

        def e2e_step():
            codes.copy_(c_h, non_blocking=True)
            step()
            o_h.copy_(y, non_blocking=True)
        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ke = max(3, args.steps // 4)
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / ke
        line["e2e"] = {"value": S * n / dt / 1e9, "unit": "GSa/s", "h2d_bytes_per_step": int(codes_h.nbytes),
                       "d2h_bytes_per_step": int(o_h.numel() * 8), "ms_per_step": dt * 1e3}
    if not args.no_cpu_baseline:
        from oracle import fde as ofde, kk as okk
        ns = 1 << 20
        t0 = time.perf_counter()
        ref_x = okk.kk_field_from_codes(ks[0].codes[:ns], scale=float(levels[0, 0]), dc=float(levels[0, 1]),
                                        fc_step=ks[0].fc_step, n_ov=w["n_ov"], floor=float(np.float32(w["floor"])))
        h_ref = e.taps()
        ref_y = ofde.apply(ref_x, h_ref, n_ov=w["fde_ov"])
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns / dt / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
                                "sample": f"the first {ns} samples of one stream (KK field, then the equaliser "
                                          f"with the GPU-trained taps), {dt:.1f} s"}
        if not args.no_parity:
            g = field[0, :ns - 1024].cpu().numpy()
            r_ = ref_x[:ns - 1024]
            err = np.abs(g - r_) / (ks[0].carrier + np.abs(r_))
            gy = y[0, :ns // 2 - 1024].cpu().numpy()
            ry = ref_y[:ns // 2 - 1024]
            rms = np.sqrt(np.mean(np.abs(ry) ** 2))
            line["parity"] = {"sample": f"stream 0, the first {ns - 1024} field / {ns // 2 - 1024} output samples",
                              "kk_max_err_rel_carrier": float(err.max()), "kk_tolerance": 2e-5,
                              "fde_max_err_rel_rms": float(np.max(np.abs(gy - ry)) / rms),
                              "fde_note": "the equaliser input differs from the oracle's by the KK rounding"}
    print(json.dumps(line), flush=True)


# ---- the paper's KK receiver end to end: KK front-end -> static equaliser -> chain ----
KKC = dict(workload="kk_receiver_dp16qam_16x2p20", fmt="dp_16qam", pairs=16, n_sym=1 << 20, distinct=4,
           cspr_db=14.0, esn0_db=20.0, kk_ov=512, floor=1e-3, fde_taps=203, fde_ov=256, fde_train=4096,
           cd_ps_per_nm=0.0, fft=1024, overlap=256, taps=15, bps_phases=32, bps_window=64, block=1 << 16,
           n_upd=1024, lag=3, mu=1e-3, n_pre=4096, cma_passes=1, n_cma=0, n_train=1024, train_passes=3,
           skip_head=16384, skip_tail=512, lms_start=1)


def _kk_pipeline_gpu(rx_mod, torch, w, codes, levels, fc_step, bits, d_train, pairs, n_sym):
    """KK, equaliser (trained on KK stream 0) and chain objects plus their buffers."""
    k = rx_mod.KK(fc_step, n_ov=w["kk_ov"], floor=w["floor"])
    e = rx_mod.FDE(w["fde_taps"], w["fde_ov"])
    field = torch.empty(tuple(codes.shape), dtype=torch.complex64, device="cuda")
    y = torch.empty((codes.shape[0], codes.shape[1] // 2), dtype=torch.complex64, device="cuda")
    k.field(codes, levels, field)
    e.train(field[0], d_train)
    r = rx_mod.Receiver(w["fmt"], cd_ps_per_nm=0.0, taps=w["taps"], bps_phases=w["bps_phases"], streams=pairs,
                        **rx_params(w), matched_filter=0)
    r.set_reference(bits)
    llr = torch.empty((pairs, n_sym, 8), dtype=torch.float32, device="cuda")
    return k, e, r, field, y, llr


def run_kk_chain(args):
    """The paper's receiver order on the GPU (Sec. 2): KK front-end (int16
    ADC codes at 4 samples per symbol -> field), trained 203-tap static
    equaliser with 4 -> 2 resampling, then the chain (butterfly LMS, phase
    search, exact LLRs, counting) with two single-polarisation KK signals as
    the X and Y of one stream and the CDC reduced to the identity.  32 KK
    signals of 2^20 16QAM symbols (CSPR 14 dB, Es/N0 20 dB) = 16 streams;
    Gbit/s of LLRs out."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = KKC
    P, n = w["pairs"], w["n_sym"]
    ks = [synth.make_kk_stream(w["fmt"], n, seed=synth.stream_seed(16, q), cspr_db=w["cspr_db"],
                               esn0_db=w["esn0_db"]) for q in range(w["distinct"])]
    src = [q % w["distinct"] for q in range(2 * P)]
    codes = torch.from_numpy(np.stack([ks[q].codes for q in src])).cuda()
    levels = np.array([[ks[q].scale, ks[q].dc] for q in src], dtype=np.float32)
    bits = torch.from_numpy(np.stack([np.concatenate([ks[src[2 * i]].bits, ks[src[2 * i + 1]].bits], axis=1)
                                      for i in range(P)])).cuda()
    d_train = torch.from_numpy(ks[0].sym[:w["fde_train"]].astype(np.complex64)).cuda()
    k, e, r, field, y, llr = _kk_pipeline_gpu(rx_mod, torch, w, codes, levels, ks[0].fc_step, bits, d_train, P, n)
    yv = y.view(P, 2, 2 * n)

    def step():
        k.field(codes, levels, field)
        e.apply(field, y)
        r.process(yv, llr, stats=False)

    ms_kk = _event_ms(lambda: k.field(codes, levels, field), args.steps, args.warmup)
    ms_fde = _event_ms(lambda: e.apply(field, y), args.steps, args.warmup)
    ms_chain = _event_ms(lambda: r.process(yv, llr, stats=False), args.steps, args.warmup)
    clk = Clocks(torch.cuda.current_device())
    clk.start()
    ms = _event_ms(step, args.steps, args.warmup)
    clocks = clk.stop()
    _, stats = r.process(yv, llr)
    bits_per_step = P * n * 8
    value = bits_per_step / (ms * 1e-3) / 1e9
    nb = sum(x["n_bits"] for x in stats)
    ne = sum(x["bit_errors"] for x in stats)
    line = {
        "metric": "KK receiver (KK front-end + static equaliser + chain) Gbit/s of LLRs out", "value": value,
        "unit": "Gbit/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["workload"], "kk_signals": 2 * P, "streams": P, "symbols_per_stream": n,
                   "format": w["fmt"], "cspr_db": w["cspr_db"], "esn0_db": w["esn0_db"], "sps_in": 4,
                   "kk_fft": 1024, "kk_overlap": w["kk_ov"], "fde_taps": w["fde_taps"], "taps": w["taps"],
                   "bps_phases": w["bps_phases"], "block": w["block"], "lag": w["lag"], "lms_start": w["lms_start"],
                   "l2": "inputs 256 MiB, field 1 GiB > L2, no flush"},
        "stages_ms": {"kk": ms_kk, "fde": ms_fde, "chain": ms_chain},
        "ber": ne / max(nb, 1), "bit_errors": int(ne), "n_bits": int(nb),
        "gpu_launches": None, "clocks": clocks,
    }
    r.set("profile", 1)
    r.process(yv, llr, stats=False)
    torch.cuda.synchronize()
    line["gpu_launches"] = 2 + int(r.launches())
    r.set("profile", 0)
    if not args.no_cpu_baseline:
        from oracle import chain, fde as ofde, kk as okk, oracle_format
        ns_sym = 1 << 15
        t0 = time.perf_counter()
        ys_o = []
        for q in (0, 1):
            x_o = okk.kk_field_from_codes(ks[q].codes[:4 * ns_sym], scale=ks[q].scale, dc=ks[q].dc,
                                          fc_step=ks[q].fc_step, n_ov=w["kk_ov"], floor=float(np.float32(w["floor"])))
            h_o = ofde.train(x_o, ks[0].sym[:w["fde_train"]] if q == 0 else ks[q].sym[:w["fde_train"]])
            ys_o.append(ofde.apply(x_o, h_o, n_ov=w["fde_ov"]))
        b_o = np.concatenate([ks[0].bits[:ns_sym], ks[1].bits[:ns_sym]], axis=1)
        res = chain.run_chain(np.stack(ys_o).astype(np.complex64), oracle_format(w["fmt"]),
                              oracle_params(w, matched_filter=False), ref_bits=b_o)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": ns_sym * 8 / dt / 1e9, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                "sample": f"one stream (two KK signals) of {ns_sym} symbols through the KK front-end, "
                                          f"equaliser training and application and the chain, {dt:.1f} s"}
        if not args.no_parity:
            c2 = torch.from_numpy(np.stack([ks[0].codes[:4 * ns_sym], ks[1].codes[:4 * ns_sym]])).cuda()
            l2 = levels[:2]
            k2, e2, r2, f2, y2, llr2 = _kk_pipeline_gpu(
                rx_mod, torch, w, c2, l2, ks[0].fc_step, torch.from_numpy(b_o[None]).cuda(), d_train, 1, ns_sym)
            e2b = rx_mod.FDE(w["fde_taps"], w["fde_ov"])
            e2b.train(f2[1], torch.from_numpy(ks[1].sym[:w["fde_train"]].astype(np.complex64)).cuda())
            e2.apply(f2[:1], y2[:1])
            e2b.apply(f2[1:], y2[1:])
            _, st2 = r2.process(y2.view(1, 2, 2 * ns_sym), llr2)
            line["parity"] = {"sample": line["cpu_baseline"]["sample"],
                              "bit_errors_gpu": int(st2[0]["bit_errors"]),
                              "bit_errors_oracle": int(res.stats["bit_errors"]),
                              "gmi_gpu": float(st2[0]["gmi"]), "gmi_oracle": float(res.stats["gmi"]),
                              "note": "GPU pipeline (KK, equaliser trained per signal, chain) against the oracle "
                                      "pipeline on the same codes; elementwise parity of each stage is in the tests"}
    print(json.dumps(line), flush=True)


def run_mlp_infer(args):
    """The learned demapper's inference alone (config 4's tensor-core
    contraction): 2^24 4D-64 symbols at 12 dB with seeded He-initialised
    weights, one rx_mlp_infer per step; the roofline counts the MLP's
    algorithmic flops, 2 (4*128 + 128*128 + 128*6) per symbol, against the
    measured bfloat16 tensor peak."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n = args.mlp_sym
    fmt = synth.tx_format("gs4d64")
    rng = np.random.default_rng(synth.stream_seed(17, 0))
    lab = rng.integers(0, 64, size=n)
    n0 = 10 ** (-12 / 10)
    z = fmt.points[lab] + np.sqrt(n0 / 2) * (rng.standard_normal((n, 2)) + 1j * rng.standard_normal((n, 2)))
    x = torch.from_numpy(np.stack([z[:, 0].real, z[:, 0].imag, z[:, 1].real, z[:, 1].imag], axis=1)
                         .astype(np.float32)).cuda()
    s2 = torch.full((n,), n0 / 2, dtype=torch.float32, device="cuda")
    m = rx_mod.Mlp(synth.mlp_init_params(LEARN["init_seed"]))
    llr = torch.empty((n, 6), dtype=torch.float32, device="cuda")
    # both inference paths: 2 = tcgen05 (the default), 1 = mma.sync
    path_ms = {}
    for path in (1, 2):
        m.set_param("infer", path)
        path_ms[path] = _event_ms(lambda: m.infer(x, s2, llr), args.steps, args.warmup)
    ms = path_ms[2]
    # one Adam step on a batch of 8192 (the training configuration's batch),
    # tcgen05 GEMMs against the float32 SIMT GEMMs
    nb = 8192
    bits = torch.from_numpy(rng.integers(0, 2, size=(nb, 6), dtype=np.uint8)).cuda()
    xb, s2b = x[:nb].contiguous(), s2[:nb].contiguous()
    train_ms = {}
    for tc in (0, 1):
        mt = rx_mod.Mlp(synth.mlp_init_params(LEARN["init_seed"]))
        mt.set_param("train_tc", tc)
        train_ms[tc] = _event_ms(lambda: mt.train_step(xb, s2b, bits, 1e-3), max(args.steps, 20), args.warmup)
        mt.close()
    pk, pk_kind = peaks()
    flops = 2.0 * (4 * 128 + 128 * 128 + 128 * 6) * n
    tf = flops / (ms * 1e-3) / 1e12
    peak = pk.get("bf16_tflops", 1900.0)
    line = {
        "metric": "learned demapper inference, 4D symbols per second", "value": n / (ms * 1e-3) / 1e9,
        "unit": "Gsym/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights / f32",
        "data": "synthetic",
        "config": {"workload": f"mlp_4x128x128x6_infer_{n}", "symbols": n, "esn0_db": 12.0,
                   "l2": f"inputs {n * 20 / 2**20:.0f} MiB, outputs {n * 24 / 2**20:.0f} MiB; no flush"},
        "roofline": {"bound": "tensor", "kernel": "infer_umma_kernel", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                     "frac": tf / peak, "traffic": None, "peak_kind": pk_kind,
                     "note": "algorithmic flops; the kernel issues 3 products per layer-2 term (bfloat16 split)"},
        "paths": {"tcgen05_gsym_s": n / (path_ms[2] * 1e-3) / 1e9, "mma_sync_gsym_s": n / (path_ms[1] * 1e-3) / 1e9},
        "train_step_ms_batch_8192": {"tcgen05": train_ms[1], "float32_simt": train_ms[0]},
        "gpu_launches": args.steps,
    }
    print(json.dumps(line), flush=True)


def run_precision(args):
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    wl = WL3
    S, n = wl["streams"], args.n_sym if args.n_sym != WL["n_sym"] else wl["n_sym"]
    rxs, bits = [], []
    for p_ in range(S):
        st = synth.make_stream(wl["fmt"], n, seed=synth.stream_seed(3, p_), esn0_db=wl["esn0_db"],
                               cd_ps_per_nm=wl["cd_ps_per_nm"], linewidth_ts=wl["linewidth_ts"])
        rxs.append(st.rx)
        bits.append(st.bits)
    samples = torch.from_numpy(np.stack(rxs)).cuda()
    bits_d = torch.from_numpy(np.stack(bits)).cuda()
    del rxs
    m = bits[0].shape[1]
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs", 6800.0)
    forms = {}
    F = max(1, min(2, args.frames_in_flight))
    for prec, name, store in ((0, "f32", 8), (1, "f16", 4), (2, "bf16", 4)):
        hs = []
        for i in range(F):
            hs.append(rx_mod.Receiver(wl["fmt"], cd_ps_per_nm=wl["cd_ps_per_nm"], taps=wl["taps"],
                                      bps_phases=wl["bps_phases"], streams=S, stream=torch.cuda.Stream(),
                                      **rx_params(wl), precision=prec))
            hs[-1].set_reference(bits_d)
        r = hs[0]
        llr = torch.empty((S, n, m), dtype=torch.float32, device="cuda")
        llr2 = torch.empty_like(llr) if F > 1 else None
        ms, stg, st_ = timed_steps(r, samples, llr, args.steps, args.warmup,
                                   hs[1] if F > 1 else None, llr2)
        ms_one = timed_steps(r, samples, llr, args.steps, 2)[0] if F > 1 else ms
        same = bool(torch.equal(llr, llr2)) if F > 1 else True
        bps = chain_bytes_per_symbol(wl, store)
        sym_s = S * n / (ms * 1e-3)
        forms[name] = {"gbps": sym_s * m / 1e9, "ms_per_step": ms, "stages_ms": stg,
                       "one_frame_at_a_time": {"gbps": S * n * m / (ms_one * 1e-3) / 1e9, "ms_per_step": ms_one},
                       "frames_identical": same,
                       "bytes_per_symbol": bps, "hbm_gbs": sym_s * bps / 1e9,
                       "hbm_frac": sym_s * bps / 1e9 / hbm,
                       "bit_errors": int(sum(x["bit_errors"] for x in st_)),
                       "n_bits": int(sum(x["n_bits"] for x in st_))}
        for h_ in hs:
            h_.close()
    be32 = forms["f32"]["bit_errors"]
    for name in ("f16", "bf16"):
        forms[name]["ber_delta_rel_vs_f32"] = (forms[name]["bit_errors"] - be32) / max(be32, 1)
    line = {
        "metric": METRIC, "value": forms["f16"]["gbps"], "unit": "Gbit/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": forms["f16"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f16 storage / f32",
        "data": "synthetic",
        "config": {"workload": wl["workload"], "streams": S, "symbols_per_stream": n, "format": wl["fmt"],
                   "fft": wl["fft"], "overlap": wl["overlap"], "taps": wl["taps"], "bps_phases": wl["bps_phases"],
                   "block": wl["block"], "lag": wl["lag"], "lms_start": wl.get("lms_start", 0),
                   "frames_in_flight": F},
        "forms": forms, "hbm_peak_gbs": hbm, "hbm_peak_kind": pk_kind,
    }
    if not args.no_cpu_baseline:
        v, dt, st_o, res_o = cpu_baseline(args.cpu_sym, wl, wl["esn0_db"], synth.stream_seed(3, 99))
        line["cpu_baseline"] = {"value": v, "unit": "Gbit/s", "cores": 1, "kind": "oracle",
                                "sample": f"one stream of {args.cpu_sym} 4D symbols, {dt:.1f} s"}
        if not args.no_parity:
            line["parity"] = {name: parity_on(rx_mod, torch, st_o, res_o, wl, prec)
                              for prec, name in ((0, "f32"), (1, "f16"), (2, "bf16"))}
            # the error against the oracle stage by stage: stored x, stored y,
            # de-rotated z, LLRs, and the bit errors against the oracle's
            per_stage = {}
            for prec, name in ((0, "f32"), (1, "f16"), (2, "bf16")):
                pe = stage_errors(rx_mod, torch, st_o, res_o, wl, prec)
                pq = line["parity"][name]
                pe.update({"z_evm": pq["evm_vs_oracle"], "max_rel_llr_err": pq["max_rel_llr_err"],
                           "ber_delta_vs_oracle": (pq["bit_errors_gpu"] - pq["bit_errors_oracle"]) /
                           max(1, pq["bit_errors_oracle"])})
                per_stage[name] = pe
            line["per_stage_error"] = per_stage
    print(json.dumps(line), flush=True)


# ---- serving (config 5): 64 streams, Poisson arrivals, mixed formats and lengths ----
SERVE = dict(n_req=64, len_log2=(14, 20), km=(80.0, 2000.0), budget=8 << 30, slots=64, load=0.8,
             esn0={"dp_qpsk": 12.0, "dp_16qam": 18.0, "gs4d64": 14.0},
             bps={"dp_qpsk": 32, "dp_16qam": 32, "gs4d64": 64}, m={"dp_qpsk": 4, "dp_16qam": 8, "gs4d64": 6}, issue=1,
             connections="32")


def serving_requests(seed: int):
    rng = np.random.default_rng(seed)
    fmts = ["dp_qpsk", "dp_16qam", "gs4d64"]
    reqs = []
    for i in range(SERVE["n_req"]):
        fmt = fmts[int(rng.integers(0, 3))]
        n = int(2 ** rng.uniform(*SERVE["len_log2"]))
        km = float(rng.uniform(*SERVE["km"]))
        st = synth.make_stream(fmt, n, seed=seed + 1 + i, esn0_db=SERVE["esn0"][fmt],
                               cd_ps_per_nm=17.0 * km, linewidth_ts=1e-5)
        reqs.append((fmt, n, km, st))
    return reqs


def run_serving(args):
    # 64 request streams share the CUDA context's hardware work queues: 32
    # (the most) instead of the default 8, set before the context is created
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", SERVE["connections"])
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    reqs = serving_requests(synth.stream_seed(5, 0))
    dev = [(torch.from_numpy(st.rx.astype(np.complex64)).cuda(), torch.from_numpy(st.bits).cuda())
           for _, _, _, st in reqs]
    total_bits = sum(n * SERVE["m"][fmt] for fmt, n, _, _ in reqs)

    # one long-lived server (its pool of idle handles carries over from the
    # warm-up to the measured runs, as in a running receiver)
    srv = rx_mod.Server(SERVE["budget"], SERVE["slots"])
    bps_default = int(srv.get_param("blocks_per_step"))     # the server's defaults for these queues
    threads_default = int(srv.get_param("issue_threads"))
    ids_last = {}

    host_ms = [0.0]       # host time inside rx_server_step (issue of the blocks)

    def serve(arrivals):
        host_ms[0] = 0.0
        llrs, ids, t_arr, t_done = {}, {}, {}, {}
        order = np.argsort(arrivals)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = 0
        while len(t_done) < len(reqs):
            now = time.perf_counter() - t0
            while k < len(order) and arrivals[order[k]] <= now:
                i = int(order[k])
                fmt, n, km, _ = reqs[i]
                llrs[i] = torch.empty((n, SERVE["m"][fmt]), dtype=torch.float32, device="cuda")
                ids[i] = srv.submit(fmt, dev[i][0], llrs[i], dev[i][1], cd_ps_per_nm=17.0 * km, taps=31,
                                    bps_phases=SERVE["bps"][fmt], fft=4096, overlap=1024, block=1 << 16)
                t_arr[i] = now
                k += 1
            th0 = time.perf_counter()
            srv.step()
            host_ms[0] += (time.perf_counter() - th0) * 1e3
            for i, rid in ids.items():
                if i not in t_done and srv.poll(rid)[0] in (rx_mod.REQ_DONE, rx_mod.REQ_FAILED):
                    t_done[i] = time.perf_counter() - t0
            if k < len(order) and not srv.info()["mem_used"]:
                time.sleep(max(0.0, min(0.001, arrivals[order[k]] - (time.perf_counter() - t0))))
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        states = [srv.poll(ids[i]) for i in range(len(reqs))]
        info = srv.info()
        lat = sorted(t_done[i] - t_arr[i] for i in range(len(reqs)))
        ids_last.clear()
        ids_last.update(ids)
        return wall, lat, states, info

    # capacity (every request present at once) in each issue mode of the
    # handles: 0 stages on their own streams with events, 1 one stream per
    # request, 2 one stream and the blocks after the first as CUDA graphs
    # (one block per step)
    srv.set_param("blocks_per_step", 1)
    cap_by_issue, host_by_issue = {}, {}
    for mode in (0, 1, 2):
        srv.set_param("issue", mode)
        for _ in range(max(1, args.warmup)):
            serve(np.zeros(len(reqs)))
        w_, _, _, _ = serve(np.zeros(len(reqs)))
        cap_by_issue[str(mode)] = total_bits / w_ / 1e9
        host_by_issue[str(mode)] = {"wall_ms": w_ * 1e3, "host_ms_in_step": host_ms[0]}
    # the same in mode 1 with 1 / 2 / 4 / 8 host issue threads (the
    # server's default blocks per step)
    cap_by_threads = {}
    srv.set_param("issue", 1)
    srv.set_param("blocks_per_step", bps_default)
    for nt in (1, 2, 4, 8):
        srv.set_param("issue_threads", nt)
        serve(np.zeros(len(reqs)))
        w_, _, _, _ = serve(np.zeros(len(reqs)))
        cap_by_threads[str(nt)] = total_bits / w_ / 1e9
    srv.set_param("issue_threads", threads_default)
    # and with 1 / 2 / 4 / all blocks of a request per step (one call each)
    cap_by_bps = {}
    for bps in (1, 2, 4, 1 << 20):
        srv.set_param("blocks_per_step", bps)
        serve(np.zeros(len(reqs)))
        w_, _, _, _ = serve(np.zeros(len(reqs)))
        cap_by_bps[str(bps)] = total_bits / w_ / 1e9
    srv.set_param("blocks_per_step", bps_default)
    srv.set_param("issue", SERVE["issue"])
    for _ in range(max(1, args.warmup)):
        serve(np.zeros(len(reqs)))
    wall0, lat0, states0, info0 = serve(np.zeros(len(reqs)))
    cap_bits = total_bits / wall0
    # Poisson arrivals at SERVE["load"] of that capacity
    rng = np.random.default_rng(7)
    rate = SERVE["load"] * cap_bits / (total_bits / len(reqs))      # requests per second
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    wall, lat, states, info = serve(arrivals)
    failed = []
    for i, (st_, _) in enumerate(states):
        if st_ != rx_mod.REQ_DONE:
            srv.poll(ids_last[i])                      # sets the server's last error to this request's
            failed.append(f"request {i} ({reqs[i][0]}, {reqs[i][1]} symbols): state {st_}: "
                          f"{rx_mod.lib().rx_server_last_error().decode()}")
    # the same arrivals again with every issue call timed on the device (an
    # event pair per call of blocks_per_step blocks): the block latency
    srv.set_param("block_latency", 1)
    serve(arrivals)
    blat = sorted(srv.block_latency())
    srv.set_param("block_latency", 0)
    # the same arrivals through the server's own loop (rx_server_start): this
    # thread only submits at the arrival times and polls
    srv.start()
    llrs_l, ids_l, t_arr_l, t_done_l = {}, {}, {}, {}
    order = np.argsort(arrivals)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 0
    while len(t_done_l) < len(reqs):
        now = time.perf_counter() - t0
        while k < len(order) and arrivals[order[k]] <= now:
            i = int(order[k])
            fmt, n, km, _ = reqs[i]
            llrs_l[i] = torch.empty((n, SERVE["m"][fmt]), dtype=torch.float32, device="cuda")
            ids_l[i] = srv.submit(fmt, dev[i][0], llrs_l[i], dev[i][1], cd_ps_per_nm=17.0 * km, taps=31,
                                  bps_phases=SERVE["bps"][fmt], fft=4096, overlap=1024, block=1 << 16)
            t_arr_l[i] = now
            k += 1
        for i, rid in ids_l.items():
            if i not in t_done_l and srv.poll(rid)[0] in (rx_mod.REQ_DONE, rx_mod.REQ_FAILED):
                t_done_l[i] = time.perf_counter() - t0
        time.sleep(0.0002)
    torch.cuda.synchronize()
    wall_l = time.perf_counter() - t0
    srv.stop()
    lat_l = sorted(t_done_l[i] - t_arr_l[i] for i in range(len(reqs)))
    loop_ok = all(srv.poll(ids_l[i])[0] == rx_mod.REQ_DONE for i in range(len(reqs)))
    handles = {k: int(srv.get_param(k)) for k in ("handles_created", "handles_destroyed", "handle_regrows")}
    srv.close()
    ok = all(s == rx_mod.REQ_DONE for s, _ in states)
    line = {
        "metric": METRIC, "value": total_bits / wall / 1e9, "unit": "Gbit/s", "n_gpus": 1,
        "steps": 1, "warmup": args.warmup, "ms_per_step": wall * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving_64_streams_poisson_mixed_formats", "requests": len(reqs),
                   "symbols": int(sum(n for _, n, _, _ in reqs)), "budget_bytes": SERVE["budget"],
                   "slots": SERVE["slots"], "load": SERVE["load"], "block": 1 << 16, "fft": 4096, "taps": 31,
                   "cuda_device_max_connections": os.environ["CUDA_DEVICE_MAX_CONNECTIONS"]},
        "capacity_gbps_all_at_once": cap_bits / 1e9,
        "capacity_gbps_by_issue_mode": cap_by_issue, "issue_mode": SERVE["issue"],
        "host_by_issue_mode": host_by_issue, "capacity_gbps_by_issue_threads_mode1": cap_by_threads,
        "capacity_gbps_by_blocks_per_step_mode1": cap_by_bps, "blocks_per_step": bps_default,
        "issue_threads": threads_default,
        "handles": handles,
        "request_latency_ms": {"p50": 1e3 * lat[len(lat) // 2], "p99": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))]},
        "request_latency_ms_all_at_once": {"p50": 1e3 * lat0[len(lat0) // 2], "p99": 1e3 * lat0[-1]},
        "block_latency_ms": {"p50": blat[len(blat) // 2], "p99": blat[min(len(blat) - 1, int(0.99 * len(blat)))],
                             "calls": len(blat), "blocks_per_call": bps_default},
        "server_loop": {"gbps": total_bits / wall_l / 1e9, "all_done": loop_ok,
                        "request_latency_ms": {"p50": 1e3 * lat_l[len(lat_l) // 2],
                                               "p99": 1e3 * lat_l[min(len(lat_l) - 1, int(0.99 * len(lat_l)))]}},
        "max_running": info["max_active"], "all_done": ok, "not_done": failed[:8],
        "ber_by_format": {f: float(np.mean([st["ber"] for (s_, st), (fm, _, _, _) in zip(states, reqs) if fm == f and st]))
                          for f in ("dp_qpsk", "dp_16qam", "gs4d64")},
    }
    print(json.dumps(line), flush=True)


# ---- learned demapper (MLP 4 -> 128 -> 128 -> 6) on the same chain ------------
# Adam at lr 1e-3; the last `decay_epochs` epochs run at lr_final (a step
# schedule that lets the network settle; 0 keeps the rate constant)
LEARN = dict(train_streams=16, train_sym=(1 << 18) + (1 << 14), skip=1 << 14, epochs=80, batch=8192,
             lr=1e-3, lr_final=1e-4, decay_epochs=20, infer_streams=16, infer_sym=1 << 20, esn0=(8.0, 16.0),
             init_seed=2108070044)


def learned_inputs(n_streams: int, n_sym: int, seed_base: int):
    """Streams of the bench channel with Es/N0 drawn uniformly in 8..16 dB."""
    rng = np.random.default_rng(seed_base)
    esn0 = rng.uniform(*LEARN["esn0"], size=n_streams)
    rxs, bits = [], []
    for p in range(n_streams):
        st = synth.make_stream(WL["fmt"], n_sym, seed=seed_base + 1 + p, esn0_db=float(esn0[p]),
                               cd_ps_per_nm=WL["cd_ps_per_nm"], linewidth_ts=WL["linewidth_ts"])
        rxs.append(st.rx)
        bits.append(st.bits)
    return np.stack(rxs), np.stack(bits), esn0


def run_learned(args):
    """Config 4: train the MLP demapper on symbols the chain itself makes, on
    the GPU's own kernels, then run the chain with it on 2^24 symbols and
    compare with the exact demapper on the same streams."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    # training data: de-rotated symbols and block sigma^2 from the exact chain
    S, N, skip = LEARN["train_streams"], LEARN["train_sym"], LEARN["skip"]
    rx_h, bits_h, _ = learned_inputs(S, N, synth.stream_seed(4, 0))
    r = rx_mod.Receiver(WL["fmt"], cd_ps_per_nm=WL["cd_ps_per_nm"], taps=WL["taps"],
                        bps_phases=WL["bps_phases"], streams=S, **rx_params())
    r.set_reference(torch.from_numpy(bits_h).cuda())
    x4 = torch.empty((S, N, 4), dtype=torch.float32, device="cuda")
    s2 = torch.empty((S, N), dtype=torch.float32, device="cuda")
    r.set_symbol_output(x4, s2)
    r.process(torch.from_numpy(rx_h).cuda(), stats=False)
    torch.cuda.synchronize()
    X = x4[:, skip:].reshape(-1, 4).contiguous()
    S2 = s2[:, skip:].reshape(-1).contiguous()
    B = torch.from_numpy(bits_h[:, skip:].reshape(-1, 6)).cuda()
    r.set_symbol_output(None, None)
    r.close()
    del rx_h
    n_train = X.shape[0]
    m = rx_mod.Mlp(synth.mlp_init_params(LEARN["init_seed"]))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(LEARN["init_seed"])
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    bs = LEARN["batch"]
    steps_per_epoch = n_train // bs
    t0 = time.perf_counter()
    losses = []
    epochs = args.learn_epochs if args.learn_epochs else LEARN["epochs"]
    decay = LEARN["decay_epochs"] if args.learn_decay is None else args.learn_decay
    for ep in range(epochs):
        lr = LEARN["lr_final"] if ep >= epochs - decay else LEARN["lr"]
        perm = torch.randperm(n_train, device="cuda", generator=gen)
        for i in range(steps_per_epoch):
            idx = perm[i * bs:(i + 1) * bs]
            m.train_step(X[idx], S2[idx], B[idx], lr, loss)
        losses.append(loss.item())
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del X, S2, B
    # inference: the chain with the exact and with the learned demapper
    S, N = LEARN["infer_streams"], args.learned_sym
    rx_h, bits_h, esn0 = learned_inputs(S, N, synth.stream_seed(4, 1))
    samples = torch.from_numpy(rx_h).cuda()
    del rx_h
    r = rx_mod.Receiver(WL["fmt"], cd_ps_per_nm=WL["cd_ps_per_nm"], taps=WL["taps"],
                        bps_phases=WL["bps_phases"], streams=S, **rx_params())
    r.set_reference(torch.from_numpy(bits_h).cuda())
    llr = torch.empty((S, N, 6), dtype=torch.float32, device="cuda")
    out = {}
    for name, dm in (("exact", None), ("learned", m)):
        r.set_demapper(dm)
        for _ in range(args.warmup):
            r.process(samples, llr, stats=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            r.process(samples, llr, stats=False)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        st = r.stats()
        out[name] = {"ms_per_step": ms, "gbps": S * N * 6 / (ms * 1e-3) / 1e9,
                     "gmi": [x["gmi"] for x in st], "ber": [x["ber"] for x in st]}
    ge, gl = np.array(out["exact"]["gmi"]), np.array(out["learned"]["gmi"])
    be, bl = np.array(out["exact"]["ber"]), np.array(out["learned"]["ber"])
    line = {
        "metric": METRIC, "value": out["learned"]["gbps"], "unit": "Gbit/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": out["learned"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32",
        "data": "synthetic",
        "config": {"workload": "learned_demapper_mlp_4x128x128x6_gs4d64", "streams": S,
                   "symbols_per_stream": N, "esn0_db": [round(float(v), 2) for v in esn0],
                   "train_symbols": int(n_train), "epochs": epochs, "batch": bs, "lr": LEARN["lr"],
                   "lr_final": LEARN["lr_final"], "decay_epochs": decay},
        "exact_chain_gbps": out["exact"]["gbps"],
        "gmi_gap_mean": float(np.mean(ge - gl)), "gmi_gap_max": float(np.max(ge - gl)),
        "ber_delta_rel_max": float(np.max(np.abs(bl - be) / np.maximum(be, 1e-12))),
        "gmi_exact": [round(float(v), 5) for v in ge], "gmi_learned": [round(float(v), 5) for v in gl],
        "ber_exact": [float(f"{v:.4g}") for v in be], "ber_learned": [float(f"{v:.4g}") for v in bl],
        "train_seconds": train_s, "train_loss_per_epoch": [round(float(v), 6) for v in losses],
    }
    print(json.dumps(line), flush=True)


def run_bps_paths(args):
    """The phase search alone at the bench's launch shape (9 streams x one
    2^16-symbol block, 64 test phases, window 64), SIMT kernel against the
    tensor-core one (bps_tc = 1): candidates per second, fraction of the
    measured FFMA issue peak, and the share of indices on which they differ."""
    import torch
    from paper_2108_07004_gb300 import rx as rx_mod
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    S, blk = 9, 1 << 16
    rng = np.random.default_rng(2108)
    pts = np.array(rx_mod.load_table("gs4d64")["points"], np.float64)
    lab = rng.integers(0, 64, size=(S, 2 * blk))
    sym = pts[lab]
    y = np.stack([sym[..., 0] + 1j * sym[..., 1], sym[..., 2] + 1j * sym[..., 3]], axis=1)
    ph = np.cumsum(rng.standard_normal((S, 2 * blk)) * 0.01, axis=1)[:, None, :]
    y = y * np.exp(1j * ph) + 0.12 * (rng.standard_normal(y.shape) + 1j * rng.standard_normal(y.shape))
    yd = torch.from_numpy(y.astype(np.complex64)).cuda()
    a, e = blk - 32, 2 * blk - 32
    cand = S * (e - a) * 64 * 64
    ipk = issue_peaks(rx_mod, 0)
    peak = ipk["ffma"]["lane_instr_per_s"]
    out, idx = {}, {}
    for tc, name in ((0, "simt"), (1, "tensor_cores")):
        r = rx_mod.Receiver("gs4d64", cd_ps_per_nm=0.0, taps=31, bps_phases=64, streams=S)
        r.set("bps_tc", tc)
        bo = torch.zeros((S, e - a), dtype=torch.uint8, device="cuda")
        for _ in range(max(3, args.warmup)):
            r.bps(yd, a, e, 2 * blk, bo)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            r.bps(yd, a, e, 2 * blk, bo)
        e1.record()
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / args.steps * 1e3
        idx[name] = bo.cpu().numpy()
        out[name] = {"us_per_launch": us, "Tcand_per_s": cand / (us * 1e-6) / 1e12,
                     "frac_of_ffma_peak": cand / (us * 1e-6) / peak}
        r.close()
    line = {"metric": "phase-search candidates per second (one (test phase, point) distance)",
            "value": out["simt"]["Tcand_per_s"], "unit": "Tcand/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic 4D-64 symbols with phase drift and noise",
            "config": {"workload": "bps_9x2p16_gs4d64_B64_W64", "streams": S, "block": blk},
            "paths": out, "differ_frac": float(np.mean(idx["simt"] != idx["tensor_cores"])),
            "peak_ffma_lane_instr_per_s": peak, "clocks": ipk["clocks"]}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-sym", type=int, default=WL["n_sym"])
    ap.add_argument("--streams", type=int, default=len(WL["esn0_db"]))
    ap.add_argument("--cpu-sym", type=int, default=1 << 17)
    ap.add_argument("--ref-sym", type=int, default=1 << 14)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--frames-in-flight", type=int, default=2,
                    help="handles whose consecutive frames overlap (1: one frame at a time)")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", default="plain", choices=["plain", "learned", "precision", "serving", "block_lms", "widely_linear", "kk", "kk_chain", "mlp_infer", "bps_paths", "gs128"],
                    help="learned: train the MLP demapper on chain output, compare with the exact one; "
                         "precision: DP-QPSK chain with CDC/FIR data in float32, half and bfloat16; "
                         "serving: 64 mixed streams with Poisson arrivals through the continuous-batching server")
    ap.add_argument("--learned-sym", type=int, default=LEARN["infer_sym"])
    ap.add_argument("--learn-epochs", type=int, default=0, help="training epochs (0: the default)")
    ap.add_argument("--learn-decay", type=int, default=None, help="final epochs at the lower rate")
    ap.add_argument("--mlp-sym", type=int, default=1 << 24)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.variant == "learned":
        run_learned(args)
    elif args.variant == "widely_linear":
        run_widely_linear(args)
    elif args.variant == "block_lms":
        run_block_lms(args)
    elif args.variant == "kk":
        run_kk(args)
    elif args.variant == "kk_chain":
        run_kk_chain(args)
    elif args.variant == "mlp_infer":
        run_mlp_infer(args)
    elif args.variant == "precision":
        run_precision(args)
    elif args.variant == "bps_paths":
        run_bps_paths(args)
    elif args.variant == "serving":
        run_serving(args)
    elif args.variant == "gs128":
        run_gs128(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
