"""Python binding of the receiver's C ABI (include/rx.h).

Argument marshalling only: torch tensors supply device memory and the CUDA
stream; every step of the chain runs in the library's kernels.  Loading
fails loudly when the compiled library is missing; there is no other path.
"""
from __future__ import annotations

import ctypes as C
import json
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librx.so")
_lib = None

RX_FMT_CUSTOM, RX_FMT_DP_QPSK, RX_FMT_DP_16QAM, RX_FMT_DP_64QAM, RX_FMT_GS4D64 = 0, 1, 2, 3, 4


class RxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rx error {code}: {msg}")
        self.code = code


class RxFormat(C.Structure):
    _fields_ = [("kind", C.c_int), ("dims", C.c_int), ("m_bits", C.c_int),
                ("sym_order", C.c_int), ("points", C.POINTER(C.c_float)),
                ("labels", C.POINTER(C.c_uint32))]


class RxRequest(C.Structure):
    _fields_ = [("format", RxFormat), ("symbol_rate", C.c_double), ("sps", C.c_int),
                ("cd_ps_per_nm", C.c_double), ("taps", C.c_int), ("bps_phases", C.c_int),
                ("fft", C.c_int), ("overlap", C.c_int), ("block", C.c_int), ("n_pre", C.c_int),
                ("samples", C.c_void_p), ("n_samples", C.c_size_t), ("llr_out", C.c_void_p),
                ("ref_bits", C.c_void_p)]


class RxStats(C.Structure):
    _fields_ = [("n_sym", C.c_uint64), ("n_bits", C.c_uint64), ("bit_errors", C.c_uint64),
                ("gmi_sum", C.c_double), ("gmi", C.c_double), ("ber", C.c_double),
                ("evm_num", C.c_double), ("evm_den", C.c_double), ("sigma2_last", C.c_double),
                ("n_out", C.c_uint64), ("blocks", C.c_uint32), ("reserved", C.c_uint32),
                ("first_valid", C.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_VP, _SZ, _I, _D = C.c_void_p, C.c_size_t, C.c_int, C.c_double
_PROTOS = {
    "rx_create": (C.c_void_p, [C.POINTER(RxFormat), _D, _I, _D, _I, _I]),
    "rx_destroy": (None, [_VP]),
    "rx_set_param": (_I, [_VP, C.c_char_p, _D]),
    "rx_get_param": (_I, [_VP, C.c_char_p, C.POINTER(_D)]),
    "rx_set_stream": (_I, [_VP, _VP]),
    "rx_set_reference": (_I, [_VP, _VP, _SZ]),
    "rx_set_reference_host": (_I, [_VP, _VP, _SZ]),
    "rx_reset": (_I, [_VP]),
    "rx_process": (_I, [_VP, _VP, _SZ, _VP, _VP]),
    "rx_process_host": (_I, [_VP, _VP, _SZ, _VP, _VP]),
    "rx_get_stats": (_I, [_VP, _VP]),
    "rx_stream_delay": (_I, [_VP, C.POINTER(_SZ)]),
    "rx_push": (_I, [_VP, _VP, _SZ, _VP, _VP]),
    "rx_flush": (_I, [_VP, _VP, C.POINTER(_SZ), _VP]),
    "rx_wait": (_I, [_VP, _D]),
    "rx_issue_rate": (_I, [_I, _I, C.POINTER(_D), C.POINTER(_D)]),
    "rx_get_profile": (_I, [_VP, C.c_char_p, C.POINTER(_D), C.POINTER(C.c_uint64)]),
    "rx_get_block_latency": (_I, [_VP, C.POINTER(_D), _SZ, C.POINTER(_SZ)]),
    "rx_get_state": (_I, [_VP, _VP, C.POINTER(_SZ)]),
    "rx_set_state": (_I, [_VP, _VP, _SZ]),
    "rx_process_blocks": (_I, [_VP, _VP, _SZ, _SZ, _SZ, _VP, _VP]),
    "rx_server_create": (_VP, [_SZ, _I]),
    "rx_server_destroy": (None, [_VP]),
    "rx_server_submit": (_I, [_VP, _VP, C.POINTER(C.c_uint64)]),
    "rx_server_step": (_I, [_VP, C.POINTER(_I)]),
    "rx_server_run": (_I, [_VP]),
    "rx_server_start": (_I, [_VP]),
    "rx_server_stop": (_I, [_VP]),
    "rx_server_poll": (_I, [_VP, C.c_uint64, C.POINTER(_I), _VP]),
    "rx_server_info": (_I, [_VP, C.POINTER(_SZ), C.POINTER(_I), C.POINTER(C.c_long)]),
    "rx_server_set_param": (_I, [_VP, C.c_char_p, _D]),
    "rx_server_get_param": (_I, [_VP, C.c_char_p, C.POINTER(_D)]),
    "rx_server_get_block_latency": (_I, [_VP, C.POINTER(_D), _SZ, C.POINTER(_SZ)]),
    "rx_server_last_error": (C.c_char_p, []),
    "rx_set_demapper": (_I, [_VP, _VP]),
    "rx_set_symbol_output": (_I, [_VP, _VP, _VP]),
    "rx_kk_create": (_VP, [_VP]),
    "rx_kk_destroy": (None, [_VP]),
    "rx_kk_set_stream": (_I, [_VP, _VP]),
    "rx_kk_field": (_I, [_VP, _VP, _SZ, _SZ, _VP, _VP]),
    "rx_fde_create": (_VP, [_I, _I]),
    "rx_fde_destroy": (None, [_VP]),
    "rx_fde_set_stream": (_I, [_VP, _VP]),
    "rx_fde_train": (_I, [_VP, _VP, _SZ, _VP, _SZ, _I, _D]),
    "rx_fde_set_taps": (_I, [_VP, _VP]),
    "rx_fde_get_taps": (_I, [_VP, _VP]),
    "rx_fde_apply": (_I, [_VP, _VP, _SZ, _SZ, _VP]),
    "rx_mlp_create": (_VP, [_VP]),
    "rx_mlp_destroy": (None, [_VP]),
    "rx_mlp_set_stream": (_I, [_VP, _VP]),
    "rx_mlp_get_params": (_I, [_VP, _VP]),
    "rx_mlp_set_params": (_I, [_VP, _VP]),
    "rx_mlp_grad": (_I, [_VP, _VP, _VP, _VP, _SZ, _VP, _VP]),
    "rx_mlp_train_step": (_I, [_VP, _VP, _VP, _VP, _SZ, C.c_float, _VP]),
    "rx_mlp_infer": (_I, [_VP, _VP, _VP, _SZ, _VP]),
    "rx_mlp_set_param": (_I, [_VP, C.c_char_p, _D]),
    "rx_mlp_get_param": (_I, [_VP, C.c_char_p, C.POINTER(_D)]),
    "rx_format_info": (_I, [_VP, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "rx_last_error": (C.c_char_p, []),
    "rx_cdc": (_I, [_VP, _VP, _VP, _SZ]),
    "rx_fir": (_I, [_VP, _VP, _SZ, _VP, _SZ, _SZ, _VP]),
    "rx_lms": (_I, [_VP, _VP, _SZ, _VP, _SZ, _SZ, _VP, _I, _I, C.c_uint64]),
    "rx_train": (_I, [_VP, _VP, _SZ, _VP, _VP]),
    "rx_bps": (_I, [_VP, _VP, _SZ, _SZ, _SZ, _SZ, _VP]),
    "rx_unwrap": (_I, [_VP, _VP, _SZ, _VP, _SZ, _SZ, _VP, _VP, _VP, _VP, _VP]),
    "rx_unwrap_static": (_I, [_VP, _VP, _SZ, _VP, _SZ, _SZ, _VP, _VP, _VP, _VP, _VP]),
    "rx_demap": (_I, [_VP, _VP, _SZ, _VP, _VP]),
}


def lib() -> C.CDLL:
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2108_07004_gb300.build`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols() -> list[str]:
    return list(_PROTOS)


def _ck(rc: int):
    if rc != 0:
        raise RxError(rc, lib().rx_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    return int(t)


# Receiver state buffer (rx_get_state / rx_set_state): header, then
# taps [L][S][2][2][T] c64, carry [S][2] int32, y_tail [S][2][W] c64,
# counters [S] (uint64 bit_errors, n_sym; float64 gmi_sum, evm_num,
# evm_den, sigma2).
STATE_MAGIC, STATE_VERSION = 0x31535852, 1
STATE_HEADER = np.dtype([("magic", "<u4"), ("version", "<u4"), ("streams", "<i4"), ("taps", "<i4"),
                         ("lag", "<i4"), ("bps_window", "<i4"), ("bps_phases", "<i4"),
                         ("m_bits", "<i4"), ("block", "<i8"), ("n_sym", "<i8"),
                         ("blocks_done", "<i8"), ("lms_updates", "<i8")])
STATE_COUNTERS = np.dtype([("bit_errors", "<u8"), ("n_sym", "<u8"), ("gmi_sum", "<f8"),
                           ("evm_num", "<f8"), ("evm_den", "<f8"), ("sigma2", "<f8")])


def pack_state(header: dict, ring: np.ndarray, carry: np.ndarray, y_tail: np.ndarray,
               counters: np.ndarray | None = None) -> bytes:
    """Lay out a receiver state from its header fields and parts (ring: the
    taps [L][S][2][2][T]; shapes as documented)."""
    hd = np.zeros(1, STATE_HEADER)
    hd["magic"], hd["version"] = STATE_MAGIC, STATE_VERSION
    for k, v in header.items():
        hd[k] = v
    S = int(hd["streams"][0])
    if counters is None:
        counters = np.zeros(S, STATE_COUNTERS)
    parts = [hd.tobytes(), np.ascontiguousarray(ring, dtype=np.complex64).tobytes(),
             np.ascontiguousarray(carry, dtype=np.int32).tobytes(),
             np.ascontiguousarray(y_tail, dtype=np.complex64).tobytes(),
             np.ascontiguousarray(counters, dtype=STATE_COUNTERS).tobytes()]
    return b"".join(parts)


def unpack_state(blob: bytes) -> dict:
    """Split a receiver state into its header fields and the arrays "ring"
    (taps), "carry", "y_tail" and "counters"."""
    hd = np.frombuffer(blob, STATE_HEADER, count=1)[0]
    S, T, L, W = int(hd["streams"]), int(hd["taps"]), int(hd["lag"]), int(hd["bps_window"])
    o = STATE_HEADER.itemsize
    out = {k: hd[k].item() for k in STATE_HEADER.names}
    n = L * S * 4 * T
    out["ring"] = np.frombuffer(blob, np.complex64, n, o).reshape(L, S, 2, 2, T)
    o += 8 * n
    out["carry"] = np.frombuffer(blob, np.int32, 2 * S, o).reshape(S, 2)
    o += 8 * S
    out["y_tail"] = np.frombuffer(blob, np.complex64, 2 * S * W, o).reshape(S, 2, W)
    o += 16 * S * W
    out["counters"] = np.frombuffer(blob, STATE_COUNTERS, S, o)
    o += STATE_COUNTERS.itemsize * S
    if o != len(blob):
        raise ValueError(f"state of {len(blob)} bytes, layout gives {o}")
    return out


def load_table(name: str) -> dict:
    with open(os.path.join(_HERE, "data", f"{name}_v1.json")) as f:
        return json.load(f)


def make_format(fmt: str):
    """rx_format for a built-in name or a table file ("table:<name>" forces
    the table file of a built-in); returns (format, arrays that must stay
    alive while it is used)."""
    f = RxFormat()
    keep = []
    if fmt == "dp_qpsk":
        f.kind = RX_FMT_DP_QPSK
    elif fmt == "dp_16qam":
        f.kind = RX_FMT_DP_16QAM
    elif fmt == "dp_64qam":
        f.kind = RX_FMT_DP_64QAM
    elif fmt == "gs4d64":
        f.kind = RX_FMT_GS4D64
    else:
        d = load_table(fmt[len("table:"):] if fmt.startswith("table:") else fmt)
        pts = np.ascontiguousarray(np.asarray(d["points"], dtype=np.float32))
        labs = np.ascontiguousarray(np.asarray(d["labels"], dtype=np.uint32))
        keep += [pts, labs]
        f.kind, f.dims, f.m_bits, f.sym_order = RX_FMT_CUSTOM, int(d["dims"]), int(d["m_bits"]), int(d["sym_order"])
        f.points = pts.ctypes.data_as(C.POINTER(C.c_float))
        f.labels = labs.ctypes.data_as(C.POINTER(C.c_uint32))
    return f, keep


class Receiver:
    """One receiver handle for `streams` streams of one format and link."""

    def __init__(self, fmt: str, *, symbol_rate: float = 28e9, sps: int = 2,
                 cd_ps_per_nm: float = 0.0, taps: int = 15, bps_phases: int = 32,
                 stream: torch.cuda.Stream | None = None, **params):
        L = lib()
        f, self._keep = make_format(fmt)
        h = L.rx_create(C.byref(f), symbol_rate, sps, cd_ps_per_nm, taps, bps_phases)
        if not h:
            raise RxError(-1, L.rx_last_error().decode())
        self.h = h
        self.fmt = fmt
        self.taps = taps
        dims, m, M = C.c_int(), C.c_int(), C.c_int()
        _ck(L.rx_format_info(h, C.byref(dims), C.byref(m), C.byref(M)))
        self.dims, self.m, self.M = dims.value, m.value, M.value
        st = stream if stream is not None else torch.cuda.current_stream()
        _ck(L.rx_set_stream(h, st.cuda_stream))
        self.stream = st
        for k, v in params.items():
            self.set(k, v)

    # ---- parameters ----
    def set(self, key: str, value: float):
        _ck(lib().rx_set_param(self.h, key.encode(), float(value)))

    def get(self, key: str) -> float:
        v = C.c_double()
        _ck(lib().rx_get_param(self.h, key.encode(), C.byref(v)))
        return v.value

    @property
    def streams(self) -> int:
        return int(self.get("streams"))

    def set_stream(self, stream: torch.cuda.Stream):
        _ck(lib().rx_set_stream(self.h, stream.cuda_stream))
        self.stream = stream

    def set_reference(self, bits: torch.Tensor):
        """bits: [S, N, m] uint8 on the device."""
        _ck(lib().rx_set_reference(self.h, _ptr(bits), bits.shape[1]))

    def set_reference_host(self, bits: torch.Tensor):
        """bits: [S, N, m] uint8 in host memory (pinned for asynchronous
        copies), taken in by the next process_host; the tensor must stay
        alive and unchanged until then."""
        if bits.is_cuda or not bits.is_contiguous() or bits.dtype != torch.uint8:
            raise ValueError("bits must be a contiguous uint8 host tensor")
        self._ref_host = bits
        _ck(lib().rx_set_reference_host(self.h, _ptr(bits), bits.shape[1]))

    def reset(self):
        _ck(lib().rx_reset(self.h))

    # ---- chain ----
    def process(self, samples: torch.Tensor, llr: torch.Tensor | None = None,
                stats: bool = True):
        """samples [S, 2, 2N] complex64 (device) -> (llr [S, N, m] float32, stats)."""
        S, _, ns = samples.shape
        if llr is None:
            llr = torch.empty((S, ns // 2, self.m), dtype=torch.float32, device=samples.device)
        st = (RxStats * S)() if stats else None
        _ck(lib().rx_process(self.h, _ptr(samples), ns, _ptr(llr),
                             C.cast(st, C.c_void_p) if st is not None else None))
        return llr, ([s.as_dict() for s in st] if st is not None else None)

    def process_blocks(self, samples: torch.Tensor, b0: int, b1: int,
                       llr: torch.Tensor | None = None, stats: bool = True):
        """Blocks b0 .. b1-1 of the streams in samples [S, 2, 2N] (device);
        b0 > 0 continues from the handle's state.  Rows outside the blocks'
        ranges of llr are left as they are."""
        S, _, ns = samples.shape
        if llr is None:
            llr = torch.zeros((S, ns // 2, self.m), dtype=torch.float32, device=samples.device)
        st = (RxStats * S)() if stats else None
        _ck(lib().rx_process_blocks(self.h, _ptr(samples), ns, b0, b1, _ptr(llr),
                                    C.cast(st, C.c_void_p) if st is not None else None))
        return llr, ([s.as_dict() for s in st] if st is not None else None)

    # ---- streaming ----
    def stream_delay(self) -> int:
        """Fixed delay d (symbols) of push(): output row r holds symbol r - d."""
        d = C.c_size_t()
        _ck(lib().rx_stream_delay(self.h, C.byref(d)))
        return d.value

    def push(self, samples: torch.Tensor, llr: torch.Tensor | None = None, stats: bool = True):
        """Next samples [S, 2, n] complex64 of a continuous stream -> n/2 LLR
        rows [S, n/2, m] (row r of the stream holds symbol r - d)."""
        S, _, n = samples.shape
        if llr is None:
            llr = torch.empty((S, n // 2, self.m), dtype=torch.float32, device="cuda")
        st = (RxStats * S)() if stats else None
        _ck(lib().rx_push(self.h, _ptr(samples), n, _ptr(llr),
                          C.cast(st, C.c_void_p) if st is not None else None))
        return llr, ([s.as_dict() for s in st] if st is not None else None)

    def flush(self, llr: torch.Tensor | None = None, stats: bool = True):
        """End the stream: the rows of the last min(N, d) symbols [S, rows, m]."""
        S = self.streams
        if llr is None:
            llr = torch.empty((S, max(1, self.stream_delay()), self.m), dtype=torch.float32, device="cuda")
        n = C.c_size_t()
        st = (RxStats * S)() if stats else None
        _ck(lib().rx_flush(self.h, _ptr(llr), C.byref(n),
                           C.cast(st, C.c_void_p) if st is not None else None))
        r = n.value                       # rows are packed: [S][r][m]
        llr = llr.reshape(-1)[: S * r * self.m].view(S, r, self.m)
        return llr, ([s.as_dict() for s in st] if st is not None else None)

    def wait(self, timeout_ms: float) -> bool:
        """True when the handle's queued work is done within timeout_ms."""
        rc = lib().rx_wait(self.h, float(timeout_ms))
        if rc == -4:
            return False
        _ck(rc)
        return True

    def set_demapper(self, mlp: "Mlp | None"):
        """Use the learned demapper (None: the exact one)."""
        _ck(lib().rx_set_demapper(self.h, mlp.h if mlp is not None else None))
        self._mlp = mlp

    def set_symbol_output(self, x4: torch.Tensor | None, sigma2: torch.Tensor | None):
        """x4 [S, N, 4] float32, sigma2 [S, N] float32 (device), or None."""
        _ck(lib().rx_set_symbol_output(self.h, _ptr(x4), _ptr(sigma2)))
        self._symout = (x4, sigma2)

    def process_host(self, samples, llr, stats: bool = True):
        """Host buffers (torch CPU tensors, pinned for overlap) in and out."""
        S, _, ns = samples.shape
        st = (RxStats * S)() if stats else None
        _ck(lib().rx_process_host(self.h, _ptr(samples), ns, _ptr(llr),
                                  C.cast(st, C.c_void_p) if st is not None else None))
        return [s.as_dict() for s in st] if st is not None else None

    def stats(self):
        S = self.streams
        st = (RxStats * S)()
        _ck(lib().rx_get_stats(self.h, C.cast(st, C.c_void_p)))
        return [s.as_dict() for s in st]

    def profile(self, stage: str = "all") -> tuple[float, int]:
        """(device ms, launches) of the last process() for one stage."""
        ms, n = C.c_double(), C.c_uint64()
        _ck(lib().rx_get_profile(self.h, stage.encode(), C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launches(self) -> int:
        n = C.c_uint64()
        _ck(lib().rx_get_profile(self.h, b"all", None, C.byref(n)))
        return n.value

    def block_latency(self) -> list[float]:
        n = C.c_size_t()
        _ck(lib().rx_get_block_latency(self.h, None, 0, C.byref(n)))
        buf = (C.c_double * max(1, n.value))()
        _ck(lib().rx_get_block_latency(self.h, buf, n.value, C.byref(n)))
        return list(buf[: n.value])

    def get_state(self) -> bytes:
        n = C.c_size_t(0)
        _ck(lib().rx_get_state(self.h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _ck(lib().rx_get_state(self.h, buf, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, blob: bytes):
        _ck(lib().rx_set_state(self.h, blob, len(blob)))

    # ---- single stages ----
    def cdc(self, x_in: torch.Tensor, x_out: torch.Tensor):
        _ck(lib().rx_cdc(self.h, _ptr(x_in), _ptr(x_out), x_in.shape[-1]))

    def fir(self, x: torch.Tensor, taps: torch.Tensor, k0: int, k1: int, y: torch.Tensor):
        _ck(lib().rx_fir(self.h, _ptr(x), x.shape[-1], _ptr(taps), k0, k1, _ptr(y)))

    def lms(self, x: torch.Tensor, taps: torch.Tensor, k0: int, n_upd: int,
            pcode: torch.Tensor | None, mode: int, passes: int = 1, u0: int = 0):
        _ck(lib().rx_lms(self.h, _ptr(x), x.shape[-1], _ptr(taps), k0, n_upd,
                         _ptr(pcode), mode, passes, u0))

    def train(self, x: torch.Tensor, taps: torch.Tensor, pcode: torch.Tensor):
        _ck(lib().rx_train(self.h, _ptr(x), x.shape[-1], _ptr(taps), _ptr(pcode)))

    def bps(self, y: torch.Tensor, a: int, e: int, n_valid: int, b_out: torch.Tensor):
        _ck(lib().rx_bps(self.h, _ptr(y), y.shape[-1], a, e, n_valid, _ptr(b_out)))

    def unwrap(self, y, b, a, e, carry_in, z, pcode, carry_out, sigma2):
        _ck(lib().rx_unwrap(self.h, _ptr(y), y.shape[-1], _ptr(b), a, e, _ptr(carry_in),
                            _ptr(z), _ptr(pcode), _ptr(carry_out), _ptr(sigma2)))

    def unwrap_static(self, y, b, a, e, carry_in, z, pcode, carry_out, sigma2):
        """unwrap() without device allocation (static 64 KiB scratch; for
        callers that may not allocate while they process)."""
        _ck(lib().rx_unwrap_static(self.h, _ptr(y), y.shape[-1], _ptr(b), a, e, _ptr(carry_in),
                                   _ptr(z), _ptr(pcode), _ptr(carry_out), _ptr(sigma2)))

    def demap(self, z: torch.Tensor, sigma2: torch.Tensor, llr: torch.Tensor):
        _ck(lib().rx_demap(self.h, _ptr(z), z.shape[-1], _ptr(sigma2), _ptr(llr)))

    def close(self):
        if getattr(self, "h", None):
            lib().rx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_PARAMS = 17926


class RxKKParams(C.Structure):
    _fields_ = [("n_ov", C.c_int), ("floor", C.c_float), ("fc_step", C.c_uint32)]


class KK:
    """Kramers-Kronig front-end: int16 ADC codes [S, n] (device) -> the
    downconverted signal field [S, n] complex64 (device)."""

    def __init__(self, fc_step: int, n_ov: int = 512, floor: float = 1e-6,
                 stream: torch.cuda.Stream | None = None):
        L = lib()
        p = RxKKParams(int(n_ov), float(floor), int(fc_step) & 0xFFFFFFFF)
        h = L.rx_kk_create(C.byref(p))
        if not h:
            raise RxError(-1, L.rx_last_error().decode())
        self.h = h
        st = stream if stream is not None else torch.cuda.current_stream()
        _ck(L.rx_kk_set_stream(h, st.cuda_stream))

    def field(self, codes: torch.Tensor, levels, out: torch.Tensor | None = None) -> torch.Tensor:
        """levels: [S, 2] (photocurrent per code, DC term) per stream."""
        if codes.dtype != torch.int16 or not codes.is_cuda or codes.dim() != 2 or not codes.is_contiguous():
            raise ValueError("codes must be a contiguous [S, n] int16 device tensor")
        S, n = codes.shape
        lv = np.ascontiguousarray(np.asarray(levels, dtype=np.float32).reshape(S, 2))
        if out is None:
            out = torch.empty((S, n), dtype=torch.complex64, device=codes.device)
        _ck(lib().rx_kk_field(self.h, _ptr(codes), S, n, lv.ctypes.data, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().rx_kk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FDE:
    """Static frequency-domain equaliser with 4 -> 2 resampling: taps
    trained by float64 least squares on known symbols, applied by the
    overlap-save kernel.  Buffers are torch complex64 device tensors."""

    def __init__(self, taps: int = 203, n_ov: int = 256, stream: torch.cuda.Stream | None = None):
        L = lib()
        h = L.rx_fde_create(int(taps), int(n_ov))
        if not h:
            raise RxError(-1, L.rx_last_error().decode())
        self.h, self.T = h, int(taps)
        st = stream if stream is not None else torch.cuda.current_stream()
        _ck(L.rx_fde_set_stream(h, st.cuda_stream))

    def train(self, x: torch.Tensor, d: torch.Tensor, sps: int = 4, delta: float = 1e-6):
        """x [n] complex64 (input rate), d [K] complex64 known symbols."""
        _ck(lib().rx_fde_train(self.h, _ptr(x), x.shape[-1], _ptr(d), d.shape[-1], int(sps), float(delta)))

    def set_taps(self, taps: np.ndarray):
        buf = np.ascontiguousarray(np.asarray(taps, dtype=np.complex128))
        if buf.shape != (self.T,):
            raise ValueError(f"expected {self.T} taps")
        _ck(lib().rx_fde_set_taps(self.h, buf.ctypes.data))

    def taps(self) -> np.ndarray:
        out = np.empty(self.T, dtype=np.complex128)
        _ck(lib().rx_fde_get_taps(self.h, out.ctypes.data))
        return out

    def apply(self, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        """x [S, n] complex64 -> y [S, n/2] complex64."""
        if x.dim() == 1:
            x = x[None]
        S, n = x.shape
        if y is None:
            y = torch.empty((S, n // 2), dtype=torch.complex64, device=x.device)
        _ck(lib().rx_fde_apply(self.h, _ptr(x), S, n, _ptr(y)))
        return y

    def close(self):
        if getattr(self, "h", None):
            lib().rx_fde_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """Learned demapper handle (MLP 4 -> 128 -> 128 -> 6); buffers are torch
    device tensors: x [n, 4] float32, sigma2 [n] float32, bits [n, 6] uint8."""

    def __init__(self, params: np.ndarray | None = None, stream: torch.cuda.Stream | None = None):
        L = lib()
        buf = None
        if params is not None:
            buf = np.ascontiguousarray(params, dtype=np.float32)
            if buf.size != MLP_PARAMS:
                raise ValueError(f"expected {MLP_PARAMS} parameters")
        h = L.rx_mlp_create(buf.ctypes.data if buf is not None else None)
        if not h:
            raise RxError(-1, L.rx_last_error().decode())
        self.h = h
        st = stream if stream is not None else torch.cuda.current_stream()
        _ck(L.rx_mlp_set_stream(h, st.cuda_stream))

    def params(self) -> np.ndarray:
        out = np.empty(MLP_PARAMS, np.float32)
        _ck(lib().rx_mlp_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, params: np.ndarray):
        buf = np.ascontiguousarray(params, dtype=np.float32)
        _ck(lib().rx_mlp_set_params(self.h, buf.ctypes.data))

    def set_param(self, key: str, value: float):
        """Kernel path: "train_tc" (1 tcgen05 GEMMs, 0 float32 SIMT) or
        "infer" (2 tcgen05, 1 mma.sync)."""
        _ck(lib().rx_mlp_set_param(self.h, key.encode(), float(value)))

    def get_param(self, key: str) -> float:
        v = C.c_double()
        _ck(lib().rx_mlp_get_param(self.h, key.encode(), C.byref(v)))
        return v.value

    def grad(self, x, sigma2, bits):
        g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _ck(lib().rx_mlp_grad(self.h, _ptr(x), _ptr(sigma2), _ptr(bits), x.shape[0], _ptr(g), _ptr(loss)))
        return g, loss

    def train_step(self, x, sigma2, bits, lr: float, loss: torch.Tensor | None = None):
        _ck(lib().rx_mlp_train_step(self.h, _ptr(x), _ptr(sigma2), _ptr(bits), x.shape[0], lr, _ptr(loss)))

    def infer(self, x, sigma2, llr: torch.Tensor | None = None):
        if llr is None:
            llr = torch.empty((x.shape[0], 6), dtype=torch.float32, device=x.device)
        _ck(lib().rx_mlp_infer(self.h, _ptr(x), _ptr(sigma2), x.shape[0], _ptr(llr)))
        return llr

    def close(self):
        if getattr(self, "h", None):
            lib().rx_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def issue_rate(kind: int, iters: int = 4096) -> tuple[float, float]:
    """(lane-instructions per second, device ms) of one FP32 instruction kind
    (0 FFMA, 1 FFMA2, 2 FMNMX) on the current device."""
    rate, ms = C.c_double(), C.c_double()
    _ck(lib().rx_issue_rate(int(kind), int(iters), C.byref(rate), C.byref(ms)))
    return rate.value, ms.value


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class Server:
    """Continuous batching over streams (rx_server_*): requests are admitted
    in arrival order as slots and the device-memory budget allow, and every
    step issues one block of each running request."""

    def __init__(self, mem_budget: int, max_slots: int):
        h = lib().rx_server_create(int(mem_budget), int(max_slots))
        if not h:
            raise RxError(-1, lib().rx_server_last_error().decode())
        self.h = h
        self._keep = {}

    def _ck(self, rc):
        if rc != 0:
            raise RxError(rc, lib().rx_server_last_error().decode())

    def set_param(self, key: str, value: float):
        """"issue" (the handles' issue mode, 0/1/2), "issue_threads", "blocks_per_step" or "block_latency"."""
        self._ck(lib().rx_server_set_param(self.h, key.encode(), float(value)))

    def get_param(self, key: str) -> float:
        """A setting, or the counters "handles_created", "handles_destroyed", "handle_regrows"."""
        v = _D()
        self._ck(lib().rx_server_get_param(self.h, key.encode(), C.byref(v)))
        return v.value

    def block_latency(self) -> list[float]:
        """Device ms of each timed issue call ("block_latency" on), retired requests only."""
        n = _SZ()
        self._ck(lib().rx_server_get_block_latency(self.h, None, 0, C.byref(n)))
        buf = (_D * max(1, n.value))()
        self._ck(lib().rx_server_get_block_latency(self.h, buf, n.value, C.byref(n)))
        return list(buf[:n.value])

    def submit(self, fmt: str, samples: torch.Tensor, llr: torch.Tensor, bits: torch.Tensor | None = None,
               *, cd_ps_per_nm: float, taps: int, bps_phases: int, symbol_rate: float = 28e9, sps: int = 2,
               fft: int = 0, overlap: int = 0, block: int = 0, n_pre: int = 0) -> int:
        """samples [2, 2N] complex64, llr [N, m] float32, bits [N, m] uint8 (device)."""
        f, keep = make_format(fmt)
        r = RxRequest(format=f, symbol_rate=symbol_rate, sps=sps, cd_ps_per_nm=cd_ps_per_nm, taps=taps,
                      bps_phases=bps_phases, fft=fft, overlap=overlap, block=block, n_pre=n_pre,
                      samples=_ptr(samples), n_samples=samples.shape[-1], llr_out=_ptr(llr),
                      ref_bits=_ptr(bits))
        rid = C.c_uint64()
        self._ck(lib().rx_server_submit(self.h, C.byref(r), C.byref(rid)))
        self._keep[rid.value] = (samples, llr, bits, keep)
        return rid.value

    def step(self) -> int:
        n = C.c_int()
        self._ck(lib().rx_server_step(self.h, C.byref(n)))
        return n.value

    def run(self):
        self._ck(lib().rx_server_run(self.h))

    def start(self):
        """The server's own loop: admits and issues without step() calls."""
        self._ck(lib().rx_server_start(self.h))

    def stop(self):
        self._ck(lib().rx_server_stop(self.h))

    def poll(self, rid: int):
        st = C.c_int()
        stats = RxStats()
        self._ck(lib().rx_server_poll(self.h, rid, C.byref(st), C.byref(stats)))
        return st.value, (stats.as_dict() if st.value == REQ_DONE else None)

    def info(self) -> dict:
        used, mx, steps = C.c_size_t(), C.c_int(), C.c_long()
        self._ck(lib().rx_server_info(self.h, C.byref(used), C.byref(mx), C.byref(steps)))
        return {"mem_used": used.value, "max_active": mx.value, "steps": steps.value}

    def close(self):
        if getattr(self, "h", None):
            lib().rx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
