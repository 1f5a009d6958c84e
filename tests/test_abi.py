"""The C-ABI library builds, loads and exports every entry point of
include/rx.h (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "rx.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rx_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2108_07004_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_chain():
    names = _declared()
    for n in ("rx_create", "rx_process", "rx_destroy", "rx_cdc", "rx_fir", "rx_lms",
              "rx_bps", "rx_unwrap", "rx_demap"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for n in _declared():
        assert hasattr(lib, n), n


def test_binding_prototypes_cover_the_header():
    from paper_2108_07004_gb300 import rx
    assert sorted(rx.exported_symbols()) == _declared()


def test_error_path_without_device(lib):
    lib.rx_last_error.restype = ctypes.c_char_p
    lib.rx_create.restype = ctypes.c_void_p
    # NULL format is rejected before any device work
    assert lib.rx_create(None, ctypes.c_double(28e9), 2, ctypes.c_double(0.0), 15, 32) is None
    assert b"format" in lib.rx_last_error()
    lib.rx_destroy(None)    # NULL-safe


def test_builtin_gs4d64_table_is_the_design_file():
    """The C arrays build.py writes for RX_FMT_GS4D64 hold exactly the float32
    points and labels of data/gs4d64_v1.json."""
    import json
    import numpy as np
    from paper_2108_07004_gb300 import build
    text = open(build.write_tables()).read()
    body = text.split("kGs4d64Points[64][4] = {", 1)[1].split("};", 1)[0]
    vals = [float.fromhex(v.strip().rstrip("f")) for v in re.findall(r"-?0x[0-9a-fp.+-]+f|0\.0f", body)]
    labs = [int(v) for v in text.split("kGs4d64Labels[64] = {", 1)[1].split("}", 1)[0].split(",")]
    d = json.load(open(os.path.join(ROOT, "paper_2108_07004_gb300", "data", "gs4d64_v1.json")))
    assert np.array_equal(np.array(vals, np.float32).reshape(64, 4), np.array(d["points"], np.float32))
    assert labs == d["labels"]


def test_server_settings_and_counters_without_device(lib):
    """The server's settings are validated and read back and its handle
    counters start at zero; none of it touches the device (no request)."""
    from paper_2108_07004_gb300 import rx
    srv = rx.Server(1 << 30, 4)
    for key, good, bad in (("issue", (0, 1, 2), (3, -1, 0.5)), ("issue_threads", (1, 3, 64), (0, 65, 1.5)),
                           ("blocks_per_step", (1, 4, 1 << 20), (0, (1 << 20) + 1, 2.5)),
                           ("block_latency", (1, 0), (2, -1, 0.5))):
        for v in good:
            srv.set_param(key, v)
            assert srv.get_param(key) == v
        for v in bad:
            with pytest.raises(rx.RxError):
                srv.set_param(key, v)
    for key in ("handles_created", "handles_destroyed", "handle_regrows"):
        assert srv.get_param(key) == 0
    assert srv.block_latency() == []
    assert srv.get_param("running") == 0
    with pytest.raises(rx.RxError):
        srv.stop()                           # no loop to stop
    for key in ("nothing", "slots"):
        with pytest.raises(rx.RxError):
            srv.get_param(key)
        with pytest.raises(rx.RxError):
            srv.set_param(key, 1)
    srv.close()


def test_server_loop_start_and_stop_without_requests(lib):
    """rx_server_start either starts the server's loop (a device is present:
    it idles with nothing submitted, and rx_server_stop ends it) or, with no
    device, fails with an error and leaves no loop running."""
    from paper_2108_07004_gb300 import rx
    srv = rx.Server(1 << 30, 4)
    try:
        srv.start()
    except rx.RxError:
        assert srv.get_param("running") == 0
    else:
        assert srv.get_param("running") == 1
        with pytest.raises(rx.RxError):
            srv.step()                       # steps come from the loop while it runs
        srv.stop()
        assert srv.get_param("running") == 0
    srv.close()
