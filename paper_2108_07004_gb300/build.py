"""Build the receiver's CUDA library (librx.so) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by its own nvcc process (in
parallel), then linked into a shared library against the shared CUDA
runtime, so that the process shares one runtime with PyTorch.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librx.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _compile(nvcc: str, src: str, verbose: bool) -> str:
    obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread",
           "-I", INCLUDE, "-I", CSRC, "-I", BUILD, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


TABLES = os.path.join(HERE, "data", "gs4d64_v1.json")


def write_tables() -> str:
    """The built-in 4D 64-ary GS table (RX_FMT_GS4D64) as C arrays from the
    frozen design file: float32 points as exact hexadecimal literals, in the
    file's row order, with their labels."""
    import json
    import struct
    with open(TABLES) as f:
        d = json.load(f)
    assert d["dims"] == 4 and d["m_bits"] == 6 and len(d["points"]) == 64

    def hexf(v: float) -> str:
        x = struct.unpack("<f", struct.pack("<f", v))[0]      # the float32 value
        return f"{float(x).hex()}f" if x != 0 else "0.0f"
    rows = ",\n".join("    {" + ", ".join(hexf(v) for v in r) + "}" for r in d["points"])
    labs = ", ".join(str(int(v)) for v in d["labels"])
    out = os.path.join(BUILD, "gs4d64_table.inc")
    text = (f"// Generated by build.py from data/gs4d64_v1.json (sha256 {d['sha256']}).\n"
            f"static const float kGs4d64Points[64][4] = {{\n{rows}}};\n"
            f"static const uint32_t kGs4d64Labels[64] = {{{labs}}};\n")
    os.makedirs(BUILD, exist_ok=True)
    if not os.path.exists(out) or open(out).read() != text:
        with open(out, "w") as f:
            f.write(text)
    return out


def build(verbose: bool = False, force: bool = False) -> str:
    srcs = sources()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".h")]
    headers.append(os.path.join(INCLUDE, "rx.h"))
    headers.append(TABLES)
    os.makedirs(BUILD, exist_ok=True)
    write_tables()
    if (not force and os.path.exists(LIB) and
            os.path.getmtime(LIB) > max(os.path.getmtime(p) for p in srcs + headers)):
        return LIB
    nvcc = _nvcc()
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(nvcc, s, verbose), srcs))
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-Xcompiler", "-pthread", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
