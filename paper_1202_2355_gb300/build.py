"""Builds the CUDA library libm2m.so in-tree for sm_103a with nvcc."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SO = os.path.join(HERE, "_build", "libm2m.so")
CSRC = os.path.join(HERE, "csrc")
SOURCES = [os.path.join(CSRC, f) for f in ("m2m_api.cu", "m2m_batch.cu", "m2m_smooth.cu", "m2m_diag.cu")]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _deps():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(ROOT, "include", "m2m.h")]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/ into _build/libm2m.so unless it is newer than every source.
    The translation units compile in parallel, then link."""
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= max(os.path.getmtime(d) for d in _deps()):
        return SO
    bdir = os.path.dirname(SO)
    os.makedirs(bdir, exist_ok=True)
    tag = f".tmp{os.getpid()}"
    # FP32 without denormals and with the hardware square root and reciprocal: the mixed
    # path's values are far from the denormal range, and its accuracy is set by FP32
    # rounding anyway; FP64 arithmetic is unaffected. No implicit contraction of a
    # multiply and an add: the code fuses with explicit fma where it means to, so that
    # every kernel inlining the same function rounds alike (a fit in a batch is
    # bit-identical to the same fit alone).
    flags = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-ftz=true", "-prec-div=false", "-prec-sqrt=false",
             "-fmad=false", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.append("-Xptxas=-v")
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + tag + ".o")
        objs.append(obj)
        procs.append(subprocess.Popen([nvcc()] + flags + ["-c", "-o", obj, src], stdout=subprocess.PIPE,
                                      stderr=subprocess.STDOUT, text=True))
    outs = [p.communicate()[0] for p in procs]
    tmp = SO + tag
    try:
        if any(p.returncode for p in procs):
            raise RuntimeError("nvcc failed:\n" + "\n".join(outs))
        r = subprocess.run([nvcc(), "-shared", ARCH, "-o", tmp] + objs, capture_output=True, text=True)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    if verbose:
        print("\n".join(outs))
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=True))
