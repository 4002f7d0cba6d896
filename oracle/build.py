"""Compile the FP64 CPU oracle (test infrastructure) with gcc.

Two shared objects come out of the D2Q9 source file: ``liblbm_oracle.so`` with
``real = double`` and ``liblbm_oracle_cs.so`` with ``real = double _Complex``
(symbols suffixed ``_cs``) for complex-step derivatives; the D3Q27 source gives
``liblbm3d_oracle.so``.  Contraction of multiply-add pairs is switched off so
that x86 and Arm hosts round alike.
"""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_build")
SRC = os.path.join(HERE, "lbm_oracle.c")
HDR = os.path.join(HERE, "lbm_oracle.h")

SRC3 = os.path.join(HERE, "lbm3d_oracle.c")
HDR3 = os.path.join(HERE, "lbm3d_oracle.h")

LIBS = {
    "real": os.path.join(OUT, "liblbm_oracle.so"),
    "complex": os.path.join(OUT, "liblbm_oracle_cs.so"),
    "d3q27": os.path.join(OUT, "liblbm3d_oracle.so"),
}

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-Wall"]


def _sources(kind: str):
    return (SRC3, HDR3) if kind == "d3q27" else (SRC, HDR)


def _stale(lib: str, kind: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(p) > t for p in (*_sources(kind), __file__))


def build(force: bool = False) -> dict:
    os.makedirs(OUT, exist_ok=True)
    for kind, lib in LIBS.items():
        if not force and not _stale(lib, kind):
            continue
        extra = ["-DORACLE_COMPLEX"] if kind == "complex" else []
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", *CFLAGS, *extra, "-I", HERE, _sources(kind)[0], "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return dict(LIBS)


if __name__ == "__main__":
    print(build(force=True))
