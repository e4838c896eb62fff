"""Planted mistakes in the oracle, to show that a pin bites.

``mutant(subs)`` compiles a copy of ``oracle/mhd_oracle.c`` with the given
source substitutions (each must match exactly once) into a temporary
directory and runs the oracle's Python wrappers on that build for the
duration of the ``with`` block.  The committed oracle is never modified; the
mistake lives only in the temporary copy, on the CPU.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import tempfile

import oracle as O


def build_mutant(subs, workdir: str) -> str:
    src = open(O._SRC).read()
    for old, new in subs:
        n = src.count(old)
        assert n == 1, f"mutation site {old!r} matches {n} times"
        src = src.replace(old, new)
    path = os.path.join(workdir, "mutant.c")
    with open(path, "w") as fh:
        fh.write(src)
    lib = os.path.join(workdir, "libmutant.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", lib, path, "-lm"])
    return lib


@contextlib.contextmanager
def mutant(subs):
    O.lib()   # the ordinary build exists, so the swap below is undone to it
    with tempfile.TemporaryDirectory() as d:
        L = O.bind(C.CDLL(build_mutant(subs, d)))
        old = O._lib
        O._lib = L
        try:
            yield L
        finally:
            O._lib = old
