"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

gcc, -O2, no fast-math and no FMA contraction (-ffp-contract=off), so the oracle rounds
every operation separately on any host (aarch64 gcc contracts by default otherwise).
OpenMP parallelises over blocks only; results do not depend on the thread count.
"""

from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "map_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


FLOPS_LIB = os.path.join(HERE, "liboracle_flops.so")


def _compile(out: str, extra, force: bool) -> str:
    if not force and os.path.exists(out) and os.path.getmtime(out) >= max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "map_oracle.h"))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           *extra, "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True, cwd=HERE)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    return _compile(LIB, ["-fopenmp"], force)


def build_flop_counter(force: bool = False) -> str:
    """The same source with its flop counters compiled in, single-threaded (the counters
    are plain globals).  Used only to count operations, never to produce results."""
    return _compile(FLOPS_LIB, ["-DORACLE_COUNT_FLOPS"], force)


if __name__ == "__main__":
    print(build(force=True))
    print(build_flop_counter(force=True))
