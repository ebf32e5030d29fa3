"""Measurement builds (in-kernel timelines), outside the library.

``python -m paper_2605_06392_gb300.trace chain [--n 608] [--tc 1] [--ctas 65]``
compiles ``trace/chain.cu``, which includes the task-graph factor's source
with its compile-time ``DAG_TRACE`` hooks defined to stamp ``%globaltimer``.
It links against the in-tree ``libbta.so`` and runs one factor of an
``n``-row SPD block. The output is one JSON line: the factor's time and the
chain's average diagonal step, phase by phase (waiting for the bulk tasks,
the triangular product, the symmetric update, the 32-pivot leaf,
publishing). ``--tc 1`` takes the tensor-core modes' tile products,
``--tc 0`` the FP64 ones; ``--ctas`` caps the persistent grid.
Needs a GPU.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess

from . import build as _build

HERE = os.path.dirname(os.path.abspath(__file__))


def chain(n: int = 608, tc: int = 1, ctas: int = 65) -> dict:
    lib = _build.build()
    out = os.path.join(_build.OUT, "chain_trace")
    src = os.path.join(HERE, "trace", "chain.cu")
    deps = [src, lib, os.path.join(_build.CSRC, "potrf_dag.cu")] + _build._headers()
    if _build._stale(out, deps):
        cmd = [_build._nvcc(), *_build.ARCH, *_build.FLAGS, src, "-L", _build.OUT, "-lbta",
               "-lcuda", "-o", out]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + r.stderr)
    env = dict(os.environ)
    env["LD_LIBRARY_PATH"] = os.pathsep.join([_build.OUT, env.get("LD_LIBRARY_PATH", "")])
    r = subprocess.run([out, str(n), str(tc), str(ctas)], capture_output=True, text=True,
                       env=env, timeout=300)
    if r.returncode != 0:
        raise RuntimeError(r.stdout + r.stderr)
    return json.loads(r.stdout.strip().splitlines()[-1])


if __name__ == "__main__":
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("what", choices=["chain"])
    ap.add_argument("--n", type=int, default=608)
    ap.add_argument("--tc", type=int, default=1)
    ap.add_argument("--ctas", type=int, default=65)
    a = ap.parse_args()
    print(json.dumps(chain(a.n, a.tc, a.ctas)))
