"""Write the stored expected values in this folder.

Every number here comes from the FP64 CPU oracle (``oracle/``) on the seeded
synthetic workloads of ``workloads``; nothing is taken from the GPU library.
The paper prints no worked numeric example, so these fixtures are
regression anchors for the oracle itself, pinned in turn by
``tests/test_oracle_pins.py``.

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402

CASES = ["st_tiny", "coreg_tiny", "coreg_k2_small"]


def main():
    for name in CASES:
        p = workloads.make_problem(name)
        r = oracle.dense.evaluate(p)
        out = {
            "workload": name,
            "source": "oracle.dense.evaluate (Eq. 1 value, Eq. 6 gradient, dense FP64)",
            "theta": p.theta.tolist(),
            "f": r.f,
            "grad": r.grad.tolist(),
            "logdet_p": r.logdet_p,
            "logdet_c": r.logdet_c,
            "quad": r.quad,
            "loglik": r.loglik,
            "phase_a": r.phase_a.tolist(),
            "phase_b": r.phase_b.tolist(),
            "phase_c": r.phase_c.tolist(),
        }
        with open(os.path.join(HERE, f"{name}.json"), "w") as fh:
            json.dump(out, fh, indent=1)
        print("wrote", name)


if __name__ == "__main__":
    main()
