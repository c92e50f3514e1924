"""Write the oracle's per-cluster ranks and phases for two small workloads.

Calls only the CPU oracle and the seeded generator.  The fixtures guard the
oracle against unintended changes; any intended change to its arithmetic must
regenerate them and cite the passage that justifies it.
Run:  python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1811_11248_gb300 import inputs  # noqa: E402

CASES = {
    "ice_16x16x8_eps1e-2": (lambda: inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1,
                                                          bc="ice", shelf=0.5), 4, 1e-2),
    "ice_16x16x8_eps1e-4": (lambda: inputs.grid_operator(16, 16, 8, ratio=1e6, sigma=1.0, seed=1,
                                                          bc="ice", shelf=0.5), 4, 1e-4),
}


def compute(name):
    make, depth, eps = CASES[name]
    p = make()
    perm, lp = oracle.partition(p, 4)
    f = oracle.Factor(p, perm, lp, depth, eps)
    lines = [f"# {name}: level cluster size0 final phase", ]
    for l in range(depth):
        s0, fi, ph = f.level_info(l)
        for c in range(len(s0)):
            lines.append(f"{l} {c} {s0[c]} {fi[c]} {ph[c]}")
    x, it, rr, rc = f.pcg(rtol=1e-8)
    lines.append(f"pcg_iterations {it}")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    for name in CASES:
        with open(os.path.join(HERE, f"oracle_{name}.txt"), "w") as fh:
            fh.write(compute(name))
