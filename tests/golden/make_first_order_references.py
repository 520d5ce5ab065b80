"""Write the first-order reference solutions of Examples 6.5, 6.6 and 6.8 (arXiv
2510.11527).

The paper compares its 1D results with a first-order scheme on 2000 cells (Section 6,
Examples 6.5 and 6.8); Example 6.6 gets the same kind of reference here. This script runs the oracle's first-order LLF + central-difference
scheme (``oracle.first_order_run``) on 2000 cells from the examples' initial data and
stores the cell averages at the final time. It calls only ``oracle`` and the seeded input
module; nothing here comes from the CUDA library.

    python tests/golden/make_first_order_references.py [file ...]   (about 3 minutes)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import af_inputs as ai  # noqa: E402
import oracle  # noqa: E402

CASES = [
    ("evje_karlsen_first_order_2000.txt", ai.evje_karlsen,
     "Example 6.5 (Evje and Karlsen): f = u^2/4, a = 0 / 5(2u-1)^2/4 / u - 11/20, [-1, 1], "
     "Dirichlet u(-1) = 1, u(1) = 0, T = 1"),
    ("strongly_degenerate_first_order_2000.txt", ai.strongly_degenerate_1d,
     "Example 6.8: f = u^2, a = 0.1 (u + 0.25) / 0 / 0.1 (u - 0.25), [-2, 2], outflow, T = 0.7"),
]
for _g in (False, True):
    for _p in ("ibvp", "rp"):
        CASES.append((f"buckley_leverett_{_p}_{'gravity' if _g else 'nogravity'}_first_order_2000.txt",
                      lambda g=_g, p=_p: ai.buckley_leverett_1d(100, g, p),
                      f"Example 6.6 ({_p}, {'with' if _g else 'without'} gravity): f = u^2/(u^2+(1-u)^2)"
                      f"{' (1 - 5(1-u)^2)' if _g else ''}, a = 0.01 (2u^2 - 4u^3/3) on [0, 1], [0, 1], "
                      f"Dirichlet {'u(0) = 1, u(1) = 0' if _p == 'ibvp' else 'u(0) = 0, u(1) = 1'}, T = 1"))


def main():
    only = set(sys.argv[1:])
    for fname, make, what in CASES:
        if only and fname not in only:
            continue
        spec = make().with_size(2000)
        ub0 = ai.initial_state(spec)[0].numpy()
        ub, nsteps = oracle.first_order_run(spec, ub0, spec.T)
        with open(os.path.join(HERE, fname), "w") as f:
            f.write(f"# {what}\n")
            f.write(f"# first-order LLF + central-difference scheme, 2000 cells, forward Euler, "
                    f"cfl 0.9, {nsteps} steps; one cell average per line, left to right\n")
            for v in ub:
                f.write(f"{v:.17g}\n")
        print(fname, nsteps, float(np.min(ub)), float(np.max(ub)))


if __name__ == "__main__":
    main()
