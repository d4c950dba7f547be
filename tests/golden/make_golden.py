"""Write the oracle regression fixtures of this folder.

The paper prints no Jacobi3D values (its figures are latencies, bandwidths and
iteration times), so these files are not the paper's numbers: they record what
the oracle computes for two small seeded cases, to show when its arithmetic
changes.  Only the oracle and the seeded input generator are called.  Run
from the repository root:

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import jacobi_inputs as J  # noqa: E402
import oracle  # noqa: E402

# (file stem, grid (nx, ny, nz), dtype, inputs, iterations)
CASES = [
    ("oracle_4x3x5_f64", (4, 3, 5), np.float64,
     dict(bc="uniform", bc_seed=11, interior="uniform", interior_seed=12), 7),
    ("oracle_5x4x3_f32", (5, 4, 3), np.float32,
     dict(bc="linear_noise", bc_seed=3, noise_amp=1e-3, interior="zero"), 9),
]


def render(grid, dtype, inputs, iters) -> str:
    """The fixture text: the interior after `iters` Jacobi iterations (x
    fastest, as exact hexadecimal floats) and the FP64 residual norms."""
    u0 = J.initial_grid(*grid, dtype=dtype, **inputs)
    u = oracle.jacobi(u0, iters)
    rn, bn, rel = oracle.residual(u)
    lines = [f"# grid {grid[0]}x{grid[1]}x{grid[2]}, {np.dtype(dtype).name}, inputs {inputs}, "
             f"{iters} iterations; written by tests/golden/make_golden.py from the oracle",
             "interior"]
    lines += [float(v).hex() for v in J.interior_of(u).astype(np.float64).ravel()]
    lines += ["residual", rn.hex(), bn.hex(), rel.hex()]
    return "\n".join(lines) + "\n"


def main():
    oracle.build()
    for stem, grid, dtype, inputs, iters in CASES:
        with open(os.path.join(HERE, stem + ".txt"), "w") as f:
            f.write(render(grid, dtype, inputs, iters))


if __name__ == "__main__":
    main()
