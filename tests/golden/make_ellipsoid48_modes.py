"""Writes ellipsoid48_modes.json: the 20 electromagnetic eigenvalues nearest
sigma = 5 of the seeded ellipsoid of the 192^3 headline configuration, solved by
the oracle (oracle.eigen.shift_invert_modes, FP64 sparse shift-invert) on the
same ellipsoid at 48^3.  The full-size GPU test compares the 192^3 eigenvalues
with these within the second-order discretisation error.  Run from the
repository root:  python tests/golden/make_ellipsoid48_modes.py"""
import json
import os
import sys

sys.path.insert(0, os.getcwd())

import workloads as W  # noqa: E402
from oracle import eigen, geometry, operators  # noqa: E402


def main():
    w = W.ellipsoid_workload(48)
    k2, _, info = eigen.shift_invert_modes(operators.DMOperators(w.grid, geometry.fractions(w.phi)), w.sigma, 20)
    out = {"workload": "ellipsoid_workload(48) (seeded semi-axes of the 192^3 headline), sigma = 5",
           "source": "oracle.eigen.shift_invert_modes, 20 modes nearest sigma",
           "semi_axes": [float(a) for a in w.meta["semi_axes"]],
           "k2": [float(v) for v in k2]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ellipsoid48_modes.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["k2"])


if __name__ == "__main__":
    main()
