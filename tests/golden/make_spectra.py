"""Writes the brute-force reference spectra used by the full-size parity tests.

Each file holds the eigenvalues of a seeded synthetic pencil that lie strictly
inside its contour, computed with ``oracle.brute`` (a dense QZ eigensolver:
the plain definition of the answer, Sec. 2 of the paper), plus the smallest
normalised distance of any eigenvalue to the contour.

    python tests/golden/make_spectra.py gaussian_pencil_n4096
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads  # noqa: E402
from oracle import brute  # noqa: E402

CASES = {
    "gaussian_pencil_n4096": lambda: workloads.gaussian_pencil(n=4096, seed=2, m0=128),
    "gaussian_pencil_n1024": lambda: workloads.gaussian_pencil(n=1024, seed=2, m0=32),
}


def write(name):
    cfg = CASES[name]()
    c = cfg["contour"]
    lam, _, _ = brute.eigenpairs(cfg["A"], cfg["B"])
    lam = lam[np.isfinite(lam)]
    dist = brute.contour_distance(lam, c["c"], c["R"], c["a"])
    inner = brute.inside_spectrum_from(lam, c["c"], c["R"], c["a"])
    path = os.path.join(HERE, name + ".txt")
    with open(path, "w") as f:
        f.write(f"# brute-force eigenvalues inside the contour of {name} (oracle.brute, scipy QZ)\n")
        f.write(f"# contour c={c['c']} R={c['R']} a={c['a']}; n_inside={len(inner)}; "
                f"min_boundary_distance={dist.min():.6e}\n")
        for z in inner:
            f.write(f"{z.real:.17e} {z.imag:.17e}\n")
    print(path, len(inner), dist.min())


if __name__ == "__main__":
    for name in sys.argv[1:] or list(CASES):
        write(name)
