"""Writes oracle/node_alpha.txt: per order N, the blend parameter alpha of
the warp & blend nodes (Section 2's node reference) that minimises their
Lebesgue constant, found with the oracle alone.

The paper names no alpha. Here it is chosen by a search over alpha in [0, 3]:
a grid of step 0.05 with the Lebesgue constant estimated on the order-30
equidistant lattice of the tetrahedron, then a golden-section search on
+-0.15 around the grid's best point with the order-60 lattice. Orders below 3
have no alpha dependence (their face nodes are fixed by symmetry or the warp
vanishes), and neither has N = 3 (its only face-interior node is the face's
centroid); they get alpha = 0.

Usage: python oracle/optimize_node_alpha.py [Nmax]   (default 9; a few minutes)
"""
from __future__ import annotations

import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402

COARSE_M, FINE_M = 30, 60


def optimise(N: int) -> tuple[float, float, float]:
    """(alpha, Lebesgue constant at alpha, Lebesgue constant at 0), order-60 lattice."""
    lam0 = O.lebesgue(N, 0.0, FINE_M)
    if N <= 3:
        return 0.0, lam0, lam0
    grid = [0.05 * i for i in range(61)]
    vals = [O.lebesgue(N, a, COARSE_M) for a in grid]
    a_best = grid[min(range(len(grid)), key=vals.__getitem__)]
    lo, hi = max(0.0, a_best - 0.15), a_best + 0.15
    g = (math.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = hi - g * (hi - lo), lo + g * (hi - lo)
    f1, f2 = O.lebesgue(N, x1, FINE_M), O.lebesgue(N, x2, FINE_M)
    while hi - lo > 1e-3:
        if f1 <= f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - g * (hi - lo)
            f1 = O.lebesgue(N, x1, FINE_M)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + g * (hi - lo)
            f2 = O.lebesgue(N, x2, FINE_M)
    a = round(0.5 * (lo + hi), 3)
    lam = O.lebesgue(N, a, FINE_M)
    if lam >= lam0:  # no gain over the plain construction
        return 0.0, lam0, lam0
    return a, lam, lam0


def main(nmax: int = 9) -> None:
    rows = [optimise(N) for N in range(1, nmax + 1)]
    with open(os.path.join(HERE, "node_alpha.txt"), "w") as f:
        f.write("# N  alpha  Lebesgue(alpha)  Lebesgue(0); Lebesgue constants on the order-60 equidistant lattice\n")
        f.write("# written by oracle/optimize_node_alpha.py (oracle only)\n")
        for N, (a, lam, lam0) in enumerate(rows, start=1):
            f.write(f"{N} {a:.3f} {lam:.6f} {lam0:.6f}\n")
            print(f"N={N}: alpha {a:.3f}  Lebesgue {lam:.4f} (alpha = 0: {lam0:.4f})", flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 9)
