"""Write the FP64 reference samples of the two precision workloads.

The benchmark compares the FP32, BF16x3 and FP16x3 paths on the workloads the
method is measured on, after the full run lengths, against the FP64 oracle:

  cavity_n5_24cube_500steps     24^3 x 6 = 82,944 jittered tetrahedra, N = 5,
                                eps = mu = 1, the (1,1,1) cavity mode at t = 0,
                                upwind flux, 500 LSERK4 steps of dt = 0.5 h / N^2
  precision_n7_32cube_200steps  32^3 x 6 = 196,608 jittered tetrahedra, N = 7,
                                eps uniform in [1, 4) per element (seed 2), mu = 1,
                                the same initial field, 200 steps

An FP64 run of these sizes takes hours on one core, so this script runs the
oracle once (its OpenMP build: the elements of each right-hand side split over
threads, the arithmetic of each element unchanged) and stores, per workload,
the reference values at 65,536 node values drawn by splitmix64 (seed 41) over
the [6][K][Np] field vector, with the reference's full-field l2 norm and
maximum. The relative l2 error over the sample estimates the full-field one.

Only the oracle and the seeded input generators are used here; nothing comes
from the CUDA library. Usage: OMP_NUM_THREADS=8 python tests/golden/make_precision_refs.py [name ...]
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

SAMPLES = 65536
SAMPLE_SEED = 41
CONFIGS = {
    "cavity_n5_24cube_500steps": dict(N=5, n=24, steps=500, eps_seed=None),
    "precision_n7_32cube_200steps": dict(N=7, n=32, steps=200, eps_seed=2),
}


def path(name: str) -> str:
    return os.path.join(HERE, f"ref_{name}.npz")


def sample_indices(K: int, Np: int) -> np.ndarray:
    """Sorted distinct flat indices into a [6][K][Np] field vector."""
    total = 6 * K * Np
    return np.unique((W.uniform(SAMPLE_SEED, SAMPLES) * total).astype(np.int64))


def setup(name: str, order: str = "lexicographic"):
    """Mesh, materials, initial field generator and step size of a workload
    (shared by this script and the benchmark; no method arithmetic). The stored
    samples index the lexicographic element order; `order` renumbers the same
    elements (each keeps its vertices and its material)."""
    c = CONFIGS[name]
    VX, VY, VZ, EToV = W.kuhn_cube(c["n"], jitter=0.1, seed=1, order=order)
    K = EToV.shape[0]
    eps = None if c["eps_seed"] is None else \
        W.element_eps(K, seed=c["eps_seed"])[W.element_permutation(c["n"], order)]
    dt = 0.5 / c["n"] / c["N"] ** 2
    return c, (VX, VY, VZ, EToV), eps, dt


def renumber_samples(idx: np.ndarray, n: int, order: str, Np: int) -> np.ndarray:
    """Flat indices into a [6][K][Np] field vector of kuhn_cube(n) in the
    lexicographic element order, moved to the numbering of kuhn_cube(n, order=order)."""
    perm = W.element_permutation(n, order)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(perm.size)
    K = perm.size
    f, rem = np.divmod(idx, K * Np)
    e, j = np.divmod(rem, Np)
    return f * K * Np + inv[e] * Np + j


def write(name: str) -> None:
    import oracle as O
    c, (VX, VY, VZ, EToV), eps, dt = setup(name)
    t0 = time.time()
    m = O.Mesh(c["N"], VX, VY, VZ, EToV, eps=None if eps is None else eps.astype(np.float64))
    x, y, z = m.coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    del x, y, z
    u, _ = m.lserk(u0, dt, c["steps"])
    idx = sample_indices(m.K, m.Np)
    flat = u.reshape(-1)
    np.savez(path(name), idx=idx, ref=flat[idx], norm_full=np.linalg.norm(flat), max_full=np.abs(flat).max(),
             N=c["N"], n=c["n"], steps=c["steps"], dt=dt, K=m.K, Np=m.Np,
             source=np.array(f"FP64 oracle (OpenMP build), {c['steps']} LSERK4 steps, upwind flux, "
                             f"written by make_precision_refs.py in {time.time() - t0:.0f} s"))
    print(f"{name}: K={m.K} steps={c['steps']} samples={idx.size} |u|={np.linalg.norm(flat):.6e} "
          f"({time.time() - t0:.0f} s)", flush=True)


def load(name: str) -> dict:
    with np.load(path(name)) as f:
        return {k: f[k] for k in f.files}


if __name__ == "__main__":
    import oracle as O
    O.use_openmp()
    for name in (sys.argv[1:] or list(CONFIGS)):
        write(name)
