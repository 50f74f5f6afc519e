"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke run.

This module holds no arithmetic of the discontinuous Galerkin method: it only
builds the input data (meshes, material fields, initial fields evaluated at
coordinates supplied by the caller, receiver indices). Both the CUDA library
and the FP64 CPU oracle consume what it produces, so neither side can bias the
other through its inputs.

Random numbers come from splitmix64 (Steele, Lea and Flood, 2014): state is
advanced by the golden-gamma constant and mixed; a uniform double in [0, 1)
is (z >> 11) * 2**-53.

Workload shapes follow the paper's "large 3D Maxwell problem" on straight-sided
tetrahedra (Section 5): a unit cube cut into n^3 hexahedra, each split into six
Kuhn tetrahedra around its main diagonal, with interior vertices jittered.

Seeds used by convention: mesh jitter 1, permittivity 2, ensemble sizes 3,
receivers 4, finite-difference directions 5, target permittivity 6, pulses 7.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int) -> np.ndarray:
    """Return `count` successive splitmix64 outputs for `seed` (uint64)."""
    with np.errstate(over="ignore"):
        idx = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """`count` doubles uniform in [0, 1) from splitmix64(seed)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def hilbert_index(x, y, z, bits: int) -> np.ndarray:
    """Position of integer points (x, y, z) in [0, 2**bits)^3 along a 3D Hilbert
    curve: the axes-to-transpose conversion of J. Skilling ("Programming the
    Hilbert curve", AIP Conf. Proc. 707, 2004), then the bits of the transposed
    coordinates interleaved, most significant first. Vectorised over arrays."""
    X = [np.asarray(x, dtype=np.int64).copy(), np.asarray(y, dtype=np.int64).copy(),
         np.asarray(z, dtype=np.int64).copy()]
    Q = 1 << (bits - 1)
    while Q > 1:  # inverse undo of the excess work
        P = Q - 1
        for i in range(3):
            flip = (X[i] & Q) != 0
            X[0] = np.where(flip, X[0] ^ P, X[0])
            t = np.where(flip, 0, (X[0] ^ X[i]) & P)
            X[0] ^= t
            X[i] ^= t
        Q >>= 1
    for i in (1, 2):  # Gray encode
        X[i] ^= X[i - 1]
    t = np.zeros_like(X[0])
    Q = 1 << (bits - 1)
    while Q > 1:
        t = np.where((X[2] & Q) != 0, t ^ (Q - 1), t)
        Q >>= 1
    for i in range(3):
        X[i] ^= t
    code = np.zeros_like(X[0])
    for b in range(bits - 1, -1, -1):
        for i in range(3):
            code = (code << 1) | ((X[i] >> b) & 1)
    return code


def hilbert_hex_order(n: int) -> np.ndarray:
    """The x-fastest indices of the n^3 hexahedra of kuhn_cube in Hilbert-curve order."""
    bits = max(1, int(math.ceil(math.log2(n))))
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.argsort(hilbert_index(i.ravel(), j.ravel(), k.ravel(), bits), kind="stable")


def element_permutation(n: int, order: str) -> np.ndarray:
    """perm with EToV(order)[e] == EToV("lexicographic")[perm[e]] for kuhn_cube(n)."""
    if order == "lexicographic":
        return np.arange(6 * n ** 3)
    return (hilbert_hex_order(n)[:, None] * 6 + np.arange(6)).reshape(-1)


def kuhn_cube(n: int, jitter: float = 0.0, seed: int = 1, order: str = "lexicographic"):
    """Unit cube, n^3 hexahedra, 6 Kuhn tetrahedra per hexahedron.

    Vertex (i, j, k) has index i + (n+1)*(j + (n+1)*k). Hexahedron (i, j, k)
    (x fastest) contributes tetrahedra 6*hex + p for the 6 permutations p of
    the axes in itertools order; tetrahedron p walks from corner (0,0,0) to
    (1,1,1) along the axes in that order, so every cube shares the same main
    diagonal and the mesh is face-conforming. Odd permutations swap their
    2nd and 3rd vertex so every tetrahedron is positively oriented.

    Jitter: 3 uniforms per vertex are drawn in vertex order (x, y, z); interior
    vertices move by (2U-1)*jitter*h per coordinate, boundary vertices stay
    (the walls remain planar). Returns (VX, VY, VZ, EToV) with EToV int32 (K, 4).

    order="hilbert" lists the hexahedra along a 3D Hilbert curve instead of x
    fastest (the six tetrahedra of a hexahedron stay together), so that runs of
    consecutive elements are compact in space (the element blocking of the
    paper's Section 4); vertices and jitter are unchanged.
    """
    h = 1.0 / n
    g = np.arange(n + 1, dtype=np.float64) * h
    VZ, VY, VX = np.meshgrid(g, g, g, indexing="ij")
    VX, VY, VZ = VX.ravel().copy(), VY.ravel().copy(), VZ.ravel().copy()
    nv = (n + 1) ** 3
    if jitter > 0.0:
        U = uniform(seed, 3 * nv).reshape(nv, 3)
        ii = np.arange(nv)
        iv, jv, kv = ii % (n + 1), (ii // (n + 1)) % (n + 1), ii // ((n + 1) ** 2)
        interior = (iv > 0) & (iv < n) & (jv > 0) & (jv < n) & (kv > 0) & (kv < n)
        d = (2.0 * U - 1.0) * jitter * h
        VX[interior] += d[interior, 0]
        VY[interior] += d[interior, 1]
        VZ[interior] += d[interior, 2]

    def vid(i, j, k):
        return i + (n + 1) * (j + (n + 1) * k)

    hk, hj, hi = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    hi, hj, hk = hi.ravel(), hj.ravel(), hk.ravel()
    if order == "hilbert":
        o = hilbert_hex_order(n)
        hi, hj, hk = hi[o], hj[o], hk[o]
    elif order != "lexicographic":
        raise ValueError(f"unknown element order {order!r}")
    tets = []
    for perm in itertools.permutations((0, 1, 2)):
        c = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            nxt = c[-1].copy()
            nxt[ax] += 1
            c.append(nxt)
        vs = [vid(hi + cc[0], hj + cc[1], hk + cc[2]) for cc in c]
        inversions = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        if inversions % 2 == 1:
            vs[1], vs[2] = vs[2], vs[1]
        tets.append(np.stack(vs, axis=1))
    EToV = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return VX, VY, VZ, EToV


def element_eps(K: int, seed: int = 2, lo: float = 1.0, hi: float = 4.0) -> np.ndarray:
    """Piecewise-constant permittivity, uniform in [lo, hi) per element (float32)."""
    return (lo + (hi - lo) * uniform(seed, K)).astype(np.float32)


CAVITY_AMPLITUDE = (1.0, -2.0, 1.0)


def cavity_mode(x, y, z, t: float, a=CAVITY_AMPLITUDE):
    """Closed-form (1,1,1) eigenmode of the unit-cube PEC cavity, eps = mu = 1.

    E = Ehat cos(w t), H = -(curl Ehat) sin(w t) / w, w = sqrt(3) pi, with
    Ehat = (ax cos(pi x) sin(pi y) sin(pi z), ay sin cos sin, az sin sin cos).
    Divergence-free because ax + ay + az = 0; tangential E vanishes on every
    wall. Returns a (6, ...) array ordered Ex, Ey, Ez, Hx, Hy, Hz.
    """
    ax, ay, az = a
    pi = math.pi
    w = math.sqrt(3.0) * pi
    Sx, Sy, Sz = np.sin(pi * x), np.sin(pi * y), np.sin(pi * z)
    Cx, Cy, Cz = np.cos(pi * x), np.cos(pi * y), np.cos(pi * z)
    ct, st = math.cos(w * t), math.sin(w * t)
    Ex = ax * Cx * Sy * Sz * ct
    Ey = ay * Sx * Cy * Sz * ct
    Ez = az * Sx * Sy * Cz * ct
    f = -st / w * pi
    Hx = f * (az - ay) * Sx * Cy * Cz
    Hy = f * (ax - az) * Cx * Sy * Cz
    Hz = f * (ay - ax) * Cx * Cy * Sz
    return np.stack([Ex, Ey, Ez, Hx, Hy, Hz])


def gaussian_pulse(x, y, z, seed: int = 7, index: int = 0, width: float | None = None):
    """Divergence-free pulse E0 = curl(p g), g = exp(-|x-c|^2 / w^2), H0 = 0.

    c in [0.3, 0.7]^3, w in [0.05, 0.15], p a unit vector; all drawn from
    splitmix64(seed) at offset 7*index (width, if given, replaces the drawn w).
    curl(p g) = grad(g) x p.
    """
    U = uniform(seed, 7 * (index + 1))[7 * index:]
    c = 0.3 + 0.4 * U[0:3]
    w = 0.05 + 0.10 * U[3] if width is None else float(width)
    p = 2.0 * U[4:7] - 1.0
    p = p / np.linalg.norm(p)
    dx, dy, dz = x - c[0], y - c[1], z - c[2]
    g = np.exp(-(dx * dx + dy * dy + dz * dz) / (w * w))
    gx, gy, gz = -2.0 * dx / (w * w) * g, -2.0 * dy / (w * w) * g, -2.0 * dz / (w * w) * g
    Ex = gy * p[2] - gz * p[1]
    Ey = gz * p[0] - gx * p[2]
    Ez = gx * p[1] - gy * p[0]
    zero = np.zeros_like(Ex)
    return np.stack([Ex, Ey, Ez, zero, zero, zero])


def receivers(K: int, Np: int, R: int = 256, seed: int = 4) -> np.ndarray:
    """R distinct node indices in [0, K*Np), drawn by splitmix64 (int64, sorted by draw)."""
    out: list[int] = []
    seen: set[int] = set()
    draws = 0
    while len(out) < R:
        u = uniform(seed, draws + 4 * R)[draws:]
        draws += 4 * R
        for v in (u * (K * Np)).astype(np.int64):
            if int(v) not in seen:
                seen.add(int(v))
                out.append(int(v))
                if len(out) == R:
                    break
    return np.asarray(out, dtype=np.int64)


def ensemble_sizes(M: int = 64, seed: int = 3, lo: int = 8, hi: int = 20) -> np.ndarray:
    """M cube resolutions n drawn uniform in {lo..hi}."""
    return (lo + np.floor(uniform(seed, M) * (hi - lo + 1))).astype(np.int64)


def directions(count: int, size: int, seed: int = 5) -> np.ndarray:
    """`count` random unit directions of length `size` (uniform entries, normalised)."""
    d = 2.0 * uniform(seed, count * size).reshape(count, size) - 1.0
    return d / np.linalg.norm(d, axis=1, keepdims=True)
