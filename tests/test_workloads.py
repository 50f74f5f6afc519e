"""The element numbering of the cube mesh: the 3D Hilbert index and the
Hilbert-ordered kuhn_cube, which lists the same tetrahedra (same vertices,
same materials) as the x-fastest one, only renumbered. The operator does not
depend on the numbering, so the oracle's right-hand side of the renumbered mesh
is the same vector, renumbered."""
import os
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W

sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
import make_precision_refs as R  # noqa: E402


@pytest.mark.parametrize("bits", [1, 2, 3, 4])
def test_hilbert_index_is_a_face_adjacent_walk(bits):
    g = np.arange(1 << bits)
    x, y, z = (a.ravel() for a in np.meshgrid(g, g, g, indexing="ij"))
    code = W.hilbert_index(x, y, z, bits)
    assert np.array_equal(np.sort(code), np.arange(1 << (3 * bits)))
    o = np.argsort(code)
    path = np.stack([x[o], y[o], z[o]], axis=1)
    # consecutive points along the curve are unit steps along one axis
    assert (np.abs(np.diff(path, axis=0)).sum(axis=1) == 1).all()
    # and every aligned sub-cube of side 2^b is a contiguous run of the curve
    for b in range(1, bits):
        block = (path >> b) @ np.array([1, 1 << bits, 1 << (2 * bits)])
        runs = np.count_nonzero(np.diff(block)) + 1
        assert runs == (1 << (3 * (bits - b)))


@pytest.mark.parametrize("n", [3, 5, 8])
def test_hilbert_mesh_is_the_same_mesh_renumbered(n):
    a = W.kuhn_cube(n, jitter=0.1, seed=1)
    b = W.kuhn_cube(n, jitter=0.1, seed=1, order="hilbert")
    perm = W.element_permutation(n, "hilbert")
    assert np.array_equal(np.sort(perm), np.arange(6 * n ** 3))
    for va, vb in zip(a[:3], b[:3]):
        assert np.array_equal(va, vb)
    assert np.array_equal(b[3], a[3][perm])
    with pytest.raises(ValueError):
        W.kuhn_cube(2, order="morton")


def _in_block_faces(EToV, block):
    """Fraction of interior faces whose two elements fall in the same run of
    `block` consecutive element numbers."""
    faces = {}
    for e, v in enumerate(EToV):
        for f in ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)):
            faces.setdefault(tuple(sorted(v[list(f)])), []).append(e)
    pairs = np.array([p for p in faces.values() if len(p) == 2])
    return np.mean(pairs[:, 0] // block == pairs[:, 1] // block)


def test_hilbert_order_keeps_more_neighbours_in_a_tile():
    n = 16
    lex = _in_block_faces(W.kuhn_cube(n)[3], 20)
    hil = _in_block_faces(W.kuhn_cube(n, order="hilbert")[3], 20)
    assert hil > lex + 0.02


def test_oracle_rhs_is_independent_of_the_numbering():
    N, n = 3, 4
    perm = W.element_permutation(n, "hilbert")
    out = []
    for order in ("lexicographic", "hilbert"):
        VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1, order=order)
        eps = W.element_eps(EToV.shape[0], seed=2)
        if order == "hilbert":
            eps = eps[perm]
        m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps.astype(np.float64))
        x, y, z = m.coords()
        out.append((m.rhs(W.gaussian_pulse(x, y, z)), m.Np))
    (r_lex, Np), (r_hil, _) = out
    idx = np.arange(r_lex.size)
    moved = R.renumber_samples(idx, n, "hilbert", Np)
    np.testing.assert_array_equal(r_hil.reshape(-1)[moved], r_lex.reshape(-1)[idx])
