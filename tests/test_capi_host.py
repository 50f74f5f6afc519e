"""Host-side checks of the C ABI (no GPU needed).

The library must load and export every entry point declared in include/*.h,
and its host-side setup (nodes, Vandermonde-based operators, LIFT, face
masks, mesh validation) must agree with the independently written oracle.
"""
import ctypes as C
import glob
import os
import re

import numpy as np
import pytest

import oracle as O
import paper_1211_0582_gb300 as dg
import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = dg.lib()
    names = declared_symbols()
    assert "dg_rhs" in names and "dg_step" in names and "dg_mesh_upload" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_host_operators_match_oracle(N):
    s = dg.Solver(N, stream=None)
    ops = s.operators()
    r, si, t = O.nodes(N)
    np.testing.assert_allclose(ops["r"], r, atol=1e-14)
    np.testing.assert_allclose(ops["s"], si, atol=1e-14)
    np.testing.assert_allclose(ops["t"], t, atol=1e-14)
    ref = O.operators(N)
    scale = max(1.0, N * N)
    for key in ("Dr", "Ds", "Dt"):
        np.testing.assert_allclose(ops[key], ref[key], atol=1e-12 * scale)
    np.testing.assert_allclose(ops["M"], ref["M"], atol=1e-13)
    np.testing.assert_allclose(ops["LIFT"], ref["LIFT"], atol=1e-11 * scale)
    np.testing.assert_array_equal(ops["Fmask"], ref["Fmask"])


@pytest.mark.parametrize("N", [5, 7, 9])
def test_host_operators_on_blended_nodes_match_oracle(N):
    # the library's table of blend parameters equals the oracle's, and the
    # operators built on those nodes match the oracle's
    alpha = dg.optimised_node_alpha(N)
    assert alpha == O.optimal_alpha(N)
    s = dg.Solver(N, stream=None, node_alpha="optimised")
    ops = s.operators()
    for got, ref in zip((ops["r"], ops["s"], ops["t"]), O.nodes(N, alpha)):
        np.testing.assert_allclose(got, ref, atol=1e-14)
    ref = O.operators(N, alpha)
    scale = max(1.0, N * N)
    for key in ("Dr", "Ds", "Dt"):
        np.testing.assert_allclose(ops[key], ref[key], atol=1e-12 * scale)
    np.testing.assert_allclose(ops["M"], ref["M"], atol=1e-13)
    np.testing.assert_allclose(ops["LIFT"], ref["LIFT"], atol=1e-11 * scale)
    np.testing.assert_array_equal(ops["Fmask"], ref["Fmask"])


def test_node_alpha_table_and_limits():
    assert [dg.optimised_node_alpha(N) for N in range(1, 10)] == [O.optimal_alpha(N) for N in range(1, 10)]
    L = dg.lib()
    assert L.dg_optimised_node_alpha(0) == -1.0 and L.dg_optimised_node_alpha(10) == -1.0
    s = dg.Solver(4, stream=None)
    assert L.dg_set_node_alpha(s._h, -0.5) == -1
    assert L.dg_set_node_alpha(s._h, 11.0) == -1
    assert L.dg_set_node_alpha(s._h, 0.7) == 0
    r = np.zeros(s.Np)
    assert L.dg_operators(s._h, r.ctypes.data, None, None, None, None, None, None, None, None) == 0
    np.testing.assert_allclose(r, O.nodes(4, 0.7)[0], atol=1e-14)


def test_create_rejects_bad_arguments():
    L = dg.lib()
    h = C.c_void_p()
    assert L.dg_create(C.byref(h), 0, 0, None) == -1
    assert L.dg_create(C.byref(h), 10, 0, None) == -1
    assert L.dg_create(C.byref(h), 3, 9, None) == -1
    assert b"precision" in L.dg_last_error(None)
    assert L.dg_create(C.byref(h), 3, 4, None) == -1
    assert L.dg_create(C.byref(h), 3, 3, None) == 0  # DG_FP32_TC
    assert L.dg_destroy(h) == 0
    assert L.dg_create(None, 3, 0, None) == -1


def test_mesh_validation_on_host():
    s = dg.Solver(2, stream=None)
    VX, VY, VZ, EToV = W.kuhn_cube(2)
    bad = EToV.copy()
    bad[3, 1] = VX.size + 5
    with pytest.raises(dg.DGError) as e:
        s.upload(VX, VY, VZ, bad)
    assert e.value.code == -2
    # a face shared by three elements: duplicate one tetrahedron
    dup = np.concatenate([EToV, EToV[:1]], axis=0)
    with pytest.raises(dg.DGError) as e:
        s.upload(VX, VY, VZ, dup)
    assert e.value.code == -2
    with pytest.raises(dg.DGError) as e:
        s.upload(VX, VY, VZ, EToV, eps=-np.ones(EToV.shape[0]))
    assert e.value.code == -1
    bc = np.zeros((EToV.shape[0], 4), dtype=np.int32)
    with pytest.raises(dg.DGError) as e:
        s.upload(VX, VY, VZ, EToV, bc=bc)
    assert e.value.code == -6
    # no mesh yet: the field entry points refuse
    L = dg.lib()
    assert L.dg_rhs(s._h, None, None, 1.0) == -1


def test_wait_limit_validation_on_host():
    s = dg.Solver(3, stream=None)
    s.set_wait_limit(0)
    s.set_wait_limit(1 << 20)
    with pytest.raises(dg.DGError) as e:
        s.set_wait_limit(-1)
    assert e.value.code == -1
    assert dg.lib().dg_set_wait_limit(None, 5) == -1
