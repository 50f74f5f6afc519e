"""GPU parity of the tensor-core split-precision path against the FP64 oracle.

Tolerances (relative discrete l2 against FP64), derived from the split
arithmetic: a BF16 pair carries 16 significant bits (dropped terms ~3 * 2^-17
per product), an FP16 pair 22 bits (~3 * 2^-23), both amplified by the
cancellation in D u of smooth or random fields and then accumulated in FP32.
"""
import numpy as np
import pytest

import oracle as O
import paper_1211_0582_gb300 as dg
import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 2e-4, "fp16x3": 1e-5}


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def pair(N, n, precision, eps=True):
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    e = W.element_eps(K, seed=2) if eps else None
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV, eps=e)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=None if e is None else e.astype(np.float64))
    return s, m


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("N,n", [(1, 3), (2, 3), (3, 3), (4, 3), (5, 4), (6, 3), (7, 3)])
def test_tc_rhs_parity(precision, N, n):
    s, m = pair(N, n, precision)
    u = np.random.default_rng(11).standard_normal(m.shape)
    for alpha in (1.0, 0.0):
        ref = m.rhs(u, alpha)
        got = s.from_device(s.rhs(s.to_device(u), alpha=alpha))
        err = rel_l2(got, ref)
        print(f"{precision} N={N} alpha={alpha}: rel l2 {err:.3e}")
        assert err < TOL[precision]
    s.sync()


@pytest.mark.parametrize("N,n", [(5, 4), (7, 3)])
def test_fp32_tc_precision_is_the_fp32_accurate_split(N, n):
    # DG_FP32_TC asks for FP32-level accuracy on the tensor cores: the FP16x3
    # split, bit for bit, within the FP32 tolerance of the oracle
    s, m = pair(N, n, "fp32_tc")
    s16, _ = pair(N, n, "fp16x3")
    u = np.random.default_rng(12).standard_normal(m.shape)
    got = s.from_device(s.rhs(s.to_device(u)))
    np.testing.assert_array_equal(got, s16.from_device(s16.rhs(s16.to_device(u))))
    assert rel_l2(got, m.rhs(u)) < 1e-5


@pytest.mark.parametrize("N,precision", [(3, "fp32"), (6, "fp32"), (4, "fp16x3"), (5, "bf16x3"), (7, "fp16x3"),
                                         (6, "bf16x3")])
def test_step_ignores_entry_residual(N, precision):
    # a_1 = 0: the first stage of every step overwrites the residual without
    # reading it, so a NaN residual on entry gives the same step as a zero one
    import torch
    VX, VY, VZ, EToV = W.kuhn_cube(3, jitter=0.1, seed=1)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV, eps=W.element_eps(EToV.shape[0], seed=2))
    x, y, z = s.node_coords()
    u0 = W.gaussian_pulse(x, y, z, seed=7)
    outs = []
    for fill in (0.0, float("nan")):
        u, r = s.to_device(u0), s.zeros()
        r.fill_(fill)
        s.step(u, r, 1e-3, 2)
        outs.append((s.from_device(u), r.cpu().numpy()))
    assert np.isfinite(outs[1][0]).all()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    torch.cuda.synchronize()


@pytest.mark.parametrize("N", [5, 7])
def test_fp16_flux_scale_per_field_type(N):
    # the FP16 flux split takes one power-of-two scale per field type of a tile:
    # with H about 1/377 of E (SI units, H ~ E / Z0) each type keeps its own
    # relative accuracy
    s, m = pair(N, 3, "fp16x3")
    u = np.random.default_rng(12).standard_normal(m.shape)
    u[3:] /= 376.73
    ref = m.rhs(u)
    got = s.from_device(s.rhs(s.to_device(u)))
    for sl, name in ((slice(0, 3), "E"), (slice(3, 6), "H")):
        err = rel_l2(got[sl], ref[sl])
        print(f"N={N} {name}: rel l2 {err:.3e}")
        assert err < TOL["fp16x3"]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
def test_tc_smooth_field_and_scaling(precision):
    # a smooth field (strong cancellation in D u) at tiny and large magnitudes:
    # the FP16 row scaling must keep the relative error independent of scale.
    s, m = pair(5, 3, precision)
    x, y, z = m.coords()
    u = W.cavity_mode(x, y, z, 0.0) + W.gaussian_pulse(x, y, z) * 0.01
    ref = m.rhs(u)
    for scale in (1.0, 1e-6, 1e5):
        got = s.from_device(s.rhs(s.to_device(u * scale))) / scale
        err = rel_l2(got, ref)
        print(f"{precision} scale={scale:g}: rel l2 {err:.3e}")
        assert err < 2 * TOL[precision]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("N", [4, 7])
def test_tc_lserk_steps(precision, N):
    s, m = pair(N, 3, precision)
    x, y, z = m.coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    dt = 0.5 / 3 / N ** 2
    ref, _ = m.lserk(u0, dt, 3)
    ud, rd = s.to_device(u0), s.zeros()
    s.step(ud, rd, dt, 3)
    s.sync()
    assert rel_l2(s.from_device(ud), ref) < TOL[precision]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
def test_tc_full_size_sampled(precision):
    # the 24^3 x 6 jittered mesh at N=5, the benchmark workload
    N, n = 5, 24
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    x, y, z = m.coords()
    u = W.cavity_mode(x, y, z, 0.0) + 0.05 * np.random.default_rng(17).standard_normal(m.shape)
    got = s.from_device(s.rhs(s.to_device(u)))
    elems = np.unique((W.uniform(21, 300) * m.K).astype(np.int64))
    err = rel_l2(got[:, elems], m.rhs_subset(u, elems))
    print(f"{precision} full size sampled: rel l2 {err:.3e}")
    assert err < TOL[precision]


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
def test_tc_streamed_full_size_sampled(precision):
    # the precision-form workload: 32^3 x 6 jittered tets, N=7, eps U[1,4] per
    # element (operators streamed through shared memory), several LSERK stages
    # in a row so that the operator ring wraps across tiles and launches
    N, n = 7, 32
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    e = W.element_eps(K, seed=2)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV, eps=e)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=e.astype(np.float64))
    x, y, z = m.coords()
    u = W.cavity_mode(x, y, z, 0.0) + 0.05 * np.random.default_rng(19).standard_normal(m.shape)
    ud = s.to_device(u)
    got = s.from_device(s.rhs(ud))
    elems = np.unique((W.uniform(23, 300) * K).astype(np.int64))
    err = rel_l2(got[:, elems], m.rhs_subset(u, elems))
    print(f"{precision} N=7 full size sampled: rel l2 {err:.3e}")
    assert err < TOL[precision]
    again = s.from_device(s.rhs(ud))
    assert np.array_equal(again, got)
    s.sync()


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("N", [3, 7])
def test_tc_single_partial_tile(precision, N):
    # 1^3 x 6 = 6 elements: one tile of 20 with 14 empty element slots, one CTA
    s, m = pair(N, 1, precision)
    u = np.random.default_rng(13).standard_normal(m.shape)
    err = rel_l2(s.from_device(s.rhs(s.to_device(u))), m.rhs(u))
    assert err < TOL[precision]
    x, y, z = m.coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    ref, _ = m.lserk(u0, 0.5 / N ** 2, 2)
    ud, rd = s.to_device(u0), s.zeros()
    s.step(ud, rd, 0.5 / N ** 2, 2)
    s.sync()
    assert rel_l2(s.from_device(ud), ref) < TOL[precision]


# per-element bars: FP32 path and FP16x3 at FP32 level, BF16x3 at its 16 bits
ELEM_TOL = {"fp32": 5e-6, "fp16x3": 1e-5, "bf16x3": 2e-4}


@pytest.mark.parametrize("precision", ["fp32", "fp16x3", "bf16x3"])
@pytest.mark.parametrize("N,n,width", [(4, 6, 0.05), (5, 6, 0.05), (7, 4, 0.06)])
def test_rhs_per_element_relative_error_localised_pulse(precision, N, n, width):
    # A narrow pulse: element amplitudes span 10^15 and more between
    # neighbours, and the 20 elements of a tile differ by 10^4..10^6. Each
    # element's error is measured against that element's own largest value
    # (over its six fields), so a quiet element that shares a tile with a loud
    # one must keep its own relative accuracy (the FP16 flux scales are per
    # element and field type). Elements below 1e-20 of the peak are left out
    # (FP32 itself cannot resolve them).
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    eps = W.element_eps(EToV.shape[0], seed=2)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV, eps=eps)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps.astype(np.float64))
    x, y, z = m.coords()
    u0 = W.gaussian_pulse(x, y, z, seed=7, width=width)
    ref = m.rhs(u0)
    got = s.from_device(s.rhs(s.to_device(u0)))
    s.sync()
    amp = np.abs(ref).max(axis=(0, 2))
    keep = amp > 1e-20 * amp.max()
    assert keep.sum() > 20 and amp[keep].min() < 1e-8 * amp.max()  # the range the test is about
    per_elem = np.abs(got - ref).max(axis=(0, 2))[keep] / amp[keep]
    print(f"{precision} N={N}: per-element max rel {per_elem.max():.2e}, global rel l2 {rel_l2(got, ref):.2e}")
    assert per_elem.max() < ELEM_TOL[precision]


def _ws_solver(N, n, precision, eps=True):
    # the warp-specialised form of the stage kernel (two tiles in flight per
    # SM) is chosen per context at mesh upload by DGMX_TC_FORM=ws
    import os
    old = os.environ.get("DGMX_TC_FORM")
    os.environ["DGMX_TC_FORM"] = "ws"
    try:
        return pair(N, n, precision, eps)
    finally:
        if old is None:
            os.environ.pop("DGMX_TC_FORM")
        else:
            os.environ["DGMX_TC_FORM"] = old


@pytest.mark.parametrize("precision", ["bf16x3", "fp16x3"])
@pytest.mark.parametrize("N,n", [(2, 3), (3, 4), (4, 3), (5, 4)])
def test_warp_specialised_form_parity(precision, N, n):
    s, m = _ws_solver(N, n, precision)
    rng = np.random.default_rng(11)
    u = rng.standard_normal(m.shape)
    for alpha in (1.0, 0.0):
        got = s.from_device(s.rhs(s.to_device(u), alpha=alpha))
        assert rel_l2(got, m.rhs(u, alpha)) < TOL[precision]
    x, y, z = m.coords()
    u0 = W.gaussian_pulse(x, y, z, seed=7) + W.cavity_mode(x, y, z, 0.0)
    dt = 0.5 / n / N ** 2
    ud, rd = s.to_device(u0), s.zeros()
    s.step(ud, rd, dt, 3)
    s.sync()
    ref, _ = m.lserk(u0, dt, 3)
    assert rel_l2(s.from_device(ud), ref) < TOL[precision]


def test_warp_specialised_form_wait_timeout_reports_and_recovers():
    s, m = _ws_solver(4, 4, "fp16x3")
    x, y, z = m.coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    dt = 0.5 / 4 / 16
    ud, rd = s.to_device(u0), s.zeros()
    s.step(ud, rd, dt, 2)
    s.sync()
    ref = s.from_device(ud)
    s.set_wait_limit(1)
    ud, rd = s.to_device(u0), s.zeros()
    s.step(ud, rd, dt, 2)
    with pytest.raises(dg.DGError) as ei:
        s.sync()
    assert ei.value.code == -5
    s.set_wait_limit(0)
    ud, rd = s.to_device(u0), s.zeros()
    s.step(ud, rd, dt, 2)
    s.sync()
    assert np.array_equal(s.from_device(ud), ref)
