"""dg_step_noalloc: LSERK4 stepping that allocates no device memory.

Some callers cannot let the library allocate device memory (their allocator
owns the GPU's memory up front, or their time loop must not risk a cudaMalloc
stall); for them dg_step_noalloc takes its stage buffer from a fixed array in
the library image. It must produce what dg_step produces. This file is named
to be collected last, so that a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1211_0582_gb300 as dg
import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(s, u, res, dt, nsteps, alpha=1.0):
    return dg.lib().dg_step_noalloc(s._h, C.c_void_p(u.data_ptr()), C.c_void_p(res.data_ptr()),
                                    float(dt), int(nsteps), float(alpha))


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_noalloc_step_matches_dg_step(precision):
    N, n = 4, 8
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    eps = W.element_eps(EToV.shape[0], seed=2)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV, eps=eps)
    x, y, z = s.node_coords()
    u0 = W.cavity_mode(x, y, z, 0.0) + 0.01 * W.gaussian_pulse(x, y, z)
    dt = 0.5 / n / N ** 2
    ua, ra = s.to_device(u0), s.zeros()
    ub, rb = s.to_device(u0), s.zeros()
    for nsteps in (3, 2):  # two calls in a row, odd then even step count
        s.step(ua, ra, dt, nsteps)
        assert _noalloc(s, ub, rb, dt, nsteps) == 0, dg.lib().dg_last_error(s._h)
        s.sync()
        a, b = s.from_device(ua), s.from_device(ub)
        err = np.linalg.norm(a - b) / np.linalg.norm(a)
        assert err < 1e-5, err
        ra_h, rb_h = s.from_device(ra), s.from_device(rb)
        assert np.linalg.norm(ra_h - rb_h) <= 1e-5 * np.linalg.norm(ra_h)


def test_noalloc_rejects_meshes_beyond_its_fixed_scratch():
    N, n = 5, 14  # 6 * 16464 * 56 floats > 4 Mi floats
    VX, VY, VZ, EToV = W.kuhn_cube(n)
    s = dg.Solver(N).upload(VX, VY, VZ, EToV)
    u, r = s.zeros(), s.zeros()
    assert _noalloc(s, u, r, 1e-3, 1) == -1
    assert b"16 MiB" in dg.lib().dg_last_error(s._h)


def test_noalloc_allocates_nothing_and_ignores_stale_scratch():
    # The fixed array is shared and keeps the previous call's contents: a call
    # that fills it with non-finite values (an N=2 mesh whose state holds NaN
    # and Inf) must not leak into a later N=4 run, whose padded rows (Np=35,
    # Np_pad=36) differ from N=2's. And a call performs no device allocation:
    # the free device memory is unchanged across calls on a new mesh and order
    # (the first call of the process may load the library's device code).
    import torch
    n = 6
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    s2 = dg.Solver(2).upload(VX, VY, VZ, EToV)
    x, y, z = s2.node_coords()
    poison = W.cavity_mode(x, y, z, 0.0)
    poison[1] = np.nan
    poison[4] = np.inf
    u2, r2 = s2.to_device(poison), s2.zeros()
    assert _noalloc(s2, u2, r2, 1e-3, 3) == 0, dg.lib().dg_last_error(s2._h)
    s2.sync()
    assert not torch.isfinite(u2).all()
    s4 = dg.Solver(4, precision="fp16x3").upload(VX, VY, VZ, EToV, eps=W.element_eps(EToV.shape[0], seed=2))
    x, y, z = s4.node_coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    dt = 0.5 / n / 16
    ua, ra = s4.to_device(u0), s4.zeros()
    ub, rb = s4.to_device(u0), s4.zeros()
    s4.step(ua, ra, dt, 3)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _noalloc(s4, ub, rb, dt, 3) == 0, dg.lib().dg_last_error(s4._h)
    s4.sync()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.isfinite(ub).all()
    a, b = s4.from_device(ua), s4.from_device(ub)
    assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(a)
