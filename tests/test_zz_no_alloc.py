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
