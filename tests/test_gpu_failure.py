"""Failure detection on the GPU without a fault.

A device wait limit shorter than the work waited for (dg_set_wait_limit) makes
the kernels give up on their bounded waits, set the device flag and return;
dg_sync then reports DG_ERR_TIMEOUT, and with the default limit restored the
same context reproduces an undisturbed run bit for bit. Covered: the
tensor-core stage with resident operators (N=3), the one with operators
streamed through shared memory (N=6), and the persistent ensemble launches
(FP32 and tensor-core forms) with their grid barrier (replayed from a CUDA
graph before and after).
"""
import numpy as np
import pytest
import torch

import paper_1211_0582_gb300 as dg
import workloads as W

pytestmark = pytest.mark.gpu

TIMEOUT = -5


def _steps(s, u0, dt, nsteps):
    u, r = s.to_device(u0), s.zeros()
    s.step(u, r, dt, nsteps)
    return u


@pytest.mark.parametrize("N,precision", [(3, "fp16x3"), (6, "bf16x3")])
def test_tensor_core_wait_timeout_reports_and_recovers(N, precision):
    VX, VY, VZ, EToV = W.kuhn_cube(3, jitter=0.1, seed=1)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV)
    x, y, z = s.node_coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    dt = 0.5 / 3 / N ** 2
    u = _steps(s, u0, dt, 2)
    s.sync()
    ref = s.from_device(u)
    s.set_wait_limit(1)
    _steps(s, u0, dt, 2)
    with pytest.raises(dg.DGError) as e:
        s.sync()
    assert e.value.code == TIMEOUT
    s.sync()  # the flag was cleared
    s.set_wait_limit(0)
    u = _steps(s, u0, dt, 2)
    s.sync()
    assert np.array_equal(s.from_device(u), ref)


@pytest.mark.parametrize("N,precision", [(2, "fp32"), (3, "fp16x3")])
def test_ensemble_grid_barrier_timeout_reports_and_recovers(N, precision):
    meshes, eps, dts = [], [], []
    for i, n in enumerate((2, 3)):
        VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=10 + i)
        meshes.append((VX, VY, VZ, EToV))
        eps.append(W.element_eps(EToV.shape[0], seed=100 + i))
        dts.append(0.5 / n / N ** 2)
    ens = dg.Solver(N, precision=precision).upload_ensemble(meshes, eps, dts)
    off = ens.ensemble_layout()
    x, y, z = ens.node_coords()
    u0 = W.gaussian_pulse(x, y, z, seed=7)

    def run():
        u = ens.to_device(u0)
        res = torch.zeros_like(u)
        ens.ensemble_step(u, res, 3)
        return u

    u = run()
    ens.sync()
    ref = ens.from_device(u)
    ens.set_wait_limit(1)
    run()
    with pytest.raises(dg.DGError) as e:
        ens.sync()
    assert e.value.code == TIMEOUT
    ens.set_wait_limit(0)
    u = run()
    ens.sync()
    assert np.array_equal(ens.from_device(u), ref)
    assert off[-1] == u.shape[1]


@pytest.mark.parametrize("N,precision", [(3, "fp32"), (4, "fp16x3"), (7, "bf16x3")])
def test_step_reports_nonfinite_state(N, precision):
    # a NaN planted in the initial state (on the host) spreads through the
    # stages; with the check on, dg_step returns DG_ERR_NONFINITE, with it off
    # it returns DG_OK; a clean state passes the check
    VX, VY, VZ, EToV = W.kuhn_cube(3, jitter=0.1, seed=1)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV)
    x, y, z = s.node_coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    dt = 0.5 / 3 / N ** 2
    s.set_nonfinite_check(True)
    u, r = s.to_device(u0), s.zeros()
    s.step(u, r, dt, 2)
    assert torch.isfinite(u).all()
    bad = u0.copy()
    bad[4, 17, 3] = np.nan
    u, r = s.to_device(bad), s.zeros()
    with pytest.raises(dg.DGError) as ei:
        s.step(u, r, dt, 1)
    assert ei.value.code == -4 and "NaN" in str(ei.value)
    s.set_nonfinite_check(False)
    u, r = s.to_device(bad), s.zeros()
    s.step(u, r, dt, 1)
    s.sync()
    assert not torch.isfinite(u).all()
