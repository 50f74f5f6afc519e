"""GPU checks of the hand-written discrete adjoint (FP32 kernels, the reverse
stage's contractions on the tensor cores or the CUDA cores, FP64 reductions).

- transpose identity <A u, v> = <u, A^T v> and parity of A^T with the oracle;
- receiver traces and the misfit gradient against the FP64 oracle's discrete
  adjoint on the 6^3 x 6 version of the adjoint workload (N=4);
- both forms of the reverse stage against the oracle at N = 1..5, and the
  tensor-core form's bounded waits (timeout reported, context reusable);
- the same gradient for every segmentation of the run (recomputed segments,
  segments aligned to the end with the last one stored, one stored segment,
  the automatic choice);
- central finite differences (step 1e-3, 16 seeded directions) of the misfit
  on the 20^3 x 6 adjoint workload (48,000 tets, N=4, 400 steps, checkpoints
  every 20 steps, 256 receivers).
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_1211_0582_gb300 as dg
import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def setup(N, n, eps_seed=2, precision="fp32"):
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=eps_seed)
    s = dg.Solver(N, precision=precision).upload(VX, VY, VZ, EToV, eps=eps)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps.astype(np.float64))
    return s, m, eps


@pytest.mark.parametrize("N,n", [(2, 3), (4, 3), (5, 2), (7, 2), (9, 1)])
def test_transpose_parity_and_identity(N, n):
    s, m, _ = setup(N, n)
    rng = np.random.default_rng(3)
    u, v = rng.standard_normal(m.shape), rng.standard_normal(m.shape)
    for alpha in (1.0, 0.0):
        got = s.from_device(s.rhs_transpose(s.to_device(v), alpha=alpha))
        assert rel(got, m.rhs_transpose(v, alpha)) < 1e-5
        Au = s.from_device(s.rhs(s.to_device(u), alpha=alpha))
        lhs, rhs = np.vdot(Au, v), np.vdot(u, got)
        assert abs(lhs - rhs) < 1e-5 * np.linalg.norm(Au) * np.linalg.norm(v)


def _misfit_problem(N, n, steps, precision="fp32"):
    s, m, eps = setup(N, n, eps_seed=2, precision=precision)
    K = m.K
    x, y, z = s.node_coords()
    u0 = W.gaussian_pulse(x, y, z, seed=7)
    recv = W.receivers(K, s.Np, 256 if K * s.Np > 4096 else 32, seed=4)
    dt = 0.5 / n / N ** 2
    eps_t = W.element_eps(K, seed=6)
    u0d = s.to_device(u0)
    rd = torch.as_tensor(recv, device="cuda")
    Eref = s.receiver_traces(u0d, rd, dt, steps, eps=torch.as_tensor(eps_t, device="cuda"))
    return s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt


def test_receiver_traces_match_oracle():
    N, n, steps = 4, 3, 6
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    ref = m.receiver_traces(u0, dt, steps, recv, eps=eps_t.astype(np.float64))
    assert rel(Eref.double().cpu().numpy(), ref) < 1e-5


def test_adjoint_gradient_matches_oracle_discrete_adjoint():
    # 6^3 x 6 = 1,296 tets at N=4, checkpoints every 5 of 12 steps (one partial segment)
    N, n, steps, ck = 4, 6, 12, 5
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    epsd = torch.as_tensor(eps, device="cuda")
    J, g_eps, g_u0 = s.adjoint(u0d, rd, Eref, dt, steps, ck, eps=epsd)
    Jo, go_eps, go_u0 = m.misfit_gradient(u0, dt, steps, recv, Eref.double().cpu().numpy(),
                                          eps=eps.astype(np.float64))
    assert abs(J - Jo) < 1e-5 * Jo
    assert rel(g_eps.cpu().numpy(), go_eps) < 1e-4
    assert rel(s.from_device(g_u0), go_u0) < 1e-4


@pytest.mark.parametrize("N,n", [(1, 3), (2, 3), (3, 3), (4, 4), (5, 2)])
def test_adjoint_forms_agree_with_the_oracle(N, n):
    # the reverse stage with its contractions on the tensor cores (FP16x3 split
    # of D^T and LIFT^T) and on the CUDA cores both give the oracle's discrete
    # adjoint; checkpoints every 3 of 7 steps (recomputed segments, a partial
    # one, the fused and the separate lifts), partial element tiles
    steps, ck = 7, 3
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    epsd = torch.as_tensor(eps, device="cuda")
    Jo, go_eps, go_u0 = m.misfit_gradient(u0, dt, steps, recv, Eref.double().cpu().numpy(),
                                          eps=eps.astype(np.float64))
    assert s.adjoint_form() == "tensor"  # the default on a GB300 for N <= 5
    out = {}
    for form in ("tensor", "cuda"):
        s.set_adjoint_form(form)
        assert s.adjoint_form() == form
        J, g_eps, g_u0 = s.adjoint(u0d, rd, Eref, dt, steps, ck, eps=epsd)
        assert abs(J - Jo) < 1e-5 * Jo
        assert rel(g_eps.cpu().numpy(), go_eps) < 1e-4, form
        assert rel(s.from_device(g_u0), go_u0) < 1e-4, form
        out[form] = (g_eps.cpu().numpy(), s.from_device(g_u0))
    assert rel(out["tensor"][0], out["cuda"][0]) < 2e-5
    assert rel(out["tensor"][1], out["cuda"][1]) < 2e-5


@pytest.mark.parametrize("N,n", [(3, 3), (4, 3), (5, 2)])
def test_adjoint_in_split_precision_context_matches_oracle(N, n):
    # an FP16x3 context: the receiver traces and the adjoint's forward sweeps
    # run the tensor-core stage (its store form keeps the stage states and
    # right-hand sides of a segment), the reverse stage the tensor-core one;
    # checkpoints every 3 of 7 steps
    steps, ck = 7, 3
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps, precision="fp16x3")
    ref = m.receiver_traces(u0, dt, steps, recv, eps=eps_t.astype(np.float64))
    assert rel(Eref.double().cpu().numpy(), ref) < 1e-5
    epsd = torch.as_tensor(eps, device="cuda")
    J, g_eps, g_u0 = s.adjoint(u0d, rd, Eref, dt, steps, ck, eps=epsd)
    Jo, go_eps, go_u0 = m.misfit_gradient(u0, dt, steps, recv, Eref.double().cpu().numpy(),
                                          eps=eps.astype(np.float64))
    assert abs(J - Jo) < 1e-5 * Jo
    assert rel(g_eps.cpu().numpy(), go_eps) < 1e-4
    assert rel(s.from_device(g_u0), go_u0) < 1e-4


def test_adjoint_tensor_form_wait_timeout_and_recovery():
    # a wait limit of one cycle makes the tensor-core reverse stage's waits run
    # out: DG_ERR_TIMEOUT, no fault; with the default limit the same context
    # gives the undisturbed gradient again
    N, n, steps = 4, 3, 4
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    epsd = torch.as_tensor(eps, device="cuda")
    s.set_adjoint_form("tensor")
    J0, ge0, gu0 = s.adjoint(u0d, rd, Eref, dt, steps, 2, eps=epsd)
    s.set_wait_limit(1)
    with pytest.raises(dg.DGError) as ei:
        s.adjoint(u0d, rd, Eref, dt, steps, 2, eps=epsd)
    assert ei.value.code == -5
    s.set_wait_limit(0)
    J1, ge1, gu1 = s.adjoint(u0d, rd, Eref, dt, steps, 2, eps=epsd)
    assert abs(J1 - J0) <= 1e-12 * J0  # the misfit's FP64 atomic sums may reorder
    assert rel(ge1.cpu().numpy(), ge0.cpu().numpy()) < 1e-6
    assert rel(s.from_device(gu1), s.from_device(gu0)) < 1e-6


def test_receiver_misfit_autograd_function():
    # torch.autograd.Function over dg_adjoint_step: backward gives the adjoint's
    # gradients scaled by dJ (here 1), equal to the oracle's discrete adjoint;
    # a forward pass with no input requiring a gradient runs the forward sweep
    # alone and gives the same misfit
    N, n, steps, ck = 4, 6, 12, 5
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    epsd = torch.as_tensor(eps, device="cuda")
    J_ref, ge_ref, gu_ref = s.adjoint(u0d, rd, Eref, dt, steps, ck, eps=epsd)
    u_in = u0d.clone().requires_grad_(True)
    e_in = epsd.clone().requires_grad_(True)
    J = dg.ReceiverMisfit.apply(u_in, e_in, s, rd, Eref, dt, steps, ck)
    assert J.dtype == torch.float64 and abs(float(J.detach()) - J_ref) <= 1e-12 * J_ref
    (3.0 * J).backward()
    # two adjoint runs: equal up to the FP32 summation order of the reverse sweep
    assert float((u_in.grad - 3.0 * gu_ref).norm()) <= 1e-6 * float((3.0 * gu_ref).norm())
    assert float((e_in.grad.double() - 3.0 * ge_ref).norm()) <= 1e-6 * float((3.0 * ge_ref).norm())
    Jo, go_eps, go_u0 = m.misfit_gradient(u0, dt, steps, recv, Eref.double().cpu().numpy(),
                                          eps=eps.astype(np.float64))
    assert rel(e_in.grad.double().cpu().numpy() / 3.0, go_eps) < 1e-4
    assert rel(s.from_device(u_in.grad) / 3.0, go_u0) < 1e-4
    with torch.no_grad():
        J0 = dg.ReceiverMisfit.apply(u0d, epsd, s, rd, Eref, dt, steps, ck)
    assert s.adjoint_segment_steps() == 0  # no checkpoints: the forward sweep alone
    assert abs(float(J0) - J_ref) <= 1e-6 * J_ref
    J1 = dg.ReceiverMisfit.apply(u0d, epsd, s, rd, Eref, dt, steps, ck)  # inputs without requires_grad
    assert not J1.requires_grad and s.adjoint_segment_steps() == 0
    assert abs(float(J1) - Jo) < 1e-5 * Jo


def test_maxwell_solve_autograd_function():
    # traces out; backward = the vector-Jacobian product through the adjoint,
    # against the oracle's discrete adjoint of the misfit whose residuals are
    # G / 2 (E_ref = traces - G / 2), and against ReceiverMisfit for
    # L = |traces - E_ref|^2 (G = 2 (traces - E_ref))
    N, n, steps, ck = 4, 6, 12, 5
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    epsd = torch.as_tensor(eps, device="cuda")
    u_in = u0d.clone().requires_grad_(True)
    e_in = epsd.clone().requires_grad_(True)
    tr = dg.MaxwellSolve.apply(u_in, e_in, s, rd, dt, steps, ck)
    assert tr.shape == (steps, 3, rd.numel()) and tr.requires_grad
    ref = m.receiver_traces(u0, dt, steps, recv, eps=eps.astype(np.float64))
    assert rel(tr.detach().double().cpu().numpy(), ref) < 1e-5
    w = torch.as_tensor(np.random.default_rng(5).standard_normal(tuple(tr.shape)), dtype=torch.float32,
                        device="cuda") * tr.detach().abs().max()
    (w * tr).sum().backward()
    Eo = ref - 0.5 * w.double().cpu().numpy()
    _, go_eps, go_u0 = m.misfit_gradient(u0, dt, steps, recv, Eo, eps=eps.astype(np.float64))
    assert rel(e_in.grad.double().cpu().numpy(), go_eps) < 1e-4
    assert rel(s.from_device(u_in.grad), go_u0) < 1e-4
    # L = misfit: the same gradients as ReceiverMisfit
    u2 = u0d.clone().requires_grad_(True)
    e2 = epsd.clone().requires_grad_(True)
    ((dg.MaxwellSolve.apply(u2, e2, s, rd, dt, steps, ck) - Eref) ** 2).sum().backward()
    _, ge_ref, gu_ref = s.adjoint(u0d, rd, Eref, dt, steps, ck, eps=epsd)
    assert rel(e2.grad.double().cpu().numpy(), ge_ref.cpu().numpy()) < 1e-5
    assert rel(s.from_device(u2.grad), s.from_device(gu_ref)) < 1e-5


def test_adjoint_segmentations_agree():
    # 4^3 x 6 tets at N=4, 12 steps: one-step segments (everything recomputed),
    # segments of 5 aligned to the end (2 + 5 + 5, the last one stored by the
    # forward sweep), one stored segment, and the automatic choice
    N, n, steps = 4, 4, 12
    s, m, eps, eps_t, u0, u0d, recv, rd, Eref, dt = _misfit_problem(N, n, steps)
    epsd = torch.as_tensor(eps, device="cuda")
    J1, ge1, gu1 = s.adjoint(u0d, rd, Eref, dt, steps, 1, eps=epsd)
    assert s.adjoint_segment_steps() == 1
    for ck, seg in ((5, 5), (12, 12), (40, 12), (0, 12)):
        J, ge, gu = s.adjoint(u0d, rd, Eref, dt, steps, ck, eps=epsd)
        assert s.adjoint_segment_steps() == seg
        assert abs(J - J1) <= 1e-12 * J1
        assert rel(ge.cpu().numpy(), ge1.cpu().numpy()) < 1e-6
        assert rel(s.from_device(gu), s.from_device(gu1)) < 1e-6
    with pytest.raises(dg.DGError):
        s.adjoint(u0d, rd, Eref, dt, steps, -1, eps=epsd)


def test_adjoint_forms_agree_full_size():
    # the adjoint workload as the bench times it (20^3 x 6 = 48,000 tets, N=4,
    # 400 steps, checkpoints every 20, 256 receivers): the tensor-core reverse
    # stage against the CUDA-core one, for J and both gradients
    N, n, steps, ck = 4, 20, 400, 20
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=2)
    s = dg.Solver(N).upload(VX, VY, VZ, EToV, eps=eps)
    x, y, z = s.node_coords()
    u0d = s.to_device(W.gaussian_pulse(x, y, z, seed=7))
    recv = torch.as_tensor(W.receivers(K, s.Np, 256, seed=4), device="cuda")
    dt = 0.5 / n / N ** 2
    epsd = torch.as_tensor(eps, device="cuda")
    Eref = s.receiver_traces(u0d, recv, dt, steps, eps=torch.as_tensor(W.element_eps(K, seed=6), device="cuda"))
    out = {}
    for form in ("tensor", "cuda"):
        s.set_adjoint_form(form)
        J, g_eps, g_u0 = s.adjoint(u0d, recv, Eref, dt, steps, ck, eps=epsd)
        out[form] = (J, g_eps.cpu().numpy(), s.from_device(g_u0))
    assert abs(out["tensor"][0] - out["cuda"][0]) <= 1e-9 * out["cuda"][0]  # the same forward sweep
    assert rel(out["tensor"][1], out["cuda"][1]) < 1e-4
    assert rel(out["tensor"][2], out["cuda"][2]) < 1e-4


def test_adjoint_finite_differences_full_size():
    # the adjoint workload: 20^3 x 6 = 48,000 jittered tets, N=4, 400 steps,
    # checkpoints every 20, 256 receivers, E_ref from the target eps (seed 6)
    N, n, steps, ck = 4, 20, 400, 20
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=2)
    s = dg.Solver(N).upload(VX, VY, VZ, EToV, eps=eps)
    x, y, z = s.node_coords()
    u0d = s.to_device(W.gaussian_pulse(x, y, z, seed=7))
    recv = torch.as_tensor(W.receivers(K, s.Np, 256, seed=4), device="cuda")
    dt = 0.5 / n / N ** 2
    epsd = torch.as_tensor(eps, device="cuda")
    Eref = s.receiver_traces(u0d, recv, dt, steps, eps=torch.as_tensor(W.element_eps(K, seed=6), device="cuda"))
    J, g_eps, g_u0 = s.adjoint(u0d, recv, Eref, dt, steps, ck, eps=epsd)
    assert J > 0

    def misfit(e):
        tr = s.receiver_traces(u0d, recv, dt, steps, eps=e)
        return float(((tr.double() - Eref.double()) ** 2).sum())

    # central differences with step 1e-3 along unit directions; eps is FP32, so
    # the realised perturbation (e+ - e-) after rounding is what J responds to
    h = 1e-3
    # directions with entries uniform in [-1, 1] (a perturbation of up to 1e-3
    # per element); unit-norm directions would move J by ~1e-8 J, far below the
    # FP32 round-off of the forward runs
    dirs = 2.0 * W.uniform(5, 16 * K).reshape(16, K) - 1.0
    worst, rels, gaps = 0.0, [], []
    for d in dirs:
        dd = torch.as_tensor(d, dtype=torch.float64, device="cuda")
        ep = (epsd.double() + h * dd).float()
        em = (epsd.double() - h * dd).float()
        fd = misfit(ep) - misfit(em)
        ad = float((g_eps * (ep.double() - em.double())).sum())
        worst = max(worst, abs(fd - ad) / max(abs(fd), 1e-30))
        rels.append(abs(fd - ad) / abs(fd))
        gaps.append(abs(fd - ad))
        print(f"  J={J:.6e} fd={fd:.6e} adjoint={ad:.6e} rel={abs(fd - ad) / abs(fd):.2e}")
    print(f"FD vs adjoint, worst relative difference over 16 directions: {worst:.3e}")
    # Each forward run is FP32 (unit round-off 6e-8, ~2000 stages), so J+ and
    # J- carry independent round-off of order 1e-7 J; the finite difference
    # cannot resolve the derivative better than that. Bound: |fd - adjoint| <=
    # 1e-6 J in every direction, and a median relative gap below 1e-3. The
    # tight check of the adjoint itself is the FP64-oracle comparison above.
    assert max(gaps) <= 1e-6 * J, (max(gaps), J)
    assert float(np.median(rels)) < 1e-3
