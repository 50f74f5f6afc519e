"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test checks the oracle against something other than itself: closed forms,
exact integrals, invariants of the discrete operator, hand-derived values.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- 1D / nodes
def test_lgl_closed_forms():
    # N=3: interior nodes +-1/sqrt(5); N=4: 0, +-sqrt(3/7).
    np.testing.assert_allclose(O.lgl(3), [-1, -1 / math.sqrt(5), 1 / math.sqrt(5), 1], atol=1e-15)
    np.testing.assert_allclose(O.lgl(4), [-1, -math.sqrt(3 / 7), 0, math.sqrt(3 / 7), 1], atol=1e-15)
    # N=5: roots of P5' = 0: x^2 = (7 -+ 2 sqrt(7)) / 21
    a, b = math.sqrt((7 - 2 * math.sqrt(7)) / 21), math.sqrt((7 + 2 * math.sqrt(7)) / 21)
    np.testing.assert_allclose(O.lgl(5), [-1, -b, -a, a, b, 1], atol=1e-15)


@pytest.mark.parametrize("N", [1, 2])
def test_nodes_equidistant_for_low_order(N):
    # LGL and equidistant points coincide for N <= 2, so no warp happens.
    r, s, t = O.nodes(N)
    lat = [(-1 + 2 * i / N, -1 + 2 * j / N, -1 + 2 * k / N)
           for k in range(N + 1) for j in range(N + 1 - k) for i in range(N + 1 - k - j)]
    np.testing.assert_allclose(np.stack([r, s, t], 1), np.array(lat), atol=1e-15)


def _bary(r, s, t):
    return np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], 1)


@pytest.mark.parametrize("N", [3, 4, 5, 7, 9])
def test_nodes_symmetric_and_edge_lgl(N):
    r, s, t = O.nodes(N)
    L = _bary(r, s, t)
    assert L.shape[0] == (N + 1) * (N + 2) * (N + 3) // 6
    key = lambda A: np.array(sorted(map(tuple, np.round(A, 12))))
    base = key(L)
    # invariant under all 24 vertex permutations (symmetry of warp & blend)
    for p in itertools.permutations(range(4)):
        np.testing.assert_allclose(key(L[:, p]), base, atol=1e-12)
    # nodes on an edge sit at the 1D LGL points
    x = O.lgl(N)
    on_edge = (np.abs(L[:, 2]) < 1e-12) & (np.abs(L[:, 3]) < 1e-12)
    pos = np.sort(L[on_edge, 1] - L[on_edge, 0])
    np.testing.assert_allclose(pos, x, atol=1e-13)
    # inside the simplex
    assert L.min() > -1e-13


# ---------------------------------------------------------------- blend parameter of the nodes
# The warp & blend construction with blend parameter alpha scales each face's
# edge warp by (1 + (alpha l_R)^2), l_R the barycentric of the face's third
# vertex. The table oracle/node_alpha.txt holds, per N, the alpha of least
# Lebesgue constant found by oracle/optimize_node_alpha.py.

def test_blend_parameter_zero_is_the_plain_construction():
    for N in (3, 6, 9):
        np.testing.assert_array_equal(np.stack(O.nodes(N, 1e-300)), np.stack(O.nodes(N)))


@pytest.mark.parametrize("N", [5, 6, 7, 8, 9])
def test_blended_nodes_symmetric_edge_lgl_and_moved(N):
    # the factor depends on the vertex opposite each edge within the face; any
    # other choice (an end of the edge, the tetrahedron's fourth vertex) breaks
    # the symmetry under the 24 vertex permutations checked here
    alpha = O.optimal_alpha(N)
    assert alpha > 0
    L = _bary(*O.nodes(N, alpha))
    L0 = _bary(*O.nodes(N))
    key = lambda A: np.array(sorted(map(tuple, np.round(A, 12))))
    base = key(L)
    for p in itertools.permutations(range(4)):
        np.testing.assert_allclose(key(L[:, p]), base, atol=1e-12)
    # edge nodes stay at the 1D LGL points (l_R = 0 on an edge), others move
    on_edge = (np.sort(L, axis=1)[:, :2] < 1e-12).all(axis=1)
    np.testing.assert_allclose(L[on_edge], L0[on_edge], atol=1e-14)
    assert np.abs(L[~on_edge] - L0[~on_edge]).max() > 1e-3
    assert L.min() > -1e-13


@pytest.mark.parametrize("N", [6, 9])
def test_blended_nodes_give_exact_operators(N):
    alpha = O.optimal_alpha(N)
    ops = O.operators(N, alpha)
    r, s, t = O.nodes(N, alpha)
    err = 0.0
    for a, b, c in [(N, 0, 0), (0, N, 0), (0, 0, N), (1, 2, N - 3), (2, 2, N - 4), (N - 1, 1, 0)]:
        f = r ** a * s ** b * t ** c
        for D, g in ((ops["Dr"], a * r ** max(a - 1, 0) * s ** b * t ** c),
                     (ops["Ds"], b * r ** a * s ** max(b - 1, 0) * t ** c),
                     (ops["Dt"], c * r ** a * s ** b * t ** max(c - 1, 0))):
            err = max(err, np.abs(D @ f - g).max())
    assert err < 1e-11 * N ** 2
    L = _bary(r, s, t)
    f, g = L[:, 1] ** N, L[:, 2] ** N
    assert abs(f @ ops["M"] @ g - _dirichlet((0, N, N, 0), 3)) < 1e-12


def _lebesgue_monomial(N, alpha, M):
    """Lebesgue constant on the order-M lattice with the Lagrange basis built
    from monomials r^a s^b t^c (not the oracle's orthonormal basis)."""
    r, s, t = O.nodes(N, alpha)
    pw = [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]
    mono = lambda x, y, z: np.stack([x ** a * y ** b * z ** c for a, b, c in pw], axis=1)
    lat = np.array([(-1 + 2 * i / M, -1 + 2 * j / M, -1 + 2 * k / M)
                    for k in range(M + 1) for j in range(M + 1 - k) for i in range(M + 1 - k - j)])
    ell = mono(*lat.T) @ np.linalg.inv(mono(r, s, t))
    return np.abs(ell).sum(axis=1).max()


def test_lebesgue_constant_closed_form_and_independent_basis():
    # N = 1: the barycentric basis is non-negative and sums to 1
    assert abs(O.lebesgue(1, 0.0, 12) - 1.0) < 1e-13
    for N, alpha in [(3, 0.0), (4, 0.7), (5, O.optimal_alpha(5))]:
        assert abs(O.lebesgue(N, alpha, 16) - _lebesgue_monomial(N, alpha, 16)) < 1e-9


def test_optimised_blend_parameter_lowers_the_lebesgue_constant():
    rows = [l.split() for l in open(os.path.join(os.path.dirname(O.__file__), "node_alpha.txt"))
            if l.strip() and not l.startswith("#")]
    assert [int(r[0]) for r in rows] == list(range(1, 10))
    for N in range(5, 10):
        a = O.optimal_alpha(N)
        # on a lattice the search did not use
        assert O.lebesgue(N, a, 45) < O.lebesgue(N, 0.0, 45)
    # N = 3: the one face-interior node is the face centroid for every alpha
    assert O.lebesgue(3, 1.3, 30) == pytest.approx(O.lebesgue(3, 0.0, 30), abs=1e-13)


# ---------------------------------------------------------------- operators
def _dirichlet(powers, dim):
    """Integral of prod(lambda_i^a_i) over the reference simplex (|T| = 4/3 or 2)."""
    vol = 4.0 / 3.0 if dim == 3 else 2.0
    num = math.prod(math.factorial(a) for a in powers) * math.factorial(dim)
    return num / math.factorial(sum(powers) + dim) * vol


@pytest.mark.parametrize("N", [1, 3, 5, 7, 9])
def test_derivative_exact_on_monomials(N):
    ops = O.operators(N)
    r, s, t = O.nodes(N)
    err = 0.0
    for a in range(N + 1):
        for b in range(N + 1 - a):
            for c in range(N + 1 - a - b):
                f = r ** a * s ** b * t ** c
                fr = a * r ** max(a - 1, 0) * s ** b * t ** c
                fs = b * r ** a * s ** max(b - 1, 0) * t ** c
                ft = c * r ** a * s ** b * t ** max(c - 1, 0)
                for D, g in ((ops["Dr"], fr), (ops["Ds"], fs), (ops["Dt"], ft)):
                    err = max(err, np.abs(D @ f - g).max())
    assert err < 1e-11 * max(1, N ** 2)


@pytest.mark.parametrize("N", [2, 4, 7, 9])
def test_mass_matrix_integrates_exactly(N):
    ops = O.operators(N)
    L = _bary(*O.nodes(N))
    one = np.ones(L.shape[0])
    cands = [(0, 0, 0, 0), (1, 0, 0, 0), (2, 1, 0, 1), (N, 0, 0, 0), (0, 1, 1, max(N - 2, 0)), (1, 1, 1, N - 3)]
    for powers in [p for p in cands if min(p) >= 0 and sum(p) <= N]:
        f = np.prod(L ** np.array(powers), axis=1)
        assert abs(one @ ops["M"] @ f - _dirichlet(powers, 3)) < 1e-13
    # product of two degree-N polynomials is still integrated exactly
    f = L[:, 1] ** N
    g = L[:, 2] ** N
    assert abs(f @ ops["M"] @ g - _dirichlet((0, N, N, 0), 3)) < 1e-12


@pytest.mark.parametrize("N", [2, 5])
def test_face_mass_and_lift(N):
    ops = O.operators(N)
    L = _bary(*O.nodes(N))
    Nfp = (N + 1) * (N + 2) // 2
    zero_bary = [3, 2, 0, 1]  # face 0: t=-1 (lambda_d=0), 1: s=-1, 2: r+s+t=-1 (lambda_a=0), 3: r=-1
    for f in range(4):
        idx = ops["Fmask"][f]
        assert np.abs(L[idx, zero_bary[f]]).max() < 1e-12
        Lf = np.delete(L[idx], zero_bary[f], axis=1)
        for powers in [p for p in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (N, 0, 0), (1, 1, N - 2)] if min(p) >= 0 and sum(p) <= N]:
            g = np.prod(Lf ** np.array(powers), axis=1)
            assert abs(np.ones(Nfp) @ ops["Mf"][f] @ g - _dirichlet(powers, 2)) < 1e-13
    # LIFT: 1^T M LIFT g = sum_f 1^T Mf g_f for arbitrary face data g
    rng = np.random.default_rng(3)
    g = rng.standard_normal(4 * Nfp)
    lhs = np.ones(L.shape[0]) @ ops["M"] @ ops["LIFT"] @ g
    rhs = sum(np.ones(Nfp) @ ops["Mf"][f] @ g[f * Nfp:(f + 1) * Nfp] for f in range(4))
    assert abs(lhs - rhs) < 1e-12


# ---------------------------------------------------------------- mesh / geometry
@pytest.fixture(scope="module")
def jittered():
    N = 3
    VX, VY, VZ, EToV = W.kuhn_cube(3, jitter=0.1, seed=1)
    eps = W.element_eps(EToV.shape[0], seed=2).astype(np.float64)
    return N, O.Mesh(N, VX, VY, VZ, EToV, eps=eps), eps, (VX, VY, VZ, EToV)


def test_connectivity_and_geometry(jittered):
    N, m, _, (VX, VY, VZ, EToV) = jittered
    x, y, z = m.coords()
    G, F, EToE, EToF = m.geometry()
    ext = m.exterior()
    Fm = O.operators(N)["Fmask"]
    # total volume of the unit cube, positive Jacobians
    assert G[:, 9].min() > 0
    assert abs((G[:, 9] * 4.0 / 3.0).sum() - 1.0) < 1e-13
    # boundary faces: exactly 2 * 6 * n^2 triangles on the cube walls
    assert (EToE < 0).sum() == 12 * 9
    X = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    for k in range(m.K):
        # sum of sJ_f n_f vanishes (closed polyhedron), normals outward
        assert np.abs((F[k, :, 3:4] * F[k, :, :3]).sum(0)).max() < 1e-14
        for f in range(4):
            k2, f2 = EToE[k, f], EToF[k, f]
            idx = k * m.Np + Fm[f]
            if k2 < 0:
                continue
            # neighbour of neighbour is the identity, normals opposite, areas equal
            assert EToE[k2, f2] == k and EToF[k2, f2] == f
            np.testing.assert_allclose(F[k2, f2, :3], -F[k, f, :3], atol=1e-14)
            assert abs(F[k2, f2, 3] - F[k, f, 3]) < 1e-15
            # exterior nodes coincide with interior nodes
            assert np.abs(X[ext[k, f]] - X[idx]).max() < 1e-14
    # face area from Heron's formula on the raw vertices
    for k in (0, 7, m.K - 1):
        for f, vs in enumerate([(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]):
            P = np.array([[VX[EToV[k, v]], VY[EToV[k, v]], VZ[EToV[k, v]]] for v in vs])
            a, b, c = (np.linalg.norm(P[i] - P[j]) for i, j in ((0, 1), (1, 2), (2, 0)))
            sp = (a + b + c) / 2
            area = math.sqrt(sp * (sp - a) * (sp - b) * (sp - c))
            assert abs(F[k, f, 3] * 2.0 - area) < 1e-14


def test_divergence_theorem_per_element(jittered):
    # int_D div w = sum_f int_f n.w for polynomial w: ties D, metric terms,
    # normals, sJ and the face mass matrices together.
    N, m, _, _ = jittered
    ops = O.operators(N)
    x, y, z = m.coords()
    G, F, _, _ = m.geometry()
    Np, Nfp = m.Np, m.Nfp
    for k in range(0, m.K, 17):
        wx = x[k] ** 2 * y[k] + z[k]
        wy = y[k] * z[k] ** 2
        wz = x[k] * y[k] * z[k]
        rx, ry, rz, sx, sy, sz, tx, ty, tz, J = G[k]
        Dx = rx * ops["Dr"] + sx * ops["Ds"] + tx * ops["Dt"]
        Dy = ry * ops["Dr"] + sy * ops["Ds"] + ty * ops["Dt"]
        Dz = rz * ops["Dr"] + sz * ops["Ds"] + tz * ops["Dt"]
        vol = J * np.ones(Np) @ ops["M"] @ (Dx @ wx + Dy @ wy + Dz @ wz)
        surf = 0.0
        for f in range(4):
            idx = ops["Fmask"][f]
            nw = F[k, f, 0] * wx[idx] + F[k, f, 1] * wy[idx] + F[k, f, 2] * wz[idx]
            surf += F[k, f, 3] * np.ones(Nfp) @ ops["Mf"][f] @ nw
        assert abs(vol - surf) < 1e-13


# ---------------------------------------------------------------- flux / RHS
def test_flux_golden():
    rows = np.loadtxt(os.path.join(GOLDEN, "maxwell_flux.txt"))
    for row in rows:
        n, qm, qp = row[0:3], row[3:9], row[9:15]
        Zm, Zp, alpha = row[15:18]
        fE, fH = O.flux(n, qm, qp, Zm, Zp, alpha)
        np.testing.assert_allclose(fE, row[18:21], atol=1e-15)
        np.testing.assert_allclose(fH, row[21:24], atol=1e-15)


def test_rhs_exact_curl_on_polynomials():
    # For a globally polynomial field of degree <= N, jumps vanish on interior
    # faces and the RHS is the exact (curl H, -curl E) on interior elements.
    N = 3
    VX, VY, VZ, EToV = W.kuhn_cube(3, jitter=0.1, seed=1)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    x, y, z = m.coords()
    u = np.stack([y * z, x * x * z, x * y * y, y ** 3, x * z, z * z * x])
    # H = (y^3, x z, x z^2): curl H = (dHz/dy - dHy/dz, dHx/dz - dHz/dx, dHy/dx - dHx/dy)
    curlH = np.stack([0 - x, 0 - z * z, z - 3 * y * y])
    # E = (y z, x^2 z, x y^2): curl E = (2 x y - x^2, y - y^2, 2 x z - z)
    curlE = np.stack([2 * x * y - x * x, y - y * y, 2 * x * z - z])
    A = m.rhs(u, 1.0)
    _, _, EToE, _ = m.geometry()
    interior = np.all(EToE >= 0, axis=1)
    assert interior.sum() > 0
    np.testing.assert_allclose(A[:3][:, interior], curlH[:, interior], atol=1e-11)
    np.testing.assert_allclose(A[3:][:, interior], -curlE[:, interior], atol=1e-11)


@pytest.mark.parametrize("alpha", [0.0, 1.0, 0.5])
def test_energy_identity(jittered, alpha):
    # d/dt E_h = u^T M_eps A u: zero for central flux, minus the closed-form
    # face dissipation (<= 0) for upwinding, with material jumps and PEC walls.
    N, m, eps, _ = jittered
    ops = O.operators(N)
    G, _, _, _ = m.geometry()
    rng = np.random.default_rng(0)
    q = rng.standard_normal(m.shape)
    A = m.rhs(q, alpha)
    rate = 0.0
    for c in range(6):
        w = G[:, 9] * (eps if c < 3 else 1.0)
        rate += np.einsum("k,ki,ij,kj->", w, q[c], ops["M"], A[c])
    diss = m.face_dissipation(q, alpha)
    E = m.energy(q)
    assert diss >= 0
    if alpha == 0.0:
        assert abs(rate) < 1e-13 * E * 100
    else:
        assert abs(rate + diss) < 1e-12 * diss
        assert diss > 1.0


# ---------------------------------------------------------------- time stepping
def _butcher():
    a, b, _ = O.lserk_coeffs()
    s = 5
    A = np.zeros((s, s))
    # stage input u_{i} = u0 + dt sum_j A[i, j] k_j, r_i = sum_j (prod a) dt k_j
    for i in range(1, s):
        for j in range(i):
            acc = 0.0
            for q in range(j, i):
                acc += b[q] * np.prod(a[j + 1:q + 1])
            A[i, j] = acc
    B = np.array([sum(b[q] * np.prod(a[j + 1:q + 1]) for q in range(j, s)) for j in range(s)])
    return A, B


def test_lserk_order_conditions():
    A, B = _butcher()
    _, _, c_given = O.lserk_coeffs()
    c = A.sum(1)
    np.testing.assert_allclose(c, c_given, atol=1e-12)
    conds = [
        (B.sum(), 1.0), (B @ c, 1 / 2), (B @ c ** 2, 1 / 3), (B @ A @ c, 1 / 6),
        (B @ c ** 3, 1 / 4), (B @ (c * (A @ c)), 1 / 8), (B @ A @ c ** 2, 1 / 12), (B @ A @ A @ c, 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-12


def test_lserk_temporal_order_on_the_semidiscrete_system():
    # Build the small operator matrix column by column and compare the oracle's
    # LSERK4 run against the exact matrix exponential: error ~ dt^4.
    scipy_linalg = pytest.importorskip("scipy.linalg")
    N = 1
    VX, VY, VZ, EToV = W.kuhn_cube(1)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    n = 6 * m.K * m.Np
    Amat = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Amat[:, j] = m.rhs(e.reshape(m.shape)).ravel()
    rng = np.random.default_rng(5)
    u0 = rng.standard_normal(n)
    T = 0.4
    exact = scipy_linalg.expm(T * Amat) @ u0
    errs = []
    for steps in (10, 20, 40):
        u, _ = m.lserk(u0.reshape(m.shape), T / steps, steps)
        errs.append(np.linalg.norm(u.ravel() - exact))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 3.7, rates


# ---------------------------------------------------------------- cavity
def _cavity_error(N, n, T=0.1):
    VX, VY, VZ, EToV = W.kuhn_cube(n)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    x, y, z = m.coords()
    u0 = W.cavity_mode(x, y, z, 0.0)
    steps = int(np.ceil(T / (0.25 / n / N ** 2)))
    u, _ = m.lserk(u0, T / steps, steps)
    e = u - W.cavity_mode(x, y, z, T)
    G, _, _, _ = m.geometry()
    M = O.operators(N)["M"]
    return math.sqrt(sum(np.einsum("k,ki,ij,kj->", G[:, 9], e[c], M, e[c]) for c in range(6)))


def test_cavity_convergence_rate():
    # Closed-form PEC cavity eigenmode: error decays like h^(N+1) with upwind flux.
    N = 2
    e1, e2 = _cavity_error(N, 3), _cavity_error(N, 6)
    rate = math.log2(e1 / e2)
    assert rate > N + 0.6, rate


def test_cavity_energy_monotone():
    N = 3
    VX, VY, VZ, EToV = W.kuhn_cube(2, jitter=0.1)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    x, y, z = m.coords()
    u = W.cavity_mode(x, y, z, 0.0)
    res = np.zeros_like(u)
    E = [m.energy(u)]
    dt = 0.5 * 0.5 / N ** 2
    for _ in range(10):
        u, res = m.lserk(u, dt, 1, res=res)
        E.append(m.energy(u))
    assert all(E[i + 1] <= E[i] * (1 + 1e-12) for i in range(10))
    # central flux: fully discrete energy never grows (normal operator, |R| <= 1)
    u = W.cavity_mode(x, y, z, 0.0)
    res = np.zeros_like(u)
    E0 = m.energy(u)
    u, res = m.lserk(u, dt, 10, alpha=0.0)
    assert m.energy(u) <= E0 * (1 + 1e-13)
    assert m.energy(u) > E0 * (1 - 1e-4)


# ---------------------------------------------------------------- adjoint
def test_transpose_dot_product(jittered):
    N, m, _, _ = jittered
    rng = np.random.default_rng(7)
    for alpha in (0.0, 1.0):
        u = rng.standard_normal(m.shape)
        v = rng.standard_normal(m.shape)
        lhs = np.vdot(m.rhs(u, alpha), v)
        rhs = np.vdot(u, m.rhs_transpose(v, alpha))
        assert abs(lhs - rhs) < 1e-12 * abs(lhs) + 1e-9


def test_misfit_gradient_finite_differences():
    N = 2
    VX, VY, VZ, EToV = W.kuhn_cube(2, jitter=0.1)
    K = EToV.shape[0]
    eps = W.element_eps(K, 2).astype(np.float64)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps)
    x, y, z = m.coords()
    u0 = 0.01 * W.gaussian_pulse(x, y, z)
    recv = W.receivers(K, m.Np, 16, 4)
    steps, dt = 6, 0.01
    Eref = m.receiver_traces(u0, dt, steps, recv, eps=W.element_eps(K, 6).astype(np.float64))
    J, ge, gu = m.misfit_gradient(u0, dt, steps, recv, Eref, eps=eps)
    h = 1e-4
    for d in W.directions(2, K, 5):
        Jp, _, _ = m.misfit_gradient(u0, dt, steps, recv, Eref, eps=eps + h * d)
        Jm, _, _ = m.misfit_gradient(u0, dt, steps, recv, Eref, eps=eps - h * d)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - ge @ d) < 1e-6 * abs(fd) + 1e-14
    du = W.directions(1, u0.size, 5)[0].reshape(u0.shape)
    Jp, _, _ = m.misfit_gradient(u0 + h * du, dt, steps, recv, Eref, eps=eps)
    Jm, _, _ = m.misfit_gradient(u0 - h * du, dt, steps, recv, Eref, eps=eps)
    fd = (Jp - Jm) / (2 * h)
    assert abs(fd - np.vdot(gu, du)) < 1e-6 * abs(fd)


# ---------------------------------------------------------------- energy (closed forms)
def _tet_volumes(VX, VY, VZ, EToV):
    P = np.stack([VX, VY, VZ], 1)[EToV]
    return np.abs(np.linalg.det(P[:, 1:] - P[:, :1])) / 6.0


def _gauss_tet(q):
    """Collapsed (Duffy) Gauss-Legendre rule on the unit simplex
    {a, b, c >= 0, a + b + c <= 1}: exact for polynomials of degree <= 2q - 3."""
    x, w = np.polynomial.legendre.leggauss(q)
    x, w = (x + 1) / 2, w / 2
    xi, eta, zeta = np.meshgrid(x, x, x, indexing="ij")
    wt = w[:, None, None] * w[None, :, None] * w[None, None, :] * (1 - xi) ** 2 * (1 - eta)
    return xi.ravel(), ((1 - xi) * eta).ravel(), ((1 - xi) * (1 - eta) * zeta).ravel(), wt.ravel()


def _materials(K):
    eps = W.element_eps(K, seed=2).astype(np.float64)
    mu = W.element_eps(K, seed=9, lo=0.5, hi=3.0).astype(np.float64)
    return eps, mu


def test_energy_piecewise_constant_fields_closed_form():
    # A field constant on each element: E_h = 1/2 sum_k |T_k| (eps_k |E_k|^2 + mu_k |H_k|^2),
    # with |T_k| from the raw vertices. Fails if J_k is dropped, eps and mu are
    # swapped, or either weights the wrong rows.
    N = 3
    VX, VY, VZ, EToV = W.kuhn_cube(3, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps, mu = _materials(K)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps, mu=mu)
    amp = 2.0 * W.uniform(11, 6 * K).reshape(6, K) - 1.0
    u = np.repeat(amp[:, :, None], m.Np, axis=2)
    vol = _tet_volumes(VX, VY, VZ, EToV)
    want = 0.5 * np.sum(vol * (eps * (amp[:3] ** 2).sum(0) + mu * (amp[3:] ** 2).sum(0)))
    assert abs(m.energy(u) - want) < 1e-13 * want


@pytest.mark.parametrize("N", [3, 4])
def test_energy_polynomial_field_exact_integral(N):
    # For a global polynomial field of degree <= N the nodal interpolant is
    # exact and M integrates the squares exactly: E_h equals the integral of
    # 1/2 (eps |E|^2 + mu |H|^2) over the mesh, here by an independent Gauss rule.
    VX, VY, VZ, EToV = W.kuhn_cube(2, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps, mu = _materials(K)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps, mu=mu)

    def fields(x, y, z):
        return np.stack([1 + x * y, z * z - x, x * y * z, y - z * z, x * x * z, 0.5 + y ** 3])

    x, y, z = m.coords()
    u = fields(x, y, z)
    a, b, c, wq = _gauss_tet(N + 3)
    P = np.stack([VX, VY, VZ], 1)[EToV]
    want = 0.0
    for k in range(K):
        v0, e1, e2, e3 = P[k, 0], P[k, 1] - P[k, 0], P[k, 2] - P[k, 0], P[k, 3] - P[k, 0]
        X = v0[:, None] + e1[:, None] * a + e2[:, None] * b + e3[:, None] * c
        f = fields(X[0], X[1], X[2])
        dens = eps[k] * (f[:3] ** 2).sum(0) + mu[k] * (f[3:] ** 2).sum(0)
        want += 0.5 * abs(np.linalg.det(np.stack([e1, e2, e3]))) * (wq @ dens)
    assert abs(m.energy(u) - want) < 1e-12 * want


# ---------------------------------------------------------------- receiver traces
@pytest.fixture(scope="module")
def small_run():
    N = 2
    VX, VY, VZ, EToV = W.kuhn_cube(2, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=2).astype(np.float64)
    m = O.Mesh(N, VX, VY, VZ, EToV, eps=eps)
    x, y, z = m.coords()
    u0 = W.gaussian_pulse(x, y, z)
    recv = W.receivers(K, m.Np, 16, 4)
    return m, eps, u0, recv, 0.01, 5


def test_receiver_traces_sampled_at_the_end_of_each_step(small_run):
    # traces[n] is E at the receivers after n + 1 full LSERK4 steps (not at
    # stages, not before the step); checked against the pinned stepper.
    m, eps, u0, recv, dt, steps = small_run
    tr = m.receiver_traces(u0, dt, steps, recv, eps=eps)
    assert tr.shape == (steps, 3, recv.size)
    for n in range(steps):
        u, _ = m.lserk(u0, dt, n + 1)
        np.testing.assert_allclose(tr[n], u[:3].reshape(3, -1)[:, recv], rtol=1e-14, atol=1e-15)
    # one step fewer or more would be a different state
    u_early, _ = m.lserk(u0, dt, 1)
    assert np.abs(tr[1] - u_early[:3].reshape(3, -1)[:, recv]).max() > 1e-6


def test_misfit_of_own_traces_is_zero_and_sums_squares(small_run):
    # J(eps; Eref = traces(eps)) = 0 exactly (same run, same sampling instants);
    # a known offset d of the reference gives J = sum d^2 (no factor 1/2).
    m, eps, u0, recv, dt, steps = small_run
    tr = m.receiver_traces(u0, dt, steps, recv, eps=eps)
    J, _, _ = m.misfit_gradient(u0, dt, steps, recv, tr, eps=eps)
    assert J == 0.0
    d = 1e-3 * (2.0 * W.uniform(12, tr.size).reshape(tr.shape) - 1.0)
    J2, _, _ = m.misfit_gradient(u0, dt, steps, recv, tr + d, eps=eps)
    assert abs(J2 - np.sum(d * d)) < 1e-12 * np.sum(d * d)


# ---------------------------------------------------------------- time-step size
def _stability_polynomial():
    """Coefficients of R(z) = sum_j g_j z^j of the LSERK4 scheme, g_j = B A^(j-1) 1."""
    A, B = _butcher()
    return [1.0] + [B @ np.linalg.matrix_power(A, j - 1) @ np.ones(5) for j in range(1, 6)]


def _extreme_eigenvalues(m, alpha):
    sla = pytest.importorskip("scipy.sparse.linalg")
    n = 6 * m.K * m.Np

    def mv(x):
        x = np.asarray(x)
        if np.iscomplexobj(x):
            return (m.rhs(np.ascontiguousarray(x.real).reshape(m.shape), alpha).ravel()
                    + 1j * m.rhs(np.ascontiguousarray(x.imag).reshape(m.shape), alpha).ravel())
        return m.rhs(np.ascontiguousarray(x).reshape(m.shape), alpha).ravel()

    op = sla.LinearOperator((n, n), matvec=mv, dtype=np.float64)
    out = []
    for which in ("LM", "LI"):  # largest modulus, largest imaginary part
        out.append(sla.eigs(op, k=4, which=which, return_eigenvectors=False, tol=1e-6, maxiter=20000,
                            v0=np.ones(n)))
    return np.concatenate(out)


def test_cfl_half_inside_the_lserk4_stability_region():
    # dt = CFL h / N^2 with CFL = 0.5 on the unit-cube mesh with 4^3 hexahedra, N = 3:
    # the extreme eigenvalues of the semi-discrete operator, scaled by dt, lie
    # inside |R(z)| <= 1 with margin. Central flux (imaginary spectrum):
    # dt rho <= 0.8 x the imaginary-axis limit of R. Upwind flux (largest
    # eigenvalues on the negative real axis): |R(dt lambda)| <= 0.5 and
    # dt rho <= 0.8 x the real-axis limit.
    g = _stability_polynomial()
    # the scheme is fourth order: R agrees with exp(z) through z^4
    np.testing.assert_allclose(g[:5], [1 / math.factorial(j) for j in range(5)], atol=1e-12)
    R = lambda z: sum(g[j] * z ** j for j in range(6))
    ys = np.linspace(0.0, 6.0, 60001)
    y_lim = ys[np.argmax(np.abs(R(1j * ys)) > 1 + 1e-13) - 1]
    xs = np.linspace(0.0, -8.0, 80001)
    x_lim = -xs[np.argmax(np.abs(R(xs)) > 1 + 1e-13) - 1]
    assert 3.3 < y_lim < 3.4 and 4.6 < x_lim < 4.7
    N, n = 3, 4
    VX, VY, VZ, EToV = W.kuhn_cube(n)
    m = O.Mesh(N, VX, VY, VZ, EToV)
    dt = 0.5 * (1.0 / n) / N ** 2
    lc = _extreme_eigenvalues(m, 0.0)
    assert np.abs(lc.real).max() < 1e-6 * np.abs(lc).max()  # central: skew in the M_eps inner product
    assert dt * np.abs(lc).max() <= 0.8 * y_lim
    lu = _extreme_eigenvalues(m, 1.0)
    assert lu.real.max() < 1e-8
    assert np.abs(R(dt * lu)).max() <= 0.5
    assert dt * np.abs(lu).max() <= 0.8 * x_lim
