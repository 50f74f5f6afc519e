"""FP64 single-threaded CPU oracle of the nodal DG Maxwell operator (ctypes front end).

TEST INFRASTRUCTURE ONLY: imported by the tests, `__graft_entry__.smoke()` and
the CPU-baseline leg of `bench.py`. The product package never imports it.

The C source (`oracle.c`) is compiled with gcc on first use (or by `build()`)
into `oracle/_build/liboracle.so`. Field arrays are float64 [6][K][Np].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_OUT_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_use_omp = False

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_ip64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (-O2, IEEE arithmetic, no host-specific flags).
    openmp=True builds the same source with OpenMP (elements of a right-hand
    side split over threads, per-element arithmetic unchanged) for long
    reference runs; the default build is single-threaded."""
    out = _OUT_OMP if openmp else _OUT
    stale = (not os.path.exists(out)) or force or any(
        os.path.getmtime(p) > os.path.getmtime(out) for p in (_SRC, _HDR))
    if stale:
        os.makedirs(os.path.dirname(out), exist_ok=True)
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared"]
                              + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


def use_openmp() -> None:
    """Load the OpenMP build instead of the single-threaded one (call before
    the first oracle call of the process; the thread count follows
    OMP_NUM_THREADS)."""
    global _use_omp
    with _lock:
        if _lib is not None and not _use_omp:
            raise RuntimeError("oracle: the single-threaded build is already loaded")
        _use_omp = True


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build(openmp=_use_omp))
            L.or_error.restype = C.c_char_p
            L.or_np.argtypes = [C.c_int]
            L.or_nfp.argtypes = [C.c_int]
            L.or_lgl.argtypes = [C.c_int, _dp]
            L.or_nodes.argtypes = [C.c_int, _dp, _dp, _dp]
            L.or_nodes_alpha.argtypes = [C.c_int, C.c_double, _dp, _dp, _dp]
            L.or_lebesgue.argtypes = [C.c_int, C.c_double, C.c_int, C.POINTER(C.c_double)]
            L.or_operators.argtypes = [C.c_int] + [C.c_void_p] * 8
            L.or_operators_alpha.argtypes = [C.c_int, C.c_double] + [C.c_void_p] * 8
            L.or_basis.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                   C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_mesh_create.restype = C.c_void_p
            L.or_mesh_create.argtypes = [C.c_int, C.c_int64, _dp, _dp, _dp, C.c_int64, _ip32,
                                         C.c_void_p, C.c_void_p]
            L.or_mesh_create_alpha.restype = C.c_void_p
            L.or_mesh_create_alpha.argtypes = [C.c_int, C.c_double, C.c_int64, _dp, _dp, _dp, C.c_int64, _ip32,
                                               C.c_void_p, C.c_void_p]
            L.or_mesh_destroy.argtypes = [C.c_void_p]
            L.or_mesh_K.argtypes = [C.c_void_p]
            L.or_mesh_K.restype = C.c_int64
            L.or_mesh_coords.argtypes = [C.c_void_p, _dp, _dp, _dp]
            L.or_mesh_geometry.argtypes = [C.c_void_p, _dp, _dp, _ip64, _ip64]
            L.or_mesh_exterior.argtypes = [C.c_void_p, _ip64]
            L.or_flux.argtypes = [_dp, _dp, _dp, C.c_double, C.c_double, C.c_double, _dp, _dp]
            L.or_rhs.argtypes = [C.c_void_p, _dp, _dp, C.c_double]
            L.or_rhs_subset.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _ip64, C.c_int64]
            L.or_lserk_coeffs.argtypes = [_dp, _dp, _dp]
            L.or_lserk.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, C.c_double]
            L.or_energy.argtypes = [C.c_void_p, _dp]
            L.or_energy.restype = C.c_double
            L.or_face_dissipation.argtypes = [C.c_void_p, _dp, C.c_double]
            L.or_face_dissipation.restype = C.c_double
            L.or_rhs_transpose.argtypes = [C.c_void_p, _dp, _dp, C.c_double]
            L.or_misfit_gradient.argtypes = [C.c_void_p, _dp, C.c_void_p, C.c_double, C.c_int,
                                             C.c_double, _ip64, C.c_int64, _dp,
                                             C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_receiver_traces.argtypes = [C.c_void_p, _dp, C.c_void_p, C.c_double, C.c_int,
                                             C.c_double, _ip64, C.c_int64, _dp]
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        raise RuntimeError("oracle: " + lib().or_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def np_count(N: int) -> int:
    return lib().or_np(N)


def nfp_count(N: int) -> int:
    return lib().or_nfp(N)


def lgl(N: int) -> np.ndarray:
    x = np.zeros(N + 1)
    _check(lib().or_lgl(N, x))
    return x


def nodes(N: int, alpha: float = 0.0):
    """Warp & blend nodes of blend parameter alpha (0: the plain construction)."""
    Np = np_count(N)
    r, s, t = np.zeros(Np), np.zeros(Np), np.zeros(Np)
    if alpha == 0.0:
        _check(lib().or_nodes(N, r, s, t))
    else:
        _check(lib().or_nodes_alpha(N, float(alpha), r, s, t))
    return r, s, t


def lebesgue(N: int, alpha: float = 0.0, M: int = 30) -> float:
    """Lebesgue constant of those nodes on the order-M equidistant lattice."""
    v = C.c_double()
    _check(lib().or_lebesgue(N, float(alpha), M, C.byref(v)))
    return v.value


def optimal_alpha(N: int) -> float:
    """Blend parameter of least Lebesgue constant, from the table written by
    oracle/optimize_node_alpha.py (0 below N = 3, where the warp vanishes or
    the nodes do not depend on it)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "node_alpha.txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                n, a = line.split()[:2]
                if int(n) == N:
                    return float(a)
    raise KeyError(f"no optimised blend parameter for N={N}")


def operators(N: int, alpha: float = 0.0) -> dict:
    Np, Nfp = np_count(N), nfp_count(N)
    out = dict(V=np.zeros((Np, Np)), Dr=np.zeros((Np, Np)), Ds=np.zeros((Np, Np)),
               Dt=np.zeros((Np, Np)), M=np.zeros((Np, Np)),
               Fmask=np.zeros((4, Nfp), dtype=np.int32), Mf=np.zeros((4, Nfp, Nfp)),
               LIFT=np.zeros((Np, 4 * Nfp)))
    _check(lib().or_operators_alpha(N, float(alpha), *[_ptr(out[k]) for k in
                                                       ("V", "Dr", "Ds", "Dt", "M", "Fmask", "Mf", "LIFT")]))
    return out


def basis(N: int, m: int, r: float, s: float, t: float):
    v, a, b, c = C.c_double(), C.c_double(), C.c_double(), C.c_double()
    _check(lib().or_basis(N, m, r, s, t, C.byref(v), C.byref(a), C.byref(b), C.byref(c)))
    return v.value, a.value, b.value, c.value


def flux(n, qm, qp, Zm=1.0, Zp=1.0, alpha=1.0):
    """n.(F - F*) at one face node: returns (flux_E, flux_H)."""
    fE, fH = np.zeros(3), np.zeros(3)
    _check(lib().or_flux(np.ascontiguousarray(n, dtype=np.float64), np.ascontiguousarray(qm, dtype=np.float64),
                         np.ascontiguousarray(qp, dtype=np.float64), float(Zm), float(Zp), float(alpha), fE, fH))
    return fE, fH


def lserk_coeffs():
    a, b, c = np.zeros(5), np.zeros(5), np.zeros(5)
    _check(lib().or_lserk_coeffs(a, b, c))
    return a, b, c


class Mesh:
    """Oracle mesh: connectivity, geometry and exterior-node map, all FP64."""

    def __init__(self, N, VX, VY, VZ, EToV, eps=None, mu=None, node_alpha: float = 0.0):
        self.N = N
        self.node_alpha = float(node_alpha)
        self.Np, self.Nfp = np_count(N), nfp_count(N)
        VX, VY, VZ = (np.ascontiguousarray(v, dtype=np.float64) for v in (VX, VY, VZ))
        EToV = np.ascontiguousarray(EToV, dtype=np.int32)
        self.K = EToV.shape[0]
        self._eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        self._mu = None if mu is None else np.ascontiguousarray(mu, dtype=np.float64)
        h = lib().or_mesh_create_alpha(N, self.node_alpha, VX.size, VX, VY, VZ, self.K, EToV,
                                       _ptr(self._eps), _ptr(self._mu))
        if not h:
            raise RuntimeError("oracle: " + lib().or_error().decode())
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_mesh_destroy(h)
            self._h = None

    @property
    def shape(self):
        return (6, self.K, self.Np)

    def coords(self):
        x, y, z = (np.zeros((self.K, self.Np)) for _ in range(3))
        _check(lib().or_mesh_coords(self._h, x, y, z))
        return x, y, z

    def geometry(self):
        G = np.zeros((self.K, 10))
        F = np.zeros((self.K, 4, 5))
        EToE = np.zeros((self.K, 4), dtype=np.int64)
        EToF = np.zeros((self.K, 4), dtype=np.int64)
        _check(lib().or_mesh_geometry(self._h, G, F, EToE, EToF))
        return G, F, EToE, EToF

    def exterior(self):
        ext = np.zeros((self.K, 4, self.Nfp), dtype=np.int64)
        _check(lib().or_mesh_exterior(self._h, ext))
        return ext

    def rhs(self, u, alpha=1.0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        out = np.zeros_like(u)
        _check(lib().or_rhs(self._h, u, out, float(alpha)))
        return out

    def rhs_subset(self, u, elems, alpha=1.0):
        u = np.ascontiguousarray(u, dtype=np.float64)
        elems = np.ascontiguousarray(elems, dtype=np.int64)
        out = np.zeros((6, elems.size, self.Np))
        _check(lib().or_rhs_subset(self._h, u, out, float(alpha), elems, elems.size))
        return out

    def rhs_transpose(self, v, alpha=1.0):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros_like(v)
        _check(lib().or_rhs_transpose(self._h, v, out, float(alpha)))
        return out

    def lserk(self, u, dt, nsteps, alpha=1.0, res=None):
        u = np.array(u, dtype=np.float64, order="C", copy=True)
        res = np.zeros_like(u) if res is None else np.array(res, dtype=np.float64, order="C", copy=True)
        _check(lib().or_lserk(self._h, u, res, float(dt), int(nsteps), float(alpha)))
        return u, res

    def energy(self, u):
        return lib().or_energy(self._h, np.ascontiguousarray(u, dtype=np.float64))

    def face_dissipation(self, u, alpha=1.0):
        return lib().or_face_dissipation(self._h, np.ascontiguousarray(u, dtype=np.float64), float(alpha))

    def receiver_traces(self, u0, dt, nsteps, recv, eps=None, alpha=1.0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        recv = np.ascontiguousarray(recv, dtype=np.int64)
        e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        out = np.zeros((nsteps, 3, recv.size))
        _check(lib().or_receiver_traces(self._h, u0, _ptr(e), float(dt), int(nsteps), float(alpha),
                                        recv, recv.size, out))
        return out

    def misfit_gradient(self, u0, dt, nsteps, recv, Eref, eps=None, alpha=1.0):
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        recv = np.ascontiguousarray(recv, dtype=np.int64)
        Eref = np.ascontiguousarray(Eref, dtype=np.float64)
        e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        J = np.zeros(1)
        g_eps = np.zeros(self.K)
        g_u0 = np.zeros_like(u0)
        _check(lib().or_misfit_gradient(self._h, u0, _ptr(e), float(dt), int(nsteps), float(alpha),
                                        recv, recv.size, Eref, _ptr(J), _ptr(g_eps), _ptr(g_u0)))
        return float(J[0]), g_eps, g_u0
