"""Python binding of libdgmx (nodal DG for 3D Maxwell on GB300).

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI declared in include/dgmx.h. PyTorch supplies device
memory and streams. There is no CPU fallback: if the library cannot be built
or loaded, the import of `lib()` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libdgmx.so")
_lock = threading.Lock()
_lib = None

DG_OK = 0
STATUS = {0: "DG_OK", -1: "DG_ERR_ARG", -2: "DG_ERR_MESH", -3: "DG_ERR_CUDA", -4: "DG_ERR_NONFINITE",
          -5: "DG_ERR_TIMEOUT", -6: "DG_ERR_UNSUPPORTED", -7: "DG_ERR_OOM"}
PRECISION = {"fp32": 0, "bf16x3": 1, "fp16x3": 2, "fp32_tc": 3}


class DGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load libdgmx.so (building it with nvcc if it is not there yet)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                from . import build as _build
                _build.build()
            L = C.CDLL(_LIB_PATH)
            vp, i64, i32, dbl, flt = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_float
            L.dg_create.argtypes = [C.POINTER(vp), i32, i32, vp]
            L.dg_destroy.argtypes = [vp]
            L.dg_last_error.argtypes = [vp]
            L.dg_last_error.restype = C.c_char_p
            L.dg_mesh_upload.argtypes = [vp, i64, vp, vp, vp, i64, vp, vp, vp, vp]
            L.dg_layout.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)]
            L.dg_operators.argtypes = [vp] + [vp] * 9
            L.dg_set_node_alpha.argtypes = [vp, dbl]
            L.dg_optimised_node_alpha.argtypes = [i32]
            L.dg_optimised_node_alpha.restype = dbl
            L.dg_node_coords.argtypes = [vp, vp]
            L.dg_set_eps.argtypes = [vp, vp]
            L.dg_rhs.argtypes = [vp, vp, vp, flt]
            L.dg_step.argtypes = [vp, vp, vp, dbl, i32, flt]
            L.dg_energy.argtypes = [vp, vp, C.POINTER(dbl)]
            L.dg_sync.argtypes = [vp]
            L.dg_set_wait_limit.argtypes = [vp, C.c_longlong]
            L.dg_step_noalloc.argtypes = [vp, vp, vp, dbl, i32, flt]
            L.dg_set_nonfinite_check.argtypes = [vp, i32]
            L.dg_rhs_transpose.argtypes = [vp, vp, vp, flt]
            L.dg_ensemble_upload.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp]
            L.dg_ensemble_layout.argtypes = [vp, C.POINTER(i32), vp]
            L.dg_ensemble_step.argtypes = [vp, vp, vp, i32, flt]
            L.dg_ensemble_tune.argtypes = [vp, i32]
            L.dg_ensemble_tuning.argtypes = [vp, C.POINTER(i32), vp, vp]
            L.dg_ensemble_tuning_grid.argtypes = [vp, C.POINTER(i32), vp, vp, vp]
            L.dg_ensemble_graph_used.argtypes = [vp]
            L.dg_receiver_traces.argtypes = [vp, vp, vp, dbl, i32, flt, vp, i64, vp]
            L.dg_adjoint_step.argtypes = [vp, vp, vp, dbl, i32, i32, flt, vp, i64, vp, C.POINTER(dbl), vp, vp]
            L.dg_adjoint_segment_steps.argtypes = [vp]
            L.dg_set_adjoint_form.argtypes = [vp, i32]
            L.dg_adjoint_form.argtypes = [vp]
            _lib = L
    return _lib


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _t_ptr(t):
    return C.c_void_p(t.data_ptr())


def optimised_node_alpha(N: int) -> float:
    """Blend parameter of least Lebesgue constant for order N (the library's table)."""
    a = lib().dg_optimised_node_alpha(N)
    if a < 0:
        raise ValueError(f"no blend parameter for N={N}")
    return a


class Solver:
    """One mesh, one polynomial order, one arithmetic, one CUDA stream."""

    def __init__(self, N: int, precision: str = "fp32", stream=None, node_alpha=0.0):
        """node_alpha: blend parameter of the warp & blend nodes, a number in
        [0, 10] or "optimised" (the built-in value of least Lebesgue constant
        for N); 0 is the plain construction."""
        import torch
        self.N = N
        self.precision = precision
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self._stream = stream
        handle = C.c_void_p()
        sp = None if stream is None else C.c_void_p(stream.cuda_stream)
        rc = lib().dg_create(C.byref(handle), N, PRECISION[precision], sp)
        if rc != DG_OK:
            raise DGError(rc, lib().dg_last_error(None).decode())
        self._h = handle
        self.K = 0
        if isinstance(node_alpha, str):
            if node_alpha != "optimised":
                raise ValueError(f"unknown node_alpha {node_alpha!r}")
            node_alpha = optimised_node_alpha(N)
        self.node_alpha = float(node_alpha)
        if self.node_alpha != 0.0:
            self._check(lib().dg_set_node_alpha(self._h, self.node_alpha))
        Np, Npad, K = C.c_int(), C.c_int(), C.c_int64()
        lib().dg_layout(self._h, C.byref(Np), C.byref(Npad), C.byref(K))
        self.Np, self.Npad = Np.value, Npad.value
        self.Nfp = (N + 1) * (N + 2) // 2

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().dg_destroy(h)
            self._h = None

    def _check(self, rc: int):
        if rc != DG_OK:
            raise DGError(rc, lib().dg_last_error(self._h).decode())

    # ---------------------------------------------------------------- setup
    def upload(self, VX, VY, VZ, EToV, eps=None, mu=None, bc=None):
        VX, VY, VZ = (np.ascontiguousarray(v, dtype=np.float64) for v in (VX, VY, VZ))
        EToV = np.ascontiguousarray(EToV, dtype=np.int32)
        eps = None if eps is None else np.ascontiguousarray(eps, dtype=np.float32)
        mu = None if mu is None else np.ascontiguousarray(mu, dtype=np.float32)
        bc = None if bc is None else np.ascontiguousarray(bc, dtype=np.int32)
        K = EToV.shape[0]
        self._check(lib().dg_mesh_upload(self._h, VX.size, _np_ptr(VX), _np_ptr(VY), _np_ptr(VZ), K,
                                         _np_ptr(EToV), _np_ptr(eps), _np_ptr(mu), _np_ptr(bc)))
        self.K = K
        return self

    def operators(self) -> dict:
        Np, Nfp = self.Np, self.Nfp
        out = dict(r=np.zeros(Np), s=np.zeros(Np), t=np.zeros(Np), Dr=np.zeros((Np, Np)),
                   Ds=np.zeros((Np, Np)), Dt=np.zeros((Np, Np)), M=np.zeros((Np, Np)),
                   LIFT=np.zeros((Np, 4 * Nfp)), Fmask=np.zeros((4, Nfp), dtype=np.int32))
        self._check(lib().dg_operators(self._h, *[_np_ptr(out[k]) for k in
                                                  ("r", "s", "t", "Dr", "Ds", "Dt", "M", "LIFT", "Fmask")]))
        return out

    def node_coords(self):
        xyz = np.zeros((3, self.K, self.Np))
        self._check(lib().dg_node_coords(self._h, _np_ptr(xyz)))
        return xyz[0], xyz[1], xyz[2]

    def set_eps(self, eps_dev):
        self._check(lib().dg_set_eps(self._h, _t_ptr(eps_dev)))

    # ---------------------------------------------------------------- fields
    def zeros(self, device="cuda"):
        import torch
        return torch.zeros((6, self.K, self.Npad), dtype=torch.float32, device=device)

    def to_device(self, u, device="cuda"):
        """[6][K][Np] array -> padded FP32 device tensor [6][K][Npad]."""
        import torch
        out = torch.zeros((6, self.K, self.Npad), dtype=torch.float32)
        out[:, :, :self.Np] = torch.as_tensor(np.asarray(u), dtype=torch.float32)
        return out.to(device)

    def from_device(self, t) -> np.ndarray:
        return t[:, :, :self.Np].double().cpu().numpy()

    # ---------------------------------------------------------------- operators
    def rhs(self, u, out=None, alpha: float = 1.0):
        out = self.zeros(u.device) if out is None else out
        self._check(lib().dg_rhs(self._h, _t_ptr(u), _t_ptr(out), float(alpha)))
        return out

    def step(self, u, res, dt: float, nsteps: int = 1, alpha: float = 1.0):
        self._check(lib().dg_step(self._h, _t_ptr(u), _t_ptr(res), float(dt), int(nsteps), float(alpha)))
        return u, res

    def rhs_transpose(self, v, out=None, alpha: float = 1.0):
        out = self.zeros(v.device) if out is None else out
        self._check(lib().dg_rhs_transpose(self._h, _t_ptr(v), _t_ptr(out), float(alpha)))
        return out

    def receiver_traces(self, u0, recv, dt: float, nsteps: int, eps=None, alpha: float = 1.0):
        import torch
        out = torch.empty((nsteps, 3, recv.numel()), dtype=torch.float32, device=u0.device)
        self._check(lib().dg_receiver_traces(self._h, _t_ptr(u0), None if eps is None else _t_ptr(eps),
                                             float(dt), int(nsteps), float(alpha), _t_ptr(recv), recv.numel(),
                                             _t_ptr(out)))
        return out

    def adjoint(self, u0, recv, Eref, dt: float, nsteps: int, ckpt_every: int = 20, eps=None, alpha: float = 1.0,
                gradients: bool = True):
        """Misfit J (float) and its gradients (dJ/deps FP64 [K], dJ/du0 [6][K][Np_pad]).
        ckpt_every = 0 lets the library choose the segment length from the free device memory.
        gradients=False computes J alone (forward run only) and returns (J, None, None)."""
        import torch
        J = C.c_double()
        g_eps = torch.empty(self.K, dtype=torch.float64, device=u0.device) if gradients else None
        g_u0 = torch.empty_like(u0) if gradients else None
        self._check(lib().dg_adjoint_step(self._h, _t_ptr(u0), None if eps is None else _t_ptr(eps), float(dt),
                                          int(nsteps), int(ckpt_every), float(alpha), _t_ptr(recv), recv.numel(),
                                          _t_ptr(Eref), C.byref(J), None if g_eps is None else _t_ptr(g_eps),
                                          None if g_u0 is None else _t_ptr(g_u0)))
        return J.value, g_eps, g_u0

    def adjoint_segment_steps(self) -> int:
        """Steps per segment used by the last adjoint call (ckpt_every = 0 chooses it)."""
        return int(lib().dg_adjoint_segment_steps(self._h))

    def set_adjoint_form(self, form: str):
        """Reverse stage of the adjoint: "tensor" (tcgen05, FP16x3 split; N <= 5) or "cuda" (FP32 CUDA cores)."""
        self._check(lib().dg_set_adjoint_form(self._h, {"cuda": 0, "tensor": 1}[form]))

    def adjoint_form(self) -> str:
        return "tensor" if lib().dg_adjoint_form(self._h) == 1 else "cuda"

    # ---------------------------------------------------------------- ensembles
    def upload_ensemble(self, meshes, eps=None, dt=None):
        """meshes: list of (VX, VY, VZ, EToV); eps: list of per-element arrays or None;
        dt: per-mesh time steps."""
        M = len(meshes)
        Nv = np.array([m[0].size for m in meshes], dtype=np.int64)
        Ks = np.array([m[3].shape[0] for m in meshes], dtype=np.int64)
        VX = np.ascontiguousarray(np.concatenate([m[0] for m in meshes]), dtype=np.float64)
        VY = np.ascontiguousarray(np.concatenate([m[1] for m in meshes]), dtype=np.float64)
        VZ = np.ascontiguousarray(np.concatenate([m[2] for m in meshes]), dtype=np.float64)
        EToV = np.ascontiguousarray(np.concatenate([m[3] for m in meshes]), dtype=np.int32)
        e = None if eps is None else np.ascontiguousarray(np.concatenate(eps), dtype=np.float32)
        dts = np.ascontiguousarray(dt, dtype=np.float64)
        self._check(lib().dg_ensemble_upload(self._h, M, _np_ptr(Nv), _np_ptr(VX), _np_ptr(VY), _np_ptr(VZ),
                                             _np_ptr(Ks), _np_ptr(EToV), _np_ptr(e), _np_ptr(dts)))
        self.K = int(Ks.sum())
        return self

    def ensemble_layout(self):
        M = C.c_int()
        self._check(lib().dg_ensemble_layout(self._h, C.byref(M), None))
        off = np.zeros(M.value + 1, dtype=np.int64)
        self._check(lib().dg_ensemble_layout(self._h, C.byref(M), _np_ptr(off)))
        return off

    def ensemble_step(self, u, res, nsteps: int, alpha: float = 1.0):
        self._check(lib().dg_ensemble_step(self._h, _t_ptr(u), _t_ptr(res), int(nsteps), float(alpha)))
        return u, res

    def ensemble_tune(self, force: bool = False):
        self._check(lib().dg_ensemble_tune(self._h, 1 if force else 0))

    def ensemble_tuning(self):
        best = C.c_int()
        eb = np.zeros(4, dtype=np.int32)
        ms = np.zeros(4, dtype=np.float32)
        self._check(lib().dg_ensemble_tuning(self._h, C.byref(best), _np_ptr(eb), _np_ptr(ms)))
        return best.value, eb.tolist(), ms.tolist()

    def ensemble_tuning_grid(self):
        """(chosen candidate, [elements per block], [blocks per SM], [ms per step]) over the 8 candidates."""
        best = C.c_int()
        eb = np.zeros(8, dtype=np.int32)
        bps = np.zeros(8, dtype=np.int32)
        ms = np.zeros(8, dtype=np.float32)
        self._check(lib().dg_ensemble_tuning_grid(self._h, C.byref(best), _np_ptr(eb), _np_ptr(bps), _np_ptr(ms)))
        return best.value, eb.tolist(), bps.tolist(), ms.tolist()

    def ensemble_graph_used(self) -> bool:
        return bool(lib().dg_ensemble_graph_used(self._h))

    def sync(self):
        self._check(lib().dg_sync(self._h))

    def set_nonfinite_check(self, enabled: bool = True):
        """dg_step checks u and res for NaN/Inf after its last stage (synchronising)."""
        self._check(lib().dg_set_nonfinite_check(self._h, 1 if enabled else 0))

    def set_wait_limit(self, cycles: int):
        """Device-side wait limit in SM cycles (0 = default, about one second)."""
        self._check(lib().dg_set_wait_limit(self._h, int(cycles)))

    def energy(self, u) -> float:
        E = C.c_double()
        self._check(lib().dg_energy(self._h, _t_ptr(u), C.byref(E)))
        return E.value


class MaxwellSolve:
    """torch.autograd.Function: the receiver traces E(recv) after each of
    nsteps LSERK4 steps from u0 with per-element permittivity eps, shape
    [nsteps][3][R] (dg_receiver_traces). backward(G), G = dL/dtraces, runs the
    library's hand-written adjoint (dg_adjoint_step) against the reference
    traces E_ref = traces - G / 2: the gradient of that misfit,
    sum_n 2 (P u_n - E_ref,n) . d(P u_n), is sum_n G_n . d traces_n, the
    vector-Jacobian product. The residuals P u_n - E_ref,n are formed in FP32
    from the same traces, so G is carried to about one FP32 ulp of the traces."""

    @staticmethod
    def _fn():
        import torch

        class _Solve(torch.autograd.Function):
            @staticmethod
            def forward(ctx, u0, eps, solver, recv, dt, nsteps, ckpt_every, alpha):
                u0c, epsc = u0.detach().contiguous(), eps.detach().contiguous()
                traces = solver.receiver_traces(u0c, recv, dt, nsteps, eps=epsc, alpha=alpha)
                ctx.save_for_backward(u0c, epsc, recv, traces)
                ctx.args = (solver, dt, nsteps, ckpt_every, alpha)
                return traces

            @staticmethod
            def backward(ctx, G):
                u0c, epsc, recv, traces = ctx.saved_tensors
                solver, dt, nsteps, ckpt_every, alpha = ctx.args
                Eref = (traces - 0.5 * G.to(traces.dtype)).contiguous()
                _, g_eps, g_u0 = solver.adjoint(u0c, recv, Eref, dt, nsteps, ckpt_every, eps=epsc, alpha=alpha)
                return g_u0, g_eps.to(torch.float32), None, None, None, None, None, None

        return _Solve

    @classmethod
    def apply(cls, u0, eps, solver, recv, dt, nsteps, ckpt_every=20, alpha=1.0):
        return cls._fn().apply(u0, eps, solver, recv, dt, nsteps, ckpt_every, alpha)


class ReceiverMisfit:
    """torch.autograd.Function: J(u0, eps) = sum over steps and receivers of
    |E - E_ref|^2 for an LSERK4 run. When u0 or eps requires a gradient the
    forward pass calls dg_adjoint_step, which returns the misfit together with
    its exact discrete gradients (the library's hand-written adjoint), and
    backward scales the saved gradients by the incoming gradient of J;
    otherwise the forward pass runs the forward sweep alone."""

    @staticmethod
    def _fn():
        import torch

        class _Misfit(torch.autograd.Function):
            @staticmethod
            def forward(ctx, u0, eps, solver, recv, Eref, dt, nsteps, ckpt_every, alpha):
                want = bool(ctx.needs_input_grad[0] or ctx.needs_input_grad[1])
                J, g_eps, g_u0 = solver.adjoint(u0.detach().contiguous(), recv, Eref, dt, nsteps, ckpt_every,
                                                eps=eps.detach().contiguous(), alpha=alpha, gradients=want)
                if want:
                    ctx.save_for_backward(g_u0, g_eps)
                return torch.tensor(J, dtype=torch.float64, device=u0.device)

            @staticmethod
            def backward(ctx, gJ):
                g_u0, g_eps = ctx.saved_tensors
                return (gJ.to(g_u0.dtype) * g_u0, (gJ * g_eps).to(torch.float32),
                        None, None, None, None, None, None, None)

        return _Misfit

    @classmethod
    def apply(cls, u0, eps, solver, recv, Eref, dt, nsteps, ckpt_every=20, alpha=1.0):
        return cls._fn().apply(u0, eps, solver, recv, Eref, dt, nsteps, ckpt_every, alpha)
