"""Per-phase cycle breakdown of the tensor-core stage kernel.

Builds a separate copy of the library with -DDGMX_STAGE_TIMING (into
_build_timing/; the library the package loads by default has no timing code),
runs a few LSERK4 steps of the jittered cube mesh, reads the phase timestamps
of the last single-stage launch (dgmx_tc_trace) and prints, per phase, thread
0's cycles averaged over all blocks and over the tiles 1 .. 30 of each block:

  0 -> 1   wait for the tile's staged fields, load them, FP16 row maxima
  1 -> 2   field split into the GEMM1 operand in tensor memory
  2 -> 3   neighbour gathers and upwind fluxes (warp 0), then the flux barrier
  4 -> 5   flux split into the GEMM2 operand (GEMM1 issued at 4, GEMM2 at 5)
  5 -> 6   GEMM1 wait; 6 -> 7 volume terms; 7 -> 12 GEMM2 and residual waits
  8 -> 9   epilogue (lifted flux, update) into the output buffer
  9 -> 0'  bulk stores issued, next tile

At N = 6, 7 (the kernel that streams its operators from L2, dgmx_tcs_trace):

  0 -> 1   fields from L2 into registers, face table
  1 -> 2   field split into the GEMM1 operand in shared memory
  2 -> 3   neighbour gathers and upwind fluxes (warp 0); 2 -> 13: GEMM1 issued
  3 -> 4   GEMM1 wait and barrier
  4 -> 5   flux split; 5 -> 14: GEMM2 issued
  5 -> 6   geometry and first residual chunk; 6 -> 7 GEMM2 wait
  8 -> 9   epilogue

The adjoint's tensor-core reverse stage (dgmx_adj_trace; case `adjoint N n`,
a few steps of the adjoint workload's problem on the n^3 x 6 mesh):

  0 -> 1   the tile's lambda_r, lambda_u and face data staged
  1 -> 2   face constants, W lambda_r split into GEMM-D's operand (GEMM-D issued at 2)
  2 -> 3   face loop: transposed flux, gradient weight terms
  3 -> 4   GEMM-D wait; 4 -> 5 epilogue (transposed curl, lambda updates)
  5 -> 6   W lambda_r split for GEMM-L; 6 -> 7 GEMM-L wait; 7 -> 8 face data stored
  8 -> 9   gradient partials, buffers cleared

Usage (on a GPU): python -m paper_1211_0582_gb300.stage_timing [precision N n] ...
e.g. `fp16x3 5 24 bf16x3 5 24 fp16x3 7 16 adjoint 4 20`. N <= 5 times the
default (single-tile) form.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TILES, EVENTS, BLOCKS = 32, 16, 160
PHASES = [(0, 1, "fields in registers"), (1, 2, "field split"), (2, 3, "fluxes (warp 0)"),
          (3, 4, "flux barrier"), (4, 5, "flux split, GEMM1 issued"), (5, 6, "GEMM1 wait"), (6, 7, "volume terms"),
          (7, 12, "GEMM2 + residual wait"), (12, 8, "barrier"), (8, 9, "epilogue")]
PHASES_STREAMED = [(0, 10, "thread 0's field loads landed (FP16)"), (0, 12, "thread 0's face table written"),
                   (0, 11, "previous tile's stores read (MMA thread)"), (0, 1, "fields and face table"), (1, 2, "field split"), (2, 3, "fluxes (warp 0)"),
                   (2, 13, "GEMM1 issued (MMA thread)"), (3, 4, "GEMM1 wait, barrier"), (4, 5, "flux split"),
                   (5, 14, "GEMM2 issued (MMA thread)"), (5, 6, "geometry, first residual"),
                   (6, 7, "GEMM2 wait"), (7, 8, "barrier"), (8, 9, "epilogue")]


def timing_library() -> str:
    from . import build as B
    return B.build(defines=["DGMX_STAGE_TIMING"], out_dir=os.path.join(HERE, "_build_timing"))


def breakdown(prec: str, N: int, n: int, order: str = "hilbert") -> dict:
    import torch

    import paper_1211_0582_gb300 as dg
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import workloads as W
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1, order=order)
    s = dg.Solver(N, precision=prec).upload(VX, VY, VZ, EToV)
    x, y, z = s.node_coords()
    u, r = s.to_device(W.cavity_mode(x, y, z, 0.0)), s.zeros()
    s.step(u, r, 0.5 / n / N ** 2, 3)
    s.sync()
    buf = np.zeros(BLOCKS * TILES * EVENTS, dtype=np.uint32)
    streamed = N >= 6
    reader = dg.lib().dgmx_tcs_trace if streamed else dg.lib().dgmx_tc_trace
    rc = reader(buf.ctypes.data_as(C.c_void_p))
    torch.cuda.synchronize()
    if rc != 0:
        raise RuntimeError(f"dgmx_tc_trace failed ({rc})")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    T = buf.reshape(BLOCKS, TILES, EVENTS).astype(np.float64)[:sms]
    nt = min(TILES, EToV.shape[0] // 20 // sms)
    if nt < 4:
        raise ValueError("the mesh gives fewer than 4 tiles per block")
    cur, nxt = T[:, 1:nt - 1], T[:, 2:nt]
    out = {"period": float((nxt[:, :, 0] - cur[:, :, 0]).mean())}
    for a, b, name in (PHASES_STREAMED if streamed else PHASES):
        out[name] = float((cur[:, :, b] - cur[:, :, a]).mean())
    out["stores, next tile"] = float((nxt[:, :, 0] - cur[:, :, 9]).mean())
    if not streamed:
        out["first warp done with fluxes (after 2)"] = float((cur[:, :, 11] - cur[:, :, 2]).mean())
        out["last warp done with fluxes (after 2)"] = float((cur[:, :, 10] - cur[:, :, 2]).mean())
    return out


ADJ_TILES, ADJ_EVENTS, ADJ_BLOCKS = 16, 12, 320
ADJ_PHASES = [(0, 1, "tile staged"), (1, 2, "face constants, split, GEMM-D issued"), (2, 3, "face loop"),
              (3, 4, "GEMM-D wait"), (4, 5, "epilogue"), (5, 6, "split for GEMM-L"), (6, 7, "GEMM-L wait"),
              (7, 8, "face data stored"), (8, 9, "gradient partials, clear")]


def adjoint_breakdown(N: int, n: int, steps: int = 3) -> dict:
    import torch

    import paper_1211_0582_gb300 as dg
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import workloads as W
    VX, VY, VZ, EToV = W.kuhn_cube(n, jitter=0.1, seed=1)
    K = EToV.shape[0]
    eps = W.element_eps(K, seed=2)
    s = dg.Solver(N).upload(VX, VY, VZ, EToV, eps=eps)
    s.set_adjoint_form("tensor")
    x, y, z = s.node_coords()
    u0 = s.to_device(W.gaussian_pulse(x, y, z, seed=7))
    recv = torch.as_tensor(W.receivers(K, s.Np, 256, seed=4), device="cuda")
    dt = 0.5 / n / N ** 2
    Eref = s.receiver_traces(u0, recv, dt, steps, eps=torch.as_tensor(W.element_eps(K, seed=6), device="cuda"))
    s.adjoint(u0, recv, Eref, dt, steps, 0, eps=torch.as_tensor(eps, device="cuda"))
    buf = np.zeros(ADJ_BLOCKS * ADJ_TILES * ADJ_EVENTS, dtype=np.uint32)
    rc = dg.lib().dgmx_adj_trace(buf.ctypes.data_as(C.c_void_p))
    torch.cuda.synchronize()
    if rc != 0:
        raise RuntimeError(f"dgmx_adj_trace failed ({rc})")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nb = min(ADJ_BLOCKS, 2 * sms)
    T = buf.reshape(ADJ_BLOCKS, ADJ_TILES, ADJ_EVENTS).astype(np.float64)[:nb]
    nt = min(ADJ_TILES, K // 20 // nb)
    if nt < 4:
        raise ValueError("the mesh gives fewer than 4 tiles per block")
    cur, nxt = T[:, 1:nt - 1], T[:, 2:nt]
    out = {"period": float((nxt[:, :, 0] - cur[:, :, 0]).mean())}
    for a, b, name in ADJ_PHASES:
        out[name] = float((cur[:, :, b] - cur[:, :, a]).mean())
    return out


def main(argv) -> None:
    import paper_1211_0582_gb300 as dg
    dg._LIB_PATH = timing_library()
    dg._lib = None
    cases = [(argv[i], int(argv[i + 1]), int(argv[i + 2])) for i in range(0, len(argv) - 2, 3)] or \
        [("fp16x3", 5, 24), ("bf16x3", 5, 24), ("fp16x3", 4, 28)]
    for prec, N, n in cases:
        if prec == "adjoint":
            b = adjoint_breakdown(N, n)
            print(f"adjoint reverse stage (tensor cores) N={N} {n}^3x6 tets: cycles per tile, thread 0 (last launch)")
        else:
            b = breakdown(prec, N, n)
            print(f"{prec} N={N} {n}^3x6 tets (Hilbert order): cycles per tile, thread 0")
        for k, v in b.items():
            pct = "" if k == "period" or k.startswith(("first", "last", "thread 0", "previous")) or "issued" in k \
                else f"  {100 * v / b['period']:5.1f}%"
            print(f"  {k:<40} {v:8.0f}{pct}")


if __name__ == "__main__":
    main(sys.argv[1:])
