"""PyTorch-facing wrapper of the batched block-tridiagonal solve of the per-ray Newton systems
(C ABI: include/vx_btd.h). All arithmetic runs in libvx_rates.so; this module checks tensors and
passes pointers, and for host data stages the copies around the device call."""
from __future__ import annotations

import torch

from . import capi


class BlockTridiagSolver:
    """Solves, for every ray, A_k x_{k-1} + B_k x_k + C_k x_{k+1} = d_k over its zones k.

    m unknowns per zone (1..128); at most ``max_zones`` zones per call; ``n_refine`` FP64
    refinement sweeps after the FP32 block factorisation (see include/vx_btd.h)."""

    def __init__(self, m: int, max_zones: int, n_refine: int = 2):
        self.m, self.max_zones, self.n_refine = int(m), int(max_zones), int(n_refine)
        self.handle = capi.vx_btd_create(self.m, self.max_zones, self.n_refine)

    def _args(self, offsets, A, B, C, d):
        m = self.m
        Z = d.shape[0]
        for name, t, shape, dt in (("A", A, (Z, m, m), torch.float64), ("B", B, (Z, m, m), torch.float64),
                                   ("C", C, (Z, m, m), torch.float64), ("d", d, (Z, m), torch.float64),
                                   ("offsets", offsets, (offsets.shape[0],), torch.int32)):
            if tuple(t.shape) != shape or t.dtype != dt or not t.is_contiguous():
                raise ValueError(f"{name}: expected contiguous {dt} {shape}, got {t.dtype} {tuple(t.shape)}")
        return int(offsets.shape[0]) - 1, Z

    def solve(self, offsets: torch.Tensor, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, d: torch.Tensor,
              out: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None) -> torch.Tensor:
        """Device tensors in, device solution out (asynchronous on ``stream``)."""
        n_rays, Z = self._args(offsets, A, B, C, d)
        for t in (offsets, A, B, C, d):
            if not t.is_cuda:
                raise ValueError("solve() takes CUDA tensors; use solve_host() for host data")
        if len({t.device for t in (offsets, A, B, C, d)}) != 1:
            raise ValueError("offsets, A, B, C and d must be on one device")
        if out is not None and (not torch.is_tensor(out) or out.dtype != torch.float64 or not out.is_contiguous()
                                or tuple(out.shape) != tuple(d.shape) or out.device != d.device):
            raise ValueError(f"out must be a contiguous float64 tensor of shape {tuple(d.shape)} on {d.device}")
        x = torch.empty_like(d) if out is None else out
        s = (stream or torch.cuda.current_stream(d.device)).cuda_stream
        capi.vx_btd_solve(self.handle, n_rays, Z, offsets.data_ptr(), A.data_ptr(), B.data_ptr(), C.data_ptr(),
                          d.data_ptr(), x.data_ptr(), s)
        return x

    def solve_host(self, offsets: torch.Tensor, A: torch.Tensor, B: torch.Tensor, C: torch.Tensor,
                   d: torch.Tensor, device: str | torch.device = "cuda") -> torch.Tensor:
        """Host tensors (pinned for asynchronous copies) in, host solution out: copies the inputs to
        the device, solves, copies x back and waits for it."""
        n_rays, Z = self._args(offsets, A, B, C, d)
        dev = [t.to(device, non_blocking=True) for t in (offsets, A, B, C, d)]
        x = self.solve(*dev)
        host = torch.empty(tuple(d.shape), dtype=torch.float64, pin_memory=d.is_pinned())
        host.copy_(x, non_blocking=True)
        torch.cuda.current_stream(x.device).synchronize()
        return host

    def check(self, stream: torch.cuda.Stream | None = None) -> bool:
        """False if a solve since the last check met a zero/non-finite pivot or invalid offsets."""
        s = (stream or torch.cuda.current_stream()).cuda_stream
        return capi.vx_btd_check(self.handle, s) == capi.VX_OK

    def close(self) -> None:
        if self.handle is not None:
            capi.vx_btd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
