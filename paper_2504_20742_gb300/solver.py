"""Thin convenience wrapper: device buffers from PyTorch, calls through the C ABI."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


class Solver:
    """One case on one GPU.  State tensors are (14, nr, nx), float64 (CT_FP64) or float32."""

    def __init__(self, case: dict, ufac_rows=None, precision: int = L.CT_FP64, device="cuda:0",
                 stream: torch.cuda.Stream | None = None):
        self.case = dict(case)
        self.precision = precision
        self.device = torch.device(device)
        self.nx = int(case["nx"])
        self.nr = int(case["nr"]) if int(case["geom"]) == 1 else 1
        self.dtype = torch.float64 if precision == L.CT_FP64 else torch.float32
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.U = torch.zeros((L.NF, self.nr, self.nx), dtype=self.dtype, device=self.device)
        self.U1 = torch.zeros_like(self.U)
        nbytes = L.ct_workspace_bytes(self.case, precision)
        if nbytes == 0:
            raise L.ContrailError(1, "invalid case: " + L.ct_last_error())
        self.work = torch.zeros(nbytes // 8 + 64, dtype=torch.float64, device=self.device)
        self.work_bytes = nbytes
        L.ct_setup(self.case, precision, ufac_rows, self.work, nbytes, self.stream)

    def init_state(self, cfl: float = 0.5):
        L.ct_init_state(self.case, self.precision, self.work, self.U, cfl, self.stream)
        return self.U

    def load_state(self, U_src: torch.Tensor, cfl: float = 0.5):
        src = U_src.to(device=self.device, dtype=self.dtype).contiguous()
        L.ct_load_state(self.case, self.precision, self.work, src, self.U, cfl, self.stream)

    def attach_surrogate(self, blob: torch.Tensor):
        """Device blob of a packed surrogate (CT_FP32_MLP solvers)."""
        self.blob = blob

    def step(self, nsteps: int, cfl: float = 0.5):
        if self.precision == L.CT_FP32_MLP:
            L.ct_step_surrogate(self.case, self.U, self.U1, self.work, self.blob, nsteps, cfl, self.stream)
        else:
            L.ct_step(self.case, self.precision, self.U, self.U1, self.work, nsteps, cfl, self.stream)

    def diagnostics(self) -> np.ndarray:
        return L.ct_diagnostics(self.work, self.stream)

    def derived(self, which: int, dt: float = 1e-6) -> torch.Tensor:
        out = torch.empty((self.nr, self.nx), dtype=torch.float64, device=self.device)
        L.ct_derived(self.case, self.precision, self.U, which, dt, out, self.stream)
        return out

    def state64(self) -> np.ndarray:
        self.stream.synchronize()
        return self.U.detach().to(torch.float64).cpu().numpy()
