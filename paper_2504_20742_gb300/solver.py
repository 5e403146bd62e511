"""Thin convenience wrapper: device buffers from PyTorch, calls through the C ABI."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


class Solver:
    """One case on one GPU.  State tensors are (nf, nr, nx), float64 (CT_FP64) or float32;
    nf = 14, or 18 with the bimodal liquid."""

    def __init__(self, case: dict, ufac_rows=None, precision: int = L.CT_FP64, device="cuda:0",
                 stream: torch.cuda.Stream | None = None):
        self.case = dict(case)
        self.precision = precision
        self.device = torch.device(device)
        self.nx = int(case["nx"])
        self.nr = int(case["nr"]) if int(case["geom"]) == 1 else 1
        self.dtype = torch.float64 if precision == L.CT_FP64 else torch.float32
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.nf = L.nfields(self.case)
        self.U = torch.zeros((self.nf, self.nr, self.nx), dtype=self.dtype, device=self.device)
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

    def autotune(self, reps: int = 5):
        """Pick the fastest tile shape for this grid (state unchanged); returns (shape, ms)."""
        return L.ct_autotune(self.case, self.precision, self.U, self.U1, self.work, getattr(self, "blob", None),
                             reps, self.stream)

    def derived(self, which: int, dt: float = 1e-6) -> torch.Tensor:
        out = torch.empty((self.nr, self.nx), dtype=torch.float64, device=self.device)
        L.ct_derived(self.case, self.precision, self.U, which, dt, out, self.stream)
        return out

    def state64(self) -> np.ndarray:
        self.stream.synchronize()
        return self.U.detach().to(torch.float64).cpu().numpy()

    def read_field(self, field: int) -> np.ndarray:
        """One field of the state as an (nr, nx) float64 host array (ct_read_field)."""
        return L.ct_read_field(self.case, self.precision, self.U, field, self.stream)


class Batch:
    """Many axisymmetric cases stepped together by the persistent, graph-captured kernel.
    The batch state is one float32 tensor; `state(k)` views case k as (nf, nr, nx)."""

    def __init__(self, cases: list, ufac_rows: list | None = None, precision: int = L.CT_FP32_MLP,
                 device="cuda:0", stream: torch.cuda.Stream | None = None, blob: torch.Tensor | None = None):
        self.cases = [dict(c) for c in cases]
        self.precision = precision
        self.device = torch.device(device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self.blob = blob
        n = L.ct_batch_state_elems(self.cases)
        if n == 0:
            raise L.ContrailError(1, "invalid batch: " + L.ct_last_error())
        self.U = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.U1 = torch.zeros_like(self.U)
        nbytes = L.ct_batch_workspace_bytes(self.cases)
        self.work = torch.zeros(nbytes // 8 + 64, dtype=torch.float64, device=self.device)
        rows = None
        if ufac_rows is not None:
            rows = np.concatenate([np.asarray(r, dtype=np.float64) for r in ufac_rows])
        self.handle = L.ct_batch_create(self.cases, precision, rows, self.work, nbytes, self.stream)
        self.offsets = []
        off = 0
        for c in self.cases:
            self.offsets.append(off)
            off += L.nfields(c) * int(c["nx"]) * int(c["nr"])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            L.ct_batch_destroy(h)
            self.handle = None

    def state(self, k: int) -> torch.Tensor:
        c = self.cases[k]
        nx, nr = int(c["nx"]), int(c["nr"])
        nf = L.nfields(c)
        return self.U[self.offsets[k]:self.offsets[k] + nf * nx * nr].view(nf, nr, nx)

    def init_state(self, cfl: float = 0.5):
        L.ct_batch_init_state(self.handle, self.U, cfl)

    def load_state(self, U_src: torch.Tensor, cfl: float = 0.5):
        L.ct_batch_load_state(self.handle, U_src, self.U, cfl)

    def autotune(self, reps: int = 3):
        return L.ct_batch_autotune(self.handle, self.U, self.U1, self.blob, reps)

    def set_tile_shape(self, shape: int):
        L.ct_batch_set_tile_shape(self.handle, shape)

    def step(self, nsteps: int, cfl: float = 0.5):
        L.ct_batch_step(self.handle, self.U, self.U1, self.blob, nsteps, cfl)

    def diagnostics(self) -> np.ndarray:
        return L.ct_batch_diagnostics(self.handle, len(self.cases))
