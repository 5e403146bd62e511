"""Training pipeline of the phase-change source surrogate (GPU, the library's kernels).

States are sampled from the library's own FP64 runs (active cells only), inputs and targets
come from its FP64 plain source (ct_mlp_dataset), and the network is trained with its own
forward/backward/Adam kernels.  This module only orchestrates: batching, index gathers and
bookkeeping use PyTorch as plumbing; every arithmetic step of the network runs in
libcontrail.so.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from .solver import Solver

LAYERS = (16, 128, 128, 128, 128, 10)


def init_params(seed: int = 0) -> np.ndarray:
    """Uniform(+-sqrt(6/fan_in)) weights and zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(LAYERS) - 1):
        fi, fo = LAYERS[l], LAYERS[l + 1]
        lim = np.sqrt(6.0 / fi) * (0.5 if l == len(LAYERS) - 2 else 1.0)
        parts.append(rng.uniform(-lim, lim, size=fo * fi))
        parts.append(np.zeros(fo))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == L.ct_mlp_param_count()
    return p


def sample_active_states(case: dict, ufac=None, nsteps: int = 200, every: int = 5, cfl: float = 0.5,
                         max_rows: int | None = None, device="cuda") -> torch.Tensor:
    """Conserved states (n x 14, float64, on the device) of the active cells of an FP64 run,
    taken every `every` steps."""
    s = Solver(case, ufac, precision=L.CT_FP64, device=device)
    s.init_state(cfl)
    rows = []
    for k in range(nsteps):
        s.step(1, cfl)
        if k % every == every - 1:
            act = s.derived(6) > 0.5
            if bool(act.any()):
                rows.append(s.U[:, act].T.contiguous())
    if not rows:
        return torch.zeros((0, 14), dtype=torch.float64, device=device)
    out = torch.cat(rows, 0)
    if max_rows is not None and out.shape[0] > max_rows:
        g = torch.Generator(device=out.device)
        g.manual_seed(0)
        out = out[torch.randperm(out.shape[0], generator=g, device=out.device)[:max_rows]]
    return out


def dataset(case: dict, U: torch.Tensor):
    """Inputs, targets and masks (float32, device) of states U for the case's physics."""
    n = U.shape[0]
    X = torch.empty((n, L.CT_MLP_IN), dtype=torch.float32, device=U.device)
    Y = torch.empty((n, L.CT_MLP_OUT), dtype=torch.float32, device=U.device)
    M = torch.empty_like(Y)
    L.ct_mlp_dataset(case, U.contiguous(), n, X, Y, M)
    return X, Y, M


def colstats(X: torch.Tensor, M: torch.Tensor | None = None) -> torch.Tensor:
    n, d = X.shape
    out = torch.empty((4, d), dtype=torch.float32, device=X.device)
    L.ct_mlp_colstats(X.contiguous(), None if M is None else M.contiguous(), n, d, out)
    return out


@dataclass
class Surrogate:
    params: np.ndarray          # flat FP32 parameters (standardised units)
    x_mean: np.ndarray
    x_sd: np.ndarray
    x_min: np.ndarray           # training hull, raw input units
    x_max: np.ndarray
    y_mean: np.ndarray
    y_sd: np.ndarray
    y_min: np.ndarray           # range of the training targets (the fused step clamps to it)
    y_max: np.ndarray
    history: np.ndarray         # loss per epoch

    def save(self, path: str):
        np.savez(path, params=self.params, x_mean=self.x_mean, x_sd=self.x_sd, x_min=self.x_min,
                 x_max=self.x_max, y_mean=self.y_mean, y_sd=self.y_sd, y_min=self.y_min, y_max=self.y_max,
                 history=self.history)

    @classmethod
    def load(cls, path: str) -> "Surrogate":
        z = np.load(path)
        keys = ("params", "x_mean", "x_sd", "x_min", "x_max", "y_mean", "y_sd", "y_min", "y_max", "history")
        return cls(**{k: z[k] for k in keys})

    def blob(self, device="cuda") -> torch.Tensor:
        """Pack into the device blob of the BF16 tensor-core kernels (ct_mlp_pack)."""
        dev = torch.device(device)
        t = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
        pad = lambda a: np.concatenate([a, np.zeros(16 - a.size, dtype=np.float32)])
        out = torch.zeros(L.ct_mlp_blob_bytes() // 4 + 16, dtype=torch.float32, device=dev)
        L.ct_mlp_pack(t(self.params), t(self.x_mean), t(self.x_sd), t(self.x_min), t(self.x_max),
                      t(pad(self.y_mean)), t(pad(self.y_sd)), t(pad(self.y_min)), t(pad(self.y_max)), out)
        return out

    def predict(self, X: torch.Tensor) -> torch.Tensor:
        """FP32 forward in raw units (for checks; the fused step runs the BF16 kernel)."""
        dev = X.device
        n = X.shape[0]
        Xn = X.clone().contiguous()
        L.ct_mlp_standardize(Xn, n, L.CT_MLP_IN, torch.tensor(self.x_mean, device=dev),
                             torch.tensor(self.x_sd, device=dev))
        p = torch.tensor(self.params, device=dev)
        Yn = torch.empty((n, L.CT_MLP_OUT), dtype=torch.float32, device=dev)
        wb = L.ct_mlp_work_bytes(n)
        work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=dev)
        L.ct_mlp_forward(p, Xn, n, Yn, work, wb)
        return Yn * torch.tensor(self.y_sd, device=dev) + torch.tensor(self.y_mean, device=dev)


def train(X: torch.Tensor, Y: torch.Tensor, M: torch.Tensor, epochs: int = 20, batch: int = 8192,
          lr: float = 2e-3, seed: int = 0, lr_final: float = 5e-5, tensor_cores: bool = False,
          out_weight=None, verbose: bool = False) -> Surrogate:
    """Adam on the masked MSE of standardised targets with a cosine learning-rate decay, run
    entirely by the library (ct_train_surrogate: statistics, standardisation, shuffles,
    batches, gradients and Adam); this wrapper allocates the device buffers."""
    dev = X.device
    n = X.shape[0]
    P = torch.tensor(init_params(seed), device=dev)
    stats = torch.zeros(4 * L.CT_MLP_IN + 4 * L.CT_MLP_OUT, dtype=torch.float32, device=dev)
    wb = L.ct_train_workspace_bytes(n, batch, epochs)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=dev)
    cfg = dict(epochs=epochs, batch=batch, lr=lr, lr_final=lr_final, seed=seed, tensor_cores=int(tensor_cores),
               out_weight=list(out_weight) if out_weight is not None else [1.0] * L.CT_MLP_OUT)
    hist = L.ct_train_surrogate(X.contiguous(), Y.contiguous(), M.contiguous(), n, cfg, P, stats, work, wb,
                                torch.cuda.current_stream(dev))
    if verbose:
        for ep, v in enumerate(hist):
            print(f"epoch {ep}: loss {v:.5f}", flush=True)
    st = stats.cpu().numpy()
    sx = st[:4 * L.CT_MLP_IN].reshape(4, L.CT_MLP_IN)
    sy = st[4 * L.CT_MLP_IN:].reshape(4, L.CT_MLP_OUT)
    return Surrogate(params=P.cpu().numpy(), x_mean=sx[0], x_sd=sx[1], x_min=sx[2], x_max=sx[3], y_mean=sy[0],
                     y_sd=sy[1], y_min=sy[2], y_max=sy[3], history=hist)


def default_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "surrogate.npz")
