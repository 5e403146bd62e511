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
          lr: float = 2e-3, seed: int = 0, lr_final: float = 5e-5, verbose: bool = False) -> Surrogate:
    """Adam on the masked MSE of standardised targets, cosine learning-rate decay."""
    dev = X.device
    n = X.shape[0]
    sx = colstats(X)
    sy = colstats(Y, M)
    x_sd = torch.where(sx[1] > 1e-6, sx[1], torch.ones_like(sx[1]))
    y_sd = torch.where(sy[1] > 1e-6, sy[1], torch.ones_like(sy[1]))
    Xn = X.clone().contiguous()
    Yn = Y.clone().contiguous()
    L.ct_mlp_standardize(Xn, n, L.CT_MLP_IN, sx[0].contiguous(), x_sd.contiguous())
    L.ct_mlp_standardize(Yn, n, L.CT_MLP_OUT, sy[0].contiguous(), y_sd.contiguous())
    Yn = Yn * M      # masked entries carry no information
    P = torch.tensor(init_params(seed), device=dev)
    G = torch.zeros_like(P)
    m1 = torch.zeros_like(P)
    m2 = torch.zeros_like(P)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    wb = L.ct_mlp_work_bytes(batch)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    nb = max(1, n // batch)
    total = epochs * nb
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=dev)
        acc = torch.zeros((), dtype=torch.float64, device=dev)
        for b in range(nb):
            idx = perm[b * batch:(b + 1) * batch]
            xb, yb, mb = Xn[idx].contiguous(), Yn[idx].contiguous(), M[idx].contiguous()
            L.ct_mlp_loss_grad(P, xb, yb, mb, xb.shape[0], G, loss, work, wb)
            step += 1
            frac = step / total
            lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + np.cos(np.pi * frac))
            L.ct_mlp_adam(P, G, m1, m2, P.numel(), float(lr_t), 0.9, 0.999, 1e-8, step)
            acc += loss[0].double()
        hist.append(float(acc) / nb)
        if verbose:
            print(f"epoch {ep}: loss {hist[-1]:.5f}", flush=True)
    return Surrogate(params=P.cpu().numpy(), x_mean=sx[0].cpu().numpy(), x_sd=x_sd.cpu().numpy(),
                     x_min=sx[2].cpu().numpy(), x_max=sx[3].cpu().numpy(), y_mean=sy[0].cpu().numpy(),
                     y_sd=y_sd.cpu().numpy(), y_min=sy[2].cpu().numpy(), y_max=sy[3].cpu().numpy(),
                     history=np.array(hist))


def default_path() -> str:
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "surrogate.npz")
