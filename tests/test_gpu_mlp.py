"""The surrogate's training kernels against the FP64 reference network (oracle/mlp_ref.py),
its dataset kernel against the oracle's source quantities, and a short training run."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from oracle import mlp_ref as R
from synth import cases

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2504_20742_gb300 as P
    return P


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, 16)).astype(np.float32)
    Y = rng.standard_normal((n, 10)).astype(np.float32)
    M = (rng.uniform(size=(n, 10)) > 0.25).astype(np.float32)
    return X, Y, M


def test_forward_and_gradient_match_fp64_reference(P):
    """FP32 device forward/backward vs the FP64 chain rule (itself pinned by finite
    differences) on 64 samples: relative error <= 1e-4 (FP32 arithmetic)."""
    theta = R.init_params(3).astype(np.float32)
    theta += 0.01 * np.random.default_rng(5).standard_normal(theta.size).astype(np.float32)
    X, Y, M = _data(64, 7)
    d = "cuda"
    p = torch.tensor(theta, device=d)
    Xt, Yt, Mt = (torch.tensor(a, device=d) for a in (X, Y, M))
    wb = P.ct_mlp_work_bytes(64)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=d)
    out = torch.empty((64, 10), dtype=torch.float32, device=d)
    P.ct_mlp_forward(p, Xt, 64, out, work, wb)
    yref, _ = R.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.allclose(out.cpu().numpy(), yref, rtol=1e-4, atol=1e-4 * np.abs(yref).max())
    g = torch.empty_like(p)
    loss = torch.zeros(1, device=d)
    P.ct_mlp_loss_grad(p, Xt, Yt, Mt, 64, g, loss, work, wb)
    Lr, gr = R.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                             M.astype(np.float64))
    assert float(loss) == pytest.approx(Lr, rel=1e-5)
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - gr) <= 1e-4 * np.linalg.norm(gr)
    scale = np.abs(gr).max()
    assert np.all(np.abs(gg - gr) <= 1e-4 * (np.abs(gr) + 1e-3 * scale))


def test_adam_step(P):
    rng = np.random.default_rng(2)
    p0 = rng.standard_normal(1000).astype(np.float32)
    g = rng.standard_normal(1000).astype(np.float32)
    m = rng.standard_normal(1000).astype(np.float32) * 0.1
    v = np.abs(rng.standard_normal(1000)).astype(np.float32) * 0.1
    tp, tg, tm, tv = (torch.tensor(a, device="cuda") for a in (p0, g, m, v))
    lr, b1, b2, eps, step = 1e-3, 0.9, 0.999, 1e-8, 7
    P.ct_mlp_adam(tp, tg, tm, tv, 1000, lr, b1, b2, eps, step)
    m1 = b1 * m + (1 - b1) * g
    v1 = b2 * v + (1 - b2) * g * g
    ref = p0 - lr * (m1 / (1 - b1 ** step)) / (np.sqrt(v1 / (1 - b2 ** step)) + eps)
    assert np.allclose(tp.cpu().numpy(), ref, rtol=1e-5, atol=1e-7)


def test_dataset_targets_match_oracle_quantities(P):
    """Targets of the training set against the oracle's own source quantities."""
    import sys, os
    sys.path.insert(0, os.path.dirname(__file__))
    from test_oracle_source import _random_states, _case
    U = _random_states(2000, seed=13)
    c = _case()
    X = torch.empty((2000, 16), device="cuda")
    Y = torch.empty((2000, 10), device="cuda")
    M = torch.empty((2000, 10), device="cuda")
    P.ct_mlp_dataset(c, torch.tensor(U, device="cuda"), 2000, X, Y, M)
    Y, M, X = Y.cpu().numpy(), M.cpu().numpy(), X.cpu().numpy()
    _, aux = O.source_batch(c, U, 1e-14)     # dt -> 0: growth rates without the stage limiter
    nuc = aux[:, 0] > 0
    assert np.array_equal(M[:, 0] > 0, nuc)
    assert np.allclose(X[:, 14], aux[:, 0], rtol=1e-5, atol=1e-5)
    assert np.allclose(X[:, 15], aux[:, 1], rtol=1e-5, atol=1e-5)
    fin = nuc & np.isfinite(aux[:, 2])
    assert np.allclose(Y[fin, 6], np.maximum(aux[fin, 2], -30.0), rtol=1e-5, atol=1e-4)
    assert np.allclose(Y[nuc, 1], np.log(aux[nuc, 5] * 1e6), rtol=1e-5, atol=1e-5)
    assert np.allclose(Y[nuc, 8], np.log1p(aux[nuc, 6]), rtol=1e-4, atol=1e-6)
    pl = M[:, 2] > 0
    assert pl.sum() > 100
    assert np.allclose(Y[pl, 2], np.arcsinh(aux[pl, 7] * 1e6), rtol=1e-4, atol=1e-4)


def test_training_reduces_loss_on_sampled_states(P):
    from paper_2504_20742_gb300 import surrogate as S
    c, uf = cases.freezing_case(nx=64, nr=32)
    U = S.sample_active_states(c, uf, nsteps=40, every=4)
    c2, uf2 = cases.mixing_layer_case(nx=64, nr=32)
    U2 = S.sample_active_states(c2, uf2, nsteps=40, every=4)
    X1, Y1, M1 = S.dataset(c, U)
    X2, Y2, M2 = S.dataset(c2, U2)
    X, Y, M = torch.cat([X1, X2]), torch.cat([Y1, Y2]), torch.cat([M1, M2])
    assert X.shape[0] > 5000 and bool(torch.isfinite(X).all()) and bool(torch.isfinite(Y).all())
    sur = S.train(X, Y, M, epochs=6, batch=2048, lr=2e-3)
    assert sur.history[-1] < 0.25 * sur.history[0], sur.history


def _sampled(P, S):
    c, uf = cases.freezing_case(nx=64, nr=32)
    U = S.sample_active_states(c, uf, nsteps=40, every=4)
    return S.dataset(c, U)


def test_train_surrogate_is_one_deterministic_library_call(P):
    """ct_train_surrogate runs statistics, standardisation, shuffles, batches, gradients and
    Adam inside the library: two calls with the same seed give the same parameters bit for
    bit, another seed other ones, and the statistics are ct_mlp_colstats' (inputs unmasked,
    targets over their mask)."""
    from paper_2504_20742_gb300 import surrogate as S
    X, Y, M = _sampled(P, S)
    n = X.shape[0]
    a = S.train(X, Y, M, epochs=3, batch=1024, lr=2e-3, seed=4)
    b = S.train(X, Y, M, epochs=3, batch=1024, lr=2e-3, seed=4)
    c = S.train(X, Y, M, epochs=3, batch=1024, lr=2e-3, seed=5)
    assert np.array_equal(a.params, b.params) and np.array_equal(a.history, b.history)
    assert not np.array_equal(a.params, c.params)
    assert np.all(np.isfinite(a.params)) and a.history[-1] < a.history[0]
    sx = S.colstats(X).cpu().numpy()
    sy = S.colstats(Y, M).cpu().numpy()
    assert np.array_equal(a.x_mean, sx[0]) and np.array_equal(a.x_min, sx[2]) and np.array_equal(a.x_max, sx[3])
    assert np.array_equal(a.y_mean, sy[0]) and np.array_equal(a.y_max, sy[3])
    assert np.array_equal(a.x_sd, np.where(sx[1] > 1e-6, sx[1], 1.0).astype(np.float32))


def test_train_surrogate_first_epoch_loss_is_the_loss_of_the_initial_network(P):
    """With one batch of all rows per epoch, the first epoch's recorded loss is the masked
    MSE of the initial parameters on the standardised rows (ct_mlp_loss_grad on the
    unshuffled rows; the two sums differ only in order)."""
    from paper_2504_20742_gb300 import surrogate as S
    X, Y, M = _sampled(P, S)
    n = X.shape[0]
    sur = S.train(X, Y, M, epochs=1, batch=n, lr=1e-3, seed=2)
    sx, sy = S.colstats(X), S.colstats(Y, M)
    sdx = torch.where(sx[1] > 1e-6, sx[1], torch.ones_like(sx[1])).contiguous()
    sdy = torch.where(sy[1] > 1e-6, sy[1], torch.ones_like(sy[1])).contiguous()
    Xn, Yn = X.clone().contiguous(), Y.clone().contiguous()
    P.ct_mlp_standardize(Xn, n, 16, sx[0].contiguous(), sdx)
    P.ct_mlp_standardize(Yn, n, 10, sy[0].contiguous(), sdy)
    Yn = (Yn * M).contiguous()
    p0 = torch.tensor(S.init_params(2), device="cuda")
    g = torch.empty_like(p0)
    loss = torch.zeros(1, device="cuda")
    wb = P.ct_mlp_work_bytes(n)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device="cuda")
    P.ct_mlp_loss_grad(p0, Xn, Yn, M.contiguous(), n, g, loss, work, wb)
    assert sur.history[0] == pytest.approx(float(loss), rel=1e-5)


def _tc_grad(P, theta, X, Y, M):
    d = "cuda"
    n = X.shape[0]
    p = torch.tensor(theta, device=d)
    Xt, Yt, Mt = (torch.tensor(a, device=d) for a in (X, Y, M))
    wb = P.ct_mlp_work_bytes(n)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=d)
    g = torch.empty_like(p)
    loss = torch.zeros(1, device=d)
    err = torch.zeros(1, dtype=torch.int32, device=d)
    P.ct_mlp_loss_grad_tc(p, Xt, Yt, Mt, n, g, loss, err, work, wb)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    return float(loss), g.cpu().numpy()


def test_tensor_core_gradient_matches_fp64_reference(P):
    """BF16 tensor-core forward and backward (FP32 accumulation, FP32 master weights) vs the
    FP64 chain rule on 64 samples: loss and gradient within 1e-2 relative (BF16 operands)."""
    theta = R.init_params(3).astype(np.float32)
    theta += 0.01 * np.random.default_rng(5).standard_normal(theta.size).astype(np.float32)
    X, Y, M = _data(64, 7)
    loss, gg = _tc_grad(P, theta, X, Y, M)
    Lr, gr = R.loss_and_grad(theta.astype(np.float64), X.astype(np.float64), Y.astype(np.float64),
                             M.astype(np.float64))
    assert loss == pytest.approx(Lr, rel=1e-2)
    assert np.linalg.norm(gg - gr) <= 1e-2 * np.linalg.norm(gr)
    # layer by layer, every weight and bias block within 2e-2 of its own norm
    off = 0
    for fi, fo in zip(R.LAYERS[:-1], R.LAYERS[1:]):
        for size in (fi * fo, fo):
            blk = slice(off, off + size)
            assert np.linalg.norm(gg[blk] - gr[blk]) <= 2e-2 * np.linalg.norm(gr[blk]) + 1e-12, (fi, fo, size)
            off += size


@pytest.mark.parametrize("n", [1000, 8192])
def test_tensor_core_gradient_matches_fp32_kernels_on_batches(P, n):
    """Full batches (split-K weight gradients over up to 32 partial tiles, ragged row counts):
    tensor-core and FP32 gradients agree within 1e-2 relative."""
    theta = R.init_params(4).astype(np.float32)
    X, Y, M = _data(n, 9)
    loss_tc, g_tc = _tc_grad(P, theta, X, Y, M)
    d = "cuda"
    p = torch.tensor(theta, device=d)
    Xt, Yt, Mt = (torch.tensor(a, device=d) for a in (X, Y, M))
    wb = P.ct_mlp_work_bytes(n)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=d)
    g = torch.empty_like(p)
    loss = torch.zeros(1, device=d)
    P.ct_mlp_loss_grad(p, Xt, Yt, Mt, n, g, loss, work, wb)
    g32 = g.cpu().numpy()
    assert loss_tc == pytest.approx(float(loss), rel=1e-2)
    assert np.linalg.norm(g_tc - g32) <= 1e-2 * np.linalg.norm(g32)


def test_tensor_core_training_reduces_loss(P):
    from paper_2504_20742_gb300 import surrogate as S
    X, Y, M = _sampled(P, S)
    sur = S.train(X, Y, M, epochs=4, batch=2048, lr=2e-3, tensor_cores=True)
    assert np.all(np.isfinite(sur.params)) and sur.history[-1] < 0.5 * sur.history[0], sur.history
