"""BF16 tensor-core inference (tcgen05) of the surrogate against (a) a numpy emulation that
rounds to BF16 at the same points and accumulates exactly, and (b) the FP32 forward."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlp_ref as R

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2504_20742_gb300 as P
    return P


def bf16(x):
    """Round float32 to bfloat16 (nearest even), returned as float32."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return b.view(np.float32)


def _setup(seed=3, n=1000):
    rng = np.random.default_rng(seed)
    theta = R.init_params(seed).astype(np.float32)
    layers = R.unpack(theta.astype(np.float64))
    # non-zero biases
    theta = theta.copy()
    off = 0
    for (o, i), _ in R.param_shapes():
        off += o * i
        theta[off:off + o] = 0.1 * rng.standard_normal(o)
        off += o
    x_mean = rng.standard_normal(16).astype(np.float32)
    x_sd = (0.5 + rng.uniform(size=16)).astype(np.float32)
    y_mean = np.concatenate([rng.standard_normal(10), np.zeros(6)]).astype(np.float32)
    y_sd = np.concatenate([0.5 + rng.uniform(size=10), np.zeros(6)]).astype(np.float32)
    X = (x_mean + x_sd * rng.standard_normal((n, 16))).astype(np.float32)
    return theta, x_mean, x_sd, y_mean, y_sd, X


def _emulate(theta, x_mean, x_sd, y_mean, y_sd, X):
    h = bf16((X - x_mean) * (1.0 / x_sd).astype(np.float32))
    layers = R.unpack(theta.astype(np.float64))
    for l, (W, b) in enumerate(layers):
        z = h.astype(np.float64) @ bf16(W.astype(np.float32)).astype(np.float64).T + b
        if l < len(layers) - 1:
            h = bf16((z / (1.0 + np.exp(-z))).astype(np.float32))
        else:
            out = z
    return out * y_sd[:10] + y_mean[:10]


def test_tensor_core_inference_matches_bf16_emulation_and_fp32(P):
    theta, x_mean, x_sd, y_mean, y_sd, X = _setup()
    d = "cuda"
    t = lambda a: torch.tensor(np.ascontiguousarray(a), device=d)
    blob = torch.zeros(P.ct_mlp_blob_bytes() // 4 + 16, dtype=torch.float32, device=d)
    P.ct_mlp_pack(t(theta), t(x_mean), t(x_sd), t(X.min(0)), t(X.max(0)), t(y_mean), t(y_sd),
                  t(np.full(16, -1e30, np.float32)), t(np.full(16, 1e30, np.float32)), blob)
    n = X.shape[0]
    Y = torch.zeros((n, 10), dtype=torch.float32, device=d)
    err = torch.zeros(1, dtype=torch.int32, device=d)
    P.ct_mlp_infer(blob, t(X), n, Y, err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    Yg = Y.cpu().numpy()
    Ye = _emulate(theta, x_mean, x_sd, y_mean, y_sd, X)
    scale = np.abs(Ye).max(axis=0)
    # same BF16 rounding points; differences come from FP32 accumulation order and the
    # rounding of activations that sit on a BF16 tie
    assert np.max(np.abs(Yg - Ye) / scale) < 2e-2, np.max(np.abs(Yg - Ye) / scale)
    assert np.median(np.abs(Yg - Ye) / scale) < 1e-3
    # FP32 forward through the library's training kernels
    Xn = ((X - x_mean) / x_sd).astype(np.float32)
    wb = P.ct_mlp_work_bytes(n)
    work = torch.empty(wb // 4 + 64, dtype=torch.float32, device=d)
    Yf = torch.empty((n, 10), dtype=torch.float32, device=d)
    P.ct_mlp_forward(t(theta), t(Xn), n, Yf, work, wb)
    Yf = Yf.cpu().numpy() * y_sd[:10] + y_mean[:10]
    assert np.max(np.abs(Yg - Yf) / scale) < 5e-2
