"""Row a7: the BF16 network kernels vs the float64 network oracle (forward,
hand-derived gradients), Adam, save/load and the feature builder."""
import os

import numpy as np
import pytest

from oracle import poisson as P
from oracle import unet as U
from paper_1112_3507_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CH = (4, 8, 8, 8)


@pytest.fixture(scope="module")
def lm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1112_3507_gb300 import build as B
    if not os.path.exists(B.LIB) or any(os.path.getmtime(s) > os.path.getmtime(B.LIB) for s in B.sources()):
        B.build()
    from paper_1112_3507_gb300 import lowmach
    return lowmach


def _bf16(a):
    """Round float64 values to bfloat16 (nearest even) and back."""
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


def _setup(seed=5, B=2, H=16, W=16):
    rng = np.random.default_rng(seed)
    Pp = U.init_params(rng, cin=3, ch=CH)
    for k in Pp:
        if k.islower():
            Pp[k] = rng.standard_normal(Pp[k].shape) * 0.1
    x = rng.standard_normal((B, H, W, 3))
    return rng, Pp, x


def _oracle_params_as_gpu_sees_them(Pp):
    """The kernels use BF16 copies of the 3x3 weights; biases and the 1x1
    output layer stay float32."""
    Q = {}
    for k, v in Pp.items():
        Q[k] = _bf16(v) if (k[0] in "ABCD") else np.float32(v).astype(np.float64)
    return Q


def test_forward_matches_oracle(lm):
    rng, Pp, x = _setup()
    net = lm.Net(CH)
    net.set_params(U.flat_params(Pp, 3, CH))
    xd = torch.as_tensor(x.astype(np.float32).ravel(), device="cuda")
    yd = torch.empty(x.shape[0] * 16 * 16, device="cuda")
    net.forward(xd, yd, x.shape[0], 16, 16)
    y = yd.cpu().numpy().astype(np.float64).reshape(x.shape[0], 16, 16, 1)
    # the oracle stores its activations at BF16 like the kernels
    y_ref, _ = U.forward(_oracle_params_as_gpu_sees_them(Pp), x, CH, rnd=_bf16)
    assert np.linalg.norm(y - y_ref) <= 1e-2 * np.linalg.norm(y_ref)
    # and stays close to the plain float64 network
    y64, _ = U.forward(Pp, x, CH)
    assert np.linalg.norm(y - y64) <= 5e-2 * np.linalg.norm(y64)
    net.close()


@pytest.mark.parametrize("ch,H,W", [((16, 32, 48, 64), 16, 16), ((8, 16, 24, 32), 24, 40)])
def test_tensor_core_forward_matches_oracle(lm, ch, H, W):
    """The production widths: every 3x3 convolution of the forward pass runs
    on the tensor cores (output widths multiples of 8), incl. ragged tiles."""
    rng = np.random.default_rng(11)
    Pp = U.init_params(rng, cin=3, ch=ch)
    for k in Pp:
        if k.islower():
            Pp[k] = rng.standard_normal(Pp[k].shape) * 0.1
    x = rng.standard_normal((2, H, W, 3))
    net = lm.Net(ch)
    net.set_params(U.flat_params(Pp, 3, ch))
    xd = torch.as_tensor(x.astype(np.float32).ravel(), device="cuda")
    yd = torch.empty(2 * H * W, device="cuda")
    net.forward(xd, yd, 2, H, W)
    y = yd.cpu().numpy().astype(np.float64).reshape(2, H, W, 1)
    y_ref, _ = U.forward(_oracle_params_as_gpu_sees_them(Pp), x, ch, rnd=_bf16)
    assert np.linalg.norm(y - y_ref) <= 1e-2 * np.linalg.norm(y_ref)
    net.close()


def test_gradients_match_oracle(lm):
    rng, Pp, x = _setup(seed=6)
    net = lm.Net(CH)
    net.set_params(U.flat_params(Pp, 3, CH))
    B = x.shape[0]
    xd = torch.as_tensor(x.astype(np.float32).ravel(), device="cuda")
    yd = torch.empty(B * 256, device="cuda")
    net.forward(xd, yd, B, 16, 16)
    gy = rng.standard_normal((B, 16, 16, 1))
    net.backward(torch.as_tensor(gy.astype(np.float32).ravel(), device="cuda"))
    g_gpu = U.unflat_params(net.grads(), 3, CH)
    Q = _oracle_params_as_gpu_sees_them(Pp)
    _, cache = U.forward(Q, x, CH, rnd=_bf16)        # same stored activations, same relu decisions
    G, _ = U.backward(Q, cache, gy, CH)
    a = np.concatenate([g_gpu[n].ravel() for n, _ in U.param_shapes(3, CH)])
    b = np.concatenate([G[n].ravel() for n, _ in U.param_shapes(3, CH)])
    assert np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.9999
    for n, _ in U.param_shapes(3, CH):
        ref = G[n]
        assert np.linalg.norm(g_gpu[n] - ref) <= 1e-2 * np.linalg.norm(ref) + 1e-6, n
    net.close()


def test_gradients_at_production_widths(lm):
    """Widths 16/32/48/64: every backward-data convolution (output widths 16
    to 112, incl. the concatenations) runs on the tensor cores with the
    split-precision input; gradients still match the oracle."""
    ch = (16, 32, 48, 64)
    rng = np.random.default_rng(12)
    Pp = U.init_params(rng, cin=3, ch=ch)
    for k in Pp:
        if k.islower():
            Pp[k] = rng.standard_normal(Pp[k].shape) * 0.1
    x = rng.standard_normal((2, 16, 16, 3))
    net = lm.Net(ch)
    net.set_params(U.flat_params(Pp, 3, ch))
    xd = torch.as_tensor(x.astype(np.float32).ravel(), device="cuda")
    yd = torch.empty(2 * 256, device="cuda")
    net.forward(xd, yd, 2, 16, 16)
    gy = rng.standard_normal((2, 16, 16, 1))
    net.backward(torch.as_tensor(gy.astype(np.float32).ravel(), device="cuda"))
    g_gpu = U.unflat_params(net.grads(), 3, ch)
    Q = _oracle_params_as_gpu_sees_them(Pp)
    _, cache = U.forward(Q, x, ch, rnd=_bf16)
    G, _ = U.backward(Q, cache, gy, ch)
    a = np.concatenate([g_gpu[n].ravel() for n, _ in U.param_shapes(3, ch)])
    b = np.concatenate([G[n].ravel() for n, _ in U.param_shapes(3, ch)])
    assert np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.9999
    for n, _ in U.param_shapes(3, ch):
        assert np.linalg.norm(g_gpu[n] - G[n]) <= 1e-2 * np.linalg.norm(G[n]) + 1e-6, n
    net.close()


def test_adam_reduces_loss_and_save_load(lm, tmp_path):
    rng, Pp, x = _setup(seed=7, B=4, H=32, W=32)
    net = lm.Net(CH)
    net.set_params(U.flat_params(Pp, 3, CH))
    B = x.shape[0]
    xd = torch.as_tensor(x.astype(np.float32).ravel(), device="cuda")
    t = torch.as_tensor(np.tanh(x[..., :1]).astype(np.float32).ravel(), device="cuda")
    y = torch.empty_like(t)
    gy = torch.empty_like(t)
    losses = []
    for _ in range(60):
        net.forward(xd, y, B, 32, 32)
        losses.append(net.mse(y, t, gy))
        net.backward(gy)
        net.adam(3e-3)
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
    path = tmp_path / "net.bin"
    net.save(path)
    net2 = lm.Net.load(path)
    assert np.array_equal(net2.params(), net.params())
    y2 = torch.empty_like(t)
    net.forward(xd, y, B, 32, 32)
    net2.forward(xd, y2, B, 32, 32)
    assert torch.equal(y, y2)
    raw = bytearray(path.read_bytes())
    raw[40] ^= 0xFF                      # corrupt a parameter byte: the checksum rejects the file
    bad = tmp_path / "bad.bin"
    bad.write_bytes(bytes(raw))
    with pytest.raises(lm.LowMachError) as e:
        lm.Net.load(bad)
    assert e.value.code == lm.LM_ERR_NETWORK
    net.close()
    net2.close()


def test_features_match_oracle(lm):
    p = I.config_training_2d(3, n=64)
    g = lm.Grid.for_problem(p)
    g.set_problem(p)
    f = torch.as_tensor(p.f.ravel(), device="cuda")
    feat = torch.empty(3 * p.size, device="cuda")
    s = g.features(f, feat)
    op = P.operator_from_problem(p)
    ct32 = op.ct.astype(np.float32).astype(np.float64)
    rho32 = p.rho_new.astype(np.float32).astype(np.float64)
    x_ref, s_ref = U.features(p.f.reshape(p.n[2], p.n[0]), rho32.reshape(p.n[2], p.n[0]),
                              ct32.reshape(p.n[2], p.n[0]), p.h[2])
    got = feat.cpu().numpy().astype(np.float64).reshape(x_ref.shape)
    assert np.allclose(got, x_ref, rtol=2e-5, atol=2e-5)
    assert s == pytest.approx(s_ref, rel=1e-6)
    g.close()
