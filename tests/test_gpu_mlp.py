"""GPU parity of the tile-error MLP kernels (bf16 tensor-core layers, fp32
accumulation) against the oracle's bf16-mode network, and an Adam training
run on a seeded regression task."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2606_15924_gb300 import binding as B
    from paper_2606_15924_gb300.predictor import TileErrorMLP
    B.device_check()
    return B, TileErrorMLP


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def _features(R, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((R, 16), np.float32)
    x[:, :5] = rng.normal(size=(R, 5)).astype(np.float32)
    return x


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("R", [1, 15, 16, 1000, 4097])
def test_forward_parity(P, orc, R, tc):
    """tc: the tcgen05 kernel (128-row tiles, accumulators in tensor memory);
    otherwise the mma.sync kernel."""
    B, TileErrorMLP = P
    mlp = TileErrorMLP(seed=R)
    x = _features(R, R)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty(R, device="cuda")
    h1 = torch.empty(R, 128, dtype=torch.int16, device="cuda")
    h2 = torch.empty(R, 128, dtype=torch.int16, device="cuda")
    if tc:
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.mlp_forward_tc(mlp.net(), xd, y, h1, h2, status=status)
        assert int(status.item()) == 0
    else:
        B.mlp_forward(mlp.net(), xd, y, h1, h2)
    yw, h1w, h2w = orc.mlp_forward(x, mlp.weights_fp(), bf16=True)
    got = y.cpu().numpy()
    print(f"mlp forward R={R} tc={tc}: y rel L2 {rel_l2(got, yw):.3e}")
    # measured on GB300: at most 1.4e-5 (4097 rows); the bound leaves a factor of 7
    assert rel_l2(got, yw) <= 1e-4
    assert np.abs(got - yw).max() <= 1e-3 * max(1.0, np.abs(yw).max())
    for hg, hw in ((h1, h1w), (h2, h2w)):
        hv = hg.view(torch.bfloat16).float().cpu().numpy().astype(np.float64)
        # fp32 vs fp64 accumulation may move a value across a bf16 rounding
        # boundary: then the two differ by one bf16 ulp
        diff = hv != hw
        assert diff.mean() < 2e-3
        ulp = np.abs(hw[diff]) * 2.0 ** -7 + 1e-30
        assert np.all(np.abs(hv[diff] - hw[diff]) <= 1.01 * ulp)


@pytest.mark.parametrize("tc", [False, True])
@pytest.mark.parametrize("R", [33, 130, 2048, 5000])
def test_backward_parity(P, orc, R, tc):
    """tc: the weight gradients as tcgen05 contractions over 128-row tiles
    (the last one ragged); otherwise on the CUDA cores."""
    B, TileErrorMLP = P
    mlp = TileErrorMLP(seed=7)
    x = _features(R, 11)
    t = np.random.default_rng(12).normal(size=R).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = torch.empty(R, device="cuda")
    h1 = torch.empty(R, 128, dtype=torch.int16, device="cuda")
    h2 = torch.empty(R, 128, dtype=torch.int16, device="cuda")
    B.mlp_forward(mlp.net(), xd, y, h1, h2)
    if tc:
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        B.mlp_backward_tc(mlp.net(), xd, h1, h2, y, td, mlp.grads, mlp.loss, status=status)
        assert int(status.item()) == 0
    else:
        B.mlp_backward(mlp.net(), xd, h1, h2, y, td, mlp.grads, mlp.loss)
    loss, gw = orc.mlp_backward(x, t, mlp.weights_fp(), bf16=True)
    # measured on GB300: loss within 2.5e-6, gradients within 4.1e-5 (2048 rows); bounds with a factor of 5
    assert float(mlp.loss.item()) == pytest.approx(loss, rel=2e-5)
    g = mlp.grads.double().cpu().numpy()
    sl = mlp._slices()
    print(f"mlp backward R={R} tc={tc}: loss rel {abs(float(mlp.loss.item()) - loss) / abs(loss):.3e}, " +
          ", ".join(f"{k} {rel_l2(g[sl[k]], gw[k].reshape(-1)):.3e}" for k in ("W1", "b1", "W2", "b2", "W3", "b3")))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert rel_l2(g[sl[name]], gw[name].reshape(-1)) <= 2e-4, (name, rel_l2(g[sl[name]], gw[name].reshape(-1)))


@pytest.mark.parametrize("R,R_dev", [(33, None), (130, None), (2048, None), (5000, None), (5000, 4321)])
def test_train_pass_parity(P, orc, R, R_dev):
    """The training pass with the forward recomputed in the same tcgen05 kernel
    (no stored activations): loss, gradients and outputs against the oracle,
    the last 128-row tile ragged; R_dev: only the first rows count."""
    B, TileErrorMLP = P
    mlp = TileErrorMLP(seed=7)
    x = _features(R, 11)
    t = np.random.default_rng(12).normal(size=R).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = torch.full((R,), float("nan"), device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rd = None if R_dev is None else torch.tensor([R_dev], dtype=torch.int32, device="cuda")
    B.mlp_train_tc(mlp.net(), xd, td, mlp.grads, mlp.loss, y=y, status=status, rows_dev=rd)
    assert int(status.item()) == 0
    Re = R if R_dev is None else R_dev
    loss, gw = orc.mlp_backward(x[:Re], t[:Re], mlp.weights_fp(), bf16=True)
    yw = orc.mlp_forward(x, mlp.weights_fp(), bf16=True)[0]
    got = y.cpu().numpy()
    # fp32 (tensor memory) against fp64 sums may move an h1 or h2 value across a
    # bf16 rounding; measured on GB300: 1.15e-4 at 2048 rows of this seed
    assert rel_l2(got, yw) <= 3e-4
    # one such flip moves y by about 2^-8 |h| |w3|: a few rows only
    assert np.mean(np.abs(got - yw) > 1e-3 * max(1.0, np.abs(yw).max())) <= 0.005
    # the forward kernel's own outputs: the same products, only the order of the
    # sum over the hidden units differs
    y_f = torch.empty(R, device="cuda")
    B.mlp_forward_tc(mlp.net(), xd, y_f, status=status)
    assert rel_l2(got, y_f.cpu().numpy()) <= 1e-6
    assert float(mlp.loss.item()) == pytest.approx(loss, rel=2e-5)
    g = mlp.grads.double().cpu().numpy()
    sl = mlp._slices()
    print(f"mlp train pass R={R}: loss rel {abs(float(mlp.loss.item()) - loss) / abs(loss):.3e}, " +
          ", ".join(f"{k} {rel_l2(g[sl[k]], gw[k].reshape(-1)):.3e}" for k in ("W1", "b1", "W2", "b2", "W3", "b3")))
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        assert rel_l2(g[sl[name]], gw[name].reshape(-1)) <= 2e-4, (name, rel_l2(g[sl[name]], gw[name].reshape(-1)))


def test_adam_step_and_training(P):
    B, TileErrorMLP = P
    mlp = TileErrorMLP(seed=3, lr=2e-3)
    p0 = mlp.params.clone()
    R = 4096
    x = torch.from_numpy(_features(R, 5)).cuda()
    # a smooth seeded target of the five features
    t = torch.tanh(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 3] ** 2 + 0.1 * x[:, 4]
    l0 = float(mlp.train_step(x, t).item())
    # first Adam step from zero moments moves every parameter with a non-zero gradient by ~lr
    d = (mlp.params - p0).abs()
    nz = mlp.grads.abs() > 1e-5
    assert torch.allclose(d[nz], torch.full_like(d[nz], 2e-3), rtol=1e-3)
    for _ in range(600):
        l = mlp.train_step(x, t)
    l1 = float(l.item())
    assert l1 < 0.1 * l0, (l0, l1)


def test_tc_wait_timeout_drill(P):
    """The tcgen05 kernel's bounded wait, made to run out on an mbarrier phase
    that nothing completes: the kernel records status 1, frees its tensor
    memory and returns, and the context stays usable (a forward right after
    succeeds with status 0 and matches the mma.sync forward)."""
    B, TileErrorMLP = P
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.mlp_tc_wait_drill(status)
    torch.cuda.synchronize()
    assert int(status.item()) == 1
    mlp = TileErrorMLP(seed=3)
    xd = torch.from_numpy(_features(300, 3)).cuda()
    y = torch.empty(300, device="cuda")
    y_ref = torch.empty(300, device="cuda")
    st2 = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.mlp_forward_tc(mlp.net(), xd, y, status=st2)
    B.mlp_forward(mlp.net(), xd, y_ref)
    torch.cuda.synchronize()
    assert int(st2.item()) == 0
    assert rel_l2(y.cpu().numpy(), y_ref.cpu().numpy()) <= 1e-3
