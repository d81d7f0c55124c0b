"""CPU pins of the learned controller's oracle (network forward/backward/Adam in FP64 and the
step-history featurisation), and the library's host-side featurisation against it.

The oracle is pinned to things other than itself: PyTorch's own float64 layers, autograd and
Adam (an independent implementation), central finite differences, and values worked out by
hand from the feature definitions."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as MO

torch = pytest.importorskip("torch")


def rand_params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    parts = []
    for name, shp in MO.SHAPES:
        fan_in = shp[1] if len(shp) == 2 else 64
        if name.startswith("W"):
            parts.append(rng.normal(0, scale * math.sqrt(2.0 / fan_in), size=shp).ravel())
        else:
            parts.append(rng.normal(0, 0.1, size=shp))
    p = np.concatenate(parts)
    assert p.size == MO.NPARAM == 10562
    return p


def torch_net(p):
    P = MO.unpack(p)
    layers = []
    for k in range(1, 5):
        W = torch.tensor(P[f"W{k}"], dtype=torch.float64, requires_grad=True)
        b = torch.tensor(P[f"b{k}"], dtype=torch.float64, requires_grad=True)
        layers += [W, b]
    return layers


def torch_forward(layers, X):
    h = torch.tensor(X, dtype=torch.float64)
    for k in range(3):
        h = torch.relu(torch.nn.functional.linear(h, layers[2 * k], layers[2 * k + 1]))
    return torch.nn.functional.linear(h, layers[6], layers[7])


def data(n=100, seed=1):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 32)), rng.normal(size=(n, 2))


def test_forward_matches_torch_layers():
    p = rand_params()
    X, _ = data()
    Y, _ = MO.forward(p, X)
    Yt = torch_forward(torch_net(p), X).detach().numpy()
    np.testing.assert_allclose(Y, Yt, rtol=1e-12, atol=1e-12)


def test_gradient_matches_autograd():
    p = rand_params(3)
    X, T = data(77, 4)
    L, g = MO.loss_and_grad(p, X, T)
    layers = torch_net(p)
    Y = torch_forward(layers, X)
    Lt = ((Y - torch.tensor(T)) ** 2).sum() / X.shape[0]
    Lt.backward()
    gt = np.concatenate([t.grad.numpy().ravel() for t in layers])
    assert abs(L - Lt.item()) <= 1e-12 * abs(L)
    np.testing.assert_allclose(g, gt, rtol=1e-10, atol=1e-13)


def test_gradient_matches_finite_differences():
    p = rand_params(5)
    X, T = data(40, 6)
    _, g = MO.loss_and_grad(p, X, T)
    rng = np.random.default_rng(7)
    for _ in range(6):
        d = rng.normal(size=p.size)
        d /= np.linalg.norm(d)
        eps = 1e-6
        Lp, _ = MO.loss_and_grad(p + eps * d, X, T)
        Lm, _ = MO.loss_and_grad(p - eps * d, X, T)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ d)
    # per-block directions: a gradient error confined to one tensor (a dropped gate, a
    # transposed product) would hide in a random global direction's average
    o = 0
    for name, shp in MO.SHAPES:
        k = int(np.prod(shp))
        d = np.zeros(p.size)
        d[o:o + k] = rng.normal(size=k)
        d /= np.linalg.norm(d)
        Lp, _ = MO.loss_and_grad(p + 1e-6 * d, X, T)
        Lm, _ = MO.loss_and_grad(p - 1e-6 * d, X, T)
        fd = (Lp - Lm) / 2e-6
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (name, fd, g @ d)
        o += k


def test_adam_matches_torch_optimizer():
    p = rand_params(8)
    X, T = data(64, 9)
    layers = torch_net(p)
    opt = torch.optim.Adam(layers, lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    q = p.copy()
    m = np.zeros_like(q)
    v = np.zeros_like(q)
    for t in range(1, 4):
        opt.zero_grad()
        Y = torch_forward(layers, X)
        ((Y - torch.tensor(T)) ** 2).sum().div(X.shape[0]).backward()
        opt.step()
        _, g = MO.loss_and_grad(q, X, T)
        q, m, v = MO.adam(q, g, m, v, t, 1e-2)
    qt = np.concatenate([t.detach().numpy().ravel() for t in layers])
    np.testing.assert_allclose(q, qt, rtol=1e-9, atol=1e-12)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(11)
    a = np.concatenate([rng.normal(size=4000).astype(np.float32),
                        np.array([0.0, -0.0, 1.0, 1.00390625, 1.01171875, -3.0e-5], np.float32)])
    ours = MO.bf16_round(a)
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


def rec(h=1e-12, h_max=1e-10, err=1e-8, E=1e-6, dF=1e-6, m=20, m_max=40, landed=0, retries=0):
    return dict(h=h, h_max=h_max, err=err, E=E, dF=dF, m=m, m_max=m_max, landed=landed,
                retries=retries)


def test_features_by_hand():
    # h/h_max = 1e-2 -> -2/3 ; m/m_max = 1/2 ; err/E = 1e-2 -> -2/3 ; dF = 1e-6 -> 0
    f = MO.features([rec()])
    assert np.allclose(f.reshape(8, 4), [[-2 / 3, 0.5, -2 / 3, 0.0]] * 8)
    # clamps: h = h_max -> 0 ; err = 0 -> -2 ; err/E = 100 -> 1/3 ; dF = 0 -> -1 ; dF = 10 -> 1
    f = MO.features([rec(h=1e-10, err=0.0, dF=0.0), rec(h=1e-20, err=1e-4, dF=10.0, m=40)])
    assert np.allclose(f[:4], [-2.0, 1.0, 1 / 3, 1.0])   # latest: h/h_max=1e-10 clamps to -6
    assert np.allclose(f[4:8], [0.0, 0.5, -2.0, -1.0])
    assert np.allclose(f[8:], np.tile(f[4:8], 6))       # older slots repeat the oldest


def test_target_by_hand():
    hist = [rec(h=1e-12)]
    # next accepted at 2h with err = E/4: headroom 0.8 * 2 = 1.6 -> log2(2) + log2(1.6)
    t = MO.target(hist, rec(h=2e-12, err=0.25e-6, m=30))
    assert np.allclose(t, [1 + math.log2(1.6), 0.75])
    # err close to E: no headroom; h halved -> -1
    t = MO.target(hist, rec(h=0.5e-12, err=0.9e-6))
    assert np.allclose(t, [-1.0, 0.5])
    # clamp at +2 and the landed exclusion
    assert np.allclose(MO.target(hist, rec(h=8e-12, err=0.0))[0], 2.0)
    assert MO.target(hist, rec(h=2e-12, landed=1)) is None


@pytest.fixture(scope="module")
def E():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers
    return ers


def random_records(rng, k):
    out = []
    for _ in range(k):
        out.append(rec(h=10 ** rng.uniform(-16, -9), h_max=10 ** rng.uniform(-11, -9),
                       err=float(rng.choice([0.0, 10 ** rng.uniform(-12, -4)])), E=1e-6,
                       dF=float(rng.choice([0.0, 10 ** rng.uniform(-14, 1)])),
                       m=int(rng.integers(1, 41)), m_max=40, landed=int(rng.integers(0, 2)),
                       retries=int(rng.integers(0, 3))))
    return out


def test_library_features_match_oracle(E):
    rng = np.random.default_rng(21)
    for trial in range(200):
        R = random_records(rng, int(rng.integers(1, 12)))
        ours = E.ctrl_features(R)
        ref = MO.features(R).astype(np.float32)
        np.testing.assert_allclose(ours, ref, rtol=0, atol=2e-7)


def test_library_targets_match_oracle(E):
    rng = np.random.default_rng(22)
    for trial in range(200):
        R = random_records(rng, int(rng.integers(1, 6)))
        nxt = random_records(rng, 1)[0]
        ours = E.ctrl_target(R, nxt)
        ref = MO.target(R, nxt)
        if ref is None:
            assert ours is None
        else:
            np.testing.assert_allclose(ours, ref.astype(np.float32), rtol=0, atol=2e-7)


def test_library_proposal_rule_by_hand(E):
    import math
    last = rec(h=1e-12, h_max=1e-10, err=0.25e-6, E=1e-6, m=10, m_max=40)
    # r* = 2 (log2 1): band [0, 2]; y0 = 0.5, no margin -> 2^0.5 h
    h, m = E.ctrl_propose([0.5, 0.25], last)
    assert h == pytest.approx(math.sqrt(2) * 1e-12, rel=1e-12) and m == 9
    # a shrink request after an easy step is held at h (lower band edge 0)
    h, _ = E.ctrl_propose([-2.0, 0.25], last)
    assert h == pytest.approx(1e-12, rel=1e-12)
    # margin shifts the request: 0.5 - 0.3
    h, _ = E.ctrl_propose([0.5, 0.25], last, margin=0.3)
    assert h == pytest.approx(2 ** 0.2 * 1e-12, rel=1e-12)
    # near the budget (err/E = 0.9): upper edge r* + 1
    hi = 1 - 0.5 * math.log2(0.9)
    h, _ = E.ctrl_propose([2.0, 0.25], rec(h=1e-12, h_max=1e-10, err=0.9e-6, E=1e-6, m_max=40))
    assert h == pytest.approx(2 ** hi * 1e-12, rel=1e-12)
    # err = 0 (linear circuit): r* capped at 2^6, so the network's 4x stands; h_max caps
    h, _ = E.ctrl_propose([2.0, 0.25], rec(h=4e-11, h_max=1e-10, err=0.0, E=1e-6, m_max=40))
    assert h == pytest.approx(1e-10, rel=1e-12)
    # m_start: round(y1 m_max) - 1 clamped to [m_min, m_max]; non-finite -> m_min
    assert E.ctrl_propose([0.0, 0.99], last)[1] == 39
    assert E.ctrl_propose([0.0, 0.0], last)[1] == 3
    h, m = E.ctrl_propose([float("nan"), float("nan")], last)
    assert m == 3 and h == pytest.approx(2e-12, rel=1e-12)   # non-finite y0: l = 1
