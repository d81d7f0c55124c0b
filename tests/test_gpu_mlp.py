"""The learned controller's network on the GPU (BF16 weights, BF16 tensor-core operands with
FP32 accumulation; activations and deltas carried as BF16 hi/lo pairs) against the FP64 oracle
evaluated on the same BF16-rounded weights, through the C ABI.

Tolerances: a hi/lo pair keeps about 16 significant bits (relative rounding <= 2^-17), sums are
FP32.  Through four layers the output error stays near 1e-5 relative; the gradient of the
first layer is a sum over samples with cancellation and the loss derivative (Y - T) can be
small, which amplifies the relative error by up to ~50 (measured on a CPU emulation of the
arithmetic), so gradients are compared per parameter tensor normwise at 5e-3 and outputs at
1e-3.  With plain BF16 activations the same comparison is off by 2-20 %, which is why the
kernels carry pairs.  Adam runs in FP32 on the same gradient the oracle is given, so its update
agrees to FP32 rounding."""
import numpy as np
import pytest

from oracle import mlp_oracle as MO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ers():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers as E
    return E


def rounded(p):
    """Weights rounded to BF16 as the kernels hold them; biases stay FP32."""
    q = np.asarray(p, np.float32).copy()
    o = 0
    for name, shp in MO.SHAPES:
        k = int(np.prod(shp))
        if name.startswith("W"):
            q[o:o + k] = MO.bf16_round(q[o:o + k])
        o += k
    return q.astype(np.float64)


def inputs(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 32)).astype(np.float32)
    T = np.stack([np.tanh(X[:, 0] + 0.5 * X[:, 1]), 0.5 / (1 + np.exp(-X[:, 2]))], 1)
    return X, T.astype(np.float32)


@pytest.mark.parametrize("n", [1, 64, 300])
def test_forward_matches_oracle(ers, n):
    M = ers.Mlp(seed=3)
    p = M.params()
    X, _ = inputs(n, 10 + n)
    Y = M.forward(X)
    Yr, _ = MO.forward(rounded(p), X.astype(np.float64))
    rms = np.sqrt(np.mean(Yr ** 2))
    assert np.linalg.norm(Y - Yr) <= 1e-3 * np.linalg.norm(Yr)
    assert np.max(np.abs(Y - Yr)) <= 3e-3 * rms
    M.close()


@pytest.mark.parametrize("n", [1, 64, 300])
def test_gradient_matches_oracle(ers, n):
    M = ers.Mlp(seed=4)
    p = M.params()
    X, T = inputs(n, 20 + n)
    g, L = M.grad(X, T)
    Lr, gr = MO.loss_and_grad(rounded(p), X.astype(np.float64), T.astype(np.float64))
    assert abs(L - Lr) <= 1e-3 * Lr
    o = 0
    for name, shp in MO.SHAPES:
        k = int(np.prod(shp))
        a, b = g[o:o + k], gr[o:o + k]
        assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b) + 1e-7, name
        o += k
    M.close()


def test_adam_steps_match_oracle(ers):
    M = ers.Mlp(seed=5)
    X, T = inputs(200, 30)
    p = M.params().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    lr = 1e-3
    for t in (1, 2, 3):
        g, _ = M.grad(X, T)            # deterministic: the step below recomputes the same one
        M.adam_step(X, T, lr)
        q = M.params().astype(np.float64)
        pr, m, v = MO.adam(p, g.astype(np.float64), m, v, t, lr)
        assert np.max(np.abs(q - pr) - (1e-6 * np.abs(p) + 1e-4 * lr)) <= 0, t
        p = q


def test_training_reduces_loss(ers):
    M = ers.Mlp(seed=6)
    X, T = inputs(4096, 40)
    _, L0 = M.grad(X, T)
    M.train(X, T, epochs=60, batch=256, lr=3e-3, seed=1)
    _, L1 = M.grad(X, T)
    assert L1 < 0.1 * L0, (L0, L1)
    # the trained network's loss agrees with the oracle's on its (rounded) weights
    Lr, _ = MO.loss_and_grad(rounded(M.params()), X.astype(np.float64), T.astype(np.float64))
    assert abs(L1 - Lr) <= 1e-3 * Lr + 1e-6
    M.close()


def test_deterministic_gradient(ers):
    M = ers.Mlp(seed=7)
    X, T = inputs(1000, 50)
    g1, L1 = M.grad(X, T)
    g2, L2 = M.grad(X, T)
    assert np.array_equal(g1, g2) and L1 == L2
    M.close()
