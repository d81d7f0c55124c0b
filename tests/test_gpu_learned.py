"""The learned (h, m) controller of batched runs, through the C ABI.

* m proposals change cost, never results: the proposed dimension only moves where the first
  residual test (Eq. 16) is taken, and the parallel test of the skipped dimensions picks the
  one the plain rule picks.  On instances small enough to be one supernode each the solves
  have no scatter between supernodes and the runs are deterministic: there every step takes
  the same dimension and the states are bit-identical.  On the inverter chains the solves
  scatter with FP64 atomics, whose order (and last-bit rounding) varies from run to run, so a
  residual within rounding of eps can flip between two plain runs as well; there the step
  counts must agree and the states to 1e-8.
* h proposals are judged by the error test (Eq. 15): a network that always asks for 4x steps
  still reaches t_end with the plain run's accuracy, its rejections falling back to h = alpha h.
* The training samples exported from plain-controller traces equal the oracle's featurisation
  of the same records.
* A network trained on plain traces of one set of circuits, run on held-out circuits of the
  same family, needs fewer rejected steps and fewer Krylov vectors than the plain controller at
  the same tolerance, and its error against a tight-tolerance run stays at the plain run's."""
import numpy as np
import pytest

from oracle import mlp_oracle as MO
from synth import circuits as S

pytestmark = pytest.mark.gpu

T_END = 0.3e-9


@pytest.fixture(scope="module")
def ers():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers as E
    return E


def family(n, seed0):
    return S.batch_family(n_inst=n, seed0=seed0, stage_lo=3, stage_hi=8, sigma=0.05,
                          t_end=T_END, tree_nodes=10)


def run(E, circs, mlp=None, parts=3, tol=1e-6, trace=False):
    sim = E.BatchSimulator(circs)
    sim.dc()
    if trace:
        sim.trace(True)
    if mlp is not None:
        sim.set_controller(mlp, parts)
    ns, nr = sim.run_batch(T_END, tol)
    xs = [sim.state_inst(k)[1] for k in range(len(circs))]
    out = dict(ns=ns, nr=nr, xs=xs, ctrl=sim.ctrl_stats(), sim=sim)
    return out


def constant_net(E, y0, y1):
    """A network whose output is (y0, y1) for every input: zero weights, output biases."""
    M = E.Mlp(seed=0)
    p = np.zeros(M.nparam, np.float32)
    p[-2:] = (y0, y1)
    M.set_params(p)
    return M


@pytest.fixture(scope="module")
def plain(ers):
    r = run(ers, family(6, 3000), trace=True)
    yield r
    r["sim"].close()


def run_linear(E, circs, t_end, mlp=None, parts=2):
    sim = E.BatchSimulator(circs, opts=E.make_opts(h_max=t_end / 50))
    sim.set_state(0.0, np.zeros(sim.n))
    sim.trace(True)
    if mlp is not None:
        sim.set_controller(mlp, parts)
    sim.run_batch(t_end, 1e-6)
    recs = [[(r["m"], r["h"]) for r in sim.records(k)] for k in range(len(circs))]
    xs = [sim.state_inst(k)[1] for k in range(len(circs))]
    st = sim.stats()
    sim.close()
    return recs, xs, st


@pytest.mark.parametrize("y1", [0.2, 0.3, 0.9])
def test_m_proposals_exact_on_single_supernode_instances(ers, y1):
    t_end = 50e-12
    # complete-graph RC networks of 32 nodes: each factors as one dense supernode
    circs = [S.random_rc(n=32, seed=s, density=1.0, t_end=t_end) for s in range(8)]
    r0, x0, st0 = run_linear(ers, circs, t_end)
    assert st0["nsn"] == len(circs)    # one supernode per instance: no scatter, deterministic
    r1, x1, _ = run_linear(ers, circs, t_end)
    assert r1 == r0 and all(np.array_equal(a, b) for a, b in zip(x1, x0))
    ms = {m for R in r0 for m, _ in R}
    assert len(ms) > 1                 # the plain rule's dimension varies over the run
    M = constant_net(ers, 1.0, y1)     # first decision at 7, 11 or 35 (past breakdown)
    r2, x2, _ = run_linear(ers, circs, t_end, M)
    assert r2 == r0
    assert all(np.array_equal(a, b) for a, b in zip(x2, x0))


@pytest.mark.parametrize("y1", [0.9, 0.2])
def test_m_proposals_keep_the_plain_steps(ers, plain, y1):
    # y1 = 0.9 -> first decision at dimension 35 (overshoot); 0.2 -> 7 (around plain's m)
    M = constant_net(ers, 1.0, y1)
    r = run(ers, family(6, 3000), M, parts=2)
    assert abs(int(r["ns"].sum()) - int(plain["ns"].sum())) <= 0.01 * plain["ns"].sum()
    for a, b in zip(r["xs"], plain["xs"]):
        assert np.max(np.abs(a - b)) <= 1e-8
    r["sim"].close()


def test_bad_step_proposals_fall_back_to_plain_rule(ers, plain):
    M = constant_net(ers, 2.0, 0.2)   # always ask for 4 h
    r = run(ers, family(6, 3000), M, parts=1)
    assert r["ctrl"]["proposals"] > 0 and r["ctrl"]["rejected"] > 0
    for k, (a, b) in enumerate(zip(r["xs"], plain["xs"])):
        assert r["sim"].state_inst(k)[0] == pytest.approx(T_END, rel=1e-12)
        assert np.max(np.abs(a - b)) <= 2e-5, k
    r["sim"].close()


def test_samples_match_oracle_featurisation(ers, plain):
    sim = plain["sim"]
    traces = [sim.records(k) for k in range(6)]
    assert all(len(R) == int(n) for R, n in zip(traces, plain["ns"]))
    X, T = sim.samples()
    Xr, Tr = MO.samples(traces)
    assert X.shape == Xr.shape and X.shape[0] > 100
    np.testing.assert_allclose(X, Xr.astype(np.float32), rtol=0, atol=2e-7)
    np.testing.assert_allclose(T, Tr.astype(np.float32), rtol=0, atol=2e-7)


def test_trained_controller_gains_on_held_out_circuits(ers, plain):
    X, T = plain["sim"].samples()
    train = run(ers, family(10, 2000), trace=True)
    X2, T2 = train["sim"].samples()
    train["sim"].close()
    X = np.concatenate([X, X2])
    T = np.concatenate([T, T2])
    M = ers.Mlp(seed=1)
    _, L0 = M.grad(X, T)
    M.train(X, T, epochs=150, batch=256, lr=2e-3, seed=1)
    _, L1 = M.grad(X, T)
    assert L1 < 0.3 * L0
    held = family(8, 5000)
    p = run(ers, held)
    lr = run(ers, held, M, parts=3)
    ref = run(ers, held, tol=1e-8)
    # fewer rejected trials and less Krylov work at the same tolerance
    assert lr["nr"].sum() < 0.5 * p["nr"].sum(), (lr["nr"].sum(), p["nr"].sum())
    assert lr["ctrl"]["krylov_vectors"] < p["ctrl"]["krylov_vectors"]
    # same accuracy: error against the tight run no larger than a few times the plain run's
    ep = max(np.max(np.abs(a - b)) for a, b in zip(p["xs"], ref["xs"]))
    el = max(np.max(np.abs(a - b)) for a, b in zip(lr["xs"], ref["xs"]))
    assert el <= 3 * ep + 1e-6, (el, ep)
    for r in (p, lr, ref):
        r["sim"].close()
