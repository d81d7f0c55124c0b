"""Singular C on the GPU path (Sec. IV-A: C is never inverted or regularised; Sec. V: the
paper's test circuits all have singular C).  Capacitor-free nodes give J^-1 = -G^-1 C the
eigenvalue 0, so H_m of Eq. 14 is singular; the small dense stage deflates every eigenvalue
|mu| <= h/700 of H_m to -h/800 (where e^{h/mu} is 0 in FP64) by a rank-one Wielandt update
before the Pade stage, the limit from the stable side that the oracle takes with an ordered
Schur form.  Checked through the C ABI against the oracle and against exact solutions."""
import numpy as np
import pytest

from synth import circuits as S
from oracle import ers_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ers():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers as E
    return E


def _pins():
    import importlib, os, sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    return importlib.import_module("test_oracle_pins")


def node_close(x, ref, rel):
    scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)) + 1e-300)
    err = np.abs(x - ref) / scale
    return bool(np.all(err <= rel)), float(np.max(err))


def _planted(mus, seed):
    """Upper Hessenberg H with the eigenvalues mus (H = P^T Q D Q^-1 P from a Hessenberg
    reduction) and f(H) e_1 = (P^T Q) f(D) (P^T Q)^-1 e_1 in FP64, with f(0) = 0 (the limit
    from the stable side); the oracle's pins check the same cases in 50-digit arithmetic."""
    import scipy.linalg as sla
    m = len(mus)
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(m, m)) + 3 * np.eye(m)
    H, P = sla.hessenberg(Q @ np.diag(mus) @ np.linalg.inv(Q), calc_q=True)
    V = P.T @ Q
    c = np.linalg.solve(V, np.eye(m)[:, 0])

    def apply(fun):
        return V @ (np.array([fun(mu) if mu != 0 else 0.0 for mu in mus]) * c)
    return H, apply


@pytest.mark.parametrize("case", ["stiff", "zero", "zero_pair"])
def test_phi_small_deflates_near_null_eigenvalues(ers, case):
    """exp(h H^-1) e_1 and e_m^T H^-1 exp(h H^-1) e_1 of the kernel for planted spectra with
    stiff, zero and double-zero eigenvalues (the oracle's pin cases), against the oracle's
    Schur-split evaluation and an evaluation from the eigendecomposition."""
    h = 1e-12
    base = [-3e-12, -1e-12, -5e-13, -2e-13, -8e-14, -3e-14]
    extra = {"stiff": [-h / 2000, -h / 1e6], "zero": [0.0], "zero_pair": [0.0, 0.0]}[case]
    H, apply = _planted(base + extra, seed=len(extra))
    m = H.shape[0]
    with np.errstate(under="ignore"):
        ref_y = apply(lambda mu: np.exp(h / mu))
        ref_g = apply(lambda mu: np.exp(h / mu) / mu)
    circ = S.random_rc(n=12, seed=3, p=2, n_alg=2)          # a context with singular C
    sim = ers.Simulator.from_circuit(circ)
    y, last = sim.phi_small(H, h)
    yo, lo = O.exp_hinv_e1(H, h, singular_c=True)
    # the oracle's Schur split and the kernel's deflation are each within 1e-12 of the
    # 50-digit values (the oracle's pins, and the FP64 eigen-evaluation below), so the two
    # differ by up to 2e-12
    assert np.max(np.abs(y - yo)) <= 3e-12 * np.max(np.abs(yo)), case
    assert abs(last - lo) <= 3e-12 * np.max(np.abs(ref_g)), case
    assert np.max(np.abs(y - ref_y)) <= 1e-11 * np.max(np.abs(ref_y)), case
    assert abs(last - ref_g[m - 1]) <= 1e-11 * np.max(np.abs(ref_g)), case
    sim.close()


@pytest.mark.parametrize("seed,alg_source", [(0, False), (1, True), (2, False)])
def test_singular_c_step_matches_oracle_and_exact_solution(ers, seed, alg_source):
    """ER steps (Eq. 13) with a full invert-Krylov space from an inconsistent random state on
    circuits with four capacitor-free nodes: per node against the oracle at the 1e-9 bar, and
    against the exact solution of the differential-algebraic system (Kron reduction)."""
    T = _pins()
    circ = S.random_rc(n=14, seed=seed, p=3, n_alg=4, alg_source=alg_source, t_end=30e-12)
    x = np.random.default_rng(seed).normal(size=circ.n) * 0.1
    sim = ers.Simulator.from_circuit(circ, opts=ers.make_opts(m_max=circ.n))
    for t, h in [(0.0, 1e-12), (6e-12, 1e-12), (9e-12, 3e-12)]:
        nb = circ.breakpoints()
        nb = nb[nb > t + 1e-18]
        h = min(h, nb[0] - t) if nb.size else h
        ref = O.er_step(circ, x, t, h, m=circ.n)
        sim.set_state(t, x)
        sim.step(h, circ.n)
        _, xg, _ = sim.state()
        ok, worst = node_close(xg, ref.x, 1e-9)
        assert ok, (t, h, worst)
        ex = T.kron_exact_step(circ, x, t, h)
        assert np.max(np.abs(xg - ex)) <= 1e-10 * np.max(np.abs(ex)), (t, h)
    sim.close()


def test_singular_c_trajectory_keeps_algebraic_kcl(ers):
    """A trajectory through every source corner with the Krylov dimension from Eq. 16, from an
    inconsistent state: it follows the oracle's trajectory and the exact solution, and the
    capacitor-free rows of KCL, (G x)_a = (B u)_a, hold from the first step on."""
    T = _pins()
    circ = S.random_rc(n=16, seed=5, p=3, n_alg=5, alg_source=True, t_end=30e-12)
    alg = circ.meta["algebraic"]
    G = circ.G.toarray()
    B = circ.B.toarray()
    x = np.random.default_rng(5).normal(size=circ.n) * 0.1
    xo, xe = x.copy(), x.copy()
    opts = O.Options(eps=1e-12, m_max=circ.n)
    sim = ers.Simulator.from_circuit(circ, opts=ers.make_opts(eps_krylov=1e-12, m_max=circ.n))
    sim.set_state(0.0, x)
    for t, h in T._linear_pieces(circ, 2e-12):
        sim.step(h, 0)
        _, xg, _ = sim.state()
        xo = O.er_step(circ, xo, t, h, m=0, opts=opts).x
        xe = T.kron_exact_step(circ, xe, t, h)
        scale = np.max(np.abs(xe))
        assert np.max(np.abs(xg - xo)) <= 1e-8 * scale, t
        assert np.max(np.abs(xg - xe)) <= 1e-8 * scale, t
        kcl = (G @ xg)[alg] - (B @ circ.u(t + h))[alg]
        assert np.max(np.abs(kcl)) <= 1e-10 * np.max(np.abs(G)) * scale, t
    sim.close()
