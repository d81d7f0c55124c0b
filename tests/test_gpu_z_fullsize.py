"""GPU parity at the full sizes of the two single-circuit benchmark workloads, in the launch
configuration bench.py times: the context is created with the bench's options, the DC point
is solved, and the solve kernels run with the resident CTAs per SM that ers_autotune picks.

* 3D RC power grid 100 x 100 x 100 (1 M nodes; 10.6 GB of factor): the oracle cannot factor
  it in seconds, so the check is a property that holds at any size, the normwise backward
  error of the supernodal solve of G x = b (a backward-stable LU leaves it at FP64 rounding
  level; a wrong block, a missed update or a race leaves it O(1)).
* Inverter chain, 2000 stages x 100-node trees (200 k nodes): the oracle runs at this size.
  DC from the logic-level nodeset against the oracle's Newton from the same guess, and one
  adaptive ER step on the input edge (Eq. 13, Krylov dimension from Eq. 16, error estimate of
  Eq. 15) against the oracle's step from the same state, per node at the 1e-9 bar."""
import numpy as np
import pytest

from synth import circuits as S
from oracle import ers_oracle as O

pytestmark = pytest.mark.gpu

REL = 1e-9


@pytest.fixture(scope="module")
def ers():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers as E
    return E


def bench_context(E, circ, t_end, nodeset=None):
    """The context as bench.py builds it: eps 1e-7, h_max = t_end / 100, DC, autotuned solves."""
    sim = E.Simulator.from_circuit(circ, opts=E.make_opts(eps_krylov=1e-7, h_max=t_end / 100))
    sim.dc(nodeset)
    sim.autotune(nrhs=2, passes=3)
    return sim


def test_mesh_100_cubed_solve_backward_error(ers):
    circ = S.rc_mesh_3d(100, 100, 100, seed=1, n_loads=10000)
    sim = bench_context(ers, circ, 2e-9)
    G = circ.G.tocsr()
    g_inf = float(abs(G).sum(axis=1).max())
    rng = np.random.default_rng(0)
    loads = circ.B @ np.full(circ.p, 1e-3)                 # every load drawing 1 mA
    for b in (rng.normal(size=circ.n), loads):
        x = sim.solve(b)
        assert np.all(np.isfinite(x))
        eta = np.max(np.abs(G @ x - b)) / (g_inf * np.max(np.abs(x)) + np.max(np.abs(b)))
        assert eta <= 1e-11, eta
    sim.close()


@pytest.fixture(scope="module")
def chain():
    circ = S.inverter_chain(stages=2000, tree_nodes=100, seed=2, t_end=5e-9)
    return circ, O.dc_solution(circ, x0=circ.nodeset)


def node_close(x, ref, rel=REL):
    scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)) + 1e-300)
    err = np.abs(x - ref) / scale
    return bool(np.all(err <= rel)), float(np.max(err))


def test_chain_2000_dc_matches_oracle(ers, chain):
    circ, xr = chain
    sim = bench_context(ers, circ, circ.t_end, circ.nodeset)
    _, xg, _ = sim.state()
    assert np.max(np.abs(xg - xr)) <= 1e-9
    sim.close()


def test_chain_2000_er_step_matches_oracle(ers, chain):
    circ, x0 = chain
    t, h = 0.105e-9, 1e-12                                 # on the input's rising edge
    sim = bench_context(ers, circ, circ.t_end, circ.nodeset)
    ref = O.er_step(circ, x0, t, h, m=0)
    sim.set_state(t, x0)
    mu, err = sim.step(h, 0)
    _, xg, _ = sim.state()
    assert mu == ref.m1
    ok, worst = node_close(xg, ref.x)
    assert ok, worst
    assert abs(err - ref.err_inf) <= 1e-6 * ref.err_inf + 1e-15, (err, ref.err_inf)
    sim.close()
