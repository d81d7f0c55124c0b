"""Batched contexts (many circuits in one context) through the C ABI, against the oracle run
instance by instance: every instance follows Algorithm 2 on its own, so its final state must
agree with the oracle's adaptive run within the run tolerance and its accepted-step count
within a few percent."""
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


def test_batch_matches_per_instance_oracle(ers):
    t_end = 0.15e-9
    circs = [S.inverter_chain(stages=st, tree_nodes=tn, seed=sd, t_end=t_end, sigma=0.05)
             for st, tn, sd in ((3, 10, 101), (5, 8, 102), (2, 20, 103), (4, 6, 104))]
    sim = ers.BatchSimulator(circs)
    x0 = np.concatenate([O.dc_solution(c) for c in circs])
    sim.set_state(0.0, x0)
    ns, nr = sim.run_batch(t_end, 1e-6)
    for k, c in enumerate(circs):
        t, xg, _ = sim.state_inst(k)
        xr, tr, st = O.er_run(c, t_end=t_end, tol=1e-6)
        assert abs(t - t_end) < 1e-20
        assert abs(int(ns[k]) - st.steps) <= max(2, 0.05 * st.steps), (k, ns[k], st.steps)
        assert np.max(np.abs(xg - xr)) <= 2e-6 * max(1.0, np.max(np.abs(xr))), k
    sim.close()


def test_batch_of_linear_meshes_matches_single_contexts(ers):
    """Linear instances: a batch step equals each instance's own step (same h, same m)."""
    t_end = 60e-12
    circs = [S.rc_mesh_2d(8, 8, seed=s, t_end=t_end) for s in (1, 2, 3)]
    sim = ers.BatchSimulator(circs, opts=ers.make_opts(h_max=4e-12))
    sim.set_state(0.0, np.zeros(sim.n))
    ns, _ = sim.run_batch(t_end, 1e-6)
    for k, c in enumerate(circs):
        single = ers.Simulator.from_circuit(c, opts=ers.make_opts(h_max=4e-12))
        single.set_state(0.0, np.zeros(c.n))
        n1, _ = single.run(t_end, 1e-6)
        _, x1, _ = single.state()
        _, xb, _ = sim.state_inst(k)
        assert n1 == ns[k]
        scale = np.maximum(np.abs(x1), 1e-3 * np.max(np.abs(x1)) + 1e-300)
        assert np.max(np.abs(xb - x1) / scale) <= 1e-9
        single.close()
    sim.close()
