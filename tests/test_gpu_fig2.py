"""Fig. 2's accuracy study through the GPU path (Sec. V): on the switching window of an
inverter chain, the kernels' ER at 0.1 ps and ER-C at 0.2 ps (ers_step, Krylov dimension from
the Eq.-16 test at eps 1e-12, gamma = 0.1) against REF = the oracle's BENR at 0.01 ps on the
most-swinging inverter output.  The paper's two claims must hold for the GPU results: ER is
more accurate than BENR at equal step, and ER-C at twice the step still is.  The GPU
trajectories also follow the oracle's ER and ER-C trajectories point by point."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

from oracle import ers_oracle as O  # noqa: E402

pytestmark = pytest.mark.gpu

GRID = 0.2e-12


@pytest.fixture(scope="module")
def ers():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers as E
    return E


def gpu_trajectory(E, circ, x0, t0, t1, h, correction):
    sim = E.Simulator.from_circuit(
        circ, opts=E.make_opts(eps_krylov=1e-12, m_max=circ.n, correction=int(correction)))
    sim.set_state(t0, x0)
    out = []
    per = int(round(GRID / h))
    for k in range(int(round((t1 - t0) / h))):
        sim.step(h, 0)
        if (k + 1) % per == 0:
            out.append(sim.state()[1])
    sim.close()
    return np.array(out)


def test_fig2_orderings_hold_on_the_gpu(ers):
    from fig2_study import be_step, er_step, trajectory
    from test_oracle_pins import _switching_window
    circ, x0, t0, t1 = _switching_window()
    ref_be = trajectory(be_step, circ, x0, t0, t1, 0.01e-12, GRID)           # REF
    be = trajectory(be_step, circ, x0, t0, t1, 0.1e-12, GRID)
    or_er = trajectory(er_step, circ, x0, t0, t1, 0.1e-12, GRID)
    or_erc = trajectory(lambda c, x, t, h: er_step(c, x, t, h, True), circ, x0, t0, t1,
                        0.2e-12, GRID)
    g_er = gpu_trajectory(ers, circ, x0, t0, t1, 0.1e-12, False)
    g_erc = gpu_trajectory(ers, circ, x0, t0, t1, 0.2e-12, True)
    drains = np.unique(circ.dev["d"][circ.dev["d"] >= 0])
    node = int(drains[np.argmax(np.ptp(ref_be[:, drains], axis=0))])
    err = lambda v: float(np.max(np.abs(v[:, node] - ref_be[:, node])))   # noqa: E731
    assert err(g_er) < err(be) / 4, (err(g_er), err(be))
    assert err(g_erc) < err(be), (err(g_erc), err(be))
    # the kernels follow the oracle's trajectories (per node, every grid point)
    for g, o in ((g_er, or_er), (g_erc, or_erc)):
        scale = np.maximum(np.abs(o), 1e-3 * np.max(np.abs(o)) + 1e-300)
        assert np.max(np.abs(g - o) / scale) <= 1e-9
