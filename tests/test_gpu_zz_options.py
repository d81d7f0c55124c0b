"""GPU parity of creation options that change the matrices: gmin added by the library equals
the oracle run on G + gmin I (one ER step of a linear circuit, per node at the 1e-9 bar)."""
import numpy as np
import pytest
import scipy.sparse as sp

from synth import circuits as S
from oracle import ers_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ers():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers as E
    return E


def test_library_gmin_equals_oracle_with_stamped_gmin(ers):
    circ = S.random_rc(n=40, seed=6)
    gmin = 2e-4
    stamped = S.Circuit(name=circ.name, n=circ.n, G=(circ.G + gmin * sp.eye(circ.n)).tocsr(),
                        C=circ.C, B=circ.B, dev=circ.dev, pwl=circ.pwl, t_end=circ.t_end,
                        meta=circ.meta)
    sim = ers.Simulator.from_circuit(circ, opts=ers.make_opts(gmin=gmin))
    x = np.random.default_rng(6).normal(size=circ.n) * 0.1
    t, h = 6e-12, 1e-12
    ref = O.er_step(stamped, x, t, h, m=0)
    sim.set_state(t, x)
    mu, _ = sim.step(h, 0)
    _, xg, _ = sim.state()
    scale = np.maximum(np.abs(ref.x), 1e-3 * np.max(np.abs(ref.x)))
    assert mu == ref.m1
    assert np.max(np.abs(xg - ref.x) / scale) <= 1e-9
    sim.close()
