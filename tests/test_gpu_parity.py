"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the same seeded
inputs.

Floating-point bar of an ER step: |x_gpu - x_or| <= 1e-9 * max(|x_or|, 1e-3 ||x_or||_inf) per
node.  It applies as written to the paper's algorithm (Krylov dimension from the Eq.-16
test) and to the 32x32 RC mesh at the config's fixed m = 20.  When a fixed m exceeds the
dimension at which the Krylov space has converged, the last directions are rounding noise of
the G_k solves and two correct FP64 implementations differ by as much as the algorithm's own
rounding sensitivity.  Those cases use the derived bar
    max(1e-9, s * cond(G_k) * eps / 1e-13),
    s = per-node change of the oracle's step when every one of its solves is perturbed by
        1e-13 relative noise (the change is linear in the noise level),
i.e. the oracle's sensitivity scaled to the size of the difference between two
backward-stable LU solves, cond(G_k) * eps."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


def node_close(x, ref, rel=REL):
    scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)) + 1e-300)
    bad = np.abs(x - ref) > rel * scale
    return not bad.any(), float(np.max(np.abs(x - ref) / scale))


def oracle_floor(circ, x, t, h, m, delta=1e-13, seeds=(1, 2, 3)):
    """Per-node sensitivity of the oracle's step to 1e-13 relative noise in its solves."""
    orig = O.Linearization.solve
    ref = O.er_step(circ, x, t, h, m=m).x
    worst = 0.0
    try:
        for sd in seeds:
            rng = np.random.default_rng(sd)

            def solve(self, b, rng=rng):
                y = orig(self, b)
                return y * (1 + delta * rng.normal(size=y.size))

            O.Linearization.solve = solve
            r1 = O.er_step(circ, x, t, h, m=m).x
            scale = np.maximum(np.abs(ref), 1e-3 * np.max(np.abs(ref)) + 1e-300)
            worst = max(worst, float(np.max(np.abs(r1 - ref) / scale)))
    finally:
        O.Linearization.solve = orig
    return worst


def make(E, circ, **kw):
    return E.Simulator.from_circuit(circ, opts=E.make_opts(**kw) if kw else None)


# --- stage tests -------------------------------------------------------------------------
@pytest.mark.parametrize("name,circ", [
    ("randrc", S.random_rc(n=40, seed=1)),
    ("rc2d", S.rc_mesh_2d(12, 9, seed=3)),
    ("rc3d", S.rc_mesh_3d(14, 13, 12, seed=2, n_loads=50)),     # several solve chunks
    ("inv", S.inverter_chain(stages=6, tree_nodes=30, seed=4)),
    # long chain of 100-node parasitic trees: most supernodes are solved by subtree tasks
    ("inv_trees", S.inverter_chain(stages=40, tree_nodes=100, seed=7)),
])
def test_solve_matches_sparse_lu(ers, name, circ):
    sim = make(ers, circ)
    x0 = O.dc_solution(circ) if circ.dev.size else np.zeros(circ.n)
    sim.set_state(0.0, x0)
    lin = O.linearize(circ, x0)
    rng = np.random.default_rng(0)
    G = lin.Gk.tocsr()
    g_inf = float(abs(G).sum(axis=1).max())
    for _ in range(3):
        b = rng.normal(size=circ.n)
        x = sim.solve(b)
        ref = lin.solve(b)
        # backward-stable LU: the normwise backward error (SuperLU and the oracle reach
        # 3e-17 .. 7e-17 on these families), and solutions within a cond-scaled bar
        eta = np.max(np.abs(G @ x - b)) / (g_inf * np.max(np.abs(x)) + np.max(np.abs(b)))
        assert eta <= 1e-14, eta
        assert np.max(np.abs(x - ref)) <= 1e-8 * np.max(np.abs(ref))
    sim.close()


def test_batch_solve_matches_per_instance_lu(ers):
    """Block-diagonal factor of many chains (subtree tasks in every instance)."""
    circs = [S.inverter_chain(stages=st, tree_nodes=50, seed=20 + st) for st in range(3, 23)]
    sim = ers.BatchSimulator(circs)
    x0 = np.concatenate([O.dc_solution(c) for c in circs])
    sim.set_state(0.0, x0)
    b = np.random.default_rng(3).normal(size=sim.n)
    x = sim.solve(b)
    o = 0
    for c in circs:
        lin = O.linearize(c, x0[o:o + c.n])
        ref = lin.solve(b[o:o + c.n])
        assert np.max(np.abs(x[o:o + c.n] - ref)) <= 1e-8 * np.max(np.abs(ref))
        o += c.n
    sim.close()


def test_autotuned_solves_match_sparse_lu(ers):
    """The autotuner times 1, 2 and 3 resident CTAs per SM and keeps one; solves stay exact."""
    circ = S.inverter_chain(stages=30, tree_nodes=40, seed=8)
    sim = make(ers, circ)
    x0 = O.dc_solution(circ, x0=circ.nodeset)
    sim.set_state(0.0, x0)
    chosen, ms = sim.autotune(nrhs=2, passes=3)
    assert chosen in (1, 2, 3) and all(t > 0 for t in ms)
    lin = O.linearize(circ, x0)
    b = np.random.default_rng(5).normal(size=circ.n)
    x = sim.solve(b)
    ref = lin.solve(b)
    assert np.max(np.abs(x - ref)) <= 1e-8 * np.max(np.abs(ref))
    sim.close()


def test_spmv_C(ers):
    circ = S.rc_mesh_2d(10, 10, seed=1)
    sim = make(ers, circ)
    v = np.random.default_rng(1).normal(size=circ.n)
    assert np.allclose(sim.spmv_C(v), circ.C @ v, rtol=1e-15, atol=0)
    sim.close()


def test_phi_small_matches_oracle(ers):
    circ = S.rc_mesh_2d(16, 16, seed=5)
    sim = make(ers, circ)
    lin = O.linearize(circ, np.zeros(circ.n))
    v = np.random.default_rng(2).normal(size=circ.n)
    K = O.arnoldi_iks(circ.C, lin, lin.Gk, v, 1e-12, 1e-7, 24, 1, 24)
    for m in (1, 5, 13, 24):
        for h in (1e-13, 1e-12, 1e-11):
            y, last = sim.phi_small(K.H[:m + 1, :m], h)
            yr, lr = O.exp_hinv_e1(K.H[:m, :m], h)
            assert np.max(np.abs(y - yr)) <= 1e-11 * max(1.0, np.max(np.abs(yr))), (m, h)
            assert abs(last - lr) <= 1e-9 * max(abs(lr), 1e-300) + 1e-12 * np.max(np.abs(K.H)) ** -1
    sim.close()


@pytest.mark.parametrize("m", [1, 8, 20])
def test_mevp_fixed_m(ers, m):
    circ = S.rc_mesh_2d(20, 20, seed=7)
    sim = make(ers, circ)
    lin = O.linearize(circ, np.zeros(circ.n))
    v = np.random.default_rng(3).normal(size=circ.n)
    h = 2e-12
    out, mu = sim.mevp(v, h, m)
    K = O.arnoldi_iks(circ.C, lin, lin.Gk, v, h, 1e-7, m, 1, m)
    ref = K.mevp(h)
    assert mu == K.m
    ok, worst = node_close(out, ref, 1e-10)
    assert ok, worst
    sim.close()


def test_mevp_adaptive(ers):
    circ = S.rc_mesh_2d(20, 20, seed=8)
    sim = make(ers, circ)
    lin = O.linearize(circ, np.zeros(circ.n))
    v = np.random.default_rng(4).normal(size=circ.n)
    for h in (1e-13, 1e-12, 1e-11):
        out, mu = sim.mevp(v, h, 0)
        K = O.arnoldi_iks(circ.C, lin, lin.Gk, v, h, 1e-7, 40, 3, 0)
        assert mu == K.m, (h, mu, K.m)
        ok, worst = node_close(out, K.mevp(h), 1e-9)
        assert ok, worst
    sim.close()


def test_zero_vector_mevp(ers):
    circ = S.random_rc(n=20, seed=2)
    sim = make(ers, circ)
    out, mu = sim.mevp(np.zeros(circ.n), 1e-12, 5)
    assert mu == 0 and np.all(out == 0.0)
    sim.close()


# --- whole ER step -----------------------------------------------------------------------
def test_single_rc_closed_form(ers):
    g, c, i0 = 1e-3, 1e-15, 1e-3
    circ = S.single_rc(g=g, c=c, i_amp=i0)
    sim = make(ers, circ)
    sim.set_state(0.0, np.zeros(1))
    mu, err = sim.step(1e-12, 3)
    t, x, _ = sim.state()
    exact = (i0 / g) * (1 - np.exp(-1e-12 * g / c))
    assert abs(x[0] - exact) <= 1e-13 * exact and mu == 1 and err == 0.0
    sim.close()


def rc2d_states():
    """Oracle trajectory of the 32x32 RC mesh at h = 1 ps, m = 20 (sampled states)."""
    circ = S.rc_mesh_2d()
    x = np.zeros(circ.n)
    states = {}
    for k in range(400):
        if k in (150, 260, 399):
            states[k] = x.copy()
        x = O.er_step(circ, x, k * 1e-12, 1e-12, m=20).x
    return circ, states


def test_er_step_rc2d_per_step(ers):
    circ, states = rc2d_states()
    sim = make(ers, circ)
    for k, xk in states.items():
        t = k * 1e-12
        ref = O.er_step(circ, xk, t, 1e-12, m=20)
        sim.set_state(t, xk)
        mu, err = sim.step(1e-12, 20)
        _, x, _ = sim.state()
        ok, worst = node_close(x, ref.x)
        assert ok, (k, worst)
        assert mu == ref.m1
    sim.close()


def test_er_step_coupled_capacitance(ers):
    """Non-diagonal C (coupling capacitors on every diagonal neighbour pair): per-step parity
    at fixed m and with the Krylov dimension from Eq. 16."""
    circ = S.coupled_rc_mesh_2d(16, 16, seed=3, n_src=8, t_end=0.3e-9)
    x = np.zeros(circ.n)
    states = {}
    for k in range(120):
        if k in (40, 119):
            states[k] = x.copy()
        x = O.er_step(circ, x, k * 1e-12, 1e-12, m=20).x
    sim = make(ers, circ)
    for k, xk in states.items():
        t = k * 1e-12
        for m in (20, 0):
            ref = O.er_step(circ, xk, t, 1e-12, m=m)
            sim.set_state(t, xk)
            mu, _ = sim.step(1e-12, m)
            _, xg, _ = sim.state()
            ok, worst = node_close(xg, ref.x)
            assert ok, (k, m, worst)
            assert mu == ref.m1
    sim.close()


def test_adaptive_run_coupled_capacitance(ers):
    circ = S.coupled_rc_mesh_2d(12, 12, seed=5, n_src=6, t_end=0.2e-9)
    sim = make(ers, circ)
    sim.set_state(0.0, np.zeros(circ.n))
    ns, nr = sim.run(circ.t_end, 1e-6)
    _, xg, _ = sim.state()
    xr, tr, st = O.er_run(circ, tol=1e-6, x0=np.zeros(circ.n))
    assert ns == st.steps
    ok, worst = node_close(xg, xr, 1e-8)
    assert ok, worst
    sim.close()


def test_er_trajectory_rc2d_full(ers):
    """Full fixed-step trajectory of the 32x32 mesh (1000 steps of 1 ps, m = 20).  Per-step
    differences accumulate along a trajectory; the oracle's own trajectory moves by up to
    1.3e-8 per node under 1e-13 solve noise, so the per-node bar is 1e-8 and the normwise
    bar ||x_gpu - x_or||_inf <= 1e-11 ||x_or||_inf."""
    circ = S.rc_mesh_2d()
    sim = make(ers, circ)
    sim.set_state(0.0, np.zeros(circ.n))
    x = np.zeros(circ.n)
    for k in range(1000):
        x = O.er_step(circ, x, k * 1e-12, 1e-12, m=20).x
        sim.step(1e-12, 20)
        if k % 50 == 49 or k == 999:
            _, xg, _ = sim.state()
            ok, w = node_close(xg, x, 1e-8)
            assert ok, (k, w)
            assert np.max(np.abs(xg - x)) <= 1e-11 * max(np.max(np.abs(x)), 1e-300), k
    sim.close()


def inv_state(stages=20, tree=20, seed=11, t=0.105e-9):
    circ = S.inverter_chain(stages=stages, tree_nodes=tree, seed=seed, t_end=1e-9)
    x = O.dc_solution(circ)
    return circ, x, t


def test_dc_matches_oracle(ers):
    circ = S.inverter_chain(stages=12, tree_nodes=15, seed=5)
    sim = make(ers, circ)
    sim.dc()
    _, x, _ = sim.state()
    ref = O.dc_solution(circ)
    assert np.max(np.abs(x - ref)) <= 1e-9
    sim.close()


def test_dc_long_chain_matches_oracle(ers):
    """DC of a 400-stage chain from its logic-level nodeset, against the oracle's Newton from
    the same guess (from 0 V the linearised chain is a 400-stage amplifier whose Newton
    system overflows, on either side)."""
    circ = S.inverter_chain(stages=400, tree_nodes=20, seed=2, t_end=1e-9)
    sim = make(ers, circ)
    sim.dc(circ.nodeset)
    _, xg, _ = sim.state()
    xr = O.dc_solution(circ, x0=circ.nodeset)
    assert np.max(np.abs(xg - xr)) <= 1e-9
    sim.close()


def test_er_step_nonlinear(ers):
    """Six consecutive steps of the 20-stage chain with the Krylov dimension of Algorithm 1."""
    circ, x0, t = inv_state()
    sim = make(ers, circ)
    x = x0.copy()
    for k in range(6):
        ref = O.er_step(circ, x, t, 1e-12, m=0)
        sim.set_state(t, x)
        mu, err = sim.step(1e-12, 0)
        _, xg, _ = sim.state()
        ok, worst = node_close(xg, ref.x)
        assert ok, (k, worst)
        assert mu == ref.m1
        assert abs(err - ref.err_inf) <= 1e-6 * ref.err_inf + 1e-15, (err, ref.err_inf)
        x = ref.x
        t += 1e-12
    sim.close()


@pytest.mark.parametrize("m", [4, 10, 15])
def test_er_step_nonlinear_fixed_m(ers, m):
    circ, x0, t = inv_state()
    sim = make(ers, circ)
    x = x0.copy()
    for k in range(4):
        ref = O.er_step(circ, x, t, 1e-12, m=m)
        lin = O.linearize(circ, x)
        scale = np.linalg.cond(lin.Gk.toarray()) * np.finfo(float).eps / 1e-13
        bar = max(REL, oracle_floor(circ, x, t, 1e-12, m) * scale)
        sim.set_state(t, x)
        mu, err = sim.step(1e-12, m)
        _, xg, _ = sim.state()
        ok, worst = node_close(xg, ref.x, bar)
        assert ok, (k, worst, bar)
        x = ref.x
        t += 1e-12
    sim.close()


def test_er_step_nonlinear_adaptive_m(ers):
    circ, x0, t = inv_state()
    sim = make(ers, circ)
    ref = O.er_step(circ, x0, t, 2e-12, m=0)
    sim.set_state(t, x0)
    mu, err = sim.step(2e-12, 0)
    _, xg, _ = sim.state()
    assert mu == ref.m1
    ok, worst = node_close(xg, ref.x)
    assert ok, worst
    sim.close()


def test_erc_correction_step(ers):
    circ, x0, t = inv_state()
    sim = make(ers, circ, correction=1)
    ref = O.er_step(circ, x0, t, 1e-12, m=10, opts=O.Options(correction=True))
    sim.set_state(t, x0)
    sim.step(1e-12, 10)
    _, xg, _ = sim.state()
    ok, worst = node_close(xg, ref.x)
    assert ok, worst
    sim.close()


def test_adaptive_run_matches_oracle(ers):
    circ = S.inverter_chain(stages=4, tree_nodes=10, seed=6, t_end=0.2e-9)
    sim = make(ers, circ)
    sim.dc()
    ns, nr = sim.run(circ.t_end, 1e-6)
    _, xg, _ = sim.state()
    xr, tr, st = O.er_run(circ, tol=1e-6)
    assert abs(ns - st.steps) <= max(2, 0.05 * st.steps), (ns, st.steps)
    assert np.max(np.abs(xg - xr)) <= 2e-6 * max(1.0, np.max(np.abs(xr)))
    stats = sim.stats()
    assert stats["refactors"] >= ns
    sim.close()


def test_adaptive_erc_run_with_rejections_matches_oracle(ers):
    """ER-C inside Algorithm 2 with rejected tries on PWL-ramp steps: every rejection
    re-exponentiates the solution bases (v1 and, on a ramp, v2) at the smaller h, so the
    correction's own basis must not share their storage.  Per-node agreement with the
    oracle's adaptive ER-C run and matching step counts."""
    circ = S.inverter_chain(stages=4, tree_nodes=10, seed=6, t_end=0.2e-9)
    sim = make(ers, circ, correction=1, h_max=5e-12)
    sim.dc()
    ns, nr = sim.run(circ.t_end, 1e-6)
    _, xg, _ = sim.state()
    xr, tr, st = O.er_run(circ, tol=1e-6, opts=O.Options(correction=True, h_max=5e-12))
    assert st.rejects > 0 and nr > 0
    assert abs(ns - st.steps) <= max(2, 0.05 * st.steps), (ns, st.steps)
    assert abs(nr - st.rejects) <= max(2, 0.05 * st.rejects), (nr, st.rejects)
    assert np.max(np.abs(xg - xr)) <= 2e-6 * max(1.0, np.max(np.abs(xr)))
    sim.close()


# --- boundary behaviour ------------------------------------------------------------------
def test_bounded_wait_reports_timeout(ers):
    """Failure detection without a GPU fault: a device wait on a flag that nothing sets gives
    up after its poll limit and reports ERS_ERR_TIMEOUT; the context keeps working."""
    circ = S.rc_mesh_2d(8, 8, seed=1)
    sim = make(ers, circ)
    sim.set_state(0.0, np.zeros(circ.n))
    assert sim.wait_selftest() == 6          # ERS_ERR_TIMEOUT
    lin = O.linearize(circ, np.zeros(circ.n))
    b = np.random.default_rng(9).normal(size=circ.n)
    x = sim.solve(b)
    ref = lin.solve(b)
    assert np.max(np.abs(x - ref)) <= 1e-8 * np.max(np.abs(ref))
    sim.close()


def test_step_across_breakpoint_rejected(ers):
    circ = S.rc_mesh_2d(8, 8, seed=1)
    sim = make(ers, circ)
    bp = circ.breakpoints()
    t0 = float(bp[2]) - 0.5e-12
    sim.set_state(t0, np.zeros(circ.n))
    with pytest.raises(ers.ErsError) as ei:
        sim.step(1e-12, 5)
    assert ei.value.status == 1
    sim.close()


def test_invalid_inputs_rejected(ers):
    circ = S.rc_mesh_2d(4, 4, seed=1)
    bad = circ.G.copy()
    bad.indices[1], bad.indices[0] = bad.indices[0], bad.indices[1]   # unsorted columns
    with pytest.raises(ers.ErsError) as ei:
        ers.Simulator(bad, circ.C, circ.B, None, circ.pwl)
    assert ei.value.status == 1


def test_singular_G_reported(ers):
    import scipy.sparse as sp
    circ = S.random_rc(n=6, seed=1)
    G = circ.G.tolil()
    G[5, :] = 0.0
    G[:, 5] = 0.0
    G[5, 5] = 0.0
    G = sp.csr_matrix(G)
    G.eliminate_zeros()
    G = G + sp.csr_matrix(([0.0], ([5], [5])), shape=G.shape)  # keep the diagonal in the pattern
    G.sort_indices()
    sim = ers.Simulator(G, circ.C, circ.B, None, circ.pwl)
    with pytest.raises(ers.ErsError) as ei:
        sim.refactor()
    assert ei.value.status == 2
    sim.close()
