"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports every
symbol include/ers.h declares, and its host-only symbolic analysis is consistent."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from synth import circuits as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def E():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers
    return ers


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ers.h")).read()
    return sorted(set(re.findall(r"\b(ers_[A-Za-z0-9_]+)\s*\(", src)))


def test_header_declares_binding_exports(E):
    assert declared_symbols() == sorted(E.EXPORTS)


def test_library_exports_every_declared_symbol(E):
    L = E.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name


def test_default_opts(E):
    o = E.default_opts()
    assert o.eps_krylov == 1e-7 and o.alpha == 0.5 and o.beta == 2.0 and o.i_grow == 5
    assert o.m_max == 40 and o.gamma == 0.1


def _pattern(c):
    rows, cols = [], []
    for d in c.dev:
        for node in (d["d"], d["s"]):
            if node < 0:
                continue
            for t in (d["d"], d["g"], d["s"]):
                if t >= 0:
                    rows.append(node)
                    cols.append(t)
    A = c.G.tocoo()
    r = np.concatenate([A.row, rows, np.arange(c.n)])
    cc = np.concatenate([A.col, cols, np.arange(c.n)])
    M = sp.csr_matrix((np.ones(r.size), (r, cc)), shape=(c.n, c.n))
    M.sum_duplicates()
    M.sort_indices()
    return M


def _chol_nnz(M, perm):
    """nnz of the Cholesky factor of the symmetrised, permuted pattern by dense elimination
    on a boolean matrix (brute force, small cases only)."""
    A = (M + M.T).toarray() != 0
    A = A[np.ix_(perm, perm)]
    n = A.shape[0]
    nnz = 0
    for k in range(n):
        nb = np.nonzero(A[k + 1:, k])[0] + k + 1
        nnz += 1 + nb.size
        A[np.ix_(nb, nb)] = True
    return nnz


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("circ", [S.rc_mesh_2d(9, 7, seed=1), S.random_rc(n=30, seed=2),
                                  S.inverter_chain(stages=5, tree_nodes=12, seed=3),
                                  S.rc_mesh_3d(6, 5, 4, seed=1, n_loads=5)])
def test_symbolic_fill_matches_brute_force(E, circ, ordering):
    M = _pattern(circ)
    d = E.analyze(M, ordering=ordering)
    perm = d["perm"]
    assert sorted(perm.tolist()) == list(range(circ.n))
    assert d["nnz_L"] == _chol_nnz(M, perm)
    assert d["nsn"] >= 1 and d["nlevels"] >= 1


@pytest.mark.parametrize("ordering", [0, 1])
def test_tree_ordering_has_no_fill(E, ordering):
    """A tree small enough for one nested-dissection leaf is ordered by exact minimum
    degree, which eliminates leaves first: zero fill."""
    circ = S.inverter_chain(stages=1, tree_nodes=30, seed=7)
    M = _pattern(circ)
    d = E.analyze(M, ordering=ordering)
    sym = ((M + M.T) != 0).astype(int)
    assert d["nnz_L"] == circ.n + (sym.nnz - circ.n) // 2


def test_ordering_1_reduces_mesh_fill(E):
    """ordering = 1 (the smallest BFS level within a 35-65 % split, from either end of the
    pseudo-diameter) against the median-level separators of ordering = 0 on 2D and 3D meshes;
    an unknown ordering is refused."""
    for G in (S.rc_mesh_2d(32, 32, seed=0).G, S.rc_mesh_3d(20, 20, 20, seed=1, n_loads=80).G):
        a, b = E.analyze(G, ordering=0), E.analyze(G, ordering=1)
        assert b["nnz_L"] < 0.95 * a["nnz_L"], (a["nnz_L"], b["nnz_L"])
        assert b["factor_doubles"] < a["factor_doubles"]
    with pytest.raises(E.ErsError):
        E.analyze(S.rc_mesh_2d(4, 4, seed=0).G, ordering=2)


def test_analyze_rejects_missing_diagonal(E):
    M = sp.csr_matrix(np.array([[0.0, 1.0], [1.0, 1.0]]))
    M.eliminate_zeros()
    with pytest.raises(E.ErsError):
        E.analyze(M)


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("name", ["rc2d", "rc3d", "chain", "batch", "randrc"])
def test_solve_plan_covers_and_orders(E, name, ordering):
    """Every supernode is computed once per direction, every wait points to an earlier entry
    (deadlock-free persistent solves); the batch of chains exercises the lane tasks."""
    if name == "rc2d":
        G = S.rc_mesh_2d(32, 32, seed=0).G
    elif name == "rc3d":
        G = S.rc_mesh_3d(20, 20, 20, seed=1, n_loads=80).G
    elif name == "chain":
        G = S.inverter_chain(stages=50, tree_nodes=100, seed=2).G
    elif name == "batch":
        circs = S.batch_family(n_inst=48, seed0=7000, stage_lo=30, stage_hi=60, tree_nodes=100)
        G = sp.block_diag([c.G for c in circs], format="csr")
    else:
        G = S.random_rc(n=60, seed=3, density=0.4).G
    G = sp.csr_matrix(G)
    G.sort_indices()
    c = E.solve_plan_check(G, ordering=ordering)
    st = E.analyze(G, ordering=ordering)
    nsn = st["nsn"]
    assert c["fwd_lane_items"] + c["fwd_warp_supernodes"] + c["fwd_diag"] == nsn
    assert c["bwd_lane_items"] + c["bwd_warp_supernodes"] + c["bwd_diag"] == nsn
    if name == "batch":
        assert c["fwd_lane_items"] > 0 and c["bwd_lane_items"] > 0


def test_batch_rejects_single_context_options(E):
    """ER-C and the combined space are single-context options: a batched context refuses them
    (checked before any device work, so this runs without a GPU)."""
    circs = [S.rc_mesh_2d(4, 4, seed=s, n_src=4) for s in range(2)]
    for kw in ({"correction": 1}, {"combined_vector": 1}):
        with pytest.raises(E.ErsError) as ei:
            E.BatchSimulator(circs, opts=E.make_opts(**kw))
        assert "single-context" in str(ei.value)


def test_create_accepts_node_without_capacitance(E):
    """A node without capacitance (singular C, Sec. IV-A) is no longer refused: the symbolic
    analysis only sees G, and the input checks pass; on this CPU-only host creation then stops
    at the first device call (ERS_ERR_CUDA), not at an argument check (ERS_ERR_INVALID)."""
    circ = S.random_rc(n=12, seed=3, p=2, n_alg=2)
    with pytest.raises(E.ErsError) as ei:
        E.Simulator.from_circuit(circ)
    assert ei.value.status == 7, ei.value


def test_coupling_capacitance_fills_c_over_h_plus_g(E):
    """Why the method factors G_k alone (Sec. II-B, Fig. 1): with coupling capacitors the
    matrix C/h + G that backward Euler factors has C's off-diagonal pattern on top of G's, and
    its LU fills more.  On the 100 x 100 mesh with a coupling capacitor per cell the symbolic
    analysis gives 1.38x the factor entries and 1.5x the refactor flops (ordering 0)."""
    c = S.coupled_rc_mesh_2d(100, 100, seed=1, n_src=16)
    G = c.G.tocsr()
    CG = (c.C + c.G).tocsr()
    CG.sort_indices()
    a, b = E.analyze(G, ordering=0), E.analyze(CG, ordering=0)
    assert CG.nnz > 1.3 * G.nnz
    assert b["nnz_L"] > 1.3 * a["nnz_L"] and b["refactor_flops"] > 1.4 * a["refactor_flops"]


def test_gmin_option_default_and_validation(E):
    """gmin (conductance from every node to ground added by the library) defaults to 0 and a
    negative or non-finite value is refused before any device work."""
    assert E.default_opts().gmin == 0.0
    circ = S.random_rc(n=8, seed=1)
    for bad in (-1e-12, float("nan"), float("inf")):
        with pytest.raises(E.ErsError) as ei:
            E.Simulator.from_circuit(circ, opts=E.make_opts(gmin=bad))
        assert ei.value.status == 1 and "gmin" in str(ei.value)


def _opt_makespan(costs, m):
    """Smallest largest-part load over all assignments (brute force, tiny inputs)."""
    import itertools
    best = float("inf")
    for assign in itertools.product(range(m), repeat=len(costs)):
        loads = [0.0] * m
        for c, p in zip(costs, assign):
            loads[p] += c
        best = min(best, max(loads))
    return best


def test_partition_lpt_rule_and_bound(E):
    """ers_partition_lpt, the device split of ers_create_batch: the hand-worked LPT assignment
    of a small case, and Graham's bound (4/3 - 1/(3m)) OPT against brute force."""
    # costs 7, 5, 4, 3, 3, 2 over 2 parts, each onto the lighter part (loads in brackets):
    # 7 -> 0 [7, 0]; 5 -> 1 [7, 5]; 4 -> 1 [7, 9]; 3 -> 0 [10, 9]; 3 -> 1 [10, 12];
    # 2 -> 0 [12, 12]
    part = E.partition_lpt([7, 5, 4, 3, 3, 2], 2)
    assert part.tolist() == [0, 1, 1, 0, 1, 0]
    rng = np.random.default_rng(4)
    for trial in range(30):
        m = int(rng.integers(2, 4))
        costs = rng.integers(1, 20, size=int(rng.integers(1, 8))).astype(float)
        part = E.partition_lpt(costs, m)
        loads = np.bincount(part, weights=costs, minlength=m)
        assert part.min() >= 0 and part.max() < m
        assert loads.max() <= (4 / 3 - 1 / (3 * m)) * _opt_makespan(costs, m) + 1e-9
    # ties: equal costs go to parts in order, lower index first
    assert E.partition_lpt([1, 1, 1, 1], 3).tolist() == [0, 1, 2, 0]
    with pytest.raises(E.ErsError):
        E.partition_lpt([1.0, -1.0], 2)
    with pytest.raises(E.ErsError):
        E.partition_lpt([1.0], 0)


def test_device_list_refusals_without_a_gpu(E):
    """A single circuit refuses more than one device; a device id that does not exist (or no
    device at all, as on a CPU-only host) is refused before any device work."""
    c = S.rc_mesh_2d(4, 4, seed=1)
    with pytest.raises(E.ErsError) as ei:
        E.Simulator.from_circuit(c, device=10 ** 6)
    assert ei.value.status == 1
    with pytest.raises(E.ErsError) as ei:
        E.BatchSimulator([c, c], devices=[0, 10 ** 6])
    assert ei.value.status == 1


def _py_pwl(tt, vv, x):
    """PWL value at x: the last corner at or before x, linear to the next (separate roundings)."""
    if x <= tt[0]:
        return vv[0]
    if x >= tt[-1]:
        return vv[-1]
    lo, hi = 0, len(tt) - 1
    while hi - lo > 1:
        mid = (lo + hi) >> 1
        if tt[mid] <= x:
            lo = mid
        else:
            hi = mid
    f = (x - tt[lo]) / (tt[hi] - tt[lo])
    prod = f * (vv[hi] - vv[lo])
    return vv[lo] + prod


def test_pwl_ramp_matches_brute_force(E):
    """The host ramp test of a step's set-up (Eq. 12-13: the v2 / w1 terms exist only when an
    input has a non-zero slope over the step) equals the brute-force evaluation of every input
    at t and t + h, including its shortcut over the ranges where some input changes: pulses
    with flat tops, steep edges, steps that start or end exactly on a corner, h = 0."""
    rng = np.random.default_rng(11)
    for trial in range(60):
        pwl = []
        corners = []
        for q in range(int(rng.integers(1, 6))):
            d = float(rng.uniform(0, 5e-10))
            rise = float(rng.choice([1e-15, 1e-11, 3e-11]))
            width = float(rng.uniform(1e-11, 2e-10))
            amp = float(rng.choice([0.0, 1e-3, -2e-3]))
            tt = [0.0, d, d + rise, d + rise + width, d + 2 * rise + width, 1e-9]
            tt = sorted(set(tt))
            vv = [0.0] * len(tt)
            for k, x in enumerate(tt):
                if d + rise <= x <= d + rise + width:
                    vv[k] = amp
            pwl.append((tt, vv))
            corners += tt
        for _ in range(40):
            if rng.random() < 0.5:
                t = float(rng.choice(corners))
                h = float(rng.choice(corners)) - t if rng.random() < 0.5 else float(rng.uniform(0, 5e-11))
            else:
                t = float(rng.uniform(0, 1e-9))
                h = float(rng.uniform(0, 5e-11))
            want = h > 0 and any(_py_pwl(tt, vv, t + h) != _py_pwl(tt, vv, t) for tt, vv in pwl)
            assert E.pwl_ramp(pwl, t, h) == want, (trial, t, h)
    assert not E.pwl_ramp([([0.0, 1e-12], [0.0, 1.0])], 0.5e-12, 0.0)
    with pytest.raises(E.ErsError):
        E.pwl_ramp([([1e-12, 1e-12], [0.0, 1.0])], 0.0, 1e-12)
