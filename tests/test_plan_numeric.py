"""Numeric execution of the symbolic plan on the CPU: the multifrontal LU of G laid out
exactly as the plan lays it out for the refactor kernels (one flat arena, fronts at their
offsets, matrix entries assigned at their assembly targets, children's update blocks added
through their relative indices in the plan's child order, each front factored without
pivoting and its Schur complement left in place for the parent), then the supernodal
triangular solves.  The result must equal a sparse direct solve of G x = b: a front placed
over a live one, a wrong relative index or assembly target, or a child added to the wrong
parent changes it.  Both orderings, five pattern families; no GPU.

The executor is test code: it uses the plan the library exports, not the library's
kernels."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from synth import circuits as S


@pytest.fixture(scope="module")
def E():
    from paper_1511_04515_gb300 import build
    build.build()
    from paper_1511_04515_gb300 import ers
    return ers


def execute(P, vals, b_new):
    """Multifrontal LU on the plan's arena, then L y = b and U x = y (new node order)."""
    nsn = P["sn_start"].size - 1
    arena = np.full(int(P["arena"][0]), np.nan)      # an unwritten read shows up as NaN
    nlev = P["lvl_slot_ptr"].size - 1
    by_level = [[] for _ in range(nlev)]
    for s in range(nsn):
        by_level[P["level"][s]].append(s)

    def dims(s):
        c0 = int(P["sn_start"][s])
        return c0, int(P["sn_start"][s + 1]) - c0, int(P["rptr"][s + 1] - P["rptr"][s])

    def front(s):
        _, w, r = dims(s)
        f = w + r
        o = int(P["front_off"][s])
        return arena[o:o + f * f].reshape((f, f), order="F")    # a view into the arena

    fac = {}
    for lev in range(nlev):
        for s in by_level[lev]:
            front(s)[:] = 0.0
        for k in range(P["lvl_slot_ptr"][lev], P["lvl_slot_ptr"][lev + 1]):
            e = P["lvl_slot"][k]
            arena[P["asm_dst"][e]] = vals[e]
        for s in by_level[lev]:
            Fp = front(s)
            for q in range(P["ch_ptr"][s], P["ch_ptr"][s + 1]):
                c = int(P["ch_list"][q])
                _, cw, _ = dims(c)
                rel = P["rel"][P["rptr"][c]:P["rptr"][c + 1]]
                Fp[np.ix_(rel, rel)] += front(c)[cw:, cw:]
        for s in by_level[lev]:
            c0, w, r = dims(s)
            F = front(s)
            U11 = F[:w, :w].copy()
            L11 = np.eye(w)
            for k in range(w):                     # LU without pivoting (static pivots)
                L11[k + 1:, k] = U11[k + 1:, k] / U11[k, k]
                U11[k + 1:, k:] -= np.outer(L11[k + 1:, k], U11[k, k:])
            U11 = np.triu(U11)
            L21 = np.linalg.solve(U11.T, F[w:, :w].T).T          # F21 U11^-1
            U12 = np.linalg.solve(L11, F[:w, w:])                # L11^-1 F12
            F[w:, w:] -= L21 @ U12                               # update block for the parent
            R = P["rows"][P["rptr"][s]:P["rptr"][s + 1]].copy()
            fac[s] = (c0, w, L11, U11, L21, U12, R)
    order = sorted(range(nsn), key=lambda s: P["level"][s])
    y = b_new.copy()
    for s in order:
        c0, w, L11, U11, L21, U12, R = fac[s]
        ys = np.linalg.solve(L11, y[c0:c0 + w])
        y[c0:c0 + w] = ys
        y[R] -= L21 @ ys
    x = y
    for s in reversed(order):
        c0, w, L11, U11, L21, U12, R = fac[s]
        x[c0:c0 + w] = np.linalg.solve(U11, x[c0:c0 + w] - U12 @ x[R])
    return x


def with_devices(c, seed):
    """G plus small conductances at the device stamp positions (the union pattern G_k has)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    for d in c.dev:
        for node in (d["d"], d["s"]):
            if node < 0:
                continue
            for t in (d["d"], d["g"], d["s"]):
                if t >= 0:
                    rows.append(node)
                    cols.append(t)
    D = sp.csr_matrix((rng.uniform(-1e-5, 1e-5, len(rows)), (rows, cols)), shape=c.G.shape)
    M = (c.G + D).tocsr()
    M.sum_duplicates()
    M.sort_indices()
    return M


def matrices():
    chain = S.inverter_chain(stages=30, tree_nodes=20, seed=3)
    batch = S.batch_family(n_inst=6, seed0=7000, stage_lo=3, stage_hi=12, tree_nodes=15)
    return {
        "rc2d": S.rc_mesh_2d(24, 20, seed=0).G,
        "rc3d": S.rc_mesh_3d(12, 11, 10, seed=1, n_loads=30).G,
        "randrc": S.random_rc(n=60, seed=3, density=0.4).G,
        "chain": with_devices(chain, 1),
        "batch": sp.block_diag([with_devices(c, k) for k, c in enumerate(batch)], format="csr"),
    }


MATS = matrices()


@pytest.mark.parametrize("ordering", [0, 1])
@pytest.mark.parametrize("name", list(MATS))
def test_plan_executes_to_the_direct_solution(E, name, ordering):
    G = sp.csr_matrix(MATS[name])
    G.sum_duplicates()
    G.sort_indices()
    P = E.plan_arrays(G, ordering=ordering)
    vals = G.data[P["a_src"]]                  # the matrix in the plan's slot order
    rng = np.random.default_rng(7)
    b = rng.normal(size=G.shape[0])
    perm = P["perm"]
    x_new = execute(P, vals, b[perm])
    x = np.empty_like(x_new)
    x[perm] = x_new
    ref = spla.spsolve(G.tocsc(), b)
    assert np.all(np.isfinite(x))
    assert np.max(np.abs(x - ref)) <= 1e-9 * np.max(np.abs(ref)), name
