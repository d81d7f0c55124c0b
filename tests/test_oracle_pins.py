"""Pins of the CPU oracle against facts that do not come from the oracle itself:
closed forms, an eigen-decomposition of the exact linear solution, the Arnoldi relation
written with a dense inverse, finite differences, convergence orders and invariants."""
import numpy as np
import pytest
import scipy.linalg as sla

from synth import circuits as S
from oracle import ers_oracle as O


def exact_linear_step(circ, x, t, h):
    """Exact solution of C x' = -G x + B u(t) over [t, t+h] with u linear on the step,
    by the generalized symmetric eigenproblem G q = lambda C q (independent of expm)."""
    G = circ.G.toarray(); C = circ.C.toarray(); B = circ.B.toarray()
    lam, Q = sla.eigh(G, C)          # Q^T C Q = I, J = -C^{-1} G = Q (-lam) Q^{-1}
    uk = circ.u(t); s = (circ.u(t + h) - uk) / h
    y0 = Q.T @ C @ x
    f = Q.T @ B @ uk
    g = Q.T @ B @ s
    e = np.exp(-lam * h)
    y = e * y0 + f * (1 - e) / lam + g * (h / lam - (1 - e) / lam ** 2)
    return Q @ y


# --- Whole ER step, linear circuits: exact up to the Krylov error (Eq. 13) ---------------
def test_single_rc_step_current_closed_form():
    g, c, i0 = 1e-3, 1e-15, 1e-3
    circ = S.single_rc(g=g, c=c, i_amp=i0)
    for h in (1e-13, 1e-12, 5e-12):
        r = O.er_step(circ, np.zeros(1), 0.0, h, m=3)
        exact = (i0 / g) * (1 - np.exp(-h * g / c))
        assert abs(r.x[0] - exact) <= 1e-13 * abs(exact)
        assert r.m1 == 1  # one-dimensional space: happy breakdown at j = 1


def test_single_rc_ramp_closed_form():
    g, c, s = 2e-3, 3e-15, 1e9
    circ = S.single_rc(g=g, c=c, ramp=s, t_end=20e-12)
    tau = c / g
    for h in (1e-13, 2e-12, 7e-12):
        r = O.er_step(circ, np.zeros(1), 0.0, h, m=3)
        exact = (s / g) * (h - tau * (1 - np.exp(-h / tau)))
        assert abs(r.x[0] - exact) <= 1e-12 * abs(exact)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_rc_step_matches_eigen_solution(seed):
    circ = S.random_rc(n=16, seed=seed)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=circ.n) * 0.1
    t, h = 3e-12, 2e-12       # inside a ramp for some sources
    nb = circ.breakpoints()
    nb = nb[nb > t]
    h = min(h, nb[0] - t) if nb.size else h      # u must be linear on the step
    r = O.er_step(circ, x, t, h, m=circ.n)
    ex = exact_linear_step(circ, x, t, h)
    assert np.max(np.abs(r.x - ex)) <= 1e-11 * np.max(np.abs(ex))


def test_coupled_capacitance_step_matches_eigen_solution():
    """Non-diagonal C (coupling capacitors): the ER step with a full Krylov space equals the
    exact solution from the generalized eigenproblem G q = lambda C q."""
    circ = S.coupled_rc_mesh_2d(5, 5, seed=4, n_src=4, t_end=50e-12)
    assert (circ.C - sp_diag(circ.C)).nnz > 0
    rng = np.random.default_rng(4)
    x = rng.normal(size=circ.n) * 0.1
    t = 0.0
    nb = circ.breakpoints()
    h = min(3e-12, float(nb[nb > t][0]) - t)
    r = O.er_step(circ, x, t, h, m=circ.n)
    ex = exact_linear_step(circ, x, t, h)
    assert np.max(np.abs(r.x - ex)) <= 1e-10 * np.max(np.abs(ex))


def sp_diag(M):
    import scipy.sparse as sp
    return sp.diags(M.diagonal())


def test_random_rc_trajectory_exact():
    circ = S.random_rc(n=12, seed=5, p=3, t_end=30e-12)
    bps = list(circ.breakpoints())
    grid = sorted(set([0.0] + [b for b in bps if b < circ.t_end] + [circ.t_end]))
    x = np.zeros(circ.n); xe = np.zeros(circ.n)
    for a, b in zip(grid[:-1], grid[1:]):
        x = O.er_step(circ, x, a, b - a, m=circ.n).x
        xe = exact_linear_step(circ, xe, a, b - a)
    # m = n spans the whole space in exact arithmetic; in floating point plain MGS (no
    # re-orthogonalisation) on a stiff spectrum (tau 3e-14 .. 7e-12 s) loses ~1e-8 on
    # some steps, while any dropped term or sign error shows up at the O(h) ~ 1e-2 level.
    assert np.max(np.abs(x - xe)) <= 1e-6 * np.max(np.abs(xe))


def test_combined_vector_equals_separate_spaces():
    circ = S.random_rc(n=16, seed=4)
    x = np.random.default_rng(1).normal(size=circ.n) * 0.05
    a = O.er_step(circ, x, 5e-12, 1e-12, m=circ.n)
    b = O.er_step(circ, x, 5e-12, 1e-12, m=circ.n, opts=O.Options(combined=True))
    assert np.max(np.abs(a.x - b.x)) <= 1e-11 * np.max(np.abs(a.x))


# --- ER formula with explicit phi functions (Eq. 9-13) ----------------------------------
def phi_step_dense(circ, x, t, h):
    """x + h phi1(hJ) g_k + h^2 phi2(hJ) b_k with J = -C^{-1} G_k, g_k and b_k of Eq. 12 and
    Eq. 12's input term, phi functions of Eq. 9 applied per eigenvalue of J."""
    lin = O.linearize(circ, x)
    C = circ.C.toarray(); Gk = lin.Gk.toarray(); Ci = np.linalg.inv(C)
    J = -Ci @ Gk
    uk = circ.u(t); s = (circ.u(t + h) - uk) / h
    g = J @ x + Ci @ (lin.F + circ.B @ uk)
    b = Ci @ (circ.B @ s)
    lam, Q = np.linalg.eig(J)
    Qi = np.linalg.inv(Q)
    z = h * lam
    phi1 = (np.exp(z) - 1) / z
    phi2 = (np.exp(z) - 1 - z) / z ** 2
    step = Q @ (h * phi1 * (Qi @ g) + h * h * phi2 * (Qi @ b))
    return x + step.real


def test_er_step_nonlinear_equals_phi_formula():
    circ = S.inverter_chain(stages=2, tree_nodes=3, seed=7, t_end=1e-9)
    x = O.dc_solution(circ)
    x = x + np.random.default_rng(0).normal(size=circ.n) * 0.05
    t = 0.1e-9 + 2e-12   # on the input's rising edge
    h = 3e-12
    r = O.er_step(circ, x, t, h, m=circ.n)
    ref = phi_step_dense(circ, x, t, h)
    assert np.max(np.abs(r.x - ref)) <= 1e-9 * max(1.0, np.max(np.abs(ref)))


# --- MEVP_IKS / Arnoldi (Algorithm 1, Eq. 14, Eq. 16) -----------------------------------
def _basis(circ, m, seed=0):
    lin = O.linearize(circ, np.zeros(circ.n))
    v = np.random.default_rng(seed).normal(size=circ.n)
    return lin, O.arnoldi_iks(circ.C, lin, lin.Gk, v, 1e-12, 1e-7, m, 1, m), v


def test_arnoldi_relation_and_orthonormality():
    circ = S.random_rc(n=30, seed=11)
    m = 10
    lin, K, v = _basis(circ, m)
    Jinv = -np.linalg.inv(circ.G.toarray()) @ circ.C.toarray()
    lhs = Jinv @ K.V[:, :m]
    rhs = K.V[:, :m + 1] @ K.H[:m + 1, :m]
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))
    assert np.max(np.abs(K.V.T @ K.V - np.eye(m + 1))) <= 1e-10
    assert np.allclose(K.V[:, 0] * K.beta, v, rtol=0, atol=1e-14 * np.max(np.abs(v)))


def test_residual_formula_matches_kcl_residual():
    circ = S.random_rc(n=30, seed=12)
    m = 6
    lin, K, v = _basis(circ, m)
    G = circ.G.toarray(); C = circ.C.toarray()
    for h in (1e-13, 1e-12, 1e-11):
        Hm = K.H[:m, :m]
        Hinv = np.linalg.inv(Hm)
        E = sla.expm(h * Hinv)
        xm = K.beta * K.V[:, :m] @ E[:, 0]
        dxm = K.beta * K.V[:, :m] @ (Hinv @ E[:, 0])
        r_explicit = C @ dxm + G @ xm                 # C (dx/dt - J x)
        r_formula = K.residual(m, h) * K.beta * np.linalg.norm(G @ K.V[:, 0])
        # the identity rests on the Arnoldi relation (1e-12 of ||J^-1 V||); the residual is
        # a small difference of large terms, so agreement to 1e-6 of its norm is the bar
        assert abs(np.linalg.norm(r_explicit) - r_formula) <= 1e-6 * np.linalg.norm(r_explicit)


def test_exp_small_against_eigendecomposition():
    rng = np.random.default_rng(3)
    m = 8
    S_ = rng.normal(size=(m, m)) + 3 * np.eye(m)
    D = -np.exp(rng.uniform(np.log(1e-15), np.log(1e-12), m))   # Ritz values: -tau_i
    Hm = S_ @ np.diag(D) @ np.linalg.inv(S_)
    h = 1e-13
    y, last = O.exp_hinv_e1(Hm, h)
    ref = S_ @ (np.exp(h / D) * np.linalg.solve(S_, np.eye(m)[:, 0]))
    assert np.max(np.abs(y - ref)) <= 1e-9 * max(1e-300, np.max(np.abs(ref))) + 1e-14
    ref_last = (S_ @ ((1 / D) * np.exp(h / D) * np.linalg.solve(S_, np.eye(m)[:, 0])))[m - 1]
    assert abs(last - ref_last) <= 1e-8 * abs(ref_last) + 1e-14 * np.max(np.abs(1 / D))


def test_exp_small_scalar():
    for mu, h in ((-1e-12, 3e-13), (-5e-15, 1e-14)):
        y, last = O.exp_hinv_e1(np.array([[mu]]), h)
        assert abs(y[0] - np.exp(h / mu)) <= 1e-15
        assert abs(last - np.exp(h / mu) / mu) <= 1e-13 * abs(1 / mu)


def test_zero_vector_mevp_is_zero():
    circ = S.random_rc(n=10, seed=1)
    lin = O.linearize(circ, np.zeros(circ.n))
    K = O.arnoldi_iks(circ.C, lin, lin.Gk, np.zeros(circ.n), 1e-12, 1e-7, 10)
    assert K.beta == 0.0 and np.all(K.mevp(1e-12) == 0.0)


def test_scaling_invariance_retry_equals_fresh_step():
    circ = S.random_rc(n=20, seed=8)
    x = np.random.default_rng(2).normal(size=circ.n) * 0.1
    t, h, m = 6e-12, 1e-12, 8
    lin = O.linearize(circ, x)
    st = O.step_setup(circ, lin, t, O.pwl_slope(circ, t, h))
    st.K1 = O.arnoldi_iks(circ.C, lin, lin.Gk, st.v1, h, 1e-7, m, 1, m)
    st.K2 = O.arnoldi_iks(circ.C, lin, lin.Gk, st.v2, h, 1e-7, m, 1, m) if np.any(st.v2) else None
    for a in (0.5, 0.25):
        reused = O.er_update(st, a * h)
        fresh = O.er_step(circ, x, t, a * h, m=m).x
        assert np.max(np.abs(reused - fresh)) <= 1e-12 * np.max(np.abs(fresh))


# --- Device model ----------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [0, 1])
def test_mosfet_partials_finite_difference(dtype):
    rng = np.random.default_rng(dtype)
    for _ in range(200):
        vd, vg, vs = rng.uniform(-0.2, 1.2, 3)
        vt, k, lam = 0.35, 1e-4, 0.05
        i0, dvd, dvg, dvs = O.mosfet_eval(dtype, vd, vg, vs, vt, k, lam)
        eps = 1e-7
        for idx, der in ((0, dvd), (1, dvg), (2, dvs)):
            vp = [vd, vg, vs]; vm = [vd, vg, vs]
            vp[idx] += eps; vm[idx] -= eps
            fd = (O.mosfet_eval(dtype, *vp, vt, k, lam)[0] - O.mosfet_eval(dtype, *vm, vt, k, lam)[0]) / (2 * eps)
            assert abs(fd - der) <= 1e-6 * k + 1e-3 * abs(der)


def test_mosfet_symmetry_and_regions():
    vt, k = 0.3, 1e-4
    # source/drain swap: I(d,g,s) = -I(s,g,d)
    a = O.mosfet_eval(0, 0.2, 1.0, 0.7, vt, k, 0.0)[0]
    b = O.mosfet_eval(0, 0.7, 1.0, 0.2, vt, k, 0.0)[0]
    assert a == -b
    # saturation value and cut-off
    assert abs(O.mosfet_eval(0, 1.0, 0.8, 0.0, vt, k, 0.0)[0] - 0.5 * k * 0.5 ** 2) < 1e-18
    assert O.mosfet_eval(0, 1.0, 0.2, 0.0, vt, k, 0.0)[0] == 0.0
    # PMOS with source at vdd, gate low, drain low: current flows from source into drain
    assert O.mosfet_eval(1, 0.0, 0.0, 1.0, vt, k, 0.0)[0] < 0.0


def test_device_jacobian_finite_difference():
    circ = S.inverter_chain(stages=3, tree_nodes=4, seed=3)
    x = np.random.default_rng(5).uniform(0, 1, circ.n)
    idev, Gdev = O.device_eval(circ, x)
    Gd = Gdev.toarray()
    eps = 1e-7
    for j in range(circ.n):
        xp = x.copy(); xp[j] += eps
        xm = x.copy(); xm[j] -= eps
        fd = (O.device_eval(circ, xp)[0] - O.device_eval(circ, xm)[0]) / (2 * eps)
        assert np.max(np.abs(fd - Gd[:, j])) <= 1e-9


# --- DC, convergence orders, error estimate --------------------------------------------
def test_dc_inverter_rails():
    circ = S.inverter_chain(stages=6, tree_nodes=5, seed=4)
    x = O.dc_solution(circ)
    outs = [int(d["d"]) for d in circ.dev[::2]]
    expect = [1.0 if s % 2 == 0 else 0.0 for s in range(len(outs))]
    assert np.max(np.abs(x[outs] - expect)) < 1e-5
    idev, _ = O.device_eval(circ, x)
    res = circ.G @ x + idev - circ.B @ circ.u(0.0)
    assert np.max(np.abs(res)) <= 1e-12


def _switching_window():
    circ = S.inverter_chain(stages=2, tree_nodes=3, seed=9, t_end=1e-9)
    x0 = O.dc_solution(circ)
    return circ, x0, 0.11e-9, 0.11e-9 + 16e-12


def _fixed_er(circ, x0, t0, t1, h, m=0, correction=False):
    """Fixed-h ER steps; m = 0 takes the Krylov dimension from the Eq.-16 test at a tight
    eps so that the Krylov error stays far below the time-discretisation error."""
    x = x0.copy(); t = t0
    nsteps = int(round((t1 - t0) / h))
    opts = O.Options(correction=correction, eps=1e-12, m_max=circ.n)
    for _ in range(nsteps):
        x = O.er_step(circ, x, t, h, m=m, opts=opts).x
        t += h
    return x


def test_er_second_order_on_nonlinear_circuit():
    circ, x0, t0, t1 = _switching_window()
    ref = _fixed_er(circ, x0, t0, t1, 0.03125e-12)
    e = [np.max(np.abs(_fixed_er(circ, x0, t0, t1, h) - ref)) for h in (2e-12, 1e-12, 0.5e-12)]
    for a, b in zip(e[:-1], e[1:]):
        assert 3.0 < a / b < 6.0, e          # order 2: error / 4 per halving of h


def test_be_first_order_and_er_beats_be():
    circ, x0, t0, t1 = _switching_window()
    ref = _fixed_er(circ, x0, t0, t1, 0.03125e-12)

    def be(h):
        x = x0.copy()
        for k in range(int(round((t1 - t0) / h))):
            x = O.be_run(_shifted(circ, t0 + k * h), h, t_end=h, x0=x)
        return x

    e_be = [np.max(np.abs(be(h) - ref)) for h in (1e-12, 0.5e-12, 0.25e-12)]
    for a, b in zip(e_be[:-1], e_be[1:]):
        assert 1.4 < a / b < 2.6, e_be            # order 1 (pre-asymptotic above 1.4)
    e_er = np.max(np.abs(_fixed_er(circ, x0, t0, t1, 1e-12) - ref))
    assert e_er < e_be[0]                         # Fig. 2: ER more accurate than BENR at equal h


def _shifted(circ, t0):
    """Same circuit with its sources shifted so that local time 0 is global time t0."""
    pwl = []
    for tt, vv in circ.pwl:
        grid = np.unique(np.concatenate([[t0], tt[tt > t0]])) - t0
        pwl.append((grid, np.interp(grid + t0, tt, vv)))
    return S.Circuit(name=circ.name, n=circ.n, G=circ.G, C=circ.C, B=circ.B, dev=circ.dev,
                     pwl=pwl, vdd=circ.vdd, t_end=circ.t_end - t0, meta=circ.meta)


def test_error_estimate_second_order():
    circ, x0, t0, _ = _switching_window()
    opts = O.Options(eps=1e-12, m_max=circ.n)
    errs = [O.er_step(circ, x0, t0 + 5e-12, h, m=0, opts=opts).err_inf for h in (2e-12, 1e-12, 0.5e-12)]
    # dF = O(h^2) since F'(x_k) = 0; h phi_1(hJ) C^{-1} is O(h) for non-stiff modes and
    # O(1) (-> G^{-1}) for stiff ones, so e_rr falls like h^2 .. h^3
    assert errs[0] > errs[1] > errs[2] > 0
    for a, b in zip(errs[:-1], errs[1:]):
        assert 2.5 < a / b < 9.0, errs


def _err_pin_case(h):
    """A state on the first switching edge of a 3-stage chain and the oracle's ER update
    from it (Krylov dimension from Eq. 16 at eps = 1e-14: the spaces are exact)."""
    circ = S.inverter_chain(stages=3, tree_nodes=6, seed=9, t_end=1e-9)
    x0 = O.dc_solution(circ)
    t0 = 0.11e-9
    t = t0 + 3e-12
    x = _fixed_er(circ, x0, t0, t, 0.25e-12)
    opts = O.Options(eps=1e-14, m_max=circ.n)
    lin = O.linearize(circ, x)
    st = O.step_setup(circ, lin, t, O.pwl_slope(circ, t, h))
    st.K1 = O.arnoldi_iks(circ.C, lin, lin.Gk, st.v1, h, opts.eps, opts.m_max, opts.m_min)
    st.K2 = O.arnoldi_iks(circ.C, lin, lin.Gk, st.v2, h, opts.eps, opts.m_max, opts.m_min) \
        if np.any(st.v2) else None
    x_new = O.er_update(st, h)
    return circ, x, st, x_new, opts


def _dense_error_estimate(circ, x, x_new, h):
    """e_rr = -(e^{hJ} - I) G_k^{-1} dF written out densely (Eq. 15 with C^{-1} cancelled):
    J = -C^{-1} G_k, G_k = G_lin + G_dev(x_k), and dF = G_dev(x_k)(x_new - x_k)
    - (i_dev(x_new) - i_dev(x_k)), the remainder F(y) = G_dev(x_k) y - i_dev(y) with the
    device Jacobian frozen at x_k (reading of Sec. III).  scipy's expm and a dense solve
    serve as independent library steps."""
    i_k, Gdev = O.device_eval(circ, x)
    i_1, _ = O.device_eval(circ, x_new)
    Gd = Gdev.toarray()
    dF = Gd @ (x_new - x) - (i_1 - i_k)
    Gk = circ.G.toarray() + Gd
    J = -np.linalg.solve(circ.C.toarray(), Gk)
    n = circ.n
    return -(sla.expm(h * J) - np.eye(n)) @ np.linalg.solve(Gk, dF)


def _err_mismatch(err_fn, h):
    circ, x, st, x_new, opts = _err_pin_case(h)
    e = err_fn(circ, st, x_new, h, circ.C, opts)[0]
    ref = _dense_error_estimate(circ, x, x_new, h)
    assert np.max(np.abs(ref)) > 0
    return float(np.max(np.abs(e - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("h", [0.5e-12, 2e-12])
def test_error_vector_equals_dense_error_estimate(h):
    """The oracle's e_rr (Eq. 15, evaluated through one more invert-Krylov MEVP as in Eq. 19)
    equals the dense -(e^{hJ} - I) G_k^{-1} dF element by element, on two step sizes on a
    switching edge."""
    assert _err_mismatch(O.error_vector, h) <= 1e-9


def test_error_vector_pin_catches_planted_mistakes():
    """The pin above fails for the plausible slips: returning the MEVP alone (dropping v_e),
    and evaluating F(x_{k+1}) with the device Jacobian at x_{k+1} instead of x_k."""
    def mevp_only(circ, st, x_new, h, C, opts, fixed_m=0):
        e, ve, Ke = O.error_vector(circ, st, x_new, h, C, opts, fixed_m)
        return Ke.mevp(h), ve, Ke

    def jacobian_at_new_state(circ, st, x_new, h, C, opts, fixed_m=0):
        i_1, Gdev1 = O.device_eval(circ, x_new)
        dF = (Gdev1 @ x_new - i_1) - st.lin.F
        ve = st.lin.solve(dF)
        Ke = O.arnoldi_iks(C, st.lin, st.lin.Gk, ve, h, opts.eps, opts.m_max, opts.m_min,
                           fixed_m)
        return ve - Ke.mevp(h), ve, Ke

    for h in (0.5e-12, 2e-12):
        assert _err_mismatch(mevp_only, h) > 1e-3
        assert _err_mismatch(jacobian_at_new_state, h) > 1e-3


def test_linear_circuit_error_estimate_is_zero():
    circ = S.random_rc(n=10, seed=3)
    r = O.er_step(circ, np.zeros(circ.n), 0.0, 1e-12, m=5)
    assert r.err_inf == 0.0


def test_adaptive_run_one_lu_per_step_and_accuracy():
    circ = S.inverter_chain(stages=3, tree_nodes=4, seed=6, t_end=0.3e-9)
    x, t, st = O.er_run(circ, tol=1e-6)
    assert abs(t - circ.t_end) < 1e-20
    assert st.lu == st.steps                       # no LU on a rejected try
    ref = _fixed_er(circ, O.dc_solution(circ), 0.0, circ.t_end, 0.05e-12)
    assert np.max(np.abs(x - ref)) < 50 * 1e-6 * st.steps ** 0.5


def test_ercorrection_runs_and_changes_solution():
    circ, x0, t0, t1 = _switching_window()
    ref = _fixed_er(circ, x0, t0, t1, 0.03125e-12)
    a = _fixed_er(circ, x0, t0, t1, 2e-12, correction=False)
    b = _fixed_er(circ, x0, t0, t1, 2e-12, correction=True)
    assert np.max(np.abs(a - b)) > 0
    assert np.all(np.isfinite(b))


def _phi2_dense(A):
    """phi_2(A) from the exponential of the block matrix [[A, I, 0], [0, 0, I], [0, 0, 0]],
    whose top-right block is phi_2(A) (Saad 1992; Al-Mohy and Higham 2011)."""
    n = A.shape[0]
    Z = np.zeros((3 * n, 3 * n))
    Z[:n, :n] = A
    Z[:n, n:2 * n] = np.eye(n)
    Z[n:2 * n, 2 * n:] = np.eye(n)
    return sla.expm(Z)[:n, 2 * n:]


@pytest.mark.parametrize("h", [0.5e-12, 2e-12])
def test_ercorrection_equals_dense_phi2(h):
    """ER-C (Eq. 17): x_c = x_ER - D with D = gamma h phi_2(hJ) C^{-1} dF, J = -C^{-1} G_k and
    dF = F(x_ER) - F(x_k).  The oracle evaluates D in the form of Eq. 20, through one more
    invert-Krylov MEVP; here phi_2 comes from a dense block exponential instead.

    Tolerance: Eq. 20 adds (e^{hJ} - I) G^{-1} C G^{-1} dF and h G^{-1} dF, which cancel to
    order (h lambda)^2 on a slow mode lambda, so the MEVP's ~1e-13 relative error grows by
    2 / (h lambda_min)^2 (about 1e6 here at h = 0.5 ps).  1e-5 relative still fails a wrong
    sign, a dropped term, gamma or 1/h misplaced, or phi_1 in place of phi_2 by orders of
    magnitude."""
    circ, x0, t0, _ = _switching_window()
    n = circ.n
    t = t0 + 4e-12
    x = _fixed_er(circ, x0, t0, t, 0.25e-12)          # a state on the switching edge
    gamma = 0.3
    # Krylov dimension from the Eq.-16 test at eps = 1e-14 (Algorithm 1): the spaces are
    # exact once invariant.  A fixed m = n would add directions past the invariant subspace
    # whose rounding-noise Ritz values (h / mu ~ -1e13) make scaling and squaring lose the
    # slow modes (error ~ u ||h H^-1||), in the dense reference's expm as in the MEVP.
    er = O.er_step(circ, x, t, h, m=0, opts=O.Options(eps=1e-14, m_max=n))
    erc = O.er_step(circ, x, t, h, m=0,
                    opts=O.Options(eps=1e-14, m_max=n, correction=True, gamma=gamma))
    D = er.x - erc.x
    lin = O.linearize(circ, x)
    dF = lin.remainder(circ, er.x) - lin.F
    Cd = circ.C.toarray()
    J = -np.linalg.solve(Cd, lin.Gk.toarray())
    ref = gamma * h * _phi2_dense(h * J) @ np.linalg.solve(Cd, dF)
    assert np.max(np.abs(ref)) > 0
    assert np.max(np.abs(D - ref)) <= 1e-5 * np.max(np.abs(ref))
    # the correction is a second-order term: far below the error estimate's h phi_1 part
    e_rr = (sla.expm(h * J) - np.eye(n)) @ np.linalg.solve(lin.Gk.toarray(), dF)
    assert np.max(np.abs(D)) < np.max(np.abs(e_rr))


def test_rc_mesh_32x32_converges_to_exact_solution():
    """The 32x32 RC mesh workload (n = 1024, h = 1 ps) against the exact solution from the
    generalized eigenproblem G q = lambda C q, over eight steps that cross a source's ramp
    corner.  The ER step of a linear circuit with u linear on the step is exact (Eq. 13), so
    the only error is the invert-Krylov one, which the Eq.-16 test bounds through eps: the
    error has to track eps down, not sit at a floor left by a wrong term."""
    circ = S.rc_mesh_2d()
    lam, Q = sla.eigh(circ.G.toarray(), circ.C.toarray())
    QtB = Q.T @ circ.B.toarray()

    def exact(y, t, h):
        uk = circ.u(t); s = (circ.u(t + h) - uk) / h
        e = np.exp(-lam * h)
        return e * y + (QtB @ uk) * (1 - e) / lam + (QtB @ s) * (h / lam - (1 - e) / lam ** 2)

    h = 1e-12
    grid = lambda t: round(t / h) * h
    y = np.zeros(circ.n); t = 0.0
    while t < 180e-12 - 1e-18:           # 5 ps into the ramp that ends at 185 ps
        y = exact(y, t, h); t = grid(t + h)
    assert np.any((circ.breakpoints() > t) & (circ.breakpoints() < t + 8 * h))
    errs = []
    for eps in (1e-6, 1e-8):
        x = Q @ y; yy = y.copy(); tt = t; err = 0.0
        for _ in range(8):
            x = O.er_step(circ, x, tt, h, m=0, opts=O.Options(m_max=120, eps=eps)).x
            yy = exact(yy, tt, h); tt = grid(tt + h)
            xe = Q @ yy
            err = max(err, np.max(np.abs(x - xe)) / np.max(np.abs(xe)))
        errs.append(err)
    assert errs[0] <= 1e-5 and errs[1] <= 1e-6, errs
    assert errs[1] <= errs[0] / 10, errs


# --- Singular C (nodes without capacitance; Sec. IV-A, Sec. V) ---------------------------
def kron_exact_step(circ, x, t, h):
    """Exact solution over [t, t+h] of C x' = -G x + B u(t) with singular diagonal C and u
    linear on the step.  The algebraic nodes a (no capacitance) obey G_a x = (B u)_a at every
    instant; eliminating them (Kron reduction) leaves the ODE
        C_dd x_d' = -(G_dd - G_da G_aa^{-1} G_ad) x_d + (B_d - G_da G_aa^{-1} B_a) u(t),
    solved by the generalized eigenproblem; x_a follows from the constraint at t + h.  Only
    x_d of the initial state matters (an inconsistent x_a is forgotten)."""
    alg = circ.meta["algebraic"]
    dyn = np.setdiff1d(np.arange(circ.n), alg)
    G = circ.G.toarray(); C = circ.C.toarray(); B = circ.B.toarray()
    Gdd, Gda = G[np.ix_(dyn, dyn)], G[np.ix_(dyn, alg)]
    Gad, Gaa = G[np.ix_(alg, dyn)], G[np.ix_(alg, alg)]
    Gr = Gdd - Gda @ np.linalg.solve(Gaa, Gad)
    Br = B[dyn] - Gda @ np.linalg.solve(Gaa, B[alg])
    Cr = C[np.ix_(dyn, dyn)]
    lam, Q = sla.eigh(Gr, Cr)
    uk = circ.u(t); s = (circ.u(t + h) - uk) / h
    y0 = Q.T @ Cr @ x[dyn]
    f = Q.T @ Br @ uk; g = Q.T @ Br @ s
    e = np.exp(-lam * h)
    xd = Q @ (e * y0 + f * (1 - e) / lam + g * (h / lam - (1 - e) / lam ** 2))
    out = np.empty(circ.n)
    out[dyn] = xd
    out[alg] = np.linalg.solve(Gaa, B[alg] @ circ.u(t + h) - Gad @ xd)
    return out


def _linear_pieces(circ, h_max):
    bps = sorted(set([0.0] + [b for b in circ.breakpoints() if b < circ.t_end] + [circ.t_end]))
    for a, b in zip(bps[:-1], bps[1:]):
        k = max(1, int(np.ceil((b - a) / h_max - 1e-9)))
        for i in range(k):
            yield a + (b - a) * i / k, (b - a) / k


@pytest.mark.parametrize("seed,alg_source", [(0, False), (1, True), (2, False)])
def test_singular_c_step_equals_kron_reduced_solution(seed, alg_source):
    """ER step (Eq. 13) with a full invert-Krylov space on a circuit with four capacitor-free
    nodes, from an inconsistent random state, against the exact solution of the
    differential-algebraic system."""
    circ = S.random_rc(n=14, seed=seed, p=3, n_alg=4, alg_source=alg_source, t_end=30e-12)
    assert circ.C.diagonal()[circ.meta["algebraic"]].tolist() == [0.0] * 4
    x = np.random.default_rng(seed).normal(size=circ.n) * 0.1
    for t, h in [(0.0, 1e-12), (6e-12, 1e-12), (9e-12, 3e-12)]:
        nb = circ.breakpoints()
        nb = nb[nb > t + 1e-18]
        h = min(h, nb[0] - t) if nb.size else h
        r = O.er_step(circ, x, t, h, m=circ.n)
        ex = kron_exact_step(circ, x, t, h)
        assert np.max(np.abs(r.x - ex)) <= 1e-10 * np.max(np.abs(ex)), (t, h)


def test_singular_c_trajectory_and_constraints():
    """A trajectory through every source corner with the adaptive Krylov dimension (Eq.-16
    test), from an inconsistent state: it follows the exact solution, and the capacitor-free
    rows of KCL, (G x)_a = (B u)_a, hold from the first step on.  (A consistent state has
    G v_1 in the range of C, so only the first step meets the eigenvalue 0.)"""
    circ = S.random_rc(n=16, seed=5, p=3, n_alg=5, alg_source=True, t_end=30e-12)
    alg = circ.meta["algebraic"]
    G = circ.G.toarray(); B = circ.B.toarray()
    x = np.random.default_rng(5).normal(size=circ.n) * 0.1
    xe = x.copy()
    opts = O.Options(eps=1e-12, m_max=circ.n)
    for t, h in _linear_pieces(circ, 2e-12):
        x = O.er_step(circ, x, t, h, m=0, opts=opts).x
        xe = kron_exact_step(circ, xe, t, h)
        scale = np.max(np.abs(xe))
        assert np.max(np.abs(x - xe)) <= 1e-8 * scale, t
        kcl = (G @ x)[alg] - (B @ circ.u(t + h))[alg]
        assert np.max(np.abs(kcl)) <= 1e-10 * np.max(np.abs(G)) * scale, t


def _planted_hessenberg(mus, seed):
    """Upper Hessenberg H = P^T Q D Q^{-1} P (P orthogonal, from a Hessenberg reduction) with
    the eigenvalues mus, and f(H) e_1 = (P^T Q) f(D) (P^T Q)^{-1} e_1 for f(mu) = e^{h/mu}
    and g(mu) = e^{h/mu} / mu evaluated in 50-digit arithmetic from that eigendecomposition,
    with f(0) = g(0) = 0 (the limit from the stable side)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    m = len(mus)
    rng = np.random.default_rng(seed)
    Q = rng.normal(size=(m, m)) + 3 * np.eye(m)
    H, P = sla.hessenberg(Q @ np.diag(mus) @ np.linalg.inv(Q), calc_q=True)
    Qm = mp.matrix((P.T @ Q).tolist())
    Qi_e1 = Qm ** -1 * mp.matrix([1] + [0] * (m - 1))

    def apply(fun):
        d = [fun(mp.mpf(v)) if v != 0 else mp.mpf(0) for v in mus]
        return Qm * mp.matrix([d[i] * Qi_e1[i] for i in range(m)])
    return H, apply, mp


@pytest.mark.parametrize("case", ["stiff", "zero", "zero_pair"])
def test_exp_hinv_e1_with_tiny_and_zero_eigenvalues(case):
    """exp(h H^{-1}) e_1 and e_m^T H^{-1} exp(h H^{-1}) e_1 against a 50-digit evaluation
    from the eigendecomposition when H has eigenvalues at or near zero (stiff modes, and the
    exact zeros of a singular C)."""
    h = 1e-12
    base = [-3e-12, -1e-12, -5e-13, -2e-13, -8e-14, -3e-14]
    extra = {"stiff": [-h / 2000, -h / 1e6], "zero": [0.0], "zero_pair": [0.0, 0.0]}[case]
    H, apply, mp = _planted_hessenberg(base + extra, seed=len(extra))
    m = H.shape[0]
    ref_y = np.array([float(v) for v in apply(lambda mu: mp.exp(h / mu))])
    ref_g = np.array([float(v) for v in apply(lambda mu: mp.exp(h / mu) / mu)])
    y, last = O.exp_hinv_e1(H, h, singular_c=True)
    # H itself is rounded (~1e-16 ||H|| cond(Q)); both bars leave room for that, and a
    # wrong limit at mu = 0 or a lost coupling block misses them by orders of magnitude
    assert np.max(np.abs(y - ref_y)) <= 1e-12 * np.max(np.abs(ref_y)), case
    assert abs(last - ref_g[m - 1]) <= 1e-12 * np.max(np.abs(ref_g)), case


def test_adaptive_step_sequence_by_hand():
    """Algorithm 2 on a linear circuit (e_rr = 0, Eq. 15, so no try is rejected): the first
    step is h_max, a step is clipped to land on the next PWL corner or t_end, and after an
    accepted step the next one is beta = 2 times it, capped at h_max.  With h_max = 0.3 ps, a
    corner at 0.35 ps and t_end = 1 ps the steps are, worked out by hand,
    0.3 | 0.05 (lands on 0.35) | 0.1 | 0.2 | 0.3 | 0.05 (lands on 1.0) ps,
    and every accepted state is the exact solution (one node: a 1-D Krylov space)."""
    circ = S.single_rc(t_end=1e-12)
    circ.pwl = [(np.array([0.0, 0.35e-12, 1e-12]), np.array([0.0, 1e-3, 1e-3]))]
    x, t, st = O.er_run(circ, t_end=1e-12, tol=1e-6, opts=O.Options(h_max=0.3e-12),
                        x0=np.zeros(1), trace=True)
    assert np.allclose(np.array(st.hs) * 1e12, [0.3, 0.05, 0.1, 0.2, 0.3, 0.05], rtol=1e-12,
                       atol=0)
    assert np.allclose(np.array(st.ts) * 1e12, [0.3, 0.35, 0.45, 0.65, 0.95, 1.0], rtol=1e-12,
                       atol=0)
    assert st.rejects == 0 and st.lu == 1 and t == 1e-12      # G factored once (linear)
    xe = np.zeros(1); ta = 0.0
    for tb in st.ts:
        xe = exact_linear_step(circ, xe, ta, tb - ta)
        ta = tb
    assert abs(x[0] - xe[0]) <= 1e-12 * abs(xe[0])


@pytest.mark.parametrize("i_grow", [5, 1])
def test_rejection_and_growth_rule_by_hand(monkeypatch, i_grow):
    """Algorithm 2's reaction to the error test, with the estimate of Eq. 15 replaced by a
    scripted sequence of ratios err / E_rr (one per try), on a corner-free window (the first
    input edge is at 0.1 ns, h_max = 1 ps).  Worked out by hand with alpha = 1/2, beta = 2:
      step 1: ratios 2, 0.5     -> reject, accept at h_max/2 (i = 1);
      step 2: ratios 3, 3, 0.1  -> reject twice, accept at the proposal / 4 (i = 2);
      step 3: ratio 0.1         -> accept the proposal (i = 0).
    A step grows the next proposal by beta only when its retry count i < i_grow:
      i_grow = 5: proposals H, H, H/2 -> accepted H/2, H/4, H/2;
      i_grow = 1: proposals H, H/2, H/8 -> accepted H/2, H/8, H/8."""
    circ = S.inverter_chain(stages=1, tree_nodes=3, seed=9, t_end=1e-9)
    ratios = iter([2.0, 0.5, 3.0, 3.0, 0.1, 0.1])
    tol = 1e-6

    def scripted(circ_, st, x_new, h, C, opts, fixed_m=0):
        E = tol * max(1.0, float(np.max(np.abs(st.lin.x))))
        e = np.zeros(circ_.n)
        e[0] = next(ratios) * E
        return e, np.zeros(circ_.n), None

    monkeypatch.setattr(O, "error_vector", scripted)
    H = 1e-12
    _, t, st = O.er_run(circ, t_end=1e-9, tol=tol, opts=O.Options(h_max=H, i_grow=i_grow),
                        max_steps=3, trace=True)
    want = [H / 2, H / 4, H / 2] if i_grow == 5 else [H / 2, H / 8, H / 8]
    assert np.allclose(st.hs, want, rtol=1e-12, atol=0), (st.hs, want)
    assert st.rejects == 3 and st.lu == 3 and abs(t - sum(want)) <= 1e-24


def test_residual_test_can_pass_falsely_at_j1_so_m_min_is_3():
    """Why the Eq. 16 test starts at m_min = 3 rather than at j = 1 as Algorithm 1 writes it.
    Two decoupled nodes with time constants 1e-16 s and 1e-10 s, v = (1, 1e-3), h = 1 ps: the
    one-dimensional Ritz value is dominated by the fast mode, e^{h/h_11} underflows, Eq. 16
    reports a zero residual and the literal loop accepts m = 1 with the result 0, while the
    slow component should be 1e-3 e^{-0.01}.  From m_min = 2 on the answer is exact."""
    import scipy.sparse as sp
    G = sp.csr_matrix(np.eye(2))
    C = sp.csr_matrix(np.diag([1e-16, 1e-10]))

    class Identity:               # G = I: the solve is the identity
        Gk = G

        def solve(self, b):
            return np.asarray(b, float).copy()

    v = np.array([1.0, 1e-3])
    h = 1e-12
    exact = np.exp(-h / np.array([1e-16, 1e-10])) * v
    K1 = O.arnoldi_iks(C, Identity(), G, v, h, 1e-7, 2, 1, 0)
    assert K1.m == 1 and np.max(np.abs(K1.mevp(h))) == 0.0           # false convergence
    K3 = O.arnoldi_iks(C, Identity(), G, v, h, 1e-7, 2, O.Options().m_min, 0)
    assert np.max(np.abs(K3.mevp(h) - exact)) <= 1e-12 * np.max(np.abs(exact))
