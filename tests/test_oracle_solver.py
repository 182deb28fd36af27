"""Pins of the oracle's linearisation, linear algebra and LM loop.

Each check compares the oracle with something other than itself: central
finite differences of its residual through the retraction, the full stacked
normal equations solved by numpy, scipy's least-squares and minimisation
routines, brute force on tiny inputs, or an invariant of the mathematics.
A planted mistake (dropped term, wrong sign, transposed block) fails at
least one of them; see test_planted_mistakes_are_caught.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

import oracle as O
from paper_2510_15271_b300 import scenes


def _problem(s):
    return O.Problem.from_arrays(s.intrinsics(), s.obs_cam, s.obs_pt, s.obs_uv, s.cam_fixed,
                                 s.n_cams, s.n_pts)


def _tiny(seed=3, n_cams=3, n_pts=12, views=3, **kw):
    s = scenes.make_scene("ring", seed=seed, n_cams=n_cams, n_pts=n_pts, views=views, **kw)
    return s, _problem(s), O.state_from_qt(s.cam_qt, s.pts)


# --------------------------------------------------------------------------- Jacobians

def _fd_jacobians(prob, st, h=1e-6):
    """Central differences of r_k through the same perturbations the solver
    uses (left SE(3) on cameras, additive on points)."""
    N = prob.n_obs
    Jc = np.zeros((N, 2, 6))
    Jp = np.zeros((N, 2, 3))
    for a in range(6):
        d = np.zeros((prob.n_cams, 6))
        d[:, a] = h
        rp, _, _ = O.residuals(prob, O.retract(st, d, np.zeros((prob.n_pts, 3))))
        rm, _, _ = O.residuals(prob, O.retract(st, -d, np.zeros((prob.n_pts, 3))))
        Jc[:, :, a] = (rp - rm) / (2 * h)
    for a in range(3):
        d = np.zeros((prob.n_pts, 3))
        d[:, a] = h
        rp, _, _ = O.residuals(prob, O.retract(st, np.zeros((prob.n_cams, 6)), d))
        rm, _, _ = O.residuals(prob, O.retract(st, np.zeros((prob.n_cams, 6)), -d))
        Jp[:, :, a] = (rp - rm) / (2 * h)
    return Jc, Jp


@pytest.mark.parametrize("name,kw", [
    ("ring", dict(n_cams=8, n_pts=200)),
    ("driving", dict(n_cams=40, n_pts=2000, length_m=80.0)),
])
def test_jacobians_match_central_differences(name, kw):
    s = scenes.make_scene(name, seed=11, **kw)
    prob = _problem(s)
    prob.cam_fixed[:] = False
    st = O.state_from_qt(s.cam_qt, s.pts)
    _, _, Jc, Jp = O.linearize(prob, st, 1.0)
    Fc, Fp = _fd_jacobians(prob, st)
    rel_c = np.linalg.norm(Jc - Fc) / np.linalg.norm(Fc)
    rel_p = np.linalg.norm(Jp - Fp) / np.linalg.norm(Fp)
    assert rel_c <= 1e-6 and rel_p <= 1e-6, (rel_c, rel_p)


def test_fixed_cameras_have_no_camera_jacobian():
    s, prob, st = _tiny()
    _, _, Jc, _ = O.linearize(prob, st, 0.0)
    assert np.all(Jc[prob.cam_fixed[prob.obs_cam]] == 0)
    assert np.any(Jc[~prob.cam_fixed[prob.obs_cam]] != 0)


# --------------------------------------------------------------------------- Huber

def test_huber_weight_is_the_derivative_of_rho():
    s = np.linspace(1e-3, 25.0, 2001)
    for delta in (0.5, 1.0, 1.5):
        h = 1e-6
        num = (O.huber_rho(s + h, delta) - O.huber_rho(s - h, delta)) / (2 * h)
        away = np.abs(s - delta * delta) > 2 * h
        np.testing.assert_allclose(O.huber_weight(s, delta)[away], num[away], rtol=1e-7)


def test_huber_is_quadratic_inside_linear_outside():
    # inside the threshold rho is the plain squared norm; outside, rho grows
    # linearly in the residual norm: rho(4s) + d^2 = 2 (rho(s) + d^2)
    d = 1.5
    s_in = np.linspace(0.0, d * d, 50)
    np.testing.assert_array_equal(O.huber_rho(s_in, d), s_in)
    s_out = np.linspace(d * d * 1.01, 100.0, 50)
    np.testing.assert_allclose(O.huber_rho(4 * s_out, d) + d * d,
                               2 * (O.huber_rho(s_out, d) + d * d), rtol=1e-13)
    # continuous at the threshold and below plain least squares beyond it
    assert abs(O.huber_rho(np.array([d * d * (1 + 1e-12)]), d)[0] - d * d) < 1e-9
    assert np.all(O.huber_rho(s_out, d) < s_out)


def test_huber_with_infinite_threshold_is_least_squares():
    s, prob, st = _tiny(seed=4, n_cams=6, n_pts=60)
    assert O.cost(prob, st, 1e9) == pytest.approx(O.cost(prob, st, 0.0), rel=1e-15)
    r1 = O.lm_solve(prob, st, O.LMOptions(huber_delta=1e9, lm_iters=4))
    r0 = O.lm_solve(prob, st, O.LMOptions(huber_delta=0.0, lm_iters=4))
    np.testing.assert_allclose(r1.costs, r0.costs, rtol=1e-12)


# --------------------------------------------------------------------------- normal equations

def _fd_normal_equations(prob, st, delta):
    """A and g from the stacked finite-difference Jacobian (free cameras then
    points) and the IRLS weights."""
    r, w, _, _ = O.linearize(prob, st, delta)
    Fc, Fp = _fd_jacobians(prob, st)
    free = np.nonzero(~prob.cam_fixed)[0]
    pos = -np.ones(prob.n_cams, dtype=int)
    pos[free] = np.arange(free.size)
    n = 6 * free.size + 3 * prob.n_pts
    J = np.zeros((2 * prob.n_obs, n))
    for k in range(prob.n_obs):
        i = pos[prob.obs_cam[k]]
        if i >= 0:
            J[2 * k:2 * k + 2, 6 * i:6 * i + 6] = Fc[k]
        o = 6 * free.size + 3 * prob.obs_pt[k]
        J[2 * k:2 * k + 2, o:o + 3] = Fp[k]
    ww = np.repeat(w, 2)
    return J.T @ (ww[:, None] * J), J.T @ (ww * r.ravel())


def test_full_normal_equations_match_finite_difference_build():
    s, prob, st = _tiny(seed=5, n_cams=3, n_pts=15, huber_delta=1.0)
    A, g = O.full_normal_equations(prob, st, 1.0)
    Af, gf = _fd_normal_equations(prob, st, 1.0)
    assert np.linalg.norm(A - Af) / np.linalg.norm(Af) < 1e-6
    assert np.linalg.norm(g - gf) / np.linalg.norm(gf) < 1e-6


@pytest.mark.parametrize("mu", [1e-4, 1.0])
@pytest.mark.parametrize("delta", [0.0, 0.7])
def test_schur_step_equals_full_normal_equation_step(mu, delta):
    """Eliminating the points through the Schur complement gives the same step
    as solving (A + mu D) h = -g over all unknowns (numpy.linalg.solve)."""
    s, prob, st = _tiny(seed=6, n_cams=3, n_pts=20, sigma=2.0)
    opts = O.LMOptions(huber_delta=delta, solver="dense")
    r, w, Jc, Jp = O.linearize(prob, st, delta)
    U, V, W, gc, gp = O.block_sums(prob, r, w, Jc, Jp)
    lin = dict(U=U, V=V, W=W, gc=gc, gp=gp)
    dc, dp, D, g, h, _ = O.solve_step(prob, lin, mu, opts)
    A, g_full = O.full_normal_equations(prob, st, delta)
    Dg = np.maximum(np.diag(A), O.DIAG_MIN)
    h_full = np.linalg.solve(A + mu * np.diag(Dg), -g_full)
    np.testing.assert_allclose(h, h_full, rtol=1e-9, atol=1e-12 * np.abs(h_full).max())
    np.testing.assert_allclose(g, g_full, rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(D, Dg, rtol=1e-12)


def test_schur_matrix_is_the_dense_elimination():
    s, prob, st = _tiny(seed=7, n_cams=4, n_pts=10)
    r, w, Jc, Jp = O.linearize(prob, st, 0.0)
    U, V, W, gc, gp = O.block_sums(prob, r, w, Jc, Jp)
    Us, Vs, _, _ = O.damped_blocks(U, V, 0.1)
    S, b, _, _ = O.schur_system(prob, Us, Vs, W, gc, gp)
    A, g = O.full_normal_equations(prob, st, 0.0)
    Dg = np.maximum(np.diag(A), O.DIAG_MIN)
    Ad = A + 0.1 * np.diag(Dg)
    nc = S.shape[0]
    Acc, Acp, App = Ad[:nc, :nc], Ad[:nc, nc:], Ad[nc:, nc:]
    S_ref = Acc - Acp @ np.linalg.solve(App, Acp.T)
    b_ref = -g[:nc] + Acp @ np.linalg.solve(App, g[nc:])
    np.testing.assert_allclose(S, S_ref, rtol=1e-10, atol=1e-9 * np.abs(S_ref).max())
    np.testing.assert_allclose(b, b_ref, rtol=1e-10, atol=1e-9 * np.abs(b_ref).max())


# --------------------------------------------------------------------------- PCG

def test_pcg_matches_cholesky_on_spd_system():
    rng = np.random.Generator(np.random.PCG64(8))
    M = rng.normal(size=(60, 60))
    S = M @ M.T + 60 * np.eye(60)
    b = rng.normal(size=60)
    x, k, rel = O.pcg_block_jacobi(S, b, 1e-12, 500)
    x_ref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(S), b)
    np.testing.assert_allclose(x, x_ref, rtol=1e-9)
    assert rel <= 1e-12 and 0 < k <= 60


def test_block_jacobi_is_exact_on_block_diagonal_system():
    rng = np.random.Generator(np.random.PCG64(9))
    blocks = []
    for _ in range(7):
        M = rng.normal(size=(6, 6))
        blocks.append(M @ M.T + np.eye(6))
    S = scipy.linalg.block_diag(*blocks)
    b = rng.normal(size=42)
    x, k, rel = O.pcg_block_jacobi(S, b, 1e-14, 50)
    assert k == 1
    np.testing.assert_allclose(S @ x, b, rtol=1e-12, atol=1e-12)


def test_pcg_zero_right_hand_side_takes_no_iterations():
    x, k, rel = O.pcg_block_jacobi(np.eye(12), np.zeros(12), 1e-6, 100)
    assert k == 0 and not x.any()


def test_pcg_counts_products_and_respects_the_cap():
    rng = np.random.Generator(np.random.PCG64(10))
    M = rng.normal(size=(120, 120))
    S = M @ M.T + 1e-3 * np.eye(120)
    b = rng.normal(size=120)
    _, k, rel = O.pcg_block_jacobi(S, b, 1e-14, 7)
    assert k == 7 and rel > 1e-14


def test_refinement_with_one_step_is_plain_pcg():
    rng = np.random.Generator(np.random.PCG64(11))
    M = rng.normal(size=(90, 90))
    S = M @ M.T + 1e-2 * np.eye(90)
    b = rng.normal(size=90)
    x1, k1, r1 = O.pcg_block_jacobi(S, b, 1e-3, 40)
    x2, k2, r2 = O.pcg_refined(S, b, 1e-3, 40, 1, 1e-12)
    np.testing.assert_array_equal(x1, x2)
    assert k1 == k2 and r2 == pytest.approx(r1, rel=1e-12)


def test_refinement_reaches_its_tolerance_and_the_direct_solution():
    """Loose inner solves (tol 1e-2) refined until the residual, recomputed
    here by numpy, is below 1e-10 relative; the solution is then within
    kappa(S) times that of the Cholesky solution."""
    rng = np.random.Generator(np.random.PCG64(12))
    M = rng.normal(size=(120, 120))
    S = M @ M.T + 0.5 * np.eye(120)
    b = rng.normal(size=120)
    x, k, rel = O.pcg_refined(S, b, 1e-2, 500, 20, 1e-10)
    true_rel = np.linalg.norm(b - S @ x) / np.linalg.norm(b)
    assert true_rel <= 1e-10 and rel == pytest.approx(true_rel, rel=1e-9)
    x_ref = scipy.linalg.cho_solve(scipy.linalg.cho_factor(S), b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= np.linalg.cond(S) * true_rel
    # each outer step cut the residual: more than one step was needed
    _, _, rel1 = O.pcg_refined(S, b, 1e-2, 500, 1, 1e-10)
    assert rel1 > 1e-4 and k > 0


def test_refined_lm_step_on_a_tiny_scene_is_the_direct_step():
    """In the LM loop, a refined PCG step with a tight outer tolerance is the
    dense Cholesky step (same costs to 1e-10)."""
    s = scenes.make_scene("city", seed=13, n_cams=12, n_pts=500)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    ref = O.lm_solve(prob, st, O.LMOptions(huber_delta=1.5, lm_iters=4, solver="dense"))
    res = O.lm_solve(prob, st, O.LMOptions(huber_delta=1.5, lm_iters=4, solver="pcg",
                                           pcg_tol=1e-3, pcg_max_iters=30, refine_max=30,
                                           refine_tol=1e-13))
    np.testing.assert_allclose(res.costs, ref.costs, rtol=1e-10)
    assert np.all(res.pcg_iters > 30)


# --------------------------------------------------------------------------- LM

@pytest.mark.parametrize("name,kw,opts", [
    ("ring", dict(n_cams=10, n_pts=400), dict(solver="dense", huber_delta=0.0)),
    ("driving", dict(n_cams=50, n_pts=3000, length_m=100.0),
     dict(solver="pcg", huber_delta=1.0)),
])
def test_lm_cost_monotone_and_model_consistent(name, kw, opts):
    s = scenes.make_scene(name, seed=12, **kw)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    res = O.lm_solve(prob, st, O.LMOptions(lm_iters=8, **opts))
    assert np.all(np.diff(res.costs) <= 0)
    assert res.accepted[0]
    assert res.costs[-1] < 0.6 * res.costs[0]
    # an accepted step's gain ratio is the measured over the predicted decrease
    for i in np.nonzero(res.accepted)[0]:
        pred = res.dL[i]
        assert pred > 0
        assert res.gain[i] == pytest.approx((res.costs[i] - res.costs[i + 1]) / pred, rel=1e-12)


def test_all_cameras_fixed_is_independent_point_refinement():
    """With every camera fixed the problem separates into one small least
    squares per point; scipy's least_squares on each point alone reaches the
    same minimum."""
    s = scenes.make_scene("ring", seed=13, n_cams=6, n_pts=25, views=4, sigma=1.0)
    prob = _problem(s)
    prob.cam_fixed[:] = True
    st = O.state_from_qt(s.cam_qt_gt, s.pts)
    res = O.lm_solve(prob, st, O.LMOptions(lm_iters=25, solver="dense"))
    np.testing.assert_array_equal(res.state.R, st.R)
    np.testing.assert_array_equal(res.state.t, st.t)
    for j in range(prob.n_pts):
        sel = prob.obs_pt == j

        def fun(X, sel=sel):
            xc = np.einsum("nij,j->ni", st.R[prob.obs_cam[sel]], X) + st.t[prob.obs_cam[sel]]
            return (np.stack([prob.fx * xc[:, 0] / xc[:, 2] + prob.cx,
                              prob.fy * xc[:, 1] / xc[:, 2] + prob.cy], 1)
                    - prob.obs_uv[sel]).ravel()
        ref = scipy.optimize.least_squares(fun, st.X[j], method="lm", xtol=1e-15, ftol=1e-15,
                                           gtol=1e-15)
        np.testing.assert_allclose(res.state.X[j], ref.x, atol=1e-7)


def _stacked_problem(prob, st0):
    """Residual function of all free unknowns around st0 (cameras through
    the left retraction) for scipy's independent solvers."""
    free = np.nonzero(~prob.cam_fixed)[0]

    def unpack(x):
        dc = np.zeros((prob.n_cams, 6))
        dc[free] = x[:6 * free.size].reshape(-1, 6)
        return O.retract(st0, dc, x[6 * free.size:].reshape(-1, 3))

    def fun(x):
        r, _, _ = O.residuals(prob, unpack(x))
        return r.ravel()
    return fun, 6 * free.size + 3 * prob.n_pts, unpack


def test_lm_reaches_scipy_least_squares_minimum_on_micro_scene():
    s = scenes.make_scene("ring", seed=14, n_cams=3, n_pts=10, views=3, sigma=0.8)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    res = O.lm_solve(prob, st, O.LMOptions(lm_iters=60, solver="dense"))
    fun, n, _ = _stacked_problem(prob, st)
    ref = scipy.optimize.least_squares(fun, np.zeros(n), method="trf", x_scale="jac",
                                       xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    assert res.costs[-1] == pytest.approx(ref.cost, rel=1e-7)


def test_lm_huber_reaches_scipy_minimiser_on_micro_scene():
    s = scenes.make_scene("ring", seed=15, n_cams=3, n_pts=10, views=3, sigma=2.0)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    delta = 1.0
    res = O.lm_solve(prob, st, O.LMOptions(lm_iters=80, solver="dense", huber_delta=delta))
    fun, n, _ = _stacked_problem(prob, st)

    def F(x):
        r = fun(x).reshape(-1, 2)
        s2 = np.sum(r * r, axis=1)
        return 0.5 * np.sum(np.where(s2 <= delta * delta, s2,
                                     2 * delta * np.sqrt(s2) - delta * delta))
    x0 = np.zeros(n)
    ref = scipy.optimize.minimize(F, x0, method="BFGS", options=dict(gtol=1e-10, maxiter=20000))
    assert res.costs[-1] <= ref.fun * (1 + 1e-6)
    assert res.costs[-1] >= ref.fun * (1 - 1e-5)


def test_cost_is_invariant_to_a_similarity_of_the_scene():
    """Rotating, translating and scaling the whole scene leaves every pixel
    residual unchanged (the 7-DoF gauge)."""
    s = scenes.make_scene("ring", seed=16, n_cams=8, n_pts=200)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    Q = O.so3_exp(np.array([[0.3, -0.2, 0.9]]))[0]
    c, d = 3.0, np.array([10.0, -4.0, 2.0])
    # X' = c Q X + d; camera x_c = R X + t = R Q^T (X' - d)/c + t
    R2 = st.R @ Q.T
    t2 = c * st.t - np.einsum("nij,j->ni", R2, d)
    st2 = O.State(R2, t2, c * st.X @ Q.T + d)
    assert O.cost(prob, st2, 1.0) == pytest.approx(O.cost(prob, st, 1.0), rel=1e-12)


def test_rejected_step_keeps_state_and_raises_damping():
    s = scenes.make_scene("ring", seed=17, n_cams=8, n_pts=300)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    res = O.lm_solve(prob, st, O.LMOptions(lm_iters=20, solver="dense"))
    rej = np.nonzero(~res.accepted)[0]
    assert rej.size > 0
    for i in rej:
        assert res.costs[i + 1] == res.costs[i]
        if i + 1 < len(res.mu):
            assert res.mu[i + 1] > res.mu[i]


# --------------------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the oracle trips one of the pins above."""
    s = scenes.make_scene("ring", seed=18, n_cams=5, n_pts=40)
    prob = _problem(s)
    prob.cam_fixed[:] = False
    st = O.state_from_qt(s.cam_qt, s.pts)
    Fc, Fp = _fd_jacobians(prob, st)
    good_lin = O.linearize

    def flipped_rotation_part(p, x, d):
        r, w, Jc, Jp = good_lin(p, x, d)
        Jc = Jc.copy()
        Jc[:, :, 3:] *= -1.0          # wrong sign of the rotational Jacobian
        return r, w, Jc, Jp

    def transposed_point_part(p, x, d):
        r, w, Jc, Jp = good_lin(p, x, d)
        Rt = np.transpose(x.R[p.obs_cam], (0, 2, 1))
        D = Jp @ Rt                   # recover dr/dx_c, then use R^T instead of R
        return r, w, Jc, D @ Rt

    for bad in (flipped_rotation_part, transposed_point_part):
        _, _, Jc, Jp = bad(prob, st, 0.0)
        err = max(np.linalg.norm(Jc - Fc) / np.linalg.norm(Fc),
                  np.linalg.norm(Jp - Fp) / np.linalg.norm(Fp))
        assert err > 1e-3, bad.__name__
    # a dropped damping term changes the step that the full system predicts
    r, w, Jc, Jp = O.linearize(prob, st, 0.0)
    U, V, W, gc, gp = O.block_sums(prob, r, w, Jc, Jp)
    lin = dict(U=U, V=V, W=W, gc=gc, gp=gp)
    _, _, _, _, h, _ = O.solve_step(prob, lin, 0.5, O.LMOptions(solver="dense"))
    monkeypatch.setattr(O, "damped_blocks",
                        lambda U_, V_, mu: (U_, V_ + mu * np.eye(3),
                                            np.maximum(np.diagonal(U_, axis1=1, axis2=2), 1e-12),
                                            np.maximum(np.diagonal(V_, axis1=1, axis2=2), 1e-12)))
    import oracle.ba_oracle as OB
    monkeypatch.setattr(OB, "damped_blocks", O.damped_blocks)
    _, _, _, _, h_bad, _ = OB.solve_step(prob, lin, 0.5, O.LMOptions(solver="dense"))
    assert np.linalg.norm(h_bad - h) > 1e-6 * np.linalg.norm(h)


# --------------------------------------------------------------------------- gain ratio and damping
#
# Each pin below is a helper that raises AssertionError when the oracle is
# wrong, so that the planted-slip test can run it against a broken oracle.

def _check_model_decrease(O_):
    """The predicted decrease of an LM step is L(0) - L(h) of the
    Gauss-Newton model L(h) = F + g^T h + 1/2 h^T A h (Madsen, Nielsen &
    Tingleff 2004, Sec. 3.2), evaluated here from its definition with the
    full stacked normal equations (A, g pinned against finite differences
    above) and numpy's solve of the damped system (A + mu D) h = -g.  The
    oracle's closed form eliminates A through the damped system, so the two
    agree only if neither the 1/2 nor a sign is lost."""
    s, prob, st = _tiny(seed=21, n_cams=3, n_pts=15, sigma=1.5)
    for delta in (0.0, 1.0):
        A, g = O_.full_normal_equations(prob, st, delta)
        D = np.maximum(np.diag(A), O_.DIAG_MIN)
        for mu in (1e-4, 0.3, 20.0):
            h = np.linalg.solve(A + mu * np.diag(D), -g)
            ref = -(g @ h) - 0.5 * h @ A @ h
            assert ref > 0
            assert O_.model_decrease(h, D, g, mu) == pytest.approx(ref, rel=1e-9), (delta, mu)
        # the LM loop reaches the same value through the Schur route
        res = O_.lm_solve(prob, st, O_.LMOptions(huber_delta=delta, lm_iters=1, solver="dense",
                                                 mu0=0.3))
        h = np.linalg.solve(A + 0.3 * np.diag(D), -g)
        assert res.dL[0] == pytest.approx(-(g @ h) - 0.5 * h @ A @ h, rel=1e-8), delta


def _check_small_step_gain(O_):
    """The Gauss-Newton model agrees with F to first order, so the gain ratio
    (measured over predicted decrease) tends to 1 as heavy damping shrinks the
    step, the gap shrinking like 1/mu.  With a dropped 1/2 in the predicted
    decrease it would tend to 1/2, with a flipped sign to -1."""
    s, prob, st = _tiny(seed=22, n_cams=4, n_pts=30, sigma=1.0)
    for delta in (0.0, 1.0):
        gaps = []
        for mu0 in (1e2, 1e3, 1e4):
            res = O_.lm_solve(prob, st, O_.LMOptions(huber_delta=delta, lm_iters=1,
                                                     solver="dense", mu0=mu0))
            gaps.append(abs(res.gain[0] - 1.0))
        assert gaps[-1] < 2e-3, (delta, gaps)
        assert gaps[0] > gaps[1] > gaps[2], (delta, gaps)
        assert gaps[1] / gaps[2] > 5.0, (delta, gaps)   # about tenfold per decade of mu


# (gain ratio, factor on mu) of an accepted step: max(1/3, 1 - (2 gain - 1)^3)
_NIELSEN_ACCEPTED = [
    (1.0, 1.0 / 3.0),     # the model predicted the decrease exactly
    (0.95, 1.0 / 3.0),    # 1 - 0.9^3 = 0.271, held at the lower bound 1/3
    (0.9, 0.488),         # 1 - 0.8^3
    (0.75, 0.875),        # 1 - 0.5^3
    (0.5, 1.0),           # halfway: damping unchanged
    (0.25, 1.125),        # 1 + 0.5^3
    (1e-12, 2.0),         # a barely useful step doubles the damping
]


def _check_damping_update(O_):
    """Nielsen's update (Madsen, Nielsen & Tingleff 2004, eq. 3.16 and the nu
    rule that follows it), as literal values of its published form."""
    for gain, factor in _NIELSEN_ACCEPTED:
        mu, nu = O_.damping_update(3.0, 8.0, gain, True)
        assert mu == pytest.approx(3.0 * factor, rel=1e-9), (gain, mu / 3.0, factor)
        assert nu == 2.0
    # a rejected step multiplies mu by nu and doubles nu, whatever the gain
    for gain in (-np.inf, -0.5, 0.7):
        assert O_.damping_update(3.0, 8.0, gain, False) == (24.0, 16.0)
    # reject, reject, accept exactly: 1e-4 -> 2e-4 -> 8e-4 -> 8e-4 / 3, nu 2 -> 4 -> 8 -> 2
    mu, nu = 1e-4, 2.0
    mu, nu = O_.damping_update(mu, nu, -1.0, False)
    mu, nu = O_.damping_update(mu, nu, -1.0, False)
    assert (mu, nu) == (pytest.approx(8e-4, rel=1e-15), 8.0)
    mu, nu = O_.damping_update(mu, nu, 1.0, True)
    assert (mu, nu) == (pytest.approx(8e-4 / 3.0, rel=1e-15), 2.0)


def test_model_decrease_is_the_decrease_of_the_quadratic_model():
    _check_model_decrease(O)


def test_gain_ratio_tends_to_one_as_the_step_shrinks():
    _check_small_step_gain(O)


def test_damping_update_matches_its_published_form():
    _check_damping_update(O)


def test_lm_loop_applies_the_pinned_damping_update():
    """The damping each iteration uses follows from the previous iteration's
    damping, gain ratio and decision through the pinned update (nu tracked
    alongside), over a run with accepted and rejected steps."""
    s = scenes.make_scene("ring", seed=17, n_cams=8, n_pts=300)
    prob = _problem(s)
    res = O.lm_solve(prob, O.state_from_qt(s.cam_qt, s.pts), O.LMOptions(lm_iters=20,
                                                                         solver="dense"))
    assert res.accepted.any() and (~res.accepted).any()
    assert res.mu[0] == O.LMOptions().mu0
    nu = O.LMOptions().nu0
    for k in range(len(res.mu) - 1):
        mu_next, nu = O.damping_update(res.mu[k], nu, res.gain[k], bool(res.accepted[k]))
        assert res.mu[k + 1] == mu_next, k


def test_damping_floor_holds_mu_and_is_inert_when_zero():
    """mu_min floors the damping after accepted steps only; with 0 (the
    default) the run is the plain schedule bit for bit."""
    s = scenes.make_scene("ring", seed=17, n_cams=8, n_pts=300)
    prob = _problem(s)
    st = O.state_from_qt(s.cam_qt, s.pts)
    plain = O.lm_solve(prob, st, O.LMOptions(lm_iters=12, solver="dense"))
    zero = O.lm_solve(prob, st, O.LMOptions(lm_iters=12, solver="dense", mu_min=0.0))
    np.testing.assert_array_equal(plain.costs, zero.costs)
    assert plain.mu.min() < 1e-4
    floored = O.lm_solve(prob, st, O.LMOptions(lm_iters=12, solver="dense", mu_min=1e-4))
    assert floored.mu.min() == pytest.approx(1e-4, rel=1e-15)
    nu = 2.0
    for k in range(len(floored.mu) - 1):
        mu_next, nu = O.damping_update(floored.mu[k], nu, floored.gain[k],
                                       bool(floored.accepted[k]))
        if floored.accepted[k]:
            mu_next = max(mu_next, 1e-4)
        assert floored.mu[k + 1] == mu_next, k


def test_planted_slips_in_gain_ratio_and_damping_are_caught(monkeypatch):
    """A dropped 1/2 or a flipped sign in the predicted decrease, and a wrong
    exponent or bound in the damping update, each fail a pin above."""
    import oracle.ba_oracle as OB
    good_dl = OB.model_decrease
    for bad in (lambda h, D, g, mu: 2.0 * good_dl(h, D, g, mu),      # 1/2 dropped
                lambda h, D, g, mu: 0.5 * float(h @ (mu * D * h + g))):  # sign of g flipped
        with monkeypatch.context() as m:
            m.setattr(OB, "model_decrease", bad)
            for pin in (_check_model_decrease, _check_small_step_gain):
                with pytest.raises(AssertionError):
                    pin(OB)
    good_du = OB.damping_update
    for bad in (lambda mu, nu, gain, acc: (mu * max(1 / 3, 1 - (2 * gain - 1) ** 2), 2.0)
                if acc else (mu * nu, 2 * nu),                        # square, not cube
                lambda mu, nu, gain, acc: (mu * max(1 / 2, 1 - (2 * gain - 1) ** 3), 2.0)
                if acc else (mu * nu, 2 * nu),                        # bound 1/2, not 1/3
                lambda mu, nu, gain, acc: good_du(mu, nu, gain, acc) if acc
                else (mu * nu, nu)):                                  # nu not doubled
        with monkeypatch.context() as m:
            m.setattr(OB, "damping_update", bad)
            with pytest.raises(AssertionError):
                _check_damping_update(OB)
