"""Pins for the oracle's solvers: closed-form special case, an independent constrained solver,
the dense operator norm, and the counter-based generator."""

import numpy as np
import pytest
from scipy.optimize import minimize

import synth
from oracle import measurement as me, solvers as so, wavelets as wv


def test_splitmix64_published_sequence():
    # first outputs of SplitMix64 from state 0 (reference sequence of the published generator)
    assert so.splitmix64(4, 0) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                                   0xF88BB8A8724C81EC]
    u = so.splitmix64_uniform(1000, 5)
    assert np.all((u >= 0) & (u < 1)) and abs(u.mean() - 0.5) < 0.05


def _closed_form(y, eps):
    """min ||x||_1 s.t. ||y - x|| <= eps, x >= 0  ->  x = max(y - lam, 0), lam by bisection."""
    lo, hi = 0.0, float(np.abs(y).max())
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.linalg.norm(y - np.maximum(y - mid, 0)) < eps:
            lo = mid
        else:
            hi = mid
    return np.maximum(y - lo, 0)


def test_identity_operator_special_case_pd_and_admm():
    y = synth.normal(200, seed=1) + 0.5
    eps = 0.5 * np.linalg.norm(np.maximum(y, 0))
    xs = _closed_form(y, eps)
    ident = lambda x: x.astype(complex)
    ident_t = lambda z: np.real(z)
    dirac = lambda a: a[0]
    dirac_t = lambda x: x[None]
    for gamma in (0.05, 1.0):
        x, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                              so.PDParams(gamma=gamma, op_norm_sq=1.0, eps=eps, max_iter=20000, rel_tol=1e-14))
        assert np.max(np.abs(x - xs)) < 1e-8
        x, _ = so.admm(y.astype(complex), ident, ident_t, dirac, dirac_t,
                       so.ADMMParams(gamma=gamma, eps=eps, rho=1.0, max_iter=20000, rel_tol=1e-14))
        assert np.max(np.abs(x - xs)) < 1e-8


def _tiny_problem():
    n, M = 8, 40
    x_true = np.zeros((n, n))
    x_true[3, 4], x_true[5, 2], x_true[2, 2] = 1.0, 0.5, 0.3
    uvw = synth.uv_coverage(M, seed=1, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    orders, L = (0, 1, 2), 2
    ops = (lambda x: me.phi(np.reshape(x, (n, n)), geo), lambda y: me.phi_adjoint(y, geo),
           lambda a: wv.psi(a, orders, L), lambda x: wv.psi_adjoint(x, orders, L))
    y0 = ops[0](x_true)
    sigma = 0.05 * np.linalg.norm(y0) / np.sqrt(M)
    y = y0 + sigma * synth.complex_normal(M, seed=2)
    return n, M, ops, y, so.epsilon_from_sigma(sigma, M)


def test_power_iteration_matches_dense_norm():
    n, M, (phi, phit, _, _), _, _ = _tiny_problem()
    A = np.stack([phi(e.reshape(n, n)) for e in np.eye(n * n)], 1)
    Ar = np.vstack([A.real, A.imag])       # Phi acts on real images
    val, _ = so.power_iteration(phi, phit, (n, n), seed=0)
    assert val == pytest.approx(np.linalg.norm(Ar, 2) ** 2, rel=1e-6)


def test_primal_dual_matches_independent_constrained_solver():
    """SLSQP on the LP-with-one-quadratic-constraint form of the analysis problem."""
    n, M, (phi, phit, psi, psit), y, eps = _tiny_problem()
    N = n * n
    A = np.stack([phi(e.reshape(n, n)) for e in np.eye(N)], 1)
    P = np.stack([psit(e.reshape(n, n)).ravel() for e in np.eye(N)], 1)
    Ar, yr = np.vstack([A.real, A.imag]), np.concatenate([y.real, y.imag])
    K = P.shape[0]
    G = np.block([[P, -np.eye(K)], [-P, -np.eye(K)]])        # |Psi^dagger x| <= t

    def qc(z):
        r = Ar @ z[:N] - yr
        return np.array([eps ** 2 - r @ r])

    def qcj(z):
        g = np.zeros((1, N + K))
        g[0, :N] = -2 * Ar.T @ (Ar @ z[:N] - yr)
        return g

    res = minimize(lambda z: z[N:].sum(), np.zeros(N + K), jac=lambda z: np.r_[np.zeros(N), np.ones(K)],
                   method="SLSQP", bounds=[(0, None)] * (N + K),
                   constraints=[{"type": "ineq", "fun": lambda z: -(G @ z), "jac": lambda z: -G},
                                {"type": "ineq", "fun": qc, "jac": qcj}],
                   options={"maxiter": 2000, "ftol": 1e-14})
    opn, _ = so.power_iteration(phi, phit, (n, n))
    gamma = so.default_gamma(y, phit, psit, opn)
    x, info = so.primal_dual(y, phi, phit, psi, psit,
                             so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=30000, rel_tol=1e-13))
    assert np.max(np.abs(x.ravel() - res.x[:N])) < 1e-6
    assert np.abs(psit(x)).sum() == pytest.approx(res.fun, rel=1e-7)
    assert info["residual_norm"] <= eps * (1 + 1e-6)
    assert np.all(x >= 0)


def test_pd_and_admm_reach_the_same_constrained_solution():
    n, M = 16, 400
    x_true = synth.sky(n, 3, 1, seed=3)
    uvw = synth.uv_coverage(M, seed=4, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    orders, L = (0, 1, 2), 2
    phi = lambda x: me.phi(x, geo)
    phit = lambda y: me.phi_adjoint(y, geo)
    psi = lambda a: wv.psi(a, orders, L)
    psit = lambda x: wv.psi_adjoint(x, orders, L)
    y0 = phi(x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = y0 + sigma * synth.complex_normal(M, seed=5)
    eps = so.epsilon_from_sigma(sigma, M)
    opn, _ = so.power_iteration(phi, phit, (n, n))
    gamma = so.default_gamma(y, phit, psit, opn, factor=1e-2)
    xp, ip = so.primal_dual(y, phi, phit, psi, psit,
                            so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=20000, rel_tol=1e-10))
    # Algorithm 1's DualFB is an inexact inner prox; with enough inner iterations its fixed point is the
    # constrained minimiser that the primal-dual iteration reaches.
    xa, ia = so.admm(y, phi, phit, psi, psit,
                     so.ADMMParams(gamma=gamma, eps=eps, rho=1.0 / opn, max_iter=20000, rel_tol=1e-10,
                                   dualfb_iters=20))
    assert np.linalg.norm(xp - xa) / np.linalg.norm(xp) < 5e-4
    for info, x in ((ip, xp), (ia, xa)):
        assert info["residual_norm"] <= eps * (1 + 1e-3)
        assert np.all(x >= 0)
    # the primal-dual objective is the smaller one (both are feasible)
    assert np.abs(psit(xp)).sum() <= np.abs(psit(xa)).sum() * (1 + 1e-9)


def test_fista_identity_operator_closed_form():
    """Phi = I, Psi = Dirac: min 1/2 ||y - x||^2 + gamma ||x||_1, x >= 0 has x = max(y - gamma, 0);
    with Psi = Dirac one DualFB step is the exact prox."""
    y = synth.normal(300, seed=7) + 0.3
    ident = lambda x: x.astype(complex)
    ident_t = lambda z: np.real(z)
    dirac = lambda a: a[0]
    dirac_t = lambda x: x[None]
    for gamma, lam in ((0.2, 1.0), (0.7, 0.4)):
        x, info = so.fista(y.astype(complex), ident, ident_t, dirac, dirac_t,
                           so.FISTAParams(gamma=gamma, lam=lam, max_iter=5000, rel_tol=1e-15))
        assert np.max(np.abs(x - np.maximum(y - gamma, 0))) < 1e-10
        assert info["iters"] < 5000


def _tiny_unconstrained(orders, L):
    n, M, (phi, phit, _, _), y, _ = _tiny_problem()
    psi = lambda a: wv.psi(a, orders, L)
    psit = lambda x: wv.psi_adjoint(x, orders, L)
    N = n * n
    A = np.stack([phi(e.reshape(n, n)) for e in np.eye(N)], 1)
    P = np.stack([psit(e.reshape(n, n)).ravel() for e in np.eye(N)], 1)
    Ar, yr = np.vstack([A.real, A.imag]), np.concatenate([y.real, y.imag])
    K = P.shape[0]
    G = np.block([[P, -np.eye(K)], [-P, -np.eye(K)]])
    gamma = 0.02 * float(np.max(np.abs(psit(phit(y)))))

    def obj(z):
        r = Ar @ z[:N] - yr
        return 0.5 * r @ r + gamma * z[N:].sum()

    def jac(z):
        return np.r_[Ar.T @ (Ar @ z[:N] - yr), gamma * np.ones(K)]

    # SLSQP on the smooth form min 1/2 ||A x - y||^2 + gamma sum t, -t <= Psi^dagger x <= t, x >= 0
    res = minimize(obj, np.zeros(N + K), jac=jac, method="SLSQP", bounds=[(0, None)] * (N + K),
                   constraints=[{"type": "ineq", "fun": lambda z: -(G @ z), "jac": lambda z: -G}],
                   options={"maxiter": 3000, "ftol": 1e-15})
    opn, _ = so.power_iteration(phi, phit, (n, n))
    return n, (phi, phit, psi, psit), y, gamma, opn, res


def test_fista_matches_independent_unconstrained_solver():
    """Dirac dictionary (the DualFB prox is exact in one step): FISTA's gradient steps and
    extrapolation reach the minimiser that SLSQP finds for the smooth reformulation."""
    n, (phi, phit, psi, psit), y, gamma, opn, res = _tiny_unconstrained((0,), 1)
    N = n * n
    x, info = so.fista(y, phi, phit, psi, psit,
                       so.FISTAParams(gamma=gamma, lam=1.0 / opn, max_iter=50000, rel_tol=1e-14))
    assert np.max(np.abs(x.ravel() - res.x[:N])) < 1e-6
    f = so.fista_objective(x, y, phi, psit, gamma)
    assert f == pytest.approx(res.fun, rel=1e-10)
    assert np.all(x >= 0)
    x10, _ = so.fista(y, phi, phit, psi, psit, so.FISTAParams(gamma=gamma, lam=1.0 / opn, max_iter=10))
    assert so.fista_objective(x10, y, phi, psit, gamma) > f  # descends overall


def test_fista_with_sara_dictionary_approaches_the_minimiser():
    """Dirac + db1 + db2 over 2 levels: with an inexact DualFB prox (30 inner iterations) the
    objective comes within 1e-5 of the SLSQP minimum."""
    n, (phi, phit, psi, psit), y, gamma, opn, res = _tiny_unconstrained((0, 1, 2), 2)
    x, info = so.fista(y, phi, phit, psi, psit,
                       so.FISTAParams(gamma=gamma, lam=1.0 / opn, dualfb_iters=30, max_iter=400))
    f = so.fista_objective(x, y, phi, psit, gamma)
    assert f == pytest.approx(res.fun, rel=1e-5)
    assert np.all(x >= 0)


def test_local_balls_identity_operator_closed_form_and_global_feasibility():
    """Phi = I, Psi = Dirac, the visibilities split into blocks: the problem separates, each block
    has the closed form max(y_j - lam_j, 0) for its own radius eps_j; the local solution also lies
    in the global ball of radius sqrt(sum eps_j^2) (Sec. 6.9).  One block is the global ball."""
    y = np.abs(synth.normal(240, seed=11)) + 0.1  # positive data: every block's constraint is feasible
    idx = np.array_split(np.random.default_rng(3).permutation(240), 4)
    eps_j = [0.5 * np.linalg.norm(y[i]) for i in idx]
    xs = np.zeros_like(y)
    for i, e in zip(idx, eps_j):
        xs[i] = _closed_form(y[i], e)
    ident = lambda x: x.astype(complex)
    ident_t = lambda z: np.real(z)
    dirac = lambda a: a[0]
    dirac_t = lambda x: x[None]
    balls = list(zip(idx, eps_j))
    eps = float(np.sqrt(np.sum(np.square(eps_j))))
    for gamma in (0.05, 0.5):
        x, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                              so.PDParams(gamma=gamma, op_norm_sq=1.0, eps=eps, max_iter=20000, rel_tol=1e-14,
                                          balls=balls))
        assert np.max(np.abs(x - xs)) < 1e-8
        xa, _ = so.admm(y.astype(complex), ident, ident_t, dirac, dirac_t,
                        so.ADMMParams(gamma=gamma, eps=eps, rho=1.0, max_iter=20000, rel_tol=1e-14, balls=balls))
        assert np.max(np.abs(xa - xs)) < 1e-8
    assert np.linalg.norm(y - x) <= eps * (1 + 1e-9)       # inside the global ball
    for i, e in balls:
        assert np.linalg.norm(y[i] - x[i]) <= e * (1 + 1e-9)
    # a single block with the whole index set is the global ball
    xg, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                           so.PDParams(gamma=0.2, op_norm_sq=1.0, eps=eps, max_iter=300))
    x1, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                           so.PDParams(gamma=0.2, op_norm_sq=1.0, eps=eps, max_iter=300,
                                       balls=[(np.arange(240), eps)]))
    assert np.array_equal(xg, x1)


def test_product_of_balls_projection_is_the_blockwise_projection():
    """proj_balls onto {||z_j - y_j|| <= eps_j}: every block is inside its ball, blocks inside
    their ball are unchanged, and the variational inequality <z - p, q - p> <= 0 holds for
    random feasible q (p is the nearest feasible point)."""
    rng = np.random.default_rng(5)
    z = synth.complex_normal(90, seed=8) * 3
    y = synth.complex_normal(90, seed=9)
    idx = np.array_split(rng.permutation(90), 3)
    eps_j = [1.0, 50.0, 2.0]
    p = so.proj_balls(z, y, None, list(zip(idx, eps_j)))
    for i, e in zip(idx, eps_j):
        assert np.linalg.norm(p[i] - y[i]) <= e * (1 + 1e-12)
    assert np.array_equal(p[idx[1]], z[idx[1]])
    for _ in range(200):
        q = y.copy()
        for i, e in zip(idx, eps_j):
            d = rng.normal(size=len(i)) + 1j * rng.normal(size=len(i))
            q[i] = y[i] + d / np.linalg.norm(d) * e * rng.uniform() ** 0.5
        assert np.real(np.vdot(z - p, q - p)) <= 1e-9


def test_weighted_l1_closed_form_and_unit_weights():
    """Phi = I, Psi = Dirac, weights w: min sum w_i x_i s.t. ||y - x|| <= eps, x >= 0 has
    x_i = max(y_i - lam w_i, 0) with lam by bisection; unit weights give the unweighted run."""
    y = np.abs(synth.normal(200, seed=21)) + 0.1
    w = 0.2 + synth.uniform(200, seed=22)
    eps = 0.5 * np.linalg.norm(y)
    lo, hi = 0.0, float(np.max(y / w))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if np.linalg.norm(y - np.maximum(y - mid * w, 0)) < eps:
            lo = mid
        else:
            hi = mid
    xs = np.maximum(y - lo * w, 0)
    ident = lambda x: x.astype(complex)
    ident_t = lambda z: np.real(z)
    dirac = lambda a: a[0]
    dirac_t = lambda x: x[None]
    x, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                          so.PDParams(gamma=0.05, op_norm_sq=1.0, eps=eps, max_iter=30000, rel_tol=1e-14,
                                      weights=w[None]))
    assert np.max(np.abs(x - xs)) < 1e-8
    xa, _ = so.admm(y.astype(complex), ident, ident_t, dirac, dirac_t,
                    so.ADMMParams(gamma=0.05, eps=eps, rho=1.0, max_iter=30000, rel_tol=1e-14, weights=w[None]))
    assert np.max(np.abs(xa - xs)) < 1e-8
    x1, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                           so.PDParams(gamma=0.05, op_norm_sq=1.0, eps=eps, max_iter=200, weights=np.ones((1, 200))))
    x0, _ = so.primal_dual(y.astype(complex), ident, ident_t, dirac, dirac_t,
                           so.PDParams(gamma=0.05, op_norm_sq=1.0, eps=eps, max_iter=200))
    assert np.array_equal(x1, x0)


def test_sara_weights():
    x = synth.normal(64, seed=3).reshape(8, 8)
    psit = lambda v: wv.psi_adjoint(v, (0, 1), 2)
    w = so.sara_weights(x, psit, 0.1)
    a = np.abs(psit(x))
    assert w.shape == a.shape and np.all((w > 0) & (w <= 1))
    assert np.allclose(w, 0.1 / (0.1 + a), rtol=0, atol=0)
    assert np.all(np.diff(w.ravel()[np.argsort(a.ravel())]) <= 0)  # larger coefficients, smaller weights
    assert np.all(so.sara_weights(np.zeros((8, 8)), psit, 0.1) == 1.0)


# ---- pins of the parameter rules (gamma, eps, SARA weights) against hand-computed values ----

def test_default_gamma_hand_computed():
    """gamma = 1e-3 max|Psi^dagger Phi^dagger y| / ||Phi||^2 (reading R8) on cases worked by hand."""
    # Phi = I (adjoint takes the real part), Psi = Dirac: max|Re y| = 2, ||Phi||^2 = 4
    y = np.array([0.5, -2.0 + 0.3j, 1.0])
    ident_t = lambda z: np.real(z)
    dirac_t = lambda x: x[None]
    assert so.default_gamma(y, ident_t, dirac_t, 4.0) == pytest.approx(5e-4, rel=1e-15)
    assert so.default_gamma(y, ident_t, dirac_t, 4.0, factor=0.1) == pytest.approx(0.05, rel=1e-15)
    # 2 x 2 image, Dirac + Haar (db1) over one level, stack scaled by 1/sqrt(2): the Haar LL
    # coefficient of [[1, 2], [3, 4]] is (1 + 2 + 3 + 4) / 2 = 5, so max = 5 / sqrt(2);
    # with ||Phi||^2 = 2: gamma = 1e-3 * 5 / (2 sqrt(2))
    y4 = np.array([1.0, 2.0, 3.0, 4.0], dtype=complex)
    g = so.default_gamma(y4, lambda z: np.real(z).reshape(2, 2), lambda v: wv.psi_adjoint(v, (0, 1), 1), 2.0)
    assert g == pytest.approx(0.0017677669529663686, rel=1e-14)


def test_default_gamma_with_brute_force_adjoint():
    """The dirty image inside gamma is Phi^dagger y: the oracle's gridding adjoint (J = 6) and the
    adjoint of the brute-force measurement equation (Eq. 1, conjugate exponentials) give the
    same gamma to the gridding error."""
    n, M = 16, 300
    uvw = synth.uv_coverage(M, seed=11, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 6, 4096)
    y = synth.complex_normal(M, seed=12)
    c = np.arange(n, dtype=np.float64) - n // 2
    u, v, w = (np.asarray(uvw[:, k], dtype=np.float64) for k in (0, 1, 3))

    def brute_adj(z):  # x[q, p] = Re sum_i w_i z_i exp(+i (u_i p' + v_i q'))
        return np.real(np.einsum("m,mq,mp->qp", w * z, np.exp(1j * v[:, None] * c[None, :]),
                                 np.exp(1j * u[:, None] * c[None, :])))

    psit = lambda x: wv.psi_adjoint(x, (0, 1, 2), 2)
    g_grid = so.default_gamma(y, lambda z: me.phi_adjoint(z, geo), psit, 3.0)
    g_brute = so.default_gamma(y, brute_adj, psit, 3.0)
    assert g_grid == pytest.approx(g_brute, rel=1e-3)


def test_epsilon_from_sigma_chi_square_rule():
    """eps^2 / sigma^2 = mean + 2 std of ||n||^2 / sigma^2 for n_i ~ CN(0, sigma^2): that ratio is
    chi^2 with 2M degrees of freedom halved (scipy's moments); a hand value; and a Monte-Carlo
    draw of the synthetic noise covers eps with the chi-square probability."""
    from scipy.stats import chi2
    for M in (1, 100, 20_000, 10_000_000):
        d = chi2(2 * M)
        ref = 0.7 * np.sqrt(d.mean() / 2 + 2 * d.std() / 2)
        assert so.epsilon_from_sigma(0.7, M) == pytest.approx(ref, rel=1e-13)
    assert so.epsilon_from_sigma(0.5, 100) == pytest.approx(0.5 * np.sqrt(120.0), rel=1e-15)  # 5.4772...
    M, draws, sigma = 400, 4000, 0.3
    n = sigma * synth.complex_normal(M * draws, seed=9).reshape(draws, M)
    sq = np.sum(np.abs(n) ** 2, axis=1)
    assert np.mean(sq) == pytest.approx(M * sigma ** 2, rel=0.01)
    assert np.std(sq) == pytest.approx(np.sqrt(M) * sigma ** 2, rel=0.05)
    covered = np.mean(np.sqrt(sq) <= so.epsilon_from_sigma(sigma, M))
    p = chi2.cdf(2 * M + 4 * np.sqrt(M), 2 * M)  # about 0.977
    assert abs(covered - p) < 0.012  # 5 binomial standard deviations


def test_sara_weights_hand_computed():
    """w = delta / (delta + |Psi^dagger x|) on [[1, 2], [3, 4]] with Dirac + Haar over one level
    (stack scaled by 1/sqrt(2)), delta = 1/2.  Coefficients: Dirac x / sqrt(2); Haar LL 5, HL -1,
    LH -2, HH 0, over sqrt(2).  So the weights are 1 / (1 + sqrt(2) |c sqrt(2)|) by hand."""
    x = np.array([[1.0, 2.0], [3.0, 4.0]])
    w = so.sara_weights(x, lambda v: wv.psi_adjoint(v, (0, 1), 1), 0.5)
    r2 = np.sqrt(2.0)
    expect = np.array([[[r2 - 1, 1 / (1 + 2 * r2)], [1 / (1 + 3 * r2), 1 / (1 + 4 * r2)]],
                       [[1 / (1 + 5 * r2), r2 - 1], [1 / (1 + 2 * r2), 1.0]]])
    assert np.allclose(w, expect, rtol=1e-13, atol=1e-15)
    assert expect[0, 0, 0] == pytest.approx(0.4142135623730951, rel=1e-15)
    assert expect[1, 0, 0] == pytest.approx(0.12389934309929541, rel=1e-15)
