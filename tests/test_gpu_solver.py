"""GPU parity of the power method and the solvers (through the C ABI) against the oracle.

Bar: the image after the solver iterations within relative L2 1e-4 of the FP64
oracle run with the same parameters (||Phi||^2, gamma, eps passed explicitly).
"""

import numpy as np
import pytest

import synth
from oracle import measurement as me, solvers as so, wavelets as wv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04502_gb300 as g
    g.library()
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem(n, M, orders, levels, seed=0, npts=5, nblobs=3):
    x_true = synth.sky(n, npts, nblobs, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, levels), lambda v: wv.psi_adjoint(v, orders, levels))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 2)).astype(np.complex64)
    return uvw, geo, ops, y, so.epsilon_from_sigma(sigma, M)


def test_power_method_matches_oracle(g):
    n, M = 64, 8000
    uvw, geo, ops, y, eps = problem(n, M, (0, 1), 2)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    val, it = g.op_norm(plan, 200, 1e-8, seed=7)
    ref, rit = so.power_iteration(ops[0], ops[1], (n, n), seed=7)
    assert val == pytest.approx(ref, rel=1e-5)


@pytest.mark.parametrize("algo,iters", [("pd", 100), ("admm", 60)])
def test_solver_iterations_match_oracle(g, algo, iters):
    """Small FP64-plain workload: 128^2 sky, M = 2e4, SARA Dirac + db1..db4, 3 levels."""
    n, M, orders, L = 128, 20_000, (0, 1, 2, 3, 4), 3
    uvw, geo, ops, y, eps = problem(n, M, orders, L)
    yd = y.astype(np.complex128)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = so.default_gamma(yd, ops[1], ops[3], opn)
    if algo == "pd":
        x_ref, info = so.primal_dual(yd, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=iters))
        kw = dict(algo=g.ALGO_PD)
    else:
        x_ref, info = so.admm(yd, *ops, so.ADMMParams(gamma=gamma, eps=eps, rho=1.0 / opn, max_iter=iters))
        kw = dict(algo=g.ALGO_ADMM)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=eps, gamma=gamma, op_norm_sq=opn, **kw)
    s.step(iters)
    x = s.x().cpu().numpy()
    assert rel(x, x_ref) <= 1e-4, rel(x, x_ref)
    r = s.report()
    assert r["iters"] == iters
    assert r["rel_change"] == pytest.approx(info["rel_change"], rel=1e-2, abs=1e-7)
    assert r["residual_norm"] == pytest.approx(np.linalg.norm(yd - ops[0](x.astype(np.float64))), rel=1e-5)


def test_default_gamma_and_op_norm_inside_solver(g):
    n, M, orders, L = 64, 6000, (0, 1, 2), 2
    uvw, geo, ops, y, eps = problem(n, M, orders, L, seed=3)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=eps, seed=0)
    r = s.report()
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n), seed=0)
    assert r["op_norm_sq"] == pytest.approx(opn, rel=1e-5)
    gam = so.default_gamma(y.astype(np.complex128), ops[1], ops[3], opn)
    assert r["gamma"] == pytest.approx(gam, rel=1e-5)


@pytest.mark.parametrize("n_balls", [0, 4])
def test_pd_forked_branches_match_serial(g, monkeypatch, n_balls):
    """A primal-dual iteration runs its wavelet branch on a second stream (graph replay and
    direct launches) and both branches on one stream while kernels are profiled.  The three
    run the same kernels on the same data; only the order of the float atomics on gridding
    tile borders differs from run to run, so the images agree to rounding (1e-5 after 40
    iterations), while a branch that read a stale iterate would be an iteration behind (the
    39-iteration image is checked to lie outside 1e-4)."""
    n, M, orders, L = 128, 20_000, (0, 1, 2, 3, 4), 3
    uvw, geo, ops, y, eps = problem(n, M, orders, L, seed=21)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    yd = torch.from_numpy(y).cuda()
    kw = dict(eps=eps, gamma=1e-3, op_norm_sq=float(g.op_norm(plan, 50, 1e-6, seed=0)[0]), n_balls=n_balls)
    xs = []
    for mode in ("graph", "direct", "profiled", "short"):
        if mode == "direct":
            monkeypatch.setenv("GBRI_GRAPHS", "0")
        s = g.Solver(plan, wav, yd, **kw)
        if mode == "profiled":
            g.profile_enable(2000)
        try:
            s.step(39 if mode == "short" else 40)
            xs.append(s.x().double().cpu().numpy())
        finally:
            if mode == "profiled":
                g.profile_enable(0)
            monkeypatch.delenv("GBRI_GRAPHS", raising=False)
        s.close()
    assert rel(xs[1], xs[0]) <= 1e-5 and rel(xs[2], xs[0]) <= 1e-5, (rel(xs[1], xs[0]), rel(xs[2], xs[0]))
    assert rel(xs[3], xs[0]) > 1e-4  # the FP64 oracle: 6.6e-4 between iterations 39 and 40


def test_pd_at_oversampling_4_matches_oracle(g):
    """n = 20 with K = 4n: the FP32 pad and primal update take their one-pixel-per-thread
    paths (n % 8 == 4), the half spectrum has K = 80 columns."""
    n, M, orders, L, os = 20, 3000, (0, 1, 2), 2, 4
    x_true = synth.sky(n, 3, 2, seed=4)
    uvw = synth.uv_coverage(M, seed=5, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, os, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=6)).astype(np.complex64)
    eps = so.epsilon_from_sigma(sigma, M)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = so.default_gamma(y.astype(np.complex128), ops[1], ops[3], opn)
    x_ref, _ = so.primal_dual(y.astype(np.complex128), *ops,
                              so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=60))
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, oversample=os)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=eps, gamma=gamma, op_norm_sq=opn)
    s.step(60)
    assert rel(s.x().cpu().numpy().astype(np.float64), x_ref) <= 1e-4


def test_pd_first_order_interpolation_matches_oracle(g):
    """Primal-dual iterations on a first-order plan against the oracle's linear mode."""
    n, M, orders, L = 64, 8000, (0, 1, 2, 3), 2
    x_true = synth.sky(n, 4, 2, seed=8)
    uvw = synth.uv_coverage(M, seed=9, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096, mode="linear")
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=10)).astype(np.complex64)
    eps = so.epsilon_from_sigma(sigma, M)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = so.default_gamma(y.astype(np.complex128), ops[1], ops[3], opn)
    x_ref, _ = so.primal_dual(y.astype(np.complex128), *ops,
                              so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=60))
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, interp_order=1)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=eps, gamma=gamma, op_norm_sq=opn)
    s.step(60)
    assert rel(s.x().cpu().numpy().astype(np.float64), x_ref) <= 1e-4


def test_pd_fused_pass_with_split_tiles_matches_oracle(g):
    """Dense small grid (heavy tiles cut into several gridding items): the primal-dual
    iteration's fused degrid + grid pass flushes those items with atomics; 30 iterations
    against the oracle."""
    n, M, orders, L = 64, 150_000, (0, 1, 2), 2
    x_true = synth.sky(n, 4, 2, seed=14)
    uvw = synth.uv_coverage(M, seed=15, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=16)).astype(np.complex64)
    eps = so.epsilon_from_sigma(sigma, M)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n), max_iter=30)  # passed to both sides
    gamma = 1e-3
    x_ref, _ = so.primal_dual(y.astype(np.complex128), *ops,
                              so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=30))
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=eps, gamma=gamma, op_norm_sq=opn)
    s.step(30)
    assert rel(s.x().cpu().numpy().astype(np.float64), x_ref) <= 1e-4


def test_solve_converges_and_is_feasible(g):
    n, M, orders, L = 64, 8000, (0, 1, 2, 3), 3
    uvw, geo, ops, y, eps = problem(n, M, orders, L, seed=11)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    x, rep = g.solve(plan, wav, torch.from_numpy(y).cuda(), eps=eps, max_iter=3000, rel_tol=1e-5, check_every=20)
    assert rep["status"] == 0 and rep["iters"] < 3000
    assert rep["residual_norm"] <= eps * 1.01
    assert float(x.min()) >= 0.0
    # the oracle's residual of the GPU image agrees with the library's FP64 norm
    xr = x.cpu().numpy().astype(np.float64)
    assert rep["residual_norm"] == pytest.approx(np.linalg.norm(y.astype(np.complex128) - ops[0](xr)), rel=1e-5)


def test_dictionary_of_the_fp32_workload_short_run(g):
    """SARA Dirac + db1..db8, 4 levels, on a 256^2 sky with 1e5 visibilities: 20 PD iterations."""
    n, M, orders, L = 256, 100_000, tuple(range(9)), 4
    uvw, geo, ops, y, eps = problem(n, M, orders, L, seed=21, npts=20, nblobs=8)
    yd = y.astype(np.complex128)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n), max_iter=50)
    gamma = so.default_gamma(yd, ops[1], ops[3], opn)
    x_ref, _ = so.primal_dual(yd, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=20))
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=eps, gamma=gamma, op_norm_sq=opn)
    s.step(20)
    assert rel(s.x().cpu().numpy(), x_ref) <= 1e-4


@pytest.mark.parametrize("prec,tol", [("f32", 1e-4), ("f64", 1e-9)])
def test_fista_matches_oracle(g, prec, tol):
    """FISTA (Algorithm 4) on the unconstrained analysis problem, 128^2 sky, M = 2e4, Dirac +
    db1..db4, 3 levels, 100 iterations with 2 DualFB inner steps: the image against the oracle
    run with the same gamma, step and starting point."""
    n, M, orders, L = 128, 20_000, (0, 1, 2, 3, 4), 3
    uvw, geo, ops, y, eps = problem(n, M, orders, L)
    yd = y.astype(np.complex128)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = 1e-3 * float(np.max(np.abs(ops[3](ops[1](yd)))))
    iters = 100
    x_ref, info = so.fista(yd, *ops, so.FISTAParams(gamma=gamma, lam=1.0 / opn, dualfb_iters=2, max_iter=iters))
    F = g.F64 if prec == "f64" else g.F32
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, precision=F)
    wav = g.Wavelet(n, L, orders, precision=F)
    ydev = torch.from_numpy(yd if prec == "f64" else y).cuda()
    s = g.Solver(plan, wav, ydev, algo=g.ALGO_FISTA, gamma=gamma, op_norm_sq=opn, rho=1.0 / opn, dualfb_iters=2)
    s.step(iters)
    x = s.x().cpu().numpy().astype(np.float64)
    assert rel(x, x_ref) <= tol, rel(x, x_ref)
    r = s.report()
    assert r["rel_change"] == pytest.approx(info["rel_change"], rel=1e-2 if prec == "f32" else 1e-6)
    assert r["residual_norm"] == pytest.approx(info["residual_norm"], rel=1e-4 if prec == "f32" else 1e-9)


@pytest.mark.parametrize("algo", ["fista", "admm"])
def test_first_order_plan_fista_and_admm_match_oracle(g, algo):
    """First-order table (reading R13) under the other solvers: FISTA runs the fused degrid +
    grid pass with its residual epilogue, ADMM the separate kernels with its epilogues; both
    against the oracle's linear mode."""
    n, M, orders, L = 64, 8000, (0, 1, 2, 3), 2
    x_true = synth.sky(n, 4, 2, seed=18)
    uvw = synth.uv_coverage(M, seed=19, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096, mode="linear")
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=20)).astype(np.complex64)
    yd = y.astype(np.complex128)
    eps = so.epsilon_from_sigma(sigma, M)
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, interp_order=1)
    wav = g.Wavelet(n, L, orders)
    if algo == "fista":
        gamma = 1e-3 * float(np.max(np.abs(ops[3](ops[1](yd)))))
        x_ref, _ = so.fista(yd, *ops, so.FISTAParams(gamma=gamma, lam=1.0 / opn, dualfb_iters=2, max_iter=60))
        s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), algo=g.ALGO_FISTA, gamma=gamma, op_norm_sq=opn,
                     rho=1.0 / opn, dualfb_iters=2)
    else:
        gamma = so.default_gamma(yd, ops[1], ops[3], opn)
        x_ref, _ = so.admm(yd, *ops, so.ADMMParams(gamma=gamma, eps=eps, rho=1.0 / opn, max_iter=60))
        s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), algo=g.ALGO_ADMM, eps=eps, gamma=gamma, op_norm_sq=opn)
    s.step(60)
    assert rel(s.x().cpu().numpy().astype(np.float64), x_ref) <= 1e-4


def test_fista_default_gamma_and_solve(g):
    n, M, orders, L = 64, 8000, (0, 1, 2), 2
    uvw, geo, ops, y, eps = problem(n, M, orders, L, seed=13)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), algo=g.ALGO_FISTA, seed=0)
    r = s.report()
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n), seed=0)
    gam = 1e-3 * float(np.max(np.abs(ops[3](ops[1](y.astype(np.complex128))))))
    assert r["gamma"] == pytest.approx(gam, rel=1e-5)
    # FISTA's momentum keeps the iterate moving on this ill-conditioned problem (the oracle's relative
    # change also levels off near 3.5e-3), so the stopping test uses 1e-2
    x, rep = g.solve(plan, wav, torch.from_numpy(y).cuda(), algo=g.ALGO_FISTA, max_iter=2000, rel_tol=1e-2,
                     check_every=5)
    assert rep["status"] == 0 and rep["iters"] < 2000 and rep["rel_change"] < 1e-2
    assert float(x.min()) >= 0.0
