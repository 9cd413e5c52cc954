"""GPU parity of the plain FP64 path (GBRI_F64 objects, through the C ABI) against the oracle,
and the mixed-precision path against the FP64 path.

Bars (derived from the arithmetic; the FP64 path rounds in a different order than the
oracle, with the same tables up to the last bit of the Bessel function):
  * Phi / Phi^dagger / Psi / Psi^dagger: relative L2 <= 1e-11.  Unit roundoff 1.1e-16,
    J^2 <= 36-term interpolation sums, log2(K^2) <= 24 FFT stages and differently rounded
    table entries (a few ulps) give errors near 1e-14; 1e-11 leaves three decades.
  * Adjoint identity Re<Phi x, y> = <x, Phi^dagger y> on the device: 1e-12 relative.
  * Solver images (100 primal-dual / 60 ADMM iterations on the 128^2, M = 2e4 plain-FP64
    workload): 1e-9.  Every step is Lipschitz with constant about 1, so rounding
    differences grow at most linearly with the iteration count.
  * Mixed precision against FP64 after 200 primal-dual iterations: 1e-4 (the stated
    final-image tolerance of the FP32 path).
"""

import numpy as np
import pytest

import synth
from oracle import measurement as me, prox, solvers as so, wavelets as wv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_OP = 1e-11
TOL_SOLVER = 1e-9


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04502_gb300 as g
    g.library()
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,M,J", [(128, 20_000, 4), (64, 5_003, 6), (96, 1_537, 4), (256, 70_001, 6)])
def test_phi_and_adjoint_fp64_match_oracle(g, n, M, J):
    x = synth.sky(n, 5, 3, seed=n) + 0.01 * synth.uniform(n * n, seed=n + 7).reshape(n, n)
    uvw = synth.uv_coverage(M, seed=n + 1, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, J, 4096)
    plan = g.Plan(dev(uvw), n, J=J, S=4096, precision=g.F64)
    assert plan.complex_dtype == torch.complex128
    y = g.phi(plan, dev(x)).cpu().numpy()
    assert y.dtype == np.complex128
    assert rel(y, me.phi(x, geo)) <= TOL_OP
    yin = synth.complex_normal(M, seed=3)
    xa = g.phi_adjoint(plan, dev(yin)).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin, geo)) <= TOL_OP
    # adjoint identity on the device alone
    lhs = float(np.real(np.vdot(yin, y)))
    rhs = float(np.dot(x.ravel(), g.phi_adjoint(plan, dev(yin)).cpu().numpy().ravel()))
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300) + 1e-12 * np.linalg.norm(x) * np.linalg.norm(yin)


def test_fp64_plan_order_and_power_method(g):
    n, M = 64, 8000
    uvw = synth.uv_coverage(M, seed=5, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    plan = g.Plan(dev(uvw), n, precision=g.F64)
    perm = plan.permutation().cpu().numpy()
    x = synth.sky(n, 5, 3, seed=2)
    y_raw = g.phi(plan, dev(x)).cpu().numpy()
    y_plan = g.phi(plan, dev(x), plan_order=True).cpu().numpy()
    assert np.array_equal(y_plan, y_raw[perm])
    assert np.array_equal(g.vis_reorder(plan, dev(y_plan), to_plan=False).cpu().numpy(), y_raw)
    val, _ = g.op_norm(plan, 200, 1e-8, seed=7)
    ref, _ = so.power_iteration(lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo), (n, n), seed=7)
    assert val == pytest.approx(ref, rel=1e-8)


@pytest.mark.parametrize("n,levels,orders", [(64, 4, tuple(range(9))), (32, 2, (8, 3, 0)), (128, 3, (0, 1, 2, 3, 4))])
def test_psi_fp64_match_oracle(g, n, levels, orders):
    wav = g.Wavelet(n, levels, orders, precision=g.F64)
    x = synth.normal(n * n, seed=n).reshape(n, n)
    al = g.psi_adjoint(wav, dev(x)).cpu().numpy()
    assert al.dtype == np.float64
    assert rel(al, wv.psi_adjoint(x, orders, levels)) <= TOL_OP
    a = synth.normal(len(orders) * n * n, seed=n + 1).reshape(len(orders), n, n)
    assert rel(g.psi(wav, dev(a)).cpu().numpy(), wv.psi(a, orders, levels)) <= TOL_OP
    assert rel(g.psi(wav, dev(al)).cpu().numpy(), x) <= 1e-13  # Psi Psi^dagger = I


def test_prox_fp64_match_oracle(g):
    n = 100_003
    x = synth.normal(n, seed=1) * 2
    out = g.prox_l1(dev(x), 0.7).cpu().numpy()
    ref = prox.soft_threshold(x, 0.7)
    assert np.array_equal(out == 0, ref == 0)  # the same entries are thresholded away
    assert rel(out, ref) <= 1e-15
    z = x + 1j * synth.normal(n, seed=2)
    outc = g.prox_l1(dev(z), 0.7).cpu().numpy()
    assert rel(outc, prox.soft_threshold(z, 0.7)) <= 1e-15
    c = synth.complex_normal(n, seed=3)
    for eps in (1.0, 1e4):
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        p = g.proj_l2ball(dev(z), dev(c), eps, norm_out=nrm).cpu().numpy()
        ref, rn = prox.proj_l2ball(z, c, eps)
        assert rel(p, ref) <= 1e-14
        assert float(nrm.item()) == pytest.approx(rn, rel=1e-13)


def test_precision_mismatch_is_rejected(g):
    n, M = 32, 500
    uvw = synth.uv_coverage(M, seed=1)
    plan = g.Plan(dev(uvw), n, precision=g.F64)
    wav = g.Wavelet(n, 2, (0, 1), precision=g.F32)
    with pytest.raises(g.GbriError):
        g.Solver(plan, wav, torch.zeros(M, dtype=torch.complex128, device="cuda"), eps=1.0, op_norm_sq=1.0,
                 gamma=1e-3)
    with pytest.raises(ValueError):  # the binding checks the dtype against the plan's precision
        g.phi(plan, torch.zeros((n, n), dtype=torch.float32, device="cuda"))


def _plain_fp64_workload():
    """128^2 sky of 5 points + 3 blobs, M = 2e4, J = 4, S = 2^12, 30 dB noise (plain FP64 workload)."""
    n, M, orders, L = 128, 20_000, (0, 1, 2, 3, 4), 3
    x_true = synth.sky(n, 5, 3, seed=0)
    uvw = synth.uv_coverage(M, seed=1, outlier_frac=0.0, weights="ones")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = y0 + sigma * synth.complex_normal(M, seed=2)
    return n, M, orders, L, uvw, ops, y, so.epsilon_from_sigma(sigma, M)


@pytest.mark.parametrize("algo,iters", [("pd", 100), ("admm", 60)])
def test_fp64_solver_matches_oracle_on_plain_workload(g, algo, iters):
    n, M, orders, L, uvw, ops, y, eps = _plain_fp64_workload()
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = so.default_gamma(y, ops[1], ops[3], opn)
    if algo == "pd":
        x_ref, info = so.primal_dual(y, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=iters))
        kw = dict(algo=g.ALGO_PD)
    else:
        x_ref, info = so.admm(y, *ops, so.ADMMParams(gamma=gamma, eps=eps, rho=1.0 / opn, max_iter=iters))
        kw = dict(algo=g.ALGO_ADMM)
    plan = g.Plan(dev(uvw), n, precision=g.F64)
    wav = g.Wavelet(n, L, orders, precision=g.F64)
    s = g.Solver(plan, wav, dev(y), eps=eps, gamma=gamma, op_norm_sq=opn, **kw)
    s.step(iters)
    x = s.x().cpu().numpy()
    assert x.dtype == np.float64
    assert rel(x, x_ref) <= TOL_SOLVER, rel(x, x_ref)
    r = s.report()
    assert r["rel_change"] == pytest.approx(info["rel_change"], rel=1e-6)
    assert r["residual_norm"] == pytest.approx(np.linalg.norm(y - ops[0](x)), rel=1e-10)


def test_fp64_defaults_match_oracle(g):
    """Power method and default gamma computed inside the FP64 solver."""
    n, M, orders, L, uvw, ops, y, eps = _plain_fp64_workload()
    plan = g.Plan(dev(uvw), n, precision=g.F64)
    wav = g.Wavelet(n, L, orders, precision=g.F64)
    r = g.Solver(plan, wav, dev(y), eps=eps, seed=0).report()
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n), seed=0)
    assert r["op_norm_sq"] == pytest.approx(opn, rel=1e-8)
    assert r["gamma"] == pytest.approx(so.default_gamma(y, ops[1], ops[3], opn), rel=1e-8)


def test_mixed_precision_matches_fp64_after_200_iterations(g):
    """256^2 sky, M = 2e5, SARA Dirac + db1..db8, 4 levels: the FP32 path's image after 200
    primal-dual iterations is within 1e-4 of the FP64 path's (same data, same parameters)."""
    n, M, orders, L = 256, 200_000, tuple(range(9)), 4
    x_true = synth.sky(n, 20, 8, seed=31)
    uvw = synth.uv_coverage(M, seed=32, outlier_frac=0.2, weights="uniform")
    p64 = g.Plan(dev(uvw), n, precision=g.F64)
    y0 = g.phi(p64, dev(x_true)).cpu().numpy()
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = y0 + sigma * synth.complex_normal(M, seed=33)
    eps = so.epsilon_from_sigma(sigma, M)
    w64 = g.Wavelet(n, L, orders, precision=g.F64)
    s64 = g.Solver(p64, w64, dev(y), eps=eps, seed=0)
    r64 = s64.report()
    p32 = g.Plan(dev(uvw), n)
    w32 = g.Wavelet(n, L, orders)
    s32 = g.Solver(p32, w32, dev(y.astype(np.complex64)), eps=eps, op_norm_sq=r64["op_norm_sq"],
                   gamma=r64["gamma"])
    s64.step(200)
    s32.step(200)
    x64 = s64.x().cpu().numpy()
    x32 = s32.x().cpu().numpy().astype(np.float64)
    assert rel(x32, x64) <= 1e-4, rel(x32, x64)
