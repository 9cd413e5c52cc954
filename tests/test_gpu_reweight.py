"""Reweighted l1 (gbri_solver_reweight) on the GPU against the oracle: the solvers run k
iterations, set SARA weights w_i = delta / (delta + |(Psi^dagger x)_i|) from the iterate
(duals kept) and continue; bars 1e-4 (FP32 path) and 1e-9 (FP64 path) on the image."""

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


def workload(n=64, M=8000, orders=(0, 1, 2, 3), L=2, seed=3):
    x_true = synth.sky(n, 5, 3, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 2)).astype(np.complex64).astype(np.complex128)
    return n, M, orders, L, uvw, ops, y, so.epsilon_from_sigma(sigma, M)


@pytest.mark.parametrize("algo,prec,tol", [("pd", "f32", 1e-4), ("pd", "f64", 1e-9), ("admm", "f64", 1e-9),
                                           ("fista", "f64", 1e-9)])
def test_reweighted_solvers_match_oracle(g, algo, prec, tol):
    n, M, orders, L, uvw, ops, y, eps = workload()
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = so.default_gamma(y, ops[1], ops[3], opn)
    k1, k2 = 30, 30
    delta = 1e-3 * float(np.max(np.abs(ops[3](ops[1](y))))) / opn
    if algo == "pd":
        x_ref, _ = so.primal_dual(y, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=k1 + k2,
                                                       reweight=(k1, delta)))
        kw = dict(algo=g.ALGO_PD, eps=eps, gamma=gamma)
    elif algo == "admm":
        x_ref, _ = so.admm(y, *ops, so.ADMMParams(gamma=gamma, eps=eps, rho=1.0 / opn, max_iter=k1 + k2,
                                                  reweight=(k1, delta)))
        kw = dict(algo=g.ALGO_ADMM, eps=eps, gamma=gamma)
    else:
        gf = 1e-3 * float(np.max(np.abs(ops[3](ops[1](y)))))
        x_ref, _ = so.fista(y, *ops, so.FISTAParams(gamma=gf, lam=1.0 / opn, max_iter=k1 + k2, reweight=(k1, delta)))
        kw = dict(algo=g.ALGO_FISTA, gamma=gf, rho=1.0 / opn)
    F = g.F64 if prec == "f64" else g.F32
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, precision=F)
    wav = g.Wavelet(n, L, orders, precision=F)
    yd = torch.from_numpy(y if prec == "f64" else y.astype(np.complex64)).cuda()
    s = g.Solver(plan, wav, yd, op_norm_sq=opn, **kw)
    s.step(k1)
    s.reweight(delta)
    s.step(k2)
    x = s.x().cpu().numpy().astype(np.float64)
    assert rel(x, x_ref) <= tol, rel(x, x_ref)


def test_reweight_inside_a_batch(g):
    """A batch member reweighted between steps: the batch rebuilds its graph and the member's
    image equals the same solver stepped alone."""
    n, M, orders, L, uvw, ops, y, eps = workload(seed=7)
    yd = torch.from_numpy(y.astype(np.complex64)).cuda()
    mk = lambda: g.Solver(g.Plan(torch.from_numpy(uvw).cuda(), n), g.Wavelet(n, L, orders), yd, eps=eps,
                          op_norm_sq=float(M), gamma=1e-3)
    a, b, ref = mk(), mk(), mk()
    batch = g.Batch()
    batch.add(a)
    batch.add(b)
    batch.step(10)
    a.reweight(1e-3)
    batch.step(10)
    ref.step(10)
    ref.reweight(1e-3)
    ref.step(10)
    xa, xr = a.x().cpu().numpy(), ref.x().cpu().numpy()
    assert rel(xa, xr) <= 1e-6
    assert rel(b.x().cpu().numpy(), xr) > 1e-6  # the other member was not reweighted


@pytest.mark.parametrize("dtype", ["float32", "complex64", "float64", "complex128"])
def test_weighted_prox_l1_matches_oracle(g, dtype):
    from oracle import prox
    n = 50_001
    x = synth.normal(n, seed=4) * 2
    if dtype.startswith("complex"):
        x = x + 1j * synth.normal(n, seed=5)
    x = x.astype(dtype)
    w = (0.1 + synth.uniform(n, seed=6)).astype("float64" if dtype in ("float64", "complex128") else "float32")
    out = g.prox_l1_weighted(torch.from_numpy(x).cuda(), torch.from_numpy(w).cuda(), 0.7).cpu().numpy()
    ref = prox.soft_threshold(x.astype(np.complex128 if x.dtype.kind == "c" else np.float64), 0.7 * w.astype(np.float64))
    tol = 1e-6 if dtype in ("float32", "complex64") else 1e-14
    assert rel(out, ref) <= tol
    if tol < 1e-10:  # FP64: the same entries are thresholded away (FP32 may differ at |x| = lam w)
        assert np.array_equal(np.abs(out) == 0, np.abs(ref) == 0)
