"""GPU parity of 200 primal-dual iterations (Appendix A.4, Algorithm 7) against stored oracle
images, and element-wise Phi^dagger at the full size of the FP32 workload.

The stored images are written by ``tests/golden/make_pd_golden.py``, which calls only
``synth`` and the FP64 oracle.  Each test regenerates the same inputs (sky, coverage and
y = complex64(Phi x_true + sigma n) with the oracle's Phi) and runs the GPU solver with the
stored ||Phi||^2, gamma and eps.

Bars: relative L2 1e-4 on the image after 200 iterations for the FP32 path (the stated
final-image tolerance); 1e-9 for the FP64 path (every iteration is Lipschitz with constant
about 1, so rounding differences of ~1e-14 per operator grow at most linearly); Phi^dagger
element by element at 1e-5 (the stated per-application tolerance).
"""

import os

import numpy as np
import pytest

import synth
from oracle import measurement as me

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_module():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_pd_golden", os.path.join(GOLDEN, "make_pd_golden.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04502_gb300 as g
    g.library()
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _load(name):
    mk = _golden_module()
    p = mk.PROBLEMS[name]
    st = np.load(os.path.join(GOLDEN, p["file"]))
    assert int(st["n"]) == p["n"] and int(st["M"]) == p["M"] and int(st["seed"]) == p["seed"]
    x_true, uvw, geo, ops, y, sigma = mk.inputs(p["n"], p["M"], p["npts"], p["nblobs"], p["seed"])
    assert float(sigma) == pytest.approx(float(st["sigma"]), rel=1e-9)
    return mk, p, st, uvw, geo, y


@pytest.fixture(scope="module")
def small():
    return _load("small")


@pytest.fixture(scope="module")
def large():
    return _load("large")


def _solve(g, mk, p, st, uvw, y, precision):
    prec = g.F64 if precision == "f64" else g.F32
    yy = y.astype(np.complex128) if precision == "f64" else y
    plan = g.Plan(torch.from_numpy(uvw).cuda(), p["n"], J=4, S=4096, precision=prec)
    wav = g.Wavelet(p["n"], mk.LEVELS, mk.ORDERS, precision=prec)
    s = g.Solver(plan, wav, torch.from_numpy(yy).cuda(), eps=float(st["eps"]), gamma=float(st["gamma"]),
                 op_norm_sq=float(st["op_norm_sq"]), algo=g.ALGO_PD)
    s.step(int(st["iters"]))
    r = s.report()
    assert r["iters"] == int(st["iters"])
    return s.x().double().cpu().numpy(), r


@pytest.mark.parametrize("precision,tol", [("f32", 1e-4), ("f64", 1e-9)])
def test_pd_200_iterations_db1_8_256sq(g, small, precision, tol):
    """256^2 sky, M = 2e5, Dirac + db1..db8 over 4 levels: the dictionary of the FP32 workload."""
    mk, p, st, uvw, geo, y = small
    x, r = _solve(g, mk, p, st, uvw, y, precision)
    x_ref = st["x"]
    assert rel(x, x_ref) <= tol, rel(x, x_ref)
    assert r["residual_norm"] == pytest.approx(float(st["residual_norm"]), rel=max(tol, 1e-7))


def test_pd_200_iterations_full_fp32_workload(g, large):
    """1024^2 sky, 2048^2 grid, J = 4, M = 1e7, Dirac + db1..db8 over 4 levels: the image the
    FP32 path reaches after 200 iterations against the stored oracle image."""
    mk, p, st, uvw, geo, y = large
    x, r = _solve(g, mk, p, st, uvw, y, "f32")
    x_ref = st["x"].astype(np.float64)
    assert rel(x, x_ref) <= 1e-4, rel(x, x_ref)
    assert r["residual_norm"] == pytest.approx(float(st["residual_norm"]), rel=1e-4)


def test_phi_adjoint_elementwise_at_full_size(g, large):
    """Phi^dagger of the full FP32 workload (M = 1e7, the dense Gaussian uv core) against the oracle's Phi^dagger pixel by pixel, in the launch
    configuration of the benchmark, for white noise and for the data vector itself."""
    mk, p, st, uvw, geo, y = large
    plan = g.Plan(torch.from_numpy(uvw).cuda(), p["n"], J=4, S=4096)
    yin = synth.complex_normal(p["M"], seed=123).astype(np.complex64)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).double().cpu().numpy()
    ref = me.phi_adjoint(yin.astype(np.complex128), geo)
    assert rel(xa, ref) <= 1e-5, rel(xa, ref)
    # the data vector (its energy sits in the dense uv core, the heaviest tiles)
    xy = g.phi_adjoint(plan, torch.from_numpy(y).cuda()).double().cpu().numpy()
    ref_y = me.phi_adjoint(y.astype(np.complex128), geo)
    assert rel(xy, ref_y) <= 1e-5, rel(xy, ref_y)
