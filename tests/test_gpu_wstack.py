"""GPU parity of the w-stacking operator (gbri_wstack_*, reading R14) against the oracle's
w-stacking (``oracle.wstack``): Phi and Phi^dagger within 1e-5 (FP32) and 1e-11 (FP64)
relative L2, the same plane assignment, empty planes, the coplanar reduction (w = 0), and the
adjoint identity on the device."""

import numpy as np
import pytest

import synth
from oracle import wstack as ws

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


@pytest.mark.parametrize("precision,tol", [("f32", 1e-5), ("f64", 1e-11)])
@pytest.mark.parametrize("n,M,J,planes,delta", [(64, 20_000, 4, 8, 0.01), (96, 9_000, 6, 3, 0.006),
                                                 (128, 30_001, 4, 16, 0.005)])
def test_wstack_matches_oracle(g, precision, tol, n, M, J, planes, delta):
    uvw = synth.uvw_noncoplanar(M, seed=n + planes, delta=delta, w_frac=0.5)
    x = synth.sky(n, 5, 3, seed=n) + 0.01 * synth.uniform(n * n, seed=n + 1).reshape(n, n)
    st = ws.WStack(uvw, n, delta, planes, J=J)
    prec = g.F64 if precision == "f64" else g.F32
    w = g.WStack(torch.from_numpy(uvw).cuda(), n, planes, delta, J=J, precision=prec)
    counts, centres = w.info()
    assert np.array_equal(counts, [len(ix) for ix in st.idx])
    assert np.allclose(centres, st.centres, rtol=0, atol=1e-9 * max(1.0, np.abs(centres).max()))
    x_in = x.astype(np.float32) if precision == "f32" else x
    y = w.phi(torch.from_numpy(x_in).cuda()).cpu().numpy()
    y_ref = ws.phi(x_in.astype(np.float64), st)
    assert rel(y, y_ref) <= tol, rel(y, y_ref)
    yin = synth.complex_normal(M, seed=n + 7)
    yd = torch.from_numpy(yin.astype(np.complex128 if precision == "f64" else np.complex64)).cuda()
    xa = w.phi_adjoint(yd).cpu().numpy()
    xa_ref = ws.phi_adjoint(yd.cpu().numpy().astype(np.complex128), st)
    assert rel(xa, xa_ref) <= tol, rel(xa, xa_ref)
    w.close()


def test_wstack_empty_planes_and_coplanar_reduction(g):
    n, M = 64, 6000
    uvw = synth.uv_coverage(M, seed=3, outlier_frac=0.2, weights="uniform")
    # two clusters of w with a gap: the middle planes are empty
    uvw[: M // 2, 2] = -20.0
    uvw[M // 2:, 2] = 30.0
    x = synth.sky(n, 4, 2, seed=4).astype(np.float32)
    w = g.WStack(torch.from_numpy(uvw).cuda(), n, 6, 0.01)
    counts, _ = w.info()
    assert counts.sum() == M and (counts == 0).sum() == 4
    st = ws.WStack(uvw, n, 0.01, 6)
    y = w.phi(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, ws.phi(x.astype(np.float64), st)) <= 1e-5
    w.close()
    # w = 0 everywhere: one populated plane with the unit screen = the coplanar plan
    uvw[:, 2] = 0.0
    w0 = g.WStack(torch.from_numpy(uvw).cuda(), n, 4, 0.01)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    xd = torch.from_numpy(x).cuda()
    assert rel(w0.phi(xd).cpu().numpy(), g.phi(plan, xd).cpu().numpy()) <= 1e-6
    yin = torch.from_numpy(synth.complex_normal(M, seed=5).astype(np.complex64)).cuda()
    assert rel(w0.phi_adjoint(yin).cpu().numpy(), g.phi_adjoint(plan, yin).cpu().numpy()) <= 1e-6
    w0.close()


def test_wstack_adjoint_identity_on_device(g):
    n, M = 128, 50_000
    uvw = synth.uvw_noncoplanar(M, seed=9, delta=0.004, w_frac=0.5)
    w = g.WStack(torch.from_numpy(uvw).cuda(), n, 12, 0.004, precision=g.F64)
    x = torch.from_numpy(synth.uniform(n * n, seed=10).reshape(n, n)).cuda()
    yin = torch.from_numpy(synth.complex_normal(M, seed=11)).cuda()
    lhs = torch.real(torch.vdot(w.phi(x), yin))
    rhs = torch.dot(x.ravel(), w.phi_adjoint(yin).ravel())
    assert abs(float(lhs - rhs)) <= 1e-12 * abs(float(lhs))
    w.close()


def test_wstack_rejects_bad_arguments(g):
    uvw = torch.from_numpy(synth.uvw_noncoplanar(100, seed=1, delta=0.01)).cuda()
    with pytest.raises(g.GbriError):
        g.WStack(uvw, 64, 0, 0.01)          # no planes
    with pytest.raises(g.GbriError):
        g.WStack(uvw, 64, 4, 0.03)          # 64 pixels of 0.03 reach the horizon
