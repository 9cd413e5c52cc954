"""Deterministic gridding (plan option ``deterministic``): Phi^dagger and the solvers give
bitwise identical results from run to run and alone or inside a batch, and stay within the
per-application tolerance of the FP64 oracle (1e-5 in FP32, 1e-11 in FP64).

The workloads put many visibilities on a small grid, so that heavy tiles are cut into
several gridding work items (the case where the default flush adds float atomics in a
run-dependent order)."""

import numpy as np
import pytest

import synth
from oracle import measurement as me, solvers as so

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


def dense(n, M, seed):
    uvw = synth.uv_coverage(M, seed=seed, outlier_frac=0.2, weights="uniform")
    y = synth.complex_normal(M, seed=seed + 1)
    return uvw, y


@pytest.mark.parametrize("taps", ["poly", "table"])
@pytest.mark.parametrize("J", [4, 6])
def test_phi_adjoint_bitwise_repeatable_fp32(g, monkeypatch, taps, J):
    n, M = 64, 300_000
    uvw, y = dense(n, M, seed=50 + J)
    if taps == "table":
        monkeypatch.setenv("GBRI_TAP_TABLE", "1")
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, deterministic=True)
    ref_plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J)
    monkeypatch.delenv("GBRI_TAP_TABLE", raising=False)
    yd = torch.from_numpy(y.astype(np.complex64)).cuda()
    outs = [g.phi_adjoint(plan, yd).cpu().numpy() for _ in range(3)]
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    xr = g.phi_adjoint(ref_plan, yd).cpu().numpy()  # default flush: same sums in another order
    assert rel(outs[0], xr) <= 1e-6
    ref = me.phi_adjoint(y.astype(np.complex64).astype(np.complex128), me.Geometry(uvw, n, 2, J, 4096))
    assert rel(outs[0], ref) <= 1e-5


def test_phi_adjoint_bitwise_repeatable_fp64(g):
    n, M = 64, 100_000
    uvw, y = dense(n, M, seed=60)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=4, precision=g.F64, deterministic=True)
    yd = torch.from_numpy(y).cuda()
    a = g.phi_adjoint(plan, yd).cpu().numpy()
    b = g.phi_adjoint(plan, yd).cpu().numpy()
    assert np.array_equal(a, b)
    ref = me.phi_adjoint(y, me.Geometry(uvw, n, 2, 4, 4096))
    assert rel(a, ref) <= 1e-11


def _pd_solver(g, n, M, seed, det=True, algo=None):
    x = synth.sky(n, 4, 2, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=0.2, weights="uniform")
    y0 = me.phi(x, me.Geometry(uvw, n, 2, 4, 4096))
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 2)).astype(np.complex64)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=4, deterministic=det)
    wav = g.Wavelet(n, 2, (0, 1, 2))
    kw = {} if algo is None else dict(algo=algo)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=so.epsilon_from_sigma(sigma, M),
                 op_norm_sq=float(M), gamma=1e-3, **kw)
    return s, plan, wav


@pytest.mark.parametrize("algo", ["pd", "fista", "admm"])
def test_solver_iterates_bitwise_repeatable(g, algo):
    a = {"pd": g.ALGO_PD, "fista": g.ALGO_FISTA, "admm": g.ALGO_ADMM}[algo]
    xs = []
    for _ in range(2):
        s, plan, wav = _pd_solver(g, 64, 200_000, seed=70, algo=a)
        s.step(25)
        xs.append(s.x().cpu().numpy())
        s.close()
    assert np.array_equal(xs[0], xs[1])


def test_batch_member_bitwise_equals_alone(g):
    """Continuous batching with deterministic plans: a member's iterates equal the same
    problem stepped alone bit for bit, while other problems share the launches."""
    alone, _, _ = _pd_solver(g, 64, 150_000, seed=80)
    mixed, _, _ = _pd_solver(g, 64, 150_000, seed=80)
    others = [_pd_solver(g, 96, 120_000, seed=90)[0], _pd_solver(g, 32, 40_000, seed=95)[0]]
    b = g.Batch()
    b.add(mixed)
    for o in others:
        b.add(o)
    b.step(12)
    torch.cuda.synchronize()
    alone.step(12)
    assert np.array_equal(alone.x().cpu().numpy(), mixed.x().cpu().numpy())
    b.close()
