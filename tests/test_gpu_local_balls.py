"""Local l2-ball constraints (Sec. 6.9) on the GPU against the oracle.

The library cuts its plan order at tile boundaries into n_balls ranges (rule in
include/gbri.h); the test derives the same partition independently from the oracle's
FP64 quantisation (tiles heaviest first, ties by index) and runs the oracle's primal-dual
and ADMM with the per-block balls eps_j = eps sqrt(M_j / M).  Bars: 1e-4 (FP32 path) and
1e-9 (FP64 path) on the image, as for the global ball.
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


def ball_partition(uvw, n, nb, S=4096, T=16):
    """Caller-order index sets of the library's local balls."""
    K = 2 * n
    kx = me.quantise(uvw[:, 0], K, S)
    ky = me.quantise(uvw[:, 1], K, S)
    cx = np.mod(np.floor_divide(kx, S), K)
    cy = np.mod(np.floor_divide(ky, S), K)
    tile = (cy // T) * (K // T) + cx // T
    counts = np.bincount(tile, minlength=(K // T) ** 2)
    tiles = np.nonzero(counts)[0]
    order = tiles[np.argsort(-counts[tiles], kind="stable")]
    M = len(uvw)
    balls, cur, cum = [], [], 0
    for t in order:
        cur.append(t)
        cum += int(counts[t])
        if len(balls) < nb - 1 and cum * nb >= (len(balls) + 1) * M:
            balls.append(cur)
            cur = []
    balls.append(cur)
    assert len(balls) == nb
    return [np.nonzero(np.isin(tile, b))[0] for b in balls]


def workload(n=128, M=20_000, orders=(0, 1, 2, 3, 4), L=3, seed=0):
    x_true = synth.sky(n, 5, 3, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, orders, L), lambda v: wv.psi_adjoint(v, orders, L))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = y0 + sigma * synth.complex_normal(M, seed=seed + 2)
    return n, M, orders, L, uvw, ops, y, so.epsilon_from_sigma(sigma, M)


@pytest.mark.parametrize("algo,iters,prec,tol", [("pd", 100, "f32", 1e-4), ("admm", 60, "f32", 1e-4),
                                                 ("pd", 100, "f64", 1e-9), ("admm", 60, "f64", 1e-9)])
def test_local_balls_match_oracle(g, algo, iters, prec, tol):
    nb = 4
    n, M, orders, L, uvw, ops, y, eps = workload()
    idx = ball_partition(uvw, n, nb)
    balls = [(i, eps * np.sqrt(len(i) / M)) for i in idx]
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n))
    gamma = so.default_gamma(y, ops[1], ops[3], opn)
    if prec == "f32":
        y = y.astype(np.complex64).astype(np.complex128)  # both sides see the same data
    if algo == "pd":
        x_ref, _ = so.primal_dual(y, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=iters,
                                                       balls=balls))
        kw = dict(algo=g.ALGO_PD)
    else:
        x_ref, _ = so.admm(y, *ops, so.ADMMParams(gamma=gamma, eps=eps, rho=1.0 / opn, max_iter=iters, balls=balls))
        kw = dict(algo=g.ALGO_ADMM)
    F = g.F64 if prec == "f64" else g.F32
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, precision=F)
    wav = g.Wavelet(n, L, orders, precision=F)
    yd = torch.from_numpy(y if prec == "f64" else y.astype(np.complex64)).cuda()
    s = g.Solver(plan, wav, yd, eps=eps, gamma=gamma, op_norm_sq=opn, n_balls=nb, **kw)
    s.step(iters)
    x = s.x().cpu().numpy().astype(np.float64)
    assert rel(x, x_ref) <= tol, rel(x, x_ref)
    # the local solution differs from the global-ball one (the constraint changed)
    s2 = g.Solver(plan, wav, yd, eps=eps, gamma=gamma, op_norm_sq=opn, **kw)
    s2.step(iters)
    assert rel(s2.x().cpu().numpy().astype(np.float64), x) > 10 * tol


def test_local_balls_with_split_tiles(g):
    """Dense small grid (heavy tiles cut into several gridding items): the per-ball scale in
    the gridding source is taken per item; PD with 4 balls against the oracle."""
    nb = 4
    n, M, orders, L, uvw, ops, y, eps = workload(n=64, M=150_000, orders=(0, 1, 2), L=2, seed=13)
    idx = ball_partition(uvw, n, nb)
    balls = [(i, eps * np.sqrt(len(i) / M)) for i in idx]
    opn, _ = so.power_iteration(ops[0], ops[1], (n, n), max_iter=30)  # passed to both sides
    gamma = so.default_gamma(y, ops[1], ops[3], opn)
    y = y.astype(np.complex64).astype(np.complex128)
    x_ref, _ = so.primal_dual(y, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=30, balls=balls))
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y.astype(np.complex64)).cuda(), eps=eps, gamma=gamma,
                 op_norm_sq=opn, n_balls=nb)
    s.step(30)
    assert rel(s.x().cpu().numpy().astype(np.float64), x_ref) <= 1e-4


def test_local_balls_reach_local_feasibility(g):
    """Converged PD with 8 local balls: every block inside its ball, hence the data inside the
    global ball of radius sqrt(sum eps_j^2) = eps (Sec. 6.9)."""
    nb = 8
    n, M, orders, L, uvw, ops, y, eps = workload(n=64, M=8000, orders=(0, 1, 2), L=2, seed=5)
    idx = ball_partition(uvw, n, nb)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    x, rep = g.solve(plan, wav, torch.from_numpy(y.astype(np.complex64)).cuda(), eps=eps, n_balls=nb,
                     max_iter=4000, rel_tol=1e-5, check_every=20)
    assert rep["status"] == 0
    xr = x.cpu().numpy().astype(np.float64)
    r = y - ops[0](xr)
    for i in idx:
        assert np.linalg.norm(r[i]) <= eps * np.sqrt(len(i) / M) * 1.01
    assert np.linalg.norm(r) <= eps * 1.01


def test_local_ball_arguments_rejected(g):
    n, M, orders, L, uvw, ops, y, eps = workload(n=32, M=500, orders=(0, 1), L=2, seed=9)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    wav = g.Wavelet(n, L, orders)
    yd = torch.from_numpy(y.astype(np.complex64)).cuda()
    with pytest.raises(g.GbriError):
        g.Solver(plan, wav, yd, eps=eps, op_norm_sq=1.0, gamma=1e-3, n_balls=65)
    with pytest.raises(g.GbriError):  # more balls than the plan has tiles
        g.Solver(plan, wav, yd, eps=eps, op_norm_sq=1.0, gamma=1e-3, n_balls=64)
