"""Batched execution (gbri_batch_*): independent problems of different sizes stepped together
in one graph launch give the same iterates as each problem stepped alone, also when members
join and leave between steps (continuous batching)."""

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


PROBLEMS = [  # (n_side, M, J, db orders, levels, seed)
    (64, 5_000, 4, (0, 1, 2), 2, 1),
    (128, 20_000, 6, (0, 1, 2, 3, 4), 3, 2),
    (32, 2_000, 4, (0, 2), 2, 3),
    (96, 9_000, 4, (0, 1, 8), 2, 4),
]


def make_solver(g, prob):
    n, M, J, orders, L, seed = prob
    x = synth.sky(n, 3, 2, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 10, outlier_frac=0.2, weights="uniform")
    y0 = me.phi(x, me.Geometry(uvw, n, 2, J, 4096))
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 20)).astype(np.complex64)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=so.epsilon_from_sigma(sigma, M),
                 op_norm_sq=float(M), gamma=1e-3)
    return s, plan, wav


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_batch_matches_alone_with_joins_and_leaves(g):
    alone = [make_solver(g, p) for p in PROBLEMS]
    mixed = [make_solver(g, p) for p in PROBLEMS]
    b = g.Batch()
    for s, _, _ in mixed[:3]:
        b.add(s)
    b.step(6)
    b.add(mixed[3][0])          # joins late
    b.remove(mixed[0][0])       # leaves early
    b.step(4)
    torch.cuda.synchronize()
    iters = [6, 10, 10, 4]
    for (sa, _, _), (sm, _, _), k in zip(alone, mixed, iters):
        sa.step(k)
        xa, xm = sa.x().cpu().numpy(), sm.x().cpu().numpy()
        assert sm.report()["iters"] == k
        assert rel(xm, xa) <= 1e-5
    assert len(b) == 3
    with pytest.raises(g.GbriError):
        b.add(mixed[1][0])      # already a member
    b.close()


def test_batch_rejects_shared_plan(g):
    s1, plan, wav = make_solver(g, PROBLEMS[0])
    y = torch.zeros(PROBLEMS[0][1], dtype=torch.complex64, device="cuda")
    s2 = g.Solver(plan, g.Wavelet(64, 2, (0, 1)), y, eps=1.0, op_norm_sq=1.0, gamma=1e-3)
    b = g.Batch()
    b.add(s1)
    with pytest.raises(g.GbriError):
        b.add(s2)
    b.close()


def test_shared_pass_members_match_alone(g):
    """The shared fused pass (gbri_batch_set_shared_pass): the J = 4 FP32 primal-dual members
    share one launch of the degridding + gridding pass, the others (J = 6, ADMM, FISTA, a
    deterministic plan) keep their own iterations; every member equals the same problem
    stepped alone (the shared pass changes only the summation order of the l2-ball norm), and
    switching the pass off gives the same iterates."""
    probs = [PROBLEMS[0], PROBLEMS[2], PROBLEMS[3], PROBLEMS[1], (64, 4_000, 4, (0, 1), 2, 7),
             (48, 3_000, 4, (0, 2), 2, 8), (64, 6_000, 4, (0, 1, 3), 2, 9)]

    def build():
        out = [make_solver(g, p) for p in probs[:4]]
        out.append(make_solver_algo(g, probs[4], g.ALGO_ADMM))
        out.append(make_solver_algo(g, probs[5], g.ALGO_FISTA))
        out.append(make_solver_det(g, probs[6]))
        return out

    runs = {}
    for shared in (True, False):
        mixed = build()
        b = g.Batch()
        b.set_shared_pass(shared)
        for s, _, _ in mixed:
            b.add(s)
        b.step(8)
        torch.cuda.synchronize()
        assert b.shared_members() == (3 if shared else 0)
        runs[shared] = [s.x().cpu().numpy() for s, _, _ in mixed]
        for s, _, _ in mixed:
            assert s.report()["iters"] == 8
        b.close()
    alone = build()
    for k, (sa, _, _) in enumerate(alone):
        sa.step(8)
        xa = sa.x().cpu().numpy()
        # ADMM and FISTA (members 4, 5) differ between any two runs by up to ~2e-5 after 8
        # iterations on these small problems (their gridding flush adds float atomics in a
        # run-dependent order): the solvers' 1e-4 bar; the primal-dual members 1e-5
        tol = 1e-4 if k in (4, 5) else 1e-5
        assert rel(runs[True][k], xa) <= tol, k
        assert rel(runs[False][k], xa) <= tol, k


def make_solver_algo(g, prob, algo):
    n, M, J, orders, L, seed = prob
    x = synth.sky(n, 3, 2, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 10, outlier_frac=0.2, weights="uniform")
    y0 = me.phi(x, me.Geometry(uvw, n, 2, J, 4096))
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 20)).astype(np.complex64)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=so.epsilon_from_sigma(sigma, M),
                 op_norm_sq=float(M), gamma=1e-3, algo=algo)
    return s, plan, wav


def make_solver_det(g, prob):
    n, M, J, orders, L, seed = prob
    x = synth.sky(n, 3, 2, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 10, outlier_frac=0.2, weights="uniform")
    y0 = me.phi(x, me.Geometry(uvw, n, 2, J, 4096))
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 20)).astype(np.complex64)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, deterministic=True)
    wav = g.Wavelet(n, L, orders)
    s = g.Solver(plan, wav, torch.from_numpy(y).cuda(), eps=so.epsilon_from_sigma(sigma, M),
                 op_norm_sq=float(M), gamma=1e-3)
    return s, plan, wav
