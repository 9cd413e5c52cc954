"""The request loop on the GPU: jobs that arrive while others run join the running batch,
memory admission holds the rest back, and every job's image is the same as when the job
runs alone for the same number of iterations."""

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


def make_job(serve, n, M, J, seed, arrival, max_iter=60, rel_tol=2e-3):
    x = synth.sky(n, 3, 2, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 100, outlier_frac=0.2, weights="uniform")
    y0 = me.phi(x, me.Geometry(uvw, n, 2, J, 4096))
    sigma = 10 ** (-30 / 20) * np.linalg.norm(y0) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 200)).astype(np.complex64)
    return serve.Job(uvw=uvw, y=y, n_side=n, eps=so.epsilon_from_sigma(sigma, M), J=J, db_orders=(0, 1, 2, 3),
                     levels=2, max_iter=max_iter, rel_tol=rel_tol, op_norm_sq=float(M), gamma=1e-3,
                     arrival=arrival)


@pytest.mark.parametrize("shared_pass", [False, True])
def test_served_jobs_match_alone(g, shared_pass):
    """Every served job equals the same job run alone; with the batch's shared fused pass on,
    the primal-dual J = 4 jobs resident together share its launch (rebuilt as jobs come and
    go, under the engine's set-up lock)."""
    from paper_1903_04502_gb300 import serve
    specs = [(64, 6000, 4), (32, 2000, 6), (96, 12000, 4), (64, 4000, 6), (32, 3000, 4), (128, 20000, 4)]
    jobs = [make_job(serve, n, M, J, seed=i + 1, arrival=0.0 if i < 3 else 0.005 * i, max_iter=300, rel_tol=1e-4)
            for i, (n, M, J) in enumerate(specs)]
    budget = 3 * max(serve.device_footprint(n, M, J, 4) for n, M, J in specs)
    srv = serve.Server(serve.GpuEngine(shared_pass=shared_pass), hbm_budget=budget, check_every=5)
    done = srv.run(jobs)
    assert len(done) == len(jobs) and not srv.failed
    assert srv.max_resident >= 2                      # jobs overlapped on the device
    st = srv.stats()
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    for j in done:
        plan = g.Plan(torch.from_numpy(j.uvw).cuda(), j.n_side, J=j.J)
        wav = g.Wavelet(j.n_side, j.levels, j.db_orders)
        s = g.Solver(plan, wav, torch.from_numpy(j.y).cuda(), eps=j.eps, op_norm_sq=j.op_norm_sq, gamma=j.gamma)
        s.step(j.iters)
        xa = s.x().cpu().numpy()
        assert np.linalg.norm(j.result - xa) <= 1e-5 * np.linalg.norm(xa)
        assert j.iters == 300 or j.rel_change < 1e-4


@pytest.mark.parametrize("n,M,J", [(256, 100_000, 4), (1024, 1_000_000, 4), (2048, 2_000_000, 6)])
def test_footprint_estimate_bounds_the_plan(g, n, M, J):
    """The admission estimate bounds what a plan really holds (its buffers, tile tables and
    both cuFFT work areas, as the library counts them)."""
    from paper_1903_04502_gb300 import serve
    uvw = torch.from_numpy(synth.uv_coverage(M, seed=1, outlier_frac=0.2, weights="uniform")).cuda()
    plan = g.Plan(uvw, n, J=J)
    try:
        assert 0 < plan.device_bytes <= serve.device_footprint(n, M, J, 1)
    finally:
        plan.close()


def test_served_jobs_bitwise_equal_alone_with_deterministic_plans(g):
    """With deterministic plans a served job's image equals the same job run alone bit for bit,
    however the other jobs overlap it on the device."""
    from paper_1903_04502_gb300 import serve
    specs = [(64, 30000, 4), (32, 8000, 6), (96, 40000, 4), (64, 20000, 4)]
    jobs = [make_job(serve, n, M, J, seed=i + 11, arrival=0.0 if i < 2 else 0.004 * i, max_iter=200, rel_tol=0.0)
            for i, (n, M, J) in enumerate(specs)]
    for j in jobs:
        j.deterministic = True
    eng = serve.GpuEngine()
    srv = serve.Server(eng, hbm_budget=1e11, check_every=5)
    done = srv.run(jobs)
    eng.close()
    assert len(done) == len(jobs) and srv.max_resident >= 2
    for j in done:
        plan = g.Plan(torch.from_numpy(j.uvw).cuda(), j.n_side, J=j.J, deterministic=True)
        wav = g.Wavelet(j.n_side, j.levels, j.db_orders)
        s = g.Solver(plan, wav, torch.from_numpy(j.y).cuda(), eps=j.eps, op_norm_sq=j.op_norm_sq, gamma=j.gamma)
        s.step(j.iters)
        assert np.array_equal(j.result, s.x().cpu().numpy())


def test_server_survives_an_out_of_memory_job(g):
    """The library's allocator is made to fail (host-side hook, no GPU fault) for the next
    device allocation, made while one job is set up: that job fails with GBRI_ENOMEM, the
    others are served normally and the server's memory reservation returns to zero."""
    from paper_1903_04502_gb300 import serve
    jobs = [make_job(serve, 64, 5000, 4, seed=i + 31, arrival=0.0) for i in range(3)]
    eng = serve.GpuEngine()
    srv = serve.Server(eng, hbm_budget=1e11, check_every=5)
    g.inject_alloc_failure(1)  # the next device allocation the library makes
    try:
        srv.run(jobs)
    finally:
        g.inject_alloc_failure(0)
        eng.close()
    assert len(srv.failed) == 1 and "-2" in srv.failed[0].error   # GBRI_ENOMEM
    assert len(srv.done) == 2 and srv.used == 0
