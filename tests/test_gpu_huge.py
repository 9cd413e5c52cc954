"""The precision-study workload at full size on the GPU: 4096^2 image, 8192^2 grid, J = 6,
M = 2e9 visibilities (uv drawn on the device, 20 % uniform-disk outliers, weights U[0.5, 1]).

Checked in the launch configuration the solvers use (FP32 path): sampled outputs of Phi
against the oracle one by one (the oracle evaluates the full 8192^2 FFT in FP64 and
degrids only the sampled visibilities) to the per-application bar 1e-5, and the adjoint
identity Re<Phi x, y> = <x, Phi^dagger y> on the device with FP64 inner products, a
property that holds at any size.  Skipped on a GPU with less than 200 GB of memory.
"""

import numpy as np
import pytest

import synth
from oracle import measurement as me

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    free, total = torch.cuda.mem_get_info()
    if free < 200 * 2 ** 30:
        pytest.skip("needs about 200 GB of free device memory")
    import paper_1903_04502_gb300 as g
    g.library()
    return g


def test_precision_study_size_sampled_parity_and_adjoint(g):
    cfg = synth.CONFIGS["huge"]
    n, M, J = cfg["n_side"], cfg["M"], cfg["J"]
    uvw = synth.uv_coverage_device(M, 11, torch.device("cuda"), outlier_frac=cfg["outlier_frac"])
    idx = np.concatenate([np.random.default_rng(0).choice(M, 3000, replace=False), [0, M - 1]])
    uvw_s = uvw[torch.from_numpy(idx).cuda()].cpu().numpy()
    plan = g.Plan(uvw, n, J=J, S=cfg["S"])
    del uvw
    torch.cuda.empty_cache()
    x = synth.sky(n, cfg["n_points"], cfg["n_blobs"], seed=0).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = g.phi(plan, xd)
    y_s = y[torch.from_numpy(idx).cuda()].cpu().numpy()
    geo = me.Geometry(uvw_s, n, 2, J, cfg["S"])
    y_ref = me.phi(x.astype(np.float64), geo)
    err = float(np.linalg.norm(y_s - y_ref) / np.linalg.norm(y_ref))
    assert err <= 1e-5, err
    # adjoint identity with FP64 inner products, taken in chunks
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)
    yin = torch.randn(M, dtype=torch.complex64, device="cuda", generator=gen)
    pty = g.phi_adjoint(plan, yin)
    lhs = 0.0
    step = 1 << 27
    for a in range(0, M, step):
        lhs += float(torch.real(torch.vdot(y[a:a + step].to(torch.complex128), yin[a:a + step].to(torch.complex128))))
    rhs = float(torch.dot(xd.double().ravel(), pty.double().ravel()))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    plan.close()
