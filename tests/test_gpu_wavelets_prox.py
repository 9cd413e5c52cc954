"""GPU parity of Psi / Psi^dagger and the proximal operators (through the C ABI) against the oracle."""

import numpy as np
import pytest

import synth
from oracle import prox, wavelets as wv

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


@pytest.mark.parametrize("n,levels,orders", [
    (64, 4, (0, 1, 2, 3, 4, 5, 6, 7, 8)),
    (128, 3, (0, 1, 2, 3, 4)),
    (32, 2, (8, 3, 0)),          # order of the stack is the caller's; filters longer than coarse blocks wrap
    (16, 3, (8,)),
    (256, 4, (1, 8)),
    (48, 1, (0, 2, 5)),          # one level: the first-level kernels alone; partial 32 x 32 blocks
    (96, 2, (3, 0, 1)),          # side not a multiple of 32, Dirac in the middle of the stack
    (40, 3, (0, 4)),
    (64, 2, (0,)),               # Dirac only
    (64, 2, tuple(range(11))),   # ten wavelet bases, db1 to db10 (20 taps, the longest filter)
])
def test_psi_adjoint_and_psi_match_oracle(g, n, levels, orders):
    x = synth.normal(n * n, seed=n).reshape(n, n).astype(np.float32)
    wav = g.Wavelet(n, levels, orders)
    al = g.psi_adjoint(wav, torch.from_numpy(x).cuda()).cpu().numpy()
    al_ref = wv.psi_adjoint(x.astype(np.float64), orders, levels)
    assert rel(al, al_ref) <= 1e-6
    a = synth.normal(len(orders) * n * n, seed=n + 1).reshape(len(orders), n, n).astype(np.float32)
    xs = g.psi(wav, torch.from_numpy(a).cuda()).cpu().numpy()
    assert rel(xs, wv.psi(a.astype(np.float64), orders, levels)) <= 1e-6
    # tight frame on the device: Psi Psi^dagger = I
    back = g.psi(wav, torch.from_numpy(al).cuda()).cpu().numpy()
    assert rel(back, x) <= 1e-6


def test_psi_full_size(g):
    n, levels, orders = 1024, 4, tuple(range(9))
    x = synth.sky(n, 50, 20, seed=0).astype(np.float32)
    wav = g.Wavelet(n, levels, orders)
    al = g.psi_adjoint(wav, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(al, wv.psi_adjoint(x.astype(np.float64), orders, levels)) <= 1e-6


@pytest.mark.parametrize("cplx", [False, True])
def test_prox_l1_matches_oracle(g, cplx):
    n = 100_003
    x = synth.normal(n, seed=1) * 2
    if cplx:
        x = (x + 1j * synth.normal(n, seed=2)).astype(np.complex64)
    else:
        x = x.astype(np.float32)
    x[:3] = [0.7, -0.7, 0.0] if not cplx else [0.7, 0.7j, 0.0]   # exact ties at |x| = lambda
    out = g.prox_l1(torch.from_numpy(x).cuda(), 0.7).cpu().numpy()
    ref = prox.soft_threshold(x.astype(np.complex128 if cplx else np.float64), 0.7)
    assert np.allclose(out, ref, rtol=1e-6, atol=1e-6)
    assert np.all(out[:3] == 0)
    # in place
    t = torch.from_numpy(x).cuda()
    g.prox_l1(t, 0.7, out=t)
    assert np.array_equal(t.cpu().numpy(), out)


@pytest.mark.parametrize("M,scale", [(1, 3.0), (100_000, 0.5), (250_001, 2.0), (4096, 10.0)])
def test_proj_l2ball_matches_oracle(g, M, scale):
    c = (synth.normal(M, seed=3) + 1j * synth.normal(M, seed=4)).astype(np.complex64)
    d = (synth.normal(M, seed=5) + 1j * synth.normal(M, seed=6)).astype(np.complex64)
    z = c + d
    eps = scale * float(np.linalg.norm(d.astype(np.complex128)))
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = g.proj_l2ball(torch.from_numpy(z).cuda(), torch.from_numpy(c).cuda(), eps, norm_out=nrm).cpu().numpy()
    ref, rn = prox.proj_l2ball(z.astype(np.complex128), c.astype(np.complex128), eps)
    assert float(nrm.item()) == pytest.approx(rn, rel=1e-7)
    assert rel(out, ref) <= 1e-6
    if scale >= 1:
        assert np.array_equal(out, z)


def test_proj_l2ball_empty_and_inplace(g):
    z = torch.zeros(0, dtype=torch.complex64, device="cuda")
    g.proj_l2ball(z, z.clone(), 1.0)
    M = 5000
    c = torch.zeros(M, dtype=torch.complex64, device="cuda")
    zz = torch.ones(M, dtype=torch.complex64, device="cuda")
    g.proj_l2ball(zz, c, 1.0, out=zz)
    assert float(torch.linalg.vector_norm(zz).item()) == pytest.approx(1.0, rel=1e-6)
