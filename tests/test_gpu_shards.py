"""Virtual shards on one GPU: the paper's distributed-image decomposition (Sec. 6.3.1,
Algorithm 2) with the visibilities split into blocks y_j, each with its own
measurement operator Phi_j (same image, same grid), checked against the operator of
the whole problem:
  * Phi_j x equals the rows of Phi x that belong to block j,
  * Phi^dagger y = sum_j Phi_j^dagger y_j (the image all-reduce of Algorithm 2),
  * ||y - Phi x||^2 = sum_j ||y_j - Phi_j x||^2 (the global l2-ball norm from block norms).
The blocks are contiguous ranges of grid-tile order (each block's gridding touches a
compact region of the grid), as a multi-GPU split would use.
"""

import numpy as np
import pytest

import synth

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


def tile_blocks(uvw, n_side, n_blocks, tile=16):
    """Indices of n_blocks contiguous ranges of the visibilities in (tile row, tile column) order."""
    K = 2 * n_side
    nT = K // tile
    cell = lambda u: np.floor((u + np.pi) / (2 * np.pi) * K).astype(np.int64) % K  # noqa: E731
    key = (cell(uvw[:, 1].astype(np.float64)) // tile) * nT + cell(uvw[:, 0].astype(np.float64)) // tile
    order = np.argsort(key, kind="stable")
    return np.array_split(order, n_blocks)


@pytest.mark.parametrize("prec,tol", [("f32", 1e-6), ("f64", 1e-12)])
def test_virtual_shards_reproduce_the_whole_operator(g, prec, tol):
    n, M, B = 128, 30_011, 4
    F = g.F64 if prec == "f64" else g.F32
    rdt = np.float64 if prec == "f64" else np.float32
    cdt = np.complex128 if prec == "f64" else np.complex64
    x = synth.sky(n, 8, 4, seed=4).astype(rdt)
    uvw = synth.uv_coverage(M, seed=5, outlier_frac=0.2, weights="uniform")
    blocks = tile_blocks(uvw, n, B)
    assert sum(len(b) for b in blocks) == M
    whole = g.Plan(torch.from_numpy(uvw).cuda(), n, precision=F)
    parts = [g.Plan(torch.from_numpy(np.ascontiguousarray(uvw[b])).cuda(), n, precision=F) for b in blocks]
    xd = torch.from_numpy(x).cuda()
    y_whole = g.phi(whole, xd).cpu().numpy()
    for b, p in zip(blocks, parts):
        assert rel(g.phi(p, xd).cpu().numpy(), y_whole[b]) <= tol
    y = synth.complex_normal(M, seed=6).astype(cdt)
    x_whole = g.phi_adjoint(whole, torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    x_sum = np.zeros((n, n))
    for b, p in zip(blocks, parts):
        x_sum += g.phi_adjoint(p, torch.from_numpy(np.ascontiguousarray(y[b])).cuda()).cpu().numpy()
    assert rel(x_sum, x_whole) <= tol
    # the global residual norm from the block norms (FP64 on the device)
    r_whole = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.proj_l2ball(torch.from_numpy(y_whole).cuda(), torch.from_numpy(y).cuda(), 0.0, norm_out=r_whole)
    sq = 0.0
    for b, p in zip(blocks, parts):
        r = torch.zeros(1, dtype=torch.float64, device="cuda")
        g.proj_l2ball(g.phi(p, xd), torch.from_numpy(np.ascontiguousarray(y[b])).cuda(), 0.0, norm_out=r)
        sq += float(r.item()) ** 2
    assert np.sqrt(sq) == pytest.approx(float(r_whole.item()), rel=tol)
