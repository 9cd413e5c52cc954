"""The allocation-free l2-ball projection, called through the C ABI, matches the allocating one.

gbri_proj_l2ball_noalloc serves callers that cannot allocate device memory when they
need the projection (their pool allocator already holds the memory, an out-of-memory
handler, a loop that must not synchronise): its reduction scratch is a fixed device
array inside the library.  Two calls in a row check that the shared scratch carries
nothing from one call into the next.  This file is collected last on purpose.
"""

import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04502_gb300 as g
    return g.library()


def _case(M, seed, scale):
    c = (synth.normal(M, seed=seed) + 1j * synth.normal(M, seed=seed + 1)).astype(np.complex64)
    d = (synth.normal(M, seed=seed + 2) + 1j * synth.normal(M, seed=seed + 3)).astype(np.complex64)
    eps = scale * float(np.linalg.norm(d.astype(np.complex128)))
    return torch.from_numpy(c + d).cuda(), torch.from_numpy(c).cuda(), eps


def _call(fn, z, c, eps, with_precision):
    out = torch.empty_like(z)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    args = [C.c_void_p(z.data_ptr()), C.c_void_p(c.data_ptr()), C.c_void_p(out.data_ptr()), z.numel(),
            float(eps), C.c_void_p(nrm.data_ptr())]
    if with_precision:
        args.append(0)  # GBRI_F32
    rc = fn(*args, stream)
    assert rc == 0
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(nrm.item())


def test_noalloc_matches_allocating_projection_twice(lib):
    # first call: large, projected (radius below the distance); second: a different size inside
    # the ball, then projected again, so stale partials from the first call would show up
    for M, seed, scale in ((1_000_003, 10, 0.3), (77_777, 20, 2.0), (250_000, 30, 0.5)):
        z, c, eps = _case(M, seed, scale)
        a, na = _call(lib.gbri_proj_l2ball, z, c, eps, True)
        b, nb = _call(lib.gbri_proj_l2ball_noalloc, z, c, eps, False)
        assert nb == pytest.approx(na, rel=1e-12)
        assert np.linalg.norm(b - a) <= 1e-6 * np.linalg.norm(a)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_against_oracle_inplace_null_norm_and_empty(lib):
    """Against the FP64 oracle projection (Sec. 4.2) at 1e-6: out separate with the norm,
    out == z (the documented in-place case) without the norm (null pointer), and M = 0."""
    from oracle import prox
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for M, seed, scale in ((500_001, 40, 0.4), (4097, 50, 3.0)):
        z, c, eps = _case(M, seed, scale)
        zc = z.cpu().numpy().astype(np.complex128)
        cc = c.cpu().numpy().astype(np.complex128)
        ref, ref_norm = prox.proj_l2ball(zc, cc, eps)
        out, nrm = _call(lib.gbri_proj_l2ball_noalloc, z, c, eps, False)
        assert _rel(out.astype(np.complex128), ref) <= 1e-6
        assert nrm == pytest.approx(ref_norm, rel=1e-9)
        zin = z.clone()
        rc = lib.gbri_proj_l2ball_noalloc(C.c_void_p(zin.data_ptr()), C.c_void_p(c.data_ptr()),
                                          C.c_void_p(zin.data_ptr()), M, float(eps), None, stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert _rel(zin.cpu().numpy().astype(np.complex128), ref) <= 1e-6
    nrm = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    rc = lib.gbri_proj_l2ball_noalloc(None, None, None, 0, 1.0, C.c_void_p(nrm.data_ptr()), stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert float(nrm.item()) == 0.0  # the empty vector is at distance 0 from the empty centre


def test_noalloc_allocates_no_device_memory(lib):
    """A warm call (kernels already loaded) leaves the device's free memory and torch's
    allocator statistics unchanged; the Python wrapper with a caller-provided out does too."""
    import paper_1903_04502_gb300 as g
    z, c, eps = _case(300_000, 60, 0.5)
    out = torch.empty_like(z)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    g.proj_l2ball_noalloc(z, c, eps, out, norm_out=nrm)  # warm-up: module loading may allocate
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for _ in range(3):
        g.proj_l2ball_noalloc(z, c, eps, out, norm_out=nrm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    alloc1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    assert free1 == free0 and alloc1 == alloc0
    ref = g.proj_l2ball(z, c, eps)
    assert _rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-6
    with pytest.raises(TypeError):
        g.proj_l2ball_noalloc(z, c, eps)  # out is required: the wrapper never allocates
