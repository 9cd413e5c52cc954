"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side tests and bench.

This module holds random draws and workload shapes only -- none of the
imaging method's arithmetic.  The paper's benchmarks draw (u, v) from a
Gaussian density spanning +-pi on each axis (Sec. 7.3); its skies are not
published, so the recipe below follows the workload descriptions (point sources
plus Gaussian blobs, 30 dB input SNR):

* sky: point sources at integer pixels, uniform in the central 80 % box, flux
  log-uniform in [0.1, 1]; Gaussian blobs with sigma uniform in [2, 6] px, peak
  log-uniform in [0.1, 1], centres in the same box.  x >= 0, float64.
* uv: isotropic 2-D Gaussian with per-axis sigma = pi/3, truncated to
  |u|, |v| <= pi by rejection; optionally a fraction of points uniform in the
  disk of radius pi.  w = 0.  Weights all 1, or uniform in [0.5, 1].  Packed as
  float32 rows {u, v, w, weight}.
* noise: standard complex normal draws CN(0, 1) (real and imaginary parts
  N(0, 1/2)); the caller scales them.

Every draw uses numpy's PCG64 seeded with (seed, stream) so that the sky, the
coverage and the noise of one problem are independent and reproducible.
"""

import numpy as np

_SKY, _UV, _NOISE, _AUX = 1, 2, 3, 4


def _rng(seed, stream):
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def sky(n_side, n_points, n_blobs, seed=0):
    """Non-negative test sky (float64, n_side x n_side)."""
    rng = _rng(seed, _SKY)
    img = np.zeros((n_side, n_side), dtype=np.float64)
    lo, hi = int(round(0.1 * n_side)), int(round(0.9 * n_side))
    for _ in range(n_points):
        q, p = rng.integers(lo, hi, size=2)
        img[q, p] += np.exp(rng.uniform(np.log(0.1), np.log(1.0)))
    yy, xx = np.mgrid[0:n_side, 0:n_side].astype(np.float64)
    for _ in range(n_blobs):
        cq, cp = rng.uniform(lo, hi, size=2)
        s = rng.uniform(2.0, 6.0)
        peak = np.exp(rng.uniform(np.log(0.1), np.log(1.0)))
        img += peak * np.exp(-((yy - cq) ** 2 + (xx - cp) ** 2) / (2.0 * s * s))
    return img


def uv_coverage(M, seed=0, outlier_frac=0.0, weights="ones", sigma=np.pi / 3.0):
    """(M, 4) float32 rows {u, v, w=0, weight} with |u|, |v| <= pi."""
    rng = _rng(seed, _UV)
    n_out = int(round(outlier_frac * M))
    n_gauss = M - n_out
    out = np.empty((M, 4), dtype=np.float32)
    got = 0
    pts = np.empty((n_gauss, 2), dtype=np.float64)
    while got < n_gauss:
        need = n_gauss - got
        cand = rng.normal(0.0, sigma, size=(int(need * 1.05) + 16, 2))
        ok = cand[np.all(np.abs(cand) <= np.pi, axis=1)][:need]
        pts[got:got + len(ok)] = ok
        got += len(ok)
    out[:n_gauss, :2] = pts
    if n_out:
        r = np.pi * np.sqrt(rng.uniform(0.0, 1.0, size=n_out))
        th = rng.uniform(0.0, 2.0 * np.pi, size=n_out)
        out[n_gauss:, 0] = np.clip(r * np.cos(th), -np.pi, np.pi)
        out[n_gauss:, 1] = np.clip(r * np.sin(th), -np.pi, np.pi)
    # the float32 cast may round a coordinate just past pi: pull it back inside
    out[:, :2] = np.clip(out[:, :2], np.float32(-np.pi), np.float32(np.pi))
    out[:, 2] = 0.0
    if weights == "ones":
        out[:, 3] = 1.0
    elif weights == "uniform":
        out[:, 3] = rng.uniform(0.5, 1.0, size=M)
    else:
        raise ValueError(weights)
    perm = rng.permutation(M)  # interleave the outliers with the core
    return out[perm]


def uvw_noncoplanar(M, seed=0, delta=0.01, w_frac=0.5, outlier_frac=0.2, weights="uniform"):
    """``uv_coverage`` rows with a w column for a non-coplanar array, in wavelengths: with
    u, v in radians per pixel the baseline length in wavelengths is |(u, v)| / (2 pi delta)
    (delta the pixel size in direction cosines), and w = w_frac |(u, v)| / (2 pi delta) s, s
    uniform in [-1, 1]: longer baselines reach larger |w|, and |w| stays below w_frac times
    the baseline length (an array tilted by up to asin(w_frac) from the plane), float32."""
    out = uv_coverage(M, seed=seed, outlier_frac=outlier_frac, weights=weights)
    rng = _rng(seed, _AUX + 1)
    r = np.sqrt(out[:, 0].astype(np.float64) ** 2 + out[:, 1].astype(np.float64) ** 2) / (2.0 * np.pi * delta)
    out[:, 2] = (w_frac * r * rng.uniform(-1.0, 1.0, size=M)).astype(np.float32)
    return out


def complex_normal(M, seed=0, stream=_NOISE):
    """Standard complex normal draws CN(0, 1), complex128."""
    rng = _rng(seed, stream)
    return (rng.normal(0.0, np.sqrt(0.5), size=M) + 1j * rng.normal(0.0, np.sqrt(0.5), size=M))


def uniform(n, seed=0, lo=0.0, hi=1.0, stream=_AUX):
    """Uniform float64 draws (auxiliary test vectors)."""
    return _rng(seed, stream).uniform(lo, hi, size=n)


def normal(n, seed=0, stream=_AUX):
    """Standard normal float64 draws (auxiliary test vectors)."""
    return _rng(seed, stream).normal(0.0, 1.0, size=n)


def uv_coverage_device(M, seed, device, outlier_frac=0.2):
    """uv coverage drawn on a torch device (for visibility counts too large for the host
    generator), with the distribution of ``uv_coverage`` (weights "uniform"): isotropic
    Gaussian, sigma = pi / 3 per axis, truncated to |u|, |v| <= pi by rejection; a fraction
    uniform in the disk of radius pi; weights uniform in [0.5, 1]; float32 [M, 4] on the
    device, w = 0.  Seeded by a torch generator on that device (its own random stream, not
    the numpy one)."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    n_out = int(round(outlier_frac * M))
    n_g = M - n_out
    out = torch.zeros((M, 4), dtype=torch.float32, device=device)
    got = 0
    while got < n_g:  # rejection in bounded batches (float64 draws, float32 storage)
        want = min(n_g - got, 1 << 27)
        c = torch.randn((int(want * 1.05) + 1024, 2), dtype=torch.float64, device=device, generator=gen)
        c = c * (np.pi / 3.0)
        c = c[(c.abs() <= np.pi).all(dim=1)][:want]
        out[got:got + c.shape[0], :2] = c.to(torch.float32)
        got += c.shape[0]
    for a in range(0, n_out, 1 << 27):
        k = min(1 << 27, n_out - a)
        r = np.pi * torch.sqrt(torch.rand(k, dtype=torch.float64, device=device, generator=gen))
        th = 2 * np.pi * torch.rand(k, dtype=torch.float64, device=device, generator=gen)
        out[n_g + a:n_g + a + k, 0] = (r * torch.cos(th)).to(torch.float32)
        out[n_g + a:n_g + a + k, 1] = (r * torch.sin(th)).to(torch.float32)
    out[:, :2].clamp_(-np.float32(np.pi), np.float32(np.pi))
    for a in range(0, M, 1 << 27):
        k = min(1 << 27, M - a)
        out[a:a + k, 3] = 0.5 + 0.5 * torch.rand(k, dtype=torch.float32, device=device, generator=gen)
    return out


# Workload shapes of the paper-shaped problems (sizes only).
CONFIGS = {
    # plain method, FP64: 128^2 sky, 5 points + 3 blobs, K = 256, J = 4, S = 2^12, M = 2e4,
    # SARA Dirac + db1..db4, 3 levels, 100 primal-dual iterations
    "small": dict(n_side=128, n_points=5, n_blobs=3, oversample=2, J=4, S=4096, M=20_000,
                  outlier_frac=0.0, weights="ones", db_orders=(0, 1, 2, 3, 4), levels=3, iters=100,
                  snr_db=30.0, seed=0),
    # FP32 on the GPU: 1024^2 sky, 50 points + 20 blobs, K = 2048, J = 4, M = 1e7, 20 % uniform-disk
    # outliers, weights U[0.5, 1], SARA Dirac + db1..db8, 4 levels, 200 iterations
    "large": dict(n_side=1024, n_points=50, n_blobs=20, oversample=2, J=4, S=4096, M=10_000_000,
                  outlier_frac=0.2, weights="uniform", db_orders=(0, 1, 2, 3, 4, 5, 6, 7, 8), levels=4,
                  iters=200, snr_db=30.0, seed=0),
    # precision study: 4096^2, K = 8192, J = 6, M = 2e9 (subsampled for the oracle)
    "huge": dict(n_side=4096, n_points=50, n_blobs=20, oversample=2, J=6, S=4096, M=2_000_000_000,
                 outlier_frac=0.2, weights="uniform", db_orders=(0, 1, 2, 3, 4, 5, 6, 7, 8), levels=4,
                 iters=200, snr_db=30.0, seed=0),
}
