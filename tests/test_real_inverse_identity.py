"""The identity the library's adjoint relies on, checked in NumPy (no GPU, no library code).

Every reader of the inverse transform of the gridded visibilities takes only its real part
(Sec. 2: the sky image is real).  The library therefore folds the grid G into its Hermitian
part H[k] = (G[k] + conj G[-k]) / 2 on the half plane kx = 0 .. K/2 and runs a
complex-to-real inverse on H.  These tests check, independently of that code, that this
gives Re(F^H G) for any complex G, including the Nyquist row and column and odd-looking
grids, and that dropping the conjugation or the mirror index (the plausible slips) does not.
"""

import numpy as np
import pytest


def hermitian_half(G):
    K = G.shape[0]
    H = np.empty((K, K // 2 + 1), dtype=complex)
    for ky in range(K):
        for kx in range(K // 2 + 1):
            a, b = G[ky, kx], G[(-ky) % K, (-kx) % K]
            H[ky, kx] = 0.5 * (a.real + b.real) + 0.5j * (a.imag - b.imag)
    return H


@pytest.mark.parametrize("K", [2, 4, 8, 16, 30])
def test_complex_to_real_of_the_hermitian_half_is_the_real_part(K):
    rng = np.random.default_rng(K)
    G = rng.normal(size=(K, K)) + 1j * rng.normal(size=(K, K))
    H = hermitian_half(G)
    # numpy's inverse transforms carry 1 / K^2; the identity holds for either normalisation
    assert np.abs(np.fft.irfft2(H, s=(K, K)) - np.fft.ifft2(G).real).max() < 1e-14


def test_hermitian_half_of_a_hermitian_grid_is_the_grid():
    K = 8
    x = np.random.default_rng(1).normal(size=(K, K))
    G = np.fft.fft2(x)  # the transform of a real image is Hermitian
    assert np.allclose(hermitian_half(G), G[:, : K // 2 + 1], atol=1e-12)


def test_slips_are_detected():
    K = 8
    rng = np.random.default_rng(2)
    G = rng.normal(size=(K, K)) + 1j * rng.normal(size=(K, K))
    ref = np.fft.ifft2(G).real
    no_conj = np.empty((K, K // 2 + 1), dtype=complex)
    no_mirror = np.empty((K, K // 2 + 1), dtype=complex)
    for ky in range(K):
        for kx in range(K // 2 + 1):
            a, b = G[ky, kx], G[(-ky) % K, (-kx) % K]
            no_conj[ky, kx] = 0.5 * (a + b)
            no_mirror[ky, kx] = 0.5 * (a + np.conj(G[ky, kx]))
    assert np.abs(np.fft.irfft2(no_conj, s=(K, K)) - ref).max() > 1e-3
    assert np.abs(np.fft.irfft2(no_mirror, s=(K, K)) - ref).max() > 1e-3
