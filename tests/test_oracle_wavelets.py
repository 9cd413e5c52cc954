"""Pins for the oracle's Daubechies filters and the SARA operators Psi / Psi^dagger."""

from math import sqrt

import numpy as np
import pytest

import synth
from oracle import wavelets as wv


@pytest.mark.parametrize("N", range(1, 9))
def test_filter_conditions(N):
    h = wv.daubechies_lowpass(N)
    g = wv.highpass(h)
    L = len(h)
    assert L == 2 * N
    assert h.sum() == pytest.approx(sqrt(2.0), abs=1e-14)
    for m in range(N):  # double-shift orthonormality
        s = sum(h[k] * h[k + 2 * m] for k in range(L - 2 * m))
        assert s == pytest.approx(1.0 if m == 0 else 0.0, abs=1e-14)
    for p in range(N):  # N vanishing moments of the wavelet
        assert abs(sum(g[k] * (k / L) ** p for k in range(L))) < 1e-13
    # H(w) = sum h_n w^n has an N-fold zero at w = -1, and the remaining factor is minimum phase
    # (all its zeros outside the unit disk)
    binom = np.poly1d([1.0, 1.0]) ** N
    q, r = np.polydiv(h[::-1], binom.coeffs)
    assert np.max(np.abs(r)) < 1e-13
    if N > 1:
        assert np.all(np.abs(np.roots(q)) > 1.0)


def test_db1_db2_db3_closed_forms():
    assert np.allclose(wv.daubechies_lowpass(1), [1 / sqrt(2), 1 / sqrt(2)], rtol=0, atol=1e-15)
    s3 = sqrt(3.0)
    d4 = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * sqrt(2.0))
    assert np.allclose(wv.daubechies_lowpass(2), d4, rtol=0, atol=1e-15)
    s10 = sqrt(10.0)
    r = sqrt(5 + 2 * s10)
    d6 = np.array([1 + s10 + r, 5 + s10 + 3 * r, 10 - 2 * s10 + 2 * r, 10 - 2 * s10 - 2 * r,
                   5 + s10 - 3 * r, 1 + s10 - r]) / (16 * sqrt(2.0))
    assert np.allclose(wv.daubechies_lowpass(3), d6, rtol=0, atol=1e-15)


def test_haar_one_level_by_hand():
    x = synth.normal(16, seed=3).reshape(4, 4)
    a = wv.dwt2(x, 1, 1)
    for i in range(2):
        for j in range(2):
            blk = x[2 * i:2 * i + 2, 2 * j:2 * j + 2]
            assert a[i, j] == pytest.approx(blk.sum() / 2)                                  # LL
            assert a[i, 2 + j] == pytest.approx((blk[:, 0] - blk[:, 1]).sum() / 2)         # rows high
            assert a[2 + i, j] == pytest.approx((blk[0, :] - blk[1, :]).sum() / 2)         # cols high
            assert a[2 + i, 2 + j] == pytest.approx((blk[0, 0] - blk[0, 1] - blk[1, 0] + blk[1, 1]) / 2)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 6, 7, 8])
@pytest.mark.parametrize("n,levels", [(32, 3), (64, 4), (16, 4)])
def test_each_basis_orthonormal(N, n, levels):
    x = synth.normal(n * n, seed=N).reshape(n, n)
    a = wv.dwt2(x, N, levels)
    assert np.linalg.norm(a) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    assert np.allclose(wv.idwt2(a, N, levels), x, rtol=0, atol=1e-12)
    b = synth.normal(n * n, seed=100 + N).reshape(n, n)
    assert np.allclose(wv.dwt2(wv.idwt2(b, N, levels), N, levels), b, rtol=0, atol=1e-12)


def test_sara_stack_tight_frame_and_adjoint():
    n, levels = 32, 3
    orders = (0, 1, 2, 3, 4, 5, 6, 7, 8)
    x = synth.normal(n * n, seed=5).reshape(n, n)
    al = wv.psi_adjoint(x, orders, levels)
    assert al.shape == (9, n, n)
    assert np.allclose(wv.psi(al, orders, levels), x, atol=1e-12)      # Psi Psi^dagger = I
    assert np.linalg.norm(al) == pytest.approx(np.linalg.norm(x), rel=1e-13)
    beta = synth.normal(9 * n * n, seed=6).reshape(9, n, n)
    assert np.vdot(al, beta) == pytest.approx(np.vdot(x, wv.psi(beta, orders, levels)), rel=1e-12)
    assert np.allclose(al[0], x / 3.0)                                    # Dirac basis / sqrt(9)


@pytest.mark.parametrize("N", [2, 5])
def test_periodic_shift_equivariance(N):
    # a cyclic shift of the image by 2^L pixels shifts every level-l subband by 2^(L-l)
    n, L = 32, 3
    x = synth.normal(n * n, seed=11).reshape(n, n)
    a = wv.dwt2(x, N, L)
    b = wv.dwt2(np.roll(x, (2 ** L, 2 ** L), axis=(0, 1)), N, L)
    for lev in range(1, L + 1):
        m = n >> lev
        s = 2 ** (L - lev)
        for (r0, c0) in ((0, m), (m, 0), (m, m)):
            sub_a = a[r0:r0 + m, c0:c0 + m]
            sub_b = b[r0:r0 + m, c0:c0 + m]
            assert np.allclose(np.roll(sub_a, (s, s), axis=(0, 1)), sub_b, atol=1e-12)
    m = n >> L
    assert np.allclose(np.roll(a[:m, :m], (1, 1), axis=(0, 1)), b[:m, :m], atol=1e-12)


def test_lowpass_of_constant_image():
    # a constant image has no detail coefficients; its LL carries the mean times 2^L
    n, L = 16, 2
    x = np.full((n, n), 3.0)
    for N in (1, 4, 8):
        a = wv.dwt2(x, N, L)
        m = n >> L
        assert np.allclose(a[:m, :m], 3.0 * 2 ** L)
        a[:m, :m] = 0
        assert np.allclose(a, 0, atol=1e-12)
