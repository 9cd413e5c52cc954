"""Pins for the oracle's Kaiser-Bessel kernel, its Fourier transform and the pre-sampled table."""

import os

import numpy as np
import pytest
from scipy import integrate

from oracle import kb

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()[:2]
        out[k] = float(v)
    return out


@pytest.mark.parametrize("J", [4, 6, 8])
def test_kernel_even_peak_and_open_support(J):
    beta = kb.default_beta(J)
    t = np.linspace(-J / 2, J / 2, 1001)
    assert np.array_equal(kb.kernel(t, J, beta), kb.kernel(-t, J, beta))  # g(u) = g(-u), Sec. 8.1
    assert kb.kernel(0.0, J, beta) == pytest.approx(1.0, abs=0.0)
    assert kb.kernel(J / 2, J, beta) == 0.0 and kb.kernel(-J / 2, J, beta) == 0.0
    assert kb.kernel(J / 2 + 0.3, J, beta) == 0.0
    # strictly decreasing on [0, J/2)
    tt = np.linspace(0, J / 2, 400, endpoint=False)
    assert np.all(np.diff(kb.kernel(tt, J, beta)) < 0)


@pytest.mark.parametrize("J", [4, 6])
@pytest.mark.parametrize("nu", [0.0, 0.05, 0.125, 0.2, 0.25, 0.4, 1.0])
def test_kernel_ft_matches_quadrature(J, nu):
    beta = kb.default_beta(J)
    f = lambda t: kb.kernel(t, J, beta) * np.cos(2 * np.pi * nu * t)
    val, err = integrate.quad(f, -J / 2, J / 2, epsabs=1e-15, epsrel=1e-14, limit=200)
    assert kb.kernel_ft(nu, J, beta) == pytest.approx(val, rel=1e-12, abs=1e-14)


def test_kernel_ft_small_beta_is_sinc():
    # beta -> 0: g -> box of width J, whose transform is J sinc(J nu)
    J = 4
    nu = np.array([0.01, 0.1, 0.2, 0.3, 0.45])
    assert np.allclose(kb.kernel_ft(nu, J, 1e-9), J * np.sinc(J * nu), rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("J,S", [(4, 4096), (6, 4096), (4, 64)])
def test_table_layout(J, S):
    beta = kb.default_beta(J)
    tab = kb.table(J, S, beta)
    assert len(tab) == (J // 2) * S + 1
    assert tab[0] == 1.0 and tab[-1] == 0.0
    assert np.all(np.diff(tab) < 0)


def test_zeroth_order_error_bound():
    # nearest-sample interpolation error <= max|g'| / (2 S), away from the jump of the open support
    # at |t| = J/2 (g(J/2 - 0) = 1 / I0(beta), g(J/2) = 0)
    J, S = 4, 4096
    beta = kb.default_beta(J)
    t = np.linspace(0, J / 2 - 1.0 / S, 200001)
    exact = kb.kernel(t, J, beta)
    idx = np.floor(t * S + 0.5).astype(int)
    approx = kb.table(J, S, beta)[idx]
    dg = np.max(np.abs(np.gradient(exact, t)))
    assert np.max(np.abs(approx - exact)) <= dg / (2 * S) * 1.01


def test_paper_presampling_claim():
    """Sec. 8.1: 2e5 samples per pixel make zeroth-order interpolation accurate to 1e-5, and J = 4
    then needs 4e5 samples (half of the symmetric support)."""
    g = golden()
    S = int(g["kb_presamples_per_pixel"])
    J = int(g["kb_support_J"])
    beta = kb.default_beta(J)
    assert (J // 2) * S == int(g["kb_presamples_total_J4"])
    t = np.random.default_rng(0).uniform(0, J / 2 - 1.0 / S, 200000)
    tab = kb.table(J, S, beta)
    approx = tab[np.floor(t * S + 0.5).astype(int)]
    assert np.max(np.abs(approx - kb.kernel(t, J, beta))) <= g["kb_presampling_accuracy"]


def test_paper_storage_arithmetic():
    """Sec. 8.1 / 8.2 bookkeeping: stored G for J = 4, M = 1e8 and the 48-byte visibility record."""
    g = golden()
    J, M = 4, 1e8
    assert J * J * M * 16 == pytest.approx(g["stored_G_bytes_J4_M1e8"])
    assert 16 + 16 + 8 + 8 == g["dataset_bytes_per_vis"]
    assert 5e10 * g["dataset_bytes_per_vis"] == pytest.approx(g["dataset_bytes_5e10_vis"])


def test_correction_is_reciprocal_ft():
    n, K, J = 16, 32, 4
    beta = kb.default_beta(J)
    c = kb.correction_1d(n, K, J, beta)
    p = np.arange(n) - n // 2
    assert np.allclose(c * kb.kernel_ft(p / K, J, beta), 1.0, rtol=1e-15)
    assert np.allclose(c, c[::-1][np.r_[n - 1, 0:n - 1]], rtol=0)  # even about p' = 0
