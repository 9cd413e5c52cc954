"""Pins for the oracle's measurement operator: brute-force NUDFT, adjoint identity, symmetries."""

import numpy as np
import pytest

import synth
from oracle import measurement as me


def _case(n, M, seed):
    x = synth.uniform(n * n, seed=seed).reshape(n, n)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=0.2, weights="uniform")
    return x, uvw


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# Band of the gridding error against the measurement equation (Eq. 1), exact kernel, oversampling 2.
# The paper states no bound for its Kaiser-Bessel choice; these bands were calibrated once and each is
# about 2-4x above the measured error, so a dropped correction, a wrong sign or a transposed axis fails.
BAND = {4: 2e-3, 6: 3e-5, 8: 5e-7}


@pytest.mark.parametrize("n", [8, 16, 32])
def test_phi_exact_kernel_matches_nudft_band_and_monotone(n):
    x, uvw = _case(n, 500, seed=10 + n)
    y_true = me.nudft(x, uvw)
    errs = []
    for J in (4, 6, 8):
        geo = me.Geometry(uvw, n, 2, J, 4096, mode="exact")
        e = _rel(me.phi(x, geo), y_true)
        assert e <= BAND[J], (J, e)
        errs.append(e)
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("J", [4, 6])
def test_table_mode_within_table_step_of_exact(J):
    n = 32
    x, uvw = _case(n, 400, seed=3)
    ex = me.phi(x, me.Geometry(uvw, n, 2, J, 4096, mode="exact"))
    tb = me.phi(x, me.Geometry(uvw, n, 2, J, 4096, mode="table"))
    # per-tap weight error <= max|g'| / (2 S) ~ 2e-4 for S = 4096; over J^2 taps in L2
    assert _rel(tb, ex) < 5e-4
    # and the nudft error of table mode is bounded by the sum of both
    assert _rel(tb, me.nudft(x, uvw)) <= BAND[J] + 5e-4


@pytest.mark.parametrize("J", [4, 6])
def test_linear_mode_weights_within_interpolation_bound(J):
    """First-order table (reading R13) against the kernel at the unquantised position.  Away
    from the support's last table step the error is at most max|g''| / (8 S^2) (linear
    interpolation) + max|g'| / (2 S F) (coordinate quantised to 1 / (S F) of a cell); in the
    last step at most the jump of the open support, g(J/2 -) = 1 / I0(beta)."""
    from oracle import kb
    K, S, F = 64, 4096, 256
    beta = kb.default_beta(J)
    tab = kb.table(J, S, beta)
    u = np.random.default_rng(1).uniform(-np.pi, np.pi, 100_000)
    cells, w = me.tap_weights_linear(u, K, J, S, tab, F)
    k = u * K / (2 * np.pi)
    ex_cells = np.floor(k).astype(np.int64)[:, None] - J // 2 + 1 + np.arange(J)[None, :]
    same = (np.mod(ex_cells, K) == cells).all(axis=1)
    assert same.mean() > 0.999
    d = np.abs(k[:, None] - ex_cells)[same]
    err = np.abs(w[same] - kb.kernel(d, J, beta))
    t = np.linspace(0.0, J / 2 - 1.0 / S, 400_001)
    g = kb.kernel(t, J, beta)
    g1 = np.abs(np.diff(g) / np.diff(t)).max()
    g2 = np.abs(np.diff(g, 2) / np.diff(t)[:-1] ** 2).max()
    inner = d < J / 2 - 1.0 / S
    assert err[inner].max() <= 1.01 * (g2 / (8 * S * S) + g1 / (2 * S * F))
    assert err[~inner].max() <= 1.0 / np.i0(beta) * 1.001
    # a wrong interpolation direction would miss by about max|g'| / S
    assert err[inner].max() < 0.01 * g1 / S


def test_linear_mode_equals_table_mode_on_samples():
    """Coordinates on table samples (k S an integer): first order reduces to zeroth order."""
    from oracle import kb
    K, S, J = 64, 4096, 4
    tab = kb.table(J, S, kb.default_beta(J))
    m = np.random.default_rng(2).integers(-K * S // 2, K * S // 2, 5000)
    u = m * (2 * np.pi / (K * S))
    c1, w1 = me.tap_weights_linear(u, K, J, S, tab, 256)
    c0, w0 = me.tap_weights_table(u, K, J, S, tab)
    assert (c1 == c0).all()
    assert np.abs(w1 - w0).max() <= 1e-15


@pytest.mark.parametrize("J", [4, 6])
def test_linear_mode_phi_closer_to_exact_than_table(J):
    """Phi's error against the exact kernel is dominated by the coordinate quantisation
    (a shift of at most half a quantisation step): 1 / (2 S) of a cell in table mode,
    1 / (2 S F) in first-order mode, so the first-order operator is about F times closer."""
    n = 32
    x, uvw = _case(n, 400, seed=3)
    ex = me.phi(x, me.Geometry(uvw, n, 2, J, 4096, mode="exact"))
    tb = me.phi(x, me.Geometry(uvw, n, 2, J, 4096, mode="table"))
    ln = me.phi(x, me.Geometry(uvw, n, 2, J, 4096, mode="linear"))
    assert _rel(ln, ex) <= 1e-6
    assert _rel(tb, ex) >= 100 * _rel(ln, ex)


@pytest.mark.parametrize("mode", ["table", "exact", "linear"])
@pytest.mark.parametrize("n,J", [(16, 4), (32, 6), (24, 4)])
def test_adjoint_identity(mode, n, J):
    x, uvw = _case(n, 700, seed=7)
    geo = me.Geometry(uvw, n, 2, J, 4096, mode=mode)
    y = synth.complex_normal(700, seed=8)
    lhs = np.real(np.vdot(me.phi(x, geo), y))
    rhs = np.vdot(x, me.phi_adjoint(y, geo))
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # complex image variant (no real part taken)
    xc = x + 1j * synth.uniform(n * n, seed=9).reshape(n, n)
    lhs = np.vdot(me.phi(xc, geo), y)
    rhs = np.vdot(xc, me.phi_adjoint(y, geo, real=False))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_adjoint_is_conjugate_transpose_of_dense_matrix():
    # brute force: build Phi column by column and compare Phi^dagger with its conjugate transpose
    n, M = 8, 40
    _, uvw = _case(n, M, seed=21)
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    A = np.zeros((M, n * n), dtype=np.complex128)
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        A[:, k] = me.phi(e.reshape(n, n), geo)
    y = synth.complex_normal(M, seed=22)
    assert np.allclose(me.phi_adjoint(y, geo).ravel(), np.real(A.conj().T @ y), rtol=1e-12, atol=1e-12)


def test_hermitian_symmetry_real_image():
    n = 16
    x, uvw = _case(n, 200, seed=31)
    mirror = uvw.copy()
    mirror[:, :2] *= -1
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    geo_m = me.Geometry(mirror, n, 2, 4, 4096)
    y = me.phi(x, geo)
    ym = me.phi(x, geo_m)
    assert np.allclose(ym, np.conj(y), rtol=1e-12, atol=1e-12 * np.abs(y).max())


def test_delta_at_origin_gives_weights():
    n = 32
    _, uvw = _case(n, 300, seed=41)
    x = np.zeros((n, n))
    x[n // 2, n // 2] = 1.0
    y = me.phi(x, me.Geometry(uvw, n, 2, 6, 4096, mode="exact"))
    assert np.allclose(y, uvw[:, 3], rtol=1e-4, atol=1e-4)


def test_nyquist_wraparound():
    # u = +pi and u = -pi land on the same grid column (k = +-K/2 wrap); the DFT agrees.
    n = 16
    x = synth.uniform(n * n, seed=51).reshape(n, n)
    uvw = np.array([[np.pi, 0.3, 0, 1], [-np.pi, 0.3, 0, 1], [0.2, np.pi, 0, 1], [0.2, -np.pi, 0, 1]],
                   dtype=np.float64)
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    y = me.phi(x, geo)
    assert y[0] == pytest.approx(y[1], rel=1e-12)
    assert y[2] == pytest.approx(y[3], rel=1e-12)
    yt = me.nudft(x, uvw)
    assert np.allclose(yt[0], yt[1]) and np.allclose(yt[2], yt[3])
    assert _rel(y, yt) < 5e-3  # the grid edge aliases a little more than the core


def test_quantisation_rounds_half_away_from_zero():
    K, S = 256, 4096
    scale = np.float64(K * S) / (2.0 * np.pi)
    u = np.array([0.5 / scale, -0.5 / scale, 1.49 / scale, -1.51 / scale, 0.0])
    q = me.quantise(u, K, S)
    # the float64 products are 0.5, -0.5, 1.49, -1.51, 0 up to one rounding
    assert list(q[2:]) == [1, -2, 0]
    assert abs(q[0]) in (0, 1) and q[0] == -q[1]


def test_phi_at_matches_full_phi():
    n = 32
    x, uvw = _case(n, 1000, seed=61)
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    idx = np.array([0, 5, 999, 500, 17])
    assert np.allclose(me.phi_at(x, geo, idx), me.phi(x, geo)[idx], rtol=1e-13, atol=0)


def test_empty_visibilities():
    n = 16
    geo = me.Geometry(np.zeros((0, 4)), n, 2, 4, 4096)
    assert me.phi(np.ones((n, n)), geo).shape == (0,)
    assert np.all(me.phi_adjoint(np.zeros(0, dtype=complex), geo) == 0)
