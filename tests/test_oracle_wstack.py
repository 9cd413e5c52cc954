"""Pins for the oracle's non-coplanar (w-stacking) operator (reading R14): the coplanar
reduction, the brute-force non-coplanar measurement equation within the gridding band plus
the w-quantisation bound, the adjoint identity, and convergence in the number of planes."""

import numpy as np
import pytest

import synth
from oracle import measurement as me, wstack as ws


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_screen_and_nudft_reduce_to_coplanar_when_w_is_zero():
    n = 16
    x = synth.uniform(n * n, seed=1).reshape(n, n)
    uvw = synth.uv_coverage(300, seed=2, weights="uniform").astype(np.float64)
    assert np.allclose(ws.screen(n, 0.02, 0.0), 1.0)
    assert np.allclose(ws.nudft_w(x, uvw, 0.02), me.nudft(x, uvw), rtol=1e-13, atol=1e-12)
    # n - 1 at the centre pixel is 0, negative elsewhere, and matches the closed form at a corner
    nm1 = ws.n_minus_1(n, 0.02)
    assert nm1[n // 2, n // 2] == 0.0 and np.all(nm1 <= 0)
    l = (0 - n // 2) * 0.02
    assert nm1[0, 0] == pytest.approx(np.sqrt(1 - 2 * l * l) - 1, rel=1e-15)


def test_all_w_equal_zero_matches_coplanar_operator():
    n, M = 32, 2000
    x = synth.uniform(n * n, seed=3).reshape(n, n)
    uvw = synth.uv_coverage(M, seed=4, outlier_frac=0.2, weights="uniform")
    st = ws.WStack(uvw, n, 0.01, n_planes=4)
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    assert np.allclose(ws.phi(x, st), me.phi(x, geo), rtol=1e-13, atol=1e-13)
    y = synth.complex_normal(M, seed=5)
    assert np.allclose(ws.phi_adjoint(y, st), me.phi_adjoint(y, geo), rtol=1e-12, atol=1e-12)


def test_adjoint_identity():
    n, M = 32, 1500
    x = synth.uniform(n * n, seed=6).reshape(n, n)
    uvw = synth.uvw_noncoplanar(M, seed=7, delta=0.02, w_frac=0.5)
    st = ws.WStack(uvw, n, 0.02, n_planes=5)
    y = synth.complex_normal(M, seed=8)
    lhs = np.real(np.vdot(ws.phi(x, st), y))
    rhs = np.vdot(x, ws.phi_adjoint(y, st))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_one_plane_at_a_common_w_matches_brute_force():
    """Every visibility at the same w: no w quantisation, so the stacked operator with the exact
    kernel is within the coplanar gridding band (J = 6: 3e-5) of the brute-force equation."""
    n, M = 32, 400
    x = synth.uniform(n * n, seed=9).reshape(n, n)
    uvw = synth.uv_coverage(M, seed=10, outlier_frac=0.2, weights="uniform").astype(np.float64)
    uvw[:, 2] = 250.0
    st = ws.WStack(uvw, n, 0.015, n_planes=1, J=6, mode="exact")
    assert _rel(ws.phi(x, st), ws.nudft_w(x, uvw, 0.015)) <= 3e-5


def test_stacked_operator_converges_to_brute_force_within_quantisation_bound():
    """The error against the brute-force equation is at most the gridding band plus the phase
    error of replacing w by its plane's centre, 2 pi (dw / 2) max|n - 1|; it shrinks as planes
    are added."""
    n, M, delta = 32, 600, 0.02
    x = synth.uniform(n * n, seed=11).reshape(n, n)
    uvw = synth.uvw_noncoplanar(M, seed=12, delta=delta, w_frac=0.5).astype(np.float64)
    y_true = ws.nudft_w(x, uvw, delta)
    max_nm1 = float(np.abs(ws.n_minus_1(n, delta)).max())
    span = float(uvw[:, 2].max() - uvw[:, 2].min())
    errs = []
    for planes in (2, 8, 32, 128, 512):
        st = ws.WStack(uvw, n, delta, n_planes=planes, J=6, mode="exact")
        e = _rel(ws.phi(x, st), y_true)
        bound = 3e-5 + 2 * np.pi * (span / planes / 2) * max_nm1
        assert e <= bound, (planes, e, bound)
        errs.append(e)
    assert all(a > b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 5e-3  # first order in dw: about 1 / planes


def test_plane_assignment_rule():
    w = np.array([-1.0, -0.5, 0.0, 0.49, 0.5, 1.0])
    k, c = ws.plane_index(w, 4)
    assert list(k) == [0, 1, 2, 2, 3, 3]          # w_hi falls in the last plane
    assert np.allclose(c, [-0.75, -0.25, 0.25, 0.75])
