"""The bounds-checked build (libgbri_debug.so, -DGBRI_DEBUG): on the parity cases of every
visibility-kernel variant (FP32 polynomial and table taps, first-order table, FP64,
deterministic gridding, J = 4 and 6, Nyquist points and a pile-up in one cell, the fused
primal-dual pass, FISTA's residual pass, a batch's shared pass over two problems) no window, accumulator, grid, half-spectrum, slot or
visibility index leaves its buffer (the plan's error word stays zero), and the results still
match the oracle.  Runs in a child process, since one process loads one library build."""

import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import os, sys
sys.path.insert(0, %(root)r)
import numpy as np, torch
import paper_1903_04502_gb300 as g
from paper_1903_04502_gb300 import _lib
import synth
from oracle import measurement as me
assert _lib.LIB_PATH.endswith("libgbri_debug.so"), _lib.LIB_PATH

def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))

def check(plan, tag):
    bits, idx = plan.debug_word()
    assert bits == 0, (tag, bits, idx)

n_cases = 0
for (n, M, J, kw, env, prec) in [
        (128, 20_000, 4, {}, None, "f32"), (64, 5_003, 6, {}, None, "f32"),
        (96, 9_000, 4, {}, "1", "f32"), (64, 6_000, 6, {"interp_order": 1}, None, "f32"),
        (64, 8_000, 4, {}, None, "f64"), (64, 120_000, 4, {"deterministic": True}, None, "f32"),
        (64, 120_000, 6, {"deterministic": True}, None, "f64")]:
    if env:
        os.environ["GBRI_TAP_TABLE"] = env
    uvw = synth.uv_coverage(M, seed=n + M, outlier_frac=0.2, weights="uniform")
    edge = np.array([[np.pi, 0.3, 0, 1], [-np.pi, 0.3, 0, 1], [0.2, np.pi, 0, 0.5], [0.2, -np.pi, 0, 0.5]],
                    dtype=np.float32)
    pile = np.tile(np.array([[0.01, -0.02, 0, 0.75]], dtype=np.float32), (500, 1))
    uvw = np.concatenate([uvw, edge, pile])
    x = synth.sky(n, 4, 2, seed=n) + 0.01 * synth.uniform(n * n, seed=n + 1).reshape(n, n)
    order = kw.get("interp_order", 0)
    geo = me.Geometry(uvw, n, 2, J, 4096, mode="linear" if order else "table")
    p = g.F64 if prec == "f64" else g.F32
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, precision=p, **kw)
    os.environ.pop("GBRI_TAP_TABLE", None)
    xin = x if prec == "f64" else x.astype(np.float32)
    y = g.phi(plan, torch.from_numpy(xin).cuda()).cpu().numpy()
    assert rel(y, me.phi(xin.astype(np.float64), geo)) <= 1e-5
    yin = synth.complex_normal(len(uvw), seed=3)
    yin = yin if prec == "f64" else yin.astype(np.complex64)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin.astype(np.complex128), geo)) <= 1e-5
    check(plan, ("operators", n, M, J, kw, env, prec))
    wav = g.Wavelet(n, 2, (0, 1, 2), precision=p)
    for algo in (g.ALGO_PD, g.ALGO_FISTA):
        s = g.Solver(plan, wav, torch.from_numpy(yin).cuda(), eps=1.0, op_norm_sq=float(len(uvw)), gamma=1e-3,
                     algo=algo)
        s.step(5)
        torch.cuda.synchronize()
        check(plan, ("solver", algo, n, M, J, kw, env, prec))
        s.close()
    n_cases += 1
# the batch's shared fused pass (k_steps_multi) over two primal-dual members
b, keep = g.Batch(), []
for k, (n, M) in enumerate([(64, 6_000), (96, 9_000)]):
    uvw = synth.uv_coverage(M, seed=50 + k, outlier_frac=0.2, weights="uniform")
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=4)
    wav = g.Wavelet(n, 2, (0, 1, 2))
    yin = synth.complex_normal(M, seed=60 + k).astype(np.complex64)
    s = g.Solver(plan, wav, torch.from_numpy(yin).cuda(), eps=1.0, op_norm_sq=float(M), gamma=1e-3)
    b.add(s)
    keep.append((plan, wav, s))
b.step(5)
torch.cuda.synchronize()
assert b.shared_members() == 2
for plan, _, _ in keep:
    check(plan, "shared pass")
b.close()
n_cases += 1
print("DEBUG_BUILD_OK", n_cases)
'''


def test_bounds_checked_build_reports_no_violation():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = os.path.join(ROOT, "paper_1903_04502_gb300", "libgbri_debug.so")
    if not os.path.exists(lib):
        from paper_1903_04502_gb300 import build
        build.build(debug=True)
    env = dict(os.environ, GBRI_DEBUG_LIB="1")
    r = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "DEBUG_BUILD_OK 8" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_default_build_has_no_checks():
    """The default library rejects the bounds-check report (its kernels carry no checks)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04502_gb300 as g
    import synth
    plan = g.Plan(torch.from_numpy(synth.uv_coverage(100, seed=1)).cuda(), 32)
    with pytest.raises(g.GbriError):
        plan.debug_word()
