"""Writes the stored oracle images of 200 primal-dual iterations (Appendix A.4, Algorithm 7).

Test infrastructure: this script calls only ``synth`` (seeded inputs) and ``oracle``
(the FP64 CPU implementation); nothing here comes from the CUDA path.  The GPU tests
regenerate the same inputs (sky, coverage, y, from the same seeds through the oracle's
own Phi) and compare the image their solver reaches with the stored one.

Problems (both with the SARA dictionary of the FP32 workload, Dirac + db1..db8 over 4
levels, weights uniform in [0.5, 1], 20 % uniform-disk outliers, 30 dB input SNR):

* ``pd200_256sq_M2e5.npz``: 256^2 sky (10 points, 4 blobs), 512^2 grid, J = 4, M = 2e5.
  ||Phi||^2 by the power method to 1e-8 (at most 200 iterations).  Image stored in FP64
  (the FP64 GPU path is held to 1e-9).
* ``pd200_1024sq_M1e7.npz``: the full FP32 workload, 1024^2 sky (50 points, 20 blobs),
  2048^2 grid, J = 4, M = 1e7.  ||Phi||^2 from 40 power iterations (a parameter passed to
  both sides; the estimate approaches the norm from below, which keeps the step-size
  condition of Algorithm 7).  Image stored in FP32 (the bar is 1e-4).  About 1.5 h on
  8 host cores.

y0 = Phi x_true is the oracle's Phi in FP64; sigma = 10^(-30/20) ||y0|| / sqrt(M); the
noise is ``synth.complex_normal(M, seed + 2)``; y = complex64(y0 + sigma n) and the
oracle runs on that rounded y (cast back to complex128), as the GPU does.  eps by the
chi-square rule, gamma = 1e-3 max|Psi^dagger Phi^dagger y| / ||Phi||^2.

Usage: python tests/golden/make_pd_golden.py [small|large|all]
"""

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import measurement as me, solvers as so, wavelets as wv  # noqa: E402

ORDERS = (0, 1, 2, 3, 4, 5, 6, 7, 8)
LEVELS = 4

PROBLEMS = {
    "small": dict(file="pd200_256sq_M2e5.npz", n=256, M=200_000, npts=10, nblobs=4, seed=40,
                  power_iters=200, power_tol=1e-8, iters=200, store=np.float64),
    "large": dict(file="pd200_1024sq_M1e7.npz", n=1024, M=10_000_000, npts=50, nblobs=20, seed=0,
                  power_iters=40, power_tol=1e-9, iters=200, store=np.float32),
}


def inputs(n, M, npts, nblobs, seed):
    """Sky, coverage, oracle geometry and operators, and the rounded data y (see the module text)."""
    x_true = synth.sky(n, npts, nblobs, seed=seed)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=0.2, weights="uniform")
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    ops = (lambda v: me.phi(v, geo), lambda v: me.phi_adjoint(v, geo),
           lambda a: wv.psi(a, ORDERS, LEVELS), lambda v: wv.psi_adjoint(v, ORDERS, LEVELS))
    y0 = ops[0](x_true)
    sigma = 10 ** (-30 / 20) * float(np.linalg.norm(y0)) / np.sqrt(M)
    y = (y0 + sigma * synth.complex_normal(M, seed=seed + 2)).astype(np.complex64)
    return x_true, uvw, geo, ops, y, sigma


def make(name):
    p = PROBLEMS[name]
    t0 = time.time()
    x_true, uvw, geo, ops, y, sigma = inputs(p["n"], p["M"], p["npts"], p["nblobs"], p["seed"])
    yd = y.astype(np.complex128)
    eps = so.epsilon_from_sigma(sigma, p["M"])
    opn, pit = so.power_iteration(ops[0], ops[1], (p["n"], p["n"]), seed=0, max_iter=p["power_iters"],
                                  tol=p["power_tol"])
    gamma = so.default_gamma(yd, ops[1], ops[3], opn)
    print(f"{name}: inputs and parameters in {time.time() - t0:.0f} s (power iterations {pit})", flush=True)
    x, info = so.primal_dual(yd, *ops, so.PDParams(gamma=gamma, op_norm_sq=opn, eps=eps, max_iter=p["iters"]))
    print(f"{name}: {p['iters']} iterations done at {time.time() - t0:.0f} s, rel change {info['rel_change']:.3e}",
          flush=True)
    np.savez_compressed(os.path.join(HERE, p["file"]), x=x.astype(p["store"]), op_norm_sq=opn, gamma=gamma,
                        eps=eps, sigma=sigma, iters=p["iters"], power_iters=pit,
                        rel_change=info["rel_change"], residual_norm=info["residual_norm"],
                        n=p["n"], M=p["M"], npts=p["npts"], nblobs=p["nblobs"], seed=p["seed"])


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    for k in (PROBLEMS if which == "all" else [which]):
        make(k)
