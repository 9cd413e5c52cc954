"""GPU parity of Phi / Phi^dagger (through the C ABI) against the FP64 oracle.

Bar: relative L2 error <= 1e-5 per application in FP32 (table mode: both sides
quantise the coordinates identically in FP64, so the tap indices and weights
agree exactly up to the FP32 rounding of the table); integer work (quantisation,
sort) bit-exact.
"""

import numpy as np
import pytest

import synth
from oracle import measurement as me

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1903_04502_gb300 as g
    g.library()
    return g


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make(n, M, J=4, seed=0, outliers=0.2, weights="uniform"):
    x = synth.sky(n, 5, 3, seed=seed) + 0.01 * synth.uniform(n * n, seed=seed + 7).reshape(n, n)
    uvw = synth.uv_coverage(M, seed=seed + 1, outlier_frac=outliers, weights=weights)
    return x.astype(np.float32), uvw


CASES = [  # (n_side, M, J): several tiles, ragged chunk tails
    (128, 20_000, 4),
    (64, 5_003, 6),
    (96, 1_537, 4),
    (256, 70_001, 4),
]


@pytest.mark.parametrize("taps", ["poly", "table", "poly-runs"])
@pytest.mark.parametrize("n,M,J", CASES)
def test_phi_and_adjoint_match_oracle(g, monkeypatch, n, M, J, taps):
    """Both ways of getting the tap weights of an FP32 plan: the polynomial fit (the default;
    at J = 4 on the step layout, or on the run layout with layout=1) and the
    shared-memory table (GBRI_TAP_TABLE=1)."""
    x, uvw = make(n, M, J, seed=n + M)
    geo = me.Geometry(uvw, n, 2, J, 4096)
    if taps == "table":
        monkeypatch.setenv("GBRI_TAP_TABLE", "1")
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, S=4096, layout=1 if taps == "poly-runs" else 0)
    monkeypatch.delenv("GBRI_TAP_TABLE", raising=False)
    assert plan.tap_mode() == (0 if taps == "table" else 2)
    y = g.phi(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    y_ref = me.phi(x.astype(np.float64), geo)
    assert rel(y, y_ref) <= TOL
    yin = synth.complex_normal(M, seed=3).astype(np.complex64)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    xa_ref = me.phi_adjoint(yin.astype(np.complex128), geo)
    assert rel(xa, xa_ref) <= TOL


@pytest.mark.parametrize("n,os,J,M,prec", [
    (48, 3, 4, 9_000, "f32"),     # K = 144: not a power of two (half spectrum, mirrored window)
    (80, 3, 6, 12_001, "f32"),
    (20, 4, 4, 3_001, "f32"),     # n % 8 == 4: the one-pixel-per-thread pad
    (36, 4, 6, 5_000, "f64"),
])
def test_oversampling_factors_match_oracle(g, n, os, J, M, prec):
    x, uvw = make(n, M, J, seed=n * os + M)
    geo = me.Geometry(uvw, n, os, J, 4096)
    F = g.F64 if prec == "f64" else g.F32
    tol = 1e-11 if prec == "f64" else TOL
    dt, ct = (np.float64, np.complex128) if prec == "f64" else (np.float32, np.complex64)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, oversample=os, J=J, S=4096, precision=F)
    assert plan.K == os * n
    y = g.phi(plan, torch.from_numpy(x.astype(dt)).cuda()).cpu().numpy()
    assert rel(y, me.phi(x.astype(np.float64), geo)) <= tol
    yin = synth.complex_normal(M, seed=5).astype(ct)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin.astype(np.complex128), geo)) <= tol


@pytest.mark.parametrize("n,M,J,prec", [
    (128, 20_000, 4, "f32"),
    (64, 5_003, 6, "f32"),
    (96, 1_537, 4, "f64"),
    (48, 9_000, 6, "f64"),
])
def test_first_order_interpolation_matches_oracle(g, n, M, J, prec):
    """First-order table mode (interp_order = 1) against the oracle's linear mode."""
    x, uvw = make(n, M, J, seed=2 * n + M)
    geo = me.Geometry(uvw, n, 2, J, 4096, mode="linear")
    F = g.F64 if prec == "f64" else g.F32
    tol = 1e-11 if prec == "f64" else TOL
    dt, ct = (np.float64, np.complex128) if prec == "f64" else (np.float32, np.complex64)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, S=4096, precision=F, interp_order=1)
    y = g.phi(plan, torch.from_numpy(x.astype(dt)).cuda()).cpu().numpy()
    assert rel(y, me.phi(x.astype(np.float64), geo)) <= tol
    yin = synth.complex_normal(M, seed=4).astype(ct)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin.astype(np.complex128), geo)) <= tol


def test_first_order_interpolation_is_closer_to_the_exact_kernel(g):
    """On the device, the FP64 first-order operator is about 256 times closer to the operator
    with the exactly evaluated kernel than the zeroth-order one (its coordinate step is
    256 times finer); both against the oracle's exact mode.  J = 6: at J = 4 the kernel's jump
    at the edge of its open support, 1 / I0(beta) = 6.5e-4, bounds the first-order gain
    (the oracle measures 14 times on this case; 263 times at J = 6)."""
    n, M, J = 64, 6_000, 6
    x, uvw = make(n, M, J, seed=17)
    y_ex = me.phi(x.astype(np.float64), me.Geometry(uvw, n, 2, J, 4096, mode="exact"))
    xd = torch.from_numpy(x.astype(np.float64)).cuda()
    errs = []
    for order in (0, 1):
        plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, S=4096, precision=g.F64, interp_order=order)
        errs.append(rel(g.phi(plan, xd).cpu().numpy(), y_ex))
    assert errs[1] <= 5e-7
    assert errs[0] >= 100 * errs[1], errs


def test_interp_order_rejected(g):
    x, uvw = make(32, 100, 4)
    with pytest.raises(g.GbriError):
        g.Plan(torch.from_numpy(uvw).cuda(), 32, interp_order=2)


@pytest.mark.parametrize("J,prec", [(4, "f32"), (6, "f32"), (4, "f64")])
def test_split_tiles_match_oracle(g, J, prec):
    """A dense small grid (128^2 cells, 2e5 visibilities: about 3000 per 16 x 16 tile against
    a per-item cap near 1000): the gridding cuts heavy tiles into several work items whose
    warps flush every cell with atomics."""
    n, M = 64, 200_000
    x, uvw = make(n, M, J, seed=31)
    geo = me.Geometry(uvw, n, 2, J, 4096)
    F = g.F64 if prec == "f64" else g.F32
    tol = 1e-11 if prec == "f64" else TOL
    ct = np.complex128 if prec == "f64" else np.complex64
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J, precision=F)
    yin = synth.complex_normal(M, seed=6).astype(ct)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin.astype(np.complex128), geo)) <= tol


def test_plan_order_and_permutation(g):
    n, M = 128, 12_345
    x, uvw = make(n, M)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    perm = plan.permutation().cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(M))
    xd = torch.from_numpy(x).cuda()
    y_raw = g.phi(plan, xd).cpu().numpy()
    y_plan = g.phi(plan, xd, plan_order=True).cpu().numpy()
    assert np.array_equal(y_plan, y_raw[perm])
    back = g.vis_reorder(plan, torch.from_numpy(y_plan).cuda(), to_plan=False).cpu().numpy()
    assert np.array_equal(back, y_raw)
    # the adjoint in plan order equals the adjoint in caller order
    yin = synth.complex_normal(M, seed=9).astype(np.complex64)
    a = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    b = g.phi_adjoint(plan, torch.from_numpy(yin[perm]).cuda(), plan_order=True).cpu().numpy()
    assert rel(b, a) <= 1e-6


def expected_plan_order(tile, cell, K, T, R, load=2, steps=True):
    """(tile, cell) of every plan position under the plan's layout rule: non-empty 16 x 16
    tiles heaviest first (ties by tile index); inside a tile the runs (up to R consecutive
    visibilities of one cell) round by round (every cell's first run, then every second
    one, ...); inside a round in bands ceil(length / 2), most first; inside a band round
    robin over the 16 shared-memory bank slots (row * 22 + col) mod 16 of the cell, in cell
    order within a slot; each round padded with empty runs to a multiple of 32.  Run layout
    (steps=False): each run's visibilities consecutive.  Step layout (FP32 polynomial-tap
    plans with J = 4): every group of 32 runs step-major, step k holding the k-th visibility
    of each run longer than k in run order."""
    counts = np.bincount(tile, minlength=(K // T) ** 2)
    tiles = np.nonzero(counts)[0]
    order = tiles[np.argsort(-counts[tiles], kind="stable")]
    exp_t, exp_c = [], []
    for t in order:
        cc = np.bincount(cell[tile == t], minlength=T * T)
        for r in range(int(-(-cc.max() // R))):
            ln = {c: min(R, cc[c] - r * R) for c in range(T * T) if cc[c] > r * R}
            bands = {c: -(-ln[c] // load) for c in ln}
            runs = []
            for b in range(max(bands.values()), 0, -1):
                buckets = [[c for c in sorted(ln) if bands[c] == b and ((c // T) * 22 + c % T) % 16 == q]
                           for q in range(16)]
                while any(buckets):
                    for q in range(16):
                        if buckets[q]:
                            runs.append(buckets[q].pop(0))
            runs += [None] * (-len(runs) % 32)
            for g0 in range(0, len(runs), 32):
                grp = runs[g0:g0 + 32]
                lens = [ln[c] if c is not None else 0 for c in grp]
                if steps:
                    for k in range(max(lens)):
                        for j, c in enumerate(grp):
                            if lens[j] > k:
                                exp_t.append(t)
                                exp_c.append(c)
                else:
                    for j, c in enumerate(grp):
                        exp_t += [t] * lens[j]
                        exp_c += [c] * lens[j]
    return np.array(exp_t), np.array(exp_c), len(tiles)


@pytest.mark.parametrize("run,layout", [(0, "steps"), (2, "steps"), (0, "runs"), (2, "runs"), (0, "runs-poly")])
def test_sort_is_bit_exact_tile_major(g, monkeypatch, run, layout):
    """The plan's visibility order follows the oracle's FP64 quantisation exactly (integer
    work, compared exactly) under the layout rule of expected_plan_order; run 0 is the
    default run length 64, run 2 splits cells into several rounds.  The default FP32 J = 4
    plan takes the step layout; the table-tap plan (GBRI_TAP_TABLE=1) and a polynomial-tap plan
    asking for layout=1 the run layout."""
    n, M, K, S, T = 128, 30_000, 256, 4096, 16
    R = run or 64
    _, uvw = make(n, M)
    if layout == "runs":
        monkeypatch.setenv("GBRI_TAP_TABLE", "1")
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, S=S, vis_per_run=run, layout=1 if layout == "runs-poly" else 0)
    monkeypatch.delenv("GBRI_TAP_TABLE", raising=False)
    assert plan.tap_mode() == (0 if layout == "runs" else 2)
    assert plan.launch_config()[0] == R
    perm = plan.permutation().cpu().numpy()
    assert np.array_equal(np.sort(perm), np.arange(M))
    kx = me.quantise(uvw[:, 0], K, S)
    ky = me.quantise(uvw[:, 1], K, S)
    cx = np.mod(np.floor_divide(kx, S), K)
    cy = np.mod(np.floor_divide(ky, S), K)
    tile = (cy // T) * (K // T) + cx // T
    cell = (cy % T) * T + (cx % T)
    exp_t, exp_c, n_tiles = expected_plan_order(tile, cell, K, T, R, steps=(layout == "steps"))
    assert np.array_equal(tile[perm], exp_t)
    assert np.array_equal(cell[perm], exp_c)
    assert plan.n_tiles == n_tiles


def test_adjoint_identity_on_gpu(g):
    n, M = 256, 100_000
    x, uvw = make(n, M, seed=5)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    y = synth.complex_normal(M, seed=6).astype(np.complex64)
    px = g.phi(plan, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    pty = g.phi_adjoint(plan, torch.from_numpy(y).cuda()).cpu().numpy().astype(np.float64)
    lhs = np.real(np.vdot(px, y.astype(np.complex128)))
    rhs = np.vdot(x.astype(np.float64), pty)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_edge_cases(g):
    n = 64
    # empty visibility set
    plan = g.Plan(torch.zeros((0, 4), dtype=torch.float32, device="cuda"), n)
    x = torch.rand((n, n), device="cuda")
    assert g.phi(plan, x).numel() == 0
    assert float(g.phi_adjoint(plan, torch.zeros(0, dtype=torch.complex64, device="cuda")).abs().max()) == 0.0
    # Nyquist edge (u, v = +-pi wrap), the origin, and a pile-up of identical points in one cell
    pts = np.array([[np.pi, 0.3, 0, 1], [-np.pi, 0.3, 0, 1], [0.2, np.pi, 0, 0.5], [0.2, -np.pi, 0, 0.5],
                    [0.0, 0.0, 0, 1.0]], dtype=np.float32)
    pile = np.tile(np.array([[0.01, -0.02, 0, 0.75]], dtype=np.float32), (3000, 1))
    uvw = np.concatenate([pts, pile])
    xs = synth.uniform(n * n, seed=2).reshape(n, n).astype(np.float32)
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n)
    y = g.phi(plan, torch.from_numpy(xs).cuda()).cpu().numpy()
    assert rel(y, me.phi(xs.astype(np.float64), geo)) <= TOL
    assert y[0] == pytest.approx(y[1], rel=1e-6)
    yin = synth.complex_normal(len(uvw), seed=4).astype(np.complex64)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin.astype(np.complex128), geo)) <= TOL


def test_invalid_inputs_rejected(g):
    n = 32
    bad = np.array([[np.nan, 0, 0, 1]], dtype=np.float32)
    with pytest.raises(g.GbriError) as e:
        g.Plan(torch.from_numpy(bad).cuda(), n)
    assert e.value.code == -6
    far = np.array([[100.0, 0, 0, 1]], dtype=np.float32)
    with pytest.raises(g.GbriError):
        g.Plan(torch.from_numpy(far).cuda(), n)
    with pytest.raises(g.GbriError):
        g.Plan(torch.zeros((4, 4), device="cuda"), n, J=5)
    with pytest.raises(g.GbriError):
        g.Plan(torch.zeros((4, 4), device="cuda"), n, layout=2)


def test_full_size_sampled_parity(g):
    """1024^2 image, 2048^2 grid, J = 4, M = 1e7 (the FP32 workload), same launch path as the
    benchmark: sampled outputs of Phi against the oracle one by one, and the adjoint identity."""
    cfg = synth.CONFIGS["large"]
    n, M = cfg["n_side"], cfg["M"]
    x = synth.sky(n, cfg["n_points"], cfg["n_blobs"], seed=0).astype(np.float32)
    uvw = synth.uv_coverage(M, seed=1, outlier_frac=cfg["outlier_frac"], weights=cfg["weights"])
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=4, S=4096)
    y = g.phi(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    idx = np.random.default_rng(0).choice(M, 4000, replace=False)
    idx = np.concatenate([idx, [0, M - 1]])
    geo = me.Geometry(uvw[idx], n, 2, 4, 4096)
    y_ref = me.phi(x.astype(np.float64), geo)
    assert rel(y[idx], y_ref) <= TOL
    yin = torch.randn(M, dtype=torch.complex64, device="cuda")
    pty = g.phi_adjoint(plan, yin).double()
    lhs = torch.real(torch.vdot(torch.from_numpy(y).cuda().to(torch.complex128), yin.to(torch.complex128)))
    rhs = torch.dot(torch.from_numpy(x).cuda().double().ravel(), pty.ravel())
    assert abs(float(lhs - rhs)) <= 1e-5 * abs(float(lhs))


@pytest.mark.parametrize("vis_per_run", [1, 2])
def test_run_length_variants_match_oracle(g, vis_per_run):
    n, M = 128, 25_000
    x, uvw = make(n, M, seed=77)
    geo = me.Geometry(uvw, n, 2, 4, 4096)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, vis_per_run=vis_per_run)
    assert plan.launch_config()[0] == vis_per_run
    y = g.phi(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, me.phi(x.astype(np.float64), geo)) <= TOL
    yin = synth.complex_normal(M, seed=78).astype(np.complex64)
    xa = g.phi_adjoint(plan, torch.from_numpy(yin).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(yin.astype(np.complex128), geo)) <= TOL


def test_autotuned_plan_matches_oracle_and_is_cached(g):
    n, M = 256, 200_000
    x, uvw = make(n, M, seed=79)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, autotune=True)
    run, dg, gr = plan.launch_config()
    assert run in (8, 16, 64) and dg >= 1 and gr >= 1
    idx = np.arange(0, M, 97)
    geo = me.Geometry(uvw[idx], n, 2, 4, 4096)
    y = g.phi(plan, torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y[idx], me.phi(x.astype(np.float64), geo)) <= TOL
    again = g.Plan(torch.from_numpy(uvw).cuda(), n, autotune=True)   # same shape: cached choice
    assert again.launch_config() == (run, dg, gr)


@pytest.mark.parametrize("n,M,J,sig", [(32, 2_000_000, 6, np.pi / 40), (64, 4_000_000, 4, np.pi / 3)])
def test_heavy_tile_density_accuracy(g, n, M, J, sig):
    """Plain FP32 accumulation at extreme densities: 2e6 visibilities on a 64^2 grid (a third of
    a million in the densest cell, 5e5 in one tile) and 4e6 on a 128^2 grid, with coherent data
    (y = Phi x of a sky) for Phi^dagger.  Each visibility's taps are summed in registers over
    its run (at most 64 visibilities of one cell) and the runs into the tile accumulator, so
    rounding grows with the number of runs per cell, not of visibilities; the FP32 path stays
    within 1e-6 of the oracle here, an order of magnitude inside the 1e-5 bar, which is why
    the sums are not compensated."""
    uvw = synth.uv_coverage(M, seed=5, outlier_frac=0.0, weights="uniform", sigma=sig)
    x = synth.sky(n, 5, 3, seed=3)
    geo = me.Geometry(uvw, n, 2, J, 4096)
    y_ref = me.phi(x, geo)
    plan = g.Plan(torch.from_numpy(uvw).cuda(), n, J=J)
    y = g.phi(plan, torch.from_numpy(x.astype(np.float32)).cuda()).cpu().numpy()
    assert rel(y, y_ref) <= 1e-6
    y32 = y_ref.astype(np.complex64)
    xa = g.phi_adjoint(plan, torch.from_numpy(y32).cuda()).cpu().numpy()
    assert rel(xa, me.phi_adjoint(y32.astype(np.complex128), geo)) <= 1e-6
