"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Sizes span several line tiles with ragged tails (tiles hold 8 lines), every
phase-encoding axis position (first, middle, last), every faces-per-lane
class (K = 3, 5, 9, 15), and lines with active constraints.  The FP64 path
must match to 1e-9 relative (Sec. 4.2 ADMM after a fixed number of
iterations); the mixed path to 1e-3 voxel in b and 1e-6 relative objective.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1607_00531_gb300 import phantoms as ph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ((37, 50), 1),          # 2D, contiguous lines, 5 tiles (ragged), K = 3
    ((9, 70, 21), 1),       # 3D, PE middle, inner tiles 8 + 8 + 5, K = 3
    ((40, 7, 9), 0),        # PE first: one outer, 63 inner lines
    ((6, 7, 100), 2),       # PE last: contiguous lines, K = 5
    ((5, 256, 11), 1),      # K = 9
    ((3, 300), 1),          # K = 15
]


@pytest.fixture(scope="module")
def sac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00531_gb300 import build, sac as S
    build.build()
    return S


def cu(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def f32(a):
    """FP32 rounding of an array, kept in FP64 (the values FP32 storage holds)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def knot_lines(og, b):
    """Per line (the faces along the PE axis, moved last and flattened): whether
    some cell's displaced position j +- A1 b / h lies within FP32 rounding of
    a knot of the image model (an integer), where an FP32 and an FP64 position
    can fall in different intervals (Sec. 3's model is piecewise linear)."""
    pe, h = og.pe, og.h[og.pe]
    bl = np.moveaxis(np.asarray(b, dtype=np.float64), pe, -1).reshape(-1, b.shape[pe])
    a = 0.5 * (bl[:, :-1] + bl[:, 1:])
    j = np.arange(a.shape[1], dtype=np.float64)
    near = np.zeros(bl.shape[0], dtype=bool)
    for sgn in (1.0, -1.0):
        t = j + sgn * a / h
        tol = 4.0 * np.spacing(np.maximum(np.abs(t), 1.0).astype(np.float32)).astype(np.float64)
        near |= np.any(np.abs(t - np.round(t)) <= tol, axis=1)
    return near


def lines_off_the_plain_oracle(og, prm, I1, I2, b, z, u, out):
    """The mixed b-step against the plain FP64 oracle (intervals decided in
    FP64) on the FP32-rounded inputs: lines off by more than 1e-3 voxel must be
    lines with a position within FP32 rounding of a knot; returns their count."""
    b_def, _ = oracle.bstep(og, prm, f32(I1), f32(I2), f32(b), f32(z), f32(u))
    pe = og.pe
    d = np.moveaxis(np.abs(np.asarray(out) - b_def), pe, -1).reshape(-1, b.shape[pe])
    off = np.max(d, axis=1) / og.h[pe] > 1e-3
    near = knot_lines(og, f32(b))
    print(f"{int(off.sum())} of {off.size} lines off the plain oracle by > 1e-3 voxel "
          f"({int(near.sum())} lines with a position at a knot)")
    assert np.all(near[off])
    return int(off.sum())


def case_data(m, pe, seed=0, max_d=0.5):
    h = tuple(1.0 / m[0] for _ in m)
    I1 = ph.random_images(m, seed + 1)
    I2 = ph.random_images(m, seed + 2)
    b = ph.random_field(m, pe, h, seed + 3, max_d=max_d)
    rng = np.random.default_rng(seed + 4)
    z = b + 0.05 * h[pe] * rng.normal(size=b.shape)
    u = 0.05 * h[pe] * rng.normal(size=b.shape)
    return h, I1, I2, b, z, u


@pytest.mark.parametrize("m,pe", CASES)
def test_objective_and_gradient_f64(sac, m, pe):
    h, I1, I2, b, _, _ = case_data(m, pe)
    og = oracle.Grid(m, h, pe)
    op = oracle.Params(alpha=0.7, beta=0.4)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=0.7, beta=0.4, prec="f64")
    ws = sac.workspace(g, p)
    o_ref = oracle.objective(og, op, I1, I2, b)
    o = sac.objective(g, p, cu(I1), cu(I2), cu(b), ws=ws)
    for k in ("J", "D", "S", "P"):
        assert o[k] == pytest.approx(o_ref[k], rel=1e-12, abs=1e-300), k
    gr = sac.gradient(g, p, cu(I1), cu(I2), cu(b), ws=ws).cpu().numpy()
    assert rel(gr, oracle.gradient(og, op, I1, I2, b)) < 1e-11


def test_objective_infinite_penalty_when_infeasible(sac):
    m, pe = (10, 12), 1
    h, I1, I2, b, _, _ = case_data(m, pe)
    b[3, 5] += 2.0 * h[1]
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=1.0, beta=1.0, prec="f64")
    o = sac.objective(g, p, cu(I1), cu(I2), cu(b))
    assert np.isinf(o["P"]) and np.isinf(o["J"])


@pytest.mark.parametrize("m,pe", CASES)
def test_bstep_f64(sac, m, pe):
    h, I1, I2, b, z, u = case_data(m, pe, seed=10)
    og = oracle.Grid(m, h, pe)
    op = oracle.Params(alpha=0.5, rho=100.0)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=0.5, rho=100.0, prec="f64")
    b_ref, st = oracle.bstep(og, op, I1, I2, b, z, u)
    out, capped = sac.bstep(g, p, cu(I1), cu(I2), cu(b), cu(z), cu(u))
    assert not capped and st["capped"] == 0
    assert rel(out.cpu().numpy(), b_ref) < 1e-10


@pytest.mark.parametrize("m,pe", [((37, 50), 1), ((9, 70, 21), 1), ((6, 7, 100), 2), ((5, 256, 11), 1)])
def test_bstep_f64_with_active_constraints(sac, m, pe):
    # steep targets z and small alpha push many cells onto |D1 b| = 1
    h, I1, I2, b, _, u = case_data(m, pe, seed=20, max_d=0.8)
    rng = np.random.default_rng(5)
    z = b + 3.0 * h[pe] * rng.normal(size=b.shape)
    og = oracle.Grid(m, h, pe)
    op = oracle.Params(alpha=1e-3, rho=1e5, n_sqp=2)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=1e-3, rho=1e5, n_sqp=2, prec="f64")
    b_ref, st = oracle.bstep(og, op, I1, I2, b, z, u)
    assert st["active"] > 0 and st["capped"] == 0
    out, capped = sac.bstep(g, p, cu(I1), cu(I2), cu(b), cu(z), cu(u))
    assert not capped
    assert rel(out.cpu().numpy(), b_ref) < 1e-9
    assert oracle.max_abs_d1(og, out.cpu().numpy()) <= 1 + 1e-9


@pytest.mark.parametrize("m,pe", CASES)
def test_zstep_f64(sac, m, pe):
    h, _, _, b, z, u = case_data(m, pe, seed=30)
    og = oracle.Grid(m, h, pe)
    op = oracle.Params(alpha=2.0, rho=50.0)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=2.0, rho=50.0, prec="f64")
    z_ref = oracle.zstep(og, op, b, u)
    u_ref = u + b - z_ref
    zt = cu(z)
    u_out, nr = sac.zstep(g, p, cu(b), cu(u), zt)
    assert rel(zt.cpu().numpy(), z_ref) < 1e-12
    assert rel(u_out.cpu().numpy(), u_ref) < 1e-11
    ref = [np.sum((b - z_ref) ** 2), np.sum((z_ref - z) ** 2), np.sum(b ** 2), np.sum(z_ref ** 2), np.sum(u_ref ** 2)]
    np.testing.assert_allclose(nr, ref, rtol=1e-10)


@pytest.mark.parametrize("m,pe,K", [((24, 40), 1, 20), ((8, 48, 13), 1, 12), ((12, 9, 50), 2, 10)])
def test_admm_f64_fixed_iterations(sac, m, pe, K):
    w = ph.small_workload(m, pe, seed=3, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    og = oracle.Grid(m, d["h"], pe)
    op = oracle.Params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0)
    ref = oracle.admm(og, op, d["I1"], d["I2"], np.zeros(og.face_shape), want_hist=True)
    g = sac.grid(m, d["h"], pe)
    p = sac.params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec="f64")
    b = cu(np.zeros(og.face_shape))
    z = cu(np.zeros(og.face_shape))
    u = cu(np.zeros(og.face_shape))
    res = sac.admm_solve(g, p, cu(d["I1"]), cu(d["I2"]), b, z, u, want_hist=True)
    assert res["iters"] == K
    bb = b.cpu().numpy()
    assert np.linalg.norm(bb - ref["b"]) <= 1e-9 * np.linalg.norm(ref["b"])
    assert rel(bb, ref["b"]) < 1e-9
    assert rel(z.cpu().numpy(), ref["z"]) < 1e-9
    np.testing.assert_allclose(res["hist"][:, :4], ref["hist"][:, :4], rtol=1e-7)


def test_admm_rejects_infeasible_start(sac):
    m, pe = (10, 12), 1
    h, I1, I2, b, _, _ = case_data(m, pe)
    b[2, 4] += 3.0 * h[1]
    g = sac.grid(m, h, pe)
    p = sac.params(prec="f64")
    with pytest.raises(sac.SacError) as e:
        sac.admm_solve(g, p, cu(I1), cu(I2), cu(b))
    assert e.value.status == sac.SAC_EINFEASIBLE


# one PE difference just above / below the bound, placed in the first, a
# middle and the last (partial) chunk of cells of the feasibility check (chunks
# of 2048 cells of one outer index: 9 x 300 x 40 cells, 6 chunks per index)
@pytest.mark.parametrize("where", [(0, 0, 0), (4, 150, 17), (8, 299, 39)])
def test_admm_feasibility_check_at_every_chunk(sac, where):
    m, pe = (9, 300, 40), 1
    h = (1.0 / 9, 1.0 / 300, 1.0 / 40)
    rng = np.random.default_rng(5)
    I1 = rng.normal(size=m)
    I2 = rng.normal(size=m)
    o, i, n = where
    for excess, infeasible in ((1e-6, True), (-1e-6, False)):
        b = np.zeros((9, 301, 40))
        b[o, i + 1:, n] = (1.0 + excess) * h[1]    # one difference (cell (o, i, n)) of (1 + excess) h
        g = sac.grid(m, h, pe)
        p = sac.params(prec="f64", max_iter=1)
        if infeasible:
            with pytest.raises(sac.SacError) as e:
                sac.admm_solve(g, p, cu(I1), cu(I2), cu(b))
            assert e.value.status == sac.SAC_EINFEASIBLE
        else:
            sac.admm_solve(g, p, cu(I1), cu(I2), cu(b))


@pytest.mark.parametrize("m,pe", [((37, 50), 1), ((9, 70, 21), 1), ((40, 7, 9), 0), ((5, 256, 11), 1)])
def test_hessvec_and_preconditioners_f64(sac, m, pe):
    h, I1, I2, b, _, _ = case_data(m, pe, seed=40)
    v = np.random.default_rng(1).normal(size=b.shape)
    og = oracle.Grid(m, h, pe)
    g = sac.grid(m, h, pe)
    for prec in (0, 1, 2):
        op = oracle.Params(alpha=0.8, beta=0.5, precond=prec)
        p = sac.params(alpha=0.8, beta=0.5, precond=prec, prec="f64")
        if prec == 2:
            Hv = sac.hessvec(g, p, cu(I1), cu(I2), cu(b), cu(v)).cpu().numpy()
            assert rel(Hv, oracle.apply(og, op, "HJGN", I1, I2, b, v)) < 1e-11
        x = sac.precond_solve(g, p, cu(I1), cu(I2), cu(b), cu(v)).cpu().numpy()
        assert rel(x, oracle.precond_solve(og, op, I1, I2, b, v)) < 1e-10


@pytest.mark.parametrize("m,pe", [((24, 40), 1), ((8, 48, 13), 1)])
def test_gnpcg_f64(sac, m, pe):
    w = ph.small_workload(m, pe, seed=4, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    og = oracle.Grid(m, d["h"], pe)
    op = oracle.Params(alpha=1.0, beta=10.0, max_gn=6, eta=0.1)
    ref = oracle.gnpcg(og, op, d["I1"], d["I2"], np.zeros(og.face_shape), want_hist=True)
    g = sac.grid(m, d["h"], pe)
    p = sac.params(alpha=1.0, beta=10.0, max_gn=6, eta=0.1, prec="f64")
    b = cu(np.zeros(og.face_shape))
    res = sac.gnpcg_solve(g, p, cu(d["I1"]), cu(d["I2"]), b, want_hist=True)
    assert res["iters"] == ref["iters"]
    np.testing.assert_array_equal(res["hist"][:, 2], ref["hist"][:, 2])     # PCG iterations
    assert rel(b.cpu().numpy(), ref["b"]) < 1e-8
    assert res["J"] == pytest.approx(ref["J"], rel=1e-10)


def test_gnpcg_jacobi_against_block_jacobi(sac):
    # Sec. 6, preconditioner comparison: the same GN-PCG with the Jacobi and
    # the block-Jacobi preconditioner; each matches the oracle's PCG counts,
    # and block-Jacobi needs fewer PCG iterations in total
    m, pe = (32, 32), 1
    w = ph.small_workload(m, pe, seed=5, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    og = oracle.Grid(m, d["h"], pe)
    g = sac.grid(m, d["h"], pe)
    total = {}
    for pc in (1, 2):
        op = oracle.Params(alpha=200.0, beta=10.0, max_gn=4, eta=0.01, max_pcg=200, precond=pc)
        ref = oracle.gnpcg(og, op, d["I1"], d["I2"], np.zeros(og.face_shape), want_hist=True)
        p = sac.params(alpha=200.0, beta=10.0, max_gn=4, eta=0.01, max_pcg=200, precond=pc, prec="f64")
        b = cu(np.zeros(og.face_shape))
        res = sac.gnpcg_solve(g, p, cu(d["I1"]), cu(d["I2"]), b, want_hist=True)
        assert res["iters"] == ref["iters"]
        np.testing.assert_array_equal(res["hist"][:, 2], ref["hist"][:, 2])
        total[pc] = int(res["hist"][:, 2].sum())
    assert total[2] < total[1]


@pytest.mark.parametrize("m,pe,K", [((24, 40), 1, 20), ((8, 48, 13), 1, 12)])
def test_admm_mixed_precision_within_stated_tolerance(sac, m, pe, K):
    w = ph.small_workload(m, pe, seed=3, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    og = oracle.Grid(m, d["h"], pe)
    op = oracle.Params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0)
    ref = oracle.admm(og, op, d["I1"], d["I2"], np.zeros(og.face_shape))
    g = sac.grid(m, d["h"], pe)
    p = sac.params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec="mixed")
    b = cu(np.zeros(og.face_shape))
    res = sac.admm_solve(g, p, cu(d["I1"], torch.float32), cu(d["I2"], torch.float32), b)
    assert res["iters"] == K
    bb = b.cpu().numpy()
    assert np.max(np.abs(bb - ref["b"])) / d["h"][pe] <= 1e-3
    J_ref = oracle.objective(og, op, d["I1"], d["I2"], ref["b"])["J"]
    J_mix = oracle.objective(og, op, d["I1"], d["I2"], bb)["J"]
    assert abs(J_mix - J_ref) <= 1e-6 * abs(J_ref)


# ---------------------------------------------------------------- adaptive augmentation parameter

@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_admm_adaptive_rho(sac, mode, prec):
    # rho from 1e6 (the paper's start) with the adaptive rule, optionally
    # bounded below; the same rho sequence and the same iterate as the oracle
    m, pe, K = (8, 48, 13), 1, 12
    w = ph.small_workload(m, pe, seed=3, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    og = oracle.Grid(m, d["h"], pe)
    kw = dict(alpha=1.0, rho=1e6, max_iter=K, eps_abs=0.0, eps_rel=0.0, adapt_rho=mode, rho_min=2e4)
    ref = oracle.admm(og, oracle.Params(**kw), d["I1"], d["I2"], np.zeros(og.face_shape), want_hist=True)
    assert len(set(ref["hist"][:, 4])) > 3          # rho changes several times
    g = sac.grid(m, d["h"], pe)
    p = sac.params(prec=prec, **kw)
    dt = torch.float64 if prec == "f64" else torch.float32
    b = cu(np.zeros(og.face_shape))
    res = sac.admm_solve(g, p, cu(d["I1"], dt), cu(d["I2"], dt), b, want_hist=True)
    assert res["iters"] == K
    np.testing.assert_allclose(res["hist"][:, 4], ref["hist"][:, 4], rtol=1e-12)
    bb = b.cpu().numpy()
    if prec == "f64":
        assert np.linalg.norm(bb - ref["b"]) <= 1e-9 * np.linalg.norm(ref["b"])
    else:
        assert np.max(np.abs(bb - ref["b"])) / d["h"][pe] <= 1e-3


# ---------------------------------------------------------------- multilevel strategy (Sec. 4.4)

@pytest.mark.parametrize("m,pe", [((8, 12), 1), ((6, 10, 8), 1), ((4, 6, 10), 2), ((10, 4, 6), 0)])
def test_restriction_and_prolongation(sac, m, pe):
    rng = np.random.default_rng(11)
    I = rng.uniform(size=m)
    g = sac.grid(m, tuple(0.1 for _ in m), pe)
    for prec, dt, tol in (("f64", torch.float64, 1e-15), ("mixed", torch.float32, 1e-6)):
        Ic = sac.restrict_image(g, sac.params(prec=prec), cu(I, dt)).double().cpu().numpy()
        assert rel(Ic, oracle.restrict(m, I)) < tol
    mc = tuple(x // 2 for x in m)
    bc = rng.normal(size=tuple(x + (1 if a == pe else 0) for a, x in enumerate(mc)))
    bf = sac.prolong_field(g, cu(bc)).cpu().numpy()
    assert rel(bf, oracle.prolong(m, pe, bc)) < 1e-15


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_multilevel_solve(sac, prec):
    # three levels (8x12x6 -> 16x24x12 -> 32x48x24), a fixed number of
    # iterations per level, adaptive rho with a lower bound carried across
    m, pe, K = (32, 48, 24), 1, 8
    w = ph.small_workload(m, pe, seed=12, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    kw = dict(alpha=1.0, rho=1e5, max_iter=K, eps_abs=0.0, eps_rel=0.0, adapt_rho=2, rho_min=1e3)
    ref = oracle.multilevel_admm(m, d["h"], pe, oracle.Params(**kw), d["I1"], d["I2"], levels=3)
    g = sac.grid(m, d["h"], pe)
    p = sac.params(prec=prec, **kw)
    dt = torch.float64 if prec == "f64" else torch.float32
    b = cu(np.zeros(sac.face_shape(g)))
    res = sac.multilevel_solve(g, 3, p, cu(d["I1"], dt), cu(d["I2"], dt), b)
    assert res["iters"] == [K, K, K]
    assert res["rho"] == pytest.approx(ref[-1]["rho"], rel=1e-12)
    bb = b.cpu().numpy()
    if prec == "f64":
        assert np.linalg.norm(bb - ref[-1]["b"]) <= 1e-9 * np.linalg.norm(ref[-1]["b"])
    else:
        assert np.max(np.abs(bb - ref[-1]["b"])) / d["h"][pe] <= 1e-3


# ---------------------------------------------------------------- corrected images, SSD, NCC (Sec. 6)

@pytest.mark.parametrize("m,pe", CASES)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_corrected_images(sac, m, pe, prec):
    h, I1, I2, b, _, _ = case_data(m, pe, seed=50, max_d=0.7)
    ref = oracle.corrected(oracle.Grid(m, h, pe), I1, I2, b)
    g = sac.grid(m, h, pe)
    p = sac.params(prec=prec)
    dt = torch.float64 if prec == "f64" else torch.float32
    out = sac.corrected_images(g, p, cu(I1, dt), cu(I2, dt), cu(b))
    T1, T2 = out["T1"].double().cpu().numpy(), out["T2"].double().cpu().numpy()
    if prec == "f64":
        assert rel(T1, ref["T1"]) < 1e-12 and rel(T2, ref["T2"]) < 1e-12
        assert out["ssd"] == pytest.approx(ref["ssd"], rel=1e-10)
        assert out["ncc"] == pytest.approx(ref["ncc"], rel=1e-12)
    else:
        # FP32 images and arithmetic: a few ulp of the image scale per cell
        assert rel(T1, ref["T1"]) < 2e-5 and rel(T2, ref["T2"]) < 2e-5
        assert out["ssd"] == pytest.approx(ref["ssd"], rel=1e-3)
        assert out["ncc"] == pytest.approx(ref["ncc"], rel=1e-5)


def test_corrected_images_measures_only(sac):
    # T1 / T2 may be left out; the measures are the same
    m, pe = (9, 70, 21), 1
    h, I1, I2, b, _, _ = case_data(m, pe, seed=51)
    g = sac.grid(m, h, pe)
    p = sac.params(prec="f64")
    full = sac.corrected_images(g, p, cu(I1), cu(I2), cu(b))
    out = (ctypes.c_double(0), ctypes.c_double(0))
    ws = sac.workspace(g, p)
    dI1, dI2, db = cu(I1), cu(I2), cu(b)
    st = sac.lib().sac_corrected_images(ctypes.byref(g), ctypes.byref(p), dI1.data_ptr(), dI2.data_ptr(),
                                        db.data_ptr(), None, None, ctypes.byref(out[0]), ctypes.byref(out[1]),
                                        ws.data_ptr(), ws.numel(), None)
    torch.cuda.synchronize()
    assert st == 0
    assert out[0].value == full["ssd"] and out[1].value == full["ncc"]


# ---------------------------------------------------------------- b-step segment kernel (mixed path)

# strided PE lines: 9 faces per segment up to 144 faces, 17 up to 272; line
# counts with ragged 32-line tiles, segment counts from 5 to 16, the last
# segment partly past the line end
SEG_CASES = [
    ((9, 70, 21), 1),       # 71 faces: 8 segments of 9, 189 lines (5 full tiles + 29)
    ((40, 7, 9), 0),        # PE first: 41 faces, 63 lines in one outer slab
    ((3, 143, 40), 1),      # 144 faces: exactly 16 segments of 9
    ((4, 145, 10), 1),      # 146 faces: 9 segments of 17
    ((5, 256, 11), 1),      # 257 faces: 16 segments of 17, 55 lines
    ((2, 271, 17), 1),      # 272 faces: exactly 16 segments of 17
    # lines a multiple of 16 apart (aligned rows): tiles staged by TMA tensor copies
    ((9, 70, 32), 1),       # 71 faces, 18 tiles
    ((24, 143, 256), 1),    # 144 faces, 384 tiles: more tiles than resident CTAs (next tile prefetched)
    ((20, 256, 256), 1),    # 257 faces, 320 tiles: the same with segments of 17
    # inner extents a multiple of 4 but not of 16: TMA-staged tiles within one
    # outer index, the index's last tile partial (its lines past the extent
    # read as zeros and are not stored)
    ((9, 70, 20), 1),       # 71 faces, 2 tiles per outer index (16 + 4 lines)
    ((6, 96, 60), 1),       # 97 faces, 4 tiles per outer index (16, 16, 16, 12): the 96 x 96 x 60 lines
    ((3, 143, 44), 1),      # 144 faces, 16 segments of 9, tiles of 16, 16, 12 lines
    ((4, 256, 36), 1),      # 257 faces, segments of 17, tiles of 16, 16, 4 lines
]


@pytest.mark.parametrize("m,pe", SEG_CASES)
def test_bstep_mixed_segment_kernel(sac, m, pe):
    # the mixed b-step (one thread per line segment) against the FP64 oracle
    # (1e-3 voxel) and against the warp-per-line FP32 kernel
    h, I1, I2, b, z, u = case_data(m, pe, seed=30)
    og = oracle.Grid(m, h, pe)
    # the model's interval at a displaced position is an integer decided in
    # floating point: the oracle takes it in FP32 as the kernels do, on the
    # FP32-rounded inputs they see (knot32); the rest of it runs in FP64
    b_ref, st = oracle.bstep(og, oracle.Params(alpha=0.5, rho=100.0, knot32=1), f32(I1), f32(I2), f32(b), f32(z),
                             f32(u))
    g = sac.grid(m, h, pe)
    outs = []
    for kern in (0, 1):
        p = sac.params(alpha=0.5, rho=100.0, prec="mixed", bstep_kernel=kern)
        out, capped = sac.bstep(g, p, cu(I1, torch.float32), cu(I2, torch.float32), cu(b), cu(z), cu(u))
        assert not capped
        outs.append(out.cpu().numpy())
        assert np.max(np.abs(outs[-1] - b_ref)) / h[pe] <= 1e-3
        lines_off_the_plain_oracle(og, oracle.Params(alpha=0.5, rho=100.0), I1, I2, b, z, u, outs[-1])
    assert np.max(np.abs(outs[0] - outs[1])) / h[pe] <= 1e-4


@pytest.mark.parametrize("m,pe", [((9, 70, 21), 1), ((5, 256, 11), 1), ((9, 70, 32), 1), ((3, 256, 32), 1),
                                  ((6, 96, 60), 1)])
def test_bstep_mixed_segment_kernel_queues_blocked_lines(sac, m, pe):
    # (the last two: TMA-staged tiles, queued lines restored in the tile's
    # shared-memory buffer before its tensor store)
    # steep targets: many lines' unconstrained steps cross |D1 b| = 1; the
    # segment kernel leaves them to the FP64 active-set method
    h, I1, I2, b, _, u = case_data(m, pe, seed=40, max_d=0.8)
    rng = np.random.default_rng(6)
    z = b + 3.0 * h[pe] * rng.normal(size=b.shape)
    og = oracle.Grid(m, h, pe)
    b_ref, st = oracle.bstep(og, oracle.Params(alpha=1e-3, rho=1e5, knot32=1), f32(I1), f32(I2), f32(b), f32(z),
                             f32(u))
    assert st["active"] > 0 and st["capped"] == 0
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=1e-3, rho=1e5, prec="mixed", bstep_kernel=0)
    out, capped = sac.bstep(g, p, cu(I1, torch.float32), cu(I2, torch.float32), cu(b), cu(z), cu(u))
    assert not capped
    out = out.cpu().numpy()
    assert np.max(np.abs(out - b_ref)) / h[pe] <= 1e-3
    assert oracle.max_abs_d1(og, out) <= 1 + 1e-5
    lines_off_the_plain_oracle(og, oracle.Params(alpha=1e-3, rho=1e5), I1, I2, b, z, u, out)


# ---------------------------------------------------------------- tensor-core z-step (mixed path)

TC_CASES = [
    ((37, 50), 1),          # 2D: contracted axis 0 has post > 1 (case A)
    ((50, 37), 0),          # 2D, PE first: contracted axis 1 is the last one (case B)
    ((9, 70, 21), 1),       # 3D PE middle: axis 0 case A, axis 2 case B
    ((40, 7, 9), 0),        # PE first: axis 1 case A (post = 9), axis 2 case B
    ((6, 7, 100), 2),       # PE last: axis 0 case A, axis 1 case A (post = 101)
    ((200, 20, 33), 1),     # two 128-row blocks (L = 200) and N = 48 (case B)
    ((300, 9, 5), 1),       # L = 300 > 256: falls back to the SIMT passes
    ((64, 30, 48), 1),      # 16-byte vector paths: post = 1488, last axis 48
    ((160, 11, 20), 1),     # two 128-row blocks with vector stores (post = 240)
    ((80, 255, 24), 1),     # more tiles than SMs on the last axis (20480 lines)
    ((6, 10, 200), 1),      # contiguous axis of 200 faces: one tile as two column halves
    ((136, 150, 130), 1),   # 154 and 161 tiles: full tiles, then the last round as column halves
    # on-chip z-step (one PE slab per CTA at a time; zstep_kernel 3 below)
    ((256, 9, 80), 1),      # full slab width: 256 x 80 (N = 256, K = 80)
    ((30, 16, 128), 0),     # PE first, 128 faces along the last axis
    ((40, 300, 12), 1),     # 301 slabs: several per CTA; K padded from 12 to 16
    ((200, 3, 37), 1),      # last axis of 37 faces: element-wise loads and stores
    ((17, 5, 6), 0),        # both slab axes padded (17 -> 32, 6 -> 16)
    ((2, 5, 3), 1),         # the smallest slabs: 2 x 3 faces
    ((3, 2, 2), 0),         # 2 x 2 faces, PE first
    ((128, 3, 128), 1),     # 128 x 128 slabs: the widest last axis
]


# Split TF32 (hi*hi + hi*lo + lo*hi, FP32 accumulation): each product carries
# a relative error of about 3 * 2^-22 (truncated lo terms and the dropped lo*lo);
# over a length-L DCT and 4 passes this stays below 1e-5 of the largest output
# for L <= 256, far inside the mixed path's 1e-3-voxel budget.
TC_TOL = 1e-5


@pytest.mark.parametrize("m,pe", TC_CASES)
def test_zstep_mixed_tensor_cores(sac, m, pe):
    h, _, _, b, z, u = case_data(m, pe, seed=50)
    og = oracle.Grid(m, h, pe)
    op = oracle.Params(alpha=2.0, rho=50.0)
    g = sac.grid(m, h, pe)
    z_ref = oracle.zstep(og, op, b, u)
    # FP32 storage: compare against the oracle run on the FP32-rounded inputs
    b32 = b.astype(np.float32).astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    z_ref32 = oracle.zstep(og, op, b32, u32)
    outs = {}
    for kern in (0, 1, 2, 3):
        p = sac.params(alpha=2.0, rho=50.0, prec="mixed", zstep_kernel=kern)
        zt = cu(z)
        u_out, nr = sac.zstep(g, p, cu(b), cu(u), zt)
        outs[kern] = zt.cpu().numpy()
        assert rel(outs[kern], z_ref32) < TC_TOL, (kern, rel(outs[kern], z_ref32))
        assert rel(u_out.cpu().numpy(), u32 + b32 - z_ref32) < 2e-5
        ref = [np.sum((b32 - z_ref32) ** 2), np.sum((z_ref32 - z) ** 2), np.sum(b32 ** 2)]
        np.testing.assert_allclose(nr[:3], ref, rtol=1e-4)
    assert rel(outs[0], outs[1]) < TC_TOL
    assert rel(outs[2], outs[1]) < TC_TOL
    assert rel(outs[3], outs[1]) < TC_TOL
    assert rel(outs[0], z_ref) < 2 * TC_TOL


@pytest.mark.parametrize("scale", [1e-12, 1e-3, 1e6, 1e18])
def test_onchip_zstep_scaling_across_magnitudes(sac, scale):
    # the on-chip z-step scales its split-FP16 operands by powers of two from
    # each row's and the slab's maximum: the same relative accuracy for inputs
    # far from unit size, and for a slab whose rows differ by 1e8 in magnitude
    m, pe = (64, 5, 48), 1
    h, _, _, b, z, u = case_data(m, pe, seed=60)
    b = b * scale
    u = u * scale
    b[:, 2, :] *= 1e-8            # one slab much smaller than the others
    b[5, :, :] *= 1e4             # one row of every slab much larger
    og = oracle.Grid(m, h, pe)
    b32 = b.astype(np.float32).astype(np.float64)
    u32 = u.astype(np.float32).astype(np.float64)
    z_ref32 = oracle.zstep(og, oracle.Params(alpha=2.0, rho=50.0), b32, u32)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=2.0, rho=50.0, prec="mixed", zstep_kernel=3)
    assert sac.zstep_fused(g, p) == 2
    zt = cu(z)
    sac.zstep(g, p, cu(b), cu(u), zt)
    out = zt.cpu().numpy()
    assert rel(out, z_ref32) < TC_TOL, rel(out, z_ref32)
    # the small slab relative to its own size
    assert rel(out[:, 2, :], z_ref32[:, 2, :]) < TC_TOL, rel(out[:, 2, :], z_ref32[:, 2, :])


# ---------------------------------------------------------------- the benchmark's volume

def test_full_size_bstep_matches_the_oracle(sac):
    # the 256 x 256 x 80 volume of the benchmark (5.26M faces) with its
    # parameters and b-step kernel: the persistent TMA-staged segment kernel
    # over 1280 tiles of 16 lines (synthetic images of that size; the oracle
    # takes the model's interval decisions in FP32 on the FP32-rounded inputs,
    # as for the smaller cases)
    m, pe = (256, 256, 80), 1
    h = tuple(1.0 / x for x in m)
    I1, I2 = ph.random_images(m, 1), ph.random_images(m, 2)
    b = f32(ph.random_field(m, pe, h, 3, max_d=0.5))
    rng = np.random.default_rng(4)
    z = f32(b + 0.05 * h[pe] * rng.normal(size=b.shape))
    u = f32(0.05 * h[pe] * rng.normal(size=b.shape))
    og = oracle.Grid(m, h, pe)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=50.0, rho=100.0, prec="mixed", near_bound=1e-3)
    out, capped = sac.bstep(g, p, cu(I1, torch.float32), cu(I2, torch.float32), cu(b), cu(z), cu(u))
    assert not capped
    b_ref, _ = oracle.bstep(og, oracle.Params(alpha=50.0, rho=100.0, knot32=1), f32(I1), f32(I2), b, z, u)
    out = out.cpu().numpy()
    err = np.max(np.abs(out - b_ref)) / h[pe]
    print(f"full-size mixed b-step: max |db| = {err:.3e} voxel")
    assert err <= 1e-3
    lines_off_the_plain_oracle(og, oracle.Params(alpha=50.0, rho=100.0), I1, I2, b, z, u, out)


@pytest.fixture(scope="module")
def full_size():
    """The benchmarked solve's inputs: the 256 x 256 x 80 phantom pair (5.26M
    faces, FP32 images), alpha 50, rho 1e2, and the oracle's K = 20 ADMM
    iterates from b = 0 with the model's intervals decided in FP64 (plain)
    and in FP32 (knot32), on the FP32 images the GPU reads."""
    w, d = ph.load_pair("3d_256x256x80", np.float32)
    og = oracle.Grid(w.m, w.h, w.pe)
    I1, I2 = d["I1"].astype(np.float64), d["I2"].astype(np.float64)
    K = 20
    ref = {}
    for k32 in (0, 1):
        op = oracle.Params(alpha=w.alpha, rho=w.rho, max_iter=K, eps_abs=0.0, eps_rel=0.0, knot32=k32)
        ref[k32] = oracle.admm(og, op, I1, I2, np.zeros(og.face_shape))["b"]
    return dict(w=w, d=d, og=og, I1=I1, I2=I2, K=K, ref=ref)


def _objective(F, b):
    return oracle.objective(F["og"], oracle.Params(alpha=F["w"].alpha), F["I1"], F["I2"], b)["J"]


def _solve(sac, F, prec, K, eps_rel=0.0):
    w = F["w"]
    g = sac.grid(w.m, w.h, w.pe)
    p = sac.params(alpha=w.alpha, rho=w.rho, max_iter=K, eps_abs=0.0, eps_rel=eps_rel, prec=prec, near_bound=1e-3)
    dt = torch.float32 if prec == "mixed" else torch.float64
    b = cu(np.zeros(F["og"].face_shape))
    res = sac.admm_solve(g, p, cu(F["d"]["I1"], dt), cu(F["d"]["I2"], dt), b)
    return res, b.cpu().numpy()


def test_full_size_admm_mixed_matches_the_oracle(sac, full_size):
    # K = 20 mixed ADMM iterations through sac_admm_solve against the FP64
    # oracle that takes the model's interval decisions in FP32 (knot32) as
    # the kernels do: 1e-3 voxel in b.  The objective of this transient
    # iterate (it changes by tens of percent from one iteration to the next)
    # is fixed by the method only to the spread between the oracle's two
    # interval rules (FP64 and FP32 positions): a displaced position within
    # rounding of a knot of the piecewise-linear model changes that line's
    # step, and each trajectory carries its own flips (the GPU's b differs
    # from the oracle's by rounding, so they flip at different cells).  The
    # mixed objective must stay within four times that spread of both
    # oracles; the 1e-6 bar is met at convergence (next tests).  Against the plain oracle the field is
    # printed beside the oracle's own spread.
    F = full_size
    h = F["w"].h[F["w"].pe]
    res, bb = _solve(sac, F, "mixed", F["K"])
    assert res["iters"] == F["K"]
    J32, J64, Jm = _objective(F, F["ref"][1]), _objective(F, F["ref"][0]), _objective(F, bb)
    err = np.max(np.abs(bb - F["ref"][1])) / h
    err64 = np.max(np.abs(bb - F["ref"][0])) / h
    own = np.max(np.abs(F["ref"][1] - F["ref"][0])) / h
    print(f"full-size mixed ADMM, K = {F['K']}: against the oracle with FP32 interval decisions "
          f"max |db| = {err:.3e} voxel, relative objective {abs(Jm - J32) / abs(J32):.3e}; against the plain "
          f"oracle {err64:.3e} voxel, {abs(Jm - J64) / abs(J64):.3e}; the oracle's two interval rules differ "
          f"by {own:.3e} voxel, {abs(J32 - J64) / abs(J64):.3e}")
    assert err <= 1e-3
    spread = abs(J32 - J64)
    assert abs(Jm - J32) <= 4.0 * spread and abs(Jm - J64) <= 4.0 * spread


def test_full_size_admm_f64_matches_the_plain_oracle(sac, full_size):
    # the plain FP64 GPU path (the comparison path of the benchmark) on the
    # same volume: 1e-9 relative in b against the plain oracle after K = 20
    F = full_size
    res, bb = _solve(sac, F, "f64", F["K"])
    assert res["iters"] == F["K"]
    ref = F["ref"][0]
    assert np.linalg.norm(bb - ref) <= 1e-9 * np.linalg.norm(ref)
    assert rel(bb, ref) < 1e-9


def test_full_size_converged_mixed_matches_converged_f64(sac, full_size):
    # both precisions run to the benchmark's stopping test (relative residual
    # 1e-4, eps_abs = 0, at most 2000 iterations); the converged mixed result
    # against the converged plain FP64 result (which decides the model's
    # intervals in FP64 as the oracle does, and matches it above): 1e-3 voxel
    # in b, 1e-6 relative objective (objectives from the oracle)
    F = full_size
    h = F["w"].h[F["w"].pe]
    rm, bm = _solve(sac, F, "mixed", 2000, eps_rel=1e-4)
    rf, bf = _solve(sac, F, "f64", 2000, eps_rel=1e-4)
    Jm, Jf = _objective(F, bm), _objective(F, bf)
    err = np.max(np.abs(bm - bf)) / h
    print(f"converged at relative residual 1e-4: mixed {rm['iters']} iterations, FP64 {rf['iters']}; "
          f"max |db| = {err:.3e} voxel, relative objective {abs(Jm - Jf) / abs(Jf):.3e}")
    assert rm["iters"] < 2000 and rf["iters"] < 2000
    assert err <= 1e-3
    assert abs(Jm - Jf) <= 1e-6 * abs(Jf)


# ---------------------------------------------------------------- FP64 parity on the configurations' grids

@pytest.mark.parametrize("name,K", [("2d_128", 50), ("3d_128x128x64", 20)])
def test_admm_f64_on_the_configurations(sac, name, K):
    # the 128 x 128 slice (alpha 50, K = 50) and the 128 x 128 x 64 volume
    # (alpha 100, K = 20), plain FP64 ADMM from b = 0: 1e-9 relative in b
    w, d = ph.load_pair(name, np.float64)
    og = oracle.Grid(w.m, w.h, w.pe)
    op = oracle.Params(alpha=w.alpha, rho=w.rho, max_iter=K, eps_abs=0.0, eps_rel=0.0)
    ref = oracle.admm(og, op, d["I1"], d["I2"], np.zeros(og.face_shape), want_hist=True)
    g = sac.grid(w.m, w.h, w.pe)
    p = sac.params(alpha=w.alpha, rho=w.rho, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec="f64")
    b = cu(np.zeros(og.face_shape))
    res = sac.admm_solve(g, p, cu(d["I1"]), cu(d["I2"]), b, want_hist=True)
    assert res["iters"] == K
    bb = b.cpu().numpy()
    assert np.linalg.norm(bb - ref["b"]) <= 1e-9 * np.linalg.norm(ref["b"])
    assert rel(bb, ref["b"]) < 1e-9
    np.testing.assert_allclose(res["hist"][:, :4], ref["hist"][:, :4], rtol=1e-7)
