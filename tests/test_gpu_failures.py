"""Failure detection through the C ABI, in forms that fault or hang no GPU:
non-finite inputs made on the host, and a bounded device wait made to give
up by setting its limit to zero (the kernel drains its copies in flight and
reports SAC_ETIMEOUT; the context stays usable)."""
import numpy as np
import pytest

from paper_1607_00531_gb300 import phantoms as ph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sac():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00531_gb300 import build, sac as S
    build.build()
    return S


def cu(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def pair_with_nan(m, pe, seed):
    w = ph.small_workload(m, pe, seed=seed, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    I1 = d["I1"].copy()
    I1[tuple(x // 2 for x in m)] = np.nan      # one cell in the middle of the volume
    return d, I1


@pytest.mark.parametrize("prec", ["f64", "mixed"])
@pytest.mark.parametrize("m,pe", [((24, 40), 1), ((9, 70, 32), 1)])
def test_nan_image_gives_enan_from_admm_solve(sac, prec, m, pe):
    d, I1 = pair_with_nan(m, pe, seed=3)
    dt = torch.float64 if prec == "f64" else torch.float32
    g = sac.grid(m, d["h"], pe)
    p = sac.params(alpha=1.0, rho=100.0, max_iter=5, eps_abs=0.0, eps_rel=0.0, prec=prec)
    b = cu(np.zeros(sac.face_shape(g)))
    with pytest.raises(sac.SacError) as e:
        sac.admm_solve(g, p, cu(I1, dt), cu(d["I2"], dt), b)
    assert e.value.status == sac.SAC_ENAN
    # the same call on finite images still works (nothing left behind)
    b.zero_()
    res = sac.admm_solve(g, p, cu(d["I1"], dt), cu(d["I2"], dt), b)
    assert res["iters"] == 5 and torch.isfinite(b).all()


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_nan_image_gives_enan_from_the_batch_engine(sac, prec):
    vols = [pair_with_nan((24, 40), 1, seed=3), pair_with_nan((10, 70, 9), 1, seed=4)]
    dt = torch.float64 if prec == "f64" else torch.float32
    p = sac.params(alpha=1.0, rho=100.0, max_iter=6, eps_abs=0.0, eps_rel=0.0, prec=prec, check_every=6)
    grids = [sac.grid(d["m"], d["h"], d["pe"]) for d, _ in vols]
    I1s = [cu(I1, dt) for _, I1 in vols[:1]] + [cu(vols[1][0]["I1"], dt)]   # NaN in the first volume only
    I2s = [cu(d["I2"], dt) for d, _ in vols]
    bs = [torch.zeros(sac.face_shape(g), dtype=torch.float64, device="cuda") for g in grids]
    bt = sac.Batch(grids, p, I1s, I2s, bs)
    try:
        with pytest.raises(sac.SacError) as e:
            bt.run(6, chunk=6)
        assert e.value.status == sac.SAC_ENAN
    finally:
        bt.close()


def test_bounded_wait_that_gives_up_returns_etimeout(sac):
    # the segment b-step stages each tile with TMA tensor copies completing
    # on an mbarrier (lines a multiple of 16 apart); with the wait limit at
    # zero every wait gives up, the kernel drains the copies in flight and
    # reports the timeout; with the default limit restored the same call runs
    m, pe = (9, 70, 32), 1
    w = ph.small_workload(m, pe, seed=8, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    h = d["h"]
    rng = np.random.default_rng(2)
    b = 0.1 * h[pe] * rng.normal(size=tuple(x + (a == pe) for a, x in enumerate(m)))
    b -= b.mean()
    z = b.copy()
    u = np.zeros_like(b)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=1.0, rho=100.0, prec="mixed")
    args = (cu(d["I1"], torch.float32), cu(d["I2"], torch.float32), cu(b), cu(z), cu(u))
    ref, _ = sac.bstep(g, p, *args)
    try:
        sac.set_wait_limit(sac.WAIT_BSTEP, 0)
        with pytest.raises(sac.SacError) as e:
            sac.bstep(g, p, *args)
        assert e.value.status == sac.SAC_ETIMEOUT
    finally:
        sac.set_wait_limit(sac.WAIT_BSTEP | sac.WAIT_ZSTEP, -1)
    out, _ = sac.bstep(g, p, *args)
    assert torch.equal(out, ref)


def test_onchip_zstep_wait_that_gives_up_returns_etimeout(sac):
    # the on-chip z-step's roles hand slabs to each other through mbarriers
    # (DCT ring, operands in shared and tensor memory, converter syncs); with
    # the wait limit at zero the first wait gives up, the roles leave their
    # loops, the MMAs and copies in flight are drained and the call reports
    # the timeout; with the default limit the same call gives the same z
    m, pe = (40, 9, 24), 1
    rng = np.random.default_rng(3)
    shape = tuple(x + (a == pe) for a, x in enumerate(m))
    h = (1.0 / 40, 1.0 / 9, 1.0 / 24)
    b = 0.01 * rng.normal(size=shape)
    u = 0.001 * rng.normal(size=shape)
    g = sac.grid(m, h, pe)
    p = sac.params(alpha=2.0, rho=50.0, prec="mixed", zstep_kernel=3)
    assert sac.zstep_fused(g, p) == 2
    z_ref = cu(np.zeros(shape))
    sac.zstep(g, p, cu(b), cu(u), z_ref)
    try:
        sac.set_wait_limit(sac.WAIT_ZSTEP, 0)
        with pytest.raises(sac.SacError) as e:
            sac.zstep(g, p, cu(b), cu(u), cu(np.zeros(shape)))
        assert e.value.status == sac.SAC_ETIMEOUT
    finally:
        sac.set_wait_limit(sac.WAIT_BSTEP | sac.WAIT_ZSTEP, -1)
    z = cu(np.zeros(shape))
    sac.zstep(g, p, cu(b), cu(u), z)
    assert torch.equal(z, z_ref)
