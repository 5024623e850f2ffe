"""Batched ADMM (one launch per phase over many volumes): each volume's
result must equal its solo result, for mixed grid sizes in one batch, and
the FP64 batch must match the CPU oracle (Sec. 4.2 per volume)."""
import numpy as np
import pytest

import oracle
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


def volumes():
    # different classes of line length (faces per lane 3, 5, 9), 2D and 3D, PE axes;
    # two volumes of the b-step segment kernel with 16 and 12 segments per line
    specs = [((24, 40), 1, 1), ((10, 70, 9), 1, 2), ((12, 150), 1, 3), ((8, 9, 30), 2, 4),
             ((6, 260, 5), 1, 5), ((30, 33), 1, 6), ((7, 200, 6), 1, 7)]
    out = []
    for m, pe, seed in specs:
        w = ph.small_workload(m, pe, seed=seed, peak_px=2.0, max_d=0.5)
        out.append(ph.make_pair(w))
    return out


def cu(a, dt):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


# zstep_kernel 3: the 3D volumes whose last axis is not the PE axis take the
# on-chip z-step (in the engine with the stopping test fused) whatever their size
@pytest.mark.parametrize("prec,kern", [("mixed", 0), ("mixed", 3), ("f64", 0)])
def test_batch_equals_solo(sac, prec, kern):
    K = 12
    vols = volumes()
    dt = torch.float32 if prec == "mixed" else torch.float64
    p = sac.params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec=prec, check_every=K,
                   zstep_kernel=kern)
    grids = [sac.grid(d["m"], d["h"], d["pe"]) for d in vols]
    I1s = [cu(d["I1"], dt) for d in vols]
    I2s = [cu(d["I2"], dt) for d in vols]
    bs = [torch.zeros(sac.face_shape(g), dtype=torch.float64, device="cuda") for g in grids]
    bt = sac.Batch(grids, p, I1s, I2s, bs)
    bt.run(K + 5, chunk=5)
    st = bt.stats()
    bt.finish()
    bt.close()
    assert np.all(st["iters"] == K)
    for g, I1, I2, bb in zip(grids, I1s, I2s, bs):
        b = torch.zeros_like(bb)
        sac.admm_solve(g, p, I1, I2, b)
        diff = (b - bb).abs().max().item()
        assert diff <= 1e-12 * max(b.abs().max().item(), 1e-30), diff


@pytest.mark.parametrize("prec,kern", [("mixed", 0), ("mixed", 3), ("f64", 0)])
def test_batch_adaptive_rho_equals_solo(sac, prec, kern):
    # the batched engine applies the adaptive rule on the device, in the
    # stopping test of each volume; the single-volume call on the host
    K = 12
    vols = volumes()[:4]
    dt = torch.float32 if prec == "mixed" else torch.float64
    p = sac.params(alpha=1.0, rho=1e6, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec=prec, adapt_rho=2, rho_min=2e4,
                   zstep_kernel=kern)
    grids = [sac.grid(d["m"], d["h"], d["pe"]) for d in vols]
    I1s = [cu(d["I1"], dt) for d in vols]
    I2s = [cu(d["I2"], dt) for d in vols]
    bs = [torch.zeros(sac.face_shape(g), dtype=torch.float64, device="cuda") for g in grids]
    bt = sac.Batch(grids, p, I1s, I2s, bs)
    bt.run(K, chunk=4)
    bt.finish()
    bt.close()
    for g, I1, I2, bb in zip(grids, I1s, I2s, bs):
        b = torch.zeros_like(bb)
        sac.admm_solve(g, p, I1, I2, b)
        diff = (b - bb).abs().max().item()
        assert diff <= 1e-12 * max(b.abs().max().item(), 1e-30), diff


def test_batch_f64_matches_oracle(sac):
    K = 10
    vols = volumes()[:3]
    p = sac.params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec="f64")
    grids = [sac.grid(d["m"], d["h"], d["pe"]) for d in vols]
    bs = [torch.zeros(sac.face_shape(g), dtype=torch.float64, device="cuda") for g in grids]
    bt = sac.Batch(grids, p, [cu(d["I1"], torch.float64) for d in vols], [cu(d["I2"], torch.float64) for d in vols], bs)
    bt.run(K)
    bt.finish()
    for d, bb in zip(vols, bs):
        og = oracle.Grid(d["m"], d["h"], d["pe"])
        ref = oracle.admm(og, oracle.Params(alpha=1.0, rho=100.0, max_iter=K, eps_abs=0.0, eps_rel=0.0),
                          d["I1"], d["I2"], np.zeros(og.face_shape))
        assert np.linalg.norm(bb.cpu().numpy() - ref["b"]) <= 1e-9 * np.linalg.norm(ref["b"])


def test_batch_stops_each_volume_on_its_own_residuals(sac):
    vols = volumes()[:4]
    p = sac.params(alpha=1.0, rho=100.0, max_iter=300, eps_abs=0.0, eps_rel=1e-3, prec="mixed", autotune=1)
    grids = [sac.grid(d["m"], d["h"], d["pe"]) for d in vols]
    bs = [torch.zeros(sac.face_shape(g), dtype=torch.float64, device="cuda") for g in grids]
    bt = sac.Batch(grids, p, [cu(d["I1"], torch.float32) for d in vols], [cu(d["I2"], torch.float32) for d in vols], bs)
    bt.run(300, chunk=10)
    st = bt.stats()
    bt.finish()
    assert np.all((st["converged"]) | (st["iters"] == 300))
    assert len(set(st["iters"].tolist())) > 1        # volumes stop at different iterations
    # a converged volume's final residuals satisfy the stopping rule it was retired by
    for g, bb, it, cv in zip(grids, bs, st["iters"], st["converged"]):
        b = torch.zeros_like(bb)
        q = sac.params(alpha=1.0, rho=100.0, max_iter=int(it), eps_abs=0.0, eps_rel=0.0, prec="mixed")
        d = vols[grids.index(g)]
        sac.admm_solve(g, q, cu(d["I1"], torch.float32), cu(d["I2"], torch.float32), b)
        assert (b - bb).abs().max().item() <= 1e-12 * max(b.abs().max().item(), 1e-30)


# ---------------------------------------------------------------- the 64-pair DTI-like batch

@pytest.fixture(scope="module")
def dti_batch():
    """The 64 pairs of 96 x 96 x 60 (independent seeded fields of 2-6 px, SNR
    10-40) of the batched workload, generated on the GPU."""
    ws = ph.batch_workloads(64)
    pairs = [ph.make_pair(w, dtype=np.float32, device="cuda") for w in ws]
    return ws, pairs


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_dti_batch_of_64_matches_the_oracle_on_sampled_pairs(sac, dti_batch, prec):
    # all 64 pairs in one engine (one launch per phase over all lines and
    # slabs, CUDA-graph replay: the launch configuration the bench times),
    # K = 8 iterations; pairs 0, 37 and 63 against the oracle run alone:
    # FP64 to 1e-9 relative in b; mixed to 1e-3 voxel against the oracle
    # with the FP32 interval decisions of the kernels (knot32)
    ws, pairs = dti_batch
    K = 8
    w0 = ws[0]
    dt = torch.float64 if prec == "f64" else torch.float32
    p = sac.params(alpha=w0.alpha, rho=w0.rho, max_iter=K, eps_abs=0.0, eps_rel=0.0, prec=prec, near_bound=1e-3)
    grids = [sac.grid(w.m, w.h, w.pe) for w in ws]
    I1s = [cu(d["I1"], dt) for d in pairs]
    I2s = [cu(d["I2"], dt) for d in pairs]
    bs = [torch.zeros(sac.face_shape(g), dtype=torch.float64, device="cuda") for g in grids]
    bt = sac.Batch(grids, p, I1s, I2s, bs)
    bt.run(K, chunk=K)
    st = bt.stats()
    bt.finish()
    bt.close()
    assert np.all(st["iters"] == K)
    for k in (0, 37, 63):
        w, d = ws[k], pairs[k]
        og = oracle.Grid(w.m, w.h, w.pe)
        op = oracle.Params(alpha=w.alpha, rho=w.rho, max_iter=K, eps_abs=0.0, eps_rel=0.0,
                           knot32=1 if prec == "mixed" else 0)
        ref = oracle.admm(og, op, d["I1"].astype(np.float64), d["I2"].astype(np.float64), np.zeros(og.face_shape))
        bb = bs[k].cpu().numpy()
        if prec == "f64":
            assert np.linalg.norm(bb - ref["b"]) <= 1e-9 * np.linalg.norm(ref["b"]), k
        else:
            assert np.max(np.abs(bb - ref["b"])) / w.h[w.pe] <= 1e-3, k
