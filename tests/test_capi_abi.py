"""The C-ABI library loads, exports every symbol include/sac.h declares, and
rejects invalid arguments before touching the GPU (no GPU needed)."""
import ctypes

import pytest

from paper_1607_00531_gb300 import build as sac_build
from paper_1607_00531_gb300 import sac


@pytest.fixture(scope="module")
def L():
    sac_build.build()
    return sac.lib()


def test_every_declared_symbol_is_exported(L):
    names = sac.header_symbols()
    assert "sac_admm_solve" in names and "sac_gnpcg_solve" in names
    for n in names:
        assert hasattr(L, n), n


def test_param_defaults_are_the_papers(L):
    p = sac.params()
    assert p.gamma == 1e-3 and p.eta == 0.1 and p.eps_obj == 1e-3 and p.eps_iter == 1e-2
    assert p.eps_grad == 1e-2 and p.max_gn == 10 and p.eps_abs == 0.2 and p.eps_rel == 0.2
    assert p.rho == 1e2 and p.beta == 10.0 and p.n_sqp == 1 and p.precond == 2
    assert L.sac_version() == 1


def test_workspace_size_and_invalid_grids(L):
    p = sac.params()
    g = sac.grid((16, 12), (0.1, 0.1), 1)
    n = sac.workspace_bytes(g, p)
    assert n > 10 * 16 * 13 * 8
    assert sac.workspace_bytes(sac.grid((16, 12), (0.1, 0.1), 2), p) == 0      # pe out of range
    assert sac.workspace_bytes(sac.grid((16, 480), (0.1, 0.1), 1), p) == 0     # PE line too long
    assert sac.workspace_bytes(sac.grid((16, 479), (0.1, 0.1), 1), p) > 0
    assert sac.workspace_bytes(sac.grid((16, 12), (0.1, -1.0), 1), p) == 0
    bad = sac.params(rho=0.0)
    assert sac.workspace_bytes(g, bad) == 0
    assert sac.workspace_bytes(g, sac.params(n_sqp=0)) == 0


def test_entry_points_reject_null_arrays(L):
    p = sac.params()
    g = sac.grid((8, 8, 4), (0.1, 0.1, 0.1), 1)
    out = (ctypes.c_double * 4)()
    assert L.sac_objective(ctypes.byref(g), ctypes.byref(p), None, None, None, out, None, 0, None) == sac.SAC_EINVAL
    assert L.sac_admm_solve(ctypes.byref(g), ctypes.byref(p), None, None, None, None, None, None, None, None, None,
                            None, 0, None) == sac.SAC_EINVAL
    assert L.sac_status_string(-4).decode() == "infeasible starting field"


def test_zstep_fusion_decision_needs_no_device(L):
    # 2: the whole z-step on the chip (3D, last axis not the PE axis, at most
    # 256 faces along the first non-PE axis and 128 along the last; mixed
    # precision, zstep_kernel 0 for slabs of at least 8192 faces, 3 for any); 1: passes 1 and 2 as one launch when both
    # DCT matrices of the second non-PE axis fit beside the rings (axes up to
    # 96 faces); 0: pass by pass
    def fused(m, pe, prec, kern=0):
        g = sac.grid(m, tuple(1.0 / x for x in m), pe)
        return sac.zstep_fused(g, sac.params(prec=prec, zstep_kernel=kern))
    assert fused((256, 256, 80), 1, "mixed") == 2
    assert fused((64, 60, 128), 1, "mixed") == 2
    assert fused((60, 64, 128), 0, "mixed") == 2
    assert fused((300, 9, 8), 1, "mixed") != 2         # 301 faces along the first non-PE axis
    assert fused((8, 9, 130), 1, "mixed") != 2         # 130 along the last
    assert fused((64, 60, 96), 2, "mixed") == 1        # PE last: per-axis passes, 1 + 2 fused
    assert fused((96, 96, 60), 1, "mixed") == 1        # 96 x 60 slabs: below 8192 faces, per-axis
    assert fused((96, 96, 60), 1, "mixed", 3) == 2     # ... on the chip when asked for
    assert fused((256, 256, 80), 1, "mixed", 2) == 1
    assert fused((64, 60, 96), 1, "mixed", 2) == 1
    assert fused((64, 60, 112), 1, "mixed", 2) == 0
    assert fused((64, 60, 128), 1, "mixed", 2) == 0
    assert fused((256, 256, 80), 1, "mixed", 1) == 0
    assert fused((256, 256, 80), 1, "f64") == 0
    assert fused((128, 128), 1, "mixed") == 0          # 2D: no second axis to fuse
    with pytest.raises(sac.SacError):
        sac.zstep_fused(sac.grid((16, 12), (0.1, 0.1), 2), sac.params())
