"""The workspace-free objective (sac_objective_noalloc), for callers that
cannot allocate device memory: it must return what sac_objective returns,
call after call, although every call reuses the same fixed scratch array
inside the library.  Collected last on purpose."""
import numpy as np
import pytest

from paper_1607_00531_gb300 import phantoms as ph

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _inputs(m, pe, seed):
    h = tuple(1.0 / m[0] for _ in m)
    I1 = ph.random_images(m, seed + 1)
    I2 = ph.random_images(m, seed + 2)
    b = ph.random_field(m, pe, h, seed + 3, max_d=0.6)
    return h, I1, I2, b


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_noalloc_objective_equals_workspace_objective_on_consecutive_calls(prec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00531_gb300 import build, sac
    build.build()
    dt = torch.float64 if prec == "f64" else torch.float32
    assert sac.lib().sac_objective_noalloc_max_bytes() == 1 << 20
    # two different problems, one call each, in a row: the second call must not
    # see anything left in the shared scratch by the first
    for m, pe, seed in (((37, 50), 1, 1), ((9, 70, 21), 1, 2)):
        h, I1, I2, b = _inputs(m, pe, seed)
        g = sac.grid(m, h, pe)
        p = sac.params(alpha=0.7, beta=0.4, prec=prec)
        tI1 = torch.as_tensor(I1, dtype=dt, device="cuda")
        tI2 = torch.as_tensor(I2, dtype=dt, device="cuda")
        tb = torch.as_tensor(b, dtype=torch.float64, device="cuda")
        ref = sac.objective(g, p, tI1, tI2, tb)
        got = sac.objective_noalloc(g, p, tI1, tI2, tb)
        for k in ("J", "D", "S", "P"):
            assert got[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-300), (k, got[k], ref[k])


def test_noalloc_objective_rejects_grids_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_00531_gb300 import build, sac
    build.build()
    m = (4096, 8, 4096)                       # far more partial sums than 1 MiB holds
    g = sac.grid(m, (1.0, 1.0, 1.0), 1)
    p = sac.params(prec="mixed")
    tiny = torch.zeros(16, dtype=torch.float32, device="cuda")
    tb = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = sac.lib().sac_objective_noalloc(__import__("ctypes").byref(g), __import__("ctypes").byref(p),
                                         sac._ptr(tiny), sac._ptr(tiny), sac._ptr(tb),
                                         (__import__("ctypes").c_double * 4)(), sac._stream(None))
    assert st == sac.SAC_ENOMEM
