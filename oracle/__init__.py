"""ctypes loader for the FP64 CPU oracle (``oracle/sac_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library never
imports, links or calls anything here, and nothing here imports the CUDA
package.  Every function below marshals numpy arrays into the C oracle; no
arithmetic of the method lives in this file.

Paper: Macdonald & Ruthotto, "Efficient Numerical Optimization for
Susceptibility Artifact Correction of EPI-MRI" (arXiv 1607.00531).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, fields

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sac_oracle.c")
_LIB = os.path.join(_HERE, "libsac_oracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over lines, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_long)
        P = ctypes.POINTER(RefParams)
        g = [ctypes.c_int, ip, dp, ctypes.c_int]
        for name, args in {
            "ref_objective": g + [P, dp, dp, dp, dp],
            "ref_residual": g + [dp, dp, dp, dp],
            "ref_gradient": g + [P, dp, dp, dp, dp],
            "ref_apply": g + [P, ctypes.c_int, dp, dp, dp, dp, dp],
            "ref_line_qp": [ctypes.c_long, ctypes.c_double, dp, dp, dp, dp, dp, ip],
            "ref_bstep": g + [P, dp, dp, dp, dp, dp, dp, lp],
            "ref_zstep": g + [P, dp, dp, dp],
            "ref_admm": g + [P, dp, dp, dp, dp, dp, dp, lp],
            "ref_precond_solve": g + [P, dp, dp, dp, dp, dp],
            "ref_pcg": g + [P, dp, dp, dp, dp, dp, dp],
            "ref_gnpcg": g + [P, dp, dp, dp, dp, lp, dp, dp],
            "ref_corrected": g + [dp, dp, dp, dp, dp, dp],
            "ref_restrict": [ctypes.c_int, ip, dp, dp],
            "ref_prolong": [ctypes.c_int, ip, ctypes.c_int, dp, dp],
            "ref_multilevel_admm": g + [P, ctypes.c_int, dp, dp, dp, dp, dp, lp, ip, dp, dp],
        }.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.ref_max_abs_d1.argtypes = g + [dp]
        L.ref_max_abs_d1.restype = ctypes.c_double
        for name in ("ref_phi", "ref_dphi", "ref_d2phi"):
            getattr(L, name).argtypes = [ctypes.c_double]
            getattr(L, name).restype = ctypes.c_double
        L.ref_dct_matrix.argtypes = [ctypes.c_long, dp]
        L.ref_dct_matrix.restype = None
        L.ref_dct_eigs.argtypes = [ctypes.c_long, ctypes.c_double, dp]
        L.ref_dct_eigs.restype = None
        L.ref_max_threads.argtypes = []
        L.ref_max_threads.restype = ctypes.c_int
        _lib = L
    return _lib


class RefParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("alpha", "beta", "gamma", "rho", "eps_abs", "eps_rel", "eta", "eps_obj",
                 "eps_iter", "eps_grad", "gn_rel_grad")] + \
               [(n, ctypes.c_int) for n in
                ("max_iter", "n_sqp", "max_pcg", "precond", "max_gn", "nthreads", "adapt_rho")] + \
               [(n, ctypes.c_double) for n in ("rho_min", "rho_tau", "rho_mu")] + \
               [("knot32", ctypes.c_int)]


@dataclass
class Params:
    """Method parameters with the paper's values as defaults.

    gamma = 1e-3 (Sec. 3), eta = 0.1 (Sec. 4.1), eps_obj = 1e-3,
    eps_iter = eps_grad = 1e-2, 10 GN iterations (Sec. 4.1),
    eps_abs = eps_rel = 0.2 (Sec. 4.2), beta = 10 (Sec. 5).
    """
    alpha: float = 50.0
    beta: float = 0.0
    gamma: float = 1e-3
    rho: float = 1e2
    eps_abs: float = 0.2
    eps_rel: float = 0.2
    eta: float = 0.1
    eps_obj: float = 1e-3
    eps_iter: float = 1e-2
    eps_grad: float = 1e-2
    gn_rel_grad: float = 0.0
    max_iter: int = 50
    n_sqp: int = 1
    max_pcg: int = 50
    precond: int = 2
    max_gn: int = 10
    nthreads: int = 0
    adapt_rho: int = 0          # 0 fixed, 1 adaptive (Boyd et al.), 2 adaptive with lower bound
    rho_min: float = 1e2
    rho_tau: float = 1.3
    rho_mu: float = 10.0
    # 1: interpolation positions formed in FP32 as the single-precision
    # kernels form them (the model's interval is an integer decided in
    # floating point; tests of FP32 kernels take that decision in FP32)
    knot32: int = 0

    def c(self) -> RefParams:
        return RefParams(**{f.name: getattr(self, f.name) for f in fields(self)})


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Cells m (2 or 3 entries), spacings h, phase-encoding axis pe (0-based)."""

    def __init__(self, m, h, pe):
        self.m = tuple(int(x) for x in m)
        self.h = tuple(float(x) for x in h)
        self.pe = int(pe)
        self.nd = len(self.m)
        self._m = (ctypes.c_int * 3)(*(list(self.m) + [1] * (3 - self.nd)))
        self._h = (ctypes.c_double * 3)(*(list(self.h) + [1.0] * (3 - self.nd)))

    @property
    def face_shape(self):
        return tuple(mm + (1 if a == self.pe else 0) for a, mm in enumerate(self.m))

    @property
    def cell_shape(self):
        return self.m

    def args(self):
        return [self.nd, self._m, self._h, self.pe]


def _check(st, name):
    if st < 0:
        raise RuntimeError(f"{name} returned status {st}")
    return st


def objective(grid, prm, I1, I2, b):
    out = np.zeros(4)
    _check(lib().ref_objective(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)),
                               _dp(_f64(b)), _dp(out)), "ref_objective")
    return dict(J=out[0], D=out[1], S=out[2], P=out[3])


def residual(grid, I1, I2, b):
    r = np.zeros(grid.cell_shape)
    _check(lib().ref_residual(*grid.args(), _dp(_f64(I1)), _dp(_f64(I2)), _dp(_f64(b)), _dp(r)),
           "ref_residual")
    return r


def gradient(grid, prm, I1, I2, b):
    gr = np.zeros(grid.face_shape)
    _check(lib().ref_gradient(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)),
                              _dp(_f64(b)), _dp(gr)), "ref_gradient")
    return gr


OPS = dict(HD=0, lapS=1, D1tD1=2, D2tD2=3, HP=4, HJGN=5, Pblock=6, D3tD3=7, M=8)


def apply(grid, prm, op, I1, I2, b, v):
    out = np.zeros(grid.face_shape)
    _check(lib().ref_apply(*grid.args(), ctypes.byref(prm.c()), OPS[op] if isinstance(op, str) else op,
                           _dp(_f64(I1)), _dp(_f64(I2)), _dp(_f64(b)), _dp(_f64(v)), _dp(out)),
           "ref_apply")
    return out


def line_qp(h, Gd, Go, c, dk):
    m = len(dk)
    x = np.zeros(m + 1)
    na = ctypes.c_int(0)
    res = lib().ref_line_qp(m, h, _dp(_f64(Gd)), _dp(_f64(Go)), _dp(_f64(c)), _dp(_f64(dk)), _dp(x),
                            ctypes.byref(na))
    return x, res, na.value


def bstep(grid, prm, I1, I2, b, z, u):
    out = np.zeros(grid.face_shape)
    stats = (ctypes.c_long * 3)()
    _check(lib().ref_bstep(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)),
                           _dp(_f64(b)), _dp(_f64(z)), _dp(_f64(u)), _dp(out), stats), "ref_bstep")
    return out, dict(capped=stats[0], active=stats[1], passes=stats[2])


def zstep(grid, prm, b, u):
    z = np.zeros(grid.face_shape)
    _check(lib().ref_zstep(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(b)), _dp(_f64(u)), _dp(z)),
           "ref_zstep")
    return z


def admm(grid, prm, I1, I2, b0, z0=None, u0=None, want_hist=False):
    b = _f64(b0).copy()
    z = b.copy() if z0 is None else _f64(z0).copy()
    u = np.zeros_like(b) if u0 is None else _f64(u0).copy()
    hist = np.zeros((max(prm.max_iter, 1), 6)) if want_hist else None
    info = (ctypes.c_long * 3)()
    st = lib().ref_admm(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)), _dp(b),
                        _dp(z), _dp(u), _dp(hist) if want_hist else None, info)
    _check(st, "ref_admm")
    res = dict(b=b, z=z, u=u, iters=info[0], converged=bool(info[1]), capped=info[2], status=st)
    if want_hist:
        res["hist"] = hist[:info[0]]
    return res


def precond_solve(grid, prm, I1, I2, b, rhs):
    out = np.zeros(grid.face_shape)
    _check(lib().ref_precond_solve(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)),
                                   _dp(_f64(b)), _dp(_f64(rhs)), _dp(out)), "ref_precond_solve")
    return out


def pcg(grid, prm, I1, I2, b, grad):
    d = np.zeros(grid.face_shape)
    rel = ctypes.c_double(0)
    its = lib().ref_pcg(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)), _dp(_f64(b)),
                        _dp(_f64(grad)), _dp(d), ctypes.byref(rel))
    return d, its, rel.value


def gnpcg(grid, prm, I1, I2, b0, want_hist=False):
    b = _f64(b0).copy()
    hist = np.zeros((max(prm.max_gn, 1), 5)) if want_hist else None
    info = (ctypes.c_long * 3)()
    J = ctypes.c_double(0)
    gn = ctypes.c_double(0)
    st = lib().ref_gnpcg(*grid.args(), ctypes.byref(prm.c()), _dp(_f64(I1)), _dp(_f64(I2)), _dp(b),
                         _dp(hist) if want_hist else None, info, ctypes.byref(J), ctypes.byref(gn))
    res = dict(b=b, iters=info[0], converged=bool(info[1]), pcg_iters=info[2], J=J.value,
               gnorm=gn.value, status=st)
    if want_hist:
        res["hist"] = hist[:info[0]]
    return res


def corrected(grid, I1, I2, b):
    """Transformed images T1 = I1(x + A b)(1 + D1 b), T2 = I2(x - A b)(1 - D1 b),
    SSD = h^d/2 |T1 - T2|^2 and NCC = <T1,T2>^2 / (|T1|^2 |T2|^2)."""
    T1 = np.zeros(grid.cell_shape)
    T2 = np.zeros(grid.cell_shape)
    out = np.zeros(2)
    _check(lib().ref_corrected(*grid.args(), _dp(_f64(I1)), _dp(_f64(I2)), _dp(_f64(b)), _dp(T1), _dp(T2),
                               _dp(out)), "ref_corrected")
    return dict(T1=T1, T2=T2, ssd=out[0], ncc=out[1])


def restrict(m, I):
    """Mean of the 2^d fine cells of every coarse cell (m: fine cells)."""
    m = tuple(int(x) for x in m)
    Ic = np.zeros(tuple(x // 2 for x in m))
    mm = (ctypes.c_int * 3)(*(list(m) + [1] * (3 - len(m))))
    _check(lib().ref_restrict(len(m), mm, _dp(_f64(I)), _dp(Ic)), "ref_restrict")
    return Ic


def prolong(m, pe, bc):
    """Fine faces from coarse faces by linear interpolation (m: fine cells)."""
    m = tuple(int(x) for x in m)
    bf = np.zeros(tuple(x + (1 if a == pe else 0) for a, x in enumerate(m)))
    mm = (ctypes.c_int * 3)(*(list(m) + [1] * (3 - len(m))))
    _check(lib().ref_prolong(len(m), mm, int(pe), _dp(_f64(bc)), _dp(bf)), "ref_prolong")
    return bf


def multilevel_admm(m, h, pe, prm, I1, I2, levels):
    """Coarse-to-fine ADMM (Sec. 4.4; ref_multilevel_admm).  Returns one dict
    per level, coarsest first, with the grid, the iterations, the converged
    flag and the augmentation parameter carried to the next level; the finest
    level's dict also holds b, z, u and the history."""
    m = tuple(int(x) for x in m)
    h = tuple(float(x) for x in h)
    g = Grid(m, h, pe)
    b = np.zeros(g.face_shape)
    z = np.zeros(g.face_shape)
    u = np.zeros(g.face_shape)
    iters = (ctypes.c_long * levels)()
    conv = (ctypes.c_int * levels)()
    rho = (ctypes.c_double * levels)()
    hist = np.zeros((max(prm.max_iter, 1), 6))
    st = lib().ref_multilevel_admm(*g.args(), ctypes.byref(prm.c()), int(levels), _dp(_f64(I1)), _dp(_f64(I2)),
                                   _dp(b), _dp(z), _dp(u), iters, conv, rho, _dp(hist))
    _check(st, "ref_multilevel_admm")
    out = []
    for lvl in range(levels):
        f = 2 ** (levels - 1 - lvl)
        out.append(dict(m=tuple(x // f for x in m), h=tuple(x * f for x in h), iters=iters[lvl],
                        converged=bool(conv[lvl]), rho=rho[lvl]))
    out[-1].update(b=b, z=z, u=u, hist=hist[:iters[levels - 1]])
    return out


def max_abs_d1(grid, b):
    return lib().ref_max_abs_d1(*grid.args(), _dp(_f64(b)))


def phi(x):
    return lib().ref_phi(float(x))


def dphi(x):
    return lib().ref_dphi(float(x))


def d2phi(x):
    return lib().ref_d2phi(float(x))


def dct_matrix(m):
    C = np.zeros((m, m))
    lib().ref_dct_matrix(m, _dp(C))
    return C


def dct_eigs(m, h):
    lam = np.zeros(m)
    lib().ref_dct_eigs(m, h, _dp(lam))
    return lam


def max_threads():
    return lib().ref_max_threads()
