"""ctypes binding of ``libsac.so`` (include/sac.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays are torch CUDA tensors (device memory and streams come
from PyTorch); results are written in place or returned as tensors.  There is
no fallback: if the library is missing or the GPU is absent the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsac.so")
HEADER = os.path.join(_HERE, "..", "include", "sac.h")

SAC_OK, SAC_ENOTCONV = 0, 1
SAC_EINVAL, SAC_ENOMEM, SAC_ECUDA, SAC_EINFEASIBLE = -1, -2, -3, -4
SAC_ETIMEOUT, SAC_ENAN, SAC_ELSFAIL = -5, -6, -7
SAC_F64, SAC_MIXED = 0, 1


class SacGrid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("m", ctypes.c_int * 3), ("h", ctypes.c_double * 3),
                ("pe_axis", ctypes.c_int)]


class SacParams(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("alpha", "beta", "gamma", "rho", "eps_abs", "eps_rel", "eta", "eps_obj", "eps_iter",
                 "eps_grad", "gn_rel_grad")] + \
               [(n, ctypes.c_int) for n in ("max_iter", "n_sqp", "max_pcg", "precond", "max_gn", "prec")] + \
               [("near_bound", ctypes.c_double), ("check_every", ctypes.c_int),
                ("zstep_kernel", ctypes.c_int), ("autotune", ctypes.c_int), ("bstep_kernel", ctypes.c_int),
                ("adapt_rho", ctypes.c_int), ("rho_min", ctypes.c_double), ("rho_tau", ctypes.c_double),
                ("rho_mu", ctypes.c_double)]


class SacError(RuntimeError):
    def __init__(self, name, status):
        extra = ""
        if status == SAC_ECUDA:
            try:
                extra = f", cudaError {int(lib().sac_last_cuda_error())}"
            except (AttributeError, OSError):
                pass
        super().__init__(f"{name} failed with status {status} ({status_string(status)}{extra})")
        self.status = status


_lib = None


def lib():
    """Load libsac.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1607_00531_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, ip, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_size_t
        G, P = ctypes.POINTER(SacGrid), ctypes.POINTER(SacParams)
        sig = {
            "sac_params_default": (None, [P]),
            "sac_version": (ctypes.c_int, []),
            "sac_status_string": (ctypes.c_char_p, [ctypes.c_int]),
            "sac_workspace_bytes": (sz, [G, P]),
            "sac_zstep_fused": (ctypes.c_int, [G, P]),
            "sac_objective": (ctypes.c_int, [G, P, vp, vp, vp, dp, vp, sz, vp]),
            "sac_gradient": (ctypes.c_int, [G, P, vp, vp, vp, vp, vp, sz, vp]),
            "sac_corrected_images": (ctypes.c_int, [G, P, vp, vp, vp, vp, vp, dp, dp, vp, sz, vp]),
            "sac_multilevel_workspace_bytes": (sz, [G, ctypes.c_int, P]),
            "sac_restrict_image": (ctypes.c_int, [G, P, vp, vp, vp]),
            "sac_prolong_field": (ctypes.c_int, [G, vp, vp, vp]),
            "sac_multilevel_solve": (ctypes.c_int, [G, ctypes.c_int, P, vp, vp, vp, ip, dp, vp, sz, vp]),
            "sac_objective_noalloc": (ctypes.c_int, [G, P, vp, vp, vp, dp, vp]),
            "sac_objective_noalloc_max_bytes": (sz, []),
            "sac_bstep": (ctypes.c_int, [G, P, vp, vp, vp, vp, vp, vp, ip, vp, sz, vp]),
            "sac_zstep": (ctypes.c_int, [G, P, vp, vp, vp, vp, dp, vp, sz, vp]),
            "sac_admm_solve": (ctypes.c_int, [G, P, vp, vp, vp, vp, vp, ip, dp, dp, dp, vp, sz, vp]),
            "sac_hessvec": (ctypes.c_int, [G, P, vp, vp, vp, vp, vp, vp, sz, vp]),
            "sac_precond_solve": (ctypes.c_int, [G, P, vp, vp, vp, vp, vp, vp, sz, vp]),
            "sac_gnpcg_solve": (ctypes.c_int, [G, P, vp, vp, vp, ip, dp, dp, dp, vp, sz, vp]),
            "sac_batch_workspace_bytes": (sz, [ctypes.c_int, G, P]),
            "sac_batch_create": (ctypes.c_int, [ctypes.c_int, G, P, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                ctypes.POINTER(vp), vp, sz, vp, ctypes.POINTER(vp)]),
            "sac_batch_run": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
            "sac_batch_stats": (ctypes.c_int, [vp, ip, ip, dp, dp]),
            "sac_batch_finish": (ctypes.c_int, [vp]),
            "sac_batch_destroy": (None, [vp]),
            "sac_batch_last_run_ms": (ctypes.c_double, [vp]),
            "sac_server_request_bytes": (sz, [P, G]),
            "sac_server_create": (ctypes.c_int, [P, vp, sz, ctypes.c_int, vp, ctypes.POINTER(vp)]),
            "sac_server_submit": (ctypes.c_int, [vp, G, vp, vp, ctypes.POINTER(ctypes.c_longlong)]),
            "sac_server_step": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, ip, ip]),
            "sac_server_poll": (ctypes.c_int, [vp, ctypes.c_longlong, ip, ip, ip, dp]),
            "sac_server_fetch": (ctypes.c_int, [vp, ctypes.c_longlong, dp]),
            "sac_server_totals": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_longlong)]),
            "sac_server_destroy": (None, [vp]),
            "sac_profile_enable": (ctypes.c_int, [ctypes.c_int]),
            "sac_profile_read": (ctypes.c_int, [dp, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int]),
            "sac_launch_count": (ctypes.c_longlong, []),
            "sac_set_wait_limit": (ctypes.c_int, [ctypes.c_int, ctypes.c_longlong]),
            "sac_last_cuda_error": (ctypes.c_int, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_symbols():
    """Function names declared in include/sac.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sac_[a-z0-9_]+)\s*\(", txt)))


def status_string(st):
    return lib().sac_status_string(int(st)).decode()


def grid(m, h, pe):
    g = SacGrid()
    g.ndim = len(m)
    for a in range(3):
        g.m[a] = int(m[a]) if a < len(m) else 1
        g.h[a] = float(h[a]) if a < len(m) else 1.0
    g.pe_axis = int(pe)
    return g


def params(**kw):
    p = SacParams()
    lib().sac_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if k == "prec" and isinstance(v, str):
            v = {"f64": SAC_F64, "mixed": SAC_MIXED}[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def face_shape(g):
    return tuple(g.m[a] + (1 if a == g.pe_axis else 0) for a in range(g.ndim))


def cell_shape(g):
    return tuple(g.m[a] for a in range(g.ndim))


def workspace_bytes(g, p):
    return int(lib().sac_workspace_bytes(ctypes.byref(g), ctypes.byref(p)))


def _torch():
    import torch
    return torch


def zstep_fused(g, p):
    """How the z-step is launched (host only): 2 on the chip in one launch per
    iteration, 1 with passes 1 and 2 as one launch, 0 pass by pass."""
    r = int(lib().sac_zstep_fused(ctypes.byref(g), ctypes.byref(p)))
    if r < 0:
        raise SacError("sac_zstep_fused", r)
    return r


def workspace(g, p, device="cuda"):
    torch = _torch()
    n = workspace_bytes(g, p)
    if n == 0:
        raise SacError("sac_workspace_bytes", SAC_EINVAL)
    return torch.empty(n, dtype=torch.uint8, device=device)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("arrays must be CUDA tensors")
    if not t.is_contiguous():
        raise ValueError("arrays must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(name, st, allow_notconv=True):
    if st < 0 or (st == SAC_ENOTCONV and not allow_notconv):
        raise SacError(name, st)
    return st


def _img_dtype(p):
    torch = _torch()
    return torch.float32 if p.prec == SAC_MIXED else torch.float64


def _check_inputs(g, p, I1, I2):
    torch = _torch()
    for I in (I1, I2):
        if tuple(I.shape) != cell_shape(g) or I.dtype != _img_dtype(p):
            raise ValueError(f"image must be {cell_shape(g)} {_img_dtype(p)}, got {tuple(I.shape)} {I.dtype}")


def _ws(g, p, ws):
    return ws if ws is not None else workspace(g, p)


def objective(g, p, I1, I2, b, ws=None, stream=None):
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    out = (ctypes.c_double * 4)()
    _check("sac_objective", lib().sac_objective(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), out,
                                                _ptr(ws), ws.numel(), _stream(stream)))
    return dict(J=out[0], D=out[1], S=out[2], P=out[3])


def corrected_images(g, p, I1, I2, b, T1=None, T2=None, ws=None, stream=None):
    """Transformed images T1, T2 (new tensors of the image dtype unless given)
    and the SSD / NCC similarity (Sec. 6)."""
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    T1 = _torch().empty_like(I1) if T1 is None else T1
    T2 = _torch().empty_like(I2) if T2 is None else T2
    ssd, ncc = ctypes.c_double(0), ctypes.c_double(0)
    _check("sac_corrected_images",
           lib().sac_corrected_images(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), _ptr(T1),
                                      _ptr(T2), ctypes.byref(ssd), ctypes.byref(ncc), _ptr(ws), ws.numel(),
                                      _stream(stream)))
    return dict(T1=T1, T2=T2, ssd=ssd.value, ncc=ncc.value)


def restrict_image(g_fine, p, I, stream=None):
    """Coarse image (block means of the fine cells)."""
    Ic = _torch().empty(tuple(int(x) // 2 for x in I.shape), dtype=I.dtype, device=I.device)
    _check("sac_restrict_image", lib().sac_restrict_image(ctypes.byref(g_fine), ctypes.byref(p), _ptr(I), _ptr(Ic),
                                                          _stream(stream)))
    return Ic


def prolong_field(g_fine, bc, stream=None):
    """Fine face array from a coarse one (linear interpolation, Sec. 4.4)."""
    bf = _torch().empty(face_shape(g_fine), dtype=_torch().float64, device=bc.device)
    _check("sac_prolong_field", lib().sac_prolong_field(ctypes.byref(g_fine), _ptr(bc), _ptr(bf), _stream(stream)))
    return bf


def multilevel_solve(g, levels, p, I1, I2, b, ws=None, stream=None):
    """Coarse-to-fine ADMM; b (fine faces, double) receives the result."""
    _check_inputs(g, p, I1, I2)
    n = int(lib().sac_multilevel_workspace_bytes(ctypes.byref(g), int(levels), ctypes.byref(p)))
    if n == 0:
        raise SacError("sac_multilevel_workspace_bytes", SAC_EINVAL)
    ws = _torch().empty(n, dtype=_torch().uint8, device="cuda") if ws is None else ws
    its = (ctypes.c_int * int(levels))()
    rho = ctypes.c_double(0)
    st = lib().sac_multilevel_solve(ctypes.byref(g), int(levels), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), its,
                                    ctypes.byref(rho), _ptr(ws), ws.numel(), _stream(stream))
    if st < 0:
        raise SacError("sac_multilevel_solve", st)
    return dict(iters=list(its), rho=rho.value, status=st)


def objective_noalloc(g, p, I1, I2, b, stream=None):
    """sac_objective without a workspace: its scratch is a fixed array inside
    the library (see include/sac.h), for callers that cannot allocate."""
    _check_inputs(g, p, I1, I2)
    out = (ctypes.c_double * 4)()
    _check("sac_objective_noalloc", lib().sac_objective_noalloc(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2),
                                                                _ptr(b), out, _stream(stream)))
    return dict(J=out[0], D=out[1], S=out[2], P=out[3])


def gradient(g, p, I1, I2, b, ws=None, stream=None):
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    out = _torch().empty_like(b)
    _check("sac_gradient", lib().sac_gradient(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b),
                                              _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def bstep(g, p, I1, I2, b, z, u, out=None, ws=None, stream=None):
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    out = _torch().empty_like(b) if out is None else out
    cap = ctypes.c_int(0)
    _check("sac_bstep", lib().sac_bstep(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), _ptr(z),
                                        _ptr(u), _ptr(out), ctypes.byref(cap), _ptr(ws), ws.numel(),
                                        _stream(stream)))
    return out, bool(cap.value)


def zstep(g, p, b, u, z, u_out=None, ws=None, stream=None):
    """z is updated in place (z^k -> z^{k+1}); returns (u_out, norms5)."""
    ws = _ws(g, p, ws)
    u_out = _torch().empty_like(u) if u_out is None else u_out
    nr = (ctypes.c_double * 5)()
    _check("sac_zstep", lib().sac_zstep(ctypes.byref(g), ctypes.byref(p), _ptr(b), _ptr(u), _ptr(z), _ptr(u_out),
                                        nr, _ptr(ws), ws.numel(), _stream(stream)))
    return u_out, np.array(nr[:])


def admm_solve(g, p, I1, I2, b, z=None, u=None, want_hist=False, ws=None, stream=None):
    """b (in: feasible b^0, out: result), z, u (in/out or None) in place."""
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    it = ctypes.c_int(0)
    rp, rd = ctypes.c_double(0), ctypes.c_double(0)
    hist = np.zeros((max(p.max_iter, 1), 6)) if want_hist else None
    st = lib().sac_admm_solve(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), _ptr(z), _ptr(u),
                              ctypes.byref(it), ctypes.byref(rp), ctypes.byref(rd),
                              hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_hist else None, _ptr(ws), ws.numel(),
                              _stream(stream))
    _check("sac_admm_solve", st)
    res = dict(iters=it.value, r_pri=rp.value, r_dual=rd.value, converged=(st == SAC_OK), status=st)
    if want_hist:
        res["hist"] = hist[:it.value]
    return res


def hessvec(g, p, I1, I2, b, v, ws=None, stream=None):
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    out = _torch().empty_like(v)
    _check("sac_hessvec", lib().sac_hessvec(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), _ptr(v),
                                            _ptr(out), _ptr(ws), ws.numel(), _stream(stream)))
    return out


def precond_solve(g, p, I1, I2, b, rhs, ws=None, stream=None):
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    out = _torch().empty_like(rhs)
    _check("sac_precond_solve", lib().sac_precond_solve(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2),
                                                        _ptr(b), _ptr(rhs), _ptr(out), _ptr(ws), ws.numel(),
                                                        _stream(stream)))
    return out


def gnpcg_solve(g, p, I1, I2, b, want_hist=False, ws=None, stream=None):
    _check_inputs(g, p, I1, I2)
    ws = _ws(g, p, ws)
    it = ctypes.c_int(0)
    J, gn = ctypes.c_double(0), ctypes.c_double(0)
    hist = np.zeros((max(p.max_gn, 1), 5)) if want_hist else None
    st = lib().sac_gnpcg_solve(ctypes.byref(g), ctypes.byref(p), _ptr(I1), _ptr(I2), _ptr(b), ctypes.byref(it),
                               ctypes.byref(J), ctypes.byref(gn),
                               hist.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if want_hist else None, _ptr(ws), ws.numel(),
                               _stream(stream))
    _check("sac_gnpcg_solve", st)
    res = dict(iters=it.value, J=J.value, gnorm=gn.value, converged=(st == SAC_OK), status=st)
    if want_hist:
        res["hist"] = hist[:it.value]
    return res


PHASES = ["bstep", "bstep_refine", "zpass0", "zpass1", "zpass2", "zpass3", "admm_update", "zslab"]


def profile_enable(on=True):
    lib().sac_profile_enable(1 if on else 0)


def profile_read(reset=True):
    ms = (ctypes.c_double * len(PHASES))()
    n = (ctypes.c_longlong * len(PHASES))()
    lib().sac_profile_read(ms, n, 1 if reset else 0)
    return {name: (ms[i], n[i]) for i, name in enumerate(PHASES)}


def launch_count():
    return int(lib().sac_launch_count())


WAIT_BSTEP, WAIT_ZSTEP = 1, 2


def set_wait_limit(which, tests):
    """Bounded-wait limit of the selected kernels on the current device
    (tests < 0: the default)."""
    _check("sac_set_wait_limit", lib().sac_set_wait_limit(int(which), int(tests)), allow_notconv=False)


def _grid_array(grids):
    arr = (SacGrid * len(grids))()
    for i, g in enumerate(grids):
        arr[i] = g
    return arr


def batch_workspace_bytes(grids, p):
    return int(lib().sac_batch_workspace_bytes(len(grids), _grid_array(grids), ctypes.byref(p)))


class Batch:
    """Many volumes solved by ADMM together (one launch per phase over all of
    them, device-side per-volume stopping, CUDA-graph replay).  bs[j] holds
    b^0 and receives the result after finish()."""

    def __init__(self, grids, p, I1s, I2s, bs, ws=None, stream=None):
        n = len(grids)
        for g, I1, I2 in zip(grids, I1s, I2s):
            _check_inputs(g, p, I1, I2)
        self.n, self.p = n, p
        self._keep = (list(I1s), list(I2s), list(bs))
        nbytes = batch_workspace_bytes(grids, p)
        if nbytes == 0:
            raise SacError("sac_batch_workspace_bytes", SAC_EINVAL)
        self.ws = ws if ws is not None else _torch().empty(nbytes, dtype=_torch().uint8, device="cuda")
        V = ctypes.c_void_p * n
        h = ctypes.c_void_p()
        _check("sac_batch_create", lib().sac_batch_create(
            n, _grid_array(grids), ctypes.byref(p), V(*[_ptr(x) for x in I1s]), V(*[_ptr(x) for x in I2s]),
            V(*[_ptr(x) for x in bs]), _ptr(self.ws), self.ws.numel(), _stream(stream), ctypes.byref(h)))
        self.h = h

    def run(self, max_iter, chunk=10):
        return _check("sac_batch_run", lib().sac_batch_run(self.h, int(max_iter), int(chunk)))

    def stats(self):
        n = self.n
        it, cv = (ctypes.c_int * n)(), (ctypes.c_int * n)()
        rp, rd = (ctypes.c_double * n)(), (ctypes.c_double * n)()
        _check("sac_batch_stats", lib().sac_batch_stats(self.h, it, cv, rp, rd))
        return dict(iters=np.array(it[:]), converged=np.array(cv[:], dtype=bool), r_pri=np.array(rp[:]),
                    r_dual=np.array(rd[:]))

    def finish(self):
        return _check("sac_batch_finish", lib().sac_batch_finish(self.h))

    def last_run_ms(self):
        return float(lib().sac_batch_last_run_ms(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().sac_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching SAC server over a device-memory pool (the
    admission budget).  submit() takes host (numpy) images; step() admits,
    iterates and retires; fetch() returns a finished field as numpy."""

    def __init__(self, p, pool_bytes, max_jobs=64, stream=None):
        torch = _torch()
        self.p = p
        self.pool = torch.empty(int(pool_bytes), dtype=torch.uint8, device="cuda")
        h = ctypes.c_void_p()
        _check("sac_server_create", lib().sac_server_create(ctypes.byref(p), _ptr(self.pool), self.pool.numel(),
                                                            int(max_jobs), _stream(stream), ctypes.byref(h)))
        self.h = h
        self.grids = {}

    def submit(self, g, I1, I2):
        dt = np.float32 if self.p.prec == SAC_MIXED else np.float64
        a1 = np.ascontiguousarray(I1, dtype=dt)
        a2 = np.ascontiguousarray(I2, dtype=dt)
        t = ctypes.c_longlong(0)
        _check("sac_server_submit", lib().sac_server_submit(self.h, ctypes.byref(g), a1.ctypes.data_as(ctypes.c_void_p),
                                                            a2.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t)))
        self.grids[t.value] = g
        return t.value

    def step(self, iters, chunk=10):
        nr, nq = ctypes.c_int(0), ctypes.c_int(0)
        _check("sac_server_step", lib().sac_server_step(self.h, int(iters), int(chunk), ctypes.byref(nr),
                                                        ctypes.byref(nq)))
        return nr.value, nq.value

    def poll(self, ticket):
        st, it, cv = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        tm = (ctypes.c_double * 3)()
        _check("sac_server_poll", lib().sac_server_poll(self.h, ticket, ctypes.byref(st), ctypes.byref(it),
                                                        ctypes.byref(cv), tm))
        return dict(state=st.value, iters=it.value, converged=bool(cv.value), t_submit=tm[0], t_admit=tm[1],
                    t_done=tm[2])

    def fetch(self, ticket):
        g = self.grids.pop(ticket)
        out = np.zeros(face_shape(g))
        _check("sac_server_fetch", lib().sac_server_fetch(self.h, ticket,
                                                          out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def request_bytes(self, g):
        return int(lib().sac_server_request_bytes(ctypes.byref(self.p), ctypes.byref(g)))

    def totals(self):
        t = (ctypes.c_longlong * 3)()
        _check("sac_server_totals", lib().sac_server_totals(self.h, t))
        return dict(iters=t[0], faces_iters=t[1], pool_used=t[2])

    def close(self):
        if getattr(self, "h", None):
            lib().sac_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
