"""Seeded synthetic inputs: a phantom, a field inhomogeneity and the two
oppositely distorted images it produces.

This module is the only code shared by the CUDA path's callers and the CPU
oracle's callers.  It holds none of the solver's arithmetic: it evaluates an
analytic phantom and an analytic field and applies the physical distortion
model (Sec. 2, Eqs. distortionModel and reversedGradient) exactly,

    I(x) = I_v(x + b(x) v) (1 + d_v b(x)) = I_-v(x - b(x) v) (1 - d_v b(x)),

by inverting x -> x +/- b(x) v along each phase-encoding line (monotone while
|d_v b| < 1):  I_v(y) = I(x)/(1 + d_v b(x)) with x + b(x) = y, and
I_-v(y) = I(x)/(1 - d_v b(x)) with x - b(x) = y.  Samples are taken at cell
centres; the field is sampled on the PE faces (Sec. 3, face-staggered grid).

Workloads stand in for the paper's 2D Muenster slice and 3D HCP pair (Sec. 5),
which are not available: Gaussian-ellipse phantoms of the same grid sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    m: tuple                 # cells per axis
    pe: int                  # phase-encoding axis (0-based)
    n_blobs: int
    n_bumps: int
    peak_px: float           # requested field peak in PE voxels
    max_d: float             # bound on max |d_v b|
    sigma: float = 0.0       # noise standard deviation (absolute)
    snr: tuple | None = None  # (lo, hi): sigma = mean foreground / SNR
    rician: bool = False
    bias: bool = False
    unit_range: bool = False  # rescale both images to [0, 1]
    alpha: float = 50.0
    rho: float = 1e2
    seed: int = 0
    bump_width: tuple = (0.06, 0.2)
    extra: dict = field(default_factory=dict)

    @property
    def h(self):
        """Isotropic voxels of edge 1/m[0]: the domain is (0,1) x (0, m1/m0) [x (0, m2/m0)]."""
        return tuple(1.0 / self.m[0] for _ in self.m)

    @property
    def face_shape(self):
        return tuple(mm + (1 if a == self.pe else 0) for a, mm in enumerate(self.m))

    @property
    def n_faces(self):
        return int(np.prod(self.face_shape))


# The workloads measured and tested (shapes of the paper's data, Sec. 5).
WORKLOADS = {
    # 2D, 128 x 128 on [0,1]^2, PE = second axis, 6 ellipses, field of 4 bumps
    # (3 px, |d b| <= 0.6), sigma 0.01, alpha 50, rho 1e2.
    "2d_128": Workload("2d_128", (128, 128), 1, 6, 4, 3.0, 0.6, sigma=0.01, alpha=50.0, seed=1),
    # 3D, 128 x 128 x 64, 12 ellipsoids + smooth bias, 6 bumps (5 px, 0.8), sigma 0.02, alpha 100.
    "3d_128x128x64": Workload("3d_128x128x64", (128, 128, 64), 1, 12, 6, 5.0, 0.8, sigma=0.02,
                              bias=True, alpha=100.0, seed=2),
    # 3D, 256 x 256 x 80 (5 263 360 faces), 20 ellipsoids, Rician 0.02, up to 8 px, 0.9.
    "3d_256x256x80": Workload("3d_256x256x80", (256, 256, 80), 1, 20, 8, 8.0, 0.9, sigma=0.02,
                              rician=True, unit_range=True, alpha=50.0, seed=3,
                              bump_width=(0.012, 0.04)),
}


def batch_workloads(n_pairs: int = 64, m=(96, 96, 60), seed0: int = 400):
    """DTI-like batch: pairs sharing one grid, independent fields (2-6 px peak)
    and per-pair SNR in [10, 40]."""
    out = []
    for k in range(n_pairs):
        rng = np.random.default_rng(seed0 + k)
        peak = float(rng.uniform(2.0, 6.0))
        out.append(Workload(f"batch_{k}", tuple(m), 1, 12, 6, peak, 0.8, snr=(10.0, 40.0),
                            alpha=50.0, seed=seed0 + k))
    return out


SERVING_KINDS = [((128, 128), 1), ((256, 256), 1), ((96, 96, 60), 1), ((128, 128, 64), 1),
                 ((256, 256, 80), 1)]


def serving_workload(kind: int, seed: int) -> Workload:
    m, pe = SERVING_KINDS[kind]
    if len(m) == 2:
        return Workload(f"serve2d_{m[0]}_{seed}", m, pe, 6, 4, 3.0, 0.6, sigma=0.01, alpha=50.0, seed=seed)
    return Workload(f"serve3d_{'x'.join(map(str, m))}_{seed}", m, pe, 12, 6, 5.0, 0.8, sigma=0.02,
                    alpha=50.0, seed=seed)


def small_workload(m, pe=1, seed=0, peak_px=2.0, max_d=0.5, sigma=0.0, n_blobs=4, n_bumps=3,
                   alpha=50.0, rho=1e2) -> Workload:
    """A small grid for tests (any shape; every axis >= 4 cells)."""
    return Workload(f"small_{'x'.join(map(str, m))}_{seed}", tuple(m), pe, n_blobs, n_bumps, peak_px,
                    max_d, sigma=sigma, alpha=alpha, rho=rho, seed=seed)


# --------------------------------------------------------------------------
# analytic phantom and field
# --------------------------------------------------------------------------

class _Numpy:
    """Array operations of the phantom evaluation on numpy arrays."""
    @staticmethod
    def asarray(a, like):
        return np.asarray(a, dtype=np.float64)
    exp = staticmethod(np.exp)
    minimum = staticmethod(np.minimum)
    where = staticmethod(np.where)

    @staticmethod
    def clip(a, lo, hi):
        return np.clip(a, lo, hi)

    @staticmethod
    def zeros(shape, like):
        return np.zeros(shape)

    @staticmethod
    def sum_last(a):
        return np.sum(a, axis=-1)

    @staticmethod
    def max_abs(a):
        return float(np.max(np.abs(a)))


class _Torch:
    """The same operations on torch tensors (float64, any device): the bench
    generates its many large phantoms on the GPU; the seeded parameters and
    the noise still come from numpy, so the pair is the same up to the
    rounding of exp."""
    @staticmethod
    def asarray(a, like):
        import torch
        return torch.as_tensor(np.asarray(a, dtype=np.float64), device=like.device)

    @staticmethod
    def exp(a):
        import torch
        return torch.exp(a)

    @staticmethod
    def minimum(a, b):
        import torch
        return torch.minimum(a, b)

    @staticmethod
    def where(c, a, b):
        import torch
        return torch.where(c, a, b)

    @staticmethod
    def clip(a, lo, hi):
        return a.clamp(lo, hi)

    @staticmethod
    def zeros(shape, like):
        import torch
        return torch.zeros(shape, dtype=torch.float64, device=like.device)

    @staticmethod
    def sum_last(a):
        return a.sum(dim=-1)

    @staticmethod
    def max_abs(a):
        return float(a.abs().max().item())


def _ns(X):
    return _Numpy if isinstance(X, np.ndarray) else _Torch


def _extent(w: Workload):
    return np.array([mm * hh for mm, hh in zip(w.m, w.h)])


def _rotation(rng, nd):
    if nd == 2:
        t = rng.uniform(0, np.pi)
        return np.array([[np.cos(t), -np.sin(t)], [np.sin(t), np.cos(t)]])
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.diag(r))


class _Phantom:
    """Sum of rotated Gaussian ellipse(oid)s, optional smooth multiplicative
    bias, tapered to exactly zero within 2 cells of the boundary (compact
    support, Sec. 2)."""

    def __init__(self, w: Workload, rng):
        nd = len(w.m)
        ext = _extent(w)
        self.nd, self.ext, self.h = nd, ext, np.array(w.h)
        self.c = [rng.uniform(0.25, 0.75, size=nd) * ext for _ in range(w.n_blobs)]
        self.R = [_rotation(rng, nd) for _ in range(w.n_blobs)]
        self.s = [rng.uniform(0.05, 0.2, size=nd) * ext.max() for _ in range(w.n_blobs)]
        self.a = [rng.uniform(0.3, 1.0) for _ in range(w.n_blobs)]
        self.bias = rng.uniform(-0.15, 0.15, size=(nd, 2)) if w.bias else None

    def __call__(self, X):
        """X: (..., nd) points in domain coordinates (numpy or torch)."""
        xp = _ns(X)
        val = xp.zeros(X.shape[:-1], X)
        for c, R, s, a in zip(self.c, self.R, self.s, self.a):
            Y = (X - xp.asarray(c, X)) @ xp.asarray(R, X)
            val += a * xp.exp(-0.5 * xp.sum_last((Y / xp.asarray(s, X)) ** 2))
        if self.bias is not None:
            t = X / xp.asarray(self.ext, X) - 0.5
            val *= 1.0 + xp.sum_last(xp.asarray(self.bias[:, 0], X) * t + xp.asarray(self.bias[:, 1], X) * t * t)
        for a in range(self.nd):
            dist = xp.minimum(X[..., a], self.ext[a] - X[..., a]) / self.h[a]
            s = xp.clip((dist - 2.0) / 4.0, 0.0, 1.0)
            val *= s * s * (3.0 - 2.0 * s)
        return val


class _Field:
    """b(x) = scale * sum_k s_k exp(-|x - c_k|^2 / (2 w_k^2)), physical units."""

    def __init__(self, w: Workload, rng):
        nd = len(w.m)
        ext = _extent(w)
        self.pe = w.pe
        self.c = np.array([rng.uniform(0.3, 0.7, size=nd) * ext for _ in range(w.n_bumps)])
        self.w = np.array([rng.uniform(*w.bump_width) * ext.max() for _ in range(w.n_bumps)])
        self.s = np.array([rng.choice([-1.0, 1.0]) * rng.uniform(0.6, 1.0) for _ in range(w.n_bumps)])
        self.scale = 1.0

    def val_and_dpe(self, X):
        return self.along_pe(X[..., self.pe], self.cross_factors(X))

    def cross_factors(self, X):
        """Per bump, the factor of the Gaussian that does not depend on the PE
        coordinate (fixed along a PE line)."""
        xp = _ns(X)
        out = []
        for c, w, s in zip(self.c, self.w, self.s):
            q = xp.zeros(X.shape[:-1], X)
            for a in range(X.shape[-1]):
                if a != self.pe:
                    q += ((X[..., a] - c[a]) / w) ** 2
            out.append(s * xp.exp(-0.5 * q))
        return out

    def along_pe(self, xpe, fac):
        xp = _ns(xpe)
        v = xp.zeros(xpe.shape, xpe)
        dv = xp.zeros(xpe.shape, xpe)
        for c, w, f in zip(self.c, self.w, fac):
            t = (xpe - c[self.pe]) / w
            e = f * xp.exp(-0.5 * t * t)
            v += e
            dv -= e * t / w
        return self.scale * v, self.scale * dv


def _grid_points(w: Workload, faces: bool, device=None):
    axes = []
    for a, (mm, hh) in enumerate(zip(w.m, w.h)):
        if faces and a == w.pe:
            axes.append(np.arange(mm + 1) * hh)
        else:
            axes.append((np.arange(mm) + 0.5) * hh)
    if device is not None:
        import torch
        G = torch.meshgrid(*[torch.as_tensor(x, dtype=torch.float64, device=device) for x in axes], indexing="ij")
        return torch.stack(G, dim=-1)
    G = np.meshgrid(*axes, indexing="ij")
    return np.stack(G, axis=-1)


def _np(a):
    return a if isinstance(a, np.ndarray) else a.cpu().numpy()


def _invert(field: _Field, X, sign, bmax):
    """Solve x + sign*b(x) = y along the PE coordinate for every point of X
    (X holds y in the PE slot): safeguarded Newton inside the bracket
    [y - bmax, y + bmax]."""
    xp = _ns(X)
    pe = field.pe
    y = X[..., pe] + 0.0
    lo, hi = y - bmax - 1e-12, y + bmax + 1e-12
    Z = X + 0.0
    x = y + 0.0
    fac = field.cross_factors(X)
    tol = 4e-16 * (1.0 + xp.max_abs(y))
    for _ in range(60):
        b, db = field.along_pe(x, fac)
        F = x + sign * b - y
        if xp.max_abs(F) <= tol:
            break
        lo = xp.where(F < 0, x, lo)
        hi = xp.where(F >= 0, x, hi)
        xn = x - F / (1.0 + sign * db)
        bad = ~((xn >= lo) & (xn <= hi))
        x = xp.where(bad, 0.5 * (lo + hi), xn)
    Z[..., pe] = x
    return Z


def make_pair(w: Workload, dtype=np.float64, chunk: int = 1 << 20, device=None):
    """Returns dict(I1, I2, b_true, h, pe, m, peak_px, max_d, sigma) for workload w.

    I1 = I_v (displaced by +b), I2 = I_-v (displaced by -b); b_true on faces in
    physical units.  Everything is a deterministic function of w.seed.  With
    a torch device the forward model is evaluated there (float64; numpy
    arrays are returned either way)."""
    rng = np.random.default_rng(w.seed)
    phantom = _Phantom(w, rng)
    fld = _Field(w, rng)
    # scale the field: peak |b| = peak_px * h_pe, then shrink until max |d_v b| <= max_d
    Xf = _grid_points(w, faces=True, device=device)
    v, dv = fld.val_and_dpe(Xf)
    hpe = w.h[w.pe]
    xp = _ns(v)
    fld.scale = w.peak_px * hpe / max(xp.max_abs(v), 1e-300)
    v, dv = fld.val_and_dpe(Xf)
    Xc = _grid_points(w, faces=False, device=device)
    _, dvc = fld.val_and_dpe(Xc)
    dmax = max(xp.max_abs(dv), xp.max_abs(dvc), float(np.max(np.abs(np.diff(_np(v), axis=w.pe)))) / hpe)
    if dmax > w.max_d:
        fld.scale *= w.max_d / dmax
    b_true = _np(fld.val_and_dpe(Xf)[0])
    bmax = float(np.max(np.abs(b_true))) * 1.001 + 1e-9
    # exact forward model at the cell centres, in chunks
    flat = Xc.reshape(-1, Xc.shape[-1])
    I1 = np.empty(flat.shape[0])
    I2 = np.empty(flat.shape[0])
    if device is not None:
        chunk = max(chunk, 1 << 23)
    for s in range(0, flat.shape[0], chunk):
        X = flat[s:s + chunk]
        for sign, out in ((1.0, I1), (-1.0, I2)):
            Z = _invert(fld, X, sign, bmax)
            _, db = fld.val_and_dpe(Z)
            out[s:s + chunk] = _np(phantom(Z) / (1.0 + sign * db))
    I1 = I1.reshape(w.m)
    I2 = I2.reshape(w.m)
    nrng = np.random.default_rng(w.seed + 1_000_003)
    sigma = w.sigma
    if w.snr is not None:
        fg = _np(phantom(Xc))
        mask = fg > 0.1 * fg.max()
        snr = nrng.uniform(*w.snr)
        sigma = float(fg[mask].mean() / snr)
    if sigma > 0:
        if w.rician:
            I1 = np.abs(I1 + sigma * nrng.normal(size=I1.shape) + 1j * sigma * nrng.normal(size=I1.shape))
            I2 = np.abs(I2 + sigma * nrng.normal(size=I2.shape) + 1j * sigma * nrng.normal(size=I2.shape))
        else:
            I1 = I1 + sigma * nrng.normal(size=I1.shape)
            I2 = I2 + sigma * nrng.normal(size=I2.shape)
    if w.unit_range:
        s = max(I1.max(), I2.max())
        I1 = np.clip(I1 / s, 0.0, 1.0)
        I2 = np.clip(I2 / s, 0.0, 1.0)
    return dict(I1=I1.astype(dtype), I2=I2.astype(dtype), b_true=b_true, h=w.h, pe=w.pe, m=w.m,
                peak_px=float(np.max(np.abs(b_true)) / hpe), max_d=float(min(dmax, w.max_d)),
                sigma=sigma, alpha=w.alpha, rho=w.rho)


def load_pair(name: str, dtype=np.float32):
    """make_pair for a named workload of WORKLOADS, cached as an .npz file in
    the temporary directory (the large phantoms take a minute to generate);
    the cached arrays are those make_pair returns for the same seed."""
    import os
    import tempfile
    w = WORKLOADS[name]
    cache = os.path.join(tempfile.gettempdir(), f"sac_{name}_seed{w.seed}_{np.dtype(dtype).name}.npz")
    if os.path.exists(cache):
        try:
            z = np.load(cache)
            d = {k: z[k] for k in z.files}
            d.update(h=w.h, pe=w.pe, m=w.m, alpha=w.alpha, rho=w.rho, sigma=float(d["sigma"]))
            d["peak_px"], d["max_d"] = float(d["peak_px"]), float(d["max_d"])
            return w, d
        except (OSError, ValueError, KeyError):
            pass
    d = make_pair(w, dtype=dtype)
    try:
        tmp = cache + f".{os.getpid()}.npz"
        np.savez(tmp, I1=d["I1"], I2=d["I2"], b_true=d["b_true"], peak_px=d["peak_px"], max_d=d["max_d"],
                 sigma=d["sigma"])
        os.replace(tmp, cache)
    except OSError:
        pass
    return w, d


def random_images(m, seed, lo=0.0, hi=1.0, zero_border=1):
    """Plain random cell images (uniform in [lo, hi]) with a zero border of
    `zero_border` cells, for unit tests that need generic data."""
    rng = np.random.default_rng(seed)
    I = rng.uniform(lo, hi, size=m)
    if zero_border:
        sl = [slice(None)] * len(m)
        for a in range(len(m)):
            s = list(sl); s[a] = slice(0, zero_border); I[tuple(s)] = 0
            s = list(sl); s[a] = slice(m[a] - zero_border, m[a]); I[tuple(s)] = 0
    return I


def random_field(m, pe, h, seed, max_d=0.5):
    """Random feasible face field with max |D1 b| <= max_d (smooth-ish: a sum
    of a few random cosines), for unit tests."""
    rng = np.random.default_rng(seed)
    fshape = tuple(mm + (1 if a == pe else 0) for a, mm in enumerate(m))
    axes = [np.linspace(0, 1, n) for n in fshape]
    G = np.meshgrid(*axes, indexing="ij")
    b = np.zeros(fshape)
    for _ in range(4):
        k = rng.uniform(0.5, 3.0, size=len(m))
        ph = rng.uniform(0, 2 * math.pi, size=len(m))
        term = np.ones(fshape)
        for a in range(len(m)):
            term = term * np.cos(math.pi * k[a] * G[a] + ph[a])
        b += rng.normal() * term
    d = np.abs(np.diff(b, axis=pe)) / h[pe]
    return b * (max_d / max(d.max(), 1e-300))
