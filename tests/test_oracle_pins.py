"""Pins of the FP64 CPU oracle to facts fixed outside the oracle itself:
closed forms, the sparsity patterns printed in the paper, library routines,
finite differences, dense brute force and exact invariants of the method.

Paper: Macdonald & Ruthotto, arXiv 1607.00531.  Each test names the passage
it pins.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.fft

import oracle
from paper_1607_00531_gb300 import phantoms as ph

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def grid_of(m, pe, h=None):
    h = h or tuple(1.0 / m[0] for _ in m)
    return oracle.Grid(m, h, pe)


def dense(grid, prm, op, I1, I2, b):
    n = int(np.prod(grid.face_shape))
    A = np.zeros((n, n))
    e = np.zeros(n)
    for k in range(n):
        e[:] = 0
        e[k] = 1
        A[:, k] = oracle.apply(grid, prm, op, I1, I2, b, e.reshape(grid.face_shape)).ravel()
    return A


# ---------------------------------------------------------------- phi (Eqs. P, dphi)

def test_phi_closed_forms_by_finite_differences():
    xs = np.linspace(-0.95, 0.95, 39)
    for x in xs:
        e = 1e-6
        fd1 = (oracle.phi(x + e) - oracle.phi(x - e)) / (2 * e)
        fd2 = (oracle.dphi(x + e) - oracle.dphi(x - e)) / (2 * e)
        assert abs(fd1 - oracle.dphi(x)) <= 1e-6 * max(1.0, abs(fd1))
        assert abs(fd2 - oracle.d2phi(x)) <= 1e-6 * max(1.0, abs(fd2))
    assert oracle.phi(0.0) == 0.0 and oracle.phi(0.5) == pytest.approx(0.0625 / 0.75)
    assert math.isinf(oracle.phi(1.0)) and math.isinf(oracle.phi(-1.2))


# ---------------------------------------------------------------- DCT (Eq. dctdiag)

@pytest.mark.parametrize("m", [1, 2, 5, 8, 13, 64])
def test_dct_matrix_is_scipy_orthonormal_dct2(m):
    C = oracle.dct_matrix(m)
    ref = scipy.fft.dct(np.eye(m), type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(C, ref, atol=1e-14)
    np.testing.assert_allclose(C @ C.T, np.eye(m), atol=1e-13)


@pytest.mark.parametrize("m,h", [(2, 0.5), (7, 0.1), (16, 1 / 16), (33, 0.03)])
def test_dct_diagonalises_neumann_difference_operator(m, h):
    Dt = np.diff(np.eye(m), axis=0) / h          # forward differences, (m-1) x m
    K = Dt.T @ Dt
    C = oracle.dct_matrix(m)
    lam = oracle.dct_eigs(m, h)
    np.testing.assert_allclose(C @ K @ C.T, np.diag(lam), atol=1e-9 * lam.max())
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(K)), np.sort(lam), atol=1e-9 * lam.max())


# ---------------------------------------------------------------- objective (Eqs. D, S, P)

def test_objective_vanishes_for_zero_field_and_identical_images():
    for m, pe in [((12, 9), 1), ((6, 7, 5), 1), ((5, 6, 4), 0), ((5, 4, 6), 2)]:
        g = grid_of(m, pe)
        I = ph.random_images(m, seed=4)
        o = oracle.objective(g, oracle.Params(alpha=3.0, beta=2.0), I, I, np.zeros(g.face_shape))
        assert o["J"] == 0.0 and o["D"] == 0.0 and o["S"] == 0.0 and o["P"] == 0.0


def test_distance_for_whole_voxel_shift_is_sample_difference():
    # b = k h constant: A1 b = k h, D1 b = 0, and the interpolant is exact at
    # the samples, so r_j = I1[j+k] - I2[j-k] with zero outside the line.
    m, pe = (7, 10), 1
    h = (0.1, 0.1)
    g = oracle.Grid(m, h, pe)
    rng = np.random.default_rng(0)
    I1, I2 = rng.uniform(size=m), rng.uniform(size=m)
    for k in (-3, -1, 1, 2, 11):
        b = np.full(g.face_shape, k * h[1])
        D = oracle.objective(g, oracle.Params(alpha=0.0), I1, I2, b)["D"]
        P1 = np.zeros((m[0], m[1] + 40)); P1[:, 20:20 + m[1]] = I1
        P2 = np.zeros((m[0], m[1] + 40)); P2[:, 20:20 + m[1]] = I2
        r = P1[:, 20 + k:20 + k + m[1]] - P2[:, 20 - k:20 - k + m[1]]
        assert D == pytest.approx(0.5 * h[0] * h[1] * np.sum(r * r), rel=1e-13, abs=1e-15)


def test_distance_for_subvoxel_shift_of_a_tent_is_closed_form():
    # piecewise-linear tent with integer knots: the linear interpolant equals it
    m = 24
    h = 1.0 / m
    t0, w = 11, 5
    tent = lambda t: np.maximum(0.0, 1.0 - np.abs(t - t0) / w)
    I = tent(np.arange(m, dtype=float))[None, :].repeat(3, axis=0)
    g = oracle.Grid((3, m), (0.2, h), 1)
    for s in (0.37, -1.6, 2.25):
        b = np.full(g.face_shape, s * h)
        D = oracle.objective(g, oracle.Params(alpha=0.0), I, I, b)["D"]
        j = np.arange(m, dtype=float)
        r = tent(j + s) - tent(j - s)
        assert D == pytest.approx(3 * 0.5 * 0.2 * h * np.sum(r * r), rel=1e-12)


# ---------------------------------------------------------------- corrected images, SSD, NCC (Sec. 6)

def _ncc(a, b):
    return float(np.sum(a * b) ** 2 / (np.sum(a * a) * np.sum(b * b)))


def test_corrected_images_for_zero_field_are_the_inputs():
    # b = 0: A1 b = D1 b = 0 and the interpolant passes through the samples
    for m, pe in [((12, 9), 1), ((6, 7, 5), 1), ((5, 6, 4), 0), ((5, 4, 6), 2)]:
        g = grid_of(m, pe)
        I1, I2 = ph.random_images(m, seed=7), ph.random_images(m, seed=8)
        c = oracle.corrected(g, I1, I2, np.zeros(g.face_shape))
        assert np.array_equal(c["T1"], I1) and np.array_equal(c["T2"], I2)
        hd = float(np.prod(g.h))
        assert c["ssd"] == pytest.approx(0.5 * hd * np.sum((I1 - I2) ** 2), rel=1e-13)
        assert c["ncc"] == pytest.approx(_ncc(I1, I2), rel=1e-13)


def test_corrected_images_for_whole_voxel_shift_are_shifted_samples():
    # b = k h constant: T1[j] = I1[j + k], T2[j] = I2[j - k], zero outside the line
    m, pe = (7, 10), 1
    h = (0.1, 0.1)
    g = oracle.Grid(m, h, pe)
    rng = np.random.default_rng(1)
    I1, I2 = rng.uniform(size=m), rng.uniform(size=m)
    for k in (-3, -1, 1, 2, 11):
        c = oracle.corrected(g, I1, I2, np.full(g.face_shape, k * h[1]))
        P1 = np.zeros((m[0], m[1] + 40)); P1[:, 20:20 + m[1]] = I1
        P2 = np.zeros((m[0], m[1] + 40)); P2[:, 20:20 + m[1]] = I2
        assert np.allclose(c["T1"], P1[:, 20 + k:20 + k + m[1]], rtol=0, atol=1e-15)
        assert np.allclose(c["T2"], P2[:, 20 - k:20 - k + m[1]], rtol=0, atol=1e-15)


def test_corrected_image_for_subvoxel_shift_of_a_tent_is_closed_form():
    m = 24
    h = 1.0 / m
    t0, w = 11, 5
    tent = lambda t: np.maximum(0.0, 1.0 - np.abs(t - t0) / w)
    I = tent(np.arange(m, dtype=float))[None, :].repeat(3, axis=0)
    g = oracle.Grid((3, m), (0.2, h), 1)
    j = np.arange(m, dtype=float)
    for sft in (0.37, -1.6, 2.25):
        c = oracle.corrected(g, I, I, np.full(g.face_shape, sft * h))
        assert np.allclose(c["T1"], tent(j + sft)[None, :], rtol=0, atol=1e-14)
        assert np.allclose(c["T2"], tent(j - sft)[None, :], rtol=0, atol=1e-14)


def test_ssd_is_the_distance_and_the_image_difference_is_the_residual():
    for m, pe in [((9, 16), 1), ((5, 12, 6), 1), ((10, 4, 5), 0), ((4, 5, 14), 2)]:
        g = grid_of(m, pe)
        I1, I2 = ph.random_images(m, seed=11), ph.random_images(m, seed=12)
        b = ph.random_field(m, pe, g.h, seed=13, max_d=0.6)
        c = oracle.corrected(g, I1, I2, b)
        D = oracle.objective(g, oracle.Params(alpha=0.0), I1, I2, b)["D"]
        assert c["ssd"] == pytest.approx(D, rel=1e-12)
        assert np.allclose(c["T1"] - c["T2"], oracle.residual(g, I1, I2, b), rtol=0, atol=1e-13)


def test_ncc_scale_invariance_swap_symmetry_and_optimum():
    m, pe = (6, 11, 5), 1
    g = grid_of(m, pe)
    I1, I2 = ph.random_images(m, seed=21), ph.random_images(m, seed=22)
    b = ph.random_field(m, pe, g.h, seed=23, max_d=0.5)
    c = oracle.corrected(g, I1, I2, b)
    assert 0.0 <= c["ncc"] <= 1.0
    assert oracle.corrected(g, I1, 3.0 * I2, b)["ncc"] == pytest.approx(c["ncc"], rel=1e-12)
    # swapping the images and negating b swaps the transformed images
    s = oracle.corrected(g, I2, I1, -b)
    assert np.allclose(s["T1"], c["T2"], rtol=0, atol=1e-14) and np.allclose(s["T2"], c["T1"], rtol=0, atol=1e-14)
    # proportional transformed images: NCC = 1
    assert oracle.corrected(g, I1, 2.0 * I1, np.zeros(g.face_shape))["ncc"] == pytest.approx(1.0, rel=1e-14)


def test_regulariser_and_penalty_of_linear_ramps():
    m, pe = (6, 8, 5), 1
    h = (0.5, 0.25, 0.2)
    g = oracle.Grid(m, h, pe)
    hd = h[0] * h[1] * h[2]
    Z = np.zeros(m)
    F = g.face_shape
    kappa = 0.4
    # ramp along PE: every cell has D1 b = kappa, no cross-line differences
    b = kappa * h[1] * np.arange(F[1])[None, :, None] * np.ones(F)
    o = oracle.objective(g, oracle.Params(alpha=1.0, beta=3.0), Z, Z, b)
    ncell = np.prod(m)
    assert o["S"] == pytest.approx(0.5 * hd * ncell * kappa ** 2, rel=1e-13)
    assert o["P"] == pytest.approx(3.0 * hd * ncell * kappa ** 4 / (1 - kappa ** 2), rel=1e-13)
    assert o["D"] == 0.0
    # ramp along axis 0 and axis 2 (cross-line): (F_a - 1) * prod(other F) differences
    for a in (0, 2):
        shape = [1, 1, 1]; shape[a] = F[a]
        b = kappa * h[a] * np.arange(F[a]).reshape(shape) * np.ones(F)
        o = oracle.objective(g, oracle.Params(alpha=1.0, beta=3.0), Z, Z, b)
        nd = (F[a] - 1) * np.prod(F) // F[a]
        assert o["S"] == pytest.approx(0.5 * hd * nd * kappa ** 2, rel=1e-13)
        assert o["P"] == 0.0


def test_swap_symmetry_of_objective_and_gradient():
    m, pe = (7, 11, 6), 1
    g = grid_of(m, pe)
    I1, I2 = ph.random_images(m, 1), ph.random_images(m, 2)
    b = ph.random_field(m, pe, g.h, 3, max_d=0.6)
    prm = oracle.Params(alpha=2.0, beta=1.5)
    o1 = oracle.objective(g, prm, I1, I2, b)
    o2 = oracle.objective(g, prm, I2, I1, -b)
    assert o1["J"] == pytest.approx(o2["J"], rel=1e-14)
    g1 = oracle.gradient(g, prm, I1, I2, b)
    g2 = oracle.gradient(g, prm, I2, I1, -b)
    np.testing.assert_allclose(g2, -g1, rtol=1e-13, atol=1e-15 * np.abs(g1).max())


# ---------------------------------------------------------------- derivatives (Sec. 3)

@pytest.mark.parametrize("m,pe", [((9, 13), 1), ((5, 7, 4), 1), ((6, 5, 4), 0), ((4, 5, 7), 2)])
def test_gradient_matches_central_differences(m, pe):
    g = grid_of(m, pe)
    I1, I2 = ph.random_images(m, 11), ph.random_images(m, 12)
    b = ph.random_field(m, pe, g.h, 13, max_d=0.5)
    prm = oracle.Params(alpha=0.7, beta=0.3)
    gr = oracle.gradient(g, prm, I1, I2, b)
    rng = np.random.default_rng(5)
    J = lambda bb: oracle.objective(g, prm, I1, I2, bb)["J"]
    eps = 1e-7 * g.h[pe]
    for _ in range(6):
        v = rng.normal(size=g.face_shape)
        fd = (J(b + eps * v) - J(b - eps * v)) / (2 * eps)
        assert fd == pytest.approx(np.sum(gr * v), rel=2e-6, abs=1e-12)


def test_jacobian_and_gauss_newton_hessian_by_finite_differences():
    m, pe = (3, 6), 1
    g = grid_of(m, pe, h=(0.3, 0.2))
    I1, I2 = ph.random_images(m, 21, zero_border=0), ph.random_images(m, 22, zero_border=0)
    b = ph.random_field(m, pe, g.h, 23, max_d=0.4)
    n = int(np.prod(g.face_shape))
    eps = 1e-7
    Jr = np.zeros((int(np.prod(m)), n))
    for k in range(n):
        e = np.zeros(n); e[k] = eps
        rp = oracle.residual(g, I1, I2, b + e.reshape(g.face_shape)).ravel()
        rm = oracle.residual(g, I1, I2, b - e.reshape(g.face_shape)).ravel()
        Jr[:, k] = (rp - rm) / (2 * eps)
    hd = g.h[0] * g.h[1]
    HD = dense(g, oracle.Params(), "HD", I1, I2, b)
    np.testing.assert_allclose(HD, hd * Jr.T @ Jr, rtol=1e-6, atol=1e-7 * np.abs(HD).max())
    # grad D = h^d J_r^T r
    r = oracle.residual(g, I1, I2, b).ravel()
    gD = oracle.gradient(g, oracle.Params(alpha=0.0, beta=0.0), I1, I2, b).ravel()
    np.testing.assert_allclose(gD, hd * Jr.T @ r, rtol=1e-6, atol=1e-8 * np.abs(gD).max())


def test_sparsity_patterns_match_the_printed_4x4_example():
    # Fig. compare_sparsity (Sec. 3), face-staggered row: 4 x 4 cells, PE index fastest
    g = oracle.Grid((4, 4), (0.25, 0.25), 1)
    I1, I2 = ph.random_images((4, 4), 31, 0.2, 1.0, 0), ph.random_images((4, 4), 32, 0.2, 1.0, 0)
    b = ph.random_field((4, 4), 1, g.h, 33, max_d=0.5) + 1e-3
    prm = oracle.Params(alpha=1.0, beta=1.0)
    for name in ("HD", "lapS", "D1tD1", "D2tD2", "HP"):
        A = dense(g, prm, name, I1, I2, b)
        nz = {(i + 1, j + 1) for i, j in zip(*np.nonzero(np.abs(A) > 1e-12 * np.abs(A).max()))}
        pts = np.loadtxt(os.path.join(GOLDEN, f"sparsity_4x4_{name}.txt"), dtype=int)
        assert nz == {tuple(p) for p in pts}, name


@pytest.mark.parametrize("m,pe,h", [((4, 5), 1, (0.2, 0.3)), ((3, 4, 5), 1, (0.3, 0.25, 0.2)),
                                    ((4, 3, 3), 0, (0.1, 0.2, 0.3))])
def test_regulariser_hessian_spectrum_is_sum_of_1d_neumann_spectra(m, pe, h):
    # grad^2 S = h^d (D1^T D1 + D2^T D2 + D3^T D3): a Kronecker sum of 1D
    # Neumann Laplacians (PE axis on m+1 faces); its eigenvalues are sums.
    g = oracle.Grid(m, h, pe)
    Z = np.zeros(m)
    A = dense(g, oracle.Params(), "lapS", Z, Z, np.zeros(g.face_shape))
    hd = float(np.prod(h))
    one_d = []
    for a, mm in enumerate(m):
        L = mm + 1 if a == pe else mm
        k = np.arange(L)
        one_d.append(4.0 / h[a] ** 2 * np.sin(np.pi * k / (2 * L)) ** 2)
    sums = one_d[0]
    for ev in one_d[1:]:
        sums = (sums[:, None] + ev[None, :]).ravel()
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(hd * sums),
                               atol=1e-10 * hd * sums.max())


def test_block_jacobi_is_the_line_block_diagonal_of_the_gn_hessian():
    # Eq. Pblock (reading: with h^d and gamma it is the block diagonal of H_JGN)
    m, pe = (3, 5, 3), 1
    g = grid_of(m, pe)
    I1, I2 = ph.random_images(m, 41, zero_border=0), ph.random_images(m, 42, zero_border=0)
    b = ph.random_field(m, pe, g.h, 43, max_d=0.5)
    prm = oracle.Params(alpha=0.8, beta=0.5, gamma=1e-3)
    H = dense(g, prm, "HJGN", I1, I2, b)
    P = dense(g, prm, "Pblock", I1, I2, b)
    F = g.face_shape
    idx = np.arange(np.prod(F)).reshape(F)
    line_of = np.zeros(np.prod(F), dtype=int)
    for i0 in range(F[0]):
        for i2 in range(F[2]):
            line_of[idx[i0, :, i2]] = i0 * F[2] + i2
    same = line_of[:, None] == line_of[None, :]
    np.testing.assert_allclose(P[same], H[same], rtol=1e-12, atol=1e-14 * np.abs(H).max())
    assert np.all(P[~same] == 0)
    # and the preconditioner solve inverts it
    rhs = np.random.default_rng(0).normal(size=F)
    x = oracle.precond_solve(g, prm, I1, I2, b, rhs)
    np.testing.assert_allclose(P @ x.ravel(), rhs.ravel(), rtol=1e-10, atol=1e-10)


def test_block_jacobi_clusters_the_spectrum_better_than_jacobi():
    # Sec. 6, spectra of the preconditioned GN Hessian: every preconditioner
    # pulls the spectrum towards 1; Jacobi least, block-Jacobi more
    import scipy.linalg
    m, pe = (12, 12), 1
    g = grid_of(m, pe)
    I1, I2 = ph.random_images(m, 51, zero_border=0), ph.random_images(m, 52, zero_border=0)
    b = ph.random_field(m, pe, g.h, 53, max_d=0.5)
    prm = oracle.Params(alpha=200.0, beta=10.0, gamma=1e-3)
    H = dense(g, prm, "HJGN", I1, I2, b)
    Pb = dense(g, prm, "Pblock", I1, I2, b)
    Pj = np.diag(np.diag(H))
    # Jacobi is the diagonal of H_JGN: the oracle's preconditioner solve agrees
    rhs = np.random.default_rng(1).normal(size=g.face_shape)
    xj = oracle.precond_solve(g, oracle.Params(alpha=200.0, beta=10.0, gamma=1e-3, precond=1), I1, I2, b, rhs)
    np.testing.assert_allclose(xj.ravel(), rhs.ravel() / np.diag(H), rtol=1e-12)

    def cond(P):
        lam = scipy.linalg.eigh(H, P, eigvals_only=True)
        return lam.max() / lam.min()
    k_none, k_jac, k_blk = np.linalg.cond(H), cond(Pj), cond(Pb)
    assert k_blk < k_jac < k_none


# ---------------------------------------------------------------- QP (Eqs. qp, schurasqp)

def _bruteforce_qp(h, Gd, Go, c, dk):
    """Unique minimiser of the strictly convex QP by enumerating working sets
    (free / lower / upper per cell) and checking the KKT conditions."""
    m = len(dk)
    n = m + 1
    G = np.diag(Gd) + np.diag(Go, 1) + np.diag(Go, -1)
    best = None
    for pat in itertools.product((0, -1, 1), repeat=m):
        rows, rhs = [], []
        for j, s in enumerate(pat):
            if s == 0:
                continue
            a = np.zeros(n); a[j + 1], a[j] = 1 / h, -1 / h
            if s < 0:
                rows.append(a); rhs.append(-1 - dk[j])
            else:
                rows.append(-a); rhs.append(-1 + dk[j])
        q = len(rows)
        K = np.zeros((n + q, n + q))
        K[:n, :n] = G
        if q:
            A = np.array(rows)
            K[:n, n:] = -A.T
            K[n:, :n] = A
        sol = np.linalg.solve(K, np.concatenate([-c, rhs]))
        x, lam = sol[:n], sol[n:]
        d = dk + np.diff(x) / h
        if np.all(d >= -1 - 1e-10) and np.all(d <= 1 + 1e-10) and np.all(lam >= -1e-10):
            assert best is None or np.allclose(best, x, atol=1e-9)
            best = x
    return best


@pytest.mark.parametrize("seed", range(12))
def test_line_qp_equals_bruteforce_kkt_point(seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 7))
    h = float(rng.uniform(0.05, 0.5))
    Jd, Ju = rng.normal(size=m), rng.normal(size=m)
    Gd = np.zeros(m + 1); Go = np.zeros(m)
    for j in range(m):
        Gd[j] += Jd[j] ** 2; Gd[j + 1] += Ju[j] ** 2; Go[j] += Jd[j] * Ju[j]
    a = rng.uniform(0.01, 1.0)
    for j in range(m):
        Gd[j] += a / h ** 2; Gd[j + 1] += a / h ** 2; Go[j] -= a / h ** 2
    Gd += rng.uniform(0.01, 0.5)
    c = rng.normal(size=m + 1) * rng.choice([0.1, 10.0, 300.0]) / h
    dk = rng.uniform(-0.95, 0.95, size=m)
    x, passes, _ = oracle.line_qp(h, Gd, Go, c, dk)
    assert passes > 0
    np.testing.assert_allclose(x, _bruteforce_qp(h, Gd, Go, c, dk), atol=1e-9, rtol=1e-8)


# ---------------------------------------------------------------- b-step (Eq. admmStep1)

def _fd_model(g, prm, I1, I2, b, z, u):
    """G and c of the b-step built by finite differences of the residual and
    of the subproblem objective (independent of the oracle's assembly)."""
    n = int(np.prod(g.face_shape))
    hd = float(np.prod(g.h))
    eps = 1e-7
    Jr = np.zeros((int(np.prod(g.m)), n))
    for k in range(n):
        e = np.zeros(n); e[k] = eps
        Jr[:, k] = (oracle.residual(g, I1, I2, b + e.reshape(g.face_shape)).ravel()
                    - oracle.residual(g, I1, I2, b - e.reshape(g.face_shape)).ravel()) / (2 * eps)
    Z = np.zeros(g.m)
    D1tD1 = dense(g, prm, "D1tD1", Z, Z, b)
    G = hd * Jr.T @ Jr + prm.alpha * hd * D1tD1 + prm.rho * hd * np.eye(n)

    def fsub(bb):
        D = oracle.objective(g, oracle.Params(alpha=0.0), I1, I2, bb)["D"]
        return D + 0.5 * prm.alpha * hd * bb.ravel() @ (D1tD1 @ bb.ravel()) \
            + 0.5 * prm.rho * hd * np.sum((bb - z + u) ** 2)
    c = np.zeros(n)
    for k in range(n):
        e = np.zeros(n); e[k] = 1e-7
        c[k] = (fsub(b + e.reshape(g.face_shape)) - fsub(b - e.reshape(g.face_shape))) / 2e-7
    return G, c


def test_bstep_unconstrained_is_the_gauss_newton_step():
    m, pe = (3, 7), 1
    g = grid_of(m, pe, h=(0.2, 0.15))
    I1, I2 = ph.random_images(m, 51, zero_border=0), ph.random_images(m, 52, zero_border=0)
    b = ph.random_field(m, pe, g.h, 53, max_d=0.2)
    z = b + 0.01 * np.random.default_rng(1).normal(size=g.face_shape)
    u = 0.01 * np.random.default_rng(2).normal(size=g.face_shape)
    prm = oracle.Params(alpha=0.05, rho=5.0)
    bn, st = oracle.bstep(g, prm, I1, I2, b, z, u)
    assert st["active"] == 0
    G, c = _fd_model(g, prm, I1, I2, b, z, u)
    x = np.linalg.solve(G, -c)
    np.testing.assert_allclose((bn - b).ravel(), x, rtol=2e-5, atol=2e-6 * np.abs(x).max())


def test_bstep_with_active_constraints_is_the_qp_kkt_point():
    m, pe = (2, 6), 1
    g = grid_of(m, pe, h=(0.3, 0.2))
    I1, I2 = ph.random_images(m, 61, zero_border=0), ph.random_images(m, 62, zero_border=0)
    b = ph.random_field(m, pe, g.h, 63, max_d=0.9)
    z = b + 0.3 * np.random.default_rng(3).normal(size=g.face_shape)
    u = np.zeros(g.face_shape)
    prm = oracle.Params(alpha=0.01, rho=200.0)
    bn, st = oracle.bstep(g, prm, I1, I2, b, z, u)
    assert st["active"] > 0 and st["capped"] == 0
    G, c = _fd_model(g, prm, I1, I2, b, z, u)
    hpe = g.h[pe]
    for line in range(m[0]):
        sl = slice(line * (m[1] + 1), (line + 1) * (m[1] + 1))
        Gl, cl = G[sl, sl], c[sl]
        dk = np.diff(b[line]) / hpe
        xb = _bruteforce_qp(hpe, np.diag(Gl).copy(), np.diag(Gl, 1).copy(), cl, dk)
        np.testing.assert_allclose(bn[line] - b[line], xb, rtol=1e-5, atol=1e-6 * np.abs(xb).max())
    assert oracle.max_abs_d1(g, bn) <= 1 + 1e-12


# ---------------------------------------------------------------- z-step (Eq. admmStep2, dctdiag)

@pytest.mark.parametrize("m,pe,h", [((5, 6), 1, (0.2, 0.2)), ((5, 6, 4), 1, (0.2, 0.25, 0.3)),
                                    ((4, 5, 6), 0, (0.3, 0.2, 0.1)), ((4, 5, 6), 2, (0.3, 0.2, 0.1))])
def test_zstep_is_the_dense_solve(m, pe, h):
    g = oracle.Grid(m, h, pe)
    rng = np.random.default_rng(7)
    b, u = rng.normal(size=g.face_shape), rng.normal(size=g.face_shape)
    prm = oracle.Params(alpha=3.0, rho=0.7)
    Z = np.zeros(m)
    n = int(np.prod(g.face_shape))
    hd = float(np.prod(h))
    A = dense(g, prm, "D2tD2", Z, Z, b) + dense(g, prm, "D3tD3", Z, Z, b)
    Gt = prm.alpha * hd * A + prm.rho * hd * np.eye(n)
    zref = np.linalg.solve(Gt, prm.rho * hd * (b + u).ravel())
    z = oracle.zstep(g, prm, b, u)
    np.testing.assert_allclose(z.ravel(), zref, rtol=1e-12, atol=1e-12 * np.abs(zref).max())


# ---------------------------------------------------------------- ADMM (Sec. 4.2, 4.3)

def test_admm_dual_equals_regulariser_gradient_after_every_iteration():
    # y^{k+1} = grad g(z^{k+1}) (Lemma zdescent): rho u = alpha (D2^T D2 + D3^T D3) z
    m, pe = (8, 10, 6), 1
    w = ph.small_workload(m, pe, seed=5)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    Z = np.zeros(m)
    for k in (1, 2, 5):
        prm = oracle.Params(alpha=2.0, rho=50.0, max_iter=k, eps_abs=0.0, eps_rel=0.0)
        r = oracle.admm(g, prm, d["I1"], d["I2"], np.zeros(g.face_shape))
        lap = oracle.apply(g, prm, "D2tD2", Z, Z, r["z"], r["z"]) + oracle.apply(g, prm, "D3tD3", Z, Z, r["z"], r["z"])
        np.testing.assert_allclose(prm.rho * r["u"], prm.alpha * lap, rtol=1e-9,
                                   atol=1e-11 * np.abs(prm.alpha * lap).max())


def _d1t_d1(g, b):
    """D1^T D1 b from differences along the phase-encoding axis (numpy)."""
    hpe = g.h[g.pe]
    w = np.diff(b, axis=g.pe) / hpe
    pad = [(0, 0)] * b.ndim
    pad[g.pe] = (1, 1)
    return -np.diff(np.pad(w, pad), axis=g.pe) / hpe


def test_admm_stopping_quantities_on_a_quadratic_problem():
    # Eq. admmStop pinned by the optimality of the b-step.  With I1 = I2 = 0
    # the distance vanishes, the b-subproblem alpha/2 h^d |D1 b|^2 + rho/2
    # h^d |b - z^k + u^k|^2 is quadratic (one Gauss-Newton step solves it) and
    # its constraint stays inactive, so
    #   alpha h^d D1^T D1 b^{k+1} + rho h^d (b^{k+1} - z^k + u^k) = 0,
    # and with u^{k+1} = u^k + b^{k+1} - z^{k+1}:
    #   |alpha h^d D1^T D1 b^{k+1} + rho h^d u^{k+1}| = rho h^d |z^{k+1} - z^k|,
    # the dual residual; the primal residual is |b^{k+1} - z^{k+1}|, and the
    # two tolerances are sqrt(n) eps_abs + eps_rel max(|b|, |z|) and
    # sqrt(n) eps_abs + eps_rel |rho h^d u| (Boyd et al. (3.12), scaled form,
    # the paper's h^d-weighted inner product)
    m, pe = (8, 12, 6), 1
    g = grid_of(m, pe)
    hd = float(np.prod(g.h))
    rng = np.random.default_rng(21)
    z0 = 0.02 * g.h[pe] * rng.normal(size=g.face_shape)
    u0 = 0.02 * g.h[pe] * rng.normal(size=g.face_shape)
    Z = np.zeros(m)
    n = z0.size
    prev_z = z0
    for k in range(1, 6):
        prm = oracle.Params(alpha=3.0, rho=40.0, max_iter=k, eps_abs=1e-14, eps_rel=1e-12)
        r = oracle.admm(g, prm, Z, Z, np.zeros(g.face_shape), z0=z0, u0=u0, want_hist=True)
        assert r["iters"] == k
        b, z, u = r["b"], r["z"], r["u"]
        assert oracle.max_abs_d1(g, b) < 0.5
        rp, rd, ep, ed = r["hist"][-1, :4]
        opt = prm.alpha * hd * _d1t_d1(g, b) + prm.rho * hd * u
        assert rd == pytest.approx(np.linalg.norm(opt), rel=1e-9)
        assert rd == pytest.approx(prm.rho * hd * np.linalg.norm(z - prev_z), rel=1e-9)
        assert rp == pytest.approx(np.linalg.norm(b - z), rel=1e-12)
        assert ep == pytest.approx(math.sqrt(n) * 1e-14 + 1e-12 * max(np.linalg.norm(b), np.linalg.norm(z)),
                                   rel=1e-12)
        assert ed == pytest.approx(math.sqrt(n) * 1e-14 + 1e-12 * np.linalg.norm(prm.rho * hd * u), rel=1e-12)
        prev_z = z


def test_admm_primal_residual_vanishes_without_regulariser():
    # alpha = 0: the z-step returns z = b + u (the spectral scale is 1), so
    # u^{k+1} = 0 and r_pri = |b^1 - z^1| = |u^0| after the first iteration,
    # then r_pri = 0 (to rounding) from the second on
    m, pe = (8, 10, 6), 1
    w = ph.small_workload(m, pe, seed=7)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    u0 = 0.05 * g.h[pe] * np.random.default_rng(3).normal(size=g.face_shape)
    prm = oracle.Params(alpha=0.0, rho=30.0, max_iter=4, eps_abs=0.0, eps_rel=0.0)
    r = oracle.admm(g, prm, d["I1"], d["I2"], np.zeros(g.face_shape), u0=u0, want_hist=True)
    hs = r["hist"]
    assert hs[0, 0] == pytest.approx(np.linalg.norm(u0), rel=1e-12)
    scale = np.linalg.norm(r["b"])
    assert np.all(hs[1:, 0] <= 1e-13 * scale)
    assert np.max(np.abs(r["u"])) <= 1e-14 * np.max(np.abs(r["b"]))


def _next_rho(prm, rho, rp, rd):
    # Boyd et al.'s varying penalty, optionally bounded below: rho times tau
    # when the primal residual exceeds mu times the dual one, divided by tau
    # in the opposite case (not below rho_min in the bounded form)
    if rp > prm.rho_mu * rd:
        return rho * prm.rho_tau
    if rd > prm.rho_mu * rp:
        r = rho / prm.rho_tau
        return rho if (prm.adapt_rho == 2 and r < prm.rho_min) else r
    return rho


@pytest.mark.parametrize("mode", [1, 2])
def test_adaptive_rho_sequence_and_rescaled_dual(mode):
    # rho follows the rule from the recorded residuals, and the rescaled dual
    # keeps y = rho u = alpha (D2^T D2 + D3^T D3) z (Lemma zdescent) through
    # every change of rho
    m, pe = (8, 10, 6), 1
    w = ph.small_workload(m, pe, seed=5)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    Z = np.zeros(m)
    for k in (1, 3, 12):
        prm = oracle.Params(alpha=2.0, rho=1e6, max_iter=k, eps_abs=0.0, eps_rel=0.0, adapt_rho=mode,
                            rho_min=1e5)
        r = oracle.admm(g, prm, d["I1"], d["I2"], np.zeros(g.face_shape), want_hist=True)
        hs = r["hist"]
        rho = prm.rho
        for it in range(k):
            assert hs[it, 4] == rho
            rho = _next_rho(prm, rho, hs[it, 0], hs[it, 1])
        if mode == 2:
            assert np.all(hs[:, 4] >= prm.rho_min)
        lap = oracle.apply(g, prm, "D2tD2", Z, Z, r["z"], r["z"]) + oracle.apply(g, prm, "D3tD3", Z, Z, r["z"], r["z"])
        np.testing.assert_allclose(rho * r["u"], prm.alpha * lap, rtol=1e-8,
                                   atol=1e-10 * np.abs(prm.alpha * lap).max())
    # from rho = 1e6 the primal residual is tiny: rho falls by tau per iteration
    # (1e6, 769 230.77, ...) until the bound stops it (mode 2)
    assert hs[1, 4] == pytest.approx(1e6 / 1.3, rel=1e-15)
    if mode == 2:
        assert hs[-1, 4] >= 1e5 and hs[-1, 4] / 1.3 < 1e5


def test_adaptive_rho_that_never_fires_is_the_fixed_method():
    m, pe = (8, 10, 6), 1
    w = ph.small_workload(m, pe, seed=6)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    fixed = oracle.admm(g, oracle.Params(alpha=2.0, rho=50.0, max_iter=6, eps_abs=0.0, eps_rel=0.0),
                        d["I1"], d["I2"], np.zeros(g.face_shape))
    never = oracle.admm(g, oracle.Params(alpha=2.0, rho=50.0, max_iter=6, eps_abs=0.0, eps_rel=0.0, adapt_rho=1,
                                         rho_mu=1e300), d["I1"], d["I2"], np.zeros(g.face_shape))
    assert np.array_equal(fixed["b"], never["b"]) and np.array_equal(fixed["u"], never["u"])


# ---------------------------------------------------------------- multilevel transfer (Sec. 4.4)

@pytest.mark.parametrize("m", [(8, 6), (6, 8, 4)])
def test_restriction_is_the_block_mean(m):
    rng = np.random.default_rng(7)
    Ic = rng.uniform(size=tuple(x // 2 for x in m))
    blocks = Ic
    for a in range(len(m)):
        blocks = np.repeat(blocks, 2, axis=a)
    assert np.allclose(oracle.restrict(m, blocks), Ic, rtol=1e-15, atol=0)   # piecewise constant at the coarse scale
    I = rng.uniform(size=m)
    assert oracle.restrict(m, I).sum() * 2 ** len(m) == pytest.approx(I.sum(), rel=1e-14)
    assert np.allclose(oracle.restrict(m, np.full(m, 0.37)), 0.37, rtol=0, atol=1e-16)


@pytest.mark.parametrize("m,pe", [((8, 6), 1), ((6, 8, 4), 1), ((4, 6, 8), 2), ((8, 4, 6), 0)])
def test_prolongation_keeps_d1_and_linear_fields(m, pe):
    rng = np.random.default_rng(8)
    mc = tuple(x // 2 for x in m)
    gc = oracle.Grid(mc, tuple(0.2 for _ in m), pe)
    gf = oracle.Grid(m, tuple(0.1 for _ in m), pe)
    bc = rng.normal(size=gc.face_shape)
    bf = oracle.prolong(m, pe, bc)
    # along PE: every fine D1 equals the coarse D1 of its coarse cell, for the
    # coarse field averaged across the other axes
    d1c = np.diff(bc, axis=pe) / 0.2
    d1f = np.diff(bf, axis=pe) / 0.1
    pair = np.take(d1f, np.arange(0, d1f.shape[pe], 2), axis=pe)
    assert np.allclose(pair, np.take(d1f, np.arange(1, d1f.shape[pe], 2), axis=pe), rtol=0, atol=1e-12)
    assert oracle.max_abs_d1(gf, bf) <= oracle.max_abs_d1(gc, bc) + 1e-12
    # constants stay constants
    assert np.allclose(oracle.prolong(m, pe, np.full(gc.face_shape, -1.25)), -1.25, rtol=0, atol=1e-15)
    # a field linear along a non-PE axis (cell centres) is reproduced away from that axis' ends
    ax = next(a for a in range(len(m)) if a != pe)
    shape = [1] * len(m); shape[ax] = gc.face_shape[ax]
    xc = ((np.arange(gc.face_shape[ax]) + 0.5) * 0.2).reshape(shape)
    shape[ax] = gf.face_shape[ax]
    xf = ((np.arange(gf.face_shape[ax]) + 0.5) * 0.1).reshape(shape)
    lin = oracle.prolong(m, pe, np.broadcast_to(3.0 * xc + 1.0, gc.face_shape).copy())
    ref = np.broadcast_to(3.0 * xf + 1.0, gf.face_shape)
    inner = [slice(None)] * len(m); inner[ax] = slice(1, -1)
    assert np.allclose(lin[tuple(inner)], ref[tuple(inner)], rtol=0, atol=1e-12)


def test_multilevel_with_one_level_is_plain_admm():
    m, pe = (8, 10, 6), 1
    w = ph.small_workload(m, pe, seed=9)
    d = ph.make_pair(w)
    prm = oracle.Params(alpha=2.0, rho=50.0, max_iter=5, eps_abs=0.0, eps_rel=0.0)
    ml = oracle.multilevel_admm(d["m"], d["h"], pe, prm, d["I1"], d["I2"], levels=1)
    g = oracle.Grid(d["m"], d["h"], pe)
    r = oracle.admm(g, prm, d["I1"], d["I2"], np.zeros(g.face_shape))
    assert np.array_equal(ml[-1]["b"], r["b"])


def test_multilevel_recovers_the_field_and_stays_feasible():
    m, pe = (32, 32), 1
    w = ph.small_workload(m, pe, seed=10, peak_px=2.0, max_d=0.5)
    d = ph.make_pair(w)
    prm = oracle.Params(alpha=0.05, rho=1e3, max_iter=150, eps_abs=0.0, eps_rel=1e-5, adapt_rho=2, rho_min=1e2)
    ml = oracle.multilevel_admm(d["m"], d["h"], pe, prm, d["I1"], d["I2"], levels=3)
    assert [x["m"] for x in ml] == [(8, 8), (16, 16), (32, 32)]
    g = oracle.Grid(d["m"], d["h"], pe)
    assert oracle.max_abs_d1(g, ml[-1]["b"]) <= 1.0
    D0 = oracle.objective(g, oracle.Params(alpha=0.0), d["I1"], d["I2"], np.zeros(g.face_shape))["D"]
    D = oracle.objective(g, oracle.Params(alpha=0.0), d["I1"], d["I2"], ml[-1]["b"])["D"]
    assert D < 0.2 * D0


def test_zstep_decreases_augmented_lagrangian():
    # Lemma zdescent: L(b, z^k, y) - L(b, z^{k+1}, y) >= rho h^d / 2 ||z^k - z^{k+1}||^2
    m, pe = (6, 7, 5), 1
    g = grid_of(m, pe)
    hd = float(np.prod(g.h))
    rng = np.random.default_rng(9)
    b, zk, u = rng.normal(size=g.face_shape), rng.normal(size=g.face_shape), rng.normal(size=g.face_shape)
    prm = oracle.Params(alpha=1.5, rho=4.0)
    Z = np.zeros(m)

    def part(z):
        lap = oracle.apply(g, prm, "D2tD2", Z, Z, z, z) + oracle.apply(g, prm, "D3tD3", Z, Z, z, z)
        gz = 0.5 * prm.alpha * hd * np.sum(z * lap)
        y = prm.rho * hd * u
        return gz + np.sum(y * (b - z)) + 0.5 * prm.rho * hd * np.sum((b - z) ** 2)
    z1 = oracle.zstep(g, prm, b, u)
    assert part(zk) - part(z1) >= 0.5 * prm.rho * hd * np.sum((zk - z1) ** 2) * (1 - 1e-10)


def test_admm_is_odd_under_swapping_the_images():
    m, pe = (10, 12), 1
    w = ph.small_workload(m, pe, seed=6)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    prm = oracle.Params(alpha=1.0, rho=100.0, max_iter=8, eps_abs=0.0, eps_rel=0.0)
    r1 = oracle.admm(g, prm, d["I1"], d["I2"], np.zeros(g.face_shape))
    r2 = oracle.admm(g, prm, d["I2"], d["I1"], np.zeros(g.face_shape))
    np.testing.assert_allclose(r2["b"], -r1["b"], rtol=1e-12, atol=1e-15)


def test_admm_and_gnpcg_reach_the_same_minimiser():
    # beta = 0 and constraints inactive: both solve min J (Sec. 5, "almost identical results")
    m, pe = (12, 16), 1
    w = ph.small_workload(m, pe, seed=7, peak_px=1.5, max_d=0.4)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    alpha = 5.0
    pa = oracle.Params(alpha=alpha, rho=1e2, max_iter=3000, eps_abs=0.0, eps_rel=1e-10)
    ra = oracle.admm(g, pa, d["I1"], d["I2"], np.zeros(g.face_shape))
    assert ra["converged"] and oracle.max_abs_d1(g, ra["b"]) < 0.95
    pg = oracle.Params(alpha=alpha, beta=0.0, eta=1e-6, max_pcg=400, max_gn=60, gn_rel_grad=1e-9)
    rg = oracle.gnpcg(g, pg, d["I1"], d["I2"], np.zeros(g.face_shape))
    rel = np.linalg.norm(ra["b"] - rg["b"]) / np.linalg.norm(rg["b"])
    assert rel < 1e-6, rel
    # and the ADMM point is stationary for J
    gr = oracle.gradient(g, oracle.Params(alpha=alpha), d["I1"], d["I2"], ra["b"])
    g0 = oracle.gradient(g, oracle.Params(alpha=alpha), d["I1"], d["I2"], np.zeros(g.face_shape))
    assert np.linalg.norm(gr) < 1e-7 * np.linalg.norm(g0)


def test_admm_recovers_a_known_field():
    m, pe = (32, 32), 1
    w = ph.small_workload(m, pe, seed=8, peak_px=2.0, max_d=0.5, n_blobs=8)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    prm = oracle.Params(alpha=0.02, rho=1e3, max_iter=400, eps_abs=0.0, eps_rel=1e-6)
    r = oracle.admm(g, prm, d["I1"], d["I2"], np.zeros(g.face_shape))
    bt = d["b_true"]
    # compare where the images carry information (the field is unobservable in the background)
    mask = np.zeros(g.face_shape, dtype=bool)
    inside = (d["I1"] + d["I2"]) > 0.05
    mask[:, :-1] |= inside
    mask[:, 1:] |= inside
    err0 = np.linalg.norm(bt[mask])
    err = np.linalg.norm((r["b"] - bt)[mask])
    assert err < 0.25 * err0, (err, err0)


# ---------------------------------------------------------------- GN-PCG (Sec. 4.1)

def test_pcg_meets_the_forcing_condition_and_gn_descends():
    m, pe = (10, 12, 6), 1
    w = ph.small_workload(m, pe, seed=9)
    d = ph.make_pair(w)
    g = oracle.Grid(d["m"], d["h"], d["pe"])
    prm = oracle.Params(alpha=0.5, beta=10.0, eta=0.1)
    b = np.zeros(g.face_shape)
    grad = oracle.gradient(g, prm, d["I1"], d["I2"], b)
    dvec, its, rel = oracle.pcg(g, prm, d["I1"], d["I2"], b, grad)
    Hd = oracle.apply(g, prm, "HJGN", d["I1"], d["I2"], b, dvec)
    assert np.linalg.norm(grad + Hd) <= 0.1 * np.linalg.norm(grad) * (1 + 1e-9)
    assert np.sum(grad * dvec) < 0
    r = oracle.gnpcg(g, prm, d["I1"], d["I2"], b, want_hist=True)
    Js = r["hist"][:, 0]
    assert np.all(np.diff(Js) <= 0) and Js[0] < oracle.objective(g, prm, d["I1"], d["I2"], b)["J"]
    assert oracle.max_abs_d1(g, r["b"]) < 1


def test_knot32_takes_the_interval_decision_in_fp32():
    # Sec. 3's piecewise-linear image model has a slope that jumps at the
    # knots.  A displacement just below a whole cell in FP64 (1 - 1e-9 cells)
    # rounds to the knot itself in FP32: with knot32 the oracle must then use
    # the interval right of the knot, as it does in FP64 for an exact knot;
    # without it, the interval left of the knot (a different gradient).
    m, pe = (8, 2), 0
    h = (1.0 / 8, 1.0 / 8)
    g = oracle.Grid(m, h, pe)
    rng = np.random.default_rng(11)
    I1 = rng.uniform(0.2, 1.0, size=m)
    I2 = rng.uniform(0.2, 1.0, size=m)
    below = np.full((9, 2), (1.0 - 1e-9) * h[0])   # positions j + 1 - 1e-9
    at = np.full((9, 2), 1.0 * h[0])               # positions exactly j + 1
    p64 = oracle.Params(alpha=0.3)
    p32 = oracle.Params(alpha=0.3, knot32=1)
    g_at = oracle.gradient(g, p64, I1, I2, at)
    g_below64 = oracle.gradient(g, p64, I1, I2, below)
    g_below32 = oracle.gradient(g, p32, I1, I2, below)
    scale = np.abs(g_at).max()
    assert np.abs(g_below32 - g_at).max() <= 1e-6 * scale
    assert np.abs(g_below64 - g_at).max() >= 1e-2 * scale
    # away from knots the two forms agree to FP32 position rounding
    mid = np.full((9, 2), 0.37 * h[0])
    assert np.allclose(oracle.gradient(g, p32, I1, I2, mid), oracle.gradient(g, p64, I1, I2, mid), rtol=1e-5,
                       atol=1e-6 * scale)
