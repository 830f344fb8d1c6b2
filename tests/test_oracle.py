"""Pins for the FP64 oracle against facts that do not come from the oracle itself.

Every test here runs on the CPU.  Each checks the oracle against something the
paper or the mathematics fixes independently of the oracle's own code: numpy's
FFT/SVD/QR/least squares (different implementations), closed forms (Parseval,
impulses, the adjoint identity), brute force on tiny dense operators, central
finite differences, invariants of Algorithm 2 and the exact-recovery guarantee
(Theorem in Sec. III-A) for Gaussian measurements.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2212_09664_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def small_mri(seed=0, ny=8, nx=8, q=6, nc=3, mask="lines", n_rand=3):
    """Tiny multi-coil problem with random masks and unit-sum-of-squares maps."""
    rng = np.random.default_rng(seed)
    smaps, _, _ = synth.coil_maps(rng, ny, nx, nc)
    if mask == "lines":
        m = synth.cartesian_lines_uniform(rng, ny, nx, q, 2, n_rand)
    elif mask == "full":
        m = np.ones((q, ny * nx), np.uint8)
    else:  # scattered 2D samples
        m = (rng.uniform(size=(q, ny * nx)) < 0.4).astype(np.uint8)
        m[:, 0] = 1
    idx, fp = synth.compact_mask(m)
    return oracle.Operator.mri(ny, nx, smaps, idx, fp), rng


def dense_dft_matrix(ny, nx):
    """Unitary 2D DFT as an explicit n x n matrix, built from numpy's FFT."""
    n = ny * nx
    eye = np.eye(n).reshape(n, ny, nx)
    return np.fft.fft2(eye, norm="ortho").reshape(n, n).T


def dense_A(op, k):
    """A_k = [H_k F D_j]_j built explicitly (numpy FFT, no oracle code)."""
    F = dense_dft_matrix(op.ny, op.nx)
    sel = op._idx[op._fp[k]:op._fp[k + 1]]
    blocks = [F[sel, :] * op._smaps[j][None, :] for j in range(op.nc)]
    return np.concatenate(blocks, axis=0)


# ---------------------------------------------------------------- DFT / operator


@pytest.mark.parametrize("shape", [(8, 16), (12, 10), (64, 64), (6, 7)])
@pytest.mark.parametrize("sign", [-1, +1])
def test_dft_matches_numpy(shape, sign):
    rng = np.random.default_rng(1)
    x = crandn(rng, *shape)
    ref = np.fft.fft2(x, norm="ortho") if sign < 0 else np.fft.ifft2(x, norm="ortho")
    assert rel(oracle.dft2(x, sign), ref) < 1e-13


def test_parseval_and_impulses():
    rng = np.random.default_rng(2)
    ny, nx = 16, 12
    x = crandn(rng, ny, nx)
    assert abs(np.linalg.norm(oracle.dft2(x)) / np.linalg.norm(x) - 1) < 1e-13
    for (a, b) in [(0, 0), (3, 5), (15, 11)]:
        d = np.zeros((ny, nx), complex)
        d[a, b] = 1.0
        ky, kx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        expect = np.exp(-2j * np.pi * (ky * a / ny + kx * b / nx)) / math.sqrt(ny * nx)
        assert np.abs(oracle.dft2(d) - expect).max() < 1e-14


def test_full_sampling_is_isometry():
    """sum_j ||F (d_j o x)||^2 = ||x||^2 when sum_j |d_j|^2 = 1 and all k-space is sampled."""
    op, rng = small_mri(3, ny=8, nx=16, q=2, nc=4, mask="full")
    x = crandn(rng, op.n)
    y = op.forward(0, x)
    assert abs(np.linalg.norm(y) ** 2 / np.linalg.norm(x) ** 2 - 1) < 1e-13
    # and A^H A = I
    assert rel(op.adjoint(0, y), x) < 1e-13


@pytest.mark.parametrize("mask", ["lines", "scatter"])
def test_adjoint_identity(mask):
    op, rng = small_mri(4, ny=16, nx=8, q=4, nc=3, mask=mask)
    for k in range(op.q):
        x = crandn(rng, op.n)
        yv = crandn(rng, op.rows(k))
        lhs = np.vdot(yv, op.forward(k, x))        # <A x, y>
        rhs = np.vdot(op.adjoint(k, yv), x)        # <x, A^H y>
        assert abs(lhs - rhs) / abs(lhs) < 1e-12


@pytest.mark.parametrize("mask", ["lines", "scatter"])
def test_operator_matches_dense_matrix(mask):
    op, rng = small_mri(5, ny=8, nx=8, q=3, nc=2, mask=mask)
    for k in range(op.q):
        A = dense_A(op, k)
        x = crandn(rng, op.n)
        yv = crandn(rng, op.rows(k))
        assert rel(op.forward(k, x), A @ x) < 1e-13
        assert rel(op.adjoint(k, yv), A.conj().T @ yv) < 1e-13


def test_generator_kspace_consistent_with_operator():
    """The generator's shift-and-sum k-space equals A_k applied to F^H zhat_k."""
    p = synth.make_problem(dict(kind="phantom", ny=16, nx=16, q=3, nc=5, rank=2,
                                mask_kind="lines_vd", accel=2.0, noise=0.0), seed=9)
    op = oracle.Operator.mri(p.ny, p.nx, p.truth["smaps128"], p.idx, p.frame_ptr)
    for k in range(p.q):
        z = oracle.dft2(p.truth["spectra"][k].reshape(p.ny, p.nx), +1).reshape(-1)
        yk = p.truth["y128"][p.nc * p.frame_ptr[k]: p.nc * p.frame_ptr[k + 1]]
        assert rel(op.forward(k, z), yk) < 1e-12


# ---------------------------------------------------------------- dense linear algebra


def test_eigh_matches_numpy():
    rng = np.random.default_rng(6)
    for q in (1, 2, 5, 17):
        A = crandn(rng, q, q)
        A = A + A.conj().T
        w, V = oracle.eigh(A)
        assert np.abs(w - np.linalg.eigvalsh(A)[::-1]).max() < 1e-12 * max(1, np.abs(w).max())
        assert np.abs(A @ V - V * w).max() < 1e-12 * max(1, np.abs(w).max())
        assert np.abs(V.conj().T @ V - np.eye(q)).max() < 1e-13


def test_qr_positive_diagonal_is_unique():
    rng = np.random.default_rng(7)
    M = crandn(rng, 30, 6)
    Q, R = oracle.qr(M)
    Qn, Rn = np.linalg.qr(M)
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    Qn = Qn * ph[None, :]
    assert np.abs(Q - Qn).max() < 1e-13
    assert np.all(np.abs(np.imag(np.diag(R))) == 0) and np.all(np.real(np.diag(R)) > 0)
    assert np.abs(Q @ R - M).max() < 1e-13
    assert np.abs(np.tril(R, -1)).max() == 0


def test_lstsq_matches_numpy():
    rng = np.random.default_rng(8)
    M = crandn(rng, 40, 5)
    yv = crandn(rng, 40)
    assert rel(oracle.lstsq(M, yv), np.linalg.lstsq(M, yv, rcond=None)[0]) < 1e-13


# ---------------------------------------------------------------- Alg. 2 steps


def test_bstep_is_pseudo_inverse_solution():
    """b_k = (A_k U)^dagger y_k against an SVD pseudo-inverse of the explicit dense A_k U."""
    op, rng = small_mri(10, ny=8, nx=8, q=5, nc=3, mask="lines")
    r = 2
    U = synth.random_orthonormal(rng, op.n, r)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    B = op.bstep(y, U)
    for k in range(op.q):
        M = dense_A(op, k) @ U
        yk = y[op.yoff(k): op.yoff(k) + op.rows(k)]
        ref = np.linalg.pinv(M) @ yk
        assert rel(B[:, k], ref) < 1e-12
        # normal equations
        res = M @ B[:, k] - yk
        assert np.linalg.norm(M.conj().T @ res) < 1e-12 * np.linalg.norm(M) * np.linalg.norm(yk)


@pytest.mark.parametrize("mask", ["lines", "scatter"])
def test_cost_is_the_residual_norm_with_dense_operators(mask):
    """f(U, B) = sum_k ||y_k - A_k U b_k||^2 with each A_k built explicitly."""
    op, rng = small_mri(13, ny=8, nx=8, q=4, nc=2, mask=mask)
    U = crandn(rng, op.n, 3)
    B = crandn(rng, 3, op.q)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    ref = 0.0
    for k in range(op.q):
        yk = y[op.nc * op._fp[k]: op.nc * op._fp[k + 1]]
        ref += np.linalg.norm(yk - dense_A(op, k) @ (U @ B[:, k])) ** 2
    assert abs(op.cost(y, U, B) - ref) < 1e-12 * ref


def test_subspace_distance_principal_angles():
    """SD(U1, U2) = ||(I - U1 U1^H) U2||_F = ||sin Theta||_F, and
    SD^2 = r - sum_i cos^2 theta_i with cos theta_i the singular values of U1^H U2."""
    rng = np.random.default_rng(14)
    n, r = 40, 3
    U1 = synth.random_orthonormal(rng, n, r)
    U2 = synth.random_orthonormal(rng, n, r)
    cos = np.linalg.svd(U1.conj().T @ U2, compute_uv=False)
    assert abs(oracle.sd(U1, U2) - math.sqrt(r - np.sum(cos ** 2))) < 1e-13
    Q = synth.random_orthonormal(rng, r, r)
    assert oracle.sd(U1, U1 @ Q) < 1e-13                     # same subspace, another basis
    W = synth.random_orthonormal(rng, n, 2 * r)              # two orthogonal subspaces
    assert abs(oracle.sd(W[:, :r], W[:, r:]) - math.sqrt(r)) < 1e-13
    # one basis vector turned by t towards an orthogonal direction: SD = |sin t|
    t = 0.3
    V = W[:, :r].copy()
    V[:, 0] = math.cos(t) * W[:, 0] + math.sin(t) * W[:, r]
    assert abs(oracle.sd(W[:, :r], V) - abs(math.sin(t))) < 1e-13


@pytest.mark.parametrize("mask", ["lines", "scatter"])
def test_gradient_central_differences(mask):
    """(f(U+eD,B) - f(U-eD,B))/2e = 2 Re tr(grad^H D) for f = sum_k ||y_k - A_k U b_k||^2."""
    op, rng = small_mri(11, ny=8, nx=8, q=4, nc=2, mask=mask)
    r = 2
    U = crandn(rng, op.n, r)
    B = crandn(rng, r, op.q)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    G = op.grad(y, U, B)
    for _ in range(3):
        D = crandn(rng, op.n, r)
        e = 1e-4      # f is quadratic in U, so the central difference has no O(e^2) term
        fd = (op.cost(y, U + e * D, B) - op.cost(y, U - e * D, B)) / (2 * e)
        an = 2 * np.real(np.vdot(G, D))
        assert abs(fd - an) / abs(an) < 1e-7


def test_gradient_envelope_on_min_over_B():
    """With B = argmin_B f(U, B), d/de min_B f(U + eD, B) = 2 Re tr(grad^H D) (envelope theorem)."""
    op, rng = small_mri(12, ny=8, nx=8, q=5, nc=2, mask="lines")
    r = 2
    U = crandn(rng, op.n, r)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    B = op.bstep(y, U)
    G = op.grad(y, U, B)
    D = crandn(rng, op.n, r)
    e = 1e-6
    fp_ = op.cost(y, U + e * D, op.bstep(y, U + e * D))
    fm_ = op.cost(y, U - e * D, op.bstep(y, U - e * D))
    an = 2 * np.real(np.vdot(G, D))
    assert abs((fp_ - fm_) / (2 * e) - an) / abs(an) < 1e-6


@pytest.mark.parametrize("mask", ["lines", "scatter"])
def test_gradient_literal_equals_summed(mask):
    op, rng = small_mri(13, ny=16, nx=8, q=5, nc=3, mask=mask)
    r = 3
    U = crandn(rng, op.n, r)
    B = crandn(rng, r, op.q)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    assert rel(op.grad(y, U, B, mode=1), op.grad(y, U, B, mode=0)) < 1e-12


def test_iteration_invariants():
    p = synth.make_problem("lines64_q32_c1_r4")
    op = oracle.Operator.from_problem(p)
    ini = op.init(p.y, rank=p.rank)
    U0 = ini["U0"]
    assert np.abs(U0.conj().T @ U0 - np.eye(p.rank)).max() < 1e-13
    B = op.bstep(p.y, U0)
    G = op.grad(p.y, U0, B)
    # LS optimality: U^H grad = 0
    assert np.linalg.norm(U0.conj().T @ G) / np.linalg.norm(G) < 1e-12
    out = op.iterate(p.y, U0, 3)
    # eta ||grad_1||_2 = 0.14
    assert abs(out["eta"] * out["gnorm"][0] - 0.14) < 1e-12
    assert abs(out["gnorm"][0] - np.linalg.norm(G, 2)) < 1e-12 * out["gnorm"][0]
    U = out["U"]
    assert np.abs(U.conj().T @ U - np.eye(p.rank)).max() < 1e-13
    assert abs(out["sd"][-1] - oracle.sd(out["Uprev"], U)) < 1e-13
    # same three iterations by hand: B-step, gradient, GD, QR
    Uh = U0
    eta = 0.14 / np.linalg.norm(G, 2)
    for _ in range(3):
        Bh = op.bstep(p.y, Uh)
        Gh = op.grad(p.y, Uh, Bh)
        Qn, Rn = np.linalg.qr(Uh - eta * Gh)
        Uh = Qn * (np.diag(Rn) / np.abs(np.diag(Rn)))[None, :]
    assert np.abs(Uh - U).max() < 1e-10


def test_full_sampling_special_case():
    """Full masks, unit-sum-of-squares maps: A^H A = I, so U0 is the SVD of X*
    and one B-step gives b_k = U^H x_k."""
    rng = np.random.default_rng(14)
    ny, nx, q, nc, r = 8, 8, 12, 3, 3
    n = ny * nx
    smaps, _, _ = synth.coil_maps(rng, ny, nx, nc)
    idx, fp = synth.compact_mask(np.ones((q, n), np.uint8))
    op = oracle.Operator.mri(ny, nx, smaps, idx, fp)
    Xs = synth.random_orthonormal(rng, n, r) @ np.diag([3.0, 2.0, 1.0]) @ crandn(rng, r, q)
    y = np.concatenate([op.forward(k, Xs[:, k]) for k in range(q)])
    ini = op.init(y, rank=r, want_x0=True)
    assert rel(ini["X0"], Xs / n) < 1e-12                  # 1/sqrt(m_k mbar) = 1/n
    Ul = np.linalg.svd(Xs)[0][:, :r]
    assert oracle.sd(Ul, ini["U0"]) < 1e-10
    sv = np.linalg.svd(Xs / n, compute_uv=False)
    assert np.abs(ini["sigma"][:r] - sv[:r]).max() < 1e-12 * sv[0]
    U = synth.random_orthonormal(rng, n, r)
    assert rel(op.bstep(y, U), U.conj().T @ Xs) < 1e-12


def test_basic_init_variant():
    """init_kind=1: top-r left singular vectors of [A_k^H y_k], no truncation."""
    op, rng = small_mri(15, ny=8, nx=8, q=10, nc=2, mask="lines")
    y = crandn(rng, int(op.nc * op._fp[-1]))
    y[5] = 50.0                                           # would be truncated by the auto init
    ini = op.init(y, oracle.Params(init_kind=1), rank=2)
    X = np.stack([op.adjoint(k, y[op.yoff(k): op.yoff(k) + op.rows(k)]) for k in range(op.q)], 1)
    assert oracle.sd(np.linalg.svd(X)[0][:, :2], ini["U0"]) < 1e-10


def test_truncation_drops_outliers():
    """gamma = 36 x mean |y|^2 over measured entries; entries above sqrt(gamma) are zeroed (Alg. 2 init)."""
    op, rng = small_mri(16, ny=8, nx=8, q=4, nc=2, mask="lines")
    tot = int(op.nc * op._fp[-1])
    y = np.ones(tot, complex)
    y[3] = 100.0
    ini = op.init(y, rank=1, want_x0=True)
    assert abs(ini["gamma"] - 36.0 * (tot - 1 + 1e4) / tot) < 1e-12 * ini["gamma"]
    yt = y.copy()
    yt[3] = 0.0
    mbar = op._fp[-1] / op.q
    for k in range(op.q):
        xk = op.adjoint(k, yt[op.yoff(k): op.yoff(k) + op.rows(k)]) / math.sqrt(op.m[k] * mbar)
        assert rel(ini["X0"][:, k], xk) < 1e-13


def test_auto_rank_hand_example():
    g = json.load(open(os.path.join(GOLD, "rank_rule_example.json")))
    rng = np.random.default_rng(17)
    ny = nx = 8
    n, q, nc = g["n"], g["q"], g["nc"]
    smaps, _, _ = synth.coil_maps(rng, ny, nx, nc)
    idx, fp = synth.compact_mask(np.ones((q, n), np.uint8))
    op = oracle.Operator.mri(ny, nx, smaps, idx, fp)
    s2 = np.zeros(q)
    s2[: len(g["sigma_sq"])] = g["sigma_sq"]
    s2[len(g["sigma_sq"]):] = 1e-4
    Ul = synth.random_orthonormal(rng, n, q)
    Vr = synth.random_orthonormal(rng, q, q)
    Xs = n * (Ul * np.sqrt(s2)[None, :]) @ Vr.conj().T      # X0 = X*/n has sigma^2 = s2
    y = np.concatenate([op.forward(k, Xs[:, k]) for k in range(q)])
    ini = op.init(y, rank=0)
    assert np.abs(ini["sigma"][:8] ** 2 - np.array(g["sigma_sq"])).max() < 1e-10
    assert ini["rank"] == g["expected_rank"]


def test_paper_constants_are_the_defaults():
    g = json.load(open(os.path.join(GOLD, "paper_constants.json")))
    p = oracle.Params()
    assert p.s.trunc_factor == g["trunc_factor"]["value"]
    assert p.s.energy_pct == g["energy_pct"]["value"]
    assert p.s.eta_c == g["eta_c"]["value"]
    assert p.s.eps_exit == g["eps_exit"]["value"]


# ---------------------------------------------------------------- recovery, invariance


def test_gaussian_exact_recovery():
    """Theorem (Sec. III-A): i.i.d. Gaussian A_k, mq >> (n+q) r^2 -> exact recovery."""
    rng = np.random.default_rng(5)
    n, q, r, m = 100, 50, 2, 40
    Us = synth.random_orthonormal(rng, n, r)
    Bs = crandn(rng, r, q)
    mats = [rng.standard_normal((m, n)) for _ in range(q)]
    op = oracle.Operator.dense(n, mats)
    y = np.concatenate([mats[k] @ (Us @ Bs[:, k]) for k in range(q)])
    ini = op.init(y, rank=r)
    out = op.iterate(y, ini["U0"], 300)
    assert oracle.sd(Us, out["U"]) < 1e-8


def _identifiable_lines_problem():
    spec = dict(kind="lowrank", ny=32, nx=32, q=32, nc=1, rank=2, mask_kind="lines_uniform",
                n_center=4, n_rand=10)
    p = synth.make_problem(spec, seed=11)
    lines = p.mask.reshape(p.q, p.ny, p.nx)[:, :, 0]
    # every line sampled by >= 2r frames -> W*[line] = sum_k b_k b_k^H has full rank
    assert lines.sum(0).min() >= 2 * p.rank
    return p


def test_fourier_exact_recovery_identifiable():
    p = _identifiable_lines_problem()
    op = oracle.Operator.from_problem(p)
    y = p.truth["y128"]
    Ustar = np.stack([oracle.dft2(p.truth["V"][:, l].reshape(p.ny, p.nx), +1).reshape(-1)
                      for l in range(p.rank)], 1)
    ini = op.init(y, rank=p.rank)
    out = op.iterate(y, ini["U0"], 1500)
    assert oracle.sd(Ustar, out["U"]) < 1e-8


def test_scale_invariance():
    """y -> c y scales B by c, grad by |c|^2 and eta by 1/|c|^2: the subspaces U_t are
    unchanged and X_t scales by c (U is defined up to column phases)."""
    p = synth.make_problem("lines64_q32_c1_r4")
    op = oracle.Operator.from_problem(p)
    y = p.y.astype(complex)
    a = op.iterate(y, op.init(y, rank=4)["U0"], 5, history=True)
    c = 3.7 - 1.2j
    b = op.iterate(c * y, op.init(c * y, rank=4)["U0"], 5, history=True)
    assert oracle.sd(a["U"], b["U"]) < 1e-11
    assert rel(b["X"], c * a["X"]) < 1e-11
    assert abs(a["eta"] / b["eta"] - abs(c) ** 2) < 1e-11 * abs(c) ** 2


def test_rotation_equivariance():
    """Starting from U0 Q (Q unitary r x r) leaves X_t = U_{t-1} B_t and SD unchanged."""
    p = synth.make_problem("lines64_q32_c1_r4")
    op = oracle.Operator.from_problem(p)
    U0 = op.init(p.y, rank=4)["U0"]
    Q = synth.random_orthonormal(np.random.default_rng(18), 4, 4)
    a = op.iterate(p.y, U0, 4, history=True)
    b = op.iterate(p.y, U0 @ Q, 4, history=True)
    assert rel(b["X"], a["X"]) < 1e-10
    assert np.abs(a["sd"] - b["sd"]).max() < 1e-10
