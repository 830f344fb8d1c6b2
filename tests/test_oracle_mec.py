"""Pins for the oracle's model-error correction (Alg. 3): MEC-1 (a few CGLS
iterations per frame) and MEC-2 (ISTA with a sparse temporal spectrum), against
facts the mathematics fixes independently of the oracle's code.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2212_09664_gb300 import synth


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def tiny(seed, mask="scatter", q=4, nc=2, ny=8, nx=8):
    """Random complex coil maps with sum_j |d_j|^2 = 1 per pixel: with these a single
    frame's A_k^H A_k is not a projection (smooth low-order maps can make it one, and
    CG then stops after one step), yet full masks still give A_k^H A_k = I."""
    rng = np.random.default_rng(seed)
    smaps = crandn(rng, nc, ny * nx)
    smaps /= np.sqrt((np.abs(smaps) ** 2).sum(0, keepdims=True))
    if mask == "full":
        m = np.ones((q, ny * nx), np.uint8)
    elif mask == "lines":
        m = synth.cartesian_lines_uniform(rng, ny, nx, q, 2, 2)
    else:
        m = (rng.uniform(size=(q, ny * nx)) < 0.3).astype(np.uint8)
    idx, fp = synth.compact_mask(m)
    return oracle.Operator.mri(ny, nx, smaps, idx, fp), rng


def dense_A(op, k):
    """A_k = [H_k F D_j]_j as an explicit matrix (numpy FFT, no oracle code)."""
    n = op.n
    F = np.fft.fft2(np.eye(n).reshape(n, op.ny, op.nx), norm="ortho").reshape(n, n).T
    sel = op._idx[op._fp[k]:op._fp[k + 1]]
    return np.concatenate([F[sel, :] * op._smaps[j][None, :] for j in range(op.nc)], axis=0)


def frame(op, v, k):
    return v[op.yoff(k): op.yoff(k) + op.rows(k)]


@pytest.mark.parametrize("mask", ["scatter", "lines"])
def test_mec1_is_least_squares_over_the_krylov_space(mask):
    """t CG steps on the normal equations from 0 minimise ||b - A e|| over the Krylov
    space span{g, N g, ..., N^{t-1} g}, g = A^H b, N = A^H A (brute force: an
    orthonormal basis of that space and a small dense least-squares problem)."""
    op, rng = tiny(21, mask)
    ytt = crandn(rng, int(op.nc * op._fp[-1]))
    E = oracle.mec1(op, ytt, iters=3)
    for k in range(op.q):
        Ak, b = dense_A(op, k), frame(op, ytt, k)
        N, g = Ak.conj().T @ Ak, Ak.conj().T @ b
        Kry = np.stack([g, N @ g, N @ (N @ g)], 1)
        Q = np.linalg.qr(Kry)[0]
        c = np.linalg.lstsq(Ak @ Q, b, rcond=None)[0]
        assert rel(E[:, k], Q @ c) < 1e-9


def test_mec1_with_full_sampling_is_the_adjoint():
    """A_k^H A_k = I (full masks, sum_j |d_j|^2 = 1): the first CGLS step is exact, e_k = A_k^H b_k."""
    op, rng = tiny(22, "full", nc=3)
    ytt = crandn(rng, int(op.nc * op._fp[-1]))
    E = oracle.mec1(op, ytt)
    for k in range(op.q):
        assert rel(E[:, k], dense_A(op, k).conj().T @ frame(op, ytt, k)) < 1e-12


def test_soft_threshold():
    M = np.array([3 + 4j, 0.5, -2.0, 1j * 1.0, 0.0])
    out = oracle.soft_threshold(M, 1.0)
    np.testing.assert_allclose(out, [(3 + 4j) * 0.8, 0.0, -1.0, 0.0, 0.0], atol=1e-15)


def test_mec2_with_full_sampling_is_one_shrinkage():
    """A_k^H A_k = I: M_0 = F_t(A^H Y), E_1 = F_t^{-1}(SThr_omega(M_0)), and M_1 = M_0, so
    ISTA stops after one update with that closed form (numpy FFT along time)."""
    op, rng = tiny(23, "full", q=6, nc=2)
    ytt = crandn(rng, int(op.nc * op._fp[-1]))
    out = oracle.mec2(op, ytt)
    AHY = np.stack([dense_A(op, k).conj().T @ frame(op, ytt, k) for k in range(op.q)], 1)
    M0 = np.fft.fft(AHY, axis=1, norm="ortho")
    omega = 0.001 * np.abs(M0).max()
    mag = np.abs(M0)
    ref = np.fft.ifft(np.where(mag > omega, M0 * (1 - omega / np.maximum(mag, 1e-300)), 0), axis=1, norm="ortho")
    assert out["iters"] == 1
    assert abs(out["omega"] - omega) < 1e-15 * omega
    assert rel(out["E"], ref) < 1e-12


def test_mec2_first_step_and_threshold_scale():
    """Scattered masks: the first update is F_t^{-1}(SThr_omega(F_t(A^H Y))) with the
    dense operators, and omega is 0.001 of the largest |M_0|.  The DFT's
    normalisation does not matter: omega scales with M."""
    op, rng = tiny(24, "scatter", q=5, nc=2)
    ytt = crandn(rng, int(op.nc * op._fp[-1]))
    one = oracle.mec2(op, ytt, max_iter=1)
    AHY = np.stack([dense_A(op, k).conj().T @ frame(op, ytt, k) for k in range(op.q)], 1)
    for norm in ("ortho", "backward"):
        M0 = np.fft.fft(AHY, axis=1, norm=norm)
        omega = 0.001 * np.abs(M0).max()
        E1 = np.fft.ifft(oracle.soft_threshold(M0, omega), axis=1, norm=norm)
        assert rel(one["E"], E1) < 1e-12
    assert one["iters"] == 1


def test_mec2_stops_at_ten_or_on_small_change():
    op, rng = tiny(25, "scatter", q=5, nc=2)
    ytt = crandn(rng, int(op.nc * op._fp[-1]))
    out = oracle.mec2(op, ytt)
    assert 1 <= out["iters"] <= 10
    loose = oracle.mec2(op, ytt, rel_change=10.0)     # any change is small: stop at the first check
    assert loose["iters"] == 1


def test_mec2_two_steps_against_dense_ista():
    """Two ISTA updates built from the dense A_k, numpy's FFT along time and a
    separately written soft threshold, with omega fixed at 0.001 max|M_0|."""
    op, rng = tiny(26, "scatter", q=5, nc=2)
    ytt = crandn(rng, int(op.nc * op._fp[-1]))
    As = [dense_A(op, k) for k in range(op.q)]
    Y = [frame(op, ytt, k) for k in range(op.q)]
    E = np.zeros((op.n, op.q), dtype=complex)
    omega = None
    for _ in range(2):
        G = np.stack([E[:, k] + As[k].conj().T @ (Y[k] - As[k] @ E[:, k]) for k in range(op.q)], 1)
        M = np.fft.fft(G, axis=1, norm="ortho")
        if omega is None:
            omega = 0.001 * np.abs(M).max()
        shrunk = np.zeros_like(M)
        big = np.abs(M) > omega
        shrunk[big] = (np.abs(M[big]) - omega) * np.exp(1j * np.angle(M[big]))
        E = np.fft.ifft(shrunk, axis=1, norm="ortho")
    out = oracle.mec2(op, ytt, max_iter=2, rel_change=0.0)
    assert out["iters"] == 2
    assert rel(out["E"], E) < 1e-12
