"""Pins for the oracle's mean step (Alg. 1 step 1: CGLS on sum_k ||y_k - A_k z||^2),
against facts the mathematics fixes independently of the oracle's code.  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2212_09664_gb300 import synth


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def tiny(seed, mask="lines", q=4, nc=2, ny=8, nx=8):
    rng = np.random.default_rng(seed)
    smaps, _, _ = synth.coil_maps(rng, ny, nx, nc)
    if mask == "lines":
        m = synth.cartesian_lines_uniform(rng, ny, nx, q, 2, 2)
    elif mask == "full":
        m = np.ones((q, ny * nx), np.uint8)
    else:
        m = (rng.uniform(size=(q, ny * nx)) < 0.3).astype(np.uint8)
    idx, fp = synth.compact_mask(m)
    return oracle.Operator.mri(ny, nx, smaps, idx, fp), rng


def dense_stack(op):
    """[A_1; ...; A_q] as an explicit matrix, each A_k = [H_k F D_j]_j from numpy's FFT."""
    n = op.n
    F = np.fft.fft2(np.eye(n).reshape(n, op.ny, op.nx), norm="ortho").reshape(n, n).T
    blocks = []
    for k in range(op.q):
        sel = op._idx[op._fp[k]:op._fp[k + 1]]
        blocks += [F[sel, :] * op._smaps[j][None, :] for j in range(op.nc)]
    return np.concatenate(blocks, axis=0)


@pytest.mark.parametrize("mask", ["lines", "scatter"])
def test_cgls_reaches_the_minimum_norm_least_squares_solution(mask):
    """Run to convergence, CGLS from z = 0 gives the minimum-norm minimiser, which is
    what numpy's SVD-based lstsq returns for the explicit stacked matrix."""
    op, rng = tiny(3, mask)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    out = oracle.mean_step(op, y, tol=1e-13, maxit=400)
    ref = np.linalg.lstsq(dense_stack(op), y, rcond=None)[0]
    assert rel(out["zbar"], ref) < 1e-9
    assert rel(out["ytil"], y - dense_stack(op) @ ref) < 1e-9


def test_first_cgls_step_is_steepest_descent():
    """z_1 = alpha A^H y with alpha = ||A^H y||^2 / ||A A^H y||^2."""
    op, rng = tiny(4)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    M = dense_stack(op)
    g = M.conj().T @ y
    alpha = np.vdot(g, g).real / np.linalg.norm(M @ g) ** 2
    out = oracle.mean_step(op, y, tol=0.0, maxit=1)
    assert out["iters"] == 1
    assert rel(out["zbar"], alpha * g) < 1e-12


def test_full_sampling_mean_is_the_average_coil_combined_image():
    """Full masks and sum_j |d_j|^2 = 1 give A^H A = q I: one CGLS step reaches
    zbar = (1/q) sum_k A_k^H y_k, the frame average of the coil-combined images."""
    op, rng = tiny(5, "full", q=5, nc=3)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    out = oracle.mean_step(op, y, tol=1e-12, maxit=10)
    avg = sum(op.adjoint(k, y[op.yoff(k): op.yoff(k) + op.rows(k)]) for k in range(op.q)) / op.q
    assert out["iters"] == 1
    assert rel(out["zbar"], avg) < 1e-12


def test_stopping_rule_and_normal_equations():
    """The paper's setting (tol 1e-3, at most 10 iterations) stops at the first t with
    ||A^H r_t|| <= 1e-3 ||A^H y|| or at t = 10; the residual satisfies A^H y~ = A^H r_t."""
    op, rng = tiny(6, "scatter", q=6, nc=2, ny=12, nx=10)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    out = oracle.mean_step(op, y)
    h = out["normal_res"]
    assert out["iters"] <= 10 and len(h) == out["iters"] + 1
    assert out["iters"] == 10 or h[-1] <= 1e-3 * h[0]
    assert all(h[t] > 1e-3 * h[0] for t in range(out["iters"]))
    M = dense_stack(op)
    assert abs(np.linalg.norm(M.conj().T @ out["ytil"]) - h[-1]) < 1e-10 * h[0]


def test_normal_operator_is_the_frame_count_weighted_form():
    """sum_k A_k^H A_k z = sum_j conj(d_j) o F^H[c o F(d_j o z)], c_i = number of frames
    sampling k-space point i: the gradient's summed form with r = 1 and b_k = 1."""
    op, rng = tiny(7, "scatter", q=5, nc=3)
    z = crandn(rng, op.n)
    lhs = sum(op.adjoint(k, op.forward(k, z)) for k in range(op.q))
    cnt = np.zeros(op.n)
    for k in range(op.q):
        cnt[op._idx[op._fp[k]:op._fp[k + 1]]] += 1
    rhs = np.zeros(op.n, dtype=complex)
    for j in range(op.nc):
        Fz = np.fft.fft2((op._smaps[j] * z).reshape(op.ny, op.nx), norm="ortho").reshape(-1)
        rhs += np.conj(op._smaps[j]) * np.fft.ifft2((cnt * Fz).reshape(op.ny, op.nx), norm="ortho").reshape(-1)
    assert rel(lhs, rhs) < 1e-12
