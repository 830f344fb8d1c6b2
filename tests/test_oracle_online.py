"""Pins for the oracle's online subspace tracking step (Alg. 5 step 2) against
facts the mathematics fixes independently of the oracle's code.  CPU only."""
import math

import numpy as np

import oracle
from paper_2212_09664_gb300 import synth


def crandn(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def setup(seed, q=5, nc=2, ny=8, nx=8, r=2):
    rng = np.random.default_rng(seed)
    smaps = crandn(rng, nc, ny * nx)
    smaps /= np.sqrt((np.abs(smaps) ** 2).sum(0, keepdims=True))
    m = (rng.uniform(size=(q, ny * nx)) < 0.4).astype(np.uint8)
    idx, fp = synth.compact_mask(m)
    op = oracle.Operator.mri(ny, nx, smaps, idx, fp)
    return op, rng, synth.random_orthonormal(rng, ny * nx, r)


def dense_A(op, k):
    n = op.n
    F = np.fft.fft2(np.eye(n).reshape(n, op.ny, op.nx), norm="ortho").reshape(n, n).T
    sel = op._idx[op._fp[k]:op._fp[k + 1]]
    return np.concatenate([F[sel, :] * op._smaps[j][None, :] for j in range(op.nc)], axis=0)


def frame(op, v, k):
    return v[op.yoff(k): op.yoff(k) + op.rows(k)]


def test_exact_frames_are_recovered_exactly():
    """y_k = A_k (zbar* + U* b*_k): the B-step returns b*_k, the residual vanishes,
    e_k = 0 and x_k = zbar* + U* b*_k."""
    op, rng, U = setup(31)
    zbar = crandn(rng, op.n)
    Bs = crandn(rng, U.shape[1], op.q)
    X = zbar[:, None] + U @ Bs
    y = np.concatenate([dense_A(op, k) @ X[:, k] for k in range(op.q)])
    out = oracle.online_frames(op, y, zbar, U)
    assert rel(out["B"], Bs) < 1e-10
    assert np.linalg.norm(out["E"]) < 1e-10 * np.linalg.norm(X)
    assert rel(out["X"], X) < 1e-10


def test_b_step_and_residual_reduction():
    """b_k is the least-squares solution of ||y_k - A_k zbar - A_k U b|| (numpy
    lstsq on the dense A_k U), and the MEC-1 correction lowers each frame's residual."""
    op, rng, U = setup(32)
    zbar = crandn(rng, op.n)
    y = crandn(rng, int(op.nc * op._fp[-1]))
    out = oracle.online_frames(op, y, zbar, U)
    for k in range(op.q):
        Ak = dense_A(op, k)
        ytil = frame(op, y, k) - Ak @ zbar
        b = np.linalg.lstsq(Ak @ U, ytil, rcond=None)[0]
        assert rel(out["B"][:, k], b) < 1e-10
        before = np.linalg.norm(ytil - Ak @ (U @ b))
        after = np.linalg.norm(frame(op, y, k) - Ak @ out["X"][:, k])
        assert after < before
