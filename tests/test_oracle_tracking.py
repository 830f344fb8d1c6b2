"""Pins for the oracle's mini-batch subspace tracking (Alg. 4), against facts the
mathematics fixes independently of the oracle's code.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2212_09664_gb300 import synth


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _batches(p, sizes):
    out, s = [], 0
    for c in sizes:
        b = synth.frames(p, s, c)
        s += c
        # FP64 maps: the data were generated with them
        out.append((oracle.Operator.mri(b.ny, b.nx, b.truth["smaps128"], b.idx, b.frame_ptr), b.truth["y128"]))
    return out


def _lowrank_sequence(q=48, seed=21):
    spec = dict(kind="lowrank", ny=32, nx=32, q=q, nc=1, rank=2, mask_kind="lines_uniform",
                n_center=4, n_rand=10)
    p = synth.make_problem(spec, seed=seed)
    # the image-domain subspace of the generator: columns F^H v*_l
    Ustar = np.stack([oracle.dft2(p.truth["V"][:, l].reshape(p.ny, p.nx), +1).reshape(-1)
                      for l in range(p.rank)], 1)
    return p, Ustar


def test_frames_slice_is_consistent():
    """A mini-batch cut from a sequence is the sequence's own frames: its data equal
    the operator applied to the sequence's ground-truth images of those frames."""
    p, Ustar = _lowrank_sequence(q=20)
    b = synth.frames(p, 12, 8)
    op = oracle.Operator.mri(b.ny, b.nx, b.truth["smaps128"], b.idx, b.frame_ptr)
    for k in range(b.q):
        xk = Ustar @ p.truth["B"][:, 12 + k]
        assert rel(op.forward(k, xk), b.truth["y128"][b.nc * b.frame_ptr[k]: b.nc * b.frame_ptr[k + 1]]) < 1e-12
    with pytest.raises(ValueError):
        synth.frames(p, 15, 8)


def test_tracking_from_true_subspace_stays_exact():
    """Noiseless exactly rank-r frames: started at U*, every mini-batch's B-step
    recovers b*_k exactly, the gradient vanishes and U stays at U*, so each
    mini-batch's X equals its ground truth (exact recovery, Sec. III-A)."""
    p, Ustar = _lowrank_sequence()
    bs = _batches(p, [8] * 6)
    # the step size Alg. 2 sets at t = 1 from the spectral initialisation of the first mini-batch
    op0, y0 = bs[0]
    eta = op0.iterate(y0, op0.init(y0, rank=2)["U0"], 1)["eta"]
    res = oracle.track_minibatches(bs, rank=2, t_next=5, U_start=Ustar, eta_start=eta)
    for j, r in enumerate(res):
        Xt = Ustar @ p.truth["B"][:, 8 * j: 8 * (j + 1)]
        assert rel(r["X"], Xt) < 1e-10
        assert oracle.sd(Ustar, r["U"]) < 1e-10
        assert r["eta"] == eta


def test_tracking_repeated_batch_continues_the_iteration():
    """Mini-batches that repeat the same frames make Alg. 4 the GDmin loop of Alg. 2
    continued: U_0 <- the previous FINAL subspace and the step size kept, so three
    mini-batches of 5 iterations equal one 15-iteration solve."""
    p = synth.make_problem(dict(kind="phantom", ny=32, nx=32, q=10, nc=3, rank=2, mask_kind="lines_vd",
                                accel=3.0, noise=0.01), seed=4)
    op = oracle.Operator.mri(p.ny, p.nx, p.truth["smaps128"], p.idx, p.frame_ptr)
    y = p.truth["y128"]
    res = oracle.track_minibatches([(op, y)] * 3, rank=2, t_first=5, t_next=5)
    full = op.iterate(y, op.init(y, rank=2)["U0"], 15, history=True)
    assert rel(res[0]["X"], full["X"][4]) < 1e-12
    assert rel(res[1]["X"], full["X"][9]) < 1e-12
    assert rel(res[2]["X"], full["X"][14]) < 1e-12
    assert oracle.sd(res[2]["U"], full["U"]) < 1e-12
    assert res[2]["eta"] == full["eta"]


def test_tracking_step_size_rule():
    """Kept: every mini-batch uses the step size set at the first mini-batch's t = 1,
    where eta ||grad_1||_2 = eta_c (Alg. 2).  Reset: each mini-batch's own first
    gradient sets it, eta_j ||grad_{j,1}||_2 = eta_c."""
    p = synth.make_problem(dict(kind="phantom", ny=32, nx=32, q=24, nc=3, rank=2, mask_kind="lines_vd",
                                accel=3.0, noise=0.01), seed=6)
    bs = _batches(p, [12, 4, 4, 4])
    keep = oracle.track_minibatches(bs, rank=2, t_first=8, t_next=3)
    assert abs(keep[0]["eta"] * keep[0]["gnorm"][0] - 0.14) < 1e-12
    for r in keep[1:]:
        assert r["eta"] == keep[0]["eta"]
    reset = oracle.track_minibatches(bs, rank=2, t_first=8, t_next=3, reset_eta=True)
    for r in reset:
        assert abs(r["eta"] * r["gnorm"][0] - 0.14) < 1e-12
    assert rel(reset[0]["X"], keep[0]["X"]) < 1e-14          # the first mini-batch is the same solve
    assert len({round(r["eta"], 12) for r in reset}) == len(reset)


def test_tracking_rotation_equivariance():
    """X = U_{t-1} B_t depends on the subspace only: starting the tracking from
    U_0 Q (Q unitary) gives the same images in every mini-batch."""
    p = synth.make_problem(dict(kind="phantom", ny=32, nx=32, q=20, nc=3, rank=3, mask_kind="lines_vd",
                                accel=3.0, noise=0.01), seed=8)
    bs = _batches(p, [8, 4, 4, 4])
    U0 = bs[0][0].init(bs[0][1], rank=3)["U0"]
    Q = synth.random_orthonormal(np.random.default_rng(3), 3, 3)
    a = oracle.track_minibatches(bs, rank=3, t_next=3, U_start=U0, eta_start=0.0)
    b = oracle.track_minibatches(bs, rank=3, t_next=3, U_start=U0 @ Q, eta_start=0.0)
    for ra, rb in zip(a, b):
        assert rel(rb["X"], ra["X"]) < 1e-10
