"""GPU tests of the launch-plan autotuner and the batched form (many
independent slices of uneven sizes run as one graph launch)."""
import os
import tempfile

import numpy as np
import pytest

import oracle
from paper_2212_09664_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2212_09664_gb300 import lrccs  # noqa: E402

DEV = torch.device("cuda:0")


def nrmse(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (p.y, p.frame_ptr, p.mask, p.smaps))


SLICES = [
    dict(kind="phantom", ny=96, nx=64, q=20, nc=4, rank=3, mask_kind="lines_vd", accel=4.0, noise=0.01),
    dict(kind="phantom", ny=64, nx=64, q=12, nc=5, rank=4, mask_kind="radial", spokes=14, noise=0.01),
    dict(kind="lowrank", ny=128, nx=96, q=24, nc=6, rank=5, mask_kind="lines_vd", accel=3.0, noise=0.01),
]


def test_autotune_keeps_the_solve_and_caches_the_plan():
    """The tuned plan changes only launch shapes: the iterates stay within
    1e-4 of the oracle's, the state after tuning is the state after init, and a
    second call finds the plan in the cache file."""
    p = synth.make_problem(SLICES[2], seed=71)
    op = oracle.Operator.from_problem(p)
    ini = op.init(p.y, rank=p.rank)
    it = op.iterate(p.y, ini["U0"], 8, history=True)
    with tempfile.TemporaryDirectory() as tmp:
        path = os.path.join(tmp, "plans.txt")
        s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
        inputs = to_dev(p)
        s.init(*inputs)
        plan = lrccs.lrccs_autotune(s.ctx, 3, path)
        assert os.path.exists(path)
        for t in range(8):
            s.iterate(1)
            U, B = s.factors()
            assert nrmse((U @ B.T).cpu().numpy().astype(np.complex128), it["X"][t]) < 1e-4
        s2 = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
        s2.init(*inputs)
        plan2 = lrccs.lrccs_autotune(s2.ctx, 3, path)
        assert (plan2.fwd_tx, plan2.coil_groups, plan2.row_groups) == (plan.fwd_tx, plan.coil_groups,
                                                                       plan.row_groups)
        assert open(path).read().count("\n") == 1
        s.close()
        s2.close()


def test_batch_equals_the_slices_solved_one_by_one():
    """Three uneven slices (line and radial masks) in one batch graph: after
    12 iterations every slice's factors equal, bit for bit, those of the same
    slice iterated on its own."""
    probs = [synth.make_problem(sp, seed=72 + i) for i, sp in enumerate(SLICES)]
    stream = torch.cuda.Stream(device=DEV)
    bs = [lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank, stream=stream) for p in probs]
    ss = [lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank, stream=torch.cuda.Stream(device=DEV)) for p in probs]
    for p, a, b in zip(probs, bs, ss):
        inp = to_dev(p)
        a.init(*inp)
        b.init(*inp)
    batch = lrccs.lrccs_batch_create([a.ctx for a in bs], stream)
    lrccs.lrccs_batch_iterate(batch, 6)
    lrccs.lrccs_batch_iterate(batch, 6)
    for b in ss:
        b.iterate(6)
        b.iterate(6)
    torch.cuda.synchronize()
    for a, b in zip(bs, ss):
        Ua, Ba = a.factors()
        Ub, Bb = b.factors()
        torch.cuda.synchronize()
        assert torch.equal(Ua, Ub) and torch.equal(Ba, Bb)
        assert a.iterate(0, info=True)["t"] == 12
    lrccs.lrccs_batch_destroy(batch)
    for x in bs + ss:
        x.close()
