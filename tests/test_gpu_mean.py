"""GPU mean step (Alg. 1 steps 1 and 2a) through the C ABI against the FP64
oracle: zbar by CGLS and the residual measurements y~ = y - A zbar, then
Alg. 2 on y~ (Alg. 1 step 2b).  96 x 64 noisy phantom, 20 frames, 4 coils,
variable-density lines.  Relative NRMSE bound 1e-4 (FP32 path)."""
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
TOL = 1e-4
SPEC = dict(kind="phantom", ny=96, nx=64, q=20, nc=4, rank=3, mask_kind="lines_vd", accel=4.0, noise=0.01)


def nrmse(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (p.y, p.frame_ptr, p.mask, p.smaps))


def host(x):
    return x.cpu().numpy().astype(np.complex128)


def test_mean_step_matches_oracle():
    """Ten CG iterations (tol 0, so neither side can stop early on rounding)."""
    p = synth.make_problem(SPEC, seed=71)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    zbar, ytil, it = s.mean_step(*to_dev(p), tol=0.0, max_iter=10)
    ref = oracle.mean_step(oracle.Operator.from_problem(p), p.y, tol=0.0, maxit=10)
    assert it == ref["iters"] == 10
    assert nrmse(host(zbar), ref["zbar"]) < TOL
    assert nrmse(host(ytil), ref["ytil"]) < TOL
    s.close()


def test_mean_step_paper_stopping_rule():
    """tol 1e-3, at most 10 iterations: the same stopping iteration up to one step
    (the decision compares FP32 and FP64 residual norms against the same bound)."""
    p = synth.make_problem(SPEC, seed=72)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    zbar, ytil, it = s.mean_step(*to_dev(p))
    ref = oracle.mean_step(oracle.Operator.from_problem(p), p.y)
    assert 1 <= it <= 10 and abs(it - ref["iters"]) <= 1
    if it == ref["iters"]:
        assert nrmse(host(zbar), ref["zbar"]) < TOL
    s.close()


def test_altgdmin_on_the_residual_measurements():
    """Alg. 1 step 2b: Alg. 2 on the GPU's y~ matches the oracle's Alg. 2 on the same y~."""
    p = synth.make_problem(SPEC, seed=73)
    y, fp, mask, sm = to_dev(p)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    zbar, ytil, it = s.mean_step(y, fp, mask, sm)
    with pytest.raises(lrccs.LrccsError) as e:
        s.iterate(1)                          # the mean step leaves no solve in the context
    assert e.value.status == lrccs.E_STATE
    s.init(ytil, fp, mask, sm)
    s.iterate(5)
    U, B = s.factors()
    X = host(U @ B.T)
    yt = ytil.cpu().numpy()
    op = oracle.Operator.from_problem(p)
    ref = op.iterate(yt, op.init(yt, rank=p.rank)["U0"], 5, history=True)
    assert nrmse(X, ref["X"][-1]) < TOL
    with pytest.raises(lrccs.LrccsError) as e:
        lrccs.lrccs_mean_step(s.ctx, y, fp, mask, sm, zbar, y)   # y~ may not overwrite y
    assert e.value.status == lrccs.E_INVALID
    s.close()
