"""GPU parity for general 2D sampling masks (Sec. V: pseudo-radial golden-angle
spokes gridded onto the Cartesian grid, and any mask with partly sampled rows)
against the FP64 oracle, which takes arbitrary sample sets.

Same bars as the line-mask path: the compaction (sample indices) bit-exact,
Z = [A_k^H y_k] and X0 within 1e-5, and every iterate X_t = U_{t-1} B_t within
relative NRMSE 1e-4 of the oracle's.
"""
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

RADIAL = dict(kind="phantom", ny=64, nx=64, q=12, nc=4, rank=3, mask_kind="radial", spokes=16, noise=0.01)


def nrmse(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (p.y, p.frame_ptr, p.mask, p.smaps))


def run_both(p, n_iter, params=None):
    op = oracle.Operator.from_problem(p)
    ini = op.init(p.y, rank=p.rank, want_x0=True)
    it = op.iterate(p.y, ini["U0"], n_iter, params=params, history=True)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    s.init(*to_dev(p))
    X, infos = [], []
    for _ in range(n_iter):
        infos.append(s.iterate(1, info=True))
        U, B = s.factors()
        X.append((U @ B.T).cpu().numpy().astype(np.complex128))
    return op, ini, it, s, X, infos


def check(p, n_iter, params=None):
    op, ini, it, s, X, infos = run_both(p, n_iter, params)
    Z = s.buffer(lrccs.BUF_Z).cpu().numpy()
    Zr = np.stack([op.adjoint(k, p.y_frame(k).reshape(-1)) for k in range(p.q)], 1)
    assert nrmse(Z, Zr) < 1e-5
    assert nrmse(s.buffer(lrccs.BUF_X0).cpu().numpy(), ini["X0"]) < 1e-5
    idx = torch.empty(int(p.frame_ptr[-1]), dtype=torch.int32, device=DEV)
    lrccs.lrccs_get_buffer(s.ctx, lrccs.BUF_IDX, idx)
    assert np.array_equal(idx.cpu().numpy(), p.idx)
    errs = [nrmse(X[t], it["X"][t]) for t in range(n_iter)]
    assert max(errs) < TOL, "per-iterate NRMSE %s" % np.array2string(np.array(errs), precision=2)
    assert abs(infos[0]["eta"] - it["eta"]) < 1e-5 * it["eta"]
    s.close()
    return errs


def test_radial_masks_iterates():
    """64 x 64, q = 12, 4 coils, r = 3, 16 golden-angle spokes per frame: 15 iterations."""
    p = synth.make_problem(RADIAL, seed=31)
    assert (p.mask.reshape(p.q, p.ny, p.nx).sum(2) % p.nx != 0).any()   # rows only partly sampled
    check(p, 15)


def test_one_broken_line_takes_the_general_path():
    """A line mask with one sample removed is a general mask: it is solved, not refused."""
    spec = dict(kind="phantom", ny=64, nx=32, q=10, nc=3, rank=2, mask_kind="lines_vd", accel=3.0, noise=0.01)
    p0 = synth.make_problem(spec, seed=32)
    mask = p0.mask.copy()
    k, i = 0, int(np.flatnonzero(mask[0])[5])
    mask[k, i] = 0
    smaps, modes, coef = synth.coil_maps(np.random.default_rng(33), p0.ny, p0.nx, p0.nc)
    p = synth.assemble("broken", p0.ny, p0.nx, p0.q, p0.nc, p0.rank, 10, mask, p0.truth["spectra"], modes, coef,
                       smaps, np.random.default_rng(34), 0.01, {})
    check(p, 8)


def test_scattered_masks_rectangular_rank_and_ragged():
    """Random 2D sample sets (about 30% density, DC always sampled) of different
    sizes per frame on a 96 x 64 image, 5 coils, r = 4."""
    rng = np.random.default_rng(35)
    ny, nx, q = 96, 64, 10
    mask = np.zeros((q, ny * nx), np.uint8)
    for k in range(q):
        mask[k] = rng.uniform(size=ny * nx) < 0.15 + 0.03 * k
        mask[k, 0] = 1
    spec = dict(kind="phantom", ny=ny, nx=nx, q=q, nc=5, rank=4, mask_kind="full", noise=0.01)
    p0 = synth.make_problem(spec, seed=36)
    smaps, modes, coef = synth.coil_maps(np.random.default_rng(37), ny, nx, 5)
    p = synth.assemble("scatter", ny, nx, q, 5, 4, 10, mask, p0.truth["spectra"], modes, coef, smaps, rng, 0.01, {})
    assert len(set(np.diff(p.frame_ptr))) == q
    check(p, 10)


def test_radial_config3_shape_first_iterates():
    """The precision-form workload's shape on the FP32 FFT path: 256 x 256,
    q = 64, 20 coils, r = 12, 16 golden-angle spokes per frame, contrast ramp.
    Init and the first 2 iterates against the oracle (summed-gradient mode,
    which a CPU pin equates with the literal per-frame adjoint to 1e-12)."""
    p = synth.make_problem("radial256_q64_c20_r12")
    errs = check(p, 2, params=oracle.Params(grad_mode=1))
    assert max(errs) < TOL


def test_mean_step_general_masks():
    """Alg. 1's mean step on radial masks: zbar and y~ against the oracle's CGLS."""
    p = synth.make_problem(RADIAL, seed=38)
    op = oracle.Operator.from_problem(p)
    ref = oracle.mean_step(op, p.y, tol=0.0, maxit=10)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    y, fp, mask, sm = to_dev(p)
    zbar, ytil, it = s.mean_step(y, fp, mask, sm, tol=0.0, max_iter=10)
    assert it == 10
    assert nrmse(zbar.cpu().numpy(), ref["zbar"]) < 1e-4
    assert nrmse(ytil.cpu().numpy(), ref["ytil"]) < 1e-4
    s.close()


def test_graph_replay_general_masks():
    """The captured iteration graph of the general path is bit-identical to
    one-by-one launches."""
    p = synth.make_problem(RADIAL, seed=39)
    stream = torch.cuda.Stream(device=DEV)
    a = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank, stream=stream)
    b = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank, stream=stream)
    inputs = to_dev(p)
    a.init(*inputs)
    b.init(*inputs)
    a.iterate(6)
    for _ in range(6):
        b.iterate(1)
    Ua, Ba = a.factors()
    Ub, Bb = b.factors()
    torch.cuda.synchronize()
    assert torch.equal(Ua, Ub) and torch.equal(Ba, Bb)
    a.close()
    b.close()
