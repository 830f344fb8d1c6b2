"""GPU tests of the precision forms: the iteration's forward transform (the
DFT along ky of d_j o U on the sampled rows) as a tcgen05 tensor-core GEMM in
BF16X3 (3-term bf16 split products) and FP16S (FP16 with per-tile scaling),
FP32 accumulation (Sec. II-A's operator with F written as a matrix).

Bounds, stated per form:
  * the transform itself against the FP32 FFT path on the same U: relative
    error 1e-5 (BF16X3: ~2^-16 per product term) and 2e-3 (FP16S: 2^-11);
  * the iterates X_t against the FP64 oracle: BF16X3 per-iterate NRMSE 1e-4
    (the FP32 path's bound); FP16S per-iterate NRMSE 2e-3, and the final
    iterate of a 20-iteration solve within 1e-3 (the metric's gate).
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

LINES = dict(kind="phantom", ny=96, nx=64, q=20, nc=4, rank=3, mask_kind="lines_vd", accel=4.0, noise=0.01)
RADIAL = dict(kind="phantom", ny=64, nx=64, q=12, nc=4, rank=3, mask_kind="radial", spokes=16, noise=0.01)
BOUND_T = {lrccs.PREC_BF16X3_GEMM: 1e-5, lrccs.PREC_FP16S_GEMM: 2e-3}
BOUND_X = {lrccs.PREC_BF16X3_GEMM: 1e-4, lrccs.PREC_FP16S_GEMM: 2e-3}
FORMS = [lrccs.PREC_BF16X3_GEMM, lrccs.PREC_FP16S_GEMM]


def nrmse(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (p.y, p.frame_ptr, p.mask, p.smaps))


def used_rows(p):
    return np.flatnonzero(p.mask.reshape(p.q, p.ny, p.nx).any(2).any(0))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("spec", ["lines", "radial", "cardiac"])
def test_gemm_transform_matches_fft(form, spec):
    """The GEMM's T_j = F_y(d_j o U) on the sampled rows against the FP32 FFT
    path's, from the same U_0 (the initialisation is the same in every form)."""
    p = synth.make_problem("cardiac192_q48_c12_r10" if spec == "cardiac" else (LINES if spec == "lines" else RADIAL),
                           seed=61)
    inputs = to_dev(p)
    ref = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank, precision=form)
    ref.init(*inputs)
    s.init(*inputs)
    Tr = torch.zeros((p.nc, p.ny, p.nx * p.rank), dtype=torch.complex64, device=DEV)
    Tg = torch.zeros_like(Tr)
    lrccs.lrccs_forward_transform(ref.ctx, Tr)
    lrccs.lrccs_forward_transform(s.ctx, Tg)
    rows = torch.from_numpy(used_rows(p)).to(DEV)
    a, b = Tg[:, rows].cpu().numpy(), Tr[:, rows].cpu().numpy()
    assert nrmse(a, b) < BOUND_T[form], nrmse(a, b)
    ref.close()
    s.close()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("spec", ["lines", "radial"])
def test_precision_form_iterates_against_oracle(form, spec):
    p = synth.make_problem(LINES if spec == "lines" else RADIAL, seed=62)
    op = oracle.Operator.from_problem(p)
    ini = op.init(p.y, rank=p.rank)
    it = op.iterate(p.y, ini["U0"], 20, history=True)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank, precision=form)
    s.init(*to_dev(p))
    errs = []
    for t in range(20):
        s.iterate(1)
        U, B = s.factors()
        errs.append(nrmse((U @ B.T).cpu().numpy().astype(np.complex128), it["X"][t]))
    assert max(errs) < BOUND_X[form], errs
    assert errs[-1] < 1e-3
    s.close()
