"""The allocation-free threshold entry point against the context path.

Some callers of this library cannot allocate device memory (a reconstruction
service that reserves its memory at start-up, or a process whose memory is
owned by another allocator).  For them lrccs_trunc_threshold_noalloc computes
the spectral initialisation's truncation threshold with a fixed scratch array
inside the library.  This file is collected last so that, if it fails, every
other test has already run.
"""
import numpy as np
import pytest

from paper_2212_09664_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2212_09664_gb300 import lrccs  # noqa: E402

DEV = torch.device("cuda:0")


def context_gamma(p):
    """gamma as lrccs_init computes it (the existing entry point)."""
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    s.init(torch.from_numpy(p.y).to(DEV), torch.from_numpy(p.frame_ptr).to(DEV),
           torch.from_numpy(p.mask).to(DEV), torch.from_numpy(p.smaps).to(DEV))
    g = float(s.buffer(lrccs.BUF_SCAL)[0].item())
    s.close()
    return g


@pytest.mark.parametrize("spec", ["cardiac192_q48_c12_r10", "lines64_q32_c1_r4"])
def test_noalloc_threshold_matches_context_path_twice(spec):
    p = synth.make_problem(spec)
    ref = context_gamma(p)
    y = torch.from_numpy(p.y).to(DEV)
    out = torch.full((1,), -1.0, dtype=torch.float64, device=DEV)
    for _ in range(2):                      # two calls in a row share the scratch
        out.fill_(-1.0)
        lrccs.lrccs_trunc_threshold_noalloc(y, y.numel(), 36.0, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * ref, (got, ref)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    """The C entry point refuses a count above its scratch capacity before any
    launch (called directly: the Python wrapper would already refuse a count
    above y.numel())."""
    y = torch.zeros(4, dtype=torch.complex64, device=DEV)
    out = torch.zeros(1, dtype=torch.float64, device=DEV)
    st = lrccs._lib.lrccs_trunc_threshold_noalloc(y.data_ptr(), (1 << 28) + 1, 36.0, out.data_ptr(), None)
    assert st == lrccs.E_INVALID
    assert "outside" in lrccs.lrccs_last_error(None)
    with pytest.raises(ValueError):
        lrccs.lrccs_trunc_threshold_noalloc(y, 5, 36.0, out)
