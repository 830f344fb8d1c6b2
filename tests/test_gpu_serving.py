"""GPU tests of the serving boundary: admission by free device memory and the
asynchronous tracking calls (Alg. 4 as a request loop) with their tickets."""
import numpy as np
import pytest

from paper_2212_09664_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2212_09664_gb300 import lrccs  # noqa: E402

DEV = torch.device("cuda:0")


def to_dev(p):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (p.y, p.frame_ptr, p.mask, p.smaps))


def test_admission_refuses_a_context_that_does_not_fit():
    """A reserve larger than the device's memory: nothing is allocated and the
    call returns LRCCS_E_ADMISSION; the default reserve admits the context."""
    prm = lrccs.default_params()
    free0 = torch.cuda.mem_get_info(DEV)[0]
    prm.admit_reserve_bytes = float(free0) * 4
    with pytest.raises(lrccs.LrccsError) as ei:
        lrccs.lrccs_create(192, 192, 48, 12, 10, params=prm)
    assert ei.value.status == lrccs.E_ADMISSION
    assert "admission" in str(ei.value)
    ctx = lrccs.lrccs_create(192, 192, 48, 12, 10)
    lrccs.lrccs_destroy(ctx)


@pytest.mark.parametrize("mask_kind", ["lines_vd", "radial"])
def test_async_tracking_matches_the_synchronous_call(mask_kind):
    """Two later mini-batches submitted back to back without a host wait in
    between (tickets), on one context: the images equal, bit for bit, those of
    the blocking call run on a second context from the same subspace."""
    spec = dict(kind="phantom", ny=64, nx=64, q=32, nc=4, rank=3, mask_kind=mask_kind, accel=4.0, spokes=16,
                noise=0.01)
    seq = synth.make_problem(spec, seed=51)
    first = synth.frames(seq, 0, 16)
    parts = [synth.frames(seq, 16, 8), synth.frames(seq, 24, 8)]
    s0 = lrccs.Solver(seq.ny, seq.nx, 16, seq.nc, seq.rank)
    s0.init(*to_dev(first))
    eta = s0.iterate(20, info=True)["eta"]
    U = s0.subspace()
    stream = torch.cuda.Stream(device=DEV)
    a = lrccs.Solver(seq.ny, seq.nx, 8, seq.nc, seq.rank, stream=stream)
    b = lrccs.Solver(seq.ny, seq.nx, 8, seq.nc, seq.rank)
    a.set_subspace(U, eta)
    b.set_subspace(U, eta)
    inputs = [to_dev(p) for p in parts]
    Xa = [torch.empty((8, seq.n), dtype=torch.complex64, device=DEV) for _ in parts]
    Xb = [torch.empty_like(x) for x in Xa]
    torch.cuda.synchronize()
    tickets = [lrccs.lrccs_track_minibatch_async(a.ctx, *inp, 5, False, X) for inp, X in zip(inputs, Xa)]
    for inp, X in zip(inputs, Xb):
        b.track(*inp, t_max=5, X=X)
    for t in tickets:
        lrccs.lrccs_ticket_wait(a.ctx, t)
        assert lrccs.lrccs_ticket_query(a.ctx, t)
    torch.cuda.synchronize()
    for x, y in zip(Xa, Xb):
        assert torch.equal(x, y)
    for s in (s0, a, b):
        s.close()


def test_unknown_ticket_is_refused():
    p = synth.make_problem(dict(kind="phantom", ny=64, nx=64, q=8, nc=2, rank=2, mask_kind="lines_vd", accel=4.0,
                                noise=0.01), seed=52)
    s = lrccs.Solver(p.ny, p.nx, p.q, p.nc, p.rank)
    with pytest.raises(lrccs.LrccsError) as ei:
        lrccs.lrccs_ticket_wait(s.ctx, lrccs.Ticket(5))
    assert ei.value.status == lrccs.E_STATE
    s.close()
