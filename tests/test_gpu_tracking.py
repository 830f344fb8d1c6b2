"""GPU mini-batch subspace tracking (Alg. 4) through the C ABI: the CUDA path
against the FP64 oracle's tracking of the same mini-batch stream, results that
do not depend on what else runs on the GPU, and checkpoint / resume of the
solver state.

The acquisition is a 96 x 64 noisy phantom (4 coils, rank 3, variable-density
lines, 1% noise): a first mini-batch of 32 frames (init + 70 iterations, Alg. 4
step 1), then mini-batches of 8 frames with 5 iterations each.  Images must
match the oracle within relative NRMSE 1e-4 (the per-iterate FP32 bound)."""
import struct

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
SEQ = dict(kind="phantom", ny=96, nx=64, nc=4, rank=3, mask_kind="lines_vd", accel=4.0, noise=0.01)
FIRST, ALPHA, NB, T_FIRST, T_NEXT = 32, 8, 3, 70, 5


def nrmse(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def sequence(seed):
    p = synth.make_problem(dict(SEQ, q=FIRST + ALPHA * NB), seed=seed)
    return [synth.frames(p, 0, FIRST)] + [synth.frames(p, FIRST + ALPHA * j, ALPHA) for j in range(NB)]


def to_dev(b):
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (b.y, b.frame_ptr, b.mask, b.smaps))


def host(x):
    return x.cpu().numpy().astype(np.complex128)


def solve_first(b, stream=None):
    s = lrccs.Solver(b.ny, b.nx, FIRST, b.nc, b.rank, stream=stream)
    s.init(*to_dev(b))
    s.iterate(T_FIRST)
    return s, s.iterate(0, info=True)["eta"]


def gpu_track(parts, stream=None):
    """Alg. 4 on the GPU: the first mini-batch solved on a q = 32 context, the later
    ones tracked on a q = 8 context that takes over U^(1) and eta.  Returns the
    images of every mini-batch (device tensors, row k = x_k), eta and the contexts."""
    with torch.cuda.stream(stream if stream is not None else torch.cuda.current_stream()):
        first, eta = solve_first(parts[0], stream)
        X = [first.images()]
        mb = lrccs.Solver(parts[0].ny, parts[0].nx, ALPHA, parts[0].nc, parts[0].rank, stream=stream)
        mb.set_subspace(first.subspace(), eta=eta)
        for b in parts[1:]:
            Xj = torch.empty((ALPHA, b.n), dtype=torch.complex64, device=DEV)
            mb.track(*to_dev(b), t_max=T_NEXT, X=Xj)
            X.append(Xj)
    return X, eta, first, mb


def test_tracking_matches_oracle():
    parts = sequence(31)
    X, eta, first, mb = gpu_track(parts)
    torch.cuda.synchronize()
    mb.sync()
    res = oracle.track_minibatches([(oracle.Operator.from_problem(b), b.y) for b in parts], rank=SEQ["rank"],
                                   t_first=T_FIRST, t_next=T_NEXT)
    assert abs(eta - res[0]["eta"]) < 1e-4 * res[0]["eta"]
    errs = [nrmse(host(x).T, r["X"]) for x, r in zip(X, res)]
    assert max(errs) < TOL, "per-mini-batch NRMSE %s" % np.array2string(np.array(errs), precision=2)
    info = mb.iterate(0, info=True)
    assert info["eta"] == eta                 # the first mini-batch's step size stays in force
    assert info["t"] == T_NEXT
    first.close()
    mb.close()


def test_tracking_reset_eta_first_step():
    """reset_eta: the tracked mini-batch's first gradient sets eta = eta_c/||grad||_2;
    X_1 = U_0 B_1 of that mini-batch matches the oracle started from the same U_0."""
    parts = sequence(33)
    X, eta, first, mb = gpu_track(parts[:2])
    U0 = host(mb.subspace())
    b = parts[2]
    Xg = torch.empty((ALPHA, b.n), dtype=torch.complex64, device=DEV)
    inf = mb.track(*to_dev(b), t_max=1, reset_eta=True, X=Xg, info=True)
    r = oracle.Operator.from_problem(b).iterate(b.y, U0, 1, eta=0.0)
    assert abs(inf["eta"] - r["eta"]) < 1e-3 * r["eta"]
    assert inf["eta"] != eta
    assert nrmse(host(Xg).T, r["Uprev"] @ r["B"]) < TOL
    first.close()
    mb.close()


def test_tracking_alone_and_in_mix_are_identical():
    """Two acquisitions tracked one after the other, each alone, and then at the
    same time on two streams with their calls interleaved: bit-identical images."""
    seqs = [sequence(41), sequence(42)]
    alone = []
    for s in seqs:
        X, _, f, m = gpu_track(s, stream=torch.cuda.Stream(device=DEV))
        torch.cuda.synchronize()
        alone.append(X)
        f.close()
        m.close()
    streams = [torch.cuda.Stream(device=DEV) for _ in seqs]
    firsts, mbs, X = [], [], [[], []]
    for s, st in zip(seqs, streams):
        with torch.cuda.stream(st):
            f = lrccs.Solver(s[0].ny, s[0].nx, FIRST, s[0].nc, s[0].rank, stream=st)
            f.init(*to_dev(s[0]))
            f.iterate(T_FIRST)                  # both first solves in flight together
            firsts.append(f)
    for i, (s, st) in enumerate(zip(seqs, streams)):
        with torch.cuda.stream(st):
            X[i].append(firsts[i].images())
            m = lrccs.Solver(s[0].ny, s[0].nx, ALPHA, s[0].nc, s[0].rank, stream=st)
            m.set_subspace(firsts[i].subspace(), eta=firsts[i].iterate(0, info=True)["eta"])
            mbs.append(m)
    for j in range(1, NB + 1):
        for i, st in enumerate(streams):
            with torch.cuda.stream(st):
                Xj = torch.empty((ALPHA, seqs[i][j].n), dtype=torch.complex64, device=DEV)
                mbs[i].track(*to_dev(seqs[i][j]), t_max=T_NEXT, X=Xj)
                X[i].append(Xj)
    torch.cuda.synchronize()
    for i in range(2):
        mbs[i].sync()
        for j, (a, b) in enumerate(zip(alone[i], X[i])):
            assert torch.equal(a, b), "acquisition %d, mini-batch %d" % (i, j)
        firsts[i].close()
        mbs[i].close()


def test_state_round_trip_and_resume():
    parts = sequence(51)
    X, eta, first, mb = gpu_track(parts[:2])
    st = mb.get_state()
    magic, version, ny, nx, r, t = struct.unpack_from("<IIiiii", st, 0)
    assert (version, ny, nx, r, t) == (1, 96, 64, 3, T_NEXT)
    assert struct.unpack_from("<d", st, 32)[0] == eta
    assert len(st) == 64 + 96 * 64 * 3 * 8
    # resume tracking in a fresh context: identical to continuing in the old one
    c = lrccs.Solver(96, 64, ALPHA, 4, 3)
    c.set_state(st)
    Xa = torch.empty((ALPHA, 96 * 64), dtype=torch.complex64, device=DEV)
    Xc = torch.empty_like(Xa)
    mb.track(*to_dev(parts[2]), t_max=T_NEXT, X=Xa)
    c.track(*to_dev(parts[2]), t_max=T_NEXT, X=Xc)
    torch.cuda.synchronize()
    assert torch.equal(Xa, Xc)
    # resume a solve: init the same data, restore U_t, t and eta, iterate on
    a, _ = solve_first(parts[0])
    s10 = a.get_state()
    d = lrccs.Solver(96, 64, FIRST, 4, 3)
    d.init(*to_dev(parts[0]))
    d.set_state(s10)
    a.iterate(5)
    d.iterate(5)
    assert a.iterate(0, info=True)["t"] == d.iterate(0, info=True)["t"] == T_FIRST + 5
    assert nrmse(host(d.images()), host(a.images())) < 1e-5
    for s in (first, mb, c, a, d):
        s.close()


def test_tracking_call_order_and_arguments():
    b = sequence(61)[1]
    s = lrccs.Solver(96, 64, ALPHA, 4, 3)
    with pytest.raises(lrccs.LrccsError) as e:
        s.track(*to_dev(b), t_max=T_NEXT)
    assert e.value.status == lrccs.E_STATE
    with pytest.raises(lrccs.LrccsError) as e:
        s.get_state()
    assert e.value.status == lrccs.E_STATE
    Q = torch.linalg.qr(torch.randn(b.n, 3, dtype=torch.complex128, device=DEV))[0].to(torch.complex64).contiguous()
    with pytest.raises(lrccs.LrccsError) as e:
        lrccs.lrccs_set_subspace(s.ctx, Q, 4, 0.0)          # above this context's rank_max
    assert e.value.status == lrccs.E_INVALID
    with pytest.raises(lrccs.LrccsError) as e:
        lrccs.lrccs_track_minibatch(s.ctx, *to_dev(b), 0)   # t_max < 1
    assert e.value.status == lrccs.E_INVALID
    with pytest.raises(lrccs.LrccsError) as e:
        s.set_state(b"\0" * 200)
    assert e.value.status == lrccs.E_INVALID
    other = lrccs.Solver(64, 64, ALPHA, 4, 3)
    other.set_subspace(Q[: 64 * 64].contiguous())
    with pytest.raises(lrccs.LrccsError) as e:
        s.set_state(other.get_state())                      # another image size
    assert e.value.status == lrccs.E_INVALID
    s.set_subspace(Q)
    with pytest.raises(lrccs.LrccsError) as e:
        s.iterate(1)                                        # a subspace but no data
    assert e.value.status == lrccs.E_STATE
    with pytest.raises(lrccs.LrccsError) as e:
        s.factors()                                         # no factors before an iteration
    assert e.value.status == lrccs.E_STATE
    s.track(*to_dev(b), t_max=2)
    s.sync()
    assert s.iterate(0, info=True)["t"] == 2
    s.close()
    other.close()
    # a fixed rank above q: tracking contexts accept it, the spectral initialisation does not
    wide = lrccs.Solver(96, 64, 4, 4, 5)
    with pytest.raises(lrccs.LrccsError) as e:
        wide.init(*to_dev(synth.frames(sequence(62)[1], 0, 4)))
    assert e.value.status == lrccs.E_INVALID
    wide.close()
