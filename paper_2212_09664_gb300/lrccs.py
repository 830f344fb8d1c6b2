"""Thin ctypes binding of liblrccs (include/lrccs.h).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  Tensors are torch CUDA tensors (torch is used for device memory and
streams); each function has the same name as the C entry point it calls.
There is no CPU fallback: if the shared library cannot be loaded, importing
this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrccs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        "liblrccs.so is not built (%s); run `python -c \"import __graft_entry__ as g; g.build()\"`" % LIB_PATH)

_lib = C.CDLL(LIB_PATH)

# status codes (lrccs_status)
OK, E_INVALID, E_NOMEM, E_CUDA, E_RANK_DEFICIENT, E_TIMEOUT, E_ADMISSION, E_STATE, E_UNSUPPORTED = range(9)
BUF_Z, BUF_X0, BUF_GRAD, BUF_SIGMA, BUF_IDX, BUF_SCAL = range(6)
PREC_FP32_FFT, PREC_BF16X3_GEMM, PREC_FP16S_GEMM = range(3)


class Dims(C.Structure):
    _fields_ = [("ny", C.c_int32), ("nx", C.c_int32), ("q", C.c_int32), ("ncoil", C.c_int32),
                ("rank", C.c_int32), ("rank_max", C.c_int32), ("precision", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("trunc_factor", C.c_double), ("energy_pct", C.c_double), ("eta_c", C.c_double),
                ("eps_exit", C.c_double), ("t_max", C.c_int32), ("exit_enabled", C.c_int32),
                ("admit_reserve_bytes", C.c_double), ("exit_patience", C.c_int32), ("reserved", C.c_int32),
                ("eta_scale0", C.c_double), ("eta_decay", C.c_double)]


class Plan(C.Structure):
    _fields_ = [("fwd_tx", C.c_int32), ("coil_groups", C.c_int32), ("row_groups", C.c_int32),
                ("bstep_form", C.c_int32)]


class Ticket(C.Structure):
    _fields_ = [("id", C.c_uint64)]


class IterInfo(C.Structure):
    _fields_ = [("t", C.c_int32), ("exited", C.c_int32), ("eta", C.c_double), ("sd", C.c_double),
                ("gnorm", C.c_double)]


class KernelStat(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_int64), ("timed", C.c_int64), ("ms", C.c_double)]


_vp = C.c_void_p
_st = C.c_int
_sig = {
    "lrccs_default_params": (None, [C.POINTER(Params)]),
    "lrccs_create": (_st, [C.POINTER(Dims), C.POINTER(Params), _vp, C.POINTER(_vp)]),
    "lrccs_init": (_st, [_vp, _vp, _vp, _vp, _vp, C.POINTER(C.c_int32)]),
    "lrccs_iterate": (_st, [_vp, C.c_int32, C.POINTER(IterInfo)]),
    "lrccs_get_factors": (_st, [_vp, _vp, _vp]),
    "lrccs_get_subspace": (_st, [_vp, _vp]),
    "lrccs_get_images": (_st, [_vp, _vp]),
    "lrccs_get_buffer": (_st, [_vp, C.c_int, _vp, C.c_size_t]),
    "lrccs_synchronize": (_st, [_vp]),
    "lrccs_profile": (_st, [_vp, C.c_char_p]),
    "lrccs_profile_read": (_st, [_vp, C.POINTER(KernelStat), C.c_int32, C.POINTER(C.c_int32)]),
    "lrccs_profile_reset": (_st, [_vp]),
    "lrccs_trunc_threshold_noalloc": (_st, [_vp, C.c_int64, C.c_double, _vp, _vp]),
    "lrccs_set_subspace": (_st, [_vp, _vp, C.c_int32, C.c_double]),
    "lrccs_mean_step": (_st, [_vp, _vp, _vp, _vp, _vp, C.c_double, C.c_int32, _vp, _vp, C.POINTER(C.c_int32)]),
    "lrccs_track_minibatch": (_st, [_vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, _vp, C.POINTER(IterInfo)]),
    "lrccs_get_state": (_st, [_vp, _vp, C.POINTER(C.c_size_t)]),
    "lrccs_set_state": (_st, [_vp, C.c_char_p, C.c_size_t]),
    "lrccs_test_wait_timeout": (_st, [_vp, C.c_int32]),
    "lrccs_gdqr_phases": (_st, [_vp, C.c_int32, C.POINTER(C.c_double)]),
    "lrccs_bstep_phases": (_st, [_vp, C.POINTER(C.c_double)]),
    "lrccs_forward_transform": (_st, [_vp, _vp, C.c_size_t]),
    "lrccs_set_plan": (_st, [_vp, C.c_void_p]),
    "lrccs_get_plan": (_st, [_vp, C.c_void_p]),
    "lrccs_autotune": (_st, [_vp, C.c_int32, C.c_char_p, C.c_void_p]),
    "lrccs_batch_create": (_st, [C.c_void_p, C.c_int32, _vp, C.POINTER(_vp)]),
    "lrccs_batch_iterate": (_st, [_vp, C.c_int32]),
    "lrccs_batch_destroy": (None, [_vp]),
    "lrccs_context_bytes": (_st, [C.c_void_p, C.POINTER(C.c_size_t)]),
    "lrccs_track_minibatch_async": (_st, [_vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, _vp, C.c_void_p]),
    "lrccs_ticket_query": (_st, [_vp, C.c_void_p, C.POINTER(C.c_int32)]),
    "lrccs_ticket_wait": (_st, [_vp, C.c_void_p]),
    "lrccs_mec1": (_st, [_vp, C.c_int32, _vp, _vp, _vp]),
    "lrccs_mec2": (_st, [_vp, C.c_int32, C.c_double, C.c_double, _vp, _vp, _vp, C.POINTER(C.c_int32)]),
    "lrccs_online_frames": (_st, [_vp, _vp, _vp, _vp, _vp, _vp, C.c_int32, _vp, _vp]),
    "lrccs_destroy": (None, [_vp]),
    "lrccs_last_error": (C.c_char_p, [_vp]),
    "lrccs_status_string": (C.c_char_p, [_st]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class LrccsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("lrccs status %d (%s): %s" % (
            status, _lib.lrccs_status_string(status).decode(), msg))
        self.status = status


def _check(ctx, st):
    if st != OK:
        raise LrccsError(st, (_lib.lrccs_last_error(ctx) or b"").decode())


def _ptr(t):
    """Device pointer of a contiguous CUDA tensor (no copies are made here)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def default_params() -> Params:
    p = Params()
    _lib.lrccs_default_params(C.byref(p))
    return p


def lrccs_context_bytes(ny, nx, q, ncoil, rank, rank_max=0, precision=PREC_FP32_FFT) -> int:
    d = Dims(ny, nx, q, ncoil, rank, rank_max, precision)
    b = C.c_size_t(0)
    _check(None, _lib.lrccs_context_bytes(C.byref(d), C.byref(b)))
    return b.value


def lrccs_create(ny, nx, q, ncoil, rank, rank_max=0, params: Params = None, stream=None, precision=PREC_FP32_FFT):
    """Returns an opaque context handle (int).  `stream` is a torch.cuda.Stream or None."""
    d = Dims(ny, nx, q, ncoil, rank, rank_max, precision)
    p = params if params is not None else default_params()
    h = _vp()
    s = None if stream is None else _vp(stream.cuda_stream)
    _check(None, _lib.lrccs_create(C.byref(d), C.byref(p), s, C.byref(h)))
    return h.value


def lrccs_init(ctx, y, frame_ptr, mask, smaps) -> int:
    r = C.c_int32(0)
    _check(ctx, _lib.lrccs_init(ctx, _ptr(y), _ptr(frame_ptr), _ptr(mask), _ptr(smaps), C.byref(r)))
    return r.value


def lrccs_iterate(ctx, n_iter: int, info: bool = False):
    inf = IterInfo() if info else None
    _check(ctx, _lib.lrccs_iterate(ctx, int(n_iter), C.byref(inf) if info else None))
    return _info_dict(inf) if info else None


def lrccs_get_factors(ctx, U=None, B=None):
    _check(ctx, _lib.lrccs_get_factors(ctx, _ptr(U), _ptr(B)))


def lrccs_get_subspace(ctx, U):
    _check(ctx, _lib.lrccs_get_subspace(ctx, _ptr(U)))


def lrccs_get_images(ctx, X):
    _check(ctx, _lib.lrccs_get_images(ctx, _ptr(X)))


def lrccs_get_buffer(ctx, which: int, dst):
    _check(ctx, _lib.lrccs_get_buffer(ctx, int(which), _ptr(dst), dst.numel() * dst.element_size()))


def lrccs_synchronize(ctx):
    _check(ctx, _lib.lrccs_synchronize(ctx))


def lrccs_destroy(ctx):
    _lib.lrccs_destroy(ctx)


def lrccs_profile(ctx, pattern):
    """Time every later launch of the kernels whose name contains `pattern`
    ("*" = all, None = none) with CUDA events on the context's stream."""
    _check(ctx, _lib.lrccs_profile(ctx, None if pattern is None else pattern.encode()))


def lrccs_profile_read(ctx):
    """Synchronise and return [{name, launches, timed, ms}] for every kernel."""
    buf = (KernelStat * 64)()
    n = C.c_int32(0)
    _check(ctx, _lib.lrccs_profile_read(ctx, buf, 64, C.byref(n)))
    return [dict(name=buf[i].name.decode(), launches=buf[i].launches, timed=buf[i].timed, ms=buf[i].ms)
            for i in range(n.value)]


def lrccs_profile_reset(ctx):
    _check(ctx, _lib.lrccs_profile_reset(ctx))


def lrccs_trunc_threshold_noalloc(y, count, trunc_factor, gamma_out, stream=None):
    """gamma = trunc_factor * sum |y_i|^2 / count into gamma_out (a CUDA float64
    tensor), computed without any device allocation (for callers that reserve
    their device memory up front and may not allocate).  The scratch is a fixed
    array inside the library shared by all calls: do not overlap calls on the GPU."""
    import torch

    # The C side can only bound count by the scratch size; everything that
    # keeps the kernel inside y's allocation is checked here, before any launch.
    if y.dtype != torch.complex64:
        raise ValueError("y must be complex64, got %s" % y.dtype)
    if gamma_out.dtype != torch.float64 or gamma_out.numel() < 1:
        raise ValueError("gamma_out must be a float64 tensor with at least one element")
    count = int(count)
    if not 1 <= count <= y.numel():
        raise ValueError("count = %d outside [1, y.numel() = %d]" % (count, y.numel()))
    if not (y.is_cuda and gamma_out.is_cuda):
        raise ValueError("y and gamma_out must be CUDA tensors")
    cur = torch.cuda.current_device()
    if y.device.index != cur or gamma_out.device.index != cur:
        raise ValueError("y and gamma_out must be on the current device (cuda:%d)" % cur)
    s = None if stream is None else _vp(stream.cuda_stream)
    _check(None, _lib.lrccs_trunc_threshold_noalloc(_ptr(y), count, float(trunc_factor), _ptr(gamma_out), s))


def lrccs_mean_step(ctx, y, frame_ptr, mask, smaps, zbar, ytil=None, tol: float = 1e-3, max_iter: int = 10) -> int:
    it = C.c_int32(0)
    _check(ctx, _lib.lrccs_mean_step(ctx, _ptr(y), _ptr(frame_ptr), _ptr(mask), _ptr(smaps), float(tol),
                                     int(max_iter), _ptr(zbar), _ptr(ytil), C.byref(it)))
    return it.value


def lrccs_set_subspace(ctx, U, rank: int, eta: float = 0.0):
    _check(ctx, _lib.lrccs_set_subspace(ctx, _ptr(U), int(rank), float(eta)))


def _info_dict(inf):
    return dict(t=inf.t, exited=inf.exited, eta=inf.eta, sd=inf.sd, gnorm=inf.gnorm)


def lrccs_track_minibatch(ctx, y, frame_ptr, mask, smaps, t_max: int, reset_eta: bool = False, X=None,
                          info: bool = False):
    inf = IterInfo() if info else None
    _check(ctx, _lib.lrccs_track_minibatch(ctx, _ptr(y), _ptr(frame_ptr), _ptr(mask), _ptr(smaps), int(t_max),
                                           1 if reset_eta else 0, _ptr(X), C.byref(inf) if info else None))
    return _info_dict(inf) if info else None


def lrccs_track_minibatch_async(ctx, y, frame_ptr, mask, smaps, t_max: int, reset_eta: bool = False, X=None):
    """Enqueue one tracking request on the context's worker; returns its Ticket."""
    t = Ticket()
    _check(ctx, _lib.lrccs_track_minibatch_async(ctx, _ptr(y), _ptr(frame_ptr), _ptr(mask), _ptr(smaps),
                                                 int(t_max), 1 if reset_eta else 0, _ptr(X), C.byref(t)))
    return t


def lrccs_ticket_query(ctx, ticket) -> bool:
    done = C.c_int32(0)
    _check(ctx, _lib.lrccs_ticket_query(ctx, C.byref(ticket), C.byref(done)))
    return bool(done.value)


def lrccs_ticket_wait(ctx, ticket):
    _check(ctx, _lib.lrccs_ticket_wait(ctx, C.byref(ticket)))


def lrccs_get_state(ctx) -> bytes:
    n = C.c_size_t(0)
    _check(ctx, _lib.lrccs_get_state(ctx, None, C.byref(n)))
    buf = C.create_string_buffer(n.value)
    _check(ctx, _lib.lrccs_get_state(ctx, buf, C.byref(n)))
    return buf.raw[: n.value]


def lrccs_set_state(ctx, state: bytes):
    _check(ctx, _lib.lrccs_set_state(ctx, state, len(state)))


def lrccs_set_plan(ctx, plan: Plan):
    _check(ctx, _lib.lrccs_set_plan(ctx, C.byref(plan)))


def lrccs_get_plan(ctx) -> Plan:
    p = Plan()
    _check(ctx, _lib.lrccs_get_plan(ctx, C.byref(p)))
    return p


def lrccs_autotune(ctx, n_iter: int = 5, cache_path: str = None) -> Plan:
    p = Plan()
    _check(ctx, _lib.lrccs_autotune(ctx, int(n_iter), None if cache_path is None else cache_path.encode(),
                                    C.byref(p)))
    return p


def lrccs_batch_create(ctxs, stream=None):
    arr = (_vp * len(ctxs))(*ctxs)
    h = _vp()
    s = None if stream is None else _vp(stream.cuda_stream)
    _check(None, _lib.lrccs_batch_create(arr, len(ctxs), s, C.byref(h)))
    return h.value


def lrccs_batch_iterate(batch, n_iter: int):
    _check(None, _lib.lrccs_batch_iterate(batch, int(n_iter)))


def lrccs_batch_destroy(batch):
    _lib.lrccs_batch_destroy(batch)


def lrccs_forward_transform(ctx, T):
    _check(ctx, _lib.lrccs_forward_transform(ctx, _ptr(T), T.numel() * T.element_size()))


def lrccs_gdqr_phases(ctx, enable: bool = True, read: bool = False):
    """Phase timing of the GD/QR kernel.  When read: [(mean, max) SM cycles] for
    each of the 8 intervals, then (first entry to last exit, spread of the
    entries) in ns."""
    out = (C.c_double * 18)() if read else None
    _check(ctx, _lib.lrccs_gdqr_phases(ctx, 1 if enable else 0, out))
    return [(out[2 * i], out[2 * i + 1]) for i in range(9)] if read else None


def lrccs_bstep_phases(ctx):
    """Phase timing of the last fused B-step launch (lrccs_gdqr_phases on):
    [(mean, max) ns] for each of the 10 intervals, then (first entry to last
    exit, spread of the entries) in ns."""
    out = (C.c_double * 22)()
    _check(ctx, _lib.lrccs_bstep_phases(ctx, out))
    return [(out[2 * i], out[2 * i + 1]) for i in range(11)]


def lrccs_test_wait_timeout(ctx, enable: bool = True):
    _check(ctx, _lib.lrccs_test_wait_timeout(ctx, 1 if enable else 0))


def lrccs_mec1(ctx, iters: int = 3, zbar=None, E=None, X=None):
    _check(ctx, _lib.lrccs_mec1(ctx, int(iters), _ptr(zbar), _ptr(E), _ptr(X)))


def lrccs_mec2(ctx, max_iter: int = 10, rel_change: float = 0.0025, omega_frac: float = 0.001, zbar=None, E=None,
               X=None) -> int:
    it = C.c_int32(0)
    _check(ctx, _lib.lrccs_mec2(ctx, int(max_iter), float(rel_change), float(omega_frac), _ptr(zbar), _ptr(E),
                                _ptr(X), C.byref(it)))
    return it.value


def lrccs_online_frames(ctx, y, frame_ptr, mask, smaps, zbar, mec_iters: int = 3, X=None, B=None):
    _check(ctx, _lib.lrccs_online_frames(ctx, _ptr(y), _ptr(frame_ptr), _ptr(mask), _ptr(smaps), _ptr(zbar),
                                         int(mec_iters), _ptr(X), _ptr(B)))


def lrccs_last_error(ctx=None) -> str:
    return (_lib.lrccs_last_error(ctx) or b"").decode()


class Solver:
    """Convenience owner of one context: create -> init -> iterate -> factors.

    All tensors live on the current CUDA device; outputs are new torch tensors.
    """

    def __init__(self, ny, nx, q, ncoil, rank, rank_max=0, params: Params = None, stream=None,
                 precision=PREC_FP32_FFT):
        import torch

        self._torch = torch
        self.ny, self.nx, self.q, self.nc = ny, nx, q, ncoil
        self.n = ny * nx
        self.stream = stream
        self.ctx = lrccs_create(ny, nx, q, ncoil, rank, rank_max, params, stream, precision)
        self.r = rank

    def close(self):
        if self.ctx:
            lrccs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, y, frame_ptr, mask, smaps) -> int:
        self.r = lrccs_init(self.ctx, y, frame_ptr, mask, smaps)
        return self.r

    def iterate(self, n_iter, info=False):
        return lrccs_iterate(self.ctx, n_iter, info)

    def mean_step(self, y, frame_ptr, mask, smaps, tol=1e-3, max_iter=10):
        """Alg. 1 steps 1 and 2a: returns (zbar (n,), y~ (like y), CG iterations run)."""
        t = self._torch
        zbar = t.empty((self.n,), dtype=t.complex64, device=y.device)
        ytil = t.empty_like(y)
        it = lrccs_mean_step(self.ctx, y, frame_ptr, mask, smaps, zbar, ytil, tol, max_iter)
        return zbar, ytil, it

    def set_subspace(self, U, eta=0.0):
        """U_0 <- U (n x r) for the next tracking call or iteration; eta > 0 fixes the step size."""
        lrccs_set_subspace(self.ctx, U, U.shape[1], eta)
        self.r = U.shape[1]

    def track(self, y, frame_ptr, mask, smaps, t_max=5, reset_eta=False, X=None, info=False):
        """One later mini-batch of Alg. 4 (warm start, t_max iterations).  X: optional
        (q, n) complex64 output, row k = x_k.  Returns the info dict when info=True."""
        return lrccs_track_minibatch(self.ctx, y, frame_ptr, mask, smaps, t_max, reset_eta, X, info)

    def mec1(self, iters=3, zbar=None):
        """Alg. 3 MEC-1 after the iterations: returns (E, X), each (q, n), row k
        = e_k and x_k = zbar + U_{t-1} b_k + e_k."""
        t = self._torch
        E = t.empty((self.q, self.n), dtype=t.complex64, device="cuda")
        X = t.empty_like(E)
        lrccs_mec1(self.ctx, iters, zbar, E, X)
        return E, X

    def mec2(self, max_iter=10, rel_change=0.0025, omega_frac=0.001, zbar=None):
        """Alg. 3 MEC-2 (ISTA, temporal DFT): returns (E, X, ISTA updates)."""
        t = self._torch
        E = t.empty((self.q, self.n), dtype=t.complex64, device="cuda")
        X = t.empty_like(E)
        it = lrccs_mec2(self.ctx, max_iter, rel_change, omega_frac, zbar, E, X)
        return E, X, it

    def online(self, y, frame_ptr, mask, smaps, zbar, mec_iters=3):
        """Alg. 5 on this context's q frames with the subspace set by set_subspace:
        returns (X (q, n), B (q, r) with row k = b_k)."""
        t = self._torch
        X = t.empty((self.q, self.n), dtype=t.complex64, device="cuda")
        B = t.empty((self.q, self.r), dtype=t.complex64, device="cuda")
        lrccs_online_frames(self.ctx, y, frame_ptr, mask, smaps, zbar, mec_iters, X, B)
        return X, B

    def get_state(self) -> bytes:
        return lrccs_get_state(self.ctx)

    def set_state(self, state: bytes):
        lrccs_set_state(self.ctx, state)
        import struct

        self.r = struct.unpack_from("<i", state, 16)[0]

    def factors(self):
        t = self._torch
        U = t.empty((self.n, self.r), dtype=t.complex64, device="cuda")
        B = t.zeros((self.q, self.r), dtype=t.complex64, device="cuda")   # row k = b_k
        lrccs_get_factors(self.ctx, U, B)
        return U, B

    def subspace(self):
        t = self._torch
        U = t.empty((self.n, self.r), dtype=t.complex64, device="cuda")
        lrccs_get_subspace(self.ctx, U)
        return U

    def images(self):
        t = self._torch
        X = t.empty((self.q, self.n), dtype=t.complex64, device="cuda")   # row k = x_k
        lrccs_get_images(self.ctx, X)
        return X

    def buffer(self, which):
        t = self._torch
        shapes = {BUF_Z: ((self.n, self.q), t.complex64), BUF_X0: ((self.n, self.q), t.complex64),
                  BUF_GRAD: ((self.n, self.r), t.complex64), BUF_SIGMA: ((self.q,), t.float64),
                  BUF_SCAL: ((8,), t.float64)}
        shape, dt = shapes[which]
        out = t.empty(shape, dtype=dt, device="cuda")
        lrccs_get_buffer(self.ctx, which, out)
        return out

    def sync(self):
        lrccs_synchronize(self.ctx)
