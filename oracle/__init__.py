"""FP64 CPU oracle for the altGDmin hot path (Alg. 2 of the paper).

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
benchmark's CPU-baseline leg may import this package.  It wraps the plain C
library built from `altgdmin_oracle.c` (numpy arrays in, numpy arrays out) and
shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "altgdmin_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libaltgdmin_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_MRI = 0
KIND_DENSE = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "altgdmin_oracle.h"))):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd, cwd=_HERE)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("kind", C.c_int32), ("ny", C.c_int32), ("nx", C.c_int32), ("q", C.c_int32),
                ("nc", C.c_int32), ("smaps", C.c_void_p), ("idx", C.c_void_p), ("fp", C.c_void_p),
                ("dense", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("trunc_factor", C.c_double), ("energy_pct", C.c_double), ("eta_c", C.c_double),
                ("eps_exit", C.c_double), ("init_kind", C.c_int32), ("exit_enabled", C.c_int32),
                ("frob_eta", C.c_int32), ("grad_mode", C.c_int32), ("exit_patience", C.c_int32),
                ("eta_scale0", C.c_double), ("eta_decay", C.c_double), ("t_offset", C.c_int32)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB_PATH)
            P = C.POINTER(_Problem)
            vp, i32, dp = C.c_void_p, C.c_int, C.POINTER(C.c_double)
            lib.orc_dft2.argtypes = [vp, vp, i32, i32, i32]
            lib.orc_forward.argtypes = [P, i32, vp, vp]
            lib.orc_adjoint.argtypes = [P, i32, vp, vp]
            lib.orc_eigh.argtypes = [vp, i32, vp, vp]
            lib.orc_eigh.restype = i32
            lib.orc_qr.argtypes = [vp, i32, i32, vp, vp]
            lib.orc_qr.restype = i32
            lib.orc_lstsq.argtypes = [vp, i32, i32, vp, vp]
            lib.orc_lstsq.restype = i32
            lib.orc_init.argtypes = [P, vp, C.POINTER(_Params), i32, i32, vp, vp, vp, dp]
            lib.orc_init.restype = i32
            lib.orc_bstep.argtypes = [P, vp, vp, i32, vp]
            lib.orc_bstep.restype = i32
            lib.orc_grad.argtypes = [P, vp, vp, vp, i32, i32, vp]
            lib.orc_cost.argtypes = [P, vp, vp, vp, i32]
            lib.orc_cost.restype = C.c_double
            lib.orc_iterate.argtypes = [P, vp, C.POINTER(_Params), vp, i32, i32, dp, vp, vp, vp, vp, vp]
            lib.orc_iterate.restype = i32
            lib.orc_sd.argtypes = [vp, vp, i32, i32]
            lib.orc_sd.restype = C.c_double
            _lib = lib
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return None if a is None else a.ctypes.data


class Params:
    """Alg. 2 constants (blue parameter settings) plus oracle switches."""

    def __init__(self, trunc_factor=36.0, energy_pct=85.0, eta_c=0.14, eps_exit=0.01,
                 init_kind=0, exit_enabled=False, frob_eta=False, grad_mode=0, exit_patience=1, eta_scale0=1.0,
                 eta_decay=1.0, t_offset=0):
        self.s = _Params(trunc_factor, energy_pct, eta_c, eps_exit, init_kind, int(exit_enabled),
                         int(frob_eta), grad_mode, int(exit_patience), float(eta_scale0), float(eta_decay),
                         int(t_offset))


class Operator:
    """One LRcCS problem: MRI operator A_k = [H_k F D_j]_j, or dense A_k.

    MRI:   Operator.mri(ny, nx, smaps (nc, n), idx int32, frame_ptr int64)
    dense: Operator.dense(n, [A_1, ..., A_q])  with A_k of shape (m_k, n)
    """

    def __init__(self, kind, ny, nx, q, nc, smaps, idx, fp, dense):
        self.kind, self.ny, self.nx, self.q, self.nc = kind, ny, nx, q, nc
        self.n = ny * nx
        self._smaps = smaps
        self._idx = idx
        self._fp = fp
        self._dense = dense
        self.m = np.diff(fp)
        self.s = _Problem(kind, ny, nx, q, nc, _ptr(smaps), _ptr(idx), _ptr(fp), _ptr(dense))

    @classmethod
    def mri(cls, ny, nx, smaps, idx, frame_ptr):
        smaps = _c128(smaps).reshape(-1, ny * nx)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        fp = np.ascontiguousarray(frame_ptr, dtype=np.int64)
        return cls(KIND_MRI, ny, nx, len(fp) - 1, smaps.shape[0], smaps, idx, fp, None)

    @classmethod
    def dense(cls, n, mats):
        fp = np.zeros(len(mats) + 1, dtype=np.int64)
        fp[1:] = np.cumsum([a.shape[0] for a in mats])
        d = _c128(np.concatenate([np.asarray(a).reshape(-1, n) for a in mats], axis=0))
        return cls(KIND_DENSE, 1, n, len(mats), 1, None, None, fp, d)

    @classmethod
    def from_problem(cls, p):
        return cls.mri(p.ny, p.nx, p.smaps, p.idx, p.frame_ptr)

    # -- operator -----------------------------------------------------------
    def rows(self, k: int) -> int:
        return int(self.nc * self.m[k])

    def yoff(self, k: int) -> int:
        return int(self.nc * self._fp[k])

    def forward(self, k: int, x) -> np.ndarray:
        x = _c128(x)
        out = np.zeros(self.rows(k), dtype=np.complex128)
        _load().orc_forward(C.byref(self.s), k, _ptr(x), _ptr(out))
        return out

    def adjoint(self, k: int, yk) -> np.ndarray:
        yk = _c128(yk)
        out = np.zeros(self.n, dtype=np.complex128)
        _load().orc_adjoint(C.byref(self.s), k, _ptr(yk), _ptr(out))
        return out

    # -- Alg. 2 pieces ------------------------------------------------------
    def init(self, y, params: Params = None, rank=0, rmax=None, want_x0=False):
        """Returns dict(U0, sigma, rank, gamma[, X0])."""
        params = params or Params()
        y = _c128(y)
        rmax = rmax or self.q
        U0 = np.zeros((self.n, rmax), dtype=np.complex128)
        sig = np.zeros(self.q, dtype=np.float64)
        X0 = np.zeros((self.n, self.q), dtype=np.complex128) if want_x0 else None
        g = C.c_double(0.0)
        r = _load().orc_init(C.byref(self.s), _ptr(y), C.byref(params.s), int(rank), int(rmax),
                             _ptr(U0), _ptr(sig), _ptr(X0), C.byref(g))
        if r < 0:
            raise RuntimeError("oracle init failed")
        out = dict(U0=np.ascontiguousarray(U0.reshape(-1)[: self.n * r].reshape(self.n, r)),
                   sigma=sig, rank=r, gamma=g.value)
        if want_x0:
            out["X0"] = X0
        return out

    def bstep(self, y, U) -> np.ndarray:
        U = _c128(U)
        r = U.shape[1]
        y = _c128(y)
        B = np.zeros((self.q, r), dtype=np.complex128)  # row k = b_k
        rc = _load().orc_bstep(C.byref(self.s), _ptr(y), _ptr(U), r, _ptr(B))
        if rc != 0:
            raise RuntimeError("rank-deficient least squares")
        return B.T.copy()

    def grad(self, y, U, B, mode=0) -> np.ndarray:
        U = _c128(U)
        r = U.shape[1]
        Bc = _c128(np.asarray(B).T)
        y = _c128(y)
        G = np.zeros_like(U)
        _load().orc_grad(C.byref(self.s), _ptr(y), _ptr(U), _ptr(Bc), r, mode, _ptr(G))
        return G

    def cost(self, y, U, B) -> float:
        U = _c128(U)
        Bc = _c128(np.asarray(B).T)
        y = _c128(y)
        return _load().orc_cost(C.byref(self.s), _ptr(y), _ptr(U), _ptr(Bc), U.shape[1])

    def iterate(self, y, U, n_iter, params: Params = None, eta=0.0, history=False):
        """Run Alg. 2 iterations from U.  Returns dict(U, Uprev, B (r x q), eta,
        sd, gnorm, iters[, X (iters, n, q)]) with X_t = U_{t-1} B_t."""
        params = params or Params()
        U = _c128(U).copy()
        r = U.shape[1]
        Bc = np.zeros((self.q, r), dtype=np.complex128)
        Uprev = np.zeros_like(U)
        Xh = np.zeros((n_iter, self.n, self.q), dtype=np.complex128) if history else None
        sd = np.zeros(n_iter)
        gn = np.zeros(n_iter)
        e = C.c_double(eta)
        y = _c128(y)
        t = _load().orc_iterate(C.byref(self.s), _ptr(y), C.byref(params.s), _ptr(U), r,
                                int(n_iter), C.byref(e), _ptr(Bc), _ptr(Uprev), _ptr(Xh),
                                _ptr(sd), _ptr(gn))
        if t < 0:
            raise RuntimeError("oracle iterate failed (%d)" % t)
        out = dict(U=U, Uprev=Uprev, B=Bc.T.copy(), eta=e.value, sd=sd[:t], gnorm=gn[:t], iters=t)
        if history:
            out["X"] = Xh[:t]
        return out


def _cgls(A, AH, b, n, tol, maxit):
    """CGLS (conjugate gradients on A^H A x = A^H b) from x = 0: at most maxit
    iterations, stopping once ||A^H r_t|| <= tol ||A^H b||.  Returns
    (x, iterations, [||A^H r_t|| for t = 0..iterations])."""
    x = np.zeros(n, dtype=np.complex128)
    res = b.copy()                      # r_0 = b - A x_0
    s = AH(res)                         # normal residual A^H r
    p = s.copy()
    gamma = np.vdot(s, s).real
    norms0 = math.sqrt(gamma)
    hist = [norms0]
    t = 0
    while t < maxit and hist[-1] > tol * norms0 and gamma > 0:
        w = A(p)
        alpha = gamma / np.vdot(w, w).real
        x = x + alpha * p
        res = res - alpha * w
        s = AH(res)
        gamma_new = np.vdot(s, s).real
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
        hist.append(math.sqrt(gamma))
        t += 1
    return x, t, np.array(hist)


def _frame(op, v, k):
    a = op.yoff(k)
    return v[a: a + op.rows(k)]


def _A_all(op, E):
    """[A_k e_k]_k concatenated in the layout of y (E: n x q)."""
    return np.concatenate([op.forward(k, E[:, k]) for k in range(op.q)])


def _AH_all(op, v):
    """n x q matrix with column k = A_k^H v_k."""
    return np.stack([op.adjoint(k, _frame(op, v, k)) for k in range(op.q)], 1)


def mean_step(op, y, tol=1e-3, maxit=10):
    """Alg. 1 step 1: zbar = argmin_z sum_k ||y_k - A_k z||^2 by CGLS on the
    stacked operator A = [A_1; ...; A_q] from z = 0, stopped after maxit
    iterations or once ||A^H r_t|| <= tol ||A^H y||; then the residual
    measurements y~_k = y_k - A_k zbar (Alg. 1 step 2a).  Returns dict(zbar,
    ytil, iters, normal_res: ||A^H r_t|| for t = 0..iters)."""
    y = _c128(y)

    def A(z):
        return np.concatenate([op.forward(k, z) for k in range(op.q)])

    def AH(v):
        return _AH_all(op, v).sum(1)

    z, t, hist = _cgls(A, AH, y, op.n, tol, maxit)
    return dict(zbar=z, ytil=y - A(z), iters=t, normal_res=hist)


def mec1(op, ytt, iters=3):
    """Alg. 3, unstructured MEC (altGDmin-MRI1): for every frame, `iters` CGLS
    iterations from e = 0 on min_e ||ytt_k - A_k e||^2 (the paper's tolerance
    1e-36 never stops them early).  ytt: residual measurements
    y_k - A_k zbar - A_k x_k in the layout of y.  Returns E (n x q)."""
    ytt = _c128(ytt)
    E = np.zeros((op.n, op.q), dtype=np.complex128)
    for k in range(op.q):
        E[:, k] = _cgls(lambda e: op.forward(k, e), lambda v: op.adjoint(k, v), _frame(op, ytt, k), op.n,
                        0.0, iters)[0]
    return E


def soft_threshold(M, omega):
    """Complex soft threshold: M_i (|M_i| - omega)/|M_i| where |M_i| > omega, else 0."""
    a = np.abs(M)
    return np.where(a > omega, M * (1.0 - omega / np.where(a > 0, a, 1.0)), 0.0)


def mec2(op, ytt, max_iter=10, rel_change=0.0025, frac=0.001):
    """Alg. 3, sparse MEC (altGDmin-MRI2): ISTA for E with a sparse temporal
    Fourier transform.  From E_0 = 0, step tau computes
        M_tau = F_t(E_tau + A^H(ytt - A(E_tau))),   F_t: DFT along the frames,
    sets omega = frac max|M_0| at tau = 0, and E_{tau+1} = F_t^{-1}(SThr_omega(M_tau));
    it stops after max_iter updates or once ||M_tau - M_{tau-1}||_F <
    rel_change ||M_{tau-1}||_F.  Returns dict(E (n x q), iters, omega)."""
    ytt = _c128(ytt)
    E = np.zeros((op.n, op.q), dtype=np.complex128)
    M_prev, omega, tau = None, None, 0
    while tau < max_iter:
        M = np.fft.fft(E + _AH_all(op, ytt - _A_all(op, E)), axis=1, norm="ortho")
        if omega is None:
            omega = frac * np.abs(M).max()
        if M_prev is not None and np.linalg.norm(M - M_prev) < rel_change * np.linalg.norm(M_prev):
            break
        E = np.fft.ifft(soft_threshold(M, omega), axis=1, norm="ortho")
        M_prev = M
        tau += 1
    return dict(E=E, iters=tau, omega=omega)


def online_frames(op, y, zbar, U, mec_iters=3):
    """Alg. 5 step 2 (online subspace tracking) for the frames of `op`, all after
    the first mini-batch: with that mini-batch's mean zbar and subspace U held
    fixed, every frame gets y~_k = y_k - A_k zbar, b_k = (A_k U)^+ y~_k (the
    B-step), e_k from `mec_iters` CGLS steps on y~_k - A_k U b_k (MEC-1), and
    x_k = zbar + U b_k + e_k.  Returns dict(X (n x q), B (r x q), E (n x q))."""
    y, zbar, U = _c128(y), _c128(zbar), _c128(U)
    ytil = y - _A_all(op, np.repeat(zbar[:, None], op.q, 1))
    B = op.bstep(ytil, U)
    E = mec1(op, ytil - _A_all(op, U @ B), mec_iters)
    return dict(X=zbar[:, None] + U @ B + E, B=B, E=E)


def track_minibatches(batches, rank, t_first=70, t_next=5, params: Params = None, reset_eta=False,
                      U_start=None, eta_start=0.0):
    """Mini-batch subspace tracking (Alg. 4) over `batches`, a list of
    (Operator, y) pairs, one per mini-batch in arrival order.

    The first mini-batch is solved by Alg. 2 (spectral initialisation, then
    t_first GDmin iterations) unless U_start is given; every later one (and
    the first, when U_start is given) starts from the previous final subspace,
    U_0 <- U^(j-1), and runs t_next GDmin iterations.  The step size is the one
    set at the first mini-batch's first iteration (or eta_start when > 0) and
    is kept; reset_eta sets it again at every mini-batch's first iteration.
    Returns one dict per mini-batch: X = U_{t-1} B_t (n x q_j), U (final),
    eta, sd, gnorm, iters."""
    params = params or Params()
    out = []
    U, eta = U_start, float(eta_start)
    for j, (op, y) in enumerate(batches):
        if U is None:
            ini = op.init(y, params, rank=rank)
            res = op.iterate(y, ini["U0"], t_first, params)
        else:
            res = op.iterate(y, U, t_next, params, eta=0.0 if reset_eta else eta)
        U, eta = res["U"], res["eta"]
        out.append(dict(X=res["Uprev"] @ res["B"], U=U, eta=eta, sd=res["sd"], gnorm=res["gnorm"],
                        iters=res["iters"]))
    return out


def dft2(x, sign=-1) -> np.ndarray:
    x = _c128(x)
    ny, nx = x.shape
    out = np.zeros_like(x)
    _load().orc_dft2(_ptr(x), _ptr(out), ny, nx, sign)
    return out


def eigh(A):
    A = _c128(A)
    q = A.shape[0]
    w = np.zeros(q)
    V = np.zeros_like(A)
    _load().orc_eigh(_ptr(A), q, _ptr(w), _ptr(V))
    return w, V


def qr(A):
    A = _c128(A)
    m, r = A.shape
    Q = np.zeros_like(A)
    R = np.zeros((r, r), dtype=np.complex128)
    if _load().orc_qr(_ptr(A), m, r, _ptr(Q), _ptr(R)) != 0:
        raise RuntimeError("rank deficient")
    return Q, R


def lstsq(M, y):
    M = _c128(M)
    m, r = M.shape
    b = np.zeros(r, dtype=np.complex128)
    y = _c128(y)
    if _load().orc_lstsq(_ptr(M), m, r, _ptr(y), _ptr(b)) != 0:
        raise RuntimeError("rank deficient")
    return b


def sd(U1, U2) -> float:
    U1, U2 = _c128(U1), _c128(U2)
    return _load().orc_sd(_ptr(U1), _ptr(U2), U1.shape[0], U1.shape[1])
