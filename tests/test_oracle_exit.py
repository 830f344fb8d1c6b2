"""Pin of the oracle's exit branch (Alg. 2: stop once SD(U_{t-1}, U_t)/sqrt(r) < eps_exit).

The pin is a problem whose iterates are known in closed form.  Take n = 4,
r = 2, q = 2, every A_k the identity, x_1 = s1 e1 and x_2 = s2 e3, and start
from U_0 = [cos th e1 + sin th e2, cos ph e3 + sin ph e4].  With A_k = I the
B-step gives b_k = U^H x_k and the gradient is -(I - U U^H) M U with
M = X X^H = s1^2 e1 e1^H + s2^2 e3 e3^H.  The two columns live in orthogonal
planes, so column 1 moves by itself:

    grad[:, 1] = -s1^2 cos th sin th w,   w = sin th e1 - cos th e2 (unit, _|_ u_1),

the GD step adds eta s1^2 cos th sin th w, and the QR step (columns already
orthogonal, R with positive diagonal) only normalises it: the angle falls to
th' = th - atan(a), a = eta s1^2 sin(2 th)/2, and the column's share of
SD(U_t, U_{t+1})^2 is sin^2(atan a) = a^2/(1 + a^2).  The same holds for
column 2 with s2 and ph.  eta = 0.14 / ||grad_1||_2, and with orthogonal
columns the spectral norm is the larger column norm.  The test runs that
scalar recursion (plain math, no oracle code) and checks the oracle against it.
"""
import math

import numpy as np
import pytest

import oracle

S1, S2, TH0, PH0, ETA_C = 1.0, 0.8, 0.5, 1.1, 0.14


def closed_form(n_iter):
    """Angles after each iteration and SD(U_{t-1}, U_t), t = 1..n_iter."""
    g1 = S1 ** 2 * math.cos(TH0) * math.sin(TH0)
    g2 = S2 ** 2 * math.cos(PH0) * math.sin(PH0)
    eta = ETA_C / max(g1, g2)
    th, ph, sds, angles = TH0, PH0, [], []
    for _ in range(n_iter):
        a = eta * S1 ** 2 * math.sin(2 * th) / 2
        b = eta * S2 ** 2 * math.sin(2 * ph) / 2
        sds.append(math.sqrt(a * a / (1 + a * a) + b * b / (1 + b * b)))
        th, ph = th - math.atan(a), ph - math.atan(b)
        angles.append((th, ph))
    return np.array(sds), angles, eta


def U_of(th, ph):
    U = np.zeros((4, 2), complex)
    U[0, 0], U[1, 0] = math.cos(th), math.sin(th)
    U[2, 1], U[3, 1] = math.cos(ph), math.sin(ph)
    return U


def problem():
    I4 = np.eye(4, dtype=complex)
    op = oracle.Operator.dense(4, [I4, I4])
    y = np.concatenate([S1 * I4[0], S2 * I4[2]])
    return op, y


def first_exit(sds, eps, r=2, sqrt_r=True, less=True):
    """Iterations run under an exit rule (t counted from 1); len(sds) if it never fires."""
    for t, d in enumerate(sds, start=1):
        v = d / math.sqrt(r) if sqrt_r else d
        if (v < eps) if less else (v > eps):
            return t
    return len(sds)


def test_iterates_follow_the_closed_form():
    op, y = problem()
    sds, angles, eta = closed_form(25)
    res = op.iterate(y, U_of(TH0, PH0), 25)
    assert res["iters"] == 25
    assert abs(res["eta"] - eta) < 1e-14 * eta
    assert np.abs(res["sd"] - sds).max() < 1e-13
    th, ph = angles[-1]
    assert np.abs(res["U"] - U_of(th, ph)).max() < 1e-13
    th1, ph1 = angles[-2]
    assert np.abs(res["Uprev"] - U_of(th1, ph1)).max() < 1e-13


@pytest.mark.parametrize("t_star", [3, 7, 12])
def test_exit_fires_at_the_first_iteration_below_the_threshold(t_star):
    """eps halfway (geometrically) between SD_{t*}/sqrt(2) and SD_{t*-1}/sqrt(2):
    the rule stops after exactly t* iterations and returns the pair of that
    iteration (U_{t*-1}, B_{t*}) and U_{t*}."""
    op, y = problem()
    sds, angles, _ = closed_form(40)
    eps = math.sqrt(sds[t_star - 1] * sds[t_star - 2]) / math.sqrt(2)
    assert first_exit(sds, eps) == t_star
    # plausible mistakes in the rule would stop elsewhere
    assert first_exit(sds, eps, sqrt_r=False) != t_star       # sqrt(r) dropped
    assert first_exit(sds, eps, less=False) != t_star         # '>' for '<'
    res = op.iterate(y, U_of(TH0, PH0), 40, params=oracle.Params(exit_enabled=True, eps_exit=eps))
    assert res["iters"] == t_star
    assert len(res["sd"]) == t_star and abs(res["sd"][-1] - sds[t_star - 1]) < 1e-13
    th, ph = angles[t_star - 1]
    assert np.abs(res["U"] - U_of(th, ph)).max() < 1e-13
    th0, ph0 = angles[t_star - 2]
    Uprev = U_of(th0, ph0)
    assert np.abs(res["Uprev"] - Uprev).max() < 1e-13
    # B_{t*} = U_{t*-1}^H x_k (the B-step of the last iteration run)
    X = np.stack([S1 * np.eye(4)[0], S2 * np.eye(4)[2]], 1)
    assert np.abs(res["B"] - Uprev.conj().T @ X).max() < 1e-13


def test_exit_never_fires_below_the_smallest_step():
    op, y = problem()
    sds, _, _ = closed_form(15)
    eps = 0.5 * sds.min() / math.sqrt(2)
    res = op.iterate(y, U_of(TH0, PH0), 15, params=oracle.Params(exit_enabled=True, eps_exit=eps))
    assert res["iters"] == 15


def test_exit_disabled_runs_every_iteration():
    op, y = problem()
    res = op.iterate(y, U_of(TH0, PH0), 15, params=oracle.Params(exit_enabled=False, eps_exit=1.0))
    assert res["iters"] == 15


# ---------------------------------------------------------------- tuning variants (discussion section)

def closed_form_schedule(n_iter, scale0=1.0, decay=1.0, t_offset=0):
    """The same recursion with the variable step eta_t = eta scale0 decay^(t_offset + t - 1)."""
    g1 = S1 ** 2 * math.cos(TH0) * math.sin(TH0)
    g2 = S2 ** 2 * math.cos(PH0) * math.sin(PH0)
    eta = ETA_C / max(g1, g2)
    th, ph, sds = TH0, PH0, []
    for t in range(n_iter):
        et = eta * scale0 * decay ** (t_offset + t)
        a = et * S1 ** 2 * math.sin(2 * th) / 2
        b = et * S2 ** 2 * math.sin(2 * ph) / 2
        sds.append(math.sqrt(a * a / (1 + a * a) + b * b / (1 + b * b)))
        th, ph = th - math.atan(a), ph - math.atan(b)
    return np.array(sds), (th, ph)


@pytest.mark.parametrize("scale0,decay,t_offset", [(2.0, 0.8, 0), (1.5, 0.9, 3), (1.0, 1.0, 5)])
def test_variable_step_size_follows_the_closed_form(scale0, decay, t_offset):
    """Larger steps first, then smaller: eta_t = eta scale0 decay^(t_offset + t - 1)
    with eta = eta_c / ||grad_1||_2 from the call's first gradient."""
    op, y = problem()
    sds, (th, ph) = closed_form_schedule(12, scale0, decay, t_offset)
    prm = oracle.Params(eta_scale0=scale0, eta_decay=decay, t_offset=t_offset)
    res = op.iterate(y, U_of(TH0, PH0), 12, params=prm)
    assert np.abs(res["sd"] - sds).max() < 1e-13
    assert np.abs(res["U"] - U_of(th, ph)).max() < 1e-13


def test_a_decaying_step_differs_from_the_constant_one():
    """A planted mistake (the schedule ignored) would leave SD unchanged; it must not."""
    sd_const, _ = closed_form_schedule(6)
    sd_var, _ = closed_form_schedule(6, 2.0, 0.8)
    assert np.abs(sd_const - sd_var).max() > 1e-2
    op, y = problem()
    res = op.iterate(y, U_of(TH0, PH0), 6, params=oracle.Params(eta_scale0=2.0, eta_decay=0.8))
    assert np.abs(res["sd"] - sd_const).max() > 1e-2


@pytest.mark.parametrize("patience", [2, 3])
def test_robust_exit_needs_consecutive_passes(patience):
    """Exit only once `patience` consecutive iterations pass the exit test.  With
    a threshold between SD_{t*} and every earlier SD, and the sequence decreasing
    after t*, the robust exit stops after t* + patience - 1 iterations."""
    op, y = problem()
    sds, _, _ = closed_form(40)
    t_star = 6
    assert np.all(np.diff(sds[t_star - 1:t_star + 4]) < 0)
    eps = math.sqrt(sds[t_star - 1] * sds[: t_star - 1].min()) / math.sqrt(2)
    res = op.iterate(y, U_of(TH0, PH0), 40,
                     params=oracle.Params(exit_enabled=True, eps_exit=eps, exit_patience=patience))
    assert res["iters"] == t_star + patience - 1
    plain = op.iterate(y, U_of(TH0, PH0), 40, params=oracle.Params(exit_enabled=True, eps_exit=eps))
    assert plain["iters"] == t_star
