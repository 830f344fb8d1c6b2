"""Seeded synthetic inputs for low-rank column-wise compressive sensing (dynamic MRI).

This module only draws random numbers and lays data out.  It implements none of
the solver's arithmetic (no DFT, no least squares, no gradient, no QR of the
iterate), so the FP64 oracle and the CUDA library can both consume what it makes
without sharing any of the method's code.

How k-space is produced without a DFT
-------------------------------------
The measurement model is y_kj = H_k F (d_j o z_k) (Sec. II-A, multi-coil model).
Ground truth is defined directly in k-space, as the spectrum zhat_k = F z_k:

* exactly low rank (the single-coil case): zhat_k = V* b*_k with V* an
  orthonormal complex Gaussian n x r matrix; since F is unitary and the complex
  Gaussian law is rotation invariant, U* = F^H V* is distributed exactly like an
  orthonormal complex Gaussian image-domain basis;
* ellipse phantoms: the continuous Fourier transform of each ellipse, evaluated
  at the integer frequencies of the grid (the standard analytic MRI phantom).

Coil maps are low-order trigonometric polynomials,
    d_j(y, x) = sum_m c_jm exp(+2 pi i (a_m y / Ny + b_m x / Nx)),
with the C x M coefficient matrix having orthogonal columns of squared norm 1/M,
which makes sum_j |d_j|^2 = 1 at every pixel exactly.  Multiplying an image by
exp(+2 pi i (a y/Ny + b x/Nx)) circularly shifts its unitary DFT by (a, b), so
    F(d_j o z)[ky, kx] = sum_m c_jm zhat[(ky - a_m) mod Ny, (kx - b_m) mod Nx],
which is how coil k-space is synthesised here: shifts and sums of the analytic
spectrum, with no transform.

Layouts (shared with the library's C ABI)
-----------------------------------------
* k-space index i = ky * Nx + kx with DC at 0 (no fftshift); masks are drawn in
  centred coordinates and stored at ky mod Ny.
* mask: uint8 (q, Ny*Nx) bitmap.
* idx: int32, the sampled indices of every frame in ascending order, frames
  concatenated; frame_ptr: int64 (q+1), offsets into idx (samples per coil).
* y: complex64, ragged, frame k / coil j / sample s at
  nc*frame_ptr[k] + j*m_k + s.
* smaps: complex64 (nc, n), pixel index i = y * Nx + x.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, Optional

import numpy as np

__all__ = [
    "Problem",
    "WORKLOADS",
    "make_problem",
    "cartesian_lines_uniform",
    "cartesian_lines_vd",
    "coil_maps",
    "random_orthonormal",
]


def _cgauss(rng: np.random.Generator, shape) -> np.ndarray:
    """Standard circular complex Gaussian, E|z|^2 = 1."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def random_orthonormal(rng: np.random.Generator, n: int, r: int) -> np.ndarray:
    """n x r matrix with orthonormal columns, Haar distributed (QR of a complex Gaussian)."""
    g = _cgauss(rng, (n, r))
    qm, rm = np.linalg.qr(g)
    ph = np.diag(rm) / np.abs(np.diag(rm))
    return qm * ph[None, :]


# ----------------------------------------------------------------------------
# Sampling masks (Sec. V: 1D Cartesian variable density, golden-angle radial)
# ----------------------------------------------------------------------------

def _centred_to_index(kc: np.ndarray, n: int) -> np.ndarray:
    return np.mod(kc, n)


def cartesian_lines_uniform(rng, ny: int, nx: int, q: int, n_center: int, n_rand: int) -> np.ndarray:
    """Per-frame phase-encode line masks: n_center central lines always, n_rand
    other lines drawn uniformly without replacement, redrawn every frame."""
    ky_c = np.arange(-ny // 2, ny - ny // 2)
    center = np.arange(-(n_center // 2), n_center - n_center // 2)
    others = np.setdiff1d(ky_c, center)
    mask = np.zeros((q, ny, nx), dtype=np.uint8)
    for k in range(q):
        pick = rng.choice(others, size=n_rand, replace=False)
        lines = _centred_to_index(np.concatenate([center, pick]), ny)
        mask[k, lines, :] = 1
    return mask.reshape(q, ny * nx)


def cartesian_lines_vd(rng, ny: int, nx: int, q: int, accel: float) -> np.ndarray:
    """Variable-density 1D Cartesian masks at acceleration `accel`.

    The paper cites a published scheme without giving its density.  Reading used
    here: a fully sampled centre block of max(4, round(Ny/(4R))) lines, plus the
    remaining round(Ny/R) - centre lines drawn without replacement with weight
    (1 - |ky|/(Ny/2))^2, redrawn every frame.
    """
    n_lines = int(round(ny / accel))
    n_center = max(4, int(round(ny / (4.0 * accel))))
    n_center = min(n_center, n_lines)
    ky_c = np.arange(-ny // 2, ny - ny // 2)
    center = np.arange(-(n_center // 2), n_center - n_center // 2)
    others = np.setdiff1d(ky_c, center)
    w = (1.0 - np.abs(others) / (ny / 2.0)) ** 2
    w = w / w.sum()
    mask = np.zeros((q, ny, nx), dtype=np.uint8)
    for k in range(q):
        pick = rng.choice(others, size=n_lines - n_center, replace=False, p=w)
        lines = _centred_to_index(np.concatenate([center, pick]), ny)
        mask[k, lines, :] = 1
    return mask.reshape(q, ny * nx)


def radial_golden(ny: int, nx: int, q: int, spokes: int, golden_deg: float = 111.25) -> np.ndarray:
    """Pseudo-radial masks on the Cartesian grid: spoke s of frame k at angle
    (s*180/S + k*golden) mod 180 degrees, points t in [-N/2, N/2) at unit step,
    rounded to the nearest grid point (deduplicated by the bitmap)."""
    n = max(ny, nx)
    t = np.arange(-n // 2, n - n // 2, dtype=np.float64)
    mask = np.zeros((q, ny, nx), dtype=np.uint8)
    for k in range(q):
        for s in range(spokes):
            th = math.radians(math.fmod(s * 180.0 / spokes + k * golden_deg, 180.0))
            kyc = np.floor(t * math.sin(th) + 0.5).astype(np.int64)
            kxc = np.floor(t * math.cos(th) + 0.5).astype(np.int64)
            ok = (kyc >= -ny // 2) & (kyc < ny - ny // 2) & (kxc >= -nx // 2) & (kxc < nx - nx // 2)
            mask[k, np.mod(kyc[ok], ny), np.mod(kxc[ok], nx)] = 1
    return mask.reshape(q, ny * nx)


# ----------------------------------------------------------------------------
# Coil maps: trigonometric polynomials with unit sum of squares
# ----------------------------------------------------------------------------

def _coil_modes(nc: int):
    cand = [(a, b) for a in range(-2, 3) for b in range(-2, 3)]
    cand.sort(key=lambda ab: (abs(ab[0]) + abs(ab[1]), abs(ab[0]), ab))
    m = min(nc, 9)
    return cand[:m]


def coil_maps(rng, ny: int, nx: int, nc: int):
    """Return (smaps (nc, n) complex128, modes [(a, b)], coef (nc, M))."""
    modes = _coil_modes(nc)
    m = len(modes)
    if nc == 1:
        coef = np.ones((1, 1), dtype=np.complex128)
    else:
        qm = random_orthonormal(rng, nc, m)
        coef = qm / math.sqrt(m)
    yy = np.arange(ny)[:, None]
    xx = np.arange(nx)[None, :]
    smaps = np.zeros((nc, ny, nx), dtype=np.complex128)
    for mi, (a, b) in enumerate(modes):
        wave = np.exp(2j * np.pi * (a * yy / ny + b * xx / nx))
        smaps += coef[:, mi][:, None, None] * wave[None]
    return smaps.reshape(nc, ny * nx), modes, coef


# ----------------------------------------------------------------------------
# Ground-truth spectra
# ----------------------------------------------------------------------------

def _freq_grid(ny: int, nx: int):
    ky = np.arange(ny)
    kx = np.arange(nx)
    kyc = np.where(ky < (ny + 1) // 2, ky, ky - ny)
    kxc = np.where(kx < (nx + 1) // 2, kx, kx - nx)
    return kyc[:, None] / ny, kxc[None, :] / nx  # cycles per pixel


def _ellipse_spectrum(nu_y, nu_x, cy, cx, ay, ax, theta, rho, n):
    """Unitary-DFT-scaled samples of the continuous FT of rho * 1{ellipse}."""
    from scipy.special import j1

    ct, st = math.cos(theta), math.sin(theta)
    uy = ct * nu_y + st * nu_x
    ux = -st * nu_y + ct * nu_x
    kap = np.sqrt((ay * uy) ** 2 + (ax * ux) ** 2)
    small = kap < 1e-12
    kap_s = np.where(small, 1.0, kap)
    val = np.where(small, math.pi * ay * ax, ay * ax * j1(2.0 * math.pi * kap_s) / kap_s)
    phase = np.exp(-2j * math.pi * (nu_y * cy + nu_x * cx))
    return rho * val * phase / math.sqrt(n)


def phantom_spectra(rng, ny: int, nx: int, q: int, n_inner: int = 5, ramp: bool = False) -> np.ndarray:
    """(q, n) complex128 spectra of an ellipse phantom whose inner ellipses
    deform sinusoidally over one period (optionally with a sigmoid contrast
    ramp per region), i.e. an approximately low-rank sequence."""
    nu_y, nu_x = _freq_grid(ny, nx)
    n = ny * nx
    cy0, cx0 = ny / 2.0, nx / 2.0
    out = np.zeros((q, ny, nx), dtype=np.complex128)
    body = _ellipse_spectrum(nu_y, nu_x, cy0, cx0, 0.42 * ny, 0.36 * nx, 0.0, 1.0, n)
    inner = []
    for e in range(n_inner):
        inner.append(dict(
            cy=cy0 + rng.uniform(-0.18, 0.18) * ny,
            cx=cx0 + rng.uniform(-0.15, 0.15) * nx,
            ay=rng.uniform(0.04, 0.12) * ny,
            ax=rng.uniform(0.04, 0.12) * nx,
            th=rng.uniform(0.0, math.pi),
            rho=rng.uniform(0.3, 0.9) * (1.0 if rng.uniform() < 0.7 else -1.0),
            phi=rng.uniform(0.0, 2.0 * math.pi),
            ramp_amp=rng.uniform(0.3, 1.0),
            ramp_mid=rng.uniform(0.3, 0.7) * q,
            ramp_w=rng.uniform(0.04, 0.12) * q,
        ))
    for k in range(q):
        acc = body.copy()
        for p in inner:
            s = 1.0 + 0.1 * math.sin(2.0 * math.pi * k / q + p["phi"])
            rho = p["rho"]
            if ramp:
                rho = rho * (1.0 + p["ramp_amp"] / (1.0 + math.exp(-(k - p["ramp_mid"]) / p["ramp_w"])))
            acc += _ellipse_spectrum(nu_y, nu_x, p["cy"], p["cx"], p["ay"] * s, p["ax"] * s, p["th"], rho, n)
        out[k] = acc
    return out.reshape(q, n)


# ----------------------------------------------------------------------------
# Problem assembly
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    name: str
    ny: int
    nx: int
    q: int
    nc: int
    rank: int
    t_iter: int
    mask: np.ndarray        # (q, n) uint8
    idx: np.ndarray         # int32, concatenated sorted sample indices
    frame_ptr: np.ndarray   # int64 (q+1)
    y: np.ndarray           # complex64 ragged
    smaps: np.ndarray       # complex64 (nc, n)
    truth: Dict[str, np.ndarray]

    @property
    def n(self) -> int:
        return self.ny * self.nx

    @property
    def m(self) -> np.ndarray:
        return np.diff(self.frame_ptr)

    def y_frame(self, k: int) -> np.ndarray:
        """(nc, m_k) view of frame k."""
        a = self.nc * int(self.frame_ptr[k])
        mk = int(self.frame_ptr[k + 1] - self.frame_ptr[k])
        return self.y[a:a + self.nc * mk].reshape(self.nc, mk)


def frames(p: Problem, start: int, count: int) -> Problem:
    """The frames [start, start + count) of `p` as a problem of their own (the
    same coil maps; masks, sample offsets, data and per-frame truth sliced).
    Mini-batches of an acquisition (Alg. 4) are cut this way."""
    if start < 0 or count < 1 or start + count > p.q:
        raise ValueError("frames %d..%d outside 0..%d" % (start, start + count, p.q))
    fp = p.frame_ptr
    a, b = int(fp[start]), int(fp[start + count])
    truth = {}
    for k, v in p.truth.items():
        if k == "spectra":
            truth[k] = v[start:start + count]
        elif k == "B":
            truth[k] = v[:, start:start + count]
        elif k == "y128":
            truth[k] = v[p.nc * a: p.nc * b]
        else:
            truth[k] = v
    return dataclasses.replace(p, name="%s[%d:%d]" % (p.name, start, start + count), q=count,
                               mask=p.mask[start:start + count], idx=p.idx[a:b], frame_ptr=fp[start:start + count + 1] - a,
                               y=p.y[p.nc * a: p.nc * b], truth=truth)


def compact_mask(mask: np.ndarray):
    """Bitmap -> (idx int32 sorted per frame, frame_ptr int64)."""
    q = mask.shape[0]
    lists = [np.flatnonzero(mask[k]).astype(np.int32) for k in range(q)]
    fp = np.zeros(q + 1, dtype=np.int64)
    fp[1:] = np.cumsum([len(l) for l in lists])
    idx = np.concatenate(lists) if q else np.zeros(0, np.int32)
    return idx, fp


def _coil_kspace_at(zhat_k: np.ndarray, ny: int, nx: int, modes, coef, sel: np.ndarray) -> np.ndarray:
    """F(d_j o z_k) at 1D indices `sel` for every coil, by the shift identity."""
    zz = zhat_k.reshape(ny, nx)
    ky = sel // nx
    kx = sel % nx
    out = np.zeros((coef.shape[0], sel.size), dtype=np.complex128)
    for mi, (a, b) in enumerate(modes):
        g = zz[(ky - a) % ny, (kx - b) % nx]
        out += coef[:, mi][:, None] * g[None, :]
    return out


def assemble(name, ny, nx, q, nc, rank, t_iter, mask, spectra, modes, coef, smaps,
             rng, noise_rel: float, truth) -> Problem:
    idx, fp = compact_mask(mask)
    y = np.zeros(nc * int(fp[-1]), dtype=np.complex128)
    y_clean = None
    for k in range(q):
        sel = idx[fp[k]:fp[k + 1]]
        yk = _coil_kspace_at(spectra[k], ny, nx, modes, coef, sel)
        y[nc * fp[k]: nc * fp[k + 1]] = yk.reshape(-1)
    if noise_rel > 0:
        rms = math.sqrt(float(np.mean(np.abs(y) ** 2)))
        y = y + noise_rel * rms * _cgauss(rng, y.shape)
    truth = dict(truth)
    truth["spectra"] = spectra
    truth["y128"] = y
    truth["smaps128"] = smaps
    return Problem(name, ny, nx, q, nc, rank, t_iter, mask, idx, fp,
                   y.astype(np.complex64), smaps.astype(np.complex64), truth)


# Named workloads (shapes of the paper's cardiac/other multi-coil scans).
WORKLOADS = {
    # exact rank-4 single-coil sequence, 16 of 64 lines per frame
    "lines64_q32_c1_r4": dict(kind="lowrank", ny=64, nx=64, q=32, nc=1, rank=4, t_iter=50,
                              n_center=4, n_rand=12),
    # cardiac-shaped multi-coil phantom, 8x variable-density Cartesian
    "cardiac192_q48_c12_r10": dict(kind="phantom", ny=192, nx=192, q=48, nc=12, rank=10, t_iter=50,
                                   accel=8.0, noise=0.01),
    # the same phantom with a contrast-uptake ramp per region, 20 coils, 16
    # golden-angle pseudo-radial spokes per frame on the Cartesian grid
    "radial256_q64_c20_r12": dict(kind="phantom", ny=256, nx=256, q=64, nc=20, rank=12, t_iter=50,
                                  mask_kind="radial", spokes=16, noise=0.01, ramp=True),
}


def make_problem(spec, seed: Optional[int] = None, **over) -> Problem:
    """Build a seeded synthetic problem.

    `spec` is a WORKLOADS key or a dict with the same fields.  kind='lowrank'
    gives y_k = H_k V* b*_k (exact rank, C=1, d=1); kind='phantom' gives the
    deforming ellipse phantom through trigonometric coil maps plus complex
    Gaussian noise at `noise` x RMS.
    """
    if isinstance(spec, str):
        name = spec
        cfg = dict(WORKLOADS[spec])
    else:
        cfg = dict(spec)
        name = cfg.pop("name", "custom")
    cfg.update(over)
    if seed is None:
        seed = 0x5EED0000 + (list(WORKLOADS).index(name) + 1 if name in WORKLOADS else 0)
    rng = np.random.default_rng(seed)
    ny, nx, q, nc = cfg["ny"], cfg["nx"], cfg["q"], cfg["nc"]
    rank, t_iter = cfg["rank"], cfg.get("t_iter", 50)
    n = ny * nx
    masks = cfg.get("mask_kind", "lines_uniform" if cfg["kind"] == "lowrank" else "lines_vd")
    if masks == "lines_uniform":
        mask = cartesian_lines_uniform(rng, ny, nx, q, cfg.get("n_center", 4), cfg.get("n_rand", 12))
    elif masks == "lines_vd":
        mask = cartesian_lines_vd(rng, ny, nx, q, cfg.get("accel", 8.0))
    elif masks == "full":
        mask = np.ones((q, n), dtype=np.uint8)
    elif masks == "radial":
        mask = radial_golden(ny, nx, q, cfg.get("spokes", 16))
    else:
        raise ValueError(masks)
    smaps, modes, coef = coil_maps(rng, ny, nx, nc)
    truth = {}
    if cfg["kind"] == "lowrank":
        vstar = random_orthonormal(rng, n, rank)
        bstar = _cgauss(rng, (rank, q))
        spectra = (vstar @ bstar).T.copy()
        truth["V"] = vstar
        truth["B"] = bstar
    elif cfg["kind"] == "phantom":
        spectra = phantom_spectra(rng, ny, nx, q, cfg.get("n_inner", 5), cfg.get("ramp", False))
    else:
        raise ValueError(cfg["kind"])
    return assemble(name, ny, nx, q, nc, rank, t_iter, mask, spectra, modes, coef, smaps,
                    rng, cfg.get("noise", 0.0), truth)
