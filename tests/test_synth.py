"""The seeded synthetic inputs follow their stated recipe: sample counts of the
workloads, the variable-density and uniform line rules, the pseudo-radial
density, unit-sum-of-squares coil maps, and per-seed determinism.  CPU only."""
import numpy as np
import pytest

from paper_2212_09664_gb300 import synth


def _lines(mask, q, ny, nx):
    m = mask.reshape(q, ny, nx)
    full = m.all(2)
    assert np.array_equal(m.any(2), full), "a row is partly sampled"
    return full


def test_workload_sample_counts():
    """cardiac192: 24 of 192 lines (R = 8) per frame, m_k = 24 x 192 = 4608 per coil,
    148 rows sampled by some frame; lines64: 16 of 64 lines, m_k = 1024."""
    p = synth.make_problem("cardiac192_q48_c12_r10")
    assert set(np.diff(p.frame_ptr).tolist()) == {4608}
    assert int(_lines(p.mask, p.q, p.ny, p.nx).any(0).sum()) == 148
    assert p.y.size == p.nc * int(p.frame_ptr[-1])
    p1 = synth.make_problem("lines64_q32_c1_r4")
    assert set(np.diff(p1.frame_ptr).tolist()) == {1024}


@pytest.mark.parametrize("ny,accel", [(192, 8.0), (96, 4.0), (256, 12.0)])
def test_variable_density_lines(ny, accel):
    """round(N/R) full lines per frame; the centre block of max(4, round(N/(4R)))
    lines (centred coordinates, stored with DC at index 0) in every frame; the
    other lines redrawn per frame."""
    q, nx = 16, 32
    mask = synth.cartesian_lines_vd(np.random.default_rng(5), ny, nx, q, accel)
    L = _lines(mask, q, ny, nx)
    assert set(L.sum(1).tolist()) == {int(round(ny / accel))}
    nc = max(4, int(round(ny / (4 * accel))))
    centre = np.mod(np.arange(-(nc // 2), nc - nc // 2), ny)
    assert L[:, centre].all()
    assert len({tuple(np.flatnonzero(L[k])) for k in range(q)}) > 1
    # lines near the centre are drawn more often than those near the edge
    freq = L.mean(0)
    inner = freq[np.mod(np.arange(-ny // 8, ny // 8), ny)].mean()
    outer = freq[np.mod(np.arange(ny // 2 - ny // 8, ny // 2 + ny // 8), ny)].mean()
    assert inner > outer


def test_uniform_lines():
    q, ny, nx = 12, 64, 16
    mask = synth.cartesian_lines_uniform(np.random.default_rng(6), ny, nx, q, 4, 12)
    L = _lines(mask, q, ny, nx)
    assert set(L.sum(1).tolist()) == {16}
    assert L[:, [0, 1, ny - 2, ny - 1]].all()          # centre 4 lines: ky_c in {-2, -1, 0, 1}


def test_pseudo_radial_density():
    """256^2, 16 spokes, golden-angle rotation: about 3822 grid points per frame
    (17x acceleration) and 44% of k-space in the union over 64 frames."""
    m = synth.radial_golden(256, 256, 64, 16)
    assert abs(m.sum(1).mean() - 3822) < 5
    assert abs(m.any(0).mean() - 0.44) < 0.01
    assert m[:, 0].all()                                 # every spoke passes DC


@pytest.mark.parametrize("nc", [1, 4, 12, 20])
def test_coil_maps_unit_sum_of_squares(nc):
    smaps, modes, coef = synth.coil_maps(np.random.default_rng(7), 48, 64, nc)
    assert smaps.shape == (nc, 48 * 64)
    assert np.abs((np.abs(smaps) ** 2).sum(0) - 1).max() < 1e-12


def test_generation_is_deterministic_per_seed():
    spec = dict(kind="phantom", ny=32, nx=32, q=6, nc=3, rank=2, mask_kind="lines_vd", accel=4.0, noise=0.01)
    a, b = synth.make_problem(spec, seed=9), synth.make_problem(spec, seed=9)
    assert np.array_equal(a.y, b.y) and np.array_equal(a.mask, b.mask) and np.array_equal(a.smaps, b.smaps)
    c = synth.make_problem(spec, seed=10)
    assert not np.array_equal(a.y, c.y)
