"""Host-side logic of bench.py that decides reported figures: algorithmic bytes
per kernel launch, the clock record's parsing, and when ncu traffic is used."""
import os
import re

import bench
from paper_2212_09664_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_algorithmic_bytes_of_the_cardiac_workload():
    """complex64 = 8 B; n = 192 * 192 = 36864, q = 48, C = 12, r = 10 and
    n_u = 148 sampled rows x 192 = 28416 k-space entries kept per coil and rank."""
    p = synth.make_problem("cardiac192_q48_c12_r10")
    n_used = int(p.mask.reshape(p.q, p.ny, p.nx)[:, :, 0].any(0).sum())
    assert n_used == 148
    kb = {k: bench.kernel_bytes(k, p, 10, n_used) for k in bench.ITER_KERNELS}
    assert kb["k_fwd_cols"] == 8 * (368640 + 442368 + 3409920)      # U, maps, sampled rows out
    assert kb["k_row_gram"] == 8 * 3409920                           # sampled rows in
    assert kb["k_row_w"] == 8 * 2 * 3409920                          # sampled rows in and out
    assert kb["k_adj_cols"] == 8 * (3409920 + 442368 + 368640)       # rows, maps in; n x r out
    assert kb["k_gdqr"] == 8 * (6 * 368640 + 1769472) == 31850496   # Gk, U, Z B^H, Z in; grad, U_t+1, U_t out
    assert kb["k_zb"] == 8 * (1769472 + 368640)                      # Z in, Z B^H out
    assert kb["k_bstep"] == kb["k_row_w"] + kb["k_zb"]               # fused: rows in and out once, Z B^H
    sep = sum(v for k, v in kb.items() if k != "k_bstep")
    assert bench.iteration_bytes(p, 10, n_used, fused=False) == sep
    assert bench.iteration_bytes(p, 10, n_used, fused=True) == sep - kb["k_row_gram"]


class _FakeProc:
    def __init__(self, out):
        self.out = out

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.out, ""


def _sampler(rows):
    c = bench.ClockSampler.__new__(bench.ClockSampler)
    c.proc = _FakeProc("\n".join(rows) + "\n")
    return c


def test_clock_record_median_max_and_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    capped = "0, 1950, 2070, 1400.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1800, 2070, 1390.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    r = _sampler([ok, ok, capped]).stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]
    r = _sampler([ok, hot, "garbage line"]).stop()
    assert r["reasons"] == ["hw_thermal_slowdown"] and r["samples"] == 2


def test_ncu_traffic_only_for_unchanged_kernel_sources(monkeypatch):
    txt = open(os.path.join(ROOT, "profiles", "k_gdqr_cardiac192.md")).read()
    stated = float(re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt).group(1))
    if "source_sha: %s" % bench.source_sha() in txt:
        assert bench.ncu_traffic("k_gdqr") == stated
    monkeypatch.setattr(bench, "source_sha", lambda: "0" * 16)
    assert bench.ncu_traffic("k_gdqr") is None          # the kernel changed since the capture
    assert bench.ncu_traffic("k_not_profiled") is None
