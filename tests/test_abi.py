"""CPU checks of the C ABI: the library loads, exports every entry point the
header declares, and the host-side argument validation works without a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")
LIB = os.path.join(ROOT, "paper_2212_09664_gb300", "liblrccs.so")


def declared_functions():
    names = set()
    for h in os.listdir(HEADER_DIR):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(HEADER_DIR, h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(lrccs_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        import __graft_entry__

        __graft_entry__.build()
    return C.CDLL(LIB)


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("lrccs_create", "lrccs_init", "lrccs_iterate", "lrccs_get_factors", "lrccs_destroy",
                     "lrccs_last_error", "lrccs_synchronize"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True, check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    missing = declared_functions() - exported
    assert not missing, "declared but not exported: %s" % sorted(missing)
    for name in declared_functions():
        getattr(lib, name)


def test_default_params_are_the_papers(lib):
    import json

    from paper_2212_09664_gb300 import lrccs

    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    p = lrccs.default_params()
    assert p.trunc_factor == g["trunc_factor"]["value"]
    assert p.energy_pct == g["energy_pct"]["value"]
    assert p.eta_c == g["eta_c"]["value"]
    assert p.eps_exit == g["eps_exit"]["value"]
    assert p.t_max == g["t_max"]["value"]


@pytest.mark.parametrize("dims", [
    (48, 64, 8, 2, 2, 0),     # ny not a multiple of 32
    (64, 64, 0, 2, 2, 0),     # no frames
    (64, 64, 8, 2, 17, 0),    # rank above 16
    (64, 64, 8, 0, 2, 0),     # no coils
    (512, 64, 8, 1, 2, 0),    # side above 256
])
def test_create_rejects_dims_outside_scope(lib, dims):
    from paper_2212_09664_gb300 import lrccs

    with pytest.raises(lrccs.LrccsError) as ei:
        lrccs.lrccs_create(*dims)
    assert ei.value.status == lrccs.E_INVALID
    assert "scope" in str(ei.value)


def test_status_strings(lib):
    from paper_2212_09664_gb300 import lrccs

    for s in range(9):
        assert lrccs._lib.lrccs_status_string(s)


def test_null_context_is_rejected_before_any_device_work(lib):
    """Every entry point that takes a context checks it before touching CUDA."""
    from paper_2212_09664_gb300 import lrccs

    L = lrccs._lib
    n = C.c_size_t(0)
    assert L.lrccs_iterate(None, 1, None) == lrccs.E_INVALID
    assert L.lrccs_set_subspace(None, None, 1, 0.0) == lrccs.E_INVALID
    assert L.lrccs_track_minibatch(None, None, None, None, None, 5, 0, None, None) == lrccs.E_INVALID
    assert L.lrccs_get_state(None, None, C.byref(n)) == lrccs.E_INVALID
    assert L.lrccs_set_state(None, b"x" * 64, 64) == lrccs.E_INVALID


def test_noalloc_wrapper_validates_before_any_launch(lib):
    """The allocation-free threshold's binding refuses, before calling the
    library, every argument that would let the kernel read outside y: a wrong
    dtype, a count above y.numel(), a gamma_out that is not float64, and
    tensors that are not on the current CUDA device."""
    import torch

    from paper_2212_09664_gb300 import lrccs

    y = torch.zeros(8, dtype=torch.complex64)
    g = torch.zeros(1, dtype=torch.float64)
    bad = [
        (torch.zeros(8, dtype=torch.complex128), 8, g),      # not complex64
        (y, 9, g),                                            # count above y.numel()
        (y, 0, g),                                            # empty count
        (y, 8, torch.zeros(1, dtype=torch.float32)),          # gamma_out not float64
        (y, 8, torch.zeros(0, dtype=torch.float64)),          # no room for gamma
        (y, 8, g),                                            # host tensors, not CUDA
    ]
    for yy, cnt, gg in bad:
        with pytest.raises(ValueError):
            lrccs.lrccs_trunc_threshold_noalloc(yy, cnt, 36.0, gg)


def test_context_bytes_without_a_gpu(lib):
    """lrccs_context_bytes sizes a context from its dims alone (no allocation):
    it grows with q, C and the rank, and covers at least Z, X0 and the
    transform work buffer (complex64)."""
    from paper_2212_09664_gb300 import lrccs

    b = lrccs.lrccs_context_bytes(192, 192, 48, 12, 10)
    n = 192 * 192
    assert b >= 8 * (2 * n * 48 + 12 * n * 10)
    assert lrccs.lrccs_context_bytes(192, 192, 96, 12, 10) > b
    assert lrccs.lrccs_context_bytes(192, 192, 48, 20, 10) > b
    assert lrccs.lrccs_context_bytes(192, 192, 48, 12, 14) > b


@pytest.mark.parametrize("prec", [3, 7, -1])
def test_unknown_precision_forms_are_refused(lib, prec):
    from paper_2212_09664_gb300 import lrccs

    with pytest.raises(lrccs.LrccsError) as ei:
        lrccs.lrccs_create(64, 64, 8, 2, 2, precision=prec)
    assert ei.value.status == lrccs.E_UNSUPPORTED


def test_ticket_calls_reject_unknown_tickets_without_a_context(lib):
    from paper_2212_09664_gb300 import lrccs

    L = lrccs._lib
    t = lrccs.Ticket(1)
    d = C.c_int32(0)
    assert L.lrccs_ticket_query(None, C.byref(t), C.byref(d)) == lrccs.E_INVALID
    assert L.lrccs_ticket_wait(None, C.byref(t)) == lrccs.E_INVALID
    assert L.lrccs_track_minibatch_async(None, None, None, None, None, 5, 0, None, C.byref(t)) == lrccs.E_INVALID
