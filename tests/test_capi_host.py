"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every entry point declared in include/ibmi.h, and rejects invalid plans before
touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2502_06377_gb300 import build as b
    b.build()
    from paper_2502_06377_gb300 import _lib
    return _lib.load()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(ibmi_\w+)\s*\(", txt))
    return names


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert "ibmi_invert" in names and "ibmi_plan" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_header(lib):
    from paper_2502_06377_gb300 import _lib
    assert declared_symbols() <= set(_lib.exported_symbols()) | set(getattr(_lib, "EXTRA_SYMBOLS", []))


def test_desc_defaults_and_status_strings(lib):
    import paper_2502_06377_gb300 as ibmi
    d = ibmi.ibmi_plan_desc_init(p=100)
    assert d.K == 2 and d.tol == 1e-10 and d.max_sweeps == 500 and d.check_every == 1
    assert ibmi.ibmi_status_string(0) == "IBMI_OK"
    assert ibmi.ibmi_status_string(2) == "IBMI_ERR_NOT_SPD"


@pytest.mark.parametrize("kw", [
    dict(p=1), dict(p=10, K=0), dict(p=10, K=11), dict(p=10, h=-1), dict(p=10, precision=7),
    dict(p=10, max_sweeps=0), dict(p=10, check_every=0), dict(p=10, tol=-1.0), dict(p=10, init=5),
])
def test_invalid_plans_rejected(lib, kw):
    import paper_2502_06377_gb300 as ibmi
    with pytest.raises(ibmi.IbmiError) as e:
        ibmi.ibmi_plan(**kw)
    assert e.value.status == ibmi.IBMI_ERR_INVALID_ARG


@pytest.mark.parametrize("lo,hi", [
    ([0, 60], [50, 100]),        # gap 50..60 not covered
    ([5, 40], [50, 100]),        # does not start at 0
    ([0, 40], [50, 90]),         # does not end at p
    ([0, 0], [50, 100]),         # not ascending
])
def test_invalid_explicit_sets(lib, lo, hi):
    import paper_2502_06377_gb300 as ibmi
    with pytest.raises(ibmi.IbmiError) as e:
        ibmi.ibmi_plan(100, lo=lo, hi=hi)
    assert e.value.status == ibmi.IBMI_ERR_INVALID_ARG


def test_batch_opts_and_plan_bytes(lib):
    import paper_2502_06377_gb300 as ibmi
    o = ibmi.ibmi_batch_opts_init()
    assert o.workers == 8 and o.autotune == 1 and o.graphs == 1 and o.tol == 1e-10 and o.precision == ibmi.IBMI_MIXED
    b = [ibmi.ibmi_plan_bytes(p, 4, 16, precision=ibmi.IBMI_MIXED) for p in (256, 1024, 4096)]
    assert b[0] < b[1] < b[2]
    assert ibmi.ibmi_plan_bytes(1) == 0


def test_batched_and_server_reject_invalid_without_gpu(lib):
    import ctypes as C
    assert lib.ibmi_invert_batched(-1, None, None, None, None, None, None, None) == 1
    h = C.c_void_p()
    assert lib.ibmi_serve_create(0, None, C.byref(h)) == 1
    assert lib.ibmi_serve_poll(None, 1, None, 0, None) == 1
