"""CPU checks of the C ABI: the library loads, exports every function that
include/porta.h declares, and rejects invalid arguments before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "porta.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(porta_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_1307_4217_gb300 as P
    L = P.lib()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n


def test_binding_has_the_c_names():
    import paper_1307_4217_gb300 as P
    for n in _declared():
        assert hasattr(P, n), n


def test_create_rejects_invalid_arguments_without_gpu():
    import paper_1307_4217_gb300 as P
    from paper_1307_4217_gb300.binding import _Grid, _Atom, _Quad, _Opts
    z = np.linspace(0, 1, 4)
    good = dict(g=_Grid(4, 4, 4, 1.0, 1.0, z.ctypes.data), a=_Atom(0, 0.0, 1.0, 25.0), q=_Quad(2, 4, 3, 4.0),
                o=_Opts(P.PORTA_FP32, 0, 0))
    bad_cases = [
        dict(good, g=_Grid(0, 4, 4, 1.0, 1.0, z.ctypes.data)),
        dict(good, g=_Grid(4, 4, 1, 1.0, 1.0, z.ctypes.data)),
        dict(good, g=_Grid(4, 4, 4, -1.0, 1.0, z.ctypes.data)),
        dict(good, g=_Grid(4, 4, 4, 1.0, 1.0, np.array([0, 1, 1, 2.0]).ctypes.data)),
        dict(good, a=_Atom(7, 0.0, 1.0, 25.0)),
        dict(good, q=_Quad(0, 4, 3, 4.0)),
        dict(good, q=_Quad(2, 4, 0, 4.0)),
        dict(good, o=_Opts(5, 0, 0)),
        dict(good, a=_Atom(1, 0.0, 1.0, 0.0)),
    ]
    for case in bad_cases:
        rc, h = P.porta_create(case["g"], case["a"], case["q"], case["o"])
        assert rc == P.PORTA_EINVAL
        assert not h.value


def test_null_context_calls_fail_cleanly():
    import paper_1307_4217_gb300 as P
    L = P.lib()
    assert L.porta_formal_solve(None) == P.PORTA_EINVAL
    assert L.porta_see_update(None, None) == P.PORTA_EINVAL
    assert L.porta_last_error(None) == b"null context"
    L.porta_destroy(None)


def test_product_path_has_no_oracle_import():
    """The CUDA package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1307_4217_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "oracle.h" not in txt, f


def test_capped_allocator_reports_enomem_without_gpu():
    """A device-memory cap below a context's needs makes porta_create fail with
    PORTA_ENOMEM before the CUDA runtime is asked for memory (so this runs on a
    host without a GPU); lifting the cap restores the default."""
    import paper_1307_4217_gb300 as P
    from paper_1307_4217_gb300.binding import _Grid, _Atom, _Quad, _Opts
    z = np.linspace(0, 1, 4)
    before = P.porta_device_bytes()
    assert P.porta_set_device_limit(1024) == P.PORTA_OK
    try:
        rc, h = P.porta_create(_Grid(4, 4, 4, 1.0, 1.0, z.ctypes.data), _Atom(0, 0.0, 1.0, 25.0),
                               _Quad(2, 4, 3, 4.0), _Opts(P.PORTA_FP32, 0, 0))
        assert rc == P.PORTA_ENOMEM
        assert not h.value
        assert P.porta_device_bytes() == before
    finally:
        assert P.porta_set_device_limit(0) == P.PORTA_OK
    assert P.porta_set_device_limit(-1) == P.PORTA_EINVAL
