"""CPU checks of the C ABI library: it builds, loads, exports every symbol the
header declares, and its host-only entry points agree with the oracle."""

import ctypes
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_1803_09876_gb300 import build as libbuild
from paper_1803_09876_gb300 import jsweep as J

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return J.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "jsweep.h")).read()
    return sorted(set(re.findall(r"^\s*(?:JSWEEP_API\s+)?(?:int|const char \*)\s*(jsweep_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 20
    assert sorted(J.EXPORTED) == syms
    for s in syms:
        assert hasattr(lib, s), s


def test_exports_nothing_else(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", libbuild.LIB], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported == set(header_symbols())


def test_bounds_checked_build_exports_the_same_symbols(lib):
    # the bounds-checked library (debug build) has the same ABI and says what it is
    import subprocess
    path = libbuild.build(bounds_check=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert exported == set(header_symbols())
    checked = ctypes.CDLL(path)
    assert checked.jsweep_bounds_checked() == 1
    assert lib.jsweep_bounds_checked() == 0
    assert lib.jsweep_bounds_error(None) == J.JSWEEP_ERR_INVALID_ARG
    w = ctypes.c_uint64(7)
    assert lib.jsweep_bounds_error(ctypes.byref(w)) == J.JSWEEP_OK and w.value == 0  # no device work


def test_version_and_options(lib):
    assert J.jsweep_version() >= 100
    o = J.jsweep_options_default()
    assert o.struct_size == ctypes.sizeof(J.jsweep_options)
    assert o.cluster_cells == 32 and o.spin_timeout_s > 0 and o.cycle_search_max == 256
    assert o.debug_block_waits == 0
    assert o.eager_search_max == 64 and o.patch_cells == 512
    assert o.no_face_stream == 0 and o.tail_units == 0


@pytest.mark.parametrize("npol,naz", [(1, 3), (2, 3), (3, 4), (4, 4), (6, 6), (8, 2)])
def test_product_quadrature_matches_oracle(lib, npol, naz):
    d, w = J.jsweep_quadrature_product(npol, naz)
    do, wo = oracle.product_quadrature(npol, naz)
    assert np.max(np.abs(d - do)) < 2e-15
    assert np.max(np.abs(w - wo)) < 2e-15
    assert abs(w.sum() - 4 * math.pi) < 1e-13


def test_quadrature_rejects_bad_sizes(lib):
    with pytest.raises(J.JsweepError) as e:
        J.jsweep_quadrature_product(0, 3)
    assert e.value.code == J.JSWEEP_ERR_INVALID_ARG
    assert "n_polar" in str(e.value)


def test_error_message_is_thread_local_and_cleared(lib):
    with pytest.raises(J.JsweepError):
        J.jsweep_quadrature_product(0, 0)
    J.jsweep_quadrature_product(1, 1)
    assert lib.jsweep_last_error() == b""


def test_multigroup_host_side_errors(lib):
    # argument checks of jsweep_source_iterate_mg return before any device work
    P = ctypes.c_void_p
    fake = P(16)  # never dereferenced: every call below fails its argument checks first
    f = lib.jsweep_source_iterate_mg
    assert f(None, 4, J.JSWEEP_F32, fake, fake, fake, None, 1e-6, 10, fake, None, None, None) == \
        J.JSWEEP_ERR_INVALID_ARG
    assert b"NULL argument" in lib.jsweep_last_error()
    assert f(fake, 4, J.JSWEEP_F32, fake, None, fake, None, 1e-6, 10, fake, None, None, None) == \
        J.JSWEEP_ERR_INVALID_ARG
    for G in (0, 9):
        assert f(fake, G, J.JSWEEP_F32, fake, fake, fake, None, 1e-6, 10, fake, None, None, None) == \
            J.JSWEEP_ERR_INVALID_ARG
        assert b"n_groups" in lib.jsweep_last_error()
    assert f(fake, 4, 7, fake, fake, fake, None, 1e-6, 10, fake, None, None, None) == J.JSWEEP_ERR_INVALID_ARG
    assert f(fake, 4, J.JSWEEP_F64, fake, fake, fake, None, -1.0, 10, fake, None, None, None) == \
        J.JSWEEP_ERR_INVALID_ARG
    assert f(fake, 4, J.JSWEEP_F64, fake, fake, fake, None, 1e-6, 0, fake, None, None, None) == \
        J.JSWEEP_ERR_INVALID_ARG


def test_batch_host_side_errors(lib):
    # host-only paths of the batch entry points (no device work is queued)
    P = ctypes.c_void_p
    h = P()
    assert lib.jsweep_batch_create(7, 1, None, ctypes.byref(h)) == J.JSWEEP_ERR_INVALID_ARG
    assert lib.jsweep_batch_create(J.JSWEEP_F32, 9, None, ctypes.byref(h)) == J.JSWEEP_ERR_INVALID_ARG
    assert lib.jsweep_batch_create(J.JSWEEP_F32, 2, None, ctypes.byref(h)) == J.JSWEEP_OK
    n = ctypes.c_int64(-1)
    assert lib.jsweep_batch_size(h, ctypes.byref(n)) == J.JSWEEP_OK and n.value == 0
    assert lib.jsweep_batch_query(h, 0, None, None, None) == J.JSWEEP_ERR_INVALID_ARG
    assert b"no problem with id 0" in lib.jsweep_last_error()
    assert lib.jsweep_batch_remove(h, 3) == J.JSWEEP_ERR_INVALID_ARG
    assert lib.jsweep_batch_add(h, None, None, None, None, None, None, 1e-6, 10, None, None) == \
        J.JSWEEP_ERR_INVALID_ARG
    assert lib.jsweep_batch_step(h, 0, None, None) == J.JSWEEP_ERR_INVALID_ARG
    # an empty batch has nothing to iterate
    assert lib.jsweep_batch_step(h, 1, ctypes.byref(n), None) == J.JSWEEP_OK and n.value == 0
    assert lib.jsweep_batch_source_iterate(h, None, None, None) == J.JSWEEP_OK
    a, b, nl = ctypes.c_double(-1), ctypes.c_double(-1), ctypes.c_int64(-1)
    assert lib.jsweep_batch_stats(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(nl), None, None) == J.JSWEEP_OK
    assert a.value == 0.0 and nl.value == 0
    assert lib.jsweep_batch_destroy(h) == J.JSWEEP_OK
    assert lib.jsweep_batch_destroy(None) == J.JSWEEP_OK
