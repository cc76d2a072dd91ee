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
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(jsweep_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    syms = header_symbols()
    assert len(syms) >= 20
    assert sorted(J.EXPORTED) == syms
    for s in syms:
        assert hasattr(lib, s), s


def test_version_and_options(lib):
    assert J.jsweep_version() >= 100
    o = J.jsweep_options_default()
    assert o.struct_size == ctypes.sizeof(J.jsweep_options)
    assert o.cluster_cells == 32 and o.spin_timeout_s > 0 and o.cycle_search_max == 256
    assert o.debug_block_waits == 0


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
