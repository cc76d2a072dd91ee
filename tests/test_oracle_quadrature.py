"""Pins of the oracle's product quadrature against closed forms and invariants."""

import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import product_quadrature


@pytest.mark.parametrize("npol,naz", [(1, 3), (2, 3), (3, 4), (4, 4), (6, 6)])
def test_moments(npol, naz):
    d, w = product_quadrature(npol, naz)
    assert d.shape == (8 * npol * naz, 3)
    assert np.all(w > 0)
    # total weight 4 pi
    assert abs(w.sum() - 4 * math.pi) < 1e-13
    # unit directions
    assert np.max(np.abs(np.linalg.norm(d, axis=1) - 1.0)) < 1e-15
    # first moments vanish, second moments (4 pi / 3) delta_ij
    assert np.max(np.abs(w @ d)) < 1e-13
    second = (d * w[:, None]).T @ d
    assert np.max(np.abs(second - (4 * math.pi / 3) * np.eye(3))) < 1e-13
    # polar moments: sum w mu^(2k) = 4 pi / (2k + 1), exact up to degree 4 npol - 1
    for k in range(0, 2 * npol):
        assert abs(np.sum(w * d[:, 2] ** (2 * k)) - 4 * math.pi / (2 * k + 1)) < 1e-12


def test_polar_nodes_are_legendre_roots():
    for npol in (1, 2, 3, 4, 6):
        d, _ = product_quadrature(npol, 3)
        mu = np.unique(np.round(np.abs(d[:, 2]), 15))
        assert mu.size == npol
        assert np.max(np.abs(eval_legendre(2 * npol, mu))) < 1e-13


def test_closed_form_nodes():
    # 2-point rule: mu = 1/sqrt(3); 4-point rule: sqrt(3/7 -+ 2/7 sqrt(6/5))
    d, _ = product_quadrature(1, 1)
    assert abs(abs(d[0, 2]) - 1 / math.sqrt(3)) < 1e-15
    d, w = product_quadrature(2, 1)
    mus = sorted(set(np.round(np.abs(d[:, 2]), 14)))
    ref = sorted([math.sqrt(3 / 7 - 2 / 7 * math.sqrt(6 / 5)), math.sqrt(3 / 7 + 2 / 7 * math.sqrt(6 / 5))])
    assert np.allclose(mus, ref, atol=1e-14, rtol=0)


def test_index_convention():
    npol, naz = 3, 4
    d, _ = product_quadrature(npol, naz)
    for octant in range(8):
        for i in range(npol):
            for j in range(naz):
                m = octant * npol * naz + i * naz + j
                s = np.sign(d[m])
                assert s[0] == (-1 if octant & 1 else 1)
                assert s[1] == (-1 if octant & 2 else 1)
                assert s[2] == (-1 if octant & 4 else 1)
                phi = math.atan2(abs(d[m, 1]), abs(d[m, 0]))
                assert abs(phi - (j + 0.5) * (math.pi / 2) / naz) < 1e-14
    # polar cosines ascend with i
    mu = np.abs(d[: npol * naz: naz, 2])
    assert np.all(np.diff(mu) > 0)
