"""Product angular quadrature for the oracle (TEST INFRASTRUCTURE ONLY).

The paper's runs use level-symmetric S_n sets (S4 = 24 directions, Sec. VI-B);
the workloads here are product sets "n_polar Gauss-Legendre polar x n_azim
azimuthal per octant":

* polar cosines mu_i: the n_polar positive nodes of the 2*n_polar-point
  Gauss-Legendre rule on [-1, 1] (ascending), with their weights w_i (which
  sum to 1 on the half range);
* azimuths phi_j = (j + 1/2) (pi/2) / n_azim, each with weight pi / (2 n_azim);
* Omega = (s_x sqrt(1-mu^2) cos phi, s_y sqrt(1-mu^2) sin phi, s_z mu) with the
  octant signs; weight w_i * pi / (2 n_azim); total weight 4 pi;
* direction index m = octant * n_polar * n_azim + i * n_azim + j, octant bits
  (bit0, bit1, bit2) set when (x, y, z) is negative.

The Gauss-Legendre rule is numpy's (a library routine serves as this step).
"""

from __future__ import annotations

import numpy as np


def product_quadrature(n_polar: int, n_azim: int):
    """Return (dirs [M, 3], weights [M]) of the product set, M = 8 n_polar n_azim."""
    x, w = np.polynomial.legendre.leggauss(2 * n_polar)
    mu = x[n_polar:]
    wmu = w[n_polar:]
    phi = (np.arange(n_azim) + 0.5) * (0.5 * np.pi) / n_azim
    wphi = 0.5 * np.pi / n_azim
    M = 8 * n_polar * n_azim
    dirs = np.empty((M, 3))
    wts = np.empty(M)
    for octant in range(8):
        sx = -1.0 if octant & 1 else 1.0
        sy = -1.0 if octant & 2 else 1.0
        sz = -1.0 if octant & 4 else 1.0
        for i in range(n_polar):
            st = np.sqrt(1.0 - mu[i] * mu[i])
            for j in range(n_azim):
                m = octant * n_polar * n_azim + i * n_azim + j
                dirs[m] = (sx * st * np.cos(phi[j]), sy * st * np.sin(phi[j]), sz * mu[i])
                wts[m] = wmu[i] * wphi
    return dirs, wts
