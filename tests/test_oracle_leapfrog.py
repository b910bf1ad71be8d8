"""Pins of the oracle integrator (O9, kick-drift-kick leapfrog with direct
forces) against facts that do not come from the oracle itself: free motion is
exact, a circular two-body orbit returns after one period with an O(dt^2)
phase error, energy errors shrink as dt^2, the scheme is time-reversible, and
momentum is conserved."""
import numpy as np
import pytest

import oracle as O
from paper_1005_5384_gb300 import workloads as W


def test_single_particle_moves_freely():
    x0 = np.array([[0.25, -1.0, 3.0]])
    v0 = np.array([[1.5, 0.5, -2.0]])
    x, v, a, phi = O.leapfrog(x0, v0, np.array([1.0]), 0.01, 0.125, 8)
    assert np.array_equal(v, v0) and np.allclose(x, x0 + v0 * 1.0, rtol=0, atol=1e-15)
    assert np.all(a == 0) and np.all(phi == 0)


def _circular_pair(eps):
    # two unit masses at distance d on a circular orbit: omega^2 d^3 = G M_tot (d^2/(d^2+eps^2))^(3/2)
    d = 1.0
    mtot = 2.0
    om = np.sqrt(mtot * d / (d * d + eps * eps) ** 1.5 / d)
    x = np.array([[-0.5, 0, 0], [0.5, 0, 0]], dtype=np.float64)
    v = np.array([[0, -0.5 * om, 0], [0, 0.5 * om, 0]], dtype=np.float64)
    return x, v, np.array([1.0, 1.0]), 2 * np.pi / om


@pytest.mark.parametrize("eps", [0.0, 0.1])
def test_circular_orbit_closes_with_second_order_error(eps):
    x0, v0, m, period = _circular_pair(eps)
    errs = []
    for k in (64, 128, 256):
        x, v, _, _ = O.leapfrog(x0, v0, m, eps, period / k, k)
        errs.append(np.abs(x - x0).max())
    assert errs[0] < 0.05
    # halving dt quarters the return error
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_energy_error_scales_as_dt_squared():
    x0, v0, m = W.plummer_pv(64, seed=5)
    e = []
    for dt in (1 / 64, 1 / 128):
        x, v, a, phi = O.leapfrog(x0, v0, m, 0.05, dt, int(0.5 / dt))
        _, phi0 = O.direct(x0, m, 0.05)
        E0 = sum(O.energies(v0, m, phi0))
        e.append(abs(sum(O.energies(v, m, phi)) - E0) / abs(E0))
    assert e[1] < 0.4 * e[0]


def test_time_reversible_and_momentum_conserving():
    x0, v0, m = W.plummer_pv(100, seed=7)
    x, v, _, _ = O.leapfrog(x0, v0, m, 0.05, 1 / 128, 40)
    xb, vb, _, _ = O.leapfrog(x, v, m, 0.05, -1 / 128, 40)
    assert np.abs(xb - x0).max() < 1e-11 and np.abs(vb - v0).max() < 1e-11
    p0 = (m[:, None] * v0).sum(0)
    p1 = (m[:, None] * v).sum(0)
    assert np.abs(p1 - p0).max() < 1e-13
