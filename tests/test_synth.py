"""Checks of the seeded input generator (vortex of Sec. 4, noise, keys)."""
import numpy as np

from synth.vortex import (VortexSpec, gaussian_vortex_scale, splitmix64_uniform,
                          tangential_wind, vortex_state)


def test_gaussian_vortex_reproduces_paper_constants():
    """Sec. 4: a Gaussian vorticity with peak 1.5e-3 1/s and maximum winds at
    50 km gives about 21.5 m/s.  With the closed-form wind profile the value
    is 21.35 m/s, within 1 % of the stated one."""
    L, zeta0, x = gaussian_vortex_scale(21.5, 50e3)
    assert abs(x - 1.12091) < 1e-5
    v = 1.5e-3 * L * L / (2 * 50e3) * (1 - np.exp(-(50e3 / L) ** 2))
    assert abs(v - 21.35) < 0.01
    assert abs(zeta0 - 1.5e-3) / 1.5e-3 < 0.01


def test_profile_maximum_and_decay():
    s = VortexSpec()
    r = np.linspace(0, 300e3, 3001)
    v = tangential_wind(r, 0.0, s)
    assert abs(r[np.argmax(v)] - 50e3) < 200.0
    assert abs(v.max() - 20.0) < 0.05
    ratio = tangential_wind(50e3, 5823.0 * np.sqrt(2.0), s) / tangential_wind(50e3, 0.0, s)
    assert abs(ratio - np.exp(-1.0)) < 1e-14


def test_noise_is_keyed_by_coordinates():
    xyz = np.array([[0.0, 1.0, 2.0], [5.0, 6.0, 7.0], [0.0, 1.0, 2.0]])
    u = splitmix64_uniform(1, xyz)
    assert u[0] == u[2] and u[0] != u[1] and np.all((u >= 0) & (u < 1))
    perm = splitmix64_uniform(1, xyz[::-1])
    assert np.array_equal(perm, u[::-1])


def test_state_independent_of_node_order():
    rng = np.random.default_rng(0)
    xyz = np.stack([rng.uniform(-3e5, 3e5, 50), rng.uniform(-3e5, 3e5, 50),
                    rng.uniform(0, 24e3, 50)], 1)
    q = vortex_state(xyz, 24e3)
    p = rng.permutation(50)
    assert np.array_equal(vortex_state(xyz[p], 24e3, Rmax=5e5), vortex_state(xyz, 24e3, Rmax=5e5)[:, p])
    assert np.all(np.isfinite(q))
