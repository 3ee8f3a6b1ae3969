"""Pins of the oracle on stretched vertical grids (layers of different
thickness; every element stays an axis-aligned box): node coupling, mass,
conservation, free stream and the convergence order carry over."""
import numpy as np
import pytest

from oracle import mesh, refstate, rhs, transfer, adapt
from synth.vortex import random_state, vortex_state
from tests.helpers import stretched_faces
from tests.test_oracle_mesh import two_level_leaves

PRM = refstate.Params()


def stretched_mesh(nc=True, nz=3, N=4, a=1.5, periodic=(True, True)):
    return mesh.OracleMesh(80e3, 80e3, 10e3, 4, 4, nz, N, periodic=periodic,
                           leaves=two_level_leaves() if nc else None,
                           z_faces=stretched_faces(10e3, nz, a))


def test_faces_and_layers():
    m = stretched_mesh()
    np.testing.assert_allclose(np.diff(m.zf), m.hzk)
    assert m.hzk[-1] > 2 * m.hzk[0]
    # element boxes follow the faces; lumped mass is the volume
    assert np.allclose(m.box[:, 4], m.zf[m.layer]) and np.allclose(m.box[:, 5], m.hzk[m.layer])
    assert abs(m.M.sum() - 80e3 * 80e3 * 10e3) < 1e-9 * 80e3 * 80e3 * 10e3
    with pytest.raises(ValueError):
        mesh.OracleMesh(80e3, 80e3, 10e3, 4, 4, 3, 4, z_faces=[0.0, 5e3, 4e3, 10e3])


def test_Q_reproduces_global_polynomials_on_stretched_layers():
    N = 4
    m = stretched_mesh(periodic=(False, False))
    rng = np.random.default_rng(9)
    C = rng.normal(size=(N + 1, N + 1))

    def f(X):
        # degree <= N in each of x, y, z
        x, y, z = X[..., 0] / 40e3, X[..., 1] / 40e3, X[..., 2] / 10e3
        return sum(C[a, b] * x ** a * y ** b * z ** ((a + b) % (N + 1))
                   for a in range(N + 1) for b in range(N + 1))

    qL = m.to_local(f(m.XG))[0]
    np.testing.assert_allclose(qL, f(m.X), rtol=0, atol=1e-11 * np.abs(f(m.X)).max())


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_rest_free_stream_and_conservation(eqset):
    m = stretched_mesh()
    assert np.all(rhs.rhs(m, np.zeros((5, m.NG)), PRM, eqset) == 0.0)
    prm = refstate.Params(f=0.0)
    ref = refstate.reference_state(m.XG[:, 2], prm)
    q = np.zeros((5, m.NG))
    q[1], q[2] = (7.0 * ref["rho0"], -3.0 * ref["rho0"]) if eqset == "C" else (7.0, -3.0)
    T = rhs.rhs(m, q, prm, eqset)
    scale = np.abs(rhs.rhs(m, random_state(m.XG, 10e3, 1, eqset), prm, eqset)).max(axis=1)
    assert np.all(np.abs(T).max(axis=1) <= 1e-12 * scale)
    T = rhs.rhs(m, random_state(m.XG, 10e3, 2, eqset), PRM, eqset)
    assert abs(np.sum(m.M * T[0])) <= 1e-13 * np.sum(np.abs(m.M * T[0]))


@pytest.mark.slow
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_manufactured_solution_convergence_on_stretched_layers(eqset):
    from tests.test_oracle_rhs import _mms
    e4, e8 = _mms(eqset, 4, stretch=1.0), _mms(eqset, 8, stretch=1.0)
    rate = np.log2(e4 / e8)
    assert np.all(e8 < 2e-3), e8
    assert np.all(rate >= 3.5), rate


def test_transfer_round_trip_on_stretched_layers():
    m = stretched_mesh(nc=False, nz=2)
    q = vortex_state(m.XG, 10e3)
    fl = np.zeros(m.Ne, dtype=np.int8)
    fl[: 4 * m.nz] = 1
    new, org = adapt.update_leaves(m.leaves, fl, m.nz, 4, 4, 2)
    m2, q2 = transfer.transfer(m, new, org, q)
    assert np.array_equal(m2.zf, m.zf)
    # a field linear in z is transferred exactly at the stretched heights
    lin = np.stack([m.XG[:, 2] * (k + 1) for k in range(5)])
    _, lin2 = transfer.transfer(m, new, org, lin)
    np.testing.assert_allclose(lin2, np.stack([m2.XG[:, 2] * (k + 1) for k in range(5)]),
                               atol=1e-9 * 10e3)
    back, org2 = adapt.update_leaves(m2.leaves, -np.ones(m2.Ne, dtype=np.int8), m2.nz, 4, 4, 2)
    m3, q3 = transfer.transfer(m2, back, org2, q2)
    np.testing.assert_allclose(q3, q, atol=1e-12 * np.abs(q).max())
