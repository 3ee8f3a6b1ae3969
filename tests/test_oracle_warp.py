"""Pins of the oracle's non-affine (warped-layer) elements: the general
isoparametric metric (Sec. 3's tensor-product LGL basis on curved
hexahedra), against what the geometry and the mathematics fix:

- without displacement the general metric reproduces the closed-form box
  operators and the same tendency;
- the metric differentiates the coordinates exactly: G_d x_e = delta_de at
  every node (a wrong inverse, a transposed Jacobian or a missing term fails);
- the lumped mass sums to the volume, which the warp leaves unchanged (the
  lids stay flat), and the lid nodes stay at z = 0 and z = Lz;
- the discrete metric identities: the assembled weak divergence of a
  constant flux vanishes to round-off on a warped conforming mesh (the
  free-stream condition); at 2:1 faces of curved elements it leaves the
  face quadrature error, which falls with the warp's amplitude;
- the rest state stays exactly at rest; mass and (rho theta)' are conserved
  to round-off across 2:1 faces of a warped mesh;
- the manufactured solution converges at about the order of the basis on
  warped meshes.
"""
import numpy as np
import pytest

from oracle import mesh, refstate, rhs
from synth.vortex import random_state
from tests.test_oracle_mesh import two_level_leaves
from tests.test_oracle_rhs import _mms

PRM = refstate.Params()
WARP = (700.0, 1, 1)


def warped_nc_mesh(warp=WARP):
    return mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves(), warp=warp)


def test_zero_warp_reproduces_the_box_operators():
    box = mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves())
    flat = warped_nc_mesh((0.0, 1, 1))
    for lev, es, G in box.op_groups():
        for e in es:
            for d in range(3):
                np.testing.assert_allclose(flat.G_elem[e, d], G[d], rtol=1e-12, atol=1e-12 * np.abs(G[d]).max())
    np.testing.assert_allclose(flat.wJ, box.wJ, rtol=1e-13)
    q = random_state(box.XG, 12e3, 3)
    np.testing.assert_allclose(rhs.rhs(flat, q, PRM), rhs.rhs(box, q, PRM), rtol=1e-11, atol=1e-12 *
                               np.abs(rhs.rhs(box, q, PRM)).max())


def test_metric_differentiates_coordinates_exactly():
    m = warped_nc_mesh()
    assert np.abs(m.X[:, :, 2] - np.repeat(m.X[:, :, 2].mean(axis=1, keepdims=True), m.P, 1)).max() > 0
    for e in range(m.Ne):
        for d in range(3):
            for c in range(3):
                want = 1.0 if c == d else 0.0
                got = m.G_elem[e, d] @ m.X[e, :, c]
                assert np.abs(got - want).max() <= 1e-12, (e, d, c)


def test_volume_and_flat_lids():
    m = warped_nc_mesh()
    assert abs(m.M.sum() - 300e3 * 300e3 * 12e3) <= 1e-12 * 300e3 * 300e3 * 12e3
    zs = m.XG[:, 2]
    assert np.count_nonzero(m.z_bottom) == np.count_nonzero(np.abs(m.XG_box[:, 2]) < 1e-6)
    assert np.count_nonzero(m.z_top) == np.count_nonzero(np.abs(m.XG_box[:, 2] - 12e3) < 1e-6)
    # interior nodes really move
    assert np.abs(zs - m.XG_box[:, 2]).max() > 0.5 * WARP[0]


def _const_flux_residual(m, Fc):
    r = np.zeros((m.Ne, m.P))
    for lev, es, G in m.op_groups():
        r[es] = sum((m.wJ[es] * Fc[d]) @ G[d] for d in range(3))
    return m.assemble(r[None])[0], np.abs(r).max()


def test_weak_divergence_of_constant_flux_vanishes_on_conforming_warped_mesh():
    """The discrete metric identities: exact free stream (round-off) on a
    warped conforming mesh, for every direction of a constant flux (the lid
    faces carry the normal flux of the z component)."""
    m = mesh.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, warp=WARP)
    interior = ~(m.z_bottom | m.z_top)
    for Fc in ((1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (3.0, -2.0, 0.5)):
        R, scale = _const_flux_residual(m, Fc)
        assert np.abs(R[interior]).max() <= 1e-12 * scale, Fc
        if Fc[2] == 0.0:
            assert np.abs(R).max() <= 1e-12 * scale, Fc


def test_free_stream_error_at_curved_2to1_faces_is_the_face_quadrature_error():
    """At a 2:1 face of curved elements the two sides' face integrals of basis
    function x metric (degree 2N along the face) are LGL quadratures of
    different points, exact only to degree 2N - 1: the constant-flux residual
    is not zero there, only small, and it shrinks with the warp's amplitude
    (to round-off for boxes); it is zero away from the 2:1 faces."""
    errs = []
    for A in (700.0, 350.0, 175.0, 0.0):
        m = warped_nc_mesh((A, 1, 1))
        R, scale = _const_flux_residual(m, (1.0, 0.0, 0.0))
        errs.append(np.abs(R).max() / scale)
        if A == 700.0:
            # global nodes that no hanging node is interpolated from: off the 2:1 faces
            hang_rows = np.nonzero(m.hang_of >= 0)[0]
            on_face = np.zeros(m.NG, dtype=bool)
            on_face[m.Q[hang_rows].nonzero()[1]] = True
            assert np.count_nonzero(on_face) > 0
            assert np.abs(R[~on_face]).max() <= 1e-12 * scale
    assert errs[0] <= 1e-4, errs
    assert errs[1] < 0.6 * errs[0] and errs[2] < 0.6 * errs[1], errs
    assert errs[3] <= 1e-13, errs


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_rest_state_exactly_steady_on_warped_mesh(eqset):
    m = warped_nc_mesh()
    assert np.all(rhs.rhs(m, np.zeros((5, m.NG)), PRM, eqset) == 0.0)


@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_mass_conserved_on_warped_nonconforming_mesh(eqset):
    m = warped_nc_mesh()
    T = rhs.rhs(m, random_state(m.XG, 12e3, 2, eqset), PRM, eqset)
    assert abs(np.sum(m.M * T[0])) <= 1e-13 * np.sum(np.abs(m.M * T[0]))
    if eqset == "C":
        assert abs(np.sum(m.M * T[4])) <= 1e-13 * np.sum(np.abs(m.M * T[4]))


@pytest.mark.slow
@pytest.mark.parametrize("eqset", ["C", "NC"])
def test_manufactured_solution_convergence_on_warped_mesh(eqset):
    """Measured 3.26 (mass, (rho theta)') to 3.94 (momentum) from 4^3 to 8^3
    elements against 3.9 on boxes: the metric is itself an interpolant and
    the integrands' degree grows, so the pre-asymptotic rate is lower."""
    e4, e8 = _mms(eqset, 4, warp=(500.0, 1, 1)), _mms(eqset, 8, warp=(500.0, 1, 1))
    rate = np.log2(e4 / e8)
    assert np.all(e8 < 2e-3), e8
    assert np.all(rate >= 3.0), rate
