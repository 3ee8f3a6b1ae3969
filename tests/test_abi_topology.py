"""CPU checks of the C ABI library: it loads, exports every declared symbol,
and its host topology (numbering, hanging rows, lumped mass, adaptation) agrees
with the oracle's brute-force construction (Sec. 3.1-3.2)."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import adapt, mesh as om
from tests.helpers import node_perm
from tests.test_oracle_mesh import ring_leaves, two_level_leaves

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sem():
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


def test_library_exports_every_declared_symbol(sem):
    hdr = open(os.path.join(ROOT, "include", "sem.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(sem_\w+)\s*\(", hdr, re.M))
    assert "sem_rhs" in declared and "sem_transfer" in declared
    for name in declared:
        assert hasattr(sem.LIB, name), name
    assert declared == set(sem.EXPORTS)


def _lib_Q(sem, m):
    """Full constraint matrix Q rebuilt from the library's host export."""
    hmap, hh, hw = sem.sem_mesh_hmap_host(m)
    leaves = sem.sem_mesh_leaves_host(m)
    N, NZ, nz = m.N, m.NZ, m.nz
    n1 = N + 1
    rows, cols, vals = [], [], []
    ii, jj, kk = np.meshgrid(np.arange(n1), np.arange(n1), np.arange(n1), indexing="ij")
    ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
    lidx = ii + n1 * jj + n1 * n1 * kk
    for c in range(m.Ncol):
        for k in range(nz):
            base = (c * nz + k) * n1 ** 3
            for i, j, kq, l in zip(ii, jj, kk, lidx):
                v = hmap[c, i + n1 * j]
                kz = k * N + kq
                if v >= 0:
                    rows.append(base + l); cols.append(v * NZ + kz); vals.append(1.0)
                else:
                    for q in range(n1):
                        if hw[-1 - v, q] != 0.0:
                            rows.append(base + l); cols.append(hh[-1 - v, q] * NZ + kz)
                            vals.append(hw[-1 - v, q])
    return sp.csr_matrix((vals, (rows, cols)), shape=(m.Ne * n1 ** 3, m.NG)), leaves


def _compare_with_oracle(sem, L, nx, nz, N, leaves, periodic, z_faces=None):
    m = sem.sem_mesh_create(L, L, 10e3, nx, nx, nz, N, leaves=leaves, periodic=periodic, lvl_max=4,
                            z_faces=z_faces)
    o = om.OracleMesh(L, L, 10e3, nx, nx, nz, N, leaves=leaves, periodic=periodic, z_faces=z_faces)
    assert m.NG == o.NG
    perm = node_perm(sem.sem_mesh_coords_host(m), o.XG)
    Q, lv = _lib_Q(sem, m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    erow = np.concatenate([np.arange((oleaf[tuple(l)] * nz + k) * o.P,
                                     (oleaf[tuple(l)] * nz + k + 1) * o.P)
                           for l in lv for k in range(nz)])
    coo = Q.tocoo()
    Qo = sp.csr_matrix((coo.data, (erow[coo.row], perm[coo.col])), shape=o.Q.shape)
    assert abs(Qo - o.Q).max() < 1e-13
    M = sem.sem_mesh_mass_host(m)
    np.testing.assert_allclose(M, o.M[perm], rtol=1e-13)
    return m, o


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("periodic", [(True, True), (False, False), (True, False)])
def test_topology_matches_oracle_two_level(sem, N, periodic):
    _compare_with_oracle(sem, 80e3, 4, 2, N, two_level_leaves(), periodic)


@pytest.mark.parametrize("N", [3, 4])
def test_topology_matches_oracle_stretched_layers(sem, N):
    """Layer faces of a stretched grid: same numbering, Q and lumped mass as
    the oracle's, and the z levels of the nodes follow the faces."""
    from tests.helpers import stretched_faces
    zf = stretched_faces(10e3, 3, 1.5)
    m, o = _compare_with_oracle(sem, 80e3, 4, 3, N, two_level_leaves(), (True, True), z_faces=zf)
    z = np.unique(np.round(sem.sem_mesh_coords_host(m)[2], 6))
    assert np.allclose(z[::N], zf)
    with pytest.raises(sem.SemError) as e:
        sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 3, 4, z_faces=[0.0, 6e3, 5e3, 10e3])
    assert e.value.code == sem.SEM_ERR_ARG


@pytest.mark.parametrize("seed", range(4))
def test_topology_matches_oracle_random_balanced(sem, seed):
    rng = np.random.default_rng(100 + seed)
    leaves = [(0, i, j) for j in range(3) for i in range(3)]
    for _ in range(5):
        fl = rng.integers(-1, 2, size=len(leaves)).astype(np.int8)
        leaves, _ = adapt.update_leaves(leaves, fl, 1, 3, 3, 3)
    _compare_with_oracle(sem, 90e3, 3, 1, 3 + seed % 2, leaves, (True, True))


@pytest.mark.parametrize("seed", range(6))
def test_adaptation_plan_matches_oracle(sem, seed):
    rng = np.random.default_rng(seed)
    nx, nz = 4, 2
    leaves = [(0, i, j) for j in range(nx) for i in range(nx)]
    for _ in range(3):
        fl = rng.integers(-1, 2, size=len(leaves)).astype(np.int8)
        leaves, _ = adapt.update_leaves(leaves, fl, 1, nx, nx, 3)
    m = sem.sem_mesh_create(80e3, 80e3, 10e3, nx, nx, nz, 4, leaves=leaves, lvl_max=3)
    lv = [tuple(x) for x in sem.sem_mesh_leaves_host(m)]
    flags = rng.integers(-1, 2, size=len(lv) * nz).astype(np.int8)
    new_lib = sem.sem_transfer_plan(m, flags)
    new_oracle, _ = adapt.update_leaves(lv, flags, nz, nx, nx, 3)
    got = sorted(tuple(x) for x in sem.sem_mesh_leaves_host(new_lib))
    assert got == sorted(new_oracle)


def test_rejects_bad_meshes(sem):
    with pytest.raises(sem.SemError) as e:     # level 0 next to level 2
        sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4,
                            leaves=[(0, 1, 0), (0, 0, 1), (0, 1, 1), (1, 1, 0), (1, 0, 1), (1, 1, 1)]
                            + [(2, a, b) for a in (0, 1) for b in (0, 1)])
    assert e.value.code == sem.SEM_ERR_TOPOLOGY
    with pytest.raises(sem.SemError) as e:     # a hole
        sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4, leaves=[(0, 0, 0), (0, 1, 0), (0, 0, 1)])
    assert e.value.code == sem.SEM_ERR_TOPOLOGY
    with pytest.raises(sem.SemError) as e:
        sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 9)
    assert e.value.code == sem.SEM_ERR_UNSUPPORTED
    m = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4)
    with pytest.raises(sem.SemError) as e:     # flags outside {-1, 0, 1}
        sem.sem_transfer_plan(m, np.full(m.Ne, 3, dtype=np.int8))
    assert e.value.code == sem.SEM_ERR_ARG


def test_autotune_select_rejects_rows_outside_the_table(sem):
    m = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4)
    sem.sem_autotune_select(m, -1)
    sem.sem_autotune_select(m, 0)
    for bad in (-2, 16, 1000):
        with pytest.raises(sem.SemError) as e:
            sem.sem_autotune_select(m, bad)
        assert e.value.code == sem.SEM_ERR_ARG
    # the paper's set has its own table (four order-4 rows)
    for row in (-1, 0, 3):
        sem.sem_autotune_select(m, row, eqset=1)
    for bad in (-2, 4, 16):
        with pytest.raises(sem.SemError) as e:
            sem.sem_autotune_select(m, bad, eqset=1)
        assert e.value.code == sem.SEM_ERR_ARG
    with pytest.raises(sem.SemError) as e:     # no such equation set
        sem.sem_autotune_select(m, 0, eqset=2)
    assert e.value.code == sem.SEM_ERR_ARG
    # warped layers: the paper's set keeps its four rows, the conservative set
    # its line-exchange rows only (five at order 4)
    w = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 2, 4, warp=(500.0, 1, 1))
    for row in (-1, 0, 3):
        sem.sem_autotune_select(w, row, eqset=1)
    sem.sem_autotune_select(w, 4, eqset=0)
    for eq, bad in ((1, 4), (0, 5)):
        with pytest.raises(sem.SemError) as e:
            sem.sem_autotune_select(w, bad, eqset=eq)
        assert e.value.code == sem.SEM_ERR_ARG


@pytest.mark.parametrize("N,n_c,n_nc", [(2, 3, 1), (3, 4, 1), (4, 10, 4), (5, 3, 1), (6, 3, 1)])
def test_variant_tables_per_order_and_set(sem, N, n_c, n_nc):
    """Every compiled order has rows in both equation sets' variant tables
    (the conservative set's z-pencil and line-exchange kernels, and order 4's
    tensor-core and TMA variants; the paper's set's line-exchange kernels):
    the last row is accepted, the one after it refused (host only)."""
    m = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, N)
    for eq, n in ((0, n_c), (1, n_nc)):
        sem.sem_autotune_select(m, n - 1, eqset=eq)
        with pytest.raises(sem.SemError) as e:
            sem.sem_autotune_select(m, n, eqset=eq)
        assert e.value.code == sem.SEM_ERR_ARG


def test_uniform_counts_and_info(sem):
    m = sem.sem_mesh_create(2048e3, 2048e3, 24e3, 64, 64, 16, 4)
    assert (m.Ne, m.NG, m.NH, m.NZ) == (65536, 4259840, 65536, 65)
    assert m.info.NL == 8192000
    assert m.info.n_hanging_h == 0


def _fake_checkpoint(path, ncol_leaves, NG, corrupt=None, warp=(0.0, 0, 0), version=3):
    """A checkpoint file in the library's layout (header with the warped-layer
    parameters, leaves, layer faces, state, FNV-1a)."""
    import struct
    head = struct.pack("<8s4d8i3q", b"SEMCKPT%d" % version, 80e3, 80e3, 10e3, 1.5, 2, 2, 1, 4, 1, 1, 0, 0,
                       len(ncol_leaves), NG, 7)
    if version >= 3:
        head += struct.pack("<d2i", float(warp[0]), int(warp[1]), int(warp[2]))
    leaves = np.asarray(ncol_leaves, dtype=np.int32).tobytes()
    faces = np.array([0.0, 10e3]).tobytes()
    state = np.arange(5 * NG, dtype=np.float64).tobytes()
    h = 1469598103934665603
    for b in head + leaves + faces + state:
        h ^= b
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    data = head + leaves + faces + state + struct.pack("<Q", h)
    if corrupt == "truncate":
        data = data[:-100]
    elif corrupt == "flip":
        data = data[:200] + bytes([data[200] ^ 1]) + data[201:]
    with open(path, "wb") as f:
        f.write(data)


def test_checkpoint_reading_rejects_bad_files(sem, tmp_path):
    leaves = [(0, i, j) for j in range(2) for i in range(2)]
    m = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4)
    good = tmp_path / "good.ckpt"
    _fake_checkpoint(good, leaves, m.NG)
    m2, t, s = sem.sem_checkpoint_read_mesh(good)
    assert (m2.NG, t, s) == (m.NG, 1.5, 7)
    for mode in ("truncate", "flip"):
        bad = tmp_path / f"{mode}.ckpt"
        _fake_checkpoint(bad, leaves, m.NG, corrupt=mode)
        with pytest.raises(sem.SemError) as e:
            sem.sem_checkpoint_read_mesh(bad)
        assert e.value.code == sem.SEM_ERR_IO
    with pytest.raises(sem.SemError) as e:
        sem.sem_checkpoint_read_mesh(tmp_path / "missing.ckpt")
    assert e.value.code == sem.SEM_ERR_IO
    garbage = tmp_path / "garbage.ckpt"
    garbage.write_bytes(b"\x00" * 300)
    with pytest.raises(sem.SemError) as e:
        sem.sem_checkpoint_read_mesh(garbage)
    assert e.value.code == sem.SEM_ERR_IO
    old = tmp_path / "v2.ckpt"                 # the format before warped layers
    _fake_checkpoint(old, leaves, m.NG, version=2)
    with pytest.raises(sem.SemError) as e:
        sem.sem_checkpoint_read_mesh(old)
    assert e.value.code == sem.SEM_ERR_IO and "earlier version" in str(e.value)


def test_checkpoint_of_a_warped_mesh_rebuilds_it(sem, tmp_path):
    """The warped-layer parameters travel in the checkpoint: the mesh read
    back has the warped node heights of the mesh that wrote it."""
    leaves = [(0, i, j) for j in range(2) for i in range(2)]
    w = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4, warp=(300.0, 1, 1))
    path = tmp_path / "warped.ckpt"
    _fake_checkpoint(path, leaves, w.NG, warp=(300.0, 1, 1))
    m2, t, s = sem.sem_checkpoint_read_mesh(path)
    np.testing.assert_array_equal(sem.sem_mesh_coords_host(m2), sem.sem_mesh_coords_host(w))
    box = sem.sem_mesh_create(80e3, 80e3, 10e3, 2, 2, 1, 4)
    assert np.abs(sem.sem_mesh_coords_host(m2)[2] - sem.sem_mesh_coords_host(box)[2]).max() > 50.0


def test_one_time_setup_runs_once_per_device(sem):
    """Constant tables and kernel attributes belong to a device: the library's
    one-time set-up must run once for each device ordinal (not once per
    process), also when several host threads make their first call at once."""
    assert sem.sem_selftest_device_once(8, 16) == [1] * 8
    assert sem.sem_selftest_device_once(64, 4) == [1] * 64
    with pytest.raises(sem.SemError):
        sem.sem_selftest_device_once(65, 1)


@pytest.mark.parametrize("nonconforming", [False, True])
def test_warped_mesh_host_tables_match_oracle(sem, nonconforming):
    """Warped layers: the library's node heights (coordinates) and per-node
    lumped mass equal the oracle's isoparametric construction."""
    leaves = two_level_leaves() if nonconforming else None
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=leaves, warp=(700.0, 1, 2))
    o = om.OracleMesh(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=leaves, warp=(700.0, 1, 2))
    xyz = sem.sem_mesh_coords_host(m)
    perm = node_perm(xyz, o.XG)
    np.testing.assert_allclose(xyz.T, o.XG[perm], rtol=0, atol=1e-9)
    np.testing.assert_allclose(sem.sem_mesh_mass_host(m), o.M[perm], rtol=1e-13)
    assert np.abs(xyz[2] - o.XG_box[perm, 2]).max() > 300.0


def test_warped_mesh_refusals(sem):
    with pytest.raises(sem.SemError):        # folds the elements
        sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, warp=(6000.0, 1, 1))
    m = sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, warp=(700.0, 1, 1), lvl_max=2)
    with pytest.raises(sem.SemError) as e:   # adaptation of warped meshes is not built
        sem.sem_transfer_plan(m, np.ones(m.Ne, dtype=np.int8))
    assert e.value.code == sem.SEM_ERR_UNSUPPORTED
