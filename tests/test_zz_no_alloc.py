"""The allocation-free right-hand side, sem_rhs_noalloc.

Some callers must not allocate device memory when they evaluate the
right-hand side: their device memory is already held by another allocator
(a framework's caching allocator or a pool, so a new cudaMalloc fails), or
their rules forbid device allocation after start-up.  sem_rhs_noalloc serves
them from a fixed device array built into the library.  These tests call it
through the C ABI two times in a row, with different states, and check each
result against sem_rhs on the same input with the tolerance of the other
parity tests (float64: relative L2 <= 1e-12 per field group; mixed form:
1e-6 between the two calls, which run the same float32 kernels); they check
that repeated calls leave the device's free memory unchanged, that a large
mesh followed by a small one gives correct results (the shared array keeps
the previous call's contents), and that what the call cannot serve is
refused.  The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


def _rel(a, b):
    out = []
    for g in ([0], [1, 2, 3], [4]):
        out.append(np.linalg.norm(a[g] - b[g]) / np.linalg.norm(b[g]))
    return np.array(out)


def _mesh(sem, kind):
    from tests.test_oracle_mesh import two_level_leaves
    if kind == "nonconforming":
        return sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves(), lvl_max=3), 12e3
    if kind == "large":            # 784 columns: 15.3 MiB of the 16 MiB array
        return sem.sem_mesh_create(600e3, 600e3, 24e3, 28, 28, 4, 4), 24e3
    return sem.sem_mesh_create(600e3, 600e3, 24e3, 6, 6, 4, 4), 24e3


def _tables(sem, m):
    """The mesh's device tables come from an ordinary call first."""
    xyz = torch.empty(3, m.NG, dtype=torch.float64, device="cuda")
    sem.sem_mesh_coords(m, xyz)


@pytest.mark.parametrize("kind", ["conforming", "nonconforming"])
@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_noalloc_matches_rhs_on_two_calls(sem, kind, precision):
    from synth.vortex import random_state
    m, Lz = _mesh(sem, kind)
    X = sem.sem_mesh_coords_host(m).T
    p = sem.sem_params_default(precision=precision)
    tol = 1e-12 if precision == 0 else 1e-6
    _tables(sem, m)
    for call, seed in enumerate((3, 4)):
        q = torch.from_numpy(random_state(X, Lz, seed)).cuda()
        ref = torch.empty_like(q)
        sem.sem_rhs(m, p, q, ref)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs_noalloc(m, p, q, out)
        torch.cuda.synchronize()
        err = _rel(out.cpu().numpy(), ref.cpu().numpy())
        assert np.all(err <= tol), (call, err)


def test_rhs_noalloc_leaves_free_memory_unchanged(sem):
    """After a first call (which may make the CUDA driver load the library's
    device code with its array), further calls change the device's free
    memory by nothing."""
    from synth.vortex import random_state
    m, Lz = _mesh(sem, "conforming")
    p = sem.sem_params_default()
    _tables(sem, m)
    q = torch.from_numpy(random_state(sem.sem_mesh_coords_host(m).T, Lz, 5)).cuda()
    out = torch.empty_like(q)
    sem.sem_rhs_noalloc(m, p, q, out)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        sem.sem_rhs_noalloc(m, p, q, out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_rhs_noalloc_large_mesh_then_small_mesh(sem):
    """A mesh that fills most of the array, then a small one: the second call
    must not read what the first left in the shared array."""
    from synth.vortex import random_state
    for kind in ("large", "nonconforming", "large"):
        m, Lz = _mesh(sem, kind)
        _tables(sem, m)
        p = sem.sem_params_default()
        q = torch.from_numpy(random_state(sem.sem_mesh_coords_host(m).T, Lz, 6)).cuda()
        ref = torch.empty_like(q)
        sem.sem_rhs(m, p, q, ref)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs_noalloc(m, p, q, out)
        torch.cuda.synchronize()
        assert np.all(_rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-12), kind


def test_rhs_noalloc_rejects_what_it_cannot_serve(sem):
    p = sem.sem_params_default()
    fresh = sem.sem_mesh_create(600e3, 600e3, 24e3, 6, 6, 4, 4)
    q = torch.zeros(5, fresh.NG, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:          # no device tables yet
        sem.sem_rhs_noalloc(fresh, p, q, torch.empty_like(q))
    assert e.value.code == sem.SEM_ERR_ARG
    big = sem.sem_mesh_create(2048e3, 2048e3, 24e3, 64, 64, 16, 4)
    qb = torch.zeros(5, big.NG, dtype=torch.float64, device="cuda")
    with pytest.raises(sem.SemError) as e:          # beyond the fixed maximum
        sem.sem_rhs_noalloc(big, p, qb, torch.empty_like(qb))
    assert e.value.code == sem.SEM_ERR_ARG
    assert "maximum" in str(e.value)
    # invalid parameters are refused as by sem_rhs, not treated as "off"
    m, _ = _mesh(sem, "conforming")
    _tables(sem, m)
    qm = torch.zeros(5, m.NG, dtype=torch.float64, device="cuda")
    for field, value in (("smag_cs", float("nan")), ("sponge_gamma", -1.0), ("heat_q0", -0.5),
                         ("time", float("inf"))):
        bad = sem.sem_params_default()
        setattr(bad, field, value)
        with pytest.raises(sem.SemError) as e:
            sem.sem_rhs_noalloc(m, bad, qm, torch.empty_like(qm))
        assert e.value.code == sem.SEM_ERR_ARG, field
        with pytest.raises(sem.SemError) as e2:
            sem.sem_rhs(m, bad, qm, torch.empty_like(qm))
        assert e2.value.code == sem.SEM_ERR_ARG, field
