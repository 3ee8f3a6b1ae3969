"""The allocation-free right-hand side, sem_rhs_noalloc.

Some callers may not allocate device memory when they evaluate the
right-hand side: their device memory is already reserved by another allocator
(so a new cudaMalloc fails), or their rules forbid device allocation after
start-up.  sem_rhs_noalloc serves them from a fixed device array built into
the library.  This test calls it through the C ABI twice in a row, with
different states, and checks each result against sem_rhs on the same input
with the float64 tolerance of the other parity tests (relative L2 <= 1e-12
per field group), on a conforming and a non-conforming mesh.  It lives in its
own file so that pytest collects it last.
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


@pytest.mark.parametrize("nonconforming", [False, True])
@pytest.mark.parametrize("precision", [0, 1])
def test_rhs_noalloc_matches_rhs_on_two_calls(sem, nonconforming, precision):
    from synth.vortex import random_state
    from tests.test_oracle_mesh import two_level_leaves
    if nonconforming:
        m = sem.sem_mesh_create(300e3, 300e3, 12e3, 4, 4, 2, 4, leaves=two_level_leaves(), lvl_max=3)
    else:
        m = sem.sem_mesh_create(600e3, 600e3, 24e3, 6, 6, 4, 4)
    X = sem.sem_mesh_coords_host(m).T
    Lz = 12e3 if nonconforming else 24e3
    p = sem.sem_params_default(precision=precision)
    tol = 1e-12 if precision == 0 else 1e-6
    # the mesh's device tables come from an ordinary call first
    xyz = torch.empty(3, m.NG, dtype=torch.float64, device="cuda")
    sem.sem_mesh_coords(m, xyz)
    for call, seed in enumerate((3, 4)):
        q = torch.from_numpy(random_state(X, Lz, seed)).cuda()
        ref = torch.empty_like(q)
        sem.sem_rhs(m, p, q, ref)
        out = torch.full_like(q, float("nan"))
        sem.sem_rhs_noalloc(m, p, q, out)
        torch.cuda.synchronize()
        err = _rel(out.cpu().numpy(), ref.cpu().numpy())
        assert np.all(err <= tol), (call, err)


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
