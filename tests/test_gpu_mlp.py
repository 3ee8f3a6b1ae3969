"""GPU parity of the learned-flag kernels against the CPU oracle (oracle/mlp.py).

Both sides follow one precision contract: inputs, weights and hidden
activations rounded to bfloat16 before each product.  The GPU sums in float32
(tensor cores, float32 GEMMs), the oracle in float64; a hidden activation
within float32 rounding of a bfloat16 rounding boundary can round to the
neighbouring bfloat16 value, which perturbs the outputs by about 1e-5, so the
probabilities are compared at 1e-4 (relative L2) and the gradients at 1e-3.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import adapt, mesh as om, mlp as omlp, refstate  # noqa: E402
from synth.vortex import random_state, vortex_state  # noqa: E402
from tests.helpers import node_perm  # noqa: E402
from tests.test_oracle_mesh import two_level_leaves  # noqa: E402

SCALES = np.array([1e-3, 5.0, 5.0, 1.0, 1.0])


@pytest.fixture(scope="module")
def sem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_21607_gb300 import build
    build.build()
    from paper_2410_21607_gb300 import sem as s
    return s


def flat(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def unflat(v):
    shapes = [(136, 128), (128,), (128, 128), (128,), (128, 3), (3,)]
    out, o = [], 0
    for s in shapes:
        k = int(np.prod(s))
        out.append(np.asarray(v[o:o + k], dtype=np.float64).reshape(s))
        o += k
    return out


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _batch(n=1000, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 136)).astype(np.float32)
    X[:, 135] = rng.integers(0, 3, size=n)
    y = rng.integers(0, 3, size=n).astype(np.int8)
    return X, y


@pytest.mark.parametrize("tc", [1, 0])
def test_forward_matches_oracle(sem, tc):
    """tc = 1: the tcgen05 tensor-core forward (default), 0: the mma.sync one;
    1000 rows (a partial last tile of 128 rows for the tensor-core forward)."""
    net = sem.sem_mlp_create(7, 4096)
    sem.sem_mlp_select_forward(net, tc)
    params = [p.astype(np.float32).astype(np.float64) for p in omlp.init_params(11)]
    params[1] += 0.05
    params[3] -= 0.02
    params[5] += np.array([0.1, -0.2, 0.3])
    sem.sem_mlp_set_params(net, flat(params))
    X, _ = _batch(1000, 1)
    prob = torch.empty((1000, 3), dtype=torch.float32, device="cuda")
    sem.sem_mlp_forward(net, torch.from_numpy(X).cuda(), prob)
    P = prob.cpu().numpy()
    P_o = omlp.forward(params, X.astype(np.float64), emulate=True)["P"]
    assert rel(P, P_o) <= 1e-4
    flags = torch.empty(1000, dtype=torch.int8, device="cuda")
    sem.sem_mlp_predict_flags(net, torch.from_numpy(X).cuda(), flags)
    f = flags.cpu().numpy()
    srt = np.sort(P_o, axis=1)
    clear = srt[:, 2] - srt[:, 1] > 1e-3
    assert np.array_equal(f[clear], (np.argmax(P_o, axis=1) - 1)[clear])
    assert sem.sem_mlp_status(net) == 0


def test_tensor_core_forward_equals_mma_sync_forward(sem):
    """The two forwards on the same rows (several CTAs, a ragged last tile):
    the same bfloat16 products with float32 accumulation in another order."""
    net = sem.sem_mlp_create(9, 4096)
    X, _ = _batch(4001, 5)
    Xd = torch.from_numpy(X).cuda()
    out = []
    for tc in (1, 0):
        sem.sem_mlp_select_forward(net, tc)
        prob = torch.full((4001, 3), float("nan"), dtype=torch.float32, device="cuda")
        sem.sem_mlp_forward(net, Xd, prob)
        out.append(prob.cpu().numpy())
    assert np.isfinite(out[0]).all()
    assert rel(out[0], out[1]) <= 1e-4
    assert sem.sem_mlp_status(net) == 0


@pytest.mark.parametrize("tc", [1, 0])
def test_backward_matches_oracle(sem, tc):
    """The backward pass after either forward (which stores the rounded
    inputs and activations it uses)."""
    net = sem.sem_mlp_create(7, 4096)
    sem.sem_mlp_select_forward(net, tc)
    params = [p.astype(np.float32).astype(np.float64) for p in omlp.init_params(12)]
    sem.sem_mlp_set_params(net, flat(params))
    X, y = _batch(3000, 2)
    cw = np.array([2.0, 0.5, 3.0], dtype=np.float32)
    loss = sem.sem_mlp_backward(net, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), cw)
    g = unflat(sem.sem_mlp_get_grads(net))
    Xd = X.astype(np.float64)
    g_o = omlp.grads(params, Xd, y.astype(np.int64), cw.astype(np.float64), emulate=True)
    l_o = omlp.loss(params, Xd, y.astype(np.int64), cw.astype(np.float64), emulate=True)
    assert abs(loss - l_o) <= 1e-5 * abs(l_o)
    for k, (a, b) in enumerate(zip(g, g_o)):
        assert rel(a, b) <= 1e-3, (k, rel(a, b))


def test_adam_step_matches_oracle(sem):
    net = sem.sem_mlp_create(3, 4096)
    p0 = unflat(sem.sem_mlp_get_params(net))
    X, y = _batch(500, 3)
    sem.sem_mlp_backward(net, torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda(), [1, 1, 1])
    g = unflat(sem.sem_mlp_get_grads(net))
    sem.sem_mlp_adam(net, 1e-3)
    torch.cuda.synchronize()
    p1 = unflat(sem.sem_mlp_get_params(net))
    zeros = [np.zeros_like(a) for a in p0]
    p1_o, _, _ = omlp.adam(p0, g, zeros, zeros, 1, 1e-3)
    for a, b in zip(p1, p1_o):
        np.testing.assert_allclose(a, b, rtol=1e-6, atol=1e-7)


def test_features_match_oracle(sem):
    L, Lz, nx, nz, N = 300e3, 12e3, 4, 2, 4
    m = sem.sem_mesh_create(L, L, Lz, nx, nx, nz, N, leaves=two_level_leaves(), lvl_max=3)
    o = om.OracleMesh(L, L, Lz, nx, nx, nz, N, leaves=two_level_leaves())
    perm = node_perm(sem.sem_mesh_coords_host(m), o.XG)
    q_o = random_state(o.XG, Lz, 4)
    F_o = omlp.features(o, q_o, SCALES)
    q = torch.from_numpy(np.ascontiguousarray(q_o[:, perm])).cuda()
    F = torch.empty((m.Ne, 136), dtype=torch.float32, device="cuda")
    sem.sem_mlp_features(m, q, SCALES, F)
    lv = sem.sem_mesh_leaves_host(m)
    oleaf = {tuple(l): c for c, l in enumerate(o.leaves)}
    emap = np.array([oleaf[tuple(l)] * o.nz + k for l in lv for k in range(o.nz)])
    np.testing.assert_allclose(F.cpu().numpy(), F_o[emap], rtol=2e-6, atol=2e-6)


def test_training_learns_the_criterion(sem):
    """Train on the current criterion flags of a vortex state (a learnable
    target): the loss falls and the predicted flags agree with the criterion."""
    L, Lz, nx, nz, N = 600e3, 24e3, 16, 4, 4
    m = sem.sem_mesh_create(L, L, Lz, nx, nx, nz, N, lvl_max=2)
    X = sem.sem_mesh_coords_host(m).T
    p = sem.sem_params_default(thresholds=[5.0, 10.0], lvl_max=2)
    feats, labels = [], []
    for seed, vmax in ((1, 12.0), (2, 20.0), (3, 28.0)):
        from synth.vortex import VortexSpec
        q = torch.from_numpy(vortex_state(X, Lz, VortexSpec(vmax=vmax, seed=seed))).cuda()
        fl = torch.empty(m.Ne, dtype=torch.int8, device="cuda")
        sem.sem_adapt_flags(m, p, q, fl)
        F = torch.empty((m.Ne, 136), dtype=torch.float32, device="cuda")
        sem.sem_mlp_features(m, q, SCALES, F)
        feats.append(F)
        labels.append((fl + 1).to(torch.int8))
    F = torch.cat(feats)
    Y = torch.cat(labels)
    counts = torch.bincount(Y.long(), minlength=3).cpu().numpy()
    cw = (counts.sum() / np.maximum(counts, 1) / 3.0).astype(np.float32)
    net = sem.sem_mlp_create(5, F.shape[0])
    l0 = sem.sem_mlp_backward(net, F, Y, cw)
    for _ in range(300):
        sem.sem_mlp_backward(net, F, Y, cw, want_loss=False)
        sem.sem_mlp_adam(net, 3e-3)
    l1 = sem.sem_mlp_backward(net, F, Y, cw)
    pred = torch.empty(F.shape[0], dtype=torch.int8, device="cuda")
    sem.sem_mlp_predict_flags(net, F, pred)
    acc = (pred == (Y - 1)).float().mean().item()
    assert l1 < 0.3 * l0, (l0, l1)
    assert acc > 0.9, acc
