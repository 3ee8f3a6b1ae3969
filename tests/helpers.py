"""Shared helpers: library <-> oracle node matching and error norms."""
import numpy as np


def node_perm(lib_xyz, oracle_xyz, scale=1e-4):
    """perm[g_lib] = g_oracle, matching global nodes by coordinates."""
    lib_xyz = np.asarray(lib_xyz)
    if lib_xyz.shape[0] == 3 and lib_xyz.shape[1] != 3:
        lib_xyz = lib_xyz.T
    kl = np.round(lib_xyz / scale).astype(np.int64)
    ko = np.round(np.asarray(oracle_xyz) / scale).astype(np.int64)
    # lexicographic sort of both key sets, then pair them up
    ol = np.lexsort(kl.T[::-1])
    oo = np.lexsort(ko.T[::-1])
    if len(ol) != len(oo) or not np.array_equal(kl[ol], ko[oo]):
        raise AssertionError("library and oracle node sets differ")
    perm = np.empty(len(ol), dtype=np.int64)
    perm[ol] = oo
    return perm


def group_rel_l2(a, b, weights=None):
    """Relative L2 error per field group {rho, momentum (joint), theta}.

    a is the result under test, b the reference, both (5, n)."""
    groups = ([0], [1, 2, 3], [4])
    w = np.ones(a.shape[1]) if weights is None else weights
    out = []
    for g in groups:
        num = np.sqrt(np.sum(w * np.sum((a[g] - b[g]) ** 2, axis=0)))
        den = np.sqrt(np.sum(w * np.sum(b[g] ** 2, axis=0)))
        out.append(num / den if den > 0 else num)
    return np.array(out)


def lib_to_oracle(q_lib, perm, n_oracle):
    out = np.zeros((q_lib.shape[0], n_oracle))
    out[:, perm] = q_lib
    return out


def stretched_faces(Lz, nz, a=1.0):
    """Layer faces z_k = Lz g(k / nz) with g(s) = (s + a s^2) / (1 + a): a
    smooth stretching, layers thickening upwards (top to bottom thickness
    ratio (nz + a (2 nz - 1)) / (nz + a))."""
    s = np.arange(nz + 1) / nz
    z = Lz * (s + a * s * s) / (1.0 + a)
    z[0], z[-1] = 0.0, Lz
    return z
