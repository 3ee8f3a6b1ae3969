"""Wind diagnostics of Sec. 4.2.

* max wind: the largest horizontal wind speed sqrt(u^2 + v^2) over the nodes
  with (x, y) in [-50, 50] km x [-50, 50] km (all heights);
* max of the horizontal mean: at every height, the mean of the horizontal wind
  speed over the same horizontal sub-domain, then the largest of these means.
  The mean at a height is weighted by the lumped mass of the nodes at that
  height (the discrete area integral divided by the area).

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np

from .refstate import reference_state


def horizontal_speed(mesh, qG, prm, eqset="C"):
    if eqset == "C":
        rho = reference_state(mesh.XG[:, 2], prm)["rho0"] + qG[0]
        return np.sqrt(qG[1] * qG[1] + qG[2] * qG[2]) / rho
    return np.sqrt(qG[1] * qG[1] + qG[2] * qG[2])


def wind_diagnostics(mesh, qG, prm, eqset="C", half_width=50.0e3):
    s = horizontal_speed(mesh, qG, prm, eqset)
    X = mesh.XG
    inside = (np.abs(X[:, 0]) <= half_width + 1e-6) & (np.abs(X[:, 1]) <= half_width + 1e-6)
    max_wind = float(s[inside].max())
    zk = np.round(X[:, 2], 6)
    best = -np.inf
    for z in np.unique(zk[inside]):
        m = inside & (zk == z)
        best = max(best, float(np.sum(mesh.M[m] * s[m]) / np.sum(mesh.M[m])))
    return dict(max_wind=max_wind, max_mean_wind=best)
