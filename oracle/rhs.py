"""Right-hand side of the split dry Euler equations on the CG spectral-element mesh.

Two equation sets share one discretisation (Sec. 3):

* "C" (conservative): state (rho', rho u, rho v, rho w, (rho theta)'), the
  flux form of Eqs. mass_split / mom_split / ent_split (multiply the velocity
  and theta equations by rho and use the mass equation):
      d rho'/dt          = -div(rho u)
      d (rho u)/dt       = -div(rho u (x) u + p' I) - rho' g e_z + f (rho v, -rho u, 0)
      d (rho theta)'/dt  = -div(rho theta u)
* "NC" (the paper's non-conservative set, Eqs. mass_split..ent_split):
  state (rho', u, v, w, theta'),
      d rho'/dt   = -div(rho u)
      d u/dt      = -u.grad u - grad p' / rho + (rho'/rho) g k + f (v, -u, 0)
      d theta'/dt = -u.grad theta0 - u.grad theta'
  with k = (0, 0, -1) (Sec. 2).  The f-plane Coriolis term is not in the
  paper's equations; it is added with the parameter f (zero turns it off).

In both, p' = p0 expm1(gamma log1p((rho theta)'/(rho theta)0)).

Optional terms of the paper's runs (Sec. 4), off unless the parameters set them:

* Rayleigh absorbing layer ("Boundary conditions"): every equation gets
  -R(z) q' with q' its own perturbation variable (for "C" the conservative
  perturbations, for "NC" rho', u, v, w, theta') and
      R(z) = min(1, max(0, gamma sin^2(pi/2 (1 - (z_top - z)/z_d))))
  for z >= z_top - z_d and R = 0 below (reading of the garbled formula: the
  layer is the top z_d of the domain, z_top = Lz; the term damps, so it
  enters with a minus sign; gamma is a rate in 1/s).  It is a collocated
  source, r_l += w_l J (-R q'_l), like the other sources.
* Synthetic latent heating (stand-in for the paper's observed heating,
  Sec. 4 "Observational heating": radially confined to r <= 60 km, largest
  at 25-30 km, introduced over the first 30 minutes by a tanh ramp):
      Q(x, t) = q0 tanh(t / tau) exp(-((r - r0) / width)^2) sin(pi z / z_top)
  for r <= r_max and z <= z_top (r from the domain centre), zero elsewhere,
  a heating rate of theta in K/s: a collocated source w J rho Q on
  (rho theta)' ("C") or w J Q on theta' ("NC"), evaluated at the time of
  the state (prm.time).
* Horizontal Smagorinsky-Lilly stress ("Sub-grid models"): with the
  element-local velocity gradients, S_h the horizontal strain of (u, v)
  (S_xx = du/dx, S_yy = dv/dy, S_xy = (du/dy + dv/dx)/2),
      nu_t = (C_s Delta)^2 sqrt(2 (S_xx^2 + S_yy^2 + 2 S_xy^2)),
  Delta = (hx + hy) / (2N) the mean horizontal node spacing of the element,
  the momentum equations get -div(tau) with the horizontal stress
  tau_{i,d} = -2 nu_t S_{i,d} for i, d in {x, y} and tau_{z,d} = -nu_t dw/dx_d,
  d in {x, y} (reading: the vertical part is the PBL scheme's, out of
  scope), in weak form with the flux rho tau ("C") or tau ("NC").

Discretisation: the divergence terms are taken in weak form,
    r_l = sum_k w_k J grad psi_l(x_k) . F(x_k)   (+ boundary terms, see below),
the remaining (source, advective and pressure-gradient) terms in collocated
strong form, r_l = w_l J s_l.  The element residuals are assembled with the
modified DSS of Sec. 3.1, R = Q^T r, and divided by the lumped mass built the
same way, M = Q^T (w J).  Lateral boundaries are periodic (Sec. 4); top and
bottom are rigid lids: the vertical-momentum (or w) tendency is set to zero
at the lid nodes, which also removes the lid boundary integrals because the
normal mass, momentum and theta fluxes vanish there with w = 0.

Test infrastructure only (see oracle/__init__.py).
"""
import numpy as np

from .refstate import reference_state, pressure_perturbation

FIELDS_C = ("rho'", "rho u", "rho v", "rho w", "(rho theta)'")
FIELDS_NC = ("rho'", "u", "v", "w", "theta'")


def sponge_rate(z, Lz, prm):
    """R(z) of the Rayleigh absorbing layer (Sec. 4), zero below Lz - z_d."""
    z = np.asarray(z, dtype=np.float64)
    zd = prm.sponge_depth
    a = np.pi / 2.0 * (1.0 - (Lz - z) / zd)
    R = np.minimum(1.0, np.maximum(0.0, prm.sponge_gamma * np.sin(a) ** 2))
    return np.where(z >= Lz - zd, R, 0.0)


def heating_rate(x, y, z, prm):
    """Q(x, t) of the synthetic heating, K/s, at points (x, y, z) and prm.time."""
    r = np.hypot(x, y)
    shape = np.exp(-((r - prm.heat_r0) / prm.heat_width) ** 2) * np.sin(np.pi * z / prm.heat_ztop)
    inside = (r <= prm.heat_rmax) & (z <= prm.heat_ztop)
    return np.where(inside, prm.heat_q0 * np.tanh(prm.time / prm.heat_ramp) * shape, 0.0)


def element_residual(mesh, qL, prm, eqset="C"):
    """Element-local residuals r_L, shape (5, Ne, P), from local values qL."""
    if eqset not in ("C", "NC"):
        raise ValueError(eqset)
    z = mesh.X[:, :, 2]
    ref = reference_state(z, prm)
    rho0, p0, rt0 = ref["rho0"], ref["p0"], ref["rhotheta0"]
    theta0, dth0 = ref["theta0"], ref["dtheta0"]
    g, f, gamma = prm.g, prm.f, prm.gamma
    wJ = mesh.wJ
    r = np.zeros_like(qL)
    for lev, es, G in mesh.op_groups():
        q = qL[:, es, :]
        rp = q[0]
        rho = rho0[es] + rp
        W_ = wJ[es]

        def weak(F):
            # sum_k wJ_k sum_d G_d[k, l] F_d[k]
            return sum((W_ * F[d]) @ G[d] for d in range(3))

        def grad(phi):
            return [phi @ G[d].T for d in range(3)]

        if eqset == "C":
            U, V, Wm, Tp = q[1], q[2], q[3], q[4]
            u, v, w = U / rho, V / rho, Wm / rho
            pp = pressure_perturbation(Tp, rt0[es], p0[es], gamma)
            rt = rt0[es] + Tp
            r[0, es] = weak((U, V, Wm))
            r[1, es] = weak((U * u + pp, U * v, U * w)) + W_ * (f * V)
            r[2, es] = weak((V * u, V * v + pp, V * w)) + W_ * (-f * U)
            r[3, es] = weak((Wm * u, Wm * v, Wm * w + pp)) + W_ * (-rp * g)
            r[4, es] = weak((rt * u, rt * v, rt * w))
        else:
            u, v, w, thp = q[1], q[2], q[3], q[4]
            rtp = rho0[es] * thp + rp * (theta0[es] + thp)
            pp = pressure_perturbation(rtp, rt0[es], p0[es], gamma)
            r[0, es] = weak((rho * u, rho * v, rho * w))
            gu, gv, gw, gp, gt = grad(u), grad(v), grad(w), grad(pp), grad(thp)
            adv = lambda gq: u * gq[0] + v * gq[1] + w * gq[2]
            su = -adv(gu) - gp[0] / rho + f * v
            sv = -adv(gv) - gp[1] / rho - f * u
            sw = -adv(gw) - gp[2] / rho - (rp / rho) * g
            st = -w * dth0[es] - adv(gt)
            r[1, es] = W_ * su
            r[2, es] = W_ * sv
            r[3, es] = W_ * sw
            r[4, es] = W_ * st
        if getattr(prm, "smag_cs", 0.0) > 0.0:
            if eqset == "C":
                uu, vv, ww, rfac = q[1] / rho, q[2] / rho, q[3] / rho, rho
            else:
                uu, vv, ww, rfac = q[1], q[2], q[3], 1.0
            gu, gv, gw = grad(uu), grad(vv), grad(ww)
            Sxx, Syy, Sxy = gu[0], gv[1], 0.5 * (gu[1] + gv[0])
            hx = mesh.Lx / (mesh.nx << int(lev))
            hy = mesh.Ly / (mesh.ny << int(lev))
            delta = (hx + hy) / (2.0 * mesh.N)
            nut = (prm.smag_cs * delta) ** 2 * np.sqrt(2.0 * (Sxx ** 2 + Syy ** 2 + 2.0 * Sxy ** 2))
            k = rfac * nut
            zero = np.zeros_like(k)
            # -div(tau) in weak form: flux rho tau (C) or tau (NC)
            r[1, es] += weak((-2.0 * k * Sxx, -2.0 * k * Sxy, zero))
            r[2, es] += weak((-2.0 * k * Sxy, -2.0 * k * Syy, zero))
            r[3, es] += weak((-k * gw[0], -k * gw[1], zero))
        if getattr(prm, "sponge_gamma", 0.0) > 0.0:
            Rz = sponge_rate(z[es], mesh.Lz, prm)
            for fl in range(5):
                r[fl, es] += W_ * (-Rz * q[fl])
        if getattr(prm, "heat_q0", 0.0) > 0.0:
            Q = heating_rate(mesh.X[es, :, 0], mesh.X[es, :, 1], z[es], prm)
            r[4, es] += W_ * (rho * Q if eqset == "C" else Q)
    return r


def rhs(mesh, qG, prm, eqset="C"):
    """Tendency dq_G/dt = (Q^T r_L) / M with the lid condition, shape (5, NG)."""
    qL = mesh.to_local(qG)
    r = element_residual(mesh, qL, prm, eqset)
    R = mesh.assemble(r)
    T = R / mesh.M[None, :]
    T[3, mesh.z_bottom | mesh.z_top] = 0.0
    return T


def scalar_advection_residual(mesh, phiG, c, form="weak"):
    """Assembled residual Q^T r of the advection of a scalar, phi_t + div(c phi) = 0
    with a constant velocity c, in the discretisation of the divergence terms
    above: "weak" r_l = sum_k w_k J grad psi_l(x_k) . c phi_k (the form the
    right-hand side uses), or the skew-symmetric split "skew" = (weak +
    strong) / 2 with the collocated strong term r_l = -w_l J c . grad phi(x_l).
    Used to study the discrete energy phi^T Q^T r (no lid condition)."""
    phiL = mesh.to_local(phiG)[0]
    r = np.zeros_like(phiL)
    for lev, es, G in mesh.op_groups():
        W = mesh.wJ[es]
        f = phiL[es]
        weak = sum((W * c[d] * f) @ G[d] for d in range(3))
        if form == "weak":
            r[es] = weak
        else:
            strong = -W * sum(c[d] * (f @ G[d].T) for d in range(3))
            r[es] = 0.5 * (weak + strong)
    return mesh.assemble(r[None])[0]
