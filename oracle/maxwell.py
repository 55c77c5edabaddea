"""Maxwell right-hand side, LSERK4 and energy (oracle, FP64).

Test infrastructure only (see the package docstring).

State u = (Ex, Ey, Ez, Hx, Hy, Hz), array (6, K, Np), eps = mu = 1, no current.
Maxwell's equations of Section 6 (Eq. maxwells-claws) read
    dE/dt = curl H,      dH/dt = -curl E.
(The flux matrix F(u) printed in Section 6 has its E and H blocks exchanged
with respect to these curl equations; the curl equations are followed.)

The semi-discrete operator (Eq. semidiscrete-dg) is split, as in Fig.
dg-subtasks, into a volume part and a lifted surface part:
  a1  U_r, U_s, U_t = Dr U, Ds U, Dt U                   (local differentiation)
  a2  d/dx = rx d/dr + sx d/ds + tx d/dt  (likewise y, z)  -> curl H, curl E
  a3  for every face node: u- at vmapM, u+ at vmapP (PEC walls: E+ = -E-,
      H+ = H-), dE = E- - E+, dH = H- - H+, and the upwind flux of Section 6
      with Z = Y = 1, written with jumps d = u- - u+:
        n.(F - F*)_E = 1/2 ( -n x dH + alpha (n (n.dE) - dE) )
        n.(F - F*)_H = 1/2 (  n x dE + alpha (n (n.dH) - dH) )
      (alpha = 1: upwind; alpha = 0: central), times Fscale = sJ / J
  a4  lifted by LIFT (Fig. lifting-matrix)
      rhs_E = curl H + LIFT fluxE,   rhs_H = -curl E + LIFT fluxH
The time stepper is the five-stage, two-register low-storage RK4 of Carpenter
and Kennedy (1994), cited in Section 6:
      res <- a_i res + dt rhs(u),   u <- u + b_i res,   i = 0..4.

Materials and boundaries (optional arguments eps, mu, bc):
  * per-element permittivity eps_k and permeability mu_k (the conservation form
    of Section 6 carries diag(eps, mu) on u_t): rhs_E is divided by eps_k and
    rhs_H by mu_k; the flux is the upwind flux of Section 6 with impedance
    Z = sqrt(mu / eps) and admittance Y = 1 / Z, written with jumps
    [u] = u+ - u-:
        n.(F - F*)_E = 1/(Z- + Z+) n x ( Z+ [H] - alpha n x [E])
        n.(F - F*)_H = 1/(Y- + Y+) n x (-Y+ [E] - alpha n x [H])
    (the 1/2 and the cross-face average {Z} of Section 6 combine into
    1/(Z- + Z+); for Z- = Z+ = 1 this is the vacuum flux above);
  * boundary faces: bc = 0 a perfect conductor (E+ = -E-, H+ = H-), bc = 1 a
    characteristic absorbing boundary (Section 6's sample calculation): the
    exterior state is zero, so no wave enters; on either, Z+ = Z-.
  * the energy weights E by eps and H by mu: 1/2 sum_k J_k (eps_k E^T M E +
    mu_k H^T M H).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np

# Carpenter & Kennedy (1994) five-stage 2N-storage RK4 coefficients
_RK_A = (Fraction(0), Fraction(-567301805773, 1357537059087),
         Fraction(-2404267990393, 2016746695238), Fraction(-3550918686646, 2091501179385),
         Fraction(-1275806237668, 842570457699))
_RK_B = (Fraction(1432997174477, 9575080441755), Fraction(5161836677717, 13612068292357),
         Fraction(1720146321549, 2090206949498), Fraction(3134564353537, 4481467310338),
         Fraction(2277821191437, 14882151754819))
_RK_C = (Fraction(0), Fraction(1432997174477, 9575080441755),
         Fraction(2526269341429, 6820363962896), Fraction(2006345519317, 3224310063776),
         Fraction(2802321613138, 2924317926251))


def lserk4_coefficients(exact: bool = False):
    """(a, b, c) of the LSERK4 scheme, as Fractions if exact else floats."""
    if exact:
        return _RK_A, _RK_B, _RK_C
    return (tuple(float(x) for x in _RK_A), tuple(float(x) for x in _RK_B),
            tuple(float(x) for x in _RK_C))


def _cross(a, b):
    return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])


def volume_term(mesh, u):
    """Steps a1-a2: (curl H, -curl E) from the reference derivatives."""
    ref = mesh.ref
    ur = np.einsum("ij,fkj->fki", ref.Dr, u)
    us = np.einsum("ij,fkj->fki", ref.Ds, u)
    ut = np.einsum("ij,fkj->fki", ref.Dt, u)
    c = lambda g: g[None, :, None]  # noqa: E731
    dx = c(mesh.rx) * ur + c(mesh.sx) * us + c(mesh.tx) * ut
    dy = c(mesh.ry) * ur + c(mesh.sy) * us + c(mesh.ty) * ut
    dz = c(mesh.rz) * ur + c(mesh.sz) * us + c(mesh.tz) * ut
    # field index: 0..2 E, 3..5 H
    curlH = np.stack([dy[5] - dz[4], dz[3] - dx[5], dx[4] - dy[3]])
    curlE = np.stack([dy[2] - dz[1], dz[0] - dx[2], dx[1] - dy[0]])
    return np.concatenate([curlH, -curlE])


def _materials(mesh, eps, mu):
    eps = np.ones(mesh.K) if eps is None else np.asarray(eps, dtype=np.float64)
    mu = np.ones(mesh.K) if mu is None else np.asarray(mu, dtype=np.float64)
    return eps, mu


def surface_flux(mesh, u, alpha: float = 1.0, eps=None, mu=None, bc=None):
    """Step a3: Fscale * n.(F - F*) at every face node, shape (6, K, 4*Nfp).

    eps, mu: per-element material (default 1); bc: (K, 4) boundary kind of
    each face, 0 perfect conductor (default), 1 absorbing (read on boundary
    faces only)."""
    K, Nfp = mesh.K, mesh.Nfp
    eps, mu = _materials(mesh, eps, mu)
    flat = u.reshape(6, -1)
    uM = flat[:, mesh.vmapM].reshape(6, K, 4, Nfp)
    uP = flat[:, mesh.vmapP].reshape(6, K, 4, Nfp).copy()
    bnd = mesh.boundary
    absorb = bnd & (np.zeros((K, 4), bool) if bc is None else np.asarray(bc) == 1)
    pec = bnd & ~absorb
    uP[:3] = np.where(pec[None, :, :, None], -uM[:3], uP[:3])      # PEC: E+ = -E-
    uP[3:] = np.where(pec[None, :, :, None], uM[3:], uP[3:])       #      H+ =  H-
    uP = np.where(absorb[None, :, :, None], 0.0, uP)               # absorbing: u+ = 0
    # impedances of both sides (the neighbour's, or the element's own on boundaries)
    Z = np.sqrt(mu / eps)
    ZM = np.repeat(Z[:, None], 4, axis=1)
    ZP = np.where(bnd, ZM, Z[mesh.EToE])
    YM, YP = 1.0 / ZM, 1.0 / ZP
    jE = uP[:3] - uM[:3]                      # [E] = E+ - E-
    jH = uP[3:] - uM[3:]
    n = (mesh.nx[:, :, None], mesh.ny[:, :, None], mesh.nz[:, :, None])
    nxjE = _cross(n, jE)
    nxjH = _cross(n, jH)
    nxnxjE = _cross(n, nxjE)
    nxnxjH = _cross(n, nxjH)
    cE = (1.0 / (ZM + ZP))[:, :, None]
    cH = (1.0 / (YM + YP))[:, :, None]
    zp, yp = ZP[:, :, None], YP[:, :, None]
    fE = [cE * (zp * nxjH[i] - alpha * nxnxjE[i]) for i in range(3)]
    fH = [cH * (-yp * nxjE[i] - alpha * nxnxjH[i]) for i in range(3)]
    flux = np.stack(fE + fH) * mesh.Fscale[None, :, :, None]
    return flux.reshape(6, K, 4 * Nfp)


def rhs(mesh, u, alpha: float = 1.0, eps=None, mu=None, bc=None):
    """Semi-discrete right-hand side du/dt, shape (6, K, Np), FP64."""
    u = np.asarray(u, dtype=np.float64)
    eps, mu = _materials(mesh, eps, mu)
    vol = volume_term(mesh, u)
    flux = surface_flux(mesh, u, alpha, eps, mu, bc)
    surf = np.einsum("im,fkm->fki", mesh.ref.LIFT, flux)
    w = np.concatenate([np.repeat(1.0 / eps[None, :], 3, axis=0),
                        np.repeat(1.0 / mu[None, :], 3, axis=0)])
    return (vol + surf) * w[:, :, None]


def stage_update(u, res, r, a, b, dt):
    """One LSERK4 stage update given the stage's right-hand side r."""
    res = a * res + dt * r
    return u + b * res, res


def lserk4_run(mesh, u, dt: float, nsteps: int, res=None, alpha: float = 1.0,
               eps=None, mu=None, bc=None):
    """Advance u by nsteps LSERK4 steps; returns (u, res)."""
    a, b, _ = lserk4_coefficients()
    u = np.array(u, dtype=np.float64)
    res = np.zeros_like(u) if res is None else np.array(res, dtype=np.float64)
    for _ in range(nsteps):
        for i in range(5):
            u, res = stage_update(u, res, rhs(mesh, u, alpha, eps, mu, bc), a[i], b[i], dt)
    return u, res


def energy(mesh, u, eps=None, mu=None):
    """Discrete energy 1/2 sum_k J_k (eps_k E_k^T M E_k + mu_k H_k^T M H_k)."""
    u = np.asarray(u, dtype=np.float64)
    eps, mu = _materials(mesh, eps, mu)
    Mu = np.einsum("ij,fkj->fki", mesh.ref.M, u)
    w = np.concatenate([np.repeat(eps[None, :], 3, axis=0), np.repeat(mu[None, :], 3, axis=0)])
    return 0.5 * float(np.sum((mesh.J[None, :] * w)[:, :, None] * u * Mu))


def cfl_dt(mesh, C: float = 1.0, eps=None, mu=None):
    """Time step dt = C * min_{k,f} (sqrt(eps_k mu_k) / Fscale) * 2/(N+1)^2 (the
    wave speed of element k is 1 / sqrt(eps_k mu_k))."""
    eps, mu = _materials(mesh, eps, mu)
    slow = np.sqrt(eps * mu)[:, None]
    return C * float(np.min(slow / mesh.Fscale)) * 2.0 / (mesh.N + 1) ** 2
