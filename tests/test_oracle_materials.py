"""Oracle pins for materials (per-element eps, mu) and absorbing boundaries.

The flux of Section 6 with impedances is pinned against an independent
derivation: the exact solution of the Riemann problem at a face, built from
the characteristics of the 1-D Maxwell system along the normal (tangential
pairs (E.t1, H.t2) and (E.t2, H.t1) travel as E.t1 +- Z H.t2 and
E.t2 -+ Z H.t1; the interface keeps tangential E and H continuous).  The upwind
flux must equal n.(F(u-) - F(u*)) = (-n x (H- - H*), n x (E- - E*)) there.  The
material weights are pinned by energy conservation (central flux, perfect
conductors) and dissipation (upwind), and the eps, mu scaling law.
"""
import numpy as np
import pytest

import oracle
from workloads import gaussian_pulse, kuhn_box_mesh, random_fields


def _riemann_flux(uM, uP, n, ZM, ZP):
    """Exact upwind n.(F - F*) per node from the characteristic solution.
    uM, uP: (6, P); n: (3, P); ZM, ZP: (P,)."""
    n = n / np.linalg.norm(n, axis=0)
    # a tangent t1 (not parallel to n) and t2 = n x t1
    a = np.where(np.abs(n[0]) < 0.9, 1.0, 0.0)
    helper = np.stack([a, 1.0 - a, np.zeros_like(a)])
    t1 = helper - n * np.sum(helper * n, axis=0)
    t1 /= np.linalg.norm(t1, axis=0)
    t2 = np.cross(n.T, t1.T).T
    dot = lambda v, w: np.sum(v * w, axis=0)  # noqa: E731
    EM, HM, EP, HP = uM[:3], uM[3:], uP[:3], uP[3:]
    # pair 1: (E.t1, H.t2): right-going invariant r = E1 + Z H2, left-going l = E1 - Z H2
    r1 = dot(EM, t1) + ZM * dot(HM, t2)
    l1 = dot(EP, t1) - ZP * dot(HP, t2)
    H2s = (r1 - l1) / (ZM + ZP)
    E1s = r1 - ZM * H2s
    # pair 2: (E.t2, H.t1): right-going r = E2 - Z H1, left-going l = E2 + Z H1
    r2 = dot(EM, t2) - ZM * dot(HM, t1)
    l2 = dot(EP, t2) + ZP * dot(HP, t1)
    H1s = (l2 - r2) / (ZM + ZP)
    E2s = r2 + ZM * H1s
    Es = E1s * t1 + E2s * t2          # tangential interface state
    Hs = H1s * t1 + H2s * t2
    # only tangential parts enter n x (.), so the normal parts of u- cancel too
    fE = -np.cross(n.T, (HM - Hs).T).T
    fH = np.cross(n.T, (EM - Es).T).T
    return np.concatenate([fE, fH])


def _face_data(om, u):
    K, Nfp = om.K, om.Nfp
    flat = u.reshape(6, -1)
    uM = flat[:, om.vmapM].reshape(6, K, 4, Nfp)
    uP = flat[:, om.vmapP].reshape(6, K, 4, Nfp)
    return uM, uP


@pytest.mark.parametrize("N", [1, 3])
def test_material_upwind_flux_is_the_exact_riemann_flux(N):
    """Interior faces between elements of different eps, mu, perfect-conductor
    faces and absorbing faces: the oracle's upwind flux equals the flux of the
    exact interface state at every face node."""
    verts, tets = kuhn_box_mesh(2, 0.15, 3)
    om = oracle.build_mesh(verts, tets, N)
    rng = np.random.default_rng(7 + N)
    eps = rng.uniform(0.5, 4.0, om.K)
    mu = rng.uniform(0.5, 3.0, om.K)
    bc = rng.integers(0, 2, (om.K, 4))
    u = random_fields(om.K, om.Np, 11 + N)
    got = oracle.maxwell.surface_flux(om, u, 1.0, eps, mu, bc).reshape(6, om.K, 4, om.Nfp)
    uM, uP = _face_data(om, u)
    uP = uP.copy()
    Z = np.sqrt(mu / eps)
    ZM = np.repeat(Z[:, None], 4, axis=1)
    ZP = np.where(om.boundary, ZM, Z[om.EToE])
    absorb = om.boundary & (bc == 1)
    pec = om.boundary & (bc == 0)
    assert absorb.any() and pec.any() and (~om.boundary).any()
    uP[:3] = np.where(pec[None, :, :, None], -uM[:3], uP[:3])
    uP[3:] = np.where(pec[None, :, :, None], uM[3:], uP[3:])
    uP = np.where(absorb[None, :, :, None], 0.0, uP)
    nvec = np.stack([om.nx, om.ny, om.nz])[:, :, :, None] * np.ones(om.Nfp)
    P = om.K * 4 * om.Nfp
    want = _riemann_flux(uM.reshape(6, P), uP.reshape(6, P), nvec.reshape(3, P),
                         np.repeat(ZM.ravel(), om.Nfp), np.repeat(ZP.ravel(), om.Nfp))
    want = want.reshape(6, om.K, 4, om.Nfp) * om.Fscale[None, :, :, None]
    assert np.max(np.abs(got - want)) < 1e-12 * np.max(np.abs(want))


def test_perfect_conductor_interface_state_has_no_tangential_e():
    """The Riemann state at a perfect-conductor face has E x n = 0: the flux
    then is (-n x (H- - H*), n x E-)."""
    rng = np.random.default_rng(3)
    P = 50
    uM = rng.standard_normal((6, P))
    uP = np.concatenate([-uM[:3], uM[3:]])
    n = rng.standard_normal((3, P))
    Z = rng.uniform(0.3, 3.0, P)
    f = _riemann_flux(uM, uP, n, Z, Z)
    nn = n / np.linalg.norm(n, axis=0)
    assert np.allclose(f[3:], np.cross(nn.T, uM[:3].T).T, atol=1e-13)


def _energy_rate(om, u, alpha, eps, mu, bc=None):
    r = oracle.rhs(om, u, alpha, eps, mu, bc)
    Mr = np.einsum("ij,fkj->fki", om.ref.M, r)
    w = np.concatenate([np.repeat(eps[None], 3, 0), np.repeat(mu[None], 3, 0)])
    return float(np.sum((om.J[None] * w)[:, :, None] * u * Mr))


@pytest.mark.parametrize("N", [2, 4])
def test_material_energy_conserved_by_central_flux_and_dissipated_by_upwind(N):
    """d/dt 1/2 sum J (eps E.M E + mu H.M H) = 0 with the central flux and
    perfect conductors (to rounding), < 0 with the upwind flux, and < 0 with
    every boundary face absorbing (no energy enters).  A missing 1/eps (or
    1/mu) weight, or Z- and Z+ swapped in one of the two flux rows, breaks the
    first identity."""
    verts, tets = kuhn_box_mesh(2, 0.15, 5)
    om = oracle.build_mesh(verts, tets, N)
    rng = np.random.default_rng(N)
    eps = rng.uniform(0.5, 4.0, om.K)
    mu = rng.uniform(0.5, 3.0, om.K)
    u = random_fields(om.K, om.Np, 21 + N)
    e = oracle.energy(om, u, eps, mu)
    scale = e * np.max(om.Fscale) * (N + 1) ** 2
    assert abs(_energy_rate(om, u, 0.0, eps, mu)) < 1e-11 * scale
    assert _energy_rate(om, u, 1.0, eps, mu) < -1e-6 * scale
    bc = np.ones((om.K, 4), int)
    assert _energy_rate(om, u, 1.0, eps, mu, bc) < -1e-6 * scale


def test_material_scaling_law():
    """eps -> c eps, mu -> c mu keeps every impedance and divides the speed by
    c: the right-hand side is divided by c."""
    verts, tets = kuhn_box_mesh(2, 0.15, 6)
    om = oracle.build_mesh(verts, tets, 3)
    rng = np.random.default_rng(9)
    eps = rng.uniform(0.5, 4.0, om.K)
    mu = rng.uniform(0.5, 3.0, om.K)
    bc = rng.integers(0, 2, (om.K, 4))
    u = random_fields(om.K, om.Np, 4)
    a = oracle.rhs(om, u, 1.0, eps, mu, bc)
    b = oracle.rhs(om, u, 1.0, 2.5 * eps, 2.5 * mu, bc)
    assert np.max(np.abs(a - 2.5 * b)) < 1e-12 * np.max(np.abs(a))
    assert oracle.maxwell.cfl_dt(om, 1.0, 2.5 * eps, 2.5 * mu) == pytest.approx(
        2.5 * oracle.maxwell.cfl_dt(om, 1.0, eps, mu), rel=1e-14)


def test_absorbing_box_lets_a_pulse_leave():
    """A divergence-free pulse E = curl(phi z), phi Gaussian, H = 0, in a box:
    with every face absorbing its energy falls below 2 % once the pulse has
    crossed the boundary (t = 2.5); with perfect conductors (upwind flux, only
    numerical dissipation) more than half remains."""
    verts, tets = kuhn_box_mesh(3, 0.1, 0)
    om = oracle.build_mesh(verts, tets, 3)
    w = 0.3
    phi = np.exp(-(om.x ** 2 + om.y ** 2 + om.z ** 2) / w ** 2)
    u0 = np.zeros((6, om.K, om.Np))
    u0[0] = -2 * om.y / w ** 2 * phi
    u0[1] = 2 * om.x / w ** 2 * phi
    dt = oracle.maxwell.cfl_dt(om, 0.9)
    steps = int(np.ceil(2.5 / dt))
    e0 = oracle.energy(om, u0)
    ua, _ = oracle.lserk4_run(om, u0, dt, steps, bc=np.ones((om.K, 4), int))
    up, _ = oracle.lserk4_run(om, u0, dt, steps)
    assert oracle.energy(om, ua) < 0.02 * e0
    assert oracle.energy(om, up) > 0.5 * e0


def test_material_energy_of_elementwise_constant_fields():
    """For fields constant on each element the energy is the exact integral
    1/2 sum_k vol_k (eps_k |E_k|^2 + mu_k |H_k|^2), with each volume taken from
    the vertices (|det| / 6), not from J or the mass matrix.  Swapped or
    missing eps, mu weights, or a lost factor 1/2, fail it."""
    verts, tets = kuhn_box_mesh(2, 0.15, 4)
    om = oracle.build_mesh(verts, tets, 3)
    rng = np.random.default_rng(17)
    eps = rng.uniform(0.5, 4.0, om.K)
    mu = rng.uniform(0.5, 3.0, om.K)
    E, H = rng.standard_normal((3, om.K)), rng.standard_normal((3, om.K))
    u = np.concatenate([E, H])[:, :, None] * np.ones(om.Np)
    X = verts[om.tets]
    vol = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 1))) / 6
    want = 0.5 * np.sum(vol * (eps * np.sum(E ** 2, 0) + mu * np.sum(H ** 2, 0)))
    assert abs(oracle.energy(om, u, eps, mu) - want) < 1e-12 * want
