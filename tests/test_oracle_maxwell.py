"""Pins for the oracle's Maxwell operator, LSERK4 and energy (CPU only)."""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
from workloads import cavity_mode, kuhn_box_mesh, random_fields


def _mesh(n, N, jitter=0.1, seed=0):
    verts, tets = kuhn_box_mesh(n, jitter, seed)
    return oracle.build_mesh(verts, tets, N), verts


def _energy_rate(m, u, r):
    """d/dt of 1/2 sum J u^T M u along du/dt = r."""
    return float(np.sum(m.J[None, :, None] * u * np.einsum("ij,fkj->fki", m.ref.M, r)))


def _poly_fields(q, x, y, z):
    """Fields of degree q (1 or 2) and their curls, written out by hand."""
    one, zero = np.ones_like(x), np.zeros_like(x)
    if q == 1:
        E = np.stack([y, z, x + y])
        H = np.stack([z - x, x, y])
        curlE = np.stack([zero, -one, -one])
        curlH = np.stack([one, one, one])
    else:
        E = np.stack([y ** 2, z * x, x + y ** 2])
        H = np.stack([z ** 2 - x, x ** 2, y * z])
        curlE = np.stack([2 * y - x, -one, z - 2 * y])
        curlH = np.stack([z, 2 * z, 2 * x])
    return E, H, curlE, curlH


@pytest.mark.parametrize("q", [1, 2])
def test_curl_fixture_consistency(q):
    """The hand-written curls of _poly_fields, checked by central differences."""
    p, h = np.array([0.3, -0.2, 0.5]), 1e-5
    E, H, cE, cH = _poly_fields(q, *[np.array([c]) for c in p])
    for i, want in ((0, cE), (1, cH)):
        J = np.zeros((3, 3))
        for d in range(3):
            e = np.zeros(3)
            e[d] = h
            fp = _poly_fields(q, *[np.array([c]) for c in p + e])[i][:, 0]
            fm = _poly_fields(q, *[np.array([c]) for c in p - e])[i][:, 0]
            J[:, d] = (fp - fm) / (2 * h)
        curl = np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])
        assert np.allclose(curl, want[:, 0], atol=1e-8)


@pytest.mark.parametrize("N", [1, 2, 3])
def test_rhs_exact_curl_on_interior_elements(N):
    """A global polynomial field of degree <= N has no jumps across interior
    faces, so on elements without a wall face the RHS is its exact curl."""
    m, _ = _mesh(3, N, 0.15, 2)
    E, H, curlE, curlH = _poly_fields(min(N, 2), m.x, m.y, m.z)
    r = oracle.rhs(m, np.concatenate([E, H]))
    interior = ~m.boundary.any(axis=1)
    assert interior.sum() > 0
    expect = np.concatenate([curlH, -curlE])
    assert np.abs(r[:, interior] - expect[:, interior]).max() < 1e-10


def _upwind_by_paper(n, uM, uP):
    """n.(F - F*) in the paper's jump notation [[u]] = u+ - u-, Z = Y = 1:
    E: 1/2 n x ([[H]] - n x [[E]]),   H: 1/2 n x (-[[E]] - n x [[H]])."""
    jE, jH = uP[:3] - uM[:3], uP[3:] - uM[3:]
    fE = 0.5 * np.cross(n, jH - np.cross(n, jE))
    fH = 0.5 * np.cross(n, -jE - np.cross(n, jH))
    return np.concatenate([fE, fH])


@pytest.mark.parametrize("N", [1, 3])
def test_upwind_flux_two_tets_by_hand(N):
    """Constant states on two tets: the volume term vanishes and
    int_{D_k} rhs = sum_faces area_f * n.(F - F*)_f (M LIFT = face mass)."""
    verts = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [0.9, 1.1, 1.2]], float)
    m = oracle.build_mesh(verts, np.array([[0, 1, 2, 3], [1, 2, 3, 4]]), N)
    rng = np.random.default_rng(7)
    uA, uB = rng.standard_normal(6), rng.standard_normal(6)
    u = np.empty((6, 2, m.Np))
    u[:, 0] = uA[:, None]
    u[:, 1] = uB[:, None]
    r = oracle.rhs(m, u)
    integ = np.einsum("k,fki->fk", m.J, np.einsum("ij,fkj->fki", m.ref.M, r))
    for k, (mine, other) in enumerate(((uA, uB), (uB, uA))):
        tot = np.zeros(6)
        for f in range(4):
            n = np.array([m.nx[k, f], m.ny[k, f], m.nz[k, f]])
            if m.boundary[k, f]:
                ghost = np.concatenate([-mine[:3], mine[3:]])     # PEC mirror
            else:
                ghost = other
            tot += 2 * m.sJ[k, f] * _upwind_by_paper(n, mine, ghost)
        assert np.allclose(integ[:, k], tot, rtol=1e-12, atol=1e-12)


def test_energy_rate_central_zero_upwind_dissipative():
    m, _ = _mesh(2, 3, 0.15, 3)
    for seed in range(3):
        u = random_fields(m.K, m.Np, seed)
        scale = np.sum(u * u)
        assert abs(_energy_rate(m, u, oracle.rhs(m, u, alpha=0.0))) < 1e-12 * scale
        assert _energy_rate(m, u, oracle.rhs(m, u, alpha=1.0)) < -1e-3 * scale / m.K


def test_rhs_is_linear():
    m, _ = _mesh(1, 2)
    u, v = random_fields(m.K, m.Np, 1), random_fields(m.K, m.Np, 2)
    assert np.allclose(oracle.rhs(m, 2 * u - 3 * v), 2 * oracle.rhs(m, u) - 3 * oracle.rhs(m, v), atol=1e-11)


def test_lserk4_order_conditions_exact():
    from fractions import Fraction
    a, b, c = oracle.lserk4_coefficients(exact=True)
    # amplification polynomial R(z) for y' = z y over one step
    poly_u, poly_r = [Fraction(1)], [Fraction(0)]
    for i in range(5):
        zr = [Fraction(0)] + poly_u
        poly_r = [(a[i] * (poly_r[j] if j < len(poly_r) else 0)) + (zr[j] if j < len(zr) else 0)
                  for j in range(max(len(poly_r), len(zr)))]
        poly_u = [(poly_u[j] if j < len(poly_u) else 0) + b[i] * poly_r[j] for j in range(len(poly_r))]
    for k in range(5):
        assert abs(poly_u[k] - Fraction(1, math.factorial(k))) < Fraction(1, 10 ** 20)
    # stage times c_i: the time reached before stage i when integrating y' = 1
    t, res = Fraction(0), Fraction(0)
    for i in range(5):
        assert abs(c[i] - t) < Fraction(1, 10 ** 20)
        res = a[i] * res + 1
        t += b[i] * res
    assert abs(t - 1) < Fraction(1, 10 ** 20)


@pytest.mark.slow
def test_lserk4_against_matrix_exponential():
    """On a tiny mesh the fully discrete solution approaches exp(T A) u0 at 4th order."""
    m, _ = _mesh(1, 1, 0.1, 4)
    n = 6 * m.K * m.Np
    A = np.empty((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1
        A[:, j] = oracle.rhs(m, e.reshape(6, m.K, m.Np)).ravel()
    u0 = random_fields(m.K, m.Np, 5)
    T = 0.5
    exact = (scipy.linalg.expm(T * A) @ u0.ravel()).reshape(u0.shape)
    errs = []
    for ns in (20, 40):
        u, _ = oracle.lserk4_run(m, u0, T / ns, ns)
        errs.append(np.linalg.norm(u - exact) / np.linalg.norm(exact))
    assert errs[1] < 1e-5
    assert 12 < errs[0] / errs[1] < 20          # ~2^4
    # the CFL step is inside the stability region: |R(dt lambda)| <= 1
    lam = np.linalg.eigvals(A)
    assert lam.real.max() < 1e-12
    a, b, _ = oracle.lserk4_coefficients()
    z = lam * oracle.cfl_dt(m)
    uu, rr = np.ones_like(z), np.zeros_like(z)
    for i in range(5):
        rr = a[i] * rr + z * uu
        uu = uu + b[i] * rr
    assert np.abs(uu).max() <= 1 + 1e-12


def _l2err(m, u, ex):
    d = u - ex
    return math.sqrt(np.sum(m.J[None, :, None] * d * np.einsum("ij,fkj->fki", m.ref.M, d)))


def _cavity_error(n, N, T=0.25):
    m, _ = _mesh(n, N)
    ns = math.ceil(T / oracle.cfl_dt(m))
    u, _ = oracle.lserk4_run(m, cavity_mode(m.x, m.y, m.z, 0.0), T / ns, ns)
    return _l2err(m, u, cavity_mode(m.x, m.y, m.z, T))


def test_cavity_eigenmode_spectral_in_N():
    errs = [_cavity_error(2, N) for N in (1, 2, 3, 4)]
    assert all(e2 < 0.35 * e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 2e-2


@pytest.mark.slow
@pytest.mark.parametrize("N", [1, 2, 3])
def test_cavity_eigenmode_h_convergence(N):
    """EOC between h = 1 and h = 1/2 approaches N+1 (the paper's h^(N+1) trend)."""
    eoc = math.log(_cavity_error(2, N) / _cavity_error(4, N)) / math.log(2)
    assert eoc > N + 0.3


def test_energy_non_increasing_and_conserved_direction():
    m, _ = _mesh(2, 3)
    u = cavity_mode(m.x, m.y, m.z, 0.0)
    dt = oracle.cfl_dt(m)
    e = [oracle.energy(m, u)]
    res = np.zeros_like(u)
    for _ in range(6):
        u, res = oracle.lserk4_run(m, u, dt, 1, res)
        e.append(oracle.energy(m, u))
    assert all(b <= a * (1 + 1e-14) for a, b in zip(e, e[1:]))
    assert e[-1] > 0.95 * e[0]
    # the exact continuous energy of the mode: 1/2 int |E|^2 + |H|^2 is constant
    assert abs(e[0] - 3.0) < 0.05


def test_cfl_dt_formula():
    m, _ = _mesh(2, 4)
    assert abs(oracle.cfl_dt(m) - np.min(1 / m.Fscale) * 2 / 25) < 1e-15
