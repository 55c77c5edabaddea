"""Pins for the oracle's reference element (CPU only).

Each check compares the oracle with something fixed independently of it:
the paper's DOF table, closed-form integrals, Gauss-Lobatto points, the
exact polynomial calculus, and the summation-by-parts identity that ties the
mass, differentiation and lifting matrices together.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle.refelem import (dof_counts, lgl_points, ref_element, warp_blend_nodes)

ORDERS = list(range(1, 10))


def test_dof_counts_match_paper_table(golden_dir):
    rows = [list(map(int, ln.split())) for ln in open(f"{golden_dir}/dof_counts.txt")
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 7
    for N, Np, Nfp, NfNfp in rows:
        assert dof_counts(N) == (Np, Nfp, NfNfp)
        ref = ref_element(N)
        assert (ref.Np, ref.Nfp, ref.LIFT.shape[1]) == (Np, Nfp, NfNfp)


def test_lgl_closed_forms():
    assert np.allclose(lgl_points(1), [-1, 1], atol=0)
    assert np.allclose(lgl_points(2), [-1, 0, 1], atol=1e-15)
    a = 1 / math.sqrt(5)
    assert np.allclose(lgl_points(3), [-1, -a, a, 1], atol=1e-15)
    b = math.sqrt(3 / 7)
    assert np.allclose(lgl_points(4), [-1, -b, 0, b, 1], atol=1e-15)


def _bary(N):
    r, s, t = warp_blend_nodes(N)
    return np.stack([-(1 + r + s + t) / 2, (1 + r) / 2, (1 + s) / 2, (1 + t) / 2], 1)


@pytest.mark.parametrize("N", ORDERS)
def test_nodes_symmetric_inside_and_lgl_on_edges(N):
    L = _bary(N)
    Np = dof_counts(N)[0]
    assert L.shape == (Np, 4)
    assert L.min() > -1e-14 and np.allclose(L.sum(1), 1)
    # the node set is invariant under all 24 vertex permutations
    key = lambda A: np.array(sorted(map(tuple, np.round(A, 11))))  # noqa: E731
    base = key(L)
    for p in itertools.permutations(range(4)):
        assert np.max(np.abs(key(L[:, list(p)]) - base)) < 1e-11
    # every edge carries the N+1 Gauss-Lobatto points
    g = (lgl_points(N) + 1) / 2
    for i, j in itertools.combinations(range(4), 2):
        others = [k for k in range(4) if k not in (i, j)]
        on = np.all(np.abs(L[:, others]) < 1e-12, axis=1)
        assert on.sum() == N + 1
        assert np.allclose(np.sort(L[on, j]), g, atol=1e-14)
    # distinct nodes
    assert len(np.unique(np.round(L, 10), axis=0)) == Np


def test_low_order_nodes_closed_form():
    # N=1: the four vertices; N=2: vertices and edge midpoints
    r, s, t = warp_blend_nodes(1)
    assert np.allclose(np.stack([r, s, t], 1),
                       [[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], atol=1e-15)
    L = _bary(2)
    vals = np.unique(np.round(L, 12))
    assert np.allclose(vals, [0, 0.5, 1])


def _monomials(N):
    return [(a, b, c) for a in range(N + 1) for b in range(N + 1 - a) for c in range(N + 1 - a - b)]


@pytest.mark.parametrize("N", ORDERS)
def test_differentiation_exact_on_polynomials(N):
    ref = ref_element(N)
    r, s, t = ref.r, ref.s, ref.t
    err = 0.0
    for a, b, c in _monomials(N):
        f = r ** a * s ** b * t ** c
        fr = a * r ** max(a - 1, 0) * s ** b * t ** c
        fs = b * r ** a * s ** max(b - 1, 0) * t ** c
        ft = c * r ** a * s ** b * t ** max(c - 1, 0)
        err = max(err, np.abs(ref.Dr @ f - fr).max(), np.abs(ref.Ds @ f - fs).max(),
                  np.abs(ref.Dt @ f - ft).max())
    assert err < 1e-11 * N ** 2


def _tet_monomial_integral(a, b, c):
    """int_I r^a s^b t^c exactly: I = 2*(unit simplex) - 1, and
    int_simplex x^p y^q z^m = p! q! m! / (p+q+m+3)!."""
    tot = Fraction(0)
    for p in range(a + 1):
        for q in range(b + 1):
            for m in range(c + 1):
                coef = (math.comb(a, p) * math.comb(b, q) * math.comb(c, m)
                        * 2 ** (p + q + m) * (-1) ** (a - p + b - q + c - m))
                tot += coef * Fraction(math.factorial(p) * math.factorial(q) * math.factorial(m),
                                       math.factorial(p + q + m + 3))
    return 8 * tot


def _tri_monomial_integral(a, b):
    """int_T p^a q^b over T = {p,q >= -1, p+q <= 0} exactly (area 2)."""
    tot = Fraction(0)
    for i in range(a + 1):
        for j in range(b + 1):
            coef = math.comb(a, i) * math.comb(b, j) * 2 ** (i + j) * (-1) ** (a - i + b - j)
            tot += coef * Fraction(math.factorial(i) * math.factorial(j), math.factorial(i + j + 2))
    return 4 * tot


def test_exact_integral_helpers():
    assert _tet_monomial_integral(0, 0, 0) == Fraction(4, 3)
    assert _tri_monomial_integral(0, 0) == 2


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 9])
def test_mass_matrix_integrates_products_exactly(N):
    ref = ref_element(N)
    r, s, t = ref.r, ref.s, ref.t
    one = np.ones(ref.Np)
    assert abs(one @ ref.M @ one - 4 / 3) < 1e-13
    mons = _monomials(N)
    rng = np.random.default_rng(N)
    for _ in range(12):
        (a1, b1, c1), (a2, b2, c2) = (mons[i] for i in rng.integers(0, len(mons), 2))
        f = r ** a1 * s ** b1 * t ** c1
        g = r ** a2 * s ** b2 * t ** c2
        exact = float(_tet_monomial_integral(a1 + a2, b1 + b2, c1 + c2))
        assert abs(f @ ref.M @ g - exact) < 1e-12 * max(1.0, abs(exact)) * N


# face parameters used by these tests (f2 deliberately projected on (s,t))
_FACE_PARAM = {0: (0, 1), 1: (0, 2), 2: (1, 2), 3: (1, 2)}


@pytest.mark.parametrize("N", [1, 2, 3, 4, 6, 9])
def test_face_mass_integrates_exactly(N):
    ref = ref_element(N)
    rst = np.stack([ref.r, ref.s, ref.t])
    for f in range(4):
        fm = ref.Fmask[f]
        i, j = _FACE_PARAM[f]
        p, q = rst[i, fm], rst[j, fm]
        Mf = ref.face_mass[f]
        assert abs(np.ones(ref.Nfp) @ Mf @ np.ones(ref.Nfp) - 2.0) < 1e-13
        for a1, b1 in [(0, 0), (1, 0), (0, 1), (N, 0), (0, N), (N // 2, N - N // 2)]:
            for a2, b2 in [(1, 1) if N >= 2 else (1, 0), (0, N), (N, 0)]:
                u, v = p ** a1 * q ** b1, p ** a2 * q ** b2
                exact = float(_tri_monomial_integral(a1 + a2, b1 + b2))
                assert abs(u @ Mf @ v - exact) < 1e-12 * max(1, abs(exact)) * N


@pytest.mark.parametrize("N", ORDERS)
def test_summation_by_parts_reference(N):
    """int_I (d_mu u) v + u (d_mu v) = sum_faces int_f u v n_mu dS on I.

    With the face measure of the parameter triangle (area 2) the reference
    outward normals times dS/dA are f0: -e_t, f1: -e_s, f2: (1,1,1), f3: -e_r,
    so M D^r + (D^r)^T M = E2 - E3, M D^s + .. = E2 - E1, M D^t + .. = E2 - E0
    with E_f the face mass scattered into the face's rows/columns.  E_f is
    taken from M @ LIFT, so this ties D, M and LIFT together.
    """
    ref = ref_element(N)
    ML = ref.M @ ref.LIFT
    E = []
    for f in range(4):
        Ef = np.zeros((ref.Np, ref.Np))
        Ef[:, ref.Fmask[f]] = ML[:, f * ref.Nfp:(f + 1) * ref.Nfp]
        E.append(Ef)
        # lifting only reads face data: off-face rows of M LIFT in block f vanish
        off = np.setdiff1d(np.arange(ref.Np), ref.Fmask[f])
        assert np.abs(ML[np.ix_(off, np.arange(f * ref.Nfp, (f + 1) * ref.Nfp))]).max() < 1e-12
        assert np.allclose(ML[np.ix_(ref.Fmask[f], np.arange(f * ref.Nfp, (f + 1) * ref.Nfp))],
                           ref.face_mass[f], atol=1e-12)
    tol = 1e-11 * N ** 2
    for D, rhs in ((ref.Dr, E[2] - E[3]), (ref.Ds, E[2] - E[1]), (ref.Dt, E[2] - E[0])):
        S = ref.M @ D
        assert np.abs(S + S.T - rhs).max() < tol
    # D = M^-1 S with S from its own definition
    for D, S in zip((ref.Dr, ref.Ds, ref.Dt), ref.S):
        assert np.abs(ref.M @ D - S).max() < tol


def test_fmask_faces():
    for N in ORDERS:
        ref = ref_element(N)
        r, s, t = ref.r, ref.s, ref.t
        assert np.allclose(t[ref.Fmask[0]], -1)
        assert np.allclose(s[ref.Fmask[1]], -1)
        assert np.allclose((r + s + t)[ref.Fmask[2]], -1)
        assert np.allclose(r[ref.Fmask[3]], -1)
        assert all(np.all(np.diff(fm) > 0) for fm in ref.Fmask)
