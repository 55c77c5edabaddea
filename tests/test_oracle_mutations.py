"""Planted mistakes in the oracle, caught by its pins (CPU only).

Each case below is a plausible slip in one oracle module: a dropped term, a
wrong sign, a transposed or swapped operand, a wrong weight, a wrong
constant.  The case builds a mutant of that module from its own source with
exactly that one substitution, swaps the mutant's functions in for the real
ones wherever the oracle package refers to them, and runs a named pin from
tests/test_oracle_*.py.  The pin must fail with an AssertionError.  The pins
compare against closed forms, exact solutions, energy identities and the
paper's own flux form, never against the oracle code itself, so a mistake
that none of them notices would show up here as a surviving mutant.
"""
import importlib.util
import os
import types

import pytest

import oracle
import oracle.maxwell
import oracle.mesh
import oracle.partition
import oracle.refelem
from workloads import kuhn_box_mesh

TESTS = os.path.dirname(os.path.abspath(__file__))
ORACLE = os.path.join(os.path.dirname(TESTS), "oracle")


def _pin_module(name):
    spec = importlib.util.spec_from_file_location(f"_pins_{name}", os.path.join(TESTS, name + ".py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = {n: _pin_module(n) for n in ("test_oracle_maxwell", "test_oracle_materials",
                                     "test_oracle_mesh", "test_oracle_refelem",
                                     "test_oracle_partition")}

# (id, oracle module, exact source text, replacement, pin module, pin, pin arguments)
CASES = [
    ("curl-H-component-sign", "maxwell", "curlH = np.stack([dy[5] - dz[4],",
     "curlH = np.stack([dz[4] - dy[5],",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("minus-curl-E-dropped", "maxwell", "return np.concatenate([curlH, -curlE])",
     "return np.concatenate([curlH, curlE])",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("metric-transposed-in-d/dx", "maxwell",
     "dx = c(mesh.rx) * ur + c(mesh.sx) * us + c(mesh.tx) * ut",
     "dx = c(mesh.rx) * ur + c(mesh.ry) * us + c(mesh.rz) * ut",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("Ds-used-for-Dt", "maxwell", 'ut = np.einsum("ij,fkj->fki", ref.Dt, u)',
     'ut = np.einsum("ij,fkj->fki", ref.Ds, u)',
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("PEC-ghost-E-not-mirrored", "maxwell",
     "uP[:3] = np.where(pec[None, :, :, None], -uM[:3], uP[:3])",
     "uP[:3] = np.where(pec[None, :, :, None], uM[:3], uP[:3])",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("upwind-penalty-sign", "maxwell", "(zp * nxjH[i] - alpha * nxnxjE[i])",
     "(zp * nxjH[i] + alpha * nxnxjE[i])",
     "test_oracle_maxwell", "test_energy_rate_central_zero_upwind_dissipative", {}),
    ("jump-taken-the-other-way", "maxwell", "jE = uP[:3] - uM[:3]", "jE = uM[:3] - uP[:3]",
     "test_oracle_maxwell", "test_energy_rate_central_zero_upwind_dissipative", {}),
    ("Fscale-dropped", "maxwell", "flux = np.stack(fE + fH) * mesh.Fscale[None, :, :, None]",
     "flux = np.stack(fE + fH)",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("Z-minus-for-Z-plus-in-E-row", "maxwell", "fE = [cE * (zp * nxjH[i]",
     "fE = [cE * (ZM[:, :, None] * nxjH[i]",
     "test_oracle_materials", "test_material_upwind_flux_is_the_exact_riemann_flux", {"N": 1}),
    ("Y-average-misweighted", "maxwell", "cH = (1.0 / (YM + YP))[:, :, None]",
     "cH = (1.0 / (ZM + ZP))[:, :, None]",
     "test_oracle_materials", "test_material_energy_conserved_by_central_flux_and_dissipated_by_upwind",
     {"N": 2}),
    ("1/eps-weight-dropped", "maxwell", "np.repeat(1.0 / eps[None, :], 3, axis=0)",
     "np.repeat(np.ones_like(eps)[None, :], 3, axis=0)",
     "test_oracle_materials", "test_material_energy_conserved_by_central_flux_and_dissipated_by_upwind",
     {"N": 2}),
    ("absorbing-face-treated-as-wall", "maxwell", "uP = np.where(absorb[None, :, :, None], 0.0, uP)",
     "uP = np.where(absorb[None, :, :, None], uP, uP)",
     "test_oracle_materials", "test_material_upwind_flux_is_the_exact_riemann_flux", {"N": 1}),
    ("dt-dropped-in-stage", "maxwell", "res = a * res + dt * r", "res = a * res + r",
     "test_oracle_maxwell", "test_energy_non_increasing_and_conserved_direction", {}),
    ("RK-coefficient-digit", "maxwell", "Fraction(5161836677717, 13612068292357)",
     "Fraction(5161836677718, 13612068292357)",
     "test_oracle_maxwell", "test_lserk4_order_conditions_exact", {}),
    ("energy-half-dropped", "maxwell", "return 0.5 * float(np.sum(", "return float(np.sum(",
     "test_oracle_maxwell", "test_energy_non_increasing_and_conserved_direction", {}),
    ("energy-mu-weight-on-E", "maxwell",
     "w = np.concatenate([np.repeat(eps[None, :], 3, axis=0), np.repeat(mu[None, :], 3, axis=0)])",
     "w = np.concatenate([np.repeat(mu[None, :], 3, axis=0), np.repeat(eps[None, :], 3, axis=0)])",
     "test_oracle_materials", "test_material_energy_of_elementwise_constant_fields", {}),
    ("CFL-wave-speed", "maxwell", "slow = np.sqrt(eps * mu)[:, None]", "slow = np.sqrt(eps / mu)[:, None]",
     "test_oracle_materials", "test_material_scaling_law", {}),
    ("metric-row-transposed", "mesh",
     "m.rx, m.ry, m.rz = inv[:, 0, 0], inv[:, 0, 1], inv[:, 0, 2]",
     "m.rx, m.ry, m.rz = inv[:, 0, 0], inv[:, 1, 0], inv[:, 2, 0]",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("normals-inward", "mesh", "n[out < 0] *= -1", "n[out > 0] *= -1",
     "test_oracle_maxwell", "test_energy_rate_central_zero_upwind_dissipative", {}),
    ("face-jacobian-not-halved", "mesh", "m.sJ = area / 2", "m.sJ = area",
     "test_oracle_mesh", "test_face_geometry", {"mesh3": None}),
    ("jacobian-scaled", "mesh", "m.J = np.linalg.det(A)  ", "m.J = 8 * np.linalg.det(A)  ",
     "test_oracle_mesh", "test_volumes_and_jacobians", {"mesh3": None}),
    ("Dr-from-s-derivative", "refelem", "self.Dr = Vr @ Vinv", "self.Dr = Vs @ Vinv",
     "test_oracle_refelem", "test_differentiation_exact_on_polynomials", {"N": 2}),
    ("mass-quadrature-too-low", "refelem", "qr, qs, qt, qw = tet_quadrature(N + 2)",
     "qr, qs, qt, qw = tet_quadrature(N)",
     "test_oracle_refelem", "test_mass_matrix_integrates_products_exactly", {"N": 3}),
    ("LIFT-without-inverse-mass", "refelem", "self.LIFT = self.Minv @ E", "self.LIFT = E",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("face-mass-on-the-next-face", "refelem", "fr, fs, ft = face_points(f, pp, pq)",
     "fr, fs, ft = face_points((f + 1) % 4, pp, pq)",
     "test_oracle_refelem", "test_face_mass_integrates_exactly", {"N": 2}),
    ("face-order-s-and-t-swapped", "refelem",
     "on_face = (np.abs(1 + t) < tol, np.abs(1 + s) < tol,",
     "on_face = (np.abs(1 + s) < tol, np.abs(1 + t) < tol,",
     "test_oracle_refelem", "test_fmask_faces", {}),
    ("neighbour-node-off-by-one", "mesh", "vmapP[k, f] = k2 * Np + idP[j2]",
     "vmapP[k, f] = k2 * Np + idP[(j2 + 1) % Nfp]",
     "test_oracle_mesh", "test_connectivity_invariants", {"N": 2}),
    ("H-row-cross-term-sign", "maxwell", "(-yp * nxjE[i] - alpha * nxnxjH[i])",
     "(yp * nxjE[i] - alpha * nxnxjH[i])",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("H-row-penalty-sign", "maxwell", "(-yp * nxjE[i] - alpha * nxnxjH[i])",
     "(-yp * nxjE[i] + alpha * nxnxjH[i])",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("PEC-ghost-H-mirrored", "maxwell", "uP[3:] = np.where(pec[None, :, :, None], uM[3:], uP[3:])",
     "uP[3:] = np.where(pec[None, :, :, None], -uM[3:], uP[3:])",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("boundary-impedance-one", "maxwell", "ZP = np.where(bnd, ZM, Z[mesh.EToE])",
     "ZP = np.where(bnd, 1.0, Z[mesh.EToE])",
     "test_oracle_materials", "test_material_upwind_flux_is_the_exact_riemann_flux", {"N": 1}),
    ("H-rows-divided-by-eps", "maxwell", "np.repeat(1.0 / mu[None, :], 3, axis=0)",
     "np.repeat(1.0 / eps[None, :], 3, axis=0)",
     "test_oracle_materials", "test_material_energy_conserved_by_central_flux_and_dissipated_by_upwind",
     {"N": 2}),
    ("curl-E-component-sign", "maxwell", "dz[0] - dx[2]", "dx[2] - dz[0]",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("metric-entry-in-d/dy", "maxwell",
     "dy = c(mesh.ry) * ur + c(mesh.sy) * us + c(mesh.ty) * ut",
     "dy = c(mesh.ry) * ur + c(mesh.sy) * us + c(mesh.tz) * ut",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("stage-advances-with-rhs", "maxwell", "return u + b * res, res", "return u + b * r, res",
     "test_oracle_maxwell", "test_energy_non_increasing_and_conserved_direction", {}),
    ("four-stages", "maxwell", "        for i in range(5):\n            u, res = stage_update(",
     "        for i in range(4):\n            u, res = stage_update(",
     "test_oracle_maxwell", "test_energy_non_increasing_and_conserved_direction", {}),
    ("energy-with-inverse-mass", "maxwell", 'Mu = np.einsum("ij,fkj->fki", mesh.ref.M, u)',
     'Mu = np.einsum("ij,fkj->fki", mesh.ref.Minv, u)',
     "test_oracle_materials", "test_material_energy_of_elementwise_constant_fields", {}),
    ("CFL-max-not-min", "maxwell", "C * float(np.min(slow / mesh.Fscale))",
     "C * float(np.max(slow / mesh.Fscale))",
     "test_oracle_maxwell", "test_cfl_dt_formula", {}),
    ("absorbing-flag-inverted", "maxwell", "else np.asarray(bc) == 1)", "else np.asarray(bc) == 0)",
     "test_oracle_materials", "test_material_upwind_flux_is_the_exact_riemann_flux", {"N": 1}),
    ("double-cross-operand-order", "maxwell", "nxnxjE = _cross(n, nxjE)", "nxnxjE = _cross(nxjE, n)",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("RK-stage-time-digit", "maxwell", "Fraction(2526269341429, 6820363962896)",
     "Fraction(2526269341428, 6820363962896)",
     "test_oracle_maxwell", "test_lserk4_order_conditions_exact", {}),
    ("Fscale-inverted", "mesh", "m.Fscale = m.sJ / m.J[:, None]", "m.Fscale = m.J[:, None] / m.sJ",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("orientation-not-fixed", "mesh", "tets[neg] = tets[neg][:, [0, 1, 3, 2]]",
     "tets[neg] = tets[neg][:, [0, 1, 2, 3]]",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("Dt-times-V-not-inverse", "refelem", "self.Dt = Vt @ Vinv", "self.Dt = Vt @ V",
     "test_oracle_maxwell", "test_rhs_exact_curl_on_interior_elements", {"N": 2}),
    ("LIFT-halved", "refelem", "self.LIFT = self.Minv @ E", "self.LIFT = self.Minv @ E * 0.5",
     "test_oracle_maxwell", "test_upwind_flux_two_tets_by_hand", {"N": 1}),
    ("face-quadrature-too-low", "refelem", "pp, pq, pw = tri_quadrature(N + 1)",
     "pp, pq, pw = tri_quadrature(N)",
     "test_oracle_refelem", "test_face_mass_integrates_exactly", {"N": 3}),
    ("queue-last-in-first-out", "partition", "queue.append(f)", "queue.insert(0, f)",
     "test_oracle_partition", "test_first_grid_block_in_queue_order", {}),
    ("one-shared-face-counted", "partition",
     "for f in face_neighbours(e):\n                    shared[f]",
     "for f in face_neighbours(e)[:1]:\n                    shared[f]",
     "test_oracle_partition", "test_grid_and_mesh_follow_the_greedy_rule", {}),
    ("greedy-ties-to-last-queued", "partition",
     "if shared.get(queue[i], 0) > shared.get(queue[best], 0):",
     "if shared.get(queue[i], 0) >= shared.get(queue[best], 0):",
     "test_oracle_partition", "test_first_grid_block_in_queue_order", {}),
    ("shared-faces-not-counted", "partition", "shared[f] = shared.get(f, 0) + 1", "shared[f] = 1",
     "test_oracle_partition", "test_grid_and_mesh_follow_the_greedy_rule", {}),
    ("next-seed-from-queue-end", "partition", "carry = queue[0] if queue else None",
     "carry = queue[-1] if queue else None",
     "test_oracle_partition", "test_next_block_seeded_by_the_first_queue_entry", {}),
]


def _mutant(modname, old, new):
    path = os.path.join(ORACLE, modname + ".py")
    src = open(path).read()
    assert src.count(old) == 1, f"mutation site not unique or gone: {old!r}"
    mod = types.ModuleType(f"oracle._mutant_{modname}")
    mod.__package__ = "oracle"
    mod.__file__ = path
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    return mod


def _install(monkeypatch, modname, mutant):
    """Every name that refers to an object of the real module (its own
    namespace, the package's re-exports, other modules' `from .x import y`,
    the pin modules' imports) is pointed at the mutant's object of that name."""
    real = getattr(oracle, modname)
    swap = {id(v): getattr(mutant, k) for k, v in vars(real).items()
            if not k.startswith("__") and hasattr(mutant, k)
            and (isinstance(v, (types.FunctionType, type)) or hasattr(v, "cache_info"))}
    for m in (oracle, oracle.maxwell, oracle.mesh, oracle.partition, oracle.refelem,
              *PINS.values()):
        for k, v in list(vars(m).items()):
            if id(v) in swap:
                monkeypatch.setattr(m, k, swap[id(v)])


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(case, monkeypatch):
    _, modname, old, new, pin_mod, pin, kwargs = case
    _install(monkeypatch, modname, _mutant(modname, old, new))
    kwargs = dict(kwargs)
    if "mesh3" in kwargs:                      # the pin's module fixture, built by the mutant
        verts, tets = kuhn_box_mesh(3, 0.15, 0)
        kwargs["mesh3"] = (oracle.build_mesh(verts, tets, 3), verts)
    with pytest.raises(AssertionError):
        getattr(PINS[pin_mod], pin)(**kwargs)


def test_unmutated_oracle_passes_the_same_pins():
    """The harness itself: with no mutation every pin used above passes."""
    seen = set()
    for _, _, _, _, pin_mod, pin, kwargs in CASES:
        key = (pin_mod, pin, tuple(sorted(kwargs)))
        if key in seen:
            continue
        seen.add(key)
        kwargs = dict(kwargs)
        if "mesh3" in kwargs:
            verts, tets = kuhn_box_mesh(3, 0.15, 0)
            kwargs["mesh3"] = (oracle.build_mesh(verts, tets, 3), verts)
        getattr(PINS[pin_mod], pin)(**kwargs)
