"""The oracle's pins catch the mistakes they are meant to catch.

Each case copies the C oracle's sources into a temporary folder, plants one mistake in
the copy by an exact text substitution (the original text must occur exactly once),
builds the copy, points the oracle module at it, runs the pin aimed at that kind of
mistake and requires it to fail. A control case builds unedited copies the same way and
requires the same pins to pass. The oracle's own sources are never edited and carry no
switch for any of this. Everything runs on the CPU.
"""
import importlib
import os
import shutil

import pytest

import oracle

D2 = "lbmrv_oracle.c"
D3 = "lbmrv_oracle3d.c"

# Planted mistakes: name -> list of (file, original text, replacement).
MUTATIONS = {
    "eq_quadratic_dropped": [
        (D2, "feq[j] = W[j] * rho * (1.0 + 3.0 * vu / l2 + 4.5 * vu * vu / (l2 * l2) - 1.5 * uu / l2);",
         "feq[j] = W[j] * rho * (1.0 + 3.0 * vu / l2 - 1.5 * uu / l2);")],
    "transport_reversed": [
        (D2, "int64_t xs = ((x - CX[j]) % nx + nx) % nx;\n"
             "                int64_t ys = ((y - CY[j]) % ny + ny) % ny;",
         "int64_t xs = ((x + CX[j]) % nx + nx) % nx;\n"
         "                int64_t ys = ((y + CY[j]) % ny + ny) % ny;")],
    "moment_matrix_transposed": [
        (D2, "orc_moment_matrix(utx, uty, l, M);\n"
             "    for (int k = 0; k < Q; ++k) {\n"
             "        double a = 0.0, b = 0.0;\n"
             "        for (int j = 0; j < Q; ++j) {\n"
             "            a += M[k * Q + j] * f[j];\n"
             "            b += M[k * Q + j] * feq[j];",
         "orc_moment_matrix(utx, uty, l, M);\n"
         "    for (int k = 0; k < Q; ++k) {\n"
         "        double a = 0.0, b = 0.0;\n"
         "        for (int j = 0; j < Q; ++j) {\n"
         "            a += M[j * Q + k] * f[j];\n"
         "            b += M[j * Q + k] * feq[j];")],
    "c3_sign": [
        (D2, "T[6 * Q + 4] = -3.0 * ux / l;", "T[6 * Q + 4] = 3.0 * ux / l;")],
    "rates_shifted_definition": [
        (D2, "ms[k] = m[k] + s[k] * (meq[k] - m[k]);\n"
             "    }\n"
             "    return orc_lu_solve(M, ms, fstar);\n"
             "}\n"
             "\n"
             "/* Shifting matrix",
         "ms[k] = m[k] + s[(k + 1) % Q] * (meq[k] - m[k]);\n"
         "    }\n"
         "    return orc_lu_solve(M, ms, fstar);\n"
         "}\n"
         "\n"
         "/* Shifting matrix")],
    "rates_shifted_geier_definition": [
        (D2, "ms[k] = m[k] + s[k] * (meq[k] - m[k]);\n"
             "    }\n"
             "    return orc_lu_solve(M, ms, fstar);\n"
             "}\n"
             "\n"
             "/* Geier's cascaded relaxation",
         "ms[k] = m[k] + s[(k + 1) % Q] * (meq[k] - m[k]);\n"
         "    }\n"
         "    return orc_lu_solve(M, ms, fstar);\n"
         "}\n"
         "\n"
         "/* Geier's cascaded relaxation")],
    "cascade_s_plus_minus_swapped": [
        (D2, "rhs[3] = sp * (meq[3] - m[3]) + sm * (meq[4] - m[4]);\n"
             "    rhs[4] = sm * (meq[3] - m[3]) + sp * (meq[4] - m[4]);",
         "rhs[3] = sm * (meq[3] - m[3]) + sp * (meq[4] - m[4]);\n"
         "    rhs[4] = sp * (meq[3] - m[3]) + sm * (meq[4] - m[4]);")],
    "d3q19_edge_weight": [
        (D3, "(nnz == 1 ? 1.0 / 18.0 : 1.0 / 36.0)", "(1.0 / 18.0)")],
    "d3q19_basis_repeated": [
        (D3, "case 15: return Z * Y * Y / l3;", "case 15: return Y * Z * Z / l3;")],
    "d3q19_transport_z_reversed": [
        (D3, "int64_t zs = ((z - CZ3[j]) % nz + nz) % nz;",
         "int64_t zs = ((z + CZ3[j]) % nz + nz) % nz;")],
}

# (mutation, pin module, pin function, pin arguments; "orc" marks the pins that take the
# oracle module as their argument)
CASES = [
    ("eq_quadratic_dropped", "test_oracle_pins", "test_equilibrium_textbook_moments",
     {"orc": True}),
    ("transport_reversed", "test_oracle_pins",
     "test_transport_moves_each_population_along_its_velocity", {"orc": True}),
    ("moment_matrix_transposed", "test_oracle_pins", "test_collision_conserves_rho_and_q",
     {"orc": True, "method": 0}),
    ("c3_sign", "test_oracle_pins", "test_shifted_form_equals_definition", {"orc": True}),
    ("rates_shifted_definition", "test_oracle_pins", "test_zero_relative_velocity_is_mrt",
     {"orc": True}),
    ("cascade_s_plus_minus_swapped", "test_oracle_geier_pins",
     "test_cascaded_scheme_is_the_relative_velocity_scheme", {"orc": True}),
    ("d3q19_edge_weight", "test_oracle3d_pins", "test_equilibrium_textbook_moments", {}),
    ("d3q19_basis_repeated", "test_oracle3d_pins",
     "test_basis_is_unisolvent_and_shift_closed", {"lam": 1.0}),
    ("d3q19_transport_z_reversed", "test_oracle3d_pins",
     "test_transport_moves_populations_along_velocities", {}),
    ("eq_quadratic_dropped", "test_oracle_bruteforce",
     "test_definition_oracle_equals_brute_force",
     {"orc": True, "nx": 3, "ny": 3, "mode": 1, "lam": 1.0}),
    ("transport_reversed", "test_oracle_bruteforce",
     "test_definition_oracle_equals_brute_force",
     {"orc": True, "nx": 4, "ny": 5, "mode": 0, "lam": 2.0}),
    ("rates_shifted_geier_definition", "test_oracle_bruteforce",
     "test_geier_definition_oracle_equals_brute_force", {"orc": True, "mode": 1, "lam": 1.0}),
    ("d3q19_edge_weight", "test_oracle3d_bruteforce", "test_d3q19_oracle_equals_brute_force",
     {"shape": (3, 3, 3), "mode": 1, "lam": 1.0}),
    ("d3q19_basis_repeated", "test_oracle3d_bruteforce",
     "test_d3q19_oracle_equals_brute_force", {"shape": (3, 3, 3), "mode": 0, "lam": 1.0}),
    ("d3q19_transport_z_reversed", "test_oracle3d_bruteforce",
     "test_d3q19_oracle_equals_brute_force", {"shape": (3, 3, 3), "mode": 2, "lam": 1.5}),
]


def _edited_sources(folder, edits):
    """Copies of the two C sources in `folder`, with `edits` applied; each original text
    must occur exactly once in its file."""
    paths = {}
    for name in (D2, D3):
        dst = os.path.join(folder, name)
        shutil.copyfile(os.path.join(os.path.dirname(oracle.__file__), name), dst)
        paths[name] = dst
    for name, old, new in edits:
        with open(paths[name]) as fh:
            text = fh.read()
        assert text.count(old) == 1, (name, old, text.count(old))
        with open(paths[name], "w") as fh:
            fh.write(text.replace(old, new))
    return [paths[D2], paths[D3]]


@pytest.fixture()
def oracle_variant(tmp_path):
    """Build the oracle from edited copies and use it for the duration of a test."""
    saved = oracle.lib()

    def use(mutation):
        folder = tmp_path / (mutation or "control")
        folder.mkdir()
        srcs = _edited_sources(str(folder), MUTATIONS[mutation] if mutation else [])
        path = str(folder / "liboracle.so")
        oracle._compile(path, srcs=srcs)
        oracle._lib = oracle._bind(path)

    yield use
    oracle._lib = saved


def _run_pin(module, name, kw):
    fn = getattr(importlib.import_module(module), name)
    args = dict(kw)
    if args.pop("orc", False):
        return fn(oracle, **args)
    return fn(**args)


def test_every_substitution_matches_once(tmp_path):
    for name, edits in MUTATIONS.items():
        folder = tmp_path / name
        folder.mkdir()
        _edited_sources(str(folder), edits)


@pytest.mark.parametrize("mutation,module,name,kw", CASES,
                         ids=[f"{c[0]}-{c[2]}" for c in CASES])
def test_pin_catches_planted_mistake(oracle_variant, mutation, module, name, kw):
    """A failed comparison, or an oracle that can no longer solve its moment system (a
    repeated basis polynomial makes M singular); the unedited control below passes."""
    oracle_variant(mutation)
    with pytest.raises((AssertionError, FloatingPointError)):
        _run_pin(module, name, kw)


def test_pins_pass_on_the_unedited_copy(oracle_variant):
    oracle_variant(None)
    for _, module, name, kw in CASES:
        _run_pin(module, name, kw)
