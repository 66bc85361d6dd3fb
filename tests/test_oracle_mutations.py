"""The oracle's pins catch the mistakes they are meant to catch.

Each case builds a copy of the C oracle with one planted mistake (ORACLE_MUTATION, a
compile-time switch that is off in the oracle every other test and tool uses), points the
oracle module at the copy, runs the pin aimed at that kind of mistake and requires it to
fail. A control case builds the copy the same way without a mistake and requires the same
pins to pass. Everything runs on the CPU.
"""
import importlib

import pytest

import oracle

# (mutation, what is planted, pin module, pin function, pin arguments; "orc" marks the
# pins that take the oracle module as their argument)
CASES = [
    (1, "the (v.u)^2 term of the equilibrium dropped", "test_oracle_pins",
     "test_equilibrium_textbook_moments", {"orc": True}),
    (2, "transport pulling from x + v_j", "test_oracle_pins",
     "test_transport_moves_each_population_along_its_velocity", {"orc": True}),
    (3, "transposed moment matrix in the definition stepper", "test_oracle_pins",
     "test_collision_conserves_rho_and_q", {"orc": True, "method": 0}),
    (4, "wrong sign in block C3 of Appendix A", "test_oracle_pins",
     "test_shifted_form_equals_definition", {"orc": True}),
    (5, "rates applied to the wrong moments", "test_oracle_pins",
     "test_zero_relative_velocity_is_mrt", {"orc": True}),
    (6, "s+ and s- swapped in Appendix B's 2x2 block", "test_oracle_geier_pins",
     "test_cascaded_scheme_is_the_relative_velocity_scheme", {"orc": True}),
    (7, "D3Q19 edge weight 1/18", "test_oracle3d_pins", "test_equilibrium_textbook_moments",
     {}),
    (8, "D3Q19 basis polynomial ZY^2 written as YZ^2", "test_oracle3d_pins",
     "test_basis_is_unisolvent_and_shift_closed", {"lam": 1.0}),
    (9, "D3Q19 transport pulling from z + v_z", "test_oracle3d_pins",
     "test_transport_moves_populations_along_velocities", {}),
    (1, "the (v.u)^2 term of the equilibrium dropped (brute force)", "test_oracle_bruteforce",
     "test_definition_oracle_equals_brute_force",
     {"orc": True, "nx": 3, "ny": 3, "mode": 1, "lam": 1.0}),
    (2, "transport pulling from x + v_j (brute force)", "test_oracle_bruteforce",
     "test_definition_oracle_equals_brute_force",
     {"orc": True, "nx": 4, "ny": 5, "mode": 0, "lam": 2.0}),
    (5, "rates applied to the wrong moments (Geier brute force)", "test_oracle_bruteforce",
     "test_geier_definition_oracle_equals_brute_force", {"orc": True, "mode": 1, "lam": 1.0}),
    (7, "D3Q19 edge weight 1/18 (brute force)", "test_oracle3d_bruteforce",
     "test_d3q19_oracle_equals_brute_force", {"shape": (3, 3, 3), "mode": 1, "lam": 1.0}),
    (8, "D3Q19 basis polynomial ZY^2 written as YZ^2 (brute force)", "test_oracle3d_bruteforce",
     "test_d3q19_oracle_equals_brute_force", {"shape": (3, 3, 3), "mode": 0, "lam": 1.0}),
    (9, "D3Q19 transport pulling from z + v_z (brute force)", "test_oracle3d_bruteforce",
     "test_d3q19_oracle_equals_brute_force", {"shape": (3, 3, 3), "mode": 2, "lam": 1.5}),
]


@pytest.fixture()
def oracle_variant(tmp_path):
    """Build the oracle with -DORACLE_MUTATION=k and use it for the duration of a test."""
    saved = oracle.lib()

    def use(k):
        path = str(tmp_path / f"liboracle_m{k}.so")
        oracle._compile(path, [f"-DORACLE_MUTATION={k}"])
        oracle._lib = oracle._bind(path)

    yield use
    oracle._lib = saved


def _run_pin(module, name, kw):
    fn = getattr(importlib.import_module(module), name)
    args = dict(kw)
    if args.pop("orc", False):
        return fn(oracle, **args)
    return fn(**args)


@pytest.mark.parametrize("k,what,module,name,kw", CASES,
                         ids=[f"{c[0]}-{c[3]}" for c in CASES])
def test_pin_catches_planted_mistake(oracle_variant, k, what, module, name, kw):
    """A failed comparison, or an oracle that can no longer solve its moment system (a
    repeated basis polynomial makes M singular); the unmutated control below passes."""
    oracle_variant(k)
    with pytest.raises((AssertionError, FloatingPointError)):
        _run_pin(module, name, kw)


def test_pins_pass_on_the_unmutated_copy(oracle_variant):
    oracle_variant(0)
    for _, _, module, name, kw in CASES:
        _run_pin(module, name, kw)
