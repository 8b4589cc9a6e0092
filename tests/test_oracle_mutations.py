"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a temporary copy of the C oracle (a dropped
term, a wrong sign or index, a transposed operand), builds it, binds it in
place of the real oracle and runs the pin tests of test_oracle_pins.py
against it: at least one pin must fail.  The real oracle is untouched.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "lpc_oracle.c")

MUTATIONS = {
    "stay term ignores the out-flow": ("s[i] = 1.0 - out;", "s[i] = 1.0;"),
    "Metropolis exponent sign": ("(dE > 0.0) ? exp(-dE) : 1.0", "(dE > 0.0) ? exp(dE) : 1.0"),
    "gather from the wrong side": ("neighbour(x, y, z, k ^ 1, nx, ny, nz, periodic)",
                                   "neighbour(x, y, z, k, nx, ny, nz, periodic)"),
    "conjugated rotation": ("m2[2 * i + 1] = c * mi + sn * mr;", "m2[2 * i + 1] = c * mi - sn * mr;"),
    "attempt factor 1/3": ("a_link / 6.0", "a_link / 3.0"),
    "link of a -a hop read at the source": ("((k & 1) ? j : i)", "i"),
    "displacement sign": ("double d = (k & 1) ? -1.0 : 1.0;", "double d = (k & 1) ? 1.0 : -1.0;"),
    "dMSD drift term sign": ("2.0 * (wp - wm)", "2.0 * (wp + wm)"),
    "walls treated as periodic": ("if (!periodic[a]) return -1;", "if (0) return -1;"),
    "transposed site index": ("return ((int64_t)z * ny + y) * nx + x;", "return ((int64_t)z * nx + x) * ny + y;"),
    "FID sums rho": ("double v[6] = {m[2 * i], ", "double v[6] = {rho[i], "),
    "solid target accepted": ("if (j >= 0 && !solid[i] && !solid[j])", "if (j >= 0 && !solid[i])"),
    "temperature dropped": ("double dE = (F[j] - F[i]) / kT;", "double dE = (F[j] - F[i]);"),
    "moment hop without rho": ("ua[a] += wk * (muj[a] + (a == axis ? d * rj : 0.0));",
                               "ua[a] += wk * muj[a];"),
    "reservoir in-weight with the out-hop's energy difference": ("double dE = (F[i] - rf[1]) / kT;",
                                                                 "double dE = (rf[1] - F[i]) / kT;"),
    "reservoir faces swapped": ("res + 5 * (2 * (k >> 1) + (k & 1))", "res + 5 * (2 * (k >> 1) + 1 - (k & 1))"),
    "no out-flow into a reservoir": ("} else if (j < 0 && !solid[i] && res) {", "} else if (0) {"),
    "reservoir magnetisation taken as its population": ("mjr = rf[3];", "mjr = rf[2];"),
    "region sums only for the first region": ("pl[6 * (1 + region[i]) + q] += v[q];",
                                              "if (region[i] == 0) pl[6 + q] += v[q];"),
    "region FID from the population": ("Mr[((int64_t)r * (nsteps + 1) + n) * 2] = t[0];",
                                       "Mr[((int64_t)r * (nsteps + 1) + n) * 2] = t[2];"),
}


def _pin_calls():
    """(name, callable) for every pin, with its parametrisations expanded."""
    calls = [
        ("detailed balance", lambda: [pins.test_weights_detailed_balance_and_walls(p)
                                      for p in [(1, 1, 1), (0, 1, 1), (1, 0, 0)]]),
        ("conservation", lambda: [pins.test_conservation(p) for p in [(1, 1, 1), (0, 1, 0)]]),
        ("boltzmann stationary", lambda: [pins.test_boltzmann_start_is_stationary(p)
                                          for p in [(1, 1, 1), (1, 0, 1)]]),
        ("boltzmann at kT", lambda: [pins.test_boltzmann_stationary_at_temperature(t) for t in (0.7, 2.5)]),
        ("uniform closed form", lambda: [pins.test_uniform_closed_form(a) for a in (0.3, 1.0)]),
        ("omega zero", pins.test_zero_omega_gives_m_equal_rho),
        ("single line", pins.test_uniform_omega_single_spectral_line),
        ("dense matrix", lambda: [pins.test_dense_matrix_power(p, s) for p, s in
                                  [((1, 1, 1), 41), ((0, 1, 1), 42), ((1, 1, 0), 43)]]),
        ("chain brute force", pins.test_msd_chain_with_walls_bruteforce),
        ("3d brute force", lambda: [pins.test_msd_3d_bruteforce(p) for p in [(1, 1, 1), (0, 1, 0)]]),
        ("one-step MSD", pins.test_one_step_msd_eq5),
        ("Kohn", lambda: [pins.test_kohn_identity_eq4(a) for a in (0, 2)]),
        ("links reduce to scalar", pins.test_links_uniform_reduce_to_scalar_alpha),
        ("links detailed balance", lambda: [pins.test_links_detailed_balance_and_boltzmann(p)
                                            for p in [(1, 1, 1), (0, 1, 1)]]),
        ("links brute force", lambda: [pins.test_links_dense_matrix_power(p) for p in [(1, 1, 1), (1, 0, 1)]]),
        ("reservoir Boltzmann", lambda: [pins.test_reservoir_boltzmann_is_stationary(p, f) for p, f in
                                         [((0, 1, 1), (0, 1)), ((0, 0, 0), (1, 2, 4))]]),
        ("reservoir chain", lambda: pins.test_reservoir_chain_linear_profile(1.0)),
        ("reservoir brute force", lambda: [pins.test_reservoir_dense_affine(p, s) for p, s in
                                           [((0, 1, 1), 81), ((0, 0, 1), 82)]]),
        ("regions", pins.test_regions_partition_the_totals_and_match_bruteforce),
        ("single region", pins.test_single_region_equals_the_totals_bitwise),
    ]
    return calls


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: " + old
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-ffp-contract=off", "-o", str(so), str(path), "-lm"])
    return str(so)


def test_real_oracle_passes_all_pins():
    for name, fn in _pin_calls():
        fn()


# a planted mistake may overflow (exp of a positive energy difference): the
# resulting inf / NaN values are expected and fail a pin
@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_each_mutation_fails_a_pin(name, tmp_path, monkeypatch):
    old, new = MUTATIONS[name]
    so = _build_mutant(tmp_path, old, new)
    monkeypatch.setattr(oracle, "_lib", oracle._bind(so))
    failed = []
    for pin, fn in _pin_calls():
        try:
            fn()
        except (AssertionError, ValueError, FloatingPointError):
            failed.append(pin)
    assert failed, "no pin caught the mutation: " + name


# Planted mistakes in the oracle's plain-Python downstream estimators: each
# replaces one function of the oracle module (for the duration of one test)
# and the pins of that estimator must fail.
def _region_diffusion_next_population(d, P, dt):
    d = np.asarray(d, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    return d / (2.0 * dt * P[1:len(d) + 1])


def _region_diffusion_initial_population(d, P, dt):
    d = np.asarray(d, dtype=np.float64)
    return d / (2.0 * dt * float(np.asarray(P)[0]))


def _region_diffusion_total_population(d, P, dt):
    d = np.asarray(d, dtype=np.float64)
    return d / (2.0 * dt * np.asarray(P, dtype=np.float64)[:len(d)].sum() / len(d))


PY_MUTATIONS = {
    "region D divides by P_r(n + 1)": ("region_diffusion", _region_diffusion_next_population),
    "region D divides by P_r(0)": ("region_diffusion", _region_diffusion_initial_population),
    "region D divides by the mean of P_r": ("region_diffusion", _region_diffusion_total_population),
}

PY_PINS = {
    "region_diffusion": [pins.test_kohn_and_region_diffusion_on_a_uniform_lattice,
                         pins.test_region_diffusion_against_dense_moments_off_equilibrium],
}


def test_real_downstream_estimators_pass_their_pins():
    for fns in PY_PINS.values():
        for fn in fns:
            fn()


@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_each_downstream_mutation_fails_a_pin(name, monkeypatch):
    attr, mutant = PY_MUTATIONS[name]
    monkeypatch.setattr(oracle, attr, mutant)
    failed = []
    for fn in PY_PINS[attr]:
        try:
            fn()
        except (AssertionError, ValueError, FloatingPointError, IndexError):
            failed.append(fn.__name__)
    assert failed, "no pin caught the mutation: " + name
