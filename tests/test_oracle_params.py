"""Pins of the parameter layer against the paper's Tables 1 and 2.

The dimensionless numbers the oracle and the library take (Ro, Re, Fr, A,
sigma, delta) are checked against the physical parameters the paper prints,
through the relations of Section 2 (Eqs. relation, Rhines, Munk, Reb, ndim,
and the two Sverdrup velocity scales).  Tolerances follow the number of
significant digits printed in the tables.
"""
import math

import pytest

from tests.golden.load import read_table

YEAR = 365.25 * 86400.0


def rel(a, b):
    return abs(a - b) / abs(b)


@pytest.mark.parametrize("col", [0, 1])
def test_one_layer_table(col):
    t = {k: v[col] for k, v in read_table("table1_one_layer.txt").items()}
    L = t["L_km"] * 1e3
    beta = t["beta"]
    # Eq. Rhines: delta_I/L = Ro^(1/2)
    assert rel(t["dI_over_L"] ** 2, t["Ro"]) < 1e-12
    # Eq. Munk: delta_M/L = (Ro/Re)^(1/3)
    assert rel(t["dM_over_L"] ** 3, t["Ro"] / t["Re"]) < 1e-12
    # Eq. Reb: Re_B = Re delta_I/L = (delta_I/delta_M)^3
    assert rel(t["Re"] * t["dI_over_L"], t["Re_B"]) < 1e-12
    assert rel((t["dI_over_L"] / t["dM_over_L"]) ** 3, t["Re_B"]) < 1e-12
    # Eq. relation: delta_M/L = (nu/(beta L^3))^(1/3)  ->  nu
    assert rel(beta * L ** 3 * t["dM_over_L"] ** 3, t["nu"]) < 1e-3
    # Eq. relation: delta_I/L = (V/(beta L^2))^(1/2)  ->  V
    assert rel(beta * L ** 2 * t["dI_over_L"] ** 2, t["V"]) < 1e-3
    # time unit L/V in years (printed to 3 digits)
    assert rel(L / t["V"] / YEAR, t["L_over_V_yr"]) < 2e-3


@pytest.mark.parametrize("col", [0, 1])
def test_two_layer_table(col):
    t = {k: v[col] for k, v in read_table("table2_two_layer.txt").items()}
    L = t["L_km"] * 1e3
    H1, H2 = t["H1_km"] * 1e3, t["H2_km"] * 1e3
    H = H1 + H2
    beta, f0, gp = t["beta"], t["f0"], t["gprime"]
    # Sverdrup velocity of the two-layer model, V = 2 pi tau0/(rho1 H1 beta L)
    V = 2.0 * math.pi * t["tau0"] / (t["rho1"] * H1 * beta * L)
    assert rel(V, t["V"]) < 5e-3
    # Eq. ndim
    assert rel(V / (beta * L ** 2), t["Ro"]) < 5e-3
    assert rel(f0 ** 2 * V / (gp * beta * H), t["Fr"]) < 1e-2
    assert rel(t["nu"] / (beta * L ** 3), t["A"]) < 1e-3
    assert rel(t["gamma"] / (beta * L), t["sigma"]) < 2e-3
    assert rel(H1 / H, t["delta"]) < 1e-12
    # Re = Ro/A (the two-layer tables quote Re this way)
    assert rel(t["Ro"] / t["A"], t["Re"]) < 5e-3
    # Section 2.2 length scales
    assert rel((t["nu"] / beta) ** (1 / 3) / 1e3, t["dM_km"]) < 1e-3
    assert rel(t["gamma"] / beta / 1e3, t["dS_km"]) < 2e-3
    assert rel(math.sqrt(V / beta) / 1e3, t["dI_km"]) < 2e-3
    assert rel(L / V / YEAR, t["L_over_V_yr"]) < 5e-3
    # L/R_d as quoted in the text equals L divided by the tabulated R_d
    assert rel(L / (t["Rd_km"] * 1e3), t["L_over_Rd"]) < 1e-3


def test_deformation_radius_experiment_1():
    """R_d = sqrt(g' H1 H2/(f0^2 H)) (Section 2.2) reproduces Table 2's
    42.79 km and, through Eq. pv-non, the baroclinic coefficient of the
    coupled solve: Fr/(Ro delta (1-delta)) = (L/R_d)^2 = 46.74^2."""
    t = {k: v[0] for k, v in read_table("table2_two_layer.txt").items()}
    H1, H2 = t["H1_km"] * 1e3, t["H2_km"] * 1e3
    Rd = math.sqrt(t["gprime"] * H1 * H2 / (t["f0"] ** 2 * (H1 + H2)))
    assert rel(Rd / 1e3, t["Rd_km"]) < 1e-3
    coeff = t["Fr"] / (t["Ro"] * t["delta"] * (1.0 - t["delta"]))
    assert rel(coeff, t["L_over_Rd"] ** 2) < 2e-3


def test_deformation_radius_experiment_2_is_inconsistent_in_print():
    """Table 2's R_d for experiment 2 (31.16 km, L/R_d = 160.5) does not
    follow from its own H1, H2, g', f0 (34.16 km).  The library uses only the
    dimensionless Fr, Ro, delta, which agree with each other; this test
    records the misprint so that nobody 'fixes' the parameter layer to it."""
    t = {k: v[1] for k, v in read_table("table2_two_layer.txt").items()}
    H1, H2 = t["H1_km"] * 1e3, t["H2_km"] * 1e3
    Rd = math.sqrt(t["gprime"] * H1 * H2 / (t["f0"] ** 2 * (H1 + H2)))
    assert rel(Rd / 1e3, 34.16) < 1e-3
    coeff = t["Fr"] / (t["Ro"] * t["delta"] * (1.0 - t["delta"]))
    L = t["L_km"] * 1e3
    assert rel(math.sqrt(coeff), L / Rd) < 5e-3
