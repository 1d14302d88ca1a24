"""Physical constants and electrolyte conversions, atomic units (oracle side).

Test infrastructure only (see the package docstring).

The ionic charge of Eq. (rhoions) is e N_A sum_i Z_i c_i with c_i in mol per
volume; in atomic units (e = 1, lengths in bohr) the number density of species
i is n_i = c_i[mol/L] * 1000 * N_A * a0^3 (bohr^-3) and kT = k_B T (Hartree).
The linear PB coefficient of Eq. (corrPB), 4 pi e^2 N_A / kT sum Z_i^2 c_i,
becomes lambda0 = 4 pi sum_i Z_i^2 n_i / kT.  The steric maximum of Eq.
(maxconc), c_max = p / ((4/3) pi R^3 N_A), is the number density
n_max = p / ((4/3) pi R^3) with R in bohr.
"""
import math

N_AVOGADRO = 6.02214076e23          # 1/mol (exact, SI 2019)
BOHR_M = 5.29177210903e-11          # m (CODATA 2018)
K_BOLTZMANN_HA = 3.1668115634556e-6  # Hartree/K (CODATA 2018)
EXP_CAP = 40.0                      # cap on the Boltzmann exponent (reading A15)
ANGSTROM_BOHR = 1e-10 / BOHR_M      # bohr per angstrom


def number_density(c_molar):
    """mol/L -> particles per bohr^3."""
    return c_molar * 1000.0 * N_AVOGADRO * BOHR_M ** 3


def kT(temperature):
    return K_BOLTZMANN_HA * temperature


def lambda0(electrolyte):
    """4 pi sum_i Z_i^2 n_i / kT (Eq. corrPB in atomic units)."""
    kt = kT(electrolyte.temperature)
    return 4.0 * math.pi * sum(z * z * number_density(c)
                               for z, c in zip(electrolyte.z, electrolyte.c_molar)) / kt


def max_number_density(radius_angstrom, packing):
    """Eq. (maxconc) as a number density: p / ((4/3) pi R^3), bohr^-3."""
    r = radius_angstrom * ANGSTROM_BOHR
    return packing / (4.0 / 3.0 * math.pi * r ** 3)
