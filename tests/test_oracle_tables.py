"""Pins of the oracle's cross-section tables against routes independent of its closed forms.

- Compton: numerical integration (scipy quad) of the Klein-Nishina *differential*
  cross section over solid angle, times the electron density.
- Thomson limit of the Klein-Nishina total cross section (CODATA sigma_T).
- Pair: zero at and below 2 mc^2, 7/(9 X0) at 1 GeV, linear in ln E.
- Photoelectric: Z^4/A scaling between materials and E^-3 scaling.
- Bremsstrahlung: node energies recovered by inverting the table; the table
  times the mean photon energy of the 1/k spectrum (numerical integral) gives
  the radiation-length loss (T - k_c)/X0.
- FP32 tables are the FP32 roundings of the FP64 ones.
"""
import numpy as np
import pytest
from scipy import integrate

import oracle

MC2 = 0.51099895
RE_CM = 2.8179403262e-13
SIGMA_THOMSON_CM2 = 6.6524587321e-25  # CODATA 2018
X0 = [5.612, 140.0]
Z = [82.0, 18.0]
A = [207.2, 39.948]
NODES = 1e-3 * 10.0 ** (8.0 * np.arange(257) / 256.0)


def kn_numeric(k):
    def dsig_dcos(c):
        eps = 1.0 / (1.0 + k * (1.0 - c))
        return 0.5 * RE_CM ** 2 * eps ** 2 * (eps + 1.0 / eps - (1.0 - c * c))
    val, _ = integrate.quad(dsig_dcos, -1.0, 1.0, epsabs=0, epsrel=1e-12, limit=200)
    return 2 * np.pi * val


@pytest.mark.parametrize("k", [1e-3, 0.02, 0.2, 1.0, 2.0, 20.0, 2000.0, 2e5])
def test_klein_nishina_total_matches_integrated_differential(k):
    assert oracle.kn_per_electron_cm2(k) == pytest.approx(kn_numeric(k), rel=1e-8)


def test_thomson_limit():
    assert oracle.kn_per_electron_cm2(1e-4) == pytest.approx(SIGMA_THOMSON_CM2, rel=3e-4)
    # first-order low-energy correction: sigma ~ sigma_T (1 - 2k)
    k = 1e-3
    assert oracle.kn_per_electron_cm2(k) == pytest.approx(SIGMA_THOMSON_CM2 * (1 - 2 * k), rel=1e-5)


def test_compton_table_equals_density_times_kn(otables):
    sig = otables["sig64"]
    for m in range(2):
        ne = oracle.electron_density_cm3(m)
        # electron density from Z, A, rho: lead 2.7e24/cm^3, argon 3.8e23/cm^3
        assert ne == pytest.approx([2.705e24, 3.788e23][m], rel=2e-3)
        for i in (0, 37, 128, 200, 256):
            expect = ne * kn_numeric(NODES[i] / MC2) / 10.0
            assert sig[m, oracle.TAB_COMPTON, i] == pytest.approx(expect, rel=1e-8)


def test_pair_table(otables):
    sig = otables["sig64"]
    for m in range(2):
        s = sig[m, oracle.TAB_PAIR]
        assert np.all(s[NODES <= 2 * MC2] == 0.0)
        assert oracle.sigma("pair", m, 1000.0) == pytest.approx(7.0 / (9.0 * X0[m]), rel=1e-14)
        e1, e2 = 5.0, 5000.0
        mid = np.sqrt(e1 * e2)
        assert oracle.sigma("pair", m, e1) + oracle.sigma("pair", m, e2) == pytest.approx(
            2 * oracle.sigma("pair", m, mid), rel=1e-12)


def test_photoelectric_scaling(otables):
    r = oracle.sigma("phot", 0, 0.3) / oracle.sigma("phot", 1, 0.3)
    rho = [11.35, 1.396]
    assert r == pytest.approx((rho[0] * Z[0] ** 4 / A[0]) / (rho[1] * Z[1] ** 4 / A[1]), rel=1e-12)
    assert oracle.sigma("phot", 0, 0.05) / oracle.sigma("phot", 0, 0.1) == pytest.approx(8.0, rel=1e-12)
    # lead mass attenuation at 100 keV ~ 2 cm^2/g by the model's choice of kappa
    assert oracle.sigma("phot", 0, 0.1) * 10.0 / rho[0] == pytest.approx(2.0, rel=0.01)


def test_brem_nodes_and_radiation_length(otables):
    sig = otables["sig64"]
    for m in range(2):
        s = sig[m, oracle.TAB_BREM]
        above = NODES > 0.01
        e_rec = 0.01 * np.exp(s[above] * X0[m])
        assert np.allclose(e_rec, NODES[above], rtol=1e-12)
        assert np.all(s[~above] == 0.0)
        for t in (0.5, 10.0, 1e4):
            mean_k = integrate.quad(lambda k: k * (1.0 / k), 0.01, t)[0] / integrate.quad(
                lambda k: 1.0 / k, 0.01, t)[0]
            assert oracle.sigma("brem", m, t) * mean_k == pytest.approx((t - 0.01) / X0[m], rel=1e-9)


def test_fp32_tables_are_rounded_fp64(otables):
    assert np.array_equal(otables["sig32"], otables["sig64"].astype(np.float32))
    assert np.array_equal(otables["dedx32"], otables["dedx64"].astype(np.float32))
    tot = otables["sig64"][:, oracle.TAB_COMPTON] + otables["sig64"][:, oracle.TAB_PAIR] + \
        otables["sig64"][:, oracle.TAB_PHOT]
    assert np.allclose(otables["sig64"][:, oracle.TAB_TOT], tot, rtol=1e-15, atol=0)
    assert otables["log_emin32"] == np.float32(np.log(1e-3))
    assert otables["inv_dlog32"] == np.float32(256.0 / np.log(1e8))
