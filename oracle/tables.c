/*
 * Oracle cross-section closed forms and table build -- TEST INFRASTRUCTURE.
 *
 * The paper's physics is G4HepEm (Sec. 1); the toy model replaces it with the
 * closed forms below, evaluated in FP64 at the table nodes and rounded to FP32
 * (the FP32 tables are what strict mode interpolates; the FP64 values serve
 * the FP64 reference mode).  Materials: 0 = lead, 1 = liquid argon, with the
 * PDG values for Z, A, density, radiation length and a fixed stopping power.
 *
 *  Compton:  Sigma_C = n_e sigma_KN(k), k = E / m_e c^2, sigma_KN the
 *            Klein-Nishina total cross section per electron.
 *  Pair:     Sigma_pair = 7/(9 X0) ln(E / 2mc^2) / ln(1000 MeV / 2mc^2), E > 2mc^2.
 *  Photo:    Sigma_pe = rho kappa Z^4/A (0.1 MeV / E)^3, kappa = 9.2e-6 cm^2/g.
 *  Total:    FP32 rounding of the FP64 sum of the three.
 *  Brems:    Sigma_brem = ln(T / k_c) / X0, T > k_c = 0.01 MeV (1/k spectrum whose
 *            mean radiative loss per unit length is (T - k_c)/X0).
 */
#include <math.h>

#include "oracle.h"

#define OR_MC2 0.51099895            /* MeV, CODATA 2018 */
#define OR_RE_CM 2.8179403262e-13    /* classical electron radius, cm */
#define OR_NA 6.02214076e23          /* 1/mol */
#define OR_KC 0.01                   /* MeV, production and tracking cut */
#define OR_PI 3.14159265358979323846
#define OR_KAPPA_PE 9.2e-6           /* cm^2/g */

typedef struct { double Z, A, rho, X0_mm, dedx; } or_material;

static const or_material OR_MATS[2] = {
    {82.0, 207.2, 11.35, 5.612, 1.274},    /* Pb */
    {18.0, 39.948, 1.396, 140.0, 0.2105},  /* liquid Ar */
};

double oracle_electron_density_cm3(int mat) {
  const or_material* m = &OR_MATS[mat];
  return m->rho * OR_NA * m->Z / m->A;
}

/* Klein-Nishina total cross section per electron (cm^2), textbook closed form. */
double oracle_kn_per_electron_cm2(double k) {
  double a = 1.0 + 2.0 * k;
  double l = log(a);
  double term1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
  double term2 = l / (2.0 * k);
  double term3 = (1.0 + 3.0 * k) / (a * a);
  return 2.0 * OR_PI * OR_RE_CM * OR_RE_CM * (term1 + term2 - term3);
}

double oracle_sigma_compton(int mat, double e) {
  double k = e / OR_MC2;
  return oracle_electron_density_cm3(mat) * oracle_kn_per_electron_cm2(k) / 10.0;
}

double oracle_sigma_pair(int mat, double e) {
  double thr = 2.0 * OR_MC2;
  if (!(e > thr)) return 0.0;
  return 7.0 / (9.0 * OR_MATS[mat].X0_mm) * log(e / thr) / log(1000.0 / thr);
}

double oracle_sigma_phot(int mat, double e) {
  const or_material* m = &OR_MATS[mat];
  double z4 = m->Z * m->Z * m->Z * m->Z;
  double q = 0.1 / e;
  return m->rho * OR_KAPPA_PE * z4 / m->A * (q * q * q) / 10.0;
}

double oracle_sigma_brem(int mat, double t) {
  if (!(t > OR_KC)) return 0.0;
  return log(t / OR_KC) / OR_MATS[mat].X0_mm;
}

double oracle_dedx(int mat) { return OR_MATS[mat].dedx; }

double oracle_x0(int mat) { return OR_MATS[mat].X0_mm; }

int oracle_build_tables(int n_mat, int n_nodes, float* sig32, double* sig64, float* dedx32,
                        double* dedx64, float* log_emin32, float* inv_dlog32, double* log_emin64,
                        double* inv_dlog64) {
  if (n_mat < 1 || n_mat > 2 || n_nodes < 2) return 1;
  const double span = log(1e8); /* ln(100 GeV / 1 keV) */
  for (int m = 0; m < n_mat; ++m) {
    for (int i = 0; i < n_nodes; ++i) {
      double e = 1e-3 * pow(10.0, 8.0 * (double)i / (double)(n_nodes - 1));
      double c = oracle_sigma_compton(m, e);
      double p = oracle_sigma_pair(m, e);
      double ph = oracle_sigma_phot(m, e);
      double vals[OR_NTAB] = {c, p, ph, c + p + ph, oracle_sigma_brem(m, e)};
      for (int t = 0; t < OR_NTAB; ++t) {
        size_t at = ((size_t)m * OR_NTAB + (size_t)t) * (size_t)n_nodes + (size_t)i;
        if (sig64) sig64[at] = vals[t];
        if (sig32) sig32[at] = (float)vals[t];
      }
    }
    if (dedx64) dedx64[m] = OR_MATS[m].dedx;
    if (dedx32) dedx32[m] = (float)OR_MATS[m].dedx;
  }
  if (log_emin64) *log_emin64 = log(1e-3);
  if (inv_dlog64) *inv_dlog64 = (double)(n_nodes - 1) / span;
  if (log_emin32) *log_emin32 = (float)log(1e-3);
  if (inv_dlog32) *inv_dlog32 = (float)((double)(n_nodes - 1) / span);
  return 0;
}
