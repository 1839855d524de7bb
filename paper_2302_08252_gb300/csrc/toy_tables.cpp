// Host-side builder of the toy EM model's cross-section tables (the stand-in
// for the G4HepEm tables the paper's AdePT runs with, Sec. 1 and Sec. 4).
// Closed forms in FP64 at 257 nodes E_i = 1e-3 * 10^(8 i / 256) MeV, rounded
// to FP32:
//   Compton   n_e * Klein-Nishina total cross section per electron
//   pair      7/(9 X0) ln(E / 2mc^2) / ln(1000 MeV / 2mc^2) above 2mc^2
//   photo     rho kappa Z^4/A (0.1 MeV / E)^3, kappa = 9.2e-6 cm^2/g
//   total     FP32 of the FP64 sum of the three
//   brems     ln(T / k_c) / X0 above k_c = 0.01 MeV
// Materials: 0 lead, 1 liquid argon (PDG Z, A, density, radiation length;
// fixed stopping powers 1.274 and 0.2105 MeV/mm).
// Built with -ffp-contract=off so that every FP64 operation rounds once.
#include <cmath>
#include <cstdint>

#include "et.h"

namespace {

struct Medium {
  double Z, A, density, x0_mm, stopping;
};

constexpr Medium kMedia[2] = {
    {82.0, 207.2, 11.35, 5.612, 1.274},
    {18.0, 39.948, 1.396, 140.0, 0.2105},
};
constexpr double kElectronMass = 0.51099895;      // MeV
constexpr double kElectronRadius = 2.8179403262e-13;  // cm
constexpr double kAvogadro = 6.02214076e23;
constexpr double kCut = 0.01;                      // MeV
constexpr double kPi = 3.14159265358979323846;
constexpr double kPhotoKappa = 9.2e-6;             // cm^2/g

double klein_nishina(double k) {
  const double a = 1.0 + 2.0 * k;
  const double l = std::log(a);
  const double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
  const double t2 = l / (2.0 * k);
  const double t3 = (1.0 + 3.0 * k) / (a * a);
  return 2.0 * kPi * kElectronRadius * kElectronRadius * (t1 + t2 - t3);
}

double compton(const Medium& m, double e) {
  const double n_e = m.density * kAvogadro * m.Z / m.A;
  return n_e * klein_nishina(e / kElectronMass) / 10.0;
}

double pair(const Medium& m, double e) {
  const double thr = 2.0 * kElectronMass;
  if (!(e > thr)) return 0.0;
  return 7.0 / (9.0 * m.x0_mm) * std::log(e / thr) / std::log(1000.0 / thr);
}

double photo(const Medium& m, double e) {
  const double z4 = m.Z * m.Z * m.Z * m.Z;
  const double q = 0.1 / e;
  return m.density * kPhotoKappa * z4 / m.A * (q * q * q) / 10.0;
}

double brems(const Medium& m, double t) {
  if (!(t > kCut)) return 0.0;
  return std::log(t / kCut) / m.x0_mm;
}

}  // namespace

extern "C" et_status et_build_toy_tables_fp64(uint32_t n_materials, uint32_t n_nodes,
                                              double* sigma_out, double* dedx_out,
                                              double* log_emin_out, double* inv_dlog_out) {
  if (n_materials < 1 || n_materials > 2 || n_nodes < 2 || !sigma_out || !dedx_out)
    return ET_ERR_INVALID;
  for (uint32_t m = 0; m < n_materials; ++m) {
    const Medium& md = kMedia[m];
    double* row = sigma_out + (size_t)m * 5 * n_nodes;
    for (uint32_t i = 0; i < n_nodes; ++i) {
      const double e = 1e-3 * std::pow(10.0, 8.0 * (double)i / (double)(n_nodes - 1));
      const double c = compton(md, e), p = pair(md, e), f = photo(md, e);
      row[0 * n_nodes + i] = c;
      row[1 * n_nodes + i] = p;
      row[2 * n_nodes + i] = f;
      row[3 * n_nodes + i] = c + p + f;
      row[4 * n_nodes + i] = brems(md, e);
    }
    dedx_out[m] = md.stopping;
  }
  if (log_emin_out) *log_emin_out = std::log(1e-3);
  if (inv_dlog_out) *inv_dlog_out = (double)(n_nodes - 1) / std::log(1e8);
  return ET_OK;
}

extern "C" et_status et_build_toy_tables(uint32_t n_materials, uint32_t n_nodes, float* sigma_out,
                                         float* dedx_out, float* log_emin_out, float* inv_dlog_out) {
  if (n_materials < 1 || n_materials > 2 || n_nodes < 2 || !sigma_out || !dedx_out)
    return ET_ERR_INVALID;
  for (uint32_t m = 0; m < n_materials; ++m) {
    const Medium& md = kMedia[m];
    float* row = sigma_out + (size_t)m * 5 * n_nodes;
    for (uint32_t i = 0; i < n_nodes; ++i) {
      const double e = 1e-3 * std::pow(10.0, 8.0 * (double)i / (double)(n_nodes - 1));
      const double c = compton(md, e), p = pair(md, e), f = photo(md, e);
      row[0 * n_nodes + i] = (float)c;
      row[1 * n_nodes + i] = (float)p;
      row[2 * n_nodes + i] = (float)f;
      row[3 * n_nodes + i] = (float)(c + p + f);
      row[4 * n_nodes + i] = (float)brems(md, e);
    }
    dedx_out[m] = (float)md.stopping;
  }
  if (log_emin_out) *log_emin_out = (float)std::log(1e-3);
  if (inv_dlog_out) *inv_dlog_out = (float)((double)(n_nodes - 1) / std::log(1e8));
  return ET_OK;
}

extern "C" et_status et_toy_radiation_lengths(uint32_t n_materials, float* x0_out) {
  if (n_materials < 1 || n_materials > 2 || !x0_out) return ET_ERR_INVALID;
  for (uint32_t m = 0; m < n_materials; ++m) x0_out[m] = (float)kMedia[m].x0_mm;
  return ET_OK;
}
