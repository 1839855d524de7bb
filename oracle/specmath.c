/*
 * Oracle strict-mode elementary functions -- TEST INFRASTRUCTURE (see oracle.h).
 *
 * The toy model fixes log, exp and sincos(2 pi u) as explicit FP32 polynomial
 * evaluations so that a CPU and a GPU evaluate them bit-identically (no FMA,
 * every operation IEEE round-to-nearest).  Each is written from the textbook
 * method named below, not from any library's implementation:
 *
 *  log:   x = m 2^e with m in (sqrt(1/2), sqrt(2)]; log m = 2 atanh r,
 *         r = (m-1)/(m+1), atanh series to r^9; e ln2 split into hi + lo
 *         (Cody & Waite, "Software Manual for the Elementary Functions", 1980).
 *  exp:   n = rint(x / ln2), r = (x - n ln2_hi) - n ln2_lo (Cody-Waite),
 *         Taylor series of e^r to degree 7 (Horner), scaled by 2^n via the
 *         exponent bits.
 *  sincos2pi: quadrant reduction of 4u to q + y with |y| <= 1/2, a = y pi/2,
 *         Taylor series of sin to a^9 and cos to a^8, quadrant rotation.
 *
 * Coefficients are the FP32 roundings of the exact series coefficients.
 * This file must be compiled with -ffp-contract=off and without fast-math.
 */
#include <math.h>
#include <string.h>

#include "oracle.h"

static uint32_t f2u(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float u2f(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/* ln 2 = LN2_HI + LN2_LO; LN2_HI has 15 significant bits, so e * LN2_HI is exact. */
static const float LN2_HI = 0.693145751953125f;       /* 0x3f317200 */
static const float LN2_LO = 1.42860682030941723e-06f; /* ln2 - LN2_HI */
static const float SQRT2 = 1.41421356237309505f;
static const float INV_LN2 = 1.44269504088896341f;
static const float HALF_PI = 1.57079632679489662f;

float oracle_spec_log(float x) {
  /* Defined for positive normal finite x (the model only takes logs of such). */
  uint32_t b = f2u(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = u2f((b & 0x007fffffu) | 0x3f800000u); /* [1, 2) */
  if (m > SQRT2) {
    m = m * 0.5f;
    e = e + 1;
  }
  float r = (m - 1.0f) / (m + 1.0f);
  float r2 = r * r;
  /* atanh(r)/r - 1 = r^2/3 + r^4/5 + r^6/7 + r^8/9 */
  float s = 1.0f / 9.0f;
  s = s * r2 + 1.0f / 7.0f;
  s = s * r2 + 1.0f / 5.0f;
  s = s * r2 + 1.0f / 3.0f;
  s = s * r2;
  float t = r + r * s; /* atanh(r) */
  float logm = t + t;
  float fe = (float)e;
  return fe * LN2_HI + (logm + fe * LN2_LO);
}

float oracle_spec_exp(float x) {
  if (x > 88.0f) return u2f(0x7f800000u);
  if (x < -87.0f) return 0.0f;
  float n = rintf(x * INV_LN2);
  float r = x - n * LN2_HI;
  r = r - n * LN2_LO;
  /* e^r = sum r^j / j!, j = 0..7 */
  float p = 1.0f / 5040.0f;
  p = p * r + 1.0f / 720.0f;
  p = p * r + 1.0f / 120.0f;
  p = p * r + 1.0f / 24.0f;
  p = p * r + 1.0f / 6.0f;
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  int ni = (int)n;
  float scale = u2f((uint32_t)(ni + 127) << 23);
  return p * scale;
}

void oracle_spec_sincos2pi(float u, float* s_out, float* c_out) {
  float v = 4.0f * u;
  float q = rintf(v);
  float y = v - q; /* exact: |y| <= 1/2 */
  float a = y * HALF_PI;
  float a2 = a * a;
  /* sin a = a (1 - a^2/3! + a^4/5! - a^6/7! + a^8/9!) */
  float ps = 1.0f / 362880.0f;
  ps = ps * a2 - 1.0f / 5040.0f;
  ps = ps * a2 + 1.0f / 120.0f;
  ps = ps * a2 - 1.0f / 6.0f;
  ps = ps * a2 + 1.0f;
  float sa = a * ps;
  /* cos a = 1 - a^2/2! + a^4/4! - a^6/6! + a^8/8! */
  float pc = 1.0f / 40320.0f;
  pc = pc * a2 - 1.0f / 720.0f;
  pc = pc * a2 + 1.0f / 24.0f;
  pc = pc * a2 - 0.5f;
  pc = pc * a2 + 1.0f;
  float ca = pc;
  int k = ((int)q) & 3;
  /* 2 pi u = k pi/2 + a */
  if (k == 0) { *s_out = sa; *c_out = ca; }
  else if (k == 1) { *s_out = ca; *c_out = -sa; }
  else if (k == 2) { *s_out = -sa; *c_out = -ca; }
  else { *s_out = -ca; *c_out = sa; }
}

/* Array forms for the pins (one call per array instead of one per element). */
void oracle_spec_log_n(const float* x, float* y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = oracle_spec_log(x[i]);
}

void oracle_spec_exp_n(const float* x, float* y, size_t n) {
  for (size_t i = 0; i < n; ++i) y[i] = oracle_spec_exp(x[i]);
}

void oracle_spec_sincos2pi_n(const float* u, float* s, float* c, size_t n) {
  for (size_t i = 0; i < n; ++i) oracle_spec_sincos2pi(u[i], &s[i], &c[i]);
}
