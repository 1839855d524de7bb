// One step of one track of the toy EM model on the GPU (the per-track work
// inside the paper's transport kernels, Sec. 2 and Sec. 4).  Strict mode
// evaluates the model's fixed operation sequence in FP32 with the spec
// polynomials (its translation units are built with --fmad=false, IEEE
// division and square root), so results are bit-identical to the model's
// definition; fast mode swaps in hardware intrinsics and allows FMA.
//
// The step is split in two so that the kernels can compact the lanes that
// need a discrete interaction (see kernels.cuh):
//   transport(): Philox block 0 of (seed, event | id, step), interaction
//     lengths, cross section from the shared-memory tables, distances to the
//     slab planes and box faces, the step limiter in fixed order, move,
//     continuous loss, boundary crossing, deaths (escape; e+- below the cut,
//     positrons annihilating at rest).  It finishes the step unless a discrete
//     interaction is due, in which case it returns the interaction context.
//   interact(): photon Compton (Butcher-Messel rejection), pair or
//     photoelectric; e+- bremsstrahlung with a 1/k spectrum; the step's FP64
//     energy balance.
// Composed, the two are exactly the model's single step.
#pragma once

#include "common.cuh"

namespace et {

constexpr float MC2 = 0x1.05a1a8p-1f;       // 0.51099895 MeV
constexpr float TWO_MC2 = 0x1.05a1a8p+0f;   // 1.0219979 MeV
constexpr float KC = 0x1.47ae14p-7f;        // 0.01 MeV, production and tracking cut
constexpr float C_LIGHT = 0x1.2bcadep+8f;   // 299.792458 mm/ns
constexpr float LOSS_FRAC = 0x1.99999ap-3f; // 0.2
// toy model v2 (multiple scattering): step limit MSC_FR max(E / dEdx, MSC_RMIN), Highland
// width 13.6 MeV / (beta c p) sqrt(x) (1 + 0.038 ln x)
constexpr float MSC_FR = 0x1.47ae14p-5f;    // 0.04
constexpr float MSC_RMIN = 0.5f;            // mm
constexpr float HIGHLAND_E = 0x1.b33334p+3f; // 13.6 MeV
constexpr float HIGHLAND_LOG = 0x1.374bc6p-5f; // 0.038
constexpr float F_INF = __builtin_huge_valf();

// Shared-memory copy of geometry and tables (block-local).
struct Tabs {
  const float* planes;   // [n_slabs + 1]
  const uint8_t* mat;    // [n_slabs]
  const float2* tot;     // [n_mat][256] {Sigma_tot, next - this}
  const float4* cp;      // [n_mat][256] {Sigma_C, dC, Sigma_pair, dP}
  const float2* brem;    // [n_mat][256]
  const float* dedx;     // [n_mat]
  const float* x0;       // [n_mat] radiation lengths (toy model v2)
  int n_slabs;
  int msc;               // toy model v2: multiple scattering of e+-
};

// A secondary's id is derived when it is written: secondary_id(parent, step, ordinal).
struct Sec {
  float e, dx, dy, dz;
};

// Terms of the step's energy balance other than the survivor and the secondaries.
enum : uint32_t { B_CUT = 1u, B_ESC = 2u, B_MC = 4u, B_MCR = 8u };

// At most 3 secondaries per step (brems photon + 2 annihilation photons; e- + 2
// annihilation photons from a pair whose positron is below the cut).  They sit in
// three named slots, never an indexed array, so that they stay in registers; their
// types are packed 2 bits each.
struct StepOut {
  int alive, death, nsec, reject, slab_cont;
  uint32_t dirty, types, bal;
  bool dep_nz;      // dep != 0
  Sec s0, s1, s2;
  double dep;       // FP64 balance: deposited in the pre-step slab
  double cut;       // below-cut energy, deposited in the end slab (B_CUT)
  double mc;        // rest mass consumed by pair production (B_MC)
  float esc;        // escaped energy (B_ESC)
  // k must be a compile-time constant after unrolling
  __device__ __forceinline__ const Sec& sec(int k) const { return k == 0 ? s0 : (k == 1 ? s1 : s2); }
  __device__ __forceinline__ int type(int k) const { return (int)((types >> (2 * k)) & 3u); }
  __device__ __forceinline__ void add_cut(float x) {
    cut = (bal & B_CUT) ? cut + f2d(x) : f2d(x);  // 0 + x == x: same as summing from 0
    bal |= B_CUT;
  }
  __device__ __forceinline__ void begin() {
    alive = 1;
    death = ALIVE;
    nsec = 0;
    reject = 0;
    types = 0;
    bal = 0;
    dep_nz = false;
  }
};

// What transport() hands to interact() when a discrete interaction is due.
struct Ctx {
  float E;              // pre-step energy
  float sig, sc, sp;    // photon: total, Compton, pair cross sections at E; e+-: brems
  float u1, u2, u3;     // Philox block 0, words 1..3
};

template <int MODE>
__device__ __forceinline__ float m_log(float x) {
  if constexpr (MODE == MODE_STRICT) return s_log(x);
  else return __logf(x);
}
template <int MODE>
__device__ __forceinline__ float m_exp(float x) {
  if constexpr (MODE == MODE_STRICT) return s_exp(x);
  else return __expf(x);
}
template <int MODE>
__device__ __forceinline__ void m_sincos2pi(float u, float* s, float* c) {
  if constexpr (MODE == MODE_STRICT) s_sincos2pi(u, s, c);
  else __sincosf(6.28318530717958648f * u, s, c);
}

__device__ __forceinline__ void add_sec(StepOut& o, int type, float e, float dx, float dy,
                                        float dz) {
  const int k = o.nsec;
  Sec s;
  s.e = e;
  s.dx = dx;
  s.dy = dy;
  s.dz = dz;
  if (k == 0) o.s0 = s;
  else if (k == 1) o.s1 = s;
  else o.s2 = s;
  o.types |= (uint32_t)type << (2 * k);
  o.nsec = k + 1;
}

// direction at polar (cost, sint) and azimuth (cphi, sphi) about unit u
__device__ __forceinline__ void rotate_about(float ux, float uy, float uz, float px, float py,
                                             float pz, float& nx, float& ny, float& nz) {
  float up = ux * ux + uy * uy;
  if (up > 0.0f) {
    up = sqrtf(up);
    nx = (ux * uz * px - uy * py) / up + ux * pz;
    ny = (uy * uz * px + ux * py) / up + uy * pz;
    nz = uz * pz - up * px;
  } else if (uz < 0.0f) {
    nx = -px; ny = py; nz = -pz;
  } else {
    nx = px; ny = py; nz = pz;
  }
}

// Toy model v2: the direction of a charged track that goes on after a step of length
// s > 0 is turned by theta, phi (Philox block 66 of the step).  Highland's width at the
// pre-step energy E and x = s / X0; 1 - cos(theta) = theta0^2 (-log u0) (small-angle
// Gaussian law), clamped at cos(theta) = -1; phi = 2 pi u1; the Compton rotation.
template <int MODE>
__device__ __forceinline__ void msc_deflect(Trk& t, uint32_t pstep, uint32_t seed, float E,
                                            float s, float x0) {
  const float pbc = E * (E + TWO_MC2) / (E + MC2);  // beta c p
  const float x = s / x0;
  const float br = 1.0f + HIGHLAND_LOG * m_log<MODE>(x);
  if (!(br > 0.0f)) return;
  const float th0 = (HIGHLAND_E / pbc) * sqrtf(x) * br;
  const uint4 r = philox((uint32_t)t.id, (uint32_t)(t.id >> 32), pstep, 66u, seed, t.event);
  const float w = (th0 * th0) * (-m_log<MODE>(u01(r.x)));
  float cost = 1.0f - w;
  if (cost < -1.0f) cost = -1.0f;
  const float sint = sqrtf((1.0f - cost) * (1.0f + cost));
  float sphi, cphi;
  m_sincos2pi<MODE>(u01(r.y), &sphi, &cphi);
  float nx, ny, nz;
  rotate_about(t.dx, t.dy, t.dz, sint * cphi, sint * sphi, cost, nx, ny, nz);
  t.dx = nx;
  t.dy = ny;
  t.dz = nz;
}

// Positron at rest: two back-to-back photons of m_e c^2, isotropic (Philox block 65).
template <int MODE>
__device__ __forceinline__ void annihilate(StepOut& o, const Trk& t, uint32_t pstep,
                                           uint32_t seed) {
  const uint4 r = philox((uint32_t)t.id, (uint32_t)(t.id >> 32), pstep, 65u, seed, t.event);
  const float cost = 2.0f * u01(r.x) - 1.0f;
  const float sint = sqrtf((1.0f - cost) * (1.0f + cost));
  float sp, cp;
  m_sincos2pi<MODE>(u01(r.y), &sp, &cp);
  const float dx = sint * cp, dy = sint * sp, dz = cost;
  add_sec(o, GAM, MC2, dx, dy, dz);
  add_sec(o, GAM, MC2, -dx, -dy, -dz);
  o.bal |= B_MCR;
}

// FP64 energy balance of the step, fixed order:
//   dep = E + mcr - E_survivor - sum E_secondaries - esc - cut - mc
__device__ __forceinline__ void balance(const Trk& t, float E, StepOut& o) {
  if (o.bal == 0 && o.nsec == 0 && o.alive) {
    // only continuous loss: the balance is E - E'.  Subtracting the zero terms leaves it
    // unchanged, and E - E' is exact in FP32 when E' >= E/2 (Sterbenz), so no FP64
    // arithmetic is needed on this, the common, path.
    const float e1 = t.e;
    o.dep_nz = e1 != E;
    if (!o.dep_nz) o.dep = 0.0;                            // E - E = +0
    else if (e1 >= 0.5f * E) o.dep = f2d(E - e1);          // exact difference
    else o.dep = f2d(E) - f2d(e1);
  } else {
    double dep = f2d(E);
    if (o.bal & B_MCR) dep = dep + (f2d(MC2) + f2d(MC2));
    if (o.alive) dep = dep - f2d(t.e);
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (k < o.nsec) dep = dep - f2d(o.sec(k).e);
    if (o.bal & B_ESC) dep = dep - f2d(o.esc);
    if (o.bal & B_CUT) dep = dep - o.cut;
    if (o.bal & B_MC) dep = dep - o.mc;
    o.dep = dep;
    o.dep_nz = dep != 0.0;
  }
}

// Whether the distance num / den (den > 0) can be below the running minimum s.  False
// only when num >= 2 s den with 2 s den a normal number: the exact quotient is then at
// least 2 s (1 - 2^-24) > s, so its rounded value is >= s and the comparison it would
// enter (quotient < s) is false.  Skipping that division leaves the step unchanged.
__device__ __forceinline__ bool may_limit(float num, float den, float s) {
  const float bound = 2.0f * s * den;
  return !(num >= bound && bound >= 0x1p-100f);
}

// Returns true when a discrete interaction is due: the step is then unfinished
// (step counter and flags unchanged) and cx holds what interact() needs.
// `type` is warp-uniform; a compile-time constant at the per-type kernels' call sites.
template <int MODE>
__device__ __forceinline__ bool transport(const int type, Trk& t, const Tabs& tb, float log_emin,
                                          float inv_dlog, float half, uint32_t seed, StepOut& o,
                                          Ctx& cx) {
  const bool charged = type != GAM;
  o.begin();
  o.dirty = D_POS | D_NIA | D_STEP | D_TIME | D_LEN | D_FLAGS;
  const uint32_t pstep = t.step;
  const uint4 r0 = philox((uint32_t)t.id, (uint32_t)(t.id >> 32), pstep, 0u, seed, t.event);
  const float E = t.e;

  // interaction lengths left
  if (t.nia < 0.0f) t.nia = -m_log<MODE>(u01(r0.x));

  // cross section at the pre-step energy
  const int s0 = t.slab;
  const int m = tb.mat[s0];
  const float lx = (m_log<MODE>(E) - log_emin) * inv_dlog;  // |lx| < 2^22 for any finite E > 0
  int bin;
  float fbin = floor_small(lx, bin);
  if (bin < 0) { bin = 0; fbin = 0.0f; }
  if (bin > NBINS - 1) { bin = NBINS - 1; fbin = (float)(NBINS - 1); }
  const float f = lx - fbin;
  float sig;
  if (charged) {
    const float2 b = tb.brem[m * NBINS + bin];
    sig = b.x + f * b.y;
  } else {
    const float2 b = tb.tot[m * NBINS + bin];
    sig = b.x + f * b.y;
  }
  // geometry: slab planes along z, box faces along x and y
  float zpl = 0.0f, sz;
  if (t.dz > 0.0f) { zpl = tb.planes[s0 + 1]; sz = (zpl - t.z) / t.dz; }
  else if (t.dz < 0.0f) { zpl = tb.planes[s0]; sz = (zpl - t.z) / t.dz; }
  else sz = F_INF;
  if (sz < 0.0f) sz = 0.0f;

  // step limiter: fixed order, earlier wins ties.  A limiter whose distance (a quotient)
  // cannot be below the running minimum skips its division (may_limit); the comparisons,
  // and so the step, are those of computing every distance.
  float s = sz;
  int lim = LIM_Z;
  if (t.dx != 0.0f) {
    const float num = (t.dx > 0.0f) ? (half - t.x) : (-half - t.x);
    if (may_limit(t.dx > 0.0f ? num : -num, fabsf(t.dx), s)) {
      float sx = num / t.dx;
      if (sx < 0.0f) sx = 0.0f;
      if (sx < s) { s = sx; lim = LIM_X; }
    }
  }
  if (t.dy != 0.0f) {
    const float num = (t.dy > 0.0f) ? (half - t.y) : (-half - t.y);
    if (may_limit(t.dy > 0.0f ? num : -num, fabsf(t.dy), s)) {
      float sy = num / t.dy;
      if (sy < 0.0f) sy = 0.0f;
      if (sy < s) { s = sy; lim = LIM_Y; }
    }
  }
  float dedx = 0.0f;
  if (charged) {
    dedx = tb.dedx[m];
    const float num = (E > 1.0f) ? LOSS_FRAC * E : E;
    if (may_limit(num, dedx, s)) {
      const float sl = num / dedx;
      if (sl < s) { s = sl; lim = LIM_LOSS; }
    }
    if (tb.msc) {  // v2: multiple-scattering step limit
      const float rng = E / dedx;
      const float sm = MSC_FR * ((rng > MSC_RMIN) ? rng : MSC_RMIN);
      if (sm < s) { s = sm; lim = LIM_MSC; }
    }
  }
  if (sig > 0.0f && may_limit(t.nia, sig, s)) {
    const float s_phys = t.nia / sig;
    if (s_phys < s) { s = s_phys; lim = LIM_PHYS; }
  }

  // move
  t.x = t.x + s * t.dx;
  t.y = t.y + s * t.dy;
  t.z = (lim == LIM_Z) ? zpl : (t.z + s * t.dz);
  if (charged) {
    const float beta = sqrtf(E * (E + TWO_MC2)) / (E + MC2);
    t.time = t.time + s / (beta * C_LIGHT);
  } else {
    t.time = t.time + s / C_LIGHT;
  }
  t.len = t.len + s;
  if (lim == LIM_PHYS) {
    t.nia = -1.0f;
  } else {
    t.nia = t.nia - s * sig;
    if (t.nia < 0.0f) t.nia = 0.0f;
  }

  // continuous loss, deposited in the pre-step slab
  float eout = E;
  if (charged) {
    const float de = (lim == LIM_LOSS && E <= 1.0f) ? E : dedx * s;
    eout = E - de;
    if (eout < 0.0f) eout = 0.0f;
    o.dirty |= D_E;
  }
  t.e = eout;
  o.slab_cont = s0;

  // boundary
  bool escaped = false;
  if (lim == LIM_Z) {
    const int s1 = (t.dz > 0.0f) ? s0 + 1 : s0 - 1;
    if (s1 < 0 || s1 >= tb.n_slabs) {
      escaped = true;
    } else {
      t.slab = s1;
      o.dirty |= D_SLAB;
    }
  } else if (lim == LIM_X || lim == LIM_Y) {
    escaped = true;
  }

  if (escaped) {
    o.esc = eout;
    o.bal |= B_ESC;
    o.alive = 0;
    o.death = DEATH_ESCAPE;
  } else if (charged && eout < KC) {
    o.add_cut(eout);
    o.alive = 0;
    o.death = DEATH_CUT;
    if (type == EP) annihilate<MODE>(o, t, pstep, seed);
  } else {
    // v2: the surviving charged track is deflected before any interaction
    if (charged && tb.msc && s > 0.0f) {
      msc_deflect<MODE>(t, pstep, seed, E, s, tb.x0[m]);
      o.dirty |= D_DIR;
    }
    if (lim == LIM_PHYS) {
    cx.E = E;
    cx.sig = sig;
    if (!charged) {
      const float4 cp = tb.cp[m * NBINS + bin];
      cx.sc = cp.x + f * cp.y;
      cx.sp = cp.z + f * cp.w;
    }
    cx.u1 = u01(r0.y);
    cx.u2 = u01(r0.z);
    cx.u3 = u01(r0.w);
    return true;
    }
  }
  balance(t, E, o);
  t.flags = (uint32_t)lim;
  t.step = pstep + 1;
  return false;
}

// The discrete interaction that ends a PHYS-limited step, then the step's balance.
// t is the post-transport state (its step counter not yet advanced); o is fresh.  `msc`:
// toy model v2, where the transport half has turned a charged track's direction.
template <int MODE>
__device__ __forceinline__ void interact(const int type, Trk& t, const Ctx& cx, uint32_t seed,
                                         StepOut& o, bool msc) {
  const bool charged = type != GAM;
  o.begin();
  o.dirty = D_POS | D_NIA | D_STEP | D_TIME | D_LEN | D_FLAGS | (charged ? D_E : 0u) |
            (charged && msc ? D_DIR : 0u);
  o.slab_cont = t.slab;
  const uint32_t pstep = t.step;
  const float E = cx.E;
  int proc;
  if (!charged) {
    const float r = cx.u1 * cx.sig;
    if (r < cx.sc) {
      // Compton (Butcher-Messel), attempt j on Philox block 1 + j, at most 64
      proc = PROC_COMPTON;
      const uint32_t idlo = (uint32_t)t.id, idhi = (uint32_t)(t.id >> 32);
      const float k = E / MC2;
      const float eps0 = 1.0f / (1.0f + 2.0f * k);
      const float eps0sq = eps0 * eps0;
      const float a1 = -m_log<MODE>(eps0);
      const float a2 = 0.5f * (1.0f - eps0sq);
      const float p1 = a1 / (a1 + a2);
      float eps = 1.0f, epssq = 1.0f, onecost = 0.0f, sint2 = 0.0f;
      int j;
      for (j = 0; j < 64; ++j) {
        const uint4 rj = philox(idlo, idhi, pstep, 1u + (uint32_t)j, seed, t.event);
        const float ua = u01(rj.x), ub = u01(rj.y), uc = u01(rj.z);
        if (p1 > ua) {
          eps = m_exp<MODE>(-(a1 * ub));
          epssq = eps * eps;
        } else {
          epssq = eps0sq + (1.0f - eps0sq) * ub;
          eps = sqrtf(epssq);
        }
        onecost = (1.0f - eps) / (k * eps);
        sint2 = onecost * (2.0f - onecost);
        const float g = 1.0f - (eps * sint2) / (1.0f + epssq);
        if (g >= uc) break;
      }
      if (j >= 64) o.reject = 1;
      if (sint2 < 0.0f) sint2 = 0.0f;
      const float cost = 1.0f - onecost;
      const float sint = sqrtf(sint2);
      float sphi, cphi;
      m_sincos2pi<MODE>(cx.u3, &sphi, &cphi);
      float nx, ny, nz;
      rotate_about(t.dx, t.dy, t.dz, sint * cphi, sint * sphi, cost, nx, ny, nz);
      const float e1 = eps * E;
      const float te = E - e1;
      if (te >= KC) {
        const float px = E * t.dx - e1 * nx;
        const float py = E * t.dy - e1 * ny;
        const float pz = E * t.dz - e1 * nz;
        const float pn = sqrtf(px * px + py * py + pz * pz);
        add_sec(o, EM, te, px / pn, py / pn, pz / pn);
      } else {
        o.add_cut(te);
      }
      t.dx = nx;
      t.dy = ny;
      t.dz = nz;
      t.e = e1;
      o.dirty |= D_DIR | D_E;
      if (!(e1 >= KC)) {
        o.add_cut(e1);
        o.alive = 0;
        o.death = DEATH_CUT;
      }
    } else if (r < cx.sc + cx.sp && E > TWO_MC2) {
      proc = PROC_PAIR;
      const float avail = E - TWO_MC2;
      const float em = cx.u2 * avail;
      const float ep = avail - em;
      o.mc = (f2d(E) - f2d(em)) - f2d(ep);
      o.bal |= B_MC;
      if (em >= KC) add_sec(o, EM, em, t.dx, t.dy, t.dz);
      else o.add_cut(em);
      if (ep >= KC) {
        add_sec(o, EP, ep, t.dx, t.dy, t.dz);
      } else {
        o.add_cut(ep);
        annihilate<MODE>(o, t, pstep, seed);
      }
      o.alive = 0;
      o.death = DEATH_ABSORB;
    } else {
      proc = PROC_PHOT;
      if (E >= KC) add_sec(o, EM, E, t.dx, t.dy, t.dz);
      else o.add_cut(E);
      o.alive = 0;
      o.death = DEATH_ABSORB;
    }
  } else {
    // bremsstrahlung, 1/k spectrum on [k_c, T'] at the post-loss energy
    proc = PROC_BREM;
    const float eout = t.e;
    if (eout > KC) {
      float kk = KC * m_exp<MODE>(cx.u2 * m_log<MODE>(eout / KC));
      if (kk < KC) kk = KC;
      if (kk > eout) kk = eout;
      add_sec(o, GAM, kk, t.dx, t.dy, t.dz);
      const float t2 = eout - kk;
      t.e = t2;
      if (t2 < KC) {
        o.add_cut(t2);
        o.alive = 0;
        o.death = DEATH_CUT;
        if (type == EP) annihilate<MODE>(o, t, pstep, seed);
      }
    }
  }
  balance(t, E, o);
  t.flags = (uint32_t)LIM_PHYS | ((uint32_t)proc << 4);
  t.step = pstep + 1;
}

// Both halves in sequence: exactly one step of the model.
template <int MODE>
__device__ __forceinline__ void step_track(const int type, Trk& t, const Tabs& tb, float log_emin,
                                           float inv_dlog, float half, uint32_t seed, StepOut& o) {
  Ctx cx;
  if (transport<MODE>(type, t, tb, log_emin, inv_dlog, half, seed, o, cx))
    interact<MODE>(type, t, cx, seed, o, tb.msc != 0);
}

}  // namespace et
