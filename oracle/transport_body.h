/*
 * Oracle transport, generic over the real type -- TEST INFRASTRUCTURE.
 *
 * Included twice by transport.c: once as the strict FP32 model (spec
 * polynomials for log/exp/sincos, FP32 tables) and once as the FP64 reference
 * (libm, FP64 tables).  Macros supplied by the includer:
 *   REAL, SFX(name), RC(literal), R_LOG, R_EXP, R_SQRT, R_FLOOR, R_SINCOS2PI,
 *   R_INF, R_SIG (table pointer in the world), R_LOGEMIN, R_INVDLOG, R_DEDX, R_X0.
 *
 * One call of SFX(step) is one step of one track: Sec. 2 of the paper (each
 * active track is advanced once per transport iteration; survivors and
 * secondaries are active in the next one).  The physics is the toy model
 * standing in for the paper's G4HepEm (Sec. 1); the order of every operation
 * below is part of the model's definition, because strict mode must be
 * reproduced bit for bit.
 */

typedef struct {
  REAL x, y, z, dx, dy, dz, e, nia;
  uint64_t id;
  uint32_t event, step;
  int32_t slab;
  REAL time, len;
  uint32_t flags;
} SFX(trk);

typedef struct {
  int alive, death, lim, proc;
  int nsec;
  int sec_type[4];
  SFX(trk) sec[4];
  double dep_cont, cut, esc, mc, mcr;
  int slab_cont, slab_cut;
  int reject_cap_hit;
} SFX(out);

typedef struct {
  uint64_t seed;
  int n_slabs, n_nodes;
  REAL planes[129]; /* z of slab boundaries: FP64 running sum of thicknesses, rounded */
  int mat[128];
  REAL half;
  REAL log_emin, inv_dlog;
  const REAL* sig; /* [n_mat][5][n_nodes] */
  REAL dedx[4];
  int msc;         /* toy model v2: multiple scattering of e+- */
  REAL x0[4];      /* radiation lengths (mm), v2 only */
} SFX(env);

/* Toy model v2: the multiple-scattering step limit is OR_MSC_FR times the larger of the
 * range E / dEdx and OR_MSC_RMIN (mm). */
#define OR_MSC_FR RC(0.04)
#define OR_MSC_RMIN RC(0.5)

static int SFX(env_init)(SFX(env) * v, const oracle_world* w) {
  if (w->n_slabs < 1 || w->n_slabs > 128 || w->n_mat < 1 || w->n_mat > 4 || w->n_nodes < 2)
    return 1;
  v->seed = w->seed;
  v->n_slabs = w->n_slabs;
  v->n_nodes = w->n_nodes;
  double z = 0.0;
  v->planes[0] = (REAL)0;
  for (int s = 0; s < w->n_slabs; ++s) {
    z = z + w->thickness[s];
    v->planes[s + 1] = (REAL)z;
    v->mat[s] = (int)w->material[s];
    if (v->mat[s] >= w->n_mat) return 1;
  }
  v->half = (REAL)w->half_xy;
  v->log_emin = R_LOGEMIN(w);
  v->inv_dlog = R_INVDLOG(w);
  v->sig = R_SIG(w);
  for (int m = 0; m < w->n_mat; ++m) v->dedx[m] = R_DEDX(w)[m];
  v->msc = w->msc != 0;
  for (int m = 0; m < 4; ++m) v->x0[m] = RC(0.0);
  if (v->msc) {
    if (!R_X0(w)) return 1;
    for (int m = 0; m < w->n_mat; ++m) {
      v->x0[m] = R_X0(w)[m];
      if (!(v->x0[m] > RC(0.0))) return 1;
    }
  }
  return 0;
}

/* Four uniforms in (0, 1] from Philox block `block` of this track's current step. */
static void SFX(draws)(uint64_t seed, uint32_t event, uint64_t id, uint32_t step, uint32_t block,
                       REAL u[4]) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, block};
  uint32_t key[2] = {(uint32_t)seed, event};
  uint32_t r[4];
  oracle_philox4x32_10(ctr, key, r);
  for (int i = 0; i < 4; ++i) u[i] = (REAL)oracle_u01(r[i]);
}

/* Linear interpolation in table `tab` of material m at node i, fraction f. */
static REAL SFX(interp)(const SFX(env) * v, int m, int tab, int i, REAL f) {
  const REAL* t = v->sig + ((size_t)m * OR_NTAB + (size_t)tab) * (size_t)v->n_nodes;
  return t[i] + f * (t[i + 1] - t[i]);
}

/* Direction with polar cosine/sine (cost, sint) and azimuth (cphi, sphi) about unit u:
 * n = px e1 + py e2 + pz u with e1 = (ux uz, uy uz, -up)/up, e2 = (-uy, ux, 0)/up. */
static void SFX(rotate)(REAL ux, REAL uy, REAL uz, REAL px, REAL py, REAL pz, REAL n[3]) {
  REAL up = ux * ux + uy * uy;
  if (up > 0) {
    up = R_SQRT(up);
    n[0] = (ux * uz * px - uy * py) / up + ux * pz;
    n[1] = (uy * uz * px + ux * py) / up + uy * pz;
    n[2] = uz * pz - up * px;
  } else if (uz < 0) {
    n[0] = -px; n[1] = py; n[2] = -pz;
  } else {
    n[0] = px; n[1] = py; n[2] = pz;
  }
}

static void SFX(add_sec)(SFX(out) * o, const SFX(trk) * parent, uint32_t pstep, int type, REAL e,
                         REAL dx, REAL dy, REAL dz) {
  int k = o->nsec++;
  SFX(trk)* s = &o->sec[k];
  s->x = parent->x; s->y = parent->y; s->z = parent->z;
  s->dx = dx; s->dy = dy; s->dz = dz;
  s->e = e;
  s->nia = RC(-1.0);
  s->id = oracle_secondary_id(parent->id, pstep, (uint32_t)k);
  s->event = parent->event;
  s->step = 0;
  s->slab = parent->slab;
  s->time = parent->time;
  s->len = RC(0.0);
  s->flags = 0;
  o->sec_type[k] = type;
}

/* Positron at rest: two back-to-back photons of m_e c^2, isotropic (Philox block 65). */
static void SFX(annihilate)(const SFX(env) * v, const SFX(trk) * t, uint32_t pstep, SFX(out) * o) {
  REAL u[4];
  SFX(draws)(v->seed, t->event, t->id, pstep, 65u, u);
  REAL cost = RC(2.0) * u[0] - RC(1.0);
  REAL sint = R_SQRT((RC(1.0) - cost) * (RC(1.0) + cost));
  REAL sp, cp;
  R_SINCOS2PI(u[1], &sp, &cp);
  REAL dx = sint * cp, dy = sint * sp, dz = cost;
  SFX(add_sec)(o, t, pstep, OR_GAMMA, RC(0.51099895), dx, dy, dz);
  SFX(add_sec)(o, t, pstep, OR_GAMMA, RC(0.51099895), -dx, -dy, -dz);
  o->mcr = (double)RC(0.51099895) + (double)RC(0.51099895);
}

/* Toy model v2, multiple scattering: the direction of a charged track that goes on after
 * a step of length s > 0 in material m is turned by a polar angle theta and an azimuth
 * phi (Philox block 66 of the step).  The width is the Highland formula of the pre-step
 * energy E, theta0 = 13.6 MeV / (beta c p) sqrt(x) (1 + 0.038 ln x), x = s / X0 (no
 * deflection when the bracket is not positive); beta c p = E (E + 2 mc^2) / (E + mc^2).
 * In the small-angle Gaussian approximation theta^2 / 2 is exponential with mean
 * theta0^2, so 1 - cos(theta) = theta0^2 (-ln u0), cos(theta) clamped at -1; phi = 2 pi u1.
 * The turn uses the same rotation as the Compton scattering. */
static void SFX(msc_deflect)(const SFX(env) * v, SFX(trk) * t, uint32_t pstep, REAL E, REAL s,
                             int m) {
  REAL pbc = E * (E + RC(1.0219979)) / (E + RC(0.51099895));
  REAL x = s / v->x0[m];
  REAL br = RC(1.0) + RC(0.038) * R_LOG(x);
  if (!(br > RC(0.0))) return;
  REAL th0 = (RC(13.6) / pbc) * R_SQRT(x) * br;
  REAL u[4];
  SFX(draws)(v->seed, t->event, t->id, pstep, 66u, u);
  REAL w = (th0 * th0) * (-R_LOG(u[0]));
  REAL cost = RC(1.0) - w;
  if (cost < RC(-1.0)) cost = RC(-1.0);
  REAL sint = R_SQRT((RC(1.0) - cost) * (RC(1.0) + cost));
  REAL sp, cp;
  R_SINCOS2PI(u[1], &sp, &cp);
  REAL n[3];
  SFX(rotate)(t->dx, t->dy, t->dz, sint * cp, sint * sp, cost, n);
  t->dx = n[0]; t->dy = n[1]; t->dz = n[2];
}

/* Butcher-Messel Klein-Nishina sampling of eps = E'/E at k = E/mc^2; attempt j uses
 * Philox block 1 + j; at most 64 attempts, after which the last candidate is kept. */
static int SFX(compton_sample)(uint64_t seed, uint32_t event, uint64_t id, uint32_t step, REAL k,
                               REAL* eps_o, REAL* onecost_o, REAL* sint2_o) {
  REAL eps0 = RC(1.0) / (RC(1.0) + RC(2.0) * k);
  REAL eps0sq = eps0 * eps0;
  REAL a1 = -R_LOG(eps0);
  REAL a2 = RC(0.5) * (RC(1.0) - eps0sq);
  REAL p1 = a1 / (a1 + a2);
  REAL eps = RC(1.0), epssq, onecost = RC(0.0), sint2 = RC(0.0);
  int j;
  for (j = 0; j < 64; ++j) {
    REAL w[4];
    SFX(draws)(seed, event, id, step, 1u + (uint32_t)j, w);
    if (p1 > w[0]) {
      eps = R_EXP(-(a1 * w[1]));
      epssq = eps * eps;
    } else {
      epssq = eps0sq + (RC(1.0) - eps0sq) * w[1];
      eps = R_SQRT(epssq);
    }
    onecost = (RC(1.0) - eps) / (k * eps);
    sint2 = onecost * (RC(2.0) - onecost);
    REAL g = RC(1.0) - (eps * sint2) / (RC(1.0) + epssq);
    if (g >= w[2]) break;
  }
  *eps_o = eps;
  *onecost_o = onecost;
  *sint2_o = sint2;
  return j; /* 64 means the cap was hit */
}

static void SFX(step)(const SFX(env) * v, int type, SFX(trk) * t, SFX(out) * o) {
  memset(o, 0, sizeof *o);
  o->alive = 1;
  const int charged = (type != OR_GAMMA);
  const uint32_t pstep = t->step;
  REAL u[4];
  SFX(draws)(v->seed, t->event, t->id, pstep, 0u, u);
  const REAL E = t->e;

  /* 1. number of interaction lengths left (-1 is the resample sentinel) */
  if (t->nia < 0) t->nia = -R_LOG(u[0]);

  /* 2-3. cross section at the pre-step energy and physics step */
  const int s0 = t->slab;
  const int m = v->mat[s0];
  REAL lx = (R_LOG(E) - v->log_emin) * v->inv_dlog;
  int i = (int)R_FLOOR(lx);
  if (i < 0) i = 0;
  if (i > v->n_nodes - 2) i = v->n_nodes - 2;
  REAL f = lx - (REAL)i;
  REAL sig = charged ? SFX(interp)(v, m, OR_TAB_BREM, i, f) : SFX(interp)(v, m, OR_TAB_TOT, i, f);
  REAL s_phys = (sig > 0) ? t->nia / sig : R_INF;

  /* 4. geometric distances: slab planes along z, box faces along x and y */
  REAL zpl = RC(0.0), sz, sx, sy;
  if (t->dz > 0) { zpl = v->planes[s0 + 1]; sz = (zpl - t->z) / t->dz; }
  else if (t->dz < 0) { zpl = v->planes[s0]; sz = (zpl - t->z) / t->dz; }
  else sz = R_INF;
  if (sz < 0) sz = RC(0.0);
  if (t->dx > 0) sx = (v->half - t->x) / t->dx;
  else if (t->dx < 0) sx = (-v->half - t->x) / t->dx;
  else sx = R_INF;
  if (sx < 0) sx = RC(0.0);
  if (t->dy > 0) sy = (v->half - t->y) / t->dy;
  else if (t->dy < 0) sy = (-v->half - t->y) / t->dy;
  else sy = R_INF;
  if (sy < 0) sy = RC(0.0);

  /* 5-6. step limit, fixed order, strict '<' (earlier limiter wins ties) */
  REAL s = sz;
  int lim = OR_LIM_Z;
  if (sx < s) { s = sx; lim = OR_LIM_X; }
  if (sy < s) { s = sy; lim = OR_LIM_Y; }
  if (charged) {
    REAL dedx = v->dedx[m];
    REAL sl = (E > RC(1.0)) ? (RC(0.2) * E) / dedx : E / dedx;
    if (sl < s) { s = sl; lim = OR_LIM_LOSS; }
    if (v->msc) {
      /* v2: multiple-scattering step limit, a fraction of the range E/dEdx (at least of
       * the minimum range) */
      REAL rng = E / dedx;
      REAL sm = OR_MSC_FR * ((rng > OR_MSC_RMIN) ? rng : OR_MSC_RMIN);
      if (sm < s) { s = sm; lim = OR_LIM_MSC; }
    }
  }
  if (s_phys < s) { s = s_phys; lim = OR_LIM_PHYS; }

  /* 7. move */
  t->x = t->x + s * t->dx;
  t->y = t->y + s * t->dy;
  t->z = (lim == OR_LIM_Z) ? zpl : (t->z + s * t->dz);
  if (charged) {
    REAL beta = R_SQRT(E * (E + RC(1.0219979))) / (E + RC(0.51099895));
    t->time = t->time + s / (beta * RC(299.792458));
  } else {
    t->time = t->time + s / RC(299.792458);
  }
  t->len = t->len + s;

  /* 8. interaction lengths */
  if (lim == OR_LIM_PHYS) {
    t->nia = RC(-1.0);
  } else {
    t->nia = t->nia - s * sig;
    if (t->nia < 0) t->nia = RC(0.0);
  }

  /* 9. continuous loss (charged), deposited in the pre-step slab */
  REAL eout = E;
  if (charged) {
    REAL de = (lim == OR_LIM_LOSS && E <= RC(1.0)) ? E : v->dedx[m] * s;
    eout = E - de;
    if (eout < 0) eout = RC(0.0);
  }
  t->e = eout;
  o->slab_cont = s0;

  /* 10. boundary */
  int escaped = 0;
  if (lim == OR_LIM_Z) {
    int s1 = (t->dz > 0) ? s0 + 1 : s0 - 1;
    if (s1 < 0 || s1 >= v->n_slabs) escaped = 1;
    else t->slab = s1;
  } else if (lim == OR_LIM_X || lim == OR_LIM_Y) {
    escaped = 1;
  }
  o->lim = lim;
  o->proc = OR_PROC_NONE;

  /* 11. deaths and interactions */
  if (escaped) {
    o->esc = (double)eout;
    o->alive = 0;
    o->death = OR_DEATH_ESCAPE;
  } else if (charged && eout < RC(0.01)) {
    o->cut = o->cut + (double)eout;
    o->alive = 0;
    o->death = OR_DEATH_CUT;
    if (type == OR_EP) SFX(annihilate)(v, t, pstep, o);
  } else {
    /* v2: the surviving charged track is deflected before any interaction */
    if (charged && v->msc && s > RC(0.0)) SFX(msc_deflect)(v, t, pstep, E, s, m);
    if (lim == OR_LIM_PHYS) {
      if (!charged) {
        REAL sc = SFX(interp)(v, m, OR_TAB_COMPTON, i, f);
        REAL sp = SFX(interp)(v, m, OR_TAB_PAIR, i, f);
        REAL r = u[1] * sig;
        if (r < sc) {
          /* Compton */
          o->proc = OR_PROC_COMPTON;
          REAL k = E / RC(0.51099895);
          REAL eps, onecost, sint2;
          int j = SFX(compton_sample)(v->seed, t->event, t->id, pstep, k, &eps, &onecost, &sint2);
          if (j >= 64) o->reject_cap_hit = 1;
          if (sint2 < 0) sint2 = RC(0.0);
          REAL cost = RC(1.0) - onecost;
          REAL sint = R_SQRT(sint2);
          REAL sphi, cphi;
          R_SINCOS2PI(u[3], &sphi, &cphi);
          REAL n[3];
          SFX(rotate)(t->dx, t->dy, t->dz, sint * cphi, sint * sphi, cost, n);
          REAL e1 = eps * E;
          REAL te = E - e1;
          if (te >= RC(0.01)) {
            REAL px = E * t->dx - e1 * n[0];
            REAL py = E * t->dy - e1 * n[1];
            REAL pz = E * t->dz - e1 * n[2];
            REAL pn = R_SQRT(px * px + py * py + pz * pz);
            SFX(add_sec)(o, t, pstep, OR_EM, te, px / pn, py / pn, pz / pn);
          } else {
            o->cut = o->cut + (double)te;
          }
          t->dx = n[0]; t->dy = n[1]; t->dz = n[2];
          t->e = e1;
          if (!(e1 >= RC(0.01))) {
            o->cut = o->cut + (double)e1;
            o->alive = 0;
            o->death = OR_DEATH_CUT;
          }
        } else if (r < sc + sp && E > RC(1.0219979)) {
          /* pair: both leptons along the photon direction */
          o->proc = OR_PROC_PAIR;
          REAL avail = E - RC(1.0219979);
          REAL em = u[2] * avail;
          REAL ep = avail - em;
          o->mc = ((double)E - (double)em) - (double)ep;
          if (em >= RC(0.01)) SFX(add_sec)(o, t, pstep, OR_EM, em, t->dx, t->dy, t->dz);
          else o->cut = o->cut + (double)em;
          if (ep >= RC(0.01)) {
            SFX(add_sec)(o, t, pstep, OR_EP, ep, t->dx, t->dy, t->dz);
          } else {
            o->cut = o->cut + (double)ep;
            SFX(annihilate)(v, t, pstep, o);
          }
          o->alive = 0;
          o->death = OR_DEATH_ABSORB;
        } else {
          /* photoelectric: electron with the full energy along the photon direction */
          o->proc = OR_PROC_PHOT;
          if (E >= RC(0.01)) SFX(add_sec)(o, t, pstep, OR_EM, E, t->dx, t->dy, t->dz);
          else o->cut = o->cut + (double)E;
          o->alive = 0;
          o->death = OR_DEATH_ABSORB;
        }
      } else {
        /* bremsstrahlung, 1/k spectrum on [k_c, T] */
        o->proc = OR_PROC_BREM;
        if (eout > RC(0.01)) {
          REAL kk = RC(0.01) * R_EXP(u[2] * R_LOG(eout / RC(0.01)));
          if (kk < RC(0.01)) kk = RC(0.01);
          if (kk > eout) kk = eout;
          SFX(add_sec)(o, t, pstep, OR_GAMMA, kk, t->dx, t->dy, t->dz);
          REAL t2 = eout - kk;
          t->e = t2;
          if (t2 < RC(0.01)) {
            o->cut = o->cut + (double)t2;
            o->alive = 0;
            o->death = OR_DEATH_CUT;
            if (type == OR_EP) SFX(annihilate)(v, t, pstep, o);
          }
        }
      }
    }
  }
  o->slab_cut = t->slab;

  /* 12. FP64 energy balance of the step, in this fixed order */
  double dep = (double)E;
  dep = dep + o->mcr;
  if (o->alive) dep = dep - (double)t->e;
  for (int k = 0; k < o->nsec; ++k) dep = dep - (double)o->sec[k].e;
  dep = dep - o->esc;
  dep = dep - o->cut;
  dep = dep - o->mc;
  o->dep_cont = dep;

  t->flags = (uint32_t)lim | ((uint32_t)o->proc << 4);
  t->step = pstep + 1;
}

/* ------------------------------------------------------------------ */
/* Per-event depth-first driver                                        */

typedef struct {
  SFX(trk) t;
  int type;
  uint64_t birth;
} SFX(item);

static int SFX(locate_slab)(const SFX(env) * v, REAL z) {
  if (!(z >= v->planes[0]) || !(z < v->planes[v->n_slabs])) return -1;
  int s = 0;
  while (s + 1 < v->n_slabs && !(z < v->planes[s + 1])) ++s;
  return s;
}

/* Runs the primaries of one event; returns 0 or an error bit mask. */
static int SFX(run_event)(const SFX(env) * v, const oracle_primary* prim, const size_t* idx,
                          size_t n, double* score, double* ledger, or_worker* wk) {
  int err = 0;
  size_t cap = 1024, top = 0;
  SFX(item)* stack = (SFX(item)*)malloc(cap * sizeof(SFX(item)));
  if (!stack) return 4;
  or_nsum* sc = (or_nsum*)calloc((size_t)v->n_slabs, sizeof(or_nsum));
  or_nsum lg[6];
  memset(lg, 0, sizeof lg);
  for (size_t q = 0; q < n; ++q) {
    const oracle_primary* p = &prim[idx[n - 1 - q]]; /* pushed in reverse: first primary first */
    SFX(item) it;
    memset(&it, 0, sizeof it);
    it.t.x = (REAL)p->pos[0]; it.t.y = (REAL)p->pos[1]; it.t.z = (REAL)p->pos[2];
    it.t.dx = (REAL)p->dir[0]; it.t.dy = (REAL)p->dir[1]; it.t.dz = (REAL)p->dir[2];
    it.t.e = (REAL)p->ekin;
    it.t.nia = RC(-1.0);
    it.t.id = p->id;
    it.t.event = p->event;
    it.t.step = 0;
    it.t.slab = SFX(locate_slab)(v, it.t.z);
    it.t.time = RC(0.0);
    it.t.len = RC(0.0);
    it.type = (int)p->type;
    it.birth = 0;
    stack[top++] = it;
    or_nsum_add(&lg[0], (double)it.t.e);
    wk->tot.tracks[it.type] += 1;
  }
  while (top > 0) {
    SFX(item) it = stack[--top];
    for (;;) {
      uint64_t iter = it.birth + it.t.step;
      if (iter < wk->max_iters) {
        if (wk->counts) wk->counts[iter * 3 + (uint64_t)it.type] += 1;
      } else {
        err |= 1;
      }
      if (iter + 1 > wk->tot.n_iters) wk->tot.n_iters = iter + 1;
      wk->tot.steps[it.type] += 1;
      SFX(out) o;
      SFX(step)(v, it.type, &it.t, &o);
      or_nsum_add(&sc[o.slab_cont], o.dep_cont);
      if (o.cut != 0.0) or_nsum_add(&sc[o.slab_cut], o.cut);
      or_nsum_add(&lg[1], o.dep_cont);
      or_nsum_add(&lg[2], o.cut);
      or_nsum_add(&lg[3], o.esc);
      or_nsum_add(&lg[4], o.mcr);
      or_nsum_add(&lg[5], o.mc);
      if (o.reject_cap_hit) wk->tot.reject_cap_hits += 1;
      for (int k = 0; k < o.nsec; ++k) {
        if (top == cap) {
          cap *= 2;
          SFX(item)* ns = (SFX(item)*)realloc(stack, cap * sizeof(SFX(item)));
          if (!ns) { free(stack); free(sc); return err | 4; }
          stack = ns;
        }
        SFX(item) child;
        child.t = o.sec[k];
        child.type = o.sec_type[k];
        child.birth = iter + 1;
        stack[top++] = child;
        wk->tot.secondaries[child.type] += 1;
        wk->tot.tracks[child.type] += 1;
      }
      if (!o.alive) {
        or_worker_idlog(wk, it.t.id, it.t.step, (uint32_t)it.type | ((uint32_t)o.death << 8));
        break;
      }
    }
  }
  for (int s = 0; s < v->n_slabs; ++s) score[s] = sc[s].s + sc[s].c;
  for (int k = 0; k < 6; ++k) ledger[k] = lg[k].s + lg[k].c;
  free(stack);
  free(sc);
  return err;
}
