/*
 * Oracle transport driver -- TEST INFRASTRUCTURE (see oracle.h).
 *
 * Instantiates the generic step/event code of transport_body.h twice:
 *   strict FP32  (spec polynomials, FP32 tables: the bit-exact target),
 *   FP64 reference (libm, FP64 tables: the precision target),
 * and runs events on a pool of POSIX threads (events are independent: every
 * draw is keyed by event and track id).  All FP64 sums are Neumaier-compensated.
 * Must be compiled with -ffp-contract=off and without fast-math.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* Neumaier compensated sum. */
typedef struct { double s, c; } or_nsum;

static void or_nsum_add(or_nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}

typedef struct {
  uint64_t* counts;      /* [max_iters][3], private to the worker */
  uint64_t max_iters;
  oracle_totals tot;
  oracle_idrec* idlog;   /* private buffer */
  uint64_t idlog_n, idlog_cap;
  int idlog_on;
} or_worker;

static void or_worker_idlog(or_worker* wk, uint64_t id, uint32_t steps, uint32_t type_death) {
  if (!wk->idlog_on) return;
  if (wk->idlog_n == wk->idlog_cap) {
    uint64_t nc = wk->idlog_cap ? wk->idlog_cap * 2 : 4096;
    oracle_idrec* p = (oracle_idrec*)realloc(wk->idlog, nc * sizeof(oracle_idrec));
    if (!p) return;
    wk->idlog = p;
    wk->idlog_cap = nc;
  }
  oracle_idrec* r = &wk->idlog[wk->idlog_n++];
  r->id = id;
  r->steps = steps;
  r->type_death = type_death;
}

/* ---- strict FP32 instantiation ---- */
#define REAL float
#define SFX(name) f32_##name
#define RC(x) x##f
#define R_LOG oracle_spec_log
#define R_EXP oracle_spec_exp
#define R_SQRT sqrtf
#define R_FLOOR floorf
#define R_SINCOS2PI oracle_spec_sincos2pi
#define R_INF ((float)INFINITY)
#define R_SIG(w) ((w)->sig32)
#define R_LOGEMIN(w) ((w)->log_emin32)
#define R_INVDLOG(w) ((w)->inv_dlog32)
#define R_DEDX(w) ((w)->dedx32)
#define R_X0(w) ((w)->x0_32)
#include "transport_body.h"
#undef REAL
#undef SFX
#undef RC
#undef R_LOG
#undef R_EXP
#undef R_SQRT
#undef R_FLOOR
#undef R_SINCOS2PI
#undef R_INF
#undef R_SIG
#undef R_LOGEMIN
#undef R_INVDLOG
#undef R_DEDX
#undef R_X0

/* ---- FP64 reference instantiation ---- */
static void or_sincos2pi64(double u, double* s, double* c) {
  double a = 2.0 * 3.14159265358979323846 * u;
  *s = sin(a);
  *c = cos(a);
}
#define REAL double
#define SFX(name) f64_##name
#define RC(x) x
#define R_LOG log
#define R_EXP exp
#define R_SQRT sqrt
#define R_FLOOR floor
#define R_SINCOS2PI or_sincos2pi64
#define R_INF ((double)INFINITY)
#define R_SIG(w) ((w)->sig64)
#define R_LOGEMIN(w) ((w)->log_emin64)
#define R_INVDLOG(w) ((w)->inv_dlog64)
#define R_DEDX(w) ((w)->dedx64)
#define R_X0(w) ((w)->x0_64)
#include "transport_body.h"

/* ------------------------------------------------------------------ */

typedef struct {
  const oracle_world* w;
  const oracle_primary* prim;
  const size_t* order;      /* primaries sorted by event */
  const size_t* ev_begin;   /* [n_events + 1] */
  uint32_t n_events;
  int mode;
  double* score;
  double* ledger;
  f32_env e32;
  f64_env e64;
  pthread_mutex_t lock;
  uint32_t next_event;
  int err;
} or_job;

typedef struct {
  or_job* job;
  or_worker wk;
} or_thread;

static void* or_thread_main(void* arg) {
  or_thread* th = (or_thread*)arg;
  or_job* job = th->job;
  for (;;) {
    pthread_mutex_lock(&job->lock);
    uint32_t ev = job->next_event++;
    pthread_mutex_unlock(&job->lock);
    if (ev >= job->n_events) break;
    size_t b = job->ev_begin[ev], e = job->ev_begin[ev + 1];
    double* sc = job->score + (size_t)ev * (size_t)job->w->n_slabs;
    double* lg = job->ledger + (size_t)ev * 6;
    int err;
    if (job->mode == OR_STRICT_FP32)
      err = f32_run_event(&job->e32, job->prim, job->order + b, e - b, sc, lg, &th->wk);
    else
      err = f64_run_event(&job->e64, job->prim, job->order + b, e - b, sc, lg, &th->wk);
    if (err) {
      pthread_mutex_lock(&job->lock);
      job->err |= err;
      pthread_mutex_unlock(&job->lock);
    }
  }
  return NULL;
}

int oracle_run(const oracle_world* w, const oracle_primary* prim, size_t n_prim, uint32_t n_events,
               int mode, int nthreads, double* score, double* ledger, uint64_t* counts,
               uint64_t max_iters, oracle_idrec* idlog, uint64_t idlog_cap, oracle_totals* totals) {
  memset(totals, 0, sizeof *totals);
  or_job job;
  memset(&job, 0, sizeof job);
  if (f32_env_init(&job.e32, w) || f64_env_init(&job.e64, w)) {
    totals->errors = 4;
    return 4;
  }
  /* validate primaries */
  for (size_t i = 0; i < n_prim; ++i) {
    const oracle_primary* p = &prim[i];
    int bad = p->type > 2 || p->event >= n_events || !(p->ekin > 0.0f) || !isfinite(p->ekin);
    bad = bad || !(fabsf(p->pos[0]) <= w->half_xy) || !(fabsf(p->pos[1]) <= w->half_xy);
    bad = bad || f32_locate_slab(&job.e32, p->pos[2]) < 0;
    if (bad) {
      totals->errors = 4;
      return 4;
    }
  }
  /* group primaries by event, stable */
  size_t* ev_begin = (size_t*)calloc((size_t)n_events + 1, sizeof(size_t));
  size_t* order = (size_t*)malloc((n_prim ? n_prim : 1) * sizeof(size_t));
  size_t* fill = (size_t*)calloc((size_t)n_events + 1, sizeof(size_t));
  if (!ev_begin || !order || !fill) { free(ev_begin); free(order); free(fill); return 4; }
  for (size_t i = 0; i < n_prim; ++i) ev_begin[prim[i].event + 1] += 1;
  for (uint32_t e = 0; e < n_events; ++e) ev_begin[e + 1] += ev_begin[e];
  for (size_t i = 0; i < n_prim; ++i) {
    uint32_t e = prim[i].event;
    order[ev_begin[e] + fill[e]++] = i;
  }
  free(fill);

  job.w = w;
  job.prim = prim;
  job.order = order;
  job.ev_begin = ev_begin;
  job.n_events = n_events;
  job.mode = mode;
  job.score = score;
  job.ledger = ledger;
  pthread_mutex_init(&job.lock, NULL);
  if (nthreads < 1) nthreads = 1;
  or_thread* th = (or_thread*)calloc((size_t)nthreads, sizeof(or_thread));
  pthread_t* tid = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int k = 0; k < nthreads; ++k) {
    th[k].job = &job;
    th[k].wk.max_iters = max_iters;
    th[k].wk.counts = counts ? (uint64_t*)calloc((size_t)max_iters * 3, sizeof(uint64_t)) : NULL;
    th[k].wk.idlog_on = idlog != NULL;
  }
  if (nthreads == 1) {
    or_thread_main(&th[0]);
  } else {
    for (int k = 0; k < nthreads; ++k) pthread_create(&tid[k], NULL, or_thread_main, &th[k]);
    for (int k = 0; k < nthreads; ++k) pthread_join(tid[k], NULL);
  }
  /* merge */
  if (counts) memset(counts, 0, (size_t)max_iters * 3 * sizeof(uint64_t));
  uint64_t nid = 0;
  for (int k = 0; k < nthreads; ++k) {
    or_worker* wk = &th[k].wk;
    if (counts)
      for (uint64_t q = 0; q < max_iters * 3; ++q) counts[q] += wk->counts[q];
    for (int t = 0; t < 3; ++t) {
      totals->steps[t] += wk->tot.steps[t];
      totals->tracks[t] += wk->tot.tracks[t];
      totals->secondaries[t] += wk->tot.secondaries[t];
    }
    totals->reject_cap_hits += wk->tot.reject_cap_hits;
    if (wk->tot.n_iters > totals->n_iters) totals->n_iters = wk->tot.n_iters;
    for (uint64_t q = 0; q < wk->idlog_n; ++q) {
      if (idlog && nid < idlog_cap) idlog[nid] = wk->idlog[q];
      nid++;
    }
    free(wk->counts);
    free(wk->idlog);
  }
  totals->idlog_n = nid;
  if (idlog && nid > idlog_cap) job.err |= 2;
  totals->errors = (uint64_t)job.err;
  pthread_mutex_destroy(&job.lock);
  free(th);
  free(tid);
  free(order);
  free(ev_begin);
  return job.err;
}

static void or_in32(const oracle_track32* a, f32_trk* t) {
  t->x = a->x; t->y = a->y; t->z = a->z;
  t->dx = a->dx; t->dy = a->dy; t->dz = a->dz;
  t->e = a->e; t->nia = a->nia;
  t->id = a->id; t->event = a->event; t->step = a->step; t->slab = a->slab;
  t->time = a->time; t->len = a->len; t->flags = a->flags;
}

static void or_out32(const f32_trk* t, oracle_track32* a) {
  a->x = t->x; a->y = t->y; a->z = t->z;
  a->dx = t->dx; a->dy = t->dy; a->dz = t->dz;
  a->e = t->e; a->nia = t->nia;
  a->id = t->id; a->event = t->event; a->step = t->step; a->slab = t->slab;
  a->time = t->time; a->len = t->len; a->flags = t->flags;
}

int oracle_step_one(const oracle_world* w, int type, const oracle_track32* in,
                    oracle_step_result* out) {
  f32_env v;
  if (f32_env_init(&v, w) || type < 0 || type > 2 || in->slab < 0 || in->slab >= w->n_slabs)
    return 4;
  f32_trk t;
  or_in32(in, &t);
  f32_out o;
  f32_step(&v, type, &t, &o);
  memset(out, 0, sizeof *out);
  or_out32(&t, &out->track);
  out->alive = o.alive;
  out->death = o.death;
  out->lim = o.lim;
  out->proc = o.proc;
  out->nsec = o.nsec;
  for (int k = 0; k < o.nsec; ++k) {
    out->sec_type[k] = o.sec_type[k];
    or_out32(&o.sec[k], &out->sec[k]);
  }
  out->dep_cont = o.dep_cont;
  out->cut = o.cut;
  out->esc = o.esc;
  out->mc = o.mc;
  out->mcr = o.mcr;
  out->slab_cont = o.slab_cont;
  out->slab_cut = o.slab_cut;
  out->reject_cap_hit = o.reject_cap_hit;
  return 0;
}

float oracle_sample_compton_eps(float k, uint64_t seed, uint32_t event, uint64_t id, uint32_t step,
                                int* attempts) {
  float eps, onecost, sint2;
  int j = f32_compton_sample(seed, event, id, step, k, &eps, &onecost, &sint2);
  if (attempts) *attempts = j;
  return eps;
}

/* Array form of the Compton sampler: eps[i] for track ids[i]. */
void oracle_sample_compton_eps_n(float k, uint64_t seed, uint32_t event, const uint64_t* ids,
                                 uint32_t step, float* eps, int32_t* attempts, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    int a;
    eps[i] = oracle_sample_compton_eps(k, seed, event, ids[i], step, &a);
    if (attempts) attempts[i] = a;
  }
}
