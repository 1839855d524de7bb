/*
 * CPU oracle for the toy electromagnetic shower transport -- TEST INFRASTRUCTURE.
 *
 * This is the plain, slow, obviously-correct definition of what one transport
 * iteration computes (Sec. 2 of the paper: the list of active tracks per
 * particle type, stepped once per iteration; Sec. 4: a 10 GeV electron gun
 * into 50 absorber/gap layers, energy deposit per layer).  The paper runs
 * AdePT's full physics; this oracle defines the fixed toy EM model that stands
 * in for it (the constants, operation order and draw assignment are listed in
 * the design notes under "Toy model").
 *
 * Only the test-suite, the smoke entry point and the CPU-baseline leg of the
 * benchmark may load this library.  It shares no code, header, helper or table
 * generator with the CUDA product path; the two meet only through the seeded
 * input generators (primaries, geometry thicknesses).
 *
 * Histories are depth-first per event: a track is stepped until it dies and
 * its secondaries are pushed on a stack.  Because every random draw is keyed
 * by (seed, event, track id, track-local step), the histories are the same as
 * the breadth-first, one-step-per-iteration histories of the GPU path, and the
 * per-iteration counts are reconstructed from each track's birth iteration.
 *
 * Parity pins (tests/test_oracle_*.py): Philox known-answer vectors, spec-math
 * error against libm, tables against numerically integrated cross sections,
 * Klein-Nishina chi-square, bremsstrahlung KS, exponential attenuation,
 * range closed form, single-interaction kinematics, energy ledger closure, and
 * for the toy model v2 (multiple scattering) the step limit's closed form and
 * the deflection against Highland's width.
 */
#ifndef ET_ORACLE_H
#define ET_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_EM = 0, OR_EP = 1, OR_GAMMA = 2, OR_NTYPES = 3 };
enum { OR_TAB_COMPTON = 0, OR_TAB_PAIR = 1, OR_TAB_PHOT = 2, OR_TAB_TOT = 3, OR_TAB_BREM = 4,
       OR_NTAB = 5 };
enum { OR_LIM_Z = 0, OR_LIM_X = 1, OR_LIM_Y = 2, OR_LIM_LOSS = 3, OR_LIM_PHYS = 4, OR_LIM_MSC = 5 };
enum { OR_PROC_NONE = 0, OR_PROC_COMPTON = 1, OR_PROC_PAIR = 2, OR_PROC_PHOT = 3,
       OR_PROC_BREM = 4 };
enum { OR_ALIVE = 0, OR_DEATH_ESCAPE = 1, OR_DEATH_CUT = 2, OR_DEATH_ABSORB = 3 };
enum { OR_STRICT_FP32 = 0, OR_REF_FP64 = 1 };

/* A primary as handed over by the input generator (48 bytes). */
typedef struct {
  uint32_t type;   /* 0 e-, 1 e+, 2 gamma */
  uint32_t event;  /* event index, < n_events */
  uint64_t id;     /* (event << 32) | index within the event */
  float pos[3];    /* mm */
  float dir[3];    /* unit vector */
  float ekin;      /* MeV (photon: energy) */
  uint32_t pad;
} oracle_primary;

/* One entry per track at its death (16 bytes). */
typedef struct {
  uint64_t id;
  uint32_t steps;       /* steps the track took */
  uint32_t type_death;  /* type | death << 8 */
} oracle_idrec;

/* Public state of one track, FP32 (64 bytes), used by the single-step entry. */
typedef struct {
  float x, y, z, dx, dy, dz, e, nia;
  uint64_t id;
  uint32_t event, step;
  int32_t slab;
  float time, len;
  uint32_t flags;
} oracle_track32;

/* Result of one step of one track (single-step entry, FP32 strict). */
typedef struct {
  oracle_track32 track;      /* post-step state */
  int32_t alive, death, lim, proc;
  int32_t nsec;
  int32_t sec_type[4];
  oracle_track32 sec[4];
  double dep_cont;           /* deposit into slab_cont */
  double cut;                /* below-cut deposit into slab_cut */
  double esc, mc, mcr;
  int32_t slab_cont, slab_cut;
  int32_t reject_cap_hit;
  int32_t pad;
} oracle_step_result;

/* ---- building blocks (exported for the pins) ---- */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
float oracle_u01(uint32_t x);
uint64_t oracle_mix64(uint64_t z);
uint64_t oracle_secondary_id(uint64_t parent, uint32_t step, uint32_t ordinal);
float oracle_spec_log(float x);
float oracle_spec_exp(float x);
void oracle_spec_sincos2pi(float u, float* s, float* c);
void oracle_spec_log_n(const float* x, float* y, size_t n);
void oracle_spec_exp_n(const float* x, float* y, size_t n);
void oracle_spec_sincos2pi_n(const float* u, float* s, float* c, size_t n);
void oracle_philox_n(const uint32_t* ctr, const uint32_t key[2], uint32_t* out, size_t n);

/* Closed-form cross sections in FP64 (1/mm), per material index (0 Pb, 1 lAr). */
double oracle_sigma_compton(int mat, double e_mev);
double oracle_sigma_pair(int mat, double e_mev);
double oracle_sigma_phot(int mat, double e_mev);
double oracle_sigma_brem(int mat, double t_mev);
double oracle_dedx(int mat);
double oracle_x0(int mat);   /* radiation length, mm */
double oracle_kn_per_electron_cm2(double k);
double oracle_electron_density_cm3(int mat);

/* Table build: node i = 0..n_nodes-1 at E_i = 1e-3 * 10^(8 i / (n_nodes-1)) MeV.
 * sig32/sig64: [n_mat][5][n_nodes]; dedx32/dedx64: [n_mat]. Returns 0. */
int oracle_build_tables(int n_mat, int n_nodes, float* sig32, double* sig64, float* dedx32,
                        double* dedx64, float* log_emin32, float* inv_dlog32, double* log_emin64,
                        double* inv_dlog64);

/* The world every step reads. */
typedef struct {
  int32_t n_slabs;           /* <= 128 */
  int32_t n_mat;             /* <= 4 */
  int32_t n_nodes;           /* table nodes (257) */
  int32_t pad0;
  const double* thickness;   /* [n_slabs] mm, front face at z = 0 */
  const uint8_t* material;   /* [n_slabs] */
  float half_xy;             /* mm */
  float log_emin32, inv_dlog32;
  float pad1;
  double log_emin64, inv_dlog64;
  const float* sig32;        /* [n_mat][5][n_nodes] */
  const double* sig64;
  const float* dedx32;       /* [n_mat] MeV/mm */
  const double* dedx64;
  uint64_t seed;
  int32_t msc;               /* 0: toy model v1; 1: v2, with multiple scattering */
  int32_t pad2;
  const float* x0_32;        /* [n_mat] radiation lengths, mm (v2 only) */
  const double* x0_64;
} oracle_world;

typedef struct {
  uint64_t steps[3];         /* per type */
  uint64_t tracks[3];        /* tracks that existed, per type */
  uint64_t secondaries[3];   /* secondaries created, per type */
  uint64_t reject_cap_hits;
  uint64_t n_iters;          /* iterations until empty */
  uint64_t idlog_n;          /* entries written (or needed, if > capacity) */
  uint64_t errors;           /* 1: iteration log too short, 2: id log too short, 4: bad input */
} oracle_totals;

/*
 * Run the given primaries to completion.
 *  mode      OR_STRICT_FP32 or OR_REF_FP64
 *  score     [n_events][n_slabs] FP64 deposits (continuous + below-cut)
 *  ledger    [n_events][6]: injected, deposited_cont, below_cut, escaped, mass_created,
 *            mass_consumed (all MeV, Neumaier-compensated sums)
 *  counts    [max_iters][3] tracks stepped per iteration and type (may be NULL)
 *  idlog     one record per track at its death (may be NULL)
 *  nthreads  worker threads over events (>= 1)
 * Returns 0, or a non-zero error code (bad input) with totals->errors set.
 */
int oracle_run(const oracle_world* w, const oracle_primary* prim, size_t n_prim, uint32_t n_events,
               int mode, int nthreads, double* score, double* ledger, uint64_t* counts,
               uint64_t max_iters, oracle_idrec* idlog, uint64_t idlog_cap, oracle_totals* totals);

/* One FP32 strict step of one track of the given type (for brute-force pins). */
int oracle_step_one(const oracle_world* w, int type, const oracle_track32* in,
                    oracle_step_result* out);

/* Compton sampler alone (FP32 strict): k = E / mc^2, draws keyed like a step. Returns eps. */
float oracle_sample_compton_eps(float k, uint64_t seed, uint32_t event, uint64_t id, uint32_t step,
                                int* attempts);
void oracle_sample_compton_eps_n(float k, uint64_t seed, uint32_t event, const uint64_t* ids,
                                 uint32_t step, float* eps, int32_t* attempts, size_t n);

#ifdef __cplusplus
}
#endif
#endif
