/*
 * et.h -- C ABI of the GB300 EM shower transport hot path.
 *
 * One transport iteration advances every active track of every particle type
 * (e-, e+, gamma) by one step; survivors and secondaries become the tracks of
 * the next iteration (paper Sec. 2).  The tracks live per type either in a
 * "dense double buffer" (two dense arrays, current and next, filled by
 * compaction, Sec. 2 / Fig. 1b) or in a "sparse single buffer" (one sparse
 * array plus two slot lists, Sec. 2 / Fig. 1a), in one of the layouts of
 * Sec. 3-4 (AoS, SoA, AoSoA-N; plus a hot/cold split), optionally instrumented to count
 * per-field reads/writes and per-word accesses (Sec. 5).  The benchmark shape
 * (an electron gun into 50 absorber/gap layers, energy scored per layer) is
 * that of Sec. 4; the physics is a fixed toy EM model.
 *
 * Conventions
 *  - Every function returns et_status; nothing aborts and nothing throws.
 *    After a failure, et_last_error(ctx) describes it.
 *  - Host pointers passed in are read during the call only (the library copies
 *    what it keeps); the caller keeps ownership.  Output pointers are host
 *    memory the caller owns, unless a name says "_device".
 *  - The library owns all device memory of a context.  It allocates through the
 *    caller's allocator callbacks when given (e.g. a framework's caching
 *    allocator), else with cudaMalloc.  All work is issued on cfg.cuda_stream
 *    (NULL: the legacy default stream).
 *  - A context is used from one host thread at a time.
 *  - Calls out of order (inject before tables, etc.) return ET_ERR_STATE.
 *  - Device-side failures (a full track buffer, a bounded wait that ran out)
 *    are recorded in a device status word and reported by the next call that
 *    synchronises (et_run_iteration, et_run_until_empty, et_read_*).
 */
#ifndef ET_H
#define ET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct et_ctx et_ctx;

typedef enum {
  ET_OK = 0,
  ET_ERR_INVALID = 1,   /* bad argument */
  ET_ERR_CAPACITY = 2,  /* a track buffer, event table or log is full */
  ET_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  ET_ERR_TIMEOUT = 4,   /* a bounded device wait ran out (persistent driver) */
  ET_ERR_STATE = 5,     /* call out of order */
  ET_ERR_NOMEM = 6      /* allocation failed */
} et_status;

enum { ET_EMINUS = 0, ET_EPLUS = 1, ET_GAMMA = 2, ET_NTYPES = 3 };
enum { ET_FORM_SPARSE = 0, ET_FORM_DENSE = 1 };
/* AoSoA-N: blocks of N records, each leaf stored N-wide inside its block (Sec. 3-4);
 * AoSoA-128 needs capacity_log2 >= 7. */
enum {
  ET_LAYOUT_AOS = 0,
  ET_LAYOUT_SOA = 1,
  ET_LAYOUT_AOSOA32 = 2,
  ET_LAYOUT_AOSOA64 = 3,
  ET_LAYOUT_AOSOA8 = 4,
  ET_LAYOUT_AOSOA16 = 5,
  ET_LAYOUT_AOSOA128 = 6,
  ET_LAYOUT_HOTCOLD = 7  /* hot 52 bytes AoSoA-32, cold time/length/flags SoA */
};
enum { ET_MODE_STRICT = 0, ET_MODE_FAST = 1 };
/* HYBRID: the persistent kernel while fewer than cfg.hybrid_tracks tracks are active,
 * the CUDA graph of per-type step kernels while at least that many are. */
enum { ET_DRIVER_HOSTLOOP = 0, ET_DRIVER_GRAPH = 1, ET_DRIVER_PERSISTENT = 2, ET_DRIVER_HYBRID = 3 };

/* Device allocator callbacks: return NULL on failure. */
typedef void* (*et_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*et_free_fn)(void* ptr, void* user);

typedef struct {
  uint32_t capacity_log2;   /* track slots per type and buffer (dense) or per type (sparse) */
  int32_t form;             /* ET_FORM_* */
  int32_t layout;           /* ET_LAYOUT_* */
  int32_t mode;             /* ET_MODE_*: strict = bit-exact toy model, fast = intrinsics + FMA */
  int32_t driver;           /* ET_DRIVER_*: how et_run_until_empty iterates */
  int32_t block_size;       /* threads per block of the step kernels (64..256, multiple of 32; 0 = 256) */
  uint64_t seed;            /* physics seed, below 2^32 (Philox key word 0); larger: ET_ERR_INVALID */
  uint32_t max_events;      /* events are numbered 0..max_events-1 */
  uint32_t max_iters;       /* length of the per-iteration count log */
  int32_t instrument;       /* 1: count per-field reads/writes and per-word accesses */
  int32_t id_log;           /* 1: record (id, steps, type|death<<8) of every track at its death */
  uint64_t id_log_capacity; /* records (when id_log) */
  void* cuda_stream;        /* cudaStream_t */
  et_alloc_fn alloc;        /* optional; both or neither */
  et_free_fn free;
  void* alloc_user;
  int32_t serving;          /* 1: report completed events (et_poll_completed, the et_serve_*
                               loop), for continuous batching; the iteration
                               count log then wraps (iteration it at entry it % max_iters)
                               instead of filling up */
  int32_t reuse_slots;      /* sparse form: 1 = slots of dead tracks are reused (from the next
                               iteration on); 0 = never reused (the plain single buffer) */
  uint32_t hybrid_tracks;   /* ET_DRIVER_HYBRID: the switch-over population (0 = 2^21) */
  int32_t split_interactions; /* 1: split step kernels (host-loop, graph and the graph phase
                               of hybrid): per type, a transport pass appends the steps that
                               end in a discrete interaction to one global queue per process,
                               then an interaction pass runs each queue with process-uniform
                               warps -- the divergent code paths of Sec. 1 sorted out of the
                               warps.  Same histories as the fused step.  Needs 96 bytes x
                               2^capacity_log2 per process queue (5 queues); not with
                               ET_DRIVER_PERSISTENT or instrument (ET_ERR_INVALID). */
  int32_t msc;              /* 0: the toy model (v1); 1: the toy model v2, which adds multiple
                               scattering of e+-: a step limit of 0.04 max(T/dEdx, 0.5 mm)
                               and a deflection of Highland's width after every step (the
                               multiple-scattering fields of the paper's Sec. 5 electron
                               trace).  Needs the radiation lengths (et_load_msc) before the
                               first injection. */
} et_config;

/* Create a context (allocates the track buffers).  *out is NULL on failure. */
et_status et_create(const et_config* cfg, et_ctx** out);
et_status et_destroy(et_ctx* ctx);
const char* et_last_error(const et_ctx* ctx);

/*
 * Calorimeter geometry (paper Sec. 4: 50 alternating absorber/gap box layers).
 * n_slabs (<= 128) slabs stacked along +z from z = 0; thickness_mm[n_slabs]
 * (FP64; the plane positions are the FP64 running sums rounded to FP32);
 * material[n_slabs] indexes the tables (< n_materials); |x|, |y| <= half_xy_mm.
 * Outside is vacuum: a track leaving the box escapes.
 */
et_status et_create_geometry(et_ctx* ctx, uint32_t n_slabs, const double* thickness_mm,
                             const uint8_t* material, float half_xy_mm);

/*
 * Cross-section tables of the toy model, per material m < n_materials (<= 4):
 * sigma[m][k][i] (1/mm) for k = 0 Compton, 1 pair, 2 photoelectric, 3 photon
 * total, 4 bremsstrahlung, at nodes i < n_nodes (257) spaced uniformly in
 * ln E; a lookup takes x = (log E - log_emin) * inv_dlog.  dedx[m] in MeV/mm.
 * The lookup constants are FP32 values (the strict model fixes them).
 * Tables are staged in shared memory by every step kernel (8 KB per material).
 */
et_status et_load_tables(et_ctx* ctx, uint32_t n_materials, uint32_t n_nodes, float log_emin,
                         float inv_dlog, const float* sigma, const float* dedx);

/*
 * Radiation lengths X0 (mm) per material, for the multiple scattering of the toy model
 * v2 (et_config.msc = 1): the width 13.6 MeV / (beta c p) sqrt(s/X0) (1 + 0.038 ln(s/X0))
 * of Highland's formula.  Call after et_load_tables (same n_materials), before the
 * first injection; ET_ERR_STATE on a v1 context or out of order, ET_ERR_INVALID for
 * values that are not positive and finite.
 */
et_status et_load_msc(et_ctx* ctx, uint32_t n_materials, const float* x0_mm);

/* The toy model's radiation lengths (FP32 of 5.612 mm lead, 140 mm liquid argon). */
et_status et_toy_radiation_lengths(uint32_t n_materials, float* x0_out);

/*
 * The toy model's own tables, computed on the host from the FP64 closed forms
 * and rounded to FP32 (Compton: Klein-Nishina; pair: log rise above 2 mc^2;
 * photoelectric: Z^4/E^3; brems: ln(T/k_c)/X0), for materials 0 = lead and
 * 1 = liquid argon.  sigma_out[n_materials][5][n_nodes], dedx_out[n_materials].
 */
et_status et_build_toy_tables(uint32_t n_materials, uint32_t n_nodes, float* sigma_out,
                              float* dedx_out, float* log_emin_out, float* inv_dlog_out);

/*
 * The same closed forms, not rounded: FP64 nodes for the all-FP64 build below.
 * sigma_out[n_materials][5][n_nodes], dedx_out[n_materials]; log_emin_out and
 * inv_dlog_out (optional) receive ln(1e-3 MeV) and (n_nodes - 1) / ln(1e8).
 */
et_status et_build_toy_tables_fp64(uint32_t n_materials, uint32_t n_nodes, double* sigma_out,
                                   double* dedx_out, double* log_emin_out, double* inv_dlog_out);

/* A primary particle (48 bytes). */
typedef struct {
  uint32_t type;   /* ET_EMINUS, ET_EPLUS, ET_GAMMA */
  uint32_t event;  /* < max_events */
  uint64_t id;     /* unique; convention (event << 32) | index in event */
  float pos[3];    /* mm, inside the calorimeter */
  float dir[3];    /* unit vector */
  float ekin;      /* MeV (kinetic; photon energy) */
  uint32_t pad;
} et_primary;

/*
 * Inject n primaries (host array, copied): they become active tracks of the
 * next iteration.  Their injected energy is added to their events' ledgers.
 * The array is copied into the context's pinned staging before the call
 * returns; the transfer to the device and the injection kernel then run
 * asynchronously on the stream (a later et_inject waits for the staging to
 * be free).
 */
et_status et_inject(et_ctx* ctx, const et_primary* primaries, size_t n);

/*
 * As et_inject, for primaries already in device memory (n records of
 * et_primary, 16-byte aligned, read by a kernel on the context's stream; the
 * caller keeps them alive until that stream passes this point).  Each record
 * is validated on the device; an invalid one is skipped and reported as
 * ET_ERR_INVALID by the next synchronising call.
 */
et_status et_inject_device(et_ctx* ctx, const et_primary* primaries_device, size_t n);

typedef struct {
  uint32_t n_active[3];     /* tracks per type active in the next iteration */
  uint32_t pad;
  uint64_t steps;           /* track steps taken (this iteration / in total) */
  uint64_t secondaries;     /* secondaries created */
} et_iter_stats;

/*
 * One transport iteration (Sec. 2): every active track takes one step; survivors and
 * secondaries become the next iteration's tracks.  Host-driven whatever the driver: the
 * per-type step kernels, then the end-of-iteration kernel.  out (may be NULL): tracks active in the next
 * iteration, steps and secondaries of this one.  ET_ERR_CAPACITY when a track buffer or
 * the iteration log overflows; ET_ERR_STATE before geometry and tables.
 */
et_status et_run_iteration(et_ctx* ctx, et_iter_stats* out);

/*
 * Iterate (Sec. 2) until no track is left or max_iters more iterations ran, with
 * the configured driver (host loop, CUDA graph, persistent kernel, hybrid).
 * Totals and the number of iterations run are optional outputs.  Errors as for
 * et_run_iteration, plus ET_ERR_TIMEOUT when a bounded wait of the persistent
 * kernel's grid barrier ran out (the context then needs et_reset).  The persistent driver
 * issues one launch and one read-back (the launch records its starting
 * counters); the others read the counters back before they start.  Returns
 * after the stream has finished the run.
 */
et_status et_run_until_empty(et_ctx* ctx, uint64_t max_iters, et_iter_stats* totals,
                             uint64_t* n_iters);

/* Energy ledger of one event (MeV). */
typedef struct {
  double injected, deposited_cont, below_cut, escaped, mass_created, mass_consumed;
} et_ledger;

/*
 * The energy scored per layer (the benchmark's observable, paper Sec. 4) for one
 * event: slab_dep[n_slabs] (host, may be NULL; n_slabs >= the geometry's) receives the
 * per-slab deposits in MeV (continuous loss in the slab a step started in, plus
 * below-cut remainders in the slab a track ended in; FP64 sums), out (may be NULL) the
 * event's ledger.  Synchronises.  ET_ERR_INVALID for event >= max_events or a short
 * buffer.
 */
et_status et_read_scoring(et_ctx* ctx, uint32_t event, double* slab_dep, size_t n_slabs,
                          et_ledger* out);

/* All events at once: score[max_events][n_slabs], ledger[max_events] (either may be NULL). */
et_status et_read_scoring_all(et_ctx* ctx, double* score, et_ledger* ledger);

/* Tracks stepped per iteration and type since the last reset: counts[n][3], n <= cap. */
et_status et_read_iteration_counts(et_ctx* ctx, uint64_t* counts, uint64_t cap, uint64_t* n);

/* Death records (16 bytes each: id, steps, type | death << 8); needs cfg.id_log. */
typedef struct {
  uint64_t id;
  uint32_t steps;
  uint32_t type_death;
} et_idrec;
et_status et_read_id_log(et_ctx* ctx, et_idrec* out, uint64_t cap, uint64_t* n);

/* Instrumented build (cfg.instrument): reads/writes per type and field,
 * counts[3][15][2] over the 15 leaf fields of the 64-byte track record. */
et_status et_read_field_trace(et_ctx* ctx, uint64_t* counts);

/* Instrumented build: accesses per 4-byte word of one track buffer (type, half
 * 0/1; the sparse form has half 0 only); out[capacity * 16] uint32. */
et_status et_read_heatmap(et_ctx* ctx, uint32_t type, uint32_t half, uint32_t* out, uint64_t cap);

/* Run counters (host copies). */
typedef struct {
  uint64_t steps[3];          /* per type */
  uint64_t secondaries[3];    /* per type */
  uint64_t iterations;        /* since reset */
  uint64_t slot_high_water[3];/* sparse: slots ever used; dense: peak next-buffer fill */
  uint64_t reject_cap_hits;   /* Compton sampler attempt cap reached */
  uint64_t kernel_launches;   /* launches issued by the library since reset */
  uint32_t status;            /* device status word (0 = fine) */
  uint32_t pad;
} et_counters;
et_status et_read_counters(et_ctx* ctx, et_counters* out);

/*
 * Checkpoint / resume.  et_snapshot copies the state of a context between iterations
 * into host memory: control block and counters, the live part of the track arrays
 * (dense: the current buffer's first n records per type; sparse: the slot array, the
 * current slot list and the reuse rings), scores, ledgers, the iteration log, the
 * serving counters, the death log and the instrumentation counts.  et_snapshot_size
 * gives the bytes it needs (cap); written receives the bytes written.  et_restore
 * loads a snapshot into a context created with the same configuration (ET_ERR_INVALID
 * otherwise, or for a damaged snapshot) after loading the same geometry and tables;
 * every draw is keyed by (event, id, step), so the restored context follows exactly the
 * histories the original would have.  Completed events reported before the snapshot
 * are not reported again.  All three synchronise the stream.
 */
et_status et_snapshot_size(et_ctx* ctx, uint64_t* bytes);
et_status et_snapshot(et_ctx* ctx, void* out, uint64_t cap, uint64_t* written);
et_status et_restore(et_ctx* ctx, const void* in, uint64_t n);

/* Forget all tracks, scores, ledgers, logs and counters (buffers stay allocated). */
et_status et_reset(et_ctx* ctx);

/*
 * Serving (cfg.serving): events whose last track died since the previous call (at most
 * cap; *n receives the number written).  An event is complete when it was injected and
 * none of the current tracks belongs to it: a scan of the active tracks' event fields
 * between launches finds them, in event-number order.  The call synchronises the
 * context's stream.
 */
et_status et_poll_completed(et_ctx* ctx, uint32_t* events, uint64_t cap, uint64_t* n);

/* Serving: clear an event's scores, ledger and completion state so that its number can be
 * given to a new event (call after reading its results). */
et_status et_release_event(et_ctx* ctx, uint32_t event);

/*
 * Native serving loop (continuous batching, the paper's AdePT offload pattern of Sec. 1
 * and 2: a host hands over events while others are in flight; each iteration advances
 * every active track of every event).  Serving contexts only (cfg.serving = 1).
 *
 * et_serve_submit queues one event's n primaries (host memory, copied; every primary's
 * .event == event < max_events) with its reserve: the track slots per type
 * (e-, e+, gamma) the event may occupy at its peak.  Requests are admitted in submission
 * order while the reserves of the events in flight fit into 90 % of the capacity per
 * type (the first one is always admitted), and never while an event of the same number
 * is in flight.  ET_ERR_CAPACITY: a reserve above the capacity.
 *
 * et_serve_round runs one round: it admits and injects what fits, runs `iters`
 * iterations with every shower in flight (the persistent driver launches them
 * asynchronously; the other drivers read counts back between iterations), and queues a
 * collection of the events completed so far (their per-slab deposits and ledgers are
 * copied out and cleared on the device, so their numbers can be given to new events).
 * It then waits for the previous round and returns that round's completions:
 * events[n_out], rows[n_out][n_slabs + 5] = per-slab deposits, then the ledger injected,
 * below-cut, escaped, mass created, mass consumed (MeV); steps (optional) the track-steps
 * the previous round took; in_flight (optional) the events admitted or queued and not yet
 * returned.  Round k's GPU work is queued before round k - 1 is waited for, so the host's
 * admission and read-back overlap the GPU.  cap >= et_serve_capacity's max_results.
 * et_serve_flush waits for the last round and returns its completions (call when no
 * more requests come, until in_flight is 0, with rounds in between).
 */
et_status et_serve_submit(et_ctx* ctx, const et_primary* primaries, size_t n, uint32_t event,
                          const uint32_t reserve[3]);
et_status et_serve_round(et_ctx* ctx, uint32_t iters, uint32_t* events, double* rows,
                         uint64_t cap, uint64_t* n_out, uint64_t* steps, uint32_t* in_flight);
et_status et_serve_flush(et_ctx* ctx, uint32_t* events, double* rows, uint64_t cap,
                         uint64_t* n_out, uint64_t* steps, uint32_t* in_flight);
/* The most completions one round returns (the result buffers' row count). */
et_status et_serve_capacity(et_ctx* ctx, uint32_t* max_results);

/*
 * Timing of the step kernels (CUDA events on the context's stream around every
 * step-kernel launch, or around the persistent kernel): total milliseconds and
 * number of timed launches since the last call.  Enabled by et_set_timing(ctx, 1).
 */
et_status et_set_timing(et_ctx* ctx, int on);
et_status et_read_timing(et_ctx* ctx, double* ms_total, uint64_t* launches);

/*
 * Transport of one batch without any device allocation.  (The paper has no
 * counterpart: this is a deployment convenience of this library.)
 *
 * For callers that cannot allocate device memory -- code running inside another
 * framework's memory pool or under a budget that forbids cudaMalloc, code that must
 * not synchronise the device (cudaMalloc/cudaFree may), plug-ins handed a stream and
 * buffers but no allocator.  All scratch (dense double buffers of the three particle
 * types, control block, iteration log, staged geometry and tables) lives in one
 * file-scope device array of ET_NOALLOC_SCRATCH_BYTES, reserved on a device when the
 * module holding it is loaded there and held by that device until the process exits.
 * The call allocates nothing itself: no cudaMalloc, no cudaFree, no allocating library
 * routine.  Under CUDA's lazy module loading (the default) the modules are loaded by
 * the first call on each device, which reserves the array then and may synchronise;
 * a caller that needs the guarantee from the very first call sets
 * CUDA_MODULE_LOADING=EAGER or makes one warm-up call.
 *
 * Inputs: geometry and tables in host memory, as for et_create_geometry and
 * et_load_tables (257 nodes per table); n_primaries records in device memory
 * (16-byte aligned), validated on the device; seed below 2^32 (the Philox key word).
 * The sizes of the device buffers cannot be checked here: score_device and
 * ledger_device must hold n_events rows.  Outputs (device memory, zeroed and
 * written by the call): score_device[n_events][n_slabs] per-slab deposits and
 * ledger_device[n_events][5] = injected, below-cut, escaped, mass created, mass
 * consumed (MeV).  steps_out (host, optional) receives the track steps taken.  The
 * physics is the strict mode, run with the dense double buffer in AoS layout by the
 * persistent kernel on `cuda_stream`; the call returns after the stream has finished.
 *
 * Limits: at most ET_NOALLOC_MAX_TRACKS active tracks per type in any iteration (and
 * that many primaries), at most ET_NOALLOC_MAX_ITERS iterations; beyond either the
 * call returns ET_ERR_CAPACITY with a message in err (err_len bytes, may be NULL).  A
 * primary the device rejects (type, event >= n_events, energy, position) is skipped and
 * the call returns ET_ERR_INVALID after the others have been transported.
 *
 * The first call on a device looks up the array's device address (once per device,
 * with that device current); make that first call before any stream capture.  Every
 * call shares the array and leaves its contents behind; a call clears what must start
 * at zero.  Calls whose work overlaps on the GPU (different streams or host threads)
 * race on the array.
 */
#define ET_NOALLOC_MAX_TRACKS 32768u
#define ET_NOALLOC_MAX_ITERS 4096u
#define ET_NOALLOC_SCRATCH_BYTES (13u << 20)
et_status et_transport_noalloc(uint32_t n_slabs, const double* thickness_mm,
                               const uint8_t* material, float half_xy_mm, uint32_t n_materials,
                               float log_emin, float inv_dlog, const float* sigma,
                               const float* dedx, const et_primary* primaries_device,
                               size_t n_primaries, uint64_t seed, uint32_t n_events,
                               double* score_device, double* ledger_device, uint64_t* steps_out,
                               void* cuda_stream, char* err, size_t err_len);

/*
 * All-FP64 transport (the precision comparison of the mixed-primary workload, which
 * sets the FP32-stepping path against a build where state, tables and arithmetic are
 * all FP64): the toy model of the strict mode with every REAL in FP64 and
 * libm-accuracy log, exp, sin and cos, i.e. the GPU counterpart of the FP64 reference
 * model, not a bit-exact mirror of it (CUDA's and the C library's log/exp may differ
 * in the last bit).  Iterations as in Sec. 2 (each active track advances one step;
 * survivors and secondaries form the next iteration), dense double buffer of 128-byte
 * AoS records, one step kernel per particle type, launched from the host until no
 * track is left.  A plain path: it allocates its buffers (cudaMalloc) per call and
 * returns only when the run is over.
 *
 * Inputs (host memory): geometry as for et_create_geometry; FP64 tables
 * sigma[n_materials][5][257] in the node layout of et_load_tables, dedx[n_materials];
 * n primaries; 2^capacity_log2 (6..26) slots per type and buffer.  Outputs (host
 * memory): score_out[n_events][n_slabs] per-slab deposits, ledger_out[n_events][5]
 * (optional) as for et_transport_noalloc, steps_out and iterations_out (optional).
 * Errors: ET_ERR_INVALID for bad arguments (a seed of 2^32 or more among them) or
 * primaries (type, event >= n_events, ekin <= 0, z outside the slabs);
 * ET_ERR_CAPACITY if the primaries or a buffer
 * exceed the capacity; ET_ERR_TIMEOUT after 65536 iterations with tracks left;
 * ET_ERR_NOMEM / ET_ERR_CUDA from the runtime.  Uses the current device's default
 * stream.
 */
et_status et_run_fp64(uint32_t n_slabs, const double* thickness_mm, const uint8_t* material,
                      double half_xy_mm, uint32_t n_materials, double log_emin, double inv_dlog,
                      const double* sigma, const double* dedx, const et_primary* primaries,
                      size_t n, uint64_t seed, uint32_t n_events, uint32_t capacity_log2,
                      double* score_out, double* ledger_out, uint64_t* steps_out,
                      uint64_t* iterations_out);

#ifdef __cplusplus
}
#endif
#endif
