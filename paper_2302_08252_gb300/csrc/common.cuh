// Shared definitions of the GPU transport path: track record, device control
// block, kernel arguments, Philox4x32-10, track ids and the strict-mode
// elementary functions of the toy model.
//
// Track record (64 bytes, 15 leaf fields): the stand-in for AdePT's track
// struct of the paper's Sec. 3 (position, navigation state, ...), here
// position, direction, kinetic energy, interaction lengths left, id, event,
// track-local step, slab (the navigation state), and three cold fields (time,
// track length, flags) so that the instrumentation sees hot and cold fields
// as the paper's heatmaps do (Sec. 5).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace et {

enum { EM = 0, EP = 1, GAM = 2, NTYPES = 3 };
enum { LIM_Z = 0, LIM_X = 1, LIM_Y = 2, LIM_LOSS = 3, LIM_PHYS = 4, LIM_MSC = 5 };
enum { PROC_NONE = 0, PROC_COMPTON = 1, PROC_PAIR = 2, PROC_PHOT = 3, PROC_BREM = 4 };
enum { ALIVE = 0, DEATH_ESCAPE = 1, DEATH_CUT = 2, DEATH_ABSORB = 3 };
enum { MODE_STRICT = 0, MODE_FAST = 1 };

// device status bits
enum : uint32_t {
  ST_CAPACITY = 1u,       // a next buffer / slot pool overflowed (writes were dropped)
  ST_TIMEOUT = 2u,        // grid barrier wait ran out
  ST_LOG_FULL = 4u,       // id log full (records dropped)
  ST_ITER_LOG_FULL = 8u,  // iteration count log full
  ST_BAD_PRIMARY = 16u,   // a device-side primary failed validation (skipped)
};

// ---- leaf fields of the track record: byte offset and size ----
enum Leaf {
  F_X = 0, F_Y, F_Z, F_DX, F_DY, F_DZ, F_E, F_NIA, F_ID, F_EVENT, F_STEP, F_SLAB, F_TIME, F_LEN,
  F_FLAGS, NLEAF
};
__host__ __device__ constexpr int leaf_off(int f) { return f <= F_NIA ? 4 * f : (f == F_ID ? 32 : 4 * f + 4); }
__host__ __device__ constexpr int leaf_size(int f) { return f == F_ID ? 8 : 4; }
static_assert(leaf_off(F_FLAGS) == 60, "record is 64 bytes");
static_assert(leaf_off(F_EVENT) == 40, "id is 8 bytes at 32");

struct Trk {
  float x, y, z, dx, dy, dz, e, nia;
  uint64_t id;
  uint32_t event, step;
  int32_t slab;
  float time, len;
  uint32_t flags;
};

// dirty-leaf bits for the sparse form's in-place update
enum : uint32_t {
  D_POS = (1u << F_X) | (1u << F_Y) | (1u << F_Z),
  D_DIR = (1u << F_DX) | (1u << F_DY) | (1u << F_DZ),
  D_E = 1u << F_E,
  D_NIA = 1u << F_NIA,
  D_STEP = 1u << F_STEP,
  D_SLAB = 1u << F_SLAB,
  D_TIME = 1u << F_TIME,
  D_LEN = 1u << F_LEN,
  D_FLAGS = 1u << F_FLAGS,
  D_ALL = (1u << NLEAF) - 1u,
};

// Count rows hold the types in the word order e-, gamma, e+ (then a pad word), so that
// the e- and gamma counters are one aligned 64-bit word: a warp reserves room for both
// (photon steps make electrons, electron steps make photons) with one atomic.
__host__ __device__ constexpr int cw(int type) { return type == EM ? 0 : (type == GAM ? 1 : 2); }

// Process queues of the split step kernels: the interactions of one iteration, sorted by
// process (e- bremsstrahlung; e+ bremsstrahlung; photon Compton, pair, photoelectric).
enum { IQ_BREM_EM = 0, IQ_BREM_EP = 1, IQ_COMPTON = 2, IQ_PAIR = 3, IQ_PHOT = 4, N_IQ = 5 };

// ---- device control block (one per context) ----
// Fields that different warps, blocks or kernels touch at the same time sit on separate
// 128-byte lines: each count row (read at an iteration's start, while the next row takes
// every warp's slot reservations), the barrier counter and generation, the chunk
// counters.  Packed into a few lines they cost 3 % on the single shower and 9 % on the
// batched events (L2 contention between the atomics and the polls).
constexpr int CTL_LINE = 32;  // 32-bit words per 128-byte line
struct alignas(128) DevCtl {
  // tracks per type (word cw(t) of the row; the rest of the line is padding); row it%3
  // current, (it+1)%3 next
  alignas(128) uint32_t cnt[3][CTL_LINE];
  alignas(128) uint32_t iter;   // iteration about to run
  uint32_t status;              // ST_* bits
  uint32_t done;                // 1 when no track is left (graph driver)
  uint32_t stop_iter;           // the graph/persistent drivers stop before this iteration
  unsigned long long secondaries[NTYPES];
  unsigned long long steps[NTYPES];
  unsigned long long reject_cap_hits;
  unsigned long long idlog_n;
  alignas(128) uint32_t hwm[4];  // word cw(t) -- sparse: slots handed out; dense: peak next fill
  alignas(128) uint32_t bar_count;  // grid barrier (persistent driver)
  alignas(128) uint32_t bar_gen;  // generation << 1 | (status non-zero at that barrier)
  alignas(128) uint32_t n_done;  // serving: events completed so far (completion ring position)
  // sparse slot reuse, per type (monotone counters; ring index = value % cap): slots in
  // [free_head, free_snap) may be taken in this iteration, slots freed in this iteration
  // are appended at free_tail and become takeable at the next iteration boundary
  uint32_t free_head[4], free_tail[4], free_snap[4];  // word cw(t)
  // persistent driver: a non-zero stop_rel stops the launch after that many iterations
  // (instead of at stop_iter); the launch records where it started, so that the host
  // needs no read-back before it
  uint32_t stop_rel;
  alignas(128) uint32_t grab[4];  // persistent driver: dynamic chunk counter of iteration it (row it % 3)
  alignas(128) uint32_t run_iter0;
  unsigned long long run_steps0[NTYPES], run_sec0[NTYPES];
  // split step kernels: entries in each process queue in this iteration (IQ_*); zeroed at
  // the iteration's end
  alignas(128) uint32_t iq_n[8];
};

// Iteration boundary bookkeeping of the slot-reuse rings (one thread, all other
// threads quiescent): heads that overshot the takeable range are pulled back, and the
// slots freed in the iteration just ended become takeable.
__device__ __forceinline__ void free_ring_boundary(DevCtl* c) {
  for (int w = 0; w < 3; ++w) {
    if ((int32_t)(c->free_head[w] - c->free_snap[w]) > 0) c->free_head[w] = c->free_snap[w];
    c->free_snap[w] = c->free_tail[w];
  }
}

struct IdRec {
  unsigned long long id;
  uint32_t steps;
  uint32_t type_death;
};

// Column of slab s in an event's row of deposits (ns slabs).  Within each complete group
// of 32 slabs, slabs alternate between the group's two 128-byte halves (s -> 16 (s mod 2)
// + (s mod 32) / 2), so that the adjacent slabs of a shower's maximum, which take most
// of its deposits, fall on different L2 lines; a shower still touches the same few lines
// of its row.  The last, incomplete group keeps its order.  A bijection on [0, ns).
__host__ __device__ __forceinline__ uint32_t score_col(uint32_t s, uint32_t ns) {
  const uint32_t g = s & ~31u;
  return g + 32u <= ns ? g + ((s & 1u) << 4) + ((s & 31u) >> 1) : s;
}

// ---- kernel arguments (passed by value) ----
struct Args {
  char* trk[NTYPES][2];         // dense: [type][half]; sparse: [type][0]
  uint32_t* idx[NTYPES][2];     // sparse: slot lists [type][parity]
  uint32_t cap;                 // slots per buffer
  DevCtl* ctl;
  uint32_t* counts_log;         // [max_iters][3]
  uint32_t max_iters;
  uint32_t iter_log_wrap;        // serving: the count log is a ring (entry it % max_iters)
  uint32_t hybrid_t;             // hybrid driver: the persistent kernel stops before an iteration
                                 // with this many tracks, the graph before one with fewer (0: off)
  uint32_t n_slabs;
  double* score;                // [max_events][n_slabs], columns in score_col order
  uint32_t score_il;            // 1: slabs interleaved in each row (score_col), 0: in order
  double* ledger;               // [max_events][5]: injected, cut, escaped, mass_created, mass_consumed
  uint32_t max_events;
  uint32_t n_mat;
  const float4* tab_cp;         // [n_mat][256] {C, C[i+1]-C[i], P, P[i+1]-P[i]}
  const float2* tab_tot;        // [n_mat][256] {T, dT}
  const float2* tab_brem;       // [n_mat][256] {B, dB}
  const float* planes;          // [n_slabs + 1]
  const uint8_t* mat;           // [n_slabs]
  float half_xy, log_emin, inv_dlog;
  float dedx[4];
  int32_t msc;                  // toy model v2: multiple scattering of e+- (0: v1)
  float x0[4];                  // radiation lengths (mm), v2 only
  uint32_t seed_lo;
  IdRec* idlog;                 // NULL: off
  unsigned long long idlog_cap;
  unsigned long long* trace;    // [3][15][2] or NULL
  uint32_t* heat[NTYPES][2];    // per-word access counts or NULL
  unsigned long long timeout_ns;// bounded waits (persistent driver)
  unsigned long long* iter_ns;  // persistent driver: %globaltimer at each iteration start, or NULL
  // serving: events with a track in the current buffers (set by k_mark_present, cleared
  // by k_scan_done), events injected and not yet reported complete, and the ring of
  // completed events (NULL: off)
  uint32_t* present;            // [max_events]
  uint32_t* done_ring;          // [done_cap] completed event ids, position n_done % done_cap
  uint32_t* ev_flag;            // [max_events] 1: injected, completion not yet reported
  uint32_t done_cap;
  // sparse form with slot reuse: ring of freed slots per type (NULL: slots never reused)
  uint32_t* free_ring[NTYPES];  // [cap] each
  // split step kernels: one global interaction queue per process (IQ_*), field-major
  // records of QW words, [QW][cap] each (NULL: the split form is off)
  uint32_t* iq[N_IQ];
};

constexpr int MAX_SLABS = 128;
constexpr int MAX_MAT = 4;
constexpr int NBINS = 256;  // table intervals (257 nodes)

// ---- Philox4x32-10 (Salmon et al., SC'11), written from its published definition ----
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  return make_uint4(c0, c1, c2, c3);
}

// ---- exact conversions without the conversion instructions ----
// On this GPU int<->float and float->double conversions and FRND issue to the FP64
// pipe (2 lanes per cycle per SM), so the hot path builds the same values with integer
// and FP32 operations instead.  Each function returns exactly what the named
// conversion returns on its stated domain.

// (float)v for an integer 0 <= v <= 2^24: the low 23 bits through the 2^23 magic
// number (2^23 + lo - 2^23 == lo), the top bits added as exact powers of two.
__device__ __forceinline__ float u24_to_float(uint32_t v) {
  const float lo = __uint_as_float(0x4B000000u | (v & 0x7FFFFFu)) - 8388608.0f;
  const uint32_t hi = v >> 23;  // 0, 1 or 2
  return lo + (hi == 0u ? 0.0f : (hi == 1u ? 8388608.0f : 16777216.0f));
}

// rintf(y) (ties to even) and its integer value, for |y| < 2^22: adding 1.5 * 2^23 rounds
// to an integer (ulp 1 in [2^23, 2^24)); the integer sits in the low mantissa bits.
__device__ __forceinline__ float rint_small(float y, int& n) {
  const float m = y + 12582912.0f;
  n = __float_as_int(m) - 0x4B400000;
  return m - 12582912.0f;
}

// floorf(y) and (int)floorf(y), for |y| < 2^22.
__device__ __forceinline__ float floor_small(float y, int& n) {
  float r = rint_small(y, n);
  if (r > y) {
    r = r - 1.0f;
    n = n - 1;
  }
  return r;
}

// (float)e for a small integer |e| < 2^22.
__device__ __forceinline__ float small_int_to_float(int e) {
  return __int_as_float(0x4B400000 + e) - 12582912.0f;
}

// (double)x for a positive normal float: re-bias the exponent, widen the mantissa.
__device__ __forceinline__ double pos_normal_to_double(float x) {
  const uint32_t u = __float_as_uint(x);
  const uint32_t e = (u >> 23) & 0xFFu;
  const uint32_t m = u & 0x7FFFFFu;
  return __hiloint2double((int)(((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// (double)x for any x >= +0 or -0 (energies): bit assembly for normal values, the
// conversion instruction only for subnormals.
__device__ __forceinline__ double f2d(float x) {
  if (x >= 0x1p-126f) return pos_normal_to_double(x);
  if (x == 0.0f) return __hiloint2double((int)(__float_as_uint(x) & 0x80000000u), 0);
  return (double)x;
}

// (x >> 8) + 1 is at most 2^24, so both the conversion and the scaling are exact.
__device__ __forceinline__ float u01(uint32_t x) {
  return u24_to_float((x >> 8) + 1u) * 0x1p-24f;
}

// SplitMix64 finalizer (Steele, Lea, Flood, OOPSLA 2014)
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t secondary_id(uint64_t parent, uint32_t step,
                                                          uint32_t ordinal) {
  const uint64_t tag = ((uint64_t)step << 2) | (uint64_t)(ordinal & 3u) | (1ull << 62);
  return mix64(parent ^ mix64(tag));
}

// ---- strict-mode elementary functions of the toy model ----
// log: x = m 2^e, m in (sqrt(1/2), sqrt(2)], log m = 2 atanh((m-1)/(m+1)) to r^9, e ln2 as hi+lo
// (Cody-Waite).  exp: n = rint(x/ln2), r = (x - n ln2_hi) - n ln2_lo, Taylor degree 7, 2^n by
// exponent bits.  sincos(2 pi u): 4u = q + y, |y| <= 1/2, a = y pi/2, Taylor sin to a^9 and
// cos to a^8, rotated by the quadrant q.  These translation units are built with --fmad=false.
__device__ __forceinline__ float s_log(float x) {
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = m * 0.5f;
    e = e + 1;
  }
  const float r = (m - 1.0f) / (m + 1.0f);
  const float r2 = r * r;
  float s = 0x1.c71c72p-4f;           // 1/9
  s = s * r2 + 0x1.24924ap-3f;        // 1/7
  s = s * r2 + 0x1.99999ap-3f;        // 1/5
  s = s * r2 + 0x1.555556p-2f;        // 1/3
  s = s * r2;
  const float t = r + r * s;
  const float lm = t + t;
  const float fe = small_int_to_float(e);
  return fe * 0x1.62e4p-1f + (lm + fe * 0x1.7f7d1cp-20f);
}

__device__ __forceinline__ float s_exp(float x) {
  if (x > 88.0f) return __uint_as_float(0x7f800000u);
  if (x < -87.0f) return 0.0f;
  int ni;
  const float n = rint_small(x * 0x1.715476p+0f, ni);  // |x / ln2| < 128
  float r = x - n * 0x1.62e4p-1f;
  r = r - n * 0x1.7f7d1cp-20f;
  float p = 0x1.a01a02p-13f;          // 1/5040
  p = p * r + 0x1.6c16c2p-10f;        // 1/720
  p = p * r + 0x1.111112p-7f;         // 1/120
  p = p * r + 0x1.555556p-5f;         // 1/24
  p = p * r + 0x1.555556p-3f;         // 1/6
  p = p * r + 0.5f;
  p = p * r + 1.0f;
  p = p * r + 1.0f;
  return p * __uint_as_float((uint32_t)(ni + 127) << 23);
}

__device__ __forceinline__ void s_sincos2pi(float u, float* so, float* co) {
  const float v = 4.0f * u;
  int qi;
  const float q = rint_small(v, qi);  // 0 <= v <= 4
  const float y = v - q;
  const float a = y * 0x1.921fb6p+0f;
  const float a2 = a * a;
  float ps = 0x1.71de3ap-19f;         // 1/9!
  ps = ps * a2 - 0x1.a01a02p-13f;     // 1/7!
  ps = ps * a2 + 0x1.111112p-7f;      // 1/5!
  ps = ps * a2 - 0x1.555556p-3f;      // 1/3!
  ps = ps * a2 + 1.0f;
  const float sa = a * ps;
  float pc = 0x1.a01a02p-16f;         // 1/8!
  pc = pc * a2 - 0x1.6c16c2p-10f;     // 1/6!
  pc = pc * a2 + 0x1.555556p-5f;      // 1/4!
  pc = pc * a2 - 0.5f;
  pc = pc * a2 + 1.0f;
  const float ca = pc;
  const int k = qi & 3;
  if (k == 0) { *so = sa; *co = ca; }
  else if (k == 1) { *so = ca; *co = -sa; }
  else if (k == 2) { *so = -sa; *co = -ca; }
  else { *so = -ca; *co = sa; }
}

}  // namespace et
