// Transport kernels: one step kernel per particle type (host-loop and graph
// drivers), one persistent kernel that loops iterations on the device, the
// end-of-iteration bookkeeping and the primary injection.  Both track-buffer
// forms of the paper's Sec. 2 are here:
//
//  dense double buffer: per type, track i of the current array is stepped and
//    its survivor and secondaries are appended to the next array.  Slots are
//    handed out by warp-aggregated allocation: ballots of the per-lane counts
//    (their population counts give the warp's total and each lane's prefix),
//    then one 64-bit atomicAdd for the e- and gamma counters and one for e+ per
//    warp, so a warp's records land contiguously.
//  sparse single buffer: per type, one slot array plus two slot lists (current,
//    next).  A survivor is updated in place (only the leaves the step changed)
//    and its slot appended to the next list; secondaries get fresh slots from a
//    high-water counter, or first from a ring of freed slots when slot reuse is on.
//
// Deposits: one fire-and-forget FP64 reduction per lane into score[event][slab];
// the rarer ledger terms (below cut, escaped, mass created/consumed) likewise.
// The step kernels return at once when the device status word is non-zero; the
// persistent kernel stops at the next iteration boundary (or the one after, when the bit
// was set just before the last block arrived at the barrier).
#pragma once

#include <cuda/atomic>

#include "common.cuh"
#include "layout.cuh"
#include "physics.cuh"

namespace et {

constexpr uint32_t FULL = 0xffffffffu;

// ---- shared-memory staging of geometry and tables ----
// layout: planes[129] | dedx[4] | x0[4] | mat[128] | tot[n_mat*256] (float2) |
//         brem[..] (float2) | cp[n_mat*256] (float4)
__host__ __device__ inline size_t smem_bytes(int n_mat) {
  return 129 * 4 + 4 * 4 + 4 * 4 + 128 + (size_t)n_mat * NBINS * (8 + 8 + 16) + 16;
}

template <bool NEED_G, bool NEED_E>
__device__ Tabs stage_tables(unsigned char* sm, const Args& a) {
  float* planes = reinterpret_cast<float*>(sm);
  float* dedx = planes + 129;
  float* x0 = dedx + 4;
  uint8_t* mat = reinterpret_cast<uint8_t*>(x0 + 4);
  float2* tot = reinterpret_cast<float2*>(mat + 128 + 12);  // 16-byte aligned: 516+32+128+12 = 688
  float2* brem = tot + a.n_mat * NBINS;
  float4* cp = reinterpret_cast<float4*>(brem + a.n_mat * NBINS);
  for (int i = threadIdx.x; i <= (int)a.n_slabs; i += blockDim.x) planes[i] = a.planes[i];
  for (int i = threadIdx.x; i < (int)a.n_slabs; i += blockDim.x) mat[i] = a.mat[i];
  if (threadIdx.x < 4) {
    dedx[threadIdx.x] = a.dedx[threadIdx.x];
    x0[threadIdx.x] = a.x0[threadIdx.x];
  }
  const int nt = (int)a.n_mat * NBINS;
  if (NEED_G) {
    for (int i = threadIdx.x; i < nt; i += blockDim.x) {
      tot[i] = a.tab_tot[i];
      cp[i] = a.tab_cp[i];
    }
  }
  if (NEED_E)
    for (int i = threadIdx.x; i < nt; i += blockDim.x) brem[i] = a.tab_brem[i];
  __syncthreads();
  Tabs tb;
  tb.planes = planes;
  tb.mat = mat;
  tb.tot = tot;
  tb.cp = cp;
  tb.brem = brem;
  tb.dedx = dedx;
  tb.x0 = x0;
  tb.n_slabs = (int)a.n_slabs;
  tb.msc = a.msc;
  return tb;
}

// %lanemask_lt: the bits of the lanes below this one
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Per-type record counts of a lane, packed 10 bits per type (e- bits 0-9, e+ 10-19,
// gamma 20-29).  A step makes at most one e- record (a survivor, or the electron of a
// Compton scattering, a pair or a photoabsorption), at most one e+ record (a survivor, or
// the positron of a pair), and at most three photons (a survivor; the two photons of a
// below-cut positron's annihilation, after a bremsstrahlung photon in a positron step),
// so the counts sit in bit 0, bit 10 and bits 20-21.  One ballot per such bit gives the
// warp's counts (population counts) and each lane's exclusive prefix (population count
// of the lanes below), the bit-1 photon ballot weighted by two.
struct WarpCounts {
  uint32_t total, below;  // the warp's counts and the lane's exclusive prefix, packed alike
  __device__ __forceinline__ WarpCounts(uint32_t packed, uint32_t lt) {
    const uint32_t be = __ballot_sync(0xffffffffu, packed & 1u);
    const uint32_t bp = __ballot_sync(0xffffffffu, packed & (1u << 10));
    const uint32_t bg0 = __ballot_sync(0xffffffffu, packed & (1u << 20));
    const uint32_t bg1 = __ballot_sync(0xffffffffu, packed & (2u << 20));
    total = __popc(be) | (__popc(bp) << 10) | ((__popc(bg0) + 2u * __popc(bg1)) << 20);
    below = __popc(be & lt) | (__popc(bp & lt) << 10) |
            ((__popc(bg0 & lt) + 2u * __popc(bg1 & lt)) << 20);
  }
};

// Reserve per-type runs for a warp: returns the lane's first index per type.  `row` is a
// count row in cw() word order: e- and gamma are reserved together by one 64-bit
// atomicAdd (the counts never reach 2^32, so no carry crosses the halves), e+ by a
// 32-bit one; a warp thus makes one atomic request in the common case.
__device__ __forceinline__ void warp_reserve(uint32_t packed, uint32_t lane, uint32_t* row,
                                             uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const WarpCounts wc(packed, lanemask_lt());
  uint32_t b0 = 0, b1 = 0, b2 = 0;
  if (lane == 0) {
    const uint32_t ne = wc.total & 1023u, np = (wc.total >> 10) & 1023u, ng = wc.total >> 20;
    if (ne | ng) {
      const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(row),
                                               (unsigned long long)ne | ((unsigned long long)ng << 32));
      b0 = (uint32_t)old;
      b2 = (uint32_t)(old >> 32);
    }
    if (np) b1 = atomicAdd(row + cw(EP), np);
  }
  p0 = __shfl_sync(FULL, b0, 0) + (wc.below & 1023u);
  p1 = __shfl_sync(FULL, b1, 0) + ((wc.below >> 10) & 1023u);
  p2 = __shfl_sync(FULL, b2, 0) + (wc.below >> 20);
}

// Next position of the run of type ty, advanced by one.  Written with selects and
// predicated increments: a reference to a dynamically chosen local would put the three
// counters on the stack.
__device__ __forceinline__ uint32_t take(int ty, uint32_t& a0, uint32_t& a1, uint32_t& a2) {
  const uint32_t v = ty == 0 ? a0 : (ty == 1 ? a1 : a2);
  a0 += (uint32_t)(ty == 0);
  a1 += (uint32_t)(ty == 1);
  a2 += (uint32_t)(ty == 2);
  return v;
}

// Sparse form: slots for a warp's new tracks.  Per type, the warp's run of k positions is
// made of `got` reused slots (the ring entries from `ring_base`) followed by fresh slots
// from the high-water counter (from `fresh`); each lane walks its own positions `pos`.
struct SlotRuns {
  uint32_t ring_base[3], got[3], fresh[3];
  uint32_t pos0, pos1, pos2;
};

template <typename T>
__device__ __forceinline__ T sel3(int ty, T v0, T v1, T v2);

__device__ __forceinline__ void sparse_reserve(const Args& a, uint32_t packed, uint32_t lane,
                                               SlotRuns& sr) {
  DevCtl* c = a.ctl;
  const WarpCounts wc(packed, lanemask_lt());
  const bool reuse = a.free_ring[0] != nullptr;
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    uint32_t rb = 0, got = 0, fresh = 0;
    const uint32_t k = (wc.total >> (10 * t)) & 1023u;
    if (lane == 0 && k) {
      if (reuse) {
        rb = atomicAdd(&c->free_head[cw(t)], k);
        const int avail = (int)(__ldcg(&c->free_snap[cw(t)]) - rb);
        got = avail <= 0 ? 0u : (avail < (int)k ? (uint32_t)avail : k);
      }
      if (k > got) fresh = atomicAdd(&c->hwm[cw(t)], k - got);
    }
    sr.ring_base[t] = __shfl_sync(FULL, rb, 0);
    sr.got[t] = __shfl_sync(FULL, got, 0);
    sr.fresh[t] = __shfl_sync(FULL, fresh, 0);
  }
  sr.pos0 = wc.below & 1023u;
  sr.pos1 = (wc.below >> 10) & 1023u;
  sr.pos2 = wc.below >> 20;
}

// The lane's next slot of type ty.
__device__ __forceinline__ uint32_t sparse_slot(const Args& a, SlotRuns& sr, int ty) {
  const uint32_t p = take(ty, sr.pos0, sr.pos1, sr.pos2);
  const uint32_t got = sel3(ty, sr.got[0], sr.got[1], sr.got[2]);
  if (p < got) {
    const uint32_t* ring = sel3(ty, a.free_ring[0], a.free_ring[1], a.free_ring[2]);
    return __ldcg(ring + ((sel3(ty, sr.ring_base[0], sr.ring_base[1], sr.ring_base[2]) + p) &
                          (a.cap - 1u)));
  }
  return sel3(ty, sr.fresh[0], sr.fresh[1], sr.fresh[2]) + (p - got);
}

// Secondary k of a parent that has just taken its step (parent.step already advanced).
__device__ __forceinline__ Trk make_secondary(const Trk& parent, const Sec& s, int k) {
  Trk r;
  r.x = parent.x; r.y = parent.y; r.z = parent.z;
  r.dx = s.dx; r.dy = s.dy; r.dz = s.dz;
  r.e = s.e;
  r.nia = -1.0f;
  r.id = secondary_id(parent.id, parent.step - 1u, (uint32_t)k);
  r.event = parent.event;
  r.step = 0;
  r.slab = parent.slab;
  r.time = parent.time;
  r.len = 0.0f;
  r.flags = 0;
  return r;
}

// Fire-and-forget FP64 add to global memory (no value comes back, so nothing waits on it).
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ void score_step(const Args& a, const Trk& t, const StepOut& o) {
  const size_t ev = t.event;
  const uint32_t c0 = a.score_il ? score_col((uint32_t)o.slab_cont, a.n_slabs) : (uint32_t)o.slab_cont;
  if (o.dep_nz) red_add(&a.score[ev * a.n_slabs + c0], o.dep);
  if (o.bal) {
    if ((o.bal & B_CUT) && o.cut != 0.0) {
      const uint32_t c1 = a.score_il ? score_col((uint32_t)t.slab, a.n_slabs) : (uint32_t)t.slab;
      red_add(&a.score[ev * a.n_slabs + c1], o.cut);
      red_add(&a.ledger[ev * 5 + 1], o.cut);
    }
    if ((o.bal & B_ESC) && o.esc != 0.0f) red_add(&a.ledger[ev * 5 + 2], f2d(o.esc));
    if (o.bal & B_MCR) red_add(&a.ledger[ev * 5 + 3], (double)MC2 + (double)MC2);
    if ((o.bal & B_MC) && o.mc != 0.0) red_add(&a.ledger[ev * 5 + 4], o.mc);
  }
}

// Warp-aggregated append of death records (test runs only).  Two entry points: inline,
// and out of line so that a kernel need not carry the code in its hot loop.  The
// arguments are scalars: a track passed by reference would have to sit in local memory
// around the call.  Which one a kernel uses is chosen by what it spills: the electron
// step kernel, at 64 registers, spills around the call and not with the inline code;
// the photon and positron kernels, and the all-type persistent kernel, run faster with
// the call (+1.9 % and +2.1 % on the batched events, +2 % on the single shower).
__device__ __forceinline__ void log_deaths_inl(IdRec* log, unsigned long long cap, DevCtl* ctl,
                                               bool dead, unsigned long long id, uint32_t steps,
                                               uint32_t type_death, uint32_t lane) {
  const uint32_t mask = __ballot_sync(FULL, dead);
  if (!mask) return;
  unsigned long long base = 0;
  const uint32_t leader = __ffs(mask) - 1;
  if (lane == leader) base = atomicAdd(&ctl->idlog_n, (unsigned long long)__popc(mask));
  base = __shfl_sync(FULL, base, leader);
  if (dead) {
    const unsigned long long at = base + __popc(mask & ((1u << lane) - 1u));
    if (at < cap) {
      IdRec r;
      r.id = id;
      r.steps = steps;
      r.type_death = type_death;
      log[at] = r;
    } else {
      atomicOr(&ctl->status, ST_LOG_FULL);
    }
  }
}
static __device__ __noinline__ void log_deaths(IdRec* log, unsigned long long cap, DevCtl* ctl,
                                               bool dead, unsigned long long id, uint32_t steps,
                                               uint32_t type_death, uint32_t lane) {
  log_deaths_inl(log, cap, ctl, dead, id, steps, type_death, lane);
}

// Per-lane tallies of secondaries per type and sampler-cap hits, kept in registers and
// added to the control block once per warp and iteration (not once per chunk: those
// counters are shared by every warp of the GPU).
struct Tally {
  uint32_t sec[3];
  uint32_t rej;
};

__device__ __forceinline__ void tally_reset(Tally& tl) {
  tl.sec[0] = tl.sec[1] = tl.sec[2] = 0;
  tl.rej = 0;
}

__device__ __forceinline__ void tally_flush(const Args& a, Tally& tl, uint32_t lane) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const uint32_t n = __reduce_add_sync(FULL, tl.sec[t]);
    if (lane == 0 && n) atomicAdd(&a.ctl->secondaries[t], (unsigned long long)n);
  }
  const uint32_t r = __reduce_add_sync(FULL, tl.rej);
  if (lane == 0 && r) atomicAdd(&a.ctl->reject_cap_hits, (unsigned long long)r);
  tally_reset(tl);
}

// Pointer tables of the kernel arguments indexed by a run-time (warp-uniform) type:
// selects between constant-offset parameter reads, no indexed parameter access.
template <typename T>
__device__ __forceinline__ T sel3(int ty, T v0, T v1, T v2) {
  return ty == 0 ? v0 : (ty == 1 ? v1 : v2);
}
__device__ __forceinline__ char* trk_of(const Args& a, int type, int half) {
  return half ? sel3(type, a.trk[0][1], a.trk[1][1], a.trk[2][1])
              : sel3(type, a.trk[0][0], a.trk[1][0], a.trk[2][0]);
}
__device__ __forceinline__ uint32_t* idx_of(const Args& a, int type, int half) {
  return half ? sel3(type, a.idx[0][1], a.idx[1][1], a.idx[2][1])
              : sel3(type, a.idx[0][0], a.idx[1][0], a.idx[2][0]);
}

template <int L, bool INSTR>
__device__ __forceinline__ View<L, INSTR> view_of(const Args& a, int type, int half) {
  View<L, INSTR> v;
  v.base = trk_of(a, type, half);
  v.cap = a.cap;
  v.ins.trace = a.trace;
  v.ins.heat = nullptr;
  if (INSTR)
    v.ins.heat = half ? sel3(type, a.heat[0][1], a.heat[1][1], a.heat[2][1])
                      : sel3(type, a.heat[0][0], a.heat[1][0], a.heat[2][0]);
  v.ins.type = type;
  return v;
}

// ---- per-warp interaction queue ----
// Photon lanes whose step ends in a discrete interaction park (post-transport track,
// interaction context, slot) in a shared-memory ring of QCAP entries per warp, stored
// field-major so that 32 lanes touch 32 consecutive words.  Whenever 32 entries wait,
// the warp drains them with every lane busy; a partial queue is drained when the warp
// moves to another particle type or runs out of chunks.  This keeps the long Compton
// sampler (rejection loop, rotation) from running with most lanes of a warp idle.  The
// same record layout, with the queue capacity as leading dimension, serves the global
// per-process queues of the split step kernels.
constexpr uint32_t QCAP = 64;
constexpr uint32_t QW = 24;  // 16 track words, 7 context words, slot

__host__ __device__ constexpr size_t queue_bytes_per_warp() { return (size_t)QW * QCAP * 4u; }
__host__ __device__ inline size_t tables_bytes_aligned(int n_mat) {
  return (smem_bytes(n_mat) + 15u) & ~(size_t)15u;
}

struct WarpQueue {
  uint32_t* q;  // [QW][QCAP]
  uint32_t head, count;  // warp-uniform
};

// One queue record: word w of entry s at q[w * ld + s] (ld = QCAP, 32-bit indexing, in
// shared memory; the queue capacity, 64-bit indexing, in global memory).
template <typename LD>
__device__ __forceinline__ void q_put(uint32_t* q, LD ld, uint32_t s, const Trk& t,
                                      const Ctx& cx, uint32_t slot) {
  q[0 * ld + s] = __float_as_uint(t.x);
  q[1 * ld + s] = __float_as_uint(t.y);
  q[2 * ld + s] = __float_as_uint(t.z);
  q[3 * ld + s] = __float_as_uint(t.dx);
  q[4 * ld + s] = __float_as_uint(t.dy);
  q[5 * ld + s] = __float_as_uint(t.dz);
  q[6 * ld + s] = __float_as_uint(t.e);
  q[7 * ld + s] = __float_as_uint(t.nia);
  q[8 * ld + s] = (uint32_t)t.id;
  q[9 * ld + s] = (uint32_t)(t.id >> 32);
  q[10 * ld + s] = t.event;
  q[11 * ld + s] = t.step;
  q[12 * ld + s] = (uint32_t)t.slab;
  q[13 * ld + s] = __float_as_uint(t.time);
  q[14 * ld + s] = __float_as_uint(t.len);
  q[15 * ld + s] = t.flags;
  q[16 * ld + s] = __float_as_uint(cx.E);
  q[17 * ld + s] = __float_as_uint(cx.sig);
  q[18 * ld + s] = __float_as_uint(cx.sc);
  q[19 * ld + s] = __float_as_uint(cx.sp);
  q[20 * ld + s] = __float_as_uint(cx.u1);
  q[21 * ld + s] = __float_as_uint(cx.u2);
  q[22 * ld + s] = __float_as_uint(cx.u3);
  q[23 * ld + s] = slot;
}

template <typename LD>
__device__ __forceinline__ void q_get(const uint32_t* q, LD ld, uint32_t s, Trk& t, Ctx& cx,
                                      uint32_t& slot) {
  t.x = __uint_as_float(q[0 * ld + s]);
  t.y = __uint_as_float(q[1 * ld + s]);
  t.z = __uint_as_float(q[2 * ld + s]);
  t.dx = __uint_as_float(q[3 * ld + s]);
  t.dy = __uint_as_float(q[4 * ld + s]);
  t.dz = __uint_as_float(q[5 * ld + s]);
  t.e = __uint_as_float(q[6 * ld + s]);
  t.nia = __uint_as_float(q[7 * ld + s]);
  t.id = (uint64_t)q[8 * ld + s] | ((uint64_t)q[9 * ld + s] << 32);
  t.event = q[10 * ld + s];
  t.step = q[11 * ld + s];
  t.slab = (int32_t)q[12 * ld + s];
  t.time = __uint_as_float(q[13 * ld + s]);
  t.len = __uint_as_float(q[14 * ld + s]);
  t.flags = q[15 * ld + s];
  cx.E = __uint_as_float(q[16 * ld + s]);
  cx.sig = __uint_as_float(q[17 * ld + s]);
  cx.sc = __uint_as_float(q[18 * ld + s]);
  cx.sp = __uint_as_float(q[19 * ld + s]);
  cx.u1 = __uint_as_float(q[20 * ld + s]);
  cx.u2 = __uint_as_float(q[21 * ld + s]);
  cx.u3 = __uint_as_float(q[22 * ld + s]);
  slot = q[23 * ld + s];
}

// Everything after the physics of a finished step, for the lanes with act == true:
// deposits, death records, counters, slot allocation and the writes of the survivor
// and the secondaries.  All 32 lanes of the warp call it together; `type` is
// warp-uniform.
template <int L, bool INSTR, bool DENSE, bool INLINE_LOG>
__device__ __forceinline__ void finish(const Args& a, const int type, uint32_t it, uint32_t lane,
                                       bool act, const Trk& t, const StepOut& o, uint32_t slot,
                                       Tally& tl) {
  const uint32_t hn = (it & 1u) ^ 1u;
  const uint32_t nslot = (it + 1) % 3;
  DevCtl* ctl = a.ctl;
  if (act) score_step(a, t, o);
  const bool alive = act && o.alive;
  const int nsec = act ? o.nsec : 0;
  if (a.idlog) {
    const uint32_t td = (uint32_t)type | ((uint32_t)(act ? o.death : 0) << 8);
    if (INLINE_LOG)
      log_deaths_inl(a.idlog, a.idlog_cap, a.ctl, act && !o.alive, (unsigned long long)t.id,
                     t.step, td, lane);
    else
      log_deaths(a.idlog, a.idlog_cap, a.ctl, act && !o.alive, (unsigned long long)t.id, t.step,
                 td, lane);
  }

  // per-type record counts of this lane: survivor + secondaries
  uint32_t packed_sec = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < nsec) {
      const int ty = o.type(k);
      packed_sec += 1u << (10 * ty);
      tl.sec[0] += ty == 0;
      tl.sec[1] += ty == 1;
      tl.sec[2] += ty == 2;
    }
  }
  const uint32_t packed = (alive ? (1u << (10 * type)) : 0u) + packed_sec;
  if (act) tl.rej += (uint32_t)o.reject;

  uint32_t q0, q1, q2;  // positions in the next arrays (dense) / next slot lists (sparse)
  warp_reserve(packed, lane, ctl->cnt[nslot], q0, q1, q2);

  if constexpr (DENSE) {
    if (alive) {
      const uint32_t at = take(type, q0, q1, q2);
      if (at < a.cap) view_of<L, INSTR>(a, type, (int)hn).store(at, t);
      else atomicOr(&ctl->status, ST_CAPACITY);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < nsec) {
        const int ty = o.type(k);
        const uint32_t at = take(ty, q0, q1, q2);
        if (at < a.cap) view_of<L, INSTR>(a, ty, (int)hn).store(at, make_secondary(t, o.sec(k), k));
        else atomicOr(&ctl->status, ST_CAPACITY);
      }
    }
  } else {
    // slots for the secondaries: reused ones first (when enabled), then fresh ones
    SlotRuns sr;
    sparse_reserve(a, packed_sec, lane, sr);
    if (alive) {
      view_of<L, INSTR>(a, type, 0).store_leaves(slot, t, o.dirty);
      const uint32_t at = take(type, q0, q1, q2);
      if (at < a.cap) idx_of(a, type, (int)hn)[at] = slot;
      else atomicOr(&ctl->status, ST_CAPACITY);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < nsec) {
        const int ty = o.type(k);
        const uint32_t ns = sparse_slot(a, sr, ty);
        const uint32_t at = take(ty, q0, q1, q2);
        if (ns < a.cap && at < a.cap) {
          view_of<L, INSTR>(a, ty, 0).store(ns, make_secondary(t, o.sec(k), k));
          idx_of(a, ty, (int)hn)[at] = ns;
        } else {
          atomicOr(&ctl->status, ST_CAPACITY);
        }
      }
    }
    // the slot of a track that died becomes reusable at the next iteration boundary
    if (a.free_ring[0]) {
      const bool freed = act && !o.alive;
      const uint32_t m = __ballot_sync(FULL, freed);
      if (m) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&ctl->free_tail[cw(type)], (uint32_t)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (freed)
          sel3(type, a.free_ring[0], a.free_ring[1], a.free_ring[2])
              [(base + __popc(m & ((1u << lane) - 1u))) & (a.cap - 1u)] = slot;
      }
    }
  }
}

// One warp transports up to 32 tracks of one type (lanes with valid == false idle).
// With `batch` set, lanes whose photon step ends in a discrete interaction go into the
// warp's queue, which is drained 32 entries at a time, or completely when `drain_all` is
// set (the warp's last chunk of this type); a call with no valid lane only drains.
// Without `batch` (iterations too small to fill a queue), and for e+- at any size, the
// interactions run in place and the whole chunk is finished in one pass: one slot
// reservation instead of two.  Only photons are queued: the Compton sampler is long and
// its rejection loop divergent, while a bremsstrahlung emission is short enough that
// parking it costs more than the idle lanes it saves (measured: 3 % on the persistent
// kernel, 5 % on the per-type kernels of the batched events).
template <int MODE, int L, bool INSTR, bool DENSE, bool INLINE_LOG>
__device__ __forceinline__ void process_warp(const Args& a, const Tabs& tb, const int type,
                                             uint32_t it, uint32_t i, bool valid, uint32_t lane,
                                             WarpQueue& wq, bool batch, bool drain_all, Tally& tl) {
  batch = batch && type == GAM;
  const uint32_t hc = it & 1u;
  Trk t;
  StepOut o;
  Ctx cx;
  uint32_t slot = 0;
  bool inter = false;
  if (valid) {
    if constexpr (DENSE) {
      slot = i;
      t = view_of<L, INSTR>(a, type, (int)hc).load(slot);
    } else {
      slot = __ldcg(idx_of(a, type, (int)hc) + i);
      t = view_of<L, INSTR>(a, type, 0).load(slot);
    }
    inter = transport<MODE>(type, t, tb, a.log_emin, a.inv_dlog, a.half_xy, a.seed_lo, o, cx);
  }
  if (batch) {
    const uint32_t mask = __ballot_sync(FULL, inter);
    if (inter) {
      const uint32_t pos = (wq.head + wq.count + __popc(mask & ((1u << lane) - 1u))) % QCAP;
      q_put(wq.q, QCAP, pos, t, cx, slot);
    }
    wq.count += (uint32_t)__popc(mask);
    __syncwarp();
  }
  // pass 0 finishes this chunk's own lanes (batch: those without an interaction, the
  // others are queued; otherwise all, interactions in place); later passes drain the queue
  bool once = true;
  while (once || wq.count >= 32u || (drain_all && wq.count)) {
    bool act, do_int;
    uint32_t n = 0, s2 = slot;
    if (once) {
      act = batch ? valid && !inter : valid;
      do_int = !batch && inter;
    } else {
      n = wq.count >= 32u ? 32u : wq.count;  // the n oldest queued entries, one per lane
      act = lane < n;
      do_int = act;
      if (act) q_get(wq.q, QCAP, (wq.head + lane) % QCAP, t, cx, s2);
    }
    if (do_int) interact<MODE>(type, t, cx, a.seed_lo, o, a.msc != 0);
    if (!once) __syncwarp();  // entries consumed before their ring slots are reused
    finish<L, INSTR, DENSE, INLINE_LOG>(a, type, it, lane, act, t, o, s2, tl);
    if (!once) {
      wq.head = (wq.head + n) % QCAP;
      wq.count -= n;
    }
    once = false;
  }
}

__device__ __forceinline__ WarpQueue warp_queue(unsigned char* smem, int n_mat) {
  WarpQueue wq;
  wq.q = reinterpret_cast<uint32_t*>(smem + tables_bytes_aligned(n_mat) +
                                     (threadIdx.x >> 5) * queue_bytes_per_warp());
  wq.head = 0;
  wq.count = 0;
  return wq;
}

// ---- per-type step kernel (host-loop and graph drivers) ----
// Dense form: three resident blocks of 256 threads per SM (<= 80 registers; the e+ and
// photon kernels spill a few bytes), 5-7 % faster than two on large iterations.  The
// sparse form keeps its free register budget: capped at 80 it runs 20 % slower.
template <int TYPE, int MODE, int L, bool INSTR, bool DENSE>
__global__ void __launch_bounds__(256, DENSE ? (TYPE == EM ? 4 : 3) : 1) k_step(const __grid_constant__ Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tabs tb = stage_tables<TYPE == GAM, TYPE != GAM>(smem, a);
  const DevCtl* ctl = a.ctl;
  if (ctl->status != 0) return;
  const uint32_t it = ctl->iter;
  uint32_t n = ctl->cnt[it % 3][cw(TYPE)];
  n = n < a.cap ? n : a.cap;
  const uint32_t lane = threadIdx.x & 31u;
  // warps numbered block-first, so that the chunks of a small iteration land on
  // different SMs instead of sharing the schedulers of the first few
  const uint32_t gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  WarpQueue wq = warp_queue(smem, (int)a.n_mat);
  const uint32_t chunks = (n + 31u) / 32u;
  const bool batch = chunks >= 2u * nw;  // each warp sees several chunks: batching pays
  Tally tl;
  tally_reset(tl);
  uint32_t c = gw;
  while (c < chunks || wq.count) {
    const bool more = c < chunks;
    const uint32_t i = c * 32u + lane;
    const bool last = !more || c + nw >= chunks;
    process_warp<MODE, L, INSTR, DENSE, TYPE == EM>(a, tb, TYPE, it, i, more && i < n, lane,
                                                    wq, batch, last, tl);
    c += nw;
  }
  tally_flush(a, tl, lane);
}

// ---- split step kernels: a transport pass, then per-process interaction passes ----
// The transport kernel of a type runs the transport half of the step for every track of
// the type.  A step that ends without a discrete interaction is finished in place; the
// others are appended, with their interaction context and slot, to the global queue of
// their process (one warp-aggregated reservation per queue, field-major records).  The
// interaction kernel of the type then runs its queues chunk by chunk, so that every warp
// executes a single process, and finishes those steps.  The histories are those of the
// fused step: the same functions run on the same values, only in two launches.

// The process an interacting photon will take (the branch `interact` takes on the same
// values); it only sorts the queues, `interact` decides again.
__device__ __forceinline__ int photon_queue(const Ctx& cx) {
  const float r = cx.u1 * cx.sig;
  if (r < cx.sc) return IQ_COMPTON;
  if (r < cx.sc + cx.sp && cx.E > TWO_MC2) return IQ_PAIR;
  return IQ_PHOT;
}

template <int TYPE>
struct TypeQueues {
  static constexpr int first = TYPE == EM ? IQ_BREM_EM : (TYPE == EP ? IQ_BREM_EP : IQ_COMPTON);
  static constexpr int count = TYPE == GAM ? 3 : 1;
};

template <int TYPE>
__device__ __forceinline__ uint32_t* queue_of(const Args& a, int k) {
  if constexpr (TYPE == GAM) return sel3(k, a.iq[IQ_COMPTON], a.iq[IQ_PAIR], a.iq[IQ_PHOT]);
  else return a.iq[TypeQueues<TYPE>::first];
}

template <int TYPE, int MODE, int L, bool DENSE>
__global__ void __launch_bounds__(256, DENSE ? 3 : 1) k_transport(const __grid_constant__ Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tabs tb = stage_tables<TYPE == GAM, TYPE != GAM>(smem, a);
  DevCtl* ctl = a.ctl;
  if (ctl->status != 0) return;
  const uint32_t it = ctl->iter;
  const uint32_t hc = it & 1u;
  uint32_t n = ctl->cnt[it % 3][cw(TYPE)];
  n = n < a.cap ? n : a.cap;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;  // block-first, as k_step
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint32_t chunks = (n + 31u) / 32u;
  using Q = TypeQueues<TYPE>;
  Tally tl;
  tally_reset(tl);
  for (uint32_t ch = gw; ch < chunks; ch += nw) {
    const uint32_t i = ch * 32u + lane;
    const bool valid = i < n;
    Trk t;
    StepOut o;
    Ctx cx;
    uint32_t slot = 0;
    bool inter = false;
    if (valid) {
      if constexpr (DENSE) {
        slot = i;
        t = view_of<L, false>(a, TYPE, (int)hc).load(slot);
      } else {
        slot = __ldcg(idx_of(a, TYPE, (int)hc) + i);
        t = view_of<L, false>(a, TYPE, 0).load(slot);
      }
      inter = transport<MODE>(TYPE, t, tb, a.log_emin, a.inv_dlog, a.half_xy, a.seed_lo, o, cx);
    }
    finish<L, false, DENSE, false>(a, TYPE, it, lane, valid && !inter, t, o, slot, tl);
    // queue positions: one ballot per queue (a lane enters at most one), then one
    // atomicAdd per non-empty queue
    const int k = (TYPE == GAM && inter) ? photon_queue(cx) - IQ_COMPTON : 0;
    const uint32_t lt = lanemask_lt();
    uint32_t b[3] = {0u, 0u, 0u}, mk[3] = {0u, 0u, 0u};
#pragma unroll
    for (int j = 0; j < Q::count; ++j) mk[j] = __ballot_sync(FULL, inter && k == j);
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < Q::count; ++j)
        if (mk[j]) b[j] = atomicAdd(&ctl->iq_n[Q::first + j], (uint32_t)__popc(mk[j]));
    }
    uint32_t base = 0, below = 0;
#pragma unroll
    for (int j = 0; j < Q::count; ++j) {
      const uint32_t bj = __shfl_sync(FULL, b[j], 0);
      if (j == k) {
        base = bj;
        below = __popc(mk[j] & lt);
      }
    }
    if (inter) {
      const uint32_t at = base + below;
      if (at < a.cap) q_put(queue_of<TYPE>(a, k), (size_t)a.cap, at, t, cx, slot);
      else atomicOr(&ctl->status, ST_CAPACITY);
    }
  }
  tally_flush(a, tl, lane);
}

template <int TYPE, int MODE, int L, bool DENSE>
__global__ void __launch_bounds__(256, DENSE ? 3 : 1) k_interact(const __grid_constant__ Args a) {
  const DevCtl* ctl = a.ctl;
  if (ctl->status != 0) return;
  const uint32_t it = ctl->iter;
  using Q = TypeQueues<TYPE>;
  uint32_t m[3] = {0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < Q::count; ++j) m[j] = min(ctl->iq_n[Q::first + j], a.cap);
  // chunk index space [queue 0 chunks][queue 1 chunks][queue 2 chunks]
  const uint32_t w0 = (m[0] + 31u) / 32u, w1 = (m[1] + 31u) / 32u, w2 = (m[2] + 31u) / 32u;
  const uint32_t wt = w0 + w1 + w2;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  Tally tl;
  tally_reset(tl);
  for (uint32_t ch = gw; ch < wt; ch += nw) {
    const int k = ch < w0 ? 0 : (ch < w0 + w1 ? 1 : 2);
    const uint32_t first = k == 0 ? 0u : (k == 1 ? w0 : w0 + w1);
    const uint32_t p = (ch - first) * 32u + lane;
    const bool act = p < sel3(k, m[0], m[1], m[2]);
    Trk t;
    StepOut o;
    Ctx cx;
    uint32_t slot = 0;
    if (act) {
      q_get(queue_of<TYPE>(a, k), (size_t)a.cap, p, t, cx, slot);
      interact<MODE>(TYPE, t, cx, a.seed_lo, o, a.msc != 0);
    }
    finish<L, false, DENSE, false>(a, TYPE, it, lane, act, t, o, slot, tl);
  }
  tally_flush(a, tl, lane);
}

#ifdef ET_HOST_TU
// ---- end of iteration (one thread): log counts, recycle the count slot, advance ----
__global__ void k_end_iteration(const __grid_constant__ Args a, cudaGraphConditionalHandle cond,
                                int use_cond) {
  DevCtl* c = a.ctl;
  const uint32_t it = c->iter;
  const uint32_t cur = it % 3, nxt = (it + 1) % 3;
  for (int t = 0; t < NTYPES; ++t) {
    c->steps[t] += c->cnt[cur][cw(t)];
    const uint32_t li = a.iter_log_wrap ? it % a.max_iters : it;
    if (li < a.max_iters) a.counts_log[(size_t)li * 3 + t] = c->cnt[cur][cw(t)];
    const uint32_t fill = c->cnt[nxt][cw(t)];
    if (a.idx[0][0] == nullptr && fill > c->hwm[cw(t)]) c->hwm[cw(t)] = fill;  // dense: peak fill
  }
  if (it >= a.max_iters && !a.iter_log_wrap) c->status |= ST_ITER_LOG_FULL;
  free_ring_boundary(c);
  for (int t = 0; t < NTYPES; ++t) c->cnt[cur][cw(t)] = 0;
  for (int q = 0; q < N_IQ; ++q) c->iq_n[q] = 0;  // split form: the queues are consumed
  c->iter = it + 1;
  const uint32_t left = c->cnt[nxt][cw(EM)] + c->cnt[nxt][cw(EP)] + c->cnt[nxt][cw(GAM)];
  const bool stop = left == 0 || c->status != 0 || it + 1 >= c->stop_iter ||
                    (a.hybrid_t != 0 && left < a.hybrid_t);
  c->done = stop ? 1u : 0u;
  if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}
#endif

#ifdef ET_HOST_TU
// ---- serving: report the events whose last track has died ----
// Between launches, after k_mark_present: an event that was injected and has no track
// in the current buffers is appended to the completion ring, once; the presence flags
// are cleared for the next scan.
__global__ void k_scan_done(const __grid_constant__ Args a) {
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < a.max_events;
       e += gridDim.x * blockDim.x) {
    if (a.ev_flag[e] != 0u && a.present[e] == 0u) {
      a.ev_flag[e] = 0u;
      const uint32_t pos = atomicAdd(&a.ctl->n_done, 1u);
      a.done_ring[pos % a.done_cap] = e;
    }
    a.present[e] = 0u;
  }
}

// ---- serving: the graph driver's iteration limit, relative to where the stream is ----
__global__ void k_round_stop(const __grid_constant__ Args a, uint32_t rel) {
  DevCtl* c = a.ctl;
  const uint32_t it = c->iter;
  c->stop_iter = it + rel < it ? 0xffffffffu : it + rel;
}

// ---- serving: collect the events completed since the last collection ----
// One block.  For at most max_out completions after *cursor (the completion ring is
// final: every iteration before this kernel has ended), copies the event's per-slab
// deposits (in slab order) and its ledger to out_rows[j] ([n_slabs + 5] doubles) and its number to
// out_events[j], clears the event's scores and ledger (its number can be given to a new
// event afterwards), advances the cursor and writes the count to out_events[max_out].
__global__ void k_serve_collect(const __grid_constant__ Args a, uint32_t* cursor,
                                uint32_t* out_events, double* out_rows, uint32_t max_out) {
  const uint32_t cur = *cursor;
  const uint32_t done = *(volatile uint32_t*)&a.ctl->n_done;
  const uint32_t n = done - cur < max_out ? done - cur : max_out;
  const uint32_t ns = a.n_slabs, row = ns + 5u;
  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t e = a.done_ring[(cur + j) % a.done_cap];
    double* sc = a.score + (size_t)e * ns;
    double* lg = a.ledger + (size_t)e * 5u;
    for (uint32_t i = threadIdx.x; i < row; i += blockDim.x) {
      if (i < ns) {
        const uint32_t col = a.score_il ? score_col(i, ns) : i;
        out_rows[(size_t)j * row + i] = sc[col];
        sc[col] = 0.0;
      } else {
        out_rows[(size_t)j * row + i] = lg[i - ns];
        lg[i - ns] = 0.0;
      }
    }
    if (threadIdx.x == 0) out_events[j] = e;
  }
  if (threadIdx.x == 0) {
    *cursor = cur + n;
    out_events[max_out] = n;
  }
}
#endif

// ---- grid barrier for the persistent kernel (bounded wait) ----
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of the persistent kernel.  Every block's thread 0 announces its arrival
// with a release reduction on a counter that only grows (nblocks per barrier); block 0's
// thread 0 waits (acquire) until the counter reaches nblocks * (gen + 1), moves the
// sparse form's slot-reuse ring boundary (`rings`) while every other block waits, and
// publishes the next generation (release); the others wait (acquire) for it.  The
// published word carries the generation (bits 1..31) and whether the status word was
// non-zero (bit 0), the snapshot that every block's next decision uses: it travels with
// the generation, so no other write has to complete before the release.  The status is
// loaded with every poll of the counter (issued before the acquire, both loads in
// flight); a bit set just before the last arrival is seen one barrier later -- the bits
// are sticky, every block still takes the same decision, and the error is reported.
// `gen` is thread 0's copy of the generation count, read once at kernel start (it cannot
// move before every block has arrived at the first barrier).  The stop flag goes to
// `stop_out` (shared memory).  Every wait is bounded: on timeout the block sets
// ST_TIMEOUT and the function returns false.
static __device__ bool grid_sync(DevCtl* c, uint32_t nblocks, unsigned long long timeout_ns,
                                 uint32_t& gen, bool rings, uint32_t* stop_out) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t g = gen;
    int ok = 1;
    uint32_t stop = 0u;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&c->bar_count) : "memory");
    const unsigned long long t0 = global_ns();
    if (blockIdx.x == 0) {
      const uint32_t target = nblocks * (g + 1u);
      uint32_t st_seen = 0u;
      for (;;) {
        uint32_t v;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(st_seen) : "l"(&c->status) : "memory");
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&c->bar_count) : "memory");
        if ((int32_t)(v - target) >= 0) break;
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(&c->status, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
      if (ok) {
        stop = st_seen != 0u ? 1u : 0u;
        if (rings) free_ring_boundary(c);
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(&c->bar_gen), "r"(((g + 1u) << 1) | stop)
                     : "memory");
      }
    } else {
      const uint32_t gw = g & 0x7fffffffu;
      for (;;) {
        uint32_t v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(&c->bar_gen) : "memory");
        if ((v >> 1) != gw) {
          stop = v & 1u;
          break;
        }
        if (global_ns() - t0 > timeout_ns) {
          atomicOr(&c->status, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    gen = g + 1u;
    *stop_out = stop;
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ---- persistent kernel: all types, all iterations, one cooperative launch ----
// Warp chunks of 32 tracks are type-uniform: the iteration's index space is
// [ceil(n_e-/32) chunks of e-][chunks of e+][chunks of gamma].  Warp w takes chunks
// w, w + nw, ... and, when the iteration gives every warp two or more chunks, the last
// round from a per-iteration counter (a counter for every chunk measured slower).
template <int MODE, int L, bool INSTR, bool DENSE>
// Three resident blocks of 256 threads per SM (<= 80 registers per thread; a handful of
// bytes spill): 24 warps per SM hide more of the step's dependent latency than 16 warps
// at 120 registers did (measured 7 % faster on the 1,000 x 10 GeV shower).
__global__ void __launch_bounds__(256, 3) k_persistent(const __grid_constant__ Args a,
                                                    int fault_skip_block) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_n[3];
  __shared__ uint32_t s_stop;
  const Tabs tb = stage_tables<true, true>(smem, a);
  WarpQueue wq = warp_queue(smem, (int)a.n_mat);
  DevCtl* c = a.ctl;
  const uint32_t lane = threadIdx.x & 31u;
  // two warp numberings: block-major for large iterations; block-first for small ones, so
  // that their few chunks land on different SMs instead of sharing the schedulers of
  // the first few
  const uint32_t gw_major = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t gw_spread = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  if ((int)blockIdx.x == fault_skip_block) return;  // host-side fault injection: never arrives
  uint32_t it = *(volatile uint32_t*)&c->iter;
  const uint32_t stop_rel = *(volatile uint32_t*)&c->stop_rel;
  const uint32_t stop_iter = stop_rel == 0u ? *(volatile uint32_t*)&c->stop_iter
                             : (it + stop_rel < it ? 0xffffffffu : it + stop_rel);
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // before this block's first barrier: no other
    c->run_iter0 = it;                        // block can have changed these yet
    for (int t = 0; t < NTYPES; ++t) {
      c->run_steps0[t] = c->steps[t];
      c->run_sec0[t] = c->secondaries[t];
    }
  }
  // the generation count (the published word holds it shifted left by one)
  uint32_t bar_gen = threadIdx.x == 0 ? (*(volatile uint32_t*)&c->bar_gen) >> 1 : 0u;
  __shared__ uint32_t s_snap_stop;
  // block 0's copy of the dense form's peak fill: it only stores, so that its thread 0
  // (lane 0 of the warp that takes a small iteration's first chunk) waits on no load
  __shared__ uint32_t s_hwm[3];
  if (DENSE && blockIdx.x == 0 && threadIdx.x == 0)
    for (int t = 0; t < 3; ++t) s_hwm[t] = c->hwm[cw(t)];
  bool first = true;
  Tally tl;  // flushed when the loop ends
  tally_reset(tl);
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t cur = it % 3;
      for (int t = 0; t < 3; ++t) s_n[t] = __ldcg(&c->cnt[cur][cw(t)]);
      // the first decision uses only what the launch started with (the same in every
      // block: a block that starts late must not see a status bit set by another block's
      // first iteration); later ones use the snapshot taken at the barrier
      const uint32_t st = first ? 0u : s_snap_stop;
      const uint32_t tot = s_n[0] + s_n[1] + s_n[2];
      s_stop = tot == 0 || it >= stop_iter || st != 0 || (a.hybrid_t != 0 && tot >= a.hybrid_t);
      // an iteration's counts are the fill of the one before (the launch's first counts
      // were recorded by the launch before, or come from injection)
      if (DENSE && blockIdx.x == 0 && !first) {
        for (int t = 0; t < 3; ++t) {
          if (s_n[t] > s_hwm[t]) {
            s_hwm[t] = s_n[t];
            c->hwm[cw(t)] = s_n[t];
          }
        }
      }
    }
    __syncthreads();
    first = false;
    if (s_stop) break;
    const uint32_t n0 = min(s_n[0], a.cap), n1 = min(s_n[1], a.cap), n2 = min(s_n[2], a.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      if (a.iter_ns && it < a.max_iters) a.iter_ns[it] = global_ns();
      for (int t = 0; t < 3; ++t) {
        c->cnt[(it + 2) % 3][cw(t)] = 0;
        atomicAdd(&c->steps[t], (unsigned long long)s_n[t]);  // a reduction: nothing waits
        const uint32_t li = a.iter_log_wrap ? it % a.max_iters : it;
        if (li < a.max_iters) a.counts_log[(size_t)li * 3 + t] = s_n[t];
      }
      if (it >= a.max_iters && !a.iter_log_wrap) atomicOr(&c->status, ST_ITER_LOG_FULL);
    }
    const uint32_t w0 = (n0 + 31) / 32, w1 = (n1 + 31) / 32, w2 = (n2 + 31) / 32;
    const uint32_t wt = w0 + w1 + w2;
    // chunk order: warp w takes chunks w, w + nw, ... below S, then the rest from a counter
    // (the last round of each iteration goes to the warps that finish first); a warp's
    // chunk indices increase, so its type changes at most twice per iteration, and the
    // queue is emptied at each change
    const bool batch = wt >= 2u * nw;  // each warp sees several chunks: batching pays
    const uint32_t S = batch ? (wt / nw - 1u) * nw : wt;
    uint32_t* grab = &c->grab[it % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0) c->grab[(it + 2) % 3] = 0u;  // last used in it - 1
    uint32_t ch = batch ? gw_major : gw_spread;
    int qtype = EM;
    while (ch < wt || wq.count) {
      int ty = qtype;
      uint32_t i = 0;
      bool valid = false, drain_all = true;
      if (ch < wt) {
        const int cty = ch < w0 ? EM : (ch < w0 + w1 ? EP : GAM);
        if (cty == qtype || wq.count == 0) {
          ty = qtype = cty;
          const uint32_t base = ty == EM ? 0u : (ty == EP ? w0 : w0 + w1);
          const uint32_t nt = ty == EM ? n0 : (ty == EP ? n1 : n2);
          i = (ch - base) * 32u + lane;
          valid = i < nt;
          uint32_t nxt = ch + nw;
          if (batch && nxt >= S) {
            uint32_t g = 0;
            if (lane == 0) g = atomicAdd(grab, 1u);
            nxt = S + __shfl_sync(FULL, g, 0);
          }
          const int nty = nxt < wt ? (nxt < w0 ? EM : (nxt < w0 + w1 ? EP : GAM)) : -1;
          drain_all = nty != ty;  // the warp's last chunk of this type
          ch = nxt;
        }
        // else: drain the previous type's queue first; this chunk is taken next round
      }
      process_warp<MODE, L, INSTR, DENSE, false>(a, tb, ty, it, i, valid, lane, wq, batch,
                                                 drain_all, tl);
    }
    if (!grid_sync(c, gridDim.x, a.timeout_ns, bar_gen, a.free_ring[0] != nullptr, &s_snap_stop))
      return;
    ++it;
  }
  tally_flush(a, tl, lane);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->iter = it;
    const uint32_t cur = it % 3;
    for (int t = 0; t < 3; ++t) c->cnt[(it + 2) % 3][cw(t)] = 0;  // between iterations only cur is non-zero
    for (int t = 0; t < 3; ++t) c->grab[t] = 0u;
    c->done = (__ldcg(&c->cnt[cur][cw(EM)]) + __ldcg(&c->cnt[cur][cw(EP)]) +
               __ldcg(&c->cnt[cur][cw(GAM)]) == 0);
  }
}

// ---- serving: which events still have tracks ----
// Between launches: every track of the current iteration marks its event present (plain
// stores of 1: idempotent).  A scan of the event field of the active tracks -- 4 bytes a
// track, coalesced -- replaces per-step live-track counting in the step kernels, whose
// atomics on the few counters of the events in flight cost more than the whole scan.
template <int L, bool DENSE>
__global__ void k_mark_present(const __grid_constant__ Args a) {
  const DevCtl* c = a.ctl;
  const uint32_t it = c->iter;
  const uint32_t hc = it & 1u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (int t = 0; t < NTYPES; ++t) {
    uint32_t n = c->cnt[it % 3][cw(t)];
    n = n < a.cap ? n : a.cap;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
      uint32_t ev;
      if constexpr (DENSE) {
        ev = view_of<L, false>(a, t, (int)hc).template ld<uint32_t>(i, F_EVENT);
      } else {
        const uint32_t slot = __ldcg(idx_of(a, t, (int)hc) + i);
        ev = view_of<L, false>(a, t, 0).template ld<uint32_t>(slot, F_EVENT);
      }
      if (ev < a.max_events) a.present[ev] = 1u;
    }
  }
}

// ---- injection of primaries into the current iteration's tracks ----
struct Primary {
  uint32_t type, event;
  unsigned long long id;
  float pos[3], dir[3], ekin;
  uint32_t pad;
};

template <int L, bool DENSE>
__global__ void k_inject(const __grid_constant__ Args a, const Primary* p, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t base_i = i0 - lane;
  if (base_i >= n) return;  // warp-uniform
  const bool valid = i0 < n;
  DevCtl* c = a.ctl;
  const uint32_t it = c->iter;
  const uint32_t cur = it % 3, hc = it & 1u;
  Trk t{};
  int type = 0;
  bool ok = false;
  if (valid) {
    const Primary q = p[i0];
    ok = q.type < 3u && q.event < a.max_events && q.ekin > 0.0f && q.ekin < 3.0e38f &&
         fabsf(q.pos[0]) <= a.half_xy && fabsf(q.pos[1]) <= a.half_xy &&
         q.pos[2] >= a.planes[0] && q.pos[2] < a.planes[a.n_slabs] && isfinite(q.dir[0]) &&
         isfinite(q.dir[1]) && isfinite(q.dir[2]);
    if (!ok) atomicOr(&c->status, ST_BAD_PRIMARY);
  }
  if (ok) {
    const Primary q = p[i0];
    type = (int)q.type;
    t.x = q.pos[0]; t.y = q.pos[1]; t.z = q.pos[2];
    t.dx = q.dir[0]; t.dy = q.dir[1]; t.dz = q.dir[2];
    t.e = q.ekin;
    t.nia = -1.0f;
    t.id = q.id;
    t.event = q.event;
    t.step = 0;
    int s = 0;  // slab s: planes[s] <= z < planes[s+1] (z validated above)
    while (s + 1 < (int)a.n_slabs && !(t.z < a.planes[s + 1])) ++s;
    t.slab = s;
    t.time = 0.0f;
    t.len = 0.0f;
    t.flags = 0;
    atomicAdd(&a.ledger[(size_t)t.event * 5 + 0], (double)t.e);
    if (a.ev_flag) a.ev_flag[t.event] = 1u;
  }
  const uint32_t packed = ok ? (1u << (10 * type)) : 0u;
  uint32_t q0, q1, q2;
  warp_reserve(packed, lane, c->cnt[cur], q0, q1, q2);
  if (DENSE) {
    if (ok) {
      const uint32_t at = sel3(type, q0, q1, q2);
      if (at < a.cap) view_of<L, false>(a, type, (int)hc).store(at, t);
      else atomicOr(&c->status, ST_CAPACITY);
    }
  } else {
    SlotRuns sr;
    sparse_reserve(a, packed, lane, sr);
    if (ok) {
      const uint32_t slot = sparse_slot(a, sr, type);
      const uint32_t at = sel3(type, q0, q1, q2);
      if (slot < a.cap && at < a.cap) {
        view_of<L, false>(a, type, 0).store(slot, t);
        (hc ? a.idx[type][1] : a.idx[type][0])[at] = slot;
      } else {
        atomicOr(&c->status, ST_CAPACITY);
      }
    }
  }
}

}  // namespace et
