// Transport kernels: one step kernel per particle type (host-loop and graph
// drivers), one persistent kernel that loops iterations on the device, the
// end-of-iteration bookkeeping and the primary injection.  Both track-buffer
// forms of the paper's Sec. 2 are here:
//
//  dense double buffer: per type, track i of the current array is stepped and
//    its survivor and secondaries are appended to the next array.  Slots are
//    handed out by warp-aggregated allocation: one inclusive warp scan over
//    per-lane counts packed 10 bits per type, then one atomicAdd per type per
//    warp (ballot/popc style), so a warp's records land contiguously.
//  sparse single buffer: per type, one slot array plus two slot lists (current,
//    next).  A survivor is updated in place (only the leaves the step changed)
//    and its slot appended to the next list; secondaries get fresh slots from a
//    high-water counter (never reused) or a free-slot stack (serving).
//
// Deposits: one FP64 atomicAdd per lane into score[event][slab]; the rarer
// ledger terms (below cut, escaped, mass created/consumed) likewise.
// Every kernel returns at once when the device status word is non-zero.
#pragma once

#include <cuda/atomic>

#include "common.cuh"
#include "layout.cuh"
#include "physics.cuh"

namespace et {

constexpr uint32_t FULL = 0xffffffffu;

// ---- shared-memory staging of geometry and tables ----
// layout: planes[129] | dedx[4] | mat[128] | tot[n_mat*256] (float2) | brem[..] (float2) |
//         cp[n_mat*256] (float4)
__host__ __device__ inline size_t smem_bytes(int n_mat) {
  return 129 * 4 + 4 * 4 + 128 + (size_t)n_mat * NBINS * (8 + 8 + 16) + 16;
}

template <bool NEED_G, bool NEED_E>
__device__ Tabs stage_tables(unsigned char* sm, const Args& a) {
  float* planes = reinterpret_cast<float*>(sm);
  float* dedx = planes + 129;
  uint8_t* mat = reinterpret_cast<uint8_t*>(dedx + 4);
  float2* tot = reinterpret_cast<float2*>(mat + 128 + 12);  // 16-byte aligned: 516+16+128+12 = 672
  float2* brem = tot + a.n_mat * NBINS;
  float4* cp = reinterpret_cast<float4*>(brem + a.n_mat * NBINS);
  for (int i = threadIdx.x; i <= (int)a.n_slabs; i += blockDim.x) planes[i] = a.planes[i];
  for (int i = threadIdx.x; i < (int)a.n_slabs; i += blockDim.x) mat[i] = a.mat[i];
  if (threadIdx.x < 4) dedx[threadIdx.x] = a.dedx[threadIdx.x];
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
  tb.n_slabs = (int)a.n_slabs;
  return tb;
}

// inclusive warp scan of packed per-type counts (10 bits per type)
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v, uint32_t lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t u = __shfl_up_sync(FULL, v, d);
    if (lane >= (uint32_t)d) v += u;
  }
  return v;
}

// Reserve per-type runs for a warp: returns the lane's first index per type.
__device__ __forceinline__ void warp_reserve(uint32_t packed, uint32_t lane, uint32_t* counters,
                                             uint32_t& p0, uint32_t& p1, uint32_t& p2) {
  const uint32_t incl = warp_incl_scan(packed, lane);
  const uint32_t total = __shfl_sync(FULL, incl, 31);
  const uint32_t excl = incl - packed;
  uint32_t base = 0;
  if (lane < 3) {
    const uint32_t n = (total >> (10 * lane)) & 1023u;
    if (n) base = atomicAdd(&counters[lane], n);
  }
  p0 = __shfl_sync(FULL, base, 0) + (excl & 1023u);
  p1 = __shfl_sync(FULL, base, 1) + ((excl >> 10) & 1023u);
  p2 = __shfl_sync(FULL, base, 2) + ((excl >> 20) & 1023u);
}

__device__ __forceinline__ uint32_t& pick(int ty, uint32_t& a0, uint32_t& a1, uint32_t& a2) {
  return ty == 0 ? a0 : (ty == 1 ? a1 : a2);
}

__device__ __forceinline__ Trk make_secondary(const Trk& parent, const Sec& s) {
  Trk r;
  r.x = parent.x; r.y = parent.y; r.z = parent.z;
  r.dx = s.dx; r.dy = s.dy; r.dz = s.dz;
  r.e = s.e;
  r.nia = -1.0f;
  r.id = s.id;
  r.event = parent.event;
  r.step = 0;
  r.slab = parent.slab;
  r.time = parent.time;
  r.len = 0.0f;
  r.flags = 0;
  return r;
}

__device__ __forceinline__ void score_step(const Args& a, const Trk& t, const StepOut& o) {
  const size_t ev = t.event;
  if (o.dep != 0.0) atomicAdd(&a.score[ev * a.n_slabs + (size_t)o.slab_cont], o.dep);
  if (o.cut != 0.0) {
    atomicAdd(&a.score[ev * a.n_slabs + (size_t)t.slab], o.cut);
    atomicAdd(&a.ledger[ev * 5 + 1], o.cut);
  }
  if (o.esc != 0.0) atomicAdd(&a.ledger[ev * 5 + 2], o.esc);
  if (o.mcr != 0.0) atomicAdd(&a.ledger[ev * 5 + 3], o.mcr);
  if (o.mc != 0.0) atomicAdd(&a.ledger[ev * 5 + 4], o.mc);
}

// warp-aggregated append of death records
__device__ __forceinline__ void log_deaths(const Args& a, bool dead, const Trk& t, int type,
                                           int death, uint32_t lane) {
  const uint32_t mask = __ballot_sync(FULL, dead);
  if (!mask) return;
  unsigned long long base = 0;
  const uint32_t leader = __ffs(mask) - 1;
  if (lane == leader) base = atomicAdd(&a.ctl->idlog_n, (unsigned long long)__popc(mask));
  base = __shfl_sync(FULL, base, leader);
  if (dead) {
    const unsigned long long at = base + __popc(mask & ((1u << lane) - 1u));
    if (at < a.idlog_cap) {
      IdRec r;
      r.id = t.id;
      r.steps = t.step;
      r.type_death = (uint32_t)type | ((uint32_t)death << 8);
      a.idlog[at] = r;
    } else {
      atomicOr(&a.ctl->status, ST_LOG_FULL);
    }
  }
}

// warp-aggregated per-type secondaries and reject-cap counters
__device__ __forceinline__ void count_secondaries(const Args& a, uint32_t packed_sec, int reject,
                                                  uint32_t lane) {
  uint32_t v = packed_sec;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(FULL, v, d);
  if (lane < 3) {
    const uint32_t n = (v >> (10 * lane)) & 1023u;
    if (n) atomicAdd(&a.ctl->secondaries[lane], (unsigned long long)n);
  }
  const uint32_t rj = __ballot_sync(FULL, reject != 0);
  if (rj && lane == 0) atomicAdd(&a.ctl->reject_cap_hits, (unsigned long long)__popc(rj));
}

template <int L, bool INSTR>
__device__ __forceinline__ View<L, INSTR> view_of(const Args& a, int type, int half) {
  View<L, INSTR> v;
  v.base = half ? a.trk[type][1] : a.trk[type][0];
  v.cap = a.cap;
  v.ins.trace = a.trace;
  v.ins.heat = INSTR ? (half ? a.heat[type][1] : a.heat[type][0]) : nullptr;
  v.ins.type = type;
  return v;
}

// One warp steps up to 32 tracks of type TYPE (lanes with valid == false idle).
template <int TYPE, int MODE, int L, bool INSTR, bool DENSE>
__device__ __forceinline__ void process_warp(const Args& a, const Tabs& tb, uint32_t it, uint32_t i,
                                             bool valid, uint32_t lane) {
  const uint32_t hc = it & 1u, hn = hc ^ 1u;
  const uint32_t nslot = (it + 1) % 3;
  DevCtl* ctl = a.ctl;
  Trk t;
  StepOut o;
  uint32_t slot = 0;
  if (valid) {
    if constexpr (DENSE) {
      slot = i;
      t = view_of<L, INSTR>(a, TYPE, (int)hc).load(slot);
    } else {
      slot = __ldcg((hc ? a.idx[TYPE][1] : a.idx[TYPE][0]) + i);
      t = view_of<L, INSTR>(a, TYPE, 0).load(slot);
    }
    step_track<TYPE, MODE>(t, tb, a.log_emin, a.inv_dlog, a.half_xy, a.seed_lo, o);
    score_step(a, t, o);
  } else {
    o.alive = 0;
    o.nsec = 0;
    o.reject = 0;
    o.death = ALIVE;
  }
  if (a.idlog) log_deaths(a, valid && !o.alive, t, TYPE, o.death, lane);

  // per-type record counts of this lane: survivor + secondaries
  uint32_t packed = (valid && o.alive) ? (1u << (10 * TYPE)) : 0u;
  uint32_t packed_sec = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < o.nsec) packed_sec += 1u << (10 * o.sec(k).type);
  packed += packed_sec;
  count_secondaries(a, packed_sec, valid ? o.reject : 0, lane);

  uint32_t q0, q1, q2;  // positions in the next arrays (dense) / next slot lists (sparse)
  warp_reserve(packed, lane, ctl->cnt[nslot], q0, q1, q2);

  if constexpr (DENSE) {
    if (valid && o.alive) {
      const uint32_t at = pick(TYPE, q0, q1, q2)++;
      if (at < a.cap) view_of<L, INSTR>(a, TYPE, (int)hn).store(at, t);
      else atomicOr(&ctl->status, ST_CAPACITY);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < o.nsec) {
        const int ty = o.sec(k).type;
        const uint32_t at = pick(ty, q0, q1, q2)++;
        if (at < a.cap) view_of<L, INSTR>(a, ty, (int)hn).store(at, make_secondary(t, o.sec(k)));
        else atomicOr(&ctl->status, ST_CAPACITY);
      }
    }
  } else {
    // fresh slots for the secondaries
    uint32_t s0, s1, s2;
    warp_reserve(packed_sec, lane, ctl->hwm, s0, s1, s2);
    if (valid && o.alive) {
      view_of<L, INSTR>(a, TYPE, 0).store_leaves(slot, t, o.dirty);
      const uint32_t at = pick(TYPE, q0, q1, q2)++;
      if (at < a.cap) (hn ? a.idx[TYPE][1] : a.idx[TYPE][0])[at] = slot;
      else atomicOr(&ctl->status, ST_CAPACITY);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < o.nsec) {
        const int ty = o.sec(k).type;
        const uint32_t ns = pick(ty, s0, s1, s2)++;
        const uint32_t at = pick(ty, q0, q1, q2)++;
        if (ns < a.cap && at < a.cap) {
          view_of<L, INSTR>(a, ty, 0).store(ns, make_secondary(t, o.sec(k)));
          (hn ? a.idx[ty][1] : a.idx[ty][0])[at] = ns;
        } else {
          atomicOr(&ctl->status, ST_CAPACITY);
        }
      }
    }
  }
}

// ---- per-type step kernel (host-loop and graph drivers) ----
template <int TYPE, int MODE, int L, bool INSTR, bool DENSE>
__global__ void __launch_bounds__(256) k_step(const __grid_constant__ Args a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tabs tb = stage_tables<TYPE == GAM, TYPE != GAM>(smem, a);
  const DevCtl* ctl = a.ctl;
  if (ctl->status != 0) return;
  const uint32_t it = ctl->iter;
  uint32_t n = ctl->cnt[it % 3][TYPE];
  n = n < a.cap ? n : a.cap;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t c = gw; c * 32u < n; c += nw) {
    const uint32_t i = c * 32u + lane;
    process_warp<TYPE, MODE, L, INSTR, DENSE>(a, tb, it, i, i < n, lane);
  }
}

#ifdef ET_HOST_TU
// ---- end of iteration (one thread): log counts, recycle the count slot, advance ----
__global__ void k_end_iteration(const __grid_constant__ Args a, cudaGraphConditionalHandle cond,
                                int use_cond) {
  DevCtl* c = a.ctl;
  const uint32_t it = c->iter;
  const uint32_t cur = it % 3, nxt = (it + 1) % 3;
  for (int t = 0; t < NTYPES; ++t) {
    c->steps[t] += c->cnt[cur][t];
    if (it < a.max_iters) a.counts_log[(size_t)it * 3 + t] = c->cnt[cur][t];
    const uint32_t fill = c->cnt[nxt][t];
    if (a.idx[0][0] == nullptr && fill > c->hwm[t]) c->hwm[t] = fill;  // dense: peak fill
  }
  if (it >= a.max_iters) c->status |= ST_ITER_LOG_FULL;
  for (int t = 0; t < NTYPES; ++t) c->cnt[cur][t] = 0;
  c->iter = it + 1;
  const uint32_t left = c->cnt[nxt][0] + c->cnt[nxt][1] + c->cnt[nxt][2];
  const bool stop = left == 0 || c->status != 0 || it + 1 >= c->stop_iter;
  c->done = stop ? 1u : 0u;
  if (use_cond) cudaGraphSetConditional(cond, stop ? 0u : 1u);
}
#endif

// ---- grid barrier for the persistent kernel (bounded wait) ----
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Returns false if this block gave up waiting (status ST_TIMEOUT is then set).
static __device__ bool grid_sync(DevCtl* c, uint32_t nblocks, unsigned long long timeout_ns,
                          uint32_t* snap_status) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> gen(c->bar_gen);
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> cnt(c->bar_count);
    cuda::atomic_ref<uint32_t, cuda::thread_scope_device> st(c->status);
    const uint32_t g = gen.load(cuda::memory_order_acquire);
    __threadfence();
    const uint32_t arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel);
    int ok = 1;
    if (arrived == nblocks - 1) {
      cnt.store(0u, cuda::memory_order_relaxed);
      *snap_status = st.load(cuda::memory_order_relaxed);
      gen.store(g + 1u, cuda::memory_order_release);
    } else {
      const unsigned long long t0 = global_ns();
      while (gen.load(cuda::memory_order_acquire) == g) {
        if (global_ns() - t0 > timeout_ns) {
          st.fetch_or(ST_TIMEOUT, cuda::memory_order_relaxed);
          ok = 0;
          break;
        }
        __nanosleep(40);
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ---- persistent kernel: all types, all iterations, one cooperative launch ----
// Warp chunks of 32 tracks are type-uniform: the iteration's index space is
// [ceil(n_e-/32) chunks of e-][chunks of e+][chunks of gamma].
template <int MODE, int L, bool INSTR, bool DENSE>
__global__ void __launch_bounds__(256) k_persistent(const __grid_constant__ Args a,
                                                    int fault_skip_block) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_n[3];
  __shared__ uint32_t s_stop;
  const Tabs tb = stage_tables<true, true>(smem, a);
  DevCtl* c = a.ctl;
  uint32_t* snap = &c->status_snap;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
  if ((int)blockIdx.x == fault_skip_block) return;  // host-side fault injection: never arrives
  uint32_t it = *(volatile uint32_t*)&c->iter;
  const uint32_t stop_iter = *(volatile uint32_t*)&c->stop_iter;
  uint32_t status0 = *(volatile uint32_t*)&c->status;
  bool first = true;
  for (;;) {
    if (threadIdx.x == 0) {
      const uint32_t cur = it % 3;
      for (int t = 0; t < 3; ++t) s_n[t] = __ldcg(&c->cnt[cur][t]);
      const uint32_t st = first ? status0 : *snap;
      s_stop = (s_n[0] + s_n[1] + s_n[2] == 0) || it >= stop_iter || st != 0;
    }
    __syncthreads();
    first = false;
    if (s_stop) break;
    const uint32_t n0 = min(s_n[0], a.cap), n1 = min(s_n[1], a.cap), n2 = min(s_n[2], a.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      for (int t = 0; t < 3; ++t) {
        c->cnt[(it + 2) % 3][t] = 0;
        c->steps[t] += s_n[t];
        if (it < a.max_iters) a.counts_log[(size_t)it * 3 + t] = s_n[t];
      }
      if (it >= a.max_iters) atomicOr(&c->status, ST_ITER_LOG_FULL);
    }
    const uint32_t w0 = (n0 + 31) / 32, w1 = (n1 + 31) / 32, w2 = (n2 + 31) / 32;
    const uint32_t wt = w0 + w1 + w2;
    for (uint32_t ch = gw; ch < wt; ch += nw) {
      if (ch < w0) {
        const uint32_t i = ch * 32u + lane;
        process_warp<EM, MODE, L, INSTR, DENSE>(a, tb, it, i, i < n0, lane);
      } else if (ch < w0 + w1) {
        const uint32_t i = (ch - w0) * 32u + lane;
        process_warp<EP, MODE, L, INSTR, DENSE>(a, tb, it, i, i < n1, lane);
      } else {
        const uint32_t i = (ch - w0 - w1) * 32u + lane;
        process_warp<GAM, MODE, L, INSTR, DENSE>(a, tb, it, i, i < n2, lane);
      }
    }
    if (!grid_sync(c, gridDim.x, a.timeout_ns, snap)) return;
    if (DENSE && blockIdx.x == 0 && threadIdx.x == 0) {
      for (int t = 0; t < 3; ++t) {
        const uint32_t fill = __ldcg(&c->cnt[(it + 1) % 3][t]);
        if (fill > c->hwm[t]) c->hwm[t] = fill;
      }
    }
    ++it;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    c->iter = it;
    const uint32_t cur = it % 3;
    for (int t = 0; t < 3; ++t) c->cnt[(it + 2) % 3][t] = 0;  // between iterations only cur is non-zero
    c->done = (__ldcg(&c->cnt[cur][0]) + __ldcg(&c->cnt[cur][1]) + __ldcg(&c->cnt[cur][2]) == 0);
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
  }
  const uint32_t packed = ok ? (1u << (10 * type)) : 0u;
  uint32_t q0, q1, q2;
  warp_reserve(packed, lane, c->cnt[cur], q0, q1, q2);
  if (DENSE) {
    if (ok) {
      const uint32_t at = pick(type, q0, q1, q2);
      if (at < a.cap) view_of<L, false>(a, type, (int)hc).store(at, t);
      else atomicOr(&c->status, ST_CAPACITY);
    }
  } else {
    uint32_t s0, s1, s2;
    warp_reserve(packed, lane, c->hwm, s0, s1, s2);
    if (ok) {
      const uint32_t slot = pick(type, s0, s1, s2);
      const uint32_t at = pick(type, q0, q1, q2);
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
