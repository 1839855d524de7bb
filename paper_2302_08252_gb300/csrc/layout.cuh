// Compile-time track layout layer (the paper's Sec. 3-4: LLAMA records,
// views and mappings AoS, SoA and AoSoA-n, switched "with a single line"),
// written as our own templates, with an instrumented accessor (Sec. 5:
// per-field read/write counts, FieldAccessCount/Trace, and per-byte access
// heatmaps).
//
// Mapping of leaf f (byte offset off_f, size s_f in the 64-byte record) of
// track i, for a buffer of `cap` slots:
//   AoS        base + 64 i + off_f
//   SoA        base + off_f cap + s_f i
//   AoSoA-N    base + 64 N (i / N) + off_f N + s_f (i mod N)
//   hot/cold   see Layout<LAYOUT_HOTCOLD>
// (AoSoA-N with N = 1 is AoS and with N = cap is SoA).  All leaves are 4 or
// 8 bytes and naturally aligned, so each access touches whole 4-byte words;
// the heatmap counts per 4-byte word, which equals the per-byte count of each
// of its bytes.
#pragma once

#include "common.cuh"

namespace et {

enum {
  LAYOUT_AOS = 0,
  LAYOUT_SOA = 1,
  LAYOUT_AOSOA32 = 2,
  LAYOUT_AOSOA64 = 3,
  LAYOUT_AOSOA8 = 4,
  LAYOUT_AOSOA16 = 5,
  LAYOUT_AOSOA128 = 6,
  LAYOUT_HOTCOLD = 7,
  N_LAYOUTS = 8
};

template <int L>
struct Layout;

template <>
struct Layout<LAYOUT_AOS> {
  static constexpr int lanes = 1;
  __device__ static size_t addr(uint32_t i, int f, uint32_t) {
    return (size_t)i * 64u + (size_t)leaf_off(f);
  }
};
template <>
struct Layout<LAYOUT_SOA> {
  static constexpr int lanes = 0;
  __device__ static size_t addr(uint32_t i, int f, uint32_t cap) {
    return (size_t)leaf_off(f) * cap + (size_t)leaf_size(f) * i;
  }
};
template <int N>
struct AoSoA {
  static constexpr int lanes = N;
  __device__ static size_t addr(uint32_t i, int f, uint32_t) {
    return (size_t)(i / N) * (64u * N) + (size_t)leaf_off(f) * N + (size_t)leaf_size(f) * (i % N);
  }
};
template <>
struct Layout<LAYOUT_AOSOA32> : AoSoA<32> {};
template <>
struct Layout<LAYOUT_AOSOA64> : AoSoA<64> {};
template <>
struct Layout<LAYOUT_AOSOA8> : AoSoA<8> {};
template <>
struct Layout<LAYOUT_AOSOA16> : AoSoA<16> {};
template <>
struct Layout<LAYOUT_AOSOA128> : AoSoA<128> {};
// Hot/cold split: the 52 bytes the step's decisions read (position, direction, energy,
// interaction lengths, id, event, step count, slab) as AoSoA-32, and the three fields
// that are only accumulated (time, track length, flags: byte offsets 52-63) as SoA
// arrays after them:
//   hot  leaf f   base + 52*32 (i / 32) + off_f 32 + s_f (i mod 32)
//   cold leaf f   base + 52 cap + (off_f - 52) cap + 4 i
// The buffer is still cap * 64 bytes; cap is a multiple of 32.
template <>
struct Layout<LAYOUT_HOTCOLD> {
  static constexpr int lanes = 32;
  static constexpr int kHot = 52;
  __device__ static size_t addr(uint32_t i, int f, uint32_t cap) {
    const int off = leaf_off(f);
    if (off < kHot)
      return (size_t)(i / 32u) * (kHot * 32u) + (size_t)off * 32u + (size_t)leaf_size(f) * (i % 32u);
    return (size_t)kHot * cap + (size_t)(off - kHot) * cap + 4u * (size_t)i;
  }
};

// Instrumentation sink: trace[type][leaf][0 read / 1 write] and a per-word heatmap.
struct Instr {
  unsigned long long* trace;
  uint32_t* heat;
  int type;
  __device__ void count(int f, int rw, const char* base, size_t a) const {
    if (trace) atomicAdd(&trace[((size_t)type * NLEAF + f) * 2 + rw], 1ull);
    if (heat) {
      const size_t w = a >> 2;
      atomicAdd(&heat[w], 1u);
      if (leaf_size(f) == 8) atomicAdd(&heat[w + 1], 1u);
    }
    (void)base;
  }
};

template <int L, bool INSTR>
struct View {
  char* base;
  uint32_t cap;
  Instr ins;

  template <typename T>
  __device__ T ld(uint32_t i, int f) const {
    const size_t a = Layout<L>::addr(i, f, cap);
    if (INSTR) ins.count(f, 0, base, a);
    return __ldcg(reinterpret_cast<const T*>(base + a));
  }
  template <typename T>
  __device__ void st(uint32_t i, int f, T v) const {
    const size_t a = Layout<L>::addr(i, f, cap);
    if (INSTR) ins.count(f, 1, base, a);
    *reinterpret_cast<T*>(base + a) = v;
  }

  __device__ Trk load(uint32_t i) const {
    Trk t;
    if (L == LAYOUT_AOS && !INSTR) {
      // one record = four 16-byte vector loads
      const uint4* p = reinterpret_cast<const uint4*>(base + (size_t)i * 64u);
      const uint4 a = __ldcg(p), b = __ldcg(p + 1), c = __ldcg(p + 2), d = __ldcg(p + 3);
      t.x = __uint_as_float(a.x); t.y = __uint_as_float(a.y);
      t.z = __uint_as_float(a.z); t.dx = __uint_as_float(a.w);
      t.dy = __uint_as_float(b.x); t.dz = __uint_as_float(b.y);
      t.e = __uint_as_float(b.z); t.nia = __uint_as_float(b.w);
      t.id = (uint64_t)c.x | ((uint64_t)c.y << 32);
      t.event = c.z; t.step = c.w;
      t.slab = (int32_t)d.x; t.time = __uint_as_float(d.y);
      t.len = __uint_as_float(d.z); t.flags = d.w;
      return t;
    }
    t.x = ld<float>(i, F_X); t.y = ld<float>(i, F_Y); t.z = ld<float>(i, F_Z);
    t.dx = ld<float>(i, F_DX); t.dy = ld<float>(i, F_DY); t.dz = ld<float>(i, F_DZ);
    t.e = ld<float>(i, F_E); t.nia = ld<float>(i, F_NIA);
    t.id = ld<unsigned long long>(i, F_ID);
    t.event = ld<uint32_t>(i, F_EVENT); t.step = ld<uint32_t>(i, F_STEP);
    t.slab = ld<int32_t>(i, F_SLAB); t.time = ld<float>(i, F_TIME);
    t.len = ld<float>(i, F_LEN); t.flags = ld<uint32_t>(i, F_FLAGS);
    return t;
  }

  __device__ void store(uint32_t i, const Trk& t) const {
    if (L == LAYOUT_AOS && !INSTR) {
      uint4* p = reinterpret_cast<uint4*>(base + (size_t)i * 64u);
      p[0] = make_uint4(__float_as_uint(t.x), __float_as_uint(t.y), __float_as_uint(t.z),
                        __float_as_uint(t.dx));
      p[1] = make_uint4(__float_as_uint(t.dy), __float_as_uint(t.dz), __float_as_uint(t.e),
                        __float_as_uint(t.nia));
      p[2] = make_uint4((uint32_t)t.id, (uint32_t)(t.id >> 32), t.event, t.step);
      p[3] = make_uint4((uint32_t)t.slab, __float_as_uint(t.time), __float_as_uint(t.len),
                        t.flags);
      return;
    }
    store_leaves(i, t, D_ALL);
  }

  // Write only the leaves named in `dirty` (sparse in-place update).
  __device__ void store_leaves(uint32_t i, const Trk& t, uint32_t dirty) const {
    if (dirty & (1u << F_X)) st<float>(i, F_X, t.x);
    if (dirty & (1u << F_Y)) st<float>(i, F_Y, t.y);
    if (dirty & (1u << F_Z)) st<float>(i, F_Z, t.z);
    if (dirty & (1u << F_DX)) st<float>(i, F_DX, t.dx);
    if (dirty & (1u << F_DY)) st<float>(i, F_DY, t.dy);
    if (dirty & (1u << F_DZ)) st<float>(i, F_DZ, t.dz);
    if (dirty & (1u << F_E)) st<float>(i, F_E, t.e);
    if (dirty & (1u << F_NIA)) st<float>(i, F_NIA, t.nia);
    if (dirty & (1u << F_ID)) st<unsigned long long>(i, F_ID, (unsigned long long)t.id);
    if (dirty & (1u << F_EVENT)) st<uint32_t>(i, F_EVENT, t.event);
    if (dirty & (1u << F_STEP)) st<uint32_t>(i, F_STEP, t.step);
    if (dirty & (1u << F_SLAB)) st<int32_t>(i, F_SLAB, t.slab);
    if (dirty & (1u << F_TIME)) st<float>(i, F_TIME, t.time);
    if (dirty & (1u << F_LEN)) st<float>(i, F_LEN, t.len);
    if (dirty & (1u << F_FLAGS)) st<uint32_t>(i, F_FLAGS, t.flags);
  }
};

}  // namespace et
