// All-FP64 GPU build of the transport (the precision comparison of the batched
// workload): the same toy model with every state variable, table and operation in FP64
// and libm-accuracy log/exp/sincos -- the GPU counterpart of the oracle's FP64
// reference mode, against which the FP32-stepping path's per-layer error is stated.
//
// This is a plain path, not a tuned one: 128-byte AoS records in a dense double
// buffer, one thread per track, warp-aggregated slot allocation, FP64 atomics for
// deposits, iterations driven from the host (counts read back each time).  FP64
// arithmetic runs at a small fraction of the FP32 rate on this GPU.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "et.h"
#include "kernels.cuh"

namespace et64 {

using et::FULL;
using et::warp_reserve;
using et::take;
using et::sel3;
using et::cw;

constexpr int NB = et::NBINS;

struct alignas(16) Trk {
  double x, y, z, dx, dy, dz, e, nia, time, len;
  unsigned long long id;
  uint32_t event, step;
  int32_t slab;
  uint32_t flags;
  uint32_t pad[6];
};
static_assert(sizeof(Trk) == 128, "128-byte record");

struct Ctl {
  uint32_t cnt[3][et::CTL_LINE];  // word cw(t), rows by iteration % 3 as in the FP32 path
  uint32_t iter, status;
  unsigned long long steps[3], secondaries[3];
};

struct Args {
  Trk* trk[3][2];
  uint32_t cap;
  Ctl* ctl;
  const double* sig;   // [n_mat][5][257]
  const double* planes;
  const uint8_t* mat;
  double dedx[4];
  double half, log_emin, inv_dlog;
  int n_slabs, n_mat;
  uint32_t seed;
  double* score;       // [max_events][n_slabs]
  double* ledger;      // [max_events][5]
  uint32_t max_events;
};

constexpr double MC2 = 0.51099895, TWO_MC2 = 1.0219979, KC = 0.01;
constexpr double C_LIGHT = 299.792458;

__device__ __forceinline__ double u01d(uint32_t x) {
  return (double)((x >> 8) + 1u) * 0x1p-24;  // the same 24-bit values as the FP32 path
}

// sin and cos of 2 pi u, the angle formed in FP64 first (as the FP64 reference does).
__device__ __forceinline__ void sincos2pi(double u, double& s, double& c) {
  sincos(2.0 * 3.14159265358979323846 * u, &s, &c);
}

__device__ __forceinline__ double interp(const Args& a, int m, int tab, int i, double f) {
  const double* t = a.sig + ((size_t)m * 5 + tab) * (NB + 1);
  return t[i] + f * (t[i + 1] - t[i]);
}

struct Out {
  int alive, death, nsec, slab_cont;
  int type[3];
  double e[3], dx[3], dy[3], dz[3];
  double dep, cut, esc, mc, mcr;
};

__device__ void add_sec(Out& o, int ty, double e, double dx, double dy, double dz) {
  const int k = o.nsec++;
  o.type[k] = ty;
  o.e[k] = e;
  o.dx[k] = dx;
  o.dy[k] = dy;
  o.dz[k] = dz;
}

__device__ void annihilate(Out& o, const Trk& t, uint32_t pstep, uint32_t seed) {
  const uint4 r = et::philox((uint32_t)t.id, (uint32_t)(t.id >> 32), pstep, 65u, seed, t.event);
  const double cost = 2.0 * u01d(r.x) - 1.0;
  const double sint = sqrt((1.0 - cost) * (1.0 + cost));
  double sp, cp;
  sincos2pi(u01d(r.y), sp, cp);
  add_sec(o, et::GAM, MC2, sint * cp, sint * sp, cost);
  add_sec(o, et::GAM, MC2, -sint * cp, -sint * sp, -cost);
  o.mcr = MC2 + MC2;
}

__device__ void rotate(double ux, double uy, double uz, double px, double py, double pz,
                       double& nx, double& ny, double& nz) {
  double up = ux * ux + uy * uy;
  if (up > 0.0) {
    up = sqrt(up);
    nx = (ux * uz * px - uy * py) / up + ux * pz;
    ny = (uy * uz * px + ux * py) / up + uy * pz;
    nz = uz * pz - up * px;
  } else if (uz < 0.0) {
    nx = -px; ny = py; nz = -pz;
  } else {
    nx = px; ny = py; nz = pz;
  }
}

// One step of the toy model in FP64 (same operation sequence as the FP32 model).
__device__ void step(const Args& a, int type, Trk& t, Out& o) {
  const bool charged = type != et::GAM;
  o.alive = 1; o.death = 0; o.nsec = 0;
  o.cut = o.esc = o.mc = o.mcr = 0.0;
  const uint32_t pstep = t.step;
  const uint4 r0 = et::philox((uint32_t)t.id, (uint32_t)(t.id >> 32), pstep, 0u, a.seed, t.event);
  const double E = t.e;
  if (t.nia < 0.0) t.nia = -log(u01d(r0.x));
  const int s0 = t.slab, m = a.mat[s0];
  const double lx = (log(E) - a.log_emin) * a.inv_dlog;
  int i = (int)floor(lx);
  i = i < 0 ? 0 : (i > NB - 1 ? NB - 1 : i);
  const double f = lx - (double)i;
  const double sig = charged ? interp(a, m, 4, i, f) : interp(a, m, 3, i, f);
  const double s_phys = sig > 0.0 ? t.nia / sig : __longlong_as_double(0x7ff0000000000000ll);
  const double INF = __longlong_as_double(0x7ff0000000000000ll);
  double zpl = 0.0, sz, sx, sy;
  if (t.dz > 0) { zpl = a.planes[s0 + 1]; sz = (zpl - t.z) / t.dz; }
  else if (t.dz < 0) { zpl = a.planes[s0]; sz = (zpl - t.z) / t.dz; }
  else sz = INF;
  if (sz < 0) sz = 0;
  if (t.dx > 0) sx = (a.half - t.x) / t.dx; else if (t.dx < 0) sx = (-a.half - t.x) / t.dx; else sx = INF;
  if (sx < 0) sx = 0;
  if (t.dy > 0) sy = (a.half - t.y) / t.dy; else if (t.dy < 0) sy = (-a.half - t.y) / t.dy; else sy = INF;
  if (sy < 0) sy = 0;
  double s = sz;
  int lim = et::LIM_Z;
  if (sx < s) { s = sx; lim = et::LIM_X; }
  if (sy < s) { s = sy; lim = et::LIM_Y; }
  if (charged) {
    const double sl = E > 1.0 ? (0.2 * E) / a.dedx[m] : E / a.dedx[m];
    if (sl < s) { s = sl; lim = et::LIM_LOSS; }
  }
  if (s_phys < s) { s = s_phys; lim = et::LIM_PHYS; }
  t.x = t.x + s * t.dx;
  t.y = t.y + s * t.dy;
  t.z = lim == et::LIM_Z ? zpl : t.z + s * t.dz;
  if (charged) t.time = t.time + s / (sqrt(E * (E + TWO_MC2)) / (E + MC2) * C_LIGHT);
  else t.time = t.time + s / C_LIGHT;
  t.len = t.len + s;
  if (lim == et::LIM_PHYS) t.nia = -1.0;
  else { t.nia = t.nia - s * sig; if (t.nia < 0) t.nia = 0.0; }
  double eout = E;
  if (charged) {
    const double de = (lim == et::LIM_LOSS && E <= 1.0) ? E : a.dedx[m] * s;
    eout = E - de;
    if (eout < 0) eout = 0.0;
  }
  t.e = eout;
  o.slab_cont = s0;
  bool escaped = false;
  if (lim == et::LIM_Z) {
    const int s1 = t.dz > 0 ? s0 + 1 : s0 - 1;
    if (s1 < 0 || s1 >= a.n_slabs) escaped = true; else t.slab = s1;
  } else if (lim == et::LIM_X || lim == et::LIM_Y) {
    escaped = true;
  }
  int proc = 0;
  if (escaped) {
    o.esc = eout; o.alive = 0; o.death = et::DEATH_ESCAPE;
  } else if (charged && eout < KC) {
    o.cut += eout; o.alive = 0; o.death = et::DEATH_CUT;
    if (type == et::EP) annihilate(o, t, pstep, a.seed);
  } else if (lim == et::LIM_PHYS) {
    if (!charged) {
      const double sc = interp(a, m, 0, i, f), sp = interp(a, m, 1, i, f);
      const double r = u01d(r0.y) * sig;
      if (r < sc) {
        proc = et::PROC_COMPTON;
        const double k = E / MC2, eps0 = 1.0 / (1.0 + 2.0 * k), eps0sq = eps0 * eps0;
        const double a1 = -log(eps0), a2 = 0.5 * (1.0 - eps0sq), p1 = a1 / (a1 + a2);
        double eps = 1.0, epssq = 1.0, onecost = 0.0, sint2 = 0.0;
        for (int j = 0; j < 64; ++j) {
          const uint4 rj = et::philox((uint32_t)t.id, (uint32_t)(t.id >> 32), pstep, 1u + j, a.seed, t.event);
          const double ua = u01d(rj.x), ub = u01d(rj.y), uc = u01d(rj.z);
          if (p1 > ua) { eps = exp(-(a1 * ub)); epssq = eps * eps; }
          else { epssq = eps0sq + (1.0 - eps0sq) * ub; eps = sqrt(epssq); }
          onecost = (1.0 - eps) / (k * eps);
          sint2 = onecost * (2.0 - onecost);
          if (1.0 - (eps * sint2) / (1.0 + epssq) >= uc) break;
        }
        if (sint2 < 0) sint2 = 0.0;
        const double cost = 1.0 - onecost, sint = sqrt(sint2);
        double sphi, cphi;
        sincos2pi(u01d(r0.w), sphi, cphi);
        double nx, ny, nz;
        rotate(t.dx, t.dy, t.dz, sint * cphi, sint * sphi, cost, nx, ny, nz);
        const double e1 = eps * E, te = E - e1;
        if (te >= KC) {
          const double px = E * t.dx - e1 * nx, py = E * t.dy - e1 * ny, pz = E * t.dz - e1 * nz;
          const double pn = sqrt(px * px + py * py + pz * pz);
          add_sec(o, et::EM, te, px / pn, py / pn, pz / pn);
        } else {
          o.cut += te;
        }
        t.dx = nx; t.dy = ny; t.dz = nz; t.e = e1;
        if (!(e1 >= KC)) { o.cut += e1; o.alive = 0; o.death = et::DEATH_CUT; }
      } else if (r < sc + sp && E > TWO_MC2) {
        proc = et::PROC_PAIR;
        const double avail = E - TWO_MC2, em = u01d(r0.z) * avail, ep = avail - em;
        o.mc = (E - em) - ep;
        if (em >= KC) add_sec(o, et::EM, em, t.dx, t.dy, t.dz); else o.cut += em;
        if (ep >= KC) add_sec(o, et::EP, ep, t.dx, t.dy, t.dz);
        else { o.cut += ep; annihilate(o, t, pstep, a.seed); }
        o.alive = 0; o.death = et::DEATH_ABSORB;
      } else {
        proc = et::PROC_PHOT;
        if (E >= KC) add_sec(o, et::EM, E, t.dx, t.dy, t.dz); else o.cut += E;
        o.alive = 0; o.death = et::DEATH_ABSORB;
      }
    } else {
      proc = et::PROC_BREM;
      if (eout > KC) {
        double kk = KC * exp(u01d(r0.z) * log(eout / KC));
        if (kk < KC) kk = KC;
        if (kk > eout) kk = eout;
        add_sec(o, et::GAM, kk, t.dx, t.dy, t.dz);
        const double t2 = eout - kk;
        t.e = t2;
        if (t2 < KC) {
          o.cut += t2; o.alive = 0; o.death = et::DEATH_CUT;
          if (type == et::EP) annihilate(o, t, pstep, a.seed);
        }
      }
    }
  }
  double dep = E + o.mcr;
  if (o.alive) dep -= t.e;
  for (int k = 0; k < o.nsec; ++k) dep -= o.e[k];
  dep = dep - o.esc - o.cut - o.mc;
  o.dep = dep;
  t.flags = (uint32_t)lim | ((uint32_t)proc << 4);
  t.step = pstep + 1;
}

__global__ void __launch_bounds__(256) k_step(const __grid_constant__ Args a, int type) {
  const uint32_t it = a.ctl->iter, cur = it % 3, nxt = (it + 1) % 3, hc = it & 1u, hn = hc ^ 1u;
  uint32_t n = a.ctl->cnt[cur][cw(type)];
  n = n < a.cap ? n : a.cap;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (uint32_t c = gw; c * 32u < n; c += nw) {
    const uint32_t i = c * 32u + lane;
    const bool valid = i < n;
    Trk t;
    Out o;
    o.alive = 0; o.nsec = 0;
    if (valid) {
      t = a.trk[type][hc][i];
      step(a, type, t, o);
      const size_t ev = t.event;
      if (o.dep != 0.0) atomicAdd(&a.score[ev * a.n_slabs + o.slab_cont], o.dep);
      if (o.cut != 0.0) { atomicAdd(&a.score[ev * a.n_slabs + t.slab], o.cut); atomicAdd(&a.ledger[ev * 5 + 1], o.cut); }
      if (o.esc != 0.0) atomicAdd(&a.ledger[ev * 5 + 2], o.esc);
      if (o.mcr != 0.0) atomicAdd(&a.ledger[ev * 5 + 3], o.mcr);
      if (o.mc != 0.0) atomicAdd(&a.ledger[ev * 5 + 4], o.mc);
    }
    uint32_t packed = (valid && o.alive) ? (1u << (10 * type)) : 0u, nsec_packed = 0;
    for (int k = 0; k < o.nsec; ++k) nsec_packed += 1u << (10 * o.type[k]);
    packed += nsec_packed;
    for (int ty = 0; ty < 3; ++ty) {
      const uint32_t cnt = (nsec_packed >> (10 * ty)) & 1023u;
      const uint32_t tot = __reduce_add_sync(FULL, cnt);
      if (lane == 0 && tot) atomicAdd(&a.ctl->secondaries[ty], (unsigned long long)tot);
    }
    uint32_t q0, q1, q2;
    warp_reserve(packed, lane, a.ctl->cnt[nxt], q0, q1, q2);
    if (valid && o.alive) {
      const uint32_t at = take(type, q0, q1, q2);
      if (at < a.cap) a.trk[type][hn][at] = t; else atomicOr(&a.ctl->status, 1u);
    }
    for (int k = 0; k < o.nsec; ++k) {
      const int ty = o.type[k];
      const uint32_t at = take(ty, q0, q1, q2);
      if (at >= a.cap) { atomicOr(&a.ctl->status, 1u); continue; }
      Trk r = t;
      r.dx = o.dx[k]; r.dy = o.dy[k]; r.dz = o.dz[k]; r.e = o.e[k];
      r.nia = -1.0; r.id = et::secondary_id(t.id, t.step - 1u, (uint32_t)k);
      r.step = 0; r.len = 0.0; r.flags = 0;
      a.trk[ty][hn][at] = r;
    }
  }
}

__global__ void k_end(Ctl* c) {
  const uint32_t it = c->iter, cur = it % 3;
  for (int t = 0; t < 3; ++t) {
    c->steps[t] += c->cnt[cur][cw(t)];
    c->cnt[cur][cw(t)] = 0;
  }
  c->iter = it + 1;
}

}  // namespace et64

extern "C" et_status et_run_fp64(uint32_t n_slabs, const double* thickness_mm,
                                 const uint8_t* material, double half_xy_mm, uint32_t n_materials,
                                 double log_emin, double inv_dlog, const double* sigma,
                                 const double* dedx, const et_primary* primaries, size_t n,
                                 uint64_t seed, uint32_t n_events, uint32_t capacity_log2,
                                 double* score_out, double* ledger_out, uint64_t* steps_out,
                                 uint64_t* iterations_out) {
  using namespace et64;
  if (n_slabs < 1 || n_slabs > (uint32_t)et::MAX_SLABS || n_materials < 1 || n_materials > 4 ||
      !thickness_mm || !material || !sigma || !dedx || (n && !primaries) || n_events == 0 ||
      capacity_log2 < 6 || capacity_log2 > 26 || !score_out || (seed >> 32) != 0)
    return ET_ERR_INVALID;
  const uint32_t cap = 1u << capacity_log2;
  if (n > cap) return ET_ERR_CAPACITY;
  std::vector<double> planes(n_slabs + 1);
  planes[0] = 0.0;
  for (uint32_t s = 0; s < n_slabs; ++s) {
    if (material[s] >= n_materials) return ET_ERR_INVALID;
    planes[s + 1] = planes[s] + thickness_mm[s];
  }
  std::vector<Trk> init(n);
  for (size_t i = 0; i < n; ++i) {
    const et_primary& p = primaries[i];
    if (p.type > 2 || p.event >= n_events || !(p.ekin > 0.0f)) return ET_ERR_INVALID;
    Trk t;
    memset(&t, 0, sizeof t);
    t.x = p.pos[0]; t.y = p.pos[1]; t.z = p.pos[2];
    t.dx = p.dir[0]; t.dy = p.dir[1]; t.dz = p.dir[2];
    t.e = p.ekin; t.nia = -1.0; t.id = p.id; t.event = p.event;
    int s = 0;
    if (!(t.z >= planes[0] && t.z < planes[n_slabs])) return ET_ERR_INVALID;
    while (s + 1 < (int)n_slabs && !(t.z < planes[s + 1])) ++s;
    t.slab = s;
    init[i] = t;
  }
  // device memory (this plain path allocates per call)
  std::vector<void*> allocs;
  auto alloc = [&](size_t b) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, b ? b : 16) != cudaSuccess) return nullptr;
    allocs.push_back(p);
    return p;
  };
  auto cleanup = [&](et_status s) {
    for (void* p : allocs) cudaFree(p);
    (void)cudaGetLastError();
    return s;
  };
  Args a;
  memset(&a, 0, sizeof a);
  for (int t = 0; t < 3; ++t)
    for (int h = 0; h < 2; ++h)
      if (!(a.trk[t][h] = (Trk*)alloc((size_t)cap * sizeof(Trk)))) return cleanup(ET_ERR_NOMEM);
  Ctl* ctl = (Ctl*)alloc(sizeof(Ctl));
  double* sig = (double*)alloc((size_t)n_materials * 5 * (et::NBINS + 1) * 8);
  double* pl = (double*)alloc(planes.size() * 8);
  uint8_t* mt = (uint8_t*)alloc(n_slabs);
  double* score = (double*)alloc((size_t)n_events * n_slabs * 8);
  double* ledger = (double*)alloc((size_t)n_events * 5 * 8);
  if (!ctl || !sig || !pl || !mt || !score || !ledger) return cleanup(ET_ERR_NOMEM);
  Ctl h;
  memset(&h, 0, sizeof h);
  uint32_t per_type[3] = {0, 0, 0};
  std::vector<Trk> by_type[3];
  for (const Trk& t : init) {
    const int ty = (int)primaries[&t - init.data()].type;
    by_type[ty].push_back(t);
    per_type[ty]++;
  }
  std::vector<double> led(n_events * 5, 0.0);
  for (size_t i = 0; i < n; ++i) led[primaries[i].event * 5] += (double)primaries[i].ekin;
  for (int t = 0; t < 3; ++t) {
    h.cnt[0][cw(t)] = per_type[t];
    if (per_type[t])
      if (cudaMemcpy(a.trk[t][0], by_type[t].data(), per_type[t] * sizeof(Trk), cudaMemcpyHostToDevice) != cudaSuccess)
        return cleanup(ET_ERR_CUDA);
  }
  if (cudaMemcpy(ctl, &h, sizeof h, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(sig, sigma, (size_t)n_materials * 5 * (et::NBINS + 1) * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(pl, planes.data(), planes.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(mt, material, n_slabs, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(score, 0, (size_t)n_events * n_slabs * 8) != cudaSuccess ||
      cudaMemcpy(ledger, led.data(), led.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return cleanup(ET_ERR_CUDA);
  a.cap = cap; a.ctl = ctl; a.sig = sig; a.planes = pl; a.mat = mt;
  for (uint32_t m = 0; m < n_materials; ++m) a.dedx[m] = dedx[m];
  a.half = half_xy_mm; a.log_emin = log_emin; a.inv_dlog = inv_dlog;
  a.n_slabs = (int)n_slabs; a.n_mat = (int)n_materials; a.seed = (uint32_t)seed;
  a.score = score; a.ledger = ledger; a.max_events = n_events;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
  uint64_t iters = 0;
  for (;;) {
    if (cudaMemcpy(&h, ctl, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) return cleanup(ET_ERR_CUDA);
    if (h.status) return cleanup(ET_ERR_CAPACITY);
    const uint32_t cur = h.iter % 3;
    const uint32_t ns[3] = {h.cnt[cur][cw(0)], h.cnt[cur][cw(1)], h.cnt[cur][cw(2)]};
    if (ns[0] + ns[1] + ns[2] == 0) break;
    if (h.iter >= (1u << 16)) return cleanup(ET_ERR_TIMEOUT);
    for (int t = 0; t < 3; ++t) {
      if (!ns[t]) continue;
      int grid = (int)((ns[t] + 255) / 256);
      if (grid > sms * 8) grid = sms * 8;
      k_step<<<grid, 256>>>(a, t);
    }
    k_end<<<1, 1>>>(ctl);
    ++iters;
  }
  if (cudaGetLastError() != cudaSuccess) return cleanup(ET_ERR_CUDA);
  if (cudaMemcpy(score_out, score, (size_t)n_events * n_slabs * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cleanup(ET_ERR_CUDA);
  if (ledger_out && cudaMemcpy(ledger_out, ledger, (size_t)n_events * 5 * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return cleanup(ET_ERR_CUDA);
  if (steps_out) *steps_out = h.steps[0] + h.steps[1] + h.steps[2];
  if (iterations_out) *iterations_out = iters;
  return cleanup(ET_OK);
}
