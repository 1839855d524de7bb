// Host side of the C ABI declared in include/et.h: context and device-memory
// management, geometry and table upload, injection, the three iteration
// drivers (host loop, CUDA graph with a device-side WHILE condition,
// persistent cooperative kernel) and the read-back calls.
//
// The iteration is the paper's transport iteration (Sec. 2): all active tracks
// of all types take one step; the device control block keeps the per-type
// counts triple-buffered (current / next / recycled) so that no host round
// trip is needed between iterations except in the host-loop driver, which
// mirrors the plain AdePT loop (launch per type, read counts back).
#define ET_HOST_TU
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <string>
#include <unordered_map>
#include <vector>

#include "et.h"
#include "et_debug.h"
#include "kernels.cuh"
#include "registry.h"

using namespace et;

static_assert(sizeof(et_primary) == 48, "primary record is 48 bytes");
static_assert(sizeof(Primary) == 48, "device primary record is 48 bytes");
static_assert(sizeof(et_idrec) == sizeof(IdRec), "id record layout");

struct EventPair {
  cudaEvent_t a, b;
};

// The native serving loop's state (et_serve_*), created on first use.
struct ServeReq {
  std::vector<Primary> p;
  uint32_t event;
  uint32_t reserve[3];
};

struct ServeState {
  std::deque<ServeReq> pending;
  std::unordered_map<uint32_t, std::array<uint32_t, 3>> inflight;  // event -> reserve
  uint64_t reserved[3] = {0, 0, 0};
  uint32_t max_out = 0;
  uint32_t* d_cursor = nullptr;  // collection cursor in the completion ring
  uint32_t* d_events = nullptr;  // [max_out + 1]
  double* d_rows = nullptr;      // [max_out][n_slabs + 5]
  uint32_t* h_events[2] = {nullptr, nullptr};  // pinned, one per round parity
  double* h_rows[2] = {nullptr, nullptr};
  DevCtl* h_ctl[2] = {nullptr, nullptr};
  uint32_t* h_rel[2] = {nullptr, nullptr};     // pinned iteration limits of the rounds
  cudaEvent_t ev[2] = {nullptr, nullptr};
  uint64_t issued = 0, delivered = 0;          // rounds
  uint64_t steps_seen = 0;                     // cumulative steps at the last delivery
  uint64_t last_pop = 0;                       // active tracks at the last delivered round's end
  std::vector<Primary> batch;
};

static void serve_free(ServeState* s) {
  if (!s) return;
  for (int k = 0; k < 2; ++k) {
    if (s->h_events[k]) cudaFreeHost(s->h_events[k]);
    if (s->h_rows[k]) cudaFreeHost(s->h_rows[k]);
    if (s->h_ctl[k]) cudaFreeHost(s->h_ctl[k]);
    if (s->h_rel[k]) cudaFreeHost(s->h_rel[k]);
    if (s->ev[k]) cudaEventDestroy(s->ev[k]);
  }
  delete s;
}


struct et_ctx {
  et_config cfg{};
  std::string err;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  uint32_t cap = 0;
  bool dense = true;
  std::vector<void*> allocs;
  KernelSet ks{};
  Args args{};
  DevCtl* d_ctl = nullptr;
  DevCtl* h_ctl = nullptr;  // pinned
  uint32_t* h_stop = nullptr;  // pinned scratch for stop_iter uploads
  double* h_ledger = nullptr;  // pinned staging of the ledgers (allocated on first read)
  bool have_geom = false, have_tables = false, have_msc = false;
  std::vector<float> planes;
  std::vector<uint8_t> mat;
  Primary* d_stage = nullptr;
  size_t stage_cap = 0;
  Primary* h_stage = nullptr;  // pinned host staging of et_inject's primaries
  size_t h_stage_cap = 0;
  cudaEvent_t h_stage_done = nullptr;  // the last copy out of h_stage
  bool h_stage_pending = false;
  int block = 256;
  int grid_fixed[3] = {0, 0, 0};  // step kernels in the graph driver (grid-stride)
  int grid_tr[3] = {0, 0, 0}, grid_ia[3] = {0, 0, 0};  // split form: transport, interaction
  int grid_persistent = 0;
  size_t smem_all = 0, smem_tab = 0;
  size_t smem_step[3] = {0, 0, 0};  // per-type step kernels: the e+- kernels queue nothing
  bool split = false;
  ServeState* serve = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph = nullptr;
  bool timing = false;
  std::vector<EventPair> evpool;
  size_t ev_used = 0;
  double ms_acc = 0.0;
  uint64_t timed = 0;
  uint64_t launches = 0;
  int fault_skip_block = -1;  // fault injection for the persistent driver's barrier (tests)
  unsigned long long* d_iter_ns = nullptr;
  uint32_t done_read = 0;     // serving: completion ring entries already returned
};

static et_status fail(et_ctx* c, et_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CUDA_TRY(c, call)                                                              \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail((c), ET_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

static void* dalloc(et_ctx* c, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  if (c->cfg.alloc) {
    p = c->cfg.alloc(bytes, c->cfg.cuda_stream, c->cfg.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    (void)cudaGetLastError();
    p = nullptr;
  }
  if (p) c->allocs.push_back(p);
  return p;
}

static void register_kernels(int mode, int layout, KernelSet* ks) {
  static void (*const fns[2][N_LAYOUTS])(KernelSet*) = {
      {et_register_kernels_0_0, et_register_kernels_0_1, et_register_kernels_0_2,
       et_register_kernels_0_3, et_register_kernels_0_4, et_register_kernels_0_5,
       et_register_kernels_0_6, et_register_kernels_0_7},
      {et_register_kernels_1_0, et_register_kernels_1_1, et_register_kernels_1_2,
       et_register_kernels_1_3, et_register_kernels_1_4, et_register_kernels_1_5,
       et_register_kernels_1_6, et_register_kernels_1_7}};
  fns[mode][layout](ks);
}

// ---- timing of step-kernel launches ----
static EventPair* timing_begin(et_ctx* c) {
  if (!c->timing) return nullptr;
  if (c->ev_used == c->evpool.size()) {
    EventPair p;
    if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) return nullptr;
    c->evpool.push_back(p);
  }
  EventPair* p = &c->evpool[c->ev_used++];
  cudaEventRecord(p->a, c->stream);
  return p;
}
static void timing_end(et_ctx* c, EventPair* p) {
  if (p) cudaEventRecord(p->b, c->stream);
}
// after a stream synchronize: accumulate and recycle the events
static void timing_collect(et_ctx* c) {
  for (size_t i = 0; i < c->ev_used; ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, c->evpool[i].a, c->evpool[i].b) == cudaSuccess) {
      c->ms_acc += ms;
      c->timed += 1;
    }
  }
  c->ev_used = 0;
}

static et_status sync_ctl(et_ctx* c) {
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  timing_collect(c);
  const uint32_t st = c->h_ctl->status;
  if (st & ST_TIMEOUT) return fail(c, ET_ERR_TIMEOUT, "device wait timed out (status 0x%x)", st);
  if (st & ST_CAPACITY)
    return fail(c, ET_ERR_CAPACITY, "track buffer capacity %u exceeded (status 0x%x)", c->cap, st);
  if (st & ST_LOG_FULL) return fail(c, ET_ERR_CAPACITY, "id log full (status 0x%x)", st);
  if (st & ST_BAD_PRIMARY) return fail(c, ET_ERR_INVALID, "invalid device-side primary (skipped)");
  if (st & ST_ITER_LOG_FULL)
    return fail(c, ET_ERR_CAPACITY, "iteration log full (max_iters %u)", c->cfg.max_iters);
  return ET_OK;
}

static et_status launch(et_ctx* c, const void* fn, int grid, int block, size_t smem, void** params) {
  CUDA_TRY(c, cudaLaunchKernel(fn, dim3(grid), dim3(block), params, smem, c->stream));
  c->launches += 1;
  return ET_OK;
}

// Serving: append the events that have ended since the last scan to the completion ring
// (mark the events of the current tracks, then report the injected ones left unmarked).
static et_status scan_done(et_ctx* c) {
  void* params[] = {(void*)&c->args};
  et_status s = launch(c, c->ks.mark_present[c->dense ? 1 : 0], c->num_sms * 4, 256, 0, params);
  if (s != ET_OK) return s;
  const int grid = (int)((c->cfg.max_events + 255u) / 256u);
  return launch(c, (const void*)k_scan_done, grid < 152 ? grid : 152, 256, 0, params);
}

// One thread per input: the primitives exactly as the step kernels use them.
__global__ void k_debug_eval(int what, const void* in, void* out, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (what == ET_EVAL_PHILOX) {
    const uint32_t* c = static_cast<const uint32_t*>(in) + 6 * i;
    const uint4 r = philox(c[0], c[1], c[2], c[3], c[4], c[5]);
    uint32_t* o = static_cast<uint32_t*>(out) + 4 * i;
    o[0] = r.x; o[1] = r.y; o[2] = r.z; o[3] = r.w;
  } else if (what == ET_EVAL_U01) {
    static_cast<float*>(out)[i] = u01(static_cast<const uint32_t*>(in)[i]);
  } else if (what == ET_EVAL_LOG) {
    static_cast<float*>(out)[i] = s_log(static_cast<const float*>(in)[i]);
  } else if (what == ET_EVAL_EXP) {
    static_cast<float*>(out)[i] = s_exp(static_cast<const float*>(in)[i]);
  } else {
    float sn, cs;
    s_sincos2pi(static_cast<const float*>(in)[i], &sn, &cs);
    static_cast<float*>(out)[2 * i] = sn;
    static_cast<float*>(out)[2 * i + 1] = cs;
  }
}

extern "C" {

const char* et_last_error(const et_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

et_status et_create(const et_config* cfg, et_ctx** out) {
  if (!out) return ET_ERR_INVALID;
  *out = nullptr;
  if (!cfg) return ET_ERR_INVALID;
  et_config k = *cfg;
  if (k.block_size == 0) k.block_size = 256;
  if (k.max_iters == 0) k.max_iters = 1u << 16;
  if (k.capacity_log2 < 6 || k.capacity_log2 > 28 || (k.form != 0 && k.form != 1) ||
      k.layout < 0 || k.layout >= N_LAYOUTS || (k.mode != 0 && k.mode != 1) || k.driver < 0 ||
      (k.layout == LAYOUT_AOSOA128 && k.capacity_log2 < 7) ||
      k.driver > 3 || k.block_size < 64 || k.block_size > 256 || (k.block_size % 32) != 0 ||
      k.max_events == 0 || (k.instrument && k.mode != ET_MODE_STRICT) || (k.seed >> 32) != 0 ||
      ((k.alloc == nullptr) != (k.free == nullptr)) ||
      (k.split_interactions != 0 && k.split_interactions != 1) ||
      (k.split_interactions && (k.driver == ET_DRIVER_PERSISTENT || k.instrument)) ||
      (k.msc != 0 && k.msc != 1))
    return ET_ERR_INVALID;
  et_ctx* c = new et_ctx();
  c->cfg = k;
  c->stream = (cudaStream_t)k.cuda_stream;
  c->cap = 1u << k.capacity_log2;
  c->dense = k.form == ET_FORM_DENSE;
  c->block = k.block_size;
  c->split = k.split_interactions != 0;
  *out = c;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(c, ET_ERR_CUDA, "no CUDA device");
  }
  register_kernels(k.mode, k.layout, &c->ks);

  Args& a = c->args;
  const size_t rec = (size_t)c->cap * 64u;
  for (int t = 0; t < 3; ++t) {
    for (int h = 0; h < (c->dense ? 2 : 1); ++h) {
      a.trk[t][h] = (char*)dalloc(c, rec);
      if (!a.trk[t][h]) return fail(c, ET_ERR_NOMEM, "track buffer of %zu bytes", rec);
    }
    if (!c->dense) {
      for (int h = 0; h < 2; ++h) {
        a.idx[t][h] = (uint32_t*)dalloc(c, (size_t)c->cap * 4u);
        if (!a.idx[t][h]) return fail(c, ET_ERR_NOMEM, "slot list");
      }
    }
    if (k.instrument) {
      for (int h = 0; h < (c->dense ? 2 : 1); ++h) {
        a.heat[t][h] = (uint32_t*)dalloc(c, (size_t)c->cap * 16u * 4u);
        if (!a.heat[t][h]) return fail(c, ET_ERR_NOMEM, "heatmap");
      }
    }
  }
  a.cap = c->cap;
  a.ctl = c->d_ctl = (DevCtl*)dalloc(c, sizeof(DevCtl));
  a.counts_log = (uint32_t*)dalloc(c, (size_t)k.max_iters * 3u * 4u);
  a.max_iters = k.max_iters;
  a.iter_log_wrap = k.serving ? 1u : 0u;
  a.hybrid_t = k.driver == ET_DRIVER_HYBRID ? (k.hybrid_tracks ? k.hybrid_tracks : 1u << 21) : 0u;
  a.max_events = k.max_events;
  a.ledger = (double*)dalloc(c, (size_t)k.max_events * 5u * 8u);
  if (!a.ctl || !a.counts_log || !a.ledger) return fail(c, ET_ERR_NOMEM, "control block");
  if (k.instrument) {
    a.trace = (unsigned long long*)dalloc(c, 3u * NLEAF * 2u * 8u);
    if (!a.trace) return fail(c, ET_ERR_NOMEM, "trace");
  }
  if (k.id_log) {
    if (k.id_log_capacity == 0) return fail(c, ET_ERR_INVALID, "id_log needs id_log_capacity");
    a.idlog = (IdRec*)dalloc(c, (size_t)k.id_log_capacity * sizeof(IdRec));
    if (!a.idlog) return fail(c, ET_ERR_NOMEM, "id log");
    a.idlog_cap = k.id_log_capacity;
  }
  if (k.serving) {
    a.present = (uint32_t*)dalloc(c, (size_t)k.max_events * 4u);
    a.done_ring = (uint32_t*)dalloc(c, (size_t)k.max_events * 4u);
    a.ev_flag = (uint32_t*)dalloc(c, (size_t)k.max_events * 4u);
    a.done_cap = k.max_events;
    if (!a.present || !a.done_ring || !a.ev_flag) return fail(c, ET_ERR_NOMEM, "serving counters");
  }
  if (k.reuse_slots && !c->dense) {
    for (int t = 0; t < 3; ++t) {
      a.free_ring[t] = (uint32_t*)dalloc(c, (size_t)c->cap * 4u);
      if (!a.free_ring[t]) return fail(c, ET_ERR_NOMEM, "free-slot ring");
    }
  }
  if (c->split) {
    for (int q = 0; q < N_IQ; ++q) {
      a.iq[q] = (uint32_t*)dalloc(c, (size_t)c->cap * QW * 4u);
      if (!a.iq[q]) return fail(c, ET_ERR_NOMEM, "interaction queue");
    }
  }
  a.seed_lo = (uint32_t)k.seed;
  a.msc = k.msc;
  a.timeout_ns = 2000000000ull;
  if (cudaMallocHost(&c->h_ctl, sizeof(DevCtl)) != cudaSuccess ||
      cudaMallocHost(&c->h_stop, 64) != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(c, ET_ERR_NOMEM, "pinned host memory");
  }
  return et_reset(c);
}

et_status et_destroy(et_ctx* c) {
  if (!c) return ET_ERR_INVALID;
  cudaStreamSynchronize(c->stream);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  for (auto& p : c->evpool) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (void* p : c->allocs) {
    if (c->cfg.free) c->cfg.free(p, c->cfg.alloc_user);
    else cudaFree(p);
  }
  if (c->h_ctl) cudaFreeHost(c->h_ctl);
  if (c->h_stop) cudaFreeHost(c->h_stop);
  if (c->h_ledger) cudaFreeHost(c->h_ledger);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  if (c->h_stage_done) cudaEventDestroy(c->h_stage_done);
  serve_free(c->serve);
  (void)cudaGetLastError();
  delete c;
  return ET_OK;
}

et_status et_reset(et_ctx* c) {
  if (!c) return ET_ERR_INVALID;
  Args& a = c->args;
  CUDA_TRY(c, cudaMemsetAsync(a.ctl, 0, sizeof(DevCtl), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(a.counts_log, 0, (size_t)a.max_iters * 3u * 4u, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(a.ledger, 0, (size_t)a.max_events * 5u * 8u, c->stream));
  if (a.score)
    CUDA_TRY(c, cudaMemsetAsync(a.score, 0, (size_t)a.max_events * a.n_slabs * 8u, c->stream));
  if (a.trace) CUDA_TRY(c, cudaMemsetAsync(a.trace, 0, 3u * NLEAF * 2u * 8u, c->stream));
  if (a.present) {
    CUDA_TRY(c, cudaMemsetAsync(a.present, 0, (size_t)a.max_events * 4u, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(a.ev_flag, 0, (size_t)a.max_events * 4u, c->stream));
  }
  c->done_read = 0;
  for (int t = 0; t < 3; ++t)
    for (int h = 0; h < 2; ++h)
      if (a.heat[t][h])
        CUDA_TRY(c, cudaMemsetAsync(a.heat[t][h], 0, (size_t)c->cap * 64u, c->stream));
  // no host synchronisation: the clears are ordered before later work on the stream, and
  // kernel timings recorded so far are collected at the next read-back
  c->launches = 0;
  memset(c->h_ctl, 0, sizeof(DevCtl));
  if (c->serve) {  // the serving loop starts over: nothing queued, in flight or collected
    ServeState* sv = c->serve;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    sv->pending.clear();
    sv->inflight.clear();
    for (int t = 0; t < 3; ++t) sv->reserved[t] = 0;
    sv->issued = sv->delivered = sv->steps_seen = 0;
    CUDA_TRY(c, cudaMemsetAsync(sv->d_cursor, 0, 4, c->stream));
  }
  return ET_OK;
}

et_status et_create_geometry(et_ctx* c, uint32_t n_slabs, const double* thickness_mm,
                             const uint8_t* material, float half_xy_mm) {
  if (!c) return ET_ERR_INVALID;
  if (c->have_geom) return fail(c, ET_ERR_STATE, "geometry already set");
  if (n_slabs < 1 || n_slabs > (uint32_t)MAX_SLABS || !thickness_mm || !material ||
      !(half_xy_mm > 0.0f) || !std::isfinite(half_xy_mm))
    return fail(c, ET_ERR_INVALID, "bad geometry arguments");
  std::vector<float> planes(n_slabs + 1);
  std::vector<uint8_t> mat(n_slabs);
  double z = 0.0;
  planes[0] = 0.0f;
  for (uint32_t s = 0; s < n_slabs; ++s) {
    if (!(thickness_mm[s] > 0.0) || !std::isfinite(thickness_mm[s]) || material[s] >= MAX_MAT)
      return fail(c, ET_ERR_INVALID, "bad slab %u", s);
    z = z + thickness_mm[s];  // FP64 running sum, rounded once
    planes[s + 1] = (float)z;
    mat[s] = material[s];
  }
  Args& a = c->args;
  float* dp = (float*)dalloc(c, planes.size() * 4);
  uint8_t* dm = (uint8_t*)dalloc(c, 128);
  double* sc = (double*)dalloc(c, (size_t)a.max_events * n_slabs * 8u);
  if (!dp || !dm || !sc) return fail(c, ET_ERR_NOMEM, "geometry");
  CUDA_TRY(c, cudaMemcpyAsync(dp, planes.data(), planes.size() * 4, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(dm, mat.data(), n_slabs, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(sc, 0, (size_t)a.max_events * n_slabs * 8u, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  a.planes = dp;
  a.mat = dm;
  a.score = sc;
  a.score_il = 1u;
  a.n_slabs = n_slabs;
  a.half_xy = half_xy_mm;
  c->planes = planes;
  c->mat = mat;
  c->have_geom = true;
  return ET_OK;
}

et_status et_load_tables(et_ctx* c, uint32_t n_materials, uint32_t n_nodes, float log_emin,
                         float inv_dlog, const float* sigma, const float* dedx) {
  if (!c) return ET_ERR_INVALID;
  if (c->have_tables) return fail(c, ET_ERR_STATE, "tables already loaded");
  if (n_materials < 1 || n_materials > (uint32_t)MAX_MAT || n_nodes != NBINS + 1 || !sigma ||
      !dedx || !std::isfinite(log_emin) || !(inv_dlog > 0.0f))
    return fail(c, ET_ERR_INVALID, "tables: need 1..4 materials and 257 nodes");
  const size_t nb = (size_t)n_materials * NBINS;
  std::vector<float2> tot(nb), brem(nb);
  std::vector<float4> cp(nb);
  for (uint32_t m = 0; m < n_materials; ++m) {
    if (!(dedx[m] > 0.0f) || !std::isfinite(dedx[m])) return fail(c, ET_ERR_INVALID, "dedx");
    const float* T = sigma + (size_t)m * 5 * n_nodes;
    for (uint32_t q = 0; q < 5 * n_nodes; ++q)
      if (!std::isfinite(T[q]) || T[q] < 0.0f) return fail(c, ET_ERR_INVALID, "table value");
    for (int i = 0; i < NBINS; ++i) {
      const float* C = T + 0 * n_nodes;
      const float* P = T + 1 * n_nodes;
      const float* S = T + 3 * n_nodes;
      const float* B = T + 4 * n_nodes;
      // {value at node i, FP32 difference to node i+1}: the interpolation
      // T[i] + f (T[i+1] - T[i]) is then one multiply and one add
      tot[m * NBINS + i] = make_float2(S[i], S[i + 1] - S[i]);
      cp[m * NBINS + i] = make_float4(C[i], C[i + 1] - C[i], P[i], P[i + 1] - P[i]);
      brem[m * NBINS + i] = make_float2(B[i], B[i + 1] - B[i]);
    }
    c->args.dedx[m] = dedx[m];
  }
  Args& a = c->args;
  float2* dt = (float2*)dalloc(c, nb * 8);
  float2* db = (float2*)dalloc(c, nb * 8);
  float4* dc = (float4*)dalloc(c, nb * 16);
  if (!dt || !db || !dc) return fail(c, ET_ERR_NOMEM, "tables");
  CUDA_TRY(c, cudaMemcpyAsync(dt, tot.data(), nb * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(db, brem.data(), nb * 8, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(dc, cp.data(), nb * 16, cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  a.tab_tot = dt;
  a.tab_brem = db;
  a.tab_cp = dc;
  a.n_mat = n_materials;
  a.log_emin = log_emin;
  a.inv_dlog = inv_dlog;
  // dynamic shared memory: tables, then one interaction queue per warp
  c->smem_all = tables_bytes_aligned((int)n_materials) + (size_t)(c->block / 32) * queue_bytes_per_warp();
  // only photon interactions are parked in the warp queues: the e+- step kernels need the
  // tables alone, which leaves room for more blocks per SM
  c->smem_tab = tables_bytes_aligned((int)n_materials);
  c->smem_step[EM] = c->smem_step[EP] = c->smem_tab;
  c->smem_step[GAM] = c->smem_all;
  const void* pf = c->ks.persistent[c->cfg.instrument ? 1 : 0][c->dense ? 1 : 0];
  CUDA_TRY(c, cudaFuncSetAttribute(pf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_all));
  // grids: grid-stride kernels sized to fill the machine
  int occ = 0;
  for (int t = 0; t < 3; ++t) {
    const void* fn = c->ks.step[c->cfg.instrument ? 1 : 0][c->dense ? 1 : 0][t];
    CUDA_TRY(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_step[t]));
    CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, c->block, c->smem_step[t]));
    c->grid_fixed[t] = (occ > 0 ? occ : 1) * c->num_sms;
  }
  if (c->split) {
    // the transport pass stages the tables only; the interaction pass needs no shared memory
    const int dn = c->dense ? 1 : 0;
    for (int t = 0; t < 3; ++t) {
      const void* ft = c->ks.transport[dn][t];
      const void* fi = c->ks.interact[dn][t];
      CUDA_TRY(c, cudaFuncSetAttribute(ft, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->smem_tab));
      CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ft, c->block, c->smem_tab));
      c->grid_tr[t] = (occ > 0 ? occ : 1) * c->num_sms;
      CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fi, c->block, 0));
      c->grid_ia[t] = (occ > 0 ? occ : 1) * c->num_sms;
    }
  }
  CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, pf, c->block, c->smem_all));
  if (occ < 1) return fail(c, ET_ERR_CUDA, "persistent kernel does not fit on an SM");
  c->grid_persistent = occ * c->num_sms;
  c->have_tables = true;
  return ET_OK;
}

et_status et_load_msc(et_ctx* c, uint32_t n_materials, const float* x0_mm) {
  if (!c) return ET_ERR_INVALID;
  if (!c->cfg.msc) return fail(c, ET_ERR_STATE, "radiation lengths: not a multiple-scattering context");
  if (!c->have_tables || c->have_msc)
    return fail(c, ET_ERR_STATE, "radiation lengths: once, after the tables");
  if (!x0_mm || n_materials != c->args.n_mat)
    return fail(c, ET_ERR_INVALID, "radiation lengths: one per material");
  for (uint32_t m = 0; m < n_materials; ++m)
    if (!(x0_mm[m] > 0.0f) || !std::isfinite(x0_mm[m]))
      return fail(c, ET_ERR_INVALID, "radiation length %u", m);
  for (uint32_t m = 0; m < n_materials; ++m) c->args.x0[m] = x0_mm[m];
  c->have_msc = true;
  return ET_OK;
}

et_status et_inject(et_ctx* c, const et_primary* p, size_t n) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  if (n == 0) return ET_OK;
  if (!p || n > c->cap) return fail(c, ET_ERR_INVALID, "bad primaries");
  const float h = c->args.half_xy;
  const uint32_t ns = c->args.n_slabs;
  for (uint32_t s = 0; s < ns; ++s)
    if (c->mat[s] >= c->args.n_mat)
      return fail(c, ET_ERR_STATE, "slab %u uses material %u but %u tables are loaded", s,
                  (unsigned)c->mat[s], c->args.n_mat);
  for (size_t i = 0; i < n; ++i) {
    const et_primary& q = p[i];
    const bool ok = q.type < 3 && q.event < c->cfg.max_events && q.ekin > 0.0f &&
                    std::isfinite(q.ekin) && std::fabs(q.pos[0]) <= h && std::fabs(q.pos[1]) <= h &&
                    q.pos[2] >= c->planes[0] && q.pos[2] < c->planes[ns] &&
                    std::isfinite(q.dir[0]) && std::isfinite(q.dir[1]) && std::isfinite(q.dir[2]);
    if (!ok) return fail(c, ET_ERR_INVALID, "primary %zu is invalid", i);
  }
  if (n > c->stage_cap) {
    c->d_stage = (Primary*)dalloc(c, n * sizeof(Primary));
    if (!c->d_stage) return fail(c, ET_ERR_NOMEM, "primary staging");
    c->stage_cap = n;
  }
  // the caller's array is copied into pinned staging before returning (it may change or
  // go away afterwards); the copy to the device then runs asynchronously on the stream
  if (c->h_stage_pending) {
    CUDA_TRY(c, cudaEventSynchronize(c->h_stage_done));  // the previous copy has read it
    c->h_stage_pending = false;
  }
  if (n > c->h_stage_cap) {
    if (c->h_stage) cudaFreeHost(c->h_stage);
    c->h_stage = nullptr;
    c->h_stage_cap = 0;
    if (cudaMallocHost(&c->h_stage, n * sizeof(Primary)) != cudaSuccess) {
      c->h_stage = nullptr;
      return fail(c, ET_ERR_NOMEM, "pinned primary staging");
    }
    c->h_stage_cap = n;
  }
  if (!c->h_stage_done)
    CUDA_TRY(c, cudaEventCreateWithFlags(&c->h_stage_done, cudaEventDisableTiming));
  memcpy(c->h_stage, p, n * sizeof(Primary));
  CUDA_TRY(c, cudaMemcpyAsync(c->d_stage, c->h_stage, n * sizeof(Primary), cudaMemcpyHostToDevice,
                              c->stream));
  CUDA_TRY(c, cudaEventRecord(c->h_stage_done, c->stream));
  c->h_stage_pending = true;
  uint32_t nn = (uint32_t)n;
  const Primary* dp = c->d_stage;
  void* params[] = {(void*)&c->args, (void*)&dp, (void*)&nn};
  const int grid = (int)((n + 255) / 256);
  return launch(c, c->ks.inject[c->dense ? 1 : 0], grid, 256, 0, params);
}

et_status et_inject_device(et_ctx* c, const et_primary* p, size_t n) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  if (n == 0) return ET_OK;
  if (!p || n > c->cap || ((uintptr_t)p & 15u) != 0) return fail(c, ET_ERR_INVALID, "bad primaries");
  for (uint32_t s = 0; s < c->args.n_slabs; ++s)
    if (c->mat[s] >= c->args.n_mat) return fail(c, ET_ERR_STATE, "slab material without table");
  uint32_t nn = (uint32_t)n;
  const Primary* dp = reinterpret_cast<const Primary*>(p);
  void* params[] = {(void*)&c->args, (void*)&dp, (void*)&nn};
  return launch(c, c->ks.inject[c->dense ? 1 : 0], (int)((n + 255) / 256), 256, 0, params);
}

// The step of type t: one step kernel, or (split form) the transport pass then the
// interaction pass.  grid: the step kernel's grid, 0 = the fixed (grid-stride) grids.
static et_status launch_type_step(et_ctx* c, int t, int grid) {
  void* params[] = {(void*)&c->args};
  const int instr = c->cfg.instrument ? 1 : 0, dn = c->dense ? 1 : 0;
  if (!c->split)
    return launch(c, c->ks.step[instr][dn][t], grid ? grid : c->grid_fixed[t], c->block,
                  c->smem_step[t], params);
  et_status s = launch(c, c->ks.transport[dn][t], grid ? std::min(grid, c->grid_tr[t]) : c->grid_tr[t],
                       c->block, c->smem_tab, params);
  if (s != ET_OK) return s;
  // at most as many interactions as tracks
  return launch(c, c->ks.interact[dn][t], grid ? std::min(grid, c->grid_ia[t]) : c->grid_ia[t],
                c->block, 0, params);
}

// Launch the step kernels of one iteration; counts from the last read-back.
static et_status launch_step_kernels(et_ctx* c, const uint32_t n[3], bool fixed_grid) {
  for (int t = 0; t < 3; ++t) {
    if (!fixed_grid && n[t] == 0) continue;
    int grid = fixed_grid ? c->grid_fixed[t] : (int)((n[t] + c->block - 1) / c->block);
    if (grid > c->grid_fixed[t]) grid = c->grid_fixed[t];
    if (grid < 1) grid = 1;
    EventPair* ev = fixed_grid ? nullptr : timing_begin(c);
    et_status s = launch_type_step(c, t, fixed_grid ? 0 : grid);
    timing_end(c, ev);
    if (s != ET_OK) return s;
  }
  return ET_OK;
}

static et_status launch_end(et_ctx* c, cudaGraphConditionalHandle h, int use) {
  void* params[] = {(void*)&c->args, (void*)&h, (void*)&use};
  return launch(c, (const void*)k_end_iteration, 1, 1, 0, params);
}

static et_status one_hostloop_iteration(et_ctx* c, bool* empty) {
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  const uint32_t it = c->h_ctl->iter;
  const uint32_t* row = c->h_ctl->cnt[it % 3];
  const uint32_t n[3] = {row[cw(EM)], row[cw(EP)], row[cw(GAM)]};
  *empty = (n[0] + n[1] + n[2]) == 0;
  if (*empty) return ET_OK;
  if (it >= c->cfg.max_iters && !c->cfg.serving) return fail(c, ET_ERR_CAPACITY, "iteration log full");
  c->h_stop[0] = 0xffffffffu;
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->stop_iter, c->h_stop, 4, cudaMemcpyHostToDevice, c->stream));
  s = launch_step_kernels(c, n, false);
  if (s != ET_OK) return s;
  return launch_end(c, 0, 0);
}

static void fill_stats(et_ctx* c, const DevCtl& before, et_iter_stats* out) {
  if (!out) return;
  const DevCtl& now = *c->h_ctl;
  const uint32_t cur = now.iter % 3;
  for (int t = 0; t < 3; ++t) out->n_active[t] = now.cnt[cur][cw(t)];
  out->pad = 0;
  out->steps = 0;
  out->secondaries = 0;
  for (int t = 0; t < 3; ++t) {
    out->steps += now.steps[t] - before.steps[t];
    out->secondaries += now.secondaries[t] - before.secondaries[t];
  }
}

et_status et_run_iteration(et_ctx* c, et_iter_stats* out) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  const DevCtl before = *c->h_ctl;
  bool empty = false;
  s = one_hostloop_iteration(c, &empty);
  if (s != ET_OK) return s;
  s = sync_ctl(c);
  if (s != ET_OK) return s;
  fill_stats(c, before, out);
  return ET_OK;
}

static et_status build_graph(et_ctx* c) {
  cudaGraph_t g;
  CUDA_TRY(c, cudaGraphCreate(&g, 0));
  c->graph = g;
  cudaGraphConditionalHandle h;
  CUDA_TRY(c, cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault));
  // the params struct holds a union of node kinds: zero-filled storage, then the conditional part
  alignas(cudaGraphNodeParams) unsigned char np_storage[sizeof(cudaGraphNodeParams)];
  memset(np_storage, 0, sizeof np_storage);
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_storage);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  CUDA_TRY(c, cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  cudaStream_t cs;
  CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = c->stream;
  const uint64_t saved_launches = c->launches;
  c->stream = cs;
  et_status s = ET_OK;
  if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess) {
    s = fail(c, ET_ERR_CUDA, "graph capture failed to start");
  } else {
    // the three per-type step kernels as parallel branches (fork/join through events), so
    // that one type's sparse tail overlaps with the others' work; then the end node
    cudaStream_t br[2] = {nullptr, nullptr};
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool ok = true;
    for (int k = 0; k < 2; ++k) ok = ok && cudaStreamCreateWithFlags(&br[k], cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 3; ++k) ok = ok && cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) s = fail(c, ET_ERR_CUDA, "graph branches");
    if (s == ET_OK && (cudaEventRecord(ev[0], cs) != cudaSuccess ||
                       cudaStreamWaitEvent(br[0], ev[0], 0) != cudaSuccess ||
                       cudaStreamWaitEvent(br[1], ev[0], 0) != cudaSuccess))
      s = fail(c, ET_ERR_CUDA, "graph fork");
    for (int t = 0; t < 3 && s == ET_OK; ++t) {
      c->stream = t == 0 ? cs : br[t - 1];
      s = launch_type_step(c, t, 0);
    }
    c->stream = cs;
    if (s == ET_OK && (cudaEventRecord(ev[1], br[0]) != cudaSuccess ||
                       cudaEventRecord(ev[2], br[1]) != cudaSuccess ||
                       cudaStreamWaitEvent(cs, ev[1], 0) != cudaSuccess ||
                       cudaStreamWaitEvent(cs, ev[2], 0) != cudaSuccess))
      s = fail(c, ET_ERR_CUDA, "graph join");
    if (s == ET_OK) s = launch_end(c, h, 1);
    cudaGraph_t out_g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &out_g);
    if (s == ET_OK && e != cudaSuccess)
      s = fail(c, ET_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    for (int k = 0; k < 2; ++k)
      if (br[k]) cudaStreamDestroy(br[k]);
    for (int k = 0; k < 3; ++k)
      if (ev[k]) cudaEventDestroy(ev[k]);
  }
  c->stream = saved;
  c->launches = saved_launches;
  cudaStreamDestroy(cs);
  if (s != ET_OK) return s;
  CUDA_TRY(c, cudaGraphInstantiate(&c->gexec, g, 0));
  return ET_OK;
}

static et_status launch_persistent(et_ctx* c, uint32_t rel) {
  c->h_stop[1] = rel;
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->stop_rel, c->h_stop + 1, 4, cudaMemcpyHostToDevice, c->stream));
  int fault = c->fault_skip_block;
  void* params[] = {(void*)&c->args, (void*)&fault};
  const void* fn = c->ks.persistent[c->cfg.instrument ? 1 : 0][c->dense ? 1 : 0];
  EventPair* ev = timing_begin(c);
  CUDA_TRY(c, cudaLaunchCooperativeKernel(fn, dim3(c->grid_persistent), dim3(c->block), params,
                                          c->smem_all, c->stream));
  timing_end(c, ev);
  c->launches += 1;
  return ET_OK;
}

static et_status launch_graph(et_ctx* c, uint32_t stop_iter) {
  c->h_stop[0] = stop_iter;
  CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->stop_iter, c->h_stop, 4, cudaMemcpyHostToDevice, c->stream));
  if (!c->gexec) {
    et_status s = build_graph(c);
    if (s != ET_OK) return s;
  }
  EventPair* ev = timing_begin(c);
  CUDA_TRY(c, cudaGraphLaunch(c->gexec, c->stream));
  timing_end(c, ev);
  c->launches += 1;
  return ET_OK;
}

// Hybrid driver: small iterations in the persistent kernel (one launch loops them on the
// device), large ones in the graph of per-type step kernels; each launch stops where the
// population crosses the threshold (the kernels check it), and runs at least one
// iteration, so every round of this loop makes progress.
static et_status run_hybrid(et_ctx* c, uint64_t max_iters, et_iter_stats* totals,
                            uint64_t* n_iters) {
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  const DevCtl before = *c->h_ctl;
  const uint32_t it0 = before.iter;
  uint64_t lim64 = (uint64_t)it0 + max_iters;
  const uint32_t lim = lim64 > 0xffffffffull ? 0xffffffffu : (uint32_t)lim64;
  for (;;) {
    const uint32_t it = c->h_ctl->iter;
    const uint32_t* row = c->h_ctl->cnt[it % 3];
    const uint64_t n = (uint64_t)row[cw(EM)] + row[cw(EP)] + row[cw(GAM)];
    if (n == 0 || it >= lim) break;
    s = n < c->args.hybrid_t ? launch_persistent(c, lim - it) : launch_graph(c, lim);
    if (s != ET_OK) return s;
    s = sync_ctl(c);
    if (s != ET_OK) return s;
  }
  fill_stats(c, before, totals);
  if (n_iters) *n_iters = c->h_ctl->iter - it0;
  return ET_OK;
}

et_status et_run_until_empty(et_ctx* c, uint64_t max_iters, et_iter_stats* totals,
                             uint64_t* n_iters) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  if (c->cfg.driver == ET_DRIVER_HYBRID) return run_hybrid(c, max_iters, totals, n_iters);
  if (c->cfg.driver == ET_DRIVER_PERSISTENT && max_iters > 0) {
    // one launch, one read-back: the kernel stops after max_iters iterations (or when no
    // track is left) and records its starting iteration and counters for the totals
    et_status s = launch_persistent(c, max_iters > 0xffffffffull ? 0xffffffffu : (uint32_t)max_iters);
    if (s != ET_OK) return s;
    s = sync_ctl(c);
    if (s != ET_OK) return s;
    DevCtl before = *c->h_ctl;
    before.iter = c->h_ctl->run_iter0;
    for (int t = 0; t < NTYPES; ++t) {
      before.steps[t] = c->h_ctl->run_steps0[t];
      before.secondaries[t] = c->h_ctl->run_sec0[t];
    }
    fill_stats(c, before, totals);
    if (n_iters) *n_iters = c->h_ctl->iter - before.iter;
    return ET_OK;
  }
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  const DevCtl before = *c->h_ctl;
  const uint32_t it0 = before.iter;
  const uint32_t* n0 = before.cnt[it0 % 3];
  const bool empty0 = (n0[0] + n0[1] + n0[2]) == 0;
  if (!empty0 && max_iters > 0) {
    uint64_t lim = (uint64_t)it0 + max_iters;
    if (lim > 0xffffffffull) lim = 0xffffffffull;
    if (c->cfg.driver == ET_DRIVER_HOSTLOOP) {
      for (uint64_t k = 0; k < max_iters; ++k) {
        bool empty = false;
        s = one_hostloop_iteration(c, &empty);
        if (s != ET_OK) return s;
        if (empty) break;
      }
    } else {  // the graph (the persistent and hybrid drivers returned above)
      s = launch_graph(c, (uint32_t)lim);
      if (s != ET_OK) return s;
    }
  }
  s = sync_ctl(c);
  if (s != ET_OK) return s;
  fill_stats(c, before, totals);
  if (n_iters) *n_iters = c->h_ctl->iter - it0;
  return ET_OK;
}

et_status et_read_scoring(et_ctx* c, uint32_t event, double* slab_dep, size_t n_slabs,
                          et_ledger* out) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom) return fail(c, ET_ERR_STATE, "no geometry");
  if (event >= c->cfg.max_events || (slab_dep && n_slabs < c->args.n_slabs))
    return fail(c, ET_ERR_INVALID, "bad event or slab buffer");
  std::vector<double> sc(c->args.n_slabs);
  double lg[5];
  CUDA_TRY(c, cudaMemcpyAsync(sc.data(), c->args.score + (size_t)event * c->args.n_slabs,
                              sc.size() * 8, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(lg, c->args.ledger + (size_t)event * 5, sizeof lg,
                              cudaMemcpyDeviceToHost, c->stream));
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  double sum = 0.0;
  const uint32_t ns = c->args.n_slabs;
  for (uint32_t i = 0; i < ns; ++i) {
    const double v = sc[c->args.score_il ? score_col(i, ns) : i];
    if (slab_dep) slab_dep[i] = v;
    sum += v;
  }
  if (out) {
    out->injected = lg[0];
    out->below_cut = lg[1];
    out->escaped = lg[2];
    out->mass_created = lg[3];
    out->mass_consumed = lg[4];
    out->deposited_cont = sum - lg[1];
  }
  return ET_OK;
}

et_status et_read_scoring_all(et_ctx* c, double* score, et_ledger* ledger) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom) return fail(c, ET_ERR_STATE, "no geometry");
  const size_t ne = c->cfg.max_events, ns = c->args.n_slabs;
  std::vector<double> sc;
  double* dst = score;
  if (!dst && ledger) {
    sc.resize(ne * ns);
    dst = sc.data();
  }
  if (ledger && !c->h_ledger && cudaMallocHost(&c->h_ledger, ne * 5 * 8) != cudaSuccess) {
    c->h_ledger = nullptr;
    return fail(c, ET_ERR_NOMEM, "pinned ledger staging");
  }
  const double* lg = c->h_ledger;
  if (dst)
    CUDA_TRY(c, cudaMemcpyAsync(dst, c->args.score, ne * ns * 8, cudaMemcpyDeviceToHost, c->stream));
  if (ledger)
    CUDA_TRY(c, cudaMemcpyAsync(c->h_ledger, c->args.ledger, ne * 5 * 8, cudaMemcpyDeviceToHost, c->stream));
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  if (dst && c->args.score_il) {  // rows back into slab order
    double row[MAX_SLABS];
    for (size_t e = 0; e < ne; ++e) {
      double* r = dst + e * ns;
      memcpy(row, r, ns * sizeof(double));
      for (uint32_t i = 0; i < (uint32_t)ns; ++i) r[i] = row[score_col(i, (uint32_t)ns)];
    }
  }
  if (ledger) {
    for (size_t e = 0; e < ne; ++e) {
      double sum = 0.0;
      for (size_t i = 0; i < ns; ++i) sum += dst[e * ns + i];
      ledger[e].injected = lg[e * 5 + 0];
      ledger[e].below_cut = lg[e * 5 + 1];
      ledger[e].escaped = lg[e * 5 + 2];
      ledger[e].mass_created = lg[e * 5 + 3];
      ledger[e].mass_consumed = lg[e * 5 + 4];
      ledger[e].deposited_cont = sum - lg[e * 5 + 1];
    }
  }
  return ET_OK;
}

et_status et_read_iteration_counts(et_ctx* c, uint64_t* counts, uint64_t cap, uint64_t* n) {
  if (!c || !n) return ET_ERR_INVALID;
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  uint64_t it = c->h_ctl->iter;
  if (it > c->cfg.max_iters) it = c->cfg.max_iters;
  *n = it;
  if (!counts) return ET_OK;
  if (cap < it) return fail(c, ET_ERR_CAPACITY, "count buffer too short (%llu < %llu)",
                           (unsigned long long)cap, (unsigned long long)it);
  std::vector<uint32_t> h(it * 3);
  if (it)
    CUDA_TRY(c, cudaMemcpyAsync(h.data(), c->args.counts_log, it * 12, cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  for (uint64_t q = 0; q < it * 3; ++q) counts[q] = h[q];
  return ET_OK;
}

et_status et_read_id_log(et_ctx* c, et_idrec* out, uint64_t cap, uint64_t* n) {
  if (!c || !n) return ET_ERR_INVALID;
  if (!c->args.idlog) return fail(c, ET_ERR_STATE, "id log not enabled");
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  uint64_t m = c->h_ctl->idlog_n;
  *n = m;
  if (!out) return ET_OK;
  if (cap < m) return fail(c, ET_ERR_CAPACITY, "id buffer too short");
  if (m)
    CUDA_TRY(c, cudaMemcpyAsync(out, c->args.idlog, m * sizeof(IdRec), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return ET_OK;
}

et_status et_read_field_trace(et_ctx* c, uint64_t* counts) {
  if (!c || !counts) return ET_ERR_INVALID;
  if (!c->args.trace) return fail(c, ET_ERR_STATE, "not an instrumented context");
  CUDA_TRY(c, cudaMemcpyAsync(counts, c->args.trace, 3u * NLEAF * 2u * 8u, cudaMemcpyDeviceToHost, c->stream));
  return sync_ctl(c);
}

et_status et_read_heatmap(et_ctx* c, uint32_t type, uint32_t half, uint32_t* out, uint64_t cap) {
  if (!c || !out || type > 2 || half > 1) return ET_ERR_INVALID;
  if (!c->args.heat[type][half]) return fail(c, ET_ERR_STATE, "no heatmap for this buffer");
  if (cap < (uint64_t)c->cap * 16u) return fail(c, ET_ERR_CAPACITY, "heatmap buffer too short");
  CUDA_TRY(c, cudaMemcpyAsync(out, c->args.heat[type][half], (size_t)c->cap * 64u, cudaMemcpyDeviceToHost, c->stream));
  return sync_ctl(c);
}

et_status et_read_counters(et_ctx* c, et_counters* out) {
  if (!c || !out) return ET_ERR_INVALID;
  CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  timing_collect(c);
  const DevCtl& d = *c->h_ctl;
  memset(out, 0, sizeof *out);
  for (int t = 0; t < 3; ++t) {
    out->steps[t] = d.steps[t];
    out->secondaries[t] = d.secondaries[t];
    out->slot_high_water[t] = d.hwm[cw(t)];
  }
  out->iterations = d.iter;
  out->reject_cap_hits = d.reject_cap_hits;
  out->kernel_launches = c->launches;
  out->status = d.status;
  return ET_OK;
}

et_status et_poll_completed(et_ctx* c, uint32_t* events, uint64_t cap, uint64_t* n) {
  if (!c || !n) return ET_ERR_INVALID;
  if (!c->args.present) return fail(c, ET_ERR_STATE, "not a serving context");
  et_status s = scan_done(c);
  if (s != ET_OK) return s;
  s = sync_ctl(c);
  if (s != ET_OK) return s;
  const uint32_t done = c->h_ctl->n_done;
  uint32_t avail = done - c->done_read;
  if (avail > c->args.done_cap) return fail(c, ET_ERR_CAPACITY, "completion ring overrun");
  if (avail > cap) avail = (uint32_t)cap;
  *n = avail;
  if (!avail) return ET_OK;
  if (!events) return fail(c, ET_ERR_INVALID, "no output buffer");
  const uint32_t dc = c->args.done_cap;
  const uint32_t first = c->done_read % dc;
  const uint32_t n1 = avail < dc - first ? avail : dc - first;
  CUDA_TRY(c, cudaMemcpyAsync(events, c->args.done_ring + first, (size_t)n1 * 4u,
                              cudaMemcpyDeviceToHost, c->stream));
  if (n1 < avail)
    CUDA_TRY(c, cudaMemcpyAsync(events + n1, c->args.done_ring, (size_t)(avail - n1) * 4u,
                                cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->done_read += avail;
  return ET_OK;
}

et_status et_release_event(et_ctx* c, uint32_t event) {
  if (!c) return ET_ERR_INVALID;
  if (!c->have_geom) return fail(c, ET_ERR_STATE, "no geometry");
  if (event >= c->cfg.max_events) return fail(c, ET_ERR_INVALID, "bad event");
  const size_t ns = c->args.n_slabs;
  CUDA_TRY(c, cudaMemsetAsync(c->args.score + (size_t)event * ns, 0, ns * 8u, c->stream));
  CUDA_TRY(c, cudaMemsetAsync(c->args.ledger + (size_t)event * 5u, 0, 5u * 8u, c->stream));
  if (c->args.present) {
    CUDA_TRY(c, cudaMemsetAsync(c->args.present + event, 0, 4u, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->args.ev_flag + event, 0, 4u, c->stream));
  }
  return ET_OK;
}

et_status et_set_timing(et_ctx* c, int on) {
  if (!c) return ET_ERR_INVALID;
  c->timing = on != 0;
  return ET_OK;
}

et_status et_read_timing(et_ctx* c, double* ms_total, uint64_t* launches) {
  if (!c) return ET_ERR_INVALID;
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  timing_collect(c);
  if (ms_total) *ms_total = c->ms_acc;
  if (launches) *launches = c->timed;
  c->ms_acc = 0.0;
  c->timed = 0;
  return ET_OK;
}

// Profiling hooks (et_debug.h): per-iteration start times of the persistent driver.
et_status et_debug_iteration_times(et_ctx* c, int enable) {
  if (!c) return ET_ERR_INVALID;
  if (enable && !c->d_iter_ns) {
    c->d_iter_ns = (unsigned long long*)dalloc(c, (size_t)c->cfg.max_iters * 8u);
    if (!c->d_iter_ns) return fail(c, ET_ERR_NOMEM, "iteration time log");
  }
  c->args.iter_ns = enable ? c->d_iter_ns : nullptr;
  return ET_OK;
}

et_status et_debug_read_iteration_times(et_ctx* c, uint64_t* out, uint64_t cap, uint64_t* n) {
  if (!c || !n) return ET_ERR_INVALID;
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  uint64_t it = c->h_ctl->iter;
  if (it > c->cfg.max_iters) it = c->cfg.max_iters;
  *n = it;
  if (!out || !c->d_iter_ns) return ET_OK;
  if (cap < it) return fail(c, ET_ERR_CAPACITY, "buffer too short");
  CUDA_TRY(c, cudaMemcpy(out, c->d_iter_ns, it * 8u, cudaMemcpyDeviceToHost));
  return ET_OK;
}

// Test hooks (et_debug.h): bounded-wait fault injection for the persistent driver.
et_status et_debug_set_barrier_fault(et_ctx* c, int skip_block, uint64_t timeout_ns) {
  if (!c) return ET_ERR_INVALID;
  c->fault_skip_block = skip_block;
  if (timeout_ns) c->args.timeout_ns = timeout_ns;
  return ET_OK;
}


// Test hook (et_debug.h): the deposit rows' column order.
et_status et_debug_score_columns(uint32_t n_slabs, uint32_t* out) {
  if (!out || n_slabs < 1 || n_slabs > (uint32_t)MAX_SLABS) return ET_ERR_INVALID;
  for (uint32_t s = 0; s < n_slabs; ++s) out[s] = score_col(s, n_slabs);
  return ET_OK;
}

// Test hook (et_debug.h): the device primitives on a batch of inputs.
et_status et_debug_eval(int what, const void* in, void* out, size_t n, void* stream) {
  if (what < ET_EVAL_PHILOX || what > ET_EVAL_SINCOS2PI || (n && (!in || !out)))
    return ET_ERR_INVALID;
  if (n == 0) return ET_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((n + 255) / 256);
  k_debug_eval<<<grid, 256, 0, s>>>(what, in, out, n);
  if (cudaGetLastError() != cudaSuccess) return ET_ERR_CUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? ET_OK : ET_ERR_CUDA;
}


// ---- checkpoint / resume ----
// A snapshot is a header (the configuration it belongs to) followed by tagged sections:
// the control block, the live part of the track arrays (dense: the current half; sparse:
// the slot array, the current slot list and the reuse rings), scores, ledgers, the
// iteration log, the serving counters, the death log and the instrumentation counts.
// Every random draw is keyed by (event, id, step), so a restored context continues with
// exactly the histories the original would have followed.
namespace {
struct SnapHeader {
  char magic[8];
  uint32_t version, form, layout, capacity_log2, mode, max_events, max_iters, n_slabs;
  uint32_t serving, reuse_slots, id_log, instrument, msc, pad;
  uint64_t id_log_capacity, seed, n_sections;
};
struct SnapSection {
  uint32_t tag, index;
  uint64_t bytes;
};
enum : uint32_t { SN_CTL = 1, SN_TRK, SN_IDX, SN_FREE, SN_SCORE, SN_LEDGER, SN_COUNTS, SN_LIVE,
                  SN_DONE, SN_IDLOG, SN_TRACE, SN_HEAT, SN_EVFLAG };
constexpr char kSnapMagic[8] = {'E', 'T', 'S', 'N', 'A', 'P', '1', 0};

struct SnapItem {
  uint32_t tag, index;
  void* dev;
  uint64_t bytes;
};

// bytes of a track array that hold its first n records
uint64_t record_prefix(int layout, uint64_t n, uint64_t cap) {
  const uint64_t lanes = layout == ET_LAYOUT_AOS ? 1 : layout == ET_LAYOUT_AOSOA8 ? 8
                         : layout == ET_LAYOUT_AOSOA16 ? 16 : layout == ET_LAYOUT_AOSOA32 ? 32
                         : layout == ET_LAYOUT_AOSOA64 ? 64 : layout == ET_LAYOUT_AOSOA128 ? 128 : 0;
  if (lanes == 0) return cap * 64u;  // SoA-like layouts spread every record over the array
  const uint64_t blocks = (n + lanes - 1) / lanes;
  return std::min(cap, blocks * lanes) * 64u;
}
}  // namespace

static std::vector<SnapItem> snapshot_items(et_ctx* c) {
  std::vector<SnapItem> v;
  Args& a = c->args;
  const DevCtl& h = *c->h_ctl;
  const uint32_t it = h.iter, cur = it % 3, half = it & 1u;
  v.push_back({SN_CTL, 0, c->d_ctl, sizeof(DevCtl)});
  for (int t = 0; t < NTYPES; ++t) {
    if (c->dense) {
      v.push_back({SN_TRK, (uint32_t)(2 * t + half), a.trk[t][half],
                   record_prefix(c->cfg.layout, h.cnt[cur][cw(t)], c->cap)});
    } else {
      v.push_back({SN_TRK, (uint32_t)(2 * t), a.trk[t][0], (uint64_t)c->cap * 64u});
      v.push_back({SN_IDX, (uint32_t)(2 * t + half), a.idx[t][half], (uint64_t)h.cnt[cur][cw(t)] * 4u});
      if (a.free_ring[t]) v.push_back({SN_FREE, (uint32_t)t, a.free_ring[t], (uint64_t)c->cap * 4u});
    }
    for (int hh = 0; hh < 2; ++hh)
      if (a.heat[t][hh]) v.push_back({SN_HEAT, (uint32_t)(2 * t + hh), a.heat[t][hh], (uint64_t)c->cap * 64u});
  }
  v.push_back({SN_SCORE, 0, a.score, (uint64_t)a.max_events * a.n_slabs * 8u});
  v.push_back({SN_LEDGER, 0, a.ledger, (uint64_t)a.max_events * 5u * 8u});
  v.push_back({SN_COUNTS, 0, a.counts_log, (uint64_t)a.max_iters * 12u});
  if (a.present) {
    v.push_back({SN_LIVE, 0, a.present, (uint64_t)a.max_events * 4u});
    v.push_back({SN_DONE, 0, a.done_ring, (uint64_t)a.done_cap * 4u});
    v.push_back({SN_EVFLAG, 0, a.ev_flag, (uint64_t)a.max_events * 4u});
  }
  if (a.idlog) {
    const uint64_t m = std::min<uint64_t>(h.idlog_n, a.idlog_cap);
    v.push_back({SN_IDLOG, 0, a.idlog, m * sizeof(IdRec)});
  }
  if (a.trace) v.push_back({SN_TRACE, 0, a.trace, 3u * NLEAF * 2u * 8u});
  return v;
}

static SnapHeader snapshot_header(const et_ctx* c, uint64_t n_sections) {
  SnapHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, kSnapMagic, 8);
  hd.version = 2;
  hd.form = (uint32_t)c->cfg.form;
  hd.layout = (uint32_t)c->cfg.layout;
  hd.capacity_log2 = c->cfg.capacity_log2;
  hd.mode = (uint32_t)c->cfg.mode;
  hd.max_events = c->cfg.max_events;
  hd.max_iters = c->cfg.max_iters;
  hd.n_slabs = c->args.n_slabs;
  hd.serving = (uint32_t)c->cfg.serving;
  hd.reuse_slots = (uint32_t)c->cfg.reuse_slots;
  hd.id_log = (uint32_t)c->cfg.id_log;
  hd.instrument = (uint32_t)c->cfg.instrument;
  hd.msc = (uint32_t)c->cfg.msc;
  hd.pad = 0;
  hd.id_log_capacity = c->cfg.id_log_capacity;
  hd.seed = c->cfg.seed;
  hd.n_sections = n_sections;
  return hd;
}

et_status et_snapshot_size(et_ctx* c, uint64_t* bytes) {
  if (!c || !bytes) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  uint64_t n = sizeof(SnapHeader);
  for (const SnapItem& it : snapshot_items(c)) n += sizeof(SnapSection) + it.bytes;
  *bytes = n;
  return ET_OK;
}

et_status et_snapshot(et_ctx* c, void* out, uint64_t cap, uint64_t* written) {
  if (!c || !out) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  et_status s = sync_ctl(c);
  if (s != ET_OK) return s;
  const std::vector<SnapItem> items = snapshot_items(c);
  uint64_t need = sizeof(SnapHeader);
  for (const SnapItem& it : items) need += sizeof(SnapSection) + it.bytes;
  if (cap < need) return fail(c, ET_ERR_CAPACITY, "snapshot needs %llu bytes", (unsigned long long)need);
  unsigned char* p = static_cast<unsigned char*>(out);
  const SnapHeader hd = snapshot_header(c, items.size());
  memcpy(p, &hd, sizeof hd);
  p += sizeof hd;
  for (const SnapItem& it : items) {
    const SnapSection sec{it.tag, it.index, it.bytes};
    memcpy(p, &sec, sizeof sec);
    p += sizeof sec;
    if (it.bytes) CUDA_TRY(c, cudaMemcpyAsync(p, it.dev, it.bytes, cudaMemcpyDeviceToHost, c->stream));
    p += it.bytes;
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (written) *written = need;
  return ET_OK;
}

et_status et_restore(et_ctx* c, const void* in, uint64_t n) {
  if (!c || !in) return ET_ERR_INVALID;
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  if (n < sizeof(SnapHeader)) return fail(c, ET_ERR_INVALID, "snapshot too short");
  SnapHeader hd;
  memcpy(&hd, in, sizeof hd);
  const SnapHeader mine = snapshot_header(c, hd.n_sections);
  if (memcmp(hd.magic, kSnapMagic, 8) != 0 || hd.version != 2)
    return fail(c, ET_ERR_INVALID, "not a snapshot of this library");
  if (memcmp(&hd, &mine, sizeof hd) != 0)
    return fail(c, ET_ERR_INVALID, "snapshot of a context with another configuration");
  et_status s = et_reset(c);
  if (s != ET_OK) return s;
  // find the device buffer of each section in this context
  Args& a = c->args;
  const unsigned char* p = static_cast<const unsigned char*>(in) + sizeof hd;
  const unsigned char* end = static_cast<const unsigned char*>(in) + n;
  for (uint64_t k = 0; k < hd.n_sections; ++k) {
    if ((uint64_t)(end - p) < sizeof(SnapSection)) return fail(c, ET_ERR_INVALID, "snapshot truncated");
    SnapSection sec;
    memcpy(&sec, p, sizeof sec);
    p += sizeof sec;
    if ((uint64_t)(end - p) < sec.bytes) return fail(c, ET_ERR_INVALID, "snapshot truncated");
    void* dev = nullptr;
    uint64_t limit = 0;
    const uint32_t t = sec.index / 2, hh = sec.index % 2;
    switch (sec.tag) {
      case SN_CTL: dev = c->d_ctl; limit = sizeof(DevCtl); break;
      case SN_TRK: if (t < 3) { dev = a.trk[t][c->dense ? hh : 0]; limit = (uint64_t)c->cap * 64u; } break;
      case SN_IDX: if (t < 3 && !c->dense) { dev = a.idx[t][hh]; limit = (uint64_t)c->cap * 4u; } break;
      case SN_FREE: if (sec.index < 3) { dev = a.free_ring[sec.index]; limit = (uint64_t)c->cap * 4u; } break;
      case SN_HEAT: if (t < 3) { dev = a.heat[t][hh]; limit = (uint64_t)c->cap * 64u; } break;
      case SN_SCORE: dev = a.score; limit = (uint64_t)a.max_events * a.n_slabs * 8u; break;
      case SN_LEDGER: dev = a.ledger; limit = (uint64_t)a.max_events * 40u; break;
      case SN_COUNTS: dev = a.counts_log; limit = (uint64_t)a.max_iters * 12u; break;
      case SN_LIVE: dev = a.present; limit = (uint64_t)a.max_events * 4u; break;
      case SN_DONE: dev = a.done_ring; limit = (uint64_t)a.done_cap * 4u; break;
      case SN_EVFLAG: dev = a.ev_flag; limit = (uint64_t)a.max_events * 4u; break;
      case SN_IDLOG: dev = a.idlog; limit = a.idlog_cap * sizeof(IdRec); break;
      case SN_TRACE: dev = a.trace; limit = 3u * NLEAF * 2u * 8u; break;
      default: break;
    }
    if (!dev || sec.bytes > limit) return fail(c, ET_ERR_INVALID, "snapshot section %u/%u does not fit", sec.tag, sec.index);
    if (sec.bytes) CUDA_TRY(c, cudaMemcpyAsync(dev, p, sec.bytes, cudaMemcpyHostToDevice, c->stream));
    p += sec.bytes;
  }
  // the grid barrier restarts from zero (the grid may differ on another GPU); launch-local
  // fields are set by the next run
  DevCtl* d = c->d_ctl;
  CUDA_TRY(c, cudaMemsetAsync(&d->bar_count, 0, sizeof(uint32_t), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(&d->bar_gen, 0, sizeof(uint32_t), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(d->grab, 0, sizeof d->grab, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  s = sync_ctl(c);
  if (s != ET_OK) return s;
  c->done_read = c->h_ctl->n_done;  // completions before the snapshot were already reported
  return ET_OK;
}


// ---- native serving loop: pipelined rounds of continuous batching ----
// Requests wait in a host queue (et_serve_submit).  Each round (et_serve_round) admits
// queued requests in order while their reserved track slots fit, injects them, runs a
// few iterations with every in-flight shower, and lets a one-block kernel copy the
// results of the events completed so far into a compact buffer (clearing their scores)
// that one copy brings to pinned host memory.  The call then waits for the round before
// it and hands back that round's results: the host's admission and read-back overlap the
// GPU's work on the next round, which is already queued on the stream.
static et_status serve_state(et_ctx* c, ServeState** out) {
  if (!c->args.present) return fail(c, ET_ERR_STATE, "not a serving context");
  if (!c->have_geom || !c->have_tables || (c->cfg.msc && !c->have_msc))
    return fail(c, ET_ERR_STATE, "geometry, tables (and radiation lengths for msc) first");
  if (!c->serve) {
    ServeState* s = new ServeState();
    s->max_out = c->cfg.max_events < 256u ? c->cfg.max_events : 256u;
    const size_t row = (size_t)c->args.n_slabs + 5u;
    s->d_cursor = (uint32_t*)dalloc(c, 256);
    s->d_events = (uint32_t*)dalloc(c, ((size_t)s->max_out + 1u) * 4u);
    s->d_rows = (double*)dalloc(c, (size_t)s->max_out * row * 8u);
    bool ok = s->d_cursor && s->d_events && s->d_rows;
    for (int k = 0; k < 2 && ok; ++k) {
      ok = cudaMallocHost(&s->h_events[k], ((size_t)s->max_out + 1u) * 4u) == cudaSuccess &&
           cudaMallocHost(&s->h_rows[k], (size_t)s->max_out * row * 8u) == cudaSuccess &&
           cudaMallocHost(&s->h_ctl[k], sizeof(DevCtl)) == cudaSuccess &&
           cudaMallocHost(&s->h_rel[k], 64) == cudaSuccess &&
           cudaEventCreateWithFlags(&s->ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      (void)cudaGetLastError();
      serve_free(s);
      return fail(c, ET_ERR_NOMEM, "serving buffers");
    }
    // the cursor starts at the completions already reported through et_poll_completed
    s->h_rel[0][0] = c->done_read;
    CUDA_TRY(c, cudaMemcpyAsync(s->d_cursor, s->h_rel[0], 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->serve = s;
  }
  *out = c->serve;
  return ET_OK;
}

et_status et_serve_submit(et_ctx* c, const et_primary* p, size_t n, uint32_t event,
                          const uint32_t reserve[3]) {
  if (!c) return ET_ERR_INVALID;
  ServeState* s = nullptr;
  et_status st = serve_state(c, &s);
  if (st != ET_OK) return st;
  if (!p || n == 0 || !reserve || event >= c->cfg.max_events)
    return fail(c, ET_ERR_INVALID, "et_serve_submit: bad request");
  for (int t = 0; t < 3; ++t)
    if (reserve[t] > c->cap) return fail(c, ET_ERR_CAPACITY, "et_serve_submit: reserve above capacity");
  ServeReq r;
  r.p.resize(n);
  memcpy(r.p.data(), p, n * sizeof(Primary));
  for (size_t i = 0; i < n; ++i)
    if (r.p[i].event != event) return fail(c, ET_ERR_INVALID, "et_serve_submit: primary of another event");
  r.event = event;
  for (int t = 0; t < 3; ++t) r.reserve[t] = reserve[t];
  s->pending.push_back(std::move(r));
  return ET_OK;
}

// Hand back the results of round `k` (complete: its event has been waited for).
static et_status serve_deliver(et_ctx* c, ServeState* s, uint64_t k, uint32_t* events,
                               double* rows, uint64_t cap, uint64_t* n_out, uint64_t* steps) {
  CUDA_TRY(c, cudaEventSynchronize(s->ev[k % 2]));
  timing_collect(c);
  const DevCtl& d = *s->h_ctl[k % 2];
  const uint32_t st = d.status;
  if (st & ST_TIMEOUT) return fail(c, ET_ERR_TIMEOUT, "device wait timed out (status 0x%x)", st);
  if (st & ST_CAPACITY) return fail(c, ET_ERR_CAPACITY, "track buffer capacity %u exceeded", c->cap);
  if (st & ST_BAD_PRIMARY) return fail(c, ET_ERR_INVALID, "invalid device-side primary (skipped)");
  const uint32_t n = s->h_events[k % 2][s->max_out];
  const size_t row = (size_t)c->args.n_slabs + 5u;
  if (n > cap) return fail(c, ET_ERR_CAPACITY, "et_serve_round: result buffer shorter than %u", n);
  for (uint32_t j = 0; j < n; ++j) {
    const uint32_t e = s->h_events[k % 2][j];
    events[j] = e;
    memcpy(rows + (size_t)j * row, s->h_rows[k % 2] + (size_t)j * row, row * 8u);
    auto it = s->inflight.find(e);
    if (it != s->inflight.end()) {
      for (int t = 0; t < 3; ++t) s->reserved[t] -= it->second[t];
      s->inflight.erase(it);
    }
  }
  *n_out += n;
  const uint64_t all = d.steps[0] + d.steps[1] + d.steps[2];
  if (steps) *steps += all - s->steps_seen;
  s->steps_seen = all;
  const uint32_t* cur = d.cnt[d.iter % 3];
  s->last_pop = (uint64_t)cur[cw(EM)] + cur[cw(EP)] + cur[cw(GAM)];
  s->delivered = k + 1;
  return ET_OK;
}

et_status et_serve_round(et_ctx* c, uint32_t iters, uint32_t* events, double* rows,
                         uint64_t cap, uint64_t* n_out, uint64_t* steps, uint32_t* in_flight) {
  if (!c || !n_out || (cap && (!events || !rows))) return ET_ERR_INVALID;
  ServeState* s = nullptr;
  et_status st = serve_state(c, &s);
  if (st != ET_OK) return st;
  *n_out = 0;
  if (steps) *steps = 0;
  if (cap < s->max_out) return fail(c, ET_ERR_INVALID, "et_serve_round: cap below %u", s->max_out);
  // 1. admission by reserved track slots (90 % of the capacity), in submission order
  s->batch.clear();
  while (!s->pending.empty()) {
    ServeReq& r = s->pending.front();
    bool fits = true;
    for (int t = 0; t < 3; ++t)
      if ((double)(s->reserved[t] + r.reserve[t]) > 0.9 * (double)c->cap) fits = false;
    if ((!fits && !s->inflight.empty()) || s->inflight.count(r.event)) break;
    for (int t = 0; t < 3; ++t) s->reserved[t] += r.reserve[t];
    s->inflight[r.event] = {r.reserve[0], r.reserve[1], r.reserve[2]};
    s->batch.insert(s->batch.end(), r.p.begin(), r.p.end());
    s->pending.pop_front();
  }
  const uint64_t k = s->issued;
  if (!s->batch.empty()) {
    st = et_inject(c, reinterpret_cast<const et_primary*>(s->batch.data()), s->batch.size());
    if (st != ET_OK) return st;
  }
  // 2. the round's iterations: the persistent kernel stops after `iters` of them; with
  // the hybrid driver, a round whose stream was last seen at or above the switch-over
  // population runs the graph of per-type step kernels instead (both stop where the
  // population crosses it, after at least one iteration)
  const bool hybrid = c->cfg.driver == ET_DRIVER_HYBRID;
  if (iters > 0 && !s->inflight.empty() && hybrid && s->last_pop >= c->args.hybrid_t) {
    void* pr[] = {(void*)&c->args, (void*)&iters};
    st = launch(c, (const void*)k_round_stop, 1, 1, 0, pr);
    if (st != ET_OK) return st;
    if (!c->gexec) {
      st = build_graph(c);
      if (st != ET_OK) return st;
    }
    EventPair* ev = timing_begin(c);
    CUDA_TRY(c, cudaGraphLaunch(c->gexec, c->stream));
    timing_end(c, ev);
    c->launches += 1;
  } else if (iters > 0 && !s->inflight.empty()) {
    if (c->cfg.driver == ET_DRIVER_PERSISTENT || hybrid) {
      s->h_rel[k % 2][0] = iters;
      CUDA_TRY(c, cudaMemcpyAsync(&c->d_ctl->stop_rel, s->h_rel[k % 2], 4, cudaMemcpyHostToDevice,
                                  c->stream));
      int fault = c->fault_skip_block;
      void* params[] = {(void*)&c->args, (void*)&fault};
      const void* fn = c->ks.persistent[c->cfg.instrument ? 1 : 0][c->dense ? 1 : 0];
      EventPair* ev = timing_begin(c);
      CUDA_TRY(c, cudaLaunchCooperativeKernel(fn, dim3(c->grid_persistent), dim3(c->block),
                                              params, c->smem_all, c->stream));
      timing_end(c, ev);
      c->launches += 1;
    } else {
      // the other drivers read the counts back between launches: a synchronous round
      et_iter_stats tot;
      uint64_t ni = 0;
      st = et_run_until_empty(c, iters, &tot, &ni);
      if (st != ET_OK) return st;
    }
  }
  // 3. collect the completed events, copy them and the counters to pinned host memory
  st = scan_done(c);
  if (st != ET_OK) return st;
  {
    void* params[] = {(void*)&c->args, (void*)&s->d_cursor, (void*)&s->d_events,
                      (void*)&s->d_rows, (void*)&s->max_out};
    st = launch(c, (const void*)k_serve_collect, 1, 128, 0, params);
    if (st != ET_OK) return st;
  }
  const size_t row = (size_t)c->args.n_slabs + 5u;
  CUDA_TRY(c, cudaMemcpyAsync(s->h_events[k % 2], s->d_events, ((size_t)s->max_out + 1u) * 4u,
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(s->h_rows[k % 2], s->d_rows, (size_t)s->max_out * row * 8u,
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(s->h_ctl[k % 2], c->d_ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost,
                              c->stream));
  CUDA_TRY(c, cudaEventRecord(s->ev[k % 2], c->stream));
  s->issued = k + 1;
  // 4. the round before this one: wait for it and hand back its results
  if (k >= 1 && s->delivered < k) {
    st = serve_deliver(c, s, k - 1, events, rows, cap, n_out, steps);
    if (st != ET_OK) return st;
  }
  if (in_flight) *in_flight = (uint32_t)(s->inflight.size() + s->pending.size());
  return ET_OK;
}

et_status et_serve_flush(et_ctx* c, uint32_t* events, double* rows, uint64_t cap,
                         uint64_t* n_out, uint64_t* steps, uint32_t* in_flight) {
  if (!c || !n_out || (cap && (!events || !rows))) return ET_ERR_INVALID;
  ServeState* s = nullptr;
  et_status st = serve_state(c, &s);
  if (st != ET_OK) return st;
  *n_out = 0;
  if (steps) *steps = 0;
  if (cap < s->max_out) return fail(c, ET_ERR_INVALID, "et_serve_flush: cap below %u", s->max_out);
  if (s->delivered < s->issued) {
    st = serve_deliver(c, s, s->issued - 1, events, rows, cap, n_out, steps);
    if (st != ET_OK) return st;
  }
  if (in_flight) *in_flight = (uint32_t)(s->inflight.size() + s->pending.size());
  return ET_OK;
}

et_status et_serve_capacity(et_ctx* c, uint32_t* max_results) {
  if (!c || !max_results) return ET_ERR_INVALID;
  ServeState* s = nullptr;
  et_status st = serve_state(c, &s);
  if (st != ET_OK) return st;
  *max_results = s->max_out;
  return ET_OK;
}

}  // extern "C"
