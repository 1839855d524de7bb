// et_transport_noalloc: the whole transport of one batch of primaries without any
// device allocation.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool or under a memory budget that forbids cudaMalloc, code that
// must not synchronise the device (cudaMalloc/cudaFree can), and plug-ins that are
// handed a stream and buffers but no allocator.  For them this entry point keeps all
// of its scratch -- the dense double buffers of the three particle types, the device
// control block, the iteration count log and the staged geometry and tables -- in one
// file-scope device array of fixed size, reserved when the module holding it is loaded
// on a device and held by that device until the process exits.  The caller passes the inputs
// (primaries in device memory, geometry and tables in host memory) and the device
// output buffers (scores, ledger).
//
// The array is shared by every call: its contents are whatever the last call left, so
// each call clears what must start at zero (the control block) and overwrites the
// rest before reading it.  Calls whose work overlaps on the GPU (on different streams,
// or from different host threads) race on the array and give wrong results.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "et.h"
#include "kernels.cuh"
#include "registry.h"

namespace {

using namespace et;

constexpr uint32_t NA_CAP = ET_NOALLOC_MAX_TRACKS;   // slots per type and buffer half
constexpr uint32_t NA_MAX_ITERS = ET_NOALLOC_MAX_ITERS;
constexpr size_t NA_HALF = (size_t)NA_CAP * 64u;      // bytes of one buffer half
constexpr size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }
constexpr size_t OFF_TRK = 0;                                           // 6 halves
constexpr size_t OFF_CTL = align256(OFF_TRK + 6u * NA_HALF);            // DevCtl
constexpr size_t OFF_LOG = align256(OFF_CTL + sizeof(DevCtl));          // counts log
constexpr size_t OFF_TOT = align256(OFF_LOG + (size_t)NA_MAX_ITERS * 12u);
constexpr size_t OFF_BREM = align256(OFF_TOT + (size_t)MAX_MAT * NBINS * sizeof(float2));
constexpr size_t OFF_CP = align256(OFF_BREM + (size_t)MAX_MAT * NBINS * sizeof(float2));
constexpr size_t OFF_PLANES = align256(OFF_CP + (size_t)MAX_MAT * NBINS * sizeof(float4));
constexpr size_t OFF_MAT = align256(OFF_PLANES + (MAX_SLABS + 1) * sizeof(float));
constexpr size_t NA_USED = align256(OFF_MAT + MAX_SLABS);
static_assert(NA_USED <= ET_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the stated size");

}  // namespace

// The scratch array.  In host code its name is only a host-side stand-in: the device
// address comes from cudaGetSymbolAddress (below), once per device.
static __device__ __align__(256) unsigned char et_noalloc_scratch[ET_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_lock;
unsigned char* g_scratch[NA_MAX_DEVICES] = {};

et_status na_fail(char* err, size_t len, et_status s, const char* msg, const char* detail = "") {
  if (err && len) snprintf(err, len, "%s%s", msg, detail);
  return s;
}

}  // namespace

extern "C" et_status et_transport_noalloc(
    uint32_t n_slabs, const double* thickness_mm, const uint8_t* material, float half_xy_mm,
    uint32_t n_materials, float log_emin, float inv_dlog, const float* sigma, const float* dedx,
    const et_primary* primaries_device, size_t n_primaries, uint64_t seed, uint32_t n_events,
    double* score_device, double* ledger_device, uint64_t* steps_out, void* cuda_stream,
    char* err, size_t err_len) {
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  // ---- sizes against the fixed maximum; arguments ----
  if (n_primaries > NA_CAP)
    return na_fail(err, err_len, ET_ERR_CAPACITY,
                   "et_transport_noalloc: more primaries than ET_NOALLOC_MAX_TRACKS");
  if (n_slabs < 1 || n_slabs > (uint32_t)MAX_SLABS || !thickness_mm || !material ||
      !(half_xy_mm > 0.0f) || n_materials < 1 || n_materials > (uint32_t)MAX_MAT || !sigma ||
      !dedx || !(inv_dlog > 0.0f) || n_events == 0 || !score_device || !ledger_device ||
      (seed >> 32) != 0 ||
      (n_primaries && !primaries_device) || ((uintptr_t)primaries_device & 15u))
    return na_fail(err, err_len, ET_ERR_INVALID, "et_transport_noalloc: invalid argument");

  // ---- once per device: the scratch array's device address ----
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
    (void)cudaGetLastError();
    return na_fail(err, err_len, ET_ERR_CUDA, "et_transport_noalloc: no usable CUDA device");
  }
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> g(g_setup_lock);
    if (!g_scratch[dev]) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, et_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return na_fail(err, err_len, ET_ERR_CUDA, "et_transport_noalloc: cudaGetSymbolAddress: ",
                       cudaGetErrorString(e));
      }
      g_scratch[dev] = static_cast<unsigned char*>(p);
    }
    base = g_scratch[dev];
  }

  // ---- geometry and tables in host stack arrays, then into the scratch ----
  float planes[MAX_SLABS + 1];
  uint8_t mat[MAX_SLABS];
  double z = 0.0;
  planes[0] = 0.0f;
  for (uint32_t s = 0; s < n_slabs; ++s) {
    if (!(thickness_mm[s] > 0.0) || !std::isfinite(thickness_mm[s]) || material[s] >= n_materials)
      return na_fail(err, err_len, ET_ERR_INVALID, "et_transport_noalloc: bad slab");
    z = z + thickness_mm[s];
    planes[s + 1] = (float)z;
    mat[s] = material[s];
  }
  float2 tot[MAX_MAT * NBINS], brem[MAX_MAT * NBINS];
  float4 cp[MAX_MAT * NBINS];
  float dedx_h[MAX_MAT] = {0.0f, 0.0f, 0.0f, 0.0f};
  const uint32_t nn = NBINS + 1;
  for (uint32_t m = 0; m < n_materials; ++m) {
    const float* T = sigma + (size_t)m * 5 * nn;
    if (!(dedx[m] > 0.0f)) return na_fail(err, err_len, ET_ERR_INVALID, "et_transport_noalloc: dedx");
    for (int i = 0; i < NBINS; ++i) {
      const float* C = T;
      const float* P = T + nn;
      const float* S = T + 3 * nn;
      const float* B = T + 4 * nn;
      tot[m * NBINS + i] = make_float2(S[i], S[i + 1] - S[i]);
      cp[m * NBINS + i] = make_float4(C[i], C[i + 1] - C[i], P[i], P[i + 1] - P[i]);
      brem[m * NBINS + i] = make_float2(B[i], B[i + 1] - B[i]);
    }
    dedx_h[m] = dedx[m];
  }

  Args a;
  memset(&a, 0, sizeof a);
  for (int t = 0; t < 3; ++t)
    for (int h = 0; h < 2; ++h) a.trk[t][h] = (char*)(base + OFF_TRK + (size_t)(2 * t + h) * NA_HALF);
  a.cap = NA_CAP;
  a.ctl = (DevCtl*)(base + OFF_CTL);
  a.counts_log = (uint32_t*)(base + OFF_LOG);
  a.max_iters = NA_MAX_ITERS;
  a.n_slabs = n_slabs;
  a.score = score_device;
  a.ledger = ledger_device;
  a.max_events = n_events;
  a.n_mat = n_materials;
  a.tab_tot = (const float2*)(base + OFF_TOT);
  a.tab_brem = (const float2*)(base + OFF_BREM);
  a.tab_cp = (const float4*)(base + OFF_CP);
  a.planes = (const float*)(base + OFF_PLANES);
  a.mat = (const uint8_t*)(base + OFF_MAT);
  a.half_xy = half_xy_mm;
  a.log_emin = log_emin;
  a.inv_dlog = inv_dlog;
  for (int m = 0; m < MAX_MAT; ++m) a.dedx[m] = dedx_h[m];
  a.seed_lo = (uint32_t)seed;
  a.timeout_ns = 2000000000ull;

  DevCtl ctl0;
  memset(&ctl0, 0, sizeof ctl0);
  ctl0.stop_iter = NA_MAX_ITERS;
  const size_t nb = (size_t)n_materials * NBINS;
#define NA_TRY(call)                                                                         \
  do {                                                                                       \
    const cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                                 \
      (void)cudaGetLastError();                                                              \
      return na_fail(err, err_len, ET_ERR_CUDA, "et_transport_noalloc: ", cudaGetErrorString(e_)); \
    }                                                                                        \
  } while (0)
  NA_TRY(cudaMemcpyAsync(a.ctl, &ctl0, sizeof ctl0, cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync((void*)a.planes, planes, (n_slabs + 1) * sizeof(float), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync((void*)a.mat, mat, n_slabs, cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync((void*)a.tab_tot, tot, nb * sizeof(float2), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync((void*)a.tab_brem, brem, nb * sizeof(float2), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemcpyAsync((void*)a.tab_cp, cp, nb * sizeof(float4), cudaMemcpyHostToDevice, stream));
  NA_TRY(cudaMemsetAsync(score_device, 0, (size_t)n_events * n_slabs * sizeof(double), stream));
  NA_TRY(cudaMemsetAsync(ledger_device, 0, (size_t)n_events * 5 * sizeof(double), stream));

  // dense double buffer, AoS layout, strict mode
  KernelSet ks;
  memset(&ks, 0, sizeof ks);
  et_register_kernels_0_0(&ks);
  if (n_primaries) {
    uint32_t n = (uint32_t)n_primaries;
    const Primary* dp = reinterpret_cast<const Primary*>(primaries_device);
    void* params[] = {(void*)&a, (void*)&dp, (void*)&n};
    NA_TRY(cudaLaunchKernel(ks.inject[1], dim3((n + 255) / 256), dim3(256), params, 0, stream));
  }
  const void* fn = ks.persistent[0][1];
  const int block = 256;
  const size_t smem = tables_bytes_aligned((int)n_materials) + (size_t)(block / 32) * queue_bytes_per_warp();
  NA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0, sms = 0;
  NA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, block, smem));
  NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (occ < 1) return na_fail(err, err_len, ET_ERR_CUDA, "et_transport_noalloc: kernel does not fit");
  int no_fault = -1;
  void* pparams[] = {(void*)&a, (void*)&no_fault};
  NA_TRY(cudaLaunchCooperativeKernel(fn, dim3(occ * sms), dim3(block), pparams, smem, stream));

  DevCtl out;
  NA_TRY(cudaMemcpyAsync(&out, a.ctl, sizeof out, cudaMemcpyDeviceToHost, stream));
  NA_TRY(cudaStreamSynchronize(stream));
#undef NA_TRY
  if (out.status & ST_TIMEOUT) return na_fail(err, err_len, ET_ERR_TIMEOUT, "et_transport_noalloc: device wait timed out");
  if (out.status & ST_CAPACITY)
    return na_fail(err, err_len, ET_ERR_CAPACITY,
                   "et_transport_noalloc: more active tracks than ET_NOALLOC_MAX_TRACKS");
  if (out.status & ST_BAD_PRIMARY)
    return na_fail(err, err_len, ET_ERR_INVALID, "et_transport_noalloc: invalid primary (skipped)");
  const uint32_t cur = out.iter % 3;
  if (out.status || out.cnt[cur][cw(EM)] + out.cnt[cur][cw(EP)] + out.cnt[cur][cw(GAM)] != 0)
    return na_fail(err, err_len, ET_ERR_CAPACITY,
                   "et_transport_noalloc: tracks left after ET_NOALLOC_MAX_ITERS iterations");
  if (steps_out) *steps_out = out.steps[0] + out.steps[1] + out.steps[2];
  if (err && err_len) err[0] = '\0';
  return ET_OK;
}
