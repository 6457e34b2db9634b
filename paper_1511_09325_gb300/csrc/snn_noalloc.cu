// snn_noalloc.cu -- one neuron-update step on caller-owned buffers, with no
// allocation of any kind.
//
// Some callers cannot let a library call cudaMalloc: a process whose device
// memory is already reserved by another framework's caching allocator or a
// fixed arena, or a real-time loop that cannot afford the implicit
// synchronisation of an allocation.  For them the
// neuron-update kernel of snn_step.cu runs here on their own state arrays; its
// scratch (step counter, spike-list cursor, per-block partial sums and the
// per-column spike counters) lives in one file-scope device array below, of a
// fixed size, which every GPU that loads the library holds until exit.
#include <cstddef>
#include <mutex>
#include <string>

#include "snn_internal.h"

using namespace snn;

namespace {

constexpr int kNoAllocMaxCols = 16384;   // columns per call
constexpr int kNoAllocMaxBlocks = 2048;  // update blocks per call
constexpr int kMaxDevices = 64;

// Byte offsets inside the scratch array.
constexpr size_t kOffCtl = 0;                                       // Ctl
constexpr size_t kOffCnt = 256;                                     // u32 spike count
constexpr size_t kOffExtSum = 264;                                  // u64 sum of ext_part
constexpr size_t kOffExt = 512;                                     // u64[blocks]
constexpr size_t kOffSpk = kOffExt + 8 * (size_t)kNoAllocMaxBlocks;  // u64[blocks]
constexpr size_t kOffRc = kOffSpk + 8 * (size_t)kNoAllocMaxBlocks;   // u64[blocks]
constexpr size_t kOffCol = kOffRc + 8 * (size_t)kNoAllocMaxBlocks;   // u64[2 * columns]
constexpr size_t kScratchBytes = kOffCol + 16 * (size_t)kNoAllocMaxCols;  // 311 808 B

static_assert(sizeof(Ctl) <= kOffCnt, "control block overlaps the counters");

__device__ __align__(256) unsigned char g_update_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on `dev` (which must be current).  The
// first call on a device looks it up; later calls reuse it, which assumes the
// device is not reset (cudaDeviceReset reloads the module) in between.
int scratch_address(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return fail_global(SNN_EINVAL, "device ordinal out of range");
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_update_scratch);
    if (e != cudaSuccess)
      return fail_global(SNN_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return SNN_OK;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

extern "C" int snn_update_noalloc(int grid_w, int grid_h, const snn_neuron_params* neuron,
                                  uint64_t seed, int64_t step, float* v, float* c,
                                  uint8_t* refractory, int32_t* input, uint32_t* spikes,
                                  int64_t* n_spikes, int64_t* ext_events,
                                  unsigned long long* col_counts, void* cuda_stream) {
  std::string why;
  const int vrc = validate_neuron_params(neuron, &why);
  if (vrc != SNN_OK) return fail_global(vrc, why);
  if (grid_w < 1 || grid_h < 1) return fail_global(SNN_EINVAL, "grid must be at least 1x1");
  const long long ncol = (long long)grid_w * grid_h;
  if (ncol > kNoAllocMaxCols)
    return fail_global(SNN_EINVAL, "snn_update_noalloc handles at most 16384 columns");
  if (step < 0 || step > 0xFFFFFFFFLL) return fail_global(SNN_EINVAL, "step must be in 0..2^32-1");
  if (!v || !c || !refractory || !input || !spikes || !n_spikes)
    return fail_global(SNN_EINVAL, "null buffer");
  if (!aligned(v, 16) || !aligned(c, 16) || !aligned(input, 16) || !aligned(refractory, 4) ||
      !aligned(spikes, 4) || !aligned(col_counts, 8))
    return fail_global(SNN_EINVAL,
                       "v, c, input must be 16-byte, refractory and spikes 4-byte, col_counts "
                       "8-byte aligned");

  HostTables tb;
  int rc = make_neuron_tables(*neuron, &tb, &why);
  if (rc != SNN_OK) return fail_global(rc, why);
  int dev = 0, num_sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail_global(SNN_ECUDA, std::string("device query: ") + cudaGetErrorString(e));
  unsigned char* base = nullptr;
  rc = scratch_address(dev, &base);
  if (rc != SNN_OK) return rc;

  const long long N = ncol * neuron->n_per_col;
  int grid = update_grid(N, num_sms);
  if (grid > kNoAllocMaxBlocks) grid = kNoAllocMaxBlocks;

  StepParams p{};
  p.N = N;
  p.npc = neuron->n_per_col;
  p.nexc = neuron->n_exc;
  p.W = grid_w;
  p.H = grid_h;
  p.nslot = 1;
  p.ncol = (int)ncol;
  p.seed_lo = (uint32_t)(seed & 0xFFFFFFFFu);
  p.seed_hi = (uint32_t)(seed >> 32);
  p.theta = neuron->theta;
  p.vr = neuron->v_reset;
  p.dc = neuron->dc;
  p.pvv = tb.pvv;
  p.pcc = tb.pcc;
  p.pvc_e = tb.pvc[0];
  p.pvc_i = tb.pvc[1];
  p.jx = tb.jx;
  p.nref = tb.nref;
  p.n_pois_thr = tb.n_pois_thr;
  for (int k = 0; k <= kMaxPoisThr; ++k) p.pois_thr[k] = tb.pois_thr[k];
  for (int k = 0; k < 256; ++k) p.pois_guide[k] = tb.pois_guide[k];
  p.V = v;
  p.C = c;
  p.R = refractory;
  p.acc = input;
  p.ids = spikes;
  p.ctl = reinterpret_cast<Ctl*>(base + kOffCtl);
  p.cnt = reinterpret_cast<unsigned*>(base + kOffCnt);
  p.ext_part = reinterpret_cast<unsigned long long*>(base + kOffExt);
  p.spk_part = reinterpret_cast<unsigned long long*>(base + kOffSpk);
  p.rcnt = reinterpret_cast<unsigned long long*>(base + kOffRc);
  p.colcnt = reinterpret_cast<unsigned long long*>(base + kOffCol);
  p.rec = nullptr;  // no spike records: the spike list is the output
  p.rec_region = 0;

  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // everything the kernel accumulates into starts at zero; the step index
  // goes into the control block
  const long long t = step;
  e = cudaMemsetAsync(base, 0, kOffCol + 16 * (size_t)ncol, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(base + kOffCtl + offsetof(Ctl, t), &t, sizeof(t), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_update(p, grid, st);
  if (e == cudaSuccess)
    e = launch_sum_parts(p.ext_part, grid, reinterpret_cast<unsigned long long*>(base + kOffExtSum), st);
  unsigned n = 0u;
  unsigned long long ext = 0ull;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, base + kOffCnt, sizeof(n), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&ext, base + kOffExtSum, sizeof(ext), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && col_counts)
    e = cudaMemcpyAsync(col_counts, base + kOffCol, 16 * (size_t)ncol, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess)
    return fail_global(SNN_ECUDA, std::string("snn_update_noalloc: ") + cudaGetErrorString(e));
  *n_spikes = (int64_t)n;
  if (ext_events) *ext_events = (int64_t)ext;
  return SNN_OK;
}
