// snn_api.cu -- the C ABI: net lifetime, graph-captured step loop, readback.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "snn_internal.h"

using namespace snn;

struct snn_net {
  // configuration
  int W = 0, H = 0, npc = 0, nexc = 0, K = 0, dmin = 0, ndel = 0, nslot = 0;
  int precision = 0, rowcap = 0, rec_size = 0, num_sms = 0, update_grid = 0;
  bool agg = true;
  int deliver_grid = 0;
  int tile = 1, ring = 0, win_cap = 0, desc_words = 8;  // delivery tiles and windows
  int part_cols = kMaxTileCols;
  size_t window_budget = 0;  // bytes of shared memory a delivery window may take
  unsigned min_items = 256;  // fewest items a delivery block takes
  unsigned win_items = kWinMinItems;  // fewest items of a windowed tile part
  unsigned cost_win = kCostWin, cost_part = kCostPart;  // range split's fixed costs
  long long N = 0, Npad = 0, ncol = 0;
  uint64_t seed = 0;
  snn_neuron_params neuron{};
  HostTables tables;
  StepParams sp{};
  // device memory
  void* syn = nullptr;
  uint8_t* bend = nullptr;
  float* V = nullptr;
  float* C = nullptr;
  uint8_t* R = nullptr;
  int32_t* acc = nullptr;
  uint32_t* desc = nullptr;               // spike descriptors
  uint32_t* vcol = nullptr;               // delivery order of the columns
  uint32_t* colv = nullptr;
  unsigned* hstatus = nullptr;            // status word (pinned, mapped)
  unsigned* hstatus_dev = nullptr;
  unsigned* cnt = nullptr;
  unsigned* ccnt = nullptr;
  uint32_t* deg = nullptr;                 // out-degree per neuron (paper law)
  unsigned long long* syn_part = nullptr;  // synaptic events per update block
  long long total_syn = 0;                 // synapses of the whole net
  int connectivity = SNN_CONN_FIXED;
  unsigned* isum = nullptr;
  unsigned* gsum = nullptr;
  Ctl* ctl = nullptr;
  unsigned long long* rec = nullptr;
  long long rec_cap = 0;     // requested total record capacity
  long long rec_region = 0;  // records per update block
  unsigned long long* rcnt = nullptr;
  unsigned long long* stage = nullptr;   // large drains on the device: ids then steps (u32)
  unsigned long long* dhdr = nullptr;    // drain header (device, 4 words)
  unsigned long long* hhdr = nullptr;    // drain header (pinned, mapped)
  unsigned long long* hhdr_dev = nullptr;
  uint32_t* hmap = nullptr;              // small drains: ids then steps (pinned, mapped)
  uint32_t* hmap_dev = nullptr;
  long long hmap_cap = 0;                // records
  uint32_t* hstage = nullptr;            // large drains: ids then steps (pinned host)
  long long hstage_cap = 0;              // records
  unsigned long long* colcnt = nullptr;
  unsigned long long* ext_part = nullptr;
  unsigned long long* spk_part = nullptr;
  size_t device_bytes = 0;
  // execution
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaGraphExec_t graph_one = nullptr;
  cudaGraphExec_t graph_many = nullptr;
  int graph_many_steps = 64;
  long long rate_window_start = 0;
  bool in_batch = false;  // stepped only through its snn_batch
  // shard (snn_build_shard): geometry, the half step due next (0 update,
  // 1 delivery), and the received spike indices (pinned host stage, device
  // copy, and an event recorded once the ingest kernel has read them)
  ShardGeo sg{};
  int shard_phase = 0;
  uint32_t* ingest = nullptr;
  uint32_t* hingest = nullptr;
  long long ingest_cap = 0;
  cudaEvent_t ingest_ev = nullptr;
  std::string err;
};

namespace {

thread_local std::string g_err;

int fail(snn_net* net, int code, const std::string& msg) {
  if (net)
    net->err = msg;
  else
    g_err = msg;
  return code;
}

}  // namespace

namespace snn {

int fail_global(int code, const std::string& msg) { return fail(nullptr, code, msg); }

int validate_neuron_params(const snn_neuron_params* n, std::string* why) {
  auto bad = [&](const char* m) {
    *why = m;
    return SNN_EINVAL;
  };
  if (!n) return bad("null parameter struct");
  if (n->n_per_col < 2 || n->n_per_col > 2048) return bad("n_per_col must be in 2..2048");
  if (n->n_exc < 0 || n->n_exc > n->n_per_col) return bad("n_exc must be in 0..n_per_col");
  if (!(n->tau_m > 0.f) || !(n->tau_c > 0.f)) return bad("time constants must be positive");
  if (!(n->t_ref >= 0.f) || n->t_ref > 200.f) return bad("t_ref must be in 0..200 ms");
  if (!(n->nu_ext_kHz >= 0.f) || n->nu_ext_kHz > 40.f) return bad("nu_ext_kHz must be in 0..40");
  if (!std::isfinite(n->theta) || !std::isfinite(n->v_reset) || !std::isfinite(n->dc) ||
      !std::isfinite(n->gc_exc) || !std::isfinite(n->gc_inh) || !std::isfinite(n->j_ext_mV))
    return bad("non-finite neuron parameter");
  return SNN_OK;
}

}  // namespace snn

namespace {

int cuda_fail(snn_net* net, cudaError_t e, const char* what) {
  return fail(net, e == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define SNN_CUDA(net, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((net), e_, #call); \
  } while (0)

template <class T>
int dalloc(snn_net* net, T** p, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes ? bytes : 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(net, e == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA,
                "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  *p = static_cast<T*>(v);
  net->device_bytes += bytes;
  return SNN_OK;
}

void free_graphs(snn_net* net) {
  if (net->graph_one) cudaGraphExecDestroy(net->graph_one);
  if (net->graph_many) cudaGraphExecDestroy(net->graph_many);
  net->graph_one = net->graph_many = nullptr;
}

void release(snn_net* net) {
  free_graphs(net);
  if (net->hhdr) cudaFreeHost(net->hhdr);
  if (net->hmap) cudaFreeHost(net->hmap);
  if (net->hstage) cudaFreeHost(net->hstage);
  if (net->hstatus) cudaFreeHost(net->hstatus);
  if (net->ingest) cudaFree(net->ingest);
  if (net->hingest) cudaFreeHost(net->hingest);
  if (net->ingest_ev) cudaEventDestroy(net->ingest_ev);
  void* ptrs[] = {net->syn, net->bend, net->V, net->C, net->R, net->acc,
                  net->desc, net->vcol, net->colv, net->cnt, net->ccnt, net->deg, net->syn_part, net->isum, net->gsum, net->ctl, net->rec, net->rcnt, net->stage, net->dhdr, net->colcnt,
                  net->ext_part, net->spk_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (net->own_stream && net->stream) cudaStreamDestroy(net->stream);
}

int validate(int gw, int gh, const snn_neuron_params* n, const snn_synapse_params* s,
             int precision, std::string* why) {
  auto bad = [&](const char* m) {
    *why = m;
    return SNN_EINVAL;
  };
  if (!n || !s) return bad("null parameter struct");
  if (gw < 1 || gh < 1) return bad("grid must be at least 1x1");
  if (gw > kMaxGridSide || gh > kMaxGridSide) return bad("grid_w and grid_h must be at most 16383");
  const int nrc = snn::validate_neuron_params(n, why);
  if (nrc != SNN_OK) return nrc;
  if (s->k_out < 1) return bad("k_out must be positive");
  if (!(s->frac_local >= 0.f && s->frac_local <= 1.f)) return bad("frac_local must be in [0, 1]");
  if (!(s->lambda_cols > 0.f)) return bad("lambda_cols must be positive");
  if (s->stencil_radius < 1 || s->stencil_radius > 3) return bad("stencil_radius must be 1..3");
  if (s->d_min < 1 || s->d_max < s->d_min || s->d_max > kMaxDelays)
    return bad("delays must satisfy 1 <= d_min <= d_max <= 32");
  if (s->periodic != 1) return bad("only periodic grids are supported");
  if (!std::isfinite(s->w_exc_mV) || !std::isfinite(s->w_inh_mV) || !std::isfinite(s->w_cv))
    return bad("non-finite weight parameter");
  if (precision != SNN_EXACT_F32W && precision != SNN_EXACT_F16W) return bad("unknown precision");
  const int ndel = s->d_max - s->d_min + 1;
  if (s->connectivity != SNN_CONN_FIXED && s->connectivity != SNN_CONN_PAPER)
    return bad("connectivity must be SNN_CONN_FIXED or SNN_CONN_PAPER");
  if (s->connectivity == SNN_CONN_FIXED &&
      (s->k_out + (kSlotUnit - 1) * ndel + kSlotUnit - 1) / kSlotUnit > 255)
    return bad("k_out too large for 8-bit bucket ends");
  if (s->connectivity == SNN_CONN_PAPER &&
      (!(s->p_local >= 0.f && s->p_local <= 1.f) || !(s->remote_a >= 0.f && s->remote_a <= 1.f) ||
       !(s->remote_sigma > 0.f) || !std::isfinite(s->remote_sigma) || !(s->remote_cutoff > 0.f)))
    return bad("paper law: p_local and remote_a in [0, 1], remote_sigma and remote_cutoff > 0");
  if (s->connectivity == SNN_CONN_PAPER &&
      (double)s->remote_a * std::exp(-16.0 / (2.0 * (double)s->remote_sigma * s->remote_sigma)) >=
          (double)s->remote_cutoff)
    return bad("the paper law keeps offsets beyond the 7x7 stencil");
  const long long N = (long long)gw * gh * n->n_per_col;
  if (N >= (1LL << 31) - 4) return bad("too many neurons");
  return SNN_OK;
}

// min(floor(2^32 / d), 2^32 - 1): the multiplier of the kernels' divisions.
uint32_t recip32(uint32_t d) {
  const unsigned long long m = (1ull << 32) / (unsigned long long)d;
  return m > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)m;
}

// Delivery tiles: the largest square tile (side <= kMaxTile) whose window --
// the tile plus a ring of kWindowRing columns, clipped to the grid -- fits the
// shared memory budget of a delivery block: one block per SM for a net of its
// own, two per SM in the batch kernel.  Measured at 96x96 (FP16, Down, middle
// and Up states): a 6x6 tile without ring (80 % of the synapses land in the
// window, each column is flushed once per part) beats a 4x4 tile with a ring
// of one (88 %, but 36 window columns flushed per 16 columns of spikes) by
// 13 %, 17 % and 3 %; 5x5 and 4x4 tiles without ring and 3x3 with a ring are
// slower still.
constexpr size_t kWindowBudget = 196 * 1024;
constexpr size_t kBatchWindowBudget = 96 * 1024;
// Fewest items a delivery block takes (fewer blocks run when a step has few
// items).  Measured on the 64-net batch: 256 per block beat 512, 2048 and
// 8192, so members use the same value as nets of their own.
constexpr unsigned kMinItems = 256;
constexpr unsigned kBatchMinItems = 256;
// Most columns of a delivery part without window (runs of sparse tiles): its
// (column, bucket) and neighbour tables take part_cols * (d_max + 64) words
// of shared memory beside the window.
constexpr int kPartCols = kMaxTileCols;
constexpr int kBatchPartCols = 16;
constexpr int kWindowRing = 0;

void choose_tiles(snn_net* net) {
  net->ring = kWindowRing;
  int t = std::min(kMaxTile, std::max(net->W, net->H));
  for (; t > 1; --t) {
    const size_t ww = (size_t)std::min(t + 2 * net->ring, net->W);
    const size_t wh = (size_t)std::min(t + 2 * net->ring, net->H);
    if (ww * wh * (size_t)net->npc * 4 <= net->window_budget) break;
  }
  net->tile = t;
  net->part_cols = std::max(net->part_cols, t * t);
  const long long ww = std::min(t + 2 * net->ring, net->W);
  const long long wh = std::min(t + 2 * net->ring, net->H);
  net->win_cap = (int)((ww * wh * net->npc + 3) / 4 * 4);
}

// Virtual (delivery) order of the columns: tile by tile, tiles and the
// columns inside a tile in row-major order.  vcol[v] = real column.
void column_order(int W, int H, int T, std::vector<uint32_t>* vcol, std::vector<uint32_t>* colv) {
  vcol->assign((size_t)W * H, 0u);
  colv->assign((size_t)W * H, 0u);
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      const int tr = y / T, tc = x / T;
      const int th = std::min(T, H - tr * T), tw = std::min(T, W - tc * T);
      const long long v = (long long)tr * T * W + (long long)tc * th * T +
                          (long long)(y - tr * T) * tw + (x - tc * T);
      const uint32_t c = (uint32_t)(y * W + x);
      (*vcol)[(size_t)v] = c;
      (*colv)[c] = (uint32_t)v;
    }
}

// A kernel found inconsistent counts: the net's stepping is no longer exact.
int check_status(snn_net* net) {
  const unsigned st = net->hstatus ? *reinterpret_cast<volatile unsigned*>(net->hstatus) : 0u;
  if (st & kStatusIngest)
    return fail(net, SNN_ESTATE,
                "a shard received a spike index beyond the network or more spikes of one column "
                "than it has neurons; the net's state is no longer exact");
  if (st != 0u)
    return fail(net, SNN_ESTATE,
                "a delivery found item counts that disagree with the spike lists; the net's "
                "state is no longer exact");
  return SNN_OK;
}

int capture(snn_net* net, int steps, cudaGraphExec_t* out) {
  cudaGraph_t g = nullptr;
  SNN_CUDA(net, cudaStreamBeginCapture(net->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int s = 0; s < steps && le == cudaSuccess; ++s) {
    le = launch_update(net->sp, net->update_grid, net->stream);
    if (le == cudaSuccess) le = launch_deliver(net->sp, net->precision, net->deliver_grid, net->stream);
  }
  cudaError_t ee = cudaStreamEndCapture(net->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(net, le, "kernel launch during capture");
  }
  if (ee != cudaSuccess) return cuda_fail(net, ee, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) return cuda_fail(net, ie, "cudaGraphInstantiate");
  return SNN_OK;
}

void fill_step_params(snn_net* net) {
  StepParams& p = net->sp;
  const HostTables& t = net->tables;
  p.N = net->N;
  p.npc = net->npc;
  p.nexc = net->nexc;
  p.W = net->W;
  p.H = net->H;
  p.K = net->K;
  p.dmin = net->dmin;
  p.ndel = net->ndel;
  p.nslot = net->nslot;
  p.rowcap = net->rowcap;
  p.ncol = (int)net->ncol;
  p.agg = net->agg ? 1 : 0;
  p.tile = net->tile;
  p.part_cols = net->part_cols;
  p.ring = net->ring;
  p.win_cap = net->win_cap;
  p.desc_words = net->desc_words;
  p.min_items = net->min_items;
  p.win_items = net->win_items;
  p.cost_win = net->cost_win;
  p.cost_part = net->cost_part;
  p.npc_m = recip32((uint32_t)net->npc);
  p.w_m = recip32((uint32_t)net->W);
  p.seed_lo = (uint32_t)(net->seed & 0xFFFFFFFFu);
  p.seed_hi = (uint32_t)(net->seed >> 32);
  p.pvv = t.pvv;
  p.pcc = t.pcc;
  p.pvc_e = t.pvc[0];
  p.pvc_i = t.pvc[1];
  p.jx = t.jx;
  p.nref = t.nref;
  p.n_pois_thr = t.n_pois_thr;
  std::memcpy(p.pois_thr, t.pois_thr, sizeof(p.pois_thr));
  std::memcpy(p.pois_guide, t.pois_guide, sizeof(p.pois_guide));
  p.V = net->V;
  p.C = net->C;
  p.R = net->R;
  p.acc = net->acc;
  p.ids = nullptr;
  p.desc = net->desc;
  p.vcol = net->vcol;
  p.colv = net->colv;
  p.hstatus = net->hstatus_dev;
  p.cnt = net->cnt;
  p.ccnt = net->ccnt;
  // a shard keeps the out-degree of its rows (synapses into its own columns)
  // for snn_row_lengths; its spikes count the full k_out synaptic events
  p.deg = net->sg.on ? nullptr : net->deg;
  p.syn_part = net->syn_part;
  p.sg = net->sg;
  p.isum = net->isum;
  p.gsum = net->gsum;
  p.bend = net->bend;
  p.syn = net->syn;
  p.ctl = net->ctl;
  p.rec = net->rec;
  p.rec_region = net->rec_region;
  p.rcnt = net->rcnt;
  p.colcnt = net->colcnt;
  p.ext_part = net->ext_part;
  p.spk_part = net->spk_part;
}

int build_impl(snn_net* net, int gw, int gh, const snn_neuron_params* np,
               const snn_synapse_params* sp, uint64_t seed, int precision) {
  std::string why;
  int rc = validate(gw, gh, np, sp, precision, &why);
  if (rc != SNN_OK) return fail(net, rc, why);
  net->W = gw;
  net->H = gh;
  net->npc = np->n_per_col;
  net->nexc = np->n_exc;
  net->K = sp->k_out;
  net->dmin = sp->d_min;
  net->ndel = sp->d_max - sp->d_min + 1;
  net->nslot = sp->d_max + 1;
  net->precision = precision;
  net->seed = seed;
  net->neuron = *np;
  net->ncol = (long long)gw * gh;
  net->N = net->ncol * np->n_per_col;
  net->Npad = (net->N + 3) / 4 * 4;
  net->rec_size = precision == SNN_EXACT_F16W ? 4 : 8;
  net->rowcap = (sp->k_out + (kSlotUnit - 1) * net->ndel + kSlotUnit - 1) / kSlotUnit * kSlotUnit;
  net->rec_cap = 1LL << 24;
  rc = make_host_tables(*np, *sp, precision, &net->tables, &why);
  if (rc != SNN_OK) return fail(net, rc, why);
  net->sp.theta = np->theta;
  net->sp.vr = np->v_reset;
  net->sp.dc = np->dc;

  int dev = 0;
  SNN_CUDA(net, cudaGetDevice(&dev));
  SNN_CUDA(net, cudaDeviceGetAttribute(&net->num_sms, cudaDevAttrMultiProcessorCount, dev));
  net->update_grid = update_grid(net->N, net->num_sms);
  choose_tiles(net);
  net->desc_words = net->ndel <= 28 ? 8 : 16;
  fill_step_params(net);
  net->deliver_grid = deliver_grid(net->sp, precision, net->num_sms);
  if (net->deliver_grid < 1) return fail(net, SNN_ECUDA, "delivery kernel does not fit on the device");
  net->rec_region = (net->rec_cap + net->update_grid - 1) / net->update_grid;

  net->connectivity = sp->connectivity;
  BuildParams bp{};
  bp.N = net->N;
  bp.npc = net->npc;
  bp.nexc = net->nexc;
  bp.W = net->W;
  bp.H = net->H;
  bp.K = net->K;
  bp.k_local = net->tables.k_local;
  bp.dmin = net->dmin;
  bp.ndel = net->ndel;
  bp.n_off = net->tables.n_off;
  bp.seed_lo = (uint32_t)(seed & 0xFFFFFFFFu);
  bp.seed_hi = (uint32_t)(seed >> 32);
  std::memcpy(bp.stencil_thr, net->tables.stencil_thr, sizeof(bp.stencil_thr));
  std::memcpy(bp.off_dx, net->tables.off_dx, sizeof(bp.off_dx));
  std::memcpy(bp.off_dy, net->tables.off_dy, sizeof(bp.off_dy));
  bp.n_poff = net->tables.n_poff;
  bp.n_cand = net->tables.n_cand;
  std::memcpy(bp.poff_thr, net->tables.poff_thr, sizeof(bp.poff_thr));
  bp.plocal_thr = net->tables.plocal_thr;
  std::memcpy(bp.poff_dx, net->tables.poff_dx, sizeof(bp.poff_dx));
  std::memcpy(bp.poff_dy, net->tables.poff_dy, sizeof(bp.poff_dy));
  bp.sg = net->sg;
  if ((rc = dalloc(net, &net->bend, (size_t)net->N * kBendStride))) return rc;
  net->total_syn = net->N * (long long)net->K;
  if (net->sg.on && (rc = dalloc(net, &net->deg, (size_t)net->N * 4))) return rc;
  if (net->connectivity == SNN_CONN_PAPER) {
    // count pass: bucket ends, out-degrees and the longest row, which sets
    // the row stride of the table
    unsigned* dmax = nullptr;
    if ((rc = dalloc(net, &net->deg, (size_t)net->N * 4))) return rc;
    if ((rc = dalloc(net, &dmax, 4))) return rc;
    net->device_bytes -= 4;
    unsigned max_units = 0u;
    bp.bend = net->bend;
    bp.deg = net->deg;
    bp.max_units = dmax;
    cudaError_t ce = cudaMemsetAsync(dmax, 0, 4, net->stream);
    if (ce == cudaSuccess) ce = launch_paper_count(bp, net->num_sms, net->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(&max_units, dmax, 4, cudaMemcpyDeviceToHost, net->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(net->stream);
    cudaFree(dmax);
    if (ce != cudaSuccess) return cuda_fail(net, ce, "connectivity count pass");
    if (max_units > 255u)
      return fail(net, SNN_EINVAL, "a row of the paper law needs more than 2040 slots");
    net->rowcap = (int)std::max(1u, max_units) * kSlotUnit;
    std::vector<uint32_t> deg((size_t)net->N);
    SNN_CUDA(net, cudaMemcpyAsync(deg.data(), net->deg, deg.size() * 4, cudaMemcpyDeviceToHost,
                                  net->stream));
    SNN_CUDA(net, cudaStreamSynchronize(net->stream));
    net->total_syn = 0;
    for (uint32_t d : deg) net->total_syn += d;
  }
  bp.rowcap = net->rowcap;
  const size_t syn_bytes = (size_t)net->N * net->rowcap * net->rec_size;
  if ((rc = dalloc(net, &net->syn, syn_bytes))) return rc;
  if ((rc = dalloc(net, &net->V, (size_t)net->Npad * 4))) return rc;
  if ((rc = dalloc(net, &net->C, (size_t)net->Npad * 4))) return rc;
  if ((rc = dalloc(net, &net->R, (size_t)net->Npad))) return rc;
  if ((rc = dalloc(net, &net->acc, (size_t)net->Npad * 4))) return rc;
  if ((rc = dalloc(net, &net->desc, (size_t)net->nslot * net->N * net->desc_words * 4))) return rc;
  if ((rc = dalloc(net, &net->vcol, (size_t)net->ncol * 4))) return rc;
  if ((rc = dalloc(net, &net->colv, (size_t)net->ncol * 4))) return rc;
  if ((rc = dalloc(net, &net->cnt, (size_t)net->nslot * 4))) return rc;
  if ((rc = dalloc(net, &net->ccnt, (size_t)net->nslot * net->ncol * 4))) return rc;
  if ((rc = dalloc(net, &net->isum, (size_t)net->ncol * 4))) return rc;
  if ((rc = dalloc(net, &net->gsum, (size_t)(net->ncol + 31) / 32 * 4))) return rc;
  if ((rc = dalloc(net, &net->ctl, sizeof(Ctl)))) return rc;
  if ((rc = dalloc(net, &net->rec, (size_t)net->rec_region * net->update_grid * 8))) return rc;
  if ((rc = dalloc(net, &net->rcnt, (size_t)net->update_grid * 8))) return rc;
  if ((rc = dalloc(net, &net->stage, (size_t)net->rec_region * net->update_grid * 8))) return rc;
  if ((rc = dalloc(net, &net->dhdr, 32))) return rc;
  SNN_CUDA(net, cudaHostAlloc(&net->hstatus, 16, cudaHostAllocMapped));
  SNN_CUDA(net, cudaHostGetDevicePointer(&net->hstatus_dev, net->hstatus, 0));
  *net->hstatus = 0u;
  SNN_CUDA(net, cudaHostAlloc(&net->hhdr, 32, cudaHostAllocMapped));
  SNN_CUDA(net, cudaHostGetDevicePointer(&net->hhdr_dev, net->hhdr, 0));
  net->hmap_cap = std::min<long long>(net->rec_region * net->update_grid, kMappedRecords);
  SNN_CUDA(net, cudaHostAlloc(&net->hmap, (size_t)net->hmap_cap * 8, cudaHostAllocMapped));
  SNN_CUDA(net, cudaHostGetDevicePointer(&net->hmap_dev, net->hmap, 0));
  if ((rc = dalloc(net, &net->colcnt, (size_t)net->ncol * 2 * 8))) return rc;
  if ((rc = dalloc(net, &net->ext_part, (size_t)net->update_grid * 8))) return rc;
  if ((rc = dalloc(net, &net->spk_part, (size_t)net->update_grid * 8))) return rc;
  if ((rc = dalloc(net, &net->syn_part, (size_t)net->update_grid * 8))) return rc;
  uint32_t* wtab = nullptr;
  if ((rc = dalloc(net, &wtab, net->tables.wtab.size() * 4))) return rc;
  net->device_bytes -= net->tables.wtab.size() * 4;

  std::vector<uint32_t> vcol, colv;
  column_order(net->W, net->H, net->tile, &vcol, &colv);
  cudaError_t e = cudaMemcpyAsync(wtab, net->tables.wtab.data(), net->tables.wtab.size() * 4,
                                  cudaMemcpyHostToDevice, net->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(net->vcol, vcol.data(), vcol.size() * 4, cudaMemcpyHostToDevice, net->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(net->colv, colv.data(), colv.size() * 4, cudaMemcpyHostToDevice, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->ctl, 0, sizeof(Ctl), net->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(net->cnt, 0, (size_t)net->nslot * 4, net->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(net->ccnt, 0, (size_t)net->nslot * net->ncol * 4, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->isum, 0, (size_t)net->ncol * 4, net->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(net->gsum, 0, (size_t)(net->ncol + 31) / 32 * 4, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->colcnt, 0, (size_t)net->ncol * 16, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->ext_part, 0, (size_t)net->update_grid * 8, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->spk_part, 0, (size_t)net->update_grid * 8, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->syn_part, 0, (size_t)net->update_grid * 8, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->rcnt, 0, (size_t)net->update_grid * 8, net->stream);
  if (e == cudaSuccess) {
    bp.wtab = wtab;
    bp.syn = net->syn;
    bp.bend = net->bend;
    bp.deg = net->deg;
    e = net->connectivity == SNN_CONN_PAPER ? launch_paper_fill(bp, precision, net->num_sms, net->stream)
                                            : launch_build(bp, precision, net->num_sms, net->stream);
  }
  fill_step_params(net);
  if (e == cudaSuccess) e = launch_init_state(net->sp, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  cudaFree(wtab);
  if (e != cudaSuccess) return cuda_fail(net, e, "network construction");
  if (net->sg.on) {
    // synapses kept by the shard: those into its own columns
    std::vector<uint32_t> deg((size_t)net->N);
    SNN_CUDA(net, cudaMemcpyAsync(deg.data(), net->deg, deg.size() * 4, cudaMemcpyDeviceToHost,
                                  net->stream));
    SNN_CUDA(net, cudaStreamSynchronize(net->stream));
    net->total_syn = 0;
    for (uint32_t d : deg) net->total_syn += d;
  }
  return SNN_OK;
}

int sync(snn_net* net) {
  SNN_CUDA(net, cudaStreamSynchronize(net->stream));
  return SNN_OK;
}

Ctl read_ctl(snn_net* net, cudaError_t* e) {
  Ctl c{};
  *e = cudaMemcpyAsync(&c, net->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, net->stream);
  if (*e == cudaSuccess) *e = cudaStreamSynchronize(net->stream);
  return c;
}

}  // namespace

namespace snn {

int net_view(snn_net* net, NetView* v) {
  if (!net) return SNN_EINVAL;
  if (net->sg.on) return SNN_ESTATE;
  v->syn = net->syn;
  v->bend = net->bend;
  v->N = net->N;
  v->npc = net->npc;
  v->nexc = net->nexc;
  v->dmin = net->dmin;
  v->ndel = net->ndel;
  v->rowcap = net->rowcap;
  v->precision = net->precision;
  v->num_sms = net->num_sms;
  v->seed = net->seed;
  v->neuron = net->neuron;
  v->stream = net->stream;
  return SNN_OK;
}

}  // namespace snn

extern "C" {

}  // extern "C"

namespace {

int build_net(int grid_w, int grid_h, const snn_neuron_params* neuron,
              const snn_synapse_params* synapse, uint64_t seed, int precision,
              void* cuda_stream, size_t window_budget, unsigned min_items, int part_cols,
              snn_net** out, const ShardGeo* shard = nullptr) {
  if (!out) return fail(nullptr, SNN_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  const int vrc = validate(grid_w, grid_h, neuron, synapse, precision, &why);
  if (vrc != SNN_OK) return fail(nullptr, vrc, why);
  snn_net* net = new (std::nothrow) snn_net();
  if (!net) return fail(nullptr, SNN_ENOMEM, "host allocation failed");
  net->window_budget = window_budget;
  net->min_items = min_items;
  net->part_cols = part_cols;
  if (shard) net->sg = *shard;
  if (cuda_stream) {
    net->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete net;
      return fail(nullptr, SNN_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    net->own_stream = true;
  }
  int rc = build_impl(net, grid_w, grid_h, neuron, synapse, seed, precision);
  if (rc != SNN_OK) {
    g_err = net->err;
    release(net);
    delete net;
    return rc;
  }
  *out = net;
  return SNN_OK;
}

}  // namespace

extern "C" {

int snn_build(int grid_w, int grid_h, const snn_neuron_params* neuron,
              const snn_synapse_params* synapse, uint64_t seed, int precision,
              void* cuda_stream, snn_net** out) {
  return build_net(grid_w, grid_h, neuron, synapse, seed, precision, cuda_stream, kWindowBudget,
                   kMinItems, kPartCols, out);
}

}  // extern "C"

namespace {

// Local grid of the shard of tile (x0, y0, w, h): the tile and a halo of R
// columns on each side, or the whole grid side where the two would meet.
// *ew, *eh receive the local grid's size.
int shard_geometry(int grid_w, int grid_h, int x0, int y0, int w, int h, int R, ShardGeo* g, int* ew,
                   int* eh) {
  if (grid_w < 1 || grid_h < 1 || grid_w > kMaxGridSide || grid_h > kMaxGridSide)
    return fail(nullptr, SNN_EINVAL, "grid_w and grid_h must be in 1..16383");
  if (x0 < 0 || y0 < 0 || w < 1 || h < 1 || x0 > grid_w - w || y0 > grid_h - h)
    return fail(nullptr, SNN_EINVAL, "the shard's tile must lie inside the grid");
  if (R < 1 || R > 3) return fail(nullptr, SNN_EINVAL, "stencil_radius must be 1..3");
  *g = ShardGeo{};
  g->on = 1;
  g->GW = grid_w;
  g->GH = grid_h;
  g->tw = w;
  g->th = h;
  *ew = grid_w;
  *eh = grid_h;
  if (w + 2 * R < grid_w) {
    *ew = w + 2 * R;
    g->ex0 = (x0 - R + grid_w) % grid_w;
    g->tx0 = R;
  } else {
    g->ex0 = 0;
    g->tx0 = x0;
  }
  if (h + 2 * R < grid_h) {
    *eh = h + 2 * R;
    g->ey0 = (y0 - R + grid_h) % grid_h;
    g->ty0 = R;
  } else {
    g->ey0 = 0;
    g->ty0 = y0;
  }
  return SNN_OK;
}

void geometry_words(const ShardGeo& g, int ew, int eh, int32_t* geo, int n) {
  const int32_t v[10] = {g.GW, g.GH, ew, eh, g.ex0, g.ey0, g.tx0, g.ty0, g.tw, g.th};
  for (int i = 0; i < n && i < 10; ++i) geo[i] = v[i];
}

}  // namespace

extern "C" {

int snn_shard_geometry(int grid_w, int grid_h, int x0, int y0, int w, int h, int stencil_radius,
                       int32_t* geo, int n) {
  if (!geo) return fail(nullptr, SNN_EINVAL, "geo is NULL");
  ShardGeo g{};
  int ew = 0, eh = 0;
  const int rc = shard_geometry(grid_w, grid_h, x0, y0, w, h, stencil_radius, &g, &ew, &eh);
  if (rc != SNN_OK) return rc;
  geometry_words(g, ew, eh, geo, n);
  return SNN_OK;
}

int snn_build_shard(int grid_w, int grid_h, int x0, int y0, int w, int h,
                    const snn_neuron_params* neuron, const snn_synapse_params* synapse,
                    uint64_t seed, int precision, void* cuda_stream, snn_net** out) {
  if (!out) return fail(nullptr, SNN_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  const int vrc = validate(grid_w, grid_h, neuron, synapse, precision, &why);
  if (vrc != SNN_OK) return fail(nullptr, vrc, why);
  if (synapse->connectivity != SNN_CONN_FIXED)
    return fail(nullptr, SNN_EINVAL, "shards support SNN_CONN_FIXED only");
  if (neuron->n_per_col % 4 != 0)
    return fail(nullptr, SNN_EINVAL, "shards need n_per_col to be a multiple of 4");
  ShardGeo g{};
  int ew = 0, eh = 0;
  const int grc = shard_geometry(grid_w, grid_h, x0, y0, w, h, synapse->stencil_radius, &g, &ew, &eh);
  if (grc != SNN_OK) return grc;
  return build_net(ew, eh, neuron, synapse, seed, precision, cuda_stream, kWindowBudget, kMinItems,
                   kPartCols, out, &g);
}

int snn_shard_update(snn_net* net) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  if (!net->sg.on) return fail(net, SNN_ESTATE, "not a shard: use snn_step");
  if (net->shard_phase != 0) return fail(net, SNN_ESTATE, "snn_shard_deliver is due first");
  int rc = check_status(net);
  if (rc) return rc;
  SNN_CUDA(net, launch_update(net->sp, net->update_grid, net->stream));
  net->shard_phase = 1;
  return SNN_OK;
}

int snn_shard_deliver(snn_net* net, const int32_t* ids, int64_t n, int32_t ids_on_device) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  if (!net->sg.on) return fail(net, SNN_ESTATE, "not a shard: use snn_step");
  if (n < 0 || (n > 0 && !ids)) return fail(net, SNN_EINVAL, "bad spike index array");
  if (net->shard_phase != 1) return fail(net, SNN_ESTATE, "snn_shard_update is due first");
  const uint32_t* src = reinterpret_cast<const uint32_t*>(ids);
  const bool staged = n > 0 && !ids_on_device;
  if (staged) {
    // the previous staged indices must have been read before the stage is reused
    if (net->ingest_ev) SNN_CUDA(net, cudaEventSynchronize(net->ingest_ev));
    else SNN_CUDA(net, cudaEventCreateWithFlags(&net->ingest_ev, cudaEventDisableTiming));
    if (n > net->ingest_cap) {
      const long long want = std::max<long long>(n, 1 << 16);
      if (net->ingest) cudaFree(net->ingest);
      if (net->hingest) cudaFreeHost(net->hingest);
      net->device_bytes -= (size_t)net->ingest_cap * 4;
      net->ingest = nullptr;
      net->hingest = nullptr;
      net->ingest_cap = 0;
      if (int rc = dalloc(net, &net->ingest, (size_t)want * 4)) return rc;
      SNN_CUDA(net, cudaMallocHost(&net->hingest, (size_t)want * 4));
      net->ingest_cap = want;
    }
    std::memcpy(net->hingest, ids, (size_t)n * 4);
    SNN_CUDA(net, cudaMemcpyAsync(net->ingest, net->hingest, (size_t)n * 4, cudaMemcpyHostToDevice,
                                  net->stream));
    src = net->ingest;
  }
  SNN_CUDA(net, launch_ingest(net->sp, src, n, net->stream));
  if (staged) SNN_CUDA(net, cudaEventRecord(net->ingest_ev, net->stream));
  SNN_CUDA(net, launch_deliver(net->sp, net->precision, net->deliver_grid, net->stream));
  net->shard_phase = 0;
  return SNN_OK;
}

int snn_shard_info(snn_net* net, int32_t* geo, int n) {
  if (!net || !geo) return fail(net, SNN_EINVAL, "null argument");
  if (!net->sg.on) return fail(net, SNN_ESTATE, "not a shard");
  geometry_words(net->sg, net->W, net->H, geo, n);
  return SNN_OK;
}

int snn_step(snn_net* net, int64_t n_steps) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  if (net->in_batch) return fail(net, SNN_ESTATE, "net belongs to a batch: use snn_batch_step");
  if (net->sg.on)
    return fail(net, SNN_ESTATE, "a shard steps by snn_shard_update and snn_shard_deliver");
  if (n_steps < 0) return fail(net, SNN_EINVAL, "n_steps must be >= 0");
  int rc = check_status(net);
  if (rc) return rc;
  if (n_steps == 0) return SNN_OK;
  if (n_steps >= net->graph_many_steps && !net->graph_many)
    if ((rc = capture(net, net->graph_many_steps, &net->graph_many))) return rc;
  if (!net->graph_one)
    if ((rc = capture(net, 1, &net->graph_one))) return rc;
  int64_t left = n_steps;
  while (left >= net->graph_many_steps) {
    SNN_CUDA(net, cudaGraphLaunch(net->graph_many, net->stream));
    left -= net->graph_many_steps;
  }
  while (left-- > 0) SNN_CUDA(net, cudaGraphLaunch(net->graph_one, net->stream));
  return SNN_OK;
}

int snn_step_profiled(snn_net* net, int64_t n_steps, double* ms, double* bytes) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  if (net->in_batch) return fail(net, SNN_ESTATE, "net belongs to a batch: use snn_batch_step");
  if (net->sg.on)
    return fail(net, SNN_ESTATE, "a shard steps by snn_shard_update and snn_shard_deliver");
  if (n_steps < 0) return fail(net, SNN_EINVAL, "n_steps must be >= 0");
  std::vector<cudaEvent_t> ev((size_t)n_steps * 3 + 1);
  unsigned long long* dspk = nullptr;  // spikes so far, after each step
  int rc = dalloc(net, &dspk, ((size_t)n_steps + 1) * 8);
  if (rc) return rc;
  net->device_bytes -= ((size_t)n_steps + 1) * 8;
  std::vector<unsigned long long> hspk((size_t)n_steps + 1, 0ull);
  size_t made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < ev.size() && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) --made;
  if (e == cudaSuccess) e = launch_sum_parts(net->spk_part, net->update_grid, dspk, net->stream);
  for (int64_t s = 0; s < n_steps && e == cudaSuccess; ++s) {
    e = cudaEventRecord(ev[3 * s], net->stream);
    if (e == cudaSuccess) e = launch_update(net->sp, net->update_grid, net->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + 1], net->stream);
    if (e == cudaSuccess)
      e = launch_deliver(net->sp, net->precision, net->deliver_grid, net->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ev[3 * s + 2], net->stream);
    if (e == cudaSuccess)
      e = launch_sum_parts(net->spk_part, net->update_grid, dspk + s + 1, net->stream);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(hspk.data(), dspk, hspk.size() * 8, cudaMemcpyDeviceToHost, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  double t_up = 0.0, t_dl = 0.0, b_up = 0.0, b_dl = 0.0;
  const double neuron_bytes = 26.0 * (double)net->N;
  for (int64_t s = 0; s < n_steps && e == cudaSuccess; ++s) {
    float a = 0.f, b = 0.f;
    e = cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[3 * s + 1], ev[3 * s + 2]);
    t_up += a;
    t_dl += b;
    const double S = (double)(hspk[s + 1] - hspk[s]);
    b_up += neuron_bytes + 12.0 * S;
    b_dl += S * ((double)net->total_syn / (double)net->N * net->rec_size + 6.0 * net->ndel);
  }
  if (e != cudaSuccess) rc = cuda_fail(net, e, "profiled step");
  for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  cudaFree(dspk);
  if (rc == SNN_OK) {
    if (ms) {
      ms[0] = t_up;
      ms[1] = t_dl;
    }
    if (bytes) {
      bytes[0] = b_up;
      bytes[1] = b_dl;
    }
  }
  return rc;
}

namespace {

// Records per region since the last drain, and the number kept.
int record_counts(snn_net* net, std::vector<unsigned long long>* cnt, long long* kept,
                  bool* lost) {
  cnt->assign((size_t)net->update_grid, 0ull);
  Ctl c{};
  SNN_CUDA(net, cudaMemcpyAsync(cnt->data(), net->rcnt, cnt->size() * 8, cudaMemcpyDeviceToHost,
                                net->stream));
  SNN_CUDA(net, cudaMemcpyAsync(&c, net->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, net->stream));
  SNN_CUDA(net, cudaStreamSynchronize(net->stream));
  *kept = 0;
  *lost = c.rec_overflow != 0u;
  for (unsigned long long v : *cnt) {
    const long long k = (long long)v < net->rec_region ? (long long)v : net->rec_region;
    *kept += k;
    if ((long long)v > net->rec_region) *lost = true;
  }
  return SNN_OK;
}

int reset_records(snn_net* net) {
  const unsigned zero32 = 0u;
  SNN_CUDA(net, cudaMemsetAsync(net->rcnt, 0, (size_t)net->update_grid * 8, net->stream));
  SNN_CUDA(net, cudaMemcpyAsync((char*)net->ctl + offsetof(Ctl, rec_overflow), &zero32, 4,
                                cudaMemcpyHostToDevice, net->stream));
  SNN_CUDA(net, cudaStreamSynchronize(net->stream));
  return SNN_OK;
}

}  // namespace

int snn_pending_spikes(snn_net* net, int64_t* n_out) {
  if (!net || !n_out) return fail(net, SNN_EINVAL, "null argument");
  std::vector<unsigned long long> cnt;
  long long kept = 0;
  bool lost = false;
  int rc = record_counts(net, &cnt, &kept, &lost);
  if (rc) return rc;
  *n_out = kept;
  return SNN_OK;
}

int snn_read_spikes(snn_net* net, int32_t* steps, int32_t* ids, int64_t cap, int64_t* n_out) {
  if (!net || !n_out || cap < 0 || (cap > 0 && (!steps || !ids)))
    return fail(net, SNN_EINVAL, "bad argument");
  *n_out = 0;
  // compact the regions on the device into id and step arrays and reset
  // them; a drain of at most hmap_cap records lands in mapped host memory
  // directly, a larger one is copied from the device stage afterwards
  const long long stage_cap = net->rec_region * net->update_grid;
  uint32_t* stage_ids = reinterpret_cast<uint32_t*>(net->stage);
  SNN_CUDA(net, launch_drain_records(net->sp, net->update_grid, stage_ids, stage_ids + stage_cap,
                                     net->dhdr, net->hhdr_dev, net->hmap_dev,
                                     net->hmap_dev + net->hmap_cap, net->hmap_cap, net->stream));
  SNN_CUDA(net, cudaStreamSynchronize(net->stream));
  if (int src = check_status(net)) return src;
  const long long kept = (long long)net->hhdr[0];
  bool lost = net->hhdr[1] != 0ull || kept > cap;
  const uint32_t tmin = (uint32_t)net->hhdr[2], tmax = (uint32_t)net->hhdr[3];
  const long long n = kept < cap ? kept : cap;
  const uint32_t* hid = net->hmap;
  const uint32_t* hst = net->hmap + net->hmap_cap;
  if (n > 0 && kept > net->hmap_cap) {
    if (n > net->hstage_cap) {
      if (net->hstage) cudaFreeHost(net->hstage);
      net->hstage = nullptr;
      net->hstage_cap = 0;
      const long long want = std::max<long long>(n, 1 << 16);
      SNN_CUDA(net, cudaMallocHost(&net->hstage, (size_t)want * 8));
      net->hstage_cap = want;
    }
    SNN_CUDA(net, cudaMemcpyAsync(net->hstage, stage_ids, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                  net->stream));
    SNN_CUDA(net, cudaMemcpyAsync(net->hstage + net->hstage_cap, stage_ids + stage_cap,
                                  (size_t)n * 4, cudaMemcpyDeviceToHost, net->stream));
    SNN_CUDA(net, cudaStreamSynchronize(net->stream));
    hid = net->hstage;
    hst = net->hstage + net->hstage_cap;
  }
  if (n > 0) {
    if (tmin == tmax) {
      // one step (the usual read after every step): the ids as they are
      std::memcpy(ids, hid, (size_t)n * 4);
      std::fill(steps, steps + n, (int32_t)tmin);
    } else {
      // each region is in step order: a counting sort by step puts the
      // window in step order (within a step the order stays unspecified)
      std::vector<long long> pos((size_t)(tmax - tmin) + 2, 0);
      for (long long k = 0; k < n; ++k) ++pos[(size_t)(hst[k] - tmin) + 1];
      for (size_t i = 1; i < pos.size(); ++i) pos[i] += pos[i - 1];
      for (long long k = 0; k < n; ++k) {
        const long long o = pos[hst[k] - tmin]++;
        steps[o] = (int32_t)hst[k];
        ids[o] = (int32_t)hid[k];
      }
    }
    *n_out = n;
  }
  if (lost) return fail(net, SNN_EOVERFLOW, "spike records dropped (buffer or cap too small)");
  return SNN_OK;
}

int snn_set_record_capacity(snn_net* net, int64_t capacity) {
  if (!net || capacity < 1) return fail(net, SNN_EINVAL, "bad argument");
  int rc = sync(net);
  if (rc) return rc;
  const long long region = (capacity + net->update_grid - 1) / net->update_grid;
  unsigned long long* nr = nullptr;
  cudaError_t e = cudaMalloc(&nr, (size_t)region * net->update_grid * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(net, e, "cudaMalloc record buffer");
  }
  unsigned long long* ns = nullptr;
  e = cudaMalloc(&ns, (size_t)region * net->update_grid * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(nr);
    return cuda_fail(net, e, "cudaMalloc record staging buffer");
  }
  cudaFree(net->rec);
  cudaFree(net->stage);
  net->device_bytes -= 2 * (size_t)net->rec_region * net->update_grid * 8;
  net->device_bytes += 2 * (size_t)region * net->update_grid * 8;
  net->rec = nr;
  net->stage = ns;
  net->rec_cap = capacity;
  net->rec_region = region;
  fill_step_params(net);
  free_graphs(net);
  return reset_records(net);
}

int snn_read_rates(snn_net* net, float* hz, int64_t n, float* pop_hz) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  if (hz && n < 2 * net->ncol) return fail(net, SNN_EINVAL, "hz array too small");
  cudaError_t e;
  Ctl c = read_ctl(net, &e);
  if (e != cudaSuccess) return cuda_fail(net, e, "read control block");
  if (int src = check_status(net)) return src;
  std::vector<unsigned long long> cnt((size_t)net->ncol * 2);
  SNN_CUDA(net, cudaMemcpyAsync(cnt.data(), net->colcnt, cnt.size() * 8, cudaMemcpyDeviceToHost,
                                net->stream));
  SNN_CUDA(net, cudaMemsetAsync(net->colcnt, 0, cnt.size() * 8, net->stream));
  SNN_CUDA(net, cudaStreamSynchronize(net->stream));
  const long long window = c.t - net->rate_window_start;
  net->rate_window_start = c.t;
  const double secs = (double)window * 1e-3;
  const double nE = (double)net->nexc, nI = (double)(net->npc - net->nexc);
  // a shard's own columns (the halo's spikes are counted by their owners)
  const double own_cols = net->sg.on ? (double)net->sg.tw * net->sg.th : (double)net->ncol;
  double totE = 0.0, totI = 0.0;
  for (long long k = 0; k < net->ncol; ++k) {
    totE += (double)cnt[2 * k];
    totI += (double)cnt[2 * k + 1];
    if (hz) {
      hz[2 * k] = (secs > 0 && nE > 0) ? (float)((double)cnt[2 * k] / (nE * secs)) : 0.f;
      hz[2 * k + 1] = (secs > 0 && nI > 0) ? (float)((double)cnt[2 * k + 1] / (nI * secs)) : 0.f;
    }
  }
  if (pop_hz) {
    pop_hz[0] = (secs > 0 && nE > 0) ? (float)(totE / (nE * own_cols * secs)) : 0.f;
    pop_hz[1] = (secs > 0 && nI > 0) ? (float)(totI / (nI * own_cols * secs)) : 0.f;
  }
  return SNN_OK;
}

int snn_stats(snn_net* net, double* recurrent_events, double* external_events, int64_t* steps) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  cudaError_t e;
  Ctl c = read_ctl(net, &e);
  if (e != cudaSuccess) return cuda_fail(net, e, "read control block");
  std::vector<unsigned long long> ext((size_t)net->update_grid), syn((size_t)net->update_grid);
  SNN_CUDA(net, cudaMemcpyAsync(ext.data(), net->ext_part, ext.size() * 8, cudaMemcpyDeviceToHost,
                                net->stream));
  SNN_CUDA(net, cudaMemcpyAsync(syn.data(), net->syn_part, syn.size() * 8, cudaMemcpyDeviceToHost,
                                net->stream));
  SNN_CUDA(net, cudaStreamSynchronize(net->stream));
  if (int src = check_status(net)) return src;
  unsigned long long se = 0ull, sy = 0ull;
  for (size_t b = 0; b < ext.size(); ++b) {
    se += ext[b];
    sy += syn[b];
  }
  // every spike counts its neuron's out-degree (k_out under the fixed law)
  if (recurrent_events) *recurrent_events = (double)sy;
  if (external_events) *external_events = (double)se;
  if (steps) *steps = (int64_t)c.t;
  return SNN_OK;
}

int snn_get_state(snn_net* net, float* v, float* c, uint8_t* refractory) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  const size_t N = (size_t)net->N;
  if (v) SNN_CUDA(net, cudaMemcpyAsync(v, net->V, N * 4, cudaMemcpyDeviceToHost, net->stream));
  if (c) SNN_CUDA(net, cudaMemcpyAsync(c, net->C, N * 4, cudaMemcpyDeviceToHost, net->stream));
  if (refractory)
    SNN_CUDA(net, cudaMemcpyAsync(refractory, net->R, N, cudaMemcpyDeviceToHost, net->stream));
  return sync(net);
}

int snn_read_synapses(snn_net* net, int64_t j0, int64_t n, int64_t* target, int32_t* delay,
                      int32_t* wfx) {
  if (!net || j0 < 0 || n < 0 || j0 + n > net->N || (n > 0 && (!target || !delay || !wfx)))
    return fail(net, SNN_EINVAL, "bad argument");
  if (n == 0) return SNN_OK;
  const size_t row_bytes = (size_t)net->rowcap * net->rec_size;
  std::vector<uint8_t> rows((size_t)n * row_bytes);
  std::vector<uint8_t> ends((size_t)n * kBendStride);
  SNN_CUDA(net, cudaMemcpyAsync(rows.data(), (const char*)net->syn + (size_t)j0 * row_bytes,
                                rows.size(), cudaMemcpyDeviceToHost, net->stream));
  SNN_CUDA(net, cudaMemcpyAsync(ends.data(), net->bend + (size_t)j0 * kBendStride, ends.size(),
                                cudaMemcpyDeviceToHost, net->stream));
  int rc = sync(net);
  if (rc) return rc;
  std::vector<int32_t> len((size_t)n);
  rc = snn_row_lengths(net, j0, n, len.data());
  if (rc) return rc;
  long long total = 0;
  for (int32_t v : len) total += v;
  long long o = 0;
  for (int64_t r = 0; r < n; ++r) {
    const long long j = j0 + r;
    const long long col = j / net->npc;
    const int cy = (int)(col / net->W), cx = (int)(col % net->W);
    const bool exc = (int)(j % net->npc) < net->nexc;
    int beg = 0;
    for (int b = 0; b < net->ndel; ++b) {
      const int end = ends[(size_t)r * kBendStride + b] * kSlotUnit;
      for (int s = beg; s < end; ++s) {
        uint32_t code, wbits;
        const uint8_t* rp = rows.data() + (size_t)r * row_bytes + (size_t)s * net->rec_size;
        int32_t w;
        if (net->precision == SNN_EXACT_F16W) {
          uint32_t rec;
          std::memcpy(&rec, rp, 4);
          if (is_pad_f16(rec)) continue;
          code = rec & 0x1FFFFu;
          __half_raw hr;
          hr.x = (unsigned short)(rec >> 17);
          const float f = __half2float(__half(hr));
          w = (int32_t)std::rint((exc ? f : -f) * 65536.0f);
        } else {
          std::memcpy(&code, rp, 4);
          std::memcpy(&wbits, rp + 4, 4);
          if (code == kPad) continue;
          w = (int32_t)wbits;
        }
        if (o >= total) return fail(net, SNN_ESTATE, "row holds too many synapses");
        if (net->precision == SNN_EXACT_F16W) {
          const int dy = (int)((code >> 14) & 7u) - 3, dx = (int)((code >> 11) & 7u) - 3;
          const int ty = ((cy + dy) % net->H + net->H) % net->H;
          const int tx = ((cx + dx) % net->W + net->W) % net->W;
          target[o] = ((long long)ty * net->W + tx) * net->npc + (code & 0x7FFu);
        } else {
          target[o] = (long long)code;
        }
        delay[o] = net->dmin + b;
        wfx[o] = w;
        ++o;
      }
      beg = end;
    }
  }
  if (o != total) return fail(net, SNN_ESTATE, "row holds too few synapses");
  return SNN_OK;
}

int snn_row_lengths(snn_net* net, int64_t j0, int64_t n, int32_t* counts) {
  if (!net || j0 < 0 || n < 0 || j0 + n > net->N || (n > 0 && !counts))
    return fail(net, SNN_EINVAL, "bad argument");
  if (n == 0) return SNN_OK;
  if (!net->deg) {
    for (int64_t r = 0; r < n; ++r) counts[r] = net->K;
    return SNN_OK;
  }
  SNN_CUDA(net, cudaMemcpyAsync(counts, net->deg + j0, (size_t)n * 4, cudaMemcpyDeviceToHost,
                                net->stream));
  return sync(net);
}

int snn_info(snn_net* net, int64_t* info, int n) {
  if (!net || !info) return fail(net, SNN_EINVAL, "null argument");
  const int64_t v[9] = {net->N, (int64_t)net->total_syn, (int64_t)net->device_bytes,
                        net->N * (int64_t)net->rowcap * net->rec_size, net->rowcap,
                        net->precision, net->tile, net->deliver_grid, net->update_grid};
  for (int i = 0; i < n && i < 9; ++i) info[i] = v[i];
  return SNN_OK;
}

const char* snn_last_error(const snn_net* net) {
  return net ? net->err.c_str() : g_err.c_str();
}

int snn_debug_offset_count(snn_net* net, int64_t column, int32_t delta, int32_t group_only) {
  if (!net) return fail(nullptr, SNN_EINVAL, "net is NULL");
  if (column < 0 || column >= net->ncol) return fail(net, SNN_EINVAL, "column out of range");
  int rc = sync(net);
  if (rc) return rc;
  uint32_t v = 0u;
  SNN_CUDA(net, cudaMemcpy(&v, net->colv + column, 4, cudaMemcpyDeviceToHost));
  unsigned word = 0u;
  if (!group_only) {
    SNN_CUDA(net, cudaMemcpy(&word, net->isum + v, 4, cudaMemcpyDeviceToHost));
    word += (unsigned)delta;
    SNN_CUDA(net, cudaMemcpy(net->isum + v, &word, 4, cudaMemcpyHostToDevice));
  }
  SNN_CUDA(net, cudaMemcpy(&word, net->gsum + (v >> 5), 4, cudaMemcpyDeviceToHost));
  word += (unsigned)delta;
  SNN_CUDA(net, cudaMemcpy(net->gsum + (v >> 5), &word, 4, cudaMemcpyHostToDevice));
  return SNN_OK;
}

void snn_destroy(snn_net* net) {
  if (!net) return;
  if (net->stream) cudaStreamSynchronize(net->stream);
  release(net);
  delete net;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched form: independent nets advanced together by one persistent launch.
// ---------------------------------------------------------------------------
struct snn_batch {
  std::vector<snn_net*> nets;
  int precision = 0, num_sms = 0, max_npc = 0;
  int infl = 4;            // 16-byte chunks in flight in the delivery loop
  int agg = 1;             // block windows for the local half of the synapses
  int dens8 = 64;          // delivery virtual blocks per 8 member columns
  int choice = -1;         // autotuner's pick (-1: not tuned)
  std::vector<int> first;  // host copy of d_first
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  StepParams* d_nets = nullptr;
  int* d_first = nullptr;  // [2][n + 1]: update, delivery virtual blocks
  unsigned* d_bar = nullptr;
  long long t = 0;
  long long spin_limit = 1LL << 25;
  unsigned extra_arrivals = 0u;
  std::string err;
};

namespace {

int bfail(snn_batch* b, int code, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_err = msg;
  return code;
}

#define SNN_BCUDA(b, call)                                                            \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return bfail((b), SNN_ECUDA, std::string(#call ": ") +     \
                                                           cudaGetErrorString(e_));   \
  } while (0)

void batch_release(snn_batch* b) {
  for (snn_net* n : b->nets) snn_destroy(n);
  b->nets.clear();
  if (b->d_nets) cudaFree(b->d_nets);
  if (b->d_first) cudaFree(b->d_first);
  if (b->d_bar) cudaFree(b->d_bar);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

// Delivery virtual blocks of member k: dens8 per 8 columns (at least one, at
// most its standalone grid).  Any count gives the same sums (the items are
// split into that many equal ranges).
void batch_delivery_firsts(snn_batch* b) {
  const size_t n = b->nets.size();
  for (size_t k = 0; k < n; ++k) {
    const snn_net* net = b->nets[k];
    const long long dg =
        std::min<long long>(net->deliver_grid, std::max<long long>(1, (long long)b->dens8 * net->ncol / 8));
    b->first[(n + 1) + k + 1] = b->first[(n + 1) + k] + (int)dg;
  }
}

// Upload the virtual-block tables (host copy in b->first).
int batch_upload_firsts(snn_batch* b) {
  SNN_BCUDA(b, cudaMemcpyAsync(b->d_first, b->first.data(), b->first.size() * sizeof(int),
                               cudaMemcpyHostToDevice, b->stream));
  SNN_BCUDA(b, cudaStreamSynchronize(b->stream));
  return SNN_OK;
}

// Upload the members' step parameters with the batch's window setting.
int batch_upload(snn_batch* b) {
  std::vector<StepParams> ps(b->nets.size());
  for (size_t k = 0; k < b->nets.size(); ++k) {
    b->nets[k]->agg = b->agg != 0;
    fill_step_params(b->nets[k]);
    ps[k] = b->nets[k]->sp;
  }
  SNN_BCUDA(b, cudaMemcpyAsync(b->d_nets, ps.data(), ps.size() * sizeof(StepParams),
                               cudaMemcpyHostToDevice, b->stream));
  SNN_BCUDA(b, cudaStreamSynchronize(b->stream));
  return SNN_OK;
}

int batch_run(snn_batch* b, long long n_steps) {
  if (n_steps == 0) return SNN_OK;
  // members' buffers may have been reallocated (record capacity): refresh
  const int urc = batch_upload(b);
  if (urc != SNN_OK) return urc;
  const int n = (int)b->nets.size();
  BatchParams bp{};
  bp.nets = b->d_nets;
  bp.u_first = b->d_first;
  bp.d_first = b->d_first + (n + 1);
  bp.n_nets = n;
  bp.t0 = b->t;
  bp.n_steps = n_steps;
  bp.bar = b->d_bar;
  bp.spin_limit = b->spin_limit;
  bp.extra_arrivals = b->extra_arrivals;
  size_t dsm = 0;
  for (const snn_net* net : b->nets) dsm = std::max(dsm, deliver_smem(net->sp, b->precision));
  const size_t smem = batch_smem(dsm);
  const int grid = batch_grid(b->precision, b->infl, b->num_sms, smem);
  if (grid < 1) return bfail(b, SNN_ECUDA, "batch kernel does not fit on the device");
  SNN_BCUDA(b, cudaMemsetAsync(b->d_bar, 0, 3 * sizeof(unsigned), b->stream));
  SNN_BCUDA(b, launch_batch(bp, b->precision, b->infl, grid, smem, b->stream));
  unsigned flags[3] = {0u, 0u, 0u};
  SNN_BCUDA(b, cudaMemcpyAsync(flags, b->d_bar, sizeof(flags), cudaMemcpyDeviceToHost, b->stream));
  SNN_BCUDA(b, cudaStreamSynchronize(b->stream));
  if (flags[2]) return bfail(b, SNN_ETIMEOUT, "a grid barrier wait gave up");
  b->t += n_steps;
  return SNN_OK;
}

}  // namespace

extern "C" {

int snn_batch_build(int n_nets, const int32_t* grid_w, const int32_t* grid_h,
                    const snn_neuron_params* neuron, const snn_synapse_params* synapse,
                    const uint64_t* seeds, int precision, void* cuda_stream, snn_batch** out) {
  if (!out) return bfail(nullptr, SNN_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_nets < 1 || n_nets > kMaxBatch) return bfail(nullptr, SNN_EINVAL, "n_nets must be in 1..256");
  if (!grid_w || !grid_h || !neuron || !synapse || !seeds)
    return bfail(nullptr, SNN_EINVAL, "null argument");
  for (int k = 0; k < n_nets; ++k) {
    std::string why;
    const int rc = validate(grid_w[k], grid_h[k], neuron + k, synapse + k, precision, &why);
    if (rc != SNN_OK) return bfail(nullptr, rc, "net " + std::to_string(k) + ": " + why);
  }
  snn_batch* b = new (std::nothrow) snn_batch();
  if (!b) return bfail(nullptr, SNN_ENOMEM, "host allocation failed");
  b->precision = precision;
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete b;
      return bfail(nullptr, SNN_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  int rc = SNN_OK;
  b->first.assign(2 * (size_t)(n_nets + 1), 0);
  for (int k = 0; k < n_nets && rc == SNN_OK; ++k) {
    snn_net* net = nullptr;
    rc = build_net(grid_w[k], grid_h[k], neuron + k, synapse + k, seeds[k], precision, b->stream,
                   kBatchWindowBudget, kBatchMinItems, kBatchPartCols, &net);
    if (rc != SNN_OK) break;
    net->in_batch = true;
    b->nets.push_back(net);
    b->max_npc = std::max(b->max_npc, net->npc);
    b->num_sms = net->num_sms;
    // update: the net's own grid (its partial sums and record regions)
    b->first[k + 1] = b->first[k] + net->update_grid;
  }
  if (rc != SNN_OK) {
    const std::string why = g_err;
    batch_release(b);
    delete b;
    return bfail(nullptr, rc, why);
  }
  batch_delivery_firsts(b);
  cudaError_t e = cudaMalloc(&b->d_nets, sizeof(StepParams) * (size_t)n_nets);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_first, b->first.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, 4 * sizeof(unsigned));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_first, b->first.data(), b->first.size() * sizeof(int),
                        cudaMemcpyHostToDevice, b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    batch_release(b);
    delete b;
    return bfail(nullptr, e == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA,
                 std::string("batch buffers: ") + cudaGetErrorString(e));
  }
  rc = batch_upload(b);
  if (rc != SNN_OK) {
    const std::string why = b->err;
    batch_release(b);
    delete b;
    return bfail(nullptr, rc, why);
  }
  *out = b;
  return SNN_OK;
}

int snn_batch_step(snn_batch* b, int64_t n_steps) {
  if (!b) return bfail(nullptr, SNN_EINVAL, "batch is NULL");
  if (n_steps < 0) return bfail(b, SNN_EINVAL, "n_steps must be >= 0");
  return batch_run(b, n_steps);
}

snn_net* snn_batch_net(snn_batch* b, int k) {
  if (!b || k < 0 || k >= (int)b->nets.size()) return nullptr;
  return b->nets[k];
}

int snn_batch_tune(snn_batch* b, int64_t steps_per_trial, int32_t* choice) {
  if (!b || steps_per_trial < 1) return bfail(b, SNN_EINVAL, "bad argument");
  // every variant computes the same sums, so the trials simply advance the
  // simulation; two interleaved rounds even out changes in activity.  Stage
  // 0 times the four delivery schedules, stage 1 the delivery densities with
  // the schedule that won.
  const int infl[4] = {4, 4, 2, 2}, agg[4] = {1, 0, 1, 0};
  const int dens8[4] = {64, 32, 16, 8};  // 8, 4, 2 and 1 blocks per column
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return bfail(b, SNN_ECUDA, std::string("tuner events: ") + cudaGetErrorString(ce));
  }
  int rc = SNN_OK;
  int pick[2] = {0, 0};
  for (int stage = 0; stage < 2 && rc == SNN_OK; ++stage) {
    double ms[4] = {0, 0, 0, 0};
    for (int round = 0; round < 2 && rc == SNN_OK; ++round) {
      for (int v = 0; v < 4 && rc == SNN_OK; ++v) {
        if (stage == 0) {
          b->infl = infl[v];
          b->agg = agg[v];
          rc = batch_upload(b);
        } else {
          b->dens8 = dens8[v];
          batch_delivery_firsts(b);
          rc = batch_upload_firsts(b);
        }
        if (rc) break;
        cudaError_t e = cudaEventRecord(e0, b->stream);
        if (e == cudaSuccess) {
          rc = batch_run(b, steps_per_trial);
          if (rc) break;
          e = cudaEventRecord(e1, b->stream);
        }
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float x = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&x, e0, e1);
        if (e != cudaSuccess) {
          rc = bfail(b, SNN_ECUDA, std::string("tuner timing: ") + cudaGetErrorString(e));
          break;
        }
        ms[v] += x;
      }
    }
    for (int v = 1; v < 4; ++v)
      if (ms[v] < ms[pick[stage]]) pick[stage] = v;
    if (rc == SNN_OK && stage == 0) {
      b->infl = infl[pick[0]];
      b->agg = agg[pick[0]];
      rc = batch_upload(b);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SNN_OK) return rc;
  b->dens8 = dens8[pick[1]];
  batch_delivery_firsts(b);
  rc = batch_upload_firsts(b);
  if (rc) return rc;
  b->choice = pick[0] + 4 * pick[1];
  if (choice) *choice = b->choice;
  return SNN_OK;
}

int snn_batch_set_wait(snn_batch* b, int64_t spin_limit, int32_t extra_arrivals) {
  if (!b || spin_limit < 1 || extra_arrivals < 0) return bfail(b, SNN_EINVAL, "bad argument");
  b->spin_limit = spin_limit;
  b->extra_arrivals = (unsigned)extra_arrivals;
  return SNN_OK;
}

const char* snn_batch_last_error(const snn_batch* b) { return b ? b->err.c_str() : g_err.c_str(); }

void snn_batch_destroy(snn_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  batch_release(b);
  delete b;
}


}  // extern "C"
