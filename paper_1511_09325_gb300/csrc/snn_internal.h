// snn_internal.h -- types shared by the translation units of the library.
//
// Device data layout of one net (all arrays are library-owned, 256 B aligned):
//   syn    outgoing-synapse table, row j at j * rowcap slots.  A row holds the
//          neuron's k_out synapses grouped by delay bucket b = d - d_min; every
//          bucket starts on a multiple of 8 slots and is padded with PAD
//          records up to the next multiple of 8 (so a bucket is a whole number
//          of 32 B sectors in the F16W layout).
//            F16W: u32 record  = half_magnitude(15) << 17 | code(17)
//            F32W: u32x2 record = { target neuron index, int32 round(w * 2^16) }
//          padding records have weight 0 (kPadF16 / {kPad, 0}).
//          (w the FP32 weight in mV, so the record holds exactly what is added)
//          code = ((dy + 3) << 3 | (dx + 3)) << 11 | l  (stencil offset of the
//          target column and index l inside it; local synapses use dx=dy=0).
//          The weight's sign is the source population's (Dale's principle),
//          so the F16W record drops the half's sign bit without loss.
//   bend   u8[N][32]: bend[j][b] = end of bucket b of row j in units of 8 slots.
//   V, C   float[Npad] membrane potential (mV) and calcium.
//   R      u8[Npad] remaining refractory steps.
//   acc    int32[Npad] recurrent input of the next step, 2^-16 mV units.
//   desc   spike descriptors of the last d_max + 1 steps (slot t % (d_max +
//          1)), desc_words u32 each: the spiker's id, then its bucket ends
//          (bend[j][0 .. ndel - 1], one byte each).  The spikes of column c
//          at step t are entries [slot][c * n_per_col + r], r < ccnt[slot][c],
//          in no fixed order.
//   ccnt   u32[d_max + 1][ncol] spikes of each slot's step per column.
//   vcol, colv  u32[ncol] delivery order of the columns: virtual column v is
//          real column vcol[v]; colv is the inverse.  Columns are numbered
//          tile by tile (tiles of `tile` x `tile` columns in row-major order,
//          row-major inside a tile), so a run of virtual columns is a compact
//          patch of the grid.
//   isum   u32[ncol] (bucket, spiker) items of each virtual column over the
//          steps that the next delivery reads (the sum of its d_max - d_min +
//          1 slots).
//   gsum   u32[ceil(ncol / 32)] isum summed over groups of 32 virtual columns.
//   cnt    u32[d_max + 1] spikes of each slot's step.
//   ctl    control block (step counter, completion counter, overflow flag,
//          status).
//   rec    u64 spike records (step << 32 | id), one region per update block,
//          rcnt[b] records in region b since the last drain.
//   colcnt u64[ncol][2] spike counts per column and population.
//   ext_part, spk_part  u64[update grid] external events and spikes counted
//          by each update block.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "snn.h"

namespace snn {

constexpr uint32_t kTagConn = 1u;  // Philox counter word 2 of each stream
constexpr uint32_t kTagExt = 2u;
constexpr uint32_t kTagInit = 3u;
constexpr uint32_t kTagSurr = 4u;  // normal draws of the differentiable form
constexpr uint32_t kTagPConn = 5u; // candidate draws of the paper connectivity law
constexpr int kMaxDelays = 32;   // d_max <= 32
constexpr int kBendStride = 32;  // bytes of bucket ends per neuron
constexpr int kSlotUnit = 8;     // buckets are padded to 8 synapse slots
constexpr int kMaxPoisThr = 127; // Poisson thresholds below 2^32
constexpr int kMaxOff = 48;      // remote stencil offsets (radius <= 3)
constexpr uint32_t kPad = 0xFFFFFFFFu;  // target of an F32W padding record (weight 0)
// F16W padding record: weight magnitude 0 and stencil field dx + 3 = 7, which
// no synapse uses (|dx| <= 3).
constexpr uint32_t kPadF16 = 7u << 11;
__host__ __device__ constexpr bool is_pad_f16(uint32_t rec) { return ((rec >> 11) & 7u) == 7u; }
constexpr int kCenterCode = (3 << 3) | 3;
constexpr int kMaxGridSide = 16383;     // columns per grid side (14-bit coordinates)
constexpr int kMaxTile = 8;             // delivery tile side, columns
constexpr int kMaxTileCols = kMaxTile * kMaxTile;
constexpr unsigned kWinMinItems = 512;  // default fewest items of a windowed tile part
// Fixed costs, in items, that the delivery's range split adds to a group of
// 32 columns with at least kWinMinItems items (window set-up and flush) and
// to one with fewer but some items (table set-up).
constexpr unsigned kCostWin = 1024;
constexpr unsigned kCostPart = 256;

// Tables computed on the host in FP64 and rounded once.
struct HostTables {
  int n_off = 0;
  int8_t off_dx[kMaxOff] = {}, off_dy[kMaxOff] = {};
  uint32_t stencil_thr[kMaxOff] = {};  // first n_off - 1 used; last is 2^32
  int n_pois_thr = 0;                  // thresholds below 2^32
  uint32_t pois_thr[kMaxPoisThr + 1] = {};
  uint8_t pois_guide[256] = {};        // #thresholds <= (b << 24)
  std::vector<uint32_t> wtab;          // [2][65536] stored weight bits
  float pvv = 0, pcc = 0, pvc[2] = {0, 0};
  int32_t jx = 0;
  int nref = 0;
  int k_local = 0;
  // paper connectivity law (SNN_CONN_PAPER)
  int n_poff = 0;
  int8_t poff_dx[kMaxOff] = {}, poff_dy[kMaxOff] = {};
  unsigned long long poff_thr[kMaxOff] = {};  // candidate kept iff word < thr
  unsigned long long plocal_thr = 0;
  long long n_cand = 0;                        // candidates per neuron
};

int make_host_tables(const snn_neuron_params& np, const snn_synapse_params& sp,
                     int precision, HostTables* out, std::string* err);
// The neuron-update part only: Poisson table, propagators, J_ext, refractory.
int make_neuron_tables(const snn_neuron_params& np, HostTables* out, std::string* err);
// Standard-normal quantiles at (m + 0.5) / 65536, m < 65536 (computed once).
const std::vector<double>& quantile_table();

// Device control block.
struct Ctl {
  long long t;                  // step index of the next update
  unsigned int drained;         // blocks done with the current record drain
  unsigned int done;            // delivery blocks finished this step
  unsigned int rec_overflow;    // set when a record did not fit its region
  unsigned int status;          // nonzero: a delivery found inconsistent counts
};

// Status codes a kernel leaves in Ctl::status (and the mapped host word).
constexpr unsigned kStatusCounts = 1u;  // item counts disagree with the spike lists
constexpr unsigned kStatusIngest = 2u;  // a shard received an index it cannot list

// A shard: a net over a local grid E of W x H columns (its own columns and a
// halo of stencil_radius columns around them, clipped to the global grid)
// whose local column (lx, ly) is global column ((ex0 + lx) mod GW,
// (ey0 + ly) mod GH).  Only the columns of T = [tx0, tx0 + tw) x [ty0, ty0 +
// th) (local coordinates) are its own: it updates their neurons and keeps the
// synapses that end in them; the halo's spikes arrive from other shards.
// Random draws and spike records use global neuron indices.  A whole network
// is the shard with on = 0 (E = T = the grid).
struct ShardGeo {
  int on;
  int GW, GH;
  int ex0, ey0;
  int tx0, ty0, tw, th;
};

// Global column of local column (lx, ly).
__host__ __device__ inline void shard_global_col(const ShardGeo& g, int lx, int ly, int* gx,
                                                 int* gy) {
  if (!g.on) {
    *gx = lx;
    *gy = ly;
    return;
  }
  *gx = (g.ex0 + lx) % g.GW;
  *gy = (g.ey0 + ly) % g.GH;
}

// Whether global column (gx, gy) is one of the shard's own columns.
__host__ __device__ inline bool shard_owns_global(const ShardGeo& g, int W, int H, int gx, int gy) {
  if (!g.on) return true;
  const int lx = ((gx - g.ex0) % g.GW + g.GW) % g.GW;
  const int ly = ((gy - g.ey0) % g.GH + g.GH) % g.GH;
  return lx < W && ly < H && lx >= g.tx0 && lx < g.tx0 + g.tw && ly >= g.ty0 && ly < g.ty0 + g.th;
}

// Everything a step kernel needs, passed by value (constant bank).
struct StepParams {
  long long N;
  int npc, nexc, W, H, K, dmin, ndel, nslot, rowcap;
  int ncol;
  int agg;  // shared-memory windows over each delivery tile and its ring
  int tile, ring;          // delivery tile side and window ring, in columns
  int part_cols;           // most columns of a delivery part without window (>= tile^2)
  int win_cap;             // ints of the window (largest tile window)
  int desc_words;          // u32 words per spike descriptor (8 or 16)
  unsigned min_items;      // fewest items a delivery block takes (fewer blocks run)
  unsigned win_items;      // fewest items of a tile part that uses the window
  unsigned cost_win, cost_part;  // fixed cost (in items) of a windowed / other group
  uint32_t npc_m, w_m;     // floor(2^32 / n_per_col), floor(2^32 / W) (capped)
  uint32_t seed_lo, seed_hi;
  float theta, vr, dc, pvv, pcc, pvc_e, pvc_i;
  int32_t jx;
  int nref;
  int n_pois_thr;
  uint32_t pois_thr[kMaxPoisThr + 1];
  uint8_t pois_guide[256];
  float* V;
  float* C;
  uint8_t* R;
  int32_t* acc;
  uint32_t* ids;   // compact spike-id list (no descriptors: noalloc form only)
  uint32_t* desc;  // spike descriptors (see above); null: write ids instead
  const uint32_t* vcol;
  const uint32_t* colv;
  unsigned* hstatus;  // mapped host copy of Ctl::status (may be null)
  unsigned* cnt;
  unsigned* ccnt;  // per-column counts (column-indexed lists); null: one compact list
  unsigned* isum;  // per-column items of the delivery window (with ccnt)
  unsigned* gsum;  // isum per group of 32 columns
  const uint8_t* bend;
  const void* syn;
  Ctl* ctl;
  unsigned long long* rec;
  long long rec_region;          // records per update block
  unsigned long long* rcnt;      // records written per region since the last drain
  unsigned long long* colcnt;
  unsigned long long* ext_part;  // external-event partial sums, one per update block
  unsigned long long* spk_part;  // spike partial sums, one per update block
  const uint32_t* deg;           // out-degree per neuron (paper law), else null
  unsigned long long* syn_part;  // synaptic events of the spikes, one per update block
  ShardGeo sg;                   // shard geometry (sg.on = 0: a whole network)
};

// A batch of nets advanced by one persistent launch (snn_batch_*).
constexpr int kMaxBatch = 256;
struct BatchParams {
  StepParams* nets;         // [n_nets], device
  const int* u_first;       // [n_nets + 1] first update virtual block of each net
  const int* d_first;       // [n_nets + 1] first delivery virtual block of each net
  int n_nets;
  long long t0, n_steps;
  unsigned* bar;            // grid barrier: arrivals, generation, error flag
  long long spin_limit;     // polls before a barrier wait gives up
  unsigned extra_arrivals;  // arrivals expected beyond the grid (0; tests only)
};

struct BuildParams {
  long long N;
  int npc, nexc, W, H, K, k_local, dmin, ndel, rowcap, n_off;
  uint32_t seed_lo, seed_hi;
  uint32_t stencil_thr[kMaxOff];
  int8_t off_dx[kMaxOff], off_dy[kMaxOff];
  const uint32_t* wtab;
  void* syn;
  uint8_t* bend;
  // paper connectivity law
  int n_poff;
  long long n_cand;
  unsigned long long poff_thr[kMaxOff];
  unsigned long long plocal_thr;
  int8_t poff_dx[kMaxOff], poff_dy[kMaxOff];
  uint32_t* deg;          // [N] out-degree of each neuron
  unsigned* max_units;    // largest row, in units of 8 slots
  ShardGeo sg;            // shard geometry (sg.on = 0: a whole network)
};

// What the differentiable form reads of a net (snn_api.cu fills it).
struct NetView {
  const void* syn;
  const uint8_t* bend;
  long long N;
  int npc, nexc, dmin, ndel, rowcap, precision, num_sms;
  uint64_t seed;
  snn_neuron_params neuron;
  cudaStream_t stream;
};
int net_view(snn_net* net, NetView* v);

// Shared host helpers (snn_api.cu).
int fail_global(int code, const std::string& msg);
int validate_neuron_params(const snn_neuron_params* n, std::string* why);

// Kernel launchers (snn_build.cu / snn_step.cu).
cudaError_t launch_build(const BuildParams& bp, int precision, int num_sms,
                         cudaStream_t st);
// Paper connectivity law: the count pass writes bend, deg and max_units; the
// fill pass (same draws) writes the rows.
cudaError_t launch_paper_count(const BuildParams& bp, int num_sms, cudaStream_t st);
cudaError_t launch_paper_fill(const BuildParams& bp, int precision, int num_sms,
                              cudaStream_t st);
cudaError_t launch_init_state(const StepParams& p, cudaStream_t st);
cudaError_t launch_update(const StepParams& p, int grid, cudaStream_t st);
int update_grid(long long N, int num_sms);
// Delivery: dynamic shared memory of one block (table, F16W neighbour table,
// window), its thread count, and the persistent grid (0 if it does not fit).
size_t deliver_smem(const StepParams& p, int precision);
int deliver_threads();
int deliver_grid(const StepParams& p, int precision, int num_sms);
cudaError_t launch_deliver(const StepParams& p, int precision, int grid, cudaStream_t st);
// Compact the per-block record regions into id and step arrays and reset
// them; header = {records kept, 1 if records were dropped, first step, last
// step}, written to header and to the mapped host header map_hdr.  The arrays
// go to the mapped host buffers when they hold at most map_cap records, else
// to the device stage.
constexpr long long kMappedRecords = 1LL << 18;  // mapped host records per net
cudaError_t launch_drain_records(const StepParams& p, int nreg, uint32_t* stage_ids,
                                 uint32_t* stage_steps, unsigned long long* header,
                                 unsigned long long* map_hdr, uint32_t* map_ids,
                                 uint32_t* map_steps, long long map_cap, cudaStream_t st);
// Batch kernel: dynamic shared memory for members whose largest delivery
// layout is max_deliver_smem, its grid (0 if it does not fit), its launch.
size_t batch_smem(size_t max_deliver_smem);
int batch_grid(int precision, int infl, int num_sms, size_t smem);
cudaError_t launch_batch(const BatchParams& b, int precision, int infl, int grid, size_t smem,
                         cudaStream_t st);
// Shard: list the received spikes (global indices ids[0 .. n)) of the halo
// columns in the step's lists, as the update kernel lists its own.
cudaError_t launch_ingest(const StepParams& p, const uint32_t* ids, long long n, cudaStream_t st);
cudaError_t launch_sum_parts(const unsigned long long* part, int n, unsigned long long* out,
                             cudaStream_t st);

}  // namespace snn
