// snn_step.cu -- the two kernels of one 1 ms step.
//
// update_kernel (neuron update, arxiv 1511.09325 Sec. 2 LIF + SFA):
//   grid-stride over tiles of 1024 neurons; one thread owns 4 consecutive
//   neurons and one Philox4x32-10 block (counter (i/4, t, EXT, 0)) whose 4
//   words give their external Poisson counts.  It reads and clears their
//   recurrent input, applies refractoriness, threshold, reset and the exact
//   propagator with explicitly rounded FP32 operations.  A tile's spikes are
//   counted per column in shared memory and written to their column's part of
//   the step's spike list (one atomic per column and tile) and to the block's
//   record region.  The per-column item counts of the next delivery (isum,
//   gsum) are kept up to date here; spike and external-event totals go to
//   per-block partial sums.
//
// deliver_kernel (event-driven delivery, Sec. 1), "pull by delay": the input
//   of step t+1 is the sum over delays d of bucket d of every neuron that
//   spiked at step t+1-d, so only one N-entry accumulator (resident in L2)
//   receives additions, not a d_max-slot ring.  The (delay bucket, spiker)
//   items of the last d_max steps, ordered by (column, bucket, spiker), form
//   one virtual list split evenly over a persistent grid.  A warp takes 32
//   consecutive items: lane e resolves item e, then the warp streams the
//   concatenated buckets in 16-byte chunks (4 synapses per lane, four chunks in
//   flight).  The item a chunk belongs to is found from a ballot over the
//   items' start offsets and the item's fields travel by shuffle, so the inner
//   loop reads no shared memory.  Each synapse's weight goes to L2 as a
//   fire-and-forget int32 reduction, except that synapses onto the first
//   columns of a block's range (where its spikers sit, so about half of their
//   synapses) are summed in shared-memory windows and flushed once per block.
//   Integer addition makes the result independent of the order.  The last
//   block to finish advances the step counter.
#include "snn_device.cuh"
#include "snn_internal.h"

namespace snn {
namespace {

constexpr int kUpdateThreads = 256;
constexpr int kDeliverThreads = 256;
constexpr int kBatchThreads = kUpdateThreads;  // the batch kernel runs both bodies
constexpr int kInflight = 4;     // 16-byte synapse chunks in flight per lane (F32W: 2 loads each)
constexpr int kInflightF16 = 4;  // the same for F16W (one load each)
constexpr int kTile = kUpdateThreads * 4;    // neurons per update tile
constexpr int kTileCols = kTile / 2 + 2;     // columns a tile can touch (npc >= 2)

struct NeuronOut {
  float v, c;
  uint32_t r;
  bool spike;
};

// One neuron, one step; every float operation rounded as written.
__device__ __forceinline__ NeuronOut neuron_step(float v, float c, uint32_t r,
                                                 int32_t I, float pvc,
                                                 const StepParams& P) {
  NeuronOut o;
  o.spike = false;
  if (r > 0u) {
    r -= 1u;
    v = P.vr;
  } else {
    v = __fadd_rn(v, __fmul_rn(__int2float_rn(I), 1.52587890625e-05f));
    if (v >= P.theta) {
      o.spike = true;
      v = P.vr;
      r = (uint32_t)P.nref;
      c = __fadd_rn(c, P.dc);
    }
  }
  o.v = __fmaf_rn(c, pvc, __fmul_rn(v, P.pvv));
  o.c = __fmul_rn(c, P.pcc);
  o.r = r;
  return o;
}

// Poisson count by inversion: the guide table gives the number of
// thresholds below the top byte of x, a short scan finishes the count.
__device__ __forceinline__ int poisson_count(uint32_t x, const uint8_t* guide,
                                             const uint32_t* thr, int n) {
  int k = guide[x >> 24];
  while (k < n && x >= thr[k]) ++k;
  return k;
}

// L2 evict-last policy for the accumulator, which the next step's update
// re-reads.
__device__ __forceinline__ uint64_t evict_last_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// Fire-and-forget int32 reduction into the accumulator under policy `pol`.
__device__ __forceinline__ void red_add(int32_t* p, int32_t v, uint64_t pol) {
  asm volatile("red.global.add.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
               : "memory");
}

// The same, issued only where `on` is nonzero: a predicated instruction, so
// lanes that take different paths do not split the warp.
__device__ __forceinline__ void red_add_if(uint32_t on, int32_t* p, int32_t v, uint64_t pol) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
      "@q red.global.add.L2::cache_hint.s32 [%1], %2, %3;\n\t}" ::"r"(on),
      "l"(p), "r"(v), "l"(pol)
      : "memory");
}

// Predicated int32 reduction into shared memory (shared-window address `a`).
__device__ __forceinline__ void red_shared_if(uint32_t on, uint32_t a, int32_t v) {
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %0, 0;\n\t"
      "@q red.shared.add.s32 [%1], %2;\n\t}" ::"r"(on),
      "r"(a), "r"(v)
      : "memory");
}

// Shared memory of one update block.
struct UpdateSmem {
  uint32_t thr[kMaxPoisThr + 1];  // Poisson thresholds
  uint8_t guide[256];            // Poisson guide table
  unsigned tpop[kTileCols][2];   // E / I spikes per column of the tile
  unsigned tpos[kTileCols];      // first record of each column's spikes in the tile
  long long lbase[kTileCols];    // list position of each column's first spike
  long long cbase;               // compact list: position of the tile's first spike
  unsigned long long rbase;      // record position of the tile's first spike
  unsigned long long rc, spk;
  unsigned long long synw[kUpdateThreads / 32];  // synaptic events per warp
  unsigned ksum[kUpdateThreads / 32];
};

// Update block vb of vgrid for step t: tiles vb, vb + vgrid, ...  Block vb
// owns ext_part[vb], spk_part[vb] and record region vb of the net, so the
// grid size must be the same every step.  Each spike goes to the step's list
// (column c's part when P.ccnt is set, else one compact list) and to the
// block's record region as (step << 32 | id).
__device__ __forceinline__ void update_body(const StepParams& P, long long t, int vb, int vgrid,
                                            UpdateSmem& S) {
  __syncthreads();  // the shared memory may still be read by a previous body
  const int slot = (int)(t % P.nslot);
  for (int m = threadIdx.x; m < 256; m += blockDim.x) S.guide[m] = P.pois_guide[m];
  for (int m = threadIdx.x; m <= kMaxPoisThr; m += blockDim.x) S.thr[m] = P.pois_thr[m];
  if (threadIdx.x == 0) {
    S.rc = P.rcnt[vb];
    S.spk = 0ull;
  }
  unsigned ksum = 0u;
  unsigned long long syn = 0ull;  // out-degrees of this thread's spikes
  const long long quads = (P.N + 3) / 4;
  const long long tiles = (quads + kUpdateThreads - 1) / kUpdateThreads;
  uint32_t* list = P.ids + (long long)slot * P.N;
  unsigned long long* region = P.rec + (long long)vb * P.rec_region;

  // Each column's item count (isum, gsum) moves from the delivery window of
  // step t - 1, steps t - d_max .. t - d_min, to that of step t: step
  // t + 1 - d_min comes in (as its spikes are counted, when d_min = 1) and
  // step t - d_max, whose slot is (t + 1) mod (d_max + 1), goes out.  The tile
  // in which a column starts applies the change for that column.
  const long long s_in = t + 1 - P.dmin;
  const unsigned* cin_ = (P.ccnt != nullptr && P.dmin >= 2 && s_in >= 0)
                             ? P.ccnt + (s_in % P.nslot) * P.ncol : nullptr;
  const unsigned* cout_ = P.ccnt != nullptr ? P.ccnt + ((t + 1) % P.nslot) * P.ncol : nullptr;

  for (long long tile = vb; tile < tiles; tile += vgrid) {
    const long long first = tile * kTile;
    const long long last = (first + kTile < P.N ? first + kTile : P.N) - 1;
    // neuron indices are below 2^31: 32-bit divisions are exact (and cheap)
    const int col0 = (int)((uint32_t)first / (uint32_t)P.npc);
    const int ncols = (int)((uint32_t)last / (uint32_t)P.npc) - col0 + 1;
    for (int k = threadIdx.x; k < ncols; k += blockDim.x) {
      S.tpop[k][0] = 0u;
      S.tpop[k][1] = 0u;
    }
    __syncthreads();

    const long long q = tile * kUpdateThreads + threadIdx.x;
    const long long i0 = q * 4;
    unsigned rank[4] = {0u, 0u, 0u, 0u};
    int scol[4] = {-1, -1, -1, -1};
    if (i0 < P.N) {
      const uint4 x = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)t, kTagExt, 0u), P.seed_lo, P.seed_hi);
      const float4 v4 = reinterpret_cast<const float4*>(P.V)[q];
      const float4 c4 = reinterpret_cast<const float4*>(P.C)[q];
      const uchar4 r4 = reinterpret_cast<const uchar4*>(P.R)[q];
      const int4 a4 = reinterpret_cast<const int4*>(P.acc)[q];
      reinterpret_cast<int4*>(P.acc)[q] = make_int4(0, 0, 0, 0);
      const float vin[4] = {v4.x, v4.y, v4.z, v4.w};
      const float cin[4] = {c4.x, c4.y, c4.z, c4.w};
      const uint32_t rin[4] = {r4.x, r4.y, r4.z, r4.w};
      const int32_t ain[4] = {a4.x, a4.y, a4.z, a4.w};
      const uint32_t xin[4] = {x.x, x.y, x.z, x.w};
      float vout[4], cout[4];
      uint32_t rout[4];
      int col = (int)((uint32_t)i0 / (uint32_t)P.npc);
      int l = (int)((uint32_t)i0 - (uint32_t)col * (uint32_t)P.npc);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = poisson_count(xin[e], S.guide, S.thr, P.n_pois_thr);
        const int32_t I = ain[e] + k * P.jx;
        const bool exc = l < P.nexc;
        const NeuronOut o = neuron_step(vin[e], cin[e], rin[e], I, exc ? P.pvc_e : P.pvc_i, P);
        vout[e] = o.v;
        cout[e] = o.c;
        rout[e] = o.r;
        if (i0 + e < P.N) {
          ksum += (unsigned)k;
          if (o.spike) {
            scol[e] = col - col0;
            rank[e] = atomicAdd(&S.tpop[col - col0][exc ? 0 : 1], 1u);
            if (!exc) rank[e] |= 0x80000000u;  // ranked among the column's I spikes
          }
        }
        if (++l == P.npc) {
          l = 0;
          ++col;
        }
      }
      reinterpret_cast<float4*>(P.V)[q] = make_float4(vout[0], vout[1], vout[2], vout[3]);
      reinterpret_cast<float4*>(P.C)[q] = make_float4(cout[0], cout[1], cout[2], cout[3]);
      reinterpret_cast<uchar4*>(P.R)[q] = make_uchar4((unsigned char)rout[0], (unsigned char)rout[1],
                                                      (unsigned char)rout[2], (unsigned char)rout[3]);
    }
    __syncthreads();
    // places: records grouped by column (E then I) in the block's region; list
    // entries in each column's part of the step's list (or the compact list)
    if (P.ccnt != nullptr) {
      for (int k = threadIdx.x; k < ncols; k += blockDim.x) {
        const unsigned n = S.tpop[k][0] + S.tpop[k][1];
        const int c = col0 + k;
        S.lbase[k] = (long long)c * P.npc +
                     (n ? (long long)atomicAdd(P.ccnt + (long long)slot * P.ncol + c, n) : 0ll);
        unsigned d = P.dmin == 1 ? n : 0u;
        if ((long long)c * P.npc >= first) d += (cin_ ? cin_[c] : 0u) - cout_[c];
        if (d) {
          atomicAdd(P.isum + c, d);
          atomicAdd(P.gsum + (c >> 5), d);
        }
      }
    }
    if (threadIdx.x == 0) {
      unsigned pos = 0u;
      for (int k = 0; k < ncols; ++k) {
        S.tpos[k] = pos;
        pos += S.tpop[k][0] + S.tpop[k][1];
      }
      S.cbase = pos ? (long long)atomicAdd(P.cnt + slot, pos) : 0ll;
      S.rbase = S.rc;
      S.rc += pos;
      S.spk += pos;
    }
    __syncthreads();
    const unsigned long long rc = S.rbase;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (scol[e] >= 0) {
        const int k = scol[e];
        const unsigned r = rank[e] & 0x7FFFFFFFu;
        const unsigned off = (rank[e] & 0x80000000u) ? S.tpop[k][0] + r : r;
        const uint32_t id = (uint32_t)(i0 + e);
        list[P.ccnt != nullptr ? S.lbase[k] + off : S.cbase + S.tpos[k] + off] = id;
        syn += P.deg != nullptr ? P.deg[id] : (uint32_t)P.K;
        const unsigned long long ri = rc + S.tpos[k] + off;
        if ((long long)ri < P.rec_region) region[ri] = ((unsigned long long)(unsigned)t << 32) | id;
      }
    }
    for (int k = threadIdx.x; k < ncols; k += blockDim.x) {
      if (S.tpop[k][0]) atomicAdd(&P.colcnt[2 * (col0 + k)], (unsigned long long)S.tpop[k][0]);
      if (S.tpop[k][1]) atomicAdd(&P.colcnt[2 * (col0 + k) + 1], (unsigned long long)S.tpop[k][1]);
    }
    __syncthreads();
  }

  // external and synaptic events: per-block partial sums, no atomics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, o);
    syn += __shfl_xor_sync(0xFFFFFFFFu, syn, o);
  }
  if ((threadIdx.x & 31) == 0) {
    S.ksum[threadIdx.x >> 5] = ksum;
    S.synw[threadIdx.x >> 5] = syn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0ull, tsyn = 0ull;
    for (int w = 0; w < kUpdateThreads / 32; ++w) {
      tot += S.ksum[w];
      tsyn += S.synw[w];
    }
    P.ext_part[vb] += tot;
    P.spk_part[vb] += S.spk;
    if (P.syn_part != nullptr) P.syn_part[vb] += tsyn;
    if ((long long)S.rc > P.rec_region) P.ctl->rec_overflow = 1u;
    P.rcnt[vb] = S.rc;
  }
}

__global__ void __launch_bounds__(kUpdateThreads, 5) update_kernel(const StepParams P) {
  __shared__ UpdateSmem S;
  update_body(P, P.ctl->t, (int)blockIdx.x, (int)gridDim.x, S);
}

// Periodic coordinate v in [-3, n + 3); one conditional correction suffices
// when the period is at least 4.
__device__ __forceinline__ int wrap_near(int v, int n) {
  if (n >= 4) {
    v += (v < 0) ? n : 0;
    v -= (v >= n) ? n : 0;
    return v;
  }
  return wrap(v, n);
}

constexpr int kWindows = 4;        // shared-memory windows (columns) per delivery block
constexpr int kBatchItems = 16;    // items per warp batch (at most 32)
// (column, bucket) entries per table piece, at most: 4 per thread
constexpr int kTabEntries = 4 * (kDeliverThreads > kBatchThreads ? kDeliverThreads : kBatchThreads);
// A piece spans at most kPieceCols columns; for F16W each has 64 entries
// (one per stencil code) in the neighbour table.
constexpr int kPieceCols = 32;
constexpr int kNbEntries = 64 * kPieceCols;

// Per-item info travelling with a chunk: the spiker's column cx | cy << 14
// and whether it is inhibitory (bit 28).
__device__ __forceinline__ uint32_t pack_info(int cx, int cy, bool inh) {
  return (uint32_t)cx | ((uint32_t)cy << 14) | ((inh ? 1u : 0u) << 28);
}

// Deliver one synapse record of a spiker whose column info is `info`.
// Targets in neurons wbase .. wbase + wlen - 1 (the block's window columns)
// are summed in the shared windows at shared address win_s, the others
// reduced into L2.  Padding records deliver nothing.  Both reductions are
// predicated, so the warp never diverges here.
template <int PREC>
__device__ __forceinline__ void deliver_record(uint32_t code, uint32_t wbits, uint32_t info,
                                               uint32_t win_s, uint32_t wbase, uint32_t wlen,
                                               uint64_t pol, const uint32_t* nb,
                                               const StepParams& P) {
  const bool valid = code != kPad;
  uint32_t target;
  int32_t wfx;
  if (PREC == SNN_EXACT_F16W) {
    const float wscale = (info >> 28) & 1u ? -65536.0f : 65536.0f;
    wfx = __float2int_rn(__fmul_rn(__half2float(__ushort_as_half((unsigned short)wbits)), wscale));
    // first neuron of the target column, from the piece's neighbour table
    const uint32_t off = (code >> 11) & 63u;
    target = nb[(info & 0x3Fu) * 64u + (valid ? off : 0u)] + (code & 0x7FFu);
  } else {
    wfx = (int32_t)wbits;
    target = code;
  }
  const uint32_t rel = target - wbase;
  const bool inwin = rel < wlen;
  red_shared_if(valid && inwin, win_s + 4u * rel, wfx);
  red_add_if(valid && !inwin, P.acc + (valid ? target : 0u), wfx, pol);
}

struct DeliverSmem {
  unsigned tab[kTabEntries + 1];  // items before each (column, bucket) entry of the piece
  int slot[kMaxDelays];           // slot of each bucket's step, -1 before step 0
  unsigned long long wsum[32];    // per-warp sums of block_scan
  unsigned long long xgp[2];      // items before the group holding lo / hi - 1
  unsigned long long p0;          // items before column c0
  int xg[2];                      // group holding lo / hi - 1
  int c0, c1;                     // first and last column of the block's items
  unsigned next;                  // next batch of the current piece
};
constexpr size_t kDeliverSmemPad = (sizeof(DeliverSmem) + 255) / 256 * 256;

// Block-wide exclusive scan of one 64-bit value per thread; *total gets the
// sum.  Uses S.wsum; contains two barriers.
__device__ __forceinline__ unsigned long long block_scan(unsigned long long v, DeliverSmem& S,
                                                         unsigned long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  unsigned long long incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) S.wsum[warp] = incl;
  __syncthreads();
  unsigned long long before = 0ull, all = 0ull;
  for (int w = 0; w < nwarps; ++w) {
    const unsigned long long s = S.wsum[w];
    before += w < warp ? s : 0ull;
    all += s;
  }
  __syncthreads();
  *total = all;
  return before + incl - v;
}

// One warp, one batch of up to 32 items [item, hi) of a table piece whose
// first column is pc: item k lies in entry e (column pc + e / ndel, bucket
// e % ndel) with tab[e] <= k < tab[e + 1].
template <int PREC, int INFL>
__device__ __forceinline__ void deliver_batch(const StepParams& P, unsigned item, unsigned hi,
                                              const DeliverSmem& S, int n_entries, int pc,
                                              uint32_t win_s, uint32_t wbase, uint32_t wlen,
                                              uint64_t pol, const uint32_t* nb) {
  const int lane = threadIdx.x & 31;
  int len = 0;
  unsigned long long base = 0ull;
  uint32_t info = 0u;
  if (item < hi) {
    int lo_e = 0, hi_e = n_entries;  // tab[lo_e] <= item < tab[hi_e]
    while (hi_e - lo_e > 1) {
      const int mid = (lo_e + hi_e) >> 1;
      if (S.tab[mid] <= item)
        lo_e = mid;
      else
        hi_e = mid;
    }
    const int k = lo_e / P.ndel;
    const int b = lo_e - k * P.ndel;
    const int c = pc + k;
    const uint32_t j = P.ids[(long long)S.slot[b] * P.N + (long long)c * P.npc + (item - S.tab[lo_e])];
    const uint8_t* be = P.bend + (long long)j * kBendStride;
    const int beg = (b ? (int)be[b - 1] : 0) * kSlotUnit;
    const int end = (int)be[b] * kSlotUnit;
    len = end - beg;
    base = (unsigned long long)j * (unsigned long long)P.rowcap + (unsigned long long)beg;
    const bool inh = (int)(j - (uint32_t)c * (uint32_t)P.npc) >= P.nexc;
    if (PREC == SNN_EXACT_F16W) {
      info = (uint32_t)k | ((inh ? 1u : 0u) << 28);  // column within the piece
    } else {
      const int cy = c / P.W;
      info = pack_info(c - cy * P.W, cy, inh);
    }
  }
  // compact the non-empty items to lanes 0..nit-1
  const unsigned cm = __ballot_sync(0xFFFFFFFFu, len > 0);
  const int nit = __popc(cm);
  const int src = lane < nit ? (int)__fns(cm, 0u, lane + 1) : 0;
  int lenc = __shfl_sync(0xFFFFFFFFu, len, src);
  const unsigned blo0 = __shfl_sync(0xFFFFFFFFu, (unsigned)base, src);
  const unsigned bhi0 = __shfl_sync(0xFFFFFFFFu, (unsigned)(base >> 32), src);
  const uint32_t infc = __shfl_sync(0xFFFFFFFFu, info, src);
  if (lane >= nit) lenc = 0;
  int incl = lenc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  const int pre = incl - lenc;  // first flat slot of compact item `lane`
  const int T = __shfl_sync(0xFFFFFFFFu, incl, 31);
  const unsigned long long bc = (((unsigned long long)bhi0 << 32) | blo0) - (unsigned long long)pre;
  const unsigned blo = (unsigned)bc, bhi = (unsigned)(bc >> 32);
  const bool mine = lane < nit;
  const unsigned le_mask = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);

  for (int f0 = 0; f0 < T; f0 += 128 * INFL) {
    // the chunks' raw words: 4 per lane for F16W, 8 for F32W; padding where
    // a lane has no chunk
    constexpr int kWords = PREC == SNN_EXACT_F16W ? 4 : 8;
    uint32_t raw[INFL][kWords];
    uint32_t inf[INFL];
#pragma unroll
    for (int u = 0; u < INFL; ++u) {
      const int fu = f0 + u * 128;
      inf[u] = 0u;
#pragma unroll
      for (int q = 0; q < kWords; ++q) raw[u][q] = kPad;
      if (fu < T) {
        // item of the chunk at flat slot fu + 4 * lane: the item holding fu,
        // plus the items that start between fu and the lane's chunk
        const int ebase = __popc(__ballot_sync(0xFFFFFFFFu, mine && pre <= fu)) - 1;
        const int pos = (pre - fu) >> 2;
        const unsigned bit = (mine && pre > fu && pos < 32) ? (1u << pos) : 0u;
        const unsigned starts = __reduce_or_sync(0xFFFFFFFFu, bit);
        const int e = ebase + __popc(starts & le_mask);
        const unsigned bl = __shfl_sync(0xFFFFFFFFu, blo, e);
        const unsigned bh = __shfl_sync(0xFFFFFFFFu, bhi, e);
        inf[u] = __shfl_sync(0xFFFFFFFFu, infc, e);
        const int f = fu + 4 * lane;
        if (f < T) {
          const long long slot = (long long)(((unsigned long long)bh << 32) | bl) + f;
          if (PREC == SNN_EXACT_F16W) {
            const uint4 r = __ldcs(reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(P.syn) + slot));
            raw[u][0] = r.x;
            raw[u][1] = r.y;
            raw[u][2] = r.z;
            raw[u][3] = r.w;
          } else {
            const uint4* p4 = reinterpret_cast<const uint4*>(static_cast<const uint2*>(P.syn) + slot);
            const uint4 r0 = __ldcs(p4);
            const uint4 r1 = __ldcs(p4 + 1);
            raw[u][0] = r0.x; raw[u][1] = r0.y; raw[u][2] = r0.z; raw[u][3] = r0.w;
            raw[u][4] = r1.x; raw[u][5] = r1.y; raw[u][6] = r1.z; raw[u][7] = r1.w;
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < INFL; ++u) {
#pragma unroll
      for (int qd = 0; qd < 4; ++qd) {
        if (PREC == SNN_EXACT_F16W) {
          const uint32_t w = raw[u][qd];
          deliver_record<PREC>(w == kPad ? kPad : (w & 0x1FFFFu), w >> 17, inf[u], win_s, wbase,
                               wlen, pol, nb, P);
        } else {
          deliver_record<PREC>(raw[u][2 * qd], raw[u][2 * qd + 1], inf[u], win_s, wbase, wlen,
                               pol, nb, P);
        }
      }
    }
  }
}

// Delivery block vb of vgrid for step t.  The step's items, ordered by
// (column, delay bucket, spiker), are split into vgrid equal contiguous
// ranges; block vb locates the first and last column of its range from the
// group and column counts (gsum, isum), tabulates the (column, bucket) counts
// of those columns (in pieces of at most kTabEntries entries) and lets its
// warps take batches of kBatchItems items.  With P.agg the synapses onto the
// first kWindows columns of each piece, from any of the piece's items, are
// summed in shared memory (win_base, kWindows * n_per_col ints) and flushed
// once per piece.
template <int PREC, int INFL>
__device__ __forceinline__ void deliver_body(const StepParams& P, long long t, int vb, int vgrid,
                                             DeliverSmem& S, int32_t* win_base, uint32_t* nb) {
  __syncthreads();  // the shared memory may still be read by a previous body
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // the slot that the next update fills holds step t - d_max: no longer read
  const long long next_slot = (t + 1) % P.nslot;
  if (vb == 0 && threadIdx.x == 0) P.cnt[next_slot] = 0u;
  for (long long c = (long long)vb * blockDim.x + threadIdx.x; c < P.ncol;
       c += (long long)vgrid * blockDim.x)
    P.ccnt[next_slot * P.ncol + c] = 0u;
  if (P.agg)
    for (int l = threadIdx.x; l < kWindows * P.npc; l += blockDim.x) win_base[l] = 0;
  if (threadIdx.x < kMaxDelays) {
    const int b = threadIdx.x;
    const long long s = t + 1 - (P.dmin + b);
    S.slot[b] = (b < P.ndel && s >= 0) ? (int)(s % P.nslot) : -1;
  }
  if (threadIdx.x == 0) {
    S.c0 = -1;
    S.c1 = -1;
    S.next = 0u;
  }

  // the block's item range, from the group counts
  const int ngrp = (P.ncol + 31) >> 5;
  const int per = (ngrp + (int)blockDim.x - 1) / (int)blockDim.x;
  const int g0 = threadIdx.x * per;
  unsigned long long mine = 0ull;
  for (int g = g0; g < g0 + per && g < ngrp; ++g) mine += P.gsum[g];
  unsigned long long total = 0ull;
  const unsigned long long excl = block_scan(mine, S, &total);
  const unsigned long long lo = total * (unsigned long long)vb / (unsigned long long)vgrid;
  const unsigned long long hi = total * (unsigned long long)(vb + 1) / (unsigned long long)vgrid;
  if (lo >= hi) return;
  for (int i = 0; i < 2; ++i) {
    const unsigned long long x = i == 0 ? lo : hi - 1;
    if (x >= excl && x < excl + mine) {
      unsigned long long run = excl;
      for (int g = g0; g < g0 + per && g < ngrp; ++g) {
        const unsigned v = P.gsum[g];
        if (x < run + v) {
          S.xg[i] = g;
          S.xgp[i] = run;
          break;
        }
        run += v;
      }
    }
  }
  __syncthreads();
  // the columns holding lo and hi - 1, from the column counts of their groups
  if (warp < 2) {
    const unsigned long long x = warp == 0 ? lo : hi - 1;
    const int c = S.xg[warp] * 32 + lane;
    const unsigned v = c < P.ncol ? P.isum[c] : 0u;
    unsigned incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += u;
    }
    const unsigned long long pos = S.xgp[warp] + incl - v;
    if (c < P.ncol && x >= pos && x < pos + v) {
      if (warp == 0) {
        S.c0 = c;
        S.p0 = pos;
      } else {
        S.c1 = c;
      }
    }
  }
  __syncthreads();
  const int c0 = S.c0, c1 = S.c1;
  if (c0 < 0 || c1 < c0) return;  // inconsistent counts: nothing is delivered

  const uint64_t pol = evict_last_policy();
  const uint32_t win_s = (uint32_t)__cvta_generic_to_shared(win_base);
  // a piece tabulates at most 4 entries per thread and kPieceCols columns
  const int cols_per_piece = min(min(kTabEntries, 4 * (int)blockDim.x) / P.ndel, kPieceCols);
  unsigned long long pbase = S.p0;  // items before the piece's first column
  for (int pc = c0; pc <= c1; pc += cols_per_piece) {
    const int ncp = min(cols_per_piece, c1 - pc + 1);
    const int n_entries = ncp * P.ndel;
    // tabulate the piece: 4 consecutive entries per thread
    unsigned v4[4];
    unsigned sum4 = 0u;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x * 4 + q;
      unsigned v = 0u;
      if (e < n_entries) {
        const int k = e / P.ndel;
        const int sl = S.slot[e - k * P.ndel];
        v = sl >= 0 ? P.ccnt[(long long)sl * P.ncol + pc + k] : 0u;
      }
      v4[q] = v;
      sum4 += v;
    }
    unsigned long long ptotal = 0ull;
    unsigned run = (unsigned)block_scan(sum4, S, &ptotal);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x * 4 + q;
      if (e < n_entries) S.tab[e] = run;
      run += v4[q];
    }
    if (threadIdx.x == 0) S.tab[n_entries] = (unsigned)ptotal;
    __syncthreads();
    const unsigned a = lo > pbase ? (unsigned)(lo - pbase) : 0u;
    const unsigned b = hi > pbase ? (unsigned)min(hi - pbase, ptotal) : 0u;
    if (PREC == SNN_EXACT_F16W) {
      // first neuron of the column at each stencil offset of each column of
      // the piece (periodic), for the records' column-relative targets
      for (int m = threadIdx.x; m < ncp * 64; m += blockDim.x) {
        const int c = pc + (m >> 6), off = m & 63;
        const int cy = c / P.W, cx = c - cy * P.W;
        const int ty = wrap(cy + (off >> 3) - 3, P.H), tx = wrap(cx + (off & 7) - 3, P.W);
        nb[m] = ((uint32_t)ty * (uint32_t)P.W + (uint32_t)tx) * (uint32_t)P.npc;
      }
      __syncthreads();
    }
    // windows: the piece's first columns, for synapses from any of its items
    const uint32_t wbase = (uint32_t)pc * (uint32_t)P.npc;
    const uint32_t wlen = P.agg ? (uint32_t)min(kWindows, ncp) * (uint32_t)P.npc : 0u;
    while (a < b) {
      unsigned k0 = 0u;
      if (lane == 0) k0 = atomicAdd(&S.next, (unsigned)kBatchItems);
      k0 = __shfl_sync(0xFFFFFFFFu, k0, 0);
      if (a + k0 >= b) break;
      const unsigned end = min(b, a + k0 + (unsigned)kBatchItems);
      deliver_batch<PREC, INFL>(P, lane < kBatchItems ? a + k0 + lane : end, end, S, n_entries, pc,
                                win_s, wbase, wlen, pol, nb);
    }
    __syncthreads();
    // flush the windows with coalesced reductions, leaving them zeroed
    for (uint32_t m = threadIdx.x; m < wlen; m += blockDim.x) {
      const int32_t v = win_base[m];
      if (v) {
        red_add(P.acc + wbase + m, v, pol);
        win_base[m] = 0;
      }
    }
    if (threadIdx.x == 0) S.next = 0u;
    pbase += ptotal;
    __syncthreads();
  }
}

template <int PREC>
__global__ void __launch_bounds__(kDeliverThreads) deliver_kernel(const StepParams P) {
  extern __shared__ int32_t s_win[];  // [kWindows][n_per_col] when P.agg
  __shared__ DeliverSmem S;
  __shared__ uint32_t s_nb[PREC == SNN_EXACT_F16W ? kNbEntries : 1];
  const long long t = P.ctl->t;
  deliver_body<PREC, PREC == SNN_EXACT_F16W ? kInflightF16 : kInflight>(
      P, t, (int)blockIdx.x, (int)gridDim.x, S, s_win, s_nb);

  // the last block to finish closes the step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&P.ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      P.ctl->done = 0u;
      P.ctl->t = t + 1;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched form: many independent nets advanced by one persistent launch.
// Every step runs the update blocks of all nets, a grid barrier, the delivery
// blocks of all nets, and a second barrier.  Virtual block g of a phase
// belongs to net k with first[k] <= g < first[k + 1]; each virtual block is the
// standalone kernel's block, so every net computes exactly what its own
// kernels compute.
// ---------------------------------------------------------------------------

// Bounded grid barrier (all blocks are co-resident: cooperative launch).  A
// block that polls spin_limit times without the generation moving sets *err
// and gives up; every later barrier then returns false at once.
__device__ __forceinline__ bool grid_barrier(const BatchParams& B, unsigned* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned ok = 1u;
    volatile unsigned* gen = B.bar + 1;
    volatile unsigned* err = B.bar + 2;
    if (*err) {
      ok = 0u;
    } else {
      const unsigned g = *gen;
      __threadfence();
      const unsigned expected = gridDim.x + B.extra_arrivals;
      if (atomicAdd(B.bar, 1u) == expected - 1u) {
        B.bar[0] = 0u;
        __threadfence();
        atomicAdd(B.bar + 1, 1u);
      } else {
        long long polls = 0;
        while (*gen == g) {
          if (*err) {
            ok = 0u;
            break;
          }
          if (++polls > B.spin_limit) {
            atomicExch(B.bar + 2, 1u);
            ok = 0u;
            break;
          }
          __nanosleep(64);
        }
      }
      __threadfence();
    }
    *s_ok = ok;
  }
  __syncthreads();
  return *s_ok != 0u;
}

// Net of virtual block g: the last k with first[k] <= g.
__device__ __forceinline__ int net_of(const int* first, int n, int g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int PREC, int INFL>
__global__ void __launch_bounds__(kBatchThreads, 3) batch_kernel(const BatchParams B) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ StepParams s_p;  // the current virtual block's net
  __shared__ uint32_t s_nb[PREC == SNN_EXACT_F16W ? kNbEntries : 1];
  __shared__ int s_uf[kMaxBatch + 1], s_df[kMaxBatch + 1];
  __shared__ unsigned s_ok;
  UpdateSmem& SU = *reinterpret_cast<UpdateSmem*>(s_dyn);
  DeliverSmem& SD = *reinterpret_cast<DeliverSmem*>(s_dyn);
  int32_t* win = reinterpret_cast<int32_t*>(s_dyn + kDeliverSmemPad);
  const int n = B.n_nets;
  for (int k = threadIdx.x; k <= n; k += blockDim.x) {
    s_uf[k] = B.u_first[k];
    s_df[k] = B.d_first[k];
  }
  __syncthreads();
  const int total_u = s_uf[n], total_d = s_df[n];
  for (long long step = 0; step < B.n_steps; ++step) {
    const long long t = B.t0 + step;
    for (int g = blockIdx.x; g < total_u; g += gridDim.x) {
      const int k = net_of(s_uf, n, g);
      __syncthreads();
      for (int w = threadIdx.x; w < (int)(sizeof(StepParams) / 4); w += blockDim.x)
        reinterpret_cast<uint32_t*>(&s_p)[w] = reinterpret_cast<const uint32_t*>(B.nets + k)[w];
      __syncthreads();
      update_body(s_p, t, g - s_uf[k], s_uf[k + 1] - s_uf[k], SU);
    }
    if (!grid_barrier(B, &s_ok)) return;
    for (int g = blockIdx.x; g < total_d; g += gridDim.x) {
      const int k = net_of(s_df, n, g);
      __syncthreads();
      for (int w = threadIdx.x; w < (int)(sizeof(StepParams) / 4); w += blockDim.x)
        reinterpret_cast<uint32_t*>(&s_p)[w] = reinterpret_cast<const uint32_t*>(B.nets + k)[w];
      __syncthreads();
      deliver_body<PREC, INFL>(s_p, t, g - s_df[k], s_df[k + 1] - s_df[k], SD, win, s_nb);
    }
    if (!grid_barrier(B, &s_ok)) return;
  }
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < n; k += blockDim.x) B.nets[k].ctl->t = B.t0 + B.n_steps;
}

// Spike-record drain, one kernel.  Block b copies the records kept in region
// b (rcnt[b], at most `region`; records are step << 32 | id) as separate id
// and step arrays, starting at the number of records kept in the regions
// before b, to the mapped host buffers when all kept records fit them
// (map_cap) and to the device stage otherwise.  Block 0 writes the header
// {records kept, 1 if any were dropped, first step, last step} to device and
// mapped host memory (each region is in step order, so its first and last
// records bound its steps).  The last block to finish resets the region
// counters and the overflow flag.
__global__ void __launch_bounds__(256) drain_records_kernel(
    unsigned long long* rcnt, int nreg, long long region, const unsigned long long* rec,
    Ctl* ctl, unsigned long long* header, unsigned long long* map_hdr, uint32_t* stage_ids,
    uint32_t* stage_steps, uint32_t* map_ids, uint32_t* map_steps, long long map_cap) {
  __shared__ unsigned long long s_pre[8], s_tot[8];
  __shared__ unsigned s_tmin[8], s_tmax[8], s_lost[8];
  __shared__ bool s_last;
  const int b = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long pre = 0ull, tot = 0ull;
  unsigned tmin = 0xFFFFFFFFu, tmax = 0u, lost = 0u;
  for (int r = threadIdx.x; r < nreg; r += blockDim.x) {
    const unsigned long long v = rcnt[r];
    const unsigned long long kept = (long long)v < region ? v : (unsigned long long)region;
    lost |= (long long)v > region ? 1u : 0u;
    tot += kept;
    if (r < b) pre += kept;
    if (b == 0 && kept > 0ull) {
      const unsigned first = (unsigned)(rec[(long long)r * region] >> 32);
      const unsigned lastt = (unsigned)(rec[(long long)r * region + (long long)kept - 1] >> 32);
      tmin = min(tmin, first);
      tmax = max(tmax, lastt);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    pre += __shfl_xor_sync(0xFFFFFFFFu, pre, o);
    tot += __shfl_xor_sync(0xFFFFFFFFu, tot, o);
    tmin = min(tmin, __shfl_xor_sync(0xFFFFFFFFu, tmin, o));
    tmax = max(tmax, __shfl_xor_sync(0xFFFFFFFFu, tmax, o));
    lost |= __shfl_xor_sync(0xFFFFFFFFu, lost, o);
  }
  if (lane == 0) {
    s_pre[w] = pre;
    s_tot[w] = tot;
    s_tmin[w] = tmin;
    s_tmax[w] = tmax;
    s_lost[w] = lost;
  }
  __syncthreads();
  pre = 0ull;
  tot = 0ull;
  tmin = 0xFFFFFFFFu;
  tmax = 0u;
  lost = 0u;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
    pre += s_pre[k];
    tot += s_tot[k];
    tmin = min(tmin, s_tmin[k]);
    tmax = max(tmax, s_tmax[k]);
    lost |= s_lost[k];
  }
  if (b == 0 && threadIdx.x == 0) {
    const unsigned long long h[4] = {tot, (lost || ctl->rec_overflow) ? 1ull : 0ull,
                                     (unsigned long long)tmin, (unsigned long long)tmax};
    for (int k = 0; k < 4; ++k) {
      header[k] = h[k];
      map_hdr[k] = h[k];
    }
  }
  const bool to_map = (long long)tot <= map_cap;
  uint32_t* ids = (to_map ? map_ids : stage_ids) + pre;
  uint32_t* steps = (to_map ? map_steps : stage_steps) + pre;
  const unsigned long long v = rcnt[b];
  const long long kept = (long long)v < region ? (long long)v : region;
  const unsigned long long* src = rec + (long long)b * region;
  for (long long k = threadIdx.x; k < kept; k += blockDim.x) {
    const unsigned long long r = src[k];
    ids[k] = (uint32_t)r;
    steps[k] = (uint32_t)(r >> 32);
  }
  // the counters are read by every block: the last one to finish resets them
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(&ctl->drained, 1u) == (unsigned)nreg - 1u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int r = threadIdx.x; r < nreg; r += blockDim.x) rcnt[r] = 0ull;
    if (threadIdx.x == 0) {
      ctl->rec_overflow = 0u;
      ctl->drained = 0u;
    }
  }
}

// Sum of the per-block spike counts (measurement helper).
__global__ void sum_parts_kernel(const unsigned long long* part, int n, unsigned long long* out) {
  unsigned long long s = 0ull;
  for (int i = threadIdx.x; i < n; i += 32) s += part[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
  if (threadIdx.x == 0) *out = s;
}

}  // namespace

int update_grid(long long N, int num_sms) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, update_kernel, kUpdateThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const long long tiles = ((N + 3) / 4 + kUpdateThreads - 1) / kUpdateThreads;
  const long long g = (long long)per_sm * num_sms;
  return (int)(tiles < g ? tiles : g);
}

cudaError_t launch_update(const StepParams& p, int grid, cudaStream_t st) {
  update_kernel<<<grid, kUpdateThreads, 0, st>>>(p);
  return cudaGetLastError();
}

size_t deliver_smem(int npc, bool agg) {
  return agg ? (size_t)kWindows * (size_t)npc * sizeof(int32_t) : 0u;
}

// Delivery grid: a persistent grid at full occupancy.
int deliver_grid(int precision, int num_sms, int npc, bool agg) {
  const size_t smem = deliver_smem(npc, agg);
  int per_sm = 0;
  if (precision == SNN_EXACT_F16W) {
    cudaFuncSetAttribute(deliver_kernel<SNN_EXACT_F16W>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_kernel<SNN_EXACT_F16W>,
                                                  kDeliverThreads, smem);
  } else {
    cudaFuncSetAttribute(deliver_kernel<SNN_EXACT_F32W>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_kernel<SNN_EXACT_F32W>,
                                                  kDeliverThreads, smem);
  }
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms;
}

cudaError_t launch_deliver(const StepParams& p, int precision, int grid, cudaStream_t st) {
  const size_t smem = deliver_smem(p.npc, p.agg != 0);
  if (precision == SNN_EXACT_F16W)
    deliver_kernel<SNN_EXACT_F16W><<<grid, kDeliverThreads, smem, st>>>(p);
  else
    deliver_kernel<SNN_EXACT_F32W><<<grid, kDeliverThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_drain_records(const StepParams& p, int nreg, uint32_t* stage_ids,
                                 uint32_t* stage_steps, unsigned long long* header,
                                 unsigned long long* map_hdr, uint32_t* map_ids,
                                 uint32_t* map_steps, long long map_cap, cudaStream_t st) {
  drain_records_kernel<<<nreg, 256, 0, st>>>(p.rcnt, nreg, p.rec_region, p.rec, p.ctl, header,
                                             map_hdr, stage_ids, stage_steps, map_ids, map_steps,
                                             map_cap);
  return cudaGetLastError();
}

namespace {
template <int PREC, int INFL>
void* batch_fn() {
  return reinterpret_cast<void*>(batch_kernel<PREC, INFL>);
}
void* batch_kernel_ptr(int precision, int infl) {
  if (precision == SNN_EXACT_F16W) return infl == 2 ? batch_fn<1, 2>() : batch_fn<1, 4>();
  return infl == 2 ? batch_fn<0, 2>() : batch_fn<0, 4>();
}
}  // namespace

size_t batch_smem(int max_npc) {
  const size_t upd = sizeof(UpdateSmem);
  const size_t del = kDeliverSmemPad + (size_t)kWindows * (size_t)max_npc * sizeof(int32_t);
  return upd > del ? upd : del;
}

int batch_grid(int precision, int infl, int num_sms, int max_npc) {
  const size_t smem = batch_smem(max_npc);
  void* fn = batch_kernel_ptr(precision, infl);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, smem);
  return per_sm * num_sms;
}

cudaError_t launch_batch(const BatchParams& b, int precision, int infl, int grid, int max_npc,
                         cudaStream_t st) {
  void* args[] = {const_cast<BatchParams*>(&b)};
  return cudaLaunchCooperativeKernel(batch_kernel_ptr(precision, infl), dim3(grid),
                                     dim3(kBatchThreads), args, batch_smem(max_npc), st);
}

cudaError_t launch_sum_parts(const unsigned long long* part, int n, unsigned long long* out,
                             cudaStream_t st) {
  sum_parts_kernel<<<1, 32, 0, st>>>(part, n, out);
  return cudaGetLastError();
}

}  // namespace snn
