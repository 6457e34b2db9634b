// snn_step.cu -- the two kernels of one 1 ms step.
//
// update_kernel (neuron update, arxiv 1511.09325 Sec. 2 LIF + SFA):
//   grid-stride over tiles of 1024 neurons; one thread owns 4 consecutive
//   neurons and one Philox4x32-10 block (counter (i/4, t, EXT, 0)) whose 4
//   words give their external Poisson counts.  It reads and clears their
//   recurrent input, applies refractoriness, threshold, reset and the exact
//   propagator with explicitly rounded FP32 operations.  A tile's spikes are
//   counted per column in shared memory and written to their column's part of
//   the step's spike list (one atomic per column and tile) as descriptors --
//   the spiker's id and its bucket ends, so that a delivery finds a bucket
//   with one load -- and to the block's record region.  The per-column item
//   counts of the next delivery (isum, gsum) are kept up to date here; spike
//   and external-event totals go to per-block partial sums.
//
// deliver_kernel (event-driven delivery, Sec. 1), "pull by delay": the input
//   of step t+1 is the sum over delays d of bucket d of every neuron that
//   spiked at step t+1-d, so only one N-entry accumulator (resident in L2)
//   receives additions, not a d_max-slot ring.  The (delay bucket, spiker)
//   items of the last d_max steps, ordered by (virtual column, bucket,
//   spiker), form one virtual list split evenly over a persistent grid of one
//   768-thread block per SM.  Virtual columns run tile by tile (tiles of
//   tile x tile columns, 6 x 6 at n_per_col = 1240), so a block's items come
//   from a compact patch of the grid.  For each tile part with enough items,
//   a block keeps a shared-memory window over the tile's columns (and a ring
//   of P.ring columns around them) -- where about four fifths of the tile's
//   synapses land (the local half and most of the near stencil) -- sums
//   those synapses there with shared-memory reductions and flushes the window
//   once into the accumulator by bulk asynchronous reductions; the other
//   synapses go to L2 as fire-and-forget int32 reductions.  A warp takes
//   batches of 32 items: lane e resolves item e (a binary search in the tile
//   part's table of (column, bucket) counts and one descriptor load); the
//   batch's buckets are then streamed as one list of 32-byte sectors dealt to
//   the lanes in balanced rounds, two rounds in flight, and the next batch is
//   resolved before the current one is streamed.  Integer addition makes the
//   result independent of the order.  The last block to finish advances the
//   step counter.
#include <algorithm>

#include "snn_device.cuh"
#include "snn_internal.h"

namespace snn {
namespace {

constexpr int kUpdateThreads = 256;
constexpr int kDeliverThreads = 768;   // one delivery block per SM (24 warps, 2 rounds in flight)
constexpr int kBatchThreads = 512;     // batch kernel: 2 update sub-blocks or one delivery block
constexpr int kUpdateSubs = kBatchThreads / kUpdateThreads;
constexpr int kDepthF32 = 2;     // rounds of 32-byte sectors in flight per lane, F32W
constexpr int kDepthF16 = 2;     // the same, F16W
constexpr int kTile = kUpdateThreads * 4;    // neurons per update tile
constexpr int kStageSpikes = 128;            // spikers per tile whose bucket ends are staged
constexpr int kTileCols = kTile / 2 + 2;     // columns a tile can touch (npc >= 2)
constexpr int kBatchItems = 32;              // items per warp batch (one per lane)

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

// Loads of the neuron state, read once per step: no L1 allocation, so that
// L1 capacity does not bound the loads a block keeps in flight.
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  float4 v;
  asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ int4 ld_stream(const int4* p) {
  int4 v;
  asm volatile("ld.global.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}
__device__ __forceinline__ uchar4 ld_stream(const uchar4* p) {
  uint32_t v;
  asm volatile("ld.global.L1::no_allocate.u32 %0, [%1];" : "=r"(v) : "l"(p));
  return make_uchar4((unsigned char)v, (unsigned char)(v >> 8), (unsigned char)(v >> 16),
                     (unsigned char)(v >> 24));
}

// Barrier of an update body: the whole block (bar 0) or one 256-thread
// sub-block of the batch kernel (named barrier `bar`).
__device__ __forceinline__ void body_sync(int bar) {
  if (bar == 0)
    __syncthreads();
  else
    asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(kUpdateThreads) : "memory");
}

// Records the first inconsistency a kernel finds; the host turns it into
// SNN_ESTATE.
__device__ __forceinline__ void set_status(const StepParams& P, unsigned code) {
  atomicOr(&P.ctl->status, code);
  if (P.hstatus != nullptr) *reinterpret_cast<volatile unsigned*>(P.hstatus) = code;
}

// Shared memory of one update body.
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
  // bucket ends of the tile's first kStageSpikes spikers, copied
  // asynchronously as soon as the spike is known, so the load's latency
  // overlaps the tile's count bookkeeping (later spikers load theirs when
  // the descriptor is written)
  unsigned nbst;
  uint4 bst[kStageSpikes][2];
};

// Update body vb of vgrid for step t, run by kUpdateThreads threads (thread
// index tid, barrier `bar`): tiles vb, vb + vgrid, ...  Body vb owns
// ext_part[vb], spk_part[vb] and record region vb of the net, so the grid
// size must be the same every step.  Each spike goes to the step's list
// (column c's part when P.ccnt is set, else one compact list) -- as a
// descriptor when P.desc is set, else as its id -- and to the body's record
// region as (step << 32 | id).  A shard (SHARD, P.sg.on) updates its own
// columns only, draws the external input with global neuron indices and
// records global indices; the halo's columns take part in the count
// bookkeeping.
template <bool SHARD>
__device__ __forceinline__ void update_body(const StepParams& P, long long t, int vb, int vgrid,
                                            UpdateSmem& S, int tid, int bar) {
  body_sync(bar);  // the shared memory may still be read by a previous body
  const int slot = (int)(t % P.nslot);
  for (int m = tid; m < 256; m += kUpdateThreads) S.guide[m] = P.pois_guide[m];
  for (int m = tid; m <= kMaxPoisThr; m += kUpdateThreads) S.thr[m] = P.pois_thr[m];
  if (tid == 0) {
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

  // the state of the body's next tile is requested before the current tile
  // is processed, so its latency overlaps the current tile's work
  float4 pv = make_float4(0.f, 0.f, 0.f, 0.f), pc = pv;
  uchar4 pr = make_uchar4(0, 0, 0, 0);
  int4 pa = make_int4(0, 0, 0, 0);
  {
    const long long q0 = (long long)vb * kUpdateThreads + tid;
    if (vb < tiles && q0 * 4 < P.N) {
      pv = ld_stream(reinterpret_cast<const float4*>(P.V) + q0);
      pc = ld_stream(reinterpret_cast<const float4*>(P.C) + q0);
      pr = ld_stream(reinterpret_cast<const uchar4*>(P.R) + q0);
      pa = ld_stream(reinterpret_cast<const int4*>(P.acc) + q0);
    }
  }
  for (long long tile = vb; tile < tiles; tile += vgrid) {
    const float4 v4 = pv, c4 = pc;
    const uchar4 r4 = pr;
    const int4 a4 = pa;
    {
      const long long qn = (tile + vgrid) * kUpdateThreads + tid;
      if (tile + vgrid < tiles && qn * 4 < P.N) {
        pv = ld_stream(reinterpret_cast<const float4*>(P.V) + qn);
        pc = ld_stream(reinterpret_cast<const float4*>(P.C) + qn);
        pr = ld_stream(reinterpret_cast<const uchar4*>(P.R) + qn);
        pa = ld_stream(reinterpret_cast<const int4*>(P.acc) + qn);
      }
    }
    const long long first = tile * kTile;
    const long long last = (first + kTile < P.N ? first + kTile : P.N) - 1;
    // neuron indices are below 2^31: 32-bit divisions are exact (and cheap)
    const int col0 = (int)((uint32_t)first / (uint32_t)P.npc);
    const int ncols = (int)((uint32_t)last / (uint32_t)P.npc) - col0 + 1;
    for (int k = tid; k < ncols; k += kUpdateThreads) {
      S.tpop[k][0] = 0u;
      S.tpop[k][1] = 0u;
    }
    if (tid == 0) S.nbst = 0u;
    body_sync(bar);

    const long long q = tile * kUpdateThreads + tid;
    const long long i0 = q * 4;
    unsigned rank[4] = {0u, 0u, 0u, 0u};
    int scol[4] = {-1, -1, -1, -1};
    uint32_t gq = (uint32_t)q;  // global quad of the four neurons
    bool own = true;
    if (SHARD && i0 < P.N) {
      const int c = (int)((uint32_t)i0 / (uint32_t)P.npc);
      const int l0 = (int)((uint32_t)i0 - (uint32_t)c * (uint32_t)P.npc);
      const int cy = c / P.W, cx = c - cy * P.W;
      own = cx >= P.sg.tx0 && cx < P.sg.tx0 + P.sg.tw && cy >= P.sg.ty0 && cy < P.sg.ty0 + P.sg.th;
      int gx, gy;
      shard_global_col(P.sg, cx, cy, &gx, &gy);
      gq = (((uint32_t)gy * (uint32_t)P.sg.GW + (uint32_t)gx) * (uint32_t)P.npc + (uint32_t)l0) >> 2;
    }
    if (i0 < P.N && own) {
      const uint4 x = philox4x32_10(make_uint4(gq, (uint32_t)t, kTagExt, 0u), P.seed_lo, P.seed_hi);
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
      if (P.desc != nullptr) {
        // stage the bucket ends of the first kStageSpikes spikers (slot in
        // bits 16..23 of the rank; 255: none)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (scol[e] >= 0) {
            const unsigned bs = atomicAdd(&S.nbst, 1u);
            if (bs < (unsigned)kStageSpikes) {
              const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&S.bst[bs][0]);
              const uint4* src = reinterpret_cast<const uint4*>(P.bend + (i0 + e) * kBendStride);
              asm volatile(
                  "cp.async.cg.shared.global [%0], [%1], 16;\n\t"
                  "cp.async.cg.shared.global [%2], [%3], 16;" ::"r"(dst),
                  "l"(src), "r"(dst + 16u), "l"(src + 1)
                  : "memory");
            }
            rank[e] |= (bs < (unsigned)kStageSpikes ? bs : 255u) << 16;
          }
        }
      }
      reinterpret_cast<float4*>(P.V)[q] = make_float4(vout[0], vout[1], vout[2], vout[3]);
      reinterpret_cast<float4*>(P.C)[q] = make_float4(cout[0], cout[1], cout[2], cout[3]);
      reinterpret_cast<uchar4*>(P.R)[q] = make_uchar4((unsigned char)rout[0], (unsigned char)rout[1],
                                                      (unsigned char)rout[2], (unsigned char)rout[3]);
    }
    body_sync(bar);
    // places: records grouped by column (E then I) in the body's region; list
    // entries in each column's part of the step's list (or the compact list)
    if (P.ccnt != nullptr) {
      for (int k = tid; k < ncols; k += kUpdateThreads) {
        const unsigned n = S.tpop[k][0] + S.tpop[k][1];
        const int c = col0 + k;
        S.lbase[k] = (long long)c * P.npc +
                     (n ? (long long)atomicAdd(P.ccnt + (long long)slot * P.ncol + c, n) : 0ll);
        unsigned d = P.dmin == 1 ? n : 0u;
        if ((long long)c * P.npc >= first) d += (cin_ ? cin_[c] : 0u) - cout_[c];
        if (d) {
          const int v = P.colv != nullptr ? (int)P.colv[c] : c;
          atomicAdd(P.isum + v, d);
          atomicAdd(P.gsum + (v >> 5), d);
        }
      }
    }
    if (tid == 0) {
      unsigned pos = 0u;
      for (int k = 0; k < ncols; ++k) {
        S.tpos[k] = pos;
        pos += S.tpop[k][0] + S.tpop[k][1];
      }
      // the compact list (no per-column lists) takes the tile's spikes at a
      // shared cursor; per-column lists need none
      S.cbase = (pos && P.ccnt == nullptr) ? (long long)atomicAdd(P.cnt + slot, pos) : 0ll;
      S.rbase = S.rc;
      S.rc += pos;
      S.spk += pos;
    }
    body_sync(bar);
    const unsigned long long rc = S.rbase;
    if (P.desc != nullptr) asm volatile("cp.async.wait_all;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (scol[e] >= 0) {
        const int k = scol[e];
        const unsigned r = rank[e] & 0xFFFFu;
        const unsigned off = (rank[e] & 0x80000000u) ? S.tpop[k][0] + r : r;
        const uint32_t id = (uint32_t)(i0 + e);
        const long long pos = P.ccnt != nullptr ? S.lbase[k] + off : S.cbase + S.tpos[k] + off;
        if (P.desc != nullptr) {
          // descriptor: id, then the bucket ends of the spiker's row
          uint4* d = reinterpret_cast<uint4*>(P.desc + ((long long)slot * P.N + pos) * P.desc_words);
          const unsigned bs = (rank[e] >> 16) & 0xFFu;
          uint4 a, b;
          if (bs != 255u) {
            a = S.bst[bs][0];
            b = S.bst[bs][1];
          } else {
            const uint4* be = reinterpret_cast<const uint4*>(P.bend + (long long)id * kBendStride);
            a = be[0];
            b = be[1];
          }
          d[0] = make_uint4(id, a.x, a.y, a.z);
          d[1] = make_uint4(a.w, b.x, b.y, b.z);
          if (P.desc_words == 16) d[2] = make_uint4(b.w, 0u, 0u, 0u);
        } else {
          list[pos] = id;
        }
        syn += P.deg != nullptr ? P.deg[id] : (uint32_t)P.K;
        const unsigned long long ri = rc + S.tpos[k] + off;
        const uint32_t gid = SHARD ? gq * 4u + (uint32_t)e : id;
        if ((long long)ri < P.rec_region) region[ri] = ((unsigned long long)(unsigned)t << 32) | gid;
      }
    }
    for (int k = tid; k < ncols; k += kUpdateThreads) {
      if (S.tpop[k][0]) atomicAdd(&P.colcnt[2 * (col0 + k)], (unsigned long long)S.tpop[k][0]);
      if (S.tpop[k][1]) atomicAdd(&P.colcnt[2 * (col0 + k) + 1], (unsigned long long)S.tpop[k][1]);
    }
    body_sync(bar);
  }

  // external and synaptic events: per-body partial sums, no atomics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, o);
    syn += __shfl_xor_sync(0xFFFFFFFFu, syn, o);
  }
  if ((tid & 31) == 0) {
    S.ksum[tid >> 5] = ksum;
    S.synw[tid >> 5] = syn;
  }
  body_sync(bar);
  if (tid == 0) {
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

template <bool SHARD>
__global__ void __launch_bounds__(kUpdateThreads, 4) update_kernel(const StepParams P) {
  __shared__ UpdateSmem S;
  update_body<SHARD>(P, P.ctl->t, (int)blockIdx.x, (int)gridDim.x, S, (int)threadIdx.x, 0);
}

// ---------------------------------------------------------------------------
// Delivery.
// ---------------------------------------------------------------------------

// Quotient of x by d from m = min(floor(2^32 / d), 2^32 - 1): the estimate
// is at most one below the quotient, so one correction step finishes it.
__device__ __forceinline__ uint32_t div_by(uint32_t x, uint32_t d, uint32_t m) {
  uint32_t q = __umulhi(x, m);
  if (x - q * d >= d) ++q;
  return q;
}

// Tile of virtual column v: tiles of P.tile x P.tile columns in row-major
// order (those of the last tile row or column may be smaller), columns
// row-major inside a tile.
struct TileGeo {
  int first;   // virtual index of the tile's first column
  int x0, y0;  // grid position of its first column
  int tw, th;  // its width and height
};

__device__ __forceinline__ TileGeo tile_geo(const StepParams& P, int v) {
  TileGeo g;
  const int rowcols = P.tile * P.W;  // columns of a full row of tiles
  const int tr = v / rowcols;
  g.y0 = tr * P.tile;
  g.th = min(P.tile, P.H - g.y0);
  const int rem = v - tr * rowcols;
  const int tc = rem / (g.th * P.tile);
  g.x0 = tc * P.tile;
  g.tw = min(P.tile, P.W - g.x0);
  g.first = tr * rowcols + tc * g.th * P.tile;
  return g;
}

// Shared-memory window of a tile: the ww x wh columns starting at (x0, y0)
// (periodic; at most the whole grid, so every column appears once).  Slot
// (rx, ry) holds column ((x0 + rx) mod W, (y0 + ry) mod H).
struct WinGeo {
  int x0, y0, ww, wh;
};

__device__ __forceinline__ WinGeo win_geo(const StepParams& P, const TileGeo& g, bool on) {
  WinGeo w;
  w.ww = min(g.tw + 2 * P.ring, P.W);
  w.wh = min(g.th + 2 * P.ring, P.H);
  w.x0 = w.ww == P.W ? 0 : wrap(g.x0 - P.ring, P.W);
  w.y0 = w.wh == P.H ? 0 : wrap(g.y0 - P.ring, P.H);
  if (!on) w.ww = w.wh = 0;
  return w;
}

struct DeliverSmem {
  unsigned long long wsum[32];    // per-warp sums of block_scan
  unsigned long long xgp[2];      // items before the group holding lo / hi - 1
  unsigned long long ipt[2];      // item positions of the block's range ends
  unsigned long long p0;          // items before virtual column v0
  int xg[2];                      // group holding lo / hi - 1
  int v0, v1;                     // first and last virtual column of the block's items
  int slot[kMaxDelays];           // slot of each bucket's step, -1 before step 0
  int pe;                         // end (exclusive) of the current part
  int pwin;                       // the current part uses the window
  int ccol[kMaxTileCols];         // real column of each column of the current tile part
  int cx[kMaxTileCols], cy[kMaxTileCols];  // its grid position
  uint32_t wbase[(kMaxTile + 2) * (kMaxTile + 2)];  // first neuron of each window slot's column
  unsigned next;                  // next batch of the current tile part
};

// Words of the (column, bucket) table and of the F16W neighbour table of a
// part of `cols` columns.  In the dynamic shared memory of a delivery block
// the tables of a windowed part (one tile, at most tile^2 columns) come first,
// then the window; a part without window (at most part_cols columns) keeps
// its tables at the start of the window area, which it does not use.
__device__ __forceinline__ int tab_words(const StepParams& P, int cols) {
  return (cols * P.ndel + 1 + 3) & ~3;
}
template <int PREC>
__device__ __forceinline__ int nb_words(int cols) {
  return PREC == SNN_EXACT_F16W ? cols * 64 : 0;
}

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

// Neighbour-table entry of F16W record w = half_magnitude(15) << 17 |
// offset(6) << 11 | l(11): in the row `nbrow` of the spiker's column, the
// offset's target column -- its shared-window address, or bit 31 set and its
// first neuron in the accumulator.  The entries of a sector's eight records
// are loaded before any of them is delivered, so the loads are not ordered
// behind the shared-memory reductions.  (Measured: one reduction with a
// generic 64-bit address instead of the two predicated ones made the
// delivery 2.6-2.8x slower: generic atomics on shared memory are slow.)
__device__ __forceinline__ uint32_t nb_entry(uint32_t w, uint32_t nbrow) {
  uint32_t e;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(e) : "r"(nbrow + ((w >> 9) & 0xFCu)));
  return e;
}

// Deliver F16W record w with its table entry e, as one PTX block: the weight
// rint(half * 2^16) comes from one rounded multiply-add (x * (+-2^16) +
// 1.5 * 2^23 lands in [2^23, 2^24), where the float grid is the integers, so
// the low mantissa bits hold the rounded product); one setp gives both
// predicates; zero weights (padding records, unused lanes) deliver nothing.
// No compiler memory barrier: nothing the loop reads aliases the window or
// the accumulator.
__device__ __forceinline__ void deliver_f16(uint32_t w, uint32_t e, float wsign,
                                            const int32_t* acc, uint64_t pol) {
  asm volatile(
      "{\n\t"
      ".reg .u32 t, l, sa, go;\n\t"
      ".reg .b16 h, hh;\n\t"
      ".reg .f32 hf, x;\n\t"
      ".reg .s32 wfx;\n\t"
      ".reg .u64 ga;\n\t"
      ".reg .pred pon, pg, ps;\n\t"
      "and.b32 l, %0, 2047;\n\t"
      "shr.b32 t, %0, 17;\n\t"
      "mov.b32 {h, hh}, t;\n\t"
      "cvt.f32.f16 hf, h;\n\t"
      "fma.rn.f32 x, hf, %2, 0f4B400000;\n\t"
      "mov.b32 wfx, x;\n\t"
      "sub.s32 wfx, wfx, 1262485504;\n\t"
      "setp.ne.s32 pon, wfx, 0;\n\t"
      "setp.lt.and.s32 pg|ps, %1, 0, pon;\n\t"
      "mad.lo.u32 sa, l, 4, %1;\n\t"
      "@ps red.shared.add.s32 [sa], wfx;\n\t"
      "add.u32 go, %1, l;\n\t"
      "and.b32 go, go, 2147483647;\n\t"
      "mad.wide.u32 ga, go, 4, %3;\n\t"
      "@pg red.global.add.L2::cache_hint.s32 [ga], wfx, %4;\n\t"
      "}" ::"r"(w),
      "r"(e), "f"(wsign), "l"(acc), "l"(pol));
}

// F32W record {target neuron, round(w * 2^16)}: the target's column is tested
// against the tile's window; then one setp gives both predicates as above.
__device__ __forceinline__ void deliver_f32(uint32_t t, int32_t wfx, const WinGeo& wg,
                                            uint32_t win_s, const StepParams& P, uint64_t pol) {
  const uint32_t col = div_by(t, (uint32_t)P.npc, P.npc_m);
  const uint32_t l = t - col * (uint32_t)P.npc;
  const uint32_t y = div_by(col, (uint32_t)P.W, P.w_m);
  const uint32_t x = col - y * (uint32_t)P.W;
  int rx = (int)x - wg.x0;
  rx += rx < 0 ? P.W : 0;
  int ry = (int)y - wg.y0;
  ry += ry < 0 ? P.H : 0;
  const uint32_t inwin = ((unsigned)rx < (unsigned)wg.ww && (unsigned)ry < (unsigned)wg.wh) ? 1u : 0u;
  const uint32_t sa = win_s + 4u * (((uint32_t)ry * (uint32_t)wg.ww + (uint32_t)rx) * (uint32_t)P.npc + l);
  const int32_t* ga = P.acc + t;
  asm volatile(
      "{\n\t.reg .pred pon, pg, ps;\n\t"
      "setp.ne.s32 pon, %2, 0;\n\t"
      "setp.eq.and.u32 ps|pg, %3, 1, pon;\n\t"
      "@ps red.shared.add.s32 [%0], %2;\n\t"
      "@pg red.global.add.L2::cache_hint.s32 [%1], %2, %4;\n\t}" ::"r"(sa),
      "l"(ga), "r"(wfx), "r"(inwin), "l"(pol));
}

// A resolved item: the bucket a lane streams.
struct Item {
  const uint4* src;  // first 16 bytes of the bucket
  int units;         // 32-byte sectors
  uint32_t nbrow;    // F16W: shared address of the neighbour-table row of its column
  float wsign;       // F16W: +-2^16, the sign of the spiker's population
};

// Lane's item `item` of a tile part whose (column, bucket) table is
// tab[0 .. n_entries] (none when item >= hi): item k lies in entry e (column
// S.ccol[e / ndel], bucket e % ndel) with tab[e] <= k < tab[e + 1].  Its
// descriptor is read here; the bucket itself is streamed by stream_items.
template <int PREC>
__device__ __forceinline__ Item resolve_item(const StepParams& P, unsigned item, unsigned hi,
                                             const DeliverSmem& S, const unsigned* tab,
                                             int n_entries, uint32_t nb_s) {
  Item it;
  it.src = nullptr;
  it.units = 0;
  it.nbrow = 0u;
  it.wsign = 65536.0f;
  if (item < hi) {
    int lo_e = 0, hi_e = n_entries;  // tab[lo_e] <= item < tab[hi_e]
    while (hi_e - lo_e > 1) {
      const int mid = (lo_e + hi_e) >> 1;
      if (tab[mid] <= item)
        lo_e = mid;
      else
        hi_e = mid;
    }
    const int k = lo_e / P.ndel;
    const int b = lo_e - k * P.ndel;
    const int c = S.ccol[k];
    const uint32_t* D =
        P.desc + ((unsigned long long)S.slot[b] * (unsigned long long)P.N +
                  (unsigned long long)c * (unsigned long long)P.npc + (item - tab[lo_e])) *
                     (unsigned long long)P.desc_words;
    // the descriptor: word 0 the spiker, bytes 4.. its bucket ends (units of
    // 8 slots); bucket b spans ends[b - 1] .. ends[b] (bytes 3 + b and 4 + b)
    const uint32_t j = D[0];
    const int w = (3 + b) >> 2, sh = (3 + b) & 3;
    const uint32_t lo_w = w == 0 ? j : D[w];
    const uint32_t hi_w = sh == 3 ? D[w + 1] : 0u;
    const uint32_t ends = __funnelshift_r(lo_w, hi_w, 8 * sh);
    const int beg = b ? (int)(ends & 0xFFu) : 0;
    const int end = (int)((ends >> 8) & 0xFFu);
    // an 8-slot unit is one sector (F16W) or two (F32W)
    it.units = (end - beg) * (PREC == SNN_EXACT_F16W ? 1 : 2);
    const unsigned long long slot0 =
        (unsigned long long)j * (unsigned long long)P.rowcap + (unsigned long long)beg * kSlotUnit;
    it.src = reinterpret_cast<const uint4*>(static_cast<const char*>(P.syn) +
                                            slot0 * (PREC == SNN_EXACT_F16W ? 4ull : 8ull));
    it.nbrow = nb_s + (uint32_t)k * 256u;
    it.wsign = (int)(j - (uint32_t)c * (uint32_t)P.npc) >= P.nexc ? -65536.0f : 65536.0f;
  }
  return it;
}

// One warp streams the buckets of its lanes' items as one list of 32-byte
// sectors (F16W: 8 records; F32W: 4), dealt to the lanes in rounds of 32, so
// no lane idles while another finishes a longer bucket.  The sector of lane L
// in round g0 belongs to the item holding g0 plus the items that start
// between g0 and g0 + L (a ballot and an or-reduction over the items' first
// sectors); the item's fields come by shuffle.  The next round's sectors are
// requested DEPTH rounds ahead of the ones being delivered.
template <int PREC, int DEPTH>
__device__ __forceinline__ void stream_items(const StepParams& P, const Item& it, uint32_t win_s,
                                             const WinGeo& wg, uint64_t pol) {
  const int lane = threadIdx.x & 31;
  // compact the non-empty items to lanes 0 .. nit - 1
  const unsigned cm = __ballot_sync(0xFFFFFFFFu, it.units > 0);
  const int nit = __popc(cm);
  if (nit == 0) return;
  const int src = lane < nit ? (int)__fns(cm, 0u, lane + 1) : 0;
  const unsigned long long sp = reinterpret_cast<unsigned long long>(it.src);
  int units = __shfl_sync(0xFFFFFFFFu, it.units, src);
  const unsigned slo = __shfl_sync(0xFFFFFFFFu, (unsigned)sp, src);
  const unsigned shi = __shfl_sync(0xFFFFFFFFu, (unsigned)(sp >> 32), src);
  const uint32_t nbr = __shfl_sync(0xFFFFFFFFu, it.nbrow, src);
  const float wsg = __shfl_sync(0xFFFFFFFFu, it.wsign, src);
  const bool mine = lane < nit;
  if (!mine) units = 0;
  int incl = units;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += v;
  }
  const int pre = incl - units;  // first sector of compact item `lane`
  const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
  const unsigned le_mask = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
  const int32_t* acc = P.acc;

  // sector of round g0 for this lane: its two 16-byte halves and its item's fields
  auto fetch = [&](int g0, uint4& r0, uint4& r1, uint32_t& nbrow, float& wsign) {
    r0 = r1 = make_uint4(0u, 0u, 0u, 0u);  // weight 0: nothing delivered
    nbrow = 0u;
    wsign = 65536.0f;
    if (g0 >= total) return;
    const int ebase = __popc(__ballot_sync(0xFFFFFFFFu, mine && pre <= g0)) - 1;
    const int pos = pre - g0;
    const unsigned bit = (mine && pos > 0 && pos < 32) ? (1u << pos) : 0u;
    const unsigned starts = __reduce_or_sync(0xFFFFFFFFu, bit);
    const int e = ebase + __popc(starts & le_mask);
    const unsigned lo = __shfl_sync(0xFFFFFFFFu, slo, e);
    const unsigned hi = __shfl_sync(0xFFFFFFFFu, shi, e);
    const int first = __shfl_sync(0xFFFFFFFFu, pre, e);
    nbrow = __shfl_sync(0xFFFFFFFFu, nbr, e);
    wsign = __shfl_sync(0xFFFFFFFFu, wsg, e);
    const int g = g0 + lane;
    if (g < total) {
      const uint4* p = reinterpret_cast<const uint4*>((((unsigned long long)hi << 32) | lo)) +
                       2 * (g - first);
      r0 = __ldcs(p);
      r1 = __ldcs(p + 1);
    }
  };

  // a ring of DEPTH stages: stage s holds the round g0 + 32 s and, once it
  // has been delivered, is refilled with the round DEPTH stages later
  uint4 a[DEPTH], b[DEPTH];
  uint32_t nbs[DEPTH];
  float wss[DEPTH];
#pragma unroll
  for (int st = 0; st < DEPTH; ++st) fetch(32 * st, a[st], b[st], nbs[st], wss[st]);
  for (int g0 = 0; g0 < total; g0 += 32 * DEPTH) {
#pragma unroll
    for (int st = 0; st < DEPTH; ++st) {
      if (g0 + 32 * st < total) {
        if (PREC == SNN_EXACT_F16W) {
          const uint32_t w8[8] = {a[st].x, a[st].y, a[st].z, a[st].w,
                                  b[st].x, b[st].y, b[st].z, b[st].w};
          uint32_t e8[8];
#pragma unroll
          for (int q = 0; q < 8; ++q) e8[q] = nb_entry(w8[q], nbs[st]);
#pragma unroll
          for (int q = 0; q < 8; ++q) deliver_f16(w8[q], e8[q], wss[st], acc, pol);
        } else {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint4 r = h ? b[st] : a[st];
            deliver_f32(r.x, (int32_t)r.y, wg, win_s, P, pol);
            deliver_f32(r.z, (int32_t)r.w, wg, win_s, P, pol);
          }
        }
      }
      fetch(g0 + 32 * (st + DEPTH), a[st], b[st], nbs[st], wss[st]);
    }
  }
}

// Adds the window's `slots` columns (n_per_col = npc words each, npc a
// multiple of 4) into the accumulator with one bulk asynchronous reduction
// (cp.reduce.async.bulk .add.s32, element-wise atomic in L2) per column,
// issued by threads 0 .. slots - 1.  The shared-memory writes of every thread
// are made visible to the bulk copies (async-proxy fence, then a barrier).
// The copies run while the block sets up its next part; flush_wait (the
// issuing threads wait until their copies have read the window, then a
// barrier) must come before anything writes the window area again.
__device__ __forceinline__ void flush_issue(const DeliverSmem& S, uint32_t win_s, int slots, int npc,
                                            int32_t* acc, int tid) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid < slots) {
    const uint32_t bytes = (uint32_t)npc * 4u;
    const uint32_t src = win_s + (uint32_t)tid * bytes;
    int32_t* dst = acc + S.wbase[tid];
    asm volatile(
        "cp.reduce.async.bulk.global.shared::cta.bulk_group.add.s32 [%0], [%1], %2;\n\t"
        "cp.async.bulk.commit_group;" ::"l"(dst),
        "r"(src), "r"(bytes)
        : "memory");
  }
}
__device__ __forceinline__ void flush_wait(int tid, int slots) {
  if (tid < slots) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncthreads();
}

// Delivery block vb of vgrid (NT threads) for step t.  The step's items,
// ordered by (virtual column, delay bucket, spiker), are split into at most
// vgrid equal contiguous ranges of at least P.min_items items; block vb
// locates the first and last virtual column of its range from the group and
// column counts (gsum, isum) and walks the tiles it meets.  For each tile
// part it tabulates the (column, bucket) counts, builds the F16W neighbour
// table, lets its warps take batches of kBatchItems items, and flushes the
// tile's window.  Counts that disagree with the spike lists set the status
// word instead of being delivered.  `dyn` is the block's dynamic shared
// memory: table, neighbour table, window.
template <int PREC, int INFL, int NT>
__device__ __forceinline__ void deliver_body(const StepParams& P, long long t, int vb, int vgrid,
                                             DeliverSmem& S, unsigned char* dyn) {
  __syncthreads();  // the shared memory may still be read by a previous body
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  unsigned* const tab_w = reinterpret_cast<unsigned*>(dyn);  // windowed parts
  uint32_t* const nb_w = tab_w + tab_words(P, P.tile * P.tile);
  int32_t* const win = reinterpret_cast<int32_t*>(nb_w + nb_words<PREC>(P.tile * P.tile));
  unsigned* const tab_s = reinterpret_cast<unsigned*>(win);  // parts without window
  uint32_t* const nb_s_ = tab_s + tab_words(P, P.part_cols);
  // the slot that the next update fills holds step t - d_max: no longer read
  const long long next_slot = (t + 1) % P.nslot;
  if (vb == 0 && tid == 0) P.cnt[next_slot] = 0u;
  for (long long c = (long long)vb * NT + tid; c < P.ncol; c += (long long)vgrid * NT)
    P.ccnt[next_slot * P.ncol + c] = 0u;
  if (tid < kMaxDelays) {
    const int b = tid;
    const long long s = t + 1 - (P.dmin + b);
    S.slot[b] = (b < P.ndel && s >= 0) ? (int)(s % P.nslot) : -1;
  }
  if (tid == 0) {
    S.v0 = -1;
    S.v1 = -1;
    S.xg[0] = S.xg[1] = -1;
    S.next = 0u;
  }

  // the block's item range, from the group counts.  The ranges split the
  // step's cost evenly: a group of 32 virtual columns costs its items plus a
  // fixed part (P.cost_win when its items reach the window threshold -- the
  // set-up and flush of a windowed part -- else P.cost_part when it has
  // items), laid out before the group's items; a cost point maps to the item
  // position it falls on (the group's first item while in the fixed part).
  // The mapping is monotone, so consecutive blocks' ranges tile the items.
  const int ngrp = (P.ncol + 31) >> 5;
  const int per = (ngrp + NT - 1) / NT;
  const int g0 = tid * per;
  auto group_cost = [&](unsigned v) -> unsigned long long {
    return (unsigned long long)v + (v >= P.win_items ? P.cost_win : (v ? P.cost_part : 0u));
  };
  unsigned long long mine = 0ull, mcost = 0ull;
  for (int g = g0; g < g0 + per && g < ngrp; ++g) {
    const unsigned v = P.gsum[g];
    mine += v;
    mcost += group_cost(v);
  }
  unsigned long long total = 0ull, ctotal = 0ull;
  const unsigned long long excl = block_scan(mine, S, &total);
  const unsigned long long cexcl = block_scan(mcost, S, &ctotal);
  const unsigned long long want = (total + P.min_items - 1) / P.min_items;
  const int nact = (int)(want < (unsigned long long)vgrid ? (want ? want : 1ull) : (unsigned long long)vgrid);
  if (vb >= nact) return;
  for (int i = 0; i < 2; ++i) {
    const unsigned long long x = ctotal * (unsigned long long)(vb + i) / (unsigned long long)nact;
    if (x >= ctotal) {
      if (tid == 0) S.ipt[i] = total;
    } else if (x >= cexcl && x < cexcl + mcost) {
      unsigned long long rc = cexcl, ri = excl;
      for (int g = g0; g < g0 + per && g < ngrp; ++g) {
        const unsigned v = P.gsum[g];
        const unsigned long long c = group_cost(v);
        if (x < rc + c) {
          const unsigned long long fixed = c - v;
          S.ipt[i] = ri + (x - rc > fixed ? x - rc - fixed : 0ull);
          break;
        }
        rc += c;
        ri += v;
      }
    }
  }
  __syncthreads();
  const unsigned long long lo = S.ipt[0];
  const unsigned long long hi = S.ipt[1];
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
  // the virtual columns holding lo and hi - 1, from the column counts of their groups
  if (warp < 2 && S.xg[warp] >= 0) {
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
        S.v0 = c;
        S.p0 = pos;
      } else {
        S.v1 = c;
      }
    }
  }
  __syncthreads();
  const int v0 = S.v0, v1 = S.v1;
  if (v0 < 0 || v1 < v0) {
    if (tid == 0) set_status(P, kStatusCounts);
    return;
  }

  const uint64_t pol = evict_last_policy();
  const uint32_t win_s = (uint32_t)__cvta_generic_to_shared(win);
  unsigned long long pbase = S.p0;  // items before the tile part's first column
  unsigned long long covered = 0ull;  // items of the range found in the spike lists
  bool win_zero = false;              // the window has been cleared in this body
  int fl_slots = 0;                   // threads whose window flush may still read the window
  for (int v = v0; v <= v1;) {
    // the part's extent: one tile whose items in the range reach the window
    // threshold (delivered through the window), else a run of consecutive
    // tiles below it, at most P.part_cols columns (delivered without one)
    if (warp == 0) {
      int e = v, tiles = 0;
      bool wnd = false;
      unsigned long long pb = pbase;  // items before column e
      while (e <= v1) {
        const TileGeo gt = tile_geo(P, e);
        const int te = min(v1, gt.first + gt.tw * gt.th - 1);
        if (tiles > 0 && te - v + 1 > P.part_cols) break;
        unsigned x = 0u;
        for (int c = e + lane; c <= te; c += 32) x += P.isum[c];
        x = __reduce_add_sync(0xFFFFFFFFu, x);
        const unsigned long long lo_in = pb > lo ? pb : lo;
        const unsigned long long hi_in = pb + x < hi ? pb + x : hi;
        const unsigned long long in = hi_in > lo_in ? hi_in - lo_in : 0ull;
        if (P.agg && in >= P.win_items) {
          if (tiles == 0) {
            wnd = true;
            e = te + 1;
          }
          break;
        }
        pb += x;
        e = te + 1;
        ++tiles;
      }
      if (lane == 0) {
        S.pe = e;
        S.pwin = wnd ? 1 : 0;
      }
    }
    __syncthreads();
    const int ve = S.pe - 1;
    const bool windowed = S.pwin != 0;
    unsigned* const tab = windowed ? tab_w : tab_s;
    uint32_t* const nb = windowed ? nb_w : nb_s_;
    const uint32_t nb_s = (uint32_t)__cvta_generic_to_shared(nb);
    if (!windowed) win_zero = false;  // the tables overwrite the window area
    const TileGeo g = tile_geo(P, v);
    const int ncv = ve - v + 1;
    const int n_entries = ncv * P.ndel;
    for (int k = tid; k < ncv; k += NT) {
      const int c = (int)P.vcol[v + k];
      const int cy = c / P.W;
      S.ccol[k] = c;
      S.cx[k] = c - cy * P.W;
      S.cy[k] = cy;
    }
    __syncthreads();
    // tabulate the tile part: consecutive entries per thread
    constexpr int kEpt = (kMaxTileCols * kMaxDelays + NT - 1) / NT;
    const int ept = (n_entries + NT - 1) / NT;
    unsigned cnt[kEpt];
    unsigned sum = 0u;
#pragma unroll
    for (int q = 0; q < kEpt; ++q) {
      const int e = tid * ept + q;
      unsigned c = 0u;
      if (q < ept && e < n_entries) {
        const int k = e / P.ndel;
        const int sl = S.slot[e - k * P.ndel];
        c = sl >= 0 ? P.ccnt[(long long)sl * P.ncol + S.ccol[k]] : 0u;
        c = min(c, (unsigned)P.npc);  // a column lists at most n_per_col spikes
      }
      cnt[q] = c;
      sum += c;
    }
    unsigned long long ptotal = 0ull;
    unsigned run = (unsigned)block_scan(sum, S, &ptotal);
    if (!windowed && fl_slots) {  // this part's tables go into the window area
      flush_wait(tid, fl_slots);
      fl_slots = 0;
    }
#pragma unroll
    for (int q = 0; q < kEpt; ++q) {
      const int e = tid * ept + q;
      if (q < ept && e < n_entries) tab[e] = run;
      run += cnt[q];
    }
    if (tid == 0) tab[n_entries] = (unsigned)ptotal;
    // the block's items of this part; a part with few items skips the window
    // (clearing and flushing it would cost more than it saves)
    const unsigned a = lo > pbase ? (unsigned)(lo - pbase) : 0u;
    const unsigned b = hi > pbase ? (unsigned)min(hi - pbase, ptotal) : 0u;
    covered += b > a ? b - a : 0u;
    const WinGeo wg = win_geo(P, g, windowed);
    if (windowed && fl_slots) {
      flush_wait(tid, fl_slots);
      fl_slots = 0;
    }
    if (windowed && !win_zero) {
      for (int i = tid; i < (P.win_cap >> 2); i += NT) reinterpret_cast<int4*>(win)[i] = make_int4(0, 0, 0, 0);
      win_zero = true;
    }
    for (int m = tid; m < wg.ww * wg.wh; m += NT) {
      const int ry = m / wg.ww, rx = m - ry * wg.ww;
      int x = wg.x0 + rx, y = wg.y0 + ry;
      x -= x >= P.W ? P.W : 0;
      y -= y >= P.H ? P.H : 0;
      S.wbase[m] = ((uint32_t)y * (uint32_t)P.W + (uint32_t)x) * (uint32_t)P.npc;
    }
    if (PREC == SNN_EXACT_F16W && b > a) {
      // the column at each stencil offset of each column of the part: its
      // shared-window address, or bit 31 set and its first neuron in the
      // accumulator (offsets with dx + 3 = 7 belong to padding records)
      for (int m = tid; m < ncv * 64; m += NT) {
        const int k = m >> 6, off = m & 63;
        const int tx = wrap(S.cx[k] + (off & 7) - 3, P.W);
        const int ty = wrap(S.cy[k] + (off >> 3) - 3, P.H);
        int rx = tx - wg.x0;
        rx += rx < 0 ? P.W : 0;
        int ry = ty - wg.y0;
        ry += ry < 0 ? P.H : 0;
        nb[m] = (rx < wg.ww && ry < wg.wh)
                    ? win_s + 4u * (((uint32_t)ry * (uint32_t)wg.ww + (uint32_t)rx) * (uint32_t)P.npc)
                    : 0x80000000u | (((uint32_t)ty * (uint32_t)P.W + (uint32_t)tx) * (uint32_t)P.npc);
      }
    }
    __syncthreads();
    // the counts of each column must equal the items the range assumed
    if (tid < ncv && tab[(tid + 1) * P.ndel] - tab[tid * P.ndel] != P.isum[v + tid])
      set_status(P, kStatusCounts);
    // warps claim batches of kBatchItems items; a warp resolves its next
    // batch (descriptor loads) before it streams the current one
    if (a < b) {
      unsigned k0 = 0u;
      if (lane == 0) k0 = atomicAdd(&S.next, (unsigned)kBatchItems);
      k0 = a + __shfl_sync(0xFFFFFFFFu, k0, 0);
      Item cur = resolve_item<PREC>(P, k0 + lane, b, S, tab, n_entries, nb_s);
      while (k0 < b) {
        unsigned k1 = 0u;
        if (lane == 0) k1 = atomicAdd(&S.next, (unsigned)kBatchItems);
        k1 = a + __shfl_sync(0xFFFFFFFFu, k1, 0);
        const Item nxt = resolve_item<PREC>(P, k1 + lane, b, S, tab, n_entries, nb_s);
        stream_items<PREC, INFL>(P, cur, win_s, wg, pol);
        cur = nxt;
        k0 = k1;
      }
    }
    const uint32_t wlen = (uint32_t)(wg.ww * wg.wh) * (uint32_t)P.npc;
    __syncthreads();  // every warp is done with the part
    if ((P.npc & 3) == 0) {
      // bulk flush: each window slot (one column, n_per_col words, 16-byte
      // aligned in both memories) is added into the accumulator by one
      // asynchronous bulk reduction, which overlaps the next part's set-up;
      // the window is cleared again before a later part uses it
      if (windowed) {
        flush_issue(S, win_s, wg.ww * wg.wh, P.npc, P.acc, tid);
        fl_slots = wg.ww * wg.wh;
        win_zero = false;
      }
    } else {
      // flush the window with coalesced reductions, leaving it zeroed: word
      // m is neuron l of slot s; (s, l) advance with m
      uint32_t fs = div_by((uint32_t)tid, (uint32_t)P.npc, P.npc_m);
      uint32_t fl = (uint32_t)tid - fs * (uint32_t)P.npc;
      for (uint32_t m = tid; m < wlen; m += NT) {
        const int32_t x = win[m];
        if (x) {
          red_add(P.acc + S.wbase[fs] + fl, x, pol);
          win[m] = 0;
        }
        fl += NT;
        while (fl >= (uint32_t)P.npc) {
          fl -= (uint32_t)P.npc;
          ++fs;
        }
      }
    }
    if (tid == 0) S.next = 0u;
    pbase += ptotal;
    v = ve + 1;
    __syncthreads();
  }
  // the body's bulk reductions must have been performed (not only have read
  // the window) before it ends: the batch kernel's next phase reads the
  // accumulator after a grid barrier
  if (tid < (kMaxTile + 2) * (kMaxTile + 2)) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncthreads();
  // every item of the range must have been found in the spike lists
  if (tid == 0 && covered != hi - lo) set_status(P, kStatusCounts);
}

template <int PREC>
__global__ void __launch_bounds__(kDeliverThreads, 1) deliver_kernel(const StepParams P) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ DeliverSmem S;
  const long long t = P.ctl->t;
  deliver_body<PREC, PREC == SNN_EXACT_F16W ? kDepthF16 : kDepthF32, kDeliverThreads>(
      P, t, (int)blockIdx.x, (int)gridDim.x, S, s_dyn);

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
// Every step runs the update bodies of all nets (two 256-thread sub-blocks
// per block, each with its own named barrier), a grid barrier, the delivery
// bodies of all nets (whole blocks), and a second barrier.  Virtual body g of
// a phase belongs to net k with first[k] <= g < first[k + 1]; each virtual
// body is the standalone kernel's block body, so every net computes exactly
// what its own kernels compute.
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

// Net of virtual body g: the last k with first[k] <= g.
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
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(const BatchParams B) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  __shared__ StepParams s_p[kUpdateSubs];  // the nets of the current virtual bodies
  __shared__ DeliverSmem SD;
  __shared__ int s_uf[kMaxBatch + 1], s_df[kMaxBatch + 1];
  __shared__ unsigned s_ok;
  UpdateSmem* SU = reinterpret_cast<UpdateSmem*>(s_dyn);  // one per sub-block
  const int sub = threadIdx.x / kUpdateThreads;
  const int stid = threadIdx.x - sub * kUpdateThreads;
  const int n = B.n_nets;
  for (int k = threadIdx.x; k <= n; k += blockDim.x) {
    s_uf[k] = B.u_first[k];
    s_df[k] = B.d_first[k];
  }
  __syncthreads();
  const int total_u = s_uf[n], total_d = s_df[n];
  constexpr int kParamWords = (int)(sizeof(StepParams) / 4);
  for (long long step = 0; step < B.n_steps; ++step) {
    const long long t = B.t0 + step;
    for (int g = blockIdx.x * kUpdateSubs + sub; g < total_u; g += gridDim.x * kUpdateSubs) {
      const int k = net_of(s_uf, n, g);
      body_sync(1 + sub);
      for (int w = stid; w < kParamWords; w += kUpdateThreads)
        reinterpret_cast<uint32_t*>(&s_p[sub])[w] = reinterpret_cast<const uint32_t*>(B.nets + k)[w];
      body_sync(1 + sub);
      update_body<false>(s_p[sub], t, g - s_uf[k], s_uf[k + 1] - s_uf[k], SU[sub], stid, 1 + sub);
    }
    if (!grid_barrier(B, &s_ok)) return;
    for (int g = blockIdx.x; g < total_d; g += gridDim.x) {
      const int k = net_of(s_df, n, g);
      __syncthreads();
      for (int w = threadIdx.x; w < kParamWords; w += blockDim.x)
        reinterpret_cast<uint32_t*>(&s_p[0])[w] = reinterpret_cast<const uint32_t*>(B.nets + k)[w];
      __syncthreads();
      deliver_body<PREC, INFL, kBatchThreads>(s_p[0], t, g - s_df[k], s_df[k + 1] - s_df[k], SD,
                                              s_dyn);
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

// Shard: the received spikes of step t (global indices ids[0 .. n)) that
// belong to halo columns join the step's per-column lists as the update
// kernel's own spikes do -- a descriptor {local index, bucket ends} at the
// next position of the column's list and, with d_min = 1, one more item for
// the column in this step's delivery (with d_min >= 2 the update kernel of
// step t + d_min - 1 moves the column's count in).  Indices of the shard's
// own columns and of columns outside its local grid are skipped.  An index
// beyond the global network, or more than n_per_col spikes for one column
// (a duplicated index), is skipped and sets the status word.
__global__ void __launch_bounds__(256) ingest_kernel(const StepParams P, const uint32_t* ids,
                                                     long long n) {
  const long long t = P.ctl->t;
  const long long slot = t % P.nslot;
  const unsigned long long ng = (unsigned long long)P.sg.GW * (unsigned long long)P.sg.GH *
                                (unsigned long long)P.npc;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    const uint32_t g = ids[k];
    if ((unsigned long long)g >= ng) {
      set_status(P, kStatusIngest);
      continue;
    }
    const uint32_t gc = g / (uint32_t)P.npc;
    const uint32_t l = g - gc * (uint32_t)P.npc;
    const int gy = (int)(gc / (uint32_t)P.sg.GW), gx = (int)gc - gy * P.sg.GW;
    const int lx = wrap(gx - P.sg.ex0, P.sg.GW), ly = wrap(gy - P.sg.ey0, P.sg.GH);
    if (lx >= P.W || ly >= P.H) continue;  // not in the local grid
    if (lx >= P.sg.tx0 && lx < P.sg.tx0 + P.sg.tw && ly >= P.sg.ty0 && ly < P.sg.ty0 + P.sg.th)
      continue;  // an own column: listed by the update kernel
    const int c = ly * P.W + lx;
    const unsigned r = atomicAdd(P.ccnt + slot * P.ncol + c, 1u);
    if (r >= (unsigned)P.npc) {
      set_status(P, kStatusIngest);
      continue;
    }
    const uint32_t id = (uint32_t)c * (uint32_t)P.npc + l;
    uint4* d = reinterpret_cast<uint4*>(
        P.desc + ((long long)slot * P.N + (long long)c * P.npc + r) * P.desc_words);
    const uint4* be = reinterpret_cast<const uint4*>(P.bend + (long long)id * kBendStride);
    const uint4 a = be[0], b = be[1];
    d[0] = make_uint4(id, a.x, a.y, a.z);
    d[1] = make_uint4(a.w, b.x, b.y, b.z);
    if (P.desc_words == 16) d[2] = make_uint4(b.w, 0u, 0u, 0u);
    if (P.dmin == 1) {
      const unsigned v = P.colv[c];
      atomicAdd(P.isum + v, 1u);
      atomicAdd(P.gsum + (v >> 5), 1u);
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
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, update_kernel<false>, kUpdateThreads, 0);
  if (per_sm < 1) per_sm = 1;
  const long long tiles = ((N + 3) / 4 + kUpdateThreads - 1) / kUpdateThreads;
  const long long g = (long long)per_sm * num_sms;
  return (int)(tiles < g ? tiles : g);
}

cudaError_t launch_update(const StepParams& p, int grid, cudaStream_t st) {
  if (p.sg.on)
    update_kernel<true><<<grid, kUpdateThreads, 0, st>>>(p);
  else
    update_kernel<false><<<grid, kUpdateThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_ingest(const StepParams& p, const uint32_t* ids, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long blocks = (n + 255) / 256;
  ingest_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0, st>>>(p, ids, n);
  return cudaGetLastError();
}

size_t deliver_smem(const StepParams& p, int precision) {
  auto tables = [&](size_t cols) {
    const size_t tabw = (cols * (size_t)p.ndel + 1 + 3) & ~(size_t)3;
    return tabw + (precision == SNN_EXACT_F16W ? cols * 64 : 0);
  };
  // windowed-part tables, then the window area (which also holds the tables
  // of a part without window)
  const size_t area = std::max((size_t)p.win_cap, tables((size_t)p.part_cols));
  return (tables((size_t)p.tile * p.tile) + area) * 4;
}

int deliver_threads() { return kDeliverThreads; }

// Delivery grid: one block per SM (a persistent grid).
int deliver_grid(const StepParams& p, int precision, int num_sms) {
  const size_t smem = deliver_smem(p, precision);
  int per_sm = 0;
  if (precision == SNN_EXACT_F16W) {
    if (cudaFuncSetAttribute(deliver_kernel<SNN_EXACT_F16W>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_kernel<SNN_EXACT_F16W>,
                                                  kDeliverThreads, smem);
  } else {
    if (cudaFuncSetAttribute(deliver_kernel<SNN_EXACT_F32W>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_kernel<SNN_EXACT_F32W>,
                                                  kDeliverThreads, smem);
  }
  return per_sm * num_sms;
}

cudaError_t launch_deliver(const StepParams& p, int precision, int grid, cudaStream_t st) {
  const size_t smem = deliver_smem(p, precision);
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
// The batch tuner's schedule `infl` (2 or 4) selects 1 or 2 rounds of
// sectors in flight per lane.
void* batch_kernel_ptr(int precision, int infl) {
  if (precision == SNN_EXACT_F16W) return infl == 2 ? batch_fn<1, 1>() : batch_fn<1, 2>();
  return infl == 2 ? batch_fn<0, 1>() : batch_fn<0, 2>();
}
}  // namespace

size_t batch_smem(size_t max_deliver_smem) {
  const size_t upd = kUpdateSubs * sizeof(UpdateSmem);
  return upd > max_deliver_smem ? upd : max_deliver_smem;
}

int batch_grid(int precision, int infl, int num_sms, size_t smem) {
  void* fn = batch_kernel_ptr(precision, infl);
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, smem);
  return per_sm * num_sms;
}

cudaError_t launch_batch(const BatchParams& b, int precision, int infl, int grid, size_t smem,
                         cudaStream_t st) {
  void* args[] = {const_cast<BatchParams*>(&b)};
  return cudaLaunchCooperativeKernel(batch_kernel_ptr(precision, infl), dim3(grid),
                                     dim3(kBatchThreads), args, smem, st);
}

cudaError_t launch_sum_parts(const unsigned long long* part, int n, unsigned long long* out,
                             cudaStream_t st) {
  sum_parts_kernel<<<1, 32, 0, st>>>(part, n, out);
  return cudaGetLastError();
}

}  // namespace snn
