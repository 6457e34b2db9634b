// snn_step.cu -- the two kernels of one 1 ms step.
//
// update_kernel (neuron update, arxiv 1511.09325 Sec. 2 LIF + SFA):
//   grid-stride over tiles of 1024 neurons; one thread owns 4 consecutive
//   neurons and one Philox4x32-10 block (counter (i/4, t, EXT, 0)) whose 4
//   words give their external Poisson counts.  It reads and clears their
//   recurrent input, applies refractoriness, threshold, reset and the exact
//   propagator with explicitly rounded FP32 operations.  Spikes are ranked per
//   (tile, column) in shared memory and appended to the per-column spike list
//   of the step with one global atomic per column and tile; the spike records
//   are buffered per block and appended with one atomic per flush.
//
// deliver_kernel (event-driven delivery, Sec. 1), "pull by delay": the input
//   of step t+1 is the sum over delays d of bucket d of every neuron that
//   spiked at step t+1-d, so only one N-entry accumulator (resident in L2)
//   receives additions, not a d_max-slot ring.  One block owns one source
//   column: it walks the (delay bucket, spiker) items of that column over the
//   last d_max steps in batches of 32 per warp, streams the concatenated
//   buckets in 16-byte chunks, adds the local half of the synapses (targets in
//   the same column) into a shared-memory copy of the column's accumulator,
//   and sends the remote half to L2 as fire-and-forget int32 reductions.  The
//   shared accumulator is flushed with coalesced reductions at the end.
//   Integer addition makes the result independent of the order.  The last
//   block to finish advances the step counter.
#include "snn_device.cuh"
#include "snn_internal.h"

namespace snn {
namespace {

constexpr int kUpdateThreads = 256;
constexpr int kDeliverThreads = 256;
constexpr int kTile = kUpdateThreads * 4;    // neurons per update tile
constexpr int kRecBuf = 3 * kTile;           // block-local spike-record buffer
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

// Fire-and-forget int32 reduction into the accumulator, with an L2
// evict-last hint: the accumulator is re-read by the next step's update.
__device__ __forceinline__ void red_add(int32_t* p, int32_t v) {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  asm volatile("red.global.add.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol)
               : "memory");
}

// Append the block's buffered records (step << 32 | id).
__device__ __forceinline__ void flush_records(const StepParams& P, long long t, uint32_t* s_rec,
                                              unsigned* s_fill, unsigned long long* s_rbase) {
  const unsigned n = *s_fill;  // block-uniform (read after a barrier)
  if (n == 0u) return;
  if (threadIdx.x == 0) {
    *s_rbase = atomicAdd(&P.ctl->rec_count, (unsigned long long)n);
    atomicAdd(&P.ctl->spikes, (unsigned long long)n);
  }
  __syncthreads();
  const unsigned long long rbase = *s_rbase;
  for (unsigned e = threadIdx.x; e < n; e += blockDim.x) {
    const unsigned long long ri = rbase + e;
    if ((long long)ri < P.rec_cap)
      P.rec[ri] = ((unsigned long long)(unsigned)t << 32) | s_rec[e];
    else
      P.ctl->rec_overflow = 1u;
  }
  __syncthreads();
  if (threadIdx.x == 0) *s_fill = 0u;
  __syncthreads();
}

// Grid-stride over tiles; the grid size is fixed per net, so block b owns
// ext_part[b].
__global__ void __launch_bounds__(kUpdateThreads) update_kernel(const StepParams P) {
  __shared__ uint32_t s_rec[kRecBuf];
  __shared__ uint32_t s_thr[kMaxPoisThr + 1];
  __shared__ uint8_t s_guide[256];
  __shared__ unsigned s_tcnt[kTileCols];     // spikes per column of the tile
  __shared__ unsigned s_tbase[kTileCols];    // their offsets in the column lists
  __shared__ unsigned s_tpop[kTileCols][2];  // E / I spikes per column
  __shared__ unsigned s_fill;
  __shared__ unsigned long long s_rbase;
  __shared__ unsigned s_ksum[kUpdateThreads / 32];

  const long long t = P.ctl->t;
  const int slot = (int)(t % P.nslot);
  for (int m = threadIdx.x; m < 256; m += blockDim.x) s_guide[m] = P.pois_guide[m];
  for (int m = threadIdx.x; m <= kMaxPoisThr; m += blockDim.x) s_thr[m] = P.pois_thr[m];
  if (threadIdx.x == 0) s_fill = 0u;
  unsigned ksum = 0u;
  const long long quads = (P.N + 3) / 4;
  const long long tiles = (quads + kUpdateThreads - 1) / kUpdateThreads;
  unsigned* cnt = P.cnt + (long long)slot * P.ncol;
  uint32_t* ids = P.ids + (long long)slot * P.N;

  for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const long long first = tile * kTile;
    const long long last = (first + kTile < P.N ? first + kTile : P.N) - 1;
    const int col0 = (int)(first / P.npc);
    const int ncols = (int)(last / P.npc) - col0 + 1;
    for (int k = threadIdx.x; k < ncols; k += blockDim.x) {
      s_tcnt[k] = 0u;
      s_tpop[k][0] = 0u;
      s_tpop[k][1] = 0u;
    }
    __syncthreads();

    const long long q = tile * kUpdateThreads + threadIdx.x;
    const long long i0 = q * 4;
    unsigned spk_rank[4] = {0u, 0u, 0u, 0u};
    int spk_col[4] = {0, 0, 0, 0};
    bool spk[4] = {false, false, false, false};
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
      int col = (int)(i0 / P.npc);
      int l = (int)(i0 - (long long)col * P.npc);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int k = poisson_count(xin[e], s_guide, s_thr, P.n_pois_thr);
        const int32_t I = ain[e] + k * P.jx;
        const bool exc = l < P.nexc;
        const NeuronOut o = neuron_step(vin[e], cin[e], rin[e], I, exc ? P.pvc_e : P.pvc_i, P);
        vout[e] = o.v;
        cout[e] = o.c;
        rout[e] = o.r;
        spk_col[e] = col;
        if (i0 + e < P.N) {
          ksum += (unsigned)k;
          if (o.spike) {
            spk[e] = true;
            spk_rank[e] = atomicAdd(&s_tcnt[col - col0], 1u);
            atomicAdd(&s_tpop[col - col0][exc ? 0 : 1], 1u);
            s_rec[atomicAdd(&s_fill, 1u)] = (uint32_t)(i0 + e);
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
    // one reservation per column of the tile in that column's spike list
    for (int k = threadIdx.x; k < ncols; k += blockDim.x) {
      const unsigned n = s_tcnt[k];
      if (n) {
        s_tbase[k] = atomicAdd(&cnt[col0 + k], n);
        if (s_tpop[k][0]) atomicAdd(&P.colcnt[2 * (col0 + k)], (unsigned long long)s_tpop[k][0]);
        if (s_tpop[k][1]) atomicAdd(&P.colcnt[2 * (col0 + k) + 1], (unsigned long long)s_tpop[k][1]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (spk[e])
        ids[(long long)spk_col[e] * P.npc + s_tbase[spk_col[e] - col0] + spk_rank[e]] =
            (uint32_t)(i0 + e);
    if (s_fill > (unsigned)(kRecBuf - kTile)) flush_records(P, t, s_rec, &s_fill, &s_rbase);
  }
  __syncthreads();
  flush_records(P, t, s_rec, &s_fill, &s_rbase);

  // external events: per-block partial sum, no atomics
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, o);
  if ((threadIdx.x & 31) == 0) s_ksum[threadIdx.x >> 5] = ksum;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long tot = 0ull;
    for (int w = 0; w < kUpdateThreads / 32; ++w) tot += s_ksum[w];
    P.ext_part[blockIdx.x] += tot;
  }
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

// Per-warp staging of one batch of 32 delivery items.
struct WarpBatch {
  int pre[33];         // exclusive prefix of the items' slot counts
  long long base[32];  // table slot of the item's first synapse, minus pre[e]
  float wscale[32];    // +-2^16: fixed-point scale with the source's sign
};

template <int PREC>
__device__ __forceinline__ void deliver_record(uint32_t code, uint32_t wbits, float wscale,
                                               int cx, int cy, int32_t* s_acc,
                                               const StepParams& P) {
  if (code == kPad) return;
  float w;
  if (PREC == SNN_EXACT_F16W)
    w = __fmul_rn(__half2float(__ushort_as_half((unsigned short)wbits)), wscale);
  else
    w = __fmul_rn(__uint_as_float(wbits), 65536.0f);
  const int32_t wfx = __float2int_rn(w);
  const int l = (int)(code & 0x7FFu);
  const uint32_t off = (code >> 11) & 63u;
  if (off == (uint32_t)kCenterCode) {
    atomicAdd(s_acc + l, wfx);
  } else {
    const int ty = wrap_near(cy + (int)(off >> 3) - 3, P.H);
    const int tx = wrap_near(cx + (int)(off & 7u) - 3, P.W);
    red_add(P.acc + (ty * P.W + tx) * P.npc + l, wfx);
  }
}

template <int PREC>
__global__ void __launch_bounds__(kDeliverThreads) deliver_kernel(const StepParams P) {
  constexpr int kWarps = kDeliverThreads / 32;
  __shared__ int32_t s_acc[2048];
  __shared__ unsigned s_pref[kMaxDelays + 1];
  __shared__ long long s_list[kMaxDelays];
  __shared__ unsigned s_next;
  __shared__ WarpBatch s_wb[kWarps];

  const long long t = P.ctl->t;
  const int c = (int)(blockIdx.x / (unsigned)P.split);
  const int part = (int)(blockIdx.x - (unsigned)c * (unsigned)P.split);
  const int cy = c / P.W;
  const int cx = c - cy * P.W;
  for (int l = threadIdx.x; l < P.npc; l += blockDim.x) s_acc[l] = 0;
  if (threadIdx.x < 32) {
    const int b = threadIdx.x;
    unsigned n = 0u;
    long long off = 0;
    if (b < P.ndel) {
      const long long s = t + 1 - (P.dmin + b);
      if (s >= 0) {
        const int slot = (int)(s % P.nslot);
        n = P.cnt[(long long)slot * P.ncol + c];
        off = (long long)slot * P.N + (long long)c * P.npc;
      }
    }
    unsigned incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (b >= o) incl += v;
    }
    s_pref[b + 1] = incl;
    if (b == 0) {
      s_pref[0] = 0u;
      s_next = 0u;
    }
    s_list[b] = off;
  }
  __syncthreads();

  const unsigned total = s_pref[P.ndel];
  const unsigned lo = (unsigned)(((unsigned long long)total * part) / P.split);
  const unsigned hi = (unsigned)(((unsigned long long)total * (part + 1)) / P.split);
  const int lane = threadIdx.x & 31;
  WarpBatch& wb = s_wb[threadIdx.x >> 5];

  while (true) {
    unsigned k0 = 0u;
    if (lane == 0) k0 = atomicAdd(&s_next, 32u);
    k0 = __shfl_sync(0xFFFFFFFFu, k0, 0);
    if (lo + k0 >= hi) break;
    // phase A: lane e resolves item e of the batch
    const unsigned item = lo + k0 + lane;
    int len = 0;
    if (item < hi) {
      int b = 0;
      while (item >= s_pref[b + 1]) ++b;
      const uint32_t j = P.ids[s_list[b] + (item - s_pref[b])];
      const uint8_t* be = P.bend + (long long)j * kBendStride;
      const int beg = (b ? (int)be[b - 1] : 0) * kSlotUnit;
      const int end = (int)be[b] * kSlotUnit;
      len = end - beg;
      wb.base[lane] = (long long)j * P.rowcap + beg;
      wb.wscale[lane] = (int)(j - (uint32_t)c * (uint32_t)P.npc) < P.nexc ? 65536.0f : -65536.0f;
    }
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    wb.pre[lane + 1] = incl;
    if (lane == 0) wb.pre[0] = 0;
    if (item < hi) wb.base[lane] -= incl - len;
    __syncwarp();
    const int T = wb.pre[32];

    // phase B: stream the concatenated buckets, 4 slots per lane per chunk,
    // two chunks in flight
    for (int f0 = 0; f0 < T; f0 += 256) {
      int e[2];
      uint32_t code[2][4], wbits[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int f = f0 + u * 128 + lane * 4;
        e[u] = -1;
        if (f < T) {
          int x = 0;
#pragma unroll
          for (int st = 16; st >= 1; st >>= 1)
            if (wb.pre[x + st] <= f) x += st;
          e[u] = x;
          const long long slot = wb.base[x] + f;
          if (PREC == SNN_EXACT_F16W) {
            const uint4 r = __ldcs(reinterpret_cast<const uint4*>(static_cast<const uint32_t*>(P.syn) + slot));
            const uint32_t rr[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
            for (int qd = 0; qd < 4; ++qd) {
              code[u][qd] = rr[qd] == kPad ? kPad : (rr[qd] & 0x1FFFFu);
              wbits[u][qd] = rr[qd] >> 17;
            }
          } else {
            const uint4* p4 = reinterpret_cast<const uint4*>(static_cast<const uint2*>(P.syn) + slot);
            const uint4 r0 = __ldcs(p4);
            const uint4 r1 = __ldcs(p4 + 1);
            code[u][0] = r0.x; wbits[u][0] = r0.y;
            code[u][1] = r0.z; wbits[u][1] = r0.w;
            code[u][2] = r1.x; wbits[u][2] = r1.y;
            code[u][3] = r1.z; wbits[u][3] = r1.w;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (e[u] >= 0) {
          const float ws = wb.wscale[e[u]];
#pragma unroll
          for (int qd = 0; qd < 4; ++qd)
            deliver_record<PREC>(code[u][qd], wbits[u][qd], ws, cx, cy, s_acc, P);
        }
      }
    }
    __syncwarp();
  }

  // flush the column's shared accumulator with coalesced reductions
  __syncthreads();
  int32_t* dst = P.acc + (long long)c * P.npc;
  for (int l = threadIdx.x; l < P.npc; l += blockDim.x) {
    const int32_t v = s_acc[l];
    if (v) red_add(dst + l, v);
  }
  // this column's count of the slot that the next update overwrites
  const int next_slot = (int)((t + 1) % P.nslot);
  if (P.split == 1 && threadIdx.x == 0) P.cnt[(long long)next_slot * P.ncol + c] = 0u;

  // the last block to finish closes the step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&P.ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      if (P.split > 1)
        for (int k = 0; k < P.ncol; ++k) P.cnt[(long long)next_slot * P.ncol + k] = 0u;
      P.ctl->done = 0u;
      P.ctl->t = t + 1;
    }
  }
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

// Blocks per source column: enough blocks for 4 per SM on small grids.
int deliver_split(long long ncol, int num_sms) {
  const long long target = 4LL * num_sms;
  long long s = (target + ncol - 1) / ncol;
  if (s < 1) s = 1;
  if (s > 64) s = 64;
  return (int)s;
}

cudaError_t launch_deliver(const StepParams& p, int precision, cudaStream_t st) {
  const unsigned grid = (unsigned)(p.ncol * p.split);
  if (precision == SNN_EXACT_F16W)
    deliver_kernel<SNN_EXACT_F16W><<<grid, kDeliverThreads, 0, st>>>(p);
  else
    deliver_kernel<SNN_EXACT_F32W><<<grid, kDeliverThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace snn
