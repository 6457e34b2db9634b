// snn_step.cu -- the two kernels of one 1 ms step.
//
// update_kernel (neuron update, arxiv 1511.09325 Sec. 2 LIF + SFA):
//   one thread owns 4 consecutive neurons and one Philox4x32-10 block
//   (counter (i/4, t, EXT, 0)) whose 4 words give their external Poisson
//   counts; it reads and clears their recurrent input, applies refractoriness,
//   threshold, reset and the exact propagator with explicitly rounded FP32
//   operations, and appends the spikes to the step's list (block-aggregated,
//   one global atomic per block), the spike records and the column counters.
//
// deliver_kernel (event-driven delivery, Sec. 1): "pull by delay".  The input
//   of step t+1 is the sum, over delays d, of bucket d of every neuron that
//   spiked at step t+1-d.  A persistent grid walks the virtual work list of
//   (delay bucket, spiker) items of the last d_max steps' spike lists; one warp
//   streams an item's bucket (a run of 32 B sectors) with coalesced loads and
//   adds each weight into acc with a fire-and-forget int32 reduction, so the
//   sum is exact and independent of the order.  Only the N-entry accumulator
//   of the next step receives atomics (it stays resident in L2), instead of a
//   d_max-slot ring.  The last block to finish advances the step counter.
#include "snn_device.cuh"
#include "snn_internal.h"

namespace snn {
namespace {

constexpr int kUpdateThreads = 256;
constexpr int kDeliverThreads = 256;

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

__device__ __forceinline__ int poisson_count(uint32_t x, const uint8_t* guide,
                                             const uint32_t* thr, int n) {
  int k = guide[x >> 24];
  while (k < n && x >= thr[k]) ++k;
  return k;
}

__global__ void __launch_bounds__(kUpdateThreads) update_kernel(const StepParams P) {
  __shared__ uint32_t s_ids[kUpdateThreads * 4];
  __shared__ uint32_t s_thr[kMaxPoisThr + 1];
  __shared__ uint8_t s_guide[256];
  __shared__ unsigned s_n, s_base;
  __shared__ unsigned long long s_k;

  const long long t = P.ctl->t;
  const int slot = (int)(t % P.nslot);
  for (int m = threadIdx.x; m < 256; m += blockDim.x) s_guide[m] = P.pois_guide[m];
  for (int m = threadIdx.x; m <= kMaxPoisThr; m += blockDim.x) s_thr[m] = P.pois_thr[m];
  if (threadIdx.x == 0) {
    s_n = 0u;
    s_k = 0ull;
  }
  __syncthreads();

  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long i0 = q * 4;
  unsigned ksum = 0u;
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
    int l = (int)(i0 % P.npc);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = poisson_count(xin[e], s_guide, s_thr, P.n_pois_thr);
      const int32_t I = ain[e] + k * P.jx;
      const NeuronOut o = neuron_step(vin[e], cin[e], rin[e], I, l < P.nexc ? P.pvc_e : P.pvc_i, P);
      vout[e] = o.v;
      cout[e] = o.c;
      rout[e] = o.r;
      if (i0 + e < P.N) {
        ksum += (unsigned)k;
        if (o.spike) s_ids[atomicAdd(&s_n, 1u)] = (uint32_t)(i0 + e);
      }
      l = (l + 1 == P.npc) ? 0 : l + 1;
    }
    reinterpret_cast<float4*>(P.V)[q] = make_float4(vout[0], vout[1], vout[2], vout[3]);
    reinterpret_cast<float4*>(P.C)[q] = make_float4(cout[0], cout[1], cout[2], cout[3]);
    reinterpret_cast<uchar4*>(P.R)[q] = make_uchar4((unsigned char)rout[0], (unsigned char)rout[1],
                                                    (unsigned char)rout[2], (unsigned char)rout[3]);
  }
  // external events: warp sum, then one shared atomic per warp
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, o);
  if ((threadIdx.x & 31) == 0 && ksum) atomicAdd(&s_k, (unsigned long long)ksum);
  __syncthreads();
  const unsigned n = s_n;
  if (threadIdx.x == 0) {
    if (n) s_base = atomicAdd(&P.ctl->count[slot], n);
    if (s_k) atomicAdd(&P.ctl->ext_events, s_k);
  }
  __syncthreads();
  if (n == 0u) return;
  const unsigned base = s_base;
  const unsigned long long rbase = P.ctl->rec_count + base;
  uint32_t* list = P.ids + (long long)slot * P.N;
  for (unsigned e = threadIdx.x; e < n; e += blockDim.x) {
    const uint32_t id = s_ids[e];
    list[base + e] = id;
    const unsigned long long ri = rbase + e;
    if ((long long)ri < P.rec_cap)
      P.rec[ri] = ((unsigned long long)(unsigned)t << 32) | id;
    else
      P.ctl->rec_overflow = 1u;
    const int col = (int)(id / (unsigned)P.npc);
    const int pop = (int)(id - (unsigned)col * (unsigned)P.npc) < P.nexc ? 0 : 1;
    atomicAdd(&P.colcnt[2 * col + pop], 1ull);
  }
}

template <int PREC>
__global__ void __launch_bounds__(kDeliverThreads) deliver_kernel(const StepParams P) {
  __shared__ unsigned s_pref[kMaxDelays + 1];
  __shared__ long long s_list[kMaxDelays];
  const long long t = P.ctl->t;
  if (threadIdx.x < 32) {
    const int b = threadIdx.x;
    unsigned cnt = 0u;
    long long off = 0;
    if (b < P.ndel) {
      const long long s = t + 1 - (P.dmin + b);
      if (s >= 0) {
        const int slot = (int)(s % P.nslot);
        cnt = P.ctl->count[slot];
        off = (long long)slot * P.N;
      }
    }
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (b >= o) incl += v;
    }
    s_pref[b + 1] = incl;
    if (b == 0) s_pref[0] = 0u;
    s_list[b] = off;
  }
  __syncthreads();

  const unsigned total = s_pref[P.ndel];
  const int lane = threadIdx.x & 31;
  const unsigned warps = gridDim.x * (kDeliverThreads / 32);
  for (unsigned item = blockIdx.x * (kDeliverThreads / 32) + (threadIdx.x >> 5); item < total;
       item += warps) {
    int b = 0;
    while (item >= s_pref[b + 1]) ++b;
    const uint32_t j = P.ids[s_list[b] + (item - s_pref[b])];
    const uint8_t* be = P.bend + (long long)j * kBendStride;
    const int beg = (b ? (int)be[b - 1] : 0) * kSlotUnit;
    const int end = (int)be[b] * kSlotUnit;
    const int col = (int)(j / (uint32_t)P.npc);
    const int lj = (int)(j - (uint32_t)col * (uint32_t)P.npc);
    const int cy = col / P.W;
    const int cx = col - cy * P.W;
    const float wscale = lj < P.nexc ? 65536.0f : -65536.0f;
    // lanes 0..6 hold the first column index of target row dy - 3,
    // lanes 8..14 the column offset of target column dx - 3
    int tab = 0;
    if (lane < 7)
      tab = wrap(cy + lane - 3, P.H) * P.W;
    else if (lane >= 8 && lane < 15)
      tab = wrap(cx + lane - 11, P.W);
    const long long row = (long long)j * P.rowcap;
    for (int p0 = beg; p0 < end; p0 += 32) {
      const int p = p0 + lane;
      const bool in = p < end;
      uint32_t code;
      float w;
      if (PREC == SNN_EXACT_F16W) {
        const uint32_t rec = in ? __ldcs(static_cast<const uint32_t*>(P.syn) + row + p) : kPad;
        code = rec == kPad ? kPad : (rec & 0x1FFFFu);
        w = __half2float(__ushort_as_half((unsigned short)(rec >> 17)));
      } else {
        const uint2 rec = in ? __ldcs(static_cast<const uint2*>(P.syn) + row + p) : make_uint2(kPad, 0u);
        code = rec.x;
        w = __uint_as_float(rec.y);
      }
      const int ry = __shfl_sync(0xFFFFFFFFu, tab, (code >> 14) & 7u);
      const int rx = __shfl_sync(0xFFFFFFFFu, tab, 8 + ((code >> 11) & 7u));
      if (code != kPad) {
        const int tgt = (ry + rx) * P.npc + (int)(code & 0x7FFu);
        const int32_t wfx = PREC == SNN_EXACT_F16W ? __float2int_rn(__fmul_rn(w, wscale))
                                                   : __float2int_rn(__fmul_rn(w, 65536.0f));
        atomicAdd(P.acc + tgt, wfx);
      }
    }
  }

  // the last block to finish closes the step
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&P.ctl->done, 1u);
    if (prev == gridDim.x - 1) {
      __threadfence();
      Ctl* c = P.ctl;
      const int slot = (int)(t % P.nslot);
      const unsigned n = *((volatile unsigned*)&c->count[slot]);
      c->rec_count += n;
      c->spikes += n;
      c->count[(int)((t + 1) % P.nslot)] = 0u;
      c->done = 0u;
      c->t = t + 1;
    }
  }
}

}  // namespace

cudaError_t launch_update(const StepParams& p, cudaStream_t st) {
  const long long quads = (p.N + 3) / 4;
  const unsigned grid = (unsigned)((quads + kUpdateThreads - 1) / kUpdateThreads);
  update_kernel<<<grid, kUpdateThreads, 0, st>>>(p);
  return cudaGetLastError();
}

int deliver_grid(int precision, int num_sms) {
  int per_sm = 0;
  if (precision == SNN_EXACT_F16W)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_kernel<SNN_EXACT_F16W>,
                                                  kDeliverThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, deliver_kernel<SNN_EXACT_F32W>,
                                                  kDeliverThreads, 0);
  if (per_sm < 1) per_sm = 1;
  return per_sm * num_sms;
}

cudaError_t launch_deliver(const StepParams& p, int precision, int grid, cudaStream_t st) {
  if (precision == SNN_EXACT_F16W)
    deliver_kernel<SNN_EXACT_F16W><<<grid, kDeliverThreads, 0, st>>>(p);
  else
    deliver_kernel<SNN_EXACT_F32W><<<grid, kDeliverThreads, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace snn
