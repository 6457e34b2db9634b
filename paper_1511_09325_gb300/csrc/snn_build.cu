// snn_build.cu -- on-device construction of the delay-bucketed synapse table.
//
// Connectivity of arxiv 1511.09325, Sec. 2, as read by this library: synapse
// k of neuron j (column (x, y), index l_j in it) draws one Philox4x32-10 block
// (counter (j, k, CONN, 0)) = (x0, x1, x2, x3):
//   k <  k_local : target in the own column, l = u_{n-1}(x0), skipping l_j;
//   k >= k_local : stencil offset = first m with x1 < thr[m] (P ~ exp(-r/lambda)),
//                  target l = u_n(x0) in column ((x+dx) mod W, (y+dy) mod H);
//   delay d = d_min + u_ndel(x2);  weight = table[population][x3 >> 16].
// F16W records keep the target as a stencil code and the weight's magnitude as
// a half; F32W records keep the target's neuron index and the FP32 weight
// already scaled to the input's fixed-point units, round(w * 2^16).
// One warp owns one row: a first pass counts the synapses of every delay
// bucket, a second pass regenerates them and stores each into its bucket in
// k order (warp match + popc rank), then the bucket tails are padded.
// A shard (see ShardGeo) draws every synapse with the neuron's global index
// and keeps only those whose target column is one of its own; an F32W record
// then holds the target's local index (local and global stencil arithmetic
// agree for such targets: the halo is as wide as the stencil, or the local
// grid spans the whole global side).
#include "snn_device.cuh"
#include "snn_internal.h"

namespace snn {
namespace {

constexpr int kBuildWarps = 8;

template <int PREC>
__global__ void __launch_bounds__(kBuildWarps * 32)
    build_rows_kernel(const BuildParams P) {
  __shared__ unsigned s_cnt[kBuildWarps][32];
  __shared__ unsigned s_cur[kBuildWarps][32];
  __shared__ uint32_t s_thr[kMaxOff];
  __shared__ int s_code[kMaxOff];
  __shared__ int s_dx[kMaxOff], s_dy[kMaxOff];
  for (int m = threadIdx.x; m < kMaxOff; m += blockDim.x) {
    s_thr[m] = P.stencil_thr[m];
    s_code[m] = m < P.n_off ? ((P.off_dy[m] + 3) << 3) | (P.off_dx[m] + 3) : kCenterCode;
    s_dx[m] = m < P.n_off ? P.off_dx[m] : 0;
    s_dy[m] = m < P.n_off ? P.off_dy[m] : 0;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * kBuildWarps;
  const uint32_t ndel = (uint32_t)P.ndel;

  for (long long j = (long long)blockIdx.x * kBuildWarps + w; j < P.N; j += nwarps) {
    const int col = (int)((uint32_t)j / (uint32_t)P.npc);
    const int lj = (int)(j - (long long)col * P.npc);
    const int cy = col / P.W, cx = col - cy * P.W;
    int gx, gy;
    shard_global_col(P.sg, cx, cy, &gx, &gy);
    const uint32_t jj = P.sg.on ? ((uint32_t)gy * (uint32_t)P.sg.GW + (uint32_t)gx) * (uint32_t)P.npc + (uint32_t)lj
                                : (uint32_t)j;
    const bool src_own = shard_owns_global(P.sg, P.W, P.H, gx, gy);
    // whether synapse k (Philox block x) ends in one of the shard's columns
    auto kept = [&](int k, const uint4& x) -> bool {
      if (!P.sg.on) return true;
      if (k < P.k_local) return src_own;
      int m = 0;
      for (int i = 0; i + 1 < P.n_off; ++i) m += (x.y >= s_thr[i]) ? 1 : 0;
      return shard_owns_global(P.sg, P.W, P.H, wrap(gx + s_dx[m], P.sg.GW), wrap(gy + s_dy[m], P.sg.GH));
    };
    s_cnt[w][lane] = 0u;
    __syncwarp();
    // pass 1: synapses per delay bucket
    unsigned nkept = 0u;
    for (int k = lane; k < P.K; k += 32) {
      const uint4 x = philox4x32_10(make_uint4(jj, (uint32_t)k, kTagConn, 0u), P.seed_lo, P.seed_hi);
      if (kept(k, x)) {
        atomicAdd(&s_cnt[w][below(x.z, ndel)], 1u);
        ++nkept;
      }
    }
    if (P.deg != nullptr) {
      nkept = __reduce_add_sync(0xFFFFFFFFu, nkept);
      if (lane == 0) P.deg[j] = nkept;
    }
    __syncwarp();
    const unsigned units = lane < P.ndel ? (s_cnt[w][lane] + (kSlotUnit - 1)) / kSlotUnit : 0u;
    unsigned incl = units;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += v;
    }
    P.bend[j * kBendStride + lane] = (uint8_t)(lane < P.ndel ? incl : 0u);
    s_cur[w][lane] = (incl - units) * kSlotUnit;
    __syncwarp();

    const long long row = j * (long long)P.rowcap;
    const uint32_t* wt = P.wtab + (lj < P.nexc ? 0 : 65536);
    // pass 2: regenerate and place every synapse
    for (int k0 = 0; k0 < P.K; k0 += 32) {
      const int k = k0 + lane;
      const uint4 x = philox4x32_10(make_uint4(jj, (uint32_t)k, kTagConn, 0u), P.seed_lo, P.seed_hi);
      const bool valid = k < P.K && kept(k, x);
      const int b = valid ? (int)below(x.z, ndel) : 63;
      uint32_t code;  // F16W: stencil code; F32W: target neuron index
      if (k < P.k_local) {
        uint32_t l = below(x.x, (uint32_t)(P.npc - 1));
        l += (l >= (uint32_t)lj) ? 1u : 0u;
        code = PREC == SNN_EXACT_F16W ? ((uint32_t)kCenterCode << 11) | l
                                      : (uint32_t)col * (uint32_t)P.npc + l;
      } else {
        int m = 0;
        for (int i = 0; i + 1 < P.n_off; ++i) m += (x.y >= s_thr[i]) ? 1 : 0;
        const uint32_t l = below(x.x, (uint32_t)P.npc);
        if (PREC == SNN_EXACT_F16W) {
          code = ((uint32_t)s_code[m] << 11) | l;
        } else {
          const int ty = wrap(cy + s_dy[m], P.H);
          const int tx = wrap(cx + s_dx[m], P.W);
          code = ((uint32_t)ty * (uint32_t)P.W + (uint32_t)tx) * (uint32_t)P.npc + l;
        }
      }
      const uint32_t wbits = wt[x.w >> 16];
      const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
      const unsigned rank = __popc(peers & ((1u << lane) - 1u));
      const unsigned pos = s_cur[w][b & 31] + rank;
      __syncwarp();
      if (valid) {
        if (PREC == SNN_EXACT_F16W) {
          static_cast<uint32_t*>(P.syn)[row + pos] = ((wbits & 0x7FFFu) << 17) | code;
        } else {
          // the FP32 weight, delivered as round(w * 2^16) in the input's units
          const int32_t wfx = __float2int_rn(__fmul_rn(__uint_as_float(wbits), 65536.0f));
          static_cast<uint2*>(P.syn)[row + pos] = make_uint2(code, (uint32_t)wfx);
        }
        if (rank == 0) s_cur[w][b] += __popc(peers);
      }
      __syncwarp();
    }
    // pad every bucket up to its 8-slot boundary
    if (lane < P.ndel) {
      const unsigned end = incl * kSlotUnit;
      for (unsigned s = s_cur[w][lane]; s < end; ++s) {
        if (PREC == SNN_EXACT_F16W)
          static_cast<uint32_t*>(P.syn)[row + s] = kPadF16;
        else
          static_cast<uint2*>(P.syn)[row + s] = make_uint2(kPad, 0u);
      }
    }
    __syncwarp();
  }
}

// Initial state: V_i uniform in [0, theta) at 24-bit resolution from word
// i mod 4 of Philox(i / 4, 0, INIT); calcium, refractoriness and input zero.
// A shard draws with the global index i (n_per_col is a multiple of 4 there,
// so a quad of local neurons is a quad of global ones).
__global__ void __launch_bounds__(256) init_state_kernel(const StepParams P) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long i0 = q * 4;
  if (i0 >= P.N) return;
  uint32_t gq = (uint32_t)q;
  if (P.sg.on) {
    const int col = (int)((uint32_t)i0 / (uint32_t)P.npc);
    const int l = (int)((uint32_t)i0 - (uint32_t)col * (uint32_t)P.npc);
    const int cy = col / P.W;
    int gx, gy;
    shard_global_col(P.sg, col - cy * P.W, cy, &gx, &gy);
    gq = (((uint32_t)gy * (uint32_t)P.sg.GW + (uint32_t)gx) * (uint32_t)P.npc + (uint32_t)l) >> 2;
  }
  const uint4 u = philox4x32_10(make_uint4(gq, 0u, kTagInit, 0u), P.seed_lo, P.seed_hi);
  const float s = 5.9604644775390625e-08f;  // 2^-24
  float4 v;
  v.x = __fmul_rn(P.theta, __fmul_rn(__uint2float_rn(u.x >> 8), s));
  v.y = __fmul_rn(P.theta, __fmul_rn(__uint2float_rn(u.y >> 8), s));
  v.z = __fmul_rn(P.theta, __fmul_rn(__uint2float_rn(u.z >> 8), s));
  v.w = __fmul_rn(P.theta, __fmul_rn(__uint2float_rn(u.w >> 8), s));
  reinterpret_cast<float4*>(P.V)[q] = v;
  reinterpret_cast<float4*>(P.C)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  reinterpret_cast<int4*>(P.acc)[q] = make_int4(0, 0, 0, 0);
  reinterpret_cast<uchar4*>(P.R)[q] = make_uchar4(0, 0, 0, 0);
}

// Paper connectivity law (Sec. 2): candidate c of neuron j -- the column's
// other neurons in ascending order, then the n_per_col neurons of each kept
// remote offset -- is kept iff word c mod 4 of Philox(j, c / 4, PCONN) is
// below its threshold.  The k-th kept candidate is synapse k, whose delay and
// weight come from Philox(j, k, CONN) as under the fixed law.  One warp per
// row; in pass it, lane e takes candidates 128 it + 4 e .. + 3, so a warp
// scan of the lanes' kept counts ranks them.  The count pass (FILL false)
// writes the bucket ends, the out-degree and the largest row; the fill pass
// makes the same draws and places every synapse (warp match + popc rank, as
// in build_rows_kernel), then pads the buckets.
template <int PREC, bool FILL>
__global__ void __launch_bounds__(kBuildWarps * 32) paper_rows_kernel(const BuildParams P) {
  __shared__ unsigned s_cnt[kBuildWarps][32];
  __shared__ unsigned s_cur[kBuildWarps][32];
  __shared__ unsigned long long s_thr[kMaxOff];
  __shared__ int s_dx[kMaxOff], s_dy[kMaxOff];
  for (int m = threadIdx.x; m < kMaxOff; m += blockDim.x) {
    s_thr[m] = m < P.n_poff ? P.poff_thr[m] : 0ull;
    s_dx[m] = m < P.n_poff ? P.poff_dx[m] : 0;
    s_dy[m] = m < P.n_poff ? P.poff_dy[m] : 0;
  }
  __syncthreads();
  const int w = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * kBuildWarps;
  const uint32_t ndel = (uint32_t)P.ndel;
  const unsigned lt_mask = (1u << lane) - 1u;

  for (long long j = (long long)blockIdx.x * kBuildWarps + w; j < P.N; j += nwarps) {
    const uint32_t jj = (uint32_t)j;
    const int col = (int)((uint32_t)j / (uint32_t)P.npc);
    const int lj = (int)(j - (long long)col * P.npc);
    const int cy = col / P.W, cx = col - cy * P.W;
    const uint32_t* wt = P.wtab + (lj < P.nexc ? 0 : 65536);
    const long long row = j * (long long)P.rowcap;
    if (FILL)
      s_cur[w][lane] = lane < P.ndel ? (lane ? (unsigned)P.bend[j * kBendStride + lane - 1] : 0u) * kSlotUnit : 0u;
    else
      s_cnt[w][lane] = 0u;
    __syncwarp();
    unsigned k_run = 0u;
    for (long long c0 = 0; c0 < P.n_cand; c0 += 128) {
      const long long cb = c0 + 4 * lane;
      const uint4 x = philox4x32_10(make_uint4(jj, (uint32_t)(cb >> 2), kTagPConn, 0u), P.seed_lo,
                                    P.seed_hi);
      const uint32_t words[4] = {x.x, x.y, x.z, x.w};
      unsigned bits = 0u;
      int lq[4], mq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long c = cb + q;
        lq[q] = 0;
        mq[q] = -1;
        if (c >= P.n_cand) continue;
        unsigned long long thr;
        if (c < P.npc - 1) {
          thr = P.plocal_thr;
          lq[q] = (int)c + ((int)c >= lj ? 1 : 0);
        } else {
          const long long r = c - (P.npc - 1);
          const int m = (int)((uint32_t)r / (uint32_t)P.npc);
          thr = s_thr[m];
          mq[q] = m;
          lq[q] = (int)(r - (long long)m * P.npc);
        }
        if ((unsigned long long)words[q] < thr) bits |= 1u << q;
      }
      const unsigned nb = (unsigned)__popc(bits);
      unsigned incl = nb;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
      }
      const unsigned kb = k_run + incl - nb;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool keep = (bits >> q) & 1u;
        int b = 63;
        uint32_t code = 0u, wbits = 0u;
        if (keep) {
          const unsigned k = kb + (unsigned)__popc(bits & ((1u << q) - 1u));
          const uint4 y = philox4x32_10(make_uint4(jj, k, kTagConn, 0u), P.seed_lo, P.seed_hi);
          b = (int)below(y.z, ndel);
          if (FILL) wbits = wt[y.w >> 16];
          const int m = mq[q];
          const int dx = m < 0 ? 0 : s_dx[m], dy = m < 0 ? 0 : s_dy[m];
          if (PREC == SNN_EXACT_F16W) {
            code = ((uint32_t)(((dy + 3) << 3) | (dx + 3)) << 11) | (uint32_t)lq[q];
          } else {
            const int ty = wrap(cy + dy, P.H), tx = wrap(cx + dx, P.W);
            code = ((uint32_t)ty * (uint32_t)P.W + (uint32_t)tx) * (uint32_t)P.npc + (uint32_t)lq[q];
          }
        }
        if (!FILL) {
          if (keep) atomicAdd(&s_cnt[w][b], 1u);
        } else {
          const unsigned peers = __match_any_sync(0xFFFFFFFFu, b);
          const unsigned rank = __popc(peers & lt_mask);
          const unsigned pos = s_cur[w][b & 31] + rank;
          __syncwarp();
          if (keep) {
            if (PREC == SNN_EXACT_F16W) {
              static_cast<uint32_t*>(P.syn)[row + pos] = ((wbits & 0x7FFFu) << 17) | code;
            } else {
              const int32_t wfx = __float2int_rn(__fmul_rn(__uint_as_float(wbits), 65536.0f));
              static_cast<uint2*>(P.syn)[row + pos] = make_uint2(code, (uint32_t)wfx);
            }
            if (rank == 0) s_cur[w][b] += __popc(peers);
          }
          __syncwarp();
        }
      }
      k_run += __shfl_sync(0xFFFFFFFFu, incl, 31);
    }
    __syncwarp();
    if (!FILL) {
      const unsigned units = lane < P.ndel ? (s_cnt[w][lane] + (kSlotUnit - 1)) / kSlotUnit : 0u;
      unsigned incl = units;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
      }
      P.bend[j * kBendStride + lane] = (uint8_t)(lane < P.ndel ? (incl < 255u ? incl : 255u) : 0u);
      if (lane == 31) atomicMax(P.max_units, incl);
      if (lane == 0) P.deg[j] = k_run;
    } else if (lane < P.ndel) {
      const unsigned end = (unsigned)P.bend[j * kBendStride + lane] * kSlotUnit;
      for (unsigned s = s_cur[w][lane]; s < end; ++s) {
        if (PREC == SNN_EXACT_F16W)
          static_cast<uint32_t*>(P.syn)[row + s] = kPadF16;
        else
          static_cast<uint2*>(P.syn)[row + s] = make_uint2(kPad, 0u);
      }
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_paper_count(const BuildParams& bp, int num_sms, cudaStream_t st) {
  paper_rows_kernel<SNN_EXACT_F32W, false><<<num_sms * 8, kBuildWarps * 32, 0, st>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_paper_fill(const BuildParams& bp, int precision, int num_sms,
                              cudaStream_t st) {
  if (precision == SNN_EXACT_F16W)
    paper_rows_kernel<SNN_EXACT_F16W, true><<<num_sms * 8, kBuildWarps * 32, 0, st>>>(bp);
  else
    paper_rows_kernel<SNN_EXACT_F32W, true><<<num_sms * 8, kBuildWarps * 32, 0, st>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_build(const BuildParams& bp, int precision, int num_sms,
                         cudaStream_t st) {
  const int grid = num_sms * 8;
  if (precision == SNN_EXACT_F16W)
    build_rows_kernel<SNN_EXACT_F16W><<<grid, kBuildWarps * 32, 0, st>>>(bp);
  else
    build_rows_kernel<SNN_EXACT_F32W><<<grid, kBuildWarps * 32, 0, st>>>(bp);
  return cudaGetLastError();
}

cudaError_t launch_init_state(const StepParams& p, cudaStream_t st) {
  const long long quads = (p.N + 3) / 4;
  const unsigned grid = (unsigned)((quads + 255) / 256);
  init_state_kernel<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace snn
