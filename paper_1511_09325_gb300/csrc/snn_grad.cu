// snn_grad.cu -- a differentiable form of the network of arxiv 1511.09325,
// Sec. 2, and its reverse-mode gradient.
//
// The paper simulates the spiking network only.  This file adds the standard
// surrogate-gradient treatment of the same recursion, on the same synapse
// table (F32W records: target index, fixed-point weight):
//
//   X_E,i(t), X_I,i(t): sums of w s_j(t - d) over excitatory / inhibitory sources
//   I_i = a[E][p_i] X_E,i + a[I][p_i] X_I,i + J (lam + sqrt(lam) xi_i(t))
//   g_i = max(0, 1 - s_i(t-1) - s_i(t-2));  U_i = g (V_i + I_i) + (1 - g) V_reset
//   s_i = [U_i >= theta] (hard) or sigmoid(beta (U_i - theta)) (soft)
//   V' = U - s (U - V_reset);  c' = c + dc s
//   V(t+1) = P_VV V' + P_VC c';  c(t+1) = P_CC c',  P_VC,E = g_c kappa
//
// with xi_i(t) the normal draw of Philox stream SURR (quantile table of the
// top 16 bits), lam = nu_ext h, and the loss (r_E - r_E*)^2 + (r_I - r_I*)^2
// on the population rates.  In hard mode the backward pass uses the
// surrogate derivative ds/dU = 1 / (1 + beta |U - theta|)^2; in soft mode the
// exact one.  Parameters: a_EE, a_EI, a_IE, a_II (a_XY scales the synapses
// from X onto Y), g_c and nu_ext.
//
// Forward: grad_deliver_kernel (one warp per source row, pull by delay: the
// input of step t is every bucket d of every row weighted by s_j(t - d), summed
// as int64 fixed point in 2^-32 mV, so the sums do not depend on the order;
// rows whose last d_max spikes are all zero leave after one load)
// and grad_update_kernel (one thread per neuron; hard mode is the spiking
// model's arithmetic, one float rounding per operation).  The state (V, c and
// the spike history of d_max + 1 steps) is checkpointed every `ckpt` steps.
// Backward: segment by segment from the end, the forward is recomputed from
// the segment's checkpoint while a tape of eight values per neuron and step is
// recorded, then the adjoint recursion runs back through the segment:
// grad_gather_kernel (one warp per source row: the adjoint of the delayed
// delivery is a gather over the row's outgoing synapses of the targets' input
// adjoints at t + d, in a fixed order) and grad_backward_kernel (one thread per
// neuron: the adjoint of every line above; parameter partials accumulate per
// neuron in FP64 and are summed on the host in a fixed order).  Every sum has a
// fixed order, so a run is reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "snn_device.cuh"
#include "snn_internal.h"

using namespace snn;

namespace {

constexpr int kThreads = 256;
constexpr int kTape = 8;  // V, I, U, g, s, c', X_E, X_I
constexpr float kTwoM32 = 2.3283064365386963e-10f;  // 2^-32
constexpr float kTwoM16 = 1.52587890625e-05f;       // 2^-16
constexpr float kTwoM24 = 5.9604644775390625e-08f;  // 2^-24

struct GradParams {
  long long N;
  int npc, nexc, dmin, ndel, nslot, rowcap, hard, T;
  uint32_t seed_lo, seed_hi;
  float beta, theta, vr, dc, pvv, pcc, pvc_e, pvc_i, kappa, J, lam, sqlam;
  float a[4];  // a_EE, a_EI, a_IE, a_II
  float dlds_e, dlds_i;
  const uint2* syn;
  const uint8_t* bend;
  const float* q;
  float* V;
  float* C;
  float* shist;               // [nslot][N] s of the last nslot steps
  unsigned long long* xe;     // [N] input sums from E sources, 2^-32 mV
  unsigned long long* xin;    // [N] the same from I sources
  float* tape;                // [ckpt][kTape][N]
  double* rate_part;          // [update blocks][2]
  float* vbar;
  float* cbar;
  float* ibe;                 // [nslot][N] a[E][p_i] * adjoint of I_i(t)
  float* ibi;                 // [nslot][N] a[I][p_i] * adjoint of I_i(t)
  float* gb;                  // [3][N] -adjoint of g_i(t) where the gate is open
  float* sg;                  // [N] gathered adjoint of s_j(t) through its synapses
  double* gacc;               // [6][N] parameter partials per neuron
};

// Ring position of step s >= 0 (steps are below 2^31: 32-bit remainder).
__device__ __forceinline__ long long ring(long long s, int n) {
  return (long long)((uint32_t)s % (uint32_t)n);
}

__device__ __forceinline__ float normal_draw(const GradParams& P, long long i, long long t) {
  const uint4 x = philox4x32_10(make_uint4((uint32_t)(i >> 2), (uint32_t)t, kTagSurr, 0u),
                                P.seed_lo, P.seed_hi);
  const uint32_t w = (i & 3) == 0 ? x.x : (i & 3) == 1 ? x.y : (i & 3) == 2 ? x.z : x.w;
  return P.q[w >> 16];
}

// Initial state: V_i uniform in [0, theta) from the spiking net's INIT
// stream (word i mod 4 of Philox(i / 4, 0, INIT)), c = 0.
__global__ void __launch_bounds__(kThreads) grad_init_kernel(const GradParams P) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const uint4 x = philox4x32_10(make_uint4((uint32_t)(i >> 2), 0u, kTagInit, 0u), P.seed_lo,
                                P.seed_hi);
  const uint32_t u = (i & 3) == 0 ? x.x : (i & 3) == 1 ? x.y : (i & 3) == 2 ? x.z : x.w;
  P.V[i] = __fmul_rn(P.theta, __fmul_rn(__uint2float_rn(u >> 8), kTwoM24));
  P.C[i] = 0.f;
}

// Bucket ends (slots) in lanes 0..ndel-1 of the warp; the bucket holding
// slot k is the first b with end_b > k, found by a fixed five-step search
// over the lanes (every lane takes part, whatever its k).
__device__ __forceinline__ int bucket_of(int k, int end_lane, int ndel) {
  int lo = 0, hi = ndel - 1;
#pragma unroll
  for (int step = 0; step < 5; ++step) {
    const int mid = (lo + hi) >> 1;
    const int e = __shfl_sync(0xFFFFFFFFu, end_lane, mid);
    if (e > k)
      hi = mid;
    else
      lo = min(mid + 1, hi);
  }
  return lo;
}

// Input of step t: every bucket d of every source row j, weighted by
// s_j(t - d), into the row's population accumulator.  One warp per row: the
// lanes first load the row's ndel spike values at once and the warp leaves
// when all are zero; otherwise it streams the row four records per lane
// (16-byte loads; a bucket is a whole number of 8-slot units, so the four
// records of a lane share a bucket).
__global__ void __launch_bounds__(kThreads) grad_deliver_kernel(const GradParams P, long long t) {
  const long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= P.N) return;
  float s_lane = 0.f;
  int end_lane = 0x7FFFFFFF;
  if (lane < P.ndel) {
    const long long src = t - (P.dmin + lane);
    s_lane = src >= 0 ? P.shist[ring(src, P.nslot) * P.N + j] : 0.f;
    end_lane = (int)P.bend[j * kBendStride + lane] * kSlotUnit;
  }
  if (__ballot_sync(0xFFFFFFFFu, s_lane != 0.f) == 0u) return;
  const bool exc = (int)((uint32_t)j % (uint32_t)P.npc) < P.nexc;
  unsigned long long* acc = exc ? P.xe : P.xin;
  const int row_end = __shfl_sync(0xFFFFFFFFu, end_lane, P.ndel - 1);
  const uint2* row = P.syn + j * (long long)P.rowcap;
  for (int k0 = 0; k0 < row_end; k0 += 128) {
    const int k = k0 + 4 * lane;
    const int b = bucket_of(k, end_lane, P.ndel);
    const float s = __shfl_sync(0xFFFFFFFFu, s_lane, b);
    if (k < row_end && s != 0.f) {
      const uint4 r01 = __ldcs(reinterpret_cast<const uint4*>(row + k));
      const uint4 r23 = __ldcs(reinterpret_cast<const uint4*>(row + k + 2));
      const uint32_t tg[4] = {r01.x, r01.z, r23.x, r23.z};
      const uint32_t wf[4] = {r01.y, r01.w, r23.y, r23.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (tg[q] == kPad) continue;
        const int32_t wfx = (int32_t)wf[q];
        const long long v = P.hard ? (long long)wfx * 65536ll
                                   : __float2ll_rn(__fmul_rn(__fmul_rn(s, (float)wfx), 65536.f));
        atomicAdd(acc + tg[q], (unsigned long long)v);
      }
    }
  }
}

// Neuron update of step t; records the tape at slot `slot` (>= 0) and adds
// the spikes of each population to this block's rate partial sums when
// `rates` is set.
__global__ void __launch_bounds__(kThreads) grad_update_kernel(const GradParams P, long long t,
                                                              int slot, int rates) {
  __shared__ float s_sum[kThreads / 32][2];
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float s = 0.f;
  bool exc = false;
  if (i < P.N) {
    const float XE = __fmul_rn(__ll2float_rn((long long)P.xe[i]), kTwoM32);
    const float XI = __fmul_rn(__ll2float_rn((long long)P.xin[i]), kTwoM32);
    P.xe[i] = 0ull;
    P.xin[i] = 0ull;
    exc = (int)((uint32_t)i % (uint32_t)P.npc) < P.nexc;
    const float xi = normal_draw(P, i, t);
    const float e = __fmul_rn(P.J, __fadd_rn(P.lam, __fmul_rn(P.sqlam, xi)));
    const float aE = exc ? P.a[0] : P.a[1];
    const float aI = exc ? P.a[2] : P.a[3];
    const float I = __fadd_rn(__fadd_rn(__fmul_rn(aE, XE), __fmul_rn(aI, XI)), e);
    const float s1 = t >= 1 ? P.shist[ring(t - 1, P.nslot) * P.N + i] : 0.f;
    const float s2 = t >= 2 ? P.shist[ring(t - 2, P.nslot) * P.N + i] : 0.f;
    const float V = P.V[i], c = P.C[i];
    float g, U, Vp, cp;
    if (P.hard) {
      g = (s1 == 0.f && s2 == 0.f) ? 1.f : 0.f;
      U = g != 0.f ? __fadd_rn(V, I) : P.vr;
      s = U >= P.theta ? 1.f : 0.f;
      Vp = s != 0.f ? P.vr : U;
      cp = s != 0.f ? __fadd_rn(c, P.dc) : c;
    } else {
      g = fmaxf(__fsub_rn(__fsub_rn(1.f, s1), s2), 0.f);
      U = __fadd_rn(__fmul_rn(g, __fadd_rn(V, I)), __fmul_rn(__fsub_rn(1.f, g), P.vr));
      const float z = __fmul_rn(P.beta, __fsub_rn(U, P.theta));
      const float ez = expf(-fabsf(z));
      s = z >= 0.f ? 1.f / (1.f + ez) : ez / (1.f + ez);
      Vp = __fsub_rn(U, __fmul_rn(s, __fsub_rn(U, P.vr)));
      cp = __fadd_rn(c, __fmul_rn(P.dc, s));
    }
    const float pvc = exc ? P.pvc_e : P.pvc_i;
    P.V[i] = __fmaf_rn(cp, pvc, __fmul_rn(Vp, P.pvv));
    P.C[i] = __fmul_rn(cp, P.pcc);
    P.shist[ring(t, P.nslot) * P.N + i] = s;
    if (slot >= 0) {
      float* tp = P.tape + (long long)slot * kTape * P.N + i;
      const float vals[kTape] = {V, I, U, g, s, cp, XE, XI};
#pragma unroll
      for (int k = 0; k < kTape; ++k) tp[(long long)k * P.N] = vals[k];
    }
  }
  if (!rates) return;
  // this block's spikes per population, in a fixed order
  float se = exc ? s : 0.f, si = (i < P.N && !exc) ? s : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    se += __shfl_xor_sync(0xFFFFFFFFu, se, o);
    si += __shfl_xor_sync(0xFFFFFFFFu, si, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s_sum[threadIdx.x >> 5][0] = se;
    s_sum[threadIdx.x >> 5][1] = si;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double te = 0.0, ti = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      te += (double)s_sum[w][0];
      ti += (double)s_sum[w][1];
    }
    P.rate_part[2 * blockIdx.x] += te;
    P.rate_part[2 * blockIdx.x + 1] += ti;
  }
}

// Adjoint of s_j(tau) through its outgoing synapses: sum over buckets d with
// tau + d < T of w * (a[p_j][p_i] * adjoint of I_i(tau + d)).  One warp per
// row, four records per lane per pass (16-byte loads), a fixed summation
// order.
__global__ void __launch_bounds__(kThreads) grad_gather_kernel(const GradParams P, long long tau) {
  const long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= P.N) return;
  const bool exc = (int)((uint32_t)j % (uint32_t)P.npc) < P.nexc;
  const float* ib = exc ? P.ibe : P.ibi;
  long long off_lane = -1;  // ring offset of bucket `lane`'s step, -1 beyond T
  int end_lane = 0x7FFFFFFF;
  if (lane < P.ndel) {
    const long long dst = tau + P.dmin + lane;
    off_lane = dst < P.T ? ring(dst, P.nslot) * P.N : -1;
    end_lane = (int)P.bend[j * kBendStride + lane] * kSlotUnit;
  }
  const int row_end = __shfl_sync(0xFFFFFFFFu, end_lane, P.ndel - 1);
  const uint2* row = P.syn + j * (long long)P.rowcap;
  float acc = 0.f;
#pragma unroll 2
  for (int k0 = 0; k0 < row_end; k0 += 128) {
    const int k = k0 + 4 * lane;
    const int b = bucket_of(k, end_lane, P.ndel);
    const long long off = __shfl_sync(0xFFFFFFFFu, off_lane, b);
    if (k < row_end && off >= 0) {
      const uint4 r01 = __ldcs(reinterpret_cast<const uint4*>(row + k));
      const uint4 r23 = __ldcs(reinterpret_cast<const uint4*>(row + k + 2));
      const float* ibs = ib + off;
      const uint32_t tg[4] = {r01.x, r01.z, r23.x, r23.z};
      const uint32_t wf[4] = {r01.y, r01.w, r23.y, r23.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (tg[q] != kPad) acc = __fmaf_rn((float)(int32_t)wf[q], ibs[tg[q]], acc);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if (lane == 0) P.sg[j] = __fmul_rn(acc, kTwoM16);
}

// One step of the adjoint recursion for step tau (tape slot `slot`): takes the
// adjoints of V(tau+1), c(tau+1) and leaves those of V(tau), c(tau).
__global__ void __launch_bounds__(kThreads) grad_backward_kernel(const GradParams P, long long tau,
                                                                int slot) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.N) return;
  const bool exc = (int)((uint32_t)i % (uint32_t)P.npc) < P.nexc;
  const float* tp = P.tape + (long long)slot * kTape * P.N + i;
  const float V = tp[0], I = tp[P.N], U = tp[2 * P.N], g = tp[3 * P.N], s = tp[4 * P.N];
  const float cp = tp[5 * P.N], XE = tp[6 * P.N], XI = tp[7 * P.N];
  float sbar = (exc ? P.dlds_e : P.dlds_i) + P.sg[i] + P.gb[ring(tau + 1, 3) * P.N + i] +
               P.gb[ring(tau + 2, 3) * P.N + i];
  const float vb1 = P.vbar[i], cb1 = P.cbar[i];
  const float pvc = exc ? P.pvc_e : P.pvc_i;
  // V(tau+1) = P_VV V' + P_VC c',  c(tau+1) = P_CC c'
  const float vpbar = P.pvv * vb1;
  const float cpbar = P.pcc * cb1 + pvc * vb1;
  double* ga = P.gacc + i;
  if (exc) ga[4 * P.N] += (double)vb1 * (double)cp * (double)P.kappa;
  // V' = U - s (U - V_reset),  c' = c + dc s
  float ubar = vpbar * (1.f - s);
  sbar += -vpbar * (U - P.vr) + cpbar * P.dc;
  // the spike nonlinearity: surrogate (hard) or exact (soft) derivative
  float dsdu;
  if (P.hard) {
    const float den = 1.f + P.beta * fabsf(U - P.theta);
    dsdu = 1.f / (den * den);
  } else {
    dsdu = P.beta * s * (1.f - s);
  }
  ubar += sbar * dsdu;
  // U = g (V + I) + (1 - g) V_reset
  const float ib = ubar * g;
  P.vbar[i] = ib;
  P.cbar[i] = cpbar;
  P.gb[ring(tau, 3) * P.N + i] = g > 0.f ? -ubar * (V + I - P.vr) : 0.f;
  const float aE = exc ? P.a[0] : P.a[1];
  const float aI = exc ? P.a[2] : P.a[3];
  P.ibe[ring(tau, P.nslot) * P.N + i] = aE * ib;
  P.ibi[ring(tau, P.nslot) * P.N + i] = aI * ib;
  // I = a[E][p] X_E + a[I][p] X_I + J (lam + sqrt(lam) xi),  h = 1 ms
  ga[(exc ? 0 : 1) * P.N] += (double)ib * (double)XE;
  ga[(exc ? 2 : 3) * P.N] += (double)ib * (double)XI;
  const float xi = normal_draw(P, i, tau);
  ga[5 * P.N] += (double)ib * (double)P.J * (1.0 + (double)xi / (2.0 * (double)P.sqlam));
}

}  // namespace

struct snn_grad {
  NetView v{};
  long long T = 0;
  int ckpt = 0, nseg = 0, hard = 1, nslot = 0, ublocks = 0, wblocks = 0;
  float beta = 5.f;
  double targets[2] = {3.0, 8.0};
  double kappa = 0.0, pvv = 0.0, pcc = 0.0;
  GradParams P{};
  float* q = nullptr;
  float* ck = nullptr;  // [nseg][(2 + nslot) N]: V, c, s history at each segment start
  std::vector<void*> bufs;
  std::string err;
};

namespace {

int gfail(snn_grad* g, int code, const std::string& msg) {
  if (g) g->err = msg;
  return code == SNN_OK ? code : fail_global(code, msg);
}

#define SNN_GCUDA(g, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return gfail((g), e_ == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA,       \
                   std::string(#call ": ") + cudaGetErrorString(e_));                   \
  } while (0)

template <class T>
int galloc(snn_grad* g, T** p, size_t count) {
  void* d = nullptr;
  const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 256;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return gfail(g, e == cudaErrorMemoryAllocation ? SNN_ENOMEM : SNN_ECUDA,
                 "cudaMalloc of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  g->bufs.push_back(d);
  *p = static_cast<T*>(d);
  return SNN_OK;
}

void grad_release(snn_grad* g) {
  for (void* p : g->bufs) cudaFree(p);
  g->bufs.clear();
}

cudaError_t launch_forward_step(snn_grad* g, long long t, int slot, int rates) {
  const GradParams& P = g->P;
  cudaStream_t st = g->v.stream;
  grad_deliver_kernel<<<g->wblocks, kThreads, 0, st>>>(P, t);
  grad_update_kernel<<<g->ublocks, kThreads, 0, st>>>(P, t, slot, rates);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int snn_grad_build(snn_net* net, int64_t n_steps, int32_t checkpoint_every, int32_t hard,
                   float beta, const double* target_rates, snn_grad** out) {
  if (!out) return fail_global(SNN_EINVAL, "out is NULL");
  *out = nullptr;
  NetView v{};
  if (!net || net_view(net, &v) != SNN_OK)
    return fail_global(SNN_EINVAL, "net is NULL or a shard");
  if (v.precision != SNN_EXACT_F32W)
    return fail_global(SNN_EINVAL, "the differentiable form needs an SNN_EXACT_F32W net");
  if (n_steps < 1 || n_steps > (1LL << 31)) return fail_global(SNN_EINVAL, "n_steps must be >= 1");
  if (checkpoint_every < 1) return fail_global(SNN_EINVAL, "checkpoint_every must be >= 1");
  if (!(beta > 0.f) || !std::isfinite(beta)) return fail_global(SNN_EINVAL, "beta must be > 0");
  if (v.neuron.tau_c == v.neuron.tau_m)
    return fail_global(SNN_EINVAL, "tau_c must differ from tau_m");
  snn_grad* g = new (std::nothrow) snn_grad();
  if (!g) return fail_global(SNN_ENOMEM, "host allocation failed");
  g->v = v;
  g->T = n_steps;
  g->ckpt = (int)std::min<long long>(checkpoint_every, n_steps);
  g->nseg = (int)((n_steps + g->ckpt - 1) / g->ckpt);
  g->hard = hard ? 1 : 0;
  g->beta = beta;
  if (target_rates) {
    g->targets[0] = target_rates[0];
    g->targets[1] = target_rates[1];
  }
  g->nslot = v.dmin + v.ndel;  // d_max + 1
  const long long N = v.N;
  g->ublocks = (int)((N + kThreads - 1) / kThreads);
  g->wblocks = (int)((N * 32 + kThreads - 1) / kThreads);
  // propagators in FP64 as the spiking tables compute them (h = 1 ms)
  const double tm = v.neuron.tau_m, tc = v.neuron.tau_c;
  g->pvv = std::exp(-1.0 / tm);
  g->pcc = std::exp(-1.0 / tc);
  g->kappa = -tm * tc / (tc - tm) * (g->pcc - g->pvv);

  GradParams& P = g->P;
  P.N = N;
  P.npc = v.npc;
  P.nexc = v.nexc;
  P.dmin = v.dmin;
  P.ndel = v.ndel;
  P.nslot = g->nslot;
  P.rowcap = v.rowcap;
  P.hard = g->hard;
  P.T = (int)n_steps;
  P.seed_lo = (uint32_t)(v.seed & 0xFFFFFFFFu);
  P.seed_hi = (uint32_t)(v.seed >> 32);
  P.beta = beta;
  P.theta = v.neuron.theta;
  P.vr = v.neuron.v_reset;
  P.dc = v.neuron.dc;
  P.pvv = (float)g->pvv;
  P.pcc = (float)g->pcc;
  P.kappa = (float)g->kappa;
  P.J = v.neuron.j_ext_mV;
  P.syn = static_cast<const uint2*>(v.syn);
  P.bend = v.bend;

  int rc = SNN_OK;
  const size_t n = (size_t)N;
  if (!rc) rc = galloc(g, &g->q, 65536);
  if (!rc) rc = galloc(g, &P.V, n);
  if (!rc) rc = galloc(g, &P.C, n);
  if (!rc) rc = galloc(g, &P.shist, n * g->nslot);
  if (!rc) rc = galloc(g, &P.xe, n);
  if (!rc) rc = galloc(g, &P.xin, n);
  if (!rc) rc = galloc(g, &P.tape, n * kTape * g->ckpt);
  if (!rc) rc = galloc(g, &P.rate_part, (size_t)g->ublocks * 2);
  if (!rc) rc = galloc(g, &P.vbar, n);
  if (!rc) rc = galloc(g, &P.cbar, n);
  if (!rc) rc = galloc(g, &P.ibe, n * g->nslot);
  if (!rc) rc = galloc(g, &P.ibi, n * g->nslot);
  if (!rc) rc = galloc(g, &P.gb, n * 3);
  if (!rc) rc = galloc(g, &P.sg, n);
  if (!rc) rc = galloc(g, &P.gacc, n * 6);
  if (!rc) rc = galloc(g, &g->ck, n * (2 + g->nslot) * g->nseg);
  if (rc) {
    const std::string why = g->err;
    grad_release(g);
    delete g;
    return fail_global(rc, why);
  }
  P.q = g->q;
  const std::vector<double>& qd = quantile_table();
  std::vector<float> qf(qd.size());
  for (size_t k = 0; k < qd.size(); ++k) qf[k] = (float)qd[k];
  cudaError_t e = cudaMemcpyAsync(g->q, qf.data(), qf.size() * 4, cudaMemcpyHostToDevice, v.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
  if (e != cudaSuccess) {
    grad_release(g);
    delete g;
    return fail_global(SNN_ECUDA, std::string("quantile table: ") + cudaGetErrorString(e));
  }
  *out = g;
  return SNN_OK;
}

int snn_grad_run(snn_grad* g, const double* theta, double* loss, double* rates, double* grad) {
  if (!g || !theta || !loss) return gfail(g, SNN_EINVAL, "null argument");
  for (int k = 0; k < 6; ++k)
    if (!std::isfinite(theta[k])) return gfail(g, SNN_EINVAL, "parameters must be finite");
  if (!(theta[5] > 0.0)) return gfail(g, SNN_EINVAL, "nu_ext must be positive");
  GradParams& P = g->P;
  for (int k = 0; k < 4; ++k) P.a[k] = (float)theta[k];
  P.pvc_e = (float)(theta[4] * g->kappa);
  P.pvc_i = (float)((double)g->v.neuron.gc_inh * g->kappa);
  const double lam = theta[5] * 1.0;  // nu_ext (kHz) * h (1 ms)
  P.lam = (float)lam;
  P.sqlam = (float)std::sqrt(lam);
  cudaStream_t st = g->v.stream;
  const long long N = g->v.N;
  const size_t n = (size_t)N;
  const size_t ckw = n * (2 + g->nslot);  // floats per checkpoint

  // forward, saving a checkpoint at the start of every segment
  grad_init_kernel<<<g->ublocks, kThreads, 0, st>>>(P);
  SNN_GCUDA(g, cudaGetLastError());
  SNN_GCUDA(g, cudaMemsetAsync(P.shist, 0, n * g->nslot * 4, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.xe, 0, n * 8, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.xin, 0, n * 8, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.rate_part, 0, (size_t)g->ublocks * 16, st));
  for (long long t = 0; t < g->T; ++t) {
    if (t % g->ckpt == 0) {
      float* ck = g->ck + (size_t)(t / g->ckpt) * ckw;
      SNN_GCUDA(g, cudaMemcpyAsync(ck, P.V, n * 4, cudaMemcpyDeviceToDevice, st));
      SNN_GCUDA(g, cudaMemcpyAsync(ck + n, P.C, n * 4, cudaMemcpyDeviceToDevice, st));
      SNN_GCUDA(g, cudaMemcpyAsync(ck + 2 * n, P.shist, n * g->nslot * 4,
                                   cudaMemcpyDeviceToDevice, st));
    }
    SNN_GCUDA(g, launch_forward_step(g, t, -1, 1));
  }
  std::vector<double> part((size_t)g->ublocks * 2);
  SNN_GCUDA(g, cudaMemcpyAsync(part.data(), P.rate_part, part.size() * 8, cudaMemcpyDeviceToHost, st));
  SNN_GCUDA(g, cudaStreamSynchronize(st));
  double se = 0.0, si = 0.0;
  for (int b = 0; b < g->ublocks; ++b) {
    se += part[2 * b];
    si += part[2 * b + 1];
  }
  const long long ncol = N / g->v.npc;
  const double NE = (double)ncol * g->v.nexc, NI = (double)N - NE;
  const double rE = NE > 0 ? 1000.0 * se / ((double)g->T * NE) : 0.0;
  const double rI = NI > 0 ? 1000.0 * si / ((double)g->T * NI) : 0.0;
  *loss = (rE - g->targets[0]) * (rE - g->targets[0]) + (rI - g->targets[1]) * (rI - g->targets[1]);
  if (rates) {
    rates[0] = rE;
    rates[1] = rI;
  }
  if (!grad) return SNN_OK;

  // backward: recompute each segment from its checkpoint, then run back
  P.dlds_e = NE > 0 ? (float)(2.0 * (rE - g->targets[0]) * 1000.0 / ((double)g->T * NE)) : 0.f;
  P.dlds_i = NI > 0 ? (float)(2.0 * (rI - g->targets[1]) * 1000.0 / ((double)g->T * NI)) : 0.f;
  SNN_GCUDA(g, cudaMemsetAsync(P.vbar, 0, n * 4, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.cbar, 0, n * 4, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.ibe, 0, n * g->nslot * 4, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.ibi, 0, n * g->nslot * 4, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.gb, 0, n * 3 * 4, st));
  SNN_GCUDA(g, cudaMemsetAsync(P.gacc, 0, n * 6 * 8, st));
  for (int seg = g->nseg - 1; seg >= 0; --seg) {
    const long long t0 = (long long)seg * g->ckpt;
    const long long t1 = std::min<long long>(g->T, t0 + g->ckpt);
    const float* ck = g->ck + (size_t)seg * ckw;
    SNN_GCUDA(g, cudaMemcpyAsync(P.V, ck, n * 4, cudaMemcpyDeviceToDevice, st));
    SNN_GCUDA(g, cudaMemcpyAsync(P.C, ck + n, n * 4, cudaMemcpyDeviceToDevice, st));
    SNN_GCUDA(g, cudaMemcpyAsync(P.shist, ck + 2 * n, n * g->nslot * 4, cudaMemcpyDeviceToDevice,
                                 st));
    for (long long t = t0; t < t1; ++t) SNN_GCUDA(g, launch_forward_step(g, t, (int)(t - t0), 0));
    for (long long tau = t1 - 1; tau >= t0; --tau) {
      grad_gather_kernel<<<g->wblocks, kThreads, 0, st>>>(P, tau);
      grad_backward_kernel<<<g->ublocks, kThreads, 0, st>>>(P, tau, (int)(tau - t0));
    }
    SNN_GCUDA(g, cudaGetLastError());
  }
  std::vector<double> acc(n * 6);
  SNN_GCUDA(g, cudaMemcpyAsync(acc.data(), P.gacc, acc.size() * 8, cudaMemcpyDeviceToHost, st));
  SNN_GCUDA(g, cudaStreamSynchronize(st));
  for (int k = 0; k < 6; ++k) {
    double sum = 0.0;
    for (size_t i = 0; i < n; ++i) sum += acc[(size_t)k * n + i];
    grad[k] = sum;
  }
  return SNN_OK;
}

const char* snn_grad_last_error(const snn_grad* g) { return g ? g->err.c_str() : ""; }

void snn_grad_destroy(snn_grad* g) {
  if (!g) return;
  cudaStreamSynchronize(g->v.stream);
  grad_release(g);
  delete g;
}

}  // extern "C"
