// snn_tables.cpp -- host-side FP64 tables of the model, rounded once.
//
// Every transcendental of the method is evaluated here on the host (and never
// on the device): the remote-offset CDF, the Poisson CDF of the external
// input, the normal quantiles of the weight distribution and the exact 1 ms
// propagator.  The operation order of each formula is fixed (the build is
// compiled with -ffp-contract=off) so that the results are reproducible.
#include <cmath>
#include <cstring>
#include <mutex>

#include "snn_internal.h"

namespace snn {
namespace {

constexpr double kTwo32 = 4294967296.0;

// Remote connectivity (arxiv 1511.09325, Sec. 2: connection probability
// decreasing with the distance between columns, cut off to a square
// stencil).  P(dx, dy) ~ exp(-r / lambda), r = sqrt(dx^2 + dy^2), over the
// offsets with |dx|, |dy| <= R except (0, 0), enumerated dy-major then dx
// ascending; the CDF is quantised to 32-bit thresholds.
void stencil_table(int R, double lambda, HostTables* t) {
  double w[kMaxOff];
  int n = 0;
  for (int dy = -R; dy <= R; ++dy) {
    for (int dx = -R; dx <= R; ++dx) {
      if (dx == 0 && dy == 0) continue;
      t->off_dx[n] = (int8_t)dx;
      t->off_dy[n] = (int8_t)dy;
      w[n] = std::exp(-std::sqrt((double)(dx * dx + dy * dy)) / lambda);
      ++n;
    }
  }
  t->n_off = n;
  double cum[kMaxOff], acc = 0.0;
  for (int m = 0; m < n; ++m) {
    acc = acc + w[m];
    cum[m] = acc;
  }
  for (int m = 0; m + 1 < n; ++m)
    t->stencil_thr[m] = (uint32_t)std::floor((cum[m] / acc) * kTwo32);
  t->stencil_thr[n - 1] = 0xFFFFFFFFu;  // unused: the last offset catches all
}

// External input (Sec. 2: extra excitatory input to every neuron): Poisson
// number of events per step with mean nu_ext * 1 ms, by inversion of the CDF
// quantised as thr[k] = floor(2^32 CDF(k)); the table ends at the first
// threshold >= 2^32 - 1, whose count absorbs the tail (< 2^-32).
int poisson_table(double lam, HostTables* t, std::string* err) {
  double pk = std::exp(-lam);
  double cdf = pk;
  int k = 0;
  double thr = std::floor(cdf * kTwo32);
  while (thr < 4294967295.0) {
    if (k >= kMaxPoisThr) {
      *err = "external rate too high for the Poisson table";
      return SNN_EINVAL;
    }
    t->pois_thr[k] = (uint32_t)thr;
    k = k + 1;
    pk = (pk * lam) / (double)k;
    cdf = cdf + pk;
    thr = std::floor(cdf * kTwo32);
  }
  t->n_pois_thr = k;  // sample = number of thresholds <= x
  for (int b = 0; b < 256; ++b) {
    uint64_t lo = (uint64_t)b << 24;
    int g = 0;
    while (g < k && (uint64_t)t->pois_thr[g] <= lo) ++g;
    t->pois_guide[b] = (uint8_t)g;
  }
  return SNN_OK;
}

// Standard-normal quantiles at (m + 0.5) / 65536 by 80 bisection steps on
// [-8, 8] against Phi(z) = erfc(-z / sqrt(2)) / 2.  They depend on no
// parameter: computed once per process.
void compute_normal_quantiles(std::vector<double>* q) {
  q->resize(65536);
  for (int m = 0; m < 65536; ++m) {
    const double target = ((double)m + 0.5) / 65536.0;
    double lo = -8.0, hi = 8.0;
    for (int step = 0; step < 80; ++step) {
      const double mid = 0.5 * (lo + hi);
      const double cdf = 0.5 * std::erfc(-mid * 0.70710678118654752440);
      if (cdf < target)
        lo = mid;
      else
        hi = mid;
    }
    (*q)[m] = 0.5 * (lo + hi);
  }
}

const std::vector<double>& normal_quantiles() {
  static std::once_flag once;
  static std::vector<double> q;
  std::call_once(once, [] { compute_normal_quantiles(&q); });
  return q;
}

// Round a double to binary16, ties to even; returns the 15 magnitude bits
// (the sign is implied by the population).  |a| must be below 65520.
uint32_t half_magnitude_rne(double a) {
  a = std::fabs(a);
  if (a == 0.0) return 0u;
  int e2 = 0;
  (void)std::frexp(a, &e2);  // a in [2^(e2-1), 2^e2)
  int E = e2 - 1;
  if (E < -14) E = -14;  // subnormal quantum 2^-24
  const double scaled = std::ldexp(a, 10 - E);
  uint32_t mant = (uint32_t)std::nearbyint(scaled);
  if (mant >= 2048u) {
    mant >>= 1;
    E += 1;
  }
  if (mant < 1024u) return mant;  // subnormal
  return ((uint32_t)(E + 15) << 10) | (mant - 1024u);
}

}  // namespace

int make_neuron_tables(const snn_neuron_params& np, HostTables* t, std::string* err) {
  int rc = poisson_table((double)np.nu_ext_kHz * 1.0, t, err);
  if (rc != SNN_OK) return rc;

  // Exact 1 ms propagator of dV/dt = -V/tau_m - g_c c, dc/dt = -c/tau_c:
  // P_vv = e^{-h/tau_m}, P_cc = e^{-h/tau_c},
  // P_vc = -g_c (tau_m tau_c / (tau_c - tau_m)) (P_cc - P_vv).
  const double h = 1.0, tm = (double)np.tau_m, tc = (double)np.tau_c;
  const double pvv = std::exp(-h / tm);
  const double pcc = std::exp(-h / tc);
  const double gcs[2] = {(double)np.gc_exc, (double)np.gc_inh};
  for (int p = 0; p < 2; ++p) {
    double v;
    if (tc == tm) {
      v = -gcs[p] * h * pvv;
    } else {
      const double prod = tm * tc;
      const double ratio = prod / (tc - tm);
      v = -(gcs[p] * ratio) * (pcc - pvv);
    }
    t->pvc[p] = (float)v;
  }
  t->pvv = (float)pvv;
  t->pcc = (float)pcc;
  t->jx = (int32_t)std::rint((double)np.j_ext_mV * 65536.0);
  t->nref = (int)std::rint((double)np.t_ref / h);
  return SNN_OK;
}

// Sec. 2's own law: offsets (dy-major, dx ascending, within 7x7) whose
// probability a exp(-r^2 / (2 sigma^2)) reaches the cut-off, each with the
// 32-bit threshold floor(P 2^32); the own column's threshold; the number of
// candidates per neuron (the column's other neurons, then n_per_col per
// offset).  Returns false when an offset beyond the 7x7 stencil would be kept.
static bool paper_table(const snn_synapse_params& sp, int npc, HostTables* t) {
  const double s2 = 2.0 * (double)sp.remote_sigma * (double)sp.remote_sigma;
  int n = 0;
  for (int dy = -3; dy <= 3; ++dy)
    for (int dx = -3; dx <= 3; ++dx) {
      if (dx == 0 && dy == 0) continue;
      const double pr = (double)sp.remote_a * std::exp(-(double)(dx * dx + dy * dy) / s2);
      if (pr < (double)sp.remote_cutoff) continue;
      t->poff_dx[n] = (int8_t)dx;
      t->poff_dy[n] = (int8_t)dy;
      t->poff_thr[n] = (unsigned long long)std::floor(pr * 4294967296.0);
      ++n;
    }
  t->n_poff = n;
  t->plocal_thr = (unsigned long long)std::floor((double)sp.p_local * 4294967296.0);
  t->n_cand = (long long)(npc - 1) + (long long)n * npc;
  return (double)sp.remote_a * std::exp(-16.0 / s2) < (double)sp.remote_cutoff;
}

int make_host_tables(const snn_neuron_params& np, const snn_synapse_params& sp,
                     int precision, HostTables* t, std::string* err) {
  stencil_table(sp.stencil_radius, (double)sp.lambda_cols, t);
  int rc = make_neuron_tables(np, t, err);
  if (rc != SNN_OK) return rc;
  t->k_local = (int)std::rint((double)sp.frac_local * (double)sp.k_out);
  if (sp.connectivity == SNN_CONN_PAPER && !paper_table(sp, np.n_per_col, t)) {
    *err = "the paper law keeps offsets beyond the 7x7 stencil";
    return SNN_EINVAL;
  }

  // Weights: w = mu (1 + cv Q), clipped to the source population's sign,
  // then stored as float bits (F32W) or half magnitude bits (F16W).
  const std::vector<double>& q = normal_quantiles();
  t->wtab.assign(2 * 65536, 0u);
  const double mus[2] = {(double)sp.w_exc_mV, (double)sp.w_inh_mV};
  for (int p = 0; p < 2; ++p) {
    for (int m = 0; m < 65536; ++m) {
      double w = mus[p] * (1.0 + (double)sp.w_cv * q[m]);
      if (p == 0 && w < 0.0) w = 0.0;
      if (p == 1 && w > 0.0) w = 0.0;
      uint32_t bits;
      if (precision == SNN_EXACT_F32W) {
        const float f = (float)w;
        std::memcpy(&bits, &f, 4);
      } else {
        if (std::fabs(w) >= 65504.0) {
          *err = "weight does not fit binary16";
          return SNN_EINVAL;
        }
        bits = half_magnitude_rne(w);
      }
      t->wtab[(size_t)p * 65536 + m] = bits;
    }
  }
  return SNN_OK;
}

const std::vector<double>& quantile_table() { return normal_quantiles(); }

}  // namespace snn
