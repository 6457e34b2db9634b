/*
 * snn_oracle.c -- plain, slow CPU oracle of the per-1 ms step of a 2-D grid of
 * cortical columns of LIF neurons with spike-frequency adaptation (arxiv
 * 1511.09325, Sec. 2 "Methods": 1240 neurons per column, 80 % excitatory /
 * 20 % inhibitory, local plus distance-dependent remote connectivity, external
 * excitatory input, plasticity disabled).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU
 * baseline of the benchmark may load this file.  The GPU library never calls
 * it and shares no code, header, table or constant generator with it.
 *
 * The paper states the model in prose only (Sec. 2) and prints no equations,
 * delays, weights or rates.  Every formula below is the reading adopted for
 * this implementation; each is marked "reading:".  Randomness is drawn from
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
 * as 1, 2, 3", SC'11), implemented here from that definition.
 *
 * Structure, deliberately event-driven and unoptimised:
 *   - no stored synapse matrix: the 1240 outgoing synapses of a spiking neuron
 *     are regenerated from the counter-based generator every time it spikes;
 *   - delivery pushes into a ring of (d_max + 1) per-step input slots;
 *   - three arithmetic modes: F32W and F16W (FP32 state, int32 fixed-point
 *     input in units of 2^-16 mV, weights rounded to float / half) and F64
 *     (double state, double input, unrounded weights).
 *
 * Compile with -ffp-contract=off: every float operation is spelled out and
 * must not be fused by the compiler.
 *
 * Pins (tests, no GPU): Philox known-answer vectors; the quantile, Poisson and
 * propagator tables against library routines; closed forms of the
 * sub-threshold and constant-drive dynamics; construction invariants and
 * Table 1 sizes; whole networks against a dense per-delay restatement, bit
 * for bit.  Parity unpinned by the paper: the network's firing rates, which
 * it does not print.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

#define ORC_MODE_F32W 0
#define ORC_MODE_F16W 1
#define ORC_MODE_F64 2

/* Philox stream tags: the third counter word (reading: key = 64-bit seed,
 * counter = (a, b, tag, 0)). */
#define TAG_CONN 1u
#define TAG_EXT 2u
#define TAG_INIT 3u
#define TAG_SURR 4u /* normal draws of the relaxed (differentiable) network */
#define TAG_PCONN 5u /* candidate draws of the paper's connectivity law       */
#define CONN_FIXED 0
#define CONN_PAPER 1

#define POIS_CAP 128 /* table entries; lambda is limited so that it saturates */
#define Q_SIZE 65536

typedef struct {
  int32_t grid_w, grid_h;  /* columns along x and y                        */
  int32_t n_per_col;       /* neurons per column (1240, Sec. 2)            */
  int32_t n_exc;           /* excitatory neurons per column (992 = 80 %)   */
  float tau_m;             /* membrane time constant, ms                   */
  float theta;             /* threshold, mV                                */
  float v_reset;           /* reset potential, mV                          */
  float t_ref;             /* absolute refractory period, ms               */
  float tau_c;             /* calcium (adaptation) time constant, ms       */
  float dc;                /* calcium increment per spike                  */
  float gc_exc, gc_inh;    /* adaptation gain, mV/ms per unit calcium      */
  float j_ext;             /* external synaptic efficacy, mV               */
  float nu_ext_khz;        /* external Poisson rate per neuron, kHz        */
  int32_t k_out;           /* outgoing synapses per neuron (1240)          */
  float frac_local;        /* fraction of them inside the own column       */
  float lambda_cols;       /* remote length constant, in grid steps        */
  int32_t stencil_radius;  /* remote cut-off: |dx|,|dy| <= radius          */
  float w_exc, w_inh;      /* mean weights, mV                             */
  float w_cv;              /* coefficient of variation of the weights      */
  int32_t d_min, d_max;    /* axonal delay range, steps                    */
  double h;                /* step, ms (1 for the network)                 */
  uint64_t seed;
  int32_t connectivity;    /* CONN_FIXED: the configs' law; CONN_PAPER: Sec. 2 */
  float p_local;           /* paper: P(synapse) to each other neuron of the column */
  float remote_a;          /* paper: P at distance r is a exp(-r^2 / 2 sigma^2) */
  float remote_sigma;      /* paper: sigma, grid steps                      */
  float remote_cutoff;     /* paper: offsets with P below this are dropped  */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 bit     */
/* multiplies whose halves are xored into the other words, with a Weyl key    */
/* schedule.                                                                 */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  int round;
  for (round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += W0;
    k1 += W1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint32_t a, uint32_t b, uint32_t tag,
                 uint32_t out[4]) {
  uint32_t ctr[4], key[2];
  ctr[0] = a; ctr[1] = b; ctr[2] = tag; ctr[3] = 0u;
  key[0] = (uint32_t)(seed & 0xFFFFFFFFu);
  key[1] = (uint32_t)(seed >> 32);
  orc_philox4x32_10(ctr, key, out);
}

/* u_n(x): uniform integer in [0, n) from one 32-bit word, (x * n) >> 32. */
static uint32_t uniform_below(uint32_t x, uint32_t n) {
  return (uint32_t)(((uint64_t)x * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Tables computed once in FP64 (reading: every transcendental of the model   */
/* is evaluated on the host, so no device transcendental enters the method).  */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n_off;                      /* remote stencil offsets                  */
  int off_dx[64], off_dy[64];     /* dy-major, dx ascending, (0,0) excluded  */
  uint64_t stencil_thr[64];       /* first m with x1 < thr[m] is drawn       */
  int n_pois;                     /* entries until the table saturates       */
  uint64_t pois_thr[POIS_CAP];    /* k = first index with x0 < thr[k]        */
  double *q;                      /* standard-normal quantiles, Q_SIZE       */
  double pvv, pcc, pvc[2];        /* 1-step propagators, [0]=E, [1]=I        */
  int32_t jx;                     /* external efficacy in 2^-16 mV units     */
  int nref;                       /* refractory steps                        */
  int k_local;                    /* synapses k < k_local stay local         */
  int n_poff;                     /* paper law: kept remote offsets          */
  int poff_dx[64], poff_dy[64];   /* dy-major, dx ascending                  */
  uint64_t poff_thr[64];          /* candidate kept iff its word < thr       */
  uint64_t plocal_thr;            /* the same for the own column             */
} orc_tables;

/* Sec. 2: remote connection probability decreases with the distance between
 * columns.  Reading (configs of this implementation): P(offset) is
 * proportional to exp(-r / lambda) over the (2R+1)^2 - 1 offsets of the
 * square cut-off stencil, r the Euclidean distance in grid steps.  The CDF is
 * quantised to 32-bit thresholds. */
static void make_stencil(const orc_params *p, orc_tables *t) {
  double e[64], s[64], total;
  int R = p->stencil_radius, n = 0, dy, dx, m;
  for (dy = -R; dy <= R; ++dy)
    for (dx = -R; dx <= R; ++dx) {
      if (dx == 0 && dy == 0) continue;
      t->off_dx[n] = dx;
      t->off_dy[n] = dy;
      e[n] = exp(-sqrt((double)(dx * dx + dy * dy)) / (double)p->lambda_cols);
      ++n;
    }
  t->n_off = n;
  total = 0.0;
  for (m = 0; m < n; ++m) {
    total = total + e[m];
    s[m] = total;
  }
  for (m = 0; m < n; ++m)
    t->stencil_thr[m] = (uint64_t)floor((s[m] / total) * 4294967296.0);
  t->stencil_thr[n - 1] = 4294967296ull;
}

/* External input: a Poisson number of events per step with mean
 * lambda = nu_ext * h, sampled by inversion of its CDF quantised to 2^-32:
 * thr[k] = floor(2^32 CDF(k)).  The table ends at the first k whose threshold
 * reaches 2^32 - 1; that entry is set to 2^32, so the tail mass beyond it
 * (below 2^-32) is folded into the last count. */
static void make_poisson(const orc_params *p, orc_tables *t) {
  double lam = (double)p->nu_ext_khz * p->h;
  double pk = exp(-lam), cdf = pk;
  int k = 0;
  t->pois_thr[0] = (uint64_t)floor(cdf * 4294967296.0);
  while (t->pois_thr[k] < 4294967295ull && k + 1 < POIS_CAP) {
    k = k + 1;
    pk = (pk * lam) / (double)k;
    cdf = cdf + pk;
    t->pois_thr[k] = (uint64_t)floor(cdf * 4294967296.0);
  }
  t->pois_thr[k] = 4294967296ull;
  t->n_pois = k + 1;
}

/* Standard-normal quantile Q[m] = Phi^-1((m + 0.5) / 65536) by 80 bisection
 * steps on [-8, 8] against Phi(z) = erfc(-z / sqrt 2) / 2. */
static void make_quantiles(double *q) {
  int m, it;
  for (m = 0; m < Q_SIZE; ++m) {
    double pr = ((double)m + 0.5) / 65536.0, lo = -8.0, hi = 8.0;
    for (it = 0; it < 80; ++it) {
      double mid = 0.5 * (lo + hi);
      if (0.5 * erfc(-mid * 0.70710678118654752440) < pr)
        lo = mid;
      else
        hi = mid;
    }
    q[m] = 0.5 * (lo + hi);
  }
}

/* Exact one-step propagator of dV/dt = -V/tau_m - g_c c, dc/dt = -c/tau_c:
 * V(h) = e^{-h/tau_m} V + P_vc c,  c(h) = e^{-h/tau_c} c, with
 * P_vc = -g_c tau_m tau_c / (tau_c - tau_m) (e^{-h/tau_c} - e^{-h/tau_m}). */
static double prop_vc(double gc, double tm, double tc, double h, double pvv,
                      double pcc) {
  double a, b;
  if (tc == tm) return -gc * h * pvv;
  a = tm * tc;
  b = a / (tc - tm);
  return -(gc * b) * (pcc - pvv);
}

/* Sec. 2's own connectivity law (reading): a neuron reaches every other
 * neuron of its column with probability p_local and every neuron of a column
 * at Euclidean grid distance r with probability a exp(-r^2 / (2 sigma^2));
 * offsets where that probability is below the cut-off are dropped (the
 * paper's "stencil").  Each probability becomes a 32-bit threshold
 * floor(P 2^32) against one Philox word per candidate. */
static void make_paper_stencil(const orc_params *p, orc_tables *t) {
  int dy, dx, n = 0;
  double s2 = 2.0 * (double)p->remote_sigma * (double)p->remote_sigma;
  for (dy = -3; dy <= 3; ++dy)
    for (dx = -3; dx <= 3; ++dx) {
      double pr;
      if (dx == 0 && dy == 0) continue;
      pr = (double)p->remote_a * exp(-(double)(dx * dx + dy * dy) / s2);
      if (pr < (double)p->remote_cutoff) continue;
      t->poff_dx[n] = dx;
      t->poff_dy[n] = dy;
      t->poff_thr[n] = (uint64_t)floor(pr * 4294967296.0);
      ++n;
    }
  t->n_poff = n;
  t->plocal_thr = (uint64_t)floor((double)p->p_local * 4294967296.0);
}

static int make_tables(const orc_params *p, orc_tables *t) {
  double tm = (double)p->tau_m, tc = (double)p->tau_c;
  memset(t, 0, sizeof(*t));
  make_stencil(p, t);
  make_paper_stencil(p, t);
  make_poisson(p, t);
  t->q = (double *)malloc(sizeof(double) * Q_SIZE);
  if (!t->q) return ORC_ENOMEM;
  make_quantiles(t->q);
  t->pvv = exp(-p->h / tm);
  t->pcc = exp(-p->h / tc);
  t->pvc[0] = prop_vc((double)p->gc_exc, tm, tc, p->h, t->pvv, t->pcc);
  t->pvc[1] = prop_vc((double)p->gc_inh, tm, tc, p->h, t->pvv, t->pcc);
  t->jx = (int32_t)rint((double)p->j_ext * 65536.0);
  t->nref = (int)rint((double)p->t_ref / p->h);
  t->k_local = (int)rint((double)p->frac_local * (double)p->k_out);
  return ORC_OK;
}

static void free_tables(orc_tables *t) {
  free(t->q);
  t->q = NULL;
}

static int validate(const orc_params *p) {
  if (p->grid_w < 1 || p->grid_h < 1) return ORC_EINVAL;
  if (p->n_per_col < 2 || p->n_per_col > 2048) return ORC_EINVAL;
  if (p->n_exc < 0 || p->n_exc > p->n_per_col) return ORC_EINVAL;
  if (p->k_out < 1) return ORC_EINVAL;
  if (p->stencil_radius < 1 || p->stencil_radius > 3) return ORC_EINVAL;
  if (p->d_min < 1 || p->d_max < p->d_min || p->d_max > 64) return ORC_EINVAL;
  if (!(p->tau_m > 0.0f) || !(p->tau_c > 0.0f) || !(p->h > 0.0)) return ORC_EINVAL;
  if (!(p->nu_ext_khz >= 0.0f) || (double)p->nu_ext_khz * p->h > 40.0) return ORC_EINVAL;
  if (!(p->lambda_cols > 0.0f)) return ORC_EINVAL;
  if (!(p->frac_local >= 0.0f && p->frac_local <= 1.0f)) return ORC_EINVAL;
  if (p->connectivity != CONN_FIXED && p->connectivity != CONN_PAPER) return ORC_EINVAL;
  if (p->connectivity == CONN_PAPER) {
    double s2 = 2.0 * (double)p->remote_sigma * (double)p->remote_sigma;
    if (!(p->p_local >= 0.0f && p->p_local <= 1.0f)) return ORC_EINVAL;
    if (!(p->remote_a >= 0.0f && p->remote_a <= 1.0f)) return ORC_EINVAL;
    if (!(p->remote_sigma > 0.0f) || !(p->remote_cutoff > 0.0f)) return ORC_EINVAL;
    /* the kept offsets must fit the 7x7 stencil: the nearest offset outside
     * it lies at r^2 = 16 */
    if ((double)p->remote_a * exp(-16.0 / s2) >= (double)p->remote_cutoff) return ORC_EINVAL;
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Half precision: round a double to the nearest binary16 (ties to even).     */
/* ------------------------------------------------------------------------ */
static float double_to_half_to_float(double w) { return (float)(_Float16)w; }

/* ------------------------------------------------------------------------ */
/* One synapse.  Reading of Sec. 2 with the configs of this implementation:   */
/* synapse k of neuron j (column (x, y), index l_j inside the column) draws   */
/* Philox(seed; j, k, CONN) = (x0, x1, x2, x3):                               */
/*   k <  k_local: target in the own column, l = u_{n-1}(x0), l += (l >= l_j) */
/*   k >= k_local: stencil offset m = first with x1 < thr[m]; target column   */
/*                 ((x+dx) mod W, (y+dy) mod H), l = u_n(x0)                  */
/*   delay  d = d_min + u_{d_max-d_min+1}(x2)                                 */
/*   weight w = mu (1 + cv Q[x3 >> 16]), clipped to the sign of the source    */
/*          population (Dale), then rounded per mode.                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t target;
  int32_t delay;
  int32_t wfx;   /* fixed-point weight, 2^-16 mV (F32W / F16W)  */
  double w;      /* weight after the mode's rounding, mV         */
  int32_t dx, dy; /* stencil offset drawn (0,0 for local)        */
} orc_syn;

static void delay_and_weight(const orc_params *p, const orc_tables *t, int mode, int exc,
                             const uint32_t x[4], orc_syn *s);

static void synapse(const orc_params *p, const orc_tables *t, int mode,
                    int64_t j, int32_t k, orc_syn *s) {
  uint32_t x[4];
  int64_t col = j / p->n_per_col;
  int32_t lj = (int32_t)(j % p->n_per_col);
  int32_t cx = (int32_t)(col % p->grid_w), cy = (int32_t)(col / p->grid_w);
  int32_t l, tx, ty;
  int exc = lj < p->n_exc;
  draw(p->seed, (uint32_t)j, (uint32_t)k, TAG_CONN, x);
  if (k < t->k_local) {
    l = (int32_t)uniform_below(x[0], (uint32_t)(p->n_per_col - 1));
    if (l >= lj) l += 1;
    tx = cx;
    ty = cy;
    s->dx = 0;
    s->dy = 0;
  } else {
    int m = 0;
    while ((uint64_t)x[1] >= t->stencil_thr[m]) ++m;
    s->dx = t->off_dx[m];
    s->dy = t->off_dy[m];
    l = (int32_t)uniform_below(x[0], (uint32_t)p->n_per_col);
    tx = ((cx + s->dx) % p->grid_w + p->grid_w) % p->grid_w;
    ty = ((cy + s->dy) % p->grid_h + p->grid_h) % p->grid_h;
  }
  s->target = ((int64_t)ty * p->grid_w + tx) * p->n_per_col + l;
  delay_and_weight(p, t, mode, exc, x, s);
}

/* Delay and weight of a synapse from its Philox block x (words 2 and 3). */
static void delay_and_weight(const orc_params *p, const orc_tables *t, int mode, int exc,
                             const uint32_t x[4], orc_syn *s) {
  double w;
  s->delay = p->d_min + (int32_t)uniform_below(x[2], (uint32_t)(p->d_max - p->d_min + 1));
  w = (double)(exc ? p->w_exc : p->w_inh) *
      (1.0 + (double)p->w_cv * t->q[x[3] >> 16]);
  if (exc) {
    if (w < 0.0) w = 0.0;
  } else {
    if (w > 0.0) w = 0.0;
  }
  if (mode == ORC_MODE_F32W) {
    float w32 = (float)w;
    s->w = (double)w32;
    s->wfx = (int32_t)rintf(w32 * 65536.0f);
  } else if (mode == ORC_MODE_F16W) {
    float w16 = double_to_half_to_float(w);
    s->w = (double)w16;
    s->wfx = (int32_t)rintf(w16 * 65536.0f);
  } else {
    s->w = w;
    s->wfx = 0;
  }
}

/* Candidates of neuron j under the paper's law, in a fixed order: the other
 * n_per_col - 1 neurons of its own column (ascending index), then for each
 * kept remote offset (dy-major, dx ascending) the n_per_col neurons of that
 * column.  Candidate c is kept iff word c mod 4 of Philox(seed; j, c / 4,
 * PCONN) is below its threshold.  The k-th kept candidate (k from 0) is
 * synapse k: its delay and weight come from Philox(seed; j, k, CONN) as in
 * the fixed law.  Writes the synapses to out (capacity: the candidate count)
 * and returns how many there are. */
static int64_t paper_row(const orc_params *p, const orc_tables *t, int mode, int64_t j,
                         orc_syn *out) {
  const int32_t npc = p->n_per_col;
  int64_t col = j / npc;
  int32_t lj = (int32_t)(j % npc);
  int32_t cx = (int32_t)(col % p->grid_w), cy = (int32_t)(col / p->grid_w);
  int exc = lj < p->n_exc;
  int64_t n_cand = (int64_t)(npc - 1) + (int64_t)t->n_poff * npc, c, k = 0;
  uint32_t word[4];
  for (c = 0; c < n_cand; ++c) {
    uint64_t thr;
    int32_t l, tx, ty, dx, dy;
    if ((c & 3) == 0) draw(p->seed, (uint32_t)j, (uint32_t)(c >> 2), TAG_PCONN, word);
    if (c < npc - 1) {
      thr = t->plocal_thr;
      l = (int32_t)c + ((int32_t)c >= lj ? 1 : 0);
      dx = 0;
      dy = 0;
    } else {
      int64_t r = c - (npc - 1);
      int m = (int)(r / npc);
      thr = t->poff_thr[m];
      l = (int32_t)(r % npc);
      dx = t->poff_dx[m];
      dy = t->poff_dy[m];
    }
    if ((uint64_t)word[c & 3] >= thr) continue;
    tx = ((cx + dx) % p->grid_w + p->grid_w) % p->grid_w;
    ty = ((cy + dy) % p->grid_h + p->grid_h) % p->grid_h;
    {
      uint32_t x[4];
      orc_syn *s = &out[k];
      s->target = ((int64_t)ty * p->grid_w + tx) * npc + l;
      s->dx = dx;
      s->dy = dy;
      draw(p->seed, (uint32_t)j, (uint32_t)k, TAG_CONN, x);
      delay_and_weight(p, t, mode, exc, x, s);
    }
    ++k;
  }
  return k;
}

static int64_t paper_candidates(const orc_params *p, const orc_tables *t) {
  return (int64_t)(p->n_per_col - 1) + (int64_t)t->n_poff * p->n_per_col;
}

/* ------------------------------------------------------------------------ */
/* Neuron update, one step.  Reading of the LIF + SFA model of Sec. 2 (the    */
/* calcium-dependent after-hyperpolarisation current g_c c):                  */
/*   1. refractory: r > 0 -> r -= 1, V = V_reset, the input is discarded;     */
/*   2. else V += I; if V >= theta: spike, V = V_reset, r = nref, c += dc;    */
/*   3. V = P_vc c + P_vv V (one fused multiply-add), c = P_cc c.             */
/* ------------------------------------------------------------------------ */
static int step_f32(float *V, float *c, uint8_t *r, int32_t I, float theta,
                    float vr, float dc, int nref, float pvv, float pvc,
                    float pcc) {
  int spk = 0;
  float v = *V, cc = *c;
  if (*r > 0) {
    *r = (uint8_t)(*r - 1);
    v = vr;
  } else {
    v = v + ((float)I * 1.52587890625e-05f); /* 2^-16 mV per unit */
    if (v >= theta) {
      spk = 1;
      v = vr;
      *r = (uint8_t)nref;
      cc = cc + dc;
    }
  }
  v = fmaf(cc, pvc, v * pvv);
  cc = cc * pcc;
  *V = v;
  *c = cc;
  return spk;
}

static int step_f64(double *V, double *c, uint8_t *r, double I, double theta,
                    double vr, double dc, int nref, double pvv, double pvc,
                    double pcc) {
  int spk = 0;
  double v = *V, cc = *c;
  if (*r > 0) {
    *r = (uint8_t)(*r - 1);
    v = vr;
  } else {
    v = v + I;
    if (v >= theta) {
      spk = 1;
      v = vr;
      *r = (uint8_t)nref;
      cc = cc + dc;
    }
  }
  v = pvc * cc + pvv * v;
  cc = cc * pcc;
  *V = v;
  *c = cc;
  return spk;
}

static int poisson_k(const orc_tables *t, uint32_t x) {
  int k = 0;
  while ((uint64_t)x >= t->pois_thr[k]) ++k;
  return k;
}

/* External events of neuron i at step t: one 32-bit word of
 * Philox(seed; i/4, t, EXT), word i mod 4. */
static uint32_t ext_word(uint64_t seed, int64_t i, int64_t t) {
  uint32_t x[4];
  draw(seed, (uint32_t)(i >> 2), (uint32_t)t, TAG_EXT, x);
  return x[i & 3];
}

/* Initial membrane potential: uniform in [0, theta), 24-bit resolution,
 * from word i mod 4 of Philox(seed; i/4, 0, INIT). */
static uint32_t init_word(uint64_t seed, int64_t i) {
  uint32_t x[4];
  draw(seed, (uint32_t)(i >> 2), 0u, TAG_INIT, x);
  return x[i & 3];
}

/* ------------------------------------------------------------------------ */
/* Public entry points (ctypes).                                             */
/* ------------------------------------------------------------------------ */

int orc_validate(const orc_params *p) { return validate(p); }

/* Tables for inspection: stencil (dx, dy, thr) x n_off, Poisson thresholds,
 * quantiles, propagators {pvv, pcc, pvc_e, pvc_i}, jx, nref, k_local. */
int orc_tables_export(const orc_params *p, int32_t *n_off, int32_t *off_dx,
                      int32_t *off_dy, uint64_t *stencil_thr, int32_t *n_pois,
                      uint64_t *pois_thr, double *q, double *props,
                      int32_t *ints) {
  orc_tables t;
  int i, rc = validate(p);
  if (rc) return rc;
  rc = make_tables(p, &t);
  if (rc) return rc;
  *n_off = t.n_off;
  for (i = 0; i < t.n_off; ++i) {
    off_dx[i] = t.off_dx[i];
    off_dy[i] = t.off_dy[i];
    stencil_thr[i] = t.stencil_thr[i];
  }
  *n_pois = t.n_pois;
  for (i = 0; i < t.n_pois; ++i) pois_thr[i] = t.pois_thr[i];
  memcpy(q, t.q, sizeof(double) * Q_SIZE);
  props[0] = t.pvv;
  props[1] = t.pcc;
  props[2] = t.pvc[0];
  props[3] = t.pvc[1];
  ints[0] = t.jx;
  ints[1] = t.nref;
  ints[2] = t.k_local;
  free_tables(&t);
  return ORC_OK;
}

/* The k_out synapses of neurons j0 .. j0+n-1 in k order: target, delay,
 * fixed-point weight, rounded weight, stencil offset. */
int orc_synapses(const orc_params *p, int mode, int64_t j0, int64_t n,
                 int64_t *target, int32_t *delay, int32_t *wfx, double *w,
                 int32_t *dx, int32_t *dy) {
  orc_tables t;
  int64_t N, j, o = 0;
  int32_t k;
  int rc = validate(p);
  if (rc) return rc;
  N = (int64_t)p->grid_w * p->grid_h * p->n_per_col;
  if (j0 < 0 || n < 0 || j0 + n > N) return ORC_EINVAL;
  if (p->connectivity != CONN_FIXED) return ORC_EINVAL; /* see orc_paper_synapses */
  rc = make_tables(p, &t);
  if (rc) return rc;
  for (j = j0; j < j0 + n; ++j)
    for (k = 0; k < p->k_out; ++k, ++o) {
      orc_syn s;
      synapse(p, &t, mode, j, k, &s);
      if (target) target[o] = s.target;
      if (delay) delay[o] = s.delay;
      if (wfx) wfx[o] = s.wfx;
      if (w) w[o] = s.w;
      if (dx) dx[o] = s.dx;
      if (dy) dy[o] = s.dy;
    }
  free_tables(&t);
  return ORC_OK;
}

/* The paper law's kept offsets and thresholds (n_off <= 48). */
int orc_paper_tables(const orc_params *p, int32_t *n_off, int32_t *dx, int32_t *dy,
                     uint64_t *thr, uint64_t *local_thr, int64_t *n_cand) {
  orc_tables t;
  int m, rc = validate(p);
  if (rc) return rc;
  rc = make_tables(p, &t);
  if (rc) return rc;
  *n_off = t.n_poff;
  for (m = 0; m < t.n_poff; ++m) {
    dx[m] = t.poff_dx[m];
    dy[m] = t.poff_dy[m];
    thr[m] = t.poff_thr[m];
  }
  *local_thr = t.plocal_thr;
  *n_cand = paper_candidates(p, &t);
  free_tables(&t);
  return ORC_OK;
}

/* Synapses of neurons j0 .. j0+n-1 under the paper law: row r's count[r]
 * synapses at [r * cap, r * cap + count[r]) of each array (cap >= the
 * candidate count), in k order. */
int orc_paper_synapses(const orc_params *p, int mode, int64_t j0, int64_t n, int64_t cap,
                       int64_t *count, int64_t *target, int32_t *delay, int32_t *wfx,
                       double *w, int32_t *dx, int32_t *dy) {
  orc_tables t;
  orc_syn *row;
  int64_t N, r, k;
  int rc = validate(p);
  if (rc) return rc;
  N = (int64_t)p->grid_w * p->grid_h * p->n_per_col;
  if (p->connectivity != CONN_PAPER || j0 < 0 || n < 0 || j0 + n > N) return ORC_EINVAL;
  rc = make_tables(p, &t);
  if (rc) return rc;
  if (cap < paper_candidates(p, &t)) {
    free_tables(&t);
    return ORC_EINVAL;
  }
  row = (orc_syn *)malloc(sizeof(orc_syn) * (size_t)paper_candidates(p, &t));
  if (!row) {
    free_tables(&t);
    return ORC_ENOMEM;
  }
  for (r = 0; r < n; ++r) {
    int64_t cnt = paper_row(p, &t, mode, j0 + r, row), o = r * cap;
    count[r] = cnt;
    for (k = 0; k < cnt; ++k, ++o) {
      if (target) target[o] = row[k].target;
      if (delay) delay[o] = row[k].delay;
      if (wfx) wfx[o] = row[k].wfx;
      if (w) w[o] = row[k].w;
      if (dx) dx[o] = row[k].dx;
      if (dy) dy[o] = row[k].dy;
    }
  }
  free(row);
  free_tables(&t);
  return ORC_OK;
}

/* External event counts k_i(t) for neurons i0..i0+n-1 at steps t0..t0+nt-1,
 * step-major. */
int orc_ext_counts(const orc_params *p, int64_t i0, int64_t n, int64_t t0,
                   int64_t nt, int32_t *k) {
  orc_tables tb;
  int64_t i, t;
  int rc = validate(p);
  if (rc) return rc;
  rc = make_tables(p, &tb);
  if (rc) return rc;
  for (t = 0; t < nt; ++t)
    for (i = 0; i < n; ++i)
      k[t * n + i] = poisson_k(&tb, ext_word(p->seed, i0 + i, t0 + t));
  free_tables(&tb);
  return ORC_OK;
}

/* Standard-normal draws of the relaxed network (reading: the external
 * Poisson input is replaced by its Gaussian approximation, whose normal
 * variate is the quantile-table value of the top 16 bits of word i mod 4 of
 * Philox(seed; i/4, t, SURR)).  xi[t][i] for t0 <= t < t0 + nt. */
int orc_surr_xi(const orc_params *p, int64_t i0, int64_t n, int64_t t0, int64_t nt,
                double *xi) {
  orc_tables tb;
  int64_t i, t;
  uint32_t x[4];
  int rc = validate(p);
  if (rc) return rc;
  rc = make_tables(p, &tb);
  if (rc) return rc;
  for (t = 0; t < nt; ++t)
    for (i = 0; i < n; ++i) {
      draw(p->seed, (uint32_t)((i0 + i) >> 2), (uint32_t)(t0 + t), TAG_SURR, x);
      xi[t * n + i] = tb.q[x[(i0 + i) & 3] >> 16];
    }
  free_tables(&tb);
  return ORC_OK;
}

/* Initial membrane potentials of neurons i0..i0+n-1 (as double). */
int orc_init_v(const orc_params *p, int mode, int64_t i0, int64_t n, double *v) {
  int64_t i;
  int rc = validate(p);
  if (rc) return rc;
  for (i = 0; i < n; ++i) {
    uint32_t u = init_word(p->seed, i0 + i);
    if (mode == ORC_MODE_F64)
      v[i] = (double)p->theta * ((double)(u >> 8) * 5.9604644775390625e-08);
    else
      v[i] = (double)(p->theta * ((float)(u >> 8) * 5.9604644775390625e-08f));
  }
  return ORC_OK;
}

/* Single-neuron trace driven by an explicit input sequence (no network, no
 * external Poisson input).  mode F32W/F16W: input_fx[t] in 2^-16 mV units;
 * mode F64: input_mv[t] in mV.  pop = 0 (E) or 1 (I).  Writes V, c after each
 * step and the spike flag of each step.  Uses the same step functions as the
 * network run. */
int orc_neuron_trace(const orc_params *p, int mode, int pop, double v0,
                     double c0, int64_t n_steps, const int32_t *input_fx,
                     const double *input_mv, double *v_out, double *c_out,
                     uint8_t *spk_out) {
  double tm = (double)p->tau_m, tc = (double)p->tau_c;
  double pvv = exp(-p->h / tm), pcc = exp(-p->h / tc);
  double gc = pop == 0 ? (double)p->gc_exc : (double)p->gc_inh;
  double pvc = prop_vc(gc, tm, tc, p->h, pvv, pcc);
  int nref = (int)rint((double)p->t_ref / p->h);
  int64_t t;
  uint8_t r = 0;
  if (!(p->tau_m > 0.0f) || !(p->tau_c > 0.0f) || !(p->h > 0.0)) return ORC_EINVAL;
  if (mode == ORC_MODE_F64) {
    double V = v0, c = c0;
    for (t = 0; t < n_steps; ++t) {
      spk_out[t] = (uint8_t)step_f64(&V, &c, &r, input_mv[t], (double)p->theta,
                                     (double)p->v_reset, (double)p->dc, nref,
                                     pvv, pvc, pcc);
      v_out[t] = V;
      c_out[t] = c;
    }
  } else {
    float V = (float)v0, c = (float)c0;
    for (t = 0; t < n_steps; ++t) {
      spk_out[t] = (uint8_t)step_f32(&V, &c, &r, input_fx[t], p->theta,
                                     p->v_reset, p->dc, nref, (float)pvv,
                                     (float)pvc, (float)pcc);
      v_out[t] = (double)V;
      c_out[t] = (double)c;
    }
  }
  return ORC_OK;
}

/* Network run for n_steps from the initial state.
 * Outputs (any may be NULL):
 *   spk_t, spk_i [cap]: raster in step order, neuron order within a step;
 *   n_spk: total spikes (may exceed cap; only cap are stored);
 *   step_spikes [n_steps], step_ext [n_steps]: spikes and external events;
 *   v_end, c_end [N] (as double), r_end [N]: final state. */
int orc_run(const orc_params *p, int mode, int64_t n_steps, int64_t cap,
            int32_t *spk_t, int32_t *spk_i, int64_t *n_spk,
            int64_t *step_spikes, int64_t *step_ext, double *v_end,
            double *c_end, uint8_t *r_end) {
  orc_tables tb;
  int64_t N, i, t, ns = 0;
  int DR, rc = validate(p);
  int32_t *R32 = NULL, *fired = NULL;
  double *R64 = NULL, *V64 = NULL, *C64 = NULL;
  float *V32 = NULL, *C32 = NULL;
  uint8_t *ref = NULL;
  orc_syn *prow = NULL; /* paper law: one row's synapses */
  float pvv32, pcc32, pvc32[2];
  if (rc) return rc;
  rc = make_tables(p, &tb);
  if (rc) return rc;
  N = (int64_t)p->grid_w * p->grid_h * p->n_per_col;
  DR = p->d_max + 1;
  if (p->connectivity == CONN_PAPER) {
    prow = (orc_syn *)malloc(sizeof(orc_syn) * (size_t)paper_candidates(p, &tb));
    if (!prow) rc = ORC_ENOMEM;
  }
  ref = (uint8_t *)calloc((size_t)N, 1);
  fired = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (mode == ORC_MODE_F64) {
    R64 = (double *)calloc((size_t)N * DR, sizeof(double));
    V64 = (double *)malloc(sizeof(double) * (size_t)N);
    C64 = (double *)calloc((size_t)N, sizeof(double));
    if (!R64 || !V64 || !C64) rc = ORC_ENOMEM;
  } else {
    R32 = (int32_t *)calloc((size_t)N * DR, sizeof(int32_t));
    V32 = (float *)malloc(sizeof(float) * (size_t)N);
    C32 = (float *)calloc((size_t)N, sizeof(float));
    if (!R32 || !V32 || !C32) rc = ORC_ENOMEM;
  }
  if (!ref || !fired) rc = ORC_ENOMEM;
  if (rc) goto done;

  pvv32 = (float)tb.pvv;
  pcc32 = (float)tb.pcc;
  pvc32[0] = (float)tb.pvc[0];
  pvc32[1] = (float)tb.pvc[1];
  for (i = 0; i < N; ++i) {
    uint32_t u = init_word(p->seed, i);
    if (mode == ORC_MODE_F64)
      V64[i] = (double)p->theta * ((double)(u >> 8) * 5.9604644775390625e-08);
    else
      V32[i] = p->theta * ((float)(u >> 8) * 5.9604644775390625e-08f);
  }

  for (t = 0; t < n_steps; ++t) {
    int slot = (int)(t % DR);
    int64_t nf = 0, kext = 0;
    /* neuron updates read and clear this step's slot */
    for (i = 0; i < N; ++i) {
      int pop = (int)(i % p->n_per_col) < p->n_exc ? 0 : 1;
      int k = poisson_k(&tb, ext_word(p->seed, i, t));
      int spk;
      kext += k;
      if (mode == ORC_MODE_F64) {
        double I = R64[(size_t)slot * N + i] + (double)k * (double)p->j_ext;
        R64[(size_t)slot * N + i] = 0.0;
        spk = step_f64(&V64[i], &C64[i], &ref[i], I, (double)p->theta,
                       (double)p->v_reset, (double)p->dc, tb.nref, tb.pvv,
                       tb.pvc[pop], tb.pcc);
      } else {
        int32_t I = R32[(size_t)slot * N + i] + k * tb.jx;
        R32[(size_t)slot * N + i] = 0;
        spk = step_f32(&V32[i], &C32[i], &ref[i], I, p->theta, p->v_reset,
                       p->dc, tb.nref, pvv32, pvc32[pop], pcc32);
      }
      if (spk) fired[nf++] = (int32_t)i;
    }
    /* every spike travels through its synapses into slot t + d */
    for (i = 0; i < nf; ++i) {
      int64_t k, cnt = p->k_out;
      if (prow) cnt = paper_row(p, &tb, mode, fired[i], prow);
      for (k = 0; k < cnt; ++k) {
        orc_syn s;
        int ds;
        if (prow)
          s = prow[k];
        else
          synapse(p, &tb, mode, fired[i], (int32_t)k, &s);
        ds = (int)((t + s.delay) % DR);
        if (mode == ORC_MODE_F64)
          R64[(size_t)ds * N + s.target] += s.w;
        else
          R32[(size_t)ds * N + s.target] += s.wfx;
      }
      if (ns < cap) {
        if (spk_t) spk_t[ns] = (int32_t)t;
        if (spk_i) spk_i[ns] = fired[i];
      }
      ++ns;
    }
    if (step_spikes) step_spikes[t] = nf;
    if (step_ext) step_ext[t] = kext;
  }
  if (n_spk) *n_spk = ns;
  for (i = 0; i < N; ++i) {
    if (v_end) v_end[i] = mode == ORC_MODE_F64 ? V64[i] : (double)V32[i];
    if (c_end) c_end[i] = mode == ORC_MODE_F64 ? C64[i] : (double)C32[i];
    if (r_end) r_end[i] = ref[i];
  }
done:
  free(R32); free(R64); free(V32); free(V64); free(C32); free(C64);
  free(ref); free(fired); free(prow);
  free_tables(&tb);
  return rc;
}
