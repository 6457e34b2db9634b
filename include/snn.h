/*
 * snn.h -- C ABI of the GB300 spiking cortical-column simulator.
 *
 * The model is the one measured in arxiv 1511.09325 (Sec. 2, "Methods"): a
 * 2-D grid of cortical columns, each holding n_per_col point neurons (1240 in
 * the paper, 80 % excitatory), leaky integrate-and-fire with spike-frequency
 * adaptation (a calcium-driven after-hyperpolarisation current), about 1240
 * outgoing synapses per neuron split between the own column and nearby columns
 * with a probability decreasing with distance, plus external excitatory input,
 * with synaptic plasticity disabled.  The simulator advances it in 1 ms steps,
 * mixing time-driven stepping with event-driven spike delivery (Sec. 1).
 *
 * One step, as this library computes it:
 *   1. every neuron i reads its input for step t (recurrent, in int32 units of
 *      2^-16 mV, plus k_i(t) * J_ext with k_i(t) ~ Poisson(nu_ext * 1 ms) drawn
 *      from Philox4x32-10 keyed on (seed, i, t)), integrates it, fires when
 *      V >= theta (reset to V_reset, refractory for t_ref, calcium += dc) and
 *      advances V and calcium by the exact 1 ms propagator of
 *      dV/dt = -V/tau_m - g_c c, dc/dt = -c/tau_c;
 *   2. every spike emitted in the last d_max steps delivers, through the
 *      synapses of the matching axonal delay, its fixed-point weights into the
 *      input of step t + 1 (integer atomics: the sum is order-independent).
 * The fixed-point/FP32 arithmetic is bit-identical to the CPU oracle of this
 * project; see the reading of each formula in the project's design notes.
 *
 * Conventions for every call:
 *   - returns an int status (SNN_OK = 0, negative on error); no C++ exception
 *     crosses the ABI; snn_last_error() gives a message for the last failure;
 *   - the library owns every device allocation of a net; the caller owns the
 *     host buffers it passes and must size them as stated;
 *   - calls on one net are not thread-safe; different nets are independent;
 *   - device work is enqueued on the net's stream (the caller's, if given);
 *     snn_read_* and snn_stats synchronise that stream.
 */
#ifndef SNN_GB300_H
#define SNN_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snn_net snn_net; /* opaque, library-owned */

/* Neuron model (Sec. 2: LIF with SFA; 1240 neurons per column, 80 % E).
 * Units: ms, mV, mV/ms; rates in kHz. */
typedef struct {
  int32_t n_per_col; /* neurons per column, 2..2048 (1240)                */
  int32_t n_exc;     /* excitatory neurons per column, first in the column */
  float tau_m;       /* membrane time constant (20 ms)                     */
  float theta;       /* firing threshold (20 mV)                           */
  float v_reset;     /* reset potential (15 mV)                            */
  float t_ref;       /* refractory period, rounded to whole steps (2 ms)   */
  float tau_c;       /* calcium time constant (500 ms)                     */
  float dc;          /* calcium increment per spike (1)                    */
  float gc_exc;      /* adaptation gain of E neurons (0.02 mV/ms)          */
  float gc_inh;      /* adaptation gain of I neurons (0)                   */
  float j_ext_mV;    /* efficacy of one external event (0.4 mV)            */
  float nu_ext_kHz;  /* external Poisson rate per neuron (2.5 kHz)         */
} snn_neuron_params;

/* Connectivity (Sec. 2: local plus distance-dependent remote synapses).
 * Two laws:
 *   SNN_CONN_FIXED: exactly k_out synapses per neuron; the first
 *     round(frac_local k_out) go to other neurons of the own column, the rest
 *     to columns of the (2 radius + 1)^2 stencil with P ~ exp(-r / lambda);
 *   SNN_CONN_PAPER: the law stated in Sec. 2: a synapse to every other neuron
 *     of the own column with probability p_local, and to every neuron of a
 *     column at Euclidean grid distance r with probability
 *     remote_a exp(-r^2 / (2 remote_sigma^2)), offsets where that is below
 *     remote_cutoff being dropped (they must all lie within the 7x7
 *     stencil); the out-degree varies from neuron to neuron (k_out,
 *     frac_local, lambda_cols and stencil_radius are then unused).
 * Delays and weights follow the same rules under both laws. */
enum { SNN_CONN_FIXED = 0, SNN_CONN_PAPER = 1 };
typedef struct {
  int32_t k_out;          /* outgoing synapses per neuron (1240)            */
  float frac_local;       /* fraction inside the own column (0.5)           */
  float lambda_cols;      /* remote P ~ exp(-r / lambda), r in grid steps   */
  int32_t stencil_radius; /* remote cut-off |dx|,|dy| <= radius, 1..3 (3)   */
  float w_exc_mV;         /* mean weight of E synapses (0.4 mV)             */
  float w_inh_mV;         /* mean weight of I synapses (-1.6 mV)            */
  float w_cv;             /* coefficient of variation of weights (0.25)     */
  int32_t d_min, d_max;   /* axonal delays, whole steps, 1 <= d_min <= d_max <= 32 */
  int32_t periodic;       /* must be 1: the grid is a torus                  */
  int32_t connectivity;   /* SNN_CONN_FIXED or SNN_CONN_PAPER               */
  float p_local;          /* paper law: own-column probability (0.8)        */
  float remote_a;         /* paper law: amplitude of the remote law (0.05)  */
  float remote_sigma;     /* paper law: its width, grid steps (1)           */
  float remote_cutoff;    /* paper law: smallest kept probability (0.001)   */
} snn_synapse_params;

enum {
  SNN_OK = 0,
  SNN_EINVAL = -1,    /* bad argument or parameter                          */
  SNN_ENOMEM = -2,    /* device or host allocation failed                   */
  SNN_ECUDA = -3,     /* a CUDA call failed (message in snn_last_error)     */
  SNN_EOVERFLOW = -4, /* spike records were dropped (counters stay exact)   */
  SNN_ETIMEOUT = -5,  /* a bounded device wait gave up                      */
  SNN_ESTATE = -6     /* call not valid in the net's current state          */
};

/* Weight storage of the outgoing-synapse table. */
enum {
  SNN_EXACT_F32W = 0, /* 8 B/synapse: target index + FP32 weight (2^-16 mV) */
  SNN_EXACT_F16W = 1  /* 4 B/synapse: packed target + FP16 weight magnitude  */
};

/*
 * snn_build -- construct a grid_w x grid_h network on the current device.
 * Sec. 2: grid of columns, n_per_col neurons each, k_out outgoing synapses.
 * seed keys every random draw (connectivity, initial V, external input).
 * precision is SNN_EXACT_F32W or SNN_EXACT_F16W.  cuda_stream is a
 * cudaStream_t (NULL: the library creates a non-blocking stream of its own).
 * On success *out receives the net (destroy with snn_destroy).  Returns
 * SNN_EINVAL for parameters outside the stated ranges, SNN_ENOMEM when the
 * synapse table does not fit, SNN_ECUDA on a CUDA error.
 */
int snn_build(int grid_w, int grid_h, const snn_neuron_params* neuron,
              const snn_synapse_params* synapse, uint64_t seed, int precision,
              void* cuda_stream, snn_net** out);

/*
 * snn_step -- advance n_steps 1 ms steps (Sec. 1: fixed network step, spikes
 * delivered event by event).  Asynchronous on the net's stream: the steps run
 * as replays of a captured CUDA graph.  n_steps >= 0.  A delivery that finds
 * its item counts disagreeing with the step's spike lists delivers nothing
 * for the disagreeing part and sets the net's status word; from then on
 * snn_step, snn_read_spikes, snn_read_rates and snn_stats return SNN_ESTATE
 * (snn_step as soon as the status has reached the host, the reads after
 * their synchronisation), and the net should be destroyed.
 */
int snn_step(snn_net* net, int64_t n_steps);

/*
 * snn_read_spikes -- drain the spike records kept since the last drain.
 * Writes up to cap pairs (steps[k], ids[k]) in step order (order within a
 * step unspecified) and *n_out = pairs written.  ids are global neuron
 * indices i = (y * grid_w + x) * n_per_col + l.  Returns SNN_EOVERFLOW if the
 * device record buffer or cap was too small; the records beyond it are lost,
 * the counters of snn_read_rates / snn_stats are not affected.
 */
int snn_read_spikes(snn_net* net, int32_t* steps, int32_t* ids, int64_t cap,
                    int64_t* n_out);

/* snn_pending_spikes -- number of records a drain would return now. */
int snn_pending_spikes(snn_net* net, int64_t* n_out);

/* snn_set_record_capacity -- resize the device spike-record buffer (records,
 * 8 B each; the default is 2^24).  Drops the pending records. */
int snn_set_record_capacity(snn_net* net, int64_t capacity);

/*
 * snn_read_rates -- firing rates over the steps since the last call.
 * hz[2 * c + p] = rate (Hz) of population p (0 = E, 1 = I) of column
 * c = y * grid_w + x; n must be >= 2 * grid_w * grid_h (hz may be NULL).
 * pop_hz[2] (may be NULL) receives the grid-wide E and I rates.
 */
int snn_read_rates(snn_net* net, float* hz, int64_t n, float* pop_hz);

/*
 * snn_stats -- totals since snn_build: recurrent synaptic events (spikes x
 * k_out), external events (sum of the Poisson counts; the paper counts both,
 * Sec. 3), and steps simulated.  Any pointer may be NULL.
 */
int snn_stats(snn_net* net, double* recurrent_events, double* external_events,
              int64_t* steps);

/*
 * snn_get_state -- copy the neuron state to host arrays of N floats / bytes:
 * membrane potential (mV), calcium, remaining refractory steps.  N = number
 * of neurons.  Any pointer may be NULL.
 */
int snn_get_state(snn_net* net, float* v, float* c, uint8_t* refractory);

/*
 * snn_read_synapses -- decode the outgoing synapses of neurons j0..j0+n-1 from
 * the device table into host arrays, grouped by neuron (neuron j0's first),
 * within a neuron by delay: target neuron, delay (steps), weight in 2^-16 mV.
 * The arrays hold the sum of the rows' lengths (snn_row_lengths): n * k_out
 * entries under SNN_CONN_FIXED.
 */
int snn_read_synapses(snn_net* net, int64_t j0, int64_t n, int64_t* target,
                      int32_t* delay, int32_t* wfx);

/* snn_row_lengths -- counts[r] = outgoing synapses of neuron j0 + r, r < n. */
int snn_row_lengths(snn_net* net, int64_t j0, int64_t n, int32_t* counts);

/*
 * snn_debug_offset_count -- testing aid with no counterpart in the paper: adds
 * delta to the number of delivery items the library has counted for `column`
 * (0 <= column < grid_w * grid_h) and to the count of its group of 32
 * columns, or to the group count only when group_only is nonzero, as a
 * bookkeeping fault would.  The spike lists are left as they are, so the next
 * delivery finds counts that disagree with them and must set the net's status
 * word (see snn_step).  Synchronises the net's stream.  SNN_EINVAL for a
 * column out of range.
 */
int snn_debug_offset_count(snn_net* net, int64_t column, int32_t delta, int32_t group_only);

/*
 * snn_info -- sizes of the net: info[0] = N neurons, [1] = synapses,
 * [2] = device bytes held, [3] = bytes of the synapse table, [4] = row
 * capacity in synapse slots, [5] = precision, [6] = side of the delivery
 * tiles in columns, [7] = delivery blocks, [8] = update blocks.  n = entries
 * available (at most 9 are written).
 */
int snn_info(snn_net* net, int64_t* info, int n);

/*
 * Column-tile shards.  The paper distributes the grid's columns over MPI
 * processes that exchange the step's spikes every step (Sec. 2, Sec. 3).  A
 * shard is the part of the network one process (one GPU) holds: the columns
 * of its tile [x0, x0 + w) x [y0, y0 + h) of the grid_w x grid_h grid, and
 * the rows of the neurons within stencil_radius columns of it (the halo,
 * periodic), restricted to the synapses that end in the tile.  Every random
 * draw uses global neuron indices, so the shards of a partition of the grid,
 * stepped together, compute exactly the raster and states of the whole
 * network built by snn_build with the same parameters and seed.
 *
 * A step of a shard has two halves.  snn_shard_update runs the neuron update
 * of the tile's columns for step t; snn_read_spikes then returns the tile's
 * spikes of step t (global indices).  The caller exchanges them among the
 * shards (any transport: every shard may receive every shard's spikes) and
 * passes the received indices to snn_shard_deliver, which lists those of the
 * halo's columns and delivers all spikes due at step t into the tile's input
 * of step t + 1.  Because d_min >= 1, one exchange per step suffices.
 */

/*
 * snn_build_shard -- build the shard of tile (x0, y0, w, h) of a grid_w x
 * grid_h network; the other arguments as for snn_build.  The local grid is
 * the tile plus a halo of stencil_radius columns on each side, or the whole
 * grid side where tile and halo would cover it.  Requires SNN_CONN_FIXED and
 * n_per_col a multiple of 4 (SNN_EINVAL otherwise, and for a tile outside the
 * grid).  On a shard, snn_get_state, snn_read_rates, snn_read_synapses,
 * snn_row_lengths and snn_debug_offset_count index the local grid (columns
 * c = ly * local_w + lx, neurons c * n_per_col + l; snn_shard_info gives the
 * mapping; a row holds only the synapses that end in the tile, F32W targets
 * as local indices); snn_read_spikes returns global indices; snn_read_rates'
 * population rates average over the tile's columns; snn_stats counts k_out
 * synaptic events per tile spike.  snn_step, snn_step_profiled and
 * snn_grad_build refuse a shard.
 */
int snn_build_shard(int grid_w, int grid_h, int x0, int y0, int w, int h,
                    const snn_neuron_params* neuron, const snn_synapse_params* synapse,
                    uint64_t seed, int precision, void* cuda_stream, snn_net** out);

/*
 * snn_shard_update -- first half of the shard's next step t: the neuron
 * update of the tile's columns (asynchronous on the net's stream).
 * SNN_ESTATE if the previous step's snn_shard_deliver has not been called,
 * for a net that is not a shard, or when the status word is set.
 */
int snn_shard_update(snn_net* net);

/*
 * snn_shard_deliver -- second half of step t: ids[0 .. n) are global indices
 * of neurons that fired at step t, each at most once (the spikes of the other
 * shards; indices of the own tile and of columns beyond the halo are
 * ignored).  ids is host memory when ids_on_device is 0 (the library copies
 * it before returning: the buffer may be reused at once), else device memory
 * that must stay unchanged until the net's stream has passed the call.
 * Lists the halo's spikes and
 * runs the step's delivery; the step counter then advances.  An index beyond
 * the network or more than n_per_col indices of one column set the status
 * word (SNN_ESTATE from the next call that checks it).  SNN_ESTATE when
 * snn_shard_update is due first.
 */
int snn_shard_deliver(snn_net* net, const int32_t* ids, int64_t n, int32_t ids_on_device);

/*
 * snn_shard_info -- geometry of a shard: geo[0..9] = grid_w, grid_h, local_w,
 * local_h, ex0, ey0, tx0, ty0, w, h: local column (lx, ly) is global column
 * ((ex0 + lx) mod grid_w, (ey0 + ly) mod grid_h); the tile is local columns
 * [tx0, tx0 + w) x [ty0, ty0 + h).  n = entries available (at most 10).
 * SNN_ESTATE for a net that is not a shard.
 */
int snn_shard_info(snn_net* net, int32_t* geo, int n);

/*
 * snn_shard_geometry -- the geometry snn_build_shard gives the shard of tile
 * (x0, y0, w, h) of a grid_w x grid_h grid with the given stencil_radius
 * (1..3), in the layout of snn_shard_info, without building anything (host
 * only, no device call).  SNN_EINVAL for a grid outside 1..16383 columns a
 * side, a tile outside the grid, a radius outside 1..3 or a NULL geo.
 */
int snn_shard_geometry(int grid_w, int grid_h, int x0, int y0, int w, int h, int stencil_radius,
                       int32_t* geo, int n);

/*
 * snn_step_profiled -- like snn_step, but each step's kernels are launched
 * one by one with CUDA events around each on the net's stream.  Writes the
 * summed device milliseconds of the neuron-update and delivery kernels and,
 * in bytes[2], their algorithmic bytes (see the design notes) over the
 * n_steps.  Synchronises the stream.  For measurement only.
 */
int snn_step_profiled(snn_net* net, int64_t n_steps, double* ms, double* bytes);

/*
 * snn_update_noalloc -- one neuron-update step on buffers the caller owns,
 * allocating nothing.  The paper has no counterpart: this entry point exists
 * for callers that cannot let a library call cudaMalloc -- a process whose
 * device memory is already reserved by another framework's allocator or a
 * fixed arena, or a real-time loop that cannot afford an allocation's
 * implicit synchronisation.
 *
 * It runs the same update kernel as snn_step for step `step` of a
 * grid_w x grid_h network of N = grid_w * grid_h * n_per_col neurons (the
 * external Poisson input is keyed on (seed, neuron, step), so the result
 * equals snn_step's update of that step given the same state and input).
 * Device buffers, each of at least ceil(N / 4) * 4 elements (the kernel reads
 * and writes whole groups of 4 neurons):
 *   v, c          float, 16-byte aligned: membrane potential and calcium, in/out;
 *   refractory    u8, 4-byte aligned: remaining refractory steps, in/out;
 *   input         int32, 16-byte aligned: recurrent input of this step in
 *                 2^-16 mV units, read and then cleared to zero;
 *   spikes        u32[N], 4-byte aligned: receives the indices of the
 *                 neurons that fired;
 *   col_counts    u64[2 * columns], 8-byte aligned, or NULL: spikes per
 *                 column (E, I).
 * Host outputs: *n_spikes (entries written to spikes), *ext_events (sum of
 * the external Poisson counts; may be NULL).  Synchronises cuda_stream
 * (a cudaStream_t; NULL is the legacy default stream).
 *
 * Its scratch is one fixed device array of 311 808 bytes inside the library
 * (held on every GPU that loads the library until the process exits), which
 * limits a call to 16 384 columns (SNN_EINVAL beyond).  Every call shares that
 * array and clears what it needs at its start, so calls whose GPU work
 * overlaps (on different streams or threads) race and must be serialised by
 * the caller.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress) and keeps it for the life of the process;
 * make that first call before any stream capture begins, and do not reset
 * the device (cudaDeviceReset) between calls, which would invalidate the kept
 * address.  Returns SNN_EINVAL for bad parameters, sizes or alignment,
 * SNN_ECUDA for a CUDA error (message in snn_last_error(NULL)).
 */
int snn_update_noalloc(int grid_w, int grid_h, const snn_neuron_params* neuron,
                       uint64_t seed, int64_t step, float* v, float* c,
                       uint8_t* refractory, int32_t* input, uint32_t* spikes,
                       int64_t* n_spikes, int64_t* ext_events,
                       unsigned long long* col_counts, void* cuda_stream);

/*
 * Batched form: many independent nets advanced together by one persistent
 * launch.  The paper runs one network on many processes (Sec. 2); a batch is
 * the other way round -- seed sweeps or stimulus sweeps of small networks that
 * alone would leave most of the GPU idle.  Every member computes exactly what
 * it computes alone (same kernels' blocks, bit-identical rasters).
 */
typedef struct snn_batch snn_batch; /* opaque, library-owned */

/*
 * snn_batch_build -- n_nets (1..256) nets on the current device: net k is a
 * grid_w[k] x grid_h[k] grid with neuron[k], synapse[k] and seeds[k] (as in
 * snn_build); all nets use `precision`.  Members are owned by the batch and
 * share its stream (cuda_stream, or a stream of its own when NULL).
 */
int snn_batch_build(int n_nets, const int32_t* grid_w, const int32_t* grid_h,
                    const snn_neuron_params* neuron, const snn_synapse_params* synapse,
                    const uint64_t* seeds, int precision, void* cuda_stream,
                    snn_batch** out);

/*
 * snn_batch_step -- advance every member n_steps steps in one cooperative
 * launch: each step runs all members' update blocks, a grid barrier, all
 * members' delivery blocks and a second barrier.  Barrier waits are bounded;
 * a wait that gives up ends the launch and the call returns SNN_ETIMEOUT (the
 * members' state is then undefined).  Synchronises the batch's stream.
 */
int snn_batch_step(snn_batch* batch, int64_t n_steps);

/* snn_batch_net -- member k, for snn_read_spikes / snn_read_rates /
 * snn_stats / snn_get_state / snn_read_synapses / snn_info (snn_step and
 * snn_step_profiled refuse a member with SNN_ESTATE).  NULL if k is out of
 * range.  The member stays owned by the batch. */
snn_net* snn_batch_net(snn_batch* batch, int k);

/*
 * snn_batch_tune -- pick the fastest delivery schedule for this batch (rounds
 * of 32-byte sectors in flight per lane: 2 or 1, i.e. 4 or 2 chunks of 16
 * bytes; shared-memory windows: on or off), then
 * the fastest delivery density (8, 4, 2 or 1 virtual delivery blocks per
 * member column, at most the member's standalone grid), each by timing two
 * interleaved rounds of steps_per_trial steps of every candidate (16 trials
 * in all).  The trial steps advance the simulation (every candidate computes
 * identical sums).  *choice (may be NULL) receives the pick, schedule (0..3)
 * + 4 x density index (0..3).
 */
int snn_batch_tune(snn_batch* batch, int64_t steps_per_trial, int32_t* choice);

/* snn_batch_set_wait -- barrier wait bound (polls of ~64 ns, default 2^25)
 * and, for tests of the timeout path only, arrivals the barrier waits for
 * beyond the launched grid (default 0). */
int snn_batch_set_wait(snn_batch* batch, int64_t spin_limit, int32_t extra_arrivals);

/* snn_batch_last_error -- message of the last failure on batch (thread-local
 * when batch is NULL). */
const char* snn_batch_last_error(const snn_batch* batch);

/* snn_batch_destroy -- free the batch and its members; NULL is a no-op. */
void snn_batch_destroy(snn_batch* batch);

/*
 * Differentiable form (surrogate gradient).  The paper simulates the spiking
 * network only (Sec. 2); this is the standard surrogate-gradient extension of
 * the same recursion, on the net's own synapse table, with respect to six
 * parameters theta = {a_EE, a_EI, a_IE, a_II, g_c, nu_ext}: a_XY multiplies
 * every synaptic weight from population X onto population Y (1 = the net as
 * built), g_c replaces the excitatory adaptation strength (mV/ms) and nu_ext
 * (kHz) the external rate.  The external input becomes its Gaussian form
 * J (lam + sqrt(lam) xi), lam = nu_ext * 1 ms, xi a normal draw of Philox
 * stream 4 (key = the net's seed, counter (i/4, t, 4, 0), word i mod 4, mapped
 * through the 65536-entry normal quantile table), so that nu_ext has a
 * pathwise derivative.  Per step, neuron i of population p:
 *   I = a[E][p] X_E + a[I][p] X_I + J (lam + sqrt(lam) xi)     (X_P: input
 *       from sources of population P, each synapse weighted by s_j(t - d))
 *   g = max(0, 1 - s(t-1) - s(t-2)),  U = g (V + I) + (1 - g) V_reset
 *   s = [U >= theta] (hard = 1) or sigmoid(beta (U - theta)) (hard = 0)
 *   V' = U - s (U - V_reset),  c' = c + dc s,
 *   V <- P_VV V' + P_VC c',  c <- P_CC c'
 * from the net's initial potentials (c = 0), for n_steps steps.  The loss is
 * (r_E - r_E*)^2 + (r_I - r_I*)^2 with r_P = 1000 * mean of s over
 * population P and all steps (Hz).  Hard mode differentiates with the
 * surrogate ds/dU = 1 / (1 + beta |U - theta|)^2 (the spikes are exactly those
 * of the threshold rule); soft mode with the exact derivative.
 *
 * snn_grad_build -- a differentiable view of `net` (which must be
 * SNN_EXACT_F32W and outlive the view).  checkpoint_every: steps between
 * stored states; the backward pass recomputes each segment from its
 * checkpoint (device memory ~ N * (8 * checkpoint_every + 23 * n_steps /
 * checkpoint_every) floats).  target_rates (Hz, E then I) may be NULL for
 * (3, 8).  Runs on the net's stream.
 */
typedef struct snn_grad snn_grad; /* opaque, library-owned */
int snn_grad_build(snn_net* net, int64_t n_steps, int32_t checkpoint_every, int32_t hard,
                   float beta, const double* target_rates, snn_grad** out);

/*
 * snn_grad_run -- forward pass for theta[6] (host doubles): *loss and, when
 * not NULL, rates[2] (Hz).  When grad is not NULL also the backward pass:
 * grad[6] = d loss / d theta.  Deterministic: every reduction has a fixed
 * order.  Synchronises the net's stream.  SNN_EINVAL for a NULL loss or
 * theta, non-finite parameters or nu_ext <= 0.
 */
int snn_grad_run(snn_grad* g, const double* theta, double* loss, double* rates, double* grad);

/* snn_grad_last_error -- message of the last failure on g ("" if none). */
const char* snn_grad_last_error(const snn_grad* g);

/* snn_grad_destroy -- free the view (not the net); NULL is a no-op. */
void snn_grad_destroy(snn_grad* g);

/* snn_last_error -- message of the last failure on net (thread-local when net
 * is NULL).  Never NULL; valid until the next call on the same net. */
const char* snn_last_error(const snn_net* net);

/* snn_destroy -- free every resource of the net; NULL is a no-op. */
void snn_destroy(snn_net* net);

#ifdef __cplusplus
}
#endif

#endif /* SNN_GB300_H */
