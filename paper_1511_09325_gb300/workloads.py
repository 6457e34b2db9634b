"""Seeded synthetic workloads: grid sizes, model parameters and seeds.

This module holds only the *inputs* of a simulation (numbers a user would
type in), none of the model's arithmetic.  Both the CUDA library binding and
the CPU oracle consume these dictionaries.

The defaults follow arxiv 1511.09325, Sec. 2: columns of 1240 LIF neurons with
spike-frequency adaptation, 80 % excitatory (992) and 20 % inhibitory (248),
about 1240 outgoing synapses per neuron, part local and part projected to
nearby columns of a 2-D grid, plus external excitatory input.  The paper leaves
time constants, weights, delays and the external rate unstated; the values
below are the ones this implementation adopts (LIF + calcium SFA with
tau_m = 20 ms, theta = 20 mV, V_reset = 15 mV, 2 ms refractory period,
tau_c = 500 ms, calcium step 1, g_c = 0.02 mV/ms for excitatory neurons,
external Poisson input 2.5 kHz x 0.4 mV, weights N(0.4, 0.25 cv) mV for
excitatory and N(-1.6, 0.25 cv) mV for inhibitory sources, integer delays
uniform in 1..20 ms, half of the synapses local and the other half spread
over a 7x7 stencil with probability proportional to exp(-d / 1.5)).
"""

NEURON = dict(
    n_per_col=1240,
    n_exc=992,
    tau_m=20.0,
    theta=20.0,
    v_reset=15.0,
    t_ref=2.0,
    tau_c=500.0,
    dc=1.0,
    gc_exc=0.02,
    gc_inh=0.0,
    j_ext_mV=0.4,
    nu_ext_kHz=2.5,
)

SYNAPSE = dict(
    k_out=1240,
    frac_local=0.5,
    lambda_cols=1.5,
    stencil_radius=3,
    w_exc_mV=0.4,
    w_inh_mV=-1.6,
    w_cv=0.25,
    d_min=1,
    d_max=20,
    periodic=1,
    # 0: the law above; 1: Sec. 2's own law (Bernoulli p_local inside the
    # column, remote_a exp(-r^2 / 2 remote_sigma^2) to each neuron of a column
    # at distance r, offsets below remote_cutoff dropped; variable out-degree)
    connectivity=0,
    p_local=0.8,
    remote_a=0.05,
    remote_sigma=1.0,
    remote_cutoff=0.001,
)

# Named workloads.  "steps" is the simulated length in 1 ms steps.
WORKLOADS = {
    # 2x2 columns, 4960 neurons, 6.15 M synapses: the parity case.
    "cols2x2_f32w": dict(grid_w=2, grid_h=2, seed=1, precision="f32w", steps=1000),
    # 12x12 columns, 178 560 neurons, 221.4 M synapses: a profiling-size case.
    "cols12x12_f32w": dict(grid_w=12, grid_h=12, seed=2, precision="f32w", steps=1000),
    "cols12x12_f16w": dict(grid_w=12, grid_h=12, seed=2, precision="f16w", steps=1000),
    # 24x24 columns, 714 240 neurons, 885.7 M synapses (Sec. 2, Table 1).
    "cols24x24_f32w": dict(grid_w=24, grid_h=24, seed=2, precision="f32w", steps=10000),
    "cols24x24_f16w": dict(grid_w=24, grid_h=24, seed=2, precision="f16w", steps=10000),
    # 48x48 columns, 2.86 M neurons, 3.54 G synapses (Table 1).
    "cols48x48_f32w": dict(grid_w=48, grid_h=48, seed=3, precision="f32w", steps=10000),
    "cols48x48_f16w": dict(grid_w=48, grid_h=48, seed=3, precision="f16w", steps=10000),
    # 96x96 columns, 11.43 M neurons, 14.17 G synapses (Table 1).
    "cols96x96_f16w": dict(grid_w=96, grid_h=96, seed=3, precision="f16w", steps=10000),
    "cols96x96_f32w": dict(grid_w=96, grid_h=96, seed=3, precision="f32w", steps=10000),
    # Sec. 2's own connectivity law (variable out-degree, ~1307 synapses).
    "cols2x2_paper_f32w": dict(grid_w=2, grid_h=2, seed=1, precision="f32w", steps=300,
                               synapse=dict(connectivity=1)),
    "cols24x24_paper_f32w": dict(grid_w=24, grid_h=24, seed=2, precision="f32w", steps=2000,
                                 synapse=dict(connectivity=1)),
    # 4x4 columns: the size used for the single-column-neighbourhood tests.
    "cols4x4_f32w": dict(grid_w=4, grid_h=4, seed=5, precision="f32w", steps=500),
}


def neuron_params(**overrides):
    """Neuron parameters with optional overrides (a new dict)."""
    p = dict(NEURON)
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return p


def synapse_params(**overrides):
    """Synapse parameters with optional overrides (a new dict)."""
    p = dict(SYNAPSE)
    for k, v in overrides.items():
        if k not in p:
            raise KeyError(k)
        p[k] = v
    return p


def n_neurons(grid_w, grid_h, n_per_col=NEURON["n_per_col"]):
    return grid_w * grid_h * n_per_col


def batch_workload(n_nets=64, seed0=100):
    """The batched form: n_nets independent networks of the default
    construction, grid sizes drawn uniformly from 1x1 to 8x8 columns (numpy
    generator seeded with 1511), seeds seed0 .. seed0 + n_nets - 1, external
    rates swept linearly over 1.5-3.5 kHz.  Returns (grids, neurons, synapses,
    seeds)."""
    import numpy as np

    rng = np.random.default_rng(1511)
    grids = [(int(a), int(b)) for a, b in rng.integers(1, 9, size=(n_nets, 2))]
    rates = [1.5 + 2.0 * k / max(n_nets - 1, 1) for k in range(n_nets)]
    neurons = [neuron_params(nu_ext_kHz=r) for r in rates]
    synapses = [synapse_params() for _ in range(n_nets)]
    seeds = [seed0 + k for k in range(n_nets)]
    return grids, neurons, synapses, seeds
