/*
 * psst.h -- C interface of the GB300 (sm_103a) library for fixed-step RK4
 * integration of networks of coupled Hodgkin-Huxley neurons with kinetic
 * synapses (Mohanta & Assisi, "Parallel scalable simulations of biological
 * neural networks using TensorFlow", arXiv:1906.03958).
 *
 * The problem statement follows the paper:
 *   - the initial value problem dy/dt = f(y, t), y(t0) = y0 (Eq. ode), with y
 *     the vectorised state X' = [V, m, h, n] of Sec. "Brain simulations as
 *     computational graphs" plus the synaptic variables;
 *   - the recursion X_{i+1} = F(X_i, t_i, eps_i) over a time grid with F the
 *     fourth-order Runge-Kutta step (same section, RK4 paragraph);
 *   - synaptic variables stored sparsely, only for existing synapses
 *     (Sec. "Circumventing memory constraints", item 1);
 *   - a long simulation split into successive calls that continue from the
 *     device-resident state (same section, item 2).
 *
 * Conventions for every function:
 *   - return 0 (PSST_OK) or a negative PSST_ERR_* code; nothing throws
 *     across this interface; psst_last_error() gives a message for the last
 *     failing call on the calling thread;
 *   - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is stream-ordered and asynchronous unless the
 *     function says it synchronises;
 *   - a handle is not thread-safe: one thread at a time per handle;
 *   - all host arrays in psst_network_desc are read during
 *     psst_create_network only; the caller keeps ownership.
 */
#ifndef PSST_H
#define PSST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSST_OK 0
#define PSST_ERR_INVALID_ARG (-1)  /* bad size, index, pointer or parameter */
#define PSST_ERR_OOM (-2)          /* device allocation failed */
#define PSST_ERR_CUDA (-3)         /* a CUDA runtime call failed */
#define PSST_ERR_NONFINITE (-4)    /* the state became NaN/Inf (device check) */
#define PSST_ERR_TIMEOUT (-5)      /* a bounded device-wide wait gave up */
#define PSST_ERR_STATE (-6)        /* call not valid in the handle's state */
#define PSST_ERR_UNSUPPORTED (-7)  /* network shape outside what a mode handles */

/* Columns of the neuron-type table (row per type), units mV, ms, uA/cm^2,
   mS/cm^2, uF/cm^2:  C, gNa, gK, gL, ENa, EK, EL, gKL, EKL.
   dV/dt = (I_ext - gNa m^3 h (V-ENa) - gK n^4 (V-EK) - gL (V-EL)
            - gKL (V-EKL) - I_syn) / C, with the squid-axon rate functions
   (-65 mV convention) for m, h, n. */
#define PSST_NEURON_NPARAM 9
/* Columns of the synapse-type table (row per type):
   kind, a, b, K3, K4, Kd, E, Vp, Kp.
   T = 1/(1+exp(-(V_pre-Vp)/Kp));
   kind 0: dr/dt = a T (1-r) - b r,                         G = r;
   kind 1: dr/dt = a T (1-r) - b r,  ds/dt = K3 r - K4 s,   G = s^4/(s^4+Kd);
   current into the postsynaptic neuron: w G (V_post - E). */
#define PSST_SYN_NPARAM 9
#define PSST_MAX_SYN_TYPES 8

/* Integration methods (Sec. "Brain simulations as computational graphs":
   Euler's method, Eq. euler, and the fourth-order Runge-Kutta method). */
#define PSST_METHOD_RK4 0    /* classic RK4 (c = 0, 1/2, 1/2, 1; b = 1/6, 1/3, 1/3, 1/6) */
#define PSST_METHOD_EULER 1  /* forward Euler: y_{n+1} = y_n + dt f(y_n, t_n) */
#define PSST_METHOD_TABLEAU 2 /* explicit Runge-Kutta map of the family both methods belong to, given by
                                 rk_stages, rk_a and rk_b: Y_1 = y, Y_s = y + dt a_s k_{s-1},
                                 k_s = f(Y_s), y_{n+1} = y + dt sum_s b_s k_s (e.g. midpoint,
                                 Heun, Ralston, Heun's third-order method; the classic RK4 and
                                 the one-stage b = 1 tableau give PSST_METHOD_RK4 and _EULER bit
                                 for bit) */

/* Execution modes. */
#define PSST_MODE_AUTO 0  /* CTA mode when every network fits one CTA, else grid */
#define PSST_MODE_CTA 1   /* each network held on chip by one CTA or a cluster of
                             2 or 4 CTAs for all steps; many networks per launch
                             (batched, ragged), one launch per size class */
#define PSST_MODE_GRID 2  /* one network spread over the whole GPU with a
                             device-wide synchronisation (per-CTA phase flags)
                             per stage (single network) */

/*
 * A batch of independent networks.  Neurons are numbered globally
 * 0..N-1 (network b owns net_neuron_off[b] .. net_neuron_off[b+1]-1);
 * synapses form one CSR matrix over the global rows, row = postsynaptic
 * neuron, with the presynaptic index local to the row's network.
 * State layout everywhere (get/set/init): [V(N), m(N), h(N), n(N), r(S), s(S)],
 * float32.  Input current of neuron i at step k (held over the step's four
 * stages, the paper's eps_i read as the step):
 *   i_const[i] + (pulse_on[b] <= k < pulse_off[b] ? pulse_amp[i] : 0)
 *   + (noise event ? noise_amp : 0),
 * where the noise event is (Philox4x32-10(counter = {k lo, k hi, i, 0},
 * key = {seed lo, seed hi}) word 0 >> 8) < noise_thresh.
 */
typedef struct {
    int32_t n_nets;
    const int32_t *net_neuron_off; /* [n_nets+1], increasing, starts at 0 */
    const int32_t *neuron_type;    /* [N], 0..n_neuron_types-1 */
    int32_t n_neuron_types;
    const float *neuron_params;    /* [n_neuron_types * PSST_NEURON_NPARAM] */
    const int64_t *row_ptr;        /* [N+1], row_ptr[0] = 0, non-decreasing */
    const int32_t *pre;            /* [S], presynaptic neuron, local to the net */
    const float *weight;           /* [S], maximal synaptic conductance */
    const int32_t *syn_type;       /* [S], 0..n_syn_types-1 */
    int32_t n_syn_types;           /* 1..PSST_MAX_SYN_TYPES */
    const float *syn_params;       /* [n_syn_types * PSST_SYN_NPARAM] */
    const float *i_const;          /* [N] */
    const float *pulse_amp;        /* [N] or NULL (no pulse) */
    const int64_t *pulse_on;       /* [n_nets] or NULL */
    const int64_t *pulse_off;      /* [n_nets] or NULL */
    uint64_t noise_seed;
    uint32_t noise_thresh;         /* 0 = no noise; at most 2^24 */
    float noise_amp;
    float dt;                      /* ms, > 0 */
    const float *init_state;       /* [4N+2S] or NULL: V=-65, gates at rest, r=s=0 */
    int32_t rec_stride;            /* record V after global step k when k % stride == 0; 0 = off */
    int64_t rec_capacity;          /* frames in the record ring buffer (>= 1 if stride > 0) */
    int32_t mode;                  /* PSST_MODE_* */
    int32_t block_threads;         /* CTA size (multiple of 32, <= 1024), 0 = tuned */
    int32_t item_chunks;           /* 4-synapse chunks per work item of the synaptic sum (1..64), 0 = tuned */
    int32_t device;                /* CUDA device ordinal, -1 = current device */
    int32_t gate_mode;             /* 0: one gate per (presynaptic neuron, type) pair whenever all
                                      its synapses' gates are equal (bitwise-identical results,
                                      less work), else one per synapse; 1: always one per synapse */
    int32_t method;                /* PSST_METHOD_RK4 (0), PSST_METHOD_EULER (1) or PSST_METHOD_TABLEAU (2) */
    int32_t min_cluster;           /* CTA mode: spread every network of at least 2 x min_cluster neurons
                                      over a cluster of at least min_cluster CTAs (1, 2 or 4; same
                                      results, shorter steps when SMs are idle); 0 = chosen by
                                      psst_autotune (default 1) */
    int32_t rk_stages;             /* PSST_METHOD_TABLEAU: stages (1..4); ignored otherwise */
    float rk_a[3];                 /* a_2, a_3, a_4: stage s+1 starts at y + dt a_{s+1} k_s (finite) */
    float rk_b[4];                 /* b_1 .. b_{rk_stages}: weights of the step (finite, not all 0) */
} psst_network_desc;

typedef struct {
    int32_t n_nets;
    int64_t n_neurons, n_synapses;
    int64_t steps_done;            /* global step index of the current state */
    int64_t rec_frames;            /* frames recorded so far (all calls) */
    int32_t mode, block_threads, item_chunks; /* CTA size and work-item chunks of the last class */
    int32_t grid_ctas;             /* CTAs of one integrate chunk (all launches) */
    int32_t smem_bytes;            /* largest dynamic shared memory per CTA */
    int32_t n_single_cta_nets;     /* CTA mode: networks held by one CTA */
    int32_t n_cluster_nets;        /* CTA mode: networks spread over a cluster of 2 or 4 CTAs */
    int32_t n_launch_classes;      /* CTA mode: launches per integrate chunk (size classes) */
    int32_t kernel_launches;       /* kernels the last psst_integrate enqueued */
    int32_t n_pair_gate_nets;      /* networks whose forward keeps one gate per (presynaptic neuron, type)
                                      pair; the others keep one gate per synapse (gate_mode) */
    int32_t n_independent_nets;    /* CTA mode: networks without synapses, integrated one thread per neuron
                                      without barriers (bitwise the same results) */
    int64_t ck_start;              /* checkpoints recorded for psst_adjoint (psst_record_checkpoints):
                                      global step at which the recorded integrate call started, or -1
                                      when no valid recording exists (none made, or the state, step,
                                      weights or neuron table changed since) */
    int64_t ck_steps;              /* steps of that recorded call (0 when ck_start is -1) */
} psst_info;

typedef struct psst_net psst_net;

/* Optional device-memory provider for a handle (for example a framework's
   caching allocator): alloc(bytes, ctx) returns device memory of the
   handle's device, aligned to at least 256 bytes, or NULL; free(ptr, ctx)
   gives it back.  Both are called on the thread that calls into the
   library; the struct is copied at psst_create_network. */
typedef struct {
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *ctx;
} psst_allocator;

/* Validate the description, build the device layout and copy everything to
   the device (synchronous).  Reads the host arrays of *d only during the
   call.  Allocates device memory owned by the handle until
   psst_destroy_network, through *a (NULL: cudaMalloc / cudaFree).  Errors:
   INVALID_ARG (with a message naming the offending field/index, or an
   allocator with a NULL function), OOM, CUDA, UNSUPPORTED. */
int psst_create_network(const psst_network_desc *d, const psst_allocator *a, psst_net **out);

/* Advance every network by n_steps steps of the handle's method (RK4,
   Euler or its tableau) from the current state
   (Sec. "Circumventing memory constraints", item 2: successive calls
   continue where the previous one stopped; results are bitwise independent
   of how the steps are split into calls).  Each step-start state variable
   is carried with the rounding remainder of its compensated step sums
   (Knuth's TwoSum; the handle keeps the remainders between calls), so the
   FP32 trajectory tracks the exact RK4 map far more closely than plain
   FP32 accumulation.  Asynchronous on `stream`;
   device-side failures (NONFINITE, TIMEOUT) are reported by psst_status.
   With the environment variable PSST_SYNC set (to anything but "0") the
   call synchronises `stream` and returns what psst_status would.
   n_steps = 0 is a no-op.  Errors: INVALID_ARG (n_steps < 0), CUDA. */
int psst_integrate(psst_net *h, int64_t n_steps, void *stream);

/* Grid mode only: time limit of one wait at the device-wide barrier between
   stages (default 2 s).  On expiry the kernel records PSST_ERR_TIMEOUT,
   every CTA returns, and the state keeps its value from before the call's
   first step that failed.  0 makes every wait give up at once (a way to
   exercise the error path without a hang). */
int psst_set_barrier_timeout(psst_net *h, int64_t timeout_ns);

/* Replay psst_integrate's launch sequence through a CUDA graph (the
   paper's Sec. "Circumventing memory constraints" item 3: run a compiled
   static graph instead of issuing operations eagerly).  While enabled, the
   first call for a given n_steps captures the launches into a graph; later
   calls with the same n_steps replay it with the step index updated.
   Results are bitwise identical to direct launches.  Not combined with
   checkpoint recording (those calls launch directly). */
int psst_set_graph_mode(psst_net *h, int enable);

/* Autotuner: when the batch needs at most half the GPU's SMs, first time
   trial_steps steps with each network spread over clusters of at least 1,
   2 and 4 CTAs (networks large enough) and keep the fastest; then, for each
   size class of a CTA-mode handle, time trial_steps steps with twice, once,
   half and a quarter of the class's default CTA size, each with the planned
   number of shared-memory copies of the per-pair gate table and with a
   single copy, and keep the fastest.  Trials start from a copy of the state
   with recording off; the state is restored.  No choice changes the
   summation order (a larger cluster keeps the work-item size of one CTA),
   so results stay bitwise identical.  Synchronises `stream`.  Grid mode:
   no-op. */
int psst_autotune(psst_net *h, int64_t trial_steps, void *stream);

/* Synchronise `stream` and return the device error word (0 if none), then
   clear it. */
int psst_status(psst_net *h, void *stream);

/* Copy the state [V, m, h, n, r, s] (4N+2S floats, the FP32 values without
   their remainders) to dst (host or device memory as dst_on_device says),
   stream-ordered; synchronises the stream when dst is on the host.
   Errors: INVALID_ARG if n < 4N+2S. */
int psst_get_state(const psst_net *h, float *dst, size_t n, int dst_on_device, void *stream);

/* Overwrite the state from src (4N+2S floats, host or device).  The
   remainders of the compensated sums restart at zero (an FP32 state given
   by the caller is exact): a run continued from a state copied out with
   psst_get_state agrees with the uninterrupted run to rounding, not bit for
   bit. */
int psst_set_state(psst_net *h, const float *src, size_t n, int src_on_device, void *stream);

/* Set the global step index (time = step * dt) used for inputs and
   recording; resets the record ring buffer. */
int psst_set_step(psst_net *h, int64_t step);

/* Copy the recorded V frames, oldest first, into dst ([frames][N] floats,
   host or device); at most min(cap_frames, rec_capacity, frames recorded)
   frames; *n_frames receives the count.  The ring keeps the newest
   rec_capacity frames. Synchronises the stream when dst is on the host. */
int psst_read_record(const psst_net *h, float *dst, size_t cap_frames, int64_t *n_frames,
                     int dst_on_device, void *stream);

/* Replace the synaptic weights ([S] floats, CSR order) or the neuron-type
   table ([n_neuron_types * PSST_NEURON_NPARAM] floats) from host or device
   memory; used by later psst_integrate / psst_adjoint calls (stream-ordered;
   synchronises when the source is on the host). */
int psst_set_weights(psst_net *h, const float *w, size_t n, int on_device, void *stream);
int psst_set_neuron_params(psst_net *h, const float *p, size_t n, int on_device, void *stream);

/* Record checkpoints for the adjoint: while every > 0, each psst_integrate
   call (of at most max_steps steps) stores the full state and its
   remainders at its start and after every `every` steps, so that
   psst_adjoint(..., ckpt_every = 0) can differentiate that call's span
   without integrating it again.  The recorded span is invalidated by
   set_state, set_step, set_weights and set_neuron_params.  every = 0 stops
   recording.  CTA mode only.  The buffers (2 x ceil(max_steps / every) full
   states) are allocated here, or reused when large enough. */
int psst_record_checkpoints(psst_net *h, int32_t every, int64_t max_steps);

/* Discrete adjoint of the integration map -- RK4, forward Euler (Eq. euler)
   or the handle's tableau, by its method -- (no counterpart in the paper;
   the differentiated form).  For the n_steps steps that a psst_integrate call
   made now would take -- from the current state and step index -- computes
   the gradient of
       L = sum_f sum_i dL_dV[f][i] * V_i(frame f)
   where frame f is the f-th recorded frame of that span (global steps k in
   (step, step + n_steps] with k % rec_stride == 0; n_frames must equal their
   count).  Outputs (device arrays, overwritten):
     grad_w              [S]   dL/dw for every synapse, CSR order;
     grad_neuron_params  [n_neuron_types * 9]  dL/d(neuron-type table);
     grad_state0         [4][N] dL/d(V, m, h, n at the start), or NULL.
   The state and step index are left unchanged.  Memory: the forward
   kernel integrates the span once, recording the full state and its
   remainders every ckpt_every steps (the record ring is not written), and
   each segment is recomputed from its checkpoint; the handle allocates the
   storage on first use and grows it as needed.  The first call also reads
   the connectivity back (synchronous copies) to plan the sweep's
   synapses by presynaptic column; later calls reuse the plan.  The recomputation uses the
   adjoint's own arithmetic, so its trajectory drifts slowly from the forward
   kernel's: spacings of up to about 1000 steps keep FP32 gradients within
   1e-3 of the exact map's on 20,000-step spiking spans.
   ckpt_every = 0 differentiates instead the span of the last psst_integrate
   call, whose checkpoints were recorded (psst_record_checkpoints); n_steps
   must equal that call's; PSST_ERR_STATE if no such checkpoints exist.
   Preconditions: CTA mode (else PSST_ERR_UNSUPPORTED); every network fits one CTA for the adjoint; all
   gates of a (presynaptic neuron, synapse type) pair hold the same value at
   the start (true from rest), else the device reports PSST_ERR_UNSUPPORTED
   through psst_status.  Each network runs on a cluster of two CTAs (forward
   recompute beside the reverse sweep).  Asynchronous on `stream`. */
int psst_adjoint(psst_net *h, int64_t n_steps, const float *dL_dV, int64_t n_frames, int32_t ckpt_every,
                 float *grad_w, float *grad_neuron_params, float *grad_state0, void *stream);

/* Sizes, progress and the launch configuration. */
int psst_query(const psst_net *h, psst_info *out);

/* Free all device memory of the handle (synchronises its device). NULL is a no-op. */
int psst_destroy_network(psst_net *h);

/* Static description of an error code. */
const char *psst_error_string(int code);

/* Message of the last failing call on this thread ("" if none). */
const char *psst_last_error(void);

/*
 * Integration without device allocation.
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc themselves or let a library do it -- code that
 * must keep every device byte inside an allocator it does not control (a
 * framework's memory pool, a memory-capped or sandboxed process), or code
 * that only receives buffers from its caller.  They pass their own device
 * arrays in the layout below, and the call allocates nothing: the grid-wide
 * kernel's extra memory (gate-map tables, per-CTA phase flags, plan) is
 * one fixed array of PSST_NOALLOC_SCRATCH_BYTES in device global memory,
 * compiled into the library.  Every GPU that loads the library holds that
 * array until the process exits.
 *
 * psst_integrate_grid_noalloc advances the single network *net by n_steps
 * RK4 steps starting at global step index step0, exactly like
 * psst_integrate in PSST_MODE_GRID with one gate per synapse (same kernel;
 * with gate_mode = 1 and the same item_chunks the results are bitwise
 * identical to a psst_integrate call made right after psst_set_state: the
 * call keeps no remainders of its compensated step sums, so each call
 * starts them at zero; the per-pair gate table of psst_integrate groups the
 * synaptic sums by type and agrees to rounding).  It runs on the current device and
 * `stream`.  Its first call on a device looks up that device's address of
 * the fixed array (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Each call synchronises `stream` once, after planning and
 * before the integration launch, and otherwise returns without waiting.
 * Every call uses the same array and finds it as the last call left it; the
 * call clears what must start at zero.  Two calls whose GPU work overlaps
 * (different streams without ordering, or different threads) race on the
 * array and give wrong results.
 *
 * The plan (rows per CTA, item_chunks when it is 0) is the one
 * psst_integrate makes in grid mode with gate_mode = 1, so item_chunks = 0
 * gives the same chunk size and bitwise the same results as psst_integrate
 * with its item_chunks left at 0.
 *
 * The array contents are checked on the device before anything else reads
 * them: row_ptr must rise from 0 to n_synapses; every syn_code must hold a
 * type below n_syn_types and a pair index pre * n_syn_types + type with the
 * same type and pre < n_neurons; every neuron_type must lie in
 * 0..n_neuron_types-1.  A failed check returns PSST_ERR_INVALID_ARG with no
 * integration launched and *state untouched.  Float contents are not
 * checked: a NaN or infinity in the state shows up as PSST_ERR_NONFINITE in
 * *err after the launch.
 *
 * Limits: n_neurons * n_syn_types < 65536 (the gate-map tables then always
 * fit the array); larger networks return PSST_ERR_UNSUPPORTED, as does a
 * network whose per-CTA share does not fit shared memory.  Errors are
 * reported by return code only (psst_last_error is not updated):
 * INVALID_ARG for a NULL pointer, a bad size/field or array contents that
 * fail the checks above, UNSUPPORTED for the limits above, CUDA for a
 * failing runtime call.  Device-side failures (TIMEOUT, NONFINITE) are
 * written to *err (the caller zeroes it).
 */
#define PSST_NOALLOC_SCRATCH_BYTES (4u << 20)

typedef struct {
    int64_t n_neurons, n_synapses;
    int32_t n_syn_types;            /* 1..PSST_MAX_SYN_TYPES */
    int32_t item_chunks;            /* 4-synapse chunks per work item, 0 = chosen by the call */
    int32_t n_neuron_types;         /* rows of neuron_params, >= 1 */
    const int64_t *row_ptr;         /* device [N+1], CSR by postsynaptic neuron */
    const uint32_t *syn_code;       /* device [S]: (syn_type << 24) | (pre * n_syn_types + syn_type) */
    const float *weight;            /* device [S] */
    const int32_t *neuron_type;     /* device [N] */
    const float *neuron_params;     /* device [n_neuron_types * PSST_NEURON_NPARAM] */
    const float *syn_params;        /* device [n_syn_types * PSST_SYN_NPARAM] */
    const float *i_const;           /* device [N] */
    const float *pulse_amp;         /* device [N] or NULL */
    int64_t pulse_on, pulse_off;    /* pulse window in steps */
    uint64_t noise_seed;
    uint32_t noise_thresh;
    float noise_amp;
    float dt;
    float *state;                   /* device [4N+2S], read and overwritten */
    float *rec;                     /* device [rec_capacity][N] or NULL */
    int32_t rec_stride;
    int64_t rec_capacity;
    int *err;                       /* device error word, written on device failure */
} psst_device_network;

int psst_integrate_grid_noalloc(const psst_device_network *net, int64_t step0, int64_t n_steps, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PSST_H */
