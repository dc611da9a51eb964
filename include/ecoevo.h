/*
 * ecoevo.h -- C ABI of libecoevo, the GB300 (sm_103a) simulation step of
 * non-episodic neuroevolution in a large multi-agent common-pool-resource
 * grid world (Hamon, Nisioti, Moulin-Frier, 2023).
 *
 * One call of eco_world_step advances a world by whole steps.  A step is,
 * in order (each part is a CUDA kernel of this library):
 *   a1 regrowth of the resource field      App. B.1, Eq. (1)
 *   a2 observation of the 7x7x3 window      App. B.2, sensorimotor ability
 *   a3 one LSTM step per agent + argmax     App. B.2, cognitive capacity
 *   a4 moves (one claim round) and eating   App. B.2
 *   a5 physiology and death                 App. B.2 physiology, App. B.3 death
 *   a6 reproduction: slot compaction and    App. B.3 reproduction
 *      Gaussian mutation of the parent's weights
 * The mutation of a step's births runs in the first kernel of the next step
 * (the same launch as its a1), or before a state read that returns weights:
 * newborns act from the step after their birth, so no result changes.
 *
 * Conventions, for every entry point:
 *   - Return ECO_OK (0) on success or a negative ECO_E* code.
 *   - Pointers named *_host are host memory; everything else handed to the
 *     library is a device pointer of the current CUDA device.
 *   - Work is enqueued on the world's CUDA stream and is asynchronous unless
 *     the comment says "synchronous".
 *   - A world is not thread-safe; distinct worlds may be used from distinct
 *     host threads.
 *   - Device-side waits are bounded: a wait that runs out sets a status bit
 *     that eco_world_sync / eco_batch_sync return as ECO_ETIMEOUT.
 *   - The checked build of this library (libecoevo_checked.so) range-checks
 *     every index it reads from device memory before using it; a failed
 *     check skips the access and eco_world_sync / eco_batch_sync return
 *     ECO_EBOUNDS.  The regular build has no such checks.
 */
#ifndef ECOEVO_H
#define ECOEVO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ECO_ABI_V2 0x45434F02u

/* Error codes. */
#define ECO_OK 0
#define ECO_EINVAL -1    /* invalid argument or parameter block            */
#define ECO_ENOMEM -2    /* arena too small, or an allocation failed       */
#define ECO_ECUDA -3     /* a CUDA runtime call failed                     */
#define ECO_ETIMEOUT -4  /* a bounded device wait ran out                  */
#define ECO_ESTATE -5    /* loaded state is inconsistent (shared cell ...) */
#define ECO_EBOUNDS -6   /* a device index was out of range (checked build)  */

/* Controllers (EcoParams.controller).
 *   ECO_CTRL_LSTM32  LSTM with 32 units on the 7x7 view (resource, other
 *                    agent, wall) + energy, 5 logits, action = first argmax
 *                    (App. B.2 form, the 200x400 workloads' controller).
 *   ECO_CTRL_PAPER   the paper's own controller (App. B.5): 15x15 view,
 *                    conv 3x3/2 (4) + average pool 2x2/1, conv 3x3/2 (8) +
 *                    pool, embedding [72 features, previous action one-hot,
 *                    ate-last-step bit], LSTM with 4 units, dense 8 + tanh on
 *                    [embedding, h], dense 5; the action is sampled from the
 *                    softmax at temperature 1/50 with the uniform
 *                    (word0 >> 8) 2^-24 of the Philox block {slot, t, 6, 0}:
 *                    the number of k < 4 whose cumulative probability is <= u. */
#define ECO_CTRL_LSTM32 0
#define ECO_CTRL_PAPER 1
#define ECO_NOBS 148
#define ECO_HIDDEN 32        /* h and c have 32 floats per slot (4 used by ECO_CTRL_PAPER) */
#define ECO_NACT 5
#define ECO_NPARAM 23333     /* parameters per agent, ECO_CTRL_LSTM32 */
#define ECO_PC_NPARAM 2445   /* parameters per agent, ECO_CTRL_PAPER   */

/* World parameters; all plain data.  Field meanings:
 *   H, W            grid rows (latitude axis, row 0 = top) and columns
 *   capacity        agent slots; births past the free slots are dropped
 *   n_agents0       agents placed at random free cells at creation
 *   border_walls    1: the outer ring of cells is wall (App. B.1)
 *   res_init_p      Bernoulli density of the initial resources
 *   nbr_shape       0: square (Chebyshev) neighbourhood, 1: diamond
 *   nbr_radius      1..3, the centre cell is never counted
 *   class_edges     count class = number of edges <= count (4 classes)
 *   p_class         p_I per count class                    Eq. (1)
 *   lat_mode        0: linear climate lat_top -> lat_bottom over the rows;
 *                   1: c = (alpha^x + 1)/(alpha + 1), x = row/(H-1)
 *   p_spont         spontaneous growth probability c        Eq. (1)
 *   e0, e_decay, e_gain, e_max   initial energy, decay per step, gain per
 *                   resource eaten, clip                    App. B.2
 *   e_repr, t_repr  reproduce after t_repr consecutive steps above e_repr
 *   e_death, t_death  die after max(t_death,1) consecutive steps at or below
 *                   e_death;  max_age: die when age exceeds it   App. B.3
 *   wall_kills      1: an agent moving into a wall or off the grid dies
 *                   (App. B.1); 0: the move is blocked
 *   w_init_std      std of the initial weights; mut_std: std sigma of the
 *                   mutation noise N(0, sigma)                  App. B.3
 *   controller      ECO_CTRL_LSTM32 or ECO_CTRL_PAPER           App. B.2, B.5
 * Sizes: 3 <= H, W <= 16384 with H*W <= 2^26; capacity <= 2^24. */
typedef struct EcoParams {
  uint32_t abi_version; /* must be ECO_ABI_V2 */
  int32_t H, W, capacity, n_agents0;
  int32_t border_walls;
  double res_init_p;
  int32_t nbr_shape, nbr_radius;
  int32_t class_edges[3];
  double p_class[4];
  int32_t lat_mode;
  double lat_top, lat_bottom, lat_alpha;
  double p_spont;
  float e0, e_decay, e_gain, e_max;
  float e_repr;
  int32_t t_repr;
  float e_death;
  int32_t t_death, max_age;
  int32_t wall_kills;
  float w_init_std, mut_std;
  int32_t controller;
} EcoParams;

/* Counters (int64), indices into EcoState.counters. */
#define ECO_C_T 0            /* steps taken                       */
#define ECO_C_POP 1          /* living agents                     */
#define ECO_C_BIRTHS 2       /* births so far                     */
#define ECO_C_DEATHS 3       /* deaths so far                     */
#define ECO_C_DROPPED 4      /* births dropped for lack of a slot */
#define ECO_C_BIRTHS_LAST 5  /* births of the last step           */
#define ECO_C_DEATHS_LAST 6
#define ECO_C_DROPPED_LAST 7
#define ECO_C_AGENT_STEPS 8  /* sum over steps of the agents alive at the step's start */
#define ECO_NCOUNTERS 9

/* Host-side view of a world's state.  Every pointer is caller-owned host
 * memory and may be NULL to skip that field.  Grid fields are unpacked
 * uint8 [H*W] row-major; per-slot fields have `capacity` entries; h, c are
 * [capacity*32]; logits [capacity*5]; weights are logical parameter
 * vectors [weights_count * P] for slots weights_first ..
 * weights_first + weights_count - 1.  ECO_CTRL_LSTM32, P = 23333:
 *   W[r][k]  r < 128 gate rows (i, f, g, o blocks of 32), k < 180
 *            (148 observation inputs, then 32 hidden inputs)   [0, 23040)
 *   b[r]                                                    [23040, 23168)
 *   Wo[a][j] a < 5, j < 32                                  [23168, 23328)
 *   bo[a]                                                   [23328, 23333)
 * ECO_CTRL_PAPER, P = 2445:
 *   conv1 [4 out][3 ky][3 kx][3 in]     [0, 108)     bias [108, 112)
 *   conv2 [8 out][3][3][4 in]           [112, 400)   bias [400, 408)
 *   LSTM input kernel [16][78]          [408, 1656)  (row = gate*4 + unit,
 *   LSTM recurrent kernel [16][4]       [1656, 1720)  gates i, f, g, o)
 *   LSTM bias [16]                      [1720, 1736)
 *   dense [8][82]                       [1736, 2392) bias [2392, 2400)
 *   dense [5][8]                        [2400, 2440) bias [2440, 2445)
 * prev_action: the action each agent moved with in its last step (0 for
 * newborns); ate: 1 if it ate in its last step.  Both are inputs of
 * ECO_CTRL_PAPER. */
typedef struct EcoState {
  int64_t counters[ECO_NCOUNTERS];
  uint8_t *res_host, *wall_host;
  int32_t *slot_map_host;  /* read only: -1 or the slot on the cell */
  uint8_t *alive_host;
  int32_t *y_host, *x_host;
  float *energy_host;
  int32_t *repr_ctr_host, *low_ctr_host, *age_host;
  float *h_host, *c_host;
  int32_t *action_host;    /* the controller's argmax of the last step */
  float *logits_host;
  float *weights_host;
  int32_t weights_first, weights_count;
  int32_t *prev_action_host;
  uint8_t *ate_host;
} EcoState;

typedef struct EcoWorld EcoWorld;
typedef struct EcoBatch EcoBatch;

/* Device bytes a world of these parameters needs (0 if they are invalid).
 * Synchronous, host only. */
size_t eco_world_bytes(const EcoParams *params);

/* Create a world (App. B.4: random walls border, random resources, random
 * placement of n_agents0 agents, random weights, all drawn from `seed`).
 *   arena, arena_bytes: caller-owned device memory of at least
 *     eco_world_bytes(params), 256-byte aligned, kept alive until
 *     eco_world_destroy; or NULL/0 to let the library allocate and own it.
 *   stream: cudaStream_t all work of the world is enqueued on; must not be
 *     the legacy default stream (0), since steps are replayed as CUDA graphs.
 * Synchronous (returns once the initial state is on the device).
 * Errors: ECO_EINVAL (params, alignment, stream), ECO_ENOMEM, ECO_ECUDA. */
int eco_world_create(const EcoParams *params, uint64_t seed, void *arena,
                     size_t arena_bytes, void *stream, EcoWorld **out);

/* Release the world (and its arena if the library allocated it). */
void eco_world_destroy(EcoWorld *world);

/* Advance the world by n_steps >= 0 whole steps (a1..a6 each step).
 * Asynchronous.  Errors: ECO_EINVAL, ECO_ECUDA. */
int eco_world_step(EcoWorld *world, int64_t n_steps);

/* One step in which moves use the given actions instead of the controller's
 * argmax; the controller still runs and its argmax is kept as `action`.
 * actions: int32 [capacity] (values 0..4; 0 = stay, 1 N, 2 S, 3 E, 4 W),
 * on the host if actions_on_host != 0, else on the device.  Synchronous
 * when actions_on_host.  Test hook for multi-step parity runs. */
int eco_world_step_forced(EcoWorld *world, const int32_t *actions,
                          int actions_on_host);

/* Copy the state into `out` (see EcoState).  Synchronous.  The weights of
 * the last step's births are written by the first kernel of the next step;
 * when weights are requested, that kernel's work for them is done first
 * (the next step then leaves them as they are). */
int eco_world_read_state(EcoWorld *world, EcoState *out);

/* Replace the state by `in`: every non-NULL field is written; slot_map,
 * the population and the free/alive lists are rebuilt from alive, y, x.
 * counters[ECO_C_T] and the cumulative counters are taken from `in` when
 * set_counters != 0.  h and c become the recurrent state for the next step.
 * A new analysis window (eco_world_analysis_async) starts at the loaded
 * state.  The births of the world's last step get their weights first, so
 * that rows `in` leaves out hold final weights.  Page-locked host buffers
 * are read by kernels through their device addresses (a weight buffer must
 * then start on a 16-byte boundary, else it is copied like pageable memory);
 * the weight rows go on a second stream of the world, created at the first
 * call, beside the rest of the state.  Synchronous: both streams are done
 * when the call returns.  Errors:
 * ECO_EINVAL, ECO_ESTATE (two agents on one
 * cell, an agent on a wall or off the grid, a negative age, res set on a
 * wall), ECO_ECUDA. */
int eco_world_load_state(EcoWorld *world, const EcoState *in, int set_counters);

/* Enqueue a copy of the world's counters (ECO_NCOUNTERS int64 in ECO_C_*
 * order, as they stand after the work enqueued so far) into out_host.
 * Asynchronous when out_host is page-locked host memory (for example from
 * cudaHostAlloc or a pinned torch tensor); the values are valid once the
 * world's stream has reached the copy (eco_world_sync).  Lets a step loop
 * stream its results without waiting for every step. */
int eco_world_counters_async(EcoWorld *world, int64_t *out_host);

/* Per-step counter log written by the step kernels themselves: from the
 * work enqueued after this call on, the kernel that ends step t (t counted
 * from 0, so counters[ECO_C_T] == t + 1 after it) writes the ECO_NCOUNTERS
 * counters, in ECO_C_* order, to row t mod rows of log_host, an array of
 * rows x ECO_NCOUNTERS int64 that the caller owns and keeps allocated and
 * page-locked while the log is on.  It must be mapped into the device's
 * address space (memory from cudaHostAlloc or cudaMallocHost, or a pinned
 * torch tensor, on a system with unified addressing).  No copy or launch is
 * added to a step, so a loop over many steps (graph chunks included) gets
 * every step's counters on the host; a row is valid once the world's stream
 * has passed that step (eco_world_sync, or an event).  log_host == NULL
 * turns the log off.  Synchronous (waits for the world's stream).
 * Errors: ECO_EINVAL (world NULL; rows <= 0; log_host not 8-byte aligned,
 * not page-locked or not mapped), ECO_ECUDA. */
int eco_world_counter_log(EcoWorld *world, int64_t *log_host, int64_t rows);

/* Metrics of the paper's analyses (App. C), for the window of steps since
 * the previous call (or since create / load_state, which start a window).
 * Life expectancy over several windows = sum(death_age_sum) / sum(deaths);
 * the paper uses 500-step windows for it and 50-step windows for movement.
 * An agent's age at death is its age counter when it dies: after the
 * step's increment when it dies of energy or age, unchanged when a wall
 * kills it.  Movement: every agent alive over the whole window (present at
 * its start and now) falls in bin floor(17 d / (L + 1)), d the Manhattan
 * distance between its cells at the window start and now, L = window_steps
 * (d <= L, so bins of three distances for L = 50). */
#define ECO_MOVE_BINS 17
typedef struct EcoAnalysis {
  int64_t t;                 /* steps taken (ECO_C_T) at the call          */
  int64_t window_steps;      /* L: steps in the window                     */
  int64_t population;        /* living agents                              */
  int64_t resources;         /* cells holding a resource                   */
  int64_t deaths;            /* deaths during the window                   */
  int64_t death_age_sum;     /* sum of their ages at death                 */
  int64_t movers;            /* agents alive over the whole window         */
  int64_t move_bins[ECO_MOVE_BINS];
} EcoAnalysis;

/* Enqueue the analysis of the window that ends now (three kernels on the
 * world's stream, after the work enqueued so far) and a copy of the record
 * into out_host; a new window starts.  Asynchronous when out_host is
 * page-locked; valid once the stream has reached the copy (eco_world_sync).
 * For a world stepped in a batch, call it when the batch's stream (the
 * first world's) has reached the point of interest (eco_batch_sync), or
 * share that stream.  Errors: ECO_EINVAL, ECO_ECUDA. */
int eco_world_analysis_async(EcoWorld *world, EcoAnalysis *out_host);

/* Life expectancy (App. C: mean age at death; the paper pools 500 steps)
 * over n consecutive analysis records (host memory, as eco_world_analysis_async
 * wrote them): sum of death_age_sum / sum of deaths, written to *out; NaN
 * when nobody died.  Host only, synchronous.  Errors: ECO_EINVAL. */
int eco_life_expectancy(const EcoAnalysis *records, int64_t n, double *out);

/* Greediness in the lab environments (App. C): G = C_r / T_r, where T_r
 * counts the windows (the paper's are 20 steps) in which a resource was in
 * the agent's field of view at the observation of some step (7x7 or 15x15
 * by controller) and C_r the windows in which it ate.  eco_world_lab_window
 * ends the current window (asynchronous, on the world's stream): every
 * living agent adds its two window flags to its T_r, C_r.  A newborn starts
 * at zero; create and load_state zero every slot.  eco_world_lab_read
 * copies T_r, C_r of every slot (int32 [capacity] each, caller-owned host
 * memory) after waiting for the stream.  Errors: ECO_EINVAL, ECO_ECUDA. */
int eco_world_lab_window(EcoWorld *world);
int eco_world_lab_read(EcoWorld *world, int32_t *seen_windows_host, int32_t *meal_windows_host);

/* Greediness G = C_r / T_r of n agents (App. C) from the two window counts
 * eco_world_lab_read returns (host memory): out[i] = meal_windows[i] /
 * seen_windows[i], NaN where seen_windows[i] = 0.  Host only, synchronous.
 * Errors: ECO_EINVAL. */
int eco_greediness(const int32_t *seen_windows, const int32_t *meal_windows, int64_t n,
                   double *out);

/* Wait for the world's stream; returns ECO_ETIMEOUT if a device wait ran
 * out, ECO_ECUDA on a CUDA error, else ECO_OK.  Synchronous. */
int eco_world_sync(EcoWorld *world);

/* Failure detection without a fault: enqueue a kernel that runs the same
 * bounded mbarrier wait the step's pipeline uses, on a barrier whose phase
 * never completes; after limit_ns (<= 10 s) it gives up and sets the
 * world's timeout status, so the next eco_world_sync returns ECO_ETIMEOUT and
 * the CUDA context stays usable.  Asynchronous.  Errors: ECO_EINVAL. */
int eco_world_selftest_timeout(EcoWorld *world, uint64_t limit_ns);

/* Clear the world's device status word (after ECO_ETIMEOUT was handled).
 * Synchronous. */
int eco_world_clear_status(EcoWorld *world);

/* The world's parameters and CUDA stream. */
const EcoParams *eco_world_params(const EcoWorld *world);
void *eco_world_stream(const EcoWorld *world);

/* Batch of independent worlds stepped together: every kernel of a step is
 * launched once for all of them (work lists over worlds and agents).  The
 * worlds must live on the current device and share one controller; the
 * batch uses the first world's stream.  The worlds must outlive the batch.
 * A member world's own calls (state I/O, counters, analysis) are ordered on
 * that world's stream: call eco_batch_sync before them. */
int eco_batch_create(EcoWorld *const *worlds, int n_worlds, EcoBatch **out);
int eco_batch_step(EcoBatch *batch, int64_t n_steps);
int eco_batch_sync(EcoBatch *batch);
void eco_batch_destroy(EcoBatch *batch);

/* Launch configuration of a batch (or of a world stepped alone).  None of
 * these choices changes any result, only how a step's work is cut into
 * launches and CTAs:
 *   fused              1: the slot phases of a step (moves, physiology,
 *                      death, birth claims, slot compaction) run as one
 *                      8-CTA cluster per world; 0: as four grid-wide
 *                      kernels.  1 is allowed only when every world's
 *                      capacity is at most 16384 (the default then).
 *   spawn_ctas_per_sm  CTAs per SM that write the children's mutated weights
 *                      (1..32, default 4).
 *   steps_per_graph    steps captured in one CUDA graph for eco_*_step
 *                      (1..1024, default 16).
 * set_config waits for the stream when the configuration changes.  Errors:
 * ECO_EINVAL (a value out of range, fused with a capacity above 16384). */
int eco_batch_set_config(EcoBatch *batch, int fused, int spawn_ctas_per_sm,
                         int steps_per_graph);
int eco_batch_get_config(const EcoBatch *batch, int *fused, int *spawn_ctas_per_sm,
                         int *steps_per_graph);

/* Kernel shapes of a batch (or of a world stepped alone); like the launch
 * configuration, no choice changes any result:
 *   regrow_rows_per_cta  8-row x 128-cell regrowth tiles stacked in one CTA
 *                        of the tail kernel: 1, 2, 4 or 8, or 0 to choose by
 *                        size (the fewest that leave at most four regrowth
 *                        CTAs per SM, one wave of the tail kernel; the
 *                        default).
 *   lstm_ctas_per_sm     CTAs per SM of the controller kernel of the LSTM(32)
 *                        controller: 1 (an 8-block weight ring, two agents in
 *                        flight; the default) or 2 (a 4-block ring each).
 * set_shape waits for the stream when a shape changes; get_shape reports
 * the stacking in use (never 0).  Errors: ECO_EINVAL (a value out of range),
 * ECO_ECUDA. */
int eco_batch_set_shape(EcoBatch *batch, int regrow_rows_per_cta, int lstm_ctas_per_sm);
int eco_batch_get_shape(const EcoBatch *batch, int *regrow_rows_per_cta,
                        int *lstm_ctas_per_sm);

/* Result of the tuner. */
typedef struct EcoTuneResult {
  int32_t fused, spawn_ctas_per_sm, steps_per_graph;
  int32_t regrow_rows_per_cta, lstm_ctas_per_sm, reserved;
  int64_t steps_taken;          /* steps every world advanced while tuning  */
  double ms_per_step_initial;   /* one trial in the configuration it started from */
  double ms_per_step_best;      /* the chosen configuration, timed once more at
                                   the end (at the population reached then)  */
} EcoTuneResult;

/* Choose the launch configuration and kernel shapes for this batch's worlds
 * by timing real steps of the batch: one knob after the other (fused, then
 * spawn_ctas_per_sm, lstm_ctas_per_sm (LSTM(32) controller only),
 * regrow_rows_per_cta, then steps_per_graph), every candidate value three
 * times round-robin, trial_steps steps per trial (a graph-length trial
 * takes trial_steps rounded up to a multiple of that length); a knob moves to
 * the candidate with the lowest median time per step only if that median is
 * more than 3% below the current value's.  Candidates: fused {1, 0},
 * spawn_ctas_per_sm {1, 2, 4, 8}, lstm_ctas_per_sm {1, 2},
 * regrow_rows_per_cta {1, 2, .., the default} (none when the default is 1),
 * steps_per_graph {1, 4, 16, 50}.  Finally the
 * chosen configuration is timed once more (ms_per_step_best).  The worlds advance by
 * out->steps_taken steps, exactly as eco_batch_step would have taken them.
 * Synchronous.  Errors: ECO_EINVAL (trial_steps outside 1..100000, profiling
 * on), ECO_ECUDA. */
int eco_batch_autotune(EcoBatch *batch, int trial_steps, EcoTuneResult *out);

/* The same for a world stepped alone (eco_world_step). */
int eco_world_set_config(EcoWorld *world, int fused, int spawn_ctas_per_sm,
                         int steps_per_graph);
int eco_world_get_config(const EcoWorld *world, int *fused, int *spawn_ctas_per_sm,
                         int *steps_per_graph);
int eco_world_set_shape(EcoWorld *world, int regrow_rows_per_cta, int lstm_ctas_per_sm);
int eco_world_get_shape(const EcoWorld *world, int *regrow_rows_per_cta,
                        int *lstm_ctas_per_sm);
int eco_world_autotune(EcoWorld *world, int trial_steps, EcoTuneResult *out);

/* Per-kernel timing with CUDA events on the world's stream.  While enabled,
 * each step (up to max_steps after each read) launches its kernels on the
 * stream with an event recorded before and after every kernel (no graph, no
 * programmatic overlap between the kernels); the elapsed times of a step are
 * added to their kernels when the next profiled step is launched (the
 * events are reused, so that launch first waits for the previous one) or
 * when they are read.  eco_world_profile_read waits for the
 * stream and returns the sums since enabling:
 * ms[k], launches[k] for k < ECO_NKERNELS (names: eco_kernel_name; a kernel
 * the world's step does not launch keeps 0 launches).  A step runs
 * "regrow_spawn" (the regrowth of the step's resource plane and the mutation
 * of the previous step's births in one launch), then "observe_lstm"
 * (ECO_CTRL_PAPER: "observe_paper"), then the slot phases (moves,
 * physiology, birth claims, compaction) as one kernel "agents_fused" for
 * worlds of capacity <= 16384 or as five kernels otherwise.  "regrow" is no
 * longer launched (kept so that the kernel ids stay stable). */
#define ECO_NKERNELS 10
int eco_world_profile(EcoWorld *world, int enable, int max_steps);
int eco_world_profile_read(EcoWorld *world, double *ms, int64_t *launches);
const char *eco_kernel_name(int k);

/* Number of the library's kernels one step of this world launches. */
int eco_kernels_per_step(const EcoWorld *world);

const char *eco_strerror(int code);

/* Move resolution that allocates no device memory.  The paper has no
 * counterpart to this entry point: it exists for callers that cannot call
 * cudaMalloc -- for example code that runs under another allocator which
 * owns all of the device's memory, or a loop that must not stall on the
 * device-wide synchronisation an allocation can cause.
 *
 * Applies one round of moves with the rule of the simulation step: agent s
 * (alive[s] != 0) with action a in {1 N, 2 S, 3 E, 4 W} moves to its target
 * cell iff the cell is on the grid, not a wall, empty in slot_map at the
 * start of the call, and s is the lowest slot claiming it; every other agent
 * stays.  With wall_kills != 0, killed[s] = 1 for an agent whose target is a
 * wall or off the grid (killed may be NULL; the caller removes such agents).
 *   wall      uint8 [H*W]  row-major, nonzero = wall              (device)
 *   alive     uint8 [capacity]                                    (device)
 *   actions   int32 [capacity], values 0..4 (others mean stay)    (device)
 *   y, x      int32 [capacity], in/out positions                  (device)
 *   slot_map  int32 [H*W], in/out: -1 or the slot on the cell     (device)
 *   killed    uint8 [capacity] or NULL, out                       (device)
 *   stream    cudaStream_t the work is enqueued on (asynchronous)
 * The per-cell claims live in one fixed array inside the library, sized for
 * at most 2^21 cells (H*W <= 2,097,152; larger grids return ECO_EINVAL with a
 * message on stderr); every GPU that loads the library keeps those 8 MiB
 * until the process exits.  The first call on each device looks up the
 * array's device address; make that first call before any stream capture.
 * Each call resets the claims it uses, but all calls share the one array:
 * calls that overlap on the GPU (other streams, other threads) race and must
 * be serialised by the caller.  Errors: ECO_EINVAL, ECO_ECUDA. */
int eco_moves_noalloc(int32_t H, int32_t W, int32_t capacity, int32_t wall_kills,
                      const uint8_t *wall, const uint8_t *alive,
                      const int32_t *actions, int32_t *y, int32_t *x,
                      int32_t *slot_map, uint8_t *killed, void *stream);

#ifdef __cplusplus
}
#endif
#endif
