/*
 * ecoevo_oracle.h -- plain, slow, single-threaded CPU simulator of the
 * non-episodic simulation step of "Eco-evolutionary Dynamics of
 * Non-episodic Neuroevolution in Large Multi-agent Environments"
 * (Hamon, Nisioti, Moulin-Frier, 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists to check the CUDA library.
 * Only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header, table or constant
 * generator with the CUDA path; it carries its own Philox4x32-10, its own
 * Box-Muller transform and its own LSTM, all written in plain loops.
 *
 * Precision: energies and weights are FP32 state (the step is FP32
 * throughout), so they are stored as float and every energy operation is a
 * single IEEE float add/sub (build with -ffp-contract=off).  Everything the
 * paper leaves to a network (gates, cell state, logits) is computed in
 * double and kept in double.
 *
 * Parity status per function (the pins live in tests/test_oracle_*.py):
 *   or_philox4x32_10   pinned: published known-answer vectors
 *   or_box_muller      pinned: moments + Kolmogorov-Smirnov vs N(0,1)
 *   or_threshold_table pinned: per-class growth frequencies (binomial bound)
 *   or_regrow          pinned: convolution-count reconstruction, invariants
 *   or_observe         pinned: numpy padded-slice reconstruction
 *   or_lstm_step       pinned: torch.nn.LSTMCell (float64), bias-only closed form
 *   or_world_step      pinned: invariants, float32 energy closed forms,
 *                      brute force on <=4x4 worlds, slot-assignment rules,
 *                      the same result for any slot visiting order
 *   or_world_analysis  pinned: hand-counted walks and lifetimes, closed
 *                      forms of the bin edges, age-based identity check
 *   or_pc_observe      pinned: numpy padded-slice reconstruction (15x15)
 *   or_pc_forward      pinned: torch conv2d/avg_pool2d/LSTMCell/linear
 *                      (float64); the layer sizes give the paper's 2445
 *                      parameters
 *   or_pc_sample       pinned: closed forms (uniform, one-hot, ties),
 *                      frequencies against softmax(50 logits)
 *   or_action_uniform  pinned: numpy Philox reconstruction
 *   or_world_lab_window pinned: hand-counted walks past placed resources,
 *                      free-run recount from the views and meals
 *   or_lstm_mag, or_pc_mag (test support: error magnitudes of the outputs)
 *                      pinned: simulated low-precision evaluations (every
 *                      operation rounded to a short mantissa) stay within
 *                      the bound and come close to it; FP32 evaluations in
 *                      several summation orders; bias-only closed form
 */
#ifndef ECOEVO_ORACLE_H
#define ECOEVO_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Fixed controller shape: 7x7x3 observation + energy, LSTM hidden 32,
 * 5 actions (App. B.2; controller of the 200x400 workloads). */
#define OR_VIEW 7
#define OR_NOBS 148              /* 7*7*3 + 1 */
#define OR_HID 32
#define OR_NIN (OR_NOBS + OR_HID) /* 180 */
#define OR_NGATE (4 * OR_HID)    /* 128 */
#define OR_NACT 5
/* Logical parameter vector of one agent. */
#define OR_OFF_B (OR_NGATE * OR_NIN)          /* 23040: gate biases   */
#define OR_OFF_WO (OR_OFF_B + OR_NGATE)       /* 23168: output matrix */
#define OR_OFF_BO (OR_OFF_WO + OR_NACT * OR_HID) /* 23328: output bias */
#define OR_NPARAM (OR_OFF_BO + OR_NACT)       /* 23333 */

/* Philox stream tags (second-to-last counter word). */
#define OR_TAG_REGROW 1u
#define OR_TAG_PLACE 2u
#define OR_TAG_RES_INIT 3u
#define OR_TAG_INIT_W 4u
#define OR_TAG_MUT 5u
#define OR_TAG_ACT 6u            /* action sampling of the paper controller */

/* Controllers (OrParams.controller). */
#define OR_CTRL_LSTM32 0         /* LSTM(32) on the 7x7 view + energy, argmax   */
#define OR_CTRL_PAPER 1          /* CNN -> LSTM(4) -> dense(8) -> dense(5),
                                    softmax at temperature 1/50, sampled (App. B.5) */

/* Paper controller (App. B.5).  Input: the 15x15 view with 3 channels
 * (resource, other agent, wall), row-major [y][x][channel]; off-grid cells
 * read as wall.  conv1 3x3 stride 2 "same" (pad 1) -> 8x8x4; average pool
 * 2x2 stride 1 -> 7x7x4; conv2 3x3 stride 2 "same" (pad 1) -> 4x4x8;
 * average pool -> 3x3x8, flattened [y][x][channel] (72); embedding = those
 * 72, the previous action one-hot (5), the ate-last-step bit (1) = 78;
 * LSTM with 4 units; [embedding, h'] (82) -> dense 8 + tanh -> dense 5.
 * Logical parameter vector (2445 floats): */
#define OR_PC_VIEW 15
#define OR_PC_NOBS (15 * 15 * 3)   /* 675 */
#define OR_PC_HID 4
#define OR_PC_EMB 78
#define OR_PC_W1 0                 /* conv1 [4 out][3 ky][3 kx][3 in]          */
#define OR_PC_B1 108               /* [4]                                      */
#define OR_PC_W2 112               /* conv2 [8 out][3][3][4 in]                */
#define OR_PC_B2 400               /* [8]                                      */
#define OR_PC_WI 408               /* LSTM input kernel [16][78], row = gate*4 + unit, gates i,f,g,o */
#define OR_PC_WH 1656              /* LSTM recurrent kernel [16][4]            */
#define OR_PC_BL 1720              /* LSTM bias [16]                           */
#define OR_PC_D1 1736              /* dense [8][82]                            */
#define OR_PC_DB1 2392             /* [8]                                      */
#define OR_PC_D2 2400              /* dense [5][8]                             */
#define OR_PC_DB2 2440             /* [5]                                      */
#define OR_PC_NPARAM 2445
#define OR_PC_INV_TEMP 50.0        /* softmax temperature 1/50                 */

typedef struct OrParams {
  int32_t H, W, capacity, n_agents0;
  int32_t border_walls;     /* 1: rows 0,H-1 and cols 0,W-1 are walls     */
  double res_init_p;        /* Bernoulli density of initial resources      */
  int32_t nbr_shape;        /* 0: square (Chebyshev) radius, 1: diamond    */
  int32_t nbr_radius;       /* 1..3                                        */
  int32_t class_edges[3];   /* class = #edges <= n                         */
  double p_class[4];        /* p_I per class                               */
  int32_t lat_mode;         /* 0: linear top->bottom, 1: (a^x+1)/(a+1)     */
  double lat_top, lat_bottom, lat_alpha;
  double p_spont;           /* spontaneous growth c                        */
  float e0, e_decay, e_gain, e_max;
  float e_repr;
  int32_t t_repr;
  float e_death;
  int32_t t_death, max_age;
  int32_t wall_kills;       /* 1: an agent moving into a wall dies         */
  float w_init_std, mut_std;
  int32_t controller;       /* OR_CTRL_*                                   */
} OrParams;

typedef struct OrWorld OrWorld;

/* Field ids for or_world_field(); each returns a pointer into the world.   */
enum {
  OR_F_RES = 0,      /* uint8  [H*W]  resource present                       */
  OR_F_WALL,         /* uint8  [H*W]                                         */
  OR_F_SLOT_MAP,     /* int32  [H*W]  slot of the agent on the cell, -1 none */
  OR_F_ALIVE,        /* uint8  [C]                                           */
  OR_F_Y,            /* int32  [C]                                           */
  OR_F_X,            /* int32  [C]                                           */
  OR_F_ENERGY,       /* float  [C]                                           */
  OR_F_REPR_CTR,     /* int32  [C]  consecutive steps with energy > e_repr   */
  OR_F_LOW_CTR,      /* int32  [C]  consecutive steps with energy <= e_death */
  OR_F_AGE,          /* int32  [C]                                           */
  OR_F_H,            /* double [C*32]                                        */
  OR_F_C,            /* double [C*32]                                        */
  OR_F_ACTION,       /* int32  [C]  argmax of the last step                  */
  OR_F_LOGITS,       /* double [C*5]                                         */
  OR_F_ATE,          /* uint8  [C]  ate during the last step                 */
  OR_F_WEIGHTS,      /* float  [C*23333] logical parameter vectors           */
  OR_F_COUNTERS,     /* int64  [OR_NCOUNTERS]  see OR_C_*                    */
  OR_F_THR,          /* uint32 [H*4] growth thresholds                       */
  OR_F_BIRTH_PARENT, /* int32  [C]  parents of the last step's births        */
  OR_F_BIRTH_CHILD,  /* int32  [C]  child slots of the last step's births    */
  OR_F_MOVE_ACTION,  /* int32  [C]  action each agent alive at the start of the
                                    last step moved with (0 for the others)  */
  OR_F_PREV_ACTION,  /* int32  [C]  action the agent moved with in its last
                                    step (0 for newborns): a paper-controller
                                    input                                    */
  OR_F_LAB_FLAGS,    /* uint8  [C]  current window: bit 0 resource in view,
                                    bit 1 ate                                */
  OR_F_LAB_T,        /* int32  [C]  windows with a resource in view (T_r)    */
  OR_F_LAB_C,        /* int32  [C]  windows with a consumption (C_r)         */
  OR_F_MAG_H,        /* double [C*32] error magnitude of h (or_lstm_mag)     */
  OR_F_MAG_C,        /* double [C*32] error magnitude of c                   */
  OR_F_MAG_LOGITS,   /* double [C*5]  error magnitude of the logits          */
  OR_NFIELDS
};
enum {
  OR_C_T = 0, OR_C_POP, OR_C_BIRTHS, OR_C_DEATHS, OR_C_DROPPED,
  OR_C_BIRTHS_LAST, OR_C_DEATHS_LAST, OR_C_DROPPED_LAST,
  OR_C_AGENT_STEPS,  /* sum over steps of the agents alive at the step's start */
  OR_NCOUNTERS
};

/* Record of or_world_analysis (App. C metrics), OR_NANALYSIS int64. */
#define OR_MOVE_BINS 17
enum {
  OR_A_T = 0,     /* steps done                                             */
  OR_A_WINDOW,    /* L: steps since the previous analysis (or create/sync)  */
  OR_A_POP,       /* agents alive                                           */
  OR_A_RES,       /* cells holding a resource                               */
  OR_A_DEATHS,    /* deaths during the window                               */
  OR_A_AGE_SUM,   /* sum of their ages at death                             */
  OR_A_MOVERS,    /* agents alive over the whole window                     */
  OR_A_BINS,      /* OR_MOVE_BINS counts: displacement d in bin 17d/(L+1)   */
  OR_NANALYSIS = OR_A_BINS + OR_MOVE_BINS
};

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]);
/* Two standard normals from two uniform words (Box and Muller, 1958). */
void or_box_muller(uint32_t x1, uint32_t x2, double *z0, double *z1);
/* Normal number j of the stream (seed, tag, t, id). */
double or_normal(uint64_t seed, uint32_t tag, uint32_t t, uint32_t id,
                 uint32_t j);
/* out[j] = base[j] + scale * N_j for the 23333 parameters (base NULL reads
 * as zero), N_j = or_normal(seed, tag, t, id, j); the mutation of App. B.3
 * (tag OR_TAG_MUT, t = step, id = parent) and the initial weights (tag
 * OR_TAG_INIT_W, t = 0, id = slot, base NULL). */
void or_fill_normals(uint64_t seed, uint32_t tag, uint32_t t, uint32_t id,
                     float scale, const float *base, float *out);
/* The same for the first n parameters only. */
void or_fill_normals_n(uint64_t seed, uint32_t tag, uint32_t t, uint32_t id,
                       float scale, const float *base, float *out, int n);
/* Parameters per agent of a controller (23333 or 2445), -1 if unknown. */
int or_param_count(int controller);
/* Paper controller (App. B.5): the 15x15x3 view of the agent at (y, x). */
void or_pc_observe(const OrParams *p, const uint8_t *res, const uint8_t *wall,
                   const int32_t *slot_map, int32_t y, int32_t x,
                   double *obs /* [675] */);
/* One forward step: h, c [4] updated in place, logits [5] written. */
void or_pc_forward(const float *w /* [2445] */, const double *obs, int prev_action,
                   int ate, double *h, double *c, double *logits);
/* Uniform of the action draw of slot s at step t: word 0 of the Philox
 * block {s, t, OR_TAG_ACT, 0}, u = (word >> 8) 2^-24. */
double or_action_uniform(uint64_t seed, uint32_t t, uint32_t slot);
/* Sampled action: probabilities softmax(50 logits); the action is the
 * number of k in 0..3 whose cumulative probability is <= u. */
int or_pc_sample(const double *logits, double u);
/* Growth thresholds thr[y*4+cls] = floor(p * 2^32), App. B.1 Eq. (1). */
int or_threshold_table(const OrParams *p, uint32_t *thr);
/* One synchronous regrowth pass, App. B.1 Eq. (1). */
void or_regrow(const OrParams *p, uint64_t seed, uint32_t t,
               const uint32_t *thr, const uint8_t *res_old,
               const uint8_t *wall, uint8_t *res_new);
/* Observation of the agent at (y, x), App. B.2 (sensorimotor ability). */
void or_observe(const OrParams *p, const uint8_t *res, const uint8_t *wall,
                const int32_t *slot_map, int32_t y, int32_t x, float energy,
                double *obs /* [148] */);
/* One LSTM step + linear read-out + argmax, App. B.2 (cognitive capacity).
 * h and c are updated in place; returns the action. */
int or_lstm_step(const float *w /* [23333] */, const double *obs,
                 double *h, double *c, double *logits);

/* Test support (not part of the method): first-order error magnitudes of
 * one controller step's outputs by running error analysis, so that an
 * evaluation whose operations each round with relative error <= eps lies
 * within eps * E of the exact outputs.  eh, ec: magnitudes of the inputs h,
 * c (0 when exact); writes E of h', c' and of the 5 logits.  The outputs
 * may alias eh, ec.  or_world_step keeps them per slot (OR_F_MAG_*). */
void or_lstm_mag(const float *w, const double *obs, const double *h, const double *c,
                 const double *eh, const double *ec, double *eh_out, double *ec_out,
                 double *el_out);
void or_pc_mag(const float *w, const double *obs, int prev_action, int ate, const double *h,
               const double *c, const double *eh, const double *ec, double *eh_out,
               double *ec_out, double *el_out);
/* Whether or_world_step keeps the magnitudes (on at create).  Off, they
 * keep their last values and nothing else of a step changes. */
void or_world_track_magnitudes(OrWorld *w, int on);

/* Initial walls, resources and agent cells (cells[s] = y*W + x of slot s,
 * s < n_agents0) of a world created from `seed`; the first part of
 * or_world_create.  Returns 0, -1 (invalid / too many agents), -2. */
int or_initial_layout(const OrParams *p, uint64_t seed, uint8_t *res, uint8_t *wall,
                      int32_t *cells);
int or_world_create(const OrParams *p, uint64_t seed, OrWorld **out);
void or_world_destroy(OrWorld *w);
/* One step.  forced: NULL, or [C] actions used for moving instead of the
 * controller's own argmax (the controller still runs). */
int or_world_step(OrWorld *w, const int32_t *forced);
void *or_world_field(OrWorld *w, int field);
/* Test hook: visit slots in the order perm[0..C-1] (a permutation of the
 * slots; NULL restores ascending order) in the per-slot loops whose result
 * the method defines independently of the order -- observation and
 * controller, move claims and moves, eating, physiology and death, birth
 * claims.  The ranking of births (k-th successful parent in ascending slot
 * order, k-th free slot) is an order the method defines and stays
 * ascending.  Returns 0, -1 (not a permutation), -2 (out of memory). */
int or_world_set_order(OrWorld *w, const int32_t *perm);
/* Rebuild slot_map from alive/y/x and the threshold table from the params,
 * after a caller has written state into the fields.  Returns 0, or -1 if
 * two agents share a cell, an agent sits on a wall or off the grid, or an
 * age is negative. */
int or_world_sync(OrWorld *w);
/* Metrics of the paper's analyses (App. C) for the window that ends now,
 * then a new window starts: out[OR_NANALYSIS], see OR_A_*.  Life
 * expectancy over a run of windows = sum of OR_A_AGE_SUM / sum of
 * OR_A_DEATHS.  create and sync start a window with fresh identities. */
int or_world_analysis(OrWorld *w, int64_t *out);
/* Lab-environment greediness G = C_r / T_r (App. C): ends the current
 * window (the paper's are 20 steps): every living agent adds 1 to T_r if a
 * resource was in its view during the window and 1 to C_r if it ate. */
void or_world_lab_window(OrWorld *w);

#ifdef __cplusplus
}
#endif
#endif
