// ecoevo_dev.cuh -- device-side data layout and helpers shared by the
// kernels of libecoevo (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ecoevo.h"

namespace eco {

// ---------------------------------------------------------------------------
// Controller shape and the physical weight layout in HBM.
// ---------------------------------------------------------------------------
constexpr int NOBS = 148;            // 7*7*3 + energy
constexpr int HID = 32;
constexpr int NIN = NOBS + HID;      // 180
constexpr int NGATE = 4 * HID;       // 128
constexpr int NACT = 5;
constexpr int NPARAM = 23333;        // logical parameter vector
constexpr int OFF_B = NGATE * NIN;   // 23040
constexpr int OFF_WO = OFF_B + NGATE;     // 23168
constexpr int OFF_BO = OFF_WO + NACT * HID; // 23328

// An agent's weights are stored as four hidden-unit blocks followed by the
// read-out.  Block q holds the 32 gate rows of hidden units 8q..8q+7, row l
// of the block being gate (l % 4) of hidden unit 8q + l/4, each row the 180
// input weights, then the 32 biases of those rows.  One block is the unit of
// work of the LSTM kernel: it carries every gate of its hidden units, so the
// cell update needs nothing from the other blocks.
constexpr int BLK_ROWS = 32;
constexpr int BLK_FLOATS = BLK_ROWS * NIN + BLK_ROWS;   // 5792
constexpr int BLK_BYTES = BLK_FLOATS * 4;               // 23168 (16-B multiple)
constexpr int NBLK = 4;
constexpr int TAIL = NBLK * BLK_FLOATS;                 // 23168 == OFF_WO
constexpr int WSTRIDE = 23360;                          // floats, 128-B multiple
static_assert(TAIL == OFF_WO, "read-out sits at its logical offset");
static_assert((WSTRIDE * 4) % 128 == 0 && WSTRIDE >= NPARAM, "stride");

// Logical gate row of row l of block q.
__host__ __device__ inline int blk_row_to_logical(int q, int l) {
  return (l & 3) * HID + 8 * q + (l >> 2);
}
// Physical float offset of logical parameter j.
__host__ __device__ inline int phys_of_logical(int j) {
  if (j >= OFF_WO) return j;
  int r = (j < OFF_B) ? j / NIN : j - OFF_B;
  int gate = r / HID, jj = r % HID;
  int q = jj >> 3, l = ((jj & 7) << 2) | gate;
  if (j < OFF_B) return q * BLK_FLOATS + l * NIN + (j % NIN);
  return q * BLK_FLOATS + BLK_ROWS * NIN + l;
}
// Logical parameter of physical float offset p, or -1 for padding.
__host__ __device__ inline int logical_of_phys(int p) {
  if (p >= TAIL) return p < NPARAM ? p : -1;
  int q = p / BLK_FLOATS, o = p % BLK_FLOATS;
  if (o < BLK_ROWS * NIN) {
    int l = o / NIN, k = o % NIN;
    return blk_row_to_logical(q, l) * NIN + k;
  }
  return OFF_B + blk_row_to_logical(q, o - BLK_ROWS * NIN);
}

// Philox stream tags (third counter word).
constexpr uint32_t TAG_REGROW = 1u, TAG_PLACE = 2u, TAG_RES_INIT = 3u,
                   TAG_INIT_W = 4u, TAG_MUT = 5u, TAG_ACT = 6u;

// The paper's controller (App. B.5): parameters in logical order, one row
// of PC_WSTRIDE floats per slot (16-byte multiple, padding zero).
constexpr int PC_NPARAM = 2445;
constexpr int PC_WSTRIDE = 2448;
constexpr int PC_OFF_W1 = 0, PC_OFF_B1 = 108, PC_OFF_W2 = 112, PC_OFF_B2 = 400,
              PC_OFF_WI = 408, PC_OFF_WH = 1656, PC_OFF_BL = 1720, PC_OFF_D1 = 1736,
              PC_OFF_DB1 = 2392, PC_OFF_D2 = 2400, PC_OFF_DB2 = 2440;
constexpr int PC_HID = 4, PC_EMB = 78, PC_VIEW = 15;

// Status bits written by kernels.
constexpr int ST_TIMEOUT = 1;
constexpr int ST_STATE = 2;
constexpr int ST_BOUNDS = 4;

// Range check of an index read from device memory.  In the checked build
// (ECO_CHECKED) a failed check sets ST_BOUNDS in the world's status word and
// the caller skips the access; otherwise the check compiles away.
#ifdef ECO_CHECKED
#define ECO_IN_RANGE(wd, cond) \
  ((cond) ? true : (atomicOr(&(wd).ctr->status, ST_BOUNDS), false))
#else
#define ECO_IN_RANGE(wd, cond) true
#endif

#ifdef __CUDACC__
struct WorldDev;
// Index i of an array of n entries, read from device memory: in the checked
// build an index out of range is reported and replaced by 0, where a kernel
// cannot skip the work item (a pipeline slot that must be filled).
template <class WD>
__device__ inline int checked_index(const WD &wd, int i, int n) {
#ifdef ECO_CHECKED
  if (i >= 0 && i < n) return i;
  atomicOr(&wd.ctr->status, ST_BOUNDS);
  return 0;
#else
  (void)wd;
  (void)n;
  return i;
#endif
}
#endif

// ---------------------------------------------------------------------------
// Per-world device structures.
// ---------------------------------------------------------------------------
struct Counters {            // mutable, updated by the kernels
  long long t, pop, births, deaths, dropped, births_last, deaths_last,
      dropped_last, agent_steps;
  int deaths_step;           // atomically accumulated during a step
  int n_births;              // births of the step, read by the spawn kernel
  unsigned births_t;         // step index the births belong to
  int use_forced;            // moves read `forced` instead of `action`
  int status;                // ST_* bits
  int pad[3];
  // analysis window (App. C): the step it started at, and the deaths and
  // summed ages at death since then
  long long snap_t, an_deaths;
  unsigned long long an_age_sum;
  // per-step counter log in mapped page-locked host memory (null: off):
  // the end of step t writes the first ECO_NCOUNTERS fields to row t % log_rows
  long long *log;
  long long log_rows;
};

// Record of the analysis kernels, in the order of the C ABI's EcoAnalysis.
constexpr int MOVE_BINS = 17;
enum { A_T = 0, A_WINDOW, A_POP, A_RES, A_DEATHS, A_AGE_SUM, A_MOVERS, A_BINS,
       ANALYSIS_WORDS = A_BINS + MOVE_BINS };

struct WorldDev {            // read-only while kernels run
  int H, W, Wp, C;
  int controller;            // ECO_CTRL_*
  int wstride, nparam;       // weight row stride (floats) and parameters per agent
  int nbr_shape, nbr_radius;
  int class_edges[3];
  int t_repr, t_death, max_age, wall_kills;
  float e0, e_decay, e_gain, e_max, e_repr, e_death, mut_std, w_init_std;
  uint32_t key0, key1;
  uint32_t *thr;             // [H][4]
  uint32_t *res0, *res1;     // bit planes [H][Wp]; current = t even ? res0 : res1
  uint32_t *wall;            // [H][Wp]
  int32_t *slot_map;         // [H*W]  -1 free
  int32_t *claim;            // [H*W]  INT32_MAX free (move claims)
  int32_t *bclaim;           // [H*W]  INT32_MAX free (birth claims)
  uint8_t *alive, *killed, *ate, *flag;
  int32_t *y, *x;
  float *energy;
  int32_t *repr_ctr, *low_ctr, *age;
  int32_t *action, *forced, *target, *birth_cell;
  uint32_t *arrive;          // LSTM block arrivals per slot
  float *h0, *h1;            // [C][32]; h read at step t = t even ? h0 : h1
  float *c;                  // [C][32]
  float *logits;             // [C][8]
  int32_t *alive_list;       // [C] slots alive at the start of the step
  uint8_t *alive_new;        // [C] alive_list[i] received a child in the last step
                             // (its weights come from the next step's tail kernel)
  int32_t *free_list, *birth_parent, *birth_child;  // [C]
  float *weights;            // [C][WSTRIDE], 256-B aligned
  Counters *ctr;
  int32_t *snap_cell;        // [C] cell of each slot's agent at the window start, -1 none
  int32_t *prev_act;         // [C] action moved with in the last step (paper controller input)
  uint8_t *lab_seen, *lab_ate;  // [C] greediness window: a resource in view / a meal
                             // (plain stores, no read-modify-write, in the hot kernels)
  int32_t *lab_t, *lab_c;    // [C] windows with a resource in view / with a meal
  int32_t *scan_blocks;      // [(ceil(C/SLOT_BLOCK) + 1) * 4] per-block counts of the
                             // split compaction (free, successful parents, survivors)
  unsigned long long *analysis;  // [ANALYSIS_WORDS] output of the analysis kernels
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11) and normals.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ inline U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
#ifdef __CUDA_ARCH__
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
#else
    uint64_t p0 = 0xD2511F53ull * c.x, p1 = 0xCD9E8D57ull * c.z;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

#ifdef __CUDACC__
// ln(u), u = (x1 + 1/2) 2^-32, in float with no branch.  u = 2^e (1 + f),
// f in [sqrt(1/2) - 1, sqrt(2) - 1), taken from the integer word: from u
// itself when x1 < 2^31 (u < 1/2); when u >= 1/2 from 1 - u = (~x1 + 1/2)
// 2^-32, which a float holds exactly, so that ln of a u close to 1 keeps its
// relative accuracy (e = 0, f = u - 1 = -(1 - u), or e = -1, f = 2u - 1).
// Then ln(1 + f) = 2 atanh(s) with s = f / (2 + f), |s| < 0.1716 (the
// quotient by the hardware's approximate division, within 2 ulp), by the
// Taylor series of atanh up to s^9 (the next term is below 2e-10 of the
// sum), and e ln 2 with ln 2 split in two (Cody and Waite) so that e ln2_hi
// is exact.
__device__ inline float ln_unit_word(uint32_t x1) {
  const bool upper = x1 >= 0x80000000u;
  const float v = ((float)(upper ? ~x1 : x1) + 0.5f) * 2.3283064365386963e-10f;  // 2^-32
  // u = v < 1/2: exponent and mantissa of v
  const uint32_t bits = __float_as_uint(v);
  int e_lo = (int)((bits >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);   // [1, 2)
  const bool big = m >= 1.41421356f;
  m = big ? 0.5f * m : m;
  e_lo += big ? 1 : 0;
  const float f_lo = m - 1.0f;                                     // exact
  // u = 1 - v >= 1/2
  const bool near_one = v <= 0.29289322f;                          // 1 - sqrt(1/2)
  const float f_up = near_one ? -v : 1.0f - 2.0f * v;              // exact
  const int e_up = near_one ? 0 : -1;
  const float f = upper ? f_up : f_lo;
  const float e = (float)(upper ? e_up : e_lo);
  const float s = __fdividef(f, 2.0f + f);
  const float s2 = s * s;
  float q = fmaf(s2, 1.0f / 9.0f, 1.0f / 7.0f);
  q = fmaf(s2, q, 1.0f / 5.0f);
  q = fmaf(s2, q, 1.0f / 3.0f);
  const float two_s = 2.0f * s;
  const float l = fmaf(two_s * s2, q, two_s);                      // ln(1 + f)
  return fmaf(e, 0.693145751953125f, fmaf(e, 1.4286067653e-06f, l));
}

// Square root of x > 0: x rsqrt(x) from the hardware's approximate
// reciprocal square root, then one Newton-Raphson (Heron) step, r + (x -
// r^2) / (2 r) with 1/r taken as rsqrt(x).
__device__ inline float sqrt_pos(float x) {
  const float y = rsqrtf(x);
  const float r = x * y;
  return fmaf(fmaf(-r, r, x), 0.5f * y, r);
}

// Box-Muller pair from two words, in float, with no branch: r = sqrt(-2 ln
// u1) (-2 ln u1 > 2e-10: u1 < 1 - 2^-33); the angle (pi/2)(quad + g), quad = the top two bits of x2 and g =
// (low 30 bits + 1/2) 2^-30, is reduced to a in (0, pi/4): a = (pi/2) g when
// g < 1/2, else the complement (pi/2)(1 - g) with 1 - g taken exactly from
// the complemented bits (and cos and sin swapped); sin a and cos a by their
// Taylor series up to a^9 and a^10 (next terms below 2e-9).
__device__ inline void box_muller_f(uint32_t x1, uint32_t x2, float &z0, float &z1) {
  const float r = sqrt_pos(-2.0f * ln_unit_word(x1));
  const uint32_t quad = x2 >> 30;
  const bool upper = (x2 >> 29) & 1u;
  const uint32_t y = (upper ? ~x2 : x2) & 0x1FFFFFFFu;
  const float a = ((float)y + 0.5f) * (1.5707963705062866f * 9.313225746154785e-10f);
  const float a2 = a * a;
  float ps = fmaf(a2, 1.0f / 362880.0f, -1.0f / 5040.0f);
  ps = fmaf(a2, ps, 1.0f / 120.0f);
  ps = fmaf(a2, ps, -1.0f / 6.0f);
  const float sa = fmaf(a * a2, ps, a);
  float pc = fmaf(a2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
  pc = fmaf(a2, pc, -1.0f / 720.0f);
  pc = fmaf(a2, pc, 1.0f / 24.0f);
  pc = fmaf(a2, pc, -0.5f);
  const float ca = fmaf(a2, pc, 1.0f);
  const float c = upper ? sa : ca, s = upper ? ca : sa;   // cos, sin of (pi/2) g
  float cs, sn;
  switch (quad) {
    case 0: cs = c; sn = s; break;
    case 1: cs = -s; sn = c; break;
    case 2: cs = -c; sn = -s; break;
    default: cs = s; sn = -c; break;
  }
  z0 = r * cs;
  z1 = r * sn;
}

// Four normals of the draw {q, t, tag, id}: (cos, sin) of lanes (0,1), then
// of lanes (2,3).
__device__ inline void normals4(uint32_t k0, uint32_t k1, uint32_t q,
                                uint32_t t, uint32_t tag, uint32_t id,
                                float z[4]) {
  U4 r = philox4x32_10(U4{q, t, tag, id}, k0, k1);
  box_muller_f(r.x, r.y, z[0], z[1]);
  box_muller_f(r.z, r.w, z[2], z[3]);
}

__device__ inline bool bit_at(const uint32_t *plane, int Wp, int y, int x) {
  return (plane[y * Wp + (x >> 5)] >> (x & 31)) & 1u;
}


#endif

// ---------------------------------------------------------------------------
// Kernel launchers (one per kernel source).
// ---------------------------------------------------------------------------
struct BatchDev {
  WorldDev w0;               // descriptor of worlds[0], carried in the launch
  WorldDev *const *worlds;   // device array [n]
  int n;
  int *tile_prefix;          // device [n+1]: regrowth tiles per world
  int regrow_k;              // 8-row tiles stacked in one regrowth CTA (1, 2, 4, 8)
  int lstm_ctas;             // controller-kernel CTAs per SM (1 or 2)
  int pdl;                   // host side: launch with programmatic dependent launch
  int *slot_block_prefix;    // device [n+1]: 256-slot blocks per world
  int total_tiles, total_slot_blocks;
  int max_capacity;
  int n_sms;
  int fused;                 // slot phases in one cluster kernel (capacity <= FUSED_MAX_C)
  int spawn_ctas;            // CTAs of the tail kernel that mutate births
  int tail_early;            // the tail kernel lets the next kernel launch at its start
                             // (its grid is at most 2 CTAs per SM), else at its end
  int controller, wstride;   // shared by every world of the batch
};

#ifdef __CUDACC__
// Programmatic dependent launch: a step kernel lets the next one be scheduled
// as soon as it starts, and waits for the previous one to complete (and its
// memory to be visible) before it reads anything.  Without the launch
// attribute both are no-ops.
__device__ inline void pdl_wait_and_release() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ inline void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ inline void pdl_release() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch a step kernel, with the programmatic-stream-serialization
// attribute unless b.pdl is 0 (kernels timed one by one between events).
template <typename Kernel>
inline void launch_step_kernel(Kernel k, int grid, int block, size_t smem, cudaStream_t s,
                               const BatchDev &b) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = b.pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, b);
}

// Descriptor of world w.  Kernels take the batch as a __grid_constant__
// parameter, so for a batch of one the descriptor is read from the launch's
// constant bank instead of global memory.
__device__ inline const WorldDev *world_ptr(const BatchDev &b, int w) {
  return b.n == 1 ? &b.w0 : b.worlds[w];
}
#endif

// Worlds up to this capacity run all slot phases of a step in one cluster.
constexpr int FUSED_MAX_C = 16384;

void launch_lstm(const BatchDev &b, cudaStream_t s);
void launch_paper_ctrl(const BatchDev &b, cudaStream_t s);   // k_paper.cu
void preload_paper();
void launch_move_apply(const BatchDev &b, cudaStream_t s);
void launch_physio(const BatchDev &b, cudaStream_t s);
void launch_birth_claim(const BatchDev &b, cudaStream_t s);
// the split compaction, for worlds of any capacity: four kernels
void launch_scan_count(const BatchDev &b, cudaStream_t s);
void launch_scan_prefix(const BatchDev &b, cudaStream_t s);
void launch_scan_lists(const BatchDev &b, cudaStream_t s);
void launch_scan_children(const BatchDev &b, cudaStream_t s);
void launch_tail(const BatchDev &b, cudaStream_t s);   // regrowth of t + births of t-1
void launch_agents_fused(const BatchDev &b, cudaStream_t s);
void configure_lstm();   // once per device, before the first launch
void launch_wait_selftest(int *status, unsigned long long limit_ns, cudaStream_t s);
// Load every step kernel's code before a step is captured in a graph.
void preload_lstm();
void preload_agents();
// set-up and state I/O
void launch_init_world(const WorldDev *wd_host, WorldDev *wd_dev, int n0,
                       const int32_t *place_y, const int32_t *place_x,
                       int border, uint32_t thr_init, int n_sms, cudaStream_t s);
void launch_rebuild(const WorldDev *wd_host, int n_sms, cudaStream_t s);
// Physical rows of `wstride` floats -> logical rows of `lpitch` floats
// (device memory or the device address of page-locked host memory);
// ECO_CTRL_LSTM32 rows are permuted, ECO_CTRL_PAPER rows are in logical order
// already (copied).
void launch_weights_to_logical(const float *physical, float *logical, size_t lpitch, int n,
                               int controller, int n_sms, cudaStream_t s);
// n packed logical rows in page-locked host memory (its device address,
// 16-byte aligned) -> the physical rows; returns a cudaError_t value
// (cudaErrorMisalignedAddress: not 16-byte aligned, nothing launched).
int launch_weights_from_host(const float *host_dev, float *rows, int n, int controller,
                             int n_sms, cudaStream_t s);
// n rows of the weight array holding logical rows (copied there) -> physical
// order, in place; returns a cudaError_t value.
int launch_rows_to_physical_inplace(float *rows, int n, int controller, int n_sms,
                                    cudaStream_t s);
// Counters of a loaded state: with set, the cumulative ones (t .. agent_steps
// but pop, which the rebuild counts); always the per-step ones zeroed.
struct LoadCounters {
  long long t, births, deaths, dropped, births_last, deaths_last, dropped_last, agent_steps;
  int set;
};
void launch_load_counters(Counters *ctr, const LoadCounters &v, cudaStream_t s);
// A plane of one byte per cell (nonzero: set; device memory or the device
// address of page-locked host memory) -> H x Wp words.
void launch_pack_plane(const uint8_t *cells, int H, int W, int Wp, uint32_t *words,
                       cudaStream_t s);
// Slot arrays of a loaded state read from page-locked host memory through
// their device addresses (null: not read here); logits are C x NACT on the
// host, C x 8 on the device; h goes to h_dst (the current buffer).
struct SlotSources {
  const uint8_t *alive, *ate;
  const int32_t *y, *x, *repr, *low, *age, *action, *prev;
  const float *energy, *logits, *h, *c;
};
void launch_load_slots(const WorldDev &wd, const SlotSources &src, float *h_dst, int n_sms,
                       cudaStream_t s);
// analysis metrics of App. C (k_analysis.cu)
void launch_analysis_reset(const WorldDev *wd_host, int n_sms, cudaStream_t s);
void launch_analysis(const WorldDev *wd_host, int n_sms, cudaStream_t s);
void launch_lab_window(const WorldDev *wd_host, int n_sms, cudaStream_t s);

constexpr int SCAN_THREADS = 1024;
constexpr int SLOT_BLOCK = 256;
constexpr int REGROW_ROWS = 8, REGROW_WORDS = 4;
constexpr int REGROW_KMAX = 8;   // 8-row tiles stacked in one regrowth CTA, at most

// Regrowth CTAs of a world (columns of k stacked tiles).
inline int regrow_tiles_of(int H, int Wp, int k) {
  const int rows = REGROW_ROWS * k;
  return ((H + rows - 1) / rows) * ((Wp + REGROW_WORDS - 1) / REGROW_WORDS);
}

}  // namespace eco
