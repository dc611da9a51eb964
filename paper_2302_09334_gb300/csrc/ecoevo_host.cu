// ecoevo_host.cu -- the C ABI of libecoevo (include/ecoevo.h): world
// layout in one device arena, creation, stepping (CUDA graphs of whole
// steps), state I/O, batches and per-kernel profiling.
#include <algorithm>
#include <cstddef>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ecoevo_dev.cuh"

using namespace eco;

namespace {

// NVTX range over one call of the C ABI (a chunk of steps, a state copy, an
// analysis): visible to profilers that record NVTX, free otherwise.
struct Trace {
  explicit Trace(const char *name) { nvtxRangePushA(name); }
  ~Trace() { nvtxRangePop(); }
  Trace(const Trace &) = delete;
  Trace &operator=(const Trace &) = delete;
};

}  // namespace

namespace {

constexpr int STEPS_PER_GRAPH = 16;     // default chunk graph length
constexpr int DEFAULT_SPAWN_PER_SM = 4;  // default mutation CTAs of the tail kernel per SM
// Weights move between host (logical order) and device (physical order)
// through a staging region of this many agents, permuted on the device.
constexpr int STAGING_AGENTS = 64;

// ---------------------------------------------------------------------------
// Parameters and the arena layout.
// ---------------------------------------------------------------------------
bool params_ok(const EcoParams *p) {
  if (!p || p->abi_version != ECO_ABI_V2) return false;
  if (p->controller != ECO_CTRL_LSTM32 && p->controller != ECO_CTRL_PAPER) return false;
  if (p->H < 1 || p->W < 1 || p->H > 16384 || p->W > 16384) return false;
  if ((long long)p->H * p->W > (1ll << 26)) return false;
  if (p->capacity < 0 || p->capacity > (1 << 24)) return false;
  if (p->n_agents0 < 0 || p->n_agents0 > p->capacity) return false;
  if (p->nbr_shape != 0 && p->nbr_shape != 1) return false;
  if (p->nbr_radius < 1 || p->nbr_radius > 3) return false;
  if (!(p->class_edges[0] <= p->class_edges[1] && p->class_edges[1] <= p->class_edges[2]))
    return false;
  if (p->lat_mode != 0 && p->lat_mode != 1) return false;
  if (p->t_repr < 0 || p->t_death < 0 || p->max_age < 0) return false;
  if (p->border_walls != 0 && p->border_walls != 1) return false;
  return true;
}

// Weight row stride (floats) and parameters per agent of a controller.
int wstride_of(int controller) { return controller == ECO_CTRL_PAPER ? PC_WSTRIDE : WSTRIDE; }
int nparam_of(int controller) { return controller == ECO_CTRL_PAPER ? PC_NPARAM : NPARAM; }

struct Layout {
  size_t ctr, wdev, tab_worlds, tab_tiles, tab_blocks, thr, res0, res1, wall,
      slot_map, claim, bclaim, alive, killed, ate, flag, y, x, energy, repr_ctr,
      low_ctr, age, action, forced, target, birth_cell, arrive, h0, h1, c,
      logits, alive_list, alive_new, free_list, birth_parent, birth_child, snap_cell, analysis,
      prev_act, lab_seen, lab_ate, lab_t, lab_c, scan_blocks, weights, staging, total;
};

Layout layout_of(const EcoParams *p) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off += (bytes + 255) & ~(size_t)255;
    return at;
  };
  const size_t H = p->H, W = p->W, Wp = (p->W + 31) / 32, C = p->capacity;
  const size_t C1 = C ? C : 1;
  L.ctr = take(sizeof(Counters));
  L.wdev = take(sizeof(WorldDev));
  L.tab_worlds = take(sizeof(WorldDev *));
  L.tab_tiles = take(2 * sizeof(int));
  L.tab_blocks = take(2 * sizeof(int));
  L.thr = take(H * 4 * 4);
  L.res0 = take(H * Wp * 4);
  L.res1 = take(H * Wp * 4);
  L.wall = take(H * Wp * 4);
  L.slot_map = take(H * W * 4);
  L.claim = take(H * W * 4);
  L.bclaim = take(H * W * 4);
  L.alive = take(C1);
  L.killed = take(C1);
  L.ate = take(C1);
  L.flag = take(C1);
  L.y = take(C1 * 4);
  L.x = take(C1 * 4);
  L.energy = take(C1 * 4);
  L.repr_ctr = take(C1 * 4);
  L.low_ctr = take(C1 * 4);
  L.age = take(C1 * 4);
  L.action = take(C1 * 4);
  L.forced = take(C1 * 4);
  L.target = take(C1 * 4);
  L.birth_cell = take(C1 * 4);
  L.arrive = take(C1 * 4);
  L.h0 = take(C1 * HID * 4);
  L.h1 = take(C1 * HID * 4);
  L.c = take(C1 * HID * 4);
  L.logits = take(C1 * 8 * 4);
  L.alive_list = take(C1 * 4);
  L.alive_new = take(C1);
  L.free_list = take(C1 * 4);
  L.birth_parent = take(C1 * 4);
  L.birth_child = take(C1 * 4);
  L.snap_cell = take(C1 * 4);
  L.analysis = take(ANALYSIS_WORDS * 8);
  L.prev_act = take(C1 * 4);
  L.lab_seen = take(C1);
  L.lab_ate = take(C1);
  L.lab_t = take(C1 * 4);
  L.lab_c = take(C1 * 4);
  L.scan_blocks = take(((C1 + SLOT_BLOCK - 1) / SLOT_BLOCK + 1) * 4 * 4);
  L.weights = take(C1 * (size_t)wstride_of(p->controller) * 4);
  L.staging = take((size_t)STAGING_AGENTS * WSTRIDE * 4);
  L.total = off;
  return L;
}

// Growth thresholds, App. B.1 Eq. (1): p = p_I[class] * climate(row) + c,
// threshold floor(p * 2^32) (0 when p <= 0, 2^32 - 1 when p >= 1); a cell
// grows when its Philox word is below the threshold.
uint32_t threshold_of(double prob) {
  if (!(prob > 0.0)) return 0u;
  if (prob >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)std::floor(prob * 4294967296.0);
}

std::vector<uint32_t> threshold_table(const EcoParams *p) {
  std::vector<uint32_t> thr((size_t)p->H * 4);
  for (int y = 0; y < p->H; ++y) {
    const double frac = (p->H > 1) ? (double)y / (double)(p->H - 1) : 0.0;
    double climate;
    if (p->lat_mode == 1)
      climate = (std::pow(p->lat_alpha, frac) + 1.0) / (p->lat_alpha + 1.0);
    else
      climate = p->lat_top + (p->lat_bottom - p->lat_top) * frac;
    for (int k = 0; k < 4; ++k) thr[(size_t)y * 4 + k] = threshold_of(p->p_class[k] * climate + p->p_spont);
  }
  return thr;
}

typedef void (*Launcher)(const BatchDev &, cudaStream_t);
struct StepKernel { int id; Launcher fn; };

// Per-kernel timing: a profiled step launches its kernels on the stream
// with an event recorded before and after every kernel (an earlier version
// launched a one-step graph with event-record nodes, which added about 7 us
// of node latency to every kernel's time).  A profiled step returns at
// once; the times of a step are added just before the next profiled step
// (its events are reused) or when they are read.
struct Profile {
  bool on = false;
  int max_steps = 0, used = 0;
  double ms[ECO_NKERNELS] = {0};
  long long launches[ECO_NKERNELS] = {0};
  cudaEvent_t ev[2 * ECO_NKERNELS] = {nullptr};
  int n_ev = 0;
  const void *owner = nullptr;   // the batch whose kernels the events bracket
  const StepKernel *list = nullptr;
  int nk = 0;
  bool pending = false;      // a launch whose times are not yet added
};

}  // namespace

// ---------------------------------------------------------------------------
// Opaque handles.
// ---------------------------------------------------------------------------
struct EcoBatch {
  std::vector<EcoWorld *> worlds;
  BatchDev bd{};
  cudaStream_t stream = nullptr;
  void *table = nullptr;  // device: worlds[], tile prefix, block prefix
  bool owns_table = false;
  cudaGraphExec_t g1 = nullptr, gk = nullptr;
  int steps_per_graph = STEPS_PER_GRAPH;  // steps in the chunk graph gk
  int regrow_cfg = 0;     // regrowth tiles stacked per CTA as set (0: chosen by size)
  Profile *prof = nullptr;  // the first world's profiler
};

struct EcoWorld {
  EcoParams p{};
  uint64_t seed = 0;
  int device = 0;
  int n_sms = 0;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  size_t arena_bytes = 0;
  bool owns_arena = false;
  Layout L{};
  WorldDev hd{};          // host copy of the device descriptor
  WorldDev *dd = nullptr; // device descriptor
  EcoBatch self;          // batch of one: this world
  Profile prof;
  // second stream of state loads (the weight rows' upload runs on it beside
  // the rest), created at the first load
  cudaStream_t io_stream = nullptr;
  cudaEvent_t io_fork = nullptr, io_join = nullptr;
};

namespace {

int cuda_err_at(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return ECO_OK;
  std::fprintf(stderr, "libecoevo: CUDA error %s in %s\n", cudaGetErrorString(e), what);
  return ECO_ECUDA;
}
#define cuda_err(call) cuda_err_at((call), #call)
#define ECO_CU(call)                                  \
  do {                                                \
    int rc__ = cuda_err_at((call), #call);            \
    if (rc__ != ECO_OK) return rc__;                  \
  } while (0)

// 8-row tiles stacked per regrowth CTA by default: the fewest (1, 2, 4, 8)
// that leave at most four CTAs per SM (one wave of the tail kernel), so that
// a large world's regrowth does not queue in waves behind itself.
int regrow_k_for(EcoWorld *const *worlds, int n, int n_sms) {
  int k = 1;
  for (; k < REGROW_KMAX; k *= 2) {
    long long tiles = 0;
    for (int i = 0; i < n; ++i)
      tiles += regrow_tiles_of(worlds[i]->hd.H, worlds[i]->hd.Wp, k);
    if (tiles <= 4ll * n_sms) break;
  }
  return k;
}
int slot_blocks_of(const WorldDev &wd) { return (wd.C + SLOT_BLOCK - 1) / SLOT_BLOCK; }

// Kernel ids for profiling (names: eco_kernel_name).
enum { K_REGROW, K_LSTM, K_MOVE_CLAIM, K_MOVE_APPLY, K_PHYSIO, K_BIRTH_CLAIM, K_SCAN,
       K_TAIL, K_AGENTS_FUSED, K_PAPER };
// A step starts with the tail kernel: the regrowth of the step's resource
// plane (App. B.1) in the same launch as the mutation of the previous step's
// births (they touch disjoint data; newborns act from the step after their
// birth, so their weights are needed only by this step's controller).  The
// observation+controller kernel also makes the move claims; the slot phases
// end the step.  In a graph, the tail kernel is thus followed by the
// controller kernel, which starts its reads of slot state and non-newborn
// weights while the tail runs (programmatic dependent launch).
// (the four kernels of the split compaction are timed together as "scan")
const StepKernel kSplitStep[] = {
    {K_TAIL, launch_tail}, {K_LSTM, launch_lstm},
    {K_MOVE_APPLY, launch_move_apply}, {K_PHYSIO, launch_physio},
    {K_BIRTH_CLAIM, launch_birth_claim}, {K_SCAN, launch_scan_count},
    {K_SCAN, launch_scan_prefix}, {K_SCAN, launch_scan_lists}, {K_SCAN, launch_scan_children}};
const StepKernel kFusedStep[] = {{K_TAIL, launch_tail},
                                 {K_LSTM, launch_lstm},
                                 {K_AGENTS_FUSED, launch_agents_fused}};
// the same with the paper's controller
const StepKernel kSplitStepPaper[] = {
    {K_TAIL, launch_tail}, {K_PAPER, launch_paper_ctrl},
    {K_MOVE_APPLY, launch_move_apply}, {K_PHYSIO, launch_physio},
    {K_BIRTH_CLAIM, launch_birth_claim}, {K_SCAN, launch_scan_count},
    {K_SCAN, launch_scan_prefix}, {K_SCAN, launch_scan_lists}, {K_SCAN, launch_scan_children}};
const StepKernel kFusedStepPaper[] = {{K_TAIL, launch_tail},
                                      {K_PAPER, launch_paper_ctrl},
                                      {K_AGENTS_FUSED, launch_agents_fused}};

static_assert(sizeof(kSplitStep) / sizeof(kSplitStep[0]) <= ECO_NKERNELS,
              "the profiler keeps two events per kernel of a step, for up to ECO_NKERNELS");

int step_kernels(const BatchDev &bd, const StepKernel **list) {
  const bool paper = bd.controller == ECO_CTRL_PAPER;
  if (bd.fused) {
    *list = paper ? kFusedStepPaper : kFusedStep;
    return (int)(sizeof(kFusedStep) / sizeof(kFusedStep[0]));
  }
  *list = paper ? kSplitStepPaper : kSplitStep;
  return (int)(sizeof(kSplitStep) / sizeof(kSplitStep[0]));
}

// One step, kernel by kernel; with `ev`, a pair of events around every
// kernel (not while capturing a graph).
// The kernels of one step; with events (profiling) each kernel is
// bracketed by two and launched without programmatic dependent launch,
// which the events between kernels rule out anyway.
void launch_step(const EcoBatch &b, cudaStream_t s, cudaEvent_t *ev) {
  const StepKernel *list;
  const int nk = step_kernels(b.bd, &list);
  BatchDev bd = b.bd;
  if (ev) bd.pdl = 0;
  for (int k = 0; k < nk; ++k) {
    if (ev) cudaEventRecord(ev[2 * k], s);
    list[k].fn(bd, s);
    if (ev) cudaEventRecord(ev[2 * k + 1], s);
  }
}

void destroy_graphs(EcoBatch &b) {
  if (b.g1) cudaGraphExecDestroy(b.g1);
  if (b.gk) cudaGraphExecDestroy(b.gk);
  b.g1 = b.gk = nullptr;
}

int capture(EcoBatch &b, int steps, cudaGraphExec_t *out) {
  cudaGraph_t g = nullptr;
  ECO_CU(cudaStreamBeginCapture(b.stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < steps; ++i) launch_step(b, b.stream, nullptr);
  cudaError_t e = cudaStreamEndCapture(b.stream, &g);
  if (e != cudaSuccess) return cuda_err(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_err(e);
  // upload now, so that the first launch does not carry it
  return cuda_err(cudaGraphUpload(*out, b.stream));
}

// The tail kernel's grid (regrowth tiles + mutation CTAs) leaves room on
// every SM for a controller CTA when it is at most 2 CTAs per SM.
int tail_early(const BatchDev &bd) {
  return bd.total_tiles + bd.spawn_ctas <= 2 * bd.n_sms ? 1 : 0;
}

// Host side of a batch: device table of descriptors and work prefixes.
int batch_init(EcoBatch &b, EcoWorld *const *worlds, int n, void *table_dev) {
  b.worlds.assign(worlds, worlds + n);
  b.stream = worlds[0]->stream;
  const size_t tab_bytes = n * sizeof(WorldDev *) + 2 * (n + 1) * sizeof(int);
  if (table_dev) {
    b.table = table_dev;
    b.owns_table = false;
  } else {
    ECO_CU(cudaMalloc(&b.table, tab_bytes));
    b.owns_table = true;
  }
  std::vector<char> host(tab_bytes);
  WorldDev **wp = reinterpret_cast<WorldDev **>(host.data());
  int *tiles = reinterpret_cast<int *>(host.data() + n * sizeof(WorldDev *));
  int *blocks = tiles + (n + 1);
  const int rk = regrow_k_for(worlds, n, worlds[0]->n_sms);
  b.regrow_cfg = 0;
  int tt = 0, bb = 0, maxc = 0;
  for (int i = 0; i < n; ++i) {
    wp[i] = worlds[i]->dd;
    tiles[i] = tt;
    blocks[i] = bb;
    tt += regrow_tiles_of(worlds[i]->hd.H, worlds[i]->hd.Wp, rk);
    bb += slot_blocks_of(worlds[i]->hd);
    maxc = std::max(maxc, worlds[i]->hd.C);
  }
  tiles[n] = tt;
  blocks[n] = bb;
  ECO_CU(cudaMemcpy(b.table, host.data(), tab_bytes, cudaMemcpyHostToDevice));
  b.bd.w0 = worlds[0]->hd;
  b.bd.worlds = reinterpret_cast<WorldDev *const *>(b.table);
  b.bd.n = n;
  b.bd.tile_prefix = reinterpret_cast<int *>((char *)b.table + n * sizeof(WorldDev *));
  b.bd.slot_block_prefix = b.bd.tile_prefix + (n + 1);
  b.bd.total_tiles = tt;
  b.bd.regrow_k = rk;
  b.bd.lstm_ctas = 1;
  b.bd.pdl = 1;
  b.bd.total_slot_blocks = bb;
  b.bd.max_capacity = maxc;
  b.bd.n_sms = worlds[0]->n_sms;
  b.bd.fused = maxc <= FUSED_MAX_C ? 1 : 0;
  b.bd.spawn_ctas = DEFAULT_SPAWN_PER_SM * b.bd.n_sms;
  b.bd.tail_early = tail_early(b.bd);
  b.bd.controller = worlds[0]->hd.controller;
  b.bd.wstride = worlds[0]->hd.wstride;
  b.prof = &worlds[0]->prof;
  return ECO_OK;
}

// Events for the kernels of the batch's step.
int profile_setup(EcoBatch &b, Profile &pr) {
  const StepKernel *list;
  const int nk = step_kernels(b.bd, &list);
  for (int k = 0; k < 2 * nk; ++k) ECO_CU(cudaEventCreate(&pr.ev[k]));
  pr.n_ev = 2 * nk;
  pr.owner = &b;
  pr.list = list;
  pr.nk = nk;
  return ECO_OK;
}

void profile_release(Profile &pr) {
  for (int k = 0; k < pr.n_ev; ++k) cudaEventDestroy(pr.ev[k]);
  pr.n_ev = 0;
  pr.owner = nullptr;
  pr.list = nullptr;
  pr.nk = 0;
  pr.pending = false;
}

// Add the per-kernel times of the pending profiled launch, if any.
int profile_collect(Profile &pr) {
  if (!pr.pending) return ECO_OK;
  ECO_CU(cudaEventSynchronize(pr.ev[2 * pr.nk - 1]));
  for (int k = 0; k < pr.nk; ++k) {
    float t = 0.f;
    ECO_CU(cudaEventElapsedTime(&t, pr.ev[2 * k], pr.ev[2 * k + 1]));
    pr.ms[pr.list[k].id] += t;
    pr.launches[pr.list[k].id] += 1;
  }
  pr.pending = false;
  return ECO_OK;
}

// One profiled step: collect the previous launch's times, launch again.
int profiled_step(EcoBatch &b, Profile &pr) {
  int rc = profile_collect(pr);
  if (rc) return rc;
  launch_step(b, b.stream, pr.ev);
  ECO_CU(cudaGetLastError());
  pr.pending = true;
  pr.used += 1;
  return ECO_OK;
}

// Capture (and upload) the graphs an unprofiled batch_step(b, n) launches:
// chunks of steps_per_graph steps, then single steps.
int prepare_graphs(EcoBatch &b, int64_t n) {
  const int k = b.steps_per_graph;
  if (k > 1 && n >= k && !b.gk) {
    int rc = capture(b, k, &b.gk);
    if (rc) return rc;
  }
  const int64_t chunks = k > 1 ? n / k : 0, singles = n - chunks * k;
  if (singles && !b.g1) {
    int rc = capture(b, 1, &b.g1);
    if (rc) return rc;
  }
  return ECO_OK;
}

int batch_step(EcoBatch &b, int64_t n) {
  if (n < 0) return ECO_EINVAL;
  Profile *prof = b.prof;
  if (prof && prof->on) {
    if (prof->owner && prof->owner != &b) {  // profiled last as part of another batch
      int rc = profile_collect(*prof);
      if (rc) return rc;
      profile_release(*prof);
    }
    if (!prof->owner) {
      int rc = profile_setup(b, *prof);
      if (rc) return rc;
    }
    for (int64_t i = 0; i < n; ++i) {
      if (prof->used < prof->max_steps) {
        int rc = profiled_step(b, *prof);
        if (rc) return rc;
      } else {
        launch_step(b, b.stream, nullptr);
      }
    }
    return cuda_err(cudaGetLastError());
  }
  int rc = prepare_graphs(b, n);
  if (rc) return rc;
  const int k = b.steps_per_graph;
  const int64_t chunks = k > 1 ? n / k : 0, singles = n - chunks * k;
  for (int64_t i = 0; i < chunks; ++i) ECO_CU(cudaGraphLaunch(b.gk, b.stream));
  for (int64_t i = 0; i < singles; ++i) ECO_CU(cudaGraphLaunch(b.g1, b.stream));
  return ECO_OK;
}

// ---------------------------------------------------------------------------
// Launch configuration and its tuner.  Every choice here leaves the results
// unchanged (the same kernels compute the same values; only how the work is
// split into launches and CTAs differs), so the tuner times real steps of the
// batch it tunes.
// ---------------------------------------------------------------------------
// Before a launch configuration changes: the stream idle, the graphs (which
// hold the old one) dropped, the profiler's events released.
int reconfigure(EcoBatch &b) {
  ECO_CU(cudaStreamSynchronize(b.stream));
  destroy_graphs(b);
  if (b.prof && b.prof->owner == &b) {  // its events bracket the old kernel list
    int rc = profile_collect(*b.prof);
    if (rc) return rc;
    profile_release(*b.prof);
  }
  return ECO_OK;
}

int set_config(EcoBatch &b, int fused, int spawn_per_sm, int steps_per_graph) {
  if (fused != 0 && fused != 1) return ECO_EINVAL;
  if (fused && b.bd.max_capacity > FUSED_MAX_C) return ECO_EINVAL;
  if (spawn_per_sm < 1 || spawn_per_sm > 32) return ECO_EINVAL;
  if (steps_per_graph < 1 || steps_per_graph > 1024) return ECO_EINVAL;
  const int spawn = spawn_per_sm * b.bd.n_sms;
  if (fused == b.bd.fused && spawn == b.bd.spawn_ctas && steps_per_graph == b.steps_per_graph)
    return ECO_OK;
  int rc = reconfigure(b);
  if (rc) return rc;
  b.bd.fused = fused;
  b.bd.spawn_ctas = spawn;
  b.bd.tail_early = tail_early(b.bd);
  b.steps_per_graph = steps_per_graph;
  return ECO_OK;
}

// Kernel shapes: regrowth tiles stacked per CTA (0: chosen by size; 1, 2,
// 4, 8) and controller-kernel CTAs per SM (1, 2).  A new stacking rewrites
// the batch's tile prefix in its device table.
int set_shape(EcoBatch &b, int regrow_rows, int lstm_ctas) {
  if (regrow_rows != 0 && regrow_rows != 1 && regrow_rows != 2 && regrow_rows != 4 &&
      regrow_rows != 8)
    return ECO_EINVAL;
  if (lstm_ctas != 1 && lstm_ctas != 2) return ECO_EINVAL;
  const int n = (int)b.worlds.size();
  const int k = regrow_rows ? regrow_rows : regrow_k_for(b.worlds.data(), n, b.bd.n_sms);
  if (k == b.bd.regrow_k && lstm_ctas == b.bd.lstm_ctas) {
    b.regrow_cfg = regrow_rows;
    return ECO_OK;
  }
  int rc = reconfigure(b);
  if (rc) return rc;
  b.regrow_cfg = regrow_rows;
  if (k != b.bd.regrow_k) {
    std::vector<int> tiles(n + 1);
    int tt = 0;
    for (int i = 0; i < n; ++i) {
      tiles[i] = tt;
      tt += regrow_tiles_of(b.worlds[i]->hd.H, b.worlds[i]->hd.Wp, k);
    }
    tiles[n] = tt;
    ECO_CU(cudaMemcpy(b.bd.tile_prefix, tiles.data(), (n + 1) * sizeof(int),
                      cudaMemcpyHostToDevice));
    b.bd.total_tiles = tt;
    b.bd.regrow_k = k;
    b.bd.tail_early = tail_early(b.bd);
  }
  b.bd.lstm_ctas = lstm_ctas;
  return ECO_OK;
}

// Milliseconds per step of `steps` steps under the batch's current config.
// The graphs are captured before the first event: a configuration change
// drops them, and their capture is host work, not part of a step.
int time_steps(EcoBatch &b, int64_t steps, cudaEvent_t e0, cudaEvent_t e1, double *ms) {
  int rc0 = prepare_graphs(b, steps);
  if (rc0) return rc0;
  ECO_CU(cudaEventRecord(e0, b.stream));
  int rc = batch_step(b, steps);
  if (rc) return rc;
  ECO_CU(cudaEventRecord(e1, b.stream));
  ECO_CU(cudaEventSynchronize(e1));
  float t = 0.f;
  ECO_CU(cudaEventElapsedTime(&t, e0, e1));
  *ms = (double)t / (double)steps;
  return ECO_OK;
}

// One coordinate of the search: every candidate value of one knob, timed
// round-robin (so that a population that drifts during the search affects
// all of them alike); the median of each candidate's trials decides, and a
// candidate replaces the current value (*best on entry, one of `cand`) only
// if it is faster by more than SWITCH_MARGIN: trials of a few steps are
// noisy, and births (which some knobs act on) come in bursts.
constexpr double SWITCH_MARGIN = 0.03;
// `trial_of(v)` is the number of steps a trial of candidate v takes (chunk
// lengths are timed over a multiple of themselves).
template <class Apply, class Trial>
int tune_knob(EcoBatch &b, const std::vector<int> &cand, Trial trial_of, int rounds, Apply apply,
              cudaEvent_t e0, cudaEvent_t e1, int64_t *steps, int *best, double *best_ms) {
  std::vector<std::vector<double>> t(cand.size());
  for (int r = 0; r < rounds; ++r) {
    for (size_t i = 0; i < cand.size(); ++i) {
      int rc = apply(cand[i]);
      if (rc) return rc;
      double ms = 0.0;
      const int64_t trial = trial_of(cand[i]);
      if ((rc = time_steps(b, trial, e0, e1, &ms))) return rc;
      *steps += trial;
      t[i].push_back(ms);
    }
  }
  std::vector<double> med(cand.size());
  double cur_ms = -1.0;
  for (size_t i = 0; i < cand.size(); ++i) {
    std::sort(t[i].begin(), t[i].end());
    med[i] = t[i][t[i].size() / 2];
    if (cand[i] == *best) cur_ms = med[i];
  }
  int choice = *best;
  double choice_ms = cur_ms;
  for (size_t i = 0; i < cand.size(); ++i) {
    // the current value is not a candidate: the fastest candidate wins
    const bool better = cur_ms < 0.0 ? (choice_ms < 0.0 || med[i] < choice_ms)
                                     : (med[i] < (1.0 - SWITCH_MARGIN) * cur_ms &&
                                        med[i] < choice_ms);
    if (better) {
      choice = cand[i];
      choice_ms = med[i];
    }
  }
  *best = choice;
  *best_ms = choice_ms;
  return apply(*best);
}

int autotune(EcoBatch &b, int trial_steps, EcoTuneResult *out) {
  if (trial_steps < 1 || trial_steps > 100000) return ECO_EINVAL;
  if (b.prof && b.prof->on) return ECO_EINVAL;  // would time the profiled graph
  *out = EcoTuneResult{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ECO_CU(cudaEventCreate(&e0));
  int rc = cuda_err(cudaEventCreate(&e1));
  const int rounds = 3;
  int64_t steps = 0;
  int fused = b.bd.fused, spawn = b.bd.spawn_ctas / b.bd.n_sms, k = b.steps_per_graph;
  int regrow = b.regrow_cfg ? b.regrow_cfg : b.bd.regrow_k, lstm = b.bd.lstm_ctas;
  double ms = 0.0;
  if (!rc) rc = set_config(b, fused, spawn, k);
  if (!rc) rc = time_steps(b, trial_steps, e0, e1, &out->ms_per_step_initial);
  if (!rc) steps += trial_steps;
  auto same = [&](int) { return (int64_t)trial_steps; };
  if (!rc && b.bd.max_capacity <= FUSED_MAX_C) {
    rc = tune_knob(b, {1, 0}, same, rounds,
                   [&](int v) { return set_config(b, v, spawn, k); }, e0, e1, &steps, &fused, &ms);
  }
  if (!rc) {
    rc = tune_knob(b, {1, 2, 4, 8}, same, rounds,
                   [&](int v) { return set_config(b, fused, v, k); }, e0, e1, &steps, &spawn, &ms);
  }
  if (!rc && b.bd.controller == ECO_CTRL_LSTM32) {
    rc = tune_knob(b, {1, 2}, same, rounds,
                   [&](int v) { return set_shape(b, b.regrow_cfg, v); }, e0, e1, &steps, &lstm,
                   &ms);
  }
  // stacking beyond the default (the fewest tiles per CTA that fit one wave)
  // only lengthens each CTA: the candidates stop there, and a batch that
  // fits one wave unstacked has no choice to make
  const int regrow_max = regrow_k_for(b.worlds.data(), (int)b.worlds.size(), b.bd.n_sms);
  if (!rc && regrow_max > 1) {
    std::vector<int> cand;
    for (int v = 1; v <= regrow_max; v *= 2) cand.push_back(v);
    rc = tune_knob(b, cand, same, rounds,
                   [&](int v) { return set_shape(b, v, lstm); }, e0, e1, &steps, &regrow, &ms);
  }
  if (!rc) {
    // a chunk length is timed over whole chunks: the multiple of it closest
    // to the trial length from above (steps per graph of the batched
    // workload: 50)
    auto whole = [&](int v) { return (int64_t)((trial_steps + v - 1) / v) * v; };
    rc = tune_knob(b, {1, 4, 16, 50}, whole, rounds,
                   [&](int v) { return set_config(b, fused, spawn, v); }, e0, e1, &steps, &k, &ms);
  }
  // the record's best time: the chosen configuration timed again now, at
  // the population the batch has reached (the knobs' medians were taken at
  // earlier, different populations)
  if (!rc) {
    const int64_t trial = ((trial_steps + k - 1) / k) * k;
    rc = time_steps(b, trial, e0, e1, &ms);
    if (!rc) steps += trial;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  out->fused = fused;
  out->spawn_ctas_per_sm = spawn;
  out->steps_per_graph = k;
  out->regrow_rows_per_cta = regrow;
  out->lstm_ctas_per_sm = lstm;
  out->steps_taken = steps;
  out->ms_per_step_best = ms;
  return ECO_OK;
}

int read_status(EcoWorld *w, int *status) {
  ECO_CU(cudaMemcpy(status, &w->hd.ctr->status, sizeof(int), cudaMemcpyDeviceToHost));
  return ECO_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------
extern "C" {

size_t eco_world_bytes(const EcoParams *p) {
  if (!params_ok(p)) return 0;
  return layout_of(p).total;
}

static void fill_descriptor(EcoWorld *w) {
  const EcoParams &p = w->p;
  const Layout &L = w->L;
  char *a = w->arena;
  WorldDev &d = w->hd;
  d.H = p.H; d.W = p.W; d.Wp = (p.W + 31) / 32; d.C = p.capacity;
  d.controller = p.controller;
  d.wstride = wstride_of(p.controller);
  d.nparam = nparam_of(p.controller);
  d.nbr_shape = p.nbr_shape; d.nbr_radius = p.nbr_radius;
  for (int i = 0; i < 3; ++i) d.class_edges[i] = p.class_edges[i];
  d.t_repr = p.t_repr; d.t_death = p.t_death; d.max_age = p.max_age;
  d.wall_kills = p.wall_kills;
  d.e0 = p.e0; d.e_decay = p.e_decay; d.e_gain = p.e_gain; d.e_max = p.e_max;
  d.e_repr = p.e_repr; d.e_death = p.e_death; d.mut_std = p.mut_std;
  d.w_init_std = p.w_init_std;
  d.key0 = (uint32_t)(w->seed & 0xFFFFFFFFu);
  d.key1 = (uint32_t)(w->seed >> 32);
  d.thr = (uint32_t *)(a + L.thr);
  d.res0 = (uint32_t *)(a + L.res0);
  d.res1 = (uint32_t *)(a + L.res1);
  d.wall = (uint32_t *)(a + L.wall);
  d.slot_map = (int32_t *)(a + L.slot_map);
  d.claim = (int32_t *)(a + L.claim);
  d.bclaim = (int32_t *)(a + L.bclaim);
  d.alive = (uint8_t *)(a + L.alive);
  d.killed = (uint8_t *)(a + L.killed);
  d.ate = (uint8_t *)(a + L.ate);
  d.flag = (uint8_t *)(a + L.flag);
  d.y = (int32_t *)(a + L.y);
  d.x = (int32_t *)(a + L.x);
  d.energy = (float *)(a + L.energy);
  d.repr_ctr = (int32_t *)(a + L.repr_ctr);
  d.low_ctr = (int32_t *)(a + L.low_ctr);
  d.age = (int32_t *)(a + L.age);
  d.action = (int32_t *)(a + L.action);
  d.forced = (int32_t *)(a + L.forced);
  d.target = (int32_t *)(a + L.target);
  d.birth_cell = (int32_t *)(a + L.birth_cell);
  d.arrive = (uint32_t *)(a + L.arrive);
  d.h0 = (float *)(a + L.h0);
  d.h1 = (float *)(a + L.h1);
  d.c = (float *)(a + L.c);
  d.logits = (float *)(a + L.logits);
  d.alive_list = (int32_t *)(a + L.alive_list);
  d.alive_new = (uint8_t *)(a + L.alive_new);
  d.free_list = (int32_t *)(a + L.free_list);
  d.birth_parent = (int32_t *)(a + L.birth_parent);
  d.birth_child = (int32_t *)(a + L.birth_child);
  d.weights = (float *)(a + L.weights);
  d.ctr = (Counters *)(a + L.ctr);
  d.snap_cell = (int32_t *)(a + L.snap_cell);
  d.prev_act = (int32_t *)(a + L.prev_act);
  d.lab_seen = (uint8_t *)(a + L.lab_seen);
  d.lab_ate = (uint8_t *)(a + L.lab_ate);
  d.lab_t = (int32_t *)(a + L.lab_t);
  d.lab_c = (int32_t *)(a + L.lab_c);
  d.scan_blocks = (int32_t *)(a + L.scan_blocks);
  d.analysis = (unsigned long long *)(a + L.analysis);
  w->dd = (WorldDev *)(a + L.wdev);
}

// Cells of the initial agents: the non-wall cells in ascending order of
// (word x%4 of the Philox draw {x/4, 0, TAG_PLACE, y}, cell index).
static bool initial_cells(const EcoParams &p, uint64_t seed, std::vector<int32_t> &py,
                          std::vector<int32_t> &px) {
  const uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
  std::vector<uint64_t> keys;
  keys.reserve((size_t)p.H * p.W);
  for (int y = 0; y < p.H; ++y) {
    for (int xq = 0; xq < p.W; xq += 4) {
      const U4 u = philox4x32_10(U4{(uint32_t)xq >> 2, 0u, TAG_PLACE, (uint32_t)y}, k0, k1);
      const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
      for (int i = 0; i < 4 && xq + i < p.W; ++i) {
        const int x = xq + i;
        const bool wall = p.border_walls && (y == 0 || y == p.H - 1 || x == 0 || x == p.W - 1);
        if (wall) continue;
        keys.push_back(((uint64_t)uw[i] << 32) | (uint64_t)((size_t)y * p.W + x));
      }
    }
  }
  const size_t n0 = (size_t)p.n_agents0;
  if (n0 > keys.size()) return false;
  std::partial_sort(keys.begin(), keys.begin() + n0, keys.end());
  py.resize(n0);
  px.resize(n0);
  for (size_t s = 0; s < n0; ++s) {
    const uint32_t cell = (uint32_t)(keys[s] & 0xFFFFFFFFu);
    py[s] = (int32_t)(cell / (uint32_t)p.W);
    px[s] = (int32_t)(cell % (uint32_t)p.W);
  }
  return true;
}

int eco_world_create(const EcoParams *params, uint64_t seed, void *arena,
                     size_t arena_bytes, void *stream, EcoWorld **out) {
  if (!out) return ECO_EINVAL;
  *out = nullptr;
  if (!params_ok(params) || !stream) return ECO_EINVAL;
  const Layout L = layout_of(params);
  if (arena && ((uintptr_t)arena & 255u)) return ECO_EINVAL;
  if (arena && arena_bytes < L.total) return ECO_ENOMEM;
  std::vector<int32_t> py, px;
  if (!initial_cells(*params, seed, py, px)) return ECO_EINVAL;

  EcoWorld *w = new (std::nothrow) EcoWorld;
  if (!w) return ECO_ENOMEM;
  w->p = *params;
  w->seed = seed;
  w->stream = (cudaStream_t)stream;
  w->L = L;
  int rc = ECO_OK;
  do {
    if ((rc = cuda_err(cudaGetDevice(&w->device)))) break;
    if ((rc = cuda_err(cudaDeviceGetAttribute(&w->n_sms, cudaDevAttrMultiProcessorCount,
                                              w->device)))) break;
    configure_lstm();
    preload_lstm();
    preload_paper();
    preload_agents();
    if (arena) {
      w->arena = (char *)arena;
      w->arena_bytes = arena_bytes;
    } else {
      if (cudaMalloc((void **)&w->arena, L.total) != cudaSuccess) {
        cudaGetLastError();
        rc = ECO_ENOMEM;
        break;
      }
      w->owns_arena = true;
      w->arena_bytes = L.total;
    }
    fill_descriptor(w);
    const std::vector<uint32_t> thr = threshold_table(params);
    cudaStream_t s = w->stream;
    if ((rc = cuda_err(cudaMemsetAsync(w->hd.ctr, 0, sizeof(Counters), s)))) break;
    if ((rc = cuda_err(cudaMemcpyAsync(w->hd.thr, thr.data(), thr.size() * 4,
                                       cudaMemcpyHostToDevice, s)))) break;
    if ((rc = cuda_err(cudaMemcpyAsync(w->dd, &w->hd, sizeof(WorldDev),
                                       cudaMemcpyHostToDevice, s)))) break;
    if (!py.empty()) {
      if ((rc = cuda_err(cudaMemcpyAsync(w->hd.free_list, py.data(), py.size() * 4,
                                         cudaMemcpyHostToDevice, s)))) break;
      if ((rc = cuda_err(cudaMemcpyAsync(w->hd.birth_parent, px.data(), px.size() * 4,
                                         cudaMemcpyHostToDevice, s)))) break;
    }
    launch_init_world(&w->hd, w->dd, params->n_agents0, w->hd.free_list,
                      w->hd.birth_parent, params->border_walls,
                      threshold_of(params->res_init_p), w->n_sms, s);
    if ((rc = cuda_err(cudaGetLastError()))) break;
    if ((rc = cuda_err(cudaStreamSynchronize(s)))) break;
    EcoWorld *self[1] = {w};
    if ((rc = batch_init(w->self, self, 1, w->arena + L.tab_worlds))) break;
  } while (0);
  if (rc != ECO_OK) {
    if (w->owns_arena && w->arena) cudaFree(w->arena);
    delete w;
    return rc;
  }
  *out = w;
  return ECO_OK;
}

void eco_world_destroy(EcoWorld *w) {
  if (!w) return;
  cudaStreamSynchronize(w->stream);
  if (w->io_stream) {
    cudaStreamSynchronize(w->io_stream);
    cudaStreamDestroy(w->io_stream);
  }
  if (w->io_fork) cudaEventDestroy(w->io_fork);
  if (w->io_join) cudaEventDestroy(w->io_join);
  destroy_graphs(w->self);
  profile_release(w->prof);
  if (w->owns_arena) cudaFree(w->arena);
  delete w;
}

int eco_world_step(EcoWorld *w, int64_t n_steps) {
  Trace trace("eco_world_step");
  if (!w) return ECO_EINVAL;
  return batch_step(w->self, n_steps);
}

int eco_world_step_forced(EcoWorld *w, const int32_t *actions, int actions_on_host) {
  Trace trace("eco_world_step_forced");
  if (!w || (!actions && w->p.capacity > 0)) return ECO_EINVAL;
  cudaStream_t s = w->stream;
  const size_t bytes = (size_t)w->p.capacity * 4;
  if (bytes)
    ECO_CU(cudaMemcpyAsync(w->hd.forced, actions, bytes,
                           actions_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  static const int one = 1;
  ECO_CU(cudaMemcpyAsync(&w->hd.ctr->use_forced, &one, sizeof(int), cudaMemcpyHostToDevice, s));
  launch_step(w->self, s, nullptr);
  ECO_CU(cudaGetLastError());
  ECO_CU(cudaMemsetAsync(&w->hd.ctr->use_forced, 0, sizeof(int), s));
  if (actions_on_host) ECO_CU(cudaStreamSynchronize(s));
  return ECO_OK;
}

int eco_world_counters_async(EcoWorld *w, int64_t *out_host) {
  if (!w || !out_host) return ECO_EINVAL;
  static_assert(offsetof(Counters, t) == 0 && offsetof(Counters, agent_steps) ==
                    (ECO_NCOUNTERS - 1) * sizeof(long long),
                "the first ECO_NCOUNTERS fields of Counters are the ECO_C_* counters");
  ECO_CU(cudaMemcpyAsync(out_host, w->hd.ctr, ECO_NCOUNTERS * sizeof(int64_t),
                         cudaMemcpyDeviceToHost, w->stream));
  return ECO_OK;
}

int eco_world_counter_log(EcoWorld *w, int64_t *log_host, int64_t rows) {
  Trace trace("eco_world_counter_log");
  if (!w) return ECO_EINVAL;
  struct {
    long long *log;
    long long rows;
  } v = {nullptr, 0};
  static_assert(offsetof(Counters, log_rows) == offsetof(Counters, log) + sizeof(long long *),
                "the log's pointer and row count are written together");
  if (log_host) {
    if (rows <= 0 || ((uintptr_t)log_host & 7u)) return ECO_EINVAL;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, log_host) != cudaSuccess) {
      (void)cudaGetLastError();
      return ECO_EINVAL;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer) return ECO_EINVAL;
    v.log = (long long *)a.devicePointer;
    v.rows = rows;
  }
  ECO_CU(cudaMemcpyAsync(&w->hd.ctr->log, &v, sizeof v, cudaMemcpyHostToDevice, w->stream));
  // the source is on the stack: the copy must have read it before returning
  ECO_CU(cudaStreamSynchronize(w->stream));
  return ECO_OK;
}

int eco_world_analysis_async(EcoWorld *w, EcoAnalysis *out_host) {
  Trace trace("eco_world_analysis_async");
  if (!w || !out_host) return ECO_EINVAL;
  static_assert(sizeof(EcoAnalysis) == ANALYSIS_WORDS * sizeof(int64_t) &&
                    offsetof(EcoAnalysis, movers) == A_MOVERS * sizeof(int64_t) &&
                    offsetof(EcoAnalysis, move_bins) == A_BINS * sizeof(int64_t) &&
                    ECO_MOVE_BINS == MOVE_BINS,
                "EcoAnalysis mirrors the analysis kernels' record");
  launch_analysis(&w->hd, w->n_sms, w->stream);
  ECO_CU(cudaGetLastError());
  ECO_CU(cudaMemcpyAsync(out_host, w->hd.analysis, sizeof(EcoAnalysis), cudaMemcpyDeviceToHost,
                         w->stream));
  return ECO_OK;
}

int eco_life_expectancy(const EcoAnalysis *records, int64_t n, double *out) {
  if (!out || n < 0 || (n > 0 && !records)) return ECO_EINVAL;
  int64_t deaths = 0, ages = 0;
  for (int64_t i = 0; i < n; ++i) {
    deaths += records[i].deaths;
    ages += records[i].death_age_sum;
  }
  *out = deaths > 0 ? (double)ages / (double)deaths : std::nan("");
  return ECO_OK;
}

int eco_greediness(const int32_t *seen_windows, const int32_t *meal_windows, int64_t n,
                   double *out) {
  if (n < 0 || (n > 0 && (!seen_windows || !meal_windows || !out))) return ECO_EINVAL;
  for (int64_t i = 0; i < n; ++i)
    out[i] = seen_windows[i] > 0 ? (double)meal_windows[i] / (double)seen_windows[i]
                                 : std::nan("");
  return ECO_OK;
}

int eco_world_lab_window(EcoWorld *w) {
  if (!w) return ECO_EINVAL;
  launch_lab_window(&w->hd, w->n_sms, w->stream);
  ECO_CU(cudaGetLastError());
  return ECO_OK;
}

int eco_world_lab_read(EcoWorld *w, int32_t *seen_windows_host, int32_t *meal_windows_host) {
  if (!w || !seen_windows_host || !meal_windows_host) return ECO_EINVAL;
  ECO_CU(cudaStreamSynchronize(w->stream));
  const size_t bytes = (size_t)w->p.capacity * 4;
  if (bytes) {
    ECO_CU(cudaMemcpy(seen_windows_host, w->hd.lab_t, bytes, cudaMemcpyDeviceToHost));
    ECO_CU(cudaMemcpy(meal_windows_host, w->hd.lab_c, bytes, cudaMemcpyDeviceToHost));
  }
  return ECO_OK;
}

int eco_world_sync(EcoWorld *w) {
  if (!w) return ECO_EINVAL;
  ECO_CU(cudaStreamSynchronize(w->stream));
  int st = 0;
  int rc = read_status(w, &st);
  if (rc) return rc;
  if (st & ST_TIMEOUT) return ECO_ETIMEOUT;
  if (st & ST_BOUNDS) return ECO_EBOUNDS;
  return ECO_OK;
}

int eco_world_selftest_timeout(EcoWorld *w, uint64_t limit_ns) {
  if (!w || limit_ns > 10000000000ull) return ECO_EINVAL;
  launch_wait_selftest(&w->hd.ctr->status, (unsigned long long)limit_ns, w->stream);
  ECO_CU(cudaGetLastError());
  return ECO_OK;
}

int eco_world_clear_status(EcoWorld *w) {
  if (!w) return ECO_EINVAL;
  ECO_CU(cudaMemsetAsync(&w->hd.ctr->status, 0, sizeof(int), w->stream));
  ECO_CU(cudaStreamSynchronize(w->stream));
  return ECO_OK;
}

const EcoParams *eco_world_params(const EcoWorld *w) { return w ? &w->p : nullptr; }
void *eco_world_stream(const EcoWorld *w) { return w ? (void *)w->stream : nullptr; }

static void counters_to_array(const Counters &c, int64_t *out) {
  out[ECO_C_T] = c.t;
  out[ECO_C_POP] = c.pop;
  out[ECO_C_BIRTHS] = c.births;
  out[ECO_C_DEATHS] = c.deaths;
  out[ECO_C_DROPPED] = c.dropped;
  out[ECO_C_BIRTHS_LAST] = c.births_last;
  out[ECO_C_DEATHS_LAST] = c.deaths_last;
  out[ECO_C_DROPPED_LAST] = c.dropped_last;
  out[ECO_C_AGENT_STEPS] = c.agent_steps;
}

// State I/O.  Every copy is enqueued on the world's stream and the call
// waits once at the end (a first version waited after each of ~20 copies).
// A copy from or to page-locked host memory is a DMA transfer that overlaps
// the others; from pageable memory the driver stages it.  Weights move
// between the host's logical order and the device's physical order by a
// permutation kernel: it reads or writes page-locked host memory directly
// through its device address, and pageable memory through a staging region
// of STAGING_AGENTS rows in the arena.
struct StateIO {
  cudaStream_t s;
  int rc = ECO_OK;
  explicit StateIO(cudaStream_t st) : s(st) {}
  void d2h(void *dst, const void *src, size_t bytes) {
    if (rc || !dst || !bytes) return;
    rc = cuda_err(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
  }
  void h2d(void *dst, const void *src, size_t bytes) {
    if (rc || !src || !bytes) return;
    rc = cuda_err(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
  }
  int wait() {
    if (rc) return rc;
    return rc = cuda_err(cudaStreamSynchronize(s));
  }
};

// Device address of a page-locked host buffer, or null for pageable memory.
static void *pinned_device_view(const void *host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return (a.type == cudaMemoryTypeHost && a.devicePointer) ? a.devicePointer : nullptr;
}

static void pack_plane(const EcoParams &p, const uint8_t *in, std::vector<uint32_t> &words) {
  const int Wp = (p.W + 31) / 32;
  words.assign((size_t)p.H * Wp, 0u);
  for (int y = 0; y < p.H; ++y)
    for (int x = 0; x < p.W; ++x)
      if (in[(size_t)y * p.W + x]) words[(size_t)y * Wp + (x >> 5)] |= 1u << (x & 31);
}
static void unpack_plane(const EcoParams &p, const std::vector<uint32_t> &words, uint8_t *out) {
  const int Wp = (p.W + 31) / 32;
  for (int y = 0; y < p.H; ++y)
    for (int x = 0; x < p.W; ++x)
      out[(size_t)y * p.W + x] = (words[(size_t)y * Wp + (x >> 5)] >> (x & 31)) & 1u;
}

// The last step's births get their weights from the tail kernel that
// starts the next step.  Reading weights, and loading a state, first run
// that kernel (its regrowth part writes the next plane from the current one:
// the same words the next step writes again) and mark the births done, so
// that they see final weights.  Nothing else a state read returns waits for
// that kernel.
static int settle_births(EcoWorld *w) {
  launch_tail(w->self.bd, w->stream);
  ECO_CU(cudaGetLastError());
  ECO_CU(cudaMemsetAsync(&w->hd.ctr->n_births, 0, sizeof(int), w->stream));
  return ECO_OK;
}

int eco_world_read_state(EcoWorld *w, EcoState *out) {
  Trace trace("eco_world_read_state");
  if (!w || !out) return ECO_EINVAL;
  const EcoParams &p = w->p;
  const WorldDev &d = w->hd;
  const size_t C = p.capacity, HW = (size_t)p.H * p.W;
  if (out->weights_host &&
      (out->weights_first < 0 || out->weights_count < 0 ||
       (size_t)out->weights_first + out->weights_count > C))
    return ECO_EINVAL;
  int rc = ECO_OK;
  const bool wts = out->weights_host && out->weights_count > 0;
  if (wts && (rc = settle_births(w))) return rc;
  StateIO io(w->stream);
  Counters c;
  io.d2h(&c, d.ctr, sizeof(Counters));
  if ((rc = io.wait())) return rc;
  counters_to_array(c, out->counters);
  const bool odd = (c.t & 1) != 0;
  const size_t nwords = (size_t)p.H * ((p.W + 31) / 32);
  std::vector<uint32_t> res_w, wall_w;
  std::vector<float> lg;
  if (out->res_host) {
    res_w.resize(nwords);
    io.d2h(res_w.data(), odd ? d.res1 : d.res0, nwords * 4);
  }
  if (out->wall_host) {
    wall_w.resize(nwords);
    io.d2h(wall_w.data(), d.wall, nwords * 4);
  }
  io.d2h(out->slot_map_host, d.slot_map, HW * 4);
  io.d2h(out->alive_host, d.alive, C);
  io.d2h(out->y_host, d.y, C * 4);
  io.d2h(out->x_host, d.x, C * 4);
  io.d2h(out->energy_host, d.energy, C * 4);
  io.d2h(out->repr_ctr_host, d.repr_ctr, C * 4);
  io.d2h(out->low_ctr_host, d.low_ctr, C * 4);
  io.d2h(out->age_host, d.age, C * 4);
  io.d2h(out->h_host, odd ? d.h1 : d.h0, C * HID * 4);
  io.d2h(out->c_host, d.c, C * HID * 4);
  io.d2h(out->action_host, d.action, C * 4);
  io.d2h(out->prev_action_host, d.prev_act, C * 4);
  io.d2h(out->ate_host, d.ate, C);
  if (out->logits_host && C) {
    lg.resize(C * 8);
    io.d2h(lg.data(), d.logits, lg.size() * 4);
  }
  if (wts && !io.rc) {
    const size_t ws = d.wstride, np = d.nparam;
    const float *src = d.weights + (size_t)out->weights_first * ws;
    if (float *dev = (float *)pinned_device_view(out->weights_host)) {
      launch_weights_to_logical(src, dev, np, out->weights_count, d.controller, w->n_sms,
                                w->stream);
      io.rc = cuda_err(cudaGetLastError());
    } else {
      float *staging = (float *)(w->arena + w->L.staging);
      for (int s0 = 0; s0 < out->weights_count && !io.rc; s0 += STAGING_AGENTS) {
        const int n = std::min(STAGING_AGENTS, out->weights_count - s0);
        launch_weights_to_logical(src + (size_t)s0 * ws, staging, ws, n, d.controller, w->n_sms,
                                  w->stream);
        io.rc = cuda_err(cudaGetLastError());
        if (!io.rc)
          io.rc = cuda_err(cudaMemcpy2DAsync(out->weights_host + (size_t)s0 * np, np * 4,
                                             staging, ws * 4, np * 4, n,
                                             cudaMemcpyDeviceToHost, w->stream));
        // the next chunk's permutation, which reuses the staging region, is
        // ordered after this copy by the stream
      }
    }
  }
  if ((rc = io.wait())) return rc;
  if (out->res_host) unpack_plane(p, res_w, out->res_host);
  if (out->wall_host) unpack_plane(p, wall_w, out->wall_host);
  if (out->logits_host)
    for (size_t s = 0; s < C; ++s)
      for (int a = 0; a < NACT; ++a) out->logits_host[s * NACT + a] = lg[s * 8 + a];
  return ECO_OK;
}

int eco_world_load_state(EcoWorld *w, const EcoState *in, int set_counters) {
  Trace trace("eco_world_load_state");
  if (!w || !in) return ECO_EINVAL;
  const EcoParams &p = w->p;
  const WorldDev &d = w->hd;
  const size_t C = p.capacity;
  if (in->weights_host &&
      (in->weights_first < 0 || in->weights_count < 0 ||
       (size_t)in->weights_first + in->weights_count > C))
    return ECO_EINVAL;
  if (set_counters && (in->counters[ECO_C_T] < 0 || in->counters[ECO_C_T] > 0xFFFFFFFFll))
    return ECO_EINVAL;
  int rc = settle_births(w);
  if (rc) return rc;
  // The weight rows, the bulk of a state (93 KB per agent over a host link
  // of about 0.2 TB/s), go first, on the world's second stream, while the
  // rest of the state is written on the world's stream; the rows' slots
  // wait for the tail kernel just launched (it writes pending children).
  const bool wts = in->weights_host && in->weights_count > 0;
  if (wts) {
    if (!w->io_stream) {
      ECO_CU(cudaStreamCreateWithFlags(&w->io_stream, cudaStreamNonBlocking));
      ECO_CU(cudaEventCreateWithFlags(&w->io_fork, cudaEventDisableTiming));
      ECO_CU(cudaEventCreateWithFlags(&w->io_join, cudaEventDisableTiming));
    }
    ECO_CU(cudaEventRecord(w->io_fork, w->stream));
    ECO_CU(cudaStreamWaitEvent(w->io_stream, w->io_fork, 0));
    const size_t ws = d.wstride, np = d.nparam;
    float *dst = d.weights + (size_t)in->weights_first * ws;
    // page-locked rows (16-byte aligned): read by a kernel through their
    // device address, stored in physical order; otherwise one 2-D copy of
    // the logical rows into their own device rows (staged by the driver
    // from pageable memory), then the permutation to the physical order in
    // place
    const float *dev = (const float *)pinned_device_view(in->weights_host);
    int wrc;
    if (dev && ((uintptr_t)dev & 15u) == 0) {
      wrc = cuda_err((cudaError_t)launch_weights_from_host(dev, dst, in->weights_count,
                                                           d.controller, w->n_sms, w->io_stream));
    } else {
      wrc = cuda_err(cudaMemcpy2DAsync(dst, ws * 4, in->weights_host, np * 4, np * 4,
                                       in->weights_count, cudaMemcpyHostToDevice, w->io_stream));
      if (!wrc)
        wrc = cuda_err((cudaError_t)launch_rows_to_physical_inplace(
            dst, in->weights_count, d.controller, w->n_sms, w->io_stream));
    }
    // joined by the world's stream before its final wait, whatever happens
    const int jrc = cuda_err(cudaEventRecord(w->io_join, w->io_stream));
    if (wrc || jrc) {
      cudaStreamSynchronize(w->io_stream);
      return wrc ? wrc : jrc;
    }
  }
  StateIO io(w->stream);
  // The step counter says which buffer of the plane and h pairs is current:
  // the caller's, or (counters kept) the device's, read back first.
  LoadCounters lc{};
  lc.set = set_counters ? 1 : 0;
  long long t_now = in->counters[ECO_C_T];
  if (set_counters) {
    lc.t = in->counters[ECO_C_T];
    lc.births = in->counters[ECO_C_BIRTHS];
    lc.deaths = in->counters[ECO_C_DEATHS];
    lc.dropped = in->counters[ECO_C_DROPPED];
    lc.births_last = in->counters[ECO_C_BIRTHS_LAST];
    lc.deaths_last = in->counters[ECO_C_DEATHS_LAST];
    lc.dropped_last = in->counters[ECO_C_DROPPED_LAST];
    lc.agent_steps = in->counters[ECO_C_AGENT_STEPS];
  } else {
    io.d2h(&t_now, &d.ctr->t, sizeof(long long));
    if ((rc = io.wait())) {
      if (wts) cudaStreamSynchronize(w->io_stream);
      return rc;
    }
  }
  launch_load_counters(d.ctr, lc, w->stream);
  const bool odd = (t_now & 1) != 0;
  // Planes: the cells' bytes are staged in the slot map (rebuilt below) or
  // read from page-locked memory, and packed into words on the device.
  const size_t HW = (size_t)p.H * p.W;
  uint8_t *stage = reinterpret_cast<uint8_t *>(d.slot_map);   // 4 HW bytes
  const uint8_t *planes_in[2] = {in->res_host, in->wall_host};
  uint32_t *planes_out[2] = {odd ? d.res1 : d.res0, d.wall};
  for (int k = 0; k < 2 && !io.rc; ++k) {
    if (!planes_in[k]) continue;
    const uint8_t *cells = (const uint8_t *)pinned_device_view(planes_in[k]);
    if (!cells) {
      io.h2d(stage + k * HW, planes_in[k], HW);
      cells = stage + k * HW;
    }
    launch_pack_plane(cells, p.H, p.W, d.Wp, planes_out[k], w->stream);
  }
  // Slot arrays: page-locked ones read by one kernel, the others copied.
  SlotSources src{};
  std::vector<float> lg;   // pageable logits repacked to C x 8, alive until the wait
  auto slot_in = [&](const void *host, void *dev, size_t bytes) -> const void * {
    if (!host || !C) return nullptr;
    if (const void *v = pinned_device_view(host)) return v;
    io.h2d(dev, host, bytes);
    return nullptr;
  };
  src.alive = (const uint8_t *)slot_in(in->alive_host, d.alive, C);
  src.y = (const int32_t *)slot_in(in->y_host, d.y, C * 4);
  src.x = (const int32_t *)slot_in(in->x_host, d.x, C * 4);
  src.energy = (const float *)slot_in(in->energy_host, d.energy, C * 4);
  src.repr = (const int32_t *)slot_in(in->repr_ctr_host, d.repr_ctr, C * 4);
  src.low = (const int32_t *)slot_in(in->low_ctr_host, d.low_ctr, C * 4);
  src.age = (const int32_t *)slot_in(in->age_host, d.age, C * 4);
  float *h_dst = odd ? d.h1 : d.h0;
  src.h = (const float *)slot_in(in->h_host, h_dst, C * HID * 4);
  src.c = (const float *)slot_in(in->c_host, d.c, C * HID * 4);
  src.action = (const int32_t *)slot_in(in->action_host, d.action, C * 4);
  src.prev = (const int32_t *)slot_in(in->prev_action_host, d.prev_act, C * 4);
  src.ate = (const uint8_t *)slot_in(in->ate_host, d.ate, C);
  if (in->logits_host && C) {
    src.logits = (const float *)pinned_device_view(in->logits_host);
    if (!src.logits) {
      lg.assign(C * 8, 0.f);
      for (size_t s = 0; s < C; ++s)
        for (int a = 0; a < NACT; ++a) lg[s * 8 + a] = in->logits_host[s * NACT + a];
      io.h2d(d.logits, lg.data(), lg.size() * 4);
    }
  }
  if (!io.rc) launch_load_slots(d, src, h_dst, w->n_sms, w->stream);
  // greediness counters start over with a loaded state
  if (!io.rc) io.rc = cuda_err(cudaMemsetAsync(d.lab_seen, 0, C ? C : 1, w->stream));
  if (!io.rc) io.rc = cuda_err(cudaMemsetAsync(d.lab_ate, 0, C ? C : 1, w->stream));
  if (!io.rc) io.rc = cuda_err(cudaMemsetAsync(d.lab_t, 0, (C ? C : 1) * 4, w->stream));
  if (!io.rc) io.rc = cuda_err(cudaMemsetAsync(d.lab_c, 0, (C ? C : 1) * 4, w->stream));
  if (!io.rc) {
    launch_rebuild(&w->hd, w->n_sms, w->stream);
    io.rc = cuda_err(cudaGetLastError());
  }
  if (wts) {
    const int jrc = cuda_err(cudaStreamWaitEvent(w->stream, w->io_join, 0));
    if (!io.rc) io.rc = jrc;
  }
  int st = 0;
  io.d2h(&st, &d.ctr->status, sizeof(int));
  if ((rc = io.wait())) {
    if (wts) cudaStreamSynchronize(w->io_stream);
    return rc;
  }
  if (st & ST_STATE) {
    st &= ~ST_STATE;
    ECO_CU(cudaMemcpy(&d.ctr->status, &st, sizeof(int), cudaMemcpyHostToDevice));
    return ECO_ESTATE;
  }
  return ECO_OK;
}

int eco_batch_create(EcoWorld *const *worlds, int n, EcoBatch **out) {
  if (!out) return ECO_EINVAL;
  *out = nullptr;
  if (!worlds || n < 1 || n > 1024) return ECO_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!worlds[i] || worlds[i]->device != worlds[0]->device ||
        worlds[i]->p.controller != worlds[0]->p.controller)
      return ECO_EINVAL;
  EcoBatch *b = new (std::nothrow) EcoBatch;
  if (!b) return ECO_ENOMEM;
  int rc = batch_init(*b, worlds, n, nullptr);
  if (rc) {
    if (b->owns_table && b->table) cudaFree(b->table);
    delete b;
    return rc;
  }
  *out = b;
  return ECO_OK;
}

int eco_batch_step(EcoBatch *b, int64_t n_steps) {
  Trace trace("eco_batch_step");
  if (!b) return ECO_EINVAL;
  return batch_step(*b, n_steps);
}

int eco_batch_set_config(EcoBatch *b, int fused, int spawn_ctas_per_sm, int steps_per_graph) {
  if (!b) return ECO_EINVAL;
  return set_config(*b, fused, spawn_ctas_per_sm, steps_per_graph);
}

int eco_batch_get_config(const EcoBatch *b, int *fused, int *spawn_ctas_per_sm,
                         int *steps_per_graph) {
  if (!b || !fused || !spawn_ctas_per_sm || !steps_per_graph) return ECO_EINVAL;
  *fused = b->bd.fused;
  *spawn_ctas_per_sm = b->bd.spawn_ctas / b->bd.n_sms;
  *steps_per_graph = b->steps_per_graph;
  return ECO_OK;
}

int eco_batch_set_shape(EcoBatch *b, int regrow_rows_per_cta, int lstm_ctas_per_sm) {
  if (!b) return ECO_EINVAL;
  return set_shape(*b, regrow_rows_per_cta, lstm_ctas_per_sm);
}

int eco_batch_get_shape(const EcoBatch *b, int *regrow_rows_per_cta, int *lstm_ctas_per_sm) {
  if (!b || !regrow_rows_per_cta || !lstm_ctas_per_sm) return ECO_EINVAL;
  *regrow_rows_per_cta = b->bd.regrow_k;
  *lstm_ctas_per_sm = b->bd.lstm_ctas;
  return ECO_OK;
}

int eco_batch_autotune(EcoBatch *b, int trial_steps, EcoTuneResult *out) {
  Trace trace("eco_batch_autotune");
  if (!b || !out) return ECO_EINVAL;
  return autotune(*b, trial_steps, out);
}

int eco_world_set_config(EcoWorld *w, int fused, int spawn_ctas_per_sm, int steps_per_graph) {
  if (!w) return ECO_EINVAL;
  return set_config(w->self, fused, spawn_ctas_per_sm, steps_per_graph);
}

int eco_world_get_config(const EcoWorld *w, int *fused, int *spawn_ctas_per_sm,
                         int *steps_per_graph) {
  if (!w) return ECO_EINVAL;
  return eco_batch_get_config(&w->self, fused, spawn_ctas_per_sm, steps_per_graph);
}

int eco_world_set_shape(EcoWorld *w, int regrow_rows_per_cta, int lstm_ctas_per_sm) {
  if (!w) return ECO_EINVAL;
  return set_shape(w->self, regrow_rows_per_cta, lstm_ctas_per_sm);
}

int eco_world_get_shape(const EcoWorld *w, int *regrow_rows_per_cta, int *lstm_ctas_per_sm) {
  if (!w) return ECO_EINVAL;
  return eco_batch_get_shape(&w->self, regrow_rows_per_cta, lstm_ctas_per_sm);
}

int eco_world_autotune(EcoWorld *w, int trial_steps, EcoTuneResult *out) {
  Trace trace("eco_world_autotune");
  if (!w || !out) return ECO_EINVAL;
  return autotune(w->self, trial_steps, out);
}

int eco_batch_sync(EcoBatch *b) {
  if (!b) return ECO_EINVAL;
  ECO_CU(cudaStreamSynchronize(b->stream));
  for (EcoWorld *w : b->worlds) {
    int st = 0;
    int rc = read_status(w, &st);
    if (rc) return rc;
    if (st & ST_TIMEOUT) return ECO_ETIMEOUT;
    if (st & ST_BOUNDS) return ECO_EBOUNDS;
  }
  return ECO_OK;
}

void eco_batch_destroy(EcoBatch *b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  destroy_graphs(*b);
  if (b->owns_table) cudaFree(b->table);
  delete b;
}

int eco_world_profile(EcoWorld *w, int enable, int max_steps) {
  if (!w || (enable && max_steps < 1)) return ECO_EINVAL;
  Profile &pr = w->prof;
  ECO_CU(cudaStreamSynchronize(w->stream));
  profile_release(pr);
  pr.pending = false;
  pr.on = false;
  pr.used = 0;
  for (int k = 0; k < ECO_NKERNELS; ++k) {
    pr.ms[k] = 0.0;
    pr.launches[k] = 0;
  }
  if (!enable) return ECO_OK;
  pr.max_steps = max_steps;
  pr.on = true;
  return ECO_OK;
}

int eco_world_profile_read(EcoWorld *w, double *ms, int64_t *launches) {
  if (!w || !ms || !launches) return ECO_EINVAL;
  Profile &pr = w->prof;
  ECO_CU(cudaStreamSynchronize(w->stream));
  int rc = profile_collect(pr);
  if (rc) return rc;
  pr.used = 0;
  for (int k = 0; k < ECO_NKERNELS; ++k) {
    ms[k] = pr.ms[k];
    launches[k] = pr.launches[k];
  }
  return ECO_OK;
}

const char *eco_kernel_name(int k) {
  static const char *names[ECO_NKERNELS] = {
      "regrow", "observe_lstm", "move_claim", "move_apply", "physio",
      "birth_claim", "scan", "regrow_spawn", "agents_fused", "observe_paper"};
  return (k >= 0 && k < ECO_NKERNELS) ? names[k] : "?";
}

int eco_kernels_per_step(const EcoWorld *w) {
  if (!w) return ECO_EINVAL;
  const StepKernel *list;
  return step_kernels(w->self.bd, &list);
}

const char *eco_strerror(int code) {
  switch (code) {
    case ECO_OK: return "ok";
    case ECO_EINVAL: return "invalid argument";
    case ECO_ENOMEM: return "out of memory";
    case ECO_ECUDA: return "CUDA error";
    case ECO_ETIMEOUT: return "device wait timed out";
    case ECO_ESTATE: return "inconsistent state";
    case ECO_EBOUNDS: return "device index out of range";
    default: return "unknown error";
  }
}

}  // extern "C"
