// k_agents.cu -- step parts a4..a6: moves and eating, physiology and death,
// reproduction (slot compaction + mutation), App. B.2 and B.3.
//
// Per-slot kernels run one thread per agent slot of every world (blocks of
// 256 slots, world found from a block prefix).  Conflicts are settled with
// order-independent atomics only (atomicMin on claim cells, atomicAnd on
// resource words), so results do not depend on thread scheduling:
//   (claims)    made by the observation+LSTM kernel as soon as an agent's
//               action is known: a valid target (on the grid, not a wall,
//               empty at the start of the phase) gets atomicMin(claim, slot)
//   move_apply  the lowest claimant moves and resets the claim cell
//   physio      eat (atomicAnd clears the resource bit), energy update with
//               exactly rounded float add/sub, death, reproduction counter
//   birth_claim first free N/S/E/W cell of each parent, atomicMin(bclaim)
//   scan_count, scan_prefix, scan_lists, scan_children
//               the compaction over 256-slot blocks: per-block counts of free
//               slots, successful parents and survivors; one CTA per world
//               scans them and writes the step's counters (t += 1); the free
//               slots the births take and the next alive list; the k-th
//               successful parent's child in the k-th free slot
//   agents_cluster  all of the above for worlds of capacity <= 16384, one
//               thread-block cluster per world (agents_single: one CTA per
//               world when every capacity is <= 2048)
//   tail        the first kernel of a step: the regrowth of the step's
//               resource plane in the same launch as the previous step's
//               births, child weights = parent weights + sigma * N(0,1) (a
//               grid-stride pass over every float4 of every birth)
#include <climits>

#include <cooperative_groups.h>

#include "ecoevo_dev.cuh"
#include "regrow_tile.cuh"

namespace cg = cooperative_groups;

namespace eco {

__device__ inline int find_world_a(const int *prefix, int n, int item) {
  if (n == 1) return 0;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Slot handled by this thread, or -1; sets wd.
__device__ inline int slot_of_thread(const BatchDev &b, const WorldDev *&wd) {
  const int w = find_world_a(b.slot_block_prefix, b.n, blockIdx.x);
  wd = world_ptr(b, w);
  const int s = (blockIdx.x - (b.n == 1 ? 0 : b.slot_block_prefix[w])) * SLOT_BLOCK + threadIdx.x;
  return s < wd->C ? s : -1;
}

__constant__ int kDY[5] = {0, -1, 1, 0, 0};  // stay, N, S, E, W
__constant__ int kDX[5] = {0, 0, 0, 1, -1};

// ---------------------------------------------------------------- a4 ------
__device__ inline void slot_move_apply(const WorldDev *wd, int s) {
  if (!wd->alive[s]) return;
  const int cell = wd->target[s];
  if (cell < 0 || !ECO_IN_RANGE(*wd, cell < wd->H * wd->W) || wd->claim[cell] != s) return;
  if (!ECO_IN_RANGE(*wd, wd->y[s] >= 0 && wd->y[s] < wd->H && wd->x[s] >= 0 &&
                         wd->x[s] < wd->W))
    return;
  wd->claim[cell] = INT_MAX;  // only the winner resets; losers compare != s
  wd->slot_map[wd->y[s] * wd->W + wd->x[s]] = -1;
  wd->slot_map[cell] = s;
  wd->y[s] = cell / wd->W;
  wd->x[s] = cell % wd->W;
}

// ---------------------------------------------------------------- a5 ------
__device__ inline void slot_physio(const WorldDev *wd, int s) {
  wd->ate[s] = 0;
  if (!wd->alive[s]) return;
  const int y = wd->y[s], x = wd->x[s];
  bool dead;
  if (wd->killed[s]) {
    dead = true;
  } else {
    const uint32_t t = (uint32_t)wd->ctr->t;
    uint32_t *res = (t & 1u) ? wd->res0 : wd->res1;  // plane after regrowth
    const uint32_t bit = 1u << (x & 31);
    const uint32_t old = atomicAnd(&res[y * wd->Wp + (x >> 5)], ~bit);
    const bool ate = (old & bit) != 0u;
    wd->ate[s] = ate ? 1 : 0;
    if (ate) wd->lab_ate[s] = 1;
    float e = wd->energy[s];
    if (ate) e = __fadd_rn(e, wd->e_gain);
    e = __fsub_rn(e, wd->e_decay);
    e = fminf(e, wd->e_max);
    wd->energy[s] = e;
    const int age = wd->age[s] + 1;
    wd->age[s] = age;
    const int low = (e <= wd->e_death) ? wd->low_ctr[s] + 1 : 0;
    wd->low_ctr[s] = low;
    dead = low >= max(wd->t_death, 1) || age > wd->max_age;
    if (!dead) wd->repr_ctr[s] = (e > wd->e_repr) ? wd->repr_ctr[s] + 1 : 0;
  }
  if (dead) {
    wd->alive[s] = 0;
    wd->slot_map[y * wd->W + x] = -1;
    atomicAdd(&wd->ctr->deaths_step, 1);
    atomicAdd(&wd->ctr->an_age_sum, (unsigned long long)wd->age[s]);  // age at death
  }
}

// First free N, S, E, W neighbour of (y, x) after moves and deaths (on the
// grid, not a wall, empty), or -1.  The four cells are read at once.
__device__ inline int first_free_neighbour(const WorldDev &wd, int y, int x) {
  int cell[4], occ[4];
  bool ok[4];
#pragma unroll
  for (int a = 1; a < NACT; ++a) {
    const int ny = y + kDY[a], nx = x + kDX[a];
    ok[a - 1] = ny >= 0 && ny < wd.H && nx >= 0 && nx < wd.W;
    cell[a - 1] = ok[a - 1] ? ny * wd.W + nx : 0;
    occ[a - 1] = ok[a - 1] ? wd.slot_map[cell[a - 1]] : 0;
    if (ok[a - 1]) ok[a - 1] = !bit_at(wd.wall, wd.Wp, ny, nx);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (ok[i] && occ[i] == -1) return cell[i];
  return -1;
}

// ---------------------------------------------------------------- a6 ------
__device__ inline void slot_birth_claim(const WorldDev *wd, int s) {
  wd->birth_cell[s] = -1;
  if (!wd->alive[s] || wd->repr_ctr[s] < wd->t_repr) return;
  const int cell = first_free_neighbour(*wd, wd->y[s], wd->x[s]);
  if (cell < 0) return;
  wd->birth_cell[s] = cell;
  atomicMin(&wd->bclaim[cell], s);
}

// Birth k of the step: parent s, child in free slot `child` on the parent's
// claimed cell; the child starts with e0, zero counters and zero recurrent
// state, the parent's reproduction counter restarts.
__device__ inline void init_child(const WorldDev &wd, int s, int cell, int k, int child,
                                  float *h_next) {
  wd.birth_parent[k] = s;
  wd.birth_child[k] = child;
  wd.repr_ctr[s] = 0;
  wd.alive[child] = 1;
  wd.y[child] = cell / wd.W;
  wd.x[child] = cell % wd.W;
  wd.slot_map[cell] = child;
  wd.energy[child] = wd.e0;
  wd.repr_ctr[child] = 0;
  wd.low_ctr[child] = 0;
  wd.age[child] = 0;
  wd.action[child] = 0;
  wd.prev_act[child] = 0;
  wd.ate[child] = 0;
  wd.lab_seen[child] = 0;
  wd.lab_ate[child] = 0;
  wd.lab_t[child] = 0;
  wd.lab_c[child] = 0;
  wd.arrive[child] = 0u;
  wd.birth_cell[child] = -1;
  float4 *hz = reinterpret_cast<float4 *>(h_next + (size_t)child * HID);
  float4 *cz = reinterpret_cast<float4 *>(wd.c + (size_t)child * HID);
  float4 *lz = reinterpret_cast<float4 *>(wd.logits + (size_t)child * 8);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int j = 0; j < HID / 4; ++j) {
    hz[j] = zero;
    cz[j] = zero;
  }
  lz[0] = zero;
  lz[1] = zero;
}

// Counters at the end of a step: S successful parents, F free slots.
__device__ inline void finish_step(const WorldDev &wd, int S, int F, int pop, uint32_t t) {
  Counters &c = *wd.ctr;
  const int births = min(S, F);
  c.births_last = births;
  c.dropped_last = S - births;
  c.deaths_last = c.deaths_step;
  c.births += births;
  c.dropped += S - births;
  c.deaths += c.deaths_step;
  c.an_deaths += c.deaths_step;
  c.deaths_step = 0;
  c.n_births = births;
  c.births_t = t;
  c.agent_steps += c.pop;  // the agents alive at the start of this step
  c.pop = pop;
  c.t = (long long)t + 1;
  if (c.log) {  // posted stores to host memory; visible once the stream passes the step
    long long *row = c.log + (size_t)((unsigned long long)t % (unsigned long long)c.log_rows) *
                                 ECO_NCOUNTERS;
    row[ECO_C_T] = c.t;
    row[ECO_C_POP] = c.pop;
    row[ECO_C_BIRTHS] = c.births;
    row[ECO_C_DEATHS] = c.deaths;
    row[ECO_C_DROPPED] = c.dropped;
    row[ECO_C_BIRTHS_LAST] = c.births_last;
    row[ECO_C_DEATHS_LAST] = c.deaths_last;
    row[ECO_C_DROPPED_LAST] = c.dropped_last;
    row[ECO_C_AGENT_STEPS] = c.agent_steps;
  }
}


__global__ void __launch_bounds__(SLOT_BLOCK) k_move_apply(const __grid_constant__ BatchDev b) {
  pdl_wait_and_release();
  const WorldDev *wd;
  const int s = slot_of_thread(b, wd);
  if (s >= 0) slot_move_apply(wd, s);
}
__global__ void __launch_bounds__(SLOT_BLOCK) k_physio(const __grid_constant__ BatchDev b) {
  pdl_wait_and_release();
  const WorldDev *wd;
  const int s = slot_of_thread(b, wd);
  if (s >= 0) slot_physio(wd, s);
}
__global__ void __launch_bounds__(SLOT_BLOCK) k_birth_claim(const __grid_constant__ BatchDev b) {
  pdl_wait_and_release();
  const WorldDev *wd;
  const int s = slot_of_thread(b, wd);
  if (s >= 0) slot_birth_claim(wd, s);
}

// Worlds of capacity <= FUSED_MAX_C: every slot phase of a step (moves,
// eating and physiology, birth claims, compaction) in one launch, one
// thread-block cluster of CLUSTER CTAs per world.  Phases are separated by
// the hardware cluster barrier (release/acquire at cluster scope, so the
// global memory one phase writes is visible to the next); the compaction
// exchanges per-CTA totals through distributed shared memory.
constexpr int CLUSTER = 8;

// Exclusive block scan of three counters over the CTA (<= 1024 threads):
// e[i] = sum over lower threads, tot[i] = block total.
__device__ inline void block_scan3(const int v[3], int e[3], int tot[3], int *sh /* [3*32+3] */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc[3] = {v[0], v[1], v[2]};
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int x = __shfl_up_sync(0xFFFFFFFFu, inc[i], o);
      if (lane >= o) inc[i] += x;
    }
  }
  if (lane == 31)
    for (int i = 0; i < 3; ++i) sh[32 * i + warp] = inc[i];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int w0 = lane < nw ? sh[32 * i + lane] : 0;
      int sc = w0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xFFFFFFFFu, sc, o);
        if (lane >= o) sc += x;
      }
      if (lane < nw) sh[32 * i + lane] = sc - w0;
      if (lane == 31) sh[96 + i] = sc;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    e[i] = sh[32 * i + warp] + inc[i] - v[i];
    tot[i] = sh[96 + i];
  }
  __syncthreads();
}

// Exclusive prefix over the cluster's CTAs of three per-CTA totals:
// out[0..2] = sum over lower ranks, out[3..5] = cluster totals.
__device__ inline void cluster_prefix3(cg::cluster_group &cl, int *pub, int *out,
                                       const int v[3]) {
  if (threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) pub[i] = v[i];
  cl.sync();
  if (threadIdx.x == 0) {
    const int me = (int)cl.block_rank();
    int base[3] = {0, 0, 0}, tot[3] = {0, 0, 0};
    for (int r = 0; r < CLUSTER; ++r) {
      const int *rp = cl.map_shared_rank(pub, r);
      for (int i = 0; i < 3; ++i) {
        if (r < me) base[i] += rp[i];
        tot[i] += rp[i];
      }
    }
    for (int i = 0; i < 3; ++i) {
      out[i] = base[i];
      out[3 + i] = tot[i];
    }
  }
  __syncthreads();
}

// Slots per thread of the fused kernel (8 CTAs x 1024 threads per world), and
// the largest capacity one CTA covers with as many slots per thread.
constexpr int CL_SPT = (FUSED_MAX_C + CLUSTER * SCAN_THREADS - 1) / (CLUSTER * SCAN_THREADS);
constexpr int SINGLE_MAX_C = CL_SPT * SCAN_THREADS;

// Every slot phase of a step for one world (the move claims are already
// made by the observation+LSTM kernel).  Each thread owns up to CL_SPT
// consecutive slots and keeps their state in registers from phase to
// phase.  Phases: moves, eating, physiology, death | birth claims |
// compaction.  Moves and physiology share a phase: a winner's target was
// empty at the start of the phase and a dying agent clears its own final
// cell, so their slot-map writes never meet.  The compaction is one scan of
// three counts per slot range -- free slots, successful parents, survivors:
// children fill the free slots of rank below the number of births in slot
// order, so a slot's place in the next alive list is the survivors before
// it plus min(free slots before it, births).
//
// NCTA = CLUSTER: one 8-CTA cluster per world, phases separated by the
// cluster barrier, per-CTA totals exchanged through distributed shared
// memory.  NCTA = 1 (every capacity <= SINGLE_MAX_C): one CTA per world, the
// same phases separated by CTA barriers.
template <int NCTA>
__device__ __forceinline__ void phase_sync() {
  if constexpr (NCTA == 1)
    __syncthreads();
  else
    cg::this_cluster().sync();
}

template <int NCTA, int THREADS>
__device__ __forceinline__ void agents_fused_body(const BatchDev &b) {
  __shared__ int sh[3 * 32 + 3];
  __shared__ int pub[3], ex[6];
  __shared__ int cta_deaths, cta_cand;
  __shared__ int busy[NCTA];   // CTA r of the cluster had a death or a candidate
  __shared__ unsigned long long cta_age_sum;
  const WorldDev &wd = *world_ptr(b, blockIdx.x / NCTA);
  const int rank = NCTA == 1 ? 0 : (int)cg::this_cluster().block_rank();
  // Every CTA of the cluster writes its quiet-step flag into the shared
  // memory of every other after the first phase; this arrival (completed
  // before those writes) makes sure they have all started.
  if constexpr (NCTA > 1) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  const int C = wd.C, W = wd.W, Wp = wd.Wp;
  const int per_cta = (C + NCTA - 1) / NCTA;
  const int c0 = min(C, rank * per_cta), c1 = min(C, c0 + per_cta);
  const int per = (c1 - c0 + THREADS - 1) / THREADS;
  const int s0 = min(c1, c0 + (int)threadIdx.x * per);
  const int ns = min(c1, s0 + per) - s0;
  if (threadIdx.x == 0) {
    cta_deaths = 0;
    cta_cand = 0;
    cta_age_sum = 0ull;
  }
  // The slot state below was last written by the previous step's slot
  // phases, which have completed when this kernel starts (the kernels in
  // between waited for them before releasing theirs), so it is read, through
  // L2, before waiting for the observation+controller kernel; its outputs
  // (targets, kills, claims) after.
  const uint32_t t = (uint32_t)__ldcg(&wd.ctr->t);
  const int pop0 = (int)__ldcg(&wd.ctr->pop);      // agents at the step's start
  uint32_t *res = (t & 1u) ? wd.res0 : wd.res1;  // plane after this step's regrowth
  float *h_next = (t & 1u) ? wd.h0 : wd.h1;

  // In a cluster the first phase takes the slots in chunks of 32, dealt
  // round-robin to the CTAs and within a CTA to its warps (chunk c = (k WARPS
  // + warp) NCTA + rank), so that the live agents, which fill the lowest
  // slots, spread over every SM of the cluster: their scattered slot-map,
  // claim and resource accesses are what the phase's time goes to, and one SM
  // took them all at 1,000 agents (5.6 µs against 2.4 spread).  The later
  // phases take contiguous ranges (their scans follow slot order) and reload
  // the slot state the first one wrote.  One CTA keeps its contiguous slots
  // throughout.
  constexpr int WARPS = THREADS / 32;
  const int lane = (int)threadIdx.x & 31, warp = (int)threadIdx.x >> 5;
  int ms[CL_SPT];   // first-phase slot of k, or -1
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    if constexpr (NCTA > 1) {
      const int s = ((k * WARPS + warp) * NCTA + rank) * 32 + lane;
      ms[k] = s < C ? s : -1;
    } else {
      ms[k] = k < ns ? s0 + k : -1;
    }
  }
  int al[CL_SPT], py[CL_SPT], px[CL_SPT], tgt[CL_SPT], age[CL_SPT], low[CL_SPT],
      rep[CL_SPT], bcell[CL_SPT];
  float en[CL_SPT];
  bool kil[CL_SPT];
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    al[k] = 0;
    if (ms[k] >= 0) {
      const int s = ms[k];
      al[k] = __ldcg(&wd.alive[s]);
      py[k] = __ldcg(&wd.y[s]);
      px[k] = __ldcg(&wd.x[s]);
      en[k] = __ldcg(&wd.energy[s]);
      age[k] = __ldcg(&wd.age[s]);
      low[k] = __ldcg(&wd.low_ctr[s]);
      rep[k] = __ldcg(&wd.repr_ctr[s]);
    }
  }
  pdl_wait_and_release();
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    if (ms[k] >= 0) {
      const int s = ms[k];
      tgt[k] = wd.target[s];
      kil[k] = wd.killed[s] != 0;
    }
  }
  __syncthreads();  // cta_deaths initialised
  // ---- moves (lowest claimant wins), eating, physiology, death
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    if (!al[k]) continue;
    const int s = ms[k];
    if (!ECO_IN_RANGE(wd, py[k] >= 0 && py[k] < wd.H && px[k] >= 0 && px[k] < W)) {
      al[k] = 0;
      wd.alive[s] = 0;   // (range-checked build) out of the step from here on
      continue;
    }
    // The claim and the resource words of both possible final cells are
    // loaded together.  Only this agent can clear its final cell's bit (one
    // agent per cell: a target was empty at the start of the phase and has
    // one winner), so the bit read here is the one it eats, and the clear
    // needs no returned value.
    const bool cand = tgt[k] >= 0 && ECO_IN_RANGE(wd, tgt[k] < wd.H * W);
    const int claimant = cand ? wd.claim[tgt[k]] : -1;
    const int ty = cand ? tgt[k] / W : 0, tx = cand ? tgt[k] % W : 0;
    uint32_t word = __ldcg(&res[py[k] * Wp + (px[k] >> 5)]);
    const uint32_t word_there = cand ? __ldcg(&res[ty * Wp + (tx >> 5)]) : 0u;
    if (cand && claimant == s) {
      wd.claim[tgt[k]] = INT_MAX;  // only the winner resets its cell
      wd.slot_map[py[k] * W + px[k]] = -1;
      wd.slot_map[tgt[k]] = s;
      py[k] = ty;
      px[k] = tx;
      wd.y[s] = py[k];
      wd.x[s] = px[k];
      word = word_there;
    }
    bool dead, ate = false;
    if (kil[k]) {
      dead = true;
    } else {
      const uint32_t bit = 1u << (px[k] & 31);
      ate = (word & bit) != 0u;
      if (ate) atomicAnd(&res[py[k] * Wp + (px[k] >> 5)], ~bit);
      float e = en[k];
      if (ate) e = __fadd_rn(e, wd.e_gain);
      e = __fsub_rn(e, wd.e_decay);
      e = fminf(e, wd.e_max);
      wd.energy[s] = e;
      age[k] += 1;
      wd.age[s] = age[k];
      low[k] = (e <= wd.e_death) ? low[k] + 1 : 0;
      wd.low_ctr[s] = low[k];
      dead = low[k] >= max(wd.t_death, 1) || age[k] > wd.max_age;
      if (!dead) {
        rep[k] = (e > wd.e_repr) ? rep[k] + 1 : 0;
        wd.repr_ctr[s] = rep[k];
        if (rep[k] >= wd.t_repr) cta_cand = 1;   // will try to give birth
      }
    }
    wd.ate[s] = ate ? 1 : 0;  // an input of the paper's controller next step
    if (ate) wd.lab_ate[s] = 1;
    if (dead) {
      al[k] = 0;
      wd.alive[s] = 0;
      wd.slot_map[py[k] * W + px[k]] = -1;
      atomicAdd(&cta_deaths, 1);
      atomicAdd(&cta_age_sum, (unsigned long long)age[k]);  // age at death
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && cta_deaths) {
    atomicAdd(&wd.ctr->deaths_step, cta_deaths);
    atomicAdd(&wd.ctr->an_age_sum, cta_age_sum);
  }
  if constexpr (NCTA > 1) {
    asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    if (threadIdx.x < NCTA)
      *cg::this_cluster().map_shared_rank(&busy[rank], (int)threadIdx.x) =
          (cta_deaths || cta_cand) ? 1 : 0;
  } else if (threadIdx.x == 0) {
    busy[0] = (cta_deaths || cta_cand) ? 1 : 0;
  }
  phase_sync<NCTA>();
  // A quiet step -- no death and no reproduction candidate in the whole
  // world (every CTA's flag is in after the barrier) -- leaves the alive
  // list as it is (survivors in slot order, no child): the birth and
  // compaction phases are skipped, last step's newborns are newborns no
  // more.
  bool quiet = true;
#pragma unroll
  for (int r = 0; r < NCTA; ++r) quiet = quiet && busy[r] == 0;
  if (quiet) {
    for (int i = rank * THREADS + (int)threadIdx.x; i < pop0; i += NCTA * THREADS)
      wd.alive_new[i] = 0;
    if (rank == 0 && threadIdx.x == 0) finish_step(wd, 0, 0, pop0, t);
    return;
  }
  // slot state of the contiguous range, as the first phase left it (the
  // barrier above makes every CTA's writes visible)
  if constexpr (NCTA > 1) {
#pragma unroll
    for (int k = 0; k < CL_SPT; ++k) {
      al[k] = 0;
      if (k < ns) {
        const int s = s0 + k;
        al[k] = __ldcg(&wd.alive[s]);
        py[k] = __ldcg(&wd.y[s]);
        px[k] = __ldcg(&wd.x[s]);
        rep[k] = __ldcg(&wd.repr_ctr[s]);
      }
    }
  }
  // ---- birth claims: first free N, S, E, W cell; lowest parent slot wins
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    bcell[k] = -1;
    if (!al[k] || rep[k] < wd.t_repr) continue;
    bcell[k] = first_free_neighbour(wd, py[k], px[k]);
    if (bcell[k] >= 0) atomicMin(&wd.bclaim[bcell[k]], s0 + k);
  }
  phase_sync<NCTA>();
  // ---- compaction (contiguous slots per thread, so ranks follow slot order)
  bool ok[CL_SPT];
  int cnt[3] = {0, 0, 0};  // free slots, successful parents, survivors
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    ok[k] = al[k] && bcell[k] >= 0 && wd.bclaim[bcell[k]] == s0 + k;
    cnt[0] += (k < ns && !al[k]) ? 1 : 0;
    cnt[1] += ok[k];
    cnt[2] += al[k];
  }
  int off[3], tot[3];
  block_scan3(cnt, off, tot, sh);
  if constexpr (NCTA == 1) {
    if (threadIdx.x == 0)
      for (int i = 0; i < 3; ++i) {
        ex[i] = 0;
        ex[3 + i] = tot[i];
      }
    __syncthreads();   // every claim cell read before any reset
  } else {
    cg::cluster_group cl = cg::this_cluster();
    cluster_prefix3(cl, pub, ex, tot);  // every claim cell read before any reset
  }
  int free_off = off[0] + ex[0], succ_off = off[1] + ex[1];
  const int surv_off = off[2] + ex[2];
  const int F = ex[3], S = ex[4], SURV = ex[5];
  const int births = min(S, F);
  int alive_pos = surv_off + min(free_off, births);
  int free_rank = free_off;
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    if (bcell[k] >= 0) wd.bclaim[bcell[k]] = INT_MAX;
    if (k < ns && !al[k]) {
      if (free_rank < S) wd.free_list[free_rank] = s0 + k;
      ++free_rank;
    }
  }
  phase_sync<NCTA>();
  free_rank = free_off;
#pragma unroll
  for (int k = 0; k < CL_SPT; ++k) {
    if (k >= ns) continue;
    const int s = s0 + k;
    if (ok[k]) {
      const int kk = succ_off++;
      if (kk < F) {
        const int child = wd.free_list[kk];
        if (ECO_IN_RANGE(wd, child >= 0 && child < wd.C))
          init_child(wd, s, bcell[k], kk, child, h_next);
      }
    }
    // the next alive list: survivors and the free slots that receive a child
    if (al[k]) {
      wd.alive_new[alive_pos] = 0;
      wd.alive_list[alive_pos++] = s;
    } else if (free_rank++ < births) {
      wd.alive_new[alive_pos] = 1;
      wd.alive_list[alive_pos++] = s;
    }
  }
  if (rank == 0 && threadIdx.x == 0) finish_step(wd, S, F, SURV + births, t);
  // no closing barrier: the last reads of another CTA's shared memory (the
  // per-CTA totals of the compaction) precede the barrier before the
  // children, so a CTA may leave as soon as it is done
}

__global__ void __cluster_dims__(CLUSTER, 1, 1) __launch_bounds__(SCAN_THREADS)
    k_agents_cluster(const __grid_constant__ BatchDev b) {
  agents_fused_body<CLUSTER, SCAN_THREADS>(b);
}

__global__ void __launch_bounds__(SCAN_THREADS) k_agents_single(const __grid_constant__ BatchDev b) {
  agents_fused_body<1, SCAN_THREADS>(b);
}

// ---------------------------------------------------------------------------
// Split compaction (worlds of any capacity): the same ranks as the cluster
// kernel's, over blocks of SLOT_BLOCK slots in four kernels --
//   count     per block: free slots, successful parents, survivors
//   prefix    per world, one CTA: exclusive prefixes of the block counts,
//             totals, and the step's counters
//   lists     per block: claim resets, the free slots the births take, the
//             next alive list (survivors before + min(free before, births))
//   children  per block: birth k (ascending parent) takes free slot k
// scan_blocks[4*blk + i] holds block blk's count i, then its prefix;
// scan_blocks[4*nb + i] the world's total i.
// ---------------------------------------------------------------------------
__device__ inline int slot_blocks(const WorldDev &wd) { return (wd.C + SLOT_BLOCK - 1) / SLOT_BLOCK; }

__global__ void __launch_bounds__(SLOT_BLOCK) k_scan_count(const __grid_constant__ BatchDev b) {
  __shared__ int sh[3 * 32 + 3];
  pdl_wait_and_release();
  const WorldDev *wdp;
  const int s = slot_of_thread(b, wdp);
  const WorldDev &wd = *wdp;
  int v[3] = {0, 0, 0};
  if (s >= 0) {
    const int a = wd.alive[s];
    const int cell = wd.birth_cell[s];
    const bool ok = a && cell >= 0 && ECO_IN_RANGE(wd, cell < wd.H * wd.W) &&
                    wd.bclaim[cell] == s;
    wd.flag[s] = ok ? 1 : 0;
    v[0] = a ? 0 : 1;
    v[1] = ok ? 1 : 0;
    v[2] = a ? 1 : 0;
  }
  int e[3], tot[3];
  block_scan3(v, e, tot, sh);
  if (threadIdx.x == 0) {   // the block's first slot exists
    const int blk = s / SLOT_BLOCK;
    for (int i = 0; i < 3; ++i) wd.scan_blocks[4 * blk + i] = tot[i];
  }
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_prefix(const __grid_constant__ BatchDev b) {
  __shared__ int sh[3 * 32 + 3];
  pdl_wait_and_release();
  const WorldDev &wd = *world_ptr(b, blockIdx.x);
  const int nb = slot_blocks(wd);
  const int per = (nb + SCAN_THREADS - 1) / SCAN_THREADS;
  const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
  int v[3] = {0, 0, 0};
  for (int k = b0; k < b1; ++k)
    for (int i = 0; i < 3; ++i) v[i] += wd.scan_blocks[4 * k + i];
  int e[3], tot[3];
  block_scan3(v, e, tot, sh);
  for (int k = b0; k < b1; ++k)
    for (int i = 0; i < 3; ++i) {
      const int c = wd.scan_blocks[4 * k + i];
      wd.scan_blocks[4 * k + i] = e[i];
      e[i] += c;
    }
  if (threadIdx.x == 0) {
    for (int i = 0; i < 3; ++i) wd.scan_blocks[4 * nb + i] = tot[i];
    const int F = tot[0], S = tot[1], SURV = tot[2];
    // counters of the step; the later kernels read births_t, never t
    finish_step(wd, S, F, SURV + min(S, F), (uint32_t)wd.ctr->t);
  }
}

__global__ void __launch_bounds__(SLOT_BLOCK) k_scan_lists(const __grid_constant__ BatchDev b) {
  __shared__ int sh[3 * 32 + 3];
  pdl_wait_and_release();
  const WorldDev *wdp;
  const int s = slot_of_thread(b, wdp);
  const WorldDev &wd = *wdp;
  const int nb = slot_blocks(wd);
  int v[3] = {0, 0, 0};
  int a = 0;
  if (s >= 0) {
    a = wd.alive[s];
    v[0] = a ? 0 : 1;
    v[1] = wd.flag[s];
    v[2] = a ? 1 : 0;
  }
  int e[3], tot[3];
  block_scan3(v, e, tot, sh);
  if (s < 0) return;
  const int blk = s / SLOT_BLOCK;
  const int F = wd.scan_blocks[4 * nb], S = wd.scan_blocks[4 * nb + 1];
  const int births = min(S, F);
  const int free_before = wd.scan_blocks[4 * blk] + e[0];
  const int surv_before = wd.scan_blocks[4 * blk + 2] + e[2];
  const int cell = wd.birth_cell[s];
  if (cell >= 0 && cell < wd.H * wd.W) wd.bclaim[cell] = INT_MAX;
  const int pos = surv_before + min(free_before, births);
  if (a) {
    wd.alive_list[pos] = s;
    wd.alive_new[pos] = 0;
  } else {
    if (free_before < S) wd.free_list[free_before] = s;
    if (free_before < births) {   // receives a child
      wd.alive_list[pos] = s;
      wd.alive_new[pos] = 1;
    }
  }
}

__global__ void __launch_bounds__(SLOT_BLOCK) k_scan_children(const __grid_constant__ BatchDev b) {
  __shared__ int sh[3 * 32 + 3];
  pdl_wait_and_release();
  const WorldDev *wdp;
  const int s = slot_of_thread(b, wdp);
  const WorldDev &wd = *wdp;
  const int nb = slot_blocks(wd);
  int v[3] = {0, 0, 0};
  if (s >= 0) v[1] = wd.flag[s];
  int e[3], tot[3];
  block_scan3(v, e, tot, sh);
  if (s < 0 || !v[1]) return;
  const int blk = s / SLOT_BLOCK;
  const int F = wd.scan_blocks[4 * nb];
  const int k = wd.scan_blocks[4 * blk + 1] + e[1];
  if (k >= F) return;   // dropped: the parent keeps its counter
  const int child = wd.free_list[k];
  if (!ECO_IN_RANGE(wd, child >= 0 && child < wd.C)) return;
  const uint32_t t = wd.ctr->births_t;   // the step's index (finish_step ran)
  init_child(wd, s, wd.birth_cell[s], k, child, (t & 1u) ? wd.h0 : wd.h1);
}

// Child weights, physical layout: W[child][p] = W[parent][p] + sigma * N_j
// with N_j normal j = logical index of p of the stream (TAG_MUT, t, parent).
// A float4 of a weight row or of the read-out holds four consecutive logical
// indices starting at a multiple of 4, so one Philox draw serves it; the
// bias rows of a block are permuted and take one draw per element.
constexpr int SPAWN_THREADS = 256;

// Four consecutive logical parameters j .. j+3 (j a multiple of 4, or -1:
// padding) plus scale * N of one Philox draw; parameters from np on are
// padding (zero).
__device__ inline float4 mutate_quad(const WorldDev &wd, float4 base, int j, int np,
                                     uint32_t tag, uint32_t t, uint32_t id, float scale) {
  if (j < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  float z[4];
  normals4(wd.key0, wd.key1, (uint32_t)j >> 2, t, tag, id, z);
  float out[4] = {base.x, base.y, base.z, base.w};
#pragma unroll
  for (int i = 0; i < 4; ++i)
    out[i] = (j + i < np) ? __fadd_rn(out[i], __fmul_rn(scale, z[i])) : 0.f;
  return make_float4(out[0], out[1], out[2], out[3]);
}

// One parameter j plus scale * N_j (normal j & 3 of draw j >> 2).
__device__ inline float mutate_one(const WorldDev &wd, float base, int j, uint32_t tag,
                                   uint32_t t, uint32_t id, float scale) {
  float z[4];
  normals4(wd.key0, wd.key1, (uint32_t)j >> 2, t, tag, id, z);
  const int i = j & 3;
  const float zi = i == 0 ? z[0] : i == 1 ? z[1] : i == 2 ? z[2] : z[3];
  return __fadd_rn(base, __fmul_rn(scale, zi));
}

// The bias float4 number b4 (0..7) of block q: rows 4 b4 .. 4 b4 + 3, whose
// logical rows are not consecutive, so each takes its own draw.
__device__ inline float4 mutate_bias4(const WorldDev &wd, float4 base, int q, int b4,
                                      uint32_t tag, uint32_t t, uint32_t id, float scale) {
  float in[4] = {base.x, base.y, base.z, base.w}, out[4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
    out[i] = mutate_one(wd, in[i], OFF_B + blk_row_to_logical(q, 4 * b4 + i), tag, t, id, scale);
  return make_float4(out[0], out[1], out[2], out[3]);
}

// Float4 number vi of an agent's physical weights after adding scale * N_j
// (stream tag, t, id) to `base` (initial weights; the mutation of births
// walks the row by parts, below).  The paper controller's rows are in
// logical order, so every float4 is four consecutive parameters.
__device__ inline float4 mutate4(const WorldDev &wd, int vi, float4 base, uint32_t tag,
                                 uint32_t t, uint32_t id, float scale) {
  const int p = vi * 4;
  if (wd.controller == ECO_CTRL_PAPER)
    return mutate_quad(wd, base, p < PC_NPARAM ? p : -1, PC_NPARAM, tag, t, id, scale);
  const int o = p % BLK_FLOATS;
  if (p < TAIL && o >= BLK_ROWS * NIN)
    return mutate_bias4(wd, base, p / BLK_FLOATS, (o - BLK_ROWS * NIN) / 4, tag, t, id, scale);
  return mutate_quad(wd, base, logical_of_phys(p), NPARAM, tag, t, id, scale);
}

// Work items of the mutation: (birth, part of its weight row), dealt to the
// CTAs round-robin.  With the LSTM(32) controller the parts are the four
// hidden-unit blocks (1,440 float4s of gate rows, a row's 45 float4s being
// consecutive logical parameters, then 8 float4s of biases) and the
// read-out; with the paper's controller, chunks of SPAWN_CHUNK float4s.  A
// CTA's threads take the float4s of an item in turn, each thread issuing the
// loads of SPAWN_UNROLL float4s before any of their arithmetic.  The birth's
// world, parent, child and step are looked up once per item (a first version
// looked them up, with a 64-bit division, for every float4; the next one
// derived each float4's logical index from its physical offset with two
// divisions).
constexpr int SPAWN_CHUNK = 1024;
constexpr int SPAWN_UNROLL = 2;
constexpr int ROW_VECS = NIN / 4;                 // 45 float4s per gate row
constexpr int BLK_VECS = BLK_FLOATS / 4;          // 1,448 float4s per block
constexpr int BLK_W_VECS = BLK_ROWS * ROW_VECS;   // 1,440 of them gate rows
static_assert(NIN % 4 == 0 && BLK_FLOATS % 4 == 0 && TAIL % 4 == 0, "float4 parts");

// Mutation of every birth of the batch by CTAs cta .. of n_cta.
__device__ inline void spawn_births(const BatchDev &b, int *pre, int cta, int n_cta) {
  if (threadIdx.x == 0) {
    int run = 0;
    for (int w = 0; w < b.n; ++w) {
      pre[w] = run;
      const WorldDev &wdw = *world_ptr(b, w);
      int nb = wdw.ctr->n_births;
      if (!ECO_IN_RANGE(wdw, nb >= 0 && nb <= wdw.C)) nb = 0;
      run += nb;
    }
    pre[b.n] = run;
  }
  __syncthreads();
  const bool lstm = b.controller != ECO_CTRL_PAPER;
  const int nvec = b.wstride / 4;
  const int per = lstm ? NBLK + 1 : (nvec + SPAWN_CHUNK - 1) / SPAWN_CHUNK;  // parts per birth
  const int items = pre[b.n] * per;
  for (int item = cta; item < items; item += n_cta) {
    const int bi = item / per, part = item - bi * per;
    int v0, v1;
    if (lstm) {
      v0 = part * BLK_VECS;
      v1 = part < NBLK ? v0 + BLK_VECS : nvec;
    } else {
      v0 = part * SPAWN_CHUNK;
      v1 = min(nvec, v0 + SPAWN_CHUNK);
    }
    int lo = 0, hi = b.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= bi) lo = mid; else hi = mid - 1;
    }
    const WorldDev &wd = *world_ptr(b, lo);
    const int k = bi - pre[lo];
    const int par = wd.birth_parent[k], child = wd.birth_child[k];
    if (!ECO_IN_RANGE(wd, par >= 0 && par < wd.C && child >= 0 && child < wd.C)) continue;
    const uint32_t t = wd.ctr->births_t;
    const float sigma = wd.mut_std;
    const float4 *src = reinterpret_cast<const float4 *>(wd.weights + (size_t)par * b.wstride);
    float4 *dst = reinterpret_cast<float4 *>(wd.weights + (size_t)child * b.wstride);
    for (int vi = v0 + (int)threadIdx.x; vi < v1; vi += SPAWN_UNROLL * (int)blockDim.x) {
      float4 in[SPAWN_UNROLL];
#pragma unroll
      for (int u = 0; u < SPAWN_UNROLL; ++u) {
        const int v = vi + u * (int)blockDim.x;
        if (v < v1) in[u] = src[v];
      }
#pragma unroll
      for (int u = 0; u < SPAWN_UNROLL; ++u) {
        const int v = vi + u * (int)blockDim.x;
        if (v >= v1) continue;
        float4 r;
        if (!lstm) {
          const int j = 4 * v;
          r = mutate_quad(wd, in[u], j < PC_NPARAM ? j : -1, PC_NPARAM, TAG_MUT, t, par, sigma);
        } else if (part == NBLK) {   // read-out, in logical order; then padding
          const int j = 4 * v;
          r = mutate_quad(wd, in[u], j < NPARAM ? j : -1, NPARAM, TAG_MUT, t, par, sigma);
        } else {
          const int f = v - v0;
          if (f < BLK_W_VECS) {
            const int l = f / ROW_VECS, k4 = f - l * ROW_VECS;
            const int j = blk_row_to_logical(part, l) * NIN + 4 * k4;
            r = mutate_quad(wd, in[u], j, NPARAM, TAG_MUT, t, par, sigma);
          } else {
            r = mutate_bias4(wd, in[u], part, f - BLK_W_VECS, TAG_MUT, t, par, sigma);
          }
        }
        dst[v] = r;
      }
    }
  }
}

// The tail of a step, launched first in the next one: the regrowth of that
// step's plane (the first total_tiles CTAs) and the mutation of the births
// of the step before (the others), in
// one launch -- they touch disjoint data (resource planes / weights).
constexpr int SPAWN_CTAS_PER_SM = 4;
static_assert(REGROW_THREADS == SPAWN_THREADS, "one block size for the tail kernel");

__global__ void __launch_bounds__(SPAWN_THREADS, 4) k_tail(const __grid_constant__ BatchDev b) {
  __shared__ union {
    RegrowSmem rg;    // regrowth CTAs
    int pre[1025];    // mutation CTAs: births per world, prefix
  } sm;
  // The controller kernel after this one starts its reads early when this
  // grid is small enough (b.tail_early) to leave room for it beside the
  // tail's CTAs; a larger grid (many worlds' regrowth tiles) lets it launch
  // only as its CTAs finish, since controller CTAs taking SMs early would
  // halve the tail's occupancy while their gather warps wait for it anyway.
  if ((int)blockIdx.x < b.total_tiles) {
    // walls and thresholds are never written by a step: read before waiting
    const RegrowPlace f = regrow_fixed(b, blockIdx.x, sm.rg);
    pdl_wait();
    if (b.tail_early) pdl_release();
    regrow_run(f, b.regrow_k, sm.rg);
  } else {
    pdl_wait();
    if (b.tail_early) pdl_release();
    spawn_births(b, sm.pre, blockIdx.x - b.total_tiles, gridDim.x - b.total_tiles);
  }
  if (!b.tail_early) pdl_release();
}

// Initial weights of slots [0, n0): w_init_std * N_j of (TAG_INIT_W, 0, slot).
__global__ void __launch_bounds__(SPAWN_THREADS) k_init_weights(const WorldDev *wdp, int n0) {
  const WorldDev &wd = *wdp;
  const int nvec = wd.wstride / 4;
  const long long total = (long long)n0 * nvec;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(g / nvec), vi = (int)(g % nvec);
    reinterpret_cast<float4 *>(wd.weights + (size_t)s * wd.wstride)[vi] =
        mutate4(wd, vi, make_float4(0.f, 0.f, 0.f, 0.f), TAG_INIT_W, 0u, (uint32_t)s,
                wd.w_init_std);
  }
}

void preload_agents() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_move_apply);
  cudaFuncGetAttributes(&a, k_physio);
  cudaFuncGetAttributes(&a, k_birth_claim);
  cudaFuncGetAttributes(&a, k_scan_count);
  cudaFuncGetAttributes(&a, k_scan_prefix);
  cudaFuncGetAttributes(&a, k_scan_lists);
  cudaFuncGetAttributes(&a, k_scan_children);
  cudaFuncGetAttributes(&a, k_agents_cluster);
  cudaFuncGetAttributes(&a, k_agents_single);
  // The tail kernel asks for the shared-memory carveout of the controller
  // kernel that follows it (the largest), so that an SM running tail CTAs
  // need not change its split between L1 and shared memory before the
  // controller kernel's CTAs start beside them (programmatic dependent
  // launch).
  cudaFuncGetAttributes(&a, k_tail);
  cudaFuncSetAttribute(k_tail, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
}

void launch_move_apply(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_move_apply, b.total_slot_blocks, SLOT_BLOCK, 0, s, b);
}
void launch_physio(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_physio, b.total_slot_blocks, SLOT_BLOCK, 0, s, b);
}
void launch_birth_claim(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_birth_claim, b.total_slot_blocks, SLOT_BLOCK, 0, s, b);
}
void launch_scan_count(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_scan_count, b.total_slot_blocks, SLOT_BLOCK, 0, s, b);
}
void launch_scan_prefix(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_scan_prefix, b.n, SCAN_THREADS, 0, s, b);
}
void launch_scan_lists(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_scan_lists, b.total_slot_blocks, SLOT_BLOCK, 0, s, b);
}
void launch_scan_children(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_scan_children, b.total_slot_blocks, SLOT_BLOCK, 0, s, b);
}
void launch_agents_fused(const BatchDev &b, cudaStream_t s) {
  if (b.max_capacity <= SINGLE_MAX_C)
    launch_step_kernel(k_agents_single, b.n, SCAN_THREADS, 0, s, b);
  else
    launch_step_kernel(k_agents_cluster, b.n * CLUSTER, SCAN_THREADS, 0, s, b);
}
void launch_tail(const BatchDev &b, cudaStream_t s) {
  const int spawn = b.spawn_ctas > 0 ? b.spawn_ctas : SPAWN_CTAS_PER_SM * b.n_sms;
  launch_step_kernel(k_tail, b.total_tiles + spawn, SPAWN_THREADS, 0, s, b);
}
void launch_init_weights(const WorldDev *wd_dev, int n0, int n_sms, cudaStream_t s) {
  if (n0 > 0) k_init_weights<<<8 * n_sms, SPAWN_THREADS, 0, s>>>(wd_dev, n0);
}

}  // namespace eco
