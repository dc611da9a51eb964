// k_lstm.cu -- step parts a2 + a3: observation gather and one LSTM step per
// agent (App. B.2, sensorimotor ability and cognitive capacity).
//
// Every agent has its own 93 KB of FP32 weights, used once per step, so the
// step is a batched GEMV bound by HBM bandwidth (about 0.5 flop per byte).
// A persistent grid of one CTA per SM (or two, each with half the ring: a
// launch-shape choice) runs a warp-specialised pipeline with no global
// synchronisation:
//   * CTA b takes the batch's agents b, b + G, b + 2G, ... (world-major,
//     alive-list order; G CTAs), so its first agent is known before the
//     population is: with one world its slot is requested together with the
//     population, and the first copy waits for one round trip;
//   * producer warp: slots and newborn flags of 32 agents at a time (one
//     lane each), and each agent's four weight blocks (a block = the 32
//     gate rows of 8 hidden units, 23,168 B; the last block also carries
//     the read-out) streamed with plain (non-multicast) cp.async.bulk copies
//     into a shared-memory ring of LSTAGES blocks (8: two agents in flight,
//     ~190 KB; 4 with two CTAs per SM);
//   * four gather warps, taking the agents in turn: slots, positions and
//     energies of 32 of their agents at a time, then per agent the 7x7x3
//     window (row masks of the bit planes staged through shared memory),
//     h and c in one round trip (about 4 us while the weight stream fills
//     the memory system: four warps keep four in flight) into an 8-entry
//     ring of inputs [obs(148); h(32)] and cell states;
//   * four compute warps, warp q on block q: lane l computes gate row l with
//     128-bit shared loads (conflict-free: rows are 720 B apart), the gate
//     nonlinearity, and lanes 0, 4, .., 28 update the cell of their hidden
//     unit; warp 3 then takes the 32 new hidden values, computes the 5
//     logits and the argmax (first maximum), and makes the agent's move
//     claim (step part a4), pipelined one agent behind.
// Every hand-off is an mbarrier with a bounded wait; a wait that runs out
// sets ST_TIMEOUT, every role leaves its loop, and the CTA waits (bounded)
// for the copies it issued before returning.
#include <cstddef>

#include "ecoevo_dev.cuh"
#include "move_claim.cuh"

namespace eco {

constexpr int VRING = 8;                   // gathered inputs in flight
constexpr int NCOMP = 4;                   // compute warps (one per block)
constexpr int NGATH = 4;                   // gather warps
constexpr int W_PROD = NCOMP + NGATH;      // producer warp index
constexpr int LTHREADS = (NCOMP + NGATH + 1) * 32;
constexpr int MAX_BATCH = 1024;
constexpr int VLEN = 184;                  // 180 inputs padded to 16 B
constexpr int STAGE_FLOATS = 5960;         // block + read-out (165) + pad
static_assert((STAGE_FLOATS * 4) % 16 == 0, "bulk copies are 16-B multiples");
static_assert(3 * BLK_FLOATS + STAGE_FLOATS <= WSTRIDE, "last copy stays in the slot");
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

// 16-byte aligned: the compute warps read v with 128-bit loads.
struct __align__(16) VEntry {
  float v[VLEN];      // [obs; h_prev]
  float c[HID];       // cell state before the step
  float hn[HID];      // new hidden state, filled by the compute warps
  float *c_row, *h_row, *logits_row;  // outputs of the agent
  int32_t *action;
  const WorldDev *wd;
  int slot, y, x;
  int forced;         // action imposed on the move (use_forced), else -1
};
static_assert(sizeof(VEntry) % 16 == 0 && offsetof(VEntry, v) == 0,
              "ring entries keep v 16-byte aligned");

// What the gather's window loads of one agent depend on: its slot, world,
// position, energy, forced action (-1: its own) and the world's step counter.
struct AgentDesc {
  int slot, world, y, x;
  float energy;
  int forced;
  uint32_t t;
};

template <int LSTAGES>
struct __align__(128) LstmSmem {
  float stage[LSTAGES][STAGE_FLOATS];
  VEntry ring[VRING];
  uint32_t masks[NGATH][16];
  unsigned long long full[LSTAGES], empty[LSTAGES];
  unsigned long long vfull[VRING], vempty[VRING], hready[VRING];
  int prefix[MAX_BATCH + 1];
  int issued;
  volatile int abort_flag;
};
static_assert(offsetof(LstmSmem<4>, ring) % 16 == 0 && offsetof(LstmSmem<8>, ring) % 16 == 0 &&
                  (STAGE_FLOATS * 4) % 16 == 0,
              "bulk-copy stages and ring entries are 16-byte aligned");

__device__ inline uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ inline unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ inline void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count)
               : "memory");
}
__device__ inline void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ inline void mbar_arrive(unsigned long long *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ inline bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity.
__device__ inline bool mbar_wait(unsigned long long *bar, uint32_t parity,
                                 unsigned long long limit_ns = WAIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
__device__ inline void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes,
                                     unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
      "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Seven cells [xs, xs+7) of a bit-plane row; cells off the grid read `fill`.
__device__ inline uint32_t row7(const uint32_t *row, int Wp, int W, int xs,
                                bool fill) {
  const int w0 = xs >> 5, off = xs & 31;
  const uint32_t lo = (w0 >= 0 && w0 < Wp) ? row[w0] : 0u;
  const uint32_t hi = (w0 + 1 >= 0 && w0 + 1 < Wp) ? row[w0 + 1] : 0u;
  uint32_t m = (uint32_t)((((uint64_t)hi << 32) | lo) >> off) & 0x7Fu;
  if (fill) {
#pragma unroll
    for (int b = 0; b < 7; ++b)
      if (xs + b < 0 || xs + b >= W) m |= 1u << b;
  }
  return m;
}

// Input of one agent into a ring entry, by one warp: [obs(148); h(32)] and
// the cell state.  The grid is the resource plane after this step's
// regrowth, the agent channel is the start-of-step occupancy without the
// agent itself, off-grid cells read as wall, the last observation is the
// agent's energy.  Every load depends only on the descriptor: gather_load
// issues them all (one round trip) before the warp waits for its ring
// entry, gather_store fills the entry.
struct GatherRegs {
  uint32_t mask;     // lanes 0..13: a row mask (resource rows, then wall rows)
  float occ0, occ1, hp, cp;
};

__device__ inline GatherRegs gather_load(const WorldDev &wd, const AgentDesc &d, int lane) {
  const int H = wd.H, W = wd.W, Wp = wd.Wp;
  const uint32_t *res = (d.t & 1u) ? wd.res0 : wd.res1;
  const float *h_prev = (d.t & 1u) ? wd.h1 : wd.h0;
  GatherRegs g;
  g.mask = 0u;
  if (lane < 14) {
    const bool is_wall = lane >= 7;
    const int yy = d.y - 3 + (is_wall ? lane - 7 : lane);
    if (yy < 0 || yy >= H)
      g.mask = is_wall ? 0x7Fu : 0u;
    else
      g.mask = row7((is_wall ? wd.wall : res) + (size_t)yy * Wp, Wp, W, d.x - 3, is_wall);
  }
  int occ[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int k = lane + 32 * r;
    const int yy = d.y + k / 7 - 3, xx = d.x + k % 7 - 3;
    occ[r] = -1;
    if (k < 49 && k != 24 && yy >= 0 && yy < H && xx >= 0 && xx < W)
      occ[r] = __ldcg(&wd.slot_map[(size_t)yy * W + xx]);
  }
  g.occ0 = occ[0] >= 0 ? 1.f : 0.f;
  g.occ1 = occ[1] >= 0 ? 1.f : 0.f;
  g.hp = __ldcg(&h_prev[(size_t)d.slot * HID + lane]);
  g.cp = __ldcg(&wd.c[(size_t)d.slot * HID + lane]);
  return g;
}

__device__ inline void gather_store(const WorldDev &wd, const AgentDesc &d, const GatherRegs &g,
                                    VEntry &e, uint32_t *masks, int lane) {
  if (lane < 14) masks[lane] = g.mask;
  __syncwarp();
  e.v[49 + lane] = g.occ0;
  if (lane + 32 < 49) e.v[49 + 32 + lane] = g.occ1;
  for (int k = lane; k < 49; k += 32) {
    const int r = k / 7, cc = k % 7;
    e.v[k] = (float)((masks[r] >> cc) & 1u);
    e.v[98 + k] = (float)((masks[7 + r] >> cc) & 1u);
  }
  if (lane == 0) {
    // greediness window: a resource in view
    uint32_t any = 0u;
#pragma unroll
    for (int r = 0; r < 7; ++r) any |= masks[r];
    if (any) wd.lab_seen[d.slot] = 1;
    e.v[147] = d.energy;
    e.slot = d.slot;
    e.y = d.y;
    e.x = d.x;
    e.forced = d.forced;
    e.wd = &wd;
    e.c_row = wd.c + (size_t)d.slot * HID;
    e.h_row = ((d.t & 1u) ? wd.h0 : wd.h1) + (size_t)d.slot * HID;
    e.logits_row = wd.logits + (size_t)d.slot * 8;
    e.action = wd.action + d.slot;
  }
  e.v[NOBS + lane] = g.hp;
  e.c[lane] = g.cp;
}

// Agent a of the batch (world-major, alive-list order): its world and its
// position in that world's alive list.
__device__ inline int local_index(const int *prefix, const BatchDev &b, int a, int *world) {
  const int w = b.n == 1 ? 0 : world_of(prefix, b.n, a);
  *world = w;
  return a - (b.n == 1 ? 0 : prefix[w]);
}

// Slot and newborn flag of batch agent a, by one lane, as loaded: nothing
// when a >= bound.  The bound is the population, or, for the loads issued
// before the population is known (one world), the capacity: an entry past
// the population is stale, so agent_valid() decides, once the population
// is known, whether the lane's agent exists before anything uses its slot.
struct AgentRef {
  int slot, fresh, world;
};
__device__ inline AgentRef agent_ref(const int *prefix, const BatchDev &b, long long a,
                                     long long bound) {
  AgentRef r{0, 0, 0};
  if (a < bound) {
    const int li = local_index(prefix, b, (int)a, &r.world);
    const WorldDev &wd = *world_ptr(b, r.world);
    r.slot = __ldcg(&wd.alive_list[li]);
    r.fresh = __ldcg(&wd.alive_new[li]);
  }
  return r;
}
// The reference of agent a if it exists (a < A, slot range-checked in the
// checked build), else slot 0 of world 0 (never stepped, loads in range).
__device__ inline AgentRef agent_valid(const BatchDev &b, AgentRef r, long long a, long long A) {
  if (a >= A) return AgentRef{0, 0, 0};
  r.slot = checked_index(*world_ptr(b, r.world), r.slot, world_ptr(b, r.world)->C);
  return r;
}

// LSTAGES weight blocks in the ring, MINB CTAs per SM.
template <int LSTAGES, int MINB>
__global__ void __launch_bounds__(LTHREADS, MINB) k_lstm(const __grid_constant__ BatchDev b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  LstmSmem<LSTAGES> &sm = *reinterpret_cast<LstmSmem<LSTAGES> *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned FULL = 0xFFFFFFFFu;
  const int G = gridDim.x;

  // The kernel before this one in a step is the tail (this step's
  // regrowth, the mutation of the last step's births); the one before that
  // (the slot phases) has completed by the time this kernel starts, since
  // every tail CTA waits for it before it lets this kernel launch.  So the
  // populations, alive lists and newborn flags, the weights of every agent
  // not born in the last step, and everything the gather reads but the
  // resource plane, are read before waiting for the tail (through L2,
  // ld.cg); the resource plane and the newborns' weights only after.
  pdl_release();

  // CTA b steps the batch's agents b, b + G, b + 2G, ...  With one world the
  // population and the first 32 slots of the producer and of each gather
  // warp are requested at once, before the barriers are set up, so the
  // first copy waits for one round trip.
  const int role_first = warp == W_PROD ? 0 : (warp >= NCOMP ? warp - NCOMP : -1);
  const int role_step = warp == W_PROD ? 1 : NGATH;   // CTA-local agents n = first + step k
  AgentRef pre{0, 0, 0};
  if (b.n == 1) {
    const WorldDev &w0 = *world_ptr(b, 0);
    const int pop = (warp == W_PROD && lane == 0) ? (int)__ldcg(&w0.ctr->pop) : 0;
    if (role_first >= 0) {
      const long long a = blockIdx.x + (long long)(role_first + role_step * lane) * G;
      pre = agent_ref(sm.prefix, b, a, w0.C);   // guarded by the capacity only
    }
    if (warp == W_PROD && lane == 0) {
      sm.prefix[0] = 0;
      sm.prefix[1] = pop;
    }
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < LSTAGES; ++i) {
      mbar_init(&sm.full[i], 1);
      mbar_init(&sm.empty[i], 1);
    }
    for (int i = 0; i < VRING; ++i) {
      mbar_init(&sm.vfull[i], 1);
      mbar_init(&sm.vempty[i], 1);
      mbar_init(&sm.hready[i], NCOMP);
    }
    sm.issued = 0;
    sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // agents per world (= alive-list length at the start of the step), for
  // batches of several worlds
  if (warp == 0 && b.n > 1) {
    const int per = (b.n + 31) / 32;
    int local = 0;
    for (int i = 0; i < per; ++i) {
      const int w = lane * per + i;
      if (w < b.n) local += (int)__ldcg(&world_ptr(b, w)->ctr->pop);
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += v;
    }
    int run = incl - local;
    for (int i = 0; i < per; ++i) {
      const int w = lane * per + i;
      if (w < b.n) {
        sm.prefix[w] = run;
        run += (int)__ldcg(&world_ptr(b, w)->ctr->pop);
      }
    }
    if (lane == 31) sm.prefix[b.n] = incl;
  }
  __syncthreads();

  const long long A = sm.prefix[b.n];
  const int n_agents = A > blockIdx.x ? (int)((A - blockIdx.x + G - 1) / G) : 0;
  int *status = &world_ptr(b, 0)->ctr->status;

  if (warp == W_PROD) {
    // ------------------------------------------------ producer -------------
    // Slots of 32 agents at a time, one lane per agent (the first 32 were
    // requested at the start with one world); lane 0 issues the copies.
    int issued = 0;
    bool waited = false, abort = false;
    AgentRef mine = pre;
    for (int n = 0; n < n_agents && !abort; ++n) {
      if ((n & 31) == 0) {
        const long long a = blockIdx.x + (long long)(n + lane) * G;
        if (n > 0 || b.n > 1) mine = agent_ref(sm.prefix, b, a, A);
        mine = agent_valid(b, mine, a, A);
      }
      const int slot = __shfl_sync(FULL, mine.slot, n & 31);
      const int fresh = __shfl_sync(FULL, mine.fresh, n & 31);
      const int world = __shfl_sync(FULL, mine.world, n & 31);
      if (!waited && fresh) {
        pdl_wait();   // a newborn's weights are written by the tail kernel
        waited = true;
      }
      if (lane == 0) {
        const float *wts = world_ptr(b, world)->weights + (size_t)slot * WSTRIDE;
        for (int q = 0; q < NBLK; ++q) {
          const int u = NBLK * n + q, st = u % LSTAGES, k = u / LSTAGES;
          if (k > 0 && !mbar_wait(&sm.empty[st], (k - 1) & 1)) {
            atomicOr(status, ST_TIMEOUT);
            sm.abort_flag = 1;
            break;
          }
          const uint32_t bytes = (q == NBLK - 1) ? STAGE_FLOATS * 4 : BLK_BYTES;
          mbar_expect_tx(&sm.full[st], bytes);
          bulk_copy_g2s(sm.stage[st], wts + q * BLK_FLOATS, bytes, &sm.full[st]);
          issued = u + 1;
        }
      }
      __syncwarp();
      abort = sm.abort_flag != 0;
    }
    if (lane == 0) sm.issued = issued;
  } else if (warp >= NCOMP) {
    // ------------------------------------------------ gather ---------------
    // Gather warp gw takes the CTA's agents gw, gw + NGATH, ...: their slots,
    // then positions, energies and forced actions, 32 agents at a time (one
    // lane per agent); then per agent the window's loads (one round trip),
    // issued before the warp waits for its ring entry.
    const int gw = warp - NCOMP;
    bool waited = false;
    AgentRef ref = pre;
    AgentDesc mine{};
    for (int m = 0;; ++m) {
      const int n = gw + NGATH * m;
      if (n >= n_agents) break;
      if ((m & 31) == 0) {
        const long long a = blockIdx.x + (long long)(gw + NGATH * (m + lane)) * G;
        if (m > 0 || b.n > 1) ref = agent_ref(sm.prefix, b, a, A);
        ref = agent_valid(b, ref, a, A);
        const WorldDev &wd = *world_ptr(b, ref.world);
        mine.slot = ref.slot;
        mine.world = ref.world;
        mine.y = __ldcg(&wd.y[ref.slot]);
        mine.x = __ldcg(&wd.x[ref.slot]);
        mine.energy = __ldcg(&wd.energy[ref.slot]);
        const int forced = __ldcg(&wd.forced[ref.slot]);
        mine.forced = __ldcg(&wd.ctr->use_forced) ? forced : -1;
        mine.t = (uint32_t)__ldcg(&wd.ctr->t);
      }
      const int src = m & 31;
      AgentDesc d;
      d.slot = __shfl_sync(FULL, mine.slot, src);
      d.world = __shfl_sync(FULL, mine.world, src);
      d.y = __shfl_sync(FULL, mine.y, src);
      d.x = __shfl_sync(FULL, mine.x, src);
      d.energy = __shfl_sync(FULL, mine.energy, src);
      d.forced = __shfl_sync(FULL, mine.forced, src);
      d.t = __shfl_sync(FULL, mine.t, src);
      if (!waited) {
        pdl_wait();   // the resource plane of this step is the tail kernel's
        waited = true;
      }
      const WorldDev &wd = *world_ptr(b, d.world);
      const GatherRegs g = gather_load(wd, d, lane);
      const int ei = n % VRING, k = n / VRING;
      bool ok = true;
      if (lane == 0 && k > 0) ok = mbar_wait(&sm.vempty[ei], (k - 1) & 1);
      if (!__shfl_sync(FULL, ok ? 1 : 0, 0)) {
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
        sm.abort_flag = 1;
        break;
      }
      gather_store(wd, d, g, sm.ring[ei], sm.masks[gw], lane);
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.vfull[ei]);
      if (sm.abort_flag) break;
    }
  } else {
    // ------------------------------------------------ compute --------------
    const int q = warp;
    MoveClaim pending;  // warp 3, lane 0: the previous agent's move claim
    for (int n = 0; n < n_agents; ++n) {
      if (sm.abort_flag) break;
      const int ei = n % VRING, kv = n / VRING;
      const int u = NBLK * n + q, st = u % LSTAGES, ks = u / LSTAGES;
      if (!mbar_wait(&sm.vfull[ei], kv & 1)) {
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
        sm.abort_flag = 1;
        break;
      }
      VEntry &E = sm.ring[ei];
      if (!mbar_wait(&sm.full[st], ks & 1)) {
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
        sm.abort_flag = 1;
        break;
      }
      const float *stg = sm.stage[st];
      // gate row `lane` of block q: z = W_row . [obs; h] + b_row
      const float4 *W4 = reinterpret_cast<const float4 *>(stg + lane * NIN);
      const float4 *V4 = reinterpret_cast<const float4 *>(E.v);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 9
      for (int k = 0; k < NIN / 4; ++k) {
        const float4 wv = W4[k], xv = V4[k];
        a0 = fmaf(wv.x, xv.x, a0);
        a1 = fmaf(wv.y, xv.y, a1);
        a2 = fmaf(wv.z, xv.z, a2);
        a3 = fmaf(wv.w, xv.w, a3);
      }
      const float z = ((a0 + a1) + (a2 + a3)) + stg[BLK_ROWS * NIN + lane];
      if (q < NCOMP - 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&sm.empty[st]);
      }
      // gate (lane % 4): 0 input, 1 forget, 2 candidate (tanh), 3 output
      const int g = lane & 3;
      const float act = (g == 2) ? tanhf(z) : 1.0f / (1.0f + expf(-z));
      const int base = lane & ~3;
      const float gi = __shfl_sync(FULL, act, base);
      const float gf = __shfl_sync(FULL, act, base + 1);
      const float gg = __shfl_sync(FULL, act, base + 2);
      const float go = __shfl_sync(FULL, act, base + 3);
      if (g == 0) {
        const int j = 8 * q + (lane >> 2);
        const float cn = gf * E.c[j] + gi * gg;
        const float hn = go * tanhf(cn);
        E.hn[j] = hn;
        E.c_row[j] = cn;
        E.h_row[j] = hn;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.hready[ei]);
      if (q == NCOMP - 1) {
        // read-out: logits = Wo h' + bo over the whole hidden state
        if (!mbar_wait(&sm.hready[ei], kv & 1)) {
          if (lane == 0) atomicOr(status, ST_TIMEOUT);
          sm.abort_flag = 1;
          break;
        }
        const float hj = E.hn[lane];
        const float *tail = stg + BLK_FLOATS;
        float lg[NACT];
#pragma unroll
        for (int a = 0; a < NACT; ++a) {
          float p = tail[a * HID + lane] * hj;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(FULL, p, o);
          lg[a] = p + tail[NACT * HID + a];
        }
        int best = 0;
        float mine = lg[0];
#pragma unroll
        for (int a = 1; a < NACT; ++a) {
          if (lg[a] > lg[best]) best = a;
          if (lane == a) mine = lg[a];
        }
        if (lane < NACT) E.logits_row[lane] = mine;
        if (lane == 0) {
          *E.action = best;
          const int moved = E.forced >= 0 ? E.forced : best;
          E.wd->prev_act[E.slot] = (moved >= 0 && moved < NACT) ? moved : 0;
          pending.resolve();
          pending.issue(*E.wd, E.slot, E.y, E.x, moved);
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&sm.empty[st]);
          mbar_arrive(&sm.vempty[ei]);
        }
      }
    }
    if (q == NCOMP - 1 && lane == 0) pending.resolve();
  }

  // Drain: wait (bounded) for every copy this CTA issued, so that no bulk
  // copy into shared memory is still in flight when the CTA exits.  A CTA
  // that had no agent has not waited for the tail kernel yet: it does so
  // here, so that this kernel never completes before the tail (the next
  // kernel waits on this one).
  __syncthreads();
  pdl_wait();
  if (threadIdx.x == 0) {
    const int issued = sm.issued;
    for (int st = 0; st < LSTAGES && st < issued; ++st) {
      const int last = st + ((issued - 1 - st) / LSTAGES) * LSTAGES;
      if (!mbar_wait(&sm.full[st], (last / LSTAGES) & 1)) atomicOr(status, ST_TIMEOUT);
    }
  }
}

// Exercises the bounded wait on a barrier whose phase never completes (two
// arrivals expected, one made): the wait gives up after limit_ns and sets
// ST_TIMEOUT, exactly as a stalled pipeline stage would.
__global__ void k_wait_selftest(int *status, unsigned long long limit_ns) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 2);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive(&bar);
    if (!mbar_wait(&bar, 0, limit_ns)) atomicOr(status, ST_TIMEOUT);
  }
}

void launch_wait_selftest(int *status, unsigned long long limit_ns, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(status, limit_ns);
}

// Two shapes: one CTA per SM with an 8-block ring (~199 KB of shared
// memory), or two CTAs per SM with a 4-block ring each (~108 KB).
static_assert(2 * (sizeof(LstmSmem<4>) + 1024) <= 228 * 1024, "two 4-stage CTAs fit an SM");

void configure_lstm() {
  cudaFuncSetAttribute(k_lstm<8, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(LstmSmem<8>));
  cudaFuncSetAttribute(k_lstm<4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(LstmSmem<4>));
}

void preload_lstm() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_lstm<8, 1>);
  cudaFuncGetAttributes(&a, k_lstm<4, 2>);
}

void launch_lstm(const BatchDev &b, cudaStream_t s) {
  if (b.lstm_ctas == 2)
    launch_step_kernel(k_lstm<4, 2>, 2 * b.n_sms, LTHREADS, sizeof(LstmSmem<4>), s, b);
  else
    launch_step_kernel(k_lstm<8, 1>, b.n_sms, LTHREADS, sizeof(LstmSmem<8>), s, b);
}

}  // namespace eco
