// k_lstm.cu -- step parts a2 + a3: observation gather and one LSTM step per
// agent (App. B.2, sensorimotor ability and cognitive capacity).
//
// Every agent has its own 93 KB of FP32 weights, used once per step, so the
// step is a batched GEMV bound by HBM bandwidth (about 0.5 flop per byte).
// Design:
//   * unit of work = one weight block of one agent (32 gate rows = all four
//     gates of 8 hidden units, 23,168 bytes); an agent is 4 units;
//   * a persistent grid of one CTA per SM; CTA b owns a contiguous range of
//     the units of all worlds of the batch (world-major, alive list order);
//   * a producer lane streams the blocks with plain (non-multicast)
//     cp.async.bulk copies into an 8-stage shared-memory ring guarded by
//     mbarriers, so about 180 KB per SM are in flight;
//   * four consumer warps take the units round-robin: each gathers the
//     agent's 7x7x3 observation (bit planes staged through shared memory)
//     and previous hidden state into a 180-float input vector while the
//     copy is in flight, then each lane computes one gate row with 128-bit
//     shared loads (conflict-free: rows are 720 B apart), applies the gate
//     nonlinearity, and lanes 0, 4, .., 28 update the cell state of their
//     hidden unit;
//   * the last of an agent's four units to finish (atomic arrival counter)
//     computes the 5 logits from the new hidden state and takes the argmax.
// Every mbarrier wait is bounded; a wait that runs out sets ST_TIMEOUT, the
// CTA stops issuing copies, waits (bounded) for the copies in flight and
// returns.
#include "ecoevo_dev.cuh"

namespace eco {

constexpr int LSTAGES = 8;
constexpr int NCONS = 4;
constexpr int LTHREADS = (NCONS + 1) * 32;
constexpr int MAX_BATCH = 1024;
constexpr int VLEN = 184;  // 180 inputs padded to a 16-byte multiple
constexpr unsigned long long WAIT_NS = 2000000000ull;  // 2 s

struct __align__(128) LstmSmem {
  float stage[LSTAGES][BLK_FLOATS];
  float v[NCONS][VLEN];
  uint32_t masks[NCONS][16];
  unsigned long long full[LSTAGES];
  unsigned long long empty[LSTAGES];
  int prefix[MAX_BATCH + 1];
  int issued;
  volatile int abort_flag;
};

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
__device__ inline bool mbar_wait(unsigned long long *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > WAIT_NS) return false;
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

// Input vector [obs(148); h(32)] of `slot` into v, by one warp.  The grid is
// the resource plane after this step's regrowth, the agent channel is the
// start-of-step occupancy without the agent itself, off-grid cells read as
// wall, the last observation is the agent's energy.
__device__ inline void gather_input(const WorldDev &wd, int slot,
                                    const uint32_t *res, const float *h_prev,
                                    float *v, uint32_t *masks, int lane) {
  const int H = wd.H, W = wd.W, Wp = wd.Wp;
  const int y = wd.y[slot], x = wd.x[slot];
  if (lane < 14) {
    const bool is_wall = lane >= 7;
    const int yy = y - 3 + (is_wall ? lane - 7 : lane);
    uint32_t m;
    if (yy < 0 || yy >= H)
      m = is_wall ? 0x7Fu : 0u;
    else
      m = row7((is_wall ? wd.wall : res) + (size_t)yy * Wp, Wp, W, x - 3, is_wall);
    masks[lane] = m;
  }
  for (int k = lane; k < 49; k += 32) {
    const int yy = y + k / 7 - 3, xx = x + k % 7 - 3;
    float a = 0.f;
    if (k != 24 && yy >= 0 && yy < H && xx >= 0 && xx < W)
      a = wd.slot_map[(size_t)yy * W + xx] >= 0 ? 1.f : 0.f;
    v[49 + k] = a;
  }
  if (lane == 0) v[147] = wd.energy[slot];
  v[NOBS + lane] = h_prev[(size_t)slot * HID + lane];
  __syncwarp();
  for (int k = lane; k < 49; k += 32) {
    const int r = k / 7, cc = k % 7;
    v[k] = (float)((masks[r] >> cc) & 1u);
    v[98 + k] = (float)((masks[7 + r] >> cc) & 1u);
  }
  __syncwarp();
}

__device__ inline void advance_world(const int *prefix, int &w, int u) {
  while (u >= prefix[w + 1]) ++w;
}

__global__ void __launch_bounds__(LTHREADS, 1) k_lstm(BatchDev b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  LstmSmem &sm = *reinterpret_cast<LstmSmem *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // units per world: 4 * population (= alive-list length at step start)
  if (warp == 0) {
    const int per = (b.n + 31) / 32;
    int local = 0;
    for (int i = 0; i < per; ++i) {
      const int w = lane * per + i;
      if (w < b.n) local += NBLK * (int)b.worlds[w]->ctr->pop;
    }
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= o) incl += t;
    }
    int run = incl - local;
    for (int i = 0; i < per; ++i) {
      const int w = lane * per + i;
      if (w < b.n) {
        sm.prefix[w] = run;
        run += NBLK * (int)b.worlds[w]->ctr->pop;
      }
    }
    if (lane == 31) sm.prefix[b.n] = incl;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < LSTAGES; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    sm.issued = 0;
    sm.abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const long long U = sm.prefix[b.n];
  const int u_begin = (int)(U * blockIdx.x / gridDim.x);
  const int u_end = (int)(U * (blockIdx.x + 1) / gridDim.x);
  int *status = &b.worlds[0]->ctr->status;

  if (warp == NCONS) {
    // ---------------- producer: one lane issues the bulk copies ----------
    if (lane == 0 && u_begin < u_end) {
      int w = 0;
      advance_world(sm.prefix, w, u_begin);
      int n = 0;
      for (int u = u_begin; u < u_end; ++u, ++n) {
        advance_world(sm.prefix, w, u);
        const WorldDev &wd = *b.worlds[w];
        const int lu = u - sm.prefix[w];
        const int slot = wd.alive_list[lu >> 2];
        const int st = n % LSTAGES;
        if (n >= LSTAGES && !mbar_wait(&sm.empty[st], ((n / LSTAGES) - 1) & 1)) {
          atomicOr(status, ST_TIMEOUT);
          sm.abort_flag = 1;
          break;
        }
        if (sm.abort_flag) break;
        const float *src = wd.weights + (size_t)slot * WSTRIDE + (lu & 3) * BLK_FLOATS;
        mbar_expect_tx(&sm.full[st], BLK_BYTES);
        bulk_copy_g2s(sm.stage[st], src, BLK_BYTES, &sm.full[st]);
        sm.issued = n + 1;
      }
    }
  } else {
    // ---------------- consumers ------------------------------------------
    float *v = sm.v[warp];
    uint32_t *masks = sm.masks[warp];
    int w = 0;
    if (u_begin < u_end) advance_world(sm.prefix, w, u_begin);
    for (int n = warp; u_begin + n < u_end; n += NCONS) {
      if (sm.abort_flag) break;
      const int u = u_begin + n;
      advance_world(sm.prefix, w, u);
      const WorldDev &wd = *b.worlds[w];
      const int lu = u - sm.prefix[w];
      const int slot = wd.alive_list[lu >> 2];
      const int q = lu & 3;
      const uint32_t t = (uint32_t)wd.ctr->t;
      const uint32_t *res_new = (t & 1u) ? wd.res0 : wd.res1;
      const float *h_prev = (t & 1u) ? wd.h1 : wd.h0;
      float *h_next = (t & 1u) ? wd.h0 : wd.h1;

      gather_input(wd, slot, res_new, h_prev, v, masks, lane);

      const int st = n % LSTAGES;
      if (!mbar_wait(&sm.full[st], (n / LSTAGES) & 1)) {
        if (lane == 0) atomicOr(status, ST_TIMEOUT);
        sm.abort_flag = 1;
        break;
      }
      // gate row `lane` of block q: z = W_row . [obs; h] + b_row
      const float4 *W4 = reinterpret_cast<const float4 *>(sm.stage[st] + lane * NIN);
      const float4 *V4 = reinterpret_cast<const float4 *>(v);
      float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll 9
      for (int k = 0; k < NIN / 4; ++k) {
        const float4 wv = W4[k], xv = V4[k];
        a0 = fmaf(wv.x, xv.x, a0);
        a1 = fmaf(wv.y, xv.y, a1);
        a2 = fmaf(wv.z, xv.z, a2);
        a3 = fmaf(wv.w, xv.w, a3);
      }
      const float z = ((a0 + a1) + (a2 + a3)) + sm.stage[st][BLK_ROWS * NIN + lane];
      __syncwarp();
      if (lane == 0) mbar_arrive(&sm.empty[st]);

      // gate (lane % 4): 0 input, 1 forget, 2 candidate (tanh), 3 output
      const int g = lane & 3;
      const float act = (g == 2) ? tanhf(z) : 1.0f / (1.0f + expf(-z));
      const int base = lane & ~3;
      const float gi = __shfl_sync(0xFFFFFFFFu, act, base);
      const float gf = __shfl_sync(0xFFFFFFFFu, act, base + 1);
      const float gg = __shfl_sync(0xFFFFFFFFu, act, base + 2);
      const float go = __shfl_sync(0xFFFFFFFFu, act, base + 3);
      if (g == 0) {
        const size_t j = (size_t)slot * HID + 8 * q + (lane >> 2);
        const float cn = gf * wd.c[j] + gi * gg;
        wd.c[j] = cn;
        h_next[j] = go * tanhf(cn);
      }
      __threadfence();
      __syncwarp();
      unsigned old = 0;
      if (lane == 0) old = atomicAdd(&wd.arrive[slot], 1u);
      old = __shfl_sync(0xFFFFFFFFu, old, 0);
      if (old == NBLK - 1) {
        // last block of the agent: read-out and argmax (first maximum)
        __threadfence();
        const float hj = __ldcg(&h_next[(size_t)slot * HID + lane]);
        const float *tail = wd.weights + (size_t)slot * WSTRIDE + TAIL;
        float lg[NACT];
#pragma unroll
        for (int a = 0; a < NACT; ++a) {
          float p = tail[a * HID + lane] * hj;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
          lg[a] = p + tail[NACT * HID + a];
        }
        int best = 0;
#pragma unroll
        for (int a = 1; a < NACT; ++a)
          if (lg[a] > lg[best]) best = a;
        float mine = lg[0];
#pragma unroll
        for (int a = 1; a < NACT; ++a)
          if (lane == a) mine = lg[a];
        if (lane < NACT) wd.logits[(size_t)slot * 8 + lane] = mine;
        if (lane == 0) {
          wd.action[slot] = best;
          wd.arrive[slot] = 0u;
        }
      }
    }
  }

  // Drain: wait (bounded) for every copy this CTA issued, so that no bulk
  // copy into shared memory is still in flight when the CTA exits.
  __syncthreads();
  if (threadIdx.x == 0) {
    const int issued = sm.issued;
    for (int st = 0; st < LSTAGES && st < issued; ++st) {
      const int last = st + ((issued - 1 - st) / LSTAGES) * LSTAGES;
      if (!mbar_wait(&sm.full[st], (last / LSTAGES) & 1)) atomicOr(status, ST_TIMEOUT);
    }
  }
}

void configure_lstm() {
  cudaFuncSetAttribute(k_lstm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(LstmSmem));
}

void preload_lstm() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_lstm);
}

void launch_lstm(const BatchDev &b, cudaStream_t s) {
  k_lstm<<<b.n_sms, LTHREADS, sizeof(LstmSmem), s>>>(b);
}

}  // namespace eco
