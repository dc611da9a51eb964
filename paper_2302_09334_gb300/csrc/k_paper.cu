// k_paper.cu -- observation, controller and move claim of the paper's own
// agent (App. B.5) for worlds with controller ECO_CTRL_PAPER.  One CTA of
// 128 threads per agent (grid-stride over the batch's agents in
// world-major alive-list order), so that an agent's work is spread wide
// (the paper's few hundred agents make this kernel latency-bound):
//   * the agent's 2445 parameters (9,792 B row) are copied to shared memory
//     with 16-byte cp.async while the threads build the 15x15x3
//     view (resource plane after this step's regrowth, start-of-step
//     occupancy without the agent itself, off-grid cells read as wall);
//   * conv 3x3 stride 2 with one cell of zero padding (15 -> 8, 4 maps),
//     2x2 average pool stride 1 (-> 7), conv 3x3 stride 2 (-> 4, 8 maps),
//     pool (-> 3): 72 features in [y][x][map] order, then the previous
//     action one-hot and the ate-last-step bit (78 inputs);
//   * LSTM with 4 units (eight threads per gate row), dense 8 + tanh on
//     [embedding, h'] (sixteen threads per row), dense 5;
//   * softmax at temperature 1/50 and the sampled action: the number of
//     k < 4 whose cumulative probability is <= u, u = (w0 >> 8) 2^-24 of
//     the Philox block {slot, t, TAG_ACT, 0};
//   * the move claim with the action moved with (forced or own), which is
//     also the next step's previous-action input.
// The parameters are used once per step (about 2.8 flop per byte), so the
// kernel is bound by HBM for large populations and by latency for the
// paper's thousand agents; tensor cores would not help.
#include "ecoevo_dev.cuh"
#include "move_claim.cuh"

namespace eco {

constexpr int PC_THREADS = 128;        // one CTA per agent
constexpr int PC_CTAS_PER_SM = 8;

struct __align__(16) PcSmem {
  float w[PC_WSTRIDE];                   // the agent's parameters
  float obs[PC_VIEW * PC_VIEW * 3 + 1];  // [y][x][channel]
  float a1[8 * 8 * 4];                   // conv1
  float p1[7 * 7 * 4];                   // pool1
  float a2[4 * 4 * 8];                   // conv2
  float emb[PC_EMB + PC_HID + 2];        // pool2 (72), one-hot (5), ate (1), h' (4)
  float hc[2 * PC_HID];                  // h and c before the step
  float z[4 * PC_HID];                   // LSTM gate pre-activations
  float d[8];                            // dense 1 after tanh
  int prefix[1025];                      // agents before world w of the batch
  int first_slot, first_new;              // one world: this CTA's first agent and its
                                         // newborn flag
};

__device__ inline void cp_async16(void *smem, const void *gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ inline void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

__device__ inline float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

// 3x3 convolution, stride 2, one cell of zero padding: in [n][n][CI],
// out [m][m][CO], weights [CO][3][3][CI]; output o = (oy*m + ox)*CO + f.
template <int CI, int CO>
__device__ inline void conv3x3_s2(const float *in, int n, const float *wt, const float *bias,
                                  float *out, int m, int tid) {
  for (int o = tid; o < m * m * CO; o += PC_THREADS) {
    const int f = o % CO, pos = o / CO, oy = pos / m, ox = pos % m;
    float acc = bias[f];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const int iy = 2 * oy + ky - 1;
      if (iy < 0 || iy >= n) continue;
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        const int ix = 2 * ox + kx - 1;
        if (ix < 0 || ix >= n) continue;
        const float *wv = wt + ((f * 3 + ky) * 3 + kx) * CI;
        const float *iv = in + (iy * n + ix) * CI;
#pragma unroll
        for (int c = 0; c < CI; ++c) acc = fmaf(wv[c], iv[c], acc);
      }
    }
    out[o] = acc;
  }
}

// 2x2 average pool, stride 1: [n][n][C] -> [n-1][n-1][C].
template <int C>
__device__ inline void avgpool2(const float *in, int n, float *out, int tid) {
  const int m = n - 1;
  for (int o = tid; o < m * m * C; o += PC_THREADS) {
    const int c = o % C, pos = o / C, y = pos / m, x = pos % m;
    const float s = ((in[(y * n + x) * C + c] + in[(y * n + x + 1) * C + c]) +
                     in[((y + 1) * n + x) * C + c]) + in[((y + 1) * n + x + 1) * C + c];
    out[o] = 0.25f * s;
  }
}

__global__ void __launch_bounds__(PC_THREADS, PC_CTAS_PER_SM)
    k_paper(const __grid_constant__ BatchDev b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PcSmem &S = *reinterpret_cast<PcSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const unsigned FULL = 0xFFFFFFFFu;
  // As in the LSTM kernel: the slot phases have completed when this kernel
  // starts (the tail kernel before it waits for them before releasing it),
  // so populations, alive lists, positions, ages and the parameters of the
  // agents not born in the last step are read (through L2) before waiting
  // for the tail; the resource plane and newborns' parameters after.
  pdl_release();

  // agents per world (= alive-list length at the start of the step); with
  // one world, the population and this CTA's first slot are loaded together
  if (warp == 0 && b.n == 1) {
    if (lane == 0) {
      const WorldDev &w0 = *world_ptr(b, 0);
      const int pop = (int)__ldcg(&w0.ctr->pop);
      const int first = (int)blockIdx.x < w0.C ? __ldcg(&w0.alive_list[blockIdx.x]) : 0;
      const int first_new = (int)blockIdx.x < w0.C ? __ldcg(&w0.alive_new[blockIdx.x]) : 1;
      S.prefix[0] = 0;
      S.prefix[1] = pop;
      S.first_slot = first;
      S.first_new = first_new;
    }
  } else if (warp == 0) {
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
        S.prefix[w] = run;
        run += (int)__ldcg(&world_ptr(b, w)->ctr->pop);
      }
    }
    if (lane == 31) S.prefix[b.n] = incl;
  }
  __syncthreads();

  const int A = S.prefix[b.n];
  for (int a = blockIdx.x; a < A; a += gridDim.x) {
    const int wi = world_of(S.prefix, b.n, a);
    const WorldDev &wd = *world_ptr(b, wi);
    const bool first = b.n == 1 && a == (int)blockIdx.x;
    const int s = checked_index(
        wd, first ? S.first_slot : __ldcg(&wd.alive_list[a - S.prefix[wi]]), wd.C);
    const int fresh = first ? S.first_new : __ldcg(&wd.alive_new[a - S.prefix[wi]]);
    const uint32_t t = (uint32_t)__ldcg(&wd.ctr->t);
    const int y = __ldcg(&wd.y[s]), x = __ldcg(&wd.x[s]);
    // a newborn's parameters are written by the tail kernel
    if (fresh) pdl_wait();

    // parameters -> shared memory, asynchronously
    const float4 *src = reinterpret_cast<const float4 *>(wd.weights + (size_t)s * PC_WSTRIDE);
    float4 *dst = reinterpret_cast<float4 *>(S.w);
    for (int i = tid; i < PC_WSTRIDE / 4; i += PC_THREADS) cp_async16(dst + i, src + i);
    pdl_wait();   // the resource plane of this step is the tail kernel's

    // the 15x15x3 view: each thread loads its (up to 2) cells, then stores
    const uint32_t *res = (t & 1u) ? wd.res0 : wd.res1;
    const int half = PC_VIEW / 2;
    constexpr int CELLS = PC_VIEW * PC_VIEW;
    constexpr int PER = (CELLS + PC_THREADS - 1) / PC_THREADS;
    uint32_t rw[PER], ww[PER];
    int occ[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = tid + PC_THREADS * i;
      const int yy = y + k / PC_VIEW - half, xx = x + k % PC_VIEW - half;
      rw[i] = 0u;
      ww[i] = 1u;   // off the grid: wall
      occ[i] = -1;
      if (k < CELLS && yy >= 0 && yy < wd.H && xx >= 0 && xx < wd.W) {
        rw[i] = res[yy * wd.Wp + (xx >> 5)] >> (xx & 31);
        ww[i] = wd.wall[yy * wd.Wp + (xx >> 5)] >> (xx & 31);
        occ[i] = (k != half * PC_VIEW + half) ? wd.slot_map[yy * wd.W + xx] : -1;
      }
    }
    int res_seen = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int k = tid + PC_THREADS * i;
      if (k < CELLS) {
        S.obs[3 * k] = (float)(rw[i] & 1u);
        S.obs[3 * k + 1] = occ[i] >= 0 ? 1.f : 0.f;
        S.obs[3 * k + 2] = (float)(ww[i] & 1u);
        res_seen |= (int)(rw[i] & 1u);
      }
    }
    const int prev = wd.prev_act[s];
    const int ate = wd.ate[s];
    const float *h_prev = ((t & 1u) ? wd.h1 : wd.h0) + (size_t)s * HID;
    float *h_next = ((t & 1u) ? wd.h0 : wd.h1) + (size_t)s * HID;
    if (tid < PC_HID) {
      S.hc[tid] = h_prev[tid];
      S.hc[PC_HID + tid] = wd.c[(size_t)s * HID + tid];
    }
    cp_async_wait_all();
    // greediness window: a resource in view (the barrier also publishes
    // the view, the parameters and h, c)
    if (__syncthreads_or(res_seen) && tid == 0) wd.lab_seen[s] = 1;

    // embedding
    conv3x3_s2<3, 4>(S.obs, PC_VIEW, S.w + PC_OFF_W1, S.w + PC_OFF_B1, S.a1, 8, tid);
    __syncthreads();
    avgpool2<4>(S.a1, 8, S.p1, tid);
    __syncthreads();
    conv3x3_s2<4, 8>(S.p1, 7, S.w + PC_OFF_W2, S.w + PC_OFF_B2, S.a2, 4, tid);
    __syncthreads();
    avgpool2<8>(S.a2, 4, S.emb, tid);
    if (tid >= 72 && tid < 72 + NACT) S.emb[tid] = (tid - 72 == prev) ? 1.f : 0.f;
    if (tid == 77) S.emb[77] = ate ? 1.f : 0.f;
    __syncthreads();

    // LSTM gate rows: row r = tid / 8, eight threads per row
    {
      const int r = tid >> 3, q = tid & 7;
      const float *wi_row = S.w + PC_OFF_WI + r * PC_EMB;
      float z = 0.f;
      for (int k = q; k < PC_EMB; k += 8) z = fmaf(wi_row[k], S.emb[k], z);
      if (q < PC_HID) z = fmaf(S.w[PC_OFF_WH + r * PC_HID + q], S.hc[q], z);
      z += __shfl_xor_sync(FULL, z, 1);
      z += __shfl_xor_sync(FULL, z, 2);
      z += __shfl_xor_sync(FULL, z, 4);
      if (q == 0) S.z[r] = z + S.w[PC_OFF_BL + r];
    }
    __syncthreads();
    // cell update of unit j (gates i, f, g, o)
    if (tid < PC_HID) {
      const float c_new =
          sigmoidf_(S.z[PC_HID + tid]) * S.hc[PC_HID + tid] +
          sigmoidf_(S.z[tid]) * tanhf(S.z[2 * PC_HID + tid]);
      const float h_new = sigmoidf_(S.z[3 * PC_HID + tid]) * tanhf(c_new);
      wd.c[(size_t)s * HID + tid] = c_new;
      h_next[tid] = h_new;
      S.emb[PC_EMB + tid] = h_new;
    }
    __syncthreads();

    // dense 8 + tanh on [embedding, h']: sixteen threads per row
    {
      const int i = tid >> 4, q = tid & 15;
      const float *row = S.w + PC_OFF_D1 + i * (PC_EMB + PC_HID);
      float acc = 0.f;
      for (int k = q; k < PC_EMB + PC_HID; k += 16) acc = fmaf(row[k], S.emb[k], acc);
      acc += __shfl_xor_sync(FULL, acc, 1);
      acc += __shfl_xor_sync(FULL, acc, 2);
      acc += __shfl_xor_sync(FULL, acc, 4);
      acc += __shfl_xor_sync(FULL, acc, 8);
      if (q == 0) S.d[i] = tanhf(acc + S.w[PC_OFF_DB1 + i]);
    }
    __syncthreads();

    if (warp == 0) {
      // dense 5
      float logit = 0.f;
      if (lane < NACT) {
        float acc = S.w[PC_OFF_DB2 + lane];
#pragma unroll
        for (int i = 0; i < 8; ++i) acc = fmaf(S.w[PC_OFF_D2 + lane * 8 + i], S.d[i], acc);
        logit = acc;
        wd.logits[(size_t)s * 8 + lane] = logit;
      }
      float lg[NACT];
#pragma unroll
      for (int k = 0; k < NACT; ++k) lg[k] = __shfl_sync(FULL, logit, k);
      if (lane == 0) {
        // softmax at temperature 1/50 and the sampled action
        float m = lg[0];
#pragma unroll
        for (int k = 1; k < NACT; ++k) m = fmaxf(m, lg[k]);
        float e[NACT], sum = 0.f;
#pragma unroll
        for (int k = 0; k < NACT; ++k) {
          e[k] = expf(50.f * (lg[k] - m));
          sum += e[k];
        }
        const U4 rnd = philox4x32_10(U4{(uint32_t)s, t, TAG_ACT, 0u}, wd.key0, wd.key1);
        const float u = (float)(rnd.x >> 8) * (1.f / 16777216.f);
        int act = 0;
        float cdf = 0.f;
#pragma unroll
        for (int k = 0; k < NACT - 1; ++k) {
          cdf += e[k] / sum;
          if (cdf <= u) act = k + 1;
        }
        wd.action[s] = act;
        const int moved = wd.ctr->use_forced ? wd.forced[s] : act;
        wd.prev_act[s] = (moved >= 0 && moved < NACT) ? moved : 0;
        // move claim (step part a4) from the view in shared memory: the
        // target's wall channel (walls and off-grid cells) and agent channel
        // (start-of-step occupancy) are the cell's state for the claim
        int tgt = -1, kill = 0;
        if (moved >= 1 && moved < NACT) {
          const int dy = moved == 1 ? -1 : moved == 2 ? 1 : 0;
          const int dx = moved == 3 ? 1 : moved == 4 ? -1 : 0;
          const int k = (half + dy) * PC_VIEW + (half + dx);
          if (S.obs[3 * k + 2] != 0.f) {
            kill = wd.wall_kills ? 1 : 0;
          } else if (S.obs[3 * k + 1] == 0.f) {
            tgt = (y + dy) * wd.W + (x + dx);
            atomicMin(&wd.claim[tgt], s);
          }
        }
        wd.target[s] = tgt;
        wd.killed[s] = kill;
      }
    }
    __syncthreads();   // the shared buffers are reused by the next agent
  }
  // a CTA without agents has not waited for the tail kernel: it does so
  // here, so that this kernel never completes before the tail (the next
  // kernel waits on this one)
  pdl_wait();
}

void preload_paper() {
  cudaFuncSetAttribute(k_paper, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(PcSmem));
  cudaFuncSetAttribute(k_paper, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
}

void launch_paper_ctrl(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_paper, PC_CTAS_PER_SM * b.n_sms, PC_THREADS, sizeof(PcSmem), s, b);
}

}  // namespace eco
