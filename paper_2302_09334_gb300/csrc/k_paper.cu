// k_paper.cu -- observation, controller and move claim of the paper's own
// agent (App. B.5) for worlds with controller ECO_CTRL_PAPER.  One warp per
// agent, agents of the batch in world-major alive-list order:
//   * the agent's 2445 parameters (9,792 B row) are copied to the warp's
//     shared memory with 16-byte cp.async while the lanes build the 15x15x3
//     view (resource plane after this step's regrowth, start-of-step
//     occupancy without the agent itself, off-grid cells read as wall);
//   * conv 3x3 stride 2 with one cell of zero padding (15 -> 8, 4 maps),
//     2x2 average pool stride 1 (-> 7), conv 3x3 stride 2 (-> 4, 8 maps),
//     pool (-> 3): 72 features in [y][x][map] order, then the previous
//     action one-hot and the ate-last-step bit (78 inputs);
//   * LSTM with 4 units (two lanes per gate row), dense 8 + tanh on
//     [embedding, h'], dense 5;
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

constexpr int PC_WARPS = 4;
constexpr int PC_THREADS = PC_WARPS * 32;
constexpr int PC_CTAS_PER_SM = 3;

struct __align__(16) PcWarp {
  float w[PC_WSTRIDE];                 // the agent's parameters
  float obs[PC_VIEW * PC_VIEW * 3 + 1];  // [y][x][channel]
  float a1[8 * 8 * 4];                 // conv1
  float p1[7 * 7 * 4];                 // pool1
  float a2[4 * 4 * 8];                 // conv2
  float emb[PC_EMB + PC_HID + 2];      // pool2 (72), one-hot (5), ate (1), h' (4)
  float d[8];                          // dense 1 after tanh
};

struct PcSmem {
  PcWarp warp[PC_WARPS];
  int prefix[1025];                    // agents before world w of the batch
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
                                  float *out, int m, int lane) {
  for (int o = lane; o < m * m * CO; o += 32) {
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
__device__ inline void avgpool2(const float *in, int n, float *out, int lane) {
  const int m = n - 1;
  for (int o = lane; o < m * m * C; o += 32) {
    const int c = o % C, pos = o / C, y = pos / m, x = pos % m;
    const float s = ((in[(y * n + x) * C + c] + in[(y * n + x + 1) * C + c]) +
                     in[((y + 1) * n + x) * C + c]) + in[((y + 1) * n + x + 1) * C + c];
    out[o] = 0.25f * s;
  }
}

__global__ void __launch_bounds__(PC_THREADS, PC_CTAS_PER_SM)
    k_paper(const __grid_constant__ BatchDev b) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  PcSmem &sm = *reinterpret_cast<PcSmem *>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned FULL = 0xFFFFFFFFu;
  pdl_wait_and_release();

  // agents per world (= alive-list length at the start of the step)
  if (warp == 0) {
    const int per = (b.n + 31) / 32;
    int local = 0;
    for (int i = 0; i < per; ++i) {
      const int w = lane * per + i;
      if (w < b.n) local += (int)world_ptr(b, w)->ctr->pop;
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
        run += (int)world_ptr(b, w)->ctr->pop;
      }
    }
    if (lane == 31) sm.prefix[b.n] = incl;
  }
  __syncthreads();

  PcWarp &S = sm.warp[warp];
  const int A = sm.prefix[b.n];
  for (int a = blockIdx.x * PC_WARPS + warp; a < A; a += gridDim.x * PC_WARPS) {
    const int wi = world_of(sm.prefix, b.n, a);
    const WorldDev &wd = *world_ptr(b, wi);
    const int s = checked_index(wd, wd.alive_list[a - sm.prefix[wi]], wd.C);
    const uint32_t t = (uint32_t)wd.ctr->t;
    const int y = wd.y[s], x = wd.x[s];

    // parameters -> shared memory, asynchronously
    const float4 *src = reinterpret_cast<const float4 *>(wd.weights + (size_t)s * PC_WSTRIDE);
    float4 *dst = reinterpret_cast<float4 *>(S.w);
    for (int i = lane; i < PC_WSTRIDE / 4; i += 32) cp_async16(dst + i, src + i);

    // the 15x15x3 view: every lane issues the loads of its (up to 8) cells
    // before it uses any of them
    const uint32_t *res = (t & 1u) ? wd.res0 : wd.res1;
    const int half = PC_VIEW / 2;
    constexpr int CELLS = PC_VIEW * PC_VIEW, PER_LANE = (CELLS + 31) / 32;
    uint32_t rw[PER_LANE], ww[PER_LANE];
    int occ[PER_LANE];
#pragma unroll
    for (int i = 0; i < PER_LANE; ++i) {
      const int k = lane + 32 * i;
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
    bool res_seen = false;
#pragma unroll
    for (int i = 0; i < PER_LANE; ++i) {
      const int k = lane + 32 * i;
      if (k < CELLS) {
        S.obs[3 * k] = (float)(rw[i] & 1u);
        S.obs[3 * k + 1] = occ[i] >= 0 ? 1.f : 0.f;
        S.obs[3 * k + 2] = (float)(ww[i] & 1u);
        res_seen |= (rw[i] & 1u) != 0u;
      }
    }
    // greediness window: a resource in view
    if (__any_sync(FULL, res_seen) && lane == 0) wd.lab_flags[s] |= 1u;
    const int prev = wd.prev_act[s];
    const int ate = wd.ate[s];
    const float *h_prev = ((t & 1u) ? wd.h1 : wd.h0) + (size_t)s * HID;
    float *h_next = ((t & 1u) ? wd.h0 : wd.h1) + (size_t)s * HID;
    const float h_old = lane < PC_HID ? h_prev[lane] : 0.f;
    const float c_old = lane < PC_HID ? wd.c[(size_t)s * HID + lane] : 0.f;
    cp_async_wait_all();
    __syncwarp();

    // embedding
    conv3x3_s2<3, 4>(S.obs, PC_VIEW, S.w + PC_OFF_W1, S.w + PC_OFF_B1, S.a1, 8, lane);
    __syncwarp();
    avgpool2<4>(S.a1, 8, S.p1, lane);
    __syncwarp();
    conv3x3_s2<4, 8>(S.p1, 7, S.w + PC_OFF_W2, S.w + PC_OFF_B2, S.a2, 4, lane);
    __syncwarp();
    avgpool2<8>(S.a2, 4, S.emb, lane);
    if (lane < NACT) S.emb[72 + lane] = (lane == prev) ? 1.f : 0.f;
    if (lane == NACT) S.emb[77] = ate ? 1.f : 0.f;
    __syncwarp();

    // LSTM gate rows: row r = lane % 16, inputs split between the two halves
    const int r = lane & 15, hf = lane >> 4;
    float z = 0.f;
    {
      const float *wi_row = S.w + PC_OFF_WI + r * PC_EMB;
      const int k0 = hf ? PC_EMB / 2 : 0, k1 = hf ? PC_EMB : PC_EMB / 2;
      for (int k = k0; k < k1; ++k) z = fmaf(wi_row[k], S.emb[k], z);
    }
#pragma unroll
    for (int j = 0; j < PC_HID; ++j) {
      const float hj = __shfl_sync(FULL, h_old, j);
      if (hf) z = fmaf(S.w[PC_OFF_WH + r * PC_HID + j], hj, z);
    }
    if (hf) z += S.w[PC_OFF_BL + r];
    z += __shfl_xor_sync(FULL, z, 16);
    // cell update of unit j = lane (lanes 0..3): gates i, f, g, o
    const int j = lane & 3;
    const float zi = __shfl_sync(FULL, z, j), zf = __shfl_sync(FULL, z, 4 + j);
    const float zg = __shfl_sync(FULL, z, 8 + j), zo = __shfl_sync(FULL, z, 12 + j);
    if (lane < PC_HID) {
      const float c_new = sigmoidf_(zf) * c_old + sigmoidf_(zi) * tanhf(zg);
      const float h_new = sigmoidf_(zo) * tanhf(c_new);
      wd.c[(size_t)s * HID + lane] = c_new;
      h_next[lane] = h_new;
      S.emb[PC_EMB + lane] = h_new;
    }
    __syncwarp();

    // dense 8 + tanh on [embedding, h']: four lanes per row
    {
      const int i = lane >> 2, q = lane & 3;
      const float *row = S.w + PC_OFF_D1 + i * (PC_EMB + PC_HID);
      float acc = 0.f;
      for (int k = q; k < PC_EMB + PC_HID; k += 4) acc = fmaf(row[k], S.emb[k], acc);
      acc += __shfl_xor_sync(FULL, acc, 1);
      acc += __shfl_xor_sync(FULL, acc, 2);
      if (q == 0) S.d[i] = tanhf(acc + S.w[PC_OFF_DB1 + i]);
    }
    __syncwarp();
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
      MoveClaim mc;
      mc.issue(wd, s, y, x, moved);
      mc.resolve();
    }
    __syncwarp();
  }
}

void preload_paper() {
  cudaFuncSetAttribute(k_paper, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(PcSmem));
}

void launch_paper_ctrl(const BatchDev &b, cudaStream_t s) {
  launch_step_kernel(k_paper, PC_CTAS_PER_SM * b.n_sms, PC_THREADS, sizeof(PcSmem), s, b);
}

}  // namespace eco
