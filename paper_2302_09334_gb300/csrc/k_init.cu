// k_init.cu -- world set-up and state rebuild (not part of the timed step).
//
// Initial state (App. B.4: walls on the border, resources and agents placed
// at random, weights drawn once at the start of the simulation):
//   walls       the outer ring of cells when border_walls
//   resources   cell (y, x) off the walls holds one iff word x%4 of the
//               Philox draw {x/4, 0, TAG_RES_INIT, y} is below
//               floor(res_init_p * 2^32)
//   agents      slots 0..n0-1 on the cells chosen by the host (ascending
//               order of the words of {x/4, 0, TAG_PLACE, y})
//   weights     w_init_std * N_j of the stream (TAG_INIT_W, 0, slot)
#include <climits>

#include "ecoevo_dev.cuh"

namespace eco {

void launch_init_weights(const WorldDev *wd_dev, int n0, int n_sms, cudaStream_t s);

__global__ void k_init_planes(WorldDev wd, int border, uint32_t thr_init) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= wd.H * wd.Wp) return;
  const int y = i / wd.Wp, ww = i % wd.Wp;
  uint32_t wall = 0, res = 0;
  for (int q = 0; q < 8; ++q) {
    const int xq = ww * 32 + q * 4;
    if (xq >= wd.W) break;
    const U4 u = philox4x32_10(U4{(uint32_t)xq >> 2, 0u, TAG_RES_INIT, (uint32_t)y},
                               wd.key0, wd.key1);
    const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
    for (int k = 0; k < 4; ++k) {
      const int x = xq + k;
      if (x >= wd.W) break;
      const bool is_wall = border && (y == 0 || y == wd.H - 1 || x == 0 || x == wd.W - 1);
      if (is_wall) wall |= 1u << (x & 31);
      else if (uw[k] < thr_init) res |= 1u << (x & 31);
    }
  }
  wd.wall[i] = wall;
  wd.res0[i] = res;
  wd.res1[i] = 0u;
}

__global__ void k_clear_cells(WorldDev wd) {
  const size_t n = (size_t)wd.H * wd.W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    wd.slot_map[i] = -1;
    wd.claim[i] = INT_MAX;
    wd.bclaim[i] = INT_MAX;
  }
}

// Fresh agents in slots [0, n0) at the given cells; every other slot empty.
__global__ void k_init_agents(WorldDev wd, int n0, const int32_t *py,
                              const int32_t *px) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= wd.C) return;
  const bool live = s < n0;
  wd.alive[s] = live ? 1 : 0;
  wd.y[s] = live ? py[s] : 0;
  wd.x[s] = live ? px[s] : 0;
  wd.energy[s] = live ? wd.e0 : 0.f;
  wd.repr_ctr[s] = 0;
  wd.low_ctr[s] = 0;
  wd.age[s] = 0;
  wd.action[s] = 0;
  wd.prev_act[s] = 0;
  wd.lab_seen[s] = 0;
  wd.lab_ate[s] = 0;
  wd.lab_t[s] = 0;
  wd.lab_c[s] = 0;
  wd.forced[s] = 0;
  wd.killed[s] = 0;
  wd.ate[s] = 0;
  wd.target[s] = -1;
  wd.birth_cell[s] = -1;
  wd.arrive[s] = 0u;
  for (int j = 0; j < HID; ++j) {
    wd.h0[(size_t)s * HID + j] = 0.f;
    wd.h1[(size_t)s * HID + j] = 0.f;
    wd.c[(size_t)s * HID + j] = 0.f;
  }
  for (int a = 0; a < 8; ++a) wd.logits[(size_t)s * 8 + a] = 0.f;
}

// Put every living agent on slot_map; a second agent on a cell, an agent on
// a wall or off the grid, a negative age, or a resource on a wall sets
// ST_STATE.
__global__ void k_place_agents(WorldDev wd) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < wd.C) {
    wd.arrive[s] = 0u;
    wd.birth_cell[s] = -1;
    wd.target[s] = -1;
    if (wd.alive[s]) {
      const int y = wd.y[s], x = wd.x[s];
      if (y < 0 || y >= wd.H || x < 0 || x >= wd.W || bit_at(wd.wall, wd.Wp, y, x) ||
          wd.age[s] < 0) {
        atomicOr(&wd.ctr->status, ST_STATE);
      } else if (atomicCAS(&wd.slot_map[y * wd.W + x], -1, s) != -1) {
        atomicOr(&wd.ctr->status, ST_STATE);
      }
    }
  }
  const int i = s;
  if (i < wd.H * wd.Wp) {
    const uint32_t t = (uint32_t)wd.ctr->t;
    const uint32_t *res = (t & 1u) ? wd.res1 : wd.res0;
    if (res[i] & wd.wall[i]) atomicOr(&wd.ctr->status, ST_STATE);
  }
}

// Alive list (ascending slots) and population, one CTA.
__global__ void __launch_bounds__(SCAN_THREADS) k_alive_list(WorldDev wd) {
  __shared__ int sh[33];
  const int C = wd.C;
  const int per = (C + SCAN_THREADS - 1) / SCAN_THREADS;
  const int s0 = min(C, (int)threadIdx.x * per), s1 = min(C, s0 + per);
  int n = 0;
  for (int s = s0; s < s1; ++s) n += wd.alive[s];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = n;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xFFFFFFFFu, inc, o);
    if (lane >= o) inc += v;
  }
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int k = 0; k < SCAN_THREADS / 32; ++k) {
      const int v = sh[k];
      sh[k] = run;
      run += v;
    }
    sh[32] = run;
  }
  __syncthreads();
  int off = sh[warp] + inc - n;
  for (int s = s0; s < s1; ++s)
    if (wd.alive[s]) {
      wd.alive_new[off] = wd.age[s] == 0 ? 1 : 0;   // never stepped: treated as newborn
      wd.alive_list[off++] = s;
    }
  if (threadIdx.x == 0) wd.ctr->pop = sh[32];
}

// Weight rows (`stride` floats apart) between the logical parameter order
// (the host's) and the physical order (the device's): the block permutation
// of the LSTM(32) controller, the identity for the paper's controller.
__device__ inline int logical_of(int controller, int p) {
  if (controller == ECO_CTRL_PAPER) return p < PC_NPARAM ? p : -1;
  return logical_of_phys(p);
}

// Weight rows from the physical order (rows of `stride` floats) to the
// logical order (rows of `lpitch` floats, the first nparam written).  The
// logical side may be page-locked host memory (its device address): writes
// along a physical row are consecutive logical parameters within each
// 180-weight gate row, so they coalesce.
__global__ void k_weights_to_logical(const float *physical, float *logical, size_t lpitch,
                                     int n, int controller, int stride) {
  const long long total = (long long)n * stride;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(g / stride), p = (int)(g % stride);
    const int j = logical_of(controller, p);
    if (j >= 0) logical[(size_t)a * lpitch + j] = physical[g];
  }
}

// Packed logical rows (n rows of nparam floats, back to back) in page-locked
// host memory, read through its device address as one flat array: 16-byte
// loads over the host link (the buffer is 16-byte aligned), the last 1..3
// floats one by one; each float is stored at its physical place in the
// device rows, and the holder of a row's last parameter zeroes the row's
// padding.
template <int CTRL>
__global__ void k_weights_from_host(const float *src, size_t total, float *rows) {
  constexpr int NP = CTRL == ECO_CTRL_PAPER ? PC_NPARAM : NPARAM;
  constexpr int STRIDE = CTRL == ECO_CTRL_PAPER ? PC_WSTRIDE : WSTRIDE;
  const size_t n_vec = (total + 3) / 4;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_vec;
       i += (size_t)gridDim.x * blockDim.x) {
    float f[4];
    if (4 * i + 4 <= total) {
      const float4 v = reinterpret_cast<const float4 *>(src)[i];
      f[0] = v.x; f[1] = v.y; f[2] = v.z; f[3] = v.w;
    } else {
      for (int c = 0; c < 4; ++c) f[c] = 4 * i + c < total ? src[4 * i + c] : 0.f;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const size_t g = 4 * i + c;
      if (g >= total) break;
      const int a = (int)(g / NP), j = (int)(g % NP);
      float *r = rows + (size_t)a * STRIDE;
      r[CTRL == ECO_CTRL_PAPER ? j : phys_of_logical(j)] = f[c];
      if (j == NP - 1)
        for (int q = NP; q < STRIDE; ++q) r[q] = 0.f;
    }
  }
}

// Rows already on the device in logical order (the first nparam floats of
// each `stride`-float row, copied there by DMA) permuted to the physical
// order in place: each CTA stages a whole row in shared memory.
__global__ void k_rows_to_physical_inplace(float *rows, int n, int controller, int stride,
                                           int nparam) {
  extern __shared__ float row[];
  for (int a = blockIdx.x; a < n; a += gridDim.x) {
    float *r = rows + (size_t)a * stride;
    for (int i = threadIdx.x; i < stride; i += blockDim.x) row[i] = i < nparam ? r[i] : 0.f;
    __syncthreads();
    for (int p = threadIdx.x; p < stride; p += blockDim.x) {
      const int j = logical_of(controller, p);
      r[p] = j >= 0 ? row[j] : 0.f;
    }
    __syncthreads();
  }
}

static int stride_of(int controller) {
  return controller == ECO_CTRL_PAPER ? PC_WSTRIDE : WSTRIDE;
}

int launch_rows_to_physical_inplace(float *rows, int n, int controller, int n_sms,
                                    cudaStream_t s) {
  if (n <= 0) return 0;
  const int stride = stride_of(controller);
  const size_t smem = (size_t)stride * sizeof(float);
  // a whole row of shared memory (the attribute is set on the current device)
  cudaError_t e = cudaFuncSetAttribute(k_rows_to_physical_inplace,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(WSTRIDE * sizeof(float)));
  if (e != cudaSuccess) return (int)e;
  const int nparam = controller == ECO_CTRL_PAPER ? PC_NPARAM : NPARAM;
  k_rows_to_physical_inplace<<<2 * n_sms, 512, smem, s>>>(rows, n, controller, stride, nparam);
  return (int)cudaGetLastError();
}

int launch_weights_from_host(const float *host_dev, float *rows, int n, int controller,
                             int n_sms, cudaStream_t s) {
  if (n <= 0) return 0;
  if (((uintptr_t)host_dev & 15u) != 0) return (int)cudaErrorMisalignedAddress;
  const size_t np = controller == ECO_CTRL_PAPER ? PC_NPARAM : NPARAM;
  const size_t total = (size_t)n * np;
  if (controller == ECO_CTRL_PAPER)
    k_weights_from_host<ECO_CTRL_PAPER><<<8 * n_sms, 256, 0, s>>>(host_dev, total, rows);
  else
    k_weights_from_host<ECO_CTRL_LSTM32><<<8 * n_sms, 256, 0, s>>>(host_dev, total, rows);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// State loads.
// ---------------------------------------------------------------------------
__global__ void k_load_counters(Counters *ctr, LoadCounters v) {
  if (v.set) {
    ctr->t = v.t;
    ctr->births = v.births;
    ctr->deaths = v.deaths;
    ctr->dropped = v.dropped;
    ctr->births_last = v.births_last;
    ctr->deaths_last = v.deaths_last;
    ctr->dropped_last = v.dropped_last;
    ctr->agent_steps = v.agent_steps;
  }
  ctr->deaths_step = 0;
  ctr->n_births = 0;
  ctr->use_forced = 0;
}

void launch_load_counters(Counters *ctr, const LoadCounters &v, cudaStream_t s) {
  k_load_counters<<<1, 1, 0, s>>>(ctr, v);
}

// One thread per word: bit b of word (y, w) is cell (y, 32 w + b).
__global__ void k_pack_plane(const uint8_t *cells, int H, int W, int Wp, uint32_t *words) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= H * Wp) return;
  const int y = i / Wp, x0 = (i % Wp) * 32;
  const uint8_t *row = cells + (size_t)y * W;
  uint32_t v = 0u;
  for (int b = 0; b < 32 && x0 + b < W; ++b)
    if (row[x0 + b]) v |= 1u << b;
  words[i] = v;
}

void launch_pack_plane(const uint8_t *cells, int H, int W, int Wp, uint32_t *words,
                       cudaStream_t s) {
  const int n = H * Wp;
  if (n > 0) k_pack_plane<<<(n + 255) / 256, 256, 0, s>>>(cells, H, W, Wp, words);
}

// Grid-stride over the C slots (scalars and logits) and over the C x HID
// elements of h and c.
__global__ void k_load_slots(WorldDev wd, SlotSources src, float *h_dst) {
  const int C = wd.C;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long i = i0; i < C; i += stride) {
    if (src.alive) wd.alive[i] = src.alive[i];
    if (src.ate) wd.ate[i] = src.ate[i];
    if (src.y) wd.y[i] = src.y[i];
    if (src.x) wd.x[i] = src.x[i];
    if (src.repr) wd.repr_ctr[i] = src.repr[i];
    if (src.low) wd.low_ctr[i] = src.low[i];
    if (src.age) wd.age[i] = src.age[i];
    if (src.action) wd.action[i] = src.action[i];
    if (src.prev) wd.prev_act[i] = src.prev[i];
    if (src.energy) wd.energy[i] = src.energy[i];
    if (src.logits)
      for (int a = 0; a < 8; ++a)
        wd.logits[i * 8 + a] = a < NACT ? src.logits[i * NACT + a] : 0.f;
  }
  const long long n = (long long)C * HID;
  for (long long i = i0; i < n; i += stride) {
    if (src.h) h_dst[i] = src.h[i];
    if (src.c) wd.c[i] = src.c[i];
  }
}

void launch_load_slots(const WorldDev &wd, const SlotSources &src, float *h_dst, int n_sms,
                       cudaStream_t s) {
  if (wd.C > 0) k_load_slots<<<4 * n_sms, 256, 0, s>>>(wd, src, h_dst);
}

void launch_weights_to_logical(const float *physical, float *logical, size_t lpitch, int n,
                               int controller, int n_sms, cudaStream_t s) {
  if (n > 0)
    k_weights_to_logical<<<8 * n_sms, 256, 0, s>>>(physical, logical, lpitch, n, controller,
                                                   stride_of(controller));
}

void launch_init_world(const WorldDev *wd_host, WorldDev *wd_dev, int n0,
                       const int32_t *place_y, const int32_t *place_x,
                       int border, uint32_t thr_init, int n_sms, cudaStream_t s) {
  const WorldDev &wd = *wd_host;
  const int nw = wd.H * wd.Wp;
  k_init_planes<<<(nw + 255) / 256, 256, 0, s>>>(wd, border, thr_init);
  k_clear_cells<<<4 * n_sms, 256, 0, s>>>(wd);
  if (wd.C > 0) {
    k_init_agents<<<(wd.C + 255) / 256, 256, 0, s>>>(wd, n0, place_y, place_x);
    k_place_agents<<<(max(wd.C, nw) + 255) / 256, 256, 0, s>>>(wd);
  }
  k_alive_list<<<1, SCAN_THREADS, 0, s>>>(wd);
  launch_init_weights(wd_dev, n0, n_sms, s);
  launch_analysis_reset(wd_host, n_sms, s);
}

void launch_rebuild(const WorldDev *wd_host, int n_sms, cudaStream_t s) {
  const WorldDev &wd = *wd_host;
  const int nw = wd.H * wd.Wp;
  k_clear_cells<<<4 * n_sms, 256, 0, s>>>(wd);
  k_place_agents<<<(max(wd.C, nw) + 255) / 256, 256, 0, s>>>(wd);
  k_alive_list<<<1, SCAN_THREADS, 0, s>>>(wd);
  launch_analysis_reset(wd_host, n_sms, s);
}

}  // namespace eco
