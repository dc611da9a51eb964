// k_analysis.cu -- the metrics the paper tracks in its analyses (App. C),
// computed on the device between steps, once per window:
//   population      agents alive
//   resources       cells holding a resource (the resource channel summed
//                   over the grid)
//   life expectancy deaths of the window and the sum of their ages at death
//                   (accumulated by the physiology phase of every step)
//   movement        for every agent alive over the whole window, the
//                   Manhattan distance between its cell now and at the
//                   window start, counted in 17 bins: bin 17 d / (L + 1) of
//                   the L + 1 possible distances of an L-step window
//                   (bins of 3 for the paper's 50-step windows)
// Agents keep their slot for life, and an agent alive over the whole window
// is exactly a living agent whose age is at least L (ages grow by one every
// step, newborns of the window are younger), so the window start needs only
// one cell per slot.
#include "ecoevo_dev.cuh"

namespace eco {

constexpr int ANALYSIS_THREADS = 256;

__global__ void k_analysis_reset(WorldDev wd) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < wd.C; s += gridDim.x * blockDim.x)
    wd.snap_cell[s] = wd.alive[s] ? wd.y[s] * wd.W + wd.x[s] : -1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Counters &c = *wd.ctr;
    c.snap_t = c.t;
    c.an_deaths = 0;
    c.an_age_sum = 0ull;
  }
}

__device__ inline unsigned long long warp_sum(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Counts over slots and plane words (grid-stride), then the next window's
// start cells.  wd.analysis is zeroed before the launch.
__global__ void __launch_bounds__(ANALYSIS_THREADS) k_analysis(WorldDev wd) {
  __shared__ unsigned long long bins[MOVE_BINS];
  __shared__ unsigned long long tot[3];
  if (threadIdx.x < MOVE_BINS) bins[threadIdx.x] = 0ull;
  if (threadIdx.x < 3) tot[threadIdx.x] = 0ull;
  __syncthreads();
  const long long t = wd.ctr->t;
  const long long L = t - wd.ctr->snap_t;
  const int W = wd.W;
  unsigned long long pop = 0, movers = 0, res = 0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < wd.C; s += gridDim.x * blockDim.x) {
    const bool alive = wd.alive[s] != 0;
    int cell = -1;
    if (alive) {
      const int y = wd.y[s], x = wd.x[s];
      cell = y * W + x;
      ++pop;
      const int start = wd.snap_cell[s];
      if ((long long)wd.age[s] >= L && start >= 0 &&
          ECO_IN_RANGE(wd, start < wd.H * wd.W)) {
        const long long d = (long long)abs(y - start / W) + abs(x - start % W);
        const long long bin = min((long long)(MOVE_BINS - 1), d * MOVE_BINS / (L + 1));
        atomicAdd(&bins[bin], 1ull);
        ++movers;
      }
    }
    wd.snap_cell[s] = cell;
  }
  const uint32_t *plane = (t & 1) ? wd.res1 : wd.res0;
  const int nwords = wd.H * wd.Wp;
  const uint32_t last_mask = (W & 31) ? ((1u << (W & 31)) - 1u) : 0xFFFFFFFFu;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nwords; i += gridDim.x * blockDim.x) {
    uint32_t v = plane[i];
    if (i % wd.Wp == wd.Wp - 1) v &= last_mask;
    res += __popc(v);
  }
  pop = warp_sum(pop);
  movers = warp_sum(movers);
  res = warp_sum(res);
  if ((threadIdx.x & 31) == 0) {
    if (pop) atomicAdd(&tot[0], pop);
    if (movers) atomicAdd(&tot[1], movers);
    if (res) atomicAdd(&tot[2], res);
  }
  __syncthreads();
  unsigned long long *out = wd.analysis;
  if (threadIdx.x < MOVE_BINS && bins[threadIdx.x])
    atomicAdd(&out[A_BINS + threadIdx.x], bins[threadIdx.x]);
  if (threadIdx.x == 0) {
    if (tot[0]) atomicAdd(&out[A_POP], tot[0]);
    if (tot[1]) atomicAdd(&out[A_MOVERS], tot[1]);
    if (tot[2]) atomicAdd(&out[A_RES], tot[2]);
  }
}

// The window's step count and deaths; the next window starts now.
__global__ void k_analysis_finish(WorldDev wd) {
  Counters &c = *wd.ctr;
  unsigned long long *out = wd.analysis;
  out[A_T] = (unsigned long long)c.t;
  out[A_WINDOW] = (unsigned long long)(c.t - c.snap_t);
  out[A_DEATHS] = (unsigned long long)c.an_deaths;
  out[A_AGE_SUM] = c.an_age_sum;
  c.snap_t = c.t;
  c.an_deaths = 0;
  c.an_age_sum = 0ull;
}

// Lab-environment greediness (App. C): a window ends; every living agent
// adds 1 to T_r if a resource was in its view during it, 1 to C_r if it ate.
__global__ void k_lab_window(WorldDev wd) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < wd.C; s += gridDim.x * blockDim.x) {
    if (wd.alive[s]) {
      wd.lab_t[s] += wd.lab_seen[s] ? 1 : 0;
      wd.lab_c[s] += wd.lab_ate[s] ? 1 : 0;
    }
    wd.lab_seen[s] = 0;
    wd.lab_ate[s] = 0;
  }
}

static int analysis_grid(const WorldDev &wd, int n_sms) {
  const int work = max(wd.C, wd.H * wd.Wp);
  const int need = (work + ANALYSIS_THREADS - 1) / ANALYSIS_THREADS;
  return max(1, min(need, 2 * n_sms));
}

void launch_analysis_reset(const WorldDev *wd_host, int n_sms, cudaStream_t s) {
  k_analysis_reset<<<analysis_grid(*wd_host, n_sms), ANALYSIS_THREADS, 0, s>>>(*wd_host);
}

void launch_lab_window(const WorldDev *wd_host, int n_sms, cudaStream_t s) {
  if (wd_host->C > 0)
    k_lab_window<<<analysis_grid(*wd_host, n_sms), ANALYSIS_THREADS, 0, s>>>(*wd_host);
}

void launch_analysis(const WorldDev *wd_host, int n_sms, cudaStream_t s) {
  cudaMemsetAsync(wd_host->analysis, 0, ANALYSIS_WORDS * sizeof(unsigned long long), s);
  k_analysis<<<analysis_grid(*wd_host, n_sms), ANALYSIS_THREADS, 0, s>>>(*wd_host);
  k_analysis_finish<<<1, 1, 0, s>>>(*wd_host);
}

}  // namespace eco
