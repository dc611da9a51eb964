// k_moves_noalloc.cu -- move resolution that allocates no device memory.
//
// The same rule as the moves of the simulation step: a move succeeds iff
// its target is on the grid, not a wall, empty at the start of the phase,
// and the mover is the lowest slot among the agents claiming that cell.
// The per-cell claims live in a fixed array in this library's own device
// memory instead of an arena, so a caller that cannot allocate device
// memory can still resolve moves on arrays it already owns.
#include <climits>
#include <cstdio>
#include <mutex>

#include "ecoevo_dev.cuh"

namespace eco {
namespace {

// Largest grid the array serves: 2^21 cells (8 MiB of int32 claims), enough
// for a 1000 x 2000 world.  Every GPU that loads the library holds it.
constexpr long long kMaxCells = 1ll << 21;
__device__ __align__(256) int32_t g_move_claims[kMaxCells];

constexpr int kMaxDevices = 64;
int32_t *g_claims_on_device[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

__constant__ int kNaDY[5] = {0, -1, 1, 0, 0};  // stay, N, S, E, W
__constant__ int kNaDX[5] = {0, 0, 0, 1, -1};

__global__ void k_na_clear(int32_t *claims, int n_cells) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cells;
       i += gridDim.x * blockDim.x)
    claims[i] = INT_MAX;
}

// Target cell of slot s, or -1 when the agent stays or cannot move.
__device__ inline int na_target(int H, int W, const uint8_t *wall, const int32_t *y,
                                const int32_t *x, int a, int s, bool &blocked) {
  blocked = false;
  if (a <= 0 || a >= NACT) return -1;
  const int ty = y[s] + kNaDY[a], tx = x[s] + kNaDX[a];
  if (ty < 0 || ty >= H || tx < 0 || tx >= W || wall[ty * W + tx]) {
    blocked = true;
    return -1;
  }
  return ty * W + tx;
}

__global__ void k_na_claim(int H, int W, int C, int wall_kills, const uint8_t *wall,
                           const uint8_t *alive, const int32_t *actions, const int32_t *y,
                           const int32_t *x, const int32_t *slot_map, uint8_t *killed,
                           int32_t *claims) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= C) return;
  if (killed) killed[s] = 0;
  if (!alive[s]) return;
  bool blocked;
  const int cell = na_target(H, W, wall, y, x, actions[s], s, blocked);
  if (blocked && wall_kills && killed) killed[s] = 1;
  if (cell < 0 || slot_map[cell] != -1) return;
  atomicMin(&claims[cell], s);
}

__global__ void k_na_apply(int H, int W, int C, const uint8_t *wall, const uint8_t *alive,
                           const int32_t *actions, int32_t *y, int32_t *x,
                           int32_t *slot_map, int32_t *claims) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= C || !alive[s]) return;
  bool blocked;
  const int cell = na_target(H, W, wall, y, x, actions[s], s, blocked);
  if (cell < 0 || claims[cell] != s) return;
  claims[cell] = INT_MAX;  // only the winner resets its cell
  slot_map[y[s] * W + x[s]] = -1;
  slot_map[cell] = s;
  y[s] = cell / W;
  x[s] = cell % W;
}

// Device address of the claim array on the current device, looked up once
// per device.  Host code must not use g_move_claims itself: on the host that
// name is only a stand-in for the device array.
int claims_pointer(int32_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ECO_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_claims_on_device[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_move_claims);
    if (e != cudaSuccess || !p) {
      std::fprintf(stderr, "libecoevo: cudaGetSymbolAddress failed: %s\n",
                   cudaGetErrorString(e));
      return ECO_ECUDA;
    }
    g_claims_on_device[dev] = static_cast<int32_t *>(p);
  }
  *out = g_claims_on_device[dev];
  return ECO_OK;
}

}  // namespace
}  // namespace eco

extern "C" int eco_moves_noalloc(int32_t H, int32_t W, int32_t capacity, int32_t wall_kills,
                                 const uint8_t *wall, const uint8_t *alive,
                                 const int32_t *actions, int32_t *y, int32_t *x,
                                 int32_t *slot_map, uint8_t *killed, void *stream) {
  using namespace eco;
  if (H < 1 || W < 1 || capacity < 0 || (long long)H * W > kMaxCells) {
    if (H >= 1 && W >= 1 && (long long)H * W > kMaxCells)
      std::fprintf(stderr, "libecoevo: eco_moves_noalloc serves at most %lld cells, got %lld\n",
                   kMaxCells, (long long)H * W);
    return ECO_EINVAL;
  }
  if (capacity > 0 && (!wall || !alive || !actions || !y || !x || !slot_map))
    return ECO_EINVAL;
  int32_t *claims = nullptr;
  int rc = claims_pointer(&claims);
  if (rc != ECO_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int n_cells = H * W;
  k_na_clear<<<(n_cells + 255) / 256 < 1024 ? (n_cells + 255) / 256 : 1024, 256, 0, s>>>(
      claims, n_cells);
  if (capacity > 0) {
    const int blocks = (capacity + 255) / 256;
    k_na_claim<<<blocks, 256, 0, s>>>(H, W, capacity, wall_kills, wall, alive, actions, y, x,
                                      slot_map, killed, claims);
    k_na_apply<<<blocks, 256, 0, s>>>(H, W, capacity, wall, alive, actions, y, x, slot_map,
                                      claims);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    std::fprintf(stderr, "libecoevo: eco_moves_noalloc launch failed: %s\n",
                 cudaGetErrorString(e));
    return ECO_ECUDA;
  }
  return ECO_OK;
}
