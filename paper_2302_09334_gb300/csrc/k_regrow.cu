// k_regrow.cu -- the regrowth of a world's first plane, after it is created
// or loaded (App. B.1, Eq. (1)); during steps the regrowth of the next step
// runs in the tail kernel (k_agents.cu).
#include "regrow_tile.cuh"

namespace eco {

__global__ void __launch_bounds__(REGROW_THREADS) k_regrow(const __grid_constant__ BatchDev b) {
  __shared__ uint32_t tile[TILE_ROWS_MAX][TILE_COLS];
  regrow_tile(b, blockIdx.x, tile);
}

void preload_regrow() {
  cudaFuncAttributes a;
  cudaFuncGetAttributes(&a, k_regrow);
}

void launch_regrow(const BatchDev &b, cudaStream_t s) {
  if (b.total_tiles > 0) k_regrow<<<b.total_tiles, 256, 0, s>>>(b);
}

}  // namespace eco
