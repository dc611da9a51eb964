// regrow_tile.cuh -- step part a1: resource regrowth, App. B.1, Eq. (1),
// one 8-row x 4-word tile per CTA.
//
// The resource field is a bit plane (one uint32 word = 32 cells of a row).
// A CTA owns a tile of 8 rows x 4 words (8 x 128 cells) and stages the rows
// and words its neighbourhoods reach (8 + 2R rows x 6 words) in shared
// memory.  Each thread owns 4 adjacent cells: one Philox draw
// {x/4, t, TAG_REGROW, y} gives their 4 words; a neighbour count is the
// popcount of a (2R+1)-bit window of each of the 2R+1 rows.  The update is
// synchronous: every count reads the plane of counter t, the new plane is
// the other buffer of the pair.
#pragma once

#include "ecoevo_dev.cuh"

namespace eco {

constexpr int REGROW_THREADS = 256;

__device__ inline int find_world(const int *prefix, int n, int item) {
  if (n == 1) return 0;
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int TILE_ROWS_MAX = REGROW_ROWS + 6;  // R <= 3
constexpr int TILE_COLS = REGROW_WORDS + 2;

// What the regrowth of a tile reads that no step writes: its world and
// place, and each thread's wall bits and growth thresholds.  The tail
// kernel reads these before waiting for the slot phases.
struct RegrowFixed {
  const WorldDev *wd;
  int y0, w0;
  uint32_t wl;       // wall bits of the thread's 4 cells
  uint32_t thr[4];   // thresholds of the thread's row, by class
};

__device__ inline RegrowFixed regrow_fixed(const BatchDev &b, int tile_id) {
  RegrowFixed f;
  const int w = find_world(b.tile_prefix, b.n, tile_id);
  f.wd = world_ptr(b, w);
  const WorldDev &wd = *f.wd;
  const int tiles_x = (wd.Wp + REGROW_WORDS - 1) / REGROW_WORDS;
  const int local = tile_id - (b.n == 1 ? 0 : b.tile_prefix[w]);
  f.y0 = (local / tiles_x) * REGROW_ROWS;
  f.w0 = (local % tiles_x) * REGROW_WORDS;
  const int y = f.y0 + (threadIdx.x >> 5), ww = f.w0 + ((threadIdx.x >> 3) & 3);
  const int xq = ww * 32 + (threadIdx.x & 7) * 4;
  f.wl = 0u;
  f.thr[0] = f.thr[1] = f.thr[2] = f.thr[3] = 0u;
  if (y < wd.H && ww < wd.Wp && xq < wd.W) {
    f.wl = (wd.wall[y * wd.Wp + ww] >> ((threadIdx.x & 7) * 4)) & 0xFu;
#pragma unroll
    for (int k = 0; k < 4; ++k) f.thr[k] = wd.thr[y * 4 + k];
  }
  return f;
}

// Regrowth of one tile by one CTA of 256 threads; `tile` is the CTA's
// staging array.  The words of both planes of the pair are loaded with the
// step counter that says which one is current.
__device__ inline void regrow_run(const RegrowFixed &f, uint32_t (*tile)[REGROW_WORDS + 2]) {
  const WorldDev &wd = *f.wd;
  const int H = wd.H, W = wd.W, Wp = wd.Wp, R = wd.nbr_radius;
  const int y0 = f.y0, w0 = f.w0;
  const uint32_t t = (uint32_t)wd.ctr->t;

  const int rows = REGROW_ROWS + 2 * R;
  for (int i = threadIdx.x; i < rows * TILE_COLS; i += blockDim.x) {
    int r = i / TILE_COLS, c = i % TILE_COLS;
    int yy = y0 - R + r, ww = w0 - 1 + c;
    uint32_t v0 = 0u, v1 = 0u;
    if (yy >= 0 && yy < H && ww >= 0 && ww < Wp) {
      v0 = wd.res0[yy * Wp + ww];
      v1 = wd.res1[yy * Wp + ww];
    }
    tile[r][c] = (t & 1u) ? v1 : v0;
  }
  __syncthreads();
  uint32_t *rout = (t & 1u) ? wd.res0 : wd.res1;

  const int r = threadIdx.x >> 5;         // row in tile
  const int wi = (threadIdx.x >> 3) & 3;  // word in tile
  const int qd = threadIdx.x & 7;         // quad (4 cells) in word
  const int y = y0 + r, ww = w0 + wi;
  const int xq = ww * 32 + qd * 4;
  uint32_t bits = 0;
  if (y < H && ww < Wp && xq < W) {
    const uint32_t own = (tile[r + R][wi + 1] >> (qd * 4)) & 0xFu;
    const int nvalid = min(4, W - xq);
    const uint32_t valid = (1u << nvalid) - 1u;
    const uint32_t cand = ~own & ~f.wl & valid;
    bits = own;
    if (cand) {
      const U4 u = philox4x32_10(U4{(uint32_t)xq >> 2, t, TAG_REGROW, (uint32_t)y},
                                 wd.key0, wd.key1);
      const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
      const uint32_t win = (1u << (2 * R + 1)) - 1u;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (!((cand >> i) & 1u)) continue;
        // bit position of the window start inside the staged 6-word row
        const int start = 32 + (xq + i - w0 * 32) - R;
        const int c0 = start >> 5, off = start & 31;
        int n = 0;
        for (int dy = -R; dy <= R; ++dy) {
          const uint32_t *row = tile[r + R + dy];
          const uint64_t v = (uint64_t)row[c0] | ((uint64_t)row[c0 + 1] << 32);
          const uint32_t wbits = (uint32_t)(v >> off) & win;
          n += __popc(wbits & nbr_mask(wd.nbr_shape, R, dy));
        }
        const int cls = (n >= wd.class_edges[0]) + (n >= wd.class_edges[1]) +
                        (n >= wd.class_edges[2]);
        const uint32_t th = cls == 0 ? f.thr[0] : cls == 1 ? f.thr[1]
                          : cls == 2 ? f.thr[2] : f.thr[3];
        if (uw[i] < th) bits |= 1u << i;
      }
    }
  }
  uint32_t word = bits << (qd * 4);
  word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
  word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
  word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
  if (qd == 0 && y < H && ww < Wp) rout[y * Wp + ww] = word;
}

}  // namespace eco
