// regrow_tile.cuh -- step part a1: resource regrowth, App. B.1, Eq. (1),
// k stacked 8-row x 4-word tiles per CTA.
//
// The resource field is a bit plane (one uint32 word = 32 cells of a row).
// A CTA owns a column of k tiles of 8 rows x 4 words (8k x 128 cells; k =
// regrow_k of the batch, 1..REGROW_KMAX) and stages the rows and words its
// neighbourhoods reach (8k + 2R rows x 6 words) in shared memory, with the
// wall words and growth thresholds of its rows.  Each thread owns 4
// adjacent cells in each of the k tiles: one Philox draw {x/4, t,
// TAG_REGROW, y} gives their 4 words; a neighbour count is the popcount of a
// (2R+1)-bit window of each of the 2R+1 rows.  The update is synchronous:
// every count reads the plane of counter t, the new plane is the other
// buffer of the pair.  Stacking tiles cuts a large world's CTAs (and their
// load round trips) by k and re-reads 2R halo rows per k tiles, not per
// tile.
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

constexpr int TILE_COLS = REGROW_WORDS + 2;
constexpr int TILE_ROWS_MAX = REGROW_ROWS * REGROW_KMAX + 6;  // R <= 3

struct RegrowSmem {
  uint32_t tile[TILE_ROWS_MAX][TILE_COLS];                // plane of counter t
  uint32_t wall[REGROW_ROWS * REGROW_KMAX][REGROW_WORDS];  // the CTA's wall words
  uint32_t thr[REGROW_ROWS * REGROW_KMAX][4];            // thresholds by class
};

struct RegrowPlace {
  const WorldDev *wd;
  int y0, w0;
};

// The CTA's world and place; its wall words and thresholds, which no step
// writes, are staged before the tail kernel waits for the slot phases (the
// barrier in regrow_run makes them visible).
__device__ inline RegrowPlace regrow_fixed(const BatchDev &b, int tile_id, RegrowSmem &s) {
  RegrowPlace f;
  const int w = find_world(b.tile_prefix, b.n, tile_id);
  f.wd = world_ptr(b, w);
  const WorldDev &wd = *f.wd;
  const int k = b.regrow_k;
  const int tiles_x = (wd.Wp + REGROW_WORDS - 1) / REGROW_WORDS;
  const int local = tile_id - (b.n == 1 ? 0 : b.tile_prefix[w]);
  f.y0 = (local / tiles_x) * (REGROW_ROWS * k);
  f.w0 = (local % tiles_x) * REGROW_WORDS;
  const int rows = REGROW_ROWS * k;
  for (int i = threadIdx.x; i < rows * REGROW_WORDS; i += blockDim.x) {
    const int r = i / REGROW_WORDS, c = i % REGROW_WORDS;
    const int y = f.y0 + r, ww = f.w0 + c;
    s.wall[r][c] = (y < wd.H && ww < wd.Wp) ? wd.wall[y * wd.Wp + ww] : 0u;
    s.thr[r][c] = y < wd.H ? wd.thr[y * 4 + c] : 0u;   // REGROW_WORDS == 4 classes
  }
  return f;
}
static_assert(REGROW_WORDS == 4, "a staging pass loads 4 thresholds per row");

// Neighbourhood bits of row offset dy in a (2R+1)-bit window, App. B.1:
// square (Chebyshev) or diamond of radius R, the centre excluded (compile-time
// shape and radius).
template <int SHAPE, int R>
__device__ constexpr uint32_t nbr_mask_c(int dy) {
  const int ady = dy < 0 ? -dy : dy;
  const int reach = SHAPE == 1 ? R - ady : R;
  uint32_t m = reach >= 0 ? ((1u << (2 * reach + 1)) - 1u) << (R - reach) : 0u;
  return dy == 0 ? (m & ~(1u << R)) : m;
}

// The new words of the CTA's k tiles from the staged plane: a thread's
// quad of cells in each tile, one Philox draw per quad with a candidate
// (an empty cell off the walls), the neighbour count of a cell the popcount
// of its window in each of the 2R+1 rows -- the quad's four windows cut from
// one funnel shift per row.
template <int SHAPE, int R>
__device__ inline void regrow_cells(const RegrowPlace &f, int k, const RegrowSmem &s,
                                    uint32_t t, uint32_t *rout) {
  const WorldDev &wd = *f.wd;
  const int H = wd.H, W = wd.W, Wp = wd.Wp;
  const int y0 = f.y0, w0 = f.w0;
  const int wi = (threadIdx.x >> 3) & 3;  // word in tile
  const int qd = threadIdx.x & 7;         // quad (4 cells) in word
  const int ww = w0 + wi;
  const int xq = ww * 32 + qd * 4;
  constexpr uint32_t WIN = (1u << (2 * R + 1)) - 1u;
  // bit position of the first cell's window start inside the staged 6-word row
  const int start = 32 + (xq - w0 * 32) - R;
  const int c0 = start >> 5, off = start & 31;
  const int e0 = wd.class_edges[0], e1 = wd.class_edges[1], e2 = wd.class_edges[2];
#pragma unroll 2
  for (int kb = 0; kb < k; ++kb) {
    const int r = kb * REGROW_ROWS + (threadIdx.x >> 5);   // row in the column
    const int y = y0 + r;
    uint32_t bits = 0;
    if (y < H && ww < Wp && xq < W) {
      const uint32_t own = (s.tile[r + R][wi + 1] >> (qd * 4)) & 0xFu;
      const uint32_t wl = (s.wall[r][wi] >> (qd * 4)) & 0xFu;
      const int nvalid = min(4, W - xq);
      const uint32_t valid = (1u << nvalid) - 1u;
      const uint32_t cand = ~own & ~wl & valid;
      bits = own;
      if (cand) {
        const U4 u = philox4x32_10(U4{(uint32_t)xq >> 2, t, TAG_REGROW, (uint32_t)y},
                                   wd.key0, wd.key1);
        const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
        int n[4] = {0, 0, 0, 0};
#pragma unroll
        for (int dy = -R; dy <= R; ++dy) {
          const uint32_t *row = s.tile[r + R + dy];
          const uint32_t win4 = __funnelshift_r(row[c0], row[c0 + 1], off);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            n[i] += __popc((win4 >> i) & WIN & nbr_mask_c<SHAPE, R>(dy));
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int cls = (n[i] >= e0) + (n[i] >= e1) + (n[i] >= e2);
          if (((cand >> i) & 1u) && uw[i] < s.thr[r][cls]) bits |= 1u << i;
        }
      }
    }
    uint32_t word = bits << (qd * 4);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 1);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 2);
    word |= __shfl_xor_sync(0xFFFFFFFFu, word, 4);
    if (qd == 0 && y < H && ww < Wp) rout[y * Wp + ww] = word;
  }
}

// Regrowth of one column of k tiles by one CTA of 256 threads.  The words
// of both planes of the pair are loaded with the step counter that says
// which one is current.
__device__ inline void regrow_run(const RegrowPlace &f, int k, RegrowSmem &s) {
  const WorldDev &wd = *f.wd;
  const int H = wd.H, Wp = wd.Wp, R = wd.nbr_radius;
  const int y0 = f.y0, w0 = f.w0;
  const uint32_t t = (uint32_t)wd.ctr->t;

  const int rows = REGROW_ROWS * k + 2 * R;
  for (int i = threadIdx.x; i < rows * TILE_COLS; i += blockDim.x) {
    int r = i / TILE_COLS, c = i % TILE_COLS;
    int yy = y0 - R + r, ww = w0 - 1 + c;
    uint32_t v0 = 0u, v1 = 0u;
    if (yy >= 0 && yy < H && ww >= 0 && ww < Wp) {
      v0 = wd.res0[yy * Wp + ww];
      v1 = wd.res1[yy * Wp + ww];
    }
    s.tile[r][c] = (t & 1u) ? v1 : v0;
  }
  __syncthreads();
  uint32_t *rout = (t & 1u) ? wd.res0 : wd.res1;
  switch (wd.nbr_shape * 4 + R) {   // radius 1..3 (checked at creation)
    case 1: regrow_cells<0, 1>(f, k, s, t, rout); break;
    case 2: regrow_cells<0, 2>(f, k, s, t, rout); break;
    case 3: regrow_cells<0, 3>(f, k, s, t, rout); break;
    case 5: regrow_cells<1, 1>(f, k, s, t, rout); break;
    case 6: regrow_cells<1, 2>(f, k, s, t, rout); break;
    default: regrow_cells<1, 3>(f, k, s, t, rout); break;
  }
}

}  // namespace eco
