// move_claim.cuh -- the move claim of step part a4, shared by the
// controller kernels, and the world lookup of a batch-wide agent index.
#pragma once

#include "ecoevo_dev.cuh"

namespace eco {

// Move claim of one agent (step part a4), made as soon as its action is
// known: a target on the grid, not a wall and empty at the start of the
// phase (the slot map does not change during this kernel) is claimed with
// atomicMin; the lowest claimant moves in the next kernel.  The loads of an
// agent's claim are issued when its action is known and used one agent
// later, so their latency hides behind the next agent's work.
struct MoveClaim {
  const WorldDev *wd = nullptr;
  int slot = -1, cell = -1, bit = 0, occ = 0;
  uint32_t wall = 0;
  bool moving = false, off_grid = false;

  __device__ void issue(const WorldDev &w, int s, int y, int x, int a) {
    wd = &w;
    slot = s;
    cell = -1;
    moving = a >= 1 && a < NACT;
    off_grid = false;
    if (!moving) return;
    const int ty = y + (a == 1 ? -1 : a == 2 ? 1 : 0);
    const int tx = x + (a == 3 ? 1 : a == 4 ? -1 : 0);
    if (ty < 0 || ty >= w.H || tx < 0 || tx >= w.W) {
      off_grid = true;
      return;
    }
    cell = ty * w.W + tx;
    bit = tx & 31;
    wall = w.wall[ty * w.Wp + (tx >> 5)];
    occ = w.slot_map[cell];
  }

  __device__ void resolve() {
    if (slot < 0) return;
    const bool blocked = off_grid || (cell >= 0 && ((wall >> bit) & 1u));
    int tgt = -1;
    if (moving && !blocked && occ == -1) {
      tgt = cell;
      atomicMin(&wd->claim[cell], slot);
    }
    wd->target[slot] = tgt;
    wd->killed[slot] = (moving && blocked && wd->wall_kills) ? 1 : 0;
    slot = -1;
  }
};

// World of global agent index a (prefix over worlds in shared memory).
__device__ inline int world_of(const int *prefix, int n, int a) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (prefix[mid] <= a) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace eco
