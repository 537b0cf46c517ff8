// Item order and slot rings of the tiled fused Myrtle form (myrtle_tiled.cu),
// written once for the device and for plain C++ (the CPU tests compile this
// header with g++ and enumerate whole queues).
//
// A queue holds blocks of 64x64 pairs first, then blocks of 32x32 pairs.
// Pair g's stage 0 is cut into tasks_per_pair(side) tasks; the items are all
// stage-0 tasks, block by block, with the stage-1 task of pair k merged LAG
// stage-0 tasks after k's last one (after all of them near the end).  Each
// image side owns a ring of S slots; pair g's slot was last used by pair
// g - S of the same side.  Functions take any struct Q with the fields
//   n, R[b], nt0[b], g0[b] (first pair of block b, g0[n] = G),
//   f0[b] (first stage-0 task of block b, f0[n] = T0), G, G64, T0, LAG, S[2].
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define NK_SCHED_HD __host__ __device__ inline
#else
#define NK_SCHED_HD inline
#endif

namespace nkf {
namespace sched {

// stage-0 tasks of a pair: 2 bands x 4 shift-t_y groups x 8 shift-t_x groups
// at 64x64, 1 x 2 x 4 at 32x32
NK_SCHED_HD constexpr int tasks_per_pair(int side) { return side == 64 ? 64 : 8; }

template <class Q>
NK_SCHED_HD int block_of_pair(const Q& q, int64_t g) {
  int b = 0;
  while (b + 1 < q.n && g >= q.g0[b + 1]) ++b;
  return b;
}

// stage-0 task index k -> block, pair, task within the pair
template <class Q>
NK_SCHED_HD void stage0_of(const Q& q, int64_t k, int* b, int64_t* g, int* sub) {
  int bb = 0;
  while (bb + 1 < q.n && k >= q.f0[bb + 1]) ++bb;
  *b = bb;
  *g = q.g0[bb] + (k - q.f0[bb]) / q.nt0[bb];
  *sub = (int)((k - q.f0[bb]) % q.nt0[bb]);
}

// position of pair k's stage-1 task in the item order
template <class Q>
NK_SCHED_HD int64_t stage1_pos(const Q& q, int64_t k) {
  const int b = block_of_pair(q, k);
  int64_t x = q.f0[b] + (k - q.g0[b] + 1) * q.nt0[b] + q.LAG;
  if (x > q.T0) x = q.T0;
  return x + k;
}

// item m -> stage-1 task of pair *k (returns 1) or stage-0 task *k (0)
template <class Q>
NK_SCHED_HD int decode(const Q& q, bool two, int64_t m, int64_t* k) {
  if (!two) {
    *k = m;
    return 0;
  }
  int64_t lo = 0, hi = q.G;  // number of stage-1 tasks at positions <= m
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    if (stage1_pos(q, mid) <= m)
      lo = mid + 1;
    else
      hi = mid;
  }
  if (lo > 0 && stage1_pos(q, lo - 1) == m) {
    *k = lo - 1;
    return 1;
  }
  *k = m - lo;
  return 0;
}

// ring (0: 64x64, 1: 32x32) and slot of pair g of block b; *prev = the pair
// that used the slot before (-1: none)
template <class Q>
NK_SCHED_HD int64_t slot(const Q& q, int b, int64_t g, int* ring, int64_t* prev) {
  const int r = q.R[b] == 64 ? 0 : 1;
  const int64_t ord = r == 0 ? g : g - q.G64;
  *ring = r;
  *prev = ord >= q.S[r] ? g - q.S[r] : -1;
  return ord % q.S[r];
}

// Lag and ring sizes of a launch of `grid` CTAs: stage-1 tasks come LAG =
// two waves after their pair's last stage-0 task; order alone needs
// S >= LAG / tasks + 1, and one more LAG between a slot's stage-1 task and
// its next user lets that task finish before it is waited for.  `tensors`
// pooled tensors per slot and global-average sums per pair (2 for the NTK:
// K and Theta).
struct Plan {
  int64_t LAG;
  int S[2];
  int64_t slot_floats[2], ring_off[2];
  uint64_t slot_bytes, bytes;
};

inline Plan make_plan(bool two, const int* R, const int64_t* npairs, int n, int grid, int tensors = 1) {
  Plan p = {};
  p.LAG = 2 * (int64_t)grid;
  int64_t G = 0;
  bool has[2] = {false, false};
  for (int b = 0; b < n; ++b) {
    has[R[b] == 64 ? 0 : 1] = true;
    G += npairs[b];
  }
  const int side[2] = {64, 32};
  int64_t off = 0;
  for (int r = 0; r < 2; ++r) {
    const int nt = tasks_per_pair(side[r]);
    const int64_t R1 = side[r] / 2;
    p.S[r] = (two && has[r]) ? (int)((2 * p.LAG + nt - 1) / nt) + 2 : 1;
    p.slot_floats[r] = (two && has[r]) ? tensors * R1 * R1 * R1 * R1 : 0;
    p.ring_off[r] = off;
    off += p.S[r] * p.slot_floats[r];
  }
  p.slot_bytes = (uint64_t)off * sizeof(float);
  p.bytes = p.slot_bytes + (uint64_t)G * (2 * sizeof(int) + tensors * sizeof(double)) + 64;
  return p;
}

}  // namespace sched
}  // namespace nkf
