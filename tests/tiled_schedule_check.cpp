// Enumerates the item order of the tiled fused form (tiled_schedule.h, the
// header the kernel uses) for several queues and checks what the kernel's
// termination argument rests on:
//   - decode is a bijection from items onto stage-0 tasks and stage-1 tasks;
//   - every stage-1 task comes after all stage-0 tasks of its pair;
//   - every stage-0 task that waits for a slot comes after the stage-1 task
//     of the slot's previous pair, which has the same image side;
//   - that stage-1 task comes at least LAG items before (so it normally has
//     finished), except where the order ends;
//   - single-stage nets: the items are the stage-0 tasks in order.
// Prints "ok" and exits 0, or prints the first violation and exits 1.
#include <cstdio>
#include <vector>

#include "tiled_schedule.h"

using namespace nkf::sched;

struct Q {
  int n;
  int R[8];
  int nt0[8];
  int64_t g0[9], f0[9];
  int64_t G, G64, T0, LAG;
  int S[2];
};

static int fail(const char* what, long long a, long long b) {
  std::printf("FAIL %s (%lld, %lld)\n", what, a, b);
  return 1;
}

static int check(const std::vector<int>& R, const std::vector<int64_t>& np, int grid, bool two) {
  Q q = {};
  q.n = (int)R.size();
  q.g0[0] = q.f0[0] = 0;
  for (int b = 0; b < q.n; ++b) {
    q.R[b] = R[b];
    q.nt0[b] = tasks_per_pair(R[b]);
    q.g0[b + 1] = q.g0[b] + np[b];
    q.f0[b + 1] = q.f0[b] + np[b] * q.nt0[b];
    if (R[b] == 64) q.G64 = q.g0[b + 1];
  }
  q.G = q.g0[q.n];
  q.T0 = q.f0[q.n];
  const Plan p = make_plan(two, R.data(), np.data(), q.n, grid);
  q.LAG = p.LAG;
  q.S[0] = p.S[0];
  q.S[1] = p.S[1];
  const int64_t nitems = q.T0 + (two ? q.G : 0);
  std::vector<int64_t> pos0(q.T0, -1), pos1(q.G, -1), first0(q.G, -1), last0(q.G, -1);
  for (int64_t m = 0; m < nitems; ++m) {
    int64_t k;
    const int st1 = decode(q, two, m, &k);
    if (st1) {
      if (k < 0 || k >= q.G || pos1[k] >= 0) return fail("stage-1 item decoded twice or out of range", m, k);
      pos1[k] = m;
    } else {
      if (k < 0 || k >= q.T0 || pos0[k] >= 0) return fail("stage-0 item decoded twice or out of range", m, k);
      if (!two && k != m) return fail("single-stage order", m, k);
      pos0[k] = m;
      int b, sub;
      int64_t g;
      stage0_of(q, k, &b, &g, &sub);
      if (g < q.g0[b] || g >= q.g0[b + 1] || sub < 0 || sub >= q.nt0[b]) return fail("stage-0 task", k, g);
      if (first0[g] < 0) first0[g] = m;
      last0[g] = m;
    }
  }
  for (int64_t k = 0; k < q.T0; ++k)
    if (pos0[k] < 0) return fail("stage-0 task missing", k, 0);
  if (!two) return 0;
  for (int64_t g = 0; g < q.G; ++g) {
    if (pos1[g] < 0) return fail("stage-1 task missing", g, 0);
    if (pos1[g] <= last0[g]) return fail("stage-1 task before its stage-0 tasks", g, pos1[g]);
    if (g > 0 && stage1_pos(q, g) <= stage1_pos(q, g - 1)) return fail("stage-1 positions not increasing", g, 0);
    const int b = block_of_pair(q, g);
    int ring;
    int64_t prev;
    const int64_t s = slot(q, b, g, &ring, &prev);
    if (s < 0 || s >= q.S[ring]) return fail("slot out of its ring", g, s);
    if (prev >= 0) {
      int ring_prev;
      int64_t prev2;
      const int64_t sp = slot(q, block_of_pair(q, prev), prev, &ring_prev, &prev2);
      if (ring_prev != ring || sp != s) return fail("previous user of the slot", g, prev);
      if (pos1[prev] >= first0[g]) return fail("slot wait on a later item", g, prev);
      if (first0[g] - pos1[prev] < q.LAG) return fail("slot wait less than LAG items back", g, prev);
    }
  }
  return 0;
}

int main() {
  struct Case {
    std::vector<int> R;
    std::vector<int64_t> np;
    int grid;
  };
  const std::vector<Case> cases = {
      {{64, 64, 32, 32}, {21, 18, 36, 30}, 152},
      {{64}, {300}, 152},
      {{32}, {500}, 304},
      {{64, 32}, {1, 2000}, 152},
      {{64, 32, 32}, {50, 7, 900}, 4},
      {{32}, {3}, 304},
      {{64}, {1}, 1},
      {{64, 32}, {2000, 1}, 152},
      // the mixed-resolution workload at full size: 512 + 128 images at 64x64 and 32x32
      {{64, 64, 32, 32}, {512 * 513 / 2, 128 * 512, 512 * 513 / 2, 128 * 512}, 152},
  };
  for (const Case& c : cases)
    for (bool two : {true, false})
      if (check(c.R, c.np, c.grid, two)) return 1;
  std::printf("ok\n");
  return 0;
}
