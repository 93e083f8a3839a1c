// Admission decision of the serving loop (host only, no CUDA): which queued request to start
// when a slot is free.  Among the `lookahead` oldest queued requests whose estimated device
// footprint fits the remaining budget (any request fits when nothing runs), the one with the
// least estimated work is chosen; the oldest is chosen once `passes` admissions have gone to
// requests behind it.  Returns the queue index (0 = oldest) or -1 when none fits.
#pragma once
#include <cstddef>

namespace efie {

inline int pick_admission(int nqueued, const size_t *footprint, const double *cost, int oldest_passed, size_t left,
                          bool idle, int lookahead) {
  auto fits = [&](int i) { return footprint[i] <= left || idle; };
  if (nqueued <= 0) return -1;
  if (oldest_passed >= lookahead && fits(0)) return 0;
  int best = -1;
  for (int i = 0; i < nqueued && i < lookahead; ++i)
    if (fits(i) && (best < 0 || cost[i] < cost[best])) best = i;
  return best;
}

}  // namespace efie
