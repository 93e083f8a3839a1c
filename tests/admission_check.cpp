// Host-only checks of the serving loop's admission decision (compiled and run by
// test_admission_cpu.py with the system C++ compiler).
#include <cstdio>
#include <deque>
#include <vector>

#include "../paper_1807_03097_gb300/csrc/admission.h"

static int failures = 0;
#define CHECK(cond)                                           \
  do {                                                        \
    if (!(cond)) {                                            \
      std::printf("FAILED line %d: %s\n", __LINE__, #cond);   \
      ++failures;                                             \
    }                                                         \
  } while (0)

int main() {
  using efie::pick_admission;
  {
    CHECK(pick_admission(0, nullptr, nullptr, 0, 100, false, 8) == -1);
  }
  {  // least work among those that fit
    size_t fp[3] = {10, 10, 10};
    double c[3] = {5, 3, 9};
    CHECK(pick_admission(3, fp, c, 0, 50, false, 8) == 1);
  }
  {  // only the oldest fits the budget
    size_t fp[2] = {10, 100};
    double c[2] = {9, 1};
    CHECK(pick_admission(2, fp, c, 0, 50, false, 8) == 0);
  }
  {  // nothing fits: only when nothing runs may a request exceed the budget
    size_t fp[3] = {100, 200, 300};
    double c[3] = {5, 3, 9};
    CHECK(pick_admission(3, fp, c, 0, 50, false, 8) == -1);
    CHECK(pick_admission(3, fp, c, 0, 50, true, 8) == 1);
  }
  {  // the window: requests behind the 8 oldest are not considered
    size_t fp[10];
    double c[10];
    for (int i = 0; i < 10; ++i) {
      fp[i] = 1;
      c[i] = 10.0 - i;  // cheapest at index 9
    }
    CHECK(pick_admission(10, fp, c, 0, 50, false, 8) == 7);
  }
  {  // the oldest goes first after 8 passes, if it fits
    size_t fp[3] = {10, 10, 10};
    double c[3] = {9, 1, 2};
    CHECK(pick_admission(3, fp, c, 8, 50, false, 8) == 0);
    CHECK(pick_admission(3, fp, c, 7, 50, false, 8) == 1);
    // once passed 8 times the oldest is next even if it does not fit yet: nothing else starts
    size_t fp2[3] = {100, 10, 10};
    CHECK(pick_admission(3, fp2, c, 8, 50, false, 8) == -1);
    CHECK(pick_admission(3, fp2, c, 7, 50, false, 8) == 1);
    CHECK(pick_admission(3, fp2, c, 8, 100, false, 8) == 0);
  }
  {  // a large request behind a steady stream of small ones: the memory released by finishing
     // requests is held for it, so it starts after a bounded number of releases
    const size_t budget = 100;
    size_t in_use = 0;
    std::deque<std::pair<size_t, double>> q;
    q.push_back({90, 1000.0});
    std::deque<size_t> running;  // footprints of running requests, oldest first
    int passed = 0, steps = 0;
    bool started = false;
    for (int i = 0; i < 200; ++i) q.push_back({30, 1.0});
    while (!started && steps < 1000) {
      ++steps;
      // admit as many as fit (slots unlimited here), then one running request finishes
      for (;;) {
        size_t fp[8];
        double c[8];
        const int n = (int)std::min<size_t>(q.size(), 8);
        for (int i = 0; i < n; ++i) {
          fp[i] = q[i].first;
          c[i] = q[i].second;
        }
        const int k = pick_admission(n, fp, c, passed, budget - in_use, running.empty(), 8);
        if (k < 0) break;
        if (k == 0) {
          started = true;
          break;
        }
        ++passed;
        in_use += q[k].first;
        running.push_back(q[k].first);
        q.erase(q.begin() + k);
      }
      if (!started && !running.empty()) {
        in_use -= running.front();
        running.pop_front();
      }
    }
    CHECK(started);
    CHECK(passed == 8);
    CHECK(steps < 20);
  }
  {  // a large request at the head of a stream of small ones is passed exactly 8 times
    std::deque<std::pair<size_t, double>> q;
    q.push_back({10, 1000.0});
    for (int i = 0; i < 30; ++i) q.push_back({10, 1.0 + 0.01 * i});
    int passed = 0, admitted_before = 0;
    for (;;) {
      size_t fp[8];
      double c[8];
      const int n = (int)std::min<size_t>(q.size(), 8);
      for (int i = 0; i < n; ++i) {
        fp[i] = q[i].first;
        c[i] = q[i].second;
      }
      const int k = pick_admission(n, fp, c, passed, 50, false, 8);
      CHECK(k >= 0);
      if (k < 0) break;
      if (k == 0) break;  // the large request
      ++passed;
      ++admitted_before;
      q.erase(q.begin() + k);
    }
    CHECK(admitted_before == 8);
  }
  {  // footprint estimate: the mixed form stores an FP32 copy of the near blocks; directions
     // solved in lockstep each hold a Krylov basis (at most 64); FP64 solves are sequential
    using efie::request_footprint;
    const size_t f64 = request_footprint(6, 5, 2, 8, 1500, 3000, false, 1, 0, 1);  // matrices evaluated
    const size_t f32 = request_footprint(6, 5, 2, 8, 1500, 3000, true, 1);
    // kept FP64 coupling matrices (the default of the FP64 form): 16 bytes per node pair
    const size_t ncl = 6 * 1365;
    CHECK(request_footprint(6, 5, 2, 8, 1500, 3000, false, 1) >= f64 + 130 * ncl * 81 * 81 * 16);
    CHECK(request_footprint(6, 5, 2, 8, 1500, 3000, true, 1, 0, 2) >= f32 + 130 * ncl * 81 * 81 * 8);
    CHECK(f32 > f64);
    const size_t ndof = 2 * 6 * 33 * 33, krylov1 = 1501 * ndof * 16;
    const size_t f32x16 = request_footprint(6, 5, 2, 8, 1500, 3000, true, 16);
    CHECK(f32x16 >= f32 + 15 * krylov1);
    CHECK(request_footprint(6, 5, 2, 8, 1500, 3000, true, 100) == request_footprint(6, 5, 2, 8, 1500, 3000, true, 64));
    CHECK(request_footprint(6, 5, 2, 8, 1500, 3000, false, 16, 0, 1) == f64);
    CHECK(request_footprint(6, 6, 2, 8, 1500, 3000, true, 1) > f32);
    CHECK(request_footprint(6, 5, 2, 8, 20, 3000, true, 1) < f32);  // shorter restart, smaller basis
    // far-field scratch: 3 complex doubles per element and direction
    const size_t nE = 6 * 32 * 32;
    CHECK(request_footprint(6, 5, 2, 8, 1500, 3000, true, 1, 64) >= f32 + 48 * 64 * nE);
    CHECK(request_footprint(6, 5, 2, 8, 1500, 3000, true, 1, 0) == f32);
  }
  if (failures == 0) std::printf("ok\n");
  return failures == 0 ? 0 : 1;
}
