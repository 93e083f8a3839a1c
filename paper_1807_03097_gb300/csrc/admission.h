// Admission of the serving loop (host only, no CUDA): the device-memory estimate of a request
// and the decision which queued request to start when a slot is free.  Among the `lookahead`
// oldest queued requests whose estimated device footprint fits the remaining budget (any
// request fits when nothing runs), the one with the least estimated work is chosen.  Once
// `lookahead` admissions have gone to requests behind the oldest, the oldest is next: nothing
// else is admitted until it fits, so that memory released by finishing requests is held for it
// and its wait is bounded.  Returns the queue index (0 = oldest) or -1 when none may start.
#pragma once
#include <algorithm>
#include <cstddef>

namespace efie {

// Device memory of one scattering request, estimated from the discretisation before anything
// is built: near-field blocks (at most 40 neighbours per element: the sphere workloads have 21 to
// 30, the tori of the serving mix up to 36; FP64 plus an FP32 copy in the
// mixed form), the Krylov bases, cluster data and work vectors, and the far-field scratch of
// ndir directions (3 complex values per element and direction, plus the output).  In the
// mixed form the directions of a request are solved in lockstep (up to 64 at a time), each
// with its own Krylov basis, and the batched product holds per-direction superspace vectors
// and cluster fields.  When the coupling matrices of the admissible blocks are kept in device
// memory (m2l_store: the FP64 form by default, the mixed form on request), they are counted
// with at most 130 admissible source clusters per cluster (the block trees of the sphere and
// torus workloads have 63 to 115).  With the leaf-level variant (leaf_dense) the admissible
// pairs of two elements are near-field blocks too: at most 130 more per element.  np patches,
// 2^level_m elements per patch direction, degree p, interpolation degree q.
inline size_t request_footprint(int np, int level_m, int p, int q, int gmres_restart, int gmres_maxit, bool mixed,
                                int nrhs, int ndir = 0, int m2l_store = 0, int leaf_dense = 0) {
  const size_t n = size_t(1) << level_m, nE = size_t(np) * n * n;
  const size_t p1 = p + 1, nb = 2 * p1 * p1, nI = size_t(q + 1) * (q + 1);
  const size_t ndof = 2 * size_t(np) * (n + p - 1) * (n + p - 1);
  const size_t near = (leaf_dense ? 160 : 40) * nE * (nb * nb * (mixed ? 24 : 16) + 8);
  const size_t kr = (size_t)std::min(gmres_restart, gmres_maxit) + 1;
  const size_t lockstep = (mixed && nrhs > 1) ? (size_t)std::min(nrhs, 64) : 1;
  const size_t krylov = lockstep * (kr * ndof * 16 + kr * kr * 16);
  const size_t ncl = nE * 4 / 3 + np;
  // per cluster: node geometry and the FMM fields; per admissible pair (at most 130 per
  // cluster): pair geometry and phase, CSR entries, the unordered-pair lists (48 bytes)
  const size_t clusters = ncl * nI * (72 + 14 * 16) + 130 * ncl * 48;
  const size_t vecs = nE * nb * 16 * 6 + ndof * 16 * 8;
  const size_t batch = lockstep > 1 ? lockstep * (5 * nE * nb * 16 + 14 * ncl * nI * 8 + 4 * ndof * 16) : 0;
  const size_t farfield = ndir > 0 ? 48 * size_t(ndir) * nE + 48 * size_t(ndir) + 24 * size_t(ndir) : 0;
  const bool stored = mixed ? m2l_store == 2 : m2l_store != 1;
  const size_t coupling = stored ? 130 * ncl * nI * nI * (mixed ? 8 : 16) : 0;
  return near + krylov + clusters + vecs + batch + farfield + coupling + (size_t(64) << 20);
}

inline int pick_admission(int nqueued, const size_t *footprint, const double *cost, int oldest_passed, size_t left,
                          bool idle, int lookahead) {
  auto fits = [&](int i) { return footprint[i] <= left || idle; };
  if (nqueued <= 0) return -1;
  if (oldest_passed >= lookahead) return fits(0) ? 0 : -1;
  int best = -1;
  for (int i = 0; i < nqueued && i < lookahead; ++i)
    if (fits(i) && (best < 0 || cost[i] < cost[best])) best = i;
  return best;
}

}  // namespace efie
