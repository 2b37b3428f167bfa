// host_opts.h -- option checks and the host-to-device option copy shared by
// every entry point of the C-ABI (plan-based solves and the allocation-free
// solve), so that the same options give the same status everywhere.
#pragma once
#include <stddef.h>

#include "fiedler.h"
#include "fz_state.h"

namespace fz {
// true if every field of u is in its documented range
bool options_valid(const fiedler_options &u);
// device copy of the options for a solve in the FP64 (type 0) or FP32 (type 1) form
void fill_opts(Opts &o, const fiedler_options &u, int type);
// arena bytes the finest level's Krylov refinement takes on top of the
// hierarchy: LOBPCG keeps six more vectors (Lx, w, Lw, p, Lp, D^-1), Lanczos
// its basis of `basis` + 1 vectors, two work vectors and D^-1 (values of
// value_bytes, FP64 on levels of at most kTinyN vertices)
// ... and with the V-cycle preconditioner the aggregate member lists and three
// vectors per level (at most 3n vertices over all levels)
inline size_t refine_bytes(long long n, size_t value_bytes, int refine, int basis, int precond) {
  if (refine == 0) return 0;
  const double v = n <= kTinyN ? 8.0 : (double)value_bytes;
  const double vecs = refine == 1 ? 7.0 : (double)basis + 4.0;
  double b = vecs * (v * (double)n + 256.0) + 4096.0;
  if (refine == 1 && precond == 1) b += 3.0 * (3.0 * 8.0 + 8.0) * (double)n + kMaxLevels * 6.0 * 256.0;
  return (size_t)b;
}
}  // namespace fz
