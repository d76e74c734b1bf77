// strata.cpp — tables of stratified importance sampling (host).
//
// Sec. 3.2 runs rare-event estimates in strata of a fixed number K of
// realised faults: stratum K is weighted by P(K faults), the
// Poisson-binomial mass of the site probabilities p_i, and each of its shots
// forces exactly K sites to fire, drawn from
//   P(F | |F| = K) = prod_{i in F} p_i prod_{i not in F} (1 - p_i) / P(K).
// The shots draw F by K conditional jumps over the sites:
//   R[j][r] = P(exactly r faults among sites j..S-1)
//           = (1 - p_j) R[j + 1][r] + p_j R[j + 1][r - 1],  R[S][r] = [r = 0];
//   W[j]    = prod_{l < j} (1 - p_l);
//   G_r(j)  = W[j] R[j][r]  (sites before j quiet, r faults from j on),
// stored as the running minimum over l <= j so that it never increases in
// floating point either. Holding r faults at site st, a shot draws u in
// [0, 1) and puts the next fault at the first j >= st with
// G_r(j + 1) <= u G_r(st); the search resumes at j + 1 with r - 1. The
// weights are R[0][K].
//
// Every value is one IEEE operation in a fixed order (products rounded, then
// sums; this file is built without floating-point contraction), so the
// tables are reproducible bit for bit.
#include <cfloat>
#include <vector>

#include "compiler.h"

namespace nc {

void build_strata(const double* p, uint32_t S, uint32_t k_max, StrataTables& out) {
  const uint32_t K1 = k_max + 1;
  std::vector<double> R((size_t)(S + 1) * K1, 0.0);  // R[j * K1 + r]
  R[(size_t)S * K1] = 1.0;
  for (uint32_t j = S; j-- > 0;) {
    const double pj = p[j], q = 1.0 - pj;
    const double* nx = &R[(size_t)(j + 1) * K1];
    double* cur = &R[(size_t)j * K1];
    cur[0] = q * nx[0];
    for (uint32_t r = 1; r < K1; r++) {
      const double a = q * nx[r];
      const double b = pj * nx[r - 1];
      cur[r] = a + b;
    }
  }
  std::vector<double> W(S + 1);
  W[0] = 1.0;
  for (uint32_t j = 0; j < S; j++) W[j + 1] = W[j] * (1.0 - p[j]);
  std::vector<uint32_t> live(S + 1, 0);
  bool certain = false;
  for (uint32_t j = S; j-- > 0;) {
    live[j] = live[j + 1] + (p[j] > 0.0 ? 1u : 0u);
    if (p[j] >= 1.0) certain = true;
  }
  out.k_max = k_max;
  out.n = S + 1;
  out.g.assign((size_t)k_max * (S + 1), 0.0);
  out.weight.assign(K1, 0.0);
  out.valid.assign(K1, 0);
  for (uint32_t r = 0; r < K1; r++) out.weight[r] = R[r];
  // first r whose table has a value that should be positive but is not a
  // normal number: strata from r on cannot be sampled exactly
  uint32_t bad_from = K1;
  for (uint32_t r = 1; r < K1; r++) {
    double* g = &out.g[(size_t)(r - 1) * (S + 1)];
    double run = 0.0;
    for (uint32_t j = 0; j <= S; j++) {
      const double v = W[j] * R[(size_t)j * K1 + r];
      run = (j == 0 || v < run) ? v : run;
      g[j] = run;
      if (live[j] >= r && !(run >= DBL_MIN) && bad_from == K1) bad_from = r;
    }
  }
  for (uint32_t K = 0; K < K1; K++) out.valid[K] = (!certain && K <= live[0] && K < bad_from) ? 1 : 0;
}

}  // namespace nc
