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
#include <algorithm>
#include <cfloat>
#include <cstring>
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

  // Guide tables for the jump search. The bit patterns of non-negative
  // doubles increase with their values, so key(t) = (bits(G_r(0)) - bits(t))
  // >> shift is a piecewise-linear log of t that grows as t falls (capped
  // at kmax, reached at the smallest positive value of the row). guide[key]
  // = the answer for the largest t of the key's bucket, a lower bound for
  // every t of the bucket; a forward scan from max(st, guide[key]) finds the
  // first j with G_r(j + 1) <= t exactly.
  out.rows.assign(k_max, StrataRow{});
  out.guide.clear();
  const uint64_t target = std::max<uint64_t>(16, 2 * (uint64_t)(S + 1));
  for (uint32_t r = 1; r < K1 && S > 0; r++) {
    const double* g = &out.g[(size_t)(r - 1) * (S + 1)];
    StrataRow& row = out.rows[r - 1];
    row.goff = (uint32_t)out.guide.size();
    uint64_t b0 = 0, bmin = 0;
    std::memcpy(&b0, &g[0], 8);
    bmin = b0;
    for (uint32_t j = 0; j < S; j++)
      if (g[j] > 0.0) std::memcpy(&bmin, &g[j], 8);
    const uint64_t range = b0 - bmin;
    uint32_t shift = 0;
    while ((range >> shift) + 1 > target) shift++;
    const uint64_t kmax = range >> shift;
    row.b = b0;
    row.shift = shift;
    row.kmax = (uint32_t)kmax;
    uint32_t j = 0;
    for (uint64_t k = 0; k <= kmax; k++) {
      const uint64_t vb = b0 - (k << shift);
      double v;
      std::memcpy(&v, &vb, 8);
      while (j < S - 1 && g[j + 1] > v) j++;
      out.guide.push_back(j);
    }
  }
}

}  // namespace nc
