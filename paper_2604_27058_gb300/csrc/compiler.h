// compiler.h — host compiler entry point (product-internal).
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "program.h"

namespace nc {

struct nc_info_counts {
  uint32_t n_static, n_random, n_active, array_ops;
  // bytes per shot the array traversals of Sec. 2.6 move at FP32 (8-byte
  // amplitudes), counted as: an expansion reads 2^k and writes 2^(k+1)
  // amplitudes, a diagonal, 2x2 or permutation pass reads and writes 2^k, an
  // active measurement reads 2^k twice and writes 2^(k-1)
  double array_bytes;
  // the part of array_bytes spent in the shared prefix (program.h prefix_end)
  double prefix_bytes;
};

struct CompiledProgram {
  std::vector<uint8_t> blob;  // ProgHeader + tables (see program.h)
  nc_info_counts counts;
};

// Compile flags (the NC_COMPILE_* bits of nc.h): each turns one HIR pass off.
constexpr uint32_t kNoPeephole = 1u;  // keep rotations whose axis is measured next
constexpr uint32_t kNoReorder = 2u;   // keep measurements and rotations in circuit order
constexpr uint32_t kNoFuse = 4u;      // no phase fusion, cancellation or Clifford re-absorption

// Returns 0 on success or an nc_status code with a message in err.
int compile_program(const std::string& text, uint32_t flags, CompiledProgram& out, std::string& err);

// Appends the record-level propagation tables (program.h) to a blob of a
// program with k_max = 0 (affine.cpp).
void append_affine(std::vector<uint8_t>& blob);

// Appends the fused array-pass instruction list (program.h OP_DIAGF /
// OP_MIXF / OP_PERMF) for the batched executor (fuse.cpp).
void append_fused(std::vector<uint8_t>& blob);

// Stratified importance sampling tables (Sec. 3.2; strata.cpp): for the
// site probabilities p[0..S), g = G_r(j) for r = 1..k_max (row r - 1, n =
// S + 1 entries per row), weight[K] = P(exactly K faults) and valid[K] = 1 if
// stratum K can be sampled (every p < 1, K live sites, no table underflow).
// rows[r - 1] / guide: the guide table of row r (strata.cpp), searched on
// the device by strat_jump (kernels.cuh).
struct StrataRow {
  uint64_t b;           // bit pattern of G_r(0)
  uint32_t shift, kmax;  // key = min(kmax, (b - bits(t)) >> shift)
  uint32_t goff, pad;    // first guide entry of the row
};
static_assert(sizeof(StrataRow) == 24, "StrataRow layout");
struct StrataTables {
  uint32_t k_max = 0, n = 0;
  std::vector<double> g, weight;
  std::vector<uint8_t> valid;
  std::vector<StrataRow> rows;
  std::vector<uint32_t> guide;
};
void build_strata(const double* p, uint32_t S, uint32_t k_max, StrataTables& out);

}  // namespace nc
