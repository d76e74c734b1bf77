// affine_kernel.cu — the sample-many phase for programs without active axes
// (k_max = 0), through the record-level propagation tables that affine.cpp
// derives from the bytecode (program.h).
//
// sample_affine<WPT, QSM>: one CTA of 32*WPT threads runs tiles of 32*WPT
// shots, one thread per shot. A tile's records live in shared memory as
// rows x WPT words (bit j of word w of a row = shot 32 w + j of the tile):
//   1. the random dormant measurement bits of the tile, m = NOT (top bit of
//      the 128-shot block draw), one Philox call per event and 128 shots;
//   2. every row starts at its constant, the detector / observable reference
//      parity and the XOR of the random bits it depends on;
//   3. each thread samples its shot's faults (the survival jump of Sec. 3.2,
//      table staged in shared memory when QSM) and XORs every fault's row
//      list into the tile with shared-memory atomics;
//   4. the tile is written out row by row, 8-byte stores, bits of shots past
//      the end cleared, plus the kept row.
// The records equal those of the executors bit for bit: same draws, same
// faults, and the tables are the executors' own frame updates propagated to
// the records once at compile time.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace nc {

template <int WPT, bool QSM>
__global__ void __launch_bounds__(32 * WPT) sample_affine(LaunchParams L) {
  extern __shared__ __align__(16) uint32_t sm[];
  const DevProg& p = L.p;
  constexpr uint32_t S = 32u * WPT, T = 32u * WPT;
  const uint32_t R = p.aff_rows, NR = p.aff_n_rand, t = threadIdx.x;
  uint64_t* QS = reinterpret_cast<uint64_t*>(sm);
  uint32_t* TILE = sm + (QSM ? 2u * p.n_sites : 0u);
  uint32_t* MW = TILE + (size_t)R * WPT;
  const uint64_t* Q = QSM ? QS : p.q;
  const bool noisy = !(L.flags & LF_NOISELESS) && p.n_sites > 0;
  const uint2 key = key_of(L.seed);
  const uint32_t n_det_end = p.n_meas + p.n_det;
  if (QSM)
    for (uint32_t i = t; i < p.n_sites; i += T) QS[i] = __ldg(p.q + i);

  for (uint32_t tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
    const uint64_t tile_s0 = L.shot_offset + (uint64_t)tile * S;  // a multiple of 128
    // 1. random dormant measurement words
    constexpr uint32_t GR = WPT / 4;  // 128-shot groups per tile
    for (uint32_t i = t; i < NR * GR; i += T) {
      const uint32_t j = i / GR, grp = i % GR;
      const uint64_t g = (tile_s0 >> 7) + grp;
      const uint4 tb = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), TAG_MT, __ldg(p.aff_rand_ev + j)), key);
      uint32_t* dst = MW + j * WPT + grp * 4u;
      dst[0] = ~tb.x;
      dst[1] = ~tb.y;
      dst[2] = ~tb.z;
      dst[3] = ~tb.w;
    }
    __syncthreads();
    // 2. constants, reference parities and random-bit terms
    for (uint32_t i = t; i < R * WPT; i += T) {
      const uint32_t r = i / WPT, w = i % WPT;
      uint32_t c = __ldg(p.aff_const + r);
      if (r >= p.n_meas) c ^= r < n_det_end ? __ldg(p.det_ref + (r - p.n_meas)) : __ldg(p.obs_ref + (r - n_det_end));
      uint32_t v = (c & 1u) ? ~0u : 0u;
      const uint32_t e0 = __ldg(p.aff_rowev_off + r), e1 = __ldg(p.aff_rowev_off + r + 1);
      for (uint32_t e = e0; e < e1; e++) v ^= MW[__ldg(p.aff_rowev + e) * WPT + w];
      TILE[i] = v;
    }
    __syncthreads();
    // 3. this thread's shot: faults and their row lists
    const uint64_t sl = (uint64_t)tile * S + t;  // call-local shot
    if (noisy && sl < L.shots) {
      const uint64_t shot = L.shot_offset + sl;
      const uint32_t w = t >> 5, bit = 1u << (t & 31u);
      uint32_t f = next_fault_tab(p, Q, L.seed, shot, 0);
      while (f != kNoFault) {
        const uint32_t site = f >> 4, c = site * kRecPerSite + (f & 15u);
        const uint32_t j0 = __ldg(p.aff_col_off + c), j1 = __ldg(p.aff_col_off + c + 1);
        for (uint32_t j = j0; j < j1; j++) atomicXor(&TILE[__ldg(p.aff_col + j) * WPT + w], bit);
        f = next_fault_tab(p, Q, L.seed, shot, site + 1);
      }
    }
    __syncthreads();
    // 4. rows out (u64 pairs of words), then the kept row
    constexpr uint32_t PR = WPT / 2;
    const uint64_t gw0 = (uint64_t)tile * WPT;
    for (uint32_t i = t; i < (R + 1) * PR; i += T) {
      const uint32_t r = i / PR, w2 = (i % PR) * 2u;
      const uint64_t gw = gw0 + w2;
      if (gw >= L.row_words32) continue;  // row_words32 is even: gw + 1 is in range too
      uint32_t m[2];
#pragma unroll
      for (uint32_t h = 0; h < 2; h++) {
        const uint64_t s0 = (gw + h) * 32u;
        m[h] = s0 + 32 <= L.shots ? ~0u : s0 < L.shots ? (1u << (uint32_t)(L.shots - s0)) - 1u : 0u;
      }
      uint32_t* dst;
      uint32_t a, b;
      if (r < R) {
        if (r < p.n_meas) {
          if (!(L.flags & LF_OUT_MEAS)) continue;
          dst = L.meas + (size_t)r * L.row_words32;
        } else if (r < n_det_end) {
          if (!(L.flags & LF_OUT_DET)) continue;
          dst = L.det + (size_t)(r - p.n_meas) * L.row_words32;
        } else {
          if (!(L.flags & LF_OUT_OBS)) continue;
          dst = L.obs + (size_t)(r - n_det_end) * L.row_words32;
        }
        a = TILE[r * WPT + w2] & m[0];
        b = TILE[r * WPT + w2 + 1] & m[1];
      } else {
        if (!(L.flags & LF_OUT_KEPT)) continue;
        dst = L.kept;
        a = m[0];
        b = m[1];
      }
      *reinterpret_cast<uint2*>(dst + gw) = make_uint2(a, b);
    }
    if (t == 0 && (uint64_t)tile * S < L.shots) {
      const uint64_t left = L.shots - (uint64_t)tile * S;
      atomicAdd(L.kept_count, (unsigned long long)(left < S ? left : S));
    }
    __syncthreads();
  }
}

// Shared memory of one CTA: staged survival table (QSM), the record tile and
// the random-bit words.
size_t affine_smem_bytes(const DevProg& p, uint32_t wpt, bool qsm) {
  return (qsm ? (size_t)p.n_sites * 8 : 0) + (size_t)wpt * 4 * ((size_t)p.aff_rows + p.aff_n_rand);
}

template <int WPT, bool QSM>
static cudaError_t aff_one(const LaunchParams& L, uint32_t grid, size_t smem, cudaStream_t st, int* per_sm) {
  auto fn = sample_affine<WPT, QSM>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, 32 * WPT, smem);
  fn<<<grid, 32 * WPT, smem, st>>>(L);
  return cudaGetLastError();
}

template <bool QSM>
static cudaError_t aff_w(const LaunchParams& L, uint32_t wpt, uint32_t grid, size_t smem, cudaStream_t st,
                         int* per_sm) {
  switch (wpt) {
    case 4: return aff_one<4, QSM>(L, grid, smem, st, per_sm);
    case 8: return aff_one<8, QSM>(L, grid, smem, st, per_sm);
    case 16: return aff_one<16, QSM>(L, grid, smem, st, per_sm);
    case 32: return aff_one<32, QSM>(L, grid, smem, st, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

// per_sm != null: report resident CTAs per SM instead of launching.
cudaError_t launch_affine(const LaunchParams& L, uint32_t wpt, bool qsm, uint32_t grid, size_t smem,
                          cudaStream_t st, int* per_sm) {
  return qsm ? aff_w<true>(L, wpt, grid, smem, st, per_sm) : aff_w<false>(L, wpt, grid, smem, st, per_sm);
}

}  // namespace nc
