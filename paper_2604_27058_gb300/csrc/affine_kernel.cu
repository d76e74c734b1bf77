// affine_kernel.cu — the sample-many phase for programs without active axes
// (k_max = 0), through the record-level propagation tables that affine.cpp
// derives from the bytecode (program.h).
//
// sample_affine<WPT>: one CTA of 16*WPT threads runs tiles of 32*WPT shots.
// A tile's records live in shared memory as rows x WPT words (bit j of word
// w of a row = shot 32 w + j of the tile; rows padded to WPT + 1 words so
// that different rows of one word fall in different banks):
//   1. the random dormant measurement bits of the tile, m = NOT (top bit of
//      the 128-shot block draw), one Philox call per event and 128 shots;
//   2. every row starts at its constant, the detector / observable reference
//      parity and the XOR of the random bits it depends on (thread per row);
//   3. fault sampling: each warp owns 64 shots and keeps its 32 lanes busy
//      by handing a finished lane the next shot, one survival-jump draw per
//      lane per step (Sec. 3.2; guide-table search of the survival table);
//      every fault appends its column's 8-row chunks to the warp's list, and
//      the warp applies a full list one chunk per lane: eight shared-memory
//      atomic XORs of the shot's bit;
//   4. the tile is written out row by row, bits of shots past the end
//      cleared, plus the kept row.
// The records equal those of the executors bit for bit: same draws, same
// faults, and the tables are the executors' own frame updates propagated to
// the records once at compile time.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace nc {

constexpr uint32_t kAffPool = 64;   // shots per warp
constexpr uint32_t kAffList = 128;  // chunk items per warp list

template <int WPT>
__global__ void __launch_bounds__(16 * WPT) sample_affine(LaunchParams L) {
  extern __shared__ __align__(16) uint32_t sm[];
  const DevProg& p = L.p;
  constexpr uint32_t S = 32u * WPT, T = 16u * WPT, STR = WPT + 1;
  const uint32_t R = p.aff_rows, NR = p.aff_n_rand, t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  // word offsets, each region 16-byte aligned (MW rows are read as uint4)
  const uint32_t o_mw = ((R + 1) * STR + 3u) & ~3u;
  uint32_t* TILE = sm;                                // (R + 1) rows; row R is scratch
  uint32_t* MW = sm + o_mw;                           // random bits [NR][WPT]
  uint32_t* LW = MW + NR * WPT + warp * kAffList;     // this warp's chunk list
  const bool noisy = !(L.flags & LF_NOISELESS) && p.n_sites > 0;
  const uint2 key = key_of(L.seed);
  const uint32_t n_det_end = p.n_meas + p.n_det;

  // eight atomic XORs of one chunk into the column of shot s (tile-local)
  auto apply_chunk = [&](uint32_t chunk, uint32_t s) {
    const uint4 ch = __ldg(p.aff_chunks + chunk);
    uint32_t* col = TILE + (s >> 5);
    const uint32_t bit = 1u << (s & 31u);
    atomicXor(col + (ch.x & 0xFFFFu) * STR, bit);
    atomicXor(col + (ch.x >> 16) * STR, bit);
    atomicXor(col + (ch.y & 0xFFFFu) * STR, bit);
    atomicXor(col + (ch.y >> 16) * STR, bit);
    atomicXor(col + (ch.z & 0xFFFFu) * STR, bit);
    atomicXor(col + (ch.z >> 16) * STR, bit);
    atomicXor(col + (ch.w & 0xFFFFu) * STR, bit);
    atomicXor(col + (ch.w >> 16) * STR, bit);
  };
  // the warp applies its list, one item per lane
  auto flush = [&](uint32_t n) {
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32) {
      const uint32_t it = LW[i];
      apply_chunk(it >> 10, it & 1023u);
    }
    __syncwarp();
  };

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
    // 2. constants, reference parities and random-bit terms, one row per thread
    for (uint32_t r = t; r < R; r += T) {
      uint32_t c = __ldg(p.aff_const + r);
      if (r >= p.n_meas) c ^= r < n_det_end ? __ldg(p.det_ref + (r - p.n_meas)) : __ldg(p.obs_ref + (r - n_det_end));
      uint32_t v[WPT];
#pragma unroll
      for (uint32_t w = 0; w < WPT; w++) v[w] = (c & 1u) ? ~0u : 0u;
      const uint32_t e0 = __ldg(p.aff_rowev_off + r), e1 = __ldg(p.aff_rowev_off + r + 1);
      for (uint32_t e = e0; e < e1; e++) {
        const uint4* mw = reinterpret_cast<const uint4*>(MW + __ldg(p.aff_rowev + e) * WPT);
#pragma unroll
        for (uint32_t w4 = 0; w4 < WPT / 4; w4++) {
          const uint4 x = mw[w4];
          v[4 * w4] ^= x.x;
          v[4 * w4 + 1] ^= x.y;
          v[4 * w4 + 2] ^= x.z;
          v[4 * w4 + 3] ^= x.w;
        }
      }
#pragma unroll
      for (uint32_t w = 0; w < WPT; w++) TILE[r * STR + w] = v[w];
    }
    __syncthreads();
    // 3. fault sampling with lane refill; chunk items through the warp list
    if (noisy) {
      const uint64_t pool0 = (uint64_t)tile * S + warp * kAffPool;  // call-local first shot of the pool
      const uint64_t left = pool0 < L.shots ? L.shots - pool0 : 0;
      const uint32_t pool_n = left < kAffPool ? (uint32_t)left : kAffPool;
      uint32_t sh = lane, nxt = 32, st = 0, cnt = 0;
      bool live = sh < pool_n;
      while (__any_sync(0xffffffffu, live)) {
        uint32_t c0 = 0, nch = 0;
        bool fin = false;
        if (live) {
          const uint64_t shot = L.shot_offset + pool0 + sh;
          uint4 w;
          const uint32_t i = jump_draw(p, key, shot, st, &w, &st);
          if (i != kNoFault) {
            const uint32_t kk = (__ldg(p.site_info + i) >> 4) & 15u;
            const uint32_t c = i * kRecPerSite + __umulhi(w.z, kk);
            c0 = __ldg(p.aff_col_off + c);
            nch = __ldg(p.aff_col_off + c + 1) - c0;
            st = i + 1;
          }
          fin = st >= p.n_sites;
        }
        // warp prefix of the chunk counts
        uint32_t incl = nch;
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
          const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += v;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t s_tile = warp * kAffPool + sh;
        if (cnt + total > kAffList) {
          flush(cnt);
          cnt = 0;
        }
        if (total > kAffList) {
          for (uint32_t j = 0; j < nch; j++) apply_chunk(c0 + j, s_tile);
        } else {
          for (uint32_t j = 0, pos = cnt + incl - nch; j < nch; j++, pos++) LW[pos] = ((c0 + j) << 10) | s_tile;
          cnt += total;
        }
        // hand finished lanes the next shots of the pool
        const uint32_t done = __ballot_sync(0xffffffffu, fin);
        if (fin) {
          sh = nxt + __popc(done & ((1u << lane) - 1u));
          st = 0;
          live = sh < pool_n;
        }
        nxt += __popc(done);
      }
      flush(cnt);
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
        a = TILE[r * STR + w2] & m[0];
        b = TILE[r * STR + w2 + 1] & m[1];
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

// Shared memory of one CTA: the record tile
// (with its scratch row and padding word), the random-bit words and one
// chunk list per warp.
size_t affine_smem_bytes(const DevProg& p, uint32_t wpt) {
  const size_t o_mw = ((size_t)(wpt + 1) * (p.aff_rows + 1) + 3) & ~(size_t)3;
  return 4 * (o_mw + (size_t)wpt * p.aff_n_rand + (size_t)(wpt / 2) * kAffList);
}

template <int WPT>
static cudaError_t aff_one(const LaunchParams& L, uint32_t grid, size_t smem, cudaStream_t st, int* per_sm) {
  auto fn = sample_affine<WPT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, 16 * WPT, smem);
  fn<<<grid, 16 * WPT, smem, st>>>(L);
  return cudaGetLastError();
}

// per_sm != null: report resident CTAs per SM instead of launching.
cudaError_t launch_affine(const LaunchParams& L, uint32_t wpt, uint32_t grid, size_t smem, cudaStream_t st,
                          int* per_sm) {
  switch (wpt) {
    case 8: return aff_one<8>(L, grid, smem, st, per_sm);
    case 16: return aff_one<16>(L, grid, smem, st, per_sm);
    case 32: return aff_one<32>(L, grid, smem, st, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace nc
