// affine_kernel.cu — the sample-many phase for programs without active axes
// (k_max = 0), through the record-level propagation tables that affine.cpp
// derives from the bytecode (program.h).
//
// sample_affine<WPT>: one CTA of 32*WPT threads runs tiles of 32*WPT shots.
// A tile's records live in shared memory as rows x WPT words (bit j of word
// w of a row = shot 32 w + j of the tile; rows padded to WPT + 1 words so
// that different rows of one word fall in different banks):
//   1. the random dormant measurement bits of the tile, m = NOT (top bit of
//      the 128-shot block draw), one Philox call per event and 128 shots;
//   2. every row starts at its constant, the detector / observable reference
//      parity and the XOR of the random bits it depends on (thread per row);
//   3. faults: the tile's chunk items from affine_items, applied with
//      shared-memory atomic XORs; or (when no item list is available) fault
//      sampling in the tile kernel, one warp per 32 shots, one survival-jump
//      draw per lane per step (Sec. 3.2; guide-table search), or one
//      conditional jump per fault for a stratified call (exactly K faults);
//      every fault appends its column's 8-row chunks to the warp's list, and
//      the warp applies a full list one chunk per lane: eight shared-memory
//      atomic XORs of the shot's bit;
//   4. rows kept as differences from a parent row (short fault columns) are
//      turned back into record rows by a running XOR down each chain;
//   5. the tile is written out row by row (16-byte stores when the rows
//      allow), bits of shots past the end cleared, plus the kept row.
// The records equal those of the executors bit for bit: same draws, same
// faults, and the tables are the executors' own frame updates propagated to
// the records once at compile time.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace nc {

constexpr uint32_t kAffTpw = 32;    // threads per 32-shot word of the tile: one warp per word
constexpr uint32_t kAffPool = 32;   // shots per warp (fused sampling): S / warps
constexpr uint32_t kAffList = 128;  // chunk items per warp list

// Chunk range of the fault column of site i with the option that option
// word wz picks (fault record fr = aff_frec[i]).
__device__ __forceinline__ void fault_chunks(const DevProg& p, uint32_t i, uint4 fr, uint32_t wz, uint32_t* c0,
                                             uint32_t* nch) {
  const uint32_t opt = __umulhi(wz, fr.y >> 28);
  if (fr.z != 0xFFFFFFFFu) {
    const uint64_t nib = (uint64_t)fr.x | ((uint64_t)(fr.y & 0x0FFFFFFFu) << 32);
    *nch = (uint32_t)(nib >> (4 * opt)) & 15u;
    uint64_t below = nib & ((1ull << (4 * opt)) - 1ull);
    below = (below & 0x0F0F0F0F0F0F0F0Full) + ((below >> 4) & 0x0F0F0F0F0F0F0F0Full);
    *c0 = fr.z + (uint32_t)((below * 0x0101010101010101ull) >> 56);
  } else {
    const uint32_t c = i * kRecPerSite + opt;
    *c0 = __ldg(p.aff_col_off + c);
    *nch = __ldg(p.aff_col_off + c + 1) - *c0;
  }
}

// One survival-jump draw from site st for `shot` (Sec. 3.2, integer form;
// kernels.cuh jump_draw with the fault record loaded beside each Q[i] of
// the scan). On a fault: *c0 / *nch = its column's chunk range, returns the
// next start site (fault + 1). Otherwise *nch = 0 and returns the segment
// end.
__device__ __forceinline__ uint32_t aff_draw(const DevProg& p, uint2 key, uint64_t shot, uint32_t st, uint32_t* c0,
                                             uint32_t* nch) {
  const uint4 r0 = __ldg(reinterpret_cast<const uint4*>(p.srch) + 2 * st);
  const uint4 r1 = __ldg(reinterpret_cast<const uint4*>(p.srch) + 2 * st + 1);
  const uint4 w = philox(make_uint4((uint32_t)shot, (uint32_t)(shot >> 32), TAG_GAP, st), key);
  const uint64_t u = (uint64_t)w.x | ((uint64_t)w.y << 32);
  const uint64_t q_end = (uint64_t)r1.x | ((uint64_t)r1.y << 32);
  const uint64_t tq = mulhi64(u, (uint64_t)r1.z | ((uint64_t)r1.w << 32));
  *nch = 0;
  if (q_end > tq) return r0.y;
  uint32_t i = __ldg(p.guide + r0.z + guide_key_dev(tq, r0.w));
  uint64_t qi = __ldg(p.q + i);
  uint4 fr = __ldg(p.aff_frec + i);
  while (qi > tq) {
    i++;
    qi = __ldg(p.q + i);
    fr = __ldg(p.aff_frec + i);
  }
  fault_chunks(p, i, fr, w.z, c0, nch);
  return i + 1;
}

// The same for a stratified shot holding r >= 1 faults (kernels.cuh
// strat_jump): always a fault; returns the next start site (fault + 1).
__device__ __forceinline__ uint32_t aff_draw_strat(const DevProg& p, uint2 key, uint64_t shot, uint32_t st,
                                                   uint32_t r, uint32_t* c0, uint32_t* nch) {
  uint32_t wz;
  const uint32_t i = strat_jump(p, key, shot, st, r, &wz);
  fault_chunks(p, i, __ldg(p.aff_frec + i), wz, c0, nch);
  return i + 1;
}

// XOR `bit` into the tile column `col` at the (up to) eight rows of a chunk;
// padding entries (row index R, the scratch row) are skipped.
template <uint32_t STR>
__device__ __forceinline__ void xor_chunk(uint32_t* col, uint4 ch, uint32_t bit, uint32_t R) {
  const uint32_t r[8] = {ch.x & 0xFFFFu, ch.x >> 16, ch.y & 0xFFFFu, ch.y >> 16,
                         ch.z & 0xFFFFu, ch.z >> 16, ch.w & 0xFFFFu, ch.w >> 16};
#pragma unroll
  for (uint32_t e = 0; e < 8; e++)
    if (r[e] < R) atomicXor(col + r[e] * STR, bit);
}

// Warp-inclusive prefix sum.
__device__ __forceinline__ uint32_t warp_incl(uint32_t v, uint32_t lane) {
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += x;
  }
  return v;
}

// affine_items: fault sampling alone, at high occupancy (no record tile).
// One warp per tile of `pool` shots (tile g of the launch = call-local shots
// (tile0 + g) * pool ...), lanes refilled as their shots end; every fault's
// chunk items (chunk << 10 | shot in the tile) go to
// the pool's list items[g * cap ...], and counts[g] receives the number of
// items (a count above cap means the list overflowed).
__global__ void __launch_bounds__(512, 2) affine_items(LaunchParams L, uint32_t pool0, uint32_t n_pools,
                                                       uint32_t* items, uint32_t cap, uint32_t* counts,
                                                       uint32_t pool) {
  const DevProg& p = L.p;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const uint2 key = key_of(L.seed);
  for (uint32_t g = wg; g < n_pools; g += nw) {
    const uint64_t s0 = (uint64_t)(pool0 + g) * pool;  // call-local first shot
    const uint64_t left = s0 < L.shots ? L.shots - s0 : 0;
    const uint32_t n = left < pool ? (uint32_t)left : pool;
    uint32_t* out = items + (size_t)g * cap;
    uint32_t sh = lane, nxt = 32, st = 0, cnt = 0, r = p.sg_k;
    const bool any = p.n_sites > 0 && (!p.sg || p.sg_k > 0);
    bool live = sh < n && any;
    while (__any_sync(0xffffffffu, live)) {
      uint32_t c0 = 0, nch = 0;
      bool fin = false;
      if (live) {
        if (p.sg) {
          st = aff_draw_strat(p, key, L.shot_offset + s0 + sh, st, r, &c0, &nch);
          fin = --r == 0 || st >= p.n_sites;
        } else {
          st = aff_draw(p, key, L.shot_offset + s0 + sh, st, &c0, &nch);
          fin = st >= p.n_sites;
        }
      }
      const uint32_t incl = warp_incl(nch, lane);
      const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
      const uint32_t it0 = sh;
      for (uint32_t j = 0, pos = cnt + incl - nch; j < nch; j++, pos++)
        if (pos < cap) out[pos] = ((c0 + j) << 10) | it0;
      cnt += total;
      const uint32_t done = __ballot_sync(0xffffffffu, fin);
      if (fin) {
        sh = nxt + __popc(done & ((1u << lane) - 1u));
        st = 0;
        r = p.sg_k;
        live = sh < n;
      }
      nxt += __popc(done);
    }
    if (lane == 0) counts[g] = cnt;
  }
}

template <int WPT>
__global__ void __launch_bounds__(kAffTpw * WPT, 65536 / (kAffTpw * WPT * 64)) sample_affine(LaunchParams L) {
  extern __shared__ __align__(16) uint32_t sm[];
  const DevProg& p = L.p;
  constexpr uint32_t S = 32u * WPT, T = kAffTpw * WPT, STR = WPT + 1;
  static_assert(S / (T / 32) == kAffPool, "one fused-sampling pool per warp");
  const uint32_t R = p.aff_rows, NR = p.aff_n_rand, t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  // word offsets, each region 16-byte aligned (MW rows are read as uint4)
  const uint32_t o_mw = ((R + 1) * STR + 3u) & ~3u;
  uint32_t* TILE = sm;                                // (R + 1) rows; row R is scratch
  uint32_t* MW = sm + o_mw;                           // random bits [NR][WPT]
  uint32_t* LW = MW + NR * WPT + warp * kAffList;     // this warp's chunk list
  // per-launch tables staged once: row info (bit 0: constant ^ reference
  // parities of the row and its parent; bits 1..: first random-event entry)
  // and the chains as u16 rows
  uint32_t* RI = MW + NR * WPT + (T / 32) * kAffList;  // [R + 1]
  uint16_t* CH = reinterpret_cast<uint16_t*>(RI + R + 1);                    // [n_chain_rows]
  uint16_t* CHOFF = CH + ((p.aff_n_chain_rows + 1) & ~1u);                  // [n_chains + 1]
  const bool noisy = !(L.flags & LF_NOISELESS) && p.n_sites > 0;
  const uint2 key = key_of(L.seed);
  const uint32_t n_det_end = p.n_meas + p.n_det;

  // eight atomic XORs of one chunk into the column of shot s (tile-local)
  auto apply_chunk = [&](uint32_t chunk, uint32_t s) {
    const uint4 ch = __ldg(p.aff_chunks + chunk);
    uint32_t* col = TILE + (s >> 5);
    const uint32_t bit = 1u << (s & 31u);
    xor_chunk<STR>(col, ch, bit, R);
  };
  // the warp applies its list (at most kAffList = 4 x 32 items), two chunk
  // loads per lane in flight before their atomics
  auto flush = [&](uint32_t n) {
    __syncwarp();
#pragma unroll
    for (uint32_t k0 = 0; k0 < kAffList / 32; k0 += 2) {
      uint4 ch[2];
      uint32_t sh[2];
#pragma unroll
      for (uint32_t u = 0; u < 2; u++) {
        const uint32_t i = lane + 32u * (k0 + u);
        if (i < n) {
          const uint32_t it = LW[i];
          ch[u] = __ldg(p.aff_chunks + (it >> 10));
          sh[u] = it & 1023u;
        }
      }
#pragma unroll
      for (uint32_t u = 0; u < 2; u++)
        if (lane + 32u * (k0 + u) < n) xor_chunk<STR>(TILE + (sh[u] >> 5), ch[u], 1u << (sh[u] & 31u), R);
    }
    __syncwarp();
  };


  {
    auto ref = [&](uint32_t r) -> uint32_t {
      return r < p.n_meas || r >= R ? 0u
             : r < n_det_end       ? __ldg(p.det_ref + (r - p.n_meas))
                                   : __ldg(p.obs_ref + (r - n_det_end));
    };
    for (uint32_t r = t; r <= R; r += T) {
      uint32_t c = 0;
      if (r < R) {
        c = __ldg(p.aff_const + r) ^ ref(r);
        const uint32_t par = __ldg(p.aff_parent + r);
        if (par != 0xFFFFFFFFu) c ^= ref(par);
      }
      RI[r] = (__ldg(p.aff_rowev_off + r) << 1) | (c & 1u);
    }
    for (uint32_t j = t; j < p.aff_n_chain_rows; j += T) CH[j] = (uint16_t)__ldg(p.aff_chain + j);
    for (uint32_t j = t; j <= p.aff_n_chains; j += T) CHOFF[j] = (uint16_t)__ldg(p.aff_chain_off + j);
    __syncthreads();
  }

  for (uint32_t tile = L.tile0 + blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
    const uint64_t tile_s0 = L.shot_offset + (uint64_t)tile * S;  // a multiple of 128
    // pre-sampled chunk items of this tile (affine_items), unless its list
    // overflowed: then the tile samples its faults itself
    const uint32_t* titems = nullptr;
    uint32_t tcnt = 0;
    if (L.aff_items) {
      tcnt = L.aff_counts[tile - L.tile0];
      if (tcnt <= L.aff_cap) titems = L.aff_items + (size_t)(tile - L.tile0) * L.aff_cap;
    }
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
    // 2. constants, reference parities and random-bit terms, four words per thread
    constexpr uint32_t QPR = WPT / 4;  // 4-word quarters per row
    for (uint32_t i = t; i < R * QPR; i += T) {
      const uint32_t r = i / QPR, q = (i % QPR) * 4u;
      const uint32_t ri = RI[r];
      const uint32_t c = (ri & 1u) ? ~0u : 0u;
      const uint32_t e0 = ri >> 1, e1 = RI[r + 1] >> 1;
      uint4 v = make_uint4(c, c, c, c);
      for (uint32_t e = e0; e < e1; e++) {
        const uint4 x = *reinterpret_cast<const uint4*>(MW + __ldg(p.aff_rowev + e) * WPT + q);
        v.x ^= x.x;
        v.y ^= x.y;
        v.z ^= x.z;
        v.w ^= x.w;
      }
      uint32_t* dst = TILE + r * STR + q;
      dst[0] = v.x;
      dst[1] = v.y;
      dst[2] = v.z;
      dst[3] = v.w;
    }
    __syncthreads();
    // 3a. apply the tile's pre-sampled items, two per thread at a time
    if (noisy && titems) {
      const uint32_t n = tcnt;
      for (uint32_t i0 = 0; i0 < n; i0 += 2 * T) {
        uint4 ch[2];
        uint32_t sh[2];
#pragma unroll
        for (uint32_t u = 0; u < 2; u++) {
          const uint32_t i = i0 + u * T + t;
          if (i < n) {
            const uint32_t it = __ldg(titems + i);
            ch[u] = __ldg(p.aff_chunks + (it >> 10));
            sh[u] = it & 1023u;
          }
        }
#pragma unroll
        for (uint32_t u = 0; u < 2; u++)
          if (i0 + u * T + t < n) xor_chunk<STR>(TILE + (sh[u] >> 5), ch[u], 1u << (sh[u] & 31u), R);
      }
    }
    // 3b. otherwise fault sampling with lane refill; chunk items through the warp list
    if (noisy && !titems) {
      const uint64_t pool0 = (uint64_t)tile * S + warp * kAffPool;  // call-local first shot of the pool
      const uint64_t left = pool0 < L.shots ? L.shots - pool0 : 0;
      const uint32_t pool_n = left < kAffPool ? (uint32_t)left : kAffPool;
      uint32_t sh = lane, nxt = 32, st = 0, cnt = 0, r = p.sg_k;
      bool live = sh < pool_n && (!p.sg || p.sg_k > 0);
      while (__any_sync(0xffffffffu, live)) {
        uint32_t c0 = 0, nch = 0;
        bool fin = false;
        if (live) {
          if (p.sg) {
            st = aff_draw_strat(p, key, L.shot_offset + pool0 + sh, st, r, &c0, &nch);
            fin = --r == 0 || st >= p.n_sites;
          } else {
            st = aff_draw(p, key, L.shot_offset + pool0 + sh, st, &c0, &nch);
            fin = st >= p.n_sites;
          }
        }
        // warp prefix of the chunk counts
        const uint32_t incl = warp_incl(nch, lane);
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
          r = p.sg_k;
          live = sh < pool_n;
        }
        nxt += __popc(done);
      }
      flush(cnt);
    }
    __syncthreads();
    // 4. delta rows to record rows: a running XOR down each chain, per word
    for (uint32_t i = t; i < p.aff_n_chains * WPT; i += T) {
      const uint32_t ch = i / WPT, w = i % WPT;
      const uint32_t j0 = CHOFF[ch], j1 = CHOFF[ch + 1];
      uint32_t v = 0, j = j0;
      for (; j + 4 <= j1; j += 4) {  // four rows' loads in flight
        uint32_t* x0 = TILE + CH[j] * STR + w;
        uint32_t* x1 = TILE + CH[j + 1] * STR + w;
        uint32_t* x2 = TILE + CH[j + 2] * STR + w;
        uint32_t* x3 = TILE + CH[j + 3] * STR + w;
        const uint32_t a0 = *x0, a1 = *x1, a2 = *x2, a3 = *x3;
        v ^= a0;
        *x0 = v;
        v ^= a1;
        *x1 = v;
        v ^= a2;
        *x2 = v;
        v ^= a3;
        *x3 = v;
      }
      for (; j < j1; j++) {
        uint32_t* x = TILE + CH[j] * STR + w;
        v ^= *x;
        *x = v;
      }
    }
    __syncthreads();
    // 5. rows out, then the kept row: four words per thread (16-byte stores)
    // when rows are 16-byte aligned (row_words32 % 4 == 0), else two. Shot
    // masks and the row-end check only in the last tile.
    const uint64_t gw0 = (uint64_t)tile * WPT;
    const bool full = (uint64_t)(tile + 1) * S <= L.shots && gw0 + WPT <= L.row_words32;
    auto valid = [&](uint64_t gw) -> uint32_t {
      const uint64_t s0 = gw * 32u;
      return s0 + 32 <= L.shots ? ~0u : s0 < L.shots ? (1u << (uint32_t)(L.shots - s0)) - 1u : 0u;
    };
    // rows [r0, r0 + nr) of the tile to base (kept row: r0 = R, constant)
    auto write_rows = [&](uint32_t* base, uint32_t r0, uint32_t nr) {
      if ((L.row_words32 & 3u) == 0) {
        constexpr uint32_t PR = WPT / 4;
        for (uint32_t i = t; i < nr * PR; i += T) {
          const uint32_t rr = i / PR, w4 = (i % PR) * 4u;
          const uint64_t gw = gw0 + w4;
          uint4 v;
          if (r0 < R) {
            const uint32_t* src = TILE + (r0 + rr) * STR + w4;
            v = make_uint4(src[0], src[1], src[2], src[3]);
          } else {
            v = make_uint4(~0u, ~0u, ~0u, ~0u);
          }
          if (!full) {
            if (gw >= L.row_words32) continue;  // gw + 3 is in range too
            v.x &= valid(gw);
            v.y &= valid(gw + 1);
            v.z &= valid(gw + 2);
            v.w &= valid(gw + 3);
          }
          *reinterpret_cast<uint4*>(base + (size_t)rr * L.row_words32 + gw) = v;
        }
      } else {
        constexpr uint32_t PR = WPT / 2;
        for (uint32_t i = t; i < nr * PR; i += T) {
          const uint32_t rr = i / PR, w2 = (i % PR) * 2u;
          const uint64_t gw = gw0 + w2;
          if (gw >= L.row_words32) continue;  // row_words32 is even
          uint2 v = r0 < R ? make_uint2(TILE[(r0 + rr) * STR + w2], TILE[(r0 + rr) * STR + w2 + 1])
                           : make_uint2(~0u, ~0u);
          v.x &= valid(gw);
          v.y &= valid(gw + 1);
          *reinterpret_cast<uint2*>(base + (size_t)rr * L.row_words32 + gw) = v;
        }
      }
    };
    if (L.flags & LF_OUT_MEAS) write_rows(L.meas, 0, p.n_meas);
    if (L.flags & LF_OUT_DET) write_rows(L.det, p.n_meas, p.n_det);
    if (L.flags & LF_OUT_OBS) write_rows(L.obs, n_det_end, p.n_obs);
    if (L.flags & LF_OUT_KEPT) write_rows(L.kept, R, 1);
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
  const size_t staged = (size_t)p.aff_rows + 1 + ((size_t)p.aff_n_chain_rows + 1) / 2 + ((size_t)p.aff_n_chains + 2) / 2;
  return 4 * (o_mw + (size_t)wpt * p.aff_n_rand + (size_t)(wpt * kAffTpw / 32) * kAffList + staged);
}

template <int WPT>
static cudaError_t aff_one(const LaunchParams& L, uint32_t grid, size_t smem, cudaStream_t st, int* per_sm) {
  auto fn = sample_affine<WPT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, kAffTpw * WPT, smem);
  fn<<<grid, kAffTpw * WPT, smem, st>>>(L);
  return cudaGetLastError();
}

// Item lists for the tiles [tile0, tile0 + n_tiles) of a call.
cudaError_t launch_affine_items(const LaunchParams& L, uint32_t tile0, uint32_t n_tiles, uint32_t* items,
                                uint32_t cap, uint32_t* counts, uint32_t tile_shots, uint32_t grid, cudaStream_t st) {
  affine_items<<<grid, 512, 0, st>>>(L, tile0, n_tiles, items, cap, counts, tile_shots);
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
