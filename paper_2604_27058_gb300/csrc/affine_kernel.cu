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

template <bool B>
struct Flag {
  static constexpr bool value = B;
};

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
// padding entries (row index R) go to `dump`, a word of the caller's that
// nothing reads, so that every entry is one unconditional atomic.
template <uint32_t STR>
__device__ __forceinline__ void xor_chunk(uint32_t* col, uint4 ch, uint32_t bit, uint32_t R, uint32_t* dump) {
  const uint32_t r[8] = {ch.x & 0xFFFFu, ch.x >> 16, ch.y & 0xFFFFu, ch.y >> 16,
                         ch.z & 0xFFFFu, ch.z >> 16, ch.w & 0xFFFFu, ch.w >> 16};
#pragma unroll
  for (uint32_t e = 0; e < 8; e++) atomicXor(r[e] < R ? col + r[e] * STR : dump, bit);
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

// Fault items of the tile kernel: (chunk << 10) | shot in the tile, one per
// 8-row chunk of a fault's column (about one per fault for the surface code),
// so that applying a list is one chunk per lane with no loop; chunks below
// 2^22.
__device__ __forceinline__ uint32_t chunk_item(uint32_t chunk, uint32_t shot) { return (chunk << 10) | shot; }

// affine_items: fault sampling alone, at high occupancy (no record tile).
// One warp per tile of `pool` shots (tile g of the launch = call-local shots
// (tile0 + g) * pool ...), lanes refilled as their shots end; every fault's
// item goes to the pool's list items[g * cap ...], and counts[g] receives
// the number of items (a count above cap means the list overflowed).
template <int MINB>
__global__ void __launch_bounds__(512, MINB) affine_items(LaunchParams L, uint32_t pool0, uint32_t n_pools,
                                                          uint32_t* items, uint32_t cap, uint32_t* counts,
                                                          uint32_t pool) {
  const DevProg& p = L.p;
  const uint32_t lane = threadIdx.x & 31u, lt = (1u << lane) - 1u;
  const uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  const uint2 key = key_of(L.seed);
  for (uint32_t g = wg; g < n_pools; g += nw) {
    const uint64_t s0 = (uint64_t)(pool0 + g) * pool;  // call-local first shot
    const uint64_t left = s0 < L.shots ? L.shots - s0 : 0;
    const uint32_t n = left < pool ? (uint32_t)left : pool;
    const uint64_t base = L.shot_offset + s0;  // global first shot
    uint32_t* out = items + (size_t)g * cap;
    // lane slot sh -> tile-local shot: in a full tile (sh mod W) * 32 + sh / W
    // with W = pool / 32 words, so that consecutive items (one per live
    // lane) name different 32-shot words of the tile and the tile kernel's
    // atomics on them fall in different banks; the identity in a ragged tile
    const uint32_t wpool = pool >> 5, wshift = __ffs(wpool) - 1;  // pool = 32 * 2^wshift
    const bool spread = n == pool;
    uint32_t sh = lane, nxt = 32, st = 0, cnt = 0, r = p.sg_k;
    const bool any = p.n_sites > 0 && (!p.sg || p.sg_k > 0);
    bool live = sh < n && any;
    while (__any_sync(0xffffffffu, live)) {
      uint32_t c0 = 0, nch = 0;
      bool fin = false;
      const uint32_t it0 = spread ? ((sh & (wpool - 1u)) << 5) | (sh >> wshift) : sh;
      if (live) {
        if (p.sg) {
          st = aff_draw_strat(p, key, base + it0, st, r, &c0, &nch);
          fin = --r == 0 || st >= p.n_sites;
        } else {
          st = aff_draw(p, key, base + it0, st, &c0, &nch);
          fin = st >= p.n_sites;
        }
      }
      // one item per chunk, placed by ballot: every lane's first chunk, then
      // one round per further chunk of the (rare) multi-chunk faults
      for (uint32_t c = 0;; c++) {
        const uint32_t has = __ballot_sync(0xffffffffu, nch > c);
        if (!has) break;
        const uint32_t pos = cnt + __popc(has & lt);
        if (nch > c && pos < cap) out[pos] = chunk_item(c0 + c, it0);
        cnt += __popc(has);
      }
      const uint32_t done = __ballot_sync(0xffffffffu, fin);
      if (fin) {
        sh = nxt + __popc(done & lt);
        st = 0;
        r = p.sg_k;
        live = sh < n;
      }
      nxt += __popc(done);
    }
    if (lane == 0) counts[g] = cnt;
  }
}

// Fault sampling inside the tile kernel (no item list for the tile): lane
// refill over the warp's 32 shots, chunk items through the warp's list LW,
// applied to TILE with atomic XORs. The warp's shots are tile-local warp,
// warp + WPT, warp + 2 WPT, ...: one per 32-shot word (WPT = 32), so the
// atomics of one list pass fall in different banks. Kept out of line so
// that its registers do not crowd the rest of the kernel.
template <int WPT>
__device__ __noinline__ void sample_tile_faults(const LaunchParams& L, uint32_t* TILE, uint32_t* LW, uint32_t* dump,
                                                uint32_t tile, uint32_t lane, uint32_t warp) {
  const DevProg& p = L.p;
  constexpr uint32_t S = 32u * WPT;
  const uint32_t R = p.aff_rows;
  const uint2 key = key_of(L.seed);
  const uint64_t tile_s0 = L.shot_offset + (uint64_t)tile * S;
  const uint64_t base = (uint64_t)tile * S;  // call-local first shot of the tile
  const uint64_t left = base < L.shots ? L.shots - base : 0;
  const uint32_t n_tile = left < S ? (uint32_t)left : S;
  const uint32_t pool_n = n_tile > warp ? min(kAffPool, (n_tile - warp + WPT - 1) / WPT) : 0u;
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
        if (lane + 32u * (k0 + u) < n) xor_chunk<WPT>(TILE + (sh[u] >> 5), ch[u], 1u << (sh[u] & 31u), R, dump);
    }
    __syncwarp();
  };
  uint32_t sh = lane, nxt = 32, st = 0, cnt = 0, r = p.sg_k;
  bool live = sh < pool_n && (!p.sg || p.sg_k > 0);
  while (__any_sync(0xffffffffu, live)) {
    uint32_t c0 = 0, nch = 0;
    bool fin = false;
    const uint32_t s_tile = sh * WPT + warp;
    if (live) {
      if (p.sg) {
        st = aff_draw_strat(p, key, tile_s0 + s_tile, st, r, &c0, &nch);
        fin = --r == 0 || st >= p.n_sites;
      } else {
        st = aff_draw(p, key, tile_s0 + s_tile, st, &c0, &nch);
        fin = st >= p.n_sites;
      }
    }
    // warp prefix of the chunk counts
    const uint32_t incl = warp_incl(nch, lane);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (cnt + total > kAffList) {
      flush(cnt);
      cnt = 0;
    }
    if (total > kAffList) {
      for (uint32_t j = 0; j < nch; j++)
        xor_chunk<WPT>(TILE + (s_tile >> 5), __ldg(p.aff_chunks + c0 + j), 1u << (s_tile & 31u), R, dump);
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

template <int WPT>
__global__ void __launch_bounds__(kAffTpw * WPT, 65536 / (kAffTpw * WPT * 64)) sample_affine(LaunchParams L) {
  extern __shared__ __align__(16) uint32_t sm[];
  const DevProg& p = L.p;
  constexpr uint32_t S = 32u * WPT, T = kAffTpw * WPT, NWARP = T / 32;
  constexpr uint32_t QPL = WPT / 4;   // lanes per row in the output pass, one 16-byte quad each
  constexpr uint32_t CPW = 32 / QPL;  // chains one warp resolves side by side
  static_assert(S / NWARP == kAffPool, "one fused-sampling pool per warp");
  const uint32_t R = p.aff_rows, NR = p.aff_n_rand, t = threadIdx.x, lane = t & 31u, warp = t >> 5;
  // word offsets; every region 16-byte aligned (WPT is a multiple of 4)
  uint32_t* TILE = sm;                                // R rows of WPT words, zero between tiles
  uint32_t* MW = sm + R * WPT;                        // random bits [NR][WPT]
  uint32_t* LW = MW + NR * WPT + warp * kAffList;     // this warp's chunk list
  // per-launch tables staged once, by chain position j (the tile keeps row
  // chain[j] at position j): the output row (null: not written), row info
  // (bit 0: constant ^ reference parities of the row and its parent; bits
  // 1..7: its number of random-bit terms; bits 8..: its first term), each
  // warp's range of single-row steps, and the chain offsets
  uint32_t** ROWP = reinterpret_cast<uint32_t**>(MW + NR * WPT + NWARP * kAffList);  // [R]
  uint32_t* RI = reinterpret_cast<uint32_t*>(ROWP + R);  // [R]
  uint32_t* SR = RI + R;                                 // [NWARP + 2]
  uint32_t* dump = SR + NWARP + 2 + lane;                // [32]: padding entries' atomics
  uint16_t* CHOFF = reinterpret_cast<uint16_t*>(SR + NWARP + 2 + 32);  // [n_chains + 1]
  const bool noisy = !(L.flags & LF_NOISELESS) && p.n_sites > 0;
  const uint2 key = key_of(L.seed);
  const uint32_t n_det_end = p.n_meas + p.n_det;

  {
    auto ref = [&](uint32_t r) -> uint32_t {
      return r < p.n_meas || r >= R ? 0u
             : r < n_det_end       ? __ldg(p.det_ref + (r - p.n_meas))
                                   : __ldg(p.obs_ref + (r - n_det_end));
    };
    for (uint32_t j = t; j < R; j += T) {
      const uint32_t r = __ldg(p.aff_chain + j);
      uint32_t c = __ldg(p.aff_const + r) ^ ref(r);
      const uint32_t par = __ldg(p.aff_parent + r);
      if (par != 0xFFFFFFFFu) c ^= ref(par);
      const uint32_t e0 = __ldg(p.aff_rowev_off + r), ne = __ldg(p.aff_rowev_off + r + 1) - e0;
      RI[j] = (e0 << 8) | (ne << 1) | (c & 1u);
      uint32_t* dst = nullptr;
      if (r < p.n_meas) {
        if (L.flags & LF_OUT_MEAS) dst = L.meas + (size_t)r * L.row_words32;
      } else if (r < n_det_end) {
        if (L.flags & LF_OUT_DET) dst = L.det + (size_t)(r - p.n_meas) * L.row_words32;
      } else if (L.flags & LF_OUT_OBS) {
        dst = L.obs + (size_t)(r - n_det_end) * L.row_words32;
      }
      ROWP[j] = dst;
    }
    for (uint32_t j = t; j <= p.aff_n_chains; j += T) CHOFF[j] = (uint16_t)__ldg(p.aff_chain_off + j);
    for (uint32_t i = t; i < R * (WPT / 4); i += T) reinterpret_cast<uint4*>(TILE)[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    // Work split of the output pass. Chains of two or more rows (the first
    // n_long, longest first) are walked CPW at a time per warp, one row per
    // step; the single rows after them are cut into steps of CPW rows, and
    // warp w takes the steps [SR[w], SR[w + 1]), sized so that every warp
    // has about the same number of steps in all.
    if (warp == 0) {
      // lane w < NWARP: warp w's chain steps; n_long by a search over the
      // chain lengths (non-increasing)
      uint32_t lo = 0, hi = p.aff_n_chains;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) / 2;
        if (CHOFF[mid + 1] - CHOFF[mid] >= 2) lo = mid + 1;
        else hi = mid;
      }
      const uint32_t n_long = lo;
      // warp w walks the chains w * CPW + cw (+ k NWARP CPW) side by side: its
      // chain steps are the lengths of the first chain of each such group
      // (chains are longest first)
      uint32_t cs = 0;
      if (lane < NWARP)
        for (uint32_t c = lane * CPW; c < n_long; c += NWARP * CPW) cs += CHOFF[c + 1] - CHOFF[c];
      const uint32_t n_ss = (R - CHOFF[n_long] + CPW - 1) / CPW;
      uint32_t tot = cs;
      for (uint32_t d = 16; d; d >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, d);
      uint32_t target = (tot + n_ss + NWARP - 1) / NWARP;
      uint32_t quota = 0;
      for (;; target++) {
        quota = lane < NWARP && cs < target ? target - cs : 0u;
        uint32_t room = quota;
        for (uint32_t d = 16; d; d >>= 1) room += __shfl_xor_sync(0xffffffffu, room, d);
        if (room >= n_ss) break;
      }
      const uint32_t incl = warp_incl(quota, lane);
      if (lane < NWARP) SR[lane] = min(n_ss, incl - quota);
      if (lane == 0) {
        SR[NWARP] = n_ss;
        SR[NWARP + 1] = n_long;
      }
    }
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
      *reinterpret_cast<uint4*>(MW + j * WPT + grp * 4u) = make_uint4(~tb.x, ~tb.y, ~tb.z, ~tb.w);
    }
    // 2. faults into the zeroed tile: pre-sampled items, one chunk per lane,
    // two chunk loads in flight before their atomics
    if (noisy && titems) {
      uint32_t i = t;
      for (; i + T < tcnt; i += 2 * T) {
        const uint32_t ia = __ldg(titems + i), ib = __ldg(titems + i + T);
        const uint4 ca = __ldg(p.aff_chunks + (ia >> 10)), cb = __ldg(p.aff_chunks + (ib >> 10));
        xor_chunk<WPT>(TILE + ((ia & 1023u) >> 5), ca, 1u << (ia & 31u), R, dump);
        xor_chunk<WPT>(TILE + ((ib & 1023u) >> 5), cb, 1u << (ib & 31u), R, dump);
      }
      if (i < tcnt) {
        const uint32_t ia = __ldg(titems + i);
        xor_chunk<WPT>(TILE + ((ia & 1023u) >> 5), __ldg(p.aff_chunks + (ia >> 10)), 1u << (ia & 31u), R, dump);
      }
    }
    // otherwise fault sampling in the tile kernel
    if (noisy && !titems) sample_tile_faults<WPT>(L, TILE, LW, dump, tile, lane, warp);
    __syncthreads();
    // 3. the output pass. Each delta row is read and zeroed for the next
    // tile, its constant and random-bit terms are added, the XOR down its
    // chain turns it into its record row, which goes straight to HBM. QPL
    // lanes cover a row (16-byte quads); a warp holds CPW row slots.
    const uint64_t gw0 = (uint64_t)tile * WPT;
    const bool full = (uint64_t)(tile + 1) * S <= L.shots && gw0 + WPT <= L.row_words32;
    const bool fast = full && (L.row_words32 & 3u) == 0;
    auto valid = [&](uint64_t gw) -> uint32_t {
      const uint64_t s0 = gw * 32u;
      return s0 + 32 <= L.shots ? ~0u : s0 < L.shots ? (1u << (uint32_t)(L.shots - s0)) - 1u : 0u;
    };
    // the quad v of a record row at words gw .. gw + 3 of dst (rows are
    // 8-byte aligned; 16-byte stores when row_words32 % 4 == 0). FAST (a
    // full tile, rows of a multiple of 4 words): the plain 16-byte store; the
    // output pass below is instantiated for both, so a full tile's loop
    // carries no ragged-edge code.
    auto put_any = [&](auto fast_tag, uint32_t* dst, uint64_t gw, uint4 v) {
      if constexpr (decltype(fast_tag)::value) {
        *reinterpret_cast<uint4*>(dst) = v;
      } else {
        if (gw >= L.row_words32) return;  // row_words32 is even: gw + 1 is out too
        v.x &= valid(gw);
        v.y &= valid(gw + 1);
        v.z &= valid(gw + 2);
        v.w &= valid(gw + 3);
        if ((L.row_words32 & 3u) == 0) {
          *reinterpret_cast<uint4*>(dst) = v;
        } else {
          *reinterpret_cast<uint2*>(dst) = make_uint2(v.x, v.y);
          if (gw + 2 < L.row_words32) *reinterpret_cast<uint2*>(dst + 2) = make_uint2(v.z, v.w);
        }
      }
    };
    auto out_pass = [&](auto fast_tag) {
      const uint32_t qd = lane % QPL, cw = lane / QPL;
      const uint64_t gw = gw0 + 4u * qd;
      // the delta at position j with its row's constant and random-bit
      // terms added (x: the tile's cell, already read; the cell is cleared)
      auto term = [&](uint32_t j, uint4 x) -> uint4 {
        const uint32_t ri = RI[j];
        const uint32_t cm = 0u - (ri & 1u);
        x.x ^= cm;
        x.y ^= cm;
        x.z ^= cm;
        x.w ^= cm;
        const uint32_t ne = (ri >> 1) & 127u;
        for (uint32_t e = ri >> 8, e1 = (ri >> 8) + ne; e < e1; e++) {
          const uint4 m = *reinterpret_cast<const uint4*>(MW + __ldg(p.aff_rowev + e) * WPT + 4u * qd);
          x.x ^= m.x;
          x.y ^= m.y;
          x.z ^= m.z;
          x.w ^= m.w;
        }
        return x;
      };
      auto cell = [&](uint32_t j) -> uint4* { return reinterpret_cast<uint4*>(TILE + j * WPT) + qd; };
      auto emit = [&](uint32_t j, uint4 v) {
        uint32_t* dst = ROWP[j];
        if (dst) put_any(fast_tag, dst + gw, gw, v);
      };
      const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
      // chains of two or more rows: lane slot cw of warp w walks chain
      // w * CPW + cw + k * NWARP * CPW down its positions, keeping the running
      // XOR of the deltas
      const uint32_t n_long = SR[NWARP + 1];
      for (uint32_t c = warp * CPW + cw; c < n_long; c += NWARP * CPW) {
        const uint32_t j1 = CHOFF[c + 1];
        uint4 v = zero;
        for (uint32_t j = CHOFF[c]; j < j1; j++) {
          const uint4 x = term(j, *cell(j));
          *cell(j) = zero;
          v.x ^= x.x;
          v.y ^= x.y;
          v.z ^= x.z;
          v.w ^= x.w;
          emit(j, v);
        }
      }
      // rows on no chain: CPW of them per step, this warp's steps, two steps
      // per pass (both cells read before either is cleared)
      {
        const uint32_t j0 = CHOFF[n_long] + cw, q1 = SR[warp + 1];
        uint32_t q = SR[warp];
        for (; q + 2 <= q1; q += 2) {
          const uint32_t ja = j0 + q * CPW, jb = ja + CPW;
          const bool oa = ja < R, ob = jb < R;
          uint4 xa = zero, xb = zero;
          if (oa) xa = *cell(ja);
          if (ob) xb = *cell(jb);
          if (oa) *cell(ja) = zero;
          if (ob) *cell(jb) = zero;
          if (oa) emit(ja, term(ja, xa));
          if (ob) emit(jb, term(jb, xb));
        }
        if (q < q1) {
          const uint32_t j = j0 + q * CPW;
          if (j < R) {
            const uint4 x = *cell(j);
            *cell(j) = zero;
            emit(j, term(j, x));
          }
        }
      }
    };
    if (fast) out_pass(Flag<true>{});
    else out_pass(Flag<false>{});
    {
      // the kept row: every shot of the tile
      if ((L.flags & LF_OUT_KEPT) && t < QPL) {
        if (fast) put_any(Flag<true>{}, L.kept + gw0 + 4u * t, gw0 + 4u * t, make_uint4(~0u, ~0u, ~0u, ~0u));
        else put_any(Flag<false>{}, L.kept + gw0 + 4u * t, gw0 + 4u * t, make_uint4(~0u, ~0u, ~0u, ~0u));
      }
    }
    if (t == 0 && (uint64_t)tile * S < L.shots) {
      const uint64_t left = L.shots - (uint64_t)tile * S;
      atomicAdd(L.kept_count, (unsigned long long)(left < S ? left : S));
    }
    __syncthreads();
  }
}

// Shared memory of one CTA: the record tile, the random-bit words, one
// chunk list per warp, the output row pointers, row info, the warps' step
// ranges, 32 dump words and the chain offsets.
size_t affine_smem_bytes(const DevProg& p, uint32_t wpt) {
  const size_t R = p.aff_rows, nwarp = wpt * kAffTpw / 32;
  const size_t staged = 2 * R + R + (nwarp + 2) + 32 + ((size_t)p.aff_n_chains + 2) / 2;
  return 4 * (R * wpt + (size_t)wpt * p.aff_n_rand + nwarp * kAffList + staged);
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

// Item lists for the tiles [tile0, tile0 + n_tiles) of a call; minb = 2, 3
// or 4 resident 512-thread CTAs per SM (register cap 64, 42, 32): more warps
// to hide the Philox and search latencies.
cudaError_t launch_affine_items(const LaunchParams& L, uint32_t tile0, uint32_t n_tiles, uint32_t* items,
                                uint32_t cap, uint32_t* counts, uint32_t tile_shots, uint32_t grid, cudaStream_t st,
                                uint32_t minb) {
  if (minb == 2) affine_items<2><<<grid, 512, 0, st>>>(L, tile0, n_tiles, items, cap, counts, tile_shots);
  else if (minb == 3) affine_items<3><<<grid, 512, 0, st>>>(L, tile0, n_tiles, items, cap, counts, tile_shots);
  else if (minb == 4) affine_items<4><<<grid, 512, 0, st>>>(L, tile0, n_tiles, items, cap, counts, tile_shots);
  else return cudaErrorInvalidValue;
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
