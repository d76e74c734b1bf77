// kernels.cuh — device-side helpers shared by the two executors: program
// view, Philox4x32-10 draws, noise-site search. Product code only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "program.h"

namespace nc {

struct DevProg {
  const Op* ops;
  const uint32_t* masks;
  const uint64_t* q;
  const uint32_t* seg_start;
  const uint32_t* seg_end;
  const uint32_t* site_info;
  const uint32_t* site_eff;
  const uint32_t* slot_list;
  const uint32_t* det_ref;
  const uint32_t* obs_ref;
  const uint32_t* site_opt;
  const uint32_t* opt_tab;
  const uint16_t* plist;
  const uint4* orec;
  const uint32_t* site_blk;
  // record-level propagation tables (program.h; null when absent)
  const uint32_t* aff_const;
  const uint32_t* aff_rowev_off;
  const uint32_t* aff_rowev;
  const uint32_t* aff_rand_ev;
  const uint32_t* aff_col_off;
  const uint4* aff_chunks;
  const uint4* aff_frec;
  const uint32_t* aff_parent;
  const uint32_t* aff_chain_off;
  const uint32_t* aff_chain;
  const uint32_t* srch;   // SrchRec per site (program.h)
  const uint32_t* guide;
  // fused array-pass list (fuse.cpp; n_fops = 0: none)
  const Op* fops;
  const FTerm* fterm;
  const uint32_t* fperm;
  uint32_t n_fops, f_perm;
  uint32_t n_qubits, nw, n_ops, n_sites, n_slots, k_max, kept_slot;
  uint32_t n_meas, n_det, n_obs, n_blocks;
  uint32_t aff_rows, aff_n_rand, aff_n_chains, aff_n_chain_rows;
  float aff_chunks_per_shot;
  // stratified noise (strata.cpp tables; set per call, null = independent
  // sites): G_r(j) at sg[(r - 1) * sg_n + j], exactly sg_k faults per shot;
  // row r's guide parameters at sgr[3 (r - 1) ..] (bits of G_r(0), shift |
  // kmax << 32, first guide entry) and its guide entries in sgg
  const double* sg;
  const unsigned long long* sgr;
  const uint32_t* sgg;
  uint32_t sg_k, sg_n;
};

enum : uint32_t {
  LF_NOISELESS = 1,   // skip every noise site
  LF_POSTSELECT = 2,  // kept &= ~detector
  LF_REFERENCE = 4,   // raw parities (no reference XOR)
  LF_OUT_MEAS = 8,
  LF_OUT_DET = 16,
  LF_OUT_OBS = 32,
  LF_OUT_KEPT = 64,
  LF_ASYNC = 128,     // host side only: no host synchronisation (stream capture)
  LF_ARGMAX = 256,    // every measurement takes its more likely outcome (0 on a tie): the reference trajectory
  LF_OUT_EXPVAL = 512,  // write the expectation probes (OP_EXPVAL) to expval
};

struct LaunchParams {
  DevProg p;
  uint64_t seed, shot_offset, shots;
  uint32_t *meas, *det, *obs, *kept;  // u32 views of the u64 record rows
  double* expval;                     // probe j of call-local shot s at expval[j * shots + s]
  uint64_t row_words32;               // u32 words per record row
  uint32_t flags;
  uint32_t G;                         // 32-shot words per tile (batched executor)
  uint32_t n_tiles;
  uint64_t work_stride;               // amplitudes per CTA workspace (batched) / per shot (plain)
  uint32_t smem_work_words;           // batched: > 0 = the CTA's vectors live in shared memory (words)
  void* work;                         // amplitude workspace
  unsigned long long* kept_count;
  uint32_t* err;
  // pre-sampled faults (batched executor; null = sample inline): fault j of
  // call-local shot s at flist[j * fstride + s] for j < fcount[s] & 127;
  // bit 7 of fcount marks a list truncated at fcap entries.
  const uint32_t* flist;
  const uint8_t* fcount;
  uint32_t fcap;
  uint64_t fstride;
  // faults bucketed by noise block (bucketed executor): warp-tile wt (1024
  // call-local shots) has its block-k entries at bents[boffs[wt*(nb+1)+k] ..
  // boffs[wt*(nb+1)+k+1]); an entry is (option record << 10) | shot in tile.
  const uint32_t* bents;
  const uint32_t* boffs;
  // record-level propagation sampler: first tile of this launch and the
  // pre-sampled chunk items of its tiles (null: sample in the kernel)
  uint32_t tile0;
  // plain executor: this launch's call-local shots [plain_base, plain_base + plain_n)
  uint64_t plain_base, plain_n;
  const uint32_t* aff_items;
  const uint32_t* aff_counts;
  uint32_t aff_cap;
  // shared prefix (batched executor): every shot starts at instruction
  // start_op of the list it runs (the fused list's f_start, or prefix_end of
  // the plain list) with the active vector init_vec (2^start_k amplitudes,
  // the executor's precision) and a zero frame; null = start at instruction
  // 0 with phi = [1]
  const void* init_vec;
  uint32_t start_op, start_k;
  uint32_t stop_event;                // debug: stop before this event (0xffffffff = never)
  uint64_t dump_shot;                 // debug: call-local shot index
  double* dump_amps;
  uint32_t* dump_frame;
  uint32_t* dump_k;
};

constexpr uint32_t kNoFault = 0xffffffffu;
constexpr uint32_t TAG_MT = 1, TAG_ML = 2, TAG_GAP = 3, TAG_STRAT = 4;

// Philox4x32-10 (Salmon et al., SC'11).
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ uint2 key_of(uint64_t seed) {
  return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
}

// Top bits of the 32 shots of the aligned word starting at global shot s0.
__device__ __forceinline__ uint32_t meas_top_word(uint64_t seed, uint64_t s0, uint32_t event) {
  uint64_t g = s0 >> 7;
  uint4 w = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), TAG_MT, event), key_of(seed));
  uint32_t sel = (uint32_t)(s0 >> 5) & 3u;
  return sel == 0 ? w.x : sel == 1 ? w.y : sel == 2 ? w.z : w.w;
}

// u of shot s (global) given its top bit: (top * 2^52 + low52) * 2^-53.
__device__ __forceinline__ double meas_u(uint64_t seed, uint64_t s, uint32_t event, uint32_t top) {
  uint4 w = philox(make_uint4((uint32_t)s, (uint32_t)(s >> 32), TAG_ML, event), key_of(seed));
  uint64_t low = ((uint64_t)w.x | ((uint64_t)w.y << 32)) & ((1ull << 52) - 1);
  uint64_t v = ((uint64_t)top << 52) | low;
  return (double)v * 0x1p-53;
}

// m = [u < p1]. When p1 == 1/2 exactly only the top bit matters.
__device__ __forceinline__ uint32_t draw_outcome(uint64_t seed, uint64_t s, uint32_t event,
                                                 uint32_t top, double p1) {
  if (p1 <= 0.0) return 0;
  if (p1 >= 1.0) return 1;
  if (p1 == 0.5) return top ? 0u : 1u;
  return meas_u(seed, s, event, top) < p1 ? 1u : 0u;
}

__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// Next fault of global shot `shot` at or after site `st` (Sec. 3.2 jump,
// integer survival form). Returns (site << 4) | option, or kNoFault.
__device__ __forceinline__ uint32_t guide_key_dev(uint64_t t, uint32_t shift) {
  t = t < (1ull << kGuideBits) ? (1ull << kGuideBits) : t;
  const uint32_t e = 63u - (uint32_t)__clzll((long long)t);
  const uint32_t m = (uint32_t)(t >> (e - kGuideBits)) & ((1u << kGuideBits) - 1u);
  const uint32_t lv = (e << kGuideBits) | m, lmax = (63u << kGuideBits) | ((1u << kGuideBits) - 1u);
  return (lmax - lv) >> shift;
}

// One survival-jump draw from site st (Sec. 3.2, integer form): returns the
// fault site (and leaves the draw in *w for the option), or kNoFault with
// *next = the end of st's segment.
__device__ __forceinline__ uint32_t jump_draw(const DevProg& p, uint2 key, uint64_t shot, uint32_t st, uint4* w,
                                              uint32_t* next) {
  const uint4 r0 = __ldg(reinterpret_cast<const uint4*>(p.srch) + 2 * st);
  const uint4 r1 = __ldg(reinterpret_cast<const uint4*>(p.srch) + 2 * st + 1);
  *w = philox(make_uint4((uint32_t)shot, (uint32_t)(shot >> 32), TAG_GAP, st), key);
  const uint64_t u = (uint64_t)w->x | ((uint64_t)w->y << 32);
  const uint64_t q_end = (uint64_t)r1.x | ((uint64_t)r1.y << 32), q_l = (uint64_t)r1.z | ((uint64_t)r1.w << 32);
  const uint64_t t = mulhi64(u, q_l);
  if (q_end > t) {
    *next = r0.y;
    return kNoFault;
  }
  uint32_t i = __ldg(p.guide + r0.z + guide_key_dev(t, r0.w));
  while (__ldg(p.q + i) > t) i++;
  return i;
}

// Next fault of a shot at or after site st: (site << 4) | option, or kNoFault.
__device__ __forceinline__ uint32_t next_fault(const DevProg& p, uint64_t seed, uint64_t shot, uint32_t st) {
  const uint2 key = key_of(seed);
  while (st < p.n_sites) {
    uint4 w;
    uint32_t nx;
    const uint32_t i = jump_draw(p, key, shot, st, &w, &nx);
    if (i != kNoFault) {
      const uint32_t k = (__ldg(p.site_info + i) >> 4) & 15u;
      return (i << 4) | __umulhi(w.z, k);
    }
    st = nx;
  }
  return kNoFault;
}

// Stratified noise (Sec. 3.2 rare-event strata): a shot holding r >= 1
// faults at site st draws u on the 53-bit grid from
// Philox(shot, TAG_STRAT, st) and puts its next fault at the first j >= st
// with G_r(j + 1) <= t, t = u * G_r(st) (one rounded FP64 product). G_r
// never increases: the row's guide entry for t is a site at or before the
// answer, and a forward scan (G_r(S) = 0 ends it) finds it exactly.
// Returns j and the option word.
__device__ __forceinline__ uint32_t strat_jump(const DevProg& p, uint2 key, uint64_t shot, uint32_t st, uint32_t r,
                                               uint32_t* wz) {
  const uint4 w = philox(make_uint4((uint32_t)shot, (uint32_t)(shot >> 32), TAG_STRAT, st), key);
  const uint64_t u53 = ((uint64_t)w.x | ((uint64_t)w.y << 32)) >> 11;
  const double* g = p.sg + (size_t)(r - 1) * p.sg_n;
  const double thr = __dmul_rn((double)u53 * 0x1p-53, __ldg(g + st));
  const unsigned long long* row = p.sgr + 3 * (size_t)(r - 1);
  const unsigned long long b = __ldg(row), sk = __ldg(row + 1), go = __ldg(row + 2);
  const unsigned long long d = (b - (unsigned long long)__double_as_longlong(thr)) >> (uint32_t)sk;
  const uint32_t kmax = (uint32_t)(sk >> 32);
  uint32_t j = __ldg(p.sgg + (uint32_t)go + (d < kmax ? (uint32_t)d : kmax));
  j = j > st ? j : st;
  while (__ldg(g + j + 1) > thr) j++;
  *wz = w.z;
  return j;
}

// Next fault at or after site st under either noise model; r counts the
// faults a stratified shot still holds (start at p.sg_k; ignored otherwise).
__device__ __forceinline__ uint32_t next_fault_r(const DevProg& p, uint64_t seed, uint64_t shot, uint32_t st,
                                                 uint32_t& r) {
  if (!p.sg) return next_fault(p, seed, shot, st);
  if (r == 0 || st >= p.n_sites) return kNoFault;
  uint32_t wz;
  const uint32_t i = strat_jump(p, key_of(seed), shot, st, r, &wz);
  r--;
  const uint32_t k = (__ldg(p.site_info + i) >> 4) & 15u;
  return (i << 4) | __umulhi(wz, k);
}

// Terms of the measurement sums S_0, S_1 (App. B.2), accumulated in FP64 by
// the caller. With FP32 amplitudes a term is formed in FP32 (|a|^2 as one
// product and one fused multiply-add: at most two roundings, relative error
// below 2^-23 per term, which does not accumulate since every term is
// non-negative) and converted once; with FP64 amplitudes it is formed in FP64.
// The FP64 units are the scarce ones on this GPU, so this keeps one
// conversion and one FP64 add per amplitude in the FP32 form.
__device__ __forceinline__ double mterm(float2 a) { return (double)fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ double mterm(double2 a) { return a.x * a.x + a.y * a.y; }
// X measurement: the folds (u + v) / sqrt 2 and (u - v) / sqrt 2, squared.
__device__ __forceinline__ void mterm_x(float2 u, float2 v, double& a0, double& a1) {
  const float px = u.x + v.x, py = u.y + v.y, mx = u.x - v.x, my = u.y - v.y;
  a0 += (double)(0.5f * fmaf(px, px, py * py));
  a1 += (double)(0.5f * fmaf(mx, mx, my * my));
}
__device__ __forceinline__ void mterm_x(double2 u, double2 v, double& a0, double& a1) {
  const double px = u.x + v.x, py = u.y + v.y, mx = u.x - v.x, my = u.y - v.y;
  a0 += 0.5 * (px * px + py * py);
  a1 += 0.5 * (mx * mx + my * my);
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t insert0(uint32_t j, uint32_t p) {
  return ((j >> p) << (p + 1)) | (j & ((1u << p) - 1u));
}

}  // namespace nc
