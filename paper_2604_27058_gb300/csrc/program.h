// program.h — compiled program layout shared by the host compiler and the
// CUDA executors (product-internal; the oracle has its own representation).
//
// A program is the SVM bytecode of Sec. 3.1 stage 3/4: a flat list of fixed
// 32-byte instructions plus side tables (virtual Pauli masks, noise-site
// survival table, detector record lists). Everything is identical for every
// shot (Thm. 1), so one copy per device serves all shots.
#pragma once
#include <stdint.h>

namespace nc {

enum OpCode : uint8_t {
  OP_END = 0,
  // Frame-only virtual Cliffords (P~ <- V P~ V^dagger), bit-sliced over shots.
  OP_FRAME_H, OP_FRAME_S, OP_FRAME_CX, OP_FRAME_CZ,
  // Virtual Cliffords between active axes: frame conjugation + array update.
  OP_ARRAY_H, OP_ARRAY_S, OP_ARRAY_CX, OP_ARRAY_CZ,
  // Pauli rotations (App. B.1); f = theta * alpha, frame sign applied per shot.
  OP_EXPAND_ROT,   // a = v, pa = new top position; phi <- phi (x) (|0> + e^{2i t}|1>)/sqrt2, t = f (-1)^{x_v}
                   // (cs, sn) = (cos 2f, sin 2f)
  OP_ROT_Z,        // a = v, pa; bit-1 amplitudes *= e^{2i t}, t = f (-1)^{x_v}; (cs, sn) = (cos 2f, sin 2f)
  OP_ROT_X,        // a = v, pa; exp(-i t X), t = f (-1)^{z_v}; (cs, sn) = (cos f, sin f)
  // Measurements (App. B.2); flags bit0 = alpha sign bit, bit1 = output now (row i3).
  OP_MEAS_STATIC,  // i0 = z-mask offset; m = sign ^ parity(x & zmask); slot i2
  OP_MEAS_RANDOM,  // a = v, i0 = event; m = [u < 1/2]; b = m^sign^z_v; H_v; x_v ^= b
  OP_MEAS_ACTIVE_Z,// a = v, pa, i0 = event; mask, renormalise, demote; x_v ^= b
  OP_MEAS_ACTIVE_X,// a = v, pa, i0 = event; fold, renormalise, demote; H_v; x_v ^= b
  // Stochastic noise (Sec. 3.2): sites [i0, i1) in physical order.
  OP_NOISE_BLOCK,
  // Conditional Paulis (App. B.3): frame ^= E (mask i0) where slot i2 is set.
  OP_FEEDFORWARD,
  // Records and classical ops (Sec. 3.2, post-selection).
  OP_REC_OUT,      // slot i2 -> meas row i3
  OP_DETECTOR,     // XOR of i1 slots at slot list i0, ^ ref(i3) -> det row i3; postselect
  OP_OBS_INCLUDE,  // obs slot i2 ^= XOR of i1 slots at slot list i0
  OP_OBS_OUT,      // obs slot i2 ^ ref -> obs row i3 (masked by kept)
  OP_KEPT_OUT,     // kept slot i2 -> kept row
  // Batch headers: the next pa instructions (same kind, mutually independent,
  // all inside one staging chunk) may run together. An executor may also
  // ignore the header and run them one by one.
  OP_BATCH,
  // Fused array passes (second instruction list, batched executor only;
  // fuse.cpp). Amplitude i of the active vector sits at p = A i ^ c.
  OP_DIAGF,  // i2 = first term, i3 = term count: apply the diagonal terms to every amplitude
  OP_MIXF,   // pair pass: partner mask i0, orientation mask i1 (bit 31: its constant), pivot
             // bit pa, pb = 0 H / 1 ROT_X; i2 = lead record (ROT_X angle, sign plane), then i3 terms
  OP_PERMF,  // gather into logical order: perm table at i0 (i1 column masks, then c), i2 / i3 terms
  // Expectation-value probe (Sec. 3.2): <P> of the shot's state into probe row i3.
  // M(P) = i^pa X^x Z^z (mask i0: x words then z words); the frame contributes
  // (-1)^{parity(fx & z) ^ parity(fz & x)}; pb = 1: x-support on a dormant
  // qubit (the value is 0); else <phi| X^i1 Z^i2 |phi> / <phi|phi> over the
  // active positions.
  OP_EXPVAL,
  OP_COUNT
};

// Terms of fused passes (32 bytes). kind bits 0..7: FT_*; bit 8 / bit 9: the
// constants of the two parities. A parity is parity(r & p) ^ constant for
// physical index p. CZ: -1 if both parities are 1; S: i if the parity is 1;
// ROTZ: (cs, sn) with sn negated when frame plane `plane` is set, if the
// parity is 1; MIX: the lead record of OP_MIXF (cs, sn and the sign plane).
enum : uint32_t { FT_CZ = 1, FT_S = 2, FT_ROTZ = 3, FT_MIX = 4 };
struct FTerm {
  uint32_t kind, plane, r1, r2;
  double cs, sn;
};
static_assert(sizeof(FTerm) == 32, "FTerm must be 32 bytes");

// FLAG_REF (DETECTOR, OBS_OUT): the noiseless reference parity is 1. It is
// set on the device copy after the reference launch (patch_ref_flags).
// Fused list only: FLAG_SUMS on an OP_PERMF gather directly before an active
// measurement: the gather also accumulates that measurement's FP64 sums
// (measured logical position in pa, pb = 1 for an X measurement), and the
// measurement carries FLAG_PRESUMMED and skips its own reduction pass.
enum : uint8_t { FLAG_SIGN = 1, FLAG_OUT = 2, FLAG_RESET = 4, FLAG_REF = 8, FLAG_SUMS = 16, FLAG_PRESUMMED = 32 };

struct Op {
  uint8_t code;
  uint8_t flags;
  uint16_t a;   // virtual qubit (control / v)
  uint16_t b;   // virtual qubit (target)
  uint8_t pa;   // array position of a; for list ops: inline entry count (kNoInline = use tables)
  uint8_t pb;   // array position of b; for a fused reset: count of its inline X-image entries
  union {
    struct { uint32_t i0, i1, i2, i3; };
    struct { uint32_t j0, j1; uint16_t r[4]; };  // fused reset: r = inline X-image planes
    struct { double cs, sn; };                   // rotations: cos / sin of the phase (see OpCode)
  };
  union {
    double f;        // rotation angle
    uint16_t e[4];   // inline entries of list ops
  };
};
static_assert(sizeof(Op) == 32, "Op must be 32 bytes");

// List ops (MEAS_STATIC, FEEDFORWARD: frame planes; DETECTOR, OBS_INCLUDE:
// record slots) carry up to kInline entries in the instruction itself. A
// frame plane index is q for the x bit of virtual qubit q and n_qubits + q
// for its z bit. Longer lists use the mask / slot-list tables.
//
// A reset whose measurement is static (a dormant Z string, App. B.2) is fused
// into one MEAS_STATIC with FLAG_RESET: m = sign ^ parity(inline planes e),
// then the frame planes r[0..pb) are XORed with m (the conditional X of the
// reset, App. B.3). It writes no record slot.
constexpr uint32_t kInline = 4;
constexpr uint8_t kNoInline = 0xFF;

// Padding of inline entries beyond the count: reads use an all-zero row
// (frame plane 2N, record slot n_slots), writes a scratch plane (2N + 1), so
// every instruction touches exactly kInline entries without branching.
// Instructions are staged in chunks of kChunk; a batch never crosses one.
constexpr uint32_t kChunk = 128;
constexpr uint32_t kMaxBatch = 8;

// Noise-site kinds (physical channel of the site).
enum SiteKind : uint8_t { SITE_X = 0, SITE_Y, SITE_Z, SITE_D1, SITE_D2, SITE_FLIP };

// Header of the device blob; all offsets are in bytes from the blob start
// and 16-byte aligned.
struct ProgHeader {
  uint32_t magic, version;
  uint32_t n_qubits, nw;          // nw = 32-bit words per virtual bit mask
  uint32_t n_ops, n_sites;
  uint32_t n_meas, n_det, n_obs, n_events;
  uint32_t n_slots, k_max;
  uint32_t kept_slot, n_mask_words, n_slot_list, n_opt;
  uint32_t n_plist;
  float mean_faults;               // sum of site probabilities (expected faults per shot)
  uint32_t n_blocks;               // NOISE_BLOCK instructions (their ordinal is in i2)
  uint32_t aff_ok;                 // 1: the record-level propagation tables below are present
  uint32_t aff_rows, aff_n_rand;   // rows = n_meas + n_det + n_obs; random dormant measurements
  uint32_t aff_n_chunks;           // 8-row chunks of the fault columns
  float aff_chunks_per_shot;       // expected chunks of a shot's faults
  uint32_t n_guide;                // survival guide-table entries
  uint32_t aff_n_chains;           // delta-row chains (every row on one; longest first)
  uint32_t aff_n_chain_rows;       // rows on those chains (= aff_rows)
  uint32_t n_probes;               // expectation-value probes (OP_EXPVAL rows)
  // shared prefix: ops [0, prefix_end) are frame / array / rotation
  // instructions only (no noise, measurement or record), so every shot
  // reaches ops[prefix_end] with the same active vector (prefix_k axes) and
  // a zero frame
  uint32_t prefix_end, prefix_k;
  // the fused list's instruction where the shots resume after the shared
  // prefix, in logical order with no pending term (fuse.cpp)
  uint32_t f_start, pad4;
  uint32_t n_fops, n_fterms;       // fused instruction list and its terms (0: none)
  uint32_t n_fperm, f_perm;        // permutation-table words; 1 if the list has OP_PERMF
  uint64_t off_ops, off_masks, off_q, off_seg_start, off_seg_end, off_site_info, off_site_eff,
      off_slot_list, off_det_ref, off_obs_ref, off_site_opt, off_opt_tab, off_plist, off_orec, off_site_blk,
      off_aff_const, off_aff_rowev_off, off_aff_rowev, off_aff_rand_ev, off_aff_col_off, off_aff_col,
      off_aff_frec, off_aff_parent, off_aff_chain_off, off_aff_chain, off_srch, off_guide, off_fops, off_fterm,
      off_fperm, off_site_p, total_bytes;
};
// site_p: the fault probability of every noise site (FP64, site order), from
// which the host builds the stratified-sampling tables (strata.cpp).
// Survival-jump search (Sec. 3.2 jump, integer form). srch[st] (32 bytes)
// holds, for a jump starting at site st: the segment [a, b), its guide-table
// base and shift, Q[b - 1] and Q_L (Q[st - 1], or 2^64 - 1 at a segment
// start). The next fault is the first i in [st, b) with Q[i] <= t; guide
// entry g[base + guide_key(t, shift)] is a site at or before it, so a short
// forward scan from there finds it exactly.
struct SrchRec {
  uint32_t a, b, gbase, shift;
  uint64_t q_end, q_l;
};
static_assert(sizeof(SrchRec) == 32, "SrchRec must be 32 bytes");
constexpr uint32_t kGuideBits = 16;
// Piecewise-linear log2 of t (exponent, then kGuideBits mantissa bits),
// non-decreasing in t; the key counts down from its value at 2^64 - 1.
// (Host form; the device form in kernels.cuh computes the same value.)
inline uint32_t guide_key(uint64_t t, uint32_t shift) {
  if (t < (1ull << kGuideBits)) t = 1ull << kGuideBits;
  uint32_t e = 63;
  while (!(t >> e)) e--;
  const uint32_t m = (uint32_t)(t >> (e - kGuideBits)) & ((1u << kGuideBits) - 1u);
  const uint32_t lv = (e << kGuideBits) | m, lmax = (63u << kGuideBits) | ((1u << kGuideBits) - 1u);
  return (lmax - lv) >> shift;
}
// Record-level propagation (programs with k_max = 0). With every frame
// update GF(2)-linear, a shot's records are an affine function of its fault
// indicators and of its random dormant measurement outcomes:
//   row r = const[r] ^ XOR_{j in rowev(r)} m_j ^ XOR_{faults f} [r in col(f)]
// where rows are meas rows, then det rows, then obs rows (detector and
// observable rows before their reference parity), m_j is the outcome of
// the j-th random dormant measurement (event rand_ev[j]) and col(f) lists
// the rows flipped by fault option f = site * kRecPerSite + option.
//   const: u32 per row (0 / 1); rowev_off: rows + 1 u32; rowev: u32 ordinals
//   rand_ev: u32 event per ordinal; col_off: n_sites * kRecPerSite + 1 u32
//   chunk offsets; col: chunks of 8 u16 chain positions (16 bytes), padded
//   with `rows` (no row).
//   Rows are stored in delta form: the value above is delta_r, and the
//   record row is delta_r ^ (record row parent[r]) (parent 0xFFFFFFFF: none);
//   chain_off / chain list the chains head first, every row on exactly one
//   (rows with neither parent nor child are chains of one), longest first;
//   position j of the concatenated list holds row chain[j], and the sampler
//   keeps row chain[j] at position j of its tile. A running XOR down a chain
//   turns deltas into rows. Detector and
//   observable reference parities apply to record rows, so delta_r takes
//   ref(r) ^ ref(parent[r]).
//   frec: 16 bytes per site, so that one load after the search gives a
//   fault's chunk range: words 0-1 hold 4-bit chunk counts of options 0..14
//   (bits 60..63: the option count K), word 2 the first chunk of option 0
//   (0xFFFFFFFF: some option has more than 15 chunks; use col_off).
// site_blk[site] = ordinal of the NOISE_BLOCK instruction that covers the site.
// Option records: orec[site * 15 + option] is 16 bytes (8 x u16). Word 0 is
// a tag: n <= 7 -> n frame-plane indices follow; kRecFlip -> the site flips
// record slot (words 1, 2) / output row (words 3, 4); kRecLong -> use
// opt_tab / plist. Indexed directly, so applying a fault is one load.
constexpr uint16_t kRecFlip = 0xFFFE, kRecLong = 0xFFFF;
constexpr uint32_t kRecPerSite = 15;
// Noise options in sparse form: site_info >> 8 indexes opt_tab;
// opt_tab[2 * (index + option)] = (plist offset, entry count); plist holds
// frame plane indices (u16). A FLIP site has one entry (record slot, record
// row): its fault flips the slot and, if the shot is kept, the output bit.

constexpr uint32_t kMagic = 0x4E435047u;  // "NCPG"
constexpr uint32_t kVersion = 14;
constexpr uint32_t kMaxK = 30;
constexpr uint32_t kMaxQubits = 4096;

// site_info word: kind (bits 0..3) | option count K (bits 4..7) | first
// opt_tab entry (bits 8..31).
inline uint32_t site_kind(uint32_t info) { return info & 15u; }
inline uint32_t site_k(uint32_t info) { return (info >> 4) & 15u; }

}  // namespace nc
