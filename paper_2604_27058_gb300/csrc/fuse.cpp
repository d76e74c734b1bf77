// fuse.cpp — fewer passes over the active vectors for the batched executor
// (compile time, host).
//
// Every array instruction of the bytecode is a pass over 2^k amplitudes per
// shot. Many of them do not need their own pass (the localisation ladders
// of App. A make CX and CZ between active axes the most common ones):
//   * ARRAY_CX is a permutation of the amplitude indices. Instead of moving
//     data, the pass keeps a GF(2)-affine index map: amplitude i of the
//     active vector is stored at p = A i ^ c. CX(v -> w) only updates A.
//   * ARRAY_CZ, ARRAY_S and ROT_Z are diagonal: a phase that depends on
//     logical bits, i.e. on parities of the physical index (rows of A^-1).
//     They are collected and applied in the next pass that touches the
//     vector anyway.
//   * ROT_X and ARRAY_H mix amplitude pairs (i, i ^ e_v), stored at p and
//     p ^ (A e_v): one pass that first applies the pending phases.
//   * Before an active measurement or an expectation probe the map is
//     materialised (one gather pass with the pending phases), so
//     measurement, demotion, probes and every record stay exactly those of
//     the plain bytecode.
// The frame parts of the array Cliffords stay as frame instructions at
// their original places. A pending ROT_Z reads its frame sign bit when the
// phases are applied, so pending phases are applied first whenever a later
// instruction could change a frame plane that one of them reads.
//
// The result is a second instruction list (program.h, fops) with its own
// term and permutation tables; the plain executor and the debug path keep
// the original list.
#include <algorithm>
#include <cstring>
#include <vector>

#include "compiler.h"

namespace nc {

namespace {

uint32_t parity(uint32_t x) { return (uint32_t)__builtin_popcount(x) & 1u; }

struct State {
  uint32_t k = 0;
  uint32_t col[32];   // physical mask of logical axis t (A e_t)
  uint32_t rinv[32];  // row t of A^-1: logical bit t = parity(rinv[t] & (p ^ c))
  uint32_t c = 0;
  bool identity() const {
    if (c) return false;
    for (uint32_t t = 0; t < k; t++)
      if (col[t] != (1u << t)) return false;
    return true;
  }
};

}  // namespace

void append_fused(std::vector<uint8_t>& blob) {
  ProgHeader h;
  std::memcpy(&h, blob.data(), sizeof(h));
  if (h.k_max == 0 || h.k_max > 30) return;
  const Op* ops = reinterpret_cast<const Op*>(blob.data() + h.off_ops);
  // only worth a second list when array Cliffords can be absorbed or deferred
  // (a rotation alone is deferred only until the next frame change)
  uint32_t saved = 0;
  for (uint32_t pc = 0; pc < h.n_ops; pc++)
    if (ops[pc].code == OP_ARRAY_CX || ops[pc].code == OP_ARRAY_CZ || ops[pc].code == OP_ARRAY_S) saved++;
  if (saved < 8) return;

  const uint32_t N = h.n_qubits;
  std::vector<Op> out;
  std::vector<FTerm> terms;
  std::vector<uint32_t> perm;
  std::vector<FTerm> pending;
  std::vector<uint32_t> read_planes;  // frame planes read by pending terms
  State s;
  bool any_perm = false;

  auto term_cz = [&](uint32_t a, uint32_t b) {
    FTerm t{};
    t.kind = FT_CZ | (parity(s.rinv[a] & s.c) << 8) | (parity(s.rinv[b] & s.c) << 9);
    t.r1 = s.rinv[a];
    t.r2 = s.rinv[b];
    pending.push_back(t);
  };
  auto term_s = [&](uint32_t a) {
    FTerm t{};
    t.kind = FT_S | (parity(s.rinv[a] & s.c) << 8);
    t.r1 = s.rinv[a];
    pending.push_back(t);
  };
  auto term_rz = [&](const Op& o) {
    FTerm t{};
    t.kind = FT_ROTZ | (parity(s.rinv[o.pa] & s.c) << 8);
    t.plane = o.a;  // x plane of the rotated qubit: the sign of the angle
    t.r1 = s.rinv[o.pa];
    t.cs = o.cs;
    t.sn = o.sn;
    pending.push_back(t);
    read_planes.push_back(o.a);
  };
  // move the pending terms into the table behind an optional lead record
  auto take_terms = [&](Op& o, const FTerm* lead) {
    o.i2 = (uint32_t)terms.size();
    if (lead) terms.push_back(*lead);
    o.i3 = (uint32_t)pending.size();
    terms.insert(terms.end(), pending.begin(), pending.end());
    pending.clear();
    read_planes.clear();
  };
  auto flush_diag = [&]() {
    if (pending.empty()) return;
    Op o{};
    o.code = OP_DIAGF;
    o.i1 = s.k;
    take_terms(o, nullptr);
    out.push_back(o);
  };
  // frame planes an instruction may write (x plane q = q, z plane = N + q)
  auto writes_read_plane = [&](const Op& o) -> bool {
    if (read_planes.empty()) return false;
    auto hit = [&](uint32_t plane) {
      return std::find(read_planes.begin(), read_planes.end(), plane) != read_planes.end();
    };
    switch (o.code) {
      case OP_FRAME_H:
        return hit(o.a);  // the x plane of a takes z's value
      case OP_FRAME_S:
      case OP_FRAME_CZ:
        return false;  // only z planes change
      case OP_FRAME_CX:
        return hit(o.b);
      case OP_MEAS_STATIC:
        return (o.flags & FLAG_RESET) != 0;  // a fused reset writes x planes
      case OP_REC_OUT:
      case OP_DETECTOR:
      case OP_OBS_INCLUDE:
      case OP_OBS_OUT:
      case OP_KEPT_OUT:
        return false;
      default:
        return true;  // noise, feed-forward, random measurements, batches: assume so
    }
  };
  auto frame_op = [&](uint8_t code, const Op& src) {
    Op o{};
    o.code = code;
    o.a = src.a;
    o.b = src.b;
    if (writes_read_plane(o)) flush_diag();
    out.push_back(o);
  };

  for (uint32_t pc = 0; pc < h.n_ops; pc++) {
    const Op& o = ops[pc];
    if (pc == h.prefix_end && h.prefix_k > 0) {
      // end of the shared prefix: logical order, no pending term, so shots
      // can resume here from the prefix's vector
      if (!s.identity()) {
        Op m{};
        m.code = OP_PERMF;
        m.i0 = (uint32_t)perm.size();
        m.i1 = s.k;
        for (uint32_t t = 0; t < s.k; t++) perm.push_back(s.col[t]);
        perm.push_back(s.c);
        take_terms(m, nullptr);
        out.push_back(m);
        any_perm = true;
        for (uint32_t t = 0; t < s.k; t++) s.col[t] = s.rinv[t] = 1u << t;
        s.c = 0;
      } else {
        flush_diag();
      }
      h.f_start = (uint32_t)out.size();
    }
    switch (o.code) {
      case OP_BATCH:
        break;  // the payloads follow as single instructions
      case OP_ARRAY_CX: {
        // logical CX(pa -> pb): A <- A C
        s.col[o.pa] ^= s.col[o.pb];
        s.rinv[o.pb] ^= s.rinv[o.pa];
        frame_op(OP_FRAME_CX, o);
        break;
      }
      case OP_ARRAY_CZ:
        term_cz(o.pa, o.pb);
        frame_op(OP_FRAME_CZ, o);
        break;
      case OP_ARRAY_S:
        term_s(o.pa);
        frame_op(OP_FRAME_S, o);
        break;
      case OP_ROT_Z:
        term_rz(o);
        break;
      case OP_ROT_X:
      case OP_ARRAY_H: {
        Op m{};
        m.code = OP_MIXF;
        m.a = o.a;
        const uint32_t mask = s.col[o.pa];
        m.pa = (uint8_t)__builtin_ctz(mask);  // pivot: a set bit of the partner mask
        m.pb = o.code == OP_ROT_X ? 1 : 0;
        m.i0 = mask;
        m.i1 = s.rinv[o.pa] | (parity(s.rinv[o.pa] & s.c) << 31);
        FTerm lead{};
        lead.kind = FT_MIX;
        lead.plane = N + o.a;  // ROT_X: the z plane gives the sign of the angle
        lead.cs = o.cs;
        lead.sn = o.sn;
        take_terms(m, &lead);
        out.push_back(m);
        if (o.code == OP_ARRAY_H) frame_op(OP_FRAME_H, o);
        break;
      }
      case OP_EXPAND_ROT: {
        flush_diag();
        s.col[s.k] = 1u << s.k;
        s.rinv[s.k] = 1u << s.k;
        s.k++;
        out.push_back(o);
        break;
      }
      case OP_EXPVAL:
      case OP_MEAS_ACTIVE_Z:
      case OP_MEAS_ACTIVE_X: {
        // the vector in logical order with every pending phase applied; a
        // gather right before a measurement also forms its sums (one pass
        // over the vector instead of two)
        Op mo = o;
        if (!s.identity()) {
          Op m{};
          m.code = OP_PERMF;
          m.i0 = (uint32_t)perm.size();
          m.i1 = s.k;
          for (uint32_t t = 0; t < s.k; t++) perm.push_back(s.col[t]);
          perm.push_back(s.c);
          take_terms(m, nullptr);
          if (o.code != OP_EXPVAL && s.k >= 1) {
            m.flags |= FLAG_SUMS;
            m.pa = o.pa;
            m.pb = o.code == OP_MEAS_ACTIVE_X ? 1 : 0;
            mo.flags |= FLAG_PRESUMMED;
          }
          out.push_back(m);
          any_perm = true;
          for (uint32_t t = 0; t < s.k; t++) s.col[t] = s.rinv[t] = 1u << t;
          s.c = 0;
        } else {
          flush_diag();
        }
        out.push_back(mo);
        if (o.code != OP_EXPVAL) s.k--;  // a probe keeps every axis
        for (uint32_t t = 0; t < s.k; t++) s.col[t] = s.rinv[t] = 1u << t;
        break;
      }
      default:
        if (writes_read_plane(o)) flush_diag();
        out.push_back(o);
        break;
    }
  }
  flush_diag();

  uint64_t off = h.total_bytes;
  auto place = [&](uint64_t bytes) {
    uint64_t at = off;
    off = (off + bytes + 15) & ~15ull;
    return at;
  };
  h.off_fops = place(out.size() * sizeof(Op));
  h.off_fterm = place(terms.size() * sizeof(FTerm));
  h.off_fperm = place(perm.size() * 4);
  h.n_fops = (uint32_t)out.size();
  h.n_fterms = (uint32_t)terms.size();
  h.n_fperm = (uint32_t)perm.size();
  h.f_perm = any_perm ? 1 : 0;
  h.total_bytes = off;
  blob.resize(off, 0);
  if (!out.empty()) std::memcpy(blob.data() + h.off_fops, out.data(), out.size() * sizeof(Op));
  if (!terms.empty()) std::memcpy(blob.data() + h.off_fterm, terms.data(), terms.size() * sizeof(FTerm));
  if (!perm.empty()) std::memcpy(blob.data() + h.off_fperm, perm.data(), perm.size() * 4);
  std::memcpy(blob.data(), &h, sizeof(h));
}

}  // namespace nc
