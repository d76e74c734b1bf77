// affine.cpp — record-level fault propagation for programs without active
// axes (k_max = 0), computed once at compile time on the host.
//
// With no active vector every instruction of the program is a GF(2)-affine
// map of the bit-packed state (virtual frame planes, record slots, output
// rows): frame Cliffords and conditional Paulis XOR planes (Sec. 2.3,
// App. B.3), a static measurement is a parity of planes (Sec. 2.4, App. B.2),
// a random dormant measurement draws a fresh bit m and then updates the frame
// affinely, and a fault XORs its fixed image M(E) into the frame (Sec. 3.2).
// The records of a shot are therefore const ^ A m ^ F f, where m are the
// shot's random measurement bits and f its fault indicators. This pass finds
// const, A and F by running the compiled program on 64 probe lanes at a time
// (lane = "no fault, all m = 0", "only m_j = 1", or "only fault option f")
// and XORing each lane's rows with the baseline's, then rewrites rows that
// overlap an earlier row as differences (chains of delta rows), which makes
// the fault columns short. The sampler then needs, per shot, only its
// faults and its random bits; the frame work is done once here instead of
// once per shot.
//
// The probe interpreter follows the bytecode as the executors run it
// (program.h); it never runs on a program with active-array instructions.
#include <algorithm>
#include <atomic>
#include <exception>
#include <mutex>
#include <thread>
#include <cstring>
#include <iterator>
#include <vector>

#include "compiler.h"

namespace nc {

namespace {

constexpr uint64_t kMaxEntries = 1ull << 26;  // 256 MB of column entries

struct Blob {
  const ProgHeader* h;
  const uint8_t* base;
  template <typename T>
  const T* at(uint64_t off) const {
    return reinterpret_cast<const T*>(base + off);
  }
};

uint32_t entry(const Op& o, uint32_t i) { return o.e[i]; }
uint32_t rentry(const Op& o, uint32_t i) { return ((i < 2 ? o.i2 : o.i3) >> (16 * (i & 1))) & 0xFFFFu; }

// State of one probe run over 64 lanes: frame planes, record slots and the
// output rows (meas, det, obs).
struct Probe {
  std::vector<uint64_t> planes, slots, rows;
};

bool supported(uint8_t code) {
  switch (code) {
    case OP_END: case OP_BATCH: case OP_FRAME_H: case OP_FRAME_S: case OP_FRAME_CX: case OP_FRAME_CZ:
    case OP_MEAS_STATIC: case OP_MEAS_RANDOM: case OP_NOISE_BLOCK: case OP_FEEDFORWARD: case OP_REC_OUT:
    case OP_DETECTOR: case OP_OBS_INCLUDE: case OP_OBS_OUT: case OP_KEPT_OUT:
      return true;
    default:
      return false;
  }
}

void run_probe(const Blob& b, const std::vector<uint32_t>& rand_ord, const std::vector<uint64_t>& rand_mask,
               const std::vector<std::vector<std::pair<uint32_t, uint64_t>>>& site_faults, Probe& pr) {
  const ProgHeader& h = *b.h;
  const uint32_t N = h.n_qubits, R = h.n_meas + h.n_det + h.n_obs;
  pr.planes.assign(2 * N + 2, 0);
  pr.slots.assign(h.n_slots + 1, 0);
  pr.rows.assign(R, 0);
  uint64_t* P = pr.planes.data();
  uint64_t* SL = pr.slots.data();
  uint64_t* RW = pr.rows.data();
  SL[h.kept_slot] = ~0ull;
  const Op* ops = b.at<Op>(h.off_ops);
  const uint32_t* masks = b.at<uint32_t>(h.off_masks);
  const uint32_t* slot_list = b.at<uint32_t>(h.off_slot_list);
  const uint32_t* site_info = b.at<uint32_t>(h.off_site_info);
  const uint32_t* opt_tab = b.at<uint32_t>(h.off_opt_tab);
  const uint16_t* plist = b.at<uint16_t>(h.off_plist);
  const uint16_t* orec = b.at<uint16_t>(h.off_orec);
  const uint64_t kept = ~0ull;
  for (uint32_t pc = 0; pc < h.n_ops; pc++) {
    const Op& o = ops[pc];
    switch (o.code) {
      case OP_FRAME_H: {
        uint64_t t = P[o.a];
        P[o.a] = P[N + o.a];
        P[N + o.a] = t;
        break;
      }
      case OP_FRAME_S:
        P[N + o.a] ^= P[o.a];
        break;
      case OP_FRAME_CX:
        P[o.b] ^= P[o.a];
        P[N + o.a] ^= P[N + o.b];
        break;
      case OP_FRAME_CZ: {
        const uint64_t xa = P[o.a], xb = P[o.b];
        P[N + o.a] ^= xb;
        P[N + o.b] ^= xa;
        break;
      }
      case OP_MEAS_STATIC: {
        uint64_t m = (o.flags & FLAG_SIGN) ? ~0ull : 0ull;
        if (o.pa != kNoInline) {
          for (uint32_t i = 0; i < kInline; i++) m ^= P[entry(o, i)];
        } else {
          for (uint32_t w = 0; w < h.nw; w++) {
            uint32_t bits = masks[o.i0 + w];
            while (bits) {
              const uint32_t q = w * 32u + (uint32_t)__builtin_ctz(bits);
              bits &= bits - 1;
              m ^= P[q];
            }
          }
        }
        if (o.flags & FLAG_RESET) {
          for (uint32_t i = 0; i < o.pb && i < kInline; i++) P[rentry(o, i)] ^= m;
        } else {
          SL[o.i2] = m;
          if (o.flags & FLAG_OUT) RW[o.i3] = m & kept;
        }
        break;
      }
      case OP_MEAS_RANDOM: {
        const uint64_t m = rand_mask[rand_ord[pc]];
        const uint64_t sg = (o.flags & FLAG_SIGN) ? ~0ull : 0ull;
        const uint64_t ox = P[o.a], oz = P[N + o.a];
        const uint64_t bb = m ^ sg ^ oz;
        P[o.a] = oz ^ bb;
        P[N + o.a] = ox;
        SL[o.i2] = m;
        if (o.flags & FLAG_OUT) RW[o.i3] = m & kept;
        break;
      }
      case OP_NOISE_BLOCK:
        for (uint32_t s = o.i0; s < o.i1; s++) {
          for (const auto& fl : site_faults[s]) {
            const uint32_t opt = fl.first;
            const uint64_t lanes = fl.second;
            const uint16_t* r = orec + ((size_t)s * kRecPerSite + opt) * 8;
            if (r[0] == kRecFlip) {
              const uint32_t slot = (uint32_t)r[1] | ((uint32_t)r[2] << 16);
              const uint32_t row = (uint32_t)r[3] | ((uint32_t)r[4] << 16);
              SL[slot] ^= lanes;
              RW[row] ^= lanes & kept;
            } else if (r[0] == kRecLong) {
              const uint32_t oi = 2 * ((site_info[s] >> 8) + opt);
              for (uint32_t q = 0; q < opt_tab[oi + 1]; q++) P[plist[opt_tab[oi] + q]] ^= lanes;
            } else {
              for (uint32_t q = 0; q < r[0]; q++) P[r[1 + q]] ^= lanes;
            }
          }
        }
        break;
      case OP_FEEDFORWARD: {
        const uint64_t c = SL[o.i2];
        if (o.pa != kNoInline) {
          for (uint32_t i = 0; i < o.pa && i < kInline; i++) P[entry(o, i)] ^= c;
        } else {
          for (uint32_t part = 0; part < 2; part++)
            for (uint32_t w = 0; w < h.nw; w++) {
              uint32_t bits = masks[o.i0 + part * h.nw + w];
              while (bits) {
                const uint32_t q = w * 32u + (uint32_t)__builtin_ctz(bits);
                bits &= bits - 1;
                P[part * N + q] ^= c;
              }
            }
        }
        break;
      }
      case OP_REC_OUT:
        RW[o.i3] = SL[o.i2] & kept;
        break;
      case OP_DETECTOR:
      case OP_OBS_INCLUDE: {
        uint64_t d = 0;
        if (o.pa != kNoInline) {
          for (uint32_t i = 0; i < kInline; i++) d ^= SL[entry(o, i)];
        } else {
          for (uint32_t j = 0; j < o.i1; j++) d ^= SL[slot_list[o.i0 + j]];
        }
        if (o.code == OP_OBS_INCLUDE) SL[o.i2] ^= d;
        else RW[h.n_meas + o.i3] = d & kept;
        break;
      }
      case OP_OBS_OUT:
        RW[h.n_meas + h.n_det + o.i3] = SL[o.i2] & kept;
        break;
      default:  // OP_END, OP_BATCH (payloads run one by one), OP_KEPT_OUT
        break;
    }
    if (o.code == OP_END) break;
  }
}

}  // namespace

// Appends the propagation tables to a compiled blob when the program has no
// active axes and the tables stay under kMaxEntries; otherwise leaves
// aff_ok = 0. Returns the (possibly reallocated) blob through `blob`.
void append_affine(std::vector<uint8_t>& blob) {
  ProgHeader h;
  std::memcpy(&h, blob.data(), sizeof(h));
  if (h.k_max != 0) return;
  Blob b{&h, blob.data()};
  const Op* ops = b.at<Op>(h.off_ops);
  for (uint32_t pc = 0; pc < h.n_ops; pc++)
    if (!supported(ops[pc].code)) return;
  const uint32_t R = h.n_meas + h.n_det + h.n_obs;
  const uint32_t* site_info = b.at<uint32_t>(h.off_site_info);

  // random dormant measurements, in program order
  std::vector<uint32_t> rand_ord(h.n_ops, 0), rand_ev;
  for (uint32_t pc = 0; pc < h.n_ops; pc++)
    if (ops[pc].code == OP_MEAS_RANDOM) {
      rand_ord[pc] = (uint32_t)rand_ev.size();
      rand_ev.push_back(ops[pc].i0);
    }
  // probes: baseline, then one per random measurement, then one per fault option
  struct Item {
    bool is_rand;
    uint32_t a, b;  // rand: ordinal; fault: site, option
  };
  std::vector<Item> items;
  for (uint32_t j = 0; j < rand_ev.size(); j++) items.push_back({true, j, 0});
  for (uint32_t s = 0; s < h.n_sites; s++) {
    const uint32_t k = site_k(site_info[s]);
    for (uint32_t o = 0; o < k; o++) items.push_back({false, s, o});
  }

  Probe base;
  std::vector<uint64_t> zero_rand(rand_ev.size(), 0);
  std::vector<std::vector<std::pair<uint32_t, uint64_t>>> site_faults(h.n_sites);
  run_probe(b, rand_ord, zero_rand, site_faults, base);

  std::vector<std::vector<uint32_t>> rand_rows(rand_ev.size());
  std::vector<uint32_t> col_off((size_t)h.n_sites * kRecPerSite + 1, 0);
  std::vector<std::vector<uint32_t>> col_rows((size_t)h.n_sites * kRecPerSite);
  // Batches of 64 items are independent, and every item's rows go to its
  // own column, so the batches run on several host threads with the same
  // result as one after the other.
  const size_t n_batches = (items.size() + 63) / 64;
  std::atomic<uint64_t> n_entries{0};
  std::atomic<bool> over{false};
  std::exception_ptr failure;
  std::mutex failure_mu;
  auto worker = [&](size_t first, size_t step) {
    try {
      Probe pr;
      std::vector<std::vector<std::pair<uint32_t, uint64_t>>> site_faults(h.n_sites);
      std::vector<uint64_t> rm(rand_ev.size(), 0);
      std::vector<uint32_t> touched;
      for (size_t bi = first; bi < n_batches && !over.load(std::memory_order_relaxed); bi += step) {
        const size_t i0 = bi * 64, n = std::min<size_t>(64, items.size() - i0);
        std::fill(rm.begin(), rm.end(), 0ull);
        touched.clear();
        for (size_t l = 0; l < n; l++) {
          const Item& it = items[i0 + l];
          if (it.is_rand) {
            rm[it.a] |= 1ull << l;
          } else {
            auto& v = site_faults[it.a];
            if (v.empty()) touched.push_back(it.a);
            v.push_back({it.b, 1ull << l});
          }
        }
        run_probe(b, rand_ord, rm, site_faults, pr);
        for (uint32_t s : touched) site_faults[s].clear();
        uint64_t k = 0;
        for (uint32_t r = 0; r < R; r++) {
          uint64_t d = pr.rows[r] ^ base.rows[r];
          while (d) {
            const uint32_t l = (uint32_t)__builtin_ctzll(d);
            d &= d - 1;
            const Item& it = items[i0 + l];
            if (it.is_rand) rand_rows[it.a].push_back(r);
            else col_rows[(size_t)it.a * kRecPerSite + it.b].push_back(r);
            k++;
          }
        }
        if (n_entries.fetch_add(k) + k > kMaxEntries) over = true;
      }
    } catch (...) {
      std::lock_guard<std::mutex> g(failure_mu);
      if (!failure) failure = std::current_exception();
      over = true;
    }
  };
  {
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t n_threads = std::min<size_t>({hw, (size_t)32, std::max<size_t>(1, n_batches / 4)});
    std::vector<std::thread> pool;
    for (size_t t = 1; t < n_threads; t++) pool.emplace_back(worker, t, n_threads);
    worker(0, n_threads);
    for (auto& th : pool) th.join();
  }
  if (failure) std::rethrow_exception(failure);
  if (over) return;

  // ---- delta rows ----
  // A row that shares most of its support with an earlier row is stored as
  // the difference: row r = delta_r ^ row parent(r). Each row is the parent
  // of at most one row, so parents form chains that the sampler resolves
  // with one running XOR per chain and word. In a memory experiment a
  // stabiliser's measurement in round t then differs from round t - 1 by its
  // detector's few faults, instead of carrying every earlier fault.
  constexpr uint32_t kNone = 0xFFFFFFFFu;
  std::vector<uint32_t> parent(R, kNone), child(R, kNone);
  {
    const uint32_t n_cols = (uint32_t)col_rows.size();
    auto rows_of = [&](uint32_t x) -> const std::vector<uint32_t>& {
      return x < n_cols ? col_rows[x] : rand_rows[x - n_cols];
    };
    std::vector<std::vector<uint32_t>> F(R);  // row -> ascending supports (faults, then random events)
    for (uint32_t c = 0; c < n_cols; c++)
      for (uint32_t r : col_rows[c]) F[r].push_back(c);
    for (uint32_t j = 0; j < rand_rows.size(); j++)
      for (uint32_t r : rand_rows[j]) F[r].push_back(n_cols + j);
    // The parent of r is the earlier row without a child that maximises
    // |F_r| - |F_r ^ F_p| = 2 |F_r & F_p| - |F_p| (> 0; the larger p on a
    // tie), so the choice depends only on the overlaps, not on the order
    // they are counted in. For up to kParR rows the overlaps of every row
    // with its earlier rows are counted on several host threads first (the
    // rows of mirror-like circuits share most of their supports, and the
    // counting is the bulk of the work); the greedy choice then runs in
    // row order as before.
    constexpr uint32_t kParR = 4096;
    auto count_overlaps = [&](uint32_t r, std::vector<uint32_t>& cnt, std::vector<uint32_t>& touched,
                              bool skip_children) {
      touched.clear();
      for (uint32_t x : F[r])
        for (uint32_t p : rows_of(x)) {
          if (p >= r) break;
          if (skip_children && child[p] != kNone) continue;
          if (!cnt[p]++) touched.push_back(p);
        }
    };
    auto choose = [&](uint32_t r, uint32_t p, uint32_t overlap, uint32_t& best, int64_t& best_gain) {
      const int64_t gain = 2 * (int64_t)overlap - (int64_t)F[p].size();
      if (gain > best_gain || (gain == best_gain && gain > 0 && p > best)) {
        best_gain = gain;
        best = p;
      }
      (void)r;
    };
    if (R <= kParR) {
      std::vector<std::vector<std::pair<uint32_t, uint32_t>>> ov(R);  // row -> (earlier row, overlap)
      auto counter = [&](uint32_t first, uint32_t step) {
        std::vector<uint32_t> cnt(R, 0), touched;
        for (uint32_t r = first; r < R; r += step) {
          if (F[r].empty()) continue;
          count_overlaps(r, cnt, touched, false);
          ov[r].reserve(touched.size());
          for (uint32_t p : touched) {
            ov[r].push_back({p, cnt[p]});
            cnt[p] = 0;
          }
        }
      };
      const uint32_t hw = std::max(1u, std::thread::hardware_concurrency());
      const uint32_t n_threads = std::min<uint32_t>({hw, 32u, std::max<uint32_t>(1, R / 16)});
      std::vector<std::thread> pool;
      std::exception_ptr err;
      std::mutex err_mu;
      auto guarded = [&](uint32_t first, uint32_t step) {
        try {
          counter(first, step);
        } catch (...) {
          std::lock_guard<std::mutex> g(err_mu);
          if (!err) err = std::current_exception();
        }
      };
      for (uint32_t t = 1; t < n_threads; t++) pool.emplace_back(guarded, t, n_threads);
      guarded(0, n_threads);
      for (auto& th : pool) th.join();
      if (err) std::rethrow_exception(err);
      for (uint32_t r = 0; r < R; r++) {
        uint32_t best = kNone;
        int64_t best_gain = 0;
        for (const auto& po : ov[r])
          if (child[po.first] == kNone) choose(r, po.first, po.second, best, best_gain);
        if (best != kNone) {
          parent[r] = best;
          child[best] = r;
        }
      }
    } else {
      std::vector<uint32_t> cnt(R, 0), touched;
      for (uint32_t r = 0; r < R; r++) {
        if (F[r].empty()) continue;
        count_overlaps(r, cnt, touched, true);
        uint32_t best = kNone;
        int64_t best_gain = 0;
        for (uint32_t p : touched) {
          choose(r, p, cnt[p], best, best_gain);
          cnt[p] = 0;
        }
        if (best != kNone) {
          parent[r] = best;
          child[best] = r;
        }
      }
    }
    // supports in delta form, then the columns again (rows ascending)
    for (auto& v : col_rows) v.clear();
    for (auto& v : rand_rows) v.clear();
    std::vector<uint32_t> d;
    for (uint32_t r = 0; r < R; r++) {
      d.clear();
      if (parent[r] == kNone) d = F[r];
      else std::set_symmetric_difference(F[r].begin(), F[r].end(), F[parent[r]].begin(), F[parent[r]].end(),
                                         std::back_inserter(d));
      for (uint32_t x : d) {
        if (x < n_cols) col_rows[x].push_back(r);
        else rand_rows[x - n_cols].push_back(r);
      }
    }
    // constants in delta form (parents come first: fix from the last row down)
    for (uint32_t r = R; r-- > 0;)
      if (parent[r] != kNone) base.rows[r] ^= base.rows[parent[r]];
  }
  // chains, head first: every row lies on exactly one (a row with neither
  // parent nor child is a chain of one), longest chains first, so that the
  // chains one warp resolves side by side have about the same length
  std::vector<uint32_t> chain_off, chain;
  {
    std::vector<std::vector<uint32_t>> chs;
    for (uint32_t r = 0; r < R; r++) {
      if (parent[r] != kNone) continue;
      chs.emplace_back();
      for (uint32_t x = r; x != kNone; x = child[x]) chs.back().push_back(x);
    }
    std::stable_sort(chs.begin(), chs.end(),
                     [](const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) { return a.size() > b.size(); });
    for (const auto& c : chs) {
      chain_off.push_back((uint32_t)chain.size());
      chain.insert(chain.end(), c.begin(), c.end());
    }
  }
  const uint32_t n_chains = (uint32_t)chain_off.size();
  chain_off.push_back((uint32_t)chain.size());

  // row-major random-event lists
  std::vector<uint32_t> rowev_off(R + 1, 0), rowev;
  {
    std::vector<std::vector<uint32_t>> per_row(R);
    for (uint32_t j = 0; j < rand_rows.size(); j++)
      for (uint32_t r : rand_rows[j]) per_row[r].push_back(j);
    for (uint32_t r = 0; r < R; r++) {
      // the sampler packs a row's term count in 7 bits and its first entry
      // in 24 (the bytecode executor serves programs beyond that)
      if (per_row[r].size() >= 128) return;
      rowev_off[r] = (uint32_t)rowev.size();
      rowev.insert(rowev.end(), per_row[r].begin(), per_row[r].end());
    }
    rowev_off[R] = (uint32_t)rowev.size();
    if (rowev.size() >= (1u << 24)) return;
  }
  // fault columns in chunks of 8 u16 chain positions (the sampler keeps
  // row chain[j] at position j of its tile; padding: R)
  if (R >= 0xFFFFu) return;
  std::vector<uint32_t> pos_of(R);
  for (uint32_t j = 0; j < (uint32_t)chain.size(); j++) pos_of[chain[j]] = j;
  std::vector<uint16_t> chunks;
  for (size_t c = 0; c < col_rows.size(); c++) {
    col_off[c] = (uint32_t)(chunks.size() / 8);
    const auto& rows = col_rows[c];
    for (size_t j = 0; j < rows.size(); j += 8)
      for (size_t e = 0; e < 8; e++) chunks.push_back((uint16_t)(j + e < rows.size() ? pos_of[rows[j + e]] : R));
  }
  col_off[col_rows.size()] = (uint32_t)(chunks.size() / 8);
  if (chunks.size() / 8 >= (1u << 22)) return;
  // expected chunks per shot: sum over sites of p * mean chunk count of its options
  double cps = 0.0;
  {
    const uint64_t* q = b.at<uint64_t>(h.off_q);
    const uint32_t* seg_start = b.at<uint32_t>(h.off_seg_start);
    for (uint32_t s = 0; s < h.n_sites; s++) {
      // the site's probability from consecutive survival thresholds
      const double qs = (double)q[s] * 0x1p-64;
      const double qp = seg_start[s] == s ? 1.0 : (double)q[s - 1] * 0x1p-64;
      const double p = qp > 0.0 ? 1.0 - qs / qp : 0.0;
      const uint32_t kk = site_k(site_info[s]);
      double mean = 0.0;
      for (uint32_t o = 0; o < kk; o++)
        mean += col_off[(size_t)s * kRecPerSite + o + 1] - col_off[(size_t)s * kRecPerSite + o];
      cps += p * (kk ? mean / kk : 0.0);
    }
  }
  std::vector<uint32_t> cst(R);
  for (uint32_t r = 0; r < R; r++) cst[r] = (uint32_t)(base.rows[r] & 1ull);

  uint64_t off = h.total_bytes;
  auto place = [&](uint64_t bytes) {
    uint64_t o = off;
    off = (off + bytes + 15) & ~15ull;
    return o;
  };
  h.off_aff_const = place((uint64_t)R * 4);
  h.off_aff_rowev_off = place((uint64_t)(R + 1) * 4);
  h.off_aff_rowev = place((uint64_t)rowev.size() * 4);
  h.off_aff_rand_ev = place((uint64_t)rand_ev.size() * 4);
  // per-site fault records: option chunk counts as nibbles, K, first chunk
  std::vector<uint32_t> frec((size_t)h.n_sites * 4, 0);
  for (uint32_t s = 0; s < h.n_sites; s++) {
    const uint32_t kk = site_k(site_info[s]);
    uint64_t nib = 0;
    bool long_site = false;
    for (uint32_t o = 0; o < kk; o++) {
      const uint32_t n = col_off[(size_t)s * kRecPerSite + o + 1] - col_off[(size_t)s * kRecPerSite + o];
      if (n > 15) long_site = true;
      nib |= (uint64_t)(n & 15u) << (4 * o);
    }
    nib |= (uint64_t)kk << 60;
    frec[4 * s] = (uint32_t)nib;
    frec[4 * s + 1] = (uint32_t)(nib >> 32);
    frec[4 * s + 2] = long_site ? 0xFFFFFFFFu : col_off[(size_t)s * kRecPerSite];
  }
  h.off_aff_col_off = place((uint64_t)col_off.size() * 4);
  h.off_aff_col = place((uint64_t)chunks.size() * 2);
  h.off_aff_frec = place((uint64_t)frec.size() * 4);
  h.off_aff_parent = place((uint64_t)R * 4);
  h.off_aff_chain_off = place((uint64_t)chain_off.size() * 4);
  h.off_aff_chain = place((uint64_t)chain.size() * 4);
  h.aff_n_chains = n_chains;
  h.aff_n_chain_rows = (uint32_t)chain.size();
  h.total_bytes = off;
  h.aff_ok = 1;
  h.aff_rows = R;
  h.aff_n_rand = (uint32_t)rand_ev.size();
  h.aff_n_chunks = (uint32_t)(chunks.size() / 8);
  h.aff_chunks_per_shot = (float)cps;
  blob.resize(off, 0);
  auto cp = [&](uint64_t o, const void* src, size_t bytes) {
    if (bytes) std::memcpy(blob.data() + o, src, bytes);
  };
  cp(h.off_aff_const, cst.data(), cst.size() * 4);
  cp(h.off_aff_rowev_off, rowev_off.data(), rowev_off.size() * 4);
  cp(h.off_aff_rowev, rowev.data(), rowev.size() * 4);
  cp(h.off_aff_rand_ev, rand_ev.data(), rand_ev.size() * 4);
  cp(h.off_aff_col_off, col_off.data(), col_off.size() * 4);
  cp(h.off_aff_col, chunks.data(), chunks.size() * 2);
  cp(h.off_aff_frec, frec.data(), frec.size() * 4);
  cp(h.off_aff_parent, parent.data(), parent.size() * 4);
  cp(h.off_aff_chain_off, chain_off.data(), chain_off.size() * 4);
  cp(h.off_aff_chain, chain.data(), chain.size() * 4);
  std::memcpy(blob.data(), &h, sizeof(h));
}

}  // namespace nc
