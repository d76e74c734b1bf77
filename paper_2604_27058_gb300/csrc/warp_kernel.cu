// warp_kernel.cu — the warp-per-shot layout of the sample-many phase
// (Sec. 3.2): exec_warp<real, NW> runs every shot on one warp.
//
// A CTA of up to 8 warps takes a 32-shot record word (a tile) at a time; its
// warps pull the tile's shots from a shared counter and run each through the
// plain instruction list, one shot per warp at a time:
//   * the shot's active vector (2^k_max amplitudes of `real`) lives in the
//     warp's slice of shared memory, and every array instruction is a loop of
//     the warp's 32 lanes over amplitude pairs;
//   * the virtual frame (x, z bits of at most 32 NW virtual qubits) sits in
//     registers, the same copy in every lane, so frame instructions and
//     noise need no shared state and no synchronisation;
//   * measurement and probe sums are accumulated in FP64 per lane and reduced
//     by a butterfly of warp shuffles (every lane ends with the same total,
//     so every lane draws the same outcome);
//   * record slots are bits in shared memory that only lane 0 touches; record
//     outputs are bits of the tile's output words in shared memory, written
//     to the record rows once per tile;
//   * a shot rejected by postselection stops at its failing detector (its
//     later records are 0 by definition), unless probes or a debug stop need
//     the rest of the instruction list.
// The vectors never leave the SM, and a shot's instruction dispatch is paid
// by one warp. The random draws and fault sets are those of the other
// executors (kernels.cuh), so the records are the same shot by shot.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace nc {

namespace {

constexpr uint32_t kFull = 0xffffffffu;

template <typename R>
struct Cw;
template <>
struct Cw<float> {
  using T = float2;
};
template <>
struct Cw<double> {
  using T = double2;
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (uint32_t d = 16; d; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

// Bit q of a frame held as NW register words (the same in every lane).
template <int NW>
__device__ __forceinline__ uint32_t fget(const uint32_t (&v)[NW], uint32_t q) {
  const uint32_t w = q >> 5;
  uint32_t x = v[0];
#pragma unroll
  for (int i = 1; i < NW; i++)
    if (w == (uint32_t)i) x = v[i];
  return (x >> (q & 31u)) & 1u;
}
template <int NW>
__device__ __forceinline__ void fflip(uint32_t (&v)[NW], uint32_t q, uint32_t b) {
  const uint32_t w = q >> 5, m = b << (q & 31u);
#pragma unroll
  for (int i = 0; i < NW; i++)
    if (w == (uint32_t)i) v[i] ^= m;
}
template <int NW>
__device__ __forceinline__ void fset(uint32_t (&v)[NW], uint32_t q, uint32_t b) {
  fflip<NW>(v, q, fget<NW>(v, q) ^ b);
}

}  // namespace

// Shared memory of one CTA of `nwarps` warps: the tile's output words (meas,
// det, obs rows, then the kept row), two counters, the instruction list when
// it is staged (at most kWarpStageOps instructions), then per warp its
// vector and its record-slot bits.
constexpr uint32_t kWarpStageOps = 1536;  // 48 KB of instructions
struct WarpLayout {
  uint32_t rows, slot_words;
  bool staged;
  size_t vec_bytes, warp_bytes, head_bytes, ops_bytes, bytes;
};
__host__ __device__ inline WarpLayout warp_layout(const DevProg& p, bool fp64, uint32_t nwarps) {
  WarpLayout w;
  w.rows = p.n_meas + p.n_det + p.n_obs + 1;
  w.slot_words = (p.n_slots + 1 + 31) / 32;
  w.staged = p.n_ops <= kWarpStageOps;
  w.vec_bytes = ((size_t)1 << p.k_max) * (fp64 ? 16 : 8);
  w.warp_bytes = (w.vec_bytes + (size_t)w.slot_words * 4 + 15) & ~(size_t)15;
  w.head_bytes = ((size_t)(w.rows + 2) * 4 + 15) & ~(size_t)15;
  w.ops_bytes = w.staged ? (size_t)p.n_ops * sizeof(Op) : 0;
  w.bytes = w.head_bytes + w.ops_bytes + (size_t)nwarps * w.warp_bytes;
  return w;
}

template <typename real, int NW>
__global__ void __launch_bounds__(256, 3) exec_warp(LaunchParams L) {
  using C = typename Cw<real>::T;
  extern __shared__ __align__(16) unsigned char wsm[];
  const DevProg& p = L.p;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const WarpLayout lay = warp_layout(p, sizeof(real) == 8, nwarps);
  uint32_t* REC = reinterpret_cast<uint32_t*>(wsm);  // [rows] output words of the tile
  uint32_t* CTR = REC + lay.rows;                     // [0] next shot of the tile, [1] kept shots
  const Op* OPS = lay.staged ? reinterpret_cast<const Op*>(wsm + lay.head_bytes) : p.ops;
  unsigned char* mine = wsm + lay.head_bytes + lay.ops_bytes + (size_t)warp * lay.warp_bytes;
  C* V = reinterpret_cast<C*>(mine);
  uint32_t* SLW = reinterpret_cast<uint32_t*>(mine + lay.vec_bytes);  // record slots (lane 0 only)
  const uint32_t r_det = p.n_meas, r_obs = p.n_meas + p.n_det, r_kept = lay.rows - 1;
  const bool noisy = !(L.flags & LF_NOISELESS) && p.n_sites > 0;
  const bool can_stop = !(L.flags & LF_OUT_EXPVAL) && L.stop_event == 0xffffffffu;
  const real rs = (real)0.70710678118654752440;

  for (uint32_t i = threadIdx.x; i < lay.rows + 2; i += blockDim.x) REC[i] = 0;
  if (lay.staged) {
    const uint4* src = reinterpret_cast<const uint4*>(p.ops);
    uint4* dst = reinterpret_cast<uint4*>(wsm + lay.head_bytes);
    for (uint32_t i = threadIdx.x; i < 2 * p.n_ops; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  for (uint64_t tile = blockIdx.x; tile < L.row_words32; tile += gridDim.x) {
    for (;;) {
      uint32_t j = 0;
      if (lane == 0) j = atomicAdd(CTR, 1u);
      j = __shfl_sync(kFull, j, 0);
      if (j >= 32) break;
      const uint64_t sl = tile * 32u + j;  // call-local shot
      if (sl >= L.shots) continue;
      const uint64_t s = L.shot_offset + sl, s0 = s & ~31ull;  // s & 31 == j (offsets are 128-aligned)
      const uint32_t bit = 1u << j;
      uint32_t x[NW], z[NW];
#pragma unroll
      for (int i = 0; i < NW; i++) x[i] = z[i] = 0;
      if (lane == 0)
        for (uint32_t w = 0; w < lay.slot_words; w++) SLW[w] = 0;
      uint32_t kept = 1, k = 0;
      if (p.k_max > 0 && lane == 0) {
        C one;
        one.x = (real)1;
        one.y = (real)0;
        V[0] = one;
      }
      uint32_t nr = p.sg_k;  // stratified: faults the shot still holds
      uint32_t nf = noisy ? next_fault_r(p, L.seed, s, 0, nr) : kNoFault;
      __syncwarp();
      // record slots: lane 0 reads and writes them; values go to every lane by shuffle
      auto slot = [&](uint32_t i) -> uint32_t {
        uint32_t v = 0;
        if (lane == 0) v = (SLW[i >> 5] >> (i & 31u)) & 1u;
        return __shfl_sync(kFull, v, 0);
      };
      auto setslot = [&](uint32_t i, uint32_t b) {
        if (lane == 0) SLW[i >> 5] = (SLW[i >> 5] & ~(1u << (i & 31u))) | (b << (i & 31u));
      };
      auto slots_xor = [&](uint32_t off, uint32_t n) -> uint32_t {
        uint32_t d = 0;
        if (lane == 0)
          for (uint32_t q = 0; q < n; q++) {
            const uint32_t i = __ldg(p.slot_list + off + q);
            d ^= (SLW[i >> 5] >> (i & 31u)) & 1u;
          }
        return __shfl_sync(kFull, d, 0);
      };
      auto rec = [&](uint32_t row, uint32_t b) {
        if (lane == 0 && b) atomicOr(REC + row, bit);
      };
      // frame ^= the mask at offset off (x words, then z words)
      auto fmask = [&](uint32_t off) {
#pragma unroll
        for (int w = 0; w < NW; w++)
          if ((uint32_t)w < p.nw) {
            x[w] ^= __ldg(p.masks + off + w);
            z[w] ^= __ldg(p.masks + off + p.nw + w);
          }
      };

      Op nxt = OPS[0];  // the next instruction is read while this one runs
      for (uint32_t pc = 0; pc < p.n_ops; pc++) {
        const Op op = nxt;
        if (pc + 1 < p.n_ops) nxt = OPS[pc + 1];
        const uint8_t code = op.code;
        if (L.stop_event != 0xffffffffu &&
            (code == OP_MEAS_STATIC || code == OP_MEAS_RANDOM || code == OP_MEAS_ACTIVE_Z ||
             code == OP_MEAS_ACTIVE_X) &&
            op.i1 == L.stop_event) {
          if (sl == L.dump_shot) {
            if (lane == 0) {
#pragma unroll
              for (int w = 0; w < NW; w++)
                if ((uint32_t)w < p.nw) {
                  L.dump_frame[w] = x[w];
                  L.dump_frame[p.nw + w] = z[w];
                }
              *L.dump_k = k;
            }
            for (uint32_t i = lane; i < (1u << k); i += 32) {
              L.dump_amps[2 * i] = (double)V[i].x;
              L.dump_amps[2 * i + 1] = (double)V[i].y;
            }
          }
          break;
        }
        const uint32_t pa = op.pa;
        bool stop = false;
        switch (code) {
          case OP_FRAME_H:
          case OP_ARRAY_H: {
            const uint32_t xa = fget<NW>(x, op.a);
            fset<NW>(x, op.a, fget<NW>(z, op.a));
            fset<NW>(z, op.a, xa);
            if (code == OP_ARRAY_H) {
              for (uint32_t jj = lane; jj < (1u << (k - 1)); jj += 32) {
                const uint32_t i0 = insert0(jj, pa), i1 = i0 | (1u << pa);
                const C a = V[i0], b = V[i1];
                C u, v;
                u.x = (a.x + b.x) * rs;
                u.y = (a.y + b.y) * rs;
                v.x = (a.x - b.x) * rs;
                v.y = (a.y - b.y) * rs;
                V[i0] = u;
                V[i1] = v;
              }
              __syncwarp();
            }
            break;
          }
          case OP_FRAME_S:
          case OP_ARRAY_S:
            fflip<NW>(z, op.a, fget<NW>(x, op.a));
            if (code == OP_ARRAY_S) {
              for (uint32_t jj = lane; jj < (1u << (k - 1)); jj += 32) {
                const uint32_t i1 = insert0(jj, pa) | (1u << pa);
                const C a = V[i1];
                C u;
                u.x = -a.y;
                u.y = a.x;
                V[i1] = u;
              }
              __syncwarp();
            }
            break;
          case OP_FRAME_CX:
          case OP_ARRAY_CX:
            fflip<NW>(x, op.b, fget<NW>(x, op.a));
            fflip<NW>(z, op.a, fget<NW>(z, op.b));
            if (code == OP_ARRAY_CX) {
              const uint32_t lo = min(pa, (uint32_t)op.pb), hi = max(pa, (uint32_t)op.pb);
              for (uint32_t jj = lane; jj < (1u << (k - 2)); jj += 32) {
                const uint32_t i0 = insert0(insert0(jj, lo), hi) | (1u << pa), i1 = i0 | (1u << op.pb);
                const C a = V[i0];
                V[i0] = V[i1];
                V[i1] = a;
              }
              __syncwarp();
            }
            break;
          case OP_FRAME_CZ:
          case OP_ARRAY_CZ: {
            const uint32_t xa = fget<NW>(x, op.a), xb = fget<NW>(x, op.b);
            fflip<NW>(z, op.a, xb);
            fflip<NW>(z, op.b, xa);
            if (code == OP_ARRAY_CZ) {
              const uint32_t lo = min(pa, (uint32_t)op.pb), hi = max(pa, (uint32_t)op.pb);
              for (uint32_t jj = lane; jj < (1u << (k - 2)); jj += 32) {
                const uint32_t i = insert0(insert0(jj, lo), hi) | (1u << pa) | (1u << op.pb);
                C a = V[i];
                a.x = -a.x;
                a.y = -a.y;
                V[i] = a;
              }
              __syncwarp();
            }
            break;
          }
          case OP_EXPAND_ROT: {
            const real c2 = (real)(op.cs * 0.70710678118654752440);
            const real s2 = (real)((fget<NW>(x, op.a) ? -op.sn : op.sn) * 0.70710678118654752440);
            const uint32_t n = 1u << k;
            for (uint32_t i = lane; i < n; i += 32) {
              const C u = V[i];
              C a, b;
              a.x = u.x * rs;
              a.y = u.y * rs;
              b.x = u.x * c2 - u.y * s2;
              b.y = u.x * s2 + u.y * c2;
              V[i] = a;
              V[i + n] = b;
            }
            k++;
            __syncwarp();
            break;
          }
          case OP_ROT_Z: {
            const real c2 = (real)op.cs, s2 = (real)(fget<NW>(x, op.a) ? -op.sn : op.sn);
            for (uint32_t jj = lane; jj < (1u << (k - 1)); jj += 32) {
              const uint32_t i1 = insert0(jj, pa) | (1u << pa);
              const C u = V[i1];
              C v;
              v.x = u.x * c2 - u.y * s2;
              v.y = u.x * s2 + u.y * c2;
              V[i1] = v;
            }
            __syncwarp();
            break;
          }
          case OP_ROT_X: {
            const real c1 = (real)op.cs, s1 = (real)(fget<NW>(z, op.a) ? -op.sn : op.sn);
            for (uint32_t jj = lane; jj < (1u << (k - 1)); jj += 32) {
              const uint32_t i0 = insert0(jj, pa), i1 = i0 | (1u << pa);
              const C a = V[i0], b = V[i1];
              C u, v;
              u.x = c1 * a.x + s1 * b.y;
              u.y = c1 * a.y - s1 * b.x;
              v.x = s1 * a.y + c1 * b.x;
              v.y = -s1 * a.x + c1 * b.y;
              V[i0] = u;
              V[i1] = v;
            }
            __syncwarp();
            break;
          }
          case OP_MEAS_STATIC: {
            uint32_t par = (op.flags & FLAG_SIGN) ? 1u : 0u;
#pragma unroll
            for (int w = 0; w < NW; w++)
              if ((uint32_t)w < p.nw) par ^= __popc(x[w] & __ldg(p.masks + op.i0 + w)) & 1u;
            if (op.flags & FLAG_RESET) {
              // fused reset: conditional X-image on the inline planes r[0..pb)
              for (uint32_t r = 0; r < op.pb; r++) {
                const uint32_t pl = ((r < 2 ? op.i2 : op.i3) >> (16 * (r & 1u))) & 0xFFFFu;
                if (pl < p.n_qubits) fflip<NW>(x, pl, par);
                else fflip<NW>(z, pl - p.n_qubits, par);
              }
            } else {
              setslot(op.i2, par);
              if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) rec(op.i3, par & kept);
            }
            break;
          }
          case OP_MEAS_RANDOM: {
            const uint32_t top = (meas_top_word(L.seed, s0, op.i0) >> j) & 1u;
            const uint32_t m = (L.flags & LF_ARGMAX) ? 0u : top ^ 1u;
            const uint32_t b = m ^ ((op.flags & FLAG_SIGN) ? 1u : 0u) ^ fget<NW>(z, op.a);
            const uint32_t xa = fget<NW>(x, op.a);
            fset<NW>(x, op.a, fget<NW>(z, op.a) ^ b);
            fset<NW>(z, op.a, xa);
            setslot(op.i2, m);
            if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) rec(op.i3, m & kept);
            break;
          }
          case OP_MEAS_ACTIVE_Z:
          case OP_MEAS_ACTIVE_X: {
            const bool xm = code == OP_MEAS_ACTIVE_X;
            const uint32_t half = 1u << (k - 1), top_pos = k - 1;
            double a0 = 0.0, a1 = 0.0;
            for (uint32_t jj = lane; jj < half; jj += 32) {
              const uint32_t i0 = insert0(jj, pa), i1 = i0 | (1u << pa);
              const C u = V[i0], v = V[i1];
              if (xm) {
                mterm_x(u, v, a0, a1);
              } else {
                a0 += mterm(u);
                a1 += mterm(v);
              }
            }
            // sums down to lane 0, which alone does the scalar FP64 work
            // (probability, draw, 1 / sqrt(S_b)): FP64 lanes are scarce
#pragma unroll
            for (uint32_t d = 16; d; d >>= 1) {
              const double b0 = __shfl_down_sync(kFull, a0, d), b1 = __shfl_down_sync(kFull, a1, d);
              if (lane < d) {
                a0 += b0;
                a1 += b1;
              }
            }
            const uint32_t pbit = xm ? fget<NW>(z, op.a) : fget<NW>(x, op.a);
            const uint32_t abit = (op.flags & FLAG_SIGN) ? 1u : 0u;
            uint32_t m = 0;
            real sc = (real)0;
            if (lane == 0) {
              const double S0 = a0, S1 = a1, tot = S0 + S1;
              const double p1 = tot > 0.0 ? ((1u ^ abit ^ pbit) ? S1 : S0) / tot : 0.0;
              const uint32_t top = (meas_top_word(L.seed, s0, op.i0) >> j) & 1u;
              m = (L.flags & LF_ARGMAX) ? (p1 > 0.5 ? 1u : 0u) : draw_outcome(L.seed, s, op.i0, top, p1);
              const double sb = (m ^ abit ^ pbit) ? S1 : S0;
              sc = (real)(sb > 0.0 ? 1.0 / sqrt(sb) : 0.0);
            }
            m = __shfl_sync(kFull, m, 0);
            sc = __shfl_sync(kFull, sc, 0);
            const uint32_t b = m ^ abit ^ pbit;
            if (pa == top_pos) {
              for (uint32_t jj = lane; jj < half; jj += 32) {
                const C o0 = V[jj], o1 = V[jj + half];
                C v;
                if (xm) {
                  const real sg = b ? (real)-1 : (real)1;
                  v.x = (o0.x + sg * o1.x) * rs;
                  v.y = (o0.y + sg * o1.y) * rs;
                } else {
                  v = b ? o1 : o0;
                }
                v.x *= sc;
                v.y *= sc;
                V[jj] = v;
              }
            } else {
              for (uint32_t jj = lane; jj < (1u << (k - 2)); jj += 32) {
                const uint32_t base = insert0(insert0(jj, pa), top_pos);
                const uint32_t p00 = base, p10 = base | (1u << pa), p01 = base | (1u << top_pos),
                               p11 = p10 | (1u << top_pos);
                C n0, n1;
                if (xm) {
                  const C o00 = V[p00], o10 = V[p10], o01 = V[p01], o11 = V[p11];
                  const real sg = b ? (real)-1 : (real)1;
                  n0.x = (o00.x + sg * o10.x) * rs;
                  n0.y = (o00.y + sg * o10.y) * rs;
                  n1.x = (o01.x + sg * o11.x) * rs;
                  n1.y = (o01.y + sg * o11.y) * rs;
                } else {
                  n0 = b ? V[p10] : V[p00];
                  n1 = b ? V[p11] : V[p01];
                }
                n0.x *= sc;
                n0.y *= sc;
                n1.x *= sc;
                n1.y *= sc;
                V[p00] = n0;
                V[p10] = n1;
              }
            }
            __syncwarp();
            k--;
            setslot(op.i2, m);
            if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) rec(op.i3, m & kept);
            if (xm) {
              const uint32_t xa = fget<NW>(x, op.a);
              fset<NW>(x, op.a, fget<NW>(z, op.a) ^ b);
              fset<NW>(z, op.a, xa);
            } else {
              fflip<NW>(x, op.a, b);
            }
            break;
          }
          case OP_NOISE_BLOCK:
            while ((nf >> 4) < op.i1) {
              const uint32_t site = nf >> 4, opt = nf & 15u;
              const uint32_t info = __ldg(p.site_info + site), eff = __ldg(p.site_eff + site);
              if ((info & 15u) == SITE_FLIP) {
                if (lane == 0) SLW[eff >> 5] ^= 1u << (eff & 31u);
                if ((L.flags & LF_OUT_MEAS) && kept && lane == 0)
                  atomicXor(REC + __ldg(p.opt_tab + 2 * (info >> 8) + 1), bit);
              } else {
                fmask(eff + opt * 2u * p.nw);
              }
              nf = next_fault_r(p, L.seed, s, site + 1, nr);
            }
            break;
          case OP_EXPVAL: {
            // (-1)^(frame sign) Re(i^pa <phi| X^i1 Z^i2 |phi>) / <phi|phi>
            if (!(L.flags & LF_OUT_EXPVAL)) break;
            double v = 0.0;
            if (!op.pb && kept) {
              const bool odd = (op.pa & 1u) != 0;
              double part = odd ? 0.0 : 1.0;
              if (k > 0) {
                double acc = 0.0, nrm = 0.0;
                for (uint32_t jj = lane; jj < (1u << k); jj += 32) {
                  const C a = V[jj], b = V[jj ^ op.i1];
                  const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
                  const double t1 = odd ? bx * ay - by * ax : bx * ax + by * ay;
                  acc += (__popc(jj & op.i2) & 1u) ? -t1 : t1;
                  nrm += ax * ax + ay * ay;
                }
                acc = wsum(acc);
                nrm = wsum(nrm);
                part = nrm > 0.0 ? acc / nrm : 0.0;
              }
              uint32_t om = 0;
#pragma unroll
              for (int w = 0; w < NW; w++)
                if ((uint32_t)w < p.nw)
                  om ^= __popc(x[w] & __ldg(p.masks + op.i0 + p.nw + w)) ^ __popc(z[w] & __ldg(p.masks + op.i0 + w));
              const double sg = (op.pa == 1 || op.pa == 2) ? -1.0 : 1.0;
              v = (om & 1u) ? -sg * part : sg * part;
            }
            if (lane == 0) L.expval[(size_t)op.i3 * L.shots + sl] = v;
            break;
          }
          case OP_FEEDFORWARD:
            if (slot(op.i2)) fmask(op.i0);
            break;
          case OP_REC_OUT:
            if (L.flags & LF_OUT_MEAS) rec(op.i3, slot(op.i2) & kept);
            break;
          case OP_DETECTOR: {
            uint32_t d = slots_xor(op.i0, op.i1);
            if (!(L.flags & LF_REFERENCE)) d ^= __ldg(p.det_ref + op.i3) ? 1u : 0u;
            if (L.flags & LF_OUT_DET) rec(r_det + op.i3, d & kept);
            if ((L.flags & LF_POSTSELECT) && d) {
              kept = 0;
              stop = can_stop;  // later records of a rejected shot are 0
            }
            break;
          }
          case OP_OBS_INCLUDE:
            if (lane == 0) {
              uint32_t d = 0;
              for (uint32_t q = 0; q < op.i1; q++) {
                const uint32_t i = __ldg(p.slot_list + op.i0 + q);
                d ^= (SLW[i >> 5] >> (i & 31u)) & 1u;
              }
              SLW[op.i2 >> 5] ^= d << (op.i2 & 31u);
            }
            break;
          case OP_OBS_OUT:
            if (L.flags & LF_OUT_OBS) {
              uint32_t v = slot(op.i2);
              if (!(L.flags & LF_REFERENCE)) v ^= __ldg(p.obs_ref + op.i3) ? 1u : 0u;
              rec(r_obs + op.i3, v & kept);
            }
            break;
          case OP_KEPT_OUT:
            if (L.flags & LF_OUT_KEPT) rec(r_kept, kept);
            if (lane == 0 && kept) atomicAdd(CTR + 1, 1u);
            break;
          default:
            break;
        }
        if (stop) break;
      }
      __syncwarp();
    }
    __syncthreads();
    // the tile's output words: word `tile` of every record row
    for (uint32_t r = threadIdx.x; r < lay.rows; r += blockDim.x) {
      const uint32_t v = REC[r];
      REC[r] = 0;
      uint32_t* dst = nullptr;
      if (r < r_det) {
        if (L.flags & LF_OUT_MEAS) dst = L.meas + (size_t)r * L.row_words32;
      } else if (r < r_obs) {
        if (L.flags & LF_OUT_DET) dst = L.det + (size_t)(r - r_det) * L.row_words32;
      } else if (r < r_kept) {
        if (L.flags & LF_OUT_OBS) dst = L.obs + (size_t)(r - r_obs) * L.row_words32;
      } else if (L.flags & LF_OUT_KEPT) {
        dst = L.kept;
      }
      if (dst) dst[tile] = v;
    }
    if (threadIdx.x == 0) {
      if (CTR[1]) atomicAdd(L.kept_count, (unsigned long long)CTR[1]);
      CTR[0] = 0;
      CTR[1] = 0;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Host side (capi.cu)
// ---------------------------------------------------------------------------
// The frame must fit NW = 4 register words (at most 128 virtual qubits).
bool warp_supported(const DevProg& p) { return p.nw <= 4; }

size_t warp_smem_bytes(const DevProg& p, bool fp64, uint32_t nwarps) { return warp_layout(p, fp64, nwarps).bytes; }

template <typename real, int NW>
static cudaError_t warp_one(const LaunchParams& L, uint32_t nwarps, uint32_t grid, size_t smem, cudaStream_t st,
                            int* per_sm) {
  auto fn = exec_warp<real, NW>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (per_sm) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, (int)(32 * nwarps), smem);
  fn<<<grid, 32 * nwarps, smem, st>>>(L);
  return cudaGetLastError();
}

template <typename real>
static cudaError_t warp_t(const LaunchParams& L, uint32_t nwarps, uint32_t grid, size_t smem, cudaStream_t st,
                          int* per_sm) {
  if (L.p.nw <= 1) return warp_one<real, 1>(L, nwarps, grid, smem, st, per_sm);
  if (L.p.nw <= 2) return warp_one<real, 2>(L, nwarps, grid, smem, st, per_sm);
  if (L.p.nw <= 4) return warp_one<real, 4>(L, nwarps, grid, smem, st, per_sm);
  return cudaErrorInvalidValue;
}

// Launch exec_warp on `grid` CTAs of `nwarps` warps (per_sm != null: report
// resident CTAs per SM instead).
cudaError_t launch_warp(const LaunchParams& L, bool fp64, uint32_t nwarps, uint32_t grid, size_t smem,
                        cudaStream_t st, int* per_sm) {
  if (nwarps < 1 || nwarps > 8) return cudaErrorInvalidValue;
  return fp64 ? warp_t<double>(L, nwarps, grid, smem, st, per_sm) : warp_t<float>(L, nwarps, grid, smem, st, per_sm);
}

}  // namespace nc
