// kernels.cu — the online sample-many phase on the GPU (Sec. 3.2).
//
// exec_batched<real>: one CTA runs a tile of 32*G shots. The virtual Pauli
//   frame and the record slots are bit-sliced over shots in shared memory
//   (word w of plane q holds bit q of the frame for the 32 shots of word w);
//   frame, noise, measurement-parity and record instructions are executed by
//   the G word-owner threads, one 32-shot word each, with no synchronisation.
//   Active-array instructions (expand, rotations, array Cliffords, active
//   measurements) run on all threads over (amplitude, shot) pairs of the
//   tile's amplitude block in global memory, laid out amplitude-major /
//   shot-minor so that consecutive threads touch consecutive shots.
//   Measurement probabilities are accumulated in FP64; amplitudes are
//   stored in `real` (float for the batched form).
//
// exec_plain: the baseline form — one thread per shot, frame and record bits
//   in thread-local arrays, FP64 amplitudes in global memory, instructions
//   read straight from global memory.
//
// Both interpret the same bytecode (program.h) and follow the same random-
// draw contract (kernels.cuh), so they produce identical records.
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace nc {

template <typename R>
struct Cx;
template <>
struct Cx<float> {
  using T = float2;
};
template <>
struct Cx<double> {
  using T = double2;
};

template <typename C>
__device__ __forceinline__ C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C, typename R>
__device__ __forceinline__ C cscale(C a, R s) {
  C r;
  r.x = a.x * s;
  r.y = a.y * s;
  return r;
}
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) {
  C r;
  r.x = a.x + b.x;
  r.y = a.y + b.y;
  return r;
}
template <typename C>
__device__ __forceinline__ C csub(C a, C b) {
  C r;
  r.x = a.x - b.x;
  r.y = a.y - b.y;
  return r;
}
template <typename C>
__device__ __forceinline__ double cnorm2(C a) {
  double x = (double)a.x, y = (double)a.y;
  return x * x + y * y;
}

__device__ __forceinline__ bool is_meas(uint8_t c) {
  return c == OP_MEAS_STATIC || c == OP_MEAS_RANDOM || c == OP_MEAS_ACTIVE_Z || c == OP_MEAS_ACTIVE_X;
}

// ---------------------------------------------------------------------------
// Batched executor
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(1024) exec_batched(LaunchParams L) {
  using C = typename Cx<real>::T;
  extern __shared__ __align__(16) uint32_t smem[];
  const DevProg& p = L.p;
  const uint32_t G = L.G, S = 32u * G, N = p.n_qubits, T = blockDim.x, t = threadIdx.x;
  uint32_t* X = smem;                  // [N][G]
  uint32_t* Z = X + N * G;             // [N][G]
  uint32_t* SL = Z + N * G;            // [n_slots][G]
  uint32_t* TMP = SL + p.n_slots * G;  // [G]
  size_t red_off = ((size_t)(2 * N + p.n_slots + 1) * G + 1) & ~(size_t)1;
  double* RED = reinterpret_cast<double*>(smem + red_off);  // [2][S] when k_max > 0
  C* work = reinterpret_cast<C*>(L.work) + (size_t)blockIdx.x * L.work_stride;

  const bool owner = t < G;
  const uint32_t R = T >= S ? T / S : 1u;  // threads per shot in array loops
  const uint32_t sub = T >= S ? t / S : 0u;
  const uint32_t noiseless = L.flags & LF_NOISELESS;

  for (uint32_t tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
    const uint64_t my_word = (uint64_t)tile * G + t;
    const bool word_ok = owner && my_word < L.row_words32;
    const uint64_t s0_local = my_word * 32u;
    const uint64_t s0 = L.shot_offset + s0_local;
    uint32_t valid = 0;
    if (word_ok) {
      if (s0_local + 32 <= L.shots) valid = ~0u;
      else if (s0_local < L.shots) valid = (1u << (uint32_t)(L.shots - s0_local)) - 1u;
    }
    uint32_t* nf = L.nf + ((size_t)blockIdx.x * S) + (size_t)t * 32u;
    uint32_t minsite = kNoFault >> 4;
    if (owner) {
      for (uint32_t q = 0; q < N; q++) {
        X[q * G + t] = 0;
        Z[q * G + t] = 0;
      }
      for (uint32_t s = 0; s < p.n_slots; s++) SL[s * G + t] = 0;
      SL[p.kept_slot * G + t] = valid;
      if (!noiseless && p.n_sites) {
        for (uint32_t j = 0; j < 32; j++) {
          uint32_t f = ((valid >> j) & 1u) ? next_fault(p, L.seed, s0 + j, 0) : kNoFault;
          nf[j] = f;
          minsite = min(minsite, f >> 4);
        }
      }
    }
    if (p.k_max > 0) {
      for (uint32_t s = t; s < S; s += T) {
        C one;
        one.x = (real)1;
        one.y = (real)0;
        work[s] = one;
      }
    }
    uint32_t k = 0;
    __syncthreads();

    auto store = [&](uint32_t* base, uint32_t row, uint32_t v) {
      if (word_ok) base[(size_t)row * L.row_words32 + my_word] = v;
    };
    auto fbit = [&](const uint32_t* plane, uint32_t s) -> uint32_t {
      return (plane[s >> 5] >> (s & 31u)) & 1u;
    };

    for (uint32_t pc = 0; pc < p.n_ops; pc++) {
      const Op op = p.ops[pc];
      const uint32_t code = op.code;
      if (L.stop_event != 0xffffffffu && is_meas(op.code) && op.i1 == L.stop_event) {
        __syncthreads();
        if (t == 0) {
          uint32_t ds = (uint32_t)(L.dump_shot - tile * (uint64_t)S);
          for (uint32_t q = 0; q < p.nw * 2; q++) L.dump_frame[q] = 0;
          for (uint32_t q = 0; q < N; q++) {
            L.dump_frame[q >> 5] |= fbit(X + q * G, ds) << (q & 31);
            L.dump_frame[p.nw + (q >> 5)] |= fbit(Z + q * G, ds) << (q & 31);
          }
          for (uint32_t i = 0; i < (1u << k); i++) {
            C a = work[(size_t)i * S + ds];
            L.dump_amps[2 * i] = (double)a.x;
            L.dump_amps[2 * i + 1] = (double)a.y;
          }
          *L.dump_k = k;
        }
        return;
      }
      switch (code) {
        case OP_FRAME_H:
        case OP_ARRAY_H:
          if (owner) {
            uint32_t a = X[op.a * G + t];
            X[op.a * G + t] = Z[op.a * G + t];
            Z[op.a * G + t] = a;
          }
          break;
        case OP_FRAME_S:
        case OP_ARRAY_S:
          if (owner) Z[op.a * G + t] ^= X[op.a * G + t];
          break;
        case OP_FRAME_CX:
        case OP_ARRAY_CX:
          if (owner) {
            X[op.b * G + t] ^= X[op.a * G + t];
            Z[op.a * G + t] ^= Z[op.b * G + t];
          }
          break;
        case OP_FRAME_CZ:
        case OP_ARRAY_CZ:
          if (owner) {
            uint32_t xa = X[op.a * G + t], xb = X[op.b * G + t];
            Z[op.a * G + t] ^= xb;
            Z[op.b * G + t] ^= xa;
          }
          break;
        case OP_MEAS_STATIC:
          if (owner) {
            uint32_t m = (op.flags & FLAG_SIGN) ? ~0u : 0u;
            const uint32_t* zm = p.masks + op.i0;
            for (uint32_t w = 0; w < p.nw; w++) {
              uint32_t bits = __ldg(zm + w);
              while (bits) {
                uint32_t q = w * 32u + (__ffs(bits) - 1);
                bits &= bits - 1;
                m ^= X[q * G + t];
              }
            }
            SL[op.i2 * G + t] = m;
            if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS))
              store(L.meas, op.i3, m & SL[p.kept_slot * G + t]);
          }
          break;
        case OP_MEAS_RANDOM:
          if (owner) {
            uint32_t top = meas_top_word(L.seed, s0, op.i0);
            uint32_t m = ~top;
            uint32_t b = m ^ ((op.flags & FLAG_SIGN) ? ~0u : 0u) ^ Z[op.a * G + t];
            uint32_t xa = X[op.a * G + t];
            X[op.a * G + t] = Z[op.a * G + t] ^ b;
            Z[op.a * G + t] = xa;
            SL[op.i2 * G + t] = m;
            if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS))
              store(L.meas, op.i3, m & SL[p.kept_slot * G + t]);
          }
          break;
        case OP_NOISE_BLOCK:
          if (owner && minsite < op.i1) {
            uint32_t nmin = kNoFault >> 4;
            for (uint32_t j = 0; j < 32; j++) {
              uint32_t f = nf[j];
              if ((f >> 4) >= op.i1) {
                nmin = min(nmin, f >> 4);
                continue;
              }
              const uint32_t bit = 1u << j;
              while ((f >> 4) < op.i1) {
                uint32_t site = f >> 4, opt = f & 15u;
                uint32_t info = __ldg(p.site_info + site), eff = __ldg(p.site_eff + site);
                if ((info & 15u) == SITE_FLIP) {
                  SL[eff * G + t] ^= bit;
                } else {
                  const uint32_t* mk = p.masks + eff + opt * 2u * p.nw;
                  for (uint32_t w = 0; w < p.nw; w++) {
                    uint32_t xb = __ldg(mk + w), zb = __ldg(mk + p.nw + w);
                    while (xb) {
                      uint32_t q = w * 32u + (__ffs(xb) - 1);
                      xb &= xb - 1;
                      X[q * G + t] ^= bit;
                    }
                    while (zb) {
                      uint32_t q = w * 32u + (__ffs(zb) - 1);
                      zb &= zb - 1;
                      Z[q * G + t] ^= bit;
                    }
                  }
                }
                f = next_fault(p, L.seed, s0 + j, site + 1);
              }
              nf[j] = f;
              nmin = min(nmin, f >> 4);
            }
            minsite = nmin;
          }
          break;
        case OP_FEEDFORWARD:
          if (owner) {
            uint32_t c = SL[op.i2 * G + t];
            if (c) {
              const uint32_t* mk = p.masks + op.i0;
              for (uint32_t w = 0; w < p.nw; w++) {
                uint32_t xb = __ldg(mk + w), zb = __ldg(mk + p.nw + w);
                while (xb) {
                  uint32_t q = w * 32u + (__ffs(xb) - 1);
                  xb &= xb - 1;
                  X[q * G + t] ^= c;
                }
                while (zb) {
                  uint32_t q = w * 32u + (__ffs(zb) - 1);
                  zb &= zb - 1;
                  Z[q * G + t] ^= c;
                }
              }
            }
          }
          break;
        case OP_REC_OUT:
          if (owner && (L.flags & LF_OUT_MEAS)) store(L.meas, op.i3, SL[op.i2 * G + t] & SL[p.kept_slot * G + t]);
          break;
        case OP_DETECTOR:
          if (owner) {
            uint32_t d = 0;
            for (uint32_t j = 0; j < op.i1; j++) d ^= SL[__ldg(p.slot_list + op.i0 + j) * G + t];
            if (!(L.flags & LF_REFERENCE) && __ldg(p.det_ref + op.i3)) d = ~d;
            uint32_t kept = SL[p.kept_slot * G + t];
            if (L.flags & LF_OUT_DET) store(L.det, op.i3, d & kept);
            if (L.flags & LF_POSTSELECT) SL[p.kept_slot * G + t] = kept & ~d;
          }
          break;
        case OP_OBS_INCLUDE:
          if (owner) {
            uint32_t d = 0;
            for (uint32_t j = 0; j < op.i1; j++) d ^= SL[__ldg(p.slot_list + op.i0 + j) * G + t];
            SL[op.i2 * G + t] ^= d;
          }
          break;
        case OP_OBS_OUT:
          if (owner && (L.flags & LF_OUT_OBS)) {
            uint32_t v = SL[op.i2 * G + t];
            if (!(L.flags & LF_REFERENCE) && __ldg(p.obs_ref + op.i3)) v = ~v;
            store(L.obs, op.i3, v & SL[p.kept_slot * G + t]);
          }
          break;
        case OP_KEPT_OUT:
          if (owner) {
            uint32_t kept = SL[p.kept_slot * G + t];
            if (L.flags & LF_OUT_KEPT) store(L.kept, 0, kept);
            if (word_ok && kept) atomicAdd(L.kept_count, (unsigned long long)__popc(kept));
          }
          break;
        default:
          break;
      }
      // ---- active-array part (all threads) ----
      if (code >= OP_ARRAY_H && code <= OP_MEAS_ACTIVE_X && code != OP_MEAS_STATIC &&
          code != OP_MEAS_RANDOM) {
        __syncthreads();
        const uint32_t pa = op.pa;
        if (code == OP_EXPAND_ROT) {
          const double c2 = cos(2.0 * op.f), s2 = sin(2.0 * op.f);
          const real rs = (real)0.70710678118654752440;
          const uint32_t n = 1u << k;
          for (uint32_t s = t % S; s < S; s += T) {
            const real sn = (real)(fbit(X + op.a * G, s) ? -s2 : s2);
            C ph;
            ph.x = (real)c2 * rs;
            ph.y = sn * rs;
            for (uint32_t j = sub; j < n; j += R) {
              C a = work[(size_t)j * S + s];
              work[(size_t)j * S + s] = cscale(a, rs);
              work[(size_t)(j + n) * S + s] = cmul(a, ph);
            }
          }
          k++;
        } else if (code == OP_ROT_Z) {
          const double c2 = cos(2.0 * op.f), s2 = sin(2.0 * op.f);
          const uint32_t half = 1u << (k - 1);
          for (uint32_t s = t % S; s < S; s += T) {
            C ph;
            ph.x = (real)c2;
            ph.y = (real)(fbit(X + op.a * G, s) ? -s2 : s2);
            for (uint32_t j = sub; j < half; j += R) {
              size_t i1 = (size_t)(insert0(j, pa) | (1u << pa)) * S + s;
              work[i1] = cmul(work[i1], ph);
            }
          }
        } else if (code == OP_ROT_X) {
          const double c1 = cos(op.f), s1 = sin(op.f);
          const uint32_t half = 1u << (k - 1);
          for (uint32_t s = t % S; s < S; s += T) {
            const real cr = (real)c1, sr = (real)(fbit(Z + op.a * G, s) ? -s1 : s1);
            for (uint32_t j = sub; j < half; j += R) {
              size_t i0 = (size_t)insert0(j, pa) * S + s, i1 = i0 + ((size_t)1 << pa) * S;
              C a = work[i0], b = work[i1], na, nb;
              na.x = cr * a.x + sr * b.y;
              na.y = cr * a.y - sr * b.x;
              nb.x = sr * a.y + cr * b.x;
              nb.y = -sr * a.x + cr * b.y;
              work[i0] = na;
              work[i1] = nb;
            }
          }
        } else if (code == OP_ARRAY_H) {
          const real rs = (real)0.70710678118654752440;
          const uint32_t half = 1u << (k - 1);
          for (uint32_t s = t % S; s < S; s += T)
            for (uint32_t j = sub; j < half; j += R) {
              size_t i0 = (size_t)insert0(j, pa) * S + s, i1 = i0 + ((size_t)1 << pa) * S;
              C a = work[i0], b = work[i1];
              work[i0] = cscale(cadd(a, b), rs);
              work[i1] = cscale(csub(a, b), rs);
            }
        } else if (code == OP_ARRAY_S) {
          const uint32_t half = 1u << (k - 1);
          for (uint32_t s = t % S; s < S; s += T)
            for (uint32_t j = sub; j < half; j += R) {
              size_t i1 = (size_t)(insert0(j, pa) | (1u << pa)) * S + s;
              C a = work[i1], r;
              r.x = -a.y;
              r.y = a.x;
              work[i1] = r;
            }
        } else if (code == OP_ARRAY_CX || code == OP_ARRAY_CZ) {
          const uint32_t pb = op.pb, lo = min(pa, pb), hi = max(pa, pb);
          const uint32_t quarter = 1u << (k - 2);
          for (uint32_t s = t % S; s < S; s += T)
            for (uint32_t j = sub; j < quarter; j += R) {
              uint32_t base = insert0(insert0(j, lo), hi);
              if (code == OP_ARRAY_CX) {
                size_t i0 = (size_t)(base | (1u << pa)) * S + s, i1 = (size_t)(base | (1u << pa) | (1u << pb)) * S + s;
                C a = work[i0];
                work[i0] = work[i1];
                work[i1] = a;
              } else {
                size_t i = (size_t)(base | (1u << pa) | (1u << pb)) * S + s;
                C a = work[i];
                a.x = -a.x;
                a.y = -a.y;
                work[i] = a;
              }
            }
        } else {  // active measurement
          const bool xm = code == OP_MEAS_ACTIVE_X;
          const uint32_t half = 1u << (k - 1);
          const real rs = (real)0.70710678118654752440;
          for (uint32_t s = t; s < S; s += T) {
            RED[s] = 0.0;
            RED[S + s] = 0.0;
          }
          __syncthreads();
          for (uint32_t s = t % S; s < S; s += T) {
            double a0 = 0.0, a1 = 0.0;
            for (uint32_t j = sub; j < half; j += R) {
              size_t i0 = (size_t)insert0(j, pa) * S + s, i1 = i0 + ((size_t)1 << pa) * S;
              C u = work[i0], v = work[i1];
              if (xm) {
                double ux = u.x, uy = u.y, vx = v.x, vy = v.y;
                double px = ux + vx, py = uy + vy, mx = ux - vx, my = uy - vy;
                a0 += 0.5 * (px * px + py * py);
                a1 += 0.5 * (mx * mx + my * my);
              } else {
                a0 += cnorm2(u);
                a1 += cnorm2(v);
              }
            }
            atomicAdd(&RED[s], a0);
            atomicAdd(&RED[S + s], a1);
          }
          __syncthreads();
          if (owner) {
            const uint32_t top = meas_top_word(L.seed, s0, op.i0);
            const uint32_t pw = xm ? Z[op.a * G + t] : X[op.a * G + t];
            const uint32_t abit = (op.flags & FLAG_SIGN) ? 1u : 0u;
            uint32_t mw = 0, bw = 0;
            for (uint32_t j = 0; j < 32; j++) {
              const uint32_t s = t * 32u + j;
              const double S0 = RED[s], S1 = RED[S + s], tot = S0 + S1;
              const uint32_t pbit = (pw >> j) & 1u;
              const double p1 = tot > 0.0 ? ((1u ^ abit ^ pbit) ? S1 : S0) / tot : 0.0;
              const uint32_t m = ((valid >> j) & 1u) ? draw_outcome(L.seed, s0 + j, op.i0, (top >> j) & 1u, p1) : 0u;
              const uint32_t b = m ^ abit ^ pbit;
              const double sb = b ? S1 : S0;
              RED[s] = sb > 0.0 ? 1.0 / sqrt(sb) : 0.0;
              mw |= m << j;
              bw |= b << j;
            }
            TMP[t] = bw;
            SL[op.i2 * G + t] = mw;
            if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS))
              store(L.meas, op.i3, mw & SL[p.kept_slot * G + t]);
            if (xm) {
              uint32_t xa = X[op.a * G + t];
              X[op.a * G + t] = Z[op.a * G + t] ^ bw;
              Z[op.a * G + t] = xa;
            } else {
              X[op.a * G + t] ^= bw;
            }
          }
          __syncthreads();
          const uint32_t top_pos = k - 1;
          for (uint32_t s = t % S; s < S; s += T) {
            const uint32_t b = fbit(TMP, s);
            const real sc = (real)RED[s];
            if (pa == top_pos) {
              for (uint32_t j = sub; j < half; j += R) {
                C o0 = work[(size_t)j * S + s], o1 = work[(size_t)(j + half) * S + s], v;
                if (xm) v = cscale(b ? csub(o0, o1) : cadd(o0, o1), rs);
                else v = b ? o1 : o0;
                work[(size_t)j * S + s] = cscale(v, sc);
              }
            } else {
              const uint32_t quarter = 1u << (k - 2);
              for (uint32_t j = sub; j < quarter; j += R) {
                uint32_t base = insert0(insert0(j, pa), top_pos);
                size_t p00 = (size_t)base * S + s, p10 = (size_t)(base | (1u << pa)) * S + s;
                size_t p01 = (size_t)(base | (1u << top_pos)) * S + s;
                size_t p11 = (size_t)(base | (1u << pa) | (1u << top_pos)) * S + s;
                C n0, n1;
                if (xm) {
                  C o00 = work[p00], o10 = work[p10], o01 = work[p01], o11 = work[p11];
                  n0 = cscale(b ? csub(o00, o10) : cadd(o00, o10), rs);
                  n1 = cscale(b ? csub(o01, o11) : cadd(o01, o11), rs);
                } else {
                  n0 = b ? work[p10] : work[p00];
                  n1 = b ? work[p11] : work[p01];
                }
                work[p00] = cscale(n0, sc);
                work[p10] = cscale(n1, sc);
              }
            }
          }
          k--;
        }
        __syncthreads();
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Plain FP64 executor: one thread per shot.
// ---------------------------------------------------------------------------
constexpr uint32_t kPlainMaxW = 8;       // N <= 256
constexpr uint32_t kPlainMaxSlots = 2048;

__global__ void __launch_bounds__(128) exec_plain(LaunchParams L) {
  const DevProg& p = L.p;
  const uint64_t sl = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t padded = L.row_words32 * 32u;
  if ((sl & ~31ull) >= padded) return;  // whole warps only
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t word = sl >> 5;
  const bool valid = sl < L.shots;
  const uint64_t s = L.shot_offset + sl;
  const uint64_t s0 = s & ~31ull;
  uint32_t x[kPlainMaxW], z[kPlainMaxW], slots[kPlainMaxSlots / 32];
  for (uint32_t w = 0; w < kPlainMaxW; w++) x[w] = z[w] = 0;
  for (uint32_t w = 0; w < kPlainMaxSlots / 32; w++) slots[w] = 0;
  double2* A = reinterpret_cast<double2*>(L.work);
  const uint64_t stride = padded;
  auto amp = [&](uint32_t i) -> double2& { return A[(size_t)i * stride + sl]; };
  auto getb = [](const uint32_t* v, uint32_t q) -> uint32_t { return (v[q >> 5] >> (q & 31)) & 1u; };
  auto setb = [](uint32_t* v, uint32_t q, uint32_t b) {
    v[q >> 5] = (v[q >> 5] & ~(1u << (q & 31))) | (b << (q & 31));
  };
  auto flipb = [](uint32_t* v, uint32_t q, uint32_t b) { v[q >> 5] ^= b << (q & 31); };
  auto store = [&](uint32_t* base, uint32_t row, uint32_t bit) {
    uint32_t w = __ballot_sync(0xffffffffu, bit);
    if (lane == 0) base[(size_t)row * L.row_words32 + word] = w;
  };
  setb(slots, p.kept_slot, valid ? 1u : 0u);
  uint32_t nf = (valid && !(L.flags & LF_NOISELESS) && p.n_sites) ? next_fault(p, L.seed, s, 0) : kNoFault;
  uint32_t k = 0;
  if (p.k_max > 0) amp(0) = make_double2(1.0, 0.0);
  const double rs = 0.70710678118654752440;

  for (uint32_t pc = 0; pc < p.n_ops; pc++) {
    const Op op = p.ops[pc];
    if (L.stop_event != 0xffffffffu && is_meas(op.code) && op.i1 == L.stop_event) {
      if (sl == L.dump_shot) {
        for (uint32_t w = 0; w < p.nw; w++) {
          L.dump_frame[w] = x[w];
          L.dump_frame[p.nw + w] = z[w];
        }
        for (uint32_t i = 0; i < (1u << k); i++) {
          L.dump_amps[2 * i] = amp(i).x;
          L.dump_amps[2 * i + 1] = amp(i).y;
        }
        *L.dump_k = k;
      }
      return;
    }
    const uint32_t kept = getb(slots, p.kept_slot);
    switch (op.code) {
      case OP_FRAME_H:
      case OP_ARRAY_H: {
        uint32_t a = getb(x, op.a);
        setb(x, op.a, getb(z, op.a));
        setb(z, op.a, a);
        if (op.code == OP_ARRAY_H) {
          const uint32_t half = 1u << (k - 1);
          for (uint32_t j = 0; j < half; j++) {
            uint32_t i0 = insert0(j, op.pa), i1 = i0 | (1u << op.pa);
            double2 u = amp(i0), v = amp(i1);
            amp(i0) = make_double2((u.x + v.x) * rs, (u.y + v.y) * rs);
            amp(i1) = make_double2((u.x - v.x) * rs, (u.y - v.y) * rs);
          }
        }
        break;
      }
      case OP_FRAME_S:
      case OP_ARRAY_S:
        flipb(z, op.a, getb(x, op.a));
        if (op.code == OP_ARRAY_S) {
          const uint32_t half = 1u << (k - 1);
          for (uint32_t j = 0; j < half; j++) {
            uint32_t i1 = insert0(j, op.pa) | (1u << op.pa);
            double2 u = amp(i1);
            amp(i1) = make_double2(-u.y, u.x);
          }
        }
        break;
      case OP_FRAME_CX:
      case OP_ARRAY_CX:
        flipb(x, op.b, getb(x, op.a));
        flipb(z, op.a, getb(z, op.b));
        if (op.code == OP_ARRAY_CX) {
          const uint32_t lo = min(op.pa, op.pb), hi = max(op.pa, op.pb);
          for (uint32_t j = 0; j < (1u << (k - 2)); j++) {
            uint32_t base = insert0(insert0(j, lo), hi);
            uint32_t i0 = base | (1u << op.pa), i1 = i0 | (1u << op.pb);
            double2 u = amp(i0);
            amp(i0) = amp(i1);
            amp(i1) = u;
          }
        }
        break;
      case OP_FRAME_CZ:
      case OP_ARRAY_CZ: {
        uint32_t xa = getb(x, op.a), xb = getb(x, op.b);
        flipb(z, op.a, xb);
        flipb(z, op.b, xa);
        if (op.code == OP_ARRAY_CZ) {
          const uint32_t lo = min(op.pa, op.pb), hi = max(op.pa, op.pb);
          for (uint32_t j = 0; j < (1u << (k - 2)); j++) {
            uint32_t i = insert0(insert0(j, lo), hi) | (1u << op.pa) | (1u << op.pb);
            double2 u = amp(i);
            amp(i) = make_double2(-u.x, -u.y);
          }
        }
        break;
      }
      case OP_EXPAND_ROT: {
        const double th = getb(x, op.a) ? -op.f : op.f;
        const double c2 = cos(2.0 * th) * rs, s2 = sin(2.0 * th) * rs;
        const uint32_t n = 1u << k;
        for (uint32_t i = 0; i < n; i++) {
          double2 u = amp(i);
          amp(i) = make_double2(u.x * rs, u.y * rs);
          amp(i + n) = make_double2(u.x * c2 - u.y * s2, u.x * s2 + u.y * c2);
        }
        k++;
        break;
      }
      case OP_ROT_Z: {
        const double th = getb(x, op.a) ? -op.f : op.f;
        const double c2 = cos(2.0 * th), s2 = sin(2.0 * th);
        for (uint32_t j = 0; j < (1u << (k - 1)); j++) {
          uint32_t i1 = insert0(j, op.pa) | (1u << op.pa);
          double2 u = amp(i1);
          amp(i1) = make_double2(u.x * c2 - u.y * s2, u.x * s2 + u.y * c2);
        }
        break;
      }
      case OP_ROT_X: {
        const double th = getb(z, op.a) ? -op.f : op.f;
        const double c1 = cos(th), s1 = sin(th);
        for (uint32_t j = 0; j < (1u << (k - 1)); j++) {
          uint32_t i0 = insert0(j, op.pa), i1 = i0 | (1u << op.pa);
          double2 a = amp(i0), b = amp(i1);
          amp(i0) = make_double2(c1 * a.x + s1 * b.y, c1 * a.y - s1 * b.x);
          amp(i1) = make_double2(s1 * a.y + c1 * b.x, -s1 * a.x + c1 * b.y);
        }
        break;
      }
      case OP_MEAS_STATIC: {
        uint32_t par = (op.flags & FLAG_SIGN) ? 1u : 0u;
        for (uint32_t w = 0; w < p.nw; w++) par ^= __popc(x[w] & __ldg(p.masks + op.i0 + w)) & 1u;
        setb(slots, op.i2, par);
        if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) store(L.meas, op.i3, par & kept);
        break;
      }
      case OP_MEAS_RANDOM: {
        uint32_t top = (meas_top_word(L.seed, s0, op.i0) >> lane) & 1u;
        uint32_t m = top ^ 1u;
        uint32_t b = m ^ (op.flags & FLAG_SIGN ? 1u : 0u) ^ getb(z, op.a);
        uint32_t xa = getb(x, op.a);
        setb(x, op.a, getb(z, op.a) ^ b);
        setb(z, op.a, xa);
        setb(slots, op.i2, m);
        if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) store(L.meas, op.i3, m & kept);
        break;
      }
      case OP_MEAS_ACTIVE_Z:
      case OP_MEAS_ACTIVE_X: {
        const bool xm = op.code == OP_MEAS_ACTIVE_X;
        const uint32_t half = 1u << (k - 1), pa = op.pa, top_pos = k - 1;
        double S0 = 0.0, S1 = 0.0;
        for (uint32_t j = 0; j < half; j++) {
          uint32_t i0 = insert0(j, pa), i1 = i0 | (1u << pa);
          double2 u = amp(i0), v = amp(i1);
          if (xm) {
            double px = u.x + v.x, py = u.y + v.y, mx = u.x - v.x, my = u.y - v.y;
            S0 += 0.5 * (px * px + py * py);
            S1 += 0.5 * (mx * mx + my * my);
          } else {
            S0 += u.x * u.x + u.y * u.y;
            S1 += v.x * v.x + v.y * v.y;
          }
        }
        const uint32_t pbit = xm ? getb(z, op.a) : getb(x, op.a);
        const uint32_t abit = (op.flags & FLAG_SIGN) ? 1u : 0u;
        const double tot = S0 + S1;
        const double p1 = tot > 0.0 ? ((1u ^ abit ^ pbit) ? S1 : S0) / tot : 0.0;
        const uint32_t top = (meas_top_word(L.seed, s0, op.i0) >> lane) & 1u;
        const uint32_t m = valid ? draw_outcome(L.seed, s, op.i0, top, p1) : 0u;
        const uint32_t b = m ^ abit ^ pbit;
        const double sb = b ? S1 : S0;
        const double sc = sb > 0.0 ? 1.0 / sqrt(sb) : 0.0;
        if (pa == top_pos) {
          for (uint32_t j = 0; j < half; j++) {
            double2 o0 = amp(j), o1 = amp(j + half), v;
            if (xm) v = b ? make_double2((o0.x - o1.x) * rs, (o0.y - o1.y) * rs)
                          : make_double2((o0.x + o1.x) * rs, (o0.y + o1.y) * rs);
            else v = b ? o1 : o0;
            amp(j) = make_double2(v.x * sc, v.y * sc);
          }
        } else {
          for (uint32_t j = 0; j < (1u << (k - 2)); j++) {
            uint32_t base = insert0(insert0(j, pa), top_pos);
            uint32_t p00 = base, p10 = base | (1u << pa), p01 = base | (1u << top_pos), p11 = p10 | (1u << top_pos);
            double2 n0, n1;
            if (xm) {
              double2 o00 = amp(p00), o10 = amp(p10), o01 = amp(p01), o11 = amp(p11);
              double sg = b ? -1.0 : 1.0;
              n0 = make_double2((o00.x + sg * o10.x) * rs, (o00.y + sg * o10.y) * rs);
              n1 = make_double2((o01.x + sg * o11.x) * rs, (o01.y + sg * o11.y) * rs);
            } else {
              n0 = b ? amp(p10) : amp(p00);
              n1 = b ? amp(p11) : amp(p01);
            }
            amp(p00) = make_double2(n0.x * sc, n0.y * sc);
            amp(p10) = make_double2(n1.x * sc, n1.y * sc);
          }
        }
        k--;
        setb(slots, op.i2, m);
        if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) store(L.meas, op.i3, m & kept);
        if (xm) {
          uint32_t xa = getb(x, op.a);
          setb(x, op.a, getb(z, op.a) ^ b);
          setb(z, op.a, xa);
        } else {
          flipb(x, op.a, b);
        }
        break;
      }
      case OP_NOISE_BLOCK:
        while ((nf >> 4) < op.i1) {
          uint32_t site = nf >> 4, opt = nf & 15u;
          uint32_t info = __ldg(p.site_info + site), eff = __ldg(p.site_eff + site);
          if ((info & 15u) == SITE_FLIP) {
            flipb(slots, eff, 1u);
          } else {
            const uint32_t* mk = p.masks + eff + opt * 2u * p.nw;
            for (uint32_t w = 0; w < p.nw; w++) {
              x[w] ^= __ldg(mk + w);
              z[w] ^= __ldg(mk + p.nw + w);
            }
          }
          nf = next_fault(p, L.seed, s, site + 1);
        }
        break;
      case OP_FEEDFORWARD:
        if (getb(slots, op.i2))
          for (uint32_t w = 0; w < p.nw; w++) {
            x[w] ^= __ldg(p.masks + op.i0 + w);
            z[w] ^= __ldg(p.masks + op.i0 + p.nw + w);
          }
        break;
      case OP_REC_OUT:
        if (L.flags & LF_OUT_MEAS) store(L.meas, op.i3, getb(slots, op.i2) & kept);
        break;
      case OP_DETECTOR: {
        uint32_t d = 0;
        for (uint32_t j = 0; j < op.i1; j++) d ^= getb(slots, __ldg(p.slot_list + op.i0 + j));
        if (!(L.flags & LF_REFERENCE)) d ^= __ldg(p.det_ref + op.i3) ? 1u : 0u;
        if (L.flags & LF_OUT_DET) store(L.det, op.i3, d & kept);
        if ((L.flags & LF_POSTSELECT) && d) setb(slots, p.kept_slot, 0u);
        break;
      }
      case OP_OBS_INCLUDE: {
        uint32_t d = 0;
        for (uint32_t j = 0; j < op.i1; j++) d ^= getb(slots, __ldg(p.slot_list + op.i0 + j));
        flipb(slots, op.i2, d);
        break;
      }
      case OP_OBS_OUT:
        if (L.flags & LF_OUT_OBS) {
          uint32_t v = getb(slots, op.i2);
          if (!(L.flags & LF_REFERENCE)) v ^= __ldg(p.obs_ref + op.i3) ? 1u : 0u;
          store(L.obs, op.i3, v & kept);
        }
        break;
      case OP_KEPT_OUT: {
        if (L.flags & LF_OUT_KEPT) store(L.kept, 0, kept);
        uint32_t w = __ballot_sync(0xffffffffu, kept);
        if (lane == 0 && w) atomicAdd(L.kept_count, (unsigned long long)__popc(w));
        break;
      }
      default:
        break;
    }
  }
}

// ---------------------------------------------------------------------------
// Host-side launchers (called from capi.cu)
// ---------------------------------------------------------------------------
size_t batched_smem_bytes(const DevProg& p, uint32_t G) {
  size_t words = ((size_t)(2 * p.n_qubits + p.n_slots + 1) * G + 1) & ~(size_t)1;
  size_t bytes = words * 4;
  if (p.k_max > 0) bytes += 2 * sizeof(double) * 32 * (size_t)G;
  return bytes;
}

cudaError_t launch_batched(const LaunchParams& L, bool fp64, uint32_t grid, uint32_t threads,
                           size_t smem, cudaStream_t st) {
  if (fp64) {
    cudaError_t e = cudaFuncSetAttribute(exec_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    exec_batched<double><<<grid, threads, smem, st>>>(L);
  } else {
    cudaError_t e = cudaFuncSetAttribute(exec_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    exec_batched<float><<<grid, threads, smem, st>>>(L);
  }
  return cudaGetLastError();
}

cudaError_t batched_occupancy(bool fp64, uint32_t threads, size_t smem, int* blocks_per_sm) {
  if (fp64) {
    cudaFuncSetAttribute(exec_batched<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, exec_batched<double>, (int)threads, smem);
  }
  cudaFuncSetAttribute(exec_batched<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, exec_batched<float>, (int)threads, smem);
}

cudaError_t launch_plain(const LaunchParams& L, cudaStream_t st) {
  const uint64_t padded = L.row_words32 * 32u;
  const uint32_t threads = 128;
  const uint64_t blocks = (padded + threads - 1) / threads;
  exec_plain<<<(uint32_t)blocks, threads, 0, st>>>(L);
  return cudaGetLastError();
}

bool plain_supported(const DevProg& p) {
  return p.nw <= kPlainMaxW && p.n_slots <= kPlainMaxSlots;
}

}  // namespace nc
