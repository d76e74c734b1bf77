// kernels.cu — the online sample-many phase on the GPU (Sec. 3.2).
//
// exec_batched<real>: one CTA runs a tile of 32*G shots. The virtual Pauli
//   frame and the record slots are bit-sliced over shots in shared memory
//   (word w of plane q holds bit q of the frame for the 32 shots of word w);
//   frame, noise, measurement-parity and record instructions are executed by
//   the G word-owner threads, one 32-shot word each, with no synchronisation.
//   Active-array instructions (expand, rotations, array Cliffords, active
//   measurements) run on all threads over (amplitude, shot) pairs of the
//   tile's amplitude block (global memory, or shared memory for small
//   tiles), laid out amplitude-major / shot-minor so that consecutive
//   threads touch consecutive shots. Measurement probabilities are
//   accumulated in FP64; amplitudes are stored in `real` (float for the
//   batched form). When the program carries a fused array-pass list
//   (fuse.cpp) the executor runs that list: pair, diagonal and gather passes
//   over an index-mapped vector.
//
// exec_plain: the baseline form — one thread per shot, frame and record bits
//   in thread-local arrays, FP64 amplitudes in global memory, instructions
//   read straight from global memory.
//
// bucket_faults / presample_faults: fault sampling ahead of the executor.
//
// The executors follow the same random-draw contract (kernels.cuh) and
// produce identical records.
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
// A tile is G 32-shot words; thread t < G / W owns words t*W .. t*W+W-1.
// Shared-memory layout of one CTA (u32 words unless noted):
//   OPS Op [2][kChunk] double-buffered instruction chunks (cp.async)
//   PL  [2N+2][G] frame planes (x bits of virtual qubit q at plane q, z bits at N + q),
//                 an all-zero plane 2N and a scratch plane 2N + 1 (padding targets)
//   SL  [n_slots+1][G] record slots and an all-zero slot n_slots
//   NF  [32][G]  next fault of shot (word w, bit j) at NF[j * G + w]
//   CUR u8 [32][G] list cursor of each shot (pre-sampled faults)
//   TMP [G]      per-word scratch (virtual outcomes of an active measurement)
//   QU  u16 [owner warps][kQueue] warp queues of due (word, bit) noise entries
//   RED f64 [2][S] measurement sums / scales (k_max > 0 only)
//   FT  FTerm [kFTermSmem] terms of the current fused pass (k_max > 0 only)
//   WORK the tile's active vectors, when they fit here (else global memory)
constexpr uint32_t kQueue = 256;

struct SmemLayout {
  size_t pl, sl, nf, cur, tmp, qu, ops, red, ft, work, bytes;
};
constexpr uint32_t kFTermSmem = 64;  // terms of a fused pass staged in shared memory

__host__ __device__ inline SmemLayout smem_layout(uint32_t n_qubits, uint32_t n_slots, uint32_t k_max, uint32_t G,
                                                  uint32_t W, bool bk = false, uint32_t work_words = 0) {
  // the bucketed executor keeps no per-shot noise state (NF, CUR, QU)
  SmemLayout L;
  size_t w = 0;
  L.ops = w;
  w += (size_t)2 * kChunk * (sizeof(Op) / 4);
  L.pl = w;
  w += (size_t)(2 * n_qubits + 2) * G;  // + zero plane (2N) and scratch plane (2N + 1)
  L.sl = w;
  w += (size_t)(n_slots + 1) * G;       // + zero slot (n_slots)
  L.nf = w;
  if (!bk) w += (size_t)32 * G;
  L.cur = w;  // u8 [32][G]: next index into the pre-sampled fault list
  if (!bk) w += (size_t)8 * G;
  L.tmp = w;
  w += G;
  w = (w + 3) & ~(size_t)3;
  L.qu = w;
  const size_t owner_warps = (G / W + 31) / 32;
  if (!bk) w += owner_warps * (kQueue / 2);
  w = (w + 3) & ~(size_t)3;
  L.red = w;
  if (k_max > 0) w += (size_t)2 * 2 * 32 * G;  // 2 doubles per shot
  w = (w + 7) & ~(size_t)7;
  L.ft = w;
  if (k_max > 0) w += (size_t)kFTermSmem * (sizeof(FTerm) / 4);
  // active vectors of the tile, when they are kept in shared memory
  w = (w + 3) & ~(size_t)3;
  L.work = w;
  w += work_words;
  L.bytes = w * 4;
  return L;
}

template <int W>
struct Vw {
  uint32_t v[W];
};

template <int W>
__device__ __forceinline__ Vw<W> vld(const uint32_t* p) {
  Vw<W> r;
  if constexpr (W == 4) {
    uint4 a = *reinterpret_cast<const uint4*>(p);
    r.v[0] = a.x; r.v[1] = a.y; r.v[2] = a.z; r.v[3] = a.w;
  } else if constexpr (W == 2) {
    uint2 a = *reinterpret_cast<const uint2*>(p);
    r.v[0] = a.x; r.v[1] = a.y;
  } else {
    r.v[0] = *p;
  }
  return r;
}

template <int W>
__device__ __forceinline__ void vst(uint32_t* p, const Vw<W>& r) {
  if constexpr (W == 4) *reinterpret_cast<uint4*>(p) = make_uint4(r.v[0], r.v[1], r.v[2], r.v[3]);
  else if constexpr (W == 2) *reinterpret_cast<uint2*>(p) = make_uint2(r.v[0], r.v[1]);
  else *p = r.v[0];
}

template <int W>
__device__ __forceinline__ Vw<W> vfill(uint32_t x) {
  Vw<W> r;
#pragma unroll
  for (int i = 0; i < W; i++) r.v[i] = x;
  return r;
}

template <int W>
__device__ __forceinline__ void vxor(Vw<W>& a, const Vw<W>& b) {
#pragma unroll
  for (int i = 0; i < W; i++) a.v[i] ^= b.v[i];
}

template <int W>
__device__ __forceinline__ Vw<W> vand(const Vw<W>& a, const Vw<W>& b) {
  Vw<W> r;
#pragma unroll
  for (int i = 0; i < W; i++) r.v[i] = a.v[i] & b.v[i];
  return r;
}

// Inline entries of list instructions, read with register bit operations
// (the u16 views of program.h would force the instruction into local memory).
__device__ __forceinline__ uint32_t ent(const Op& op, uint32_t i) {
  return (uint32_t)((unsigned long long)__double_as_longlong(op.f) >> (16 * i)) & 0xFFFFu;
}
__device__ __forceinline__ uint32_t rent(const Op& op, uint32_t i) {
  return ((i < 2 ? op.i2 : op.i3) >> (16 * (i & 1))) & 0xFFFFu;
}

__device__ __forceinline__ uint32_t pick4(const uint4& v, uint32_t i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}

// BIG variants allow 1024 threads per CTA (large-k tiles, at most 64
// registers per thread); the others allow 256 threads and more registers.
template <typename real, int W, bool BIG, bool BK>
__global__ void __launch_bounds__(BIG ? 1024 : 256, 1) exec_batched(LaunchParams L) {
  using C = typename Cx<real>::T;
  extern __shared__ __align__(16) uint32_t smem[];
  const DevProg& p = L.p;
  const uint32_t G = L.G, S = 32u * G, N = p.n_qubits, T = blockDim.x, t = threadIdx.x;
  const SmemLayout lay = smem_layout(N, p.n_slots, p.k_max, G, W, BK, L.smem_work_words);
  uint32_t* PL = smem + lay.pl;
  uint32_t* X = PL;
  uint32_t* Z = PL + (size_t)N * G;
  uint32_t* SL = smem + lay.sl;
  uint32_t* NF = smem + lay.nf;
  uint8_t* CUR = reinterpret_cast<uint8_t*>(smem + lay.cur);
  uint32_t* TMP = smem + lay.tmp;
  const uint32_t lane = t & 31u, warp = t >> 5;
  uint16_t* QU = reinterpret_cast<uint16_t*>(smem + lay.qu) + (size_t)warp * kQueue;
  double* RED = reinterpret_cast<double*>(smem + lay.red);
  // the fused array-pass list (fuse.cpp) unless a debug stop needs the
  // original one; with gather passes each CTA owns two vector buffers
  const bool fused = p.n_fops > 0 && L.stop_event == 0xffffffffu;
  const Op* OPS = fused ? p.fops : p.ops;
  const uint32_t n_ops = fused ? p.n_fops : p.n_ops;
  // active vectors: in shared memory when they fit (small tiles), else in
  // this CTA's slice of the global workspace
  C* const work_base = L.smem_work_words
                           ? reinterpret_cast<C*>(smem + lay.work)
                           : reinterpret_cast<C*>(L.work) + (size_t)blockIdx.x * L.work_stride * (fused && p.f_perm ? 2 : 1);
  C* work = work_base;
  C* work2 = work_base + L.work_stride;
  Op* OPB = reinterpret_cast<Op*>(smem + lay.ops);

  const uint32_t n_owners = G / W;
  const bool owner = t < n_owners;
  const bool owner_warp = (t & ~31u) < n_owners;
  const uint32_t tw = t * W;  // first word of this thread
  const uint32_t R = T >= S ? T / S : 1u;  // threads per shot in array loops
  const uint32_t sub = T >= S ? t / S : 0u;
  const bool noisy = !(L.flags & LF_NOISELESS) && p.n_sites > 0;
  const uint32_t kept_off = p.kept_slot * G;
  const uint32_t n_chunks = (n_ops + kChunk - 1) / kChunk;

  auto load_chunk = [&](uint32_t c) {
    const uint32_t first = c * kChunk, cnt = min(kChunk, n_ops - first);
    const uint4* src = reinterpret_cast<const uint4*>(OPS + first);
    uint4* dst = reinterpret_cast<uint4*>(OPB + (c & 1u) * kChunk);
    for (uint32_t i = t; i < 2 * cnt; i += T) cp_async16(dst + i, src + i);
    cp_async_commit();
  };
  __syncthreads();

  for (uint32_t tile = blockIdx.x; tile < L.n_tiles; tile += gridDim.x) {
    const uint64_t word0 = (uint64_t)tile * G + tw;  // call-local index of my first word
    const uint64_t tile_s0 = L.shot_offset + (uint64_t)tile * S;
    const uint64_t s0 = tile_s0 + (uint64_t)tw * 32u;  // global shot of my first word
    Vw<W> valid = vfill<W>(0u);
    if (owner) {
#pragma unroll
      for (int i = 0; i < W; i++) {
        const uint64_t sl0 = (word0 + i) * 32u;
        if (word0 + i < L.row_words32) {
          if (sl0 + 32 <= L.shots) valid.v[i] = ~0u;
          else if (sl0 < L.shots) valid.v[i] = (1u << (uint32_t)(L.shots - sl0)) - 1u;
        }
      }
    }
    uint32_t minsite = kNoFault >> 4;
    if (owner) {
      for (uint32_t q = 0; q < 2 * N + 2; q++) vst<W>(PL + q * G + tw, vfill<W>(0u));
      for (uint32_t s = 0; s <= p.n_slots; s++) vst<W>(SL + s * G + tw, vfill<W>(0u));
      vst<W>(SL + kept_off + tw, valid);
#pragma unroll
      for (int i = 0; i < W && !BK; i++) {
        const uint64_t sl0 = (word0 + i) * 32u;  // call-local shot of bit 0
        for (uint32_t j = 0; j < 32; j++) {
          uint32_t f = kNoFault;
          if (noisy && ((valid.v[i] >> j) & 1u)) {
            if (L.flist) {
              const uint32_t c = L.fcount[sl0 + j];
              if (c & 127u) f = L.flist[sl0 + j];
              else if (c & 128u) f = next_fault(p, L.seed, s0 + (uint64_t)i * 32u + j, 0);
            } else {
              f = next_fault(p, L.seed, s0 + (uint64_t)i * 32u + j, 0);
            }
            // stratified shots come only from complete pre-sampled lists
            if (p.sg && (!L.flist || (L.fcount[sl0 + j] & 128u))) atomicOr(L.err, 4u);
          }
          NF[j * G + tw + i] = f;
          CUR[j * G + tw + i] = 1;
          minsite = min(minsite, f >> 4);
        }
      }
    }
    work = work_base;
    work2 = work_base + L.work_stride;
    if (p.k_max > 0 && !L.init_vec) {
      for (uint32_t s = t; s < S; s += T) {
        C one;
        one.x = (real)1;
        one.y = (real)0;
        work[s] = one;
      }
    }
    uint32_t k = 0;
    if (L.init_vec) {
      // the shared prefix's state (frame zero, no record): every shot's copy
      const C* iv = reinterpret_cast<const C*>(L.init_vec);
      const uint32_t dim = 1u << L.start_k;
      for (uint32_t s = t % S; s < S; s += T)
        for (uint32_t j = sub; j < dim; j += R) work[(size_t)j * S + s] = iv[j];
      k = L.start_k;
    }

    auto store = [&](uint32_t* base, uint32_t row, const Vw<W>& v) {
      uint32_t* dst = base + (size_t)row * L.row_words32 + word0;
#pragma unroll
      for (int i = 0; i < W; i++)
        if (word0 + i < L.row_words32) dst[i] = v.v[i];
    };
    auto fbit = [&](const uint32_t* plane, uint32_t s) -> uint32_t {
      return (plane[s >> 5] >> (s & 31u)) & 1u;
    };
    auto plane = [&](uint32_t q) -> uint32_t* { return PL + q * G + tw; };
    auto slot = [&](uint32_t s) -> uint32_t* { return SL + s * G + tw; };

    const uint32_t op0 = L.init_vec ? L.start_op : 0u;  // past the shared prefix
    load_chunk(op0 / kChunk);
    cp_async_wait_all();
    __syncthreads();
    for (uint32_t ch = op0 / kChunk; ch < n_chunks; ch++) {
      if (ch + 1 < n_chunks) load_chunk(ch + 1);
      const Op* ops = OPB + (ch & 1u) * kChunk;
      const uint32_t n_here = min(kChunk, n_ops - ch * kChunk);
      const uint32_t pi0 = ch == op0 / kChunk ? op0 % kChunk : 0u;
      Op nxt = ops[pi0];
      uint32_t skip = 0;  // payload instructions consumed by a batch
      for (uint32_t pi = pi0; pi < n_here; pi += 1 + skip) {
        const Op op = nxt;
        skip = 0;
        if (op.code == OP_BATCH && L.stop_event == 0xffffffffu) skip = op.pa;
        if (pi + 1 + skip < n_here) nxt = ops[pi + 1 + skip];
        switch (op.code) {
          case OP_BATCH:
            // skip == 0 in debug-stop mode: the payloads then run one by one
            if (owner && skip) {
              const Op* b = ops + pi + 1;
              const uint32_t n = skip;
              if (op.a == 1 || op.a == 2) {
                // static measurements (a = 1) or fused static resets (a = 2):
                // all loads of the batch first, then all stores
                Vw<W> m[kMaxBatch];
#pragma unroll
                for (uint32_t u = 0; u < kMaxBatch; u++) {
                  if (u < n) {
                    const Op o = b[u];
                    m[u] = vfill<W>((o.flags & FLAG_SIGN) ? ~0u : 0u);
                    vxor<W>(m[u], vld<W>(plane(ent(o, 0))));
                    vxor<W>(m[u], vld<W>(plane(ent(o, 1))));
                    vxor<W>(m[u], vld<W>(plane(ent(o, 2))));
                    vxor<W>(m[u], vld<W>(plane(ent(o, 3))));
                  }
                }
                if (op.a == 1) {
                  const Vw<W> kept = vld<W>(slot(p.kept_slot));
#pragma unroll
                  for (uint32_t u = 0; u < kMaxBatch; u++) {
                    if (u < n) {
                      const Op o = b[u];
                      vst<W>(slot(o.i2), m[u]);
                      if ((o.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) store(L.meas, o.i3, vand<W>(m[u], kept));
                    }
                  }
                } else {
                  // conditional X-images; members write disjoint planes
                  // (scratch plane padding aside), checked by the compiler
#pragma unroll
                  for (uint32_t u = 0; u < kMaxBatch; u++) {
                    if (u < n) {
                      const Op o = b[u];
#pragma unroll
                      for (uint32_t e = 0; e < 4; e++) {
                        const uint32_t pl = rent(o, e);
                        Vw<W> v = vld<W>(plane(pl));
                        vxor<W>(v, m[u]);
                        vst<W>(plane(pl), v);
                      }
                    }
                  }
                }
              } else {
                // detectors: parities, reference, kept chain in registers
                Vw<W> d[kMaxBatch];
#pragma unroll
                for (uint32_t u = 0; u < kMaxBatch; u++) {
                  if (u < n) {
                    const Op o = b[u];
                    d[u] = vld<W>(slot(ent(o, 0)));
                    vxor<W>(d[u], vld<W>(slot(ent(o, 1))));
                    vxor<W>(d[u], vld<W>(slot(ent(o, 2))));
                    vxor<W>(d[u], vld<W>(slot(ent(o, 3))));
                  }
                }
                Vw<W> kept = vld<W>(slot(p.kept_slot));
#pragma unroll
                for (uint32_t u = 0; u < kMaxBatch; u++) {
                  if (u < n) {
                    const Op o = b[u];
                    if (!(L.flags & LF_REFERENCE) && (o.flags & FLAG_REF)) vxor<W>(d[u], vfill<W>(~0u));
                    if (L.flags & LF_OUT_DET) store(L.det, o.i3, vand<W>(d[u], kept));
                    if (L.flags & LF_POSTSELECT) {
#pragma unroll
                      for (int i = 0; i < W; i++) kept.v[i] &= ~d[u].v[i];
                    }
                  }
                }
                if (L.flags & LF_POSTSELECT) vst<W>(slot(p.kept_slot), kept);
              }
            }
            break;
          case OP_FRAME_H:
          case OP_FRAME_S:
          case OP_FRAME_CX:
          case OP_FRAME_CZ:
            if (owner) {
              if (op.code == OP_FRAME_H) {
                Vw<W> a = vld<W>(plane(op.a)), b = vld<W>(plane(N + op.a));
                vst<W>(plane(op.a), b);
                vst<W>(plane(N + op.a), a);
              } else if (op.code == OP_FRAME_S) {
                Vw<W> zz = vld<W>(plane(N + op.a));
                vxor<W>(zz, vld<W>(plane(op.a)));
                vst<W>(plane(N + op.a), zz);
              } else if (op.code == OP_FRAME_CX) {
                Vw<W> xb = vld<W>(plane(op.b)), za = vld<W>(plane(N + op.a));
                vxor<W>(xb, vld<W>(plane(op.a)));
                vxor<W>(za, vld<W>(plane(N + op.b)));
                vst<W>(plane(op.b), xb);
                vst<W>(plane(N + op.a), za);
              } else {
                Vw<W> xa = vld<W>(plane(op.a)), xb = vld<W>(plane(op.b));
                Vw<W> za = vld<W>(plane(N + op.a)), zb = vld<W>(plane(N + op.b));
                vxor<W>(za, xb);
                vxor<W>(zb, xa);
                vst<W>(plane(N + op.a), za);
                vst<W>(plane(N + op.b), zb);
              }
            }
            break;
          case OP_MEAS_STATIC:
            if (L.stop_event != 0xffffffffu && op.i1 == L.stop_event) goto dump;
            if (owner) {
              Vw<W> m = vfill<W>((op.flags & FLAG_SIGN) ? ~0u : 0u);
              if (op.pa != kNoInline) {
                // entries past the count point at the zero plane
                vxor<W>(m, vld<W>(plane(ent(op, 0))));
                vxor<W>(m, vld<W>(plane(ent(op, 1))));
                vxor<W>(m, vld<W>(plane(ent(op, 2))));
                vxor<W>(m, vld<W>(plane(ent(op, 3))));
              } else {
                const uint32_t* zm = p.masks + op.i0;
                for (uint32_t w = 0; w < p.nw; w++) {
                  uint32_t bits = __ldg(zm + w);
                  while (bits) {
                    uint32_t q = w * 32u + (__ffs(bits) - 1);
                    bits &= bits - 1;
                    vxor<W>(m, vld<W>(plane(q)));
                  }
                }
              }
              if (op.flags & FLAG_RESET) {
                // fused reset: frame ^= X-image where m is set
                auto flip = [&](uint32_t pl) {
                  Vw<W> v = vld<W>(plane(pl));
                  vxor<W>(v, m);
                  vst<W>(plane(pl), v);
                };
                switch (op.pb) {
                  case 4: flip(rent(op, 3)); [[fallthrough]];
                  case 3: flip(rent(op, 2)); [[fallthrough]];
                  case 2: flip(rent(op, 1)); [[fallthrough]];
                  case 1: flip(rent(op, 0)); [[fallthrough]];
                  default: break;
                }
              } else {
                vst<W>(slot(op.i2), m);
                if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS))
                  store(L.meas, op.i3, vand<W>(m, vld<W>(slot(p.kept_slot))));
              }
            }
            break;
          case OP_MEAS_RANDOM:
            if (L.stop_event != 0xffffffffu && op.i1 == L.stop_event) goto dump;
            if (owner) {
              const uint64_t g = s0 >> 7;
              const uint4 tb = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), TAG_MT, op.i0), key_of(L.seed));
              const uint32_t sel = (uint32_t)(s0 >> 5) & 3u;
              Vw<W> m, xa, za;
              const uint32_t sg = (op.flags & FLAG_SIGN) ? ~0u : 0u;
#pragma unroll
              for (int i = 0; i < W; i++) m.v[i] = (L.flags & LF_ARGMAX) ? 0u : ~pick4(tb, (sel + i) & 3u);
              // H_v then x_v ^= b: new x = old z ^ b, new z = old x
              Vw<W> ox = vld<W>(plane(op.a)), oz = vld<W>(plane(N + op.a));
#pragma unroll
              for (int i = 0; i < W; i++) {
                const uint32_t b = m.v[i] ^ sg ^ oz.v[i];
                xa.v[i] = oz.v[i] ^ b;
                za.v[i] = ox.v[i];
              }
              vst<W>(plane(op.a), xa);
              vst<W>(plane(N + op.a), za);
              vst<W>(slot(op.i2), m);
              if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS))
                store(L.meas, op.i3, vand<W>(m, vld<W>(slot(p.kept_slot))));
            }
            break;
          case OP_NOISE_BLOCK:
            if constexpr (BK) {
              // faults of this warp's 1024 shots in this block, one per lane
              if (owner_warp) {
                const uint32_t wt = tile * (G / 32u) + warp;
                const uint32_t* bo = L.boffs + (size_t)wt * (p.n_blocks + 1) + op.i2;
                const uint32_t beg = bo[0], end = bo[1];
                for (uint32_t e = beg + lane; e < end; e += 32) {
                  const uint32_t ent = L.bents[e];
                  const uint32_t sl = ent & 1023u;
                  const uint32_t w = warp * 32u + (sl >> 5), bit = 1u << (sl & 31u);
                  const uint4 r = __ldg(p.orec + (ent >> 10));
                  const uint32_t tag = r.x & 0xFFFFu;
                  if (tag == kRecFlip) {
                    const uint32_t sl_idx = (r.x >> 16) | ((r.y & 0xFFFFu) << 16);
                    const uint32_t row = (r.y >> 16) | ((r.z & 0xFFFFu) << 16);
                    atomicXor(&SL[sl_idx * G + w], bit);
                    if ((L.flags & LF_OUT_MEAS) && (SL[kept_off + w] & bit) &&
                        (uint64_t)w + (uint64_t)tile * G < L.row_words32)
                      atomicXor(&L.meas[(size_t)row * L.row_words32 + (uint64_t)tile * G + w], bit);
                  } else if (tag == kRecLong) {
                    const uint32_t site = (ent >> 10) / kRecPerSite, opt = (ent >> 10) % kRecPerSite;
                    const uint32_t info = __ldg(p.site_info + site);
                    const uint2 o2 = __ldg(reinterpret_cast<const uint2*>(p.opt_tab) + (info >> 8) + opt);
                    for (uint32_t q = 0; q < o2.y; q++)
                      atomicXor(&PL[(uint32_t)__ldg(p.plist + o2.x + q) * G + w], bit);
                  } else {
                    const uint32_t ent7[7] = {r.x >> 16, r.y & 0xFFFFu, r.y >> 16, r.z & 0xFFFFu,
                                              r.z >> 16, r.w & 0xFFFFu, r.w >> 16};
#pragma unroll
                    for (uint32_t q = 0; q < 7; q++)
                      if (q < tag) atomicXor(&PL[ent7[q] * G + w], bit);
                  }
                }
                __syncwarp();
              }
              break;
            }
            if (owner_warp) {
              while (true) {
                // due entries of this lane's words (site < block end) and the
                // minimum site among the others, then warp-wide compaction
                uint32_t due[W];
                uint32_t cnt = 0, nmin = kNoFault >> 4;
                const bool scanned = owner && minsite < op.i1;
#pragma unroll
                for (int i = 0; i < W; i++) {
                  due[i] = 0;
                  if (scanned)
                    for (uint32_t j = 0; j < 32; j++) {
                      const uint32_t sv = NF[j * G + tw + i] >> 4;
                      if (sv < op.i1) due[i] |= 1u << j;
                      else nmin = min(nmin, sv);
                    }
                  cnt += __popc(due[i]);
                }
                uint32_t incl = cnt;
#pragma unroll
                for (uint32_t d = 1; d < 32; d <<= 1) {
                  uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
                  if (lane >= d) incl += v;
                }
                const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
                if (total == 0) break;
                uint32_t pos = incl - cnt;
#pragma unroll
                for (int i = 0; i < W; i++) {
                  uint32_t d = due[i];
                  while (d && pos < kQueue) {
                    uint32_t j = __ffs(d) - 1;
                    d &= d - 1;
                    QU[pos++] = (uint16_t)((((lane * W) + i) << 5) | j);
                  }
                }
                __syncwarp();
                const uint32_t n_q = min(total, kQueue);
                for (uint32_t qi = lane; qi < n_q; qi += 32) {
                  const uint32_t e = QU[qi];
                  const uint32_t w = (warp * 32u * W) + (e >> 5), j = e & 31u, bit = 1u << j;
                  const uint64_t shot = tile_s0 + (uint64_t)w * 32u + j;
                  const uint64_t sl = ((uint64_t)tile * G + w) * 32u + j;  // call-local shot
                  uint32_t f = NF[j * G + w];
                  do {
                    const uint32_t site = f >> 4, opt = f & 15u;
                    // next fault of this shot (independent of the application below)
                    uint32_t fn = kNoFault;
                    bool search = false;
                    if (L.flist) {
                      const uint32_t c = CUR[j * G + w];
                      const uint32_t cn = L.fcount[sl];
                      if (c < (cn & 127u)) {
                        fn = L.flist[(uint64_t)c * L.fstride + sl];
                        CUR[j * G + w] = (uint8_t)(c + 1);
                      } else {
                        search = (cn & 128u) != 0;
                      }
                    } else {
                      search = true;
                    }
                    const uint4 r = __ldg(p.orec + (size_t)site * kRecPerSite + opt);
                    const uint32_t tag = r.x & 0xFFFFu;
                    if (tag == kRecFlip) {
                      const uint32_t sl_idx = (r.x >> 16) | ((r.y & 0xFFFFu) << 16);
                      const uint32_t row = (r.y >> 16) | ((r.z & 0xFFFFu) << 16);
                      atomicXor(&SL[sl_idx * G + w], bit);
                      if ((L.flags & LF_OUT_MEAS) && (SL[kept_off + w] & bit) &&
                          (uint64_t)w + (uint64_t)tile * G < L.row_words32)
                        atomicXor(&L.meas[(size_t)row * L.row_words32 + (uint64_t)tile * G + w], bit);
                    } else if (tag == kRecLong) {
                      const uint32_t info = __ldg(p.site_info + site);
                      const uint2 o2 = __ldg(reinterpret_cast<const uint2*>(p.opt_tab) + (info >> 8) + opt);
                      for (uint32_t q = 0; q < o2.y; q++)
                        atomicXor(&PL[(uint32_t)__ldg(p.plist + o2.x + q) * G + w], bit);
                    } else {
                      const uint32_t ent7[7] = {r.x >> 16, r.y & 0xFFFFu, r.y >> 16, r.z & 0xFFFFu,
                                                r.z >> 16, r.w & 0xFFFFu, r.w >> 16};
#pragma unroll
                      for (uint32_t q = 0; q < 7; q++)
                        if (q < tag) atomicXor(&PL[ent7[q] * G + w], bit);
                    }
                    if (search) fn = next_fault(p, L.seed, shot, site + 1);
                    f = fn;
                  } while ((f >> 4) < op.i1);
                  NF[j * G + w] = f;
                }
                __syncwarp();
                if (scanned) {
                  // only the entries just processed can have moved
                  uint32_t m = nmin;
#pragma unroll
                  for (int i = 0; i < W; i++) {
                    uint32_t d = due[i];
                    while (d) {
                      uint32_t j = __ffs(d) - 1;
                      d &= d - 1;
                      m = min(m, NF[j * G + tw + i] >> 4);
                    }
                  }
                  minsite = m;
                }
                if (total <= kQueue) break;
              }
            }
            break;
          case OP_FEEDFORWARD:
            if (owner) {
              const Vw<W> c = vld<W>(slot(op.i2));
              if (op.pa != kNoInline) {
                auto flip = [&](uint32_t pl) {
                  Vw<W> v = vld<W>(plane(pl));
                  vxor<W>(v, c);
                  vst<W>(plane(pl), v);
                };
                switch (op.pa) {
                  case 4: flip(ent(op, 3)); [[fallthrough]];
                  case 3: flip(ent(op, 2)); [[fallthrough]];
                  case 2: flip(ent(op, 1)); [[fallthrough]];
                  case 1: flip(ent(op, 0)); [[fallthrough]];
                  default: break;
                }
              } else {
                const uint32_t* mk = p.masks + op.i0;
                for (uint32_t part = 0; part < 2; part++)
                  for (uint32_t w = 0; w < p.nw; w++) {
                    uint32_t bits = __ldg(mk + part * p.nw + w);
                    while (bits) {
                      uint32_t q = w * 32u + (__ffs(bits) - 1);
                      bits &= bits - 1;
                      Vw<W> v = vld<W>(plane(part * N + q));
                      vxor<W>(v, c);
                      vst<W>(plane(part * N + q), v);
                    }
                  }
              }
            }
            break;
          case OP_REC_OUT:
            if (owner && (L.flags & LF_OUT_MEAS))
              store(L.meas, op.i3, vand<W>(vld<W>(slot(op.i2)), vld<W>(slot(p.kept_slot))));
            break;
          case OP_DETECTOR:
          case OP_OBS_INCLUDE:
            if (owner) {
              Vw<W> d = vfill<W>(0u);
              if (op.pa != kNoInline) {
                // entries past the count point at the zero slot
                vxor<W>(d, vld<W>(slot(ent(op, 0))));
                vxor<W>(d, vld<W>(slot(ent(op, 1))));
                vxor<W>(d, vld<W>(slot(ent(op, 2))));
                vxor<W>(d, vld<W>(slot(ent(op, 3))));
              } else {
                for (uint32_t j = 0; j < op.i1; j++) vxor<W>(d, vld<W>(slot(__ldg(p.slot_list + op.i0 + j))));
              }
              if (op.code == OP_OBS_INCLUDE) {
                Vw<W> o = vld<W>(slot(op.i2));
                vxor<W>(o, d);
                vst<W>(slot(op.i2), o);
              } else {
                if (!(L.flags & LF_REFERENCE) && (op.flags & FLAG_REF)) vxor<W>(d, vfill<W>(~0u));
                Vw<W> kept = vld<W>(slot(p.kept_slot));
                if (L.flags & LF_OUT_DET) store(L.det, op.i3, vand<W>(d, kept));
                if (L.flags & LF_POSTSELECT) {
#pragma unroll
                  for (int i = 0; i < W; i++) kept.v[i] &= ~d.v[i];
                  vst<W>(slot(p.kept_slot), kept);
                }
              }
            }
            break;
          case OP_OBS_OUT:
            if (owner && (L.flags & LF_OUT_OBS)) {
              Vw<W> v = vld<W>(slot(op.i2));
              if (!(L.flags & LF_REFERENCE) && (op.flags & FLAG_REF)) vxor<W>(v, vfill<W>(~0u));
              store(L.obs, op.i3, vand<W>(v, vld<W>(slot(p.kept_slot))));
            }
            break;
          case OP_KEPT_OUT:
            if (owner) {
              const Vw<W> kept = vld<W>(slot(p.kept_slot));
              if (L.flags & LF_OUT_KEPT) store(L.kept, 0, kept);
              uint32_t c = 0;
#pragma unroll
              for (int i = 0; i < W; i++) c += __popc(kept.v[i]);
              if (c) atomicAdd(L.kept_count, (unsigned long long)c);
            }
            break;
          case OP_EXPVAL: {
            // ---- expectation probe (Sec. 3.2): <P> = (-1)^(frame sign) Re(i^pa
            // <phi| X^i1 Z^i2 |phi>) / <phi|phi>, FP64 sums per shot ----
            if (!(L.flags & LF_OUT_EXPVAL)) break;
            __syncthreads();
            const bool odd = (op.pa & 1u) != 0;
            if (!op.pb && k > 0) {
              for (uint32_t s = t; s < S; s += T) {
                RED[s] = 0.0;
                RED[S + s] = 0.0;
              }
              __syncthreads();
              const uint32_t dim = 1u << k, mx = op.i1, mz = op.i2;
              for (uint32_t s = t % S; s < S; s += T) {
                double acc = 0.0, nrm = 0.0;
                for (uint32_t j = sub; j < dim; j += R) {
                  const C a = work[(size_t)j * S + s], b = work[(size_t)(j ^ mx) * S + s];
                  const double ax = a.x, ay = a.y, bx = b.x, by = b.y;
                  const double v = odd ? bx * ay - by * ax : bx * ax + by * ay;  // conj(b) a
                  acc += (__popc(j & mz) & 1u) ? -v : v;
                  nrm += ax * ax + ay * ay;
                }
                atomicAdd(&RED[s], acc);
                atomicAdd(&RED[S + s], nrm);
              }
              __syncthreads();
            }
            if (owner) {
              // frame sign: parity(fx & z) ^ parity(fz & x) of the image M(P)
              const uint32_t* mk = p.masks + op.i0;
              Vw<W> om = vfill<W>(0u);
              for (uint32_t w = 0; w < p.nw; w++) {
                uint32_t bx = __ldg(mk + w), bz = __ldg(mk + p.nw + w);
                while (bz) {
                  vxor<W>(om, vld<W>(plane(w * 32u + (__ffs(bz) - 1))));
                  bz &= bz - 1;
                }
                while (bx) {
                  vxor<W>(om, vld<W>(plane(N + w * 32u + (__ffs(bx) - 1))));
                  bx &= bx - 1;
                }
              }
              const Vw<W> kept = vld<W>(slot(p.kept_slot));
              const double sg = (op.pa == 1 || op.pa == 2) ? -1.0 : 1.0;
#pragma unroll
              for (int i = 0; i < W; i++)
                for (uint32_t j = 0; j < 32; j++) {
                  const uint64_t sl = (word0 + i) * 32u + j;  // call-local shot
                  if (sl >= L.shots) break;
                  const uint32_t s = (tw + i) * 32u + j;      // shot in the tile
                  double v = 0.0;
                  if (!op.pb && ((kept.v[i] >> j) & 1u)) {
                    double part = odd ? 0.0 : 1.0;
                    if (k > 0) part = RED[S + s] > 0.0 ? RED[s] / RED[S + s] : 0.0;
                    v = ((om.v[i] >> j) & 1u) ? -sg * part : sg * part;
                  }
                  L.expval[(size_t)op.i3 * L.shots + sl] = v;
                }
            }
            __syncthreads();
            break;
          }
          case OP_DIAGF:
          case OP_MIXF:
          case OP_PERMF: {
            // ---- fused array passes (fuse.cpp): amplitude i at p = A i ^ c ----
            __syncthreads();
            const FTerm* TG = p.fterm + op.i2 + (op.code == OP_MIXF ? 1u : 0u);
            const uint32_t nt = op.i3, ns = min(nt, kFTermSmem);
            FTerm* FT = reinterpret_cast<FTerm*>(smem + lay.ft);
            for (uint32_t e = t; e < 2 * ns; e += T)
              reinterpret_cast<uint4*>(FT)[e] = __ldg(reinterpret_cast<const uint4*>(TG) + e);
            __syncthreads();
            // product of the deferred diagonal phases at physical indices q0 and
            // q1 (a pair, or the same index twice): quarter turns from CZ / S,
            // complex factors from ROTZ
            auto phase2 = [&](C& v0, C& v1, uint32_t q0, uint32_t q1, uint32_t s, bool pair) {
              uint32_t qt0 = 0, qt1 = 0;
              for (uint32_t e = 0; e < nt; e++) {
                const FTerm& tm = e < ns ? FT[e] : TG[e];
                const uint32_t kind = tm.kind & 255u;
                const uint32_t a0 = (__popc(q0 & tm.r1) ^ (tm.kind >> 8)) & 1u;
                const uint32_t a1 = pair ? (__popc(q1 & tm.r1) ^ (tm.kind >> 8)) & 1u : 0u;
                if (!(a0 | a1)) continue;
                if (kind == FT_CZ) {
                  qt0 += (a0 & (__popc(q0 & tm.r2) ^ (tm.kind >> 9))) << 1;
                  if (pair) qt1 += (a1 & (__popc(q1 & tm.r2) ^ (tm.kind >> 9))) << 1;
                } else if (kind == FT_S) {
                  qt0 += a0;
                  qt1 += a1;
                } else {
                  C ph;
                  ph.x = (real)tm.cs;
                  ph.y = (real)(fbit(PL + tm.plane * G, s) ? -tm.sn : tm.sn);
                  if (a0) v0 = cmul(v0, ph);
                  if (a1) v1 = cmul(v1, ph);
                }
              }
              auto turn = [](C v, uint32_t q) {
                C r = v;
                switch (q & 3u) {
                  case 1: r.x = -v.y; r.y = v.x; break;
                  case 2: r.x = -v.x; r.y = -v.y; break;
                  case 3: r.x = v.y; r.y = -v.x; break;
                  default: break;
                }
                return r;
              };
              v0 = turn(v0, qt0);
              if (pair) v1 = turn(v1, qt1);
            };
            const uint32_t dim = 1u << k;
            if (op.code == OP_DIAGF) {
              for (uint32_t s = t % S; s < S; s += T)
                for (uint32_t j = sub; j < dim; j += R) {
                  C v = work[(size_t)j * S + s], dummy = v;
                  phase2(v, dummy, j, j, s, false);
                  work[(size_t)j * S + s] = v;
                }
            } else if (op.code == OP_MIXF) {
              const FTerm lead = p.fterm[op.i2];
              const uint32_t m = op.i0, r = op.i1 & 0x7FFFFFFFu, rc = op.i1 >> 31, piv = op.pa;
              const real rs = (real)0.70710678118654752440;
              for (uint32_t s = t % S; s < S; s += T) {
                const real cr = (real)lead.cs, sr = (real)(fbit(PL + lead.plane * G, s) ? -lead.sn : lead.sn);
                for (uint32_t j = sub; j < dim / 2; j += R) {
                  uint32_t q0 = insert0(j, piv), q1 = q0 ^ m;
                  if ((__popc(q0 & r) ^ rc) & 1u) {
                    const uint32_t x = q0;
                    q0 = q1;
                    q1 = x;
                  }
                  if ((q0 | q1) >= dim) {  // cannot happen for a well-formed list
                    atomicOr(L.err, 2u);
                    continue;
                  }
                  const size_t i0 = (size_t)q0 * S + s, i1 = (size_t)q1 * S + s;
                  C a = work[i0], b = work[i1];
                  phase2(a, b, q0, q1, s, true);
                  C na, nb;
                  if (op.pb == 0) {
                    na = cscale(cadd(a, b), rs);
                    nb = cscale(csub(a, b), rs);
                  } else {
                    na.x = cr * a.x + sr * b.y;
                    na.y = cr * a.y - sr * b.x;
                    nb.x = sr * a.y + cr * b.x;
                    nb.y = -sr * a.x + cr * b.y;
                  }
                  work[i0] = na;
                  work[i1] = nb;
                }
              }
            } else {
              // gather into logical order: new[i] = phase(q) old[q], q = A i ^ c
              const uint32_t* cols = p.fperm + op.i0;
              const uint32_t kk = op.i1, c0 = __ldg(cols + kk);
              auto src = [&](uint32_t j) -> uint32_t {
                uint32_t q = c0, bits = j;
                while (bits) {
                  q ^= __ldg(cols + (__ffs(bits) - 1));
                  bits &= bits - 1;
                }
                return q;
              };
              if (op.flags & FLAG_SUMS) {
                // gathered in the next measurement's amplitude pairs, whose
                // FP64 sums are formed on the way (the measurement's own
                // reduction, same pairs in the same order per thread)
                const uint32_t mpa = op.pa;
                const bool xm = op.pb != 0;
                for (uint32_t s = t; s < S; s += T) {
                  RED[s] = 0.0;
                  RED[S + s] = 0.0;
                }
                __syncthreads();
                for (uint32_t s = t % S; s < S; s += T) {
                  double a0 = 0.0, a1 = 0.0;
                  for (uint32_t j = sub; j < dim / 2; j += R) {
                    const uint32_t j0 = insert0(j, mpa), j1 = j0 | (1u << mpa);
                    const uint32_t q0 = src(j0), q1 = src(j1);
                    if ((q0 | q1) >= dim) {  // cannot happen for a well-formed list
                      atomicOr(L.err, 2u);
                      continue;
                    }
                    C v0 = work[(size_t)q0 * S + s], v1 = work[(size_t)q1 * S + s], d0 = v0, d1 = v1;
                    phase2(v0, d0, q0, q0, s, false);
                    phase2(v1, d1, q1, q1, s, false);
                    work2[(size_t)j0 * S + s] = v0;
                    work2[(size_t)j1 * S + s] = v1;
                    if (xm) {
                      mterm_x(v0, v1, a0, a1);
                    } else {
                      a0 += mterm(v0);
                      a1 += mterm(v1);
                    }
                  }
                  atomicAdd(&RED[s], a0);
                  atomicAdd(&RED[S + s], a1);
                }
              } else {
                for (uint32_t s = t % S; s < S; s += T)
                  for (uint32_t j = sub; j < dim; j += R) {
                    const uint32_t q = src(j);
                    if (q >= dim) {  // cannot happen for a well-formed list
                      atomicOr(L.err, 2u);
                      continue;
                    }
                    C v = work[(size_t)q * S + s], dummy = v;
                    phase2(v, dummy, q, q, s, false);
                    work2[(size_t)j * S + s] = v;
                  }
              }
              __syncthreads();
              C* const x = work;
              work = work2;
              work2 = x;
            }
            __syncthreads();
            break;
          }
          default: {
            // ---- instructions on the active array (all threads) ----
            if (is_meas(op.code) && L.stop_event != 0xffffffffu && op.i1 == L.stop_event) goto dump;
            const uint32_t code = op.code;
            if (owner && code >= OP_ARRAY_H && code <= OP_ARRAY_CZ) {
              // frame part of the array Clifford
              if (code == OP_ARRAY_H) {
                Vw<W> a = vld<W>(plane(op.a)), b = vld<W>(plane(N + op.a));
                vst<W>(plane(op.a), b);
                vst<W>(plane(N + op.a), a);
              } else if (code == OP_ARRAY_S) {
                Vw<W> zz = vld<W>(plane(N + op.a));
                vxor<W>(zz, vld<W>(plane(op.a)));
                vst<W>(plane(N + op.a), zz);
              } else if (code == OP_ARRAY_CX) {
                Vw<W> xb = vld<W>(plane(op.b)), za = vld<W>(plane(N + op.a));
                vxor<W>(xb, vld<W>(plane(op.a)));
                vxor<W>(za, vld<W>(plane(N + op.b)));
                vst<W>(plane(op.b), xb);
                vst<W>(plane(N + op.a), za);
              } else {
                Vw<W> xa = vld<W>(plane(op.a)), xb = vld<W>(plane(op.b));
                Vw<W> za = vld<W>(plane(N + op.a)), zb = vld<W>(plane(N + op.b));
                vxor<W>(za, xb);
                vxor<W>(zb, xa);
                vst<W>(plane(N + op.a), za);
                vst<W>(plane(N + op.b), zb);
              }
            }
            if (code < OP_ARRAY_H || code > OP_MEAS_ACTIVE_X) break;
            __syncthreads();
            const uint32_t pa = op.pa;
            if (code == OP_EXPAND_ROT) {
              const double c2 = op.cs, s2 = op.sn;
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
              const double c2 = op.cs, s2 = op.sn;
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
              const double c1 = op.cs, s1 = op.sn;
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
                    size_t i0 = (size_t)(base | (1u << pa)) * S + s;
                    size_t i1 = (size_t)(base | (1u << pa) | (1u << pb)) * S + s;
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
              if (!(op.flags & FLAG_PRESUMMED)) {  // else the gather before formed the sums
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
                      mterm_x(u, v, a0, a1);
                    } else {
                      a0 += mterm(u);
                      a1 += mterm(v);
                    }
                  }
                  atomicAdd(&RED[s], a0);
                  atomicAdd(&RED[S + s], a1);
                }
              }
              __syncthreads();
              if (owner) {
                const uint64_t g = s0 >> 7;
                const uint4 tb = philox(make_uint4((uint32_t)g, (uint32_t)(g >> 32), TAG_MT, op.i0), key_of(L.seed));
                const uint32_t sel = (uint32_t)(s0 >> 5) & 3u;
                const uint32_t abit = (op.flags & FLAG_SIGN) ? 1u : 0u;
                const Vw<W> kept = vld<W>(slot(p.kept_slot));
                Vw<W> mw, xa = vld<W>(plane(op.a)), za = vld<W>(plane(N + op.a));
#pragma unroll
                for (int i = 0; i < W; i++) {
                  const uint32_t top = pick4(tb, (sel + i) & 3u);
                  const uint32_t pw = xm ? za.v[i] : xa.v[i];
                  uint32_t m32 = 0, b32 = 0;
                  for (uint32_t j = 0; j < 32; j++) {
                    const uint32_t s = (tw + i) * 32u + j;
                    const double S0 = RED[s], S1 = RED[S + s], tot = S0 + S1;
                    const uint32_t pbit = (pw >> j) & 1u;
                    const double p1 = tot > 0.0 ? ((1u ^ abit ^ pbit) ? S1 : S0) / tot : 0.0;
                    const uint32_t m = !((valid.v[i] >> j) & 1u) ? 0u
                                       : (L.flags & LF_ARGMAX)     ? (p1 > 0.5 ? 1u : 0u)
                                           : draw_outcome(L.seed, s0 + (uint64_t)i * 32u + j, op.i0, (top >> j) & 1u, p1);
                    const uint32_t b = m ^ abit ^ pbit;
                    const double sb = b ? S1 : S0;
                    RED[s] = sb > 0.0 ? 1.0 / sqrt(sb) : 0.0;
                    m32 |= m << j;
                    b32 |= b << j;
                  }
                  mw.v[i] = m32;
                  TMP[tw + i] = b32;
                  if (xm) {
                    const uint32_t ox = xa.v[i];
                    xa.v[i] = za.v[i] ^ b32;
                    za.v[i] = ox;
                  } else {
                    xa.v[i] ^= b32;
                  }
                }
                vst<W>(plane(op.a), xa);
                vst<W>(plane(N + op.a), za);
                vst<W>(slot(op.i2), mw);
                if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) store(L.meas, op.i3, vand<W>(mw, kept));
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
            break;
          }
        }
        continue;
      dump:
        // debug stop: copy the frame and amplitudes of one shot, then leave
        cp_async_wait_all();
        __syncthreads();
        if (t == 0) {
          const uint32_t ds = (uint32_t)(L.dump_shot - tile * (uint64_t)S);
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
      cp_async_wait_all();
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Reference parities into instruction flags: FLAG_REF on DETECTOR / OBS_OUT
// instructions whose det_ref / obs_ref entry is 1 (cleared otherwise).
// ---------------------------------------------------------------------------
__global__ void patch_ref_flags(Op* ops, uint32_t n_ops, const uint32_t* det_ref, const uint32_t* obs_ref) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_ops) return;
  const uint8_t c = ops[i].code;
  if (c != OP_DETECTOR && c != OP_OBS_OUT) return;
  const uint32_t r = c == OP_DETECTOR ? det_ref[ops[i].i3] : obs_ref[ops[i].i3];
  ops[i].flags = (uint8_t)((ops[i].flags & ~FLAG_REF) | (r ? FLAG_REF : 0));
}

cudaError_t launch_patch_ref(Op* ops, uint32_t n_ops, const uint32_t* det_ref, const uint32_t* obs_ref,
                             cudaStream_t st) {
  if (!n_ops) return cudaSuccess;
  patch_ref_flags<<<(n_ops + 255) / 256, 256, 0, st>>>(ops, n_ops, det_ref, obs_ref);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fault bucketing: one CTA of 1024 threads per 1024-shot warp-tile, one
// thread per shot. Each thread samples its shot's faults (Sec. 3.2 jump),
// then the CTA counting-sorts them by noise block into a compact global
// array (the order inside a block is free: fault effects are XORs). A shot
// with more than kBucketCap faults or a full global array sets *ovf, and the
// host then uses the per-shot path.
// ---------------------------------------------------------------------------
constexpr uint32_t kBucketCap = 32;

__global__ void __launch_bounds__(1024) bucket_faults(LaunchParams L, uint32_t* ents, uint32_t* offs,
                                                      uint64_t cap_total, unsigned long long* total,
                                                      uint32_t* ovf) {
  extern __shared__ uint32_t bsm[];
  const uint32_t nb = L.p.n_blocks;
  uint32_t* cnt = bsm;            // [nb]
  uint32_t* pre = bsm + nb;       // [nb + 1]
  __shared__ uint32_t wsum[32];
  __shared__ unsigned long long base_s;
  const uint32_t t = threadIdx.x, wt = blockIdx.x;
  for (uint32_t i = t; i < nb; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const uint64_t sl = (uint64_t)wt * 1024u + t;
  uint32_t loc[kBucketCap];
  uint32_t n = 0;
  if (sl < L.shots) {
    const uint64_t shot = L.shot_offset + sl;
    uint32_t r = L.p.sg_k;
    uint32_t f = next_fault_r(L.p, L.seed, shot, 0, r);
    while (f != kNoFault) {
      if (n == kBucketCap) {
        atomicOr(ovf, 1u);
        break;
      }
      const uint32_t site = f >> 4;
      loc[n++] = f;
      atomicAdd(&cnt[__ldg(L.p.site_blk + site)], 1u);
      f = next_fault_r(L.p, L.seed, shot, site + 1, r);
    }
  }
  __syncthreads();
  // exclusive scan of cnt: each thread sums a contiguous run, then a block scan
  const uint32_t per = (nb + blockDim.x - 1) / blockDim.x;
  const uint32_t lo = min(nb, t * per), hi = min(nb, lo + per);
  uint32_t s = 0;
  for (uint32_t i = lo; i < hi; i++) s += cnt[i];
  uint32_t incl = s;
  const uint32_t lane = t & 31u, wid = t >> 5;
#pragma unroll
  for (uint32_t d = 1; d < 32; d <<= 1) {
    uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t v = lane < (blockDim.x >> 5) ? wsum[lane] : 0u, inc = v;
#pragma unroll
    for (uint32_t d = 1; d < 32; d <<= 1) {
      uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
      if (lane >= d) inc += u;
    }
    wsum[lane] = inc - v;  // exclusive warp offsets
    if (lane == 31) {
      const unsigned long long b = atomicAdd(total, (unsigned long long)inc);
      base_s = b;
      if (b + inc > cap_total) atomicOr(ovf, 1u);
    }
  }
  __syncthreads();
  uint32_t run = wsum[wid] + incl - s;
  for (uint32_t i = lo; i < hi; i++) {
    pre[i] = run;
    run += cnt[i];
  }
  if (hi == nb && lo < hi) pre[nb] = run;
  if (nb == 0 && t == 0) pre[0] = 0;
  __syncthreads();
  const unsigned long long base = base_s;
  for (uint32_t i = t; i <= nb; i += blockDim.x) offs[(size_t)wt * (nb + 1) + i] = (uint32_t)(base + pre[i]);
  __syncthreads();
  // cursors start at the block offsets
  for (uint32_t i = t; i < nb; i += blockDim.x) cnt[i] = pre[i];
  __syncthreads();
  for (uint32_t i = 0; i < n; i++) {
    const uint32_t site = loc[i] >> 4, opt = loc[i] & 15u;
    const uint32_t pos = atomicAdd(&cnt[__ldg(L.p.site_blk + site)], 1u);
    if (base + pos < cap_total) ents[base + pos] = ((site * kRecPerSite + opt) << 10) | t;
  }
}

cudaError_t launch_bucket(const LaunchParams& L, uint32_t n_wt, uint32_t* ents, uint32_t* offs, uint64_t cap_total,
                          unsigned long long* total, uint32_t* ovf, cudaStream_t st) {
  const size_t smem = (size_t)(2 * L.p.n_blocks + 1) * 4;
  cudaError_t e = cudaFuncSetAttribute(bucket_faults, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  bucket_faults<<<n_wt, 1024, smem, st>>>(L, ents, offs, cap_total, total, ovf);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fault pre-sampling: one thread per shot, no shared memory, so the latency-
// bound search of Sec. 3.2's jump runs at full occupancy. Fault j of shot s
// is stored at flist[j * fstride + s] (shot-minor: coalesced stores).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) presample_faults(LaunchParams L) {
  const uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= L.fstride) return;
  uint32_t n = 0;
  bool ovf = false;
  if (s < L.shots) {
    const uint64_t shot = L.shot_offset + s;
    uint32_t r = L.p.sg_k;
    uint32_t f = next_fault_r(L.p, L.seed, shot, 0, r);
    uint32_t* dst = const_cast<uint32_t*>(L.flist);
    while (f != kNoFault) {
      if (n == L.fcap) {
        ovf = true;
        break;
      }
      dst[(uint64_t)n * L.fstride + s] = f;
      n++;
      f = next_fault_r(L.p, L.seed, shot, (f >> 4) + 1, r);
    }
  }
  const_cast<uint8_t*>(L.fcount)[s] = (uint8_t)(n | (ovf ? 128u : 0u));
}

cudaError_t launch_presample(const LaunchParams& L, cudaStream_t st) {
  const uint32_t threads = 256;
  const uint64_t blocks = (L.fstride + threads - 1) / threads;
  presample_faults<<<(uint32_t)blocks, threads, 0, st>>>(L);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Thread-per-shot executor: one thread per shot, its 2^k amplitudes in global
// memory (amplitude-major, shot-minor, so a warp's accesses coalesce).
// exec_plain<double> is the plain FP64 form; exec_plain<float> keeps FP32
// amplitudes with FP64 measurement sums (the batched form's precision), a
// layout for small vectors and short calls.
// ---------------------------------------------------------------------------
constexpr uint32_t kPlainMaxW = 8;       // N <= 256
constexpr uint32_t kPlainMaxSlots = 2048;

// Call-local shot sl of the program L describes, by one thread of a full
// warp (32 consecutive shots); amplitude i of the shot lives at
// work[i * stride + slot].
template <typename real>
__device__ __forceinline__ void plain_shot(const LaunchParams& L, uint64_t sl, void* work, uint64_t stride,
                                           uint64_t slot) {
  using C = typename Cx<real>::T;
  const DevProg& p = L.p;
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t word = sl >> 5;
  const bool valid = sl < L.shots;
  const uint64_t s = L.shot_offset + sl;
  const uint64_t s0 = s & ~31ull;
  uint32_t x[kPlainMaxW], z[kPlainMaxW], slots[kPlainMaxSlots / 32];
  for (uint32_t w = 0; w < kPlainMaxW; w++) x[w] = z[w] = 0;
  for (uint32_t w = 0; w < kPlainMaxSlots / 32; w++) slots[w] = 0;
  C* A = reinterpret_cast<C*>(work);
  auto amp = [&](uint32_t i) -> C& { return A[(size_t)i * stride + slot]; };
  auto mk = [](real re, real im) -> C {
    C c;
    c.x = re;
    c.y = im;
    return c;
  };
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
  uint32_t nr = p.sg_k;  // stratified: faults this shot still holds
  uint32_t nf = (valid && !(L.flags & LF_NOISELESS) && p.n_sites) ? next_fault_r(p, L.seed, s, 0, nr) : kNoFault;
  uint32_t k = 0;
  if (p.k_max > 0) amp(0) = mk((real)1, (real)0);
  const real rs = (real)0.70710678118654752440;

  for (uint32_t pc = 0; pc < p.n_ops; pc++) {
    const Op op = p.ops[pc];
    if (L.stop_event != 0xffffffffu && is_meas(op.code) && op.i1 == L.stop_event) {
      if (sl == L.dump_shot) {
        for (uint32_t w = 0; w < p.nw; w++) {
          L.dump_frame[w] = x[w];
          L.dump_frame[p.nw + w] = z[w];
        }
        for (uint32_t i = 0; i < (1u << k); i++) {
          L.dump_amps[2 * i] = (double)amp(i).x;
          L.dump_amps[2 * i + 1] = (double)amp(i).y;
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
            C u = amp(i0), v = amp(i1);
            amp(i0) = mk((u.x + v.x) * rs, (u.y + v.y) * rs);
            amp(i1) = mk((u.x - v.x) * rs, (u.y - v.y) * rs);
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
            C u = amp(i1);
            amp(i1) = mk(-u.y, u.x);
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
            C u = amp(i0);
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
            C u = amp(i);
            amp(i) = mk(-u.x, -u.y);
          }
        }
        break;
      }
      case OP_EXPAND_ROT: {
        const real c2 = (real)(op.cs * 0.70710678118654752440),
                   s2 = (real)((getb(x, op.a) ? -op.sn : op.sn) * 0.70710678118654752440);
        const uint32_t n = 1u << k;
        for (uint32_t i = 0; i < n; i++) {
          C u = amp(i);
          amp(i) = mk(u.x * rs, u.y * rs);
          amp(i + n) = mk(u.x * c2 - u.y * s2, u.x * s2 + u.y * c2);
        }
        k++;
        break;
      }
      case OP_ROT_Z: {
        const real c2 = (real)op.cs, s2 = (real)(getb(x, op.a) ? -op.sn : op.sn);
        for (uint32_t j = 0; j < (1u << (k - 1)); j++) {
          uint32_t i1 = insert0(j, op.pa) | (1u << op.pa);
          C u = amp(i1);
          amp(i1) = mk(u.x * c2 - u.y * s2, u.x * s2 + u.y * c2);
        }
        break;
      }
      case OP_ROT_X: {
        const real c1 = (real)op.cs, s1 = (real)(getb(z, op.a) ? -op.sn : op.sn);
        for (uint32_t j = 0; j < (1u << (k - 1)); j++) {
          uint32_t i0 = insert0(j, op.pa), i1 = i0 | (1u << op.pa);
          C a = amp(i0), b = amp(i1);
          amp(i0) = mk(c1 * a.x + s1 * b.y, c1 * a.y - s1 * b.x);
          amp(i1) = mk(s1 * a.y + c1 * b.x, -s1 * a.x + c1 * b.y);
        }
        break;
      }
      case OP_MEAS_STATIC: {
        uint32_t par = (op.flags & FLAG_SIGN) ? 1u : 0u;
        for (uint32_t w = 0; w < p.nw; w++) par ^= __popc(x[w] & __ldg(p.masks + op.i0 + w)) & 1u;
        if (op.flags & FLAG_RESET) {
          // fused reset: conditional X-image on the inline planes r[0..pb)
          for (uint32_t r = 0; r < op.pb; r++) {
            const uint32_t pl = rent(op, r);
            if (pl < p.n_qubits) flipb(x, pl, par);
            else flipb(z, pl - p.n_qubits, par);
          }
        } else {
          setb(slots, op.i2, par);
          if ((op.flags & FLAG_OUT) && (L.flags & LF_OUT_MEAS)) store(L.meas, op.i3, par & kept);
        }
        break;
      }
      case OP_MEAS_RANDOM: {
        uint32_t top = (meas_top_word(L.seed, s0, op.i0) >> lane) & 1u;
        uint32_t m = (L.flags & LF_ARGMAX) ? 0u : top ^ 1u;
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
          C u = amp(i0), v = amp(i1);
          if (xm) {
            const real px = u.x + v.x, py = u.y + v.y, mx = u.x - v.x, my = u.y - v.y;
            S0 += 0.5 * (double)(px * px + py * py);
            S1 += 0.5 * (double)(mx * mx + my * my);
          } else {
            S0 += (double)(u.x * u.x + u.y * u.y);
            S1 += (double)(v.x * v.x + v.y * v.y);
          }
        }
        const uint32_t pbit = xm ? getb(z, op.a) : getb(x, op.a);
        const uint32_t abit = (op.flags & FLAG_SIGN) ? 1u : 0u;
        const double tot = S0 + S1;
        const double p1 = tot > 0.0 ? ((1u ^ abit ^ pbit) ? S1 : S0) / tot : 0.0;
        const uint32_t top = (meas_top_word(L.seed, s0, op.i0) >> lane) & 1u;
        const uint32_t m = !valid ? 0u : (L.flags & LF_ARGMAX) ? (p1 > 0.5 ? 1u : 0u) : draw_outcome(L.seed, s, op.i0, top, p1);
        const uint32_t b = m ^ abit ^ pbit;
        const double sb = b ? S1 : S0;
        const real sc = (real)(sb > 0.0 ? 1.0 / sqrt(sb) : 0.0);
        if (pa == top_pos) {
          for (uint32_t j = 0; j < half; j++) {
            C o0 = amp(j), o1 = amp(j + half), v;
            if (xm) v = b ? mk((o0.x - o1.x) * rs, (o0.y - o1.y) * rs) : mk((o0.x + o1.x) * rs, (o0.y + o1.y) * rs);
            else v = b ? o1 : o0;
            amp(j) = mk(v.x * sc, v.y * sc);
          }
        } else {
          for (uint32_t j = 0; j < (1u << (k - 2)); j++) {
            uint32_t base = insert0(insert0(j, pa), top_pos);
            uint32_t p00 = base, p10 = base | (1u << pa), p01 = base | (1u << top_pos), p11 = p10 | (1u << top_pos);
            C n0, n1;
            if (xm) {
              C o00 = amp(p00), o10 = amp(p10), o01 = amp(p01), o11 = amp(p11);
              const real sg = b ? (real)-1 : (real)1;
              n0 = mk((o00.x + sg * o10.x) * rs, (o00.y + sg * o10.y) * rs);
              n1 = mk((o01.x + sg * o11.x) * rs, (o01.y + sg * o11.y) * rs);
            } else {
              n0 = b ? amp(p10) : amp(p00);
              n1 = b ? amp(p11) : amp(p01);
            }
            amp(p00) = mk(n0.x * sc, n0.y * sc);
            amp(p10) = mk(n1.x * sc, n1.y * sc);
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
            if ((L.flags & LF_OUT_MEAS) && getb(slots, p.kept_slot)) {
              const uint32_t row = __ldg(p.opt_tab + 2 * (info >> 8) + 1);
              atomicXor(&L.meas[(size_t)row * L.row_words32 + word], 1u << lane);
            }
          } else {
            const uint32_t* mk = p.masks + eff + opt * 2u * p.nw;
            for (uint32_t w = 0; w < p.nw; w++) {
              x[w] ^= __ldg(mk + w);
              z[w] ^= __ldg(mk + p.nw + w);
            }
          }
          nf = next_fault_r(p, L.seed, s, site + 1, nr);
        }
        break;
      case OP_EXPVAL: {
        // expectation probe: (-1)^(frame sign) Re(i^pa <phi| X^i1 Z^i2 |phi>) / <phi|phi>
        if (!(L.flags & LF_OUT_EXPVAL) || !valid) break;
        double v = 0.0;
        if (!op.pb && getb(slots, p.kept_slot)) {
          const bool odd = (op.pa & 1u) != 0;
          double part = odd ? 0.0 : 1.0;
          if (k > 0) {
            double acc = 0.0, nrm = 0.0;
            for (uint32_t j = 0; j < (1u << k); j++) {
              const C ac = amp(j), bc = amp(j ^ op.i1);
              const double2 a = make_double2((double)ac.x, (double)ac.y), b = make_double2((double)bc.x, (double)bc.y);
              const double t1 = odd ? b.x * a.y - b.y * a.x : b.x * a.x + b.y * a.y;
              acc += (__popc(j & op.i2) & 1u) ? -t1 : t1;
              nrm += a.x * a.x + a.y * a.y;
            }
            part = nrm > 0.0 ? acc / nrm : 0.0;
          }
          uint32_t om = 0;
          for (uint32_t w = 0; w < p.nw; w++)
            om ^= __popc(x[w] & __ldg(p.masks + op.i0 + p.nw + w)) ^ __popc(z[w] & __ldg(p.masks + op.i0 + w));
          const double sg = (op.pa == 1 || op.pa == 2) ? -1.0 : 1.0;
          v = (om & 1u) ? -sg * part : sg * part;
        }
        L.expval[(size_t)op.i3 * L.shots + sl] = v;
        break;
      }
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
size_t batched_smem_bytes(const DevProg& p, uint32_t G, uint32_t W, bool bk, uint32_t work_words) {
  return smem_layout(p.n_qubits, p.n_slots, p.k_max, G, W, bk, work_words).bytes;
}

template <typename real, int W, bool BIG, bool BK>
static cudaError_t launch_one(const LaunchParams& L, uint32_t grid, uint32_t threads, size_t smem, cudaStream_t st) {
  auto fn = exec_batched<real, W, BIG, BK>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, threads, smem, st>>>(L);
  return cudaGetLastError();
}

template <typename real, int W, bool BIG, bool BK>
static cudaError_t occ_one(uint32_t threads, size_t smem, int* per_sm) {
  auto fn = exec_batched<real, W, BIG, BK>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, (int)threads, smem);
}

// Dispatch over (precision, words per thread, CTA size class, bucketed
// noise). W > 1 and the bucketed variant exist only for CTAs of at most 256
// threads; the bucketed variant only for W = 1.
template <typename real>
static cudaError_t launch_t(const LaunchParams& L, uint32_t W, bool bk, uint32_t grid, uint32_t threads, size_t smem,
                            cudaStream_t st) {
  if (threads > 256) return launch_one<real, 1, true, false>(L, grid, threads, smem, st);
  if (bk) return launch_one<real, 1, false, true>(L, grid, threads, smem, st);
  if (W == 4) return launch_one<real, 4, false, false>(L, grid, threads, smem, st);
  if (W == 2) return launch_one<real, 2, false, false>(L, grid, threads, smem, st);
  return launch_one<real, 1, false, false>(L, grid, threads, smem, st);
}

template <typename real>
static cudaError_t occ_t(uint32_t W, bool bk, uint32_t threads, size_t smem, int* per_sm) {
  if (threads > 256) return occ_one<real, 1, true, false>(threads, smem, per_sm);
  if (bk) return occ_one<real, 1, false, true>(threads, smem, per_sm);
  if (W == 4) return occ_one<real, 4, false, false>(threads, smem, per_sm);
  if (W == 2) return occ_one<real, 2, false, false>(threads, smem, per_sm);
  return occ_one<real, 1, false, false>(threads, smem, per_sm);
}

cudaError_t launch_batched(const LaunchParams& L, bool fp64, uint32_t W, bool bk, uint32_t grid, uint32_t threads,
                           size_t smem, cudaStream_t st) {
  return fp64 ? launch_t<double>(L, W, bk, grid, threads, smem, st)
              : launch_t<float>(L, W, bk, grid, threads, smem, st);
}

cudaError_t batched_occupancy(bool fp64, uint32_t W, bool bk, uint32_t threads, size_t smem, int* per_sm) {
  return fp64 ? occ_t<double>(W, bk, threads, smem, per_sm) : occ_t<float>(W, bk, threads, smem, per_sm);
}

// ---------------------------------------------------------------------------
// Shared prefix: the frame, array and rotation instructions before the first
// noise, measurement or record instruction act alike on every shot (the frame
// stays zero, so every rotation takes its unsigned angle). They run once per
// call on one vector spread over the whole grid, one launch per instruction,
// with the executor's own update formulas; the executor then starts every
// shot from that vector.
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(256) prefix_init(typename Cx<real>::T* v) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    v[0].x = (real)1;
    v[0].y = (real)0;
  }
}

template <typename real>
__global__ void __launch_bounds__(256) prefix_pass(const Op op, typename Cx<real>::T* v, uint32_t k) {
  using C = typename Cx<real>::T;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  const real rs = (real)0.70710678118654752440;
  const uint32_t pa = op.pa;
  switch (op.code) {
    case OP_EXPAND_ROT: {
      const uint32_t n = 1u << k;
      C ph;
      ph.x = (real)op.cs * rs;
      ph.y = (real)op.sn * rs;
      for (uint32_t j = tid; j < n; j += nt) {
        const C a = v[j];
        v[j] = cscale(a, rs);
        v[j + n] = cmul(a, ph);
      }
      break;
    }
    case OP_ROT_Z: {
      C ph;
      ph.x = (real)op.cs;
      ph.y = (real)op.sn;
      for (uint32_t j = tid; j < (1u << (k - 1)); j += nt) {
        const uint32_t i1 = insert0(j, pa) | (1u << pa);
        v[i1] = cmul(v[i1], ph);
      }
      break;
    }
    case OP_ROT_X: {
      const real cr = (real)op.cs, sr = (real)op.sn;
      for (uint32_t j = tid; j < (1u << (k - 1)); j += nt) {
        const uint32_t i0 = insert0(j, pa), i1 = i0 | (1u << pa);
        const C a = v[i0], b = v[i1];
        C na, nb;
        na.x = cr * a.x + sr * b.y;
        na.y = cr * a.y - sr * b.x;
        nb.x = sr * a.y + cr * b.x;
        nb.y = -sr * a.x + cr * b.y;
        v[i0] = na;
        v[i1] = nb;
      }
      break;
    }
    case OP_ARRAY_H:
      for (uint32_t j = tid; j < (1u << (k - 1)); j += nt) {
        const uint32_t i0 = insert0(j, pa), i1 = i0 | (1u << pa);
        const C a = v[i0], b = v[i1];
        v[i0] = cscale(cadd(a, b), rs);
        v[i1] = cscale(csub(a, b), rs);
      }
      break;
    case OP_ARRAY_S:
      for (uint32_t j = tid; j < (1u << (k - 1)); j += nt) {
        const uint32_t i1 = insert0(j, pa) | (1u << pa);
        const C a = v[i1];
        C r;
        r.x = -a.y;
        r.y = a.x;
        v[i1] = r;
      }
      break;
    case OP_ARRAY_CX:
    case OP_ARRAY_CZ: {
      const uint32_t pb = op.pb, lo = min(pa, pb), hi = max(pa, pb);
      for (uint32_t j = tid; j < (1u << (k - 2)); j += nt) {
        const uint32_t base = insert0(insert0(j, lo), hi);
        if (op.code == OP_ARRAY_CX) {
          const uint32_t i0 = base | (1u << pa), i1 = i0 | (1u << pb);
          const C a = v[i0];
          v[i0] = v[i1];
          v[i1] = a;
        } else {
          const uint32_t i = base | (1u << pa) | (1u << pb);
          C a = v[i];
          a.x = -a.x;
          a.y = -a.y;
          v[i] = a;
        }
      }
      break;
    }
    default:
      break;  // frame instructions: the frame stays zero
  }
}

// Runs ops [0, p.prefix_end) of the program on vec (2^k_max amplitudes of the
// given precision); returns the launches made.
cudaError_t launch_prefix(const Op* host_ops, uint32_t n, bool fp64, void* vec, int n_sm, cudaStream_t st,
                          uint32_t* launches) {
  *launches = 0;
  if (fp64) prefix_init<double><<<1, 32, 0, st>>>(reinterpret_cast<double2*>(vec));
  else prefix_init<float><<<1, 32, 0, st>>>(reinterpret_cast<float2*>(vec));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  (*launches)++;
  uint32_t k = 0;
  for (uint32_t pc = 0; pc < n; pc++) {
    const Op& o = host_ops[pc];
    if (o.code < OP_ARRAY_H || o.code > OP_ROT_X) continue;  // frame instructions
    const uint32_t work = o.code == OP_EXPAND_ROT ? (1u << k)
                          : (o.code == OP_ARRAY_CX || o.code == OP_ARRAY_CZ) ? (1u << (k - 2)) : (1u << (k - 1));
    uint32_t grid = (work + 255) / 256;
    if (grid > 8u * (uint32_t)n_sm) grid = 8u * (uint32_t)n_sm;
    if (grid < 1) grid = 1;
    if (fp64) prefix_pass<double><<<grid, 256, 0, st>>>(o, reinterpret_cast<double2*>(vec), k);
    else prefix_pass<float><<<grid, 256, 0, st>>>(o, reinterpret_cast<float2*>(vec), k);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    (*launches)++;
    if (o.code == OP_EXPAND_ROT) k++;
  }
  return cudaSuccess;
}

template <typename real>
__global__ void __launch_bounds__(128) exec_plain(const __grid_constant__ LaunchParams L) {
  // this launch covers call-local shots [plain_base, plain_base + plain_n)
  const uint64_t sl = L.plain_base + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t padded = L.row_words32 * 32u;
  if ((sl & ~31ull) >= padded || sl - L.plain_base >= L.plain_n) return;  // whole warps only
  plain_shot<real>(L, sl, L.work, L.plain_n, sl - L.plain_base);
}

// Many programs in one persistent launch (the batching row of Sec. 3.2):
// item j is 128 shots of one program, program i owning items
// [item0[i], item0[i + 1]) (programs ordered longest first by the host).
// CTAs take items from the counter `next`, stage the item's launch
// parameters in shared memory, and run one shot per thread; each thread
// keeps one vector slot of the workspace (2^k_max of the batch amplitudes,
// slot = global thread index, stride = threads of the launch).
template <typename real>
__global__ void __launch_bounds__(128) exec_plain_multi(const LaunchParams* __restrict__ Ls,
                                                        const unsigned long long* __restrict__ item0,
                                                        uint32_t n_progs, unsigned long long* next, void* work) {
  static_assert(sizeof(LaunchParams) % 4 == 0, "launch parameters copied as words");
  __shared__ __align__(16) uint32_t lsh[sizeof(LaunchParams) / 4];
  __shared__ unsigned long long it_sh;
  __shared__ uint32_t prog_sh;
  const LaunchParams& L = *reinterpret_cast<const LaunchParams*>(lsh);
  const uint64_t n_items = item0[n_progs];
  const uint64_t slot = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t cur = 0xffffffffu;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned long long it = atomicAdd(next, 1ull);
      uint32_t lo = 0, hi = n_progs;  // the program with item0[i] <= it < item0[i + 1]
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (item0[mid] <= it) lo = mid;
        else hi = mid;
      }
      it_sh = it;
      prog_sh = lo;
    }
    __syncthreads();
    const unsigned long long it = it_sh;
    const uint32_t pi = prog_sh;
    if (it >= n_items) break;
    if (pi != cur) {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(Ls + pi);
      for (uint32_t w = threadIdx.x; w < sizeof(LaunchParams) / 4; w += blockDim.x) lsh[w] = src[w];
      cur = pi;
      __syncthreads();
    }
    const uint64_t sl = (it - item0[pi]) * blockDim.x + threadIdx.x;
    if ((sl & ~31ull) < L.row_words32 * 32u) plain_shot<real>(L, sl, work, stride, slot);
    __syncthreads();  // the item and parameters stay until every thread is done
  }
}

// Stores one program's launch parameters (and its first item) for the
// multi-program launch: a kernel, so that a captured graph needs no host
// memory at replay.
__global__ void store_params(const __grid_constant__ LaunchParams L, LaunchParams* dst, unsigned long long* item0,
                             unsigned long long first, unsigned long long end, uint32_t last) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&L);
  uint32_t* d = reinterpret_cast<uint32_t*>(dst);
  for (uint32_t w = threadIdx.x; w < sizeof(LaunchParams) / 4; w += blockDim.x) d[w] = src[w];
  if (threadIdx.x == 0) {
    item0[0] = first;
    if (last) item0[1] = end;
  }
}

// fp32: FP32 amplitudes (the thread-per-shot layout of the batched form),
// else the plain FP64 form.
cudaError_t launch_plain(const LaunchParams& L, cudaStream_t st, bool fp32) {
  const uint32_t threads = 128;
  const uint64_t blocks = (L.plain_n + threads - 1) / threads;
  if (fp32) exec_plain<float><<<(uint32_t)blocks, threads, 0, st>>>(L);
  else exec_plain<double><<<(uint32_t)blocks, threads, 0, st>>>(L);
  return cudaGetLastError();
}

// The multi-program thread-per-shot launch: parameters stored by one small
// launch per program, then one persistent launch of `grid` CTAs over every
// program's items. Ls: n device LaunchParams; item0: n + 1 device u64; next:
// a device u64 zeroed here; work: grid * 128 * 2^k_max amplitudes.
cudaError_t launch_plain_multi(const LaunchParams* hLs, uint32_t n, const uint64_t* h_items, LaunchParams* dLs,
                               unsigned long long* item0, unsigned long long* next, void* work, uint32_t grid,
                               bool fp32, cudaStream_t st) {
  uint64_t acc = 0;
  for (uint32_t i = 0; i < n; i++) {
    store_params<<<1, 128, 0, st>>>(hLs[i], dLs + i, item0 + i, acc, acc + h_items[i], i + 1 == n);
    acc += h_items[i];
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = cudaMemsetAsync(next, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (fp32) exec_plain_multi<float><<<grid, 128, 0, st>>>(dLs, item0, n, next, work);
  else exec_plain_multi<double><<<grid, 128, 0, st>>>(dLs, item0, n, next, work);
  return cudaGetLastError();
}

// resident CTAs of the multi-program launch per SM
cudaError_t plain_multi_occupancy(bool fp32, int* per_sm) {
  return fp32 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, exec_plain_multi<float>, 128, 0)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, exec_plain_multi<double>, 128, 0);
}

bool plain_supported(const DevProg& p) {
  return p.nw <= kPlainMaxW && p.n_slots <= kPlainMaxSlots;
}

}  // namespace nc
