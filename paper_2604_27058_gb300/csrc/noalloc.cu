// noalloc.cu — nc_sample_noalloc: FP32 batched sampling without any device
// allocation, for callers that cannot allocate device memory while they run
// (their device memory belongs to another framework's pool, or allocations
// are only allowed at start-up, or an allocation's implicit synchronisation
// is not acceptable in their loop).
//
// Every device byte the call needs comes from g_noalloc_scratch, a fixed
// file-scope device array of NC_NOALLOC_SCRATCH_BYTES that each device
// holds from module load until process exit. Host code cannot use the
// array's name as a device pointer (it is a host-side stand-in), so the
// device address is looked up once per device with cudaGetSymbolAddress, with
// that device current, on the first call there.
//
// Layout of the array for one call (each part 256-byte aligned):
//   [program blob][kept counter, error word][reference det/obs rows][amplitudes]
// Each call overwrites it; calls that overlap on the GPU race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/nc.h"
#include "kernels.cuh"

namespace nc {
size_t batched_smem_bytes(const DevProg& p, uint32_t G, uint32_t W, bool bk, uint32_t work_words = 0);
cudaError_t launch_batched(const LaunchParams& L, bool fp64, uint32_t W, bool bk, uint32_t grid, uint32_t threads,
                           size_t smem, cudaStream_t st);
cudaError_t batched_occupancy(bool fp64, uint32_t W, bool bk, uint32_t threads, size_t smem, int* blocks_per_sm);
const std::vector<uint8_t>& program_blob(const nc_program* p);
cudaError_t launch_patch_ref(Op* ops, uint32_t n_ops, const uint32_t* det_ref, const uint32_t* obs_ref,
                             cudaStream_t st);
}  // namespace nc

using namespace nc;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NC_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_addr[kMaxDevices];  // device address of g_noalloc_scratch per device (set-up once)

// Device address of g_noalloc_scratch on the current device (looked up once).
nc_status scratch_base(uint8_t** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NC_E_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NC_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return NC_E_CUDA;
    g_addr[dev] = (uint8_t*)p;
  }
  *out = g_addr[dev];
  return NC_OK;
}

uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

DevProg view(const ProgHeader& h, const uint8_t* base) {
  DevProg d{};
  d.ops = reinterpret_cast<const Op*>(base + h.off_ops);
  d.masks = reinterpret_cast<const uint32_t*>(base + h.off_masks);
  d.q = reinterpret_cast<const uint64_t*>(base + h.off_q);
  d.seg_start = reinterpret_cast<const uint32_t*>(base + h.off_seg_start);
  d.seg_end = reinterpret_cast<const uint32_t*>(base + h.off_seg_end);
  d.site_info = reinterpret_cast<const uint32_t*>(base + h.off_site_info);
  d.site_eff = reinterpret_cast<const uint32_t*>(base + h.off_site_eff);
  d.slot_list = reinterpret_cast<const uint32_t*>(base + h.off_slot_list);
  d.det_ref = reinterpret_cast<const uint32_t*>(base + h.off_det_ref);
  d.obs_ref = reinterpret_cast<const uint32_t*>(base + h.off_obs_ref);
  d.site_opt = reinterpret_cast<const uint32_t*>(base + h.off_site_opt);
  d.opt_tab = reinterpret_cast<const uint32_t*>(base + h.off_opt_tab);
  d.plist = reinterpret_cast<const uint16_t*>(base + h.off_plist);
  d.orec = reinterpret_cast<const uint4*>(base + h.off_orec);
  d.site_blk = reinterpret_cast<const uint32_t*>(base + h.off_site_blk);
  d.n_qubits = h.n_qubits;
  d.nw = h.nw;
  d.n_ops = h.n_ops;
  d.n_sites = h.n_sites;
  d.n_slots = h.n_slots;
  d.k_max = h.k_max;
  d.kept_slot = h.kept_slot;
  d.n_meas = h.n_meas;
  d.n_det = h.n_det;
  d.n_obs = h.n_obs;
  d.n_blocks = h.n_blocks;
  d.srch = reinterpret_cast<const uint32_t*>(base + h.off_srch);
  if (h.n_fops) {
    d.fops = reinterpret_cast<const Op*>(base + h.off_fops);
    d.fterm = reinterpret_cast<const FTerm*>(base + h.off_fterm);
    d.fperm = reinterpret_cast<const uint32_t*>(base + h.off_fperm);
    d.n_fops = h.n_fops;
    d.f_perm = h.f_perm;
  }
  d.guide = reinterpret_cast<const uint32_t*>(base + h.off_guide);
  if (h.aff_ok) {
    d.aff_const = reinterpret_cast<const uint32_t*>(base + h.off_aff_const);
    d.aff_rowev_off = reinterpret_cast<const uint32_t*>(base + h.off_aff_rowev_off);
    d.aff_rowev = reinterpret_cast<const uint32_t*>(base + h.off_aff_rowev);
    d.aff_rand_ev = reinterpret_cast<const uint32_t*>(base + h.off_aff_rand_ev);
    d.aff_col_off = reinterpret_cast<const uint32_t*>(base + h.off_aff_col_off);
    d.aff_chunks = reinterpret_cast<const uint4*>(base + h.off_aff_col);
    d.aff_frec = reinterpret_cast<const uint4*>(base + h.off_aff_frec);
    d.aff_parent = reinterpret_cast<const uint32_t*>(base + h.off_aff_parent);
    d.aff_chain_off = reinterpret_cast<const uint32_t*>(base + h.off_aff_chain_off);
    d.aff_chain = reinterpret_cast<const uint32_t*>(base + h.off_aff_chain);
    d.aff_n_chains = h.aff_n_chains;
    d.aff_n_chain_rows = h.aff_n_chain_rows;
    d.aff_chunks_per_shot = h.aff_chunks_per_shot;
    d.aff_rows = h.aff_rows;
    d.aff_n_rand = h.aff_n_rand;
  }
  return d;
}

// Launch shape by peak active dimension. This is a fixed table of its own,
// not nc_sample's tuned choice: its tiles are smaller for small k_max, and
// the speed-ups of nc_sample that need allocations (active vectors in shared
// memory, the shared noiseless prefix, pre-sampled noise) are not used. The
// records do not depend on the launch shape.
void shape(uint32_t k_max, uint32_t* G, uint32_t* T) {
  if (k_max == 0) { *G = 128; *T = 128; }
  else if (k_max <= 6) { *G = 32; *T = 256; }
  else if (k_max <= 10) { *G = 8; *T = 256; }
  else if (k_max <= 13) { *G = 2; *T = 512; }
  else { *G = 1; *T = 1024; }
}

// One executor launch (FP32 amplitudes, or FP64 for the reference launches
// as in nc_sample) whose amplitude workspace starts at `work` and may use
// `work_bytes`.
nc_status launch(const DevProg& d, bool fp64, uint64_t shots, uint64_t seed, uint64_t shot_offset, uint32_t flags,
                 uint32_t* meas, uint32_t* det, uint32_t* obs, uint32_t* kept, unsigned long long* kept_count,
                 uint32_t* err, uint8_t* work, uint64_t work_bytes, cudaStream_t stream) {
  LaunchParams L;
  std::memset(&L, 0, sizeof(L));
  L.p = d;
  L.seed = seed;
  L.shot_offset = shot_offset;
  L.shots = shots;
  L.meas = meas;
  L.det = det;
  L.obs = obs;
  L.kept = kept;
  L.row_words32 = 2 * ((shots + 63) / 64);
  L.flags = flags;
  L.kept_count = kept_count;
  L.err = err;
  L.stop_event = 0xffffffffu;
  uint32_t G, T;
  shape(d.k_max, &G, &T);
  while (G > 1 && batched_smem_bytes(d, G, 1, false) > 220 * 1024) G >>= 1;
  if (batched_smem_bytes(d, G, 1, false) > 220 * 1024) return NC_E_UNSUPPORTED;  // frame planes too large
  if (T < G) T = G;
  L.G = G;
  L.n_tiles = (uint32_t)((L.row_words32 + G - 1) / G);
  const size_t smem = batched_smem_bytes(d, G, 1, false);
  int per_sm = 0, n_sm = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NC_E_CUDA;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return NC_E_CUDA;
  if (batched_occupancy(fp64, 1, false, T, smem, &per_sm) != cudaSuccess) return NC_E_CUDA;
  if (per_sm < 1) return NC_E_UNSUPPORTED;
  uint64_t grid = std::min<uint64_t>(L.n_tiles, (uint64_t)per_sm * n_sm);
  if (d.k_max > 0) {
    L.work_stride = ((uint64_t)1 << d.k_max) * 32ull * G;
    const uint64_t per_cta = L.work_stride * (fp64 ? sizeof(double) : sizeof(float)) * 2 * (d.n_fops && d.f_perm ? 2 : 1);
    const uint64_t fit = work_bytes / per_cta;
    if (fit == 0) return NC_E_ARG;  // one tile's amplitudes exceed the fixed scratch
    grid = std::min<uint64_t>(grid, fit);
    L.work = work;
  }
  if (grid == 0) return NC_OK;
  if (launch_batched(L, fp64, 1, false, (uint32_t)grid, T, smem, stream) != cudaSuccess) return NC_E_CUDA;
  return NC_OK;
}

}  // namespace

extern "C" nc_status nc_sample_noalloc(const nc_program* prog, uint64_t shots, uint64_t seed,
                                       const nc_sample_opts* opts, nc_records* out, void* cuda_stream) {
  if (!prog || !out) return NC_E_ARG;
  nc_sample_opts o;
  std::memset(&o, 0, sizeof(o));
  o.precision = NC_FP32_BATCHED;
  o.outputs = NC_OUT_MEAS | NC_OUT_DET | NC_OUT_OBS | NC_OUT_KEPT;
  if (opts) o = *opts;
  if (o.precision != NC_FP32_BATCHED || (o.outputs & NC_OUT_HOST) || o.shot_offset % 128) return NC_E_ARG;
  if (o.postselect != NC_PS_NONE && o.postselect != NC_PS_ALL_DETECTORS) return NC_E_ARG;
  if (o.stratified) return NC_E_UNSUPPORTED;  // its tables are allocated on demand
  const std::vector<uint8_t>& blob = program_blob(prog);
  ProgHeader h;
  std::memcpy(&h, blob.data(), sizeof(h));
  if ((o.outputs & NC_OUT_EXPVAL) && h.n_probes) return NC_E_UNSUPPORTED;  // probes: nc_sample
  if (out->words_per_record != (shots + 63) / 64) return NC_E_ARG;
  if ((o.outputs & NC_OUT_MEAS) && h.n_meas && !out->meas) return NC_E_ARG;
  if ((o.outputs & NC_OUT_DET) && h.n_det && !out->det) return NC_E_ARG;
  if ((o.outputs & NC_OUT_OBS) && h.n_obs && !out->obs) return NC_E_ARG;
  if ((o.outputs & NC_OUT_KEPT) && !out->kept) return NC_E_ARG;
  if (h.n_sites >= (1u << 28) - 1) return NC_E_UNSUPPORTED;

  // carve the fixed array
  const uint64_t off_blob = 0;
  const uint64_t off_cnt = align256(off_blob + blob.size());
  const uint64_t off_ref = align256(off_cnt + 16);
  const uint64_t ref_bytes = (uint64_t)(h.n_det + h.n_obs) * 8;
  const uint64_t off_work = align256(off_ref + ref_bytes);
  if (off_work > NC_NOALLOC_SCRATCH_BYTES) return NC_E_ARG;  // program too large for the fixed scratch
  const uint64_t work_bytes = NC_NOALLOC_SCRATCH_BYTES - off_work;

  uint8_t* base = nullptr;
  nc_status st = scratch_base(&base);
  if (st != NC_OK) return st;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  uint8_t* dblob = base + off_blob;
  unsigned long long* cnt = (unsigned long long*)(base + off_cnt);
  uint32_t* err = (uint32_t*)(base + off_cnt + 8);
  const DevProg d = view(h, dblob);

  if (cudaMemcpyAsync(dblob, blob.data(), blob.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return NC_E_CUDA;
  // kept counter and error word; the error word is cleared once here and
  // read after the last launch, so it reports every launch of the call
  if (cudaMemsetAsync(cnt, 0, 16, stream) != cudaSuccess) return NC_E_CUDA;
  // reference parities of detectors / observables (64 noiseless shots)
  if (h.n_det + h.n_obs) {
    uint32_t* rdet = (uint32_t*)(base + off_ref);
    uint32_t* robs = rdet + 2 * h.n_det;
    // the reference trajectory: every measurement takes its more likely
    // outcome (0 on a tie), so all 64 shots agree; FP64 amplitudes, as in
    // nc_sample, so that a near-even choice is taken the same way
    st = launch(d, true, 64, 0, 0, LF_NOISELESS | LF_REFERENCE | LF_ARGMAX | LF_OUT_DET | LF_OUT_OBS, nullptr, rdet,
                robs, nullptr, cnt, err, base + off_work, work_bytes, stream);
    if (st != NC_OK) return st;
    // rows are read back and checked in fixed stack chunks (no host heap use)
    constexpr uint32_t kRows = 256;
    uint64_t rows[kRows];
    uint32_t ref[kRows];
    const uint32_t n_rows = h.n_det + h.n_obs;
    for (uint32_t r0 = 0; r0 < n_rows; r0 += kRows) {
      const uint32_t nr = std::min(kRows, n_rows - r0);
      if (cudaMemcpyAsync(rows, rdet + 2 * (size_t)r0, nr * 8, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess)
        return NC_E_CUDA;
      for (uint32_t i = 0; i < nr; i++) {
        if (rows[i] != 0 && rows[i] != ~0ull) return NC_E_INTERNAL;
        ref[i] = (uint32_t)(rows[i] & 1);
      }
      // detector rows come first, then observable rows; the blob keeps them apart
      for (uint32_t i = 0; i < nr;) {
        const uint32_t r = r0 + i;
        const bool is_det = r < h.n_det;
        const uint32_t run = is_det ? std::min(nr - i, h.n_det - r) : nr - i;
        uint8_t* dst = is_det ? dblob + h.off_det_ref + (size_t)r * 4 : dblob + h.off_obs_ref + (size_t)(r - h.n_det) * 4;
        if (cudaMemcpyAsync(dst, ref + i, run * 4, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
            cudaStreamSynchronize(stream) != cudaSuccess)
          return NC_E_CUDA;
        i += run;
      }
    }
    // 64 sampled noiseless shots: a detector that differs from its
    // reference in more than a quarter of them is not deterministic
    st = launch(d, true, 64, 0, 0, LF_NOISELESS | LF_REFERENCE | LF_OUT_DET | LF_OUT_OBS, nullptr, rdet, robs, nullptr,
                cnt, err, base + off_work, work_bytes, stream);
    if (st != NC_OK) return st;
    for (uint32_t r0 = 0; r0 < n_rows; r0 += kRows) {
      const uint32_t nr = std::min(kRows, n_rows - r0);
      if (cudaMemcpyAsync(rows, rdet + 2 * (size_t)r0, nr * 8, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return NC_E_CUDA;
      for (uint32_t i = 0; i < nr;) {
        const uint32_t r = r0 + i;
        const bool is_det = r < h.n_det;
        const uint32_t run = is_det ? std::min(nr - i, h.n_det - r) : nr - i;
        const uint8_t* src = is_det ? dblob + h.off_det_ref + (size_t)r * 4 : dblob + h.off_obs_ref + (size_t)(r - h.n_det) * 4;
        if (cudaMemcpyAsync(ref + i, src, run * 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess) return NC_E_CUDA;
        i += run;
      }
      if (cudaStreamSynchronize(stream) != cudaSuccess) return NC_E_CUDA;
      for (uint32_t i = 0; i < nr; i++)
        if (__builtin_popcountll(rows[i] ^ (ref[i] ? ~0ull : 0ull)) > 16) return NC_E_NONDET_DETECTOR;
    }
    if (launch_patch_ref(reinterpret_cast<Op*>(dblob + h.off_ops), h.n_ops,
                         reinterpret_cast<const uint32_t*>(dblob + h.off_det_ref),
                         reinterpret_cast<const uint32_t*>(dblob + h.off_obs_ref), stream) != cudaSuccess)
      return NC_E_CUDA;
  }
  if (cudaMemsetAsync(cnt, 0, 8, stream) != cudaSuccess) return NC_E_CUDA;  // the counter only
  uint32_t flags = 0;
  if (o.outputs & NC_OUT_MEAS) flags |= LF_OUT_MEAS;
  if (o.outputs & NC_OUT_DET) flags |= LF_OUT_DET;
  if (o.outputs & NC_OUT_OBS) flags |= LF_OUT_OBS;
  if (o.outputs & NC_OUT_KEPT) flags |= LF_OUT_KEPT;
  if (o.postselect == NC_PS_ALL_DETECTORS) flags |= LF_POSTSELECT;
  if (o.noiseless) flags |= LF_NOISELESS;
  if (shots) {
    st = launch(d, false, shots, seed, o.shot_offset, flags, (uint32_t*)out->meas, (uint32_t*)out->det,
                (uint32_t*)out->obs, (uint32_t*)out->kept, cnt, err, base + off_work, work_bytes, stream);
    if (st != NC_OK) return st;
  }
  unsigned long long kept = 0;
  uint32_t herr = 0;
  if (cudaMemcpyAsync(&kept, cnt, 8, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return NC_E_CUDA;
  out->shots_run = shots;
  out->shots_kept = shots ? kept : 0;
  out->kernel_ms = 0.0;
  out->exec_ms = 0.0;
  out->launches = (h.n_det + h.n_obs ? 2u : 0u) + (shots ? 1u : 0u);
  return herr ? NC_E_INTERNAL : NC_OK;
}
