// capi.cu — the C ABI declared in include/nc.h.
//
// Host-side orchestration only: compile (compiler.cpp), upload the program
// blob once per device, run the noiseless reference launch that fixes the
// detector / observable reference parities, size the launch, enqueue one of
// the two executors (kernels.cu) and read back the counters. No sampling is
// ever done on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/nc.h"
#include "compiler.h"
#include "kernels.cuh"

namespace nc {
size_t batched_smem_bytes(const DevProg& p, uint32_t G, uint32_t W, bool bk, uint32_t work_words = 0);
cudaError_t launch_batched(const LaunchParams& L, bool fp64, uint32_t W, bool bk, uint32_t grid, uint32_t threads,
                           size_t smem, cudaStream_t st);
cudaError_t batched_occupancy(bool fp64, uint32_t W, bool bk, uint32_t threads, size_t smem, int* blocks_per_sm);
cudaError_t launch_plain(const LaunchParams& L, cudaStream_t st, bool fp32);
cudaError_t launch_plain_multi(const LaunchParams* hLs, uint32_t n, const uint64_t* h_items, LaunchParams* dLs,
                               unsigned long long* item0, unsigned long long* next, void* work, uint32_t grid,
                               bool fp32, cudaStream_t st);
cudaError_t plain_multi_occupancy(bool fp32, int* per_sm);
cudaError_t launch_patch_ref(Op* ops, uint32_t n_ops, const uint32_t* det_ref, const uint32_t* obs_ref,
                             cudaStream_t st);
cudaError_t launch_presample(const LaunchParams& L, cudaStream_t st);
cudaError_t launch_prefix(const Op* host_ops, uint32_t n, bool fp64, void* vec, int n_sm, cudaStream_t st,
                          uint32_t* launches);
size_t affine_smem_bytes(const DevProg& p, uint32_t wpt);
bool warp_supported(const DevProg& p);
size_t warp_smem_bytes(const DevProg& p, bool fp64, uint32_t nwarps);
cudaError_t launch_warp(const LaunchParams& L, bool fp64, uint32_t nwarps, uint32_t grid, size_t smem,
                        cudaStream_t st, int* per_sm);
cudaError_t launch_affine(const LaunchParams& L, uint32_t wpt, uint32_t grid, size_t smem, cudaStream_t st,
                          int* per_sm);
cudaError_t launch_affine_items(const LaunchParams& L, uint32_t tile0, uint32_t n_tiles, uint32_t* items,
                                uint32_t cap, uint32_t* counts, uint32_t tile_shots, uint32_t grid, cudaStream_t st,
                                uint32_t minb);
cudaError_t launch_bucket(const LaunchParams& L, uint32_t n_wt, uint32_t* ents, uint32_t* offs, uint64_t cap_total,
                          unsigned long long* total, uint32_t* ovf, cudaStream_t st);
bool plain_supported(const DevProg& p);
}  // namespace nc

using namespace nc;

namespace {

struct DevCopy {
  int device = -1;
  uint8_t* blob = nullptr;
  bool ref_ready = false;
  nc_status ref_status = NC_OK;
  std::string tuned;  // launch shape chosen by nc_autotune ("" = heuristic)
  // stratified tables (strata.cpp) in one allocation: G_r rows r = 1..sg_rows,
  // then the guide parameters (3 u64 per row), then the guide entries
  double* sg = nullptr;
  const unsigned long long* sgr = nullptr;
  const uint32_t* sgg = nullptr;
  uint32_t sg_rows = 0;
};

}  // namespace

struct nc_program {
  CompiledProgram cp;
  nc_info info{};
  std::mutex mu;
  std::vector<DevCopy> devs;
  StrataTables strata;  // host stratified tables, built on first use (under mu)
};

namespace {

const ProgHeader& header(const nc_program* p) {
  return *reinterpret_cast<const ProgHeader*>(p->cp.blob.data());
}

DevProg dev_view(const ProgHeader& h, const uint8_t* base) {
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

void fill_info(nc_program* p) {
  const ProgHeader& h = header(p);
  nc_info& i = p->info;
  i.n_qubits = h.n_qubits;
  i.n_meas = h.n_meas;
  i.n_det = h.n_det;
  i.n_obs = h.n_obs;
  i.k_max = h.k_max;
  i.n_noise_sites = h.n_sites;
  i.n_ops = h.n_ops;
  i.n_events = h.n_events;
  i.n_slots = h.n_slots;
  i.n_probes = h.n_probes;
  i.array_bytes_fp32 = p->cp.counts.array_bytes;
  i.prefix_ops = h.prefix_end;
  i.prefix_k = h.prefix_k;
  i.prefix_bytes_fp32 = p->cp.counts.prefix_bytes;
  i.n_static = p->cp.counts.n_static;
  i.n_random = p->cp.counts.n_random;
  i.n_active_meas = p->cp.counts.n_active;
  i.n_array_ops = p->cp.counts.array_ops;
}

nc_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return NC_OK;
  if (e == cudaErrorMemoryAllocation) return NC_E_OOM;
  return NC_E_CUDA;
}

#define NC_TRY(expr)                        \
  do {                                      \
    cudaError_t _e = (expr);                \
    if (_e != cudaSuccess) {                \
      st = cuda_status(_e);                 \
      goto done;                            \
    }                                       \
  } while (0)

// Scratch allocations made on the caller's stream and released on it.
struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t get(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// Launch shape of the batched executor: G 32-shot words per tile, W words
// per owner thread (G / W owners), T threads per CTA; B = 0 turns the
// bucketed noise path off. A = 0 turns the record-level propagation path
// (programs with k_max = 0) off; AW forces its 32-shot words per tile; AI = 0
// makes it sample faults inside the tile kernel instead of in a separate
// high-occupancy pass; AV is the shots per pass pair (0: default); AC
// overrides the item-list capacity per tile (tiles whose list overflows
// sample in the tile kernel); AO = 1 overlaps the item passes (side stream,
// two item buffers) with the tile kernel, which then keeps one CTA per SM
// (slower on GB300 for the surface-code workload, so off by default).
struct Tuning {
  uint32_t G, T, W, B, A, AW, AI, AV, AC, PS, AO;  // PS = 1: pre-sample faults even for small calls
  uint32_t SW = 1;                                 // SW = 0: active vectors never in shared memory
  uint32_t PX = 1;  // shared prefix: 0 off, 1 when it saves enough traffic, 2 whenever it has array work
  uint32_t LW = 0;  // 1: warp-per-shot layout (exec_warp) for programs with active axes
  uint32_t LP = 0;  // 1: thread-per-shot layout (exec_plain<float>) for programs with active axes
  uint32_t AQ = 4;  // resident item-kernel CTAs per SM (2, 3, 4)
  uint32_t WN = 0;  // its warps per CTA (0: 8, fewer if the vectors do not fit)
};

Tuning choose_tuning(const DevProg& d, const char* tune, uint64_t shots, int n_sm) {
  Tuning t;
  if (d.k_max == 0) t = {128, 128, 1, 1, 1, 0, 1, 0, 0, 0, 0};
  else if (d.k_max <= 6) t = {64, 512, 1, 1, 1, 0, 1, 0, 0, 0, 0};
  else if (d.k_max <= 10) t = {16, 512, 1, 1, 1, 0, 1, 0, 0, 0, 0};
  else if (d.k_max <= 13) t = {2, 512, 1, 1, 1, 0, 1, 0, 0, 0, 0};
  else t = {1, 1024, 1, 1, 1, 0, 1, 0, 0, 0, 0};
  // small calls: smaller tiles, so that every SM gets one
  while (t.G > 1 && (shots + 32 * t.G - 1) / (32 * t.G) < (uint64_t)n_sm) t.G >>= 1;
  if (tune) {
    unsigned v = 0;
    const char* s = tune;
    while (*s) {
      if (sscanf(s, "g=%u", &v) == 1) t.G = v;
      else if (sscanf(s, "t=%u", &v) == 1) t.T = v;
      else if (sscanf(s, "w=%u", &v) == 1) t.W = v;
      else if (sscanf(s, "b=%u", &v) == 1) t.B = v;
      else if (sscanf(s, "a=%u", &v) == 1) t.A = v;
      else if (sscanf(s, "aw=%u", &v) == 1) t.AW = v;
      else if (sscanf(s, "ai=%u", &v) == 1) t.AI = v;
      else if (sscanf(s, "av=%u", &v) == 1) t.AV = v;
      else if (sscanf(s, "ac=%u", &v) == 1) t.AC = v;
      else if (sscanf(s, "ps=%u", &v) == 1) t.PS = v;
      else if (sscanf(s, "ao=%u", &v) == 1) t.AO = v;
      else if (sscanf(s, "sw=%u", &v) == 1) t.SW = v;
      else if (sscanf(s, "px=%u", &v) == 1) t.PX = v;
      else if (sscanf(s, "lw=%u", &v) == 1) t.LW = v;
      else if (sscanf(s, "lp=%u", &v) == 1) t.LP = v;
      else if (sscanf(s, "aq=%u", &v) == 1) t.AQ = v;
      else if (sscanf(s, "wn=%u", &v) == 1) t.WN = v;
      const char* c = strchr(s, ',');
      if (!c) break;
      s = c + 1;
    }
  }
  if (t.W != 1 && t.W != 2 && t.W != 4) t.W = 1;
  if (t.AQ < 2 || t.AQ > 4) t.AQ = 4;
  if (t.G < t.W) t.W = t.G;
  // keep the shared-memory footprint under the opt-in limit
  while (t.G > t.W && batched_smem_bytes(d, t.G, t.W, false) > 220 * 1024) t.G >>= 1;
  if (t.T < t.G / t.W) t.T = t.G / t.W;
  if (t.T < 32) t.T = 32;
  return t;
}

bool pow2(uint32_t v) { return v && !(v & (v - 1)); }

// Free device memory for sizing scratch. Under LF_ASYNC (possibly inside a
// stream capture) the device's total memory stands in, and an allocation
// that does not fit fails as NC_E_OOM.
cudaError_t free_memory(uint32_t lflags, size_t* free_b) {
  size_t total_b = 0;
  if (lflags & LF_ASYNC) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaDeviceProp pr;
    e = cudaGetDeviceProperties(&pr, dev);
    *free_b = pr.totalGlobalMem / 2;
    return e;
  }
  return cudaMemGetInfo(free_b, &total_b);
}

// Internal side streams (one per concurrent call and device), kept for
// reuse. A call orders its side-stream work after the caller's stream and
// makes the caller's stream wait for it before anything that depends on it.
struct SideStream {
  int dev = -1;
  cudaStream_t s = nullptr;
  SideStream() = default;
  SideStream(const SideStream&) = delete;
  SideStream& operator=(const SideStream&) = delete;
  static std::mutex& mu() {
    static std::mutex m;
    return m;
  }
  static std::vector<std::pair<int, cudaStream_t>>& pool() {
    static std::vector<std::pair<int, cudaStream_t>> v;
    return v;
  }
  cudaError_t acquire(int device) {
    dev = device;
    {
      std::lock_guard<std::mutex> g(mu());
      auto& v = pool();
      for (size_t i = 0; i < v.size(); i++)
        if (v[i].first == device) {
          s = v[i].second;
          v.erase(v.begin() + i);
          return cudaSuccess;
        }
    }
    return cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  }
  ~SideStream() {
    if (!s) return;
    std::lock_guard<std::mutex> g(mu());
    pool().push_back({dev, s});
  }
};

// A few events for ordering work between the caller's stream and a side
// stream (timing disabled), destroyed with the holder.
struct Events {
  std::vector<cudaEvent_t> ev;
  cudaError_t make(size_t n) {
    for (size_t i = 0; i < n; i++) {
      cudaEvent_t e = nullptr;
      cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (r != cudaSuccess) return r;
      ev.push_back(e);
    }
    return cudaSuccess;
  }
  ~Events() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

// Per-call scratch comes from the device's default stream-ordered pool. By
// default the pool hands freed memory back at every synchronisation, so a
// call would map its scratch (up to a few GB) anew each time; keeping it
// cached in the pool makes the next call's allocation free. This changes
// only this process's default pool, once per device.
void keep_pool_memory(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> g(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  done.push_back(dev);
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  uint64_t keep = ~0ull;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
}

// Get (uploading once) the device copy of a program for the current device.
nc_status device_copy(nc_program* p, DevCopy** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NC_E_CUDA;
  for (auto& c : p->devs)
    if (c.device == dev) {
      *out = &c;
      return NC_OK;
    }
  DevCopy c;
  c.device = dev;
  keep_pool_memory(dev);
  cudaError_t e = cudaMalloc(&c.blob, p->cp.blob.size());
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpy(c.blob, p->cp.blob.data(), p->cp.blob.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(c.blob);
    return cuda_status(e);
  }
  p->devs.push_back(c);
  *out = &p->devs.back();
  return NC_OK;
}

struct CallOut {
  uint32_t *meas, *det, *obs, *kept;
  double* expval = nullptr;
};

// Optional per-program timing: events around the executor launch and the
// number of kernels launched.
struct Timing {
  std::vector<cudaEvent_t> ev;  // pairs around each launch of the dominant kernel
  uint32_t launches = 0;
  uint32_t path = 0;  // bit 0: the shared prefix ran once for the call
  cudaError_t begin(cudaStream_t s) { return mark(s); }
  cudaError_t end(cudaStream_t s) { return mark(s); }
  cudaError_t mark(cudaStream_t s) {
    cudaEvent_t e = nullptr;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ev.push_back(e);
    return cudaEventRecord(e, s);
  }
  // summed device time of the bracketed launches (after the stream synced)
  float ms() const {
    float tot = 0.f;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float x = 0.f;
      if (cudaEventElapsedTime(&x, ev[i], ev[i + 1]) == cudaSuccess) tot += x;
    }
    return tot;
  }
  ~Timing() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
};

constexpr uint32_t kNoStratum = 0xffffffffu;
constexpr uint32_t kMaxStratum = 127;  // per-shot fault lists hold up to 127 entries

nc_status enqueue_multi_flags(const nc_program* const* progs, const std::vector<DevCopy*>& dcs,
                              const uint64_t* shots, const uint64_t* seeds, uint32_t n, const nc_sample_opts& o,
                              uint32_t lflags, const CallOut* cos, unsigned long long* kept_count, uint32_t* err,
                              Scratch& scratch, cudaStream_t stream, Timing* tm);

// Enqueue one sampling launch. kept_count must point to a zeroed device u64.
nc_status enqueue(const nc_program* prog, const DevCopy& dc, uint64_t shots, uint64_t seed,
                  uint64_t shot_offset, int precision, uint32_t lflags, const char* tune, CallOut o,
                  unsigned long long* kept_count, uint32_t* err, Scratch& scratch, cudaStream_t stream,
                  uint32_t stop_event = 0xffffffffu, uint64_t dump_shot = 0, double* dump_amps = nullptr,
                  uint32_t* dump_frame = nullptr, uint32_t* dump_k = nullptr, Timing* tm = nullptr,
                  uint32_t stratum = kNoStratum) {
  nc_status st = NC_OK;
  const ProgHeader& h = header(prog);
  LaunchParams L;
  std::memset(&L, 0, sizeof(L));
  L.p = dev_view(h, dc.blob);
  // stratified call (stratum K >= 1; K = 0 runs as noiseless): exactly K
  // faults per shot from the device tables
  const bool strat = stratum != kNoStratum && stratum > 0 && !(lflags & LF_NOISELESS);
  if (stratum == 0) lflags |= LF_NOISELESS;
  if (strat) {
    if (!dc.sg || dc.sg_rows < stratum || stop_event != 0xffffffffu) return NC_E_INTERNAL;
    L.p.sg = dc.sg;
    L.p.sgr = dc.sgr;
    L.p.sgg = dc.sgg;
    L.p.sg_k = stratum;
    L.p.sg_n = h.n_sites + 1;
  }
  L.seed = seed;
  L.shot_offset = shot_offset;
  L.shots = shots;
  L.meas = o.meas;
  L.expval = o.expval;
  if (!o.expval || !h.n_probes) lflags &= ~(uint32_t)LF_OUT_EXPVAL;
  L.det = o.det;
  L.obs = o.obs;
  L.kept = o.kept;
  L.row_words32 = 2 * ((shots + 63) / 64);
  L.flags = lflags;
  L.kept_count = kept_count;
  L.err = err;
  L.stop_event = stop_event;
  L.dump_shot = dump_shot;
  L.dump_amps = dump_amps;
  L.dump_frame = dump_frame;
  L.dump_k = dump_k;
  // the persistent thread-per-shot launch for one program (tune mp=1; mg=
  // sets its resident CTAs per SM)
  if (precision == NC_FP32_BATCHED && tune && strstr(tune, "mp=1") && !strat && stop_event == 0xffffffffu &&
      h.k_max > 0 && plain_supported(L.p)) {
    nc_sample_opts o1;
    std::memset(&o1, 0, sizeof(o1));
    o1.precision = NC_FP32_BATCHED;
    o1.shot_offset = shot_offset;
    o1.tune = tune;
    const nc_program* one = prog;
    std::vector<DevCopy*> d1{const_cast<DevCopy*>(&dc)};
    CallOut c1 = o;
    if (!(lflags & LF_OUT_EXPVAL)) c1.expval = nullptr;
    st = enqueue_multi_flags(&one, d1, &shots, &seed, 1, o1, lflags, &c1, kept_count, err, scratch, stream, tm);
    if (st != NC_E_UNSUPPORTED) return st;
    st = NC_OK;
  }
  // thread-per-shot layout: the plain FP64 form, or the FP32 batched form's
  // layout for small vectors (tune lp=1)
  bool lp32 = false;
  if (precision == NC_FP32_BATCHED && h.k_max > 0 && !strat && tune && strstr(tune, "lp=1")) {
    int n_sm_q = 0, dev_q = 0;
    NC_TRY(cudaGetDevice(&dev_q));
    NC_TRY(cudaDeviceGetAttribute(&n_sm_q, cudaDevAttrMultiProcessorCount, dev_q));
    lp32 = choose_tuning(L.p, tune, shots, n_sm_q).LP == 1 && plain_supported(L.p);
  }
  if (precision == NC_FP64_PLAIN || lp32) {
    if (!plain_supported(L.p)) return NC_E_UNSUPPORTED;
    // one vector of 2^k amplitudes per shot: launches over shot ranges whose
    // vectors fit in a quarter of the free memory
    const uint64_t padded = L.row_words32 * 32;
    uint64_t chunk = padded;
    if (h.k_max > 0) {
      size_t free_b = 0;
      NC_TRY(free_memory(lflags, &free_b));
      const uint64_t per_shot = ((uint64_t)1 << h.k_max) * (lp32 ? sizeof(float) : sizeof(double)) * 2;
      chunk = std::min<uint64_t>(padded, std::max<uint64_t>(128, (free_b / 4 / per_shot) & ~127ull));
      NC_TRY(scratch.get(&L.work, per_shot * chunk));
    }
    for (uint64_t b0 = 0; b0 < padded; b0 += chunk) {
      L.plain_base = b0;
      L.plain_n = std::min(chunk, padded - b0);
      if (tm) NC_TRY(tm->begin(stream));
      NC_TRY(launch_plain(L, stream, lp32));
      if (tm) {
        NC_TRY(tm->end(stream));
        tm->launches += 1;
      }
    }
  } else {
    int n_sm_dev = 0, dev_id = 0;
    NC_TRY(cudaGetDevice(&dev_id));
    NC_TRY(cudaDeviceGetAttribute(&n_sm_dev, cudaDevAttrMultiProcessorCount, dev_id));
    Tuning tu = choose_tuning(L.p, tune, shots, n_sm_dev);
    if (h.aff_ok && tu.A && !(lflags & (LF_POSTSELECT | LF_REFERENCE)) && stop_event == 0xffffffffu) {
      // record-level propagation sampler: tile of 32 * wpt shots per CTA of
      // 32 * wpt threads; the shape with the most resident warps wins
      int n_sm = 0, dev = 0;
      NC_TRY(cudaGetDevice(&dev));
      NC_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
      // with the item passes overlapped, the tile kernel keeps one CTA of
      // 512 threads per SM so that an item-pass CTA fits beside it
      // (item lists name chunks below 2^22: affine_kernel.cu chunk_item)
      const bool items = tu.AI && !(lflags & LF_NOISELESS) && h.n_sites > 0 && h.aff_n_chunks < (1u << 22);
      const bool overlap = items && tu.AO;
      uint32_t wpt = 0;
      int best_warps = 0, best_ctas = 0;
      for (uint32_t c : {32u, 16u, 8u}) {
        if (tu.AW && tu.AW != c) continue;
        if (overlap && !tu.AW && c != 16) continue;
        const size_t smem = affine_smem_bytes(L.p, c);
        if (smem > 227 * 1024) continue;
        int per_sm = 0;
        NC_TRY(launch_affine(L, c, 0, smem, stream, &per_sm));
        const int warps = per_sm * (int)c;
        if (per_sm > 0 && warps > best_warps) {
          best_warps = warps;
          best_ctas = per_sm;
          wpt = c;
        }
      }
      if (wpt) {
        const size_t smem = affine_smem_bytes(L.p, wpt);
        const uint32_t n_tiles = (uint32_t)((L.row_words32 + wpt - 1) / wpt);
        const uint32_t tile_shots = 32 * wpt;
        if (overlap) best_ctas = 1;
        // faults sampled by affine_items in passes of `wave` tiles, each
        // followed by the tile kernel on the same tiles
        uint32_t wave = n_tiles;
        uint32_t cap = 0;
        uint32_t *ibuf = nullptr, *cbuf = nullptr;
        if (items) {
          // default pass: one tile per warp of the item kernel (AQ CTAs of 16
          // warps per SM), so no warp is left with a second tile while the
          // others idle; the pass's item lists (16 KB per tile for the surface
          // code) then mostly stay in L2 for the tile kernel
          const uint64_t wave_shots = tu.AV ? tu.AV : 16ull * tu.AQ * (uint64_t)n_sm * tile_shots;
          wave = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, wave_shots / tile_shots));
          // list capacity per tile: mean + 10 sigma (a chunk count per fault
          // of at most 15, so the variance is below 16 x the mean) + slack
          // (stratified: K faults of the average chunk count per fault)
          const double per_shot = strat && h.mean_faults > 0.f
                                      ? (double)h.aff_chunks_per_shot / h.mean_faults * stratum
                                      : (double)h.aff_chunks_per_shot;
          const double mean = per_shot * tile_shots;
          cap = (uint32_t)(mean * 1.1 + 10.0 * std::sqrt(mean * 16.0) + 64.0);
          if (tu.AC) cap = tu.AC;
          // two buffers when the passes overlap: pass j + 1 fills one while
          // the tile kernel of pass j reads the other
          const size_t nbuf = overlap ? 2 : 1;
          void *a = nullptr, *b = nullptr;
          NC_TRY(scratch.get(&a, nbuf * wave * cap * 4));
          NC_TRY(scratch.get(&b, nbuf * wave * 4));
          ibuf = (uint32_t*)a;
          cbuf = (uint32_t*)b;
        }
        SideStream side;
        Events ev;  // [0] start, [1..2] items ready, [3..4] tile kernel done with a buffer
        cudaStream_t istream = stream;
        if (overlap) {
          NC_TRY(side.acquire(dev));
          NC_TRY(ev.make(5));
          istream = side.s;
          NC_TRY(cudaEventRecord(ev.ev[0], stream));
          NC_TRY(cudaStreamWaitEvent(istream, ev.ev[0], 0));
        }
        uint32_t pass = 0;
        for (uint32_t t0 = 0; t0 < n_tiles; t0 += wave, pass++) {
          const uint32_t nt = std::min(wave, n_tiles - t0);
          const uint32_t bsel = overlap ? (pass & 1u) : 0u;
          L.tile0 = t0;
          L.n_tiles = t0 + nt;
          if (items) {
            uint32_t* ib = ibuf + (size_t)bsel * wave * cap;
            uint32_t* cb = cbuf + (size_t)bsel * wave;
            if (overlap && pass >= 2) NC_TRY(cudaStreamWaitEvent(istream, ev.ev[3 + bsel], 0));
            const uint32_t grid = std::min<uint32_t>((nt + 15) / 16, tu.AQ * (uint32_t)n_sm);
            NC_TRY(launch_affine_items(L, t0, nt, ib, cap, cb, tile_shots, grid, istream, tu.AQ));
            if (overlap) {
              NC_TRY(cudaEventRecord(ev.ev[1 + bsel], istream));
              NC_TRY(cudaStreamWaitEvent(stream, ev.ev[1 + bsel], 0));
            }
            L.aff_items = ib;
            L.aff_counts = cb;
            L.aff_cap = cap;
            if (tm) tm->launches += 1;
          }
          const uint64_t grid = std::min<uint64_t>(nt, (uint64_t)best_ctas * n_sm);
          if (tm) NC_TRY(tm->begin(stream));
          NC_TRY(launch_affine(L, wpt, (uint32_t)grid, smem, stream, nullptr));
          if (tm) {
            NC_TRY(tm->end(stream));
            tm->launches += 1;
          }
          if (overlap) NC_TRY(cudaEventRecord(ev.ev[3 + bsel], stream));
        }
        return NC_OK;
      }
    }
    // warp-per-shot layout: one warp per shot, its vector in shared memory
    if (tu.LW == 1 && h.k_max > 0 && warp_supported(L.p)) {
      const bool fp64w = precision == NC_FP64_BATCHED;
      uint32_t nw = tu.WN ? std::min<uint32_t>(tu.WN, 8) : 8;
      while (nw > 1 && warp_smem_bytes(L.p, fp64w, nw) > 200 * 1024) nw--;
      const size_t smem = warp_smem_bytes(L.p, fp64w, nw);
      int per_sm = 0;
      if (smem <= 227 * 1024 && launch_warp(L, fp64w, nw, 0, smem, stream, &per_sm) == cudaSuccess && per_sm > 0) {
        int n_sm = 0, dev = 0;
        NC_TRY(cudaGetDevice(&dev));
        NC_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
        const uint64_t grid = std::min<uint64_t>(L.row_words32, (uint64_t)per_sm * n_sm);
        if (grid == 0) return NC_OK;
        if (tm) NC_TRY(tm->begin(stream));
        NC_TRY(launch_warp(L, fp64w, nw, (uint32_t)grid, smem, stream, nullptr));
        if (tm) {
          NC_TRY(tm->end(stream));
          tm->launches += 1;
        }
        return NC_OK;
      }
    }
    if (!pow2(tu.G) || !pow2(tu.T) || !pow2(tu.W) || tu.T > (tu.W == 1 ? 1024u : 256u) || tu.T < 32)
      return NC_E_ARG;
    L.G = tu.G;
    const uint64_t S = 32ull * tu.G;
    L.n_tiles = (uint32_t)((L.row_words32 + tu.G - 1) / tu.G);
    // fault pre-sampling (bucketed or per-shot lists) pays off only for
    // large calls; small ones sample faults inside the executor
    // (stratified shots are always pre-sampled: exactly K faults each)
    const bool noisy = !(lflags & LF_NOISELESS) && h.n_sites && stop_event == 0xffffffffu &&
                       (shots >= (1u << 20) || tu.PS || strat);
    const double mean = strat ? (double)stratum : (double)h.mean_faults;
    const double per_shot_cap = strat ? mean : std::ceil(mean + 6.0 * std::sqrt(mean) + 4.0);
    // Bucketed noise: every shot's faults sampled up front and sorted by
    // noise block per 1024-shot warp-tile (one owner word per lane).
    bool bk = false;
    if (noisy && tu.B && !(lflags & LF_ASYNC) && tu.W == 1 && tu.T <= 256 && tu.G >= 32 && h.n_blocks <= 8192 &&
        (uint64_t)h.n_sites * kRecPerSite < (1ull << 22) && per_shot_cap <= 32.0) {
      const uint32_t n_wt = L.n_tiles * (tu.G / 32);
      const double lam = mean * (double)shots;
      const uint64_t cap_total =
          strat ? (uint64_t)lam + 65536 : (uint64_t)(lam * 1.02 + 12.0 * std::sqrt(lam) + 65536.0);
      const size_t ents_b = cap_total * 4, offs_b = (size_t)n_wt * (h.n_blocks + 1) * 4;
      size_t free_b = 0;
      NC_TRY(free_memory(lflags, &free_b));
      if (cap_total < (1ull << 32) && ents_b + offs_b < free_b / 2) {
        void *ents = nullptr, *offs = nullptr, *ctr = nullptr;
        NC_TRY(scratch.get(&ents, ents_b));
        NC_TRY(scratch.get(&offs, offs_b));
        NC_TRY(scratch.get(&ctr, 16));
        NC_TRY(cudaMemsetAsync(ctr, 0, 16, stream));
        unsigned long long* total = (unsigned long long*)ctr;
        uint32_t* ovf = (uint32_t*)((char*)ctr + 8);
        NC_TRY(launch_bucket(L, n_wt, (uint32_t*)ents, (uint32_t*)offs, cap_total, total, ovf, stream));
        if (tm) tm->launches += 1;
        uint32_t h_ovf = 1;
        NC_TRY(cudaMemcpyAsync(&h_ovf, ovf, 4, cudaMemcpyDeviceToHost, stream));
        NC_TRY(cudaStreamSynchronize(stream));
        if (!h_ovf) {
          bk = true;
          L.bents = (const uint32_t*)ents;
          L.boffs = (const uint32_t*)offs;
        }
      }
    }
    const bool fp64 = precision == NC_FP64_BATCHED;
    // the tile's active vectors: shared memory when they fit beside the
    // planes (small tiles: latency-bound calls), else the global workspace;
    // two buffers per CTA when the fused list gathers (debug stops use the
    // original list)
    const bool two = h.n_fops && h.f_perm && stop_event == 0xffffffffu;
    size_t per_cta = 0;
    if (h.k_max > 0) {
      L.work_stride = ((size_t)1 << h.k_max) * S;
      per_cta = L.work_stride * (fp64 ? sizeof(double) : sizeof(float)) * 2 * (two ? 2 : 1);
      if (tu.SW && per_cta <= 64 * 1024 && batched_smem_bytes(L.p, tu.G, tu.W, bk, 0) + per_cta <= 200 * 1024)
        L.smem_work_words = (uint32_t)(per_cta / 4);
    }
    const size_t smem = batched_smem_bytes(L.p, tu.G, tu.W, bk, L.smem_work_words);
    int per_sm = 0, n_sm = 0, dev = 0;
    NC_TRY(cudaGetDevice(&dev));
    NC_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    NC_TRY(batched_occupancy(fp64, tu.W, bk, tu.T, smem, &per_sm));
    if (per_sm < 1) return NC_E_UNSUPPORTED;
    uint64_t grid = std::min<uint64_t>(L.n_tiles, (uint64_t)per_sm * n_sm);
    if (h.k_max > 0 && !L.smem_work_words) {
      size_t free_b = 0;
      NC_TRY(free_memory(lflags, &free_b));
      uint64_t cap = std::max<uint64_t>(1, (uint64_t)(free_b * 0.6) / per_cta);
      grid = std::min(grid, cap);
      NC_TRY(scratch.get(&L.work, per_cta * grid));
    }
    // otherwise pre-sample every shot's faults when the list buffer fits
    if (noisy && !bk) {
      const uint32_t cap = (uint32_t)std::min(127.0, per_shot_cap);
      const uint64_t padded = L.row_words32 * 32;
      const size_t bytes = (size_t)cap * padded * 4 + padded;
      size_t free_b = 0;
      NC_TRY(free_memory(lflags, &free_b));
      if (bytes < free_b / 2) {
        void* buf = nullptr;
        NC_TRY(scratch.get(&buf, bytes));
        L.flist = (const uint32_t*)buf;
        L.fcount = (const uint8_t*)buf + (size_t)cap * padded * 4;
        L.fcap = cap;
        L.fstride = padded;
        NC_TRY(launch_presample(L, stream));
        if (tm) tm->launches += 1;
      }
    }
    if (strat && !bk && !L.flist) return NC_E_OOM;  // stratified shots need their fault lists
    // the shared prefix (program.h prefix_end) once for the whole call, when
    // its traffic over all shots outweighs one launch per instruction; a
    // debug stop (the unfused list, from prefix_end) takes it only when forced
    if (h.prefix_end > 0 && h.prefix_k > 0 && tu.PX && (stop_event == 0xffffffffu || tu.PX == 2)) {
      const double saved = (double)prog->cp.counts.prefix_bytes * (fp64 ? 2.0 : 1.0) * (double)shots;
      if (tu.PX == 2 || (h.prefix_k >= 6 && saved > 64.0 * 1024 * 1024)) {
        void* vec = nullptr;
        NC_TRY(scratch.get(&vec, ((size_t)1 << h.prefix_k) * (fp64 ? 16 : 8)));
        uint32_t nl = 0;
        NC_TRY(launch_prefix(reinterpret_cast<const Op*>(prog->cp.blob.data() + h.off_ops), h.prefix_end, fp64, vec,
                             n_sm, stream, &nl));
        L.init_vec = vec;
        // the executor runs the fused list when there is one, except at a debug stop
        L.start_op = h.n_fops && stop_event == 0xffffffffu ? h.f_start : h.prefix_end;
        L.start_k = h.prefix_k;
        if (tm) {
          tm->launches += nl;
          tm->path |= 1u;
        }
      }
    }
    if (tm) NC_TRY(tm->begin(stream));
    NC_TRY(launch_batched(L, fp64, tu.W, bk, (uint32_t)grid, tu.T, smem, stream));
    if (tm) {
      NC_TRY(tm->end(stream));
      tm->launches += 1;
    }
  }
done:
  return st;
}

uint32_t launch_flags(const nc_sample_opts& o);

// Many programs in ONE executor launch (tune "mp=1" on a batch): the
// thread-per-shot layout over a work list of 128-shot items, programs
// ordered by their estimated cost per shot (longest first) so that the
// persistent CTAs finish together. FP32 amplitudes (NC_FP32_BATCHED) or
// FP64 (NC_FP64_PLAIN); no stratified calls, host outputs or debug stops.
// Returns NC_E_UNSUPPORTED when a program does not fit the layout.
nc_status enqueue_multi_flags(const nc_program* const* progs, const std::vector<DevCopy*>& dcs,
                              const uint64_t* shots, const uint64_t* seeds, uint32_t n, const nc_sample_opts& o,
                              uint32_t lflags, const CallOut* cos, unsigned long long* kept_count, uint32_t* err,
                              Scratch& scratch, cudaStream_t stream, Timing* tm) {
  nc_status st = NC_OK;
  const bool fp32 = o.precision == NC_FP32_BATCHED;
  if (!fp32 && o.precision != NC_FP64_PLAIN) return NC_E_UNSUPPORTED;
  if (o.stratified || (o.outputs & NC_OUT_HOST)) return NC_E_UNSUPPORTED;
  std::vector<uint32_t> order;
  std::vector<double> cost(n, 0.0);
  uint32_t kmax = 0;
  for (uint32_t i = 0; i < n; i++) {
    const ProgHeader& h = header(progs[i]);
    const DevProg d = dev_view(h, dcs[i]->blob);
    if (!plain_supported(d) || h.k_max > 20) return NC_E_UNSUPPORTED;
    if (!shots[i]) continue;
    order.push_back(i);
    kmax = std::max(kmax, h.k_max);
    cost[i] = progs[i]->cp.counts.array_bytes + 64.0 * h.n_ops;
  }
  if (order.empty()) return NC_OK;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return cost[a] > cost[b]; });
  std::vector<LaunchParams> Ls(order.size());
  std::vector<uint64_t> items(order.size());
  for (size_t j = 0; j < order.size(); j++) {
    const uint32_t i = order[j];
    const ProgHeader& h = header(progs[i]);
    LaunchParams& L = Ls[j];
    std::memset(&L, 0, sizeof(L));
    L.p = dev_view(h, dcs[i]->blob);
    L.seed = seeds[i];
    L.shot_offset = o.shot_offset;
    L.shots = shots[i];
    L.meas = cos[i].meas;
    L.det = cos[i].det;
    L.obs = cos[i].obs;
    L.kept = cos[i].kept;
    L.expval = cos[i].expval;
    uint32_t lf = lflags;
    if (!cos[i].expval || !h.n_probes) lf &= ~(uint32_t)LF_OUT_EXPVAL;
    L.flags = lf;
    L.row_words32 = 2 * ((shots[i] + 63) / 64);
    L.kept_count = kept_count + (n == 1 ? 0 : i);
    L.err = err;
    L.stop_event = 0xffffffffu;
    items[j] = (L.row_words32 * 32 + 127) / 128;
  }
  int per_sm = 0, n_sm = 0, dev = 0;
  NC_TRY(cudaGetDevice(&dev));
  NC_TRY(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
  NC_TRY(plain_multi_occupancy(fp32, &per_sm));
  if (per_sm < 1) return NC_E_UNSUPPORTED;
  {
    // mg: resident CTAs per SM (fewer vector slots: a working set that stays in L2)
    const char* mg = o.tune ? strstr(o.tune, "mg=") : nullptr;
    unsigned v = 0;
    if (mg && sscanf(mg, "mg=%u", &v) == 1 && v >= 1) per_sm = std::min<int>(per_sm, (int)v);
  }
  {
    uint64_t total_items = 0;
    for (uint64_t v : items) total_items += v;
    uint64_t grid = std::min<uint64_t>((uint64_t)per_sm * n_sm, total_items);
    // one vector slot per thread of the launch, within half the free memory
    const uint64_t per_slot = kmax ? ((uint64_t)1 << kmax) * (fp32 ? 8 : 16) : 0;
    if (per_slot) {
      size_t free_b = 0;
      NC_TRY(free_memory(LF_ASYNC, &free_b));
      grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, free_b / 2 / (per_slot * 128)));
    }
    void *dLs = nullptr, *item0 = nullptr, *next = nullptr, *work = nullptr;
    NC_TRY(scratch.get(&dLs, Ls.size() * sizeof(LaunchParams)));
    NC_TRY(scratch.get(&item0, (Ls.size() + 1) * 8));
    NC_TRY(scratch.get(&next, 8));
    if (per_slot) NC_TRY(scratch.get(&work, per_slot * 128 * grid));
    if (tm) NC_TRY(tm->begin(stream));
    NC_TRY(launch_plain_multi(Ls.data(), (uint32_t)Ls.size(), items.data(), (LaunchParams*)dLs,
                              (unsigned long long*)item0, (unsigned long long*)next, work, (uint32_t)grid, fp32,
                              stream));
    if (tm) {
      NC_TRY(tm->end(stream));
      tm->launches += 1 + (uint32_t)Ls.size();
      tm->path |= 8u;
    }
  }
done:
  return st;
}

nc_status enqueue_multi(const nc_program* const* progs, const std::vector<DevCopy*>& dcs, const uint64_t* shots,
                        const uint64_t* seeds, uint32_t n, const nc_sample_opts& o, const CallOut* cos,
                        unsigned long long* kept_count, uint32_t* err, Scratch& scratch, cudaStream_t stream,
                        Timing* tm) {
  return enqueue_multi_flags(progs, dcs, shots, seeds, n, o, launch_flags(o), cos, kept_count, err, scratch, stream,
                             tm);
}

// Noiseless 64-shot reference launch: raw detector / observable parities.
nc_status ensure_reference(nc_program* p, DevCopy& dc, cudaStream_t stream) {
  if (dc.ref_ready) return dc.ref_status;
  const ProgHeader& h = header(p);
  nc_status st = NC_OK;
  if (h.n_det + h.n_obs == 0) {
    dc.ref_ready = true;
    return NC_OK;
  }
  {
    Scratch scratch(stream);
    void *det = nullptr, *obs = nullptr, *cnt = nullptr, *err = nullptr;
    const uint64_t shots = 64;
    NC_TRY(scratch.get(&det, (size_t)std::max<uint32_t>(h.n_det, 1) * 8));
    NC_TRY(scratch.get(&obs, (size_t)std::max<uint32_t>(h.n_obs, 1) * 8));
    NC_TRY(scratch.get(&cnt, 8));
    NC_TRY(scratch.get(&err, 4));
    NC_TRY(cudaMemsetAsync(cnt, 0, 8, stream));
    // raw parities of 64 noiseless shots: along the reference trajectory
    // (every measurement takes its more likely outcome, 0 on a tie: all 64
    // shots agree), then sampled
    std::vector<uint64_t> hd(h.n_det), ho(h.n_obs), sd(h.n_det), so(h.n_obs);
    for (int pass = 0; pass < 2; pass++) {
      CallOut o{nullptr, (uint32_t*)det, (uint32_t*)obs, nullptr};
      const uint32_t fl = LF_NOISELESS | LF_REFERENCE | LF_OUT_DET | LF_OUT_OBS | (pass == 0 ? LF_ARGMAX : 0u);
      st = enqueue(p, dc, shots, 0, 0, NC_FP64_BATCHED, fl, nullptr, o, (unsigned long long*)cnt, (uint32_t*)err,
                   scratch, stream);
      if (st != NC_OK) goto done;
      uint64_t* dd = pass == 0 ? hd.data() : sd.data();
      uint64_t* oo = pass == 0 ? ho.data() : so.data();
      if (h.n_det) NC_TRY(cudaMemcpyAsync(dd, det, h.n_det * 8, cudaMemcpyDeviceToHost, stream));
      if (h.n_obs) NC_TRY(cudaMemcpyAsync(oo, obs, h.n_obs * 8, cudaMemcpyDeviceToHost, stream));
      NC_TRY(cudaStreamSynchronize(stream));
    }
    // a detector that differs from its reference in more than a quarter of
    // the sampled shots is not deterministic (one that near-deterministic
    // coherent rotations flip now and then is)
    std::vector<uint32_t> rd(h.n_det), ro(h.n_obs);
    for (uint32_t d = 0; d < h.n_det; d++) {
      if (hd[d] != 0 && hd[d] != ~0ull) st = NC_E_INTERNAL;
      rd[d] = (uint32_t)(hd[d] & 1);
      if (__builtin_popcountll(sd[d] ^ hd[d]) > 16 && st == NC_OK) st = NC_E_NONDET_DETECTOR;
    }
    for (uint32_t d = 0; d < h.n_obs; d++) {
      if (ho[d] != 0 && ho[d] != ~0ull) st = NC_E_INTERNAL;
      ro[d] = (uint32_t)(ho[d] & 1);
      if (__builtin_popcountll(so[d] ^ ho[d]) > 16 && st == NC_OK) st = NC_E_NONDET_DETECTOR;
    }
    if (st == NC_E_INTERNAL) goto done;
    if (h.n_det) NC_TRY(cudaMemcpy(dc.blob + h.off_det_ref, rd.data(), h.n_det * 4, cudaMemcpyHostToDevice));
    if (h.n_obs) NC_TRY(cudaMemcpy(dc.blob + h.off_obs_ref, ro.data(), h.n_obs * 4, cudaMemcpyHostToDevice));
    NC_TRY(launch_patch_ref(reinterpret_cast<Op*>(dc.blob + h.off_ops), h.n_ops,
                            reinterpret_cast<const uint32_t*>(dc.blob + h.off_det_ref),
                            reinterpret_cast<const uint32_t*>(dc.blob + h.off_obs_ref), stream));
    NC_TRY(cudaStreamSynchronize(stream));
  }
done:
  if (st == NC_OK || st == NC_E_NONDET_DETECTOR) {
    dc.ref_ready = true;
    dc.ref_status = st;
  }
  return st;
}

nc_status prepare(const nc_program* cprog, DevCopy** dc_out, cudaStream_t stream) {
  nc_program* prog = const_cast<nc_program*>(cprog);
  std::lock_guard<std::mutex> lock(prog->mu);
  DevCopy* dc = nullptr;
  nc_status st = device_copy(prog, &dc);
  if (st != NC_OK) return st;
  st = ensure_reference(prog, *dc, stream);
  if (st != NC_OK) return st;
  *dc_out = dc;
  return NC_OK;
}

// Host stratified tables covering strata 0..k: built on first use, grown on
// demand (rows of smaller strata do not change). Caller holds p->mu.
nc_status host_strata(nc_program* p, uint32_t k) {
  if (p->strata.valid.size() >= (size_t)k + 1) return NC_OK;
  const ProgHeader& h = header(p);
  try {
    build_strata(reinterpret_cast<const double*>(p->cp.blob.data() + h.off_site_p), h.n_sites,
                 std::max<uint32_t>(k, 16), p->strata);
  } catch (std::bad_alloc&) {
    return NC_E_OOM;
  }
  return NC_OK;
}

// The tables for stratum k and, with dc, their copy on dc's device.
// NC_E_ARG for a stratum that cannot be sampled.
nc_status strata_tables(nc_program* p, uint32_t k, DevCopy* dc) {
  std::lock_guard<std::mutex> lock(p->mu);
  if (k > kMaxStratum) return NC_E_ARG;
  nc_status st = host_strata(p, k);
  if (st != NC_OK) return st;
  if (!p->strata.valid[k]) return NC_E_ARG;
  if (dc && k > 0 && dc->sg_rows < k) {
    const StrataTables& t = p->strata;
    const size_t bg = t.g.size() * sizeof(double), br = t.rows.size() * sizeof(StrataRow),
                 bu = t.guide.size() * 4;
    const size_t og = 0, orow = (bg + 15) & ~(size_t)15, ogd = (orow + br + 15) & ~(size_t)15;
    static_assert(sizeof(StrataRow) == 3 * sizeof(unsigned long long), "row = 3 u64 on the device");
    uint8_t* base = nullptr;
    cudaError_t e = cudaMalloc(&base, ogd + bu);
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemcpy(base + og, t.g.data(), bg, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + orow, t.rows.data(), br, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(base + ogd, t.guide.data(), bu, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(base);
      return cuda_status(e);
    }
    if (dc->sg) cudaFree(dc->sg);  // synchronises the device: no launch still reads it
    dc->sg = reinterpret_cast<double*>(base + og);
    dc->sgr = reinterpret_cast<const unsigned long long*>(base + orow);
    dc->sgg = reinterpret_cast<const uint32_t*>(base + ogd);
    dc->sg_rows = t.k_max;
  }
  return NC_OK;
}

uint32_t launch_flags(const nc_sample_opts& o) {
  uint32_t f = 0;
  if (o.outputs & NC_OUT_MEAS) f |= LF_OUT_MEAS;
  if (o.outputs & NC_OUT_DET) f |= LF_OUT_DET;
  if (o.outputs & NC_OUT_OBS) f |= LF_OUT_OBS;
  if (o.outputs & NC_OUT_KEPT) f |= LF_OUT_KEPT;
  if (o.postselect == NC_PS_ALL_DETECTORS) f |= LF_POSTSELECT;
  if (o.noiseless) f |= LF_NOISELESS;
  if (o.outputs & NC_OUT_EXPVAL) f |= LF_OUT_EXPVAL;
  return f;
}

nc_sample_opts default_opts() {
  nc_sample_opts o;
  std::memset(&o, 0, sizeof(o));
  o.precision = NC_FP32_BATCHED;
  o.outputs = NC_OUT_MEAS | NC_OUT_DET | NC_OUT_OBS | NC_OUT_KEPT;
  o.postselect = NC_PS_NONE;
  return o;
}

// Host outputs the device cannot address: the call's shots run in chunks
// (global shot offsets advance with the chunk, so the records are those of
// one call), each into one of two device staging buffers, and each finished
// chunk's record columns are copied to the caller's rows on a side stream
// while the next chunk runs. The caller's stream waits for the last copy.
nc_status sample_staged(const nc_program* prog, DevCopy& dc, uint64_t shots, uint64_t seed, const nc_sample_opts& o,
                        uint32_t lflags, const char* tune, CallOut host, unsigned long long* kept_count, uint32_t* err,
                        Scratch& scratch, cudaStream_t stream, Timing* tm, uint32_t stratum) {
  nc_status st = NC_OK;
  const ProgHeader& h = header(prog);
  const uint64_t wpr = (shots + 63) / 64;
  const uint32_t rows[4] = {host.meas ? h.n_meas : 0u, host.det ? h.n_det : 0u, host.obs ? h.n_obs : 0u,
                            host.kept ? 1u : 0u};
  const uint32_t n_rows = rows[0] + rows[1] + rows[2] + rows[3];
  const uint32_t n_probes = host.expval ? h.n_probes : 0u;
  // chunk: at most 2^24 shots and 1 GiB of staging per buffer, 128-aligned
  const uint64_t per_shot = (uint64_t)n_rows / 8 + 1 + (uint64_t)n_probes * 8;
  uint64_t chunk = std::min<uint64_t>(1ull << 24, std::max<uint64_t>(128, (1ull << 30) / per_shot)) & ~127ull;
  {
    const char* hc = tune ? strstr(tune, "hc=") : nullptr;  // chunk override (tests)
    unsigned long long v = 0;
    if (hc && sscanf(hc, "hc=%llu", &v) == 1 && v >= 128) chunk = (uint64_t)v & ~127ull;
  }
  chunk = std::min<uint64_t>(chunk, (shots + 127) & ~127ull);
  const uint64_t cw = (chunk + 63) / 64;  // words per staged row
  const size_t rec_b = (size_t)n_rows * cw * 8, ev_b = (size_t)n_probes * chunk * 8;
  void* buf[2] = {nullptr, nullptr};
  SideStream side;
  Events ev;  // [0] start, [1..2] chunk computed into buffer b, [3..4] buffer b copied out
  NC_TRY(scratch.get(&buf[0], rec_b + ev_b));
  NC_TRY(scratch.get(&buf[1], rec_b + ev_b));
  {
    int dev = 0;
    NC_TRY(cudaGetDevice(&dev));
    NC_TRY(side.acquire(dev));
  }
  NC_TRY(ev.make(5));
  NC_TRY(cudaEventRecord(ev.ev[0], stream));
  NC_TRY(cudaStreamWaitEvent(side.s, ev.ev[0], 0));
  for (uint64_t c0 = 0, ci = 0; c0 < shots; c0 += chunk, ci++) {
    const uint64_t cs = std::min(chunk, shots - c0), csw = (cs + 63) / 64;
    const uint32_t b = (uint32_t)(ci & 1);
    uint8_t* base = (uint8_t*)buf[b];
    if (ci >= 2) NC_TRY(cudaStreamWaitEvent(stream, ev.ev[3 + b], 0));  // buffer b drained
    CallOut d{nullptr, nullptr, nullptr, nullptr, nullptr};
    uint32_t* r = (uint32_t*)base;
    const size_t rstride = csw * 2;  // u32 words per staged row of this chunk
    if (rows[0]) { d.meas = r; r += rows[0] * rstride; }
    if (rows[1]) { d.det = r; r += rows[1] * rstride; }
    if (rows[2]) { d.obs = r; r += rows[2] * rstride; }
    if (rows[3]) { d.kept = r; r += rows[3] * rstride; }
    if (n_probes) d.expval = (double*)(base + rec_b);
    st = enqueue(prog, dc, cs, seed, o.shot_offset + c0, o.precision, lflags, tune, d, kept_count, err, scratch, stream,
                 0xffffffffu, 0, nullptr, nullptr, nullptr, tm, stratum);
    if (st != NC_OK) goto done;
    NC_TRY(cudaEventRecord(ev.ev[1 + b], stream));
    NC_TRY(cudaStreamWaitEvent(side.s, ev.ev[1 + b], 0));
    {
      const uint32_t* src = (const uint32_t*)base;
      uint32_t* dst[4] = {host.meas, host.det, host.obs, host.kept};
      for (int j = 0; j < 4; j++) {
        if (!rows[j]) continue;
        NC_TRY(cudaMemcpy2DAsync((uint64_t*)dst[j] + c0 / 64, wpr * 8, src, csw * 8, csw * 8, rows[j],
                                 cudaMemcpyDeviceToHost, side.s));
        src += rows[j] * rstride;
      }
      if (n_probes)
        NC_TRY(cudaMemcpy2DAsync(host.expval + c0, shots * 8, base + rec_b, cs * 8, cs * 8, n_probes,
                                 cudaMemcpyDeviceToHost, side.s));
    }
    NC_TRY(cudaEventRecord(ev.ev[3 + b], side.s));
  }
  // the caller's stream (and with it the scratch release) waits for every copy
  NC_TRY(cudaEventRecord(ev.ev[0], side.s));
  NC_TRY(cudaStreamWaitEvent(stream, ev.ev[0], 0));
  if (tm) tm->path |= 4u;
done:
  return st;
}

nc_status sample_many(const nc_program* const* progs, const uint64_t* shots, const uint64_t* seeds, uint32_t n,
                      const nc_sample_opts* opts_in, nc_records* outs, cudaStream_t stream) {
  if (!progs || !shots || !seeds || !outs) return NC_E_ARG;
  nc_sample_opts o = opts_in ? *opts_in : default_opts();
  if (o.precision != NC_FP32_BATCHED && o.precision != NC_FP64_PLAIN && o.precision != NC_FP64_BATCHED)
    return NC_E_ARG;
  if (o.shot_offset % 128) return NC_E_ARG;
  if (o.postselect != NC_PS_NONE && o.postselect != NC_PS_ALL_DETECTORS) return NC_E_ARG;
  if (o.stratified > 1 || (o.stratified && o.stratum > kMaxStratum)) return NC_E_ARG;
  const uint32_t stratum = o.stratified ? o.stratum : kNoStratum;
  const bool host = (o.outputs & NC_OUT_HOST) != 0;
  nc_status st = NC_OK;
  std::vector<DevCopy*> dcs(n, nullptr);
  for (uint32_t i = 0; i < n; i++) {
    if (!progs[i]) return NC_E_ARG;
    const ProgHeader& h = header(progs[i]);
    uint64_t wpr = (shots[i] + 63) / 64;
    if (outs[i].words_per_record != wpr) return NC_E_ARG;
    if ((o.outputs & NC_OUT_MEAS) && h.n_meas && !outs[i].meas) return NC_E_ARG;
    if ((o.outputs & NC_OUT_DET) && h.n_det && !outs[i].det) return NC_E_ARG;
    if ((o.outputs & NC_OUT_OBS) && h.n_obs && !outs[i].obs) return NC_E_ARG;
    if ((o.outputs & NC_OUT_KEPT) && !outs[i].kept) return NC_E_ARG;
    if ((o.outputs & NC_OUT_EXPVAL) && h.n_probes && !outs[i].expval) return NC_E_ARG;
    if (h.n_sites >= (1u << 28) - 1) return NC_E_UNSUPPORTED;
    st = prepare(progs[i], &dcs[i], stream);
    if (st != NC_OK) return st;
    if (o.stratified) {
      st = strata_tables(const_cast<nc_program*>(progs[i]), o.stratum, dcs[i]);
      if (st != NC_OK) return st;
    }
  }
  std::vector<unsigned long long> kept(n, 0);
  float kernel_ms = 0.f;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<Timing> tms(n);
  if (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0);
    return NC_E_CUDA;
  }
  {
    Scratch scratch(stream);
    void* counters = nullptr;
    void* err = nullptr;
    NC_TRY(scratch.get(&counters, 8 * (size_t)std::max<uint32_t>(n, 1)));
    NC_TRY(scratch.get(&err, 4));
    NC_TRY(cudaMemsetAsync(counters, 0, 8 * (size_t)std::max<uint32_t>(n, 1), stream));
    NC_TRY(cudaMemsetAsync(err, 0, 4, stream));
    NC_TRY(cudaEventRecord(ev0, stream));
    // every program in one executor launch
    const bool mp = o.tune && strstr(o.tune, "mp=1") && !host && !o.stratified;
    if (mp) {
      std::vector<CallOut> cos(n);
      for (uint32_t i = 0; i < n; i++)
        cos[i] = CallOut{(uint32_t*)outs[i].meas, (uint32_t*)outs[i].det, (uint32_t*)outs[i].obs,
                         (uint32_t*)outs[i].kept, (o.outputs & NC_OUT_EXPVAL) ? outs[i].expval : nullptr};
      st = enqueue_multi(progs, dcs, shots, seeds, n, o, cos.data(), (unsigned long long*)counters, (uint32_t*)err,
                         scratch, stream, &tms[0]);
      if (st != NC_OK) goto done;
      NC_TRY(cudaEventRecord(ev1, stream));
    }
    for (uint32_t i = 0; i < n && !mp; i++) {
      if (shots[i] == 0) continue;
      const ProgHeader& h = header(progs[i]);
      CallOut co{(uint32_t*)outs[i].meas, (uint32_t*)outs[i].det, (uint32_t*)outs[i].obs,
                 (uint32_t*)outs[i].kept, (o.outputs & NC_OUT_EXPVAL) ? outs[i].expval : nullptr};
      const char* tn = o.tune ? o.tune : (dcs[i]->tuned.empty() ? nullptr : dcs[i]->tuned.c_str());
      const uint32_t lf = launch_flags(o);
      if (host) {
        // host outputs: written by the kernels themselves when the device can
        // address the caller's (pinned) buffers, else staged in device
        // memory chunk by chunk with the copies overlapped
        // (the executors' record-flip atomics need native host atomics)
        int native_atomics = 0, cur_dev = 0;
        NC_TRY(cudaGetDevice(&cur_dev));
        NC_TRY(cudaDeviceGetAttribute(&native_atomics, cudaDevAttrHostNativeAtomicSupported, cur_dev));
        bool direct = native_atomics && !(tn && strstr(tn, "hd=0"));
        CallOut dv = co;
        auto dev_ptr = [&](void* hp, void** dp) {
          if (!hp) return;
          cudaPointerAttributes a;
          if (cudaPointerGetAttributes(&a, hp) != cudaSuccess || a.type != cudaMemoryTypeHost || !a.devicePointer) {
            cudaGetLastError();
            direct = false;
            return;
          }
          *dp = a.devicePointer;
        };
        if (direct) {
          dev_ptr(co.meas, (void**)&dv.meas);
          dev_ptr(co.det, (void**)&dv.det);
          dev_ptr(co.obs, (void**)&dv.obs);
          dev_ptr(co.kept, (void**)&dv.kept);
          dev_ptr(co.expval, (void**)&dv.expval);
        }
        if (direct) {
          st = enqueue(progs[i], *dcs[i], shots[i], seeds[i], o.shot_offset, o.precision, lf, tn, dv,
                       (unsigned long long*)counters + i, (uint32_t*)err, scratch, stream, 0xffffffffu, 0, nullptr,
                       nullptr, nullptr, &tms[i], stratum);
          if (st != NC_OK) goto done;
          tms[i].path |= 2u;
        } else {
          st = sample_staged(progs[i], *dcs[i], shots[i], seeds[i], o, lf, tn, co, (unsigned long long*)counters + i,
                             (uint32_t*)err, scratch, stream, &tms[i], stratum);
          if (st != NC_OK) goto done;
        }
      } else {
        st = enqueue(progs[i], *dcs[i], shots[i], seeds[i], o.shot_offset, o.precision, lf, tn, co,
                     (unsigned long long*)counters + i, (uint32_t*)err, scratch, stream, 0xffffffffu, 0, nullptr,
                     nullptr, nullptr, &tms[i], stratum);
        if (st != NC_OK) goto done;
      }
      if (i + 1 == n) NC_TRY(cudaEventRecord(ev1, stream));
    }
    NC_TRY(cudaMemcpyAsync(kept.data(), counters, 8 * (size_t)n, cudaMemcpyDeviceToHost, stream));
    uint32_t herr = 0;
    NC_TRY(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, stream));
    NC_TRY(cudaStreamSynchronize(stream));
    if (herr) st = NC_E_INTERNAL;
    if ((shots[n - 1] != 0 || mp) && cudaEventElapsedTime(&kernel_ms, ev0, ev1) != cudaSuccess) kernel_ms = 0.f;
    if (mp)
      for (uint32_t i = 1; i < n; i++) tms[i].path = tms[0].path;
  }
  NC_TRY(cudaStreamSynchronize(stream));
  for (uint32_t i = 0; i < n; i++) {
    outs[i].shots_run = shots[i];
    outs[i].shots_kept = kept[i];
    outs[i].kernel_ms = kernel_ms;
    outs[i].exec_ms = shots[i] ? (tms[i].path & 8u ? tms[0].ms() : tms[i].ms()) : 0.0;
    outs[i].launches = tms[i].launches;
    outs[i].path = tms[i].path;
  }
done:
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  return st;
}

}  // namespace

extern "C" {

nc_status nc_compile(const char* text, size_t len, nc_program** out, char* err, size_t err_len) {
  return nc_compile_ex(text, len, 0u, out, err, err_len);
}

nc_status nc_compile_ex(const char* text, size_t len, uint32_t flags, nc_program** out, char* err,
                        size_t err_len) {
  if (out) *out = nullptr;
  if (!text || !out || (flags & ~(uint32_t)NC_COMPILE_FLAGS_ALL)) return NC_E_ARG;
  nc_program* p = new (std::nothrow) nc_program();
  if (!p) return NC_E_OOM;
  std::string msg;
  int rc = compile_program(std::string(text, len), flags, p->cp, msg);
  if (rc != 0) {
    if (err && err_len) snprintf(err, err_len, "%s", msg.c_str());
    delete p;
    return (nc_status)rc;
  }
  fill_info(p);
  *out = p;
  return NC_OK;
}

nc_status nc_program_info(const nc_program* prog, nc_info* info) {
  if (!prog || !info) return NC_E_ARG;
  *info = prog->info;
  return NC_OK;
}

nc_status nc_program_serialize(const nc_program* prog, void* buf, size_t* len) {
  if (!prog || !len) return NC_E_ARG;
  const size_t need = prog->cp.blob.size() + sizeof(nc_info_counts);
  if (!buf) {
    *len = need;
    return NC_OK;
  }
  if (*len < need) return NC_E_ARG;
  std::memcpy(buf, prog->cp.blob.data(), prog->cp.blob.size());
  std::memcpy((uint8_t*)buf + prog->cp.blob.size(), &prog->cp.counts, sizeof(nc_info_counts));
  *len = need;
  return NC_OK;
}

nc_status nc_program_deserialize(const void* buf, size_t len, nc_program** out) {
  if (out) *out = nullptr;
  if (!buf || !out || len < sizeof(ProgHeader) + sizeof(nc_info_counts)) return NC_E_ARG;
  ProgHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kMagic || h.version != kVersion || h.total_bytes + sizeof(nc_info_counts) != len) return NC_E_ARG;
  uint64_t offs[] = {h.off_ops, h.off_masks, h.off_q, h.off_seg_start, h.off_seg_end, h.off_site_info,
                     h.off_site_eff, h.off_slot_list, h.off_det_ref, h.off_obs_ref,
                     h.off_site_opt, h.off_opt_tab, h.off_plist, h.off_orec, h.off_site_blk,
                     h.off_aff_const, h.off_aff_rowev_off, h.off_aff_rowev, h.off_aff_rand_ev,
                     h.off_aff_col_off, h.off_aff_col, h.off_aff_frec, h.off_aff_parent, h.off_aff_chain_off,
                     h.off_aff_chain, h.off_srch, h.off_guide, h.off_fops, h.off_fterm, h.off_fperm,
                     h.off_site_p};
  for (uint64_t o : offs)
    if (o > h.total_bytes || (o & 15)) return NC_E_ARG;
  if (h.off_ops + (uint64_t)h.n_ops * sizeof(Op) > h.total_bytes || h.k_max > kMaxK || h.n_qubits > kMaxQubits)
    return NC_E_ARG;
  nc_program* p = new (std::nothrow) nc_program();
  if (!p) return NC_E_OOM;
  p->cp.blob.assign((const uint8_t*)buf, (const uint8_t*)buf + h.total_bytes);
  std::memcpy(&p->cp.counts, (const uint8_t*)buf + h.total_bytes, sizeof(nc_info_counts));
  // reference parities are recomputed on first use
  std::memset(p->cp.blob.data() + h.off_det_ref, 0, (size_t)h.n_det * 4);
  std::memset(p->cp.blob.data() + h.off_obs_ref, 0, (size_t)h.n_obs * 4);
  fill_info(p);
  *out = p;
  return NC_OK;
}

nc_status nc_sample(const nc_program* prog, uint64_t shots, uint64_t seed, const nc_sample_opts* opts,
                    nc_records* out, void* cuda_stream) {
  if (!prog || !out) return NC_E_ARG;
  return sample_many(&prog, &shots, &seed, 1, opts, out, (cudaStream_t)cuda_stream);
}

nc_status nc_sample_batch(const nc_program* const* progs, const uint64_t* shots, const uint64_t* seeds, uint32_t n,
                          const nc_sample_opts* opts, nc_records* outs, void* cuda_stream) {
  if (n == 0) return NC_OK;
  return sample_many(progs, shots, seeds, n, opts, outs, (cudaStream_t)cuda_stream);
}

nc_status nc_program_prepare(const nc_program* prog, void* cuda_stream) {
  if (!prog) return NC_E_ARG;
  DevCopy* dc = nullptr;
  return prepare(prog, &dc, (cudaStream_t)cuda_stream);
}

nc_status nc_stratum_weights(const nc_program* prog, uint32_t k_max, double* weights, uint8_t* valid) {
  if (!prog || !weights || k_max > kMaxStratum) return NC_E_ARG;
  nc_program* p = const_cast<nc_program*>(prog);
  std::lock_guard<std::mutex> lock(p->mu);
  nc_status st = host_strata(p, k_max);
  if (st != NC_OK) return st;
  for (uint32_t k = 0; k <= k_max; k++) {
    weights[k] = p->strata.weight[k];
    if (valid) valid[k] = p->strata.valid[k];
  }
  return NC_OK;
}

nc_status nc_strata_prepare(const nc_program* prog, uint32_t k_max, void* cuda_stream) {
  if (!prog || k_max > kMaxStratum) return NC_E_ARG;
  DevCopy* dc = nullptr;
  nc_status st = prepare(prog, &dc, (cudaStream_t)cuda_stream);
  if (st != NC_OK) return st;
  nc_program* p = const_cast<nc_program*>(prog);
  uint32_t top = 0;  // largest stratum <= k_max that can be sampled
  {
    std::lock_guard<std::mutex> lock(p->mu);
    st = host_strata(p, k_max);
    if (st != NC_OK) return st;
    for (uint32_t k = 1; k <= k_max; k++)
      if (p->strata.valid[k]) top = k;
  }
  return top ? strata_tables(p, top, dc) : NC_OK;
}

nc_status nc_sample_batch_async(const nc_program* const* progs, const uint64_t* shots, const uint64_t* seeds,
                                uint32_t n, const nc_sample_opts* opts_in, nc_records* outs,
                                unsigned long long* kept_dev, uint32_t* err_dev, void* cuda_stream) {
  if (n == 0) return NC_OK;
  if (!progs || !shots || !seeds || !outs || !kept_dev || !err_dev) return NC_E_ARG;
  nc_sample_opts o = opts_in ? *opts_in : default_opts();
  if (o.precision != NC_FP32_BATCHED && o.precision != NC_FP64_PLAIN && o.precision != NC_FP64_BATCHED)
    return NC_E_ARG;
  if (o.shot_offset % 128 || (o.outputs & NC_OUT_HOST)) return NC_E_ARG;
  if (o.postselect != NC_PS_NONE && o.postselect != NC_PS_ALL_DETECTORS) return NC_E_ARG;
  if (o.stratified > 1 || (o.stratified && o.stratum > kMaxStratum)) return NC_E_ARG;
  const uint32_t stratum = o.stratified ? o.stratum : kNoStratum;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return NC_E_CUDA;
  std::vector<DevCopy*> dcs(n, nullptr);
  for (uint32_t i = 0; i < n; i++) {
    if (!progs[i]) return NC_E_ARG;
    const ProgHeader& h = header(progs[i]);
    if (outs[i].words_per_record != (shots[i] + 63) / 64) return NC_E_ARG;
    if ((o.outputs & NC_OUT_MEAS) && h.n_meas && !outs[i].meas) return NC_E_ARG;
    if ((o.outputs & NC_OUT_DET) && h.n_det && !outs[i].det) return NC_E_ARG;
    if ((o.outputs & NC_OUT_OBS) && h.n_obs && !outs[i].obs) return NC_E_ARG;
    if ((o.outputs & NC_OUT_KEPT) && !outs[i].kept) return NC_E_ARG;
    if ((o.outputs & NC_OUT_EXPVAL) && h.n_probes && !outs[i].expval) return NC_E_ARG;
    nc_program* p = const_cast<nc_program*>(progs[i]);
    std::lock_guard<std::mutex> lock(p->mu);
    for (auto& c : p->devs)
      if (c.device == dev && c.ref_ready) dcs[i] = &c;
    if (!dcs[i]) return NC_E_ARG;  // not prepared on this device
    if (dcs[i]->ref_status != NC_OK) return dcs[i]->ref_status;
    // stratified: tables uploaded by nc_strata_prepare, stratum checked
    if (o.stratified && o.stratum > 0 &&
        (dcs[i]->sg_rows < o.stratum || p->strata.valid.size() <= o.stratum || !p->strata.valid[o.stratum]))
      return NC_E_ARG;
  }
  // The programs run on up to kBranches side streams forked from the
  // caller's stream and joined back into it (program i on branch i mod the
  // branch count, in order within a branch), so that a captured graph holds
  // independent branches and small programs run beside large ones.
  constexpr uint32_t kBranches = 16;
  std::vector<uint32_t> live;
  for (uint32_t i = 0; i < n; i++) {
    outs[i].shots_run = shots[i];
    outs[i].shots_kept = 0;
    outs[i].kernel_ms = outs[i].exec_ms = 0.0;
    outs[i].launches = 0;
    outs[i].path = 0;
    if (shots[i]) live.push_back(i);
  }
  if (live.empty()) return NC_OK;
  nc_status st = NC_OK;
  if (o.tune && strstr(o.tune, "mp=1") && !o.stratified) {
    // every program in one executor launch on the caller's stream
    std::vector<CallOut> cos(n);
    for (uint32_t i = 0; i < n; i++)
      cos[i] = CallOut{(uint32_t*)outs[i].meas, (uint32_t*)outs[i].det, (uint32_t*)outs[i].obs,
                       (uint32_t*)outs[i].kept, (o.outputs & NC_OUT_EXPVAL) ? outs[i].expval : nullptr};
    Scratch scratch(stream);
    return enqueue_multi(progs, dcs, shots, seeds, n, o, cos.data(), kept_dev, err_dev, scratch, stream, nullptr);
  }
  const uint32_t nb = std::min<uint32_t>(kBranches, (uint32_t)live.size());
  std::vector<SideStream> side(nb);
  Events ev;
  NC_TRY(ev.make(1 + nb));
  NC_TRY(cudaEventRecord(ev.ev[0], stream));
  for (uint32_t b = 0; b < nb; b++) {
    NC_TRY(side[b].acquire(dev));
    NC_TRY(cudaStreamWaitEvent(side[b].s, ev.ev[0], 0));
  }
  for (uint32_t b = 0; b < nb; b++) {
    {
      Scratch scratch(side[b].s);  // released on its branch, before the join
      for (size_t j = b; j < live.size() && st == NC_OK; j += nb) {
        const uint32_t i = live[j];
        CallOut co{(uint32_t*)outs[i].meas, (uint32_t*)outs[i].det, (uint32_t*)outs[i].obs,
                   (uint32_t*)outs[i].kept, (o.outputs & NC_OUT_EXPVAL) ? outs[i].expval : nullptr};
        const char* tn = o.tune ? o.tune : (dcs[i]->tuned.empty() ? nullptr : dcs[i]->tuned.c_str());
        st = enqueue(progs[i], *dcs[i], shots[i], seeds[i], o.shot_offset, o.precision,
                     launch_flags(o) | LF_ASYNC, tn, co, kept_dev + i, err_dev, scratch, side[b].s, 0xffffffffu, 0,
                     nullptr, nullptr, nullptr, nullptr, stratum);
      }
    }
    // every branch is joined, also after an error, so that a capture can end
    cudaError_t e1 = cudaEventRecord(ev.ev[1 + b], side[b].s);
    cudaError_t e2 = e1 == cudaSuccess ? cudaStreamWaitEvent(stream, ev.ev[1 + b], 0) : e1;
    if (e2 != cudaSuccess && st == NC_OK) st = cuda_status(e2);
  }
done:
  return st;
}

nc_status nc_autotune(nc_program* prog, uint64_t shots, const nc_sample_opts* opts_in, void* cuda_stream,
                      char* best, size_t best_len) {
  if (!prog || shots == 0) return NC_E_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  DevCopy* dc = nullptr;
  nc_status st = prepare(prog, &dc, stream);
  if (st != NC_OK) return st;
  nc_sample_opts o = opts_in ? *opts_in : default_opts();
  o.outputs &= ~(uint32_t)NC_OUT_HOST;
  const ProgHeader& h = header(prog);
  const uint64_t n = std::min<uint64_t>(std::max<uint64_t>(shots, 128), 4ull << 20);
  const uint64_t wpr = (n + 63) / 64;
  // candidate launch shapes
  std::vector<std::string> cand;
  if (h.k_max == 0 && h.aff_ok) {
    // (the item kernel's residency, aq, stays at its default of 4: 2 and 3
    // were slower in longer timings than the autotuner's short ones resolve)
    for (const char* c : {"aw=32", "aw=16", "aw=8", "aw=32,ai=0", "a=0"}) cand.push_back(c);
  } else {
    const uint32_t gs[] = {1, 2, 4, 8, 16, 32, 64, 128};
    const uint32_t ts[] = {256, 512, 1024};
    const DevProg d = dev_view(h, dc->blob);
    for (uint32_t g : gs)
      for (uint32_t t : ts) {
        if (batched_smem_bytes(d, g, 1, false) > 220 * 1024 || g > 1024u * 1024u / (1u << std::min(h.k_max, 20u)))
          continue;
        cand.push_back("g=" + std::to_string(g) + ",t=" + std::to_string(t));
      }
    // the warp-per-shot layout (vectors in shared memory, frame in registers)
    if (warp_supported(d) && h.k_max <= 13)
      for (const char* c : {"lw=1", "lw=1,wn=4", "lw=1,wn=2"}) cand.push_back(c);
    // the thread-per-shot layout (vectors in global memory, no barriers), and
    // its persistent form with one vector slot per resident thread (fewer
    // resident CTAs: the vectors stay in L2)
    if (plain_supported(d) && h.k_max <= 12)
      for (const char* c : {"lp=1", "mp=1", "mp=1,mg=4", "mp=1,mg=2", "mp=1,mg=1"}) cand.push_back(c);
  }
  Scratch scratch(stream);
  void *meas = nullptr, *det = nullptr, *obs = nullptr, *kept = nullptr;
  cudaError_t e = cudaSuccess;
  if (h.n_meas) e = scratch.get(&meas, (size_t)h.n_meas * wpr * 8);
  if (e == cudaSuccess && h.n_det) e = scratch.get(&det, (size_t)h.n_det * wpr * 8);
  if (e == cudaSuccess && h.n_obs) e = scratch.get(&obs, (size_t)h.n_obs * wpr * 8);
  if (e == cudaSuccess) e = scratch.get(&kept, wpr * 8);
  if (e != cudaSuccess) return cuda_status(e);
  nc_records r;
  std::memset(&r, 0, sizeof(r));
  r.meas = (uint64_t*)meas;
  r.det = (uint64_t*)det;
  r.obs = (uint64_t*)obs;
  r.kept = (uint64_t*)kept;
  r.words_per_record = wpr;
  std::string win;
  double win_ms = 1e30;
  const uint64_t seed = 1;
  for (const auto& c : cand) {
    nc_sample_opts oc = o;
    oc.tune = c.c_str();
    const nc_program* cp = prog;
    if (sample_many(&cp, &n, &seed, 1, &oc, &r, stream) != NC_OK) continue;  // warm-up; skips unusable shapes
    double ms = 1e30;
    for (int rep = 0; rep < 2; rep++) {
      if (sample_many(&cp, &n, &seed, 1, &oc, &r, stream) != NC_OK) break;
      ms = std::min(ms, r.kernel_ms);
    }
    if (ms < win_ms) {
      win_ms = ms;
      win = c;
    }
  }
  if (win.empty()) return NC_E_UNSUPPORTED;
  {
    std::lock_guard<std::mutex> lock(prog->mu);
    dc->tuned = win;
  }
  if (best && best_len) snprintf(best, best_len, "%s", win.c_str());
  return NC_OK;
}

void nc_program_free(nc_program* prog) {
  if (!prog) return;
  int cur = 0;
  bool have = cudaGetDevice(&cur) == cudaSuccess;
  for (auto& c : prog->devs) {
    if (c.blob || c.sg) {
      cudaSetDevice(c.device);
      if (c.blob) cudaFree(c.blob);
      if (c.sg) cudaFree(c.sg);
    }
  }
  if (have) cudaSetDevice(cur);
  delete prog;
}

const char* nc_status_str(nc_status st) {
  switch (st) {
    case NC_OK: return "ok";
    case NC_E_PARSE: return "parse error";
    case NC_E_UNSUPPORTED: return "unsupported";
    case NC_E_KMAX: return "active dimension above the limit";
    case NC_E_NONDET_DETECTOR: return "non-deterministic detector or observable";
    case NC_E_ARG: return "invalid argument";
    case NC_E_OOM: return "out of memory";
    case NC_E_CUDA: return "CUDA error";
    case NC_E_TIMEOUT: return "device wait timed out";
    case NC_E_INTERNAL: return "internal error";
  }
  return "unknown status";
}

nc_status nc_debug_dump(const nc_program* prog, uint64_t seed, uint64_t shot, uint32_t event, int precision,
                        uint32_t* frame_xz, double* amps, uint32_t* k, void* cuda_stream) {
  if (!prog || !frame_xz || !amps || !k) return NC_E_ARG;
  if (precision != NC_FP32_BATCHED && precision != NC_FP64_PLAIN && precision != NC_FP64_BATCHED)
    return NC_E_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  DevCopy* dc = nullptr;
  nc_status st = prepare(prog, &dc, stream);
  if (st != NC_OK) return st;
  const ProgHeader& h = header(prog);
  const uint64_t base = shot & ~127ull;
  const size_t n_amp = (size_t)1 << h.k_max;
  {
    Scratch scratch(stream);
    void *d_amps = nullptr, *d_frame = nullptr, *d_k = nullptr, *cnt = nullptr, *err = nullptr;
    NC_TRY(scratch.get(&d_amps, n_amp * 2 * sizeof(double)));
    NC_TRY(scratch.get(&d_frame, (size_t)2 * h.nw * 4));
    NC_TRY(scratch.get(&d_k, 4));
    NC_TRY(scratch.get(&cnt, 8));
    NC_TRY(scratch.get(&err, 4));
    NC_TRY(cudaMemsetAsync(d_amps, 0, n_amp * 2 * sizeof(double), stream));
    NC_TRY(cudaMemsetAsync(d_frame, 0, (size_t)2 * h.nw * 4, stream));
    NC_TRY(cudaMemsetAsync(d_k, 0xff, 4, stream));
    NC_TRY(cudaMemsetAsync(cnt, 0, 8, stream));
    {
      CallOut o{nullptr, nullptr, nullptr, nullptr};
      // vectors of 2^15 amplitudes and more live in HBM: their noiseless
      // prefix is computed once (as a sampling call does), not per shot
      char tune[32];
      snprintf(tune, sizeof(tune), "g=4,t=%u,px=%u", h.k_max > 10 ? 512u : 128u, h.prefix_k >= 15 ? 2u : 0u);
      st = enqueue(prog, *dc, 128, seed, base, precision, 0, tune, o, (unsigned long long*)cnt, (uint32_t*)err,
                   scratch, stream, event, shot - base, (double*)d_amps, (uint32_t*)d_frame, (uint32_t*)d_k);
      if (st != NC_OK) goto done;
    }
    NC_TRY(cudaMemcpyAsync(amps, d_amps, n_amp * 2 * sizeof(double), cudaMemcpyDeviceToHost, stream));
    NC_TRY(cudaMemcpyAsync(frame_xz, d_frame, (size_t)2 * h.nw * 4, cudaMemcpyDeviceToHost, stream));
    NC_TRY(cudaMemcpyAsync(k, d_k, 4, cudaMemcpyDeviceToHost, stream));
    NC_TRY(cudaStreamSynchronize(stream));
  }
  NC_TRY(cudaStreamSynchronize(stream));
done:
  return st;
}

uint32_t nc_abi_version(void) { return (kVersion << 16) | 5u; }

}  // extern "C"

// Host blob of a program, for the allocation-free entry point (noalloc.cu).
namespace nc {
const std::vector<uint8_t>& program_blob(const nc_program* p) { return p->cp.blob; }
}  // namespace nc

extern "C" {

}  // extern "C"
