/*
 * nc.h — C ABI of the GB300 near-Clifford shot sampler.
 *
 * The library implements the online "sample-many" phase of frame-factored
 * near-Clifford simulation (Clifft, arXiv 2604.27058): a circuit is compiled
 * once on the host (Sec. 3.1: Heisenberg mapping, Pauli localisation,
 * bytecode emission) and then sampled for many independent shots on one GPU
 * (Sec. 3.2: Pauli-frame updates, sampled noise, active state vector).
 *
 * Conventions for every entry point:
 *   - Functions return nc_status; they never abort or throw across the ABI.
 *   - Programs are library-owned and immutable after nc_compile (device
 *     copies are made lazily, once per device, under an internal lock).
 *   - Record buffers are caller-owned. Unless NC_OUT_HOST is set they are
 *     DEVICE pointers (e.g. from torch) on the current CUDA device.
 *   - cuda_stream is a cudaStream_t (NULL = legacy default stream). Device
 *     work is enqueued on it; nc_sample returns after it has completed
 *     (the device-side error word and counters are read back).
 *   - Random draws follow a counter-based Philox4x32-10 contract keyed by
 *     (seed, global shot index, physical event / site index), so shot s of a
 *     call is global shot shot_offset + s and results do not depend on the
 *     launch layout, the precision choice or how shots are split into calls.
 */
#ifndef NC_H
#define NC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NC_OK = 0,
  NC_E_PARSE = 1,            /* circuit text could not be parsed */
  NC_E_UNSUPPORTED = 2,      /* instruction or configuration not supported */
  NC_E_KMAX = 3,             /* peak active dimension above the limit */
  NC_E_NONDET_DETECTOR = 4,  /* a detector/observable is not deterministic */
  NC_E_ARG = 5,              /* invalid argument (NULL, size, alignment) */
  NC_E_OOM = 6,              /* host or device allocation failed */
  NC_E_CUDA = 7,             /* a CUDA runtime call failed */
  NC_E_TIMEOUT = 8,          /* a bounded device wait gave up */
  NC_E_INTERNAL = 9          /* internal invariant violated (a bug) */
} nc_status;

typedef struct nc_program nc_program;

/* Summary of a compiled program. k_max is the peak active dimension fixed
 * at compile time (Thm. 1); n_ops the number of bytecode instructions. */
typedef struct {
  uint32_t n_qubits, n_meas, n_det, n_obs, k_max, n_noise_sites, n_ops;
  uint32_t n_events, n_slots, n_static, n_random, n_active_meas, n_array_ops;
  uint32_t n_probes;  /* EXPVAL probes (rows of nc_records.expval) */
  double array_bytes_fp32;  /* active-vector bytes one shot's array traversals
                               (Sec. 2.6) move at FP32, counted as: expansion
                               3 * 2^k amplitudes, a 1- or 2-axis pass 2 * 2^k,
                               an active measurement 2.5 * 2^k; 8 bytes each */
  uint32_t prefix_ops, prefix_k;  /* shared prefix: the first prefix_ops
                               instructions hold no noise, measurement or
                               record, so every shot leaves them with the same
                               state (prefix_k active axes, zero frame); the
                               batched forms compute that state once per call */
  double prefix_bytes_fp32;  /* the part of array_bytes_fp32 spent in it */
} nc_info;

/* precision */
#define NC_FP32_BATCHED 0  /* bit-sliced frame tiles, FP32 amplitudes, FP64 reductions */
#define NC_FP64_PLAIN 1    /* one thread per shot, FP64 amplitudes (baseline form) */
#define NC_FP64_BATCHED 2  /* the batched layout with FP64 amplitudes (accuracy reference) */

/* outputs bitmask */
#define NC_OUT_MEAS 1u
#define NC_OUT_DET 2u
#define NC_OUT_OBS 4u
#define NC_OUT_KEPT 8u
#define NC_OUT_HOST 16u    /* record pointers are host memory: the kernels write
                              them directly when the device can address them
                              (pinned memory, native host atomics; path bit 2),
                              else the call runs in shot chunks through two
                              device staging buffers whose copies overlap the
                              next chunk (path bit 4; tune "hd=0" forces it) */
#define NC_OUT_EXPVAL 32u  /* expectation-value probes (nc_records.expval) */

/* postselect */
#define NC_PS_NONE 0
#define NC_PS_ALL_DETECTORS 1

typedef struct {
  int precision;          /* NC_FP32_BATCHED, NC_FP64_PLAIN or NC_FP64_BATCHED */
  uint32_t outputs;       /* NC_OUT_* bits */
  int postselect;         /* NC_PS_NONE or NC_PS_ALL_DETECTORS */
  uint64_t shot_offset;   /* global index of this call's first shot */
  const char* tune;       /* NULL = the shape nc_autotune chose, else the
                             built-in heuristic. Otherwise comma-separated
                             key=value pairs: g (32-shot words per executor
                             tile), t (threads per CTA), w (words per owner
                             thread: 1, 2, 4), b (0: no bucketed noise),
                             ps (1: pre-sample faults even for small calls),
                             sw (0: active vectors never in shared memory),
                             px (shared prefix: 0 off, 2 always), a (0: no
                             record-level path for k_max = 0), aw (its words
                             per tile: 8, 16, 32), ai (0: faults sampled in
                             the tile kernel), av (shots per item pass), ac
                             (item-list capacity per tile), ao (1: item
                             passes overlapped on a side stream), lw (1:
                             warp-per-shot layout), wn (its warps per CTA),
                             lp (1: FP32 thread-per-shot layout), mp (1:
                             its persistent form, one vector slot per
                             resident thread; on a batch, every program in
                             one launch), mg (resident CTAs per SM of that
                             launch), hd (0:
                             host outputs staged, not written directly), hc
                             (shots per staged chunk), aq (resident
                             item-kernel CTAs per SM: 2, 3, 4) */
  int noiseless;          /* 1 = disable every noise site (reference runs) */
  uint32_t stratified;    /* 0 = independent noise sites (default);
                             1 = stratified importance sampling: every shot
                             has exactly `stratum` faults (see
                             nc_stratum_weights) */
  uint32_t stratum;       /* faults per shot when stratified (K <= 127) */
} nc_sample_opts;

/*
 * Records layout (record-major, shot-minor, bit-packed):
 *   bit (s % 64) of word [r * words_per_record + s / 64] of a row buffer
 *   holds record r of shot s. words_per_record = ceil(shots / 64); bits of
 *   the last word beyond `shots` are written as 0.
 *   meas: n_meas rows, det: n_det rows, obs: n_obs rows, kept: 1 row.
 * Circuit text: the extended Stim subset of Sec. 3.1 plus EXPVAL, whose
 * targets are Pauli products (Stim's product syntax, e.g. "EXPVAL X0*Y1 Z2":
 * two probes).
 * A rejected (postselected-out) shot reports its failing detector as 1,
 * every later record and detector as 0, all observables 0 and kept = 0.
 * shots_run, shots_kept, kernel_ms, exec_ms and launches are filled by
 * nc_sample.
 */
typedef struct {
  uint64_t *meas, *det, *obs, *kept;
  uint64_t words_per_record;
  uint64_t shots_run, shots_kept;
  double kernel_ms;       /* filled: device time of the whole sampling call
                             (fault bucketing, executors), CUDA events on
                             cuda_stream */
  double exec_ms;         /* filled: device time of this program's dominant
                             kernel (the executor, or the record-tile kernel
                             of the k_max = 0 path), summed over its
                             launches, CUDA events on cuda_stream */
  uint32_t launches;      /* filled: kernels this call launched for this
                             program (memsets and copies not counted) */
  uint32_t path;          /* filled: bit 0 = the shared prefix was computed
                             once for the call (nc_info.prefix_ops) */
  double* expval;         /* NC_OUT_EXPVAL: n_probes rows of `shots` FP64
                             values, probe j of shot s at expval[j * shots + s]:
                             <psi|P|psi> / <psi|psi> of the shot's state where
                             the EXPVAL target P stands (Sec. 3.2, expectation
                             probes on the runtime state); 0 for a shot already
                             rejected by postselection there. NULL is allowed
                             when the program has no probes. */
} nc_records;

/* Compile extended-Stim text (Sec. 3.1). On failure *out is NULL and a
 * message is written to err (if err_len > 0). The text is not retained. */
nc_status nc_compile(const char* text, size_t len, nc_program** out, char* err, size_t err_len);

/* Compile flags. The compiler's HIR passes (Sec. 3.1, stage 2) act on every
 * active operation written as a Pauli of the t = 0 frame (the Heisenberg
 * image through the physical Cliffords before it); two operations commute iff
 * their Paulis do. The passes change the bytecode, the k-schedule and the
 * intermediate states, never a probability or a record; each flag turns one
 * pass off, so that a program can be compared step by step with a plain run
 * of the method (App. B). NC_COMPILE_PLAIN turns them all off.
 *   NC_COMPILE_NO_PEEPHOLE: keep every rotation. By default a rotation whose
 *     axis is measured later, with every operation in between commuting with
 *     it (for instance a T before its qubit's Z measurement), is dropped: next
 *     to the measurement it contributes a phase per outcome branch only.
 *   NC_COMPILE_NO_REORDER: keep circuit order. By default a measurement moves
 *     ahead of the rotations it commutes with, and a rotation after the
 *     measurements it commutes with, so the active dimension contracts
 *     before it grows; noise sites keep their order, measurements keep their
 *     place among detectors, nothing passes an EXPVAL probe.
 *   NC_COMPILE_NO_FUSE: no phase fusion. By default two rotations about the
 *     same axis with only commuting operations between them become one (T T
 *     is one pi/4 rotation), and a rotation whose angle is then a multiple of
 *     pi/4 (a Clifford, a Pauli or the identity, e.g. T T_DAG) leaves the list
 *     after conjugating every later operation. */
#define NC_COMPILE_NO_PEEPHOLE 1u
#define NC_COMPILE_NO_REORDER 2u
#define NC_COMPILE_NO_FUSE 4u
#define NC_COMPILE_PLAIN 7u
#define NC_COMPILE_FLAGS_ALL 7u

/* nc_compile with compile flags (NC_COMPILE_* bits; nc_compile passes 0).
 * An unknown flag bit is NC_E_ARG. */
nc_status nc_compile_ex(const char* text, size_t len, uint32_t flags, nc_program** out, char* err,
                        size_t err_len);

/* Fill *info for a compiled program. */
nc_status nc_program_info(const nc_program* prog, nc_info* info);

/* Serialize a program to a versioned byte blob. With buf == NULL, *len
 * receives the size needed; otherwise *len is the capacity of buf and
 * receives the bytes written (NC_E_ARG if too small). */
nc_status nc_program_serialize(const nc_program* prog, void* buf, size_t* len);

/* Rebuild a program from nc_program_serialize output. */
nc_status nc_program_deserialize(const void* buf, size_t len, nc_program** out);

/* Sample `shots` shots (Sec. 3.2). opts may be NULL (FP32 batched, all
 * outputs, no postselection, shot_offset 0). Synchronises cuda_stream before
 * returning. The first call on a device uploads the program and runs a
 * 64-shot noiseless reference launch that fixes the detector/observable
 * reference parities (NC_E_NONDET_DETECTOR if those shots disagree). */
nc_status nc_sample(const nc_program* prog, uint64_t shots, uint64_t seed,
                    const nc_sample_opts* opts, nc_records* out, void* cuda_stream);

/* Sample n programs on one stream: program i runs shots[i] shots with
 * seeds[i] into outs[i]. Same semantics as n calls of nc_sample. */
nc_status nc_sample_batch(const nc_program* const* progs, const uint64_t* shots,
                          const uint64_t* seeds, uint32_t n, const nc_sample_opts* opts,
                          nc_records* outs, void* cuda_stream);

/* Upload a program to the current device and run its 64-shot noiseless
 * reference launch (Sec. 3.2 records: detector / observable references);
 * synchronises cuda_stream. nc_sample does this on first use; call it
 * explicitly before nc_sample_batch_async. */
nc_status nc_program_prepare(const nc_program* prog, void* cuda_stream);

/* nc_sample_batch for stream capture (a CUDA graph of many circuits, the
 * batching row of Sec. 3.2): only enqueues work on cuda_stream and never
 * synchronises the host. Requirements: every program prepared on the
 * current device (else NC_E_ARG); device outputs only (NC_OUT_HOST is
 * NC_E_ARG). kept_dev (n device u64) and err_dev (one device u32) are
 * caller-owned and zeroed by the caller: kept_dev[i] accumulates program
 * i's kept shots and err_dev receives a nonzero value if a kernel reported
 * an internal error. outs[i].shots_run is set; shots_kept, kernel_ms,
 * exec_ms and launches are 0. Scratch comes from the stream-ordered pool.
 * The programs run on up to 16 internal streams forked from cuda_stream (an
 * event recorded on it) and joined back into it (events it waits for), so
 * that small programs run beside large ones and a captured graph holds one
 * branch per group of programs; all work is ordered after what cuda_stream
 * held at the call and before what it is given next. */
nc_status nc_sample_batch_async(const nc_program* const* progs, const uint64_t* shots,
                                const uint64_t* seeds, uint32_t n, const nc_sample_opts* opts,
                                nc_records* outs, unsigned long long* kept_dev, uint32_t* err_dev,
                                void* cuda_stream);

/*
 * Stratified importance sampling (Sec. 3.2, the rare-event mode used for
 * Sec. 4.2.1): a call with opts->stratified = 1 runs stratum K =
 * opts->stratum, whose shots each have exactly K realised faults drawn from
 * the independent-site distribution conditioned on K faults,
 *   P(F | |F| = K) = prod_{i in F} p_i prod_{i not in F} (1 - p_i) / P(K).
 * An estimate over strata weights the stratum-K mean by P(K), the
 * Poisson-binomial mass that nc_stratum_weights returns. Each fault's Pauli
 * option is drawn as for independent noise; everything else is unchanged.
 * Draw contract: shot s holding r faults at site index st draws
 * Philox(key, (s lo, s hi, 4, st)); u = ((w0 | w1 << 32) >> 11) * 2^-53; the
 * fault is the first j >= st with G_r(j + 1) <= u * G_r(st) (FP64), where
 * G_r(j) = prod_{l<j}(1 - p_l) * P(r faults among sites j..) as a running
 * minimum over j; its option is floor(w2 * K_j / 2^32).
 * A stratum is refused (NC_E_ARG) if some site has p >= 1, if K exceeds the
 * number of sites with p > 0, or if the tables underflow the FP64 normal
 * range. K = 0 is the noiseless run. nc_sample_noalloc does not support it
 * (NC_E_UNSUPPORTED).
 */

/* weights[K] = P(exactly K faults) for K = 0..k_max (k_max + 1 doubles, host
 * memory); valid (optional, k_max + 1 bytes) receives 1 for every stratum
 * that can be sampled. Host computation only. */
nc_status nc_stratum_weights(const nc_program* prog, uint32_t k_max, double* weights, uint8_t* valid);

/* Upload the stratified tables for strata up to k_max to the current device
 * (and prepare the program as nc_program_prepare does). nc_sample does this
 * on demand; nc_sample_batch_async requires it (NC_E_ARG otherwise). */
nc_status nc_strata_prepare(const nc_program* prog, uint32_t k_max, void* cuda_stream);

/* Launch-shape autotuner (shots per CTA, CTA size, warp- or word-per-shot
 * layout of the record tile, fault pre-sampling; for programs with active
 * axes also the warp-per-shot layout "lw=1" and the FP32 thread-per-shot
 * layout "lp=1"): times the candidates for
 * this program on min(shots, 2^22) shots with opts' outputs and keeps the
 * fastest for later calls on this device whose opts->tune is NULL. best
 * (if best_len > 0) receives the chosen shape as a tune string. The
 * program must not be sampled concurrently while it is tuned. */
nc_status nc_autotune(nc_program* prog, uint64_t shots, const nc_sample_opts* opts, void* cuda_stream,
                      char* best, size_t best_len);

/*
 * Allocation-free sampling. Some callers cannot allocate device memory once
 * they are running: an application whose device memory is owned entirely by
 * another framework's caching pool, code that must not hit the implicit
 * synchronisation of an allocation inside a latency-critical loop, or a
 * process that is only allowed to allocate during start-up. For them
 * nc_sample_noalloc behaves like nc_sample with precision NC_FP32_BATCHED,
 * but it calls no cudaMalloc / cudaFree (nor any allocating library routine):
 * the device copy of the program, the reference-parity launch, the counters
 * and the amplitude workspace all live in one fixed array that the library
 * reserves statically on every device that loads it (NC_NOALLOC_SCRATCH_BYTES,
 * held until the process exits). The paper has no counterpart of this entry
 * point; it is an integration convenience.
 *   - Record buffers are caller-owned device memory (NC_OUT_HOST: NC_E_ARG).
 *   - opts->precision must be NC_FP32_BATCHED (else NC_E_ARG); opts->tune is
 *     ignored.
 *   - NC_E_ARG if the program blob plus its workspace cannot fit in
 *     NC_NOALLOC_SCRATCH_BYTES (large k_max or very long programs). The
 *     64-shot reference launch runs with FP64 amplitudes, as nc_sample's
 *     does, and needs twice the FP32 workspace of one tile.
 *   - NC_E_UNSUPPORTED if one 32-shot tile's frame planes and record slots
 *     exceed the shared memory of a CTA (tens of thousands of qubits).
 *   - Launch shapes come from a fixed table by k_max, and the speed-ups of
 *     nc_sample that need allocations (vectors in shared memory, the shared
 *     noiseless prefix, pre-sampled noise) are not used: records equal
 *     nc_sample's, speed can differ.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Every call reuses the same array and leaves the last call's contents in
 *     it; calls whose work overlaps on the GPU (different streams, or host
 *     threads without ordering) race on it and must be serialised by the
 *     caller. Each call synchronises cuda_stream before returning.
 */
#define NC_NOALLOC_SCRATCH_BYTES (64u << 20)
nc_status nc_sample_noalloc(const nc_program* prog, uint64_t shots, uint64_t seed,
                            const nc_sample_opts* opts, nc_records* out, void* cuda_stream);

/* Free a program and its device copies. NULL is a no-op. */
void nc_program_free(nc_program* prog);

/* Static string for a status code. */
const char* nc_status_str(nc_status st);

/* Test hook: run shot `shot` (global index) of `seed` up to, not including,
 * measurement event `event` and return its frame and active state vector.
 * frame_xz: 2 * ceil(n_qubits / 32) words (x bits of virtual qubits, then z
 * bits); amps: at least 2 * 2^k_max doubles (re, im interleaved), converted
 * to FP64; *k: active dimension at that point. Host pointers. A program
 * whose noiseless prefix (nc_info.prefix_ops) ends with 15 or more active
 * axes starts from that prefix's state computed once, as sampling calls do;
 * otherwise the shot runs the instruction list from the start. */
nc_status nc_debug_dump(const nc_program* prog, uint64_t seed, uint64_t shot, uint32_t event,
                        int precision, uint32_t* frame_xz, double* amps, uint32_t* k,
                        void* cuda_stream);

/* Version of the serialized program format and of the ABI. */
uint32_t nc_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NC_H */
