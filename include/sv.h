/*
 * sv.h — C ABI of libsv.so, the GB300 (sm_103a) compressed state-vector simulator.
 *
 * The library implements the per-gate slice update of Algorithm 1 of Wu, Di, Cappello,
 * Finkel, Alexeev and Chong, "Memory-Efficient Quantum Circuit Simulation by Using Lossy
 * Data Compression" (PMES 2018): the state vector of n qubits (Sec. I: 2^n complex
 * amplitudes) is kept divided into slices, every slice stored compressed by an SZ-style
 * error-bounded lossy codec (Sec. II); each gate is applied by decompressing, normalizing,
 * applying the gate and recompressing every slice (Algorithm 1). On the GPU one kernel
 * launch performs this for all slices at once; decompressed amplitudes live only in
 * shared memory and registers.
 *
 * Conventions
 *   - Qubit q is bit q of the amplitude index (little-endian).
 *   - A slice is 2^slice_log2 consecutive amplitudes; it is coded as 2^(slice_log2 -
 *     block_log2) independent blocks of B = 2^block_log2 amplitudes (the parallel unit).
 *   - Amplitudes are interleaved (re, im): complex128 (SV_C128, FP64 gate arithmetic) or
 *     complex64 (SV_C64, FP32 gate arithmetic; quantization and the norm stay FP64).
 *   - Gates: G is a row-major 2^k x 2^k complex matrix given as (re, im) FP64 pairs;
 *     targets[0] is the least significant bit of G's basis index. Controls are qubits that
 *     must all be 1; they are disjoint from the targets. G is copied during the call; the
 *     caller keeps ownership of every host buffer it passes.
 *   - error_bound > 0 selects the compressed path; error_bound == 0 selects the plain
 *     (uncompressed) path, the comparison baseline, with the same calls.
 *   - Device memory: the library allocates none. The caller hands it one device buffer
 *     (sv_pool_create); every state's arenas, tables and scalars are sub-allocated there.
 *   - Streams: every call is ordered on the state's CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream). Calls that return host data synchronize that
 *     stream; the others are asynchronous.
 *   - Host threads: a state or a batch is used by one host thread at a time; states on one
 *     pool may be used from different threads (the pool's allocator is locked).
 *   - Errors: every call returns 0 (SV_OK) or a negative SV_ERR_* code. An error raised
 *     inside a kernel (stream corruption, arena overflow, norm collapse) is recorded on the
 *     device and returned by the next synchronizing call; later passes of that state are
 *     skipped until then. Arena overflow is recovered inside sv_sync by growing the arena
 *     and replaying the logged gates, so callers only see SV_ERR_OOM when the pool is full.
 */
#ifndef SV_H
#define SV_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SV_OK 0
#define SV_ERR_ARG (-1)         /* invalid argument */
#define SV_ERR_OOM (-2)         /* pool exhausted */
#define SV_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define SV_ERR_NORM (-4)        /* stored norm is zero or not finite */
#define SV_ERR_CORRUPT (-5)     /* a block stream failed the decoder's bounds checks */
#define SV_ERR_UNSUPPORTED (-6) /* outside the library's limits (see each call) */
#define SV_ERR_TIMEOUT (-7)     /* a bounded device wait ran out */
#define SV_ERR_INTERNAL (-8)    /* a device-side consistency check failed (a library bug) */

#define SV_C64 1
#define SV_C128 2

typedef struct sv_pool sv_pool;
typedef struct sv_state sv_state;

/* Statistics of the most recent gate pass (or of sv_create's initial compression). */
typedef struct {
  uint64_t pass_index;       /* passes completed on this state */
  uint64_t compressed_bytes; /* sum of all block streams (headers, codebooks, payload) */
  uint64_t table_bytes;      /* block offset/length tables */
  uint64_t n_blocks;
  uint64_t blocks_const, blocks_huff, blocks_pack; /* block modes */
  uint64_t n_verbatim, n_escape;
  double norm;               /* N of the stored state after the pass */
  double sigma;              /* scale the next pass applies, 1/sqrt(norm) */
  uint64_t blocks_reused;    /* blocks whose stream the pass re-emitted unchanged: the pass
                                provably reproduced their codes (or a partner block's), so
                                the stream is what recoding would have written */
  uint64_t replayed_passes;  /* passes re-run after an arena overflow, since creation */
  uint64_t peak_compressed_bytes; /* largest compressed_bytes of any pass since the last
                                     sv_reset_basis: the paper's minimum compression ratio over
                                     a run (Sec. III) is the raw size divided by this */
  uint64_t spill_arena_bytes;  /* capacity of the state's arenas held in its spill pool */
} sv_stats_t;

/* ---------------------------------------------------------------------------------------
 * Pool. dev_base: device pointer to `bytes` bytes owned by the caller (e.g. a torch
 * tensor), 256-byte aligned, valid until sv_pool_destroy. The pool hands out page runs
 * (2 MiB pages) to states. Returns SV_ERR_ARG on a NULL/misaligned pointer.
 * ------------------------------------------------------------------------------------- */
int sv_pool_create(void* dev_base, size_t bytes, sv_pool** out);
int sv_pool_destroy(sv_pool* pool); /* fails with SV_ERR_ARG while states or their pages remain */

/* Spill pool (the paper's aim of fitting more qubits into a given memory, Sec. I and IV):
 * sv_pool_create also accepts pinned host memory that the device can address (e.g. a pinned
 * torch CPU tensor); the kernels then read and write its pages in host memory (over
 * NVLink-C2C on a Grace system). sv_set_spill_pool(s, spill): arenas (the compressed streams)
 * and measurement buffers of state s that do not fit in its pool are taken from `spill`
 * (NULL: none); metadata and block tables stay in the state's pool. Results do not depend on
 * where the arenas are. SV_ERR_ARG for a plain state or spill == the state's pool. The spill
 * pool must outlive the state's use of it (sv_pool_destroy refuses while pages are held). */
int sv_set_spill_pool(sv_state* s, sv_pool* spill);
int sv_pool_usage(const sv_pool* pool, size_t* used_bytes, size_t* capacity_bytes);

/* ---------------------------------------------------------------------------------------
 * sv_create — a state of n_qubits initialized to |0...0>, compressed (Algorithm 1's input;
 * Sec. II error bound).
 *   n_qubits   1..40 (compressed: block_log2 <= n_qubits), slice_log2 in [block_log2, n].
 *   error_bound absolute bound on every real and imaginary part after each compression,
 *              > 0; or 0 for the plain path (no codec).
 *   dtype      SV_C64 or SV_C128.
 *   stream     cudaStream_t (as void*) all work of this state is ordered on.
 * Block size: min(slice_log2, 12) unless sv_create_ex sets it (5..12; -1 = default).
 * arena_bytes (sv_create_ex): capacity of each of the two arenas (0 = default: 64 bytes
 *   per block, at least one 2 MiB page, and at every status check the arena the next pass
 *   writes is reserved at twice the live state); arenas grow on overflow (sv_sync), and a
 *   caller-given size grows on overflow only.
 * Returns SV_ERR_OOM when the pool cannot hold the state's initial arenas.
 * ------------------------------------------------------------------------------------- */
int sv_create(sv_pool* pool, int n_qubits, int slice_log2, double error_bound, int dtype,
              void* stream, sv_state** out);
int sv_create_ex(sv_pool* pool, int n_qubits, int slice_log2, int block_log2,
                 double error_bound, int dtype, size_t arena_bytes, void* stream,
                 sv_state** out);
int sv_destroy(sv_state* s);

/* Re-initialize to the computational basis state |index> (index < 2^n). Asynchronous. */
int sv_reset_basis(sv_state* s, uint64_t index);

/* ---------------------------------------------------------------------------------------
 * sv_apply_gate — one gate pass of Algorithm 1 over every slice: Decompress(S),
 * Normalize(S) (global scale 1/sqrt(N) of the stored norm N), GateComputation(G, S),
 * Compress(S). Slices are processed in every pass, also where the controls make the gate
 * the identity. Targets at or above block_log2 pair the 2^h coupled blocks inside one CTA
 * (h <= 2: SV_ERR_UNSUPPORTED otherwise). k in 1..5 targets (Sec. II applies any gate; the
 * paper does not bound k): G is a dense 2^k x 2^k complex matrix, e.g. several gates fused
 * into one; with k >= 4 the CTA also keeps the matrix in fixed point, and 4096-amplitude
 * blocks (block_log2 12) with two high targets then exceed the shared memory of a CTA
 * (SV_ERR_UNSUPPORTED). SV_ERR_ARG: k outside 1..5, a qubit outside 0..n-1, repeated or
 * shared between targets and controls.
 * Plain path: G applied in place to the uncompressed vector (no normalization).
 * Asynchronous; errors raised on the device are reported by the next synchronizing call.
 * ------------------------------------------------------------------------------------- */
int sv_apply_gate(sv_state* s, const double* G, const int* targets, int k,
                  const int* controls, int n_controls);

/* ---------------------------------------------------------------------------------------
 * Batching: one gate pass for many states in one launch (the pass kernel walks the
 * block-groups of all of them), for serving many small simulations at once.
 * sv_batch_create: max_states per step; device descriptors come from the pool, host staging
 *   is pinned memory; all work goes to `stream`, which every state of a step must use.
 * sv_batch_apply: gates[i] to states[i] for i < count: each state gets one Algorithm 1 pass
 *   exactly as sv_apply_gate would give it (bit-identical results). States must be compressed,
 *   of one dtype and one block size, each at most once per call; gates of at most 3 qubits
 *   (SV_ERR_UNSUPPORTED for 4 and 5). Asynchronous; each state's errors and overflow replay
 *   are handled by its own sv_sync.
 * sv_batch_use_graphs: capture the step (descriptor copy, pass, norm kernels) as CUDA graphs,
 *   one per batch shape (count, gate width, coupled blocks, groups) and replay them.
 * ------------------------------------------------------------------------------------- */
typedef struct {
  const double* G;      /* row-major 2^k x 2^k complex (re, im) FP64 */
  const int* targets;
  int k;
  const int* controls;
  int n_controls;
} sv_gate_t;
typedef struct sv_batch sv_batch;
int sv_batch_create(sv_pool* pool, int max_states, void* stream, sv_batch** out);
int sv_batch_destroy(sv_batch* batch);
int sv_batch_use_graphs(sv_batch* batch, int on);
/* 1 when sv_batch_apply would not wait for the host staging buffer of an earlier step
 * (lets a host loop serve other batches meanwhile), 0 otherwise, <0 on error. */
int sv_batch_ready(sv_batch* batch);
int sv_batch_apply(sv_batch* batch, sv_state* const* states, const sv_gate_t* gates, int count);

/* Wait for the state's stream, resolve arena overflow (grow + replay) and return any
 * error recorded on the device. */
int sv_sync(sv_state* s);

/* ---------------------------------------------------------------------------------------
 * Measurements (synchronizing). The paper judges a compressed simulation by the fidelity of
 * its final state to the uncompressed simulator's and by the compression ratio, whose minimum
 * over a run sets how many extra qubits fit in memory (Sec. III; the ratio as the measure of
 * the method's scalability: Sec. I). Arguments are host pointers owned by the caller; errors:
 * SV_ERR_ARG for bad arguments, SV_ERR_NORM when the state's norm is zero, otherwise any error
 * the state has recorded on the device.
 * sv_measure_probs: marginal probabilities of the m (<= 14) given qubits of the normalized
 *   stored state (the Born rule on the state Sec. II keeps, normalized by its stored norm N);
 *   out[2^m] (host), out[v] = P(bits of the listed qubits = v, qubits[0] least significant).
 *   The paper prints no probabilities; for its QFT benchmark (Sec. III) on a basis state
 *   every outcome has probability 2^-n, which these marginals check.
 * sv_amplitudes: the stored (reconstructed, not rescaled) amplitudes x' at host indices
 *   idx[] into out[2*cnt] (re, im FP64). The stored state has norm sv_norm(); multiply by
 *   1/sqrt(norm) for the normalized amplitudes.
 * sv_read_amplitudes: stored amplitudes [start, start+count) into host out[2*count].
 * sv_fidelity: F = |<a|b>|^2 / (<a|a><b|b>) of two states of equal n (either path), the
 *   state fidelity of Sec. III (1 for identical states) in its squared pure-state form; the
 *   paper compares the compressed run's final amplitudes with the original simulator's,
 *   which is this call with b on the plain path (error_bound 0). *out receives F.
 * sv_compressed_bytes: bytes of all block streams of the current state (headers, codebooks,
 *   payload, verbatim values; plain path: the vector's bytes). The compression ratio of
 *   Sec. I / III is 2^(n+4) (complex128) or 2^(n+3) (complex64) divided by this; the paper
 *   reports its minimum over the run (Sec. III), i.e. this call after every gate.
 * ------------------------------------------------------------------------------------- */
int sv_measure_probs(sv_state* s, const int* qubits, int m, double* out);
int sv_amplitudes(sv_state* s, const uint64_t* idx, size_t cnt, double* out);
int sv_read_amplitudes(sv_state* s, uint64_t start, uint64_t count, double* out);
int sv_fidelity(sv_state* a, sv_state* b, double* out);
int sv_compressed_bytes(sv_state* s, uint64_t* out);
int sv_stats(sv_state* s, sv_stats_t* out);

/* Threads per CTA of the fused pass for this state (an autotuning knob; the paper has no
 * counterpart): 0 restores the default (one thread per 32-value decode chunk, 32..256);
 * otherwise a power of two T, 32 <= T <= 256, with 2 <= 2^(block_log2+1) / T <= 32 and
 * 2^(block_log2+1) / chunk <= T (sv_set_chunk). Results (streams, norms) do not depend on
 * it. SV_ERR_ARG for other values or a plain state. A batch runs with the setting of its
 * first state. */
int sv_set_threads(sv_state* s, int threads);

/* Select (on != 0) the register-capped build of the fused pass for 1- and 2-qubit gates
 * (1-qubit gates: 64 registers per thread, so that four 256-thread CTAs fit on an SM; 2-qubit
 * gates: 85, three CTAs; larger gates keep the default build). An autotuning knob with no counterpart in the paper; results do not
 * depend on it. SV_ERR_ARG for a plain state. Batches ignore it. */
int sv_set_compact(sv_state* s, int on);

/* Apply 4- and 5-qubit complex128 gates on the tensor cores (on != 0, the default) or on the
 * CUDA cores. An implementation choice with no counterpart in the paper: the tensor cores
 * compute the fixed-point gate sums exactly through FP16 digit products (with the same
 * tie-margin fallback to the FP64 chain), so streams and norms do not depend on it; passes on
 * the tensor cores use 256-thread CTAs. SV_ERR_ARG for a plain state. */
int sv_set_tensor_cores(sv_state* s, int on);

/* Huffman chunk size of the state's block format: the number of symbols per stored chunk bit
 * count, each chunk decoded by one thread (16, 32 or 64; the default 32). Smaller chunks
 * decode with more threads in parallel and cost 16 more bits per chunk of stream. It changes
 * the bytes of the streams (not the decoded values), so the state is reset to |0...0>
 * (synchronizing). Needs 2^(block_log2+1) / chunk <= the state's CTA size (sv_set_threads),
 * SV_ERR_ARG otherwise; batched states must share it. An autotuning knob. */
int sv_set_chunk(sv_state* s, int chunk);
int sv_norm(sv_state* s, double* out);

/* Overlap with the exact QFT of the basis state |x> (the closed form
 * 2^{-n/2} sum_y exp(2 pi i (x y mod 2^n) / 2^n) |y>, which the plain simulator reaches):
 * out[0], out[1] = re, im of <ref|psi>, out[2] = <psi|psi> (psi the stored amplitudes), so
 * the fidelity is (out[0]^2 + out[1]^2) / out[2]. Streams the state in decoded chunks; a
 * validation service for states too large for a plain reference. Synchronizing. */
int sv_overlap_qft(sv_state* s, uint64_t x, double* out);

/* Copy block `b`'s stream (current state) to host `out` (capacity `cap` bytes); *len gets
 * its length. SV_ERR_ARG when cap is too small. Used to compare streams byte by byte. */
int sv_block_stream(sv_state* s, uint64_t b, uint8_t* out, size_t cap, size_t* len);

/* ---------------------------------------------------------------------------------------
 * Standalone block codec (Sec. II), the same device code the gate pass uses.
 * sv_codec_compress: nblocks blocks of 2^block_log2 amplitudes from device `values`
 *   (interleaved, dtype's component type) into device `out` (capacity `cap` bytes); block
 *   i's stream is written at out + offsets[i] with length lengths[i] (device arrays of
 *   nblocks u64/u32). Streams are packed in an order that is not specified. *used (host)
 *   receives the total bytes. SV_ERR_OOM when cap is too small (nothing is valid then).
 * sv_codec_decompress: the inverse, from device streams at in + offsets[i] into device
 *   `values`. SV_ERR_CORRUPT when a stream fails the bounds checks.
 * Both synchronize `stream`. The scratch they need (a few counters) is the caller's
 *   `scratch` device buffer of at least sv_codec_scratch_bytes() bytes. nblocks == 0 is a
 *   no-op that returns SV_OK (compress: *used = 0); the buffers may then be NULL.
 * ------------------------------------------------------------------------------------- */
size_t sv_codec_scratch_bytes(void);
int sv_codec_compress(const void* values, uint64_t nblocks, int block_log2, int dtype,
                      double error_bound, void* out, uint64_t cap, uint64_t* offsets,
                      uint32_t* lengths, void* scratch, void* stream, uint64_t* used);
int sv_codec_decompress(const void* in, const uint64_t* offsets, const uint32_t* lengths,
                        uint64_t nblocks, int block_log2, int dtype, double error_bound,
                        void* values, void* scratch, void* stream);

/* ---------------------------------------------------------------------------------------
 * sv_codec_compress_static — sv_codec_compress for callers that cannot allocate device
 * memory (no scratch argument). The paper has no counterpart: this is a library service.
 * Who needs it: code that runs where device allocation is forbidden or unavailable, e.g. a
 * runtime that owns every allocation up front, or a caller without access to an allocator;
 * such a caller still owns the inputs and outputs (values, out, offsets, lengths) but
 * cannot provide sv_codec_scratch_bytes() of scratch.
 * The scratch lives in a fixed array compiled into libsv.so (about 513 KB; every GPU that
 * loads the library holds it until the process exits): a 256-byte bookkeeping record plus
 * one double per block. At most SV_STATIC_MAX_BLOCKS blocks per call (SV_ERR_UNSUPPORTED
 * beyond). Outputs as sv_codec_compress (same streams, same `used`), plus *norm (if not
 * NULL): the stored norm of the compressed values, N = fl(fl(Sd*(2eb)^2) + V), with Sd the
 * exact sum of the squared codes and V the pairwise sum of the per-block squares of the
 * verbatim values (list padded with zeros to a power of two).
 * The first call on a device looks the array's device address up (once per device, with
 * that device current) and caches it for the life of the process; after a cudaDeviceReset
 * of that device the cached address is stale, so do not call this function on a device the
 * process has reset. Every call clears the record it uses at its start; the array is shared
 * by all calls on a device and keeps the last call's contents, so calls that overlap on the
 * GPU (other streams or threads) race and must be serialized by the caller. Every call reads
 * its results back and synchronizes `stream`, so it cannot be recorded into a CUDA graph: on a
 * stream that is capturing (or whose capture state cannot be read) it returns SV_ERR_ARG
 * before enqueueing anything. nblocks == 0: SV_OK with *used = 0 and *norm = 0, nothing
 * launched (the buffers may then be NULL). No memory is allocated.
 * ------------------------------------------------------------------------------------- */
#define SV_STATIC_MAX_BLOCKS 65536
int sv_codec_compress_static(const void* values, uint64_t nblocks, int block_log2, int dtype,
                             double error_bound, void* out, uint64_t cap, uint64_t* offsets,
                             uint32_t* lengths, void* stream, uint64_t* used, double* norm);

/* ---------------------------------------------------------------------------------------
 * Tracing. sv_set_pass_timing(s, 1) records CUDA events on the state's stream around every
 * fused pass kernel from then on and zeroes the counters (0 stops recording).
 * sv_get_pass_timing synchronizes and returns the summed kernel time of the recorded
 * passes (ms), their number, and their algorithmic bytes: compressed bytes read plus
 * written, plus 64 bytes per block of table traffic (offset and length read and written,
 * the block summary read and written, the verbatim sum written).
 * ------------------------------------------------------------------------------------- */
int sv_set_pass_timing(sv_state* s, int on);
int sv_get_pass_timing(sv_state* s, double* kernel_ms, uint64_t* passes, uint64_t* bytes);

/* Self-check of the bounded device wait (failure detection; no counterpart in the paper).
 * The tensor-core pass waits for its matrix multiplies on an mbarrier and gives up after a
 * bounded number of polls, recording a timeout that the next sv_sync returns as
 * SV_ERR_TIMEOUT instead of hanging. This call runs that wait on an mbarrier nothing arrives
 * on, polling `polls` times (1 <= polls <= 2^24), on `stream` (a cudaStream_t; NULL: the
 * legacy default stream), synchronizes the stream and sets *timed_out to 1 when the wait gave
 * up (the expected result) and 0 when the phase completed. The context stays usable.
 * SV_ERR_ARG for a NULL output or polls out of range; SV_ERR_CUDA if a CUDA call failed. */
int sv_check_bounded_wait(long long polls, void* stream, int* timed_out);

/* Library version string and the sm architecture it was built for. */
const char* sv_version(void);

#ifdef __cplusplus
}
#endif
#endif
