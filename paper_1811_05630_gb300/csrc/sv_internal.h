// sv_internal.h — launchers shared by the host API and the kernels translation unit.
#pragma once
#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>

#include "sv_block.cuh"

namespace sv {

// Per-device one-time setup of a kernel's launch attributes: `done` is a bit set over device
// ordinals (0..63) owned by the caller (one per kernel instantiation). Returns the error of the
// first failing setup call, cudaSuccess once the current device is set up.
template <typename F>
inline cudaError_t once_per_device(std::atomic<unsigned long long>& done, F setup) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = setup();
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Fused gate pass (Algorithm 1 over every slice) for one state; Real by dtype (1 = float).
cudaError_t launch_pass(const PassArgs& a, int dtype, cudaStream_t st);
// The same pass built with a register cap for 1- and 2-qubit gates (others: launch_pass).
cudaError_t launch_pass_compact(const PassArgs& a, int dtype, cudaStream_t st);
// The fused pass over the block-groups of many states (one descriptor each).
cudaError_t launch_pass_batch(const PassArgs* descs, const unsigned long long* gprefix, int nstates,
                              unsigned long long total_groups, int b, int Gmax, int Kmax, int dtype,
                              int threads, int chunk, cudaStream_t st);
// Norm finalization after a pass (one CTA per state): verbatim-sum tree when needed, N, sigma,
// statistics; resets the bump of the arena the next pass writes.
cudaError_t launch_norm(DevScalars* sc, const double* vsum, unsigned long long nb, double* tree, double two2,
                        int out_id, unsigned int seq, cudaStream_t st);
cudaError_t launch_norm_batch(const PassArgs* descs, int nstates, cudaStream_t st);

// Standalone codec.
cudaError_t launch_codec_compress(const void* values, unsigned long long nblocks, int b,
                                  int dtype, QuantP qp, uint8_t* out, unsigned long long cap,
                                  unsigned long long* offsets, unsigned int* lengths,
                                  DevScalars* sc, double* vsum, cudaStream_t st);
cudaError_t launch_codec_decompress(const uint8_t* in, const unsigned long long* offsets,
                                    const unsigned int* lengths, unsigned long long nblocks,
                                    int b, int dtype, QuantP qp, void* values, DevScalars* sc,
                                    cudaStream_t st);
// Decoded (reconstructed) amplitudes of blocks [b0, b0 + nb) as FP64 (re, im) into out.
cudaError_t launch_read_blocks(const uint8_t* arena, const unsigned long long* offs,
                               const unsigned int* lens, unsigned long long b0,
                               unsigned long long nb, int b, int dtype, QuantP qp,
                               double* out, DevScalars* sc, cudaStream_t st);

// Reductions over FP64 (re, im) chunks.
cudaError_t launch_probs_chunk(const double* amp, unsigned long long start,
                               unsigned long long count, const int* qubits_dev, int m,
                               double* bins, cudaStream_t st);
cudaError_t launch_dot_chunk(const double* a, const double* b, unsigned long long count,
                             double* acc4, cudaStream_t st);

cudaError_t launch_qft_overlap_chunk(const double* amp, unsigned long long start, unsigned long long count,
                                     unsigned long long x, int n, double* acc, cudaStream_t st);

// Plain (uncompressed) path.
// G: host matrix (k <= 3) ; G_dev: the same matrix in device memory (read for k = 4, 5)
cudaError_t launch_plain_gate(void* psi, int n, int dtype, const double* G, const int* targets,
                              int k, unsigned long long cmask, const double* G_dev, cudaStream_t st);
cudaError_t launch_plain_basis(void* psi, int n, int dtype, unsigned long long index,
                               cudaStream_t st);
cudaError_t launch_plain_read(const void* psi, int dtype, unsigned long long start,
                              unsigned long long count, double* out, cudaStream_t st);

}  // namespace sv
