// sv_static.cu — the block compressor for callers that cannot allocate device memory.
//
// sv_codec_compress needs a small caller-provided scratch buffer (a bump counter, status
// flags and statistics). Some callers cannot provide one: code that runs where device
// allocation is forbidden or unavailable (inside a region whose memory was fixed up front,
// or in a runtime that owns every allocation). sv_codec_compress_static does the same
// compression with its scratch in a fixed array compiled into the library instead, and also
// reports the stored norm of what it compressed. It allocates nothing.
//
// The array is shared by every call on a device and keeps the last call's contents; each
// call clears the part that must start at zero. Calls that overlap on the GPU (two streams,
// or two host threads) race on it and must be serialized by the caller. Every call reads its
// results back to the host and synchronizes the stream, so it cannot be recorded into a CUDA
// graph: a call on a stream that is capturing is refused (SV_ERR_ARG) before any work.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/sv.h"
#include "sv_internal.h"

using namespace sv;

namespace {

constexpr unsigned long long kMaxBlocks = SV_STATIC_MAX_BLOCKS;
constexpr size_t kRecordBytes = 256;  // DevScalars, padded
static_assert(sizeof(DevScalars) <= kRecordBytes, "record must fit its slot");

// [0, 256): the bookkeeping record; then one double per block (verbatim sums) and a few
// words for the norm. Every GPU that loads the library holds this until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kRecordBytes + 8 * kMaxBlocks + 256];

constexpr int kMaxDevices = 64;
void* g_dev_ptr[kMaxDevices] = {nullptr};
std::mutex g_mu;

// Device address of g_scratch on the current device (looked up once per device, then
// cached for the life of the process: after a cudaDeviceReset the cached address is stale,
// so a process that resets a device must not call this entry point on it again).
cudaError_t scratch_ptr(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_dev_ptr[dev] = p;
  }
  *out = g_dev_ptr[dev];
  return cudaSuccess;
}

// Stored norm of the compressed blocks, with the same definition as a state's norm:
// N = fl(fl(Sd * two2) + V), Sd from the exact 128-bit sum of q^2, V the level-by-level
// pairwise sum of the per-block verbatim sums, the list padded with zeros to a power of two
// (adding +0.0 is exact). One CTA; nblocks <= kMaxBlocks.
__global__ void __launch_bounds__(1024) k_static_norm(DevScalars* sc, double* vsum,
                                                      unsigned long long nblocks, double two2,
                                                      double* out) {
  unsigned long long n = 1;
  while (n < nblocks) n <<= 1;
  for (unsigned long long i = nblocks + threadIdx.x; i < n; i += blockDim.x) vsum[i] = 0.0;
  __syncthreads();
  for (unsigned long long cnt = n; cnt > 1; cnt >>= 1) {
    const unsigned long long half = cnt >> 1;
    double v[64];  // half <= 32768 = 1024 threads x 32 pairs
    int k = 0;
    for (unsigned long long i = threadIdx.x; i < half && k < 64; i += blockDim.x, ++k)
      v[k] = __dadd_rn(vsum[2 * i], vsum[2 * i + 1]);
    __syncthreads();
    k = 0;
    for (unsigned long long i = threadIdx.x; i < half && k < 64; i += blockDim.x, ++k) vsum[i] = v[k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double V = vsum[0];
    const double Sd = __dadd_rn(__dmul_rn(__ull2double_rn(sc->acc.sq_hi), 18446744073709551616.0),
                                __ull2double_rn(sc->acc.sq_lo));
    *out = __dadd_rn(__dmul_rn(Sd, two2), V);
  }
}

}  // namespace

extern "C" int sv_codec_compress_static(const void* values, uint64_t nblocks, int bl, int dtype,
                                        double eb, void* out, uint64_t cap, uint64_t* offsets,
                                        uint32_t* lengths, void* stream, uint64_t* used,
                                        double* norm) {
  if (bl < 5 || bl > 12 || (dtype != SV_C64 && dtype != SV_C128) || !(eb > 0.0) || !std::isfinite(eb))
    return SV_ERR_ARG;
  if (nblocks > kMaxBlocks) return SV_ERR_UNSUPPORTED;
  if (nblocks && (!values || !out || !offsets || !lengths || ((uintptr_t)out & 15))) return SV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the call ends with a read-back and a stream synchronization, neither of which a capturing
  // stream accepts: refuse before enqueueing anything (an error here means the stream's
  // capture state could not be read, e.g. the legacy stream while another stream captures)
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap_st) != cudaSuccess) {
    cudaGetLastError();
    return SV_ERR_ARG;
  }
  if (cap_st != cudaStreamCaptureStatusNone) return SV_ERR_ARG;
  if (nblocks == 0) {  // nothing to compress (the same result as sv_codec_compress)
    if (used) *used = 0;
    if (norm) *norm = 0.0;
    return SV_OK;
  }
  void* base = nullptr;
  cudaError_t e = scratch_ptr(&base);
  if (e != cudaSuccess) return SV_ERR_CUDA;
  DevScalars* sc = (DevScalars*)base;
  double* vsum = (double*)((unsigned char*)base + kRecordBytes);
  double* nout = vsum + kMaxBlocks;
  QuantP qp;
  qp.eb = eb;
  qp.two = 2.0 * eb;
  qp.r = 1.0 / qp.two;
  // the record must start at zero (the previous call left its counters there)
  e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), st);
  if (e == cudaSuccess)
    e = launch_codec_compress(values, nblocks, bl, dtype == SV_C64 ? 1 : 2, qp, (uint8_t*)out, cap,
                              (unsigned long long*)offsets, lengths, sc, vsum, st);
  if (e == cudaSuccess) {
    k_static_norm<<<1, 1024, 0, st>>>(sc, vsum, nblocks, qp.two * qp.two, nout);
    e = cudaGetLastError();
  }
  DevScalars h;
  double hn = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hn, nout, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return SV_ERR_CUDA;
  if (used) *used = h.bump[0];
  if (norm) *norm = hn;
  if (h.status & kStInternal) return SV_ERR_INTERNAL;
  if (h.status & kStCorrupt) return SV_ERR_CORRUPT;
  if (h.status & kStVerbatim) return SV_ERR_UNSUPPORTED;
  if (h.status & kStOverflow) return SV_ERR_OOM;
  return SV_OK;
}
