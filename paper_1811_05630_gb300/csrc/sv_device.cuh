// sv_device.cuh — device-side block codec and helpers (sm_103a).
//
// The block codec is the SZ-style error-bounded compressor of Sec. II of Wu et al. (PMES
// 2018), restated for the GPU:
//   quantization  t = fl(v r), q = rint(t), x' = fl(q 2eb) (complex64: rounded to float);
//                 a value is stored verbatim when |t| >= 2^29 or |fl(v - x')| > eb;
//   prediction    1-D Lorenzo per plane on the integer codes (dual quantization): the
//                 delta of value j is q_j - q_{j-2} (re and im are interleaved), q_{-2} = 0;
//   symbols       delta + 32768 for |delta| <= 32767, else the escape symbol 0 followed by
//                 the 32-bit delta in the bit stream;
//   entropy code  canonical Huffman per block (two-queue construction, leaves ordered by
//                 (frequency, symbol), leaf first on ties), or PACK (zigzag deltas at a fixed
//                 width) when that is not larger, or CONST (header only) when every code of
//                 a plane is equal and nothing is verbatim.
// Every floating-point step uses the _rn intrinsics so that no multiply-add is contracted:
// the results are the IEEE results of the written operation order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sv {

// ---- format constants -----------------------------------------------------------------
constexpr int kHdr = 16;
constexpr int kRadius = 32767;
// Huffman symbols per stored chunk bit count (one decoding thread per chunk): a format
// parameter of the state, 16, 32 or 64
constexpr int kChunkDefault = 32, kChunkMin = 16;
constexpr int kHuffMaxD = 256;        // more distinct symbols: PACK
constexpr int kHashSlots = 512;       // >= 2 * kHuffMaxD
constexpr int kBinsMax = 2048;        // direct histogram bins (symbols 32768 +- 1024)
constexpr int kLutBits = 10;          // decode table width
constexpr int kVmax = 128;            // GPU limit: verbatim values per block
constexpr int kModeConst = 0, kModeHuff = 1, kModePack = 2;
constexpr int32_t kSentinel = INT32_MIN;  // q slot of a verbatim value
constexpr uint32_t kEmpty = 0xFFFFFFFFu;

// device status bits
constexpr uint32_t kStOverflow = 1u, kStCorrupt = 2u, kStNorm = 4u, kStVerbatim = 8u,
                   kStTimeout = 16u, kStInternal = 32u;

struct PassAcc {
  unsigned long long sq_lo, sq_hi;  // exact sum of q^2 (128-bit)
  unsigned long long n_verbatim, n_escape;
  unsigned long long modes[3];
  unsigned long long reused;  // blocks whose stream was re-emitted unchanged (pass-through)
};

struct DevScalars {
  unsigned long long bump[2];  // bytes used in arena 0 / 1
  PassAcc acc;                 // accumulated by the running pass
  PassAcc last;                // of the last finalized pass
  unsigned long long last_bytes;
  unsigned long long pass_index;
  unsigned long long io_bytes;   // compressed bytes read + written, summed over passes
  unsigned long long peak_bytes; // largest stored state (compressed bytes) since the reset
  double sigma;                // scale for the next pass, 1/sqrt(norm)
  double norm;                 // N of the current stored state
  unsigned int status;
  unsigned int fail_seq;
};

struct QuantP {
  double eb, two, r;
};

__host__ __device__ inline size_t pad_to(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---- quantization ---------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ Real dequant(int32_t q, const QuantP& p);
template <>
__device__ __forceinline__ double dequant<double>(int32_t q, const QuantP& p) {
  return __dmul_rn((double)q, p.two);
}
template <>
__device__ __forceinline__ float dequant<float>(int32_t q, const QuantP& p) {
  return __double2float_rn(__dmul_rn((double)q, p.two));
}

// true: verbatim. Otherwise *q receives the code.
template <typename Real>
__device__ __forceinline__ bool quantize(Real v, const QuantP& p, int32_t* q) {
  const double vd = (double)v;
  const double t = __dmul_rn(vd, p.r);
  if (!(fabs(t) < 536870912.0)) return true;
  const int32_t qq = __double2int_rn(t);
  const double xr = (double)dequant<Real>(qq, p);
  const double d = __dsub_rn(vd, xr);
  if (fabs(d) > p.eb) return true;
  *q = qq;
  return false;
}

template <typename Real>
struct RawBits;
template <>
struct RawBits<double> {
  __device__ static uint64_t to(double v) { return (uint64_t)__double_as_longlong(v); }
  __device__ static double from(uint64_t b) { return __longlong_as_double((long long)b); }
};
template <>
struct RawBits<float> {
  __device__ static uint64_t to(float v) { return (uint64_t)__float_as_uint(v); }
  __device__ static float from(uint64_t b) { return __uint_as_float((uint32_t)b); }
};

// ---- small block-level helpers --------------------------------------------------------
__device__ __forceinline__ uint32_t zigzag(int32_t d) {
  return d >= 0 ? (uint32_t)d << 1 : (((uint32_t)(-(int64_t)d)) << 1) - 1u;
}
__device__ __forceinline__ int32_t unzigzag(uint32_t z) {
  return (z & 1u) ? (int32_t)(-(int64_t)((z >> 1) + 1u)) : (int32_t)(z >> 1);
}
__device__ __forceinline__ int bit_width(uint32_t z) { return z ? 32 - __clz(z) : 0; }

__device__ __forceinline__ uint32_t hash_sym(uint32_t s) { return (s * 0x9E3779B1u) >> (32 - 11); }

// Block-wide exclusive scan of a 32-bit unsigned value. `ws` holds >= 33 words.
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t* ws, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < nw ? ws[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    ws[lane] = w;
  }
  __syncthreads();
  const uint32_t off = wid ? ws[wid - 1] : 0u;
  if (total) *total = ws[nw - 1];
  __syncthreads();
  return off + x - v;
}

// Block-wide exclusive scan of two int32 lanes (the two Lorenzo planes).
__device__ __forceinline__ int2 block_excl_scan_i2(int2 v, int2* ws) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int2 x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int yx = __shfl_up_sync(0xffffffffu, x.x, o);
    int yy = __shfl_up_sync(0xffffffffu, x.y, o);
    if (lane >= o) {
      x.x += yx;
      x.y += yy;
    }
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int2 w = lane < nw ? ws[lane] : make_int2(0, 0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int yx = __shfl_up_sync(0xffffffffu, w.x, o);
      int yy = __shfl_up_sync(0xffffffffu, w.y, o);
      if (lane >= o) {
        w.x += yx;
        w.y += yy;
      }
    }
    ws[lane] = w;
  }
  __syncthreads();
  int2 off = wid ? ws[wid - 1] : make_int2(0, 0);
  __syncthreads();
  return make_int2(off.x + x.x - v.x, off.y + x.y - v.y);
}

template <typename T>
__device__ __forceinline__ T block_reduce_max(T v, T* ws) {
  for (int o = 16; o > 0; o >>= 1) {
    T y = __shfl_xor_sync(0xffffffffu, v, o);
    v = v > y ? v : y;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    T w = lane < nw ? ws[lane] : (T)0;
    for (int o = 16; o > 0; o >>= 1) {
      T y = __shfl_xor_sync(0xffffffffu, w, o);
      w = w > y ? w : y;
    }
    if (lane == 0) ws[0] = w;
  }
  __syncthreads();
  T r = ws[0];
  __syncthreads();
  return r;
}

// Per-block statistics of a code block, reduced across the CTA with one pair of barriers:
// sums of the high/low 32-bit halves of q^2 and of escapes, maxima of zigzag(delta) and |q|,
// AND of the constant-block test. ws: one entry per warp (at most 8).
struct BlkStats {
  unsigned long long sqh, sql;
  uint32_t zmax, amax;
  int nesc, cst;
};

__device__ __forceinline__ void block_reduce_stats(BlkStats& v, BlkStats* ws) {
  for (int o = 16; o > 0; o >>= 1) {
    v.sqh += __shfl_xor_sync(0xffffffffu, v.sqh, o);
    v.sql += __shfl_xor_sync(0xffffffffu, v.sql, o);
    const uint32_t z = __shfl_xor_sync(0xffffffffu, v.zmax, o), a = __shfl_xor_sync(0xffffffffu, v.amax, o);
    v.zmax = z > v.zmax ? z : v.zmax;
    v.amax = a > v.amax ? a : v.amax;
    v.nesc += __shfl_xor_sync(0xffffffffu, v.nesc, o);
    v.cst &= __shfl_xor_sync(0xffffffffu, v.cst, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  BlkStats r = ws[0];
  for (int w = 1; w < nw; ++w) {
    const BlkStats& x = ws[w];
    r.sqh += x.sqh;
    r.sql += x.sql;
    r.zmax = x.zmax > r.zmax ? x.zmax : r.zmax;
    r.amax = x.amax > r.amax ? x.amax : r.amax;
    r.nesc += x.nesc;
    r.cst &= x.cst;
  }
  __syncthreads();
  v = r;
}

__device__ __forceinline__ unsigned long long block_reduce_sum_u64(unsigned long long v,
                                                                   unsigned long long* ws) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) ws[wid] = v;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < nw ? ws[lane] : 0ull;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if (lane == 0) ws[0] = w;
  }
  __syncthreads();
  unsigned long long r = ws[0];
  __syncthreads();
  return r;
}

// Bitonic sort of n (power of two) (key, val) pairs in shared memory, ascending by key.
inline __device__ __noinline__ void bitonic_sort(uint32_t* key, uint32_t* val, int n) {
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const uint32_t a = key[i], b = key[ixj];
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
            const uint32_t t = val[i];
            val[i] = val[ixj];
            val[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

// MSB-first bit writer into shared-memory words that were zeroed beforehand. The first
// and the last word a thread touches may be shared with its neighbours (atomicOr); the
// words strictly inside its range are plain stores.
struct BitWriter {
  uint32_t* w;
  uint32_t word;  // index of the word the accumulator maps to
  uint64_t acc;
  int nacc;       // bits in acc, counted from the MSB
  bool first;
  __device__ void start(uint32_t* words, uint32_t bitpos) {
    w = words;
    word = bitpos >> 5;
    nacc = (int)(bitpos & 31);
    acc = 0;
    first = true;
  }
  __device__ __forceinline__ void put(uint32_t val, int n) {  // 0 <= n <= 32
    if (n == 0) return;
    const uint64_t v = n == 32 ? (uint64_t)val : (uint64_t)(val & ((1u << n) - 1u));
    acc |= v << (64 - nacc - n);
    nacc += n;
    if (nacc >= 32) {
      const uint32_t hi = (uint32_t)(acc >> 32);
      if (first) {
        atomicOr(&w[word], hi);
        first = false;
      } else {
        w[word] = hi;
      }
      word++;
      acc <<= 32;
      nacc -= 32;
    }
  }
  __device__ void finish() {
    if (nacc > 0) atomicOr(&w[word], (uint32_t)(acc >> 32));
  }
};

// 32 stream bits starting at bit `pos` of a word array (zeros past `nwords`).
__device__ __forceinline__ uint32_t peek32(const uint32_t* w, uint64_t pos, uint32_t nwords) {
  const uint32_t i = (uint32_t)(pos >> 5), s = (uint32_t)(pos & 31);
  const uint32_t a = i < nwords ? __ldg(w + i) : 0u;
  if (s == 0) return a;
  const uint32_t b = i + 1 < nwords ? __ldg(w + i + 1) : 0u;
  return (a << s) | (b >> (32 - s));
}

}  // namespace sv
