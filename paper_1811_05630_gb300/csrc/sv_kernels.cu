// sv_kernels.cu — the kernels of libsv.so and their launchers.
//
//   k_pass            Algorithm 1, one gate pass over every block-group (Wu et al. PMES 2018)
//   k_pass_batch      the same pass over the block-groups of many states
//   k_norm[_batch]    per state: the stored norm N and the next pass's scale sigma = 1/sqrt(N)
//                     (with the pairwise sum of the per-block verbatim squares)
//   k_codec_*         the block codec on its own (Sec. II), same device code as k_pass
//   k_read_blocks     decoded amplitudes for measurements
//   k_plain_*         the plain (uncompressed) full amplitude-vector update (Sec. I)
#include "../../include/sv.h"
#include "sv_internal.h"
#include "sv_pass.cuh"

namespace sv {

// N and sigma from the pass's accumulators (one thread); V the verbatim sum (0 without any).
// Loads bypass L1: the accumulators were written by other CTAs' atomics.
__device__ void finalize_state(DevScalars* sc, double V, double two2, int reset_id, unsigned int seq) {
  const unsigned long long sq_hi = __ldcg(&sc->acc.sq_hi), sq_lo = __ldcg(&sc->acc.sq_lo);
  const double Sd = __dadd_rn(__dmul_rn(__ull2double_rn(sq_hi), 18446744073709551616.0), __ull2double_rn(sq_lo));
  const double N = __dadd_rn(__dmul_rn(Sd, two2), V);
  if (!(N > 0.0) || isinf(N)) {
    sc->status |= kStNorm;
    if (seq < sc->fail_seq) sc->fail_seq = seq;
    return;
  }
  sc->norm = N;
  sc->sigma = __ddiv_rn(1.0, __dsqrt_rn(N));
  sc->last.sq_lo = sq_lo;
  sc->last.sq_hi = sq_hi;
  sc->last.n_verbatim = __ldcg(&sc->acc.n_verbatim);
  sc->last.n_escape = __ldcg(&sc->acc.n_escape);
  for (int i = 0; i < 3; ++i) sc->last.modes[i] = __ldcg(&sc->acc.modes[i]);
  sc->last.reused = __ldcg(&sc->acc.reused);
  const unsigned long long used_out = __ldcg(&sc->bump[reset_id ^ 1]), used_in = __ldcg(&sc->bump[reset_id]);
  sc->last_bytes = used_out;
  if (used_out > sc->peak_bytes) sc->peak_bytes = used_out;
  sc->io_bytes += used_in + used_out;
  sc->acc.sq_lo = sc->acc.sq_hi = 0;
  sc->acc.n_verbatim = sc->acc.n_escape = 0;
  sc->acc.modes[0] = sc->acc.modes[1] = sc->acc.modes[2] = 0;
  sc->acc.reused = 0;
  sc->bump[reset_id] = 0;
  sc->pass_index++;
}

// Level-by-level pairwise sum of n = 2^k doubles (the norm definition's verbatim sum) by one
// CTA: chunks of 256 through shared memory `sm`, chunk results into the global ping-pong
// buffers buf0/buf1 (n / 256 + 1 doubles each). Power-of-two chunks compose to the same tree.
__device__ double cta_pairwise_sum(const double* in, unsigned long long n, double* buf0, double* buf1, double* sm) {
  const int tid = threadIdx.x, T = blockDim.x;
  int which = 0;
  while (true) {
    const unsigned long long chunk = n < 256 ? n : 256, nchunks = n / chunk;
    double* out = which ? buf1 : buf0;
    for (unsigned long long c = 0; c < nchunks; ++c) {
      for (unsigned long long i = tid; i < chunk; i += T) sm[i] = __ldcg(in + c * chunk + i);
      __syncthreads();
      for (unsigned long long cnt = chunk; cnt > 1; cnt >>= 1) {
        const unsigned long long half = cnt >> 1;
        double v[4];
        int nv = 0;
        for (unsigned long long p = tid; p < half; p += T) v[nv++] = __dadd_rn(sm[2 * p], sm[2 * p + 1]);
        __syncthreads();
        nv = 0;
        for (unsigned long long p = tid; p < half; p += T) sm[p] = v[nv++];
        __syncthreads();
      }
      if (tid == 0) out[c] = sm[0];
      __syncthreads();
    }
    if (nchunks == 1) return __ldcg(out);
    in = out;
    n = nchunks;
    which ^= 1;
  }
}

// The same pass for a batch of states (one gate each; equal dtype and block size). Group g of
// the launch belongs to the state s with gprefix[s] <= g < gprefix[s+1]; a CTA copies that
// state's descriptor into shared memory when it reaches the state's first group.
template <typename Real, int KM>
__global__ void __launch_bounds__(256) k_pass_batch(const PassArgs* __restrict__ descs,
                                                    const unsigned long long* __restrict__ gprefix,
                                                    int nstates, int b, int Gmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(b, Gmax, (int)sizeof(Real), true);
  PassArgs* as = (PassArgs*)(smem + L.off_desc);
  Worker<Real> w;
  QuantP q0{0.0, 0.0, 0.0};
  w.init(smem, L, b, q0);
  FastGate* fg = (FastGate*)(smem + L.off_fast);
  const unsigned long long total = gprefix[nstates];
  int cur = -1;
  double sigma = 1.0;
  for (unsigned long long g = blockIdx.x; g < total; g += gridDim.x) {
    int lo = 0, hi = nstates;  // largest s with gprefix[s] <= g
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (gprefix[mid] <= g) lo = mid;
      else hi = mid;
    }
    if (lo != cur) {
      __syncthreads();
      if (cur >= 0 && threadIdx.x == 0 && w.m->err) {
        atomicOr(&as->sc->status, w.m->err);
        atomicMin(&as->sc->fail_seq, as->seq);
      }
      __syncthreads();
      const uint4* src = (const uint4*)(descs + lo);
      uint4* dst = (uint4*)as;
      for (int i = threadIdx.x; i < (int)(sizeof(PassArgs) / 16); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      if (threadIdx.x == 0) {
        w.m->err = 0;
        w.m->live = *(volatile unsigned int*)&as->sc->status == 0;
      }
      __syncthreads();
      cur = lo;
      w.qp = as->qp;
      w.kc = as->chunk ? as->chunk : kChunkDefault;
      sigma = as->use_sigma ? *(volatile double*)&as->sc->sigma : 1.0;
      if (w.m->live && sizeof(Real) == 8 && threadIdx.x == 0) fast_prepare(fg, *as, sigma);
    }
    if (!w.m->live) continue;
    pass_group<Real, KM>(w, *as, fg, sigma, g - gprefix[lo]);
  }
  __syncthreads();
  if (cur >= 0 && threadIdx.x == 0 && w.m->err) {
    atomicOr(&as->sc->status, w.m->err);
    atomicMin(&as->sc->fail_seq, as->seq);
  }
}

template <typename Real, int KM>
static cudaError_t launch_pass_batch_k(const PassArgs* descs, const unsigned long long* gprefix, int nstates,
                                       unsigned long long total_groups, int b, int Gmax, int threads, int chunk,
                                       cudaStream_t st) {
  const Layout L = make_layout(b, Gmax, (int)sizeof(Real), true);  // the kernel's layout
  static std::atomic<unsigned long long> configured{0};  // devices set up
  cudaError_t ce = once_per_device(configured, [] {
    return cudaFuncSetAttribute(k_pass_batch<Real, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  if (ce != cudaSuccess) return ce;
  if (L.total > 227 * 1024) return cudaErrorInvalidValue;
  const int T = threads_ok(b, threads) ? threads : worker_threads(b);
  if (!chunk_ok(b, chunk, T)) return cudaErrorInvalidValue;
  unsigned long long grid = total_groups;
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  if (grid == 0) return cudaSuccess;
  k_pass_batch<Real, KM><<<(unsigned int)grid, T, L.total, st>>>(descs, gprefix, nstates, b, Gmax);
  return cudaGetLastError();
}

cudaError_t launch_pass_batch(const PassArgs* descs, const unsigned long long* gprefix, int nstates,
                              unsigned long long total_groups, int b, int Gmax, int Kmax, int dtype,
                              int threads, int chunk, cudaStream_t st) {
  const unsigned long long tg = total_groups;
  const int c = chunk ? chunk : kChunkDefault;
  if (dtype == 1) {
    if (Kmax <= 2) return launch_pass_batch_k<float, 2>(descs, gprefix, nstates, tg, b, Gmax, threads, c, st);
    if (Kmax <= 4) return launch_pass_batch_k<float, 4>(descs, gprefix, nstates, tg, b, Gmax, threads, c, st);
    return launch_pass_batch_k<float, 8>(descs, gprefix, nstates, tg, b, Gmax, threads, c, st);
  }
  if (Kmax <= 2) return launch_pass_batch_k<double, 2>(descs, gprefix, nstates, tg, b, Gmax, threads, c, st);
  if (Kmax <= 4) return launch_pass_batch_k<double, 4>(descs, gprefix, nstates, tg, b, Gmax, threads, c, st);
  return launch_pass_batch_k<double, 8>(descs, gprefix, nstates, tg, b, Gmax, threads, c, st);
}

cudaError_t launch_pass(const PassArgs& a, int dtype, cudaStream_t st) {
  return dtype == 1 ? launch_pass_t<float>(a, st) : launch_pass_t<double>(a, st);
}

// ---------------------------------------------------------------------------------------
// Norm of the stored state (the reading of Normalize(S) in Algorithm 1: one global scale
// per pass from the exact norm of what is stored):
//   N = fl( fl(Sd * two2) + V ),  Sd = fl( fl((double)S_hi * 2^64) + (double)S_lo ),
//   V = level-by-level pairwise sum over blocks of the per-block verbatim sums.
// ---------------------------------------------------------------------------------------
// Norm finalization after a pass, one CTA per state: the level-by-level pairwise verbatim sum
// (only when the pass stored a verbatim value), then N and sigma by thread 0.
__device__ void norm_cta(DevScalars* sc, const double* vsum, unsigned long long nb, double* tree, double two2,
                         int out_id, unsigned int seq, double* sm) {
  __shared__ int live;
  __shared__ unsigned long long nverb;
  if (threadIdx.x == 0) {
    live = sc->status == 0;
    nverb = sc->acc.n_verbatim;
  }
  __syncthreads();
  if (!live) return;
  double V = 0.0;
  if (nverb > 0) V = cta_pairwise_sum(vsum, nb, tree, tree + (nb / 256 + 1), sm);
  if (threadIdx.x == 0) finalize_state(sc, V, two2, out_id ^ 1, seq);
}

__global__ void __launch_bounds__(256) k_norm(DevScalars* sc, const double* vsum, unsigned long long nb, double* tree,
                                              double two2, int out_id, unsigned int seq) {
  __shared__ double sm[256];
  norm_cta(sc, vsum, nb, tree, two2, out_id, seq, sm);
}

__global__ void __launch_bounds__(256) k_norm_batch(const PassArgs* __restrict__ descs) {
  __shared__ double sm[256];
  const PassArgs& a = descs[blockIdx.x];
  norm_cta(a.sc, a.vsum, a.ngroups << a.h, a.tree, a.two2, a.out_id, a.seq, sm);
}

cudaError_t launch_norm(DevScalars* sc, const double* vsum, unsigned long long nb, double* tree, double two2,
                        int out_id, unsigned int seq, cudaStream_t st) {
  k_norm<<<1, 256, 0, st>>>(sc, vsum, nb, tree, two2, out_id, seq);
  return cudaGetLastError();
}

cudaError_t launch_norm_batch(const PassArgs* descs, int nstates, cudaStream_t st) {
  k_norm_batch<<<nstates, 256, 0, st>>>(descs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Standalone codec: quantize raw values (Compress) / decode to raw values (Decompress).
// ---------------------------------------------------------------------------------------
template <typename Real>
__global__ void __launch_bounds__(256) k_codec_compress(const Real* values, PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(a.b, 1, (int)sizeof(Real));
  Worker<Real> w;
  w.init(smem, L, a.b, a.qp);
  if (threadIdx.x == 0) w.m->err = 0;
  for (unsigned long long blk = blockIdx.x; blk < a.ngroups; blk += gridDim.x) {
    __syncthreads();
    if (threadIdx.x == 0) {
      w.vout_cnt[0] = 0;
      w.m->vbig[0] = 0;
      w.m->any_big = 0;
      w.m->fix = 0;
    }
    for (int i = threadIdx.x; i < (L.nv >> 5); i += blockDim.x) {
      w.vmask[i] = 0u;
      w.vomask[i] = 0u;
    }
    __syncthreads();
    const Real* v = values + blk * (unsigned long long)L.nv;
    for (int j = threadIdx.x; j < L.nv; j += blockDim.x) w.put_value(0, j, v[j]);
    __syncthreads();
    w.encode(0, blk, a);
    if (w.m->any_big) {  // complex128 with many verbatim values: raw values, then their sum
      w.prepare_out_ranks(0);
      if (threadIdx.x == 0) w.m->fix = 1;
      __syncthreads();
      for (int j = threadIdx.x; j < L.nv; j += blockDim.x) w.put_value(0, j, v[j]);
      __syncthreads();
      const double vs = w.verbatim_square_tree(0);
      if (threadIdx.x == 0 && a.vsum) a.vsum[blk] = vs;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && w.m->err) atomicOr(&a.sc->status, w.m->err);
}

template <typename Real>
__global__ void __launch_bounds__(256) k_codec_decompress(Real* values, PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(a.b, 1, (int)sizeof(Real));
  Worker<Real> w;
  w.init(smem, L, a.b, a.qp);
  if (threadIdx.x == 0) w.m->err = 0;
  for (unsigned long long blk = blockIdx.x; blk < a.ngroups; blk += gridDim.x) {
    __syncthreads();
    w.decode(0, a.in_arena + a.in_off[blk], a.in_len[blk]);
    Real* v = values + blk * (unsigned long long)L.nv;
    for (int j = threadIdx.x; j < L.nv; j += blockDim.x) v[j] = w.value_at(0, j);
  }
  if (threadIdx.x == 0 && w.m->err) atomicOr(&a.sc->status, w.m->err);
}

template <typename Real>
__global__ void __launch_bounds__(256) k_read_blocks(PassArgs a, unsigned long long b0,
                                                     double* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(a.b, 1, (int)sizeof(Real));
  Worker<Real> w;
  w.init(smem, L, a.b, a.qp);
  if (threadIdx.x == 0) w.m->err = 0;
  for (unsigned long long i = blockIdx.x; i < a.ngroups; i += gridDim.x) {
    __syncthreads();
    const unsigned long long blk = b0 + i;
    w.decode(0, a.in_arena + a.in_off[blk], a.in_len[blk]);
    double* o = out + i * (unsigned long long)L.nv;
    for (int j = threadIdx.x; j < L.nv; j += blockDim.x) o[j] = (double)w.value_at(0, j);
  }
  if (threadIdx.x == 0 && w.m->err) atomicOr(&a.sc->status, w.m->err);
}

template <typename Real, typename K>
static cudaError_t launch_worker(K kern, int b, unsigned long long n, cudaStream_t st,
                                 const PassArgs& a, int* smem_out) {
  const Layout L = make_layout(b, 1, (int)sizeof(Real));
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
  if (e != cudaSuccess) return e;
  *smem_out = (int)L.total;
  (void)a;
  (void)n;
  (void)st;
  return cudaSuccess;
}

static PassArgs codec_args(int b, QuantP qp, unsigned long long nblocks, DevScalars* sc) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.b = b;
  a.nv = 2 << b;
  a.G = 1;
  a.K = 1;
  a.qp = qp;
  a.ngroups = nblocks;
  a.sc = sc;
  a.out_id = 0;
  return a;
}

static unsigned int grid_for(unsigned long long n) {
  const unsigned long long cap = 152ull * 64ull;
  return (unsigned int)(n < cap ? n : cap);
}

cudaError_t launch_codec_compress(const void* values, unsigned long long nblocks, int b,
                                  int dtype, QuantP qp, uint8_t* out, unsigned long long cap,
                                  unsigned long long* offsets, unsigned int* lengths,
                                  DevScalars* sc, double* vsum, cudaStream_t st) {
  PassArgs a = codec_args(b, qp, nblocks, sc);
  a.out_arena = out;
  a.out_cap = cap;
  a.out_off = offsets;
  a.out_len = lengths;
  a.vsum = vsum;
  int smem = 0;
  const int T = worker_threads(b);
  cudaError_t e;
  if (dtype == 1) {
    e = launch_worker<float>(k_codec_compress<float>, b, nblocks, st, a, &smem);
    if (e == cudaSuccess) k_codec_compress<float><<<grid_for(nblocks), T, smem, st>>>((const float*)values, a);
  } else {
    e = launch_worker<double>(k_codec_compress<double>, b, nblocks, st, a, &smem);
    if (e == cudaSuccess) k_codec_compress<double><<<grid_for(nblocks), T, smem, st>>>((const double*)values, a);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_codec_decompress(const uint8_t* in, const unsigned long long* offsets,
                                    const unsigned int* lengths, unsigned long long nblocks,
                                    int b, int dtype, QuantP qp, void* values, DevScalars* sc,
                                    cudaStream_t st) {
  PassArgs a = codec_args(b, qp, nblocks, sc);
  a.in_arena = in;
  a.in_off = offsets;
  a.in_len = lengths;
  int smem = 0;
  const int T = worker_threads(b);
  cudaError_t e;
  if (dtype == 1) {
    e = launch_worker<float>(k_codec_decompress<float>, b, nblocks, st, a, &smem);
    if (e == cudaSuccess) k_codec_decompress<float><<<grid_for(nblocks), T, smem, st>>>((float*)values, a);
  } else {
    e = launch_worker<double>(k_codec_decompress<double>, b, nblocks, st, a, &smem);
    if (e == cudaSuccess) k_codec_decompress<double><<<grid_for(nblocks), T, smem, st>>>((double*)values, a);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_read_blocks(const uint8_t* arena, const unsigned long long* offs,
                               const unsigned int* lens, unsigned long long b0,
                               unsigned long long nb, int b, int dtype, QuantP qp,
                               double* out, DevScalars* sc, cudaStream_t st) {
  PassArgs a = codec_args(b, qp, nb, sc);
  a.in_arena = arena;
  a.in_off = offs;
  a.in_len = lens;
  int smem = 0;
  const int T = worker_threads(b);
  cudaError_t e;
  if (dtype == 1) {
    e = launch_worker<float>(k_read_blocks<float>, b, nb, st, a, &smem);
    if (e == cudaSuccess) k_read_blocks<float><<<grid_for(nb), T, smem, st>>>(a, b0, out);
  } else {
    e = launch_worker<double>(k_read_blocks<double>, b, nb, st, a, &smem);
    if (e == cudaSuccess) k_read_blocks<double><<<grid_for(nb), T, smem, st>>>(a, b0, out);
  }
  return e != cudaSuccess ? e : cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Reductions over decoded FP64 chunks (measurements; not on the gate path).
// ---------------------------------------------------------------------------------------
__global__ void k_probs_chunk(const double* amp, unsigned long long start, unsigned long long count,
                              const int* qubits, int m, double* bins) {
  extern __shared__ double sb[];
  const int nb = 1 << m;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) sb[i] = 0.0;
  __syncthreads();
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long gi = start + i;
    int v = 0;
    for (int l = 0; l < m; ++l) v |= (int)((gi >> qubits[l]) & 1ull) << l;
    const double re = amp[2 * i], im = amp[2 * i + 1];
    atomicAdd(&sb[v], re * re + im * im);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x)
    if (sb[i] != 0.0) atomicAdd(&bins[i], sb[i]);
}

cudaError_t launch_probs_chunk(const double* amp, unsigned long long start,
                               unsigned long long count, const int* qubits_dev, int m,
                               double* bins, cudaStream_t st) {
  const size_t smem = sizeof(double) << m;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_probs_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  unsigned long long blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) blocks = 1;
  k_probs_chunk<<<(unsigned int)blocks, 256, smem, st>>>(amp, start, count, qubits_dev, m, bins);
  return cudaGetLastError();
}

__global__ void k_dot_chunk(const double* a, const double* b, unsigned long long count,
                            double* acc) {
  double s[4] = {0, 0, 0, 0};
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const double ar = a[2 * i], ai = a[2 * i + 1], br = b[2 * i], bi = b[2 * i + 1];
    s[0] += ar * br + ai * bi;  // re <a|b>
    s[1] += ar * bi - ai * br;  // im <a|b>
    s[2] += ar * ar + ai * ai;
    s[3] += br * br + bi * bi;
  }
  for (int k = 0; k < 4; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], v);
  }
}

cudaError_t launch_dot_chunk(const double* a, const double* b, unsigned long long count,
                             double* acc4, cudaStream_t st) {
  unsigned long long blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) blocks = 1;
  k_dot_chunk<<<(unsigned int)blocks, 256, 0, st>>>(a, b, count, acc4);
  return cudaGetLastError();
}

// Overlap with the QFT of a basis state, 2^{-n/2} exp(2 pi i (x y mod 2^n) / 2^n) (the
// closed form the exact simulator reaches): acc[0..1] += conj(ref) . psi, acc[2] += |psi|^2.
__global__ void k_qft_overlap_chunk(const double* amp, unsigned long long start, unsigned long long count,
                                    unsigned long long x, int n, double* acc) {
  double s[3] = {0, 0, 0};
  const unsigned long long mask = n >= 64 ? ~0ull : ((1ull << n) - 1ull);
  const double inv_half = 1.0 / (double)(1ull << (n - 1));  // exact power of two
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < count;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long y = start + i;
    const unsigned long long t = (x * y) & mask;  // x y mod 2^n (the low n bits of the product)
    double sn, cs;
    sincospi((double)t * inv_half, &sn, &cs);
    const double pr = amp[2 * i], pi = amp[2 * i + 1];
    s[0] += cs * pr + sn * pi;
    s[1] += cs * pi - sn * pr;
    s[2] += pr * pr + pi * pi;
  }
  for (int k = 0; k < 3; ++k) {
    double v = s[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], v);
  }
}

cudaError_t launch_qft_overlap_chunk(const double* amp, unsigned long long start, unsigned long long count,
                                     unsigned long long x, int n, double* acc, cudaStream_t st) {
  unsigned long long blocks = (count + 255) / 256;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) blocks = 1;
  k_qft_overlap_chunk<<<(unsigned int)blocks, 256, 0, st>>>(amp, start, count, x, n, acc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Plain path: the full amplitude vector updated in place (the comparison baseline).
// ---------------------------------------------------------------------------------------
// The gate acts on tuples whose control bits are all 1: the launch enumerates exactly those
// (free bits = all bits but targets and controls), so no thread idles on a skipped tuple.
// Three forms: a diagonal gate touches only the members whose entry is not exactly 1; a
// permutation (unit rows, coefficient exactly 1) moves values without arithmetic; a real
// matrix multiplies both components by real coefficients; any other gate is the dense complex
// matrix-vector product (FMA).
struct PlainGate {
  int k, K, n, nfix;
  int fixsorted[40];                // target and control bits, ascending
  unsigned long long cmask;
  int form;                         // 0 dense, 1 diagonal, 2 permutation, 3 real dense
  int nm;                           // diagonal / permutation: members touched
  int mem[32];                      // their member indices
  int src[32];                      // permutation: source member of each touched member
  unsigned long long delta[32];     // member offset (target bits) from the tuple base
  double g[2 * 64];
};

__device__ __forceinline__ unsigned long long plain_base(unsigned long long u, const PlainGate& pg) {
  for (int l = 0; l < pg.nfix; ++l) u = insert_zero_bit(u, pg.fixsorted[l]);
  return u | pg.cmask;
}

template <typename Real>
__device__ __forceinline__ Real pfma(Real a, Real b, Real c);
template <>
__device__ __forceinline__ double pfma<double>(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float pfma<float>(float a, float b, float c) { return fmaf(a, b, c); }

template <typename Real>
__global__ void k_plain_gate(Real* psi, const PlainGate pg) {
  const unsigned long long ntup = 1ull << (pg.n - pg.nfix);
  for (unsigned long long u = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; u < ntup;
       u += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long base = plain_base(u, pg);
    if (pg.form == 1) {
      for (int j = 0; j < pg.nm; ++j) {
        const int m = pg.mem[j];
        const unsigned long long i = base + pg.delta[m];
        const Real dr = (Real)pg.g[2 * (m * pg.K + m)], di = (Real)pg.g[2 * (m * pg.K + m) + 1];
        const Real xr = psi[2 * i], xi = psi[2 * i + 1];
        psi[2 * i] = pfma<Real>(dr, xr, -di * xi);
        psi[2 * i + 1] = pfma<Real>(dr, xi, di * xr);
      }
      continue;
    }
    Real yr[8], yi[8];
    if (pg.form == 2) {
      for (int j = 0; j < pg.nm; ++j) {
        const unsigned long long i = base + pg.delta[pg.src[j]];
        yr[j] = psi[2 * i];
        yi[j] = psi[2 * i + 1];
      }
      for (int j = 0; j < pg.nm; ++j) {
        const unsigned long long i = base + pg.delta[pg.mem[j]];
        psi[2 * i] = yr[j];
        psi[2 * i + 1] = yi[j];
      }
      continue;
    }
#pragma unroll
    for (int mm = 0; mm < 8; ++mm)
      if (mm < pg.K) {
        const unsigned long long i = base + pg.delta[mm];
        yr[mm] = psi[2 * i];
        yi[mm] = psi[2 * i + 1];
      }
    if (pg.form == 3) {  // real matrix (H, real rotations): half the multiply-adds
#pragma unroll
      for (int jj = 0; jj < 8; ++jj)
        if (jj < pg.K) {
          Real ar = 0, ai = 0;
#pragma unroll
          for (int mm = 0; mm < 8; ++mm)
            if (mm < pg.K) {
              const Real gr = (Real)pg.g[2 * (jj * pg.K + mm)];
              ar = pfma<Real>(gr, yr[mm], ar);
              ai = pfma<Real>(gr, yi[mm], ai);
            }
          const unsigned long long i = base + pg.delta[jj];
          psi[2 * i] = ar;
          psi[2 * i + 1] = ai;
        }
      continue;
    }
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (jj < pg.K) {
        Real ar = 0, ai = 0;
#pragma unroll
        for (int mm = 0; mm < 8; ++mm)
          if (mm < pg.K) {
            const Real gr = (Real)pg.g[2 * (jj * pg.K + mm)], gi = (Real)pg.g[2 * (jj * pg.K + mm) + 1];
            ar = pfma<Real>(gr, yr[mm], pfma<Real>(-gi, yi[mm], ar));
            ai = pfma<Real>(gr, yi[mm], pfma<Real>(gi, yr[mm], ai));
          }
        const unsigned long long i = base + pg.delta[jj];
        psi[2 * i] = ar;
        psi[2 * i + 1] = ai;
      }
  }
}

// 4- and 5-qubit gates (K = 16 or 32) on the plain vector: K lanes of a warp own the K
// members of one tuple; each lane loads its member, the members are exchanged by shuffles (so
// every input is read before any lane writes), and lane j computes output row j from the matrix
// kept in shared memory in transposed order (lanes read consecutive entries).
template <typename Real>
__global__ void __launch_bounds__(256) k_plain_gate_big(Real* psi, const PlainGate pg, const double* __restrict__ G) {
  __shared__ Real gs[2 * 32 * 32];
  const int K = pg.K;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int j = e / K, m = e % K;
    gs[2 * (m * K + j)] = (Real)G[2 * e];
    gs[2 * (m * K + j) + 1] = (Real)G[2 * e + 1];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, j = lane % K, lead = lane - j;
  const int tpw = 32 / K;
  const unsigned long long ntup = 1ull << (pg.n - pg.nfix);
  const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
  for (unsigned long long u0 = warp * tpw; u0 < ntup; u0 += nwarps * tpw) {
    const unsigned long long u = u0 + (unsigned long long)(lane / K);
    const bool valid = u < ntup;
    unsigned long long i = 0;
    Real yr = 0, yi = 0;
    if (valid) {
      i = plain_base(u, pg) + pg.delta[j];
      yr = psi[2 * i];
      yi = psi[2 * i + 1];
    }
    Real ar = 0, ai = 0;
    for (int m = 0; m < K; ++m) {
      const Real xr = __shfl_sync(0xffffffffu, yr, lead + m), xi = __shfl_sync(0xffffffffu, yi, lead + m);
      const Real gr = gs[2 * (m * K + j)], gi = gs[2 * (m * K + j) + 1];
      ar = pfma<Real>(gr, xr, pfma<Real>(-gi, xi, ar));
      ai = pfma<Real>(gr, xi, pfma<Real>(gi, xr, ai));
    }
    if (valid) {
      psi[2 * i] = ar;
      psi[2 * i + 1] = ai;
    }
  }
}

cudaError_t launch_plain_gate(void* psi, int n, int dtype, const double* G, const int* targets,
                              int k, unsigned long long cmask, const double* G_dev, cudaStream_t st) {
  PlainGate pg;
  memset(&pg, 0, sizeof(pg));
  pg.k = k;
  pg.K = 1 << k;
  pg.n = n;
  pg.cmask = cmask;
  unsigned long long fix = cmask;
  for (int l = 0; l < k; ++l) fix |= 1ull << targets[l];
  for (int q = 0; q < n; ++q)
    if ((fix >> q) & 1ull) pg.fixsorted[pg.nfix++] = q;
  for (int mm = 0; mm < pg.K; ++mm) {
    unsigned long long d = 0;
    for (int l = 0; l < k; ++l)
      if ((mm >> l) & 1) d |= 1ull << targets[l];
    pg.delta[mm] = d;
  }
  if (k > 3) {  // the matrix is read from G_dev
    const unsigned long long ntup = 1ull << (n - pg.nfix);
    const unsigned long long warps = (ntup * pg.K + 31) / 32;
    unsigned long long blocks = (warps + 7) / 8;
    if (blocks > 152ull * 8) blocks = 152ull * 8;
    if (blocks == 0) blocks = 1;
    if (dtype == 1) k_plain_gate_big<float><<<(unsigned int)blocks, 256, 0, st>>>((float*)psi, pg, G_dev);
    else k_plain_gate_big<double><<<(unsigned int)blocks, 256, 0, st>>>((double*)psi, pg, G_dev);
    return cudaGetLastError();
  }
  for (int e = 0; e < 2 * pg.K * pg.K; ++e) pg.g[e] = G[e];
  // classify: diagonal, permutation (unit rows with coefficient exactly 1), or dense
  bool diag = true, perm = true;
  int src[32];
  for (int j = 0; j < pg.K; ++j) {
    int nz = 0;
    src[j] = -1;
    for (int m = 0; m < pg.K; ++m) {
      const double gr = G[2 * (j * pg.K + m)], gi = G[2 * (j * pg.K + m) + 1];
      if (gr != 0.0 || gi != 0.0) {
        ++nz;
        if (m != j) diag = false;
        if (gr == 1.0 && gi == 0.0) src[j] = m;
        else perm = false;
      }
    }
    if (nz != 1) perm = false;
  }
  if (diag) {
    pg.form = 1;
    for (int m = 0; m < pg.K; ++m)
      if (!(G[2 * (m * pg.K + m)] == 1.0 && G[2 * (m * pg.K + m) + 1] == 0.0)) pg.mem[pg.nm++] = m;
    if (pg.nm == 0) return cudaSuccess;  // the identity
  } else if (perm) {
    pg.form = 2;
    for (int j = 0; j < pg.K; ++j)
      if (src[j] != j) {
        pg.mem[pg.nm] = j;
        pg.src[pg.nm] = src[j];
        ++pg.nm;
      }
  } else {
    bool real = true;
    for (int e = 0; e < pg.K * pg.K; ++e) real = real && G[2 * e + 1] == 0.0;
    if (real) pg.form = 3;
  }
  const unsigned long long ntup = 1ull << (n - pg.nfix);
  unsigned long long blocks = (ntup + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  if (blocks == 0) blocks = 1;
  if (dtype == 1) k_plain_gate<float><<<(unsigned int)blocks, 256, 0, st>>>((float*)psi, pg);
  else k_plain_gate<double><<<(unsigned int)blocks, 256, 0, st>>>((double*)psi, pg);
  return cudaGetLastError();
}

template <typename Real>
__global__ void k_plain_basis(Real* psi, unsigned long long dim, unsigned long long index) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < dim;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    psi[2 * i] = (Real)(i == index ? 1.0 : 0.0);
    psi[2 * i + 1] = (Real)0.0;
  }
}

cudaError_t launch_plain_basis(void* psi, int n, int dtype, unsigned long long index,
                               cudaStream_t st) {
  const unsigned long long dim = 1ull << n;
  unsigned long long blocks = (dim + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  if (dtype == 1) k_plain_basis<float><<<(unsigned int)blocks, 256, 0, st>>>((float*)psi, dim, index);
  else k_plain_basis<double><<<(unsigned int)blocks, 256, 0, st>>>((double*)psi, dim, index);
  return cudaGetLastError();
}

template <typename Real>
__global__ void k_plain_read(const Real* psi, unsigned long long start, unsigned long long count,
                             double* out) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < 2 * count;
       i += (unsigned long long)gridDim.x * blockDim.x)
    out[i] = (double)psi[2 * start + i];
}

cudaError_t launch_plain_read(const void* psi, int dtype, unsigned long long start,
                              unsigned long long count, double* out, cudaStream_t st) {
  unsigned long long blocks = (2 * count + 255) / 256;
  if (blocks > 152ull * 16) blocks = 152ull * 16;
  if (blocks == 0) blocks = 1;
  if (dtype == 1) k_plain_read<float><<<(unsigned int)blocks, 256, 0, st>>>((const float*)psi, start, count, out);
  else k_plain_read<double><<<(unsigned int)blocks, 256, 0, st>>>((const double*)psi, start, count, out);
  return cudaGetLastError();
}

// Self-check of the bounded device wait: one thread initializes an mbarrier that expects one
// arrival, which nothing makes, and waits for its first phase with the tensor-core pass's
// wait, at most `polls` times. Status 2: the wait gave up, as it must; 1: the phase completed.
static __device__ unsigned int g_wait_status;

__global__ void k_wait_check(long long polls) {
  __shared__ unsigned long long mbar;
  if (threadIdx.x == 0) {
    tc_mbar_init(&mbar);
    g_wait_status = tc_wait_bounded(&mbar, 0u, polls) ? 1u : 2u;
  }
}

}  // namespace sv

int sv_check_bounded_wait(long long polls, void* stream, int* timed_out) {
  if (!timed_out || polls < 1 || polls > sv::kTcWaitLimit) return SV_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned int zero = 0;
  cudaError_t e = cudaMemcpyToSymbolAsync(sv::g_wait_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    sv::k_wait_check<<<1, 32, 0, st>>>(polls);
    e = cudaGetLastError();
  }
  unsigned int status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyFromSymbolAsync(&status, sv::g_wait_status, sizeof(status), 0, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return SV_ERR_CUDA;
  if (status != 1u && status != 2u) return SV_ERR_INTERNAL;
  *timed_out = status == 2u;
  return SV_OK;
}
