// sv_kernels.cu — the kernels of libsv.so and their launchers.
//
//   k_pass            Algorithm 1, one gate pass over every block-group (Wu et al. PMES 2018)
//   k_vsum_tree       pairwise sum of the per-block verbatim squares (norm definition)
//   k_finalize        stored norm N and the next pass's scale sigma = 1/sqrt(N)
//   k_codec_*         the block codec on its own (Sec. II), same device code as k_pass
//   k_read_blocks     decoded amplitudes for measurements
//   k_plain_*         the plain (uncompressed) full amplitude-vector update (Sec. I)
#include "sv_internal.h"

namespace sv {

template <typename Real>
struct Arith;
template <>
struct Arith<double> {
  __device__ static double mul(double a, double b) { return __dmul_rn(a, b); }
  __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
};
template <>
struct Arith<float> {
  __device__ static float mul(float a, float b) { return __fmul_rn(a, b); }
  __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
};

template <typename Real>
__device__ __forceinline__ Real gate_coef(const PassArgs& a, int e);
template <>
__device__ __forceinline__ double gate_coef<double>(const PassArgs& a, int e) { return a.g[e]; }
template <>
__device__ __forceinline__ float gate_coef<float>(const PassArgs& a, int e) { return a.gf[e]; }

__device__ __forceinline__ unsigned long long insert_zero_bit(unsigned long long v, int p) {
  return ((v >> p) << (p + 1)) | (v & ((1ull << p) - 1ull));
}

// ---------------------------------------------------------------------------------------
// complex128 fast path. The exact step chain of a pass (x' = fl(q 2eb), y = fl(sigma x'),
// z = ordered sum of fl products, t = fl(z r), q' = rint(t)) lands within 2^-48 R Q of the
// real number T = sum c q with c = sigma G (2eb r) (R: largest row sum of |c|, Q = 2^29 the
// code limit). W below is T in fixed point with error at most 3 2^-F. Where W is farther
// than the sum of both bounds (plus 2^-21 for the verbatim test) from a rounding tie and
// inside the code range, rint(t) = round(W) and the value is not verbatim; otherwise that
// component is recomputed with the exact step chain. Results are identical either way.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int ceil_log2(double x) {
  const int e = ilogb(x);  // 2^e <= x < 2^(e+1)
  return scalbn(1.0, e) == x ? e : e + 1;
}

__device__ void fast_prepare(FastGate* fg, const PassArgs& a, double sigma) {
  const double s1 = __dmul_rn(a.use_sigma ? sigma : 1.0, a.two_r);
  const int K = a.K;
  double R = fabs(s1);
  if (a.apply_gate) {
    for (int jj = 0; jj < K; ++jj) {
      double row = 0.0;
      for (int m = 0; m < K; ++m)
        row += fabs(__dmul_rn(a.g[2 * (jj * K + m)], s1)) + fabs(__dmul_rn(a.g[2 * (jj * K + m) + 1], s1));
      R = row > R ? row : R;
    }
  }
  const int cl = R > 0.0 ? ceil_log2(R) : 0;
  int F = 30 - (cl > 0 ? cl : 0);
  if (!(R > 0.0) || cl > 16 || !isfinite(R)) F = -1;  // fast path off
  fg->F = F;
  if (F < 0) return;
  fg->margin = (long long)ceil(R * scalbn(1.0, F - 19)) + 3 + (1ll << (F > 21 ? F - 21 : 0));
  const double scale = scalbn(1.0, F + 31);
  auto fix = [&](double c, int32_t* hi, int32_t* lo) {
    const long long v = __double2ll_rn(__dmul_rn(c, scale));
    *hi = (int32_t)(v >> 31);
    *lo = (int32_t)(v & 0x7fffffffll);
  };
  fix(s1, &fg->idhi, &fg->idlo);
  // |q| <= qsafe gives rint of the exact chain for q * s1 equal to q: |q| |s1' - 1| plus the
  // chain's error (<= 2^-19 R here) stays below 1/2 - 2^-18 (s1' the exact scale, within
  // 2^-51 of s1)
  {
    const double dev = fabs(s1 - 1.0) + scalbn(1.0, -50);
    const double lim = (0.5 - scalbn(1.0, -18) - R * scalbn(1.0, -19)) / dev;
    fg->qsafe = lim >= 536870000.0 ? 536870000 : (lim > 0.0 ? (int)lim : -1);
  }
  for (int jj = 0; jj < 8; ++jj)
    for (int p = 0; p < 2; ++p) {
      fg->ssrc[jj][p] = -1;
      fg->ssgn[jj][p] = 1;
    }
  if (!a.apply_gate) return;
  for (int jj = 0; jj < K; ++jj) {
    int nz = 0, mz = -1;
    for (int m = 0; m < K; ++m)
      if (a.g[2 * (jj * K + m)] != 0.0 || a.g[2 * (jj * K + m) + 1] != 0.0) {
        ++nz;
        mz = m;
      }
    if (nz != 1) continue;
    const double gr = a.g[2 * (jj * K + mz)], gi = a.g[2 * (jj * K + mz) + 1];
    if (gi == 0.0 && (gr == 1.0 || gr == -1.0)) {  // (+-1) (x + iy)
      const int sg = gr > 0 ? 1 : -1;
      fg->ssrc[jj][0] = (int8_t)(2 * mz);
      fg->ssgn[jj][0] = (int8_t)sg;
      fg->ssrc[jj][1] = (int8_t)(2 * mz + 1);
      fg->ssgn[jj][1] = (int8_t)sg;
    } else if (gr == 0.0 && (gi == 1.0 || gi == -1.0)) {  // (+-i) (x + iy) = -+y +- ix
      const int sg = gi > 0 ? 1 : -1;
      fg->ssrc[jj][0] = (int8_t)(2 * mz + 1);
      fg->ssgn[jj][0] = (int8_t)-sg;
      fg->ssrc[jj][1] = (int8_t)(2 * mz);
      fg->ssgn[jj][1] = (int8_t)sg;
    }
  }
  int diag = 1;
  for (int jj = 0; jj < K; ++jj)
    for (int m = 0; m < K; ++m) {
      const double A = __dmul_rn(a.g[2 * (jj * K + m)], s1);
      const double Bc = __dmul_rn(a.g[2 * (jj * K + m) + 1], s1);
      if (m != jj && (A != 0.0 || Bc != 0.0)) diag = 0;
      // re += A q_re - B q_im ; im += B q_re + A q_im
      fix(A, &fg->chi[jj][0][m][0], &fg->clo[jj][0][m][0]);
      fix(-Bc, &fg->chi[jj][0][m][1], &fg->clo[jj][0][m][1]);
      fix(Bc, &fg->chi[jj][1][m][0], &fg->clo[jj][1][m][0]);
      fix(A, &fg->chi[jj][1][m][1], &fg->clo[jj][1][m][1]);
    }
  fg->diag = diag;
}

// round(W / 2^F) when it provably equals the exact chain's code; false otherwise
__device__ __forceinline__ bool fast_round(long long W, int F, long long margin, int32_t* q) {
  const long long half = 1ll << (F - 1);
  const long long qn = (W + half) >> F;
  const long long frac = W - (qn << F);
  if (frac < margin - half || frac >= half - margin) return false;
  if (qn >= (1ll << 29) - 1 || qn <= -((1ll << 29) - 1)) return false;
  *q = (int32_t)qn;
  return true;
}

// the exact step chain for one output component of a tuple (no verbatim input)
__device__ __forceinline__ double exact_component(const PassArgs& a, double sigma, const int32_t* qv,
                                                  int jj, int p, bool ctrl) {
  if (!ctrl) {
    const double x = __dmul_rn((double)qv[2 * jj + p], a.qp.two);
    return a.use_sigma ? __dmul_rn(sigma, x) : x;
  }
  double ar = 0.0, ai = 0.0;
  for (int m = 0; m < a.K; ++m) {
    double yr = __dmul_rn((double)qv[2 * m], a.qp.two), yi = __dmul_rn((double)qv[2 * m + 1], a.qp.two);
    if (a.use_sigma) {
      yr = __dmul_rn(sigma, yr);
      yi = __dmul_rn(sigma, yi);
    }
    const double gr = a.g[2 * (jj * a.K + m)], gi = a.g[2 * (jj * a.K + m) + 1];
    const double pr = __dsub_rn(__dmul_rn(gr, yr), __dmul_rn(gi, yi));
    const double pi = __dadd_rn(__dmul_rn(gr, yi), __dmul_rn(gi, yr));
    if (m == 0) {
      ar = pr;
      ai = pi;
    } else {
      ar = __dadd_rn(ar, pr);
      ai = __dadd_rn(ai, pi);
    }
  }
  return p ? ai : ar;
}

// One tuple through the exact step chain in the value type (verbatim inputs; complex64).
template <typename Real, int KM>
__device__ __forceinline__ void tuple_exact(Worker<Real>& w, const PassArgs& a, Real sg, int bp, bool ctrl) {
  using A = Arith<Real>;
  const Layout& L = w.L;
  Real yr[KM], yi[KM];
  int gs[KM], js[KM];
#pragma unroll
  for (int mm = 0; mm < KM; ++mm) {
    if (mm < a.K) {
      const int p = bp + a.pos_delta[mm];
      const int g = p / L.nv;
      const int j = p - g * L.nv;
      gs[mm] = g;
      js[mm] = j;
      const Real xr = w.value_at(g, j), xi = w.value_at(g, j + 1);
      yr[mm] = a.use_sigma ? A::mul(sg, xr) : xr;
      yi[mm] = a.use_sigma ? A::mul(sg, xi) : xi;
    }
  }
  if (ctrl) {
    Real zr[KM], zi[KM];
#pragma unroll
    for (int jj = 0; jj < KM; ++jj) {
      if (jj < a.K) {
        Real ar = 0, ai = 0;
#pragma unroll
        for (int mm = 0; mm < KM; ++mm) {
          if (mm < a.K) {
            const Real gr = gate_coef<Real>(a, 2 * (jj * a.K + mm));
            const Real gi = gate_coef<Real>(a, 2 * (jj * a.K + mm) + 1);
            const Real pr = A::sub(A::mul(gr, yr[mm]), A::mul(gi, yi[mm]));
            const Real pi = A::add(A::mul(gr, yi[mm]), A::mul(gi, yr[mm]));
            if (mm == 0) {
              ar = pr;
              ai = pi;
            } else {
              ar = A::add(ar, pr);
              ai = A::add(ai, pi);
            }
          }
        }
        zr[jj] = ar;
        zi[jj] = ai;
      }
    }
#pragma unroll
    for (int mm = 0; mm < KM; ++mm)
      if (mm < a.K) {
        yr[mm] = zr[mm];
        yi[mm] = zi[mm];
      }
  }
#pragma unroll
  for (int mm = 0; mm < KM; ++mm)
    if (mm < a.K) {
      w.put_value(gs[mm], js[mm], yr[mm]);
      w.put_value(gs[mm], js[mm] + 1, yi[mm]);
    }
}

// ---------------------------------------------------------------------------------------
// Algorithm 1: for the gate G, for every slice: Decompress, Normalize, GateComputation,
// Compress. One CTA per group of 2^h coupled blocks (grid-stride over the groups).
// ---------------------------------------------------------------------------------------
// One group of 2^h coupled blocks of one state: Decompress, Normalize + GateComputation,
// Compress (shared by the single-state and the batched pass kernels).
template <typename Real, int KM>
__device__ __forceinline__ void pass_group(Worker<Real>& w, const PassArgs& a, const FastGate* fg,
                                           double sigma, unsigned long long grp) {
  using A = Arith<Real>;
  const Layout& L = w.L;
  const Real sg = (Real)sigma;  // complex64: sigma rounded to float once
  const int B = L.nv / 2;
  constexpr bool kFast = sizeof(Real) == 8;
  unsigned long long base = grp;
  for (int l = 0; l < a.h; ++l) base = insert_zero_bit(base, a.high_pos[l]);
  unsigned long long blks[4];
  for (int g = 0; g < a.G; ++g) {
    unsigned long long bid = base;
    for (int l = 0; l < a.h; ++l)
      if ((g >> l) & 1) bid |= 1ull << a.slot_shift[l];
    blks[g] = bid;
  }
  __syncthreads();
  if (threadIdx.x < 4) w.vout_cnt[threadIdx.x] = 0;
  // ---- stream pass-through (complex128) ----
  // Block slot g keeps the codes of slot src (src = g where the gate acts as the identity on
  // it: the group's high controls are not all 1, or its rows are unit rows; another slot for
  // a +1 permutation across blocks) when that slot holds no verbatim value and every |q| is
  // within qsafe: then each output code equals its input code exactly (the same argument as
  // the single-term shortcut below), and the block's stream is the source stream.
  bool any_pt = false;
  if (kFast && a.pt_ok && fg->F >= 0) {
    if (threadIdx.x == 0) {
      const bool hc = ((blks[0] << a.b) & a.cmask_high) == a.cmask_high;
      unsigned int dmask = 0;
      int npt = 0;
      for (int g = 0; g < a.G; ++g) {
        int src = hc ? a.pt_src[g] : g;
        if (src >= 0) {
          const unsigned int mm = a.in_info[blks[src]].maxq_mode;
          if ((mm & 0x80000000u) || (long long)(mm & 0x1FFFFFFFu) > (long long)fg->qsafe) src = -1;
        }
        w.m->pt[g] = src;
        if (src >= 0) ++npt;
        else dmask |= hc ? a.need[g] : (1u << g);
      }
      w.m->dmask = dmask;
      w.m->npt = npt;
    }
    __syncthreads();
    any_pt = w.m->npt > 0;
    if (w.m->npt == a.G) {
      for (int g = 0; g < a.G; ++g) w.pass_through(blks[w.m->pt[g]], blks[g], a);
      return;
    }
  }
  // ---- Decompress(S) ----
  for (int g = 0; g < a.G; ++g) {
    if (a.input_basis) {
      const int pos = ((a.basis >> a.b) == blks[g]) ? 2 * (int)(a.basis & (unsigned long long)(B - 1)) : -1;
      w.load_basis(g, pos);
    } else if (any_pt && !((w.m->dmask >> g) & 1u)) {
      w.load_basis(g, -1);  // read by no recoded block: zeros
    } else {
      w.decode(g, a.in_arena + a.in_off[blks[g]], a.in_len[blks[g]]);
    }
  }
  // ---- Normalize(S) and GateComputation(G, S), tuple by tuple, in place ----
  const int ntup = B >> a.nlow;
  for (int u = threadIdx.x; u < ntup; u += blockDim.x) {
    unsigned long long o = (unsigned long long)u;
    for (int l = 0; l < a.nlow; ++l) o = insert_zero_bit(o, a.low_t[l]);
    const unsigned long long gidx = (blks[0] << a.b) | o;
    const bool ctrl = a.apply_gate && ((gidx & a.cmask) == a.cmask);
    const int bp = 2 * (int)o;
    if (kFast && fg->F >= 0) {
      int32_t qv[2 * KM];
      int gq[KM], jq[KM];
      bool sentinel = false;
#pragma unroll
      for (int mm = 0; mm < KM; ++mm)
        if (mm < a.K) {
          const int p = bp + a.pos_delta[mm];
          gq[mm] = p / L.nv;
          jq[mm] = p - gq[mm] * L.nv;
          qv[2 * mm] = w.q[p];
          qv[2 * mm + 1] = w.q[p + 1];
          sentinel |= qv[2 * mm] == kSentinel || qv[2 * mm + 1] == kSentinel;
        }
      if (!sentinel) {
        const int F = fg->F;
        const long long margin = fg->margin;
        int32_t out[2 * KM];
        unsigned int exact_mask = 0;
#pragma unroll
        for (int jj = 0; jj < KM; ++jj)
          if (jj < a.K) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              // outputs that are +-1 times one input: exact without arithmetic when small
              const int ssrc = ctrl ? fg->ssrc[jj][p] : 2 * jj + p;
              bool done = false;
              if (ssrc >= 0) {
                int32_t qq = 0;
#pragma unroll
                for (int e = 0; e < 2 * KM; ++e)
                  if (e == ssrc) qq = qv[e];
                if ((qq < 0 ? -qq : qq) <= fg->qsafe) {
                  out[2 * jj + p] = (ctrl && fg->ssgn[jj][p] < 0) ? -qq : qq;
                  done = true;
                }
              }
              if (!done) {
                long long sh = 0, sl = 0;
                if (ctrl && fg->diag) {
  #pragma unroll
                  for (int c = 0; c < 2; ++c) {
                    const long long qq = qv[2 * jj + c];
                    sh += qq * fg->chi[jj][p][jj][c];
                    sl += (qq * fg->clo[jj][p][jj][c]) >> 4;
                  }
                } else if (ctrl) {
  #pragma unroll
                  for (int m = 0; m < KM; ++m)
                    if (m < a.K) {
  #pragma unroll
                      for (int c = 0; c < 2; ++c) {
                        const long long qq = qv[2 * m + c];
                        sh += qq * fg->chi[jj][p][m][c];
                        sl += (qq * fg->clo[jj][p][m][c]) >> 4;
                      }
                    }
                } else {
                  const long long qq = qv[2 * jj + p];
                  sh = qq * fg->idhi;
                  sl = (qq * fg->idlo) >> 4;
                }
                if (!fast_round(sh + (sl >> 27), F, margin, &out[2 * jj + p])) exact_mask |= 1u << (2 * jj + p);
              }
            }
          }
        double zx[2 * KM];
        if (exact_mask) {
#pragma unroll
          for (int e = 0; e < 2 * KM; ++e)
            if ((exact_mask >> e) & 1u) zx[e] = exact_component(a, sigma, qv, e >> 1, e & 1, ctrl);
        }
#pragma unroll
        for (int mm = 0; mm < KM; ++mm)
          if (mm < a.K) {
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              const int e = 2 * mm + p;
              if ((exact_mask >> e) & 1u) w.put_value(gq[mm], jq[mm] + p, (Real)zx[e]);
              else w.q[gq[mm] * L.nv + jq[mm] + p] = out[e];
            }
          }
        continue;
      }
    }
    tuple_exact<Real, KM>(w, a, sg, bp, ctrl);
  }
  __syncthreads();
  // ---- Compress(S) ----
  for (int g = 0; g < a.G; ++g) {
    if (any_pt && w.m->pt[g] >= 0) w.pass_through(blks[w.m->pt[g]], blks[g], a);
    else w.encode(g, blks[g], a);
  }
}

template <typename Real, int KM>
__global__ void __launch_bounds__(256) k_pass(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(a.b, a.G, (int)sizeof(Real));
  Worker<Real> w;
  w.init(smem, L, a.b, a.qp);
  // A state poisoned by an earlier pass (or by another CTA of this one) is skipped. One
  // thread reads the flag so that the whole CTA takes the same branch.
  if (threadIdx.x == 0) {
    w.m->err = 0;
    w.m->live = *(volatile unsigned int*)&a.sc->status == 0;
  }
  __syncthreads();
  if (!w.m->live) return;
  const double sigma = a.use_sigma ? *(volatile double*)&a.sc->sigma : 1.0;
  FastGate* fg = (FastGate*)(smem + L.off_fast);
  if (sizeof(Real) == 8 && threadIdx.x == 0) fast_prepare(fg, a, sigma);  // visible after pass_group's barrier
  for (unsigned long long grp = blockIdx.x; grp < a.ngroups; grp += gridDim.x)
    pass_group<Real, KM>(w, a, fg, sigma, grp);
  if (threadIdx.x == 0 && w.m->err) {
    atomicOr(&a.sc->status, w.m->err);
    atomicMin(&a.sc->fail_seq, a.seq);
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
  const Layout L = make_layout(b, Gmax, (int)sizeof(Real));
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
                                       unsigned long long total_groups, int b, int Gmax, int threads,
                                       cudaStream_t st) {
  const Layout L = make_layout(b, Gmax, (int)sizeof(Real));
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_pass_batch<Real, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (L.total > 227 * 1024) return cudaErrorInvalidValue;
  const int T = threads_ok(b, threads) ? threads : worker_threads(b);
  unsigned long long grid = total_groups;
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  if (grid == 0) return cudaSuccess;
  k_pass_batch<Real, KM><<<(unsigned int)grid, T, L.total, st>>>(descs, gprefix, nstates, b, Gmax);
  return cudaGetLastError();
}

cudaError_t launch_pass_batch(const PassArgs* descs, const unsigned long long* gprefix, int nstates,
                              unsigned long long total_groups, int b, int Gmax, int Kmax, int dtype,
                              int threads, cudaStream_t st) {
  const unsigned long long tg = total_groups;
  if (dtype == 1) {
    if (Kmax <= 2) return launch_pass_batch_k<float, 2>(descs, gprefix, nstates, tg, b, Gmax, threads, st);
    if (Kmax <= 4) return launch_pass_batch_k<float, 4>(descs, gprefix, nstates, tg, b, Gmax, threads, st);
    return launch_pass_batch_k<float, 8>(descs, gprefix, nstates, tg, b, Gmax, threads, st);
  }
  if (Kmax <= 2) return launch_pass_batch_k<double, 2>(descs, gprefix, nstates, tg, b, Gmax, threads, st);
  if (Kmax <= 4) return launch_pass_batch_k<double, 4>(descs, gprefix, nstates, tg, b, Gmax, threads, st);
  return launch_pass_batch_k<double, 8>(descs, gprefix, nstates, tg, b, Gmax, threads, st);
}

template <typename Real, int KM>
static cudaError_t launch_pass_k(const PassArgs& a, cudaStream_t st) {
  const Layout L = make_layout(a.b, a.G, (int)sizeof(Real));
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_pass<Real, KM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (L.total > 227 * 1024) return cudaErrorInvalidValue;
  const int T = threads_ok(a.b, a.threads) ? a.threads : worker_threads(a.b);
  unsigned long long grid = a.ngroups;
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  k_pass<Real, KM><<<(unsigned int)grid, T, L.total, st>>>(a);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t launch_pass_t(const PassArgs& a, cudaStream_t st) {
  if (a.K <= 2) return launch_pass_k<Real, 2>(a, st);
  if (a.K <= 4) return launch_pass_k<Real, 4>(a, st);
  return launch_pass_k<Real, 8>(a, st);
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
__global__ void __launch_bounds__(1024) k_vsum_tree(const double* in, double* out,
                                                    unsigned long long chunk,
                                                    const DevScalars* sc) {
  if (sc->acc.n_verbatim == 0 || sc->status) return;
  __shared__ double s[2048];
  const unsigned long long base = (unsigned long long)blockIdx.x * chunk;
  for (unsigned long long i = threadIdx.x; i < chunk; i += blockDim.x) s[i] = in[base + i];
  __syncthreads();
  for (unsigned long long cnt = chunk; cnt > 1; cnt >>= 1) {
    double v = 0.0;
    const unsigned long long half = cnt >> 1;
    // chunk <= 2048 and blockDim == 1024: each thread owns at most one pair per level
    if (threadIdx.x < half) v = __dadd_rn(s[2 * threadIdx.x], s[2 * threadIdx.x + 1]);
    __syncthreads();
    if (threadIdx.x < half) s[threadIdx.x] = v;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s[0];
}

cudaError_t launch_vsum_tree(const double* vsum, unsigned long long n, double* scratch,
                             double* root, const DevScalars* sc, cudaStream_t st) {
  // scratch: ping-pong levels; the final value lands in root
  const double* in = vsum;
  double* bufs[2] = {scratch, scratch + (n / 2048 + 1)};
  int which = 0;
  while (true) {
    const unsigned long long chunk = n < 2048 ? n : 2048;
    const unsigned long long nblk = n / chunk;
    double* out = nblk == 1 ? root : bufs[which];
    k_vsum_tree<<<(unsigned int)nblk, 1024, 0, st>>>(in, out, chunk, sc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nblk == 1) break;
    in = out;
    which ^= 1;
    n = nblk;
  }
  return cudaSuccess;
}

__global__ void k_finalize(DevScalars* sc, const double* root, double two2, int reset_id,
                           unsigned int seq) {
  if (threadIdx.x != 0 || sc->status) return;
  const double V = sc->acc.n_verbatim ? *root : 0.0;
  const double Sd = __dadd_rn(__dmul_rn(__ull2double_rn(sc->acc.sq_hi), 18446744073709551616.0),
                              __ull2double_rn(sc->acc.sq_lo));
  const double N = __dadd_rn(__dmul_rn(Sd, two2), V);
  if (!(N > 0.0) || isinf(N)) {
    sc->status |= kStNorm;
    if (seq < sc->fail_seq) sc->fail_seq = seq;
    return;
  }
  sc->norm = N;
  sc->sigma = __ddiv_rn(1.0, __dsqrt_rn(N));
  sc->last = sc->acc;
  sc->last_bytes = sc->bump[reset_id ^ 1];
  sc->io_bytes += sc->bump[reset_id] + sc->bump[reset_id ^ 1];
  sc->acc.sq_lo = sc->acc.sq_hi = 0;
  sc->acc.n_verbatim = sc->acc.n_escape = 0;
  sc->acc.modes[0] = sc->acc.modes[1] = sc->acc.modes[2] = 0;
  sc->acc.reused = 0;
  sc->bump[reset_id] = 0;
  sc->pass_index++;
}

cudaError_t launch_finalize(DevScalars* sc, const double* root, double two2, int reset_id,
                            unsigned int seq, cudaStream_t st) {
  k_finalize<<<1, 32, 0, st>>>(sc, root, two2, reset_id, seq);
  return cudaGetLastError();
}

// Batched norm finalization: one CTA per state computes that state's pairwise verbatim sum
// (chunks of 2048 level by level, the same tree as the multi-launch version) when the pass
// stored a verbatim value; then one thread per state finalizes N and sigma.
__global__ void __launch_bounds__(1024) k_vsum_batch(const PassArgs* __restrict__ descs,
                                                     const double* const* __restrict__ trees,
                                                     const unsigned long long* __restrict__ nblocks) {
  const PassArgs& a = descs[blockIdx.x];
  if (a.sc->acc.n_verbatim == 0 || a.sc->status) return;
  __shared__ double sm[2048];
  double* tree = (double*)trees[blockIdx.x];
  const double* in = a.vsum;
  unsigned long long n = nblocks[blockIdx.x];
  double* bufs[2] = {tree, tree + (n / 2048 + 1)};
  int which = 0;
  double* out = bufs[0];
  while (true) {
    const unsigned long long chunk = n < 2048 ? n : 2048;
    const unsigned long long nch = n / chunk;
    out = bufs[which];
    for (unsigned long long c = 0; c < nch; ++c) {
      for (unsigned long long i = threadIdx.x; i < chunk; i += blockDim.x) sm[i] = in[c * chunk + i];
      __syncthreads();
      for (unsigned long long cnt = chunk; cnt > 1; cnt >>= 1) {
        const unsigned long long half = cnt >> 1;
        double v = 0.0;
        if (threadIdx.x < half) v = __dadd_rn(sm[2 * threadIdx.x], sm[2 * threadIdx.x + 1]);
        __syncthreads();
        if (threadIdx.x < half) sm[threadIdx.x] = v;
        __syncthreads();
      }
      if (threadIdx.x == 0) out[c] = sm[0];
      __syncthreads();
    }
    if (nch == 1) break;
    in = out;
    which ^= 1;
    n = nch;
  }
  if (threadIdx.x == 0) tree[0] = out[0];  // the root, wherever the last level left it
}

__global__ void k_finalize_batch(const PassArgs* __restrict__ descs, const double* const* __restrict__ trees,
                                 int nstates) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nstates) return;
  const PassArgs& a = descs[i];
  DevScalars* sc = a.sc;
  if (sc->status) return;
  const double V = sc->acc.n_verbatim ? trees[i][0] : 0.0;
  const double Sd = __dadd_rn(__dmul_rn(__ull2double_rn(sc->acc.sq_hi), 18446744073709551616.0),
                              __ull2double_rn(sc->acc.sq_lo));
  const double N = __dadd_rn(__dmul_rn(Sd, a.two2), V);
  if (!(N > 0.0) || isinf(N)) {
    sc->status |= kStNorm;
    if (a.seq < sc->fail_seq) sc->fail_seq = a.seq;
    return;
  }
  const int reset_id = a.out_id ^ 1;
  sc->norm = N;
  sc->sigma = __ddiv_rn(1.0, __dsqrt_rn(N));
  sc->last = sc->acc;
  sc->last_bytes = sc->bump[reset_id ^ 1];
  sc->io_bytes += sc->bump[reset_id] + sc->bump[reset_id ^ 1];
  sc->acc.sq_lo = sc->acc.sq_hi = 0;
  sc->acc.n_verbatim = sc->acc.n_escape = 0;
  sc->acc.modes[0] = sc->acc.modes[1] = sc->acc.modes[2] = 0;
  sc->acc.reused = 0;
  sc->bump[reset_id] = 0;
  sc->pass_index++;
}

cudaError_t launch_norm_batch(const PassArgs* descs, const double* const* trees, const unsigned long long* nblocks,
                              int nstates, cudaStream_t st) {
  k_vsum_batch<<<nstates, 1024, 0, st>>>(descs, trees, nblocks);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_finalize_batch<<<(nstates + 63) / 64, 64, 0, st>>>(descs, trees, nstates);
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
    if (threadIdx.x == 0) w.vout_cnt[0] = 0;
    for (int i = threadIdx.x; i < (L.nv >> 5); i += blockDim.x) w.vmask[i] = 0u;
    __syncthreads();
    const Real* v = values + blk * (unsigned long long)L.nv;
    for (int j = threadIdx.x; j < L.nv; j += blockDim.x) w.put_value(0, j, v[j]);
    __syncthreads();
    w.encode(0, blk, a);
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
struct PlainGate {
  int k, K, n;
  int tsorted[5];
  int delta_log[5];
  unsigned long long delta[32];
  unsigned long long cmask;
  double g[2 * 64];
};

template <typename Real>
__global__ void k_plain_gate(Real* psi, const PlainGate pg) {
  const unsigned long long ntup = (1ull << pg.n) >> pg.k;
  for (unsigned long long u = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; u < ntup;
       u += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long base = u;
    for (int l = 0; l < pg.k; ++l) base = insert_zero_bit(base, pg.tsorted[l]);
    if ((base & pg.cmask) != pg.cmask) continue;
    double yr[8], yi[8];
#pragma unroll
    for (int mm = 0; mm < 8; ++mm)
      if (mm < pg.K) {
        const unsigned long long i = base + pg.delta[mm];
        yr[mm] = (double)psi[2 * i];
        yi[mm] = (double)psi[2 * i + 1];
      }
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (jj < pg.K) {
        double ar = 0, ai = 0;
#pragma unroll
        for (int mm = 0; mm < 8; ++mm)
          if (mm < pg.K) {
            const double gr = pg.g[2 * (jj * pg.K + mm)], gi = pg.g[2 * (jj * pg.K + mm) + 1];
            ar = fma(gr, yr[mm], fma(-gi, yi[mm], ar));
            ai = fma(gr, yi[mm], fma(gi, yr[mm], ai));
          }
        const unsigned long long i = base + pg.delta[jj];
        psi[2 * i] = (Real)ar;
        psi[2 * i + 1] = (Real)ai;
      }
  }
}

// complex64 plain path keeps FP32 gate arithmetic
template <>
__global__ void k_plain_gate<float>(float* psi, const PlainGate pg) {
  const unsigned long long ntup = (1ull << pg.n) >> pg.k;
  for (unsigned long long u = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; u < ntup;
       u += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long base = u;
    for (int l = 0; l < pg.k; ++l) base = insert_zero_bit(base, pg.tsorted[l]);
    if ((base & pg.cmask) != pg.cmask) continue;
    float yr[8], yi[8];
#pragma unroll
    for (int mm = 0; mm < 8; ++mm)
      if (mm < pg.K) {
        const unsigned long long i = base + pg.delta[mm];
        yr[mm] = psi[2 * i];
        yi[mm] = psi[2 * i + 1];
      }
#pragma unroll
    for (int jj = 0; jj < 8; ++jj)
      if (jj < pg.K) {
        float ar = 0, ai = 0;
#pragma unroll
        for (int mm = 0; mm < 8; ++mm)
          if (mm < pg.K) {
            const float gr = (float)pg.g[2 * (jj * pg.K + mm)], gi = (float)pg.g[2 * (jj * pg.K + mm) + 1];
            ar = fmaf(gr, yr[mm], fmaf(-gi, yi[mm], ar));
            ai = fmaf(gr, yi[mm], fmaf(gi, yr[mm], ai));
          }
        const unsigned long long i = base + pg.delta[jj];
        psi[2 * i] = ar;
        psi[2 * i + 1] = ai;
      }
  }
}

cudaError_t launch_plain_gate(void* psi, int n, int dtype, const double* G, const int* targets,
                              int k, unsigned long long cmask, cudaStream_t st) {
  PlainGate pg;
  memset(&pg, 0, sizeof(pg));
  pg.k = k;
  pg.K = 1 << k;
  pg.n = n;
  pg.cmask = cmask;
  int ts[5];
  for (int l = 0; l < k; ++l) ts[l] = targets[l];
  for (int i = 0; i < k; ++i)
    for (int j = i + 1; j < k; ++j)
      if (ts[j] < ts[i]) {
        int t = ts[i];
        ts[i] = ts[j];
        ts[j] = t;
      }
  for (int l = 0; l < k; ++l) pg.tsorted[l] = ts[l];
  for (int mm = 0; mm < pg.K; ++mm) {
    unsigned long long d = 0;
    for (int l = 0; l < k; ++l)
      if ((mm >> l) & 1) d |= 1ull << targets[l];
    pg.delta[mm] = d;
  }
  for (int e = 0; e < 2 * pg.K * pg.K; ++e) pg.g[e] = G[e];
  const unsigned long long ntup = (1ull << n) >> k;
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

}  // namespace sv
