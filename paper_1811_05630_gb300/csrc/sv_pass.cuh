// sv_pass.cuh — the fused gate pass (Algorithm 1 of Wu et al., PMES 2018): gate arithmetic,
// the complex128 fixed-point path, stream pass-through and the k_pass kernel. Included by the
// translation units that instantiate k_pass (with and without a register cap).
#pragma once
#include "sv_internal.h"
#include "sv_tc.cuh"

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

__device__ inline void fast_prepare(FastGate* fg, const PassArgs& a, double sigma) {
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
  int diag = 1, real = 1;
  for (int jj = 0; jj < K; ++jj)
    for (int m = 0; m < K; ++m) {
      const double A = __dmul_rn(a.g[2 * (jj * K + m)], s1);
      const double Bc = __dmul_rn(a.g[2 * (jj * K + m) + 1], s1);
      if (m != jj && (A != 0.0 || Bc != 0.0)) diag = 0;
      if (Bc != 0.0) real = 0;
      // re += A q_re - B q_im ; im += B q_re + A q_im
      fix(A, &fg->chi[jj][0][m][0], &fg->clo[jj][0][m][0]);
      fix(-Bc, &fg->chi[jj][0][m][1], &fg->clo[jj][0][m][1]);
      fix(Bc, &fg->chi[jj][1][m][0], &fg->clo[jj][1][m][0]);
      fix(A, &fg->chi[jj][1][m][1], &fg->clo[jj][1][m][1]);
    }
  fg->diag = diag;
  fg->real = real;
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

// the exact step chain for one output component of a tuple (no verbatim input). The member
// loop is unrolled to KM with a guard so that the caller's code array stays in registers.
template <int KM>
__device__ __forceinline__ double exact_component(const PassArgs& a, double sigma, const int32_t (&qv)[2 * KM],
                                                  int jj, int p, bool ctrl) {
  if (!ctrl) {
    const double x = __dmul_rn((double)qv[2 * jj + p], a.qp.two);
    return a.use_sigma ? __dmul_rn(sigma, x) : x;
  }
  double ar = 0.0, ai = 0.0;
#pragma unroll
  for (int m = 0; m < KM; ++m) {
    if (m >= a.K) break;
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
      const int g = p >> (w.b + 1);  // block slot (2^(b+1) values per block)
      const int j = p & (L.nv - 1);
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
#include "sv_pass_big.cuh"

// fgv: the CTA's FastGate (KM <= 8) or BigGate (KM = 32), prepared before the first group
template <typename Real, int KM>
__device__ __forceinline__ void pass_group(Worker<Real>& w, const PassArgs& a, const void* __restrict__ fgv,
                                           double sigma, unsigned long long grp, uint32_t* tc_par = nullptr) {
  using A = Arith<Real>;
  const Layout& L = w.L;
  const FastGate* __restrict__ fg = (const FastGate*)fgv;
  int fF, fqsafe;  // fixed-point form available (F >= 0) and the single-term code limit
  if constexpr (KM > 8) {
    fF = ((const BigGate*)fgv)->F;
    fqsafe = ((const BigGate*)fgv)->qsafe;
  } else {
    fF = fg->F;
    fqsafe = fg->qsafe;
  }
  const Real sg = (Real)sigma;  // complex64: sigma rounded to float once
  const int B = L.nv / 2;
  constexpr bool kFast = sizeof(Real) == 8;
  unsigned long long base = grp;
  for (int l = 0; l < a.h; ++l) base = insert_zero_bit(base, a.high_pos[l]);
  // block id of group slot g (a function rather than an array indexed at run time, which
  // would live in local memory)
  auto blk_of = [&](int g) -> unsigned long long {
    unsigned long long bid = base;
    for (int l = 0; l < a.h; ++l)
      if ((g >> l) & 1) bid |= 1ull << a.slot_shift[l];
    return bid;
  };
  __syncthreads();
  if (threadIdx.x < 4) {
    w.vout_cnt[threadIdx.x] = 0;
    w.m->vbig[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) {
    w.m->any_big = 0;
    w.m->fix = 0;
  }
  for (int i = threadIdx.x; i < a.G * (L.nv >> 5); i += blockDim.x) w.vomask[i] = 0u;  // output verbatim bitmap
  // ---- stream pass-through ----
  // complex128: block slot g keeps the codes of slot src (src = g where the gate acts as the identity on
  // it: the group's high controls are not all 1, or its rows are unit rows; another slot for
  // a +1 permutation across blocks) when that slot holds no verbatim value and every |q| is
  // within qsafe: then each output code equals its input code exactly (the same argument as
  // the single-term shortcut below), and the block's stream is the source stream.
  // A block whose inputs (the blocks it reads) are all zero codes with no verbatim value
  // has zero outputs under any gate (every step of the chain maps 0 to 0): it keeps its
  // own all-zero stream, in either precision.
  bool any_pt = false;
  if (a.pt_ok) {
    if (threadIdx.x == 0) {
      const bool hc = ((blk_of(0) << a.b) & a.cmask_high) == a.cmask_high;
      const bool unit_rule = kFast && (a.pt_ok & 2) && fF >= 0;
      unsigned int dmask = 0;
      int npt = 0;
      for (int g = 0; g < a.G; ++g) {
        const unsigned int reads = hc ? a.need[g] : (1u << g);
        int src = -1;
        if (unit_rule) {
          const int c = hc ? a.pt_src[g] : g;
          if (c >= 0) {
            const unsigned int mm = a.in_info[blk_of(c)].maxq_mode;
            if (!(mm & 0x80000000u) && (long long)(mm & 0x1FFFFFFFu) <= (long long)fqsafe) src = c;
          }
        }
        if (src < 0) {
          bool zero = true;
          for (int h = 0; h < a.G; ++h)
            if (((reads >> h) & 1u) && (a.in_info[blk_of(h)].maxq_mode & 0x9FFFFFFFu)) zero = false;
          if (zero) src = g;
        }
        w.m->pt[g] = src;
        if (src >= 0) ++npt;
        else dmask |= reads;
      }
      w.m->dmask = dmask;
      w.m->npt = npt;
    }
    __syncthreads();
    any_pt = w.m->npt > 0;
    if (w.m->npt == a.G) {
      for (int g = 0; g < a.G; ++g) w.pass_through(blk_of(w.m->pt[g]), blk_of(g), a);
      return;
    }
  }
  // A second round (fix) runs only when a complex128 block stored more verbatim values than
  // its lists hold: the same decode and transform again, writing just those raw values into
  // the output streams the first round wrote (every step is deterministic, so the second
  // round finds the same values).
  for (int round = 0; round < 2; ++round) {
    if (round == 1) {
      __syncthreads();
      if (!w.m->any_big) break;
      for (int g = 0; g < a.G; ++g)
        if (w.m->vbig[g]) w.prepare_out_ranks(g);
      if (threadIdx.x == 0) w.m->fix = 1;
      __syncthreads();
    }
    // ---- Decompress(S) ----
    for (int g = 0; g < a.G; ++g) {
      if (a.input_basis) {
        const int pos = ((a.basis >> a.b) == blk_of(g)) ? 2 * (int)(a.basis & (unsigned long long)(B - 1)) : -1;
        w.load_basis(g, pos);
      } else if (any_pt && !((w.m->dmask >> g) & 1u)) {
        w.load_basis(g, -1);  // read by no recoded block: zeros
      } else {
        w.decode(g, a.in_arena + a.in_off[blk_of(g)], a.in_len[blk_of(g)]);
      }
    }
    // ---- Normalize(S) and GateComputation(G, S), tuple by tuple, in place ----
    if constexpr (KM > 8) {
      __syncthreads();  // every block of the group is decoded
      big_gate_stage<Real>(w, a, (BigGate*)fgv, sigma, blk_of(0), tc_par);
    }
    if constexpr (KM <= 8) {
    const int ntup = B >> a.nlow;
    // the gate's scalars in registers for the whole loop (the code stores below would
    // otherwise make the compiler read them again for every tuple)
    int gF = -1, gqsafe = 0, gdiag = 0, greal = 0;
    long long gmargin = 0;
    int32_t gidhi = 0, gidlo = 0;
    if (kFast) {
      gF = fg->F;
      gqsafe = fg->qsafe;
      gdiag = fg->diag;
      greal = fg->real;
      gmargin = fg->margin;
      gidhi = fg->idhi;
      gidlo = fg->idlo;
    }
    const unsigned long long blk0 = blk_of(0);
    for (int u = threadIdx.x; u < ntup; u += blockDim.x) {
      unsigned long long o = (unsigned long long)u;
      for (int l = 0; l < a.nlow; ++l) o = insert_zero_bit(o, a.low_t[l]);
      const unsigned long long gidx = (blk0 << a.b) | o;
      const bool ctrl = a.apply_gate && ((gidx & a.cmask) == a.cmask);
      const int bp = 2 * (int)o;
      if (kFast && gF >= 0) {
        // member m's values sit at bp + pos_delta[m] (+1) of the group's code array, whose
        // blocks are contiguous
        int32_t qv[2 * KM];
        bool sentinel = false;
  #pragma unroll
        for (int mm = 0; mm < KM; ++mm)
          if (mm < a.K) {
            const int p = bp + a.pos_delta[mm];
            qv[2 * mm] = w.q[p];
            qv[2 * mm + 1] = w.q[p + 1];
            sentinel |= qv[2 * mm] == kSentinel || qv[2 * mm + 1] == kSentinel;
          }
        if (!sentinel) {
          // every input of the tuple is in registers: each output is stored as soon as it is
          // known (the tuples' positions are disjoint)
  #pragma unroll
          for (int jj = 0; jj < KM; ++jj)
            if (jj < a.K) {
              const int pj = bp + a.pos_delta[jj];
  #pragma unroll
              for (int p = 0; p < 2; ++p) {
                int32_t oc = 0;
                bool done = false;
                // outputs that are +-1 times one input: exact without arithmetic when small
                const int ssrc = ctrl ? fg->ssrc[jj][p] : 2 * jj + p;
                if (ssrc >= 0) {
                  int32_t qq = 0;
  #pragma unroll
                  for (int e = 0; e < 2 * KM; ++e)
                    if (e == ssrc) qq = qv[e];
                  if ((qq < 0 ? -qq : qq) <= gqsafe) {
                    oc = (ctrl && fg->ssgn[jj][p] < 0) ? -qq : qq;
                    done = true;
                  }
                }
                if (!done) {
                  long long sh = 0, sl = 0;
                  if (ctrl && gdiag) {
  #pragma unroll
                    for (int c = 0; c < 2; ++c) {
                      const long long qq = qv[2 * jj + c];
                      sh += qq * fg->chi[jj][p][jj][c];
                      sl += (qq * fg->clo[jj][p][jj][c]) >> 4;
                    }
                  } else if (ctrl && greal) {  // real matrix: the cross terms are exactly 0
  #pragma unroll
                    for (int m = 0; m < KM; ++m)
                      if (m < a.K) {
                        const long long qq = qv[2 * m + p];
                        sh += qq * fg->chi[jj][p][m][p];
                        sl += (qq * fg->clo[jj][p][m][p]) >> 4;
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
                    sh = qq * gidhi;
                    sl = (qq * gidlo) >> 4;
                  }
                  done = fast_round(sh + (sl >> 27), gF, gmargin, &oc);
                }
                if (done) w.q[pj + p] = oc;
                else  // near a rounding tie or at the code range: the exact step chain
                  w.put_value(pj >> (w.b + 1), (pj & (L.nv - 1)) + p,
                              (Real)exact_component<KM>(a, sigma, qv, jj, p, ctrl));
              }
            }
          continue;
        }
      }
      tuple_exact<Real, KM>(w, a, sg, bp, ctrl);
    }
    }
    __syncthreads();
    if (round == 0) {
      // ---- Compress(S) ----
      for (int g = 0; g < a.G; ++g) {
        if (any_pt && w.m->pt[g] >= 0) w.pass_through(blk_of(w.m->pt[g]), blk_of(g), a);
        else w.encode(g, blk_of(g), a);
      }
    } else {
      // the raw values are in place: the verbatim sums of those blocks
      for (int g = 0; g < a.G; ++g)
        if (w.m->vbig[g]) {
          const double vs = w.verbatim_square_tree(g);
          if (threadIdx.x == 0 && a.vsum) a.vsum[blk_of(g)] = vs;
        }
      __syncthreads();
      if (threadIdx.x == 0) w.m->fix = 0;
    }
  }
}

template <typename Real, int KM>
__device__ __forceinline__ void pass_body(const PassArgs& a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Layout L = make_layout(a.b, a.G, (int)sizeof(Real), false, KM > 8);
  Worker<Real> w;
  w.init(smem, L, a.b, a.qp);
  if (a.chunk) w.kc = a.chunk;
  // A state poisoned by an earlier pass (or by another CTA of this one) is skipped. One
  // thread reads the flag so that the whole CTA takes the same branch.
  uint32_t tc_par = 0;  // phase of the CTA's tensor-core completion barrier
  if constexpr (KM > 8) {
    if (a.tc) {  // tensor-memory columns and the completion barrier for the whole kernel
      BigGate* bgp = (BigGate*)(smem + L.off_fast);
      if (threadIdx.x < 32) tc_alloc(&bgp->tmem);
      if (threadIdx.x == 0) tc_mbar_init(&bgp->mbar);
      tc_fence_before_sync();
      __syncthreads();
      tc_fence_after_sync();
    }
  }
  if (threadIdx.x == 0) {
    w.m->err = 0;
    w.m->live = *(volatile unsigned int*)&a.sc->status == 0;
  }
  __syncthreads();
  if (w.m->live) {
    const double sigma = a.use_sigma ? *(volatile double*)&a.sc->sigma : 1.0;
    void* fg = smem + L.off_fast;
    if constexpr (KM > 8) {
      big_prepare<Real>((BigGate*)fg, a, sigma);  // all threads; ends with a barrier
    } else {
      if (sizeof(Real) == 8 && threadIdx.x == 0) fast_prepare((FastGate*)fg, a, sigma);  // visible after pass_group's barrier
    }
    for (unsigned long long grp = blockIdx.x; grp < a.ngroups; grp += gridDim.x)
      pass_group<Real, KM>(w, a, fg, sigma, grp, &tc_par);
    if (threadIdx.x == 0 && w.m->err) {
      atomicOr(&a.sc->status, w.m->err);
      atomicMin(&a.sc->fail_seq, a.seq);
    }
  }
  if constexpr (KM > 8) {
    if (a.tc) {  // every MMA has completed (each was waited for) and every load is done
      tc_fence_before_sync();
      __syncthreads();
      if (threadIdx.x < 32) tc_dealloc(((BigGate*)(smem + L.off_fast))->tmem);
    }
  }
}

// The pass kernel without a register cap (the compiler picks the count), and (COMPACT) with
// one. 1-qubit gates (one block per CTA, 55 KB of shared memory at 2048-amplitude blocks): 64
// registers per thread, spilling, so that four 256-thread CTAs fit on an SM. 2-qubit gates
// (up to two coupled blocks, 75 KB): 85 registers, so that the three CTAs the shared memory
// admits also fit the register file.
template <typename Real, int KM>
__global__ void __launch_bounds__(256) k_pass(const PassArgs a) {
  pass_body<Real, KM>(a);
}
template <typename Real, int KM>
__global__ void __launch_bounds__(256, 4) k_pass_c(const PassArgs a) {
  pass_body<Real, KM>(a);
}
template <typename Real, int KM>
__global__ void __launch_bounds__(256, 3) k_pass_c3(const PassArgs a) {
  pass_body<Real, KM>(a);
}
// 4- and 5-qubit gates: at most 128 registers, so that the two CTAs per SM that the shared
// memory admits also fit the register file. A kernel of its own: a minimum of one CTA per SM
// on k_pass lets the compiler take up to 255 registers for the smaller gates too, which
// halves their resident CTAs.
template <typename Real>
__global__ void __launch_bounds__(256, 2) k_pass_big(const PassArgs a) {
  pass_body<Real, 32>(a);
}

template <typename Real, int KM, bool COMPACT>
constexpr auto pass_kernel() {
  if constexpr (KM > 8) return k_pass_big<Real>;
  else if constexpr (COMPACT && KM == 4) return k_pass_c3<Real, KM>;
  else if constexpr (COMPACT) return k_pass_c<Real, KM>;
  else return k_pass<Real, KM>;
}

template <typename Real, int KM, bool COMPACT>
static cudaError_t launch_pass_k(const PassArgs& a, cudaStream_t st) {
  const Layout L = make_layout(a.b, a.G, (int)sizeof(Real), false, KM > 8);
  static std::atomic<unsigned long long> configured{0};  // devices set up
  cudaError_t ce = once_per_device(configured, [] {
    return cudaFuncSetAttribute(pass_kernel<Real, KM, COMPACT>(), cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  });
  if (ce != cudaSuccess) return ce;
  if (L.total > 227 * 1024) return cudaErrorInvalidValue;
  const int T = threads_ok(a.b, a.threads) ? a.threads : worker_threads(a.b);
  if (!chunk_ok(a.b, a.chunk ? a.chunk : kChunkDefault, T)) return cudaErrorInvalidValue;
  unsigned long long grid = a.ngroups;
  if constexpr (KM > 8) {
    // 4- and 5-qubit gates: as many CTAs as fit at once, each walking many groups, so that the
    // per-CTA preparation of the gate's coefficient tables (and tensor memory) is amortized
    // (resident CTAs per SM: what the 228 KB of shared memory holds, each CTA with the 1 KB the
    // hardware reserves, and at most two by the 128-register cap of this build)
    int dev = 0, sms = 0;
    int per_sm = (int)((228u * 1024u) / (L.total + 1024u));
    if (per_sm > 2) per_sm = 2;
    if (per_sm < 1) per_sm = 1;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        sms > 0 && grid > (unsigned long long)sms * per_sm)
      grid = (unsigned long long)sms * per_sm;
  }
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  const auto kern = pass_kernel<Real, KM, COMPACT>();
  kern<<<(unsigned int)grid, T, L.total, st>>>(a);
  return cudaGetLastError();
}

template <typename Real>
static cudaError_t launch_pass_t(const PassArgs& a, cudaStream_t st) {
  if (a.K <= 2) return launch_pass_k<Real, 2, false>(a, st);
  if (a.K <= 4) return launch_pass_k<Real, 4, false>(a, st);
  if (a.K <= 8) return launch_pass_k<Real, 8, false>(a, st);
  return launch_pass_k<Real, 32, false>(a, st);  // 4- and 5-qubit gates
}

}  // namespace sv
