// sv_pass_big.cuh — GateComputation(G, S) of Algorithm 1 (Wu et al., PMES 2018) for dense
// 4- and 5-qubit gates (K = 16 or 32 amplitudes per tuple), e.g. gates fused from several
// 1- and 2-qubit gates. Included by sv_pass.cuh; used by the KM = 32 build of the fused pass.
//
// A tuple's K output rows are computed by K consecutive threads. The CTA walks the group's
// tuples in rounds of blockDim.x rows (whole tuples, since K divides the CTA size): every
// thread computes its row from the codes in shared memory, the CTA synchronizes, and then the
// rows are written back in place. Tuples of different rounds share no member, so the in-place
// update needs one barrier per round.
//
// complex128 rows use the fixed-point form of the fast path (FastGate's argument, with the
// error terms grown for 32-term sums, below); a row whose fixed-point value lies too close to a
// rounding tie, or a tuple with a verbatim input, runs the exact FP64 step chain (decoded value,
// scale, ordered complex sum). complex64 rows always run the FP32 chain. Results are those of
// the chain in either case, so every stream equals the oracle's.
#pragma once
// (included inside namespace sv, after the helpers of sv_pass.cuh it uses)

// All threads: the fixed-point coefficients of sigma * G * fl(2eb r) (complex128) or the FP32
// matrix in transposed order (complex64). Ends with a barrier.
template <typename Real>
__device__ inline void big_prepare(BigGate* bg, const PassArgs& a, double sigma) {
  const int K = a.K, tid = threadIdx.x, T = blockDim.x;
  if (sizeof(Real) == 4) {
    float* gfs = (float*)bg->tab;
    for (int e = tid; e < K * K; e += T) {
      const int jj = e / K, m = e % K;  // row-major input: entry e = jj K + m
      gfs[2 * (m * K + jj)] = a.gfbig[2 * e];
      gfs[2 * (m * K + jj) + 1] = a.gfbig[2 * e + 1];
    }
    if (tid == 0) {
      bg->F = -1;
      bg->tc = 0;
    }
    __syncthreads();
    return;
  }
  const double s1 = __dmul_rn(a.use_sigma ? sigma : 1.0, a.two_r);
  // row sums of |c| in the order fast_prepare uses (one thread per row)
  if (tid < K) {
    double row = 0.0;
    for (int m = 0; m < K; ++m)
      row += fabs(__dmul_rn(__ldg(a.gbig + 2 * (tid * K + m)), s1)) +
             fabs(__dmul_rn(__ldg(a.gbig + 2 * (tid * K + m) + 1), s1));
    bg->rows[tid] = row;
    // outputs that are +-1 or +-i times one input
    int nz = 0, mz = -1;
    for (int m = 0; m < K; ++m)
      if (__ldg(a.gbig + 2 * (tid * K + m)) != 0.0 || __ldg(a.gbig + 2 * (tid * K + m) + 1) != 0.0) {
        ++nz;
        mz = m;
      }
    bg->ssrc[tid][0] = bg->ssrc[tid][1] = -1;
    bg->ssgn[tid][0] = bg->ssgn[tid][1] = 1;
    if (nz == 1) {
      const double gr = __ldg(a.gbig + 2 * (tid * K + mz)), gi = __ldg(a.gbig + 2 * (tid * K + mz) + 1);
      if (gi == 0.0 && (gr == 1.0 || gr == -1.0)) {
        const int sg = gr > 0 ? 1 : -1;
        bg->ssrc[tid][0] = (int8_t)(2 * mz);
        bg->ssgn[tid][0] = (int8_t)sg;
        bg->ssrc[tid][1] = (int8_t)(2 * mz + 1);
        bg->ssgn[tid][1] = (int8_t)sg;
      } else if (gr == 0.0 && (gi == 1.0 || gi == -1.0)) {
        const int sg = gi > 0 ? 1 : -1;
        bg->ssrc[tid][0] = (int8_t)(2 * mz + 1);
        bg->ssgn[tid][0] = (int8_t)-sg;
        bg->ssrc[tid][1] = (int8_t)(2 * mz);
        bg->ssgn[tid][1] = (int8_t)sg;
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    double R = fabs(s1);
    for (int jj = 0; jj < K; ++jj) R = bg->rows[jj] > R ? bg->rows[jj] : R;
    const int cl = R > 0.0 ? ceil_log2(R) : 0;
    int F = 30 - (cl > 0 ? cl : 0);
    if (!(R > 0.0) || cl > 16 || !isfinite(R)) F = -1;  // fast path off
    bg->F = F;
    bg->diag = 1;
    bg->real = 1;
    bg->tc = 0;
    if (F >= 0) {
      // the exact chain lands within (K + 7) 2^-53 R Q of T (K - 1 ordered additions, the
      // decode, scale, product, difference and requantization roundings, and the roundings of
      // the coefficients); with Q = 2^29 that is R 2^(F-19) in units of W for K <= 16 and
      // R 2^(F-18) for K = 32. Rounding each of the 2K coefficients to 2^-(F+31) moves W by at
      // most 2K 2^29 2^-(F+32) = K/4 units, and the two truncating shifts by one more unit.
      const int chain = K > 16 ? F - 18 : F - 19;
      bg->margin = (long long)ceil(R * scalbn(1.0, chain)) + (K / 4 + 2) + (1ll << (F > 21 ? F - 21 : 0));
      const long long v = __double2ll_rn(__dmul_rn(s1, scalbn(1.0, F + 31)));
      bg->idhi = (int32_t)(v >> 31);
      bg->idlo = (int32_t)(v & 0x7fffffffll);
      const double dev = fabs(s1 - 1.0) + scalbn(1.0, -50);
      const double lim = (0.5 - scalbn(1.0, -18) - R * scalbn(1.0, chain - F)) / dev;
      bg->qsafe = lim >= 536870000.0 ? 536870000 : (lim > 0.0 ? (int)lim : -1);
    }
  }
  __syncthreads();
  const int F = bg->F;
  if (F >= 0 && a.tc) {
    // tensor-core form: the digits of v for output row o = 2 jj + p and input column
    // i = 2 m + c, one FP16 matrix per digit in the no-swizzle K-major layout
    if (tid == 0) {
      bg->tc = 1;
      bg->diag = 0;  // the diagonal and real shortcuts read the CUDA-core tables
      bg->real = 0;
    }
    const double scale = scalbn(1.0, F + 31);
    const int kin = 2 * K;
    uint16_t* dig = (uint16_t*)bg->tab;
    for (int e = tid; e < K * K; e += T) {
      const int jj = e / K, m = e % K;
      const double A = __dmul_rn(__ldg(a.gbig + 2 * e), s1);
      const double Bc = __dmul_rn(__ldg(a.gbig + 2 * e + 1), s1);
      const double cv[4] = {A, Bc, -Bc, A};  // (c, p) = (0, 0), (0, 1), (1, 0), (1, 1)
      for (int cp = 0; cp < 4; ++cp) {
        long long v = __double2ll_rn(__dmul_rn(cv[cp], scale));
        const int o = 2 * jj + (cp & 1), i = 2 * m + (cp >> 1);
        for (int d = 0; d < kTcDigits; ++d) {
          const long long t = v + 256;
          const long long hi = t >> 9;  // floor
          const int digit = (int)(t - (hi << 9)) - 256;
          v = hi;
          dig[d * kin * kin + tc_tile_index(o, i, kin)] = __half_as_ushort(__int2half_rn(digit));
        }
      }
    }
    tc_fence_operands();
    __syncthreads();
    return;
  }
  if (F >= 0) {
    if (tid == 0) bg->tc = 0;
    const double scale = scalbn(1.0, F + 31);
    bool diag = true, real = true;
    for (int e = tid; e < K * K; e += T) {
      const int jj = e / K, m = e % K;
      const double A = __dmul_rn(__ldg(a.gbig + 2 * e), s1);
      const double Bc = __dmul_rn(__ldg(a.gbig + 2 * e + 1), s1);
      if (m != jj && (A != 0.0 || Bc != 0.0)) diag = false;
      if (Bc != 0.0) real = false;
      // re += A q_re - B q_im ; im += B q_re + A q_im ; entry ((m 2 + c) 2 + p) K + jj
      const double cv[4] = {A, Bc, -Bc, A};  // (c, p) = (0, 0), (0, 1), (1, 0), (1, 1)
      for (int cp = 0; cp < 4; ++cp) {
        const long long v = __double2ll_rn(__dmul_rn(cv[cp], scale));
        const int idx = (m * 4 + cp) * K + jj;
        bg->tab[idx] = (int32_t)(v >> 31);
        bg->tab[4096 + idx] = (int32_t)(v & 0x7fffffffll);
      }
    }
    if (!diag) atomicAnd(&bg->diag, 0);
    if (!real) atomicAnd(&bg->real, 0);
  }
  __syncthreads();
}

// Row jj of the tuple with value base bp through the exact step chain in the value type: the
// decoded values (verbatim ones included), the scale, the ordered complex sum over members.
template <typename Real>
__device__ __forceinline__ void big_exact_row(const Worker<Real>& w, const PassArgs& a, const BigGate* bg,
                                              Real sg, int bp, int jj, bool ctrl, Real* zr, Real* zi) {
  using A = Arith<Real>;
  const int K = a.K, nvm = w.L.nv - 1, sh = w.b + 1;
  if (!ctrl) {
    const int p = bp + a.pos_delta[jj];
    const Real xr = w.value_at(p >> sh, p & nvm), xi = w.value_at(p >> sh, (p & nvm) + 1);
    *zr = a.use_sigma ? A::mul(sg, xr) : xr;
    *zi = a.use_sigma ? A::mul(sg, xi) : xi;
    return;
  }
  const float* gfs = (const float*)bg->tab;
  Real ar = 0, ai = 0;
  for (int m = 0; m < K; ++m) {
    const int p = bp + a.pos_delta[m];
    Real yr = w.value_at(p >> sh, p & nvm), yi = w.value_at(p >> sh, (p & nvm) + 1);
    if (a.use_sigma) {
      yr = A::mul(sg, yr);
      yi = A::mul(sg, yi);
    }
    Real gr, gi;
    if (sizeof(Real) == 8) {
      gr = (Real)__ldg(a.gbig + 2 * (jj * K + m));
      gi = (Real)__ldg(a.gbig + 2 * (jj * K + m) + 1);
    } else {
      gr = (Real)gfs[2 * (m * K + jj)];
      gi = (Real)gfs[2 * (m * K + jj) + 1];
    }
    const Real pr = A::sub(A::mul(gr, yr), A::mul(gi, yi));
    const Real pi = A::add(A::mul(gr, yi), A::mul(gi, yr));
    if (m == 0) {
      ar = pr;
      ai = pi;
    } else {
      ar = A::add(ar, pr);
      ai = A::add(ai, pi);
    }
  }
  *zr = ar;
  *zi = ai;
}

// GateComputation for the tuples [u0, u1) of one group (codes decoded in w.q), in place, on
// the CUDA cores: rounds of blockDim.x output rows. `tables`: the CTA holds the CUDA-core form
// of the fixed-point coefficients (otherwise every row runs the exact chain). All threads call
// it; it ends with a barrier.
template <typename Real>
__device__ void big_rounds(Worker<Real>& w, const PassArgs& a, const BigGate* bg, double sigma,
                           unsigned long long blk0, int u0, int u1, bool tables) {
  const int K = a.K, T = blockDim.x, tid = threadIdx.x;
  const int nv = w.L.nv;
  const Real sg = (Real)sigma;
  const bool fast = sizeof(Real) == 8 && bg->F >= 0 && tables;
  for (int r0 = u0 * K; r0 < u1 * K; r0 += T) {
    const int it = r0 + tid;
    const bool act = it < u1 * K;  // rows past the range recompute row u0 * K and write nothing
    const int u = act ? it / K : u0, jj = act ? it % K : 0;
    unsigned long long o = (unsigned long long)u;
    for (int l = 0; l < a.nlow; ++l) o = insert_zero_bit(o, a.low_t[l]);
    const bool ctrl = ((((blk0 << a.b) | o) & a.cmask) == a.cmask);
    const int bp = 2 * (int)o;
    bool sentinel = false;
    if (sizeof(Real) == 8) {
      for (int m = 0; m < K; ++m) {
        const int p = bp + a.pos_delta[m];
        sentinel |= w.q[p] == kSentinel || w.q[p + 1] == kSentinel;
      }
    }
    int32_t oc[2] = {0, 0};
    bool exact = !fast || sentinel;
    if (!exact) {
      const int F = bg->F;
      const long long margin = bg->margin;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const int ssrc = ctrl ? bg->ssrc[jj][p] : 2 * jj + p;
        if (ssrc >= 0) {
          const int q0 = bp + a.pos_delta[ssrc >> 1] + (ssrc & 1);
          const int32_t qq = w.q[q0];
          if ((qq < 0 ? -qq : qq) <= bg->qsafe) {
            oc[p] = (ctrl && bg->ssgn[jj][p] < 0) ? -qq : qq;
            continue;
          }
        }
        long long sh = 0, sl = 0;
        if (!ctrl) {
          const long long qq = w.q[bp + a.pos_delta[jj] + p];
          sh = qq * bg->idhi;
          sl = (qq * bg->idlo) >> 4;
        } else if (bg->diag) {
          const int pm = bp + a.pos_delta[jj];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const long long qq = w.q[pm + c];
            const int idx = (jj * 4 + c * 2 + p) * K + jj;
            sh += qq * bg->tab[idx];
            sl += (qq * bg->tab[4096 + idx]) >> 4;
          }
        } else {
          for (int m = 0; m < K; ++m) {
            const int pm = bp + a.pos_delta[m];
            const long long qr = w.q[pm], qi = w.q[pm + 1];
            const int i0 = (m * 4 + p) * K + jj, i1 = (m * 4 + 2 + p) * K + jj;
            sh += qr * bg->tab[i0] + qi * bg->tab[i1];
            sl += ((qr * bg->tab[4096 + i0]) >> 4) + ((qi * bg->tab[4096 + i1]) >> 4);
          }
        }
        if (!fast_round(sh + (sl >> 27), F, margin, &oc[p])) exact = true;
      }
    }
    Real zr = 0, zi = 0;
    if (exact) big_exact_row<Real>(w, a, bg, sg, bp, jj, ctrl, &zr, &zi);
    __syncthreads();  // every row of this round has read its inputs
    const int pj = bp + a.pos_delta[jj];
    const int g = pj >> (w.b + 1), j = pj & (nv - 1);
    if (!act) {
    } else if (exact) {
      w.put_value(g, j, zr);
      w.put_value(g, j + 1, zi);
    } else {
      w.q[pj] = oc[0];
      w.q[pj + 1] = oc[1];
    }
  }
  __syncthreads();
}

#include "sv_pass_tc.cuh"

// GateComputation for one group (codes decoded in w.q), in place: on the tensor cores when the
// CTA holds the tensor-core form and the group's codes are small enough, else on the CUDA
// cores. All threads call it; it ends with a barrier. tc_par: the CTA's mbarrier phase.
template <typename Real>
__device__ void big_gate_stage(Worker<Real>& w, const PassArgs& a, BigGate* bg, double sigma,
                               unsigned long long blk0, uint32_t* tc_par) {
  const int ntup = (w.L.nv / 2 << a.h) / a.K;
  if (sizeof(Real) == 8 && bg->tc) {
    if (tc_gate_stage<Real>(w, a, bg, sigma, blk0, tc_par)) return;
    big_rounds<Real>(w, a, bg, sigma, blk0, 0, ntup, false);
    return;
  }
  big_rounds<Real>(w, a, bg, sigma, blk0, 0, ntup, true);
}
