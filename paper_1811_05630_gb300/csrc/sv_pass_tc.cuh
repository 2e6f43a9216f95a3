// sv_pass_tc.cuh — GateComputation(G, S) of Algorithm 1 (Wu et al., PMES 2018) for dense
// 4- and 5-qubit gates on the tensor cores (tcgen05), complex128. Included by sv_pass_big.cuh
// (inside namespace sv).
//
// The fast path's fixed-point value of output component o of a tuple is
//   W = floor(sum_i q_i v_oi / 2^31),  v_oi = round(c_oi 2^(F+31))
// (c = sigma G fl(2eb r), q the tuple's 2K input codes; W in units of 2^-F). The products are
// made exact on the FP16 tensor pipe by digits: v = sum_d v_d 512^d (seven balanced digits,
// |v_d| <= 256, kept per CTA as FP16 matrices) and q = sum_e q_e 512^e (one digit when every
// |q| < 256, two when every |q| < 2^17). Each MMA multiplies a 128-tuple tile of one code digit
// (A, 128 x 2K) by a 32-column slice of one coefficient digit (B, 32 x 2K) into FP32 tensor
// memory; the MMAs of equal weight s = d + e share an accumulator. Every product is at most
// 257 * 256 in magnitude and an accumulator sums at most 2 x 64 of them, below 2^24, so the FP32
// sums are exact integers. The low coefficient digits are dropped (d < 2 for one code digit,
// d < 1 for two): that moves W by at most 64 * 256 * 256 / 2^31 < 1 unit (two digits: 64 * 2^17
// * 512 / 2^32 = 1 unit), and the final floor by less than one more; the fast path's margin for
// K-member tuples allows K/4 + 2 units here, so its rounding decisions stay those of the exact
// chain. Outputs it cannot decide (near a rounding tie, a verbatim input) run the exact FP64
// chain; tuples whose controls are not all set take the identity form. Results are those of the
// CUDA-core form bit for bit.
#pragma once

// One code digit of q (e = 0: the balanced low digit in [-256, 255]; e = 1: the rest).
__device__ __forceinline__ int tc_code_digit(int32_t q, int e) {
  const int lo = ((q + 256) & 511) - 256;
  return e ? (q - lo) >> 9 : lo;
}

template <typename Real>
__device__ bool tc_gate_stage(Worker<Real>& w, const PassArgs& a, BigGate* bg, double sigma,
                              unsigned long long blk0, uint32_t* tc_par);

template <>
__device__ inline bool tc_gate_stage<float>(Worker<float>&, const PassArgs&, BigGate*, double, unsigned long long,
                                     uint32_t*) {
  return false;
}

// All threads call it after the group's codes are decoded. Returns false, having changed
// nothing, when the codes are too large for the digit form (the caller then runs the CUDA-core
// rounds); otherwise the group's tuples are updated in place and it ends with a barrier.
template <>
__device__ inline bool tc_gate_stage<double>(Worker<double>& w, const PassArgs& a, BigGate* bg, double sigma,
                                      unsigned long long blk0, uint32_t* tc_par) {
  if (blockDim.x != 256) return false;  // two warps per lane quarter cover a slice's 32 columns
  const int K = a.K, kin = 2 * K, T = blockDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nv = w.L.nv, ntup = ((nv / 2) << a.h) / K;
  const double sg = sigma;
  // the group's largest |code| (verbatim slots excluded)
  uint32_t am = 0;
  for (int i = tid; i < (nv << a.h); i += T) {
    const int32_t c = w.q[i];
    if (c != kSentinel) {
      const uint32_t ac = c < 0 ? (uint32_t)(-(int64_t)c) : (uint32_t)c;
      am = ac > am ? ac : am;
    }
  }
  am = block_reduce_max<uint32_t>(am, (uint32_t*)w.m->red);
  const int nq = am < 256u ? 1 : (am < 131072u ? 2 : 0);
  if (nq == 0) return false;
  const int d0 = nq == 1 ? 2 : 1;                  // lowest coefficient digit kept
  const int nacc = kTcDigits - d0 + nq - 1;        // accumulators: weights s = d0 .. 6 + nq - 1
  const int nhalf = kin / kTcN;                    // 32-column slices of the 2K outputs
  const int F = bg->F;
  const long long margin = bg->margin;
  uint16_t* At = (uint16_t*)w.stage;               // A tile: kTcM tuples x 2K inputs
  const uint16_t* dig = (const uint16_t*)bg->tab;  // B: digit d at d * kin * kin
  int* xlist = (int*)w.hval;                       // outputs for the exact chain (u << 8 | o)
  double* xval = (double*)(w.hval + 128);          // and their values
  constexpr int kXmax = 128;
  const int q4 = warp & 3, cg = warp >> 2;         // lane quarter (tuple rows), column group
  const uint32_t sbo = (uint32_t)(kin / 8) * 128u, idesc = tc_idesc(kTcM, kTcN);
  bool tc_ok = true;

  for (int u0 = 0; u0 < ntup; u0 += kTcM) {
    const int nt = ntup - u0 < kTcM ? ntup - u0 : kTcM;
    // this thread's tuple row and its properties
    const int r = 32 * q4 + lane, u = u0 + r;
    const bool row = r < nt;
    unsigned long long ob = (unsigned long long)(row ? u : u0);
    for (int l = 0; l < a.nlow; ++l) ob = insert_zero_bit(ob, a.low_t[l]);
    const int bp = 2 * (int)ob;
    const bool ctrl = ((((blk0 << a.b) | ob) & a.cmask) == a.cmask);
    bool sentinel = false;
    for (int m = 0; m < K; ++m) {
      const int p = bp + a.pos_delta[m];
      sentinel |= w.q[p] == kSentinel || w.q[p + 1] == kSentinel;
    }
    if (tid == 0) {
      w.m->tc_nx = 0;
      w.m->tc_over = 0;
    }
    int32_t oc[32];            // codes of this thread's outputs (half h, column c: [h * 16 + c])
    uint32_t xm = 0;           // those that run the exact chain
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h >= nhalf) break;
      for (int e = 0; e < nq; ++e) {
        if (h == 0 || nq > 1) {
          // A tile of code digit e (rows past the chunk and verbatim slots are 0)
          {
            // thread t fills row t % 128, inputs [half * K, half * K + K) with half = t / 128
            const int rr = tid & (kTcM - 1), i0 = (tid >> 7) * K;
            int bpr = 0;
            if (rr < nt) {
              unsigned long long o2 = (unsigned long long)(u0 + rr);
              for (int l = 0; l < a.nlow; ++l) o2 = insert_zero_bit(o2, a.low_t[l]);
              bpr = 2 * (int)o2;
            }
            for (int i = i0; i < i0 + K; ++i) {
              int dv = 0;
              if (rr < nt) {
                const int32_t c = w.q[bpr + a.pos_delta[i >> 1] + (i & 1)];
                if (c != kSentinel) dv = tc_code_digit(c, e);
              }
              At[tc_tile_index(rr, i, kin)] = __half_as_ushort(__int2half_rn(dv));
            }
          }
          tc_fence_operands();
        }
        tc_fence_before_sync();
        __syncthreads();
        if (tid == 0) {
          tc_fence_after_sync();
          const uint32_t abase = tc_smem_u32(At);
          for (int d = d0; d < kTcDigits; ++d) {
            const int acc = d + e - d0;
            // an accumulator is new in this slice unless an earlier code digit wrote it
            const bool first = e == 0 || d == kTcDigits - 1;
            const uint32_t bbase = tc_smem_u32(dig + d * kin * kin + tc_tile_index(h * kTcN, 0, kin));
            for (int k0 = 0; k0 < kin; k0 += 16)
              tc_mma(bg->tmem + (uint32_t)(acc * kTcN), tc_desc(abase + 16u * k0, 128u, sbo),
                     tc_desc(bbase + 16u * k0, 128u, sbo), idesc, (k0 > 0 || !first) ? 1 : 0);
          }
          tc_commit(&bg->mbar);
        }
        if (!tc_wait(&bg->mbar, *tc_par & 1u)) tc_ok = false;
        *tc_par += 1;
      }
      // this slice's outputs: the accumulators of the thread's tuple row, 16 columns of its
      // column group, four at a time; W = sum_s acc_s 512^s / 2^31, the terms below 2^31
      // summed first so that one floor is taken
      tc_fence_after_sync();
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        long long hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
        uint32_t v[kTcMaxAcc - 1][4];  // every accumulator's four columns, one wait for all
#pragma unroll
        for (int acc = 0; acc < kTcMaxAcc - 1; ++acc)
          if (acc < nacc) tc_ld4(bg->tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(acc * kTcN + cg * 16 + c4 * 4), v[acc]);
        tc_ld_wait();
#pragma unroll
        for (int acc = 0; acc < kTcMaxAcc - 1; ++acc) {
          if (acc >= nacc) break;
          const int s9 = 9 * (acc + d0);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const long long x = (long long)__uint_as_float(v[acc][j]);
            if (s9 >= 31) hi[j] += x << (s9 - 31);
            else lo[j] += x << s9;
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int o = h * kTcN + cg * 16 + c4 * 4 + j, jj = o >> 1, p = o & 1;
          int32_t code = 0;
          bool ex = sentinel;
          if (!ex && ctrl) {
            ex = !fast_round(hi[j] + (lo[j] >> 31), F, margin, &code);
          } else if (!ex) {  // controls not all 1: the identity, scaled
            const int32_t qq = w.q[bp + a.pos_delta[jj] + p];
            if ((qq < 0 ? -qq : qq) <= bg->qsafe) {
              code = qq;
            } else {
              const long long sh = (long long)qq * bg->idhi, sl = ((long long)qq * bg->idlo) >> 4;
              ex = !fast_round(sh + (sl >> 27), F, margin, &code);
            }
          }
          oc[(h & 1) * 16 + c4 * 4 + j] = code;
          if (ex && row) {
            xm |= 1u << ((h & 1) * 16 + c4 * 4 + j);
            const int k = atomicAdd(&w.m->tc_nx, 1);
            if (k < kXmax) xlist[k] = (r << 8) | o;
            else w.m->tc_over = 1;
          }
        }
      }
      tc_fence_before_sync();
    }
    // every tensor-memory load is done and the list is complete
    if (__syncthreads_or(!tc_ok)) {
      if (tid == 0) atomicOr(&w.m->err, kStTimeout);
      __syncthreads();
      return true;
    }
    if (w.m->tc_over) {  // many outputs for the exact chain: the chunk runs the CUDA-core rounds
      big_rounds<double>(w, a, bg, sigma, blk0, u0, u0 + nt, false);
      continue;
    }
    const int nx = w.m->tc_nx;
    for (int i = tid; i < nx; i += T) {
      const int rr = xlist[i] >> 8, o = xlist[i] & 255;
      unsigned long long o2 = (unsigned long long)(u0 + rr);
      for (int l = 0; l < a.nlow; ++l) o2 = insert_zero_bit(o2, a.low_t[l]);
      const bool c2 = ((((blk0 << a.b) | o2) & a.cmask) == a.cmask);
      double zr, zi;
      big_exact_row<double>(w, a, bg, sg, 2 * (int)o2, o >> 1, c2, &zr, &zi);
      xval[i] = (o & 1) ? zi : zr;
    }
    __syncthreads();  // every input of the chunk has been read
    if (row) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        if (hh >= nhalf) break;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int o = hh * kTcN + cg * 16 + c;
          if (!((xm >> (hh * 16 + c)) & 1u)) w.q[bp + a.pos_delta[o >> 1] + (o & 1)] = oc[hh * 16 + c];
        }
      }
    }
    for (int i = tid; i < nx; i += T) {
      const int rr = xlist[i] >> 8, o = xlist[i] & 255;
      unsigned long long o2 = (unsigned long long)(u0 + rr);
      for (int l = 0; l < a.nlow; ++l) o2 = insert_zero_bit(o2, a.low_t[l]);
      const int pj = 2 * (int)o2 + a.pos_delta[o >> 1] + (o & 1);
      w.put_value(pj >> (w.b + 1), pj & (nv - 1), xval[i]);
    }
    __syncthreads();
  }
  return true;
}
