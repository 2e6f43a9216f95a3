// sv_block.cuh — one CTA's work on a group of codec blocks: decode, transform, encode.
//
// Algorithm 1 of Wu et al. (PMES 2018) processes, for every gate, every slice in four
// steps: Decompress(S), Normalize(S), GateComputation(G, S), Compress(S). On the GPU a
// slice is cut into independent blocks of B = 2^b amplitudes and one CTA owns the 2^h
// blocks that a gate couples (h = number of targets >= b). The decompressed amplitudes
// never leave shared memory: the integer codes q (one int32 per real value) are decoded
// into shared memory, the gate is applied tuple by tuple, the results are re-quantized in
// place, and the new stream is assembled in shared memory and copied out with 16-byte
// stores into a bump-allocated output arena.
#pragma once
#include "sv_device.cuh"

namespace sv {

// Per-CTA scalars in the misc area.
struct Misc {
  uint32_t scan[40];
  unsigned long long red[40];
  int vin_cnt[4], vout_cnt[4];
  unsigned int err;
  int live;  // the state being processed is not poisoned
  int D;
  int nesc;
  int cnt;
  int mode, lmax, width;
  uint32_t pbits;
  uint32_t size;
  unsigned long long out_off;
  int ok;
  // complex128 blocks with more verbatim values than the lists hold: inputs are read from
  // the stream by rank; outputs are found again by a second transform (fix) that writes
  // their raw values straight into the already written output stream
  int vin_big[4];
  const uint64_t* vin_vals[4];
  int vbig[4];
  int any_big;
  int fix;
  uint8_t* vsec_base[4];
  uint32_t vsec_valoff[4];
  int pt[4];       // pass-through source slot per block of the group (-1: recode)
  unsigned int dmask;  // blocks of the group to decode
  int npt;
  int tc_nx, tc_over;  // tensor-core gate: outputs listed for the exact chain, list overflow
  int first[34];   // canonical first code per length
  int offs[34];    // first canonical index per length
  int lcount[34];  // codes per length
};

// Summary of one stored block stream, written with it by every pass and read by the next:
// enough to re-emit the stream unchanged (with its norm and statistics contributions) when
// the next pass provably reproduces the block's codes.
struct BlkInfo {
  unsigned long long sq_lo;  // exact sum of q^2 over the block (< 2^71), low 64 bits
  unsigned int sq_hi_nesc;   // bits 0..7: bits 64..71 of the sum; bits 8..31: escapes
  unsigned int maxq_mode;    // bits 0..28: max |q|; bits 29..30: mode; bit 31: verbatim values
};

struct __align__(16) PassArgs {
  int b, nv, G, h, k, K, nlow;
  int low_t[5];       // low targets ascending (for base enumeration)
  int high_pos[5];    // (high target - b) ascending (block-id expansion)
  int slot_shift[5];  // for slot bit l (target order of high targets): block-id bit
  int pos_delta[32];  // value-position offset of tuple member m within the group
  unsigned long long cmask;
  int apply_gate;     // 0: identity (initial compression)
  int input_basis;    // 1: the input is the basis state |basis>
  unsigned long long basis;
  int use_sigma;
  double g[2 * 64];   // gate matrix (re, im), row-major K x K, for K <= 8
  float gf[2 * 64];
  // K = 16 or 32 (4- and 5-qubit gates): the matrix in device memory (the state's gate slot,
  // written on the state's stream before the launch), FP64 and its FP32 rounding
  const double* gbig;
  const float* gfbig;
  QuantP qp;
  double two2;
  double two_r;       // fl(2eb * r), the dequantize-requantize factor (about 1)
  unsigned long long ngroups;
  int tc;  // 4- and 5-qubit gates of complex128 on the tensor cores (256-thread CTAs)
  const uint8_t* in_arena;
  const unsigned long long* in_off;
  const unsigned int* in_len;
  uint8_t* out_arena;
  unsigned long long out_cap;
  int out_id;
  unsigned long long* out_off;
  unsigned int* out_len;
  DevScalars* sc;
  double* vsum;
  double* tree;  // scratch of the norm kernel's verbatim-sum tree (2 (nblocks / 256 + 1) doubles)
  unsigned int seq;
  int threads;  // CTA size (0: worker_threads(b)); results do not depend on it
  int chunk;    // Huffman chunk size (0: 32); 2^(b+1) / chunk <= CTA size
  // stream pass-through: pt_ok bit 0 re-emits blocks whose inputs are all zero, bit 1
  // (complex128) blocks whose rows are unit rows: slot g of a group whose high controls are
  // all 1 takes the codes of slot pt_src[g] (-1: never); need[g] is the mask of the slots
  // its outputs read
  int pt_ok;
  int pt_src[4];
  unsigned int need[4];
  unsigned long long cmask_high;  // control bits at or above b
  const BlkInfo* in_info;
  BlkInfo* out_info;
};

// Fixed-point form of one gate pass for complex128 (computed once per CTA): output jj, part
// p (0 re, 1 im) is W = sum over members m and components c of coef[jj][p][m][c] * q[m][c],
// with coef = sigma * G * fl(2eb * r) in units of 2^-(F+31), split as hi * 2^31 + lo
// (lo in [0, 2^31)). Diagonal gates use only m = jj.
struct FastGate {
  int F;              // fractional bits of W
  int diag;           // the gate matrix is diagonal
  int real;           // every entry of sigma * G * fl(2eb r) has a zero imaginary part
  long long margin;   // half-width of the band around a rounding tie sent to the exact path
  // outputs that are one input times +-1 (identity rows, permutations, phase +-1 / +-i):
  // source index (member * 2 + component, -1 if not such an output) and sign; their code is
  // exactly +-q whenever |q| <= qsafe
  int8_t ssrc[8][2], ssgn[8][2];
  int qsafe;
  int32_t chi[8][2][8][2], clo[8][2][8][2];
  int32_t idhi, idlo; // the identity scaled by sigma (members whose controls are not all 1)
};

// Fixed-point form of a 4- or 5-qubit gate (K = 16 or 32 members per tuple) for complex128,
// prepared by all threads of a CTA: the same quantities as FastGate. The table area holds one
// of two forms of the coefficients v = round(c 2^(F+31)) (c = sigma G fl(2eb r)):
//  - CUDA-core form: v split as hi 2^31 + lo, transposed (entry ((m * 2 + c) * 2 + p) * K + jj,
//    hi in tab[0, 4096), lo in tab[4096, 8192)) so that the lanes of a warp, which take
//    consecutive output rows jj of one tuple, read consecutive words;
//  - tensor-core form: v as 7 balanced base-512 digits (v = sum_d dig_d 512^d, |dig_d| <= 256),
//    each digit an FP16 matrix of 2K output rows by 2K input columns in the tensor cores'
//    no-swizzle K-major layout (see sv_pass_tc.cuh), digit d at byte 2 d (2K)^2.
// complex64 keeps the FP32 matrix in the table area instead (entry 2 (m K + jj) + {0: re, 1: im}).
struct __align__(128) BigGate {
  int32_t tab[7 * 64 * 64 / 2];  // 56 KB: 7 FP16 matrices of 64 x 64 (the larger form)
  int F, diag, real, qsafe;
  long long margin;
  int32_t idhi, idlo;
  double rows[32];  // row sums of |c| (scratch of the preparation)
  int8_t ssrc[32][2], ssgn[32][2];
  unsigned long long mbar;  // tensor-core form: completion barrier of the CTA's MMAs
  uint32_t tmem;            // tensor-core form: the CTA's tensor-memory columns
  int tc;                   // the table holds the tensor-core form
};

// Dynamic shared-memory layout of a worker CTA (host and device agree on it).
struct Layout {
  int nv, G, hs, dcap, p2cap;
  uint32_t off_q, off_vin_pos, off_vin_bits, off_vout_pos, off_vout_bits, off_hkey, off_hval,
      off_stage, off_build, off_misc, off_fast, off_desc, off_vmask, off_vtree, off_vomask, off_vpre_in,
      off_vpre_out, total;
  uint32_t stage_bytes, build_bytes;
  uint32_t sort_off, sort_n;  // rank-sort scratch inside the build area
  uint32_t off_wint, off_parent, off_parent2, off_lens, off_lens2;
};

__host__ __device__ inline int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// `batch`: the batched pass also keeps the current state's descriptor in shared memory.
// `big`: the pass applies 4- or 5-qubit gates (the fixed-point area holds a BigGate).
__host__ __device__ inline Layout make_layout(int b, int G, int csize, bool batch = false, bool big = false) {
  Layout L;
  L.nv = 2 << b;
  L.G = G;
  L.hs = L.nv * 2 < kHashSlots ? L.nv * 2 : kHashSlots;
  L.dcap = L.nv < kHuffMaxD ? L.nv : kHuffMaxD;
  L.p2cap = next_pow2(L.dcap);
  uint32_t o = 0;
  L.off_q = o;
  o += (uint32_t)(G * L.nv * 4);
  L.off_vin_bits = o;
  o += (uint32_t)(G * kVmax * 8);
  L.off_vout_bits = o;
  o += (uint32_t)(G * kVmax * 8);
  L.off_vin_pos = o;
  o += (uint32_t)pad_to((size_t)G * kVmax * 2, 16);
  L.off_vout_pos = o;
  o += (uint32_t)pad_to((size_t)G * kVmax * 2, 16);
  L.off_hkey = o;
  o += (uint32_t)(L.hs * 4);
  L.off_hval = o;
  o += (uint32_t)(L.hs * 4);
  // stream image: header + largest body (PACK at 32 bits) + verbatim section
  L.stage_bytes = (uint32_t)pad_to(kHdr + (size_t)L.nv * 4 + 2 * kVmax + 8 + (size_t)kVmax * csize + 16, 16);
  if (big) o = (uint32_t)pad_to(o, 128);  // the stage doubles as a tensor-core operand tile
  L.off_stage = o;
  o += L.stage_bytes;
  // codebook build: keys, vals (p2cap each), internal weights (dcap), parent and its
  // ping-pong copy (2 dcap u16 each), depths and copy (2 dcap u8 each), rank-sort scratch
  // (2 x min(256, dcap) u32). Decode: table (2^kLutBits u32), chunk starts.
  L.off_wint = (uint32_t)(8 * L.p2cap);
  // the internal-weight array doubles as the table of 257 thread start bits (pass 2)
  L.off_parent = L.off_wint + (uint32_t)(4 * (L.dcap > 257 ? L.dcap : 257));
  L.off_parent2 = L.off_parent + (uint32_t)(4 * L.dcap);
  L.off_lens = L.off_parent2 + (uint32_t)(4 * L.dcap);
  L.off_lens2 = L.off_lens + (uint32_t)pad_to(2 * L.dcap, 4);
  L.sort_off = L.off_lens2 + (uint32_t)pad_to(2 * L.dcap, 4);
  L.sort_n = L.dcap < 256 ? L.dcap : 256;
  uint32_t build = L.sort_off + (uint32_t)(8 * L.sort_n);
  uint32_t dec = (uint32_t)(4 * (1 << kLutBits) + 4 * (L.nv / kChunkMin + 1));
  L.build_bytes = (uint32_t)pad_to(build > dec ? build : dec, 16);
  L.off_build = o;
  o += L.build_bytes;
  L.off_misc = o;
  o += (uint32_t)pad_to(sizeof(Misc), 16);  // scalars and scan workspace
  if (big) o = (uint32_t)pad_to(o, 128);    // tensor-core operand tables
  L.off_fast = o;
  o += (uint32_t)pad_to(big ? sizeof(BigGate) : sizeof(FastGate), 16);
  L.off_desc = o;  // the batched pass keeps the current state's descriptor here
  if (batch) o += (uint32_t)pad_to(sizeof(PassArgs), 16);
  L.off_vmask = o;  // complex64: one bit per value marks a verbatim value kept in place
  o += (uint32_t)pad_to((size_t)G * (L.nv / 32) * 4, 16);
  L.off_vtree = o;  // pairwise verbatim-square tree across threads
  o += 256 * 8;
  // complex128: output verbatim bitmap; per-word prefix counts of the input and output
  // bitmaps (ranks of verbatim values in their stream sections) live in the hash table's
  // space, which is idle while they are used (decode to transform; the second round)
  L.off_vomask = o;
  o += (uint32_t)pad_to((size_t)G * (L.nv / 32) * 4, 16);
  L.off_vpre_in = L.off_hkey;
  L.off_vpre_out = L.off_hkey + (uint32_t)pad_to((size_t)G * (L.nv / 32) * 2, 16);
  L.total = o;
  return L;
}

// Default CTA size: one thread per 32-value decode chunk, 32 to 256 threads. Any power of
// two T with 32 <= T <= 256 and 2 <= 2^(b+1) / T <= 32 works (threads beyond the chunk count
// idle while decoding); results do not depend on T.
__host__ __device__ inline bool threads_ok(int b, int t) {
  const int nv = 2 << b;
  return t >= 32 && t <= 256 && (t & (t - 1)) == 0 && nv / t >= 2 && nv / t <= 32;
}
// Huffman chunk size `chunk` works with CTA size T when every chunk has its decoding thread
// and spans whole threads' value runs: 2^(b+1) / chunk <= T.
__host__ __device__ inline bool chunk_ok(int b, int chunk, int t) {
  return (chunk == 16 || chunk == 32 || chunk == 64) && (2 << b) / chunk <= t;
}
__host__ __device__ inline int worker_threads(int b) {
  int nv = 2 << b;
  int t = nv / kChunkDefault;
  if (t > 256) t = 256;
  if (t < 32) t = 32;
  return t;
}

// Pairwise sum (every node fl(left + right)) of x*x over the aligned run [j0, j0 + vpt) of a
// block's values, x the value if it is verbatim and +0 otherwise. complex64 (mask, no ranks):
// verbatim values are flagged in `mask` with their float bits in the code slot q[j];
// complex128 with ranks (many verbatim values): `mask` flags them and their raw values sit in
// `sec` at their rank (prefix counts `pre`); complex128 otherwise: the (pos, bits) list.
// Kept out of line: it runs only for blocks with verbatim values, and its stack of pending
// subtrees stays out of the pass's registers.
template <typename Real>
__device__ __noinline__ double square_run(int j0, int vpt, const uint32_t* mask, const int32_t* q,
                                          const uint16_t* pre, const uint8_t* sec, int nlist,
                                          const uint16_t* lpos, const uint64_t* lbits) {
  constexpr bool kMask = sizeof(Real) == 4;
  double stk[7];
  int lvl[7], top = 0;
  for (int i = 0; i < vpt; ++i) {
    const int j = j0 + i;
    double x2 = 0.0;
    if (kMask) {
      if ((mask[j >> 5] >> (j & 31)) & 1u) {
        const double x = (double)__uint_as_float((uint32_t)q[j]);
        x2 = __dmul_rn(x, x);
      }
    } else if (pre) {
      const uint32_t wd = mask[j >> 5];
      if ((wd >> (j & 31)) & 1u) {
        const uint32_t rank = pre[j >> 5] + (uint32_t)__popc(wd & ((1u << (j & 31)) - 1u));
        const double x = __longlong_as_double(*(const long long*)(sec + 8 * rank));
        x2 = __dmul_rn(x, x);
      }
    } else {
      for (int e = 0; e < nlist; ++e)
        if (lpos[e] == j) {
          const double x = __longlong_as_double((long long)lbits[e]);
          x2 = __dmul_rn(x, x);
        }
    }
    double v = x2;
    int l = 0;
    while (top > 0 && lvl[top - 1] == l) {
      v = __dadd_rn(stk[top - 1], v);
      --top;
      ++l;
    }
    stk[top] = v;
    lvl[top] = l;
    ++top;
  }
  return stk[0];
}

template <typename Real>
struct Worker {
  Layout L;
  int T, vpt, b;
  int kc;  // Huffman chunk size of the state (symbols per stored chunk bit count)
  QuantP qp;
  int32_t* q;
  uint16_t *vin_pos, *vout_pos;
  uint64_t *vin_bits, *vout_bits;
  int *vin_cnt, *vout_cnt;
  uint32_t *hkey, *hval, *stage;
  uint8_t* build;
  Misc* m;
  // complex64 keeps verbatim values in place (float bits in the code slot, flagged here);
  // complex128 keeps them in the vin/vout lists (at most kVmax per block)
  static constexpr bool kMask = sizeof(Real) == 4;
  uint32_t* vmask;
  double* vtree;
  uint32_t* vomask;
  uint16_t *vpre_in, *vpre_out;

  __device__ __forceinline__ void init(unsigned char* smem, const Layout& lay, int b_, const QuantP& p) {
    L = lay;
    b = b_;
    T = blockDim.x;
    vpt = L.nv / T;
    kc = kChunkDefault;
    qp = p;
    q = (int32_t*)(smem + L.off_q);
    vin_bits = (uint64_t*)(smem + L.off_vin_bits);
    vout_bits = (uint64_t*)(smem + L.off_vout_bits);
    vin_pos = (uint16_t*)(smem + L.off_vin_pos);
    vout_pos = (uint16_t*)(smem + L.off_vout_pos);
    hkey = (uint32_t*)(smem + L.off_hkey);
    hval = (uint32_t*)(smem + L.off_hval);
    stage = (uint32_t*)(smem + L.off_stage);
    build = smem + L.off_build;
    m = (Misc*)(smem + L.off_misc);
    vmask = (uint32_t*)(smem + L.off_vmask);
    vtree = (double*)(smem + L.off_vtree);
    vomask = (uint32_t*)(smem + L.off_vomask);
    vpre_in = (uint16_t*)(smem + L.off_vpre_in);
    vpre_out = (uint16_t*)(smem + L.off_vpre_out);
    vin_cnt = m->vin_cnt;
    vout_cnt = m->vout_cnt;
  }

  // ------------------------------------------------------------------------------------
  // Decompress(S) for one block: stream -> q codes (verbatim slots hold kSentinel and
  // their raw values go to the vin list). The stream is first copied into the stage buffer
  // with 16-byte loads; every later read is from shared memory. Errors set m->err.
  // ------------------------------------------------------------------------------------
  __device__ __forceinline__ void decode(int g, const uint8_t* s, uint32_t len) {
    const int tid = threadIdx.x, nv = L.nv;
    int32_t* qb = q + g * nv;
    for (int i = tid; i < (nv >> 5); i += T) vmask[g * (nv >> 5) + i] = 0u;
    if (tid == 0) m->vin_big[g] = 0;
    // header and body are staged (they always fit); a complex64 verbatim section can be
    // longer than the stage and is read from the stream in global memory
    const bool fits = len >= kHdr && (len & 15) == 0;
    const uint32_t staged = fits ? (len < (L.stage_bytes & ~15u) ? len : (L.stage_bytes & ~15u)) : 0u;
    if (fits) {
      const uint4* src = (const uint4*)s;
      uint4* dst = (uint4*)stage;
      for (uint32_t i = tid; i < staged / 16; i += T) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    const uint8_t* sm = (const uint8_t*)stage;
    uint32_t h0 = 0, h1 = 0, h2 = 0, h3 = 0;
    if (fits) {
      h0 = stage[0];
      h1 = stage[1];
      h2 = stage[2];
      h3 = stage[3];
    }
    const int mode = h0 & 0xff, dt = (h0 >> 8) & 0xff, bl = (h0 >> 16) & 0xff, param = h0 >> 24;
    const int nverb = h1 & 0xffff, D = h1 >> 16;
    const int want_dt = sizeof(Real) == 8 ? 2 : 1;
    bool bad = !fits || dt != want_dt || bl != b || mode > kModePack;
    uint32_t body_end = kHdr;
    if (!bad && mode == kModeConst) {
      if (nverb != 0) bad = true;
      const int32_t qre = (int32_t)h2, qim = (int32_t)h3;
      for (int j = tid; j < nv; j += T) qb[j] = (j & 1) ? qim : qre;
      if (tid == 0) vin_cnt[g] = 0;
      __syncthreads();
      if (bad && tid == 0) atomicOr(&m->err, kStCorrupt);
      return;
    }
    const uint32_t pbits = h2, total = h3;
    if (!bad && (total > len || (total & 15))) bad = true;
    if (!bad && mode == kModePack) {
      const int width = param;
      if (width > 32 || pbits != (uint32_t)nv * (uint32_t)width) bad = true;
      const uint32_t nwords = (pbits + 31) / 32;
      body_end = kHdr + 4 * nwords;
      if (body_end > total || body_end > staged) bad = true;
      if (!bad) {
        const uint32_t* w = (const uint32_t*)(sm + kHdr);
        for (int i = 0; i < vpt; ++i) {
          const int j = tid * vpt + i;
          uint32_t z = 0;
          if (width) {
            const uint32_t pos = (uint32_t)j * (uint32_t)width, wi = pos >> 5, sh = pos & 31;
            const uint32_t a0 = w[wi], a1 = wi + 1 < nwords ? w[wi + 1] : 0u;
            const uint32_t pk = sh ? (a0 << sh) | (a1 >> (32 - sh)) : a0;
            z = pk >> (32 - width);
          }
          qb[j] = unzigzag(z);
        }
      }
    } else if (!bad && mode == kModeHuff) {
      const int lmax = param;
      const int C = nv / kc;
      const uint32_t off_sym = kHdr + (uint32_t)pad_to(2 * lmax, 4);
      const uint32_t off_chunk = off_sym + (uint32_t)pad_to(2 * D, 4);
      const uint32_t off_pay = off_chunk + (uint32_t)pad_to(2 * C, 4);
      const uint32_t nwords = (pbits + 31) / 32;
      body_end = off_pay + 4 * nwords;
      if (lmax < 1 || lmax > 24 || D < 1 || D > L.dcap || body_end > total || body_end > staged) bad = true;
      uint32_t* lut = (uint32_t*)build;
      uint32_t* cstart = (uint32_t*)(build + 4 * (1 << kLutBits));
      const uint16_t* symtab = (const uint16_t*)(sm + off_sym);
      if (!bad) {
        if (tid == 0) {
          int code = 0, idx = 0;
          const uint16_t* cnt = (const uint16_t*)(sm + kHdr);
          for (int l = 1; l <= lmax; ++l) {
            const int c = cnt[l - 1];
            m->first[l] = code;
            m->offs[l] = idx;
            m->lcount[l] = c;
            code = (code + c) << 1;
            idx += c;
          }
          if (idx != D) atomicOr(&m->err, kStCorrupt);
        }
      }
      uint32_t cb = 0;
      if (!bad && tid < C) cb = ((const uint16_t*)(sm + off_chunk))[tid];
      uint32_t ctot = 0;
      const uint32_t cs = block_excl_scan_u32(cb, m->scan, &ctot);  // syncs
      if (!bad && ctot != pbits) bad = true;
      if (!bad) {
        if (tid < C) cstart[tid] = cs;
        if (tid == 0) cstart[C] = pbits;
        // decode table, one entry per thread step: the kLutBits-bit prefix e starts the code
        // of length l <= kLutBits whose canonical value is e >> (kLutBits - l) (at most one l
        // matches: the code is prefix-free); entry (canonical index + 1) << 8 | length, or 0
        // when the code is longer
        // canonical codes left-justified to kLutBits bits increase with their length and index,
        // so the prefix e starts a code of length l exactly when lim[l-1] <= e < lim[l], with
        // lim[l] = (first[l] + lcount[l]) << (kLutBits - l) (an empty length repeats the
        // previous limit); the limits and the per-length bases live in registers
        const int lshort = lmax < kLutBits ? lmax : kLutBits;
        int lim[kLutBits + 1], base[kLutBits + 1];
#pragma unroll
        for (int l = 1; l <= kLutBits; ++l) {
          const int fl = l <= lshort ? m->first[l] : 0, lc = l <= lshort ? m->lcount[l] : 0;
          lim[l] = l <= lshort ? (fl + lc) << (kLutBits - l) : 0;
          base[l] = l <= lshort ? m->offs[l] - fl + 1 : 0;
        }
        for (int e = tid; e < (1 << kLutBits); e += T) {
          uint32_t v = 0;
#pragma unroll
          for (int l = kLutBits; l >= 1; --l)
            if (l <= lshort && e < lim[l]) v = ((uint32_t)(base[l] + (e >> (kLutBits - l))) << 8) | (uint32_t)l;
          lut[e] = v;
        }
      }
      __syncthreads();
      if (!bad && tid < C && !m->err) decode_chunk(qb + tid * kc, (const uint32_t*)(sm + off_pay), nwords,
                                                   cstart[tid], cstart[tid + 1], lut, symtab, D, lmax);
    }
    if (bad && tid == 0) atomicOr(&m->err, kStCorrupt);
    __syncthreads();
    // inverse Lorenzo: q_j = q_{j-2} + delta_j, one running sum per plane: each thread sums
    // its run, a block scan gives the run's offsets, then it reads the run again and writes the
    // codes (no run held in registers across the scan). Runs of 4 or more values move as
    // 16-byte words: a thread's run starts vpt words after its neighbour's, and word-wide
    // accesses at that stride would share banks vpt/2 ways.
    int32_t* run = qb + tid * vpt;
    const bool wide = (vpt & 3) == 0;
    int2 loc = make_int2(0, 0);
    if (wide) {
      for (int i = 0; i < vpt; i += 4) {
        const int4 v = *(const int4*)(run + i);
        loc.x += v.x;
        loc.y += v.y;
        loc.x += v.z;
        loc.y += v.w;
      }
    } else {
      for (int i = 0; i < vpt; i += 2) {
        const int2 v = *(const int2*)(run + i);
        loc.x += v.x;
        loc.y += v.y;
      }
    }
    int2 off = block_excl_scan_i2(loc, (int2*)m->red);  // syncs: every run is summed
    if (wide) {
      for (int i = 0; i < vpt; i += 4) {
        const int4 v = *(const int4*)(run + i);
        int4 o;
        off.x += v.x;
        o.x = off.x;
        off.y += v.y;
        o.y = off.y;
        off.x += v.z;
        o.z = off.x;
        off.y += v.w;
        o.w = off.y;
        *(int4*)(run + i) = o;
      }
    } else {
      for (int i = 0; i < vpt; i += 2) {
        const int2 v = *(const int2*)(run + i);
        off.x += v.x;
        off.y += v.y;
        *(int2*)(run + i) = make_int2(off.x, off.y);
      }
    }
    // verbatim section: ascending positions, then raw values (aligned to the value size)
    if (nverb > nv) {
      if (tid == 0) atomicOr(&m->err, kStCorrupt);
    } else if (nverb > 0 && !bad) {
      __syncthreads();
      read_verbatim(g, s, body_end, total, nverb);
      if (!kMask && nverb > kVmax) {
        // rank of a verbatim value = verbatim positions before it: per-word prefix counts
        __syncthreads();
        const int W = nv >> 5;  // <= blockDim.x (threads_ok)
        const uint32_t pc = tid < W ? (uint32_t)__popc(vmask[g * W + tid]) : 0u;
        uint32_t tot = 0;
        const uint32_t pre = block_excl_scan_u32(pc, m->scan, &tot);
        if (tid < W) vpre_in[g * W + tid] = (uint16_t)pre;
        if (tid == 0) {
          m->vin_big[g] = 1;
          m->vin_vals[g] = (const uint64_t*)(s + pad_to(body_end + 2 * nverb, 8));
        }
      }
    }
    if (tid == 0) vin_cnt[g] = (!kMask && nverb <= kVmax) ? nverb : 0;
    __syncthreads();
  }

  __device__ __forceinline__ void read_verbatim(int g, const uint8_t* sm, uint32_t posoff, uint32_t total,
                                                int nverb) {  // sm: the stream in global memory
    const uint32_t valoff = (uint32_t)pad_to(posoff + 2 * nverb, sizeof(Real));
    if (valoff + sizeof(Real) * nverb > total) {
      if (threadIdx.x == 0) atomicOr(&m->err, kStCorrupt);
      return;
    }
    for (int i = threadIdx.x; i < nverb; i += T) {
      const int j = ((const uint16_t*)(sm + posoff))[i];
      uint64_t bits;
      if (sizeof(Real) == 8) bits = ((const uint64_t*)(sm + valoff))[i];
      else bits = ((const uint32_t*)(sm + valoff))[i];
      if (j >= L.nv) {
        atomicOr(&m->err, kStCorrupt);
      } else if (kMask) {
        q[g * L.nv + j] = (int32_t)(uint32_t)bits;
        atomicOr(&vmask[g * (L.nv >> 5) + (j >> 5)], 1u << (j & 31));
      } else if (nverb > kVmax) {  // looked up by rank in the stream (value_at)
        q[g * L.nv + j] = kSentinel;
        atomicOr(&vmask[g * (L.nv >> 5) + (j >> 5)], 1u << (j & 31));
      } else {
        vin_pos[g * kVmax + i] = (uint16_t)j;
        vin_bits[g * kVmax + i] = bits;
        q[g * L.nv + j] = kSentinel;
      }
    }
  }

  // One K-symbol chunk of a Huffman payload (shared-memory words), through a 64-bit bit
  // buffer that holds at least 32 unread bits before every symbol. The deltas leave in
  // 16-byte words of four (chunks start K words apart, so word-wide stores of all threads
  // would share one bank).
  __device__ __forceinline__ void decode_chunk(int32_t* out, const uint32_t* w, uint32_t nwords,
                                               uint32_t pos, uint32_t end, const uint32_t* lut,
                                               const uint16_t* symtab, int D, int lmax) {
    uint32_t wi = pos >> 5;
    const int sh = (int)(pos & 31);
    const uint64_t w0 = wi < nwords ? w[wi] : 0u, w1 = wi + 1 < nwords ? w[wi + 1] : 0u;
    uint64_t buf = ((w0 << 32) | w1) << sh;
    int nbuf = 64 - sh;
    wi += 2;
    bool cerr = false;
    for (int i4 = 0; i4 < kc && !cerr; i4 += 4) {
      int32_t r4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (nbuf < 32) {
          buf |= (uint64_t)(wi < nwords ? w[wi] : 0u) << (32 - nbuf);
          ++wi;
          nbuf += 32;
        }
        const uint32_t pk = (uint32_t)(buf >> 32);
        const uint32_t e = lut[pk >> (32 - kLutBits)];
        int idx = -1, l = 0;
        if (e) {
          idx = (int)(e >> 8) - 1;
          l = (int)(e & 0xff);
        } else {
          for (l = kLutBits + 1; l <= lmax; ++l) {
            const int c = (int)(pk >> (32 - l));
            if (m->lcount[l] && c >= m->first[l] && c - m->first[l] < m->lcount[l]) {
              idx = m->offs[l] + c - m->first[l];
              break;
            }
          }
        }
        if (idx < 0 || idx >= D) {
          cerr = true;
          r4[u] = 0;
          continue;
        }
        buf <<= l;
        nbuf -= l;
        pos += (uint32_t)l;
        const int sym = symtab[idx];
        int32_t d;
        if (sym == 0) {
          if (nbuf < 32) {
            buf |= (uint64_t)(wi < nwords ? w[wi] : 0u) << (32 - nbuf);
            ++wi;
            nbuf += 32;
          }
          d = (int32_t)(uint32_t)(buf >> 32);
          buf <<= 32;
          nbuf -= 32;
          pos += 32;
        } else {
          d = sym - 32768;
        }
        r4[u] = d;
      }
      *(int4*)(out + i4) = make_int4(r4[0], r4[1], r4[2], r4[3]);
    }
    if (cerr || pos != end) atomicOr(&m->err, kStCorrupt);
  }

  // Basis input: every code 0 except the value 1.0 at `pos` (given raw, as verbatim input).
  __device__ __forceinline__ void load_basis(int g, int pos) {
    const int tid = threadIdx.x;
    int32_t* qb = q + g * L.nv;
    for (int j = tid; j < L.nv; j += T) qb[j] = 0;
    for (int i = tid; i < (L.nv >> 5); i += T) vmask[g * (L.nv >> 5) + i] = 0u;
    if (tid == 0) m->vin_big[g] = 0;
    __syncthreads();
    if (kMask) {
      if (tid == 0) {
        vin_cnt[g] = 0;
        if (pos >= 0) {  // the value 1.0, given raw
          qb[pos] = (int32_t)RawBits<Real>::to((Real)1.0);
          vmask[g * (L.nv >> 5) + (pos >> 5)] |= 1u << (pos & 31);
        }
      }
      __syncthreads();
      return;
    }
    if (tid == 0) {
      if (pos >= 0) {
        qb[pos] = kSentinel;
        vin_pos[g * kVmax] = (uint16_t)pos;
        vin_bits[g * kVmax] = RawBits<Real>::to((Real)1.0);
        vin_cnt[g] = 1;
      } else {
        vin_cnt[g] = 0;
      }
    }
    __syncthreads();
  }

  __device__ __forceinline__ bool is_verb(int g, int j) const {
    return kMask && ((vmask[g * (L.nv >> 5) + (j >> 5)] >> (j & 31)) & 1u);
  }

  // code of value j for prediction (verbatim values count as 0)
  __device__ __forceinline__ int32_t code(int g, int j) const {
    return is_verb(g, j) ? 0 : q[g * L.nv + j];
  }

  __device__ __forceinline__ Real value_at(int g, int j) const {
    const int32_t c = q[g * L.nv + j];
    if (kMask) return is_verb(g, j) ? RawBits<Real>::from((uint32_t)c) : dequant<Real>(c, qp);
    if (c != kSentinel) return dequant<Real>(c, qp);
    if (m->vin_big[g]) {
      const int W = L.nv >> 5;
      const uint32_t wd = vmask[g * W + (j >> 5)];
      const uint32_t rank = vpre_in[g * W + (j >> 5)] + (uint32_t)__popc(wd & ((1u << (j & 31)) - 1u));
      return RawBits<Real>::from(__ldg(m->vin_vals[g] + rank));
    }
    const int n = vin_cnt[g];
    for (int i = 0; i < n; ++i)
      if (vin_pos[g * kVmax + i] == j) return RawBits<Real>::from(vin_bits[g * kVmax + i]);
    return (Real)0;
  }

  // Hash slot of a symbol that the histogram inserted; L.hs (and an error flag) when it is
  // missing, which only a logic error can cause: the probe is bounded either way.
  __device__ __forceinline__ uint32_t find_slot(uint32_t sym) const {
    uint32_t h = hash_sym(sym) & (uint32_t)(L.hs - 1);
    for (int probe = 0; probe < L.hs; ++probe) {
      const uint32_t k = hkey[h];
      if (k == sym) return h;
      if (k == kEmpty) break;
      h = (h + 1) & (uint32_t)(L.hs - 1);
    }
    atomicOr(&m->err, kStInternal);
    return (uint32_t)L.hs;
  }

  // Add `cnt` occurrences of symbol `sym` to the histogram's hash table, unless the block
  // already has more distinct symbols than Huffman mode takes (m->D then exceeds kHuffMaxD
  // and the block is packed).
  __device__ __forceinline__ void hash_add(uint32_t sym, uint32_t cnt) {
    if (*(volatile int*)&m->D > kHuffMaxD) return;
    uint32_t hslot = hash_sym(sym) & (uint32_t)(L.hs - 1);
    for (int probe = 0; probe < L.hs; ++probe) {
      const uint32_t k = hkey[hslot];
      if (k == sym) {
        atomicAdd(&hval[hslot], cnt);
        return;
      }
      if (k == kEmpty) {
        const uint32_t old = atomicCAS(&hkey[hslot], kEmpty, sym);
        if (old == kEmpty) {
          atomicAdd(&m->D, 1);
          atomicAdd(&hval[hslot], cnt);
          return;
        }
        if (old == sym) {
          atomicAdd(&hval[hslot], cnt);
          return;
        }
      }
      hslot = (hslot + 1) & (uint32_t)(L.hs - 1);
    }
  }

  // Quantize one result into slot g position j (Compress(S), first step).
  __device__ __forceinline__ void put_value(int g, int j, Real v) {
    int32_t c;
    if (kMask) {
      uint32_t* w = &vmask[g * (L.nv >> 5) + (j >> 5)];
      if (quantize<Real>(v, qp, &c)) {
        q[g * L.nv + j] = (int32_t)(uint32_t)RawBits<Real>::to(v);
        atomicOr(w, 1u << (j & 31));
      } else {
        q[g * L.nv + j] = c;
        atomicAnd(w, ~(1u << (j & 31)));
      }
      return;
    }
    const bool verb = quantize<Real>(v, qp, &c);
    if (m->fix) {  // second transform of a block with many verbatim values: raw values only
      if (verb && m->vbig[g]) {
        const int W = L.nv >> 5;
        const uint32_t wd = vomask[g * W + (j >> 5)];
        const uint32_t rank = vpre_out[g * W + (j >> 5)] + (uint32_t)__popc(wd & ((1u << (j & 31)) - 1u));
        *(uint64_t*)(m->vsec_base[g] + m->vsec_valoff[g] + 8 * rank) = RawBits<Real>::to(v);
      }
      return;
    }
    if (verb) {
      const int i = atomicAdd(&vout_cnt[g], 1);
      if (i < kVmax) {
        vout_pos[g * kVmax + i] = (uint16_t)j;
        vout_bits[g * kVmax + i] = RawBits<Real>::to(v);
      }
      atomicOr(&vomask[g * (L.nv >> 5) + (j >> 5)], 1u << (j & 31));
      c = 0;
    }
    q[g * L.nv + j] = c;
  }

  // ------------------------------------------------------------------------------------
  // Compress(S) for one block: q codes + verbatim list -> stream in the output arena.
  // ------------------------------------------------------------------------------------
  __device__ __forceinline__ void encode(int g, unsigned long long blk, const PassArgs& a);

  // Re-emit the input stream of block sb as the output stream of block db: the pass has
  // been shown to reproduce sb's codes exactly at db's positions, and encoding is a function
  // of the codes alone, so the recoded stream would be these bytes. The norm partial and
  // statistics come from sb's summary, as the recode would have added them.
  __device__ __forceinline__ void pass_through(unsigned long long sb, unsigned long long db, const PassArgs& a) {
    const int tid = threadIdx.x;
    const uint32_t len = a.in_len[sb];
    if (tid == 0) {
      const unsigned long long off = atomicAdd(&a.sc->bump[a.out_id], (unsigned long long)len);
      m->out_off = off;
      m->ok = off + len <= a.out_cap;
      if (!m->ok) {
        atomicOr(&a.sc->status, kStOverflow);
        atomicMin(&a.sc->fail_seq, a.seq);
      }
      const BlkInfo bi = a.in_info[sb];
      const unsigned long long lo = bi.sq_lo, hi = bi.sq_hi_nesc & 0xFFu;
      const unsigned long long old = atomicAdd(&a.sc->acc.sq_lo, lo);
      const unsigned long long c1 = (old + lo < old) ? 1ull : 0ull;
      if (hi + c1) atomicAdd(&a.sc->acc.sq_hi, hi + c1);
      const int mode = (int)((bi.maxq_mode >> 29) & 3u);
      if (mode != kModeConst) atomicAdd(&a.sc->acc.n_escape, (unsigned long long)(bi.sq_hi_nesc >> 8));
      atomicAdd(&a.sc->acc.modes[mode], 1ull);
      atomicAdd(&a.sc->acc.reused, 1ull);
      a.out_info[db] = bi;
      if (a.vsum) a.vsum[db] = 0.0;
    }
    __syncthreads();
    if (m->ok) {
      const uint4* src = (const uint4*)(a.in_arena + a.in_off[sb]);
      uint4* dst = (uint4*)(a.out_arena + m->out_off);
      for (uint32_t i = tid; i < len / 16; i += T) dst[i] = src[i];
      if (tid == 0) {
        a.out_off[db] = m->out_off;
        a.out_len[db] = len;
      }
    }
    __syncthreads();
  }

  // complex128 second round: rank of every output verbatim position of block g (per-word
  // prefix counts of the output bitmap). All threads call it.
  __device__ __forceinline__ void prepare_out_ranks(int g) {
    const int W = L.nv >> 5;  // <= blockDim.x
    const uint32_t pc = (int)threadIdx.x < W ? (uint32_t)__popc(vomask[g * W + threadIdx.x]) : 0u;
    uint32_t tot = 0;
    const uint32_t pre = block_excl_scan_u32(pc, m->scan, &tot);
    if ((int)threadIdx.x < W) vpre_out[g * W + threadIdx.x] = (uint16_t)pre;
    __syncthreads();
  }

  // complex64: write the verbatim section (u16 positions ascending, raw floats) of block g
  // into its stream at `out`, after the zero fill of the section
  // (complex128 with many verbatim values: positions now; the section's address is kept for
  // the second transform that writes the raw values)
  __device__ __forceinline__ void write_verbatim_inplace(int g, uint8_t* out, uint32_t body_end, int nverb) {
    const int tid = threadIdx.x, nv = L.nv, j0 = tid * vpt;
    const uint32_t* bm = kMask ? vmask : vomask;
    const uint32_t w = bm[g * (nv >> 5) + (j0 >> 5)];
    const uint32_t mine = vpt >= 32 ? w : ((w >> (j0 & 31)) & ((1u << vpt) - 1u));
    uint32_t tot = 0;
    uint32_t k = block_excl_scan_u32((uint32_t)__popc(mine), m->scan, &tot);
    const uint32_t valoff = (uint32_t)pad_to(body_end + 2 * nverb, sizeof(Real));
    if (!kMask && tid == 0) {
      m->vsec_base[g] = out;
      m->vsec_valoff[g] = valoff;
    }
    for (int i = 0; i < vpt; ++i) {
      if (!((mine >> i) & 1u)) continue;
      const int j = j0 + i;
      *(uint16_t*)(out + body_end + 2 * k) = (uint16_t)j;
      if (kMask) *(uint32_t*)(out + valoff + 4 * k) = (uint32_t)q[g * nv + j];
      ++k;
    }
  }

  // Pairwise sum of x*x over the block's values (x verbatim) and +0 (others), level by
  // level: each thread reduces its aligned run of vpt values (square_run, below), then the
  // runs are reduced across threads. All threads call it; the result is returned to all.
  __device__ __forceinline__ double verbatim_square_tree(int g) {
    const int tid = threadIdx.x, nv = L.nv, W = nv >> 5;
    const double top = square_run<Real>(tid * vpt, vpt, kMask ? vmask + g * W : vomask + g * W,
                                        q + g * nv, (!kMask && m->vbig[g]) ? vpre_out + g * W : nullptr,
                                        kMask ? nullptr : m->vsec_base[g] + m->vsec_valoff[g],
                                        vout_cnt[g] < kVmax ? vout_cnt[g] : kVmax, vout_pos + g * kVmax,
                                        vout_bits + g * kVmax);
    vtree[tid] = top;
    __syncthreads();
    for (int cnt = T; cnt > 1; cnt >>= 1) {
      const int half = cnt >> 1;
      double v = 0.0;
      if (tid < half) v = __dadd_rn(vtree[2 * tid], vtree[2 * tid + 1]);
      __syncthreads();
      if (tid < half) vtree[tid] = v;
      __syncthreads();
    }
    const double r = vtree[0];
    __syncthreads();
    return r;
  }
};

// Two-queue Huffman merge over D >= 2 leaves sorted by (frequency, symbol) in keys (frequency
// in the upper 16 bits): each step joins the two lightest queue heads, the leaf queue first on
// equal weight. Writes parent[v] for every node but the root (2D - 2), and wint[k] (internal
// node k = node D + k) for the nodes formed before the last leaf is consumed.
//
// In rounds rather than D - 1 serial steps. The steps consume the nodes in the order of S, the
// merge of the leaf list with the internal-node list (leaves first on equal weight), and
// internal node k joins S[2k] and S[2k + 1]. With m entries of S placed, the internal nodes
// 0 .. m/2 - 1 are known, and every node not yet formed weighs at least thr = S[m-1] + v0
// (m odd) or v0 + v1 (m even), v0 <= v1 the two lightest nodes available now. Every available
// node of weight <= thr therefore precedes every unformed one (a leaf wins a tie; a known internal
// node was formed earlier), so one round places all of them at once, each at its merge
// position, and forms the internal nodes their pairs complete. thr at least doubles every
// round, so a block (total weight < 2^16) needs at most 17 rounds; once the last leaf is
// placed the remaining pairs are fixed by position and need no round. One warp runs the rounds
// (warp votes and warp barriers only); the CTA waits once, after it. sw, sid: scratch for S
// (weights and node ids, 2D - 2 entries each).
__device__ inline void huffman_merge(const uint32_t* keys, int D, uint32_t* wint, uint16_t* parent,
                                     uint32_t* sw, uint16_t* sid) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int m = 0, lp = 0, ip = 0;  // S entries placed, leaves and internal nodes consumed (uniform)
    while (m < 2 * D - 2) {
      const int nk = m >> 1;  // internal nodes formed
      if (lp == D) {
        // every leaf is placed: the rest of S is the internal-node queue in order, so the
        // entry at position p >= m is internal node p - D (node id p), and every pair
        // (2k, 2k + 1) from 2 nk on forms internal node k without any weight being needed
        for (int p = 2 * nk + lane; p < 2 * D - 2; p += 32) parent[p < m ? sid[p] : p] = (uint16_t)(D + (p >> 1));
        __syncwarp();
        break;
      }
      // the next 32 nodes of each queue (one load each) and the pending entry S[m - 1]
      constexpr unsigned kAll = 0xffffffffu;
      const uint32_t kl = lp + lane < D ? keys[lp + lane] >> 16 : 0xFFFFFFFFu;
      const uint32_t wl = ip + lane < nk ? wint[ip + lane] : 0xFFFFFFFFu;
      const uint32_t pend = (m & 1) ? sw[m - 1] : 0u;
      const uint32_t l0 = __shfl_sync(kAll, kl, 0), l1 = __shfl_sync(kAll, kl, 1);
      const uint32_t i0 = __shfl_sync(kAll, wl, 0), i1 = __shfl_sync(kAll, wl, 1);
      // v0 <= v1: the two lightest available nodes (a leaf first on equal weight). The next
      // internal node joins S[m - 1] and v0 (m odd) or v0 and v1 (m even), and no node
      // formed after it is lighter: thr bounds every node not yet formed from below.
      uint32_t v0, v1;
      if (l0 <= i0) {
        v0 = l0;
        v1 = l1 < i0 ? l1 : i0;
      } else {
        v0 = i0;
        v1 = i1 < l0 ? i1 : l0;
      }
      const uint32_t thr = (m & 1) ? pend + v0 : (v1 != 0xFFFFFFFFu ? v0 + v1 : 2u * v0);
      // available nodes at or below thr (each list is sorted, so they form prefixes)
      unsigned vb = __ballot_sync(kAll, kl <= thr);
      int cl = __popc(vb);
      for (int t0 = 32; vb == kAll && t0 < D - lp; t0 += 32) {
        vb = __ballot_sync(kAll, t0 + lane < D - lp && (keys[lp + t0 + lane] >> 16) <= thr);
        cl += __popc(vb);
      }
      vb = __ballot_sync(kAll, wl <= thr);
      int ci = __popc(vb);
      for (int t0 = 32; vb == kAll && t0 < nk - ip; t0 += 32) {
        vb = __ballot_sync(kAll, t0 + lane < nk - ip && wint[ip + t0 + lane] <= thr);
        ci += __popc(vb);
      }
      // merge positions: a leaf follows the internal nodes lighter than it, an internal node
      // follows the leaves not heavier than it
      for (int t = lane; t < cl; t += 32) {
        const uint32_t x = keys[lp + t] >> 16;
        int lo = ip, hi = ip + ci;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (wint[mid] < x) lo = mid + 1;
          else hi = mid;
        }
        sw[m + t + (lo - ip)] = x;
        sid[m + t + (lo - ip)] = (uint16_t)(lp + t);
      }
      for (int t = lane; t < ci; t += 32) {
        const uint32_t x = wint[ip + t];
        int lo = lp, hi = lp + cl;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if ((keys[mid] >> 16) <= x) lo = mid + 1;
          else hi = mid;
        }
        sw[m + t + (lo - lp)] = x;
        sid[m + t + (lo - lp)] = (uint16_t)(D + ip + t);
      }
      __syncwarp();
      const int mn = m + cl + ci;
      for (int k = nk + lane; k < (mn >> 1); k += 32) {
        wint[k] = sw[2 * k] + sw[2 * k + 1];
        parent[sid[2 * k]] = (uint16_t)(D + k);
        parent[sid[2 * k + 1]] = (uint16_t)(D + k);
      }
      __syncwarp();
      m = mn;
      lp += cl;
      ip += ci;
    }
  }
  __syncthreads();
}

// Depth of every node of the merged tree by pointer jumping (all threads): d[v] += d[p[v]],
// p[v] = p[p[v]], ping-ponging between two copies. A tree over D leaves is at most D - 1
// deep, and a Huffman tree over the <= 8192 symbols of a block at most 18 (a code of length L
// needs total weight >= Fibonacci(L + 2)); after k rounds every node has jumped 2^k levels, so
// the first k with 2^k >= min(D - 1, 18) suffices. Returns the array holding the depths.
__device__ inline uint8_t* tree_depths(int D, uint16_t* parent, uint8_t* depth, uint16_t* parent2,
                                       uint8_t* depth2) {
  const int total = 2 * D - 1, root = total - 1;
  for (int v = threadIdx.x; v < total; v += blockDim.x) {
    depth[v] = v == root ? 0 : 1;
    if (v == root) parent[v] = (uint16_t)root;
  }
  __syncthreads();
  const int maxd = D - 1 < 18 ? D - 1 : 18;
  int rounds = 0;
  while ((1 << rounds) < maxd) ++rounds;
  uint16_t *pa = parent, *pb = parent2;
  uint8_t *da = depth, *db = depth2;
  for (int round = 0; round < rounds; ++round) {
    for (int v = threadIdx.x; v < total; v += blockDim.x) {
      const int p = pa[v];
      db[v] = (uint8_t)(da[v] + da[p]);
      pb[v] = pa[p];
    }
    __syncthreads();
    uint16_t* tp = pa;
    pa = pb;
    pb = tp;
    uint8_t* td = da;
    da = db;
    db = td;
  }
  return da;
}

// Sort n (key, val) pairs ascending by key (keys distinct). Up to 256: every element finds
// its rank in one pass (scratch tk/tv); larger lists: bitonic over the padded power p2.
__device__ inline void sort_pairs(uint32_t* key, uint32_t* val, int n, int p2, uint32_t* tk,
                                  uint32_t* tv) {
  if (n <= 256) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t k = key[i];
      int r = 0;
      for (int j = 0; j < n; ++j) r += key[j] < k;
      tk[r] = k;
      tv[r] = val[i];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      key[i] = tk[i];
      val[i] = tv[i];
    }
    __syncthreads();
  } else {
    bitonic_sort(key, val, p2);
  }
}

template <typename Real>
__device__ __forceinline__ void Worker<Real>::encode(int g, unsigned long long blk, const PassArgs& a) {
  const int tid = threadIdx.x, nv = L.nv;
  const int32_t* qb = q + g * nv;
  int nverb_raw, nverb;
  if (kMask) {  // verbatim values flagged in place: count the flags
    const unsigned long long c1 = tid < (nv >> 5) ? (unsigned long long)__popc(vmask[g * (nv >> 5) + tid]) : 0ull;
    nverb_raw = nverb = (int)block_reduce_sum_u64(c1, m->red);
  } else {
    nverb_raw = nverb = vout_cnt[g];
  }
  // complex128 with more verbatim values than the lists hold: the section goes straight to
  // the output like complex64's; the raw values come from a second transform (pass_group)
  const bool big = !kMask && nverb > kVmax;
  const int C = nv / kc;
  // ---- pass 1: statistics and the symbol histogram over this thread's values ----
  // Symbols near 32768 (small deltas) are counted in direct bins in the stage buffer, which
  // is idle until the stream image is assembled; the others go to the hash table (runs of
  // equal symbols merged before an insert; inserts stop once the block has more distinct
  // symbols than Huffman mode takes). After the pass every nonzero bin enters the hash table
  // with its count, so the codebook build and the code lookup see one table.
  uint32_t* bins = stage;
  int nbin = kBinsMax;
  while (nbin > 32 && (uint32_t)nbin * 4u > L.stage_bytes) nbin >>= 1;
  const uint32_t bin0 = 32768u - (uint32_t)(nbin >> 1);  // symbol of bin 0
  for (int i = tid; i < L.hs; i += T) {
    hkey[i] = kEmpty;
    hval[i] = 0;
  }
  for (int i = tid; i < nbin; i += T) bins[i] = 0;
  if (tid == 0) {
    m->D = 0;
    m->cnt = 0;
  }
  __syncthreads();
  const int j0 = tid * vpt;
  const int32_t q0 = qb[0], q1 = qb[1];
  BlkStats bs;
  bs.sqh = bs.sql = 0;
  bs.zmax = bs.amax = 0;
  bs.nesc = 0;
  bs.cst = 1;
  {
    // Every quantity of this pass is independent of the order in which a thread visits its
    // run, so thread t starts at offset (lane(t) * vpt / 32) of its run and wraps around: the
    // 32 lanes of a warp then read 32 different banks at every step (runs start vpt words
    // apart, and in-order visits would share banks vpt/2 ways). d_j = c_j - c_{j-2} reads both
    // codes from shared memory.
    const int rot = ((tid & 31) * vpt) >> 5;
    uint32_t run_sym = 0xFFFFFFFFu, run = 0;
    for (int k = 0; k <= vpt; ++k) {
      uint32_t sym = 0xFFFFFFFEu;
      if (k < vpt) {
        const int j = j0 + ((k + rot) & (vpt - 1));
        const int32_t c = code(g, j);
        const int32_t d = c - (j >= 2 ? code(g, j - 2) : 0);
        const uint64_t s2 = (uint64_t)((int64_t)c * (int64_t)c);
        bs.sqh += s2 >> 32;
        bs.sql += s2 & 0xffffffffull;
        const uint32_t z = zigzag(d);
        bs.zmax = z > bs.zmax ? z : bs.zmax;
        const uint32_t ac = (uint32_t)(c < 0 ? -c : c);
        bs.amax = ac > bs.amax ? ac : bs.amax;
        const bool esc = d < -kRadius || d > kRadius;
        bs.nesc += esc ? 1 : 0;
        bs.cst &= (c == ((j & 1) ? q1 : q0)) ? 1 : 0;
        sym = esc ? 0u : (uint32_t)(d + 32768);
      }
      if (sym == run_sym) {
        run++;
        continue;
      }
      if (run) {
        if (run_sym - bin0 < (uint32_t)nbin) atomicAdd(&bins[run_sym - bin0], run);
        else hash_add(run_sym, run);
      }
      run_sym = sym;
      run = 1;
    }
  }
  block_reduce_stats(bs, (BlkStats*)m->red);  // syncs: every value is counted after it
  for (int i = tid; i < nbin; i += T)
    if (bins[i]) hash_add(bin0 + (uint32_t)i, bins[i]);
  __syncthreads();
  const bool is_const = bs.cst && nverb_raw == 0;
  const unsigned long long Sh = bs.sqh, Sl = bs.sql;
  uint32_t amax = bs.amax;
  const int nesc_blk = bs.nesc;
  int mode = kModeConst, lmax = 0, width = 0, D = 0;
  uint32_t pbits = 0, body = 0;
  uint32_t* keys = (uint32_t*)build;
  uint32_t* vals = (uint32_t*)(build + 4 * L.p2cap);
  uint32_t* wint = (uint32_t*)(build + L.off_wint);
  uint16_t* parent = (uint16_t*)(build + L.off_parent);
  uint16_t* parent2 = (uint16_t*)(build + L.off_parent2);
  uint8_t* lens = build + L.off_lens;
  uint8_t* lens2 = build + L.off_lens2;
  uint32_t* tsk = (uint32_t*)(build + L.sort_off);  // rank-sort scratch
  uint32_t* tsv = tsk + L.sort_n;
  if (!is_const) {
    width = bit_width(bs.zmax);
    const uint32_t pack_body = 4u * (((uint32_t)nv * (uint32_t)width + 31u) / 32u);
    D = m->D;
    const int ne = nesc_blk;
    bool use_huff = false;
    if (D <= L.dcap && D <= kHuffMaxD) {
      const int P2 = next_pow2(D);
      for (int i = tid; i < L.hs; i += T) {
        if (hkey[i] != kEmpty) {
          const int k = atomicAdd(&m->cnt, 1);
          keys[k] = (hval[i] << 16) | hkey[i];
          vals[k] = (uint32_t)i;
        }
      }
      __syncthreads();
      for (int i = D + tid; i < P2; i += T) {
        keys[i] = 0xFFFFFFFFu;
        vals[i] = 0;
      }
      __syncthreads();
      sort_pairs(keys, vals, D, P2, tsk, tsv);
      if (D == 1) {
        if (tid == 0) lens[0] = 1;
      } else {
        // S of the merge in the rank-sort scratch (weights) and the second parent array (ids),
        // both idle until the depth computation
        huffman_merge(keys, D, wint, parent, tsk, parent2);
        lens = tree_depths(D, parent, lens, parent2, lens2);
      }
      if (tid == 0) m->lmax = 0;
      __syncthreads();
      for (int i = tid; i < D; i += T) atomicMax(&m->lmax, (int)lens[i]);
      __syncthreads();
      lmax = m->lmax;
      unsigned long long pb = 0;
      for (int i = tid; i < D; i += T) pb += (unsigned long long)(keys[i] >> 16) * lens[i];
      pb = block_reduce_sum_u64(pb, m->red) + 32ull * (unsigned long long)ne;
      pbits = (uint32_t)pb;
      const uint32_t huff_body = (uint32_t)(pad_to(2 * lmax, 4) + pad_to(2 * D, 4) +
                                            pad_to(2 * C, 4) + 4 * ((pb + 31) / 32));
      use_huff = huff_body < pack_body;
      if (use_huff) {
        body = huff_body;
        // canonical order: (length, symbol) ascending
        if (tid < 34) m->lcount[tid] = 0;
        for (int i = tid; i < D; i += T) keys[i] = ((uint32_t)lens[i] << 16) | (keys[i] & 0xFFFFu);
        __syncthreads();
        for (int i = tid; i < D; i += T) atomicAdd(&m->lcount[lens[i]], 1);
        sort_pairs(keys, vals, D, P2, tsk, tsv);
        if (tid == 0) {
          int code = 0, idx = 0;
          for (int l = 1; l <= lmax; ++l) {
            m->first[l] = code;
            m->offs[l] = idx;
            code = (code + m->lcount[l]) << 1;
            idx += m->lcount[l];
          }
        }
        __syncthreads();
        for (int i = tid; i < D; i += T) {
          const int l = (int)(keys[i] >> 16);
          const uint32_t code = (uint32_t)(m->first[l] + (i - m->offs[l]));
          hval[vals[i]] = (code << 5) | (uint32_t)l;
        }
        __syncthreads();
      }
    }
    if (use_huff) {
      mode = kModeHuff;
    } else {
      mode = kModePack;
      body = pack_body;
      pbits = (uint32_t)nv * (uint32_t)width;
    }
  }
  // ---- size and allocation ----
  const uint32_t body_end = kHdr + body;
  uint32_t size;
  if (mode == kModeConst) size = kHdr;
  else size = (uint32_t)pad_to(pad_to(body_end + 2 * nverb, sizeof(Real)) + sizeof(Real) * nverb, 16);
  if (tid == 0) {
    const unsigned long long off = atomicAdd(&a.sc->bump[a.out_id], (unsigned long long)size);
    m->out_off = off;
    m->ok = off + size <= a.out_cap;
    if (!m->ok) {
      atomicOr(&a.sc->status, kStOverflow);
      atomicMin(&a.sc->fail_seq, a.seq);
    }
  }
  __syncthreads();
  const bool ok = m->ok;
  // complex64: the stream image in shared memory ends with the body; the verbatim section is
  // written straight to the output (it can be as large as the whole block)
  const uint32_t span = ((kMask || big) && mode != kModeConst) ? (uint32_t)pad_to(body_end, 16) : size;
  if (ok) {
    for (uint32_t i = tid; i < span / 4; i += T) stage[i] = 0;
    __syncthreads();
    if (tid == 0) {
      const int want_dt = sizeof(Real) == 8 ? 2 : 1;
      const int param = mode == kModeHuff ? lmax : (mode == kModePack ? width : 0);
      stage[0] = (uint32_t)mode | ((uint32_t)want_dt << 8) | ((uint32_t)b << 16) | ((uint32_t)param << 24);
      stage[1] = (uint32_t)nverb | ((uint32_t)(mode == kModeHuff ? D : 0) << 16);
      if (mode == kModeConst) {
        stage[2] = (uint32_t)q0;
        stage[3] = (uint32_t)q1;
      } else {
        stage[2] = pbits;
        stage[3] = size;
      }
    }
    if (mode != kModeConst) {
      uint32_t* pay;
      if (mode == kModeHuff) {
        uint16_t* st16 = (uint16_t*)stage;
        const uint32_t off_sym = kHdr + (uint32_t)pad_to(2 * lmax, 4);
        const uint32_t off_chunk = off_sym + (uint32_t)pad_to(2 * D, 4);
        const uint32_t off_pay = off_chunk + (uint32_t)pad_to(2 * C, 4);
        for (int l = tid + 1; l <= lmax; l += T) st16[kHdr / 2 + l - 1] = (uint16_t)m->lcount[l];
        for (int i = tid; i < D; i += T) st16[off_sym / 2 + i] = (uint16_t)(keys[i] & 0xFFFFu);
        // pass 2: bits per thread, then positions. Without escapes (and without complex64
        // verbatim values, whose raw bits live in the code slots) each value's code word
        // replaces its code in place, so the bit writer needs no second lookup.
        const bool keep_cw = nesc_blk == 0 && (!kMask || nverb_raw == 0);
        uint32_t nb = 0;
        {
          int32_t pr2 = j0 >= 2 ? code(g, j0 - 2) : 0, pi2 = j0 >= 2 ? code(g, j0 - 1) : 0;
          __syncthreads();  // every thread has its two preceding codes before any slot is rewritten
          int32_t* qw = q + g * nv;
          for (int i = 0; i < vpt; ++i) {
            const int j = j0 + i;
            const int32_t c = code(g, j);
            const int32_t d = c - ((j & 1) ? pi2 : pr2);
            if (j & 1) pi2 = c;
            else pr2 = c;
            const uint32_t sym = (d < -kRadius || d > kRadius) ? 0u : (uint32_t)(d + 32768);
            const uint32_t hs_ = find_slot(sym);
            const uint32_t cl = hs_ < (uint32_t)L.hs ? hval[hs_] : 0u;
            nb += (cl & 31u) + (sym == 0 ? 32u : 0u);
            if (keep_cw) qw[j] = (int32_t)cl;
          }
        }
        uint32_t tot = 0;
        const uint32_t start = block_excl_scan_u32(nb, m->scan, &tot);
        // chunk c covers threads [c*64/vpt, (c+1)*64/vpt)
        // chunk c covers threads [c*tpc, (c+1)*tpc); the thread starts go to the (now free)
        // internal-weight array
        const int tpc = kc / vpt;
        uint32_t* tstart = wint;
        tstart[tid] = start;
        if (tid == 0) tstart[T] = tot;
        __syncthreads();
        for (int c = tid; c < C; c += T) st16[off_chunk / 2 + c] = (uint16_t)(tstart[(c + 1) * tpc] - tstart[c * tpc]);
        pay = stage + off_pay / 4;
        BitWriter bw;
        bw.start(pay, start);
        if (keep_cw) {
          const uint32_t* cw = (const uint32_t*)(q + g * nv) + j0;
          for (int i = 0; i < vpt; ++i) {
            const uint32_t cl = cw[i];
            bw.put(cl >> 5, (int)(cl & 31u));
          }
        } else {
          int32_t pr2 = j0 >= 2 ? code(g, j0 - 2) : 0, pi2 = j0 >= 2 ? code(g, j0 - 1) : 0;
          for (int i = 0; i < vpt; ++i) {
            const int j = j0 + i;
            const int32_t c = code(g, j);
            const int32_t d = c - ((j & 1) ? pi2 : pr2);
            if (j & 1) pi2 = c;
            else pr2 = c;
            const uint32_t sym = (d < -kRadius || d > kRadius) ? 0u : (uint32_t)(d + 32768);
            const uint32_t hs_ = find_slot(sym);
            const uint32_t cl = hs_ < (uint32_t)L.hs ? hval[hs_] : 0u;
            bw.put(cl >> 5, (int)(cl & 31u));
            if (sym == 0) bw.put((uint32_t)d, 32);
          }
        }
        bw.finish();
      } else {
        pay = stage + kHdr / 4;
        BitWriter bw;
        bw.start(pay, (uint32_t)(j0 * width));
        int32_t pr2 = j0 >= 2 ? code(g, j0 - 2) : 0, pi2 = j0 >= 2 ? code(g, j0 - 1) : 0;
        for (int i = 0; i < vpt; ++i) {
          const int j = j0 + i;
          const int32_t c = code(g, j);
          const int32_t d = c - ((j & 1) ? pi2 : pr2);
          if (j & 1) pi2 = c;
          else pr2 = c;
          bw.put(zigzag(d), width);
        }
        bw.finish();
      }
      // verbatim section (positions ascending)
      if (!kMask && nverb > 0 && !big) {
        __syncthreads();
        if (tid == 0) {
          // insertion sort of the (rare) verbatim list by position
          uint16_t* vp = vout_pos + g * kVmax;
          uint64_t* vb = vout_bits + g * kVmax;
          for (int i = 1; i < nverb; ++i) {
            const uint16_t kp = vp[i];
            const uint64_t kb = vb[i];
            int j = i - 1;
            while (j >= 0 && vp[j] > kp) {
              vp[j + 1] = vp[j];
              vb[j + 1] = vb[j];
              --j;
            }
            vp[j + 1] = kp;
            vb[j + 1] = kb;
          }
          uint16_t* st16 = (uint16_t*)stage;
          for (int i = 0; i < nverb; ++i) st16[body_end / 2 + i] = vp[i];
          const uint32_t valoff = (uint32_t)pad_to(body_end + 2 * nverb, sizeof(Real));
          for (int i = 0; i < nverb; ++i) {
            if (sizeof(Real) == 8) ((uint64_t*)((uint8_t*)stage + valoff))[i] = vb[i];
            else ((uint32_t*)((uint8_t*)stage + valoff))[i] = (uint32_t)vb[i];
          }
        }
      }
    }
    __syncthreads();
    uint4* dst = (uint4*)(a.out_arena + m->out_off);
    const uint4* src = (const uint4*)stage;
    for (uint32_t i = tid; i < span / 16; i += T) dst[i] = src[i];
    if ((kMask || big) && mode != kModeConst && nverb > 0) {
      for (uint32_t i = span / 16 + tid; i < size / 16; i += T) dst[i] = make_uint4(0u, 0u, 0u, 0u);
      __syncthreads();  // the zero fill lands before the positions and values below
      write_verbatim_inplace(g, a.out_arena + m->out_off, body_end, nverb);
    }
    if (tid == 0) {
      a.out_off[blk] = m->out_off;
      a.out_len[blk] = size;
    }
  }
  // ---- norm partials and statistics ----
  if (tid == 0) {
    // exact sum of q^2: Sh * 2^32 + Sl as a 128-bit value
    const unsigned long long lo = (Sh << 32) + Sl;
    const unsigned long long carry0 = (lo < Sl) ? 1ull : 0ull;
    const unsigned long long hi = (Sh >> 32) + carry0;
    const unsigned long long old = atomicAdd(&a.sc->acc.sq_lo, lo);
    const unsigned long long c1 = (old + lo < old) ? 1ull : 0ull;
    if (hi + c1) atomicAdd(&a.sc->acc.sq_hi, hi + c1);
    if (nverb) atomicAdd(&a.sc->acc.n_verbatim, (unsigned long long)nverb);
    if (mode != kModeConst) atomicAdd(&a.sc->acc.n_escape, (unsigned long long)nesc_blk);
    atomicAdd(&a.sc->acc.modes[mode], 1ull);
    if (a.out_info) {
      if (is_const) {
        const uint32_t a0 = (uint32_t)(q0 < 0 ? -q0 : q0), a1 = (uint32_t)(q1 < 0 ? -q1 : q1);
        amax = a0 > a1 ? a0 : a1;
      }
      BlkInfo bi;
      bi.sq_lo = lo;
      bi.sq_hi_nesc = (unsigned int)(hi & 0xFFull) | ((unsigned int)(mode != kModeConst ? nesc_blk : 0) << 8);
      bi.maxq_mode = (amax & 0x1FFFFFFFu) | ((unsigned int)mode << 29) | (nverb_raw ? 0x80000000u : 0u);
      a.out_info[blk] = bi;
    }
  }
  if (big) {  // values and the verbatim sum follow the second transform
    if (tid == 0) {
      m->vbig[g] = 1;
      m->any_big = 1;
    }
    __syncthreads();
    return;
  }
  const double vs = nverb > 0 ? verbatim_square_tree(g) : 0.0;
  if (tid == 0 && a.vsum) a.vsum[blk] = vs;
  __syncthreads();
}

}  // namespace sv
