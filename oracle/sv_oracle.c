/*
 * sv_oracle.c — plain, slow CPU oracle. TEST INFRASTRUCTURE ONLY: the product never
 * links or loads it. Compile with -ffp-contract=off: every floating-point step below is
 * one IEEE operation, in the order written.
 *
 * Paper: Wu et al., "Memory-Efficient Quantum Circuit Simulation by Using Lossy Data
 * Compression" (PMES 2018).
 *   Sec. I    — full amplitude-vector update; 2^n complex doubles (O1 below).
 *   Sec. II   — SZ error-bounded lossy compression of state-vector slices, error bound set
 *               by the user (the codec below, restated: quantization, Lorenzo, Huffman).
 *   Alg. 1    — for each gate, for each slice: Decompress, Normalize, GateComputation,
 *               Compress (O2 below); O2L, its second mode, skips the slices a gate leaves
 *               unchanged and keeps their normalization as a per-slice scale.
 * Where the paper is silent (error-bound mode, what "Normalize" scales by, the codec's
 * internals, gates whose targets span slices) this file follows the readings recorded in
 * the design notes; each such place says which reading it takes.
 */
#include "sv_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------------------
 * Format constants (the block stream layout).
 * ---------------------------------------------------------------------------------- */
#define HDR_BYTES 16
#define SYM_RADIUS 32767   /* |delta| <= 32767 maps to symbol delta + 32768 */
#define SYM_ESCAPE 0       /* symbol 0: delta follows as 32 raw bits */
#define CHUNK_DEFAULT 32   /* symbols per decode chunk unless the caller picks 16 or 64 */
#define HUFF_MAX_DISTINCT 256
#define Q_LIMIT 536870912.0 /* 2^29: |x*r| must be below this to be quantized */

static size_t pad_to(size_t x, size_t a) { return (x + a - 1) / a * a; }

/* ------------------------------------------------------------------------------------
 * Linear quantization under an absolute error bound (Sec. II, "error bound for each
 * amplitude"; absolute mode per the design notes' reading).
 *   t  = fl(v * r),  r = fl(1 / fl(2 eb))
 *   q  = rint(t)                     (round half to even)
 *   x' = fl(q * fl(2 eb))            (complex64: then rounded to float)
 *   verbatim when |t| >= 2^29 (or t is NaN) or |fl(v - x')| > eb
 * ---------------------------------------------------------------------------------- */
typedef struct {
  double eb, two, r;
  int dtype;
} quant_params;

static quant_params qparams(double eb, int dtype) {
  quant_params p;
  p.eb = eb;
  p.two = 2.0 * eb;
  p.r = 1.0 / p.two;
  p.dtype = dtype;
  return p;
}

static double recon(int32_t q, const quant_params* p) {
  double x = (double)q * p->two;
  if (p->dtype == ORC_C64) x = (double)(float)x;
  return x;
}

/* Returns 1 when v must be stored verbatim; otherwise writes q. */
static int quantize(double v, const quant_params* p, int32_t* q_out) {
  double t = v * p->r;
  if (!(fabs(t) < Q_LIMIT)) return 1;
  double qd = rint(t);
  int32_t q = (int32_t)qd;
  double xr = recon(q, p);
  double d = v - xr;
  if (fabs(d) > p->eb) return 1;
  *q_out = q;
  return 0;
}

/* ------------------------------------------------------------------------------------
 * MSB-first bit stream in little-endian 32-bit words: stream bit k is bit (31 - k % 32)
 * of word k / 32.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  uint32_t* w;
  uint64_t bit;
} bitw;

static void put_bits(bitw* b, uint32_t val, int n) {
  for (int i = n - 1; i >= 0; --i) {
    if ((val >> i) & 1u) b->w[b->bit >> 5] |= 0x80000000u >> (b->bit & 31);
    b->bit++;
  }
}

typedef struct {
  const uint32_t* w;
  uint64_t bit, limit;
} bitr;

static int get_bit(bitr* b, int* err) {
  if (b->bit >= b->limit) {
    *err = 1;
    return 0;
  }
  int v = (int)((b->w[b->bit >> 5] >> (31 - (b->bit & 31))) & 1u);
  b->bit++;
  return v;
}

static uint32_t get_bits(bitr* b, int n, int* err) {
  uint32_t v = 0;
  for (int i = 0; i < n; ++i) v = (v << 1) | (uint32_t)get_bit(b, err);
  return v;
}

static void wr16(uint8_t* p, uint16_t v) { memcpy(p, &v, 2); }
static void wr32(uint8_t* p, uint32_t v) { memcpy(p, &v, 4); }
static uint16_t rd16(const uint8_t* p) { uint16_t v; memcpy(&v, p, 2); return v; }
static uint32_t rd32(const uint8_t* p) { uint32_t v; memcpy(&v, p, 4); return v; }

/* ------------------------------------------------------------------------------------
 * Huffman code lengths (Sec. II: SZ entropy-codes its quantization codes with Huffman).
 * Two-queue construction: leaves in increasing (frequency, symbol) order; internal nodes
 * are created in non-decreasing weight order, so the two queues stay sorted. Each merge
 * takes the two lightest heads; on equal weight the leaf queue is taken first.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  uint32_t f, s;
  int pos;
} leaf_t;

static int cmp_leaf(const void* a, const void* b) {
  const leaf_t* x = (const leaf_t*)a;
  const leaf_t* y = (const leaf_t*)b;
  if (x->f != y->f) return x->f < y->f ? -1 : 1;
  if (x->s != y->s) return x->s < y->s ? -1 : 1;
  return 0;
}

int orc_huffman_lengths(const uint32_t* freq, const uint32_t* sym, int n, int* lens_out) {
  if (n <= 0) return 0;
  if (n == 1) {
    lens_out[0] = 1;
    return 1;
  }
  leaf_t* leaf = (leaf_t*)malloc(sizeof(leaf_t) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    leaf[i].f = freq[i];
    leaf[i].s = sym[i];
    leaf[i].pos = i;
  }
  qsort(leaf, (size_t)n, sizeof(leaf_t), cmp_leaf);
  const int total = 2 * n - 1; /* nodes 0..n-1 leaves (sorted), n..2n-2 internal */
  uint64_t* w = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)total);
  int* parent = (int*)malloc(sizeof(int) * (size_t)total);
  int* depth = (int*)malloc(sizeof(int) * (size_t)total);
  for (int i = 0; i < n; ++i) w[i] = leaf[i].f;
  int lp = 0;   /* head of the leaf queue */
  int ip = n;   /* head of the internal-node queue */
  int next = n; /* next internal node to create */
  for (int m = 0; m < n - 1; ++m) {
    int pick[2];
    for (int t = 0; t < 2; ++t) {
      if (lp < n && (ip >= next || w[lp] <= w[ip])) pick[t] = lp++;
      else pick[t] = ip++;
    }
    w[next] = w[pick[0]] + w[pick[1]];
    parent[pick[0]] = next;
    parent[pick[1]] = next;
    next++;
  }
  /* every parent has a larger index than its children: depths top-down */
  depth[total - 1] = 0;
  for (int v = total - 2; v >= 0; --v) depth[v] = depth[parent[v]] + 1;
  int maxlen = 0;
  for (int i = 0; i < n; ++i) {
    lens_out[leaf[i].pos] = depth[i];
    if (depth[i] > maxlen) maxlen = depth[i];
  }
  free(w);
  free(parent);
  free(depth);
  free(leaf);
  return maxlen;
}

/* ------------------------------------------------------------------------------------
 * Block codec.
 * Stream = 16-byte header, body, verbatim section, zero padding to 16 bytes.
 *   header: u8 mode, u8 dtype, u8 block_log2, u8 param, u16 n_verbatim, u16 D,
 *           CONST: i32 q_re, i32 q_im;  HUFF/PACK: u32 payload_bits, u32 total_bytes.
 *   HUFF body: u16 count[1..Lmax] | u16 symbols (canonical order) | u16 chunk_bits[C]
 *              | u32 payload words     (each part padded to 4 bytes)
 *   PACK body: u32 payload words (2B zigzag deltas of `param` bits each)
 *   verbatim: u16 positions (ascending), padded to the value size, then raw values.
 * ---------------------------------------------------------------------------------- */
static int comp_size(int dtype) { return dtype == ORC_C64 ? 4 : 8; }

size_t orc_block_bound(int block_log2, int dtype) {
  size_t B = (size_t)1 << block_log2;
  size_t nv = 2 * B;
  /* PACK with 32-bit width is the largest body the mode rule can choose */
  size_t body = nv * 4;
  size_t verb = pad_to(nv * 2, 8) + nv * (size_t)comp_size(dtype);
  return pad_to(HDR_BYTES + body + verb, 16);
}

static double load_val(const void* v, int dtype, size_t j) {
  if (dtype == ORC_C64) return (double)((const float*)v)[j];
  return ((const double*)v)[j];
}

static void store_val(void* v, int dtype, size_t j, double x) {
  if (dtype == ORC_C64) ((float*)v)[j] = (float)x;
  else ((double*)v)[j] = x;
}

static uint32_t zigzag(int32_t d) {
  return d >= 0 ? (uint32_t)d << 1 : (((uint32_t)(-(int64_t)d) << 1) - 1u);
}

static int32_t unzigzag(uint32_t z) {
  return (z & 1u) ? (int32_t)(-(int64_t)((z >> 1) + 1u)) : (int32_t)(z >> 1);
}

static int bit_width(uint32_t z) {
  int w = 0;
  while (z) {
    w++;
    z >>= 1;
  }
  return w;
}

static int chunk_ok(int chunk) { return chunk == 16 || chunk == 32 || chunk == 64; }

size_t orc_compress_block(const void* values, int block_log2, int dtype, double eb,
                          uint8_t* out, orc_block_info* info) {
  return orc_compress_block_k(values, block_log2, dtype, eb, CHUNK_DEFAULT, out, info);
}

size_t orc_compress_block_k(const void* values, int block_log2, int dtype, double eb, int chunk,
                            uint8_t* out, orc_block_info* info) {
  if (block_log2 < 5 || block_log2 > 12 || !(eb > 0) || (dtype != ORC_C64 && dtype != ORC_C128) ||
      !chunk_ok(chunk))
    return 0;
  const size_t B = (size_t)1 << block_log2;
  const size_t nv = 2 * B; /* values in the block: re, im interleaved */
  quant_params p = qparams(eb, dtype);
  int32_t* q = (int32_t*)calloc(nv, sizeof(int32_t));
  uint8_t* verb = (uint8_t*)calloc(nv, 1);
  int32_t* delta = (int32_t*)calloc(nv, sizeof(int32_t));
  uint32_t* symb = (uint32_t*)calloc(nv, sizeof(uint32_t));
  orc_block_info inf;
  memset(&inf, 0, sizeof(inf));
  u128 sq = 0;
  /* squares of the verbatim values (zero elsewhere), summed below by a pairwise tree */
  double* vsq = (double*)calloc(nv, sizeof(double));
  for (size_t j = 0; j < nv; ++j) {
    double v = load_val(values, dtype, j);
    int32_t qq = 0;
    if (quantize(v, &p, &qq)) {
      verb[j] = 1;
      q[j] = 0;
      inf.n_verbatim++;
      vsq[j] = v * v;
    } else {
      q[j] = qq;
      sq += (u128)((int64_t)qq * (int64_t)qq);
    }
  }
  /* Lorenzo 1-D per plane: value j predicts from value j-2 (same plane); first from 0 */
  for (size_t j = 0; j < nv; ++j) {
    int32_t prev = j >= 2 ? q[j - 2] : 0;
    delta[j] = q[j] - prev;
    if (delta[j] >= -SYM_RADIUS && delta[j] <= SYM_RADIUS) {
      symb[j] = (uint32_t)(delta[j] + 32768);
    } else {
      symb[j] = SYM_ESCAPE;
      inf.n_escape++;
    }
  }
  inf.sq_lo = (uint64_t)sq;
  inf.sq_hi = (uint64_t)(sq >> 64);
  /* verbatim part of the block's norm: level-by-level pairwise sum over the 2B values,
     vsq[i] = vsq[2i] + vsq[2i+1] until one remains (entries of non-verbatim values are +0) */
  for (size_t cnt = nv; cnt > 1; cnt /= 2)
    for (size_t i = 0; i < cnt / 2; ++i) vsq[i] = vsq[2 * i] + vsq[2 * i + 1];
  inf.vsum = vsq[0];
  free(vsq);

  memset(out, 0, orc_block_bound(block_log2, dtype));
  out[1] = (uint8_t)dtype;
  out[2] = (uint8_t)block_log2;

  /* CONST: no verbatim value and every q equal within each plane */
  int is_const = inf.n_verbatim == 0;
  for (size_t j = 2; j < nv && is_const; ++j)
    if (q[j] != q[j - 2]) is_const = 0;
  size_t total;
  if (is_const) {
    out[0] = ORC_MODE_CONST;
    wr32(out + 8, (uint32_t)q[0]);
    wr32(out + 12, (uint32_t)q[1]);
    inf.mode = ORC_MODE_CONST;
    total = HDR_BYTES;
  } else {
    /* histogram over the 65536 symbols */
    uint32_t* hist = (uint32_t*)calloc(65536, sizeof(uint32_t));
    for (size_t j = 0; j < nv; ++j) hist[symb[j]]++;
    int D = 0;
    for (int s = 0; s < 65536; ++s) D += hist[s] ? 1 : 0;
    inf.n_distinct = D;
    /* PACK size */
    uint32_t zmax = 0;
    for (size_t j = 0; j < nv; ++j) {
      uint32_t z = zigzag(delta[j]);
      if (z > zmax) zmax = z;
    }
    int width = bit_width(zmax);
    size_t pack_body = 4 * ((nv * (size_t)width + 31) / 32);
    /* HUFF size when allowed */
    int use_huff = 0;
    int* len_of = NULL;
    uint32_t* syms = NULL;
    int Lmax = 0;
    uint64_t payload_bits = 0;
    size_t nchunks = nv / (size_t)chunk;
    size_t huff_body = 0;
    if (D <= HUFF_MAX_DISTINCT) {
      syms = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)D);
      uint32_t* fr = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)D);
      int* lens = (int*)malloc(sizeof(int) * (size_t)D);
      int d = 0;
      for (int s = 0; s < 65536; ++s)
        if (hist[s]) {
          syms[d] = (uint32_t)s;
          fr[d] = hist[s];
          d++;
        }
      Lmax = orc_huffman_lengths(fr, syms, D, lens);
      len_of = (int*)calloc(65536, sizeof(int));
      for (int i = 0; i < D; ++i) len_of[syms[i]] = lens[i];
      for (int i = 0; i < D; ++i) payload_bits += (uint64_t)fr[i] * (uint64_t)lens[i];
      payload_bits += 32u * (uint64_t)inf.n_escape;
      huff_body = pad_to(2 * (size_t)Lmax, 4) + pad_to(2 * (size_t)D, 4) +
                  pad_to(2 * nchunks, 4) + 4 * (size_t)((payload_bits + 31) / 32);
      use_huff = huff_body < pack_body;
      free(fr);
      free(lens);
    }
    size_t body_end;
    uint32_t pbits;
    if (use_huff) {
      out[0] = ORC_MODE_HUFF;
      out[3] = (uint8_t)Lmax;
      wr16(out + 6, (uint16_t)D);
      inf.mode = ORC_MODE_HUFF;
      /* canonical order: (length, symbol) ascending */
      uint32_t* canon = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)D);
      int c = 0;
      for (int L = 1; L <= Lmax; ++L)
        for (int s = 0; s < 65536; ++s)
          if (hist[s] && len_of[s] == L) canon[c++] = (uint32_t)s;
      uint32_t* code_of = (uint32_t*)calloc(65536, sizeof(uint32_t));
      uint32_t code = 0;
      for (int i = 0; i < D; ++i) {
        if (i > 0) code = (code + 1u) << (len_of[canon[i]] - len_of[canon[i - 1]]);
        code_of[canon[i]] = code;
      }
      uint8_t* ptr = out + HDR_BYTES;
      for (int L = 1; L <= Lmax; ++L) {
        int cnt = 0;
        for (int i = 0; i < D; ++i) cnt += len_of[canon[i]] == L;
        wr16(ptr + 2 * (size_t)(L - 1), (uint16_t)cnt);
      }
      ptr += pad_to(2 * (size_t)Lmax, 4);
      for (int i = 0; i < D; ++i) wr16(ptr + 2 * (size_t)i, (uint16_t)canon[i]);
      ptr += pad_to(2 * (size_t)D, 4);
      uint8_t* chunk_tab = ptr;
      ptr += pad_to(2 * nchunks, 4);
      bitw bw;
      bw.w = (uint32_t*)ptr; /* 4-byte aligned: out is 16-aligned, offsets are multiples of 4 */
      bw.bit = 0;
      for (size_t j = 0; j < nv; ++j) {
        put_bits(&bw, code_of[symb[j]], len_of[symb[j]]);
        if (symb[j] == SYM_ESCAPE) put_bits(&bw, (uint32_t)delta[j], 32);
      }
      /* chunk sizes: re-walk and measure */
      uint64_t pos = 0;
      for (size_t ch = 0; ch < nchunks; ++ch) {
        uint64_t start = pos;
        for (size_t j = ch * (size_t)chunk; j < (ch + 1) * (size_t)chunk; ++j) {
          pos += (uint64_t)len_of[symb[j]];
          if (symb[j] == SYM_ESCAPE) pos += 32;
        }
        wr16(chunk_tab + 2 * ch, (uint16_t)(pos - start));
      }
      pbits = (uint32_t)payload_bits;
      body_end = HDR_BYTES + huff_body;
      free(canon);
      free(code_of);
    } else {
      out[0] = ORC_MODE_PACK;
      out[3] = (uint8_t)width;
      inf.mode = ORC_MODE_PACK;
      bitw bw;
      bw.w = (uint32_t*)(out + HDR_BYTES);
      bw.bit = 0;
      for (size_t j = 0; j < nv; ++j) put_bits(&bw, zigzag(delta[j]), width);
      pbits = (uint32_t)(nv * (size_t)width);
      body_end = HDR_BYTES + pack_body;
    }
    /* verbatim section */
    size_t pos = body_end;
    size_t k = 0;
    for (size_t j = 0; j < nv; ++j)
      if (verb[j]) wr16(out + pos + 2 * (k++), (uint16_t)j);
    pos = pad_to(pos + 2 * (size_t)inf.n_verbatim, (size_t)comp_size(dtype));
    for (size_t j = 0; j < nv; ++j) {
      if (!verb[j]) continue;
      if (dtype == ORC_C64) {
        float f = ((const float*)values)[j];
        memcpy(out + pos, &f, 4);
        pos += 4;
      } else {
        double f = ((const double*)values)[j];
        memcpy(out + pos, &f, 8);
        pos += 8;
      }
    }
    total = pad_to(pos, 16);
    wr16(out + 4, (uint16_t)inf.n_verbatim);
    wr32(out + 8, pbits);
    wr32(out + 12, (uint32_t)total);
    free(hist);
    free(len_of);
    free(syms);
  }
  if (info) *info = inf;
  free(q);
  free(verb);
  free(delta);
  free(symb);
  return total;
}

int orc_decompress_block(const uint8_t* in, size_t len, int block_log2, int dtype, double eb,
                         void* values_out) {
  return orc_decompress_block_k(in, len, block_log2, dtype, eb, CHUNK_DEFAULT, values_out);
}

int orc_decompress_block_k(const uint8_t* in, size_t len, int block_log2, int dtype, double eb,
                           int chunk, void* values_out) {
  if (len < HDR_BYTES || !chunk_ok(chunk)) return -1;
  const size_t B = (size_t)1 << block_log2;
  const size_t nv = 2 * B;
  quant_params p = qparams(eb, dtype);
  int mode = in[0];
  if (in[1] != dtype || in[2] != block_log2) return -2;
  int32_t* q = (int32_t*)calloc(nv, sizeof(int32_t));
  int rc = 0;
  size_t body_end = HDR_BYTES;
  int nverb = rd16(in + 4);
  if (mode == ORC_MODE_CONST) {
    int32_t qre = (int32_t)rd32(in + 8), qim = (int32_t)rd32(in + 12);
    for (size_t i = 0; i < B; ++i) {
      q[2 * i] = qre;
      q[2 * i + 1] = qim;
    }
    if (nverb != 0) rc = -3;
  } else if (mode == ORC_MODE_HUFF || mode == ORC_MODE_PACK) {
    uint32_t pbits = rd32(in + 8);
    uint32_t total = rd32(in + 12);
    if (total > len) {
      free(q);
      return -4;
    }
    int32_t* delta = (int32_t*)calloc(nv, sizeof(int32_t));
    int err = 0;
    if (mode == ORC_MODE_PACK) {
      int width = in[3];
      bitr br;
      br.w = (const uint32_t*)(in + HDR_BYTES);
      br.bit = 0;
      br.limit = pbits;
      for (size_t j = 0; j < nv; ++j) delta[j] = unzigzag(get_bits(&br, width, &err));
      body_end = HDR_BYTES + 4 * ((pbits + 31) / 32);
    } else {
      int Lmax = in[3];
      int D = rd16(in + 6);
      const uint8_t* ptr = in + HDR_BYTES;
      int count[33] = {0};
      for (int L = 1; L <= Lmax; ++L) count[L] = rd16(ptr + 2 * (size_t)(L - 1));
      ptr += pad_to(2 * (size_t)Lmax, 4);
      const uint8_t* symtab = ptr;
      ptr += pad_to(2 * (size_t)D, 4);
      size_t nchunks = nv / (size_t)chunk;
      ptr += pad_to(2 * nchunks, 4);
      /* canonical decoding: first code and first index of every length */
      uint32_t first[34];
      int offs[34];
      uint32_t code = 0;
      int idx = 0;
      for (int L = 1; L <= Lmax; ++L) {
        first[L] = code;
        offs[L] = idx;
        code = (code + (uint32_t)count[L]) << 1;
        idx += count[L];
      }
      bitr br;
      br.w = (const uint32_t*)ptr;
      br.bit = 0;
      br.limit = pbits;
      for (size_t j = 0; j < nv && !err; ++j) {
        uint32_t c = 0;
        int sym = -1;
        for (int L = 1; L <= Lmax; ++L) {
          c = (c << 1) | (uint32_t)get_bit(&br, &err);
          if (count[L] && c >= first[L] && c - first[L] < (uint32_t)count[L]) {
            sym = rd16(symtab + 2 * (size_t)(offs[L] + (int)(c - first[L])));
            break;
          }
        }
        if (sym < 0) {
          err = 1;
          break;
        }
        if (sym == SYM_ESCAPE) delta[j] = (int32_t)get_bits(&br, 32, &err);
        else delta[j] = sym - 32768;
      }
      body_end = (size_t)(ptr - in) + 4 * ((pbits + 31) / 32);
    }
    if (err) rc = -5;
    for (size_t j = 0; j < nv; ++j) q[j] = (j >= 2 ? q[j - 2] : 0) + delta[j];
    free(delta);
  } else {
    rc = -6;
  }
  if (rc == 0) {
    for (size_t j = 0; j < nv; ++j) store_val(values_out, dtype, j, recon(q[j], &p));
    if (nverb) {
      size_t pos = body_end;
      const uint8_t* posp = in + pos;
      pos = pad_to(pos + 2 * (size_t)nverb, (size_t)comp_size(dtype));
      for (int k = 0; k < nverb; ++k) {
        size_t j = rd16(posp + 2 * (size_t)k);
        if (j >= nv) {
          rc = -7;
          break;
        }
        if (dtype == ORC_C64) {
          float f;
          memcpy(&f, in + pos + 4 * (size_t)k, 4);
          ((float*)values_out)[j] = f;
        } else {
          double f;
          memcpy(&f, in + pos + 8 * (size_t)k, 8);
          ((double*)values_out)[j] = f;
        }
      }
    }
  }
  free(q);
  return rc;
}

/* ------------------------------------------------------------------------------------
 * Gate computation (Alg. 1 GateComputation; Sec. I full amplitude-vector update).
 * For every index i whose target bits are zero, the 2^k amplitudes
 * y_m = a[i + sum_l bit_l(m) 2^{t_l}] are replaced by z_j = sum_m G[j][m] y_m when every
 * control bit of i is one. Complex product (a+ib)(c+id) = (ac - bd) + i(ad + bc); the sum
 * over m runs m = 0, 1, ... left to right. complex64 runs the same steps in float with G
 * rounded to float.
 * ---------------------------------------------------------------------------------- */
typedef struct {
  double re, im;
} cd;
typedef struct {
  float re, im;
} cf;

static void gate_tuple_d(const double* G, int k, const cd* y, cd* z) {
  int K = 1 << k;
  for (int j = 0; j < K; ++j) {
    double ar = 0, ai = 0;
    for (int m = 0; m < K; ++m) {
      double gr = G[2 * (j * K + m)], gi = G[2 * (j * K + m) + 1];
      double pr = gr * y[m].re - gi * y[m].im;
      double pi = gr * y[m].im + gi * y[m].re;
      if (m == 0) {
        ar = pr;
        ai = pi;
      } else {
        ar = ar + pr;
        ai = ai + pi;
      }
    }
    z[j].re = ar;
    z[j].im = ai;
  }
}

static void gate_tuple_f(const float* Gf, int k, const cf* y, cf* z) {
  int K = 1 << k;
  for (int j = 0; j < K; ++j) {
    float ar = 0, ai = 0;
    for (int m = 0; m < K; ++m) {
      float gr = Gf[2 * (j * K + m)], gi = Gf[2 * (j * K + m) + 1];
      float pr = gr * y[m].re - gi * y[m].im;
      float pi = gr * y[m].im + gi * y[m].re;
      if (m == 0) {
        ar = pr;
        ai = pi;
      } else {
        ar = ar + pr;
        ai = ai + pi;
      }
    }
    z[j].re = ar;
    z[j].im = ai;
  }
}

static uint64_t tuple_index(uint64_t base, const int* targets, int k, int m) {
  uint64_t i = base;
  for (int l = 0; l < k; ++l)
    if ((m >> l) & 1) i |= (uint64_t)1 << targets[l];
  return i;
}

static int gate_args_ok(int n, const int* targets, int k, const int* controls, int nc) {
  if (k < 1 || k > 5 || nc < 0) return 0;
  uint64_t seen = 0;
  for (int l = 0; l < k; ++l) {
    if (targets[l] < 0 || targets[l] >= n || ((seen >> targets[l]) & 1)) return 0;
    seen |= (uint64_t)1 << targets[l];
  }
  for (int l = 0; l < nc; ++l) {
    if (controls[l] < 0 || controls[l] >= n || ((seen >> controls[l]) & 1)) return 0;
    seen |= (uint64_t)1 << controls[l];
  }
  return 1;
}

void orc_plain_apply(void* state, int n, int dtype, const double* G, const int* targets, int k,
                     const int* controls, int nc) {
  if (!gate_args_ok(n, targets, k, controls, nc)) return;
  uint64_t tmask = 0, cmask = 0;
  for (int l = 0; l < k; ++l) tmask |= (uint64_t)1 << targets[l];
  for (int l = 0; l < nc; ++l) cmask |= (uint64_t)1 << controls[l];
  int K = 1 << k;
  uint64_t dim = (uint64_t)1 << n;
  float Gf[2 * 32 * 32];
  for (int e = 0; e < 2 * K * K; ++e) Gf[e] = (float)G[e];
  for (uint64_t base = 0; base < dim; ++base) {
    if (base & tmask) continue;
    if ((base & cmask) != cmask) continue;
    if (dtype == ORC_C128) {
      cd y[32], z[32];
      double* a = (double*)state;
      for (int m = 0; m < K; ++m) {
        uint64_t i = tuple_index(base, targets, k, m);
        y[m].re = a[2 * i];
        y[m].im = a[2 * i + 1];
      }
      gate_tuple_d(G, k, y, z);
      for (int m = 0; m < K; ++m) {
        uint64_t i = tuple_index(base, targets, k, m);
        a[2 * i] = z[m].re;
        a[2 * i + 1] = z[m].im;
      }
    } else {
      cf y[32], z[32];
      float* a = (float*)state;
      for (int m = 0; m < K; ++m) {
        uint64_t i = tuple_index(base, targets, k, m);
        y[m].re = a[2 * i];
        y[m].im = a[2 * i + 1];
      }
      gate_tuple_f(Gf, k, y, z);
      for (int m = 0; m < K; ++m) {
        uint64_t i = tuple_index(base, targets, k, m);
        a[2 * i] = z[m].re;
        a[2 * i + 1] = z[m].im;
      }
    }
  }
}

/* ------------------------------------------------------------------------------------
 * O2: Algorithm 1 over a block-compressed state.
 * Slices are 2^slice_log2 amplitudes (Alg. 1's unit); each slice is stored as
 * 2^(slice_log2 - block_log2) independently coded blocks.
 * ---------------------------------------------------------------------------------- */
struct orc_csim {
  int n, slice_log2, block_log2, dtype, chunk;
  double eb;
  quant_params qp;
  uint64_t nblocks;
  uint8_t** streams;
  size_t* lens;
  orc_block_info* infos;
  double norm;
  /* the second mode (lazy normalization with slice skipping): a slice the gate leaves
   * unchanged keeps its stream, and its pending normalization is a scale c_s; the state
   * it represents is c_s x' (x' the stored values). Outside the mode every c_s is 1. */
  int lazy;
  double* scale;     /* one per slice */
  uint64_t skipped;  /* slices left unchanged by the passes so far */
};

/* Norm of the stored state (Alg. 1 Normalize; reading: one global scale per gate pass,
 * from the exact norm of what is stored):
 *   N = fl( fl(Sd * fl(two*two)) + V )
 *   Sd = fl( fl((double)S_hi * 2^64) + (double)S_lo ),  S = exact sum of q^2
 *   V  = pairwise sum over blocks (level by level, a[i] = a[2i] + a[2i+1]) of the
 *        per-block verbatim sums.                                                     */
/* The same formula over blocks [b0, b1) (a power-of-two count) whose slices are selected by
 * `keep` (NULL: all): S and V sum only the kept blocks (the others count as 0 in V's tree). */
static double norm_of_blocks(const orc_csim* s, uint64_t b0, uint64_t b1, const unsigned char* keep) {
  const uint64_t per_slice = (uint64_t)1 << (s->slice_log2 - s->block_log2);
  u128 S = 0;
  for (uint64_t b = b0; b < b1; ++b)
    if (!keep || keep[b / per_slice]) S += ((u128)s->infos[b].sq_hi << 64) | (u128)s->infos[b].sq_lo;
  uint64_t hi = (uint64_t)(S >> 64), lo = (uint64_t)S;
  double Sd = (double)hi * 18446744073709551616.0 + (double)lo;
  uint64_t cnt = b1 - b0;
  double* a = (double*)malloc(sizeof(double) * cnt);
  for (uint64_t b = b0; b < b1; ++b) a[b - b0] = (!keep || keep[b / per_slice]) ? s->infos[b].vsum : 0.0;
  while (cnt > 1) {
    for (uint64_t i = 0; i < cnt / 2; ++i) a[i] = a[2 * i] + a[2 * i + 1];
    cnt /= 2;
  }
  double V = a[0];
  free(a);
  double two2 = s->qp.two * s->qp.two;
  double t = Sd * two2;
  return t + V;
}

/* Second mode: N = fl(N_1 + R), N_1 the formula above over the slices whose scale is exactly
 * 1, R the pairwise sum over slices (level by level, 0 for slices of scale 1) of
 * fl(fl(c_s c_s) N_s), N_s the formula over slice s's own blocks. With every scale 1 this is
 * the formula above exactly. */
static double stored_norm(const orc_csim* s) {
  if (!s->lazy) return norm_of_blocks(s, 0, s->nblocks, NULL);
  const uint64_t ns = (uint64_t)1 << (s->n - s->slice_log2);
  const uint64_t per_slice = (uint64_t)1 << (s->slice_log2 - s->block_log2);
  unsigned char* one = (unsigned char*)malloc(ns);
  double* r = (double*)malloc(sizeof(double) * ns);
  for (uint64_t i = 0; i < ns; ++i) {
    one[i] = s->scale[i] == 1.0;
    r[i] = 0.0;
    if (!one[i]) {
      const double Ns = norm_of_blocks(s, i * per_slice, (i + 1) * per_slice, NULL);
      r[i] = (s->scale[i] * s->scale[i]) * Ns;
    }
  }
  const double N1 = norm_of_blocks(s, 0, s->nblocks, one);
  uint64_t cnt = ns;
  while (cnt > 1) {
    for (uint64_t i = 0; i < cnt / 2; ++i) r[i] = r[2 * i] + r[2 * i + 1];
    cnt /= 2;
  }
  const double R = r[0];
  free(one);
  free(r);
  return N1 + R;
}

static void set_block(orc_csim* s, uint64_t b, const void* vals) {
  size_t bound = orc_block_bound(s->block_log2, s->dtype);
  uint8_t* tmp = (uint8_t*)malloc(bound);
  size_t len = orc_compress_block_k(vals, s->block_log2, s->dtype, s->eb, s->chunk, tmp, &s->infos[b]);
  free(s->streams[b]);
  s->streams[b] = (uint8_t*)malloc(len);
  memcpy(s->streams[b], tmp, len);
  s->lens[b] = len;
  free(tmp);
}

orc_csim* orc_csim_create(int n, int slice_log2, int block_log2, int dtype, double eb,
                          uint64_t basis_index) {
  return orc_csim_create_k(n, slice_log2, block_log2, dtype, eb, basis_index, CHUNK_DEFAULT);
}

orc_csim* orc_csim_create_k(int n, int slice_log2, int block_log2, int dtype, double eb,
                            uint64_t basis_index, int chunk) {
  if (n < block_log2 || slice_log2 < block_log2 || slice_log2 > n || block_log2 < 5 ||
      block_log2 > 12 || !(eb > 0) || (dtype != ORC_C64 && dtype != ORC_C128) || n > 40 ||
      !chunk_ok(chunk))
    return NULL;
  if (basis_index >> n) return NULL;
  orc_csim* s = (orc_csim*)calloc(1, sizeof(orc_csim));
  s->n = n;
  s->slice_log2 = slice_log2;
  s->block_log2 = block_log2;
  s->dtype = dtype;
  s->chunk = chunk;
  s->eb = eb;
  s->qp = qparams(eb, dtype);
  s->nblocks = (uint64_t)1 << (n - block_log2);
  s->streams = (uint8_t**)calloc(s->nblocks, sizeof(uint8_t*));
  s->lens = (size_t*)calloc(s->nblocks, sizeof(size_t));
  s->infos = (orc_block_info*)calloc(s->nblocks, sizeof(orc_block_info));
  s->scale = (double*)malloc(sizeof(double) * ((size_t)1 << (n - slice_log2)));
  for (uint64_t i = 0; i < ((uint64_t)1 << (n - slice_log2)); ++i) s->scale[i] = 1.0;
  size_t B = (size_t)1 << block_log2;
  size_t cs = (size_t)comp_size(dtype);
  void* vals = calloc(2 * B, cs);
  /* the initial state |x>: every block zero except the one holding x */
  for (uint64_t b = 0; b < s->nblocks; ++b) {
    memset(vals, 0, 2 * B * cs);
    if ((basis_index >> block_log2) == b) store_val(vals, dtype, 2 * (basis_index & (B - 1)), 1.0);
    set_block(s, b, vals);
  }
  free(vals);
  s->norm = stored_norm(s);
  return s;
}

void orc_csim_destroy(orc_csim* s) {
  if (!s) return;
  for (uint64_t b = 0; b < s->nblocks; ++b) free(s->streams[b]);
  free(s->streams);
  free(s->lens);
  free(s->infos);
  free(s->scale);
  free(s);
}

int orc_csim_set_lazy(orc_csim* s, int on) {
  const uint64_t ns = (uint64_t)1 << (s->n - s->slice_log2);
  for (uint64_t i = 0; i < ns; ++i)
    if (s->scale[i] != 1.0) return -1; /* a pending scale belongs to the mode */
  s->lazy = on != 0;
  return 0;
}
void orc_csim_scales(const orc_csim* s, double* out) {
  const uint64_t ns = (uint64_t)1 << (s->n - s->slice_log2);
  for (uint64_t i = 0; i < ns; ++i) out[i] = s->scale[i];
}
uint64_t orc_csim_skipped(const orc_csim* s) { return s->skipped; }

/* The represented amplitudes c_s x' as FP64 (re, im) pairs, for either dtype. */
void orc_csim_read_values(const orc_csim* s, double* out) {
  const size_t B = (size_t)1 << s->block_log2;
  const size_t cs = (size_t)comp_size(s->dtype);
  const uint64_t per_slice = (uint64_t)1 << (s->slice_log2 - s->block_log2);
  uint8_t* tmp = (uint8_t*)malloc(2 * B * cs);
  for (uint64_t b = 0; b < s->nblocks; ++b) {
    orc_decompress_block_k(s->streams[b], s->lens[b], s->block_log2, s->dtype, s->eb, s->chunk, tmp);
    const double c = s->scale[b / per_slice];
    for (size_t j = 0; j < 2 * B; ++j) out[b * 2 * B + j] = c * load_val(tmp, s->dtype, j);
  }
  free(tmp);
}

double orc_csim_norm(const orc_csim* s) { return s->norm; }
uint64_t orc_csim_nblocks(const orc_csim* s) { return s->nblocks; }
size_t orc_csim_block_stream(const orc_csim* s, uint64_t b, const uint8_t** ptr) {
  *ptr = s->streams[b];
  return s->lens[b];
}
uint64_t orc_csim_total_bytes(const orc_csim* s) {
  uint64_t t = 0;
  for (uint64_t b = 0; b < s->nblocks; ++b) t += s->lens[b];
  return t;
}

void orc_csim_read(const orc_csim* s, void* out) {
  size_t B = (size_t)1 << s->block_log2;
  size_t cs = (size_t)comp_size(s->dtype);
  for (uint64_t b = 0; b < s->nblocks; ++b)
    orc_decompress_block_k(s->streams[b], s->lens[b], s->block_log2, s->dtype, s->eb, s->chunk,
                           (uint8_t*)out + b * 2 * B * cs);
}

void orc_csim_load(orc_csim* s, const void* values) {
  size_t B = (size_t)1 << s->block_log2;
  size_t cs = (size_t)comp_size(s->dtype);
  for (uint64_t b = 0; b < s->nblocks; ++b)
    set_block(s, b, (const uint8_t*)values + b * 2 * B * cs);
  for (uint64_t i = 0; i < ((uint64_t)1 << (s->n - s->slice_log2)); ++i) s->scale[i] = 1.0;
  s->norm = stored_norm(s);
}

int orc_csim_apply(orc_csim* s, const double* G, const int* targets, int k, const int* controls,
                   int nc) {
  if (!gate_args_ok(s->n, targets, k, controls, nc)) return -1;
  if (!(s->norm > 0) || !isfinite(s->norm)) return -2;
  const int n = s->n, sl = s->slice_log2, bl = s->block_log2;
  const size_t S = (size_t)1 << sl;          /* amplitudes per slice */
  const size_t B = (size_t)1 << bl;          /* amplitudes per block */
  const size_t cs = (size_t)comp_size(s->dtype);
  const int K = 1 << k;
  /* Normalize(S): sigma = 1 / sqrt(N) of the stored state (one scale for every slice) */
  const double sigma = 1.0 / sqrt(s->norm);
  const float sigma_f = (float)sigma;
  float Gf[2 * 32 * 32];
  for (int e = 0; e < 2 * K * K; ++e) Gf[e] = (float)G[e];
  uint64_t cmask = 0;
  for (int l = 0; l < nc; ++l) cmask |= (uint64_t)1 << controls[l];
  /* targets at or above slice_log2 couple 2^h slices; they are processed together */
  int high[5], h = 0;
  for (int l = 0; l < k; ++l)
    if (targets[l] >= sl) high[h++] = targets[l];
  uint64_t hmask = 0;
  for (int l = 0; l < h; ++l) hmask |= (uint64_t)1 << (high[l] - sl);
  const uint64_t nslices = (uint64_t)1 << (n - sl);
  const int G_ = 1 << h; /* slices per group */
  uint8_t* buf = (uint8_t*)malloc((size_t)G_ * S * 2 * cs);
  uint64_t* slice_ids = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)G_);
  orc_block_info* new_infos = (orc_block_info*)calloc(s->nblocks, sizeof(orc_block_info));
  uint8_t** new_streams = (uint8_t**)calloc(s->nblocks, sizeof(uint8_t*));
  size_t* new_lens = (size_t*)calloc(s->nblocks, sizeof(size_t));
  size_t bound = orc_block_bound(bl, s->dtype);
  uint8_t* tmp = (uint8_t*)malloc(bound);
  /* second mode: slot g of a group is left unchanged when the group's controls above the
   * slice are not all 1, or when G is diagonal with every entry of the slot's rows (the rows
   * whose high-target bits are g) exactly 1 */
  const uint64_t chigh = cmask >> sl;  /* controls above the slice, as slice-index bits */
  int unit_slot[32];
  {
    int diag = 1;
    for (int j = 0; j < K; ++j)
      for (int m = 0; m < K; ++m)
        if (j != m && (G[2 * (j * K + m)] != 0.0 || G[2 * (j * K + m) + 1] != 0.0)) diag = 0;
    int tl[5];
    for (int lh = 0; lh < h; ++lh)
      for (int l = 0; l < k; ++l)
        if (targets[l] == high[lh]) tl[lh] = l;
    for (int g = 0; g < G_; ++g) unit_slot[g] = diag;
    for (int j = 0; j < K; ++j) {
      int g = 0;
      for (int lh = 0; lh < h; ++lh) g |= ((j >> tl[lh]) & 1) << lh;
      if (!(G[2 * (j * K + j)] == 1.0 && G[2 * (j * K + j) + 1] == 0.0)) unit_slot[g] = 0;
    }
  }

  for (uint64_t base_slice = 0; base_slice < nslices; ++base_slice) {
    if (base_slice & hmask) continue;
    for (int g = 0; g < G_; ++g) {
      uint64_t sid = base_slice;
      for (int l = 0; l < h; ++l)
        if ((g >> l) & 1) sid |= (uint64_t)1 << (high[l] - sl);
      slice_ids[g] = sid;
    }
    int untouched[32], any_touched = 0;
    for (int g = 0; g < G_; ++g) {
      untouched[g] = s->lazy && ((base_slice & chigh) != chigh || unit_slot[g]);
      if (!untouched[g]) any_touched = 1;
    }
    if (!any_touched) {
      /* the group keeps its streams; each slice's pending scale takes this pass's sigma */
      for (int g = 0; g < G_; ++g) {
        for (size_t bi = 0; bi < S / B; ++bi) {
          uint64_t blk = (slice_ids[g] << (sl - bl)) + bi;
          new_streams[blk] = s->streams[blk];
          new_lens[blk] = s->lens[blk];
          new_infos[blk] = s->infos[blk];
          s->streams[blk] = NULL;
        }
        s->scale[slice_ids[g]] = s->scale[slice_ids[g]] * sigma;
        s->skipped++;
      }
      continue;
    }
    /* Decompress(S) for every slice of the group */
    for (int g = 0; g < G_; ++g)
      for (size_t bi = 0; bi < S / B; ++bi) {
        uint64_t blk = (slice_ids[g] << (sl - bl)) + bi;
        orc_decompress_block_k(s->streams[blk], s->lens[blk], bl, s->dtype, s->eb, s->chunk,
                               buf + ((size_t)g * S + bi * B) * 2 * cs);
      }
    /* Normalize(S); second mode: the slice's pending scale joins sigma, t = fl(sigma c_s),
     * and a slice left unchanged is not scaled (only a diagonal gate leaves some slots of a
     * processed group unchanged, and those slots' values then pass the gate unmixed) */
    for (int g = 0; g < G_; ++g) {
      if (untouched[g]) continue;
      const double t = s->lazy ? sigma * s->scale[slice_ids[g]] : sigma;
      const float t_f = s->lazy ? (float)t : sigma_f;
      for (size_t e = (size_t)g * S * 2; e < (size_t)(g + 1) * S * 2; ++e) {
        if (s->dtype == ORC_C128) ((double*)buf)[e] = t * ((double*)buf)[e];
        else ((float*)buf)[e] = t_f * ((float*)buf)[e];
      }
    }
    /* GateComputation(G, S): global index i lives in group slot g (its high-target bits)
     * at offset i mod S */
    {
      /* tuples are enumerated from the group slot whose high-target bits are zero */
      for (size_t off = 0; off < S; ++off) {
        uint64_t base = (slice_ids[0] << sl) | off;
        int skip = 0;
        for (int l = 0; l < k; ++l)
          if (targets[l] < sl && ((base >> targets[l]) & 1)) skip = 1;
        if (skip || (base & cmask) != cmask) continue;
        size_t pos[32];
        for (int m = 0; m < K; ++m) {
          uint64_t gi = tuple_index(base, targets, k, m);
          int slot = 0;
          for (int l = 0; l < h; ++l)
            if ((gi >> high[l]) & 1) slot |= 1 << l;
          pos[m] = (size_t)slot * S + (size_t)(gi & (S - 1));
        }
        if (s->dtype == ORC_C128) {
          double* a = (double*)buf;
          cd y[32], z[32];
          for (int m = 0; m < K; ++m) {
            y[m].re = a[2 * pos[m]];
            y[m].im = a[2 * pos[m] + 1];
          }
          gate_tuple_d(G, k, y, z);
          for (int m = 0; m < K; ++m) {
            a[2 * pos[m]] = z[m].re;
            a[2 * pos[m] + 1] = z[m].im;
          }
        } else {
          float* a = (float*)buf;
          cf y[32], z[32];
          for (int m = 0; m < K; ++m) {
            y[m].re = a[2 * pos[m]];
            y[m].im = a[2 * pos[m] + 1];
          }
          gate_tuple_f(Gf, k, y, z);
          for (int m = 0; m < K; ++m) {
            a[2 * pos[m]] = z[m].re;
            a[2 * pos[m] + 1] = z[m].im;
          }
        }
      }
    }
    /* Compress(S) */
    for (int g = 0; g < G_; ++g) {
      if (untouched[g]) {  /* second mode: the stream stays, the scale takes sigma */
        for (size_t bi = 0; bi < S / B; ++bi) {
          uint64_t blk = (slice_ids[g] << (sl - bl)) + bi;
          new_streams[blk] = s->streams[blk];
          new_lens[blk] = s->lens[blk];
          new_infos[blk] = s->infos[blk];
          s->streams[blk] = NULL;
        }
        s->scale[slice_ids[g]] = s->scale[slice_ids[g]] * sigma;
        s->skipped++;
        continue;
      }
      for (size_t bi = 0; bi < S / B; ++bi) {
        uint64_t blk = (slice_ids[g] << (sl - bl)) + bi;
        size_t len = orc_compress_block_k(buf + ((size_t)g * S + bi * B) * 2 * cs, bl, s->dtype,
                                          s->eb, s->chunk, tmp, &new_infos[blk]);
        new_streams[blk] = (uint8_t*)malloc(len);
        memcpy(new_streams[blk], tmp, len);
        new_lens[blk] = len;
      }
      s->scale[slice_ids[g]] = 1.0;
    }
  }
  for (uint64_t b = 0; b < s->nblocks; ++b) free(s->streams[b]);
  free(s->streams);
  free(s->lens);
  free(s->infos);
  s->streams = new_streams;
  s->lens = new_lens;
  s->infos = new_infos;
  free(buf);
  free(slice_ids);
  free(tmp);
  s->norm = stored_norm(s);
  if (!(s->norm > 0) || !isfinite(s->norm)) return -2;
  return 0;
}
