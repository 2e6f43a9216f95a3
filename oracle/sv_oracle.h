/*
 * sv_oracle.h — CPU oracle for the compressed state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, the smoke check and the bench's CPU baseline
 * may call anything declared here. The product (the CUDA library) shares no code,
 * header, table or constant with this file.
 *
 * What it computes (Wu, Di, Cappello, Finkel, Alexeev, Chong, "Memory-Efficient
 * Quantum Circuit Simulation by Using Lossy Data Compression", PMES 2018):
 *   - O1, the "original simulator": a plain full-amplitude state vector updated gate by
 *     gate (Sec. I: full amplitude-vector update, 2^n complex doubles).
 *   - the block codec: SZ-style error-bounded lossy compression (Sec. II), restated as
 *     linear quantization under an absolute bound, a 1-D Lorenzo predictor on the
 *     integer codes, 16-bit quantization symbols, canonical Huffman coding.
 *   - O2, Algorithm 1: for each gate, for each slice: Decompress, Normalize,
 *     GateComputation, Compress.
 *
 * The byte layout of a block stream and every rounding step are fixed by the format
 * description in the repository's design notes; this file implements it independently.
 */
#ifndef SV_ORACLE_H
#define SV_ORACLE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_C64 1  /* complex64: float components, FP32 gate arithmetic */
#define ORC_C128 2 /* complex128: double components, FP64 gate arithmetic */

#define ORC_MODE_CONST 0
#define ORC_MODE_HUFF 1
#define ORC_MODE_PACK 2

/* Per-block side results of compressing one block. */
typedef struct {
  int mode;          /* ORC_MODE_* */
  int n_verbatim;    /* values stored raw */
  int n_escape;      /* Lorenzo deltas outside the 16-bit symbol range */
  int n_distinct;    /* distinct 16-bit symbols (0 for CONST) */
  uint64_t sq_lo;    /* exact sum of q^2 over non-verbatim values, low 64 bits */
  uint64_t sq_hi;    /* ... high 64 bits */
  double vsum;       /* pairwise sum over the block's values of x*x (verbatim) or 0 (others) */
} orc_block_info;

/* Upper bound of one block stream in bytes. */
size_t orc_block_bound(int block_log2, int dtype);

/* Compress one block of B = 2^block_log2 amplitudes (2B interleaved re/im values of the
 * dtype's component type). Returns the stream length in bytes (multiple of 16), or 0
 * on an argument error. `out` must hold orc_block_bound() bytes. */
size_t orc_compress_block(const void* values, int block_log2, int dtype, double eb,
                          uint8_t* out, orc_block_info* info);

/* Decompress one block stream into 2B values of the dtype's component type.
 * Returns 0 on success, a negative number when the stream is malformed. */
int orc_decompress_block(const uint8_t* stream, size_t len, int block_log2, int dtype,
                         double eb, void* values_out);

/* The same with the Huffman decode-chunk size (symbols per stored chunk bit count: 16, 32 or
 * 64; the functions above use 32). It changes the bytes of HUFF streams. */
size_t orc_compress_block_k(const void* values, int block_log2, int dtype, double eb, int chunk,
                            uint8_t* out, orc_block_info* info);
int orc_decompress_block_k(const uint8_t* stream, size_t len, int block_log2, int dtype,
                           double eb, int chunk, void* values_out);

/* Huffman code lengths by the two-queue method (leaves sorted by frequency, then symbol;
 * ties between queue heads go to the leaf). freq[i] > 0 for i < n; lens_out[i] receives
 * the length of symbol i. Exposed for tests. Returns the maximum length. */
int orc_huffman_lengths(const uint32_t* freq, const uint32_t* sym, int n, int* lens_out);

/* ---- O1: plain state vector ---- */
/* Apply a k-qubit gate G (row-major 2^k x 2^k complex, (re,im) pairs, FP64) to the
 * amplitudes `state` (2^n interleaved values of the dtype's component type).
 * targets[0] is the least significant bit of G's basis index. Controls must be 1. */
void orc_plain_apply(void* state, int n, int dtype, const double* G, const int* targets,
                     int k, const int* controls, int n_controls);

/* ---- O2: Algorithm 1 ---- */
typedef struct orc_csim orc_csim;
orc_csim* orc_csim_create(int n, int slice_log2, int block_log2, int dtype, double eb,
                          uint64_t basis_index);
orc_csim* orc_csim_create_k(int n, int slice_log2, int block_log2, int dtype, double eb,
                            uint64_t basis_index, int chunk);
void orc_csim_destroy(orc_csim* s);
/* One gate pass over every slice. Returns 0, or -1 on an argument error, -2 when the
 * stored norm collapses to zero or is not finite. */
int orc_csim_apply(orc_csim* s, const double* G, const int* targets, int k,
                   const int* controls, int n_controls);
/* Decompressed (reconstructed, un-normalized) amplitudes of the whole state. */
void orc_csim_read(const orc_csim* s, void* out);
double orc_csim_norm(const orc_csim* s);  /* N of the stored state */
uint64_t orc_csim_nblocks(const orc_csim* s);
size_t orc_csim_block_stream(const orc_csim* s, uint64_t block, const uint8_t** ptr);
uint64_t orc_csim_total_bytes(const orc_csim* s);
/* Replace the stored state by the compression of `values` (2^n amplitudes). */
void orc_csim_load(orc_csim* s, const void* values);

/* ---- O2L: the second mode, lazy normalization with slice skipping ----
 * Algorithm 1 visits every slice with every gate. In this mode a slice the gate leaves
 * unchanged (the group's controls above the slice are not all 1, or G is diagonal with every
 * entry of the slice's rows exactly 1) is not decompressed or recompressed: its stream stays
 * and its pending normalization is kept as a scale c_s (c_s <- fl(c_s sigma)); the state it
 * represents is c_s x'. A slice the gate changes is normalized with t = fl(sigma c_s) in
 * place of sigma and recompressed with c_s = 1. The stored norm becomes fl(N_1 + R): N_1 the
 * O2 formula over the slices of scale 1, R the pairwise sum over slices of fl(fl(c_s c_s) N_s).
 * With every scale 1 and no slice skipped a pass is O2's pass exactly. Results differ from
 * O2 otherwise (skipped slices are not requantized).
 * set_lazy: switch the mode (-1 while a scale is pending). scales: c_s per slice (2^(n -
 * slice_log2) doubles). skipped: slices left unchanged so far. read_values: c_s x' as FP64
 * (re, im) pairs for either dtype. */
int orc_csim_set_lazy(orc_csim* s, int on);
void orc_csim_scales(const orc_csim* s, double* out);
uint64_t orc_csim_skipped(const orc_csim* s);
void orc_csim_read_values(const orc_csim* s, double* out);

#ifdef __cplusplus
}
#endif
#endif
