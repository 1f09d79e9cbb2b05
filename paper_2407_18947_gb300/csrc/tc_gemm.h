// Tensor-core (tcgen05, sm_103a) path for the large complex contractions.
//
// A complex contraction C[m,n] (+)= alpha sum_k A[m,k] B[n,k] is run as one
// real GEMM: A is packed K-major with (re, im) interleaved along K (M x 2K
// real), B is packed as its real 2x2 embedding ([Br -Bi; Bi Br] per
// element, 2N x 2K real), and the real product M x 2N is the interleaved
// complex result.  Operands are rounded to TF32 (split into hi + lo parts,
// three products) or converted to BF16; accumulation is FP32 in tensor
// memory.  The epilogue scatters into any strided output view through the
// contraction's offset tables (or writes FP32 partials for split-K).  Long
// TF32 sums read A straight from its source through the offset tables
// (tc_gemm_direct) instead of a packed copy.
#pragma once

#include "common.h"

namespace rtcc3 {

struct TcOperands {
  int M = 0, N = 0, K = 0;  // complex extents
  int Kp = 0;               // packed real K of A (multiple of the K tile)
  int elem_bytes = 4;       // 4: TF32 operands, 2: BF16 operands
  // TF32: A is packed as raw FP32 and split into hi + lo TF32 parts in the
  // GEMM's shared memory, B is packed as [hi | lo] (width 2 Kp); one GEMM
  // sums hi.hi + hi.lo + lo.hi (FP32-level products at three times the
  // tensor work, A read once).
  bool split = false;
  // the product is bound by its output (short sum): two CTAs per SM with
  // narrower tiles, so that epilogues overlap main loops
  bool out_bound = false;
  // A packed in tiles of 128 rows x 128 bytes of K, each stored as the
  // 128-byte-swizzled shared-memory image the MMA reads and the tiles of one
  // row block consecutive along K, so a long sum streams A as contiguous
  // 16 KB blocks (set iff tc_chained)
  bool a_tiled = false;
  // clock cycles a wait on another warp's progress may spin before the
  // kernel gives up (raises its error flag, drains its own copies and MMAs,
  // frees its tensor memory and returns); 0: the default of about 2 s
  long long wait_budget = 0;
};

// GEMM column tile (real columns) for Nr = 2N real output columns: the
// narrowest of 64 / 128 / 256 that holds them (one column tile, the A tile
// read once), at most 128 for output-bound products.
inline int tc_tile_n(int Nr, bool out_bound) {
  if (out_bound) return Nr <= 64 ? 64 : 128;
  // long sums with narrow outputs: the tile's unused columns are tensor-core
  // work the operand stream has to wait for (N = 10 complex -> 20 real
  // columns, N = 38 -> 76)
  if (Nr <= 32) return 32;
  if (Nr <= 64) return 64;
  if (Nr <= 96) return 96;
  if (Nr <= 128) return 128;
  return 256;
}
// CTAs resident per SM for the two variants.
inline int tc_ctas_per_sm(bool out_bound) { return out_bound ? 2 : 1; }

// Whether a long sum split into nsplit accumulation chains runs as the
// chained kernel (several chains per CTA, tiled A): every chain non-empty and
// an N tile of at most 128 real columns.
inline bool tc_chained(const TcOperands& op, int nsplit) {
  if (op.out_bound || nsplit < 2 || tc_tile_n(2 * op.N, false) > 128) return false;
  const int nkb = op.Kp / (128 / op.elem_bytes);
  const int per = (nkb + nsplit - 1) / nsplit;
  return (nkb + per - 1) / per == nsplit;
}

// Whether a TF32 long sum runs as the direct kernel (A gathered from its
// source through its tables, no packed copy): the chained kernel's shapes.
inline bool tc_direct(const TcOperands& op, int nsplit) {
  return op.split && op.elem_bytes == 4 && tc_chained(op, nsplit);
}

// Pack A (complex, addressed by tables) into a K-major real buffer of packed
// width Kp: raw FP32 for TF32 (elem_bytes 4), BF16 otherwise.  kfast: the
// source is contiguous along k (else along the row index); the packing
// kernel reads along that index and writes packed rows along k.
// tiled: the TcOperands::a_tiled layout (rows rounded up to 128).
void tc_pack_a(const float2* A, const long long* aM, const long long* aK, long long aoff, int M,
               int K, int Kp, int elem_bytes, bool kfast, bool tiled, void* out, cudaStream_t s);
// Pack B as its 2x2 real embedding: rows 2n (real part) and 2n+1 (imaginary
// part); for TF32 as [hi | lo] K segments (row width 2 Kp).
void tc_pack_b(const float2* B, const long long* bN, const long long* bK, long long boff, int N,
               int K, int Kp, int elem_bytes, bool kfast, void* out, cudaStream_t s);

// C[cB + cM[m] + cN[n]] (+)= alpha * (Apack Bpack^T)[m, 2n..2n+1] as complex.
// nsplit > 1: K is split over CTAs; partial sums (M x 2N FP32 per split) go
// to `partial` and tc_split_finish reduces them into C.  Returns false if the
// shape is not supported by the tensor-core path.
bool tc_gemm(const void* Apack, const void* Bpack, const TcOperands& op, float2* C,
             const long long* cM, const long long* cN, long long coff, float alpha, bool accumulate,
             int nsplit, float* partial, int* err_flag, cudaStream_t s);
// The long sum C = A B (TF32 split, nsplit chains into `partial`, reduced by
// tc_split_finish) with A read from its source: element (m, k) at
// A[aoff + aM[m] + aK[k]] (a_kc: the source is contiguous along k).
bool tc_gemm_direct(const float2* A, long long aoff, const long long* aM, const long long* aK,
                    bool a_kc, const void* Bpack, const TcOperands& op, int nsplit, float* partial,
                    int* err_flag, cudaStream_t s);
void tc_split_finish(const float* partial, int nsplit, int M, int N, float2* C, const long long* cM,
                     const long long* cN, long long coff, float alpha, bool accumulate,
                     cudaStream_t s);

// Packed K for a complex K at the given element size (K tile = 128 bytes).
// Measured dense rate (TFLOP/s) of one pipe on the current device: 0 TF32
// tcgen05 MMA, 1 BF16 tcgen05 MMA, 2 FP32 FMA, 3 FP64 FMA (probe kernels, no
// global memory traffic).
double measure_pipe_tflops(int which, int* err_flag, cudaStream_t s);

inline int tc_packed_k(int K, int elem_bytes) {
  const int tile = 128 / elem_bytes;
  return ((2 * K + tile - 1) / tile) * tile;
}

}  // namespace rtcc3
