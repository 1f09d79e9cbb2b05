// Contractions whose output is small or a single column, where the generic
// 64 x 64 tiled kernel wastes most of its tile and re-reads the long operand.
//
//   reduce_small: C[m,n] = sum_k A[m,k] B[n,k] with the whole M x N output held
//     by every CTA (M, N <= 64, or N = 1 and M <= 512); each CTA sums one K
//     chunk, so both operands stream from HBM exactly once.  Used for the
//     triples slot densities (ijkabc,ijkdbc->ad; ijkabc,ljkabc->li) and the
//     X1-type back-contractions (ijkabc,jkbc->ia).
//   gemv: C[m] = sum_k A[m,k] B[k] for a long output column (M > 512): one
//     warp per output when A is contiguous along k, else one thread per output
//     with consecutive threads on consecutive m.
// Addresses come from the contraction's offset tables (element offsets):
// A[aoff + aM[m] + aK[k]], B[boff + bN[n] + bK[k]], C[coff + cM[m] + cN[n]].
#pragma once

#include "common.h"

namespace rtcc3 {

// Output-tile configurations of reduce_small (0 = not applicable).
enum SmallCfg : int {
  kSmallNone = 0, kSmall48 = 1, kSmall16 = 2, kSmallCol256 = 3, kSmallCol512 = 4, kSmall64 = 5,
  kSmall10 = 6, kSmall40 = 7
};

// Configuration for an M x N output (N <= M expected; returns kSmallNone
// when the shape is not small).
int small_output_config(long long M, long long N);
// Depth of one K slice for a configuration (chunks are multiples of it).
int small_output_bk(int cfg, int elem_bytes);

// nsplit > 1: CTA s sums K range [s kchunk, (s+1) kchunk) into
// part[m][n][s] and a second kernel adds the splits in a fixed order into C
// (deterministic); nsplit == 1: C (+)= alpha * result directly.
template <typename R>
void launch_reduce_small(int cfg, bool a_kc, bool b_kc, const Cx<R>* A, long long aoff,
                         const long long* aM, const long long* aK, const Cx<R>* B, long long boff,
                         const long long* bN, const long long* bK, Cx<R>* C, long long coff,
                         const long long* cM, const long long* cN, int M, int N, int K, int nsplit,
                         int kchunk, double alpha, bool accumulate, Cx<R>* part, cudaStream_t s);

// Outer products (K = 1): C[coff + cM[m] + cN[n]] (+)= alpha A[aoff + aM[m] +
// aK[0]] B[boff + bN[n] + bK[0]], n along the output's contiguous index: a
// streaming pass over C (the reverse-pass products that spread a vector over
// the o^3 v^3 cotangent).
template <typename R>
void launch_outer(const Cx<R>* A, long long aoff, const long long* aM, const long long* aK,
                  const Cx<R>* B, long long boff, const long long* bN, const long long* bK,
                  Cx<R>* C, long long coff, const long long* cM, const long long* cN, int M, int N,
                  double alpha, bool accumulate, cudaStream_t s);

template <typename R>
void launch_gemv(bool a_kc, const Cx<R>* A, long long aoff, const long long* aM, const long long* aK,
                 const Cx<R>* B, long long boff, const long long* bK, Cx<R>* C, long long coff,
                 const long long* cM, int M, int K, double alpha, bool accumulate, cudaStream_t s);

}  // namespace rtcc3
