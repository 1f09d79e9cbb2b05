// Field-dressed eigenbasis of the triples equation.
//
// With a field, the triples solve eps3 t3 + [V~, T3] = rhs (Eq. 4 / Eq. A12 with
// dt3/dt = 0) couples every triple through the dressed perturbation on each
// index: A = sum over virtual slots of V - sum over occupied slots of O with
//   V = diag(e_vir) + v~_vv          (acting as (V t)_a = sum_d V_ad t_d)
//   O = diag(e_occ) + (v~_oo)^T      (acting as (O t)_i = sum_l v~_li t_l + e_i t_i).
// A is a Kronecker sum, so with V = S_v L_v S_v^-1 and O = S_o L_o S_o^-1 the
// change of basis t3 = K t3' (S_o on each occupied, S_v on each virtual index)
// makes it diagonal with complex denominators l_a + l_b + l_c - l_i - l_j - l_k:
// the triples are formed, divided and contracted in that basis exactly as in
// the field-free case, with the small inputs (t2, integral blocks) rotated in
// O(N^5) and no iteration.
#pragma once

#include "common.h"

namespace rtcc3 {

constexpr int kEigMaxN = 112;  // matrix in shared memory (112^2 complex128 = 196 KiB)
// A failed decomposition raises the shared device error flag with a code that
// says why: kEigStatusBase | reason << 20 | n << 10 | row of the active block.
constexpr int kEigStatusBase = 1 << 24;
constexpr int kEigNoConvergence = 1, kEigNonFinite = 2;
__host__ __device__ constexpr int eig_status(int reason, int n, int row) {
  return kEigStatusBase | (reason << 20) | (n << 10) | row;
}

// One matrix M[n][n] (row-major, complex128) -> S, S^-1 (row-major, complex128)
// and eigenvalues lam[n]; ws holds 3 n^2 complex128 of scratch.
struct EigJob {
  const double2* M;
  int n;
  double2* S;
  double2* Sinv;
  double2* lam;
  double2* ws;
  int max_sweeps = 0;  // QR sweeps before giving up (0: 60 n + 100)
};
// Both matrices of a stage in one launch (one warp each).  fp32: complex64
// arithmetic (for the complex64 graphs), else complex128.  *status is raised
// if the QR sweeps do not converge or a matrix is not finite.
void launch_eig(const EigJob& a, const EigJob& b, bool fp32, int* status, cudaStream_t s);

// The eigenbasis of one stage computed ahead of it (complex128, owned by the
// caller and kept between stages): M* the matrices, S*, Si* = S^-1, l* the
// eigenvalues, ws* the eigensolver scratch (3 n^2 each).
struct BasisBuffers {
  double2 *Mo = nullptr, *Mv = nullptr, *So = nullptr, *Sio = nullptr, *Sv = nullptr,
          *Siv = nullptr, *lo = nullptr, *lv = nullptr, *wso = nullptr, *wsv = nullptr;
};

// O (o x o) and V (v x v) of the current stage from the dressed perturbation w~
// (n x n, compute precision) and the orbital energies.
template <typename R>
void launch_field_matrices(const Cx<R>* wt, const double* eps, int o, int v, double2* Mo,
                           double2* Mv, cudaStream_t s);
// osum[(i o + j) o + k] = l_i + l_j + l_k and vsum likewise (summed in FP64,
// rounded once to the compute precision R).
template <typename R>
void launch_lambda_sums(const double2* lo, const double2* lv, int o, int v, double shift,
                        Cx<R>* osum, Cx<R>* vsum, cudaStream_t s);
// dst (compute precision) = src (complex128), n elements.
template <typename R>
void launch_to_precision(const double2* src, Cx<R>* dst, size_t n, cudaStream_t s);

}  // namespace rtcc3
