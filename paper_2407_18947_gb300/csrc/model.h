// The RT-CC3 residual graph (one RK4 stage for one field) and the small
// device kernels of the integrator around it.
#pragma once

#include "common.h"
#include "engine.h"
#include "rotation.h"

namespace rtcc3 {

// Field profile (Eq. 14 cosine, Eq. 32 Gaussian, static), one per batch slot.
struct FieldDev {
  int kind;  // 0 none, 1 static, 2 cos, 3 gauss, 4 linear-ramped cos, 5 quadratic-ramped cos
  double amp, omega, center, width;
  double dir[3];
};

// Hamiltonian constants on the device in the compute precision R, plus the
// FP64 copies used by denominators and reductions.
template <typename R>
struct Hamil {
  int o = 0, v = 0, n = 0, naux = 0;
  Cx<R>* L = nullptr;     // naux x n x n, DF factors (real, stored complex)
  Cx<R>* h = nullptr;     // n x n core Hamiltonian h = f - G[D_ref]
  Cx<R>* ones = nullptr;  // n ones (for traces)
  double* eps = nullptr;  // n orbital energies (FP64)
  double* mu = nullptr;   // 3 x n x n dipole matrices (FP64)
  double* osum = nullptr;  // o^3 sums e_i + e_j + e_k (FP64)
  double* vsum = nullptr;  // v^3 sums e_a + e_b + e_c (FP64)
  R* osum_r = nullptr;     // the same sums rounded once to R
  R* vsum_r = nullptr;
  int* orbit_order = nullptr;  // o^3 occupied blocks, permutation orbits consecutive
  // mid-gap energy c = (e_homo + e_lumo) / 2 subtracted from every orbital
  // energy (and every field-dressed eigenvalue) entering a sum table: the
  // denominators D = vsum - osum are unchanged (three terms on each side),
  // and with occupied sums below zero and virtual sums above, the one
  // rounding of each sum to the compute precision cannot cancel in D
  double eshift = 0.0;
};

// Node ids of one recorded stage.
struct StageNodes {
  int t1 = -1, t2 = -1, w = -1;  // leaves
  int r1 = -1, r2 = -1, e = -1;  // T residuals and the correlation part of the energy
  int t3 = -1;                   // final triples amplitudes (for diagnostics)
};

struct StageOptions {
  bool ccsd = true;  // false: R1, R2 hold only the triples terms X1, X2
  bool triples = true;
  // split-TF32 tensor cores beyond the triples: 0 triples only, 1 also the
  // dressed-integral product g = L~^T L~ (and its adjoints), 2 every
  // contraction of the stage
  int tc_scope = 0;
  bool need_grad = true;
  bool field_terms = true;  // include the V-coupling of the triples equation
  bool rotation = true;     // field-dressed eigenbasis (else fixed-point sweeps)
  int field_iters = 1;      // fixed-point sweeps of the triples equation
  // 0: the triples tensors are stored whole (o^3 v^3 each); k > 0: blocked,
  // slabs of k first occupied indices with W and t3 recomputed in the
  // reverse pass (the fixed-point field solver always stores)
  int triples_chunk = 0;
  // eigenbasis of this stage's O and V already decomposed on the engine's side
  // stream (enqueued there before this stage), else null: decomposed in-stage
  const BasisBuffers* basis = nullptr;
};

// Records dressing, the CCSD residual, the triples and the energy (the same
// equations as the paper's Appendix A: Eqs. A4, A8, A10-A12, A21, A22, A25,
// A30) onto the engine's tape.  `fill` is called right after the leaves are
// created so the caller can write t1, t2 and w before any operation reads them.
template <typename R, typename Fill>
StageNodes record_stage(Engine<R>& E, const Hamil<R>& H, const StageOptions& opt, Fill&& fill);

// ---- integrator kernels (model.cu) --------------------------------------
// Write the stage inputs: t = y + ch * kprev (FP64 -> R), lambda stage values
// (kept for the seeds) and w = -E(t_s) dir . mu.
template <typename R>
void launch_stage_inputs(const double2* y, const double2* kprev, double ch, Cx<R>* t1, Cx<R>* t2,
                         Cx<R>* l1s, Cx<R>* l2s, Cx<R>* w, const double* mu, const FieldDev* f,
                         const double* tdev, double dt, int o, int v, int n, cudaStream_t s);
// O and V (as launch_field_matrices) of the NEXT Runge-Kutta stage from this
// stage's forward residual: that stage's t1 = y1 + ch * (-i r1) (y1 alone if
// r1 is null) and
// w = -E(*tdev + dt) dir . mu, both rounded to R exactly as the stage inputs
// are, dressed as w~ = (1 - tau) w (1 + tau) with the FP64 sums
//   O[i][l] = e_i d_il + w_li + sum_a w_l,a t1_ia,
//   V[a][d] = e_a d_ad + w_ad - sum_i t1_ia w_i,d.
template <typename R>
void launch_next_field_matrices(const double2* y, const Cx<R>* r1, double ch, const double* mu,
                                const FieldDev* f, const double* tdev, double dt,
                                const double* eps, int o, int v, double2* Mo, double2* Mv,
                                cudaStream_t s);
// grad(e) = 1, grad(r1) = l1s, grad(r2) = l2s / 2 (Lagrangian E + l1.R1 + 1/2 l2.R2).
template <typename R>
void launch_seeds(Cx<R>* ge, Cx<R>* gr1, Cx<R>* gr2, const Cx<R>* l1s, const Cx<R>* l2s, int o,
                  int v, cudaStream_t s);
// k = (-i R1, -i R2, +i (g1 + 2 w_ov), +i (g2 + g2^T)); acc += hw * k; optional
// k copy. w_ov is the FP64 field operator's occupied-virtual block at time
// *tdev + dt (the t1 derivative of the energy's field term, kept out of the
// graph).
template <typename R>
void launch_stage_output(const Cx<R>* r1, const Cx<R>* r2, const Cx<R>* g1, const Cx<R>* g2,
                         double2* kout, double2* acc, double hw, const double* mu,
                         const FieldDev* f, const double* tdev, double dt, int o, int v,
                         cudaStream_t s);
// Where a propagation writes its observables (device struct, so a captured
// step graph does not depend on the output buffers of one call): entry
// (slot * stride + step) of dip (x3) and en.
struct TrajDesc {
  double2* dip;
  double2* en;
  long long stride;
  // additional one-electron observables sum_pq D_pq O_pq (e.g. the magnetic
  // dipole of Section 2.2.3): nobs complex n x n operators, values at
  // obs[entry * nobs + k]
  double2* obs = nullptr;
  const double2* ops = nullptr;
  int nobs = 0;
};
// dipole[3] = sum_pq D_pq mu^x_pq + 2 sum_i mu^x_ii + 2 sum_ia t1_ia mu^x_ia,
// each additional observable the same with its operator, and energy =
// e + 2 sum_i w_ii + 2 sum_ia t1_ia w_ia (w at time *tdev + dt), all in FP64:
// the graph's density D and energy e leave out the field-dressed reference
// terms. t1 is the FP64 state the stage was evaluated at (its first o*v
// entries). Written at entry (slot * td->stride + *step) (step may be NULL:
// entry slot * stride).
template <typename R>
void launch_observables(const Cx<R>* D, const Cx<R>* e, const double2* t1, const double* mu,
                        const FieldDev* f, const double* tdev, double dt, int o, int v, int nobs,
                        const TrajDesc* td, int slot, const int* step, cudaStream_t s);
// Host-readable FP64 copy of the residuals: out = [r1, r2, g1 + 2 w_ov, g2 + g2^T]
// (w at time *tdev).
template <typename R>
void launch_residual_export(const Cx<R>* r1, const Cx<R>* r2, const Cx<R>* g1, const Cx<R>* g2,
                            const double* mu, const FieldDev* f, const double* tdev, double2* out,
                            int o, int v, bool have_grad, cudaStream_t s);
// Jacobi update of one amplitude pair: x1 -= r1 / D1, x2 -= r2 / D2 (orbital-
// energy denominators, FP64) and max |r| into *maxr.
void launch_jacobi(double2* x1, double2* x2, const double2* r1, const double2* r2,
                   const double* eps, int o, int v, double* maxr, cudaStream_t s);
// DIIS support (ground state): e = -r / D, xs = x + e over one contiguous
// amplitude block [x1 | x2]; max |r| into *maxr.
void launch_diis_step(const double2* x, const double2* r, const double* eps, int o, int v,
                      double2* xs, double2* es, double* maxr, cudaStream_t s);
// out[k] = sum conj(E_k) . e for k < m (vectors of length len, stride len).
void launch_dots(const double2* E, const double2* e, int m, size_t len, double2* out, cudaStream_t s);
// x = sum_k c_k X_k.
void launch_lincomb(const double2* X, const double2* c, int m, size_t len, double2* x, cudaStream_t s);
// y = acc and flag non-finite entries (first bad step index kept in *bad_step).
void launch_step_finish(double2* y, const double2* acc, size_t ny, const int* step, int* bad_step,
                        bool c64,
                        cudaStream_t s);
// *t += h; ++*step.
void launch_step_advance(double* tdev, double h, int* step, cudaStream_t s);
// Load t1, t2 (complex128 device arrays) into compute-precision leaves.
template <typename R>
void launch_load_amplitudes(const double2* t1, const double2* t2, Cx<R>* d1, Cx<R>* d2, int o,
                            int v, cudaStream_t s);
// out (complex128) = in (compute precision), n elements.
template <typename R>
void launch_export(const Cx<R>* in, double2* out, size_t n, cudaStream_t s);
// w = -E(t) dir . mu for the field of one slot at time *tdev + dt.
template <typename R>
void launch_field_operator(Cx<R>* w, const double* mu, const FieldDev* f, const double* tdev,
                           double dt, int n, cudaStream_t s);
void launch_copy_c128(double2* dst, const double2* src, size_t n, cudaStream_t s);
void launch_stage_prep_acc(double2* acc, const double2* y, size_t ny, cudaStream_t s);

}  // namespace rtcc3
