/*
 * librtcc3 -- real-time CC3 (RT-CC3) approximate-triples hot path on one GPU.
 *
 * The library evaluates, for a closed-shell molecule in a time-dependent
 * electric field, the right-hand sides of the RT-CC3 equations of motion
 *
 *     i dt_mu/dt      = <mu| H + [H,T2] + [H,T3] (+ 1/2[[H,T2],T2]) |0>     (Eqs. 2, A10-A11)
 *    -i dlambda_mu/dt = dL_CC3/dt_mu                                      (Eqs. 3, A13-A14)
 *
 * where H is the T1-transformed Hamiltonian (Eq. 8, Eq. A4), the triples t3
 * solve their stationarity condition (Eq. 4 / Eq. A12 with dt3/dt = 0) and
 * L_CC3 is the CC3 Lagrangian of Eq. A6, and propagates (t1, t2, lambda1,
 * lambda2) with classical fourth-order Runge-Kutta, returning the dipole
 * moment sum_pq D_pq mu_pq (D the one-electron density, dL/dV) and the
 * energy <0|H + [H,T2]|0> - E_ref (Eq. A8) at every step.
 *
 * Conventions
 *   - nocc occupied and nvir virtual spatial orbitals, nmo = nocc + nvir,
 *     occupied first; canonical reference with orbital energies eps (Eq. A2).
 *   - two-electron integrals are density fitted: (pq|rs) = sum_P L[P][p][q] L[P][r][s]
 *     (chemists' order; the paper's <pq|rs> is (pr|qs)).
 *   - the field couples as V = -E(t) . mu (Eq. 10).
 *   - complex numbers are interleaved (re, im) pairs of double (C99
 *     "double _Complex" compatible), row-major arrays:
 *       t1[i][a] = t_i^a, t2[i][j][a][b] = t_ij^ab (= t_ji^ba),
 *       l1[i][a] = lambda_a^i, l2[i][j][a][b] = lambda_ab^ij,
 *     with the Lagrangian normalised as L = E + sum l1 R1 + 1/2 sum l2 R2.
 *
 * Errors: every call returns RTCC3_OK (0) or a negative status; no exception
 * or abort crosses the ABI.  rtcc3_last_error() returns a message for the last
 * failing call on a context.  A context is used by one host thread at a time.
 * Host buffers passed in are copied; the caller keeps ownership.
 */
#ifndef RTCC3_H
#define RTCC3_H

#ifdef __cplusplus
extern "C" {
#endif

#define RTCC3_OK 0
#define RTCC3_ERR_ARG (-1)           /* invalid argument or size */
#define RTCC3_ERR_OOM (-2)           /* device allocation failed */
#define RTCC3_ERR_CUDA (-3)          /* CUDA runtime error */
#define RTCC3_ERR_NONFINITE (-4)     /* NaN/Inf appeared in the propagated state */
#define RTCC3_ERR_TIMEOUT (-5)       /* a bounded device wait gave up */
#define RTCC3_ERR_NOT_CONVERGED (-6) /* ground-state iterations did not converge */
#define RTCC3_ERR_STATE (-7)         /* call out of order (e.g. no Hamiltonian set) */

/* Arithmetic of the residual evaluation.  The RK4 state, its update, the
 * orbital-energy divisions and the dipole/energy reductions are FP64 in every
 * mode. */
#define RTCC3_PREC_FP64 0 /* complex128 throughout */
#define RTCC3_PREC_FP32 1 /* complex64 residual graph on CUDA cores */
#define RTCC3_PREC_TF32 2 /* complex64 graph, triples contractions on tcgen05 TF32 */
#define RTCC3_PREC_BF16 3 /* complex64 graph, triples contractions on tcgen05 BF16 */

#define RTCC3_STORAGE_C128 0
#define RTCC3_STORAGE_C64 1

#define RTCC3_FIELD_NONE 0
#define RTCC3_FIELD_STATIC 1 /* E(t) = A                                   */
#define RTCC3_FIELD_COS 2    /* E(t) = A cos(omega t)                (Eq. 14) */
#define RTCC3_FIELD_GAUSS 3  /* E(t) = A exp(-(t - c)^2 / (2 w^2))   (Eq. 32) */
/* Ramped continuous waves (Section 2.2.4), ramp duration t_r = width, zero
 * for t < 0 and A cos(omega t) from t_r on:                                  */
#define RTCC3_FIELD_LRCW 4   /* E(t) = A (t / t_r) cos(omega t), t < t_r          */
#define RTCC3_FIELD_QRCW 5   /* E(t) = A 2 t^2 / t_r^2 cos(omega t), t < t_r / 2;
                                A [1 - 2 (t - t_r)^2 / t_r^2] cos(omega t), t < t_r */

typedef struct rtcc3_ctx rtcc3_ctx;

typedef struct rtcc3_options {
  int precision;     /* RTCC3_PREC_*                                          */
  int triples;       /* 1: CC3 (default); 0: CCSD only                       */
  int device;        /* CUDA device ordinal                                  */
  int use_graphs;    /* 1: capture one RK4 step as a CUDA graph and replay   */
  double field_tol;  /* target relative error of the field-coupled triples
                        fixed point (0: 1e-14 in FP64, 1e-8 otherwise)       */
  int field_solver;  /* field-coupled triples: 0 = field-dressed eigenbasis
                        (exact, default), 1 = fixed-point sweeps on the
                        stored triples (the paper's scheme)                   */
  int triples_chunk; /* triples storage: 0 = automatic (whole o^3 v^3
                        tensors when about 24 of them fit in 70% of the free
                        device memory, else blocked), -1 = always whole,
                        k > 0 = blocked: the (i,j,k) blocks in slabs of k
                        first occupied indices, W and t3 recomputed in the
                        reverse pass and never stored (Section 2.1 computes
                        the triples per (i,j,k) block); field_solver = 1
                        always stores                                         */
  long long spin_budget; /* clock cycles a bounded device wait (tensor-core
                        pipeline barriers) may spin before the kernel gives
                        up, drains its copies and the call returns
                        RTCC3_ERR_TIMEOUT; 0 = default (4e9, about 2 s)      */
  int eig_sweep_cap; /* QR sweeps the field eigensolver may take per matrix
                        before the call returns RTCC3_ERR_TIMEOUT; 0 =
                        default (60 n + 100)                                   */
  int tc_scope;      /* RTCC3_PREC_TF32 only, split-TF32 tensor cores for: 0 =
                        the triples (default; the rest on FP32 CUDA cores),
                        1 = also the dressed two-electron integrals
                        g = L~^T L~ and their adjoints, 2 = every
                        contraction of the stage                              */
  int storage;       /* propagated state: RTCC3_STORAGE_C128 (default) or
                        RTCC3_STORAGE_C64 (rounded to complex64 after every
                        RK4 step; the step itself is FP64)                    */
  int checked;       /* 1: every device tensor of a stage gets a 256-byte
                        canary, verified after the stage (RTCC3_ERR_STATE on
                        an overrun); no CUDA graphs.  Independently of this,
                        every operation's index ranges are checked on the
                        host against its tensors before it is launched       */
  int serial;        /* 1: every operation of a stage on the context's one
                        stream in recording order; 0 (default): independent
                        work (the two adjoints of a CUDA-core product, the
                        CCSD part beside the triples) on streams of its own,
                        joined before its results are read                    */
} rtcc3_options;

/* Fill *opt with defaults (FP64, triples on, device 0, graphs on, automatic
 * triples storage, default wait budgets). */
void rtcc3_default_options(rtcc3_options* opt);

/* Create a context for nbatch independent propagations (field slots).
 * nocc >= 1, nvir >= 1, 1 <= nbatch <= 64.  *out receives the handle. */
int rtcc3_create(int nocc, int nvir, int nbatch, const rtcc3_options* opt, rtcc3_ctx** out);
/* Release all device memory of the context.  NULL is accepted. */
int rtcc3_destroy(rtcc3_ctx* ctx);
const char* rtcc3_last_error(const rtcc3_ctx* ctx);

/* Hamiltonian (Eqs. A1-A3): eps[nmo] canonical orbital energies, Lfac[naux][nmo][nmo]
 * real DF factors symmetric in (p,q), dipole[3][nmo][nmo] real symmetric.  The
 * core operator is h = diag(eps) - G[D_ref], G_pq = sum_k 2(pq|kk) - (pk|kq),
 * so the reference is a canonical Hartree-Fock determinant.  Resets all slots
 * to zero amplitudes and time 0. */
int rtcc3_set_hamiltonian(rtcc3_ctx* ctx, const double* eps, int naux, const double* Lfac,
                          const double* dipole);

/* Hamiltonian from dense chemists' integrals eri[nmo][nmo][nmo][nmo] = (pq|rs)
 * (real, with the symmetries (pq|rs) = (qp|rs) = (rs|pq), positive
 * semidefinite as a matrix over the pairs (pq)), otherwise as
 * rtcc3_set_hamiltonian.  The integrals enter through their pivoted Cholesky
 * factors (rtcc3_eri_cholesky with tol 1e-12: every integral reproduced to
 * 1e-12), which the T1 transformation of Eq. A4 then dresses as DF factors.
 * RTCC3_ERR_ARG if eri is non-finite, not symmetric or not positive
 * semidefinite. */
int rtcc3_set_hamiltonian_eri(rtcc3_ctx* ctx, const double* eps, const double* eri,
                              const double* dipole);

/* Pivoted (incomplete) Cholesky factorisation of the integral matrix
 * V[(pq)][(rs)] = (pq|rs) on the host, no context or GPU needed: L[k][p][q],
 * k < *rank, with V - sum_k L_k L_k^T positive semidefinite and its largest
 * diagonal element <= tol (so every integral is reproduced to within tol).
 * Each step takes the largest remaining diagonal element as the pivot.
 * Lfac holds max_rank x nmo x nmo doubles (caller-owned).  Returns
 * RTCC3_ERR_ARG for bad sizes, non-finite, asymmetric or indefinite input
 * (a remaining diagonal element below -tol), RTCC3_ERR_NOT_CONVERGED if
 * max_rank factors do not reach tol (*rank = max_rank, the factors so far
 * in Lfac). */
int rtcc3_eri_cholesky(int nmo, const double* eri, double tol, int max_rank, double* Lfac,
                       int* rank);

/* Field of slot b (0 <= b < nbatch): kind RTCC3_FIELD_*, amplitude A (au),
 * omega, center, width (au; the ramp duration t_r for LRCW / QRCW) and a
 * Cartesian direction dir[3]; the perturbation is V = -E(t) dir . mu. */
int rtcc3_set_field(rtcc3_ctx* ctx, int b, int kind, double amplitude, double omega,
                    double center, double width, const double* dir);

/* Amplitudes of slot b (host, interleaved complex; layouts above).  Any of
 * the pointers may be NULL on get. */
int rtcc3_set_amplitudes(rtcc3_ctx* ctx, int b, const double* t1, const double* t2,
                         const double* l1, const double* l2);
int rtcc3_get_amplitudes(const rtcc3_ctx* ctx, int b, double* t1, double* t2, double* l1,
                         double* l2);
/* Simulation time of the context (shared by all slots). */
int rtcc3_set_time(rtcc3_ctx* ctx, double time);
int rtcc3_get_time(const rtcc3_ctx* ctx, double* time);

/* One residual evaluation (one RK4 stage) of slot b at the given time:
 * r_t1, r_t2 = T residuals (Eqs. A10-A11), r_l1, r_l2 = lambda residuals
 * (Eqs. A13-A14), energy[2] (complex), dipole[6] (3 complex components).
 * Any output pointer may be NULL. */
int rtcc3_compute_residuals(rtcc3_ctx* ctx, int b, double time, double* r_t1, double* r_t2,
                            double* r_l1, double* r_l2, double* energy, double* dipole);

/* Zero-field ground state by Jacobi iterations t <- t - R/D, then lambda,
 * until max|R| < tol; copies the result to every slot and sets time 0. */
int rtcc3_solve_ground_state(rtcc3_ctx* ctx, double tol, int maxiter);

/* Convergence record of the last rtcc3_solve_ground_state call (also when
 * it failed): out[k] = max |R| of iteration k, the T iterations first
 * (*t_iterations of them), then the lambda iterations; *count = iterations
 * made (out receives at most max_entries of them). */
int rtcc3_ground_state_history(const rtcc3_ctx* ctx, double* out, int max_entries, int* count,
                               int* t_iterations);

/* Advance every slot nsteps RK4 steps of size h (stage times t, t+h/2,
 * t+h/2, t+h).  dipole: nbatch x (nsteps+1) x 3 complex, energy: nbatch x
 * (nsteps+1) complex (either may be NULL); entry n is evaluated from the
 * state at t0 + n h.  Returns RTCC3_ERR_NONFINITE if the state became
 * non-finite (the state is then left at the failing step). */
int rtcc3_propagate_rk4(rtcc3_ctx* ctx, double h, int nsteps, double* dipole, double* energy);

/* As above with DEVICE output buffers (double2 layout as above), on the CUDA
 * stream `stream` (cudaStream_t, may be NULL for the context stream).  The
 * call returns after the work is enqueued and the stream synchronised. */
int rtcc3_propagate_rk4_dev(rtcc3_ctx* ctx, double h, int nsteps, void* dipole_dev,
                            void* energy_dev, void* stream);

/* Trajectory in chunks: as rtcc3_propagate_rk4 / rtcc3_propagate_rk4_dev
 * but without the evaluation of the final state, so dipole holds nbatch x
 * nsteps x 3 and energy nbatch x nsteps complex entries, entry n from the
 * state at t0 + n h (n < nsteps).  The state the chunk ends in is entry 0 of
 * the next chunk: consecutive chunks give the rtcc3_propagate_rk4 trajectory
 * with every RK4 step evaluated once (Section 2.1: four stage evaluations
 * per step, the observables of the step's start state from its first stage). */
int rtcc3_propagate_rk4_chunk(rtcc3_ctx* ctx, double h, int nsteps, double* dipole,
                              double* energy);
int rtcc3_propagate_rk4_chunk_dev(rtcc3_ctx* ctx, double h, int nsteps, void* dipole_dev,
                                  void* energy_dev, void* stream);

/* Triples map of slot b's Hamiltonian at `time` (device buffers, interleaved
 * complex double): (t1, t2) -> (X1, X2), the triples contributions to the T
 * residuals (Eqs. A21-A22), and its holomorphic vector-Jacobian product
 * g = u^T J for cotangents (u1, u2) (the lambda-side triples terms, Eqs. A23-A24
 * when u = (lambda1, lambda2/2)).  Buffers sized o*v and o*o*v*v. */
int rtcc3_triples_forward_dev(rtcc3_ctx* ctx, int b, double time, const void* t1,
                              const void* t2, void* x1, void* x2, void* stream);
int rtcc3_triples_vjp_dev(rtcc3_ctx* ctx, int b, double time, const void* t1, const void* t2,
                          const void* u1, const void* u2, void* g1, void* g2, void* stream);

/* Allocation-free variant of rtcc3_triples_forward_dev (no counterpart in the
 * paper; it exists for callers that cannot allocate device memory when they
 * call, e.g. code whose allocator is locked between pre-planned stages or
 * which must not trigger cudaMalloc/cudaFree on its hot path).  Same inputs,
 * outputs and results, but every piece of device workspace (intermediate
 * tensors, contraction tables, split-K partial sums, tensor-core operand
 * buffers) is taken from one static device array of 64 MiB compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.  Systems whose workspace would exceed it are rejected with
 * RTCC3_ERR_ARG and a message naming the size.  The call makes no
 * cudaMalloc/cudaFree (it still needs the context created earlier).  The
 * first call on a device looks up the array's device address (make it before
 * any stream capture).  All calls share the array and overwrite it: calls that
 * overlap on the GPU (other threads, other streams) race.  Work runs on
 * `stream` (NULL: the context stream) and the call returns after it is done. */
int rtcc3_triples_forward_noalloc_dev(rtcc3_ctx* ctx, int b, double time, const void* t1,
                                      const void* t2, void* x1, void* x2, void* stream);

/* Autotuner of the (i,j,k) slab size of the triples (Section 2.1 evaluates
 * the triples per (i,j,k) block; the slab groups the blocks of `k` first
 * occupied indices).  For slot b at its current state and time, times one
 * full stage (forward and reverse pass, CUDA events on the context stream,
 * after one untimed evaluation that builds the contraction plans) for every
 * storage form that fits in the device memory free at set-up: the whole
 * o^3 v^3 tensors (reported as -1) when about 24 of them fit in 70 % of it,
 * and slabs of o, o/2, o/4, ..., 1 occupied indices whose four slab buffers
 * fit in a quarter of it.  The fastest becomes the context's triples_chunk
 * option.  Outputs (any may be NULL): *chunk the choice, *ms its time,
 * candidates[] / candidate_ms[] the first max_candidates forms tried and
 * their times, *count how many were tried.  The slot's state is not
 * changed.  RTCC3_ERR_STATE without triples or with field_solver = 1. */
int rtcc3_autotune_triples(rtcc3_ctx* ctx, int b, int* chunk, float* ms, int max_candidates,
                           int* candidates, float* candidate_ms, int* count);

/* Additional one-electron observables, recorded with the same density as
 * the dipole (Section 2.2.3: the magnetic dipole moment is the density
 * contracted with the magnetic dipole matrix elements; in a real orbital
 * basis those are imaginary and antisymmetric): ops holds nops complex
 * nmo x nmo matrices O_k (interleaved, row-major, [k][p][q]), and every
 * compute or propagate call then also records sum_pq D_pq O_k,pq at each
 * entry where it records the dipole.  nops = 0 (ops may be NULL) removes
 * them; 0 <= nops <= 64.  The library copies ops. */
int rtcc3_set_observables(rtcc3_ctx* ctx, int nops, const double* ops);
/* Values recorded by the last compute (1 entry) or propagate call (nbatch x
 * (nsteps + 1) entries, slot-major like the dipole): out[entry][k] complex.
 * `entries` is the capacity of out in entries; RTCC3_ERR_ARG if it is smaller
 * than what the last call recorded, RTCC3_ERR_STATE if nothing was recorded. */
int rtcc3_get_observables(const rtcc3_ctx* ctx, double* out, long long entries);

/* Measured dense arithmetic rates of device `device` in TFLOP/s, the
 * denominators of the roofline fractions the benchmark reports (no
 * counterpart in the paper): tflops[0] TF32 and tflops[1] BF16 tcgen05 MMA
 * issue rate (128 x 256 tiles from shared memory into tensor memory, one CTA
 * per SM), tflops[2] FP32 and tflops[3] FP64 fused multiply-add on the CUDA
 * cores.  Each probe runs once untimed and once timed with CUDA events
 * (about 0.1 s in all).  No context needed. */
int rtcc3_measure_peaks(int device, double* tflops);

/* Change the wait budgets of an existing context (the rtcc3_options fields
 * spin_budget and eig_sweep_cap; 0 restores a default); later calls use them.
 * A wait that runs out of its budget does not hang or poison the context: the
 * kernel drains its own copies and MMAs, frees its tensor memory and returns,
 * the call returns RTCC3_ERR_TIMEOUT (the outputs of that call are
 * undefined), and a later call with a sufficient budget succeeds. */
int rtcc3_set_wait_budgets(rtcc3_ctx* ctx, long long spin_budget, int eig_sweep_cap);

/* Checkpoint: FP64 state of all slots plus time and step counter, as a flat
 * byte image with a version word and checksum.  Query the size with
 * buf == NULL.  Restoring checks size, version and checksum. */
int rtcc3_state_size(const rtcc3_ctx* ctx, long long* bytes);
int rtcc3_get_state(const rtcc3_ctx* ctx, void* buf, long long bytes);
int rtcc3_set_state(rtcc3_ctx* ctx, const void* buf, long long bytes);

/* Diagnostics: number of kernel launches issued by the last propagate or
 * compute call, and bytes of device memory reserved by the context. */
int rtcc3_stats(const rtcc3_ctx* ctx, long long* launches, long long* device_bytes);

/* Per-kernel timing.  While enabled, every launch of the library is
 * bracketed by CUDA events on its stream and CUDA graphs are not used;
 * rtcc3_kernel_stats returns, per kernel name, the launch count, total
 * device milliseconds and the algorithmic flops and bytes of those launches
 * (operands read once, results written once).  Enabling resets the tallies. */
typedef struct rtcc3_kernel_stat {
  char name[48];
  long long launches;
  double ms;
  double flops;
  double bytes;
} rtcc3_kernel_stat;
int rtcc3_set_profiling(rtcc3_ctx* ctx, int enable);
int rtcc3_kernel_stats(rtcc3_ctx* ctx, rtcc3_kernel_stat* out, int max_entries, int* count);

#ifdef __cplusplus
}
#endif

#endif /* RTCC3_H */
