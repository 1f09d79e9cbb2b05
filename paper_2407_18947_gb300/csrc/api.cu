// C ABI of librtcc3 (include/rtcc3.h): context, Hamiltonian, fields, state,
// residual evaluation, ground state, RK4 propagation and checkpoints.
#include "../../include/rtcc3.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <new>
#include <mutex>
#include <string>
#include <vector>

#include "common.h"
#include "engine.h"
#include "model.h"
#include "stage_graph.h"
#include "tc_gemm.h"

using namespace rtcc3;

namespace {

struct Base {
  virtual ~Base() {}
};

// Everything that depends on the compute precision R.
template <typename R>
struct Runner : Base {
  int o, v, n;
  cudaStream_t stream;
  Engine<R> E;
  Hamil<R> H;
  Cx<R>* l1s = nullptr;  // stage lambda values (seeds)
  Cx<R>* l2s = nullptr;
  std::vector<void*> owned;
  Runner(int o_, int v_, cudaStream_t s) : o(o_), v(v_), n(o_ + v_), stream(s), E(s) {
    const size_t n1 = size_t(o) * v;
    l1s = alloc<Cx<R>>(n1);
    l2s = alloc<Cx<R>>(n1 * n1);
  }
  ~Runner() override {
    for (void* p : owned) cudaFree(p);
  }
  // FP64 eigenbases decomposed ahead of their stage: set 0 for the stages
  // inside a Runge-Kutta step, set 1 + b for the first stage of slot b's next
  // step (allocated on first use, before any graph capture)
  std::deque<BasisBuffers> ahead;  // growing keeps references valid
  const BasisBuffers* ahead_buffers(int set) {
    if (int(ahead.size()) <= set) ahead.resize(set + 1);
    BasisBuffers& bb = ahead[set];
    if (!bb.Mo) {
      const size_t oo = size_t(o) * o, vv = size_t(v) * v;
      bb.Mo = alloc<double2>(oo);
      bb.So = alloc<double2>(oo);
      bb.Sio = alloc<double2>(oo);
      bb.wso = alloc<double2>(3 * oo);
      bb.lo = alloc<double2>(o);
      bb.Mv = alloc<double2>(vv);
      bb.Sv = alloc<double2>(vv);
      bb.Siv = alloc<double2>(vv);
      bb.wsv = alloc<double2>(3 * vv);
      bb.lv = alloc<double2>(v);
    }
    return &bb;
  }
  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    RTCC3_CUDA(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
    owned.push_back(p);
    return static_cast<T*>(p);
  }
};

}  // namespace

struct rtcc3_ctx {
  int o = 0, v = 0, n = 0, nb = 0, naux = 0;
  rtcc3_options opt{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool have_ham = false;
  std::unique_ptr<Base> runner;
  // FP64 constants
  double* eps = nullptr;
  double* mu = nullptr;
  std::vector<double> eps_h, mu_h;
  // state: nb slots of [t1, t2, l1, l2] (complex128)
  size_t n1 = 0, n2 = 0, ny = 0;
  double2* y = nullptr;
  double2* acc = nullptr;
  double2* kbuf = nullptr;
  double2* res = nullptr;  // FP64 residual export (ny)
  FieldDev* fdev = nullptr;
  FieldDev* fnone = nullptr;
  std::vector<FieldDev> fhost;
  double* tdev = nullptr;
  double* teval = nullptr;
  int* stepdev = nullptr;
  int* baddev = nullptr;
  double* maxr = nullptr;
  double2* dip_traj = nullptr;
  double2* en_traj = nullptr;
  size_t traj_cap = 0;
  // additional one-electron observables (rtcc3_set_observables)
  int nobs = 0;
  double2* obs_ops = nullptr;     // nobs x n x n
  double2* obs_traj = nullptr;    // entries x nobs
  size_t obs_cap = 0;             // entries
  long long obs_last = 0;         // entries written by the last call
  size_t free_at_setup = 0;  // free device memory when the Hamiltonian was set
  // max |R| per iteration of the last ground-state solve (T, then lambda)
  std::vector<double> gs_history;
  int gs_t_iters = 0;
  double time = 0.0;
  long long step_total = 0;
  long long last_launches = 0;
  Profiler prof;
  TrajDesc* tdesc = nullptr;
  int* checkflag = nullptr;  // raised by the canary check (checked mode)
  // cached CUDA graph of one RK4 step (all slots)
  cudaGraphExec_t gexec = nullptr;
  double gh = 0.0;
  std::vector<int> gsweeps;
  int ggen = -1;
  long long gsteplaunches = 0;
  std::vector<void*> owned;

  template <typename T>
  T* dalloc(size_t count) {
    void* p = nullptr;
    RTCC3_CUDA(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
    owned.push_back(p);
    return static_cast<T*>(p);
  }
  bool fp64() const { return opt.precision == RTCC3_PREC_FP64; }
  template <typename R>
  Runner<R>& run() { return *static_cast<Runner<R>*>(runner.get()); }
  ~rtcc3_ctx() {
    if (gexec) cudaGraphExecDestroy(gexec);
    runner.reset();
    if (dip_traj) cudaFree(dip_traj);
    if (en_traj) cudaFree(en_traj);
    if (obs_ops) cudaFree(obs_ops);
    if (obs_traj) cudaFree(obs_traj);
    for (void* p : owned) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

// Times the launches issued inside its scope when profiling is enabled.
struct PScope {
  Profiler& p;
  cudaStream_t s;
  const char* name;
  double flops, bytes;
  int k;
  PScope(Profiler& p_, cudaStream_t s_, const char* n, double f, double b)
      : p(p_), s(s_), name(n), flops(f), bytes(b), k(p_.begin(s_)) {}
  ~PScope() { p.end(k, s, name, flops, bytes); }
};

int fail(rtcc3_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

template <typename F>
int guarded(rtcc3_ctx* ctx, F&& f) {
  try {
    f();
    if (ctx) ctx->err.clear();
    return RTCC3_OK;
  } catch (const Error& e) {
    return fail(ctx, e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(ctx, RTCC3_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(ctx, RTCC3_ERR_CUDA, e.what());
  }
}

double frob_block(const std::vector<double>& mu, const double* dir, int n, int r0, int r1, int c0,
                  int c1) {
  double s = 0.0;
  const size_t nn = size_t(n) * n;
  for (int p = r0; p < r1; ++p)
    for (int q = c0; q < c1; ++q) {
      const double m = dir[0] * mu[p * n + q] + dir[1] * mu[nn + p * n + q] + dir[2] * mu[2 * nn + p * n + q];
      s += m * m;
    }
  return std::sqrt(s);
}

// Fixed-point sweeps of the field-coupled triples equation needed for a
// relative error below tol: contraction factor rho bounded with Frobenius
// norms of the field blocks (|t1| <= 1 assumed for the dressing terms).
int field_sweeps(const rtcc3_ctx* ctx, int b) {
  const FieldDev& f = ctx->fhost[b];
  if (f.kind == RTCC3_FIELD_NONE || f.amp == 0.0) return 1;
  const int o = ctx->o, n = ctx->n;
  const double A = std::fabs(f.amp);
  const double wvv = A * frob_block(ctx->mu_h, f.dir, n, o, n, o, n);
  const double woo = A * frob_block(ctx->mu_h, f.dir, n, 0, o, 0, o);
  const double wov = A * frob_block(ctx->mu_h, f.dir, n, 0, o, o, n);
  double emax_o = -1e300, emin_v = 1e300;
  for (int p = 0; p < o; ++p) emax_o = std::max(emax_o, ctx->eps_h[p]);
  for (int p = o; p < n; ++p) emin_v = std::min(emin_v, ctx->eps_h[p]);
  const double e3 = 3.0 * (emin_v - emax_o);
  const double rho = 3.0 * (wvv + woo + 2.0 * wov) / e3;
  RTCC3_CHECK(rho < 0.9, RTCC3_ERR_ARG, "field too strong for the triples fixed point (rho >= 0.9)");
  double tol = ctx->opt.field_tol;
  if (tol <= 0.0) tol = ctx->fp64() ? 1e-14 : 1e-8;
  if (rho <= 0.0) return 1;
  const int k = int(std::ceil(std::log(tol) / std::log(rho))) + 1;
  return std::max(1, std::min(k, 200));
}

// Field eigenbasis look-ahead: the next stage's O and V depend only on its t1
// (known once this stage's forward residual r1 is) and its field, so their
// decomposition runs on the side stream during this stage's backward pass
// instead of stalling the next stage.  The next stage's t1 = base + ch (-i r1)
// with base = y inside a step and base = the RK4 accumulator at its last stage.
struct Ahead {
  const BasisBuffers* use = nullptr;   // this stage's basis, decomposed ahead
  const BasisBuffers* make = nullptr;  // decompose the next stage's basis into these
  const double2* base = nullptr;
  double ch = 0.0, dt = 0.0;  // the next stage's input step and time offset
};

// Whether propagation stages use the field-dressed eigenbasis (the condition
// under which record_stage starts one).
bool basis_stages(const rtcc3_ctx* ctx) {
  return ctx->opt.triples != 0 && ctx->opt.field_solver == 0;
}

// M and its decomposition into bb for a stage with t1 = base + ch (-i r1)
// (r1 may be null: t1 = base) and the field of slot `f` at *tdev + dt.
template <typename R>
void launch_basis_ahead(rtcc3_ctx* ctx, const BasisBuffers& bb, const double2* base,
                        const Cx<R>* r1, double ch, const FieldDev* f, double dt) {
  Engine<R>& E = ctx->run<R>().E;
  {
    PScope ps(ctx->prof, ctx->stream, "field_matrices_ahead", 0.0, 0.0);
    launch_next_field_matrices<R>(base, r1, ch, ctx->mu, f, ctx->tdev, dt, ctx->eps, ctx->o,
                                  ctx->v, bb.Mo, bb.Mv, ctx->stream);
  }
  // M is written on the main stream (r1 lives in the stage's arena); the
  // decomposition runs on the side stream, which the consuming stage joins
  E.fork();
  const cudaStream_t ss = E.side_stream();
  const int pk = E.prof_begin(ss);
  const EigJob jo{bb.Mo, ctx->o, bb.So, bb.Sio, bb.lo, bb.wso, E.eig_sweep_cap()};
  const EigJob jv{bb.Mv, ctx->v, bb.Sv, bb.Siv, bb.lv, bb.wsv, E.eig_sweep_cap()};
  launch_eig(jo, jv, sizeof(R) == 4, E.error_flag(), ss);
  E.prof_end(pk, ss, "field_eig_ahead", 0.0, 0.0);
  E.add_launches(2);
}

// Slab size of the blocked triples for this context (0: stored whole).
// Automatic: the stored form keeps about a dozen o^3 v^3 tensors and their
// cotangents alive in a stage; when 24 of them do not fit in 70% of the
// device memory free at set-up, the triples are blocked in slabs of k first
// occupied indices with the four slab buffers within a quarter of that
// memory (at most 32 GB).
int triples_chunk(const rtcc3_ctx* ctx) {
  if (!ctx->opt.triples || ctx->opt.field_solver != 0) return 0;
  const int o = ctx->o, v = ctx->v;
  if (ctx->opt.triples_chunk > 0) return std::min(ctx->opt.triples_chunk, o);
  if (ctx->opt.triples_chunk < 0) return 0;
  const double elem = ctx->fp64() ? 16.0 : 8.0;
  const double t3 = double(o) * o * o * v * v * v * elem;
  const double freeb = double(ctx->free_at_setup);
  if (24.0 * t3 <= 0.7 * freeb) return 0;
  const double budget = std::min(0.25 * freeb, 32.0 * (1ull << 30));
  const double slab = 4.0 * double(o) * o * v * v * v * elem;
  return std::max(1, std::min(o, int(budget / slab)));
}

// One stage evaluation for slot b: records the graph with inputs
// y_b + ch * kprev at time *tsrc + dt and, if need_grad, runs the backward
// pass with the Lagrangian seeds.
template <typename R>
StageNodes eval_stage(rtcc3_ctx* ctx, int b, const double2* ybase, const double2* kprev, double ch,
                      const double* tsrc, double dt, bool need_grad, const FieldDev* f,
                      bool field_terms, int sweeps, bool ccsd_terms = true,
                      const Ahead& ahead = Ahead{}) {
  Runner<R>& Rn = ctx->run<R>();
  Engine<R>& E = Rn.E;
  E.begin();
  StageOptions so;
  so.triples = ctx->opt.triples != 0;
  so.need_grad = need_grad;
  so.field_terms = field_terms;
  so.field_iters = sweeps;
  so.rotation = ctx->opt.field_solver == 0;
  so.triples_chunk = triples_chunk(ctx);
  so.tc_scope = ctx->opt.tc_scope;
  const bool basis_stage = so.triples && so.field_terms && so.rotation;
  if (basis_stage) so.basis = ahead.use;
  (void)ccsd_terms;
  StageNodes S = record_stage<R>(E, Rn.H, so, [&](const StageNodes& s) {
    PScope ps(ctx->prof, ctx->stream, "stage_inputs", 0.0,
              double(ctx->ny) * (kprev ? 32.0 : 16.0) + double(ctx->ny) * sizeof(Cx<R>));
    launch_stage_inputs<R>(ybase, kprev, ch, E.data(s.t1), E.data(s.t2), Rn.l1s, Rn.l2s,
                           E.data(s.w), ctx->mu, f, tsrc, dt, ctx->o, ctx->v, ctx->n, ctx->stream);
    E.add_launches(1);
  });
  if (ahead.make && basis_stage)
    launch_basis_ahead<R>(ctx, *ahead.make, ahead.base, E.data(S.r1), ahead.ch, f, ahead.dt);
  if (need_grad) {
    E.prepare_backward();
    {
      PScope ps(ctx->prof, ctx->stream, "seeds", 0.0, double(ctx->ny) * sizeof(Cx<R>));
      launch_seeds<R>(E.grad(S.e), E.grad(S.r1), E.grad(S.r2), Rn.l1s, Rn.l2s, ctx->o, ctx->v,
                      ctx->stream);
      E.add_launches(1);
      E.mark_grad_written(S.e);
      E.mark_grad_written(S.r1);
      E.mark_grad_written(S.r2);
    }
    E.backward();
    E.ensure_grad(S.t1);  // read outside the engine
    E.ensure_grad(S.t2);
    E.ensure_grad(S.w);
  }
  if (E.checked()) {
    // checked mode: no tensor of the stage was written past its end
    E.verify_canaries(ctx->checkflag);
    int bad = 0;
    RTCC3_CUDA(cudaMemcpy(&bad, ctx->checkflag, sizeof(int), cudaMemcpyDeviceToHost));
    if (bad) {
      RTCC3_CUDA(cudaMemset(ctx->checkflag, 0, sizeof(int)));
      throw Error(RTCC3_ERR_STATE, "checked mode: a device tensor was written past its end");
    }
  }
  return S;
}

template <typename R>
void setup_runner(rtcc3_ctx* ctx, const double* Lfac) {
  auto rn = std::make_unique<Runner<R>>(ctx->o, ctx->v, ctx->stream);
  const int n = ctx->n, na = ctx->naux;
  Hamil<R>& H = rn->H;
  H.o = ctx->o; H.v = ctx->v; H.n = n; H.naux = na;
  H.eps = ctx->eps;
  H.mu = ctx->mu;
  // h = diag(eps) - (2J - K) with J, K from the DF factors (FP64 on host:
  // set-up only, O(naux n^2 o))
  std::vector<double> h(size_t(n) * n, 0.0);
  for (int p = 0; p < n; ++p) h[p * n + p] = ctx->eps_h[p];
  const int o = ctx->o;
  std::vector<double> dk(na, 0.0);
  for (int P = 0; P < na; ++P)
    for (int k = 0; k < o; ++k) dk[P] += Lfac[(size_t(P) * n + k) * n + k];
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double J = 0.0, K = 0.0;
      for (int P = 0; P < na; ++P) {
        const double* LP = Lfac + size_t(P) * n * n;
        J += LP[p * n + q] * dk[P];
        for (int k = 0; k < o; ++k) K += LP[p * n + k] * LP[k * n + q];
      }
      h[p * n + q] -= 2.0 * J - K;
    }
  std::vector<Cx<R>> hc(size_t(n) * n), Lc(size_t(na) * n * n), ones(n);
  for (size_t t = 0; t < hc.size(); ++t) hc[t] = cmake<R>(R(h[t]), R(0));
  for (size_t t = 0; t < Lc.size(); ++t) Lc[t] = cmake<R>(R(Lfac[t]), R(0));
  for (int t = 0; t < n; ++t) ones[t] = cmake<R>(R(1), R(0));
  {
    // FP64 sums of three occupied / three virtual orbital energies (Eq. A16),
    // each energy taken relative to the mid-gap energy (see Hamil::eshift)
    const int v = ctx->v;
    double emax_o = -1e300, emin_v = 1e300;
    for (int p = 0; p < o; ++p) emax_o = std::max(emax_o, ctx->eps_h[p]);
    for (int p = o; p < n; ++p) emin_v = std::min(emin_v, ctx->eps_h[p]);
    const double shift = 0.5 * (emax_o + emin_v);
    H.eshift = shift;
    std::vector<double> os(size_t(o) * o * o), vs(size_t(v) * v * v);
    for (int i = 0; i < o; ++i)
      for (int j = 0; j < o; ++j)
        for (int k = 0; k < o; ++k)
          os[(size_t(i) * o + j) * o + k] =
              (ctx->eps_h[i] - shift) + (ctx->eps_h[j] - shift) + (ctx->eps_h[k] - shift);
    for (int a = 0; a < v; ++a)
      for (int b = 0; b < v; ++b)
        for (int c = 0; c < v; ++c)
          vs[(size_t(a) * v + b) * v + c] =
              (ctx->eps_h[o + a] - shift) + (ctx->eps_h[o + b] - shift) +
              (ctx->eps_h[o + c] - shift);
    H.osum = rn->template alloc<double>(os.size());
    H.vsum = rn->template alloc<double>(vs.size());
    RTCC3_CUDA(cudaMemcpy(H.osum, os.data(), os.size() * sizeof(double), cudaMemcpyHostToDevice));
    RTCC3_CUDA(cudaMemcpy(H.vsum, vs.data(), vs.size() * sizeof(double), cudaMemcpyHostToDevice));
    // the sums rounded once to the compute precision (the dense triples
    // kernels divide in R; after the mid-gap shift every occupied sum is
    // negative and every virtual sum positive, so D = vsum - osum adds two
    // terms of one sign whatever the absolute orbital energies)
    std::vector<R> osr(os.begin(), os.end()), vsr(vs.begin(), vs.end());
    H.osum_r = rn->template alloc<R>(osr.size());
    H.vsum_r = rn->template alloc<R>(vsr.size());
    RTCC3_CUDA(cudaMemcpy(H.osum_r, osr.data(), osr.size() * sizeof(R), cudaMemcpyHostToDevice));
    RTCC3_CUDA(cudaMemcpy(H.vsum_r, vsr.data(), vsr.size() * sizeof(R), cudaMemcpyHostToDevice));
    // occupied blocks in orbit order: for each i <= j <= k its distinct
    // permutations, one after the other
    std::vector<int> order;
    order.reserve(size_t(o) * o * o);
    for (int i = 0; i < o; ++i)
      for (int j = i; j < o; ++j)
        for (int k = j; k < o; ++k) {
          const int p[6][3] = {{i, j, k}, {j, i, k}, {i, k, j}, {k, j, i}, {k, i, j}, {j, k, i}};
          const size_t first = order.size();
          for (auto& q : p) {
            const int id = (q[0] * o + q[1]) * o + q[2];
            if (std::find(order.begin() + first, order.end(), id) == order.end()) order.push_back(id);
          }
        }
    RTCC3_CHECK(order.size() == size_t(o) * o * o, kErrState, "orbit order incomplete");
    H.orbit_order = rn->template alloc<int>(order.size());
    RTCC3_CUDA(cudaMemcpy(H.orbit_order, order.data(), order.size() * sizeof(int),
                          cudaMemcpyHostToDevice));
  }
  H.h = rn->template alloc<Cx<R>>(hc.size());
  H.L = rn->template alloc<Cx<R>>(Lc.size());
  H.ones = rn->template alloc<Cx<R>>(n);
  RTCC3_CUDA(cudaMemcpy(H.h, hc.data(), hc.size() * sizeof(Cx<R>), cudaMemcpyHostToDevice));
  RTCC3_CUDA(cudaMemcpy(H.L, Lc.data(), Lc.size() * sizeof(Cx<R>), cudaMemcpyHostToDevice));
  RTCC3_CUDA(cudaMemcpy(H.ones, ones.data(), ones.size() * sizeof(Cx<R>), cudaMemcpyHostToDevice));
  rn->E.set_profiler(&ctx->prof);
  rn->E.set_wait_budget(ctx->opt.spin_budget);
  rn->E.set_checked(ctx->opt.checked != 0);
  rn->E.set_branches(ctx->opt.serial == 0);
  rn->E.set_eig_sweep_cap(ctx->opt.eig_sweep_cap);
  if (ctx->opt.precision == RTCC3_PREC_TF32) rn->E.set_tensor_cores(4);
  if (ctx->opt.precision == RTCC3_PREC_BF16) rn->E.set_tensor_cores(2);
  ctx->runner = std::move(rn);
}

// Room for `entries` values of every additional observable.
void ensure_obs(rtcc3_ctx* ctx, size_t entries) {
  if (ctx->nobs == 0 || entries <= ctx->obs_cap) return;
  if (ctx->obs_traj) cudaFree(ctx->obs_traj);
  ctx->obs_traj = nullptr;
  ctx->obs_cap = 0;
  RTCC3_CUDA(cudaMalloc(&ctx->obs_traj, entries * ctx->nobs * sizeof(double2)));
  ctx->obs_cap = entries;
}

// Trajectory descriptor with the context's additional observables.
TrajDesc traj_desc(const rtcc3_ctx* ctx, double2* dip, double2* en, long long stride) {
  TrajDesc td{dip, en, stride};
  if (ctx->nobs > 0) {
    td.obs = ctx->obs_traj;
    td.ops = ctx->obs_ops;
    td.nobs = ctx->nobs;
  }
  return td;
}

void ensure_traj(rtcc3_ctx* ctx, size_t entries) {
  if (entries <= ctx->traj_cap) return;
  if (ctx->dip_traj) cudaFree(ctx->dip_traj);
  if (ctx->en_traj) cudaFree(ctx->en_traj);
  ctx->dip_traj = nullptr;
  ctx->en_traj = nullptr;
  RTCC3_CUDA(cudaMalloc(&ctx->dip_traj, entries * 3 * sizeof(double2)));
  RTCC3_CUDA(cudaMalloc(&ctx->en_traj, entries * sizeof(double2)));
  ctx->traj_cap = entries;
}

// One RK4 step for every slot; observables of the step-start state go to
// trajectory entry *stepdev of slot b (arrays strided by `stride`).
template <typename R>
void rk4_step(rtcc3_ctx* ctx, double h, const std::vector<int>& sweeps) {
  Runner<R>& Rn = ctx->run<R>();
  Engine<R>& E = Rn.E;
  const double cs[4] = {0.0, 0.5, 0.5, 1.0};
  const double ws[4] = {1.0, 2.0, 2.0, 1.0};
  for (int b = 0; b < ctx->nb; ++b) {
    double2* yb = ctx->y + size_t(b) * ctx->ny;
    const double ybytes = double(ctx->ny) * 16.0;
    {
      PScope ps(ctx->prof, ctx->stream, "rk4_update", 0.0, 2.0 * ybytes);
      launch_stage_prep_acc(ctx->acc, yb, ctx->ny, ctx->stream);
      E.add_launches(1);
    }
    for (int s = 0; s < 4; ++s) {
      Ahead ah;
      if (basis_stages(ctx)) {
        // stage 0 was decomposed by the previous step (or by prime_basis_ahead)
        ah.use = Rn.ahead_buffers(s == 0 ? 1 + b : 0);
        ah.make = Rn.ahead_buffers(s == 3 ? 1 + b : 0);
        ah.base = s == 3 ? ctx->acc : yb;
        ah.ch = s == 3 ? h * ws[3] / 6.0 : cs[s + 1] * h;
        ah.dt = s == 3 ? h : cs[s + 1] * h;
      }
      StageNodes S = eval_stage<R>(ctx, b, yb, s == 0 ? nullptr : ctx->kbuf, cs[s] * h, ctx->tdev,
                                   cs[s] * h, true, ctx->fdev + b, true, sweeps[b], true, ah);
      if (s == 0) {
        PScope ps(ctx->prof, ctx->stream, "observables", 8.0 * ctx->n * ctx->n,
                  double(ctx->n) * ctx->n * (sizeof(Cx<R>) + 24.0));
        launch_observables<R>(E.grad(S.w), E.data(S.e), yb, ctx->mu, ctx->fdev + b, ctx->tdev,
                              0.0, ctx->o, ctx->v, ctx->nobs, ctx->tdesc, b, ctx->stepdev,
                              ctx->stream);
        E.add_launches(1);
      }
      PScope ps(ctx->prof, ctx->stream, "rk4_update", 4.0 * ctx->ny,
                double(ctx->ny) * sizeof(Cx<R>) + (s < 3 ? 3.0 : 2.0) * ybytes);
      launch_stage_output<R>(E.data(S.r1), E.data(S.r2), E.grad(S.t1), E.grad(S.t2),
                             s < 3 ? ctx->kbuf : nullptr, ctx->acc, h * ws[s] / 6.0, ctx->mu,
                             ctx->fdev + b, ctx->tdev, cs[s] * h, ctx->o, ctx->v, ctx->stream);
      E.add_launches(1);
    }
    PScope ps(ctx->prof, ctx->stream, "rk4_update", 0.0, 2.0 * ybytes);
    launch_step_finish(yb, ctx->acc, ctx->ny, ctx->stepdev, ctx->baddev,
                       ctx->opt.storage == RTCC3_STORAGE_C64, ctx->stream);
    E.add_launches(1);
  }
  launch_step_advance(ctx->tdev, h, ctx->stepdev, ctx->stream);
  E.add_launches(1);
  // the next step's first-stage bases were decomposed during the last stages'
  // backward passes; a captured step must not leave side-stream work unjoined
  E.join();
}

// Decompose the first-stage basis of every slot's next step from its current
// state (the state or the field may have changed since the last step).
template <typename R>
void prime_basis_ahead(rtcc3_ctx* ctx) {
  if (!basis_stages(ctx)) return;
  Runner<R>& Rn = ctx->run<R>();
  for (int b = 0; b < ctx->nb; ++b)
    launch_basis_ahead<R>(ctx, *Rn.ahead_buffers(1 + b), ctx->y + size_t(b) * ctx->ny, nullptr,
                          0.0, ctx->fdev + b, 0.0);
  // a captured step graph orders itself after the main stream only
  Rn.E.join();
}

template <typename R>
void final_observables(rtcc3_ctx* ctx, const std::vector<int>& sweeps) {
  Runner<R>& Rn = ctx->run<R>();
  Engine<R>& E = Rn.E;
  for (int b = 0; b < ctx->nb; ++b) {
    double2* yb = ctx->y + size_t(b) * ctx->ny;
    StageNodes S = eval_stage<R>(ctx, b, yb, nullptr, 0.0, ctx->tdev, 0.0, true, ctx->fdev + b,
                                 true, sweeps[b]);
    PScope ps(ctx->prof, ctx->stream, "observables", 8.0 * ctx->n * ctx->n,
              double(ctx->n) * ctx->n * (sizeof(Cx<R>) + 24.0));
    launch_observables<R>(E.grad(S.w), E.data(S.e), yb, ctx->mu, ctx->fdev + b, ctx->tdev, 0.0,
                          ctx->o, ctx->v, ctx->nobs, ctx->tdesc, b, ctx->stepdev, ctx->stream);
  }
}

// A bounded device wait that gave up leaves a flag; report it and clear it.
template <typename R>
void check_device_timeout(rtcc3_ctx* ctx) {
  Engine<R>& E = ctx->run<R>().E;
  int flag = 0;
  RTCC3_CUDA(cudaMemcpy(&flag, E.error_flag(), sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    RTCC3_CUDA(cudaMemset(E.error_flag(), 0, sizeof(int)));
    if (flag & kEigStatusBase) {
      const int reason = (flag >> 20) & 0xf, n = (flag >> 10) & 0x3ff, row = flag & 0x3ff;
      throw Error(reason == kEigNonFinite ? RTCC3_ERR_NONFINITE : RTCC3_ERR_TIMEOUT,
                  std::string("field eigensolver (order ") + std::to_string(n) + "): " +
                      (reason == kEigNonFinite ? "non-finite dressed field matrix"
                                               : "QR sweeps did not converge at row " +
                                                     std::to_string(row)));
    }
    throw Error(RTCC3_ERR_TIMEOUT, "a tensor-core pipeline wait gave up");
  }
}

void drop_graph(rtcc3_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
  ctx->gsweeps.clear();
}

template <typename R>
void propagate_impl(rtcc3_ctx* ctx, double h, int nsteps, double2* dip, double2* en, size_t stride,
                    bool final) {
  Engine<R>& E = ctx->run<R>().E;
  std::vector<int> sweeps(ctx->nb);
  for (int b = 0; b < ctx->nb; ++b) sweeps[b] = field_sweeps(ctx, b);
  ensure_obs(ctx, stride * ctx->nb);
  ctx->obs_last = (long long)(stride * ctx->nb);
  const TrajDesc td = traj_desc(ctx, dip, en, (long long)stride);
  RTCC3_CUDA(cudaMemcpyAsync(ctx->tdesc, &td, sizeof(td), cudaMemcpyHostToDevice, ctx->stream));
  RTCC3_CUDA(cudaMemsetAsync(ctx->stepdev, 0, sizeof(int), ctx->stream));
  const int minus1 = -1;
  RTCC3_CUDA(cudaMemcpyAsync(ctx->baddev, &minus1, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  // stage-local buffers must not be overwritten before the copies above land
  RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
  E.reset_launch_count();
  const bool graphs = ctx->opt.use_graphs && !ctx->prof.enabled && !ctx->opt.checked;
  // the captured step depends on h, the sweep counts and the engine's
  // persistent buffers; anything else is read from device memory
  if (ctx->gexec && (!graphs || ctx->gh != h || ctx->gsweeps != sweeps || ctx->ggen != E.generation()))
    drop_graph(ctx);
  int done = 0;
  long long launches = 0;
  if (nsteps > 0) {
    prime_basis_ahead<R>(ctx);
    launches += E.launches();
    E.reset_launch_count();
  }
  if (graphs && !ctx->gexec && nsteps > 0) {
    rk4_step<R>(ctx, h, sweeps);  // eager first step: builds plans, arena and scratch
    done = 1;
    launches += E.launches();
    cudaGraph_t graph = nullptr;
    E.freeze_plans(true);
    const int before = E.launches();
    try {
      RTCC3_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      try {
        rk4_step<R>(ctx, h, sweeps);
      } catch (...) {
        cudaStreamEndCapture(ctx->stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        throw;
      }
      RTCC3_CUDA(cudaStreamEndCapture(ctx->stream, &graph));
      cudaGraphExec_t exec = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      RTCC3_CUDA(ie);
      ctx->gexec = exec;
    } catch (...) {
      E.freeze_plans(false);
      throw;
    }
    E.freeze_plans(false);
    ctx->gsteplaunches = E.launches() - before;
    ctx->gh = h;
    ctx->gsweeps = sweeps;
    ctx->ggen = E.generation();
  }
  if (graphs && ctx->gexec) {
    for (; done < nsteps; ++done) {
      RTCC3_CUDA(cudaGraphLaunch(ctx->gexec, ctx->stream));
      launches += ctx->gsteplaunches;
    }
  } else {
    E.reset_launch_count();
    for (; done < nsteps; ++done) rk4_step<R>(ctx, h, sweeps);
    launches += E.launches();
  }
  E.reset_launch_count();
  if (final) final_observables<R>(ctx, sweeps);
  ctx->last_launches = launches + E.launches();
  RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->time += h * nsteps;
  ctx->step_total += nsteps;
  check_device_timeout<R>(ctx);
  int bad = -1;
  RTCC3_CUDA(cudaMemcpy(&bad, ctx->baddev, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad >= 0)
    throw Error(RTCC3_ERR_NONFINITE, "non-finite amplitudes after RK4 step " + std::to_string(bad));
}

void check_slot(const rtcc3_ctx* ctx, int b) {
  RTCC3_CHECK(b >= 0 && b < ctx->nb, RTCC3_ERR_ARG, "slot index out of range");
}

void require_ham(const rtcc3_ctx* ctx) {
  RTCC3_CHECK(ctx->have_ham, RTCC3_ERR_STATE, "rtcc3_set_hamiltonian has not been called");
}

template <typename R>
void residuals_impl(rtcc3_ctx* ctx, int b, double time, double* r_t1, double* r_t2, double* r_l1,
                    double* r_l2, double* energy, double* dipole) {
  Engine<R>& E = ctx->run<R>().E;
  RTCC3_CUDA(cudaMemcpyAsync(ctx->teval, &time, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  const bool need_grad = r_l1 || r_l2 || dipole;
  E.reset_launch_count();
  StageNodes S = eval_stage<R>(ctx, b, ctx->y + size_t(b) * ctx->ny, nullptr, 0.0, ctx->teval, 0.0,
                               need_grad, ctx->fdev + b, need_grad || ctx->fhost[b].kind != 0,
                               field_sweeps(ctx, b));
  launch_residual_export<R>(E.data(S.r1), E.data(S.r2), need_grad ? E.grad(S.t1) : nullptr,
                            need_grad ? E.grad(S.t2) : nullptr, ctx->mu, ctx->fdev + b, ctx->teval,
                            ctx->res, ctx->o, ctx->v, need_grad, ctx->stream);
  ensure_traj(ctx, 1);
  ensure_obs(ctx, 1);
  ctx->obs_last = 1;
  const TrajDesc td = traj_desc(ctx, ctx->dip_traj, ctx->en_traj, 0);
  RTCC3_CUDA(cudaMemcpyAsync(ctx->tdesc, &td, sizeof(td), cudaMemcpyHostToDevice, ctx->stream));
  launch_observables<R>(need_grad ? E.grad(S.w) : E.data(S.w), E.data(S.e),
                        ctx->y + size_t(b) * ctx->ny, ctx->mu, ctx->fdev + b, ctx->teval, 0.0,
                        ctx->o, ctx->v, ctx->nobs, ctx->tdesc, 0, nullptr, ctx->stream);
  RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->last_launches = E.launches();
  check_device_timeout<R>(ctx);
  const size_t n1 = ctx->n1, n2 = ctx->n2;
  auto get = [&](double* dst, size_t off, size_t cnt) {
    if (dst)
      RTCC3_CUDA(cudaMemcpy(dst, ctx->res + off, cnt * sizeof(double2), cudaMemcpyDeviceToHost));
  };
  get(r_t1, 0, n1);
  get(r_t2, n1, n2);
  get(r_l1, n1 + n2, n1);
  get(r_l2, 2 * n1 + n2, n2);
  if (energy) RTCC3_CUDA(cudaMemcpy(energy, ctx->en_traj, sizeof(double2), cudaMemcpyDeviceToHost));
  if (dipole) RTCC3_CUDA(cudaMemcpy(dipole, ctx->dip_traj, 3 * sizeof(double2), cudaMemcpyDeviceToHost));
}

// Solve the (m+1)x(m+1) complex DIIS system by Gaussian elimination with
// partial pivoting (host; m <= 8).
std::vector<double2> diis_coefficients(const std::vector<double2>& Bm, int m) {
  const int N = m + 1;
  std::vector<double> ar(size_t(N) * N), ai(size_t(N) * N), br(N, 0.0), bi(N, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) { ar[i * N + j] = Bm[i * m + j].x; ai[i * N + j] = Bm[i * m + j].y; }
  for (int i = 0; i < m; ++i) { ar[i * N + m] = -1.0; ar[m * N + i] = -1.0; }
  br[m] = -1.0;
  for (int c = 0; c < N; ++c) {
    int piv = c;
    double best = -1.0;
    for (int r = c; r < N; ++r) {
      const double mag = std::hypot(ar[r * N + c], ai[r * N + c]);
      if (mag > best) { best = mag; piv = r; }
    }
    RTCC3_CHECK(best > 0.0, RTCC3_ERR_NOT_CONVERGED, "singular DIIS matrix");
    if (piv != c) {
      for (int k = 0; k < N; ++k) { std::swap(ar[c * N + k], ar[piv * N + k]); std::swap(ai[c * N + k], ai[piv * N + k]); }
      std::swap(br[c], br[piv]); std::swap(bi[c], bi[piv]);
    }
    const double pr = ar[c * N + c], pi = ai[c * N + c], pd = pr * pr + pi * pi;
    for (int r = c + 1; r < N; ++r) {
      const double xr = ar[r * N + c], xi = ai[r * N + c];
      const double fr = (xr * pr + xi * pi) / pd, fi = (xi * pr - xr * pi) / pd;
      for (int k = c; k < N; ++k) {
        const double yr = ar[c * N + k], yi = ai[c * N + k];
        ar[r * N + k] -= fr * yr - fi * yi;
        ai[r * N + k] -= fr * yi + fi * yr;
      }
      br[r] -= fr * br[c] - fi * bi[c];
      bi[r] -= fr * bi[c] + fi * br[c];
    }
  }
  std::vector<double> xr(N), xi(N);
  for (int r = N - 1; r >= 0; --r) {
    double sr = br[r], si = bi[r];
    for (int k = r + 1; k < N; ++k) {
      sr -= ar[r * N + k] * xr[k] - ai[r * N + k] * xi[k];
      si -= ar[r * N + k] * xi[k] + ai[r * N + k] * xr[k];
    }
    const double pr = ar[r * N + r], pi = ai[r * N + r], pd = pr * pr + pi * pi;
    xr[r] = (sr * pr + si * pi) / pd;
    xi[r] = (si * pr - sr * pi) / pd;
  }
  std::vector<double2> c(m);
  for (int k = 0; k < m; ++k) c[k] = make_double2(xr[k], xi[k]);
  return c;
}

template <typename R>
void ground_state_impl(rtcc3_ctx* ctx, double tol, int maxiter) {
  Engine<R>& E = ctx->run<R>().E;
  double2* y0 = ctx->y;
  RTCC3_CUDA(cudaMemsetAsync(y0, 0, ctx->ny * sizeof(double2), ctx->stream));
  const double zero = 0.0;
  RTCC3_CUDA(cudaMemcpyAsync(ctx->teval, &zero, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  const size_t n1 = ctx->n1, n2 = ctx->n2, len = n1 + n2;
  const int kDiis = 8;
  double2* X = ctx->dalloc<double2>(len * kDiis);
  double2* Ev = ctx->dalloc<double2>(len * kDiis);
  double2* dots = ctx->dalloc<double2>(kDiis);
  double2* coef = ctx->dalloc<double2>(kDiis);
  ctx->gs_history.clear();
  ctx->gs_t_iters = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const bool lam = pass == 1;
    const size_t off = lam ? len : 0;
    bool conv = false;
    int m = 0, head = 0;  // ring buffer of DIIS vectors
    std::vector<double2> B(kDiis * kDiis, make_double2(0.0, 0.0));
    for (int it = 0; it < maxiter; ++it) {
      StageNodes S = eval_stage<R>(ctx, 0, y0, nullptr, 0.0, ctx->teval, 0.0, lam, ctx->fnone, false, 1);
      launch_residual_export<R>(E.data(S.r1), E.data(S.r2), lam ? E.grad(S.t1) : nullptr,
                                lam ? E.grad(S.t2) : nullptr, ctx->mu, ctx->fnone, ctx->teval,
                                ctx->res, ctx->o, ctx->v, lam, ctx->stream);
      RTCC3_CUDA(cudaMemsetAsync(ctx->maxr, 0, sizeof(double), ctx->stream));
      const int slot = head;
      launch_diis_step(y0 + off, ctx->res + off, ctx->eps, ctx->o, ctx->v, X + slot * len,
                       Ev + slot * len, ctx->maxr, ctx->stream);
      const int mm = std::min(m + 1, kDiis);
      launch_dots(Ev, Ev + slot * len, mm, len, dots, ctx->stream);
      double mx = 0.0;
      std::vector<double2> d(mm);
      RTCC3_CUDA(cudaMemcpyAsync(&mx, ctx->maxr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      RTCC3_CUDA(cudaMemcpyAsync(d.data(), dots, mm * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
      RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
      ctx->gs_history.push_back(mx);
      if (!lam) ctx->gs_t_iters = int(ctx->gs_history.size());
      if (!std::isfinite(mx)) {
        check_device_timeout<R>(ctx);  // a device-side cause is reported (and its flag cleared) first
        throw Error(RTCC3_ERR_NONFINITE, "non-finite residual in the ground-state solve");
      }
      if (mx < tol) { conv = true; break; }
      m = mm;
      head = (head + 1) % kDiis;
      // B[k][slot] = <E_k|E_slot>, B[slot][k] = conj
      for (int k = 0; k < m; ++k) {
        B[k * kDiis + slot] = d[k];
        B[slot * kDiis + k] = make_double2(d[k].x, -d[k].y);
      }
      std::vector<double2> Bm(size_t(m) * m);
      for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Bm[i * m + j] = B[i * kDiis + j];
      std::vector<double2> c = m >= 2 ? diis_coefficients(Bm, m) : std::vector<double2>();
      if (m < 2) {
        c.assign(m, make_double2(0.0, 0.0));
        c[slot] = make_double2(1.0, 0.0);
      }
      RTCC3_CUDA(cudaMemcpyAsync(coef, c.data(), m * sizeof(double2), cudaMemcpyHostToDevice, ctx->stream));
      launch_lincomb(X, coef, m, len, y0 + off, ctx->stream);
    }
    if (!conv)
      throw Error(RTCC3_ERR_NOT_CONVERGED,
                  std::string(lam ? "lambda" : "T") + " equations did not converge");
  }
  for (int b = 1; b < ctx->nb; ++b)
    RTCC3_CUDA(cudaMemcpyAsync(ctx->y + size_t(b) * ctx->ny, y0, ctx->ny * sizeof(double2),
                               cudaMemcpyDeviceToDevice, ctx->stream));
  RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->time = 0.0;
  ctx->step_total = 0;
  RTCC3_CUDA(cudaMemcpy(ctx->tdev, &ctx->time, sizeof(double), cudaMemcpyHostToDevice));
}

// Triples-only map (t1, t2) -> (X1, X2) and its vector-Jacobian product.
template <typename R>
void triples_impl(rtcc3_ctx* ctx, int b, double time, const double2* t1, const double2* t2,
                  const double2* u1, const double2* u2, double2* x1, double2* x2, double2* g1,
                  double2* g2, cudaStream_t st) {
  Runner<R>& Rn = ctx->run<R>();
  Engine<R>& E = Rn.E;
  const bool vjp = (g1 || g2);
  RTCC3_CUDA(cudaMemcpyAsync(ctx->teval, &time, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  E.begin();
  StageOptions so;
  so.ccsd = false;  // R1, R2 = X1, X2 only
  so.triples = true;
  so.need_grad = vjp;
  so.field_terms = true;
  so.field_iters = field_sweeps(ctx, b);
  so.rotation = ctx->opt.field_solver == 0;
  so.triples_chunk = triples_chunk(ctx);
  so.tc_scope = ctx->opt.tc_scope;
  auto fill = [&](const StageNodes& s) {
    launch_load_amplitudes<R>(t1, t2, E.data(s.t1), E.data(s.t2), ctx->o, ctx->v, ctx->stream);
    launch_field_operator<R>(E.data(s.w), ctx->mu, ctx->fdev + b, ctx->teval, 0.0, ctx->n, ctx->stream);
  };
  (void)st;
  const size_t n1 = ctx->n1, n2 = ctx->n2;
  StageNodes S = record_stage<R>(E, Rn.H, so, fill);
  if (vjp) {
    E.prepare_backward();  // grad(e) stays zero: only u . X is differentiated
    launch_load_amplitudes<R>(u1, u2, E.grad(S.r1), E.grad(S.r2), ctx->o, ctx->v, ctx->stream);
    E.mark_grad_written(S.r1);
    E.mark_grad_written(S.r2);
    E.backward();
    E.ensure_grad(S.t1);  // read outside the engine
    E.ensure_grad(S.t2);
    launch_export<R>(E.grad(S.t1), g1, n1, ctx->stream);
    launch_export<R>(E.grad(S.t2), g2, n2, ctx->stream);
  } else {
    launch_export<R>(E.data(S.r1), x1, n1, ctx->stream);
    launch_export<R>(E.data(S.r2), x2, n2, ctx->stream);
  }
  RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
}

// ---- allocation-free triples map ------------------------------------------
// For callers that cannot allocate device memory at the point of the call
// (for example code running between pre-allocated pipeline stages, or
// embedders whose allocator forbids cudaMalloc on their hot path), the
// triples map also runs out of a fixed device region compiled into this
// library: kNoAllocBytes per device, held by every GPU that loads the
// library until the process exits.  All calls share the region.
constexpr size_t kNoAllocBytes = size_t(64) << 20;
}  // namespace

static __device__ __align__(256) unsigned char g_rtcc3_noalloc_scratch[kNoAllocBytes];

namespace {

// Device address of the static region for `dev` (which must be the current
// device), looked up once per device.  The first call on a device performs this
// lookup, so it should come before any stream capture.
char* noalloc_scratch_address(int dev) {
  static std::mutex mu;
  static std::vector<char*> addr;
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= int(addr.size())) addr.resize(dev + 1, nullptr);
  if (!addr[dev]) {
    void* p = nullptr;
    RTCC3_CUDA(cudaGetSymbolAddress(&p, g_rtcc3_noalloc_scratch));
    addr[dev] = static_cast<char*>(p);
  }
  return addr[dev];
}

// Conservative workspace of one triples-map evaluation: dressed integrals,
// the o^3 v^3 triples intermediates, small tensors, plus room for
// contraction tables and split-K partial sums.
template <typename R>
size_t noalloc_estimate(const rtcc3_ctx* ctx) {
  const size_t o = ctx->o, v = ctx->v, n = ctx->n, na = ctx->naux;
  const size_t elems = 2 * na * n * n + 12 * n * n + n * n * n * n + 12 * o * o * v * v +
                       10 * o * o * o * v * v * v + 2 * o * o * o * v;
  return elems * sizeof(Cx<R>) + (size_t(16) << 20);
}

template <typename R>
void triples_noalloc_impl(rtcc3_ctx* ctx, int b, double time, const double2* t1, const double2* t2,
                          double2* x1, double2* x2, char* base, cudaStream_t st) {
  Runner<R>& Rn = ctx->run<R>();
  DevicePool pool;
  pool.base = base;
  pool.cap = kNoAllocBytes;
  Engine<R> E(st);
  E.use_pool(&pool);
  E.set_tensor_cores(Rn.E.tensor_cores());
  E.set_wait_budget(Rn.E.wait_budget());
  E.set_eig_sweep_cap(Rn.E.eig_sweep_cap());
  E.set_profiler(&ctx->prof);  // records events only while profiling is enabled
  try {
    // the evaluation time lives in the region too (nothing else is written
    // before the recorded graph reads it)
    double* tdev = static_cast<double*>(pool.take(sizeof(double)));
    RTCC3_CUDA(cudaMemcpyAsync(tdev, &time, sizeof(double), cudaMemcpyHostToDevice, st));
    E.begin();
    StageOptions so;
    so.ccsd = false;
    so.triples = true;
    so.need_grad = false;
    so.field_terms = true;
    so.field_iters = field_sweeps(ctx, b);
    so.rotation = ctx->opt.field_solver == 0;
    StageNodes S = record_stage<R>(E, Rn.H, so, [&](const StageNodes& s) {
      launch_load_amplitudes<R>(t1, t2, E.data(s.t1), E.data(s.t2), ctx->o, ctx->v, st);
      launch_field_operator<R>(E.data(s.w), ctx->mu, ctx->fdev + b, tdev, 0.0, ctx->n, st);
    });
    launch_export<R>(E.data(S.r1), x1, ctx->n1, st);
    launch_export<R>(E.data(S.r2), x2, ctx->n2, st);
  } catch (...) {
    // a request the region cannot serve (or any other failure) may come
    // after kernels that write the region were enqueued: let them finish
    // before the error returns, so the next call does not race with them
    cudaStreamSynchronize(st);
    throw;
  }
  // the engine's host-side tables must outlive the copies it enqueued
  RTCC3_CUDA(cudaStreamSynchronize(st));
  if (E.tensor_cores()) {
    int flag = 0;
    RTCC3_CUDA(cudaMemcpy(&flag, E.error_flag(), sizeof(int), cudaMemcpyDeviceToHost));
    RTCC3_CHECK(flag == 0, RTCC3_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on its pipeline");
  }
}

// Candidate storage forms of the triples for this context, in the order
// they are timed: whole tensors when 24 of them fit in 70% of the free
// memory (-1), then slabs of o, o/2, o/4, ..., 1 first occupied indices
// whose four slab buffers fit in a quarter of it.
std::vector<int> chunk_candidates(const rtcc3_ctx* ctx) {
  std::vector<int> c;
  const int o = ctx->o, v = ctx->v;
  const double elem = ctx->fp64() ? 16.0 : 8.0;
  const double freeb = double(ctx->free_at_setup);
  if (24.0 * double(o) * o * o * v * v * v * elem <= 0.7 * freeb) c.push_back(-1);
  for (int k = o; k >= 1; k = (k + 1) / 2) {
    if (4.0 * double(k) * o * o * v * v * v * elem <= 0.25 * freeb &&
        std::find(c.begin(), c.end(), k) == c.end())
      c.push_back(k);
    if (k == 1) break;
  }
  return c;
}

// Times one full stage (forward and reverse pass) of slot b for every
// candidate triples storage form and keeps the fastest in the options.
template <typename R>
void autotune_impl(rtcc3_ctx* ctx, int b, int* best_chunk, float* best_ms, int max_out,
                   int* cand_out, float* ms_out, int* count) {
  Engine<R>& E = ctx->run<R>().E;
  const std::vector<int> cands = chunk_candidates(ctx);
  RTCC3_CHECK(!cands.empty(), RTCC3_ERR_OOM, "no triples storage form fits in device memory");
  const int saved = ctx->opt.triples_chunk;
  cudaEvent_t e0, e1;
  RTCC3_CUDA(cudaEventCreate(&e0));
  RTCC3_CUDA(cudaEventCreate(&e1));
  int best = 0;
  float bms = 0.f;
  int k = 0;
  try {
    for (int c : cands) {
      ctx->opt.triples_chunk = c;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first evaluation builds the plans
        RTCC3_CUDA(cudaEventRecord(e0, ctx->stream));
        eval_stage<R>(ctx, b, ctx->y + size_t(b) * ctx->ny, nullptr, 0.0, ctx->tdev, 0.0, true,
                      ctx->fdev + b, true, field_sweeps(ctx, b));
        RTCC3_CUDA(cudaEventRecord(e1, ctx->stream));
        RTCC3_CUDA(cudaEventSynchronize(e1));
        RTCC3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      }
      check_device_timeout<R>(ctx);
      if (k < max_out) {
        if (cand_out) cand_out[k] = c;
        if (ms_out) ms_out[k] = ms;
      }
      ++k;
      if (best == 0 || ms < bms) {
        best = c;
        bms = ms;
      }
    }
  } catch (...) {
    ctx->opt.triples_chunk = saved;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->opt.triples_chunk = best;
  drop_graph(ctx);
  if (best_chunk) *best_chunk = best;
  if (best_ms) *best_ms = bms;
  if (count) *count = k;
  E.reset_launch_count();
}

uint64_t fnv1a(const unsigned char* p, size_t n) {
  uint64_t h = 1469598103934665603ULL;
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 1099511628211ULL; }
  return h;
}

struct StateHeader {
  char magic[8];
  int version, o, v, nb;
  long long ny;
  double time;
  long long step;
};

}  // namespace

extern "C" {

void rtcc3_default_options(rtcc3_options* opt) {
  if (!opt) return;
  opt->precision = RTCC3_PREC_FP64;
  opt->triples = 1;
  opt->device = 0;
  opt->use_graphs = 1;
  opt->field_tol = 0.0;
  opt->field_solver = 0;
  opt->triples_chunk = 0;
  opt->spin_budget = 0;
  opt->eig_sweep_cap = 0;
  opt->storage = RTCC3_STORAGE_C128;
  opt->tc_scope = 0;
  opt->checked = 0;
  opt->serial = 0;
}

int rtcc3_create(int nocc, int nvir, int nbatch, const rtcc3_options* opt, rtcc3_ctx** out) {
  if (!out) return RTCC3_ERR_ARG;
  *out = nullptr;
  if (nocc < 1 || nvir < 1 || nbatch < 1 || nbatch > 64) return RTCC3_ERR_ARG;
  auto ctx = std::make_unique<rtcc3_ctx>();
  if (opt) ctx->opt = *opt; else rtcc3_default_options(&ctx->opt);
  if (ctx->opt.precision < RTCC3_PREC_FP64 || ctx->opt.precision > RTCC3_PREC_BF16)
    return RTCC3_ERR_ARG;
  if (ctx->opt.storage != RTCC3_STORAGE_C128 && ctx->opt.storage != RTCC3_STORAGE_C64)
    return RTCC3_ERR_ARG;
  if (ctx->opt.tc_scope < 0 || ctx->opt.tc_scope > 2) return RTCC3_ERR_ARG;
  ctx->o = nocc; ctx->v = nvir; ctx->n = nocc + nvir; ctx->nb = nbatch;
  ctx->n1 = size_t(nocc) * nvir;
  ctx->n2 = ctx->n1 * ctx->n1;
  ctx->ny = 2 * (ctx->n1 + ctx->n2);
  rtcc3_ctx* raw = ctx.get();
  const int rc = guarded(raw, [&] {
    RTCC3_CUDA(cudaSetDevice(raw->opt.device));
    RTCC3_CUDA(cudaStreamCreateWithFlags(&raw->stream, cudaStreamNonBlocking));
    raw->y = raw->dalloc<double2>(raw->ny * nbatch);
    raw->acc = raw->dalloc<double2>(raw->ny);
    raw->kbuf = raw->dalloc<double2>(raw->ny);
    raw->res = raw->dalloc<double2>(raw->ny);
    raw->fdev = raw->dalloc<FieldDev>(nbatch);
    raw->fnone = raw->dalloc<FieldDev>(1);
    raw->tdev = raw->dalloc<double>(1);
    raw->teval = raw->dalloc<double>(1);
    raw->stepdev = raw->dalloc<int>(1);
    raw->baddev = raw->dalloc<int>(1);
    raw->maxr = raw->dalloc<double>(1);
    raw->tdesc = raw->dalloc<TrajDesc>(1);
    raw->checkflag = raw->dalloc<int>(1);
    RTCC3_CUDA(cudaMemset(raw->checkflag, 0, sizeof(int)));
    raw->fhost.assign(nbatch, FieldDev{0, 0.0, 0.0, 0.0, 1.0, {0.0, 0.0, 1.0}});
    RTCC3_CUDA(cudaMemcpy(raw->fdev, raw->fhost.data(), nbatch * sizeof(FieldDev), cudaMemcpyHostToDevice));
    RTCC3_CUDA(cudaMemcpy(raw->fnone, raw->fhost.data(), sizeof(FieldDev), cudaMemcpyHostToDevice));
    RTCC3_CUDA(cudaMemset(raw->y, 0, raw->ny * nbatch * sizeof(double2)));
    RTCC3_CUDA(cudaMemset(raw->tdev, 0, sizeof(double)));
  });
  if (rc != RTCC3_OK) return rc;
  *out = ctx.release();
  return RTCC3_OK;
}

int rtcc3_destroy(rtcc3_ctx* ctx) {
  delete ctx;
  return RTCC3_OK;
}

const char* rtcc3_last_error(const rtcc3_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int rtcc3_set_hamiltonian(rtcc3_ctx* ctx, const double* eps, int naux, const double* Lfac,
                          const double* dipole) {
  if (!ctx) return RTCC3_ERR_ARG;
  if (!eps || !Lfac || !dipole || naux < 1) return fail(ctx, RTCC3_ERR_ARG, "null input or naux < 1");
  return guarded(ctx, [&] {
    RTCC3_CUDA(cudaSetDevice(ctx->opt.device));
    const int n = ctx->n;
    for (int p = 0; p < n; ++p) RTCC3_CHECK(std::isfinite(eps[p]), RTCC3_ERR_ARG, "non-finite eps");
    double emax_o = -1e300, emin_v = 1e300;
    for (int p = 0; p < ctx->o; ++p) emax_o = std::max(emax_o, eps[p]);
    for (int p = ctx->o; p < n; ++p) emin_v = std::min(emin_v, eps[p]);
    RTCC3_CHECK(emax_o < emin_v, RTCC3_ERR_ARG,
                "highest occupied orbital energy must lie below the lowest virtual");
    ctx->naux = naux;
    ctx->eps_h.assign(eps, eps + n);
    ctx->mu_h.assign(dipole, dipole + size_t(3) * n * n);
    if (!ctx->eps) ctx->eps = ctx->dalloc<double>(n);
    if (!ctx->mu) ctx->mu = ctx->dalloc<double>(size_t(3) * n * n);
    RTCC3_CUDA(cudaMemcpy(ctx->eps, eps, n * sizeof(double), cudaMemcpyHostToDevice));
    RTCC3_CUDA(cudaMemcpy(ctx->mu, dipole, size_t(3) * n * n * sizeof(double), cudaMemcpyHostToDevice));
    drop_graph(ctx);
    ctx->runner.reset();
    if (ctx->fp64()) setup_runner<double>(ctx, Lfac);
    else setup_runner<float>(ctx, Lfac);
    RTCC3_CUDA(cudaMemset(ctx->y, 0, ctx->ny * ctx->nb * sizeof(double2)));
    ctx->time = 0.0;
    ctx->step_total = 0;
    RTCC3_CUDA(cudaMemcpy(ctx->tdev, &ctx->time, sizeof(double), cudaMemcpyHostToDevice));
    size_t fr = 0, tot = 0;
    RTCC3_CUDA(cudaMemGetInfo(&fr, &tot));
    ctx->free_at_setup = fr;
    ctx->have_ham = true;
  });
}

namespace {

// Pivoted Cholesky factors of V[(pq)][(rs)] = (pq|rs): the pivot is the
// largest remaining diagonal element, the new factor the pivot's residual
// column over its square root, until every remaining diagonal element is
// <= tol (the residual is positive semidefinite, so no integral then differs
// by more than tol).  Row p of V is read for column p (V symmetric).
int eri_cholesky_impl(int n, const double* eri, double tol, int max_rank,
                      std::vector<double>& L, int& rank) {
  rank = 0;
  if (n < 1 || !eri || !(tol > 0.0) || max_rank < 1) return RTCC3_ERR_ARG;
  const size_t N = size_t(n) * n;
  double vmax = 0.0;
  for (size_t i = 0; i < N * N; ++i) {
    if (!std::isfinite(eri[i])) return RTCC3_ERR_ARG;
    vmax = std::max(vmax, std::fabs(eri[i]));
  }
  const double symtol = 1e-12 * std::max(1.0, vmax);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
          const double x = eri[((size_t(p) * n + q) * n + r) * n + s];
          if (std::fabs(x - eri[((size_t(q) * n + p) * n + r) * n + s]) > symtol ||
              std::fabs(x - eri[((size_t(r) * n + s) * n + p) * n + q]) > symtol)
            return RTCC3_ERR_ARG;
        }
  std::vector<double> d(N);
  for (size_t i = 0; i < N; ++i) d[i] = eri[i * N + i];
  L.clear();
  while (true) {
    size_t piv = 0;
    for (size_t i = 1; i < N; ++i)
      if (d[i] > d[piv]) piv = i;
    const double dp = d[piv];
    if (dp <= tol) break;
    if (rank >= max_rank) return RTCC3_ERR_NOT_CONVERGED;
    L.resize(size_t(rank + 1) * N);
    double* Lr = L.data() + size_t(rank) * N;
    const double* row = eri + piv * N;
    for (size_t i = 0; i < N; ++i) Lr[i] = row[i];
    for (int k = 0; k < rank; ++k) {
      const double* Lk = L.data() + size_t(k) * N;
      const double lk = Lk[piv];
      if (lk != 0.0)
        for (size_t i = 0; i < N; ++i) Lr[i] -= lk * Lk[i];
    }
    const double sc = 1.0 / std::sqrt(dp);
    for (size_t i = 0; i < N; ++i) {
      Lr[i] *= sc;
      d[i] -= Lr[i] * Lr[i];
    }
    d[piv] = 0.0;
    ++rank;
  }
  for (size_t i = 0; i < N; ++i)
    if (d[i] < -tol) return RTCC3_ERR_ARG;  // not positive semidefinite
  return RTCC3_OK;
}

}  // namespace

int rtcc3_eri_cholesky(int nmo, const double* eri, double tol, int max_rank, double* Lfac,
                       int* rank) {
  if (!Lfac || !rank) return RTCC3_ERR_ARG;
  try {
    std::vector<double> L;
    int r = 0;
    const int rc = eri_cholesky_impl(nmo, eri, tol, max_rank, L, r);
    *rank = r;
    if (r > 0) std::copy(L.begin(), L.begin() + size_t(r) * nmo * nmo, Lfac);
    return rc;
  } catch (const std::bad_alloc&) {
    return RTCC3_ERR_OOM;
  } catch (...) {
    return RTCC3_ERR_ARG;
  }
}

int rtcc3_set_hamiltonian_eri(rtcc3_ctx* ctx, const double* eps, const double* eri,
                              const double* dipole) {
  if (!ctx) return RTCC3_ERR_ARG;
  if (!eps || !eri || !dipole) return fail(ctx, RTCC3_ERR_ARG, "null input");
  std::vector<double> L;
  int rank = 0;
  int rc;
  try {
    rc = eri_cholesky_impl(ctx->n, eri, 1e-12, ctx->n * ctx->n, L, rank);
  } catch (const std::bad_alloc&) {
    return fail(ctx, RTCC3_ERR_OOM, "host allocation failed in the Cholesky factorisation");
  }
  if (rc != RTCC3_OK)
    return fail(ctx, rc, "two-electron integrals not finite, not symmetric or not positive semidefinite");
  if (rank == 0) {  // all integrals below the tolerance: one zero factor
    rank = 1;
    L.assign(size_t(ctx->n) * ctx->n, 0.0);
  }
  return rtcc3_set_hamiltonian(ctx, eps, rank, L.data(), dipole);
}

int rtcc3_set_field(rtcc3_ctx* ctx, int b, int kind, double amplitude, double omega, double center,
                    double width, const double* dir) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    check_slot(ctx, b);
    RTCC3_CHECK(kind >= RTCC3_FIELD_NONE && kind <= RTCC3_FIELD_QRCW, RTCC3_ERR_ARG, "unknown field kind");
    RTCC3_CHECK(std::isfinite(amplitude) && std::isfinite(omega) && std::isfinite(center) &&
                    std::isfinite(width), RTCC3_ERR_ARG, "non-finite field parameter");
    RTCC3_CHECK(kind != RTCC3_FIELD_GAUSS || width > 0.0, RTCC3_ERR_ARG, "Gaussian width must be > 0");
    RTCC3_CHECK((kind != RTCC3_FIELD_LRCW && kind != RTCC3_FIELD_QRCW) || width > 0.0, RTCC3_ERR_ARG,
                "ramp duration (width) must be > 0");
    FieldDev f{kind, amplitude, omega, center, width, {0.0, 0.0, 1.0}};
    if (dir) { f.dir[0] = dir[0]; f.dir[1] = dir[1]; f.dir[2] = dir[2]; }
    ctx->fhost[b] = f;
    drop_graph(ctx);  // field parameters live on the device, sweep counts do not
    RTCC3_CUDA(cudaMemcpy(ctx->fdev + b, &f, sizeof(FieldDev), cudaMemcpyHostToDevice));
  });
}

int rtcc3_set_amplitudes(rtcc3_ctx* ctx, int b, const double* t1, const double* t2,
                         const double* l1, const double* l2) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    check_slot(ctx, b);
    double2* yb = ctx->y + size_t(b) * ctx->ny;
    const size_t n1 = ctx->n1, n2 = ctx->n2;
    const double* src[4] = {t1, t2, l1, l2};
    const size_t off[4] = {0, n1, n1 + n2, 2 * n1 + n2};
    const size_t cnt[4] = {n1, n2, n1, n2};
    for (int k = 0; k < 4; ++k) {
      if (!src[k]) continue;
      for (size_t t = 0; t < 2 * cnt[k]; ++t)
        RTCC3_CHECK(std::isfinite(src[k][t]), RTCC3_ERR_ARG, "non-finite amplitude");
      RTCC3_CUDA(cudaMemcpy(yb + off[k], src[k], cnt[k] * sizeof(double2), cudaMemcpyHostToDevice));
    }
  });
}

int rtcc3_get_amplitudes(const rtcc3_ctx* cctx, int b, double* t1, double* t2, double* l1,
                         double* l2) {
  rtcc3_ctx* ctx = const_cast<rtcc3_ctx*>(cctx);
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    check_slot(ctx, b);
    RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
    const double2* yb = ctx->y + size_t(b) * ctx->ny;
    const size_t n1 = ctx->n1, n2 = ctx->n2;
    double* dst[4] = {t1, t2, l1, l2};
    const size_t off[4] = {0, n1, n1 + n2, 2 * n1 + n2};
    const size_t cnt[4] = {n1, n2, n1, n2};
    for (int k = 0; k < 4; ++k)
      if (dst[k]) RTCC3_CUDA(cudaMemcpy(dst[k], yb + off[k], cnt[k] * sizeof(double2), cudaMemcpyDeviceToHost));
  });
}

int rtcc3_set_time(rtcc3_ctx* ctx, double time) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    RTCC3_CHECK(std::isfinite(time), RTCC3_ERR_ARG, "non-finite time");
    ctx->time = time;
    RTCC3_CUDA(cudaMemcpy(ctx->tdev, &time, sizeof(double), cudaMemcpyHostToDevice));
  });
}

int rtcc3_get_time(const rtcc3_ctx* ctx, double* time) {
  if (!ctx || !time) return RTCC3_ERR_ARG;
  *time = ctx->time;
  return RTCC3_OK;
}

int rtcc3_compute_residuals(rtcc3_ctx* ctx, int b, double time, double* r_t1, double* r_t2,
                            double* r_l1, double* r_l2, double* energy, double* dipole) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    require_ham(ctx);
    check_slot(ctx, b);
    RTCC3_CHECK(std::isfinite(time), RTCC3_ERR_ARG, "non-finite time");
    if (ctx->fp64()) residuals_impl<double>(ctx, b, time, r_t1, r_t2, r_l1, r_l2, energy, dipole);
    else residuals_impl<float>(ctx, b, time, r_t1, r_t2, r_l1, r_l2, energy, dipole);
  });
}

int rtcc3_solve_ground_state(rtcc3_ctx* ctx, double tol, int maxiter) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    require_ham(ctx);
    RTCC3_CHECK(tol > 0.0 && maxiter > 0, RTCC3_ERR_ARG, "tol must be > 0 and maxiter > 0");
    if (ctx->fp64()) ground_state_impl<double>(ctx, tol, maxiter);
    else ground_state_impl<float>(ctx, tol, maxiter);
  });
}

static int propagate_common(rtcc3_ctx* ctx, double h, int nsteps, double2* dip, double2* en,
                            bool host, double* dip_h, double* en_h, bool final) {
  return guarded(ctx, [&] {
    require_ham(ctx);
    RTCC3_CHECK(nsteps >= 0 && std::isfinite(h) && h != 0.0, RTCC3_ERR_ARG, "bad step size or count");
    // a chunk records the state at the start of each step only; the state it
    // ends in is entry 0 of the next chunk
    const size_t entries = size_t(nsteps) + (final ? 1 : 0);
    if (entries == 0) return;
    double2* d = dip;
    double2* e = en;
    if (host) {
      ensure_traj(ctx, entries * ctx->nb);
      d = ctx->dip_traj;
      e = ctx->en_traj;
    }
    if (ctx->fp64()) propagate_impl<double>(ctx, h, nsteps, d, e, entries, final);
    else propagate_impl<float>(ctx, h, nsteps, d, e, entries, final);
    if (host) {
      if (dip_h)
        RTCC3_CUDA(cudaMemcpy(dip_h, d, entries * ctx->nb * 3 * sizeof(double2), cudaMemcpyDeviceToHost));
      if (en_h)
        RTCC3_CUDA(cudaMemcpy(en_h, e, entries * ctx->nb * sizeof(double2), cudaMemcpyDeviceToHost));
    }
  });
}

static int propagate_dev_common(rtcc3_ctx* ctx, double h, int nsteps, void* dipole_dev,
                                void* energy_dev, void* stream, bool final) {
  // the work runs on the context stream; an external stream is ordered
  // before and after it with events
  cudaStream_t ext = static_cast<cudaStream_t>(stream);
  return guarded(ctx, [&] {
    if (ext) {
      cudaEvent_t ev;
      RTCC3_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      RTCC3_CUDA(cudaEventRecord(ev, ext));
      RTCC3_CUDA(cudaStreamWaitEvent(ctx->stream, ev, 0));
      cudaEventDestroy(ev);
    }
    const int rc = propagate_common(ctx, h, nsteps, static_cast<double2*>(dipole_dev),
                                    static_cast<double2*>(energy_dev), false, nullptr, nullptr,
                                    final);
    if (rc != RTCC3_OK) throw Error(rc, ctx->err);
    if (ext) {
      cudaEvent_t ev;
      RTCC3_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      RTCC3_CUDA(cudaEventRecord(ev, ctx->stream));
      RTCC3_CUDA(cudaStreamWaitEvent(ext, ev, 0));
      cudaEventDestroy(ev);
    }
  });
}

int rtcc3_propagate_rk4(rtcc3_ctx* ctx, double h, int nsteps, double* dipole, double* energy) {
  if (!ctx) return RTCC3_ERR_ARG;
  return propagate_common(ctx, h, nsteps, nullptr, nullptr, true, dipole, energy, true);
}

int rtcc3_propagate_rk4_dev(rtcc3_ctx* ctx, double h, int nsteps, void* dipole_dev,
                            void* energy_dev, void* stream) {
  if (!ctx) return RTCC3_ERR_ARG;
  return propagate_dev_common(ctx, h, nsteps, dipole_dev, energy_dev, stream, true);
}

int rtcc3_propagate_rk4_chunk(rtcc3_ctx* ctx, double h, int nsteps, double* dipole,
                              double* energy) {
  if (!ctx) return RTCC3_ERR_ARG;
  return propagate_common(ctx, h, nsteps, nullptr, nullptr, true, dipole, energy, false);
}

int rtcc3_propagate_rk4_chunk_dev(rtcc3_ctx* ctx, double h, int nsteps, void* dipole_dev,
                                  void* energy_dev, void* stream) {
  if (!ctx) return RTCC3_ERR_ARG;
  return propagate_dev_common(ctx, h, nsteps, dipole_dev, energy_dev, stream, false);
}

int rtcc3_triples_forward_dev(rtcc3_ctx* ctx, int b, double time, const void* t1, const void* t2,
                              void* x1, void* x2, void* stream) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    require_ham(ctx);
    check_slot(ctx, b);
    RTCC3_CHECK(t1 && t2 && x1 && x2, RTCC3_ERR_ARG, "null device buffer");
    RTCC3_CHECK(ctx->opt.triples, RTCC3_ERR_STATE, "context created without triples");
    if (stream) RTCC3_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    auto f = [&](auto tag) {
      using R = decltype(tag);
      triples_impl<R>(ctx, b, time, static_cast<const double2*>(t1), static_cast<const double2*>(t2),
                      nullptr, nullptr, static_cast<double2*>(x1), static_cast<double2*>(x2),
                      nullptr, nullptr, static_cast<cudaStream_t>(stream));
    };
    if (ctx->fp64()) f(double()); else f(float());
  });
}

int rtcc3_triples_vjp_dev(rtcc3_ctx* ctx, int b, double time, const void* t1, const void* t2,
                          const void* u1, const void* u2, void* g1, void* g2, void* stream) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    require_ham(ctx);
    check_slot(ctx, b);
    RTCC3_CHECK(t1 && t2 && u1 && u2 && g1 && g2, RTCC3_ERR_ARG, "null device buffer");
    RTCC3_CHECK(ctx->opt.triples, RTCC3_ERR_STATE, "context created without triples");
    if (stream) RTCC3_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    auto f = [&](auto tag) {
      using R = decltype(tag);
      triples_impl<R>(ctx, b, time, static_cast<const double2*>(t1), static_cast<const double2*>(t2),
                      static_cast<const double2*>(u1), static_cast<const double2*>(u2), nullptr,
                      nullptr, static_cast<double2*>(g1), static_cast<double2*>(g2),
                      static_cast<cudaStream_t>(stream));
    };
    if (ctx->fp64()) f(double()); else f(float());
  });
}

int rtcc3_triples_forward_noalloc_dev(rtcc3_ctx* ctx, int b, double time, const void* t1,
                                      const void* t2, void* x1, void* x2, void* stream) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    require_ham(ctx);
    check_slot(ctx, b);
    RTCC3_CHECK(t1 && t2 && x1 && x2, RTCC3_ERR_ARG, "null device buffer");
    RTCC3_CHECK(ctx->opt.triples, RTCC3_ERR_STATE, "context created without triples");
    // the context's device: its Hamiltonian, stream and the region's copy
    // used below all live there, whatever device the caller has current
    const int dev = ctx->opt.device;
    RTCC3_CUDA(cudaSetDevice(dev));
    char* base = noalloc_scratch_address(dev);
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : ctx->stream;
    auto f = [&](auto tag) {
      using R = decltype(tag);
      const size_t need = noalloc_estimate<R>(ctx);
      RTCC3_CHECK(need <= kNoAllocBytes, RTCC3_ERR_ARG,
                  "system too large for the allocation-free path: needs about " +
                      std::to_string(need >> 20) + " MiB of workspace, the static region holds " +
                      std::to_string(kNoAllocBytes >> 20) + " MiB");
      triples_noalloc_impl<R>(ctx, b, time, static_cast<const double2*>(t1),
                              static_cast<const double2*>(t2), static_cast<double2*>(x1),
                              static_cast<double2*>(x2), base, st);
    };
    if (ctx->fp64()) f(double()); else f(float());
  });
}

int rtcc3_state_size(const rtcc3_ctx* ctx, long long* bytes) {
  if (!ctx || !bytes) return RTCC3_ERR_ARG;
  *bytes = (long long)(sizeof(StateHeader) + ctx->ny * ctx->nb * sizeof(double2) + sizeof(uint64_t));
  return RTCC3_OK;
}

int rtcc3_get_state(const rtcc3_ctx* cctx, void* buf, long long bytes) {
  rtcc3_ctx* ctx = const_cast<rtcc3_ctx*>(cctx);
  if (!ctx || !buf) return RTCC3_ERR_ARG;
  long long need = 0;
  rtcc3_state_size(ctx, &need);
  if (bytes < need) return fail(ctx, RTCC3_ERR_ARG, "state buffer too small");
  return guarded(ctx, [&] {
    RTCC3_CUDA(cudaStreamSynchronize(ctx->stream));
    unsigned char* p = static_cast<unsigned char*>(buf);
    StateHeader hd{};
    std::memcpy(hd.magic, "RTCC3ST1", 8);
    hd.version = 1; hd.o = ctx->o; hd.v = ctx->v; hd.nb = ctx->nb;
    hd.ny = (long long)ctx->ny; hd.time = ctx->time; hd.step = ctx->step_total;
    std::memcpy(p, &hd, sizeof(hd));
    const size_t body = ctx->ny * ctx->nb * sizeof(double2);
    RTCC3_CUDA(cudaMemcpy(p + sizeof(hd), ctx->y, body, cudaMemcpyDeviceToHost));
    const uint64_t h = fnv1a(p, sizeof(hd) + body);
    std::memcpy(p + sizeof(hd) + body, &h, sizeof(h));
  });
}

int rtcc3_set_state(rtcc3_ctx* ctx, const void* buf, long long bytes) {
  if (!ctx || !buf) return RTCC3_ERR_ARG;
  long long need = 0;
  rtcc3_state_size(ctx, &need);
  if (bytes != need) return fail(ctx, RTCC3_ERR_ARG, "state image has the wrong size");
  return guarded(ctx, [&] {
    const unsigned char* p = static_cast<const unsigned char*>(buf);
    StateHeader hd{};
    std::memcpy(&hd, p, sizeof(hd));
    RTCC3_CHECK(std::memcmp(hd.magic, "RTCC3ST1", 8) == 0 && hd.version == 1, RTCC3_ERR_ARG,
                "not an rtcc3 state image (magic/version)");
    RTCC3_CHECK(hd.o == ctx->o && hd.v == ctx->v && hd.nb == ctx->nb && hd.ny == (long long)ctx->ny,
                RTCC3_ERR_ARG, "state image was written for different sizes");
    const size_t body = ctx->ny * ctx->nb * sizeof(double2);
    uint64_t h = 0;
    std::memcpy(&h, p + sizeof(hd) + body, sizeof(h));
    RTCC3_CHECK(h == fnv1a(p, sizeof(hd) + body), RTCC3_ERR_ARG, "state image checksum mismatch");
    RTCC3_CUDA(cudaMemcpy(ctx->y, p + sizeof(hd), body, cudaMemcpyHostToDevice));
    ctx->time = hd.time;
    ctx->step_total = hd.step;
    RTCC3_CUDA(cudaMemcpy(ctx->tdev, &ctx->time, sizeof(double), cudaMemcpyHostToDevice));
  });
}

int rtcc3_autotune_triples(rtcc3_ctx* ctx, int b, int* chunk, float* ms, int max_candidates,
                           int* candidates, float* candidate_ms, int* count) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    require_ham(ctx);
    check_slot(ctx, b);
    RTCC3_CHECK(ctx->opt.triples && ctx->opt.field_solver == 0, RTCC3_ERR_STATE,
                "autotuning needs the triples with the field-dressed eigenbasis solver");
    RTCC3_CHECK(max_candidates >= 0, RTCC3_ERR_ARG, "max_candidates < 0");
    if (ctx->fp64())
      autotune_impl<double>(ctx, b, chunk, ms, max_candidates, candidates, candidate_ms, count);
    else
      autotune_impl<float>(ctx, b, chunk, ms, max_candidates, candidates, candidate_ms, count);
  });
}

int rtcc3_ground_state_history(const rtcc3_ctx* ctx, double* out, int max_entries, int* count,
                               int* t_iterations) {
  if (!ctx || max_entries < 0 || (max_entries > 0 && !out)) return RTCC3_ERR_ARG;
  const int n = int(ctx->gs_history.size());
  for (int k = 0; k < std::min(n, max_entries); ++k) out[k] = ctx->gs_history[size_t(k)];
  if (count) *count = n;
  if (t_iterations) *t_iterations = ctx->gs_t_iters;
  return RTCC3_OK;
}

int rtcc3_set_observables(rtcc3_ctx* ctx, int nops, const double* ops) {
  if (!ctx) return RTCC3_ERR_ARG;
  if (nops < 0 || nops > 64 || (nops > 0 && !ops))
    return fail(ctx, RTCC3_ERR_ARG, "0 <= nops <= 64 with a non-null operator array");
  return guarded(ctx, [&] {
    RTCC3_CUDA(cudaSetDevice(ctx->opt.device));
    const size_t nn = size_t(ctx->n) * ctx->n;
    for (size_t t = 0; t < 2 * nn * size_t(nops); ++t)
      RTCC3_CHECK(std::isfinite(ops[t]), RTCC3_ERR_ARG, "non-finite observable matrix element");
    if (ctx->obs_ops) cudaFree(ctx->obs_ops);
    if (ctx->obs_traj) cudaFree(ctx->obs_traj);
    ctx->obs_ops = nullptr;
    ctx->obs_traj = nullptr;
    ctx->obs_cap = 0;
    ctx->obs_last = 0;
    ctx->nobs = 0;
    if (nops > 0) {
      RTCC3_CUDA(cudaMalloc(&ctx->obs_ops, nn * nops * sizeof(double2)));
      RTCC3_CUDA(cudaMemcpy(ctx->obs_ops, ops, nn * nops * sizeof(double2), cudaMemcpyHostToDevice));
      ctx->nobs = nops;
    }
    drop_graph(ctx);  // the observables kernel's grid depends on nops
  });
}

int rtcc3_get_observables(const rtcc3_ctx* cctx, double* out, long long entries) {
  rtcc3_ctx* ctx = const_cast<rtcc3_ctx*>(cctx);
  if (!ctx || !out || entries < 0) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    RTCC3_CHECK(ctx->nobs > 0 && ctx->obs_last > 0, RTCC3_ERR_STATE,
                "no observables recorded (rtcc3_set_observables, then a compute or propagate call)");
    RTCC3_CHECK(entries >= ctx->obs_last, RTCC3_ERR_ARG,
                "output holds fewer entries than the last call recorded (" +
                    std::to_string(ctx->obs_last) + ")");
    RTCC3_CUDA(cudaMemcpy(out, ctx->obs_traj, size_t(ctx->obs_last) * ctx->nobs * sizeof(double2),
                          cudaMemcpyDeviceToHost));
  });
}

int rtcc3_measure_peaks(int device, double* tflops) {
  if (!tflops) return RTCC3_ERR_ARG;
  return guarded(nullptr, [&] {
    RTCC3_CUDA(cudaSetDevice(device));
    cudaStream_t s = nullptr;
    int* flag = nullptr;
    RTCC3_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    RTCC3_CUDA(cudaMalloc(&flag, sizeof(int)));
    RTCC3_CUDA(cudaMemset(flag, 0, sizeof(int)));
    try {
      for (int w = 0; w < 4; ++w) tflops[w] = measure_pipe_tflops(w, flag, s);
      int f = 0;
      RTCC3_CUDA(cudaMemcpy(&f, flag, sizeof(int), cudaMemcpyDeviceToHost));
      RTCC3_CHECK(f == 0, RTCC3_ERR_TIMEOUT, "a rate probe gave up waiting on its MMAs");
    } catch (...) {
      cudaStreamSynchronize(s);
      cudaFree(flag);
      cudaStreamDestroy(s);
      throw;
    }
    cudaFree(flag);
    cudaStreamDestroy(s);
  });
}

int rtcc3_set_wait_budgets(rtcc3_ctx* ctx, long long spin_budget, int eig_sweep_cap) {
  if (!ctx) return RTCC3_ERR_ARG;
  if (spin_budget < 0 || eig_sweep_cap < 0)
    return fail(ctx, RTCC3_ERR_ARG, "negative wait budget");
  return guarded(ctx, [&] {
    ctx->opt.spin_budget = spin_budget;
    ctx->opt.eig_sweep_cap = eig_sweep_cap;
    if (ctx->runner) {
      auto f = [&](auto tag) {
        using R = decltype(tag);
        ctx->run<R>().E.set_wait_budget(spin_budget);
        ctx->run<R>().E.set_eig_sweep_cap(eig_sweep_cap);
      };
      if (ctx->fp64()) f(double()); else f(float());
    }
    drop_graph(ctx);  // a captured step holds the budgets as kernel arguments
  });
}

int rtcc3_set_profiling(rtcc3_ctx* ctx, int enable) {
  if (!ctx) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    ctx->prof.reset();
    ctx->prof.enabled = enable != 0;
    const char* det = std::getenv("RTCC3_PROFILE_DETAIL");
    ctx->prof.set_detail(det && det[0] == '1');
    drop_graph(ctx);
  });
}

int rtcc3_kernel_stats(rtcc3_ctx* ctx, rtcc3_kernel_stat* out, int max_entries, int* count) {
  if (!ctx || !count) return RTCC3_ERR_ARG;
  return guarded(ctx, [&] {
    ctx->prof.collect();
    const auto& st = ctx->prof.stats();
    *count = int(st.size());
    for (int i = 0; i < int(st.size()) && i < max_entries && out; ++i) {
      std::memset(&out[i], 0, sizeof(rtcc3_kernel_stat));
      std::strncpy(out[i].name, st[i].name.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = st[i].launches;
      out[i].ms = st[i].ms;
      out[i].flops = st[i].flops;
      out[i].bytes = st[i].bytes;
    }
  });
}

int rtcc3_stats(const rtcc3_ctx* ctx, long long* launches, long long* device_bytes) {
  if (!ctx) return RTCC3_ERR_ARG;
  if (launches) *launches = ctx->last_launches;
  if (device_bytes) {
    long long s = 0;
    if (ctx->runner) {
      if (ctx->fp64()) s += (long long)static_cast<Runner<double>*>(ctx->runner.get())->E.arena().reserved();
      else s += (long long)static_cast<Runner<float>*>(ctx->runner.get())->E.arena().reserved();
    }
    *device_bytes = s;
  }
  return RTCC3_OK;
}

}  // extern "C"
