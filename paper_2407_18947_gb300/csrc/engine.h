// Reverse-mode tensor engine for the RT-CC3 residual graph.
//
// A residual evaluation is recorded as a list of operations on dense complex
// tensors ("nodes") living in a device arena:
//   * contract:  C (+)= alpha * sum_K A[..] B[..]   (einsum with two operands)
//   * axpy:      Y += alpha * X                      (X, Y arbitrary strided views)
//   * mulc:      Y += X .* c                         (c a constant tensor)
// Views carry an element offset and strides, so slices of the dressed
// integral tensor, index permutations and diagonals cost nothing.
// backward() replays the list in reverse and accumulates holomorphic
// vector-Jacobian products (plain transposes, no conjugation): for a
// contraction "a,b->c", grad(A) += alpha einsum("c,b->a", grad(C), B) and
// grad(B) += alpha einsum("a,c->b", A, grad(C)).
#pragma once

#include <functional>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.h"

namespace rtcc3 {

// Most sources one pass of a combine (and one merged reverse-pass gather)
// sums.
constexpr int kCombineSources = 8;

constexpr int kMaxDim = 8;

struct View {
  int node = -1;
  long long off = 0;
  int nd = 0;
  int shape[kMaxDim] = {0};
  long long stride[kMaxDim] = {0};
  size_t numel() const {
    size_t n = 1;
    for (int d = 0; d < nd; ++d) n *= size_t(shape[d]);
    return n;
  }
  // Slice [start, start+len) of dimension dim.
  View sub(int dim, int start, int len) const {
    View r = *this;
    r.off += (long long)start * stride[dim];
    r.shape[dim] = len;
    return r;
  }
};

// Offset tables of a planned contraction (device memory, cached per shape).
struct ContractPlan {
  int M = 1, N = 1, K = 1, nb = 1;
  int nsplit = 1, kchunk = 1;
  bool a_kcontig = false, b_kcontig = false;
  bool small_tile = false;  // 16x16 output tiles with 64-deep K slices (skinny shapes)
  int tile = 0;             // 0: 64 x 64, 1: 16 x 256, 2: 256 x 16 output tiles
  // kind 0: tiled gather-GEMM; 1: small output held whole by every CTA
  // (reduce_small, config small_cfg); 2: single long output column (gemv);
  // 3: outer product (K = 1, a streaming pass over C).
  // small_swap: the kernels run with A and B exchanged (kinds 1, 2: larger
  // side first; kind 3: the output's contiguous index on the second side).
  int kind = 0, small_cfg = 0;
  bool small_swap = false;
  long long gemv_boff = 0, gemv_coff = 0;  // B and C offsets of the single column
  // tensor-core route (complex64 graphs with TF32/BF16 operands)
  bool use_tc = false, tc_swap = false;
  int tc_nsplit = 1, tc_kp = 0;
  bool tc_out = false;  // short sum bound by its output (two CTAs per SM)
  long long a_off0 = 0, b_off0 = 0, c_off0 = 0;  // batch-0 offsets (host copies)
  long long *aM = nullptr, *aK = nullptr, *bN = nullptr, *bK = nullptr;
  long long *cM = nullptr, *cN = nullptr, *aB = nullptr, *bB = nullptr, *cB = nullptr;
  std::vector<long long> host;  // backing store for the uploaded tables
  void* dev = nullptr;
};

template <typename R>
class Engine {
 public:
  using C = Cx<R>;
  struct Node {
    C* data = nullptr;
    C* grad = nullptr;
    size_t numel = 0;
    std::vector<int> shape;
    bool needs_grad = false;
    bool grad_ready = false;  // grad holds valid values (zeroed or written)
  };

  explicit Engine(cudaStream_t s) : stream_(s) {}
  ~Engine();
  void set_stream(cudaStream_t s) { stream_ = s; }
  cudaStream_t stream() const { return stream_; }

  // Start a new graph: resets the arena cursor and the tape.
  void begin();
  // New tensor (zero-filled on the stream); a leaf may require gradients.
  // zero = false skips the fill when the first writer overwrites every element.
  int node(const std::vector<int>& shape, bool needs_grad = false, bool zero = true);
  // Register persistent device memory (a constant of the graph, no gradient).
  int external(C* data, const std::vector<int>& shape);
  View v(int node) const;
  // Permuted / diagonal view: spec like "jikbac->ijkabc" or "pqkk->pqk".
  View ev(const char* spec, const View& x) const;

  void contract(const char* spec, double alpha, const View& A, const View& B, const View& Cv,
                bool accumulate);
  void axpy(double alpha, const View& X, const View& Y);
  // Y (+)= sum_s alpha_s X_s in one pass (up to eight strided sources).
  void combine(std::initializer_list<std::pair<double, View>> srcs, const View& Y, bool overwrite);
  // Several overwriting combines at once (Y_o = sum_s alpha_os X_os): one
  // pass reading each distinct source once when the outputs are dense
  // (..., v, v, v) tensors and the sources permute their last three indices,
  // else one combine after another; the tape records one combine per output.
  void combine_multi(const std::vector<std::vector<std::pair<double, View>>>& srcs,
                     const std::vector<View>& ys);
  // Y (+)= alpha P_ijk^abc X for 6-index tensors (o,o,o,v,v,v); self-adjoint.
  void sym6(double alpha, const View& X, const View& Y, bool overwrite);
  void mulc(const View& X, const View& Cst, const View& Y);
  // Y += X / eps(index) with eps(index) = sum_d sign[d] * eps_dev[base[d] + index_d],
  // the orbital-energy denominators; the division is carried out in FP64.
  struct EpsSpec {
    const double* eps = nullptr;
    int sign[kMaxDim] = {0};
    int base[kMaxDim] = {0};
    // Triples shortcut (o,o,o,v,v,v): precomputed FP64 sums
    // osum[(i o + j) o + k] = e_i + e_j + e_k, vsum[(a v + b) v + c] = e_a + e_b + e_c.
    const double* osum = nullptr;
    const double* vsum = nullptr;
    int o = 0, v = 0;
    // Complex sums of eigenvalues in the field-dressed basis (take precedence).
    const double2* osum_c = nullptr;
    const double2* vsum_c = nullptr;
    // The sums in the compute precision, for the fused P_ijk^abc + division
    // kernels (real, or complex when osum_cr / vsum_cr are set).
    const R* osum_r = nullptr;
    const R* vsum_r = nullptr;
    const Cx<R>* osum_cr = nullptr;
    const Cx<R>* vsum_cr = nullptr;
    // o^3 occupied-block indices (i o + j) o + k in orbit order (the distinct
    // permutations of each i <= j <= k consecutively), the visiting order of
    // the fused kernels; null: natural order
    const int* order = nullptr;
  };
  void div_eps(const View& X, const EpsSpec& es, const View& Y, bool overwrite = false);
  // Y = alpha P_ijk^abc(X) / D (Eq. A30 and the denominators of Eq. 6 in one
  // pass; X, Y dense triples, es with FP64 sum tables; Y is overwritten).
  void sym6_div(double alpha, const View& X, const EpsSpec& es, const View& Y);
  // Non-differentiable initialisation.
  void fill_identity(int node);
  void fill_ones(int node);

  // Allocate gradient buffers of every node that needs one (small ones
  // zeroed; large ones are left unset: their first full-coverage write
  // overwrites, a partial first write zeroes them first, and an adjoint whose
  // cotangent was never written contributes nothing and is skipped).  After
  // writing the seeds into grad() and calling mark_grad_written() on them,
  // call backward().
  void prepare_backward();
  void mark_grad_written(int node) { nodes_[node].grad_ready = true; }
  // Zero a gradient that no operation wrote (before reading it outside the engine).
  void ensure_grad(int node) { zero_grad_if_unset(node); }
  bool grad_ready(int node) const { return nodes_[node].grad_ready; }
  void backward();

  // Untaped execution on data (g = false) or gradient (g = true) buffers,
  // for custom operations whose adjoint is written by hand.
  void exec_contract(const char* spec, double alpha, const View& A, bool ag, const View& B,
                     bool bg, const View& Cv, bool cg) {
    cur_tc_ = tc_region_;
    run_contract(spec, alpha, A, ag, B, bg, Cv, cg, true);
  }
  // As exec_contract, with each operand's data (or gradient) pointer moved by
  // sa / sb / sc elements and an explicit accumulate flag.  The plan is made
  // for the views as given, so a loop over slices of equal extent that
  // differ only in their start (views at start 0 plus the start as a shift)
  // reuses one plan.  Every kernel takes per-address decisions on
  // alignment, so any whole-element shift is valid.
  void exec_contract_at(const char* spec, double alpha, const View& A, bool ag, long long sa,
                        const View& B, bool bg, long long sb, const View& Cv, bool cg, long long sc,
                        bool accumulate) {
    cur_tc_ = tc_region_;
    run_contract(spec, alpha, A, ag, B, bg, Cv, cg, accumulate, sa, sb, sc);
  }
  // Slab of the triples (dense I x o x o x v x v x v, its first occupied
  // index running over i0 .. i0+I-1): Y = alpha X / D with the triples
  // denominators D[ijk abc] = vsum[abc] - osum[ijk] of es (the sum tables in
  // the compute precision, real or complex); X and Y on data buffers, Y may
  // be X.  Untaped.
  void exec_slab_div(double alpha, const View& X, int i0, const EpsSpec& es, const View& Y);
  void exec_axpy(double alpha, const View& X, bool xg, const View& Y, bool yg) {
    run_axpy(alpha, X, xg, Y, yg);
  }
  void exec_div(const View& X, bool xg, const EpsSpec& es, const View& Y, bool yg,
                bool overwrite = false) {
    run_div(X, xg, es, Y, yg, overwrite);
  }
  // Y = (X + X(jik,bac) + X(kji,cba)) / D over dense triples (X on its data
  // or gradient buffer; untaped; es with FP64 sum tables).
  // The forward of sym6_div without recording it (the caller's custom
  // adjoint then owns its reverse), and that reverse fused with the
  // three-term sum of the same cotangent: grad(X) (+)= alpha P6(grad(Y)) / D
  // and Y3 = P3(grad(Y)) / D (data of a dense node) in one pass.
  void exec_sym6_div(double alpha, const View& X, const EpsSpec& es, const View& Y) {
    run_sym6_div(alpha, X, false, es, Y, false, true, 6);
  }
  void exec_sym6_div_adjoint_pair(double alpha, const View& Yg, const EpsSpec& es, const View& Xg,
                                  const View& Y3) {
    run_sym6_div(alpha, Yg, true, es, Xg, true, false, 6, &Y3);
  }
  // grad(dst) (+)= a1 grad(x1)[i,a] y1[j,k,b,c] + a2 grad(x2)[i,j,a,b] y2[k,c]
  // over dense (o,o,o,v,v,v) in one pass (untaped; a zero coefficient drops
  // its term unread).
  void exec_outer_pair(double a1, const View& x1g, const View& y1, double a2, const View& x2g,
                       const View& y2, const View& dstg);
  void exec_sym3_div(const View& X, bool xg, const EpsSpec& es, const View& Y) {
    run_sym6_div(1.0, X, xg, es, Y, false, true, 3);
  }
  // Y = X (X on its data or gradient buffer; untaped).
  void exec_copy(const View& X, bool xg, const View& Y) {
    const double one = 1.0;
    run_combine(&X, &xg, &one, 1, Y, false, true, "copy");
  }
  // Y (+)= sum_s alpha_s X_s over data buffers (untaped).
  void exec_combine(std::initializer_list<std::pair<double, View>> srcs, const View& Y,
                    bool overwrite) {
    View xs[kCombineSources];
    bool xg[kCombineSources] = {};
    double al[kCombineSources];
    int ns = 0;
    for (auto& s : srcs) {
      RTCC3_CHECK(ns < kCombineSources, kErrArg, "combine takes at most 8 sources");
      xs[ns] = s.second;
      al[ns] = s.first;
      ++ns;
    }
    run_combine(xs, xg, al, ns, Y, false, overwrite, "combine");
  }
  // Record a custom operation: `bwd` runs at its place in the reverse sweep
  // (all gradients of tensors it produced are complete by then).
  void custom(std::function<void()> bwd, bool tc) {
    Op op{kCustom, "", 0.0, View(), View(), View(), EpsSpec()};
    op.tc = tc;
    op.fn = std::move(bwd);
    tape_.push_back(std::move(op));
  }
  void zero(int node, bool grad = false) {
    if (grad) nodes_[node].grad_ready = true;
    RTCC3_CUDA(cudaMemsetAsync(grad ? nodes_[node].grad : nodes_[node].data, 0,
                               nodes_[node].numel * sizeof(C), stream_));
  }
  void set_needs_grad(int node, bool g) { nodes_[node].needs_grad = g; }
  bool needs_grad(int node) const { return nodes_[node].needs_grad; }

  C* data(int n) const { return nodes_[n].data; }
  C* grad(int n) const { return nodes_[n].grad; }
  const Node& info(int n) const { return nodes_[n]; }
  Arena& arena() { return arena_; }
  size_t num_plans() const { return plans_.size(); }
  int launches() const { return launches_; }
  void reset_launch_count() { launches_ = 0; }
  // When true, creating a new contraction plan raises (used while a CUDA
  // graph is being captured: plans upload tables synchronously).
  void freeze_plans(bool f) { frozen_ = f; }
  // Persistent scratch buffers by slot: 0 split-K partials, 1/2 packed
  // tensor-core operands, 3 tensor-core split-K partials, 4 split-K partials
  // of the branch stream, 5 those of a concurrent region, 6-8 the branch
  // stream's tensor-core buffers.
  void* scratch(int slot, size_t bytes);
  // Route large contractions of a complex64 graph to the tcgen05 GEMM with
  // TF32 (elem_bytes 4) or BF16 (2) operands; 0 keeps the CUDA-core kernel.
  void set_tensor_cores(int elem_bytes) { tc_eb_ = elem_bytes; }
  int tensor_cores() const { return tc_eb_; }
  // Contractions recorded while the region is open (and their adjoints) may
  // take the tensor-core route; everything else stays on CUDA cores in FP32.
  void set_tc_region(bool open) { tc_region_ = open; }
  // Device word raised by a bounded wait that gave up (tensor-core kernel).
  int* error_flag();
  // Clock cycles a tensor-core kernel's wait on another warp may spin before
  // it gives up and raises the error flag (0: the kernels' default).
  // Checked mode: every tensor gets a canary after it, verified (raising
  // *flag) by verify_canaries() after the stage.
  void set_checked(bool c) { checked_ = c; }
  bool checked() const { return checked_; }
  void verify_canaries(int* flag);
  void set_wait_budget(long long cycles) { wait_budget_ = cycles; }
  long long wait_budget() const { return wait_budget_; }
  // QR sweeps the field eigensolver may take per matrix (0: its default).
  void set_eig_sweep_cap(int sweeps) { eig_cap_ = sweeps; }
  int eig_sweep_cap() const { return eig_cap_; }
  // Take every device buffer (arena, tables, scratch, flag) from `p` instead
  // of cudaMalloc; the engine then frees nothing either.
  void use_pool(DevicePool* p) {
    pool_ = p;
    arena_.use_pool(p);
  }
  // Incremented whenever a persistent buffer (the split-K scratch) moves:
  // a captured CUDA graph recorded under an older generation is stale.
  int generation() const { return generation_; }
  void set_profiler(Profiler* p) { prof_ = p; }
  // Reverse pass: the A and B adjoints of a CUDA-core product as parallel
  // branches, and concurrent regions (default on; off runs everything on
  // the engine's stream in recording order).
  void set_branches(bool on) { branches_ = on; }
  // Concurrent region: operations recorded between region_begin() and
  // region_end() run on a stream of their own, forked from the engine's
  // stream at region_begin(), concurrently with the operations recorded
  // after region_end() up to region_join(), which joins it back.  The
  // reverse pass mirrors it: the region's adjoints run on its stream,
  // forked where the reverse pass meets region_join() and joined where it
  // meets region_begin().  Every node the region writes, values or
  // cotangents, must be private to it (inputs shared with the rest of the
  // stage are copied before region_begin()).  regions() is false, and the
  // three calls do nothing, while profiling, with a caller's pool or with
  // branches off.
  bool regions() const { return branches_ && !pool_ && !(prof_ && prof_->enabled); }
  // Two-sided branch inside a stage or a custom adjoint: work issued between
  // branch_begin() and branch_switch() runs on the branch stream (forked from
  // the engine's stream, with its own split-K scratch), work issued between
  // branch_switch() and branch_join() on the engine's stream concurrently,
  // and branch_join() joins the two.  The two sides must not write the same
  // tensor (nor the same cotangent).  Everything stays on the engine's
  // stream when regions() is false or inside a concurrent region.
  void branch_begin();
  void branch_switch();
  void branch_join();
  void region_begin();
  void region_end();
  void region_join();
  // A second stream for independent work (created on first use; with a
  // caller-owned pool the engine's own stream is used instead), and the
  // points where it forks from and joins back into the engine's stream (also
  // valid during stream capture).
  cudaStream_t side_stream();
  void fork();
  void join();
  int prof_begin(cudaStream_t s) { return prof_ ? prof_->begin(s) : -1; }
  void prof_end(int k, cudaStream_t s, const char* name, double flops, double bytes) {
    if (prof_) prof_->end(k, s, name, flops, bytes);
  }
  void add_launches(int n) { launches_ += n; }

 private:
  Profiler* prof_ = nullptr;
  int pbegin() { return prof_ ? prof_->begin(stream_) : -1; }
  void pend(int k, const char* name, double flops, double bytes,
            const std::string& detail = std::string()) {
    if (prof_) prof_->end(k, stream_, name, flops, bytes, detail);
  }
  std::string cur_detail_;  // spec and extents of the operation being run (profiling)
  // Before writing into the gradient of dst.node: returns the accumulate flag
  // to use (false = overwrite when the write covers a gradient not yet set).
  bool begin_grad_write(const View& dst, bool accumulate);
  void zero_grad_if_unset(int node);
  enum OpKind { kContract, kAxpy, kMulc, kDiv, kCustom, kSym6, kSym6Div, kRegionBegin, kRegionEnd,
                kRegionJoin };
  struct Op {
    OpKind kind;
    std::string spec;
    double alpha;
    View a, b, c;
    EpsSpec es;
    bool tc = false;  // recorded inside the tensor-core region
    std::function<void()> fn;  // kCustom backward
  };
  bool cur_tc_ = false;  // tensor-core permission of the contraction being run
  void run_div(const View& X, bool xg, const EpsSpec& es, const View& Y, bool yg,
               bool overwrite = false);
  void run_combine(const View* xs, const bool* xg, const double* alphas, int ns, const View& Y,
                   bool yg, bool overwrite, const char* name);
  // run_combine (overwriting) for dense (..., v, v, v) operands whose
  // sources permute the last three indices, when the brick thread layout
  // touches fewer sectors; false: not that form, nothing launched
  bool run_combine_brick(const View* xs, const bool* xg, const double* alphas, int ns,
                         const View& Y, bool yg, bool overwrite, const char* name);
  void run_sym6(double alpha, const View& X, bool xg, const View& Y, bool yg, bool overwrite);
  void run_sym6_div(double alpha, const View& X, bool xg, const EpsSpec& es, const View& Y, bool yg,
                    bool overwrite, int np, const View* Y3 = nullptr);
  void run_contract(const std::string& spec, double alpha, const View& A, bool a_grad, const View& B,
                    bool b_grad, const View& Cv, bool c_grad, bool accumulate, long long sa = 0,
                    long long sb = 0, long long sc = 0);
  void run_axpy(double alpha, const View& X, bool xg, const View& Y, bool yg);
  void run_mulc(const View& X, bool xg, const View& Cst, const View& Y, bool yg);
  ContractPlan& plan(const std::string& spec, const View& A, const View& B, const View& Cv);

  cudaStream_t stream_;
  Arena arena_;
  std::vector<Node> nodes_;
  std::vector<Op> tape_;
  std::map<std::string, std::unique_ptr<ContractPlan>> plans_;
  static constexpr int kScratchSlots = 9;
  void* scratch_[kScratchSlots] = {};
  size_t scratch_bytes_[kScratchSlots] = {};
  // tensor-core scratch (packed A, packed B, split partials): slots 1-3 on
  // the engine's stream, 6-8 on the branch stream
  int tc_slot_ = 1;
  // split-K partials of CUDA-core contractions: slot 0 on the engine's
  // stream, slot 4 on the branch stream of the reverse pass, slot 5 in a
  // concurrent region
  int split_slot_ = 0;
  // concurrent region (region_begin / region_end / region_join)
  cudaStream_t region_ = nullptr, region_main_ = nullptr;
  cudaEvent_t region_fork_ = nullptr, region_join_ = nullptr;
  bool in_region_ = false, region_pending_ = false;
  void region_enter();
  void region_leave();
  // reverse pass: the two adjoints of one product (different outputs, same
  // inputs) run as parallel branches (a stream of their own, forked from and
  // joined into the engine's stream, also under graph capture)
  cudaStream_t branch_ = nullptr, branch_main_ = nullptr;
  cudaEvent_t branch_fork_ = nullptr, branch_join_ = nullptr;
  int branch_state_ = 0;  // 1: on the branch stream, 2: back on the engine's stream
  void ensure_branch_stream();
  bool branches_ = true;
  bool run_adjoints_branched(const Op& op);
  // reverse pass: gathers (adjoints of permuted sums) into one destination
  // view are held back and merged, up to kMaxSrc sources per pass, until the
  // destination's cotangent is read or the pass ends
  struct PendingGather {
    View dst;
    int ns = 0;
    View xs[kCombineSources];
    double al[kCombineSources];
  };
  std::vector<PendingGather> gathers_;
  void defer_gather(const View* xs, const double* al, int ns, const View& dst);
  void flush_gathers(int node);  // node < 0: all
  int tc_eb_ = 0;
  long long wait_budget_ = 0;
  bool checked_ = false;
  std::vector<unsigned char*> canaries_;
  void* canary_list_ = nullptr;
  size_t canary_list_bytes_ = 0;
  void check_view(const View& v, long long shift, const char* what) const;
  int eig_cap_ = 0;
  bool tc_region_ = false;
  int* err_ = nullptr;
  cudaStream_t side_ = nullptr;
  cudaEvent_t fork_ev_ = nullptr, join_ev_ = nullptr;
  DevicePool* pool_ = nullptr;
  void run_contract_small(ContractPlan& P, double alpha, const C* pa, const C* pb, C* pc,
                          bool accumulate);
  void run_contract_tc(ContractPlan& P, double alpha, const C* pa, const C* pb, C* pc,
                       bool accumulate);
  int launches_ = 0;
  int generation_ = 0;
  bool frozen_ = false;
};

// Small elementwise kernels used by the model and the integrator.
template <typename R>
void launch_fill(Cx<R>* p, size_t n, double re, double im, cudaStream_t s);

}  // namespace rtcc3
