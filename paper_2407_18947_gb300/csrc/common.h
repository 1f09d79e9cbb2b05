// Shared helpers for the RT-CC3 CUDA library: complex storage types, error
// propagation and the device arena.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

namespace rtcc3 {

// Complex numbers are interleaved (re, im) pairs: double2 / float2.
template <typename R> struct CxT;
template <> struct CxT<double> { using type = double2; };
template <> struct CxT<float> { using type = float2; };
template <typename R> using Cx = typename CxT<R>::type;

template <typename R> __host__ __device__ inline Cx<R> cmake(R re, R im) {
  Cx<R> z; z.x = re; z.y = im; return z;
}

// Error carried across the C ABI as a status code plus message.
struct Error : public std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

enum Status {
  kOk = 0, kErrArg = -1, kErrOom = -2, kErrCuda = -3, kErrNonfinite = -4,
  kErrTimeout = -5, kErrNotConverged = -6, kErrState = -7
};

#define RTCC3_CUDA(expr)                                                          \
  do {                                                                            \
    cudaError_t e__ = (expr);                                                     \
    if (e__ != cudaSuccess) {                                                     \
      throw ::rtcc3::Error(e__ == cudaErrorMemoryAllocation ? ::rtcc3::kErrOom    \
                                                            : ::rtcc3::kErrCuda,  \
                           std::string(#expr) + ": " + cudaGetErrorString(e__));  \
    }                                                                             \
  } while (0)

#define RTCC3_CHECK(cond, code, msg)                                              \
  do { if (!(cond)) throw ::rtcc3::Error((code), (msg)); } while (0)

// Optional per-kernel timing with CUDA events (eager launches only: CUDA
// graphs are not used while it is enabled).  Each launch is bracketed by an
// event pair on the launching stream; collect() synchronises and adds the
// elapsed times, the algorithmic flops and bytes per kernel name.
class Profiler {
 public:
  struct Stat { std::string name; long long launches = 0; double ms = 0.0, flops = 0.0, bytes = 0.0; };
  ~Profiler() { for (auto e : pool_) cudaEventDestroy(e); }
  bool enabled = false;
  int begin(cudaStream_t s) {
    if (!enabled) return -1;
    const int k = next_event();
    cudaEventRecord(pool_[k], s);
    return k;
  }
  void end(int k0, cudaStream_t s, const char* name, double flops, double bytes,
           const std::string& detail = std::string()) {
    if (k0 < 0) return;
    const int k1 = next_event();
    cudaEventRecord(pool_[k1], s);
    if (detail_ && !detail.empty())
      pending_.push_back({k0, k1, find((std::string(name) + "|" + detail).c_str()), flops, bytes});
    else
      pending_.push_back({k0, k1, find(name), flops, bytes});
  }
  // Per-operation names (kernel|spec) when the environment sets
  // RTCC3_PROFILE_DETAIL=1; used for tuning, not by the benchmark.
  void set_detail(bool d) { detail_ = d; }
  bool detail() const { return detail_; }
  void collect() {
    if (pending_.empty()) return;
    for (auto& p : pending_) cudaEventSynchronize(pool_[p.e1]);
    for (auto& p : pending_) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, pool_[p.e0], pool_[p.e1]);
      Stat& s = stats_[p.stat];
      s.launches += 1;
      s.ms += ms;
      s.flops += p.flops;
      s.bytes += p.bytes;
    }
    pending_.clear();
    used_ = 0;
  }
  void reset() { collect(); stats_.clear(); }
  const std::vector<Stat>& stats() const { return stats_; }

 private:
  struct Pending { int e0, e1, stat; double flops, bytes; };
  int next_event() {
    if (used_ == pool_.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool_.push_back(e);
    }
    return int(used_++);
  }
  int find(const char* name) {
    for (size_t i = 0; i < stats_.size(); ++i) if (stats_[i].name == name) return int(i);
    stats_.push_back(Stat());
    stats_.back().name = name;
    return int(stats_.size()) - 1;
  }
  std::vector<cudaEvent_t> pool_;
  size_t used_ = 0;
  bool detail_ = false;
  std::vector<Pending> pending_;
  std::vector<Stat> stats_;
};

// A fixed device region handed out by bumping a cursor; used instead of
// cudaMalloc by an engine that must not allocate (take() fails with
// kErrArg once the region is exhausted).
struct DevicePool {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  void* take(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    if (used + bytes > cap)
      throw Error(kErrArg, "workspace needs more than the " + std::to_string(cap >> 20) +
                               " MiB static scratch region");
    void* p = base + used;
    used += bytes;
    return p;
  }
};

// Bump allocator over device blocks.  Every evaluation of a residual graph
// requests the same sequence of sizes, so after reset() the same addresses are
// handed out again: buffers are stable across evaluations, which lets a whole
// RK4 step be captured once as a CUDA graph and replayed.
class Arena {
 public:
  ~Arena() { release(); }
  // Serve every request from `p` (no device allocation of its own).
  void use_pool(DevicePool* p) { pool_ = p; }
  void* alloc(size_t bytes) {
    if (pool_) return pool_->take(bytes);
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    while (true) {
      if (cur_ < blocks_.size()) {
        Block& b = blocks_[cur_];
        if (off_ + bytes <= b.size) {
          void* p = static_cast<char*>(b.ptr) + off_;
          off_ += bytes;
          used_ = std::max(used_, total_before(cur_) + off_);
          return p;
        }
        ++cur_;
        off_ = 0;
        continue;
      }
      size_t sz = std::max(bytes, size_t(256) << 20);
      void* p = nullptr;
      RTCC3_CUDA(cudaMalloc(&p, sz));
      blocks_.push_back({p, sz});
    }
  }
  void reset() { cur_ = 0; off_ = 0; }
  void release() {
    for (auto& b : blocks_) cudaFree(b.ptr);
    blocks_.clear();
    cur_ = 0; off_ = 0;
  }
  size_t reserved() const { size_t s = 0; for (auto& b : blocks_) s += b.size; return s; }
  size_t high_water() const { return used_; }

 private:
  DevicePool* pool_ = nullptr;
  struct Block { void* ptr; size_t size; };
  size_t total_before(size_t k) const { size_t s = 0; for (size_t i = 0; i < k; ++i) s += blocks_[i].size; return s; }
  std::vector<Block> blocks_;
  size_t cur_ = 0, off_ = 0, used_ = 0;
};

}  // namespace rtcc3
