// tcgen05 GEMMs for the complex contractions (see tc_gemm.h).
//
// k_tc_gemm: one CTA computes a 128 x BN tile of the real product Apack
// (M x Kp) times Bpack^T (Nr x Kp), both K-major, staged by TMA (128-byte
// swizzle) through a shared-memory ring.  Warp 0 issues the TMA loads, warp 1
// allocates tensor memory and issues tcgen05.mma (one elected thread), the
// epilogue warps first split each TF32 A tile into hi + lo parts in shared
// memory (the MMA warp then issues hi.hi, hi.lo and lo.hi) and afterwards
// read the FP32 accumulator back with tcgen05.ld and write the complex result
// (coalesced through a per-warp shared-memory transpose, 16 stores in flight
// per warp) or FP32 split-K partials.  Used for the short sums bound by their
// output.
//
// k_tc_gemm_direct (TF32 long sums) and k_tc_gemm_chains (BF16 long sums)
// cut the sum into accumulation chains and let one CTA stream several chains
// through two TMEM accumulators (one filled while the other is drained to its
// partial); the direct kernel gathers A from its source tensor with cp.async
// (no packed copy) and keeps A's TF32 hi/lo parts in tensor memory.
//
// Every mbarrier wait is bounded by a clock budget; on expiry the kernel
// raises *err and winds down, releasing its tensor memory.
#include "tc_gemm.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

namespace rtcc3 {

namespace {

constexpr int kBM = 128;
// Waits on other warps' progress spin for at most a budget of clock cycles
// (a kernel argument, kWaitBudget by default, about 2 s).  Waits for this
// CTA's own asynchronous work to land (its TMA / bulk copies, its MMAs) at
// exit use kDrainBudget: that work completes by itself, so these waits end
// whatever the progress budget was; they are what makes giving up safe
// (no copy or MMA may still target the CTA's shared or tensor memory when it
// frees them).
constexpr long long kWaitBudget = 4000000000LL;
constexpr long long kDrainBudget = 4000000000LL;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > budget) return false;
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// Contiguous global -> shared copy (16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}

// 8-byte asynchronous global -> shared copy; src_bytes 0 writes zeros.
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(src_bytes)
               : "memory");
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
               "l"(reinterpret_cast<uint64_t>(src))
               : "memory");
}

// Arrive on `bar` once this thread's earlier cp.async copies have landed (the
// arrival is one of the barrier's expected arrivals).
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t(1) << 16;                    // leading byte offset (unused for this layout)
  d |= uint64_t((1024 >> 4) & 0x3FFF) << 32;  // stride byte offset
  d |= uint64_t(1) << 46;                    // version
  d |= uint64_t(2) << 61;                    // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D = F32, A/B format (2 = TF32 for kind::tf32,
// 1 = BF16 for kind::f16), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <bool BF16>
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (uint32_t(BF16 ? 1 : 2) << 7) | (uint32_t(BF16 ? 1 : 2) << 10) |
         (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
  if (BF16) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  } else {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
  }
}

// D (+)= A B with A (128 rows = TMEM lanes, K = 8 TF32 columns) in tensor
// memory and B from shared memory.
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, "
      "%29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory plan of one CTA.  SPLIT (TF32 with a hi + lo split done in
// shared memory): A arrives as raw FP32 and a second A buffer takes the low
// parts; B arrives pre-split as [hi | lo] K halves.  EW epilogue warps: 8
// with a ring of up to four stages in 192 KB (one CTA per SM, long sums), or
// 4 with the ring in 80 KB (two CTAs per SM: one CTA's epilogue overlaps the
// other's main loop, for products bound by their output).
template <int BN, bool SPLIT, int EW>
struct TcSmem {
  // TMEM columns of the FP32 accumulator (an allocation is a power of two >= 32)
  static constexpr int kTmemCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  static constexpr int kABytes = kBM * 128;
  static constexpr int kALoBytes = SPLIT ? kBM * 128 : 0;
  static constexpr int kBBytes = BN * 128;
  static constexpr int kBLoBytes = SPLIT ? BN * 128 : 0;
  static constexpr int kStageBytes = kABytes + kALoBytes + kBBytes + kBLoBytes;
  static constexpr int kTmaBytes = kABytes + kBBytes + kBLoBytes;  // bytes the TMA delivers
  static constexpr int kRing = EW == 8 ? 196608 : 81920;
  static constexpr int kStages = kRing / kStageBytes < 4 ? kRing / kStageBytes : 4;
  static constexpr int kBarOff = kStages * kStageBytes;
  static constexpr int kStageOutOff = kBarOff + 256;
  static constexpr int kStageOutBytes = EW * 32 * 33 * 4;
  static constexpr int kTotal = kStageOutOff + kStageOutBytes + 1024;  // + alignment slack
  static constexpr int kThreads = 64 + 32 * EW;  // TMA warp, MMA warp, EW epilogue warps
  static_assert(kStages >= 1, "ring depth");
  static_assert(kTotal <= (EW == 8 ? 232448 : 116224), "shared memory per CTA");
};

template <int BN, bool BF16, bool SPLIT, int EW>
__global__ void __launch_bounds__(64 + 32 * EW, EW == 4 ? 2 : 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          int M, int Nr, int nkb_total, int kb_per_split, int kb_lo, float2* __restrict__ C,
          const long long* __restrict__ cM, const long long* __restrict__ cN, long long coff,
          float alpha, int accumulate, float* __restrict__ partial, int* __restrict__ err,
          long long budget) {
  using L = TcSmem<BN, SPLIT, EW>;
  constexpr int kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* conv = bars + 2 * kStages;  // SPLIT: low parts of A written
  uint64_t* done = bars + 3 * kStages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3 * kStages + 1);
  float* stage_out = reinterpret_cast<float*>(smem + L::kStageOutOff);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int split = blockIdx.z;
  const int kb0 = split * kb_per_split;
  const int nkb = max(0, min(nkb_total, kb0 + kb_per_split) - kb0);
  constexpr int kElemPerK = BF16 ? 64 : 32;  // elements per 128-byte K tile

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(smem_u32(&full[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
      mbar_init(smem_u32(&conv[s]), EW);  // one arrival per converter warp
    }
    mbar_init(smem_u32(done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(L::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nkb && ok; ++i) {
        const int s = i % kStages;
        if (i >= kStages) ok = mbar_wait(smem_u32(&empty[s]), ((i / kStages) - 1) & 1, budget);
        if (!ok) break;
        const uint32_t fb = smem_u32(&full[s]);
        mbar_expect_tx(fb, L::kTmaBytes);
        uint8_t* sa = smem + s * L::kStageBytes;
        uint8_t* sb = sa + L::kABytes + L::kALoBytes;
        const int kx = (kb0 + i) * kElemPerK;
        tma_load_2d(smem_u32(sa), &tmA, kx, m0, fb);
        tma_load_2d(smem_u32(sb), &tmB, kx, n0, fb);
        if (SPLIT) tma_load_2d(smem_u32(sb + L::kBBytes), &tmB, kx + kb_lo * kElemPerK, n0, fb);
        issued = i + 1;
      }
      // drain: every copy issued into this CTA's shared memory has landed
      // before it exits (the last ring round; earlier rounds were consumed
      // before their stage was reused), also after giving up
      for (int i = max(0, issued - kStages); i < issued; ++i)
        if (!mbar_wait(smem_u32(&full[i % kStages]), (i / kStages) & 1, kDrainBudget)) ok = false;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<BF16>(kBM, BN);
      for (int i = 0; i < nkb && ok; ++i) {
        const int s = i % kStages;
        ok = mbar_wait(smem_u32(SPLIT ? &conv[s] : &full[s]), (i / kStages) & 1, budget);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = smem_u32(smem + s * L::kStageBytes);
        const uint32_t sb = sa + L::kABytes + L::kALoBytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
          mma<BF16>(tmem, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), idesc, acc);
          if (SPLIT) {
            // hi.lo and lo.hi: the leading corrections of the split product
            mma<BF16>(tmem, smem_desc(sa + kk * 32), smem_desc(sb + L::kBBytes + kk * 32), idesc, 1u);
            mma<BF16>(tmem, smem_desc(sa + L::kABytes + kk * 32), smem_desc(sb + kk * 32), idesc, 1u);
          }
        }
        mma_commit(smem_u32(&empty[s]));
      }
      // committed also after giving up: `done` completes once every MMA
      // issued has, and nothing leaves before that
      mma_commit(smem_u32(done));
      if (!mbar_wait(smem_u32(done), 0, kDrainBudget)) ok = false;
    }
  } else {
    if (SPLIT) {
      // converters (warps 2..9) while the main loop runs: A tile -> TF32 hi in
      // place, the remainder x - hi into the low buffer (same offsets, so the
      // swizzled layout is kept), then a proxy fence for the tensor cores
      const int ct = threadIdx.x - 64;  // 0 .. 32 EW - 1
      for (int i = 0; i < nkb && ok; ++i) {
        const int s = i % kStages;
        ok = mbar_wait(smem_u32(&full[s]), (i / kStages) & 1, budget);
        if (!ok) break;
        float4* ah = reinterpret_cast<float4*>(smem + s * L::kStageBytes);
        float4* al = reinterpret_cast<float4*>(smem + s * L::kStageBytes + L::kABytes);
#pragma unroll
        for (int u = 0; u < L::kABytes / 16 / (32 * EW); ++u) {
          const int e = ct + 32 * EW * u;
          const float4 x = ah[e];
          float4 h, lo;
          h.x = __uint_as_float(to_tf32(x.x)); lo.x = x.x - h.x;
          h.y = __uint_as_float(to_tf32(x.y)); lo.y = x.y - h.y;
          h.z = __uint_as_float(to_tf32(x.z)); lo.z = x.z - h.z;
          h.w = __uint_as_float(to_tf32(x.w)); lo.w = x.w - h.w;
          ah[e] = h;
          al[e] = lo;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&conv[s]));
      }
    }
    // epilogue: warps 2 .. 1 + EW, EW / 4 per TMEM lane quarter (warp % 4),
    // taking every (EW / 4)-th 32-column chunk
    const int q = warp & 3, ew = warp - 2, half = ew >> 2;
    // the MMA warp always commits `done`: wait for it even after giving up
    const bool dn = (nkb == 0) ? true : mbar_wait(smem_u32(done), 0, kDrainBudget);
    ok = ok && dn;
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* st = stage_out + ew * 32 * 33;
    const int row = q * 32 + lane;
    const int m = m0 + row;
    // output row offsets of this warp's 32 rows, one per lane
    const long long cm_lane = (!partial && m < M) ? cM[m] : 0;
    for (int c0 = 32 * half; c0 < BN && ok; c0 += 32 * (EW / 4)) {
      uint32_t r[32];
      if (nkb > 0) {
        tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(c0), r);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) r[j] = 0u;
      }
      if (partial) {
        if (m < M) {
          float* dst = partial + (size_t(split) * M + m) * size_t(Nr) + n0 + c0;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (n0 + c0 + j < Nr) dst[j] = __uint_as_float(r[j]);
        }
        continue;
      }
      // transpose through shared memory so a warp stores runs of the output row
#pragma unroll
      for (int j = 0; j < 32; ++j) st[lane * 33 + j] = __uint_as_float(r[j]);
      __syncwarp();
      const int jc = lane & 15;   // complex column within the 16-column chunk
      const int rh = lane >> 4;   // row parity handled by this half-warp
      const int n = (n0 + c0) / 2 + jc;
      const bool ncol = (2 * n) < Nr;
      const long long cn = ncol ? cN[n] : 0;
      // all addresses and values first, then (for accumulation) all loads,
      // then all stores: the warp keeps 16 memory operations in flight
      long long idx[16];
      float2 val[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int rr = rh + 2 * u;
        const long long cmr = __shfl_sync(0xffffffffu, cm_lane, rr);
        const bool in = ncol && (m0 + q * 32 + rr < M);
        idx[u] = in ? coff + cmr + cn : -1;
        val[u] = make_float2(alpha * st[rr * 33 + 2 * jc], alpha * st[rr * 33 + 2 * jc + 1]);
      }
      if (accumulate) {
        float2 old[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) old[u] = idx[u] >= 0 ? C[idx[u]] : make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          val[u].x += old[u].x;
          val[u].y += old[u].y;
        }
      }
#pragma unroll
      for (int u = 0; u < 16; ++u)
        if (idx[u] >= 0) C[idx[u]] = val[u];
      __syncwarp();
    }
  }
  if (!ok && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::kTmemCols)
                 : "memory");
  }
}


// Shared-memory plan of the chained long-sum kernel: the same stage layout as
// TcSmem, a ring of up to 224 KB (no transpose staging), two accumulators.
// SPLIT: a stage holds the raw A tile and B [hi | lo]; the A tile's TF32 hi
// and lo parts go to tensor memory (the MMAs read A from there, so the three
// products of a K tile do not re-read A from shared memory).
template <int BN, bool SPLIT>
struct TcChainSmem {
  static constexpr int kABytes = kBM * 128;
  static constexpr int kBBytes = BN * 128;
  static constexpr int kStageBytes = kABytes + (SPLIT ? 2 : 1) * kBBytes;
  static constexpr int kRing = 229376;
  // two accumulators at columns 0 and kAccStride; SPLIT: A stages (64 TMEM
  // columns each: hi, lo) from column kACol, as many as the 512 columns hold
  static constexpr int kAccStride = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
  static constexpr int kACol = 2 * kAccStride;
  static constexpr int kMaxStages = SPLIT ? ((512 - kACol) / 64 < 6 ? (512 - kACol) / 64 : 6) : 6;
  static constexpr int kStages = kRing / kStageBytes < kMaxStages ? kRing / kStageBytes : kMaxStages;
  static constexpr int kBarOff = kStages * kStageBytes;
  static constexpr int kTotal = kBarOff + 256 + 1024;  // barriers + alignment slack
  static constexpr int kTmemCols = SPLIT ? 512 : (2 * kAccStride < 64 ? 64 : 2 * kAccStride);
  static_assert(!SPLIT || BN <= 128, "accumulators and A stages share 512 TMEM columns");
  static_assert(kStages >= 2 && kTotal <= 232448, "shared memory per CTA");
};

// Long sums split into accumulation chains of at most `per` K tiles (the
// FP32 accumulator's error grows with the chain).  One CTA streams the K
// tiles of `cpc` consecutive chains through its ring without draining the
// pipeline between them: the MMA warp alternates two TMEM accumulators and,
// while it fills one, four drain warps copy the other's finished chain to its
// FP32 partial (partial[(chain M + m) Nr + n], summed later by
// tc_split_finish).  A comes tiled (TcOperands::a_tiled) by bulk copies;
// with the TF32 split its hi and lo parts are staged in tensor memory, so the
// three products of a K tile read A from there instead of shared memory.
// Warps: 0 TMA, 1 MMA, 2-5 TF32 hi/lo split of A, 6-9 drain.  The chains and
// the products in each are those of the one-chain-per-CTA kernel.
template <int BN, bool BF16, bool SPLIT>
__global__ void __launch_bounds__(320, 1)
k_tc_gemm_chains(const uint8_t* __restrict__ Atiled, const __grid_constant__ CUtensorMap tmB,
                 int M, int Nr, int nkb_total, int per, int nchains, int cpc, int kb_lo,
                 float* __restrict__ partial, int* __restrict__ err, long long budget) {
  using L = TcChainSmem<BN, SPLIT>;
  constexpr int kStages = L::kStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint64_t* full = bars;
  uint64_t* empty = bars + kStages;
  uint64_t* conv = bars + 2 * kStages;   // SPLIT: low parts of A written
  uint64_t* cfull = bars + 3 * kStages;  // [2] accumulator holds a finished chain
  uint64_t* cfree = cfull + 2;           // [2] accumulator drained
  uint64_t* fin = cfree + 2;             // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int ch0 = blockIdx.z * cpc;
  const int nch = max(0, min(nchains, ch0 + cpc) - ch0);
  const int kb0 = ch0 * per;
  const int nkb = max(0, min(nkb_total, kb0 + nch * per) - kb0);
  constexpr int kElemPerK = BF16 ? 64 : 32;

  if (threadIdx.x == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(smem_u32(&full[st]), 1);
      mbar_init(smem_u32(&empty[st]), 1);
      mbar_init(smem_u32(&conv[st]), 4);  // one arrival per splitting warp
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&cfull[b]), 1);
      mbar_init(smem_u32(&cfree[b]), 4);  // one arrival per drain warp
    }
    mbar_init(smem_u32(fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(L::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nkb && ok; ++i) {
        const int st = i % kStages;
        if (i >= kStages) ok = mbar_wait(smem_u32(&empty[st]), ((i / kStages) - 1) & 1, budget);
        if (!ok) break;
        issued = i + 1;
        const uint32_t fb = smem_u32(&full[st]);
        mbar_expect_tx(fb, L::kStageBytes);
        uint8_t* sa = smem + st * L::kStageBytes;
        uint8_t* sb = sa + L::kABytes;
        const int kx = (kb0 + i) * kElemPerK;
        // A tile (row block blockIdx.y, K tile kb0 + i): one contiguous 16 KB
        // block already in its swizzled shared-memory image
        bulk_load(smem_u32(sa), Atiled + ((size_t(blockIdx.y) * nkb_total + kb0 + i) << 14),
                  L::kABytes, fb);
        tma_load_2d(smem_u32(sb), &tmB, kx, n0, fb);
        if (SPLIT) tma_load_2d(smem_u32(sb + L::kBBytes), &tmB, kx + kb_lo * kElemPerK, n0, fb);
      }
      // no copy into shared memory may be outstanding at exit (also after
      // giving up): the last ring round of copies has landed
      for (int i = max(0, issued - kStages); i < issued; ++i)
        if (!mbar_wait(smem_u32(&full[i % kStages]), (i / kStages) & 1, kDrainBudget)) ok = false;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<BF16>(kBM, BN);
      for (int i = 0; i < nkb && ok; ++i) {
        const int st = i % kStages, j = i / per, pos = i - j * per, b = j & 1;
        // the accumulator's previous chain (j - 2) must have been drained
        if (pos == 0 && j >= 2) ok = mbar_wait(smem_u32(&cfree[b]), ((j >> 1) - 1) & 1, budget);
        if (!ok) break;
        ok = mbar_wait(smem_u32(SPLIT ? &conv[st] : &full[st]), (i / kStages) & 1, budget);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_t = tmem + uint32_t(b * L::kAccStride);
        const uint32_t sa = smem_u32(smem + st * L::kStageBytes);
        const uint32_t sb = sa + L::kABytes;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc = (pos > 0 || kk > 0) ? 1u : 0u;
          if (SPLIT) {
            // A hi at columns kACol + 64 st, lo 32 columns further; 8 per K step
            const uint32_t ah = tmem + uint32_t(L::kACol + 64 * st + 8 * kk);
            mma_tf32_ta(acc_t, ah, smem_desc(sb + kk * 32), idesc, acc);
            mma_tf32_ta(acc_t, ah, smem_desc(sb + L::kBBytes + kk * 32), idesc, 1u);
            mma_tf32_ta(acc_t, ah + 32, smem_desc(sb + kk * 32), idesc, 1u);
          } else {
            mma<BF16>(acc_t, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), idesc, acc);
          }
        }
        mma_commit(smem_u32(&empty[st]));
        if (pos == per - 1 || i == nkb - 1) mma_commit(smem_u32(&cfull[b]));
      }
      // every MMA issued has completed before tensor memory is freed (also
      // after giving up)
      mma_commit(smem_u32(fin));
      if (!mbar_wait(smem_u32(fin), 0, kDrainBudget)) ok = false;
    }
  } else if (warp < 6) {
    if (SPLIT) {
      // warp % 4 owns TMEM lanes (A rows) 32 (warp % 4) .. + 31: each thread
      // reads its row's 32 FP32 values from the swizzled tile (16-byte chunk
      // c of row r sits at chunk c ^ (r % 8)) and stores hi = tf32(x) and
      // lo = x - hi to its TMEM lane
      const int r = 32 * (warp & 3) + lane;
      const uint32_t lane_base = uint32_t(32 * (warp & 3)) << 16;
      for (int i = 0; i < nkb && ok; ++i) {
        const int st = i % kStages;
        ok = mbar_wait(smem_u32(&full[st]), (i / kStages) & 1, budget);
        if (!ok) break;
        const float4* row = reinterpret_cast<const float4*>(smem + st * L::kStageBytes + r * 128);
        uint32_t hi[32], lo[32];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 x = row[c ^ (r & 7)];
          const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            hi[4 * c + e] = to_tf32(xv[e]);
            lo[4 * c + e] = __float_as_uint(xv[e] - __uint_as_float(hi[4 * c + e]));
          }
        }
        const uint32_t ta = tmem + lane_base + uint32_t(L::kACol + 64 * st);
        tmem_st32(ta, hi);
        tmem_st32(ta + 32, lo);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&conv[st]));
      }
    }
  } else {
    // drain warps 6-9: TMEM lane quarter warp % 4, all BN columns
    const int q = warp & 3;
    const int m = m0 + q * 32 + lane;
    const bool vec = (Nr & 3) == 0;
    for (int j = 0; j < nch && ok; ++j) {
      const int b = j & 1;
      ok = mbar_wait(smem_u32(&cfull[b]), (j >> 1) & 1, budget);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* dst = partial + (size_t(ch0 + j) * M + (m < M ? m : 0)) * size_t(Nr) + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(b * L::kAccStride + c0), r);
        if (m < M) {
          if (vec && n0 + c0 + 32 <= Nr) {
#pragma unroll
            for (int jj = 0; jj < 32; jj += 4)
              *reinterpret_cast<float4*>(dst + c0 + jj) =
                  make_float4(__uint_as_float(r[jj]), __uint_as_float(r[jj + 1]),
                              __uint_as_float(r[jj + 2]), __uint_as_float(r[jj + 3]));
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              if (n0 + c0 + jj < Nr) dst[c0 + jj] = __uint_as_float(r[jj]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&cfree[b]));
    }
  }
  if (!ok && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::kTmemCols)
                 : "memory");
  }
}

// One thread per complex source element: its (re, im) pair is written to
// every K segment (and, for B, to both rows of its 2x2 embedding) with one
// vector store each.  I is the index type of the flattened (row, k) loop.
template <int EB>
__device__ __forceinline__ void put_pair(void* out, size_t idx, float x, float y) {
  if (EB == 4) {
    *reinterpret_cast<uint2*>(static_cast<uint32_t*>(out) + idx) = make_uint2(to_tf32(x), to_tf32(y));
  } else {
    const uint32_t ux = __float_as_uint(x), uy = __float_as_uint(y);
    // round to nearest even on the upper 16 bits (finite inputs)
    const uint32_t rx = (ux + 0x7FFFu + ((ux >> 16) & 1u)) >> 16;
    const uint32_t ry = (uy + 0x7FFFu + ((uy >> 16) & 1u)) >> 16;
    *reinterpret_cast<uint32_t*>(static_cast<unsigned short*>(out) + idx) = rx | (ry << 16);
  }
}

// Packing runs on 32 x 32 (row, complex k) tiles staged in shared memory:
// the source is read with consecutive threads on its contiguous index (k when
// KFAST, else the row), the packed rows are written with consecutive threads
// along k.  B rows expand to the two rows of their 2x2 real embedding.
// TF32 (EB 4): A is written as raw FP32 (split into hi + lo in the GEMM's
// shared memory) and B as two K segments [hi | lo]; BF16 (EB 2): one
// segment, rounded to nearest even.
template <int EB, bool KFAST, bool IS_B, bool TILED>
__global__ void __launch_bounds__(256)
k_pack(const float2* __restrict__ X, const long long* __restrict__ xR, const long long* __restrict__ xK,
       long long xoff, int R, int K, int Kp, int segs, void* out) {
  __shared__ float2 tile[32][33];
  const int seg_w = Kp / segs, hw = seg_w >> 1;
  const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int a = w + 8 * u;
    const int rr = KFAST ? a : lane, kk = KFAST ? lane : a;
    const int r = r0 + rr, k = k0 + kk;
    tile[rr][kk] = (r < R && k < K) ? X[xoff + xR[r] + xK[k]] : make_float2(0.f, 0.f);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = w + 8 * u, r = r0 + rr, k = k0 + lane;
    if (r >= R || k >= hw) continue;
    const float2 v = tile[rr][lane];
    const size_t row = (IS_B ? size_t(2 * r) : size_t(r)) * Kp + 2 * size_t(k);
    if (TILED) {
      // tile (r / 128, kr / kpt) of 16 KB; row r % 128 at 128 bytes; its
      // 16-byte chunks permuted by the 128-byte swizzle (chunk ^ row % 8)
      constexpr int kpt = 128 / EB, epc = 16 / EB;
      const int kr = 2 * k, kt = kr / kpt, kc = kr % kpt, rr = r & 127;
      const size_t elem = ((size_t(r >> 7) * (Kp / kpt) + kt) << 14) / EB + size_t(rr) * kpt +
                          size_t(((kc / epc) ^ (rr & 7)) * epc + kc % epc);
      if (EB == 4) *reinterpret_cast<float2*>(static_cast<float*>(out) + elem) = v;  // raw FP32
      else put_pair<EB>(out, elem, v.x, v.y);
    } else if (!IS_B) {
      if (EB == 4) *reinterpret_cast<float2*>(static_cast<float*>(out) + row) = v;  // raw FP32
      else put_pair<EB>(out, row, v.x, v.y);
    } else {
      // row 2n: (Br, -Bi); row 2n+1: (Bi, Br) along (re, im) of K
      const size_t r1 = row + Kp;
      if (EB == 4) {
        const float hx = __uint_as_float(to_tf32(v.x)), hy = __uint_as_float(to_tf32(v.y));
        const float lx = v.x - hx, ly = v.y - hy;
        put_pair<EB>(out, row, hx, -hy);
        put_pair<EB>(out, r1, hy, hx);
        put_pair<EB>(out, row + seg_w, lx, -ly);
        put_pair<EB>(out, r1 + seg_w, ly, lx);
      } else {
        put_pair<EB>(out, row, v.x, -v.y);
        put_pair<EB>(out, r1, v.y, v.x);
      }
    }
  }
}

template <bool IS_B, bool TILED>
void launch_pack(const float2* X, const long long* xR, const long long* xK, long long xoff, int R,
                 int K, int Kp, int segs, int elem_bytes, bool kfast, void* out, cudaStream_t s) {
  const int hw = Kp / segs / 2;
  dim3 grid((hw + 31) / 32, (R + 31) / 32);
  RTCC3_CHECK(grid.y < 65536, kErrArg, "packed operand has too many rows");
#define RTCC3_PK(EBV, KF) k_pack<EBV, KF, IS_B, TILED><<<grid, 256, 0, s>>>(X, xR, xK, xoff, R, K, Kp, segs, out)
  if (elem_bytes == 4) {
    if (kfast) RTCC3_PK(4, true);
    else RTCC3_PK(4, false);
  } else {
    if (kfast) RTCC3_PK(2, true);
    else RTCC3_PK(2, false);
  }
#undef RTCC3_PK
  RTCC3_CUDA(cudaGetLastError());
}

__global__ void k_split_finish(const float* __restrict__ partial, int nsplit, int M, int N,
                               float2* __restrict__ C, const long long* __restrict__ cM,
                               const long long* __restrict__ cN, long long coff, float alpha,
                               int accumulate) {
  const size_t total = size_t(M) * N;
  const size_t plane = size_t(M) * 2 * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int n = int(t % N), m = int(t / N);
    float re = 0.f, im = 0.f;
    for (int s = 0; s < nsplit; ++s) {
      const float* p = partial + s * plane + size_t(m) * 2 * N + 2 * n;
      re += p[0];
      im += p[1];
    }
    const long long idx = coff + cM[m] + cN[n];
    float2 v = make_float2(alpha * re, alpha * im);
    if (accumulate) { v.x += C[idx].x; v.y += C[idx].y; }
    C[idx] = v;
  }
}

int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return int(std::max<size_t>(1, std::min<size_t>(g, 152 * 8)));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

bool make_map(CUtensorMap* map, const void* base, int elem_bytes, int Kp, int rows, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {cuuint64_t(Kp), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(Kp) * elem_bytes};
  const cuuint32_t box[2] = {cuuint32_t(128 / elem_bytes), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(map, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                        2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int BN, bool BF16, bool SPLIT, int EW>
void launch(const CUtensorMap& ma, const CUtensorMap& mb, const TcOperands& op, float2* C,
            const long long* cM, const long long* cN, long long coff, float alpha, bool accumulate,
            int nsplit, float* partial, int* err, cudaStream_t s) {
  using L = TcSmem<BN, SPLIT, EW>;
  static bool attr = false;
  if (!attr) {
    RTCC3_CUDA(cudaFuncSetAttribute(k_tc_gemm<BN, BF16, SPLIT, EW>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal));
    attr = true;
  }
  const int Nr = 2 * op.N;
  const int nkb = op.Kp / (128 / op.elem_bytes);
  const int per = (nkb + nsplit - 1) / nsplit;
  dim3 grid((Nr + BN - 1) / BN, (op.M + kBM - 1) / kBM, nsplit);
  k_tc_gemm<BN, BF16, SPLIT, EW><<<grid, L::kThreads, L::kTotal, s>>>(
      ma, mb, op.M, Nr, nkb, per, nkb, C, cM, cN, coff, alpha, accumulate ? 1 : 0,
      nsplit > 1 ? partial : nullptr, err, op.wait_budget > 0 ? op.wait_budget : kWaitBudget);
  RTCC3_CUDA(cudaGetLastError());
}

// Chains per CTA for `tiles` output tiles and `nchains` chains: the fewest
// CTAs per tile that fill whole waves of one CTA per SM to 90 % (else the
// best fill).
int chains_per_cta(long long tiles, int nchains) {
  int z = 1;
  double best = 0.0;
  for (int c = 1; c <= nchains; ++c) {
    const long long ctas = tiles * c;
    const double eff = double(ctas) / double(((ctas + 151) / 152) * 152);
    if (eff > best + 1e-9) {
      best = eff;
      z = c;
    }
    if (eff >= 0.9) break;
  }
  return (nchains + z - 1) / z;
}

// Shared-memory plan of the direct long-sum kernel: an A ring (raw FP32
// tiles gathered by cp.async, freed once split into TMEM) and a B ring
// ([hi | lo] by TMA, freed by the MMA commit) whose depth is the number of
// TMEM A stages.
template <int BN>
struct TcDirectSmem {
  static constexpr int kABytes = kBM * 128;
  static constexpr int kBStage = 2 * BN * 128;
  static constexpr int kAccStride = BN <= 32 ? 32 : (BN <= 64 ? 64 : 128);
  static constexpr int kACol = 2 * kAccStride;
  static constexpr int kBStages = (512 - kACol) / 64 < 6 ? (512 - kACol) / 64 : 6;
  static constexpr int kRing = 229376;
  static constexpr int kAStages0 = (kRing - kBStages * kBStage) / kABytes;
  static constexpr int kAStages = kAStages0 < 8 ? kAStages0 : 8;
  static constexpr int kBOff = kAStages * kABytes;
  static constexpr int kBarOff = kBOff + kBStages * kBStage;
  static constexpr int kTotal = kBarOff + 512 + 1024;  // barriers + alignment slack
  static_assert(BN <= 128 && kAStages >= 2 && kBStages >= 2 && kTotal <= 232448, "plan");
};

// The chained long sum with A read straight from its source tensor through
// its offset tables (TF32 split): no packed copy of the big operand is
// written.  Warps 2-9 gather the 128 x 16 complex A tile of each K tile with
// 8-byte cp.async copies into a shared-memory ring (zeros outside M and K),
// consecutive threads on the source's contiguous index (a_kc: along k, else
// along rows), in the swizzled row layout; warps 10-13 split each tile into
// TF32 hi and lo in tensor memory; warp 0 brings B by TMA, warp 1 issues the
// MMAs (A from TMEM), warps 14-17 drain the accumulators to the chain
// partials as in k_tc_gemm_chains.
template <int BN, bool AKC>
__global__ void __launch_bounds__(576, 1)
k_tc_gemm_direct(const float2* __restrict__ A, long long aoff, const long long* __restrict__ aM,
                 const long long* __restrict__ aK, int K, const __grid_constant__ CUtensorMap tmB,
                 int M, int Nr, int nkb_total, int per, int nchains, int cpc,
                 float* __restrict__ partial, int* __restrict__ err, long long budget) {
  using L = TcDirectSmem<BN>;
  constexpr int SA = L::kAStages, SB = L::kBStages;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L::kBarOff);
  uint64_t* afull = bars;            // [SA] A tile landed (256 loader threads)
  uint64_t* aempty = afull + SA;     // [SA] A tile split into TMEM (4 warps)
  uint64_t* bfull = aempty + SA;     // [SB] B tile landed (TMA)
  uint64_t* empty = bfull + SB;      // [SB] MMAs of the stage done (commit)
  uint64_t* conv = empty + SB;       // [SB] TMEM A stage written (4 warps)
  uint64_t* cfull = conv + SB;       // [2] accumulator holds a finished chain
  uint64_t* cfree = cfull + 2;       // [2] accumulator drained
  uint64_t* fin = cfree + 2;         // every MMA issued has completed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
  const int ch0 = blockIdx.z * cpc;
  const int nch = max(0, min(nchains, ch0 + cpc) - ch0);
  const int kb0 = ch0 * per;
  const int nkb = max(0, min(nkb_total, kb0 + nch * per) - kb0);

  if (threadIdx.x == 0) {
    for (int st = 0; st < SA; ++st) {
      mbar_init(smem_u32(&afull[st]), 256);
      mbar_init(smem_u32(&aempty[st]), 4);
    }
    for (int st = 0; st < SB; ++st) {
      mbar_init(smem_u32(&bfull[st]), 1);
      mbar_init(smem_u32(&empty[st]), 1);
      mbar_init(smem_u32(&conv[st]), 4);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&cfull[b]), 1);
      mbar_init(smem_u32(&cfree[b]), 4);
    }
    mbar_init(smem_u32(fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  bool ok = true;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int i = 0; i < nkb && ok; ++i) {
        const int st = i % SB;
        if (i >= SB) ok = mbar_wait(smem_u32(&empty[st]), ((i / SB) - 1) & 1, budget);
        if (!ok) break;
        issued = i + 1;
        const uint32_t fb = smem_u32(&bfull[st]);
        mbar_expect_tx(fb, L::kBStage);
        const uint32_t sb = smem_u32(smem + L::kBOff + st * L::kBStage);
        const int kx = (kb0 + i) * 32;
        tma_load_2d(sb, &tmB, kx, n0, fb);
        tma_load_2d(sb + BN * 128, &tmB, kx + nkb_total * 32, n0, fb);
      }
      // the last ring round of B copies has landed (also after giving up)
      for (int i = max(0, issued - SB); i < issued; ++i)
        if (!mbar_wait(smem_u32(&bfull[i % SB]), (i / SB) & 1, kDrainBudget)) ok = false;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = instr_desc<false>(kBM, BN);
      for (int i = 0; i < nkb && ok; ++i) {
        const int st = i % SB, j = i / per, pos = i - j * per, b = j & 1;
        if (pos == 0 && j >= 2) ok = mbar_wait(smem_u32(&cfree[b]), ((j >> 1) - 1) & 1, budget);
        if (ok) ok = mbar_wait(smem_u32(&conv[st]), (i / SB) & 1, budget);
        if (ok) ok = mbar_wait(smem_u32(&bfull[st]), (i / SB) & 1, budget);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc_t = tmem + uint32_t(b * L::kAccStride);
        const uint32_t sb = smem_u32(smem + L::kBOff + st * L::kBStage);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint32_t acc = (pos > 0 || kk > 0) ? 1u : 0u;
          const uint32_t ah = tmem + uint32_t(L::kACol + 64 * st + 8 * kk);
          mma_tf32_ta(acc_t, ah, smem_desc(sb + kk * 32), idesc, acc);
          mma_tf32_ta(acc_t, ah, smem_desc(sb + BN * 128 + kk * 32), idesc, 1u);
          mma_tf32_ta(acc_t, ah + 32, smem_desc(sb + kk * 32), idesc, 1u);
        }
        mma_commit(smem_u32(&empty[st]));
        if (pos == per - 1 || i == nkb - 1) mma_commit(smem_u32(&cfull[b]));
      }
      // every MMA issued has completed before tensor memory is freed (also
      // after giving up)
      mma_commit(smem_u32(fin));
      if (!mbar_wait(smem_u32(fin), 0, kDrainBudget)) ok = false;
    }
  } else if (warp < 10) {
    // loaders.  AKC: pairs of consecutive k, pair p = t + 256 u (u < 4),
    // k pair (p % 8) (constant per thread), row p / 8, one 16-byte copy when
    // the pair is contiguous and aligned in the source; else element
    // e = t + 256 u (u < 8), row e % 128 (constant), j = e / 128
    const int t = threadIdx.x - 64;
    constexpr int NU = AKC ? 4 : 8;
    long long rowoff[NU];
    bool rowok[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int r = AKC ? (t >> 3) + 32 * u : (t & 127);
      const int m = m0 + r;
      rowok[u] = m < M;
      rowoff[u] = rowok[u] ? aoff + aM[m] : 0;
    }
    for (int i = 0; i < nkb && ok; ++i) {
      const int st = i % SA;
      if (i >= SA) ok = mbar_wait(smem_u32(&aempty[st]), ((i / SA) - 1) & 1, budget);
      if (!ok) break;
      const uint32_t sa = smem_u32(smem + st * L::kABytes);
      const int kbase = (kb0 + i) * 16;
      if (AKC) {
        const int j2 = t & 7, k = kbase + 2 * j2;
        const bool k0in = k < K, k1in = k + 1 < K;
        const long long o0 = k0in ? aK[k] : 0, o1 = k1in ? aK[k + 1] : 0;
        const bool pair = k1in && o1 == o0 + 1;
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int r = (t >> 3) + 32 * u;
          // floats 4 j2 .. 4 j2 + 3 of row r: 16-byte chunk j2 at j2 ^ (r % 8)
          const uint32_t dst = sa + uint32_t(r * 128 + ((j2 ^ (r & 7)) << 4));
          const long long a0 = rowoff[u] + o0;
          if (rowok[u] && pair && (reinterpret_cast<uintptr_t>(A + a0) & 15) == 0) {
            cp_async16(dst, A + a0);
          } else {
            const bool in0 = rowok[u] && k0in, in1 = rowok[u] && k1in;
            cp_async8(dst, in0 ? A + a0 : A, in0 ? 8u : 0u);
            cp_async8(dst + 8, in1 ? A + rowoff[u] + o1 : A, in1 ? 8u : 0u);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < NU; ++u) {
          const int r = t & 127;
          const int j = (t >> 7) + 2 * u;
          const int k = kbase + j;
          const bool in = rowok[u] && k < K;
          const float2* src = in ? A + rowoff[u] + aK[k] : A;
          // float 2j of row r: 16-byte chunk j / 2 at position (j / 2) ^ (r % 8)
          const uint32_t dst = sa + uint32_t(r * 128 + ((((j >> 1) ^ (r & 7)) << 4) | ((j & 1) << 3)));
          cp_async8(dst, src, in ? 8u : 0u);
        }
      }
      cp_async_arrive(smem_u32(&afull[st]));
    }
    // no copy may be outstanding at exit
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp < 14) {
    // splitters: TMEM lanes 32 (warp % 4) .. + 31 = rows of the A tile
    const int r = 32 * (warp & 3) + lane;
    const uint32_t lane_base = uint32_t(32 * (warp & 3)) << 16;
    for (int i = 0; i < nkb && ok; ++i) {
      const int sa_i = i % SA, st = i % SB;
      ok = mbar_wait(smem_u32(&afull[sa_i]), (i / SA) & 1, budget);
      // the TMEM stage's previous MMAs (K tile i - SB) must be done
      if (ok && i >= SB) ok = mbar_wait(smem_u32(&empty[st]), ((i / SB) - 1) & 1, budget);
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.st below is warp-collective
      if (!ok) break;
      const float4* row = reinterpret_cast<const float4*>(smem + sa_i * L::kABytes + r * 128);
      uint32_t hi[32], lo[32];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 x = row[c ^ (r & 7)];
        const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          hi[4 * c + e] = to_tf32(xv[e]);
          lo[4 * c + e] = __float_as_uint(xv[e] - __uint_as_float(hi[4 * c + e]));
        }
      }
      const uint32_t ta = tmem + lane_base + uint32_t(L::kACol + 64 * st);
      tmem_st32(ta, hi);
      tmem_st32(ta + 32, lo);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(smem_u32(&aempty[sa_i]));
        mbar_arrive(smem_u32(&conv[st]));
      }
    }
  } else {
    // drain warps 14-17: TMEM lane quarter warp % 4, all BN columns
    const int q = warp & 3;
    const int m = m0 + q * 32 + lane;
    const bool vec = (Nr & 3) == 0;
    for (int j = 0; j < nch && ok; ++j) {
      const int b = j & 1;
      ok = mbar_wait(smem_u32(&cfull[b]), (j >> 1) & 1, budget);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* dst = partial + (size_t(ch0 + j) * M + (m < M ? m : 0)) * size_t(Nr) + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(tmem + (uint32_t(q * 32) << 16) + uint32_t(b * L::kAccStride + c0), r);
        if (m < M) {
          if (vec && n0 + c0 + 32 <= Nr) {
#pragma unroll
            for (int jj = 0; jj < 32; jj += 4)
              *reinterpret_cast<float4*>(dst + c0 + jj) =
                  make_float4(__uint_as_float(r[jj]), __uint_as_float(r[jj + 1]),
                              __uint_as_float(r[jj + 2]), __uint_as_float(r[jj + 3]));
          } else {
#pragma unroll
            for (int jj = 0; jj < 32; ++jj)
              if (n0 + c0 + jj < Nr) dst[c0 + jj] = __uint_as_float(r[jj]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&cfree[b]));
    }
  }
  if (!ok && err) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

template <int BN>
void launch_direct(const float2* A, long long aoff, const long long* aM, const long long* aK,
                   bool a_kc, const CUtensorMap& mb, const TcOperands& op, int nsplit,
                   float* partial, int* err, cudaStream_t s) {
  using L = TcDirectSmem<BN>;
  const int Nr = 2 * op.N;
  const int nkb = op.Kp / 32;
  const int per = (nkb + nsplit - 1) / nsplit;
  const int nchains = (nkb + per - 1) / per;
  static bool attr = false;
  if (!attr) {
    RTCC3_CUDA(cudaFuncSetAttribute(k_tc_gemm_direct<BN, true>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal));
    RTCC3_CUDA(cudaFuncSetAttribute(k_tc_gemm_direct<BN, false>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal));
    attr = true;
  }
  const long long tiles = (long long)((Nr + BN - 1) / BN) * ((op.M + kBM - 1) / kBM);
  const int cpc = chains_per_cta(tiles, nchains);
  const int zz = (nchains + cpc - 1) / cpc;
  dim3 grid((Nr + BN - 1) / BN, (op.M + kBM - 1) / kBM, zz);
  const long long budget = op.wait_budget > 0 ? op.wait_budget : kWaitBudget;
  if (a_kc)
    k_tc_gemm_direct<BN, true><<<grid, 576, L::kTotal, s>>>(A, aoff, aM, aK, op.K, mb, op.M, Nr,
                                                            nkb, per, nchains, cpc, partial, err,
                                                            budget);
  else
    k_tc_gemm_direct<BN, false><<<grid, 576, L::kTotal, s>>>(A, aoff, aM, aK, op.K, mb, op.M, Nr,
                                                             nkb, per, nchains, cpc, partial, err,
                                                             budget);
  RTCC3_CUDA(cudaGetLastError());
}

// Chained long-sum launch (see k_tc_gemm_chains); false if the split does
// not map onto whole chains.
template <int BN, bool BF16, bool SPLIT>
bool launch_chains(const void* Atiled, const CUtensorMap& mb, const TcOperands& op, int nsplit,
                   float* partial, int* err, cudaStream_t s) {
  using L = TcChainSmem<BN, SPLIT>;
  const int Nr = 2 * op.N;
  const int nkb = op.Kp / (128 / op.elem_bytes);
  const int per = (nkb + nsplit - 1) / nsplit;
  const int nchains = (nkb + per - 1) / per;
  if (nchains != nsplit) return false;  // every partial slice must be written
  static bool attr = false;
  if (!attr) {
    RTCC3_CUDA(cudaFuncSetAttribute(k_tc_gemm_chains<BN, BF16, SPLIT>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, L::kTotal));
    attr = true;
  }
  const long long tiles = (long long)((Nr + BN - 1) / BN) * ((op.M + kBM - 1) / kBM);
  const int cpc = chains_per_cta(tiles, nchains);
  const int zz = (nchains + cpc - 1) / cpc;
  dim3 grid((Nr + BN - 1) / BN, (op.M + kBM - 1) / kBM, zz);
  k_tc_gemm_chains<BN, BF16, SPLIT><<<grid, 320, L::kTotal, s>>>(
      static_cast<const uint8_t*>(Atiled), mb, op.M, Nr, nkb, per, nchains, cpc, nkb, partial, err,
      op.wait_budget > 0 ? op.wait_budget : kWaitBudget);
  RTCC3_CUDA(cudaGetLastError());
  return true;
}

// ---- pipe-rate probes (roofline denominators) -------------------------------
// Tensor pipe: one CTA per SM issues `iters` K tiles of a 128 x 256 MMA (four
// 32-byte K steps per tile: K = 32 TF32 or 64 BF16 elements) from zeroed
// shared-memory tiles into one TMEM accumulator: no global traffic, the
// issue rate of dense tcgen05 MMAs.  The kernel waits (drain budget) for its
// MMAs before freeing tensor memory.
template <bool BF16>
__global__ void __launch_bounds__(128, 1) k_mma_rate(int iters, int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kA = 128 * 128, kB = 256 * 128;
  uint64_t* fin = reinterpret_cast<uint64_t*>(smem + kA + kB);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(fin + 1);
  for (int t = threadIdx.x; t < (kA + kB) / 16; t += blockDim.x)
    reinterpret_cast<uint4*>(smem)[t] = make_uint4(0u, 0u, 0u, 0u);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(fin), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)), "r"(256) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = instr_desc<BF16>(128, 256);
    const uint32_t sa = smem_u32(smem), sb = sa + kA;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)
        mma<BF16>(tmem, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), idesc, (i | kk) ? 1u : 0u);
    }
    mma_commit(smem_u32(fin));
    if (!mbar_wait(smem_u32(fin), 0, kDrainBudget) && err) atomicExch(err, 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                 : "memory");
  }
}

// CUDA-core FMA pipes: eight independent multiply-add chains per thread.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_rate(T* __restrict__ sink, int iters) {
  T a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = T(threadIdx.x + j) * T(1e-3);
  const T b = T(0.999999), c = T(1e-7);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  T sum = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) sum += a[j];
  if (sum == T(-1)) sink[0] = sum;  // never true; keeps the chains alive
}

}  // namespace

// Measured dense rate (TFLOP/s) of one pipe on the current device: 0 TF32
// tcgen05 MMA, 1 BF16 tcgen05 MMA, 2 FP32 FMA, 3 FP64 FMA.  One untimed
// launch, then one launch timed with CUDA events.
double measure_pipe_tflops(int which, int* err_flag, cudaStream_t s) {
  int dev = 0, sms = 0;
  RTCC3_CUDA(cudaGetDevice(&dev));
  RTCC3_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaEvent_t e0, e1;
  RTCC3_CUDA(cudaEventCreate(&e0));
  RTCC3_CUDA(cudaEventCreate(&e1));
  double flops = 0.0;
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    RTCC3_CUDA(cudaEventRecord(e0, s));
    if (which <= 1) {
      const int iters = 4096;
      const int smem = 128 * 128 + 256 * 128 + 64 + 1024;
      if (which == 0) {
        RTCC3_CUDA(cudaFuncSetAttribute(k_mma_rate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_mma_rate<false><<<sms, 128, smem, s>>>(iters, err_flag);
      } else {
        RTCC3_CUDA(cudaFuncSetAttribute(k_mma_rate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        k_mma_rate<true><<<sms, 128, smem, s>>>(iters, err_flag);
      }
      const double k = which == 0 ? 32.0 : 64.0;  // K elements per tile
      flops = 2.0 * 128.0 * 256.0 * k * iters * sms;
    } else {
      const int iters = which == 2 ? 8192 : 1024;
      const int blocks = sms * 8;
      if (which == 2) k_fma_rate<float><<<blocks, 256, 0, s>>>(nullptr, iters);
      else k_fma_rate<double><<<blocks, 256, 0, s>>>(nullptr, iters);
      flops = 2.0 * 8.0 * iters * 256.0 * blocks;
    }
    RTCC3_CUDA(cudaGetLastError());
    RTCC3_CUDA(cudaEventRecord(e1, s));
    RTCC3_CUDA(cudaEventSynchronize(e1));
    RTCC3_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return flops / (double(ms) * 1e-3) / 1e12;
}

void tc_pack_a(const float2* A, const long long* aM, const long long* aK, long long aoff, int M,
               int K, int Kp, int elem_bytes, bool kfast, bool tiled, void* out, cudaStream_t s) {
  if (tiled) launch_pack<false, true>(A, aM, aK, aoff, M, K, Kp, 1, elem_bytes, kfast, out, s);
  else launch_pack<false, false>(A, aM, aK, aoff, M, K, Kp, 1, elem_bytes, kfast, out, s);
}

void tc_pack_b(const float2* B, const long long* bN, const long long* bK, long long boff, int N,
               int K, int Kp, int elem_bytes, bool kfast, void* out, cudaStream_t s) {
  const int segs = elem_bytes == 4 ? 2 : 1;
  launch_pack<true, false>(B, bN, bK, boff, N, K, segs * Kp, segs, elem_bytes, kfast, out, s);
}

bool tc_gemm(const void* Apack, const void* Bpack, const TcOperands& op, float2* C,
             const long long* cM, const long long* cN, long long coff, float alpha, bool accumulate,
             int nsplit, float* partial, int* err_flag, cudaStream_t s) {
  const int Nr = 2 * op.N;
  if (op.M <= 0 || op.N <= 0 || op.Kp <= 0) return false;
  if (op.Kp % (128 / op.elem_bytes) != 0) return false;
  const int BN = tc_tile_n(Nr, op.out_bound);
  CUtensorMap ma, mb;
  if (!op.a_tiled && !make_map(&ma, Apack, op.elem_bytes, op.Kp, op.M, kBM)) return false;
  if (!make_map(&mb, Bpack, op.elem_bytes, op.split ? 2 * op.Kp : op.Kp, Nr, BN)) return false;
  const bool bf16 = op.elem_bytes == 2;
  RTCC3_CHECK(bf16 || op.split, kErrArg, "TF32 operands are split in the GEMM (pack B as hi | lo)");
#define RTCC3_TC(BNV, EWV)                                                                        \
  (bf16 ? launch<BNV, true, false, EWV>(ma, mb, op, C, cM, cN, coff, alpha, accumulate, nsplit, partial, err_flag, s) \
        : launch<BNV, false, true, EWV>(ma, mb, op, C, cM, cN, coff, alpha, accumulate, nsplit, partial, err_flag, s))
#define RTCC3_CH(BNV)                                                                     \
  (bf16 ? launch_chains<BNV, true, false>(Apack, mb, op, nsplit, partial, err_flag, s)     \
        : launch_chains<BNV, false, true>(Apack, mb, op, nsplit, partial, err_flag, s))
  if (op.a_tiled) {
    RTCC3_CHECK(tc_chained(op, nsplit) && partial, kErrArg,
                "tiled A is for chained long sums with split partials");
    bool launched = false;
    if (BN == 128) launched = RTCC3_CH(128);
    else if (BN == 96) launched = RTCC3_CH(96);
    else if (BN == 64) launched = RTCC3_CH(64);
    else if (BN == 32) launched = RTCC3_CH(32);
    RTCC3_CHECK(launched, kErrArg, "chained long sum: unsupported tile");
  } else if (op.out_bound) {
    if (BN == 128) RTCC3_TC(128, 4);
    else RTCC3_TC(64, 4);
  } else {
    if (BN == 256) RTCC3_TC(256, 8);
    else if (BN == 128) RTCC3_TC(128, 8);
    else if (BN == 96) RTCC3_TC(96, 8);
    else if (BN == 64) RTCC3_TC(64, 8);
    else RTCC3_TC(32, 8);
  }
#undef RTCC3_TC
#undef RTCC3_CH
  return true;
}

bool tc_gemm_direct(const float2* A, long long aoff, const long long* aM, const long long* aK,
                    bool a_kc, const void* Bpack, const TcOperands& op, int nsplit, float* partial,
                    int* err_flag, cudaStream_t s) {
  RTCC3_CHECK(tc_direct(op, nsplit) && partial, kErrArg, "direct long sum: unsupported shape");
  const int Nr = 2 * op.N;
  const int BN = tc_tile_n(Nr, false);
  CUtensorMap mb;
  if (!make_map(&mb, Bpack, 4, 2 * op.Kp, Nr, BN)) return false;
  if (BN == 128) launch_direct<128>(A, aoff, aM, aK, a_kc, mb, op, nsplit, partial, err_flag, s);
  else if (BN == 96) launch_direct<96>(A, aoff, aM, aK, a_kc, mb, op, nsplit, partial, err_flag, s);
  else if (BN == 64) launch_direct<64>(A, aoff, aM, aK, a_kc, mb, op, nsplit, partial, err_flag, s);
  else launch_direct<32>(A, aoff, aM, aK, a_kc, mb, op, nsplit, partial, err_flag, s);
  return true;
}

void tc_split_finish(const float* partial, int nsplit, int M, int N, float2* C, const long long* cM,
                     const long long* cN, long long coff, float alpha, bool accumulate,
                     cudaStream_t s) {
  k_split_finish<<<grid_for(size_t(M) * N), 256, 0, s>>>(partial, nsplit, M, N, C, cM, cN, coff,
                                                          alpha, accumulate ? 1 : 0);
  RTCC3_CUDA(cudaGetLastError());
}

}  // namespace rtcc3
