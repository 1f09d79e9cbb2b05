// Small-output and single-column contractions (see contract_small.h).
#include "contract_small.h"

#include <algorithm>

namespace rtcc3 {

namespace {

constexpr int kThreads = 256;

template <typename R>
__device__ __forceinline__ void cfma(R& ar, R& ai, Cx<R> a, Cx<R> b) {
  ar = fma(a.x, b.x, ar);
  ar = fma(-a.y, b.y, ar);
  ai = fma(a.x, b.y, ai);
  ai = fma(a.y, b.x, ai);
}

// RM x RN threads own UM x UN outputs each (rows rm + RM i, columns rn + RN j);
// the remaining G = 256 / (RM RN) thread groups take interleaved k of every
// slice and are summed in a fixed order at the end.
template <typename R, int RM, int RN, int UM, int UN>
struct SmallShape {
  static constexpr int MP = RM * UM, NP = RN * UN, G = kThreads / (RM * RN);
  static constexpr int EB = int(sizeof(Cx<R>));
  static constexpr int BK0 = 40960 / ((MP + NP + 2) * EB);
  // deep slices keep more loads in flight per thread (128 for the 16 x 16 tile)
  static constexpr int BK = BK0 >= 128 ? 128 : (BK0 >= 64 ? 64 : (BK0 >= 32 ? 32 : (BK0 >= 16 ? 16 : (BK0 >= 8 ? 8 : 4))));
  // thread groups sharing a warp (summed by shuffles) and the rest (by shared memory)
  static constexpr int WG = RM * RN >= 32 ? 1 : 32 / (RM * RN);
  static constexpr int GS = G / WG;
  // slices are stored [k][m] with an odd row pitch so that the transposing
  // stores of K-contiguous loads do not hit one bank
  static constexpr int MS = MP + 1, NS = NP + 1;
  static constexpr int TILE_BYTES = BK * (MS + NS) * EB;
  static constexpr int RED_BYTES = GS > 1 ? MP * NP * EB : 0;
  static constexpr int SMEM = TILE_BYTES > RED_BYTES ? TILE_BYTES : RED_BYTES;
  static_assert(G >= 1 && BK >= G, "slice shallower than the thread groups");
  static_assert(SMEM <= 48 * 1024, "static shared memory");
};

template <typename R, bool A_KC, bool B_KC, int RM, int RN, int UM, int UN>
__global__ void __launch_bounds__(kThreads)
k_reduce_small(const Cx<R>* __restrict__ A, long long aoff, const long long* __restrict__ aM,
               const long long* __restrict__ aK, const Cx<R>* __restrict__ B, long long boff,
               const long long* __restrict__ bN, const long long* __restrict__ bK,
               Cx<R>* __restrict__ Cp, long long coff, const long long* __restrict__ cM,
               const long long* __restrict__ cN, int M, int N, int K, int kchunk, R alpha,
               int accumulate, Cx<R>* __restrict__ part) {
  using S = SmallShape<R, RM, RN, UM, UN>;
  constexpr int MP = S::MP, NP = S::NP, G = S::G, BK = S::BK;
  __shared__ __align__(16) unsigned char smem[S::SMEM];
  constexpr int MS = S::MS, NS = S::NS;
  Cx<R>* As = reinterpret_cast<Cx<R>*>(smem);  // [BK][MS]
  Cx<R>* Bs = As + BK * MS;                      // [BK][NS]
  const int tid = threadIdx.x;
  const int rn = tid % RN, rm = (tid / RN) % RM, g = tid / (RM * RN);
  const int split = blockIdx.x;
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  R accr[UM][UN], acci[UM][UN];
#pragma unroll
  for (int i = 0; i < UM; ++i)
#pragma unroll
    for (int j = 0; j < UN; ++j) { accr[i][j] = R(0); acci[i][j] = R(0); }
  const Cx<R> zero = cmake<R>(R(0), R(0));
  const Cx<R>* Ab = A + aoff;
  const Cx<R>* Bb = B + boff;
  // the next slice is fetched into registers while the current one is used
  constexpr int LA = (MP * BK + kThreads - 1) / kThreads, LB = (NP * BK + kThreads - 1) / kThreads;
  Cx<R> ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = tid + u * kThreads;
      int mm, kk;
      if (A_KC) { kk = e % BK; mm = e / BK; } else { mm = e % MP; kk = e / MP; }
      const int k = k0 + kk;
      ra[u] = (e < MP * BK && mm < M && k < kend) ? Ab[aM[mm] + aK[k]] : zero;
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = tid + u * kThreads;
      int nn, kk;
      if (B_KC) { kk = e % BK; nn = e / BK; } else { nn = e % NP; kk = e / NP; }
      const int k = k0 + kk;
      rb[u] = (e < NP * BK && nn < N && k < kend) ? Bb[bN[nn] + bK[k]] : zero;
    }
  };
  if (kbeg < kend) fetch(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      const int e = tid + u * kThreads;
      int mm, kk;
      if (A_KC) { kk = e % BK; mm = e / BK; } else { mm = e % MP; kk = e / MP; }
      if (e < MP * BK) As[kk * MS + mm] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      const int e = tid + u * kThreads;
      int nn, kk;
      if (B_KC) { kk = e % BK; nn = e / BK; } else { nn = e % NP; kk = e / NP; }
      if (e < NP * BK) Bs[kk * NS + nn] = rb[u];
    }
    __syncthreads();
    if (k0 + BK < kend) fetch(k0 + BK);
#pragma unroll 4
    for (int kk = g; kk < BK; kk += G) {
      Cx<R> a[UM], b[UN];
#pragma unroll
      for (int i = 0; i < UM; ++i) a[i] = As[kk * MS + rm + RM * i];
#pragma unroll
      for (int j = 0; j < UN; ++j) b[j] = Bs[kk * NS + rn + RN * j];
#pragma unroll
      for (int i = 0; i < UM; ++i)
#pragma unroll
        for (int j = 0; j < UN; ++j) cfma<R>(accr[i][j], acci[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  // fixed-order sum over the thread groups: shuffles within a warp, then
  // shared memory across warps
  if (S::WG > 1) {
#pragma unroll
    for (int off = RM * RN; off < 32; off <<= 1)
#pragma unroll
      for (int i = 0; i < UM; ++i)
#pragma unroll
        for (int j = 0; j < UN; ++j) {
          accr[i][j] += __shfl_xor_sync(0xffffffffu, accr[i][j], off);
          acci[i][j] += __shfl_xor_sync(0xffffffffu, acci[i][j], off);
        }
  }
  auto store = [&](int m, int n, R re, R im) {
    if (m >= M || n >= N) return;
    if (part) {
      part[(size_t(m) * N + n) * gridDim.x + split] = cmake<R>(re, im);
    } else {
      const long long idx = coff + cM[m] + cN[n];
      Cx<R> v = cmake<R>(alpha * re, alpha * im);
      if (accumulate) { v.x += Cp[idx].x; v.y += Cp[idx].y; }
      Cp[idx] = v;
    }
  };
  if (S::GS == 1) {
    if (g != 0) return;
#pragma unroll
    for (int i = 0; i < UM; ++i)
#pragma unroll
      for (int j = 0; j < UN; ++j) store(rm + RM * i, rn + RN * j, accr[i][j], acci[i][j]);
    return;
  }
  // one [MP][NP] tile in shared memory, the warp-level partials added into it
  // one group after another (fixed order)
  Cx<R>* red = reinterpret_cast<Cx<R>*>(smem);
  for (int gs = 0; gs < S::GS; ++gs) {
    if (g % S::WG == 0 && g / S::WG == gs) {
#pragma unroll
      for (int i = 0; i < UM; ++i)
#pragma unroll
        for (int j = 0; j < UN; ++j) {
          Cx<R>& r = red[(rm + RM * i) * NP + rn + RN * j];
          r = gs == 0 ? cmake<R>(accr[i][j], acci[i][j])
                      : cmake<R>(r.x + accr[i][j], r.y + acci[i][j]);
        }
    }
    __syncthreads();
  }
  for (int t = tid; t < MP * NP; t += kThreads) store(t / NP, t % NP, red[t].x, red[t].y);
}

// C[cM[m] + cN[n]] (+)= alpha sum_s part[m][n][s]: one warp per output, the
// splits summed in a fixed order (lane-strided, then a shuffle tree).
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_split_sum(const Cx<R>* __restrict__ part, int nsplit, Cx<R>* __restrict__ Cp, long long coff,
            const long long* __restrict__ cM, const long long* __restrict__ cN, int M, int N,
            R alpha, int accumulate) {
  const int lane = threadIdx.x & 31;
  const long long w0 = (long long)blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  const long long nw = (long long)gridDim.x * (kThreads / 32);
  for (long long t = w0; t < (long long)M * N; t += nw) {
    const Cx<R>* p = part + t * nsplit;
    R re = 0, im = 0;
    for (int sp = lane; sp < nsplit; sp += 32) {
      re += p[sp].x;
      im += p[sp].y;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, off);
      im += __shfl_xor_sync(0xffffffffu, im, off);
    }
    if (lane == 0) {
      const int m = int(t / N), n = int(t - (long long)m * N);
      const long long idx = coff + cM[m] + cN[n];
      Cx<R> v = cmake<R>(alpha * re, alpha * im);
      if (accumulate) { v.x += Cp[idx].x; v.y += Cp[idx].y; }
      Cp[idx] = v;
    }
  }
}

// One output per warp (A contiguous along k: lanes stride k) or per thread.
template <typename R, bool A_KC>
__global__ void __launch_bounds__(kThreads)
k_gemv(const Cx<R>* __restrict__ A, long long aoff, const long long* __restrict__ aM,
       const long long* __restrict__ aK, const Cx<R>* __restrict__ B, long long boff,
       const long long* __restrict__ bK, Cx<R>* __restrict__ Cp, long long coff,
       const long long* __restrict__ cM, int M, int K, R alpha, int accumulate) {
  const Cx<R>* Ab = A + aoff;
  const Cx<R>* Bb = B + boff;
  if (A_KC) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (long long)(blockIdx.x * (kThreads / 32)) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (kThreads / 32);
    for (long long m = w0; m < M; m += nw) {
      const Cx<R>* row = Ab + aM[m];
      R re = 0, im = 0;
      for (int k = lane; k < K; k += 32) cfma<R>(re, im, row[aK[k]], Bb[bK[k]]);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, off);
        im += __shfl_xor_sync(0xffffffffu, im, off);
      }
      if (lane == 0) {
        const long long idx = coff + cM[m];
        Cx<R> v = cmake<R>(alpha * re, alpha * im);
        if (accumulate) { v.x += Cp[idx].x; v.y += Cp[idx].y; }
        Cp[idx] = v;
      }
    }
  } else {
    for (long long m = (long long)blockIdx.x * kThreads + threadIdx.x; m < M;
         m += (long long)gridDim.x * kThreads) {
      const Cx<R>* row = Ab + aM[m];
      R re = 0, im = 0;
#pragma unroll 4
      for (int k = 0; k < K; ++k) cfma<R>(re, im, row[aK[k]], Bb[bK[k]]);
      const long long idx = coff + cM[m];
      Cx<R> v = cmake<R>(alpha * re, alpha * im);
      if (accumulate) { v.x += Cp[idx].x; v.y += Cp[idx].y; }
      Cp[idx] = v;
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_outer(const Cx<R>* __restrict__ A, long long aoff, const long long* __restrict__ aM,
        const long long* __restrict__ aK, const Cx<R>* __restrict__ B, long long boff,
        const long long* __restrict__ bN, const long long* __restrict__ bK, Cx<R>* __restrict__ Cp,
        long long coff, const long long* __restrict__ cM, const long long* __restrict__ cN, int M,
        int N, R alpha, int accumulate) {
  const long long ak = aK[0], bk = bK[0];
  for (int m = blockIdx.y; m < M; m += gridDim.y) {
    const Cx<R> a = A[aoff + aM[m] + ak];
    const R ar = alpha * a.x, ai = alpha * a.y;
    const long long cm = coff + cM[m];
    for (int n = blockIdx.x * kThreads + threadIdx.x; n < N; n += gridDim.x * kThreads) {
      const Cx<R> b = B[boff + bN[n] + bk];
      const long long idx = cm + cN[n];
      Cx<R> v = cmake<R>(ar * b.x - ai * b.y, ar * b.y + ai * b.x);
      if (accumulate) {
        const Cx<R> c = Cp[idx];
        v.x += c.x;
        v.y += c.y;
      }
      Cp[idx] = v;
    }
  }
}

template <typename R, int RM, int RN, int UM, int UN>
void launch_cfg(bool a_kc, bool b_kc, const Cx<R>* A, long long aoff, const long long* aM,
                const long long* aK, const Cx<R>* B, long long boff, const long long* bN,
                const long long* bK, Cx<R>* C, long long coff, const long long* cM,
                const long long* cN, int M, int N, int K, int nsplit, int kchunk, double alpha,
                bool accumulate, Cx<R>* part, cudaStream_t s) {
  Cx<R>* p = nsplit > 1 ? part : nullptr;
#define RTCC3_RS(AK, BK_)                                                                        \
  k_reduce_small<R, AK, BK_, RM, RN, UM, UN><<<nsplit, kThreads, 0, s>>>(                        \
      A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N, K, kchunk, R(alpha),              \
      accumulate ? 1 : 0, p)
  if (a_kc && b_kc) RTCC3_RS(true, true);
  else if (a_kc) RTCC3_RS(true, false);
  else if (b_kc) RTCC3_RS(false, true);
  else RTCC3_RS(false, false);
#undef RTCC3_RS
  RTCC3_CUDA(cudaGetLastError());
  if (nsplit > 1) {
    const long long warps = (long long)M * N;
    const int grid = int(std::max<long long>(1, std::min<long long>((warps * 32 + kThreads - 1) / kThreads,
                                                                     152LL * 16)));
    k_split_sum<R><<<grid, kThreads, 0, s>>>(part, nsplit, C, coff, cM, cN, M, N, R(alpha),
                                             accumulate ? 1 : 0);
    RTCC3_CUDA(cudaGetLastError());
  }
}

}  // namespace

template <typename R>
void launch_outer(const Cx<R>* A, long long aoff, const long long* aM, const long long* aK,
                  const Cx<R>* B, long long boff, const long long* bN, const long long* bK,
                  Cx<R>* C, long long coff, const long long* cM, const long long* cN, int M, int N,
                  double alpha, bool accumulate, cudaStream_t s) {
  // about four outputs per thread along n, rows spread over grid.y
  const int gx = std::max(1, std::min(1024, (N + 4 * kThreads - 1) / (4 * kThreads)));
  const int gy = std::max(1, std::min(M, std::max(1, 152 * 32 / gx)));
  k_outer<R><<<dim3(gx, gy), kThreads, 0, s>>>(A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN,
                                               M, N, R(alpha), accumulate ? 1 : 0);
  RTCC3_CUDA(cudaGetLastError());
}

int small_output_config(long long M, long long N) {
  if (M <= 10 && N <= 10) return kSmall10;
  if (M <= 16 && N <= 16) return kSmall16;
  if (M <= 40 && N <= 40) return kSmall40;
  if (M <= 48 && N <= 48) return kSmall48;
  if (M <= 64 && N <= 64) return kSmall64;
  if (N == 1 && M <= 256) return kSmallCol256;
  if (N == 1 && M <= 512) return kSmallCol512;
  return kSmallNone;
}

int small_output_bk(int cfg, int elem_bytes) {
  const bool d = elem_bytes == 16;
  switch (cfg) {
    case kSmall10: return d ? SmallShape<double, 2, 2, 5, 5>::BK : SmallShape<float, 2, 2, 5, 5>::BK;
    case kSmall16: return d ? SmallShape<double, 4, 4, 4, 4>::BK : SmallShape<float, 4, 4, 4, 4>::BK;
    case kSmall40: return d ? SmallShape<double, 8, 8, 5, 5>::BK : SmallShape<float, 8, 8, 5, 5>::BK;
    case kSmall48: return d ? SmallShape<double, 16, 16, 3, 3>::BK : SmallShape<float, 16, 16, 3, 3>::BK;
    case kSmall64: return d ? SmallShape<double, 16, 16, 4, 4>::BK : SmallShape<float, 16, 16, 4, 4>::BK;
    case kSmallCol256: return d ? SmallShape<double, 64, 1, 4, 1>::BK : SmallShape<float, 64, 1, 4, 1>::BK;
    case kSmallCol512: return d ? SmallShape<double, 128, 1, 4, 1>::BK : SmallShape<float, 128, 1, 4, 1>::BK;
    default: return 0;
  }
}

template <typename R>
void launch_reduce_small(int cfg, bool a_kc, bool b_kc, const Cx<R>* A, long long aoff,
                         const long long* aM, const long long* aK, const Cx<R>* B, long long boff,
                         const long long* bN, const long long* bK, Cx<R>* C, long long coff,
                         const long long* cM, const long long* cN, int M, int N, int K, int nsplit,
                         int kchunk, double alpha, bool accumulate, Cx<R>* part, cudaStream_t s) {
  switch (cfg) {
    case kSmall10:
      launch_cfg<R, 2, 2, 5, 5>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N, K,
                                nsplit, kchunk, alpha, accumulate, part, s);
      break;
    case kSmall40:
      launch_cfg<R, 8, 8, 5, 5>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N, K,
                                nsplit, kchunk, alpha, accumulate, part, s);
      break;
    case kSmall16:
      launch_cfg<R, 4, 4, 4, 4>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N, K,
                                nsplit, kchunk, alpha, accumulate, part, s);
      break;
    case kSmall48:
      launch_cfg<R, 16, 16, 3, 3>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N,
                                  K, nsplit, kchunk, alpha, accumulate, part, s);
      break;
    case kSmall64:
      launch_cfg<R, 16, 16, 4, 4>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N,
                                  K, nsplit, kchunk, alpha, accumulate, part, s);
      break;
    case kSmallCol256:
      launch_cfg<R, 64, 1, 4, 1>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N, K,
                                 nsplit, kchunk, alpha, accumulate, part, s);
      break;
    case kSmallCol512:
      launch_cfg<R, 128, 1, 4, 1>(a_kc, b_kc, A, aoff, aM, aK, B, boff, bN, bK, C, coff, cM, cN, M, N,
                                  K, nsplit, kchunk, alpha, accumulate, part, s);
      break;
    default:
      throw Error(kErrArg, "reduce_small: unsupported output shape");
  }
}

template <typename R>
void launch_gemv(bool a_kc, const Cx<R>* A, long long aoff, const long long* aM, const long long* aK,
                 const Cx<R>* B, long long boff, const long long* bK, Cx<R>* C, long long coff,
                 const long long* cM, int M, int K, double alpha, bool accumulate, cudaStream_t s) {
  const long long units = a_kc ? (long long)M * 32 : (long long)M;
  const int grid = int(std::max<long long>(1, std::min<long long>((units + kThreads - 1) / kThreads,
                                                                   152LL * 16)));
  if (a_kc)
    k_gemv<R, true><<<grid, kThreads, 0, s>>>(A, aoff, aM, aK, B, boff, bK, C, coff, cM, M, K, R(alpha),
                                              accumulate ? 1 : 0);
  else
    k_gemv<R, false><<<grid, kThreads, 0, s>>>(A, aoff, aM, aK, B, boff, bK, C, coff, cM, M, K, R(alpha),
                                               accumulate ? 1 : 0);
  RTCC3_CUDA(cudaGetLastError());
}

#define RTCC3_INST(R)                                                                              \
  template void launch_reduce_small<R>(int, bool, bool, const Cx<R>*, long long, const long long*,  \
                                       const long long*, const Cx<R>*, long long, const long long*, \
                                       const long long*, Cx<R>*, long long, const long long*,       \
                                       const long long*, int, int, int, int, int, double, bool,     \
                                       Cx<R>*, cudaStream_t);                                       \
  template void launch_gemv<R>(bool, const Cx<R>*, long long, const long long*, const long long*,   \
                               const Cx<R>*, long long, const long long*, Cx<R>*, long long,        \
                               const long long*, int, int, double, bool, cudaStream_t);         \
  template void launch_outer<R>(const Cx<R>*, long long, const long long*, const long long*,       \
                                const Cx<R>*, long long, const long long*, const long long*,       \
                                Cx<R>*, long long, const long long*, const long long*, int, int,   \
                                double, bool, cudaStream_t);
RTCC3_INST(float)
RTCC3_INST(double)
#undef RTCC3_INST

}  // namespace rtcc3
