// Kernels and host logic of the reverse-mode tensor engine (see engine.h).
#include "engine.h"

#include <algorithm>
#include <type_traits>

#include "contract_small.h"
#include "tc_gemm.h"
#include <cstring>
#include <sstream>

namespace rtcc3 {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16, kThreads = 256;
constexpr int kSBM = 16, kSBK = 64;  // small-tile variant
constexpr int kTBK = 8;               // thin (16 x 256) tiles
constexpr int kTcMaxKbPerSplit = 16;  // K tiles per tensor-core accumulation chain
constexpr size_t kLazyGradMin = 65536;  // gradients this large are not zero-filled up front

// Division of 32-bit n < 2^31 by an invariant d >= 1 with one multiply-high
// (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994; round-up variant): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(n, m) + n) >> l.
struct FastDiv {
  unsigned d = 1, m = 1;
  int l = 0;
  FastDiv() = default;
  explicit FastDiv(unsigned dv) : d(dv) {
    l = 0;
    while ((1ull << l) < dv) ++l;
    m = unsigned(((1ull << 32) * ((1ull << l) - dv)) / dv + 1);
  }
  __device__ __forceinline__ unsigned div(unsigned n) const { return (__umulhi(n, m) + n) >> l; }
};

struct EpsArgs {
  int sign[kMaxDim];
  int base[kMaxDim];
  const double* osum;
  const double* vsum;
  int o, v;
};

// Triples denominators from the precomputed FP64 occupied / virtual sums, for
// X and Y both in the dense (o,o,o,v,v,v) layout: one FP64 subtraction per
// element instead of six FP64 additions (GB300's FP64 rate is low).
// Complex denominators (field-dressed eigenvalue sums), dense layout:
// y (+)= x / (vsum[abc] - osum[ijk]); the sums are FP64, the division in R.
template <typename R, typename I>
__global__ void k_div_lambda_dense6(const Cx<R>* __restrict__ X, Cx<R>* __restrict__ Y,
                                    long long offx, long long offy,
                                    const double2* __restrict__ osum,
                                    const double2* __restrict__ vsum, I v3, I n, int overwrite) {
  for (I t = I(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += I(gridDim.x) * blockDim.x) {
    const I ijk = t / v3;
    const I abc = t - ijk * v3;
    const double2 vs = vsum[abc], os = osum[ijk];
    const R dr = R(vs.x - os.x), di = R(vs.y - os.y);
    const R m = R(1) / (dr * dr + di * di);
    const R ir = dr * m, ii = -di * m;  // 1 / (dr + i di)
    const Cx<R> x = X[offx + t];
    Cx<R> y = overwrite ? cmake<R>(R(0), R(0)) : Y[offy + t];
    y.x += x.x * ir - x.y * ii;
    y.y += x.x * ii + x.y * ir;
    Y[offy + t] = y;
  }
}

template <typename R, typename I>
__global__ void k_div_eps_dense6(const Cx<R>* __restrict__ X, Cx<R>* __restrict__ Y, long long offx,
                                 long long offy, const double* __restrict__ osum,
                                 const double* __restrict__ vsum, I v3, I n, int overwrite) {
  for (I t = I(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += I(gridDim.x) * blockDim.x) {
    const I ijk = t / v3;
    const I abc = t - ijk * v3;
    const R inv = R(1) / R(vsum[abc] - osum[ijk]);
    const Cx<R> x = X[offx + t];
    Cx<R> y = overwrite ? cmake<R>(R(0), R(0)) : Y[offy + t];
    y.x += x.x * inv;
    y.y += x.y * inv;
    Y[offy + t] = y;
  }
}

// One slab of the triples, dense (I, o, o, v, v, v) with its first occupied
// index starting at i0: Y = alpha X / D, D[ijk abc] = vsum[abc] - osum[ijk]
// with the sums in the compute precision (complex when CPLX).  X may be Y.
template <typename R, bool CPLX>
__global__ void k_slab_div(const Cx<R>* X, Cx<R>* Y, const R* __restrict__ osum,
                           const R* __restrict__ vsum, const Cx<R>* __restrict__ osum_c,
                           const Cx<R>* __restrict__ vsum_c, size_t o2base, size_t v3, size_t n,
                           R alpha) {
  for (size_t t = size_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n;
       t += size_t(gridDim.x) * blockDim.x) {
    const size_t ijk = t / v3;
    const size_t abc = t - ijk * v3;
    const Cx<R> x = X[t];
    Cx<R> y;
    if (CPLX) {
      const Cx<R> vs = vsum_c[abc], os = osum_c[o2base + ijk];
      const R dr = vs.x - os.x, di = vs.y - os.y;
      const R m = alpha / (dr * dr + di * di);
      const R ir = dr * m, ii = -di * m;  // alpha / (dr + i di)
      y.x = x.x * ir - x.y * ii;
      y.y = x.x * ii + x.y * ir;
    } else {
      const R inv = alpha / (vsum[abc] - osum[o2base + ijk]);
      y.x = x.x * inv;
      y.y = x.y * inv;
    }
    Y[t] = y;
  }
}

// Thread layout of a 4 (a) x 8 (b) x 8 (c) brick, 256 threads (LAYOUT 0: a
// warp on 4 x 4 x 2 elements, a fastest; 1: on 2 x 4 x 4, c fastest), first
// c of the thread (stepping by 8).
template <int LAYOUT>
__device__ __forceinline__ void brick_coords(int v, unsigned& a, unsigned& b, unsigned& c0) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nbb = (v + 7) / 8;
  const unsigned ta = unsigned(blockIdx.x / nbb) * 4, tb = unsigned(blockIdx.x % nbb) * 8;
  if (LAYOUT == 0) {
    a = ta + (lane & 3);
    b = tb + (w & 1) * 4 + ((lane >> 2) & 3);
    c0 = unsigned((w >> 1) * 2 + (lane >> 4));
  } else {
    a = ta + (w & 1) * 2 + (lane >> 4);
    b = tb + ((w >> 1) & 1) * 4 + ((lane >> 2) & 3);
    c0 = unsigned((w >> 2) * 4 + (lane & 3));
  }
}

// Y (+)= alpha P(X) / D for X, Y dense (o,o,o,v,v,v): P sums the six
// simultaneous permutations of (ijk, abc) (NP = 6) or the identity and the
// exchanges of slot 1 with slots 2 and 3 (NP = 3), then divides by the
// triples denominator D[ijk abc] = vsum[abc] - osum[ijk] (sums in the compute
// precision; complex when CPLX).  D is invariant under those permutations, so
// for NP = 6 the same kernel is its own adjoint.  Grid: ((a, b) bricks,
// occupied blocks); the occupied blocks are visited in `order` (the distinct
// permutations of each i <= j <= k consecutively), so the source blocks of
// one orbit are read while they are resident in L2.
template <typename R, bool CPLX, int NP>
__global__ void __launch_bounds__(256)
k_sym6_div(const Cx<R>* __restrict__ X, Cx<R>* __restrict__ Y, long long offx, long long offy,
           const R* __restrict__ osum, const R* __restrict__ vsum, const Cx<R>* __restrict__ osum_c,
           const Cx<R>* __restrict__ vsum_c, const int* __restrict__ order, int o, int v, R alpha,
           int overwrite, const FastDiv fv2, const FastDiv fv, Cx<R>* __restrict__ Y3) {
  const int ijk = order ? order[blockIdx.y] : int(blockIdx.y);
  const int i = ijk / (o * o), j = (ijk / o) % o, k = ijk % o;
  const unsigned v2 = unsigned(v) * v, v3 = v2 * v;
  auto O = [&](int x, int y, int z) { return (long long)((x * o + y) * o + z) * v3; };
  const Cx<R>* b0 = X + offx + O(i, j, k);
  const Cx<R>* b1 = X + offx + O(j, i, k);
  const Cx<R>* b2 = X + offx + O(i, k, j);
  const Cx<R>* b3 = X + offx + O(k, j, i);
  const Cx<R>* b4 = X + offx + O(k, i, j);
  const Cx<R>* b5 = X + offx + O(j, k, i);
  Cx<R>* yb = Y + offy + O(i, j, k);
  // NP = 6 with Y3: also Y3 = (x0 + x1 + x3) / D, the NP = 3 sum of the same
  // sources (overwritten; dense, no offset)
  Cx<R>* y3b = Y3 ? Y3 + O(i, j, k) : nullptr;
  auto V = [&](unsigned x, unsigned y, unsigned z) { return (x * v + y) * v + z; };
  auto element = [&](unsigned a, unsigned b, unsigned c, unsigned abc) {
    const Cx<R> x0 = b0[abc];
    const Cx<R> x1 = b1[V(b, a, c)];
    const Cx<R> x3 = b3[V(c, b, a)];
    R sr, si;
    if (NP == 6) {
      const Cx<R> x2 = b2[V(a, c, b)];
      const Cx<R> x4 = b4[V(c, a, b)];
      const Cx<R> x5 = b5[V(b, c, a)];
      sr = alpha * (((x0.x + x1.x) + (x2.x + x3.x)) + (x4.x + x5.x));
      si = alpha * (((x0.y + x1.y) + (x2.y + x3.y)) + (x4.y + x5.y));
      if (y3b) {
        const R tr = (x0.x + x1.x) + x3.x, ti = (x0.y + x1.y) + x3.y;
        Cx<R> z;
        if (CPLX) {
          const Cx<R> vs = vsum_c[abc], os = osum_c[ijk];
          const R dr = vs.x - os.x, di = vs.y - os.y;
          const R m = R(1) / (dr * dr + di * di);
          const R ir = dr * m, ii = -di * m;
          z.x = tr * ir - ti * ii;
          z.y = tr * ii + ti * ir;
        } else {
          const R inv = R(1) / (vsum[abc] - osum[ijk]);
          z.x = tr * inv;
          z.y = ti * inv;
        }
        y3b[abc] = z;
      }
    } else {
      // identity, (ij)(ab) and (ik)(ac): the three slot exchanges with slot 1
      sr = alpha * ((x0.x + x1.x) + x3.x);
      si = alpha * ((x0.y + x1.y) + x3.y);
    }
    Cx<R> y = overwrite ? cmake<R>(R(0), R(0)) : yb[abc];
    if (CPLX) {
      const Cx<R> vs = vsum_c[abc], os = osum_c[ijk];
      const R dr = vs.x - os.x, di = vs.y - os.y;
      const R m = R(1) / (dr * dr + di * di);
      const R ir = dr * m, ii = -di * m;
      y.x += sr * ir - si * ii;
      y.y += sr * ii + si * ir;
    } else {
      const R inv = R(1) / (vsum[abc] - osum[ijk]);
      y.x += sr * inv;
      y.y += si * inv;
    }
    yb[abc] = y;
  };
  if (NP == 6) {
    // a CTA covers a 4 (a) x 8 (b) x 8 (c) brick, stepping over c; a warp
    // covers 2 x 4 x 4 of it, so every source is read in runs of 2 to 4
    // consecutive elements along its own fastest index (the sources permute
    // a, b, c)
    unsigned a, b, c0;
    brick_coords<1>(v, a, b, c0);
    if (a >= unsigned(v) || b >= unsigned(v)) return;
    for (unsigned c = c0; c < unsigned(v); c += 8) element(a, b, c, (a * v + b) * v + c);
  } else {
    // two of the three sources keep c fastest: consecutive threads on
    // consecutive abc
    for (unsigned abc = blockIdx.x * blockDim.x + threadIdx.x; abc < v3;
         abc += gridDim.x * blockDim.x) {
      const unsigned a = fv2.div(abc), bc = abc - a * v2, b = fv.div(bc), c = bc - b * v;
      element(a, b, c, abc);
    }
  }
}

struct StridedDesc {
  int nd;
  int shape[kMaxDim];
  long long s0[kMaxDim];
  long long s1[kMaxDim];
  long long s2[kMaxDim];
  long long off0, off1, off2;
};

template <typename R>
__device__ __forceinline__ void cfma(R& ar, R& ai, Cx<R> a, Cx<R> b) {
  ar = fma(a.x, b.x, ar);
  ar = fma(-a.y, b.y, ar);
  ai = fma(a.x, b.y, ai);
  ai = fma(a.y, b.x, ai);
}

// Generic strided complex contraction as a gather-GEMM: C[b,m,n] (+)= alpha *
// sum_k A[b,m,k] B[b,n,k] with every (b,m,n,k) -> address mapping given by
// offset tables.  BM x BN output tile per CTA, BK-deep K slices in shared
// memory (odd row pitch: the transposing stores of K-contiguous loads do not
// share a bank), TM x TN complex micro-tile per thread on a (BM/TM) x (BN/TN)
// thread grid.  With nsplit > 1 each CTA sums a K chunk into a partial buffer
// and k_split_reduce adds the chunks in fixed order (deterministic results).
template <typename R, bool A_KC, bool B_KC, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__(kThreads)
k_contract(const Cx<R>* __restrict__ A, const Cx<R>* __restrict__ B, Cx<R>* __restrict__ Cp,
           const long long* __restrict__ aM, const long long* __restrict__ aK,
           const long long* __restrict__ bN, const long long* __restrict__ bK,
           const long long* __restrict__ cM, const long long* __restrict__ cN,
           const long long* __restrict__ aB, const long long* __restrict__ bB,
           const long long* __restrict__ cB, int M, int N, int K, int nsplit, int kchunk,
           R alpha, int accumulate, Cx<R>* __restrict__ part) {
  constexpr int RY = BM / TM, RX = BN / TN;  // thread grid, TM x TN outputs each
  static_assert(RY * RX == kThreads, "thread grid");
  __shared__ Cx<R> As[BK][BM + 1];
  __shared__ Cx<R> Bs[BK][BN + 1];
  const int bz = blockIdx.z;
  const int b = bz / nsplit, split = bz % nsplit;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = split * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const Cx<R>* Ab = A + aB[b];
  const Cx<R>* Bb = B + bB[b];
  const int tid = threadIdx.x, tx = tid % RX, ty = tid / RX;
  R accr[TM][TN], acci[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) { accr[i][j] = R(0); acci[i][j] = R(0); }
  const Cx<R> zero = cmake<R>(R(0), R(0));
  // each thread stages the same (row, k-offset) slots of every K slice: the
  // row offsets are looked up once, and the next slice is loaded into
  // registers while the current one is multiplied
  constexpr int LA = (BM * BK + kThreads - 1) / kThreads;
  constexpr int LB = (BN * BK + kThreads - 1) / kThreads;
  long long arow[LA], brow[LB];
  bool aok[LA], bok[LB];
  Cx<R> ra[LA], rb[LB];
#pragma unroll
  for (int l = 0; l < LA; ++l) {
    const int e = l * kThreads + tid;
    const int mm = A_KC ? e / BK : e % BM;
    aok[l] = e < BM * BK && m0 + mm < M;
    arow[l] = aok[l] ? aM[m0 + mm] : 0;
  }
#pragma unroll
  for (int l = 0; l < LB; ++l) {
    const int e = l * kThreads + tid;
    const int nn = B_KC ? e / BK : e % BN;
    bok[l] = e < BN * BK && n0 + nn < N;
    brow[l] = bok[l] ? bN[n0 + nn] : 0;
  }
  auto load = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = l * kThreads + tid;
      const int k = k0 + (A_KC ? e % BK : e / BM);
      ra[l] = (aok[l] && k < kend) ? Ab[arow[l] + aK[k]] : zero;
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = l * kThreads + tid;
      const int k = k0 + (B_KC ? e % BK : e / BN);
      rb[l] = (bok[l] && k < kend) ? Bb[brow[l] + bK[k]] : zero;
    }
  };
  if (kbeg < kend) load(kbeg);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int l = 0; l < LA; ++l) {
      const int e = l * kThreads + tid;
      if ((BM * BK) % kThreads != 0 && e >= BM * BK) break;
      if (A_KC) As[e % BK][e / BK] = ra[l];
      else As[e / BM][e % BM] = ra[l];
    }
#pragma unroll
    for (int l = 0; l < LB; ++l) {
      const int e = l * kThreads + tid;
      if ((BN * BK) % kThreads != 0 && e >= BN * BK) break;
      if (B_KC) Bs[e % BK][e / BK] = rb[l];
      else Bs[e / BN][e % BN] = rb[l];
    }
    __syncthreads();
    if (k0 + BK < kend) load(k0 + BK);
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      Cx<R> a[TM], bv[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + RY * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + RX * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma<R>(accr[i][j], acci[i][j], a[i], bv[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int m = m0 + ty + RY * i;
    if (m >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int n = n0 + tx + RX * j;
      if (n >= N) continue;
      if (nsplit == 1) {
        const long long idx = cB[b] + cM[m] + cN[n];
        Cx<R> val = cmake<R>(alpha * accr[i][j], alpha * acci[i][j]);
        if (accumulate) { val.x += Cp[idx].x; val.y += Cp[idx].y; }
        Cp[idx] = val;
      } else {
        part[((size_t)bz * M + m) * N + n] = cmake<R>(accr[i][j], acci[i][j]);
      }
    }
  }
}

template <typename R>
__global__ void k_split_reduce(const Cx<R>* __restrict__ part, Cx<R>* __restrict__ Cp,
                               const long long* __restrict__ cM, const long long* __restrict__ cN,
                               const long long* __restrict__ cB, int M, int N, int nb, int nsplit,
                               R alpha, int accumulate) {
  const size_t total = (size_t)nb * M * N;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    const int n = int(t % N);
    const int m = int((t / N) % M);
    const int b = int(t / ((size_t)M * N));
    R sr = 0, si = 0;
    for (int s = 0; s < nsplit; ++s) {
      const Cx<R> p = part[(((size_t)b * nsplit + s) * M + m) * N + n];
      sr += p.x;
      si += p.y;
    }
    const long long idx = cB[b] + cM[m] + cN[n];
    Cx<R> val = cmake<R>(alpha * sr, alpha * si);
    if (accumulate) { val.x += Cp[idx].x; val.y += Cp[idx].y; }
    Cp[idx] = val;
  }
}

__device__ __forceinline__ void decode(const StridedDesc& d, size_t t, long long& o0, long long& o1,
                                       long long& o2) {
  o0 = d.off0; o1 = d.off1; o2 = d.off2;
  for (int k = d.nd - 1; k >= 0; --k) {
    const long long i = (long long)(t % (size_t)d.shape[k]);
    t /= (size_t)d.shape[k];
    o0 += i * d.s0[k];
    o1 += i * d.s1[k];
    o2 += i * d.s2[k];
  }
}

// Y[.] += alpha X[.] over Y's shape (desc slots: 0 = X, 1 = Y).
template <typename R>
__global__ void k_axpy(const Cx<R>* __restrict__ X, Cx<R>* __restrict__ Y, StridedDesc d, R alpha,
                       size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    long long ox, oy, oz;
    decode(d, t, ox, oy, oz);
    const Cx<R> x = X[ox];
    Cx<R> y = Y[oy];
    y.x += alpha * x.x;
    y.y += alpha * x.y;
    Y[oy] = y;
  }
}

// Y[.] += X[.] * c[.] (complex product; slots 0 = X, 1 = Y, 2 = c).
template <typename R>
__global__ void k_mulc(const Cx<R>* __restrict__ X, const Cx<R>* __restrict__ Cst,
                       Cx<R>* __restrict__ Y, StridedDesc d, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x) {
    long long ox, oy, oc;
    decode(d, t, ox, oy, oc);
    const Cx<R> x = X[ox], c = Cst[oc];
    Cx<R> y = Y[oy];
    y.x += x.x * c.x - x.y * c.y;
    y.y += x.x * c.y + x.y * c.x;
    Y[oy] = y;
  }
}

// Y[.] += X[.] / eps(index) in FP64 (slot 0 = X, 1 = Y).
template <typename R, typename I>
__global__ void k_div_eps(const Cx<R>* __restrict__ X, Cx<R>* __restrict__ Y, StridedDesc d,
                          const double* __restrict__ eps, EpsArgs ea, I n, int overwrite) {
  for (I t = I(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += I(gridDim.x) * blockDim.x) {
    long long ox = d.off0, oy = d.off1;
    double den = 0.0;
    I rem = t;
    for (int k = d.nd - 1; k >= 0; --k) {
      const I sh = I(d.shape[k]);
      const long long i = (long long)(rem % sh);
      rem /= sh;
      ox += i * d.s0[k];
      oy += i * d.s1[k];
      if (ea.sign[k]) den += ea.sign[k] * eps[ea.base[k] + i];
    }
    const Cx<R> x = X[ox];
    Cx<R> y = overwrite ? cmake<R>(R(0), R(0)) : Y[oy];
    // the orbital-energy sum is formed in FP64; the division runs in the
    // graph's precision (R = float: one FP32 reciprocal instead of two FP64
    // divisions, which GB300's reduced FP64 rate makes the costliest step)
    const R inv = R(1) / R(den);
    y.x += x.x * inv;
    y.y += x.y * inv;
    Y[oy] = y;
  }
}

// Y[.] (+)= sum_s alpha_s X_s[.] over Y's shape: up to kMaxSrc strided
// sources, one pass, coalesced on Y (threads walk Y's last index fastest).
constexpr int kMaxSrc = kCombineSources;
template <typename R>
struct CombDesc {
  int nd, nsrc, overwrite;
  int shape[kMaxDim];
  FastDiv fd[kMaxDim];  // divisors of the extents (32-bit index path)
  long long sy[kMaxDim];
  long long sx[kMaxSrc][kMaxDim];
  long long offy;
  long long offx[kMaxSrc];
  R alpha[kMaxSrc];
  const Cx<R>* src[kMaxSrc];
};

template <typename R, typename I>
__global__ void k_combine(Cx<R>* __restrict__ Y, const CombDesc<R> d, I n) {
  for (I t = I(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += I(gridDim.x) * blockDim.x) {
    I rem = t;
    long long oy = d.offy;
    long long ox[kMaxSrc];
#pragma unroll
    for (int s = 0; s < kMaxSrc; ++s) ox[s] = d.offx[s];
    for (int k = d.nd - 1; k >= 0; --k) {
      const I sh = I(d.shape[k]);
      I q;
      if constexpr (sizeof(I) == 4) q = I(d.fd[k].div(unsigned(rem)));
      else q = rem / sh;
      const I i = rem - q * sh;
      rem = q;
      oy += (long long)i * d.sy[k];
#pragma unroll
      for (int s = 0; s < kMaxSrc; ++s)
        if (s < d.nsrc) ox[s] += (long long)i * d.sx[s][k];
    }
    R re = R(0), im = R(0);
#pragma unroll
    for (int s = 0; s < kMaxSrc; ++s)
      if (s < d.nsrc) {
        const Cx<R> x = d.src[s][ox[s]];
        re += d.alpha[s] * x.x;
        im += d.alpha[s] * x.y;
      }
    if (!d.overwrite) {
      const Cx<R> y = Y[oy];
      re += y.x;
      im += y.y;
    }
    Y[oy] = cmake<R>(re, im);
  }
}

// k_combine with the rank ND a compile-time constant (every descriptor index
// constant: the strides stay in the parameter bank, no local-memory copy) and
// OFF32: all element offsets fit 31 bits (32-bit index arithmetic).
template <typename R, int ND, bool OFF32>
__global__ void __launch_bounds__(256) k_combine_nd(Cx<R>* __restrict__ Y, const CombDesc<R> d, unsigned n) {
  using O = typename std::conditional<OFF32, int, long long>::type;
  for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    unsigned rem = t;
    O oy = O(d.offy);
    O ox[kMaxSrc];
#pragma unroll
    for (int s = 0; s < kMaxSrc; ++s) ox[s] = O(d.offx[s]);
#pragma unroll
    for (int k = ND - 1; k >= 0; --k) {
      const unsigned q = k > 0 ? d.fd[k].div(rem) : 0u;
      const O i = O(rem - q * unsigned(d.shape[k]));
      rem = q;
      oy += i * O(d.sy[k]);
#pragma unroll
      for (int s = 0; s < kMaxSrc; ++s)
        if (s < d.nsrc) ox[s] += i * O(d.sx[s][k]);
    }
    R re = R(0), im = R(0);
#pragma unroll
    for (int s = 0; s < kMaxSrc; ++s)
      if (s < d.nsrc) {
        const Cx<R> x = d.src[s][ox[s]];
        re += d.alpha[s] * x.x;
        im += d.alpha[s] * x.y;
      }
    if (!d.overwrite) {
      const Cx<R> y = Y[oy];
      re += y.x;
      im += y.y;
    }
    Y[oy] = cmake<R>(re, im);
  }
}

// Y[blk][abc] (+)= sum_s alpha_s X_s[blk][sigma_s(abc)] over dense
// (nblk, v, v, v) tensors whose sources permute the last three indices, in
// brick thread layouts (a CTA per 4 x 8 (a, b) brick of a block, stepping
// over c; a warp on 4 x 4 x 2 or 2 x 4 x 4 elements), so sources whose
// fastest index is a or b are read in runs of 2 to 4 instead of one element
// per lane.  Source s has stride 1, v or v^2 for a, b, c as encoded
// in lv (bits 0-1, 2-3, 4-5: 0 stride 1, 1 stride v, 2 stride v^2).
template <typename R>
struct BrickDesc {
  const Cx<R>* src[kMaxSrc];  // at the source's view offset
  R alpha[kMaxSrc];
  int lv[kMaxSrc];
  int nsrc;
  Cx<R>* y;  // at the output's view offset
  int overwrite;
  int v;
};

template <typename R, int NS, int LAYOUT>
__global__ void __launch_bounds__(256) k_combine_brick(const BrickDesc<R> d) {
  const int v = d.v;
  const unsigned v2 = unsigned(v) * unsigned(v);
  const size_t v3 = size_t(v2) * v;
  unsigned a, b, c0;
  brick_coords<LAYOUT>(v, a, b, c0);
  if (a >= unsigned(v) || b >= unsigned(v)) return;
  const size_t blk = size_t(blockIdx.y) * v3;
  unsigned sa[NS], sb[NS], sc[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int lv = d.lv[s];
    const int la = lv & 3, lb = (lv >> 2) & 3, lc = (lv >> 4) & 3;
    sa[s] = la == 0 ? 1u : (la == 1 ? unsigned(v) : v2);
    sb[s] = lb == 0 ? 1u : (lb == 1 ? unsigned(v) : v2);
    sc[s] = lc == 0 ? 1u : (lc == 1 ? unsigned(v) : v2);
  }
  for (unsigned c = c0; c < unsigned(v); c += 8) {
    R re = R(0), im = R(0);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const Cx<R> x = d.src[s][blk + a * sa[s] + b * sb[s] + c * sc[s]];
      re += d.alpha[s] * x.x;
      im += d.alpha[s] * x.y;
    }
    Cx<R>* py = d.y + blk + (a * v + b) * v + c;
    if (!d.overwrite) {
      const Cx<R> o = *py;
      re += o.x;
      im += o.y;
    }
    *py = cmake<R>(re, im);
  }
}

// Several outputs of one pass over shared permuted sources (layout as
// k_combine_brick): Y_o[blk][abc] = sum_u coef[o][u] X_u[blk][sigma_u(abc)],
// each source element loaded once for all outputs.
constexpr int kMultiOut = 3;
template <typename R>
struct BrickMultiDesc {
  const Cx<R>* src[6];
  int lv[6];
  R coef[kMultiOut][6];
  Cx<R>* y[kMultiOut];
  int v;
};

template <typename R, int NU, int NO, int LAYOUT>
__global__ void __launch_bounds__(256) k_combine_brick_multi(const BrickMultiDesc<R> d) {
  const int v = d.v;
  const unsigned v2 = unsigned(v) * unsigned(v);
  const size_t v3 = size_t(v2) * v;
  unsigned a, b, c0;
  brick_coords<LAYOUT>(v, a, b, c0);
  if (a >= unsigned(v) || b >= unsigned(v)) return;
  const size_t blk = size_t(blockIdx.y) * v3;
  unsigned sa[NU], sb[NU], sc[NU];
#pragma unroll
  for (int u = 0; u < NU; ++u) {
    const int lv = d.lv[u];
    const int la = lv & 3, lb = (lv >> 2) & 3, lc = (lv >> 4) & 3;
    sa[u] = la == 0 ? 1u : (la == 1 ? unsigned(v) : v2);
    sb[u] = lb == 0 ? 1u : (lb == 1 ? unsigned(v) : v2);
    sc[u] = lc == 0 ? 1u : (lc == 1 ? unsigned(v) : v2);
  }
  for (unsigned c = c0; c < unsigned(v); c += 8) {
    Cx<R> x[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) x[u] = d.src[u][blk + a * sa[u] + b * sb[u] + c * sc[u]];
    const size_t out = blk + (a * v + b) * v + c;
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      R re = R(0), im = R(0);
#pragma unroll
      for (int u = 0; u < NU; ++u) {
        re += d.coef[o][u] * x[u].x;
        im += d.coef[o][u] * x[u].y;
      }
      d.y[o][out] = cmake<R>(re, im);
    }
  }
}

// Y[ijk][abc] (+)= a1 x1[i,a] y1[j,k,b,c] + a2 x2[i,j,a,b] y2[k,c] over
// dense (o,o,o,v,v,v): the two outer products of the adjoints of X1 and of
// the first X2 term (Eqs. A21-A22) in one pass (a term with a zero
// coefficient is not read).  One block row per (i,j,k), consecutive threads
// on consecutive abc.
template <typename R>
__global__ void __launch_bounds__(256)
k_outer_pair(Cx<R>* __restrict__ Y, const Cx<R>* __restrict__ x1, const Cx<R>* __restrict__ y1,
             const Cx<R>* __restrict__ x2, const Cx<R>* __restrict__ y2, R a1, R a2, int o, int v,
             int accumulate, const FastDiv fv2, const FastDiv fv) {
  const int ijk = blockIdx.y;
  const int i = ijk / (o * o), j = (ijk / o) % o, k = ijk % o;
  const unsigned v2 = unsigned(v) * v, v3 = v2 * v;
  Cx<R>* yb = Y + size_t(ijk) * v3;
  const Cx<R>* x1i = x1 + size_t(i) * v;
  const Cx<R>* y1jk = y1 + (size_t(j) * o + k) * v2;
  const Cx<R>* x2ij = x2 + (size_t(i) * o + j) * v2;
  const Cx<R>* y2k = y2 + size_t(k) * v;
  for (unsigned abc = blockIdx.x * blockDim.x + threadIdx.x; abc < v3; abc += gridDim.x * blockDim.x) {
    const unsigned a = fv2.div(abc), bc = abc - a * v2, b = fv.div(bc), c = bc - b * v;
    R re = R(0), im = R(0);
    if (a1 != R(0)) {
      const Cx<R> p = x1i[a], q = y1jk[bc];
      re += a1 * (p.x * q.x - p.y * q.y);
      im += a1 * (p.x * q.y + p.y * q.x);
    }
    if (a2 != R(0)) {
      const Cx<R> p = x2ij[a * v + b], q = y2k[c];
      re += a2 * (p.x * q.x - p.y * q.y);
      im += a2 * (p.x * q.y + p.y * q.x);
    }
    if (accumulate) {
      const Cx<R> y = yb[abc];
      re += y.x;
      im += y.y;
    }
    yb[abc] = cmake<R>(re, im);
  }
}

template <typename R>
__global__ void k_fill(Cx<R>* p, size_t n, R re, R im) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    p[t] = cmake<R>(re, im);
}

template <typename R>
__global__ void k_identity(Cx<R>* p, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n * n) p[t] = cmake<R>((t / n) == (t % n) ? R(1) : R(0), R(0));
}

int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return int(std::max<size_t>(1, std::min<size_t>(g, 152 * 16)));
}

struct Spec {
  std::string a, b, c;
};

Spec parse(const std::string& s) {
  Spec r;
  const size_t comma = s.find(','), arrow = s.find("->");
  if (comma == std::string::npos || arrow == std::string::npos || comma > arrow)
    throw Error(kErrArg, "bad contraction spec " + s);
  r.a = s.substr(0, comma);
  r.b = s.substr(comma + 1, arrow - comma - 1);
  r.c = s.substr(arrow + 2);
  return r;
}

std::string view_key(const View& v) {
  std::ostringstream o;
  o << v.off << ':';
  for (int d = 0; d < v.nd; ++d) o << v.shape[d] << '/' << v.stride[d] << ',';
  return o.str();
}

}  // namespace

static bool same_view(const View& a, const View& b) {
  if (a.node != b.node || a.off != b.off || a.nd != b.nd) return false;
  for (int d = 0; d < a.nd; ++d)
    if (a.shape[d] != b.shape[d] || a.stride[d] != b.stride[d]) return false;
  return true;
}

// If X covers its whole node as a permutation of the node's dense layout,
// reorder the dimensions of X and of the same-shaped view Y so that X
// becomes that dense layout (returned as `dense`, Y's matching view as
// `src`); extent-1 dimensions are dropped.  Returns false otherwise.
static bool invert_view(const View& X, const View& Y, View& dense, View& src) {
  if (X.off != 0 || X.nd != Y.nd) return false;
  int idx[kMaxDim];
  int nd = 0;
  for (int d = 0; d < X.nd; ++d) {
    if (X.shape[d] != Y.shape[d]) return false;
    if (X.shape[d] == 0) return false;
    if (X.shape[d] > 1) idx[nd++] = d;
  }
  std::stable_sort(idx, idx + nd, [&](int p, int q) { return X.stride[p] > X.stride[q]; });
  long long expect = 1;
  for (int k = nd - 1; k >= 0; --k) {
    if (X.stride[idx[k]] != expect) return false;
    expect *= X.shape[idx[k]];
  }
  dense = View();
  dense.node = X.node;
  dense.off = 0;
  src = View();
  src.node = Y.node;
  src.off = Y.off;
  dense.nd = src.nd = nd > 0 ? nd : 1;
  if (nd == 0) {
    dense.shape[0] = src.shape[0] = 1;
    dense.stride[0] = src.stride[0] = 1;
  }
  for (int k = 0; k < nd; ++k) {
    dense.shape[k] = src.shape[k] = X.shape[idx[k]];
    dense.stride[k] = X.stride[idx[k]];
    src.stride[k] = Y.stride[idx[k]];
  }
  return true;
}

template <typename R>
void launch_fill(Cx<R>* p, size_t n, double re, double im, cudaStream_t s) {
  if (n == 0) return;
  k_fill<R><<<grid_for(n), 256, 0, s>>>(p, n, R(re), R(im));
}

template <typename R>
Engine<R>::~Engine() {
  if (canary_list_) cudaFree(canary_list_);
  if (side_) cudaStreamDestroy(side_);
  if (fork_ev_) cudaEventDestroy(fork_ev_);
  if (join_ev_) cudaEventDestroy(join_ev_);
  if (branch_) cudaStreamDestroy(branch_);
  if (branch_fork_) cudaEventDestroy(branch_fork_);
  if (branch_join_) cudaEventDestroy(branch_join_);
  if (region_) cudaStreamDestroy(region_);
  if (region_fork_) cudaEventDestroy(region_fork_);
  if (region_join_) cudaEventDestroy(region_join_);
  if (pool_) return;  // everything lives in the caller's pool
  for (auto& kv : plans_)
    if (kv.second->dev) cudaFree(kv.second->dev);
  for (int s = 0; s < kScratchSlots; ++s)
    if (scratch_[s]) cudaFree(scratch_[s]);
  if (err_) cudaFree(err_);
}

template <typename R>
cudaStream_t Engine<R>::side_stream() {
  if (pool_) return stream_;
  if (!side_) {
    RTCC3_CUDA(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking));
    RTCC3_CUDA(cudaEventCreateWithFlags(&fork_ev_, cudaEventDisableTiming));
    RTCC3_CUDA(cudaEventCreateWithFlags(&join_ev_, cudaEventDisableTiming));
  }
  return side_;
}

template <typename R>
void Engine<R>::fork() {
  cudaStream_t s = side_stream();
  if (s == stream_) return;
  RTCC3_CUDA(cudaEventRecord(fork_ev_, stream_));
  RTCC3_CUDA(cudaStreamWaitEvent(s, fork_ev_, 0));
}

template <typename R>
void Engine<R>::join() {
  if (!side_ || pool_) return;
  RTCC3_CUDA(cudaEventRecord(join_ev_, side_));
  RTCC3_CUDA(cudaStreamWaitEvent(stream_, join_ev_, 0));
}

template <typename R>
int* Engine<R>::error_flag() {
  if (!err_) {
    if (pool_) {
      err_ = static_cast<int*>(pool_->take(sizeof(int)));
      RTCC3_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), stream_));
    } else {
      RTCC3_CUDA(cudaMalloc(&err_, sizeof(int)));
      RTCC3_CUDA(cudaMemset(err_, 0, sizeof(int)));
    }
  }
  return err_;
}

template <typename R>
void Engine<R>::begin() {
  tc_region_ = false;
  // a stage abandoned inside a concurrent region (an error) leaves it here
  if (in_region_) region_leave();
  region_pending_ = false;
  if (branch_state_ != 0) {
    stream_ = branch_main_;
    split_slot_ = 0;
    tc_slot_ = 1;
    branch_state_ = 0;
  }
  arena_.reset();
  nodes_.clear();
  tape_.clear();
  canaries_.clear();
}

// Every element a view (moved by `shift` elements) addresses lies inside its
// node: checked on the host for every operation before it is launched, so a
// planning error is reported (kErrState) instead of reaching memory.
template <typename R>
void Engine<R>::check_view(const View& v, long long shift, const char* what) const {
  RTCC3_CHECK(v.node >= 0 && v.node < int(nodes_.size()), kErrState,
              std::string("view of an unknown tensor in ") + what);
  if (v.numel() == 0) return;
  long long lo = v.off + shift, hi = v.off + shift;
  for (int d = 0; d < v.nd; ++d) {
    const long long span = (long long)(v.shape[d] - 1) * v.stride[d];
    if (span < 0) lo += span; else hi += span;
  }
  RTCC3_CHECK(lo >= 0 && hi < (long long)nodes_[v.node].numel, kErrState,
              std::string("view outside its tensor in ") + what + " (elements " +
                  std::to_string(lo) + ".." + std::to_string(hi) + " of " +
                  std::to_string(nodes_[v.node].numel) + ")");
}

namespace {
constexpr unsigned char kCanary = 0xA5;
constexpr size_t kCanaryBytes = 256;

// One block per guarded tensor: every byte of its canary must still hold the
// pattern written when the tensor was created.
__global__ void k_check_canaries(unsigned char* const* __restrict__ pads, int* __restrict__ flag) {
  const unsigned char* p = pads[blockIdx.x];
  bool bad = false;
  for (size_t t = threadIdx.x; t < kCanaryBytes; t += blockDim.x) bad |= p[t] != kCanary;
  if (bad) atomicOr(flag, 1);
}
}  // namespace

template <typename R>
void Engine<R>::verify_canaries(int* flag) {
  if (canaries_.empty()) return;
  const size_t bytes = canaries_.size() * sizeof(unsigned char*);
  if (bytes > canary_list_bytes_) {
    if (canary_list_) cudaFree(canary_list_);
    canary_list_ = nullptr;
    RTCC3_CUDA(cudaMalloc(&canary_list_, bytes));
    canary_list_bytes_ = bytes;
  }
  RTCC3_CUDA(cudaMemcpyAsync(canary_list_, canaries_.data(), bytes, cudaMemcpyHostToDevice, stream_));
  k_check_canaries<<<int(canaries_.size()), 128, 0, stream_>>>(
      static_cast<unsigned char* const*>(canary_list_), flag);
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
  // the host list must outlive the copy
  RTCC3_CUDA(cudaStreamSynchronize(stream_));
}

template <typename R>
int Engine<R>::node(const std::vector<int>& shape, bool needs_grad, bool zero) {
  Node nd;
  nd.shape = shape;
  nd.numel = 1;
  for (int s : shape) nd.numel *= size_t(s);
  RTCC3_CHECK((int)shape.size() <= kMaxDim, kErrArg, "tensor rank too large");
  nd.data = static_cast<C*>(arena_.alloc(nd.numel * sizeof(C) + (checked_ ? kCanaryBytes : 0)));
  if (zero) RTCC3_CUDA(cudaMemsetAsync(nd.data, 0, nd.numel * sizeof(C), stream_));
  if (checked_) {
    // canary right after the tensor (checked mode): verified after the stage
    unsigned char* pad = reinterpret_cast<unsigned char*>(nd.data + nd.numel);
    RTCC3_CUDA(cudaMemsetAsync(pad, kCanary, kCanaryBytes, stream_));
    canaries_.push_back(pad);
  }
  nd.needs_grad = needs_grad;
  nodes_.push_back(nd);
  return int(nodes_.size()) - 1;
}

template <typename R>
int Engine<R>::external(C* data, const std::vector<int>& shape) {
  Node nd;
  nd.shape = shape;
  nd.numel = 1;
  for (int s : shape) nd.numel *= size_t(s);
  nd.data = data;
  nd.needs_grad = false;
  nodes_.push_back(nd);
  return int(nodes_.size()) - 1;
}

template <typename R>
View Engine<R>::v(int n) const {
  const Node& nd = nodes_[n];
  View r;
  r.node = n;
  r.off = 0;
  r.nd = int(nd.shape.size());
  long long st = 1;
  for (int d = r.nd - 1; d >= 0; --d) {
    r.shape[d] = nd.shape[d];
    r.stride[d] = st;
    st *= nd.shape[d];
  }
  return r;
}

template <typename R>
View Engine<R>::ev(const char* spec_c, const View& x) const {
  const std::string spec(spec_c);
  const size_t arrow = spec.find("->");
  RTCC3_CHECK(arrow != std::string::npos, kErrArg, "bad view spec");
  const std::string in = spec.substr(0, arrow), out = spec.substr(arrow + 2);
  RTCC3_CHECK((int)in.size() == x.nd, kErrArg, "view spec rank mismatch: " + spec);
  View r;
  r.node = x.node;
  r.off = x.off;
  r.nd = int(out.size());
  for (int d = 0; d < r.nd; ++d) {
    long long st = 0;
    int ext = -1;
    for (int k = 0; k < x.nd; ++k)
      if (in[k] == out[d]) {
        st += x.stride[k];
        RTCC3_CHECK(ext < 0 || ext == x.shape[k], kErrArg, "diagonal extents differ: " + spec);
        ext = x.shape[k];
      }
    RTCC3_CHECK(ext >= 0, kErrArg, "view output letter missing: " + spec);
    r.shape[d] = ext;
    r.stride[d] = st;
  }
  for (size_t k = 0; k < in.size(); ++k)
    RTCC3_CHECK(out.find(in[k]) != std::string::npos, kErrArg, "view drops a letter: " + spec);
  return r;
}

template <typename R>
void* Engine<R>::scratch(int slot, size_t bytes) {
  if (bytes > scratch_bytes_[slot]) {
    RTCC3_CHECK(!frozen_, kErrState, "scratch growth during graph capture");
    if (pool_) {
      scratch_[slot] = pool_->take(bytes);
      scratch_bytes_[slot] = bytes;
      ++generation_;
      return scratch_[slot];
    }
    if (scratch_[slot]) cudaFree(scratch_[slot]);
    scratch_[slot] = nullptr;
    RTCC3_CUDA(cudaMalloc(&scratch_[slot], bytes));
    scratch_bytes_[slot] = bytes;
    ++generation_;
  }
  return scratch_[slot];
}

// Resident CTAs per SM of the k_contract instantiation a plan launches
// (registers decide it; cached per tile shape and operand layout).
template <typename R>
int simt_ctas_per_sm(bool small_tile, int tile, bool akc, bool bkc) {
  static int cache[4][2][2] = {};
  int& c = cache[small_tile ? 3 : tile][akc ? 1 : 0][bkc ? 1 : 0];
  if (c > 0) return c;
  auto q = [&](auto kern) {
    RTCC3_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kern, kThreads, 0));
  };
#define RTCC3_OCC(TBM, TBN, TBK, TTM, TTN)                                       \
  if (akc && bkc) q(k_contract<R, true, true, TBM, TBN, TBK, TTM, TTN>);        \
  else if (akc) q(k_contract<R, true, false, TBM, TBN, TBK, TTM, TTN>);         \
  else if (bkc) q(k_contract<R, false, true, TBM, TBN, TBK, TTM, TTN>);         \
  else q(k_contract<R, false, false, TBM, TBN, TBK, TTM, TTN>)
  if (small_tile) {
    RTCC3_OCC(kSBM, kSBM, kSBK, 1, 1);
  } else if (tile == 1) {
    RTCC3_OCC(16, 256, kTBK, 4, 4);
  } else if (tile == 2) {
    RTCC3_OCC(256, 16, kTBK, 4, 4);
  } else {
    RTCC3_OCC(kBM, kBN, kBK, 4, 4);
  }
#undef RTCC3_OCC
  c = std::max(c, 1);
  return c;
}

template <typename R>
ContractPlan& Engine<R>::plan(const std::string& spec, const View& A, const View& B, const View& Cv) {
  // tensor cores only inside the tensor-core region (the triples): the
  // split-TF32 products (about 5e-7 relative) are accurate enough for the
  // small triples terms, not for the CCSD part at its full magnitude
  const bool tc_ok = cur_tc_ && tc_eb_ > 0;
  const std::string key = spec + "|" + view_key(A) + "|" + view_key(B) + "|" + view_key(Cv) +
                          (tc_ok ? "|tc" : "");
  auto it = plans_.find(key);
  if (it != plans_.end()) return *it->second;
  RTCC3_CHECK(!frozen_, kErrState, "new contraction plan during graph capture: " + spec);
  const Spec s = parse(spec);
  RTCC3_CHECK((int)s.a.size() == A.nd && (int)s.b.size() == B.nd && (int)s.c.size() == Cv.nd,
              kErrArg, "contraction rank mismatch: " + spec);
  struct Letter { char ch; int ext; long long sa, sb, sc; bool ia, ib, ic; };
  std::vector<Letter> letters;
  auto find = [&](char ch) -> Letter& {
    for (auto& l : letters) if (l.ch == ch) return l;
    letters.push_back({ch, -1, 0, 0, 0, false, false, false});
    return letters.back();
  };
  auto add = [&](const std::string& str, const View& vw, int which) {
    for (int d = 0; d < (int)str.size(); ++d) {
      Letter& l = find(str[d]);
      bool& seen = which == 0 ? l.ia : (which == 1 ? l.ib : l.ic);
      RTCC3_CHECK(!seen, kErrArg, "repeated index in one operand (use a diagonal view): " + spec);
      seen = true;
      RTCC3_CHECK(l.ext < 0 || l.ext == vw.shape[d], kErrArg, "extent mismatch in " + spec);
      l.ext = vw.shape[d];
      (which == 0 ? l.sa : (which == 1 ? l.sb : l.sc)) = vw.stride[d];
    }
  };
  add(s.a, A, 0);
  add(s.b, B, 1);
  add(s.c, Cv, 2);
  std::vector<Letter> gb, gm, gn, gk;
  for (char ch : s.c) {
    Letter& l = find(ch);
    if (l.ia && l.ib) gb.push_back(l);
    else if (l.ia) gm.push_back(l);
    else if (l.ib) gn.push_back(l);
    else throw Error(kErrArg, "output index in no operand: " + spec);
  }
  for (auto& l : letters) {
    if (l.ic) continue;
    RTCC3_CHECK(l.ia && l.ib, kErrArg, "index summed in one operand only: " + spec);
    gk.push_back(l);
  }
  // Letter order inside each group: the larger of the two tensors that carry
  // the group decides (its smallest stride fastest), so the loads or stores
  // of the big tensor run along its contiguous index.
  const double nA = double(A.numel()), nB = double(B.numel()), nC = double(Cv.numel());
  auto by = [](int which) {
    return [which](const Letter& x, const Letter& y) {
      const long long sx = which == 0 ? x.sa : (which == 1 ? x.sb : x.sc);
      const long long sy = which == 0 ? y.sa : (which == 1 ? y.sb : y.sc);
      return std::llabs(sx) > std::llabs(sy);
    };
  };
  std::stable_sort(gk.begin(), gk.end(), by(nA >= nB ? 0 : 1));
  std::stable_sort(gm.begin(), gm.end(), by(nA > nC ? 0 : 2));
  std::stable_sort(gn.begin(), gn.end(), by(nB > nC ? 1 : 2));
  auto P = std::make_unique<ContractPlan>();
  auto count = [](const std::vector<Letter>& g) {
    long long n = 1;
    for (auto& l : g) n *= l.ext;
    return n;
  };
  const long long M = count(gm), N = count(gn), K = count(gk), NB = count(gb);
  RTCC3_CHECK(M < (1LL << 31) && N < (1LL << 31) && K < (1LL << 31) && NB < (1LL << 31), kErrArg,
              "contraction too large: " + spec);
  P->M = int(M); P->N = int(N); P->K = int(K); P->nb = int(NB);
  // tables (row-major decode over each group, last letter fastest)
  auto table = [](const std::vector<Letter>& g, int which, std::vector<long long>& out) {
    long long n = 1;
    for (auto& l : g) n *= l.ext;
    const size_t base = out.size();
    out.resize(base + size_t(n));
    for (long long t = 0; t < n; ++t) {
      long long rem = t, off = 0;
      for (int k = int(g.size()) - 1; k >= 0; --k) {
        const long long i = rem % g[k].ext;
        rem /= g[k].ext;
        off += i * (which == 0 ? g[k].sa : (which == 1 ? g[k].sb : g[k].sc));
      }
      out[base + size_t(t)] = off;
    }
    return base;
  };
  std::vector<long long>& h = P->host;
  const size_t iaM = table(gm, 0, h), iaK = table(gk, 0, h), ibN = table(gn, 1, h),
               ibK = table(gk, 1, h), icM = table(gm, 2, h), icN = table(gn, 2, h);
  const size_t iaB = table(gb, 0, h), ibB = table(gb, 1, h), icB = table(gb, 2, h);
  for (size_t t = iaB; t < iaB + size_t(NB); ++t) h[t] += A.off;
  for (size_t t = ibB; t < ibB + size_t(NB); ++t) h[t] += B.off;
  for (size_t t = icB; t < icB + size_t(NB); ++t) h[t] += Cv.off;
  P->a_kcontig = !gk.empty() && std::llabs(gk.back().sa) == 1;
  P->b_kcontig = !gk.empty() && std::llabs(gk.back().sb) == 1;
  if (pool_) {
    // tables go into the pool; the host copy lives in the plan until the
    // engine is destroyed, after the stream has drained
    P->dev = pool_->take(h.size() * sizeof(long long));
    RTCC3_CUDA(cudaMemcpyAsync(P->dev, h.data(), h.size() * sizeof(long long),
                               cudaMemcpyHostToDevice, stream_));
  } else {
    RTCC3_CUDA(cudaMalloc(&P->dev, h.size() * sizeof(long long)));
    RTCC3_CUDA(cudaMemcpy(P->dev, h.data(), h.size() * sizeof(long long), cudaMemcpyHostToDevice));
  }
  long long* d = static_cast<long long*>(P->dev);
  P->aM = d + iaM; P->aK = d + iaK; P->bN = d + ibN; P->bK = d + ibK;
  P->cM = d + icM; P->cN = d + icN; P->aB = d + iaB; P->bB = d + ibB; P->cB = d + icB;
  P->a_off0 = h[iaB];
  P->b_off0 = h[ibB];
  P->c_off0 = h[icB];
  // small outputs (held whole by every CTA, K split over the GPU) and single
  // long output columns get their own kernels
  {
    const long long mx = std::max(M, N), mn = std::min(M, N);
    if (NB == 1 && K == 1 && M * N >= 65536) {
      // outer product: a streaming pass over C with n on its contiguous index
      P->kind = 3;
      P->small_swap = !gm.empty() && std::llabs(gm.back().sc) == 1;
    } else if (NB == 1 && mn == 1 && mx > 512 && K <= 65536) {
      P->kind = 2;
      P->small_swap = M == 1;
      P->gemv_boff = P->small_swap ? P->a_off0 + h[iaM] : P->b_off0 + h[ibN];
      P->gemv_coff = P->c_off0 + (P->small_swap ? h[icM] : h[icN]);
    } else if (NB == 1 && K >= 256 && small_output_config(mx, mn) != kSmallNone) {
      P->kind = 1;
      P->small_cfg = small_output_config(mx, mn);
      P->small_swap = N > M;
      const int bk = small_output_bk(P->small_cfg, int(sizeof(C)));
      const long long want = 4 * 152;
      const long long maxs = (K + 4 * bk - 1) / (4 * bk);  // at least four slices per CTA
      int ns = int(std::max<long long>(1, std::min(want, maxs)));
      int kc = int((K + ns - 1) / ns);
      kc = ((kc + bk - 1) / bk) * bk;
      P->nsplit = int((K + kc - 1) / kc);
      P->kchunk = kc;
    }
  }
  if (P->kind != 0) {
    ContractPlan& ref = *P;
    plans_[key] = std::move(P);
    return ref;
  }
  // tile shape: 64 x 64; 16 x 256 (256 x 16) when one side is at most 16;
  // 16 x 16 with 64-deep K slices for small outputs with long sums, and for
  // small products whose whole sum is one such slice (more CTAs, one pass)
  P->small_tile = std::max(M, N) <= 48 && (K >= 1024 || K <= kSBK);
  if (!P->small_tile && M <= 16 && N > 64) P->tile = 1;
  else if (!P->small_tile && N <= 16 && M > 64) P->tile = 2;
  int bmm = kBM, bnn = kBN, bk = kBK;
  if (P->small_tile) { bmm = bnn = kSBM; bk = kSBK; }
  else if (P->tile == 1) { bmm = 16; bnn = 256; bk = kTBK; }
  else if (P->tile == 2) { bmm = 256; bnn = 16; bk = kTBK; }
  // split-K when the output tiles alone do not fill the GPU: from about four
  // CTAs per SM up, the fewest splits (each at least four K slices) whose
  // CTAs fill their last wave of resident CTAs to 90 %, else the best-filled
  // count
  const long long tiles = ((M + bmm - 1) / bmm) * ((N + bnn - 1) / bnn) * NB;
  int nsplit = 1;
  if (tiles < 2 * 152 && K > 4 * bk) {
    const long long maxs = (K + 4 * bk - 1) / (4 * bk);
    const long long slots = 152LL * simt_ctas_per_sm<R>(P->small_tile, P->tile, P->a_kcontig,
                                                         P->b_kcontig);
    // at least enough splits for four CTAs per SM (more CTAs hide latency)
    const long long want = std::min(maxs, (4 * 152 + tiles - 1) / tiles);
    double best_eff = -1.0;
    for (long long ns = std::max<long long>(1, want); ns <= maxs; ++ns) {
      long long kc = (K + ns - 1) / ns;
      kc = ((kc + bk - 1) / bk) * bk;
      const long long used = (K + kc - 1) / kc;
      const long long ctas = tiles * used, waves = (ctas + slots - 1) / slots;
      const double eff = double(ctas) / double(waves * slots);
      if (eff >= 0.9 && ctas >= slots) {
        nsplit = int(used);
        break;
      }
      if (eff > best_eff + 1e-9) {
        best_eff = eff;
        nsplit = int(used);
      }
    }
  }
  int kchunk = int((K + nsplit - 1) / nsplit);
  kchunk = ((kchunk + bk - 1) / bk) * bk;
  nsplit = int((K + kchunk - 1) / kchunk);
  P->nsplit = nsplit;
  P->kchunk = kchunk;
  // tensor-core route: one batch, a large output side and enough work
  // (a short K would make the packed operands cost more traffic than the
  // product saves: those stay on CUDA cores)
  // With split TF32 operands (FP32-level products) short sums that write a
  // large output (outer-product-like, e.g. the connected triples Z) go to
  // the tensor cores too: their packed operands are small and the product
  // is bound by the output write.  BF16 keeps them on the CUDA cores (FP32),
  // so the connected triples stay accurate enough for the amplitude
  // equations to converge.
  const long long kp_tc = tc_ok ? 2LL * tc_packed_k(int(K), 4) : 0;
  const bool long_k = K >= 64 && M * N * K >= (1LL << 21);
  const bool out_bound = tc_eb_ == 4 && M * N >= (1LL << 22) && M * N >= 2 * (M + 2 * N) * kp_tc;
  if (std::is_same<R, float>::value && tc_ok && NB == 1 && std::max(M, N) >= 128 &&
      std::min(M, N) >= 4 && (long_k || out_bound)) {
    P->use_tc = true;
    // long sums: the expanded (2x2 real) operand is the smaller one; short
    // sums: the output's contiguous index goes to the GEMM columns, which
    // the epilogue stores in runs
    const bool c_unit_m = !gm.empty() && std::llabs(gm.back().sc) == 1;
    P->tc_swap = long_k ? (N > M) : c_unit_m;
    P->tc_out = !long_k;
    const long long Mg = P->tc_swap ? N : M, Ng = P->tc_swap ? M : N;
    P->tc_kp = tc_packed_k(int(K), tc_eb_);
    const int nkb = P->tc_kp / (128 / tc_eb_);
    const long long nr = 2 * Ng;
    const long long bn = tc_tile_n(int(std::min<long long>(nr, 1 << 30)), P->tc_out);
    const long long tcs = ((nr + bn - 1) / bn) * ((Mg + 127) / 128);
    // split K so that the CTAs fill whole waves of the GPU (each split sums
    // at least 32 K tiles; a larger split must gain 3% of wave occupancy)
    int ts = 1;
    if (!P->tc_out && nkb >= 64) {
      const long long slots = 152LL * tc_ctas_per_sm(false);
      double best = double(tcs) / double(((tcs + slots - 1) / slots) * slots);
      for (int c = 2; c <= nkb / 32 && c <= 64; ++c) {
        const long long ctas = tcs * c;
        const double eff = double(ctas) / double(((ctas + slots - 1) / slots) * slots);
        if (eff > best + 0.03) {
          best = eff;
          ts = c;
        }
      }
    }
    // bounded accumulation chains: the tensor-core FP32 accumulator adds
    // every product of a CTA's K range in place, and its error grows with
    // the chain length, so no split sums more than 64 K tiles; the splits
    // are added in FP32 by tc_split_finish
    if (!P->tc_out) ts = std::max(ts, (nkb + kTcMaxKbPerSplit - 1) / kTcMaxKbPerSplit);
    P->tc_nsplit = ts;
  }
  ContractPlan& ref = *P;
  plans_[key] = std::move(P);
  return ref;
}

template <typename R>
void Engine<R>::run_contract(const std::string& spec, double alpha, const View& A, bool a_grad,
                             const View& B, bool b_grad, const View& Cv, bool c_grad,
                             bool accumulate, long long sa, long long sb, long long sc) {
  ContractPlan& P = plan(spec, A, B, Cv);
  if (prof_ && prof_->detail())
    cur_detail_ = spec + " M=" + std::to_string(P.M) + " N=" + std::to_string(P.N) +
                  " K=" + std::to_string(P.K) + (P.use_tc ? (P.tc_swap ? " tc-swap" : " tc") : "");
  if ((a_grad && !nodes_[A.node].grad_ready) || (b_grad && !nodes_[B.node].grad_ready)) {
    // a cotangent never written is zero: nothing to add; an overwriting
    // product needs its zeros, so the cotangent is zero-filled first
    if (accumulate) return;
    if (a_grad) zero_grad_if_unset(A.node);
    if (b_grad) zero_grad_if_unset(B.node);
  }
  if (c_grad) accumulate = begin_grad_write(Cv, accumulate);
  const C* pa = (a_grad ? nodes_[A.node].grad : nodes_[A.node].data);
  const C* pb = (b_grad ? nodes_[B.node].grad : nodes_[B.node].data);
  C* pc = (c_grad ? nodes_[Cv.node].grad : nodes_[Cv.node].data);
  RTCC3_CHECK(pa && pb && pc, kErrState, "contraction on an unallocated buffer: " + spec);
  check_view(A, sa, spec.c_str());
  check_view(B, sb, spec.c_str());
  check_view(Cv, sc, spec.c_str());
  pa += sa;
  pb += sb;
  pc += sc;
  if (P.use_tc) {
    run_contract_tc(P, alpha, pa, pb, pc, accumulate);
    return;
  }
  if (P.kind != 0) {
    run_contract_small(P, alpha, pa, pb, pc, accumulate);
    return;
  }
  C* part = nullptr;
  if (P.nsplit > 1)
    part = static_cast<C*>(scratch(split_slot_, size_t(P.nb) * P.nsplit * P.M * P.N * sizeof(C)));
  int bmm = kBM, bnn = kBN;
  if (P.small_tile) bmm = bnn = kSBM;
  else if (P.tile == 1) { bmm = 16; bnn = 256; }
  else if (P.tile == 2) { bmm = 256; bnn = 16; }
  dim3 grid((P.N + bnn - 1) / bnn, (P.M + bmm - 1) / bmm, P.nb * P.nsplit);
  RTCC3_CHECK(grid.y < 65536 && grid.z < 65536, kErrArg, "contraction grid too large: " + spec);
  const int pk = pbegin();
#define RTCC3_LAUNCH(AK, BK, TBM, TBN, TBK, TTM, TTN)                                            \
  k_contract<R, AK, BK, TBM, TBN, TBK, TTM, TTN><<<grid, kThreads, 0, stream_>>>(                \
      pa, pb, pc, P.aM, P.aK, P.bN, P.bK, P.cM, P.cN, P.aB, P.bB, P.cB, P.M, P.N, P.K, P.nsplit, \
      P.kchunk, R(alpha), accumulate ? 1 : 0, part)
#define RTCC3_LAUNCH4(...)                                                       \
  if (P.a_kcontig && P.b_kcontig) RTCC3_LAUNCH(true, true, __VA_ARGS__);          \
  else if (P.a_kcontig) RTCC3_LAUNCH(true, false, __VA_ARGS__);                  \
  else if (P.b_kcontig) RTCC3_LAUNCH(false, true, __VA_ARGS__);                  \
  else RTCC3_LAUNCH(false, false, __VA_ARGS__)
  if (P.small_tile) {
    RTCC3_LAUNCH4(kSBM, kSBM, kSBK, 1, 1);
  } else if (P.tile == 1) {
    RTCC3_LAUNCH4(16, 256, kTBK, 4, 4);
  } else if (P.tile == 2) {
    RTCC3_LAUNCH4(256, 16, kTBK, 4, 4);
  } else {
    RTCC3_LAUNCH4(kBM, kBN, kBK, 4, 4);
  }
#undef RTCC3_LAUNCH4
#undef RTCC3_LAUNCH
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
  {
    const double mnk = double(P.M) * P.N * P.K * P.nb;
    const double bytes = (double(P.M) * P.K + double(P.N) * P.K +
                          double(P.M) * P.N * (accumulate ? 2.0 : 1.0)) * P.nb * sizeof(C);
    pend(pk, sizeof(R) == 8 ? "contract_simt_c128" : "contract_simt_c64", 8.0 * mnk, bytes,
         cur_detail_);
  }
  if (P.nsplit > 1) {
    const size_t n = size_t(P.nb) * P.M * P.N;
    const int pr = pbegin();
    k_split_reduce<R><<<grid_for(n), 256, 0, stream_>>>(part, pc, P.cM, P.cN, P.cB, P.M, P.N, P.nb,
                                                        P.nsplit, R(alpha), accumulate ? 1 : 0);
    ++launches_;
    RTCC3_CUDA(cudaGetLastError());
    pend(pr, "split_reduce", 2.0 * n * P.nsplit, double(n) * (P.nsplit + 2) * sizeof(C));
  }
}

template <typename R>
void Engine<R>::run_contract_small(ContractPlan& P, double alpha, const C* pa, const C* pb, C* pc,
                                   bool accumulate) {
  const bool sw = P.small_swap;
  const int Mk = sw ? P.N : P.M, Nk = sw ? P.M : P.N;
  const long long* kM = sw ? P.cN : P.cM;
  const long long* kN = sw ? P.cM : P.cN;
  const double mnk = double(P.M) * P.N * P.K;
  const double bytes = (double(P.M) * P.K + double(P.N) * P.K +
                        double(P.M) * P.N * (accumulate ? 2.0 : 1.0)) * sizeof(C);
  const char* tag = sizeof(R) == 8 ? "c128" : "c64";
  if (P.kind == 3) {
    const int pk = pbegin();
    launch_outer<R>(sw ? pb : pa, sw ? P.b_off0 : P.a_off0, sw ? P.bN : P.aM, sw ? P.bK : P.aK,
                    sw ? pa : pb, sw ? P.a_off0 : P.b_off0, sw ? P.aM : P.bN, sw ? P.aK : P.bK,
                    pc, P.c_off0, kM, kN, Mk, Nk, alpha, accumulate, stream_);
    ++launches_;
    pend(pk, (std::string("contract_outer_") + tag).c_str(), 8.0 * mnk, bytes, cur_detail_);
    return;
  }
  if (P.kind == 2) {
    const int pk = pbegin();
    launch_gemv<R>(sw ? P.b_kcontig : P.a_kcontig, sw ? pb : pa, sw ? P.b_off0 : P.a_off0,
                   sw ? P.bN : P.aM, sw ? P.bK : P.aK, sw ? pa : pb, P.gemv_boff, sw ? P.aK : P.bK,
                   pc, P.gemv_coff, kM, Mk, P.K, alpha, accumulate, stream_);
    ++launches_;
    pend(pk, (std::string("contract_gemv_") + tag).c_str(), 8.0 * mnk, bytes, cur_detail_);
    return;
  }
  C* part = nullptr;
  if (P.nsplit > 1)
    part = static_cast<C*>(scratch(split_slot_, size_t(P.nsplit) * P.M * P.N * sizeof(C)));
  const int pk = pbegin();
  launch_reduce_small<R>(P.small_cfg, sw ? P.b_kcontig : P.a_kcontig, sw ? P.a_kcontig : P.b_kcontig,
                         sw ? pb : pa, sw ? P.b_off0 : P.a_off0, sw ? P.bN : P.aM, sw ? P.bK : P.aK,
                         sw ? pa : pb, sw ? P.a_off0 : P.b_off0, sw ? P.aM : P.bN, sw ? P.aK : P.bK,
                         pc, P.c_off0, kM, kN, Mk, Nk, P.K, P.nsplit, P.kchunk, alpha, accumulate,
                         part, stream_);
  launches_ += P.nsplit > 1 ? 2 : 1;
  pend(pk, (std::string("contract_small_") + tag).c_str(), 8.0 * mnk, bytes, cur_detail_);
}

template <typename R>
void Engine<R>::run_contract_tc(ContractPlan& P, double alpha, const C* pa, const C* pb, C* pc,
                                bool accumulate) {
  if constexpr (std::is_same<R, float>::value) {
    const bool sw = P.tc_swap;
    TcOperands op;
    op.M = sw ? P.N : P.M;
    op.N = sw ? P.M : P.N;
    op.K = P.K;
    op.Kp = P.tc_kp;
    op.elem_bytes = tc_eb_;
    op.split = tc_eb_ == 4;
    op.out_bound = P.tc_out;
    op.wait_budget = wait_budget_;
    const float2* ga = sw ? pb : pa;
    const float2* gb = sw ? pa : pb;
    const long long* gaM = sw ? P.bN : P.aM;
    const long long* gaK = sw ? P.bK : P.aK;
    const long long* gbN = sw ? P.aM : P.bN;
    const long long* gbK = sw ? P.aK : P.bK;
    const long long* gcM = sw ? P.cN : P.cM;
    const long long* gcN = sw ? P.cM : P.cN;
    const long long goa = sw ? P.b_off0 : P.a_off0;
    const long long gob = sw ? P.a_off0 : P.b_off0;
    // TF32 long sums read the big operand A straight from its source (no
    // packed copy); the others pack A (tiled for chained long sums)
    const bool direct = tc_direct(op, P.tc_nsplit);
    op.a_tiled = !direct && tc_chained(op, P.tc_nsplit);
    const size_t a_rows = op.a_tiled ? size_t((op.M + 127) / 128) * 128 : size_t(op.M);
    void* apk = direct ? nullptr : scratch(tc_slot_, a_rows * op.Kp * tc_eb_);
    void* bpk = scratch(tc_slot_ + 1, size_t(2 * op.N) * op.Kp * tc_eb_ * (op.split ? 2 : 1));
    float* part = nullptr;
    if (P.tc_nsplit > 1)
      part = static_cast<float*>(
          scratch(tc_slot_ + 2, size_t(P.tc_nsplit) * op.M * 2 * op.N * sizeof(float)));
    int* err = error_flag();
    const bool a_kc = sw ? P.b_kcontig : P.a_kcontig;
    const double rows_packed = direct ? 2.0 * op.N : op.M + 2.0 * op.N;
    int pk = pbegin();
    if (!direct) tc_pack_a(ga, gaM, gaK, goa, op.M, op.K, op.Kp, tc_eb_, a_kc, op.a_tiled, apk, stream_);
    tc_pack_b(gb, gbN, gbK, gob, op.N, op.K, op.Kp, tc_eb_, sw ? P.a_kcontig : P.b_kcontig, bpk,
              stream_);
    pend(pk, "tc_pack", 0.0, rows_packed * op.K * 8.0 + rows_packed * op.Kp * tc_eb_, cur_detail_);
    launches_ += direct ? 1 : 2;
    pk = pbegin();
    const bool ok = direct ? tc_gemm_direct(ga, goa, gaM, gaK, a_kc, bpk, op, P.tc_nsplit, part,
                                            err, stream_)
                           : tc_gemm(apk, bpk, op, pc, gcM, gcN, P.c_off0, float(alpha),
                                     accumulate, P.tc_nsplit, part, err, stream_);
    RTCC3_CHECK(ok, kErrCuda, "tensor-core GEMM set-up failed (tensor map encoding)");
    const double mnk = double(op.M) * op.N * op.K;
    const double bytes = (direct ? double(op.M) * op.K * 8.0 : double(op.M) * op.Kp * tc_eb_) +
                         2.0 * op.N * op.Kp * tc_eb_ * (op.split ? 2 : 1) +
                         (P.tc_nsplit > 1 ? double(P.tc_nsplit) * op.M * 2 * op.N * 4.0
                                          : double(op.M) * op.N * sizeof(C) * (accumulate ? 2.0 : 1.0));
    pend(pk, direct ? "contract_tc_direct_tf32" : (tc_eb_ == 4 ? "contract_tc_tf32" : "contract_tc_bf16"),
         8.0 * mnk, bytes, cur_detail_);
    ++launches_;
    if (P.tc_nsplit > 1) {
      pk = pbegin();
      tc_split_finish(part, P.tc_nsplit, op.M, op.N, pc, gcM, gcN, P.c_off0, float(alpha),
                      accumulate, stream_);
      pend(pk, "tc_split_finish", 0.0,
           double(P.tc_nsplit) * op.M * 2 * op.N * 4.0 + double(op.M) * op.N * sizeof(C) * 2.0);
      ++launches_;
    }
  } else {
    (void)P; (void)alpha; (void)pa; (void)pb; (void)pc; (void)accumulate;
    throw Error(kErrState, "tensor-core route requires a complex64 graph");
  }
}

template <typename R>
void Engine<R>::contract(const char* spec, double alpha, const View& A, const View& B,
                         const View& Cv, bool accumulate) {
  RTCC3_CHECK(Cv.node != A.node && Cv.node != B.node, kErrArg, "contraction output aliases input");
  cur_tc_ = tc_region_;
  run_contract(spec, alpha, A, false, B, false, Cv, false, accumulate);
  if (nodes_[A.node].needs_grad || nodes_[B.node].needs_grad) nodes_[Cv.node].needs_grad = true;
  Op op{kContract, spec, alpha, A, B, Cv, EpsSpec()};
  op.tc = tc_region_;
  tape_.push_back(op);
}

template <typename R>
void Engine<R>::run_axpy(double alpha, const View& X, bool xg, const View& Y, bool yg) {
  run_combine(&X, &xg, &alpha, 1, Y, yg, false, "axpy_strided");
}

template <typename R>
void Engine<R>::run_combine(const View* xs, const bool* xg, const double* alphas, int ns,
                            const View& Y, bool yg, bool overwrite, const char* name) {
  RTCC3_CHECK(ns >= 1 && ns <= kMaxSrc, kErrArg, "combine takes 1..8 sources");
  for (int k = 0; k < ns; ++k) check_view(xs[k], 0, name);
  check_view(Y, 0, name);
  {
    // sources on unset (zero) gradients drop out; none left: nothing to add
    View keep[kMaxSrc];
    bool kg[kMaxSrc];
    double ka[kMaxSrc];
    int nk = 0;
    for (int s = 0; s < ns; ++s) {
      if (xg[s] && !nodes_[xs[s].node].grad_ready) continue;
      keep[nk] = xs[s];
      kg[nk] = xg[s];
      ka[nk] = alphas[s];
      ++nk;
    }
    if (nk < ns) {
      if (nk == 0) {
        if (!overwrite) return;
        zero_grad_if_unset(xs[0].node);  // an overwrite still needs its zeros
        run_combine(xs, xg, alphas, 1, Y, yg, overwrite, name);
        return;
      }
      run_combine(keep, kg, ka, nk, Y, yg, overwrite, name);
      return;
    }
  }
  if (yg) overwrite = !begin_grad_write(Y, !overwrite);
  if (run_combine_brick(xs, xg, alphas, ns, Y, yg, overwrite, name)) return;
  CombDesc<R> d{};
  d.nsrc = ns;
  d.overwrite = overwrite ? 1 : 0;
  d.offy = Y.off;
  // copy dims in the destination's memory order (largest stride first: the
  // writes stay coalesced whatever the sources' order), then merge
  // neighbours that are contiguous in every operand
  int nd = Y.nd;
  int shape[kMaxDim];
  long long sy[kMaxDim], sx[kMaxSrc][kMaxDim];
  // stable insertion sort of the (at most kMaxDim) dims by decreasing |stride|
  int ord[kMaxDim];
  for (int k = 0; k < nd; ++k) {
    int m = k;
    while (m > 0 && std::llabs(Y.stride[ord[m - 1]]) < std::llabs(Y.stride[k])) {
      ord[m] = ord[m - 1];
      --m;
    }
    ord[m] = k;
  }
  for (int k = 0; k < nd; ++k) {
    shape[k] = Y.shape[ord[k]];
    sy[k] = Y.stride[ord[k]];
  }
  for (int s = 0; s < ns; ++s) {
    RTCC3_CHECK(xs[s].nd == Y.nd, kErrArg, "combine rank mismatch");
    for (int k = 0; k < nd; ++k) {
      RTCC3_CHECK(xs[s].shape[ord[k]] == Y.shape[ord[k]], kErrArg, "combine shape mismatch");
      sx[s][k] = xs[s].stride[ord[k]];
    }
    d.offx[s] = xs[s].off;
    d.alpha[s] = R(alphas[s]);
    d.src[s] = xg[s] ? nodes_[xs[s].node].grad : nodes_[xs[s].node].data;
  }
  int w = 0;
  for (int k = 0; k < nd; ++k) {
    if (w > 0) {
      bool merge = sy[w - 1] == sy[k] * shape[k];
      for (int s = 0; s < ns && merge; ++s) merge = sx[s][w - 1] == sx[s][k] * shape[k];
      if (merge) {
        shape[w - 1] *= shape[k];
        sy[w - 1] = sy[k];
        for (int s = 0; s < ns; ++s) sx[s][w - 1] = sx[s][k];
        continue;
      }
    }
    shape[w] = shape[k];
    sy[w] = sy[k];
    for (int s = 0; s < ns; ++s) sx[s][w] = sx[s][k];
    ++w;
  }
  d.nd = w;
  for (int k = 0; k < w; ++k) {
    d.shape[k] = shape[k];
    d.fd[k] = FastDiv(unsigned(shape[k]));
    d.sy[k] = sy[k];
    for (int s = 0; s < ns; ++s) d.sx[s][k] = sx[s][k];
  }
  const size_t n = Y.numel();
  if (n == 0) return;
  C* py = yg ? nodes_[Y.node].grad : nodes_[Y.node].data;
  const int pk = pbegin();
  // largest element offset any operand reaches (decides 32-bit indexing)
  long long span = std::llabs(d.offy);
  {
    long long ey = std::llabs(d.offy);
    for (int k = 0; k < w; ++k) ey += std::llabs(d.sy[k]) * (d.shape[k] - 1);
    span = ey;
    for (int s = 0; s < ns; ++s) {
      long long e = std::llabs(d.offx[s]);
      for (int k = 0; k < w; ++k) e += std::llabs(d.sx[s][k]) * (d.shape[k] - 1);
      span = std::max(span, e);
    }
  }
  const bool off32 = span < (1LL << 31);
  if (n < (size_t(1) << 31) && w <= 6) {
#define RTCC3_CND(NDV)                                                                       \
  if (off32) k_combine_nd<R, NDV, true><<<grid_for(n), 256, 0, stream_>>>(py, d, unsigned(n)); \
  else k_combine_nd<R, NDV, false><<<grid_for(n), 256, 0, stream_>>>(py, d, unsigned(n))
    switch (w) {
      case 1: RTCC3_CND(1); break;
      case 2: RTCC3_CND(2); break;
      case 3: RTCC3_CND(3); break;
      case 4: RTCC3_CND(4); break;
      case 5: RTCC3_CND(5); break;
      default: RTCC3_CND(6); break;
    }
#undef RTCC3_CND
  } else if (n < (size_t(1) << 31)) {
    k_combine<R, unsigned><<<grid_for(n), 256, 0, stream_>>>(py, d, unsigned(n));
  } else {
    k_combine<R, size_t><<<grid_for(n), 256, 0, stream_>>>(py, d, n);
  }
  pend(pk, name, 2.0 * ns * n, double(n) * sizeof(C) * (ns + (overwrite ? 1 : 2)),
       prof_ && prof_->detail() ? "n=" + std::to_string(n) + " nsrc=" + std::to_string(ns) +
                                      " nd=" + std::to_string(w)
                                : std::string());
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
bool Engine<R>::run_combine_brick(const View* xs, const bool* xg, const double* alphas, int ns,
                                  const View& Y, bool yg, bool overwrite, const char* name) {
  // dense (..., v, v, v) operands that share the leading indices and permute
  // the last three
  // (overwriting sums only: accumulating into the output measured no faster
  // (three sources) or twice as slow (two) in both brick layouts at (H2O)2
  // size, against the flat layout)
  const int nd = Y.nd;
  const size_t n = Y.numel();
  if (!overwrite || nd < 3 || n < (size_t(1) << 16)) return false;
  const int v = Y.shape[nd - 1];
  if (v < 4 || Y.shape[nd - 2] != v || Y.shape[nd - 3] != v) return false;
  {
    long long st = 1;
    for (int k = nd - 1; k >= 0; --k) {
      if (Y.stride[k] != st) return false;
      st *= Y.shape[k];
    }
  }
  const long long vl = v, v2 = vl * vl;
  BrickDesc<R> d{};
  d.nsrc = ns;
  // 32-byte sectors a warp touches per 32 elements: flat layout 8 for a
  // source whose fastest index is c, 32 otherwise, output 8; 4x4x2 warps 16
  // (c fastest), 8 (a or b), output 16; 2x4x4 warps 8 (c or b), 16 (a),
  // output 8
  int flat = 8, brick0 = 16, brick1 = 8;
  for (int s = 0; s < ns; ++s) {
    const View& x = xs[s];
    if (x.nd != nd) return false;
    for (int k = 0; k < nd; ++k)
      if (x.shape[k] != Y.shape[k] || (k < nd - 3 && x.stride[k] != Y.stride[k])) return false;
    int lev[3];
    for (int q = 0; q < 3; ++q) {
      const long long st = x.stride[nd - 3 + q];
      lev[q] = st == 1 ? 0 : (st == vl ? 1 : (st == v2 ? 2 : -1));
      if (lev[q] < 0) return false;
    }
    if (lev[0] == lev[1] || lev[0] == lev[2] || lev[1] == lev[2]) return false;
    flat += lev[2] == 0 ? 8 : 32;
    brick0 += lev[2] == 0 ? 16 : 8;
    brick1 += lev[0] == 0 ? 16 : 8;
    d.src[s] = (xg[s] ? nodes_[x.node].grad : nodes_[x.node].data) + x.off;
    d.alpha[s] = R(alphas[s]);
    d.lv[s] = lev[0] | (lev[1] << 2) | (lev[2] << 4);
  }
  if (std::min(brick0, brick1) >= flat) return false;
  const int layout = brick1 <= brick0 ? 1 : 0;
  const size_t nblk = n / size_t(v2 * vl);
  if (nblk >= 65536) return false;
  d.y = (yg ? nodes_[Y.node].grad : nodes_[Y.node].data) + Y.off;
  d.overwrite = overwrite ? 1 : 0;
  d.v = v;
  const dim3 grid(unsigned((v + 3) / 4) * unsigned((v + 7) / 8), unsigned(nblk));
  const int pk = pbegin();
#define RTCC3_BRK(NSV)                                                     \
  if (layout == 1) k_combine_brick<R, NSV, 1><<<grid, 256, 0, stream_>>>(d); \
  else k_combine_brick<R, NSV, 0><<<grid, 256, 0, stream_>>>(d)
  switch (ns) {
    case 1: RTCC3_BRK(1); break;
    case 2: RTCC3_BRK(2); break;
    case 3: RTCC3_BRK(3); break;
    case 4: RTCC3_BRK(4); break;
    case 5: RTCC3_BRK(5); break;
    case 6: RTCC3_BRK(6); break;
    case 7: RTCC3_BRK(7); break;
    default: RTCC3_BRK(8); break;
  }
#undef RTCC3_BRK
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
  pend(pk, "combine_brick", 2.0 * ns * n, double(n) * sizeof(C) * (ns + (overwrite ? 1 : 2)),
       prof_ && prof_->detail() ? std::string(name) + " n=" + std::to_string(n) +
                                      " nsrc=" + std::to_string(ns)
                                : std::string());
  return true;
}

template <typename R>
void Engine<R>::combine(std::initializer_list<std::pair<double, View>> srcs, const View& Y,
                        bool overwrite) {
  View xs[kMaxSrc];
  bool xg[kMaxSrc] = {};
  double al[kMaxSrc] = {};
  int ns = 0;
  bool g = false;
  for (auto& s : srcs) {
    RTCC3_CHECK(ns < kMaxSrc, kErrArg, "combine takes at most 8 sources");
    RTCC3_CHECK(s.second.node != Y.node, kErrArg, "combine output aliases an input");
    xs[ns] = s.second;
    al[ns] = s.first;
    g = g || nodes_[s.second.node].needs_grad;
    ++ns;
  }
  run_combine(xs, xg, al, ns, Y, false, overwrite, "combine");
  if (g) nodes_[Y.node].needs_grad = true;
  for (int s = 0; s < ns; ++s) {
    Op op{kAxpy, "", al[s], xs[s], View(), Y, EpsSpec()};
    tape_.push_back(op);  // adjoint: grad(X_s) += alpha_s grad(Y)
  }
}

template <typename R>
void Engine<R>::combine_multi(const std::vector<std::vector<std::pair<double, View>>>& srcs,
                              const std::vector<View>& ys) {
  RTCC3_CHECK(srcs.size() == ys.size() && !ys.empty(), kErrArg, "combine_multi: one source list per output");
  // the fused pass: overwriting outputs of one dense (..., v, v, v) shape,
  // at most six distinct sources (views of data, not cotangents) that share
  // the leading indices and permute the last three
  bool fused = ys.size() <= size_t(kMultiOut);
  const View& Y0 = ys[0];
  const int nd = Y0.nd;
  int v = nd >= 3 ? Y0.shape[nd - 1] : 0;
  fused = fused && nd >= 3 && v >= 4 && Y0.shape[nd - 2] == v && Y0.shape[nd - 3] == v &&
          Y0.numel() >= (size_t(1) << 16);
  std::vector<View> uniq;
  BrickMultiDesc<R> d{};
  const long long vl = v, v2 = vl * vl;
  for (size_t o = 0; fused && o < ys.size(); ++o) {
    const View& Y = ys[o];
    if (Y.nd != nd) { fused = false; break; }
    long long st = 1;
    for (int k = nd - 1; k >= 0; --k) {
      if (Y.shape[k] != Y0.shape[k] || Y.stride[k] != st) { fused = false; break; }
      st *= Y.shape[k];
    }
    for (auto& sv : srcs[o]) {
      if (!fused) break;
      const View& x = sv.second;
      if (x.nd != nd || x.node == Y.node) { fused = false; break; }
      size_t u = 0;
      while (u < uniq.size() && !same_view(uniq[u], x)) ++u;
      if (u == uniq.size()) {
        if (uniq.size() == 6) { fused = false; break; }
        int lev[3];
        for (int k = 0; k < nd; ++k)
          if (x.shape[k] != Y0.shape[k] || (k < nd - 3 && x.stride[k] != Y0.stride[k])) fused = false;
        for (int q = 0; q < 3 && fused; ++q) {
          const long long sq = x.stride[nd - 3 + q];
          lev[q] = sq == 1 ? 0 : (sq == vl ? 1 : (sq == v2 ? 2 : -1));
          if (lev[q] < 0) fused = false;
        }
        if (!fused || lev[0] == lev[1] || lev[0] == lev[2] || lev[1] == lev[2]) { fused = false; break; }
        d.src[u] = nodes_[x.node].data + x.off;
        d.lv[u] = lev[0] | (lev[1] << 2) | (lev[2] << 4);
        uniq.push_back(x);
      }
      d.coef[o][u] += R(sv.first);
    }
  }
  const size_t nblk = fused ? Y0.numel() / size_t(v2 * vl) : 0;
  fused = fused && nblk < 65536;
  if (!fused) {
    for (size_t o = 0; o < ys.size(); ++o) {
      View xs[kMaxSrc];
      bool xg[kMaxSrc] = {};
      double al[kMaxSrc];
      int ns = 0;
      for (auto& sv : srcs[o]) {
        RTCC3_CHECK(ns < kMaxSrc, kErrArg, "combine takes at most 8 sources");
        xs[ns] = sv.second;
        al[ns] = sv.first;
        ++ns;
      }
      run_combine(xs, xg, al, ns, ys[o], false, true, "combine");
    }
  } else {
    for (auto& x : uniq) check_view(x, 0, "combine_multi");
    for (size_t o = 0; o < ys.size(); ++o) {
      check_view(ys[o], 0, "combine_multi");
      d.y[o] = nodes_[ys[o].node].data + ys[o].off;
    }
    d.v = v;
    // layout by 32-byte sectors per warp and 32 elements (see run_combine_brick)
    int b0 = 16 * int(ys.size()), b1 = 8 * int(ys.size());
    for (auto& x : uniq) {
      const long long sa = x.stride[nd - 3], sc = x.stride[nd - 1];
      b0 += sc == 1 ? 16 : 8;
      b1 += sa == 1 ? 16 : 8;
    }
    const int layout = b1 <= b0 ? 1 : 0;
    const dim3 grid(unsigned((v + 3) / 4) * unsigned((v + 7) / 8), unsigned(nblk));
    const int pk = pbegin();
    const int nu = int(uniq.size()), no = int(ys.size());
#define RTCC3_BM(NUV, NOV)                                                                   \
  if (layout == 1) k_combine_brick_multi<R, NUV, NOV, 1><<<grid, 256, 0, stream_>>>(d);      \
  else k_combine_brick_multi<R, NUV, NOV, 0><<<grid, 256, 0, stream_>>>(d)
#define RTCC3_BMO(NUV)                                \
  if (no == 1) { RTCC3_BM(NUV, 1); }                 \
  else if (no == 2) { RTCC3_BM(NUV, 2); }            \
  else { RTCC3_BM(NUV, 3); }
    switch (nu) {
      case 1: RTCC3_BMO(1); break;
      case 2: RTCC3_BMO(2); break;
      case 3: RTCC3_BMO(3); break;
      case 4: RTCC3_BMO(4); break;
      case 5: RTCC3_BMO(5); break;
      default: RTCC3_BMO(6); break;
    }
#undef RTCC3_BMO
#undef RTCC3_BM
    ++launches_;
    RTCC3_CUDA(cudaGetLastError());
    const size_t n = Y0.numel();
    pend(pk, "combine_brick", 2.0 * n * nu * no, double(n) * sizeof(C) * (nu + no),
         prof_ && prof_->detail() ? "multi n=" + std::to_string(n) + " nsrc=" + std::to_string(nu) +
                                        " nout=" + std::to_string(no)
                                  : std::string());
  }
  // the tape holds one combine per output, as if each had run alone
  for (size_t o = 0; o < ys.size(); ++o) {
    bool g = false;
    for (auto& sv : srcs[o]) g = g || nodes_[sv.second.node].needs_grad;
    if (g) nodes_[ys[o].node].needs_grad = true;
    for (auto& sv : srcs[o]) {
      Op op{kAxpy, "", sv.first, sv.second, View(), ys[o], EpsSpec()};
      tape_.push_back(op);
    }
  }
}

template <typename R>
void Engine<R>::exec_outer_pair(double a1, const View& x1g, const View& y1, double a2,
                                const View& x2g, const View& y2, const View& dstg) {
  auto dense = [](const View& w, std::initializer_list<int> dims) {
    if (w.nd != int(dims.size())) return false;
    long long st = 1;
    int k = w.nd - 1;
    std::vector<int> d(dims);
    for (; k >= 0; --k) {
      if (w.shape[k] != d[k] || w.stride[k] != st) return false;
      st *= d[k];
    }
    return true;
  };
  const int o = dstg.shape[0], v = dstg.shape[3];
  RTCC3_CHECK(dense(dstg, {o, o, o, v, v, v}) && dense(x1g, {o, v}) && dense(y1, {o, o, v, v}) &&
                  dense(x2g, {o, o, v, v}) && dense(y2, {o, v}) && dstg.off == 0,
              kErrArg, "outer_pair needs dense operands");
  check_view(x1g, 0, "outer_pair");
  check_view(y1, 0, "outer_pair");
  check_view(x2g, 0, "outer_pair");
  check_view(y2, 0, "outer_pair");
  check_view(dstg, 0, "outer_pair");
  if (a1 == 0.0 && a2 == 0.0) return;
  const bool acc = begin_grad_write(dstg, true);
  const unsigned v2 = unsigned(v) * unsigned(v), v3 = v2 * unsigned(v);
  RTCC3_CHECK(size_t(o) * o * o < 65536u, kErrArg, "outer_pair: too many occupied blocks");
  const dim3 grid(std::max(1u, (v3 + 1023u) / 1024u), unsigned(o) * o * o);
  const int pk = pbegin();
  k_outer_pair<R><<<grid, 256, 0, stream_>>>(
      nodes_[dstg.node].grad, a1 != 0.0 ? nodes_[x1g.node].grad + x1g.off : nullptr,
      nodes_[y1.node].data + y1.off, a2 != 0.0 ? nodes_[x2g.node].grad + x2g.off : nullptr,
      nodes_[y2.node].data + y2.off, R(a1), R(a2), o, v, acc ? 1 : 0, FastDiv(v2),
      FastDiv(unsigned(v)));
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
  const double n = double(dstg.numel());
  pend(pk, "outer_pair", 16.0 * n, n * sizeof(C) * (acc ? 2.0 : 1.0));
}

template <typename R>
void Engine<R>::sym6(double alpha, const View& X, const View& Y, bool overwrite) {
  RTCC3_CHECK(X.node != Y.node, kErrArg, "sym6 output aliases input");
  run_sym6(alpha, X, false, Y, false, overwrite);
  if (nodes_[X.node].needs_grad) nodes_[Y.node].needs_grad = true;
  Op op{kSym6, "", alpha, X, View(), Y, EpsSpec()};
  tape_.push_back(op);
}

template <typename R>
void Engine<R>::sym6_div(double alpha, const View& X, const EpsSpec& es, const View& Y) {
  RTCC3_CHECK(X.node != Y.node, kErrArg, "sym6_div output aliases input");
  run_sym6_div(alpha, X, false, es, Y, false, true, 6);
  if (nodes_[X.node].needs_grad) nodes_[Y.node].needs_grad = true;
  Op op{kSym6Div, "", alpha, X, View(), Y, es};
  tape_.push_back(op);
}

template <typename R>
void Engine<R>::run_sym6_div(double alpha, const View& X, bool xg, const EpsSpec& es, const View& Y,
                             bool yg, bool overwrite, int np, const View* Y3) {
  check_view(X, 0, "sym6_div");
  check_view(Y, 0, "sym6_div");
  if (Y3) check_view(*Y3, 0, "sym6_div");
  const bool cplx = es.osum_cr && es.vsum_cr;
  RTCC3_CHECK(cplx || (es.osum_r && es.vsum_r), kErrArg, "sym6_div needs denominator sum tables");
  auto dense6 = [&](const View& w) {
    if (w.nd != 6) return false;
    const int dims[6] = {es.o, es.o, es.o, es.v, es.v, es.v};
    long long st = 1;
    for (int k = 5; k >= 0; --k) {
      if (w.shape[k] != dims[k] || w.stride[k] != st) return false;
      st *= dims[k];
    }
    return true;
  };
  RTCC3_CHECK(dense6(X) && dense6(Y), kErrArg, "sym6_div needs dense triples views");
  RTCC3_CHECK(!Y3 || (np == 6 && dense6(*Y3) && Y3->off == 0), kErrArg,
              "sym6_div: the three-term output needs NP = 6 and a dense tensor");
  if (xg && !nodes_[X.node].grad_ready) {
    if (!overwrite && !Y3) return;  // zero cotangent
    zero_grad_if_unset(X.node);
  }
  if (yg) overwrite = !begin_grad_write(Y, !overwrite);
  const size_t n = Y.numel();
  if (n == 0) return;
  const C* px = xg ? nodes_[X.node].grad : nodes_[X.node].data;
  C* py = yg ? nodes_[Y.node].grad : nodes_[Y.node].data;
  const int pk = pbegin();
  const unsigned v2 = unsigned(es.v) * unsigned(es.v), v3 = v2 * unsigned(es.v);
  const FastDiv fv2(v2), fv(unsigned(es.v));
  // about four elements per thread along abc; one grid row per occupied block
  // NP = 6: one CTA per 4 x 8 (a, b) brick of each block; NP = 3: about four
  // elements per thread along abc
  dim3 grid(np == 6 ? unsigned((es.v + 3) / 4) * unsigned((es.v + 7) / 8)
                    : std::max(1u, (v3 + 1023u) / 1024u),
            unsigned(es.o) * es.o * es.o);
  RTCC3_CHECK(grid.y < 65536u, kErrArg, "sym6_div: too many occupied blocks");
#define RTCC3_S6D(CP, NPV)                                                                         \
  k_sym6_div<R, CP, NPV><<<grid, 256, 0, stream_>>>(px, py, X.off, Y.off, es.osum_r, es.vsum_r,     \
                                                    es.osum_cr, es.vsum_cr, es.order, es.o, es.v,  \
                                                    R(alpha), overwrite ? 1 : 0, fv2, fv,    \
                                                    Y3 ? nodes_[Y3->node].data : nullptr)
  if (cplx) {
    if (np == 6) RTCC3_S6D(true, 6);
    else RTCC3_S6D(true, 3);
  } else {
    if (np == 6) RTCC3_S6D(false, 6);
    else RTCC3_S6D(false, 3);
  }
#undef RTCC3_S6D
  pend(pk, np == 6 ? "sym6_div" : "sym3_div", (np * 2.0 + 8.0) * n,
       double(n) * sizeof(C) * (np + (overwrite ? 1 : 2)));
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void Engine<R>::run_sym6(double alpha, const View& X, bool xg, const View& Y, bool yg,
                         bool overwrite) {
  // P_ijk^abc (Eq. A30): the six simultaneous permutations of (ijk, abc)
  static const char* perms[6] = {"ijkabc->ijkabc", "jikbac->ijkabc", "ikjacb->ijkabc",
                                 "kjicba->ijkabc", "kijcab->ijkabc", "jkibca->ijkabc"};
  View xs[6];
  bool xgs[6];
  double al[6];
  for (int s = 0; s < 6; ++s) {
    xs[s] = ev(perms[s], X);
    xgs[s] = xg;
    al[s] = alpha;
  }
  run_combine(xs, xgs, al, 6, Y, yg, overwrite, "sym6");
}

template <typename R>
void Engine<R>::axpy(double alpha, const View& X, const View& Y) {
  RTCC3_CHECK(X.node != Y.node, kErrArg, "axpy output aliases input");
  run_axpy(alpha, X, false, Y, false);
  if (nodes_[X.node].needs_grad) nodes_[Y.node].needs_grad = true;
  Op op{kAxpy, "", alpha, X, View(), Y, EpsSpec()};
  tape_.push_back(op);
}

template <typename R>
void Engine<R>::run_mulc(const View& X, bool xg, const View& Cst, const View& Y, bool yg) {
  RTCC3_CHECK(X.nd == Y.nd && Cst.nd == Y.nd, kErrArg, "mulc rank mismatch");
  if (xg && !nodes_[X.node].grad_ready) return;  // zero cotangent (mulc accumulates)
  if (yg) zero_grad_if_unset(Y.node);  // k_mulc always accumulates
  StridedDesc d{};
  d.nd = Y.nd;
  for (int k = 0; k < Y.nd; ++k) {
    RTCC3_CHECK(X.shape[k] == Y.shape[k] && Cst.shape[k] == Y.shape[k], kErrArg, "mulc shape mismatch");
    d.shape[k] = Y.shape[k];
    d.s0[k] = X.stride[k];
    d.s1[k] = Y.stride[k];
    d.s2[k] = Cst.stride[k];
  }
  d.off0 = X.off; d.off1 = Y.off; d.off2 = Cst.off;
  const size_t n = Y.numel();
  if (n == 0) return;
  const C* px = xg ? nodes_[X.node].grad : nodes_[X.node].data;
  C* py = yg ? nodes_[Y.node].grad : nodes_[Y.node].data;
  const int pk = pbegin();
  k_mulc<R><<<grid_for(n), 256, 0, stream_>>>(px, nodes_[Cst.node].data, py, d, n);
  pend(pk, "mulc_strided", 8.0 * n, 4.0 * n * sizeof(C));
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void Engine<R>::mulc(const View& X, const View& Cst, const View& Y) {
  RTCC3_CHECK(X.node != Y.node, kErrArg, "mulc output aliases input");
  RTCC3_CHECK(!nodes_[Cst.node].needs_grad, kErrArg, "mulc constant must not need gradients");
  run_mulc(X, false, Cst, Y, false);
  if (nodes_[X.node].needs_grad) nodes_[Y.node].needs_grad = true;
  Op op{kMulc, "", 1.0, X, Cst, Y, EpsSpec()};
  tape_.push_back(op);
}

template <typename R>
void Engine<R>::run_div(const View& X, bool xg, const EpsSpec& es, const View& Y, bool yg,
                        bool overwrite) {
  check_view(X, 0, "div_eps");
  check_view(Y, 0, "div_eps");
  RTCC3_CHECK(X.nd == Y.nd, kErrArg, "div_eps rank mismatch");
  if (xg && !nodes_[X.node].grad_ready) {
    if (!overwrite) return;  // zero cotangent
    zero_grad_if_unset(X.node);
  }
  if (yg) overwrite = !begin_grad_write(Y, !overwrite);
  if (es.osum_c && es.vsum_c) {
    auto dense6 = [&](const View& w) {
      if (w.nd != 6) return false;
      const int dims[6] = {es.o, es.o, es.o, es.v, es.v, es.v};
      long long st = 1;
      for (int k = 5; k >= 0; --k) {
        if (w.shape[k] != dims[k] || w.stride[k] != st) return false;
        st *= dims[k];
      }
      return true;
    };
    RTCC3_CHECK(dense6(X) && dense6(Y), kErrArg, "complex denominators need dense triples views");
    const size_t n = Y.numel();
    const C* px = xg ? nodes_[X.node].grad : nodes_[X.node].data;
    C* py = yg ? nodes_[Y.node].grad : nodes_[Y.node].data;
    const long long v3 = (long long)es.v * es.v * es.v;
    const int pk = pbegin();
    if (n < (size_t(1) << 31))
      k_div_lambda_dense6<R, unsigned><<<grid_for(n), 256, 0, stream_>>>(
          px, py, X.off, Y.off, es.osum_c, es.vsum_c, unsigned(v3), unsigned(n), overwrite ? 1 : 0);
    else
      k_div_lambda_dense6<R, size_t><<<grid_for(n), 256, 0, stream_>>>(
          px, py, X.off, Y.off, es.osum_c, es.vsum_c, size_t(v3), n, overwrite ? 1 : 0);
    pend(pk, "div_eps", 8.0 * n, (overwrite ? 2.0 : 3.0) * n * sizeof(C));
    ++launches_;
    RTCC3_CUDA(cudaGetLastError());
    return;
  }
  if (es.osum && es.vsum && Y.nd == 6) {
    auto dense6 = [&](const View& w) {
      const int dims[6] = {es.o, es.o, es.o, es.v, es.v, es.v};
      long long st = 1;
      for (int k = 5; k >= 0; --k) {
        if (w.shape[k] != dims[k] || w.stride[k] != st) return false;
        st *= dims[k];
      }
      return true;
    };
    if (dense6(X) && dense6(Y)) {
      const size_t n = Y.numel();
      const C* px = xg ? nodes_[X.node].grad : nodes_[X.node].data;
      C* py = yg ? nodes_[Y.node].grad : nodes_[Y.node].data;
      const long long v3 = (long long)es.v * es.v * es.v;
      const int pk = pbegin();
      if (n < (size_t(1) << 31))
        k_div_eps_dense6<R, unsigned><<<grid_for(n), 256, 0, stream_>>>(
            px, py, X.off, Y.off, es.osum, es.vsum, unsigned(v3), unsigned(n), overwrite ? 1 : 0);
      else
        k_div_eps_dense6<R, size_t><<<grid_for(n), 256, 0, stream_>>>(
            px, py, X.off, Y.off, es.osum, es.vsum, size_t(v3), n, overwrite ? 1 : 0);
      pend(pk, "div_eps", 4.0 * n, (overwrite ? 2.0 : 3.0) * n * sizeof(C));
      ++launches_;
      RTCC3_CUDA(cudaGetLastError());
      return;
    }
  }
  StridedDesc d{};
  EpsArgs ea{};
  d.nd = Y.nd;
  for (int k = 0; k < Y.nd; ++k) {
    RTCC3_CHECK(X.shape[k] == Y.shape[k], kErrArg, "div_eps shape mismatch");
    d.shape[k] = Y.shape[k];
    d.s0[k] = X.stride[k];
    d.s1[k] = Y.stride[k];
    ea.sign[k] = es.sign[k];
    ea.base[k] = es.base[k];
  }
  d.off0 = X.off;
  d.off1 = Y.off;
  const size_t n = Y.numel();
  if (n == 0) return;
  const C* px = xg ? nodes_[X.node].grad : nodes_[X.node].data;
  C* py = yg ? nodes_[Y.node].grad : nodes_[Y.node].data;
  const int pk = pbegin();
  if (n < (size_t(1) << 31))
    k_div_eps<R, unsigned><<<grid_for(n), 256, 0, stream_>>>(px, py, d, es.eps, ea, unsigned(n),
                                                              overwrite ? 1 : 0);
  else
    k_div_eps<R, size_t><<<grid_for(n), 256, 0, stream_>>>(px, py, d, es.eps, ea, n, overwrite ? 1 : 0);
  pend(pk, "div_eps", 4.0 * n, (overwrite ? 2.0 : 3.0) * n * sizeof(C));
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void Engine<R>::div_eps(const View& X, const EpsSpec& es, const View& Y, bool overwrite) {
  RTCC3_CHECK(X.node != Y.node, kErrArg, "div_eps output aliases input");
  run_div(X, false, es, Y, false, overwrite);
  if (nodes_[X.node].needs_grad) nodes_[Y.node].needs_grad = true;
  Op op{kDiv, "", 1.0, X, View(), Y, es};
  tape_.push_back(op);
}

template <typename R>
void Engine<R>::fill_identity(int n) {
  const Node& nd = nodes_[n];
  RTCC3_CHECK(nd.shape.size() == 2 && nd.shape[0] == nd.shape[1], kErrArg, "identity needs a square node");
  const int m = nd.shape[0];
  k_identity<R><<<(m * m + 255) / 256, 256, 0, stream_>>>(nd.data, m);
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void Engine<R>::fill_ones(int n) {
  launch_fill<R>(nodes_[n].data, nodes_[n].numel, 1.0, 0.0, stream_);
  ++launches_;
}

template <typename R>
void Engine<R>::prepare_backward() {
  for (auto& nd : nodes_) {
    if (!nd.needs_grad) continue;
    nd.grad = static_cast<C*>(arena_.alloc(nd.numel * sizeof(C)));
    nd.grad_ready = nd.numel < kLazyGradMin;
    if (nd.grad_ready) RTCC3_CUDA(cudaMemsetAsync(nd.grad, 0, nd.numel * sizeof(C), stream_));
  }
}

template <typename R>
bool Engine<R>::begin_grad_write(const View& dst, bool accumulate) {
  Node& nd = nodes_[dst.node];
  if (nd.grad_ready) return accumulate;
  nd.grad_ready = true;
  // does the view cover the whole node, each element once?
  bool covers = dst.off == 0 && dst.numel() == nd.numel;
  if (covers) {
    long long st[kMaxDim];
    int ext[kMaxDim], m = 0;
    for (int d = 0; d < dst.nd; ++d)
      if (dst.shape[d] > 1) { st[m] = std::llabs(dst.stride[d]); ext[m] = dst.shape[d]; ++m; }
    int idx[kMaxDim];
    for (int d = 0; d < m; ++d) idx[d] = d;
    std::sort(idx, idx + m, [&](int p, int q) { return st[p] > st[q]; });
    long long expect = 1;
    for (int d = m - 1; d >= 0 && covers; --d) {
      covers = st[idx[d]] == expect;
      expect *= ext[idx[d]];
    }
  }
  if (covers) return false;
  RTCC3_CUDA(cudaMemsetAsync(nd.grad, 0, nd.numel * sizeof(C), stream_));
  return accumulate;
}

template <typename R>
void Engine<R>::zero_grad_if_unset(int node) {
  Node& nd = nodes_[node];
  if (nd.grad_ready) return;
  RTCC3_CUDA(cudaMemsetAsync(nd.grad, 0, nd.numel * sizeof(C), stream_));
  nd.grad_ready = true;
}

template <typename R>
void Engine<R>::exec_slab_div(double alpha, const View& X, int i0, const EpsSpec& es,
                              const View& Y) {
  check_view(X, 0, "slab_div");
  check_view(Y, 0, "slab_div");
  const bool cplx = es.osum_cr && es.vsum_cr;
  RTCC3_CHECK(cplx || (es.osum_r && es.vsum_r), kErrArg, "slab division needs sum tables");
  RTCC3_CHECK(X.nd == 6 && Y.nd == 6 && X.off == 0 && Y.off == 0, kErrArg,
              "slab division takes whole dense slab nodes");
  const size_t v3 = size_t(es.v) * es.v * es.v;
  const size_t n = Y.numel();
  RTCC3_CHECK(X.numel() == n && n % (v3 * es.o * es.o) == 0, kErrArg, "slab division extents");
  RTCC3_CHECK(i0 >= 0 && i0 + int(n / (v3 * es.o * es.o)) <= es.o, kErrArg, "slab start");
  const int pk = pbegin();
  const size_t o2base = size_t(i0) * es.o * es.o;
  if (cplx)
    k_slab_div<R, true><<<grid_for(n), 256, 0, stream_>>>(nodes_[X.node].data, nodes_[Y.node].data,
                                                          nullptr, nullptr, es.osum_cr, es.vsum_cr,
                                                          o2base, v3, n, R(alpha));
  else
    k_slab_div<R, false><<<grid_for(n), 256, 0, stream_>>>(nodes_[X.node].data,
                                                           nodes_[Y.node].data, es.osum_r,
                                                           es.vsum_r, nullptr, nullptr, o2base, v3,
                                                           n, R(alpha));
  ++launches_;
  RTCC3_CUDA(cudaGetLastError());
  pend(pk, "slab_div", 8.0 * double(n), 2.0 * double(n) * sizeof(C));
}

// The adjoints dA = dC . B and dB = A . dC of one product read the same
// inputs and write different cotangents: they are launched as two branches
// (dB on the branch stream with its own split-K and tensor-core scratch, dA
// on the engine's stream) that join before the next operation.
// Not while profiling (per-operation timings stay serial), with a caller's
// pool (one stream) or when A and B are one node (both adjoints add into it).
template <typename R>
void Engine<R>::region_enter() {
  if (!region_) {
    RTCC3_CUDA(cudaStreamCreateWithFlags(&region_, cudaStreamNonBlocking));
    RTCC3_CUDA(cudaEventCreateWithFlags(&region_fork_, cudaEventDisableTiming));
    RTCC3_CUDA(cudaEventCreateWithFlags(&region_join_, cudaEventDisableTiming));
  }
  RTCC3_CUDA(cudaEventRecord(region_fork_, stream_));
  RTCC3_CUDA(cudaStreamWaitEvent(region_, region_fork_, 0));
  region_main_ = stream_;
  stream_ = region_;
  split_slot_ = 5;
  in_region_ = true;
}

template <typename R>
void Engine<R>::region_leave() {
  stream_ = region_main_;
  split_slot_ = 0;
  in_region_ = false;
}

template <typename R>
void Engine<R>::region_begin() {
  if (!regions() || in_region_ || region_pending_) return;
  region_enter();
  region_pending_ = true;
  tape_.push_back(Op{kRegionBegin, "", 0.0, View(), View(), View(), EpsSpec()});
}

template <typename R>
void Engine<R>::region_end() {
  if (!in_region_) return;
  region_leave();
  tape_.push_back(Op{kRegionEnd, "", 0.0, View(), View(), View(), EpsSpec()});
}

template <typename R>
void Engine<R>::region_join() {
  if (!region_pending_ || in_region_) return;
  RTCC3_CUDA(cudaEventRecord(region_join_, region_));
  RTCC3_CUDA(cudaStreamWaitEvent(stream_, region_join_, 0));
  region_pending_ = false;
  tape_.push_back(Op{kRegionJoin, "", 0.0, View(), View(), View(), EpsSpec()});
}

template <typename R>
void Engine<R>::ensure_branch_stream() {
  if (branch_) return;
  RTCC3_CUDA(cudaStreamCreateWithFlags(&branch_, cudaStreamNonBlocking));
  RTCC3_CUDA(cudaEventCreateWithFlags(&branch_fork_, cudaEventDisableTiming));
  RTCC3_CUDA(cudaEventCreateWithFlags(&branch_join_, cudaEventDisableTiming));
}

template <typename R>
void Engine<R>::branch_begin() {
  if (!regions() || in_region_ || branch_state_ != 0) return;
  ensure_branch_stream();
  RTCC3_CUDA(cudaEventRecord(branch_fork_, stream_));
  RTCC3_CUDA(cudaStreamWaitEvent(branch_, branch_fork_, 0));
  branch_main_ = stream_;
  stream_ = branch_;
  split_slot_ = 4;
  tc_slot_ = 6;
  branch_state_ = 1;
}

template <typename R>
void Engine<R>::branch_switch() {
  if (branch_state_ != 1) return;
  stream_ = branch_main_;
  split_slot_ = 0;
  tc_slot_ = 1;
  branch_state_ = 2;
}

template <typename R>
void Engine<R>::branch_join() {
  if (branch_state_ == 0) return;
  if (branch_state_ == 1) branch_switch();
  RTCC3_CUDA(cudaEventRecord(branch_join_, branch_));
  RTCC3_CUDA(cudaStreamWaitEvent(stream_, branch_join_, 0));
  branch_state_ = 0;
}

template <typename R>
bool Engine<R>::run_adjoints_branched(const Op& op) {
  if (!branches_ || pool_ || (prof_ && prof_->enabled) || in_region_ || branch_state_ != 0)
    return false;
  if (op.a.node == op.b.node || !nodes_[op.a.node].needs_grad || !nodes_[op.b.node].needs_grad)
    return false;
  const Spec s = parse(op.spec);
  const std::string sa = s.c + "," + s.b + "->" + s.a, sb = s.a + "," + s.c + "->" + s.b;
  ensure_branch_stream();
  RTCC3_CUDA(cudaEventRecord(branch_fork_, stream_));
  RTCC3_CUDA(cudaStreamWaitEvent(branch_, branch_fork_, 0));
  cudaStream_t main = stream_;
  stream_ = branch_;
  split_slot_ = 4;
  tc_slot_ = 6;
  try {
    run_contract(sb, op.alpha, op.a, false, op.c, true, op.b, true, true);
  } catch (...) {
    stream_ = main;
    split_slot_ = 0;
    tc_slot_ = 1;
    throw;
  }
  stream_ = main;
  split_slot_ = 0;
  tc_slot_ = 1;
  run_contract(sa, op.alpha, op.c, true, op.b, false, op.a, true, true);
  RTCC3_CUDA(cudaEventRecord(branch_join_, branch_));
  RTCC3_CUDA(cudaStreamWaitEvent(stream_, branch_join_, 0));
  return true;
}

template <typename R>
void Engine<R>::defer_gather(const View* xs, const double* al, int ns, const View& dst) {
  for (size_t k = 0; k < gathers_.size(); ++k) {
    PendingGather& p = gathers_[k];
    if (!same_view(p.dst, dst)) continue;
    if (p.ns + ns <= kMaxSrc) {
      for (int s = 0; s < ns; ++s) {
        p.xs[p.ns] = xs[s];
        p.al[p.ns] = al[s];
        ++p.ns;
      }
      return;
    }
    flush_gathers(dst.node);
    break;
  }
  PendingGather p;
  p.dst = dst;
  p.ns = ns;
  for (int s = 0; s < ns; ++s) {
    p.xs[s] = xs[s];
    p.al[s] = al[s];
  }
  gathers_.push_back(p);
}

template <typename R>
void Engine<R>::flush_gathers(int node) {
  std::vector<PendingGather> keep;
  std::vector<PendingGather> run;
  for (auto& p : gathers_) (node < 0 || p.dst.node == node ? run : keep).push_back(p);
  gathers_.swap(keep);
  for (auto& p : run) {
    bool xg[kMaxSrc];
    for (int s = 0; s < kMaxSrc; ++s) xg[s] = true;
    run_combine(p.xs, xg, p.al, p.ns, p.dst, true, false, "axpy_gather");
  }
}

template <typename R>
void Engine<R>::backward() {
  gathers_.clear();
  for (auto it = tape_.rbegin(); it != tape_.rend(); ++it) {
    const Op& op = *it;
    // a held-back gather completes a cotangent before anything reads it: the
    // adjoint of the operation that produced its node, any custom adjoint,
    // and a change of stream
    if (op.kind == kContract || op.kind == kAxpy || op.kind == kMulc || op.kind == kDiv ||
        op.kind == kSym6 || op.kind == kSym6Div) {
      if (!gathers_.empty()) flush_gathers(op.c.node);
    } else if (!gathers_.empty()) {
      flush_gathers(-1);
    }
    if (op.kind == kContract) {
      if (!nodes_[op.c.node].needs_grad) continue;
      const Spec s = parse(op.spec);
      cur_tc_ = op.tc;
      if (run_adjoints_branched(op)) continue;
      if (nodes_[op.a.node].needs_grad)
        run_contract(s.c + "," + s.b + "->" + s.a, op.alpha, op.c, true, op.b, false, op.a, true, true);
      if (nodes_[op.b.node].needs_grad)
        run_contract(s.a + "," + s.c + "->" + s.b, op.alpha, op.a, false, op.c, true, op.b, true, true);
    } else if (op.kind == kAxpy) {
      // the run of axpy ops recorded by one combine share their gradient
      // source; their adjoints into one node become one gather pass over
      // that node in its own memory order
      auto jt = it;
      std::vector<const Op*> run;
      while (jt != tape_.rend() && jt->kind == kAxpy && same_view(jt->c, op.c)) {
        run.push_back(&*jt);
        ++jt;
      }
      it = std::prev(jt);
      if (!nodes_[op.c.node].needs_grad) continue;
      std::vector<bool> done(run.size(), false);
      for (size_t i = 0; i < run.size(); ++i) {
        if (done[i] || !nodes_[run[i]->a.node].needs_grad) continue;
        View dense, src;
        if (!invert_view(run[i]->a, run[i]->c, dense, src)) {
          run_axpy(run[i]->alpha, run[i]->c, true, run[i]->a, true);
          continue;
        }
        View xs[kMaxSrc];
        double al[kMaxSrc];
        int ns = 0;
        for (size_t j = i; j < run.size() && ns < kMaxSrc; ++j) {
          if (done[j] || run[j]->a.node != run[i]->a.node) continue;
          View dj, sj;
          if (!invert_view(run[j]->a, run[j]->c, dj, sj) || !same_view(dj, dense)) continue;
          xs[ns] = sj;
          al[ns] = run[j]->alpha;
          ++ns;
          done[j] = true;
        }
        defer_gather(xs, al, ns, dense);
      }
    } else if (op.kind == kMulc) {
      if (!nodes_[op.c.node].needs_grad || !nodes_[op.a.node].needs_grad) continue;
      run_mulc(op.c, true, op.b, op.a, true);
    } else if (op.kind == kDiv) {
      if (!nodes_[op.c.node].needs_grad || !nodes_[op.a.node].needs_grad) continue;
      run_div(op.c, true, op.es, op.a, true);
    } else if (op.kind == kSym6) {
      if (!nodes_[op.c.node].needs_grad || !nodes_[op.a.node].needs_grad) continue;
      run_sym6(op.alpha, op.c, true, op.a, true, false);
    } else if (op.kind == kSym6Div) {
      if (!nodes_[op.c.node].needs_grad || !nodes_[op.a.node].needs_grad) continue;
      run_sym6_div(op.alpha, op.c, true, op.es, op.a, true, false, 6);
    } else if (op.kind == kRegionJoin) {
      // the region's adjoints may start once everything after it is done
      RTCC3_CUDA(cudaEventRecord(region_fork_, stream_));
      RTCC3_CUDA(cudaStreamWaitEvent(region_, region_fork_, 0));
    } else if (op.kind == kRegionEnd) {
      region_main_ = stream_;
      stream_ = region_;
      split_slot_ = 5;
      in_region_ = true;
    } else if (op.kind == kRegionBegin) {
      region_leave();
      RTCC3_CUDA(cudaEventRecord(region_join_, region_));
      RTCC3_CUDA(cudaStreamWaitEvent(stream_, region_join_, 0));
    } else {
      const bool saved = tc_region_;
      tc_region_ = op.tc;
      op.fn();
      tc_region_ = saved;
    }
  }
  flush_gathers(-1);
}

template class Engine<double>;
template class Engine<float>;
template void launch_fill<double>(Cx<double>*, size_t, double, double, cudaStream_t);
template void launch_fill<float>(Cx<float>*, size_t, double, double, cudaStream_t);

}  // namespace rtcc3
