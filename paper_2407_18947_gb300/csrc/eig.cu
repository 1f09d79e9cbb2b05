// Eigendecomposition of the small complex non-Hermitian matrices that carry
// the field coupling of the triples equation (see rotation.h).
//
// One warp per matrix, no block-wide barriers: M is reduced to upper
// Hessenberg form by Householder reflections, then to Schur form
// T = Q^H M Q by single-shift QR sweeps (Wilkinson shift, Givens rotations,
// deflation of negligible subdiagonal entries, an exceptional shift every
// eleventh sweep); the eigenvectors X of the upper-triangular T follow by back
// substitution (unit diagonal), so S = Q X, S^-1 = X^-1 Q^H and
// M = S diag(T_kk) S^-1.  Every lane computes the rotation parameters itself
// from the same shared-memory values (identical control flow), then the lanes
// update disjoint rows and columns.  The arithmetic type T is float for the
// complex64 graphs and double for the complex128 one.  H lives in shared
// memory, Q, X and X^-1 in a global workspace; a non-converging sweep count or
// a non-finite matrix raises *status (codes in rotation.h) instead of looping.
#include "rotation.h"

#include <algorithm>

namespace rtcc3 {

namespace {

template <typename T> struct C2T;
template <> struct C2T<float> { using type = float2; };
template <> struct C2T<double> { using type = double2; };

template <typename T>
struct Cplx {
  using V = typename C2T<T>::type;
  static __device__ __forceinline__ V mk(T a, T b) { V r; r.x = a; r.y = b; return r; }
  static __device__ __forceinline__ V mul(V a, V b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
  static __device__ __forceinline__ V conj(V a) { return mk(a.x, -a.y); }
  static __device__ __forceinline__ V add(V a, V b) { return mk(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ V sub(V a, V b) { return mk(a.x - b.x, a.y - b.y); }
  static __device__ __forceinline__ V scale(V a, T s) { return mk(a.x * s, a.y * s); }
  static __device__ __forceinline__ T abs(V a) { return sqrt(a.x * a.x + a.y * a.y); }
  // Smith's algorithm
  static __device__ __forceinline__ V div(V a, V b) {
    if (fabs(b.x) >= fabs(b.y)) {
      const T r = b.y / b.x, d = b.x + b.y * r;
      return mk((a.x + a.y * r) / d, (a.y - a.x * r) / d);
    }
    const T r = b.x / b.y, d = b.y + b.x * r;
    return mk((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
  // principal square root without cancellation: t = sqrt((|x| + |z|) / 2) is
  // the larger of |Re|, |Im| and the other part follows as y / (2 t)
  static __device__ __forceinline__ V sqrt_(V z) {
    const T m = abs(z);
    if (m == T(0)) return mk(T(0), T(0));
    const T t = sqrt(T(0.5) * (fabs(z.x) + m));
    if (z.x >= T(0)) return mk(t, z.y / (T(2) * t));
    return mk(fabs(z.y) / (T(2) * t), copysign(t, z.y));
  }
};

// Sum over the warp, returned identically in every lane (lane 0's value:
// the lanes' butterfly sums may round differently, and every lane takes the
// same branches on the result).
// 1/sqrt(x) from the correctly rounded square root and division: the rotation
// stays unitary to rounding, with no systematic drift of |c|^2 + |s|^2 over the
// thousands of rotations accumulated into Q
template <typename T>
__device__ __forceinline__ T rsqrt_(T x) { return T(1) / sqrt(x); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return __shfl_sync(0xffffffffu, v, 0);
}

// level: 2 = H, Q, X and X^-1 in shared memory, 1 = H and Q, 0 = H only (the
// rest in the workspace).
template <typename T>
__global__ void __launch_bounds__(32) k_eig_warp(EigJob ja, EigJob jb, int level,
                                                 int* __restrict__ status) {
  using X = Cplx<T>;
  using V = typename C2T<T>::type;
  const EigJob J = blockIdx.x == 0 ? ja : jb;
  const int n = J.n;
  if (n <= 0) return;
  const int lane = threadIdx.x;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int nn = n * n;
  V* H = reinterpret_cast<V*>(sm_raw);  // n x n, row-major
  V* vb = H + nn;                       // Householder vector
  V* wsv = reinterpret_cast<V*>(J.ws);
  V* Q = level >= 1 ? vb + n : wsv;
  V* Xv = level >= 2 ? Q + nn : wsv + nn;
  V* Xi = Xv + nn;
  T fro = T(0);
  for (int t = lane; t < nn; t += 32) {
    const double2 m = J.M[t];
    H[t] = X::mk(T(m.x), T(m.y));
    Q[t] = X::mk((t / n) == (t % n) ? T(1) : T(0), T(0));
    fro += T(m.x) * T(m.x) + T(m.y) * T(m.y);
  }
  fro = sqrt(warp_sum(fro));
  __syncwarp();
  if (!isfinite(fro)) {
    if (lane == 0) atomicExch(status, eig_status(kEigNonFinite, n, n - 1));
    return;
  }
  const T tiny = sizeof(T) == 4 ? T(1e-30) : T(1e-300);
  const T eps = sizeof(T) == 4 ? T(1.2e-7) : T(2.2e-16);

  // ---- Householder reduction to upper Hessenberg form -------------------------
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    T s2 = T(0);
    for (int i = lane; i < m; i += 32) {
      const V x = H[(k + 1 + i) * n + k];
      s2 += x.x * x.x + x.y * x.y;
    }
    s2 = warp_sum(s2);
    const T xnorm = sqrt(s2);
    const V x0 = H[(k + 1) * n + k];
    const T ax0 = X::abs(x0);
    if (xnorm <= tiny || s2 - ax0 * ax0 <= T(1e-30) * s2) continue;  // column already reduced
    const V ph = ax0 > T(0) ? X::scale(x0, T(1) / ax0) : X::mk(T(1), T(0));
    const V alpha = X::scale(ph, -xnorm);
    for (int i = lane; i < m; i += 32) vb[i] = i == 0 ? X::sub(x0, alpha) : H[(k + 1 + i) * n + k];
    __syncwarp();
    T vv = T(0);
    for (int i = lane; i < m; i += 32) vv += vb[i].x * vb[i].x + vb[i].y * vb[i].y;
    const T beta = T(2) / warp_sum(vv);
    // left: rows k+1.., columns k..n-1 (one column per lane)
    for (int j = k + lane; j < n; j += 32) {
      V sd = X::mk(T(0), T(0));
      for (int i = 0; i < m; ++i) sd = X::add(sd, X::mul(X::conj(vb[i]), H[(k + 1 + i) * n + j]));
      sd = X::scale(sd, beta);
      for (int i = 0; i < m; ++i) H[(k + 1 + i) * n + j] = X::sub(H[(k + 1 + i) * n + j], X::mul(vb[i], sd));
    }
    __syncwarp();
    // right: all rows of H and Q, columns k+1..n-1 (one row per lane)
    for (int r = lane; r < 2 * n; r += 32) {
      V* row = r < n ? &H[r * n] : &Q[size_t(r - n) * n];
      V sd = X::mk(T(0), T(0));
      for (int j = 0; j < m; ++j) sd = X::add(sd, X::mul(row[k + 1 + j], vb[j]));
      sd = X::scale(sd, beta);
      for (int j = 0; j < m; ++j) row[k + 1 + j] = X::sub(row[k + 1 + j], X::mul(sd, X::conj(vb[j])));
    }
    __syncwarp();
    for (int i = 1 + lane; i < m; i += 32) H[(k + 1 + i) * n + k] = X::mk(T(0), T(0));
    __syncwarp();
  }

  // ---- shifted QR sweeps to Schur form ---------------------------------------
  int hi = n - 1, iter = 0, its_here = 0;
  const int max_iter = J.max_sweeps > 0 ? J.max_sweeps : 60 * n + 100;
  bool failed = false;
  while (hi > 0) {
    int l = hi;
    while (l > 0) {
      const T off = X::abs(H[l * n + l - 1]);
      const T dg = X::abs(H[l * n + l]) + X::abs(H[(l - 1) * n + l - 1]);
      if (off <= eps * (dg > T(0) ? dg : fro)) break;
      --l;
    }
    __syncwarp();
    if (l > 0 && lane == 0) H[l * n + l - 1] = X::mk(T(0), T(0));
    __syncwarp();
    if (l == hi) {
      --hi;
      its_here = 0;
      continue;
    }
    if (++iter > max_iter) {
      failed = true;
      break;
    }
    ++its_here;
    for (int k = l; k < hi; ++k) {
      V x, y;
      if (k == l) {
        // Wilkinson shift: eigenvalue of the trailing 2x2 closest to H[hi][hi]
        const V a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
        const V c = H[hi * n + hi - 1], d = H[hi * n + hi];
        const V tr2 = X::scale(X::add(a, d), T(0.5));
        const V hd = X::scale(X::sub(a, d), T(0.5));
        const V disc = X::sqrt_(X::add(X::mul(hd, hd), X::mul(b, c)));
        const V l1 = X::add(tr2, disc), l2 = X::sub(tr2, disc);
        V mu = X::abs(X::sub(l1, d)) < X::abs(X::sub(l2, d)) ? l1 : l2;
        if (its_here % 11 == 10 || !isfinite(mu.x) || !isfinite(mu.y))  // exceptional shift
          mu = X::add(d, X::mk(T(0.75) * X::abs(c), T(0)));
        x = X::sub(H[l * n + l], mu);
        y = H[(l + 1) * n + l];
      } else {
        x = H[k * n + k - 1];
        y = H[(k + 1) * n + k - 1];
      }
      // G = [[c, s], [-conj(s), conj(c)]] with c = conj(x) / r, s = conj(y) / r,
      // r = |(x, y)|: unitary, maps (x, y) to (r, 0); one reciprocal square root
      T r2 = x.x * x.x + x.y * x.y + y.x * y.x + y.y * y.y;
      V c, s;
      if (!(r2 > tiny && r2 < T(1) / tiny)) {  // rescale out of the under/overflow range
        const T m = fmax(fmax(fabs(x.x), fabs(x.y)), fmax(fabs(y.x), fabs(y.y)));
        if (m > T(0) && isfinite(m)) {
          x = X::scale(x, T(1) / m);
          y = X::scale(y, T(1) / m);
        } else {
          x = X::mk(T(1), T(0));
          y = X::mk(T(0), T(0));
        }
        r2 = x.x * x.x + x.y * x.y + y.x * y.x + y.y * y.y;
      }
      const T ri = rsqrt_(r2);
      c = X::mk(x.x * ri, -x.y * ri);
      s = X::mk(y.x * ri, -y.y * ri);
      __syncwarp();  // every lane has read the entries the rotation is built from
      // rows k, k+1 <- G rows; the bulge H[k+1][k-1] becomes exactly zero
      for (int j = (k == l ? k : k - 1) + lane; j < n; j += 32) {
        const V a = H[k * n + j], b = H[(k + 1) * n + j];
        H[k * n + j] = X::add(X::mul(c, a), X::mul(s, b));
        H[(k + 1) * n + j] = (k > l && j == k - 1)
                                 ? X::mk(T(0), T(0))
                                 : X::sub(X::mul(X::conj(c), b), X::mul(X::conj(s), a));
      }
      __syncwarp();
      // columns k, k+1 <- columns times G^H (H rows 0..min(k+2,hi), all rows of Q)
      const int rmax = min(k + 2, hi);
      for (int rr = lane; rr <= rmax + n; rr += 32) {
        V* row = rr <= rmax ? &H[rr * n] : &Q[size_t(rr - rmax - 1) * n];
        const V a = row[k], b = row[k + 1];
        row[k] = X::add(X::mul(a, X::conj(c)), X::mul(b, X::conj(s)));
        row[k + 1] = X::sub(X::mul(b, c), X::mul(a, s));
      }
      __syncwarp();
    }
  }
  if (failed) {
    if (lane == 0) atomicExch(status, eig_status(kEigNoConvergence, n, hi));
    return;
  }

  // ---- eigenvectors of T (unit upper triangular X), S = Q X, S^-1 = X^-1 Q^H --
  const T smin = fmax(eps * fro, tiny);
  for (int k = lane; k < n; k += 32) {
    const V tk = H[k * n + k];
    J.lam[k] = make_double2(double(tk.x), double(tk.y));
    for (int i = 0; i < n; ++i) Xv[size_t(i) * n + k] = X::mk(i == k ? T(1) : T(0), T(0));
    for (int i = k - 1; i >= 0; --i) {
      V acc = X::mk(T(0), T(0));
      for (int j = i + 1; j <= k; ++j) acc = X::add(acc, X::mul(H[i * n + j], Xv[size_t(j) * n + k]));
      V den = X::sub(H[i * n + i], tk);
      if (X::abs(den) < smin) den = X::mk(smin, T(0));
      Xv[size_t(i) * n + k] = X::scale(X::div(acc, den), T(-1));
    }
  }
  __syncwarp();
  for (int k = lane; k < n; k += 32) {
    // column k of X^-1: unit upper triangular back substitution
    for (int i = 0; i < n; ++i) Xi[size_t(i) * n + k] = X::mk(i == k ? T(1) : T(0), T(0));
    for (int i = k - 1; i >= 0; --i) {
      V acc = X::mk(T(0), T(0));
      for (int j = i + 1; j <= k; ++j) acc = X::add(acc, X::mul(Xv[size_t(i) * n + j], Xi[size_t(j) * n + k]));
      Xi[size_t(i) * n + k] = X::scale(acc, T(-1));
    }
  }
  __syncwarp();
  for (int t = lane; t < nn; t += 32) {
    const int i = t / n, k = t % n;
    V a = X::mk(T(0), T(0)), b = X::mk(T(0), T(0));
    for (int j = 0; j <= k; ++j) a = X::add(a, X::mul(Q[size_t(i) * n + j], Xv[size_t(j) * n + k]));
    for (int j = i; j < n; ++j) b = X::add(b, X::mul(Xi[size_t(i) * n + j], X::conj(Q[size_t(k) * n + j])));
    J.S[t] = make_double2(double(a.x), double(a.y));
    J.Sinv[t] = make_double2(double(b.x), double(b.y));
  }
}

template <typename T>
void launch_t(const EigJob& a, const EigJob& b, int* status, cudaStream_t s) {
  constexpr size_t kMaxSmem = 200 * 1024;
  const size_t nmax = size_t(std::max(a.n, b.n));
  const size_t vs = sizeof(typename C2T<T>::type);
  int level = 0;
  size_t smem = (nmax * nmax + nmax) * vs;
  if ((4 * nmax * nmax + nmax) * vs <= kMaxSmem) {
    level = 2;
    smem = (4 * nmax * nmax + nmax) * vs;
  } else if ((2 * nmax * nmax + nmax) * vs <= kMaxSmem) {
    level = 1;
    smem = (2 * nmax * nmax + nmax) * vs;
  }
  static bool attr = false;
  if (!attr) {
    RTCC3_CUDA(cudaFuncSetAttribute(k_eig_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(kMaxSmem)));
    attr = true;
  }
  k_eig_warp<T><<<2, 32, smem, s>>>(a, b, level, status);
  RTCC3_CUDA(cudaGetLastError());
}

}  // namespace

void launch_eig(const EigJob& a, const EigJob& b, bool fp32, int* status, cudaStream_t s) {
  RTCC3_CHECK(a.n >= 1 && a.n <= kEigMaxN && b.n >= 1 && b.n <= kEigMaxN, kErrArg,
              "eigensolver supports n <= " + std::to_string(kEigMaxN));
  if (fp32) launch_t<float>(a, b, status, s);
  else launch_t<double>(a, b, status, s);
}

}  // namespace rtcc3
