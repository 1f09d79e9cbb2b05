// Eigendecomposition of the small complex non-Hermitian matrices that carry
// the field coupling of the triples equation (see rotation.h).
//
// One CTA per matrix, FP64 complex.  M is reduced to upper Hessenberg form by
// Householder reflections, then to Schur form T = Q^H M Q by single-shift QR
// sweeps (Wilkinson shift, Givens rotations, deflation of negligible
// subdiagonal entries); the eigenvectors X of the upper-triangular T are found
// by back substitution (unit diagonal), so S = Q X, S^-1 = X^-1 Q^H and
// M = S diag(T_kk) S^-1.  H lives in shared memory; Q, X and X^-1 in a global
// workspace.  A non-converging sweep count raises *status instead of looping.
#include "rotation.h"

namespace rtcc3 {

namespace {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.y + b.x * r;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
// Principal square root without cancellation: t = sqrt((|x| + |z|) / 2) is
// the larger of |Re|, |Im| and the other part follows as y / (2 t).
__device__ __forceinline__ double2 csqrt(double2 z) {
  const double m = cabs2(z);
  if (m == 0.0) return make_double2(0.0, 0.0);
  const double t = sqrt(0.5 * (fabs(z.x) + m));
  if (z.x >= 0.0) return make_double2(t, z.y / (2.0 * t));
  return make_double2(fabs(z.y) / (2.0 * t), copysign(t, z.y));
}

// Block-wide sum of one double (blockDim.x <= 1024).
__device__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int i = 0; i < nw; ++i) s += red[i];
  return s;
}

__global__ void k_eig(const double2* __restrict__ Min, int n, double2* __restrict__ S,
                      double2* __restrict__ Sinv, double2* __restrict__ lam,
                      double2* __restrict__ ws, int* __restrict__ status) {
  extern __shared__ double2 H[];  // n x n, row-major
  __shared__ double red[32];
  __shared__ double2 v[kEigMaxN];
  __shared__ double2 gcs[2];  // (c, 0), s
  __shared__ int ctl[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t nn = size_t(n) * n;
  const double2* M = Min + size_t(blockIdx.x) * nn;
  double2* Q = ws + size_t(blockIdx.x) * 3 * nn;
  double2* X = Q + nn;
  double2* Xi = X + nn;
  S += size_t(blockIdx.x) * nn;
  Sinv += size_t(blockIdx.x) * nn;
  lam += size_t(blockIdx.x) * n;
  for (size_t t = tid; t < nn; t += nt) {
    H[t] = M[t];
    Q[t] = make_double2((t / n) == (t % n) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  double fro = 0.0;
  for (size_t t = tid; t < nn; t += nt) fro += H[t].x * H[t].x + H[t].y * H[t].y;
  fro = sqrt(block_sum(fro, red));
  const double tiny = 1e-300;
  if (!isfinite(fro)) {
    if (tid == 0) atomicExch(status, eig_status(kEigNonFinite, n, n - 1));
    return;
  }

  // ---- Householder reduction to upper Hessenberg form -------------------------
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double s2 = 0.0;
    for (int i = tid; i < m; i += nt) {
      const double2 x = H[(k + 1 + i) * n + k];
      s2 += x.x * x.x + x.y * x.y;
    }
    const double xnorm = sqrt(block_sum(s2, red));
    const double2 x0 = H[(k + 1) * n + k];
    const double ax0 = cabs2(x0);
    double tail = xnorm * xnorm - ax0 * ax0;
    if (xnorm <= tiny || tail <= 1e-30 * xnorm * xnorm) {
      __syncthreads();
      continue;  // column already reduced
    }
    const double2 ph = ax0 > 0.0 ? cscale(x0, 1.0 / ax0) : make_double2(1.0, 0.0);
    const double2 alpha = cscale(ph, -xnorm);
    for (int i = tid; i < m; i += nt) v[i] = H[(k + 1 + i) * n + k];
    __syncthreads();
    if (tid == 0) v[0] = csub(x0, alpha);
    __syncthreads();
    double vv = 0.0;
    for (int i = tid; i < m; i += nt) vv += v[i].x * v[i].x + v[i].y * v[i].y;
    vv = block_sum(vv, red);
    const double beta = 2.0 / vv;
    // left: rows k+1.., columns k..n-1
    for (int j = k + tid; j < n; j += nt) {
      double2 sdot = make_double2(0.0, 0.0);
      for (int i = 0; i < m; ++i) sdot = cadd(sdot, cmul(cconj(v[i]), H[(k + 1 + i) * n + j]));
      sdot = cscale(sdot, beta);
      for (int i = 0; i < m; ++i) H[(k + 1 + i) * n + j] = csub(H[(k + 1 + i) * n + j], cmul(v[i], sdot));
    }
    __syncthreads();
    // right: all rows, columns k+1..n-1 (H and Q)
    for (int r = tid; r < 2 * n; r += nt) {
      double2* row = r < n ? &H[r * n] : &Q[size_t(r - n) * n];
      double2 sdot = make_double2(0.0, 0.0);
      for (int j = 0; j < m; ++j) sdot = cadd(sdot, cmul(row[k + 1 + j], v[j]));
      sdot = cscale(sdot, beta);
      for (int j = 0; j < m; ++j) row[k + 1 + j] = csub(row[k + 1 + j], cmul(sdot, cconj(v[j])));
    }
    __syncthreads();
    for (int i = tid; i < m; i += nt)
      if (i > 0) H[(k + 1 + i) * n + k] = make_double2(0.0, 0.0);
    __syncthreads();
  }

  // ---- shifted QR sweeps to Schur form ---------------------------------------
  const double eps = 2.2e-16;
  int hi = n - 1, iter = 0, its_here = 0;
  const int max_iter = 60 * n + 100;
  while (hi > 0) {
    if (tid == 0) {
      int l = hi;
      while (l > 0) {
        const double off = cabs2(H[l * n + l - 1]);
        const double dg = cabs2(H[l * n + l]) + cabs2(H[(l - 1) * n + l - 1]);
        if (off <= eps * (dg > 0.0 ? dg : fro)) {
          H[l * n + l - 1] = make_double2(0.0, 0.0);
          break;
        }
        --l;
      }
      ctl[0] = l;
    }
    __syncthreads();
    const int l = ctl[0];
    if (l == hi) {
      --hi;
      its_here = 0;
      __syncthreads();
      continue;
    }
    if (++iter > max_iter) {
      if (tid == 0) atomicExch(status, eig_status(kEigNoConvergence, n, hi));
      break;
    }
    ++its_here;
    for (int k = l; k < hi; ++k) {
      if (tid == 0) {
        double2 x, y;
        if (k == l) {
          // Wilkinson shift: eigenvalue of the trailing 2x2 closest to H[hi][hi]
          const double2 a = H[(hi - 1) * n + hi - 1], b = H[(hi - 1) * n + hi];
          const double2 c = H[hi * n + hi - 1], d = H[hi * n + hi];
          const double2 tr2 = cscale(cadd(a, d), 0.5);
          const double2 hd = cscale(csub(a, d), 0.5);
          const double2 disc = csqrt(cadd(cmul(hd, hd), cmul(b, c)));
          const double2 l1 = cadd(tr2, disc), l2 = csub(tr2, disc);
          double2 mu = cabs2(csub(l1, d)) < cabs2(csub(l2, d)) ? l1 : l2;
          if (its_here % 11 == 10 || !isfinite(mu.x) || !isfinite(mu.y)) {  // exceptional shift
            mu = cadd(d, make_double2(0.75 * cabs2(c), 0.0));
          }
          x = csub(H[l * n + l], mu);
          y = H[(l + 1) * n + l];
        } else {
          x = H[k * n + k - 1];
          y = H[(k + 1) * n + k - 1];
        }
        const double ax = cabs2(x), ay = cabs2(y);
        const double r = hypot(ax, ay);
        double c;
        double2 s;
        if (r == 0.0) {
          c = 1.0;
          s = make_double2(0.0, 0.0);
        } else if (ax == 0.0) {
          c = 0.0;
          s = cscale(cconj(y), 1.0 / ay);
        } else {
          c = ax / r;
          s = cscale(cmul(cscale(x, 1.0 / ax), cconj(y)), 1.0 / r);
        }
        gcs[0] = make_double2(c, 0.0);
        gcs[1] = s;
      }
      __syncthreads();
      const double c = gcs[0].x;
      const double2 s = gcs[1];
      // rows k, k+1 <- G rows
      for (int j = (k == l ? k : k - 1) + tid; j < n; j += nt) {
        const double2 a = H[k * n + j], b = H[(k + 1) * n + j];
        H[k * n + j] = cadd(cscale(a, c), cmul(s, b));
        H[(k + 1) * n + j] = csub(cscale(b, c), cmul(cconj(s), a));
      }
      __syncthreads();
      // columns k, k+1 <- columns G^H (H rows 0..min(k+2,hi), all of Q)
      const int rmax = min(k + 2, hi);
      for (int r = tid; r <= rmax + n; r += nt) {
        double2* row;
        if (r <= rmax) row = &H[r * n];
        else row = &Q[size_t(r - rmax - 1) * n];
        const double2 a = row[k], b = row[k + 1];
        row[k] = cadd(cscale(a, c), cmul(cconj(s), b));
        row[k + 1] = csub(cscale(b, c), cmul(s, a));
      }
      __syncthreads();
      if (k > l && tid == 0) H[(k + 1) * n + k - 1] = make_double2(0.0, 0.0);
      __syncthreads();
    }
  }
  __syncthreads();

  // ---- eigenvectors of T (unit upper triangular X), S = Q X, S^-1 = X^-1 Q^H --
  const double smin = fmax(eps * fro, tiny);
  for (int k = tid; k < n; k += nt) {
    const double2 tk = H[k * n + k];
    lam[k] = tk;
    for (int i = 0; i < n; ++i) X[size_t(i) * n + k] = make_double2(i == k ? 1.0 : 0.0, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int j = i + 1; j <= k; ++j) acc = cadd(acc, cmul(H[i * n + j], X[size_t(j) * n + k]));
      double2 den = csub(H[i * n + i], tk);
      if (cabs2(den) < smin) den = make_double2(smin, 0.0);
      X[size_t(i) * n + k] = cscale(cdiv(acc, den), -1.0);
    }
  }
  __syncthreads();
  for (int k = tid; k < n; k += nt) {
    // column k of X^-1: unit upper triangular back substitution
    for (int i = 0; i < n; ++i) Xi[size_t(i) * n + k] = make_double2(i == k ? 1.0 : 0.0, 0.0);
    for (int i = k - 1; i >= 0; --i) {
      double2 acc = make_double2(0.0, 0.0);
      for (int j = i + 1; j <= k; ++j) acc = cadd(acc, cmul(X[size_t(i) * n + j], Xi[size_t(j) * n + k]));
      Xi[size_t(i) * n + k] = cscale(acc, -1.0);
    }
  }
  __syncthreads();
  for (size_t t = tid; t < nn; t += nt) {
    const int i = int(t / n), k = int(t % n);
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    for (int j = 0; j <= k; ++j) a = cadd(a, cmul(Q[size_t(i) * n + j], X[size_t(j) * n + k]));
    for (int j = i; j < n; ++j) b = cadd(b, cmul(Xi[size_t(i) * n + j], cconj(Q[size_t(k) * n + j])));
    S[t] = a;
    Sinv[t] = b;
  }
}

}  // namespace

void launch_eig(const double2* M, int n, int count, double2* S, double2* Sinv, double2* lam,
                double2* ws, int* status, cudaStream_t s) {
  RTCC3_CHECK(n >= 1 && n <= kEigMaxN, kErrArg, "eigensolver supports n <= " + std::to_string(kEigMaxN));
  const size_t smem = size_t(n) * n * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    RTCC3_CUDA(cudaFuncSetAttribute(k_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(size_t(kEigMaxN) * kEigMaxN * sizeof(double2))));
    attr = true;
  }
  k_eig<<<count, 256, smem, s>>>(M, n, S, Sinv, lam, ws, status);
  RTCC3_CUDA(cudaGetLastError());
}

}  // namespace rtcc3
