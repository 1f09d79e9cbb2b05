// Integrator kernels around the residual graph: stage inputs, seeds, RK4
// accumulation in FP64, observables (dipole, energy) and Jacobi updates.
#include "model.h"

#include <cmath>

namespace rtcc3 {

namespace {

int grid_n(size_t n) {
  size_t g = (n + 255) / 256;
  return int(std::max<size_t>(1, std::min<size_t>(g, 152 * 8)));
}

// E(t) of one field slot: static, A cos(wt) (Eq. 14), Gaussian pulse
// (Eq. 32), and the ramped continuous waves of Section 2.2.4 with ramp
// duration t_r = width: linear (t / t_r) cos(wt) for t < t_r, and quadratic
// 2 t^2 / t_r^2 cos(wt) for t < t_r / 2, [1 - 2 (t - t_r)^2 / t_r^2] cos(wt)
// for t_r / 2 <= t < t_r; both A cos(wt) from t_r on and zero before t = 0.
__device__ double field_strength(const FieldDev& f, double t) {
  switch (f.kind) {
    case 1: return f.amp;
    case 2: return f.amp * cos(f.omega * t);
    case 3: return f.amp * exp(-(t - f.center) * (t - f.center) / (2.0 * f.width * f.width));
    case 4:
    case 5: {
      if (t < 0.0) return 0.0;
      const double tr = f.width;
      double ramp = 1.0;
      if (t < tr) {
        if (f.kind == 4) {
          ramp = t / tr;
        } else if (t < 0.5 * tr) {
          ramp = 2.0 * t * t / (tr * tr);
        } else {
          ramp = 1.0 - 2.0 * (t - tr) * (t - tr) / (tr * tr);
        }
      }
      return f.amp * ramp * cos(f.omega * t);
    }
    default: return 0.0;
  }
}

template <typename R>
__global__ void k_stage_inputs(const double2* __restrict__ y, const double2* __restrict__ kprev,
                               double ch, Cx<R>* __restrict__ t1, Cx<R>* __restrict__ t2,
                               Cx<R>* __restrict__ l1s, Cx<R>* __restrict__ l2s,
                               Cx<R>* __restrict__ w, const double* __restrict__ mu,
                               const FieldDev* __restrict__ f, const double* __restrict__ tdev,
                               double dt, int o, int v, int n) {
  const size_t n1 = size_t(o) * v, n2 = n1 * n1, nn = size_t(n) * n;
  const size_t total = 2 * (n1 + n2) + nn;
  const double E = field_strength(*f, *tdev + dt);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    if (t < 2 * (n1 + n2)) {
      double2 val = y[t];
      if (kprev) { val.x += ch * kprev[t].x; val.y += ch * kprev[t].y; }
      const Cx<R> c = cmake<R>(R(val.x), R(val.y));
      if (t < n1) t1[t] = c;
      else if (t < n1 + n2) t2[t - n1] = c;
      else if (t < 2 * n1 + n2) l1s[t - n1 - n2] = c;
      else l2s[t - 2 * n1 - n2] = c;
    } else {
      const size_t pq = t - 2 * (n1 + n2);
      const double m = f->dir[0] * mu[pq] + f->dir[1] * mu[nn + pq] + f->dir[2] * mu[2 * nn + pq];
      w[pq] = cmake<R>(R(-E * m), R(0));
    }
  }
}

template <typename R>
__global__ void k_seeds(Cx<R>* ge, Cx<R>* gr1, Cx<R>* gr2, const Cx<R>* l1s, const Cx<R>* l2s,
                        size_t n1, size_t n2) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n1 + n2 + 1;
       t += (size_t)gridDim.x * blockDim.x) {
    if (t < n1) gr1[t] = l1s[t];
    else if (t < n1 + n2) {
      const Cx<R> x = l2s[t - n1];
      gr2[t - n1] = cmake<R>(R(0.5) * x.x, R(0.5) * x.y);
    } else ge[0] = cmake<R>(R(1), R(0));
  }
}

// pair transpose index of t2[i,j,a,b] -> [j,i,b,a]
__device__ __forceinline__ size_t pairT(size_t t, int o, int v) {
  const int b = int(t % v), a = int((t / v) % v), j = int((t / v / v) % o), i = int(t / v / v / o);
  return ((size_t(j) * o + i) * v + b) * v + a;
}

// w_ia = -E(t) dir . mu_ia (FP64) of the field at the time *tdev + dt.
__device__ __forceinline__ double field_element(const FieldDev& f, const double* mu, double E,
                                                size_t nn, size_t pq) {
  return -E * (f.dir[0] * mu[pq] + f.dir[1] * mu[nn + pq] + f.dir[2] * mu[2 * nn + pq]);
}

template <typename R>
__global__ void k_stage_output(const Cx<R>* __restrict__ r1, const Cx<R>* __restrict__ r2,
                               const Cx<R>* __restrict__ g1, const Cx<R>* __restrict__ g2,
                               double2* __restrict__ kout, double2* __restrict__ acc, double hw,
                               const double* __restrict__ mu, const FieldDev* __restrict__ f,
                               const double* __restrict__ tdev, double dt, int o, int v) {
  const size_t n1 = size_t(o) * v, n2 = n1 * n1;
  const size_t total = 2 * (n1 + n2);
  const int n = o + v;
  const double E = field_strength(*f, *tdev + dt);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    double re, im;  // residual value R; k = -i R (T part) or +i R (lambda part)
    double sgn;
    if (t < n1) { re = r1[t].x; im = r1[t].y; sgn = -1.0; }
    else if (t < n1 + n2) { re = r2[t - n1].x; im = r2[t - n1].y; sgn = -1.0; }
    else if (t < 2 * n1 + n2) {
      const size_t q = t - n1 - n2;
      // the energy's field term 2 sum_ia w_ia t_ia is kept out of the graph:
      // its t1 derivative 2 w_ia joins the lambda residual here, in FP64
      const size_t pq = (q / v) * size_t(n) + o + q % v;
      re = double(g1[q].x) + 2.0 * field_element(*f, mu, E, size_t(n) * n, pq);
      im = g1[q].y;
      sgn = 1.0;
    } else {
      const size_t q = t - 2 * n1 - n2;
      const size_t p = pairT(q, o, v);
      re = double(g2[q].x) + double(g2[p].x);
      im = double(g2[q].y) + double(g2[p].y);
      sgn = 1.0;
    }
    // sgn * i * (re + i im) = sgn * (-im + i re)
    const double2 k = make_double2(-sgn * im, sgn * re);
    if (kout) kout[t] = k;
    if (acc) { acc[t].x += hw * k.x; acc[t].y += hw * k.y; }
  }
}

template <typename R>
__global__ void k_observables(const Cx<R>* __restrict__ D, const Cx<R>* __restrict__ e,
                              const double2* __restrict__ t1, const double* __restrict__ mu,
                              const FieldDev* __restrict__ f, const double* __restrict__ tdev,
                              double dt, int o, int v, const TrajDesc* __restrict__ td, int slot,
                              const int* step) {
  // one block per Cartesian component of the dipole, one per additional
  // observable, and the last for the energy; FP64 reductions in fixed order.
  // The graph's density and energy leave out the field-dressed reference
  // terms, added here in FP64: the energy's 2 sum_i w_ii + 2 sum_ia w_ia t_ia
  // and, for an operator O, its derivative part 2 sum_i O_ii + 2 sum_ia t_ia O_ia.
  __shared__ double sr[256], si[256];
  const int x = blockIdx.x, nobs = td->nobs;
  const int n = o + v;
  const size_t nn = size_t(n) * n, n1 = size_t(o) * v;
  double ar = 0.0, ai = 0.0;
  if (x < 3) {
    const double* m = mu + x * nn;
    for (size_t pq = threadIdx.x; pq < nn; pq += blockDim.x) {
      ar += double(D[pq].x) * m[pq];
      ai += double(D[pq].y) * m[pq];
    }
    for (size_t q = threadIdx.x; q < n1 + o; q += blockDim.x) {
      if (q < n1) {
        const double mia = m[(q / v) * size_t(n) + o + q % v];
        ar += 2.0 * t1[q].x * mia;
        ai += 2.0 * t1[q].y * mia;
      } else {
        ar += 2.0 * m[(q - n1) * size_t(n + 1)];
      }
    }
  } else if (x < int(gridDim.x) - 1) {
    if (x - 3 >= nobs) return;  // block-uniform
    const double2* op = td->ops + size_t(x - 3) * nn;
    for (size_t pq = threadIdx.x; pq < nn; pq += blockDim.x) {
      const double2 m = op[pq];
      const double dr = double(D[pq].x), di = double(D[pq].y);
      ar += dr * m.x - di * m.y;
      ai += dr * m.y + di * m.x;
    }
    for (size_t q = threadIdx.x; q < n1 + o; q += blockDim.x) {
      if (q < n1) {
        const double2 m = op[(q / v) * size_t(n) + o + q % v], tq = t1[q];
        ar += 2.0 * (tq.x * m.x - tq.y * m.y);
        ai += 2.0 * (tq.x * m.y + tq.y * m.x);
      } else {
        const double2 m = op[(q - n1) * size_t(n + 1)];
        ar += 2.0 * m.x;
        ai += 2.0 * m.y;
      }
    }
  } else {
    const double E = field_strength(*f, *tdev + dt);
    for (size_t q = threadIdx.x; q < n1 + o; q += blockDim.x) {
      if (q < n1) {
        const double wia = field_element(*f, mu, E, nn, (q / v) * size_t(n) + o + q % v);
        ar += 2.0 * t1[q].x * wia;
        ai += 2.0 * t1[q].y * wia;
      } else {
        ar += 2.0 * field_element(*f, mu, E, nn, (q - n1) * size_t(n + 1));
      }
    }
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long ent = (long long)slot * td->stride + (step ? *step : 0);
    if (x < 3) {
      if (td->dip) td->dip[size_t(ent) * 3 + x] = make_double2(sr[0], si[0]);
    } else if (x < int(gridDim.x) - 1) {
      if (td->obs) td->obs[size_t(ent) * nobs + (x - 3)] = make_double2(sr[0], si[0]);
    } else if (td->en) {
      td->en[ent] = make_double2(double(e[0].x) + sr[0], double(e[0].y) + si[0]);
    }
  }
}

template <typename R>
__global__ void k_residual_export(const Cx<R>* r1, const Cx<R>* r2, const Cx<R>* g1,
                                  const Cx<R>* g2, const double* __restrict__ mu,
                                  const FieldDev* __restrict__ f, const double* __restrict__ tdev,
                                  double2* out, int o, int v, int have_grad) {
  const size_t n1 = size_t(o) * v, n2 = n1 * n1;
  const size_t total = 2 * (n1 + n2);
  const int n = o + v;
  const double E = field_strength(*f, *tdev);
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total;
       t += (size_t)gridDim.x * blockDim.x) {
    double2 r = make_double2(0.0, 0.0);
    if (t < n1) r = make_double2(r1[t].x, r1[t].y);
    else if (t < n1 + n2) r = make_double2(r2[t - n1].x, r2[t - n1].y);
    else if (have_grad && t < 2 * n1 + n2) {
      // plus the t1 derivative 2 w_ia of the energy's field term (FP64)
      const size_t q = t - n1 - n2, pq = (q / v) * size_t(n) + o + q % v;
      r = make_double2(double(g1[q].x) + 2.0 * field_element(*f, mu, E, size_t(n) * n, pq),
                       g1[q].y);
    } else if (have_grad) {
      const size_t q = t - 2 * n1 - n2, p = pairT(q, o, v);
      r = make_double2(double(g2[q].x) + double(g2[p].x), double(g2[q].y) + double(g2[p].y));
    }
    out[t] = r;
  }
}

__device__ __forceinline__ void atomic_max_pos(double* addr, double val) {
  // val >= 0: the bit pattern of a non-negative double orders like an integer
  atomicMax(reinterpret_cast<unsigned long long*>(addr), __double_as_longlong(val));
}

__global__ void k_jacobi(double2* __restrict__ x1, double2* __restrict__ x2,
                         const double2* __restrict__ r1, const double2* __restrict__ r2,
                         const double* __restrict__ eps, int o, int v, double* maxr) {
  const size_t n1 = size_t(o) * v, n2 = n1 * n1;
  double m = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n1 + n2;
       t += (size_t)gridDim.x * blockDim.x) {
    double den;
    double2 r;
    double2* dst;
    if (t < n1) {
      const int a = int(t % v), i = int(t / v);
      den = eps[o + a] - eps[i];
      r = r1[t];
      dst = x1 + t;
    } else {
      const size_t q = t - n1;
      const int b = int(q % v), a = int((q / v) % v), j = int((q / v / v) % o), i = int(q / v / v / o);
      den = eps[o + a] + eps[o + b] - eps[i] - eps[j];
      r = r2[q];
      dst = x2 + q;
    }
    dst->x -= r.x / den;
    dst->y -= r.y / den;
    m = fmax(m, fmax(fabs(r.x), fabs(r.y)));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(maxr, m);
}

__global__ void k_diis_step(const double2* __restrict__ x, const double2* __restrict__ r,
                            const double* __restrict__ eps, int o, int v, double2* __restrict__ xs,
                            double2* __restrict__ es, double* maxr) {
  const size_t n1 = size_t(o) * v, n2 = n1 * n1;
  double m = 0.0;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n1 + n2;
       t += (size_t)gridDim.x * blockDim.x) {
    double den;
    if (t < n1) {
      const int a = int(t % v), i = int(t / v);
      den = eps[o + a] - eps[i];
    } else {
      const size_t q = t - n1;
      const int b = int(q % v), a = int((q / v) % v), j = int((q / v / v) % o), i = int(q / v / v / o);
      den = eps[o + a] + eps[o + b] - eps[i] - eps[j];
    }
    const double2 rr = r[t];
    const double2 e = make_double2(-rr.x / den, -rr.y / den);
    es[t] = e;
    xs[t] = make_double2(x[t].x + e.x, x[t].y + e.y);
    m = fmax(m, fmax(fabs(rr.x), fabs(rr.y)));
  }
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomic_max_pos(maxr, m);
}

__global__ void k_dots(const double2* __restrict__ E, const double2* __restrict__ e, size_t len,
                       double2* out) {
  __shared__ double sr[256], si[256];
  const double2* Ek = E + size_t(blockIdx.x) * len;
  double ar = 0.0, ai = 0.0;
  for (size_t t = threadIdx.x; t < len; t += blockDim.x) {
    const double2 a = Ek[t], b = e[t];
    ar += a.x * b.x + a.y * b.y;  // conj(a) * b
    ai += a.x * b.y - a.y * b.x;
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = make_double2(sr[0], si[0]);
}

__global__ void k_lincomb(const double2* __restrict__ X, const double2* __restrict__ c, int m,
                          size_t len, double2* __restrict__ x) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < len;
       t += (size_t)gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int k = 0; k < m; ++k) {
      const double2 a = X[size_t(k) * len + t], ck = c[k];
      re += ck.x * a.x - ck.y * a.y;
      im += ck.x * a.y + ck.y * a.x;
    }
    x[t] = make_double2(re, im);
  }
}

// y = acc (the RK4 result); with complex64 storage the state is rounded to
// complex64 after every step (FP64 arithmetic inside the step).
__global__ void k_step_finish(double2* __restrict__ y, const double2* __restrict__ acc, size_t ny,
                              const int* step, int* bad_step, int c64) {
  bool bad = false;
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < ny;
       t += (size_t)gridDim.x * blockDim.x) {
    double2 a = acc[t];
    if (!isfinite(a.x) || !isfinite(a.y)) bad = true;
    if (c64) a = make_double2(double(float(a.x)), double(float(a.y)));
    y[t] = a;
  }
  if (bad) atomicCAS(bad_step, -1, *step);
}

__global__ void k_step_advance(double* tdev, double h, int* step) {
  *tdev += h;
  *step += 1;
}

template <typename R>
__global__ void k_load_amplitudes(const double2* __restrict__ t1, const double2* __restrict__ t2,
                                  Cx<R>* __restrict__ d1, Cx<R>* __restrict__ d2, size_t n1,
                                  size_t n2) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n1 + n2;
       t += (size_t)gridDim.x * blockDim.x) {
    if (t < n1) d1[t] = cmake<R>(R(t1[t].x), R(t1[t].y));
    else d2[t - n1] = cmake<R>(R(t2[t - n1].x), R(t2[t - n1].y));
  }
}

template <typename R>
__global__ void k_export(const Cx<R>* __restrict__ in, double2* __restrict__ out, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    out[t] = make_double2(in[t].x, in[t].y);
}

template <typename R>
__global__ void k_field_operator(Cx<R>* __restrict__ w, const double* __restrict__ mu,
                                 const FieldDev* __restrict__ f, const double* __restrict__ tdev,
                                 double dt, int n) {
  const size_t nn = size_t(n) * n;
  const double E = field_strength(*f, *tdev + dt);
  for (size_t pq = blockIdx.x * (size_t)blockDim.x + threadIdx.x; pq < nn;
       pq += (size_t)gridDim.x * blockDim.x) {
    const double m = f->dir[0] * mu[pq] + f->dir[1] * mu[nn + pq] + f->dir[2] * mu[2 * nn + pq];
    w[pq] = cmake<R>(R(-E * m), R(0));
  }
}

__global__ void k_copy(double2* dst, const double2* src, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

}  // namespace

template <typename R>
void launch_stage_inputs(const double2* y, const double2* kprev, double ch, Cx<R>* t1, Cx<R>* t2,
                         Cx<R>* l1s, Cx<R>* l2s, Cx<R>* w, const double* mu, const FieldDev* f,
                         const double* tdev, double dt, int o, int v, int n, cudaStream_t s) {
  const size_t n1 = size_t(o) * v;
  const size_t total = 2 * (n1 + n1 * n1) + size_t(n) * n;
  k_stage_inputs<R><<<grid_n(total), 256, 0, s>>>(y, kprev, ch, t1, t2, l1s, l2s, w, mu, f, tdev,
                                                   dt, o, v, n);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_seeds(Cx<R>* ge, Cx<R>* gr1, Cx<R>* gr2, const Cx<R>* l1s, const Cx<R>* l2s, int o,
                  int v, cudaStream_t s) {
  const size_t n1 = size_t(o) * v;
  k_seeds<R><<<grid_n(n1 + n1 * n1 + 1), 256, 0, s>>>(ge, gr1, gr2, l1s, l2s, n1, n1 * n1);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_stage_output(const Cx<R>* r1, const Cx<R>* r2, const Cx<R>* g1, const Cx<R>* g2,
                         double2* kout, double2* acc, double hw, const double* mu,
                         const FieldDev* f, const double* tdev, double dt, int o, int v,
                         cudaStream_t s) {
  const size_t n1 = size_t(o) * v;
  k_stage_output<R><<<grid_n(2 * (n1 + n1 * n1)), 256, 0, s>>>(r1, r2, g1, g2, kout, acc, hw, mu,
                                                               f, tdev, dt, o, v);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_observables(const Cx<R>* D, const Cx<R>* e, const double2* t1, const double* mu,
                        const FieldDev* f, const double* tdev, double dt, int o, int v, int nobs,
                        const TrajDesc* td, int slot, const int* step, cudaStream_t s) {
  k_observables<R><<<4 + nobs, 256, 0, s>>>(D, e, t1, mu, f, tdev, dt, o, v, td, slot, step);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_residual_export(const Cx<R>* r1, const Cx<R>* r2, const Cx<R>* g1, const Cx<R>* g2,
                            const double* mu, const FieldDev* f, const double* tdev, double2* out,
                            int o, int v, bool have_grad, cudaStream_t s) {
  const size_t n1 = size_t(o) * v;
  k_residual_export<R><<<grid_n(2 * (n1 + n1 * n1)), 256, 0, s>>>(r1, r2, g1, g2, mu, f, tdev,
                                                                   out, o, v, have_grad ? 1 : 0);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_jacobi(double2* x1, double2* x2, const double2* r1, const double2* r2,
                   const double* eps, int o, int v, double* maxr, cudaStream_t s) {
  const size_t n1 = size_t(o) * v;
  k_jacobi<<<grid_n(n1 + n1 * n1), 256, 0, s>>>(x1, x2, r1, r2, eps, o, v, maxr);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_diis_step(const double2* x, const double2* r, const double* eps, int o, int v,
                      double2* xs, double2* es, double* maxr, cudaStream_t s) {
  const size_t n1 = size_t(o) * v;
  k_diis_step<<<grid_n(n1 + n1 * n1), 256, 0, s>>>(x, r, eps, o, v, xs, es, maxr);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_dots(const double2* E, const double2* e, int m, size_t len, double2* out, cudaStream_t s) {
  if (m <= 0) return;
  k_dots<<<m, 256, 0, s>>>(E, e, len, out);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_lincomb(const double2* X, const double2* c, int m, size_t len, double2* x, cudaStream_t s) {
  k_lincomb<<<grid_n(len), 256, 0, s>>>(X, c, m, len, x);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_step_finish(double2* y, const double2* acc, size_t ny, const int* step, int* bad_step,
                        bool c64, cudaStream_t s) {
  k_step_finish<<<grid_n(ny), 256, 0, s>>>(y, acc, ny, step, bad_step, c64 ? 1 : 0);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_step_advance(double* tdev, double h, int* step, cudaStream_t s) {
  k_step_advance<<<1, 1, 0, s>>>(tdev, h, step);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_load_amplitudes(const double2* t1, const double2* t2, Cx<R>* d1, Cx<R>* d2, int o,
                            int v, cudaStream_t s) {
  const size_t n1 = size_t(o) * v, n2 = n1 * n1;
  k_load_amplitudes<R><<<grid_n(n1 + n2), 256, 0, s>>>(t1, t2, d1, d2, n1, n2);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_export(const Cx<R>* in, double2* out, size_t n, cudaStream_t s) {
  k_export<R><<<grid_n(n), 256, 0, s>>>(in, out, n);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
__global__ void k_next_field_matrices(const double2* __restrict__ y, const Cx<R>* __restrict__ r1,
                                      double ch, const double* __restrict__ mu,
                                      const FieldDev* __restrict__ f,
                                      const double* __restrict__ tdev, double dt,
                                      const double* __restrict__ eps, int o, int v,
                                      double2* __restrict__ Mo, double2* __restrict__ Mv) {
  const int n = o + v;
  const size_t nn = size_t(n) * n;
  const double E = field_strength(*f, *tdev + dt);
  // the next stage's inputs, rounded as k_stage_inputs rounds them
  auto t1 = [&](int i, int a) {
    const size_t t = size_t(i) * v + a;
    double vx = y[t].x, vy = y[t].y;
    if (r1) {
      vx += ch * double(r1[t].y);  // k = -i r1
      vy += ch * -double(r1[t].x);
    }
    return make_double2(double(R(vx)), double(R(vy)));
  };
  auto w = [&](int p, int q) {
    const size_t pq = size_t(p) * n + q;
    const double m = f->dir[0] * mu[pq] + f->dir[1] * mu[nn + pq] + f->dir[2] * mu[2 * nn + pq];
    return double(R(-E * m));
  };
  const int total = o * o + v * v;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    if (t < o * o) {
      const int i = t / o, l = t % o;
      double re = w(l, i) + (i == l ? eps[i] : 0.0), im = 0.0;
      for (int a = 0; a < v; ++a) {
        const double2 x = t1(i, a);
        const double wl = w(l, o + a);
        re += wl * x.x;
        im += wl * x.y;
      }
      Mo[t] = make_double2(re, im);
    } else {
      const int q = t - o * o, a = q / v, d = q % v;
      double re = w(o + a, o + d) + (a == d ? eps[o + a] : 0.0), im = 0.0;
      for (int i = 0; i < o; ++i) {
        const double2 x = t1(i, a);
        const double wi = w(i, o + d);
        re -= x.x * wi;
        im -= x.y * wi;
      }
      Mv[q] = make_double2(re, im);
    }
  }
}

template <typename R>
void launch_next_field_matrices(const double2* y, const Cx<R>* r1, double ch, const double* mu,
                                const FieldDev* f, const double* tdev, double dt,
                                const double* eps, int o, int v, double2* Mo, double2* Mv,
                                cudaStream_t s) {
  const size_t total = size_t(o) * o + size_t(v) * v;
  k_next_field_matrices<R><<<int((total + 127) / 128), 128, 0, s>>>(y, r1, ch, mu, f, tdev, dt,
                                                                   eps, o, v, Mo, Mv);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_field_operator(Cx<R>* w, const double* mu, const FieldDev* f, const double* tdev,
                           double dt, int n, cudaStream_t s) {
  k_field_operator<R><<<grid_n(size_t(n) * n), 256, 0, s>>>(w, mu, f, tdev, dt, n);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_copy_c128(double2* dst, const double2* src, size_t n, cudaStream_t s) {
  k_copy<<<grid_n(n), 256, 0, s>>>(dst, src, n);
  RTCC3_CUDA(cudaGetLastError());
}

void launch_stage_prep_acc(double2* acc, const double2* y, size_t ny, cudaStream_t s) {
  launch_copy_c128(acc, y, ny, s);
}

#define RTCC3_INST(R)                                                                             \
  template void launch_stage_inputs<R>(const double2*, const double2*, double, Cx<R>*, Cx<R>*,    \
                                       Cx<R>*, Cx<R>*, Cx<R>*, const double*, const FieldDev*,    \
                                       const double*, double, int, int, int, cudaStream_t);       \
  template void launch_seeds<R>(Cx<R>*, Cx<R>*, Cx<R>*, const Cx<R>*, const Cx<R>*, int, int,     \
                                cudaStream_t);                                                    \
  template void launch_stage_output<R>(const Cx<R>*, const Cx<R>*, const Cx<R>*, const Cx<R>*,    \
                                       double2*, double2*, double, const double*,                 \
                                       const FieldDev*, const double*, double, int, int,          \
                                       cudaStream_t);                                             \
  template void launch_observables<R>(const Cx<R>*, const Cx<R>*, const double2*, const double*,  \
                                      const FieldDev*, const double*, double, int, int, int,      \
                                      const TrajDesc*, int, const int*, cudaStream_t);            \
  template void launch_residual_export<R>(const Cx<R>*, const Cx<R>*, const Cx<R>*, const Cx<R>*, \
                                          const double*, const FieldDev*, const double*, double2*, \
                                          int, int, bool, cudaStream_t);                          \
  template void launch_load_amplitudes<R>(const double2*, const double2*, Cx<R>*, Cx<R>*, int,  \
                                          int, cudaStream_t);                                     \
  template void launch_export<R>(const Cx<R>*, double2*, size_t, cudaStream_t);                   \
  template void launch_field_operator<R>(Cx<R>*, const double*, const FieldDev*, const double*,   \
                                         double, int, cudaStream_t);                              \
  template void launch_next_field_matrices<R>(const double2*, const Cx<R>*, double, const double*, \
                                              const FieldDev*, const double*, double,             \
                                              const double*, int, int, double2*, double2*,        \
                                              cudaStream_t);
RTCC3_INST(double)
RTCC3_INST(float)
#undef RTCC3_INST

}  // namespace rtcc3
