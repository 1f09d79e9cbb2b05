// Small kernels around the field-dressed eigenbasis (see rotation.h).
#include "rotation.h"

namespace rtcc3 {

namespace {

template <typename R>
__global__ void k_field_matrices(const Cx<R>* __restrict__ wt, const double* __restrict__ eps,
                                 int o, int v, double2* __restrict__ Mo,
                                 double2* __restrict__ Mv) {
  const int n = o + v;
  const int total = o * o + v * v;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    if (t < o * o) {
      const int i = t / o, l = t % o;
      // O[i][l] = e_i delta_il + w~_li
      const Cx<R> w = wt[l * n + i];
      Mo[t] = make_double2(double(w.x) + (i == l ? eps[i] : 0.0), double(w.y));
    } else {
      const int q = t - o * o;
      const int a = q / v, d = q % v;
      // V[a][d] = e_a delta_ad + w~_ad
      const Cx<R> w = wt[(o + a) * n + o + d];
      Mv[q] = make_double2(double(w.x) + (a == d ? eps[o + a] : 0.0), double(w.y));
    }
  }
}

template <typename R>
__global__ void k_lambda_sums(const double2* __restrict__ lo, const double2* __restrict__ lv, int o,
                              int v, double c, Cx<R>* __restrict__ os, Cx<R>* __restrict__ vs) {
  const int no = o * o * o, nv = v * v * v;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < no + nv; t += gridDim.x * blockDim.x) {
    if (t < no) {
      const int k = t % o, j = (t / o) % o, i = t / (o * o);
      os[t] = cmake<R>(R((lo[i].x - c) + (lo[j].x - c) + (lo[k].x - c)),
                       R(lo[i].y + lo[j].y + lo[k].y));
    } else {
      const int q = t - no;
      const int cc = q % v, b = (q / v) % v, a = q / (v * v);
      vs[q] = cmake<R>(R((lv[a].x - c) + (lv[b].x - c) + (lv[cc].x - c)),
                       R(lv[a].y + lv[b].y + lv[cc].y));
    }
  }
}

template <typename R>
__global__ void k_to_precision(const double2* __restrict__ src, Cx<R>* __restrict__ dst, size_t n) {
  for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < n;
       t += (size_t)gridDim.x * blockDim.x)
    dst[t] = cmake<R>(R(src[t].x), R(src[t].y));
}

int blocks_for(size_t n) { return int(std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 1216))); }

}  // namespace

template <typename R>
void launch_field_matrices(const Cx<R>* wt, const double* eps, int o, int v, double2* Mo,
                           double2* Mv, cudaStream_t s) {
  k_field_matrices<R><<<blocks_for(size_t(o) * o + size_t(v) * v), 256, 0, s>>>(wt, eps, o, v, Mo, Mv);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_lambda_sums(const double2* lo, const double2* lv, int o, int v, double shift,
                        Cx<R>* osum, Cx<R>* vsum, cudaStream_t s) {
  const size_t n = size_t(o) * o * o + size_t(v) * v * v;
  k_lambda_sums<R><<<blocks_for(n), 256, 0, s>>>(lo, lv, o, v, shift, osum, vsum);
  RTCC3_CUDA(cudaGetLastError());
}

template <typename R>
void launch_to_precision(const double2* src, Cx<R>* dst, size_t n, cudaStream_t s) {
  k_to_precision<R><<<blocks_for(n), 256, 0, s>>>(src, dst, n);
  RTCC3_CUDA(cudaGetLastError());
}

template void launch_field_matrices<double>(const Cx<double>*, const double*, int, int, double2*,
                                            double2*, cudaStream_t);
template void launch_field_matrices<float>(const Cx<float>*, const double*, int, int, double2*,
                                           double2*, cudaStream_t);
template void launch_to_precision<double>(const double2*, Cx<double>*, size_t, cudaStream_t);
template void launch_lambda_sums<double>(const double2*, const double2*, int, int, double,
                                         Cx<double>*,
                                         Cx<double>*, cudaStream_t);
template void launch_lambda_sums<float>(const double2*, const double2*, int, int, double,
                                        Cx<float>*,
                                        Cx<float>*, cudaStream_t);
template void launch_to_precision<float>(const double2*, Cx<float>*, size_t, cudaStream_t);

}  // namespace rtcc3
