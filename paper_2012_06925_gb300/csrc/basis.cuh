// Lagrange basis on Chebyshev proxy grids (Sec. 2.1, Eqs. (3)-(5)) and a
// compensated float dot product, shared by the SIMT and the tensor-core
// forms of the leaf passes.
#pragma once

#include "internal.cuh"

namespace bldtt {

// Barycentric weight of Chebyshev points of the 2nd kind, Eq. (5).
__device__ __forceinline__ double bary_weight(int k, int n) {
  double w = (k == 0 || k == n) ? 0.5 : 1.0;
  return (k & 1) ? -w : w;
}

// L_k(x), k = 0..n, of the 1D grid `nodes` (Eq. (3)), written to out[k*stride].
// If x - t_k == 0 for some k, the result is one-hot at the first such k.
template <typename T>
__device__ __forceinline__ void basis_1d(double x, const double* nodes, int n, T* out, int stride) {
  double r[kMaxP];
  int hit = -1;
  double sum = 0.0;
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) {
    if (k <= n) {
      double d = x - nodes[k];
      if (d == 0.0 && hit < 0) hit = k;
      r[k] = d == 0.0 ? 0.0 : bary_weight(k, n) / d;
      sum += r[k];
    }
  }
  double inv = 1.0 / sum;
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) {
    if (k <= n) out[k * stride] = (T)(hit >= 0 ? (k == hit ? 1.0 : 0.0) : r[k] * inv);
  }
}

// FP32_BULK form of the same basis: x and the nodes are split into float
// pairs (hi = fl(v), lo = fl(v - hi)), so d_k = (x_hi - t_hi) + (x_lo - t_lo)
// is x - t_k to within u |d_k| + u^2 |x|; d_k == 0 (x and t_k equal to ~48
// bits) takes the guard.  The weights are exact; the quotients and their sum
// are float.  nodes_hl: [2][n+1] (hi row, lo row).
__device__ __forceinline__ void basis_1d_f32(double x, const float* nodes_hl, int n, float* out,
                                             int stride) {
  float xh, xl;
  split_f64(x, xh, xl);
  float r[kMaxP];
  int hit = -1;
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) {
    if (k <= n) {
      const float d = __fadd_rn(__fsub_rn(xh, nodes_hl[k]), __fsub_rn(xl, nodes_hl[kMaxP + k]));
      if (d == 0.f && hit < 0) hit = k;
      r[k] = d == 0.f ? 0.f : __fdividef((float)bary_weight(k, n), d);
      sum += r[k];
    }
  }
  const float inv = __fdividef(1.f, sum);
#pragma unroll
  for (int k = 0; k < kMaxP; ++k) {
    if (k <= n) out[k * stride] = hit >= 0 ? (k == hit ? 1.f : 0.f) : r[k] * inv;
  }
}

// basis_1d_f32 for a grid of P points fixed at compile time, into registers
// (the same operations in the same order).
template <int P>
__device__ __forceinline__ void basis_f32_fixed(double x, const float* nodes_hl, float (&out)[P]) {
  float xh, xl;
  split_f64(x, xh, xl);
  float r[P];
  int hit = -1;
  float sum = 0.f;
#pragma unroll
  for (int k = 0; k < P; ++k) {
    const float d = __fadd_rn(__fsub_rn(xh, nodes_hl[k]), __fsub_rn(xl, nodes_hl[kMaxP + k]));
    if (d == 0.f && hit < 0) hit = k;
    r[k] = d == 0.f ? 0.f : __fdividef((float)bary_weight(k, P - 1), d);
    sum += r[k];
  }
  const float inv = __fdividef(1.f, sum);
#pragma unroll
  for (int k = 0; k < P; ++k) out[k] = hit >= 0 ? (k == hit ? 1.f : 0.f) : r[k] * inv;
}

// Compensated float sum of products: s + c carries sum a_i b_i with the
// rounding errors of every product (FMA) and every addition (TwoSum).
struct CompSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    c = __fadd_rn(c, __fadd_rn(e, pe));
    s = t;
  }
};

}  // namespace bldtt
