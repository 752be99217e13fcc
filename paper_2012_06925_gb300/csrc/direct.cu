// FP64 direct summation, Eq. (1), for error measurements on sampled targets.
// One thread per target; sources are staged through shared memory.  Pairs at
// distance 0 contribute nothing.
#include "internal.cuh"

namespace bldtt {

constexpr int kDirectThreads = 256;

template <int KERN>
__global__ void __launch_bounds__(kDirectThreads) k_direct(const double* __restrict__ t, int64_t M,
                                                           const double* __restrict__ src, int64_t N,
                                                           const double* __restrict__ q, double kappa,
                                                           double* __restrict__ phi) {
  __shared__ double4 tile[kDirectThreads];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x = 0, y = 0, z = 0;
  if (i < M) {
    x = t[i];
    y = t[M + i];
    z = t[2 * M + i];
  }
  double acc = 0.0;
  for (int64_t base = 0; base < N; base += kDirectThreads) {
    int64_t j = base + threadIdx.x;
    tile[threadIdx.x] = j < N ? make_double4(src[j], src[N + j], src[2 * N + j], q[j])
                              : make_double4(0, 0, 0, 0);
    __syncthreads();
    int cnt = (int)min((int64_t)kDirectThreads, N - base);
    for (int k = 0; k < cnt; ++k) {
      double4 p = tile[k];
      double dx = x - p.x, dy = y - p.y, dz = z - p.z;
      double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 > 0.0) {
        double g;
        if (KERN == BLDTT_COULOMB) {
          g = rsqrt(r2);
        } else if (KERN == BLDTT_YUKAWA) {
          double r = sqrt(r2);
          g = exp(-kappa * r) / r;
        } else if (KERN == BLDTT_OSCILLATORY) {
          double r = sqrt(r2);
          g = sin(kappa * r) / r;
        } else if (KERN == BLDTT_REG_COULOMB) {
          g = rsqrt(r2 + kappa * kappa);
        } else {
          g = 1.0 + dx - 2.0 * dy + 3.0 * dz + dx * dy - dy * dz + dx * dx * dz * dz - 0.5 * dy * dy;
        }
        acc += g * p.w;
      }
    }
    __syncthreads();
  }
  if (i < M) phi[i] = acc;
}

int direct_sum(const double* targets, int64_t M, const double* sources, int64_t N,
               const double* charges, int kernel, double kappa, double* phi, cudaStream_t s) {
  unsigned blocks = (unsigned)((M + kDirectThreads - 1) / kDirectThreads);
  if (kernel == BLDTT_COULOMB)
    k_direct<BLDTT_COULOMB><<<blocks, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, phi);
  else if (kernel == BLDTT_YUKAWA)
    k_direct<BLDTT_YUKAWA><<<blocks, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, phi);
  else if (kernel == BLDTT_OSCILLATORY)
    k_direct<BLDTT_OSCILLATORY><<<blocks, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, phi);
  else if (kernel == BLDTT_REG_COULOMB)
    k_direct<BLDTT_REG_COULOMB><<<blocks, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, phi);
  else
    k_direct<BLDTT_TEST_POLY><<<blocks, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, phi);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  return BLDTT_OK;
}

}  // namespace bldtt
