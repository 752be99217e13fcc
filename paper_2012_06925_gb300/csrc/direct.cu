// FP64 direct summation, Eq. (1), for error measurements on sampled targets.
// One thread per target and source split (the sources are split so that few
// targets still fill the device); sources are staged through shared memory
// and the splits are summed in order.  Pairs at distance 0 contribute nothing.
#include "internal.cuh"

namespace bldtt {

constexpr int kDirectThreads = 256;

template <int KERN>
__global__ void __launch_bounds__(kDirectThreads) k_direct(const double* __restrict__ t, int64_t M,
                                                           const double* __restrict__ src, int64_t N,
                                                           const double* __restrict__ q, double kappa,
                                                           int64_t span, double* __restrict__ part) {
  // blockIdx.y takes sources [y * span, min(N, (y + 1) * span)); part[y][i]
  __shared__ double4 tile[kDirectThreads];
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double x = 0, y = 0, z = 0;
  if (i < M) {
    x = t[i];
    y = t[M + i];
    z = t[2 * M + i];
  }
  const int64_t s0 = (int64_t)blockIdx.y * span, s1 = min(N, s0 + span);
  double acc = 0.0;
  for (int64_t base = s0; base < s1; base += kDirectThreads) {
    int64_t j = base + threadIdx.x;
    tile[threadIdx.x] = j < s1 ? make_double4(src[j], src[N + j], src[2 * N + j], q[j])
                               : make_double4(0, 0, 0, 0);
    __syncthreads();
    int cnt = (int)min((int64_t)kDirectThreads, s1 - base);
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
  if (i < M) part[(int64_t)blockIdx.y * M + i] = acc;
}

// phi[i] = sum over the source splits, in split order.
__global__ void k_direct_reduce(const double* __restrict__ part, int64_t M, int splits,
                                double* __restrict__ phi) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  double a = 0.0;
  for (int k = 0; k < splits; ++k) a += part[(int64_t)k * M + i];
  phi[i] = a;
}

int direct_sum(const double* targets, int64_t M, const double* sources, int64_t N,
               const double* charges, int kernel, double kappa, double* phi, cudaStream_t s) {
  const unsigned blocks = (unsigned)((M + kDirectThreads - 1) / kDirectThreads);
  // Split the sources so that the grid fills the device (few targets, many sources).
  int dev = 0, sms = 0;
  BL_CUDA(cudaGetDevice(&dev));
  BL_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int64_t splits = ((int64_t)4 * sms + blocks - 1) / blocks;
  const int64_t max_splits = (N + kDirectThreads - 1) / kDirectThreads;
  if (splits > max_splits) splits = max_splits;
  if (splits > 1024) splits = 1024;
  if (splits < 1) splits = 1;
  const int64_t span = (N + splits - 1) / splits;
  double* part = phi;
  if (splits > 1) BL_TRY(dalloc_n(&part, (size_t)(splits * M), s));
  const dim3 grid(blocks, (unsigned)splits);
  if (kernel == BLDTT_COULOMB)
    k_direct<BLDTT_COULOMB><<<grid, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, span, part);
  else if (kernel == BLDTT_YUKAWA)
    k_direct<BLDTT_YUKAWA><<<grid, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, span, part);
  else if (kernel == BLDTT_OSCILLATORY)
    k_direct<BLDTT_OSCILLATORY><<<grid, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, span, part);
  else if (kernel == BLDTT_REG_COULOMB)
    k_direct<BLDTT_REG_COULOMB><<<grid, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, span, part);
  else
    k_direct<BLDTT_TEST_POLY><<<grid, kDirectThreads, 0, s>>>(targets, M, sources, N, charges, kappa, span, part);
  int64_t dummy = 0;
  BL_LAUNCHED(dummy);
  if (splits > 1) {
    k_direct_reduce<<<blocks, kDirectThreads, 0, s>>>(part, M, (int)splits, phi);
    BL_LAUNCHED(dummy);
    dfree(part, s);
  }
  return BLDTT_OK;
}

}  // namespace bldtt
