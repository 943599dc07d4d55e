// Interpolation of FP64 coarse vectors with the FP64 locally orthonormal test
// vectors (P phi, Sec. 3): the second set-up part interpolates the harmonic
// Ritz vectors of D_c exactly, whatever format P is stored in for the solve.
#include "internal.h"

namespace sapmg {

// out(x) = sum_k v_k(x)|_chi phi[blk(x)][chi N + k], chi = 0 for spins 0, 1 and
// 1 for spins 2, 3 (the aggregates are the 4^4 blocks times chirality).
// v: N fine fields in the blocked layout; phi: [nblocks][2N]; one CTA per block.
__global__ void __launch_bounds__(256) prolong_v64_kernel(const double2* __restrict__ v, int N, size_t n,
                                                          const double2* __restrict__ phi, double2* __restrict__ out) {
  const int blk = blockIdx.x, loc = threadIdx.x;
  const double2* ph = phi + (size_t)blk * 2 * N;
  for (int c = 0; c < 12; ++c) {
    const size_t i = ((size_t)blk * 12 + c) * 256 + loc;
    const int off = (c < 6 ? 0 : N);
    double re = 0, im = 0;
    for (int k = 0; k < N; ++k) {
      const double2 a = v[(size_t)k * n + i], b = ph[off + k];
      re += a.x * b.x - a.y * b.y;
      im += a.x * b.y + a.y * b.x;
    }
    out[i] = make_double2(re, im);
  }
}

int launch_prolong_v64(const Geom& g, const void* v64, int N, const void* phi, void* out, cudaStream_t s) {
  if (N < 1) return MG_ERR_ARG;
  prolong_v64_kernel<<<(unsigned)g.nblocks, 256, 0, s>>>((const double2*)v64, N, (size_t)g.V * 12,
                                                         (const double2*)phi, (double2*)out);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
