// Interpolation of FP64 coarse vectors with the FP64 locally orthonormal test
// vectors (P phi, Sec. 3): the second set-up part interpolates the harmonic
// Ritz vectors of D_c exactly, whatever format P is stored in for the solve;
// and the matching restriction P^dagger x, which the three-level set-up uses.
#include "internal.h"

namespace sapmg {

// out(x) = sum_k v_k(x)|_chi phi[blk(x)][chi N + k], chi = 0 for spins 0, 1 and
// 1 for spins 2, 3 (the aggregates are the 4^4 blocks times chirality).
// v: N fine fields in the blocked layout; phi: [nblocks][2N]; one CTA per block.
__global__ void __launch_bounds__(256) prolong_v64_kernel(const double2* __restrict__ v, int N, size_t n,
                                                          const double2* __restrict__ phi, double2* __restrict__ out) {
  const int blk = MG_CLAMP(kBlock, blockIdx.x, n / (12 * 256)), loc = threadIdx.x;
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

// The restriction with the same vectors, out[blk][chi N + k] = <v_k|_(blk, chi), x>
// (P^dagger x, Sec. 3), reading v in its vector-major layout: the set-up
// restricts fine fields this way without a block-major copy of P (at 48^3 x 96
// with N = 24 that copy would be another 49 GB).  One CTA per block; the sums
// over the block's sites run in a fixed order.
__global__ void __launch_bounds__(256) restrict_v64_kernel(const double2* __restrict__ v, int N, size_t n,
                                                           const double2* __restrict__ x, double2* __restrict__ out) {
  __shared__ double red[8][4];
  const int blk = MG_CLAMP(kBlock, blockIdx.x, n / (12 * 256)), loc = threadIdx.x, w = loc >> 5, lane = loc & 31;
  double2 xs[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) xs[c] = x[((size_t)blk * 12 + c) * 256 + loc];
  for (int k = 0; k < N; ++k) {
    double s[4] = {0, 0, 0, 0};                        // (re, im) for chirality 0, then 1
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const double2 a = v[(size_t)k * n + ((size_t)blk * 12 + c) * 256 + loc];
      const int h = c < 6 ? 0 : 2;
      s[h] += a.x * xs[c].x + a.y * xs[c].y;          // conj(a) x
      s[h + 1] += a.x * xs[c].y - a.y * xs[c].x;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
      for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
    if (lane == 0)
      for (int q = 0; q < 4; ++q) red[w][q] = s[q];
    __syncthreads();
    if (loc == 0) {
      double t[4] = {0, 0, 0, 0};
      for (int q = 0; q < 8; ++q)
        for (int e = 0; e < 4; ++e) t[e] += red[q][e];
      out[(size_t)blk * 2 * N + k] = make_double2(t[0], t[1]);
      out[(size_t)blk * 2 * N + N + k] = make_double2(t[2], t[3]);
    }
    __syncthreads();
  }
}

int launch_restrict_v64(const Geom& g, const void* v64, int N, const void* x, void* out, cudaStream_t s) {
  if (N < 1) return MG_ERR_ARG;
  restrict_v64_kernel<<<(unsigned)g.nblocks, 256, 0, s>>>((const double2*)v64, N, (size_t)g.V * 12,
                                                          (const double2*)x, (double2*)out);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
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
