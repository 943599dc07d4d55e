// K1, paired form: the clover-Wilson operator D over the whole lattice (Sec. 1,
// Eq. 1.1) for an even number of right-hand sides, two per thread, FP32
// arithmetic on FP32/FP16/BF16 fields.  One CTA per (4^4 block, pair of
// right-hand sides), one thread per site; each link and clover entry is loaded
// and converted once for both right-hand sides of the pair and every add,
// multiply and FMA is the packed two-wide instruction (pair.cuh), with the -1/2
// of the hopping term folded into the reconstruction FMAs.  The pairs of one
// block are adjacent CTAs, so the block's fields are shared through L1/L2.
#include "internal.h"
#include "pair.cuh"

namespace sapmg {
namespace {
using namespace pair;

template <class TG>
__global__ void __launch_bounds__(256, 2)
    dirac_pair_kernel(float2* __restrict__ out, const float2* __restrict__ in, const TG* __restrict__ U,
                      const TG* __restrict__ A, Geom g, int npairs) {
  const int blk = MG_CLAMP(kBlock, blockIdx.x / npairs, g.nblocks);
  const int loc = threadIdx.x;
  const size_t stride = (size_t)g.V * 12;
  const size_t off = (size_t)(blockIdx.x % npairs) * 2 * stride;
  in += off;
  out += off;
  const size_t site0 = (size_t)blk * 12 * 256 + loc;
  // acc = A psi - 1/2 sum(hops) = D psi
  P2 acc[12];
  clover2<TG>(A, blk, loc, [&](int k) { return ldg2(in, stride, site0 + k * 256); }, acc);
  global_hops2<0>(g, in, stride, U, blk, loc, acc);
  global_hops2<1>(g, in, stride, U, blk, loc, acc);
  global_hops2<2>(g, in, stride, U, blk, loc, acc);
  global_hops2<3>(g, in, stride, U, blk, loc, acc);
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const size_t i = site0 + c * 256;
    out[i] = make_float2(acc[c].re.x, acc[c].im.x);
    out[i + stride] = make_float2(acc[c].re.y, acc[c].im.y);
  }
}

template <class TG>
static int run_pair(const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs, cudaStream_t s) {
  const int npairs = nrhs / 2;
  dirac_pair_kernel<TG><<<(unsigned)(g.nblocks * npairs), 256, 0, s>>>((float2*)out, (const float2*)in,
                                                                        (const TG*)U, (const TG*)A, g, npairs);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace

int launch_dirac_pair(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                      cudaStream_t s) {
  if (nrhs < 2 || nrhs % 2 != 0) return MG_ERR_ARG;
  switch (prec) {
    case P32: return run_pair<float2>(g, out, in, U, A, nrhs, s);
    case P16: return run_pair<__half2>(g, out, in, U, A, nrhs, s);
    case PBF: return run_pair<__nv_bfloat162>(g, out, in, U, A, nrhs, s);
    default: return MG_ERR_ARG;
  }
}

}  // namespace sapmg
