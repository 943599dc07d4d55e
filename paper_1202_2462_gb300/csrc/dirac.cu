// K1: the clover-Wilson operator D over the whole lattice (Sec. 1, Eq. 1.1).
//
// One CTA per 4^4 block, one thread per site, fields in the blocked
// structure-of-arrays layout so that a warp's loads of one component are 256
// contiguous bytes (float2).  Hops are spin-projected (6 complex per
// neighbour instead of 12) and the antiperiodic time boundary, if any, is
// folded into the stored links.
#include "internal.h"
#include "stencil.cuh"

namespace sapmg {

template <class R, class TS, class TG>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 ? 3 : 1)) dirac_kernel(TS* __restrict__ out, const TS* __restrict__ in,
                                                    const TG* __restrict__ U, const TG* __restrict__ A, Geom g,
                                                    int nrhs) {
  // right-hand side fastest in the grid: the CTAs of one block run back to
  // back and share its links and clover through L2
  const int blk = blockIdx.x / nrhs;
  const int loc = threadIdx.x;
  const size_t off = (size_t)(blockIdx.x % nrhs) * g.V * 12;
  in += off;
  out += off;
  // acc = -2 A psi + sum of hops, so D psi = -acc / 2
  Cplx<R> acc[12];
  {
    Cplx<R> p[12];
    load_spinor<R>(in, blk, loc, p);
    clover_apply<R>(A, blk, loc, p, acc);
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = (R)(-2) * acc[c];
  hops_global_dir<0>(g, in, U, blk, loc, acc);
  hops_global_dir<1>(g, in, U, blk, loc, acc);
  hops_global_dir<2>(g, in, U, blk, loc, acc);
  hops_global_dir<3>(g, in, U, blk, loc, acc);
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = (R)(-0.5) * acc[c];
  store_spinor<R>(out, blk, loc, acc);
}

template <class R, class TS, class TG>
static void run(const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs, cudaStream_t s) {
  dirac_kernel<R, TS, TG><<<(unsigned)(g.nblocks * nrhs), 256, 0, s>>>((TS*)out, (const TS*)in, (const TG*)U,
                                                                      (const TG*)A, g, nrhs); count_launches(1);
}

int launch_dirac(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                 cudaStream_t s) {
  switch (prec) {
    case P64: run<double, double2, double2>(g, out, in, U, A, nrhs, s); break;
    case P32: run<float, float2, float2>(g, out, in, U, A, nrhs, s); break;
    case P16: run<float, float2, __half2>(g, out, in, U, A, nrhs, s); break;
    case PBF: run<float, float2, __nv_bfloat162>(g, out, in, U, A, nrhs, s); break;
    default: return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
