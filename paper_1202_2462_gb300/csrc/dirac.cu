// K1: the clover-Wilson operator D over the whole lattice (Sec. 1, Eq. 1.1).
//
// One CTA per 4^4 block, one thread per site, fields in the blocked
// structure-of-arrays layout so that a warp's loads of one component are 256
// contiguous bytes (float2).  Hops are spin-projected (6 complex per
// neighbour instead of 12) and the antiperiodic time boundary, if any, is
// folded into the stored links.
#include "internal.h"
#include "stencil.cuh"
#include "dfloat.cuh"

namespace sapmg {

// DAG: apply D^dagger = gamma5 D gamma5 instead (the operator of the normal
// equations).  NORM: also write the CTA's share of ||out||^2 to
// part[blockIdx.x] (CTA index = block * nrhs + right-hand side), reduced in a
// fixed order so that the result does not depend on scheduling.
template <class R, class TS, class TG, bool DAG, bool NORM>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 ? 3 : 1)) dirac_kernel(TS* __restrict__ out, const TS* __restrict__ in,
                                                    const TG* __restrict__ U, const TG* __restrict__ A, Geom g,
                                                    int nrhs, double* __restrict__ part) {
  // right-hand side fastest in the grid: the CTAs of one block run back to
  // back and share its links and clover through L2
  const int blk = MG_CLAMP(kBlock, blockIdx.x / nrhs, g.nblocks);
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
  hops_global_dir<0, R, TS, TG, DAG>(g, in, U, blk, loc, acc);
  hops_global_dir<1, R, TS, TG, DAG>(g, in, U, blk, loc, acc);
  hops_global_dir<2, R, TS, TG, DAG>(g, in, U, blk, loc, acc);
  hops_global_dir<3, R, TS, TG, DAG>(g, in, U, blk, loc, acc);
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = (R)(-0.5) * acc[c];
  store_spinor<R>(out, blk, loc, acc);
  if constexpr (NORM) {
    __shared__ double ws[8];
    R t = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) t += acc[c].re * acc[c].re + acc[c].im * acc[c].im;
    t = warp_sum(t);
    if ((loc & 31) == 0) ws[loc >> 5] = (double)t;
    __syncthreads();
    if (loc == 0) {
      double sum = 0;
      for (int w = 0; w < 8; ++w) sum += ws[w];
      part[blockIdx.x] = sum;
    }
  }
}

template <class R, class TS, class TG, bool DAG, bool NORM>
static void run(const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs, double* part,
                cudaStream_t s) {
  dirac_kernel<R, TS, TG, DAG, NORM><<<(unsigned)(g.nblocks * nrhs), 256, 0, s>>>(
      (TS*)out, (const TS*)in, (const TG*)U, (const TG*)A, g, nrhs, part);
  count_launches(1);
}

template <class R, class TS, class TG>
static void run_ex(const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs, bool dag,
                   double* part, cudaStream_t s) {
  if (dag) {
    if (part) run<R, TS, TG, true, true>(g, out, in, U, A, nrhs, part, s);
    else run<R, TS, TG, true, false>(g, out, in, U, A, nrhs, part, s);
  } else {
    if (part) run<R, TS, TG, false, true>(g, out, in, U, A, nrhs, part, s);
    else run<R, TS, TG, false, false>(g, out, in, U, A, nrhs, part, s);
  }
}

int launch_dirac_ex(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                    bool dag, double* part, cudaStream_t s) {
  switch (prec) {
    case P64: run_ex<double, double2, double2>(g, out, in, U, A, nrhs, dag, part, s); break;
    case P64E:                             // FP64 data, double-float arithmetic (dfloat.cuh)
      if (dag || part) return MG_ERR_ARG;
      run<DF, double2, double2, false, false>(g, out, in, U, A, nrhs, nullptr, s);
      break;
    case P32: run_ex<float, float2, float2>(g, out, in, U, A, nrhs, dag, part, s); break;
    case P16:
      if (dag || part) return MG_ERR_ARG;
      run<float, float2, __half2, false, false>(g, out, in, U, A, nrhs, nullptr, s);
      break;
    case PBF:
      if (dag || part) return MG_ERR_ARG;
      run<float, float2, __nv_bfloat162, false, false>(g, out, in, U, A, nrhs, nullptr, s);
      break;
    default: return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_dirac(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                 cudaStream_t s) {
  return launch_dirac_ex(prec, g, out, in, U, A, nrhs, false, nullptr, s);
}

}  // namespace sapmg
