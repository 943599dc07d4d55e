// K2: one colour pass of red-black Schwarz (Sec. 2, Algorithm 1).
//
// For every block i of colour c (blocks of one colour never touch, so they
// run as independent CTAs of one launch):
//   r = b - D z on the block's sites (full operator: halo z from the
//       neighbouring blocks of the other colour),
//   e ~ D_i^{-1} r by n_MR minimal-residual steps with the Dirichlet block
//       operator D_i = I^T D I (hops leaving the block dropped),
//   z += e.
// One CTA per block, one thread per site.  The MR iterate rho lives in shared
// memory for the neighbour accesses of D_i, and so does the correction e; the
// block-wide dots are warp shuffles plus one shared-memory exchange.  The two
// colours are two launches in stream order.
#include "internal.h"
#include "stencil.cuh"

namespace sapmg {

template <class R>
__device__ __forceinline__ void load_smem_spinor(const Cplx<R>* __restrict__ s, int loc, Cplx<R> (&p)[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) p[c] = s[c * 256 + loc];
}

// Sum of the hops of D_i at loc (neighbours inside the block only, from shared memory).
template <int MU, class R, class TG>
__device__ __forceinline__ void block_hops_dir(const TG* __restrict__ U, const Cplx<R>* __restrict__ rs, int blk,
                                               int loc, Cplx<R> (&acc)[12]) {
  const int ls = 1 << (2 * MU);
  const int c = (loc >> (2 * MU)) & 3;
  Cplx<R> h[6], gg[6], u[9];
  if (c < 3) {
    const Cplx<R>* q = rs + loc + ls;
    spin_project_ld<MU, -1, R>([&](int k) { return q[k * 256]; }, h);
    load_link<R>(U, blk, MU, loc, u);
    su3_mul(u, h, gg);
    spin_reconstruct_add<MU, -1>(gg, acc);
  }
  if (c > 0) {
    const Cplx<R>* q = rs + loc - ls;
    spin_project_ld<MU, 1, R>([&](int k) { return q[k * 256]; }, h);
    load_link<R>(U, blk, MU, loc - ls, u);
    su3_dag_mul(u, h, gg);
    spin_reconstruct_add<MU, 1>(gg, acc);
  }
}

template <class R>
__device__ __forceinline__ void block_reduce3(R& a, R& b, R& c, R (*red)[4]) {
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[w][0] = a; red[w][1] = b; red[w][2] = c; }
  __syncthreads();
  a = b = c = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) { a += red[k][0]; b += red[k][1]; c += red[k][2]; }
}

// Shared memory per CTA: the MR iterate rho and the block correction e
// (12 x 256 complex each, structure of arrays), and the reduction scratch.
// Registers hold one site's operator image p and the stencil temporaries only,
// so that two CTAs fit on an SM in FP32.
template <class R, class TS, class TG>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 ? 2 : 1))
    sap_colour_kernel(TS* __restrict__ z, const TS* __restrict__ b, const TG* __restrict__ U,
                      const TG* __restrict__ A, Geom g, int colour, int n_mr, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* rs = reinterpret_cast<Cplx<R>*>(smem_raw);                    // [12][256]
  Cplx<R>* es = rs + 12 * 256;                                            // [12][256]
  R (*red)[4] = reinterpret_cast<R (*)[4]>(smem_raw + sizeof(Cplx<R>) * 24 * 256);
  // right-hand side fastest in the grid (links and clover of a block shared through L2)
  const size_t off = (size_t)(blockIdx.x % nrhs) * g.V * 12;
  z += off;
  b += off;
  const int blk = colour_block(g, blockIdx.x / nrhs, colour);
  const int loc = threadIdx.x;

  // residual r = b - D z (Algorithm 1: residual update before the colour's block solves);
  // with acc = -2 A z + sum of hops, D z = -acc/2 and r = b + acc/2
  {
    Cplx<R> acc[12];
    {
      Cplx<R> zz[12];
      load_spinor<R>(z, blk, loc, zz);
      clover_apply<R>(A, blk, loc, zz, acc);
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = (R)(-2) * acc[c];
    hops_global_dir<0>(g, z, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    hops_global_dir<1>(g, z, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    hops_global_dir<2>(g, z, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    hops_global_dir<3>(g, z, U, blk, loc, acc);
    const TS* bq = b + (size_t)blk * 12 * 256 + loc;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      rs[c * 256 + loc] = Io<R, TS>::ldc(bq + c * 256) + (R)0.5 * acc[c];
      es[c * 256 + loc] = cmk<R>(0, 0);
    }
  }

  // n_MR minimal-residual steps on D_i e = r, D_i the block operator (hops leaving the block dropped)
  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();                                   // rho of every site written
    Cplx<R> p[12];
    {
      Cplx<R> ro[12];
      load_smem_spinor(rs, loc, ro);
      clover_apply<R>(A, blk, loc, ro, p);
    }
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = (R)(-2) * p[c];
    // the empty asm statements keep the compiler from hoisting the next
    // direction's loads (which would raise register pressure past the limit)
    block_hops_dir<0>(U, rs, blk, loc, p);
    asm volatile("" ::: "memory");
    block_hops_dir<1>(U, rs, blk, loc, p);
    asm volatile("" ::: "memory");
    block_hops_dir<2>(U, rs, blk, loc, p);
    asm volatile("" ::: "memory");
    block_hops_dir<3>(U, rs, blk, loc, p);
    R pr_re = 0, pr_im = 0, pp = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      p[c] = (R)(-0.5) * p[c];
      const Cplx<R> ro = rs[c * 256 + loc];
      pr_re += p[c].re * ro.re + p[c].im * ro.im;
      pr_im += p[c].re * ro.im - p[c].im * ro.re;
      pp += p[c].re * p[c].re + p[c].im * p[c].im;
    }
    block_reduce3(pr_re, pr_im, pp, red);            // contains the barrier after all neighbour reads
    Cplx<R> alpha = cmk<R>(0, 0);
    if (pp > (R)0) alpha = cmk(pr_re / pp, pr_im / pp);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const Cplx<R> ro = rs[c * 256 + loc];
      es[c * 256 + loc] = es[c * 256 + loc] + alpha * ro;
      rs[c * 256 + loc] = ro - alpha * p[c];
    }
  }
  // z += e on the block (own site only: no barrier needed)
  TS* zq = z + (size_t)blk * 12 * 256 + loc;
#pragma unroll
  for (int c = 0; c < 12; ++c) Io<R, TS>::st(zq + c * 256, Io<R, TS>::ldc(zq + c * 256) + es[c * 256 + loc]);
}

template <class R, class TS, class TG>
static int run(const Geom& g, void* z, const void* b, const void* U, const void* A, int colour, int n_mr, int nrhs,
               cudaStream_t s) {
  const size_t smem = sizeof(Cplx<R>) * 24 * 256 + sizeof(R) * 8 * 4;
  static bool attr = false;
  if (!attr) {
    SAPMG_CUDA_TRY(cudaFuncSetAttribute(sap_colour_kernel<R, TS, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  sap_colour_kernel<R, TS, TG><<<(unsigned)(g.nblocks / 2 * nrhs), 256, smem, s>>>(
      (TS*)z, (const TS*)b, (const TG*)U, (const TG*)A, g, colour, n_mr, nrhs); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_sap_colour(int prec, const Geom& g, void* z, const void* b, const void* U, const void* A, int colour,
                      int n_mr, int nrhs, cudaStream_t s, int pair_shape, int* err) {
  // an even number of FP32-arithmetic right-hand sides goes to the paired
  // kernel (sap2.cu) unless pair_shape < 0
  if (pair_shape >= 0 && prec != P64 && nrhs >= 2 && nrhs % 2 == 0 && n_mr >= 1)
    return launch_sap_colour_pair(prec, g, z, b, U, A, colour, n_mr, nrhs, s, pair_shape, err);
  switch (prec) {
    case P64: return run<double, double2, double2>(g, z, b, U, A, colour, n_mr, nrhs, s);
    case P32: return run<float, float2, float2>(g, z, b, U, A, colour, n_mr, nrhs, s);
    case P16: return run<float, float2, __half2>(g, z, b, U, A, colour, n_mr, nrhs, s);
    case PBF: return run<float, float2, __nv_bfloat162>(g, z, b, U, A, colour, n_mr, nrhs, s);
    default: return MG_ERR_ARG;
  }
}

}  // namespace sapmg
