// One colour pass of red-black Schwarz for the shifted operator D - lambda
// (lambda per right-hand side): the smoother S(lambda) of the set-up's second
// part (Sec. 3), whose block solves are B_j(lambda) = I [I^T (D - lambda) I]^{-1} I^T,
// here n_MR minimal-residual steps on the shifted block systems.
//
// The layout and the steps are those of the solve's Schwarz pass
// (r = b - (D - lambda) z on the block, n_MR MR steps with D_j - lambda, z += e);
// it runs a few times per set-up, so it is written plainly (no tuning of
// its register use) and kept apart from the solve's kernel.
#include "internal.h"
#include "stencil.cuh"

namespace sapmg {

namespace {

// hops of the Dirichlet block operator D_j at loc (neighbours from shared memory)
template <int MU, class R, class TG>
__device__ __forceinline__ void shifted_block_hops(const TG* __restrict__ U, const Cplx<R>* __restrict__ rs, int blk,
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

template <class R, class TS, class TG>
__global__ void __launch_bounds__(256) sap_shifted_kernel(TS* __restrict__ z, const TS* __restrict__ b,
                                                          const TG* __restrict__ U, const TG* __restrict__ A, Geom g,
                                                          int colour, int n_mr, int nrhs,
                                                          const double2* __restrict__ shift) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* rs = reinterpret_cast<Cplx<R>*>(smem_raw);        // MR iterate rho [12][256]
  Cplx<R>* es = rs + 12 * 256;                                // correction e [12][256]
  R* red = reinterpret_cast<R*>(es + 12 * 256);               // [8][3]
  const int r_ = blockIdx.x % nrhs;
  const size_t off = (size_t)r_ * g.V * 12;
  z += off;
  b += off;
  const int blk = colour_block(g, blockIdx.x / nrhs, colour);
  const int loc = threadIdx.x;
  const Cplx<R> lam = cmk<R>((R)shift[r_].x, (R)shift[r_].y);

  // r = b - (D - lambda) z; with acc = -2 A z + hops, D z = -acc / 2
  {
    Cplx<R> acc[12], zz[12];
    load_spinor<R>(z, blk, loc, zz);
    clover_apply<R>(A, blk, loc, zz, acc);
#pragma unroll
    for (int c = 0; c < 12; ++c) acc[c] = (R)(-2) * acc[c];
    hops_global_dir<0>(g, z, U, blk, loc, acc);
    hops_global_dir<1>(g, z, U, blk, loc, acc);
    hops_global_dir<2>(g, z, U, blk, loc, acc);
    hops_global_dir<3>(g, z, U, blk, loc, acc);
    const TS* bq = b + (size_t)blk * 12 * 256 + loc;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      rs[c * 256 + loc] = Io<R, TS>::ldc(bq + c * 256) + (R)0.5 * acc[c] + lam * zz[c];
      es[c * 256 + loc] = cmk<R>(0, 0);
    }
  }
  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();
    Cplx<R> p[12], ro[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) ro[c] = rs[c * 256 + loc];
    clover_apply<R>(A, blk, loc, ro, p);
#pragma unroll
    for (int c = 0; c < 12; ++c) p[c] = (R)(-2) * p[c];
    shifted_block_hops<0>(U, rs, blk, loc, p);
    shifted_block_hops<1>(U, rs, blk, loc, p);
    shifted_block_hops<2>(U, rs, blk, loc, p);
    shifted_block_hops<3>(U, rs, blk, loc, p);
    // p = (D_j - lambda) rho; <p, rho> and <p, p> over the block
    R pr_re = 0, pr_im = 0, pp = 0;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      p[c] = (R)(-0.5) * p[c] - lam * ro[c];
      pr_re += p[c].re * ro[c].re + p[c].im * ro[c].im;
      pr_im += p[c].re * ro[c].im - p[c].im * ro[c].re;
      pp += p[c].re * p[c].re + p[c].im * p[c].im;
    }
    pr_re = warp_sum(pr_re);
    pr_im = warp_sum(pr_im);
    pp = warp_sum(pp);
    const int w = loc >> 5;
    if ((loc & 31) == 0) { red[w * 3] = pr_re; red[w * 3 + 1] = pr_im; red[w * 3 + 2] = pp; }
    __syncthreads();                                   // also: every neighbour read of rho is done
    pr_re = pr_im = pp = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) { pr_re += red[k * 3]; pr_im += red[k * 3 + 1]; pp += red[k * 3 + 2]; }
    Cplx<R> alpha = cmk<R>(0, 0);
    if (pp > (R)0) alpha = cmk(pr_re / pp, pr_im / pp);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      es[c * 256 + loc] = es[c * 256 + loc] + alpha * ro[c];
      rs[c * 256 + loc] = ro[c] - alpha * p[c];
    }
    __syncthreads();                                   // red is rewritten in the next step
  }
  TS* zq = z + (size_t)blk * 12 * 256 + loc;
#pragma unroll
  for (int c = 0; c < 12; ++c) Io<R, TS>::st(zq + c * 256, Io<R, TS>::ldc(zq + c * 256) + es[c * 256 + loc]);
}

template <class R, class TS, class TG>
int run_shifted(const Geom& g, void* z, const void* b, const void* U, const void* A, int colour, int n_mr, int nrhs,
                const double2* shift, cudaStream_t s) {
  const size_t smem = sizeof(Cplx<R>) * 24 * 256 + sizeof(R) * 8 * 3;
  static bool attr = false;
  if (!attr) {
    SAPMG_CUDA_TRY(cudaFuncSetAttribute(sap_shifted_kernel<R, TS, TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  sap_shifted_kernel<R, TS, TG><<<(unsigned)(g.nblocks / 2 * nrhs), 256, smem, s>>>(
      (TS*)z, (const TS*)b, (const TG*)U, (const TG*)A, g, colour, n_mr, nrhs, shift);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace

int launch_sap_colour_shifted(int prec, const Geom& g, void* z, const void* b, const void* U, const void* A,
                              int colour, int n_mr, int nrhs, const double2* shift, cudaStream_t s) {
  if (!shift || nrhs < 1) return MG_ERR_ARG;
  switch (prec) {
    case P64: return run_shifted<double, double2, double2>(g, z, b, U, A, colour, n_mr, nrhs, shift, s);
    case P32: return run_shifted<float, float2, float2>(g, z, b, U, A, colour, n_mr, nrhs, shift, s);
    case P16: return run_shifted<float, float2, __half2>(g, z, b, U, A, colour, n_mr, nrhs, shift, s);
    case PBF: return run_shifted<float, float2, __nv_bfloat162>(g, z, b, U, A, colour, n_mr, nrhs, shift, s);
    default: return MG_ERR_ARG;
  }
}

}  // namespace sapmg
