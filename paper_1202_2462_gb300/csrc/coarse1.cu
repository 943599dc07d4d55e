// Kernels of the intermediate level of a three-level hierarchy (Sec. 3: the
// two-level construction applied recursively to the coarse equation).
//
// Level-1 fields are canonical on the lattice of 4^4 aggregates: [site][n2]
// (n2 = 2 N0 dof, chirality chi = dof / N0).  Level-1 Schwarz blocks and
// level-2 aggregates are boxes of coarse sites (Box4).  Level-1 test vectors
// are vector-major [k][site][n2]; the level-2 operator uses the stencil layout
// M[site][d][j][i] of every coarse level.
#include "internal.h"
#include "coarse.h"

namespace sapmg {

__device__ __forceinline__ int c_coord(const CGeom& c, int site, int mu) {
  int s = site;
  for (int m = 0; m < mu; ++m) s /= c.L[m];
  return s % c.L[mu];
}

__device__ __forceinline__ int c_site(const CGeom& c, const int (&x)[4]) {
  return MG_CLAMP(kCoarseSite, ((x[3] * c.L[2] + x[2]) * c.L[1] + x[1]) * c.L[0] + x[0], c.nsites);
}

// Box index and box coordinates -> the k-th box of a colour ((sum of box coords) mod 2).
__device__ __forceinline__ int colour_box(const Box4& bx, int k, int colour, int (&bc)[4]) {
  k = MG_CLAMP(kBlock, k, bx.nboxes >> 1);
  const int half = bx.nb[0] >> 1;
  const int j = k % half;
  int rest = k / half;
  bc[1] = rest % bx.nb[1];
  rest /= bx.nb[1];
  bc[2] = rest % bx.nb[2];
  bc[3] = rest / bx.nb[2];
  bc[0] = 2 * j + ((bc[1] + bc[2] + bc[3] + colour) & 1);
  return ((bc[3] * bx.nb[2] + bc[2]) * bx.nb[1] + bc[1]) * bx.nb[0] + bc[0];
}

// Site of local index s inside box with box coordinates bc.
__device__ __forceinline__ int box_site(const CGeom& c, const Box4& bx, const int (&bc)[4], int s, int (&lc)[4]) {
  int x[4];
  int q = s;
  for (int mu = 0; mu < 4; ++mu) {
    lc[mu] = q % bx.b[mu];
    q /= bx.b[mu];
    x[mu] = bc[mu] * bx.b[mu] + lc[mu];
  }
  return c_site(c, x);
}

__device__ __forceinline__ int stencil_nb(const CGeom& c, int site, int d) {
  if (d == 0) return site;
  const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
  int stride = 1;
  for (int m = 0; m < mu; ++m) stride *= c.L[m];
  const int x = (site / stride) % c.L[mu];
  return MG_CLAMP(kCoarseNeighbour, site + (((x + step + c.L[mu]) % c.L[mu]) - x) * stride, c.nsites);
}

// The MR step's scalar products and updates with every product and sum rounded
// on its own (no contraction into FMAs), so that the one-RHS and all-RHS forms
// of the coarse Schwarz pass give the same bits whatever the compiler fuses.
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
// (re <p, rho>, im <p, rho>, <p, p>) of one element
template <class R>
__device__ __forceinline__ void mr_dots(const Cplx<R>& p, const Cplx<R>& ro, R (&v)[3]) {
  v[0] = add_rn(mul_rn(p.re, ro.re), mul_rn(p.im, ro.im));
  v[1] = sub_rn(mul_rn(p.re, ro.im), mul_rn(p.im, ro.re));
  v[2] = add_rn(mul_rn(p.re, p.re), mul_rn(p.im, p.im));
}
// e += alpha rho, rho -= alpha p
template <class R>
__device__ __forceinline__ void mr_update(const Cplx<R>& alpha, const Cplx<R>& p, Cplx<R>& e, Cplx<R>& ro) {
  const R ar = sub_rn(mul_rn(alpha.re, ro.re), mul_rn(alpha.im, ro.im));
  const R ai = add_rn(mul_rn(alpha.re, ro.im), mul_rn(alpha.im, ro.re));
  const R pr = sub_rn(mul_rn(alpha.re, p.re), mul_rn(alpha.im, p.im));
  const R pi = add_rn(mul_rn(alpha.re, p.im), mul_rn(alpha.im, p.re));
  e = cmk(add_rn(e.re, ar), add_rn(e.im, ai));
  ro = cmk(sub_rn(ro.re, pr), sub_rn(ro.im, pi));
}

template <class R>
__device__ __forceinline__ void block_reduce_n(R (&v)[3], R (*red)[4]) {
  const int nw = (blockDim.x + 31) >> 5;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < 3; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) { red[w][0] = v[0]; red[w][1] = v[1]; red[w][2] = v[2]; }
  __syncthreads();
  v[0] = v[1] = v[2] = 0;
  for (int k = 0; k < nw; ++k) { v[0] += red[k][0]; v[1] += red[k][1]; v[2] += red[k][2]; }
}

// ------------------------------------------------------------ Schwarz colour pass on a coarse level
// For every box of colour c: r = b - D_c z on the box, n_MR MR steps with the
// box operator (couplings leaving the box dropped), z += e.  Thread (s, i):
// row i of box site s.  rho and e in shared memory [bsites][n2].
template <class R, class TM, class TX>
__global__ void __launch_bounds__(1024) coarse_sap_kernel(const TM* __restrict__ M, TX* __restrict__ z,
                                                          const TX* __restrict__ b, CGeom c, Box4 bx, int colour,
                                                          int n_mr, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n2 = c.n2, bs = bx.sites;
  Cplx<R>* rs = reinterpret_cast<Cplx<R>*>(smem_raw);
  Cplx<R>* es = rs + bs * n2;
  R (*red)[4] = reinterpret_cast<R (*)[4]>(es + bs * n2);
  const int rhs = blockIdx.x % nrhs;
  int bc[4];
  colour_box(bx, blockIdx.x / nrhs, colour, bc);
  const size_t fs = (size_t)c.nsites * n2;
  z += rhs * fs;
  b += rhs * fs;
  const int tid = threadIdx.x;
  const bool act = tid < bs * n2;
  const int s = act ? tid / n2 : 0, i = act ? tid % n2 : 0;
  int lc[4];
  const int site = box_site(c, bx, bc, s, lc);

  // residual
  if (act) {
    Cplx<R> acc = Io<R, TX>::ldc(b + (size_t)site * n2 + i);
    for (int d = 0; d < 9; ++d) {
      const TX* xn = z + (size_t)stencil_nb(c, site, d) * n2;
      const TM* m = M + (((size_t)site * 9 + d) * n2) * n2 + i;
      Cplx<R> t = cmk<R>(0, 0);
      for (int j = 0; j < n2; ++j) cfma(t, Io<R, TM>::ld(m + (size_t)j * n2), Io<R, TX>::ldc(xn + j));
      acc = acc - t;
    }
    rs[tid] = acc;
    es[tid] = cmk<R>(0, 0);
  }
  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();
    Cplx<R> p = cmk<R>(0, 0);
    R v[3] = {0, 0, 0};
    if (act) {
      for (int d = 0; d < 9; ++d) {
        int ln = s;
        if (d > 0) {
          const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
          const int l2 = lc[mu] + step;
          if (l2 < 0 || l2 >= bx.b[mu]) continue;                 // coupling leaves the box
          int stride = 1;
          for (int m = 0; m < mu; ++m) stride *= bx.b[m];
          ln = s + step * stride;
        }
        const TM* m = M + (((size_t)site * 9 + d) * n2) * n2 + i;
        const Cplx<R>* rn = rs + ln * n2;
        for (int j = 0; j < n2; ++j) cfma(p, Io<R, TM>::ld(m + (size_t)j * n2), rn[j]);
      }
      mr_dots(p, rs[tid], v);
    }
    block_reduce_n(v, red);
    Cplx<R> alpha = cmk<R>(0, 0);
    if (v[2] > (R)0) alpha = cmk(v[0] / v[2], v[1] / v[2]);
    if (act) {
      Cplx<R> e = es[tid], ro = rs[tid];
      mr_update(alpha, p, e, ro);
      es[tid] = e;
      rs[tid] = ro;
    }
    __syncthreads();                      // red reused by the next reduction
  }
  if (act) {
    TX* zq = z + (size_t)site * n2 + i;
    Io<R, TX>::st(zq, Io<R, TX>::ldc(zq) + es[tid]);
  }
}

template <class R, class TM, class TX>
static int coarse_sap_t(const CGeom& c, const Box4& bx, const void* M, void* z, const void* b, int colour, int n_mr,
                        int nrhs, cudaStream_t s) {
  const int threads = ((bx.sites * c.n2 + 31) / 32) * 32;
  if (threads > 1024) return MG_ERR_ARG;
  const size_t smem = sizeof(Cplx<R>) * 2 * bx.sites * c.n2 + sizeof(R) * 4 * 32;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(coarse_sap_kernel<R, TM, TX>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    attr = true;
  }
  coarse_sap_kernel<R, TM, TX><<<(unsigned)(bx.nboxes / 2 * nrhs), threads, smem, s>>>(
      (const TM*)M, (TX*)z, (const TX*)b, c, bx, colour, n_mr, nrhs); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// The same colour pass for all right-hand sides in one CTA per box (FP32
// vectors, FP32 or FP16 operator): each operator entry is loaded once for every
// right-hand side, where the one-RHS-per-CTA form above reads the box's
// operator (16 sites x 9 x n2^2 entries) once per right-hand side and MR step
// from memory.  Per right-hand side every sum runs in the order of the kernel
// above (the same residual and MR sums, the same block reduction), so the two
// give the same results bit for bit.  rho and e in shared memory as
// [box site][n2][NR]; NR >= nrhs, an even compile-time bound on the right-hand
// sides.
template <int NR, class TM, int MAXT>
__global__ void __launch_bounds__(MAXT) coarse_sap_mrhs_kernel(const TM* __restrict__ M, float2* __restrict__ z,
                                                               const float2* __restrict__ b, CGeom c, Box4 bx,
                                                               int colour, int n_mr, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n2 = c.n2, bs = bx.sites;
  Cplx<float>* rs = reinterpret_cast<Cplx<float>*>(smem_raw);
  Cplx<float>* es = rs + bs * n2 * NR;
  float (*red)[3 * NR] = reinterpret_cast<float (*)[3 * NR]>(es + bs * n2 * NR);
  int bc[4];
  colour_box(bx, blockIdx.x, colour, bc);
  const size_t fs = (size_t)c.nsites * n2;
  const int tid = threadIdx.x;
  const bool act = tid < bs * n2;
  const int s = act ? tid / n2 : 0, i = act ? tid % n2 : 0;
  int lc[4];
  const int site = box_site(c, bx, bc, s, lc);
  const int nw = (blockDim.x + 31) >> 5, w = tid >> 5, lane = tid & 31;

  // residual of every right-hand side, four at a time (registers)
  if (act) {
#pragma unroll
    for (int r0 = 0; r0 < NR; r0 += 4) {
      Cplx<float> acc[4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
        acc[r] = r0 + r < nrhs ? Io<float, float2>::ldc(b + (r0 + r) * fs + (size_t)site * n2 + i) : cmk(0.f, 0.f);
      for (int d = 0; d < 9; ++d) {
        const size_t xo = (size_t)stencil_nb(c, site, d) * n2;
        const TM* m = M + (((size_t)site * 9 + d) * n2) * n2 + i;
        Cplx<float> t[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) t[r] = cmk(0.f, 0.f);
        for (int j = 0; j < n2; ++j) {
          const Cplx<float> mv = Io<float, TM>::ld(m + (size_t)j * n2);
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (r0 + r < nrhs) cfma(t[r], mv, Io<float, float2>::ldc(z + (r0 + r) * fs + xo + j));
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = acc[r] - t[r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (r0 + r < NR) {
          rs[tid * NR + r0 + r] = acc[r];
          es[tid * NR + r0 + r] = cmk(0.f, 0.f);
        }
    }
  }
  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();
    // p = D_box rho: the right-hand sides in pairs, each FMA the packed two-wide
    // FP32 instruction (lane by lane the cfma of the kernel above: the same
    // products in the same order), the pair's rho read as one 16-byte word
    float2 pre[NR / 2], pim[NR / 2];
#pragma unroll
    for (int q = 0; q < NR / 2; ++q) { pre[q] = make_float2(0.f, 0.f); pim[q] = make_float2(0.f, 0.f); }
    if (act) {
      for (int d = 0; d < 9; ++d) {
        int ln = s;
        if (d > 0) {
          const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
          const int l2 = lc[mu] + step;
          if (l2 < 0 || l2 >= bx.b[mu]) continue;                 // coupling leaves the box
          int stride = 1;
          for (int m = 0; m < mu; ++m) stride *= bx.b[m];
          ln = s + step * stride;
        }
        const TM* m = M + (((size_t)site * 9 + d) * n2) * n2 + i;
        const float4* rn = reinterpret_cast<const float4*>(rs + (size_t)ln * n2 * NR);
        for (int j = 0; j < n2; ++j) {
          const Cplx<float> mv = Io<float, TM>::ld(m + (size_t)j * n2);
          const float2 mr = make_float2(mv.re, mv.re), mi = make_float2(mv.im, mv.im);
          const float2 nmi = make_float2(-mv.im, -mv.im);
#pragma unroll
          for (int q = 0; q < NR / 2; ++q) {
            const float4 x = rn[j * (NR / 2) + q];                // (re_r, im_r, re_r+1, im_r+1)
            const float2 xre = make_float2(x.x, x.z), xim = make_float2(x.y, x.w);
            pre[q] = __ffma2_rn(mr, xre, pre[q]);
            pre[q] = __ffma2_rn(nmi, xim, pre[q]);
            pim[q] = __ffma2_rn(mr, xim, pim[q]);
            pim[q] = __ffma2_rn(mi, xre, pim[q]);
          }
        }
      }
    }
    Cplx<float> p[NR];
#pragma unroll
    for (int q = 0; q < NR / 2; ++q) {
      p[2 * q] = cmk(pre[q].x, pim[q].x);
      p[2 * q + 1] = cmk(pre[q].y, pim[q].y);
    }
    // block sums, per right-hand side as block_reduce_n forms them
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float v[3] = {0.f, 0.f, 0.f};
      if (act) mr_dots(p[r], rs[tid * NR + r], v);
#pragma unroll
      for (int q = 0; q < 3; ++q) v[q] = warp_sum(v[q]);
      if (lane == 0)
#pragma unroll
        for (int q = 0; q < 3; ++q) red[w][3 * r + q] = v[q];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      float a0 = 0, a1 = 0, a2 = 0;
      for (int k = 0; k < nw; ++k) { a0 += red[k][3 * r]; a1 += red[k][3 * r + 1]; a2 += red[k][3 * r + 2]; }
      Cplx<float> alpha = cmk(0.f, 0.f);
      if (a2 > 0.f) alpha = cmk(a0 / a2, a1 / a2);
      if (act) {
        Cplx<float> e = es[tid * NR + r], ro = rs[tid * NR + r];
        mr_update(alpha, p[r], e, ro);
        es[tid * NR + r] = e;
        rs[tid * NR + r] = ro;
      }
    }
    __syncthreads();                      // red reused by the next reduction
  }
  if (act)
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) {
        float2* zq = z + r * fs + (size_t)site * n2 + i;
        Io<float, float2>::st(zq, Io<float, float2>::ldc(zq) + es[tid * NR + r]);
      }
}

// MAXT: the block size the kernel is compiled for (768 leaves 85 registers a
// thread, enough for 12 right-hand sides without spills; 1024 for 2N > 48)
template <int NR, class TM, int MAXT>
static int coarse_sap_mrhs_launch(const CGeom& c, const Box4& bx, const void* M, void* z, const void* b,
                                  int colour, int n_mr, int nrhs, cudaStream_t s, int threads, size_t smem) {
  static bool attr = false;
  if (!attr) {
    SAPMG_CUDA_TRY(cudaFuncSetAttribute(coarse_sap_mrhs_kernel<NR, TM, MAXT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    attr = true;
  }
  coarse_sap_mrhs_kernel<NR, TM, MAXT><<<(unsigned)(bx.nboxes / 2), threads, smem, s>>>(
      (const TM*)M, (float2*)z, (const float2*)b, c, bx, colour, n_mr, nrhs);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

template <int NR, class TM>
static int coarse_sap_mrhs_t(const CGeom& c, const Box4& bx, const void* M, void* z, const void* b, int colour,
                             int n_mr, int nrhs, cudaStream_t s) {
  const int threads = ((bx.sites * c.n2 + 31) / 32) * 32;
  if (threads > 1024 || nrhs > NR) return MG_ERR_ARG;
  const size_t smem = sizeof(Cplx<float>) * 2 * bx.sites * c.n2 * NR + sizeof(float) * 3 * NR * 32;
  if (smem > 227 * 1024) return MG_ERR_ARG;
  return threads <= 768 ? coarse_sap_mrhs_launch<NR, TM, 768>(c, bx, M, z, b, colour, n_mr, nrhs, s, threads, smem)
                        : coarse_sap_mrhs_launch<NR, TM, 1024>(c, bx, M, z, b, colour, n_mr, nrhs, s, threads, smem);
}

template <class TM>
static int coarse_sap_mrhs_any(const CGeom& c, const Box4& bx, const void* M, void* z, const void* b, int colour,
                               int n_mr, int nrhs, cudaStream_t s) {
  if (nrhs <= 2) return coarse_sap_mrhs_t<2, TM>(c, bx, M, z, b, colour, n_mr, nrhs, s);
  if (nrhs <= 4) return coarse_sap_mrhs_t<4, TM>(c, bx, M, z, b, colour, n_mr, nrhs, s);
  if (nrhs <= 8) return coarse_sap_mrhs_t<8, TM>(c, bx, M, z, b, colour, n_mr, nrhs, s);
  if (nrhs <= 12) return coarse_sap_mrhs_t<12, TM>(c, bx, M, z, b, colour, n_mr, nrhs, s);
  return MG_ERR_ARG;
}

int launch_coarse_sap_mrhs(const CGeom& c, const Box4& bx, const void* M, bool m16, void* z, const void* b,
                           int colour, int n_mr, int nrhs, cudaStream_t s) {
  return m16 ? coarse_sap_mrhs_any<__half2>(c, bx, M, z, b, colour, n_mr, nrhs, s)
             : coarse_sap_mrhs_any<float2>(c, bx, M, z, b, colour, n_mr, nrhs, s);
}

int launch_coarse_sap(int prec, const CGeom& c, const Box4& bx, const void* M, void* z, const void* b, int colour,
                      int n_mr, int nrhs, cudaStream_t s, bool m16) {
  if (m16 && prec != P32) return MG_ERR_ARG;
  switch (prec) {
    case P64: return coarse_sap_t<double, double2, double2>(c, bx, M, z, b, colour, n_mr, nrhs, s);
    case P32:
      return m16 ? coarse_sap_t<float, __half2, float2>(c, bx, M, z, b, colour, n_mr, nrhs, s)
                 : coarse_sap_t<float, float2, float2>(c, bx, M, z, b, colour, n_mr, nrhs, s);
    default: return MG_ERR_ARG;
  }
}

// ------------------------------------------------------------ level 1 -> 2 transfers
// restriction: out[A][chi*N1 + k] = sum_{s in A, i in chi} conj(W_k[s][i]) x[s][i]
template <class R, class TX, class TV>
__global__ void __launch_bounds__(1024) restrict1_kernel(const TX* __restrict__ x, TX* __restrict__ out,
                                                         const TV* __restrict__ W, CGeom c, Box4 ag, int N1,
                                                         int nrhs, int nsites2) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R (*red)[4] = reinterpret_cast<R (*)[4]>(smem_raw);               // [nwarps * N1][4]
  const int n2 = c.n2, N0 = n2 / 2;
  const int rhs = blockIdx.x % nrhs, A = MG_CLAMP(kAggregate, blockIdx.x / nrhs, ag.nboxes);
  int bc[4];
  {
    int q = A;
    for (int mu = 0; mu < 4; ++mu) { bc[mu] = q % ag.nb[mu]; q /= ag.nb[mu]; }
  }
  const int tid = threadIdx.x;
  const bool act = tid < ag.sites * n2;
  const int s = act ? tid / n2 : 0, i = act ? tid % n2 : 0;
  int lc[4];
  const int site = box_site(c, ag, bc, s, lc);
  const size_t fs = (size_t)c.nsites * n2;
  const Cplx<R> xv = act ? Io<R, TX>::ldc(x + rhs * fs + (size_t)site * n2 + i) : cmk<R>(0, 0);
  const int chi = i / N0;
  const int w = tid >> 5, lane = tid & 31, nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < N1; ++k) {
    Cplx<R> d = cmk<R>(0, 0);
    if (act) cfma_conj(d, Io<R, TV>::ld(W + (size_t)k * fs + (size_t)site * n2 + i), xv);
    R a0 = chi == 0 ? d.re : (R)0, a1 = chi == 0 ? d.im : (R)0;
    R a2 = chi == 1 ? d.re : (R)0, a3 = chi == 1 ? d.im : (R)0;
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3);
    if (lane == 0) { R* q = red[w * N1 + k]; q[0] = a0; q[1] = a1; q[2] = a2; q[3] = a3; }
  }
  __syncthreads();
  const int m2 = 2 * N1;
  for (int t = tid; t < m2; t += blockDim.x) {
    const int ch = t / N1, k = t % N1;
    R sr = 0, si = 0;
    for (int q = 0; q < nw; ++q) { sr += red[q * N1 + k][2 * ch]; si += red[q * N1 + k][2 * ch + 1]; }
    Io<R, TX>::st(out + (size_t)rhs * nsites2 * m2 + (size_t)A * m2 + t, cmk(sr, si));
  }
}

// interpolation: out[s][i] = sum_k W_k[s][i] e[A(s)][chi(i)*N1 + k]   (overwrites)
template <class R, class TX, class TV>
__global__ void prolong1_kernel(const TX* __restrict__ e, TX* __restrict__ out, const TV* __restrict__ W, CGeom c,
                                Box4 ag, int N1, int nrhs, int nsites2) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n2 = c.n2, N0 = n2 / 2;
  const size_t fs = (size_t)c.nsites * n2;
  if (t >= (long long)fs * nrhs) return;
  const int rhs = (int)(t / fs);
  const size_t rem = (size_t)(t % fs);
  const int site = (int)(rem / n2), i = (int)(rem % n2);
  int A = 0, stride = 1;
  for (int mu = 0; mu < 4; ++mu) {
    A += (c_coord(c, site, mu) / ag.b[mu]) * stride;
    stride *= ag.nb[mu];
  }
  A = MG_CLAMP(kAggregate, A, nsites2);
  const int chi = i / N0;
  const TX* ea = e + (size_t)rhs * nsites2 * 2 * N1 + (size_t)A * 2 * N1 + chi * N1;
  Cplx<R> acc = cmk<R>(0, 0);
  for (int k = 0; k < N1; ++k) cfma(acc, Io<R, TV>::ld(W + (size_t)k * fs + rem), Io<R, TX>::ldc(ea + k));
  Io<R, TX>::st(out + t, acc);
}

template <class R, class TX, class TV>
static int transfer1_t(bool restrict_, const CGeom& c, const Box4& ag, const void* in, void* out, const void* W,
                       int N1, int nrhs, cudaStream_t s) {
  const int nsites2 = ag.nboxes;
  if (restrict_) {
    const int threads = ((ag.sites * c.n2 + 31) / 32) * 32;
    if (threads > 1024) return MG_ERR_ARG;
    const size_t smem = sizeof(R) * 4 * (threads / 32) * N1;
    restrict1_kernel<R, TX, TV><<<(unsigned)(ag.nboxes * nrhs), threads, smem, s>>>(
        (const TX*)in, (TX*)out, (const TV*)W, c, ag, N1, nrhs, nsites2); count_launches(1);
  } else {
    const long long n = (long long)c.nsites * c.n2 * nrhs;
    prolong1_kernel<R, TX, TV><<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const TX*)in, (TX*)out, (const TV*)W, c,
                                                                         ag, N1, nrhs, nsites2); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_transfer1(bool restrict_, int prec, const CGeom& c, const Box4& ag, const void* in, void* out,
                     const void* W, int N1, int nrhs, cudaStream_t s) {
  switch (prec) {
    case P64: return transfer1_t<double, double2, double2>(restrict_, c, ag, in, out, W, N1, nrhs, s);
    case P32: return transfer1_t<float, float2, float2>(restrict_, c, ag, in, out, W, N1, nrhs, s);
    default: return MG_ERR_ARG;
  }
}

// ------------------------------------------------------------ level-1 local orthonormalisation (FP64)
// Modified Gram-Schmidt of W_0..W_{N1-1} on every (aggregate, chirality), in order.
__global__ void __launch_bounds__(1024) block_gs1_kernel(double2* __restrict__ W, CGeom c, Box4 ag, int N1) {
  __shared__ double red[32][2];
  const int A = MG_CLAMP(kAggregate, blockIdx.x, ag.nboxes), chi = blockIdx.y;
  const int n2 = c.n2, N0 = n2 / 2;
  int bc[4];
  {
    int q = A;
    for (int mu = 0; mu < 4; ++mu) { bc[mu] = q % ag.nb[mu]; q /= ag.nb[mu]; }
  }
  const int tid = threadIdx.x;
  const bool act = tid < ag.sites * N0;
  const int s = act ? tid / N0 : 0, h = act ? tid % N0 : 0;
  int lc[4];
  const int site = box_site(c, ag, bc, s, lc);
  const size_t fs = (size_t)c.nsites * n2;
  const size_t off = (size_t)site * n2 + chi * N0 + h;
  const int nw = (blockDim.x + 31) >> 5, w = tid >> 5, lane = tid & 31;
  auto bsum = [&](double a, double b2) {
    a = warp_sum(a);
    b2 = warp_sum(b2);
    if (lane == 0) { red[w][0] = a; red[w][1] = b2; }
    __syncthreads();
    double sa = 0, sb = 0;
    for (int q = 0; q < nw; ++q) { sa += red[q][0]; sb += red[q][1]; }
    __syncthreads();
    return make_double2(sa, sb);
  };
  for (int k = 0; k < N1; ++k) {
    Cplx<double> xk = cmk(0.0, 0.0);
    if (act) { const double2 t = W[k * fs + off]; xk = cmk(t.x, t.y); }
    for (int j = 0; j < k; ++j) {
      Cplx<double> qj = cmk(0.0, 0.0), d = cmk(0.0, 0.0);
      if (act) { const double2 t = W[j * fs + off]; qj = cmk(t.x, t.y); cfma_conj(d, qj, xk); }
      const double2 sum = bsum(d.re, d.im);
      xk = xk - cmk(sum.x, sum.y) * qj;
    }
    const double2 nn = bsum(xk.re * xk.re + xk.im * xk.im, 0.0);
    const double inv = nn.x > 0 ? 1.0 / sqrt(nn.x) : 0.0;
    if (act) W[k * fs + off] = make_double2(xk.re * inv, xk.im * inv);
  }
}

int launch_block_gs1(const CGeom& c, const Box4& ag, void* W64, int N1, cudaStream_t s) {
  const int threads = ((ag.sites * (c.n2 / 2) + 31) / 32) * 32;
  if (threads > 1024) return MG_ERR_ARG;
  dim3 grid(ag.nboxes, 2);
  block_gs1_kernel<<<grid, threads, 0, s>>>((double2*)W64, c, ag, N1); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// ------------------------------------------------------------ Galerkin assembly D_c2 = P1^dagger D_c1 P1 (FP64)
// CTA (A, j), column j = (chi', k): u = W_k restricted to chirality chi'.  Thread
// (s, i) forms row i at site s of each of the 9 partial images (self: the
// couplings that stay inside A; +-mu: the coupling from the neighbouring
// aggregate across A's face) and the projections onto W_k'|chi on A are summed.
__global__ void __launch_bounds__(1024) assemble1_kernel(const double2* __restrict__ W,
                                                         const double2* __restrict__ M1,
                                                         double2* __restrict__ M2, CGeom c, CGeom c2, Box4 ag,
                                                         int N1) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double (*red)[4] = reinterpret_cast<double (*)[4]>(smem_raw);     // [nwarps * N1][4]
  const int A = MG_CLAMP(kAggregate, blockIdx.x, ag.nboxes), j = blockIdx.y;
  const int n2 = c.n2, N0 = n2 / 2, m2 = 2 * N1;
  const int chi_p = j / N1, k = j % N1;
  int bc[4];
  {
    int q = A;
    for (int mu = 0; mu < 4; ++mu) { bc[mu] = q % ag.nb[mu]; q /= ag.nb[mu]; }
  }
  const int tid = threadIdx.x;
  const bool act = tid < ag.sites * n2;
  const int s = act ? tid / n2 : 0, i = act ? tid % n2 : 0;
  int lc[4];
  const int site = box_site(c, ag, bc, s, lc);
  const size_t fs = (size_t)c.nsites * n2;
  const int nw = (blockDim.x + 31) >> 5, w = tid >> 5, lane = tid & 31;
  for (int dout = 0; dout < 9; ++dout) {
    Cplx<double> acc = cmk(0.0, 0.0);
    if (act) {
      for (int d = 0; d < 9; ++d) {
        bool inside = true;
        if (d > 0) {
          const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
          const int l2 = lc[mu] + step;
          inside = (l2 >= 0 && l2 < ag.b[mu]);
        }
        if (dout == 0 ? !inside : (d != dout || inside)) continue;
        const int nb = stencil_nb(c, site, d);
        const double2* m = M1 + (((size_t)site * 9 + d) * n2) * n2 + i;
        const double2* u = W + (size_t)k * fs + (size_t)nb * n2 + chi_p * N0;
        for (int jj = 0; jj < N0; ++jj) {
          const double2 mv = m[(size_t)(chi_p * N0 + jj) * n2], uv = u[jj];
          cfma(acc, cmk(mv.x, mv.y), cmk(uv.x, uv.y));
        }
      }
    }
    const int chi = i / N0;
    for (int kk = 0; kk < N1; ++kk) {
      Cplx<double> d = cmk(0.0, 0.0);
      if (act) {
        const double2 wv = W[(size_t)kk * fs + (size_t)site * n2 + i];
        cfma_conj(d, cmk(wv.x, wv.y), acc);
      }
      double a0 = chi == 0 ? d.re : 0.0, a1 = chi == 0 ? d.im : 0.0;
      double a2 = chi == 1 ? d.re : 0.0, a3 = chi == 1 ? d.im : 0.0;
      a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2); a3 = warp_sum(a3);
      if (lane == 0) { double* q = red[w * N1 + kk]; q[0] = a0; q[1] = a1; q[2] = a2; q[3] = a3; }
    }
    __syncthreads();
    double2* col = M2 + (((size_t)A * 9 + dout) * m2 + j) * m2;
    for (int t = tid; t < m2; t += blockDim.x) {
      const int ch = t / N1, kk = t % N1;
      double sr = 0, si = 0;
      for (int q = 0; q < nw; ++q) { sr += red[q * N1 + kk][2 * ch]; si += red[q * N1 + kk][2 * ch + 1]; }
      col[t] = make_double2(sr, si);
    }
    __syncthreads();
  }
}

int launch_assemble1(const CGeom& c, const CGeom& c2, const Box4& ag, const void* W64, const void* M1_64, void* M2_64,
                     int N1, cudaStream_t s) {
  const int threads = ((ag.sites * c.n2 + 31) / 32) * 32;
  if (threads > 1024) return MG_ERR_ARG;
  const size_t smem = sizeof(double) * 4 * (threads / 32) * N1;
  dim3 grid(ag.nboxes, 2 * N1);
  assemble1_kernel<<<grid, threads, smem, s>>>((const double2*)W64, (const double2*)M1_64, (double2*)M2_64, c, c2, ag,
                                               N1); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
