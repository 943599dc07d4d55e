// Vector and scalar kernels of CG on the normal equations D^dagger D x =
// D^dagger b (CGN), the method the paper's solver is compared with (Sec. 4,
// Tables 1-2).  R systems run together; every per-system scalar lives on the
// device (CgnState), so an iteration needs no host round trip: the kernels
// read alpha, beta and the active flag of their system from there.
//
// Partial sums: a vector kernel with G CTAs per system writes one double per
// CTA at part[r * G + cta]; the Dirac kernel's norm epilogue writes
// part[block * R + r].  The scalar kernels add them up in a fixed order.
#include <algorithm>

#include "internal.h"

namespace sapmg {

namespace {

template <class T> struct CgVec;
template <> struct CgVec<float> { using V = float4; static constexpr int per = 2; };   // two complex per load
template <> struct CgVec<double> { using V = double2; static constexpr int per = 1; };

__device__ __forceinline__ float4 axpy(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ double2 axpy(double a, double2 x, double2 y) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}
__device__ __forceinline__ float nrm(float4 v) { return v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w; }
__device__ __forceinline__ double nrm(double2 v) { return v.x * v.x + v.y * v.y; }

// The CTA's sum of t (one value per thread, 256 threads) to part[slot].
template <class A>
__device__ __forceinline__ void cta_partial(A t, double* part, size_t slot) {
  __shared__ double ws[8];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = (double)t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0;
    for (int w = 0; w < 8; ++w) sum += ws[w];
    part[slot] = sum;
  }
}

// Fixed-order sum of count values p[k * stride] by one 256-thread CTA.
__device__ double cta_sum(const double* __restrict__ p, int count, int stride) {
  __shared__ double sh[256];
  double t = 0;
  for (int k = threadIdx.x; k < count; k += 256) t += p[(size_t)k * stride];
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double res = sh[0];
  __syncthreads();
  return res;
}

// r = b - t (FP64 in, stored as T), part = ||b - t||^2 in FP64.
template <class T>
__global__ void __launch_bounds__(256) cgn_residual_kernel(const double2* __restrict__ b, const double2* __restrict__ t,
                                                           T* __restrict__ r, size_t n, double* __restrict__ part, int G) {
  const int sys = blockIdx.y;
  b += (size_t)sys * n;
  t += (size_t)sys * n;
  r += (size_t)sys * n * 2;
  double acc = 0;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)G * 256) {
    const double2 bv = b[i], tv = t[i];
    const double2 d = make_double2(bv.x - tv.x, bv.y - tv.y);
    r[2 * i] = (T)d.x;
    r[2 * i + 1] = (T)d.y;
    acc += d.x * d.x + d.y * d.y;
  }
  cta_partial(acc, part, (size_t)sys * G + blockIdx.x);
}

// x += alpha p, r -= alpha q for the active systems; part = ||r_new||^2.
template <class T>
__global__ void __launch_bounds__(256) cgn_xr_kernel(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ p,
                                                     const T* __restrict__ q, size_t nv, const CgnState* __restrict__ st,
                                                     double* __restrict__ part, int G) {
  using V = typename CgVec<T>::V;
  const int sys = blockIdx.y;
  if (!st[sys].act) return;   // the scalar kernels read part only for active systems
  const T a = (T)st[sys].alpha;
  V* xv = (V*)x + (size_t)sys * nv;
  V* rv = (V*)r + (size_t)sys * nv;
  const V* pv = (const V*)p + (size_t)sys * nv;
  const V* qv = (const V*)q + (size_t)sys * nv;
  T acc = 0;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < nv; i += (size_t)G * 256) {
    xv[i] = axpy(a, pv[i], xv[i]);
    const V rn = axpy(-a, qv[i], rv[i]);
    rv[i] = rn;
    acc += nrm(rn);
  }
  cta_partial(acc, part, (size_t)sys * G + blockIdx.x);
}

// p = s + beta p for the active systems (p = s for every system when init,
// without reading p).
template <class T>
__global__ void __launch_bounds__(256) cgn_p_kernel(T* __restrict__ p, const T* __restrict__ s, size_t nv,
                                                    const CgnState* __restrict__ st, int init, int G) {
  using V = typename CgVec<T>::V;
  const int sys = blockIdx.y;
  if (!init && !st[sys].act) return;
  const T beta = init ? (T)0 : (T)st[sys].beta;
  V* pv = (V*)p + (size_t)sys * nv;
  const V* sv = (const V*)s + (size_t)sys * nv;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < nv; i += (size_t)G * 256)
    pv[i] = beta == (T)0 ? sv[i] : axpy(beta, pv[i], sv[i]);
}

// x64 += x32, x32 = 0 (the FP64 update of the mixed form).
__global__ void __launch_bounds__(256) cgn_accum_kernel(double2* __restrict__ x64, float2* __restrict__ x32, size_t n,
                                                        int G) {
  const int sys = blockIdx.y;
  x64 += (size_t)sys * n;
  x32 += (size_t)sys * n;
  for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (size_t)G * 256) {
    const float2 e = x32[i];
    double2 v = x64[i];
    v.x += (double)e.x;
    v.y += (double)e.y;
    x64[i] = v;
    x32[i] = make_float2(0.f, 0.f);
  }
}

// gam = ||s||^2 (Dirac norm partials); init: also rr = ||r||^2, the stopping
// threshold tol^2 ||b||^2 (r = b at the start) and a zero iteration count.
__global__ void __launch_bounds__(256) cgn_gamma_kernel(const double* __restrict__ part_s, int nb,
                                                        const double* __restrict__ part_r, int G, int R,
                                                        CgnState* __restrict__ st, double tol2, int init) {
  const int sys = blockIdx.x;
  const double ss = cta_sum(part_s + sys, nb, R);
  const double rr = init ? cta_sum(part_r + (size_t)sys * G, G, 1) : 0.0;
  if (threadIdx.x == 0) {
    CgnState& q = st[sys];
    q.gam = ss;
    q.beta = 0;
    if (init) {
      q.rr = rr;
      q.thr = tol2 * rr;
      q.alpha = 0;
      q.act = 0;
      q.its = 0;
    }
  }
}

// Start of an iteration: qq = ||D p||^2; a system is active while its residual
// is above the threshold and it has iterations left; alpha = gam / qq.
__global__ void __launch_bounds__(256) cgn_alpha_kernel(const double* __restrict__ part_q, int nb, int R,
                                                        CgnState* __restrict__ st, int maxiter) {
  const int sys = blockIdx.x;
  const double qq = cta_sum(part_q + sys, nb, R);
  if (threadIdx.x == 0) {
    CgnState& q = st[sys];
    const int act = q.rr > q.thr && q.its < maxiter && qq > 0 && isfinite(qq) && isfinite(q.gam);
    q.act = act;
    q.alpha = act ? q.gam / qq : 0.0;
    q.its += act;
  }
}

// End of an iteration: rr = ||r_new||^2, beta = ||s_new||^2 / gam, gam = ||s_new||^2.
__global__ void __launch_bounds__(256) cgn_beta_kernel(const double* __restrict__ part_s, int nb,
                                                       const double* __restrict__ part_r, int G, int R,
                                                       CgnState* __restrict__ st) {
  const int sys = blockIdx.x;
  if (!st[sys].act) return;
  const double ss = cta_sum(part_s + sys, nb, R);
  const double rr = cta_sum(part_r + (size_t)sys * G, G, 1);
  if (threadIdx.x == 0) {
    CgnState& q = st[sys];
    q.rr = rr;
    q.beta = q.gam > 0 ? ss / q.gam : 0.0;
    q.gam = ss;
  }
}

// rr = ||r||^2 for every system (after r was replaced by the true residual).
__global__ void __launch_bounds__(256) cgn_rr_kernel(const double* __restrict__ part_r, int G,
                                                     CgnState* __restrict__ st) {
  const int sys = blockIdx.x;
  const double rr = cta_sum(part_r + (size_t)sys * G, G, 1);
  if (threadIdx.x == 0) st[sys].rr = rr;
}

}  // namespace

int cgn_grid(size_t n) {
  const size_t g = (n + 1023) / 1024;
  return (int)std::min<size_t>(std::max<size_t>(g, 1), kCgnMaxG);
}

int launch_cgn_residual(int type, const void* b64, const void* t64, void* r, size_t n, int R, double* part, int G,
                        cudaStream_t s) {
  const dim3 grid(G, R);
  if (type == P64)
    cgn_residual_kernel<double><<<grid, 256, 0, s>>>((const double2*)b64, (const double2*)t64, (double*)r, n, part, G);
  else if (type == P32)
    cgn_residual_kernel<float><<<grid, 256, 0, s>>>((const double2*)b64, (const double2*)t64, (float*)r, n, part, G);
  else
    return MG_ERR_ARG;
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_xr(int type, void* x, void* r, const void* p, const void* q, size_t n, int R, const CgnState* st,
                  double* part, int G, cudaStream_t s) {
  const dim3 grid(G, R);
  if (type == P64)
    cgn_xr_kernel<double><<<grid, 256, 0, s>>>((double*)x, (double*)r, (const double*)p, (const double*)q, n, st,
                                                part, G);
  else if (type == P32)
    cgn_xr_kernel<float><<<grid, 256, 0, s>>>((float*)x, (float*)r, (const float*)p, (const float*)q, n / 2, st,
                                               part, G);
  else
    return MG_ERR_ARG;
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_p(int type, void* p, const void* sv, size_t n, int R, const CgnState* st, bool init, int G,
                 cudaStream_t s) {
  const dim3 grid(G, R);
  if (type == P64)
    cgn_p_kernel<double><<<grid, 256, 0, s>>>((double*)p, (const double*)sv, n, st, init ? 1 : 0, G);
  else if (type == P32)
    cgn_p_kernel<float><<<grid, 256, 0, s>>>((float*)p, (const float*)sv, n / 2, st, init ? 1 : 0, G);
  else
    return MG_ERR_ARG;
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_accum(void* x64, void* x32, size_t n, int R, int G, cudaStream_t s) {
  cgn_accum_kernel<<<dim3(G, R), 256, 0, s>>>((double2*)x64, (float2*)x32, n, G);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_gamma(const double* part_s, int nb, const double* part_r, int G, int R, CgnState* st, double tol2,
                     bool init, cudaStream_t s) {
  cgn_gamma_kernel<<<R, 256, 0, s>>>(part_s, nb, part_r, G, R, st, tol2, init ? 1 : 0);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_alpha(const double* part_q, int nb, int R, CgnState* st, int maxiter, cudaStream_t s) {
  cgn_alpha_kernel<<<R, 256, 0, s>>>(part_q, nb, R, st, maxiter);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_beta(const double* part_s, int nb, const double* part_r, int G, int R, CgnState* st, cudaStream_t s) {
  cgn_beta_kernel<<<R, 256, 0, s>>>(part_s, nb, part_r, G, R, st);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_cgn_rr(const double* part_r, int G, int R, CgnState* st, cudaStream_t s) {
  cgn_rr_kernel<<<R, 256, 0, s>>>(part_r, G, st);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
