// K8: vector kernels of the Krylov solvers (Sec. 2 and Sec. 4: GMRES on the
// coarse grid, flexible GMRES outside), batched over right-hand sides: one
// launch serves all R systems, each with its own vectors and scalars.
//
// A batched vector is R fields stored back to back (field r at base + r*stride).
// Reductions are deterministic: every CTA writes its partial sums, one CTA per
// right-hand side adds them in a fixed order.  Per-thread and per-warp partial
// sums use the vector's own precision; CTA-level and final sums use FP64.
#include "internal.h"
#include "blas.h"

#include <type_traits>

namespace sapmg {

template <class T2> struct RealOf;
template <> struct RealOf<double2> { typedef double R; };
template <> struct RealOf<float2> { typedef float R; };

// up to 16 vectors per launch
constexpr int kChunk = 16;
template <class T2> struct Ptrs8 { const T2* p[kChunk]; };

// CTAs per right-hand side of a reduction: at least 8 elements per thread, and
// R * CTAs within the partial buffer.
static int reduce_ctas(size_t n, int R) {
  const size_t per = std::max<size_t>(1, (size_t)kMaxReduceCta / (size_t)std::max(R, 1));
  return (int)std::max<size_t>(1, std::min<size_t>((n + 2047) / 2048, per));
}

template <class T2, int K>
__global__ void __launch_bounds__(256) multidot_partial(Ptrs8<T2> v, const T2* __restrict__ w, size_t n,
                                                        size_t vstride, size_t wstride,
                                                        double2* __restrict__ partial) {
  typedef typename RealOf<T2>::R R;
  const int r = blockIdx.y;
  const T2* wr = w + r * wstride;
  R are[K], aim[K];
#pragma unroll
  for (int j = 0; j < K; ++j) are[j] = aim[j] = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    // issue every load of the element before any arithmetic (memory-level parallelism)
    T2 a[K];
#pragma unroll
    for (int j = 0; j < K; ++j) a[j] = __ldg(&v.p[j][r * vstride + i]);
    const T2 x = __ldg(&wr[i]);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      are[j] = fma(a[j].x, x.x, fma(a[j].y, x.y, are[j]));
      aim[j] = fma(a[j].x, x.y, fma(-a[j].y, x.x, aim[j]));
    }
  }
  __shared__ double red[8][2 * K];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // warp trees in the vector's precision (FP64 arithmetic is scarce), CTA sum in FP64
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const R s = warp_sum(are[j]);
    const R m = warp_sum(aim[j]);
    if (lane == 0) { red[wid][2 * j] = (double)s; red[wid][2 * j + 1] = (double)m; }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0, m = 0;
    for (int q = 0; q < 8; ++q) { s += red[q][2 * threadIdx.x]; m += red[q][2 * threadIdx.x + 1]; }
    partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk + threadIdx.x] = make_double2(s, m);
  }
}

// FP32 vectors with an even length: two complex numbers per 16-byte load.
template <int K>
__global__ void __launch_bounds__(256) multidot_partial_f4(Ptrs8<float2> v, const float2* __restrict__ w, size_t n,
                                                           size_t vstride, size_t wstride,
                                                           double2* __restrict__ partial) {
  const int r = blockIdx.y;
  const float4* wr = reinterpret_cast<const float4*>(w + r * wstride);
  const size_t n4 = n / 2;
  float are[K], aim[K];
#pragma unroll
  for (int j = 0; j < K; ++j) are[j] = aim[j] = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (size_t)gridDim.x * blockDim.x) {
    float4 a[K];
#pragma unroll
    for (int j = 0; j < K; ++j) a[j] = __ldg(reinterpret_cast<const float4*>(v.p[j] + r * vstride) + i);
    const float4 x = __ldg(wr + i);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      are[j] = fmaf(a[j].x, x.x, fmaf(a[j].y, x.y, fmaf(a[j].z, x.z, fmaf(a[j].w, x.w, are[j]))));
      aim[j] = fmaf(a[j].x, x.y, fmaf(-a[j].y, x.x, fmaf(a[j].z, x.w, fmaf(-a[j].w, x.z, aim[j]))));
    }
  }
  __shared__ double red[8][2 * K];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float s = warp_sum(are[j]);
    const float m = warp_sum(aim[j]);
    if (lane == 0) { red[wid][2 * j] = (double)s; red[wid][2 * j + 1] = (double)m; }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double s = 0, m = 0;
    for (int q = 0; q < 8; ++q) { s += red[q][2 * threadIdx.x]; m += red[q][2 * threadIdx.x + 1]; }
    partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk + threadIdx.x] = make_double2(s, m);
  }
}

// out[r*ldo + j] = (mode 1: out +) sum over CTAs; out2[r*ldo + j] = the sum if out2 != nullptr.
__global__ void multidot_finalize(const double2* __restrict__ partial, int ncta, int k, double2* out, int ldo,
                                  int mode, double2* out2) {
  __shared__ double red[8][2];
  const int r = blockIdx.x;
  for (int j = 0; j < k; ++j) {
    double s = 0, m = 0;
    for (int c = threadIdx.x; c < ncta; c += blockDim.x) {
      const double2 v = partial[((size_t)r * ncta + c) * kChunk + j];
      s += v.x;
      m += v.y;
    }
    s = warp_sum(s);
    m = warp_sum(m);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[wid][0] = s; red[wid][1] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ss = 0, sm = 0;
      for (int q = 0; q < 8; ++q) { ss += red[q][0]; sm += red[q][1]; }
      if (out) {
        double2* o = out + (size_t)r * ldo + j;
        if (mode == 1) { o->x += ss; o->y += sm; }
        else *o = make_double2(ss, sm);
      }
      if (out2) out2[(size_t)r * ldo + j] = make_double2(ss, sm);
    }
    __syncthreads();
  }
}

template <class T2, int K>
static void md_launch(dim3 grid, const Ptrs8<T2>& p, const T2* w, size_t n, size_t vs, size_t ws, double2* part,
                      cudaStream_t s) {
  multidot_partial<T2, K><<<grid, 256, 0, s>>>(p, w, n, vs, ws, part); count_launches(1);
}

template <class T2, int K>
static void md_launch_any(bool vec4, dim3 grid, const Ptrs8<T2>& p, const T2* w, size_t n, size_t vs, size_t ws,
                          double2* part, cudaStream_t s) {
  if constexpr (std::is_same<T2, float2>::value) {
    if (vec4) {
      multidot_partial_f4<K><<<grid, 256, 0, s>>>(p, w, n, vs, ws, part); count_launches(1);
      return;
    }
  }
  md_launch<T2, K>(grid, p, w, n, vs, ws, part, s);
}

template <class T2>
static int multidot_t(const BVec& b, const void* const* v, int k, const void* w, double2* out, int ldo, int mode,
                      double2* out2, double2* partial, cudaStream_t s) {
  // two complex numbers per load when every vector is 16-byte aligned and n is even
  bool vec4 = (b.n % 2 == 0) && (b.vstride % 2 == 0) && (b.wstride % 2 == 0) &&
              ((reinterpret_cast<uintptr_t>(w) & 15) == 0);
  for (int j = 0; j < k; ++j) vec4 = vec4 && ((reinterpret_cast<uintptr_t>(v[j]) & 15) == 0);
  const int ncta = reduce_ctas(vec4 ? b.n / 2 : b.n, b.R);
  const dim3 grid(ncta, b.R);
  for (int j0 = 0; j0 < k; j0 += kChunk) {
    const int kk = std::min(kChunk, k - j0);
    Ptrs8<T2> p;
    for (int j = 0; j < kChunk; ++j) p.p[j] = (const T2*)v[j0 + std::min(j, kk - 1)];
    const T2* wp = (const T2*)w;
#define SAPMG_MD(K) case K: md_launch_any<T2, K>(vec4, grid, p, wp, b.n, b.vstride, b.wstride, partial, s); break;
    switch (kk) {
      SAPMG_MD(1) SAPMG_MD(2) SAPMG_MD(3) SAPMG_MD(4) SAPMG_MD(5) SAPMG_MD(6) SAPMG_MD(7) SAPMG_MD(8)
      SAPMG_MD(9) SAPMG_MD(10) SAPMG_MD(11) SAPMG_MD(12) SAPMG_MD(13) SAPMG_MD(14) SAPMG_MD(15)
      default: md_launch_any<T2, 16>(vec4, grid, p, wp, b.n, b.vstride, b.wstride, partial, s); break;
    }
#undef SAPMG_MD
    multidot_finalize<<<b.R, 256, 0, s>>>(partial, ncta, kk, out ? out + j0 : nullptr, ldo, mode,
                                          out2 ? out2 + j0 : nullptr); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_multidot(int type, const BVec& b, const void* const* v, int k, const void* w, double2* out, int ldo,
                  int mode, double2* out2, double2* partial, cudaStream_t s) {
  if (k <= 0 || b.R <= 0) return MG_OK;
  count_bytes((double)(k + (v[k - 1] == w ? 0 : 1)) * b.n * b.R * (type == P64 ? 16 : 8));
  if (type == P64) return multidot_t<double2>(b, v, k, w, out, ldo, mode, out2, partial, s);
  if (type == P32) return multidot_t<float2>(b, v, k, w, out, ldo, mode, out2, partial, s);
  return MG_ERR_ARG;
}

// w[r] += sign * sum_j coeff[r*ldc + j] v_j[r]; with partial != nullptr the
// CTA also writes its part of ||w_new||^2 (finished by multidot_finalize).
template <class T2, int K>
__global__ void __launch_bounds__(256) multiaxpy_kernel(T2* __restrict__ w, Ptrs8<T2> v,
                                                        const double2* __restrict__ coeff, int ldc, double sign,
                                                        size_t n, size_t vstride, size_t wstride,
                                                        double2* __restrict__ partial) {
  typedef typename RealOf<T2>::R R;
  const int r = blockIdx.y;
  R cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const double2 c = coeff[(size_t)r * ldc + j];
    cr[j] = (R)(sign * c.x);
    ci[j] = (R)(sign * c.y);
  }
  T2* wr = w + r * wstride;
  R nn = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T2 x = wr[i];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const T2 a = v.p[j][r * vstride + i];
      x.x = fma(cr[j], a.x, fma(-ci[j], a.y, x.x));
      x.y = fma(cr[j], a.y, fma(ci[j], a.x, x.y));
    }
    wr[i] = x;
    nn = fma(x.x, x.x, fma(x.y, x.y, nn));
  }
  if (partial) {
    __shared__ double red[8];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R t = warp_sum(nn);
    if (lane == 0) red[wid] = (double)t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0;
      for (int q = 0; q < 8; ++q) sum += red[q];
      partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk] = make_double2(sum, 0.0);
    }
  }
}

// Streaming kernels: about 8 CTAs of 256 threads per SM over all right-hand sides.
static dim3 stream_grid(size_t n, int R) {
  const size_t per = std::max<size_t>(16, (size_t)152 * 8 / (size_t)std::max(R, 1));
  return dim3((unsigned)std::max<size_t>(1, std::min<size_t>((n + 1023) / 1024, per)), R);
}

template <class T2, int K>
static void ma_launch(dim3 g, T2* w, const Ptrs8<T2>& p, const double2* c, int ldc, double sign, const BVec& b,
                      double2* partial, cudaStream_t s) {
  multiaxpy_kernel<T2, K><<<g, 256, 0, s>>>(w, p, c, ldc, sign, b.n, b.vstride, b.wstride, partial); count_launches(1);
}

template <class T2>
static int multiaxpy_t(const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc,
                       double sign, double2* nrm2, int ldn, double2* partial, cudaStream_t s) {
  const dim3 g = nrm2 ? dim3(reduce_ctas(b.n, b.R), b.R) : stream_grid(b.n, b.R);
  for (int j0 = 0; j0 < k; j0 += kChunk) {
    const int kk = std::min(kChunk, k - j0);
    const bool last = j0 + kChunk >= k;
    Ptrs8<T2> p;
    for (int j = 0; j < kChunk; ++j) p.p[j] = (const T2*)v[j0 + std::min(j, kk - 1)];
    const double2* c = coeff + j0;
    double2* part = (last && nrm2) ? partial : nullptr;
#define SAPMG_MA(K) case K: ma_launch<T2, K>(g, (T2*)w, p, c, ldc, sign, b, part, s); break;
    switch (kk) {
      SAPMG_MA(1) SAPMG_MA(2) SAPMG_MA(3) SAPMG_MA(4) SAPMG_MA(5) SAPMG_MA(6) SAPMG_MA(7) SAPMG_MA(8)
      SAPMG_MA(9) SAPMG_MA(10) SAPMG_MA(11) SAPMG_MA(12) SAPMG_MA(13) SAPMG_MA(14) SAPMG_MA(15)
      default: ma_launch<T2, 16>(g, (T2*)w, p, c, ldc, sign, b, part, s); break;
    }
#undef SAPMG_MA
  }
  if (nrm2) {
    multidot_finalize<<<b.R, 256, 0, s>>>(partial, (int)g.x, 1, nrm2, ldn, 0, nullptr); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_multiaxpy(int type, const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc,
                   double sign, cudaStream_t s) {
  if (k <= 0 || b.R <= 0) return MG_OK;
  count_bytes((double)(k + 2) * b.n * b.R * (type == P64 ? 16 : 8));
  if (type == P64) return multiaxpy_t<double2>(b, w, v, k, coeff, ldc, sign, nullptr, 0, nullptr, s);
  if (type == P32) return multiaxpy_t<float2>(b, w, v, k, coeff, ldc, sign, nullptr, 0, nullptr, s);
  return MG_ERR_ARG;
}

int blas_multiaxpy_norm(int type, const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc,
                        double sign, double2* nrm2, int ldn, double2* partial, cudaStream_t s) {
  if (k <= 0 || b.R <= 0) return MG_OK;
  count_bytes((double)(k + 2) * b.n * b.R * (type == P64 ? 16 : 8));
  if (type == P64) return multiaxpy_t<double2>(b, w, v, k, coeff, ldc, sign, nrm2, ldn, partial, s);
  if (type == P32) return multiaxpy_t<float2>(b, w, v, k, coeff, ldc, sign, nrm2, ldn, partial, s);
  return MG_ERR_ARG;
}

// y[r] = a_r x[r] + b_r y[r] with per-RHS scalars passed by value; x and y may
// differ in element type; b_r = 0 means y[r] is not read.
template <class TX, class TY>
__global__ void axpby_kernel(Scal32 a, const TX* __restrict__ x, Scal32 b, TY* __restrict__ y, size_t n,
                             size_t xs, size_t ys) {
  typedef typename RealOf<TY>::R R;
  const int r = blockIdx.y;
  const R ar = (R)a.v[r].x, ai = (R)a.v[r].y, br = (R)b.v[r].x, bi = (R)b.v[r].y;
  const bool yz = (b.v[r].x == 0.0 && b.v[r].y == 0.0);
  const TX* xr = x + r * xs;
  TY* yr = y + r * ys;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const TX u = xr[i];
    const R ux = (R)u.x, uy = (R)u.y;
    TY o;
    if (yz) {
      o.x = ar * ux - ai * uy;
      o.y = ar * uy + ai * ux;
    } else {
      const TY v = yr[i];
      o.x = ar * ux - ai * uy + br * v.x - bi * v.y;
      o.y = ar * uy + ai * ux + br * v.y + bi * v.x;
    }
    yr[i] = o;
  }
}

int blas_axpby2(int tx, const Scal32& a, const void* x, size_t xs, int ty, const Scal32& b, void* y, size_t ys,
                size_t n, int R, cudaStream_t s) {
  if (n == 0 || R == 0) return MG_OK;
  if (R > 32) return MG_ERR_ARG;
  bool yread = false;
  for (int r = 0; r < R; ++r) yread = yread || b.v[r].x != 0.0 || b.v[r].y != 0.0;
  count_bytes((double)n * R * ((tx == P64 ? 16 : 8) + (ty == P64 ? 16 : 8) * (yread ? 2 : 1)));
  const dim3 g = stream_grid(n, R);
  if (tx == P64 && ty == P64) { axpby_kernel<double2, double2><<<g, 256, 0, s>>>(a, (const double2*)x, b, (double2*)y, n, xs, ys); count_launches(1); }
  else if (tx == P32 && ty == P32) { axpby_kernel<float2, float2><<<g, 256, 0, s>>>(a, (const float2*)x, b, (float2*)y, n, xs, ys); count_launches(1); }
  else if (tx == P32 && ty == P64) { axpby_kernel<float2, double2><<<g, 256, 0, s>>>(a, (const float2*)x, b, (double2*)y, n, xs, ys); count_launches(1); }
  else if (tx == P64 && ty == P32) { axpby_kernel<double2, float2><<<g, 256, 0, s>>>(a, (const double2*)x, b, (float2*)y, n, xs, ys); count_launches(1); }
  else return MG_ERR_ARG;
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// out[r] = x[r] / sqrt(nrm2[r*ldn].x); store[r*lds] = (sqrt(...), 0).  A vanishing
// norm gives a zero vector and a zero stored norm (invariant Krylov space).
template <class T2>
__global__ void normalize_kernel(const T2* __restrict__ x, T2* __restrict__ out, const double2* __restrict__ nrm2,
                                 int ldn, double2* __restrict__ store, int lds, size_t n, size_t stride) {
  typedef typename RealOf<T2>::R R;
  const int r = blockIdx.y;
  const double nn = sqrt(fmax(nrm2[(size_t)r * ldn].x, 0.0));
  const R inv = nn > 0.0 ? (R)(1.0 / nn) : (R)0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && store) store[(size_t)r * lds] = make_double2(nn, 0.0);
  const T2* xr = x + r * stride;
  T2* o = out + r * stride;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T2 u = xr[i];
    u.x *= inv;
    u.y *= inv;
    o[i] = u;
  }
}

int blas_normalize(int type, const BVec& b, const void* x, void* out, const double2* nrm2, int ldn, double2* store,
                   int lds, cudaStream_t s) {
  count_bytes(2.0 * b.n * b.R * (type == P64 ? 16 : 8));
  const dim3 g = stream_grid(b.n, b.R);
  if (type == P64) { normalize_kernel<double2><<<g, 256, 0, s>>>((const double2*)x, (double2*)out, nrm2, ldn, store, lds, b.n, b.wstride); count_launches(1); }
  else if (type == P32) { normalize_kernel<float2><<<g, 256, 0, s>>>((const float2*)x, (float2*)out, nrm2, ldn, store, lds, b.n, b.wstride); count_launches(1); }
  else return MG_ERR_ARG;
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Least-squares solve of the (m+1) x m Hessenberg system min ||beta e1 - H y||
// of fixed-step GMRES, one right-hand side per thread block (thread 0): Givens
// rotations and back substitution.  H for RHS r at H + r*ldr, column-major with
// leading dimension ldh; beta2[r].x = ||b_r||^2; y[r*ldy + j].  Columns after a
// zero subdiagonal entry are unused.  m <= 32.
__global__ void hessenberg_solve_kernel(const double2* __restrict__ Hall, int ldh, int ldr, int m,
                                        const double2* __restrict__ beta2, double2* __restrict__ yall, int ldy) {
  if (threadIdx.x != 0) return;
  const int r = blockIdx.x;
  const double2* Hin = Hall + (size_t)r * ldr;
  double2* y = yall + (size_t)r * ldy;
  double hr[33 * 32], hi[33 * 32];
  double gr[33], gi[33];
  for (int j = 0; j < m; ++j) y[j] = make_double2(0, 0);
  const double beta = sqrt(fmax(beta2[r].x, 0.0));
  if (beta == 0.0) return;
  int mm = m;
  for (int j = 0; j < m; ++j)
    if (Hin[(j + 1) + j * ldh].x == 0.0) { mm = j + 1; break; }
  for (int j = 0; j < mm; ++j)
    for (int i = 0; i <= j + 1; ++i) { hr[i + j * 33] = Hin[i + j * ldh].x; hi[i + j * 33] = Hin[i + j * ldh].y; }
  for (int i = 0; i <= mm; ++i) gr[i] = gi[i] = 0;
  gr[0] = beta;
  for (int j = 0; j < mm; ++j) {
    const double ar = hr[j + j * 33], ai = hi[j + j * 33];
    const double br = hr[j + 1 + j * 33], bi = hi[j + 1 + j * 33];
    const double na = sqrt(ar * ar + ai * ai), nb = sqrt(br * br + bi * bi);
    const double den = sqrt(na * na + nb * nb);
    double c, sr, si;
    if (den == 0.0) { c = 1; sr = si = 0; }
    else if (na == 0.0) { c = 0; sr = 1; si = 0; }
    else {
      c = na / den;
      const double pr = ar / na, pi = ai / na;    // s = (a/|a|) conj(b) / den
      sr = (pr * br + pi * bi) / den;
      si = (pi * br - pr * bi) / den;
    }
    for (int k = j; k < mm; ++k) {                  // rotate rows j, j+1
      const double xr = hr[j + k * 33], xi = hi[j + k * 33];
      const double zr = hr[j + 1 + k * 33], zi = hi[j + 1 + k * 33];
      hr[j + k * 33] = c * xr + (sr * zr - si * zi);
      hi[j + k * 33] = c * xi + (sr * zi + si * zr);
      hr[j + 1 + k * 33] = -(sr * xr + si * xi) + c * zr;
      hi[j + 1 + k * 33] = -(sr * xi - si * xr) + c * zi;
    }
    const double xr = gr[j], xi = gi[j];
    gr[j] = c * xr;
    gi[j] = c * xi;
    gr[j + 1] = -(sr * xr + si * xi);
    gi[j + 1] = -(sr * xi - si * xr);
  }
  for (int i = mm - 1; i >= 0; --i) {
    double sr = gr[i], si = gi[i];
    for (int k = i + 1; k < mm; ++k) {
      const double hr_ = hr[i + k * 33], hi_ = hi[i + k * 33];
      const double yr = y[k].x, yi = y[k].y;
      sr -= hr_ * yr - hi_ * yi;
      si -= hr_ * yi + hi_ * yr;
    }
    const double dr = hr[i + i * 33], di = hi[i + i * 33];
    const double d2 = dr * dr + di * di;
    y[i] = d2 > 0 ? make_double2((sr * dr + si * di) / d2, (si * dr - sr * di) / d2) : make_double2(0, 0);
  }
}

int blas_hessenberg_solve(const double2* H, int ldh, int ldr, int m, const double2* beta2, double2* y, int ldy,
                          int R, cudaStream_t s) {
  if (m > 32) return MG_ERR_ARG;
  hessenberg_solve_kernel<<<R, 32, 0, s>>>(H, ldh, ldr, m, beta2, y, ldy); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
