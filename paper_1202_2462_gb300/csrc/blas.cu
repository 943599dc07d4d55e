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
// of fixed-step GMRES, one warp per right-hand side: H in shared memory, each
// Givens rotation computed by every lane (same values) and applied to the
// columns in parallel, back substitution with warp-reduced row sums.  H for
// RHS r at H + r*ldr, column-major with leading dimension ldh; beta2[r].x =
// ||b_r||^2; y[r*ldy + j].  Columns after a zero subdiagonal entry are
// unused.  m <= 32.
__global__ void __launch_bounds__(32) hessenberg_solve_kernel(const double2* __restrict__ Hall, int ldh, int ldr,
                                                              int m, const double2* __restrict__ beta2,
                                                              double2* __restrict__ yall, int ldy) {
  __shared__ double hr[33 * 32], hi[33 * 32];
  __shared__ double gr[33], gi[33], yr[32], yi[32];
  const int r = blockIdx.x, lane = threadIdx.x;
  const double2* Hin = Hall + (size_t)r * ldr;
  double2* y = yall + (size_t)r * ldy;
  const double beta = sqrt(fmax(beta2[r].x, 0.0));
  if (beta == 0.0) {
    for (int j = lane; j < m; j += 32) y[j] = make_double2(0, 0);
    return;
  }
  int mm = m;
  for (int j = 0; j < m; ++j)
    if (Hin[(j + 1) + j * ldh].x == 0.0) { mm = j + 1; break; }
  for (int idx = lane; idx < 33 * mm; idx += 32) {
    const int k = idx / 33, i = idx % 33;
    const bool in = i <= k + 1;
    hr[idx] = in ? Hin[i + k * ldh].x : 0.0;
    hi[idx] = in ? Hin[i + k * ldh].y : 0.0;
  }
  for (int i = lane; i <= mm; i += 32) { gr[i] = i == 0 ? beta : 0.0; gi[i] = 0.0; }
  __syncwarp();
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
    __syncwarp();                                   // every lane has read column j
    for (int k = j + lane; k < mm; k += 32) {       // rotate rows j, j+1 of column k
      const double xr = hr[j + k * 33], xi = hi[j + k * 33];
      const double zr = hr[j + 1 + k * 33], zi = hi[j + 1 + k * 33];
      hr[j + k * 33] = c * xr + (sr * zr - si * zi);
      hi[j + k * 33] = c * xi + (sr * zi + si * zr);
      hr[j + 1 + k * 33] = -(sr * xr + si * xi) + c * zr;
      hi[j + 1 + k * 33] = -(sr * xi - si * xr) + c * zi;
    }
    if (lane == 0) {
      const double xr = gr[j], xi = gi[j];
      gr[j] = c * xr;
      gi[j] = c * xi;
      gr[j + 1] = -(sr * xr + si * xi);
      gi[j + 1] = -(sr * xi - si * xr);
    }
    __syncwarp();
  }
  for (int i = mm - 1; i >= 0; --i) {
    double sr = 0, si = 0;
    for (int k = i + 1 + lane; k < mm; k += 32) {
      const double hr_ = hr[i + k * 33], hi_ = hi[i + k * 33];
      sr += hr_ * yr[k] - hi_ * yi[k];
      si += hr_ * yi[k] + hi_ * yr[k];
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if (lane == 0) {
      const double tr = gr[i] - sr, ti = gi[i] - si;
      const double dr = hr[i + i * 33], di = hi[i + i * 33];
      const double d2 = dr * dr + di * di;
      yr[i] = d2 > 0 ? (tr * dr + ti * di) / d2 : 0.0;
      yi[i] = d2 > 0 ? (ti * dr - tr * di) / d2 : 0.0;
    }
    __syncwarp();
  }
  for (int j = lane; j < m; j += 32) y[j] = j < mm ? make_double2(yr[j], yi[j]) : make_double2(0, 0);
}

// ------------------------------------------------------------ delayed reorthogonalisation
// One Arnoldi step with classical Gram-Schmidt whose second pass is delayed by
// one step (low-synchronisation CGS2, Bielich, Langou, Thomas, Swirydowicz,
// Yamazaki, Boman, Parallel Computing 2022): the previous basis vector u (one
// pass done) is reorthogonalised in the same sweeps that orthogonalise the new
// vector w, so each step reads the basis twice instead of four times.
//   pass 1: A_i = <v_i, u>, B_i = <v_i, w> (i < j), d = <u, u>, c = <u, w>, <w, w>;
//   coefficients: beta = sqrt(d - sum |A_i|^2), v_j = (u - sum A_i v_i) / beta,
//                 h_j = (c - sum conj(A_i) B_i) / beta;
//   pass 2: u <- v_j, w <- w - sum_i B_i v_i - h_j v_j (and both norms).

// A load unit: two FP32 complex numbers (float4) or one FP64 complex (double2).
template <class T2> struct Unit;
template <> struct Unit<float2> { typedef float4 V; typedef float R; static constexpr int C = 2; };
template <> struct Unit<double2> { typedef double2 V; typedef double R; static constexpr int C = 1; };

__device__ __forceinline__ void cdot_acc(const float4& a, const float4& x, float& re, float& im) {
  re = fmaf(a.x, x.x, fmaf(a.y, x.y, fmaf(a.z, x.z, fmaf(a.w, x.w, re))));
  im = fmaf(a.x, x.y, fmaf(-a.y, x.x, fmaf(a.z, x.w, fmaf(-a.w, x.z, im))));
}
__device__ __forceinline__ void cdot_acc(const double2& a, const double2& x, double& re, double& im) {
  re = fma(a.x, x.x, fma(a.y, x.y, re));
  im = fma(a.x, x.y, fma(-a.y, x.x, im));
}
__device__ __forceinline__ void caxpy(float cr, float ci, const float4& a, float4& y) {
  y.x = fmaf(cr, a.x, fmaf(-ci, a.y, y.x));
  y.y = fmaf(cr, a.y, fmaf(ci, a.x, y.y));
  y.z = fmaf(cr, a.z, fmaf(-ci, a.w, y.z));
  y.w = fmaf(cr, a.w, fmaf(ci, a.z, y.w));
}
__device__ __forceinline__ void caxpy(double cr, double ci, const double2& a, double2& y) {
  y.x = fma(cr, a.x, fma(-ci, a.y, y.x));
  y.y = fma(cr, a.y, fma(ci, a.x, y.y));
}
__device__ __forceinline__ float nrm_of(const float4& y) { return y.x * y.x + y.y * y.y + y.z * y.z + y.w * y.w; }
__device__ __forceinline__ double nrm_of(const double2& y) { return y.x * y.x + y.y * y.y; }
template <class V> __device__ __forceinline__ V vzero();
template <> __device__ __forceinline__ float4 vzero<float4>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double2>() { return make_double2(0.0, 0.0); }

constexpr int kDots2Max = 12;      // basis vectors per pass-1 launch
constexpr int kDots2Slots = 32;    // partial slots per (right-hand side, CTA)
template <class V> struct PtrsV { const V* p[16]; };

// slots: [i] = <v_i, u>, [K + i] = <v_i, w>, [2K + 0..2] = <u,u>, <u,w>, <w,w> (EXTRA only)
template <class T2, int K, bool EXTRA>
__global__ void __launch_bounds__(256) dots2_partial(PtrsV<typename Unit<T2>::V> v,
                                                     const typename Unit<T2>::V* __restrict__ u,
                                                     const typename Unit<T2>::V* __restrict__ w, size_t nu,
                                                     size_t stride, double2* __restrict__ partial) {
  typedef typename Unit<T2>::V V;
  typedef typename Unit<T2>::R R;
  constexpr int NS = 2 * K + (EXTRA ? 3 : 0);
  const int r = blockIdx.y;
  const V* ur = u + r * stride;
  const V* wr = w + r * stride;
  R re[NS > 0 ? NS : 1], im[NS > 0 ? NS : 1];
#pragma unroll
  for (int q = 0; q < NS; ++q) re[q] = im[q] = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    V a[K > 0 ? K : 1];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = __ldg(v.p[q] + r * stride + i);
    const V x = __ldg(ur + i);
    const V y = __ldg(wr + i);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      cdot_acc(a[q], x, re[q], im[q]);
      cdot_acc(a[q], y, re[K + q], im[K + q]);
    }
    if (EXTRA) {
      cdot_acc(x, x, re[2 * K], im[2 * K]);
      cdot_acc(x, y, re[2 * K + 1], im[2 * K + 1]);
      cdot_acc(y, y, re[2 * K + 2], im[2 * K + 2]);
    }
  }
  __shared__ double red[8][2 * kDots2Slots];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const R s = warp_sum(re[q]);
    const R m = warp_sum(im[q]);
    if (lane == 0) { red[wid][2 * q] = (double)s; red[wid][2 * q + 1] = (double)m; }
  }
  __syncthreads();
  if ((int)threadIdx.x < NS) {
    double s = 0, m = 0;
    for (int q = 0; q < 8; ++q) { s += red[q][2 * threadIdx.x]; m += red[q][2 * threadIdx.x + 1]; }
    partial[((size_t)r * gridDim.x + blockIdx.x) * kDots2Slots + threadIdx.x] = make_double2(s, m);
  }
}

// Sums the CTAs' slots: A[r*ld + j0 + i], B[r*ld + j0 + i] (i < K), X[r*4 + e].
__global__ void dots2_finalize(const double2* __restrict__ partial, int ncta, int K, bool extra, double2* A,
                               double2* B, double2* X, int ld, int j0) {
  __shared__ double red[8][2];
  const int r = blockIdx.x;
  const int ns = 2 * K + (extra ? 3 : 0);
  for (int q = 0; q < ns; ++q) {
    double s = 0, m = 0;
    for (int c = threadIdx.x; c < ncta; c += blockDim.x) {
      const double2 v = partial[((size_t)r * ncta + c) * kDots2Slots + q];
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
      for (int k = 0; k < 8; ++k) { ss += red[k][0]; sm += red[k][1]; }
      const double2 o = make_double2(ss, sm);
      if (q < K) A[(size_t)r * ld + j0 + q] = o;
      else if (q < 2 * K) B[(size_t)r * ld + j0 + q - K] = o;
      else X[(size_t)r * 4 + q - 2 * K] = o;
    }
    __syncthreads();
  }
}

// Per right-hand side (one thread): beta, h_j and the pass-2 coefficients for
// the vector list [u, w, v_0 .. v_{j-1}]: c1 makes v_j, c2 makes the new w.
// hcol[0..j] = (B_0 .. B_{j-1}, h_j); acol[0..j] = (A_0 .. A_{j-1}, beta).  A
// vanishing beta (u in the span of the basis: a zero or invariant direction)
// gives zero coefficients.
__global__ void dcgs2_coeff_kernel(int j, const double2* __restrict__ A, const double2* __restrict__ B,
                                   const double2* __restrict__ X, int ld, double2* c1, double2* c2, int ldc,
                                   double2* hcol, double2* acol) {
  if (threadIdx.x != 0) return;
  const int r = blockIdx.x;
  const double2* a = A + (size_t)r * ld;
  const double2* b = B + (size_t)r * ld;
  const double2* x = X + (size_t)r * 4;
  double2* o1 = c1 + (size_t)r * ldc;
  double2* o2 = c2 + (size_t)r * ldc;
  double2* hc = hcol + (size_t)r * ld;
  double2* ac = acol + (size_t)r * ld;
  double na = 0;
  for (int i = 0; i < j; ++i) na += a[i].x * a[i].x + a[i].y * a[i].y;
  const double d = x[0].x;
  const double beta2 = d - na;
  if (!(beta2 > 1e-24 * d) || !(d > 0)) {
    for (int i = 0; i < j + 2; ++i) { o1[i] = make_double2(0, 0); o2[i] = make_double2(0, 0); }
    for (int i = 0; i <= j; ++i) { hc[i] = make_double2(0, 0); ac[i] = make_double2(0, 0); }
    return;
  }
  const double beta = sqrt(beta2), ib = 1.0 / beta;
  double sr = x[1].x, si = x[1].y;                          // c - sum conj(a_i) b_i
  for (int i = 0; i < j; ++i) {
    sr -= a[i].x * b[i].x + a[i].y * b[i].y;
    si -= a[i].x * b[i].y - a[i].y * b[i].x;
  }
  const double hr = sr * ib, hi = si * ib;                  // h_j
  const double gr = hr * ib, gi = hi * ib;                  // h_j / beta
  o1[0] = make_double2(ib, 0);
  o1[1] = make_double2(0, 0);
  o2[0] = make_double2(-gr, -gi);
  o2[1] = make_double2(1, 0);
  for (int i = 0; i < j; ++i) {
    o1[2 + i] = make_double2(-a[i].x * ib, -a[i].y * ib);
    // -(b_i - (h_j / beta) a_i)
    o2[2 + i] = make_double2(-(b[i].x - (gr * a[i].x - gi * a[i].y)), -(b[i].y - (gr * a[i].y + gi * a[i].x)));
    hc[i] = b[i];
    ac[i] = a[i];
  }
  hc[j] = make_double2(hr, hi);
  ac[j] = make_double2(beta, 0);
}

// y1 = (acc ? y1 : 0) + sum c1_q v_q, y2 likewise; y1 and y2 may be v_0, v_1
// (every element is read before it is written, by the same thread).  With
// partial != nullptr the CTA writes its parts of ||y1||^2 and ||y2||^2.
template <class T2, int K>
__global__ void __launch_bounds__(256) axpy2_kernel(PtrsV<typename Unit<T2>::V> v, const double2* __restrict__ c1,
                                                    const double2* __restrict__ c2, int ldc, int j0,
                                                    typename Unit<T2>::V* y1, typename Unit<T2>::V* y2, size_t nu,
                                                    size_t stride, int acc, double2* __restrict__ partial) {
  typedef typename Unit<T2>::V V;
  typedef typename Unit<T2>::R R;
  __shared__ R cf[4][16];
  const int r = blockIdx.y;
  if (threadIdx.x < K) {
    const double2 p = c1[(size_t)r * ldc + j0 + threadIdx.x], q = c2[(size_t)r * ldc + j0 + threadIdx.x];
    cf[0][threadIdx.x] = (R)p.x;
    cf[1][threadIdx.x] = (R)p.y;
    cf[2][threadIdx.x] = (R)q.x;
    cf[3][threadIdx.x] = (R)q.y;
  }
  __syncthreads();
  V* o1 = y1 + r * stride;
  V* o2 = y2 + r * stride;
  R n1 = 0, n2 = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    V a[K];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = v.p[q][r * stride + i];
    V s1 = acc ? o1[i] : vzero<V>();
    V s2 = acc ? o2[i] : vzero<V>();
#pragma unroll
    for (int q = 0; q < K; ++q) {
      caxpy(cf[0][q], cf[1][q], a[q], s1);
      caxpy(cf[2][q], cf[3][q], a[q], s2);
    }
    o1[i] = s1;
    o2[i] = s2;
    n1 += nrm_of(s1);
    n2 += nrm_of(s2);
  }
  if (partial) {
    __shared__ double red[8][2];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const R t1 = warp_sum(n1), t2 = warp_sum(n2);
    if (lane == 0) { red[wid][0] = (double)t1; red[wid][1] = (double)t2; }
    __syncthreads();
    if (threadIdx.x < 2) {
      double sum = 0;
      for (int q = 0; q < 8; ++q) sum += red[q][threadIdx.x];
      partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk + threadIdx.x] = make_double2(sum, 0.0);
    }
  }
}

template <class T2>
static int dcgs2_step_t(const BVec& b, const void* const* v, int j, void* u, void* w, const DcgsWork& ws,
                        cudaStream_t s) {
  typedef typename Unit<T2>::V V;
  constexpr int C = Unit<T2>::C;
  const size_t nu = b.n / C, stride = b.vstride / C;
  const int R = b.R;
  // pass 1: dots of u and w with the basis (chunks of kDots2Max) and with each other
  const int ncta1 = std::max(1, std::min(reduce_ctas(nu, R), (int)(kPartialDouble2 / kDots2Slots / (size_t)R)));
  const dim3 g1(ncta1, R);
  int j0 = 0;
  do {
    const int kk = std::min(kDots2Max, j - j0);
    const bool extra = (j0 == 0);
    PtrsV<V> p;
    for (int q = 0; q < 16; ++q) p.p[q] = j > 0 ? (const V*)v[std::max(0, std::min(j0 + q, j - 1))] : (const V*)u;
#define SAPMG_D2(K)                                                                                          \
  case K:                                                                                                    \
    if (extra) { dots2_partial<T2, K, true><<<g1, 256, 0, s>>>(p, (const V*)u, (const V*)w, nu, stride, ws.partial); } \
    else { dots2_partial<T2, K, false><<<g1, 256, 0, s>>>(p, (const V*)u, (const V*)w, nu, stride, ws.partial); } \
    count_launches(1);                                                                                       \
    break;
    switch (kk) {
      SAPMG_D2(0) SAPMG_D2(1) SAPMG_D2(2) SAPMG_D2(3) SAPMG_D2(4) SAPMG_D2(5) SAPMG_D2(6)
      SAPMG_D2(7) SAPMG_D2(8) SAPMG_D2(9) SAPMG_D2(10) SAPMG_D2(11) SAPMG_D2(12)
      default: return MG_ERR_ARG;
    }
#undef SAPMG_D2
    dots2_finalize<<<R, 256, 0, s>>>(ws.partial, ncta1, kk, extra, ws.A, ws.B, ws.X, ws.ld, j0); count_launches(1);
    j0 += kk;
  } while (j0 < j);
  dcgs2_coeff_kernel<<<R, 32, 0, s>>>(j, ws.A, ws.B, ws.X, ws.ld, ws.c1, ws.c2, ws.ld, ws.hcol, ws.acol);
  count_launches(1);
  // pass 2 over the list [u, w, v_0 .. v_{j-1}] in chunks of 16
  const dim3 g2(reduce_ctas(nu, R), R);
  const int total = j + 2;
  for (int q0 = 0; q0 < total; q0 += 16) {
    const int kk = std::min(16, total - q0);
    const bool last = q0 + 16 >= total;
    PtrsV<V> p;
    for (int q = 0; q < 16; ++q) {
      const int t = q0 + std::min(q, kk - 1);
      p.p[q] = (const V*)(t == 0 ? u : (t == 1 ? w : v[t - 2]));
    }
    double2* part = last ? ws.partial : nullptr;
    const int acc = q0 > 0;
#define SAPMG_A2(K)                                                                                            \
  case K:                                                                                                      \
    axpy2_kernel<T2, K><<<g2, 256, 0, s>>>(p, ws.c1, ws.c2, ws.ld, q0, (V*)u, (V*)w, nu, stride, acc, part); \
    count_launches(1);                                                                                         \
    break;
    switch (kk) {
      SAPMG_A2(1) SAPMG_A2(2) SAPMG_A2(3) SAPMG_A2(4) SAPMG_A2(5) SAPMG_A2(6) SAPMG_A2(7) SAPMG_A2(8)
      SAPMG_A2(9) SAPMG_A2(10) SAPMG_A2(11) SAPMG_A2(12) SAPMG_A2(13) SAPMG_A2(14) SAPMG_A2(15) SAPMG_A2(16)
      default: return MG_ERR_ARG;
    }
#undef SAPMG_A2
  }
  multidot_finalize<<<R, 256, 0, s>>>(ws.partial, (int)g2.x, 2, ws.nrm, ws.ld, 0, nullptr); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_dcgs2_step(int type, const BVec& b, const void* const* v, int j, void* u, void* w, const DcgsWork& ws,
                    cudaStream_t s) {
  if (b.R <= 0) return MG_OK;
  if (j < 0 || j + 2 > ws.ld || b.R > 32) return MG_ERR_ARG;
  // pass 1 reads the j basis vectors, u and w; pass 2 reads them again and writes u and w
  count_bytes((double)(2 * j + 6) * b.n * b.R * (type == P64 ? 16 : 8));
  if (type == P32) {
    bool al = (b.n % 2 == 0) && (b.vstride == b.n) && ((reinterpret_cast<uintptr_t>(u) & 15) == 0) &&
              ((reinterpret_cast<uintptr_t>(w) & 15) == 0);
    for (int q = 0; q < j; ++q) al = al && ((reinterpret_cast<uintptr_t>(v[q]) & 15) == 0);
    if (!al) return MG_ERR_ARG;
    return dcgs2_step_t<float2>(b, v, j, u, w, ws, s);
  }
  if (type == P64) {
    if (b.vstride != b.n) return MG_ERR_ARG;
    return dcgs2_step_t<double2>(b, v, j, u, w, ws, s);
  }
  return MG_ERR_ARG;
}

// ------------------------------------------------------------ FP16 basis
// The finished basis vectors of the mixed form's outer Arnoldi may be kept in
// FP16, scaled by kBasisScale = 2^10 (a unit vector's entries stay below 1, so
// the scaled values stay in FP16's normal range and the scaling is exact).
// Eight bytes = two complex numbers per load unit.

__device__ __forceinline__ float4 h4_to_f4(uint2 u) {
  const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
  const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  constexpr float is = 1.f / kBasisScale;
  return make_float4(a.x * is, a.y * is, b.x * is, b.y * is);
}

__device__ __forceinline__ uint2 f4_to_h4(float4 v) {
  const __half2 a = __floats2half2_rn(v.x * kBasisScale, v.y * kBasisScale);
  const __half2 b = __floats2half2_rn(v.z * kBasisScale, v.w * kBasisScale);
  uint2 u;
  u.x = *reinterpret_cast<const unsigned int*>(&a);
  u.y = *reinterpret_cast<const unsigned int*>(&b);
  return u;
}

// pass 1 with an FP16 basis: slots as dots2_partial
template <int K, bool EXTRA>
__global__ void __launch_bounds__(256) dots2h_partial(PtrsV<uint2> v, const float4* __restrict__ u,
                                                      const float4* __restrict__ w, size_t nu, size_t stride,
                                                      double2* __restrict__ partial) {
  constexpr int NS = 2 * K + (EXTRA ? 3 : 0);
  const int r = blockIdx.y;
  const float4* ur = u + r * stride;
  const float4* wr = w + r * stride;
  float re[NS > 0 ? NS : 1], im[NS > 0 ? NS : 1];
#pragma unroll
  for (int q = 0; q < NS; ++q) re[q] = im[q] = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    uint2 a[K > 0 ? K : 1];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = __ldg(v.p[q] + r * stride + i);
    const float4 x = __ldg(ur + i);
    const float4 y = __ldg(wr + i);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const float4 av = h4_to_f4(a[q]);
      cdot_acc(av, x, re[q], im[q]);
      cdot_acc(av, y, re[K + q], im[K + q]);
    }
    if (EXTRA) {
      cdot_acc(x, x, re[2 * K], im[2 * K]);
      cdot_acc(x, y, re[2 * K + 1], im[2 * K + 1]);
      cdot_acc(y, y, re[2 * K + 2], im[2 * K + 2]);
    }
  }
  __shared__ double red[8][2 * kDots2Slots];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    const float a = warp_sum(re[q]);
    const float b = warp_sum(im[q]);
    if (lane == 0) { red[wid][2 * q] = (double)a; red[wid][2 * q + 1] = (double)b; }
  }
  __syncthreads();
  if ((int)threadIdx.x < NS) {
    double a = 0, b = 0;
    for (int q = 0; q < 8; ++q) { a += red[q][2 * threadIdx.x]; b += red[q][2 * threadIdx.x + 1]; }
    partial[((size_t)r * gridDim.x + blockIdx.x) * kDots2Slots + threadIdx.x] = make_double2(a, b);
  }
}

// pass 2 with an FP16 basis.  Coefficient q of c1/c2 belongs to [u, w, v_0, ...].
// first: y1 = c1_u u + c1_w w + sum, y2 likewise; otherwise y1 += sum (y1 kept
// in u), y2 += sum (in w).  vout != nullptr (last chunk): v_j = y1 is
// written to the FP16 basis and to u only if keep_u; partial: ||y1||^2, ||y2||^2.
template <int K>
__global__ void __launch_bounds__(256) axpy2h_kernel(PtrsV<uint2> v, const double2* __restrict__ c1,
                                                     const double2* __restrict__ c2, int ldc, int q0, float4* u,
                                                     float4* w, uint2* __restrict__ vout, size_t nu, size_t stride,
                                                     int first, int keep_u, double2* __restrict__ partial) {
  __shared__ float cf[4][18];
  const int r = blockIdx.y;
  if ((int)threadIdx.x < K + 2) {
    const int q = threadIdx.x;                       // 0, 1: u, w (first chunk); 2..: basis entries
    const int ci = q < 2 ? q : 2 + q0 + (q - 2);
    const double2 p = c1[(size_t)r * ldc + ci], t = c2[(size_t)r * ldc + ci];
    cf[0][q] = (float)p.x;
    cf[1][q] = (float)p.y;
    cf[2][q] = (float)t.x;
    cf[3][q] = (float)t.y;
  }
  __syncthreads();
  float4* o1 = u + r * stride;
  float4* o2 = w + r * stride;
  uint2* ov = vout ? vout + r * stride : nullptr;
  float n1 = 0.f, n2 = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    uint2 a[K > 0 ? K : 1];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = __ldg(v.p[q] + r * stride + i);
    const float4 uu = o1[i], ww = o2[i];
    float4 s1, s2;
    if (first) {
      s1 = vzero<float4>();
      s2 = vzero<float4>();
      caxpy(cf[0][0], cf[1][0], uu, s1);
      caxpy(cf[0][1], cf[1][1], ww, s1);
      caxpy(cf[2][0], cf[3][0], uu, s2);
      caxpy(cf[2][1], cf[3][1], ww, s2);
    } else {
      s1 = uu;
      s2 = ww;
    }
#pragma unroll
    for (int q = 0; q < K; ++q) {
      const float4 av = h4_to_f4(a[q]);
      caxpy(cf[0][2 + q], cf[1][2 + q], av, s1);
      caxpy(cf[2][2 + q], cf[3][2 + q], av, s2);
    }
    if (!ov || keep_u) o1[i] = s1;
    o2[i] = s2;
    if (ov) ov[i] = f4_to_h4(s1);
    n1 += nrm_of(s1);
    n2 += nrm_of(s2);
  }
  if (partial) {
    __shared__ double red[8][2];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float t1 = warp_sum(n1), t2 = warp_sum(n2);
    if (lane == 0) { red[wid][0] = (double)t1; red[wid][1] = (double)t2; }
    __syncthreads();
    if (threadIdx.x < 2) {
      double sum = 0;
      for (int q = 0; q < 8; ++q) sum += red[q][threadIdx.x];
      partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk + threadIdx.x] = make_double2(sum, 0.0);
    }
  }
}

int blas_dcgs2_step_h(const BVec& b, const void* const* vh, int j, void* u, void* w, void* vout, const DcgsWork& ws,
                      cudaStream_t s) {
  if (b.R <= 0) return MG_OK;
  if (j < 0 || j + 2 > ws.ld || b.R > 32 || b.n % 2 != 0 || b.vstride != b.n) return MG_ERR_ARG;
  bool al = ((reinterpret_cast<uintptr_t>(u) & 15) == 0) && ((reinterpret_cast<uintptr_t>(w) & 15) == 0) &&
            ((reinterpret_cast<uintptr_t>(vout) & 7) == 0);
  for (int q = 0; q < j; ++q) al = al && ((reinterpret_cast<uintptr_t>(vh[q]) & 7) == 0);
  if (!al) return MG_ERR_ARG;
  // pass 1: j FP16 basis vectors + u, w; pass 2: the same + w written + v_j in FP16
  // (u is written back only between chunks, when j > 16)
  count_bytes(((double)2 * j * 4 + 5 * 8 + 4) * b.n * b.R);
  const size_t nu = b.n / 2, stride = b.vstride / 2;
  const int R = b.R;
  const int ncta1 = std::max(1, std::min(reduce_ctas(nu, R), (int)(kPartialDouble2 / kDots2Slots / (size_t)R)));
  const dim3 g1(ncta1, R);
  const float4* uf = (const float4*)u;
  const float4* wf = (const float4*)w;
  int j0 = 0;
  do {
    const int kk = std::min(kDots2Max, j - j0);
    const bool extra = (j0 == 0);
    PtrsV<uint2> p;
    for (int q = 0; q < 16; ++q) p.p[q] = j > 0 ? (const uint2*)vh[std::max(0, std::min(j0 + q, j - 1))] : (const uint2*)vout;
#define SAPMG_D2H(K)                                                                                              \
  case K:                                                                                                         \
    if (extra) { dots2h_partial<K, true><<<g1, 256, 0, s>>>(p, uf, wf, nu, stride, ws.partial); }                \
    else { dots2h_partial<K, false><<<g1, 256, 0, s>>>(p, uf, wf, nu, stride, ws.partial); }                     \
    count_launches(1);                                                                                            \
    break;
    switch (kk) {
      SAPMG_D2H(0) SAPMG_D2H(1) SAPMG_D2H(2) SAPMG_D2H(3) SAPMG_D2H(4) SAPMG_D2H(5) SAPMG_D2H(6)
      SAPMG_D2H(7) SAPMG_D2H(8) SAPMG_D2H(9) SAPMG_D2H(10) SAPMG_D2H(11) SAPMG_D2H(12)
      default: return MG_ERR_ARG;
    }
#undef SAPMG_D2H
    dots2_finalize<<<R, 256, 0, s>>>(ws.partial, ncta1, kk, extra, ws.A, ws.B, ws.X, ws.ld, j0); count_launches(1);
    j0 += kk;
  } while (j0 < j);
  dcgs2_coeff_kernel<<<R, 32, 0, s>>>(j, ws.A, ws.B, ws.X, ws.ld, ws.c1, ws.c2, ws.ld, ws.hcol, ws.acol);
  count_launches(1);
  const dim3 g2(reduce_ctas(nu, R), R);
  int q0 = 0;
  bool first = true;
  do {
    const int kk = std::min(16, j - q0);
    const bool last = q0 + kk >= j;
    PtrsV<uint2> p;
    for (int q = 0; q < 16; ++q) p.p[q] = j > 0 ? (const uint2*)vh[std::max(0, std::min(q0 + q, j - 1))] : (const uint2*)vout;
    double2* part = last ? ws.partial : nullptr;
    uint2* vo = last ? (uint2*)vout : nullptr;
#define SAPMG_A2H(K)                                                                                                \
  case K:                                                                                                           \
    axpy2h_kernel<K><<<g2, 256, 0, s>>>(p, ws.c1, ws.c2, ws.ld, q0, (float4*)u, (float4*)w, vo, nu, stride, first, \
                                        0, part);                                                                   \
    count_launches(1);                                                                                              \
    break;
    switch (kk) {
      SAPMG_A2H(0) SAPMG_A2H(1) SAPMG_A2H(2) SAPMG_A2H(3) SAPMG_A2H(4) SAPMG_A2H(5) SAPMG_A2H(6) SAPMG_A2H(7)
      SAPMG_A2H(8) SAPMG_A2H(9) SAPMG_A2H(10) SAPMG_A2H(11) SAPMG_A2H(12) SAPMG_A2H(13) SAPMG_A2H(14)
      SAPMG_A2H(15) SAPMG_A2H(16)
      default: return MG_ERR_ARG;
    }
#undef SAPMG_A2H
    q0 += kk;
    first = false;
  } while (q0 < j);
  multidot_finalize<<<R, 256, 0, s>>>(ws.partial, (int)g2.x, 2, ws.nrm, ws.ld, 0, nullptr); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// The coarse-level GMRES with an FP16 basis (same format): <v_j, w> for a list
// of FP16 vectors, w += sign sum c_j v_j (FP32 w, optional norm), and
// out = x / ||x|| written in FP16.
template <int K>
__global__ void __launch_bounds__(256) multidot_h_partial(PtrsV<uint2> v, const float4* __restrict__ w, size_t nu,
                                                          size_t stride, double2* __restrict__ partial) {
  const int r = blockIdx.y;
  const float4* wr = w + r * stride;
  float re[K], im[K];
#pragma unroll
  for (int q = 0; q < K; ++q) re[q] = im[q] = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    uint2 a[K];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = __ldg(v.p[q] + r * stride + i);
    const float4 x = __ldg(wr + i);
#pragma unroll
    for (int q = 0; q < K; ++q) cdot_acc(h4_to_f4(a[q]), x, re[q], im[q]);
  }
  __shared__ double red[8][2 * K];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const float a = warp_sum(re[q]);
    const float b = warp_sum(im[q]);
    if (lane == 0) { red[wid][2 * q] = (double)a; red[wid][2 * q + 1] = (double)b; }
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    double a = 0, b = 0;
    for (int q = 0; q < 8; ++q) { a += red[q][2 * threadIdx.x]; b += red[q][2 * threadIdx.x + 1]; }
    partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk + threadIdx.x] = make_double2(a, b);
  }
}

template <int K>
__global__ void __launch_bounds__(256) multiaxpy_h_kernel(float4* __restrict__ w, PtrsV<uint2> v,
                                                          const double2* __restrict__ coeff, int ldc, double sign,
                                                          size_t nu, size_t stride, double2* __restrict__ partial) {
  __shared__ float cf[2][16];
  const int r = blockIdx.y;
  if ((int)threadIdx.x < K) {
    const double2 c = coeff[(size_t)r * ldc + threadIdx.x];
    cf[0][threadIdx.x] = (float)(sign * c.x);
    cf[1][threadIdx.x] = (float)(sign * c.y);
  }
  __syncthreads();
  float4* wr = w + r * stride;
  float nn = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    uint2 a[K];
#pragma unroll
    for (int q = 0; q < K; ++q) a[q] = __ldg(v.p[q] + r * stride + i);
    float4 x = wr[i];
#pragma unroll
    for (int q = 0; q < K; ++q) caxpy(cf[0][q], cf[1][q], h4_to_f4(a[q]), x);
    wr[i] = x;
    nn += nrm_of(x);
  }
  if (partial) {
    __shared__ double red[8];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float t = warp_sum(nn);
    if (lane == 0) red[wid] = (double)t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0;
      for (int q = 0; q < 8; ++q) sum += red[q];
      partial[((size_t)r * gridDim.x + blockIdx.x) * kChunk] = make_double2(sum, 0.0);
    }
  }
}

__global__ void normalize_h_kernel(const float4* __restrict__ x, uint2* __restrict__ out,
                                   const double2* __restrict__ nrm2, int ldn, double2* __restrict__ store, int lds,
                                   size_t nu, size_t stride) {
  const int r = blockIdx.y;
  const double nn = sqrt(fmax(nrm2[(size_t)r * ldn].x, 0.0));
  const float inv = nn > 0.0 ? (float)(1.0 / nn) : 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0 && store) store[(size_t)r * lds] = make_double2(nn, 0.0);
  const float4* xr = x + r * stride;
  uint2* o = out + r * stride;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nu; i += (size_t)gridDim.x * blockDim.x) {
    float4 u = xr[i];
    u.x *= inv;
    u.y *= inv;
    u.z *= inv;
    u.w *= inv;
    o[i] = f4_to_h4(u);
  }
}

static bool half_ok(const BVec& b, const void* w, const void* const* v, int k) {
  bool al = (b.n % 2 == 0) && (b.vstride == b.n) && ((reinterpret_cast<uintptr_t>(w) & 15) == 0);
  for (int q = 0; q < k; ++q) al = al && ((reinterpret_cast<uintptr_t>(v[q]) & 7) == 0);
  return al;
}

int blas_multidot_h(const BVec& b, const void* const* v, int k, const void* w, double2* out, int ldo,
                    double2* partial, cudaStream_t s) {
  if (k <= 0 || b.R <= 0) return MG_OK;
  if (!half_ok(b, w, v, k)) return MG_ERR_ARG;
  count_bytes(((double)k * 4 + 8) * b.n * b.R);
  const size_t nu = b.n / 2, stride = b.vstride / 2;
  const int ncta = reduce_ctas(nu, b.R);
  const dim3 grid(ncta, b.R);
  for (int j0 = 0; j0 < k; j0 += kChunk) {
    const int kk = std::min(kChunk, k - j0);
    PtrsV<uint2> p;
    for (int q = 0; q < 16; ++q) p.p[q] = (const uint2*)v[j0 + std::min(q, kk - 1)];
#define SAPMG_MDH(K) case K: multidot_h_partial<K><<<grid, 256, 0, s>>>(p, (const float4*)w, nu, stride, partial); count_launches(1); break;
    switch (kk) {
      SAPMG_MDH(1) SAPMG_MDH(2) SAPMG_MDH(3) SAPMG_MDH(4) SAPMG_MDH(5) SAPMG_MDH(6) SAPMG_MDH(7) SAPMG_MDH(8)
      SAPMG_MDH(9) SAPMG_MDH(10) SAPMG_MDH(11) SAPMG_MDH(12) SAPMG_MDH(13) SAPMG_MDH(14) SAPMG_MDH(15)
      default: multidot_h_partial<16><<<grid, 256, 0, s>>>(p, (const float4*)w, nu, stride, partial); count_launches(1); break;
    }
#undef SAPMG_MDH
    multidot_finalize<<<b.R, 256, 0, s>>>(partial, ncta, kk, out + j0, ldo, 0, nullptr); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_multiaxpy_h(const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc, double sign,
                     double2* nrm2, int ldn, double2* partial, cudaStream_t s) {
  if (k <= 0 || b.R <= 0) return MG_OK;
  if (!half_ok(b, w, v, k)) return MG_ERR_ARG;
  count_bytes(((double)k * 4 + 16) * b.n * b.R);
  const size_t nu = b.n / 2, stride = b.vstride / 2;
  const dim3 g = nrm2 ? dim3(reduce_ctas(nu, b.R), b.R) : stream_grid(nu, b.R);
  for (int j0 = 0; j0 < k; j0 += kChunk) {
    const int kk = std::min(kChunk, k - j0);
    const bool last = j0 + kChunk >= k;
    PtrsV<uint2> p;
    for (int q = 0; q < 16; ++q) p.p[q] = (const uint2*)v[j0 + std::min(q, kk - 1)];
    double2* part = (last && nrm2) ? partial : nullptr;
    const double2* c = coeff + j0;
#define SAPMG_MAH(K) case K: multiaxpy_h_kernel<K><<<g, 256, 0, s>>>((float4*)w, p, c, ldc, sign, nu, stride, part); count_launches(1); break;
    switch (kk) {
      SAPMG_MAH(1) SAPMG_MAH(2) SAPMG_MAH(3) SAPMG_MAH(4) SAPMG_MAH(5) SAPMG_MAH(6) SAPMG_MAH(7) SAPMG_MAH(8)
      SAPMG_MAH(9) SAPMG_MAH(10) SAPMG_MAH(11) SAPMG_MAH(12) SAPMG_MAH(13) SAPMG_MAH(14) SAPMG_MAH(15)
      default: multiaxpy_h_kernel<16><<<g, 256, 0, s>>>((float4*)w, p, c, ldc, sign, nu, stride, part); count_launches(1); break;
    }
#undef SAPMG_MAH
  }
  if (nrm2) {
    multidot_finalize<<<b.R, 256, 0, s>>>(partial, (int)g.x, 1, nrm2, ldn, 0, nullptr); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_normalize_h(const BVec& b, const void* x, void* out, const double2* nrm2, int ldn, double2* store, int lds,
                     cudaStream_t s) {
  if (b.n % 2 != 0 || b.wstride != b.n) return MG_ERR_ARG;
  count_bytes(12.0 * b.n * b.R);
  const size_t nu = b.n / 2;
  const dim3 g = stream_grid(nu, b.R);
  normalize_h_kernel<<<g, 256, 0, s>>>((const float4*)x, (uint2*)out, nrm2, ldn, store, lds, nu, b.wstride / 2);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}


int blas_hessenberg_solve(const double2* H, int ldh, int ldr, int m, const double2* beta2, double2* y, int ldy,
                          int R, cudaStream_t s) {
  if (m > 32) return MG_ERR_ARG;
  hessenberg_solve_kernel<<<R, 32, 0, s>>>(H, ldh, ldr, m, beta2, y, ldy); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
