// K8: vector kernels of the Krylov solvers (Sec. 2 and Sec. 4: GMRES on the
// coarse grid, flexible GMRES outside): fused multi-dot products, fused
// multi-axpy, scaled copies and normalisation with device-resident scalars so
// that the coarse GMRES runs without host round trips.
//
// Reductions are deterministic: every CTA writes its partial sums, one CTA
// adds the partials in a fixed order.  Per-thread partial sums use the
// vector's own precision; CTA-level and final sums use FP64.
#include "internal.h"
#include "blas.h"

namespace sapmg {

template <class T2> struct RealOf;
template <> struct RealOf<double2> { typedef double R; };
template <> struct RealOf<float2> { typedef float R; };

template <class T2> struct Ptrs8 { const T2* p[8]; };

template <class T2, int K>
__global__ void __launch_bounds__(256) multidot_partial(Ptrs8<T2> v, const T2* __restrict__ w, size_t n,
                                                        double2* __restrict__ partial) {
  typedef typename RealOf<T2>::R R;
  R are[K], aim[K];
#pragma unroll
  for (int j = 0; j < K; ++j) are[j] = aim[j] = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T2 x = w[i];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const T2 a = v.p[j][i];
      are[j] = fma(a.x, x.x, fma(a.y, x.y, are[j]));
      aim[j] = fma(a.x, x.y, fma(-a.y, x.x, aim[j]));
    }
  }
  __shared__ double red[8][2 * K];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    double r = warp_sum((double)are[j]);
    double m = warp_sum((double)aim[j]);
    if (lane == 0) { red[wid][2 * j] = r; red[wid][2 * j + 1] = m; }
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double r = 0, m = 0;
    for (int q = 0; q < 8; ++q) { r += red[q][2 * threadIdx.x]; m += red[q][2 * threadIdx.x + 1]; }
    partial[(size_t)blockIdx.x * 8 + threadIdx.x] = make_double2(r, m);
  }
}

// out[j] = (mode 1: out[j] +) sum over CTAs; out2[j] = the sum if out2 != nullptr.
__global__ void multidot_finalize(const double2* __restrict__ partial, int ncta, int k, double2* out, int mode,
                                  double2* out2) {
  __shared__ double red[8][2];
  for (int j = 0; j < k; ++j) {
    double r = 0, m = 0;
    for (int c = threadIdx.x; c < ncta; c += blockDim.x) {
      const double2 v = partial[(size_t)c * 8 + j];
      r += v.x;
      m += v.y;
    }
    r = warp_sum(r);
    m = warp_sum(m);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { red[wid][0] = r; red[wid][1] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0, sm = 0;
      for (int q = 0; q < 8; ++q) { sr += red[q][0]; sm += red[q][1]; }
      if (out) {
        if (mode == 1) { out[j].x += sr; out[j].y += sm; }
        else out[j] = make_double2(sr, sm);
      }
      if (out2) out2[j] = make_double2(sr, sm);
    }
    __syncthreads();
  }
}

static int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(g, kMaxReduceCta));
}

template <class T2, int K>
static void md_launch(int ncta, const Ptrs8<T2>& p, const T2* w, size_t n, double2* part, cudaStream_t s) {
  multidot_partial<T2, K><<<ncta, 256, 0, s>>>(p, w, n, part); count_launches(1);
}

template <class T2>
static int multidot_t(const void* const* v, int k, const void* w, size_t n, double2* out, int mode, double2* out2,
                      double2* partial, cudaStream_t s) {
  const int ncta = grid_for(n);
  for (int j0 = 0; j0 < k; j0 += 8) {
    const int kk = std::min(8, k - j0);
    Ptrs8<T2> p;
    for (int j = 0; j < 8; ++j) p.p[j] = (const T2*)v[j0 + std::min(j, kk - 1)];
    switch (kk) {
      case 1: md_launch<T2, 1>(ncta, p, (const T2*)w, n, partial, s); break;
      case 2: md_launch<T2, 2>(ncta, p, (const T2*)w, n, partial, s); break;
      case 3: md_launch<T2, 3>(ncta, p, (const T2*)w, n, partial, s); break;
      case 4: md_launch<T2, 4>(ncta, p, (const T2*)w, n, partial, s); break;
      case 5: md_launch<T2, 5>(ncta, p, (const T2*)w, n, partial, s); break;
      case 6: md_launch<T2, 6>(ncta, p, (const T2*)w, n, partial, s); break;
      case 7: md_launch<T2, 7>(ncta, p, (const T2*)w, n, partial, s); break;
      default: md_launch<T2, 8>(ncta, p, (const T2*)w, n, partial, s); break;
    }
    multidot_finalize<<<1, 256, 0, s>>>(partial, ncta, kk, out ? out + j0 : nullptr, mode,
                                        out2 ? out2 + j0 : nullptr); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_multidot(int type, const void* const* v, int k, const void* w, size_t n, double2* out, int mode,
                  double2* out2, double2* partial, cudaStream_t s) {
  if (k <= 0) return MG_OK;
  if (type == P64) return multidot_t<double2>(v, k, w, n, out, mode, out2, partial, s);
  if (type == P32) return multidot_t<float2>(v, k, w, n, out, mode, out2, partial, s);
  return MG_ERR_ARG;
}

// w += sign * sum_j coeff[j] v_j
template <class T2, int K>
__global__ void __launch_bounds__(256) multiaxpy_kernel(T2* __restrict__ w, Ptrs8<T2> v,
                                                        const double2* __restrict__ coeff, double sign, size_t n) {
  typedef typename RealOf<T2>::R R;
  R cr[K], ci[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const double2 c = coeff[j];
    cr[j] = (R)(sign * c.x);
    ci[j] = (R)(sign * c.y);
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T2 x = w[i];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const T2 a = v.p[j][i];
      x.x = fma(cr[j], a.x, fma(-ci[j], a.y, x.x));
      x.y = fma(cr[j], a.y, fma(ci[j], a.x, x.y));
    }
    w[i] = x;
  }
}

template <class T2, int K>
static void ma_launch(T2* w, const Ptrs8<T2>& p, const double2* c, double sign, size_t n, cudaStream_t s) {
  const int ncta = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8));
  multiaxpy_kernel<T2, K><<<ncta, 256, 0, s>>>(w, p, c, sign, n); count_launches(1);
}

template <class T2>
static int multiaxpy_t(void* w, const void* const* v, int k, const double2* coeff, double sign, size_t n,
                       cudaStream_t s) {
  for (int j0 = 0; j0 < k; j0 += 8) {
    const int kk = std::min(8, k - j0);
    Ptrs8<T2> p;
    for (int j = 0; j < 8; ++j) p.p[j] = (const T2*)v[j0 + std::min(j, kk - 1)];
    const double2* c = coeff + j0;
    switch (kk) {
      case 1: ma_launch<T2, 1>((T2*)w, p, c, sign, n, s); break;
      case 2: ma_launch<T2, 2>((T2*)w, p, c, sign, n, s); break;
      case 3: ma_launch<T2, 3>((T2*)w, p, c, sign, n, s); break;
      case 4: ma_launch<T2, 4>((T2*)w, p, c, sign, n, s); break;
      case 5: ma_launch<T2, 5>((T2*)w, p, c, sign, n, s); break;
      case 6: ma_launch<T2, 6>((T2*)w, p, c, sign, n, s); break;
      case 7: ma_launch<T2, 7>((T2*)w, p, c, sign, n, s); break;
      default: ma_launch<T2, 8>((T2*)w, p, c, sign, n, s); break;
    }
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_multiaxpy(int type, void* w, const void* const* v, int k, const double2* coeff, double sign, size_t n,
                   cudaStream_t s) {
  if (k <= 0) return MG_OK;
  if (type == P64) return multiaxpy_t<double2>(w, v, k, coeff, sign, n, s);
  if (type == P32) return multiaxpy_t<float2>(w, v, k, coeff, sign, n, s);
  return MG_ERR_ARG;
}

// y = a x + b y (host scalars); x and y may differ in element type.
template <class TX, class TY>
__global__ void axpby_kernel(double ar, double ai, const TX* __restrict__ x, double br, double bi, TY* __restrict__ y,
                             size_t n, int y_is_zero) {
  typedef typename RealOf<TY>::R R;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const TX u = x[i];
    TY o;
    const R ux = (R)u.x, uy = (R)u.y;
    if (y_is_zero) {
      o.x = (R)ar * ux - (R)ai * uy;
      o.y = (R)ar * uy + (R)ai * ux;
    } else {
      const TY v = y[i];
      o.x = (R)ar * ux - (R)ai * uy + (R)br * v.x - (R)bi * v.y;
      o.y = (R)ar * uy + (R)ai * ux + (R)br * v.y + (R)bi * v.x;
    }
    y[i] = o;
  }
}

int blas_axpby2(int tx, double2 a, const void* x, int ty, double2 b, void* y, size_t n, cudaStream_t s) {
  if (n == 0) return MG_OK;
  const int ncta = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8));
  const int z = (b.x == 0.0 && b.y == 0.0) ? 1 : 0;
  if (tx == P64 && ty == P64) { axpby_kernel<double2, double2><<<ncta, 256, 0, s>>>(a.x, a.y, (const double2*)x, b.x, b.y, (double2*)y, n, z); count_launches(1); }
  else if (tx == P32 && ty == P32) { axpby_kernel<float2, float2><<<ncta, 256, 0, s>>>(a.x, a.y, (const float2*)x, b.x, b.y, (float2*)y, n, z); count_launches(1); }
  else if (tx == P32 && ty == P64) { axpby_kernel<float2, double2><<<ncta, 256, 0, s>>>(a.x, a.y, (const float2*)x, b.x, b.y, (double2*)y, n, z); count_launches(1); }
  else if (tx == P64 && ty == P32) { axpby_kernel<double2, float2><<<ncta, 256, 0, s>>>(a.x, a.y, (const double2*)x, b.x, b.y, (float2*)y, n, z); count_launches(1); }
  else return MG_ERR_ARG;
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int blas_axpby(int type, double2 a, const void* x, double2 b, void* y, size_t n, cudaStream_t s) {
  return blas_axpby2(type, a, x, type, b, y, n, s);
}

// out = x / sqrt(nrm2->x); *store = (sqrt(nrm2->x), 0).  Zero output (and a zero
// stored norm) when the norm vanishes: the Krylov space is invariant.
template <class T2>
__global__ void normalize_kernel(const T2* __restrict__ x, T2* __restrict__ out, const double2* __restrict__ nrm2,
                                 double2* __restrict__ store, size_t n) {
  typedef typename RealOf<T2>::R R;
  const double nn = sqrt(fmax(nrm2->x, 0.0));
  const R inv = nn > 0.0 ? (R)(1.0 / nn) : (R)0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && store) *store = make_double2(nn, 0.0);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T2 u = x[i];
    u.x *= inv;
    u.y *= inv;
    out[i] = u;
  }
}

int blas_normalize(int type, const void* x, void* out, const double2* nrm2, double2* store, size_t n,
                   cudaStream_t s) {
  const int ncta = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 152 * 8));
  if (type == P64) { normalize_kernel<double2><<<ncta, 256, 0, s>>>((const double2*)x, (double2*)out, nrm2, store, n); count_launches(1); }
  else if (type == P32) { normalize_kernel<float2><<<ncta, 256, 0, s>>>((const float2*)x, (float2*)out, nrm2, store, n); count_launches(1); }
  else return MG_ERR_ARG;
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Least-squares solve of the (m+1) x m Hessenberg system min ||beta e1 - H y||
// for the fixed-step GMRES: Givens rotations and back substitution by one
// thread (m <= 32).  H is column-major with leading dimension ldh (H[i + j*ldh]);
// beta2 holds ||b||^2.  Columns after a zero subdiagonal entry are unused.
__global__ void hessenberg_solve_kernel(const double2* __restrict__ Hin, int ldh, int m,
                                        const double2* __restrict__ beta2, double2* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double hr[33 * 32], hi[33 * 32];
  double gr[33], gi[33];
  for (int j = 0; j < m; ++j) y[j] = make_double2(0, 0);
  const double beta = sqrt(fmax(beta2->x, 0.0));
  if (beta == 0.0) return;
  int mm = m;
  for (int j = 0; j < m; ++j)
    if (Hin[(j + 1) + j * ldh].x == 0.0) { mm = j + 1; break; }
  for (int j = 0; j < mm; ++j)
    for (int i = 0; i <= j + 1; ++i) { hr[i + j * 33] = Hin[i + j * ldh].x; hi[i + j * 33] = Hin[i + j * ldh].y; }
  for (int i = 0; i <= mm; ++i) gr[i] = gi[i] = 0;
  gr[0] = beta;
  for (int j = 0; j < mm; ++j) {
    // apply previous rotations were applied column by column below
    const double ar = hr[j + j * 33], ai = hi[j + j * 33];
    const double br = hr[j + 1 + j * 33], bi = hi[j + 1 + j * 33];
    const double na = sqrt(ar * ar + ai * ai), nb = sqrt(br * br + bi * bi);
    const double den = sqrt(na * na + nb * nb);
    double c, sr, si;
    if (den == 0.0) { c = 1; sr = si = 0; }
    else if (na == 0.0) { c = 0; sr = 1; si = 0; }
    else {
      c = na / den;
      // s = (a/|a|) conj(b) / den
      const double pr = ar / na, pi = ai / na;
      sr = (pr * br + pi * bi) / den;
      si = (pi * br - pr * bi) / den;
    }
    // rotate rows j, j+1 of columns j..mm-1
    for (int k = j; k < mm; ++k) {
      const double xr = hr[j + k * 33], xi = hi[j + k * 33];
      const double zr = hr[j + 1 + k * 33], zi = hi[j + 1 + k * 33];
      // t = c x + s z ; z' = -conj(s) x + c z
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

int blas_hessenberg_solve(const double2* H, int ldh, int m, const double2* beta2, double2* y, cudaStream_t s) {
  if (m > 32) return MG_ERR_ARG;
  hessenberg_solve_kernel<<<1, 32, 0, s>>>(H, ldh, m, beta2, y); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
