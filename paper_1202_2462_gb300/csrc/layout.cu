// Field layouts and set-up kernels: gauge packing, the clover term (K9),
// storage-precision conversion, spinor pack/unpack between the canonical and
// the blocked layout, and the counter-based draw of random test vectors.
#include "internal.h"

namespace sapmg {

// ------------------------------------------------------------ coordinates
struct Coord { int x[4]; };

__device__ __forceinline__ Coord canon_coord(const Geom& g, long long s) {
  Coord c;
  c.x[0] = (int)(s % g.L[0]); s /= g.L[0];
  c.x[1] = (int)(s % g.L[1]); s /= g.L[1];
  c.x[2] = (int)(s % g.L[2]); s /= g.L[2];
  c.x[3] = (int)s;
  return c;
}

__device__ __forceinline__ long long canon_index(const Geom& g, const Coord& c) {
  return (((long long)c.x[3] * g.L[2] + c.x[2]) * g.L[1] + c.x[1]) * g.L[0] + c.x[0];
}

__device__ __forceinline__ void blocked_of(const Geom& g, const Coord& c, int& blk, int& loc) {
  blk = (c.x[0] >> 2) + g.nb[0] * ((c.x[1] >> 2) + g.nb[1] * ((c.x[2] >> 2) + g.nb[2] * (c.x[3] >> 2)));
  loc = (c.x[0] & 3) + 4 * ((c.x[1] & 3) + 4 * ((c.x[2] & 3) + 4 * (c.x[3] & 3)));
  blk = MG_CLAMP(kBlock, blk, g.nblocks);
}

__device__ __forceinline__ long long shifted(const Geom& g, Coord c, int mu, int step) {
  c.x[mu] = (c.x[mu] + step + g.L[mu]) % g.L[mu];
  return MG_CLAMP(kNeighbourSite, canon_index(g, c), g.V);
}

// ------------------------------------------------------------ gauge packing
template <class TG>
__global__ void pack_gauge_kernel(const double2* __restrict__ Uc, TG* __restrict__ Ub, Geom g, int antiperiodic_t) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V * 4) return;
  const long long s = i >> 2;
  const int mu = (int)(i & 3);
  Coord c = canon_coord(g, s);
  int blk, loc;
  blocked_of(g, c, blk, loc);
  const double sign = (antiperiodic_t && mu == 3 && c.x[3] == g.L[3] - 1) ? -1.0 : 1.0;
  const double2* src = Uc + i * 9;
  TG* dst = Ub + ((size_t)(blk * 4 + mu) * 9) * 256 + loc;
  for (int k = 0; k < 9; ++k) {
    double2 v = src[k];
    Io<double, TG>::st(dst + k * 256, cmk(sign * v.x, sign * v.y));
  }
}

int launch_pack_gauge(int prec, const Geom& g, const double* Uc, void* Ub, int antiperiodic_t, cudaStream_t s) {
  const long long n = g.V * 4;
  const int th = 256;
  const unsigned nb = (unsigned)((n + th - 1) / th);
  const double2* u = (const double2*)Uc;
  switch (prec) {
    case P64: pack_gauge_kernel<double2><<<nb, th, 0, s>>>(u, (double2*)Ub, g, antiperiodic_t); count_launches(1); break;
    case P32: pack_gauge_kernel<float2><<<nb, th, 0, s>>>(u, (float2*)Ub, g, antiperiodic_t); count_launches(1); break;
    case P16: pack_gauge_kernel<__half2><<<nb, th, 0, s>>>(u, (__half2*)Ub, g, antiperiodic_t); count_launches(1); break;
    case PBF: pack_gauge_kernel<__nv_bfloat162><<<nb, th, 0, s>>>(u, (__nv_bfloat162*)Ub, g, antiperiodic_t); count_launches(1); break;
    default: return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// ------------------------------------------------------------ clover term (K9)
struct M3 { Cplx<double> e[9]; };

__device__ __forceinline__ M3 ld_link(const double2* Uc, long long s, int mu) {
  M3 m;
  const double2* p = Uc + (s * 4 + mu) * 9;
  for (int k = 0; k < 9; ++k) { double2 v = p[k]; m.e[k] = cmk(v.x, v.y); }
  return m;
}
__device__ __forceinline__ M3 mm(const M3& a, const M3& b) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Cplx<double> acc = a.e[i * 3] * b.e[j];
      cfma(acc, a.e[i * 3 + 1], b.e[3 + j]);
      cfma(acc, a.e[i * 3 + 2], b.e[6 + j]);
      c.e[i * 3 + j] = acc;
    }
  return c;
}
__device__ __forceinline__ M3 dag(const M3& a) {
  M3 c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.e[i * 3 + j] = conj(a.e[j * 3 + i]);
  return c;
}
__device__ __forceinline__ M3 madd(const M3& a, const M3& b) {
  M3 c;
  for (int k = 0; k < 9; ++k) c.e[k] = a.e[k] + b.e[k];
  return c;
}

// G = c_sw (i/2) Fhat with Fhat = (Q - Q^dagger)/8, Q the four same-sense mu-nu leaves at x.
__device__ M3 clover_g(const double2* Uc, const Geom& g, const Coord& c, int mu, int nu, double csw) {
  const long long x = canon_index(g, c);
  const long long xpm = shifted(g, c, mu, 1), xpn = shifted(g, c, nu, 1);
  const long long xmm = shifted(g, c, mu, -1), xmn = shifted(g, c, nu, -1);
  Coord cm = c; cm.x[mu] = (c.x[mu] - 1 + g.L[mu]) % g.L[mu];
  const long long xmm_pn = shifted(g, cm, nu, 1), xmm_mn = shifted(g, cm, nu, -1);
  Coord cn = c; cn.x[nu] = (c.x[nu] - 1 + g.L[nu]) % g.L[nu];
  const long long xmn_pm = shifted(g, cn, mu, 1);
  // leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x
  M3 q = mm(mm(ld_link(Uc, x, mu), ld_link(Uc, xpm, nu)), mm(dag(ld_link(Uc, xpn, mu)), dag(ld_link(Uc, x, nu))));
  // leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x
  q = madd(q, mm(mm(ld_link(Uc, x, nu), dag(ld_link(Uc, xmm_pn, mu))), mm(dag(ld_link(Uc, xmm, nu)), ld_link(Uc, xmm, mu))));
  // leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x
  q = madd(q, mm(mm(dag(ld_link(Uc, xmm, mu)), dag(ld_link(Uc, xmm_mn, nu))), mm(ld_link(Uc, xmm_mn, mu), ld_link(Uc, xmn, nu))));
  // leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x
  q = madd(q, mm(mm(dag(ld_link(Uc, xmn, nu)), ld_link(Uc, xmn, mu)), mm(ld_link(Uc, xmn_pm, nu), dag(ld_link(Uc, x, mu)))));
  M3 G;
  // (i/2) c_sw (Q - Q^dagger)/8
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      Cplx<double> f = (1.0 / 8.0) * (q.e[i * 3 + j] - conj(q.e[j * 3 + i]));
      G.e[i * 3 + j] = (0.5 * csw) * mul_i(f);
    }
  return G;
}

// In the chiral basis sigma_{mu nu} = diag(s+, s-) with 2x2 blocks
//   xy: -s3, -s3   xz: s2, s2   yz: -s1, -s1   xt: s1, -s1   yt: s2, -s2   zt: s3, -s3
// so chirality block chi of the clover sum is sum_k s_k (x) B_k^chi with
//   B1 = G_xt - G_yz (+), -G_yz - G_xt (-);  B2 = G_xz + G_yt (+), G_xz - G_yt (-);
//   B3 = G_zt - G_xy (+), -G_xy - G_zt (-)
// and s1 (x) B1 + s2 (x) B2 + s3 (x) B3 = [[B3, B1 - i B2], [B1 + i B2, -B3]].
__global__ void clover_build_kernel(const double2* __restrict__ Uc, double2* __restrict__ Ab, Geom g, double diag,
                                    double csw) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Coord c = canon_coord(g, s);
  int blk, loc;
  blocked_of(g, c, blk, loc);
  const M3 gxy = clover_g(Uc, g, c, 0, 1, csw), gxz = clover_g(Uc, g, c, 0, 2, csw);
  const M3 gyz = clover_g(Uc, g, c, 1, 2, csw), gxt = clover_g(Uc, g, c, 0, 3, csw);
  const M3 gyt = clover_g(Uc, g, c, 1, 3, csw), gzt = clover_g(Uc, g, c, 2, 3, csw);
  for (int chi = 0; chi < 2; ++chi) {
    const double sg = chi == 0 ? 1.0 : -1.0;
    Cplx<double> m[36];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const int k = i * 3 + j;
        const Cplx<double> b1 = sg * gxt.e[k] - gyz.e[k];
        const Cplx<double> b2 = gxz.e[k] + sg * gyt.e[k];
        const Cplx<double> b3 = sg * gzt.e[k] - gxy.e[k];
        m[i * 6 + j] = b3;
        m[(3 + i) * 6 + (3 + j)] = cmk(-b3.re, -b3.im);
        m[i * 6 + 3 + j] = b1 - mul_i(b2);
        m[(3 + i) * 6 + j] = b1 + mul_i(b2);
      }
    double2* a = Ab + ((size_t)(blk * 36 + chi * 18)) * 256 + loc;
    for (int q = 0; q < 3; ++q)
      a[q * 256] = make_double2(diag + m[(2 * q) * 6 + 2 * q].re, diag + m[(2 * q + 1) * 6 + 2 * q + 1].re);
    int q = 3;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j, ++q) a[q * 256] = make_double2(m[i * 6 + j].re, m[i * 6 + j].im);
  }
}

int launch_clover_build(const Geom& g, const double* Uc, void* Ab64, double m0, double c_sw, cudaStream_t s) {
  const int th = 128;
  clover_build_kernel<<<(unsigned)((g.V + th - 1) / th), th, 0, s>>>((const double2*)Uc, (double2*)Ab64, g,
                                                                     4.0 + m0, c_sw); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Dense export of the blocked FP64 clover: [V][chi][6][6] complex, canonical order.
__global__ void clover_export_kernel(const double2* __restrict__ Ab, double2* __restrict__ out, Geom g) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Coord c = canon_coord(g, s);
  int blk, loc;
  blocked_of(g, c, blk, loc);
  for (int chi = 0; chi < 2; ++chi) {
    const double2* a = Ab + ((size_t)(blk * 36 + chi * 18)) * 256 + loc;
    double2* o = out + (s * 2 + chi) * 36;
    for (int q = 0; q < 3; ++q) {
      double2 d = a[q * 256];
      o[(2 * q) * 6 + 2 * q] = make_double2(d.x, 0.0);
      o[(2 * q + 1) * 6 + 2 * q + 1] = make_double2(d.y, 0.0);
    }
    int q = 3;
    for (int i = 0; i < 6; ++i)
      for (int j = i + 1; j < 6; ++j, ++q) {
        double2 v = a[q * 256];
        o[i * 6 + j] = v;
        o[j * 6 + i] = make_double2(v.x, -v.y);
      }
  }
}

int launch_clover_export(const Geom& g, const void* Ab64, double* out, cudaStream_t s) {
  const int th = 128;
  clover_export_kernel<<<(unsigned)((g.V + th - 1) / th), th, 0, s>>>((const double2*)Ab64, (double2*)out, g); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// ------------------------------------------------------------ conversion
template <class TI, class TO>
__global__ void convert_kernel(const TI* __restrict__ in, TO* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    Io<double, TO>::st(out + i, Io<double, TI>::ld(in + i));
}

template <class TI>
static int convert_from(const TI* in, int to, void* out, size_t n, cudaStream_t s) {
  const int th = 256;
  const unsigned nb = (unsigned)std::min<size_t>((n + th - 1) / th, 152 * 64);
  switch (to) {
    case P64: convert_kernel<TI, double2><<<nb, th, 0, s>>>(in, (double2*)out, n); count_launches(1); break;
    case P32: convert_kernel<TI, float2><<<nb, th, 0, s>>>(in, (float2*)out, n); count_launches(1); break;
    case P16: convert_kernel<TI, __half2><<<nb, th, 0, s>>>(in, (__half2*)out, n); count_launches(1); break;
    case PBF: convert_kernel<TI, __nv_bfloat162><<<nb, th, 0, s>>>(in, (__nv_bfloat162*)out, n); count_launches(1); break;
    default: return MG_ERR_ARG;
  }
  return MG_OK;
}

int launch_convert(int from, const void* in, int to, void* out, size_t n_complex, cudaStream_t s) {
  if (n_complex == 0) return MG_OK;
  int rc;
  switch (from) {
    case P64: rc = convert_from((const double2*)in, to, out, n_complex, s); break;
    case P32: rc = convert_from((const float2*)in, to, out, n_complex, s); break;
    case P16: rc = convert_from((const __half2*)in, to, out, n_complex, s); break;
    case PBF: rc = convert_from((const __nv_bfloat162*)in, to, out, n_complex, s); break;
    default: return MG_ERR_ARG;
  }
  if (rc) return rc;
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// ------------------------------------------------------------ spinor layouts
// canonical [r][site][12] <-> blocked [r][blk][12][256]
template <class TI, class TO>
__global__ void pack_spinor_kernel(const TI* __restrict__ in, TO* __restrict__ out, Geom g, int nrhs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V * nrhs) return;
  const long long r = i / g.V, s = i % g.V;
  Coord c = canon_coord(g, s);
  int blk, loc;
  blocked_of(g, c, blk, loc);
  const TI* src = in + (r * g.V + s) * 12;
  TO* dst = out + r * g.V * 12 + ((size_t)blk * 12) * 256 + loc;
  for (int k = 0; k < 12; ++k) Io<double, TO>::st(dst + k * 256, Io<double, TI>::ldc(src + k));
}

template <class TI, class TO>
__global__ void unpack_spinor_kernel(const TI* __restrict__ in, TO* __restrict__ out, Geom g, int nrhs) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V * nrhs) return;
  const long long r = i / g.V, s = i % g.V;
  Coord c = canon_coord(g, s);
  int blk, loc;
  blocked_of(g, c, blk, loc);
  const TI* src = in + r * g.V * 12 + ((size_t)blk * 12) * 256 + loc;
  TO* dst = out + (r * g.V + s) * 12;
  for (int k = 0; k < 12; ++k) Io<double, TO>::st(dst + k, Io<double, TI>::ldc(src + k * 256));
}

template <class TI, class TO>
static void layout_launch(bool pack, unsigned nb, int th, const void* in, void* out, const Geom& g, int nrhs,
                          cudaStream_t s) {
  if (pack) { pack_spinor_kernel<TI, TO><<<nb, th, 0, s>>>((const TI*)in, (TO*)out, g, nrhs); count_launches(1); }
  else { unpack_spinor_kernel<TI, TO><<<nb, th, 0, s>>>((const TI*)in, (TO*)out, g, nrhs); count_launches(1); }
}

static int layout_dispatch(bool pack, int pin, const void* in, int pout, void* out, const Geom& g, int nrhs,
                           cudaStream_t s) {
  const long long n = g.V * nrhs;
  const int th = 128;
  const unsigned nb = (unsigned)((n + th - 1) / th);
  if (n == 0) return MG_OK;
  if (pin == P64 && pout == P64) layout_launch<double2, double2>(pack, nb, th, in, out, g, nrhs, s);
  else if (pin == P64 && pout == P32) layout_launch<double2, float2>(pack, nb, th, in, out, g, nrhs, s);
  else if (pin == P32 && pout == P64) layout_launch<float2, double2>(pack, nb, th, in, out, g, nrhs, s);
  else if (pin == P32 && pout == P32) layout_launch<float2, float2>(pack, nb, th, in, out, g, nrhs, s);
  else return MG_ERR_ARG;
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_pack_spinor(int pin, const void* canon, int pout, void* blocked, const Geom& g, int nrhs, cudaStream_t s) {
  return layout_dispatch(true, pin, canon, pout, blocked, g, nrhs, s);
}
int launch_unpack_spinor(int pin, const void* blocked, int pout, void* canon, const Geom& g, int nrhs,
                         cudaStream_t s) {
  return layout_dispatch(false, pin, blocked, pout, canon, g, nrhs, s);
}

// ------------------------------------------------------------ random test vectors
// SplitMix64 (Steele, Lea, Flood 2014): golden-ratio increment, then xor-shift-
// multiply rounds with shifts 30, 27, 31.  Value i of stream (seed, stream) is
// mix(mix(mix(seed) + stream) + i); uniform in [-1, 1) as (u >> 11) 2^-52 - 1,
// exactly representable, so host and device draws agree bit for bit.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void draw_vectors_kernel(double2* __restrict__ out, Geom g, int nvec, uint64_t key) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V * nvec) return;
  const long long k = i / g.V, s = i % g.V;
  Coord c = canon_coord(g, s);
  int blk, loc;
  blocked_of(g, c, blk, loc);
  double2* dst = out + k * g.V * 12 + ((size_t)blk * 12) * 256 + loc;
  for (int q = 0; q < 12; ++q) {
    const uint64_t base = (uint64_t)(((k * g.V + s) * 12 + q) * 2);
    const double re = (double)(splitmix64(key + base) >> 11) * 0x1.0p-52 - 1.0;
    const double im = (double)(splitmix64(key + base + 1) >> 11) * 0x1.0p-52 - 1.0;
    dst[q * 256] = make_double2(re, im);
  }
}

uint64_t host_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int launch_draw_vectors(const Geom& g, void* out64, int nvec, unsigned long long seed, unsigned long long stream,
                        cudaStream_t s) {
  const uint64_t key = host_splitmix64(host_splitmix64(seed) + stream);
  const long long n = g.V * nvec;
  const int th = 128;
  draw_vectors_kernel<<<(unsigned)((n + th - 1) / th), th, 0, s>>>((double2*)out64, g, nvec, key); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
