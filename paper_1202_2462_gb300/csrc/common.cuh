// Shared device helpers of the SAP-multilevel library: complex arithmetic in
// the compute precision, loads/stores through the storage types, the lattice
// geometry of the internal blocked layout, and error checking.
//
// Internal blocked layout (every fine field):
//   * the lattice (Lx, Ly, Lz, Lt) is cut into 4^4 blocks, block index
//     blk = bx + nb0*(by + nb1*(bz + nb2*bt)); inside a block the local index is
//     loc = lx + 4*(ly + 4*(lz + 4*lt)) (256 sites);
//   * spinor fields are structure-of-arrays per block: complex component c
//     (c = spin*3 + colour) of site (blk, loc) sits at (blk*12 + c)*256 + loc;
//   * links: U_mu(x) entry (a, b) at ((blk*4 + mu)*9 + a*3 + b)*256 + loc;
//   * clover: two 6x6 Hermitian chiral blocks per site stored as 18 complex
//     slots each (slots 0-2: the real diagonal in pairs, slots 3-17: the upper
//     off-diagonals (0,1),(0,2),...,(4,5)), slot q of chirality chi at
//     ((blk*36 + chi*18 + q)*256 + loc).
// The 4^4 blocks are both the Schwarz blocks and the first-level aggregates.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "debug.cuh"

namespace sapmg {

// ---------------------------------------------------------------- complex
template <class R> struct Cplx { R re, im; };

template <class R> __host__ __device__ __forceinline__ Cplx<R> cmk(R a, R b) { Cplx<R> c; c.re = a; c.im = b; return c; }
template <class R> __device__ __forceinline__ Cplx<R> operator+(Cplx<R> a, Cplx<R> b) { return cmk(a.re + b.re, a.im + b.im); }
template <class R> __device__ __forceinline__ Cplx<R> operator-(Cplx<R> a, Cplx<R> b) { return cmk(a.re - b.re, a.im - b.im); }
template <class R> __device__ __forceinline__ Cplx<R> operator*(Cplx<R> a, Cplx<R> b) {
  return cmk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> __device__ __forceinline__ Cplx<R> operator*(R s, Cplx<R> a) { return cmk(s * a.re, s * a.im); }
template <class R> __device__ __forceinline__ Cplx<R> conj(Cplx<R> a) { return cmk(a.re, -a.im); }
// conj(a) * b
template <class R> __device__ __forceinline__ Cplx<R> cdot(Cplx<R> a, Cplx<R> b) {
  return cmk(a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re);
}
// i * a and -i * a
template <class R> __device__ __forceinline__ Cplx<R> mul_i(Cplx<R> a) { return cmk(-a.im, a.re); }
template <class R> __device__ __forceinline__ Cplx<R> mul_mi(Cplx<R> a) { return cmk(a.im, -a.re); }
template <class R> __device__ __forceinline__ void cfma(Cplx<R>& acc, Cplx<R> a, Cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <class R> __device__ __forceinline__ void cfma_conj(Cplx<R>& acc, Cplx<R> a, Cplx<R> b) {
  acc.re = fma(a.re, b.re, acc.re); acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im); acc.im = fma(-a.im, b.re, acc.im);
}

// ---------------------------------------------------------------- storage
// Storage types hold one complex number: double2, float2, __half2, __nv_bfloat162.
template <class R, class S> struct Io;
template <class R> struct Io<R, double2> {
  static __device__ __forceinline__ Cplx<R> ld(const double2* p) { double2 v = __ldg(p); return cmk<R>((R)v.x, (R)v.y); }
  static __device__ __forceinline__ Cplx<R> ldc(const double2* p) { double2 v = *p; return cmk<R>((R)v.x, (R)v.y); }
  static __device__ __forceinline__ void st(double2* p, Cplx<R> c) { *p = make_double2((double)c.re, (double)c.im); }
};
template <class R> struct Io<R, float2> {
  static __device__ __forceinline__ Cplx<R> ld(const float2* p) { float2 v = __ldg(p); return cmk<R>((R)v.x, (R)v.y); }
  static __device__ __forceinline__ Cplx<R> ldc(const float2* p) { float2 v = *p; return cmk<R>((R)v.x, (R)v.y); }
  static __device__ __forceinline__ void st(float2* p, Cplx<R> c) { *p = make_float2((float)c.re, (float)c.im); }
};
// Half-precision loads go through 32-bit integer loads and value conversions
// (no address-taken temporaries, which would end up in local memory under
// register pressure).
__device__ __forceinline__ float2 half2_bits_to_float2(unsigned int u) {
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}
__device__ __forceinline__ float2 bf162_bits_to_float2(unsigned int u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}
template <class R> struct Io<R, __half2> {
  static __device__ __forceinline__ Cplx<R> ld(const __half2* p) {
    float2 v = half2_bits_to_float2(__ldg(reinterpret_cast<const unsigned int*>(p)));
    return cmk<R>((R)v.x, (R)v.y);
  }
  static __device__ __forceinline__ Cplx<R> ldc(const __half2* p) { float2 v = __half22float2(*p); return cmk<R>((R)v.x, (R)v.y); }
  static __device__ __forceinline__ void st(__half2* p, Cplx<R> c) { *p = __floats2half2_rn((float)c.re, (float)c.im); }
};
template <class R> struct Io<R, __nv_bfloat162> {
  static __device__ __forceinline__ Cplx<R> ld(const __nv_bfloat162* p) {
    float2 v = bf162_bits_to_float2(__ldg(reinterpret_cast<const unsigned int*>(p)));
    return cmk<R>((R)v.x, (R)v.y);
  }
  static __device__ __forceinline__ Cplx<R> ldc(const __nv_bfloat162* p) { float2 v = __bfloat1622float2(*p); return cmk<R>((R)v.x, (R)v.y); }
  static __device__ __forceinline__ void st(__nv_bfloat162* p, Cplx<R> c) { *p = __floats2bfloat162_rn((float)c.re, (float)c.im); }
};

// ---------------------------------------------------------------- geometry
struct Geom {
  int L[4];        // Lx, Ly, Lz, Lt
  int nb[4];       // 4^4 blocks per direction
  int bstride[4];  // block-index stride per direction
  int nblocks;
  long long V;
};

__host__ inline Geom make_geom(const int dims[4]) {
  Geom g;
  int s = 1;
  for (int mu = 0; mu < 4; ++mu) {
    g.L[mu] = dims[mu];
    g.nb[mu] = dims[mu] / 4;
    g.bstride[mu] = s;
    s *= g.nb[mu];
  }
  g.nblocks = s;
  g.V = (long long)s * 256;
  return g;
}

__device__ __forceinline__ int loc_stride(int mu) { return 1 << (2 * mu); }

// Block coordinate of block index blk in direction mu.
__device__ __forceinline__ int block_coord(const Geom& g, int blk, int mu) {
  return (blk / g.bstride[mu]) % g.nb[mu];
}

// Neighbour (blk', loc') of (blk, loc) one step in direction mu (step = +1 / -1).
__device__ __forceinline__ void neighbour_unchecked(const Geom& g, int blk, int loc, int mu, int step, int& nblk,
                                                    int& nloc) {
  const int ls = loc_stride(mu);
  const int c = (loc >> (2 * mu)) & 3;
  if (step > 0) {
    if (c < 3) { nblk = blk; nloc = loc + ls; return; }
    const int bc = block_coord(g, blk, mu);
    nblk = blk + (bc == g.nb[mu] - 1 ? -(g.nb[mu] - 1) : 1) * g.bstride[mu];
    nloc = loc - 3 * ls;
  } else {
    if (c > 0) { nblk = blk; nloc = loc - ls; return; }
    const int bc = block_coord(g, blk, mu);
    nblk = blk + (bc == 0 ? (g.nb[mu] - 1) : -1) * g.bstride[mu];
    nloc = loc + 3 * ls;
  }
}
__device__ __forceinline__ void neighbour(const Geom& g, int blk, int loc, int mu, int step, int& nblk, int& nloc) {
  neighbour_unchecked(g, blk, loc, mu, step, nblk, nloc);
#ifdef MG_DEBUG
  nblk = MG_CLAMP(kNeighbourBlock, nblk, g.nblocks);
  nloc = MG_CLAMP(kNeighbourSite, nloc, 256);
#endif
}

// The k-th block of colour c ((bx+by+bz+bt) mod 2 == c); nb[0] is even.
__device__ __forceinline__ int colour_block(const Geom& g, int k, int colour) {
  k = MG_CLAMP(kColourBlock, k, g.nblocks >> 1);
  const int half = g.nb[0] >> 1;
  const int j = k % half;
  const int rest = k / half;               // = by + nb1*(bz + nb2*bt)
  const int by = rest % g.nb[1];
  const int bz = (rest / g.nb[1]) % g.nb[2];
  const int bt = rest / (g.nb[1] * g.nb[2]);
  const int bx = 2 * j + ((by + bz + bt + colour) & 1);
  const int blk = bx + g.nb[0] * rest;
  return MG_CLAMP(kColourBlock, blk, g.nblocks);
}

// Canonical site index of (blk, loc).
__device__ __forceinline__ long long canonical_site(const Geom& g, int blk, int loc) {
  long long x = (long long)block_coord(g, blk, 0) * 4 + (loc & 3);
  long long y = (long long)block_coord(g, blk, 1) * 4 + ((loc >> 2) & 3);
  long long z = (long long)block_coord(g, blk, 2) * 4 + ((loc >> 4) & 3);
  long long t = (long long)block_coord(g, blk, 3) * 4 + ((loc >> 6) & 3);
  return ((t * g.L[2] + z) * g.L[1] + y) * g.L[0] + x;
}

// ---------------------------------------------------------------- reductions
template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace sapmg

// ---------------------------------------------------------------- errors
#define SAPMG_CUDA_TRY(expr)                                  \
  do {                                                        \
    cudaError_t err__ = (expr);                               \
    if (err__ != cudaSuccess) {                               \
      sapmg::set_last_error(cudaGetErrorString(err__), __FILE__, __LINE__); \
      return MG_ERR_CUDA;                                     \
    }                                                         \
  } while (0)

namespace sapmg {
void set_last_error(const char* msg, const char* file, int line);
// Count of kernel launches issued by the library (diagnostics).
void count_launches(int n);
// Running total of the algorithmic bytes (distinct operands read + results
// written) of the vector kernels, for their roofline.
void count_bytes(double bytes);
long long bytes_counted();
}
