// K2, paired form: one colour pass of red-black Schwarz (Sec. 2, Algorithm 1)
// for two right-hand sides per thread, FP32 arithmetic on FP32/FP16/BF16
// fields.
//
// For every block i of colour c and every pair (r, r+1) of right-hand sides:
//   rho = b - D z on the block's sites (halo z from the neighbouring blocks),
//   n_MR minimal-residual steps on D_i e = rho with the Dirichlet block
//   operator D_i (hops leaving the block dropped):
//     p = D_i rho, alpha = <p, rho>/<p, p>, e += alpha rho, rho -= alpha p,
//   z += e.
// The arithmetic is the single-pair kernel's (sap.cu), reorganised for the
// issue and load limits of sm_103a:
//   * every value is a pair (right-hand side r, right-hand side r+1) and every
//     add, multiply and FMA is the packed two-wide FP32 instruction, so one
//     issue slot does the work of two;
//   * a link or clover entry is loaded and converted once for both right-hand
//     sides (a broadcast pair), halving the field traffic through L1;
//   * the -1/2 of the hopping term is folded into the reconstruction FMAs, so
//     p = A rho - 1/2 sum(hops) needs no separate scaling pass;
//   * the last MR step adds alpha rho straight into z (no write of the last
//     rho or e); the first writes e = alpha rho without reading e.
// Shared memory holds rho and e of the block for the pair, one 16-byte word
// (re_r, re_r+1, im_r, im_r+1) per site and spin-colour component.
#include "internal.h"
#include "stencil.cuh"

namespace sapmg {
namespace {

struct P2 { float2 re, im; };                      // one complex component for two right-hand sides
struct B2 { float2 r, i, ni; };                    // a broadcast complex field entry: (re,re), (im,im), (-im,-im)

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one FMA with an exact product: b * (-1) + a
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, f2(-1.f), a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

template <int SG> __device__ __forceinline__ float2 addsg(float2 a, float2 b) { return SG > 0 ? add2(a, b) : sub2(a, b); }

// Field entries (links, clover) in storage type TG as a broadcast pair.
template <class TG> struct Fld;
template <> struct Fld<__nv_bfloat162> {
  static __device__ __forceinline__ B2 ld(const __nv_bfloat162* p) {
    const unsigned w = __ldg(reinterpret_cast<const unsigned*>(p));
    const float re = __uint_as_float(w << 16), im = __uint_as_float(w & 0xffff0000u);
    B2 b; b.r = f2(re); b.i = f2(im); b.ni = f2(-im); return b;
  }
};
template <> struct Fld<__half2> {
  static __device__ __forceinline__ B2 ld(const __half2* p) {
    const float2 v = half2_bits_to_float2(__ldg(reinterpret_cast<const unsigned*>(p)));
    B2 b; b.r = f2(v.x); b.i = f2(v.y); b.ni = f2(-v.y); return b;
  }
};
template <> struct Fld<float2> {
  static __device__ __forceinline__ B2 ld(const float2* p) {
    const float2 v = __ldg(p);
    B2 b; b.r = f2(v.x); b.i = f2(v.y); b.ni = f2(-v.y); return b;
  }
};

// acc = u h, acc += u h, acc += conj(u) h
__device__ __forceinline__ P2 cmul(const B2& u, const P2& h) {
  P2 a;
  a.re = fma2(u.ni, h.im, mul2(u.r, h.re));
  a.im = fma2(u.i, h.re, mul2(u.r, h.im));
  return a;
}
__device__ __forceinline__ void cmac(P2& a, const B2& u, const P2& h) {
  a.re = fma2(u.r, h.re, a.re); a.re = fma2(u.ni, h.im, a.re);
  a.im = fma2(u.r, h.im, a.im); a.im = fma2(u.i, h.re, a.im);
}
__device__ __forceinline__ P2 cmul_conj(const B2& u, const P2& h) {
  P2 a;
  a.re = fma2(u.i, h.im, mul2(u.r, h.re));
  a.im = fma2(u.ni, h.re, mul2(u.r, h.im));
  return a;
}
__device__ __forceinline__ void cmac_conj(P2& a, const B2& u, const P2& h) {
  a.re = fma2(u.r, h.re, a.re); a.re = fma2(u.i, h.im, a.re);
  a.im = fma2(u.r, h.im, a.im); a.im = fma2(u.ni, h.re, a.im);
}

// Spin projection h = psi_u + S X_MU psi_l (X_MU as in stencil.cuh), reading
// components through ld(c).
template <int MU, int S, class LD>
__device__ __forceinline__ void project2(LD ld, P2 (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const P2 l0 = ld(6 + c), l1 = ld(9 + c), u0 = ld(c), u1 = ld(3 + c);
    P2 a, b;
    if (MU == 0) {            // x0 = -i l1, x1 = -i l0
      a.re = addsg<S>(u0.re, l1.im); a.im = addsg<-S>(u0.im, l1.re);
      b.re = addsg<S>(u1.re, l0.im); b.im = addsg<-S>(u1.im, l0.re);
    } else if (MU == 1) {     // x0 = -l1, x1 = l0
      a.re = addsg<-S>(u0.re, l1.re); a.im = addsg<-S>(u0.im, l1.im);
      b.re = addsg<S>(u1.re, l0.re); b.im = addsg<S>(u1.im, l0.im);
    } else if (MU == 2) {     // x0 = -i l0, x1 = i l1
      a.re = addsg<S>(u0.re, l0.im); a.im = addsg<-S>(u0.im, l0.re);
      b.re = addsg<-S>(u1.re, l1.im); b.im = addsg<S>(u1.im, l1.re);
    } else {                  // x0 = l0, x1 = l1
      a.re = addsg<S>(u0.re, l0.re); a.im = addsg<S>(u0.im, l0.im);
      b.re = addsg<S>(u1.re, l1.re); b.im = addsg<S>(u1.im, l1.im);
    }
    h[c] = a;
    h[3 + c] = b;
  }
}

// acc_u[a] += k g0, acc_u[3+a] += k g1, acc_l += k S X_MU^dagger (g0, g1) for colour a,
// with k = -1/2 (the hopping term's coefficient): kp = (k, k), km = (-k, -k).
template <int MU, int S>
__device__ __forceinline__ void reconstruct2(const P2& g0, const P2& g1, int a, P2 (&acc)[12]) {
  const float2 kp = f2(-0.5f), km = f2(0.5f);
  acc[a].re = fma2(g0.re, kp, acc[a].re); acc[a].im = fma2(g0.im, kp, acc[a].im);
  acc[3 + a].re = fma2(g1.re, kp, acc[3 + a].re); acc[3 + a].im = fma2(g1.im, kp, acc[3 + a].im);
  // the lower components receive S * X^dagger g scaled by k; k S = -S/2
  const float2 ks = S > 0 ? kp : km, nks = S > 0 ? km : kp;
  P2& l0 = acc[6 + a];
  P2& l1 = acc[9 + a];
  if (MU == 0) {              // x0 = i g1, x1 = i g0
    l0.re = fma2(g1.im, nks, l0.re); l0.im = fma2(g1.re, ks, l0.im);
    l1.re = fma2(g0.im, nks, l1.re); l1.im = fma2(g0.re, ks, l1.im);
  } else if (MU == 1) {       // x0 = g1, x1 = -g0
    l0.re = fma2(g1.re, ks, l0.re); l0.im = fma2(g1.im, ks, l0.im);
    l1.re = fma2(g0.re, nks, l1.re); l1.im = fma2(g0.im, nks, l1.im);
  } else if (MU == 2) {       // x0 = i g0, x1 = -i g1
    l0.re = fma2(g0.im, nks, l0.re); l0.im = fma2(g0.re, ks, l0.im);
    l1.re = fma2(g1.im, ks, l1.re); l1.im = fma2(g1.re, nks, l1.im);
  } else {                    // x0 = g0, x1 = g1
    l0.re = fma2(g0.re, ks, l0.re); l0.im = fma2(g0.im, ks, l0.im);
    l1.re = fma2(g1.re, ks, l1.re); l1.im = fma2(g1.im, ks, l1.im);
  }
}

// One hop: acc += -1/2 (1 + S gamma_MU) W h, W = U_MU(x) (S = -1, forward) or
// U_MU(x - MU)^dagger (S = +1, backward); the link sits at (lblk, lloc).
template <int MU, int S, class TG, class LD>
__device__ __forceinline__ void hop2(LD ld, const TG* __restrict__ U, int lblk, int lloc, P2 (&acc)[12]) {
  P2 h[6];
  project2<MU, S>(ld, h);
  const TG* lp = U + ((size_t)(lblk * 4 + MU) * 9) * 256 + lloc;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P2 g0, g1;
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      // U h: row a of U; U^dagger h: column a, conjugated
      const B2 u = Fld<TG>::ld(lp + (S < 0 ? 3 * a + bb : 3 * bb + a) * 256);
      if (S < 0) {
        if (bb == 0) { g0 = cmul(u, h[0]); g1 = cmul(u, h[3]); }
        else { cmac(g0, u, h[bb]); cmac(g1, u, h[3 + bb]); }
      } else {
        if (bb == 0) { g0 = cmul_conj(u, h[0]); g1 = cmul_conj(u, h[3]); }
        else { cmac_conj(g0, u, h[bb]); cmac_conj(g1, u, h[3 + bb]); }
      }
    }
    reconstruct2<MU, S>(g0, g1, a, acc);
  }
}

// out = A psi for one chirality (two Hermitian 6x6 blocks, stored as in
// common.cuh: 3 slots of real diagonal pairs, then the 15 upper entries).
template <class TG>
__device__ __forceinline__ void clover2_chi(const TG* __restrict__ a, const P2 (&p)[6], P2 (&out)[6]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const B2 d = Fld<TG>::ld(a + q * 256);
    out[2 * q].re = mul2(d.r, p[2 * q].re); out[2 * q].im = mul2(d.r, p[2 * q].im);
    out[2 * q + 1].re = mul2(d.i, p[2 * q + 1].re); out[2 * q + 1].im = mul2(d.i, p[2 * q + 1].im);
  }
  int q = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j, ++q) {
      const B2 o = Fld<TG>::ld(a + q * 256);
      cmac(out[i], o, p[j]);
      cmac_conj(out[j], o, p[i]);
    }
}

__device__ __forceinline__ P2 lds2(const float4* __restrict__ s, int idx) {
  const float4 v = s[idx];
  P2 p; p.re = make_float2(v.x, v.y); p.im = make_float2(v.z, v.w); return p;
}
__device__ __forceinline__ void sts2(float4* __restrict__ s, int idx, const P2& p) {
  s[idx] = make_float4(p.re.x, p.re.y, p.im.x, p.im.y);
}
// a component of two right-hand sides in the global FP32 layout (r and r + 1 are 12 V apart)
__device__ __forceinline__ P2 ldg2(const float2* __restrict__ f, size_t stride, size_t idx) {
  const float2 a = f[idx], b = f[idx + stride];
  P2 p; p.re = make_float2(a.x, b.x); p.im = make_float2(a.y, b.y); return p;
}

template <int MU, class TG>
__device__ __forceinline__ void block_hops2(const TG* __restrict__ U, const float4* __restrict__ rs, int blk, int loc,
                                            P2 (&acc)[12]) {
  const int ls = 1 << (2 * MU);
  const int c = (loc >> (2 * MU)) & 3;
  if (c < 3) hop2<MU, -1>([&](int k) { return lds2(rs, k * 256 + loc + ls); }, U, blk, loc, acc);
  if (c > 0) hop2<MU, 1>([&](int k) { return lds2(rs, k * 256 + loc - ls); }, U, blk, loc - ls, acc);
}

template <int MU, class TG>
__device__ __forceinline__ void global_hops2(const Geom& g, const float2* __restrict__ z, size_t stride,
                                             const TG* __restrict__ U, int blk, int loc, P2 (&acc)[12]) {
  int nb, nl;
  neighbour(g, blk, loc, MU, 1, nb, nl);
  hop2<MU, -1>([&](int k) { return ldg2(z, stride, ((size_t)nb * 12 + k) * 256 + nl); }, U, blk, loc, acc);
  neighbour(g, blk, loc, MU, -1, nb, nl);
  hop2<MU, 1>([&](int k) { return ldg2(z, stride, ((size_t)nb * 12 + k) * 256 + nl); }, U, nb, nl, acc);
}

// p = A psi for the whole site, psi read component by component through ld
template <class TG, class LD>
__device__ __forceinline__ void clover2(const TG* __restrict__ A, int blk, int loc, LD ld, P2 (&out)[12]) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    P2 p[6], o[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = ld(chi * 6 + k);
    clover2_chi<TG>(A + ((size_t)(blk * 36 + chi * 18)) * 256 + loc, p, o);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[chi * 6 + k] = o[k];
  }
}

// Sum of six floats (three pairs) over the CTA: warp shuffles, one word per
// warp in shared memory, every thread adds the eight warps' words.
__device__ __forceinline__ void block_reduce6(float2& a, float2& b, float2& c, float4 (*red)[2]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a.x += __shfl_xor_sync(0xffffffffu, a.x, o); a.y += __shfl_xor_sync(0xffffffffu, a.y, o);
    b.x += __shfl_xor_sync(0xffffffffu, b.x, o); b.y += __shfl_xor_sync(0xffffffffu, b.y, o);
    c.x += __shfl_xor_sync(0xffffffffu, c.x, o); c.y += __shfl_xor_sync(0xffffffffu, c.y, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    red[w][0] = make_float4(a.x, a.y, b.x, b.y);
    red[w][1] = make_float4(c.x, c.y, 0.f, 0.f);
  }
  __syncthreads();
  float4 s0 = red[0][0], s1 = red[0][1];
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const float4 t0 = red[k][0], t1 = red[k][1];
    const float2 u = add2(make_float2(s0.x, s0.y), make_float2(t0.x, t0.y));
    const float2 v = add2(make_float2(s0.z, s0.w), make_float2(t0.z, t0.w));
    const float2 x = add2(make_float2(s1.x, s1.y), make_float2(t1.x, t1.y));
    s0 = make_float4(u.x, u.y, v.x, v.y);
    s1 = make_float4(x.x, x.y, 0.f, 0.f);
  }
  a = make_float2(s0.x, s0.y);
  b = make_float2(s0.z, s0.w);
  c = make_float2(s1.x, s1.y);
}

template <class TG, bool KEEP_RHO, int MINB>
__global__ void __launch_bounds__(256, MINB)
    sap_colour_pair_kernel(float2* __restrict__ z, const float2* __restrict__ b, const TG* __restrict__ U,
                           const TG* __restrict__ A, Geom g, int colour, int n_mr, int npairs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* rs = reinterpret_cast<float4*>(smem_raw);                      // rho [12][256]
  float4* es = rs + 12 * 256;                                            // e   [12][256]
  float4 (*red)[2] = reinterpret_cast<float4 (*)[2]>(es + 12 * 256);     // [8][2]
  const size_t stride = (size_t)g.V * 12;                                // one right-hand side
  const size_t off = (size_t)(blockIdx.x % npairs) * 2 * stride;
  z += off;
  b += off;
  const int blk = colour_block(g, blockIdx.x / npairs, colour);
  const int loc = threadIdx.x;
  const size_t site0 = (size_t)blk * 12 * 256 + loc;

  // rho = b - D z = b - A z + 1/2 sum(hops): acc = A z - 1/2 sum(hops), rho = b - acc
  {
    P2 acc[12];
    clover2<TG>(A, blk, loc, [&](int k) { return ldg2(z, stride, site0 + k * 256); }, acc);
    global_hops2<0>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<1>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<2>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<3>(g, z, stride, U, blk, loc, acc);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const P2 bb = ldg2(b, stride, site0 + c * 256);
      P2 r;
      r.re = sub2(bb.re, acc[c].re);
      r.im = sub2(bb.im, acc[c].im);
      sts2(rs, c * 256 + loc, r);
    }
  }

  for (int it = 0; it < n_mr; ++it) {
    __syncthreads();                                   // rho of every site written
    P2 p[12];
    clover2<TG>(A, blk, loc, [&](int k) { return lds2(rs, k * 256 + loc); }, p);
    block_hops2<0>(U, rs, blk, loc, p);
    asm volatile("" ::: "memory");
    block_hops2<1>(U, rs, blk, loc, p);
    asm volatile("" ::: "memory");
    block_hops2<2>(U, rs, blk, loc, p);
    asm volatile("" ::: "memory");
    block_hops2<3>(U, rs, blk, loc, p);
    // <p, rho> and <p, p> per right-hand side (KEEP_RHO: own rho stays in registers for the update)
    P2 ro[12];
    float2 pr_re = f2(0.f), pr_im = f2(0.f), pp = f2(0.f);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const P2 r = lds2(rs, c * 256 + loc);
      if (KEEP_RHO) ro[c] = r;
      pr_re = fma2(p[c].re, r.re, pr_re); pr_re = fma2(p[c].im, r.im, pr_re);
      pr_im = fma2(p[c].re, r.im, pr_im); pr_im = fma2(p[c].im, sub2(f2(0.f), r.re), pr_im);
      pp = fma2(p[c].re, p[c].re, pp); pp = fma2(p[c].im, p[c].im, pp);
    }
    block_reduce6(pr_re, pr_im, pp, red);             // its barrier follows every neighbour read of rho
    float2 al_re = f2(0.f), al_im = f2(0.f);
    if (pp.x > 0.f) { const float q = 1.f / pp.x; al_re.x = pr_re.x * q; al_im.x = pr_im.x * q; }
    if (pp.y > 0.f) { const float q = 1.f / pp.y; al_re.y = pr_re.y * q; al_im.y = pr_im.y * q; }
    const float2 nal_im = make_float2(-al_im.x, -al_im.y);
    const bool first = it == 0, last = it == n_mr - 1;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      if (!KEEP_RHO) ro[c] = lds2(rs, c * 256 + loc);
      // alpha rho and rho - alpha p
      P2 ar, rn;
      ar.re = fma2(nal_im, ro[c].im, mul2(al_re, ro[c].re));
      ar.im = fma2(al_im, ro[c].re, mul2(al_re, ro[c].im));
      P2 e = ar;
      if (!first) {
        const P2 eo = lds2(es, c * 256 + loc);
        e.re = add2(eo.re, ar.re); e.im = add2(eo.im, ar.im);
      }
      if (last) {
        // z += e on the block (own site only)
        const size_t i = site0 + c * 256;
        const float2 za = z[i], zb = z[i + stride];
        z[i] = make_float2(za.x + e.re.x, za.y + e.im.x);
        z[i + stride] = make_float2(zb.x + e.re.y, zb.y + e.im.y);
      } else {
        sts2(es, c * 256 + loc, e);
        rn.re = fma2(al_im, p[c].im, fma2(sub2(f2(0.f), al_re), p[c].re, ro[c].re));
        rn.im = fma2(nal_im, p[c].re, fma2(sub2(f2(0.f), al_re), p[c].im, ro[c].im));
        sts2(rs, c * 256 + loc, rn);
      }
    }
  }
  if (n_mr == 0) return;
}

template <class TG, bool KEEP_RHO, int MINB>
static int run_pair(const Geom& g, void* z, const void* b, const void* U, const void* A, int colour, int n_mr,
                    int nrhs, cudaStream_t s) {
  const size_t smem = sizeof(float4) * (24 * 256 + 16);
  static bool attr = false;
  if (!attr) {
    SAPMG_CUDA_TRY(cudaFuncSetAttribute(sap_colour_pair_kernel<TG, KEEP_RHO, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  const int npairs = nrhs / 2;
  sap_colour_pair_kernel<TG, KEEP_RHO, MINB><<<(unsigned)(g.nblocks / 2 * npairs), 256, smem, s>>>(
      (float2*)z, (const float2*)b, (const TG*)U, (const TG*)A, g, colour, n_mr, npairs);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace

int launch_sap_colour_pair(int prec, const Geom& g, void* z, const void* b, const void* U, const void* A, int colour,
                           int n_mr, int nrhs, cudaStream_t s, int shape) {
  if (nrhs < 2 || nrhs % 2 != 0 || n_mr < 1) return MG_ERR_ARG;
#define SAPMG_PAIR_CASE(T)                                                                   \
  return shape == 2 ? run_pair<T, true, 1>(g, z, b, U, A, colour, n_mr, nrhs, s)             \
       : shape == 1 ? run_pair<T, true, 2>(g, z, b, U, A, colour, n_mr, nrhs, s)             \
                    : run_pair<T, false, 2>(g, z, b, U, A, colour, n_mr, nrhs, s)
  switch (prec) {
    case P32: SAPMG_PAIR_CASE(float2);
    case P16: SAPMG_PAIR_CASE(__half2);
    case PBF: SAPMG_PAIR_CASE(__nv_bfloat162);
    default: return MG_ERR_ARG;
  }
#undef SAPMG_PAIR_CASE
}

}  // namespace sapmg
