// Arithmetic on pairs of right-hand sides for the clover-Wilson operator
// (Sec. 1, Eq. 1.1) in packed two-wide FP32: every value is a pair (right-hand
// side r, right-hand side r+1) and every add, multiply and FMA is one packed
// instruction (sm_100 and later); a link or clover entry, shared by the two
// right-hand sides, is a broadcast pair.  Gamma matrices, spin projection and
// the blocked layouts are those of stencil.cuh and common.cuh.  Used by the
// paired Schwarz kernels (sap2.cu) and the paired Dirac kernel (dirac2.cu).
#pragma once
#include "stencil.cuh"

namespace sapmg {
namespace pair {


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

// The same from a copy in shared memory (the block-resident kernel).
template <class TG> struct FldS;
template <> struct FldS<__nv_bfloat162> {
  static __device__ __forceinline__ B2 ld(const __nv_bfloat162* p) {
    const unsigned w = *reinterpret_cast<const unsigned*>(p);
    const float re = __uint_as_float(w << 16), im = __uint_as_float(w & 0xffff0000u);
    B2 b; b.r = f2(re); b.i = f2(im); b.ni = f2(-im); return b;
  }
};
template <> struct FldS<__half2> {
  static __device__ __forceinline__ B2 ld(const __half2* p) {
    const float2 v = half2_bits_to_float2(*reinterpret_cast<const unsigned*>(p));
    B2 b; b.r = f2(v.x); b.i = f2(v.y); b.ni = f2(-v.y); return b;
  }
};
template <> struct FldS<float2> {
  static __device__ __forceinline__ B2 ld(const float2* p) {
    const float2 v = *p;
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
// with k = -1/2 (the hopping term's coefficient; 0 drops the hop): kp = (k, k), km = (-k, -k).
template <int MU, int S>
__device__ __forceinline__ void reconstruct2(const P2& g0, const P2& g1, int a, P2 (&acc)[12], float k = -0.5f) {
  const float2 kp = f2(k), km = f2(-k);
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
// U_MU(x - MU)^dagger (S = +1, backward); fl(k) returns entry k = 3 a + b of
// that link as a broadcast pair, ld(c) component c of the neighbour.
template <int MU, int S, class LD, class FL>
__device__ __forceinline__ void hop2(LD ld, FL fl, P2 (&acc)[12], float k = -0.5f) {
  P2 h[6];
  project2<MU, S>(ld, h);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    P2 g0, g1;
#pragma unroll
    for (int bb = 0; bb < 3; ++bb) {
      // U h: row a of U; U^dagger h: column a, conjugated
      const B2 u = fl(S < 0 ? 3 * a + bb : 3 * bb + a);
      if (S < 0) {
        if (bb == 0) { g0 = cmul(u, h[0]); g1 = cmul(u, h[3]); }
        else { cmac(g0, u, h[bb]); cmac(g1, u, h[3 + bb]); }
      } else {
        if (bb == 0) { g0 = cmul_conj(u, h[0]); g1 = cmul_conj(u, h[3]); }
        else { cmac_conj(g0, u, h[bb]); cmac_conj(g1, u, h[3 + bb]); }
      }
    }
    reconstruct2<MU, S>(g0, g1, a, acc, k);
  }
}

// a link entry k of U_MU at (blk, loc) from global memory, and from the block's copy in shared memory
template <int MU, class TG>
struct LinkG {
  const TG* p;
  __device__ __forceinline__ LinkG(const TG* U, int blk, int loc) : p(U + ((size_t)(blk * 4 + MU) * 9) * 256 + loc) {}
  __device__ __forceinline__ B2 operator()(int k) const { return Fld<TG>::ld(p + k * 256); }
};
template <int MU, class TG>
struct LinkS {
  const TG* p;
  __device__ __forceinline__ LinkS(const TG* Us, int loc) : p(Us + (MU * 9) * 256 + loc) {}
  __device__ __forceinline__ B2 operator()(int k) const { return FldS<TG>::ld(p + k * 256); }
};

// out = A psi for one chirality (two Hermitian 6x6 blocks, stored as in
// common.cuh: 3 slots of real diagonal pairs, then the 15 upper entries);
// fl(q) returns slot q as a broadcast pair.
template <class FL>
__device__ __forceinline__ void clover2_chi(FL fl, const P2 (&p)[6], P2 (&out)[6]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const B2 d = fl(q);
    out[2 * q].re = mul2(d.r, p[2 * q].re); out[2 * q].im = mul2(d.r, p[2 * q].im);
    out[2 * q + 1].re = mul2(d.i, p[2 * q + 1].re); out[2 * q + 1].im = mul2(d.i, p[2 * q + 1].im);
  }
  int q = 3;
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = i + 1; j < 6; ++j, ++q) {
      const B2 o = fl(q);
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
__device__ __forceinline__ void global_hops2(const Geom& g, const float2* __restrict__ z, size_t stride,
                                             const TG* __restrict__ U, int blk, int loc, P2 (&acc)[12]) {
  int nb, nl;
  neighbour(g, blk, loc, MU, 1, nb, nl);
  hop2<MU, -1>([&](int k) { return ldg2(z, stride, ((size_t)nb * 12 + k) * 256 + nl); }, LinkG<MU, TG>(U, blk, loc),
               acc);
  neighbour(g, blk, loc, MU, -1, nb, nl);
  hop2<MU, 1>([&](int k) { return ldg2(z, stride, ((size_t)nb * 12 + k) * 256 + nl); }, LinkG<MU, TG>(U, nb, nl), acc);
}

// p = A psi for the whole site, psi read component by component through ld
template <class TG, class LD>
__device__ __forceinline__ void clover2(const TG* __restrict__ A, int blk, int loc, LD ld, P2 (&out)[12]) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    P2 p[6], o[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = ld(chi * 6 + k);
    const TG* a = A + ((size_t)(blk * 36 + chi * 18)) * 256 + loc;
    clover2_chi([&](int q) { return Fld<TG>::ld(a + q * 256); }, p, o);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[chi * 6 + k] = o[k];
  }
}

}  // namespace pair
}  // namespace sapmg
