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
#include "async.cuh"
#include "internal.h"
#include "pair.cuh"

namespace sapmg {
namespace {
using namespace pair;
template <int MU, class TG>
__device__ __forceinline__ void block_hops2(const TG* __restrict__ U, const float4* __restrict__ rs, int blk, int loc,
                                            P2 (&acc)[12]) {
  const int ls = 1 << (2 * MU);
  const int c = (loc >> (2 * MU)) & 3;
  if (c < 3) hop2<MU, -1>([&](int k) { return lds2(rs, k * 256 + loc + ls); }, LinkG<MU, TG>(U, blk, loc), acc);
  if (c > 0) hop2<MU, 1>([&](int k) { return lds2(rs, k * 256 + loc - ls); }, LinkG<MU, TG>(U, blk, loc - ls), acc);
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
    // alpha = <p, rho> / <p, p> by division (a reciprocal of a tiny denormal <p, p>
    // overflows, and 0 * inf would be NaN; the quotient is scale-invariant)
    float2 al_re = f2(0.f), al_im = f2(0.f);
    if (pp.x > 0.f) { al_re.x = pr_re.x / pp.x; al_im.x = pr_im.x / pp.x; }
    if (pp.y > 0.f) { al_re.y = pr_re.y / pp.y; al_im.y = pr_im.y / pp.y; }
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

// ---------------------------------------------------------------------------
// Block-resident form: one CTA per block of the colour copies the block's links
// and clover into shared memory once (two 1-D bulk copies completing on one
// mbarrier; the first pair's residual is computed from global memory while
// they land) and runs every pair of right-hand sides through the block in
// turn.  Every field load of the MR steps is then a shared-memory load and
// each field crosses HBM once per colour pass, whatever the number of
// right-hand sides.  rho lives in shared memory (the neighbours read it); the
// correction e and the thread's own rho live in registers (one CTA per SM).

// link entry k of U_MU at (blk, loc) through a generic pointer: the block's copy in shared
// memory when the site lies in the block, global memory otherwise
template <int MU, class TG>
struct LinkP {
  const TG* p;
  __device__ __forceinline__ explicit LinkP(const TG* q) : p(q) {}
  __device__ __forceinline__ B2 operator()(int k) const { return FldS<TG>::ld(p + k * 256); }
};

template <class TG, class LD>
__device__ __forceinline__ void clover2s(const TG* __restrict__ As, int loc, LD ld, P2 (&out)[12]) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    P2 p[6], o[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) p[k] = ld(chi * 6 + k);
    const TG* a = As + (chi * 18) * 256 + loc;
    clover2_chi([&](int q) { return FldS<TG>::ld(a + q * 256); }, p, o);
#pragma unroll
    for (int k = 0; k < 6; ++k) out[chi * 6 + k] = o[k];
  }
}

// the hops of D at (blk, loc) with neighbours from global z; links from the
// block's copy in shared memory where they lie in the block
template <int MU, class TG>
__device__ __forceinline__ void global_hops2s(const Geom& g, const float2* __restrict__ z, size_t stride,
                                              const TG* __restrict__ U, const TG* Us, int blk, int loc,
                                              P2 (&acc)[12]) {
  const int ls = 1 << (2 * MU);
  const int c = (loc >> (2 * MU)) & 3;
  int nb, nl;
  neighbour(g, blk, loc, MU, 1, nb, nl);
  hop2<MU, -1>([&](int k) { return ldg2(z, stride, ((size_t)nb * 12 + k) * 256 + nl); },
               LinkS<MU, TG>(Us, loc), acc);
  neighbour(g, blk, loc, MU, -1, nb, nl);
  const TG* lp = c > 0 ? Us + (MU * 9) * 256 + (loc - ls) : U + ((size_t)(nb * 4 + MU) * 9) * 256 + nl;
  hop2<MU, 1>([&](int k) { return ldg2(z, stride, ((size_t)nb * 12 + k) * 256 + nl); }, LinkP<MU, TG>(lp), acc);
}

// Both hops of direction MU without a branch: a hop that leaves the block is
// computed from the site itself and weighted by 0 (acc + 0 * g = acc), so the
// two hops' loads and products are independent work the scheduler can
// interleave.  Used for x, y, z, whose block faces cut through every warp
// (a branch there runs both hops anyway); t keeps the branch (warp-uniform).
template <int MU, class TG>
__device__ __forceinline__ void block_hops2s_both(const TG* Us, const float4* __restrict__ rs, int loc,
                                                  P2 (&acc)[12]) {
  const int ls = 1 << (2 * MU);
  const int c = (loc >> (2 * MU)) & 3;
  const int lf = c < 3 ? loc + ls : loc, lb = c > 0 ? loc - ls : loc;
  const float kf = c < 3 ? -0.5f : 0.f, kb = c > 0 ? -0.5f : 0.f;
  hop2<MU, -1>([&](int k) { return lds2(rs, k * 256 + lf); }, LinkS<MU, TG>(Us, loc), acc, kf);
  hop2<MU, 1>([&](int k) { return lds2(rs, k * 256 + lb); }, LinkS<MU, TG>(Us, lb), acc, kb);
}

template <int MU, class TG>
__device__ __forceinline__ void block_hops2s(const TG* Us, const float4* __restrict__ rs, int loc, P2 (&acc)[12]) {
  const int ls = 1 << (2 * MU);
  const int c = (loc >> (2 * MU)) & 3;
  if (c < 3) hop2<MU, -1>([&](int k) { return lds2(rs, k * 256 + loc + ls); }, LinkS<MU, TG>(Us, loc), acc);
  if (c > 0) hop2<MU, 1>([&](int k) { return lds2(rs, k * 256 + loc - ls); }, LinkS<MU, TG>(Us, loc - ls), acc);
}

// rho = b - D z for one pair of right-hand sides, written to shared memory;
// FS: fields from the block's shared copy (else from global memory)
template <bool FS, class TG>
__device__ __forceinline__ void residual_pair(const Geom& g, const float2* __restrict__ z,
                                              const float2* __restrict__ b, size_t stride, const TG* __restrict__ U,
                                              const TG* __restrict__ A, const TG* Us, const TG* As, int blk, int loc,
                                              float4* rs) {
  const size_t site0 = (size_t)blk * 12 * 256 + loc;
  P2 acc[12];
  auto zl = [&](int k) { return ldg2(z, stride, site0 + k * 256); };
  if (FS) clover2s<TG>(As, loc, zl, acc);
  else clover2<TG>(A, blk, loc, zl, acc);
  if (FS) {
    global_hops2s<0>(g, z, stride, U, Us, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2s<1>(g, z, stride, U, Us, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2s<2>(g, z, stride, U, Us, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2s<3>(g, z, stride, U, Us, blk, loc, acc);
  } else {
    global_hops2<0>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<1>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<2>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<3>(g, z, stride, U, blk, loc, acc);
  }
#pragma unroll
  for (int c = 0; c < 12; ++c) {
    const P2 bb = ldg2(b, stride, site0 + c * 256);
    P2 r;
    r.re = sub2(bb.re, acc[c].re);
    r.im = sub2(bb.im, acc[c].im);
    sts2(rs, c * 256 + loc, r);
  }
}

template <class TG, int BF>
__global__ void __launch_bounds__(256, 1)
    sap_block_kernel(float2* __restrict__ z, const float2* __restrict__ b, const TG* __restrict__ U,
                     const TG* __restrict__ A, Geom g, int colour, int n_mr, int npairs, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TG* Us = reinterpret_cast<TG*>(smem_raw);                               // links of the block [4][9][256]
  TG* As = Us + 36 * 256;                                                 // clover of the block [36][256]
  float4* rs = reinterpret_cast<float4*>(As + 36 * 256);                 // rho [12][256]
  float4 (*red)[2] = reinterpret_cast<float4 (*)[2]>(rs + 12 * 256);     // [8][2]
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 8);
  constexpr uint32_t kFieldBytes = 36 * 256 * sizeof(TG);
  const size_t stride = (size_t)g.V * 12;
  const int blk = colour_block(g, blockIdx.x, colour);
  const int loc = threadIdx.x;
  const size_t site0 = (size_t)blk * 12 * 256 + loc;
  if (loc == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (loc == 0) {
    mbar_expect_tx(bar, 2 * kFieldBytes);
    bulk_copy_g2s(Us, U + (size_t)blk * 36 * 256, kFieldBytes, bar);
    bulk_copy_g2s(As, A + (size_t)blk * 36 * 256, kFieldBytes, bar);
  }
  const int spins = wait_spins(err);
  residual_pair<false>(g, z, b, stride, U, A, Us, As, blk, loc, rs);
  const bool waited = mbar_wait(bar, 0, spins);
  if (__syncthreads_or(!waited)) {          // uniform decision: every thread leaves together
    if (loc == 0) {
      atomicExch(err, 1);
      mbar_wait(bar, 0);                    // let the copies in flight land (bounded as well)
    }
    __syncthreads();
    return;
  }
  for (int pr = 0; pr < npairs; ++pr) {
    float2* zp = z + (size_t)pr * 2 * stride;
    if (pr > 0) residual_pair<true>(g, zp, b + (size_t)pr * 2 * stride, stride, U, A, Us, As, blk, loc, rs);
    P2 e[12];
    for (int it = 0; it < n_mr; ++it) {
      __syncthreads();                                 // rho of every site written
      P2 p[12];
      clover2s<TG>(As, loc, [&](int k) { return lds2(rs, k * 256 + loc); }, p);
      if (BF) {                                        // BF 1: branch-free x, y, z hops; 2: also t
        block_hops2s_both<0>(Us, rs, loc, p);
        block_hops2s_both<1>(Us, rs, loc, p);
        block_hops2s_both<2>(Us, rs, loc, p);
        if (BF == 2) block_hops2s_both<3>(Us, rs, loc, p);
        else block_hops2s<3>(Us, rs, loc, p);
      } else {
        block_hops2s<0>(Us, rs, loc, p);
        asm volatile("" ::: "memory");
        block_hops2s<1>(Us, rs, loc, p);
        asm volatile("" ::: "memory");
        block_hops2s<2>(Us, rs, loc, p);
        asm volatile("" ::: "memory");
        block_hops2s<3>(Us, rs, loc, p);
      }
      P2 ro[12];
      float2 pr_re = f2(0.f), pr_im = f2(0.f), pp = f2(0.f);
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        ro[c] = lds2(rs, c * 256 + loc);
        pr_re = fma2(p[c].re, ro[c].re, pr_re); pr_re = fma2(p[c].im, ro[c].im, pr_re);
        pr_im = fma2(p[c].re, ro[c].im, pr_im); pr_im = fma2(p[c].im, sub2(f2(0.f), ro[c].re), pr_im);
        pp = fma2(p[c].re, p[c].re, pp); pp = fma2(p[c].im, p[c].im, pp);
      }
      block_reduce6(pr_re, pr_im, pp, red);           // its barrier follows every neighbour read of rho
      // alpha by division, as in the pair kernel above
      float2 al_re = f2(0.f), al_im = f2(0.f);
      if (pp.x > 0.f) { al_re.x = pr_re.x / pp.x; al_im.x = pr_im.x / pp.x; }
      if (pp.y > 0.f) { al_re.y = pr_re.y / pp.y; al_im.y = pr_im.y / pp.y; }
      const float2 nal_im = make_float2(-al_im.x, -al_im.y);
      const float2 nal_re = make_float2(-al_re.x, -al_re.y);
      const bool last = it == n_mr - 1;
#pragma unroll
      for (int c = 0; c < 12; ++c) {
        P2 ar;
        ar.re = fma2(nal_im, ro[c].im, mul2(al_re, ro[c].re));
        ar.im = fma2(al_im, ro[c].re, mul2(al_re, ro[c].im));
        if (it == 0) e[c] = ar;
        else { e[c].re = add2(e[c].re, ar.re); e[c].im = add2(e[c].im, ar.im); }
        if (!last) {
          P2 rn;
          rn.re = fma2(al_im, p[c].im, fma2(nal_re, p[c].re, ro[c].re));
          rn.im = fma2(nal_im, p[c].re, fma2(nal_re, p[c].im, ro[c].im));
          sts2(rs, c * 256 + loc, rn);
        }
      }
    }
    // z += e on the block (own site only)
#pragma unroll
    for (int c = 0; c < 12; ++c) {
      const size_t i = site0 + c * 256;
      const float2 za = zp[i], zb = zp[i + stride];
      zp[i] = make_float2(za.x + e[c].re.x, za.y + e[c].im.x);
      zp[i + stride] = make_float2(zb.x + e[c].re.y, zb.y + e[c].im.y);
    }
  }
}

// ---------------------------------------------------------------------------
// Shape 6: the block-resident pass with two threads per site.  The CTA has 512
// threads; thread half H (0: threads 0-255, 1: 256-511) of site loc applies
// the clover block of chirality H (spin-colour components 6H .. 6H+5) and the
// hops of directions 2H and 2H+1, into a full 12-component partial sum; the
// halves swap the partial sums of each other's components through shared
// memory, and from there on each thread owns the 6 components of its
// chirality: its share of <p, rho> and <p, p>, its part of e and rho.  The same
// work as shape 5 on twice the warps per SM (16 instead of 8), to hide the
// latency of dependent FMA chains and shared-memory loads, at the cost of one
// more barrier and the 192-byte swap per site and MR step.

__device__ __forceinline__ void block_reduce6_16(float2& a, float2& b, float2& c, float4 (*red)[2]) {
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
  for (int k = 1; k < 16; ++k) {
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

// acc = A_H psi on the components of chirality H (psi through ld), zero on the others
template <int H, class FL, class LD>
__device__ __forceinline__ void clover_half(FL fl, LD ld, P2 (&acc)[12]) {
  P2 p[6], o[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) p[k] = ld(6 * H + k);
  clover2_chi(fl, p, o);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    acc[6 * H + k] = o[k];
    acc[6 * (1 - H) + k].re = f2(0.f);
    acc[6 * (1 - H) + k].im = f2(0.f);
  }
}

// partial sums of the other chirality out to the swap buffer xs; after a barrier,
// swap_in adds the partner's partial sums of this chirality
template <int H>
__device__ __forceinline__ void swap_out(float4* xs, int loc, const P2 (&acc)[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) sts2(xs, (6 * (1 - H) + k) * 256 + loc, acc[6 * (1 - H) + k]);
}
template <int H>
__device__ __forceinline__ void swap_in(const float4* xs, int loc, P2 (&acc)[12]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const P2 x = lds2(xs, (6 * H + k) * 256 + loc);
    acc[6 * H + k].re = add2(acc[6 * H + k].re, x.re);
    acc[6 * H + k].im = add2(acc[6 * H + k].im, x.im);
  }
}

// Every barrier below sits in code all 512 threads run; the work between two
// barriers branches on the (warp-uniform) half into instances with a
// compile-time chirality H.

// first part of rho = b - D z for chirality H: clover block H and the hops of
// directions 2H, 2H+1 into acc, the other chirality's partial sums out to xs;
// FS: fields from the block's copy in shared memory
template <int H, bool FS, class TG>
__device__ __forceinline__ void residual_a(const Geom& g, const float2* __restrict__ z, size_t stride,
                                           const TG* __restrict__ U, const TG* __restrict__ A, const TG* Us,
                                           const TG* As, int blk, int loc, float4* xs, P2 (&acc)[12]) {
  const size_t site0 = (size_t)blk * 12 * 256 + loc;
  auto zl = [&](int k) { return ldg2(z, stride, site0 + k * 256); };
  if (FS) {
    const TG* a = As + (H * 18) * 256 + loc;
    clover_half<H>([&](int q) { return FldS<TG>::ld(a + q * 256); }, zl, acc);
    global_hops2s<2 * H>(g, z, stride, U, Us, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2s<2 * H + 1>(g, z, stride, U, Us, blk, loc, acc);
  } else {
    const TG* a = A + ((size_t)(blk * 36 + H * 18)) * 256 + loc;
    clover_half<H>([&](int q) { return Fld<TG>::ld(a + q * 256); }, zl, acc);
    global_hops2<2 * H>(g, z, stride, U, blk, loc, acc);
    asm volatile("" ::: "memory");
    global_hops2<2 * H + 1>(g, z, stride, U, blk, loc, acc);
  }
  swap_out<H>(xs, loc, acc);
}

// second part: the partner's partial sums in, rho = b - acc on chirality H
template <int H>
__device__ __forceinline__ void residual_b(const float2* __restrict__ b, size_t stride, size_t site0, int loc,
                                           float4* rs, const float4* xs, P2 (&acc)[12]) {
  swap_in<H>(xs, loc, acc);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int c = 6 * H + k;
    const P2 bb = ldg2(b, stride, site0 + c * 256);
    P2 r;
    r.re = sub2(bb.re, acc[c].re);
    r.im = sub2(bb.im, acc[c].im);
    sts2(rs, c * 256 + loc, r);
  }
}

// MR step, first part: p = D_i rho partially (clover block H, hops 2H, 2H+1), swap out
template <int H, class TG>
__device__ __forceinline__ void mr_a(const TG* Us, const TG* As, const float4* rs, float4* xs, int loc,
                                     P2 (&p)[12]) {
  const TG* a = As + (H * 18) * 256 + loc;
  clover_half<H>([&](int q) { return FldS<TG>::ld(a + q * 256); }, [&](int k) { return lds2(rs, k * 256 + loc); },
                 p);
  block_hops2s_both<2 * H>(Us, rs, loc, p);
  block_hops2s_both<2 * H + 1>(Us, rs, loc, p);
  swap_out<H>(xs, loc, p);
}

// second part: swap in, this thread's share of <p, rho> and <p, p>
template <int H>
__device__ __forceinline__ void mr_b(const float4* rs, const float4* xs, int loc, P2 (&p)[12], P2 (&ro)[6],
                                     float2& pr_re, float2& pr_im, float2& pp) {
  swap_in<H>(xs, loc, p);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const P2 q = p[6 * H + k];
    ro[k] = lds2(rs, (6 * H + k) * 256 + loc);
    pr_re = fma2(q.re, ro[k].re, pr_re); pr_re = fma2(q.im, ro[k].im, pr_re);
    pr_im = fma2(q.re, ro[k].im, pr_im); pr_im = fma2(q.im, sub2(f2(0.f), ro[k].re), pr_im);
    pp = fma2(q.re, q.re, pp); pp = fma2(q.im, q.im, pp);
  }
}

// third part: e += alpha rho and rho -= alpha p on chirality H (e in es, read
// and written by this thread only); on the last step z += e instead
template <int H>
__device__ __forceinline__ void mr_c(float2* zp, size_t stride, size_t site0, float4* rs, float4* es, int loc,
                                     const P2 (&p)[12], const P2 (&ro)[6], float2 al_re, float2 al_im, bool first,
                                     bool last) {
  const float2 nal_im = make_float2(-al_im.x, -al_im.y);
  const float2 nal_re = make_float2(-al_re.x, -al_re.y);
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const int c = (6 * H + k) * 256 + loc;
    P2 ar;
    ar.re = fma2(nal_im, ro[k].im, mul2(al_re, ro[k].re));
    ar.im = fma2(al_im, ro[k].re, mul2(al_re, ro[k].im));
    if (!first) {
      const P2 e = lds2(es, c);
      ar.re = add2(e.re, ar.re); ar.im = add2(e.im, ar.im);
    }
    if (!last) {
      sts2(es, c, ar);
      const P2 q = p[6 * H + k];
      P2 rn;
      rn.re = fma2(al_im, q.im, fma2(nal_re, q.re, ro[k].re));
      rn.im = fma2(nal_im, q.re, fma2(nal_re, q.im, ro[k].im));
      sts2(rs, c, rn);
    } else {
      const size_t i = site0 + (6 * H + k) * 256;
      const float2 za = zp[i], zb = zp[i + stride];
      zp[i] = make_float2(za.x + ar.re.x, za.y + ar.im.x);
      zp[i + stride] = make_float2(zb.x + ar.re.y, zb.y + ar.im.y);
    }
  }
}

template <class TG>
__global__ void __launch_bounds__(512, 1)
    sap_split_kernel(float2* __restrict__ z, const float2* __restrict__ b, const TG* __restrict__ U,
                     const TG* __restrict__ A, Geom g, int colour, int n_mr, int npairs, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  TG* Us = reinterpret_cast<TG*>(smem_raw);                               // links of the block [4][9][256]
  TG* As = Us + 36 * 256;                                                 // clover of the block [36][256]
  float4* rs = reinterpret_cast<float4*>(As + 36 * 256);                 // rho [12][256]
  float4* xs = rs + 12 * 256;                                             // swap buffer [12][256]
  float4* es = xs + 12 * 256;                                             // e [12][256]
  float4 (*red)[2] = reinterpret_cast<float4 (*)[2]>(es + 12 * 256);     // [16][2]
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 16);
  constexpr uint32_t kFieldBytes = 36 * 256 * sizeof(TG);
  const size_t stride = (size_t)g.V * 12;
  const int blk = colour_block(g, blockIdx.x, colour);
  const bool h0 = threadIdx.x < 256;                                      // warp-uniform half
  const int loc = threadIdx.x & 255;
  const size_t site0 = (size_t)blk * 12 * 256 + loc;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, 2 * kFieldBytes);
    bulk_copy_g2s(Us, U + (size_t)blk * 36 * 256, kFieldBytes, bar);
    bulk_copy_g2s(As, A + (size_t)blk * 36 * 256, kFieldBytes, bar);
  }
  const int spins = wait_spins(err);
  P2 acc[12];
  // the first pair's residual from global fields while the copies land
  if (h0) residual_a<0, false>(g, z, stride, U, A, Us, As, blk, loc, xs, acc);
  else residual_a<1, false>(g, z, stride, U, A, Us, As, blk, loc, xs, acc);
  __syncthreads();
  if (h0) residual_b<0>(b, stride, site0, loc, rs, xs, acc);
  else residual_b<1>(b, stride, site0, loc, rs, xs, acc);
  const bool waited = mbar_wait(bar, 0, spins);
  if (__syncthreads_or(!waited)) {          // uniform decision: every thread leaves together
    if (threadIdx.x == 0) {
      atomicExch(err, 1);
      mbar_wait(bar, 0);                    // let the copies in flight land (bounded as well)
    }
    __syncthreads();
    return;
  }
  for (int pr = 0; pr < npairs; ++pr) {
    float2* zp = z + (size_t)pr * 2 * stride;
    if (pr > 0) {
      const float2* bp = b + (size_t)pr * 2 * stride;
      __syncthreads();                      // every read of the previous pair's swap buffer done
      if (h0) residual_a<0, true>(g, zp, stride, U, A, Us, As, blk, loc, xs, acc);
      else residual_a<1, true>(g, zp, stride, U, A, Us, As, blk, loc, xs, acc);
      __syncthreads();
      if (h0) residual_b<0>(bp, stride, site0, loc, rs, xs, acc);
      else residual_b<1>(bp, stride, site0, loc, rs, xs, acc);
    }
    for (int it = 0; it < n_mr; ++it) {
      __syncthreads();                      // rho of every site written
      if (h0) mr_a<0>(Us, As, rs, xs, loc, acc);
      else mr_a<1>(Us, As, rs, xs, loc, acc);
      __syncthreads();                      // partial sums swapped
      P2 ro[6];
      float2 pr_re = f2(0.f), pr_im = f2(0.f), pp = f2(0.f);
      if (h0) mr_b<0>(rs, xs, loc, acc, ro, pr_re, pr_im, pp);
      else mr_b<1>(rs, xs, loc, acc, ro, pr_re, pr_im, pp);
      block_reduce6_16(pr_re, pr_im, pp, red);       // its barrier follows every neighbour read of rho
      // alpha by division, as in the pair kernel above
      float2 al_re = f2(0.f), al_im = f2(0.f);
      if (pp.x > 0.f) { al_re.x = pr_re.x / pp.x; al_im.x = pr_im.x / pp.x; }
      if (pp.y > 0.f) { al_re.y = pr_re.y / pp.y; al_im.y = pr_im.y / pp.y; }
      if (h0) mr_c<0>(zp, stride, site0, rs, es, loc, acc, ro, al_re, al_im, it == 0, it == n_mr - 1);
      else mr_c<1>(zp, stride, site0, rs, es, loc, acc, ro, al_re, al_im, it == 0, it == n_mr - 1);
    }
  }
}

template <class TG>
static int run_split(const Geom& g, void* z, const void* b, const void* U, const void* A, int colour, int n_mr,
                     int nrhs, int* err, cudaStream_t s) {
  const size_t smem = 2 * 36 * 256 * sizeof(TG) + sizeof(float4) * (36 * 256 + 32) + 16;
  if (smem > 227 * 1024) return MG_ERR_ARG;          // FP32 fields: the block's copy does not fit
  static bool attr = false;
  if (!attr) {
    SAPMG_CUDA_TRY(cudaFuncSetAttribute(sap_split_kernel<TG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  sap_split_kernel<TG><<<(unsigned)(g.nblocks / 2), 512, smem, s>>>(
      (float2*)z, (const float2*)b, (const TG*)U, (const TG*)A, g, colour, n_mr, nrhs / 2, err);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

template <class TG, int BF>
static int run_block(const Geom& g, void* z, const void* b, const void* U, const void* A, int colour, int n_mr,
                     int nrhs, int* err, cudaStream_t s) {
  const size_t smem = 2 * 36 * 256 * sizeof(TG) + sizeof(float4) * (12 * 256 + 16) + 16;
  static bool attr = false;
  if (!attr) {
    SAPMG_CUDA_TRY(cudaFuncSetAttribute(sap_block_kernel<TG, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    attr = true;
  }
  sap_block_kernel<TG, BF><<<(unsigned)(g.nblocks / 2), 256, smem, s>>>(
      (float2*)z, (const float2*)b, (const TG*)U, (const TG*)A, g, colour, n_mr, nrhs / 2, err);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
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
                           int n_mr, int nrhs, cudaStream_t s, int shape, int* err) {
  if (shape >= 3 && !err) return MG_ERR_ARG;
  if (nrhs < 2 || nrhs % 2 != 0 || n_mr < 1) return MG_ERR_ARG;
#define SAPMG_PAIR_CASE(T)                                                                   \
  return shape == 6 ? run_split<T>(g, z, b, U, A, colour, n_mr, nrhs, err, s)               \
       : shape == 5 ? run_block<T, 2>(g, z, b, U, A, colour, n_mr, nrhs, err, s)             \
       : shape == 4 ? run_block<T, 1>(g, z, b, U, A, colour, n_mr, nrhs, err, s)             \
       : shape == 3 ? run_block<T, 0>(g, z, b, U, A, colour, n_mr, nrhs, err, s)             \
       : shape == 2 ? run_pair<T, true, 1>(g, z, b, U, A, colour, n_mr, nrhs, s)             \
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
