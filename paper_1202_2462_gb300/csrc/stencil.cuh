// Site-level pieces of the clover-Wilson operator
//   (D psi)(x) = A(x) psi(x) - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x+mu)
//                                        + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu) ]
// (Sec. 1, Eq. 1.1), where A(x) holds 4 + m0 and the clover term.  Gamma
// matrices are in the chiral basis gamma_mu = [[0, X_mu], [X_mu^dagger, 0]] with
// X_k = -i sigma_k (k = x, y, z) and X_t = 1, so (1 + s gamma_mu) psi =
// [h; s X_mu^dagger h] with the half spinor h = psi_upper + s X_mu psi_lower:
// every hop multiplies only two spin rows by the link (spin projection).
#pragma once
#include "common.cuh"

namespace sapmg {

// h = psi_u + S * X_MU psi_l  (S = -1: forward hop, S = +1: backward hop)
template <int MU, int S, class R>
__device__ __forceinline__ void spin_project(const Cplx<R> (&p)[12], Cplx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cplx<R> l0 = p[6 + c], l1 = p[9 + c];
    Cplx<R> x0, x1;
    if (MU == 0) { x0 = mul_mi(l1); x1 = mul_mi(l0); }
    else if (MU == 1) { x0 = cmk(-l1.re, -l1.im); x1 = l0; }
    else if (MU == 2) { x0 = mul_mi(l0); x1 = mul_i(l1); }
    else { x0 = l0; x1 = l1; }
    if (S > 0) { h[c] = p[c] + x0; h[3 + c] = p[3 + c] + x1; }
    else { h[c] = p[c] - x0; h[3 + c] = p[3 + c] - x1; }
  }
}

// The same projection reading the four-spinor component by component from a
// loader (global or shared memory), so that only the half spinor is live.
template <int MU, int S, class R, class LD>
__device__ __forceinline__ void spin_project_ld(LD ld, Cplx<R> (&h)[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cplx<R> l0 = ld(6 + c), l1 = ld(9 + c);
    Cplx<R> x0, x1;
    if (MU == 0) { x0 = mul_mi(l1); x1 = mul_mi(l0); }
    else if (MU == 1) { x0 = cmk(-l1.re, -l1.im); x1 = l0; }
    else if (MU == 2) { x0 = mul_mi(l0); x1 = mul_i(l1); }
    else { x0 = l0; x1 = l1; }
    const Cplx<R> u0 = ld(c), u1 = ld(3 + c);
    if (S > 0) { h[c] = u0 + x0; h[3 + c] = u1 + x1; }
    else { h[c] = u0 - x0; h[3 + c] = u1 - x1; }
  }
}

// acc_u += g, acc_l += S * X_MU^dagger g
template <int MU, int S, class R>
__device__ __forceinline__ void spin_reconstruct_add(const Cplx<R> (&g)[6], Cplx<R> (&acc)[12]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const Cplx<R> g0 = g[c], g1 = g[3 + c];
    acc[c] = acc[c] + g0;
    acc[3 + c] = acc[3 + c] + g1;
    Cplx<R> x0, x1;
    if (MU == 0) { x0 = mul_i(g1); x1 = mul_i(g0); }
    else if (MU == 1) { x0 = g1; x1 = cmk(-g0.re, -g0.im); }
    else if (MU == 2) { x0 = mul_i(g0); x1 = mul_mi(g1); }
    else { x0 = g0; x1 = g1; }
    if (S > 0) { acc[6 + c] = acc[6 + c] + x0; acc[9 + c] = acc[9 + c] + x1; }
    else { acc[6 + c] = acc[6 + c] - x0; acc[9 + c] = acc[9 + c] - x1; }
  }
}

template <class R, class TG>
__device__ __forceinline__ void load_link(const TG* __restrict__ U, int blk, int mu, int loc, Cplx<R> (&u)[9]) {
  const TG* p = U + ((size_t)(blk * 4 + mu) * 9) * 256 + loc;
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = Io<R, TG>::ld(p + k * 256);
}

// g = U h on both spin rows
template <class R>
__device__ __forceinline__ void su3_mul(const Cplx<R> (&u)[9], const Cplx<R> (&h)[6], Cplx<R> (&g)[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cplx<R> acc = u[a * 3] * h[s * 3];
      cfma(acc, u[a * 3 + 1], h[s * 3 + 1]);
      cfma(acc, u[a * 3 + 2], h[s * 3 + 2]);
      g[s * 3 + a] = acc;
    }
}

// g = U^dagger h on both spin rows
template <class R>
__device__ __forceinline__ void su3_dag_mul(const Cplx<R> (&u)[9], const Cplx<R> (&h)[6], Cplx<R> (&g)[6]) {
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cplx<R> acc = cmk<R>(0, 0);
      cfma_conj(acc, u[a], h[s * 3]);
      cfma_conj(acc, u[3 + a], h[s * 3 + 1]);
      cfma_conj(acc, u[6 + a], h[s * 3 + 2]);
      g[s * 3 + a] = acc;
    }
}

template <class R, class TS>
__device__ __forceinline__ void load_spinor(const TS* __restrict__ f, int blk, int loc, Cplx<R> (&p)[12]) {
  const TS* q = f + (size_t)blk * 12 * 256 + loc;
#pragma unroll
  for (int c = 0; c < 12; ++c) p[c] = Io<R, TS>::ldc(q + c * 256);
}

template <class R, class TS>
__device__ __forceinline__ void store_spinor(TS* __restrict__ f, int blk, int loc, const Cplx<R> (&p)[12]) {
  TS* q = f + (size_t)blk * 12 * 256 + loc;
#pragma unroll
  for (int c = 0; c < 12; ++c) Io<R, TS>::st(q + c * 256, p[c]);
}

__device__ __forceinline__ int offdiag_index(int i, int j) {  // i < j, 0..14
  return i * 6 - (i * (i + 1)) / 2 + (j - i - 1);
}

// out = A(x) psi: two Hermitian 6x6 chiral blocks.  Each stored off-diagonal
// entry a_ij (i < j) is loaded once and used for both a_ij psi_j and
// conj(a_ij) psi_i, so only one entry is live at a time.
template <class R, class TG>
__device__ __forceinline__ void clover_apply(const TG* __restrict__ A, int blk, int loc, const Cplx<R> (&p)[12],
                                             Cplx<R> (&out)[12]) {
#pragma unroll
  for (int chi = 0; chi < 2; ++chi) {
    const TG* a = A + ((size_t)(blk * 36 + chi * 18)) * 256 + loc;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const Cplx<R> d = Io<R, TG>::ld(a + q * 256);
      out[chi * 6 + 2 * q] = d.re * p[chi * 6 + 2 * q];
      out[chi * 6 + 2 * q + 1] = d.im * p[chi * 6 + 2 * q + 1];
    }
    int q = 3;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int j = i + 1; j < 6; ++j, ++q) {
        const Cplx<R> o = Io<R, TG>::ld(a + q * 256);
        cfma(out[chi * 6 + i], o, p[chi * 6 + j]);
        cfma_conj(out[chi * 6 + j], o, p[chi * 6 + i]);
      }
  }
}

// Forward (+mu) hop contribution (1 - gamma_mu) U_mu(x) psi_n accumulated into acc.
template <int MU, class R, class TG>
__device__ __forceinline__ void hop_fwd(const TG* __restrict__ U, int blk, int loc, const Cplx<R> (&pn)[12],
                                        Cplx<R> (&acc)[12]) {
  Cplx<R> h[6], g[6], u[9];
  spin_project<MU, -1>(pn, h);
  load_link<R>(U, blk, MU, loc, u);
  su3_mul(u, h, g);
  spin_reconstruct_add<MU, -1>(g, acc);
}

// Backward (-mu) hop contribution (1 + gamma_mu) U_mu(x-mu)^dagger psi_n; (nblk, nloc) = x - mu.
template <int MU, class R, class TG>
__device__ __forceinline__ void hop_bwd(const TG* __restrict__ U, int nblk, int nloc, const Cplx<R> (&pn)[12],
                                        Cplx<R> (&acc)[12]) {
  Cplx<R> h[6], g[6], u[9];
  spin_project<MU, 1>(pn, h);
  load_link<R>(U, nblk, MU, nloc, u);
  su3_dag_mul(u, h, g);
  spin_reconstruct_add<MU, 1>(g, acc);
}

// Sum of all eight hops at (blk, loc) with neighbours read from global field f.
// DAG: the hops of D^dagger = gamma5 D gamma5, whose projectors are
// gamma5 (1 -+ gamma_mu) gamma5 = (1 +- gamma_mu) (gamma5 anticommutes with
// gamma_mu; the clover term commutes with gamma5 and is Hermitian, so it is
// the same in D and D^dagger).
template <int MU, class R, class TS, class TG, bool DAG = false>
__device__ __forceinline__ void hops_global_dir(const Geom& g, const TS* __restrict__ f, const TG* __restrict__ U,
                                                int blk, int loc, Cplx<R> (&acc)[12]) {
  constexpr int SF = DAG ? 1 : -1;   // projector sign of the forward hop
  int nb, nl;
  Cplx<R> h[6], gg[6], u[9];
  neighbour(g, blk, loc, MU, 1, nb, nl);
  {
    const TS* q = f + (size_t)nb * 12 * 256 + nl;
    spin_project_ld<MU, SF, R>([&](int c) { return Io<R, TS>::ldc(q + c * 256); }, h);
  }
  load_link<R>(U, blk, MU, loc, u);
  su3_mul(u, h, gg);
  spin_reconstruct_add<MU, SF>(gg, acc);
  neighbour(g, blk, loc, MU, -1, nb, nl);
  {
    const TS* q = f + (size_t)nb * 12 * 256 + nl;
    spin_project_ld<MU, -SF, R>([&](int c) { return Io<R, TS>::ldc(q + c * 256); }, h);
  }
  load_link<R>(U, nb, MU, nl, u);
  su3_dag_mul(u, h, gg);
  spin_reconstruct_add<MU, -SF>(gg, acc);
}

template <class R, class TS, class TG>
__device__ __forceinline__ void hops_global(const Geom& g, const TS* __restrict__ f, const TG* __restrict__ U,
                                            int blk, int loc, Cplx<R> (&acc)[12]) {
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = cmk<R>(0, 0);
  hops_global_dir<0>(g, f, U, blk, loc, acc);
  hops_global_dir<1>(g, f, U, blk, loc, acc);
  hops_global_dir<2>(g, f, U, blk, loc, acc);
  hops_global_dir<3>(g, f, U, blk, loc, acc);
}

}  // namespace sapmg
