// Aggregation and coarse-grid kernels (Sec. 3):
//   K3 restriction P^dagger, K4 interpolation P, K7 local orthonormalisation of
//   the test vectors, K6 Galerkin assembly D_c = P^dagger D P, K5 the coarse
//   stencil (D_c x)(a) = sum_d M_d(a) x(a + offset_d).
//
// Level 0 -> 1: aggregates are the 4^4 blocks of the fine layout, split by
// chirality (spins {0,1} / {2,3}); coarse dof chi*N + k.  P is stored as the
// locally orthonormal test vectors, block-major: Pv[blk][k][12][256].
// Levels >= 1: fields are canonical [site][n2]; aggregates are a^4 boxes of
// coarse sites; level-1 vectors are stored vector-major [k][site][n2].
// Coarse operators: M[site][d][j][i] (column j, row i contiguous in i), with
// d = 0 self, 1 + 2 mu the +mu neighbour, 2 + 2 mu the -mu neighbour.
#include "internal.h"
#include "coarse.h"
#include "stencil.cuh"

namespace sapmg {

// ============================================================ level 0 -> 1
// K3: rc[blk][chi*N + k] = sum over the block's sites and chirality chi of conj(v_k) r
template <class R, class TS, class TV, class TC>
__global__ void __launch_bounds__(256) restrict0_kernel(const TS* __restrict__ in, TC* __restrict__ out,
                                                        const TV* __restrict__ Pv, int N, int nrhs, int nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R (*red)[4] = reinterpret_cast<R (*)[4]>(smem_raw);        // [8 * N][4]
  const int blk = MG_CLAMP(kAggregate, blockIdx.x / nrhs, nblocks), rhs = blockIdx.x % nrhs, loc = threadIdx.x;
  const int wid = loc >> 5, lane = loc & 31;
  const size_t off = (size_t)rhs * nblocks * 12 * 256;       // rhs stride (one field)
  Cplx<R> r[12];
  load_spinor<R>(in + off, blk, loc, r);
  for (int k = 0; k < N; ++k) {
    const TV* v = Pv + ((size_t)(blk * N + k) * 12) * 256 + loc;
    Cplx<R> d0 = cmk<R>(0, 0), d1 = cmk<R>(0, 0);
#pragma unroll
    for (int c = 0; c < 6; ++c) cfma_conj(d0, Io<R, TV>::ld(v + c * 256), r[c]);
#pragma unroll
    for (int c = 6; c < 12; ++c) cfma_conj(d1, Io<R, TV>::ld(v + c * 256), r[c]);
    R a = warp_sum(d0.re), b = warp_sum(d0.im), c2 = warp_sum(d1.re), d = warp_sum(d1.im);
    if (lane == 0) { R* q = red[wid * N + k]; q[0] = a; q[1] = b; q[2] = c2; q[3] = d; }
  }
  __syncthreads();
  const int n2 = 2 * N;
  TC* o = out + (size_t)rhs * nblocks * n2 + (size_t)blk * n2;
  for (int t = loc; t < n2; t += 256) {
    const int chi = t / N, k = t % N;
    R sr = 0, si = 0;
    for (int w = 0; w < 8; ++w) { sr += red[w * N + k][2 * chi]; si += red[w * N + k][2 * chi + 1]; }
    Io<R, TC>::st(o + t, cmk(sr, si));
  }
}

// K4: out(x) = sum_k v_k(x)|_chi e[blk][chi*N + k]   (overwrites out)
template <class R, class TS, class TV, class TC>
__global__ void __launch_bounds__(256) prolong0_kernel(const TC* __restrict__ in, TS* __restrict__ out,
                                                       const TV* __restrict__ Pv, int N, int nrhs, int nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Cplx<R>* e = reinterpret_cast<Cplx<R>*>(smem_raw);             // [2N]
  const int blk = MG_CLAMP(kAggregate, blockIdx.x / nrhs, nblocks), rhs = blockIdx.x % nrhs, loc = threadIdx.x;
  const int n2 = 2 * N;
  const TC* ein = in + (size_t)rhs * nblocks * n2 + (size_t)blk * n2;
  for (int t = loc; t < n2; t += 256) e[t] = Io<R, TC>::ldc(ein + t);
  __syncthreads();
  Cplx<R> o[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) o[c] = cmk<R>(0, 0);
  for (int k = 0; k < N; ++k) {
    const TV* v = Pv + ((size_t)(blk * N + k) * 12) * 256 + loc;
    const Cplx<R> e0 = e[k], e1 = e[N + k];
#pragma unroll
    for (int c = 0; c < 6; ++c) cfma(o[c], Io<R, TV>::ld(v + c * 256), e0);
#pragma unroll
    for (int c = 6; c < 12; ++c) cfma(o[c], Io<R, TV>::ld(v + c * 256), e1);
  }
  store_spinor<R>(out + (size_t)rhs * nblocks * 12 * 256, blk, loc, o);
}

// Multi-RHS forms for the mixed precision (FP32 vectors):
//
// K3': CTA (block, chirality, group of RG right-hand sides).  The group's
// residual half-spinors (6 components x 256 sites each) are staged in shared
// memory; warp w owns the outputs (k, r) with k = w, w+8, w+16, ... and lane l
// sums the terms K = l, l+32, ... of the 1536-term dot products, then the
// lanes are reduced.  P is read once per group (not once per right-hand side).
template <int RG, class TV>
__global__ void __launch_bounds__(256) restrict0_mrhs_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                             const TV* __restrict__ Pv, int N, int nrhs,
                                                             int nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* rs = reinterpret_cast<float2*>(smem_raw);             // [RG][1536]
  // right-hand-side group fastest in the grid: the groups of one (block,
  // chirality) run back to back and share its P rows through L2
  const int ngrp = (nrhs + RG - 1) / RG;
  const int r0 = (blockIdx.x % ngrp) * RG;
  const int blk = MG_CLAMP(kAggregate, blockIdx.x / ngrp / 2, nblocks), chi = (blockIdx.x / ngrp) % 2;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const size_t fs = (size_t)nblocks * 12 * 256;
  const int rg = min(RG, nrhs - r0);
#pragma unroll 8
  for (int e = tid; e < RG * 1536; e += 256) {
    const int r = e / 1536, K = e % 1536;
    rs[e] = r < rg ? in[(size_t)(r0 + r) * fs + ((size_t)blk * 12 + 6 * chi) * 256 + K] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  constexpr int KW = 3;                                           // k = w + 8*q, q < KW (N <= 24)
  float are[KW][RG], aim[KW][RG];
#pragma unroll
  for (int q = 0; q < KW; ++q)
#pragma unroll
    for (int r = 0; r < RG; ++r) are[q][r] = aim[q][r] = 0.f;
#pragma unroll 4
  for (int K = lane; K < 1536; K += 32) {
    float2 x[RG];
#pragma unroll
    for (int r = 0; r < RG; ++r) x[r] = rs[r * 1536 + K];
#pragma unroll
    for (int q = 0; q < KW; ++q) {
      const int k = w + 8 * q;
      if (k < N) {
        const Cplx<float> v = Io<float, TV>::ld(Pv + ((size_t)(blk * N + k) * 12 + 6 * chi) * 256 + K);
#pragma unroll
        for (int r = 0; r < RG; ++r) {
          are[q][r] = fmaf(v.re, x[r].x, fmaf(v.im, x[r].y, are[q][r]));
          aim[q][r] = fmaf(v.re, x[r].y, fmaf(-v.im, x[r].x, aim[q][r]));
        }
      }
    }
  }
  const int n2 = 2 * N;
#pragma unroll
  for (int q = 0; q < KW; ++q) {
    const int k = w + 8 * q;
#pragma unroll
    for (int r = 0; r < RG; ++r) {
      const float sr = warp_sum(are[q][r]), si = warp_sum(aim[q][r]);
      if (lane == 0 && k < N && r < rg)
        out[(size_t)(r0 + r) * nblocks * n2 + (size_t)blk * n2 + chi * N + k] = make_float2(sr, si);
    }
  }
}

// K4': CTA (block, spin-colour component c): thread = site; out_r[c] =
// sum_k v_k[c] e_r[blk][chi(c)*N + k] for all right-hand sides; P read once.
template <class TV>
__global__ void __launch_bounds__(256) prolong0_mrhs_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                            const TV* __restrict__ Pv, int N, int nrhs,
                                                            int nblocks) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* es = reinterpret_cast<float2*>(smem_raw);              // [nrhs][N] of this chirality
  const int blk = MG_CLAMP(kAggregate, blockIdx.x, nblocks), c = blockIdx.y, loc = threadIdx.x;
  const int chi = c / 6, n2 = 2 * N;
  for (int e = loc; e < nrhs * N; e += 256) {
    const int r = e / N, k = e % N;
    es[e] = in[(size_t)r * nblocks * n2 + (size_t)blk * n2 + chi * N + k];
  }
  __syncthreads();
  const size_t fs = (size_t)nblocks * 12 * 256;
  for (int r0 = 0; r0 < nrhs; r0 += 12) {
    const int rc = min(12, nrhs - r0);
    float2 acc[12];
#pragma unroll
    for (int r = 0; r < 12; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < N; ++k) {
      const Cplx<float> v = Io<float, TV>::ld(Pv + ((size_t)(blk * N + k) * 12 + c) * 256 + loc);
#pragma unroll
      for (int r = 0; r < 12; ++r) {
        if (r < rc) {
          const float2 e = es[(r0 + r) * N + k];
          acc[r].x = fmaf(v.re, e.x, fmaf(-v.im, e.y, acc[r].x));
          acc[r].y = fmaf(v.re, e.y, fmaf(v.im, e.x, acc[r].y));
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 12; ++r)
      if (r < rc) out[(size_t)(r0 + r) * fs + ((size_t)blk * 12 + c) * 256 + loc] = acc[r];
  }
}

// K3'' (tensor cores): CTA (block, chirality), all right-hand sides (<= 16).
// With K' = 2K + (0 re, 1 im) over the 1536 complex entries of the chiral
// half-block, C = A B with A[k][K'] = the stored v_k (re/im interleaved, as P
// is stored) and B[2K][2r] = Re x_r(K), B[2K+1][2r] = Im x_r(K),
// B[2K][2r+1] = Im x_r(K), B[2K+1][2r+1] = -Re x_r(K) gives
// C[k][2r] = Re <v_k, x_r>, C[k][2r+1] = Im <v_k, x_r>.  mma.sync m16n8k8 TF32
// (FP16-stored P converts exactly); warp w takes the K steps w, w+8, ...;
// the warps' partial products are added in shared memory.
__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_m16n8k8_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                 uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Operands are staged in shared memory by asynchronous 16-byte copies
// (cp.async, kRStages-deep ring over K chunks of kRKC complex entries), so
// every global load is a coalesced 16-byte piece and the fragments come from
// shared memory.  Rows N..31 of P and R..15 of x stay zero in every stage.
constexpr int kRKC = 128;
constexpr int kRStages = 3;
template <class TV> struct RPad { static constexpr int sp = 132; };           // 4-byte P entries
template <> struct RPad<float2> { static constexpr int sp = 130; };           // 8-byte P entries
constexpr int kRSX = 132;                                                      // x row stride (float2)

template <class TV> __device__ __forceinline__ float2 p_ld(const TV* p) {
  const Cplx<float> v = Io<float, TV>::ldc(p);
  return make_float2(v.re, v.im);
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <class TV>
__host__ __device__ constexpr size_t restrict_stage_bytes() {
  return (size_t)32 * RPad<TV>::sp * sizeof(TV) + (size_t)16 * kRSX * sizeof(float2);
}

template <int NT, class TV>
__global__ void __launch_bounds__(256) restrict0_mma_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                            const TV* __restrict__ Pv, int N, int nrhs,
                                                            int nblocks) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int SP = RPad<TV>::sp;
  constexpr size_t PB = (size_t)32 * SP * sizeof(TV);
  constexpr size_t STAGE = restrict_stage_bytes<TV>();
  auto sP = [&](int st) { return reinterpret_cast<TV*>(smem_raw + st * STAGE); };
  auto sX = [&](int st) { return reinterpret_cast<float2*>(smem_raw + st * STAGE + PB); };
  const int blk = MG_CLAMP(kAggregate, blockIdx.x >> 1, nblocks), chi = blockIdx.x & 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tig = lane & 3, p1 = tig & 1;
  const size_t fs = (size_t)nblocks * 12 * 256;
  const size_t off = ((size_t)blk * 12 + 6 * chi) * 256;      // start of the chiral half-block
  // zero rows of P (>= N) and of x (>= nrhs) in every stage
  for (int st = 0; st < kRStages; ++st) {
    TV* P = sP(st);
    float2* X = sX(st);
    uint32_t* pz = reinterpret_cast<uint32_t*>(P + N * SP);
    for (int e = tid; e < (32 - N) * SP * (int)sizeof(TV) / 4; e += 256) pz[e] = 0u;
    for (int e = tid; e < (16 - nrhs) * kRSX; e += 256) X[nrhs * kRSX + e] = make_float2(0.f, 0.f);
  }
  constexpr int PP = kRKC * (int)sizeof(TV) / 16;             // 16-byte pieces per P row chunk
  constexpr int XP = kRKC * 8 / 16;                           // per x row chunk
  auto load = [&](int st, int kc0) {
    TV* P = sP(st);
    float2* X = sX(st);
    const int np = N * PP, total = np + nrhs * XP;
    for (int e = tid; e < total; e += 256) {
      if (e < np) {
        const int row = e / PP, pc = e % PP;
        const TV* src = Pv + ((size_t)(blk * N + row) * 12 + 6 * chi) * 256 + kc0;
        cp_async16(reinterpret_cast<unsigned char*>(P + row * SP) + pc * 16,
                   reinterpret_cast<const unsigned char*>(src) + pc * 16);
      } else {
        const int f = e - np, row = f / XP, pc = f % XP;
        const float2* src = in + (size_t)row * fs + off + kc0;
        cp_async16(reinterpret_cast<unsigned char*>(X + row * kRSX) + pc * 16,
                   reinterpret_cast<const unsigned char*>(src) + pc * 16);
      }
    }
  };
  constexpr int NC = 1536 / kRKC;
#pragma unroll
  for (int st = 0; st < kRStages - 1; ++st) {
    load(st, st * kRKC);
    cp_async_commit();
  }
  float acc[2][NT][4];
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < NT; ++q) acc[m][q][0] = acc[m][q][1] = acc[m][q][2] = acc[m][q][3] = 0.f;
  for (int c = 0; c < NC; ++c) {
    cp_async_wait<kRStages - 2>();
    __syncthreads();
    if (c + kRStages - 1 < NC) load((c + kRStages - 1) % kRStages, (c + kRStages - 1) * kRKC);
    cp_async_commit();
    const TV* P = sP(c % kRStages);
    const float2* X = sX(c % kRStages);
#pragma unroll
    for (int i = 0; i < kRKC / 32; ++i) {                     // this warp's k8 steps: warp + 8 i
      const int K = 4 * (warp + 8 * i) + (tig >> 1);          // complex entry of columns tig (and tig + 4: K + 2)
      uint32_t a[2][4];
#pragma unroll
      for (int m = 0; m < 2; ++m) {
        const int r0 = 16 * m + g, r1 = r0 + 8;
        const float2 x00 = p_ld(P + r0 * SP + K), x01 = p_ld(P + r0 * SP + K + 2);
        const float2 x10 = p_ld(P + r1 * SP + K), x11 = p_ld(P + r1 * SP + K + 2);
        a[m][0] = f32_to_tf32(p1 ? x00.y : x00.x);
        a[m][1] = f32_to_tf32(p1 ? x10.y : x10.x);
        a[m][2] = f32_to_tf32(p1 ? x01.y : x01.x);
        a[m][3] = f32_to_tf32(p1 ? x11.y : x11.x);
      }
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        const int col = 8 * q + g, r = col >> 1, pc = col & 1;
        const float2 x = X[r * kRSX + K], y = X[r * kRSX + K + 2];
        // B[2K+p1][2r+pc]: (pc, p1) = (0,0) re, (0,1) im, (1,0) im, (1,1) -re
        const float b0 = pc ? (p1 ? -x.x : x.y) : (p1 ? x.y : x.x);
        const float b1 = pc ? (p1 ? -y.x : y.y) : (p1 ? y.y : y.x);
        const uint32_t tb0 = f32_to_tf32(b0), tb1 = f32_to_tf32(b1);
#pragma unroll
        for (int m = 0; m < 2; ++m) mma_m16n8k8_tf32(acc[m][q], a[m][0], a[m][1], a[m][2], a[m][3], tb0, tb1);
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();
  // the warps' partial products, added by warp 0 in a fixed order
  float* red = reinterpret_cast<float*>(smem_raw);            // [8][2][NT][4][32]
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < NT; ++q)
#pragma unroll
      for (int f = 0; f < 4; ++f) red[(((warp * 2 + m) * NT + q) * 4 + f) * 32 + lane] = acc[m][q][f];
  __syncthreads();
  if (warp == 0) {
    const int n2 = 2 * N;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int q = 0; q < NT; ++q) {
        float sum[4] = {0.f, 0.f, 0.f, 0.f};
        for (int w = 0; w < 8; ++w)
#pragma unroll
          for (int f = 0; f < 4; ++f) sum[f] += red[(((w * 2 + m) * NT + q) * 4 + f) * 32 + lane];
        const int r = (8 * q + 2 * tig) >> 1;                  // columns 2 tig (re) and 2 tig + 1 (im)
        const int k0 = 16 * m + g, k1 = k0 + 8;
        if (r < nrhs) {
          float2* o = out + (size_t)r * nblocks * n2 + (size_t)blk * n2 + chi * N;
          if (k0 < N) o[k0] = make_float2(sum[0], sum[1]);
          if (k1 < N) o[k1] = make_float2(sum[2], sum[3]);
        }
      }
  }
}

// K4'' (tensor cores): interpolation of all right-hand sides (<= 16) for one
// (aggregate, chirality) per CTA.  With the real embedding A[2K+a][2k+b] of P
// ((0,0) Re, (0,1) -Im, (1,0) Im, (1,1) Re of P(K, k)) and B[2k][r] = Re e_r(k),
// B[2k+1][r] = Im e_r(k), Y = A B gives Y[2K][r] = Re out_r(K) and
// Y[2K+1][r] = Im out_r(K).  mma.sync m16n8k8 TF32 (FP16-stored P converts
// exactly); P is staged per chunk of kRKC entries by cp.async; B is loaded
// into registers once.  Neighbouring lanes (real and imaginary rows of one K)
// swap halves by a shuffle so that each stores whole complex numbers.
__device__ __forceinline__ float embed_pr(float2 m, int a, int b) { return a == b ? m.x : (a ? m.y : -m.y); }

template <class TV>
__host__ __device__ constexpr size_t prolong_stage_bytes(int Np) {
  return (size_t)Np * RPad<TV>::sp * sizeof(TV);
}

template <int NT, class TV>
__global__ void __launch_bounds__(256) prolong0_mma_kernel(const float2* __restrict__ in, float2* __restrict__ out,
                                                           const TV* __restrict__ Pv, int N, int nrhs, int nblocks) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int SP = RPad<TV>::sp;
  const int Np = (N + 3) & ~3;                                 // k padded to whole k8 steps of the embedding
  const size_t PB = prolong_stage_bytes<TV>(Np);
  auto sP = [&](int st) { return reinterpret_cast<TV*>(smem_raw + st * PB); };
  float* eb = reinterpret_cast<float*>(smem_raw + kRStages * PB);   // [2 Np][16]
  const int blk = MG_CLAMP(kAggregate, blockIdx.x >> 1, nblocks), chi = blockIdx.x & 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tig = lane & 3, a = g & 1;
  const size_t fs = (size_t)nblocks * 12 * 256;
  const size_t off = ((size_t)blk * 12 + 6 * chi) * 256;
  const int n2 = 2 * N;
  for (int e = tid; e < 2 * Np * 16; e += 256) {
    const int kk = e >> 4, r = e & 15, k = kk >> 1;
    float v = 0.f;
    if (k < N && r < nrhs) {
      const float2 x = in[(size_t)r * nblocks * n2 + (size_t)blk * n2 + chi * N + k];
      v = (kk & 1) ? x.y : x.x;
    }
    eb[e] = v;
  }
  for (int st = 0; st < kRStages; ++st) {
    uint32_t* pz = reinterpret_cast<uint32_t*>(sP(st) + N * SP);
    for (int e = tid; e < (Np - N) * SP * (int)sizeof(TV) / 4; e += 256) pz[e] = 0u;
  }
  constexpr int PP = kRKC * (int)sizeof(TV) / 16;
  auto load = [&](int st, int kc0) {
    TV* P = sP(st);
    for (int e = tid; e < N * PP; e += 256) {
      const int row = e / PP, pc = e % PP;
      const TV* src = Pv + ((size_t)(blk * N + row) * 12 + 6 * chi) * 256 + kc0;
      cp_async16(reinterpret_cast<unsigned char*>(P + row * SP) + pc * 16,
                 reinterpret_cast<const unsigned char*>(src) + pc * 16);
    }
  };
  constexpr int NC = 1536 / kRKC;
#pragma unroll
  for (int st = 0; st < kRStages - 1; ++st) {
    load(st, st * kRKC);
    cp_async_commit();
  }
  __syncthreads();                                             // eb written
  const int KS = Np / 4;                                       // k8 steps (<= 8)
  uint32_t bf[8][NT][2];
#pragma unroll
  for (int ks = 0; ks < 8; ++ks)
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
      if (ks < KS) {
        bf[ks][nt][0] = f32_to_tf32(eb[(8 * ks + tig) * 16 + 8 * nt + g]);
        bf[ks][nt][1] = f32_to_tf32(eb[(8 * ks + tig + 4) * 16 + 8 * nt + g]);
      } else {
        bf[ks][nt][0] = bf[ks][nt][1] = 0u;
      }
    }
  for (int c = 0; c < NC; ++c) {
    cp_async_wait<kRStages - 2>();
    __syncthreads();
    if (c + kRStages - 1 < NC) load((c + kRStages - 1) % kRStages, (c + kRStages - 1) * kRKC);
    cp_async_commit();
    const TV* P = sP(c % kRStages);
    for (int mt = warp; mt < kRKC / 8; mt += 8) {              // 16-row tiles of the 2 kRKC real rows
      const int Kl = 8 * mt + (g >> 1);                        // rows g (K = Kl) and g + 8 (K = Kl + 4)
      float acc[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        if (ks < KS) {
          const int k = 4 * ks + (tig >> 1), b = tig & 1;       // columns tig (k) and tig + 4 (k + 2)
          const uint32_t a0 = f32_to_tf32(embed_pr(p_ld(P + k * SP + Kl), a, b));
          const uint32_t a1 = f32_to_tf32(embed_pr(p_ld(P + k * SP + Kl + 4), a, b));
          const uint32_t a2 = f32_to_tf32(embed_pr(p_ld(P + (k + 2) * SP + Kl), a, b));
          const uint32_t a3 = f32_to_tf32(embed_pr(p_ld(P + (k + 2) * SP + Kl + 4), a, b));
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma_m16n8k8_tf32(acc[nt], a0, a1, a2, a3, bf[ks][nt][0], bf[ks][nt][1]);
        }
      }
      // lane with a = 0 holds Re, its partner (lane ^ 4) Im, of out_r(K) for r = r0, r0 + 1
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) {
        const int r0 = 8 * nt + 2 * tig, rw = r0 + a;
#pragma unroll
        for (int h = 0; h < 2; ++h) {                          // rows K = Kl (h = 0) and Kl + 4
          const float v0 = acc[nt][2 * h], v1 = acc[nt][2 * h + 1];
          const float send = a ? v0 : v1;
          const float recv = __shfl_xor_sync(0xffffffffu, send, 4);
          const float2 o = a ? make_float2(recv, v1) : make_float2(v0, recv);
          if (rw < nrhs) out[(size_t)rw * fs + off + c * kRKC + Kl + 4 * h] = o;
        }
      }
    }
  }
  cp_async_wait<0>();
}

template <class TV>
static int transfer0_mrhs(bool restrict_, const Geom& g, const void* in, void* out, const void* Pv, int N, int nrhs,
                          bool tf32, cudaStream_t s) {
  if (restrict_ && tf32 && nrhs <= 16 && N <= 32) {
    const unsigned grid = (unsigned)(g.nblocks * 2);
    const size_t smem = kRStages * restrict_stage_bytes<TV>();
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(restrict0_mma_kernel<1, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(restrict0_mma_kernel<2, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(restrict0_mma_kernel<3, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      cudaFuncSetAttribute(restrict0_mma_kernel<4, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    const float2* xi = (const float2*)in;
    float2* xo = (float2*)out;
    const TV* pv = (const TV*)Pv;
    if (nrhs <= 4) { restrict0_mma_kernel<1, TV><<<grid, 256, smem, s>>>(xi, xo, pv, N, nrhs, g.nblocks); count_launches(1); }
    else if (nrhs <= 8) { restrict0_mma_kernel<2, TV><<<grid, 256, smem, s>>>(xi, xo, pv, N, nrhs, g.nblocks); count_launches(1); }
    else if (nrhs <= 12) { restrict0_mma_kernel<3, TV><<<grid, 256, smem, s>>>(xi, xo, pv, N, nrhs, g.nblocks); count_launches(1); }
    else { restrict0_mma_kernel<4, TV><<<grid, 256, smem, s>>>(xi, xo, pv, N, nrhs, g.nblocks); count_launches(1); }
    SAPMG_CUDA_TRY(cudaGetLastError());
    return MG_OK;
  }
  if (restrict_) {
    constexpr int RG = 4;
    const size_t smem = sizeof(float2) * RG * 1536;
    const unsigned grid = (unsigned)(g.nblocks * 2 * ((nrhs + RG - 1) / RG));
    restrict0_mrhs_kernel<RG, TV><<<grid, 256, smem, s>>>((const float2*)in, (float2*)out, (const TV*)Pv, N, nrhs,
                                                          g.nblocks); count_launches(1);
  } else if (tf32 && nrhs <= 16 && N <= 32) {
    const int Np = (N + 3) & ~3;
    const size_t smem = kRStages * prolong_stage_bytes<TV>(Np) + sizeof(float) * 2 * Np * 16;
    const unsigned grid = (unsigned)(g.nblocks * 2);
    static bool pattr = false;
    if (!pattr) {                                 // enough for N = 32
      const int mx = (int)(kRStages * prolong_stage_bytes<TV>(32) + sizeof(float) * 2 * 32 * 16);
      cudaFuncSetAttribute(prolong0_mma_kernel<1, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      cudaFuncSetAttribute(prolong0_mma_kernel<2, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
      pattr = true;
    }
    if (nrhs <= 8) {
      prolong0_mma_kernel<1, TV><<<grid, 256, smem, s>>>((const float2*)in, (float2*)out, (const TV*)Pv, N, nrhs,
                                                          g.nblocks); count_launches(1);
    } else {
      prolong0_mma_kernel<2, TV><<<grid, 256, smem, s>>>((const float2*)in, (float2*)out, (const TV*)Pv, N, nrhs,
                                                          g.nblocks); count_launches(1);
    }
  } else {
    const size_t smem = sizeof(float2) * nrhs * N;
    dim3 grid(g.nblocks, 12);
    prolong0_mrhs_kernel<TV><<<grid, 256, smem, s>>>((const float2*)in, (float2*)out, (const TV*)Pv, N, nrhs,
                                                     g.nblocks); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

template <class R, class TS, class TV, class TC>
static int transfer0_run(bool restrict_, const Geom& g, const void* in, void* out, const void* Pv, int N, int nrhs,
                         cudaStream_t s) {
  const unsigned grid = (unsigned)(g.nblocks * nrhs);   // right-hand side fastest: P shared through L2
  if (restrict_) {
    const size_t smem = sizeof(R) * 4 * 8 * N;
    restrict0_kernel<R, TS, TV, TC><<<grid, 256, smem, s>>>((const TS*)in, (TC*)out, (const TV*)Pv, N, nrhs,
                                                            g.nblocks); count_launches(1);
  } else {
    const size_t smem = sizeof(Cplx<R>) * 2 * N;
    prolong0_kernel<R, TS, TV, TC><<<grid, 256, smem, s>>>((const TC*)in, (TS*)out, (const TV*)Pv, N, nrhs,
                                                           g.nblocks); count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_transfer0(bool restrict_, int prec, const Geom& g, const void* in, void* out, const void* Pv, int N,
                     int nrhs, bool tf32, cudaStream_t s) {
  // several right-hand sides in the mixed form: the forms that read P once
  if (nrhs > 1 && prec != P64 && N <= 24) {
    switch (prec) {
      case P32: return transfer0_mrhs<float2>(restrict_, g, in, out, Pv, N, nrhs, tf32, s);
      case P16: return transfer0_mrhs<__half2>(restrict_, g, in, out, Pv, N, nrhs, tf32, s);
      case PBF: return transfer0_mrhs<__nv_bfloat162>(restrict_, g, in, out, Pv, N, nrhs, tf32, s);
      default: break;
    }
  }
  switch (prec) {
    case P64: return transfer0_run<double, double2, double2, double2>(restrict_, g, in, out, Pv, N, nrhs, s);
    case P32: return transfer0_run<float, float2, float2, float2>(restrict_, g, in, out, Pv, N, nrhs, s);
    case P16: return transfer0_run<float, float2, __half2, float2>(restrict_, g, in, out, Pv, N, nrhs, s);
    case PBF: return transfer0_run<float, float2, __nv_bfloat162, float2>(restrict_, g, in, out, Pv, N, nrhs, s);
    default: return MG_ERR_ARG;
  }
}

// K7: modified Gram-Schmidt of the N vectors on every (block, chirality),
// vectors k = 0..N-1 in order, each normalised to a positive real norm.
// V: FP64 vector-major blocked fields [k][blk][12][256].
__device__ __forceinline__ double2 block_sum2(double a, double b, double (*red)[2]) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[w][0] = a; red[w][1] = b; }
  __syncthreads();
  double sa = 0, sb = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { sa += red[q][0]; sb += red[q][1]; }
  __syncthreads();
  return make_double2(sa, sb);
}

__global__ void __launch_bounds__(256) block_gs0_kernel(double2* __restrict__ V, int N, long long fstride) {
  __shared__ double red[8][2];
  const int blk = blockIdx.x, chi = blockIdx.y, loc = threadIdx.x;
  const size_t base = ((size_t)blk * 12 + 6 * chi) * 256 + loc;
  for (int k = 0; k < N; ++k) {
    double2* vk = V + k * fstride + base;
    Cplx<double> x[6];
    for (int c = 0; c < 6; ++c) { double2 t = vk[c * 256]; x[c] = cmk(t.x, t.y); }
    for (int j = 0; j < k; ++j) {
      const double2* vj = V + j * fstride + base;
      Cplx<double> q[6], d = cmk(0.0, 0.0);
      for (int c = 0; c < 6; ++c) { double2 t = vj[c * 256]; q[c] = cmk(t.x, t.y); cfma_conj(d, q[c], x[c]); }
      const double2 s = block_sum2(d.re, d.im, red);
      const Cplx<double> cs = cmk(s.x, s.y);
      for (int c = 0; c < 6; ++c) x[c] = x[c] - cs * q[c];
    }
    double nn = 0;
    for (int c = 0; c < 6; ++c) nn += x[c].re * x[c].re + x[c].im * x[c].im;
    const double2 s = block_sum2(nn, 0.0, red);
    const double inv = s.x > 0 ? 1.0 / sqrt(s.x) : 0.0;
    for (int c = 0; c < 6; ++c) vk[c * 256] = make_double2(x[c].re * inv, x[c].im * inv);
  }
}

int launch_block_gs0(const Geom& g, void* V64, int N, cudaStream_t s) {
  dim3 grid(g.nblocks, 2);
  block_gs0_kernel<<<grid, 256, 0, s>>>((double2*)V64, N, (long long)g.V * 12); count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Reorder the FP64 vector-major vectors into the block-major storage Pv[blk][k][12][256].
template <class TV>
__global__ void store_p0_kernel(const double2* __restrict__ V, TV* __restrict__ Pv, int N, long long fstride) {
  const int blk = blockIdx.x, k = blockIdx.y, loc = threadIdx.x;
  const double2* src = V + k * fstride + (size_t)blk * 12 * 256 + loc;
  TV* dst = Pv + ((size_t)(blk * N + k) * 12) * 256 + loc;
  for (int c = 0; c < 12; ++c) {
    const double2 t = src[c * 256];
    Io<double, TV>::st(dst + c * 256, cmk(t.x, t.y));
  }
}

int launch_store_p0(int prec, const Geom& g, const void* V64, void* Pv, int N, cudaStream_t s) {
  dim3 grid(g.nblocks, N);
  const long long fs = (long long)g.V * 12;
  switch (prec) {
    case P64: store_p0_kernel<double2><<<grid, 256, 0, s>>>((const double2*)V64, (double2*)Pv, N, fs); count_launches(1); break;
    case P32: store_p0_kernel<float2><<<grid, 256, 0, s>>>((const double2*)V64, (float2*)Pv, N, fs); count_launches(1); break;
    case P16: store_p0_kernel<__half2><<<grid, 256, 0, s>>>((const double2*)V64, (__half2*)Pv, N, fs); count_launches(1); break;
    case PBF: store_p0_kernel<__nv_bfloat162><<<grid, 256, 0, s>>>((const double2*)V64, (__nv_bfloat162*)Pv, N, fs); count_launches(1); break;
    default: return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// K6: D_c = P^dagger D P for level 0 -> 1, FP64.  CTA (a, j): column j = (chi', k)
// of every 2N x 2N block row of aggregate a.  Each thread (site x of a) forms
// the 9 partial images of u = v_k|_chi' (self: clover and hops inside a; +-mu:
// the hop from the neighbouring aggregate across a's face) and projects each
// onto the 2N columns of P on a.
template <int MU, int S, class R, class T2>
__device__ __forceinline__ void assemble_hop(const Geom& g, const T2* __restrict__ U, const T2* vk,
                                             int chi_p, int blk, int loc, bool inside, Cplx<R> (&w)[12]) {
  int nb, nl;
  neighbour(g, blk, loc, MU, S, nb, nl);
  if ((nb == blk) != inside) return;
  Cplx<R> u[12];
  load_spinor<R>(vk, nb, nl, u);
#pragma unroll
  for (int c = 0; c < 12; ++c)
    if ((c / 6) != chi_p) u[c] = cmk<R>(0, 0);
  Cplx<R> acc[12];
#pragma unroll
  for (int c = 0; c < 12; ++c) acc[c] = cmk<R>(0, 0);
  if (S > 0) hop_fwd<MU>(U, blk, loc, u, acc);
  else hop_bwd<MU>(U, nb, nl, u, acc);
#pragma unroll
  for (int c = 0; c < 12; ++c) w[c] = w[c] - (R)0.5 * acc[c];
}

template <int MU, class R, class T2>
__device__ __forceinline__ void assemble_dir(const Geom& g, const T2* U, const T2* vk, int chi_p, int blk,
                                             int loc, int d, Cplx<R> (&w)[12]) {
  if (d == 0) {
    assemble_hop<MU, 1>(g, U, vk, chi_p, blk, loc, true, w);
    assemble_hop<MU, -1>(g, U, vk, chi_p, blk, loc, true, w);
  } else if (d == 1 + 2 * MU) {
    assemble_hop<MU, 1>(g, U, vk, chi_p, blk, loc, false, w);
  } else if (d == 2 + 2 * MU) {
    assemble_hop<MU, -1>(g, U, vk, chi_p, blk, loc, false, w);
  }
}

// R = double with FP64 vectors and fields (the plain form, exact to rounding);
// R = float with FP32 copies (the mixed form, whose coarse operator is stored
// in FP32 and FP16: FP64 arithmetic is scarce on this GPU).  The entries are
// written in FP64 either way.
template <class R, class T2>
__global__ void __launch_bounds__(256) assemble0_kernel(const T2* __restrict__ V, const T2* __restrict__ U,
                                                        const T2* __restrict__ A, double2* __restrict__ M,
                                                        Geom g, int N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double (*red)[4] = reinterpret_cast<double (*)[4]>(smem_raw);   // [8 * N][4]
  const int blk = MG_CLAMP(kAggregate, blockIdx.x, g.nblocks), j = blockIdx.y, loc = threadIdx.x;
  const int n2 = 2 * N, chi_p = j / N, k = j % N;
  const int wid = loc >> 5, lane = loc & 31;
  const long long fs = g.V * 12;
  const T2* vk = V + k * fs;
  for (int d = 0; d < 9; ++d) {
    Cplx<R> w[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) w[c] = cmk<R>(0, 0);
    if (d == 0) {
      Cplx<R> u[12];
      load_spinor<R>(vk, blk, loc, u);
#pragma unroll
      for (int c = 0; c < 12; ++c)
        if ((c / 6) != chi_p) u[c] = cmk<R>(0, 0);
      clover_apply<R>(A, blk, loc, u, w);
    }
    assemble_dir<0>(g, U, vk, chi_p, blk, loc, d, w);
    assemble_dir<1>(g, U, vk, chi_p, blk, loc, d, w);
    assemble_dir<2>(g, U, vk, chi_p, blk, loc, d, w);
    assemble_dir<3>(g, U, vk, chi_p, blk, loc, d, w);
    // project onto v_i|_chi on this block; for d > 0 only the sites on the
    // block's face towards direction d have a non-zero image (the others would
    // add exact zeros, so skipping them changes no bit)
    bool live = true;
    if (d > 0) {
      const int mu = (d - 1) >> 1, cmu = (loc >> (2 * mu)) & 3;
      live = (d & 1) ? cmu == 3 : cmu == 0;
    }
    for (int i = 0; i < N; ++i) {
      const T2* vi = V + i * fs + (size_t)blk * 12 * 256 + loc;
      Cplx<R> d0 = cmk<R>(0, 0), d1 = cmk<R>(0, 0);
      if (live) {
#pragma unroll
        for (int c = 0; c < 6; ++c) { const T2 t = vi[c * 256]; cfma_conj(d0, cmk<R>(t.x, t.y), w[c]); }
#pragma unroll
        for (int c = 6; c < 12; ++c) { const T2 t = vi[c * 256]; cfma_conj(d1, cmk<R>(t.x, t.y), w[c]); }
      }
      const R a = warp_sum(d0.re), b = warp_sum(d0.im), c2 = warp_sum(d1.re), e = warp_sum(d1.im);
      if (lane == 0) { double* q = red[wid * N + i]; q[0] = a; q[1] = b; q[2] = c2; q[3] = e; }
    }
    __syncthreads();
    double2* col = M + (((size_t)blk * 9 + d) * n2 + j) * n2;
    for (int t = loc; t < n2; t += 256) {
      const int chi = t / N, i = t % N;
      double sr = 0, si = 0;
      for (int q = 0; q < 8; ++q) { sr += red[q * N + i][2 * chi]; si += red[q * N + i][2 * chi + 1]; }
      col[t] = make_double2(sr, si);
    }
    __syncthreads();
  }
}

int launch_assemble0(const Geom& g, int prec, const void* V, const void* U, const void* A, void* M64, int N,
                     cudaStream_t s) {
  dim3 grid(g.nblocks, 2 * N);
  const size_t smem = sizeof(double) * 4 * 8 * N;
  if (prec == P64)
    assemble0_kernel<double, double2><<<grid, 256, smem, s>>>((const double2*)V, (const double2*)U,
                                                              (const double2*)A, (double2*)M64, g, N);
  else if (prec == P32)
    assemble0_kernel<float, float2><<<grid, 256, smem, s>>>((const float2*)V, (const float2*)U, (const float2*)A,
                                                            (double2*)M64, g, N);
  else
    return MG_ERR_ARG;
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// ============================================================ coarse levels
__device__ __forceinline__ int cg_coord(const CGeom& c, int site, int mu) {
  int s = site;
  for (int m = 0; m < mu; ++m) s /= c.L[m];
  return s % c.L[mu];
}

// Site index of the neighbour of `site` in direction d (0 self, 1+2mu: +mu, 2+2mu: -mu).
__device__ __forceinline__ int cg_neighbour(const CGeom& c, int site, int d) {
  if (d == 0) return site;
  const int mu = (d - 1) >> 1;
  const int step = (d & 1) ? 1 : -1;
  int stride = 1;
  for (int m = 0; m < mu; ++m) stride *= c.L[m];
  const int x = (site / stride) % c.L[mu];
  const int nx = (x + step + c.L[mu]) % c.L[mu];
  return MG_CLAMP(kCoarseNeighbour, site + (nx - x) * stride, c.nsites);
}

// K5: out_r[site][i] = sum_d sum_j M[site][d][j][i] x_r[nb_d(site)][j] for RB
// right-hand sides at once: every matrix entry is loaded once and applied to
// all RB vectors (the operator dominates the traffic; the vectors stay in L2).
template <class R, class TM, class TX, int RB>
__global__ void __launch_bounds__(256) coarse_apply_kernel(const TM* __restrict__ M, const TX* __restrict__ x,
                                                           TX* __restrict__ out, CGeom c, int r0) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int n2 = c.n2;
  if (t >= (long long)c.nsites * n2) return;
  const int site = (int)(t / n2), i = (int)(t % n2);
  const size_t fs = (size_t)c.nsites * n2;
  const TX* xr = x + (size_t)r0 * fs;
  Cplx<R> acc[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) acc[r] = cmk<R>(0, 0);
  for (int d = 0; d < 9; ++d) {
    const int nb = cg_neighbour(c, site, d);
    const TM* m = M + (((size_t)site * 9 + d) * n2) * n2 + i;
    const TX* xn = xr + (size_t)nb * n2;
#pragma unroll 4
    for (int j = 0; j < n2; ++j) {
      const Cplx<R> mv = Io<R, TM>::ld(m + (size_t)j * n2);
#pragma unroll
      for (int r = 0; r < RB; ++r) cfma(acc[r], mv, Io<R, TX>::ld(xn + r * fs + j));
    }
  }
#pragma unroll
  for (int r = 0; r < RB; ++r) Io<R, TX>::st(out + (size_t)(r0 + r) * fs + t, acc[r]);
}

template <class R, class TM, class TX>
static void coarse_apply_t(const CGeom& c, const void* M, const void* x, void* out, int nrhs, cudaStream_t s) {
  const long long n = (long long)c.nsites * c.n2;
  const unsigned grid = (unsigned)((n + 255) / 256);
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    const TM* m = (const TM*)M;
    const TX* xi = (const TX*)x;
    TX* o = (TX*)out;
    if (left >= 12) { coarse_apply_kernel<R, TM, TX, 12><<<grid, 256, 0, s>>>(m, xi, o, c, r0); count_launches(1); r0 += 12; }
    else if (left >= 4) { coarse_apply_kernel<R, TM, TX, 4><<<grid, 256, 0, s>>>(m, xi, o, c, r0); count_launches(1); r0 += 4; }
    else if (left >= 2) { coarse_apply_kernel<R, TM, TX, 2><<<grid, 256, 0, s>>>(m, xi, o, c, r0); count_launches(1); r0 += 2; }
    else { coarse_apply_kernel<R, TM, TX, 1><<<grid, 256, 0, s>>>(m, xi, o, c, r0); count_launches(1); r0 += 1; }
  }
}

int launch_coarse_apply(int prec, const CGeom& c, const void* M, const void* x, void* out, int nrhs, cudaStream_t s) {
  switch (prec) {
    case P64: coarse_apply_t<double, double2, double2>(c, M, x, out, nrhs, s); break;
    case P32: coarse_apply_t<float, float2, float2>(c, M, x, out, nrhs, s); break;
    case P16: coarse_apply_t<float, __half2, float2>(c, M, x, out, nrhs, s); break;
    case PBF: coarse_apply_t<float, __nv_bfloat162, float2>(c, M, x, out, nrhs, s); break;
    default: return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Dense row-major FP64 export [site][9][i][j] of a column-major operator.
template <class TM>
__global__ void coarse_export_kernel(const TM* __restrict__ M, double2* __restrict__ out, CGeom c) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n2 = c.n2;
  if (t >= (long long)c.nsites * 9 * n2 * n2) return;
  const long long sd = t / (n2 * n2);
  const int i = (int)((t / n2) % n2), j = (int)(t % n2);
  const Cplx<double> v = Io<double, TM>::ld(M + (sd * n2 + j) * n2 + i);
  out[t] = make_double2(v.re, v.im);
}

int launch_coarse_export(int prec, const CGeom& c, const void* M, double* out, cudaStream_t s) {
  const long long n = (long long)c.nsites * 9 * c.n2 * c.n2;
  const unsigned nb = (unsigned)((n + 255) / 256);
  switch (prec) {
    case P64: coarse_export_kernel<double2><<<nb, 256, 0, s>>>((const double2*)M, (double2*)out, c); count_launches(1); break;
    case P32: coarse_export_kernel<float2><<<nb, 256, 0, s>>>((const float2*)M, (double2*)out, c); count_launches(1); break;
    case P16: coarse_export_kernel<__half2><<<nb, 256, 0, s>>>((const __half2*)M, (double2*)out, c); count_launches(1); break;
    case PBF: coarse_export_kernel<__nv_bfloat162><<<nb, 256, 0, s>>>((const __nv_bfloat162*)M, (double2*)out, c); count_launches(1); break;
    default: return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Blocked FP64 vector-major -> canonical FP64 export of the level-0 vectors.
}  // namespace sapmg
