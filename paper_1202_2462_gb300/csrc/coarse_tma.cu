// K5 (FP32 operator): the coarse stencil (D_c x)(a) = sum_d M_d(a) x(a + offset_d)
// (Sec. 3: D_c couples nearest-neighbour aggregates only) for up to 12
// right-hand sides, with every 2N x 2N block M_d(a) streamed from HBM once.
//
// Each CTA walks its sites and, per site, the 9 blocks (self, +-mu).  One
// elected thread copies block k+1 into shared memory with a bulk asynchronous
// copy (cp.async.bulk, completion counted on an mbarrier) while all threads
// compute with block k (double buffering).  The right-hand sides' neighbour
// vectors are staged in shared memory; thread (group gq, row i) owns APT
// accumulators out_r[i] for r = gq*APT .. gq*APT+APT-1.  Every wait on an
// mbarrier is bounded: when it gives up the kernel raises an error flag that
// the host turns into MG_ERR_TIMEOUT.
#include "internal.h"
#include "coarse.h"
#include "async.cuh"

namespace sapmg {


template <int RB, int APT>
__global__ void __launch_bounds__(256) coarse_apply_tma_kernel(const float2* __restrict__ M,
                                                               const float2* __restrict__ x,
                                                               float2* __restrict__ out, CGeom c, int r0,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int spins = wait_spins(err);
  __shared__ __align__(8) uint64_t bar[2];
  const int n2 = c.n2;
  const int tile = n2 * n2;                                   // complex entries per block
  const uint32_t tile_bytes = (uint32_t)tile * sizeof(float2);
  float2* buf0 = reinterpret_cast<float2*>(smem);
  float2* buf1 = buf0 + tile;
  float2* xs = buf1 + tile;                                   // [RB][n2]
  const int tid = threadIdx.x;
  const int gq = tid / n2, i = tid % n2;
  const bool active = (gq * APT < RB) && (tid < ((RB + APT - 1) / APT) * n2);
  const size_t fs = (size_t)c.nsites * n2;
  const float2* xr = x + (size_t)r0 * fs;

  const int nsite_cta = (c.nsites - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int T = 9 * nsite_cta;
  if (T <= 0) return;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto tile_src = [&](int t) {
    const int site = MG_CLAMP(kCoarseSite, (int)blockIdx.x + (t / 9) * (int)gridDim.x, c.nsites);
    return M + ((size_t)site * 9 + (t % 9)) * tile;
  };
  if (tid == 0) {
    mbar_expect_tx(&bar[0], tile_bytes);
    bulk_copy_g2s(buf0, tile_src(0), tile_bytes, &bar[0]);
  }
  float acc_re[APT], acc_im[APT];
  int tfail = -1;
  for (int t = 0; t < T; ++t) {
    const int d = t % 9;
    const int site = MG_CLAMP(kCoarseSite, (int)blockIdx.x + (t / 9) * (int)gridDim.x, c.nsites);
    if (d == 0) {
#pragma unroll
      for (int a = 0; a < APT; ++a) acc_re[a] = acc_im[a] = 0.f;
    }
    // prefetch block t+1 into the other buffer (its last readers finished at the
    // barrier that closed step t-1)
    if (tid == 0 && t + 1 < T) {
      uint64_t* b = &bar[(t + 1) & 1];
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(b, tile_bytes);
      bulk_copy_g2s(((t + 1) & 1) ? buf1 : buf0, tile_src(t + 1), tile_bytes, b);
    }
    // stage the neighbour vectors of every right-hand side
    {
      int nb = site;
      if (d > 0) {
        const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
        int stride = 1;
        for (int m = 0; m < mu; ++m) stride *= c.L[m];
        const int xc = (site / stride) % c.L[mu];
        nb = site + (((xc + step + c.L[mu]) % c.L[mu]) - xc) * stride;
      }
      nb = MG_CLAMP(kCoarseNeighbour, nb, c.nsites);
      for (int e = tid; e < RB * n2; e += blockDim.x) xs[e] = xr[(size_t)(e / n2) * fs + (size_t)nb * n2 + e % n2];
    }
    const bool waited = mbar_wait(&bar[t & 1], (uint32_t)((t >> 1) & 1), spins);
    if (__syncthreads_or(!waited)) {          // uniform decision: every thread leaves together
      tfail = t;
      break;
    }
    const float2* mt = (t & 1) ? buf1 : buf0;
    if (active) {
#pragma unroll 4
      for (int j = 0; j < n2; ++j) {
        const float2 mv = mt[j * n2 + i];
#pragma unroll
        for (int a = 0; a < APT; ++a) {
          const int r = gq * APT + a;
          if (r < RB) {
            const float2 xv = xs[r * n2 + j];
            acc_re[a] = fmaf(mv.x, xv.x, fmaf(-mv.y, xv.y, acc_re[a]));
            acc_im[a] = fmaf(mv.x, xv.y, fmaf(mv.y, xv.x, acc_im[a]));
          }
        }
      }
    }
    if (d == 8 && active) {
#pragma unroll
      for (int a = 0; a < APT; ++a) {
        const int r = gq * APT + a;
        if (r < RB) out[(size_t)(r0 + r) * fs + (size_t)site * n2 + i] = make_float2(acc_re[a], acc_im[a]);
      }
    }
    __syncthreads();
  }
  if (tfail >= 0) {
    // let the copies still in flight (blocks tfail and tfail + 1) land before
    // the CTA exits; these waits are bounded as well
    if (tid == 0) {
      atomicExch(err, 1);
      mbar_wait(&bar[tfail & 1], (uint32_t)((tfail >> 1) & 1));
      if (tfail + 1 < T) mbar_wait(&bar[(tfail + 1) & 1], (uint32_t)(((tfail + 1) >> 1) & 1));
    }
    __syncthreads();
  }
}

template <int RB, int APT>
static void launch_tma(const CGeom& c, const float2* M, const float2* x, float2* out, int r0, int* err,
                       cudaStream_t s) {
  const size_t smem = (size_t)(2 * c.n2 * c.n2 + RB * c.n2) * sizeof(float2);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(coarse_apply_tma_kernel<RB, APT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (220 * 1024) / (smem + 1024)));
  const int grid = std::min(c.nsites, 152 * per_sm);
  coarse_apply_tma_kernel<RB, APT><<<grid, 256, smem, s>>>(M, x, out, c, r0, err); count_launches(1);
}

// ---------------------------------------------------------------- tensor-core form
// The same stencil with the per-block products on tensor cores
// (mma.sync m16n8k8, TF32 inputs, FP32 accumulation).  For one block M_d(a)
// and the RB right-hand sides the complex product out += M x is the real
// product Y += A X with
//   A[2i][2j] = Re M_ij, A[2i][2j+1] = -Im M_ij, A[2i+1][2j] = Im M_ij,
//   A[2i+1][2j+1] = Re M_ij,   X[2j][r] = Re x_r(j), X[2j+1][r] = Im x_r(j),
// Y[2i][r] = Re out_r(i), Y[2i+1][r] = Im out_r(i): 2n2 x 2n2 times 2n2 x 16.
// Warp w owns rows 16w..16w+15 of Y (both 8-column tiles); the 9 blocks of a
// site accumulate in the same fragments.  Needs n2 % 8 == 0.  The operator may
// be stored in FP16 (half the HBM traffic; FP16 values are exact in TF32).
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// component (a, b) of the real embedding of complex m: (0,0) re, (0,1) -im, (1,0) im, (1,1) re
__device__ __forceinline__ float embed(float2 m, int a, int b) {
  return a == b ? m.x : (a ? m.y : -m.y);
}

__device__ __forceinline__ float2 tile_ld(const float2* t, int k) { return t[k]; }
__device__ __forceinline__ float2 tile_ld(const __half2* t, int k) { return __half22float2(t[k]); }

// Pipeline: a ring of kStages stages, each holding one operator block (FP32
// or FP16 entries; FP16 converts exactly to TF32) and the RB neighbour
// vectors it multiplies.  One thread issues all bulk copies of block
// t + kStages - 1 (block + RB vector rows, one transaction count on that
// stage's mbarrier) while the warps multiply block t; a block's stage is
// refilled only after the CTA-wide barrier that ends its use.  Two stages keep
// a CTA's shared memory small, so that many CTAs share an SM (measured faster
// than deeper rings with fewer CTAs).
constexpr int kStages = 2;

template <int RB, class TM>
__global__ void __launch_bounds__(256) coarse_apply_mma_kernel(const TM* __restrict__ M,
                                                               const float2* __restrict__ x,
                                                               float2* __restrict__ out, CGeom c, int r0, int nr,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int spins = wait_spins(err);
  __shared__ __align__(8) uint64_t bar[kStages];
  const int n2 = c.n2;
  const int xst = n2 + 2;                                     // padded row stride of the staged vectors
  const int tile = n2 * n2;
  const uint32_t tile_bytes = (uint32_t)tile * sizeof(TM);
  const uint32_t row_bytes = (uint32_t)n2 * sizeof(float2);
  const size_t stage_bytes = tile_bytes + (size_t)16 * xst * sizeof(float2);
  auto stage_tile = [&](int st) { return reinterpret_cast<TM*>(smem + st * stage_bytes); };
  auto stage_x = [&](int st) { return reinterpret_cast<float2*>(smem + st * stage_bytes + tile_bytes); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tig = lane & 3;
  const size_t fs = (size_t)c.nsites * n2;
  const float2* xr = x + (size_t)r0 * fs;
  const int nsite_cta = (c.nsites - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int T = 9 * nsite_cta;
  if (T <= 0) return;
  // rows nr..15 of every stage's vectors stay zero (the copies fill rows < nr only)
  for (int st = 0; st < kStages; ++st)
    for (int e = tid; e < (16 - nr) * xst; e += blockDim.x) stage_x(st)[nr * xst + e] = make_float2(0.f, 0.f);
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(&bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto site_of = [&](int t) { return (int)blockIdx.x + (t / 9) * (int)gridDim.x; };
  auto neighbour = [&](int site, int d) {
    if (d == 0) return site;
    const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
    int stride = 1;
    for (int m = 0; m < mu; ++m) stride *= c.L[m];
    const int xc = (site / stride) % c.L[mu];
    return site + (((xc + step + c.L[mu]) % c.L[mu]) - xc) * stride;
  };
  // thread 0: all copies of block t into stage t % kStages
  auto issue = [&](int t) {
    const int st = t % kStages;
    const int site = MG_CLAMP(kCoarseSite, site_of(t), c.nsites), d = t % 9;
    uint64_t* b = &bar[st];
    mbar_expect_tx(b, tile_bytes + nr * row_bytes);
    bulk_copy_g2s(stage_tile(st), M + ((size_t)site * 9 + d) * tile, tile_bytes, b);
    const int nb = MG_CLAMP(kCoarseNeighbour, neighbour(site, d), c.nsites);
    float2* xs = stage_x(st);
    for (int r = 0; r < nr; ++r) bulk_copy_g2s(xs + r * xst, xr + (size_t)r * fs + (size_t)nb * n2, row_bytes, b);
  };
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int t = 0; t < kStages - 1 && t < T; ++t) issue(t);
  }
  const int m0 = warp * 16;                                   // rows of Y owned by this warp
  float acc[2][4];
  int tfail = -1;
  for (int t = 0; t < T; ++t) {
    const int d = t % 9;
    const int site = MG_CLAMP(kCoarseSite, site_of(t), c.nsites);
    if (d == 0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    }
    if (tid == 0 && t + kStages - 1 < T) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + kStages - 1);
    }
    const int st = t % kStages;
    const bool waited = mbar_wait(&bar[st], (uint32_t)((t / kStages) & 1), spins);
    if (__syncthreads_or(!waited)) {
      tfail = t;
      break;
    }
    const TM* mt = stage_tile(st);
    const float2* xs = stage_x(st);
    if (m0 < 2 * n2) {
      const int i0 = (m0 >> 1) + (g >> 1), a = g & 1;        // output row pair of A rows m0+g, m0+g+8
      for (int k0 = 0; k0 < 2 * n2; k0 += 8) {
        const int j0 = (k0 >> 1) + (tig >> 1), bb = tig & 1;  // input column pair of A cols k0+tig, +4
        const uint32_t a0 = to_tf32(embed(tile_ld(mt, j0 * n2 + i0), a, bb));
        const uint32_t a1 = to_tf32(embed(tile_ld(mt, j0 * n2 + i0 + 4), a, bb));
        const uint32_t a2 = to_tf32(embed(tile_ld(mt, (j0 + 2) * n2 + i0), a, bb));
        const uint32_t a3 = to_tf32(embed(tile_ld(mt, (j0 + 2) * n2 + i0 + 4), a, bb));
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q == 1 && RB <= 8) continue;                    // columns 8..15 are zero
          const float2 x0 = xs[(8 * q + g) * xst + j0];
          const float2 x1 = xs[(8 * q + g) * xst + j0 + 2];
          const uint32_t b0 = to_tf32(bb ? x0.y : x0.x);
          const uint32_t b1 = to_tf32(bb ? x1.y : x1.x);
          mma_tf32(acc[q], a0, a1, a2, a3, b0, b1);
        }
      }
      if (d == 8) {
        // Y rows m0+g (and +8) = (re or im) of out_r(i0) (and out_r(i0 + 4)), columns 2 tig, 2 tig + 1
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 8 * q + 2 * tig + h;
            if (r < nr) {
              float* o = reinterpret_cast<float*>(out + (size_t)(r0 + r) * fs + (size_t)site * n2);
              o[2 * i0 + a] = acc[q][h];
              o[2 * (i0 + 4) + a] = acc[q][2 + h];
            }
          }
      }
    }
    __syncthreads();
  }
  if (tfail >= 0) {
    // wait (bounded) for this CTA's copies still in flight before leaving
    if (tid == 0) {
      atomicExch(err, 1);
      // stages tfail .. tfail + kStages - 1 were issued (the copy of t + kStages - 1
      // goes out before the wait of t): let every one of them land
      for (int u = tfail; u < T && u < tfail + kStages; ++u) mbar_wait(&bar[u % kStages], (uint32_t)((u / kStages) & 1));
    }
    __syncthreads();
  }
}

// FP16 operator: mma.sync m16n8k16 with FP16 inputs and FP32 accumulation.
// Fragment registers are pairs of real-embedding entries along k, so a stored
// complex entry m = (re, im) gives the A pair (re, -im) (even row) or (im, re)
// (odd row) with one bit or byte operation, and a vector entry x_r(j) is the B
// pair (re, im) itself, rounded to FP16 when the fragment is built.
__device__ __forceinline__ void mma_f16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                        uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t emb16(uint32_t m, int a) {
  return a ? __byte_perm(m, 0u, 0x1032) : (m ^ 0x80000000u);
}

__device__ __forceinline__ uint32_t pack16(float2 v) {
  const __half2 h = __floats2half2_rn(v.x, v.y);
  return *reinterpret_cast<const uint32_t*>(&h);
}

template <int RB, int N2, int ST, bool XH>
__global__ void __launch_bounds__(256) coarse_apply_mma16_kernel(const __half2* __restrict__ M,
                                                                 const void* __restrict__ xv,
                                                                 float2* __restrict__ out, CGeom c, int r0, int nr,
                                                                 int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int spins = wait_spins(err);
  __shared__ __align__(8) uint64_t bar[ST];
  const int n2 = N2 > 0 ? N2 : c.n2;                         // N2 > 0: block size fixed at compile time
  const int xst = n2 + 4;                                     // padded row stride (conflict-free fragment loads)
  const int tile = n2 * n2;
  const uint32_t tile_bytes = (uint32_t)tile * sizeof(__half2);
  // XH: the vectors are FP16 basis vectors (scaled by kBasisScale), staged as
  // half2 and used as B fragments directly; otherwise FP32, packed per fragment
  constexpr int xb = XH ? 4 : 8;                              // bytes per staged complex entry
  const uint32_t row_bytes = (uint32_t)n2 * xb;
  const size_t stage_bytes = tile_bytes + (size_t)16 * xst * xb;
  auto stage_tile = [&](int st) { return reinterpret_cast<const uint32_t*>(smem + st * stage_bytes); };
  auto stage_x = [&](int st) { return reinterpret_cast<float2*>(smem + st * stage_bytes + tile_bytes); };
  auto stage_xh = [&](int st) { return reinterpret_cast<uint32_t*>(smem + st * stage_bytes + tile_bytes); };
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, tig = lane & 3;
  const size_t fs = (size_t)c.nsites * n2;
  const unsigned char* xr = reinterpret_cast<const unsigned char*>(xv) + (size_t)r0 * fs * xb;
  const int nsite_cta = (c.nsites - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int T = 9 * nsite_cta;
  if (T <= 0) return;
  for (int st = 0; st < ST; ++st) {
    uint32_t* z = reinterpret_cast<uint32_t*>(smem + st * stage_bytes + tile_bytes + (size_t)nr * xst * xb);
    for (int e = tid; e < (16 - nr) * xst * xb / 4; e += blockDim.x) z[e] = 0u;
  }
  if (tid == 0) {
    for (int st = 0; st < ST; ++st) mbar_init(&bar[st], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  auto site_of = [&](int t) { return (int)blockIdx.x + (t / 9) * (int)gridDim.x; };
  auto neighbour = [&](int site, int d) {
    if (d == 0) return site;
    const int mu = (d - 1) >> 1, step = (d & 1) ? 1 : -1;
    int stride = 1;
    for (int m = 0; m < mu; ++m) stride *= c.L[m];
    const int xc = (site / stride) % c.L[mu];
    return site + (((xc + step + c.L[mu]) % c.L[mu]) - xc) * stride;
  };
  auto issue = [&](int t) {
    const int st = t % ST;
    const int site = MG_CLAMP(kCoarseSite, site_of(t), c.nsites), d = t % 9;
    uint64_t* b = &bar[st];
    mbar_expect_tx(b, tile_bytes + nr * row_bytes);
    bulk_copy_g2s((void*)stage_tile(st), M + ((size_t)site * 9 + d) * tile, tile_bytes, b);
    const int nb = MG_CLAMP(kCoarseNeighbour, neighbour(site, d), c.nsites);
    unsigned char* xs = smem + st * stage_bytes + tile_bytes;
    for (int r = 0; r < nr; ++r)
      bulk_copy_g2s(xs + (size_t)r * xst * xb, xr + ((size_t)r * fs + (size_t)nb * n2) * xb, row_bytes, b);
  };
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int t = 0; t < ST - 1 && t < T; ++t) issue(t);
  }
  const int m0 = warp * 16;
  const int i0 = (m0 >> 1) + (g >> 1), a = g & 1;            // output rows i0 (fragment row g) and i0 + 4 (g + 8)
  float acc[2][4];
  int tfail = -1;
  for (int t = 0; t < T; ++t) {
    const int d = t % 9;
    const int site = MG_CLAMP(kCoarseSite, site_of(t), c.nsites);
    if (d == 0) {
#pragma unroll
      for (int q = 0; q < 2; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
    }
    if (tid == 0 && t + ST - 1 < T) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(t + ST - 1);
    }
    const int st = t % ST;
    const bool waited = mbar_wait(&bar[st], (uint32_t)((t / ST) & 1), spins);
    if (__syncthreads_or(!waited)) {
      tfail = t;
      break;
    }
    const uint32_t* mt = stage_tile(st);
    const float2* xs = stage_x(st);
    const uint32_t* xsh = stage_xh(st);
    if (m0 < 2 * n2) {
#pragma unroll
      for (int k0 = 0; k0 < 2 * n2; k0 += 16) {
        const int j = (k0 >> 1) + tig;                        // input columns j (k pair 2 tig) and j + 4
        const uint32_t a0 = emb16(mt[j * n2 + i0], a);
        const uint32_t a1 = emb16(mt[j * n2 + i0 + 4], a);
        const uint32_t a2 = emb16(mt[(j + 4) * n2 + i0], a);
        const uint32_t a3 = emb16(mt[(j + 4) * n2 + i0 + 4], a);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (q == 1 && RB <= 8) continue;                    // columns 8..15 are zero
          const uint32_t b0 = XH ? xsh[(8 * q + g) * xst + j] : pack16(xs[(8 * q + g) * xst + j]);
          const uint32_t b1 = XH ? xsh[(8 * q + g) * xst + j + 4] : pack16(xs[(8 * q + g) * xst + j + 4]);
          mma_f16(acc[q], a0, a1, a2, a3, b0, b1);
        }
      }
      if (d == 8) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int r = 8 * q + 2 * tig + h;
            if (r < nr) {
              float* o = reinterpret_cast<float*>(out + (size_t)(r0 + r) * fs + (size_t)site * n2);
              constexpr float os = XH ? 1.f / kBasisScale : 1.f;
              o[2 * i0 + a] = os * acc[q][h];
              o[2 * (i0 + 4) + a] = os * acc[q][2 + h];
            }
          }
      }
    }
    __syncthreads();
  }
  if (tfail >= 0) {
    if (tid == 0) {
      atomicExch(err, 1);
      // stages tfail .. tfail + ST - 1 were issued (the copy of t + ST - 1 goes out
      // before the wait of t): let every one of them land
      for (int u = tfail; u < T && u < tfail + ST; ++u) mbar_wait(&bar[u % ST], (uint32_t)((u / ST) & 1));
    }
    __syncthreads();
  }
}

template <int RB, int N2, int ST, bool XH>
static void launch_mma16_t(const CGeom& c, const __half2* M, const void* x, float2* out, int r0, int nr, int* err,
                           int ctas, cudaStream_t s) {
  const size_t stage = (size_t)c.n2 * c.n2 * sizeof(__half2) + (size_t)16 * (c.n2 + 4) * (XH ? 4 : 8);
  const size_t smem = ST * stage;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(coarse_apply_mma16_kernel<RB, N2, ST, XH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    attr = true;
  }
  const int threads = 32 * (c.n2 / 8);
  int per_sm = (int)std::max<size_t>(1, std::min<size_t>(16, (220 * 1024) / (smem + 1024)));
  if (ctas > 0) per_sm = std::min(per_sm, ctas);
  const int grid = std::min(c.nsites, 152 * per_sm);
  coarse_apply_mma16_kernel<RB, N2, ST, XH><<<grid, threads, smem, s>>>(M, x, out, c, r0, nr, err); count_launches(1);
}

// Two stages (one block in flight while the previous is multiplied) keep the
// shared memory per CTA small enough for eight CTAs per SM, which measured
// faster than deeper rings with fewer CTAs; 2N = 40 has a specialised
// instance with the k loop unrolled.
template <int RB, bool XH>
static void launch_mma16(const CGeom& c, const __half2* M, const void* x, float2* out, int r0, int nr, int* err,
                         const CoarseTune& t, cudaStream_t s) {
  if (c.n2 == 40 && t.stages == 3) launch_mma16_t<RB, 40, 3, XH>(c, M, x, out, r0, nr, err, t.ctas, s);
  else if (c.n2 == 40) launch_mma16_t<RB, 40, 2, XH>(c, M, x, out, r0, nr, err, t.ctas, s);
  else launch_mma16_t<RB, 0, 2, XH>(c, M, x, out, r0, nr, err, t.ctas, s);
}

template <int RB, class TM>
static void launch_mma(const CGeom& c, const TM* M, const float2* x, float2* out, int r0, int nr, int* err,
                       cudaStream_t s) {
  const size_t stage = (size_t)c.n2 * c.n2 * sizeof(TM) + (size_t)16 * (c.n2 + 2) * sizeof(float2);
  const size_t smem = kStages * stage;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(coarse_apply_mma_kernel<RB, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  const int threads = 32 * (c.n2 / 8);                        // one warp per 16 rows of the 2 n2 real rows
  const int per_sm = (int)std::max<size_t>(1, std::min<size_t>(16, (220 * 1024) / (smem + 1024)));
  const int grid = std::min(c.nsites, 152 * per_sm);
  coarse_apply_mma_kernel<RB, TM><<<grid, threads, smem, s>>>(M, x, out, c, r0, nr, err); count_launches(1);
}

template <class TM>
static void launch_mma_all(const CGeom& c, const TM* M, const float2* x, float2* out, int nrhs, int* err,
                           cudaStream_t s) {
  for (int r0 = 0; r0 < nrhs; r0 += 16) {
    const int rb = std::min(16, nrhs - r0);
    if (rb > 12) launch_mma<16, TM>(c, M, x, out, r0, rb, err, s);
    else if (rb > 8) launch_mma<12, TM>(c, M, x, out, r0, rb, err, s);
    else if (rb > 4) launch_mma<8, TM>(c, M, x, out, r0, rb, err, s);
    else if (rb > 1) launch_mma<4, TM>(c, M, x, out, r0, rb, err, s);
    else launch_mma<1, TM>(c, M, x, out, r0, rb, err, s);
  }
}

// Tensor-core form: n2 % 8 == 0 and n2 <= 64; up to 16 right-hand sides per
// launch (nr of them, the template width RB >= nr fixes the fragment count);
// the operator in FP32 (store P32) or FP16 (store P16).
int launch_coarse_apply_mma(const CGeom& c, int store, const void* M, const void* x, void* out, int nrhs, int* err,
                            bool x_half, cudaStream_t s, const CoarseTune& t) {
  if (x_half && store != P16) return MG_ERR_ARG;
  if (c.n2 % 8 != 0 || c.n2 > 64) return MG_ERR_ARG;
  if (store == P32) {
    launch_mma_all(c, (const float2*)M, (const float2*)x, (float2*)out, nrhs, err, s);
  } else if (store == P16) {
    const __half2* m = (const __half2*)M;
    const size_t xe = x_half ? 4 : 8;                         // bytes per complex vector entry
    const int batch = std::max(1, std::min(16, t.batch));
    for (int r0 = 0; r0 < nrhs; r0 += batch) {
      const int rb = std::min(batch, nrhs - r0);
      const void* xs = x;
      float2* o = (float2*)out;
      (void)xe;
#define SAPMG_M16(RB_)                                                                       \
  if (x_half) launch_mma16<RB_, true>(c, m, xs, o, r0, rb, err, t, s);                       \
  else launch_mma16<RB_, false>(c, m, xs, o, r0, rb, err, t, s);
      if (rb > 12) { SAPMG_M16(16) }
      else if (rb > 8) { SAPMG_M16(12) }
      else if (rb > 4) { SAPMG_M16(8) }
      else if (rb > 1) { SAPMG_M16(4) }
      else { SAPMG_M16(1) }
#undef SAPMG_M16
    }
  } else {
    return MG_ERR_ARG;
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

// Requires 16-byte aligned blocks (n2 even) and n2 <= 64; the caller routes
// other shapes to the generic kernel.
int launch_coarse_apply_tma(const CGeom& c, const void* M, const void* x, void* out, int nrhs, int* err,
                            cudaStream_t s) {
  if (c.n2 % 2 != 0 || c.n2 > 64) return MG_ERR_ARG;
  const float2* m = (const float2*)M;
  const float2* xi = (const float2*)x;
  float2* o = (float2*)out;
  for (int r0 = 0; r0 < nrhs;) {
    const int left = nrhs - r0;
    if (left >= 12) {
      if (c.n2 <= 42) launch_tma<12, 2>(c, m, xi, o, r0, err, s);
      else launch_tma<12, 3>(c, m, xi, o, r0, err, s);
      r0 += 12;
    } else if (left >= 4) {
      launch_tma<4, 1>(c, m, xi, o, r0, err, s);
      r0 += 4;
    } else {
      launch_tma<1, 1>(c, m, xi, o, r0, err, s);
      r0 += 1;
    }
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
