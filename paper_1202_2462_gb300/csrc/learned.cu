// Kernels of the learned set-up: a gauge-covariant convolutional network that
// proposes near-kernel test vectors (trained to imitate the bootstrap set-up
// of Sec. 3; the bootstrap stays the fallback).
//
// Layer: out_a(x) = sum_b sum_h W[a][b][h] (T_h in_b)(x), with the parallel
// transports T_0 psi = psi, T_{+mu} psi(x) = U_mu(x) psi(x + mu),
// T_{-mu} psi(x) = U_mu(x - mu)^dagger psi(x - mu) (hop h = 0, 1 + 2 mu,
// 2 + 2 mu) and W[a][b][h] a complex 4 x 4 matrix on the spin index.  Gate
// between layers: psi(x) -> psi(x) / sqrt(1 + |psi(x)|^2) per channel and
// site.  Gradients: G_z = dL/dRe z + i dL/dIm z.
//
// Fields are FP32 complex in the blocked layout, channel c at c * 12V; links
// are the context's FP32 copy.  One thread per (site, output channel) in the
// forward pass and per (site, input channel) in the input gradient; the weight
// gradient is one CTA per (a, b, h) reducing over all sites in a fixed order
// (deterministic).
#include "internal.h"
#include "stencil.cuh"

namespace sapmg {

namespace {

// T_h psi_b at (blk, loc) into v (4 spins x 3 colours); links in storage type TG
template <class TG = float2>
__device__ __forceinline__ void transport_at(const Geom& g, const TG* __restrict__ U,
                                             const float2* __restrict__ f, int blk, int loc, int h,
                                             Cplx<float> (&v)[12]) {
  if (h == 0) {
    load_spinor<float>(f, blk, loc, v);
    return;
  }
  const int mu = (h - 1) >> 1;
  const int step = ((h - 1) & 1) ? -1 : 1;
  int nb, nl;
  neighbour(g, blk, loc, mu, step, nb, nl);
  Cplx<float> p[12], u[9];
  load_spinor<float>(f, nb, nl, p);
  if (step > 0) {
    load_link<float>(U, blk, mu, loc, u);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Cplx<float> acc = u[a * 3] * p[s * 3];
        cfma(acc, u[a * 3 + 1], p[s * 3 + 1]);
        cfma(acc, u[a * 3 + 2], p[s * 3 + 2]);
        v[s * 3 + a] = acc;
      }
  } else {
    load_link<float>(U, nb, mu, nl, u);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        Cplx<float> acc = cmk(0.f, 0.f);
        cfma_conj(acc, u[a], p[s * 3]);
        cfma_conj(acc, u[3 + a], p[s * 3 + 1]);
        cfma_conj(acc, u[6 + a], p[s * 3 + 2]);
        v[s * 3 + a] = acc;
      }
  }
}

__device__ __forceinline__ int adjoint_hop(int h) { return h == 0 ? 0 : (((h - 1) & 1) ? h - 1 : h + 1); }

}  // namespace

// y_a = sum_b sum_h W[a][b][h] T_h x_b; grid (nblocks, cout), W[a] staged in shared memory.
// TG, TW: storage of the links and of the weights (FP32, or BF16 for inference);
// activations and accumulation in FP32.
template <class TG, class TW>
__global__ void __launch_bounds__(256) gconv_forward_kernel(Geom g, const TG* __restrict__ U,
                                                            const TW* __restrict__ W,
                                                            const float2* __restrict__ x, float2* __restrict__ y,
                                                            int cin) {
  extern __shared__ float2 ws[];                                // [cin][9][16]
  const int blk = MG_CLAMP(kBlock, blockIdx.x, g.nblocks), a = blockIdx.y, loc = threadIdx.x;
  const size_t fs = (size_t)g.V * 12;
  for (int e = loc; e < cin * 9 * 16; e += 256) {
    const Cplx<float> w = Io<float, TW>::ldc(W + (size_t)a * cin * 9 * 16 + e);
    ws[e] = make_float2(w.re, w.im);
  }
  __syncthreads();
  Cplx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cmk(0.f, 0.f);
  for (int b = 0; b < cin; ++b) {
    for (int h = 0; h < 9; ++h) {
      Cplx<float> v[12];
      transport_at<TG>(g, U, x + (size_t)b * fs, blk, loc, h, v);
      const float2* w = ws + (b * 9 + h) * 16;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const Cplx<float> m = cmk(w[s * 4 + t].x, w[s * 4 + t].y);
#pragma unroll
          for (int c = 0; c < 3; ++c) cfma(acc[s * 3 + c], m, v[t * 3 + c]);
        }
    }
  }
  store_spinor<float>(y + (size_t)a * fs, blk, loc, acc);
}

// G_x_b = sum_h T_h^dagger (sum_a W[a][b][h]^dagger G_y_a); T_h^dagger = T_{adjoint hop}.
// grid (nblocks, cin), W[.][b] staged in shared memory.
__global__ void __launch_bounds__(256) gconv_backward_input_kernel(Geom g, const float2* __restrict__ U,
                                                                   const float2* __restrict__ W,
                                                                   const float2* __restrict__ gy,
                                                                   float2* __restrict__ gx, int cin, int cout) {
  extern __shared__ float2 ws[];                                // [cout][9][16] for this b
  const int blk = MG_CLAMP(kBlock, blockIdx.x, g.nblocks), b = blockIdx.y, loc = threadIdx.x;
  const size_t fs = (size_t)g.V * 12;
  for (int e = loc; e < cout * 9 * 16; e += 256) {
    const int a = e / (9 * 16), r = e % (9 * 16);
    ws[e] = W[((size_t)a * cin + b) * 9 * 16 + r];
  }
  __syncthreads();
  Cplx<float> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = cmk(0.f, 0.f);
  for (int h = 0; h < 9; ++h) {
    // q(y) = sum_a W[a][b][h]^dagger G_y_a(y) at y = the site T_{adjoint hop} reads from,
    // then transported: (T_adj q)(x)
    const int ha = adjoint_hop(h);
    int nb = blk, nl = loc;
    if (ha != 0) neighbour(g, blk, loc, (ha - 1) >> 1, ((ha - 1) & 1) ? -1 : 1, nb, nl);
    Cplx<float> q[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = cmk(0.f, 0.f);
    for (int a = 0; a < cout; ++a) {
      Cplx<float> p[12];
      load_spinor<float>(gy + (size_t)a * fs, nb, nl, p);
      const float2* w = ws + (a * 9 + h) * 16;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const Cplx<float> m = cmk(w[t * 4 + s].x, w[t * 4 + s].y);   // (W^dagger)[s][t] = conj(W[t][s])
#pragma unroll
          for (int c = 0; c < 3; ++c) cfma_conj(q[s * 3 + c], m, p[t * 3 + c]);
        }
    }
    if (ha == 0) {
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = acc[k] + q[k];
    } else {
      const int mu = (ha - 1) >> 1;
      Cplx<float> u[9];
      if (((ha - 1) & 1) == 0) {                                // +mu: U_mu(x) q(x + mu)
        load_link<float>(U, blk, mu, loc, u);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cfma(acc[s * 3 + c], u[c * 3], q[s * 3]);
            cfma(acc[s * 3 + c], u[c * 3 + 1], q[s * 3 + 1]);
            cfma(acc[s * 3 + c], u[c * 3 + 2], q[s * 3 + 2]);
          }
      } else {                                                  // -mu: U_mu(x - mu)^dagger q(x - mu)
        load_link<float>(U, nb, mu, nl, u);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            cfma_conj(acc[s * 3 + c], u[c], q[s * 3]);
            cfma_conj(acc[s * 3 + c], u[3 + c], q[s * 3 + 1]);
            cfma_conj(acc[s * 3 + c], u[6 + c], q[s * 3 + 2]);
          }
      }
    }
  }
  store_spinor<float>(gx + (size_t)b * fs, blk, loc, acc);
}

// G_W[a][b][h][s][t] = sum_x sum_c G_y_a(x)[s][c] conj((T_h x_b)(x)[t][c]);
// one CTA per (a, b, h), fixed-order reduction (per-thread sums over a
// grid-stride of sites, then warps, then the CTA).
__global__ void __launch_bounds__(256) gconv_backward_weight_kernel(Geom g, const float2* __restrict__ U,
                                                                    const float2* __restrict__ x,
                                                                    const float2* __restrict__ gy,
                                                                    float2* __restrict__ gW, int cin) {
  const int id = blockIdx.x;
  const int h = id % 9, b = (id / 9) % cin, a = id / (9 * cin);
  const size_t fs = (size_t)g.V * 12;
  float re[16], im[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) re[k] = im[k] = 0.f;
  for (long long i = threadIdx.x; i < g.V; i += blockDim.x) {
    const int blk = (int)(i >> 8), loc = (int)(i & 255);
    Cplx<float> v[12], p[12];
    transport_at(g, U, x + (size_t)b * fs, blk, loc, h, v);
    load_spinor<float>(gy + (size_t)a * fs, blk, loc, p);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          // p[s][c] * conj(v[t][c])
          const Cplx<float> l = p[s * 3 + c], r = v[t * 3 + c];
          re[s * 4 + t] += l.re * r.re + l.im * r.im;
          im[s * 4 + t] += l.im * r.re - l.re * r.im;
        }
  }
  __shared__ float red[8][32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const float sr = warp_sum(re[k]), si = warp_sum(im[k]);
    if (lane == 0) { red[w][2 * k] = sr; red[w][2 * k + 1] = si; }
  }
  __syncthreads();
  if (threadIdx.x < 16) {
    float sr = 0.f, si = 0.f;
    for (int q = 0; q < 8; ++q) { sr += red[q][2 * threadIdx.x]; si += red[q][2 * threadIdx.x + 1]; }
    gW[(size_t)id * 16 + threadIdx.x] = make_float2(sr, si);
  }
}

// y = x / sqrt(1 + |x(site)|^2) per channel and site
__global__ void gate_forward_kernel(Geom g, const float2* __restrict__ x, float2* __restrict__ y, int channels) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V * channels) return;
  const int ch = (int)(i / g.V);
  const long long site = i % g.V;
  const int blk = (int)(site >> 8), loc = (int)(site & 255);
  const size_t fs = (size_t)g.V * 12;
  Cplx<float> p[12];
  load_spinor<float>(x + (size_t)ch * fs, blk, loc, p);
  float n = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) n += p[k].re * p[k].re + p[k].im * p[k].im;
  const float s = rsqrtf(1.f + n);
#pragma unroll
  for (int k = 0; k < 12; ++k) p[k] = s * p[k];
  store_spinor<float>(y + (size_t)ch * fs, blk, loc, p);
}

// G_x = s G_y - (1 + n)^(-3/2) Re<G_y, x>_site x, s = (1 + n)^(-1/2), n = |x(site)|^2
__global__ void gate_backward_kernel(Geom g, const float2* __restrict__ x, const float2* __restrict__ gy,
                                     float2* __restrict__ gx, int channels) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.V * channels) return;
  const int ch = (int)(i / g.V);
  const long long site = i % g.V;
  const int blk = (int)(site >> 8), loc = (int)(site & 255);
  const size_t fs = (size_t)g.V * 12;
  Cplx<float> p[12], q[12];
  load_spinor<float>(x + (size_t)ch * fs, blk, loc, p);
  load_spinor<float>(gy + (size_t)ch * fs, blk, loc, q);
  float n = 0.f, re = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    n += p[k].re * p[k].re + p[k].im * p[k].im;
    re += q[k].re * p[k].re + q[k].im * p[k].im;
  }
  const float s = rsqrtf(1.f + n);
  const float c = re * s * s * s;
#pragma unroll
  for (int k = 0; k < 12; ++k) q[k] = s * q[k] + (-c) * p[k];
  store_spinor<float>(gx + (size_t)ch * fs, blk, loc, q);
}

// Adam on n real parameters (bias-corrected moments; step >= 1).
__global__ void adam_kernel(size_t n, float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

template <class TG, class TW>
static int gconv_forward(const Geom& g, const void* U, const void* W, const void* x, void* y, int cin, int cout,
                         cudaStream_t s) {
  const size_t smem = sizeof(float2) * cin * 9 * 16;
  if (smem > 200 * 1024) return MG_ERR_ARG;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gconv_forward_kernel<TG, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  gconv_forward_kernel<TG, TW><<<dim3(g.nblocks, cout), 256, smem, s>>>(g, (const TG*)U, (const TW*)W,
                                                                         (const float2*)x, (float2*)y, cin);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_gconv_forward(const Geom& g, const void* U, const void* W, const void* x, void* y, int cin, int cout,
                         cudaStream_t s) {
  return gconv_forward<float2, float2>(g, U, W, x, y, cin, cout, s);
}

int launch_gconv_forward_bf16(const Geom& g, const void* U, const void* W, const void* x, void* y, int cin, int cout,
                              cudaStream_t s) {
  return gconv_forward<__nv_bfloat162, __nv_bfloat162>(g, U, W, x, y, cin, cout, s);
}

int launch_gconv_backward(const Geom& g, const void* U, const void* W, const void* x, const void* gy, void* gx,
                          void* gW, int cin, int cout, cudaStream_t s) {
  const size_t smem = sizeof(float2) * cout * 9 * 16;
  if (smem > 200 * 1024) return MG_ERR_ARG;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(gconv_backward_input_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  if (gx) {
    gconv_backward_input_kernel<<<dim3(g.nblocks, cin), 256, smem, s>>>(g, (const float2*)U, (const float2*)W,
                                                                       (const float2*)gy, (float2*)gx, cin, cout);
    count_launches(1);
  }
  if (gW) {
    gconv_backward_weight_kernel<<<cout * cin * 9, 256, 0, s>>>(g, (const float2*)U, (const float2*)x,
                                                               (const float2*)gy, (float2*)gW, cin);
    count_launches(1);
  }
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_gate(const Geom& g, const void* x, const void* gy, void* out, int channels, cudaStream_t s) {
  const long long n = g.V * channels;
  const unsigned grid = (unsigned)((n + 255) / 256);
  if (gy) {
    gate_backward_kernel<<<grid, 256, 0, s>>>(g, (const float2*)x, (const float2*)gy, (float2*)out, channels);
  } else {
    gate_forward_kernel<<<grid, 256, 0, s>>>(g, (const float2*)x, (float2*)out, channels);
  }
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

int launch_adam(size_t n, float* p, const float* gr, float* m, float* v, double lr, double b1, double b2,
                double eps, int step, cudaStream_t s) {
  if (step < 1) return MG_ERR_ARG;
  const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 152 * 8);
  adam_kernel<<<std::max(1u, grid), 256, 0, s>>>(n, p, gr, m, v, (float)lr, (float)b1, (float)b2, (float)eps, c1,
                                                  c2);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
}

}  // namespace sapmg
