// Measured compute and shared-memory peaks of the current GPU (the
// denominators of the roofline of the CUDA-core kernels: the Schwarz colour
// pass is bound by FP32 arithmetic and by shared-memory/L1 traffic, neither of
// which a copy or a GEMM measures).
//
//  * fp32: every thread runs 16 independent chains x = fma(x, a, b) (scalar
//    FFMA); 2 flop per FMA.
//  * fp32x2: the same with 8 chains of the packed two-wide FMA (__ffma2_rn,
//    sm_100 and later), 4 flop per instruction.
//  * smem: every thread reads 16-byte words of a 16 KB shared array at
//    conflict-free addresses (a warp covers 512 consecutive bytes) and folds
//    them with integer xor (one instruction per two words), so the loads, not
//    the arithmetic, bound the loop.
// Each probe runs on every SM with full occupancy (8 CTAs of 256 threads per
// SM), three warm-up launches, then the best of ten timed with CUDA events on
// the given stream.
#include "internal.h"

namespace sapmg {

__global__ void __launch_bounds__(256) probe_fma_kernel(float* out, float a, float b, int iters) {
  float x[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) x[i] = threadIdx.x * 1e-3f + (float)i;
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += x[i];
  if (s == -1.2345f) out[blockIdx.x] = s;      // never true: keeps the chains alive
}

__global__ void __launch_bounds__(256) probe_fma2_kernel(float* out, float a, float b, int iters) {
  float2 x[8];
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = make_float2(threadIdx.x * 1e-3f + (float)i, (float)i + 0.5f);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i].x + x[i].y;
  if (s == -1.2345f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) probe_smem_kernel(unsigned* out, int iters) {
  __shared__ uint4 buf[1024];
  for (int i = threadIdx.x; i < 1024; i += blockDim.x) buf[i] = make_uint4(i, 3 * i, 5 * i, 7 * i);
  __syncthreads();
  unsigned acc0 = 0, acc1 = 0;
  const int t = threadIdx.x;
#pragma unroll 2
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint4 v = buf[(t + 256 * k + it) & 1023];
      acc0 ^= v.x ^ v.y;
      acc1 ^= v.z ^ v.w;
    }
  }
  if ((acc0 ^ acc1) == 0x9e3779b9u) out[blockIdx.x] = acc0;
}

template <class F>
static int best_ms(cudaStream_t s, F launch, float* ms_out) {
  cudaEvent_t e0, e1;
  SAPMG_CUDA_TRY(cudaEventCreate(&e0));
  SAPMG_CUDA_TRY(cudaEventCreate(&e1));
  for (int i = 0; i < 3; ++i) launch();
  float best = 1e30f;
  for (int i = 0; i < 10; ++i) {
    SAPMG_CUDA_TRY(cudaEventRecord(e0, s));
    launch();
    SAPMG_CUDA_TRY(cudaEventRecord(e1, s));
    SAPMG_CUDA_TRY(cudaEventSynchronize(e1));
    float ms = 0.f;
    SAPMG_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  *ms_out = best;
  return MG_OK;
}

int probe_peaks(cudaStream_t s, double* fp32_tflops, double* fp32x2_tflops, double* smem_gbs) {
  int dev = 0, nsm = 0;
  SAPMG_CUDA_TRY(cudaGetDevice(&dev));
  SAPMG_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)nsm * 8;
  const double threads = (double)grid * 256;
  void* out = nullptr;
  SAPMG_CUDA_TRY(cudaMallocAsync(&out, grid * sizeof(float), s));
  const int it_fma = 8192, it_smem = 4096;
  float ms = 0.f;
  int rc = best_ms(s, [&] { probe_fma_kernel<<<grid, 256, 0, s>>>((float*)out, 0.9999f, 1e-4f, it_fma); }, &ms);
  if (rc == MG_OK) *fp32_tflops = 2.0 * 16 * it_fma * threads / (ms * 1e-3) / 1e12;
  if (rc == MG_OK)
    rc = best_ms(s, [&] { probe_fma2_kernel<<<grid, 256, 0, s>>>((float*)out, 0.9999f, 1e-4f, it_fma); }, &ms);
  if (rc == MG_OK) *fp32x2_tflops = 2.0 * 16 * it_fma * threads / (ms * 1e-3) / 1e12;
  if (rc == MG_OK)
    rc = best_ms(s, [&] { probe_smem_kernel<<<grid, 256, 0, s>>>((unsigned*)out, it_smem); }, &ms);
  if (rc == MG_OK) *smem_gbs = 16.0 * 4 * it_smem * threads / (ms * 1e-3) / 1e9;
  cudaFreeAsync(out, s);
  SAPMG_CUDA_TRY(cudaStreamSynchronize(s));
  return rc;
}

}  // namespace sapmg
