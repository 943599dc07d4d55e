// Aggregation and coarse-grid kernels (internal).
#pragma once
#include "internal.h"

namespace sapmg {

// A coarse lattice: dims, sites, dof per site (2N of the finer level).
struct CGeom {
  int L[4];
  int nsites;
  int n2;
};

// A decomposition of a coarse lattice into boxes of b[0] x .. x b[3] sites.
struct Box4 {
  int b[4];
  int nb[4];
  int nboxes;
  int sites;
};
inline Box4 make_box(const CGeom& c, const int b[4]) {
  Box4 x;
  x.nboxes = 1;
  x.sites = 1;
  for (int mu = 0; mu < 4; ++mu) {
    x.b[mu] = b[mu];
    x.nb[mu] = c.L[mu] / b[mu];
    x.nboxes *= x.nb[mu];
    x.sites *= b[mu];
  }
  return x;
}

// Level 0 -> 1 (4^4 aggregates = the fine blocks).  tf32: several FP32
// right-hand sides are restricted on the tensor cores (TF32 inputs, FP32 sums).
int launch_transfer0(bool restrict_, int prec, const Geom& g, const void* in, void* out, const void* Pv, int N,
                     int nrhs, bool tf32, cudaStream_t s);
int launch_block_gs0(const Geom& g, void* V64, int N, cudaStream_t s);
int launch_store_p0(int prec, const Geom& g, const void* V64, void* Pv, int N, cudaStream_t s);
// D_c = P^dagger D P into the FP64 M64 from the locally orthonormal vectors V,
// links U and clover A, all of type prec (P64: FP64 arithmetic; P32: FP32
// copies and FP32 arithmetic, the mixed form).
int launch_assemble0(const Geom& g, int prec, const void* V, const void* U, const void* A, void* M64, int N,
                     cudaStream_t s);

// Coarse levels.
int launch_coarse_apply(int prec, const CGeom& c, const void* M, const void* x, void* out, int nrhs, cudaStream_t s);
int launch_coarse_export(int prec, const CGeom& c, const void* M, double* out, cudaStream_t s);
// FP32 operator, FP32 vectors: the stencil fed by bulk asynchronous copies (n2 even, <= 64).
// err: device flag raised when a bounded wait gives up.
int launch_coarse_apply_tma(const CGeom& c, const void* M, const void* x, void* out, int nrhs, int* err,
                            cudaStream_t s);
// Launch shape of the FP16 tensor-core stencil (chosen by the autotuner; every
// choice computes each output with the same operations): right-hand sides per
// launch (1..16), depth of the bulk-copy ring (2 or 3; 3 only for 2N = 40)
// and a cap on the CTAs per SM (0: as many as shared memory allows).
struct CoarseTune {
  int batch = 16;
  int stages = 2;
  int ctas = 0;
};
// The same stencil with the block products on tensor cores (TF32 inputs, FP32
// accumulation; n2 % 8 == 0, n2 <= 64); operator stored in FP32 (P32) or FP16 (P16).
// x_half (FP16 operator only): x holds FP16 basis vectors scaled by kBasisScale.
int launch_coarse_apply_mma(const CGeom& c, int store, const void* M, const void* x, void* out, int nrhs, int* err,
                            bool x_half, cudaStream_t s, const CoarseTune& t = CoarseTune());

// Intermediate level of a three-level hierarchy (coarse1.cu).
// The colour pass of launch_coarse_sap for 1 <= nrhs <= 12 right-hand sides in one
// CTA per box (FP32 vectors; FP32 operator, or its FP16 copy with m16; each
// operator entry loaded once for all of them); bit for bit the one-RHS-per-CTA
// results with the same operator.
int launch_coarse_sap_mrhs(const CGeom& c, const Box4& bx, const void* M, bool m16, void* z, const void* b,
                           int colour, int n_mr, int nrhs, cudaStream_t s);
int launch_coarse_sap(int prec, const CGeom& c, const Box4& bx, const void* M, void* z, const void* b, int colour,
                      int n_mr, int nrhs, cudaStream_t s, bool m16 = false);
int launch_transfer1(bool restrict_, int prec, const CGeom& c, const Box4& ag, const void* in, void* out,
                     const void* W, int N1, int nrhs, cudaStream_t s);
int launch_block_gs1(const CGeom& c, const Box4& ag, void* W64, int N1, cudaStream_t s);
int launch_assemble1(const CGeom& c, const CGeom& c2, const Box4& ag, const void* W64, const void* M1_64, void* M2_64,
                     int N1, cudaStream_t s);

}  // namespace sapmg
