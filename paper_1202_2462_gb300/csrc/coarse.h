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

// Level 0 -> 1 (4^4 aggregates = the fine blocks).
int launch_transfer0(bool restrict_, int prec, const Geom& g, const void* in, void* out, const void* Pv, int N,
                     int nrhs, cudaStream_t s);
int launch_block_gs0(const Geom& g, void* V64, int N, cudaStream_t s);
int launch_store_p0(int prec, const Geom& g, const void* V64, void* Pv, int N, cudaStream_t s);
int launch_assemble0(const Geom& g, const void* V64, const void* U64, const void* A64, void* M64, int N,
                     cudaStream_t s);

// Coarse levels.
int launch_coarse_apply(int prec, const CGeom& c, const void* M, const void* x, void* out, int nrhs, cudaStream_t s);
int launch_coarse_export(int prec, const CGeom& c, const void* M, double* out, cudaStream_t s);
// FP32 operator, FP32 vectors: the stencil fed by bulk asynchronous copies (n2 even, <= 64).
// err: device flag raised when a bounded wait gives up.
int launch_coarse_apply_tma(const CGeom& c, const void* M, const void* x, void* out, int nrhs, int* err,
                            cudaStream_t s);

}  // namespace sapmg
