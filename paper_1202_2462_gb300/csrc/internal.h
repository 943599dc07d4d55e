// Internal declarations of the SAP-multilevel library (not part of the C-ABI).
#pragma once
#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "sapmg.h"
#include "common.cuh"

namespace sapmg {

// Storage precisions of fields; equal to the public MG_FP64 ... MG_BF16.
enum { P64 = MG_FP64, P32 = MG_FP32, P16 = MG_FP16, PBF = MG_BF16 };
// FP64 data with double-float arithmetic on the FP32 units (dirac.cu only)
enum { P64E = 16 };

inline size_t complex_bytes(int prec) { return prec == P64 ? 16 : (prec == P32 ? 8 : 4); }
// Krylov basis vectors kept in FP16 are stored multiplied by this power of two
// (unit vectors: entries below 1, so the scaled values stay normal in FP16).
constexpr float kBasisScale = 1024.f;

// layout.cu
int launch_pack_gauge(int prec, const Geom& g, const double* Uc, void* Ub, int antiperiodic_t, cudaStream_t s);
int launch_clover_build(const Geom& g, const double* Uc, void* Ab64, double m0, double c_sw, cudaStream_t s);
int launch_clover_export(const Geom& g, const void* Ab64, double* out, cudaStream_t s);
int launch_convert(int from, const void* in, int to, void* out, size_t n_complex, cudaStream_t s);
int launch_pack_spinor(int pin, const void* canon, int pout, void* blocked, const Geom& g, int nrhs, cudaStream_t s);
int launch_unpack_spinor(int pin, const void* blocked, int pout, void* canon, const Geom& g, int nrhs, cudaStream_t s);
int launch_draw_vectors(const Geom& g, void* out64, int nvec, unsigned long long seed, unsigned long long stream,
                        cudaStream_t s);
uint64_t host_splitmix64(uint64_t x);

// dirac.cu
int launch_dirac(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                 cudaStream_t s);
// The same for an even number of right-hand sides in FP32 arithmetic, two per thread (dirac2.cu).
int launch_dirac_pair(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                      cudaStream_t s);
// dag: D^dagger = gamma5 D gamma5; part != nullptr: also the per-CTA partial
// sums of ||out||^2 at part[block * nrhs + r] (FP64 and FP32 fields only).
int launch_dirac_ex(int prec, const Geom& g, void* out, const void* in, const void* U, const void* A, int nrhs,
                    bool dag, double* part, cudaStream_t s);

// setup2.cu: out = P phi with the FP64 vector-major test vectors v64 (N fine
// fields, blocked layout) and an FP64 coarse vector phi [nblocks][2N]
int launch_prolong_v64(const Geom& g, const void* v64, int N, const void* phi, void* out, cudaStream_t s);
int launch_restrict_v64(const Geom& g, const void* v64, int N, const void* x, void* out, cudaStream_t s);

// dense_eig.cu: host eigen-solvers of the set-up's second part (column-major
// complex, re/im interleaved)
int harmonic_ritz_host(int m, const double* hbar, double* theta, double* y);
int eigh_host(int n, const double* a, double* w, double* v);

// cgn.cu: CG on the normal equations, R systems at once; every per-system
// scalar on the device
struct CgnState {
  double thr;    // stop when rr <= thr = tol^2 ||b||^2
  double rr;     // ||r||^2, r = b - D x (recursively updated)
  double gam;    // ||D^dagger r||^2
  double alpha, beta;
  int act;       // the system iterates in the current iteration
  int its;       // iterations the system has taken
};
constexpr int kCgnMaxG = 304;   // CTAs per system of the vector kernels (2 per SM)
int cgn_grid(size_t n);
int launch_cgn_residual(int type, const void* b64, const void* t64, void* r, size_t n, int R, double* part, int G,
                        cudaStream_t s);
int launch_cgn_xr(int type, void* x, void* r, const void* p, const void* q, size_t n, int R, const CgnState* st,
                  double* part, int G, cudaStream_t s);
int launch_cgn_p(int type, void* p, const void* sv, size_t n, int R, const CgnState* st, bool init, int G,
                 cudaStream_t s);
int launch_cgn_accum(void* x64, void* x32, size_t n, int R, int G, cudaStream_t s);
int launch_cgn_gamma(const double* part_s, int nb, const double* part_r, int G, int R, CgnState* st, double tol2,
                     bool init, cudaStream_t s);
int launch_cgn_alpha(const double* part_q, int nb, int R, CgnState* st, int maxiter, cudaStream_t s);
int launch_cgn_beta(const double* part_s, int nb, const double* part_r, int G, int R, CgnState* st, cudaStream_t s);
int launch_cgn_rr(const double* part_r, int G, int R, CgnState* st, cudaStream_t s);

// learned.cu: the set-up network's layers, gate and optimiser
int launch_gconv_forward(const Geom& g, const void* U, const void* W, const void* x, void* y, int cin, int cout,
                         cudaStream_t s);
// The same with BF16 links and BF16 weights (inference), FP32 activations and accumulation.
int launch_gconv_forward_bf16(const Geom& g, const void* U, const void* W, const void* x, void* y, int cin, int cout,
                              cudaStream_t s);
int launch_gconv_backward(const Geom& g, const void* U, const void* W, const void* x, const void* gy, void* gx,
                          void* gW, int cin, int cout, cudaStream_t s);
int launch_gate(const Geom& g, const void* x, const void* gy, void* out, int channels, cudaStream_t s);
int launch_adam(size_t n, float* p, const float* gr, float* m, float* v, double lr, double b1, double b2,
                double eps, int step, cudaStream_t s);

// sap.cu
// pair_shape >= 0: an even number of right-hand sides in FP32 arithmetic
// goes to the paired kernel with that launch shape; < 0: the one-RHS-per-CTA kernel.
int launch_sap_colour(int prec, const Geom& g, void* z, const void* b, const void* U, const void* A, int colour,
                      int n_mr, int nrhs, cudaStream_t s, int pair_shape = 0, int* err = nullptr);
// The paired kernels: two right-hand sides per thread (sap2.cu).  shape 0: two
// CTAs per SM, rho re-read from shared memory for the update; 1: two CTAs per
// SM, rho kept in registers; 2: one CTA per SM, rho kept in registers; 3: one
// CTA per block holding the block's fields in shared memory for every pair;
// 4: shape 3 with the x, y, z hops of the MR steps computed without branches;
// 5: all four directions without branches; 6: shape 5 with two threads per
// site (512 per CTA, each thread one chirality and two directions; FP16/BF16
// fields only, MG_ERR_ARG for FP32 fields, whose copy would not fit in shared
// memory) (err: the device flag a bounded wait that gives up raises; needed by
// shapes 3-6).
int launch_sap_colour_pair(int prec, const Geom& g, void* z, const void* b, const void* U, const void* A, int colour,
                           int n_mr, int nrhs, cudaStream_t s, int shape, int* err);
// sap_shift.cu: the same pass for D - shift[r] (per right-hand side r; device
// array of nrhs values), the set-up's S(lambda)
int launch_sap_colour_shifted(int prec, const Geom& g, void* z, const void* b, const void* U, const void* A,
                              int colour, int n_mr, int nrhs, const double2* shift, cudaStream_t s);

// Measured FP32 FMA (scalar and packed two-wide) and shared-memory peaks (probe.cu).
int probe_peaks(cudaStream_t s, double* fp32_tflops, double* fp32x2_tflops, double* smem_gbs);

}  // namespace sapmg
