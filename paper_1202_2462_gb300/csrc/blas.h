// Vector kernels of the Krylov solvers, batched over right-hand sides (internal).
#pragma once
#include "internal.h"

namespace sapmg {

// Upper bound on the CTAs of one reduction over all right-hand sides; the
// partial buffer holds kMaxReduceCta * 16 double2.
constexpr int kMaxReduceCta = 4096;
constexpr size_t kPartialDouble2 = (size_t)kMaxReduceCta * 16;

// Geometry of a batched vector operation: R systems, n elements each; the
// vector v_j of system r is at v_j + r*vstride, w of system r at w + r*wstride.
struct BVec {
  size_t n;
  int R;
  size_t vstride;
  size_t wstride;
};
inline BVec bvec(size_t n, int R, size_t stride) { return BVec{n, R, stride, stride}; }

// Per-system complex scalars passed by value (R <= 32).
struct Scal32 { double2 v[32]; };

// out[r*ldo + j] = <v_j[r], w[r]> = sum conj(v_j) w (out2 too if non-null); mode 1 adds into out.
int blas_multidot(int type, const BVec& b, const void* const* v, int k, const void* w, double2* out, int ldo,
                  int mode, double2* out2, double2* partial, cudaStream_t s);
// w[r] += sign * sum_j coeff[r*ldc + j] v_j[r] with device coefficients.
int blas_multiaxpy(int type, const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc,
                   double sign, cudaStream_t s);
// The same, and nrm2[r*ldn] = ||w_new[r]||^2 computed in the same pass.
int blas_multiaxpy_norm(int type, const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc,
                        double sign, double2* nrm2, int ldn, double2* partial, cudaStream_t s);
// y[r] = a_r x[r] + b_r y[r]; element types tx, ty (P64 / P32); b_r = 0: y not read.
int blas_axpby2(int tx, const Scal32& a, const void* x, size_t xs, int ty, const Scal32& b, void* y, size_t ys,
                size_t n, int R, cudaStream_t s);
// out[r] = x[r] / sqrt(nrm2[r*ldn]); store[r*lds] = sqrt(nrm2[r*ldn]) if store != nullptr.
int blas_normalize(int type, const BVec& b, const void* x, void* out, const double2* nrm2, int ldn, double2* store,
                   int lds, cudaStream_t s);
// Work areas of one delayed-reorthogonalisation Arnoldi step (device, each [R][ld]
// double2 except X = [R][4]): dot products A, B, X, pass-2 coefficients c1, c2,
// and the results hcol (Hessenberg column: <v_i, w> for i < j, h_j), acol
// (<v_i, u> for i < j, beta) and nrm (||v_j||^2, ||w_new||^2).
struct DcgsWork {
  double2 *A, *B, *X, *c1, *c2, *hcol, *acol, *nrm;
  int ld;
  double2* partial;
};
// One Arnoldi step with the second Gram-Schmidt pass delayed by one step: u (the
// last basis vector, one pass done) becomes v_j, w (the operator image of the
// step) becomes w - sum_{i<=j} <v_i, w> v_i; v = the j finished basis vectors.
int blas_dcgs2_step(int type, const BVec& b, const void* const* v, int j, void* u, void* w, const DcgsWork& ws,
                    cudaStream_t s);
// The same step (FP32 u and w) with the finished basis vectors stored in FP16,
// scaled by 2^10: vh = v_0 .. v_{j-1}; the new v_j is written to vout in the
// same format only (u's contents are undefined afterwards); u need not be
// normalised.
int blas_dcgs2_step_h(const BVec& b, const void* const* vh, int j, void* u, void* w, void* vout, const DcgsWork& ws,
                      cudaStream_t s);
// Kernels on FP16 basis vectors (scaled by 2^10, as blas_dcgs2_step_h stores
// them) with FP32 w / x: <v_j, w>; w += sign sum c_j v_j (and ||w_new||^2 when
// nrm2 != nullptr); out = x / ||x|| stored in the FP16 format.
int blas_multidot_h(const BVec& b, const void* const* v, int k, const void* w, double2* out, int ldo,
                    double2* partial, cudaStream_t s);
int blas_multiaxpy_h(const BVec& b, void* w, const void* const* v, int k, const double2* coeff, int ldc, double sign,
                     double2* nrm2, int ldn, double2* partial, cudaStream_t s);
int blas_normalize_h(const BVec& b, const void* x, void* out, const double2* nrm2, int ldn, double2* store, int lds,
                     cudaStream_t s);
// y[r] = argmin || sqrt(beta2[r]) e1 - H_r y || for (m+1) x m Hessenberg H_r (column-major, ldh; H_r at H + r*ldr).
int blas_hessenberg_solve(const double2* H, int ldh, int ldr, int m, const double2* beta2, double2* y, int ldy,
                          int R, cudaStream_t s);

}  // namespace sapmg
