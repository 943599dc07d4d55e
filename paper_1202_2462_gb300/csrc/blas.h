// Vector kernels of the Krylov solvers (internal).
#pragma once
#include "internal.h"

namespace sapmg {

// Upper bound on the CTAs of a reduction; partial buffers hold kMaxReduceCta * 8 double2.
constexpr int kMaxReduceCta = 1024;

// out[j] = <v_j, w> = sum conj(v_j) w for j < k (out2[j] too if non-null); mode 1 adds into out.
int blas_multidot(int type, const void* const* v, int k, const void* w, size_t n, double2* out, int mode,
                  double2* out2, double2* partial, cudaStream_t s);
// w += sign * sum_j coeff[j] v_j with device coefficients.
int blas_multiaxpy(int type, void* w, const void* const* v, int k, const double2* coeff, double sign, size_t n,
                   cudaStream_t s);
// y = a x + b y (b = 0: y is not read).
int blas_axpby(int type, double2 a, const void* x, double2 b, void* y, size_t n, cudaStream_t s);
// The same with element types tx of x and ty of y (P64 / P32 each).
int blas_axpby2(int tx, double2 a, const void* x, int ty, double2 b, void* y, size_t n, cudaStream_t s);
// out = x / sqrt(*nrm2); *store = sqrt(*nrm2).
int blas_normalize(int type, const void* x, void* out, const double2* nrm2, double2* store, size_t n, cudaStream_t s);
// y = argmin || sqrt(*beta2) e1 - H y || for the (m+1) x m Hessenberg H (column-major, ldh), m <= 32.
int blas_hessenberg_solve(const double2* H, int ldh, int m, const double2* beta2, double2* y, cudaStream_t s);

}  // namespace sapmg
