/*
 * sapmg.h -- C-ABI of the GB300 SAP-multilevel solver for the clover-improved
 * Wilson-Dirac equation D z = b (Frommer, Kahl, Krieg, Leder, Rottmann,
 * "Aggregation-based Multilevel Methods for Lattice QCD", Lattice 2011).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Lattice dims (Lx, Ly, Lz, Lt), x fastest, periodic; the fermion field may be
 * antiperiodic in t.  Every dim must be a multiple of 8 (an even number of
 * 4^4 Schwarz blocks per direction, Sec. 2: two-colouring).
 *
 * Canonical layouts (what the caller passes unless MG_BLOCKED is set):
 *   gauge  U : [V][mu = x,y,z,t][3][3] complex128, the forward links U_mu(x);
 *   spinor   : [nrhs][V][spin 4][colour 3] complex (complex128 for MG_FP64,
 *              complex64 otherwise), site = ((t*Lz + z)*Ly + y)*Lx + x;
 *   coarse   : [nrhs][coarse site][2N] complex, coarse site canonical on the
 *              lattice of aggregates, dof index chi*N + k (chirality chi of
 *              gamma_5^c = diag(+1_N, -1_N), test vector k).
 * Gamma matrices are in the chiral basis: gamma_k = [[0, -i s_k], [i s_k, 0]]
 * (k = x, y, z), gamma_t = [[0, 1], [1, 0]], gamma_5 = diag(1, 1, -1, -1).
 *
 * Pointers: every field argument is a DEVICE pointer owned by the caller (for
 * instance a torch tensor's data_ptr()), except where stated.  The library
 * copies what it keeps; it never frees caller memory.  All work is issued on
 * the stream given in mg_params.stream (NULL = legacy default stream) and is
 * asynchronous unless stated; mg_solve synchronises.  A context is not
 * thread-safe.
 *
 * Errors: 0 = MG_OK.  Negative codes are errors and leave outputs undefined;
 * mg_last_error() returns a message.  MG_NOT_CONVERGED (positive) means the
 * solve hit its iteration cap; the output holds the best iterate.
 */
#ifndef SAPMG_H
#define SAPMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MG_OK 0
#define MG_NOT_CONVERGED 1
#define MG_ERR_ARG (-1)       /* null pointer, bad dims, unsupported option */
#define MG_ERR_NONFINITE (-2) /* NaN or Inf in an input field */
#define MG_ERR_OOM (-3)       /* device allocation failed */
#define MG_ERR_CUDA (-4)      /* a CUDA call failed; see mg_last_error() */
#define MG_ERR_TIMEOUT (-5)   /* a bounded device wait gave up */
#define MG_ERR_STATE (-6)     /* the call needs a part the context was not set up with */
#define MG_ERR_BOUNDS (-7)    /* MG_DEBUG builds only: a device-side index check failed */

/* Precisions.  MG_FP64: storage and arithmetic in binary64 (the plain form).
 * MG_FP32 / MG_FP16 / MG_BF16: binary32 arithmetic with links, clover blocks,
 * test vectors and coarse operators stored in that format (the mixed form).  */
#define MG_FP64 0
#define MG_FP32 1
#define MG_FP16 2
#define MG_BF16 3
/* OR-ed into a prec argument: spinors are in the library's internal blocked
 * layout (see mg_pack_spinor) instead of the canonical one. */
#define MG_BLOCKED 0x100
/* OR-ed into dirac_apply's prec: apply D^dagger = gamma5 D gamma5 instead of D
 * (MG_FP64 or MG_FP32 only). */
#define MG_DAGGER 0x200
/* OR-ed into dirac_apply's prec with MG_FP64 (not with MG_DAGGER): the same
 * FP64 operator on FP64 data, with the arithmetic in double-float (pairs of
 * FP32 numbers, about 48 significand bits) on the FP32 units.  Measured
 * slower than the FP64 units on GB300 (96 against 51 ms for 12 right-hand
 * sides at 32^3 x 64), so the solver does not use it unless the environment
 * sets SAPMG_FP64_ON_FP32=1. */
#define MG_FP64_ON_FP32 0x400

typedef struct mg_ctx mg_ctx;

typedef struct {
  int dims[4];              /* Lx, Ly, Lz, Lt; each a multiple of 8 */
  int antiperiodic_t;       /* 1: fermion field antiperiodic in t */
  int n_levels;             /* 1 (Schwarz-preconditioned FGMRES), 2 or 3 */
  int agg2[4];              /* 3 levels: level-1 aggregate in coarse sites (default 2^4) */
  int sap_block2[4];        /* 3 levels: level-1 Schwarz block in coarse sites (default 2^4) */
  int n_vec[2];             /* test vectors N per non-coarsest level (Sec. 3) */
  int setup_iters;          /* bootstrap part 1: smoother sweeps per level (Sec. 3) */
  int n_mr;                 /* MR steps per Schwarz block solve (Sec. 2) */
  int nu_post;              /* Schwarz sweeps per multilevel cycle */
  int coarse_iters;         /* GMRES steps on the coarsest level (Sec. 4: 12) */
  int inner_iters;          /* 3 levels: flexible GMRES steps on level 1 */
  int fgmres_m;             /* outer restart length (Sec. 4: 25) */
  double tol;               /* relative residual target (Sec. 4: 1e-10) */
  int maxiter;              /* cap on preconditioned iterations per right-hand side */
  int precision;            /* MG_FP64 (plain form) or MG_FP32 / MG_FP16 / MG_BF16 */
  int nrhs_max;             /* right-hand sides solved together by mg_solve */
  unsigned long long seed;  /* seed of the random initial test vectors */
  void* stream;             /* cudaStream_t; NULL = default stream */
  const double* init_vectors; /* optional device pointer: n_vec[0] canonical
                                 complex128 fine fields used instead of the
                                 random initial test vectors */
  int verbose;
  int setup2_iters;         /* set-up part 2 (Sec. 3; two or three levels):
                               Schwarz sweeps iota of S(lambda) per harmonic
                               Ritz vector; 0 = part 1 only */
  const double* setup2_start; /* optional device pointer: start vector of the
                                 part-2 Arnoldi process on the coarsest
                                 operator, complex128 [coarse site][2N] of the
                                 coarsest level (sites in block order);
                                 NULL = drawn from seed */
  int autotune;             /* 1: at the end of mg_setup, time the candidate
                               launch shapes of the mixed form's multi-RHS
                               kernels for nrhs_max right-hand sides and keep
                               the fastest (see mg_get_tuning); 0 = defaults */
  int init_vectors_prec;    /* type of init_vectors: MG_FP64 (complex128,
                               the default) or MG_FP32 (complex64, half the
                               caller's memory; widened to FP64 on entry) */
} mg_params;

typedef struct {
  int iterations;      /* preconditioned Krylov iterations, summed over right-hand sides */
  int restarts;        /* plain form: FGMRES restarts; mixed form: FP64 defect corrections (summed) */
  double relres;       /* largest final true relative residual ||b - D z||/||b|| (FP64) */
  double seconds;      /* wall time of the call */
  double precond_seconds;  /* device time in the multilevel preconditioner (profiling on) */
} mg_solve_info;

/* Fill *p with defaults: 1 level, 4 MR steps, 2 post sweeps, N = 8, 3 set-up
 * sweeps, 12 coarse steps, 8 inner steps, FGMRES(20), tol 1e-10, maxiter 1000,
 * MG_FP64, nrhs_max 1, agg2 = sap_block2 = 2^4.  dims must still be set. */
int mg_default_params(mg_params* p);

/* Build a solver context (Sec. 3, set-up part 1).
 * U: device, canonical gauge field, complex128 (read during the call only; the
 *    caller may free it afterwards).  c_sw: clover coefficient; m0: bare mass,
 *    D = 4 + m0 - hopping/2 + clover (kappa = 1/(2 m0 + 8)).
 * Builds the clover term, packs U in every precision the context needs, runs
 * the bootstrap set-up (Schwarz sweeps on random or given test vectors, kept
 * orthonormal; local orthonormalisation; D_c = P^dagger D P, recursively),
 * with setup2_iters > 0 also its second part, run once from the coarsest
 * level (harmonic Ritz vectors of the coarsest operator interpolated to the
 * fine level, smoothed by S(lambda), merged with the part-1 vectors by the
 * (DV)^dagger DV reduction; P and D_c rebuilt; with three levels, level 1 is
 * then rebuilt from the new vectors as part 1 builds it), and allocates all
 * solve workspace.  The plain form does all of this in FP64; the mixed form
 * keeps the test vectors FP32 through the part-1 sweeps and their global
 * Gram-Schmidt and assembles the level-1 D_c in FP32 arithmetic (the local
 * orthonormalisation stays FP64).  Synchronises.  *out receives the context.
 * Errors: MG_ERR_ARG (dims, params), MG_ERR_NONFINITE (U), MG_ERR_OOM, MG_ERR_CUDA. */
int mg_setup(const double* U, double c_sw, double m0, const mg_params* p, mg_ctx** out);

/* out = D in (Sec. 1, Eq. 1.1) for nrhs fields.  prec: MG_FP64 (complex128
 * fields, FP64 links) or the context's mixed precision / MG_FP32 (complex64
 * fields; links and clover stored in that precision), optionally | MG_BLOCKED,
 * and | MG_DAGGER for D^dagger = gamma5 D gamma5 (MG_FP64 / MG_FP32 only).
 * in and out must not overlap.  Asynchronous. */
int dirac_apply(mg_ctx* ctx, const void* in, void* out, int prec, int nrhs);

/* n_sweeps red-black Schwarz sweeps (Sec. 2, Algorithm 1) on D z = b, updating z
 * in place (z is the starting guess).  Each sweep: for colour 0 then 1,
 * r = b - D z and z += (n_MR MR steps of the block system) on every block of
 * that colour.  prec and layout as for dirac_apply.  Asynchronous (a bounded
 * device wait that gives up is reported by the next synchronising call, e.g.
 * mg_sync). */
int sap_smooth(mg_ctx* ctx, const void* b, void* z, int n_sweeps, int prec, int nrhs);

/* Solve D z = b for nrhs right-hand sides to ||b - D z|| <= tol ||b|| (Sec. 4).
 * b, z: device, canonical complex128.  Plain form (MG_FP64): FGMRES(m) in FP64
 * with the FP64 multilevel cycle as right preconditioner.  Mixed form: FP64
 * defect correction (r = b - D z recomputed in FP64) around FP32 FGMRES(m)
 * whose preconditioner is the FP32/FP16/BF16 cycle.  Synchronises.
 * info may be NULL.  Returns MG_OK, MG_NOT_CONVERGED or an error;
 * MG_ERR_NONFINITE if the recomputed residual is not finite (NaN or Inf in b,
 * or a breakdown of the reduced-precision iteration). */
int mg_solve(mg_ctx* ctx, const double* b, double* z, int nrhs, mg_solve_info* info);

/* Solve D z = b by CG on the normal equations D^dagger D z = D^dagger b (CGN,
 * the method the multilevel solver is compared with in Sec. 4, Tables 1-2),
 * from z = 0, until ||b - D z|| <= tol ||b|| for every right-hand side, where
 * the residual is the one the CG recursion updates and is recomputed in FP64
 * (b - D z) before the call returns.  No preconditioner and no multilevel
 * set-up are used, so any context serves.  b, z: device, canonical
 * complex128, nrhs fields, solved nrhs_max at a time.
 * prec: MG_FP64 (every vector, the links and the clover in FP64) or MG_FP32
 *   (FP32 iteration with the FP32 links and clover of a mixed-form context;
 *   the iterate is added to the FP64 solution and the residual recomputed in
 *   FP64 each time it has fallen by 1e-2, keeping the search direction).
 * maxiter: cap on CG iterations per right-hand side.
 * info (may be NULL): iterations summed over right-hand sides, restarts = the
 * FP64 residual recomputations, relres = the largest final FP64 relative
 * residual.  Allocates 48 bytes per complex entry per right-hand side on the
 * first call (kept by the context).  Synchronises.  Returns MG_OK,
 * MG_NOT_CONVERGED (z holds the last iterate), MG_ERR_ARG (tol <= 0,
 * maxiter < 1, other prec), MG_ERR_STATE (MG_FP32 in a plain-form context),
 * MG_ERR_NONFINITE, MG_ERR_OOM or MG_ERR_CUDA. */
int mg_cgn_solve(mg_ctx* ctx, const double* b, double* z, int nrhs, int prec, double tol, int maxiter,
                 mg_solve_info* info);

/* Harmonic Ritz pairs (Sec. 3, set-up part 2) of an Arnoldi relation
 * A V_m = V_{m+1} Hbar, on the host: the pairs (theta, y) with
 * Hbar^H Hbar y = theta H_m^H y (H_m the top m x m part), i.e. A V_m y - theta
 * V_m y orthogonal to A V_m.  hbar: (m+1) x m complex, column-major, re/im
 * interleaved (host).  theta: m complex, sorted by |theta|; y: m x m complex,
 * column k the unit-norm coefficient vector of theta_k (host, caller-owned).
 * Returns MG_OK, MG_ERR_ARG, or MG_ERR_NONFINITE (H_m singular or the QR
 * iteration did not converge).  Used by the set-up; exported for checking. */
int mg_harmonic_ritz(int m, const double* hbar, double* theta, double* y);

/* Eigen-decomposition of a Hermitian n x n complex matrix on the host (the
 * (DV)^dagger DV reduction of set-up part 2): a column-major, re/im
 * interleaved; w: n ascending eigenvalues; v: n x n orthonormal eigenvectors
 * (column k for w[k]).  Returns MG_OK or MG_ERR_ARG.  Used by the set-up;
 * exported for checking. */
int mg_eigh(int n, const double* a, double* w, double* v);

/* Free every device buffer the context owns. */
/* Checkpoint of a set-up (no paper counterpart; Sec. 3's set-up is built
 * once and serves every later solve): write the context's test vectors --
 * the locally orthonormal vectors defining P on level 0 and, with three
 * levels, on level 1, in FP64 -- with the lattice, levels, N, blocking, m0 and
 * c_sw they belong to and a checksum, to the file `path`.  Synchronises. */
int mg_save(mg_ctx* ctx, const char* path);
/* Build a context as mg_setup does, except that the test vectors come from a
 * file written by mg_save instead of the bootstrap set-up (both parts): P and
 * the coarse operators are rebuilt from them and the links U given here.
 * The file's lattice, levels, N, blocking, m0 and c_sw must equal the
 * arguments (MG_ERR_ARG otherwise, also for a truncated or corrupted file);
 * precision, nrhs_max and the solver parameters may differ.  Synchronises. */
int mg_setup_load(const double* U, double c_sw, double m0, const mg_params* p, const char* path, mg_ctx** out);

void mg_destroy(mg_ctx* ctx);

/* Message of the last error (thread-local, valid until the next call). */
const char* mg_last_error(void);

/* sizeof(mg_params), for bindings that mirror the struct. */
unsigned long mg_sizeof_params(void);

/* ---- inspection and component entry points (used by the parity tests) ---- */

/* Spinor layout conversion canonical <-> internal blocked (prec: MG_FP64 or
 * MG_FP32 element type, same on both sides). */
int mg_pack_spinor(mg_ctx* ctx, const void* canonical, void* blocked, int prec, int nrhs);
int mg_unpack_spinor(mg_ctx* ctx, const void* blocked, void* canonical, int prec, int nrhs);

/* The clover matrix A(x) = (4 + m0) + c_sw (i/2) sum sigma F (FP64) as two dense
 * 6x6 chiral blocks: out device [V][chi][6][6] complex128, canonical sites,
 * index within a block (spin - 2 chi)*3 + colour. */
int mg_clover_export(mg_ctx* ctx, double* out);

/* The locally orthonormalised test vectors defining P of level `level` (0:
 * fine -> level 1, 1: level 1 -> level 2) as FP64 fields: out device
 * [N][fine-level field] complex128 in that level's canonical layout. */
int mg_get_vectors(mg_ctx* ctx, int level, double* out);

/* The coarse operator of level `level` (1 or 2) as FP64 stencil: out device
 * [coarse site][9][2N][2N] complex128, row-major (row i, column j); direction
 * 0 = self, 1 + 2 mu = +mu, 2 + 2 mu = -mu (mu = x, y, z, t), i.e.
 * (D_c x)(a) = sum_d M_d(a) x(a + offset_d).  The plain (FP64) form
 * assembles it in FP64 arithmetic; the mixed form, which stores and applies
 * it in FP32 and FP16, assembles level 1 in FP32 arithmetic from FP32 copies
 * of the vectors, links and clover (relative accuracy about 1e-6). */
int mg_get_coarse_op(mg_ctx* ctx, int level, double* out);

/* v_c = P^dagger v (restriction) and v = P v_c (interpolation) between level
 * `level` and level + 1, and v_out = D_c v_in on level `level` >= 1.
 * Element type: complex128 for MG_FP64, complex64 otherwise (fine side
 * canonical unless MG_BLOCKED).  Asynchronous. */
int mg_restrict(mg_ctx* ctx, int level, const void* in, void* out, int prec);
int mg_prolong(mg_ctx* ctx, int level, const void* in, void* out, int prec);
int mg_coarse_apply(mg_ctx* ctx, int level, const void* in, void* out, int prec);
/* Restriction and interpolation of nrhs <= nrhs_max vectors stored back to
 * back (fine side [nrhs][field], coarse side [nrhs][sites][2N]), the batched
 * form the cycle uses.  In the mixed form with 1 < nrhs <= 16 the level-0
 * restriction and interpolation run on the tensor cores: the FP32 vectors and
 * the stored P enter as TF32 (10-bit mantissa, rounded to nearest), sums are
 * FP32 (environment SAPMG_RESTRICT_TF32=0 selects the FP32 forms).
 * Asynchronous. */
int mg_restrict_batch(mg_ctx* ctx, int level, const void* in, void* out, int prec, int nrhs);
int mg_prolong_batch(mg_ctx* ctx, int level, const void* in, void* out, int prec, int nrhs);
/* The same for nrhs coarse vectors stored back to back ([nrhs][sites][2N]);
 * synchronises (it checks the device error flag of the bounded waits). */
int mg_coarse_apply_batch(mg_ctx* ctx, int level, const void* in, void* out, int prec, int nrhs);

/* Approximate solve on coarse level `level` >= 1 exactly as the cycle does it
 * (fixed-step GMRES on the coarsest level, fixed-step flexible GMRES with the
 * level's cycle otherwise), from zero. */
int mg_coarse_solve(mg_ctx* ctx, int level, const void* in, void* out, int prec);

/* The coarse solve of mg_coarse_solve without any device allocation.
 * The paper has no counterpart: this entry point is for callers that cannot
 * call cudaMalloc at the time they solve -- code running under an allocator
 * that forbids new device memory (a memory pool sized up front, or an
 * allowance that another framework owns), or on a real-time path where an allocation's
 * implicit synchronisation or its failure is not acceptable.  Its Krylov
 * basis, Hessenberg matrix and reduction partials live in a fixed 8 MiB array
 * inside the library's own device memory (every device that loads the library
 * holds it until the process exits); the result is written straight to `out`,
 * which starts from zero.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) with the device current.  Every call
 * shares the one array,
 * which keeps the previous call's contents, so calls that overlap on the GPU
 * (other streams, other contexts on the same device) race: serialise them.
 * Two-level contexts only (level 1 is then the coarsest level, solved by
 * fixed-step GMRES); a three-level context gets MG_ERR_STATE.  The Krylov
 * basis is kept in the context's vector precision (FP64, or FP32 in the mixed
 * form): where mg_coarse_solve keeps the mixed form's basis in FP16 (the FP16
 * operator copy exists, 2N a multiple of 8), the two results differ by the
 * FP16 rounding of that basis.  A coarse system whose basis does not fit
 * (about (coarse_iters + 2) vectors of the level's size) is rejected with
 * MG_ERR_ARG and a message naming the sizes.  Synchronises. */
int mg_coarse_solve_noalloc(mg_ctx* ctx, int level, const void* in, void* out, int prec);

/* One application of the multilevel cycle z = M v on the fine level (the
 * outer solver's preconditioner).  prec: MG_FP64 for a plain-form context,
 * MG_FP32 for a mixed one.  Asynchronous. */
int mg_precondition(mg_ctx* ctx, const void* v, void* z, int prec);

/* ---- Learned set-up (not in the paper): a gauge-covariant convolutional
 * network that proposes near-kernel test vectors from noise, trained to
 * imitate the bootstrap set-up (Sec. 3), which stays the fallback.
 * Layer: out_a(x) = sum_b sum_h W[a][b][h] (T_h in_b)(x), T_0 = identity,
 * T_{+mu} psi(x) = U_mu(x) psi(x + mu), T_{-mu} psi(x) = U_mu(x - mu)^dagger
 * psi(x - mu), hop h = 0, 1 + 2 mu (+mu), 2 + 2 mu (-mu), mu = x, y, z, t;
 * W[a][b][h] a complex 4 x 4 spin matrix.  W: device complex64
 * [cout][cin][9][4][4] (row s, column t).  Fields: device complex64, blocked
 * layout (mg_pack_spinor), channel c at c * 12V.  The transports use the
 * context's FP32 links (mixed-form contexts only; MG_ERR_STATE otherwise),
 * including an antiperiodic t sign if the context has one.  Gradients follow
 * G_z = dL/dRe z + i dL/dIm z.  Asynchronous except mg_net_loss. */
int mg_net_layer_forward(mg_ctx* ctx, int cin, int cout, const void* W, const void* x, void* y);
/* The same layer for inference with BF16 storage: W device BF16 complex pairs
 * [cout][cin][9][4][4] (re, im), the context's BF16 links (a context of
 * precision MG_BF16; MG_ERR_STATE otherwise), FP32 activations x, y and FP32
 * accumulation. */
int mg_net_layer_forward_bf16(mg_ctx* ctx, int cin, int cout, const void* W, const void* x, void* y);
/* gx = sum_h T_h^dagger sum_a W[a][b][h]^dagger gy_a (skipped if gx is NULL);
 * gW[a][b][h] = sum_x gy_a(x) (T_h x_b)(x)^dagger (skipped if gW is NULL;
 * a fixed-order reduction, deterministic). */
int mg_net_layer_backward(mg_ctx* ctx, int cin, int cout, const void* W, const void* x, const void* gy, void* gx,
                          void* gW);
/* Gate between layers: y = x / sqrt(1 + |x(site)|^2) per channel and site;
 * backward gx = s gy - (1 + n)^(-3/2) Re<gy, x>_site x. */
int mg_net_gate_forward(mg_ctx* ctx, int channels, const void* x, void* y);
int mg_net_gate_backward(mg_ctx* ctx, int channels, const void* x, const void* gy, void* gx);
/* loss = ||y - t||^2 / ||t||^2 (returned on the host; synchronises) and
 * gy = 2 (y - t) / ||t||^2 (one channel). */
int mg_net_loss(mg_ctx* ctx, const void* y, const void* t, void* gy, double* loss);
/* Adam on n FP32 parameters (first and second moments m, v; step >= 1). */
int mg_adam_step(mg_ctx* ctx, size_t n, float* p, const float* g, float* m, float* v, double lr, double beta1,
                 double beta2, double eps, int step);

/* Per-kernel device timing with CUDA events recorded on the context's stream
 * around every launch of the selected kernel families.  mask: 0 = off, 1 = all
 * families, otherwise bit (f + 1) selects family f (0 dirac, 1 Schwarz colour
 * pass, 2 coarse apply, 3 restrict, 4 prolong, 5 fine-level vector kernels
 * of the outer solver, 6 vector kernels of the coarse-level solves, 7 the
 * level-1 Schwarz colour pass of a three-level hierarchy).  mg_get_profile
 * returns a family's timed launch count and summed milliseconds (it
 * synchronises on the pending events). */
int mg_set_profiling(mg_ctx* ctx, int mask);
int mg_get_profile(mg_ctx* ctx, int family, long long* launches, double* ms);
/* The algorithmic bytes of the timed launches of a level-0 family (every
 * operand read once and every result written once: fields in storage
 * precision, the right-hand sides' vectors, P, the coarse operator), summed
 * like mg_get_profile's milliseconds; their ratio is the family's achieved
 * bandwidth.  The level-1 Schwarz passes count their operator reads (every
 * MR step reads the box's operator; once for all right-hand sides in the
 * multi-RHS form, once per right-hand side otherwise); the level-1 transfers
 * add no bytes. */
int mg_get_profile_bytes(mg_ctx* ctx, int family, double* bytes);
int mg_reset_profile(mg_ctx* ctx);

/* Number of kernel launches the library has issued in this process. */
long long mg_launch_count(void);

/* The launch shapes a context uses (no paper counterpart): out[0] = how they
 * were chosen (0 defaults, 1 timed by the autotuner at set-up, 2 taken from
 * the autotuner's cache of an earlier context with the same lattice, N,
 * nrhs_max, precision and levels), out[1] = Schwarz launch shape (0: two CTAs
 * per SM, rho re-read for the update; 1: rho in registers; 2: one CTA per SM;
 * 3: one CTA per block with the block's fields in shared memory, every pair
 * of right-hand sides in turn; 4, 5: shape 3 with the x, y, z (4) or all (5)
 * hops computed without branches; 6: shape 5 with two threads per site, each
 * one chirality and two directions, FP16/BF16 fields only), out[2] =
 * right-hand sides per transfer launch, out[3] = ring depth, out[4] =
 * CTA-per-SM cap (0: none) and out[5] = right-hand sides per launch of the
 * FP16 tensor-core coarse stencil.  Every choice computes the same results bit
 * for bit, except Schwarz shape 6, which adds a site's hops in another order
 * (the results agree to FP32 rounding); only the time differs. */
int mg_get_tuning(mg_ctx* ctx, int* out);

/* Residual history of the context's last mg_solve (no paper counterpart;
 * metrics): entries of three doubles (iteration, right-hand side, relative
 * residual).  iteration >= 1: the least-squares residual estimate of the
 * flexible GMRES after that many preconditioned iterations of that
 * right-hand side, scaled to ||b - D x|| / ||b|| (in the mixed form through
 * the FP64 correction's ||r||); iteration = -(k + 1): the FP64-recomputed
 * ||b - D x|| / ||b|| after k iterations (every restart or defect
 * correction, and the final one).  Copies at most max_entries entries to out
 * (out may be NULL) and returns the number stored. */
int mg_get_history(mg_ctx* ctx, double* out, int max_entries);

/* Wait for the context's stream and report a device-side wait that gave up
 * since the last check (MG_ERR_TIMEOUT; the flag is then cleared).  The
 * asynchronous entry points (sap_smooth, dirac_apply, the transfers) leave
 * such a flag for the next synchronising call; this one only checks it.
 * In an MG_DEBUG build the synchronising calls also report a failed
 * device-side index check (MG_ERR_BOUNDS, see mg_debug_failures). */
int mg_sync(mg_ctx* ctx);

/* The MG_DEBUG build (libsapmg_debug.so, compiled with -DMG_DEBUG) checks in
 * its kernels the indices they compute -- neighbour sites and blocks, the
 * blocks of a colour, coarse sites and their neighbours, aggregates, kernel
 * block indices -- and the 16-byte alignment of every bulk copy.  A failed
 * check never traps: it is recorded on the device and the kernel carries on
 * with index 0 (or skips the copy), so results are then wrong but every
 * barrier and wait behaves as in the release build.  This call synchronises
 * the device and returns the number of failed checks since the previous call
 * (clearing them), with mg_last_error() describing the first one (file, kind,
 * value, source line); MG_ERR_CUDA if the records cannot be read.  In the
 * release build (libsapmg.so) it returns -1: no checks are compiled. */
long long mg_debug_failures(void);

/* MG_DEBUG build: one device-side check of value against [0, bound) in a
 * one-thread kernel that touches no memory (a failure is recorded as a
 * "block" check of solver.cu), for tests of the reporting path.
 * Asynchronous on the legacy default stream; MG_OK.  Release build:
 * MG_ERR_STATE. */
int mg_debug_check(long long value, long long bound);

/* Bound on the main-loop waits of the kernels that stage data with bulk
 * copies (the coarse stencils, the block-resident Schwarz pass): a wait that
 * has not completed after `spins` tries gives up, the kernel drains its copies
 * in flight (those waits keep the default bound) and raises the flag that the
 * synchronising calls report as MG_ERR_TIMEOUT.  spins < 0 restores the
 * default (2^22 tries); 0 makes every such wait give up at once, which tests
 * of the timeout path use.  Diagnostics only.  Synchronises. */
int mg_set_wait_limit(mg_ctx* ctx, int spins);

/* Measured peaks of the current device, the denominators of the roofline of
 * the CUDA-core kernels (no paper counterpart; measurement only): FP32 FMA
 * throughput with scalar FMAs and with the packed two-wide FMA (TFLOP/s,
 * 2 flop per FMA), and shared-memory load bandwidth (GB/s), each the best of
 * ten timed launches of a probe kernel that fills every SM, after three
 * warm-up launches.  stream: a cudaStream_t (NULL: the legacy default
 * stream).  Allocates a few KB with cudaMallocAsync; synchronises; takes
 * about a tenth of a second. */
int mg_probe_peaks(void* stream, double* fp32_tflops, double* fp32x2_tflops, double* smem_gbs);

#ifdef __cplusplus
}
#endif

#endif /* SAPMG_H */
