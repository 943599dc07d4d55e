// Host orchestration and the C-ABI: context and set-up (Sec. 3, bootstrap part
// 1), the multilevel cycle, the device-resident fixed-step coarse GMRES, the
// outer flexible GMRES (Sec. 2, Sec. 4) and FP64 defect correction.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <string>
#include <vector>
#include <atomic>
#include <mutex>

#include "async.cuh"
#include "internal.h"
#include "blas.h"
#include "coarse.h"

namespace sapmg {

static thread_local std::string g_err;
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
static std::atomic<long long> g_bytes{0};
void count_bytes(double bytes) { g_bytes.fetch_add((long long)bytes, std::memory_order_relaxed); }
long long bytes_counted() { return g_bytes.load(std::memory_order_relaxed); }
void set_last_error(const char* msg, const char* file, int line) {
  g_err = std::string(msg) + " (" + file + ":" + std::to_string(line) + ")";
}
static int fail(int code, const std::string& m) {
  g_err = m;
  return code;
}

// ---- device-side index checks (MG_DEBUG builds; debug.cuh)
namespace dbg {
const char* kind_name(int kind) {
  static const char* names[kKinds] = {"none",        "neighbour block",  "neighbour site",
                                      "block of a colour", "block",      "coarse site",
                                      "coarse neighbour",  "aggregate",  "bulk-copy alignment"};
  return (kind > 0 && kind < kKinds) ? names[kind] : "unknown";
}
struct ReaderEntry {
  Reader read;
  const char* unit;
};
static std::vector<ReaderEntry>& readers() {
  static std::vector<ReaderEntry> r;
  return r;
}
int add_reader(Reader r, const char* unit) {
  readers().push_back({r, unit});
  return (int)readers().size();
}
// Failed checks of every unit since the last collection (the records are
// cleared); msg describes the first one.  -1 if a record could not be read.
static long long collect(std::string* msg) {
  long long total = 0;
  for (const ReaderEntry& e : readers()) {
    unsigned long long first = 0, fails = 0;
    if (e.read(&first, &fails) != 0) return -1;
    if (fails && total == 0 && msg) {
      const char* base = std::strrchr(e.unit, '/');
      *msg = std::string("device-side index check failed in ") + (base ? base + 1 : e.unit) + ": " +
             kind_name((int)(first >> 56)) + " " + std::to_string((int)(uint32_t)first) + " out of range (line " +
             std::to_string((int)((first >> 32) & 0xffffff)) + ")";
    }
    total += (long long)fails;
  }
  if (total && msg) *msg += ", " + std::to_string(total) + " failed check(s) in all";
  return total;
}
#ifdef MG_DEBUG
// one check of v against [0, n) by one thread, with no memory access
__global__ void selftest_kernel(long long v, long long n) { (void)MG_CHECK(kBlock, v, n); }
#endif
}  // namespace dbg

#define TRY(x)                  \
  do {                          \
    int rc__ = (x);             \
    if (rc__ < 0) return rc__;  \
  } while (0)

// TRY for a vector-kernel call, timed as the fine-level (BLAS) or coarse-level
// (CBLAS) vector family when profiling is on
#define BLAS(x)                                     \
  do {                                              \
    ProfScope ps__(c->prof, FAM_BLAS, c->s);        \
    int rc__ = (x);                                 \
    if (rc__ < 0) return rc__;                      \
  } while (0)
#define CBLAS(x)                                    \
  do {                                              \
    ProfScope ps__(c->prof, FAM_CBLAS, c->s);       \
    int rc__ = (x);                                 \
    if (rc__ < 0) return rc__;                      \
  } while (0)

enum {
  FAM_DIRAC = 0, FAM_SAP = 1, FAM_COARSE = 2, FAM_RESTRICT = 3, FAM_PROLONG = 4, FAM_BLAS = 5, FAM_CBLAS = 6,
  FAM_SAP1 = 7, FAM_N = 8
};

struct Prof {
  bool on = false;
  unsigned mask = 0;   // families timed (bit f = family f)
  struct Rec { int fam; cudaEvent_t a, b; long long bytes; };
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> pending;
  long long launches[FAM_N] = {};
  double ms[FAM_N] = {};
  double bytes[FAM_N] = {};
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& r : pending) {
      float t = 0;
      cudaEventSynchronize(r.b);
      cudaEventElapsedTime(&t, r.a, r.b);
      ms[r.fam] += t;
      launches[r.fam] += 1;
      bytes[r.fam] += (double)r.bytes;
      pool.push_back(r.a);
      pool.push_back(r.b);
    }
    pending.clear();
  }
  ~Prof() {
    for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct ProfScope {
  Prof& p;
  int fam;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  long long b0 = 0;
  bool act;
  ProfScope(Prof& p_, int f, cudaStream_t s_) : p(p_), fam(f), s(s_), act(p_.on && ((p_.mask >> f) & 1u)) {
    if (act) { a = p.get(); cudaEventRecord(a, s); b0 = bytes_counted(); }
  }
  ~ProfScope() {
    if (act) {
      cudaEvent_t b = p.get();
      cudaEventRecord(b, s);
      p.pending.push_back({fam, a, b, bytes_counted() - b0});
      if (p.pending.size() > 4096) p.drain();
    }
  }
};

struct CoarseLevel {
  CGeom cg;
  int store = P64;           // storage precision of M
  void* M64 = nullptr;       // FP64 operator (set-up result, export)
  void* M = nullptr;         // operator used by the solver (== M64 in FP64)
  void* Mh = nullptr;        // FP16 copy for the tensor-core stencil (mixed form, SAPMG_COARSE_FP16=0: none)
  void* Vh = nullptr;        // FP16 Krylov basis of the coarse GMRES (with Mh; SAPMG_COARSE_BASIS_FP16=0: none)
  // fixed-step GMRES workspace for R right-hand sides (vector type = the cycle's)
  void* V = nullptr;         // (kmax + 1) batched vectors, vector j at V + j*R*n
  void* w = nullptr;         // batched [R][n]
  void* x = nullptr;
  void* b = nullptr;
  double2* H = nullptr;      // [R][33 x 33] column-major
  double2* tmp = nullptr;    // [R][64] scratch scalars
  double2* beta2 = nullptr;  // [R]
  double2* y = nullptr;      // [R][33]
  size_t n() const { return (size_t)cg.nsites * cg.n2; }
};

}  // namespace sapmg

using namespace sapmg;

struct mg_ctx {
  mg_params p;
  Geom g;
  cudaStream_t s = nullptr;
  int prec = P64;    // MG_FP64 or the mixed storage precision of links and clover
  int vt = P64;      // vector type of the cycle (P64 plain, P32 mixed)
  int pv_prec = P64; // storage of the interpolation P (FP16 for both half modes)
  int coarse_reorth = 0;  // second Gram-Schmidt pass in the coarse GMRES (SAPMG_COARSE_REORTH=1)
  int generic_coarse = 0; // use the generic coarse stencil kernel (SAPMG_GENERIC_COARSE=1)
  int coarse_tf32 = 1;    // tensor-core (TF32) coarse stencil in the mixed form (SAPMG_COARSE_TF32=0 disables)
  int sap_shape = 0;      // Schwarz launch shape for an even number of RHS (SAPMG_SAP_SHAPE; -1: one RHS per CTA)
  int dirac_pair = 1;     // paired Dirac kernel for an even number of FP32-arithmetic RHS (SAPMG_DIRAC_PAIR=0: off)
  int graphs = 1;         // coarse solves of the mixed form replayed as CUDA graphs (SAPMG_GRAPHS=0: plain launches)
  int coarse_sap_mrhs = 1; // level-1 Schwarz with all RHS per CTA (SAPMG_COARSE_SAP_MRHS=0: one RHS per CTA)
  int coarse_sap_fp16 = 1; // level-1 Schwarz reads the FP16 operator copy (SAPMG_COARSE_SAP_FP16=0: FP32)
  int setup_fp32 = 1;      // mixed form: set-up part 1 on FP32 vectors (SAPMG_SETUP_FP32=0: FP64 vectors)
  int fp64_on_fp32 = 0;    // mixed form: FP64 residuals in double-float arithmetic (SAPMG_FP64_ON_FP32=1; slower)
  cudaStream_t cap_s = nullptr;            // stream the coarse-solve graphs are captured on
  cudaGraphExec_t cgraph[3][33] = {};      // [level][right-hand sides]: the captured fixed-step coarse GMRES
  int cgraph_kernels[3][33] = {};          // kernels in each graph (for the launch counter)
  unsigned char cgraph_state[3][33] = {};  // 0: not run yet, 1: ran once with plain launches
  int xfer_batch = 16;    // right-hand sides per level-0 transfer launch (autotuned)
  CoarseTune ctune;       // launch shape of the FP16 tensor-core coarse stencil (autotuned)
  // residual history of the last mg_solve: (iteration, right-hand side, relative residual) triples;
  // the cycles add their least-squares estimates times hist_scale[q] at hist_base + step
  std::vector<double> hist, hist_scale;
  int hist_base = 0, hist_r0 = 0;
  int tune_source = 0;    // 0: default launch shapes, 1: chosen by the autotuner, 2: taken from its cache
  int restrict_tf32 = 1;  // tensor-core (TF32) multi-RHS level-0 transfers in the mixed form (SAPMG_RESTRICT_TF32=0 disables)
  int coarse_fp16 = 1;    // FP16-stored operator for the tensor-core coarse stencil (SAPMG_COARSE_FP16=0: FP32)
  int dc_prec = P64; // storage of the coarse operators (FP32 in the mixed form)
  double m0 = 0, csw = 0;
  std::vector<void*> allocs;
  void *U64 = nullptr, *A64 = nullptr;     // blocked FP64 links (boundary sign folded in) and clover
  void *U32 = nullptr, *A32 = nullptr;     // FP32 copies (mixed form)
  void *Us = nullptr, *As = nullptr;       // smoother precision (== U64/A64 or U32/A32 or half)
  int N0 = 0;
  void* V64 = nullptr;                     // locally orthonormal test vectors, FP64 vector-major
  void* Vs64 = nullptr;                    // set-up only: the smoothed vectors before local orthonormalisation
  void* part2_buf = nullptr;               // set-up only (three levels): part-1 vectors kept for set-up part 2
  const std::vector<double2>* load_v0 = nullptr;  // mg_setup_load: the saved level-0 vectors (host)
  const std::vector<double2>* load_w1 = nullptr;  // mg_setup_load: the saved level-1 vectors (host, three levels)
  void* Pv = nullptr;                      // P in cycle storage, block-major
  CoarseLevel c1;
  // three levels: level-1 Schwarz boxes, level-2 aggregates, level-1 vectors, level 2
  Box4 sap1, agg1;
  int N1 = 0;
  void* W64 = nullptr;                     // level-1 locally orthonormal vectors, FP64 [N1][site][n2]
  void* W = nullptr;                       // the same in the cycle's vector type
  CoarseLevel c2;
  // level-1 fixed-step flexible GMRES workspace
  void *f1V = nullptr, *f1Z = nullptr, *f1w = nullptr;
  double2 *f1H = nullptr, *f1tmp = nullptr, *f1beta2 = nullptr, *f1y = nullptr;
  // fine workspace
  void* zero_f = nullptr;                  // a zero fine field (cycle type)
  void* io_a = nullptr;                    // canonical <-> blocked staging (FP64, nrhs_max fields)
  void* io_b = nullptr;
  double2* partial = nullptr;
  int* dev_err = nullptr;                  // [0] raised by kernels whose bounded waits gave up, [1] their bound
  // Krylov workspace
  int m = 0;
  void *V = nullptr, *Z = nullptr, *w = nullptr;       // outer (plain: FP64; mixed: FP32 inner)
  void *x64 = nullptr, *r64 = nullptr, *t64 = nullptr, *b64 = nullptr;   // [nrhs_max] fine fields
  void* e32 = nullptr;                                                    // inner correction (mixed form)
  int ldh = 0;                             // per-RHS stride of the scalar buffers
  double2* hd = nullptr;                   // device scalars [nrhs_max][ldh]
  double2* hh = nullptr;                   // pinned host mirror
  double2* dcg = nullptr;                  // delayed-reorthogonalisation work [8][nrhs_max][ldh] (device)
  double2* dch = nullptr;                  // pinned mirror of its hcol, acol, nrm parts [3][nrhs_max][ldh]
  int outer_dcgs2 = 1;                     // outer Arnoldi with the delayed second pass (SAPMG_DCGS2=0: two passes)
  int outer_half = 0;                      // mixed form: finished outer basis vectors in FP16 (SAPMG_OUTER_FP16=0: FP32)
  void* Vh = nullptr;                      // the FP16 basis [m][nrhs_max][fine field] (V then holds only the newest vector)
  // CG on the normal equations (comparison solver; allocated on first use)
  void* cg = nullptr;                      // its vectors: 48 bytes per complex per system
  double* cg_part = nullptr;               // partial sums: 2 x [nblocks][nrhs_max] (Dirac), [nrhs_max][kCgnMaxG]
  CgnState* cg_st = nullptr;               // per-system scalars (device)
  CgnState* cg_host = nullptr;             // two pinned copies of them
  Prof prof;

  void release(void* ptr) {
    for (auto& q : allocs)
      if (q == ptr) { cudaFree(q); q = nullptr; }
  }
  void* alloc(size_t bytes) {
    void* ptr = nullptr;
    if (bytes == 0) bytes = 16;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    allocs.push_back(ptr);
    // SAPMG_POISON=1: fill every workspace with NaN bytes (0xff), so that a read
    // of memory no kernel has written shows up in the results (debugging aid)
    static const bool poison = std::getenv("SAPMG_POISON") && std::atoi(std::getenv("SAPMG_POISON"));
    if (poison) cudaMemset(ptr, 0xff, bytes);
    return ptr;
  }
  ~mg_ctx() {
    for (auto& row : cgraph)
      for (auto& x : row)
        if (x) cudaGraphExecDestroy(x);
    if (cap_s) cudaStreamDestroy(cap_s);
    for (void* q : allocs)
      if (q) cudaFree(q);
    if (hh) cudaFreeHost(hh);
    if (dch) cudaFreeHost(dch);
    if (cg_host) cudaFreeHost(cg_host);
  }
  size_t fine_n() const { return (size_t)g.V * 12; }
};

namespace sapmg {

// ------------------------------------------------------------ helpers
// Algorithmic bytes of the level-0 kernels (each operand read once, each
// result written once): links (4 x 9 complex) and clover (2 x 36 real) per
// site in storage precision, spinors (12 complex per site and system).
static double fields_bytes(int store) { return 72.0 * complex_bytes(store); }
static double vec_bytes(int prec) { return prec == P64 ? 16.0 : 8.0; }

static int smoother_sweeps(mg_ctx* c, const void* b, void* z, int n_sweeps, int nrhs) {
  for (int it = 0; it < n_sweeps; ++it)
    for (int col = 0; col < 2; ++col) {
      ProfScope ps(c->prof, FAM_SAP, c->s);
      // one colour: half the sites; b and z read, z written, z read across the block faces
      count_bytes(0.5 * c->g.V * (nrhs * 4 * 12 * vec_bytes(c->prec) + fields_bytes(c->prec)));
      TRY(launch_sap_colour(c->prec, c->g, z, b, c->Us, c->As, col, c->p.n_mr, nrhs, c->s, c->sap_shape, c->dev_err));
    }
  return MG_OK;
}

static int fine_dirac(mg_ctx* c, int prec, void* out, const void* in, int nrhs) {
  const bool f64 = prec == P64 || prec == P64E;
  const void* U = f64 ? c->U64 : (prec == P32 ? c->U32 : c->Us);
  const void* A = f64 ? c->A64 : (prec == P32 ? c->A32 : c->As);
  if (!U || !A) return fail(MG_ERR_STATE, "requested precision not set up in this context");
  ProfScope ps(c->prof, FAM_DIRAC, c->s);
  const int bp = f64 ? P64 : prec;
  count_bytes((double)c->g.V * (nrhs * 2 * 12 * vec_bytes(bp) + fields_bytes(bp)));
  if (c->dirac_pair && !f64 && nrhs >= 2 && nrhs % 2 == 0)
    return launch_dirac_pair(prec, c->g, out, in, U, A, nrhs, c->s);
  return launch_dirac(prec, c->g, out, in, U, A, nrhs, c->s);
}

static int dot_to(mg_ctx* c, int type, const BVec& b, const void* x, const void* y, double2* out, int ldo) {
  const void* v[1] = {x};
  return blas_multidot(type, b, v, 1, y, out, ldo, 0, nullptr, c->partial, c->s);
}

// D_c x on a coarse level: the tensor-core kernel (FP16 or FP32 operator) in
// the mixed form, the bulk-copy kernel for an FP32 operator, else the generic
// one.  xh: x holds FP16 basis vectors (scaled by kBasisScale); needs the FP16
// operator copy.
static int coarse_apply(mg_ctx* c, CoarseLevel& L, const void* x, void* out, int R, bool xh = false) {
  ProfScope ps(c->prof, FAM_COARSE, c->s);
  const bool mma = L.store == P32 && c->vt == P32 && c->coarse_tf32 && L.cg.n2 % 8 == 0 && L.cg.n2 <= 64 &&
                   !c->generic_coarse;
  const int store = (mma && L.Mh) ? P16 : L.store;
  if (xh && store != P16) return fail(MG_ERR_STATE, "FP16 coarse vectors need the FP16 operator");
  count_bytes((double)L.cg.nsites * (9.0 * L.cg.n2 * L.cg.n2 * complex_bytes(store) +
                                     R * L.cg.n2 * (complex_bytes(c->vt) + (xh ? 4.0 : complex_bytes(c->vt)))));
  if (mma)
    return launch_coarse_apply_mma(L.cg, store, store == P16 ? L.Mh : L.M, x, out, R, c->dev_err, xh, c->s,
                                   store == P16 ? c->ctune : CoarseTune());
  if (L.store == P32 && c->vt == P32 && L.cg.n2 % 2 == 0 && L.cg.n2 <= 64 && !c->generic_coarse)
    return launch_coarse_apply_tma(L.cg, L.M, x, out, R, c->dev_err, c->s);
  return launch_coarse_apply(L.store, L.cg, L.M, x, out, R, c->s);
}

static int check_device_error(mg_ctx* c) {
  int h = 0;
  SAPMG_CUDA_TRY(cudaMemcpyAsync(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  if (h) {
    SAPMG_CUDA_TRY(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->s));
    return fail(MG_ERR_TIMEOUT, "a bounded device wait gave up");
  }
#ifdef MG_DEBUG
  std::string msg;
  const long long n = dbg::collect(&msg);
  if (n < 0) return fail(MG_ERR_CUDA, "could not read the device-side index checks");
  if (n > 0) return fail(MG_ERR_BOUNDS, msg);
#endif
  return MG_OK;
}

static Scal32 scal_all(double re, int R) {
  Scal32 s;
  for (int r = 0; r < 32; ++r) s.v[r] = make_double2(r < R ? re : 0.0, 0.0);
  return s;
}

// The level-0 transfers of R right-hand sides in launches of at most
// xfer_batch of them (mixed form; each launch reads P once for its batch).
// A batch of one would take the one-vector kernel, which rounds differently,
// so a last batch of one joins the previous one.
static int transfer0(mg_ctx* c, bool restrict_, const void* in, void* out, int R) {
  int bsz = (c->vt == P32 && c->xfer_batch > 0) ? std::min(c->xfer_batch, R) : R;
  const size_t fb = c->fine_n() * complex_bytes(c->vt), cb = c->c1.n() * complex_bytes(c->vt);
  for (int r0 = 0; r0 < R;) {
    int nr = std::min(bsz, R - r0);
    if (R - r0 - nr == 1) nr += 1;
    const char* src = (const char*)in + (size_t)r0 * (restrict_ ? fb : cb);
    char* dst = (char*)out + (size_t)r0 * (restrict_ ? cb : fb);
    TRY(launch_transfer0(restrict_, c->pv_prec, c->g, src, dst, c->Pv, c->N0, nr, c->restrict_tf32, c->s));
    r0 += nr;
  }
  return MG_OK;
}

// Fixed-step GMRES from zero on a coarse level for R right-hand sides at once
// (Sec. 4: 12 steps on the coarse grid): Arnoldi with classical Gram-Schmidt
// (a second pass when coarse_reorth is set), all scalars on the device, one
// operator application per step serving every right-hand side.
static int coarse_gmres(mg_ctx* c, CoarseLevel& L, int k, int R) {
  const size_t n = L.n();
  const int vt = c->vt;
  const size_t eb = complex_bytes(vt);
  const BVec bv = bvec(n, R, n);
  auto Vj = [&](int j) { return (void*)((char*)L.V + (size_t)j * R * n * eb); };
  CBLAS(dot_to(c, vt, bv, L.b, L.b, L.beta2, 1));
  CBLAS(blas_normalize(vt, bv, L.b, Vj(0), L.beta2, 1, nullptr, 0, c->s));
  std::vector<const void*> vl;
  for (int j = 0; j < k; ++j) {
    TRY(coarse_apply(c, L, Vj(j), L.w, R));
    vl.push_back(Vj(j));
    double2* hcol = L.H + (size_t)j * 33;
    CBLAS(blas_multidot(vt, bv, vl.data(), j + 1, L.w, hcol, 33 * 33, 0, nullptr, c->partial, c->s));
    if (c->coarse_reorth) {
      CBLAS(blas_multiaxpy(vt, bv, L.w, vl.data(), j + 1, hcol, 33 * 33, -1.0, c->s));
      CBLAS(blas_multidot(vt, bv, vl.data(), j + 1, L.w, hcol, 33 * 33, 1, L.tmp, c->partial, c->s));
      CBLAS(blas_multiaxpy_norm(vt, bv, L.w, vl.data(), j + 1, L.tmp, 33 * 33, -1.0, L.tmp + 40, 33 * 33, c->partial,
                              c->s));
    } else {
      CBLAS(blas_multiaxpy_norm(vt, bv, L.w, vl.data(), j + 1, hcol, 33 * 33, -1.0, L.tmp + 40, 33 * 33, c->partial,
                              c->s));
    }
    CBLAS(blas_normalize(vt, bv, L.w, Vj(j + 1), L.tmp + 40, 33 * 33, hcol + j + 1, 33 * 33, c->s));
  }
  CBLAS(blas_hessenberg_solve(L.H, 33, 33 * 33, k, L.beta2, L.y, 33, R, c->s));
  SAPMG_CUDA_TRY(cudaMemsetAsync(L.x, 0, (size_t)R * n * eb, c->s));
  CBLAS(blas_multiaxpy(vt, bv, L.x, vl.data(), k, L.y, 33, 1.0, c->s));
  return MG_OK;
}

// The same fixed-step GMRES with the Krylov basis kept in FP16 (scaled by
// kBasisScale; the mixed form's two-level coarse solve when the FP16 operator
// copy exists): half the basis traffic of the orthogonalisation, FP32 w, x.
static int coarse_gmres_h(mg_ctx* c, CoarseLevel& L, int k, int R) {
  const size_t n = L.n();
  const BVec bv = bvec(n, R, n);
  auto Vj = [&](int j) { return (void*)((char*)L.Vh + (size_t)j * R * n * 4); };
  CBLAS(dot_to(c, P32, bv, L.b, L.b, L.beta2, 1));
  CBLAS(blas_normalize_h(bv, L.b, Vj(0), L.beta2, 1, nullptr, 0, c->s));
  std::vector<const void*> vl;
  for (int j = 0; j < k; ++j) {
    TRY(coarse_apply(c, L, Vj(j), L.w, R, true));
    vl.push_back(Vj(j));
    double2* hcol = L.H + (size_t)j * 33;
    CBLAS(blas_multidot_h(bv, vl.data(), j + 1, L.w, hcol, 33 * 33, c->partial, c->s));
    CBLAS(blas_multiaxpy_h(bv, L.w, vl.data(), j + 1, hcol, 33 * 33, -1.0, L.tmp + 40, 33 * 33, c->partial, c->s));
    CBLAS(blas_normalize_h(bv, L.w, Vj(j + 1), L.tmp + 40, 33 * 33, hcol + j + 1, 33 * 33, c->s));
  }
  CBLAS(blas_hessenberg_solve(L.H, 33, 33 * 33, k, L.beta2, L.y, 33, R, c->s));
  SAPMG_CUDA_TRY(cudaMemsetAsync(L.x, 0, (size_t)R * n * 8, c->s));
  CBLAS(blas_multiaxpy_h(bv, L.x, vl.data(), k, L.y, 33, 1.0, nullptr, 0, c->partial, c->s));
  return MG_OK;
}

static int cycle1(mg_ctx* c, const void* v, void* z, int R);

// Fixed-step flexible GMRES from zero on level 1 of a three-level hierarchy,
// right-preconditioned by the level-1 cycle (the two-level method applied to
// the coarse equation, Sec. 3): b = c1.b -> x = c1.x for R systems.
static int fgmres_fixed1(mg_ctx* c, int k, int R) {
  CoarseLevel& L = c->c1;
  const size_t n = L.n();
  const int vt = c->vt;
  const size_t eb = complex_bytes(vt);
  const BVec bv = bvec(n, R, n);
  auto Vj = [&](int j) { return (void*)((char*)c->f1V + (size_t)j * R * n * eb); };
  auto Zj = [&](int j) { return (void*)((char*)c->f1Z + (size_t)j * R * n * eb); };
  CBLAS(dot_to(c, vt, bv, L.b, L.b, c->f1beta2, 1));
  CBLAS(blas_normalize(vt, bv, L.b, Vj(0), c->f1beta2, 1, nullptr, 0, c->s));
  std::vector<const void*> vl, zl;
  for (int j = 0; j < k; ++j) {
    TRY(cycle1(c, Vj(j), Zj(j), R));
    TRY(coarse_apply(c, L, Zj(j), c->f1w, R));
    vl.push_back(Vj(j));
    zl.push_back(Zj(j));
    double2* hcol = c->f1H + (size_t)j * 33;
    CBLAS(blas_multidot(vt, bv, vl.data(), j + 1, c->f1w, hcol, 33 * 33, 0, nullptr, c->partial, c->s));
    if (c->coarse_reorth) {
      CBLAS(blas_multiaxpy(vt, bv, c->f1w, vl.data(), j + 1, hcol, 33 * 33, -1.0, c->s));
      CBLAS(blas_multidot(vt, bv, vl.data(), j + 1, c->f1w, hcol, 33 * 33, 1, c->f1tmp, c->partial, c->s));
      CBLAS(blas_multiaxpy_norm(vt, bv, c->f1w, vl.data(), j + 1, c->f1tmp, 33 * 33, -1.0, c->f1tmp + 40, 33 * 33,
                              c->partial, c->s));
    } else {
      CBLAS(blas_multiaxpy_norm(vt, bv, c->f1w, vl.data(), j + 1, hcol, 33 * 33, -1.0, c->f1tmp + 40, 33 * 33,
                              c->partial, c->s));
    }
    CBLAS(blas_normalize(vt, bv, c->f1w, Vj(j + 1), c->f1tmp + 40, 33 * 33, hcol + j + 1, 33 * 33, c->s));
  }
  CBLAS(blas_hessenberg_solve(c->f1H, 33, 33 * 33, k, c->f1beta2, c->f1y, 33, R, c->s));
  SAPMG_CUDA_TRY(cudaMemsetAsync(L.x, 0, (size_t)R * n * eb, c->s));
  CBLAS(blas_multiaxpy(vt, bv, L.x, zl.data(), k, c->f1y, 33, 1.0, c->s));
  return MG_OK;
}

// The FP16-basis coarse GMRES as a CUDA graph: its ~4k+3 launches use fixed
// buffers and no host synchronisation, so after one run with plain launches
// (which also sets every kernel attribute) the sequence is captured once per
// (level, R) on a stream of the context's own and replayed on the context's
// stream, saving the launch gaps between the short dependent kernels.  The
// replay computes what the plain launches compute, bit for bit.  Plain
// launches while the coarse families are being profiled (the profile times
// every launch with events on the host's side).
static int coarse_gmres_h_graph(mg_ctx* c, int level, CoarseLevel& L, int k, int R) {
  const bool prof = c->prof.on && ((((c->prof.mask >> FAM_COARSE) | (c->prof.mask >> FAM_CBLAS)) & 1u) != 0);
  if (!c->graphs || prof || R < 1 || R > 32) return coarse_gmres_h(c, L, k, R);
  if (c->cgraph_state[level][R] == 0) {
    c->cgraph_state[level][R] = 1;
    return coarse_gmres_h(c, L, k, R);
  }
  if (!c->cgraph[level][R]) {
    if (!c->cap_s) SAPMG_CUDA_TRY(cudaStreamCreateWithFlags(&c->cap_s, cudaStreamNonBlocking));
    const cudaStream_t s0 = c->s;
    const long long l0 = mg_launch_count();
    SAPMG_CUDA_TRY(cudaStreamBeginCapture(c->cap_s, cudaStreamCaptureModeThreadLocal));
    c->s = c->cap_s;
    const int rc = coarse_gmres_h(c, L, k, R);
    c->s = s0;
    cudaGraph_t gr = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->cap_s, &gr);
    const long long nk = mg_launch_count() - l0;
    count_launches(-(int)nk);                           // captured, not launched
    if (rc < 0 || e != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      if (rc < 0) return rc;
      return fail(MG_ERR_CUDA, std::string("coarse-solve graph capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t x = nullptr;
    const cudaError_t e2 = cudaGraphInstantiate(&x, gr, 0);
    cudaGraphDestroy(gr);
    if (e2 != cudaSuccess) return fail(MG_ERR_CUDA, std::string("coarse-solve graph: ") + cudaGetErrorString(e2));
    c->cgraph[level][R] = x;
    c->cgraph_kernels[level][R] = (int)nk;
  }
  SAPMG_CUDA_TRY(cudaGraphLaunch(c->cgraph[level][R], c->s));
  count_launches(c->cgraph_kernels[level][R]);
  return MG_OK;
}

static int coarse_solve(mg_ctx* c, int level, int R) {
  if (level == 1 && c->p.n_levels == 2 && c->c1.Vh) return coarse_gmres_h_graph(c, 1, c->c1, c->p.coarse_iters, R);
  if (level == 1 && c->p.n_levels == 2) return coarse_gmres(c, c->c1, c->p.coarse_iters, R);
  if (level == 1 && c->p.n_levels == 3) return fgmres_fixed1(c, c->p.inner_iters, R);
  if (level == 2 && c->p.n_levels == 3 && c->c2.Vh) return coarse_gmres_h_graph(c, 2, c->c2, c->p.coarse_iters, R);
  if (level == 2 && c->p.n_levels == 3) return coarse_gmres(c, c->c2, c->p.coarse_iters, R);
  return fail(MG_ERR_ARG, "coarse level out of range");
}

// Schwarz sweeps on level 1 (boxes of coarse sites, red-black as on the fine level).
// Mixed form: all right-hand sides in one CTA per box (each operator entry
// loaded once for all of them), unless SAPMG_COARSE_SAP_MRHS=0, reading the
// FP16 copy of the level-1 operator that the level-1 Krylov operator already
// uses (the pass reads the box's operator once per MR step: half the bytes),
// unless SAPMG_COARSE_SAP_FP16=0.
static int smoother_sweeps1(mg_ctx* c, const void* b, void* z, int n_sweeps, int R) {
  const bool mrhs = c->coarse_sap_mrhs && c->c1.store == P32 && R >= 2 && R <= 12;
  const bool m16 = c->coarse_sap_fp16 && c->c1.store == P32 && c->c1.Mh != nullptr;
  const void* M = m16 ? c->c1.Mh : c->c1.M;
  for (int it = 0; it < n_sweeps; ++it)
    for (int col = 0; col < 2; ++col) {
      ProfScope ps(c->prof, FAM_SAP1, c->s);
      count_bytes((double)c->c1.cg.nsites / 2 * 9.0 * c->c1.cg.n2 * c->c1.cg.n2 *
                  complex_bytes(m16 ? P16 : c->c1.store) * (mrhs ? 1.0 : R) * (c->p.n_mr + 1));
      if (mrhs) TRY(launch_coarse_sap_mrhs(c->c1.cg, c->sap1, M, m16, z, b, col, c->p.n_mr, R, c->s));
      else TRY(launch_coarse_sap(c->c1.store == P64 ? P64 : P32, c->c1.cg, c->sap1, M, z, b, col, c->p.n_mr, R, c->s,
                                 m16));
    }
  return MG_OK;
}

// The level-1 cycle z = M1 v: restrict to level 2, fixed-step GMRES there,
// interpolate, nu_post Schwarz sweeps on level 1.
static int cycle1(mg_ctx* c, const void* v, void* z, int R) {
  {
    ProfScope ps(c->prof, FAM_RESTRICT, c->s);
    TRY(launch_transfer1(true, c->vt, c->c1.cg, c->agg1, v, c->c2.b, c->W, c->N1, R, c->s));
  }
  TRY(coarse_solve(c, 2, R));
  {
    ProfScope ps(c->prof, FAM_PROLONG, c->s);
    TRY(launch_transfer1(false, c->vt, c->c1.cg, c->agg1, c->c2.x, z, c->W, c->N1, R, c->s));
  }
  return smoother_sweeps1(c, v, z, c->p.nu_post, R);
}

// The multilevel cycle z = M v on the fine level for R right-hand sides (cycle vector type).
static int cycle(mg_ctx* c, const void* v, void* z, int R) {
  const size_t n = c->fine_n();
  if (c->p.n_levels == 1) {
    SAPMG_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)R * n * complex_bytes(c->vt), c->s));
    return smoother_sweeps(c, v, z, c->p.nu_post, R);
  }
  // P (N vectors of 12 complex per site), the fine and the coarse vectors
  const double tbytes = (double)c->g.V * (c->N0 * 12.0 * complex_bytes(c->pv_prec) + R * 12.0 * complex_bytes(c->vt)) +
                        (double)c->g.nblocks * 2 * c->N0 * R * complex_bytes(c->vt);
  {
    ProfScope ps(c->prof, FAM_RESTRICT, c->s);
    count_bytes(tbytes);
    TRY(transfer0(c, true, v, c->c1.b, R));
  }
  TRY(coarse_solve(c, 1, R));
  {
    ProfScope ps(c->prof, FAM_PROLONG, c->s);
    count_bytes(tbytes);
    TRY(transfer0(c, false, c->c1.x, z, R));
  }
  return smoother_sweeps(c, v, z, c->p.nu_post, R);
}

// One entry of the residual history: the least-squares residual estimate of a
// cycle's system q scaled to ||b - D x|| / ||b|| of the solve's system.
static void record_history(mg_ctx* c, int q, int iteration, double est) {
  if (q >= (int)c->hist_scale.size()) return;
  c->hist.push_back((double)iteration);
  c->hist.push_back((double)(c->hist_r0 + q));
  c->hist.push_back(est * c->hist_scale[q]);
}

// Least squares min || g0 e1 - H y || for the (n+1) x n upper Hessenberg H
// (column-major, leading dimension ld) by Givens rotations applied from
// scratch; returns the residual norm and, if y != nullptr, the solution.
static double hessenberg_lsq(const std::complex<double>* H, int ld, int n, double g0, std::complex<double>* y) {
  typedef std::complex<double> cd;
  std::vector<cd> h(H, H + (size_t)ld * n), g(n + 1, 0.0);
  g[0] = g0;
  for (int j = 0; j < n; ++j) {
    const cd u = h[j + (size_t)j * ld], v = h[j + 1 + (size_t)j * ld];
    const double na = std::abs(u), nb = std::abs(v), den = std::sqrt(na * na + nb * nb);
    double cs;
    cd sn;
    if (den == 0.0) { cs = 1; sn = 0; }
    else if (na == 0.0) { cs = 0; sn = 1; }
    else { cs = na / den; sn = (u / na) * std::conj(v) / den; }
    for (int k = j; k < n; ++k) {
      cd& p = h[j + (size_t)k * ld];
      cd& q = h[j + 1 + (size_t)k * ld];
      const cd t = cs * p + sn * q;
      q = -std::conj(sn) * p + cs * q;
      p = t;
    }
    g[j + 1] = -std::conj(sn) * g[j];
    g[j] = cs * g[j];
  }
  if (y) {
    for (int i = n - 1; i >= 0; --i) {
      cd acc = g[i];
      for (int k = i + 1; k < n; ++k) acc -= h[i + (size_t)k * ld] * y[k];
      const cd d = h[i + (size_t)i * ld];
      y[i] = std::abs(d) > 0 ? acc / d : 0.0;
    }
  }
  return std::abs(g[n]);
}

// The same cycle as fgmres_cycle with the delayed second Gram-Schmidt pass
// (blas_dcgs2_step): step j reorthogonalises v_j and orthogonalises w = A z_j
// in one dot pass and one update pass over the basis.  The second pass of v_j
// rewrites column j-1 of the Hessenberg matrix (A z_{j-1} was expanded in the
// once-orthogonalised v_j); the least-squares problem is re-solved from the
// stored columns at every step.
static int fgmres_cycle_dcgs2(mg_ctx* c, int ft, int aprec, int R, const void* r, const std::vector<double>& rnorm,
                              void* x, const std::vector<double>& abs_tol, int iters_left, std::vector<int>& done,
                              std::vector<double>& est) {
  typedef std::complex<double> cd;
  const size_t n = c->fine_n();
  const size_t eb = complex_bytes(ft);
  const int m = std::min(c->m, std::max(1, iters_left));
  const int ld = c->ldh;
  const int lh = m + 1;
  const BVec bv = bvec(n, R, n);
  auto Vj = [&](int j) { return (void*)((char*)c->V + (size_t)j * R * n * eb); };
  auto Zj = [&](int j) { return (void*)((char*)c->Z + (size_t)j * R * n * eb); };
  std::vector<cd> H((size_t)R * lh * m, 0.0);
  auto Hq = [&](int q, int i, int j) -> cd& { return H[(size_t)q * lh * m + i + (size_t)j * lh]; };
  std::vector<char> active(R, 0);
  done.assign(R, 0);
  est.assign(R, 0.0);
  Scal32 a = scal_all(0, R), zero = scal_all(0, R);
  int n_active = 0;
  for (int q = 0; q < R; ++q) {
    est[q] = rnorm[q];
    if (rnorm[q] > 0 && rnorm[q] > abs_tol[q]) { active[q] = 1; ++n_active; a.v[q].x = 1.0 / rnorm[q]; }
  }
  if (n_active == 0) return MG_OK;
  // With an FP16 basis the finished vectors live in Vh and the newest,
  // once-orthogonalised one in FP32 in one of two buffers (V, w) that swap
  // roles every step: step j's new w (not normalised: the second pass
  // normalises it, and the cycle is homogeneous of degree one) is step j+1's u.
  const bool hb = c->outer_half != 0;
  void* ucur = hb ? c->V : Vj(0);
  void* wcur = c->w;
  auto Vhj = [&](int j) { return (void*)((char*)c->Vh + (size_t)j * R * n * 4); };
  BLAS(blas_axpby2(ft, a, r, n, ft, zero, ucur, n, n, R, c->s));
  const size_t rl = (size_t)R * ld;
  DcgsWork ws;
  ws.A = c->dcg;
  ws.B = c->dcg + rl;
  ws.X = c->dcg + 2 * rl;
  ws.c1 = c->dcg + 3 * rl;
  ws.c2 = c->dcg + 4 * rl;
  ws.hcol = c->dcg + 5 * rl;
  ws.acol = c->dcg + 6 * rl;
  ws.nrm = c->dcg + 7 * rl;
  ws.ld = ld;
  ws.partial = c->partial;
  std::vector<const void*> vl;   // finished basis vectors v_0 .. v_{j-1}
  for (int j = 0; j < m; ++j) {
    if (!hb) ucur = Vj(j);
    TRY(cycle(c, ucur, Zj(j), R));
    TRY(fine_dirac(c, aprec, wcur, Zj(j), R));
    if (hb) BLAS(blas_dcgs2_step_h(bv, vl.data(), j, ucur, wcur, Vhj(j), ws, c->s));
    else BLAS(blas_dcgs2_step(ft, bv, vl.data(), j, ucur, wcur, ws, c->s));
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->dch, ws.hcol, sizeof(double2) * 3 * rl, cudaMemcpyDeviceToHost, c->s));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
    n_active = 0;
    for (int q = 0; q < R; ++q) {
      a.v[q] = make_double2(0, 0);
      if (!active[q]) continue;
      const double2* hc = c->dch + (size_t)q * ld;
      const double2* ac = c->dch + rl + (size_t)q * ld;
      const double2* nr = c->dch + 2 * rl + (size_t)q * ld;
      if (j > 0) {
        // u was hs * (normalised u) (the normalised form) or the unnormalised
        // new w itself (FP16 basis), whose coefficients a_i, beta carry the scale
        const cd hs = hb ? cd(1.0, 0.0) : Hq(q, j, j - 1);
        for (int i = 0; i < j; ++i) Hq(q, i, j - 1) += hs * cd(ac[i].x, ac[i].y);
        Hq(q, j, j - 1) = hs * ac[j].x;
      }
      for (int i = 0; i <= j; ++i) Hq(q, i, j) = cd(hc[i].x, hc[i].y);
      const double hn = std::sqrt(std::max(nr[1].x, 0.0));
      Hq(q, j + 1, j) = hn;
      done[q] = j + 1;
      est[q] = hessenberg_lsq(&Hq(q, 0, 0), lh, j + 1, rnorm[q], nullptr);
      record_history(c, q, c->hist_base + j + 1, est[q]);
      if (est[q] <= abs_tol[q] || hn == 0.0 || ac[j].x == 0.0) { active[q] = 0; continue; }
      a.v[q].x = 1.0 / hn;
      ++n_active;
    }
    if (n_active == 0 || j + 1 == m) break;
    if (hb) {
      std::swap(ucur, wcur);
    } else {
      BLAS(blas_axpby2(ft, a, wcur, n, ft, zero, Vj(j + 1), n, n, R, c->s));
    }
    vl.push_back(hb ? Vhj(j) : Vj(j));
  }
  // least squares per system and x += Z y
  int jmax = 0;
  for (int q = 0; q < R; ++q) {
    jmax = std::max(jmax, done[q]);
    std::vector<cd> y(std::max(done[q], 1));
    if (done[q] > 0) hessenberg_lsq(&Hq(q, 0, 0), lh, done[q], rnorm[q], y.data());
    double2* hq = c->hh + (size_t)q * ld;
    for (int i = 0; i < ld; ++i) hq[i] = i < done[q] ? make_double2(y[i].real(), y[i].imag()) : make_double2(0, 0);
  }
  SAPMG_CUDA_TRY(cudaMemcpyAsync(c->hd, c->hh, sizeof(double2) * R * ld, cudaMemcpyHostToDevice, c->s));
  std::vector<const void*> zl;
  for (int i = 0; i < jmax; ++i) zl.push_back(Zj(i));
  BLAS(blas_multiaxpy(ft, bv, x, zl.data(), jmax, c->hd, ld, 1.0, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));   // hh is reused by the next cycle
  return MG_OK;
}

// One cycle of flexible GMRES(m) for R systems in lockstep, A e = r from e = x
// (x updated in place, x += Z y).  r: current residuals (type ft); rnorm[r]
// their norms (0 = system inactive).  System r stops when its least-squares
// residual estimate <= abs_tol[r]; the cycle ends when every system has stopped,
// after m steps or at iters_left.  Orthogonalisation: classical Gram-Schmidt
// with a second pass when a norm drops below 1/sqrt(2) of its value (the
// Daniel-Gragg-Kaufman-Stewart criterion).  done[r] = steps taken by system r.
static int fgmres_cycle(mg_ctx* c, int ft, int aprec, int R, const void* r, const std::vector<double>& rnorm,
                        void* x, const std::vector<double>& abs_tol, int iters_left, std::vector<int>& done,
                        std::vector<double>& est) {
  if (c->outer_dcgs2) return fgmres_cycle_dcgs2(c, ft, aprec, R, r, rnorm, x, abs_tol, iters_left, done, est);
  typedef std::complex<double> cd;
  const size_t n = c->fine_n();
  const size_t eb = complex_bytes(ft);
  const int m = std::min(c->m, std::max(1, iters_left));
  const int ld = c->ldh;
  const BVec bv = bvec(n, R, n);
  auto Vj = [&](int j) { return (void*)((char*)c->V + (size_t)j * R * n * eb); };
  auto Zj = [&](int j) { return (void*)((char*)c->Z + (size_t)j * R * n * eb); };
  std::vector<cd> H((size_t)R * (m + 1) * m, 0.0), g((size_t)R * (m + 1), 0.0), sn((size_t)R * m, 0.0);
  std::vector<double> cs((size_t)R * m, 0.0), hn(R, 0.0);
  std::vector<char> active(R, 0);
  done.assign(R, 0);
  est.assign(R, 0.0);
  Scal32 a = scal_all(0, R), zero = scal_all(0, R);
  int n_active = 0;
  for (int q = 0; q < R; ++q) {
    est[q] = rnorm[q];
    if (rnorm[q] > 0 && rnorm[q] > abs_tol[q]) { active[q] = 1; ++n_active; a.v[q].x = 1.0 / rnorm[q]; }
    g[(size_t)q * (m + 1)] = rnorm[q];
  }
  if (n_active == 0) return MG_OK;
  BLAS(blas_axpby2(ft, a, r, n, ft, zero, Vj(0), n, n, R, c->s));
  auto Hq = [&](int q, int i, int j) -> cd& { return H[(size_t)q * (m + 1) * m + i + (size_t)j * (m + 1)]; };
  std::vector<const void*> vl;
  for (int j = 0; j < m; ++j) {
    TRY(cycle(c, Vj(j), Zj(j), R));
    TRY(fine_dirac(c, aprec, c->w, Zj(j), R));
    vl.push_back(Vj(j));
    vl.push_back(c->w);                  // h = V^dagger w and ||w||^2 in one pass
    BLAS(blas_multidot(ft, bv, vl.data(), j + 2, c->w, c->hd, ld, 0, nullptr, c->partial, c->s));
    vl.pop_back();
    BLAS(blas_multiaxpy_norm(ft, bv, c->w, vl.data(), j + 1, c->hd, ld, -1.0, c->hd + j + 2, ld, c->partial, c->s));
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->hh, c->hd, sizeof(double2) * R * ld, cudaMemcpyDeviceToHost, c->s));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
    bool again = false;
    for (int q = 0; q < R; ++q) {
      const double2* h = c->hh + (size_t)q * ld;
      for (int i = 0; i <= j; ++i) Hq(q, i, j) = cd(h[i].x, h[i].y);
      hn[q] = h[j + 2].x;
      if (active[q] && h[j + 2].x < 0.5 * h[j + 1].x) again = true;
    }
    if (again) {
      BLAS(blas_multidot(ft, bv, vl.data(), j + 1, c->w, c->hd, ld, 0, nullptr, c->partial, c->s));
      BLAS(blas_multiaxpy_norm(ft, bv, c->w, vl.data(), j + 1, c->hd, ld, -1.0, c->hd + j + 2, ld, c->partial, c->s));
      SAPMG_CUDA_TRY(cudaMemcpyAsync(c->hh, c->hd, sizeof(double2) * R * ld, cudaMemcpyDeviceToHost, c->s));
      SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
      for (int q = 0; q < R; ++q) {
        const double2* h = c->hh + (size_t)q * ld;
        for (int i = 0; i <= j; ++i) Hq(q, i, j) += cd(h[i].x, h[i].y);
        hn[q] = h[j + 2].x;
      }
    }
    n_active = 0;
    for (int q = 0; q < R; ++q) {
      a.v[q] = make_double2(0, 0);
      if (!active[q]) continue;
      const double hq = std::sqrt(std::max(hn[q], 0.0));
      Hq(q, j + 1, j) = hq;
      double* csq = &cs[(size_t)q * m];
      cd* snq = &sn[(size_t)q * m];
      cd* gq = &g[(size_t)q * (m + 1)];
      for (int i = 0; i < j; ++i) {
        cd& u = Hq(q, i, j);
        cd& v = Hq(q, i + 1, j);
        const cd t = csq[i] * u + snq[i] * v;
        v = -std::conj(snq[i]) * u + csq[i] * v;
        u = t;
      }
      cd& u = Hq(q, j, j);
      cd& v = Hq(q, j + 1, j);
      const double na = std::abs(u), nb = std::abs(v), den = std::sqrt(na * na + nb * nb);
      if (den == 0.0) { csq[j] = 1; snq[j] = 0; }
      else if (na == 0.0) { csq[j] = 0; snq[j] = 1; }
      else { csq[j] = na / den; snq[j] = (u / na) * std::conj(v) / den; }
      u = csq[j] * u + snq[j] * v;
      v = 0.0;
      gq[j + 1] = -std::conj(snq[j]) * gq[j];
      gq[j] = csq[j] * gq[j];
      done[q] = j + 1;
      est[q] = std::abs(gq[j + 1]);
      record_history(c, q, c->hist_base + j + 1, est[q]);
      if (est[q] <= abs_tol[q] || hq == 0.0) { active[q] = 0; continue; }
      a.v[q].x = 1.0 / hq;
      ++n_active;
    }
    if (n_active == 0 || j + 1 == m) break;
    BLAS(blas_axpby2(ft, a, c->w, n, ft, zero, Vj(j + 1), n, n, R, c->s));
  }
  // back substitution per system and x += Z y
  int jmax = 0;
  for (int q = 0; q < R; ++q) {
    jmax = std::max(jmax, done[q]);
    std::vector<cd> y(done[q]);
    const cd* gq = &g[(size_t)q * (m + 1)];
    for (int i = done[q] - 1; i >= 0; --i) {
      cd acc = gq[i];
      for (int k = i + 1; k < done[q]; ++k) acc -= Hq(q, i, k) * y[k];
      const cd d = Hq(q, i, i);
      y[i] = std::abs(d) > 0 ? acc / d : 0.0;
    }
    double2* hq = c->hh + (size_t)q * ld;
    for (int i = 0; i < ld; ++i) hq[i] = i < done[q] ? make_double2(y[i].real(), y[i].imag()) : make_double2(0, 0);
  }
  SAPMG_CUDA_TRY(cudaMemcpyAsync(c->hd, c->hh, sizeof(double2) * R * ld, cudaMemcpyHostToDevice, c->s));
  std::vector<const void*> zl;
  for (int i = 0; i < jmax; ++i) zl.push_back(Zj(i));
  BLAS(blas_multiaxpy(ft, bv, x, zl.data(), jmax, c->hd, ld, 1.0, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));   // hh is reused by the next cycle
  return MG_OK;
}

static int host_norms(mg_ctx* c, int type, const void* x, int R, std::vector<double>& out) {
  const size_t n = c->fine_n();
  TRY(dot_to(c, type, bvec(n, R, n), x, x, c->hd, c->ldh));
  SAPMG_CUDA_TRY(cudaMemcpyAsync(c->hh, c->hd, sizeof(double2) * R * c->ldh, cudaMemcpyDeviceToHost, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  out.resize(R);
  for (int q = 0; q < R; ++q) out[q] = std::sqrt(std::max(c->hh[(size_t)q * c->ldh].x, 0.0));
  return MG_OK;
}

// Solve R right-hand sides together: b64 (batched blocked FP64) -> x64.
// Restart cycles of the mixed form's FP32 flexible GMRES per FP64 correction.
constexpr int kInnerCycles = 12;

static int solve_batch(mg_ctx* c, int R, int& iters, int& restarts, double& relres) {
  const size_t n = c->fine_n();
  std::vector<double> bn, rn, tol(R), ones(R, 1.0), inner(R), est;
  std::vector<int> done;
  BLAS(host_norms(c, P64, c->b64, R, bn));
  SAPMG_CUDA_TRY(cudaMemsetAsync(c->x64, 0, (size_t)R * n * 16, c->s));
  SAPMG_CUDA_TRY(cudaMemcpyAsync(c->r64, c->b64, (size_t)R * n * 16, cudaMemcpyDeviceToDevice, c->s));
  for (int q = 0; q < R; ++q) tol[q] = c->p.tol * bn[q];
  iters = 0;
  restarts = 0;
  const Scal32 one = scal_all(1.0, R), zero = scal_all(0.0, R), minus = scal_all(-1.0, R);
  for (;;) {
    BLAS(host_norms(c, P64, c->r64, R, rn));
    relres = 0;
    bool all = true;
    for (int q = 0; q < R; ++q) {
      if (!std::isfinite(rn[q])) {
        relres = rn[q];
        return fail(MG_ERR_NONFINITE, "the residual became non-finite");
      }
      const double rel = bn[q] > 0 ? rn[q] / bn[q] : 0.0;
      relres = std::max(relres, rel);
      if (rn[q] > tol[q]) all = false;
    }
    // the FP64 residual of every system at this restart / defect correction (entries
    // with a negative iteration mark the recomputed residuals)
    for (int q = 0; q < R; ++q) {
      c->hist.push_back(-(double)iters - 1.0);
      c->hist.push_back((double)(c->hist_r0 + q));
      c->hist.push_back(bn[q] > 0 ? rn[q] / bn[q] : 0.0);
    }
    if (c->p.verbose) std::fprintf(stderr, "[sapmg] outer %d iters %d max relres %.3e\n", restarts, iters, relres);
    if (all) return MG_OK;
    if (iters >= c->p.maxiter) return MG_NOT_CONVERGED;
    std::vector<double> act(R);
    for (int q = 0; q < R; ++q) act[q] = rn[q] > tol[q] ? rn[q] : 0.0;
    c->hist_base = iters;
    c->hist_scale.assign(R, 0.0);
    if (c->prec == P64) {
      for (int q = 0; q < R; ++q) c->hist_scale[q] = bn[q] > 0 ? 1.0 / bn[q] : 0.0;
      TRY(fgmres_cycle(c, P64, P64, R, c->r64, act, c->x64, tol, c->p.maxiter - iters, done, est));
    } else {
      // the inner systems D e = r / ||r|| scale back by ||r|| / ||b||
      for (int q = 0; q < R; ++q) c->hist_scale[q] = bn[q] > 0 ? act[q] / bn[q] : 0.0;
      // FP64 defect correction: flexible GMRES in FP32 on D e = t, t = the
      // normalised residual, restarted on its own FP32 residual t - D e until
      // that is below the inner tolerance (or no longer falls), then x and r
      // are updated in FP64
      Scal32 a = zero;
      for (int q = 0; q < R; ++q) {
        if (act[q] > 0) a.v[q].x = 1.0 / act[q];
        inner[q] = act[q] > 0 ? std::max(2e-6, 0.5 * tol[q] / act[q]) : 1.0;
      }
      std::vector<double> rin(R), rin_prev(R, 2.0), aim(R);
      for (int q = 0; q < R; ++q) rin[q] = act[q] > 0 ? 1.0 : 0.0;
      BLAS(blas_axpby2(P64, a, c->r64, n, P32, zero, c->t64, n, n, R, c->s));
      SAPMG_CUDA_TRY(cudaMemsetAsync(c->e32, 0, (size_t)R * n * 8, c->s));
      const void* rcur = c->t64;
      int step = 0;
      for (int cyc = 0; cyc < kInnerCycles; ++cyc) {
        bool any = false;
        for (int q = 0; q < R; ++q) {
          // stop a system at its tolerance or when a cycle gained less than 10%
          aim[q] = rin[q] > inner[q] && rin[q] < 0.9 * rin_prev[q] ? rin[q] : 0.0;
          any = any || aim[q] > 0;
        }
        if (!any || iters + step >= c->p.maxiter) break;
        c->hist_base = iters + step;
        TRY(fgmres_cycle(c, P32, P32, R, rcur, aim, c->e32, inner, c->p.maxiter - iters - step, done, est));
        int cs = 0;
        for (int q = 0; q < R; ++q) cs = std::max(cs, done[q]);
        step += cs;
        if (cs == 0) break;
        // w = t - D e in FP32 (the Arnoldi work vector is free between cycles)
        TRY(fine_dirac(c, P32, c->w, c->e32, R));
        BLAS(blas_axpby2(P32, one, c->t64, n, P32, minus, c->w, n, n, R, c->s));
        rin_prev = rin;
        BLAS(host_norms(c, P32, c->w, R, rin));
        for (int q = 0; q < R; ++q)
          if (act[q] == 0) rin[q] = 0;
        rcur = c->w;
      }
      for (int q = 0; q < R; ++q) done[q] = step;
      Scal32 sc = zero;
      for (int q = 0; q < R; ++q) sc.v[q].x = act[q];
      BLAS(blas_axpby2(P32, sc, c->e32, n, P64, one, c->x64, n, n, R, c->s));
    }
    int step = 0;
    for (int q = 0; q < R; ++q) step = std::max(step, done[q]);
    iters += step;
    restarts += 1;
    TRY(fine_dirac(c, c->fp64_on_fp32 ? P64E : P64, c->r64, c->x64, R));
    BLAS(blas_axpby2(P64, one, c->b64, n, P64, minus, c->r64, n, n, R, c->s));
    if (step == 0) return MG_NOT_CONVERGED;
  }
}

// ------------------------------------------------------------ CGN
// CG on the normal equations D^dagger D x = D^dagger b, the method Sec. 4
// compares the multilevel solver with (Tables 1-2), R systems at once, from
// x = 0, stopping when ||b - D x|| <= tol ||b||.  The residual r = b - D x is
// updated by the recursion r -= alpha D p, so the test costs nothing extra.
// FP64 form: vectors, links and clover in FP64.  FP32 form: the iteration in
// FP32 with the FP32 links and clover; the FP32 iterate is added to the FP64
// solution and r replaced by the FP64 residual b - D x whenever a system's
// residual has fallen by kCgnUpdate since the last such update (reliable
// updates), keeping the search direction.  Either form ends with the FP64
// residual; if a system is then above the tolerance, CG restarts from it.
constexpr double kCgnUpdate = 1e-2;
constexpr int kCgnMaxRefresh = 20;

static int cgn_alloc(mg_ctx* c) {
  const size_t n = c->fine_n();
  const int R = c->p.nrhs_max;
  if (!c->cg) c->cg = c->alloc((size_t)R * n * 48);
  if (!c->cg_part) c->cg_part = (double*)c->alloc(sizeof(double) * (2 * (size_t)c->g.nblocks * R + (size_t)R * kCgnMaxG));
  if (!c->cg_st) c->cg_st = (CgnState*)c->alloc(sizeof(CgnState) * R);
  if (!c->cg || !c->cg_part || !c->cg_st) return fail(MG_ERR_OOM, "CGN workspace");
  if (!c->cg_host && cudaMallocHost((void**)&c->cg_host, sizeof(CgnState) * 2 * R) != cudaSuccess) {
    c->cg_host = nullptr;
    return fail(MG_ERR_OOM, "CGN host buffer");
  }
  return MG_OK;
}

static int cgn_dirac(mg_ctx* c, int type, void* out, const void* in, int R, bool dag, double* part) {
  ProfScope ps(c->prof, FAM_DIRAC, c->s);
  count_bytes((double)c->g.V * (R * 2 * 12 * vec_bytes(type) + fields_bytes(type)));
  return launch_dirac_ex(type, c->g, out, in, type == P64 ? c->U64 : c->U32, type == P64 ? c->A64 : c->A32, R, dag,
                         part, c->s);
}

// RAII pair of events for the pipelined convergence check.
struct EventPair {
  cudaEvent_t e[2] = {nullptr, nullptr};
  ~EventPair() {
    for (auto& q : e)
      if (q) cudaEventDestroy(q);
  }
};

static int cgn_batch(mg_ctx* c, int type, int R, double tol, int maxiter, int& iters, int& updates, double& relres) {
  const size_t n = c->fine_n();
  const int nb = c->g.nblocks;
  const int G = cgn_grid(type == P64 ? n : n / 2);
  cudaStream_t s = c->s;
  char* w = (char*)c->cg;
  const size_t vb = (size_t)R * n * (type == P64 ? 16 : 8);
  void* x = type == P64 ? c->x64 : (void*)w;
  void* r = type == P64 ? c->r64 : (void*)(w + vb);
  void* p = w + (type == P64 ? 0 : 2) * vb;
  void* q = w + (type == P64 ? 1 : 3) * vb;
  void* sv = w + (type == P64 ? 2 : 4) * vb;
  double* part_q = c->cg_part;
  double* part_s = part_q + (size_t)nb * R;
  double* part_r = part_s + (size_t)nb * R;
  CgnState* st = c->cg_st;
  CgnState* hs = c->cg_host;
  EventPair ev;
  for (auto& e : ev.e) SAPMG_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));

  // x = 0, r = b, s = D^dagger r, p = s
  SAPMG_CUDA_TRY(cudaMemsetAsync(c->x64, 0, (size_t)R * n * 16, s));
  if (type == P32) SAPMG_CUDA_TRY(cudaMemsetAsync(x, 0, vb, s));
  SAPMG_CUDA_TRY(cudaMemsetAsync(c->t64, 0, (size_t)R * n * 16, s));
  BLAS(launch_cgn_residual(type, c->b64, c->t64, r, n, R, part_r, G, s));
  TRY(cgn_dirac(c, type, sv, r, R, true, part_s));
  BLAS(launch_cgn_gamma(part_s, nb, part_r, G, R, st, tol * tol, true, s));
  BLAS(launch_cgn_p(type, p, sv, n, R, st, true, G, s));
  SAPMG_CUDA_TRY(cudaMemcpyAsync(hs, st, sizeof(CgnState) * R, cudaMemcpyDeviceToHost, s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<double> bb(R), ref(R);
  for (int k = 0; k < R; ++k) {
    bb[k] = hs[k].rr;
    ref[k] = hs[k].rr;
    if (!std::isfinite(bb[k])) return fail(MG_ERR_NONFINITE, "non-finite right-hand side");
  }
  // x64 += x32 (FP32 form), r = b - D x64 in FP64, rr of every system
  auto refresh = [&]() -> int {
    if (type == P32) BLAS(launch_cgn_accum(c->x64, x, n, R, G, s));
    TRY(cgn_dirac(c, P64, c->t64, c->x64, R, false, nullptr));
    BLAS(launch_cgn_residual(type, c->b64, c->t64, r, n, R, part_r, G, s));
    BLAS(launch_cgn_rr(part_r, G, R, st, s));
    return MG_OK;
  };
  updates = 0;
  int refreshes = 0, it = 0;
  bool update_now = false;
  for (;;) {
    // iterate until no system is active; the host reads the scalars of the
    // previous iteration while the device runs the current one
    for (int k = 0;; ++k, ++it) {
      TRY(cgn_dirac(c, type, q, p, R, false, part_q));
      BLAS(launch_cgn_alpha(part_q, nb, R, st, maxiter, s));
      SAPMG_CUDA_TRY(cudaMemcpyAsync(hs + (it & 1) * R, st, sizeof(CgnState) * R, cudaMemcpyDeviceToHost, s));
      SAPMG_CUDA_TRY(cudaEventRecord(ev.e[it & 1], s));
      BLAS(launch_cgn_xr(type, x, r, p, q, n, R, st, part_r, G, s));
      if (update_now) {
        TRY(refresh());
        ++updates;
        update_now = false;
      }
      TRY(cgn_dirac(c, type, sv, r, R, true, part_s));
      BLAS(launch_cgn_beta(part_s, nb, part_r, G, R, st, s));
      BLAS(launch_cgn_p(type, p, sv, n, R, st, false, G, s));
      if (k == 0) continue;
      SAPMG_CUDA_TRY(cudaEventSynchronize(ev.e[(it - 1) & 1]));
      const CgnState* h = hs + ((it - 1) & 1) * R;
      bool any = false;
      for (int j = 0; j < R; ++j) {
        if (!h[j].act) continue;
        any = true;
        if (type == P32 && h[j].rr < kCgnUpdate * kCgnUpdate * ref[j]) update_now = true;
      }
      if (!any) break;
      if (update_now)
        for (int j = 0; j < R; ++j) ref[j] = h[j].rr;
    }
    TRY(refresh());
    ++refreshes;
    ++updates;
    SAPMG_CUDA_TRY(cudaMemcpyAsync(hs, st, sizeof(CgnState) * R, cudaMemcpyDeviceToHost, s));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(s));
    bool conv = true, left = false;
    relres = 0;
    iters = 0;
    for (int j = 0; j < R; ++j) {
      const double rr = hs[j].rr;
      if (!std::isfinite(rr)) {
        relres = rr;
        return fail(MG_ERR_NONFINITE, "the residual became non-finite");
      }
      relres = std::max(relres, bb[j] > 0 ? std::sqrt(rr / bb[j]) : 0.0);
      iters += hs[j].its;
      if (rr > hs[j].thr) {
        conv = false;
        if (hs[j].its < maxiter) left = true;
      }
      ref[j] = rr;
    }
    if (c->p.verbose)
      std::fprintf(stderr, "[sapmg] CGN %d iterations (summed), %d updates, max relres %.3e\n", iters, updates, relres);
    if (conv) return MG_OK;
    if (!left || refreshes >= kCgnMaxRefresh) return MG_NOT_CONVERGED;
    // CG again from the FP64 residual: s = D^dagger r, p = s
    TRY(cgn_dirac(c, type, sv, r, R, true, part_s));
    BLAS(launch_cgn_gamma(part_s, nb, part_r, G, R, st, 0.0, false, s));
    BLAS(launch_cgn_p(type, p, sv, n, R, st, true, G, s));
  }
}

// ------------------------------------------------------------ set-up
__global__ void nonfinite_kernel(const double* __restrict__ x, size_t n, int* flag) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) *flag = 1;
}

static int check_finite(mg_ctx* c, const double* x, size_t n_doubles) {
  int* flag = (int*)c->alloc(sizeof(int));
  if (!flag) return fail(MG_ERR_OOM, "allocation failed");
  SAPMG_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), c->s));
  nonfinite_kernel<<<1024, 256, 0, c->s>>>(x, n_doubles, flag); count_launches(1);
  int h = 0;
  SAPMG_CUDA_TRY(cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  return h ? fail(MG_ERR_NONFINITE, "non-finite value in input field") : MG_OK;
}

// Global orthonormalisation of the N set-up vectors (FP64): classical
// Gram-Schmidt against the previous vectors, applied twice, then normalise.
// Classical Gram-Schmidt with a second pass of N vectors (type P64, or P32
// for the mixed form's set-up vectors).
static int orthonormalise(mg_ctx* c, void* V, int N, size_t n, int type = P64) {
  const BVec one = bvec(n, 1, n);
  const size_t eb = type == P64 ? 16 : 8;
  auto Vk = [&](int k) { return (void*)((char*)V + (size_t)k * n * eb); };
  std::vector<const void*> vl;
  for (int k = 0; k < N; ++k) {
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      TRY(blas_multidot(type, one, vl.data(), k, Vk(k), c->hd, c->ldh, 0, nullptr, c->partial, c->s));
      TRY(blas_multiaxpy(type, one, Vk(k), vl.data(), k, c->hd, c->ldh, -1.0, c->s));
    }
    TRY(dot_to(c, type, one, Vk(k), Vk(k), c->hd + c->ldh - 1, 1));
    TRY(blas_normalize(type, one, Vk(k), Vk(k), c->hd + c->ldh - 1, 1, nullptr, 0, c->s));
    vl.push_back(Vk(k));
  }
  return MG_OK;
}

// P (in the cycle's storage) and D_c = P^dagger D P from the global test
// vectors in V64, which are locally orthonormalised in place (buffers
// allocated on the first call, refilled on later ones).
static int build_level0_operators(mg_ctx* c) {
  const size_t n = c->fine_n();
  const int N = c->N0;
  TRY(launch_block_gs0(c->g, c->V64, N, c->s));
  if (!c->Pv) c->Pv = c->alloc((size_t)N * n * complex_bytes(c->pv_prec));
  if (!c->Pv) return fail(MG_ERR_OOM, "interpolation");
  TRY(launch_store_p0(c->pv_prec, c->g, c->V64, c->Pv, N, c->s));
  // Galerkin coarse operator
  CoarseLevel& L = c->c1;
  for (int mu = 0; mu < 4; ++mu) L.cg.L[mu] = c->g.nb[mu];
  L.cg.nsites = c->g.nblocks;
  L.cg.n2 = 2 * N;
  const size_t msz = (size_t)L.cg.nsites * 9 * L.cg.n2 * L.cg.n2;
  if (!L.M64) L.M64 = c->alloc(msz * 16);
  if (!L.M64) return fail(MG_ERR_OOM, "coarse operator");
  // the mixed form stores D_c in FP32 and FP16: assemble it from FP32 copies in
  // FP32 arithmetic (the flexible basis, free during the set-up, holds the
  // vectors) unless SAPMG_SETUP_FP32=0 or the basis is too small
  const bool f32 = c->vt == P32 && c->setup_fp32 && c->U32 && c->A32 && c->Z &&
                   (size_t)c->m * c->p.nrhs_max >= (size_t)N;
  if (f32) {
    TRY(blas_axpby2(P64, scal_all(1.0, N), c->V64, n, P32, scal_all(0.0, N), c->Z, n, n, N, c->s));
    TRY(launch_assemble0(c->g, P32, c->Z, c->U32, c->A32, L.M64, N, c->s));
  } else {
    TRY(launch_assemble0(c->g, P64, c->V64, c->U64, c->A64, L.M64, N, c->s));
  }
  L.store = c->dc_prec;
  if (c->dc_prec == P64) {
    L.M = L.M64;
  } else {
    if (!L.M) L.M = c->alloc(msz * complex_bytes(c->dc_prec));
    if (!L.M) return fail(MG_ERR_OOM, "coarse operator");
    TRY(launch_convert(P64, L.M64, c->dc_prec, L.M, msz, c->s));
    if (c->dc_prec == P32 && c->coarse_fp16 && L.cg.n2 % 8 == 0 && L.cg.n2 <= 64) {
      if (!L.Mh) L.Mh = c->alloc(msz * complex_bytes(P16));
      if (!L.Mh) return fail(MG_ERR_OOM, "coarse operator");
      TRY(launch_convert(P64, L.M64, P16, L.Mh, msz, c->s));
    }
  }
  return MG_OK;
}

// Bootstrap set-up part 2 (Sec. 3), run once on a two-level hierarchy:
//  1. N harmonic Ritz pairs (theta_i, phi_i) of D_c from the Arnoldi space of
//     dimension 2N of a start vector (FP64, two Gram-Schmidt passes; a
//     subdiagonal entry below 1e-12 of the largest ends the space, which is
//     then invariant); the small eigenproblem on the host;
//  2. x_i = S(theta_i)^iota P phi_i: P phi_i with the FP64 local vectors, then
//     iota sweeps of the shifted Schwarz pass on (D - theta_i) x = 0;
//  3. V = {x_i} followed by the part-1 vectors (the second half of V2),
//     orthonormalised (two classical Gram-Schmidt passes, FP64);
//  4. the N eigenvectors y_k of (DV)^dagger DV (= V^dagger D^dagger D V) with
//     the smallest eigenvalues give the new test vectors V y_k;
//  5. P and D_c rebuilt from them.
static int setup_level1(mg_ctx* c);
static int finish_level1(mg_ctx* c);

static int setup_part2(mg_ctx* c, void* V2) {
  const mg_params& p = c->p;
  const size_t n = c->fine_n();
  const int N = c->N0;
  const bool three = p.n_levels == 3;        // the Ritz pairs come from the coarsest operator
  CoarseLevel& L = three ? c->c2 : c->c1;
  const size_t nc = L.n();
  const int m = (int)std::min<size_t>((size_t)2 * N, nc);
  const BVec bc = bvec(nc, 1, nc), bf = bvec(n, 1, n);
  cudaStream_t s = c->s;
  void* Q = c->alloc((size_t)(m + 2) * nc * 16);            // basis q_0..q_m and phi
  double2* d = (double2*)c->alloc(sizeof(double2) * 320);   // device scalars
  void* phi1 = three ? c->alloc(c->c1.n() * 16) : nullptr;  // three levels: phi interpolated to level 1
  if (!Q || !d || (three && !phi1)) return fail(MG_ERR_OOM, "set-up part 2 workspace");
  double2 *h1 = d, *h2 = d + 72, *coef = d + 144, *nrm = d + 216, *shift = d + 224;
  auto Qj = [&](int j) { return (void*)((char*)Q + (size_t)j * nc * 16); };
  auto Vk = [&](int k) { return (void*)((char*)V2 + (size_t)k * n * 16); };
  void* phi = Qj(m + 1);
  auto to_dev = [&](double2* dst, const std::vector<double2>& src) -> int {
    SAPMG_CUDA_TRY(cudaMemcpyAsync(dst, src.data(), sizeof(double2) * src.size(), cudaMemcpyHostToDevice, s));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(s));
    return MG_OK;
  };
  auto to_host = [&](std::vector<double2>& dst, const double2* src, size_t cnt) -> int {
    dst.resize(cnt);
    SAPMG_CUDA_TRY(cudaMemcpyAsync(dst.data(), src, sizeof(double2) * cnt, cudaMemcpyDeviceToHost, s));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(s));
    return MG_OK;
  };

  // 1. Arnoldi on D_c from the start vector
  if (p.setup2_start) {
    SAPMG_CUDA_TRY(cudaMemcpyAsync(Qj(0), p.setup2_start, nc * 16, cudaMemcpyDeviceToDevice, s));
  } else {
    // uniform in [-1, 1) per real component from SplitMix64 counters (stream 6)
    std::vector<double2> h0(nc);
    const uint64_t key = host_splitmix64(host_splitmix64(p.seed) + 6ull);
    for (size_t i = 0; i < nc; ++i) {
      const double re = (double)(host_splitmix64(key + 2 * i) >> 11) * 0x1.0p-52 - 1.0;
      const double im = (double)(host_splitmix64(key + 2 * i + 1) >> 11) * 0x1.0p-52 - 1.0;
      h0[i] = make_double2(re, im);
    }
    TRY(to_dev((double2*)Qj(0), h0));
  }
  TRY(dot_to(c, P64, bc, Qj(0), Qj(0), nrm, 1));
  TRY(blas_normalize(P64, bc, Qj(0), Qj(0), nrm, 1, nullptr, 0, s));
  std::vector<double2> H((size_t)(m + 1) * m, make_double2(0, 0)), t1, t2, tn;
  std::vector<const void*> vl;
  int steps = m;
  double hmax = 0;
  for (int j = 0; j < m; ++j) {
    vl.push_back(Qj(j));
    void* w = Qj(j + 1);
    TRY(launch_coarse_apply(P64, L.cg, L.M64, Qj(j), w, 1, s));
    TRY(blas_multidot(P64, bc, vl.data(), j + 1, w, h1, 1, 0, nullptr, c->partial, s));
    TRY(blas_multiaxpy(P64, bc, w, vl.data(), j + 1, h1, 1, -1.0, s));
    TRY(blas_multidot(P64, bc, vl.data(), j + 1, w, h2, 1, 0, nullptr, c->partial, s));
    TRY(blas_multiaxpy(P64, bc, w, vl.data(), j + 1, h2, 1, -1.0, s));
    TRY(dot_to(c, P64, bc, w, w, nrm, 1));
    TRY(to_host(t1, h1, j + 1));
    TRY(to_host(t2, h2, j + 1));
    TRY(to_host(tn, nrm, 1));
    for (int i = 0; i <= j; ++i) {
      H[(size_t)j * (m + 1) + i] = make_double2(t1[i].x + t2[i].x, t1[i].y + t2[i].y);
      hmax = std::max(hmax, std::hypot(t1[i].x + t2[i].x, t1[i].y + t2[i].y));
    }
    const double beta = std::sqrt(std::max(tn[0].x, 0.0));
    if (!std::isfinite(beta)) return fail(MG_ERR_NONFINITE, "set-up part 2: non-finite Arnoldi vector");
    hmax = std::max(hmax, beta);
    if (beta <= 1e-12 * hmax) {            // invariant space: stop here
      steps = j + 1;
      break;
    }
    H[(size_t)j * (m + 1) + j + 1] = make_double2(beta, 0);
    TRY(blas_normalize(P64, bc, w, w, nrm, 1, nullptr, 0, s));
  }
  std::vector<double> hb((size_t)2 * (steps + 1) * steps, 0.0), th(2 * (size_t)steps), Y((size_t)2 * steps * steps);
  for (int j = 0; j < steps; ++j)
    for (int i = 0; i <= steps; ++i) {
      const double2 v = H[(size_t)j * (m + 1) + i];
      hb[2 * ((size_t)j * (steps + 1) + i)] = v.x;
      hb[2 * ((size_t)j * (steps + 1) + i) + 1] = v.y;
    }
  if (harmonic_ritz_host(steps, hb.data(), th.data(), Y.data()) != MG_OK)
    return fail(MG_ERR_NONFINITE, "set-up part 2: the harmonic Ritz problem failed");
  const int nr = std::min(N, steps);

  // 2. x_i = S(theta_i)^iota P phi_i into the first nr slots of V2
  for (int i = 0; i < nr; ++i) {
    std::vector<double2> y(steps);
    for (int k = 0; k < steps; ++k) y[k] = make_double2(Y[2 * ((size_t)i * steps + k)], Y[2 * ((size_t)i * steps + k) + 1]);
    TRY(to_dev(coef, y));
    SAPMG_CUDA_TRY(cudaMemsetAsync(phi, 0, nc * 16, s));
    TRY(blas_multiaxpy(P64, bc, phi, vl.data(), steps, coef, 1, 1.0, s));
    void* xi = Vk(i);
    if (three) {
      TRY(launch_transfer1(false, P64, c->c1.cg, c->agg1, phi, phi1, c->W64, c->N1, 1, s));
      TRY(launch_prolong_v64(c->g, c->V64, N, phi1, xi, s));
    } else {
      TRY(launch_prolong_v64(c->g, c->V64, N, phi, xi, s));
    }
    TRY(to_dev(shift, std::vector<double2>{make_double2(th[2 * i], th[2 * i + 1])}));
    if (c->vt == P64) {
      for (int it = 0; it < p.setup2_iters; ++it)
        for (int col = 0; col < 2; ++col)
          TRY(launch_sap_colour_shifted(P64, c->g, xi, c->zero_f, c->U64, c->A64, col, p.n_mr, 1, shift, s));
    } else {
      const Scal32 one = scal_all(1.0, 1), zero = scal_all(0.0, 1);
      TRY(blas_axpby2(P64, one, xi, n, P32, zero, c->io_b, n, n, 1, s));
      for (int it = 0; it < p.setup2_iters; ++it)
        for (int col = 0; col < 2; ++col)
          TRY(launch_sap_colour_shifted(c->prec, c->g, c->io_b, c->zero_f, c->Us, c->As, col, p.n_mr, 1, shift, s));
      TRY(blas_axpby2(P32, one, c->io_b, n, P64, zero, xi, n, n, 1, s));
    }
  }
  // the part-1 vectors follow the nr new ones (one vector at a time, upwards: no overlap)
  if (nr < N)
    for (int k = 0; k < N; ++k)
      SAPMG_CUDA_TRY(cudaMemcpyAsync(Vk(nr + k), Vk(N + k), n * 16, cudaMemcpyDeviceToDevice, s));
  const int nv = nr + N;

  // 3. orthonormalise V (classical Gram-Schmidt, two passes)
  std::vector<const void*> vall;
  for (int k = 0; k < nv; ++k) {
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      TRY(blas_multidot(P64, bf, vall.data(), k, Vk(k), h1, 1, 0, nullptr, c->partial, s));
      TRY(blas_multiaxpy(P64, bf, Vk(k), vall.data(), k, h1, 1, -1.0, s));
    }
    TRY(dot_to(c, P64, bf, Vk(k), Vk(k), nrm, 1));
    TRY(blas_normalize(P64, bf, Vk(k), Vk(k), nrm, 1, nullptr, 0, s));
    vall.push_back(Vk(k));
  }
  // 4. G = V^dagger D^dagger D V, its N lowest eigenvectors
  std::vector<double> G((size_t)2 * nv * nv), ev(nv), EV((size_t)2 * nv * nv);
  for (int k = 0; k < nv; ++k) {
    TRY(fine_dirac(c, P64, c->t64, Vk(k), 1));
    TRY(cgn_dirac(c, P64, c->r64, c->t64, 1, true, nullptr));
    TRY(blas_multidot(P64, bf, vall.data(), nv, c->r64, h1, 1, 0, nullptr, c->partial, s));
    TRY(to_host(t1, h1, nv));
    for (int j = 0; j < nv; ++j) {
      G[2 * ((size_t)k * nv + j)] = t1[j].x;
      G[2 * ((size_t)k * nv + j) + 1] = t1[j].y;
    }
  }
  TRY(eigh_host(nv, G.data(), ev.data(), EV.data()));
  // 5. new test vectors and the rebuilt hierarchy
  for (int k = 0; k < N; ++k) {
    std::vector<double2> y(nv);
    for (int j = 0; j < nv; ++j) y[j] = make_double2(EV[2 * ((size_t)k * nv + j)], EV[2 * ((size_t)k * nv + j) + 1]);
    TRY(to_dev(coef, y));
    void* vk = (char*)c->V64 + (size_t)k * n * 16;
    SAPMG_CUDA_TRY(cudaMemsetAsync(vk, 0, n * 16, s));
    TRY(blas_multiaxpy(P64, bf, vk, vall.data(), nv, coef, 1, 1.0, s));
  }
  if (three) {                               // the new vectors also start level 1 again (restricted)
    c->Vs64 = c->alloc((size_t)N * n * 16);
    if (!c->Vs64) return fail(MG_ERR_OOM, "set-up vectors");
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->Vs64, c->V64, (size_t)N * n * 16, cudaMemcpyDeviceToDevice, s));
  }
  TRY(build_level0_operators(c));
  if (three) TRY(setup_level1(c));           // level 1 rebuilt as part 1 builds it
  SAPMG_CUDA_TRY(cudaStreamSynchronize(s));
  c->release(Q);
  c->release(d);
  if (phi1) c->release(phi1);
  return MG_OK;
}

// verbose: wall time of the set-up's phases (synchronising the stream; only then)
struct PhaseClock {
  const mg_ctx* c;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  explicit PhaseClock(const mg_ctx* c_) : c(c_) {}
  double lap() {
    if (!c->p.verbose) return 0.0;
    cudaStreamSynchronize(c->s);
    const auto n = std::chrono::steady_clock::now();
    const double s = std::chrono::duration<double>(n - t).count();
    t = n;
    return s;
  }
};

static int setup_level0(mg_ctx* c) {
  const size_t n = c->fine_n();
  const int N = c->N0;
  const mg_params& p = c->p;
  c->V64 = c->alloc((size_t)N * n * 16);
  if (!c->V64) return fail(MG_ERR_OOM, "test vectors");
  if (c->load_v0) {                        // a saved set-up: its vectors replace both bootstrap parts
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->V64, c->load_v0->data(), (size_t)N * n * 16, cudaMemcpyHostToDevice, c->s));
    return build_level0_operators(c);
  }
  if (p.init_vectors) {
    TRY(launch_pack_spinor(p.init_vectors_prec == P32 ? P32 : P64, p.init_vectors, P64, c->V64, c->g, N, c->s));
  } else {
    TRY(launch_draw_vectors(c->g, c->V64, N, p.seed, 3ull /* test-vector stream */, c->s));
  }
  // bootstrap part 1: nu sweeps of the smoother's iteration matrix (SAP on D x = 0), kept orthonormal
  PhaseClock clk(c);
  double t_sweep = 0, t_orth = 0;
  // Mixed form: the vectors stay FP32 through part 1 (in the flexible basis,
  // free until the first solve) and are orthonormalised in FP32; the sweeps
  // are FP32 anyway, and FP64 arithmetic is scarce on this GPU.  The FP64
  // form, or a basis too small for N vectors, keeps them FP64.
  const bool f32 = c->vt == P32 && c->setup_fp32 && p.setup_iters > 0 && (size_t)c->m * p.nrhs_max >= (size_t)N;
  if (f32) {
    TRY(blas_axpby2(P64, scal_all(1.0, N), c->V64, n, P32, scal_all(0.0, N), c->Z, n, n, N, c->s));
    for (int it = 0; it < p.setup_iters; ++it) {
      for (int k = 0; k < N; ++k) TRY(smoother_sweeps(c, c->zero_f, (char*)c->Z + (size_t)k * n * 8, 1, 1));
      t_sweep += clk.lap();
      TRY(orthonormalise(c, c->Z, N, n, P32));
      t_orth += clk.lap();
    }
    TRY(blas_axpby2(P32, scal_all(1.0, N), c->Z, n, P64, scal_all(0.0, N), c->V64, n, n, N, c->s));
  }
  for (int it = 0; it < p.setup_iters && !f32; ++it) {
    for (int k = 0; k < N; ++k) {
      void* vk = (char*)c->V64 + (size_t)k * n * 16;
      if (c->vt == P64) {
        TRY(smoother_sweeps(c, c->zero_f, vk, 1, 1));
      } else {
        const Scal32 one = scal_all(1.0, 1), zero = scal_all(0.0, 1);
        TRY(blas_axpby2(P64, one, vk, n, P32, zero, c->io_b, n, n, 1, c->s));
        TRY(smoother_sweeps(c, c->zero_f, c->io_b, 1, 1));
        TRY(blas_axpby2(P32, one, c->io_b, n, P64, zero, vk, n, n, 1, c->s));
      }
    }
    t_sweep += clk.lap();
    TRY(orthonormalise(c, c->V64, N, n));
    t_orth += clk.lap();
  }
  if (p.verbose)
    std::fprintf(stderr, "[sapmg] set-up part 1: %d sweeps of %d vectors %.3f s, orthonormalisation %.3f s\n",
                 p.setup_iters, N, t_sweep, t_orth);
  if (p.n_levels == 3) {                   // the smoothed vectors start level 1 (restricted below)
    c->Vs64 = c->alloc((size_t)N * n * 16);
    if (!c->Vs64) return fail(MG_ERR_OOM, "set-up vectors");
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->Vs64, c->V64, (size_t)N * n * 16, cudaMemcpyDeviceToDevice, c->s));
  }
  void* V2 = nullptr;
  if (p.setup2_iters > 0) {                // part 2 keeps the part-1 vectors as the second half of its set
    V2 = c->alloc((size_t)2 * N * n * 16);
    if (!V2) return fail(MG_ERR_OOM, "set-up part 2 vectors");
    SAPMG_CUDA_TRY(cudaMemcpyAsync((char*)V2 + (size_t)N * n * 16, c->V64, (size_t)N * n * 16,
                                   cudaMemcpyDeviceToDevice, c->s));
  }
  clk.lap();
  TRY(build_level0_operators(c));
  if (p.verbose) std::fprintf(stderr, "[sapmg] block Gram-Schmidt, P and D_c %.3f s\n", clk.lap());
  if (p.setup2_iters > 0 && p.n_levels == 2) {
    TRY(setup_part2(c, V2));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
    c->release(V2);
  } else if (p.setup2_iters > 0) {
    c->part2_buf = V2;                     // three levels: part 2 runs once level 2 exists
  }
  return MG_OK;
}

// Bootstrap part 1 on level 1 (Sec. 3: the procedure continues recursively on
// the coarser grid): the smoothed fine vectors restricted with P^dagger start
// N1 level-1 vectors; setup_iters Schwarz sweeps of the level-1 smoother on
// D_c x = 0 each, kept orthonormal; local orthonormalisation on the level-2
// aggregates; D_c2 = P1^dagger D_c1 P1.
static int setup_level1(mg_ctx* c) {
  const mg_params& p = c->p;
  const size_t nf = c->fine_n();
  CoarseLevel& L1 = c->c1;
  const size_t n1 = L1.n();
  const int N0 = c->N0, N1 = c->N1;
  c->sap1 = make_box(L1.cg, p.sap_block2);
  c->agg1 = make_box(L1.cg, p.agg2);
  if (!c->W64) c->W64 = c->alloc((size_t)N1 * n1 * 16);         // reused when set-up part 2 rebuilds level 1
  if (!c->W64) return fail(MG_ERR_OOM, "level-1 vectors");
  if (c->load_w1) {                        // a saved set-up: the level-1 vectors as saved
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->W64, c->load_w1->data(), (size_t)N1 * n1 * 16, cudaMemcpyHostToDevice, c->s));
    return finish_level1(c);
  }
  // the smoothed fine vectors restricted with the FP64 P0, read in place
  for (int k = 0; k < N1; ++k)
    TRY(launch_restrict_v64(c->g, c->V64, N0, (char*)c->Vs64 + (size_t)k * nf * 16,
                            (char*)c->W64 + (size_t)k * n1 * 16, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  c->release(c->Vs64);
  c->Vs64 = nullptr;
  // level-1 smoothing of the vectors (S^nu on D_c1 x = 0), kept orthonormal
  void* zero1 = c->alloc(n1 * 16);
  void* t32 = c->alloc(n1 * 8);
  if (!zero1 || !t32) return fail(MG_ERR_OOM, "level-1 set-up");
  SAPMG_CUDA_TRY(cudaMemsetAsync(zero1, 0, n1 * 16, c->s));
  const Scal32 one = scal_all(1.0, 1), zero = scal_all(0.0, 1);
  for (int it = 0; it < p.setup_iters; ++it) {
    for (int k = 0; k < N1; ++k) {
      void* wk = (char*)c->W64 + (size_t)k * n1 * 16;
      if (c->vt == P64) {
        TRY(smoother_sweeps1(c, zero1, wk, 1, 1));
      } else {
        TRY(blas_axpby2(P64, one, wk, n1, P32, zero, t32, n1, n1, 1, c->s));
        TRY(smoother_sweeps1(c, zero1, t32, 1, 1));
        TRY(blas_axpby2(P32, one, t32, n1, P64, zero, wk, n1, n1, 1, c->s));
      }
    }
    TRY(orthonormalise(c, c->W64, N1, n1));
  }
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  c->release(zero1);
  c->release(t32);
  return finish_level1(c);
}

// Level 1's local orthonormalisation on the level-2 aggregates, its vectors in
// the cycle's type and the level-2 Galerkin operator D_c2 = P1^dagger D_c1 P1.
static int finish_level1(mg_ctx* c) {
  CoarseLevel& L1 = c->c1;
  const size_t n1 = L1.n();
  const int N1 = c->N1;
  TRY(launch_block_gs1(L1.cg, c->agg1, c->W64, N1, c->s));
  if (c->vt == P64) {
    c->W = c->W64;
  } else {
    if (!c->W) c->W = c->alloc((size_t)N1 * n1 * 8);
    if (!c->W) return fail(MG_ERR_OOM, "level-1 vectors");
    TRY(launch_convert(P64, c->W64, P32, c->W, (size_t)N1 * n1, c->s));
  }
  // level 2
  CoarseLevel& L2 = c->c2;
  for (int mu = 0; mu < 4; ++mu) L2.cg.L[mu] = c->agg1.nb[mu];
  L2.cg.nsites = c->agg1.nboxes;
  L2.cg.n2 = 2 * N1;
  const size_t msz = (size_t)L2.cg.nsites * 9 * L2.cg.n2 * L2.cg.n2;
  if (!L2.M64) L2.M64 = c->alloc(msz * 16);
  if (!L2.M64) return fail(MG_ERR_OOM, "level-2 operator");
  TRY(launch_assemble1(L1.cg, L2.cg, c->agg1, c->W64, L1.M64, L2.M64, N1, c->s));
  L2.store = c->dc_prec;
  if (c->dc_prec == P64) {
    L2.M = L2.M64;
  } else {
    if (!L2.M) L2.M = c->alloc(msz * complex_bytes(c->dc_prec));
    if (!L2.M) return fail(MG_ERR_OOM, "level-2 operator");
    TRY(launch_convert(P64, L2.M64, c->dc_prec, L2.M, msz, c->s));
    if (c->dc_prec == P32 && c->coarse_fp16 && L2.cg.n2 % 8 == 0 && L2.cg.n2 <= 64) {
      if (!L2.Mh) L2.Mh = c->alloc(msz * complex_bytes(P16));
      if (!L2.Mh) return fail(MG_ERR_OOM, "level-2 operator");
      TRY(launch_convert(P64, L2.M64, P16, L2.Mh, msz, c->s));
    }
  }
  return MG_OK;
}

static int alloc_fgmres1_ws(mg_ctx* c, int k, int R) {
  const size_t n = c->c1.n(), eb = complex_bytes(c->vt);
  c->f1V = c->alloc((size_t)(k + 1) * R * n * eb);
  c->f1Z = c->alloc((size_t)k * R * n * eb);
  c->f1w = c->alloc((size_t)R * n * eb);
  c->f1H = (double2*)c->alloc(sizeof(double2) * 33 * 33 * R);
  c->f1tmp = (double2*)c->alloc(sizeof(double2) * 33 * 33 * R);
  c->f1beta2 = (double2*)c->alloc(sizeof(double2) * R);
  c->f1y = (double2*)c->alloc(sizeof(double2) * 33 * R);
  if (!c->f1V || !c->f1Z || !c->f1w || !c->f1H || !c->f1tmp || !c->f1beta2 || !c->f1y)
    return fail(MG_ERR_OOM, "level-1 workspace");
  SAPMG_CUDA_TRY(cudaMemsetAsync(c->f1H, 0, sizeof(double2) * 33 * 33 * R, c->s));
  return MG_OK;
}

static int alloc_coarse_ws(mg_ctx* c, CoarseLevel& L, int kmax, int R) {
  const size_t n = L.n(), eb = complex_bytes(c->vt);
  const char* hb = std::getenv("SAPMG_COARSE_BASIS_FP16");
  if (L.Mh && c->vt == P32 && n % 2 == 0 && (hb ? std::atoi(hb) : 1)) {
    L.Vh = c->alloc((size_t)(kmax + 1) * R * n * 4);
    if (!L.Vh) return fail(MG_ERR_OOM, "coarse workspace");
  }
  if (!L.Vh) L.V = c->alloc((size_t)(kmax + 1) * R * n * eb);
  L.w = c->alloc((size_t)R * n * eb);
  L.x = c->alloc((size_t)R * n * eb);
  L.b = c->alloc((size_t)R * n * eb);
  L.H = (double2*)c->alloc(sizeof(double2) * 33 * 33 * R);
  L.tmp = (double2*)c->alloc(sizeof(double2) * 33 * 33 * R);
  L.beta2 = (double2*)c->alloc(sizeof(double2) * R);
  L.y = (double2*)c->alloc(sizeof(double2) * 33 * R);
  if ((!L.V && !L.Vh) || !L.w || !L.x || !L.b || !L.H || !L.tmp || !L.beta2 || !L.y)
    return fail(MG_ERR_OOM, "coarse workspace");
  SAPMG_CUDA_TRY(cudaMemsetAsync(L.H, 0, sizeof(double2) * 33 * 33 * R, c->s));
  return MG_OK;
}

static int validate(const mg_params* p) {
  for (int mu = 0; mu < 4; ++mu)
    if (p->dims[mu] <= 0 || p->dims[mu] % 8 != 0)
      return fail(MG_ERR_ARG, "every lattice dim must be a positive multiple of 8 (even number of 4^4 blocks)");
  if (p->n_levels < 1 || p->n_levels > 3) return fail(MG_ERR_ARG, "n_levels must be 1, 2 or 3");
  if (p->n_levels == 3) {
    if (p->n_vec[1] < 1 || p->n_vec[1] > p->n_vec[0]) return fail(MG_ERR_ARG, "n_vec[1] must be in 1..n_vec[0]");
    if (p->inner_iters < 1 || p->inner_iters > 32) return fail(MG_ERR_ARG, "inner_iters must be in 1..32");
    int sb = 1, ab = 1;
    for (int mu = 0; mu < 4; ++mu) {
      const int l1 = p->dims[mu] / 4;
      if (p->sap_block2[mu] < 1 || l1 % p->sap_block2[mu] != 0 || (l1 / p->sap_block2[mu]) % 2 != 0)
        return fail(MG_ERR_ARG, "level-1 Schwarz blocks must cut the level-1 lattice into an even number per dim");
      if (p->agg2[mu] < 1 || l1 % p->agg2[mu] != 0)
        return fail(MG_ERR_ARG, "level-2 aggregates must divide the level-1 lattice");
      sb *= p->sap_block2[mu];
      ab *= p->agg2[mu];
    }
    if (sb * 2 * p->n_vec[0] > 1024 || ab * 2 * p->n_vec[0] > 1024)
      return fail(MG_ERR_ARG, "level-1 block or aggregate too large (sites x 2N must be <= 1024)");
  }
  if (p->n_levels >= 2 && (p->n_vec[0] < 1 || p->n_vec[0] > 32)) return fail(MG_ERR_ARG, "n_vec[0] must be in 1..32");
  if (p->setup_iters < 0 || p->n_mr < 0 || p->nu_post < 0) return fail(MG_ERR_ARG, "negative iteration count");
  if (p->coarse_iters < 1 || p->coarse_iters > 32) return fail(MG_ERR_ARG, "coarse_iters must be in 1..32");
  if (p->fgmres_m < 1 || p->fgmres_m > 256) return fail(MG_ERR_ARG, "fgmres_m must be in 1..256");
  if (!(p->tol > 0)) return fail(MG_ERR_ARG, "tol must be positive");
  if (p->maxiter < 1) return fail(MG_ERR_ARG, "maxiter must be positive");
  if (p->precision < MG_FP64 || p->precision > MG_BF16) return fail(MG_ERR_ARG, "unknown precision");
  if (p->nrhs_max < 1 || p->nrhs_max > 32) return fail(MG_ERR_ARG, "nrhs_max must be in 1..32");
  if (p->init_vectors_prec != P64 && p->init_vectors_prec != P32)
    return fail(MG_ERR_ARG, "init_vectors_prec must be MG_FP64 or MG_FP32");
  if (p->setup2_iters < 0) return fail(MG_ERR_ARG, "negative iteration count");
  if (p->setup2_iters > 0 && p->n_levels < 2) return fail(MG_ERR_ARG, "set-up part 2 needs a coarse level");
  return MG_OK;
}

static int autotune(mg_ctx* c);

static int do_setup(mg_ctx* c, const double* U) {
  const mg_params& p = c->p;
  const size_t n = c->fine_n();
  const size_t ulinks = (size_t)c->g.V * 4 * 9, aslots = (size_t)c->g.V * 36;
  TRY(check_finite(c, U, ulinks * 2));
  c->U64 = c->alloc(ulinks * 16);
  c->A64 = c->alloc(aslots * 16);
  if (!c->U64 || !c->A64) return fail(MG_ERR_OOM, "gauge field");
  TRY(launch_pack_gauge(P64, c->g, U, c->U64, p.antiperiodic_t, c->s));
  TRY(launch_clover_build(c->g, U, c->A64, c->m0, c->csw, c->s));
  if (c->prec != P64) {
    c->U32 = c->alloc(ulinks * 8);
    c->A32 = c->alloc(aslots * 8);
    if (!c->U32 || !c->A32) return fail(MG_ERR_OOM, "gauge field");
    TRY(launch_convert(P64, c->U64, P32, c->U32, ulinks, c->s));
    TRY(launch_convert(P64, c->A64, P32, c->A32, aslots, c->s));
    if (c->prec == P32) {
      c->Us = c->U32;
      c->As = c->A32;
    } else {
      c->Us = c->alloc(ulinks * 4);
      c->As = c->alloc(aslots * 4);
      if (!c->Us || !c->As) return fail(MG_ERR_OOM, "gauge field");
      TRY(launch_convert(P64, c->U64, c->prec, c->Us, ulinks, c->s));
      TRY(launch_convert(P64, c->A64, c->prec, c->As, aslots, c->s));
    }
  } else {
    c->Us = c->U64;
    c->As = c->A64;
  }
  // workspace
  const size_t eb = complex_bytes(c->vt);
  const int R = p.nrhs_max;
  c->partial = (double2*)c->alloc(sizeof(double2) * kPartialDouble2);
  c->dev_err = (int*)c->alloc(2 * sizeof(int));
  if (!c->dev_err) return fail(MG_ERR_OOM, "workspace");
  {
    const int init[2] = {0, kMaxSpins};
    SAPMG_CUDA_TRY(cudaMemcpyAsync(c->dev_err, init, sizeof(init), cudaMemcpyHostToDevice, c->s));
    SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  }
  c->zero_f = c->alloc(n * eb);
  c->io_a = c->alloc((size_t)R * n * 16);
  c->io_b = c->alloc((size_t)R * n * 16);
  c->m = p.fgmres_m;
  c->ldh = std::max(c->m, 32) + 8;
  const size_t ft = complex_bytes(c->vt);
  const char* oh = std::getenv("SAPMG_OUTER_FP16");
  c->outer_half = c->vt == P32 && c->outer_dcgs2 && (oh ? std::atoi(oh) : 1);
  if (c->outer_half) {
    c->V = c->alloc((size_t)R * n * ft);
    c->Vh = c->alloc((size_t)c->m * R * n * 4);
    if (!c->Vh) return fail(MG_ERR_OOM, "workspace");
  } else {
    c->V = c->alloc((size_t)(c->m + 1) * R * n * ft);
  }
  c->Z = c->alloc((size_t)c->m * R * n * ft);
  c->w = c->alloc((size_t)R * n * ft);
  c->x64 = c->alloc((size_t)R * n * 16);
  c->r64 = c->alloc((size_t)R * n * 16);
  c->t64 = c->alloc((size_t)R * n * 16);
  c->b64 = c->alloc((size_t)R * n * 16);
  c->e32 = c->vt == P64 ? c->t64 : c->alloc((size_t)R * n * 8);
  c->hd = (double2*)c->alloc(sizeof(double2) * R * c->ldh);
  c->dcg = (double2*)c->alloc(sizeof(double2) * 8 * R * c->ldh);
  if (!c->partial || !c->zero_f || !c->io_a || !c->io_b || !c->V || !c->Z || !c->w || !c->x64 || !c->r64 ||
      !c->t64 || !c->b64 || !c->hd || !c->e32 || !c->dcg)
    return fail(MG_ERR_OOM, "workspace");
  if (cudaMallocHost((void**)&c->hh, sizeof(double2) * R * c->ldh) != cudaSuccess) return fail(MG_ERR_OOM, "host");
  if (cudaMallocHost((void**)&c->dch, sizeof(double2) * 3 * R * c->ldh) != cudaSuccess) return fail(MG_ERR_OOM, "host");
  SAPMG_CUDA_TRY(cudaMemsetAsync(c->zero_f, 0, n * eb, c->s));
  if (p.n_levels >= 2) {
    c->N0 = p.n_vec[0];
    TRY(setup_level0(c));
    TRY(alloc_coarse_ws(c, c->c1, p.coarse_iters, R));
  }
  if (p.n_levels == 3) {
    c->N1 = p.n_vec[1];
    TRY(setup_level1(c));
    if (c->part2_buf) {
      TRY(setup_part2(c, c->part2_buf));
      c->release(c->part2_buf);
      c->part2_buf = nullptr;
    }
    TRY(alloc_coarse_ws(c, c->c2, p.coarse_iters, R));
    TRY(alloc_fgmres1_ws(c, p.inner_iters, R));
  }
  PhaseClock clk(c);
  if (p.autotune) TRY(autotune(c));
  if (p.verbose && p.autotune) std::fprintf(stderr, "[sapmg] autotune %.3f s\n", clk.lap());
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  return MG_OK;
}

// ------------------------------------------------------------ autotuner
// The launch shapes of the mixed form's multi-RHS kernels, chosen by timing
// every candidate on the context's own fields, P and D_c with nrhs_max
// right-hand sides (CUDA events on the context's stream, best of three after a
// warm-up launch), one knob at a time: the Schwarz pass's launch shape, the
// right-hand sides per transfer launch, and the coarse stencil's ring depth,
// CTAs per SM and right-hand sides per launch.  Every candidate of a knob
// computes each output with the same operations in the same order, so a tuned
// context gives the default's results bit for bit, except Schwarz shape 6
// (two threads per site), whose sums of a site's hops run in another order
// and agree to FP32 rounding.  The choice is cached per
// (lattice, N, nrhs_max, precision, levels) for the life of the process; a
// later context with the same key takes it without timing.
struct TuneChoice {
  int sap_shape, xfer_batch;
  CoarseTune ct;
};
static std::mutex g_tune_mutex;
static std::vector<std::pair<std::vector<int>, TuneChoice>> g_tune_cache;

static std::vector<int> tune_key(const mg_ctx* c) {
  const mg_params& p = c->p;
  return {p.dims[0], p.dims[1], p.dims[2], p.dims[3], p.n_vec[0], p.nrhs_max, p.precision, p.n_levels};
}

static int autotune(mg_ctx* c) {
  if (c->vt != P32 || c->p.n_levels < 2 || !c->Pv) return MG_OK;       // the knobs exist in the mixed form only
  const std::vector<int> key = tune_key(c);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& e : g_tune_cache)
      if (e.first == key) {
        c->sap_shape = e.second.sap_shape;
        c->xfer_batch = e.second.xfer_batch;
        c->ctune = e.second.ct;
        c->tune_source = 2;
        return MG_OK;
      }
  }
  const int R = c->p.nrhs_max;
  const size_t n = c->fine_n();
  // scratch vectors: the outer solver's flexible basis and w (free until the first solve)
  void* b = c->Z;
  void* z = c->w;
  SAPMG_CUDA_TRY(cudaMemsetAsync(b, 0, (size_t)R * n * 8, c->s));
  SAPMG_CUDA_TRY(cudaMemsetAsync(z, 0, (size_t)R * n * 8, c->s));
  cudaEvent_t e0, e1;
  SAPMG_CUDA_TRY(cudaEventCreate(&e0));
  SAPMG_CUDA_TRY(cudaEventCreate(&e1));
  int rc = MG_OK;
  auto timed = [&](auto&& fn) -> float {
    float best = 1e30f;
    if (rc != MG_OK) return best;
    if ((rc = fn()) != MG_OK) return best;
    for (int rep = 0; rep < 3 && rc == MG_OK; ++rep) {
      cudaEventRecord(e0, c->s);
      rc = fn();
      cudaEventRecord(e1, c->s);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
    return best;
  };
  // 1. Schwarz launch shape (the paired kernels: an even number of right-hand sides)
  if (R >= 2 && R % 2 == 0 && c->sap_shape >= 0) {
    int best_shape = c->sap_shape;
    float best = 1e30f;
    for (int shape = 0; shape <= 6; ++shape) {
      if (shape == 6 && c->prec == P32) continue;     // shape 6 holds FP16/BF16 fields only
      c->sap_shape = shape;
      const float ms = timed([&] { return smoother_sweeps(c, b, z, 1, R); });
      if (ms < best) { best = ms; best_shape = shape; }
    }
    c->sap_shape = best_shape;
  }
  // 2. right-hand sides per transfer launch (restriction and interpolation)
  if (R >= 2) {
    int best_b = c->xfer_batch;
    float best = 1e30f;
    for (int bsz : {16, 12, 8, 6, 4}) {
      if (bsz > R && bsz != 16) continue;
      c->xfer_batch = bsz;
      const float ms = timed([&] {
        const int r = transfer0(c, true, b, c->c1.b, R);
        return r != MG_OK ? r : transfer0(c, false, c->c1.b, z, R);
      });
      if (ms < best) { best = ms; best_b = bsz; }
    }
    c->xfer_batch = best_b;
  }
  // 3. coarse stencil: ring depth, CTAs per SM, right-hand sides per launch (the
  //    form the coarse GMRES uses: FP16 basis vectors when that basis exists)
  CoarseLevel& L = c->c1;
  if (L.Mh) {
    const bool xh = L.Vh != nullptr;
    const void* x = xh ? L.Vh : L.b;
    CoarseTune best_t = c->ctune;
    float best = 1e30f;
    for (int st : {2, 3}) {
      if (st == 3 && L.cg.n2 != 40) continue;
      for (int ctas : {0, 8, 4})
        for (int bsz : {16, 8, 4}) {
          if (bsz > R && bsz != 16) continue;
          c->ctune = CoarseTune{bsz, st, ctas};
          const float ms = timed([&] { return coarse_apply(c, L, x, L.w, R, xh); });
          if (ms < best) { best = ms; best_t = c->ctune; }
        }
    }
    c->ctune = best_t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MG_OK) return rc;
  TRY(check_device_error(c));
  c->tune_source = 1;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune_cache.push_back({key, TuneChoice{c->sap_shape, c->xfer_batch, c->ctune}});
  return MG_OK;
}

// canonical <-> blocked staging for the component entry points
static int stage_in(mg_ctx* c, const void* in, int prec, bool blocked, int nrhs, const void** out_ptr) {
  if (blocked) { *out_ptr = in; return MG_OK; }
  const int t = prec == P64 ? P64 : P32;
  TRY(launch_pack_spinor(t, in, t, c->io_a, c->g, nrhs, c->s));
  *out_ptr = c->io_a;
  return MG_OK;
}

}  // namespace sapmg

// ------------------------------------------------------------ no-allocation coarse solve
// Scratch of mg_coarse_solve_noalloc: a fixed array in the library's own device
// memory (every device that loads the library holds it until the process
// exits), so that this entry point never allocates.  Host code cannot use the
// symbol as an address; its device address is looked up once per device.
constexpr size_t kNoAllocBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];
static void* g_noalloc_addr[64] = {};
static std::mutex g_noalloc_mutex;

static int noalloc_scratch(void** out) {
  int dev = 0;
  SAPMG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(MG_ERR_ARG, "device index beyond the no-alloc table");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    SAPMG_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return MG_OK;
}

// ------------------------------------------------------------ saved set-ups
// File layout (little-endian, as the host writes it): 8-byte magic, then the
// int32 header below, the doubles m0 and c_sw, the int64 counts of complex
// numbers in the level-0 and level-1 vector sets, the FP64 vectors (level 0:
// the locally orthonormal test vectors, N0 x V x 12 in the blocked layout;
// level 1 when there are three levels: N1 x n1), and an FNV-1a 64-bit hash of
// everything before it.
static const char kSaveMagic[8] = {'S', 'A', 'P', 'M', 'G', 'S', 'U', '1'};
struct SaveHeader {
  int32_t dims[4], antiperiodic_t, n_levels, n_vec[2], agg2[4], sap_block2[4];
};

static uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < n; ++i) { h ^= p[i]; h *= 0x100000001b3ull; }
  return h;
}

static SaveHeader save_header(const mg_params& p) {
  SaveHeader h;
  std::memset(&h, 0, sizeof(h));
  for (int mu = 0; mu < 4; ++mu) {
    h.dims[mu] = p.dims[mu];
    h.agg2[mu] = p.n_levels == 3 ? p.agg2[mu] : 0;
    h.sap_block2[mu] = p.n_levels == 3 ? p.sap_block2[mu] : 0;
  }
  h.antiperiodic_t = p.antiperiodic_t;
  h.n_levels = p.n_levels;
  h.n_vec[0] = p.n_vec[0];
  h.n_vec[1] = p.n_levels == 3 ? p.n_vec[1] : 0;
  return h;
}

// Everything mg_setup does once the parameters are valid (also the body of
// mg_setup_load, whose context carries the saved vectors).
static int setup_context(mg_ctx* c, const double* U, double c_sw, double m0, const mg_params* p) {
  c->p = *p;
  c->g = make_geom(p->dims);
  c->s = (cudaStream_t)p->stream;
  c->prec = p->precision;
  c->vt = p->precision == MG_FP64 ? P64 : P32;
  c->pv_prec = p->precision == MG_BF16 ? P16 : p->precision;
  c->dc_prec = p->precision == MG_FP64 ? P64 : P32;
  c->coarse_reorth = std::getenv("SAPMG_COARSE_REORTH") ? std::atoi(std::getenv("SAPMG_COARSE_REORTH")) : 0;
  c->generic_coarse = std::getenv("SAPMG_GENERIC_COARSE") ? std::atoi(std::getenv("SAPMG_GENERIC_COARSE")) : 0;
  c->coarse_tf32 = std::getenv("SAPMG_COARSE_TF32") ? std::atoi(std::getenv("SAPMG_COARSE_TF32")) : 1;
  c->sap_shape = std::getenv("SAPMG_SAP_SHAPE") ? std::atoi(std::getenv("SAPMG_SAP_SHAPE")) : 0;
  c->dirac_pair = std::getenv("SAPMG_DIRAC_PAIR") ? std::atoi(std::getenv("SAPMG_DIRAC_PAIR")) : 1;
  c->graphs = std::getenv("SAPMG_GRAPHS") ? std::atoi(std::getenv("SAPMG_GRAPHS")) : 1;
  c->coarse_sap_mrhs = std::getenv("SAPMG_COARSE_SAP_MRHS") ? std::atoi(std::getenv("SAPMG_COARSE_SAP_MRHS")) : 1;
  c->coarse_sap_fp16 = std::getenv("SAPMG_COARSE_SAP_FP16") ? std::atoi(std::getenv("SAPMG_COARSE_SAP_FP16")) : 1;
  c->setup_fp32 = std::getenv("SAPMG_SETUP_FP32") ? std::atoi(std::getenv("SAPMG_SETUP_FP32")) : 1;
  c->fp64_on_fp32 = c->vt == P32 && std::getenv("SAPMG_FP64_ON_FP32") && std::atoi(std::getenv("SAPMG_FP64_ON_FP32"));
  c->xfer_batch = std::getenv("SAPMG_XFER_BATCH") ? std::max(1, std::atoi(std::getenv("SAPMG_XFER_BATCH"))) : 16;
  if (const char* ct = std::getenv("SAPMG_COARSE_TUNE")) {        // "batch,stages,ctas"
    int b = 16, st = 2, k = 0;
    if (std::sscanf(ct, "%d,%d,%d", &b, &st, &k) == 3) c->ctune = CoarseTune{std::max(1, b), st == 3 ? 3 : 2, k};
  }
  c->restrict_tf32 = std::getenv("SAPMG_RESTRICT_TF32") ? std::atoi(std::getenv("SAPMG_RESTRICT_TF32")) : 1;
  c->outer_dcgs2 = std::getenv("SAPMG_DCGS2") ? std::atoi(std::getenv("SAPMG_DCGS2")) : 1;
  c->coarse_fp16 = std::getenv("SAPMG_COARSE_FP16") ? std::atoi(std::getenv("SAPMG_COARSE_FP16")) : 1;
  c->m0 = m0;
  c->csw = c_sw;
  return do_setup(c, U);
}

// ============================================================ C-ABI
extern "C" {

int mg_default_params(mg_params* p) {
  if (!p) return fail(MG_ERR_ARG, "null params");
  std::memset(p, 0, sizeof(*p));
  p->n_levels = 1;
  for (int mu = 0; mu < 4; ++mu) { p->agg2[mu] = 2; p->sap_block2[mu] = 2; }
  p->n_vec[0] = 8;
  p->n_vec[1] = 8;
  p->setup_iters = 3;
  p->n_mr = 4;
  p->nu_post = 2;
  p->coarse_iters = 12;
  p->inner_iters = 8;
  p->fgmres_m = 20;
  p->tol = 1e-10;
  p->maxiter = 1000;
  p->precision = MG_FP64;
  p->nrhs_max = 1;
  p->seed = 1;
  return MG_OK;
}

const char* mg_last_error(void) { return g_err.c_str(); }

unsigned long mg_sizeof_params(void) { return (unsigned long)sizeof(mg_params); }

int mg_setup(const double* U, double c_sw, double m0, const mg_params* p, mg_ctx** out) {
  if (!U || !p || !out) return fail(MG_ERR_ARG, "null argument");
  *out = nullptr;
  TRY(validate(p));
  mg_ctx* c = new mg_ctx();
  const int rc = setup_context(c, U, c_sw, m0, p);
  if (rc < 0) {
    cudaStreamSynchronize(c->s);
    delete c;
    return rc;
  }
  *out = c;
  return MG_OK;
}

int mg_save(mg_ctx* c, const char* path) {
  if (!c || !path) return fail(MG_ERR_ARG, "bad argument");
  if (!c->V64 || c->p.n_levels < 2) return fail(MG_ERR_STATE, "no multilevel set-up to save");
  const SaveHeader h = save_header(c->p);
  const int64_t n0 = (int64_t)c->N0 * (int64_t)c->fine_n();
  const int64_t n1 = c->p.n_levels == 3 ? (int64_t)c->N1 * (int64_t)c->c1.n() : 0;
  std::vector<double2> v0((size_t)n0), w1((size_t)n1);
  SAPMG_CUDA_TRY(cudaMemcpyAsync(v0.data(), c->V64, (size_t)n0 * 16, cudaMemcpyDeviceToHost, c->s));
  if (n1) SAPMG_CUDA_TRY(cudaMemcpyAsync(w1.data(), c->W64, (size_t)n1 * 16, cudaMemcpyDeviceToHost, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(MG_ERR_ARG, std::string("cannot open ") + path + " for writing");
  uint64_t hash = 0xcbf29ce484222325ull;
  bool ok = true;
  auto put = [&](const void* d, size_t bytes) {
    hash = fnv1a(hash, d, bytes);
    ok = ok && std::fwrite(d, 1, bytes, f) == bytes;
  };
  put(kSaveMagic, sizeof(kSaveMagic));
  put(&h, sizeof(h));
  put(&c->m0, sizeof(double));
  put(&c->csw, sizeof(double));
  put(&n0, sizeof(n0));
  put(&n1, sizeof(n1));
  put(v0.data(), (size_t)n0 * 16);
  if (n1) put(w1.data(), (size_t)n1 * 16);
  ok = ok && std::fwrite(&hash, 1, sizeof(hash), f) == sizeof(hash);
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MG_OK : fail(MG_ERR_ARG, std::string("writing ") + path + " failed");
}

int mg_setup_load(const double* U, double c_sw, double m0, const mg_params* p, const char* path, mg_ctx** out) {
  if (!U || !p || !path || !out) return fail(MG_ERR_ARG, "null argument");
  *out = nullptr;
  TRY(validate(p));
  if (p->n_levels < 2) return fail(MG_ERR_ARG, "a saved set-up needs n_levels 2 or 3");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(MG_ERR_ARG, std::string("cannot open ") + path);
  uint64_t hash = 0xcbf29ce484222325ull;
  bool ok = true;
  auto get = [&](void* d, size_t bytes) {
    ok = ok && std::fread(d, 1, bytes, f) == bytes;
    if (ok) hash = fnv1a(hash, d, bytes);
  };
  char magic[8];
  SaveHeader h;
  double fm0 = 0, fcsw = 0;
  int64_t n0 = 0, n1 = 0;
  get(magic, sizeof(magic));
  get(&h, sizeof(h));
  get(&fm0, sizeof(double));
  get(&fcsw, sizeof(double));
  get(&n0, sizeof(n0));
  get(&n1, sizeof(n1));
  const SaveHeader want = save_header(*p);
  const Geom g = make_geom(p->dims);
  const int64_t want0 = (int64_t)p->n_vec[0] * g.V * 12;
  std::string why;
  if (!ok || std::memcmp(magic, kSaveMagic, sizeof(magic)) != 0) why = "not a saved set-up";
  else if (std::memcmp(&h, &want, sizeof(h)) != 0) why = "lattice, levels, N or blocking differ from the parameters";
  else if (fm0 != m0 || fcsw != c_sw) why = "m0 or c_sw differ from the saved set-up";
  else if (n0 != want0 || n1 < 0 || (p->n_levels == 2 && n1 != 0)) why = "vector counts do not match";
  std::vector<double2> v0, w1;
  if (why.empty()) {
    v0.resize((size_t)n0);
    w1.resize((size_t)n1);
    get(v0.data(), (size_t)n0 * 16);
    if (n1) get(w1.data(), (size_t)n1 * 16);
    uint64_t stored = 0;
    const uint64_t computed = hash;
    ok = ok && std::fread(&stored, 1, sizeof(stored), f) == sizeof(stored);
    if (!ok) why = "the file is truncated";
    else if (stored != computed) why = "checksum mismatch (the file is corrupted)";
  }
  std::fclose(f);
  if (!why.empty()) return fail(MG_ERR_ARG, std::string(path) + ": " + why);
  mg_ctx* c = new mg_ctx();
  c->load_v0 = &v0;
  c->load_w1 = n1 ? &w1 : nullptr;
  const int rc = setup_context(c, U, c_sw, m0, p);
  c->load_v0 = c->load_w1 = nullptr;
  if (rc < 0) {
    cudaStreamSynchronize(c->s);
    delete c;
    return rc;
  }
  *out = c;
  return MG_OK;
}

void mg_destroy(mg_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->s);
  delete c;
}

int dirac_apply(mg_ctx* c, const void* in, void* out, int prec, int nrhs) {
  if (!c || !in || !out || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  const bool blocked = (prec & MG_BLOCKED) != 0;
  const bool dag = (prec & MG_DAGGER) != 0;
  const bool emul = (prec & MG_FP64_ON_FP32) != 0;
  prec &= 0xff;
  if (prec < MG_FP64 || prec > MG_BF16) return fail(MG_ERR_ARG, "unknown precision");
  if (emul && (prec != MG_FP64 || dag)) return fail(MG_ERR_ARG, "MG_FP64_ON_FP32 goes with MG_FP64 and without MG_DAGGER");
  if (dag && prec != MG_FP64 && prec != MG_FP32) return fail(MG_ERR_ARG, "D^dagger is applied in MG_FP64 or MG_FP32");
  if (dag && prec == MG_FP32 && !c->U32) return fail(MG_ERR_STATE, "requested precision not set up in this context");
  if (!blocked && nrhs > c->p.nrhs_max) return fail(MG_ERR_ARG, "nrhs exceeds nrhs_max for canonical layout");
  const int t = prec == P64 ? P64 : P32;
  const void* src;
  TRY(stage_in(c, in, prec, blocked, nrhs, &src));
  void* dst = blocked ? out : c->io_b;
  if (dag)
    TRY(cgn_dirac(c, prec, dst, src, nrhs, true, nullptr));
  else
    TRY(fine_dirac(c, emul ? P64E : prec, dst, src, nrhs));
  if (!blocked) TRY(launch_unpack_spinor(t, dst, t, out, c->g, nrhs, c->s));
  return MG_OK;
}

int sap_smooth(mg_ctx* c, const void* b, void* z, int n_sweeps, int prec, int nrhs) {
  if (!c || !b || !z || nrhs < 1 || n_sweeps < 0) return fail(MG_ERR_ARG, "bad argument");
  const bool blocked = (prec & MG_BLOCKED) != 0;
  prec &= 0xff;
  if (prec != c->prec) return fail(MG_ERR_STATE, "sap_smooth runs in the context's smoother precision");
  if (!blocked && nrhs > c->p.nrhs_max) return fail(MG_ERR_ARG, "nrhs exceeds nrhs_max for canonical layout");
  const int t = prec == P64 ? P64 : P32;
  if (blocked) return smoother_sweeps(c, b, z, n_sweeps, nrhs);
  TRY(launch_pack_spinor(t, b, t, c->io_a, c->g, nrhs, c->s));
  TRY(launch_pack_spinor(t, z, t, c->io_b, c->g, nrhs, c->s));
  TRY(smoother_sweeps(c, c->io_a, c->io_b, n_sweeps, nrhs));
  return launch_unpack_spinor(t, c->io_b, t, z, c->g, nrhs, c->s);
}

int mg_solve(mg_ctx* c, const double* b, double* z, int nrhs, mg_solve_info* info) {
  if (!c || !b || !z || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t n = c->fine_n();
  int status = MG_OK, it_sum = 0, rs_sum = 0;
  double worst = 0;
  c->hist.clear();
  for (int r0 = 0; r0 < nrhs; r0 += c->p.nrhs_max) {
    const int R = std::min(c->p.nrhs_max, nrhs - r0);
    c->hist_r0 = r0;
    TRY(launch_pack_spinor(P64, b + (size_t)r0 * n * 2, P64, c->b64, c->g, R, c->s));
    int it = 0, rs = 0;
    double rel = 0;
    const int rc = solve_batch(c, R, it, rs, rel);
    if (rc < 0) return rc;
    if (rc == MG_NOT_CONVERGED) status = MG_NOT_CONVERGED;
    TRY(launch_unpack_spinor(P64, c->x64, P64, z + (size_t)r0 * n * 2, c->g, R, c->s));
    it_sum += it * R;
    rs_sum += rs;
    worst = std::max(worst, rel);
  }
  TRY(check_device_error(c));
  if (info) {
    info->iterations = it_sum;
    info->restarts = rs_sum;
    info->relres = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->precond_seconds = 0;
  }
  return status;
}

int mg_cgn_solve(mg_ctx* c, const double* b, double* z, int nrhs, int prec, double tol, int maxiter,
                 mg_solve_info* info) {
  if (!c || !b || !z || nrhs < 1 || !(tol > 0) || maxiter < 1) return fail(MG_ERR_ARG, "bad argument");
  const int type = prec == MG_FP64 ? P64 : (prec == MG_FP32 ? P32 : -1);
  if (type < 0) return fail(MG_ERR_ARG, "CGN runs in MG_FP64 or MG_FP32");
  if (type == P32 && (!c->U32 || !c->A32)) return fail(MG_ERR_STATE, "the FP32 form needs a mixed-precision context");
  TRY(cgn_alloc(c));
  const auto t0 = std::chrono::steady_clock::now();
  const size_t n = c->fine_n();
  int status = MG_OK, it_sum = 0, up_sum = 0;
  double worst = 0;
  c->hist.clear();
  for (int r0 = 0; r0 < nrhs; r0 += c->p.nrhs_max) {
    const int R = std::min(c->p.nrhs_max, nrhs - r0);
    c->hist_r0 = r0;
    TRY(launch_pack_spinor(P64, b + (size_t)r0 * n * 2, P64, c->b64, c->g, R, c->s));
    int it = 0, up = 0;
    double rel = 0;
    const int rc = cgn_batch(c, type, R, tol, maxiter, it, up, rel);
    if (rc < 0) return rc;
    if (rc == MG_NOT_CONVERGED) status = MG_NOT_CONVERGED;
    TRY(launch_unpack_spinor(P64, c->x64, P64, z + (size_t)r0 * n * 2, c->g, R, c->s));
    it_sum += it;
    up_sum += up;
    worst = std::max(worst, rel);
  }
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  if (info) {
    info->iterations = it_sum;
    info->restarts = up_sum;
    info->relres = worst;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->precond_seconds = 0;
  }
  return status;
}

int mg_harmonic_ritz(int m, const double* hbar, double* theta, double* y) {
  const int rc = harmonic_ritz_host(m, hbar, theta, y);
  if (rc == MG_ERR_ARG) return fail(rc, "bad argument");
  if (rc == MG_ERR_NONFINITE) return fail(rc, "the harmonic Ritz problem did not converge or is singular");
  return rc;
}

int mg_eigh(int n, const double* a, double* w, double* v) {
  const int rc = eigh_host(n, a, w, v);
  if (rc == MG_ERR_ARG) return fail(rc, "bad argument");
  return rc;
}

int mg_pack_spinor(mg_ctx* c, const void* canonical, void* blocked, int prec, int nrhs) {
  if (!c || !canonical || !blocked || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  const int t = (prec & 0xff) == P64 ? P64 : P32;
  return launch_pack_spinor(t, canonical, t, blocked, c->g, nrhs, c->s);
}

int mg_unpack_spinor(mg_ctx* c, const void* blocked, void* canonical, int prec, int nrhs) {
  if (!c || !canonical || !blocked || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  const int t = (prec & 0xff) == P64 ? P64 : P32;
  return launch_unpack_spinor(t, blocked, t, canonical, c->g, nrhs, c->s);
}

int mg_clover_export(mg_ctx* c, double* out) {
  if (!c || !out) return fail(MG_ERR_ARG, "bad argument");
  return launch_clover_export(c->g, c->A64, out, c->s);
}

int mg_get_vectors(mg_ctx* c, int level, double* out) {
  if (!c || !out) return fail(MG_ERR_ARG, "bad argument");
  if (level == 0 && c->V64) return launch_unpack_spinor(P64, c->V64, P64, out, c->g, c->N0, c->s);
  if (level == 1 && c->W64) {
    SAPMG_CUDA_TRY(cudaMemcpyAsync(out, c->W64, (size_t)c->N1 * c->c1.n() * 16, cudaMemcpyDeviceToDevice, c->s));
    return MG_OK;
  }
  return fail(MG_ERR_STATE, "no test vectors on that level");
}

static CoarseLevel* coarse_level(mg_ctx* c, int level) {
  if (level == 1 && c->c1.M) return &c->c1;
  if (level == 2 && c->c2.M) return &c->c2;
  return nullptr;
}

int mg_get_coarse_op(mg_ctx* c, int level, double* out) {
  if (!c || !out) return fail(MG_ERR_ARG, "bad argument");
  CoarseLevel* L = coarse_level(c, level);
  if (!L) return fail(MG_ERR_STATE, "no coarse operator on that level");
  return launch_coarse_export(P64, L->cg, L->M64, out, c->s);
}

int mg_restrict(mg_ctx* c, int level, const void* in, void* out, int prec) {
  return mg_restrict_batch(c, level, in, out, prec, 1);
}

int mg_prolong(mg_ctx* c, int level, const void* in, void* out, int prec) {
  return mg_prolong_batch(c, level, in, out, prec, 1);
}

int mg_restrict_batch(mg_ctx* c, int level, const void* in, void* out, int prec, int nrhs) {
  if (!c || !in || !out || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  if (nrhs > c->p.nrhs_max) return fail(MG_ERR_ARG, "more right-hand sides than nrhs_max");
  const bool blocked = (prec & MG_BLOCKED) != 0;
  prec &= 0xff;
  if ((prec == P64) != (c->prec == P64)) return fail(MG_ERR_STATE, "precision does not match the context");
  if (level == 1 && c->W) {
    ProfScope ps(c->prof, FAM_RESTRICT, c->s);
    return launch_transfer1(true, c->vt, c->c1.cg, c->agg1, in, out, c->W, c->N1, nrhs, c->s);
  }
  if (level != 0 || !c->Pv) return fail(MG_ERR_STATE, "no interpolation on that level");
  const void* src;
  TRY(stage_in(c, in, prec, blocked, nrhs, &src));
  ProfScope ps(c->prof, FAM_RESTRICT, c->s);
  return transfer0(c, true, src, out, nrhs);
}

int mg_prolong_batch(mg_ctx* c, int level, const void* in, void* out, int prec, int nrhs) {
  if (!c || !in || !out || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  if (nrhs > c->p.nrhs_max) return fail(MG_ERR_ARG, "more right-hand sides than nrhs_max");
  const bool blocked = (prec & MG_BLOCKED) != 0;
  prec &= 0xff;
  if ((prec == P64) != (c->prec == P64)) return fail(MG_ERR_STATE, "precision does not match the context");
  if (level == 1 && c->W) {
    ProfScope ps(c->prof, FAM_PROLONG, c->s);
    return launch_transfer1(false, c->vt, c->c1.cg, c->agg1, in, out, c->W, c->N1, nrhs, c->s);
  }
  if (level != 0 || !c->Pv) return fail(MG_ERR_STATE, "no interpolation on that level");
  void* dst = blocked ? out : c->io_b;
  {
    ProfScope ps(c->prof, FAM_PROLONG, c->s);
    TRY(transfer0(c, false, in, dst, nrhs));
  }
  if (!blocked) {
    const int t = prec == P64 ? P64 : P32;
    TRY(launch_unpack_spinor(t, dst, t, out, c->g, nrhs, c->s));
  }
  return MG_OK;
}

int mg_coarse_apply(mg_ctx* c, int level, const void* in, void* out, int prec) {
  return mg_coarse_apply_batch(c, level, in, out, prec, 1);
}

int mg_coarse_apply_batch(mg_ctx* c, int level, const void* in, void* out, int prec, int nrhs) {
  if (!c || !in || !out || nrhs < 1) return fail(MG_ERR_ARG, "bad argument");
  prec &= 0xff;
  CoarseLevel* L = coarse_level(c, level);
  if (!L) return fail(MG_ERR_STATE, "no coarse operator on that level");
  if ((prec == P64) != (c->prec == P64)) return fail(MG_ERR_STATE, "precision does not match the context");
  TRY(coarse_apply(c, *L, in, out, nrhs));
  return check_device_error(c);
}

int mg_coarse_solve(mg_ctx* c, int level, const void* in, void* out, int prec) {
  if (!c || !in || !out) return fail(MG_ERR_ARG, "bad argument");
  prec &= 0xff;
  CoarseLevel* L = coarse_level(c, level);
  if (!L) return fail(MG_ERR_STATE, "no coarse operator on that level");
  if ((prec == P64) != (c->prec == P64)) return fail(MG_ERR_STATE, "precision does not match the context");
  const size_t bytes = L->n() * complex_bytes(c->vt);
  SAPMG_CUDA_TRY(cudaMemcpyAsync(L->b, in, bytes, cudaMemcpyDeviceToDevice, c->s));
  TRY(coarse_solve(c, level, 1));
  SAPMG_CUDA_TRY(cudaMemcpyAsync(out, L->x, bytes, cudaMemcpyDeviceToDevice, c->s));
  return check_device_error(c);
}

int mg_coarse_solve_noalloc(mg_ctx* c, int level, const void* in, void* out, int prec) {
  if (!c || !in || !out) return fail(MG_ERR_ARG, "bad argument");
  prec &= 0xff;
  if (level != 1 || !c->c1.M) return fail(MG_ERR_STATE, "no coarse operator on that level");
  if (c->p.n_levels != 2)
    return fail(MG_ERR_STATE, "the no-alloc coarse solve serves two-level contexts only (on a three-level "
                              "context level 1 is solved by flexible GMRES with the level-1 cycle)");
  if ((prec == P64) != (c->prec == P64)) return fail(MG_ERR_STATE, "precision does not match the context");
  CoarseLevel& L = c->c1;
  const size_t n = L.n();
  const int vt = c->vt;
  const size_t eb = complex_bytes(vt);
  const int k = c->p.coarse_iters;
  // carve the scratch: partial sums | H | H scratch | ||b||^2 | y | basis V (k+1) | w
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t o_part = 0;
  const size_t o_h = o_part + up(sizeof(double2) * kPartialDouble2);
  const size_t o_tmp = o_h + up(sizeof(double2) * 33 * 33);
  const size_t o_beta = o_tmp + up(sizeof(double2) * 33 * 33);
  const size_t o_y = o_beta + up(sizeof(double2));
  const size_t o_v = o_y + up(sizeof(double2) * 33);
  const size_t o_w = o_v + up((size_t)(k + 1) * n * eb);
  const size_t need = o_w + up(n * eb);
  if (need > kNoAllocBytes)
    return fail(MG_ERR_ARG, "coarse system too large for the no-alloc scratch (" + std::to_string(need) +
                                " bytes needed, limit " + std::to_string(kNoAllocBytes) + ")");
  void* base = nullptr;
  TRY(noalloc_scratch(&base));
  char* sb = (char*)base;
  double2* partial = (double2*)(sb + o_part);
  double2* H = (double2*)(sb + o_h);
  double2* tmp = (double2*)(sb + o_tmp);
  double2* beta2 = (double2*)(sb + o_beta);
  double2* y = (double2*)(sb + o_y);
  void* V = sb + o_v;
  void* w = sb + o_w;
  auto Vj = [&](int j) { return (void*)((char*)V + (size_t)j * n * eb); };
  const BVec bv = bvec(n, 1, n);
  // the same fixed-step GMRES as the cycle's coarse solve, on the scratch buffers
  {
    const void* v1[1] = {in};
    TRY(blas_multidot(vt, bv, v1, 1, in, beta2, 1, 0, nullptr, partial, c->s));
  }
  TRY(blas_normalize(vt, bv, in, Vj(0), beta2, 1, nullptr, 0, c->s));
  std::vector<const void*> vl;
  for (int j = 0; j < k; ++j) {
    TRY(coarse_apply(c, L, Vj(j), w, 1));
    vl.push_back(Vj(j));
    double2* hcol = H + (size_t)j * 33;
    TRY(blas_multidot(vt, bv, vl.data(), j + 1, w, hcol, 33 * 33, 0, nullptr, partial, c->s));
    TRY(blas_multiaxpy(vt, bv, w, vl.data(), j + 1, hcol, 33 * 33, -1.0, c->s));
    if (c->coarse_reorth) {
      TRY(blas_multidot(vt, bv, vl.data(), j + 1, w, hcol, 33 * 33, 1, tmp, partial, c->s));
      TRY(blas_multiaxpy(vt, bv, w, vl.data(), j + 1, tmp, 33 * 33, -1.0, c->s));
    }
    const void* wl[1] = {w};
    TRY(blas_multidot(vt, bv, wl, 1, w, tmp + 40, 33 * 33, 0, nullptr, partial, c->s));
    TRY(blas_normalize(vt, bv, w, Vj(j + 1), tmp + 40, 33 * 33, hcol + j + 1, 33 * 33, c->s));
  }
  TRY(blas_hessenberg_solve(H, 33, 33 * 33, k, beta2, y, 33, 1, c->s));
  SAPMG_CUDA_TRY(cudaMemsetAsync(out, 0, n * eb, c->s));     // the result starts from zero
  TRY(blas_multiaxpy(vt, bv, out, vl.data(), k, y, 33, 1.0, c->s));
  return check_device_error(c);
}

int mg_precondition(mg_ctx* c, const void* v, void* z, int prec) {
  if (!c || !v || !z) return fail(MG_ERR_ARG, "bad argument");
  const bool blocked = (prec & MG_BLOCKED) != 0;
  prec &= 0xff;
  if ((prec == P64) != (c->prec == P64)) return fail(MG_ERR_STATE, "precision does not match the context");
  const void* src;
  TRY(stage_in(c, v, prec, blocked, 1, &src));
  void* dst = blocked ? z : c->io_b;
  TRY(cycle(c, src, dst, 1));
  if (!blocked) {
    const int t = prec == P64 ? P64 : P32;
    TRY(launch_unpack_spinor(t, dst, t, z, c->g, 1, c->s));
  }
  return MG_OK;
}

// ------------------------------------------------------------ learned set-up
static int net_state(mg_ctx* c, int a, int b) {
  if (!c) return fail(MG_ERR_ARG, "bad argument");
  if (!c->U32) return fail(MG_ERR_STATE, "the network needs a mixed-form context (FP32 links)");
  if (a < 1 || b < 1 || a > 64 || b > 64) return fail(MG_ERR_ARG, "channel counts must be in 1..64");
  return MG_OK;
}

int mg_net_layer_forward(mg_ctx* c, int cin, int cout, const void* W, const void* x, void* y) {
  TRY(net_state(c, cin, cout));
  if (!W || !x || !y) return fail(MG_ERR_ARG, "bad argument");
  return launch_gconv_forward(c->g, c->U32, W, x, y, cin, cout, c->s);
}

int mg_net_layer_forward_bf16(mg_ctx* c, int cin, int cout, const void* W, const void* x, void* y) {
  TRY(net_state(c, cin, cout));
  if (!W || !x || !y) return fail(MG_ERR_ARG, "bad argument");
  if (c->prec != MG_BF16) return fail(MG_ERR_STATE, "BF16 inference needs a BF16 context (BF16 links)");
  return launch_gconv_forward_bf16(c->g, c->Us, W, x, y, cin, cout, c->s);
}

int mg_net_layer_backward(mg_ctx* c, int cin, int cout, const void* W, const void* x, const void* gy, void* gx,
                          void* gW) {
  TRY(net_state(c, cin, cout));
  if (!W || !x || !gy || (!gx && !gW)) return fail(MG_ERR_ARG, "bad argument");
  return launch_gconv_backward(c->g, c->U32, W, x, gy, gx, gW, cin, cout, c->s);
}

int mg_net_gate_forward(mg_ctx* c, int channels, const void* x, void* y) {
  TRY(net_state(c, channels, 1));
  if (!x || !y) return fail(MG_ERR_ARG, "bad argument");
  return launch_gate(c->g, x, nullptr, y, channels, c->s);
}

int mg_net_gate_backward(mg_ctx* c, int channels, const void* x, const void* gy, void* gx) {
  TRY(net_state(c, channels, 1));
  if (!x || !gy || !gx) return fail(MG_ERR_ARG, "bad argument");
  return launch_gate(c->g, x, gy, gx, channels, c->s);
}

int mg_net_loss(mg_ctx* c, const void* y, const void* t, void* gy, double* loss) {
  TRY(net_state(c, 1, 1));
  if (!y || !t || !gy || !loss) return fail(MG_ERR_ARG, "bad argument");
  const size_t n = c->fine_n();
  const BVec bv = bvec(n, 1, n);
  const Scal32 one = scal_all(1.0, 1), zero = scal_all(0.0, 1), minus = scal_all(-1.0, 1);
  TRY(blas_axpby2(P32, one, y, n, P32, zero, gy, n, n, 1, c->s));           // gy = y
  TRY(blas_axpby2(P32, minus, t, n, P32, one, gy, n, n, 1, c->s));          // gy = y - t
  TRY(dot_to(c, P32, bv, gy, gy, c->hd, 1));
  TRY(dot_to(c, P32, bv, t, t, c->hd + 1, 1));
  SAPMG_CUDA_TRY(cudaMemcpyAsync(c->hh, c->hd, 2 * sizeof(double2), cudaMemcpyDeviceToHost, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  const double dn = c->hh[0].x, tn = c->hh[1].x;
  if (!(tn > 0)) return fail(MG_ERR_ARG, "target vector is zero");
  *loss = dn / tn;
  const Scal32 sc = scal_all(2.0 / tn, 1);
  return blas_axpby2(P32, sc, gy, n, P32, zero, gy, n, n, 1, c->s);       // G = 2 (y - t) / ||t||^2
}

int mg_adam_step(mg_ctx* c, size_t n, float* p, const float* g, float* m, float* v, double lr, double beta1,
                 double beta2, double eps, int step) {
  if (!c || !p || !g || !m || !v) return fail(MG_ERR_ARG, "bad argument");
  return launch_adam(n, p, g, m, v, lr, beta1, beta2, eps, step, c->s);
}

int mg_set_profiling(mg_ctx* c, int mask) {
  if (!c) return fail(MG_ERR_ARG, "bad argument");
  c->prof.on = mask != 0;
  c->prof.mask = (mask == 1) ? 0xffffffffu : (unsigned)mask >> 1;
  return MG_OK;
}

long long mg_launch_count(void) { return g_launches.load(); }

int mg_set_wait_limit(mg_ctx* c, int spins) {
  if (!c) return fail(MG_ERR_ARG, "bad argument");
  const int v = spins < 0 ? kMaxSpins : spins;
  SAPMG_CUDA_TRY(cudaMemcpyAsync(c->dev_err + 1, &v, sizeof(int), cudaMemcpyHostToDevice, c->s));
  SAPMG_CUDA_TRY(cudaStreamSynchronize(c->s));
  return MG_OK;
}

int mg_get_tuning(mg_ctx* c, int* out) {
  if (!c || !out) return fail(MG_ERR_ARG, "bad argument");
  out[0] = c->tune_source;
  out[1] = c->sap_shape;
  out[2] = c->xfer_batch;
  out[3] = c->ctune.stages;
  out[4] = c->ctune.ctas;
  out[5] = c->ctune.batch;
  return MG_OK;
}

int mg_get_history(mg_ctx* c, double* out, int max_entries) {
  if (!c || max_entries < 0) return fail(MG_ERR_ARG, "bad argument");
  const int n = (int)(c->hist.size() / 3);
  if (out) std::memcpy(out, c->hist.data(), sizeof(double) * 3 * (size_t)std::min(n, max_entries));
  return n;
}

int mg_sync(mg_ctx* c) {
  if (!c) return fail(MG_ERR_ARG, "bad argument");
  return check_device_error(c);
}

int mg_debug_check(long long value, long long bound) {
#ifdef MG_DEBUG
  dbg::selftest_kernel<<<1, 1>>>(value, bound);
  count_launches(1);
  SAPMG_CUDA_TRY(cudaGetLastError());
  return MG_OK;
#else
  (void)value;
  (void)bound;
  return fail(MG_ERR_STATE, "mg_debug_check needs the MG_DEBUG build");
#endif
}

long long mg_debug_failures(void) {
#ifdef MG_DEBUG
  SAPMG_CUDA_TRY(cudaDeviceSynchronize());
  std::string msg;
  const long long n = dbg::collect(&msg);
  if (n < 0) return fail(MG_ERR_CUDA, "could not read the device-side index checks");
  if (n > 0) g_err = msg;
  return n;
#else
  return -1;
#endif
}

int mg_probe_peaks(void* stream, double* fp32_tflops, double* fp32x2_tflops, double* smem_gbs) {
  if (!fp32_tflops || !fp32x2_tflops || !smem_gbs) return fail(MG_ERR_ARG, "bad argument");
  return probe_peaks((cudaStream_t)stream, fp32_tflops, fp32x2_tflops, smem_gbs);
}

int mg_get_profile(mg_ctx* c, int family, long long* launches, double* ms) {
  if (!c || family < 0 || family >= FAM_N) return fail(MG_ERR_ARG, "bad argument");
  c->prof.drain();
  if (launches) *launches = c->prof.launches[family];
  if (ms) *ms = c->prof.ms[family];
  return MG_OK;
}

int mg_get_profile_bytes(mg_ctx* c, int family, double* bytes) {
  if (!c || !bytes || family < 0 || family >= FAM_N) return fail(MG_ERR_ARG, "bad argument");
  c->prof.drain();
  *bytes = c->prof.bytes[family];
  return MG_OK;
}

int mg_reset_profile(mg_ctx* c) {
  if (!c) return fail(MG_ERR_ARG, "bad argument");
  c->prof.drain();
  for (int f = 0; f < FAM_N; ++f) { c->prof.launches[f] = 0; c->prof.ms[f] = 0; c->prof.bytes[f] = 0; }
  return MG_OK;
}

}  // extern "C"
