// Device-side index checks of the MG_DEBUG build.
//
// Built with -DMG_DEBUG (libsapmg_debug.so), the kernels test the indices they
// compute -- neighbour sites and blocks, the blocks of a colour, coarse sites
// and their neighbours, aggregates, kernel block indices -- and the alignment of
// every bulk copy before they use them.  A failed check never traps: it
// records itself in a per-translation-unit device word (the first failure's
// kind, source line and value, and a count) and the kernel goes on with an
// in-range substitute (index 0, or a bulk copy skipped with its transaction
// bytes completed by hand), so the control flow, every barrier and every wait
// stay as in the release build.  The host reads the records at the next
// synchronising call (MG_ERR_BOUNDS) or through mg_debug_failures().  In the
// release build every check compiles to nothing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sapmg {
namespace dbg {

enum Kind : int {
  kNeighbourBlock = 1,  // fine neighbour block outside [0, nblocks)
  kNeighbourSite,       // fine neighbour site out of range (in its block, or canonical)
  kColourBlock,         // k-th block of a colour outside [0, nblocks)
  kBlock,               // a kernel's own block (box, or blocked site) index out of range
  kCoarseSite,          // coarse site outside [0, nsites)
  kCoarseNeighbour,     // coarse neighbour site outside [0, nsites)
  kAggregate,           // aggregate (or aggregate row) out of range
  kBulkCopy,            // bulk copy address or size not a multiple of 16 bytes
  kKinds
};

// Host side (defined in solver.cu in every build): the name of a kind, and the
// registry of the per-unit readers (each reader copies its unit's first record
// and failure count to the host and clears them).
const char* kind_name(int kind);
typedef int (*Reader)(unsigned long long* first, unsigned long long* fails);
int add_reader(Reader r, const char* unit);

}  // namespace dbg
}  // namespace sapmg

#ifdef MG_DEBUG
namespace sapmg {
namespace dbg {

// first failure: kind << 56 | (line & 0xffffff) << 32 | low 32 bits of the value
static __device__ unsigned long long g_first;
static __device__ unsigned long long g_fails;

static __device__ __noinline__ void record(int kind, int line, long long value) {
  const unsigned long long rec = ((unsigned long long)kind << 56) |
                                 ((unsigned long long)(line & 0xffffff) << 32) | (unsigned long long)(uint32_t)value;
  atomicCAS(&g_first, 0ull, rec);
  atomicAdd(&g_fails, 1ull);
}

__device__ __forceinline__ bool in_range(int kind, int line, long long v, long long n) {
  if (v >= 0 && v < n) return true;
  record(kind, line, v);
  return false;
}

static int read_unit(unsigned long long* first, unsigned long long* fails) {
  if (cudaMemcpyFromSymbol(first, g_first, sizeof(*first)) != cudaSuccess) return -1;
  if (cudaMemcpyFromSymbol(fails, g_fails, sizeof(*fails)) != cudaSuccess) return -1;
  if (*fails) {
    const unsigned long long zero = 0;
    if (cudaMemcpyToSymbol(g_first, &zero, sizeof(zero)) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(g_fails, &zero, sizeof(zero)) != cudaSuccess) return -1;
  }
  return 0;
}
static const int g_reader_slot = add_reader(read_unit, __BASE_FILE__);

}  // namespace dbg
}  // namespace sapmg

// true if 0 <= v < n; otherwise records the failure and gives false
#define MG_CHECK(kind, v, n) ::sapmg::dbg::in_range(::sapmg::dbg::kind, __LINE__, (long long)(v), (long long)(n))
// v if 0 <= v < n, otherwise 0 (after recording the failure); v is evaluated twice
#define MG_CLAMP(kind, v, n) (MG_CHECK(kind, v, n) ? (v) : 0)
#else
#define MG_CHECK(kind, v, n) true
#define MG_CLAMP(kind, v, n) (v)
#endif
