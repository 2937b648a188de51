// internal.h -- host-side internals shared by the translation units of libmpk.
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/mpk.h"

namespace mpk {

// Error reporting (thread-local last error; see mpk_last_error).
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
// Multi-component vectors (and complex matrix values) are read and written with 16-byte accesses:
// every entry point refuses a misaligned device pointer (MPK_INVALID_ARG) before any launch.
inline bool misaligned(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }
#define MPK_CUDA(call)                                                                      \
  do {                                                                                      \
    cudaError_t err_ = (call);                                                              \
    if (err_ != cudaSuccess)                                                                \
      return ::mpk::fail(MPK_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(err_)); \
  } while (0)

struct Csr {  // device CSR view
  int n = 0, nnz = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const double* val = nullptr;  // c doubles per entry
  int cplx = 0;
  const int* order = nullptr;   // SpMV: thread t computes row order[t] (nullptr: row t)
  bool mm = false;              // SpMV with the entries promoted to the vectors' w components
};

// Scalar slots of a solve: each slot holds one number (up to 8 doubles).
enum Slot : int {
  S_ONE = 0, S_MONE, S_ZERO,
  S_RHO, S_RHO_OLD, S_SIG, S_ALPHA, S_NALPHA, S_NCALPHA, S_BETA, S_CBETA,
  S_OMEGA, S_NOMEGA, S_ZETA, S_NZETA, S_ETA, S_NETA,
  S_NORM,           // last ||r|| (number; leading component used)
  S_R0N, S_TOL,     // plain doubles in component 0
  S_D0, S_D1, S_D2, S_D3, S_D4, S_D5,  // dot outputs
  S_COUNT
};
constexpr int kSlotDoubles = 8;
// Integer state of a solve on the device.
// ST_PERIOD: the replacement period (0: off).  ST_NOCHK / ST_NOREPL: 0 while the true-residual
// check / the replacement copy of the current iteration is to run (the gates of those launches),
// else 1.  ST_CHECK: 1 periodic check, 2 the recursive norm passed the test; ST_CHK_IT: the
// iteration checked; ST_NREP: replacements so far.
enum StateIdx : int {
  ST_DONE = 0, ST_STATUS, ST_ITERS, ST_IT, ST_MAXIT, ST_FLAGS,
  ST_PERIOD, ST_NOCHK, ST_NOREPL, ST_CHECK, ST_CHK_IT, ST_NREP,
  ST_TRUEKNOWN,  // 1: the solve ended on an accepted check, whose true norm is already in S_D4
  ST_COUNT
};

// Phases of the single-thread scalar kernel.
enum Phase : int {
  PH_INIT = 0,    // after ||r0||^2 in S_D0: r0 norm, tolerance, hist[0], early exit
  PH_RHO,         // after <r~,r> (or BiCG's <z~,r>) in S_D0
  PH_SIG,         // after the alpha denominator in S_D0
  PH_OMEGA,       // BiCGSTAB: <t,s>, <t,t> in S_D0, S_D1
  PH_ZETA,        // GPBiCG: cc, ct, yy, yt, cy, yc in S_D0..S_D5
  PH_NORM,        // after ||r||^2 in S_D0: history, convergence, breakdown checks
  PH_BETA,        // BiCG / GPBiCG: after the new rho in S_D0
  PH_STORE_RHO,   // store S_D0 as rho (BiCG / GPBiCG initialisation)
  PH_TRUE,        // ||b - A x|| from S_D5 (final true residual)
  PH_TRUECHK      // replacement rule: ||b - A x_k||^2 in S_D5 (true_res_period)
};

struct DotWs {           // workspace of the fixed-order reduction
  double* partial = nullptr;  // dot_partial_doubles(n) doubles
  unsigned* counter = nullptr;
};
constexpr int kMaxDots = 6;
// Fixed summation order of the inner products: leaves of kDotLeaf consecutive products, one leaf
// per thread of a kDotBlockLeaves-thread block; dot_blocks(n) blocks for n entries.
constexpr int kDotLeaf = 16;
constexpr int kDotBlockLeaves = 256;
inline int dot_blocks(int n) {
  const int m = (n + kDotLeaf - 1) / kDotLeaf;
  return m < 1 ? 1 : (m + kDotBlockLeaves - 1) / kDotBlockLeaves;
}
// doubles of per-block partials needed by up to kMaxDots simultaneous inner products of length n
inline size_t dot_partial_doubles(int n) { return ((size_t)(n > 0 ? n : 1) + 4095) / 4096 * kMaxDots * 8; }

struct IluHandleView;  // forward
}  // namespace mpk
struct mpk_ilu;
namespace mpk {

// nsys independent systems stored as consecutive row blocks of one block-diagonal matrix.  Each
// system has its own scalar slots (S + s * kSysDoubles) and integer state (st + s * ST_COUNT); a
// system whose ST_DONE is set keeps its iterate and residual (its rows are skipped).
constexpr int kSysDoubles = S_COUNT * kSlotDoubles;
struct Batch {
  int nsys = 1;
  const int* sysid = nullptr;        // row -> system
  const int* roff = nullptr;         // nsys + 1 row offsets
  const int* boff = nullptr;         // nsys + 1: first inner-product block of each system
  const int* bsys = nullptr;         // inner-product block -> system
  int nblocks = 0;                   // boff[nsys]
  const int* st = nullptr;           // per-system state (nullptr: skip no system)
  int gate = -1;                     // >= 0: also skip systems whose st[gate] is nonzero
  unsigned long long* absmax = nullptr;  // nsys scale accumulators of the binary32 substitutions
};

// Level order of one triangle for the chunk dataflow (see chunk_rows).
struct LevelOrder {
  const int* perm = nullptr;     // position -> row (-1: padding); levels padded to 32 rows
  const int* pos = nullptr;      // row -> position
  int* flags = nullptr;          // per chunk: epoch of the last pass that finished it
  const int* nchunks = nullptr;  // device int: number of chunks
  const int* lstart = nullptr;   // nlev + 1: first chunk of every level (the last: nchunks)
  int nlev = 0;
};

// A dependency-respecting row order of one triangle (see syncfree_rows).
struct Order {
  const int* perm = nullptr;  // position -> row (-1: empty position)
  const int* pos = nullptr;   // row -> position
  int npos = 0;               // number of positions
};

// Kernel launchers for one (w, c) pair.  `done` (nullable) is the device flag that turns every
// launch into a no-op once a solve has finished.
struct Ops {
  int w, cp;
  // bt (nullable): rows of systems whose ST_DONE is set are skipped
  void (*spmv)(const Csr& A, const double* x, double* y, const double* b_or_null, const int* done, const Batch* bt,
               cudaStream_t s);
  void (*dots)(int n, int k, const double* const* a, const double* const* b, double* const* out, const DotWs& ws,
               const int* done, cudaStream_t s);
  // per-system inner products of a batch: system s's k-th result goes to its slot slot0 + k (same
  // summation order as `dots` on the system alone); partial: nblocks * k entries, counters: nsys
  void (*dots_seg)(const Batch& bt, int k, const double* const* a, const double* const* b, double* S, int slot0,
                   double* partial, unsigned* counters, const int* done, cudaStream_t s);
  // y = sum_k coef_k * v_k evaluated left to right; coef == nullptr means exactly 1
  // copy_at_first (nullable, the solve's int state): y = v_0 when the iteration counter is 1
  // bt (nullable): coefficients per system (coef_k + s * kSysDoubles), done systems skipped
  void (*lincomb)(int n, double* y, int nt, const double* const* coef, const double* const* v,
                  const int* copy_at_first, const int* done, const Batch* bt, cudaStream_t s);
  // y = v0 + s2 * (v1 + s1 * v2)
  void (*nested)(int n, double* y, const double* v0, const double* v1, const double* v2, const double* s1,
                 const double* s2, const int* copy_at_first, const int* done, const Batch* bt, cudaStream_t s);
  void (*copy)(int n, double* y, const double* x, const int* done, cudaStream_t s);
  // nsys systems (one thread each); fin (nsys > 1): count of finished systems, and *alldone set
  // when it reaches nsys; hist: hist_stride doubles per system
  void (*scalar)(int method, int phase, double* S, int* st, double* hist, const int* done, int nsys, int hist_stride,
                 int* fin, int* alldone, cudaStream_t s);
  // Substitutions with a binary64 factor and w-component vectors (the paper's "_d"), or, for a
  // MPK_ILU_MP handle, with a w-component factor.
  int (*trsv_mp)(const IluHandleView& M, bool lower, bool unit, const double* in, double* out, const int* done,
                 cudaStream_t s);
  // Substitutions with a binary32 / bfloat16 factor: lower (in: w-component, out: the handle's
  // binary32 vector), upper (in: that vector, out: w-component); scaling by a power of two.
  int (*trsv32)(const IluHandleView& M, bool lower, bool unit, const double* in, double* out, const int* done,
                cudaStream_t s);
  // bt (nullable): one accumulator per system (out + s)
  void (*absmax)(int n, const double* v, unsigned long long* out, const int* done, const Batch* bt, cudaStream_t s);
  // 1 if the substitution kernel for factor precision prec, block size wpb warps and schedule
  // sched can be launched with all its blocks co-resident
  int (*trsv_fits)(int prec, int wpb, int sched, int nblocks);
};
const Ops* get_ops(int w, int cp);

// One triangle of the factor repacked for the static chunk schedule of the substitutions
// (SELL-32): positions are the level order's (32 rows per chunk, levels padded to whole chunks);
// chunk c owns slot blocks coff[c] .. coff[c+1]-1, and slot k of the row at lane l of chunk c is
// entry (coff[c] + k) * 32 + l of col / val, its entries in CSR order.  Values have the factor's
// storage type (double, float or bfloat16 bits).
//
// Owner-block variant (ob != 0): the positions are grouped by owner block first (block b of the
// cooperative grid owns a contiguous range of rows, balanced by work), then by level, each
// (block, level) group padded to whole chunks.  Block b runs its groups goff[bgrp[b]] ..
// goff[bgrp[b+1]] in order, its warps sharing a group's chunks, with a block barrier between
// groups.  A dependency computed earlier by the same block and still held in the block's
// shared-memory ring of kRing values is encoded as col = -2 - slot (slot = its position minus
// bstart[b], modulo kRing); the others keep their column and are polled in global memory; rep
// then names the latest of those (-1: none).
// Cluster variants (schedules 2, 3): a block is a thread-block cluster of csize CTAs (one per
// SM) sharing the group's chunks (chunk m of a group goes to CTA m mod csize); every CTA keeps
// the values it computed in its own ring, and a local dependency is encoded as
// -2 - (rank * kRing + slot), read from CTA `rank`'s ring through distributed shared memory
// after the cluster barrier that ends the producing group.
constexpr int kRing = 2048;  // values kept per CTA in shared memory (owner-block schedules)
constexpr int kScheds = 4;   // 0 static, 1 owner-block per SM, 2 / 3 owner-block per cluster of 8 / 16
constexpr int kClusterSmem = 116 * 1024;  // dynamic shared memory of a cluster CTA: one CTA per SM
inline int sched_csize(int sched) { return sched == 2 ? 8 : (sched == 3 ? 16 : 1); }
struct SellTri {
  const int* perm = nullptr;    // 32 * nchunks: row at each position (-1: padding)
  const int* coff = nullptr;    // nchunks + 1
  const int* col = nullptr;     // 32 * coff[nchunks]: column of the slot (-1 past the row's end)
  const void* val = nullptr;    // 32 * coff[nchunks] * cp: factor value of the slot
  const void* dia = nullptr;    // 32 * nchunks * cp: the row's diagonal factor value (1 for padding)
  const int* rep = nullptr;     // nchunks: the chunk's dependency latest in the level order (-1: none)
  int nchunks = 0;
  int ob = 0;                   // 1: owner-block layout (fields below)
  const int* goff = nullptr;    // groups + 1: first chunk of each (block, level) group
  const int* bgrp = nullptr;    // blocks + 1: first group of each block
  const int* bstart = nullptr;  // blocks + 1: first position of each block
  int nblocks = 0;              // the grid the layout was built for (blocks or clusters)
  int csize = 1;                // CTAs per block (cluster schedules: 8 or 16)
};

// Device-side view of an ILU(0) handle used by the substitution kernels (one triangle pair:
// either the factor itself or its conjugate transpose).
struct IluHandleView {
  int n = 0, nnz = 0, cp = 1, prec = 0;
  const int* rp = nullptr;
  const int* ci = nullptr;
  const int* diag = nullptr;
  const void* fac = nullptr;   // double / float / uint16 (bfloat16), cp values per entry;
                               // MPK_ILU_MP: cp * w doubles (w real components, then imaginary)
  int* flags = nullptr;        // n: epoch stamps of finished rows
  int* ctl = nullptr;          // device control words, see CtlIdx
  float* v32 = nullptr;        // n*cp binary32 intermediate
  double* vmp = nullptr;       // n*cp*w multi-component intermediate (capacity for w = 4)
  unsigned long long* absmax = nullptr;
  unsigned long long* pk = nullptr;  // packed (epoch << 32 | 32 payload bits) words, 8*cp per row
  LevelOrder lv_lo, lv_up;           // level orders of the two triangles
  SellTri sl_lo, sl_up;              // repacked triangles of the substitutions
  const int* sysid = nullptr;        // batch: row -> system (absmax holds one scale per system)
  int wpb = 4;                       // warps per block (per SM) of the substitution kernels
  int sched = 0;                     // see kScheds
  int withhold = -1;                 // testing aid: a row whose value is never published
  int poll = 0;                      // 0: lane 0 polls the chunk's latest dependency, then every lane
                                     // loads its own; 1: every lane polls its own from the start;
                                     // 2: as 1 with a short sleep between polling rounds
  int poll_ns = 256;                 // that sleep (MPK_SUBST_POLL_SLEEP_NS, default 256 ns)
};
enum CtlIdx : int {
  CTL_EPOCH = 0,
  CTL_TICKET_LO,
  CTL_TICKET_UP,
  CTL_ERR,
  CTL_FAIL_ROW,
  CTL_BAR_COUNT,  // grid barrier of the level-synchronous kernels: arrivals
  CTL_BAR_GEN,    // and generation
  CTL_COUNT
};

// Launch helpers shared by the instantiation units.
int sm_count();
int resident_warps_per_sm();        // MPK_RESIDENT_WARPS (default 32): dependency-driven kernels
void count_launch(unsigned k = 1);  // every kernel launch of the library is counted
unsigned long long launch_count();
void uncount_launch(unsigned long long k);  // launches recorded into a graph run only when it is launched
void launch_trsv_prep(const IluHandleView& M, const int* done, cudaStream_t s);
// Fingerprint of a CSR pattern (row_ptr[0..n], col_idx[0..nnz)), synchronises s: the key of the
// tuning caches (two patterns that differ anywhere collide with probability about 2^-64).
int pattern_fingerprint(int n, int nnz, const int* rp, const int* ci, uint64_t* out, cudaStream_t s);
// Pick the substitution kernels' warps per SM for this handle and w by timing the candidates
// (r, z: scratch vectors of n*c*w doubles); cached per (matrix pattern, factor precision, w, c).
int tune_substitution(mpk_ilu* M, const Ops* o, int w, double* r, double* z, cudaStream_t s);
// Repacked triangles t0, t0 + 1 (0: the factor, 2: its conjugate transpose) for schedule `sched`,
// built if missing (not inside a graph capture).
int ensure_layout(mpk_ilu* M, int t0, int sched, cudaStream_t s);
// ints of the order buffer of one triangle with n rows and `nlevels` levels:
// level perm (P = n + 32*nlevels) | level pos (n) | chunk flags (P/32 + 1) | nchunks (1)
size_t level_buf_ints(int n, int nlevels);
LevelOrder level_view(int* buf, int n, int nlevels);

}  // namespace mpk

// The opaque handle.
struct mpk_ilu {
  int n = 0, nnz = 0, cp = 1, prec = 0;
  int wf = 1;  // components per factor value (MPK_ILU_MP: the w it was built for)
  int* rp = nullptr;
  int* ci = nullptr;
  int* diag = nullptr;
  void* fac = nullptr;
  // conjugate transpose (built on first M^H use)
  int* rpT = nullptr;
  int* ciT = nullptr;
  int* diagT = nullptr;
  void* facT = nullptr;
  int* flags = nullptr;
  int* ctl = nullptr;
  float* v32 = nullptr;
  double* vmp = nullptr;
  unsigned long long* absmax = nullptr;
  unsigned long long* pk = nullptr;
  int* lvbuf[4] = {nullptr, nullptr, nullptr, nullptr};  // level orders: lower, upper, transposed lower / upper
  int nlevels[4] = {0, 0, 0, 0};
  // repacked triangles per schedule (see mpk::kScheds) and orientation (lower, upper, transposed
  // lower / upper): the repack buffer and, owner-block schedules, the order buffer
  void* laybuf[mpk::kScheds][4] = {};
  void* ordbuf[mpk::kScheds][4] = {};
  mpk::SellTri lay[mpk::kScheds][4];
  int* depth[4] = {nullptr, nullptr, nullptr, nullptr};      // level of every row, per triangle
  int wpb = 4;                   // warps per SM of the substitution kernels (autotuned per pattern)
  int sched = 0;                 // substitution schedule (autotuned per pattern)
  int poll = 0;                  // dependency polling of the substitutions (autotuned; see IluHandleView)
  int withhold = -1;             // testing aid (mpk_ilu0_test_withhold): a row left unpublished
  uint64_t pattern_fp = 0;       // fingerprint of the factored matrix's pattern: the tuning cache's key
  mpk::IluHandleView view(bool trans) const;
  int vals_per_entry() const { return cp * wf; }  // doubles (or narrower values) per factor entry
};
