// krylov.cu -- product-type Krylov solvers (Sec. 3): BiCG (Algorithm 3), CGS, BiCGSTAB and
// GPBiCG with an optional ILU(0) preconditioner, in w-component real or complex arithmetic.
//
// All scalars (rho, alpha, beta, omega, zeta, eta, norms) stay on the device; the host queues
// `check_every` iterations of kernels and then reads the device "done" flag once.  Kernels
// queued after convergence return immediately.  Every vector step below names the exact
// left-to-right evaluation it performs, term by term, so that each element sees the same
// sequence of w-component operations as the CPU restatement of the method.
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"

namespace mpk {
int precond_apply(const mpk_ilu* M, const Ops* o, bool trans, const double* r, double* z, const int* done,
                  const Batch* bt, cudaStream_t s);
int prepare_trans(mpk_ilu* M, cudaStream_t s);
int read_ctl_err(const mpk_ilu* M, cudaStream_t s);
int transpose_matrix(const Csr& A, int* rpT, int* ciT, double* vT, cudaStream_t s);
}  // namespace mpk

using namespace mpk;

// one word of device state set from the stream (graph-capturable)
__global__ void k_set_flag(int* p, int v) { *p = v; }

namespace {

// A solve of nsys systems (nsys == 1: the plain single-system solve; a batch otherwise, with
// per-system scalars, segmented inner products and finished systems frozen).
struct Ctx {
  const Ops* o;
  Csr A, AH;
  const mpk_ilu* M;
  int method, n;
  cudaStream_t s;
  double* S;
  int* st;
  const int* done;  // single: st[ST_DONE]; batch: the "all systems finished" flag
  double* hist;
  int hist_stride = 0;
  DotWs dws;
  const Batch* bt = nullptr;  // nullptr for a single system
  double* seg_partial = nullptr;
  unsigned* seg_counters = nullptr;
  int* fin = nullptr;
  int* alldone = nullptr;
  int err = MPK_OK;
  // residual replacement (true_res_period > 0): b, the iterate, scratch for b - A x, the
  // true-residual history
  int period = 0;
  const double* b = nullptr;
  double* x = nullptr;
  double* rtrue = nullptr;
  double* hist_true = nullptr;

  int nsys() const { return bt ? bt->nsys : 1; }
  double* slot(int k) const { return S + k * kSlotDoubles; }
  void dot(const double* a, const double* b, int out_slot) {
    const double* av[1] = {a};
    const double* bv[1] = {b};
    if (bt) {
      o->dots_seg(*bt, 1, av, bv, S, out_slot, seg_partial, seg_counters, done, s);
      return;
    }
    double* ov[1] = {slot(out_slot)};
    o->dots(n, 1, av, bv, ov, dws, done, s);
  }
  void dots(int k, const double* const* a, const double* const* b, int first_slot) {
    if (bt) {
      o->dots_seg(*bt, k, a, b, S, first_slot, seg_partial, seg_counters, done, s);
      return;
    }
    double* ov[kMaxDots];
    for (int q = 0; q < k; ++q) ov[q] = slot(first_slot + q);
    o->dots(n, k, a, b, ov, dws, done, s);
  }
  // y = t0 + t1 + t2, term k = coef_k * v_k (coef slot < 0: the vector itself)
  void lin(double* y, int c0, const double* v0, int c1 = -2, const double* v1 = nullptr, int c2 = -2,
           const double* v2 = nullptr, bool copy_at_first = false) {
    const double* coef[3] = {c0 >= 0 ? slot(c0) : nullptr, c1 >= 0 ? slot(c1) : nullptr, c2 >= 0 ? slot(c2) : nullptr};
    const double* v[3] = {v0, v1, v2};
    const int nt = (c1 == -2) ? 1 : ((c2 == -2) ? 2 : 3);
    o->lincomb(n, y, nt, coef, v, copy_at_first ? st : nullptr, done, bt, s);
  }
  // y = v0 + s2 (v1 + s1 v2); copy_at_first: y = v0 at iteration 1
  void nested(double* y, const double* v0, const double* v1, const double* v2, int s1, int s2, bool copy_at_first) {
    o->nested(n, y, v0, v1, v2, slot(s1), slot(s2), copy_at_first ? st : nullptr, done, bt, s);
  }
  void scalar(int phase) { o->scalar(method, phase, S, st, hist, done, nsys(), hist_stride, fin, alldone, s); }
  // The replacement rule after PH_NORM: when the iteration is checked (a multiple of the period,
  // or the recursive norm passed the test), rtrue = b - A x and its norm decide whether r becomes
  // rtrue.  The launches are gated on the state words ST_NOCHK / ST_NOREPL (per system in a batch).
  void truechk(double* r) {
    if (period <= 0) return;
    const double* av[1] = {rtrue};
    if (bt) {
      // every launch leaves at once unless some system asked for a check (nopend == 0); within
      // them, the systems that did not are skipped by their own state words
      int* nopend = alldone + 1;
      Batch g = *bt;
      g.gate = ST_NOCHK;
      o->spmv(A, x, rtrue, b, nopend, &g, s);
      o->dots_seg(g, 1, av, av, S, S_D5, seg_partial, seg_counters, nopend, s);
      o->scalar(method, PH_TRUECHK, S, st, hist_true, nopend, nsys(), hist_stride, fin, alldone, s);
      Batch gr = *bt;
      gr.gate = ST_NOREPL;
      const double* coef[1] = {nullptr};
      const double* v[1] = {rtrue};
      o->lincomb(n, r, 1, coef, v, nullptr, nopend, &gr, s);
      count_launch();
      k_set_flag<<<1, 1, 0, s>>>(nopend, 1);
      return;
    }
    const int* g1 = st + ST_NOCHK;
    o->spmv(A, x, rtrue, b, g1, nullptr, s);
    double* ov[1] = {slot(S_D5)};
    o->dots(n, 1, av, av, ov, dws, g1, s);
    o->scalar(method, PH_TRUECHK, S, st, hist_true, g1, 1, hist_stride, nullptr, nullptr, s);
    o->copy(n, r, rtrue, st + ST_NOREPL, s);
  }
  void mv(const double* x, double* y) { o->spmv(A, x, y, nullptr, done, bt, s); }
  void mvh(const double* x, double* y) { o->spmv(AH, x, y, nullptr, done, bt, s); }
  void prec(bool trans, const double* r, double* z) {
    if (M == nullptr) {
      o->copy(n, z, r, done, s);
      return;
    }
    int st_ = precond_apply(M, o, trans, r, z, done, bt, s);
    if (st_ != MPK_OK && err == MPK_OK) err = st_;
  }
};
constexpr int ONE = -1;  // coefficient "exactly one"

// ---- BiCGSTAB (van der Vorst), right-preconditioned, r = b - A x -----------------------------
struct BiCGSTAB {
  double *r, *rt, *p, *v, *ph, *sv, *sh, *tv;
  void iter(Ctx& c) {
    c.dot(rt, r, S_D0);                       // rho = <r~, r>
    c.scalar(PH_RHO);                         // beta = (rho/rho_old)(alpha/omega); 0 at it = 1
    c.nested(p, r, p, v, S_NOMEGA, S_BETA, true);  // p = r at it = 1, else r + beta (p + (-omega) v)
    c.prec(false, p, ph);                     // p^ = M^-1 p
    c.mv(ph, v);                              // v = A p^
    c.dot(rt, v, S_D0);                       // <r~, v>
    c.scalar(PH_SIG);                         // alpha = rho / <r~, v>
    c.lin(sv, ONE, r, S_NALPHA, v);           // s = r + (-alpha) v
    c.prec(false, sv, sh);                    // s^ = M^-1 s
    c.mv(sh, tv);                             // t = A s^
    const double* a[2] = {tv, tv};
    const double* b[2] = {sv, tv};
    c.dots(2, a, b, S_D0);                    // <t, s>, <t, t>
    c.scalar(PH_OMEGA);                       // omega = <t,s> / <t,t> (0 if <t,t> = 0)
    c.lin(xptr, ONE, xptr, S_ALPHA, ph, S_OMEGA, sh);  // x = (x + alpha p^) + omega s^
    c.lin(r, ONE, sv, S_NOMEGA, tv);          // r = s + (-omega) t
    c.dot(r, r, S_D0);
    c.scalar(PH_NORM);                        // ||r||, stopping rule, omega = 0 breakdown
    c.truechk(r);                             // replacement rule (true_res_period)
  }
  double* xptr;
};

// ---- CGS (Sonneveld), right-preconditioned ---------------------------------------------------
struct CGS {
  double *r, *rt, *u, *p, *q, *ph, *v, *uh, *uq, *tmp, *xptr;
  void iter(Ctx& c) {
    c.dot(rt, r, S_D0);                       // rho = <r~, r>
    c.scalar(PH_RHO);                         // beta = rho / rho_old; 0 at it = 1
    c.lin(u, ONE, r, S_BETA, q, -2, nullptr, true);  // u = r at it = 1, else r + beta q
    c.nested(p, u, q, p, S_BETA, S_BETA, true);      // p = u at it = 1, else u + beta (q + beta p)
    c.prec(false, p, ph);
    c.mv(ph, v);                              // v = A M^-1 p
    c.dot(rt, v, S_D0);
    c.scalar(PH_SIG);                         // alpha = rho / <r~, v>
    c.lin(q, ONE, u, S_NALPHA, v);            // q = u + (-alpha) v
    c.lin(uq, ONE, u, S_ONE, q);              // u + 1 q
    c.prec(false, uq, uh);                    // u^ = M^-1 (u + q)
    c.lin(xptr, ONE, xptr, S_ALPHA, uh);      // x = x + alpha u^
    c.mv(uh, tmp);
    c.lin(r, ONE, r, S_NALPHA, tmp);          // r = r + (-alpha) A u^
    c.dot(r, r, S_D0);
    c.scalar(PH_NORM);
    c.truechk(r);                             // replacement rule (true_res_period)
  }
};

// ---- BiCG, Algorithm 3 -----------------------------------------------------------------------
struct BiCG {
  double *r, *rt, *z, *zt, *p, *pt, *q, *qt, *xptr;
  void init(Ctx& c) {
    c.prec(false, r, z);                      // M z = r
    c.prec(true, rt, zt);                     // M^H z~ = r~
    c.o->copy(c.n, p, z, c.done, c.s);        // p = z
    c.o->copy(c.n, pt, zt, c.done, c.s);      // p~ = z~
    c.dot(zt, r, S_D0);                       // rho = <z~, r>
    c.scalar(PH_STORE_RHO);
  }
  void iter(Ctx& c) {
    c.mv(p, q);                               // q = A p
    c.mvh(pt, qt);                            // q~ = A^H p~
    c.dot(pt, q, S_D0);
    c.scalar(PH_SIG);                         // alpha = rho / <p~, q>
    c.lin(xptr, ONE, xptr, S_ALPHA, p);       // x = x + alpha p
    c.lin(r, ONE, r, S_NALPHA, q);            // r = r + (-alpha) q
    c.lin(rt, ONE, rt, S_NCALPHA, qt);        // r~ = r~ + (-conj(alpha)) q~
    c.dot(r, r, S_D0);
    c.scalar(PH_NORM);
    c.truechk(r);                             // replacement rule (true_res_period)
    c.prec(false, r, z);
    c.prec(true, rt, zt);
    c.dot(zt, r, S_D0);                       // rho_new = <z~, r>
    c.scalar(PH_BETA);                        // beta = rho_new / rho
    c.lin(p, ONE, z, S_BETA, p);              // p = z + beta p
    c.lin(pt, ONE, zt, S_CBETA, pt);          // p~ = z~ + conj(beta) p~
  }
};

// ---- GPBiCG (Zhang) on A M^-1, carried in M^-1-images ("hat" vectors) ------------------------
struct GPBiCG {
  double *r, *rt, *rh, *ph, *q, *qh, *tv, *th, *cv, *y, *uh, *zh, *wv, *tprev, *thprev, *tmp, *xptr;
  void init(Ctx& c) {
    c.dot(rt, r, S_D0);
    c.scalar(PH_STORE_RHO);                   // rho = <r~, r0>
  }
  void iter(Ctx& c) {
    c.scalar(PH_RHO);                         // rho = 0 -> breakdown
    c.prec(false, r, rh);                     // r^ = M^-1 r
    c.nested(ph, rh, ph, uh, S_MONE, S_BETA, false);  // p^ = r^ + beta (p^ + (-1) u^)
    c.mv(ph, q);                              // q = A p^
    c.dot(rt, q, S_D0);
    c.scalar(PH_SIG);                         // alpha = rho / <r~, q>
    c.prec(false, q, qh);                     // q^ = M^-1 q
    c.lin(tv, ONE, r, S_NALPHA, q);           // t = r + (-alpha) q
    c.lin(th, ONE, rh, S_NALPHA, qh);         // t^ = r^ + (-alpha) q^
    c.mv(th, cv);                             // c = A t^
    c.lin(y, ONE, tprev, S_MONE, tv, S_NALPHA, wv);  // y = (t_prev + (-1) t) + (-alpha) w
    const double* a[6] = {cv, cv, y, y, cv, y};
    const double* b[6] = {cv, tv, y, tv, y, cv};
    c.dots(6, a, b, S_D0);                    // cc, ct, yy, yt, cy, yc
    c.scalar(PH_ZETA);                        // zeta, eta (eta = 0 at it = 1)
    c.lin(tmp, ONE, thprev, S_MONE, rh, S_BETA, uh);  // (t^_prev + (-1) r^) + beta u^
    c.lin(uh, S_ZETA, qh, S_ETA, tmp);        // u^ = zeta q^ + eta (...)
    c.lin(zh, S_ZETA, rh, S_ETA, zh, S_NALPHA, uh);  // z^ = (zeta r^ + eta z^) + (-alpha) u^
    c.lin(xptr, ONE, xptr, S_ALPHA, ph, S_ONE, zh);  // x = (x + alpha p^) + 1 z^
    c.lin(r, ONE, tv, S_NETA, y, S_NZETA, cv);       // r = (t + (-eta) y) + (-zeta) c
    c.dot(r, r, S_D0);
    c.scalar(PH_NORM);
    c.truechk(r);                             // replacement rule (true_res_period)
    c.dot(rt, r, S_D0);
    c.scalar(PH_BETA);                        // beta = (alpha/zeta) <r~,r_new>/<r~,r>
    c.lin(wv, ONE, cv, S_BETA, q);            // w = c + beta q
    c.o->copy(c.n, tprev, tv, c.done, c.s);
    c.o->copy(c.n, thprev, th, c.done, c.s);
  }
};

}  // namespace

static int validate_csr(const mpk_csr* A) {
  if (A == nullptr) return fail(MPK_INVALID_ARG, "null matrix");
  if (A->n < 1 || A->nnz < 0 || A->row_ptr == nullptr || (A->nnz > 0 && (A->col_idx == nullptr || A->val == nullptr)))
    return fail(MPK_INVALID_ARG, "invalid CSR descriptor");
  if (A->is_complex != 0 && A->is_complex != 1) return fail(MPK_INVALID_ARG, "is_complex must be 0 or 1");
  if (A->is_complex && misaligned(A->val)) return fail(MPK_INVALID_ARG, "complex values must be 16-byte aligned");
  return MPK_OK;
}

// ---------------------------------------------------------------------------------------------
// Autotuner of the SpMV row order.  Candidates: natural order, and rows grouped by length
// (longest first; counting sort on the row lengths).  Both compute every row in CSR order, so the
// choice changes timing only.  The decision (and the order) is cached per matrix pattern (its
// fingerprint, n, nnz, w, c) for the process.
// ---------------------------------------------------------------------------------------------
constexpr int kLenBuckets = 1024;
__global__ void k_len_hist(int n, const int* __restrict__ rp, int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int len = min(rp[i + 1] - rp[i], kLenBuckets - 1);
    atomicAdd(cnt + (kLenBuckets - 1 - len), 1);
  }
}
__global__ void k_len_scan(int* __restrict__ cnt) {  // one thread: exclusive scan in place
  int run = 0;
  for (int b = 0; b < kLenBuckets; ++b) {
    const int v = cnt[b];
    cnt[b] = run;
    run += v;
  }
}
__global__ void k_len_scatter(int n, const int* __restrict__ rp, int* __restrict__ off, int* __restrict__ order) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int len = min(rp[i + 1] - rp[i], kLenBuckets - 1);
    order[atomicAdd(off + (kLenBuckets - 1 - len), 1)] = i;
  }
}
struct SpmvTune {
  uint64_t fp;
  int n, nnz, w, cp;
  int* order;  // nullptr: natural order wins
};
static std::mutex g_tune_mu;
static std::vector<SpmvTune> g_tune;

static const int* spmv_order(const Ops* o, const Csr& A, int w, int cp, double* x, double* y, cudaStream_t s) {
  uint64_t fp = 0;
  if (pattern_fingerprint(A.n, A.nnz, A.rp, A.ci, &fp, s) != MPK_OK) {
    cudaGetLastError();
    return nullptr;
  }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const SpmvTune& t : g_tune)
      if (t.fp == fp && t.n == A.n && t.nnz == A.nnz && t.w == w && t.cp == cp) return t.order;
  }
  int* order = nullptr;
  int* cnt = nullptr;
  if (cudaMalloc((void**)&order, sizeof(int) * (size_t)A.n) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaMallocAsync((void**)&cnt, sizeof(int) * kLenBuckets, s) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(order);
    return nullptr;
  }
  cudaMemsetAsync(cnt, 0, sizeof(int) * kLenBuckets, s);
  const int g = (A.n + 255) / 256 < 4096 ? (A.n + 255) / 256 : 4096;
  count_launch(3);
  k_len_hist<<<g, 256, 0, s>>>(A.n, A.rp, cnt);
  k_len_scan<<<1, 1, 0, s>>>(cnt);
  k_len_scatter<<<g, 256, 0, s>>>(A.n, A.rp, cnt, order);
  cudaFreeAsync(cnt, s);
  // time both candidates (x, y: scratch vectors; the cost does not depend on the values)
  cudaEvent_t ev[4];
  for (auto& e : ev) cudaEventCreate(&e);
  Csr nat = A, srt = A;
  nat.order = nullptr;
  srt.order = order;
  float t[2] = {0.f, 0.f};
  for (int rep = 0; rep < 2; ++rep) {
    for (int v = 0; v < 2; ++v) {
      const Csr& M = v == 0 ? nat : srt;
      o->spmv(M, x, y, nullptr, nullptr, nullptr, s);  // warm
      cudaEventRecord(ev[2 * v], s);
      o->spmv(M, x, y, nullptr, nullptr, nullptr, s);
      o->spmv(M, x, y, nullptr, nullptr, nullptr, s);
      cudaEventRecord(ev[2 * v + 1], s);
    }
    cudaEventSynchronize(ev[3]);
    for (int v = 0; v < 2; ++v) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * v], ev[2 * v + 1]);
      t[v] += ms;
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (cudaGetLastError() != cudaSuccess) {
    cudaFree(order);
    return nullptr;
  }
  const bool use = t[1] < 0.97f * t[0];
  if (!use) {
    cudaFree(order);
    order = nullptr;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (g_tune.size() < 64) g_tune.push_back(SpmvTune{fp, A.n, A.nnz, w, cp, order});
  else if (order != nullptr) {
    // cache full: keep this solve untuned rather than grow without bound
    cudaFree(order);
    order = nullptr;
  }
  return order;
}

// Rows -> system, and the segmented inner products' block layout, of a batch with row offsets roff.
__global__ void k_batch_sysid(int n, int nsys, const int* __restrict__ roff, int* __restrict__ sysid,
                              int* __restrict__ bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int lo = 0, hi = nsys;  // largest sy with roff[sy] <= i
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (roff[mid] <= i) lo = mid;
      else hi = mid;
    }
    sysid[i] = lo;
  }
  (void)bad;
}
// Every stored column of row i lies in row i's system block (block-diagonal structure).
__global__ void k_batch_check(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const int* __restrict__ roff, const int* __restrict__ sysid, int* __restrict__ bad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int sy = sysid[i], lo = roff[sy], hi = roff[sy + 1];
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] < lo || ci[p] >= hi) atomicMin(bad, i);
  }
}
__global__ void k_batch_bsys(int nsys, const int* __restrict__ boff, int* __restrict__ bsys) {
  for (int sy = blockIdx.x; sy < nsys; sy += gridDim.x)
    for (int b = boff[sy] + threadIdx.x; b < boff[sy + 1]; b += blockDim.x) bsys[b] = sy;
}

// Whether A equals its conjugate transpose: every entry (i, j) has its mirror (j, i) with the
// conjugate value (compared as numbers).  Columns are sorted within rows (validated), so the
// mirror is found by bisection.  *not_h is set to 1 on the first mismatch.
__global__ void k_hermitian(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                            const double* __restrict__ val, int cplx, int* __restrict__ not_h) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p];
      if (j < 0 || j >= n) {
        atomicOr(not_h, 1);
        return;
      }
      int lo = rp[j], hi = rp[j + 1];  // first position in row j with column >= i
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ci[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      bool ok = lo < rp[j + 1] && ci[lo] == i;
      if (ok) ok = cplx ? (val[2 * (int64_t)lo] == val[2 * (int64_t)p] && val[2 * (int64_t)lo + 1] == -val[2 * (int64_t)p + 1])
                        : val[lo] == val[p];
      if (!ok) {
        atomicOr(not_h, 1);
        return;
      }
    }
  }
}

// nsys == 1 and roff_host == nullptr: one system.  Otherwise A is block-diagonal with the systems'
// rows at roff_host[s] .. roff_host[s+1]-1 (host copy) / roff_dev (device copy); infos has nsys
// entries; hist_dev (nullable) nsys * (maxit + 1) doubles.
// The solve runs on a private stream joined to the caller's stream at both ends (stream capture
// into a CUDA graph is not possible on the legacy default stream).
struct StreamJoin {
  cudaStream_t caller = nullptr, own = nullptr;
  cudaEvent_t ev = nullptr;
  bool ok = false;
  explicit StreamJoin(cudaStream_t c) : caller(c) {
    ok = cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventRecord(ev, caller) == cudaSuccess && cudaStreamWaitEvent(own, ev, 0) == cudaSuccess;
  }
  ~StreamJoin() {
    if (own != nullptr) {
      if (ev != nullptr && cudaEventRecord(ev, own) == cudaSuccess) cudaStreamWaitEvent(caller, ev, 0);
      cudaStreamDestroy(own);
    }
    if (ev != nullptr) cudaEventDestroy(ev);
  }
};
static bool graphs_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("MPK_NO_GRAPH");
    return !(e != nullptr && e[0] == '1');
  }();
  return on;
}

static int solve_impl(int method, int w, const mpk_csr* Ac, const mpk_ilu* Mc, const double* b, double* x,
                      const mpk_opts* opts, mpk_info* infos, cudaStream_t caller, int nsys, const int* roff_host,
                      const int* roff_dev) {
  StreamJoin join(caller);
  if (!join.ok) return fail(MPK_CUDA_ERROR, "could not create the solve's stream");
  cudaStream_t s = join.own;
  const int n = Ac->n, cp = Ac->is_complex ? 2 : 1;
  const int64_t vlen = (int64_t)n * cp * w;
  mpk_ilu* M = const_cast<mpk_ilu*>(Mc);
  const Ops* o = get_ops(w, cp);
  if (o == nullptr) return fail(MPK_INVALID_ARG, "unsupported (w, complex)");
  const int check_every = opts->check_every > 0 ? opts->check_every : 25;
  const int maxit = opts->maxit;
  const bool batched = roff_host != nullptr;

  Ctx c;
  c.o = o;
  c.A = Csr{n, Ac->nnz, Ac->row_ptr, Ac->col_idx, Ac->val, Ac->is_complex};
  c.A.mm = (opts->flags & MPK_FLAG_MP_MATRIX) != 0;
  c.M = M;
  c.method = method;
  c.n = n;
  c.s = s;
  c.hist = opts->hist_dev;
  c.hist_stride = maxit + 1;

  cudaEvent_t e0, e1;
  MPK_CUDA(cudaEventCreate(&e0));
  MPK_CUDA(cudaEventCreate(&e1));
  MPK_CUDA(cudaEventRecord(e0, s));

  if (method == MPK_BICG && M != nullptr) {
    int st = prepare_trans(M, s);
    if (st != MPK_OK) return st;
  }
  // batch layout: inner-product blocks per system (host scan of the row offsets)
  std::vector<int> boff_h;
  int nblocks = 0;
  if (batched) {
    boff_h.resize((size_t)nsys + 1);
    for (int sy = 0; sy < nsys; ++sy) {
      boff_h[sy] = nblocks;
      nblocks += dot_blocks(roff_host[sy + 1] - roff_host[sy]);
    }
    boff_h[nsys] = nblocks;
  }
  const int nvec = 17;
  const size_t vec_bytes = (sizeof(double) * (size_t)vlen + 255) & ~(size_t)255;
  const size_t S_bytes = (sizeof(double) * (size_t)kSysDoubles * nsys + 255) & ~(size_t)255;
  const size_t part_bytes = batched ? (sizeof(double) * (size_t)nblocks * kMaxDots * 8 + 255) & ~(size_t)255
                                    : (sizeof(double) * dot_partial_doubles(n) + 255) & ~(size_t)255;
  const size_t st_bytes = (sizeof(int) * ((size_t)ST_COUNT * nsys + 8) + 255) & ~(size_t)255;
  const size_t cnt_bytes = (sizeof(unsigned) * ((size_t)nsys + 8) + 255) & ~(size_t)255;
  const size_t batch_bytes = batched ? (sizeof(int) * ((size_t)n + 2 * ((size_t)nsys + 1) + nblocks) +
                                        sizeof(unsigned long long) * (size_t)nsys + 1024)
                                     : 0;
  const size_t total = vec_bytes * nvec + S_bytes + part_bytes + st_bytes + cnt_bytes + batch_bytes + 256;
  char* base = nullptr;
  MPK_CUDA(cudaMallocAsync((void**)&base, total, s));
  MPK_CUDA(cudaMemsetAsync(base + vec_bytes * nvec, 0, total - vec_bytes * nvec, s));
  MPK_CUDA(cudaMemsetAsync(base, 0, vec_bytes * nvec, s));
  std::vector<double*> V(nvec);
  for (int k = 0; k < nvec; ++k) V[k] = (double*)(base + vec_bytes * k);
  char* tail = base + vec_bytes * nvec;
  c.S = (double*)tail;
  tail += S_bytes;
  double* partial = (double*)tail;
  tail += part_bytes;
  c.st = (int*)tail;
  // [0] finished systems, [1] all finished, [2] no replacement check pending in any system (the
  // gate of the batch's check launches; k_scalar's PH_NORM clears it at alldone + 1)
  int* gstate = c.st + (size_t)ST_COUNT * nsys;
  tail += st_bytes;
  unsigned* counters = (unsigned*)tail;
  tail += cnt_bytes;
  c.dws.partial = partial;
  c.dws.counter = counters;
  Batch bt;
  if (batched) {
    unsigned long long* amax = (unsigned long long*)(((uintptr_t)tail + 15) & ~(uintptr_t)15);
    int* sysid = (int*)(amax + nsys);
    int* boff = sysid + n;
    int* bsys = boff + nsys + 1;
    int* bad = bsys + nblocks;
    MPK_CUDA(cudaMemcpyAsync(boff, boff_h.data(), sizeof(int) * ((size_t)nsys + 1), cudaMemcpyHostToDevice, s));
    int bad0 = INT_MAX;
    MPK_CUDA(cudaMemcpyAsync(bad, &bad0, sizeof(int), cudaMemcpyHostToDevice, s));
    count_launch(3);
    k_batch_sysid<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(n, nsys, roff_dev, sysid, bad);
    k_batch_check<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(n, Ac->row_ptr, Ac->col_idx,
                                                                                   roff_dev, sysid, bad);
    k_batch_bsys<<<nsys < 1024 ? nsys : 1024, 128, 0, s>>>(nsys, boff, bsys);
    MPK_CUDA(cudaGetLastError());
    int badh = INT_MAX;
    MPK_CUDA(cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    MPK_CUDA(cudaStreamSynchronize(s));
    if (badh != INT_MAX) {
      cudaFreeAsync(base, s);
      return fail(MPK_INVALID_ARG, "row " + std::to_string(badh) + " has a column outside its system's block");
    }
    bt.nsys = nsys;
    bt.sysid = sysid;
    bt.roff = roff_dev;
    bt.boff = boff;
    bt.bsys = bsys;
    bt.nblocks = nblocks;
    bt.st = c.st;
    bt.absmax = amax;
    c.bt = &bt;
    c.seg_partial = partial;
    c.seg_counters = counters;
    c.fin = gstate;
    c.alldone = gstate + 1;
    c.done = gstate + 1;
  } else {
    c.done = c.st + ST_DONE;
  }

  int* ahbuf = nullptr;
  int hermitian = 0;
  if (method == MPK_BICG) {  // A = A^H: q~ = A^H p~ multiplies by A itself (its rows are A^H's)
    int* flag = nullptr;
    MPK_CUDA(cudaMallocAsync((void**)&flag, sizeof(int), s));
    MPK_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), s));
    count_launch();
    k_hermitian<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(n, Ac->row_ptr, Ac->col_idx, Ac->val, Ac->is_complex, flag);
    int not_h = 1;
    MPK_CUDA(cudaMemcpyAsync(&not_h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    MPK_CUDA(cudaFreeAsync(flag, s));
    MPK_CUDA(cudaStreamSynchronize(s));
    hermitian = not_h == 0;
    if (hermitian) c.AH = c.A;
  }
  if (method == MPK_BICG && !hermitian) {  // A^H for q~ = A^H p~ (block-diagonal stays block-diagonal)
    const size_t nnz = (size_t)Ac->nnz;
    MPK_CUDA(cudaMallocAsync((void**)&ahbuf, sizeof(int) * ((size_t)n + 1 + nnz) + sizeof(double) * nnz * cp + 16, s));
    int* rpT = ahbuf;
    int* ciT = ahbuf + n + 1;
    double* vT = (double*)(((uintptr_t)(ciT + nnz) + 15) & ~(uintptr_t)15);
    int st = transpose_matrix(c.A, rpT, ciT, vT, s);
    if (st != MPK_OK) return st;
    c.AH = Csr{n, Ac->nnz, rpT, ciT, vT, Ac->is_complex};
    c.AH.mm = c.A.mm;
  }

  {
    std::vector<int> st_init((size_t)ST_COUNT * nsys);
    for (int sy = 0; sy < nsys; ++sy) {
      int* q = st_init.data() + (size_t)sy * ST_COUNT;
      q[ST_DONE] = 0;
      q[ST_STATUS] = MPK_MAXIT;
      q[ST_ITERS] = 0;
      q[ST_IT] = 0;
      q[ST_MAXIT] = maxit;
      q[ST_FLAGS] = opts->flags;
      q[ST_PERIOD] = opts->true_res_period > 0 ? opts->true_res_period : 0;
      q[ST_NOCHK] = 1;
      q[ST_NOREPL] = 1;
      q[ST_CHECK] = 0;
      q[ST_CHK_IT] = 0;
      q[ST_NREP] = 0;
      q[ST_TRUEKNOWN] = 0;
    }
    MPK_CUDA(cudaMemcpyAsync(c.st, st_init.data(), sizeof(int) * st_init.size(), cudaMemcpyHostToDevice, s));
    const int one = 1;
    MPK_CUDA(cudaMemcpyAsync(gstate + 2, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    std::vector<double> tolv((size_t)2 * nsys);
    for (int sy = 0; sy < nsys; ++sy) {
      tolv[2 * sy] = opts->tol_rel;
      tolv[2 * sy + 1] = opts->tol_abs;
    }
    MPK_CUDA(cudaMemcpy2DAsync(c.slot(S_TOL) + 1, sizeof(double) * kSysDoubles, tolv.data(), 2 * sizeof(double),
                               2 * sizeof(double), nsys, cudaMemcpyHostToDevice, s));
    MPK_CUDA(cudaStreamSynchronize(s));  // the host buffers above go out of scope
  }

  // SpMV row order and substitution warps per SM for this matrix pattern (autotuned once per
  // pattern and cached; V[15], V[16] serve as scratch: zero in, zero out)
  c.A.order = spmv_order(o, c.A, w, cp, V[15], V[16], s);
  if (M != nullptr) {
    const int st = tune_substitution(M, o, w, V[15], V[16], s);
    if (st != MPK_OK) {
      cudaFreeAsync(base, s);
      return st;
    }
  }

  double* r = V[0];
  double* rt = V[1];
  c.period = opts->true_res_period > 0 ? opts->true_res_period : 0;
  c.b = b;
  c.x = x;
  c.rtrue = V[16];  // free during the iterations (tuner scratch before, final residual after)
  c.hist_true = opts->hist_true_dev;
  // r = b - A x0, r~ = r, ||r0||
  o->spmv(c.A, x, r, b, c.done, nullptr, s);
  o->copy(n, rt, r, c.done, s);
  c.dot(r, r, S_D0);
  c.scalar(PH_INIT);

  BiCGSTAB m_stab{r, rt, V[2], V[3], V[4], V[5], V[6], V[7], x};
  CGS m_cgs{r, rt, V[2], V[3], V[4], V[5], V[6], V[7], V[8], V[9], x};
  BiCG m_bicg{r, rt, V[2], V[3], V[4], V[5], V[6], V[7], x};
  GPBiCG m_gp{r, rt, V[2], V[3], V[4], V[5], V[6], V[7], V[8], V[9], V[10], V[11], V[12], V[13], V[14], V[15], x};
  switch (method) {
    case MPK_BICG: m_bicg.init(c); break;
    case MPK_GPBICG: m_gp.init(c); break;
    default: break;
  }
  auto one_iter = [&]() {
    switch (method) {
      case MPK_BICG: m_bicg.iter(c); break;
      case MPK_CGS: m_cgs.iter(c); break;
      case MPK_BICGSTAB: m_stab.iter(c); break;
      default: m_gp.iter(c); break;
    }
  };
  // One iteration captured into a CUDA graph and replayed; every kernel reads its state from device
  // memory, so the replays are the iterations.  If capture is not possible the launches go direct.
  cudaGraphExec_t gexec = nullptr;
  unsigned long long per_iter = 0;
  if (graphs_enabled() && c.err == MPK_OK) {
    const unsigned long long l0 = launch_count();
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      one_iter();
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (e == cudaSuccess && c.err == MPK_OK) e = cudaGraphInstantiate(&gexec, g, 0);
      if (g != nullptr) cudaGraphDestroy(g);
      if (e != cudaSuccess || c.err != MPK_OK) {
        if (gexec != nullptr) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        c.err = MPK_OK;
      }
    }
    cudaGetLastError();  // a failed capture leaves no error behind: the launches then go direct
    per_iter = launch_count() - l0;
    uncount_launch(per_iter);
  }
  int hflag = 0;
  int queued = 0;
  for (;;) {
    for (int k = 0; k < check_every; ++k) {
      if (gexec != nullptr) {
        if (cudaGraphLaunch(gexec, s) != cudaSuccess) {
          c.err = fail(MPK_CUDA_ERROR, "graph launch failed");
          break;
        }
        count_launch((unsigned)per_iter);
      } else {
        one_iter();
      }
    }
    queued += check_every;
    if (c.err != MPK_OK) break;
    MPK_CUDA(cudaGetLastError());
    MPK_CUDA(cudaMemcpyAsync(&hflag, c.done, sizeof(int), cudaMemcpyDeviceToHost, s));
    MPK_CUDA(cudaStreamSynchronize(s));
    if (hflag || queued > maxit + check_every) break;
  }
  const bool gexec_used = gexec != nullptr;
  if (gexec != nullptr) cudaGraphExecDestroy(gexec);
  if (c.err != MPK_OK) {
    cudaFreeAsync(base, s);
    if (ahbuf) cudaFreeAsync(ahbuf, s);
    return c.err;
  }
  int dev_err = MPK_OK;
  if (M != nullptr) dev_err = read_ctl_err(M, s);

  // true residual b - A x with the final x, for every system that did not end on an accepted
  // replacement check (those have it already).  The batch launches skip a system through the
  // state word they read as ST_DONE, here shifted to ST_TRUEKNOWN (every system is done now).
  {
    const double* av[1] = {V[16]};
    const double* bv[1] = {V[16]};
    if (batched) {
      Batch all = bt;
      all.st = c.st + (ST_TRUEKNOWN - ST_DONE);
      all.gate = -1;
      o->spmv(c.A, x, V[16], b, nullptr, &all, s);
      o->dots_seg(all, 1, av, bv, c.S, S_D5, partial, counters, nullptr, s);
    } else {
      const int* known = c.st + ST_TRUEKNOWN;
      o->spmv(c.A, x, V[16], b, known, nullptr, s);
      double* ov[1] = {c.slot(S_D5)};
      o->dots(n, 1, av, bv, ov, c.dws, known, s);
    }
    o->scalar(method, PH_TRUE, c.S, c.st, nullptr, nullptr, nsys, 0, nullptr, nullptr, s);
  }
  MPK_CUDA(cudaEventRecord(e1, s));
  std::vector<int> hst((size_t)ST_COUNT * nsys);
  std::vector<double> hS((size_t)kSysDoubles * nsys);
  MPK_CUDA(cudaMemcpyAsync(hst.data(), c.st, sizeof(int) * hst.size(), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaMemcpyAsync(hS.data(), c.S, sizeof(double) * hS.size(), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MPK_CUDA(cudaFreeAsync(base, s));
  if (ahbuf) MPK_CUDA(cudaFreeAsync(ahbuf, s));

  int worst = MPK_OK;
  for (int sy = 0; sy < nsys; ++sy) {
    const int* q = hst.data() + (size_t)sy * ST_COUNT;
    const double* Sy = hS.data() + (size_t)sy * kSysDoubles;
    mpk_info& info = infos[sy];
    const double r0n = Sy[S_R0N * kSlotDoubles];
    info.status = q[ST_DONE] ? q[ST_STATUS] : MPK_MAXIT;
    info.iters = q[ST_DONE] ? q[ST_ITERS] : maxit;
    if (dev_err != MPK_OK) info.status = dev_err;
    info.fail_row = -1;
    info.graph = gexec_used ? 1 : 0;
    info.hermitian = hermitian;
    info.replacements = q[ST_NREP];
    info.res0 = r0n;
    info.relres_rec = r0n > 0 ? Sy[S_NORM * kSlotDoubles] / r0n : 0.0;
    info.relres_true = r0n > 0 ? Sy[S_D4 * kSlotDoubles] / r0n : 0.0;
    info.ms_solve = ms;
    if (info.status != MPK_OK && worst == MPK_OK) worst = info.status;
  }
  if (dev_err != MPK_OK) return fail(dev_err, "solve failed on the device");
  if (!batched) {
    const int st = infos[0].status;
    if (st != MPK_OK && st != MPK_MAXIT && st != MPK_BREAKDOWN && st != MPK_NAN)
      return fail(st, "solve failed on the device");
    return st;
  }
  return worst;
}

extern "C" int mpk_krylov_solve(int method, int w, const mpk_csr* A, const mpk_ilu* M, const double* b_dev,
                                double* x_dev, const mpk_opts* opts, mpk_info* info, void* stream) {
  mpk_info dummy;
  if (info == nullptr) info = &dummy;
  std::memset(info, 0, sizeof(*info));
  info->fail_row = -1;
  info->status = MPK_INVALID_ARG;
  int v = validate_csr(A);
  if (v != MPK_OK) return v;
  if (method < MPK_BICG || method > MPK_GPBICG) return fail(MPK_INVALID_ARG, "unknown method");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  if (b_dev == nullptr || x_dev == nullptr || opts == nullptr || b_dev == x_dev)
    return fail(MPK_INVALID_ARG, "null or aliased vector / options");
  if (misaligned(b_dev) || misaligned(x_dev)) return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  if (opts->maxit < 0) return fail(MPK_INVALID_ARG, "maxit must be >= 0");
  if (M != nullptr && (M->n != A->n || M->cp != (A->is_complex ? 2 : 1)))
    return fail(MPK_INVALID_ARG, "preconditioner does not match the matrix");
  if (M != nullptr && M->prec == MPK_ILU_MP && M->wf != w)
    return fail(MPK_INVALID_ARG, "a w-component factor serves solves with the same w");
  int st = solve_impl(method, w, A, M, b_dev, x_dev, opts, info, (cudaStream_t)stream, 1, nullptr, nullptr);
  info->status = st;
  return st;
}

extern "C" int mpk_krylov_solve_batched(int method, int w, const mpk_csr* A, int nsys, const int32_t* sys_rows_host,
                                        const int32_t* sys_rows_dev, const mpk_ilu* M, const double* b_dev,
                                        double* x_dev, const mpk_opts* opts, mpk_info* infos, void* stream) {
  if (infos == nullptr || nsys < 1) return fail(MPK_INVALID_ARG, "null infos or nsys < 1");
  for (int sy = 0; sy < nsys; ++sy) {
    std::memset(infos + sy, 0, sizeof(mpk_info));
    infos[sy].fail_row = -1;
    infos[sy].status = MPK_INVALID_ARG;
  }
  int v = validate_csr(A);
  if (v != MPK_OK) return v;
  if (method < MPK_BICG || method > MPK_GPBICG) return fail(MPK_INVALID_ARG, "unknown method");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  if (b_dev == nullptr || x_dev == nullptr || opts == nullptr || b_dev == x_dev)
    return fail(MPK_INVALID_ARG, "null or aliased vector / options");
  if (misaligned(b_dev) || misaligned(x_dev)) return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  if (sys_rows_host == nullptr || sys_rows_dev == nullptr) return fail(MPK_INVALID_ARG, "null system row offsets");
  if (sys_rows_host[0] != 0 || sys_rows_host[nsys] != A->n)
    return fail(MPK_INVALID_ARG, "system row offsets must start at 0 and end at n");
  for (int sy = 0; sy < nsys; ++sy)
    if (sys_rows_host[sy + 1] <= sys_rows_host[sy]) return fail(MPK_INVALID_ARG, "empty or decreasing system");
  if (opts->maxit < 0) return fail(MPK_INVALID_ARG, "maxit must be >= 0");
  if (M != nullptr && (M->n != A->n || M->cp != (A->is_complex ? 2 : 1)))
    return fail(MPK_INVALID_ARG, "preconditioner does not match the matrix");
  if (M != nullptr && M->prec == MPK_ILU_MP && M->wf != w)
    return fail(MPK_INVALID_ARG, "a w-component factor serves solves with the same w");
  return solve_impl(method, w, A, M, b_dev, x_dev, opts, infos, (cudaStream_t)stream, nsys, sys_rows_host,
                    sys_rows_dev);
}

extern "C" int mpk_solve_host(int method, int w, int prec, int32_t n, int32_t is_complex, const int32_t* rp_h,
                              const int32_t* ci_h, const double* val_h, const double* b_h, double* x_h,
                              const mpk_opts* opts, mpk_info* info) {
  mpk_info dummy;
  if (info == nullptr) info = &dummy;
  std::memset(info, 0, sizeof(*info));
  info->fail_row = -1;
  if (n < 1 || rp_h == nullptr || b_h == nullptr || x_h == nullptr || opts == nullptr)
    return fail(MPK_INVALID_ARG, "null argument");
  if (w < 1 || w > 4 || (is_complex != 0 && is_complex != 1)) return fail(MPK_INVALID_ARG, "bad w / is_complex");
  const int nnz = rp_h[n];
  const int cp = is_complex ? 2 : 1;
  if (nnz < 0 || (nnz > 0 && (ci_h == nullptr || val_h == nullptr))) return fail(MPK_INVALID_ARG, "bad nnz");
  cudaStream_t s;
  MPK_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  MPK_CUDA(cudaEventCreate(&e0));
  MPK_CUDA(cudaEventCreate(&e1));
  MPK_CUDA(cudaEventRecord(e0, s));
  const size_t vb = sizeof(double) * (size_t)n * cp * w;
  char* buf = nullptr;
  const size_t bytes = sizeof(int) * ((size_t)n + 1 + nnz) + 16 + sizeof(double) * (size_t)nnz * cp + 2 * vb + 64;
  MPK_CUDA(cudaMallocAsync((void**)&buf, bytes, s));
  int* rp = (int*)buf;
  int* ci = rp + n + 1;
  double* val = (double*)(((uintptr_t)(ci + nnz) + 15) & ~(uintptr_t)15);
  double* b = (double*)(((uintptr_t)(val + (size_t)nnz * cp) + 15) & ~(uintptr_t)15);
  double* x = b + (size_t)n * cp * w;
  MPK_CUDA(cudaMemcpyAsync(rp, rp_h, sizeof(int) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
  MPK_CUDA(cudaMemcpyAsync(ci, ci_h, sizeof(int) * (size_t)nnz, cudaMemcpyHostToDevice, s));
  MPK_CUDA(cudaMemcpyAsync(val, val_h, sizeof(double) * (size_t)nnz * cp, cudaMemcpyHostToDevice, s));
  MPK_CUDA(cudaMemcpyAsync(b, b_h, vb, cudaMemcpyHostToDevice, s));
  MPK_CUDA(cudaMemcpyAsync(x, x_h, vb, cudaMemcpyHostToDevice, s));
  mpk_csr A{n, nnz, rp, ci, val, is_complex};
  mpk_ilu* M = nullptr;
  int st = MPK_OK;
  if (prec == MPK_ILU_MP) st = mpk_ilu0_factor_mp(&A, w, &M, &info->fail_row, s);
  else if (prec != MPK_ILU_NONE) st = mpk_ilu0_factor(&A, prec, &M, &info->fail_row, s);
  if (st == MPK_OK) st = mpk_krylov_solve(method, w, &A, M, b, x, opts, info, s);
  if (M) mpk_ilu0_destroy(M);
  int fr = info->fail_row;
  MPK_CUDA(cudaMemcpyAsync(x_h, x, vb, cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaFreeAsync(buf, s));
  MPK_CUDA(cudaEventRecord(e1, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  info->ms_solve = ms;
  info->fail_row = fr;
  info->status = st;
  return st;
}
