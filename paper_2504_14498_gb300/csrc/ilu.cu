// ilu.cu -- ILU(0) factorisation (Algorithm 1) and the substitutions of Algorithm 2 as C-ABI
// entry points, plus the device transposition used by BiCG's M^H solve (Algorithm 3).
#include <climits>
#include <cstdint>
#include <cstring>

#include "kernels.cuh"

namespace mpk {

// ---------------------------------------------------------------------------------------------
// Pattern validation: rows monotone and inside [0, nnz], columns in range and strictly
// ascending, diagonal present.  code = min over failing rows of 2*row (+1 if only the
// diagonal is missing).
// ---------------------------------------------------------------------------------------------
__global__ void k_check_pattern(int n, int nnz, const int* __restrict__ rp, const int* __restrict__ ci,
                                int* __restrict__ diag, int* __restrict__ code) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = rp[i], b = rp[i + 1];
  if (a < 0 || b < a || b > nnz) { atomicMin(code, 2 * i); return; }
  int d = -1, prev = -1;
  for (int p = a; p < b; ++p) {
    const int c = ci[p];
    if (c < 0 || c >= n || c <= prev) { atomicMin(code, 2 * i); return; }
    if (c == i) d = p;
    prev = c;
  }
  if (d < 0) atomicMin(code, 2 * i + 1);
  else diag[i] = d;
}

template <typename T>
__global__ void k_narrow(int64_t m, const double* __restrict__ v, T* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = (T)v[k];
}
__device__ __forceinline__ uint16_t bf16_rne(float f) {
  unsigned u = __float_as_uint(f);
  if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0u) return (uint16_t)((u | 0x00400000u) >> 16);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
__global__ void k_to_bf16(int64_t m, const float* __restrict__ v, uint16_t* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = bf16_rne(v[k]);
}
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return (double)x; }
__device__ __forceinline__ double widen(uint16_t x) { return (double)__uint_as_float(((unsigned)x) << 16); }
template <typename T>
__global__ void k_widen(int64_t m, const T* __restrict__ v, double* __restrict__ out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x)
    out[k] = widen(v[k]);
}

// ---------------------------------------------------------------------------------------------
// ILU(0) by rows (row-IKJ): for each k < i in row i, ascending: a_ik := a_ik / a_kk, then for
// every j > k in row k that is also in row i: a_ij := fma(-a_ik, a_kj, a_ij).  Entry a_ij
// receives exactly the updates of the KIJ listing, in the same (ascending k) order, so the
// result equals Algorithm 1 bit for bit.  Complex steps use the operation order
//   x/y: den = fma(yr,yr,yi*yi), nr = fma(xr,yr,xi*yi), ni = fma(xi,yr,-(xr*yi)), (nr/den, ni/den)
//   a -= l*u: re = fma(-lr,ur,ar), re = fma(li,ui,re), im = fma(-lr,ui,ai), im = fma(-li,ur,im).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ float fm(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fm(double a, double b, double c) { return fma(a, b, c); }

template <typename T, int CP>
struct RowIlu {
  const int* rp;
  const int* ci;
  const int* diag;
  T* a;
  int* ctl;
  __device__ void begin(int i, int& p, int& pend) {
    p = rp[i];
    pend = diag[i];
  }
  __device__ void consume(int i, int p, int k) {
    const int dk = diag[k], ek = rp[k + 1], ei = rp[i + 1];
    T lr, li = T(0);
    if constexpr (CP == 1) {
      lr = a[p] / a[dk];
      a[p] = lr;
    } else {
      const T xr = a[2 * (int64_t)p], xi = a[2 * (int64_t)p + 1];
      const T yr = a[2 * (int64_t)dk], yi = a[2 * (int64_t)dk + 1];
      const T den = fm(yr, yr, yi * yi), nr = fm(xr, yr, xi * yi), ni = fm(xi, yr, -(xr * yi));
      lr = nr / den;
      li = ni / den;
      a[2 * (int64_t)p] = lr;
      a[2 * (int64_t)p + 1] = li;
    }
    int r = p + 1;
    for (int q = dk + 1; q < ek; ++q) {
      const int j = ci[q];
      while (r < ei && ci[r] < j) ++r;
      if (r >= ei) break;
      if (ci[r] != j) continue;
      if constexpr (CP == 1) {
        a[r] = fm(-lr, a[q], a[r]);
      } else {
        const T ur = a[2 * (int64_t)q], ui = a[2 * (int64_t)q + 1];
        T re = fm(-lr, ur, a[2 * (int64_t)r]), im = fm(-lr, ui, a[2 * (int64_t)r + 1]);
        re = fm(li, ui, re);
        im = fm(-li, ur, im);
        a[2 * (int64_t)r] = re;
        a[2 * (int64_t)r + 1] = im;
      }
    }
  }
  __device__ void finish(int i) {
    const int d = diag[i];
    bool zero;
    if constexpr (CP == 1) zero = a[d] == T(0);
    else zero = a[2 * (int64_t)d] == T(0) && a[2 * (int64_t)d + 1] == T(0);
    if (zero) atomicMin(ctl + CTL_FAIL_ROW, i);
  }
};
constexpr int kIluEpoch = 1;  // substitution epochs are >= 2

template <typename T, int CP>
__global__ void __launch_bounds__(kBlock) k_ilu(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const int* __restrict__ diag, T* a, int* flags, int* ctl) {
  RowIlu<T, CP> row{rp, ci, diag, a, ctl};
  syncfree_rows(n, true, ci, flags, kIluEpoch, ctl + CTL_TICKET_LO, ctl, row);
}

__global__ void k_trsv_prep(int* ctl, unsigned long long* absmax, const int* done) {
  if (is_done(done)) return;
  ctl[CTL_EPOCH] += 2;
  ctl[CTL_TICKET_LO] = 0;
  ctl[CTL_TICKET_UP] = 0;
  *absmax = 0ull;
}

// ---------------------------------------------------------------------------------------------
// Conjugate transpose of a CSR matrix with CP values of type T per entry: counts, a single-
// block scan, scatter, then an insertion sort of every row so columns are ascending.
// ---------------------------------------------------------------------------------------------
__global__ void k_count_cols(int nnz, const int* __restrict__ ci, int* __restrict__ cnt) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += gridDim.x * blockDim.x) atomicAdd(cnt + ci[p], 1);
}
__global__ void k_scan_single(int n, const int* __restrict__ cnt, int* __restrict__ out) {  // out[0..n], blockDim 1024
  __shared__ int part[1024];
  const int t = threadIdx.x, T_ = blockDim.x;
  const int per = (n + T_ - 1) / T_;
  const int lo = t * per, hi = min(n, lo + per);
  int s = 0;
  for (int k = lo; k < hi; ++k) s += cnt[k];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int k = 0; k < T_; ++k) { int v = part[k]; part[k] = run; run += v; }
    out[n] = run;
  }
  __syncthreads();
  int run = part[t];
  for (int k = lo; k < hi; ++k) { out[k] = run; run += cnt[k]; }
}
__device__ __forceinline__ double conj_part(double x) { return -x; }
__device__ __forceinline__ float conj_part(float x) { return -x; }
__device__ __forceinline__ uint16_t conj_part(uint16_t x) { return (uint16_t)(x ^ 0x8000u); }
template <typename T, int CP>
__global__ void k_scatter_t(int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
                            const int* __restrict__ rpT, int* __restrict__ fill, int* __restrict__ ciT,
                            T* __restrict__ vT) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    const int dst = rpT[j] + atomicAdd(fill + j, 1);
    ciT[dst] = i;
    vT[(int64_t)dst * CP] = v[(int64_t)p * CP];
    if constexpr (CP == 2) vT[(int64_t)dst * CP + 1] = conj_part(v[(int64_t)p * CP + 1]);
  }
}
template <typename T, int CP>
__global__ void k_sort_rows(int n, const int* __restrict__ rp, int* __restrict__ ci, T* __restrict__ v,
                            int* __restrict__ diag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = rp[i], b = rp[i + 1];
  for (int p = a + 1; p < b; ++p) {
    const int c = ci[p];
    T x0 = v[(int64_t)p * CP], x1 = CP == 2 ? v[(int64_t)p * CP + 1] : T(0);
    int q = p - 1;
    while (q >= a && ci[q] > c) {
      ci[q + 1] = ci[q];
      v[(int64_t)(q + 1) * CP] = v[(int64_t)q * CP];
      if constexpr (CP == 2) v[(int64_t)(q + 1) * CP + 1] = v[(int64_t)q * CP + 1];
      --q;
    }
    ci[q + 1] = c;
    v[(int64_t)(q + 1) * CP] = x0;
    if constexpr (CP == 2) v[(int64_t)(q + 1) * CP + 1] = x1;
  }
  if (diag != nullptr) {
    int d = -1;
    for (int p = a; p < b; ++p)
      if (ci[p] == i) d = p;
    diag[i] = d;
  }
}

template <typename T, int CP>
static int transpose_t(int n, int nnz, const int* rp, const int* ci, const T* v, int* rpT, int* ciT, T* vT, int* diagT,
                       cudaStream_t s) {
  int* cnt = nullptr;
  MPK_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int) * (size_t)n * 2, s));
  int* fill = cnt + n;
  MPK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n * 2, s));
  k_count_cols<<<grid_for(nnz), kBlock, 0, s>>>(nnz, ci, cnt);
  k_scan_single<<<1, 1024, 0, s>>>(n, cnt, rpT);
  k_scatter_t<T, CP><<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(n, rp, ci, v, rpT, fill, ciT, vT);
  k_sort_rows<T, CP><<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(n, rpT, ciT, vT, diagT);
  MPK_CUDA(cudaFreeAsync(cnt, s));
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}

int transpose_matrix(const Csr& A, int* rpT, int* ciT, double* vT, cudaStream_t s) {
  if (A.cplx) return transpose_t<double, 2>(A.n, A.nnz, A.rp, A.ci, A.val, rpT, ciT, vT, nullptr, s);
  return transpose_t<double, 1>(A.n, A.nnz, A.rp, A.ci, A.val, rpT, ciT, vT, nullptr, s);
}

void launch_trsv_prep(const IluHandleView& M, const int* done, cudaStream_t s) {
  k_trsv_prep<<<1, 1, 0, s>>>(M.ctl, M.absmax, done);
}

static size_t fac_elem_size(int prec) { return prec == MPK_ILU_FP64 ? 8 : (prec == MPK_ILU_FP32 ? 4 : 2); }

static int build_transpose(mpk_ilu* M, cudaStream_t s) {
  if (M->rpT != nullptr) return MPK_OK;
  const size_t es = fac_elem_size(M->prec);
  MPK_CUDA(cudaMalloc((void**)&M->rpT, sizeof(int) * ((size_t)M->n + 1)));
  MPK_CUDA(cudaMalloc((void**)&M->ciT, sizeof(int) * (size_t)M->nnz));
  MPK_CUDA(cudaMalloc((void**)&M->diagT, sizeof(int) * (size_t)M->n));
  MPK_CUDA(cudaMalloc(&M->facT, es * (size_t)M->nnz * M->cp));
  int st;
  if (M->prec == MPK_ILU_FP64) {
    st = M->cp == 2 ? transpose_t<double, 2>(M->n, M->nnz, M->rp, M->ci, (const double*)M->fac, M->rpT, M->ciT,
                                             (double*)M->facT, M->diagT, s)
                    : transpose_t<double, 1>(M->n, M->nnz, M->rp, M->ci, (const double*)M->fac, M->rpT, M->ciT,
                                             (double*)M->facT, M->diagT, s);
  } else if (M->prec == MPK_ILU_FP32) {
    st = M->cp == 2 ? transpose_t<float, 2>(M->n, M->nnz, M->rp, M->ci, (const float*)M->fac, M->rpT, M->ciT,
                                            (float*)M->facT, M->diagT, s)
                    : transpose_t<float, 1>(M->n, M->nnz, M->rp, M->ci, (const float*)M->fac, M->rpT, M->ciT,
                                            (float*)M->facT, M->diagT, s);
  } else {
    st = M->cp == 2 ? transpose_t<uint16_t, 2>(M->n, M->nnz, M->rp, M->ci, (const uint16_t*)M->fac, M->rpT,
                                               M->ciT, (uint16_t*)M->facT, M->diagT, s)
                    : transpose_t<uint16_t, 1>(M->n, M->nnz, M->rp, M->ci, (const uint16_t*)M->fac, M->rpT,
                                               M->ciT, (uint16_t*)M->facT, M->diagT, s);
  }
  return st;
}

int prepare_trans(mpk_ilu* M, cudaStream_t s) { return build_transpose(M, s); }

// z = M^-1 r or M^-H r, stream-ordered; `done` may be null.
int precond_apply(const mpk_ilu* M, const Ops* o, bool trans, const double* r, double* z, const int* done,
                  cudaStream_t s) {
  if (trans && M->rpT == nullptr) return fail(MPK_INVALID_ARG, "M^H solve needs the transposed factor");
  const IluHandleView v = M->view(trans);
  launch_trsv_prep(v, done, s);
  int st;
  if (M->prec == MPK_ILU_FP64) {
    st = o->trsv_mp(v, true, !trans, r, M->vmp, done, s);
    if (st == MPK_OK) st = o->trsv_mp(v, false, trans, M->vmp, z, done, s);
  } else {
    o->absmax(M->n, r, v.absmax, done, s);
    st = o->trsv_lo32(v, !trans, r, done, s);
    if (st == MPK_OK) st = o->trsv_up32(v, trans, z, done, s);
  }
  if (st != MPK_OK) return fail(st, "substitution launch failed");
  return MPK_OK;
}

int read_ctl_err(const mpk_ilu* M, cudaStream_t s) {
  int err = 0;
  MPK_CUDA(cudaMemcpyAsync(&err, M->ctl + CTL_ERR, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  if (err != 0) return fail(err, "a bounded device wait ran out in a substitution kernel");
  return MPK_OK;
}

static void free_handle(mpk_ilu* M) {
  if (M == nullptr) return;
  void* ptrs[] = {M->rp, M->ci, M->diag, M->fac, M->rpT, M->ciT, M->diagT, M->facT, M->flags, M->ctl, M->v32, M->vmp,
                  M->absmax};
  for (void* p : ptrs)
    if (p != nullptr) cudaFree(p);
  delete M;
}

}  // namespace mpk

using namespace mpk;

IluHandleView mpk_ilu::view(bool trans) const {
  IluHandleView v;
  v.n = n;
  v.nnz = nnz;
  v.cp = cp;
  v.prec = prec;
  v.rp = trans ? rpT : rp;
  v.ci = trans ? ciT : ci;
  v.diag = trans ? diagT : diag;
  v.fac = trans ? facT : fac;
  v.flags = flags;
  v.ctl = ctl;
  v.v32 = v32;
  v.vmp = vmp;
  v.absmax = absmax;
  return v;
}

static int factor_impl(const mpk_csr* A, int prec, mpk_ilu** out, int* fail_row, cudaStream_t s) {
  const int n = A->n, nnz = A->nnz, cp = A->is_complex ? 2 : 1;
  int head[2] = {-1, -1};
  MPK_CUDA(cudaMemcpyAsync(&head[0], A->row_ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaMemcpyAsync(&head[1], A->row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  if (head[0] != 0 || head[1] != nnz) return fail(MPK_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] == nnz");

  mpk_ilu* M = new mpk_ilu();
  M->n = n;
  M->nnz = nnz;
  M->cp = cp;
  M->prec = prec;
  auto bail = [&](int st) {
    free_handle(M);
    return st;
  };
#define MPK_TRY(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return bail(fail(MPK_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_))); \
  } while (0)
  MPK_TRY(cudaMalloc((void**)&M->rp, sizeof(int) * ((size_t)n + 1)));
  MPK_TRY(cudaMalloc((void**)&M->ci, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1)));
  MPK_TRY(cudaMalloc((void**)&M->diag, sizeof(int) * (size_t)n));
  MPK_TRY(cudaMalloc((void**)&M->flags, sizeof(int) * (size_t)n));
  MPK_TRY(cudaMalloc((void**)&M->ctl, sizeof(int) * CTL_COUNT));
  MPK_TRY(cudaMalloc((void**)&M->absmax, sizeof(unsigned long long)));
  MPK_TRY(cudaMemcpyAsync(M->rp, A->row_ptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
  MPK_TRY(cudaMemcpyAsync(M->ci, A->col_idx, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, s));
  MPK_TRY(cudaMemsetAsync(M->flags, 0, sizeof(int) * (size_t)n, s));
  int ctl0[CTL_COUNT] = {0, 0, 0, 0, INT_MAX};
  MPK_TRY(cudaMemcpyAsync(M->ctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, s));
  int code = INT_MAX;
  MPK_TRY(cudaMemcpyAsync(M->ctl + CTL_FAIL_ROW, &code, sizeof(int), cudaMemcpyHostToDevice, s));
  // pattern check writes its code into CTL_FAIL_ROW (reset afterwards)
  k_check_pattern<<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(n, nnz, M->rp, M->ci, M->diag, M->ctl + CTL_FAIL_ROW);
  MPK_TRY(cudaGetLastError());
  MPK_TRY(cudaMemcpyAsync(&code, M->ctl + CTL_FAIL_ROW, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_TRY(cudaStreamSynchronize(s));
  if (code != INT_MAX) {
    if (fail_row) *fail_row = code / 2;
    return bail(fail((code & 1) ? MPK_MISSING_DIAG : MPK_INVALID_ARG,
                     (code & 1) ? "row without a stored diagonal" : "invalid CSR row (range or column order)"));
  }
  MPK_TRY(cudaMemcpyAsync(M->ctl, ctl0, sizeof(ctl0), cudaMemcpyHostToDevice, s));

  const int64_t m = (int64_t)nnz * cp;
  void* work = nullptr;  // factor in its computation type
  if (prec == MPK_ILU_FP64) {
    MPK_TRY(cudaMalloc(&work, sizeof(double) * (size_t)(m > 0 ? m : 1)));
    MPK_TRY(cudaMemcpyAsync(work, A->val, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s));
  } else {
    MPK_TRY(cudaMalloc(&work, sizeof(float) * (size_t)(m > 0 ? m : 1)));
    k_narrow<float><<<grid_for((int)((m + 3) / 4)), kBlock, 0, s>>>(m, A->val, (float*)work);
  }
  M->fac = work;
  static int blocks_d1 = persistent_blocks(k_ilu<double, 1>), blocks_d2 = persistent_blocks(k_ilu<double, 2>);
  static int blocks_f1 = persistent_blocks(k_ilu<float, 1>), blocks_f2 = persistent_blocks(k_ilu<float, 2>);
  if (prec == MPK_ILU_FP64) {
    if (cp == 1) k_ilu<double, 1><<<blocks_d1, kBlock, 0, s>>>(n, M->rp, M->ci, M->diag, (double*)work, M->flags, M->ctl);
    else k_ilu<double, 2><<<blocks_d2, kBlock, 0, s>>>(n, M->rp, M->ci, M->diag, (double*)work, M->flags, M->ctl);
  } else {
    if (cp == 1) k_ilu<float, 1><<<blocks_f1, kBlock, 0, s>>>(n, M->rp, M->ci, M->diag, (float*)work, M->flags, M->ctl);
    else k_ilu<float, 2><<<blocks_f2, kBlock, 0, s>>>(n, M->rp, M->ci, M->diag, (float*)work, M->flags, M->ctl);
  }
  MPK_TRY(cudaGetLastError());
  int ctl1[CTL_COUNT];
  MPK_TRY(cudaMemcpyAsync(ctl1, M->ctl, sizeof(ctl1), cudaMemcpyDeviceToHost, s));
  MPK_TRY(cudaStreamSynchronize(s));
  if (ctl1[CTL_ERR] != 0) return bail(fail(MPK_TIMEOUT, "a bounded device wait ran out in the ILU(0) kernel"));
  if (ctl1[CTL_FAIL_ROW] != INT_MAX) {
    if (fail_row) *fail_row = ctl1[CTL_FAIL_ROW];
    return bail(fail(MPK_ZERO_PIVOT, "zero pivot U_kk in ILU(0)"));
  }
  if (prec == MPK_ILU_BF16) {
    uint16_t* h = nullptr;
    MPK_TRY(cudaMalloc((void**)&h, sizeof(uint16_t) * (size_t)(m > 0 ? m : 1)));
    k_to_bf16<<<grid_for((int)((m + 3) / 4)), kBlock, 0, s>>>(m, (const float*)work, h);
    MPK_TRY(cudaGetLastError());
    MPK_TRY(cudaStreamSynchronize(s));
    cudaFree(work);
    M->fac = h;
  }
  if (prec == MPK_ILU_FP64) {
    MPK_TRY(cudaMalloc((void**)&M->vmp, sizeof(double) * (size_t)n * cp * 4));
  } else {
    MPK_TRY(cudaMalloc((void**)&M->v32, sizeof(float) * (size_t)n * cp));
  }
  MPK_TRY(cudaMemcpyAsync(M->ctl, ctl0, sizeof(int) * 4, cudaMemcpyHostToDevice, s));
  MPK_TRY(cudaStreamSynchronize(s));
#undef MPK_TRY
  *out = M;
  return MPK_OK;
}

extern "C" int mpk_ilu0_factor(const mpk_csr* A, int prec, mpk_ilu** out, int* fail_row, void* stream) {
  if (fail_row) *fail_row = -1;
  if (out) *out = nullptr;
  if (A == nullptr || out == nullptr) return fail(MPK_INVALID_ARG, "null argument");
  if (A->n < 1 || A->nnz < 0 || A->row_ptr == nullptr || (A->nnz > 0 && (A->col_idx == nullptr || A->val == nullptr)))
    return fail(MPK_INVALID_ARG, "invalid CSR descriptor");
  if (A->is_complex != 0 && A->is_complex != 1) return fail(MPK_INVALID_ARG, "is_complex must be 0 or 1");
  if (prec != MPK_ILU_FP64 && prec != MPK_ILU_FP32 && prec != MPK_ILU_BF16)
    return fail(MPK_INVALID_ARG, "prec must be MPK_ILU_FP64, MPK_ILU_FP32 or MPK_ILU_BF16");
  return factor_impl(A, prec, out, fail_row, (cudaStream_t)stream);
}

extern "C" int mpk_ilu0_values(const mpk_ilu* M, double* out_dev, void* stream) {
  if (M == nullptr || out_dev == nullptr) return fail(MPK_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t m = (int64_t)M->nnz * M->cp;
  if (m == 0) return MPK_OK;
  const int g = grid_for((int)((m + 3) / 4));
  if (M->prec == MPK_ILU_FP64) k_widen<double><<<g, kBlock, 0, s>>>(m, (const double*)M->fac, out_dev);
  else if (M->prec == MPK_ILU_FP32) k_widen<float><<<g, kBlock, 0, s>>>(m, (const float*)M->fac, out_dev);
  else k_widen<uint16_t><<<g, kBlock, 0, s>>>(m, (const uint16_t*)M->fac, out_dev);
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}

extern "C" int mpk_ilu0_prec(const mpk_ilu* M) { return M == nullptr ? -2 : M->prec; }

extern "C" void mpk_ilu0_destroy(mpk_ilu* M) { free_handle(M); }

extern "C" int mpk_precond_apply(const mpk_ilu* M, int w, int trans, const double* r_dev, double* z_dev,
                                 void* stream) {
  if (M == nullptr || r_dev == nullptr || z_dev == nullptr || r_dev == z_dev)
    return fail(MPK_INVALID_ARG, "null or aliased argument");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  cudaStream_t s = (cudaStream_t)stream;
  if (trans) {
    int st = build_transpose(const_cast<mpk_ilu*>(M), s);
    if (st != MPK_OK) return st;
  }
  const Ops* o = get_ops(w, M->cp);
  int st = precond_apply(M, o, trans != 0, r_dev, z_dev, nullptr, s);
  if (st != MPK_OK) return st;
  MPK_CUDA(cudaGetLastError());
  return read_ctl_err(M, s);
}
