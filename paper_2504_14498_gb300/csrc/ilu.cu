// ilu.cu -- ILU(0) factorisation (Algorithm 1) and the substitutions of Algorithm 2 as C-ABI
// entry points, plus the device transposition used by BiCG's M^H solve (Algorithm 3).
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

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

template <typename T, int CP, bool LONG = false>
struct RowIlu {
  // Rows of up to RI entries are held in registers while they are factored, and a finished row
  // k's pivot and first RK upper entries are fetched ahead of consume (Val), so that the
  // eliminations need no memory round trip per entry; longer rows take the memory path, with
  // the same operations in the same order.  LONG (matrices whose rows average more than RI
  // entries): the memory path only, without the registers of the short-row path, so that more
  // warps fit on an SM.
  static constexpr int RI = LONG ? 1 : 8, RK = LONG ? 1 : 4, kMG = 8;
  struct Val {
    int dk, ek;
    int uc[RK];       // columns of row k's upper entries dk+1 .. (-1 past its end)
    T uv[RK * CP];    // their values
    T piv[CP];        // U_kk
  };
  const int* rp;
  const int* ci;
  const int* diag;
  T* a;
  int* ctl;
  int i, p0, len;
  bool reg;          // row i is held in rc / rv
  int rc[RI];
  T rv[RI * CP];
  __device__ void begin(int i_, int& p, int& pend) {
    i = i_;
    p0 = rp[i_];
    len = rp[i_ + 1] - p0;
    reg = !LONG && len <= RI;
#pragma unroll
    for (int t = 0; t < RI; ++t) {
      rc[t] = -1;
#pragma unroll
      for (int h = 0; h < CP; ++h) rv[t * CP + h] = T(0);
      if (reg && t < len) {
        rc[t] = ci[p0 + t];
#pragma unroll
        for (int h = 0; h < CP; ++h) rv[t * CP + h] = a[(int64_t)(p0 + t) * CP + h];
      }
    }
    p = p0;
    pend = diag[i_];
  }
  __device__ Val load(int k) {
    Val v;
    v.dk = diag[k];
    v.ek = rp[k + 1];
#pragma unroll
    for (int h = 0; h < CP; ++h) v.piv[h] = a[(int64_t)v.dk * CP + h];
    if constexpr (!LONG) {
#pragma unroll
      for (int u = 0; u < RK; ++u) {
        const int q = v.dk + 1 + u;
        v.uc[u] = q < v.ek ? ci[q] : -1;
#pragma unroll
        for (int h = 0; h < CP; ++h) v.uv[u * CP + h] = q < v.ek ? a[(int64_t)q * CP + h] : T(0);
      }
    }
    return v;
  }
  // l = x / y in the factor's type, complex steps as documented above
  __device__ static void divide(const T* x, const T* y, T& lr, T& li) {
    if constexpr (CP == 1) {
      lr = x[0] / y[0];
      li = T(0);
    } else {
      const T den = fm(y[0], y[0], y[1] * y[1]), nr = fm(x[0], y[0], x[1] * y[1]), ni = fm(x[1], y[0], -(x[0] * y[1]));
      lr = nr / den;
      li = ni / den;
    }
  }
  // a := a - l * u
  __device__ static void update(T lr, T li, const T* u, T* av) {
    if constexpr (CP == 1) {
      av[0] = fm(-lr, u[0], av[0]);
    } else {
      T re = fm(-lr, u[0], av[0]), im = fm(-lr, u[1], av[1]);
      re = fm(li, u[1], re);
      im = fm(-li, u[0], im);
      av[0] = re;
      av[1] = im;
    }
  }
  __device__ void spill() {  // row i back to memory; the memory path continues from there
#pragma unroll
    for (int t = 0; t < RI; ++t)
      if (t < len)
#pragma unroll
        for (int h = 0; h < CP; ++h) a[(int64_t)(p0 + t) * CP + h] = rv[t * CP + h];
    reg = false;
  }
  __device__ void consume(int p, int k, const Val& vk) {
    if constexpr (!LONG) {
      if (reg && vk.ek - vk.dk - 1 > RK) spill();
    }
    if (!LONG && reg) {
      const int tk = p - p0;  // position of (i, k) in row i
      T x[CP];
#pragma unroll
      for (int t = 0; t < RI; ++t)
        if (t == tk)
#pragma unroll
          for (int h = 0; h < CP; ++h) x[h] = rv[t * CP + h];
      T lr, li;
      divide(x, vk.piv, lr, li);
#pragma unroll
      for (int t = 0; t < RI; ++t)
        if (t == tk) {
          rv[t * CP] = lr;
          if constexpr (CP == 2) rv[t * CP + 1] = li;
        }
#pragma unroll
      for (int u = 0; u < RK; ++u) {
        if (vk.uc[u] < 0) continue;
#pragma unroll
        for (int t = 0; t < RI; ++t)
          if (t > tk && t < len && rc[t] == vk.uc[u]) update(lr, li, vk.uv + u * CP, rv + t * CP);
      }
      return;
    }
    const int dk = vk.dk, ek = vk.ek, ei = rp[i + 1];
    T lr, li;
    {
      T x[CP];
#pragma unroll
      for (int h = 0; h < CP; ++h) x[h] = a[(int64_t)p * CP + h];
      divide(x, vk.piv, lr, li);
      a[(int64_t)p * CP] = lr;
      if constexpr (CP == 2) a[(int64_t)p * CP + 1] = li;
    }
    // row k's upper columns are loaded kMG at a time (one round trip per group instead of one per
    // entry), then merged with row i's remaining columns in ascending order as before
    int r = p + 1;
    for (int q0 = dk + 1; q0 < ek && r < ei; q0 += kMG) {
      int jq[kMG];
#pragma unroll
      for (int g = 0; g < kMG; ++g) jq[g] = q0 + g < ek ? ci[q0 + g] : INT_MAX;
#pragma unroll
      for (int g = 0; g < kMG; ++g) {
        const int j = jq[g];
        if (j == INT_MAX) break;
        while (r < ei && ci[r] < j) ++r;
        if (r >= ei) break;
        if (ci[r] != j) continue;
        const int q = q0 + g;
        T u[CP], av[CP];
#pragma unroll
        for (int h = 0; h < CP; ++h) {
          u[h] = a[(int64_t)q * CP + h];
          av[h] = a[(int64_t)r * CP + h];
        }
        update(lr, li, u, av);
#pragma unroll
        for (int h = 0; h < CP; ++h) a[(int64_t)r * CP + h] = av[h];
      }
    }
  }
  __device__ Val finish() {
    if (!LONG && reg) spill();
    const int d = diag[i];
    bool zero;
    if constexpr (CP == 1) zero = a[d] == T(0);
    else zero = a[2 * (int64_t)d] == T(0) && a[2 * (int64_t)d + 1] == T(0);
    if (zero) atomicMin(ctl + CTL_FAIL_ROW, i);
    return Val{};
  }
  __device__ void store(const Val&) {}
};

constexpr int kIluEpoch = 1;  // the substitutions use epochs >= 2 on the same chunk flags

template <typename T, int CP, bool LONG>
__global__ void __launch_bounds__(kBlock) k_ilu(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const int* __restrict__ diag, const LevelOrder lo, T* a, int* ctl) {
  RowIlu<T, CP, LONG> row;
  row.rp = rp;
  row.ci = ci;
  row.diag = diag;
  row.a = a;
  row.ctl = ctl;
  chunk_rows(lo, ci, kIluEpoch, ctl + CTL_TICKET_LO, ctl, row);
}

// The same rows level by level (level_rows): a cooperative launch, grid barriers between levels.
template <typename T, int CP, bool LONG>
__global__ void __launch_bounds__(kBlock) k_ilu_lv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const int* __restrict__ diag, const LevelOrder lo, T* a, int* ctl) {
  RowIlu<T, CP, LONG> row;
  row.rp = rp;
  row.ci = ci;
  row.diag = diag;
  row.a = a;
  row.ctl = ctl;
  level_rows(lo, ci, ctl, row);
}

// ILU(0) in w-component arithmetic (MPK_ILU_MP): the same row-IKJ dataflow, entries of CP * W
// doubles; for each k < i in row i, ascending: a_ik := a_ik / a_kk (the format's division), then
// a_ij := a_ij - a_ik * a_kj for every j > k of row k also in row i (product with a_ik first,
// then the subtraction, each rounded to W components).  Every entry receives the updates of the
// KIJ listing in its order, so the result is the sequential one bit for bit.
template <int W, int CP>
struct RowIluMp {
  using Val = Empty;
  const int* rp;
  const int* ci;
  const int* diag;
  double* a;
  int* ctl;
  int i;
  __device__ void begin(int i_, int& p, int& pend) {
    i = i_;
    p = rp[i_];
    pend = diag[i_];
  }
  __device__ Val load(int) { return Val{}; }
  __device__ void consume(int p, int k, const Val&) {
    const int dk = diag[k], ek = rp[k + 1], ei = rp[i + 1];
    const N<W, CP> l = n_div<W, CP>(n_load<W, CP>(a, p), n_load<W, CP>(a, dk));
    n_store<W, CP>(a, p, l);
    int r = p + 1;
    for (int q = dk + 1; q < ek; ++q) {
      const int j = ci[q];
      while (r < ei && ci[r] < j) ++r;
      if (r >= ei) break;
      if (ci[r] != j) continue;
      n_store<W, CP>(a, r, n_sub<W, CP>(n_load<W, CP>(a, r), n_mul<W, CP>(l, n_load<W, CP>(a, q))));
    }
  }
  __device__ Val finish() {
    if (n_is_zero<W, CP>(n_load<W, CP>(a, diag[i]))) atomicMin(ctl + CTL_FAIL_ROW, i);
    return Val{};
  }
  __device__ void store(const Val&) {}
};

template <int W, int CP>
__global__ void __launch_bounds__(kBlock) k_ilu_mp(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                   const int* __restrict__ diag, const LevelOrder lo, double* a,
                                                   int* ctl) {
  RowIluMp<W, CP> row;
  row.rp = rp;
  row.ci = ci;
  row.diag = diag;
  row.a = a;
  row.ctl = ctl;
  chunk_rows(lo, ci, kIluEpoch, ctl + CTL_TICKET_LO, ctl, row);
}

// A's binary64 values as w-component numbers: entry p, value t of CP (real, imaginary) goes to
// component 0 of its part, the other components are 0.
__global__ void k_to_mp(int64_t nnz, int cp, int w, const double* __restrict__ v, double* __restrict__ out) {
  const int64_t m = nnz * cp * w;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = k / (cp * w);
    const int r = (int)(k - p * cp * w), t = r / w, c = r - t * w;
    out[k] = c == 0 ? v[p * cp + t] : 0.0;
  }
}

template <int W, int CP>
__global__ void __launch_bounds__(kBlock) k_ilu_mp_lv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                      const int* __restrict__ diag, const LevelOrder lo, double* a,
                                                      int* ctl) {
  RowIluMp<W, CP> row;
  row.rp = rp;
  row.ci = ci;
  row.diag = diag;
  row.a = a;
  row.ctl = ctl;
  level_rows(lo, ci, ctl, row);
}

// Schedule of the ILU(0) kernels: level-synchronous (level_rows) or the dataflow over chunk flags
// (chunk_rows).  Both compute every row with the same operations in the same order: identical
// factors.  Measured on GB300: levels of a few hundred chunks (the 128^3 mesh: 382 levels of 172
// chunks on average) factor faster level by level (12.1 against 12.8 ms for the whole
// factorisation), while wide levels (the 512-system batch: 61 levels of ~10,000 chunks) want the
// dataflow, which overlaps consecutive levels (133 against 153 ms).  So the levels schedule is
// taken when a level averages no more chunks than the grid has warps; MPK_ILU_SCHEDULE=levels|
// dataflow, read at every factorisation, forces one.
static bool ilu_levels(int n, int nlev, int warps) {
  const char* e = std::getenv("MPK_ILU_SCHEDULE");
  if (e != nullptr && std::strcmp(e, "dataflow") == 0) return false;
  if (e != nullptr && std::strcmp(e, "levels") == 0) return true;
  return (double)n / (32.0 * (nlev > 0 ? nlev : 1)) <= (double)warps;
}
// One launch of the level-synchronous kernel `lv` (cooperative: its grid barriers need every
// block resident) or of the dataflow kernel `df`, over the lower level order.
template <typename T>
static int launch_ilu_kernel(const void* lv, const void* df, int blocks_lv, int blocks_df, int n, const int* rp,
                             const int* ci, const int* diag, LevelOrder lo, T* a, int* ctl, cudaStream_t s) {
  void* args[] = {(void*)&n, (void*)&rp, (void*)&ci, (void*)&diag, (void*)&lo, (void*)&a, (void*)&ctl};
  count_launch();
  if (ilu_levels(n, lo.nlev, blocks_lv * (kBlock / 32))) {
    MPK_CUDA(cudaMemsetAsync(ctl + CTL_BAR_COUNT, 0, sizeof(int), s));
    MPK_CUDA(cudaLaunchCooperativeKernel(lv, dim3(blocks_lv), dim3(kBlock), args, 0, s));
  } else {
    MPK_CUDA(cudaMemsetAsync(ctl + CTL_TICKET_LO, 0, sizeof(int), s));
    MPK_CUDA(cudaLaunchKernel(df, dim3(blocks_df), dim3(kBlock), args, 0, s));
  }
  return MPK_OK;
}
// long_rows: rows average more than RowIlu's register capacity (the memory-path-only kernels)
template <typename T, int CP>
static int launch_ilu(int n, int nnz, const int* rp, const int* ci, const int* diag, const LevelOrder& lo, T* a,
                      int* ctl, cudaStream_t s) {
  if ((int64_t)nnz > (int64_t)RowIlu<T, CP>::RI * n) {
    static const int blv = persistent_blocks(k_ilu_lv<T, CP, true>), bdf = persistent_blocks(k_ilu<T, CP, true>);
    return launch_ilu_kernel<T>((const void*)k_ilu_lv<T, CP, true>, (const void*)k_ilu<T, CP, true>, blv, bdf, n, rp,
                                ci, diag, lo, a, ctl, s);
  }
  static const int blv = persistent_blocks(k_ilu_lv<T, CP, false>), bdf = persistent_blocks(k_ilu<T, CP, false>);
  return launch_ilu_kernel<T>((const void*)k_ilu_lv<T, CP, false>, (const void*)k_ilu<T, CP, false>, blv, bdf, n, rp,
                              ci, diag, lo, a, ctl, s);
}
template <int W, int CP>
static int launch_ilu_mp_wc(int n, const int* rp, const int* ci, const int* diag, const LevelOrder& lo, double* a,
                            int* ctl, cudaStream_t s) {
  static const int blv = persistent_blocks(k_ilu_mp_lv<W, CP>), bdf = persistent_blocks(k_ilu_mp<W, CP>);
  return launch_ilu_kernel<double>((const void*)k_ilu_mp_lv<W, CP>, (const void*)k_ilu_mp<W, CP>, blv, bdf, n, rp,
                                   ci, diag, lo, a, ctl, s);
}
static int launch_ilu_mp(int w, int cp, int n, const int* rp, const int* ci, const int* diag, const LevelOrder& lo,
                         double* a, int* ctl, cudaStream_t s) {
  switch (w * 2 + cp - 1) {
    case 2: return launch_ilu_mp_wc<1, 1>(n, rp, ci, diag, lo, a, ctl, s);
    case 3: return launch_ilu_mp_wc<1, 2>(n, rp, ci, diag, lo, a, ctl, s);
    case 4: return launch_ilu_mp_wc<2, 1>(n, rp, ci, diag, lo, a, ctl, s);
    case 5: return launch_ilu_mp_wc<2, 2>(n, rp, ci, diag, lo, a, ctl, s);
    case 6: return launch_ilu_mp_wc<3, 1>(n, rp, ci, diag, lo, a, ctl, s);
    case 7: return launch_ilu_mp_wc<3, 2>(n, rp, ci, diag, lo, a, ctl, s);
    case 8: return launch_ilu_mp_wc<4, 1>(n, rp, ci, diag, lo, a, ctl, s);
    default: return launch_ilu_mp_wc<4, 2>(n, rp, ci, diag, lo, a, ctl, s);
  }
}

// New epoch pair (lower: even, upper: odd) and reset tickets and the scale accumulator.
__global__ void k_trsv_prep(int* ctl, unsigned long long* absmax, const int* done) {
  if (is_done(done)) return;
  ctl[CTL_EPOCH] += 2;
  ctl[CTL_TICKET_LO] = 0;
  ctl[CTL_TICKET_UP] = 0;
  *absmax = 0ull;
}

constexpr unsigned kDepthEpoch0 = 0x40000000u;  // epochs of the ordering passes, distinct from others

// counts per depth; cnt[L] (L = array length - 1, passed as maxslot) collects the largest depth
// Levels below kHistBins are counted per block in shared memory and added once per block (a few
// dozen levels over millions of rows would otherwise serialise on a few global counters).
constexpr int kHistBins = 4096;
__global__ void k_depth_count(int m, const int* __restrict__ depth, int* __restrict__ cnt, int* __restrict__ maxd) {
  __shared__ int h[kHistBins];
  for (int t = threadIdx.x; t < kHistBins; t += blockDim.x) h[t] = 0;
  __syncthreads();
  int mx = 0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
    const int d = depth[c];
    if (d < kHistBins) atomicAdd(&h[d], 1);
    else atomicAdd(cnt + d, 1);
    mx = max(mx, d);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kHistBins; t += blockDim.x)
    if (h[t] != 0) atomicAdd(cnt + t, h[t]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) atomicMax(maxd, mx);
}
__global__ void k_scan_single(int n, const int* __restrict__ cnt, int* __restrict__ out);

// Fingerprint of a sparsity pattern (row pointers and column indices): the XOR over all entries
// of a 64-bit mix (splitmix64's finaliser) of (array, position, value).  Order-independent, so a
// grid-stride loop with atomic XOR gives the same value every time; two patterns that differ
// anywhere differ in their fingerprints except with probability about 2^-64.
__device__ __forceinline__ unsigned long long fp_mix(unsigned long long z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
__global__ void k_pattern_fp(int n, int nnz, const int* __restrict__ rp, const int* __restrict__ ci,
                             unsigned long long* __restrict__ out) {
  unsigned long long h = 0ull;
  const int64_t total = (int64_t)n + 1 + nnz;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const bool is_rp = k <= n;
    const unsigned v = (unsigned)(is_rp ? rp[k] : ci[k - n - 1]);
    h ^= fp_mix(((unsigned long long)k << 32) ^ v ^ (is_rp ? 0ull : 0x8000000000000000ull));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) h ^= __shfl_xor_sync(0xffffffffu, h, off);
  if ((threadIdx.x & 31) == 0 && h != 0ull) atomicXor(out, h);
}
int pattern_fingerprint(int n, int nnz, const int* rp, const int* ci, uint64_t* out, cudaStream_t s) {
  unsigned long long* d = nullptr;
  MPK_CUDA(cudaMallocAsync((void**)&d, sizeof(unsigned long long), s));
  MPK_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), s));
  count_launch();
  const int64_t total = (int64_t)n + 1 + nnz;
  int g = (int)((total + kBlock - 1) / kBlock);
  if (g > sm_count() * 8) g = sm_count() * 8;
  k_pattern_fp<<<g < 1 ? 1 : g, kBlock, 0, s>>>(n, nnz, rp, ci, d);
  unsigned long long h = 0ull;
  MPK_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaFreeAsync(d, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  *out = (uint64_t)h;
  return MPK_OK;
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
// Entries of S values each; the last NNEG of them (the imaginary components) change sign.
template <typename T, int S, int NNEG>
__global__ void k_scatter_t(int n, const int* __restrict__ rp, const int* __restrict__ ci, const T* __restrict__ v,
                            const int* __restrict__ rpT, int* __restrict__ fill, int* __restrict__ ciT,
                            T* __restrict__ vT) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int p = rp[i]; p < rp[i + 1]; ++p) {
    const int j = ci[p];
    const int dst = rpT[j] + atomicAdd(fill + j, 1);
    ciT[dst] = i;
#pragma unroll
    for (int t = 0; t < S; ++t) {
      const T x = v[(int64_t)p * S + t];
      vT[(int64_t)dst * S + t] = t >= S - NNEG ? conj_part(x) : x;
    }
  }
}
template <typename T, int S>
__global__ void k_sort_rows(int n, const int* __restrict__ rp, int* __restrict__ ci, T* __restrict__ v,
                            int* __restrict__ diag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = rp[i], b = rp[i + 1];
  for (int p = a + 1; p < b; ++p) {
    const int c = ci[p];
    T x[S];
#pragma unroll
    for (int t = 0; t < S; ++t) x[t] = v[(int64_t)p * S + t];
    int q = p - 1;
    while (q >= a && ci[q] > c) {
      ci[q + 1] = ci[q];
#pragma unroll
      for (int t = 0; t < S; ++t) v[(int64_t)(q + 1) * S + t] = v[(int64_t)q * S + t];
      --q;
    }
    ci[q + 1] = c;
#pragma unroll
    for (int t = 0; t < S; ++t) v[(int64_t)(q + 1) * S + t] = x[t];
  }
  if (diag != nullptr) {
    int d = -1;
    for (int p = a; p < b; ++p)
      if (ci[p] == i) d = p;
    diag[i] = d;
  }
}

// Conjugate transpose of a CSR matrix whose entries hold S values, the last NNEG negated.
template <typename T, int S, int NNEG>
static int transpose_t(int n, int nnz, const int* rp, const int* ci, const T* v, int* rpT, int* ciT, T* vT, int* diagT,
                       cudaStream_t s) {
  int* cnt = nullptr;
  MPK_CUDA(cudaMallocAsync((void**)&cnt, sizeof(int) * (size_t)n * 2, s));
  int* fill = cnt + n;
  MPK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n * 2, s));
  count_launch(4);  // count, scan, scatter, sort
  k_count_cols<<<grid_for(nnz), kBlock, 0, s>>>(nnz, ci, cnt);
  k_scan_single<<<1, 1024, 0, s>>>(n, cnt, rpT);
  k_scatter_t<T, S, NNEG><<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(n, rp, ci, v, rpT, fill, ciT, vT);
  k_sort_rows<T, S><<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(n, rpT, ciT, vT, diagT);
  MPK_CUDA(cudaFreeAsync(cnt, s));
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}

int transpose_matrix(const Csr& A, int* rpT, int* ciT, double* vT, cudaStream_t s) {
  if (A.cplx) return transpose_t<double, 2, 1>(A.n, A.nnz, A.rp, A.ci, A.val, rpT, ciT, vT, nullptr, s);
  return transpose_t<double, 1, 0>(A.n, A.nnz, A.rp, A.ci, A.val, rpT, ciT, vT, nullptr, s);
}

// Level of every row of one triangle: 0 without dependencies, else 1 + the largest level of the
// rows it depends on; computed by the dependency-driven scheme over the chunk order.
struct RowDepth {
  using Val = int;
  const int* rp;
  const int* diag;
  bool lower;
  unsigned long long* pk;
  unsigned epoch;
  int* depth;
  int i, d;
  __device__ void begin(int i_, int& p, int& pend) {
    i = i_;
    d = 0;
    if (lower) { p = rp[i_]; pend = diag[i_]; }
    else { p = diag[i_] + 1; pend = rp[i_ + 1]; }
  }
  static constexpr int kLook = 3;  // a 7-point row's 3 entries per triangle; 32 registers in all
  static constexpr int kBatch = 0;
  struct Raw { unsigned long long w; };
  __device__ void issue(int j, Raw& r) { r.w = ld_relaxed_u64(pk + j); }
  __device__ bool check(int, const Raw& r, Val& v) {
    if ((unsigned)(r.w >> 32) != epoch) return false;
    v = (int)(unsigned)r.w;
    return true;
  }
  __device__ void consume(int, int, const Val& v) { d = max(d, v + 1); }
  __device__ Val finish() { return d; }
  __device__ void publish(const Val& v) {
    depth[i] = v;
    st_relaxed_u64(pk + i, ((unsigned long long)epoch << 32) | (unsigned)v);
  }
};
// Both triangles at once: the first half of the blocks runs the lower triangle's pass, the second
// half the upper one's, each with its own order, ticket, packed words and result (the two passes
// are independent; each half's warps are resident, so each pass progresses as alone).
struct DepthPass {
  Order ord;
  unsigned long long* pk;
  unsigned epoch;
  int* depth;
  int* ticket;
};
__global__ void __launch_bounds__(kBlock, 8) k_row_depth(DepthPass lo_pass, DepthPass up_pass, const int* __restrict__ ci,
                                                      const int* __restrict__ rp, const int* __restrict__ diag,
                                                      int* ctl) {
  const bool lower = blockIdx.x < (gridDim.x >> 1);
  const DepthPass& P = lower ? lo_pass : up_pass;
  RowDepth row;
  row.rp = rp;
  row.diag = diag;
  row.lower = lower;
  row.pk = P.pk;
  row.epoch = P.epoch;
  row.depth = P.depth;
  syncfree_rows(P.ord, ci, P.ticket, ctl, row);
}
// Natural row order of a triangle as an Order: position q holds row q (lower) or n-1-q (upper).
__global__ void k_natural_order(int n, bool lower, int npos, int* __restrict__ perm, int* __restrict__ pos) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < npos; q += gridDim.x * blockDim.x) {
    if (q < n) {
      const int row = lower ? q : n - 1 - q;
      perm[q] = row;
      pos[row] = q;
    } else {
      perm[q] = -1;
    }
  }
}
__global__ void k_inverse(int n, const int* __restrict__ perm, int* __restrict__ pos) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) pos[perm[q]] = q;
}

size_t level_buf_ints(int n, int nlevels) {
  const size_t P = (size_t)n + 32 * (size_t)nlevels;
  return P + (size_t)n + (P / 32 + 1) + 1 + (size_t)nlevels + 1;
}
LevelOrder level_view(int* buf, int n, int nlevels) {
  const size_t P = (size_t)n + 32 * (size_t)nlevels;
  LevelOrder o;
  o.perm = buf;
  o.pos = buf + P;
  o.flags = buf + P + n;
  o.nchunks = buf + P + n + (P / 32 + 1);
  o.lstart = o.nchunks + 1;
  o.nlev = nlevels;
  return o;
}

// Level layout: level_size = cnt, padded starts (exclusive scan of 32-rounded sizes, in `off`),
// each level's first chunk (lstart) and nchunks; one block of 1024 threads.
__global__ void k_level_layout(int nlevels, const int* __restrict__ cnt, int* __restrict__ off, LevelOrder lo) {
  __shared__ int part[1024];
  const int t = threadIdx.x, T_ = blockDim.x;
  const int per = (nlevels + T_ - 1) / T_;
  const int lo_ = min(nlevels, t * per), hi = min(nlevels, lo_ + per);
  int s = 0;
  for (int k = lo_; k < hi; ++k) s += (cnt[k] + 31) & ~31;
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int k = 0; k < T_; ++k) { int v = part[k]; part[k] = run; run += v; }
    *const_cast<int*>(lo.nchunks) = run / 32;
    const_cast<int*>(lo.lstart)[nlevels] = run / 32;
  }
  __syncthreads();
  int run = part[t];
  for (int k = lo_; k < hi; ++k) {
    off[k] = run;
    const_cast<int*>(lo.lstart)[k] = run / 32;
    run += (cnt[k] + 31) & ~31;
  }
}
// Within a level the rows are sorted by their length in the triangle (longest first, lengths
// bucketed by kLenB): the 32 rows of a chunk then have similar lengths and the repacked chunk few
// padding slots.  key = level * kLenB + (kLenB - 1 - min(len, kLenB - 1)).
constexpr int kLenB = 32;
__device__ __forceinline__ int tri_len(const int* rp, const int* diag, bool lower, int i) {
  return lower ? diag[i] - rp[i] : rp[i + 1] - diag[i] - 1;
}
__global__ void k_key_count(int n, const int* __restrict__ depth, const int* __restrict__ rp,
                            const int* __restrict__ diag, bool lower, int* __restrict__ cnt2) {
  __shared__ int h[kHistBins];  // keys below kHistBins counted per block first
  for (int t = threadIdx.x; t < kHistBins; t += blockDim.x) h[t] = 0;
  __syncthreads();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int key = depth[i] * kLenB + (kLenB - 1 - min(tri_len(rp, diag, lower, i), kLenB - 1));
    if (key < kHistBins) atomicAdd(&h[key], 1);
    else atomicAdd(cnt2 + key, 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kHistBins; t += blockDim.x)
    if (h[t] != 0) atomicAdd(cnt2 + t, h[t]);
}
__global__ void k_key_offsets(int nlevels, const int* __restrict__ off, const int* __restrict__ cnt2,
                              int* __restrict__ sub) {
  for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < nlevels; d += gridDim.x * blockDim.x) {
    int run = off[d];
    for (int b = 0; b < kLenB; ++b) {
      sub[d * kLenB + b] = run;
      run += cnt2[d * kLenB + b];
    }
  }
}
__global__ void k_level_scatter(int n, const int* __restrict__ depth, const int* __restrict__ rp,
                                const int* __restrict__ diag, bool lower, int* __restrict__ sub,
                                int* __restrict__ perm, int* __restrict__ pos) {
  // the lanes of a warp with equal keys take their positions with one reservation (the order
  // inside a key's group is arbitrary either way)
  const int lane = threadIdx.x & 31;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int key = depth[i] * kLenB + (kLenB - 1 - min(tri_len(rp, diag, lower, i), kLenB - 1));
    const unsigned peers = __match_any_sync(__activemask(), key);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(sub + key, __popc(peers));
    base = __shfl_sync(peers, base, leader);
    const int q = base + __popc(peers & ((1u << lane) - 1u));
    perm[q] = i;
    pos[i] = q;
  }
}

// Level orders of the two triangles of (rp, ci, diag) into bufs[0] (lower) and bufs[1] (upper),
// allocated here.  Row levels come from the dependency-driven pass over the natural row order
// (every row depends on earlier rows only: a valid order for it), then a counting sort by
// (level, length) places them, every level padded to whole 32-row chunks.
static int build_levels(int n, const int* rp, const int* ci, const int* diag, unsigned long long* pk, int* ctl,
                        int which, int** bufs, int* nlev, int** depths, cudaStream_t s) {
  const int m = (n + 31) >> 5;
  const size_t L = (size_t)n + 1;
  // per triangle: level counts (L), natural order perm (32 m) and pos (n), largest level (1);
  // packed words of the upper pass (the lower pass uses pk)
  int* tmp = nullptr;
  const size_t per = L + (size_t)m * 32 + (size_t)n + 1;
  MPK_CUDA(cudaMallocAsync((void**)&tmp, sizeof(int) * (2 * per + 16) + sizeof(unsigned long long) * L, s));
  int* cnt[2];
  int* perm_c[2];
  int* pos_c[2];
  int* maxd[2];
  for (int tri = 0; tri < 2; ++tri) {
    int* base = tmp + tri * per;
    cnt[tri] = base;
    perm_c[tri] = base + L;
    pos_c[tri] = perm_c[tri] + (size_t)m * 32;
    maxd[tri] = pos_c[tri] + n;
  }
  unsigned long long* pk_up = (unsigned long long*)(((uintptr_t)(tmp + 2 * per + 8)) & ~(uintptr_t)7);
  MPK_CUDA(cudaMemsetAsync(tmp, 0, sizeof(int) * 2 * per, s));
  MPK_CUDA(cudaMemsetAsync(pk_up, 0, sizeof(unsigned long long) * L, s));
  MPK_CUDA(cudaMemsetAsync(ctl + CTL_TICKET_LO, 0, sizeof(int) * 2, s));  // CTL_TICKET_LO, CTL_TICKET_UP
  DepthPass pass[2];
  for (int tri = 0; tri < 2; ++tri) {
    int* depth = nullptr;  // kept: the owner-block layout groups rows by level
    MPK_CUDA(cudaMalloc((void**)&depth, sizeof(int) * L));
    depths[tri] = depth;
    count_launch();
    k_natural_order<<<grid_for(m * 32), kBlock, 0, s>>>(n, tri == 0, m * 32, perm_c[tri], pos_c[tri]);
    pass[tri].ord.perm = perm_c[tri];
    pass[tri].ord.pos = pos_c[tri];
    pass[tri].ord.npos = m * 32;
    pass[tri].pk = tri == 0 ? pk : pk_up;
    pass[tri].epoch = kDepthEpoch0 + 4u * which + 2u + tri;
    pass[tri].depth = depth;
    pass[tri].ticket = ctl + (tri == 0 ? CTL_TICKET_LO : CTL_TICKET_UP);
  }
  // The pass is bound by its window of rows in flight (it follows the natural row order, in which
  // the rows that are ready at any moment are spread over the whole matrix), so it runs as many
  // warps as fit: 32 registers a thread, 64 warps per SM.  Even: two halves.
  static int blocks_rd = [] {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_row_depth, kBlock, 0) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    return (per_sm * sm_count() + 1) & ~1;
  }();
  count_launch(3);
  k_row_depth<<<blocks_rd, kBlock, 0, s>>>(pass[0], pass[1], ci, rp, diag, ctl);
  for (int tri = 0; tri < 2; ++tri) k_depth_count<<<grid_for(n), kBlock, 0, s>>>(n, depths[tri], cnt[tri], maxd[tri]);
  int hmax[2] = {0, 0}, herr = 0;
  MPK_CUDA(cudaMemcpyAsync(&hmax[0], maxd[0], sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaMemcpyAsync(&hmax[1], maxd[1], sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaMemcpyAsync(&herr, ctl + CTL_ERR, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  if (herr != 0) {
    cudaFreeAsync(tmp, s);
    return fail(MPK_TIMEOUT, "a bounded device wait ran out while ordering the triangles");
  }
  for (int tri = 0; tri < 2; ++tri) {
    const bool lower = tri == 0;
    const int nl = hmax[tri] + 1;
    int* depth = depths[tri];
    int* buf = nullptr;
    MPK_CUDA(cudaMalloc((void**)&buf, sizeof(int) * level_buf_ints(n, nl)));
    const LevelOrder lo = level_view(buf, n, nl);
    const size_t P = (size_t)n + 32 * (size_t)nl;
    MPK_CUDA(cudaMemsetAsync(buf, 0xff, sizeof(int) * P, s));  // padding positions: -1
    MPK_CUDA(cudaMemsetAsync(lo.flags, 0, sizeof(int) * (P / 32 + 1), s));
    int* keys = nullptr;  // off[nl] | cnt2[nl*kLenB] | sub[nl*kLenB]
    MPK_CUDA(cudaMallocAsync((void**)&keys, sizeof(int) * ((size_t)nl * (2 * kLenB + 1)), s));
    int* off = keys;
    int* cnt2 = off + nl;
    int* sub = cnt2 + (size_t)nl * kLenB;
    MPK_CUDA(cudaMemsetAsync(cnt2, 0, sizeof(int) * (size_t)nl * kLenB, s));
    count_launch(4);
    k_level_layout<<<1, 1024, 0, s>>>(nl, cnt[tri], off, lo);
    k_key_count<<<grid_for(n), kBlock, 0, s>>>(n, depth, rp, diag, lower, cnt2);
    k_key_offsets<<<(nl + 255) / 256, 256, 0, s>>>(nl, off, cnt2, sub);
    k_level_scatter<<<grid_for(n), kBlock, 0, s>>>(n, depth, rp, diag, lower, sub, buf, const_cast<int*>(lo.pos));
    MPK_CUDA(cudaFreeAsync(keys, s));
    bufs[tri] = buf;
    nlev[tri] = nl;
  }
  MPK_CUDA(cudaMemsetAsync(ctl + CTL_TICKET_LO, 0, sizeof(int) * 2, s));
  MPK_CUDA(cudaGetLastError());
  MPK_CUDA(cudaFreeAsync(tmp, s));
  return MPK_OK;
}

// ---------------------------------------------------------------------------------------------
// Repacking of a binary64 triangle into the SELL-32 layout of the static substitution schedule
// (see SellTri): one warp per chunk computes its width (the longest row of the triangle among
// its 32 rows), a scan gives the slot-block offsets, then every position copies its row.
// ---------------------------------------------------------------------------------------------
__global__ void k_sell_width(int nchunks, const int* __restrict__ perm, const int* __restrict__ rp,
                             const int* __restrict__ diag, bool lower, int* __restrict__ width) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += warps) {
    const int i = perm[c * 32 + lane];
    int len = 0;
    if (i >= 0) len = lower ? diag[i] - rp[i] : rp[i + 1] - diag[i] - 1;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) len = max(len, __shfl_xor_sync(0xffffffffu, len, off));
    if (lane == 0) width[c] = len;
  }
}
// Also records, per chunk, the dependency with the largest level-order position (rep): the
// substitution polls that one value before checking all the others.  The 32 positions of a chunk
// are the 32 lanes of one warp (blockDim and the stride are multiples of 32).
// Owner-block layout (enc.blk != nullptr): a dependency on a row of the same block whose value
// is still in the block's ring when this row's group runs (its position + kRing reaches the end
// of the group, enc.cgend of the chunk) is encoded as -2 - ring slot and left out of rep.
struct ObEnc {
  const int* blk = nullptr;      // row -> owner block
  const int* bstart = nullptr;   // block -> first position
  const int* cgend = nullptr;    // chunk -> end position of its group
  const int* cgstart = nullptr;  // chunk -> first chunk of its group (the CTA of a chunk in a cluster)
  int csize = 1;                 // CTAs per block
};
__device__ __forceinline__ double one_of(double) { return 1.0; }
__device__ __forceinline__ float one_of(float) { return 1.0f; }
__device__ __forceinline__ uint16_t one_of(uint16_t) { return (uint16_t)0x3F80u; }  // bfloat16 1.0
template <typename T, int CP>
__global__ void k_sell_fill(int nchunks, const int* __restrict__ perm, const int* __restrict__ pos,
                            const int* __restrict__ rp, const int* __restrict__ ci, const int* __restrict__ diag,
                            const T* __restrict__ fac, bool lower, const int* __restrict__ coff, ObEnc enc,
                            int* __restrict__ col, T* __restrict__ val, T* __restrict__ dia, int* __restrict__ rep) {
  const int64_t P = (int64_t)nchunks * 32;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < P; q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q >> 5), lane = (int)(q & 31);
    const int i = perm[q];
    int p = 0, len = 0;
    if (i >= 0) {
      p = lower ? rp[i] : diag[i] + 1;
      len = lower ? diag[i] - rp[i] : rp[i + 1] - diag[i] - 1;
    }
    const int b0 = coff[c], w = coff[c + 1] - b0;
    const int bi = (enc.blk != nullptr && i >= 0) ? enc.blk[i] : -1;
    const int gend = enc.blk != nullptr ? enc.cgend[c] : 0;
    int last = -1;
    // four entries at a time: their columns, then the columns' positions and the values, each
    // loaded together (a chain of dependent loads per entry otherwise)
    for (int k0 = 0; k0 < w; k0 += 4) {
      int j4[4], q4[4];
      T v4[4][CP];
#pragma unroll
      for (int u = 0; u < 4; ++u) j4[u] = k0 + u < len ? ci[p + k0 + u] : -1;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        q4[u] = j4[u] >= 0 ? pos[j4[u]] : -1;
#pragma unroll
        for (int t = 0; t < CP; ++t) v4[u][t] = j4[u] >= 0 ? fac[(int64_t)(p + k0 + u) * CP + t] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = k0 + u;
        if (k >= w) break;
        const int64_t e = ((int64_t)(b0 + k) << 5) + lane;
        int cv = -1;
        if (k < len) {
          const int j = j4[u], qj = q4[u];
          if (bi >= 0 && enc.blk[j] == bi && qj + kRing >= gend) {
            const int rank = ((qj >> 5) - enc.cgstart[qj >> 5]) % enc.csize;
            cv = -2 - (rank * kRing + (qj - enc.bstart[bi]) % kRing);
          } else {
            cv = j;
            last = max(last, qj);
          }
        }
        col[e] = cv;
#pragma unroll
        for (int t = 0; t < CP; ++t) val[e * CP + t] = v4[u][t];
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) last = max(last, __shfl_xor_sync(0xffffffffu, last, off));
    if (lane == 0) rep[c] = last >= 0 ? perm[last] : -1;
#pragma unroll
    for (int t = 0; t < CP; ++t) dia[q * CP + t] = i >= 0 ? fac[(int64_t)diag[i] * CP + t] : (t == 0 ? one_of(T(0)) : T(0));
  }
}

// Repack one triangle of (rp, ci, diag, fac) in the positions of the order (perm, pos, nch
// chunks) into *buf (allocated here) and describe it in *out; cp values of type T per entry.
template <typename T>
static int build_sell(int n, int cp, const int* rp, const int* ci, const int* diag, const T* fac, const int* perm,
                      const int* pos, int nch, bool lower, const ObEnc& enc, void** buf, SellTri* out,
                      cudaStream_t s) {
  (void)n;
  int* width = nullptr;
  MPK_CUDA(cudaMallocAsync((void**)&width, sizeof(int) * ((size_t)nch + 1) * 2, s));
  int* coff_tmp = width + nch + 1;
  count_launch(2);
  k_sell_width<<<grid_for(nch * 32), kBlock, 0, s>>>(nch, perm, rp, diag, lower, width);
  k_scan_single<<<1, 1024, 0, s>>>(nch, width, coff_tmp);
  int total = 0;
  MPK_CUDA(cudaMemcpyAsync(&total, coff_tmp + nch, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  const size_t slots = (size_t)total * 32;
  const size_t coff_b = ((sizeof(int) * ((size_t)nch + 1)) + 255) & ~(size_t)255;
  const size_t col_b = ((sizeof(int) * slots) + 255) & ~(size_t)255;
  const size_t val_b = ((sizeof(T) * slots * cp) + 255) & ~(size_t)255;
  const size_t dia_b = ((sizeof(T) * (size_t)nch * 32 * cp) + 255) & ~(size_t)255;
  const size_t rep_b = sizeof(int) * (size_t)nch;
  char* b = nullptr;
  MPK_CUDA(cudaMalloc((void**)&b, coff_b + col_b + val_b + dia_b + rep_b + 256));
  int* coff = (int*)b;
  int* col = (int*)(b + coff_b);
  T* val = (T*)(b + coff_b + col_b);
  T* dia = (T*)(b + coff_b + col_b + val_b);
  int* rep = (int*)(b + coff_b + col_b + val_b + dia_b);
  MPK_CUDA(cudaMemcpyAsync(coff, coff_tmp, sizeof(int) * ((size_t)nch + 1), cudaMemcpyDeviceToDevice, s));
  count_launch();
  const int g = grid_for(nch * 32);
#define MPK_SELL_FILL(CPX) \
  k_sell_fill<T, CPX><<<g, kBlock, 0, s>>>(nch, perm, pos, rp, ci, diag, fac, lower, coff, enc, col, val, dia, rep)
  switch (cp) {  // values per entry: c, or c * w for a w-component factor
    case 1: MPK_SELL_FILL(1); break;
    case 2: MPK_SELL_FILL(2); break;
    case 3: MPK_SELL_FILL(3); break;
    case 4: MPK_SELL_FILL(4); break;
    case 6: MPK_SELL_FILL(6); break;
    case 8: MPK_SELL_FILL(8); break;
    default: cudaFree(b); cudaFreeAsync(width, s); return fail(MPK_INVALID_ARG, "unsupported values per entry");
  }
#undef MPK_SELL_FILL
  MPK_CUDA(cudaGetLastError());
  MPK_CUDA(cudaFreeAsync(width, s));
  *buf = b;
  out->perm = perm;
  out->coff = coff;
  out->col = col;
  out->val = val;
  out->dia = dia;
  out->rep = rep;
  out->nchunks = nch;
  return MPK_OK;
}

// ---------------------------------------------------------------------------------------------
// Owner-block order of one triangle (see SellTri): rows are dealt to the B blocks of the
// substitution grid in contiguous ranges of equal work (row length + 1), then grouped by
// (block, level), each group padded to whole chunks; inside a group rows keep no particular
// order.  Keys k = block * nlevels + level; counts, padded offsets and group numbers by scans.
// ---------------------------------------------------------------------------------------------
__global__ void k_ob_work(int n, const int* __restrict__ rp, const int* __restrict__ diag, bool lower,
                          int* __restrict__ work) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    work[i] = (lower ? diag[i] - rp[i] : rp[i + 1] - diag[i] - 1) + 1;
}
__global__ void k_ob_keys(int n, int B, int nl, const int* __restrict__ wcum, const int* __restrict__ depth,
                          int* __restrict__ blk, int* __restrict__ cnt) {
  const long long W = wcum[n];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int b = min(B - 1, (int)((long long)wcum[i] * B / (W > 0 ? W : 1)));
    blk[i] = b;
    atomicAdd(cnt + (int64_t)b * nl + depth[i], 1);
  }
}
__global__ void k_ob_pad(int K, const int* __restrict__ cnt, int* __restrict__ pc, int* __restrict__ fl) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    pc[k] = (cnt[k] + 31) & ~31;
    fl[k] = cnt[k] > 0 ? 1 : 0;
  }
}
// off: K + 1 padded position offsets; gid: K + 1 group numbers (exclusive scans)
__global__ void k_ob_groups(int K, int B, int nl, const int* __restrict__ cnt, const int* __restrict__ off,
                            const int* __restrict__ gid, int* __restrict__ goff, int* __restrict__ bgrp,
                            int* __restrict__ bstart, int* __restrict__ cgend, int* __restrict__ cgstart) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
    if (k == K) {
      goff[gid[K]] = off[K] >> 5;
      bgrp[B] = gid[K];
      bstart[B] = off[K];
      continue;
    }
    if (k % nl == 0) {
      bgrp[k / nl] = gid[k];
      bstart[k / nl] = off[k];
    }
    if (cnt[k] > 0) {
      goff[gid[k]] = off[k] >> 5;
      for (int c = off[k] >> 5; c < (off[k + 1] >> 5); ++c) {
        cgend[c] = off[k + 1];
        cgstart[c] = off[k] >> 5;
      }
    }
  }
}
__global__ void k_ob_scatter(int n, int nl, const int* __restrict__ blk, const int* __restrict__ depth,
                             int* __restrict__ sub, int* __restrict__ perm, int* __restrict__ pos) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int q = atomicAdd(sub + (int64_t)blk[i] * nl + depth[i], 1);
    perm[q] = i;
    pos[i] = q;
  }
}

// Orientation t of the handle: 0, 1 the factor's lower / upper triangle, 2, 3 the conjugate
// transpose's.
struct Orient {
  const int *rp, *ci, *diag;
  const void* fac;
};
static Orient orient(const mpk_ilu* M, int t) {
  if (t < 2) return Orient{M->rp, M->ci, M->diag, M->fac};
  return Orient{M->rpT, M->ciT, M->diagT, M->facT};
}

// Empty kernel whose launch configuration (one CTA per SM through its shared memory, clusters
// of csize) gives the number of clusters that can be co-resident.
__global__ void k_cluster_slot() {}
static int cluster_count(int csize) {
  static std::mutex mu;
  static int known[17] = {0};
  std::lock_guard<std::mutex> lk(mu);
  if (known[csize] != 0) return known[csize];
  int n = -1;
  cudaFuncSetAttribute(k_cluster_slot, cudaFuncAttributeMaxDynamicSharedMemorySize, kClusterSmem);
  if (csize > 8) cudaFuncSetAttribute(k_cluster_slot, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = csize;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(128);
  cfg.dynamicSmemBytes = kClusterSmem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int active = 0;
  if (cudaOccupancyMaxActiveClusters(&active, k_cluster_slot, &cfg) == cudaSuccess && active > 0)
    n = active < sm_count() / csize ? active : sm_count() / csize;
  cudaGetLastError();
  known[csize] = n;
  return n;
}

template <typename T>
static int build_ob_t(mpk_ilu* M, int t, int sched, cudaStream_t s) {
  const Orient o = orient(M, t);
  const bool lower = (t % 2) == 0;
  const int csize = sched_csize(sched);
  const int n = M->n, nl = M->nlevels[t], B = sched == 1 ? sm_count() : cluster_count(csize);
  if (B < 1) return fail(MPK_INVALID_ARG, "no co-resident clusters of this size");
  const int64_t K64 = (int64_t)B * nl;
  if (K64 > (1 << 28)) return fail(MPK_INVALID_ARG, "too many levels for the owner-block layout");
  const int K = (int)K64;
  // temporaries: work/wcum (n + 1), blk (n), cnt, pc, fl (K each), off, gid (K + 1 each)
  int* tmp = nullptr;
  const size_t tmp_ints = 2 * ((size_t)n + 1) + (size_t)n + 3 * (size_t)K + 2 * ((size_t)K + 1);
  MPK_CUDA(cudaMallocAsync((void**)&tmp, sizeof(int) * tmp_ints, s));
  int* work = tmp;
  int* wcum = work + n + 1;
  int* blk = wcum + n + 1;
  int* cnt = blk + n;
  int* pc = cnt + K;
  int* fl = pc + K;
  int* off = fl + K;
  int* gid = off + K + 1;
  MPK_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)K, s));
  count_launch(6);
  k_ob_work<<<grid_for(n), kBlock, 0, s>>>(n, o.rp, o.diag, lower, work);
  k_scan_single<<<1, 1024, 0, s>>>(n, work, wcum);
  k_ob_keys<<<grid_for(n), kBlock, 0, s>>>(n, B, nl, wcum, M->depth[t], blk, cnt);
  k_ob_pad<<<grid_for(K), kBlock, 0, s>>>(K, cnt, pc, fl);
  k_scan_single<<<1, 1024, 0, s>>>(K, pc, off);
  k_scan_single<<<1, 1024, 0, s>>>(K, fl, gid);
  int tot[2] = {0, 0};
  MPK_CUDA(cudaMemcpyAsync(&tot[0], off + K, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaMemcpyAsync(&tot[1], gid + K, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  const int P = tot[0], G = tot[1], nch = P / 32;
  // persistent order buffer: perm (P) | pos (n) | goff (G + 1) | bgrp (B + 1) | bstart (B + 1) |
  // cgend, cgstart (nch each; needed only while repacking)
  int* ob = nullptr;
  const size_t ob_ints = (size_t)P + n + (size_t)G + 1 + 2 * ((size_t)B + 1) + 2 * (size_t)nch;
  MPK_CUDA(cudaMalloc((void**)&ob, sizeof(int) * ob_ints));
  int* perm = ob;
  int* pos = perm + P;
  int* goff = pos + n;
  int* bgrp = goff + G + 1;
  int* bstart = bgrp + B + 1;
  int* cgend = bstart + B + 1;
  int* cgstart = cgend + nch;
  MPK_CUDA(cudaMemsetAsync(perm, 0xff, sizeof(int) * (size_t)P, s));  // padding positions: -1
  count_launch(2);
  k_ob_groups<<<grid_for(K + 1), kBlock, 0, s>>>(K, B, nl, cnt, off, gid, goff, bgrp, bstart, cgend, cgstart);
  k_ob_scatter<<<grid_for(n), kBlock, 0, s>>>(n, nl, blk, M->depth[t], off, perm, pos);  // off becomes ends
  MPK_CUDA(cudaGetLastError());
  ObEnc enc;
  enc.blk = blk;
  enc.bstart = bstart;
  enc.cgend = cgend;
  enc.cgstart = cgstart;
  enc.csize = csize;
  M->ordbuf[sched][t] = ob;
  int st = build_sell<T>(n, M->vals_per_entry(), o.rp, o.ci, o.diag, (const T*)o.fac, perm, pos, nch, lower, enc,
                         &M->laybuf[sched][t], &M->lay[sched][t], s);
  MPK_CUDA(cudaFreeAsync(tmp, s));
  if (st != MPK_OK) return st;
  SellTri& L = M->lay[sched][t];
  L.ob = 1;
  L.goff = goff;
  L.bgrp = bgrp;
  L.bstart = bstart;
  L.nblocks = B;
  L.csize = csize;
  return MPK_OK;
}

// Classic (static chunk schedule) repack of orientation t from its level order.
template <typename T>
static int build_classic_t(mpk_ilu* M, int t, cudaStream_t s) {
  const Orient o = orient(M, t);
  const LevelOrder lo = level_view(M->lvbuf[t], M->n, M->nlevels[t]);
  int nch = 0;
  MPK_CUDA(cudaMemcpyAsync(&nch, lo.nchunks, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  return build_sell<T>(M->n, M->vals_per_entry(), o.rp, o.ci, o.diag, (const T*)o.fac, lo.perm, lo.pos, nch,
                       (t % 2) == 0, ObEnc(), &M->laybuf[0][t], &M->lay[0][t], s);
}

template <typename T>
static int build_layout_t(mpk_ilu* M, int t, int sched, cudaStream_t s) {
  return sched >= 1 ? build_ob_t<T>(M, t, sched, s) : build_classic_t<T>(M, t, s);
}

static void drop_layout(mpk_ilu* M, int t, int sched) {
  if (M->laybuf[sched][t] != nullptr) cudaFree(M->laybuf[sched][t]);
  if (M->ordbuf[sched][t] != nullptr) cudaFree(M->ordbuf[sched][t]);
  M->laybuf[sched][t] = nullptr;
  M->ordbuf[sched][t] = nullptr;
  M->lay[sched][t] = SellTri();
}

int ensure_layout(mpk_ilu* M, int t0, int sched, cudaStream_t s) {
  for (int t = t0; t < t0 + 2; ++t) {
    if (M->laybuf[sched][t] != nullptr) continue;
    if (t >= 2 && M->rpT == nullptr) return fail(MPK_INVALID_ARG, "the conjugate transpose is not built");
    int st;
    if (M->prec == MPK_ILU_FP64 || M->prec == MPK_ILU_MP) st = build_layout_t<double>(M, t, sched, s);
    else if (M->prec == MPK_ILU_FP32) st = build_layout_t<float>(M, t, sched, s);
    else st = build_layout_t<uint16_t>(M, t, sched, s);
    if (st != MPK_OK) return st;
  }
  return MPK_OK;
}

void launch_trsv_prep(const IluHandleView& M, const int* done, cudaStream_t s) {
  count_launch();
  k_trsv_prep<<<1, 1, 0, s>>>(M.ctl, M.absmax, done);
}

static size_t fac_elem_size(int prec) {
  return (prec == MPK_ILU_FP64 || prec == MPK_ILU_MP) ? 8 : (prec == MPK_ILU_FP32 ? 4 : 2);
}

static int build_transpose(mpk_ilu* M, cudaStream_t s) {
  if (M->rpT != nullptr) return MPK_OK;
  const size_t es = fac_elem_size(M->prec);
  MPK_CUDA(cudaMalloc((void**)&M->rpT, sizeof(int) * ((size_t)M->n + 1)));
  MPK_CUDA(cudaMalloc((void**)&M->ciT, sizeof(int) * (size_t)M->nnz));
  MPK_CUDA(cudaMalloc((void**)&M->diagT, sizeof(int) * (size_t)M->n));
  MPK_CUDA(cudaMalloc(&M->facT, es * (size_t)M->nnz * M->vals_per_entry()));
  int st;
#define MPK_TRANSPOSE(T, S, NNEG)                                                                            \
  transpose_t<T, S, NNEG>(M->n, M->nnz, M->rp, M->ci, (const T*)M->fac, M->rpT, M->ciT, (T*)M->facT, M->diagT, s)
  if (M->prec == MPK_ILU_MP) {
    // w-component entries: the w imaginary components change sign
    switch (M->wf * 2 + M->cp - 1) {
      case 2: st = MPK_TRANSPOSE(double, 1, 0); break;
      case 3: st = MPK_TRANSPOSE(double, 2, 1); break;
      case 4: st = MPK_TRANSPOSE(double, 2, 0); break;
      case 5: st = MPK_TRANSPOSE(double, 4, 2); break;
      case 6: st = MPK_TRANSPOSE(double, 3, 0); break;
      case 7: st = MPK_TRANSPOSE(double, 6, 3); break;
      case 8: st = MPK_TRANSPOSE(double, 4, 0); break;
      default: st = MPK_TRANSPOSE(double, 8, 4); break;
    }
  } else if (M->prec == MPK_ILU_FP64) {
    st = M->cp == 2 ? MPK_TRANSPOSE(double, 2, 1) : MPK_TRANSPOSE(double, 1, 0);
  } else if (M->prec == MPK_ILU_FP32) {
    st = M->cp == 2 ? MPK_TRANSPOSE(float, 2, 1) : MPK_TRANSPOSE(float, 1, 0);
  } else {
    st = M->cp == 2 ? MPK_TRANSPOSE(uint16_t, 2, 1) : MPK_TRANSPOSE(uint16_t, 1, 0);
  }
#undef MPK_TRANSPOSE
  if (st != MPK_OK) return st;
  // pk also serves as the binary32 substitutions' result buffer: clear it before the epoch-stamped
  // ordering passes read it
  MPK_CUDA(cudaMemsetAsync(M->pk, 0, sizeof(unsigned long long) * (size_t)M->n * M->cp, s));
  return build_levels(M->n, M->rpT, M->ciT, M->diagT, M->pk, M->ctl, 1, M->lvbuf + 2, M->nlevels + 2, M->depth + 2, s);
}

int prepare_trans(mpk_ilu* M, cudaStream_t s) { return build_transpose(M, s); }

// z = M^-1 r or M^-H r, stream-ordered; `done` may be null.
// bt (nullable): a batch of systems, each with its own binary32 scaling (bt->absmax)
int precond_apply(const mpk_ilu* M, const Ops* o, bool trans, const double* r, double* z, const int* done,
                  const Batch* bt, cudaStream_t s) {
  if (trans && M->rpT == nullptr) return fail(MPK_INVALID_ARG, "M^H solve needs the transposed factor");
  IluHandleView v = M->view(trans);
  if (v.sl_lo.coff == nullptr || v.sl_up.coff == nullptr)
    return fail(MPK_INVALID_ARG, "the substitution layout of this schedule is not built");
  launch_trsv_prep(v, done, s);
  int st;
  // M: unit lower L~ then upper U~ with division; M^H: lower U~^H with division then unit upper L~^H
  if (M->prec == MPK_ILU_MP && M->wf != o->w) return fail(MPK_INVALID_ARG, "a w-component factor needs the same w");
  if (M->prec == MPK_ILU_FP64 || M->prec == MPK_ILU_MP) {
    st = o->trsv_mp(v, true, !trans, r, M->vmp, done, s);
    if (st == MPK_OK) st = o->trsv_mp(v, false, trans, M->vmp, z, done, s);
  } else {
    if (bt != nullptr && bt->sysid != nullptr) {
      v.sysid = bt->sysid;
      v.absmax = bt->absmax;
      MPK_CUDA(cudaMemsetAsync(bt->absmax, 0, sizeof(unsigned long long) * (size_t)bt->nsys, s));
    }
    o->absmax(M->n, r, v.absmax, done, bt, s);
    st = o->trsv32(v, true, !trans, r, nullptr, done, s);
    if (st == MPK_OK) st = o->trsv32(v, false, trans, nullptr, z, done, s);
  }
  if (st != MPK_OK) return fail(st, "substitution launch failed");
  return MPK_OK;
}

// New factor values on the same pattern (after a learned correction): drop every repacked
// triangle and the conjugate transpose (all rebuilt on their next use).
int refresh_factor(mpk_ilu* M, cudaStream_t s) {
  MPK_CUDA(cudaStreamSynchronize(s));
  for (int t = 0; t < 4; ++t)
    for (int sc = 0; sc < kScheds; ++sc) drop_layout(M, t, sc);
  void* tp[] = {M->rpT, M->ciT, M->diagT, M->facT, M->lvbuf[2], M->lvbuf[3], M->depth[2], M->depth[3]};
  for (void* p : tp)
    if (p != nullptr) cudaFree(p);
  M->rpT = M->ciT = M->diagT = nullptr;
  M->facT = nullptr;
  M->lvbuf[2] = M->lvbuf[3] = nullptr;
  M->depth[2] = M->depth[3] = nullptr;
  M->nlevels[2] = M->nlevels[3] = 0;
  return MPK_OK;
}

// ---- substitution autotuner ---------------------------------------------------------------------
// Candidates: the static chunk schedule and the owner-block schedule per SM with 4, 8, 16 or 32
// warps per SM, each timed on two applications of M^-1; the choice is cached per (matrix
// pattern, factor precision, w, c).  MPK_SUBST_SCHEDULE=static|owner|cluster8|cluster16 selects
// one schedule instead (the owner-block schedule per cluster of 8 or 16 SMs, with 4 or 8 warps
// per SM, runs only when selected so; tests use it to cover each).
int read_ctl_err(const mpk_ilu* M, cudaStream_t s);
struct TrsvTune {
  uint64_t fp;  // pattern fingerprint of the factored matrix
  int n, nnz, prec, w, cp, forced, wpb, sched, poll;
};
static std::mutex g_trsv_mu;
static std::vector<TrsvTune> g_trsv;
// MPK_SUBST_POLL=lane0|all|allsleep forces the dependency polling of the substitutions (-1: tuned).
static int forced_poll() {
  const char* e = std::getenv("MPK_SUBST_POLL");
  if (e == nullptr) return -1;
  if (std::strcmp(e, "lane0") == 0) return 0;
  if (std::strcmp(e, "all") == 0) return 1;
  if (std::strcmp(e, "allsleep") == 0) return 2;
  return -1;
}
// MPK_SUBST_POLL_SLEEP_NS=16..4096: the sleep between polling rounds of polling mode 2 (256 ns).
static int poll_sleep_ns() {
  const char* e = std::getenv("MPK_SUBST_POLL_SLEEP_NS");
  if (e == nullptr) return 256;
  const int v = std::atoi(e);
  return v < 16 ? 16 : (v > 4096 ? 4096 : v);
}
static int forced_schedule() {
  const char* e = std::getenv("MPK_SUBST_SCHEDULE");
  if (e == nullptr) return -1;
  if (std::strcmp(e, "static") == 0) return 0;
  if (std::strcmp(e, "owner") == 0) return 1;
  if (std::strcmp(e, "cluster8") == 0) return 2;
  if (std::strcmp(e, "cluster16") == 0) return 3;
  return -1;
}
// applications of M^-1 timed per candidate (after one untimed): candidates within a few percent
// of each other need more than two to be told apart
constexpr int kTuneReps = 4;
static bool cached_choice(const mpk_ilu* M, int w, int forced, int fpoll, int* wpb, int* sched, int* poll) {
  std::lock_guard<std::mutex> lk(g_trsv_mu);
  for (const TrsvTune& t : g_trsv)
    if (t.fp == M->pattern_fp && t.n == M->n && t.nnz == M->nnz && t.prec == M->prec && t.w == w && t.cp == M->cp &&
        t.forced == forced && (fpoll < 0 || t.poll == fpoll)) {
      *wpb = t.wpb;
      *sched = t.sched;
      *poll = t.poll;
      return true;
    }
  return false;
}
// the handle's layouts for its current schedule (factor, and the conjugate transpose if built)
static int ensure_current(mpk_ilu* M, cudaStream_t s) {
  int st = ensure_layout(M, 0, M->sched, s);
  if (st == MPK_OK && M->rpT != nullptr) st = ensure_layout(M, 2, M->sched, s);
  return st;
}
int tune_substitution(mpk_ilu* M, const Ops* o, int w, double* r, double* z, cudaStream_t s) {
  const int forced = forced_schedule(), fpoll = forced_poll();
  int wpb = 0, sched = 0, poll = 0;
  if (cached_choice(M, w, forced, fpoll, &wpb, &sched, &poll)) {
    M->wpb = wpb;
    M->sched = sched;
    M->poll = poll;
    return ensure_current(M, s);
  }
  static const int cands[4] = {4, 8, 16, 32};
  cudaEvent_t e0, e1;
  MPK_CUDA(cudaEventCreate(&e0));
  MPK_CUDA(cudaEventCreate(&e1));
  float best = 0.f;
  int best_wpb = 4, best_sched = forced >= 0 ? forced : 0, best_poll = fpoll >= 0 ? fpoll : 0;
  for (int sc = 0; sc < kScheds; ++sc) {
    // the cluster schedules (2, 3) are candidates only when asked for: they lost on every
    // workload measured, and their cooperative cluster launches cannot run under ncu
    if (forced >= 0 ? sc != forced : sc >= 2) continue;
    if (ensure_layout(M, 0, sc, s) != MPK_OK) {
      cudaGetLastError();
      drop_layout(M, 0, sc);
      drop_layout(M, 1, sc);
      continue;
    }
    M->sched = sc;
    for (int wp : cands) {
      if (sc >= 2 && wp > 8) continue;  // cluster CTAs: one per SM, 4 or 8 warps
      if (!o->trsv_fits(M->prec, wp, sc, M->lay[sc][0].nblocks)) continue;
      M->wpb = wp;
      for (int pm = 0; pm < 3; ++pm) {
        // polling: lane 0 on the latest dependency first, or every lane on its own, spinning or
        // sleeping between rounds (the static schedule only for 1 and 2; measured: each wins on
        // some workloads)
        if ((fpoll >= 0 && pm != fpoll) || (fpoll < 0 && pm >= 1 && sc != 0)) continue;
        M->poll = pm;
        int st = precond_apply(M, o, false, r, z, nullptr, nullptr, s);  // warm
        if (st != MPK_OK) continue;
        cudaEventRecord(e0, s);
        for (int k = 0; k < kTuneReps; ++k) precond_apply(M, o, false, r, z, nullptr, nullptr, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0.f || ms < best) {
          best = ms;
          best_wpb = wp;
          best_sched = sc;
          best_poll = pm;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  M->wpb = best_wpb;
  M->sched = best_sched;
  M->poll = best_poll;
  const int err = read_ctl_err(M, s);
  if (err != MPK_OK) return err;
  for (int sc = 0; sc < kScheds; ++sc)  // keep the chosen repack only
    if (sc != best_sched)
      for (int t = 0; t < 4; ++t) drop_layout(M, t, sc);
  {
    std::lock_guard<std::mutex> lk(g_trsv_mu);
    if (g_trsv.size() < 256)
      g_trsv.push_back(TrsvTune{M->pattern_fp, M->n, M->nnz, M->prec, w, M->cp, forced, best_wpb, best_sched,
                                best_poll});
  }
  return ensure_current(M, s);
}

// Device error of the handle's last kernels; reported once (cleared after reading, so the handle
// serves the next call).
int read_ctl_err(const mpk_ilu* M, cudaStream_t s) {
  int err = 0;
  MPK_CUDA(cudaMemcpyAsync(&err, M->ctl + CTL_ERR, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  if (err != 0) {
    MPK_CUDA(cudaMemsetAsync(M->ctl + CTL_ERR, 0, sizeof(int), s));
    MPK_CUDA(cudaStreamSynchronize(s));
    return fail(err, "a bounded device wait ran out in a substitution kernel");
  }
  return MPK_OK;
}

static void free_handle(mpk_ilu* M) {
  if (M == nullptr) return;
  void* ptrs[] = {M->rp, M->ci, M->diag, M->fac, M->rpT, M->ciT, M->diagT, M->facT, M->flags, M->ctl, M->v32, M->vmp,
                  M->absmax, M->pk, M->lvbuf[0], M->lvbuf[1], M->lvbuf[2], M->lvbuf[3],
                  M->depth[0], M->depth[1], M->depth[2], M->depth[3]};
  for (void* p : ptrs)
    if (p != nullptr) cudaFree(p);
  for (int sc = 0; sc < kScheds; ++sc)
    for (int t = 0; t < 4; ++t) drop_layout(M, t, sc);
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
  v.pk = pk;
  const int t = trans ? 2 : 0;
  v.lv_lo = level_view(lvbuf[t], n, nlevels[t]);
  v.lv_up = level_view(lvbuf[t + 1], n, nlevels[t + 1]);
  v.sl_lo = lay[sched][t];
  v.sl_up = lay[sched][t + 1];
  v.wpb = wpb;
  v.sched = sched;
  v.withhold = withhold;
  v.poll = poll;
  v.poll_ns = poll_sleep_ns();
  return v;
}

static int factor_impl(const mpk_csr* A, int prec, int w, mpk_ilu** out, int* fail_row, cudaStream_t s) {
  const int n = A->n, nnz = A->nnz, cp = A->is_complex ? 2 : 1;
  int head[2] = {-1, -1};
  MPK_CUDA(cudaMemcpyAsync(&head[0], A->row_ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaMemcpyAsync(&head[1], A->row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  if (head[0] != 0 || head[1] != nnz) return fail(MPK_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] == nnz");

  uint64_t pfp = 0;
  {
    const int st_fp = pattern_fingerprint(n, nnz, A->row_ptr, A->col_idx, &pfp, s);
    if (st_fp != MPK_OK) return st_fp;
  }
  mpk_ilu* M = new mpk_ilu();
  M->pattern_fp = pfp;
  M->n = n;
  M->nnz = nnz;
  M->cp = cp;
  M->prec = prec;
  M->wf = prec == MPK_ILU_MP ? w : 1;
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
  count_launch();
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
  {
    const int nch = (n + 31) >> 5;
    MPK_TRY(cudaMalloc((void**)&M->pk, sizeof(unsigned long long) * (size_t)n * cp));
    MPK_TRY(cudaMemsetAsync(M->pk, 0, sizeof(unsigned long long) * (size_t)n * cp, s));
    (void)nch;
    int st = build_levels(n, M->rp, M->ci, M->diag, M->pk, M->ctl, 0, M->lvbuf, M->nlevels, M->depth, s);
    if (st != MPK_OK) return bail(st);
  }

  const int64_t m = (int64_t)nnz * cp;
  void* work = nullptr;  // factor in its computation type
  if (prec == MPK_ILU_MP) {
    const int64_t mw = m * w;
    MPK_TRY(cudaMalloc(&work, sizeof(double) * (size_t)(mw > 0 ? mw : 1)));
    count_launch();
    k_to_mp<<<grid_for((int)((mw + 3) / 4)), kBlock, 0, s>>>(nnz, cp, w, A->val, (double*)work);
  } else if (prec == MPK_ILU_FP64) {
    MPK_TRY(cudaMalloc(&work, sizeof(double) * (size_t)(m > 0 ? m : 1)));
    MPK_TRY(cudaMemcpyAsync(work, A->val, sizeof(double) * (size_t)m, cudaMemcpyDeviceToDevice, s));
  } else {
    MPK_TRY(cudaMalloc(&work, sizeof(float) * (size_t)(m > 0 ? m : 1)));
    count_launch();
    k_narrow<float><<<grid_for((int)((m + 3) / 4)), kBlock, 0, s>>>(m, A->val, (float*)work);
  }
  M->fac = work;
  const LevelOrder lv_lo = M->view(false).lv_lo;
  int lst = MPK_OK;
  if (prec == MPK_ILU_MP) {
    lst = launch_ilu_mp(w, cp, n, M->rp, M->ci, M->diag, lv_lo, (double*)work, M->ctl, s);
  } else if (prec == MPK_ILU_FP64) {
    if (cp == 1) lst = launch_ilu<double, 1>(n, M->nnz, M->rp, M->ci, M->diag, lv_lo, (double*)work, M->ctl, s);
    else lst = launch_ilu<double, 2>(n, M->nnz, M->rp, M->ci, M->diag, lv_lo, (double*)work, M->ctl, s);
  } else {
    if (cp == 1) lst = launch_ilu<float, 1>(n, M->nnz, M->rp, M->ci, M->diag, lv_lo, (float*)work, M->ctl, s);
    else lst = launch_ilu<float, 2>(n, M->nnz, M->rp, M->ci, M->diag, lv_lo, (float*)work, M->ctl, s);
  }
  if (lst != MPK_OK) return bail(lst);
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
    count_launch();
    k_to_bf16<<<grid_for((int)((m + 3) / 4)), kBlock, 0, s>>>(m, (const float*)work, h);
    MPK_TRY(cudaGetLastError());
    MPK_TRY(cudaStreamSynchronize(s));
    cudaFree(work);
    M->fac = h;
  }
  if (prec == MPK_ILU_FP64 || prec == MPK_ILU_MP) {
    MPK_TRY(cudaMalloc((void**)&M->vmp, sizeof(double) * (size_t)n * cp * 4));
  } else {
    MPK_TRY(cudaMalloc((void**)&M->v32, sizeof(float) * (size_t)n * cp));
  }
  // the repacked triangles are built on first use, for the schedule the tuner picks
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
  if (A->is_complex && misaligned(A->val)) return fail(MPK_INVALID_ARG, "complex values must be 16-byte aligned");
  if (prec != MPK_ILU_FP64 && prec != MPK_ILU_FP32 && prec != MPK_ILU_BF16)
    return fail(MPK_INVALID_ARG, "prec must be MPK_ILU_FP64, MPK_ILU_FP32 or MPK_ILU_BF16");
  return factor_impl(A, prec, 1, out, fail_row, (cudaStream_t)stream);
}

extern "C" int mpk_ilu0_factor_mp(const mpk_csr* A, int w, mpk_ilu** out, int* fail_row, void* stream) {
  if (fail_row) *fail_row = -1;
  if (out) *out = nullptr;
  if (A == nullptr || out == nullptr) return fail(MPK_INVALID_ARG, "null argument");
  if (A->n < 1 || A->nnz < 0 || A->row_ptr == nullptr || (A->nnz > 0 && (A->col_idx == nullptr || A->val == nullptr)))
    return fail(MPK_INVALID_ARG, "invalid CSR descriptor");
  if (A->is_complex != 0 && A->is_complex != 1) return fail(MPK_INVALID_ARG, "is_complex must be 0 or 1");
  if (A->is_complex && misaligned(A->val)) return fail(MPK_INVALID_ARG, "complex values must be 16-byte aligned");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  return factor_impl(A, MPK_ILU_MP, w, out, fail_row, (cudaStream_t)stream);
}

extern "C" int mpk_ilu0_values(const mpk_ilu* M, double* out_dev, void* stream) {
  if (M == nullptr || out_dev == nullptr) return fail(MPK_INVALID_ARG, "null argument");
  if (misaligned(out_dev)) return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t m = (int64_t)M->nnz * M->cp;
  if (m == 0) return MPK_OK;
  if (M->prec == MPK_ILU_MP) {
    MPK_CUDA(cudaMemcpyAsync(out_dev, M->fac, sizeof(double) * (size_t)m * M->wf, cudaMemcpyDeviceToDevice, s));
    return MPK_OK;
  }
  const int g = grid_for((int)((m + 3) / 4));
  count_launch();
  if (M->prec == MPK_ILU_FP64) k_widen<double><<<g, kBlock, 0, s>>>(m, (const double*)M->fac, out_dev);
  else if (M->prec == MPK_ILU_FP32) k_widen<float><<<g, kBlock, 0, s>>>(m, (const float*)M->fac, out_dev);
  else k_widen<uint16_t><<<g, kBlock, 0, s>>>(m, (const uint16_t*)M->fac, out_dev);
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}

extern "C" int mpk_ilu0_prec(const mpk_ilu* M) { return M == nullptr ? -2 : M->prec; }

extern "C" int mpk_ilu0_width(const mpk_ilu* M) { return M == nullptr ? -2 : M->wf; }

extern "C" int mpk_ilu0_levels(const mpk_ilu* M, int tri, int* nlevels_out, int* depth_dev, void* stream) {
  if (M == nullptr || tri < 0 || tri > 1) return fail(MPK_INVALID_ARG, "bad handle or triangle");
  if (nlevels_out != nullptr) *nlevels_out = M->nlevels[tri];
  if (depth_dev != nullptr && M->n > 0) {
    if (M->depth[tri] == nullptr) return fail(MPK_INVALID_ARG, "the handle holds no level record");
    MPK_CUDA(cudaMemcpyAsync(depth_dev, M->depth[tri], sizeof(int) * (size_t)M->n, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
  }
  return MPK_OK;
}

extern "C" int mpk_ilu0_test_withhold(mpk_ilu* M, int row) {
  if (M == nullptr || row < -1 || row >= M->n) return fail(MPK_INVALID_ARG, "bad handle or row");
  M->withhold = row;
  return MPK_OK;
}

extern "C" int mpk_ilu0_schedule(const mpk_ilu* M, int* wpb_out) {
  if (M == nullptr) return -2;
  if (wpb_out != nullptr) *wpb_out = M->wpb;
  return M->sched;
}

extern "C" int mpk_ilu0_polling(const mpk_ilu* M) { return M == nullptr ? -2 : M->poll; }

extern "C" void mpk_ilu0_destroy(mpk_ilu* M) { free_handle(M); }

extern "C" int mpk_precond_apply(const mpk_ilu* M, int w, int trans, const double* r_dev, double* z_dev,
                                 void* stream) {
  if (M == nullptr || r_dev == nullptr || z_dev == nullptr || r_dev == z_dev)
    return fail(MPK_INVALID_ARG, "null or aliased argument");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  if (misaligned(r_dev) || misaligned(z_dev)) return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  if (trans) {
    int st = build_transpose(const_cast<mpk_ilu*>(M), s);
    if (st != MPK_OK) return st;
  }
  const Ops* o = get_ops(w, M->cp);
  mpk_ilu* Mm = const_cast<mpk_ilu*>(M);
  {
    const int forced = forced_schedule(), fpoll = forced_poll();
    int wpb = 0, sched = 0, poll = 0;
    if (cached_choice(M, w, forced, fpoll, &wpb, &sched, &poll)) {
      Mm->wpb = wpb;
      Mm->sched = sched;
      Mm->poll = poll;
    } else {
      if (forced >= 0) Mm->sched = forced;
      if (fpoll >= 0) Mm->poll = fpoll;
    }
    int st = ensure_layout(Mm, trans ? 2 : 0, M->sched, s);
    if (st != MPK_OK) return st;
  }
  int st = precond_apply(M, o, trans != 0, r_dev, z_dev, nullptr, nullptr, s);
  if (st != MPK_OK) return st;
  MPK_CUDA(cudaGetLastError());
  return read_ctl_err(M, s);
}
