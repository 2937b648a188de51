// kernels.cuh -- templated CUDA kernels of the Krylov iteration (instantiated per w in
// inst_w*.cu).  Every kernel takes the solve's `done` flag (nullable) and returns at once when
// it is set, so the host can queue several iterations ahead of its convergence check.
#pragma once
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "mp.cuh"

namespace mpk {

constexpr int kBlock = 256;
constexpr long long kWaitCycles = 1ll << 31;  // ~1 s at 2 GHz: bound of every device wait

__device__ __forceinline__ bool is_done(const int* done) { return done != nullptr && *done != 0; }

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

template <int W, int CP>
__device__ __forceinline__ N<W, CP> shfl_down_n(const N<W, CP>& a, int off) {
  N<W, CP> z;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    z.re.c[k] = __shfl_down_sync(0xffffffffu, a.re.c[k], off);
    z.im.c[k] = CP == 2 ? __shfl_down_sync(0xffffffffu, a.im.c[k], off) : 0.0;
  }
  return z;
}
template <int W, int CP>
__device__ __forceinline__ N<W, CP> warp_sum(N<W, CP> a) {  // fixed tree order
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) a = n_add<W, CP>(a, shfl_down_n<W, CP>(a, off));
  return a;
}

// ---------------------------------------------------------------------------------------------
// y = A x  (b != nullptr: y = b - A x), one thread per row, CSR order from 0.  A real D row
// accumulates each entry with one fused multiply-add (one binary64 instruction per nonzero).
// ---------------------------------------------------------------------------------------------
// A batch (sysid != nullptr) skips the rows of systems whose state sst has ST_DONE set, or, with
// gate >= 0, a nonzero sst[gate].
// MM: the matrix entry is promoted to a W-component number (a, 0, ..., 0), same value, and the
// product is the format's full multiplication with the matrix entry first (the paper's rows
// without "_d", whose matrices are held in the vectors' type).
template <int W, int CP, bool MM>
__global__ void __launch_bounds__(kBlock) k_spmv(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                                 const double* __restrict__ val, const double* __restrict__ x,
                                                 double* __restrict__ y, const double* __restrict__ b,
                                                 const int* __restrict__ done, const int* __restrict__ sysid,
                                                 const int* __restrict__ sst, const int* __restrict__ order,
                                                 int gate) {
  if (is_done(done)) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  // order (nullable): rows grouped by length so that the lanes of a warp do equal work (every
  // binary64 warp instruction costs its full pipe time however many lanes are active)
  const int i = order != nullptr ? order[t] : t;
  if (sysid != nullptr && sst != nullptr) {
    const int* q = sst + sysid[i] * ST_COUNT;
    if (q[ST_DONE] != 0 || (gate >= 0 && q[gate] != 0)) return;
  }
  N<W, CP> acc = n_zero<W, CP>();
  const int p1 = rp[i + 1];
  int p = rp[i];
  if constexpr (W == 2 && CP == 1 && !MM) {
    // Real DD: the row's first product is its sum so far.  Adding a normalised double-word p to
    // (+0, +0) returns p with any -0 word as +0 -- bit for bit (checked on 5e7 products of
    // normalised double-words, zeros and subnormals included), so the first entry's DW+DW
    // addition (14 binary64 instructions) is skipped.  Inputs follow the library's convention
    // (normalised components); the zero test is an integer one.
    if (p < p1) {
      const N<W, CP> q = n_mul_fp<W, CP>(n_load<W, CP>(x, ci[p]), val[p], 0.0);
#pragma unroll
      for (int k = 0; k < W; ++k)
        acc.re.c[k] = (__double_as_longlong(q.re.c[k]) << 1) == 0 ? 0.0 : q.re.c[k];
      ++p;
    }
  }
  for (; p < p1; ++p) {
    const int j = ci[p];
    double ar, ai = 0.0;
    if constexpr (CP == 1) {
      ar = val[p];
    } else {
      double2 v = reinterpret_cast<const double2*>(val)[p];
      ar = v.x;
      ai = v.y;
    }
    if constexpr (W == 1 && CP == 1) {
      acc.re.c[0] = fma(ar, x[j], acc.re.c[0]);  // D, real: one fused multiply-add per entry
    } else if constexpr (MM) {
      N<W, CP> a = n_zero<W, CP>();
      a.re.c[0] = ar;
      a.im.c[0] = ai;
      acc = n_add<W, CP>(acc, n_mul<W, CP>(a, n_load<W, CP>(x, j)));
    } else {
      acc = n_add<W, CP>(acc, n_mul_fp<W, CP>(n_load<W, CP>(x, j), ar, ai));
    }
  }
  if (b != nullptr) acc = n_add<W, CP>(n_load<W, CP>(b, i), n_mul<W, CP>(n_real<W, CP>(-1.0), acc));
  n_store<W, CP>(y, i, acc);
}

// ---------------------------------------------------------------------------------------------
// K inner products <a_k, b_k> = sum_i conj(a_k,i) b_k,i in the library's fixed summation order:
// leaves of kDotLeaf consecutive products summed left to right (from the first product), leaf
// sums combined by a stride-doubling pairwise tree (level d adds s_{j+d} into s_j for j a
// multiple of 2d, j + d < m).  Thread t owns leaf t; levels d < 32 run across the lanes of a
// warp, d = 32..128 across the warps of a block, d >= 256 across blocks (the last block to
// finish walks the per-block partials).  The result depends on n only, not on the hardware.
// ---------------------------------------------------------------------------------------------
constexpr int kLeavesPerBlock = kBlock;  // one leaf per thread
static_assert(kLeavesPerBlock == kDotBlockLeaves, "inner-product block layout");

template <int K>
struct DotArgs {
  const double* a[K];
  const double* b[K];
  double* out[K];
};

// One block of the fixed-order reduction of K inner products of length n: block lb of G
// (a, b already offset to the first entry), partials[0 .. G*K) and counter private to these n
// entries.  The last block to finish reduces the partials and writes out[k].
template <int W, int CP, int K>
__device__ __forceinline__ void dots_block(int n, int lb, int G, const double* const* a, const double* const* b,
                                           double* const* out, double* __restrict__ partial,
                                           unsigned* __restrict__ counter) {
  __shared__ __align__(16) double sh[(kBlock / 32) * K * CP * W];
  __shared__ bool last;
  const int m = (n + kDotLeaf - 1) / kDotLeaf;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int block_leaf0 = lb * kLeavesPerBlock;
  const int leaf = block_leaf0 + threadIdx.x;
  N<W, CP> acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = n_zero<W, CP>();
  if (leaf < m) {
    const int i0 = leaf * kDotLeaf, i1 = min(n, i0 + kDotLeaf);
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = n_mul_conj<W, CP>(n_load<W, CP>(a[k], i0), n_load<W, CP>(b[k], i0));
    for (int i = i0 + 1; i < i1; ++i) {
#pragma unroll
      for (int k = 0; k < K; ++k)
        acc[k] = n_add<W, CP>(acc[k], n_mul_conj<W, CP>(n_load<W, CP>(a[k], i), n_load<W, CP>(b[k], i)));
    }
  }
  // levels d = 1..16 across lanes
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      N<W, CP> o = shfl_down_n<W, CP>(acc[k], d);
      if ((lane & (2 * d - 1)) == 0 && leaf + d < m) acc[k] = n_add<W, CP>(acc[k], o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) n_store<W, CP>(sh, (int64_t)wid * K + k, acc[k]);
  }
  __syncthreads();
  // levels d = 32, 64, 128 across the warps of the block
  if (wid == 0) {
    constexpr int NW = kBlock / 32;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = lane < NW ? n_load<W, CP>(sh, (int64_t)lane * K + k) : n_zero<W, CP>();
#pragma unroll
    for (int d = 1; d < NW; d <<= 1) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        N<W, CP> o = shfl_down_n<W, CP>(acc[k], d);
        if (lane < NW && (lane & (2 * d - 1)) == 0 && block_leaf0 + 32 * (lane + d) < m)
          acc[k] = n_add<W, CP>(acc[k], o);
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < K; ++k) n_store<W, CP>(partial, (int64_t)lb * K + k, acc[k]);
      __threadfence();
      const unsigned t = atomicAdd(counter, 1u);
      last = (t == (unsigned)G - 1);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // levels d >= 256 across blocks, on the partials
  for (int e = 1; e < G; e <<= 1) {
    for (int bb = threadIdx.x * 2 * e; bb + e < G; bb += blockDim.x * 2 * e) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        N<W, CP> x = n_load<W, CP>(partial, (int64_t)bb * K + k);
        N<W, CP> y = n_load<W, CP>(partial, (int64_t)(bb + e) * K + k);
        n_store<W, CP>(partial, (int64_t)bb * K + k, n_add<W, CP>(x, y));
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) n_store<W, CP>(out[k], 0, n_load<W, CP>(partial, k));
    *counter = 0u;
  }
}

template <int W, int CP, int K>
__global__ void __launch_bounds__(kBlock) k_dots(int n, DotArgs<K> args, double* __restrict__ partial,
                                                 unsigned* __restrict__ counter, const int* __restrict__ done) {
  if (is_done(done)) return;
  dots_block<W, CP, K>(n, blockIdx.x, gridDim.x, args.a, args.b, args.out, partial, counter);
}

// Segmented: block b belongs to system bsys[b] (blocks boff[s] .. boff[s+1]-1); every system is
// reduced exactly as k_dots would reduce it alone.  Systems whose state has ST_DONE set are skipped
// by all their blocks (the state does not change during the launch).
template <int W, int CP, int K>
__global__ void __launch_bounds__(kBlock) k_dots_seg(Batch bt, DotArgs<K> args, double* __restrict__ S, int slot0,
                                                     double* __restrict__ partial, unsigned* __restrict__ counters,
                                                     const int* __restrict__ done) {
  if (is_done(done)) return;
  const int sy = bt.bsys[blockIdx.x];
  if (bt.st != nullptr &&
      (bt.st[sy * ST_COUNT + ST_DONE] != 0 || (bt.gate >= 0 && bt.st[sy * ST_COUNT + bt.gate] != 0)))
    return;
  const int r0 = bt.roff[sy], n = bt.roff[sy + 1] - r0;
  const int b0 = bt.boff[sy], G = bt.boff[sy + 1] - b0;
  const double* a[K];
  const double* b[K];
  double* out[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    a[k] = args.a[k] + (int64_t)r0 * CP * W;
    b[k] = args.b[k] + (int64_t)r0 * CP * W;
    out[k] = S + (int64_t)sy * kSysDoubles + (slot0 + k) * kSlotDoubles;
  }
  dots_block<W, CP, K>(n, blockIdx.x - b0, G, a, b, out, partial + (int64_t)b0 * K * CP * W, counters + sy);
}

// ---------------------------------------------------------------------------------------------
// Vector updates
// ---------------------------------------------------------------------------------------------
struct LinArgs {
  double* y;
  const double* v[3];
  const double* s[3];  // nullptr: the vector itself (no multiplication)
  int nt;
  const int* copy_at_first;  // non-null: at iteration 1 (st[ST_IT] == 1) y = v[0] instead
};
// Batch (sysid != nullptr): coefficients of system s at a.s[k] + s * kSysDoubles, its iteration
// counter in sst, and the rows of finished systems (or, gate >= 0, of systems whose sst[gate] is
// nonzero) left untouched.
template <int W, int CP>
__global__ void __launch_bounds__(kBlock) k_lincomb(int n, LinArgs a, const int* __restrict__ done,
                                                    const int* __restrict__ sysid, const int* __restrict__ sst,
                                                    int gate) {
  if (is_done(done)) return;
  if (sysid != nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const int sy = sysid[i];
      const int* st = sst + sy * ST_COUNT;
      if (st[ST_DONE] != 0 || (gate >= 0 && st[gate] != 0)) continue;
      if (a.copy_at_first != nullptr && st[ST_IT] == 1) {
        n_store<W, CP>(a.y, i, n_load<W, CP>(a.v[0], i));
        continue;
      }
      const int64_t so = (int64_t)sy * kSysDoubles;
      N<W, CP> acc = n_load<W, CP>(a.v[0], i);
      if (a.s[0] != nullptr) acc = n_mul<W, CP>(n_load<W, CP>(a.s[0] + so, 0), acc);
#pragma unroll
      for (int k = 1; k < 3; ++k) {
        if (k < a.nt) {
          N<W, CP> t = n_load<W, CP>(a.v[k], i);
          if (a.s[k] != nullptr) t = n_mul<W, CP>(n_load<W, CP>(a.s[k] + so, 0), t);
          acc = n_add<W, CP>(acc, t);
        }
      }
      n_store<W, CP>(a.y, i, acc);
    }
    return;
  }
  if (a.copy_at_first != nullptr && a.copy_at_first[ST_IT] == 1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      n_store<W, CP>(a.y, i, n_load<W, CP>(a.v[0], i));
    return;
  }
  N<W, CP> s[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    if (k < a.nt && a.s[k] != nullptr) s[k] = n_load<W, CP>(a.s[k], 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    N<W, CP> acc = n_load<W, CP>(a.v[0], i);
    if (a.s[0] != nullptr) acc = n_mul<W, CP>(s[0], acc);
#pragma unroll
    for (int k = 1; k < 3; ++k) {
      if (k < a.nt) {
        N<W, CP> t = n_load<W, CP>(a.v[k], i);
        if (a.s[k] != nullptr) t = n_mul<W, CP>(s[k], t);
        acc = n_add<W, CP>(acc, t);
      }
    }
    n_store<W, CP>(a.y, i, acc);
  }
}
template <int W, int CP>
__global__ void __launch_bounds__(kBlock) k_nested(int n, double* y, const double* v0, const double* v1,
                                                   const double* v2, const double* s1p, const double* s2p,
                                                   const int* copy_at_first, const int* __restrict__ done,
                                                   const int* __restrict__ sysid, const int* __restrict__ sst) {
  if (is_done(done)) return;
  if (sysid != nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const int sy = sysid[i];
      const int* st = sst + sy * ST_COUNT;
      if (st[ST_DONE] != 0) continue;
      if (copy_at_first != nullptr && st[ST_IT] == 1) {
        n_store<W, CP>(y, i, n_load<W, CP>(v0, i));
        continue;
      }
      const int64_t so = (int64_t)sy * kSysDoubles;
      const N<W, CP> s1 = n_load<W, CP>(s1p + so, 0), s2 = n_load<W, CP>(s2p + so, 0);
      N<W, CP> inner = n_add<W, CP>(n_load<W, CP>(v1, i), n_mul<W, CP>(s1, n_load<W, CP>(v2, i)));
      n_store<W, CP>(y, i, n_add<W, CP>(n_load<W, CP>(v0, i), n_mul<W, CP>(s2, inner)));
    }
    return;
  }
  if (copy_at_first != nullptr && copy_at_first[ST_IT] == 1) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      n_store<W, CP>(y, i, n_load<W, CP>(v0, i));
    return;
  }
  const N<W, CP> s1 = n_load<W, CP>(s1p, 0), s2 = n_load<W, CP>(s2p, 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    N<W, CP> inner = n_add<W, CP>(n_load<W, CP>(v1, i), n_mul<W, CP>(s1, n_load<W, CP>(v2, i)));
    n_store<W, CP>(y, i, n_add<W, CP>(n_load<W, CP>(v0, i), n_mul<W, CP>(s2, inner)));
  }
}
template <int W, int CP>
__global__ void __launch_bounds__(kBlock) k_copy(int n, double* __restrict__ y, const double* __restrict__ x,
                                                 const int* __restrict__ done) {
  if (is_done(done)) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    n_store<W, CP>(y, i, n_load<W, CP>(x, i));
}

// Largest |leading component| (real and imaginary parts) as the bit pattern of a nonnegative
// double, combined with atomicMax (bit order equals numeric order for nonnegative doubles).
// Batch (sysid != nullptr): one accumulator per system, out[sysid[i]].
template <int W, int CP>
__global__ void __launch_bounds__(kBlock) k_absmax(int n, const double* __restrict__ v,
                                                   unsigned long long* __restrict__ out,
                                                   const int* __restrict__ done, const int* __restrict__ sysid) {
  if (is_done(done)) return;
  if (sysid != nullptr) {  // warp-uniform loop: a warp whose rows share one system reduces first
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += gridDim.x * blockDim.x) {
      const int i = base + lane;
      unsigned long long a = 0ull;
      int sy = -1;
      if (i < n) {
        const double* p = v + (int64_t)i * CP * W;
        a = (unsigned long long)__double_as_longlong(fabs(p[0]));
        if constexpr (CP == 2) {
          unsigned long long b = (unsigned long long)__double_as_longlong(fabs(p[W]));
          a = b > a ? b : a;
        }
        sy = sysid[i];
      }
      const int sy0 = __shfl_sync(FULL, sy, 0);
      if (__all_sync(FULL, sy < 0 || sy == sy0)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          const unsigned long long o = __shfl_down_sync(FULL, a, off);
          a = o > a ? o : a;
        }
        if (lane == 0 && a != 0ull) atomicMax(out + sy0, a);
      } else if (sy >= 0 && a != 0ull) {
        atomicMax(out + sy, a);
      }
    }
    return;
  }
  unsigned long long m = 0ull;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double* p = v + (int64_t)i * CP * W;
    unsigned long long a = (unsigned long long)__double_as_longlong(fabs(p[0]));
    m = a > m ? a : m;
    if constexpr (CP == 2) {
      unsigned long long b = (unsigned long long)__double_as_longlong(fabs(p[W]));
      m = b > m ? b : m;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    unsigned long long o = __shfl_down_sync(0xffffffffu, m, off);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31) == 0 && m != 0ull) atomicMax(out, m);
}

// ---------------------------------------------------------------------------------------------
// Scalar logic of the methods (one thread).  Mirrors the control flow of BiCG (Algorithm 3),
// CGS, BiCGSTAB and GPBiCG; see krylov.cu for the vector steps between phases.
// ---------------------------------------------------------------------------------------------
template <int W, int CP>
__device__ __forceinline__ N<W, CP> slot(const double* S, int k) {
  return n_load<W, CP>(S + k * kSlotDoubles, 0);
}
template <int W, int CP>
__device__ __forceinline__ void set_slot(double* S, int k, const N<W, CP>& v) {
  n_store<W, CP>(S + k * kSlotDoubles, 0, v);
}
__device__ __forceinline__ void finish(int* st, int status, int iters) {
  st[ST_STATUS] = status;
  st[ST_ITERS] = iters;
  st[ST_DONE] = 1;
}
__device__ __forceinline__ void next_iter(int* st) {
  const int it = st[ST_IT] + 1;
  st[ST_IT] = it;
  if (it > st[ST_MAXIT]) finish(st, MPK_MAXIT, st[ST_MAXIT]);
}
// What follows a stopping test that did not stop iteration `it`: BiCGSTAB's omega = 0 and
// GPBiCG's zeta = 0 breakdowns, rho_old, and (BiCGSTAB, CGS) the next iteration.
template <int W, int CP>
__device__ __forceinline__ void after_norm(int method, double* __restrict__ S, int* __restrict__ st, int it) {
  if (method == MPK_BICGSTAB) {
    if (n_is_zero<W, CP>(n_load<W, CP>(S + S_OMEGA * kSlotDoubles, 0))) { finish(st, MPK_BREAKDOWN, it); return; }
    n_store<W, CP>(S + S_RHO_OLD * kSlotDoubles, 0, n_load<W, CP>(S + S_RHO * kSlotDoubles, 0));
    next_iter(st);
  } else if (method == MPK_CGS) {
    n_store<W, CP>(S + S_RHO_OLD * kSlotDoubles, 0, n_load<W, CP>(S + S_RHO * kSlotDoubles, 0));
    next_iter(st);
  } else if (method == MPK_GPBICG) {
    if (n_is_zero<W, CP>(n_load<W, CP>(S + S_ZETA * kSlotDoubles, 0))) finish(st, MPK_BREAKDOWN, it);
  }
}

// One thread per system: system sy uses S + sy * kSysDoubles, st + sy * ST_COUNT and
// hist + sy * hist_stride.  With done != nullptr a finished system is skipped; when a system
// finishes in a batch (fin != nullptr) it is counted, and the last one sets *alldone.
template <int W, int CP>
__device__ void scalar_phase(int method, int phase, double* __restrict__ S, int* __restrict__ st,
                             double* __restrict__ hist);
template <int W, int CP>
__global__ void k_scalar(int method, int phase, double* __restrict__ S, int* __restrict__ st,
                         double* __restrict__ hist, const int* __restrict__ done, int nsys, int hist_stride,
                         int* __restrict__ fin, int* __restrict__ alldone) {
  const int sy = blockIdx.x * blockDim.x + threadIdx.x;
  if (sy >= nsys || is_done(done)) return;
  int* sst = st + (int64_t)sy * ST_COUNT;
  if (done != nullptr && sst[ST_DONE] != 0) return;
  scalar_phase<W, CP>(method, phase, S + (int64_t)sy * kSysDoubles, sst,
                      hist != nullptr ? hist + (int64_t)sy * hist_stride : nullptr);
  // batch: a system that asked for a replacement check opens the check launches' gate, the word
  // after *alldone (cleared again at the end of the check)
  if (alldone != nullptr && phase == PH_NORM && sst[ST_NOCHK] == 0) alldone[1] = 0;
  if (fin != nullptr && sst[ST_DONE] != 0 && atomicAdd(fin, 1) == nsys - 1) *alldone = 1;
}
template <int W, int CP>
__device__ void scalar_phase(int method, int phase, double* __restrict__ S, int* __restrict__ st,
                             double* __restrict__ hist) {
  using Num = N<W, CP>;
  const int it = st[ST_IT];
  switch (phase) {
    case PH_INIT: {
      Num d = slot<W, CP>(S, S_D0);
      R<W> nr = rsqrt_mp<W>(d.re);
      const double r0n = nr.c[0];
      const double tol = S[S_TOL * kSlotDoubles + 1] * r0n + S[S_TOL * kSlotDoubles + 2];
      S[S_R0N * kSlotDoubles] = r0n;
      S[S_TOL * kSlotDoubles] = tol;
      Num nn = n_zero<W, CP>();
      nn.re = nr;
      set_slot<W, CP>(S, S_NORM, nn);
      if (hist) hist[0] = r0n;
      set_slot<W, CP>(S, S_ONE, n_real<W, CP>(1.0));
      set_slot<W, CP>(S, S_MONE, n_real<W, CP>(-1.0));
      set_slot<W, CP>(S, S_ZERO, n_zero<W, CP>());
      set_slot<W, CP>(S, S_BETA, n_zero<W, CP>());
      set_slot<W, CP>(S, S_NOMEGA, n_zero<W, CP>());
      st[ST_IT] = 1;
      if (r0n != r0n) finish(st, MPK_NAN, 0);
      else if (r0n < tol || r0n == 0.0) finish(st, MPK_OK, 0);
      else if (st[ST_MAXIT] < 1) finish(st, MPK_MAXIT, 0);
      break;
    }
    case PH_TRUE: {  // ||b - A x|| of the final iterate (S_D5) into S_D4 component 0
      if (st[ST_TRUEKNOWN] != 0) break;  // already there from the accepted check
      R<W> nr = rsqrt_mp<W>(slot<W, CP>(S, S_D5).re);
      S[S_D4 * kSlotDoubles] = nr.c[0];
      break;
    }
    case PH_STORE_RHO:
      set_slot<W, CP>(S, S_RHO, slot<W, CP>(S, S_D0));
      break;
    case PH_RHO: {
      Num rho = (method == MPK_GPBICG) ? slot<W, CP>(S, S_RHO) : slot<W, CP>(S, S_D0);
      if (n_is_zero<W, CP>(rho)) { finish(st, MPK_BREAKDOWN, it - 1); break; }
      set_slot<W, CP>(S, S_RHO, rho);
      if (method == MPK_BICGSTAB) {
        if (it == 1) {
          set_slot<W, CP>(S, S_BETA, n_zero<W, CP>());
          set_slot<W, CP>(S, S_NOMEGA, n_zero<W, CP>());
        } else {
          Num beta = n_mul<W, CP>(n_div<W, CP>(rho, slot<W, CP>(S, S_RHO_OLD)),
                                  n_div<W, CP>(slot<W, CP>(S, S_ALPHA), slot<W, CP>(S, S_OMEGA)));
          set_slot<W, CP>(S, S_BETA, beta);
        }
      } else if (method == MPK_CGS) {
        set_slot<W, CP>(S, S_BETA, it == 1 ? n_zero<W, CP>() : n_div<W, CP>(rho, slot<W, CP>(S, S_RHO_OLD)));
      }
      break;
    }
    case PH_SIG: {
      Num sig = slot<W, CP>(S, S_D0), rho = slot<W, CP>(S, S_RHO);
      if (n_is_zero<W, CP>(sig) || (method == MPK_BICG && n_is_zero<W, CP>(rho))) {
        finish(st, MPK_BREAKDOWN, it - 1);
        break;
      }
      Num alpha = n_div<W, CP>(rho, sig);
      set_slot<W, CP>(S, S_SIG, sig);
      set_slot<W, CP>(S, S_ALPHA, alpha);
      set_slot<W, CP>(S, S_NALPHA, n_neg<W, CP>(alpha));
      set_slot<W, CP>(S, S_NCALPHA, n_neg<W, CP>(n_conj<W, CP>(alpha)));
      break;
    }
    case PH_OMEGA: {
      Num ts = slot<W, CP>(S, S_D0), tt = slot<W, CP>(S, S_D1);
      Num om = n_is_zero<W, CP>(tt) ? n_zero<W, CP>() : n_div<W, CP>(ts, tt);
      set_slot<W, CP>(S, S_OMEGA, om);
      set_slot<W, CP>(S, S_NOMEGA, n_neg<W, CP>(om));
      break;
    }
    case PH_ZETA: {
      Num cc = slot<W, CP>(S, S_D0), ct = slot<W, CP>(S, S_D1);
      Num zeta, eta;
      if (n_is_zero<W, CP>(cc)) {
        zeta = n_zero<W, CP>();
        eta = n_zero<W, CP>();
      } else if (it == 1 || (st[ST_FLAGS] & 1)) {
        zeta = n_div<W, CP>(ct, cc);
        eta = n_zero<W, CP>();
      } else {
        Num yy = slot<W, CP>(S, S_D2), yt = slot<W, CP>(S, S_D3), cy = slot<W, CP>(S, S_D4), yc = slot<W, CP>(S, S_D5);
        Num det = n_sub<W, CP>(n_mul<W, CP>(cc, yy), n_mul<W, CP>(cy, yc));
        if (n_is_zero<W, CP>(det)) { finish(st, MPK_BREAKDOWN, it - 1); break; }
        zeta = n_div<W, CP>(n_sub<W, CP>(n_mul<W, CP>(yy, ct), n_mul<W, CP>(cy, yt)), det);
        eta = n_div<W, CP>(n_sub<W, CP>(n_mul<W, CP>(cc, yt), n_mul<W, CP>(yc, ct)), det);
      }
      set_slot<W, CP>(S, S_ZETA, zeta);
      set_slot<W, CP>(S, S_NZETA, n_neg<W, CP>(zeta));
      set_slot<W, CP>(S, S_ETA, eta);
      set_slot<W, CP>(S, S_NETA, n_neg<W, CP>(eta));
      break;
    }
    case PH_NORM: {
      R<W> nr = rsqrt_mp<W>(slot<W, CP>(S, S_D0).re);
      Num nn = n_zero<W, CP>();
      nn.re = nr;
      set_slot<W, CP>(S, S_NORM, nn);
      if (hist) hist[it] = nr.c[0];
      st[ST_NOCHK] = 1;
      st[ST_NOREPL] = 1;
      if (nr.c[0] != nr.c[0]) { finish(st, MPK_NAN, it); break; }
      const int period = st[ST_PERIOD];
      if (nr.c[0] < S[S_TOL * kSlotDoubles]) {
        if (period <= 0) { finish(st, MPK_OK, it); break; }
        st[ST_CHECK] = 2;  // the test passed: it stands only if the true residual agrees
        st[ST_CHK_IT] = it;
        st[ST_NOCHK] = 0;
        break;
      }
      if (period > 0 && it % period == 0) {
        st[ST_CHECK] = 1;
        st[ST_CHK_IT] = it;
        st[ST_NOCHK] = 0;
      }
      after_norm<W, CP>(method, S, st, it);
      break;
    }
    case PH_TRUECHK: {  // ||b - A x_k||^2 in S_D5; hist: the true-residual history
      if (st[ST_NOCHK] != 0) break;
      st[ST_NOCHK] = 1;
      const int k = st[ST_CHK_IT];
      const bool passed = st[ST_CHECK] == 2;
      st[ST_CHECK] = 0;
      R<W> nt = rsqrt_mp<W>(slot<W, CP>(S, S_D5).re);
      if (hist) hist[k] = nt.c[0];
      if (nt.c[0] > 10.0 * S[S_TOL * kSlotDoubles]) {
        st[ST_NOREPL] = 0;  // r := b - A x_k (the launch after this one)
        st[ST_NREP] += 1;
        if (passed) after_norm<W, CP>(method, S, st, k);
      } else if (passed) {
        S[S_D4 * kSlotDoubles] = nt.c[0];  // the final true norm: no recomputation after the loop
        st[ST_TRUEKNOWN] = 1;
        finish(st, MPK_OK, k);
      }
      break;
    }
    case PH_BETA: {
      Num rhon = slot<W, CP>(S, S_D0), rho = slot<W, CP>(S, S_RHO), beta;
      if (method == MPK_BICG) {
        beta = n_div<W, CP>(rhon, rho);
        set_slot<W, CP>(S, S_CBETA, n_conj<W, CP>(beta));
      } else {
        beta = n_mul<W, CP>(n_div<W, CP>(slot<W, CP>(S, S_ALPHA), slot<W, CP>(S, S_ZETA)), n_div<W, CP>(rhon, rho));
      }
      set_slot<W, CP>(S, S_BETA, beta);
      set_slot<W, CP>(S, S_RHO, rhon);
      next_iter(st);
      break;
    }
    default:
      break;
  }
}

// ---------------------------------------------------------------------------------------------
// Dependency-driven ("sync-free") row processing shared by the ILU(0) factorisation and the
// substitutions.  Rows are taken in the order of a permutation `perm` (position -> row, -1 for
// an empty position; `pos` is the inverse) in which every row comes after the rows it depends
// on: the library uses rows sorted by their level in the dependency graph, so the 32 lanes of a
// warp hold 32 independent rows of one wavefront.  A warp takes 32 consecutive positions at a
// time through a ticket counter.  Each lane owns one row and consumes its entries strictly in
// CSR order (so every row sees the same operation sequence as the sequential algorithm), but
// fetches the values of rows owned by other warps ahead of time into a small lookahead window
// as soon as they are published; rows of its own warp are passed by warp shuffle.  A warp only
// waits for rows at earlier positions, taken by running warps, so the scheme cannot deadlock;
// every wait is still bounded by kWaitCycles, after which the kernel records MPK_TIMEOUT in
// ctl[CTL_ERR] and all warps leave.  Warps that make no progress back off with __nanosleep.
// `Row` provides: type Val; begin(i, p, pend); fetch(j, Val&) (row j owned by another warp:
// published yet? value); consume(p, j, const Val&); finish() -> Val; publish(const Val&).
// ---------------------------------------------------------------------------------------------
struct Empty {};
__device__ __forceinline__ Empty shfl_val(const Empty& v, int) { return v; }
__device__ __forceinline__ float shfl_val(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ int shfl_val(int v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ float2 shfl_val(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
template <int W, int CP>
__device__ __forceinline__ N<W, CP> shfl_val(const N<W, CP>& a, int src) {
  N<W, CP> z;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    z.re.c[k] = __shfl_sync(0xffffffffu, a.re.c[k], src);
    z.im.c[k] = CP == 2 ? __shfl_sync(0xffffffffu, a.im.c[k], src) : 0.0;
  }
  return z;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}


template <class Row>
__device__ __forceinline__ void syncfree_rows(const Order ord, const int* __restrict__ ci, int* ticket, int* ctl,
                                              Row& row) {
  using V = typename Row::Val;
  using Raw = typename Row::Raw;
  constexpr int K = Row::kLook;  // lookahead window (entries fetched ahead of use)
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nchunks = (ord.npos + 31) >> 5;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(ticket, 1);
    chunk = __shfl_sync(FULL, chunk, 0);
    if (chunk >= nchunks) return;
    const int base = chunk << 5;
    const int k = base + lane;
    const int ik = k < ord.npos ? ord.perm[k] : -1;
    const bool valid = ik >= 0;
    const int i = valid ? ik : 0;
    int p = 0, pend = 0;
    if (valid) row.begin(i, p, pend);
    // window q <-> entry p + q: column, position of that row, fetched value
    int wj[K], wk[K];
    V win[K];
    unsigned have = 0u;
#pragma unroll
    for (int q = 0; q < K; ++q) {
      wj[q] = (valid && p + q < pend) ? ci[p + q] : -1;
      wk[q] = wj[q] >= 0 ? ord.pos[wj[q]] : INT_MAX;
    }
    V mine{};
    bool fin = !valid;
    if (valid && p >= pend) {
      mine = row.finish();
      row.publish(mine);
      fin = true;
    }
    unsigned finmask = __ballot_sync(FULL, fin);
    long long t0 = clock64();
    unsigned backoff = 0u;
    int rounds = 0, patience = 0;
    while (finmask != FULL) {
      bool progressed = false;
      // (1) fetch published out-of-warp entries of the window: issue every load, then check
      if (!fin) {
        Raw raw[K];
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (wj[q] >= 0 && wk[q] < base && !((have >> q) & 1u)) row.issue(wj[q], raw[q]);
#pragma unroll
        for (int q = 0; q < K; ++q)
          if (wj[q] >= 0 && wk[q] < base && !((have >> q) & 1u) && row.check(wj[q], raw[q], win[q])) {
            have |= 1u << q;
            progressed = true;
          }
      }
      // (2) consume in CSR order while possible; in-warp values arrive by shuffle.  Rows with
      // expensive arithmetic (Row::kBatch rounds of patience) wait until every unfinished lane of
      // the warp can proceed, so that their arithmetic runs with all lanes active.
      bool go = true;
      if constexpr (Row::kBatch > 0) {
        bool lane_ok = true;  // every window entry fetched, or owned by a lane of this warp
        if (!fin) {
#pragma unroll
          for (int q = 0; q < K; ++q)
            if (wj[q] >= 0 && wk[q] < base && !((have >> q) & 1u)) lane_ok = false;
        }
        if (!__all_sync(FULL, lane_ok) && ++patience <= Row::kBatch) go = false;
        else patience = 0;
      }
      for (; go;) {
        int src = lane;
        bool can = false, from_lane = false;
        if (!fin && p < pend) {
          if (have & 1u) {
            can = true;
          } else if (wk[0] >= base && ((finmask >> (wk[0] - base)) & 1u)) {
            can = true;
            from_lane = true;
            src = wk[0] - base;
          }
        }
        const V sv = shfl_val(mine, src);
        bool step = false;
        if (can) {
          row.consume(p, wj[0], from_lane ? sv : win[0]);
          ++p;
#pragma unroll
          for (int q = 0; q < K - 1; ++q) {
            win[q] = win[q + 1];
            wj[q] = wj[q + 1];
            wk[q] = wk[q + 1];
          }
          wj[K - 1] = p + K - 1 < pend ? ci[p + K - 1] : -1;
          wk[K - 1] = wj[K - 1] >= 0 ? ord.pos[wj[K - 1]] : INT_MAX;
          have >>= 1;
          step = true;
          if (p >= pend) {
            mine = row.finish();
            row.publish(mine);
            fin = true;
          }
        }
        __syncwarp();
        finmask = __ballot_sync(FULL, fin);
        if (!__any_sync(FULL, step)) break;
        progressed = true;
      }
      if (finmask == FULL) break;
      // (3) bounded waiting, error propagation, backoff
      const bool any_prog = __any_sync(FULL, progressed);
      if (any_prog) {
        t0 = clock64();
        backoff = 0u;
      } else {
        int stop = 0;
        if (lane == 0) {
          if (clock64() - t0 > kWaitCycles) {
            atomicCAS(ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
            stop = 1;
          } else if ((++rounds & 15) == 0 && ld_relaxed(ctl + CTL_ERR) != 0) {
            stop = 1;
          }
        }
        if (__shfl_sync(FULL, stop, 0)) return;
        backoff = backoff == 0u ? 32u : (backoff < 1024u ? 2u * backoff : 1024u);
        __nanosleep(backoff);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------------
// binary32 / bfloat16 factor access
__device__ __forceinline__ float ld_fac(const float* f, int64_t idx) { return f[idx]; }
__device__ __forceinline__ float ld_fac(const uint16_t* f, int64_t idx) {
  return __uint_as_float(((unsigned)f[idx]) << 16);
}

__device__ __forceinline__ int scale_exponent(const unsigned long long* absmax) {
  const double mx = __longlong_as_double((long long)*absmax);
  int e = 0;
  if (mx > 0.0 && isfinite(mx)) frexp(mx, &e);
  return e;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// ---------------------------------------------------------------------------------------------
// Chunk dataflow for the substitutions and the ILU(0) factorisation.  Rows are sorted by their
// level in the dependency graph (0: no dependency, else 1 + the largest level of the rows they
// depend on) and every level is padded to whole 32-row chunks, so the lanes of a warp hold
// independent rows and compute in lockstep.  Warps take chunks in level order through a ticket
// counter.  Before computing, every lane polls (relaxed loads, backoff) the completion flags of
// the chunks holding its row's dependencies; once all lanes are satisfied the warp executes one
// acquire fence, computes its rows with ordinary loads and stores, and lane 0 stamps the
// chunk's flag with the current epoch by a release store.  Dependencies lie in earlier levels,
// whose chunks have earlier tickets and belong to running warps: no deadlock.  Every wait is
// bounded by kWaitCycles (then MPK_TIMEOUT in ctl[CTL_ERR] and all warps leave).  `Row`
// provides: type Val; begin(i, p, pend); Val load(j); consume(p, j, Val); Val finish();
// store(Val).
// ---------------------------------------------------------------------------------------------
template <class Row>
__device__ __forceinline__ void chunk_rows(const LevelOrder lo, const int* __restrict__ ci, int epoch, int* ticket,
                                           int* ctl, Row& row) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nchunks = *lo.nchunks;
  for (;;) {
    int chunk = 0;
    if (lane == 0) chunk = atomicAdd(ticket, 1);
    chunk = __shfl_sync(FULL, chunk, 0);
    if (chunk >= nchunks) return;
    const int i = lo.perm[(chunk << 5) + lane];
    int p = 0, pend = 0;
    if (i >= 0) row.begin(i, p, pend);
    // wait for the chunks this row depends on, kDepBatch dependencies at a time: their columns,
    // positions and flags are each loaded together (one memory round trip per step, not per
    // dependency)
    constexpr int kDepBatch = 4;
    bool timeout = false;
    {
      const long long t0 = clock64();
      unsigned backoff = 0u;
      int rounds = 0;
      for (int q0 = p; q0 < pend && !timeout; q0 += kDepBatch) {
        int cc[kDepBatch];
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k) cc[k] = q0 + k < pend ? ci[q0 + k] : -1;
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k) cc[k] = cc[k] >= 0 ? (lo.pos[cc[k]] >> 5) : -1;
        unsigned need = 0u;
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k)
          if (cc[k] >= 0) need |= 1u << k;
        while (need != 0u) {
          int f[kDepBatch];
#pragma unroll
          for (int k = 0; k < kDepBatch; ++k) f[k] = ((need >> k) & 1u) ? ld_relaxed(lo.flags + cc[k]) : epoch;
#pragma unroll
          for (int k = 0; k < kDepBatch; ++k)
            if (f[k] == epoch) need &= ~(1u << k);
          if (need == 0u) break;
          if (clock64() - t0 > kWaitCycles) { timeout = true; break; }
          if ((++rounds & 31) == 0 && ld_relaxed(ctl + CTL_ERR) != 0) { timeout = true; break; }
          backoff = backoff == 0u ? 32u : (backoff < 512u ? 2u * backoff : 512u);
          __nanosleep(backoff);
        }
      }
    }
    if (__any_sync(FULL, timeout)) {
      if (lane == 0) atomicCAS(ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
      return;
    }
    fence_acq_rel();
    if (i >= 0) {
      // the rows' finished data (Row::load) is fetched for a batch of dependencies before the
      // batch is consumed in order
      for (int q0 = p; q0 < pend; q0 += kDepBatch) {
        int jj[kDepBatch];
        typename Row::Val v[kDepBatch];
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k) jj[k] = q0 + k < pend ? ci[q0 + k] : -1;
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k)
          if (jj[k] >= 0) v[k] = row.load(jj[k]);
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k)
          if (jj[k] >= 0) row.consume(q0 + k, jj[k], v[k]);
      }
      row.store(row.finish());
    }
    __syncwarp();
    if (lane == 0) st_release(lo.flags + chunk, epoch);
  }
}

// Grid-wide barrier of a co-resident (cooperative) grid on the control words CTL_BAR_COUNT
// (arrivals) and CTL_BAR_GEN (generation).  Thread 0 of every block reads the generation, makes
// the block's writes visible (fence after the block barrier) and arrives; the last arrival
// resets the count and publishes the next generation, the others wait for it.  Every wait is
// bounded by kWaitCycles (then MPK_TIMEOUT) and ends early once a block has reported an error.
// Returns false when the grid must stop.
__device__ __forceinline__ bool grid_barrier(int* ctl) {
  __shared__ int s_go;
  __syncthreads();
  if (threadIdx.x == 0) {
    int go = 1;
    unsigned* cnt = (unsigned*)(ctl + CTL_BAR_COUNT);
    const int gen = ld_acquire(ctl + CTL_BAR_GEN);
    __threadfence();
    if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
      atomicExch(cnt, 0u);
      __threadfence();
      st_release(ctl + CTL_BAR_GEN, gen + 1);
    } else {
      const long long t0 = clock64();
      int rounds = 0;
      while (ld_acquire(ctl + CTL_BAR_GEN) == gen) {
        if (clock64() - t0 > kWaitCycles) {
          atomicCAS(ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
          go = 0;
          break;
        }
        if ((++rounds & 15) == 0 && ld_relaxed(ctl + CTL_ERR) != 0) {
          go = 0;
          break;
        }
        if (rounds > 64) __nanosleep(64);
      }
    }
    __threadfence();
    s_go = go;
  }
  __syncthreads();
  return s_go != 0;
}

// Level-synchronous form of chunk_rows for a co-resident (cooperative) grid: the chunks of level
// l (lo.lstart[l] .. lo.lstart[l + 1]) are dealt over all warps, warp g taking lstart[l] + g,
// + G, ... (g numbered so that consecutive chunks fall on different SMs), and a grid barrier
// separates the levels.  A row depends on rows of earlier levels only, which are final after the
// barrier: no flags, no polling, no fences per chunk.  The Row calls are those of chunk_rows.
template <class Row>
__device__ __forceinline__ void level_rows(const LevelOrder lo, const int* __restrict__ ci, int* ctl, Row& row) {
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x * (blockDim.x >> 5);
  const int g = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  constexpr int kDepBatch = 4;
  for (int l = 0; l < lo.nlev; ++l) {
    const int c1 = lo.lstart[l + 1];
    for (int c = lo.lstart[l] + g; c < c1; c += G) {
      const int i = lo.perm[(c << 5) + lane];
      if (i < 0) continue;
      int p = 0, pend = 0;
      row.begin(i, p, pend);
      for (int q0 = p; q0 < pend; q0 += kDepBatch) {
        int jj[kDepBatch];
        typename Row::Val v[kDepBatch];
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k) jj[k] = q0 + k < pend ? ci[q0 + k] : -1;
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k)
          if (jj[k] >= 0) v[k] = row.load(jj[k]);
#pragma unroll
        for (int k = 0; k < kDepBatch; ++k)
          if (jj[k] >= 0) row.consume(q0 + k, jj[k], v[k]);
      }
      row.store(row.finish());
    }
    if (l + 1 < lo.nlev && !grid_barrier(ctl)) return;
  }
}

// Binary64 factor, w-component vectors (paper's "_d" substitutions): row i computes
//   acc = in_i;  acc -= f_ij * out_j  for the row's entries of the triangle in CSR order;
//   upper triangle: acc /= f_ii;  out_i = acc,
// every product and difference in w-component arithmetic (the sequential order of Algorithm 2).
//
// Schedule (static, balanced): the rows come in their triangle's level order, every level
// padded to whole 32-row chunks and sorted by row length within the level, from the repacked
// triangle (SellTri: coalesced columns and values per chunk).  The grid has one block per SM and
// WPB warps per block, all co-resident (cooperative launch); chunk c belongs to warp c mod G
// (G = warps in the grid), numbered so that consecutive chunks of a level fall on different SMs
// and, once every SM has one, on the next sub-partition.  A level of up to 4 x 152 chunks thus
// puts at most one chunk on each FP64 unit: on this GPU an FP64 warp instruction holds its
// sub-partition's unit for 64 cycles whatever the number of active lanes, so a level costs one
// chunk's instruction count, not a multiple of it.  Wide, shallow level structures (many chunks
// per level) want more warps per SM to overlap their memory latency: WPB is chosen per matrix
// pattern by the autotuner.  Each warp walks its chunks in increasing order; every dependency of
// a chunk lies in an earlier level, i.e. in a smaller chunk, so the smallest unfinished chunk can
// always proceed (no deadlock).
// Completion is carried by the values themselves: before the pass, `out` is filled with the
// sentinel bit pattern kSent (k_fill_sent), a finished row stores its w-component value with
// strong relaxed 64-bit stores (a computed value equal to kSent is stored as another NaN), and a
// dependent row polls those words with strong relaxed loads until none is kSent.  Each word is
// written once per pass, so a word that is not kSent is final: no flag, no fence.  Entries are
// handled in groups of KG: the group's columns and values are loaded together, all its
// dependencies polled together (warp-uniform loop: lanes that are ready early do not run the
// FP64 arithmetic as a separate divergent group), then consumed in CSR order.  The first group
// of a chunk and the next chunk's position are fetched ahead; lane 0 first polls the chunk's
// latest dependency alone.  Every wait is bounded by kWaitCycles (then MPK_TIMEOUT in
// ctl[CTL_ERR] and all warps leave).
constexpr int kTrsvWpbChoices[4] = {4, 8, 16, 32};  // candidate warps per block (per SM)
constexpr long long kSpinCycles = 40000;            // ~20 us of polling without sleeping
constexpr unsigned long long kSent = 0xFFFFFFFFFFFFFFFFull;

__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return __longlong_as_double((long long)v);
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double x) {
  unsigned long long v = (unsigned long long)__double_as_longlong(x);
  if (v == kSent) v = 0x7FF8000000000000ull;  // never publish the sentinel
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Double-word (and quad-word) values as one (two) 16-byte strong accesses where the vector is
// 16-byte aligned (half the requests; each word is still checked on its own, so a value seen
// half-written is polled again), else word by word.
__device__ __forceinline__ void ld_relaxed_f64x2(const double* p, double& a, double& b) {
  asm volatile("ld.relaxed.gpu.global.v2.f64 {%0, %1}, [%2];" : "=d"(a), "=d"(b) : "l"(p) : "memory");
}
__device__ __forceinline__ void st_relaxed_f64x2(double* p, double a, double b) {
  unsigned long long ua = (unsigned long long)__double_as_longlong(a), ub = (unsigned long long)__double_as_longlong(b);
  if (ua == kSent) ua = 0x7FF8000000000000ull;  // never publish the sentinel
  if (ub == kSent) ub = 0x7FF8000000000000ull;
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(ua), "l"(ub) : "memory");
}
__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
template <int W, int CP>
__device__ __forceinline__ void n_fetch(const double* __restrict__ v, int64_t i, N<W, CP>& z) {
  const double* p = v + i * (CP * W);
  if constexpr (W == 2 || W == 4) {  // (a TD value's 24-byte stride breaks the alignment)
    if (aligned16(v)) {
#pragma unroll
      for (int k = 0; k < W; k += 2) ld_relaxed_f64x2(p + k, z.re.c[k], z.re.c[k + 1]);
      if constexpr (CP == 2) {
#pragma unroll
        for (int k = 0; k < W; k += 2) ld_relaxed_f64x2(p + W + k, z.im.c[k], z.im.c[k + 1]);
      }
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) z.re.c[k] = ld_relaxed_f64(p + k);
  if constexpr (CP == 2) {
#pragma unroll
    for (int k = 0; k < W; ++k) z.im.c[k] = ld_relaxed_f64(p + W + k);
  }
}
template <int W, int CP>
__device__ __forceinline__ bool n_ready(const N<W, CP>& z) {  // no word is the sentinel
  bool ok = true;
#pragma unroll
  for (int k = 0; k < W; ++k) ok = ok && (unsigned long long)__double_as_longlong(z.re.c[k]) != kSent;
  if constexpr (CP == 2) {
#pragma unroll
    for (int k = 0; k < W; ++k) ok = ok && (unsigned long long)__double_as_longlong(z.im.c[k]) != kSent;
  }
  return ok;
}
template <int W, int CP>
__device__ __forceinline__ bool n_poll(const double* __restrict__ v, int64_t i, N<W, CP>& z) {
  n_fetch<W, CP>(v, i, z);
  return n_ready<W, CP>(z);
}
template <int W, int CP>
__device__ __forceinline__ void n_publish(double* __restrict__ v, int64_t i, const N<W, CP>& z) {
  double* p = v + i * (CP * W);
  if constexpr (W == 2 || W == 4) {
    if (aligned16(v)) {
#pragma unroll
      for (int k = 0; k < W; k += 2) st_relaxed_f64x2(p + k, z.re.c[k], z.re.c[k + 1]);
      if constexpr (CP == 2) {
#pragma unroll
        for (int k = 0; k < W; k += 2) st_relaxed_f64x2(p + W + k, z.im.c[k], z.im.c[k + 1]);
      }
      return;
    }
  }
#pragma unroll
  for (int k = 0; k < W; ++k) st_relaxed_f64(p + k, z.re.c[k]);
  if constexpr (CP == 2) {
#pragma unroll
    for (int k = 0; k < W; ++k) st_relaxed_f64(p + W + k, z.im.c[k]);
  }
}
static __global__ void __launch_bounds__(kBlock) k_fill_sent(int64_t m, double* __restrict__ a, int64_t mb,
                                                             double* __restrict__ b, const int* __restrict__ done) {
  if (is_done(done)) return;
  const double s = __longlong_as_double((long long)kSent);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m + mb; k += (int64_t)gridDim.x * blockDim.x) {
    if (k < m) a[k] = s;
    else b[k - m] = s;
  }
}

// Bounded wait bookkeeping shared by the substitution kernels: true once the wait must end.
__device__ __forceinline__ bool wait_expired(long long t0, int& polls, const int* ctl) {
  const long long dt = clock64() - t0;
  return dt > kWaitCycles || ((++polls & 63) == 0 && ld_relaxed(ctl + CTL_ERR) != 0);
}
__device__ __forceinline__ void wait_pause(long long t0, int ns) {
  if (clock64() - t0 > kSpinCycles) __nanosleep(ns);
}

// MF (MPK_ILU_MP handle): the factor values are w-component numbers (CP * W doubles per slot)
// and row i computes acc -= f_ij * out_j with the factor first in the product, then
// acc /= f_ii, both in w-component arithmetic; fewer entries per group keep the values in
// registers.
//
// One chunk (32 rows) of the substitution, shared by both schedules, in three steps so that a
// schedule can load a chunk's operands ahead of its dependencies: mp_meta (the row and slot
// range), mp_operands (the first group of entries, the right-hand side, the diagonal) and
// mp_finish (dependency waits, arithmetic, publication).  ring (owner-block schedule; nullptr
// otherwise): the block's shared-memory values, read for the entries encoded as local
// (col <= -2) and written at own_slot.  mp_finish returns the warp-uniform timeout flag.
// Shared-memory ring of an owner-block schedule as seen by one CTA: its own ring (base, and its
// 32-bit shared address sa) and its rank in the cluster; a local dependency code
// rank * kRing + slot names a slot of CTA `rank` (rank 0 and csize 1 without clusters).
struct RingRef {
  void* base = nullptr;  // nullptr: static schedule, no ring
  unsigned sa = 0;
  unsigned rank = 0;
};
__device__ __forceinline__ unsigned cta_rank_in_cluster() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cluster_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {  // release / acquire: orders shared-memory values
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_addr(unsigned sa, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(sa), "r"(rank));
  return r;
}
__device__ __forceinline__ double ld_cluster_f64(unsigned a) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float ld_cluster_f32(unsigned a) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_cluster_s32(unsigned a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
template <int W, int CP>
__device__ __forceinline__ N<W, CP> ring_read(const RingRef& R, int code) {
  const unsigned rank = (unsigned)(code / kRing);
  const int slot = code - (int)rank * kRing;
  if (rank == R.rank) return n_load<W, CP>((const double*)R.base, slot);
  N<W, CP> z = n_zero<W, CP>();
  const unsigned a = cluster_addr(R.sa + (unsigned)slot * (CP * W * 8), rank);
#pragma unroll
  for (int k = 0; k < W; ++k) z.re.c[k] = ld_cluster_f64(a + 8u * k);
  if constexpr (CP == 2) {
#pragma unroll
    for (int k = 0; k < W; ++k) z.im.c[k] = ld_cluster_f64(a + 8u * (W + k));
  }
  return z;
}
template <int CP>
__device__ __forceinline__ void ring_read32(const RingRef& R, int code, float& xr, float& xi) {
  const unsigned rank = (unsigned)(code / kRing);
  const int slot = code - (int)rank * kRing;
  if (rank == R.rank) {
    const float* b = (const float*)R.base;
    xr = b[slot * CP];
    xi = CP == 2 ? b[slot * CP + 1] : 0.0f;
    return;
  }
  const unsigned a = cluster_addr(R.sa + (unsigned)slot * (CP * 4), rank);
  xr = ld_cluster_f32(a);
  xi = CP == 2 ? ld_cluster_f32(a + 4u) : 0.0f;
}

template <int W, int CP, bool MF>
struct MpChunk {
  static constexpr int KG = (MF && W * CP >= 4) ? 2 : 4;  // entries per group
  int i, b0, w, rep;
  int jj[KG];
  double fr[KG], fi[KG];
  N<W, CP> fv[MF ? KG : 1];
  N<W, CP> acc, dv;
  double dr, di;
};
template <int W, int CP, bool MF>
__device__ __forceinline__ void mp_meta(const SellTri& T, int chunk, MpChunk<W, CP, MF>& c) {
  const int lane = threadIdx.x & 31;
  c.i = T.perm[(chunk << 5) + lane];
  c.b0 = T.coff[chunk];
  c.w = T.coff[chunk + 1] - c.b0;
  c.rep = T.rep[chunk];
}
template <int W, int CP, bool MF>
__device__ __forceinline__ void mp_group(const SellTri& T, int k0, MpChunk<W, CP, MF>& c) {
  const double* __restrict__ tval = (const double*)T.val;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < MpChunk<W, CP, MF>::KG; ++k) {
    c.jj[k] = -1;
    c.fr[k] = 0.0;
    c.fi[k] = 0.0;
    if constexpr (MF) c.fv[k] = n_zero<W, CP>();
    if (k0 + k < c.w) {
      const int64_t e = ((int64_t)(c.b0 + k0 + k) << 5) + lane;
      c.jj[k] = T.col[e];
      if constexpr (MF) c.fv[k] = n_load<W, CP>(tval, e);
      else if constexpr (CP == 1) c.fr[k] = tval[e];
      else { c.fr[k] = tval[2 * e]; c.fi[k] = tval[2 * e + 1]; }
    }
  }
}
template <int W, int CP, bool MF>
__device__ __forceinline__ void mp_operands(const SellTri& T, bool unit, const double* __restrict__ in, int chunk,
                                            MpChunk<W, CP, MF>& c) {
  const double* __restrict__ tdia = (const double*)T.dia;
  const int lane = threadIdx.x & 31;
  mp_group<W, CP, MF>(T, 0, c);
  c.acc = n_zero<W, CP>();
  c.dr = 1.0;
  c.di = 0.0;
  c.dv = n_real<W, CP>(1.0);
  if (c.i >= 0) {
    c.acc = n_load<W, CP>(in, c.i);
    if (!unit) {
      const int64_t q = ((int64_t)chunk << 5) + lane;
      if constexpr (MF) c.dv = n_load<W, CP>(tdia, q);
      else if constexpr (CP == 1) c.dr = tdia[q];
      else { c.dr = tdia[2 * q]; c.di = tdia[2 * q + 1]; }
    }
  }
}
template <int W, int CP, bool MF, bool RING>
__device__ __forceinline__ bool mp_finish(const SellTri& T, const IluHandleView& M, bool unit,
                                          double* __restrict__ out, MpChunk<W, CP, MF>& c, const RingRef& R,
                                          int own_slot) {
  constexpr int KG = MpChunk<W, CP, MF>::KG;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool timeout = false;
  const long long t0 = clock64();
  int polls = 0;
  if (lane == 0 && c.rep >= 0 && M.poll == 0) {  // the chunk's latest dependency, polled by one lane
    N<W, CP> r;
    while (!n_poll<W, CP>(out, c.rep, r)) {
      if (wait_expired(t0, polls, M.ctl)) { timeout = true; break; }
      wait_pause(t0, 128);
    }
  }
  __syncwarp();
  N<W, CP> acc = c.acc;
  for (int k0 = 0; k0 < c.w; k0 += KG) {
    if (k0 > 0) mp_group<W, CP, MF>(T, k0, c);
    N<W, CP> v[KG];
    unsigned need = 0u;
#pragma unroll
    for (int k = 0; k < KG; ++k) {
      v[k] = n_zero<W, CP>();
      if (c.jj[k] >= 0) need |= 1u << k;
      else if (RING && c.jj[k] <= -2) v[k] = ring_read<W, CP>(R, -2 - c.jj[k]);  // computed by this block
    }
    while (__any_sync(FULL, need != 0u && !timeout)) {
      // every outstanding load of the round is issued before any is checked
#pragma unroll
      for (int k = 0; k < KG; ++k)
        if ((need >> k) & 1u) n_fetch<W, CP>(out, c.jj[k], v[k]);
      unsigned got = 0u;
#pragma unroll
      for (int k = 0; k < KG; ++k)
        if (((need >> k) & 1u) && n_ready<W, CP>(v[k])) got |= 1u << k;
      need &= ~got;
      if (need != 0u && !timeout && wait_expired(t0, polls, M.ctl)) timeout = true;
      if (__any_sync(FULL, need != 0u)) {
        if (M.poll == 1) wait_pause(t0, 64);
        else __nanosleep(M.poll == 2 ? (unsigned)M.poll_ns : 64u);
      }
    }
    __syncwarp();
    if (!timeout && c.i >= 0) {
#pragma unroll
      for (int k = 0; k < KG; ++k) {
        if (c.jj[k] == -1) continue;
        if constexpr (MF) acc = n_sub<W, CP>(acc, n_mul<W, CP>(c.fv[k], v[k]));
        else acc = n_sub<W, CP>(acc, n_mul_fp<W, CP>(v[k], c.fr[k], c.fi[k]));
      }
    }
  }
  if (!timeout && c.i >= 0 && c.i != M.withhold) {
    if (!unit) {
      if constexpr (MF) acc = n_div<W, CP>(acc, c.dv);
      else acc = n_div_fp<W, CP>(acc, c.dr, c.di);
    }
    n_publish<W, CP>(out, c.i, acc);
    if constexpr (RING) n_store<W, CP>((double*)R.base, own_slot, acc);
  }
  return __any_sync(FULL, timeout);
}

template <int W, int CP, int WPB, bool MF>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_mp(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
              const int* __restrict__ done) {
  if (is_done(done)) return;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x * (blockDim.x >> 5);
  const int g = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  // Two chunks ahead: the next chunk's operands (right-hand side, diagonal, first group of
  // factor entries; none of them written by this launch) and the rows of the one after it are
  // loaded before the current chunk waits, so a warp that finishes a chunk late starts the next
  // one without a load round trip.  At 32 warps per SM (64 registers a thread) the warps hide
  // that latency instead, and only the next chunk's rows are loaded ahead.
  constexpr bool AHEAD = WPB < 32;
  MpChunk<W, CP, MF> c, nx, mm;
  if (g < T.nchunks) {
    mp_meta<W, CP, MF>(T, g, nx);
    if constexpr (AHEAD) mp_operands<W, CP, MF>(T, unit, in, g, nx);
  }
  if (AHEAD && g + G < T.nchunks) mp_meta<W, CP, MF>(T, g + G, mm);
  for (int chunk = g; chunk < T.nchunks; chunk += G) {
    if constexpr (AHEAD) {
      c = nx;
      if (chunk + G < T.nchunks) {
        nx.i = mm.i;
        nx.b0 = mm.b0;
        nx.w = mm.w;
        nx.rep = mm.rep;
        mp_operands<W, CP, MF>(T, unit, in, chunk + G, nx);
      }
      if (chunk + 2 * G < T.nchunks) mp_meta<W, CP, MF>(T, chunk + 2 * G, mm);
    } else {
      c.i = nx.i;
      c.b0 = nx.b0;
      c.w = nx.w;
      c.rep = nx.rep;
      mp_operands<W, CP, MF>(T, unit, in, chunk, c);
      if (chunk + G < T.nchunks) mp_meta<W, CP, MF>(T, chunk + G, nx);
    }
    if (mp_finish<W, CP, MF, false>(T, M, unit, out, c, RingRef(), 0)) {
      if (lane == 0) atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
      return;
    }
  }
}

// Complex substitution with a binary64 factor, each 32-row chunk shared by a pair of warps of one
// block (consecutive warps, so different sub-partitions): the even warp computes the real parts
// of the chunk's rows, the odd warp the imaginary parts.  Every step is the one the single-warp
// kernel performs for that part -- the product's part re = a.re fr - a.im fi or
// im = a.im fr + a.re fi, then acc_part - product_part, in CSR order -- so the results are the
// same bits; the division by the diagonal needs both parts of the accumulator, which the two
// warps exchange through shared memory (double-buffered, one named barrier per chunk).  A binary64
// warp instruction costs its sub-partition 64 cycles however many lanes run, so splitting a row's
// chain over two sub-partitions halves the time of a narrow level.  Both warps poll the chunk's
// dependencies (both parts of each value are needed) and publish their own part; a consumer sees
// a value once all its words are published.  Deadlock-free as the single-warp kernel (pairs walk
// their chunks in increasing order, dependencies lie in earlier chunks); a timed-out wait ends
// both warps of the pair after the barrier they share.
__device__ __forceinline__ void pair_barrier(int id) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(64) : "memory");
}
template <int W, int WPB>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_mp_cx(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
                 const int* __restrict__ done) {
  static_assert(WPB % 2 == 0 && WPB / 2 <= 14, "pairs of warps, named barriers 1..14");
  constexpr int CP = 2, NP = WPB / 2;
  constexpr int KG = MpChunk<W, CP, false>::KG;
  __shared__ __align__(16) double xch[2][NP][2][W][32];  // [buffer][pair][part][component][lane]
  __shared__ int xto[2][NP][2];                           // timeout flags, same buffering
  if (is_done(done)) return;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int pair = warp >> 1, part = warp & 1;
  const int G = gridDim.x * NP;
  const int g = pair * gridDim.x + blockIdx.x;
  MpChunk<W, CP, false> c, nx, mm;  // two chunks ahead, as in k_trsv_mp
  if (g < T.nchunks) {
    mp_meta<W, CP, false>(T, g, nx);
    mp_operands<W, CP, false>(T, unit, in, g, nx);
  }
  if (g + G < T.nchunks) mp_meta<W, CP, false>(T, g + G, mm);
  int buf = 0;
  for (int chunk = g; chunk < T.nchunks; chunk += G) {
    c = nx;
    if (chunk + G < T.nchunks) {
      nx.i = mm.i;
      nx.b0 = mm.b0;
      nx.w = mm.w;
      nx.rep = mm.rep;
      mp_operands<W, CP, false>(T, unit, in, chunk + G, nx);
    }
    if (chunk + 2 * G < T.nchunks) mp_meta<W, CP, false>(T, chunk + 2 * G, mm);
    // |f_ii|^2 depends on the factor alone: formed while the dependencies are outstanding, not
    // on the chain after them (the sub-partition's binary64 unit is idle during the wait)
    R<W> den = r_from<W>(1.0);
    if (!unit) den = add<W>(mul_fp<W>(r_from<W>(c.dr), c.dr), mul_fp<W>(r_from<W>(c.di), c.di));
    bool timeout = false;
    const long long t0 = clock64();
    int polls = 0;
    if (lane == 0 && c.rep >= 0 && M.poll == 0) {  // lane 0 first on the latest dependency
      N<W, CP> r;
      while (!n_poll<W, CP>(out, c.rep, r)) {
        if (wait_expired(t0, polls, M.ctl)) { timeout = true; break; }
        wait_pause(t0, 128);
      }
    }
    timeout = __any_sync(FULL, timeout);
    R<W> acc = part == 0 ? c.acc.re : c.acc.im;
    for (int k0 = 0; k0 < c.w && !timeout; k0 += KG) {
      if (k0 > 0) mp_group<W, CP, false>(T, k0, c);
      N<W, CP> v[KG];
      unsigned need = 0u;
#pragma unroll
      for (int k = 0; k < KG; ++k) {
        v[k] = n_zero<W, CP>();
        if (c.jj[k] >= 0) need |= 1u << k;
      }
      while (__any_sync(FULL, need != 0u && !timeout)) {
#pragma unroll
        for (int k = 0; k < KG; ++k)
          if ((need >> k) & 1u) n_fetch<W, CP>(out, c.jj[k], v[k]);
        unsigned got = 0u;
#pragma unroll
        for (int k = 0; k < KG; ++k)
          if (((need >> k) & 1u) && n_ready<W, CP>(v[k])) got |= 1u << k;
        need &= ~got;
        if (need != 0u && !timeout && wait_expired(t0, polls, M.ctl)) timeout = true;
        if (__any_sync(FULL, need != 0u)) {
          if (M.poll == 1) wait_pause(t0, 64);
          else __nanosleep(M.poll == 2 ? (unsigned)M.poll_ns : 64u);
        }
      }
      timeout = __any_sync(FULL, timeout);
      if (!timeout && c.i >= 0) {
#pragma unroll
        for (int k = 0; k < KG; ++k) {
          if (c.jj[k] == -1) continue;
          const R<W> p = part == 0 ? sub<W>(mul_fp<W>(v[k].re, c.fr[k]), mul_fp<W>(v[k].im, c.fi[k]))
                                   : add<W>(mul_fp<W>(v[k].im, c.fr[k]), mul_fp<W>(v[k].re, c.fi[k]));
          acc = sub<W>(acc, p);
        }
      }
    }
    if (!unit) {  // the division needs the partner's part: exchange, then each warp its own part
#pragma unroll
      for (int k = 0; k < W; ++k) xch[buf][pair][part][k][lane] = acc.c[k];
      if (lane == 0) xto[buf][pair][part] = timeout ? 1 : 0;
      pair_barrier(1 + pair);
      timeout = timeout || xto[buf][pair][part ^ 1] != 0;
      if (!timeout && c.i >= 0) {
        R<W> other;
#pragma unroll
        for (int k = 0; k < W; ++k) other.c[k] = xch[buf][pair][part ^ 1][k][lane];
        const R<W> are = part == 0 ? acc : other, aim = part == 0 ? other : acc;
        const R<W> num = part == 0 ? add<W>(mul_fp<W>(are, c.dr), mul_fp<W>(aim, c.di))
                                   : sub<W>(mul_fp<W>(aim, c.dr), mul_fp<W>(are, c.di));
        acc = div<W>(num, den);
      }
      buf ^= 1;
    }
    if (timeout) {
      if (lane == 0) atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
      return;
    }
    if (c.i >= 0 && c.i != M.withhold) {
      double* p = out + (int64_t)c.i * (CP * W) + part * W;
#pragma unroll
      for (int k = 0; k < W; ++k) st_relaxed_f64(p + k, acc.c[k]);
    }
  }
}

// Owner-block schedule (SellTri::ob): block b runs its (block, level) groups in order; the
// block's warps share a group's chunks (chunk goff[g] + k for warp k mod WPB), then meet at a
// block barrier, after which the group's values are in the block's shared-memory ring.  Only
// dependencies on other blocks' rows (or on own rows that left the ring) are polled in global
// memory: on a mesh in natural order with contiguous row blocks those are the rows of the
// neighbouring block, so such levels cost a barrier instead of a cross-SM notification.  A
// warp loads its next chunk's rows before computing the current one and that chunk's operands
// right after (they do not depend on the current values), so no load latency sits between a
// barrier and the arithmetic.  Deadlock-free with all blocks resident (cooperative launch): a
// block waits only for rows of lower levels, and the block with the lowest current level waits
// for nothing unfinished.  A timed-out wait sets MPK_TIMEOUT and a block flag; every warp still
// reaches the barrier, then the block leaves.
template <int W, int CP, int WPB, bool MF>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_mp_ob(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
                 const int* __restrict__ done) {
  if (is_done(done)) return;
  extern __shared__ double ring_mp[];
  __shared__ int abort_blk;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x;
  if (threadIdx.x == 0) abort_blk = 0;
  __syncthreads();
  if (b >= T.nblocks) return;
  RingRef R;
  R.base = ring_mp;
  const int bs = T.bstart[b], gbeg = T.bgrp[b], gend = T.bgrp[b + 1];
  // chunk bounds of the current group and the next one: [cg0, cg1), [cg1, cg2)
  int cg0 = 0, cg1 = 0, cg2 = 0;
  if (gbeg < gend) {
    cg0 = T.goff[gbeg];
    cg1 = T.goff[gbeg + 1];
    cg2 = gbeg + 1 < gend ? T.goff[gbeg + 2] : cg1;
  }
  MpChunk<W, CP, MF> c, nx;
  bool ahead = false;  // c holds the operands of this warp's next chunk
  for (int g = gbeg; g < gend; ++g) {
    const int cg3 = g + 2 < gend ? T.goff[g + 3] : cg2;
    for (int chunk = cg0 + warp; chunk < cg1; chunk += WPB) {
      if (!ahead) {
        mp_meta<W, CP, MF>(T, chunk, c);
        mp_operands<W, CP, MF>(T, unit, in, chunk, c);
      }
      int nxt = chunk + WPB;  // this warp's next chunk: in this group, else its chunk of the next group
      if (nxt >= cg1) nxt = (g + 1 < gend && cg1 + warp < cg2) ? cg1 + warp : -1;
      if (nxt >= 0) mp_meta<W, CP, MF>(T, nxt, nx);
      const int own = ((chunk << 5) + lane - bs) % kRing;
      if (mp_finish<W, CP, MF, true>(T, M, unit, out, c, R, own)) {
        if (lane == 0) {
          atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
          abort_blk = 1;
        }
        ahead = false;
        break;
      }
      ahead = nxt >= 0;
      if (ahead) {
        mp_operands<W, CP, MF>(T, unit, in, nxt, nx);
        c = nx;
      }
    }
    __syncthreads();
    if (abort_blk) return;
    cg0 = cg1;
    cg1 = cg2;
    cg2 = cg3;
  }
}

// Owner-block schedule per thread-block cluster of CS CTAs (one per SM): cluster b runs its
// groups in order; chunk m of a group goes to CTA m mod CS, warp (m / CS) mod WPB; a CTA keeps
// its values in its own ring, and a dependency computed by another CTA of the cluster is read
// through distributed shared memory.  Groups are separated by cluster barriers (release /
// acquire).  A timed-out wait sets MPK_TIMEOUT and writes the abort flag of every CTA of the
// cluster before the barrier, so all of them leave after it; no CTA touches another's shared
// memory after the last barrier it passes.
template <int W, int CP, int WPB, bool MF, int CS>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_mp_cl(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
                 const int* __restrict__ done) {
  if (is_done(done)) return;  // the same for every CTA: no barrier is left waiting
  extern __shared__ double ring_mc[];
  __shared__ int abort_blk;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RingRef R;
  R.base = ring_mc;
  R.sa = (unsigned)__cvta_generic_to_shared(ring_mc);
  R.rank = cta_rank_in_cluster();
  const int b = (int)cluster_index();
  if (threadIdx.x == 0) abort_blk = 0;
  cluster_barrier();  // every CTA's flag is set before any CTA may write it
  if (b >= T.nblocks) return;  // the whole cluster
  const unsigned abort_sa = (unsigned)__cvta_generic_to_shared(&abort_blk);
  const int bs = T.bstart[b], gbeg = T.bgrp[b], gend = T.bgrp[b + 1];
  int cg0 = 0, cg1 = 0, cg2 = 0;
  if (gbeg < gend) {
    cg0 = T.goff[gbeg];
    cg1 = T.goff[gbeg + 1];
    cg2 = gbeg + 1 < gend ? T.goff[gbeg + 2] : cg1;
  }
  const int first = (int)R.rank + CS * warp, stride = CS * WPB;
  MpChunk<W, CP, MF> c, nx;
  bool ahead = false;
  for (int g = gbeg; g < gend; ++g) {
    const int cg3 = g + 2 < gend ? T.goff[g + 3] : cg2;
    for (int chunk = cg0 + first; chunk < cg1; chunk += stride) {
      if (!ahead) {
        mp_meta<W, CP, MF>(T, chunk, c);
        mp_operands<W, CP, MF>(T, unit, in, chunk, c);
      }
      int nxt = chunk + stride;
      if (nxt >= cg1) nxt = (g + 1 < gend && cg1 + first < cg2) ? cg1 + first : -1;
      if (nxt >= 0) mp_meta<W, CP, MF>(T, nxt, nx);
      const int own = ((chunk << 5) + lane - bs) % kRing;
      if (mp_finish<W, CP, MF, true>(T, M, unit, out, c, R, own)) {
        if (lane == 0) {
          atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
          for (int r = 0; r < CS; ++r) st_cluster_s32(cluster_addr(abort_sa, (unsigned)r), 1);
        }
        ahead = false;
        break;
      }
      ahead = nxt >= 0;
      if (ahead) {
        mp_operands<W, CP, MF>(T, unit, in, nxt, nx);
        c = nx;
      }
    }
    cluster_barrier();
    if (abort_blk) return;
    cg0 = cg1;
    cg1 = cg2;
    cg2 = cg3;
  }
}

// Binary32 / bfloat16 factor (substitutions in binary32): the same static balanced schedule and
// value-carried completion as k_trsv_mp, with binary32 values and the sentinel kSent32.  Row i:
//   lower: a = fl32(2^-e in_i) (leading components), a -= f_ij v_j (fmaf, CSR order), v_i = a;
//   upper: a = lower result of row i, a -= f_ij v_j, a /= f_ii, v_i = a, out_i = 2^e v_i,
// e = frexp exponent of the largest leading component of the right-hand side (of the row's
// system in a batch): the scaling keeps residuals far below binary32's range representable.
// Complex steps: a -= l*v as re = fmaf(-lr, vr, re), re = fmaf(li, vi, re), im = fmaf(-lr, vi, im),
// im = fmaf(-li, vr, im); a / d as den = fmaf(dr, dr, di*di), (fmaf(ar, dr, ai*di), fmaf(ai, dr,
// -(ar*di))) / den.  Lower results go to M.v32, upper results to M.pk read as binary32.
constexpr unsigned kSent32 = 0xFFFFFFFFu;
__device__ __forceinline__ float ld_relaxed_f32(const float* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return __uint_as_float(v);
}
__device__ __forceinline__ void st_relaxed_f32(float* p, float x) {
  unsigned v = __float_as_uint(x);
  if (v == kSent32) v = 0x7FC00000u;  // never publish the sentinel
  asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// A complex binary32 value (real, imaginary) as one 8-byte strong access where it is 8-byte
// aligned (the handle's own buffers always are); each half is still checked on its own.
__device__ __forceinline__ bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }
__device__ __forceinline__ void ld_relaxed_f32x2(const float* p, float& a, float& b) {
  unsigned x, y;
  if (aligned8(p)) {
    asm volatile("ld.relaxed.gpu.global.v2.b32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "l"(p) : "memory");
    a = __uint_as_float(x);
    b = __uint_as_float(y);
  } else {
    a = ld_relaxed_f32(p);
    b = ld_relaxed_f32(p + 1);
  }
}
__device__ __forceinline__ void st_relaxed_f32x2(float* p, float a, float b) {
  if (!aligned8(p)) {
    st_relaxed_f32(p, a);
    st_relaxed_f32(p + 1, b);
    return;
  }
  unsigned x = __float_as_uint(a), y = __float_as_uint(b);
  if (x == kSent32) x = 0x7FC00000u;  // never publish the sentinel
  if (y == kSent32) y = 0x7FC00000u;
  asm volatile("st.relaxed.gpu.global.v2.b32 [%0], {%1, %2};" ::"l"(p), "r"(x), "r"(y) : "memory");
}
static __global__ void __launch_bounds__(kBlock) k_fill_sent32(int64_t m, float* __restrict__ a,
                                                              const int* __restrict__ done) {
  if (is_done(done)) return;
  const float s = __uint_as_float(kSent32);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) a[k] = s;
}
template <int CP>
__device__ __forceinline__ bool f_poll(const float* __restrict__ v, int j, float& xr, float& xi) {
  if constexpr (CP == 2) {
    ld_relaxed_f32x2(v + (int64_t)j * CP, xr, xi);
  } else {
    xr = ld_relaxed_f32(v + (int64_t)j);
    xi = 0.0f;
  }
  return __float_as_uint(xr) != kSent32 && (CP == 1 || __float_as_uint(xi) != kSent32);
}

// One chunk of the binary32 substitution, shared by both schedules, in the three steps of the
// binary64 one (lp_meta, lp_operands, lp_finish; ring: see mp_finish).  e1: the scale exponent
// of a single system (a batch reads each row's system's).
template <typename TS>
struct LpChunk {
  static constexpr int KG = 8;  // entries per group
  int i, b0, w, rep, e;
  int jj[KG];
  float fr[KG], fi[KG];
  float ar, ai, dr, di;
};
template <typename TS>
__device__ __forceinline__ void lp_meta(const SellTri& T, int chunk, LpChunk<TS>& c) {
  const int lane = threadIdx.x & 31;
  c.i = T.perm[(chunk << 5) + lane];
  c.b0 = T.coff[chunk];
  c.w = T.coff[chunk + 1] - c.b0;
  c.rep = T.rep[chunk];
}
template <int CP, typename TS>
__device__ __forceinline__ void lp_group(const SellTri& T, int k0, LpChunk<TS>& c) {
  const TS* __restrict__ tval = (const TS*)T.val;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < LpChunk<TS>::KG; ++k) {
    c.jj[k] = -1;
    c.fr[k] = 0.0f;
    c.fi[k] = 0.0f;
    if (k0 + k < c.w) {
      const int64_t s = ((int64_t)(c.b0 + k0 + k) << 5) + lane;
      c.jj[k] = T.col[s];
      if constexpr (CP == 1) c.fr[k] = ld_fac(tval, s);
      else { c.fr[k] = ld_fac(tval, 2 * s); c.fi[k] = ld_fac(tval, 2 * s + 1); }
    }
  }
}
template <int W, int CP, typename TS>
__device__ __forceinline__ void lp_operands(const SellTri& T, const IluHandleView& M, bool lower, bool unit,
                                            const double* __restrict__ in, int chunk, int e1, LpChunk<TS>& c) {
  const TS* __restrict__ tdia = (const TS*)T.dia;
  const int lane = threadIdx.x & 31;
  lp_group<CP, TS>(T, 0, c);
  c.ar = 0.0f;
  c.ai = 0.0f;
  c.dr = 1.0f;
  c.di = 0.0f;
  c.e = (M.sysid != nullptr && c.i >= 0) ? scale_exponent(M.absmax + M.sysid[c.i]) : e1;
  if (c.i >= 0) {
    if (lower) {
      const double* q = in + (int64_t)c.i * CP * W;
      c.ar = __double2float_rn(ldexp(q[0], -c.e));
      c.ai = CP == 2 ? __double2float_rn(ldexp(q[W], -c.e)) : 0.0f;
    } else {
      c.ar = M.v32[(int64_t)c.i * CP];
      c.ai = CP == 2 ? M.v32[(int64_t)c.i * CP + 1] : 0.0f;
    }
    if (!unit) {
      const int64_t q = ((int64_t)chunk << 5) + lane;
      if constexpr (CP == 1) c.dr = ld_fac(tdia, q);
      else { c.dr = ld_fac(tdia, 2 * q); c.di = ld_fac(tdia, 2 * q + 1); }
    }
  }
}
template <int W, int CP, typename TS, bool RING>
__device__ __forceinline__ bool lp_finish(const SellTri& T, const IluHandleView& M, bool lower, bool unit,
                                          double* __restrict__ out, LpChunk<TS>& c, const RingRef& R,
                                          int own_slot) {
  constexpr int KG = LpChunk<TS>::KG;
  const unsigned FULL = 0xffffffffu;
  float* __restrict__ mine = lower ? M.v32 : reinterpret_cast<float*>(M.pk);
  const int lane = threadIdx.x & 31;
  bool timeout = false;
  const long long t0 = clock64();
  int polls = 0;
  if (lane == 0 && c.rep >= 0 && M.poll == 0) {  // the chunk's latest dependency, polled by one lane
    float xr, xi;
    while (!f_poll<CP>(mine, c.rep, xr, xi)) {
      if (wait_expired(t0, polls, M.ctl)) { timeout = true; break; }
      wait_pause(t0, 128);
    }
  }
  __syncwarp();
  float ar = c.ar, ai = c.ai;
  for (int k0 = 0; k0 < c.w; k0 += KG) {
    if (k0 > 0) lp_group<CP, TS>(T, k0, c);
    float vr[KG], vi[KG];
    unsigned need = 0u;
#pragma unroll
    for (int k = 0; k < KG; ++k) {
      vr[k] = 0.0f;
      vi[k] = 0.0f;
      if (c.jj[k] >= 0) {
        need |= 1u << k;
      } else if (RING && c.jj[k] <= -2) {  // computed by this block
        ring_read32<CP>(R, -2 - c.jj[k], vr[k], vi[k]);
      }
    }
    while (__any_sync(FULL, need != 0u && !timeout)) {
#pragma unroll
      for (int k = 0; k < KG; ++k)
        if ((need >> k) & 1u) {
          if constexpr (CP == 2) ld_relaxed_f32x2(mine + (int64_t)c.jj[k] * CP, vr[k], vi[k]);
          else vr[k] = ld_relaxed_f32(mine + (int64_t)c.jj[k]);
        }
      unsigned got = 0u;
#pragma unroll
      for (int k = 0; k < KG; ++k)
        if (((need >> k) & 1u) && __float_as_uint(vr[k]) != kSent32 &&
            (CP == 1 || __float_as_uint(vi[k]) != kSent32))
          got |= 1u << k;
      need &= ~got;
      if (need != 0u && !timeout && wait_expired(t0, polls, M.ctl)) timeout = true;
      if (__any_sync(FULL, need != 0u)) {
        if (M.poll == 1) wait_pause(t0, 64);
        else __nanosleep(M.poll == 2 ? (unsigned)M.poll_ns : 64u);
      }
    }
    __syncwarp();
    if (!timeout && c.i >= 0) {
#pragma unroll
      for (int k = 0; k < KG; ++k) {
        if (c.jj[k] == -1) continue;
        if constexpr (CP == 1) {
          ar = fmaf(-c.fr[k], vr[k], ar);
        } else {
          ar = fmaf(-c.fr[k], vr[k], ar);
          ar = fmaf(c.fi[k], vi[k], ar);
          ai = fmaf(-c.fr[k], vi[k], ai);
          ai = fmaf(-c.fi[k], vr[k], ai);
        }
      }
    }
  }
  if (!timeout && c.i >= 0 && c.i != M.withhold) {
    if (!unit) {
      if constexpr (CP == 1) {
        ar = ar / c.dr;
      } else {
        const float den = fmaf(c.dr, c.dr, c.di * c.di), nr = fmaf(ar, c.dr, ai * c.di);
        const float ni = fmaf(ai, c.dr, -(ar * c.di));
        ar = nr / den;
        ai = ni / den;
      }
    }
    if constexpr (CP == 2) st_relaxed_f32x2(mine + (int64_t)c.i * CP, ar, ai);
    else st_relaxed_f32(mine + (int64_t)c.i, ar);
    if constexpr (RING) {
      float* ring = (float*)R.base;
      ring[own_slot * CP] = ar;
      if constexpr (CP == 2) ring[own_slot * CP + 1] = ai;
    }
    if (!lower) {
      N<W, CP> z = n_zero<W, CP>();
      z.re.c[0] = ldexp((double)ar, c.e);
      if constexpr (CP == 2) z.im.c[0] = ldexp((double)ai, c.e);
      n_store<W, CP>(out, c.i, z);
    }
  }
  return __any_sync(FULL, timeout);
}

template <int W, int CP, typename TS, int WPB>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_lp(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
              const int* __restrict__ done) {
  if (is_done(done)) return;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const int e1 = M.sysid == nullptr ? scale_exponent(M.absmax) : 0;  // one system: one scale
  const int lane = threadIdx.x & 31;
  const int G = gridDim.x * (blockDim.x >> 5);
  const int g = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
  // Two chunks ahead below 32 warps per SM, as in k_trsv_mp: the operands read here (the
  // right-hand side, or the lower pass's binary32 output, and the factor) are not written by
  // this launch.
  constexpr bool AHEAD = WPB < 32;
  LpChunk<TS> c, nx, mm;
  if (g < T.nchunks) {
    lp_meta<TS>(T, g, nx);
    if constexpr (AHEAD) lp_operands<W, CP, TS>(T, M, lower, unit, in, g, e1, nx);
  }
  if (AHEAD && g + G < T.nchunks) lp_meta<TS>(T, g + G, mm);
  for (int chunk = g; chunk < T.nchunks; chunk += G) {
    if constexpr (AHEAD) {
      c = nx;
      if (chunk + G < T.nchunks) {
        nx.i = mm.i;
        nx.b0 = mm.b0;
        nx.w = mm.w;
        nx.rep = mm.rep;
        lp_operands<W, CP, TS>(T, M, lower, unit, in, chunk + G, e1, nx);
      }
      if (chunk + 2 * G < T.nchunks) lp_meta<TS>(T, chunk + 2 * G, mm);
    } else {
      c.i = nx.i;
      c.b0 = nx.b0;
      c.w = nx.w;
      c.rep = nx.rep;
      lp_operands<W, CP, TS>(T, M, lower, unit, in, chunk, e1, c);
      if (chunk + G < T.nchunks) lp_meta<TS>(T, chunk + G, nx);
    }
    if (lp_finish<W, CP, TS, false>(T, M, lower, unit, out, c, RingRef(), 0)) {
      if (lane == 0) atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
      return;
    }
  }
}

// Owner-block schedule of the binary32 substitution (see k_trsv_mp_ob).
template <int W, int CP, typename TS, int WPB>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_lp_ob(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
                 const int* __restrict__ done) {
  if (is_done(done)) return;
  extern __shared__ float ring_lp[];
  __shared__ int abort_blk;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const int e1 = M.sysid == nullptr ? scale_exponent(M.absmax) : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int b = blockIdx.x;
  if (threadIdx.x == 0) abort_blk = 0;
  __syncthreads();
  if (b >= T.nblocks) return;
  RingRef R;
  R.base = ring_lp;
  const int bs = T.bstart[b], gbeg = T.bgrp[b], gend = T.bgrp[b + 1];
  int cg0 = 0, cg1 = 0, cg2 = 0;
  if (gbeg < gend) {
    cg0 = T.goff[gbeg];
    cg1 = T.goff[gbeg + 1];
    cg2 = gbeg + 1 < gend ? T.goff[gbeg + 2] : cg1;
  }
  LpChunk<TS> c, nx;
  bool ahead = false;
  for (int g = gbeg; g < gend; ++g) {
    const int cg3 = g + 2 < gend ? T.goff[g + 3] : cg2;
    for (int chunk = cg0 + warp; chunk < cg1; chunk += WPB) {
      if (!ahead) {
        lp_meta<TS>(T, chunk, c);
        lp_operands<W, CP, TS>(T, M, lower, unit, in, chunk, e1, c);
      }
      int nxt = chunk + WPB;
      if (nxt >= cg1) nxt = (g + 1 < gend && cg1 + warp < cg2) ? cg1 + warp : -1;
      if (nxt >= 0) lp_meta<TS>(T, nxt, nx);
      const int own = ((chunk << 5) + lane - bs) % kRing;
      if (lp_finish<W, CP, TS, true>(T, M, lower, unit, out, c, R, own)) {
        if (lane == 0) {
          atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
          abort_blk = 1;
        }
        ahead = false;
        break;
      }
      ahead = nxt >= 0;
      if (ahead) {
        lp_operands<W, CP, TS>(T, M, lower, unit, in, nxt, e1, nx);
        c = nx;
      }
    }
    __syncthreads();
    if (abort_blk) return;
    cg0 = cg1;
    cg1 = cg2;
    cg2 = cg3;
  }
}

// Owner-block schedule per cluster of the binary32 substitution (see k_trsv_mp_cl).
template <int W, int CP, typename TS, int WPB, int CS>
__global__ void __launch_bounds__(WPB * 32, 1)
    k_trsv_lp_cl(IluHandleView M, bool lower, bool unit, const double* __restrict__ in, double* __restrict__ out,
                 const int* __restrict__ done) {
  if (is_done(done)) return;
  extern __shared__ float ring_lc[];
  __shared__ int abort_blk;
  const SellTri T = lower ? M.sl_lo : M.sl_up;
  const int e1 = M.sysid == nullptr ? scale_exponent(M.absmax) : 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  RingRef R;
  R.base = ring_lc;
  R.sa = (unsigned)__cvta_generic_to_shared(ring_lc);
  R.rank = cta_rank_in_cluster();
  const int b = (int)cluster_index();
  if (threadIdx.x == 0) abort_blk = 0;
  cluster_barrier();
  if (b >= T.nblocks) return;
  const unsigned abort_sa = (unsigned)__cvta_generic_to_shared(&abort_blk);
  const int bs = T.bstart[b], gbeg = T.bgrp[b], gend = T.bgrp[b + 1];
  int cg0 = 0, cg1 = 0, cg2 = 0;
  if (gbeg < gend) {
    cg0 = T.goff[gbeg];
    cg1 = T.goff[gbeg + 1];
    cg2 = gbeg + 1 < gend ? T.goff[gbeg + 2] : cg1;
  }
  const int first = (int)R.rank + CS * warp, stride = CS * WPB;
  LpChunk<TS> c, nx;
  bool ahead = false;
  for (int g = gbeg; g < gend; ++g) {
    const int cg3 = g + 2 < gend ? T.goff[g + 3] : cg2;
    for (int chunk = cg0 + first; chunk < cg1; chunk += stride) {
      if (!ahead) {
        lp_meta<TS>(T, chunk, c);
        lp_operands<W, CP, TS>(T, M, lower, unit, in, chunk, e1, c);
      }
      int nxt = chunk + stride;
      if (nxt >= cg1) nxt = (g + 1 < gend && cg1 + first < cg2) ? cg1 + first : -1;
      if (nxt >= 0) lp_meta<TS>(T, nxt, nx);
      const int own = ((chunk << 5) + lane - bs) % kRing;
      if (lp_finish<W, CP, TS, true>(T, M, lower, unit, out, c, R, own)) {
        if (lane == 0) {
          atomicCAS(M.ctl + CTL_ERR, 0, (int)MPK_TIMEOUT);
          for (int r = 0; r < CS; ++r) st_cluster_s32(cluster_addr(abort_sa, (unsigned)r), 1);
        }
        ahead = false;
        break;
      }
      ahead = nxt >= 0;
      if (ahead) {
        lp_operands<W, CP, TS>(T, M, lower, unit, in, nxt, e1, nx);
        c = nx;
      }
    }
    cluster_barrier();
    if (abort_blk) return;
    cg0 = cg1;
    cg1 = cg2;
    cg2 = cg3;
  }
}

// ---------------------------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------------------------
inline int grid_for(int n) {
  int g = (n + kBlock - 1) / kBlock;
  const int cap = sm_count() * 8;
  return g < 1 ? 1 : (g > cap ? cap : g);
}
// Blocks of the dependency-driven kernels: at most `resident_warps_per_sm()` warps per SM (fewer
// waiting warps poll less), capped by occupancy.
template <class KernelT>
inline int persistent_blocks(KernelT kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  int want = resident_warps_per_sm() / (kBlock / 32);
  if (want < 1) want = 1;
  if (want < per_sm) per_sm = want;
  return per_sm * sm_count();
}

template <int W, int CP>
struct Launch {
  static void spmv(const Csr& A, const double* x, double* y, const double* b, const int* done, const Batch* bt,
                   cudaStream_t s) {
    count_launch();
    auto fn = A.mm ? k_spmv<W, CP, true> : k_spmv<W, CP, false>;
    fn<<<(A.n + kBlock - 1) / kBlock, kBlock, 0, s>>>(A.n, A.rp, A.ci, A.val, x, y, b, done, bt ? bt->sysid : nullptr,
                                                       bt ? bt->st : nullptr, A.order, bt ? bt->gate : -1);
  }
  template <int K>
  static void dotsK(int n, const double* const* a, const double* const* b, double* const* out, const DotWs& ws,
                    const int* done, cudaStream_t s) {
    DotArgs<K> args;
    for (int k = 0; k < K; ++k) {
      args.a[k] = a[k];
      args.b[k] = b[k];
      args.out[k] = out[k];
    }
    count_launch();
    k_dots<W, CP, K><<<dot_blocks(n), kBlock, 0, s>>>(n, args, ws.partial, ws.counter, done);
  }
  static void dots(int n, int k, const double* const* a, const double* const* b, double* const* out, const DotWs& ws,
                   const int* done, cudaStream_t s) {
    if (k == 1) dotsK<1>(n, a, b, out, ws, done, s);
    else if (k == 2) dotsK<2>(n, a, b, out, ws, done, s);
    else dotsK<6>(n, a, b, out, ws, done, s);
  }
  template <int K>
  static void dotsSegK(const Batch& bt, const double* const* a, const double* const* b, double* S, int slot0,
                       double* partial, unsigned* counters, const int* done, cudaStream_t s) {
    DotArgs<K> args;
    for (int k = 0; k < K; ++k) {
      args.a[k] = a[k];
      args.b[k] = b[k];
      args.out[k] = nullptr;
    }
    count_launch();
    k_dots_seg<W, CP, K><<<bt.nblocks, kBlock, 0, s>>>(bt, args, S, slot0, partial, counters, done);
  }
  static void dots_seg(const Batch& bt, int k, const double* const* a, const double* const* b, double* S, int slot0,
                       double* partial, unsigned* counters, const int* done, cudaStream_t s) {
    if (k == 1) dotsSegK<1>(bt, a, b, S, slot0, partial, counters, done, s);
    else if (k == 2) dotsSegK<2>(bt, a, b, S, slot0, partial, counters, done, s);
    else dotsSegK<6>(bt, a, b, S, slot0, partial, counters, done, s);
  }
  static void lincomb(int n, double* y, int nt, const double* const* coef, const double* const* v,
                      const int* copy_at_first, const int* done, const Batch* bt, cudaStream_t s) {
    LinArgs a;
    a.y = y;
    a.nt = nt;
    a.copy_at_first = copy_at_first;
    for (int k = 0; k < 3; ++k) {
      a.v[k] = k < nt ? v[k] : nullptr;
      a.s[k] = k < nt ? coef[k] : nullptr;
    }
    count_launch();
    k_lincomb<W, CP><<<grid_for(n), kBlock, 0, s>>>(n, a, done, bt ? bt->sysid : nullptr, bt ? bt->st : nullptr,
                                                     bt ? bt->gate : -1);
  }
  static void nested(int n, double* y, const double* v0, const double* v1, const double* v2, const double* s1,
                     const double* s2, const int* copy_at_first, const int* done, const Batch* bt, cudaStream_t s) {
    count_launch();
    k_nested<W, CP><<<grid_for(n), kBlock, 0, s>>>(n, y, v0, v1, v2, s1, s2, copy_at_first, done,
                                                    bt ? bt->sysid : nullptr, bt ? bt->st : nullptr);
  }
  static void copy(int n, double* y, const double* x, const int* done, cudaStream_t s) {
    count_launch();
    k_copy<W, CP><<<grid_for(n), kBlock, 0, s>>>(n, y, x, done);
  }
  static void scalar(int method, int phase, double* S, int* st, double* hist, const int* done, int nsys,
                     int hist_stride, int* fin, int* alldone, cudaStream_t s) {
    count_launch();
    k_scalar<W, CP><<<(nsys + 63) / 64, 64, 0, s>>>(method, phase, S, st, hist, done, nsys, hist_stride, fin, alldone);
  }
  static void absmax(int n, const double* v, unsigned long long* out, const int* done, const Batch* bt,
                     cudaStream_t s) {
    count_launch();
    k_absmax<W, CP><<<grid_for(n), kBlock, 0, s>>>(n, v, out, done, bt ? bt->sysid : nullptr);
  }
  // Launch of a substitution kernel with wpb warps per block, all blocks co-resident (cooperative
  // launch): one block per SM, or (cluster schedules) nblocks clusters of csize CTAs, one CTA per
  // SM; smem: dynamic shared memory (the owner-block ring)
  static int coop(const void* fn, int wpb, size_t smem, int sched, int nblocks, const IluHandleView& M, bool lower,
                  bool unit, const double* in, double* out, const int* done, cudaStream_t s) {
    void* args[] = {(void*)&M, (void*)&lower, (void*)&unit, (void*)&in, (void*)&out, (void*)&done};
    count_launch();
    if (sched < 2) {
      const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(sm_count()), dim3(wpb * 32), args, smem, s);
      return e == cudaSuccess ? MPK_OK : MPK_CUDA_ERROR;
    }
    const int cs = sched_csize(sched);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.gridDim = dim3(nblocks * cs);
    cfg.blockDim = dim3(wpb * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    const cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    return e == cudaSuccess ? MPK_OK : MPK_CUDA_ERROR;
  }
  static size_t ring_bytes(int prec) {  // the owner-block kernels' shared-memory ring
    return (size_t)kRing * CP * ((prec == MPK_ILU_FP64 || prec == MPK_ILU_MP) ? W * sizeof(double) : sizeof(float));
  }
  template <bool MF, int S>
  static const void* mp_fn_t(int wpb) {
    if constexpr (S == 2 || S == 3) {
      constexpr int C = S == 2 ? 8 : 16;
      return wpb == 8 ? (const void*)k_trsv_mp_cl<W, CP, 8, MF, C> : (const void*)k_trsv_mp_cl<W, CP, 4, MF, C>;
    } else if constexpr (S == 1) {
      switch (wpb) {
        case 8: return (const void*)k_trsv_mp_ob<W, CP, 8, MF>;
        case 16: return (const void*)k_trsv_mp_ob<W, CP, 16, MF>;
        case 32: return (const void*)k_trsv_mp_ob<W, CP, 32, MF>;
        default: return (const void*)k_trsv_mp_ob<W, CP, 4, MF>;
      }
    } else {
      if constexpr (CP == 2 && !MF) {  // complex, binary64 factor: a pair of warps per chunk
        switch (wpb) {
          case 8: return (const void*)k_trsv_mp_cx<W, 8>;
          case 16: return (const void*)k_trsv_mp_cx<W, 16>;
          case 32: return (const void*)k_trsv_mp<W, CP, 32, MF>;
          default: return (const void*)k_trsv_mp_cx<W, 4>;
        }
      }
      switch (wpb) {
        case 8: return (const void*)k_trsv_mp<W, CP, 8, MF>;
        case 16: return (const void*)k_trsv_mp<W, CP, 16, MF>;
        case 32: return (const void*)k_trsv_mp<W, CP, 32, MF>;
        default: return (const void*)k_trsv_mp<W, CP, 4, MF>;
      }
    }
  }
  template <typename TS, int S>
  static const void* lp_fn_t(int wpb) {
    if constexpr (S == 2 || S == 3) {
      constexpr int C = S == 2 ? 8 : 16;
      return wpb == 8 ? (const void*)k_trsv_lp_cl<W, CP, TS, 8, C> : (const void*)k_trsv_lp_cl<W, CP, TS, 4, C>;
    } else if constexpr (S == 1) {
      switch (wpb) {
        case 8: return (const void*)k_trsv_lp_ob<W, CP, TS, 8>;
        case 16: return (const void*)k_trsv_lp_ob<W, CP, TS, 16>;
        case 32: return (const void*)k_trsv_lp_ob<W, CP, TS, 32>;
        default: return (const void*)k_trsv_lp_ob<W, CP, TS, 4>;
      }
    } else {
      switch (wpb) {
        case 8: return (const void*)k_trsv_lp<W, CP, TS, 8>;
        case 16: return (const void*)k_trsv_lp<W, CP, TS, 16>;
        case 32: return (const void*)k_trsv_lp<W, CP, TS, 32>;
        default: return (const void*)k_trsv_lp<W, CP, TS, 4>;
      }
    }
  }
  template <int S>
  static const void* trsv_fn_s(int prec, int wpb) {
    if (prec == MPK_ILU_FP64) return mp_fn_t<false, S>(wpb);
    if (prec == MPK_ILU_MP) return mp_fn_t<true, S>(wpb);
    if (prec == MPK_ILU_BF16) return lp_fn_t<uint16_t, S>(wpb);
    return lp_fn_t<float, S>(wpb);
  }
  // the substitution kernel of a factor precision, schedule and block size (cluster schedules:
  // 4 or 8 warps; launch_wpb gives the block size to launch with)
  static int launch_wpb(int sched, int wpb) { return sched >= 2 ? (wpb == 8 ? 8 : 4) : wpb; }
  static const void* trsv_fn(int prec, int sched, int wpb) {
    switch (sched) {
      case 1: return trsv_fn_s<1>(prec, wpb);
      case 2: return trsv_fn_s<2>(prec, wpb);
      case 3: return trsv_fn_s<3>(prec, wpb);
      default: return trsv_fn_s<0>(prec, wpb);
    }
  }
  // dynamic shared memory of a schedule's kernel; above the default 48 KB the kernel opts in,
  // once (the first call comes from the tuner, outside any graph capture)
  static size_t prepare_fn(const void* fn, int prec, int sched) {
    if (sched == 0) return 0;
    size_t rb = ring_bytes(prec);
    if (sched >= 2 && rb < (size_t)kClusterSmem) rb = kClusterSmem;  // one CTA per SM
    if (rb > 48 * 1024 || sched == 3) {
      static std::mutex mu;
      static const void* seen[128];
      static int nseen = 0;
      std::lock_guard<std::mutex> lk(mu);
      bool found = false;
      for (int k = 0; k < nseen; ++k) found = found || seen[k] == fn;
      if (!found) {
        if (rb > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rb);
        if (sched == 3) cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (nseen < 128) seen[nseen++] = fn;
      }
    }
    return rb;
  }
  static int trsv_mp(const IluHandleView& M, bool lower, bool unit, const double* in, double* out, const int* done,
                     cudaStream_t s) {
    // out starts as sentinels: completion is read from the values
    count_launch();
    k_fill_sent<<<grid_for(M.n), kBlock, 0, s>>>((int64_t)M.n * CP * W, out, 0, nullptr, done);
    const int wpb = launch_wpb(M.sched, M.wpb);
    const void* fn = trsv_fn(M.prec, M.sched, wpb);
    return coop(fn, wpb, prepare_fn(fn, M.prec, M.sched), M.sched, M.sl_lo.nblocks, M, lower, unit, in, out, done,
                s);
  }
  static int trsv32(const IluHandleView& M, bool lower, bool unit, const double* in, double* out, const int* done,
                    cudaStream_t s) {
    // this pass's binary32 results start as sentinels: completion is read from the values
    count_launch();
    float* mine = lower ? M.v32 : reinterpret_cast<float*>(M.pk);
    k_fill_sent32<<<grid_for(M.n), kBlock, 0, s>>>((int64_t)M.n * CP, mine, done);
    const int wpb = launch_wpb(M.sched, M.wpb);
    const void* fn = trsv_fn(M.prec, M.sched, wpb);
    return coop(fn, wpb, prepare_fn(fn, M.prec, M.sched), M.sched, M.sl_lo.nblocks, M, lower, unit, in, out, done,
                s);
  }
  // 1 if the kernel of (prec, wpb, sched) can run all its blocks co-resident: one block per SM,
  // or (cluster schedules) nblocks clusters
  static int trsv_fits(int prec, int wpb, int sched, int nblocks) {
    wpb = launch_wpb(sched, wpb);
    const void* fn = trsv_fn(prec, sched, wpb);
    const size_t smem = prepare_fn(fn, prec, sched);
    if (sched < 2) {
      int per_sm = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, wpb * 32, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
      }
      return per_sm >= 1 ? 1 : 0;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = sched_csize(sched);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(sched_csize(sched));
    cfg.blockDim = dim3(wpb * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, fn, &cfg) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return (nblocks >= 1 && active >= nblocks) ? 1 : 0;
  }
  static Ops table() {
    Ops o;
    o.w = W;
    o.cp = CP;
    o.spmv = &spmv;
    o.dots = &dots;
    o.dots_seg = &dots_seg;
    o.lincomb = &lincomb;
    o.nested = &nested;
    o.copy = &copy;
    o.scalar = &scalar;
    o.trsv_mp = &trsv_mp;
    o.trsv32 = &trsv32;
    o.absmax = &absmax;
    o.trsv_fits = &trsv_fits;
    return o;
  }
};

}  // namespace mpk
