// capi.cu -- library-wide helpers and the stateless C-ABI entry points (SpMV, inner product,
// elementwise multi-component arithmetic).
#include <atomic>
#include <cstdlib>
#include <string>

#include "internal.h"
#include "mp.cuh"

namespace mpk {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int status, const std::string& msg) {
  g_last_error = msg;
  return status;
}

static std::atomic<unsigned long long> g_launches{0};
void count_launch(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }
void uncount_launch(unsigned long long k) { g_launches.fetch_sub(k, std::memory_order_relaxed); }

int resident_warps_per_sm() {
  static int w = [] {
    const char* e = std::getenv("MPK_RESIDENT_WARPS");
    int v = e ? std::atoi(e) : 0;
    return v > 0 ? v : 32;
  }();
  return w;
}

int sm_count() {
  static int count = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) return 1;
    return v;
  }();
  return count;
}

const Ops* ops_w1(int cp);
const Ops* ops_w2(int cp);
const Ops* ops_w3(int cp);
const Ops* ops_w4(int cp);

const Ops* get_ops(int w, int cp) {
  if (cp != 1 && cp != 2) return nullptr;
  switch (w) {
    case 1: return ops_w1(cp);
    case 2: return ops_w2(cp);
    case 3: return ops_w3(cp);
    case 4: return ops_w4(cp);
    default: return nullptr;
  }
}

}  // namespace mpk

using namespace mpk;

extern "C" int mpk_version(void) { return 100; }

extern "C" const char* mpk_last_error(void) { return g_last_error.c_str(); }

extern "C" uint64_t mpk_kernel_launches(void) { return (uint64_t)g_launches.load(); }

static int spmv_entry(const mpk_csr* A, int w, const double* x_dev, double* y_dev, bool mm, void* stream) {
  if (A == nullptr || x_dev == nullptr || y_dev == nullptr || x_dev == y_dev)
    return fail(MPK_INVALID_ARG, "null or aliased argument");
  if (A->n < 1 || A->nnz < 0 || A->row_ptr == nullptr || (A->nnz > 0 && (A->col_idx == nullptr || A->val == nullptr)))
    return fail(MPK_INVALID_ARG, "invalid CSR descriptor");
  if (A->is_complex != 0 && A->is_complex != 1) return fail(MPK_INVALID_ARG, "is_complex must be 0 or 1");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  if (misaligned(x_dev) || misaligned(y_dev) || (A->is_complex && misaligned(A->val)))
    return fail(MPK_INVALID_ARG, "device vectors (and complex values) must be 16-byte aligned");
  const Ops* o = get_ops(w, A->is_complex ? 2 : 1);
  Csr c{A->n, A->nnz, A->row_ptr, A->col_idx, A->val, A->is_complex};
  c.mm = mm;
  o->spmv(c, x_dev, y_dev, nullptr, nullptr, nullptr, (cudaStream_t)stream);
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}

extern "C" int mpk_spmv_mp(const mpk_csr* A, int w, const double* x_dev, double* y_dev, void* stream) {
  return spmv_entry(A, w, x_dev, y_dev, false, stream);
}

extern "C" int mpk_spmv_mp_matrix(const mpk_csr* A, int w, const double* x_dev, double* y_dev, void* stream) {
  return spmv_entry(A, w, x_dev, y_dev, true, stream);
}

extern "C" int mpk_dot(int n, int is_complex, int w, const double* a_dev, const double* b_dev, double* out_dev,
                       void* stream) {
  if (n < 1 || a_dev == nullptr || b_dev == nullptr || out_dev == nullptr) return fail(MPK_INVALID_ARG, "bad argument");
  if (w < 1 || w > 4 || (is_complex != 0 && is_complex != 1)) return fail(MPK_INVALID_ARG, "bad w / is_complex");
  if (misaligned(a_dev) || misaligned(b_dev) || misaligned(out_dev))
    return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  const Ops* o = get_ops(w, is_complex ? 2 : 1);
  DotWs ws;
  char* buf = nullptr;
  const size_t pb = sizeof(double) * dot_partial_doubles(n);
  MPK_CUDA(cudaMallocAsync((void**)&buf, pb + 64, s));
  ws.partial = (double*)buf;
  ws.counter = (unsigned*)(buf + pb);
  MPK_CUDA(cudaMemsetAsync(ws.counter, 0, sizeof(unsigned), s));
  const double* av[1] = {a_dev};
  const double* bv[1] = {b_dev};
  double* ov[1] = {out_dev};
  o->dots(n, 1, av, bv, ov, ws, nullptr, s);
  MPK_CUDA(cudaGetLastError());
  MPK_CUDA(cudaFreeAsync(buf, s));
  return MPK_OK;
}

// Elementwise real w-component arithmetic (the operations of mp.cuh every kernel uses).
template <int W>
__global__ void k_mp_op(int op, int n, const double* __restrict__ a, const double* __restrict__ b,
                        double* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    R<W> x, y;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      x.c[k] = a[(int64_t)i * W + k];
      y.c[k] = b != nullptr ? b[(int64_t)i * W + k] : 0.0;
    }
    R<W> z;
    switch (op) {
      case MPK_OP_ADD: z = add<W>(x, y); break;
      case MPK_OP_SUB: z = sub<W>(x, y); break;
      case MPK_OP_MUL: z = mul<W>(x, y); break;
      case MPK_OP_MUL_FP: z = mul_fp<W>(x, y.c[0]); break;
      case MPK_OP_DIV: z = div<W>(x, y); break;
      case MPK_OP_DIV_FP: z = div_fp<W>(x, y.c[0]); break;
      default: z = rsqrt_mp<W>(x); break;
    }
#pragma unroll
    for (int k = 0; k < W; ++k) out[(int64_t)i * W + k] = z.c[k];
  }
}

extern "C" int mpk_mp_op(int op, int w, int n, const double* a_dev, const double* b_dev, double* out_dev,
                         void* stream) {
  if (op < MPK_OP_ADD || op > MPK_OP_SQRT) return fail(MPK_INVALID_ARG, "unknown operation");
  if (w < 1 || w > 4) return fail(MPK_INVALID_ARG, "w must be 1..4");
  if (n < 0 || a_dev == nullptr || out_dev == nullptr || (b_dev == nullptr && op != MPK_OP_SQRT))
    return fail(MPK_INVALID_ARG, "bad argument");
  if (misaligned(a_dev) || (b_dev != nullptr && misaligned(b_dev)) || misaligned(out_dev))
    return fail(MPK_INVALID_ARG, "device vectors must be 16-byte aligned");
  if (n == 0) return MPK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int g = (n + 255) / 256;
  if (g > 4096) g = 4096;
  count_launch();
  switch (w) {
    case 1: k_mp_op<1><<<g, 256, 0, s>>>(op, n, a_dev, b_dev, out_dev); break;
    case 2: k_mp_op<2><<<g, 256, 0, s>>>(op, n, a_dev, b_dev, out_dev); break;
    case 3: k_mp_op<3><<<g, 256, 0, s>>>(op, n, a_dev, b_dev, out_dev); break;
    default: k_mp_op<4><<<g, 256, 0, s>>>(op, n, a_dev, b_dev, out_dev); break;
  }
  MPK_CUDA(cudaGetLastError());
  return MPK_OK;
}

// Cross-SM notification latency: block 0 and block `partner` of a cooperative grid of partner + 1
// blocks (each asks for more than half an SM's shared memory, so every block sits on its own SM)
// pass a counter back and forth through one word of global memory with the strong relaxed loads
// and stores the dependency-driven kernels use; the other blocks leave at once.  Block 0 times
// `rounds` round trips with the global timer.  Every wait is bounded (kProbeSpin polls); a wait
// that runs out records the failure and both blocks leave.
constexpr long long kProbeSpin = 1ll << 20;  // about a second of polls
__global__ void k_probe_hop(int rounds, int partner, int* __restrict__ word, unsigned long long* __restrict__ res) {
  if (threadIdx.x != 0) return;
  if (blockIdx.x != 0 && (int)blockIdx.x != partner) return;
  const int me = blockIdx.x == 0 ? 0 : 1;
  unsigned long long t0 = 0, t1 = 0;
  if (me == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  bool ok = true;
  for (int r = 0; r < rounds && ok; ++r) {
    const int want = 2 * r + me;  // block 0 waits for even values, the partner for odd ones
    long long spins = 0;
    int v;
    do {
      asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(word) : "memory");
      if (++spins > kProbeSpin) {
        ok = false;
        break;
      }
    } while (v != want);
    if (!ok) break;
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(word), "r"(want + 1) : "memory");
  }
  unsigned sm;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(sm));
  res[2 + me] = sm;
  if (me == 0) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    res[0] = t1 - t0;
    res[1] = ok ? 1ull : 0ull;
  }
  if (!ok) atomicExch(word, -1);  // release the other block's wait
}

extern "C" int mpk_probe_notify_ns(int rounds, int partner, double* one_way_ns, int* sm_pair, void* stream) {
  if (rounds < 1 || rounds > 1000000 || one_way_ns == nullptr) return fail(MPK_INVALID_ARG, "bad argument");
  if (partner < 1 || partner >= sm_count()) return fail(MPK_INVALID_ARG, "partner must be 1 .. SMs - 1");
  cudaStream_t s = (cudaStream_t)stream;
  char* buf = nullptr;
  MPK_CUDA(cudaMallocAsync((void**)&buf, 64, s));
  int* word = (int*)buf;  // res: elapsed ns, ok, the two blocks' SM ids
  unsigned long long* res = (unsigned long long*)(buf + 16);
  MPK_CUDA(cudaMemsetAsync(buf, 0, 64, s));
  void* args[] = {(void*)&rounds, (void*)&partner, (void*)&word, (void*)&res};
  constexpr int kSmem = 160 * 1024;  // more than half of an SM: one block per SM
  MPK_CUDA(cudaFuncSetAttribute((const void*)k_probe_hop, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem));
  count_launch();
  MPK_CUDA(cudaLaunchCooperativeKernel((const void*)k_probe_hop, dim3(partner + 1), dim3(32), args, kSmem, s));
  unsigned long long h[4] = {0, 0, 0, 0};
  MPK_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s));
  MPK_CUDA(cudaFreeAsync(buf, s));
  MPK_CUDA(cudaStreamSynchronize(s));
  if (h[1] != 1ull) return fail(MPK_TIMEOUT, "notification probe: a bounded wait ran out");
  if (h[2] == h[3]) return fail(MPK_INVALID_ARG, "notification probe: both blocks ran on one SM");
  *one_way_ns = (double)h[0] / (2.0 * rounds);
  if (sm_pair != nullptr) {
    sm_pair[0] = (int)h[2];
    sm_pair[1] = (int)h[3];
  }
  return MPK_OK;
}
