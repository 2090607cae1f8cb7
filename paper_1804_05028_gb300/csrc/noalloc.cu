// noalloc.cu -- a dot product that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need a reduction: a
// host loop that must not stall other work on the device (cudaMalloc and cudaFree may
// synchronise the whole device), or an embedding framework that owns every byte of device
// memory through its own pool and forbids allocations it does not make.  ed_dot (capi.cu)
// keeps its block partials in scratch that ed_build_basis allocated; this variant keeps
// them in a fixed array compiled into the library instead, so a call needs no basis and
// performs no allocation of any kind.
//
// The array lives on every device that loads the library, until the process exits.  All
// calls share it and it keeps the last call's partials; every slot a call reads was
// written earlier in that same call, so nothing has to be cleared.  Two calls whose work
// overlaps on the device (different streams, no ordering between them) race on it.
#include "sced_internal.cuh"

#include <mutex>

namespace {

constexpr int kThreads = 256;
constexpr int64_t kPerThread = 64;                          // elements per thread
constexpr int64_t kPerBlock = kThreads * kPerThread;        // 16384 elements per block
constexpr int kMaxBlocks = 65536;                           // partials kept in the array
constexpr int64_t kMaxN = (int64_t)kMaxBlocks * kPerBlock;  // 2^30 elements

// (re, im) of every block's partial sum: 65536 x 2 doubles = 1 MiB
static __device__ __align__(256) double g_dot_scratch[2 * kMaxBlocks];

std::mutex g_mu;
double *g_ptr[64] = {nullptr};   // device address of g_dot_scratch, per device ordinal

template <typename V> struct Cx { static constexpr bool cplx = false; };
template <> struct Cx<double2> { static constexpr bool cplx = true; };
template <> struct Cx<float2> { static constexpr bool cplx = true; };

// one fixed slice of kPerBlock elements per block; strided so that loads coalesce
template <typename V>
__global__ void __launch_bounds__(kThreads) dot_fixed_partials(const V *x, const V *y, int64_t n,
                                                               double *part) {
  const int64_t base = (int64_t)blockIdx.x * kPerBlock;
  double re = 0.0, im = 0.0;
#pragma unroll 4
  for (int64_t k = threadIdx.x; k < kPerBlock; k += kThreads) {
    const int64_t i = base + k;
    if (i >= n) break;
    if constexpr (Cx<V>::cplx) {
      const V a = x[i], b = y[i];
      re += (double)a.x * b.x + (double)a.y * b.y;
      im += (double)a.x * b.y - (double)a.y * b.x;
    } else {
      re += (double)x[i] * (double)y[i];
    }
  }
  __shared__ double sr[kThreads / 32], si[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xFFFFFFFFu, re, o);
    im += __shfl_down_sync(0xFFFFFFFFu, im, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sr[wid] = re; si[wid] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kThreads / 32; w++) { a += sr[w]; b += si[w]; }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// sum of the partials in block order (one block; fixed order, deterministic)
__global__ void __launch_bounds__(kThreads) dot_fixed_final(const double *part, int nblk,
                                                            double *out) {
  __shared__ double sr[kThreads], si[kThreads];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblk; k += kThreads) { a += part[2 * k]; b += part[2 * k + 1]; }
  sr[threadIdx.x] = a;
  si[threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x == 0) {
    double ra = 0.0, rb = 0.0;
    for (int k = 0; k < kThreads; k++) { ra += sr[k]; rb += si[k]; }
    out[0] = ra;
    out[1] = rb;
  }
}

// Address of g_dot_scratch on the current device.  The host-side name of a __device__
// array is only a stand-in, so the device address is asked for once per device (with that
// device current) and remembered.
int scratch_on_current_device(double **ptr) {
  int dev = 0;
  ED_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return ed_fail(ED_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_dot_scratch);
    if (e != cudaSuccess) return ed_cuda_fail(e, "cudaGetSymbolAddress(g_dot_scratch)");
    g_ptr[dev] = static_cast<double *>(p);
  }
  *ptr = g_ptr[dev];
  return ED_OK;
}

template <typename V>
int launch(const void *x, const void *y, int64_t n, double *part, int nblk, double *out,
           cudaStream_t st) {
  if (nblk > 0) {
    dot_fixed_partials<V><<<nblk, kThreads, 0, st>>>((const V *)x, (const V *)y, n, part);
    ED_CK(cudaGetLastError());
  }
  dot_fixed_final<<<1, kThreads, 0, st>>>(part, nblk, out);
  ED_CK(cudaGetLastError());
  return ED_OK;
}

}  // namespace

extern "C" int ed_dot_noalloc(const void *x, const void *y, int64_t n, int32_t dtype, double *out,
                              void *stream) {
  if (!out) return ed_fail(ED_ERR_INVALID, "out is null");
  if (n < 0) return ed_fail(ED_ERR_INVALID, "n is negative");
  if (n > kMaxN)
    return ed_fail(ED_ERR_INVALID, "ed_dot_noalloc handles at most 2^30 elements (its fixed "
                                   "scratch holds 65536 block partials of 16384 elements); got " +
                                       std::to_string(n));
  if (n > 0 && (!x || !y)) return ed_fail(ED_ERR_INVALID, "null vector");
  double *part = nullptr;
  int rc = scratch_on_current_device(&part);
  if (rc) return rc;
  const int nblk = (int)((n + kPerBlock - 1) / kPerBlock);
  cudaStream_t st = (cudaStream_t)stream;
  switch (dtype) {
    case ED_F64: return launch<double>(x, y, n, part, nblk, out, st);
    case ED_F32: return launch<float>(x, y, n, part, nblk, out, st);
    case ED_C128: return launch<double2>(x, y, n, part, nblk, out, st);
    case ED_C64: return launch<float2>(x, y, n, part, nblk, out, st);
  }
  return ed_fail(ED_ERR_INVALID, "unknown dtype");
}
