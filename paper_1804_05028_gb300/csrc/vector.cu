// vector.cu -- the Lanczos vector operations on a caller's slice of a vector (Sec. IV: the
// product dominates Lanczos; the scalings, updates and dot products around it are
// streaming passes).  The single-device ed_lanczos keeps its vectors inside the library;
// these entry points serve a driver that holds only a slice of every vector, such as a
// row-sharded Lanczos across ranks, so that its rank-local arithmetic also runs in the
// library's kernels.  fp32 vectors use double-float accumulation (dfloat.cuh), fp64
// vectors fp64; reductions are in a fixed order.
#include "sced_internal.cuh"
#include "dfloat.cuh"
#include <algorithm>

namespace {

template <typename V> struct Vv;
template <> struct Vv<double> { using A = double; static constexpr bool cplx = false; };
template <> struct Vv<float> { using A = float; static constexpr bool cplx = false; };
template <> struct Vv<double2> { using A = double; static constexpr bool cplx = true; };
template <> struct Vv<float2> { using A = float; static constexpr bool cplx = true; };

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double d) {
  __shared__ double red[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  double a = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kThreads / 32; q++) a += red[q];
  return a;
}

// w <- w - a v - b vprev (vprev may be null), rounded once; partial[blk] = the block's
// ||w||^2 (as the single-device three-term update)
template <typename V>
__global__ void __launch_bounds__(kThreads) slice_axpy_norm(V *w, const V *v, const V *vprev,
                                                            double a, double b, int64_t n,
                                                            double *partial) {
  using A = typename Vv<V>::A;
  constexpr bool kF = sizeof(A) == 4;
  constexpr bool kC = Vv<V>::cplx;
  float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f, nh = 0.f, nl = 0.f;
  double acc = 0.0;
  if constexpr (kF) { df_split(a, ah, al); df_split(b, bh, bl); }
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    if constexpr (kF && kC) {
      const V w0 = w[i], v0 = v[i];
      float rh = w0.x, rl = 0.f, ih = w0.y, il = 0.f;
      df_sub_scaled(rh, rl, ah, al, v0.x);
      df_sub_scaled(ih, il, ah, al, v0.y);
      if (vprev) {
        const V p0 = vprev[i];
        df_sub_scaled(rh, rl, bh, bl, p0.x);
        df_sub_scaled(ih, il, bh, bl, p0.y);
      }
      V o; o.x = df_round(rh, rl); o.y = df_round(ih, il);
      w[i] = o;
      df_add_prod(nh, nl, o.x, o.x);
      df_add_prod(nh, nl, o.y, o.y);
    } else if constexpr (kF) {
      float hi = w[i], lo = 0.f;
      df_sub_scaled(hi, lo, ah, al, v[i]);
      if (vprev) df_sub_scaled(hi, lo, bh, bl, vprev[i]);
      const float o = df_round(hi, lo);
      w[i] = o;
      df_add_prod(nh, nl, o, o);
    } else if constexpr (kC) {
      double wr = w[i].x - a * v[i].x, wi = w[i].y - a * v[i].y;
      if (vprev) { wr -= b * vprev[i].x; wi -= b * vprev[i].y; }
      V o; o.x = wr; o.y = wi;
      w[i] = o;
      acc += wr * wr + wi * wi;
    } else {
      double t = w[i] - a * v[i];
      if (vprev) t -= b * vprev[i];
      w[i] = t;
      acc += t * t;
    }
  }
  if constexpr (kF) acc = df_value(nh, nl);
  const double s = block_sum(acc);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// out[0] = sum of partial[0 .. n) in a fixed order
__global__ void __launch_bounds__(kThreads) sum_partials(const double *partial, int n, double *out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += kThreads) s += partial[k];
  s = block_sum(s);
  if (threadIdx.x == 0) out[0] = s;
}

template <typename V>
__global__ void __launch_bounds__(kThreads) slice_scale(V *x, double s, int64_t n) {
  using A = typename Vv<V>::A;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    if constexpr (Vv<V>::cplx) {
      V o = x[i];
      o.x = (A)(o.x * s);
      o.y = (A)(o.y * s);
      x[i] = o;
    } else {
      x[i] = (A)(x[i] * s);
    }
  }
}

#define VV_DISPATCH(dtype, ...)                                    \
  switch (dtype) {                                                 \
    case ED_F64: { using V = double; __VA_ARGS__; break; }         \
    case ED_F32: { using V = float; __VA_ARGS__; break; }          \
    case ED_C128: { using V = double2; __VA_ARGS__; break; }       \
    case ED_C64: { using V = float2; __VA_ARGS__; break; }         \
    default: return ed_fail(ED_ERR_INVALID, "unknown dtype");      \
  }

int grid_for_slice(int64_t n, int cap) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)sms * 4);
  g = std::min<int64_t>(g, cap);
  return (int)std::max<int64_t>(g, 1);
}

}  // namespace

extern "C" int ed_axpy_norm(void *w, const void *v, const void *vprev, double a, double b,
                            int64_t n, int32_t dtype, double *scratch, int64_t scratch_len,
                            double *norm2, void *stream) {
  if (n < 0) return ed_fail(ED_ERR_INVALID, "negative length");
  if (!scratch || scratch_len < 1 || !norm2) return ed_fail(ED_ERR_INVALID, "scratch and norm2 are required");
  if (n > 0 && (!w || !v)) return ed_fail(ED_ERR_INVALID, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  const int grid = grid_for_slice(n, (int)std::min<int64_t>(scratch_len, 1 << 20));
  if (n > 0) {
    VV_DISPATCH(dtype, slice_axpy_norm<V><<<grid, kThreads, 0, st>>>((V *)w, (const V *)v,
                                                                     (const V *)vprev, a, b, n, scratch));
    ED_CK(cudaGetLastError());
    sum_partials<<<1, kThreads, 0, st>>>(scratch, grid, norm2);
  } else {
    ED_CK(cudaMemsetAsync(norm2, 0, sizeof(double), st));
  }
  ED_CK(cudaGetLastError());
  return ED_OK;
}

extern "C" int ed_scale(void *x, double s, int64_t n, int32_t dtype, void *stream) {
  if (n < 0) return ed_fail(ED_ERR_INVALID, "negative length");
  if (n == 0) return ED_OK;
  if (!x) return ed_fail(ED_ERR_INVALID, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  VV_DISPATCH(dtype, slice_scale<V><<<grid_for_slice(n, 1 << 20), kThreads, 0, st>>>((V *)x, s, n));
  ED_CK(cudaGetLastError());
  return ED_OK;
}
