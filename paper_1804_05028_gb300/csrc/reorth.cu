// reorth.cu -- the fp64 reorthogonalisation of the Lanczos iteration (Sec. IV's Lanczos
// paragraph: the product dominates, so the vector work around it may be made accurate
// at little cost).
//
// After the three-term update w = H v_j - alpha_j v_j - beta_{j-1} v_{j-1}, a
// Gram-Schmidt sweep against m vectors u_0 .. u_{m-1} computes c_k = <u_k, w> and then
// w <- w - sum_k c_k u_k with ||w||^2.  Vectors may be fp32 or fp64 (real or complex);
// every dot, every coefficient and the update are accumulated in fp64 and w is rounded
// once.  Reductions run in a fixed order (per warp, then per block, then over blocks),
// so a sweep is bit-for-bit reproducible -- the second Lanczos pass that rebuilds the
// ground state relies on that.
//
// Kernels (all HBM streams, no tensor cores: m dot products and one m-term axpy):
//   multidot_kernel   partial[k][blk] = sum over the block's rows of conj(u_k) w
//   coef_kernel       c[k] = sum over blocks of partial[k][.], one block per k
//   update_kernel     w -= sum_k c_k u_k, partial ||w||^2 per block
//   combine_kernel    psi = sum_k s_k u_k (the Ritz vector from a stored Krylov basis)
#include "sced_internal.cuh"

namespace {

template <typename V> struct Rv;
template <> struct Rv<double> { using A = double; static constexpr bool cplx = false; };
template <> struct Rv<float> { using A = float; static constexpr bool cplx = false; };
template <> struct Rv<double2> { using A = double; static constexpr bool cplx = true; };
template <> struct Rv<float2> { using A = float; static constexpr bool cplx = true; };

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRows = 8;      // rows per lane in one pass of a warp over its chunk

// the m vectors: base + k * stride (a Krylov store), or the two explicit pointers p0, p1
struct VecSet {
  const void *base;
  int64_t stride;
  const void *p0, *p1;
  int m;
};

template <typename V>
__device__ __forceinline__ const V *vec(const VecSet &S, int k) {
  if (S.base) return reinterpret_cast<const V *>(S.base) + (size_t)k * (size_t)S.stride;
  return reinterpret_cast<const V *>(k ? S.p1 : S.p0);
}

__device__ __forceinline__ double warp_sum(double d) {
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
  return d;
}

// Each warp walks chunks of 32 * kRows rows (grid-stride over chunks), holding w in
// registers; for every k it reduces conj(u_k) w over the chunk and lane 0 adds the sum to
// its own shared slot acc[k][warp].  At the end the block sums its warps' slots in warp
// order into partial[(k * P + part) * nblk + blk], P = 2 for complex (re, im) else 1.
template <typename V>
__global__ void __launch_bounds__(kThreads) multidot_kernel(VecSet S, const V *w, int64_t n,
                                                            double *partial) {
  constexpr bool kC = Rv<V>::cplx;
  constexpr int P = kC ? 2 : 1;
  extern __shared__ double acc[];   // [m][P][kWarps]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < S.m * P * kWarps; t += kThreads) acc[t] = 0.0;
  __syncthreads();
  const int64_t chunk = 32 * kRows;
  const int64_t n_chunks = (n + chunk - 1) / chunk;
  for (int64_t c = (int64_t)blockIdx.x * kWarps + wid; c < n_chunks;
       c += (int64_t)gridDim.x * kWarps) {
    const int64_t r0 = c * chunk + lane;
    V wv[kRows];
#pragma unroll
    for (int r = 0; r < kRows; r++) {
      const int64_t i = r0 + 32 * r;
      if (i < n) wv[r] = w[i];
      else if constexpr (kC) { wv[r].x = 0; wv[r].y = 0; } else wv[r] = 0;
    }
    for (int k = 0; k < S.m; k++) {
      const V *u = vec<V>(S, k);
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int r = 0; r < kRows; r++) {
        const int64_t i = r0 + 32 * r;
        if (i < n) {
          const V a = u[i];
          if constexpr (kC) {   // conj(a) * w
            re += (double)a.x * wv[r].x + (double)a.y * wv[r].y;
            im += (double)a.x * wv[r].y - (double)a.y * wv[r].x;
          } else {
            re += (double)a * (double)wv[r];
          }
        }
      }
      re = warp_sum(re);
      if constexpr (kC) im = warp_sum(im);
      if (lane == 0) {
        acc[(k * P) * kWarps + wid] += re;
        if constexpr (kC) acc[(k * P + 1) * kWarps + wid] += im;
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < S.m * P; t += kThreads) {
    double s = 0.0;
    for (int q = 0; q < kWarps; q++) s += acc[t * kWarps + q];
    partial[(size_t)t * gridDim.x + blockIdx.x] = s;
  }
}

// c[t] = sum_b partial[t * nblk + b] for t < m * P, one block per t: every thread sums a
// fixed stride of blocks, then a fixed-shape tree.
__global__ void __launch_bounds__(kThreads) coef_kernel(const double *partial, int nblk, double *c) {
  __shared__ double red[kWarps];
  const int t = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += kThreads) s += partial[(size_t)t * nblk + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < kWarps; q++) a += red[q];
    c[t] = a;
  }
}

__device__ __forceinline__ void block_sum_store(double d, double *out, int slot) {
  __shared__ double red[kWarps];
  d = warp_sum(d);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int q = 0; q < kWarps; q++) a += red[q];
    out[slot] = a;
  }
}

// w <- w - sum_k c_k u_k in fp64, rounded once; partial[blk] = the block's ||w||^2.
template <typename V>
__global__ void __launch_bounds__(kThreads) update_kernel(VecSet S, const double *c, V *w,
                                                          int64_t n, double *partial) {
  using A = typename Rv<V>::A;
  constexpr bool kC = Rv<V>::cplx;
  extern __shared__ double cs[];   // [m][P]
  const int P = kC ? 2 : 1;
  for (int t = threadIdx.x; t < S.m * P; t += kThreads) cs[t] = c[t];
  __syncthreads();
  double nrm = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    if constexpr (kC) {
      double wr = w[i].x, wi = w[i].y;
      for (int k = 0; k < S.m; k++) {
        const V a = vec<V>(S, k)[i];
        const double cr = cs[2 * k], ci = cs[2 * k + 1];
        wr -= cr * (double)a.x - ci * (double)a.y;
        wi -= cr * (double)a.y + ci * (double)a.x;
      }
      V o;
      o.x = (A)wr;
      o.y = (A)wi;
      w[i] = o;
      nrm += (double)o.x * o.x + (double)o.y * o.y;
    } else {
      double t = (double)w[i];
      for (int k = 0; k < S.m; k++) t -= cs[k] * (double)vec<V>(S, k)[i];
      const A o = (A)t;
      w[i] = o;
      nrm += (double)o * (double)o;
    }
  }
  block_sum_store(nrm, partial, blockIdx.x);
}

// psi = sum_k s_k u_k (real coefficients: the tridiagonal matrix is real symmetric)
template <typename V>
__global__ void __launch_bounds__(kThreads) combine_kernel(VecSet S, const double *s, V *psi,
                                                           int64_t n) {
  using A = typename Rv<V>::A;
  constexpr bool kC = Rv<V>::cplx;
  extern __shared__ double cs[];
  for (int t = threadIdx.x; t < S.m; t += kThreads) cs[t] = s[t];
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    if constexpr (kC) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < S.m; k++) {
        const V a = vec<V>(S, k)[i];
        re += cs[k] * (double)a.x;
        im += cs[k] * (double)a.y;
      }
      V o;
      o.x = (A)re;
      o.y = (A)im;
      psi[i] = o;
    } else {
      double t = 0.0;
      for (int k = 0; k < S.m; k++) t += cs[k] * (double)vec<V>(S, k)[i];
      psi[i] = (A)t;
    }
  }
}

#define RO_DISPATCH(dtype, ...)                                   \
  switch (dtype) {                                                \
    case ED_F64: { using V = double; __VA_ARGS__; break; }        \
    case ED_F32: { using V = float; __VA_ARGS__; break; }         \
    case ED_C128: { using V = double2; __VA_ARGS__; break; }      \
    case ED_C64: { using V = float2; __VA_ARGS__; break; }        \
    default: return ed_fail(ED_ERR_INVALID, "unknown dtype");     \
  }

VecSet make_set(const void *base, int64_t stride, const void *p0, const void *p1, int m) {
  VecSet S;
  S.base = base;
  S.stride = stride;
  S.p0 = p0;
  S.p1 = p1;
  S.m = m;
  return S;
}

}  // namespace

int ed_reorth_grid(const ed_basis *B) { return 4 * B->sm_count; }

// One Gram-Schmidt sweep of w against m vectors (base + k * D, or p0 and p1 when base is
// null): coefficients c (device, m * P doubles, P = 2 for complex) and ||w||^2 block
// partials in partial[0 .. grid).  partial must hold m * P * grid doubles.
int ed_launch_reorth_sweep(const ed_basis *B, void *w, const void *base, const void *p0,
                           const void *p1, int m, int dtype, double *partial, double *c,
                           cudaStream_t st) {
  if (m <= 0) return ED_OK;
  const bool cplx = dtype == ED_C128 || dtype == ED_C64;
  const int P = cplx ? 2 : 1;
  const int grid = ed_reorth_grid(B);
  const VecSet S = make_set(base, B->D, p0, p1, m);
  const size_t smem_dot = sizeof(double) * (size_t)m * P * kWarps;
  const size_t smem_upd = sizeof(double) * (size_t)m * P;
  if (smem_dot > 200 * 1024) return ed_fail(ED_ERR_UNSUPPORTED, "too many vectors in one sweep");
  RO_DISPATCH(dtype, {
    auto kd = multidot_kernel<V>;
    if (smem_dot > 48 * 1024)
      ED_CK(cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_dot));
    kd<<<grid, kThreads, smem_dot, st>>>(S, (const V *)w, B->D, partial);
    ED_CK(cudaGetLastError());
    coef_kernel<<<m * P, kThreads, 0, st>>>(partial, grid, c);
    ED_CK(cudaGetLastError());
    update_kernel<V><<<grid, kThreads, smem_upd, st>>>(S, c, (V *)w, B->D, partial);
    ED_CK(cudaGetLastError());
  });
  return ED_OK;
}

// psi = sum_k s[k] (base + k * D), s a DEVICE array of m doubles.
int ed_launch_combine(const ed_basis *B, void *psi, const void *base, int m, const double *s,
                      int dtype, cudaStream_t st) {
  const VecSet S = make_set(base, B->D, nullptr, nullptr, m);
  const size_t smem = sizeof(double) * (size_t)m;
  if (smem > 200 * 1024) return ed_fail(ED_ERR_UNSUPPORTED, "too many vectors to combine");
  RO_DISPATCH(dtype, {
    auto k = combine_kernel<V>;
    if (smem > 48 * 1024)
      ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k<<<ed_reorth_grid(B), kThreads, smem, st>>>(S, s, (V *)psi, B->D);
    ED_CK(cudaGetLastError());
  });
  return ED_OK;
}
