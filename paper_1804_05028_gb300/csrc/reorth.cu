// reorth.cu -- the fp64 reorthogonalisation of the Lanczos iteration (Sec. IV's Lanczos
// paragraph: the product dominates, so the vector work around it may be made accurate
// at little cost).
//
// After the three-term update w = H v_j - alpha_j v_j - beta_{j-1} v_{j-1}, a
// Gram-Schmidt sweep against m vectors u_0 .. u_{m-1} computes c_k = <u_k, w> and then
// w <- w - sum_k c_k u_k with ||w||^2.  Vectors may be fp32 or fp64 (real or complex).
// With fp64 vectors every operation is fp64.  With fp32 vectors the per-thread sums run
// in double-float (dfloat.cuh: exact fp32 products, about 48 significant bits; this
// GPU's fp64 pipe is far too slow for a sweep over 10^9 products), the coefficients are
// fp64 and split into two fp32 words for the update, and all cross-thread reductions are
// fp64; w is rounded once.  Reductions run in a fixed order (per warp, then per block,
// then over blocks), so a sweep is bit-for-bit reproducible -- the second Lanczos pass
// that rebuilds the ground state relies on that.
//
// Kernels (all HBM streams, no tensor cores: m dot products and one m-term axpy):
//   multidot_kernel   partial[k][blk] = sum over the block's rows of conj(u_k) w, for
//                     groups of 8 vectors (one group per blockIdx.y)
//   coef_kernel       c[k] = sum over blocks of partial[k][.], one block per k
//   update_kernel     w -= sum_k c_k u_k, partial ||w||^2 per block
//   combine_kernel    psi = sum_k s_k u_k (the Ritz vector from a stored Krylov basis)
#include "sced_internal.cuh"
#include "dfloat.cuh"
#include <type_traits>

namespace {

template <typename V> struct Rv;
template <> struct Rv<double> { using A = double; static constexpr bool cplx = false; };
template <> struct Rv<float> { using A = float; static constexpr bool cplx = false; };
template <> struct Rv<double2> { using A = double; static constexpr bool cplx = true; };
template <> struct Rv<float2> { using A = float; static constexpr bool cplx = true; };

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kGroup = 8;     // vectors per block of the multi-dot (blockIdx.y)

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

// Rows per thread and iteration: the loads of U rows (U grid-stride apart, so every load
// stays coalesced) are issued together, which keeps enough bytes in flight to stream
// from HBM; a thread still visits its rows in increasing order, so the sums do not
// depend on U.
template <typename V> struct RowsPer { static constexpr int U = 1; };
template <> struct RowsPer<float> { static constexpr int U = 4; };
template <> struct RowsPer<double> { static constexpr int U = 2; };
template <> struct RowsPer<float2> { static constexpr int U = 2; };

// conj(a) (w + wl) into one accumulator (double-float for fp32 vectors)
template <typename V>
__device__ __forceinline__ void md_acc(double &re, double &im, float &rh, float &rl, float &ih,
                                       float &il, const V a, const V wv, const V wl) {
  using A = typename Rv<V>::A;
  constexpr bool kC = Rv<V>::cplx;
  constexpr bool kF = std::is_same<A, float>::value;
  if constexpr (kF && kC) {
    df_add_prod(rh, rl, a.x, wv.x);
    df_add_prod(rh, rl, a.y, wv.y);
    df_add_prod(ih, il, a.x, wv.y);
    df_add_prod(ih, il, -a.y, wv.x);
    rl = __fmaf_rn(a.x, wl.x, __fmaf_rn(a.y, wl.y, rl));
    il = __fmaf_rn(a.x, wl.y, __fmaf_rn(-a.y, wl.x, il));
  } else if constexpr (kF) {
    df_add_prod(rh, rl, a, wv);
    rl = __fmaf_rn(a, wl, rl);
  } else if constexpr (kC) {
    re += a.x * wv.x + a.y * wv.y;
    im += a.x * wv.y - a.y * wv.x;
  } else {
    re += a * wv;
  }
}

template <typename V>
__device__ __forceinline__ V zero_v() {
  if constexpr (Rv<V>::cplx) { V z; z.x = 0; z.y = 0; return z; } else { return V(0); }
}

// Every thread keeps accumulators for a group of kGroup vectors (blockIdx.y selects the
// group) over its grid-stride rows: w[i] is read once per group and the kGroup loads of
// u_k[i] are independent.  fp32 vectors accumulate exact products in double-float, fp64
// vectors in fp64.  At the end the block reduces each accumulator in fp64 (warps, then the
// block's warps in order) into partial[(k * P + part) * nblk + blk], P = 2 for complex
// (re, im) else 1.
template <typename V>
__global__ void __launch_bounds__(kThreads, 4) multidot_kernel(VecSet S, const V *w, const V *wlo,
                                                            int64_t n, double *partial) {
  using A = typename Rv<V>::A;
  constexpr bool kC = Rv<V>::cplx;
  constexpr bool kF = std::is_same<A, float>::value;
  constexpr int P = kC ? 2 : 1;
  constexpr int U = RowsPer<V>::U;
  __shared__ double red[kGroup * P][kWarps];
  const int k0 = blockIdx.y * kGroup;
  const int kn = min(kGroup, S.m - k0);
  double re[kGroup], im[kGroup];        // fp64 vectors
  float rh[kGroup], rl[kGroup], ih[kGroup], il[kGroup];   // fp32 vectors: double-float
#pragma unroll
  for (int q = 0; q < kGroup; q++) { re[q] = im[q] = 0.0; rh[q] = rl[q] = ih[q] = il[q] = 0.f; }
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  for (; i + (U - 1) * stride < n; i += U * stride) {
    V wv[U], wl[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      wv[u] = w[i + u * stride];
      wl[u] = (kF && wlo) ? wlo[i + u * stride] : zero_v<V>();
    }
#pragma unroll
    for (int q = 0; q < kGroup; q++) {
      if (q < kn) {
        const V *uk = vec<V>(S, k0 + q);
        V a[U];
#pragma unroll
        for (int u = 0; u < U; u++) a[u] = uk[i + u * stride];
#pragma unroll
        for (int u = 0; u < U; u++) md_acc<V>(re[q], im[q], rh[q], rl[q], ih[q], il[q], a[u], wv[u], wl[u]);
      }
    }
  }
  for (; i < n; i += stride) {
    const V wv = w[i];
    const V wl = (kF && wlo) ? wlo[i] : zero_v<V>();
#pragma unroll
    for (int q = 0; q < kGroup; q++)
      if (q < kn) md_acc<V>(re[q], im[q], rh[q], rl[q], ih[q], il[q], vec<V>(S, k0 + q)[i], wv, wl);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kGroup; q++) {
    double a0 = re[q], b0 = im[q];
    if constexpr (kF) { a0 = df_value(rh[q], rl[q]); b0 = df_value(ih[q], il[q]); }
    const double a = warp_sum(a0);
    double b = 0.0;
    if constexpr (kC) b = warp_sum(b0);
    if (lane == 0) {
      red[q * P][wid] = a;
      if constexpr (kC) red[q * P + 1][wid] = b;
    }
  }
  __syncthreads();
  if (threadIdx.x < kn * P) {
    double sacc = 0.0;
    for (int q = 0; q < kWarps; q++) sacc += red[threadIdx.x][q];
    partial[(size_t)(k0 * P + threadIdx.x) * gridDim.x + blockIdx.x] = sacc;
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

// w <- w - sum_k c_k u_k, rounded once; partial[blk] = the block's ||w||^2.  fp32 vectors:
// every coefficient split into two fp32 words and the sum carried in double-float; fp64
// vectors: fp64.
// The running value of one row of w during the update: double-float words for fp32
// vectors (real and imaginary parts), fp64 otherwise.
template <typename V> struct Row;
template <> struct Row<float> { float h, l; };
template <> struct Row<float2> { float rh, rl, ih, il; };
template <> struct Row<double> { double t; };
template <> struct Row<double2> { double r, i; };

template <typename V>
__device__ __forceinline__ Row<V> row_load(const V *w, const V *wlo, int64_t i) {
  Row<V> R;
  if constexpr (std::is_same<V, float>::value) {
    R.h = w[i];
    R.l = wlo ? wlo[i] : 0.f;
  } else if constexpr (std::is_same<V, float2>::value) {
    const V w0 = w[i];
    R.rh = w0.x; R.ih = w0.y; R.rl = 0.f; R.il = 0.f;
    if (wlo) { const V l0 = wlo[i]; R.rl = l0.x; R.il = l0.y; }
  } else if constexpr (std::is_same<V, double>::value) {
    R.t = w[i];
  } else {
    const V w0 = w[i];
    R.r = w0.x; R.i = w0.y;
  }
  return R;
}

// R -= c_k a (cs: fp64 coefficients [m][P]; cf: the same as two fp32 words each)
template <typename V>
__device__ __forceinline__ void row_sub(Row<V> &R, const double *cs, const float *cf, int k, const V a) {
  if constexpr (std::is_same<V, float>::value) {
    df_sub_scaled(R.h, R.l, cf[2 * k], cf[2 * k + 1], a);
  } else if constexpr (std::is_same<V, float2>::value) {
    const float crh = cf[4 * k], crl = cf[4 * k + 1], cih = cf[4 * k + 2], cil = cf[4 * k + 3];
    df_sub_scaled(R.rh, R.rl, crh, crl, a.x);     // - cr a.x
    df_sub_scaled(R.rh, R.rl, -cih, -cil, a.y);   // + ci a.y
    df_sub_scaled(R.ih, R.il, crh, crl, a.y);     // - cr a.y
    df_sub_scaled(R.ih, R.il, cih, cil, a.x);     // - ci a.x
  } else if constexpr (std::is_same<V, double>::value) {
    R.t -= cs[k] * a;
  } else {
    const double cr = cs[2 * k], ci = cs[2 * k + 1];
    R.r -= cr * a.x - ci * a.y;
    R.i -= cr * a.y + ci * a.x;
  }
}

// w[i] (and wlo[i]) from R, rounded once; ||w||^2 accumulated
template <typename V>
__device__ __forceinline__ void row_store(const Row<V> &R, V *w, V *wlo, int64_t i, float &nh,
                                          float &nl, double &nrm) {
  if constexpr (std::is_same<V, float>::value) {
    float o, r;
    df_store(R.h, R.l, o, r);
    w[i] = o;
    if (wlo) wlo[i] = r; else r = 0.f;
    df_add_sq(nh, nl, o, r);
  } else if constexpr (std::is_same<V, float2>::value) {
    V o, r;
    df_store(R.rh, R.rl, o.x, r.x);
    df_store(R.ih, R.il, o.y, r.y);
    w[i] = o;
    if (wlo) wlo[i] = r; else { r.x = 0.f; r.y = 0.f; }
    df_add_sq(nh, nl, o.x, r.x);
    df_add_sq(nh, nl, o.y, r.y);
  } else if constexpr (std::is_same<V, double>::value) {
    w[i] = R.t;
    nrm += R.t * R.t;
  } else {
    V o;
    o.x = R.r;
    o.y = R.i;
    w[i] = o;
    nrm += R.r * R.r + R.i * R.i;
  }
}

// w <- w - sum_k c_k u_k, rounded once; partial[blk] = the block's ||w||^2.  fp32 vectors:
// every coefficient split into two fp32 words and the sum carried in double-float; fp64
// vectors: fp64.  Every row subtracts c_0 u_0, c_1 u_1, ... in that order; the loads of
// kK vectors for U rows are issued before the arithmetic that uses them.
template <typename V>
__global__ void __launch_bounds__(kThreads, 4) update_kernel(VecSet S, const double *c, V *w,
                                                          V *wlo, int64_t n, double *partial) {
  using A = typename Rv<V>::A;
  constexpr bool kC = Rv<V>::cplx;
  constexpr bool kF = std::is_same<A, float>::value;
  constexpr int P = kC ? 2 : 1;
  constexpr int U = RowsPer<V>::U;
  constexpr int kK = 8;
  extern __shared__ double cs[];   // [m][P] fp64, then (fp32 vectors) [m][P][2] words
  float *cf = reinterpret_cast<float *>(cs + S.m * P);
  for (int t = threadIdx.x; t < S.m * P; t += kThreads) {
    cs[t] = c[t];
    if constexpr (kF) df_split(c[t], cf[2 * t], cf[2 * t + 1]);
  }
  __syncthreads();
  float nh = 0.f, nl = 0.f;
  double nrm = 0.0;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  for (; i + (U - 1) * stride < n; i += U * stride) {
    Row<V> R[U];
#pragma unroll
    for (int u = 0; u < U; u++) R[u] = row_load<V>(w, wlo, i + u * stride);
    for (int k = 0; k < S.m; k += kK) {
      V a[kK][U];
#pragma unroll
      for (int kk = 0; kk < kK; kk++)
        if (k + kk < S.m) {
          const V *uk = vec<V>(S, k + kk);
#pragma unroll
          for (int u = 0; u < U; u++) a[kk][u] = uk[i + u * stride];
        }
#pragma unroll
      for (int kk = 0; kk < kK; kk++)
        if (k + kk < S.m) {
#pragma unroll
          for (int u = 0; u < U; u++) row_sub<V>(R[u], cs, cf, k + kk, a[kk][u]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; u++) row_store<V>(R[u], w, wlo, i + u * stride, nh, nl, nrm);
  }
  for (; i < n; i += stride) {
    Row<V> R = row_load<V>(w, wlo, i);
    for (int k = 0; k < S.m; k++) row_sub<V>(R, cs, cf, k, vec<V>(S, k)[i]);
    row_store<V>(R, w, wlo, i, nh, nl, nrm);
  }
  if constexpr (kF) nrm = df_value(nh, nl);
  block_sum_store(nrm, partial, blockIdx.x);
}

// psi = sum_k s_k u_k (real coefficients: the tridiagonal matrix is real symmetric)
template <typename V>
__global__ void __launch_bounds__(kThreads) combine_kernel(VecSet S, const double *s, V *psi,
                                                           int64_t n) {
  using A = typename Rv<V>::A;
  constexpr bool kC = Rv<V>::cplx;
  constexpr bool kF = std::is_same<A, float>::value;
  extern __shared__ double cs[];
  float *cf = reinterpret_cast<float *>(cs + S.m);
  for (int t = threadIdx.x; t < S.m; t += kThreads) {
    cs[t] = s[t];
    if constexpr (kF) df_split(s[t], cf[2 * t], cf[2 * t + 1]);
  }
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    if constexpr (kF && kC) {
      float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
      for (int k = 0; k < S.m; k++) {
        const V a = vec<V>(S, k)[i];
        df_sub_scaled(rh, rl, -cf[2 * k], -cf[2 * k + 1], a.x);
        df_sub_scaled(ih, il, -cf[2 * k], -cf[2 * k + 1], a.y);
      }
      V o;
      o.x = df_round(rh, rl);
      o.y = df_round(ih, il);
      psi[i] = o;
    } else if constexpr (kF) {
      float hi = 0.f, lo = 0.f;
      for (int k = 0; k < S.m; k++) df_sub_scaled(hi, lo, -cf[2 * k], -cf[2 * k + 1], vec<V>(S, k)[i]);
      psi[i] = df_round(hi, lo);
    } else if constexpr (kC) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < S.m; k++) {
        const V a = vec<V>(S, k)[i];
        re += cs[k] * a.x;
        im += cs[k] * a.y;
      }
      V o;
      o.x = re;
      o.y = im;
      psi[i] = o;
    } else {
      double t = 0.0;
      for (int k = 0; k < S.m; k++) t += cs[k] * vec<V>(S, k)[i];
      psi[i] = t;
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
                           cudaStream_t st, void *wlo) {
  if (m <= 0) return ED_OK;
  const bool cplx = dtype == ED_C128 || dtype == ED_C64;
  const int P = cplx ? 2 : 1;
  const int grid = ed_reorth_grid(B);
  const VecSet S = make_set(base, B->D, p0, p1, m);
  const size_t smem_upd = 2 * sizeof(double) * (size_t)m * P;   // fp64 + two fp32 words
  if (smem_upd > 48 * 1024) return ed_fail(ED_ERR_UNSUPPORTED, "too many vectors in one sweep");
  const dim3 dgrid(grid, (m + kGroup - 1) / kGroup);
  RO_DISPATCH(dtype, {
    multidot_kernel<V><<<dgrid, kThreads, 0, st>>>(S, (const V *)w, (const V *)wlo, B->D, partial);
    ED_CK(cudaGetLastError());
    coef_kernel<<<m * P, kThreads, 0, st>>>(partial, grid, c);
    ED_CK(cudaGetLastError());
    update_kernel<V><<<grid, kThreads, smem_upd, st>>>(S, c, (V *)w, (V *)wlo, B->D, partial);
    ED_CK(cudaGetLastError());
  });
  return ED_OK;
}

// psi = sum_k s[k] (base + k * D), s a DEVICE array of m doubles.
int ed_launch_combine(const ed_basis *B, void *psi, const void *base, int m, const double *s,
                      int dtype, cudaStream_t st) {
  const VecSet S = make_set(base, B->D, nullptr, nullptr, m);
  const size_t smem = 2 * sizeof(double) * (size_t)m;
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
