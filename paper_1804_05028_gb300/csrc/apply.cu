// apply.cu -- the matrix-free product y = H x on the symmetry-adapted basis
// (Sec. IV, Eqs. 12-17 of arXiv:1804.05028, restated as a row-wise pull), the
// find_rep test hook, and the streaming vector kernels of the Lanczos iteration.
//
// Row-wise pull: row i owns y_i.  For every antiparallel bond of its representative
// s_i the exchanged configuration s' is mapped to its representative s_j = h s' by
// sublattice coding (Alg. 2), s_j is located in Basis through Limits (Sec. IV), and
// y_i += (J_c/2) chi(h) sqrt(|Stab_j|/|Stab_i|) x_j -- the conjugate-transposed form
// of the push of Alg. 4, exact because H is Hermitian.  Each y_i is written once:
// no atomics, no inter-block communication, fixed summation order.
#include "sced_internal.cuh"
#include "dfloat.cuh"
#include <cstdlib>

namespace {

template <typename V> struct Vt;
template <> struct Vt<double> { using A = double; static constexpr bool cplx = false; };
template <> struct Vt<float> { using A = float; static constexpr bool cplx = false; };
template <> struct Vt<double2> { using A = double; static constexpr bool cplx = true; };
template <> struct Vt<float2> { using A = float; static constexpr bool cplx = true; };

struct ApplyParams {
  DevTables T;
  DevIndex I;
  int n_classes;
  int cls_off[ED_MAXCLS + 1];
  double jh[ED_MAXCLS];    // J_c / 2, amplitude of the exchange term
  double jzq[ED_MAXCLS];   // J_c Jz_c / 4, S^z S^z of a parallel pair
  const uint8_t *bond_pos; // [n_bonds][2] bit positions (N-1-label), class-sorted
  const double *sqrt_tab;  // sqrt(t), t = 0..nsym
  const double *rsqrt_tab; // 1/sqrt(t)
  const double *cs;        // [denom][2] cos, sin (complex sectors)
  const void *x;
  void *y;
  int64_t r0, r1;          // rows [r0, r1); y[0] is row r0
  double *partial;         // optional [gridDim.x] (or 2x for complex) partial <x_rows, y>
  // shared-memory layout (bytes)
  int stage_tables;
  uint32_t sym_list_bytes;
  uint32_t off_rep, off_symoff, off_phase, off_symlist, off_dest, off_bond, off_sqrt, off_cs;
  uint32_t smem_bytes;
};

template <typename A>
__device__ __forceinline__ void block_reduce_store(A v, double *out, int slot) {
  __shared__ double red[32];
  double d = (double)v;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = d;
  __syncthreads();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    d = lane < nw ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
    if (lane == 0) out[slot] = d;
  }
}

// Stage Rep_X, Sym_X offsets and lists, dest, phases, bond positions and the norm /
// character tables in shared memory (they are small: O(nsub 2^n) entries).
template <typename A, bool kStage>
__device__ __forceinline__ void stage(const ApplyParams &P, unsigned char *sm) {
  const DevTables &T = P.T;
  auto cp32 = [&](uint32_t off, const void *src, size_t bytes) {
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(sm + off);
    for (size_t k = threadIdx.x; k < bytes / 4; k += blockDim.x) d[k] = s[k];
  };
  auto cp8 = [&](uint32_t off, const void *src, size_t bytes) {
    const unsigned char *s = reinterpret_cast<const unsigned char *>(src);
    for (size_t k = threadIdx.x; k < bytes; k += blockDim.x) sm[off + k] = s[k];
  };
  if (kStage) {
    const size_t nn = (size_t)1 << T.n;
    cp32(P.off_rep, T.rep, (size_t)T.nsub * nn * 4);
    cp32(P.off_symoff, T.sym_off, (size_t)T.nsub * (nn + 1) * 4);
    cp32(P.off_phase, T.phase, (size_t)T.nsym * 4);
    cp8(P.off_symlist, T.sym_list, (size_t)P.sym_list_bytes);
    cp8(P.off_dest, T.dest, (size_t)T.nsym * T.nsub);
  }
  cp8(P.off_bond, P.bond_pos, (size_t)P.cls_off[P.n_classes] * 2);
  A *sq = reinterpret_cast<A *>(sm + P.off_sqrt);
  for (int k = threadIdx.x; k <= T.nsym; k += blockDim.x) {
    sq[2 * k] = (A)P.sqrt_tab[k];
    sq[2 * k + 1] = (A)P.rsqrt_tab[k];
  }
  if (P.cs) {
    A *c = reinterpret_cast<A *>(sm + P.off_cs);
    for (int k = threadIdx.x; k < 2 * T.denom; k += blockDim.x) c[k] = (A)P.cs[k];
  }
  __syncthreads();
}

// kMode 0: y = H x (and the optional <x, y> partials).  kMode 1: no y; per coupling class
// c the partial sums of Re <x | H_c x> with unit exchange (P.jh, P.jzq set for J_c = 1)
// into P.partial[c * gridDim.x + block] (Hellmann-Feynman derivative dE0/dJ_c).
template <typename V, bool kStage, int kMode>
__global__ void __launch_bounds__(256) apply_h_kernel(const ApplyParams P) {
  using A = typename Vt<V>::A;
  constexpr bool kC = Vt<V>::cplx;
  extern __shared__ __align__(16) unsigned char sm[];
  stage<A, kStage>(P, sm);
  const DevTables &T = P.T;
  const uint32_t *rep_s = kStage ? reinterpret_cast<const uint32_t *>(sm + P.off_rep) : T.rep;
  const uint32_t *symoff_s =
      kStage ? reinterpret_cast<const uint32_t *>(sm + P.off_symoff) : T.sym_off;
  const uint16_t *symlist_s =
      kStage ? reinterpret_cast<const uint16_t *>(sm + P.off_symlist) : T.sym_list;
  const uint8_t *dest_s = kStage ? reinterpret_cast<const uint8_t *>(sm + P.off_dest) : T.dest;
  const int32_t *phase_s =
      kStage ? reinterpret_cast<const int32_t *>(sm + P.off_phase) : T.phase;
  const uint8_t *bond_s = sm + P.off_bond;
  const A *sq = reinterpret_cast<const A *>(sm + P.off_sqrt);
  const A *cs = reinterpret_cast<const A *>(sm + P.off_cs);
  const V *x = reinterpret_cast<const V *>(P.x);
  V *y = reinterpret_cast<V *>(P.y);

  double dot_re = 0.0, dot_im = 0.0;
  double cls_dot[kMode == 1 ? ED_MAXCLS : 1];
  for (int c = 0; c < (kMode == 1 ? ED_MAXCLS : 1); c++) cls_dot[c] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = P.r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.r1; i += stride) {
    const uint64_t s = __ldg(P.I.basis + i);
    const int ti = __ldg(P.I.stab + i);
    A row_re = 0, row_im = 0;
    double diag = 0.0;
    for (int c = 0; c < P.n_classes; c++) {
      A acc_re = 0, acc_im = 0;
      int nanti = 0;
      const int b1 = P.cls_off[c + 1];
      for (int b = P.cls_off[c]; b < b1; b++) {
        const int pa = bond_s[2 * b], pb = bond_s[2 * b + 1];
        if ((((s >> pa) ^ (s >> pb)) & 1ULL) == 0) continue;
        nanti++;
        const uint64_t s2 = s ^ ((1ULL << pa) | (1ULL << pb));
        const RepOut R = find_rep(T, rep_s, symoff_s, symlist_s, dest_s, phase_s, s2);
        if (R.mixed) continue;
        const int64_t j = lookup_index(P.I, R.rep);
        if (j < 0) continue;
        const A w = sq[2 * R.t];
        const int ph = phase_s[R.g];
        if constexpr (!kC) {
          const A v = w * x[j];
          acc_re += (ph == 0) ? v : -v;   // real sector: chi(h) = +1 or -1
        } else {
          const V xj = x[j];
          const A cr = cs[2 * ph] * w, ci = cs[2 * ph + 1] * w;
          acc_re += cr * xj.x - ci * xj.y;
          acc_im += cr * xj.y + ci * xj.x;
        }
      }
      const double dg = P.jzq[c] * (double)((b1 - P.cls_off[c]) - 2 * nanti);
      diag += dg;
      row_re += (A)P.jh[c] * acc_re;
      if constexpr (kC) row_im += (A)P.jh[c] * acc_im;
      if constexpr (kMode == 1) {
        const double rsd = (double)sq[2 * ti + 1];
        if constexpr (!kC) {
          const double xv = (double)x[i];
          cls_dot[c] += dg * xv * xv + P.jh[c] * rsd * xv * (double)acc_re;
        } else {
          const V xv = x[i];
          cls_dot[c] += dg * ((double)xv.x * xv.x + (double)xv.y * xv.y) +
                        P.jh[c] * rsd * ((double)xv.x * acc_re + (double)xv.y * acc_im);
        }
      }
    }
    if constexpr (kMode == 1) continue;
    const A rs = sq[2 * ti + 1];
    if constexpr (!kC) {
      const V xi = x[i];
      const V yi = (A)diag * xi + row_re * rs;
      y[i - P.r0] = yi;
      if (P.partial) dot_re += (double)xi * (double)yi;
    } else {
      const V xi = x[i];
      V yi;
      yi.x = (A)diag * xi.x + row_re * rs;
      yi.y = (A)diag * xi.y + row_im * rs;
      y[i - P.r0] = yi;
      if (P.partial) {
        dot_re += (double)xi.x * yi.x + (double)xi.y * yi.y;
        dot_im += (double)xi.x * yi.y - (double)xi.y * yi.x;
      }
    }
  }
  if constexpr (kMode == 1) {
    for (int c = 0; c < P.n_classes; c++)
      block_reduce_store<double>(cls_dot[c], P.partial, c * gridDim.x + blockIdx.x);
    return;
  }
  if (P.partial) {
    block_reduce_store<double>(dot_re, P.partial, blockIdx.x);
    if (kC) block_reduce_store<double>(dot_im, P.partial, gridDim.x + blockIdx.x);
  }
}

template <typename V, bool kStage, int kMode = 0>
int launch_apply_t(const ApplyParams &P, int grid, cudaStream_t st) {
  auto k = apply_h_kernel<V, kStage, kMode>;
  if (P.smem_bytes > 48 * 1024)
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes));
  k<<<grid, 256, P.smem_bytes, st>>>(P);
  ED_CK(cudaGetLastError());
  return ED_OK;
}

__global__ void find_rep_kernel(const DevTables T, const DevIndex I, const uint64_t *states,
                                int64_t n, uint64_t *rep, int32_t *sym, int32_t *phase,
                                int32_t *stab, int64_t *index) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const RepOut R = find_rep(T, T.rep, T.sym_off, T.sym_list, T.dest, T.phase, states[i]);
    if (rep) rep[i] = R.rep;
    if (sym) sym[i] = R.g;
    if (phase) phase[i] = R.g >= 0 ? T.phase[R.g] : 0;
    if (stab) stab[i] = R.t;
    if (index) index[i] = (R.mixed || I.D == 0) ? -1 : lookup_index(I, R.rep);
  }
}

// number of exchange terms per product: every antiparallel bond, and those whose
// representative is a basis state
__global__ void count_terms_kernel(const DevTables T, const DevIndex I, const uint8_t *bond_pos,
                                   int n_bonds, unsigned long long *out) {
  unsigned long long nf = 0, no = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I.D;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t s = I.basis[i];
    for (int b = 0; b < n_bonds; b++) {
      const int pa = bond_pos[2 * b], pb = bond_pos[2 * b + 1];
      if ((((s >> pa) ^ (s >> pb)) & 1ULL) == 0) continue;
      nf++;
      const RepOut R = find_rep(T, T.rep, T.sym_off, T.sym_list, T.dest, T.phase,
                                s ^ ((1ULL << pa) | (1ULL << pb)));
      if (!R.mixed && lookup_index(I, R.rep) >= 0) no++;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    nf += __shfl_down_sync(0xFFFFFFFFu, nf, o);
    no += __shfl_down_sync(0xFFFFFFFFu, no, o);
  }
  if ((threadIdx.x & 31) == 0) { atomicAdd(out, nf); atomicAdd(out + 1, no); }
}

// ------------------------------ vector kernels -------------------------------------
template <typename V>
__global__ void dot_kernel(const V *x, const V *y, int64_t n, double *partial) {
  double re = 0, im = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (Vt<V>::cplx) {
      const V a = x[i], b = y[i];
      re += (double)a.x * b.x + (double)a.y * b.y;
      im += (double)a.x * b.y - (double)a.y * b.x;
    } else {
      re += (double)x[i] * (double)y[i];
    }
  }
  block_reduce_store<double>(re, partial, blockIdx.x);
  if (Vt<V>::cplx) block_reduce_store<double>(im, partial, gridDim.x + blockIdx.x);
}

// w <- w - a v - b vprev ; partial ||w||^2   (vprev may be null).  fp64 vectors in fp64;
// fp32 vectors in double-float (a and b split into two fp32 words each, exact products):
// with wlo (may be null) w enters as the pair (w, wlo) -- the product's value and its
// rounding remainder -- and leaves the same way, so that the update rounds nothing; the
// norm is that of the pair.  The fp64 pipe of this GPU is too slow for a pass of fp64
// arithmetic over the whole vector.
template <typename V>
__global__ void axpy_norm_kernel(V *w, const V *v, const V *vprev, double a, double b,
                                 int64_t n, double *partial, V *wlo) {
  using A = typename Vt<V>::A;
  constexpr bool kF = sizeof(A) == 4;
  double acc = 0;
  float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f, nh = 0.f, nl = 0.f;
  if constexpr (kF) {
    df_split(a, ah, al);
    df_split(b, bh, bl);
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (Vt<V>::cplx && kF) {
      // a and b are real (Hermitian tridiagonal)
      const V w0 = w[i], v0 = v[i];
      float rh = w0.x, rl = 0.f, ih = w0.y, il = 0.f;
      if (wlo) { const V l0 = wlo[i]; rl = l0.x; il = l0.y; }
      df_sub_scaled(rh, rl, ah, al, v0.x);
      df_sub_scaled(ih, il, ah, al, v0.y);
      if (vprev) {
        const V p0 = vprev[i];
        df_sub_scaled(rh, rl, bh, bl, p0.x);
        df_sub_scaled(ih, il, bh, bl, p0.y);
      }
      V o, r;
      df_store(rh, rl, o.x, r.x);
      df_store(ih, il, o.y, r.y);
      w[i] = o;
      if (wlo) wlo[i] = r; else { r.x = 0.f; r.y = 0.f; }
      df_add_sq(nh, nl, o.x, r.x);
      df_add_sq(nh, nl, o.y, r.y);
    } else if constexpr (kF) {
      float hi = w[i], lo = wlo ? wlo[i] : 0.f;
      df_sub_scaled(hi, lo, ah, al, v[i]);
      if (vprev) df_sub_scaled(hi, lo, bh, bl, vprev[i]);
      float o, r;
      df_store(hi, lo, o, r);
      w[i] = o;
      if (wlo) wlo[i] = r; else r = 0.f;
      df_add_sq(nh, nl, o, r);
    } else if constexpr (Vt<V>::cplx) {
      double wr = (double)w[i].x - a * (double)v[i].x;
      double wi = (double)w[i].y - a * (double)v[i].y;
      if (vprev) { wr -= b * (double)vprev[i].x; wi -= b * (double)vprev[i].y; }
      V o; o.x = (A)wr; o.y = (A)wi;
      w[i] = o;
      acc += (double)o.x * o.x + (double)o.y * o.y;
    } else {
      double t = (double)w[i] - a * (double)v[i];
      if (vprev) t -= b * (double)vprev[i];
      const A o = (A)t;
      w[i] = o;
      acc += (double)o * (double)o;
    }
  }
  if constexpr (kF) acc = df_value(nh, nl);
  block_reduce_store<double>(acc, partial, blockIdx.x);
}

// v <- s v; with vlo (fp32 vectors, may be null) v enters as the pair (v, vlo) and the
// product is rounded once
template <typename V>
__global__ void scale_kernel(V *v, double s, int64_t n, const V *vlo) {
  using A = typename Vt<V>::A;
  constexpr bool kF = sizeof(A) == 4;
  float sh = 0.f, sl = 0.f;
  if constexpr (kF) df_split(s, sh, sl);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (kF) {
      if (vlo) {
        if constexpr (Vt<V>::cplx) {
          const V a = v[i], l = vlo[i];
          float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
          df_sub_scaled(rh, rl, -sh, -sl, a.x);
          df_sub_scaled(rh, rl, -sh, -sl, l.x);
          df_sub_scaled(ih, il, -sh, -sl, a.y);
          df_sub_scaled(ih, il, -sh, -sl, l.y);
          V o; o.x = df_round(rh, rl); o.y = df_round(ih, il);
          v[i] = o;
        } else {
          float hi = 0.f, lo = 0.f;
          df_sub_scaled(hi, lo, -sh, -sl, v[i]);
          df_sub_scaled(hi, lo, -sh, -sl, vlo[i]);
          v[i] = df_round(hi, lo);
        }
        continue;
      }
    }
    if constexpr (Vt<V>::cplx) { V o = v[i]; o.x = (A)(o.x * s); o.y = (A)(o.y * s); v[i] = o; }
    else v[i] = (A)((double)v[i] * s);
  }
}

template <typename V>
__global__ void axpy_kernel(V *y, const V *x, double a, int64_t n) {
  using A = typename Vt<V>::A;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (Vt<V>::cplx) {
      V o = y[i]; o.x = (A)(o.x + a * x[i].x); o.y = (A)(o.y + a * x[i].y); y[i] = o;
    } else y[i] = (A)((double)y[i] + a * (double)x[i]);
  }
}

// start vector v_i = uniform[-1, 1) keyed by the basis state (real part; imaginary part
// from a second stream for complex types)
template <typename V>
__global__ void start_kernel(V *v, const uint64_t *basis, int64_t n, uint64_t seed) {
  using A = typename Vt<V>::A;
  const uint64_t off0 = (seed * 2 + 1) * 0x9E3779B97F4A7C15ULL;
  const uint64_t off1 = (seed * 2 + 2) * 0x9E3779B97F4A7C15ULL;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t s = basis[i];
    const double u0 = (double)(splitmix64_mix(s + off0) >> 11) * (1.0 / 9007199254740992.0);
    if constexpr (Vt<V>::cplx) {
      const double u1 = (double)(splitmix64_mix(s + off1) >> 11) * (1.0 / 9007199254740992.0);
      V o; o.x = (A)(2.0 * u0 - 1.0); o.y = (A)(2.0 * u1 - 1.0); v[i] = o;
    } else {
      v[i] = (A)(2.0 * u0 - 1.0);
    }
  }
}

int grid_for(const ed_basis *B, int64_t n, int per_sm) {
  int64_t g = (int64_t)B->sm_count * per_sm;
  int64_t need = (n + 255) / 256;
  if (need < g) g = need;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

// --------------------------------- launchers ---------------------------------------
static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

int ed_launch_apply(const ed_basis *B, const double *J, const double *Jz, const void *x,
                    void *y, int dtype, int64_t r0, int64_t r1, double *partial,
                    cudaStream_t st, int mode, void *ylo) {
  if (r1 <= r0) return ED_OK;
  {  // the specialised two-level kernels first; the generic kernel serves what they cannot
    bool done = false;
    const int rc = ed_launch_apply_fast(B, J, Jz, x, y, dtype, r0, r1, partial, st, mode, ylo, &done);
    if (rc != ED_ERR_UNSUPPORTED) {
      if (!rc && ylo && !done)
        ED_CK(cudaMemsetAsync(ylo, 0, (size_t)(r1 - r0) * (dtype == ED_C64 ? 8 : 4), st));
      return rc;
    }
  }
  if (ylo) ED_CK(cudaMemsetAsync(ylo, 0, (size_t)(r1 - r0) * (dtype == ED_C64 ? 8 : 4), st));
  ApplyParams P{};
  P.T = B->T;
  P.I = B->I;
  P.n_classes = B->n_classes;
  for (int c = 0; c <= B->n_classes; c++) P.cls_off[c] = B->cls_off[c];
  for (int c = 0; c < B->n_classes; c++) {
    P.jh[c] = 0.5 * J[c];
    P.jzq[c] = 0.25 * J[c] * Jz[c];
  }
  P.bond_pos = B->d_bond_pos;
  P.sqrt_tab = B->d_sqrt;
  P.rsqrt_tab = B->d_rsqrt;
  const bool cplx = (dtype == ED_C128 || dtype == ED_C64);
  P.cs = cplx ? B->d_cs : nullptr;
  P.x = x;
  P.y = y;
  P.r0 = r0;
  P.r1 = r1;
  P.partial = partial;
  // shared-memory layout
  const size_t nn = (size_t)1 << B->n;
  const size_t abytes = (dtype == ED_F64 || dtype == ED_C128) ? 8 : 4;
  size_t off = 0;
  const size_t tab_bytes = align16((size_t)B->nsub * nn * 4) +
                           align16((size_t)B->nsub * (nn + 1) * 4) +
                           align16((size_t)B->nsym * 4) + align16(B->sym_list_len * 2) +
                           align16((size_t)B->nsym * B->nsub);
  const size_t rest = align16((size_t)B->n_bonds * 2) + align16((size_t)(B->nsym + 1) * 2 * abytes) +
                      align16((size_t)B->denom * 2 * abytes);
  const size_t kMaxSmem = 200 * 1024;
  // a one-sublattice split reads the whole table from global memory and has no
  // Rep/Sym/dest tables to stage
  P.stage_tables = (!B->T.full && tab_bytes + rest <= kMaxSmem) ? 1 : 0;
  P.sym_list_bytes = (uint32_t)(B->sym_list_len * 2);
  if (P.stage_tables) {
    P.off_rep = (uint32_t)off; off += align16((size_t)B->nsub * nn * 4);
    P.off_symoff = (uint32_t)off; off += align16((size_t)B->nsub * (nn + 1) * 4);
    P.off_phase = (uint32_t)off; off += align16((size_t)B->nsym * 4);
    P.off_symlist = (uint32_t)off; off += align16(B->sym_list_len * 2);
    P.off_dest = (uint32_t)off; off += align16((size_t)B->nsym * B->nsub);
  } else {
    P.off_symlist = P.off_dest = 0;
  }
  P.off_bond = (uint32_t)off; off += align16((size_t)B->n_bonds * 2);
  P.off_sqrt = (uint32_t)off; off += align16((size_t)(B->nsym + 1) * 2 * abytes);
  P.off_cs = (uint32_t)off; off += align16((size_t)B->denom * 2 * abytes);
  P.smem_bytes = (uint32_t)off;
  // fixed grid: a whole number of CTAs per SM, grid-stride over rows
  const int grid = grid_for(B, r1 - r0, 8);
  if (partial && grid > B->n_partial / 2) return ed_fail(ED_ERR_INVALID, "partial buffer too small");
  B->last_apply_grid = grid;
  const bool sg = P.stage_tables != 0;
  if (mode == 1) {
    if (!partial || B->n_classes * grid > B->n_partial) return ed_fail(ED_ERR_INVALID, "partial buffer too small");
    switch (dtype) {
      case ED_F64: return sg ? launch_apply_t<double, true, 1>(P, grid, st) : launch_apply_t<double, false, 1>(P, grid, st);
      case ED_F32: return sg ? launch_apply_t<float, true, 1>(P, grid, st) : launch_apply_t<float, false, 1>(P, grid, st);
      case ED_C128: return sg ? launch_apply_t<double2, true, 1>(P, grid, st) : launch_apply_t<double2, false, 1>(P, grid, st);
      case ED_C64: return sg ? launch_apply_t<float2, true, 1>(P, grid, st) : launch_apply_t<float2, false, 1>(P, grid, st);
    }
    return ed_fail(ED_ERR_INVALID, "unknown dtype");
  }
  switch (dtype) {
    case ED_F64: return sg ? launch_apply_t<double, true>(P, grid, st) : launch_apply_t<double, false>(P, grid, st);
    case ED_F32: return sg ? launch_apply_t<float, true>(P, grid, st) : launch_apply_t<float, false>(P, grid, st);
    case ED_C128: return sg ? launch_apply_t<double2, true>(P, grid, st) : launch_apply_t<double2, false>(P, grid, st);
    case ED_C64: return sg ? launch_apply_t<float2, true>(P, grid, st) : launch_apply_t<float2, false>(P, grid, st);
  }
  return ed_fail(ED_ERR_INVALID, "unknown dtype");
}

int ed_apply_grid(const ed_basis *B, int64_t rows) { return grid_for(B, rows, 8); }

int ed_launch_find_rep(const ed_basis *B, const uint64_t *states, int64_t n, uint64_t *rep,
                       int32_t *sym, int32_t *phase, int32_t *stab, int64_t *index,
                       cudaStream_t st) {
  if (n <= 0) return ED_OK;
  const int grid = grid_for(B, n, 8);
  find_rep_kernel<<<grid, 256, 0, st>>>(B->T, B->I, states, n, rep, sym, phase, stab, index);
  ED_CK(cudaGetLastError());
  return ED_OK;
}

int ed_launch_count(const ed_basis *B, unsigned long long *d_out, cudaStream_t st) {
  if (B->D == 0) return ED_OK;
  count_terms_kernel<<<grid_for(B, B->D, 8), 256, 0, st>>>(B->T, B->I, B->d_bond_pos,
                                                            B->n_bonds, d_out);
  ED_CK(cudaGetLastError());
  return ED_OK;
}

#define ED_DISPATCH(dtype, CALL)                                 \
  switch (dtype) {                                               \
    case ED_F64: { using V = double; CALL; break; }              \
    case ED_F32: { using V = float; CALL; break; }               \
    case ED_C128: { using V = double2; CALL; break; }            \
    case ED_C64: { using V = float2; CALL; break; }              \
    default: return ed_fail(ED_ERR_INVALID, "unknown dtype");    \
  }

int ed_launch_dot(const ed_basis *B, const void *x, const void *y, int dtype, double *partial,
                  int nblk, cudaStream_t st) {
  ED_DISPATCH(dtype, (dot_kernel<V><<<nblk, 256, 0, st>>>((const V *)x, (const V *)y, B->D, partial)));
  ED_CK(cudaGetLastError());
  return ED_OK;
}

int ed_launch_axpy_norm(const ed_basis *B, void *w, const void *v, const void *vprev, double a,
                        double b, int dtype, double *partial, int nblk, cudaStream_t st,
                        void *wlo) {
  ED_DISPATCH(dtype, (axpy_norm_kernel<V><<<nblk, 256, 0, st>>>((V *)w, (const V *)v,
                                                                (const V *)vprev, a, b, B->D,
                                                                partial, (V *)wlo)));
  ED_CK(cudaGetLastError());
  return ED_OK;
}

int ed_launch_scale(const ed_basis *B, void *v, double s, int dtype, cudaStream_t st,
                    const void *vlo) {
  const int grid = grid_for(B, B->D, 8);
  ED_DISPATCH(dtype, (scale_kernel<V><<<grid, 256, 0, st>>>((V *)v, s, B->D, (const V *)vlo)));
  ED_CK(cudaGetLastError());
  return ED_OK;
}

int ed_launch_axpy(const ed_basis *B, void *y, const void *x, double a, int dtype,
                   cudaStream_t st) {
  const int grid = grid_for(B, B->D, 8);
  ED_DISPATCH(dtype, (axpy_kernel<V><<<grid, 256, 0, st>>>((V *)y, (const V *)x, a, B->D)));
  ED_CK(cudaGetLastError());
  return ED_OK;
}

int ed_launch_start(const ed_basis *B, void *v, uint64_t seed, int dtype, cudaStream_t st) {
  const int grid = grid_for(B, B->D, 8);
  ED_DISPATCH(dtype, (start_kernel<V><<<grid, 256, 0, st>>>((V *)v, B->d_basis, B->D, seed)));
  ED_CK(cudaGetLastError());
  return ED_OK;
}

int ed_launch_copy(const ed_basis *B, void *dst, const void *src, int dtype, cudaStream_t st) {
  const size_t es = (dtype == ED_F64) ? 8 : (dtype == ED_F32) ? 4 : (dtype == ED_C128) ? 16 : 8;
  ED_CK(cudaMemcpyAsync(dst, src, es * (size_t)B->D, cudaMemcpyDeviceToDevice, st));
  return ED_OK;
}
