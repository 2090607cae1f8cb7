// apply_fast.cu -- the row-pull product y = H x with a two-level representative search.
//
// Two-level search.  In Alg. 2 of arXiv:1804.05028 the candidates of a minimal block Y
// are Sym_Y(s_Y) = K_R h: the coset of the stabiliser K_R = {k in G_0 : k R = R} of
// R = MinRep through the first element h.  Hence min over Sym_Y of g s =
// min over k in K_R of k (h s), and that inner minimum is again a sublattice-coding
// problem (Eqs. 8-10) for the group K_R acting on blocks 1.., with block 1 in the role
// of block 0.  Level 1 looks up (Rep_X, h) per block, applies h once; level 2 looks up
// (Rep^R_X, Sym^R_X) of the images and scans only those candidates.  The candidate
// scans shrink from ~20 to ~3 entries on the 6x6 C4v sector.  Every minimiser of the
// orbit is still visited (all of them lie in the scanned sets), so |Stab| and the
// character check are exact, as in the single-level search.
//
// Two kernels share the search:
//   apply_tile_kernel  the product: a warp owns 32 consecutive rows and resolves their
//                      exchange terms 32 at a time from term lists in shared memory (see
//                      the comment above tile_round); the index of a representative is
//                      one ranked Limits record (first index + popcount of a bitmap).
//   apply_two_kernel   one thread per row, one term at a time; it serves the
//                      class-resolved expectations <x|H_c|x> (the adjoint).
// Antiparallel bonds come as 32-bit masks (one coupling class per word), from per-nibble
// XOR tables; each exchange flips one bit in the block of each end.  Tables: Rep_X /
// first of Sym_X, stabiliser ids, the level-2 tables (when they fit), prefix ranks,
// bonds and weights in shared memory; SymmetryAction_X in global memory (L1/L2), and the
// level-2 tables there too when they do not fit.  Each y_i is written once; no atomics.
#include "sced_internal.cuh"
#include "dfloat.cuh"
#include <algorithm>
#include <cstdlib>
#include <type_traits>

namespace {

template <typename V> struct Vf;
template <> struct Vf<double> { using A = double; static constexpr bool cplx = false; };
template <> struct Vf<float> { using A = float; static constexpr bool cplx = false; };
template <> struct Vf<double2> { using A = double; static constexpr bool cplx = true; };
template <> struct Vf<float2> { using A = float; static constexpr bool cplx = true; };

struct TwoParams {
  int N, n, nsym, denom;
  int n_classes;
  int cls_word[ED_MAXCLS + 1];   // words [cls_word[c], cls_word[c+1]) hold class c
  int nb_cls[ED_MAXCLS];         // real bonds per class (diagonal term)
  double jh[ED_MAXCLS], jzq[ED_MAXCLS];
  const uint32_t *e1, *e2, *off2, *top_rank, *limits;
  const uint16_t *list2, *act;
  const uint8_t *rid, *dest, *src, *bond_pos;
  const uint32_t *bond_blk;      // per padded bond: block of each end, bit inside the block
  const int32_t *phase;
  const double *sqrt_tab, *rsqrt_tab, *cs;
  const uint64_t *basis;
  const uint16_t *stab;
  const void *postfix;
  int r_bits, q_bits, post_bits, post_bytes;
  int L;                         // bits below the top block: (NSUB - 1) n <= 32
  int id_g;                      // index of the identity element
  uint32_t qmask, pmask;
  int64_t D;
  const void *x;
  void *y;
  void *ylo;                     // fp32 vectors: optional low words of y (double-float y)
  int64_t r0, r1;
  double *partial;
  uint32_t n_e1, n_e2, n_rid, n_dest, n_bond, n_top, n_sq, n_cs;
  uint32_t off_bblk, off_e2, off_e1, off_rid, off_dest, off_src, off_phase, off_bond, off_top, off_sq, off_cs,
      smem_bytes;
  // term-parallel kernel: fp32 weight / character tables and the per-warp row states and
  // term lists (0 when the layout has no tile region)
  uint32_t off_sqf, off_csf, off_tile, tile_warps;
  const uint32_t *nib;           // antiparallel masks by nibbles, [word][n_nib][16]
  uint32_t n_nib, off_nib;
  const uint4 *rlim;             // ranked Limits records (null: search the buckets)
  int rq_bits, rpost_bits;
  uint32_t rqmask, rpmask;
};

struct Sm2 {
  const uint32_t *e2;    // level-2 tables (shared-memory copy), when staged
  const uint32_t *bblk;
  const uint32_t *e1;
  const uint16_t *top;   // prefix rank (< 4096), 0xFFFF where no representative has that top
  const uint8_t *rid, *dest, *src, *bond;
  const int32_t *phase;
};

// per-warp shared memory of the term-parallel kernel: 32 row states, 32 row accumulators
// (real and imaginary parts, up to fp64), then a list of at most 32 x 16 terms of 16 bits
constexpr uint32_t kTileWarpBytes = 32 * 8 + 32 * 16 + 32 * 16 * 2;

struct Rep2 {
  uint32_t minrep;   // top block of the representative
  uint32_t low;      // the lower NSUB-1 blocks, block 1 most significant
  int t, ph, mixed;
};

template <typename T>
__device__ __forceinline__ void cp(unsigned char *sm, uint32_t off, const T *g, uint32_t n) {
  T *d = reinterpret_cast<T *>(sm + off);
  for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) d[k] = g[k];
}

// g s restricted to block X: an n-bit value on block dest(g, X) (SymmetryAction_X, Eq. 11).
// The identity leaves every block in place, so its lookups are skipped: level 1 meets it
// whenever the minimal block is already its own Rep (often, as the exchanged state
// differs from a representative in two sites), level 2 whenever the images are already
// minimal for K_R.
// The table (|G| 2^n entries per sublattice, about 1 MB for 4 x 2^9 x 144) is read at
// random by every thread: the load asks L1 to keep its lines over the streamed data.
__device__ __forceinline__ uint32_t act(const TwoParams &P, int X, uint32_t sub, int g) {
  if (g == P.id_g) return sub;
  const unsigned short *a = P.act + (((uint32_t)X << P.n) | sub) * (uint32_t)P.nsym + (uint32_t)g;
  unsigned short r;
  asm volatile("ld.global.nc.L1::evict_last.u16 %0, [%1];" : "=h"(r) : "l"(a));
  return r;
}

// x_j of a found representative: a gather with no reuse to speak of, kept out of L1.
template <typename V>
__device__ __forceinline__ V gather_x(const V *x, int64_t j) {
  if constexpr (std::is_same<V, float>::value) {
    float f;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(f) : "l"(x + j));
    return f;
  } else if constexpr (std::is_same<V, double>::value) {
    double f;
    asm volatile("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(f) : "l"(x + j));
    return f;
  } else {
    return x[j];
  }
}

__device__ __forceinline__ void consider(Rep2 &o, uint32_t low, int ph) {
  if (low < o.low) { o.low = low; o.t = 1; o.ph = ph; o.mixed = 0; }
  else if (low == o.low) { o.t++; o.mixed |= (ph != o.ph); }
}

template <int NSUB>
__device__ __forceinline__ uint32_t pick(const uint32_t (&a)[NSUB], int i) {
  uint32_t v = a[0];
#pragma unroll
  for (int k = 1; k < NSUB; k++) v = (i == k) ? a[k] : v;
  return v;
}

// Two-level search (see the file comment) on a configuration given block by block
// (sub[X] = the n-bit substate of block X).  Candidates share the top block MinRep, so
// they are compared on the lower NSUB-1 blocks only, packed in 32 bits (block 1 most
// significant); the result is rep = MinRep << L | low with L = (NSUB-1) n.  Loops run
// over bitmasks of the minimal blocks so that one copy of each step is emitted.
template <int NSUB, bool kE2>
__device__ __forceinline__ Rep2 find_rep_blocks(const Sm2 &S, const TwoParams &P,
                                                const uint32_t (&sub)[NSUB]) {
  const int n = P.n;
  uint32_t e[NSUB];
  uint32_t minrep = 0xFFFFFFFFu, ymask = 0;
#pragma unroll
  for (int X = 0; X < NSUB; X++) {
    e[X] = S.e1[(X << n) | sub[X]];
    const uint32_t r = e[X] & 0xFFFu;
    if (r < minrep) { minrep = r; ymask = 1u << X; }
    else if (r == minrep) ymask |= 1u << X;
  }
  Rep2 o;
  o.minrep = minrep; o.low = 0xFFFFFFFFu; o.t = 0; o.ph = 0; o.mixed = 0;
  const int rid = S.rid[minrep];
  while (ymask) {
    const int Y = __ffs(ymask) - 1;
    ymask &= ymask - 1;
    const int h = (pick<NSUB>(e, Y) >> 12) & 0xFFF;
    const int phh = S.phase[h];
    uint32_t tau[NSUB];   // tau[d] = block d of h s
    tau[0] = minrep;
#pragma unroll
    for (int d = 1; d < NSUB; d++) {
      const int X = S.src[h * NSUB + d];
      tau[d] = act(P, X, pick<NSUB>(sub, X), h);
    }
    if (rid == 0xFF) {   // K_R = {e}: h is the only candidate of this block
      uint32_t low = 0;
#pragma unroll
      for (int d = 1; d < NSUB; d++) low |= tau[d] << ((NSUB - 1 - d) * n);
      consider(o, low, phh);
      continue;
    }
    const uint32_t rbase = (uint32_t)rid * (NSUB - 1);
    uint32_t f[NSUB];
    uint32_t m2 = 0xFFFFFFFFu, dmask = 0;
#pragma unroll
    for (int d = 1; d < NSUB; d++) {
      const uint32_t ei = ((rbase + d - 1) << n) | tau[d];
      f[d] = kE2 ? S.e2[ei] : __ldg(P.e2 + ei);
      const uint32_t r2 = f[d] & 0xFFFu;
      if (r2 < m2) { m2 = r2; dmask = 1u << d; }
      else if (r2 == m2) dmask |= 1u << d;
    }
    f[0] = 0;
    const uint32_t low2 = m2 << ((NSUB - 2) * n);
    while (dmask) {
      const int d2 = __ffs(dmask) - 1;
      dmask &= dmask - 1;
      const uint32_t fd = pick<NSUB>(f, d2);
      const int cnt = fd >> 24;
      const uint32_t base =
          cnt > 1 ? __ldg(P.off2 + (((rbase + d2 - 1) << n) | pick<NSUB>(tau, d2))) : 0u;
      for (int c = 0; c < cnt; c++) {
        const int k = c == 0 ? (int)((fd >> 12) & 0xFFF) : (int)__ldg(P.list2 + base + c);
        uint32_t low = low2;
#pragma unroll
        for (int d = 1; d < NSUB; d++) {
          if (d == d2) continue;
          const int dd = S.dest[k * NSUB + d];
          low |= act(P, d, tau[d], k) << ((NSUB - 1 - dd) * n);
        }
        int ph = phh + S.phase[k];
        if (ph >= P.denom) ph -= P.denom;
        consider(o, low, ph);
      }
    }
  }
  return o;
}

__device__ __forceinline__ uint32_t ld_post(const TwoParams &P, uint32_t i) {
  switch (P.post_bytes) {
    case 1: return __ldg(reinterpret_cast<const uint8_t *>(P.postfix) + i);
    case 2: return __ldg(reinterpret_cast<const uint16_t *>(P.postfix) + i);
  }
  return __ldg(reinterpret_cast<const uint32_t *>(P.postfix) + i);
}

__device__ __forceinline__ void two_sum(float &hi, float &lo, float v) {
  const float s = hi + v;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (v - bb);
  hi = s;
}

__device__ __forceinline__ Sm2 stage_two(const TwoParams &P, unsigned char *sm, bool cplx,
                                         bool e2) {
  cp(sm, P.off_e1, P.e1, P.n_e1);
  cp(sm, P.off_rid, P.rid, P.n_rid);
  cp(sm, P.off_dest, P.dest, P.n_dest);
  cp(sm, P.off_src, P.src, P.n_dest);
  cp(sm, P.off_phase, P.phase, (uint32_t)P.nsym);
  cp(sm, P.off_bond, P.bond_pos, P.n_bond);
  cp(sm, P.off_bblk, P.bond_blk, P.n_bond / 2);
  {   // the prefix rank staged as 16 bits: ranks are below 2^12
    uint16_t *d = reinterpret_cast<uint16_t *>(sm + P.off_top);
    for (uint32_t k = threadIdx.x; k < P.n_top; k += blockDim.x) {
      const uint32_t v = P.top_rank[k];
      d[k] = v == ED_NO_RANK ? (uint16_t)0xFFFFu : (uint16_t)v;
    }
  }
  cp(sm, P.off_sq, P.sqrt_tab, P.n_sq);
  cp(sm, P.off_sq + 8 * P.n_sq, P.rsqrt_tab, P.n_sq);
  if (cplx) cp(sm, P.off_cs, P.cs, P.n_cs);
  if (e2) cp(sm, P.off_e2, P.e2, P.n_e2);
  __syncthreads();
  Sm2 S;
  S.e2 = reinterpret_cast<const uint32_t *>(sm + P.off_e2);
  S.bblk = reinterpret_cast<const uint32_t *>(sm + P.off_bblk);
  S.e1 = reinterpret_cast<const uint32_t *>(sm + P.off_e1);
  S.rid = sm + P.off_rid;
  S.dest = sm + P.off_dest;
  S.src = sm + P.off_src;
  S.phase = reinterpret_cast<const int32_t *>(sm + P.off_phase);
  S.bond = sm + P.off_bond;
  S.top = reinterpret_cast<const uint16_t *>(sm + P.off_top);
  return S;
}

// Index of the representative MinRep << L | low in Basis: prefix rank (shared memory),
// Limits bucket, binary search of the postfixes in the bucket (Sec. IV); -1 when absent.
// The fast path has N - r_bits <= 32, so the bucket key's raw bits and the postfix are
// taken from the low 32 bits of the state.
__device__ __forceinline__ int64_t lookup_ranked(const Sm2 &S, const TwoParams &P,
                                                 uint32_t minrep, uint32_t low);

__device__ __forceinline__ int64_t lookup_two(const Sm2 &S, const TwoParams &P, uint32_t minrep,
                                              uint32_t low) {
  if (P.rlim) return lookup_ranked(S, P, minrep, low);
  const uint64_t r = ((uint64_t)minrep << P.L) | low;
  const uint32_t rk = S.top[(uint32_t)(r >> (P.N - P.r_bits))];
  if (rk == 0xFFFFu) return -1;
  const uint32_t key = (rk << P.q_bits) | ((uint32_t)(r >> P.post_bits) & P.qmask);
  uint32_t lo = __ldg(P.limits + key), hi = __ldg(P.limits + key + 1);
  const uint32_t tg = (uint32_t)r & P.pmask;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t pv = ld_post(P, mid);
    if (pv < tg) lo = mid + 1;
    else if (pv > tg) hi = mid;
    else return mid;
  }
  return -1;
}

// Index of the representative through the ranked Limits: one 16-byte record per key
// {first index of the bucket, 0, bitmap of the postfixes present}; the state is present
// when its postfix bit is set, and its index is the first index plus the number of
// present postfixes below it.  One dependent global load instead of a binary search.
__device__ __forceinline__ int64_t lookup_ranked(const Sm2 &S, const TwoParams &P,
                                                 uint32_t minrep, uint32_t low) {
  const uint64_t r = ((uint64_t)minrep << P.L) | low;
  const uint32_t rk = S.top[(uint32_t)(r >> (P.N - P.r_bits))];
  if (rk == 0xFFFFu) return -1;
  const uint32_t key = (rk << P.rq_bits) | ((uint32_t)(r >> P.rpost_bits) & P.rqmask);
  uint4 rec;
  asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(rec.x), "=r"(rec.y), "=r"(rec.z), "=r"(rec.w) : "l"(P.rlim + key));
  const uint32_t pf = (uint32_t)r & P.rpmask;
  const uint64_t bits = ((uint64_t)rec.w << 32) | rec.z;
  if (!((bits >> pf) & 1ULL)) return -1;
  return (int64_t)rec.x + __popcll(bits & ((1ULL << pf) - 1ULL));
}

// Kernel without level-2 tables in shared memory: two 768-thread blocks per SM, i.e. 48
// warps at 40 registers.  48 warps hide more of the dependent table loads than 32 at 64
// registers; and two blocks stage the shared tables twice where three 512-thread blocks
// stage them three times, which leaves L1 more room for the SymmetryAction and level-2
// lines (3-4% faster; six 256-thread blocks were 29% slower).
constexpr int kThreads = 768;
constexpr int kMinBlocks = 2;

// kMode 0: y = H x (and optional <x, y> partials); kMode 1: per coupling class the
// partial sums of Re <x | H_c x> with unit exchange, into partial[c * grid + block].
template <typename V, int NSUB, bool kE2, int kMode>
__global__ void __launch_bounds__(kE2 ? 1024 : kThreads, kE2 ? 1 : kMinBlocks) apply_two_kernel(const TwoParams P) {
  using A = typename Vf<V>::A;
  constexpr bool kC = Vf<V>::cplx;
  constexpr bool kF32 = sizeof(A) == 4;
  extern __shared__ __align__(16) unsigned char sm[];
  const Sm2 S = stage_two(P, sm, kC, kE2);
  const double *sqd = reinterpret_cast<const double *>(sm + P.off_sq);
  const double *rsd = sqd + P.n_sq;
  const double *csd = reinterpret_cast<const double *>(sm + P.off_cs);
  const V *x = reinterpret_cast<const V *>(P.x);
  V *y = reinterpret_cast<V *>(P.y);
  const int N = P.N, n = P.n;
  const uint32_t bmask = (1u << n) - 1u;

  double dot_re = 0.0, dot_im = 0.0;
  double cls_dot[kMode == 1 ? ED_MAXCLS : 1];
  for (int c = 0; c < (kMode == 1 ? ED_MAXCLS : 1); c++) cls_dot[c] = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = P.r0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.r1; i += stride) {
    // the row's own state, stabiliser order and y_i are touched once: streamed (evict
    // first) so that they do not push the gathered x out of L2
    const uint64_t s = __ldcs(reinterpret_cast<const unsigned long long *>(P.basis) + i);
    const int ti = __ldcs(P.stab + i);
    uint32_t sub[NSUB];
#pragma unroll
    for (int X = 0; X < NSUB; X++) sub[X] = (uint32_t)(s >> (N - (X + 1) * n)) & bmask;
    double row_re = 0.0, row_im = 0.0, diag = 0.0;
    for (int c = 0; c < P.n_classes; c++) {
      A acc_re = 0, acc_im = 0;
      float lo_re = 0.f;   // compensation (fp32 real vectors)
      int nanti = 0;
      for (int wd = P.cls_word[c]; wd < P.cls_word[c + 1]; wd++) {
        const uint8_t *bp = S.bond + wd * 64;
        uint32_t m = 0;
#pragma unroll 8
        for (int k = 0; k < 32; k++)
          m |= (uint32_t)(((s >> bp[2 * k]) ^ (s >> bp[2 * k + 1])) & 1ULL) << k;
        nanti += __popc(m);
        while (m) {
          const int k = __ffs(m) - 1;
          m &= m - 1;
          // the exchanged configuration, block by block: one bit flips in the block of
          // each end of the bond
          const uint32_t bi = S.bblk[wd * 32 + k];
          const int xa = bi & 15, xb = (bi >> 4) & 15;
          const uint32_t fa = 1u << ((bi >> 8) & 255), fb = 1u << (bi >> 16);
          uint32_t s2[NSUB];
#pragma unroll
          for (int X = 0; X < NSUB; X++) s2[X] = sub[X] ^ (X == xa ? fa : 0u) ^ (X == xb ? fb : 0u);
          const Rep2 R = find_rep_blocks<NSUB, kE2>(S, P, s2);
          if (R.mixed) continue;
          const int64_t j = lookup_two(S, P, R.minrep, R.low);
          if (j < 0) continue;
          const V xj = gather_x(x, j);
          const int t = R.t, ph = R.ph;
          if constexpr (!kC) {
            if constexpr (kF32) {
              if (t == 1) {
                two_sum(acc_re, lo_re, ph == 0 ? xj : -xj);
              } else {
                const double w = sqd[t];
                const float wh = (float)w, wl = (float)(w - (double)wh);
                const float p = wh * xj;
                const float pe = fmaf(wh, xj, -p) + wl * xj;
                two_sum(acc_re, lo_re, ph == 0 ? p : -p);
                lo_re += ph == 0 ? pe : -pe;
              }
            } else {
              const double v = (t == 1) ? (double)xj : sqd[t] * (double)xj;
              acc_re += ph == 0 ? v : -v;
            }
          } else {
            const A wgt = (A)sqd[t];
            const A cr = (A)csd[2 * ph] * wgt, ci = (A)csd[2 * ph + 1] * wgt;
            acc_re += cr * xj.x - ci * xj.y;
            acc_im += cr * xj.y + ci * xj.x;
          }
        }
      }
      const double dg = P.jzq[c] * (double)(P.nb_cls[c] - 2 * nanti);
      diag += dg;
      row_re += P.jh[c] * ((double)acc_re + (double)lo_re);
      if (kC) row_im += P.jh[c] * (double)acc_im;
      if constexpr (kMode == 1) {
        if constexpr (!kC) {
          const double xv = (double)x[i];
          cls_dot[c] += dg * xv * xv + P.jh[c] * rsd[ti] * xv * ((double)acc_re + (double)lo_re);
        } else {
          const V xv = x[i];
          cls_dot[c] += dg * ((double)xv.x * xv.x + (double)xv.y * xv.y) +
                        P.jh[c] * rsd[ti] * ((double)xv.x * acc_re + (double)xv.y * acc_im);
        }
      }
    }
    if constexpr (kMode == 1) continue;
    const double rs = rsd[ti];
    if constexpr (!kC) {
      const double xi = (double)x[i];
      const A yi = (A)(diag * xi + row_re * rs);
      __stcs(y + (i - P.r0), yi);
      if (P.partial) dot_re += xi * (double)yi;
    } else {
      const V xv = x[i];
      V yv;
      yv.x = (A)(diag * (double)xv.x + row_re * rs);
      yv.y = (A)(diag * (double)xv.y + row_im * rs);
      y[i - P.r0] = yv;
      if (P.partial) {
        dot_re += (double)xv.x * yv.x + (double)xv.y * yv.y;
        dot_im += (double)xv.x * yv.y - (double)xv.y * yv.x;
      }
    }
  }
  if (P.partial) {
    __shared__ double red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nparts = kMode == 1 ? P.n_classes : (kC ? 2 : 1);
    for (int part = 0; part < nparts; part++) {
      double d = kMode == 1 ? cls_dot[part] : (part ? dot_im : dot_re);
      for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
      __syncthreads();
      if (lane == 0) red[wid] = d;
      __syncthreads();
      if (wid == 0) {
        d = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xFFFFFFFFu, d, o);
        if (lane == 0) P.partial[part * gridDim.x + blockIdx.x] = d;
      }
    }
  }
}

constexpr int kTileChunk = 16;
constexpr int kTileThreads = 768;      // level-2 tables in global memory: 2 blocks per SM
constexpr int kTileMinBlocks = 2;
constexpr int kTileThreadsE2 = 1024;   // level-2 tables staged: 1 block per SM

// The common cases of the two-level search, without loops: one minimal block at level 1
// and one or two candidates at level 2 (a Sym^R list of one or two elements; two equal
// images are a stabiliser of order 2, whose characters must agree).  Returns false,
// leaving R unset, when the term needs the general search (several minimal blocks,
// several level-2 minimal blocks, or a longer Sym^R list).
template <int NSUB, bool kE2>
__device__ __forceinline__ bool find_rep_simple(const Sm2 &S, const TwoParams &P,
                                                const uint32_t (&sub)[NSUB], Rep2 &R) {
  const int n = P.n;
  // level 1: only the entry of the minimal block is kept (one minimal block is the case
  // handled here)
  uint32_t minrep = 0xFFFFFFFFu, ymask = 0, eY = 0;
#pragma unroll
  for (int X = 0; X < NSUB; X++) {
    const uint32_t ex = S.e1[(X << n) | sub[X]];
    const uint32_t r = ex & 0xFFFu;
    if (r < minrep) { minrep = r; ymask = 1u << X; eY = ex; }
    else if (r == minrep) ymask |= 1u << X;
  }
  if (ymask & (ymask - 1)) return false;
  const int h = (eY >> 12) & 0xFFF;
  uint32_t tau[NSUB];
  tau[0] = minrep;
#pragma unroll
  for (int d = 1; d < NSUB; d++) {
    const int X = S.src[h * NSUB + d];
    tau[d] = act(P, X, pick<NSUB>(sub, X), h);
  }
  const int phh = S.phase[h];
  R.minrep = minrep;
  R.t = 1;
  R.mixed = 0;
  const int rid = S.rid[minrep];
  if (rid == 0xFF) {   // K_R = {e}: h is the only candidate
    uint32_t low = 0;
#pragma unroll
    for (int d = 1; d < NSUB; d++) low |= tau[d] << ((NSUB - 1 - d) * n);
    R.low = low;
    R.ph = phh;
    return true;
  }
  // level 2: again only the entry of the minimal block is kept
  const uint32_t rbase = (uint32_t)rid * (NSUB - 1);
  uint32_t m2 = 0xFFFFFFFFu, dmask = 0, fd = 0;
  int d2 = 1;
#pragma unroll
  for (int d = 1; d < NSUB; d++) {
    const uint32_t ei = ((rbase + d - 1) << n) | tau[d];
    const uint32_t fv = kE2 ? S.e2[ei] : __ldg(P.e2 + ei);
    const uint32_t r2 = fv & 0xFFFu;
    if (r2 < m2) { m2 = r2; dmask = 1u << d; fd = fv; d2 = d; }
    else if (r2 == m2) dmask |= 1u << d;
  }
  const uint32_t cnt = fd >> 24;
  if ((dmask & (dmask - 1)) || cnt > 2) return false;
  const int k = (int)((fd >> 12) & 0xFFF);
  uint32_t low = m2 << ((NSUB - 2) * n);
  const uint32_t low2 = low;
#pragma unroll
  for (int d = 1; d < NSUB; d++) {
    if (d == d2) continue;
    const int dd = S.dest[k * NSUB + d];
    low |= act(P, d, tau[d], k) << ((NSUB - 1 - dd) * n);
  }
  int ph = phh + S.phase[k];
  if (ph >= P.denom) ph -= P.denom;
  R.low = low;
  R.ph = ph;
  if (cnt == 2) {   // Sym^R holds a second element: compare its image, count a tie
    const uint32_t base = __ldg(P.off2 + (((rbase + d2 - 1) << n) | pick<NSUB>(tau, d2)));
    const int k2 = (int)__ldg(P.list2 + base + 1);
    uint32_t lowb = low2;
#pragma unroll
    for (int d = 1; d < NSUB; d++) {
      if (d == d2) continue;
      const int dd = S.dest[k2 * NSUB + d];
      lowb |= act(P, d, tau[d], k2) << ((NSUB - 1 - dd) * n);
    }
    int phb = phh + S.phase[k2];
    if (phb >= P.denom) phb -= P.denom;
    if (lowb < low) {
      R.low = lowb;
      R.ph = phb;
    } else if (lowb == low) {
      R.t = 2;
      R.mixed = phb != ph;
    }
  }
  return true;
}

// ---------------------------------------------------------------------------------------
// Term-parallel product (fp32 and complex fp32 vectors).
//
// A warp owns a tile of 32 consecutive rows (lane l owns row l of the tile).  The bonds
// are taken in chunks of 16 (half a padded word, one coupling class); for each chunk
// every lane appends its row's antiparallel bonds to a warp-private list in shared
// memory, in row order, and the warp then works through the list 32 terms at a time:
// lane l takes term base + l whatever row it belongs to.  Rows of unequal length no
// longer leave lanes idle (a row-per-lane loop runs as long as the longest row of the
// warp).
//
// A term whose search needs more than the common case (several minimal blocks or
// several level-2 candidates, see find_rep_simple) is not resolved in its round: it is
// appended to a second list (written over the part of the chunk list already consumed)
// and the deferred terms are resolved together, 32 at a time, by the general search.
// The rare long searches then run with every lane busy instead of stalling 31 lanes of
// each round.  Both lists stay in row order.
//
// A term's value goes back to its row by a segmented inclusive scan over the 32 lanes
// (rows are non-decreasing along a list, so equal neighbouring rows form one segment);
// the lane holding a segment's last term adds the sum to the row's shared accumulator.
// A round holds terms of one chunk only, so a row has at most kTileChunk terms in it and
// log2(kTileChunk) scan steps cover every segment.  Every step has a fixed order, so the
// product is deterministic; no atomics.  The accumulators of fp32 rows are double-float
// pairs: this GPU's fp64 pipe is slow enough that one fp64 update per segment of every
// round kept it 30% busy.
// ---------------------------------------------------------------------------------------
// weights of the term-parallel kernel (shared memory): per coupling class c and
// stabiliser order t, J_c / 2 sqrt(t), split into two fp32 words for fp32 vectors and as
// one fp64 word for fp64 vectors (in the same 8-byte slots); complex fp32 sectors add
// (cos, remainder, sin, remainder) per character, complex fp64 sectors use the fp64
// character table
struct TileW {
  const float2 *wf;
  const float4 *csf4;
  const double *csd;
  int n_sq;
};

template <typename V, int NSUB, bool kE2, bool kGeneral>
__device__ __forceinline__ void tile_round(const Sm2 &S, const TwoParams &P, const V *x,
                                           const TileW &W, int c, const uint64_t *rowst,
                                           uint16_t *list, int base, int T, int bbase,
                                           double *racc, int *n_def) {
  using A = typename Vf<V>::A;
  constexpr bool kC = Vf<V>::cplx;
  constexpr bool kF = sizeof(A) == 4;
  const unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const int N = P.N, n = P.n;
  const uint32_t bmask = (1u << n) - 1u;
  const int t = base + lane;
  int r = 32;
  uint32_t e = 0;
  bool defer = false;
  A v_re = 0, v_im = 0;
  float l_re = 0.f, l_im = 0.f;   // fp32 vectors: low words of the values (double-float)
  if (t < T) {
    e = list[t];
    r = (int)(e >> 5);
    const uint64_t sr = rowst[r];
    // the exchanged configuration, block by block: one bit flips in the block of each
    // end of the bond
    const uint32_t bi = S.bblk[bbase + (e & 31)];
    const int xa = bi & 15, xb = (bi >> 4) & 15;
    const uint32_t fa = 1u << ((bi >> 8) & 255), fb = 1u << (bi >> 16);
    uint32_t s2[NSUB];
#pragma unroll
    for (int X = 0; X < NSUB; X++)
      s2[X] = ((uint32_t)(sr >> (N - (X + 1) * n)) & bmask) ^ (X == xa ? fa : 0u) ^
              (X == xb ? fb : 0u);
    Rep2 R;
    if constexpr (kGeneral) {
      R = find_rep_blocks<NSUB, kE2>(S, P, s2);
    } else {
      defer = !find_rep_simple<NSUB, kE2>(S, P, s2, R);
    }
    if (!defer && !R.mixed) {
      const int64_t j = lookup_two(S, P, R.minrep, R.low);
      if (j >= 0) {
        const V xj = gather_x(x, j);
        if constexpr (kF) {
          // the weight J_c / 2 sqrt(|Stab_j|) as two fp32 words, so that no rounding of it
          // is repeated in every term with the same class and stabiliser order (a bias
          // that would not average out over the sector)
          const float2 wv = W.wf[c * W.n_sq + R.t];
          if constexpr (!kC) {   // (wh + wl) xj as an unevaluated pair
            const float ph_ = __fmul_rn(wv.x, xj);
            const float pl_ = __fmaf_rn(wv.y, xj, __fmaf_rn(wv.x, xj, -ph_));
            v_re = R.ph == 0 ? ph_ : -ph_;
            l_re = R.ph == 0 ? pl_ : -pl_;
          } else {
            const float4 cs = W.csf4[R.ph];   // cos, its remainder, sin, its remainder
            const float crh = wv.x * cs.x, crl = fmaf(wv.x, cs.x, -crh) + fmaf(wv.x, cs.y, wv.y * cs.x);
            const float cih = wv.x * cs.z, cil = fmaf(wv.x, cs.z, -cih) + fmaf(wv.x, cs.w, wv.y * cs.z);
            v_re = fmaf(crh, xj.x, fmaf(crl, xj.x, -fmaf(cih, xj.y, cil * xj.y)));
            v_im = fmaf(crh, xj.y, fmaf(crl, xj.y, fmaf(cih, xj.x, cil * xj.x)));
          }
        } else {
          const double wgt = reinterpret_cast<const double *>(W.wf)[c * W.n_sq + R.t];   // J_c / 2 sqrt(|Stab_j|)
          if constexpr (!kC) {
            const double pv = wgt * xj;
            v_re = R.ph == 0 ? pv : -pv;
          } else {
            const double cr = W.csd[2 * R.ph] * wgt, ci = W.csd[2 * R.ph + 1] * wgt;
            v_re = cr * xj.x - ci * xj.y;
            v_im = cr * xj.y + ci * xj.x;
          }
        }
      }
    }
  }
  if constexpr (!kGeneral) {
    // deferred terms go, in lane (= list) order, to the front of the list, over entries
    // every lane has read already (one deferred entry per consumed entry at most)
    const unsigned dm = __ballot_sync(FULL, defer);
    if (defer) list[*n_def + __popc(dm & ((1u << lane) - 1u))] = (uint16_t)e;
    *n_def += __popc(dm);
  }
  // segmented inclusive scan: lanes with the same row form one segment, at most kTileChunk
  // lanes long (fp32 values are summed in double-float, so the sum of a segment carries
  // no fp32 rounding)
#pragma unroll
  for (int d = 1; d < kTileChunk; d <<= 1) {
    const int ru = __shfl_up_sync(FULL, r, d);
    const A a = __shfl_up_sync(FULL, v_re, d);
    A b = 0;
    if constexpr (kC) b = __shfl_up_sync(FULL, v_im, d);
    float al = 0.f, bl = 0.f;
    if constexpr (kF) {
      al = __shfl_up_sync(FULL, l_re, d);
      if constexpr (kC) bl = __shfl_up_sync(FULL, l_im, d);
    }
    if (lane >= d && ru == r) {
      if constexpr (kF) {
        df_add(v_re, l_re, a);
        l_re = __fadd_rn(l_re, al);
        if constexpr (kC) {
          df_add(v_im, l_im, b);
          l_im = __fadd_rn(l_im, bl);
        }
      } else {
        v_re += a;
        if constexpr (kC) v_im += b;
      }
    }
  }
  const int rn = __shfl_down_sync(FULL, r, 1);
  __syncwarp();   // the previous round's accumulator updates are visible
  if (r < 32 && (lane == 31 || rn != r)) {   // last lane of its segment
    if constexpr (kF) {
      float *rf = reinterpret_cast<float *>(racc);
      float h = rf[r], l = rf[32 + r];
      df_add(h, l, v_re);
      rf[r] = h;
      rf[32 + r] = __fadd_rn(l, l_re);
      if constexpr (kC) {
        h = rf[64 + r];
        l = rf[96 + r];
        df_add(h, l, v_im);
        rf[64 + r] = h;
        rf[96 + r] = __fadd_rn(l, l_im);
      }
    } else {
      racc[r] += (double)v_re + (double)l_re;
      if constexpr (kC) racc[32 + r] += (double)v_im + (double)l_im;
    }
  }
}

template <typename V, int NSUB, bool kE2>
__global__ void __launch_bounds__(kE2 ? kTileThreadsE2 : kTileThreads, kE2 ? 1 : kTileMinBlocks)
    apply_tile_kernel(const __grid_constant__ TwoParams P) {
  constexpr bool kC = Vf<V>::cplx;
  extern __shared__ __align__(16) unsigned char sm[];
  const Sm2 S = stage_two(P, sm, kC, kE2);
  {
    const double *sqd = reinterpret_cast<const double *>(sm + P.off_sq);
    const double *csd = reinterpret_cast<const double *>(sm + P.off_cs);
    float2 *wf = reinterpret_cast<float2 *>(sm + P.off_sqf);
    float4 *csf4 = reinterpret_cast<float4 *>(sm + P.off_csf);
    for (uint32_t k = threadIdx.x; k < (uint32_t)P.n_classes * P.n_sq; k += blockDim.x) {
      const double wv = P.jh[k / P.n_sq] * sqd[k % P.n_sq];
      const float hi = (float)wv;
      if (sizeof(typename Vf<V>::A) == 4) wf[k] = make_float2(hi, (float)(wv - (double)hi));
      else reinterpret_cast<double *>(wf)[k] = wv;
    }
    if (kC)
      for (uint32_t k = threadIdx.x; k < P.n_cs / 2; k += blockDim.x) {
        const double cv = csd[2 * k], sv = csd[2 * k + 1];
        const float ch = (float)cv, sh = (float)sv;
        csf4[k] = make_float4(ch, (float)(cv - (double)ch), sh, (float)(sv - (double)sh));
      }
    uint32_t *nb = reinterpret_cast<uint32_t *>(sm + P.off_nib);
    const uint32_t n_nibtab = (uint32_t)P.cls_word[P.n_classes] * P.n_nib * 16;
    for (uint32_t k = threadIdx.x; k < n_nibtab; k += blockDim.x) nb[k] = P.nib[k];
    __syncthreads();
  }
  const uint32_t *nibs = reinterpret_cast<const uint32_t *>(sm + P.off_nib);
  TileW W;
  W.wf = reinterpret_cast<const float2 *>(sm + P.off_sqf);
  W.csf4 = reinterpret_cast<const float4 *>(sm + P.off_csf);
  W.csd = reinterpret_cast<const double *>(sm + P.off_cs);
  W.n_sq = (int)P.n_sq;
  using A = typename Vf<V>::A;
  constexpr bool kF = sizeof(A) == 4;
  const double *rsd = reinterpret_cast<const double *>(sm + P.off_sq) + P.n_sq;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char *tw = sm + P.off_tile + (size_t)wid * kTileWarpBytes;
  uint64_t *rowst = reinterpret_cast<uint64_t *>(tw);
  // row accumulators: fp64 [re 32][im 32], or for fp32 rows double-float words as floats
  // [re hi 32][re lo 32][im hi 32][im lo 32]
  double *racc = reinterpret_cast<double *>(tw + 32 * 8);
  uint16_t *list = reinterpret_cast<uint16_t *>(tw + 32 * 8 + 32 * 16);
  const V *x = reinterpret_cast<const V *>(P.x);
  V *y = reinterpret_cast<V *>(P.y);
  const unsigned FULL = 0xFFFFFFFFu;
  const int64_t n_tiles = (P.r1 - P.r0 + 31) >> 5;
  const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
  double dot_re = 0.0, dot_im = 0.0;
  for (int64_t tile = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid; tile < n_tiles; tile += wstride) {
    {
      const int64_t i = P.r0 + (tile << 5) + lane;
      rowst[lane] = i < P.r1 ? __ldcs(reinterpret_cast<const unsigned long long *>(P.basis) + i) : 0ULL;
      racc[lane] = 0.0;
      if (kC) racc[32 + lane] = 0.0;
    }
    const bool valid = P.r0 + (tile << 5) + lane < P.r1;
    double diag = 0.0;
    for (int c = 0; c < P.n_classes; c++) {
      int nanti = 0;
      for (int wd = P.cls_word[c]; wd < P.cls_word[c + 1]; wd++) {
        uint32_t m = 0;
        {   // antiparallel bonds of the word: XOR of the state's nibbles' contributions
          const uint64_t s = rowst[lane];
          const uint32_t *nw = nibs + (uint32_t)wd * P.n_nib * 16;
          for (uint32_t q = 0; q < P.n_nib; q++) m ^= nw[q * 16 + (uint32_t)((s >> (4 * q)) & 15u)];
        }
        if (!valid) m = 0;
        nanti += __popc(m);
#pragma unroll 1
        for (int h = 0; h < 32 / kTileChunk; h++) {
          const uint32_t cm = (m >> (kTileChunk * h)) & ((1u << kTileChunk) - 1u);
          const int cnt = __popc(cm);
          int incl = cnt;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += u;
          }
          const int T = __shfl_sync(FULL, incl, 31);
          if (T == 0) continue;
          {   // this lane's terms, in bond order, at its place in the row-major list
            uint32_t mm = cm;
            int pos = incl - cnt;
            while (mm) {
              const int k = __ffs(mm) - 1;
              mm &= mm - 1;
              list[pos++] = (uint16_t)((lane << 5) | k);
            }
          }
          __syncwarp();
          const int bbase = wd * 32 + kTileChunk * h;
          int n_def = 0;
          for (int base = 0; base < T; base += 32)
            tile_round<V, NSUB, kE2, false>(S, P, x, W, c, rowst, list, base, T, bbase, racc, &n_def);
          __syncwarp();
          for (int base = 0; base < n_def; base += 32)
            tile_round<V, NSUB, kE2, true>(S, P, x, W, c, rowst, list, base, n_def, bbase, racc, &n_def);
          __syncwarp();   // the list is rewritten by the next chunk
        }
      }
      diag += P.jzq[c] * (double)(P.nb_cls[c] - 2 * nanti);
    }
    __syncwarp();
    if (valid) {
      const int64_t i = P.r0 + (tile << 5) + lane;
      const double rs = rsd[__ldcs(P.stab + i)];
      const float *rf = reinterpret_cast<const float *>(racc);
      const double row_re = kF ? (double)rf[lane] + (double)rf[32 + lane] : (double)racc[lane];
      // y_i in fp64, rounded once to the vector type; for fp32 vectors the rounding's
      // remainder goes to ylo when asked (the mixed Lanczos keeps y as a double-float
      // pair for its update), and <x, y> uses the unrounded value
      if constexpr (!kC) {
        const double xi = (double)x[i];
        const double yd = diag * xi + row_re * rs;
        const A yi = (A)yd;
        __stcs(y + (i - P.r0), yi);
        if (kF && P.ylo) reinterpret_cast<float *>(P.ylo)[i - P.r0] = (float)(yd - (double)yi);
        if (P.partial) dot_re += xi * (kF && P.ylo ? yd : (double)yi);
      } else {
        const double row_im = kF ? (double)rf[64 + lane] + (double)rf[96 + lane] : (double)racc[32 + lane];
        const V xv = x[i];
        const double yr = diag * (double)xv.x + row_re * rs;
        const double yim = diag * (double)xv.y + row_im * rs;
        V yv;
        yv.x = (A)yr;
        yv.y = (A)yim;
        y[i - P.r0] = yv;
        double ur = (double)yv.x, ui = (double)yv.y;
        if (kF && P.ylo) {
          float2 lo;
          lo.x = (float)(yr - ur);
          lo.y = (float)(yim - ui);
          reinterpret_cast<float2 *>(P.ylo)[i - P.r0] = lo;
          ur = yr;
          ui = yim;
        }
        if (P.partial) {
          dot_re += (double)xv.x * ur + (double)xv.y * ui;
          dot_im += (double)xv.x * ui - (double)xv.y * ur;
        }
      }
    }
    __syncwarp();   // rowst and racc are rewritten by the next tile
  }
  if (P.partial) {
    __shared__ double red[32];
    const int nparts = kC ? 2 : 1;
    for (int part = 0; part < nparts; part++) {
      double d = part ? dot_im : dot_re;
      for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(FULL, d, o);
      __syncthreads();
      if (lane == 0) red[wid] = d;
      __syncthreads();
      if (wid == 0) {
        d = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(FULL, d, o);
        if (lane == 0) P.partial[part * gridDim.x + blockIdx.x] = d;
      }
    }
  }
}

// test hook: the two-level search alone
template <int NSUB, bool kE2>
__global__ void find_rep_two_kernel(const TwoParams P, const DevIndex I, const uint64_t *states,
                                    int64_t n, uint64_t *rep, int32_t *phase, int32_t *stab,
                                    int64_t *index) {
  extern __shared__ __align__(16) unsigned char sm[];
  const Sm2 S = stage_two(P, sm, false, kE2);
  const uint32_t bmask = (1u << P.n) - 1u;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t sub[NSUB];
#pragma unroll
    for (int X = 0; X < NSUB; X++) sub[X] = (uint32_t)(states[i] >> (P.N - (X + 1) * P.n)) & bmask;
    const Rep2 R = find_rep_blocks<NSUB, kE2>(S, P, sub);
    const uint64_t r = ((uint64_t)R.minrep << P.L) | R.low;
    if (rep) rep[i] = r;
    if (phase) phase[i] = R.ph;
    if (stab) stab[i] = R.t;
    if (index) index[i] = (R.mixed || I.D == 0) ? -1 : lookup_index(I, r);
  }
}

size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }

// Parameters and shared-memory layout; e2 = stage the level-2 tables in shared memory.
int make_params(const ed_basis *B, const double *J, const double *Jz, bool e2, TwoParams &P,
                int tile_warps = 0) {
  if (!B->two_level || B->nsub < 2 || B->nsub > 4 || B->I.r_bits > 12 || B->D == 0 ||
      (B->nsub - 1) * B->n > 32 || B->N - B->I.r_bits > 32)
    return ED_ERR_UNSUPPORTED;
  P = TwoParams{};
  P.N = B->N; P.n = B->n; P.nsym = B->nsym; P.denom = B->denom;
  P.n_classes = B->n_classes;
  for (int c = 0; c <= B->n_classes; c++) P.cls_word[c] = B->cls_word[c];
  for (int c = 0; c < B->n_classes; c++) {
    P.nb_cls[c] = B->cls_off[c + 1] - B->cls_off[c];
    P.jh[c] = J ? 0.5 * J[c] : 0.0;
    P.jzq[c] = J ? 0.25 * J[c] * Jz[c] : 0.0;
  }
  P.e1 = B->d_e1; P.e2 = B->d_e2; P.off2 = B->d_off2; P.list2 = B->d_list2; P.rid = B->d_rid;
  P.act = (const uint16_t *)B->d_action;
  P.dest = B->d_dest; P.src = B->d_src; P.phase = B->d_phase;
  P.bond_pos = B->d_bond_pad; P.top_rank = B->d_top_rank; P.limits = B->d_limits;
  P.sqrt_tab = B->d_sqrt; P.rsqrt_tab = B->d_rsqrt; P.cs = B->d_cs;
  P.basis = B->d_basis; P.stab = B->d_stab; P.postfix = B->d_postfix;
  P.r_bits = B->I.r_bits; P.q_bits = B->I.q_bits; P.post_bits = B->I.post_bits;
  P.post_bytes = B->I.post_bytes; P.D = B->D;
  P.L = (B->nsub - 1) * B->n;
  P.id_g = B->id_g;
  P.qmask = P.q_bits >= 32 ? 0xFFFFFFFFu : ((1u << P.q_bits) - 1u);
  P.pmask = P.post_bits >= 32 ? 0xFFFFFFFFu : ((1u << P.post_bits) - 1u);
  P.bond_blk = B->d_bond_blk;
  const uint32_t nn = 1u << B->n;
  P.n_e1 = (uint32_t)B->nsub * nn;
  P.n_rid = nn;
  P.n_dest = (uint32_t)B->nsym * B->nsub;
  P.n_bond = (uint32_t)B->cls_word[B->n_classes] * 64;
  P.n_top = 1u << B->I.r_bits;
  P.n_sq = (uint32_t)B->nsym + 1;
  P.n_cs = 2u * B->denom;
  P.n_e2 = e2 ? (uint32_t)B->n_rid * (B->nsub - 1) * nn : 0u;
  size_t off = 0;
  auto put = [&](uint32_t &o, size_t bytes) { o = (uint32_t)off; off += a16(bytes); };
  put(P.off_sq, 16 * (size_t)P.n_sq);
  put(P.off_cs, 8 * (size_t)P.n_cs);
  put(P.off_e1, 4 * (size_t)P.n_e1);
  put(P.off_top, 2 * (size_t)P.n_top);
  put(P.off_phase, 4 * (size_t)P.nsym);
  put(P.off_e2, 4 * (size_t)P.n_e2);
  put(P.off_bblk, 2 * (size_t)P.n_bond);
  put(P.off_rid, P.n_rid);
  put(P.off_dest, P.n_dest);
  put(P.off_src, P.n_dest);
  put(P.off_bond, P.n_bond);
  P.tile_warps = (uint32_t)tile_warps;
  P.rlim = reinterpret_cast<const uint4 *>(B->d_rlim);
  P.rq_bits = B->rq_bits;
  P.rpost_bits = B->rpost_bits;
  P.rqmask = B->rq_bits >= 32 ? 0xFFFFFFFFu : ((1u << B->rq_bits) - 1u);
  P.rpmask = (1u << B->rpost_bits) - 1u;
  P.nib = B->d_nib;
  P.n_nib = (uint32_t)B->n_nib;
  if (tile_warps) {
    put(P.off_sqf, 8 * (size_t)P.n_sq * B->n_classes);   // J_c/2 sqrt(t) as float2
    put(P.off_csf, 8 * (size_t)P.n_cs);                  // (cos, rem, sin, rem) as float4
    put(P.off_nib, 4 * B->nib.size());
    put(P.off_tile, (size_t)tile_warps * kTileWarpBytes);
  }
  P.smem_bytes = (uint32_t)off;
  if (off > (e2 ? (tile_warps ? 220 : 180) : 100) * 1024) return ED_ERR_UNSUPPORTED;
  return ED_OK;
}

// e2 staged: one 1024-thread CTA per SM (the tables take most of shared memory), 32
// warps at 64 registers; otherwise two 768-thread CTAs per SM, 48 warps at 40 registers.
template <typename V, int NSUB, int kMode = 0>
int launch_t(const TwoParams &P, bool e2, int grid, cudaStream_t st) {
  if (e2) {
    auto k = apply_two_kernel<V, NSUB, true, kMode>;
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes));
    k<<<grid, 1024, P.smem_bytes, st>>>(P);
  } else {
    auto k = apply_two_kernel<V, NSUB, false, kMode>;
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes));
    // ask for just the shared memory of kMinBlocks resident blocks (plus the per-block
    // reserve); the rest of the SM's 256 KB stays L1 for the SymmetryAction and level-2
    // lines (about 1% faster than the default split)
    const int need = kMinBlocks * ((int)P.smem_bytes + 1536);
    const int pct = std::min(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    k<<<grid, kThreads, P.smem_bytes, st>>>(P);
  }
  ED_CK(cudaGetLastError());
  return ED_OK;
}

template <typename V, int kMode = 0>
int launch_v(const TwoParams &P, bool e2, int nsub, int grid, cudaStream_t st) {
  switch (nsub) {
    case 2: return launch_t<V, 2, kMode>(P, e2, grid, st);
    case 3: return launch_t<V, 3, kMode>(P, e2, grid, st);
    case 4: return launch_t<V, 4, kMode>(P, e2, grid, st);
  }
  return ED_ERR_UNSUPPORTED;
}

}  // namespace

template <typename V, int NSUB>
int launch_tile_t(const TwoParams &P, bool e2, int grid, cudaStream_t st) {
  if (e2) {
    auto k = apply_tile_kernel<V, NSUB, true>;
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes));
    k<<<grid, kTileThreadsE2, P.smem_bytes, st>>>(P);
  } else {
    auto k = apply_tile_kernel<V, NSUB, false>;
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes));
    const int need = kTileMinBlocks * ((int)P.smem_bytes + 1536);
    const int pct = std::min(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
    k<<<grid, kTileThreads, P.smem_bytes, st>>>(P);
  }
  ED_CK(cudaGetLastError());
  return ED_OK;
}

template <typename V>
int launch_tile_v(const TwoParams &P, bool e2, int nsub, int grid, cudaStream_t st) {
  switch (nsub) {
    case 2: return launch_tile_t<V, 2>(P, e2, grid, st);
    case 3: return launch_tile_t<V, 3>(P, e2, grid, st);
    case 4: return launch_tile_t<V, 4>(P, e2, grid, st);
  }
  return ED_ERR_UNSUPPORTED;
}

// The two-level path applies when its tables exist (2..4 sublattices of <= 11 sites,
// |G| <= 4096); returns ED_ERR_UNSUPPORTED otherwise (the caller uses the generic kernel).
int ed_launch_apply_fast(const ed_basis *B, const double *J, const double *Jz, const void *x,
                         void *y, int dtype, int64_t r0, int64_t r1, double *partial,
                         cudaStream_t st, int mode, void *ylo, bool *ylo_done) {
  TwoParams P;
  bool e2 = true;
  int rc = make_params(B, J, Jz, e2, P);
  if (rc == ED_ERR_UNSUPPORTED) { e2 = false; rc = make_params(B, J, Jz, false, P); }
  if (rc) return rc;
  // the product: the term-parallel kernel (level-2 tables staged when they fit with the
  // per-warp term lists, else read from global memory)
  if (mode == 0) {
    TwoParams Q;
    bool qe2 = e2;
    int qrc = make_params(B, J, Jz, qe2, Q, (qe2 ? kTileThreadsE2 : kTileThreads) / 32);
    if (qrc == ED_ERR_UNSUPPORTED && qe2) {
      qe2 = false;
      qrc = make_params(B, J, Jz, false, Q, kTileThreads / 32);
    }
    if (qrc == ED_OK) {
      Q.x = x; Q.y = y; Q.r0 = r0; Q.r1 = r1; Q.partial = partial;
      Q.ylo = (dtype == ED_F32 || dtype == ED_C64) ? ylo : nullptr;
      if (ylo_done) *ylo_done = Q.ylo != nullptr;
      const int bs = qe2 ? kTileThreadsE2 : kTileThreads;
      int grid = B->sm_count * (qe2 ? 1 : kTileMinBlocks);
      const int64_t need = (r1 - r0 + bs - 1) / bs;
      if (need < grid) grid = (int)need;
      if (grid < 1) grid = 1;
      if (partial && grid > B->n_partial / 2) return ed_fail(ED_ERR_INVALID, "partial buffer too small");
      B->last_apply_grid = grid;
      switch (dtype) {
        case ED_F32: return launch_tile_v<float>(Q, qe2, B->nsub, grid, st);
        case ED_C64: return launch_tile_v<float2>(Q, qe2, B->nsub, grid, st);
        case ED_F64: return launch_tile_v<double>(Q, qe2, B->nsub, grid, st);
        case ED_C128: return launch_tile_v<double2>(Q, qe2, B->nsub, grid, st);
      }
      return ed_fail(ED_ERR_INVALID, "unknown dtype");
    }
  }
  P.x = x; P.y = y; P.r0 = r0; P.r1 = r1; P.partial = partial;
  const int bs = e2 ? 1024 : kThreads;
  int grid = B->sm_count * (e2 ? 1 : kMinBlocks);
  const int64_t need = (r1 - r0 + bs - 1) / bs;
  if (need < grid) grid = (int)need;
  if (grid < 1) grid = 1;
  if (partial && grid > B->n_partial / 2) return ed_fail(ED_ERR_INVALID, "partial buffer too small");
  B->last_apply_grid = grid;
  if (mode == 1) {
    if (!partial || B->n_classes * grid > B->n_partial) return ed_fail(ED_ERR_INVALID, "partial buffer too small");
    switch (dtype) {
      case ED_F64: return launch_v<double, 1>(P, e2, B->nsub, grid, st);
      case ED_F32: return launch_v<float, 1>(P, e2, B->nsub, grid, st);
      case ED_C128: return launch_v<double2, 1>(P, e2, B->nsub, grid, st);
      case ED_C64: return launch_v<float2, 1>(P, e2, B->nsub, grid, st);
    }
    return ed_fail(ED_ERR_INVALID, "unknown dtype");
  }
  switch (dtype) {
    case ED_F64: return launch_v<double>(P, e2, B->nsub, grid, st);
    case ED_F32: return launch_v<float>(P, e2, B->nsub, grid, st);
    case ED_C128: return launch_v<double2>(P, e2, B->nsub, grid, st);
    case ED_C64: return launch_v<float2>(P, e2, B->nsub, grid, st);
  }
  return ed_fail(ED_ERR_INVALID, "unknown dtype");
}

int ed_launch_find_rep_two(const ed_basis *B, const uint64_t *states, int64_t n, uint64_t *rep,
                           int32_t *phase, int32_t *stab, int64_t *index, cudaStream_t st) {
  TwoParams P;
  bool e2 = true;
  int rc = make_params(B, nullptr, nullptr, e2, P);
  if (rc == ED_ERR_UNSUPPORTED) { e2 = false; rc = make_params(B, nullptr, nullptr, false, P); }
  if (rc == ED_ERR_UNSUPPORTED) return ed_fail(rc, "two-level search not available for this sector");
  if (rc) return rc;
  if (n <= 0) return ED_OK;
  int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)B->sm_count * 4);
  switch (B->nsub * 2 + (e2 ? 1 : 0)) {
#define L2CASE(K, C)                                                                           \
  case K * 2 + C: {                                                                            \
    auto k = find_rep_two_kernel<K, C>;                                                        \
    ED_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, P.smem_bytes)); \
    k<<<grid, 256, P.smem_bytes, st>>>(P, B->I, states, n, rep, phase, stab, index);           \
    break;                                                                                     \
  }
    L2CASE(2, 0)
    L2CASE(3, 0)
    L2CASE(4, 0)
    L2CASE(2, 1)
    L2CASE(3, 1)
    L2CASE(4, 1)
#undef L2CASE
  }
  ED_CK(cudaGetLastError());
  return ED_OK;
}
