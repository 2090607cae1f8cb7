// sced_internal.cuh -- data layout and device building blocks shared by the kernels of
// libsced: the sublattice-coding representative search (Alg. 2 of arXiv:1804.05028),
// the Limits lookup (Sec. IV) and small helpers.  Host-only declarations are at the end.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/sced.h"

#define ED_MAXSUB 8
#define ED_MAXCLS 8
#define ED_MAXBONDS 4096

// ---------------------------------------------------------------------------------
// Lookup tables of the sublattice coding (Eqs. 8-11), device resident.
//   n = N / nsub bits per sublattice block; block X holds bits [N-(X+1)n, N-Xn).
//   rep[X<<n | sub]           Rep_X(sub): the smallest g sub over g in G_X, read on block 0
//   sym_off[X*(2^n+1) + sub]  start of Sym_X(sub) in sym_list (end = next entry)
//   sym_list[...]             group elements of Sym_X(sub), increasing g
//   action[((X<<n)|sub)*nsym + g]   g sub as an n-bit value on block dest[g*nsub+X]
//                             (SymmetryAction_X, Eq. 11); uint16 when n <= 16 else uint32
//   dest[g*nsub + X]          block that g carries block X onto
//   phase[g]                  numerator of chi(g) over the irrep's denominator
// ---------------------------------------------------------------------------------
struct DevTables {
  int N, nsub, n, nsym;
  int denom;
  int action_u16;
  int chi_trivial;           // every character is 1 (no projection check needed)
  // one sublattice: the whole lookup table (Sec. III, second option), per configuration
  // rep | first minimising g << 32 | number of minimisers << 48, and the permutations as
  // bit maps pbit[g*N + b] = bit that bit b is carried to (for the projection check)
  const uint64_t *full;
  const uint8_t *pbit;
  const uint8_t *flip;       // [nsym] spin reversal of each element (one-sublattice table)
  const uint32_t *rep;
  const uint32_t *sym_off;
  const uint16_t *sym_list;
  const void *action;
  const uint8_t *dest;
  const int32_t *phase;
};

// Basis and its prefix index.
//   basis[D]  sorted representatives (Basis of Sec. IV), stab[D] = |Stab|
//   key(s) = top_rank[s >> (N - r_bits)] << q_bits | (s >> post_bits) & (2^q - 1)
//   limits[key] .. limits[key+1]: half-open range of Basis holding that key (Limits)
//   postfix[i] = basis[i] & (2^post_bits - 1): what the in-bucket binary search compares
//   rlim[key'] = {first index, 0, 64-bit bitmap of postfixes}: the ranked Limits over
//   rq_bits raw bits and rpost_bits (<= 6) postfix bits, when built (else null)
struct DevIndex {
  int N, r_bits, q_bits, post_bits;
  int post_bytes;  // 1, 2, 4 or 8
  int64_t D;
  const uint64_t *basis;
  const uint16_t *stab;
  const uint32_t *top_rank;
  const uint32_t *limits;
  const void *postfix;
  const uint4 *rlim;
  int rq_bits, rpost_bits;
};

#define ED_NO_RANK 0xFFFFFFFFu

struct RepOut {
  uint64_t rep;
  int g;       // first minimising element in (Y, Sym_Y) order
  int t;       // number of minimisers = |Stab(rep)|
  int mixed;   // 1 when two minimisers have different characters (rep is dropped)
};

__device__ __forceinline__ uint32_t ld_action(const DevTables &T, int X, uint32_t sub, int g) {
  size_t off = ((size_t)((X << T.n) | sub)) * (size_t)T.nsym + (size_t)g;
  if (T.action_u16) return __ldg(reinterpret_cast<const uint16_t *>(T.action) + off);
  return __ldg(reinterpret_cast<const uint32_t *>(T.action) + off);
}

// Alg. 2: MinRep = min_X Rep_X(s_X); for every Y attaining it and every g in
// Sym_Y(s_Y), assemble g s from SymmetryAction and keep the strict minimum.  All
// minimisers are among these candidates (the top block of the orbit minimum is MinRep),
// so counting ties gives |Stab(rep)| and comparing their characters tells whether the
// projected state vanishes.  rep_s / symoff_s / symlist_s / dest_s / phase_s may point
// to shared-memory copies of the tables.
__device__ __forceinline__ RepOut find_rep(const DevTables &T, const uint32_t *rep_s,
                                           const uint32_t *symoff_s, const uint16_t *symlist_s,
                                           const uint8_t *dest_s, const int32_t *phase_s,
                                           uint64_t s) {
  if (T.full) {   // one block: the table holds the answer (a representative that the
                  // projection removes is simply absent from Basis)
    RepOut f;
    if (s >> T.N) { f.rep = ~0ULL; f.g = -1; f.t = 0; f.mixed = 1; return f; }
    const uint64_t e = __ldg(T.full + s);
    f.rep = e & 0xFFFFFFFFull;
    f.g = (int)((e >> 32) & 0xFFFF);
    f.t = (int)(e >> 48);
    f.mixed = 0;
    return f;
  }
  const int n = T.n, nsub = T.nsub, N = T.N;
  const uint32_t mask = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  uint32_t sub[ED_MAXSUB], r[ED_MAXSUB];
  uint32_t minrep = 0xFFFFFFFFu;
#pragma unroll
  for (int X = 0; X < ED_MAXSUB; X++) {
    if (X < nsub) {
      sub[X] = (uint32_t)(s >> (N - (X + 1) * n)) & mask;
      r[X] = rep_s[(X << n) | sub[X]];
      minrep = min(minrep, r[X]);
    }
  }
  RepOut o;
  o.rep = ~0ULL;
  o.g = -1;
  o.t = 0;
  o.mixed = 0;
  int ph = 0;
  const uint64_t top = (uint64_t)minrep << (N - n);
  const size_t stride = ((size_t)1 << n) + 1;
#pragma unroll
  for (int Y = 0; Y < ED_MAXSUB; Y++) {
    if (Y >= nsub || r[Y] != minrep) continue;
    const uint32_t b = symoff_s[Y * stride + sub[Y]];
    const uint32_t e = symoff_s[Y * stride + sub[Y] + 1];
    for (uint32_t k = b; k < e; k++) {
      const int g = symlist_s[k];
      uint64_t v = top;
#pragma unroll
      for (int X = 0; X < ED_MAXSUB; X++) {
        if (X < nsub && X != Y) {
          const int d = dest_s[g * nsub + X];
          v |= (uint64_t)ld_action(T, X, sub[X], g) << (N - (d + 1) * n);
        }
      }
      const int pg = phase_s[g];
      if (v < o.rep) {
        o.rep = v; o.g = g; o.t = 1; o.mixed = 0; ph = pg;
      } else if (v == o.rep) {
        o.t++;
        o.mixed |= (pg != ph);
      }
    }
  }
  return o;
}

// Is s its own representative with a surviving projection?  Same search as find_rep
// but stops at the first candidate below s.  On success *t = |Stab(s)|.
__device__ __forceinline__ bool is_kept_rep(const DevTables &T, const uint32_t *rep_s,
                                            const uint32_t *symoff_s, const uint16_t *symlist_s,
                                            const uint8_t *dest_s, const int32_t *phase_s,
                                            uint64_t s, int *t_out) {
  if (T.full) {
    const uint64_t e = __ldg(T.full + s);
    if ((e & 0xFFFFFFFFull) != s) return false;
    if (!T.chi_trivial) {   // the projection survives iff chi = 1 on the stabiliser
      for (int g = 0; g < T.nsym; g++) {
        if (phase_s[g] == 0) continue;
        uint64_t v = 0, m = s;
        while (m) {
          const int b = __ffsll((long long)m) - 1;
          m &= m - 1;
          v |= 1ULL << T.pbit[g * T.N + b];
        }
        if (T.flip && T.flip[g]) v ^= (T.N == 64) ? ~0ULL : ((1ULL << T.N) - 1ULL);
        if (v == s) return false;
      }
    }
    *t_out = (int)(e >> 48);
    return true;
  }
  const int n = T.n, nsub = T.nsub, N = T.N;
  const uint32_t mask = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  uint32_t sub[ED_MAXSUB], r[ED_MAXSUB];
  const uint32_t topv = (uint32_t)(s >> (N - n)) & mask;
  uint32_t minrep = 0xFFFFFFFFu;
#pragma unroll
  for (int X = 0; X < ED_MAXSUB; X++) {
    if (X < nsub) {
      sub[X] = (uint32_t)(s >> (N - (X + 1) * n)) & mask;
      r[X] = rep_s[(X << n) | sub[X]];
      minrep = min(minrep, r[X]);
    }
  }
  if (minrep < topv) return false;   // some g gives a smaller top block
  const uint64_t top = (uint64_t)minrep << (N - n);
  const size_t stride = ((size_t)1 << n) + 1;
  int t = 0;
#pragma unroll
  for (int Y = 0; Y < ED_MAXSUB; Y++) {
    if (Y >= nsub || r[Y] != minrep) continue;
    const uint32_t b = symoff_s[Y * stride + sub[Y]];
    const uint32_t e = symoff_s[Y * stride + sub[Y] + 1];
    for (uint32_t k = b; k < e; k++) {
      const int g = symlist_s[k];
      uint64_t v = top;
#pragma unroll
      for (int X = 0; X < ED_MAXSUB; X++) {
        if (X < nsub && X != Y) {
          const int d = dest_s[g * nsub + X];
          v |= (uint64_t)ld_action(T, X, sub[X], g) << (N - (d + 1) * n);
        }
      }
      if (v < s) return false;
      if (v == s) {
        if (phase_s[g] != 0) return false;   // chi not trivial on Stab(s): state vanishes
        t++;
      }
    }
  }
  *t_out = t;
  return true;
}

template <typename PT>
__device__ __forceinline__ int64_t bucket_search(const PT *post, uint32_t lo, uint32_t hi,
                                                 PT target) {
  const uint32_t end = hi;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(post + mid) < target) lo = mid + 1; else hi = mid;
  }
  return (lo < end && __ldg(post + lo) == target) ? (int64_t)lo : -1;
}

// Index of representative s in Basis, or -1 (Limits lookup + binary search, Sec. IV).
__device__ __forceinline__ int64_t lookup_index(const DevIndex &I, uint64_t s) {
  if (I.N < 64 && (s >> I.N) != 0) return -1;   // not an N-site configuration
  const uint32_t top = (uint32_t)(s >> (I.N - I.r_bits));
  const uint32_t rk = __ldg(I.top_rank + top);
  if (rk == ED_NO_RANK) return -1;
  if (I.rlim) {   // ranked Limits: first index + rank of the postfix in the bucket's bitmap
    const uint64_t key = ((uint64_t)rk << I.rq_bits) |
                         ((s >> I.rpost_bits) & ((1ULL << I.rq_bits) - 1ULL));
    const uint4 rec = __ldg(I.rlim + key);
    const uint32_t pf = (uint32_t)(s & ((1ULL << I.rpost_bits) - 1ULL));
    const uint64_t bits = ((uint64_t)rec.w << 32) | rec.z;
    if (!((bits >> pf) & 1ULL)) return -1;
    return (int64_t)rec.x + __popcll(bits & ((1ULL << pf) - 1ULL));
  }
  const uint64_t qmask = (I.q_bits >= 64) ? ~0ULL : ((1ULL << I.q_bits) - 1ULL);
  const uint64_t key = ((uint64_t)rk << I.q_bits) | ((s >> I.post_bits) & qmask);
  const uint32_t lo = __ldg(I.limits + key), hi = __ldg(I.limits + key + 1);
  const uint64_t pmask = (I.post_bits >= 64) ? ~0ULL : ((1ULL << I.post_bits) - 1ULL);
  const uint64_t p = s & pmask;
  if (I.post_bytes == 1)
    return bucket_search<uint8_t>(reinterpret_cast<const uint8_t *>(I.postfix), lo, hi,
                                  (uint8_t)p);
  if (I.post_bytes == 2)
    return bucket_search<uint16_t>(reinterpret_cast<const uint16_t *>(I.postfix), lo, hi,
                                   (uint16_t)p);
  if (I.post_bytes == 4)
    return bucket_search<uint32_t>(reinterpret_cast<const uint32_t *>(I.postfix), lo, hi,
                                   (uint32_t)p);
  return bucket_search<uint64_t>(reinterpret_cast<const uint64_t *>(I.postfix), lo, hi, p);
}

// SplitMix64 output function (Steele, Lea & Flood 2014) for state-keyed start vectors.
__device__ __forceinline__ uint64_t splitmix64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------
#include <memory>
#include <string>
#include <vector>

struct ed_basis {
  int device = 0;
  int sm_count = 0;
  // problem
  int N = 0, nsub = 1, n = 0, nsym = 0, n_up = 0, denom = 1, n_bonds = 0, n_classes = 0;
  bool is_real = true;
  std::vector<int32_t> perm, phase;
  std::vector<uint8_t> flip;           // [nsym] spin reversal (empty: none)
  int id_g = 0;                        // index of the identity element
  std::vector<uint8_t> bond_pos;       // [n_bonds][2] bit positions (class-sorted)
  std::vector<int32_t> cls_off;        // [n_classes+1] bond ranges per class
  std::vector<uint8_t> bond_pad;       // bonds padded per class to words of 32 (inert (0,0))
  std::vector<int32_t> cls_word;       // [n_classes+1] word ranges per class
  std::vector<uint32_t> bond_blk;      // padded bonds: block | block << 4 | bit << 8 | bit << 16
  int n_nib = 0;                       // 4-bit nibbles of a state, (N + 3) / 4
  std::vector<uint32_t> nib;           // [word][nibble][16]: antiparallel-mask contributions
  // tables
  DevTables T{};
  uint32_t *d_rep = nullptr, *d_sym_off = nullptr;
  uint16_t *d_sym_list = nullptr;
  void *d_action = nullptr;
  uint8_t *d_dest = nullptr;
  uint8_t *d_src = nullptr;            // [nsym][nsub]: block carried onto block d
  // two-level search (level 1: Rep_X | first of Sym_X << 12; level 2 per stabiliser K_R)
  bool two_level = false;
  int n_rid = 0;
  uint32_t *d_e1 = nullptr, *d_e2 = nullptr, *d_off2 = nullptr;
  uint8_t *d_rid = nullptr;
  uint16_t *d_list2 = nullptr;
  uint8_t *d_bond_pad = nullptr;
  uint32_t *d_bond_blk = nullptr;
  uint32_t *d_nib = nullptr;
  int32_t *d_phase = nullptr;
  std::shared_ptr<uint64_t> full_tab;  // one-sublattice table, shareable between sectors
  uint8_t *d_pbit = nullptr;
  uint8_t *d_flip = nullptr;
  size_t sym_list_len = 0;
  size_t table_bytes = 0;
  // basis + index
  DevIndex I{};
  int64_t D = 0;
  uint64_t *d_basis = nullptr;
  uint16_t *d_stab = nullptr;
  uint32_t *d_top_rank = nullptr, *d_limits = nullptr;
  void *d_postfix = nullptr;
  int64_t n_keys = 0, max_bucket = 0;
  // ranked Limits: per key {first index, 0, 64-bit bitmap of the postfixes present}
  void *d_rlim = nullptr;
  int rq_bits = 0, rpost_bits = 0;
  int64_t n_rkeys = 0;
  size_t index_bytes = 0;
  // per-class bond data and norm tables for apply_H
  double *d_sqrt = nullptr, *d_rsqrt = nullptr;   // [nsym+1]
  double *d_cs = nullptr;                         // [denom][2] cos, sin of 2 pi k / denom
  uint8_t *d_bond_pos = nullptr;
  // scratch
  double *d_partial = nullptr;
  int n_partial = 0;
  mutable int last_apply_grid = 0;     // grid of the last product (number of dot partials)
  double *h_partial = nullptr;   // pinned
  void *d_stage_x = nullptr, *d_stage_y = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t copy_stream = nullptr;   // device-to-host copies of ed_apply_H_host
  std::vector<cudaEvent_t> chunk_done;  // one per row chunk of ed_apply_H_host
  double build_ms = 0;
};

// error reporting (capi.cu)
int ed_fail(int code, const std::string &msg);
int ed_cuda_fail(cudaError_t e, const char *what);
#define ED_CK(call)                                                   \
  do {                                                                \
    cudaError_t _e = (call);                                          \
    if (_e != cudaSuccess) return ed_cuda_fail(_e, #call);            \
  } while (0)

// kernels.cu / basis.cu entry points used by capi.cu
int ed_build_device(ed_basis *B, cudaStream_t st, int bucket_target);
// mode 0: y = H x (partial: optional <x, y> block partials); mode 1: per-class block partials
// of Re <x | H_c x> (J, Jz: unit couplings) into partial[c * grid + block], y unused
// ylo (fp32 / complex fp32 vectors only, may be null): receives the remainder of rounding
// each y_i to fp32, so that y + ylo holds the product to about 48 bits; zeroed when the
// kernel that runs cannot produce it
int ed_launch_apply(const ed_basis *B, const double *J, const double *Jz, const void *x, void *y,
                    int dtype, int64_t r0, int64_t r1, double *partial, cudaStream_t st,
                    int mode = 0, void *ylo = nullptr);
int ed_launch_find_rep(const ed_basis *B, const uint64_t *states, int64_t n, uint64_t *rep,
                       int32_t *sym, int32_t *phase, int32_t *stab, int64_t *index,
                       cudaStream_t st);
int ed_launch_find_rep_two(const ed_basis *B, const uint64_t *states, int64_t n, uint64_t *rep,
                           int32_t *phase, int32_t *stab, int64_t *index, cudaStream_t st);
int ed_launch_dot(const ed_basis *B, const void *x, const void *y, int dtype, double *partial,
                  int nblk, cudaStream_t st);
// (w, wlo) <- (w + wlo) - a v - b vprev, ||w + wlo||^2 partials; wlo (fp32 vectors, may
// be null) holds the low words of w: on entry those of the product (ed_launch_apply's
// ylo), on exit those of the update
int ed_launch_axpy_norm(const ed_basis *B, void *w, const void *v, const void *vprev, double a,
                        double b, int dtype, double *partial, int nblk, cudaStream_t st,
                        void *wlo = nullptr);
// v <- s (v + vlo), rounded once (vlo: fp32 vectors, may be null)
int ed_launch_scale(const ed_basis *B, void *v, double s, int dtype, cudaStream_t st,
                    const void *vlo = nullptr);
int ed_launch_axpy(const ed_basis *B, void *y, const void *x, double a, int dtype,
                   cudaStream_t st);
int ed_launch_start(const ed_basis *B, void *v, uint64_t seed, int dtype, cudaStream_t st);
int ed_launch_apply_fast(const ed_basis *B, const double *J, const double *Jz, const void *x,
                         void *y, int dtype, int64_t r0, int64_t r1, double *partial,
                         cudaStream_t st, int mode, void *ylo = nullptr, bool *ylo_done = nullptr);
int ed_build_full_table(const uint8_t *d_pbit, const uint8_t *d_flip, int N, int nsym,
                        uint64_t *out, cudaStream_t st);
struct ed_batch;
extern "C" void ed_batch_free(ed_batch *batch);
int ed_launch_count(const ed_basis *B, unsigned long long *d_out, cudaStream_t st);
int ed_launch_copy(const ed_basis *B, void *dst, const void *src, int dtype, cudaStream_t st);
// reorth.cu: one Gram-Schmidt sweep of w against m vectors (base + k * D, or p0 / p1),
// coefficients into c (m, or 2m for complex), ||w||^2 block partials into partial[0, grid)
int ed_reorth_grid(const ed_basis *B);
int ed_launch_reorth_sweep(const ed_basis *B, void *w, const void *base, const void *p0,
                           const void *p1, int m, int dtype, double *partial, double *c,
                           cudaStream_t st, void *wlo = nullptr);
int ed_launch_combine(const ed_basis *B, void *psi, const void *base, int m, const double *s,
                      int dtype, cudaStream_t st);
