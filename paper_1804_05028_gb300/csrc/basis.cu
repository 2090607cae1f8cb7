// basis.cu -- construction of the symmetry-adapted basis on one GPU (Alg. 3 of
// arXiv:1804.05028 without the process split) and of its prefix index (Basis and
// Limits, Sec. IV).
//
// Enumeration.  A representative's top block equals MinRep = min_X Rep_X, and MinRep
// is its own Rep_0; so only top blocks v with Rep_0(v) == v are enumerated (for a
// single sublattice: every top-P-bit prefix).  For each such v the remaining bits run
// over all patterns with the right number of up spins, in increasing order, split into
// work items of 1024 consecutive ranks.  One warp owns an item; lane l owns ranks
// [32 l, 32 l + 32) of it, so lanes are ordered like the states they produce.
//   pass 1 (count): every kept representative is counted per item;
//   scan: exclusive prefix sums of the item counts give each item's output offset;
//   pass 2 (fill): each lane records a 32-bit hit mask, the warp scans the popcounts,
//   and every lane writes its hits in order -- the output is sorted with no sort.
// Index.  top_rank compresses the occupied values of the top r bits to a dense rank;
// key = rank << q | next q bits; limits[key] = first position whose key is >= key
// (lower bound in the sorted basis); the remaining low bits go to a narrow postfix
// array searched inside the bucket.  Where they fit (4x the basis's bytes, or 64 MB),
// ranked records replace the search: one record per prefix rank and value of every bit
// but the low 6, holding the first basis position and a 64-bit bitmap of the low-6-bit
// values present, so that the index is first + popcount(bitmap below the value) -- one
// 16-byte load.
#include "sced_internal.cuh"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

namespace {

constexpr int kRun = 32;               // ranks per lane
constexpr int kItem = 32 * kRun;       // ranks per work item (one warp)

struct EnumParams {
  DevTables T;
  int S;                 // suffix bits (below the enumerated prefix)
  int n_tops;
  const uint32_t *top_v;       // prefix value
  const uint8_t *top_k;        // up spins in the suffix
  const uint64_t *top_total;   // C(S, k)
  const uint64_t *top_item0;   // first item of this prefix (exclusive scan of item counts)
  uint64_t n_items;
  const uint64_t *binom;       // [65][65]
};

__device__ __forceinline__ uint64_t unrank(const uint64_t *binom, int S, int k, uint64_t r) {
  // r-th S-bit pattern with k ones in increasing order: patterns whose bit pos is 0
  // come first and there are C(pos, k) of them.
  uint64_t x = 0;
  for (int pos = S - 1; pos >= 0 && k > 0; pos--) {
    const uint64_t c = __ldg(binom + pos * 65 + k);
    if (r >= c) { x |= 1ULL << pos; r -= c; k--; }
  }
  return x;
}

// next larger integer with the same number of ones: move the lowest run of ones up by
// one place, keeping all but one of its ones at the bottom
__device__ __forceinline__ uint64_t next_comb(uint64_t x) {
  if (x == 0) return 0;
  const int p = __ffsll((long long)x) - 1;
  const uint64_t y = x >> p;
  const int run = __ffsll((long long)~y) - 1;   // length of the run of ones
  const int q = p + run;                          // first zero above the run
  uint64_t hi = (q >= 64) ? 0 : (x & ~((q >= 63 ? ~0ULL : ((1ULL << (q + 1)) - 1ULL))));
  hi |= (q >= 64) ? 0 : (1ULL << q);
  return hi | ((run - 1) >= 64 ? ~0ULL : ((1ULL << (run - 1)) - 1ULL));
}

__device__ __forceinline__ int find_top(const EnumParams &E, uint64_t item) {
  int lo = 0, hi = E.n_tops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (E.top_item0[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <bool kFill>
__global__ void __launch_bounds__(256) enum_kernel(const EnumParams E, uint32_t *counts,
                                                   const uint64_t *offsets, uint64_t *basis,
                                                   uint16_t *stab) {
  const DevTables &T = E.T;
  const int lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t item = (((uint64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5);
       item < E.n_items; item += nwarps) {
    const int t = find_top(E, item);
    const uint64_t base = (item - E.top_item0[t]) * kItem;
    const uint64_t total = E.top_total[t];
    const int k = E.top_k[t];
    const uint64_t pre = (uint64_t)E.top_v[t] << E.S;
    const uint64_t r0 = base + (uint64_t)lane * kRun;
    int len = 0;
    if (r0 < total) len = (total - r0 < (uint64_t)kRun) ? (int)(total - r0) : kRun;
    uint32_t hits = 0;
    uint64_t x = len ? unrank(E.binom, E.S, k, r0) : 0;
    const uint64_t x0 = x;
    for (int u = 0; u < len; u++) {
      int tt;
      if (is_kept_rep(T, T.rep, T.sym_off, T.sym_list, T.dest, T.phase, pre | x, &tt))
        hits |= 1u << u;
      x = next_comb(x);
    }
    const int c = __popc(hits);
    if (!kFill) {
      int tot = c;
      for (int o = 16; o > 0; o >>= 1) tot += __shfl_down_sync(0xFFFFFFFFu, tot, o);
      if (lane == 0) counts[item] = (uint32_t)tot;
    } else {
      int incl = c;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
      }
      uint64_t w = offsets[item] + (uint64_t)(incl - c);
      x = x0;
      for (int u = 0; u < len; u++) {
        if (hits & (1u << u)) {
          int tt = 0;
          is_kept_rep(T, T.rep, T.sym_off, T.sym_list, T.dest, T.phase, pre | x, &tt);
          basis[w] = pre | x;
          stab[w] = (uint16_t)tt;
          w++;
        }
        x = next_comb(x);
      }
    }
  }
}

// ------------------------------ exclusive scan -------------------------------------
constexpr int kScanBlock = 1024;   // elements per CTA (256 threads x 4)

template <typename T>
__device__ T block_exclusive_scan(T v, T *total) {
  __shared__ T ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const T u = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) ws[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    T a = lane < nw ? ws[lane] : 0;
    T ai = a;
    for (int o = 1; o < 32; o <<= 1) {
      const T u = __shfl_up_sync(0xFFFFFFFFu, ai, o);
      if (lane >= o) ai += u;
    }
    if (lane < nw) ws[lane] = ai - a;
    if (lane == nw - 1) ws[31] = ai;
  }
  __syncthreads();
  const T r = ws[wid] + incl - v;
  if (total) *total = ws[31];
  __syncthreads();
  return r;
}

template <typename TI>
__global__ void scan_block_sums(const TI *in, uint64_t n, uint64_t *sums) {
  const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x * 4;
  uint64_t s = 0;
  for (int u = 0; u < 4; u++) if (b0 + u < n) s += in[b0 + u];
  uint64_t tot;
  block_exclusive_scan<uint64_t>(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename TI>
__global__ void scan_block_apply(const TI *in, uint64_t n, const uint64_t *block_off,
                                 uint64_t *out) {
  const uint64_t b0 = (uint64_t)blockIdx.x * kScanBlock + threadIdx.x * 4;
  uint64_t v[4], s = 0;
  for (int u = 0; u < 4; u++) { v[u] = (b0 + u < n) ? (uint64_t)in[b0 + u] : 0; s += v[u]; }
  uint64_t run = block_exclusive_scan<uint64_t>(s, nullptr) + (block_off ? block_off[blockIdx.x] : 0);
  for (int u = 0; u < 4; u++) {
    if (b0 + u < n) out[b0 + u] = run;
    run += v[u];
  }
}

// out[i] = sum_{j<i} in[j] (uint64), returns the total.  Scratch is allocated here.
template <typename TI>
int exclusive_scan(const TI *in, uint64_t n, uint64_t *out, uint64_t *total, cudaStream_t st) {
  if (n == 0) { *total = 0; return ED_OK; }
  const uint64_t nb = (n + kScanBlock - 1) / kScanBlock;
  if (nb == 1) {
    scan_block_apply<TI><<<1, 256, 0, st>>>(in, n, nullptr, out);
    ED_CK(cudaGetLastError());
  } else {
    uint64_t *sums = nullptr, *offs = nullptr;
    ED_CK(cudaMallocAsync(&sums, nb * 8, st));
    ED_CK(cudaMallocAsync(&offs, nb * 8, st));
    scan_block_sums<TI><<<(unsigned)nb, 256, 0, st>>>(in, n, sums);
    ED_CK(cudaGetLastError());
    uint64_t sub_total = 0;
    int rc = exclusive_scan<uint64_t>(sums, nb, offs, &sub_total, st);
    if (rc) return rc;
    scan_block_apply<TI><<<(unsigned)nb, 256, 0, st>>>(in, n, offs, out);
    ED_CK(cudaGetLastError());
    ED_CK(cudaFreeAsync(sums, st));
    ED_CK(cudaFreeAsync(offs, st));
  }
  // total = out[n-1] + in[n-1]
  uint64_t last_out = 0;
  TI last_in = 0;
  ED_CK(cudaMemcpyAsync(&last_out, out + n - 1, 8, cudaMemcpyDeviceToHost, st));
  ED_CK(cudaMemcpyAsync(&last_in, in + n - 1, sizeof(TI), cudaMemcpyDeviceToHost, st));
  ED_CK(cudaStreamSynchronize(st));
  *total = last_out + (uint64_t)last_in;
  return ED_OK;
}

// ------------------------------ index kernels --------------------------------------
__global__ void mark_tops(const uint64_t *basis, int64_t D, int shift, uint32_t *flags) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D;
       i += (int64_t)gridDim.x * blockDim.x)
    flags[basis[i] >> shift] = 1u;   // every writer stores the same value
}

__global__ void make_rank(const uint32_t *flags, const uint64_t *scan, uint64_t n,
                          uint32_t *top_rank, uint32_t *rank_top) {
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[v]) { top_rank[v] = (uint32_t)scan[v]; rank_top[scan[v]] = (uint32_t)v; }
    else top_rank[v] = ED_NO_RANK;
  }
}

// limits[k] = first position whose key is >= k, by binary search for the smallest state
// carrying key k
__global__ void make_limits(const uint64_t *basis, int64_t D, const uint32_t *rank_top,
                            int r_shift, int q_bits, int post_bits, uint64_t n_keys,
                            uint32_t *limits) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n_keys;
       k += (uint64_t)gridDim.x * blockDim.x) {
    if (k == n_keys) { limits[k] = (uint32_t)D; continue; }
    const uint64_t rk = k >> q_bits;
    const uint64_t mid = k & ((1ULL << q_bits) - 1ULL);
    const uint64_t thr = ((uint64_t)rank_top[rk] << r_shift) | (mid << post_bits);
    int64_t lo = 0, hi = D;
    while (lo < hi) {
      const int64_t m = (lo + hi) >> 1;
      if (basis[m] < thr) lo = m + 1; else hi = m;
    }
    limits[k] = (uint32_t)lo;
  }
}

// Ranked Limits (Sec. IV's Limits with the in-bucket search replaced by a rank): with at
// most 6 postfix bits a bucket is a subset of 64 values, kept as a 64-bit occupancy
// bitmap next to the bucket's first index; the index of a state is then
// start + popcount(bitmap below its postfix).  One 16-byte record per key:
// {start, 0, bitmap low word, bitmap high word}.
__global__ void ranked_starts(const uint64_t *basis, int64_t D, const uint32_t *rank_top,
                              int r_shift, int q_bits, int post_bits, uint64_t n_keys,
                              uint4 *rec) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_keys;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t rk = k >> q_bits;
    const uint64_t mid = k & ((1ULL << q_bits) - 1ULL);
    const uint64_t thr = ((uint64_t)rank_top[rk] << r_shift) | (mid << post_bits);
    int64_t lo = 0, hi = D;
    while (lo < hi) {
      const int64_t m = (lo + hi) >> 1;
      if (basis[m] < thr) lo = m + 1; else hi = m;
    }
    rec[k] = make_uint4((uint32_t)lo, 0u, 0u, 0u);
  }
}

__global__ void ranked_bits(const uint64_t *basis, int64_t D, const uint32_t *top_rank,
                            int r_shift, int q_bits, int post_bits, uint4 *rec) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t s = basis[i];
    const uint64_t rk = top_rank[s >> r_shift];
    const uint64_t k = (rk << q_bits) | ((s >> post_bits) & ((1ULL << q_bits) - 1ULL));
    const uint32_t pf = (uint32_t)(s & ((1ULL << post_bits) - 1ULL));
    unsigned int *w = reinterpret_cast<unsigned int *>(rec + k) + (pf < 32 ? 2 : 3);
    atomicOr(w, 1u << (pf & 31));
  }
}

__global__ void max_bucket_kernel(const uint32_t *limits, uint64_t n_keys,
                                  unsigned long long *out) {
  unsigned long long m = 0;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_keys;
       k += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)(limits[k + 1] - limits[k]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xFFFFFFFFu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

template <typename PT>
__global__ void make_postfix(const uint64_t *basis, int64_t D, uint64_t mask, PT *post) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D;
       i += (int64_t)gridDim.x * blockDim.x)
    post[i] = (PT)(basis[i] & mask);
}

// The whole lookup table of a one-sublattice split: every configuration s < 2^N gets its
// representative (Eq. 4, every group element applied), the first minimising element and
// the number of minimisers.  pbit[g*N + b] is the bit that g carries bit b to.
__global__ void full_table_kernel(const uint8_t *pbit, const uint8_t *flip, int N, int nsym,
                                  uint64_t *out) {
  extern __shared__ uint8_t sp[];
  uint8_t *sf = sp + nsym * N;
  for (int k = threadIdx.x; k < nsym * N; k += blockDim.x) sp[k] = pbit[k];
  for (int k = threadIdx.x; k < nsym; k += blockDim.x) sf[k] = flip ? flip[k] : 0;
  __syncthreads();
  const uint64_t total = 1ULL << N;
  const uint64_t all = total - 1ULL;
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < total;
       s += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t best = ~0ULL;
    uint32_t gb = 0, cnt = 0;
    for (int g = 0; g < nsym; g++) {
      const uint8_t *pg = sp + g * N;
      uint64_t v = 0, m = s;
      while (m) {
        const int b = __ffsll((long long)m) - 1;
        m &= m - 1;
        v |= 1ULL << pg[b];
      }
      if (sf[g]) v ^= all;   // the element also reverses every spin
      if (v < best) { best = v; gb = g; cnt = 1; }
      else if (v == best) cnt++;
    }
    out[s] = best | ((uint64_t)gb << 32) | ((uint64_t)cnt << 48);
  }
}

uint64_t binom_host(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; i++) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

}  // namespace

int ed_build_full_table(const uint8_t *d_pbit, const uint8_t *d_flip, int N, int nsym,
                        uint64_t *out, cudaStream_t st) {
  const size_t sm = (size_t)nsym * N + nsym;
  if (sm > 200 * 1024) return ed_fail(ED_ERR_UNSUPPORTED, "group too large for the one-block table");
  if (sm > 48 * 1024)
    ED_CK(cudaFuncSetAttribute(full_table_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  int dev = 0, nsm = 0;
  ED_CK(cudaGetDevice(&dev));
  ED_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  full_table_kernel<<<nsm * 8, 256, sm, st>>>(d_pbit, d_flip, N, nsym, out);
  ED_CK(cudaGetLastError());
  return ED_OK;
}

// Build Basis, |Stab| and the index on the device.  Tables (B->T) must be in place.
int ed_build_device(ed_basis *B, cudaStream_t st, int bucket_target) {
  const int N = B->N;
  const int P = (B->nsub >= 2) ? B->n : std::min(N, 12);
  const int S = N - P;
  // prefixes to enumerate: Rep_0(v) == v when there are several sublattices
  std::vector<uint32_t> rep0;
  if (B->nsub >= 2) {
    rep0.resize((size_t)1 << B->n);
    ED_CK(cudaMemcpyAsync(rep0.data(), B->d_rep, rep0.size() * 4, cudaMemcpyDeviceToHost, st));
    ED_CK(cudaStreamSynchronize(st));
  }
  std::vector<uint32_t> tv;
  std::vector<uint8_t> tk;
  std::vector<uint64_t> ttot, titem;
  uint64_t n_items = 0;
  for (uint64_t v = 0; v < (1ULL << P); v++) {
    if (B->nsub >= 2 && rep0[v] != v) continue;
    const int k = B->n_up - __builtin_popcountll(v);
    if (k < 0 || k > S) continue;
    const uint64_t tot = binom_host(S, k);
    tv.push_back((uint32_t)v);
    tk.push_back((uint8_t)k);
    ttot.push_back(tot);
    titem.push_back(n_items);
    n_items += (tot + kItem - 1) / kItem;
  }
  B->D = 0;
  if (n_items == 0) return ED_OK;
  std::vector<uint64_t> binom(65 * 65);
  for (int a = 0; a <= 64; a++)
    for (int b = 0; b <= 64; b++) binom[a * 65 + b] = binom_host(a, b);

  uint32_t *d_tv = nullptr, *d_counts = nullptr;
  uint8_t *d_tk = nullptr;
  uint64_t *d_ttot = nullptr, *d_titem = nullptr, *d_binom = nullptr, *d_off = nullptr;
  const size_t nt = tv.size();
  ED_CK(cudaMallocAsync(&d_tv, nt * 4, st));
  ED_CK(cudaMallocAsync(&d_tk, nt, st));
  ED_CK(cudaMallocAsync(&d_ttot, nt * 8, st));
  ED_CK(cudaMallocAsync(&d_titem, nt * 8, st));
  ED_CK(cudaMallocAsync(&d_binom, binom.size() * 8, st));
  ED_CK(cudaMallocAsync(&d_counts, n_items * 4, st));
  ED_CK(cudaMallocAsync(&d_off, n_items * 8, st));
  ED_CK(cudaMemcpyAsync(d_tv, tv.data(), nt * 4, cudaMemcpyHostToDevice, st));
  ED_CK(cudaMemcpyAsync(d_tk, tk.data(), nt, cudaMemcpyHostToDevice, st));
  ED_CK(cudaMemcpyAsync(d_ttot, ttot.data(), nt * 8, cudaMemcpyHostToDevice, st));
  ED_CK(cudaMemcpyAsync(d_titem, titem.data(), nt * 8, cudaMemcpyHostToDevice, st));
  ED_CK(cudaMemcpyAsync(d_binom, binom.data(), binom.size() * 8, cudaMemcpyHostToDevice, st));

  EnumParams E{};
  E.T = B->T;
  E.S = S;
  E.n_tops = (int)nt;
  E.top_v = d_tv;
  E.top_k = d_tk;
  E.top_total = d_ttot;
  E.top_item0 = d_titem;
  E.n_items = n_items;
  E.binom = d_binom;
  const uint64_t warps_needed = n_items;
  uint64_t grid64 = (warps_needed + 7) / 8;
  const uint64_t cap = (uint64_t)B->sm_count * 16;
  if (grid64 > cap) grid64 = cap;
  const unsigned grid = (unsigned)std::max<uint64_t>(grid64, 1);
  enum_kernel<false><<<grid, 256, 0, st>>>(E, d_counts, nullptr, nullptr, nullptr);
  ED_CK(cudaGetLastError());
  uint64_t D = 0;
  int rc = exclusive_scan<uint32_t>(d_counts, n_items, d_off, &D, st);
  if (rc) return rc;
  if (D >= 0xFFFFFFFFull)
    return ed_fail(ED_ERR_UNSUPPORTED, "sector dimension must be below 2^32");
  B->D = (int64_t)D;
  if (D > 0) {
    if (cudaMalloc(&B->d_basis, D * 8) != cudaSuccess || cudaMalloc(&B->d_stab, D * 2) != cudaSuccess) {
      cudaGetLastError();
      return ed_fail(ED_ERR_OOM, "cannot allocate the basis on the device");
    }
    enum_kernel<true><<<grid, 256, 0, st>>>(E, nullptr, d_off, B->d_basis, B->d_stab);
    ED_CK(cudaGetLastError());
  }
  ED_CK(cudaFreeAsync(d_tv, st));
  ED_CK(cudaFreeAsync(d_tk, st));
  ED_CK(cudaFreeAsync(d_ttot, st));
  ED_CK(cudaFreeAsync(d_titem, st));
  ED_CK(cudaFreeAsync(d_binom, st));
  ED_CK(cudaFreeAsync(d_counts, st));
  ED_CK(cudaFreeAsync(d_off, st));
  if (D == 0) return ED_OK;

  // ---- prefix index ----
  const int r_bits = std::min(N, 12);
  const uint64_t ntop = 1ULL << r_bits;
  uint32_t *d_flags = nullptr, *d_rank_top = nullptr;
  uint64_t *d_scan = nullptr;
  ED_CK(cudaMallocAsync(&d_flags, ntop * 4, st));
  ED_CK(cudaMallocAsync(&d_scan, ntop * 8, st));
  ED_CK(cudaMemsetAsync(d_flags, 0, ntop * 4, st));
  const int g1 = B->sm_count * 8;
  mark_tops<<<g1, 256, 0, st>>>(B->d_basis, B->D, N - r_bits, d_flags);
  ED_CK(cudaGetLastError());
  uint64_t R = 0;
  rc = exclusive_scan<uint32_t>(d_flags, ntop, d_scan, &R, st);
  if (rc) return rc;
  if (cudaMalloc(&B->d_top_rank, ntop * 4) != cudaSuccess) {
    cudaGetLastError();
    return ed_fail(ED_ERR_OOM, "cannot allocate the prefix rank table");
  }
  ED_CK(cudaMallocAsync(&d_rank_top, R * 4, st));
  make_rank<<<g1, 256, 0, st>>>(d_flags, d_scan, ntop, B->d_top_rank, d_rank_top);
  ED_CK(cudaGetLastError());
  // q: about bucket_target states per key, limited by the bits left
  int q = 0;
  const double want = (double)D / ((double)std::max(1, bucket_target) * (double)R);
  if (want > 1.0) q = (int)std::lround(std::log2(want));
  q = std::max(0, std::min(q, N - r_bits));
  while ((double)R * std::ldexp(1.0, q) > 4.0e9) q--;   // keys must fit in uint32
  const int post_bits = N - r_bits - q;
  const uint64_t n_keys = R << q;
  if (cudaMalloc(&B->d_limits, (n_keys + 1) * 4) != cudaSuccess) {
    cudaGetLastError();
    return ed_fail(ED_ERR_OOM, "cannot allocate Limits");
  }
  make_limits<<<g1, 256, 0, st>>>(B->d_basis, B->D, d_rank_top, N - r_bits, q, post_bits,
                                    n_keys, B->d_limits);
  ED_CK(cudaGetLastError());
  unsigned long long *d_max = nullptr;
  ED_CK(cudaMallocAsync(&d_max, 8, st));
  ED_CK(cudaMemsetAsync(d_max, 0, 8, st));
  max_bucket_kernel<<<g1, 256, 0, st>>>(B->d_limits, n_keys, d_max);
  ED_CK(cudaGetLastError());
  unsigned long long mb = 0;
  ED_CK(cudaMemcpyAsync(&mb, d_max, 8, cudaMemcpyDeviceToHost, st));
  const int post_bytes = post_bits <= 8 ? 1 : post_bits <= 16 ? 2 : post_bits <= 32 ? 4 : 8;
  const uint64_t pmask = post_bits >= 64 ? ~0ULL : ((1ULL << post_bits) - 1ULL);
  if (post_bytes == 8) {
    B->d_postfix = B->d_basis;   // full states are the postfixes
  } else {
    // 32 bytes of zero padding: the bucket reader loads whole 16-byte chunks
    if (cudaMalloc(&B->d_postfix, (size_t)D * post_bytes + 32) != cudaSuccess) {
      cudaGetLastError();
      return ed_fail(ED_ERR_OOM, "cannot allocate postfixes");
    }
    ED_CK(cudaMemsetAsync((char *)B->d_postfix + (size_t)D * post_bytes, 0, 32, st));
    if (post_bytes == 1)
      make_postfix<uint8_t><<<g1, 256, 0, st>>>(B->d_basis, B->D, pmask, (uint8_t *)B->d_postfix);
    else if (post_bytes == 2)
      make_postfix<uint16_t><<<g1, 256, 0, st>>>(B->d_basis, B->D, pmask, (uint16_t *)B->d_postfix);
    else
      make_postfix<uint32_t><<<g1, 256, 0, st>>>(B->d_basis, B->D, pmask, (uint32_t *)B->d_postfix);
    ED_CK(cudaGetLastError());
  }
  // ranked Limits: 6 postfix bits (fewer when N - r_bits < 6), if the records fit (one
  // record per key; at most 2^32 keys and 16 bytes per key, no more than 4x the basis)
  {
    const int rq = std::max(0, N - r_bits - 6);
    const int rpost = N - r_bits - rq;
    const uint64_t rkeys = R << rq;
    if (rkeys < (1ULL << 32) && rkeys * 16 <= std::max<uint64_t>(4 * (uint64_t)D * 8, 1ULL << 26)) {
      if (cudaMalloc(&B->d_rlim, rkeys * 16) == cudaSuccess) {
        ranked_starts<<<g1, 256, 0, st>>>(B->d_basis, B->D, d_rank_top, N - r_bits, rq, rpost, rkeys,
                                          reinterpret_cast<uint4 *>(B->d_rlim));
        ED_CK(cudaGetLastError());
        ranked_bits<<<g1, 256, 0, st>>>(B->d_basis, B->D, B->d_top_rank, N - r_bits, rq, rpost,
                                        reinterpret_cast<uint4 *>(B->d_rlim));
        ED_CK(cudaGetLastError());
        B->rq_bits = rq;
        B->rpost_bits = rpost;
        B->n_rkeys = (int64_t)rkeys;
      } else {
        cudaGetLastError();   // no ranked index: the kernels search the buckets instead
        B->d_rlim = nullptr;
      }
    }
  }
  ED_CK(cudaFreeAsync(d_flags, st));
  ED_CK(cudaFreeAsync(d_scan, st));
  ED_CK(cudaFreeAsync(d_rank_top, st));
  ED_CK(cudaFreeAsync(d_max, st));
  ED_CK(cudaStreamSynchronize(st));
  B->n_keys = (int64_t)n_keys;
  B->max_bucket = (int64_t)mb;
  B->index_bytes = ntop * 4 + (n_keys + 1) * 4 + (post_bytes == 8 ? 0 : (size_t)D * post_bytes) +
                   (size_t)B->n_rkeys * 16;
  DevIndex &I = B->I;
  I.N = N;
  I.r_bits = r_bits;
  I.q_bits = q;
  I.post_bits = post_bits;
  I.post_bytes = post_bytes;
  I.D = B->D;
  I.basis = B->d_basis;
  I.stab = B->d_stab;
  I.top_rank = B->d_top_rank;
  I.limits = B->d_limits;
  I.postfix = B->d_postfix;
  I.rlim = reinterpret_cast<const uint4 *>(B->d_rlim);
  I.rq_bits = B->rq_bits;
  I.rpost_bits = B->rpost_bits;
  return ED_OK;
}
