// batch.cu -- the product over many symmetry sectors at once, with block vectors.
//
// A batch holds sectors of one lattice (same sites, bonds and couplings) that differ in
// symmetry group, irrep and n_up, and so in dimension (from 0 to ~2e5 on the 5x5 torus).
// One persistent launch covers all of them: every warp takes work items -- (sector,
// block of consecutive rows) -- from a device counter with atomicAdd until none are
// left, so uneven sectors balance themselves and no warp waits on another.  Each row's
// exchange terms go through the representative search and the Limits lookup once and
// are applied to k vectors stored row-major ([D][k], so the k values of a gathered row
// are contiguous), amortising the search over the block.  Vectors are fp32 for real
// sectors and complex fp32 for sectors with complex characters.  After the first call
// the counter reset and the launch are replayed from a captured CUDA graph.  The number
// of rows per work item is picked by timing a few candidates on the first call.
#include "sced_internal.cuh"

#include <algorithm>
#include <cmath>
#include <chrono>
#include <vector>

struct BatchSector {
  DevTables T;
  DevIndex I;
  // fp32 copies of sqrt(t), 1/sqrt(t) and (cos, sin)(2 pi k / denom): converting the fp64
  // tables term by term would run on the FP64 pipe
  const float *sqrt_f, *rsqrt_f, *cs_f;
  const void *x;
  void *y;
  int64_t D;
  int64_t item0;     // first work item of this sector
  int cplx;
  int pad;
};

struct ed_batch {
  int n = 0, k = 1, n_classes = 0, n_bonds = 0;
  std::vector<ed_basis *> bases;
  std::vector<BatchSector> host;
  BatchSector *d_sec = nullptr;
  int64_t *d_item0 = nullptr;
  unsigned long long *d_counter = nullptr;
  uint8_t *d_bond = nullptr;
  float *d_ftab = nullptr;   // the sectors' fp32 norm and phase tables, back to back
  bool all_full = false;     // every sector has a one-sublattice (whole) table
  int cls_off[ED_MAXCLS + 1];
  double jh[ED_MAXCLS], jzq[ED_MAXCLS];
  const uint32_t *nib = nullptr;   // the first basis's nibble tables (shared lattice)
  int n_nib = 0;
  int cls_word[ED_MAXCLS + 1];
  int rows_per_item = 0;   // chosen tile
  int64_t n_items = 0;
  int sm_count = 0;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t done = nullptr;  // recorded after every launch: set_vectors waits on it
  bool vectors_set = false;
};

namespace {

struct BatchParams {
  const BatchSector *sec;
  const int64_t *item0;
  int n_sec;
  int64_t n_items;
  int rows_per_item;
  unsigned long long *counter;
  const uint8_t *bond;
  int n_classes;
  int cls_off[ED_MAXCLS + 1];
  float jh[ED_MAXCLS], jzq[ED_MAXCLS];
  const uint32_t *nib;             // antiparallel masks by nibbles, [word][n_nib][16]
  int n_nib;
  int cls_word[ED_MAXCLS + 1];     // words of class c: [cls_word[c], cls_word[c + 1])
};

__device__ __forceinline__ int sector_of(const BatchParams &P, int64_t item) {
  int lo = 0, hi = P.n_sec - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.item0[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

constexpr int kBatchThreads = 256;

// Index of a representative of a sector with at most 26 sites (whole-table sectors):
// the Limits lookup and bucket search of Sec. IV in 32-bit arithmetic.
__device__ __forceinline__ int64_t lookup_index32(const DevIndex &I, uint32_t s) {
  const uint32_t rk = __ldg(I.top_rank + (s >> (I.N - I.r_bits)));
  if (rk == ED_NO_RANK) return -1;
  if (I.rlim) {   // ranked Limits: first index + rank of the postfix in the bucket's bitmap
    const uint32_t key = (rk << I.rq_bits) | ((s >> I.rpost_bits) & ((1u << I.rq_bits) - 1u));
    const uint4 rec = __ldg(I.rlim + key);
    const uint32_t pf = s & ((1u << I.rpost_bits) - 1u);
    const uint64_t bits = ((uint64_t)rec.w << 32) | rec.z;
    if (!((bits >> pf) & 1ULL)) return -1;
    return (int64_t)rec.x + __popcll(bits & ((1ULL << pf) - 1ULL));
  }
  const uint32_t key = (rk << I.q_bits) | ((s >> I.post_bits) & ((1u << I.q_bits) - 1u));
  uint32_t lo = __ldg(I.limits + key), hi = __ldg(I.limits + key + 1);
  const uint32_t p = s & ((1u << I.post_bits) - 1u);
  const uint32_t end = hi;
  if (I.post_bytes == 1) {
    const uint8_t *post = reinterpret_cast<const uint8_t *>(I.postfix);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if ((uint32_t)__ldg(post + mid) < p) lo = mid + 1; else hi = mid;
    }
    return (lo < end && (uint32_t)__ldg(post + lo) == p) ? (int64_t)lo : -1;
  }
  if (I.post_bytes == 2) {
    const uint16_t *post = reinterpret_cast<const uint16_t *>(I.postfix);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if ((uint32_t)__ldg(post + mid) < p) lo = mid + 1; else hi = mid;
    }
    return (lo < end && (uint32_t)__ldg(post + lo) == p) ? (int64_t)lo : -1;
  }
  const uint32_t *post = reinterpret_cast<const uint32_t *>(I.postfix);
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(post + mid) < p) lo = mid + 1; else hi = mid;
  }
  return (lo < end && __ldg(post + lo) == p) ? (int64_t)lo : -1;
}

// Eight fp32 values (32 bytes, 32-byte aligned) in one 256-bit load: a gathered row of
// k >= 8 real or k >= 4 complex entries then costs one L1 request per lane, not two.
struct F8 { float v[8]; };
__device__ __forceinline__ F8 ld8(const float *p) {
  F8 r;
  asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]),
                 "=f"(r.v[5]), "=f"(r.v[6]), "=f"(r.v[7])
               : "l"(p));
  return r;
}
static_assert(sizeof(BatchSector) % 4 == 0, "sector descriptors are copied as 32-bit words");

// kFull: every sector looks its representatives up in a whole table (one sublattice), so
// the block-wise search is not compiled in and the kernel needs far fewer registers.
// Resident blocks per SM: 6 up to k = 4; 5 for k = 8 (48 registers and a small spill),
// which beat 4 (63 registers) by 5% and 6 (42 registers) by 3%.
template <int K, bool kFull>
__global__ void __launch_bounds__(kBatchThreads, kFull ? (K <= 4 ? 6 : 5) : 1)
    batch_kernel(const BatchParams P) {
  // each warp takes its own work items and keeps its own copy of the sector descriptor,
  // so no warp waits at a block-wide barrier for another warp's rows
  __shared__ BatchSector S_w[kBatchThreads / 32];
  __shared__ uint8_t bond_s[2 * ED_MAXBONDS / 8];
  const int nb = P.cls_off[P.n_classes];
  for (int q = threadIdx.x; q < 2 * nb; q += blockDim.x) bond_s[q] = P.bond[q];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  BatchSector &S = S_w[threadIdx.x >> 5];
  int cur = -1;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(P.counter, 1ULL);
    const int64_t item = (int64_t)__shfl_sync(0xFFFFFFFFu, it, 0);
    if (item >= P.n_items) break;
    const int sid = sector_of(P, item);
    if (sid != cur) {
      __syncwarp();
      const uint32_t *src = reinterpret_cast<const uint32_t *>(P.sec + sid);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&S);
      for (int q = lane; q < (int)(sizeof(BatchSector) / 4); q += 32) dst[q] = __ldg(src + q);
      __syncwarp();
      cur = sid;
    }
    for (int64_t i = (item - S.item0) * P.rows_per_item + lane;
         i < S.D && i < (item - S.item0 + 1) * P.rows_per_item; i += 32) {
      const uint64_t s = __ldcs(reinterpret_cast<const unsigned long long *>(S.I.basis) + i);
      const int ti = __ldcs(S.I.stab + i);
      float yr[K], yi[K];
#pragma unroll
      for (int v = 0; v < K; v++) { yr[v] = 0.f; yi[v] = 0.f; }
      float diag = 0.f;
      for (int c = 0; c < P.n_classes; c++) {
        const float jh = P.jh[c];   // the class's J/2 goes into every term's weight
        int nanti = 0;
        for (int wd = P.cls_word[c]; wd < P.cls_word[c + 1]; wd++) {
          const int b0 = P.cls_off[c] + (wd - P.cls_word[c]) * 32;
          // the row's antiparallel bonds among b0 .. b0 + 31 as a mask (XOR of the state's
          // nibbles' table entries), then one pass per set bit: lanes run the term body
          // together instead of one bond test at a time (with a branch per bond, about
          // half the lanes of every term body were idle)
          uint32_t am = 0;
          const uint32_t *nw = P.nib + (uint32_t)wd * P.n_nib * 16;
          for (int q = 0; q < P.n_nib; q++) am ^= __ldg(nw + q * 16 + (uint32_t)((s >> (4 * q)) & 15u));
          nanti += __popc(am);
          while (am) {
            const int b = b0 + __ffs(am) - 1;
            am &= am - 1;
            const int pa = bond_s[2 * b], pb = bond_s[2 * b + 1];
            const uint64_t s2 = s ^ ((1ULL << pa) | (1ULL << pb));
            RepOut R;
            if constexpr (kFull) {
              const uint64_t e = __ldg(S.T.full + s2);
              R.rep = e & 0xFFFFFFFFull;
              R.g = (int)((e >> 32) & 0xFFFF);
              R.t = (int)(e >> 48);
            } else {
              R = find_rep(S.T, S.T.rep, S.T.sym_off, S.T.sym_list, S.T.dest, S.T.phase, s2);
              if (R.mixed) continue;
            }
            const int64_t j = kFull ? lookup_index32(S.I, (uint32_t)R.rep) : lookup_index(S.I, R.rep);
            if (j < 0) continue;
            float w = jh;
            if (R.t != 1) w *= __ldg(S.sqrt_f + R.t);   // t = |Stab| of the target, mostly 1
            const int ph = __ldg(S.T.phase + R.g);
            if (!S.cplx) {
              const float sg = ph == 0 ? w : -w;
              const float *xr = reinterpret_cast<const float *>(S.x) + j * K;
              if constexpr (K % 8 == 0) {
  #pragma unroll
                for (int v = 0; v < K; v += 8) {
                  const F8 q = ld8(xr + v);
  #pragma unroll
                  for (int u = 0; u < 8; u++) yr[v + u] += sg * q.v[u];
                }
              } else if constexpr (K % 4 == 0) {
  #pragma unroll
                for (int v = 0; v < K; v += 4) {
                  const float4 q = *reinterpret_cast<const float4 *>(xr + v);
                  yr[v] += sg * q.x; yr[v + 1] += sg * q.y; yr[v + 2] += sg * q.z; yr[v + 3] += sg * q.w;
                }
              } else {
  #pragma unroll
                for (int v = 0; v < K; v++) yr[v] += sg * xr[v];
              }
            } else {
              const float cr = __ldg(S.cs_f + 2 * ph) * w, ci = __ldg(S.cs_f + 2 * ph + 1) * w;
              const float2 *xc = reinterpret_cast<const float2 *>(S.x) + j * K;
              if constexpr (K % 4 == 0) {   // four complex entries per 32-byte load
  #pragma unroll
                for (int v = 0; v < K; v += 4) {
                  const F8 q = ld8(reinterpret_cast<const float *>(xc + v));
  #pragma unroll
                  for (int u = 0; u < 4; u++) {
                    yr[v + u] += cr * q.v[2 * u] - ci * q.v[2 * u + 1];
                    yi[v + u] += cr * q.v[2 * u + 1] + ci * q.v[2 * u];
                  }
                }
              } else if constexpr (K % 2 == 0) {   // two complex entries per 16-byte load
  #pragma unroll
                for (int v = 0; v < K; v += 2) {
                  const float4 q = *reinterpret_cast<const float4 *>(xc + v);
                  yr[v] += cr * q.x - ci * q.y;
                  yi[v] += cr * q.y + ci * q.x;
                  yr[v + 1] += cr * q.z - ci * q.w;
                  yi[v + 1] += cr * q.w + ci * q.z;
                }
              } else {
                const float2 q = xc[0];
                yr[0] += cr * q.x - ci * q.y;
                yi[0] += cr * q.y + ci * q.x;
              }
            }
          }
        }
        diag += P.jzq[c] * (float)((P.cls_off[c + 1] - P.cls_off[c]) - 2 * nanti);
      }
      const float rs = __ldg(S.rsqrt_f + ti);
      if (!S.cplx) {
        const float *xi = reinterpret_cast<const float *>(S.x) + i * K;
        float *yo = reinterpret_cast<float *>(S.y) + i * K;
        if constexpr (K % 4 == 0) {
#pragma unroll
          for (int v = 0; v < K; v += 4) {
            const float4 q = *reinterpret_cast<const float4 *>(xi + v);
            *reinterpret_cast<float4 *>(yo + v) =
                make_float4(diag * q.x + yr[v] * rs, diag * q.y + yr[v + 1] * rs,
                            diag * q.z + yr[v + 2] * rs, diag * q.w + yr[v + 3] * rs);
          }
        } else {
#pragma unroll
          for (int v = 0; v < K; v++) yo[v] = diag * xi[v] + yr[v] * rs;
        }
      } else {
        const float2 *xi = reinterpret_cast<const float2 *>(S.x) + i * K;
        float2 *yo = reinterpret_cast<float2 *>(S.y) + i * K;
        if constexpr (K % 2 == 0) {
#pragma unroll
          for (int v = 0; v < K; v += 2) {
            const float4 q = *reinterpret_cast<const float4 *>(xi + v);
            *reinterpret_cast<float4 *>(yo + v) =
                make_float4(diag * q.x + yr[v] * rs, diag * q.y + yi[v] * rs,
                            diag * q.z + yr[v + 1] * rs, diag * q.w + yi[v + 1] * rs);
          }
        } else {
          const float2 q = xi[0];
          yo[0] = make_float2(diag * q.x + yr[0] * rs, diag * q.y + yi[0] * rs);
        }
      }
    }
  }
}

// Work-item prefix sums for a tile, and the sector table, to the device (synchronous).
int upload(ed_batch *Bt, int rows_per_item) {
  std::vector<int64_t> item0(Bt->n);
  int64_t acc = 0;
  for (int s = 0; s < Bt->n; s++) {
    item0[s] = acc;
    Bt->host[s].item0 = acc;
    acc += (Bt->host[s].D + rows_per_item - 1) / rows_per_item;
  }
  Bt->n_items = acc;
  ED_CK(cudaMemcpy(Bt->d_item0, item0.data(), (size_t)Bt->n * 8, cudaMemcpyHostToDevice));
  ED_CK(cudaMemcpy(Bt->d_sec, Bt->host.data(), sizeof(BatchSector) * Bt->n, cudaMemcpyHostToDevice));
  return ED_OK;
}

// Counter reset and the persistent kernel (the part that is captured in the graph).
int launch(ed_batch *Bt, int rows_per_item, cudaStream_t st) {
  BatchParams P{};
  P.sec = Bt->d_sec;
  P.item0 = Bt->d_item0;
  P.n_sec = Bt->n;
  P.n_items = Bt->n_items;
  P.rows_per_item = rows_per_item;
  P.counter = Bt->d_counter;
  P.bond = Bt->d_bond;
  P.n_classes = Bt->n_classes;
  for (int c = 0; c <= Bt->n_classes; c++) P.cls_off[c] = Bt->cls_off[c];
  for (int c = 0; c <= Bt->n_classes; c++) P.cls_word[c] = Bt->cls_word[c];
  P.nib = Bt->nib;
  P.n_nib = Bt->n_nib;
  for (int c = 0; c < Bt->n_classes; c++) { P.jh[c] = (float)Bt->jh[c]; P.jzq[c] = (float)Bt->jzq[c]; }
  ED_CK(cudaMemsetAsync(Bt->d_counter, 0, 8, st));
  const int grid = Bt->sm_count * 8;
  switch (Bt->k * 2 + (Bt->all_full ? 1 : 0)) {
#define BCASE(K)                                                     \
  case 2 * K: batch_kernel<K, false><<<grid, kBatchThreads, 0, st>>>(P); break; \
  case 2 * K + 1: batch_kernel<K, true><<<grid, kBatchThreads, 0, st>>>(P); break;
    BCASE(1)
    BCASE(2)
    BCASE(4)
    BCASE(8)
#undef BCASE
    default: return ed_fail(ED_ERR_INVALID, "block width k must be 1, 2, 4 or 8");
  }
  ED_CK(cudaGetLastError());
  return ED_OK;
}

}  // namespace

extern "C" int ed_batch_create(ed_basis *const *bases, int32_t n, const double *J, const double *Jz,
                               int32_t k, ed_batch **out) {
  if (!bases || n < 1 || !J || !Jz || !out) return ed_fail(ED_ERR_INVALID, "null argument");
  if (k != 1 && k != 2 && k != 4 && k != 8) return ed_fail(ED_ERR_INVALID, "block width k must be 1, 2, 4 or 8");
  *out = nullptr;
  const ed_basis *b0 = bases[0];
  if (!b0) return ed_fail(ED_ERR_INVALID, "null basis");
  if (2 * b0->n_bonds > 2 * ED_MAXBONDS / 8) return ed_fail(ED_ERR_UNSUPPORTED, "at most 512 bonds in a batch");
  for (int s = 1; s < n; s++) {
    if (!bases[s]) return ed_fail(ED_ERR_INVALID, "null basis");
    if (bases[s]->N != b0->N || bases[s]->bond_pos != b0->bond_pos || bases[s]->cls_off != b0->cls_off)
      return ed_fail(ED_ERR_INVALID, "sectors of a batch must share sites, bonds and classes");
  }
  ed_batch *Bt = new (std::nothrow) ed_batch();
  if (!Bt) return ed_fail(ED_ERR_OOM, "host allocation failed");
  Bt->n = n;
  Bt->k = k;
  Bt->n_classes = b0->n_classes;
  Bt->n_bonds = b0->n_bonds;
  Bt->sm_count = b0->sm_count;
  Bt->bases.assign(bases, bases + n);
  for (int c = 0; c <= b0->n_classes; c++) Bt->cls_off[c] = b0->cls_off[c];
  for (int c = 0; c <= b0->n_classes; c++) Bt->cls_word[c] = b0->cls_word[c];
  Bt->nib = b0->d_nib;
  Bt->n_nib = b0->n_nib;
  for (int c = 0; c < b0->n_classes; c++) { Bt->jh[c] = 0.5 * J[c]; Bt->jzq[c] = 0.25 * J[c] * Jz[c]; }
  Bt->host.resize(n);
  std::vector<float> ftab;
  std::vector<size_t> foff(n);
  Bt->all_full = true;
  for (int s = 0; s < n; s++) {
    const ed_basis *B = bases[s];
    BatchSector &S = Bt->host[s];
    S.T = B->T;
    S.I = B->I;
    S.D = B->D;
    S.cplx = B->is_real ? 0 : 1;
    if (!B->T.full) Bt->all_full = false;
    foff[s] = ftab.size();   // sqrt [nsym+1], rsqrt [nsym+1], cs [2 denom]
    for (int t = 0; t <= B->nsym; t++) ftab.push_back((float)std::sqrt((double)t));
    for (int t = 0; t <= B->nsym; t++) ftab.push_back(t ? (float)(1.0 / std::sqrt((double)t)) : 0.f);
    for (int q = 0; q < B->denom; q++) {
      const double a = 2.0 * M_PI * (double)q / (double)B->denom;
      ftab.push_back((float)std::cos(a));
      ftab.push_back((float)std::sin(a));
    }
  }
  if (cudaMalloc(&Bt->d_sec, sizeof(BatchSector) * n) != cudaSuccess ||
      cudaMalloc(&Bt->d_item0, 8 * (size_t)n) != cudaSuccess || cudaMalloc(&Bt->d_counter, 8) != cudaSuccess ||
      cudaMalloc(&Bt->d_bond, std::max<size_t>(b0->bond_pos.size(), 1)) != cudaSuccess ||
      cudaMalloc(&Bt->d_ftab, ftab.size() * 4) != cudaSuccess) {
    cudaGetLastError();
    ed_batch_free(Bt);
    return ed_fail(ED_ERR_OOM, "cannot allocate the batch");
  }
  if (cudaMemcpy(Bt->d_bond, b0->bond_pos.data(), b0->bond_pos.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(Bt->d_ftab, ftab.data(), ftab.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    ed_batch_free(Bt);
    return ed_fail(ED_ERR_CUDA, "cannot upload bonds and tables");
  }
  for (int s = 0; s < n; s++) {
    BatchSector &S = Bt->host[s];
    const int ns = bases[s]->nsym;
    S.sqrt_f = Bt->d_ftab + foff[s];
    S.rsqrt_f = S.sqrt_f + ns + 1;
    S.cs_f = S.rsqrt_f + ns + 1;
  }
  *out = Bt;
  return ED_OK;
}

extern "C" int ed_batch_set_vectors(ed_batch *Bt, void *const *x, void *const *y) {
  if (!Bt || !x || !y) return ed_fail(ED_ERR_INVALID, "null argument");
  for (int s = 0; s < Bt->n; s++) {   // check every sector before changing any
    if (Bt->host[s].D > 0 && (!x[s] || !y[s])) return ed_fail(ED_ERR_INVALID, "null vector of a non-empty sector");
    if (Bt->host[s].D > 0 && Bt->k >= 2 && (((uintptr_t)x[s] | (uintptr_t)y[s]) & 15u))
      return ed_fail(ED_ERR_INVALID, "vectors must be 16-byte aligned for k >= 2");
    const int row_bytes = Bt->k * (Bt->host[s].cplx ? 8 : 4);
    if (Bt->host[s].D > 0 && row_bytes >= 32 && ((uintptr_t)x[s] & 31u))
      return ed_fail(ED_ERR_INVALID, "x must be 32-byte aligned when a row holds 32 bytes or more");
  }
  for (int s = 0; s < Bt->n; s++) {
    Bt->host[s].x = x[s];
    Bt->host[s].y = y[s];
  }
  Bt->vectors_set = true;
  if (Bt->rows_per_item) {   // the kernel reads the sector table from device memory
    // a launch still in flight on the caller's stream reads that table: let it finish
    // before overwriting it (a pageable copy is not ordered against other streams)
    if (Bt->done) ED_CK(cudaEventSynchronize(Bt->done));
    ED_CK(cudaMemcpy(Bt->d_sec, Bt->host.data(), sizeof(BatchSector) * Bt->n, cudaMemcpyHostToDevice));
  }
  return ED_OK;
}

extern "C" int ed_batch_apply(ed_batch *Bt, void *stream) {
  if (!Bt) return ed_fail(ED_ERR_INVALID, "null batch");
  if (!Bt->vectors_set) return ed_fail(ED_ERR_INVALID, "ed_batch_set_vectors first");
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if (!Bt->rows_per_item) {
    // pick the tile: time each candidate (second of two runs) and keep the fastest
    const int cand[] = {32, 64, 128, 256};   // rows per work item of one warp
    struct Events {   // destroyed on every exit path
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      ~Events() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
      }
    } ev;
    ED_CK(cudaEventCreate(&ev.e0));
    ED_CK(cudaEventCreate(&ev.e1));
    float best = 1e30f;
    int pick = 256;
    for (int c : cand) {
      float ms = 0;
      if ((rc = upload(Bt, c))) return rc;
      for (int rep = 0; rep < 2; rep++) {
        ED_CK(cudaEventRecord(ev.e0, st));
        if ((rc = launch(Bt, c, st))) return rc;
        ED_CK(cudaEventRecord(ev.e1, st));
        ED_CK(cudaEventSynchronize(ev.e1));
        ED_CK(cudaEventElapsedTime(&ms, ev.e0, ev.e1));
      }
      if (ms < best) { best = ms; pick = c; }
    }
    Bt->rows_per_item = pick;
    if ((rc = upload(Bt, pick))) return rc;
  }
  if (!Bt->exec) {   // capture counter reset + launch once, replay afterwards
    cudaStream_t cs;
    ED_CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t g;
    ED_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    rc = launch(Bt, Bt->rows_per_item, cs);
    cudaGraph_t gg = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &gg);
    if (rc) { if (gg) cudaGraphDestroy(gg); cudaStreamDestroy(cs); return rc; }
    if (ce != cudaSuccess) { cudaStreamDestroy(cs); return ed_cuda_fail(ce, "cudaStreamEndCapture"); }
    g = gg;
    const cudaError_t ie = cudaGraphInstantiate(&Bt->exec, g, 0);
    cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (ie != cudaSuccess) return ed_cuda_fail(ie, "cudaGraphInstantiate");
  }
  if (!Bt->done) ED_CK(cudaEventCreateWithFlags(&Bt->done, cudaEventDisableTiming));
  ED_CK(cudaGraphLaunch(Bt->exec, st));
  ED_CK(cudaEventRecord(Bt->done, st));
  return ED_OK;
}

extern "C" int ed_batch_info(const ed_batch *Bt, int32_t *rows_per_item, int64_t *n_items) {
  if (!Bt) return ed_fail(ED_ERR_INVALID, "null batch");
  if (rows_per_item) *rows_per_item = Bt->rows_per_item;
  if (n_items) *n_items = Bt->n_items;
  return ED_OK;
}

extern "C" void ed_batch_free(ed_batch *Bt) {
  if (!Bt) return;
  if (Bt->done) {
    cudaEventSynchronize(Bt->done);
    cudaEventDestroy(Bt->done);
  }
  if (Bt->exec) cudaGraphExecDestroy(Bt->exec);
  if (Bt->d_sec) cudaFree(Bt->d_sec);
  if (Bt->d_item0) cudaFree(Bt->d_item0);
  if (Bt->d_counter) cudaFree(Bt->d_counter);
  if (Bt->d_bond) cudaFree(Bt->d_bond);
  if (Bt->d_ftab) cudaFree(Bt->d_ftab);
  delete Bt;
}
