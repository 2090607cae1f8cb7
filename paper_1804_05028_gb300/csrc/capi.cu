// capi.cu -- the C ABI of libsced (include/sced.h): descriptor validation, the lookup
// tables of the sublattice coding (Alg. 1 of arXiv:1804.05028), basis life cycle, the
// H x entry points and the Lanczos driver (Sec. IV: the product dominates; dots,
// scalings and the tridiagonal eigenproblem are cheap and stay simple).
#include "sced_internal.cuh"
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

static thread_local std::string g_err;

int ed_fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

int ed_cuda_fail(cudaError_t e, const char *what) {
  g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
  return ED_ERR_CUDA;
}


extern "C" const char *ed_last_error(void) { return g_err.c_str(); }
extern "C" const char *ed_version(void) { return "sced 0.1 (sm_103a)"; }

namespace {

using Perm = std::vector<int32_t>;

uint64_t hash_perm(const int32_t *p, int N) {
  uint64_t h = 1469598103934665603ULL;
  for (int i = 0; i < N; i++) { h ^= (uint64_t)(uint32_t)p[i]; h *= 1099511628211ULL; }
  return h;
}

int mod(int64_t a, int m) { int64_t r = a % m; return (int)(r < 0 ? r + m : r); }

// Validate the descriptor; fills B's problem fields.
int validate(ed_basis *B, const ed_lattice *L, const ed_group *G, const ed_irrep *R, int n_up) {
  if (!L || !G || !R) return ed_fail(ED_ERR_INVALID, "null descriptor");
  const int N = L->n_sites;
  if (N < 1 || N > 64) return ed_fail(ED_ERR_INVALID, "n_sites must be in 1..64");
  if (L->n_sublat < 1 || L->n_sublat > ED_MAXSUB)
    return ed_fail(ED_ERR_INVALID, "n_sublat must be in 1..8");
  if (N % L->n_sublat) return ed_fail(ED_ERR_UNSTABLE, "n_sublat does not divide n_sites");
  const int n = N / L->n_sublat;
  if (L->n_sublat > 1 && n > 20) return ed_fail(ED_ERR_UNSUPPORTED, "sublattice blocks above 20 sites");
  if (L->n_sublat == 1 && N > 26) return ed_fail(ED_ERR_UNSUPPORTED, "a single sublattice needs N <= 26");
  if (L->n_bonds < 1 || L->n_bonds > ED_MAXBONDS || !L->bonds || !L->bond_class)
    return ed_fail(ED_ERR_INVALID, "bonds missing or more than 4096");
  if (L->n_classes < 1 || L->n_classes > ED_MAXCLS)
    return ed_fail(ED_ERR_INVALID, "n_classes must be in 1..8");
  if (G->n_sym < 1 || G->n_sym > 65535 || !G->perm)
    return ed_fail(ED_ERR_INVALID, "n_sym must be in 1..65535");
  if (R->phase_denom < 1 || !R->phase_num) return ed_fail(ED_ERR_INVALID, "bad irrep");
  if (n_up < 0 || n_up > N) return ed_fail(ED_ERR_INVALID, "n_up out of range");
  const int ns = G->n_sym;
  // permutations are bijections
  std::vector<int> seen(N);
  for (int g = 0; g < ns; g++) {
    std::fill(seen.begin(), seen.end(), 0);
    for (int p = 0; p < N; p++) {
      const int q = G->perm[(size_t)g * N + p];
      if (q < 0 || q >= N || seen[q]++) return ed_fail(ED_ERR_INVALID, "permutation " + std::to_string(g) + " is not a bijection");
    }
  }
  // closure and homomorphism: (g h)[p] = g[h[p]], flips add mod 2,
  // phase(g h) = phase(g) + phase(h)
  auto fl = [&](int g) -> int { return G->flip ? (G->flip[g] ? 1 : 0) : 0; };
  bool any_flip = false;
  for (int g = 0; g < ns; g++) any_flip = any_flip || fl(g);
  if (any_flip && 2 * n_up != N)
    return ed_fail(ED_ERR_INVALID, "the spin flip needs n_up = N/2");
  std::unordered_multimap<uint64_t, int> index;
  for (int g = 0; g < ns; g++) index.emplace(hash_perm(G->perm + (size_t)g * N, N) ^ (uint64_t)fl(g), g);
  auto find = [&](const int32_t *p, int f) -> int {
    auto rng = index.equal_range(hash_perm(p, N) ^ (uint64_t)f);
    for (auto it = rng.first; it != rng.second; ++it)
      if (fl(it->second) == f && !memcmp(G->perm + (size_t)it->second * N, p, sizeof(int32_t) * N))
        return it->second;
    return -1;
  };
  bool has_id = false;
  for (int g = 0; g < ns && !has_id; g++) {
    bool id = fl(g) == 0;
    for (int p = 0; p < N && id; p++) id = G->perm[(size_t)g * N + p] == p;
    if (id) {
      has_id = true;
      B->id_g = g;
      if (mod(R->phase_num[g], R->phase_denom)) return ed_fail(ED_ERR_INVALID, "chi(identity) != 1");
    }
  }
  if (!has_id) return ed_fail(ED_ERR_INVALID, "group has no identity");
  if ((double)ns * ns * N <= 4e9) {
    std::vector<int32_t> c(N);
    for (int g = 0; g < ns; g++)
      for (int h = 0; h < ns; h++) {
        for (int p = 0; p < N; p++) c[p] = G->perm[(size_t)g * N + G->perm[(size_t)h * N + p]];
        const int k = find(c.data(), fl(g) ^ fl(h));
        if (k < 0) return ed_fail(ED_ERR_INVALID, "group is not closed");
        if (mod((int64_t)R->phase_num[g] + R->phase_num[h] - R->phase_num[k], R->phase_denom))
          return ed_fail(ED_ERR_INVALID, "characters are not a homomorphism");
      }
  }
  // bonds: distinct endpoints, invariant as a set of (pair, class) under the group
  std::unordered_map<uint64_t, int> bset;
  for (int b = 0; b < L->n_bonds; b++) {
    int a = L->bonds[2 * b], c = L->bonds[2 * b + 1], k = L->bond_class[b];
    if (a < 0 || a >= N || c < 0 || c >= N || a == c) return ed_fail(ED_ERR_INVALID, "bad bond");
    if (k < 0 || k >= L->n_classes) return ed_fail(ED_ERR_INVALID, "bad bond class");
    if (a > c) std::swap(a, c);
    const uint64_t key = ((uint64_t)a << 8) | (uint64_t)c;
    if (bset.count(key)) return ed_fail(ED_ERR_INVALID, "duplicate bond");
    bset[key] = k;
  }
  for (int g = 0; g < ns; g++)
    for (int b = 0; b < L->n_bonds; b++) {
      int a = G->perm[(size_t)g * N + L->bonds[2 * b]], c = G->perm[(size_t)g * N + L->bonds[2 * b + 1]];
      if (a > c) std::swap(a, c);
      auto it = bset.find(((uint64_t)a << 8) | (uint64_t)c);
      if (it == bset.end() || it->second != L->bond_class[b])
        return ed_fail(ED_ERR_INVALID, "bonds are not invariant under the group");
    }
  // sublattice stability (Sec. III B): each g carries each block onto one block
  for (int g = 0; g < ns; g++)
    for (int X = 0; X < L->n_sublat; X++) {
      const int d = G->perm[(size_t)g * N + X * n] / n;
      for (int k = 1; k < n; k++)
        if (G->perm[(size_t)g * N + X * n + k] / n != d)
          return ed_fail(ED_ERR_UNSTABLE, "sublattice split is not stable under group element " + std::to_string(g));
    }
  B->N = N;
  B->nsub = L->n_sublat;
  B->n = n;
  B->nsym = ns;
  B->n_up = n_up;
  B->denom = R->phase_denom;
  B->n_bonds = L->n_bonds;
  B->n_classes = L->n_classes;
  B->perm.assign(G->perm, G->perm + (size_t)ns * N);
  B->flip.assign(ns, 0);
  for (int g = 0; g < ns; g++) B->flip[g] = (uint8_t)fl(g);
  B->phase.resize(ns);
  bool real = true;
  for (int g = 0; g < ns; g++) {
    B->phase[g] = mod(R->phase_num[g], R->phase_denom);
    if (mod(2 * (int64_t)B->phase[g], R->phase_denom)) real = false;
  }
  B->is_real = real;
  // bonds sorted by class, as bit positions
  B->cls_off.assign(B->n_classes + 1, 0);
  B->bond_pos.clear();
  for (int c = 0; c < B->n_classes; c++) {
    B->cls_off[c] = (int)B->bond_pos.size() / 2;
    for (int b = 0; b < L->n_bonds; b++)
      if (L->bond_class[b] == c) {
        B->bond_pos.push_back((uint8_t)(N - 1 - L->bonds[2 * b]));
        B->bond_pos.push_back((uint8_t)(N - 1 - L->bonds[2 * b + 1]));
      }
  }
  B->cls_off[B->n_classes] = (int)B->bond_pos.size() / 2;
  // the same bonds padded per class to whole words of 32 with inert bonds (0, 0)
  B->cls_word.assign(B->n_classes + 1, 0);
  B->bond_pad.clear();
  for (int c = 0; c < B->n_classes; c++) {
    B->cls_word[c] = (int)B->bond_pad.size() / 64;
    for (int b = B->cls_off[c]; b < B->cls_off[c + 1]; b++) {
      B->bond_pad.push_back(B->bond_pos[2 * b]);
      B->bond_pad.push_back(B->bond_pos[2 * b + 1]);
    }
    while (B->bond_pad.size() % 64) B->bond_pad.push_back(0);
  }
  B->cls_word[B->n_classes] = (int)B->bond_pad.size() / 64;
  // the same bonds as (block, bit inside the block) pairs, bit counted from the block's LSB
  B->bond_blk.assign(B->bond_pad.size() / 2, 0);
  for (size_t b = 0; b < B->bond_blk.size(); b++) {
    const int pa = B->bond_pad[2 * b], pb = B->bond_pad[2 * b + 1];
    if (pa == pb) continue;   // inert padding
    const int la = N - 1 - pa, lb = N - 1 - pb;
    B->bond_blk[b] = (uint32_t)(la / n) | ((uint32_t)(lb / n) << 4) |
                     ((uint32_t)(n - 1 - la % n) << 8) | ((uint32_t)(n - 1 - lb % n) << 16);
  }
  // Antiparallel masks by nibbles: bit k of word w is s_a XOR s_b for bond k = (a, b), a
  // linear map of the state's bits over GF(2), so the mask is the XOR over the state's
  // 4-bit nibbles q of nib[(w * n_nib + q) * 16 + nibble_q(s)], where each entry XORs in
  // bit k for every endpoint of bond k that lies in nibble q and is up.
  const int n_words = B->cls_word[B->n_classes];
  B->n_nib = (N + 3) / 4;
  B->nib.assign((size_t)n_words * B->n_nib * 16, 0u);
  for (int w = 0; w < n_words; w++)
    for (int k = 0; k < 32; k++) {
      const int pa = B->bond_pad[2 * (w * 32 + k)], pb = B->bond_pad[2 * (w * 32 + k) + 1];
      if (pa == pb) continue;   // inert padding
      for (int p : {pa, pb})
        for (int v = 0; v < 16; v++)
          if ((v >> (p % 4)) & 1) B->nib[((size_t)w * B->n_nib + p / 4) * 16 + v] ^= 1u << k;
    }
  return ED_OK;
}

// norm and character tables, bond positions (every split)
int build_norm_tables(ed_basis *B, cudaStream_t st) {
  const int ns = B->nsym;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    if (bytes == 0) { *dst = nullptr; return ED_OK; }
    if (cudaMalloc(dst, bytes) != cudaSuccess) { cudaGetLastError(); return ed_fail(ED_ERR_OOM, "cannot allocate lookup tables"); }
    ED_CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
    B->table_bytes += bytes;
    return ED_OK;
  };
  int rc;
  std::vector<double> sq(ns + 1), rs(ns + 1), cs(2 * (size_t)B->denom);
  for (int t = 0; t <= ns; t++) { sq[t] = std::sqrt((double)t); rs[t] = t ? 1.0 / std::sqrt((double)t) : 0.0; }
  for (int k = 0; k < B->denom; k++) {
    const double a = 2.0 * M_PI * (double)k / (double)B->denom;
    cs[2 * k] = std::cos(a);
    cs[2 * k + 1] = std::sin(a);
  }
  if ((rc = up((void **)&B->d_sqrt, sq.data(), sq.size() * 8))) return rc;
  if ((rc = up((void **)&B->d_rsqrt, rs.data(), rs.size() * 8))) return rc;
  if ((rc = up((void **)&B->d_cs, cs.data(), cs.size() * 8))) return rc;
  if ((rc = up((void **)&B->d_bond_pos, B->bond_pos.data(), B->bond_pos.size()))) return rc;
  if ((rc = up((void **)&B->d_bond_pad, B->bond_pad.data(), B->bond_pad.size()))) return rc;
  if ((rc = up((void **)&B->d_bond_blk, B->bond_blk.data(), B->bond_blk.size() * 4))) return rc;
  if ((rc = up((void **)&B->d_nib, B->nib.data(), B->nib.size() * 4))) return rc;
  ED_CK(cudaStreamSynchronize(st));
  return ED_OK;
}

// One sublattice: the whole table (Sec. III, "store the representative and g for every
// state"), built on the device, or shared with another basis of the same group.
int build_full_table(ed_basis *B, cudaStream_t st, const ed_basis *share) {
  const int N = B->N, ns = B->nsym;
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    if (cudaMalloc(dst, bytes) != cudaSuccess) { cudaGetLastError(); return ed_fail(ED_ERR_OOM, "cannot allocate lookup tables"); }
    ED_CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
    B->table_bytes += bytes;
    return ED_OK;
  };
  std::vector<uint8_t> pbit((size_t)ns * N);
  for (int g = 0; g < ns; g++)
    for (int b = 0; b < N; b++)   // bit b is label N-1-b; its image label perm[g][N-1-b]
      pbit[(size_t)g * N + b] = (uint8_t)(N - 1 - B->perm[(size_t)g * N + (N - 1 - b)]);
  int rc;
  if ((rc = up((void **)&B->d_pbit, pbit.data(), pbit.size()))) return rc;
  if ((rc = up((void **)&B->d_phase, B->phase.data(), B->phase.size() * 4))) return rc;
  if ((rc = up((void **)&B->d_flip, B->flip.data(), B->flip.size()))) return rc;
  if (share && share->full_tab && share->N == N && share->nsym == ns && share->perm == B->perm &&
      share->flip == B->flip) {
    B->full_tab = share->full_tab;
  } else {
    uint64_t *t = nullptr;
    if (cudaMalloc(&t, ((size_t)1 << N) * 8) != cudaSuccess) {
      cudaGetLastError();
      return ed_fail(ED_ERR_OOM, "cannot allocate the one-sublattice table");
    }
    B->full_tab = std::shared_ptr<uint64_t>(t, [](uint64_t *q) { cudaFree(q); });
    B->table_bytes += ((size_t)1 << N) * 8;
    if ((rc = ed_build_full_table(B->d_pbit, B->d_flip, N, ns, t, st))) return rc;
  }
  bool triv = true;
  for (int g = 0; g < ns; g++) triv = triv && B->phase[g] == 0;
  DevTables &T = B->T;
  T.N = N; T.nsub = 1; T.n = N; T.nsym = ns; T.denom = B->denom;
  T.chi_trivial = triv ? 1 : 0;
  T.full = B->full_tab.get();
  T.pbit = B->d_pbit;
  T.flip = B->d_flip;
  T.phase = B->d_phase;
  return build_norm_tables(B, st);
}

// Alg. 1: for every sublattice X, substate and group element, SymmetryAction_X; then
// Rep_X = min over G_X (elements carrying X onto block 0) and Sym_X = its minimisers.
int build_tables(ed_basis *B, cudaStream_t st, const ed_basis *share) {
  const int N = B->N, nsub = B->nsub, n = B->n, ns = B->nsym;
  if (nsub == 1) return build_full_table(B, st, share);
  const size_t nn = (size_t)1 << n;
  std::vector<uint8_t> dest((size_t)ns * nsub);
  for (int g = 0; g < ns; g++)
    for (int X = 0; X < nsub; X++) dest[(size_t)g * nsub + X] = (uint8_t)(B->perm[(size_t)g * N + X * n] / n);
  const bool u16 = n <= 16;
  const bool need_action = nsub > 1;
  std::vector<uint32_t> act32;
  std::vector<uint16_t> act16;
  if (need_action) {
    if (u16) act16.resize((size_t)nsub * nn * ns); else act32.resize((size_t)nsub * nn * ns);
  }
  std::vector<uint32_t> rep((size_t)nsub * nn, 0xFFFFFFFFu);
  std::vector<uint32_t> symoff((size_t)nsub * (nn + 1));
  std::vector<uint16_t> symlist;
  std::vector<uint32_t> val(ns);
  std::vector<int> pos(n);
  for (int X = 0; X < nsub; X++) {
    std::vector<std::vector<int>> posg(ns, std::vector<int>(n));
    for (int g = 0; g < ns; g++)
      for (int k = 0; k < n; k++) posg[g][k] = B->perm[(size_t)g * N + X * n + k] % n;
    for (size_t sub = 0; sub < nn; sub++) {
      uint32_t best = 0xFFFFFFFFu;
      for (int g = 0; g < ns; g++) {
        uint32_t v = 0;
        for (int k = 0; k < n; k++)
          if ((sub >> (n - 1 - k)) & 1) v |= 1u << (n - 1 - posg[g][k]);
        if (B->flip[g]) v ^= (uint32_t)(nn - 1);   // the element also reverses every spin
        val[g] = v;
        if (need_action) {
          const size_t o = ((size_t)X * nn + sub) * ns + g;
          if (u16) act16[o] = (uint16_t)v; else act32[o] = v;
        }
        if (dest[(size_t)g * nsub + X] == 0 && v < best) best = v;
      }
      rep[(size_t)X * nn + sub] = best;
      symoff[(size_t)X * (nn + 1) + sub] = (uint32_t)symlist.size();
      for (int g = 0; g < ns; g++)
        if (dest[(size_t)g * nsub + X] == 0 && val[g] == best) symlist.push_back((uint16_t)g);
    }
    symoff[(size_t)X * (nn + 1) + nn] = (uint32_t)symlist.size();
  }
  if (symlist.size() >= 0xFFFFFFFFull) return ed_fail(ED_ERR_UNSUPPORTED, "Sym lists too long");
  // Two-level search tables.  Sym_Y(s_Y) is the coset K_R h of the stabiliser
  // K_R = {k in G_0 : k R = R} of R = Rep_Y(s_Y), h its first element; so
  // min over Sym_Y of g s = min over k in K_R of k (h s), and the inner minimum is again
  // a sublattice-coding problem, for the group K_R on blocks 1.. (Eqs. 8-10 with
  // block 1 in the role of block 0).  Level 1 keeps only (Rep_X, first element of
  // Sym_X); level 2 holds, for every R with a nontrivial K_R, Rep^R_X and Sym^R_X.
  // Entries: level 1 rep | h << 12;  level 2 rep | first << 12 | count << 24, and the
  // offset of the full list; a block that no element of K_R carries onto block 1 gets the
  // sentinel rep 0xFFF (above every n-bit value).  Needs n <= 11, |G| <= 4096, lists <=
  // 255 entries and fewer than 255 such R.
  std::vector<uint32_t> e1, e2, off2;
  std::vector<uint16_t> list2;
  std::vector<uint8_t> rid, src((size_t)ns * nsub, 0);
  for (int g = 0; g < ns; g++)
    for (int X = 0; X < nsub; X++) src[(size_t)g * nsub + dest[(size_t)g * nsub + X]] = (uint8_t)X;
  bool two = need_action && nsub <= 4 && n <= 11 && ns <= 4096;
  int nrid = 0;
  if (two) {
    e1.resize((size_t)nsub * nn);
    for (int X = 0; X < nsub; X++)
      for (size_t sub = 0; sub < nn; sub++)
        e1[(size_t)X * nn + sub] = rep[(size_t)X * nn + sub] |
                                   ((uint32_t)symlist[symoff[(size_t)X * (nn + 1) + sub]] << 12);
    rid.assign(nn, 0xFF);
    std::vector<int> G0;
    for (int g = 0; g < ns; g++) if (dest[(size_t)g * nsub] == 0) G0.push_back(g);
    for (size_t R = 0; R < nn && two; R++) {
      if (rep[R] != R) continue;   // only Rep_0 fixed points can be MinRep
      std::vector<int> K;
      for (int g : G0) if (act16[((size_t)0 * nn + R) * ns + g] == R) K.push_back(g);
      if (K.size() <= 1) continue;
      if (nrid >= 254) { two = false; break; }
      rid[R] = (uint8_t)nrid++;
      for (int d = 1; d < nsub && two; d++)
        for (size_t sub = 0; sub < nn; sub++) {
          uint32_t best = 0xFFFFFFFFu;
          for (int k : K)
            if (dest[(size_t)k * nsub + d] == 1) best = std::min<uint32_t>(best, act16[((size_t)d * nn + sub) * ns + k]);
          const uint32_t o = (uint32_t)list2.size();
          for (int k : K)
            if (dest[(size_t)k * nsub + d] == 1 && act16[((size_t)d * nn + sub) * ns + k] == best) list2.push_back((uint16_t)k);
          const uint32_t cnt = (uint32_t)list2.size() - o;
          if (cnt > 255) { two = false; break; }
          e2.push_back(cnt ? (best | ((uint32_t)list2[o] << 12) | (cnt << 24)) : 0xFFFu);
          off2.push_back(o);
        }
    }
  }
  auto up = [&](void **dst, const void *src, size_t bytes) -> int {
    if (bytes == 0) { *dst = nullptr; return ED_OK; }
    if (cudaMalloc(dst, bytes) != cudaSuccess) { cudaGetLastError(); return ed_fail(ED_ERR_OOM, "cannot allocate lookup tables"); }
    ED_CK(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, st));
    B->table_bytes += bytes;
    return ED_OK;
  };
  int rc;
  if ((rc = up((void **)&B->d_rep, rep.data(), rep.size() * 4))) return rc;
  if ((rc = up((void **)&B->d_sym_off, symoff.data(), symoff.size() * 4))) return rc;
  if (symlist.empty()) symlist.push_back(0);
  if ((rc = up((void **)&B->d_sym_list, symlist.data(), symlist.size() * 2))) return rc;
  if ((rc = up((void **)&B->d_dest, dest.data(), dest.size()))) return rc;
  if ((rc = up((void **)&B->d_phase, B->phase.data(), B->phase.size() * 4))) return rc;
  if ((rc = up((void **)&B->d_src, src.data(), src.size()))) return rc;
  if (two) {
    if (e2.empty()) { e2.push_back(0xFFFu); off2.push_back(0); }
    if (list2.empty()) list2.push_back(0);
    if ((rc = up((void **)&B->d_e1, e1.data(), e1.size() * 4))) return rc;
    if ((rc = up((void **)&B->d_rid, rid.data(), rid.size()))) return rc;
    if ((rc = up((void **)&B->d_e2, e2.data(), e2.size() * 4))) return rc;
    if ((rc = up((void **)&B->d_off2, off2.data(), off2.size() * 4))) return rc;
    if ((rc = up((void **)&B->d_list2, list2.data(), list2.size() * 2))) return rc;
    B->two_level = true;
    B->n_rid = nrid;
  }
  if (need_action) {
    if (u16) { if ((rc = up(&B->d_action, act16.data(), act16.size() * 2))) return rc; }
    else { if ((rc = up(&B->d_action, act32.data(), act32.size() * 4))) return rc; }
  }
  B->sym_list_len = symlist.size();
  DevTables &T = B->T;
  T.N = N; T.nsub = nsub; T.n = n; T.nsym = ns; T.denom = B->denom;
  T.action_u16 = u16 ? 1 : 0;
  T.rep = B->d_rep; T.sym_off = B->d_sym_off; T.sym_list = B->d_sym_list;
  T.action = B->d_action; T.dest = B->d_dest; T.phase = B->d_phase;
  T.chi_trivial = 0;
  return build_norm_tables(B, st);
}

void free_all(ed_basis *B) {
  void *ptrs[] = {B->d_rep, B->d_sym_off, B->d_sym_list, B->d_action, B->d_dest, B->d_phase,
                  B->d_src, B->d_e1, B->d_rid, B->d_e2, B->d_off2, B->d_list2, B->d_bond_pad,
                  B->d_bond_blk, B->d_nib, B->d_pbit, B->d_flip,
                  B->d_basis, B->d_stab, B->d_top_rank, B->d_limits, B->d_rlim,
                  B->d_postfix == B->d_basis ? nullptr : B->d_postfix,
                  B->d_sqrt, B->d_rsqrt, B->d_cs, B->d_bond_pos, B->d_partial,
                  B->d_stage_x, B->d_stage_y};
  for (void *p : ptrs) if (p) cudaFree(p);
  if (B->h_partial) cudaFreeHost(B->h_partial);
  B->full_tab.reset();
  for (cudaEvent_t e : B->chunk_done) cudaEventDestroy(e);
  B->chunk_done.clear();
  if (B->copy_stream) cudaStreamDestroy(B->copy_stream);
  B->copy_stream = nullptr;
}

size_t elem_size(int dtype) {
  switch (dtype) {
    case ED_F64: return 8;
    case ED_F32: return 4;
    case ED_C128: return 16;
    case ED_C64: return 8;
  }
  return 0;
}

int check_dtype(const ed_basis *B, int dtype) {
  if (!elem_size(dtype)) return ed_fail(ED_ERR_INVALID, "unknown dtype");
  const bool cplx = dtype == ED_C128 || dtype == ED_C64;
  if (!B->is_real && !cplx) return ed_fail(ED_ERR_INVALID, "complex characters need a complex dtype");
  return ED_OK;
}

// sum of per-block partials, in block order (deterministic)
int reduce_partials(const ed_basis *B, const double *d_part, int nblk, bool cplx, cudaStream_t st,
                    double *re, double *im) {
  const int cnt = cplx ? 2 * nblk : nblk;
  ED_CK(cudaMemcpyAsync(B->h_partial, d_part, (size_t)cnt * 8, cudaMemcpyDeviceToHost, st));
  ED_CK(cudaStreamSynchronize(st));
  double a = 0, b = 0;
  for (int k = 0; k < nblk; k++) a += B->h_partial[k];
  if (cplx) for (int k = 0; k < nblk; k++) b += B->h_partial[nblk + k];
  *re = a;
  if (im) *im = b;
  return ED_OK;
}

// ---------------- symmetric tridiagonal helpers (host, double) ----------------------
// number of eigenvalues below x (Sturm sequence of the LDL^T factorisation)
int sturm_count(const std::vector<double> &a, const std::vector<double> &b, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; i++) {
    const double bb = i ? b[i - 1] * b[i - 1] : 0.0;
    q = a[i] - x - (i ? bb / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0) cnt++;
  }
  return cnt;
}

double lowest_eigenvalue(const std::vector<double> &a, const std::vector<double> &b, int m) {
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; i++) {
    const double r = (i ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count(a, b, m, mid) >= 1) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// eigenvector of T for eigenvalue lam by inverse iteration; each solve is Gaussian
// elimination of the tridiagonal T - shift with partial pivoting (one extra band)
std::vector<double> tri_eigvec(const std::vector<double> &a, const std::vector<double> &b, int m,
                               double lam) {
  std::vector<double> z(m, 1.0);
  if (m == 1) return z;
  const double shift = lam - 1e-10 * std::max(1.0, std::fabs(lam));
  for (int iter = 0; iter < 4; iter++) {
    std::vector<double> d(m), u(m, 0.0), u2(m, 0.0), l(m, 0.0), r = z;
    for (int i = 0; i < m; i++) d[i] = a[i] - shift;
    for (int i = 0; i + 1 < m; i++) { u[i] = b[i]; l[i] = b[i]; }
    for (int i = 0; i + 1 < m; i++) {
      if (std::fabs(d[i]) >= std::fabs(l[i])) {
        if (d[i] == 0.0) d[i] = 1e-300;
        const double f = l[i] / d[i];
        d[i + 1] -= f * u[i];
        r[i + 1] -= f * r[i];
      } else {   // swap rows i and i+1, then eliminate
        const double f = d[i] / l[i];
        d[i] = l[i];
        const double t = d[i + 1];
        d[i + 1] = u[i] - f * t;
        u[i] = t;
        if (i + 2 < m) { u2[i] = u[i + 1]; u[i + 1] = -f * u2[i]; }
        std::swap(r[i], r[i + 1]);
        r[i + 1] -= f * r[i];
      }
    }
    if (d[m - 1] == 0.0) d[m - 1] = 1e-300;
    z[m - 1] = r[m - 1] / d[m - 1];
    z[m - 2] = (r[m - 2] - u[m - 2] * z[m - 1]) / d[m - 2];
    for (int i = m - 3; i >= 0; i--) z[i] = (r[i] - u[i] * z[i + 1] - u2[i] * z[i + 2]) / d[i];
    double nrm = 0;
    for (double v : z) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (double &v : z) v /= nrm;
  }
  return z;
}

}  // namespace

// --------------------------------------------------------------------------------------
extern "C" int ed_build_basis(const ed_lattice *L, const ed_group *G, const ed_irrep *R,
                              int32_t n_up, const ed_basis_opts *opts, void *stream,
                              ed_basis **out) {
  if (!out) return ed_fail(ED_ERR_INVALID, "out is null");
  *out = nullptr;
  auto t0 = std::chrono::steady_clock::now();
  ed_basis *B = new (std::nothrow) ed_basis();
  if (!B) return ed_fail(ED_ERR_OOM, "host allocation failed");
  int rc = validate(B, L, G, R, n_up);
  if (rc) { delete B; return rc; }
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&B->device);
  if (e != cudaSuccess) { delete B; return ed_cuda_fail(e, "cudaGetDevice"); }
  e = cudaDeviceGetAttribute(&B->sm_count, cudaDevAttrMultiProcessorCount, B->device);
  if (e != cudaSuccess) { delete B; return ed_cuda_fail(e, "cudaDeviceGetAttribute"); }
  if ((rc = build_tables(B, st, opts ? opts->share_tables : nullptr))) { free_all(B); delete B; return rc; }
  const int bucket = (opts && opts->bucket_target > 0) ? opts->bucket_target : 1;
  if ((rc = ed_build_device(B, st, bucket))) { free_all(B); delete B; return rc; }
  B->n_partial = ED_MAXCLS * B->sm_count * 8;   // per-class partials of the widest grid
  if (cudaMalloc(&B->d_partial, (size_t)B->n_partial * 8) != cudaSuccess ||
      cudaMallocHost(&B->h_partial, (size_t)B->n_partial * 8) != cudaSuccess) {
    cudaGetLastError();
    free_all(B);
    delete B;
    return ed_fail(ED_ERR_OOM, "cannot allocate reduction scratch");
  }
  B->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  *out = B;
  return ED_OK;
}

extern "C" void ed_free_basis(ed_basis *B) {
  if (!B) return;
  free_all(B);
  delete B;
}

extern "C" int ed_basis_info(const ed_basis *B, ed_basis_info_t *info) {
  if (!B || !info) return ed_fail(ED_ERR_INVALID, "null argument");
  memset(info, 0, sizeof(*info));
  info->dim = B->D;
  info->is_real = B->is_real ? 1 : 0;
  info->n_sites = B->N;
  info->n_sublat = B->nsub;
  info->n_sym = B->nsym;
  info->n_up = B->n_up;
  info->n_bonds = B->n_bonds;
  info->n_classes = B->n_classes;
  info->prefix_rank_bits = B->I.r_bits;
  info->prefix_raw_bits = B->I.q_bits;
  info->postfix_bits = B->I.post_bits;
  info->n_keys = B->n_keys;
  info->max_bucket = B->max_bucket;
  info->table_bytes = (int64_t)B->table_bytes;
  info->index_bytes = (int64_t)B->index_bytes;
  info->basis_bytes = B->D * 10;
  info->sym_list_len = (int64_t)B->sym_list_len;
  info->build_ms = B->build_ms;
  return ED_OK;
}

extern "C" int ed_basis_export(const ed_basis *B, uint64_t *states, uint16_t *stab) {
  if (!B) return ed_fail(ED_ERR_INVALID, "null basis");
  if (B->D == 0) return ED_OK;
  if (states) ED_CK(cudaMemcpy(states, B->d_basis, (size_t)B->D * 8, cudaMemcpyDeviceToHost));
  if (stab) ED_CK(cudaMemcpy(stab, B->d_stab, (size_t)B->D * 2, cudaMemcpyDeviceToHost));
  return ED_OK;
}

extern "C" int ed_find_rep(const ed_basis *B, const uint64_t *states, int64_t n, int32_t method,
                           uint64_t *rep, int32_t *sym, int32_t *phase, int32_t *stab,
                           int64_t *index, void *stream) {
  if (!B || (n > 0 && !states)) return ed_fail(ED_ERR_INVALID, "null argument");
  if (method == 0)
    return ed_launch_find_rep(B, states, n, rep, sym, phase, stab, index, (cudaStream_t)stream);
  if (method != 1) return ed_fail(ED_ERR_INVALID, "method must be 0 or 1");
  if (sym && n > 0) ED_CK(cudaMemsetAsync(sym, 0xFF, (size_t)n * 4, (cudaStream_t)stream));
  return ed_launch_find_rep_two(B, states, n, rep, phase, stab, index, (cudaStream_t)stream);
}

extern "C" int ed_apply_H_rows(const ed_basis *B, const double *J, const double *Jz,
                               const void *x, void *y, int32_t dtype, int64_t r0, int64_t r1,
                               void *stream) {
  if (!B || !J || !Jz) return ed_fail(ED_ERR_INVALID, "null argument");
  int rc = check_dtype(B, dtype);
  if (rc) return rc;
  if (r0 < 0 || r1 > B->D || r0 > r1) return ed_fail(ED_ERR_INVALID, "row range outside the basis");
  if (r1 == r0) return ED_OK;
  if (!x || !y) return ed_fail(ED_ERR_INVALID, "null vector");
  return ed_launch_apply(B, J, Jz, x, y, dtype, r0, r1, nullptr, (cudaStream_t)stream);
}

extern "C" int ed_apply_H(const ed_basis *B, const double *J, const double *Jz, const void *x,
                          void *y, int32_t dtype, void *stream) {
  if (!B) return ed_fail(ED_ERR_INVALID, "null basis");
  return ed_apply_H_rows(B, J, Jz, x, y, dtype, 0, B->D, stream);
}

extern "C" int ed_apply_H_host(ed_basis *B, const double *J, const double *Jz, const void *xh,
                               void *yh, int32_t dtype, void *stream) {
  if (!B || !J || !Jz) return ed_fail(ED_ERR_INVALID, "null argument");
  int rc = check_dtype(B, dtype);
  if (rc) return rc;
  if (B->D == 0) return ED_OK;
  if (!xh || !yh) return ed_fail(ED_ERR_INVALID, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = elem_size(dtype) * (size_t)B->D;
  if (B->stage_bytes < bytes) {
    if (B->d_stage_x) cudaFree(B->d_stage_x);
    if (B->d_stage_y) cudaFree(B->d_stage_y);
    B->d_stage_x = B->d_stage_y = nullptr;
    B->stage_bytes = 0;
    if (cudaMalloc(&B->d_stage_x, bytes) != cudaSuccess || cudaMalloc(&B->d_stage_y, bytes) != cudaSuccess) {
      cudaGetLastError();
      return ed_fail(ED_ERR_OOM, "cannot allocate staging vectors");
    }
    B->stage_bytes = bytes;
  }
  // The product needs the whole of x, so the host-to-device copy comes first.  y goes
  // back in row chunks: the copy of chunk c (on a second stream) runs while chunk c+1
  // is computed, so only the last chunk's copy is exposed.
  const int64_t kMinChunkRows = (int64_t)1 << 24;   // ~64 rows per thread: chunk tails stay small
  const int n_chunks = (int)std::min<int64_t>(8, std::max<int64_t>(1, B->D / kMinChunkRows));
  if (n_chunks > 1 && !B->copy_stream) {
    ED_CK(cudaStreamCreateWithFlags(&B->copy_stream, cudaStreamNonBlocking));
  }
  while ((int)B->chunk_done.size() < n_chunks) {
    cudaEvent_t e;
    ED_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    B->chunk_done.push_back(e);
  }
  const size_t es = elem_size(dtype);
  ED_CK(cudaMemcpyAsync(B->d_stage_x, xh, bytes, cudaMemcpyHostToDevice, st));
  // on an error after some chunks were queued, their copies into the caller's y are
  // drained before the call returns
  auto drain = [&](int code) {
    if (n_chunks > 1) cudaStreamSynchronize(B->copy_stream);
    cudaStreamSynchronize(st);
    return code;
  };
  for (int c = 0; c < n_chunks; c++) {
    const int64_t r0 = B->D * c / n_chunks, r1 = B->D * (c + 1) / n_chunks;
    char *yd = (char *)B->d_stage_y + (size_t)r0 * es;
    if ((rc = ed_launch_apply(B, J, Jz, B->d_stage_x, yd, dtype, r0, r1, nullptr, st))) return drain(rc);
    cudaError_t e;
    if (n_chunks == 1) {
      e = cudaMemcpyAsync(yh, B->d_stage_y, bytes, cudaMemcpyDeviceToHost, st);
      if (e != cudaSuccess) return drain(ed_cuda_fail(e, "cudaMemcpyAsync"));
    } else {
      if ((e = cudaEventRecord(B->chunk_done[c], st)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(B->copy_stream, B->chunk_done[c], 0)) != cudaSuccess ||
          (e = cudaMemcpyAsync((char *)yh + (size_t)r0 * es, yd, (size_t)(r1 - r0) * es,
                               cudaMemcpyDeviceToHost, B->copy_stream)) != cudaSuccess)
        return drain(ed_cuda_fail(e, "chunked copy of y"));
    }
  }
  if (n_chunks > 1) ED_CK(cudaStreamSynchronize(B->copy_stream));
  ED_CK(cudaStreamSynchronize(st));
  return ED_OK;
}

extern "C" int ed_dot(ed_basis *B, const void *x, const void *y, int32_t dtype, double *out,
                      void *stream) {
  if (!B || !out) return ed_fail(ED_ERR_INVALID, "null argument");
  if (!elem_size(dtype)) return ed_fail(ED_ERR_INVALID, "unknown dtype");
  out[0] = out[1] = 0;
  if (B->D == 0) return ED_OK;
  if (!x || !y) return ed_fail(ED_ERR_INVALID, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  const int nblk = B->n_partial / 2;
  int rc = ed_launch_dot(B, x, y, dtype, B->d_partial, nblk, st);
  if (rc) return rc;
  const bool cplx = dtype == ED_C128 || dtype == ED_C64;
  return reduce_partials(B, B->d_partial, nblk, cplx, st, &out[0], &out[1]);
}

extern "C" int ed_count_terms(const ed_basis *B, int64_t *n_flip, int64_t *n_offdiag,
                              void *stream) {
  if (!B || !n_flip || !n_offdiag) return ed_fail(ED_ERR_INVALID, "null argument");
  *n_flip = *n_offdiag = 0;
  if (B->D == 0) return ED_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *d = nullptr, h[2] = {0, 0};
  ED_CK(cudaMallocAsync(&d, 16, st));
  ED_CK(cudaMemsetAsync(d, 0, 16, st));
  int rc = ed_launch_count(B, d, st);
  if (rc) return rc;
  ED_CK(cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, st));
  ED_CK(cudaFreeAsync(d, st));
  ED_CK(cudaStreamSynchronize(st));
  *n_flip = (int64_t)h[0];
  *n_offdiag = (int64_t)h[1];
  return ED_OK;
}

extern "C" int ed_expect_classes(ed_basis *B, const double *Jz, const void *x, int32_t dtype,
                                 double *out, void *stream) {
  if (!B || !Jz || !out) return ed_fail(ED_ERR_INVALID, "null argument");
  int rc = check_dtype(B, dtype);
  if (rc) return rc;
  for (int c = 0; c < B->n_classes; c++) out[c] = 0.0;
  if (B->D == 0) return ED_OK;
  if (!x) return ed_fail(ED_ERR_INVALID, "null vector");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> unit(B->n_classes, 1.0);
  if ((rc = ed_launch_apply(B, unit.data(), Jz, x, nullptr, dtype, 0, B->D, B->d_partial, st, 1))) return rc;
  const int g = B->last_apply_grid;
  ED_CK(cudaMemcpyAsync(B->h_partial, B->d_partial, (size_t)B->n_classes * g * 8,
                        cudaMemcpyDeviceToHost, st));
  ED_CK(cudaStreamSynchronize(st));
  for (int c = 0; c < B->n_classes; c++) {
    double a = 0;
    for (int k = 0; k < g; k++) a += B->h_partial[(size_t)c * g + k];
    out[c] = a;
  }
  return ED_OK;
}

// --------------------------------------------------------------------------------------
// Lanczos
// --------------------------------------------------------------------------------------
namespace {

struct LanczosRun {
  ed_basis *B;
  const double *J, *Jz;
  int dtype;
  bool cplx;
  cudaStream_t st;
  void *v[3];        // rotating: vprev, v, w (local or no reorthogonalisation)
  void *ylo = nullptr;     // fp32 vectors: low words of the product (w is a double-float pair)
  bool own_ylo = false;
  char *store = nullptr;   // full reorthogonalisation: slot k holds v_k
  int store_slots = 0;
  int reorth = ED_REORTH_LOCAL;
  double *d_ro = nullptr;  // sweep partials [m_cap * P * grid], then coefficients [m_cap * P]
  size_t ro_coef_off = 0;
  cudaEvent_t e0, e1, r0, r1;
  double ms_apply = 0, ms_reorth = 0;
  void *slot(int k) const { return store + (size_t)k * elem_bytes(); }
  size_t elem_bytes() const {
    return (dtype == ED_F64 ? 8 : dtype == ED_F32 ? 4 : dtype == ED_C128 ? 16 : 8) * (size_t)B->D;
  }
};

// The sweeps of step j after the three-term update of w.  Local: one sweep against v_j and
// v_{j-1} (the second Gram-Schmidt pass of the recurrence's own projection).  Full: two
// sweeps against every stored v_0 .. v_j (classical Gram-Schmidt, twice).  *corr gets
// Re <v_j, w> summed over the sweeps (added to alpha_j so that the tridiagonal matrix stays
// the projection of H), *b2 the new ||w||^2; both only when want_host (the replay pass
// reuses the stored alpha and beta and skips the copies).
int reorth_step(LanczosRun &L, int j, void *w, const void *v, const void *vprev, bool want_host,
                double *corr, double *b2) {
  ed_basis *B = L.B;
  const int P = L.cplx ? 2 : 1;
  const int grid = ed_reorth_grid(B);
  double *c = L.d_ro + L.ro_coef_off;
  ED_CK(cudaEventRecord(L.r0, L.st));
  const int sweeps = L.reorth == ED_REORTH_FULL ? 2 : 1;
  double cj = 0.0;
  for (int sw = 0; sw < sweeps; sw++) {
    int rc, jj;
    if (L.reorth == ED_REORTH_FULL) {
      rc = ed_launch_reorth_sweep(B, w, L.store, nullptr, nullptr, j + 1, L.dtype, L.d_ro, c, L.st, L.ylo);
      jj = j;
    } else {
      rc = ed_launch_reorth_sweep(B, w, nullptr, v, vprev, j ? 2 : 1, L.dtype, L.d_ro, c, L.st, L.ylo);
      jj = 0;
    }
    if (rc) return rc;
    if (want_host) {
      double h = 0;
      ED_CK(cudaMemcpyAsync(&B->h_partial[0], c + (size_t)jj * P, 8, cudaMemcpyDeviceToHost, L.st));
      ED_CK(cudaStreamSynchronize(L.st));
      h = B->h_partial[0];
      cj += h;
    }
  }
  ED_CK(cudaEventRecord(L.r1, L.st));
  if (want_host) {
    double nn = 0, im = 0;
    int rc = reduce_partials(B, L.d_ro, grid, false, L.st, &nn, &im);
    if (rc) return rc;
    float ms = 0;
    ED_CK(cudaEventElapsedTime(&ms, L.r0, L.r1));
    L.ms_reorth += ms;
    *corr = cj;
    *b2 = nn;
  }
  return ED_OK;
}

// one Lanczos pass; when coef != null, also accumulates psi += coef[j] v_j (replay of the
// first pass from its stored alpha / beta: same operations, so the same vectors)
int lanczos_pass(LanczosRun &L, const ed_lanczos_opts *o, int max_steps, bool fixed, double tol,
                 std::vector<double> &alpha, std::vector<double> &alpha_rec,
                 std::vector<double> &beta, double *E0, int *steps, int *converged,
                 const std::vector<double> *coef, void *psi) {
  ed_basis *B = L.B;
  const int nblk = B->n_partial / 2;
  const bool full = L.reorth == ED_REORTH_FULL;
  void *vprev = full ? nullptr : L.v[0], *v = full ? L.slot(0) : L.v[1], *w = full ? nullptr : L.v[2];
  int rc;
  // start vector, normalised
  if (o->v0) { if ((rc = ed_launch_copy(B, v, o->v0, L.dtype, L.st))) return rc; }
  else if ((rc = ed_launch_start(B, v, o->seed, L.dtype, L.st))) return rc;
  double nn, im;
  if ((rc = ed_launch_dot(B, v, v, L.dtype, B->d_partial, nblk, L.st))) return rc;
  if ((rc = reduce_partials(B, B->d_partial, nblk, L.cplx, L.st, &nn, &im))) return rc;
  if (!(nn > 0)) return ed_fail(ED_ERR_INVALID, "start vector is zero");
  if ((rc = ed_launch_scale(B, v, 1.0 / std::sqrt(nn), L.dtype, L.st))) return rc;
  const bool replay = coef != nullptr;
  const int m_total = replay ? (int)coef->size() : max_steps;
  if (replay) {
    ED_CK(cudaMemsetAsync(psi, 0, elem_size(L.dtype) * (size_t)B->D, L.st));
  }
  double e_old = 0;
  bool have_old = false;
  *converged = 0;
  for (int j = 0; j < m_total; j++) {
    if (full) { v = L.slot(j); vprev = j ? L.slot(j - 1) : nullptr; w = L.slot(j + 1); }
    if (replay) { if ((rc = ed_launch_axpy(B, psi, v, (*coef)[j], L.dtype, L.st))) return rc; }
    if (replay && j == m_total - 1) break;
    ED_CK(cudaEventRecord(L.e0, L.st));
    if ((rc = ed_launch_apply(B, L.J, L.Jz, v, w, L.dtype, 0, B->D, B->d_partial, L.st, 0, L.ylo))) return rc;
    ED_CK(cudaEventRecord(L.e1, L.st));
    double a;
    if (replay) {
      a = alpha_rec[j];
    } else {
      if ((rc = reduce_partials(B, B->d_partial, B->last_apply_grid, L.cplx, L.st, &a, nullptr))) return rc;
    }
    float ms = 0;
    ED_CK(cudaEventSynchronize(L.e1));
    ED_CK(cudaEventElapsedTime(&ms, L.e0, L.e1));
    L.ms_apply += ms;
    const double bprev = j ? beta[j - 1] : 0.0;
    if ((rc = ed_launch_axpy_norm(B, w, v, j ? vprev : nullptr, a, bprev, L.dtype, B->d_partial, nblk, L.st, L.ylo))) return rc;
    double b2 = 0, corr = 0;
    if (L.reorth != ED_REORTH_NONE) {
      if ((rc = reorth_step(L, j, w, v, j ? vprev : nullptr, !replay, &corr, &b2))) return rc;
    } else if (!replay) {
      if ((rc = reduce_partials(B, B->d_partial, nblk, false, L.st, &b2, nullptr))) return rc;
    }
    double b = replay ? beta[j] : std::sqrt(std::max(b2, 0.0));
    if (!replay) {
      alpha_rec.push_back(a);
      alpha.push_back(a + corr);
      const double e = lowest_eigenvalue(alpha, beta, (int)alpha.size());
      *E0 = e;
      *steps = j + 1;
      bool stop = false;
      if (!fixed && have_old && std::fabs(e - e_old) < tol * std::max(1.0, std::fabs(e))) {
        bool res_ok = true;
        if (o->tol_residual > 0) {   // residual of the lowest Ritz pair: beta_m |s_m|
          const std::vector<double> s = tri_eigvec(alpha, beta, (int)alpha.size(), e);
          res_ok = b * std::fabs(s.back()) < o->tol_residual * std::max(1.0, std::fabs(e));
        }
        if (res_ok) {
          *converged = 1;
          stop = true;
        }
      }
      if (b < 1e-14 * std::max(1.0, std::fabs(a)) || (int64_t)alpha.size() >= B->D) {
        *converged = 1;   // invariant subspace: T holds exact eigenvalues
        stop = true;
      }
      e_old = e;
      have_old = true;
      if (stop || j + 1 == max_steps) break;
      beta.push_back(b);
    }
    if ((rc = ed_launch_scale(B, w, 1.0 / b, L.dtype, L.st, L.ylo))) return rc;
    if (!full) { void *t = vprev; vprev = v; v = w; w = t; }
  }
  return ED_OK;
}

}  // namespace

extern "C" int ed_lanczos(ed_basis *B, const double *J, const double *Jz,
                          const ed_lanczos_opts *opts, ed_lanczos_result *res) {
  if (!B || !J || !Jz || !res) return ed_fail(ED_ERR_INVALID, "null argument");
  memset(res, 0, sizeof(*res));
  ed_lanczos_opts o{};
  if (opts) o = *opts;
  if (B->D == 0) return ed_fail(ED_ERR_EMPTY, "sector has dimension 0");
  int rc = check_dtype(B, o.dtype);
  if (rc) return rc;
  if (o.reorth != ED_REORTH_LOCAL && o.reorth != ED_REORTH_NONE && o.reorth != ED_REORTH_FULL)
    return ed_fail(ED_ERR_INVALID, "reorth must be ED_REORTH_LOCAL, ED_REORTH_NONE or ED_REORTH_FULL");
  int max_steps = o.fixed_steps > 0 ? o.fixed_steps : (o.max_steps > 0 ? o.max_steps : 300);
  const double tol = o.tol > 0 ? o.tol : 1e-13;
  auto t0 = std::chrono::steady_clock::now();
  LanczosRun L{};
  L.B = B; L.J = J; L.Jz = Jz; L.dtype = o.dtype;
  L.cplx = o.dtype == ED_C128 || o.dtype == ED_C64;
  L.st = (cudaStream_t)o.stream;
  L.reorth = o.reorth;
  const size_t bytes = elem_size(o.dtype) * (size_t)B->D;
  const bool full = o.reorth == ED_REORTH_FULL;
  const bool own = !full && o.work == nullptr;
  if (full) {
    if (!o.krylov) return ed_fail(ED_ERR_INVALID, "ED_REORTH_FULL needs a Krylov store");
    const int64_t slots = o.krylov_bytes / (int64_t)bytes;
    if (slots < 2) return ed_fail(ED_ERR_INVALID, "Krylov store smaller than 2 vectors");
    L.store = (char *)o.krylov;
    L.store_slots = (int)std::min<int64_t>(slots, 100000);
    // step j writes w into slot j + 1; the sweeps' shared memory bounds the store too
    max_steps = std::min(max_steps, std::min(L.store_slots - 1, 1024));
    if (o.fixed_steps > 0 && o.fixed_steps > max_steps)
      return ed_fail(ED_ERR_INVALID, "Krylov store too small for fixed_steps");
  } else if (!own && o.work_bytes < (int64_t)(3 * bytes)) {
    return ed_fail(ED_ERR_INVALID, "Lanczos workspace smaller than 3 vectors");
  }
  for (int k = 0; k < 3 && !full; k++) {
    if (!own) { L.v[k] = (char *)o.work + k * bytes; continue; }
    if (cudaMalloc(&L.v[k], bytes) != cudaSuccess) {
      cudaGetLastError();
      for (int q = 0; q < k; q++) cudaFree(L.v[q]);
      return ed_fail(ED_ERR_OOM, "cannot allocate Lanczos vectors");
    }
  }
  // fp32 vectors: the product's low words, so that the three-term update starts from y to
  // about 48 bits (the fourth vector of the caller's workspace when it has one)
  if (o.dtype == ED_F32 || o.dtype == ED_C64) {
    if (!full && !own && o.work_bytes >= (int64_t)(4 * bytes)) {
      L.ylo = (char *)o.work + 3 * bytes;
    } else if (cudaMalloc(&L.ylo, bytes) == cudaSuccess) {
      L.own_ylo = true;
    } else {
      cudaGetLastError();
      if (own) for (int k = 0; k < 3; k++) cudaFree(L.v[k]);
      return ed_fail(ED_ERR_OOM, "cannot allocate the low words of the product");
    }
  }
  // sweep scratch: partials of up to m_cap vectors per block, then their coefficients
  const int m_cap = full ? max_steps + 1 : 2;
  const int P = L.cplx ? 2 : 1;
  L.ro_coef_off = (size_t)m_cap * P * ed_reorth_grid(B);
  if (o.reorth != ED_REORTH_NONE &&
      cudaMalloc(&L.d_ro, sizeof(double) * (L.ro_coef_off + (size_t)m_cap * P)) != cudaSuccess) {
    cudaGetLastError();
    if (own) for (int k = 0; k < 3; k++) cudaFree(L.v[k]);
    if (L.own_ylo) cudaFree(L.ylo);
    return ed_fail(ED_ERR_OOM, "cannot allocate the reorthogonalisation scratch");
  }
  if (cudaEventCreate(&L.e0) != cudaSuccess || cudaEventCreate(&L.e1) != cudaSuccess ||
      cudaEventCreate(&L.r0) != cudaSuccess || cudaEventCreate(&L.r1) != cudaSuccess) {
    cudaGetLastError();
    rc = ed_fail(ED_ERR_CUDA, "cannot create the timing events");
  }
  std::vector<double> alpha, alpha_rec, beta;
  double E0 = 0;
  int steps = 0, conv = 0;
  if (!rc)
    rc = lanczos_pass(L, &o, max_steps, o.fixed_steps > 0, tol, alpha, alpha_rec, beta, &E0,
                      &steps, &conv, nullptr, nullptr);
  if (!rc && o.psi) {
    const int m = (int)alpha.size();
    std::vector<double> bt(beta.begin(), beta.begin() + std::max(0, m - 1));
    std::vector<double> s = tri_eigvec(alpha, bt, m, E0);
    if (full) {   // the Krylov basis is stored: psi = sum_k s_k v_k, no second pass
      double *d_s = L.d_ro;   // the sweep partials are free again
      rc = ED_OK;
      if (cudaMemcpyAsync(d_s, s.data(), sizeof(double) * m, cudaMemcpyHostToDevice, L.st) != cudaSuccess)
        rc = ed_fail(ED_ERR_CUDA, "copy of the Ritz coefficients");
      if (!rc) rc = ed_launch_combine(B, o.psi, L.store, m, d_s, o.dtype, L.st);
      if (!rc && cudaStreamSynchronize(L.st) != cudaSuccess) rc = ed_fail(ED_ERR_CUDA, "combine");
    } else {
      std::vector<double> a2 = alpha, ar2 = alpha_rec, b2 = bt;
      double e_dummy;
      int st_dummy, cv_dummy;
      rc = lanczos_pass(L, &o, m, true, tol, a2, ar2, b2, &e_dummy, &st_dummy, &cv_dummy, &s, o.psi);
    }
    if (!rc) {
      // normalise psi and take its Rayleigh quotient
      double nn, im;
      const int nblk = B->n_partial / 2;
      void *scratch = full ? L.slot(std::min(m, L.store_slots - 1)) : L.v[0];
      rc = ed_launch_dot(B, o.psi, o.psi, o.dtype, B->d_partial, nblk, L.st);
      if (!rc) rc = reduce_partials(B, B->d_partial, nblk, L.cplx, L.st, &nn, &im);
      if (!rc) rc = ed_launch_scale(B, o.psi, 1.0 / std::sqrt(nn), o.dtype, L.st);
      if (!rc) rc = ed_launch_apply(B, J, Jz, o.psi, scratch, o.dtype, 0, B->D, B->d_partial, L.st);
      double rq = 0;
      if (!rc) rc = reduce_partials(B, B->d_partial, B->last_apply_grid, L.cplx, L.st, &rq, nullptr);
      res->rq = rq;
    }
  }
  if (!rc) {
    res->E0 = E0;
    res->steps = steps;
    res->converged = conv;
    res->ms_apply = L.ms_apply;
    res->ms_reorth = L.ms_reorth;
    if (o.alpha) for (size_t k = 0; k < alpha.size(); k++) o.alpha[k] = alpha[k];
    if (o.beta) for (size_t k = 0; k < beta.size(); k++) o.beta[k] = beta[k];
  }
  cudaStreamSynchronize(L.st);
  if (own) for (int k = 0; k < 3; k++) cudaFree(L.v[k]);
  if (L.own_ylo) cudaFree(L.ylo);
  if (L.d_ro) cudaFree(L.d_ro);
  for (cudaEvent_t e : {L.e0, L.e1, L.r0, L.r1})
    if (e) cudaEventDestroy(e);
  res->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return rc;
}
