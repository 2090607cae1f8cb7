/*
 * sced.h -- C ABI of libsced: the symmetry-adapted, matrix-free Hamiltonian-vector
 * product of Wietek & Laeuchli, "Sublattice coding algorithm and distributed memory
 * parallelization for large-scale exact diagonalizations of quantum many-body
 * systems" (arXiv:1804.05028), on one NVIDIA GB300 (sm_103a).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Spin configurations are uint64 integers.  Site label 0 is the most significant
 *    of the N used bits (bit N-1), an up spin is a 1, and states are ordered by
 *    their integer value (Sec. II, Eq. 1 and the ordering by int).
 *  - Sublattice X (0-based) is the block of labels [X*N/n_sublat, (X+1)*N/n_sublat);
 *    sublattice 0 holds the most significant bits (Sec. III B, site numbering).
 *  - Group element g carries the spin on label p to label perm[g*N + p]:
 *    (g s)[perm[g*N+p]] = s[p].  One-dimensional irrep: chi(g) = exp(2 pi i
 *    phase_num[g] / phase_denom) (Sec. II, Eq. 2, 1-D irreps only).
 *  - Hamiltonian: H = sum_b J[c(b)] ( Jz[c(b)] S^z_i S^z_j + (S^+_i S^-_j + h.c.)/2 )
 *    over bonds b = (i, j) of coupling class c(b) (Eq. 21 split into classes).
 *  - Basis state |s_rho> = (1/N_s) sum_g chi(g)^* g|s> for each representative s
 *    (Eq. 2) that survives the projection (chi = 1 on the stabiliser of s);
 *    N_s = sqrt(|G| |Stab(s)|).  Its matrix elements are
 *    <j|H_k|i> = c chi(h)^* N_j/N_i with s_j = h s' (Eq. 5; conjugation as implied
 *    by Eq. 2).
 *
 * Errors: every call returns ED_OK (0) or one of the ED_ERR_* codes below and, on
 * error, leaves a message for ed_last_error() (thread-local).  No call aborts the
 * process.  Device work is enqueued on the caller's stream (a cudaStream_t passed
 * as void*, NULL = the legacy default stream) on the device that is current when
 * ed_build_basis ran; calls marked "synchronous" wait for it.
 */
#ifndef SCED_H
#define SCED_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ED_OK 0
#define ED_ERR_INVALID 1     /* bad descriptor: N>64, non-bijective permutation, group not
                                closed, bonds not invariant, chi not a homomorphism, ... */
#define ED_ERR_UNSTABLE 2    /* sublattice split not stable under the group (Sec. III B,
                                "Sublattice stability") or n_sublat does not divide N */
#define ED_ERR_OOM 3         /* device or host allocation failed */
#define ED_ERR_CUDA 4        /* a CUDA runtime call failed (message has the CUDA error) */
#define ED_ERR_TIMEOUT 5     /* reserved: a bounded device wait gave up */
#define ED_ERR_EMPTY 6       /* the sector has dimension 0 (Lanczos has nothing to do) */
#define ED_ERR_UNSUPPORTED 7 /* valid request outside what this build implements */

/* Vector element types of apply_H / lanczos. */
#define ED_F64 0   /* double   */
#define ED_F32 1   /* float    */
#define ED_C128 2  /* complex double, interleaved (re, im) */
#define ED_C64 3   /* complex float, interleaved (re, im) */

/* Lattice: sites, sublattice split and bonds (Eq. 21).  Host memory, read only
 * during ed_build_basis. */
typedef struct {
  int32_t n_sites;            /* N, 1..64 */
  int32_t n_sublat;           /* number of sublattices, divides N; N/n_sublat <= 20 when > 1,
                                 N <= 26 when 1 (the whole lookup table of Sec. III, built
                                 on the device: 2^N entries of 8 bytes) */
  int32_t n_bonds;            /* 1..4096 */
  int32_t n_classes;          /* coupling classes, 1..8 */
  const int32_t *bonds;       /* [n_bonds][2] site labels, distinct */
  const int32_t *bond_class;  /* [n_bonds] in [0, n_classes) */
} ed_lattice;

/* Symmetry group as site permutations, optionally combined with the reversal of every
 * spin (the spin-flip symmetry of the S^z = 0 sector, Sec. V, Table 1) (host memory). */
typedef struct {
  int32_t n_sym;              /* |G|, 1..65535 */
  const int32_t *perm;        /* [n_sym][n_sites] */
  const uint8_t *flip;        /* NULL, or [n_sym]: 1 when element g also reverses every spin,
                                 (g s) = perm(s) XOR (all ones); needs n_up = N/2 */
} ed_group;

/* One-dimensional irrep as exact phases (host memory). */
typedef struct {
  int32_t phase_denom;        /* >= 1 */
  const int32_t *phase_num;   /* [n_sym] */
} ed_irrep;

typedef struct ed_basis ed_basis;   /* opaque; owns (or shares) every device table it uses */

/* Tuning of the basis and its index; pass NULL for defaults. */
typedef struct {
  int32_t bucket_target;      /* average states per Limits bucket (default 1) */
  int32_t reserved0;
  const ed_basis *share_tables; /* optional: a basis of the same lattice and group whose
                                   one-sublattice table (n_sublat == 1) is reused instead of
                                   building a copy; it stays valid until every basis that
                                   uses it is freed */
  int64_t reserved[2];
} ed_basis_opts;

typedef struct {
  int64_t dim;                /* D, number of basis states */
  int32_t is_real;            /* 1 when every character is +1 or -1 */
  int32_t n_sites, n_sublat, n_sym, n_up, n_bonds, n_classes;
  int32_t prefix_rank_bits;   /* top bits mapped through the prefix rank table */
  int32_t prefix_raw_bits;    /* further bits of the Limits key */
  int32_t postfix_bits;       /* bits compared by the in-bucket binary search */
  int64_t n_keys;             /* Limits buckets */
  int64_t max_bucket;         /* largest bucket */
  int64_t table_bytes;        /* device bytes of Rep/Sym/SymmetryAction tables */
  int64_t index_bytes;        /* device bytes of the prefix rank table, Limits and postfixes */
  int64_t basis_bytes;        /* device bytes of Basis and |Stab| */
  int64_t sym_list_len;       /* total entries of the Sym_X lists */
  double build_ms;            /* wall time of ed_build_basis */
} ed_basis_info_t;

/*
 * ed_build_basis -- validate the descriptor, build the sublattice-coding lookup
 * tables (Alg. 1: Rep_X, Sym_X, SymmetryAction_X of Eqs. 8-11) on the host, then on
 * the device enumerate every configuration with n_up up spins whose top block is its
 * own Rep_0, keep those that are their own representative (Alg. 2) and survive the
 * projection, in increasing integer order (Alg. 3 on one GPU: count, scan, fill), and
 * build the index used by apply_H (Basis, |Stab| and the prefix map Limits of
 * Sec. IV, with half-open buckets).
 *   lattice, group, irrep: host descriptors (copied; caller keeps ownership).
 *   n_up: number of up spins (S^z = n_up - N/2).
 *   opts: NULL or tuning.  stream: enqueue on this stream; the call is synchronous.
 *   out: receives the new basis (free with ed_free_basis), NULL on error.
 * A sector of dimension 0 is valid: *out is a basis with dim 0.
 * Errors: ED_ERR_INVALID (malformed descriptor: not a group, characters not a
 * homomorphism, bonds not invariant, n_up out of range, spin flip away from n_up = N/2),
 * ED_ERR_UNSTABLE (n_sublat does not divide N, or a group element splits a block),
 * ED_ERR_UNSUPPORTED (blocks above 20 sites, one block above 26 sites, dimension of
 * 2^32 or more), ED_ERR_OOM, ED_ERR_CUDA.
 */
int ed_build_basis(const ed_lattice *lattice, const ed_group *group, const ed_irrep *irrep,
                   int32_t n_up, const ed_basis_opts *opts, void *stream, ed_basis **out);

/* ed_free_basis -- release every device and host buffer of the basis (NULL is a no-op). */
void ed_free_basis(ed_basis *basis);

/* ed_basis_info -- sizes and index parameters of a basis (host struct, caller-owned). */
int ed_basis_info(const ed_basis *basis, ed_basis_info_t *info);

/* ed_basis_export -- synchronous copy of Basis (uint64[dim]) and |Stab| (uint16[dim]) to
 * caller-owned HOST arrays; either pointer may be NULL. */
int ed_basis_export(const ed_basis *basis, uint64_t *states, uint16_t *stab);

/*
 * ed_find_rep -- the representative search alone, plus the Limits lookup, for n arbitrary
 * configurations.  method 0 is Alg. 2 as printed: MinRep = min_X Rep_X, then every g of
 * Sym_Y for every minimal Y; method 1 is the two-level search the product uses (Sym_Y is
 * a coset of the stabiliser of MinRep, searched again by sublattice coding; available for
 * 2..4 sublattices of <= 11 sites, else ED_ERR_UNSUPPORTED).
 * All pointers are DEVICE arrays of length n owned by the caller: states (in), rep (out,
 * Eq. 4 representative), sym (out, method 0: the first minimising element in Sym_Y order,
 * unique up to the stabiliser; method 1: -1), phase (out, numerator of chi of that
 * minimiser), stab (out, |Stab(rep)| = number of minimisers), index (out, position of rep
 * in Basis, or -1 when rep is not a basis state: not a surviving representative or a
 * different n_up).  Asynchronous on stream.  Output pointers may be NULL to skip.
 */
int ed_find_rep(const ed_basis *basis, const uint64_t *states, int64_t n, int32_t method,
                uint64_t *rep, int32_t *sym, int32_t *phase, int32_t *stab, int64_t *index,
                void *stream);

/*
 * ed_apply_H -- y = H x on the symmetry-adapted basis, matrix-free (Sec. IV,
 * Eqs. 12-17 restated as a row-wise pull): for each row i, its diagonal, then for
 * each antiparallel bond the exchanged configuration, its representative by sublattice
 * coding (Alg. 2), its index through Limits (the bucket's first index plus the rank of
 * the postfix in the bucket's bitmap, or a binary search in the bucket), and
 * y_i += (J/2) chi(h) sqrt(|Stab_j|/|Stab_i|) x_j.  No atomics; every y_i is written
 * once.  Deterministic: the same call gives the same bits.  The terms of 32
 * consecutive rows are summed together, so a row range that starts elsewhere
 * (ed_apply_H_rows, the chunks of ed_apply_H_host) may differ in the last bit.
 *   J, Jz: HOST arrays [n_classes].
 *   x, y: DEVICE arrays of dim elements of `dtype` (ED_F64 or ED_F32; the complex types
 *   for sectors with complex characters), caller-owned, must not overlap.
 *   dtype ED_F32 stores vectors in float; each row is summed to about 48 bits
 *   (double-float) and rounded once.
 *   Asynchronous on stream.  dim 0: no-op.
 * Errors: ED_ERR_INVALID (null pointers, dtype not matching the sector), ED_ERR_CUDA.
 */
int ed_apply_H(const ed_basis *basis, const double *J, const double *Jz, const void *x,
               void *y, int32_t dtype, void *stream);

/*
 * ed_apply_H_rows -- as ed_apply_H restricted to rows [row_begin, row_end): y holds
 * those rows only (y[0] is row row_begin), x is the whole vector.  Building block of a
 * row-sharded product across devices.
 */
int ed_apply_H_rows(const ed_basis *basis, const double *J, const double *Jz, const void *x,
                    void *y, int32_t dtype, int64_t row_begin, int64_t row_end, void *stream);

/*
 * ed_apply_H_host -- ed_apply_H on HOST arrays x, y (dim elements of dtype): copies x
 * to device staging buffers owned by the basis, runs the product, copies y back.  Above
 * 2^25 rows the product runs in up to 8 row chunks and each chunk of y is copied back
 * (on a stream of the basis) while the next one is computed; with pinned host arrays
 * the copies then overlap the product.  Synchronous.  Not safe to call concurrently on
 * the same basis.
 */
int ed_apply_H_host(ed_basis *basis, const double *J, const double *Jz, const void *x_host,
                    void *y_host, int32_t dtype, void *stream);

/* Reorthogonalisation of the Lanczos vectors (ed_lanczos_opts.reorth).  Every dot,
 * coefficient and update of a sweep is accumulated in double, whatever the vector type. */
#define ED_REORTH_LOCAL 0  /* default: after the three-term update, one more Gram-Schmidt sweep
                              against v_j and v_{j-1} (two extra dots, one extra update) */
#define ED_REORTH_NONE 1   /* the plain three-term recurrence */
#define ED_REORTH_FULL 2   /* two classical Gram-Schmidt sweeps against every earlier Lanczos
                              vector, which the caller's Krylov store keeps; the ground state
                              is then formed from the store, without a second pass */

/* Lanczos options; zero-initialise and set what you need. */
typedef struct {
  int32_t max_steps;          /* default 300 when 0 */
  int32_t fixed_steps;        /* > 0: run exactly this many steps, no convergence test */
  double tol;                 /* stop when the lowest Ritz value moves by < tol*max(1,|E0|);
                                 default 1e-13 when 0 */
  int32_t dtype;              /* ED_F64 or ED_F32 vectors; alpha, beta and the tridiagonal
                                 eigenproblem are always double */
  int32_t reserved0;
  uint64_t seed;              /* start vector x(s) = uniform[-1,1) from SplitMix64 of
                                 (s + (2 seed + 1) * 0x9E3779B97F4A7C15), unless v0 given */
  const void *v0;             /* optional DEVICE start vector (dtype, dim) */
  void *psi;                  /* optional DEVICE output (dtype, dim): normalised ground
                                 state from a second Lanczos pass */
  double *alpha;              /* optional HOST output of M doubles, where M = fixed_steps
                                 when fixed_steps > 0, else max_steps, else 300 */
  double *beta;               /* optional HOST output of M doubles (M as for alpha) */
  void *stream;
  void *work;                 /* optional DEVICE workspace of >= 3 * dim elements of dtype,
                                 caller-owned; when NULL the call allocates its own.  With
                                 fp32 vectors a fourth dim-element slice, when the workspace
                                 holds one, keeps the low words of the product (y as a
                                 double-float pair); otherwise the call allocates it */
  int64_t work_bytes;         /* size of work in bytes */
  double tol_residual;        /* > 0: also require the Ritz residual beta_m |s_m| of the lowest
                                 pair to fall below tol_residual * max(1, |E0|) (for an
                                 accurate ground state, e.g. derivatives); 0: energy only */
  int32_t reorth;             /* ED_REORTH_LOCAL (0), ED_REORTH_NONE or ED_REORTH_FULL */
  int32_t reserved1;
  void *krylov;               /* ED_REORTH_FULL only: caller-owned DEVICE store of krylov_bytes
                                 bytes; slot k (dim elements of dtype, slot k at byte
                                 k * dim * element size) receives v_k.  The run takes at most
                                 min(slots - 1, 1024) steps; work is not used */
  int64_t krylov_bytes;
} ed_lanczos_opts;

typedef struct {
  double E0;                  /* lowest Ritz value */
  int32_t steps;              /* Lanczos steps taken */
  int32_t converged;          /* 1 when the tolerance was met (or breakdown: invariant
                                 subspace found) */
  double rq;                  /* <psi|H|psi> with fp64 accumulation when psi was
                                 requested (Rayleigh quotient), else 0 */
  double ms_total;            /* wall time */
  double ms_apply;            /* device time spent in apply_H (CUDA events) */
  double ms_reorth;           /* device time spent in reorthogonalisation sweeps */
} ed_lanczos_result;

/*
 * ed_lanczos -- ground-state energy by the Lanczos iteration with apply_H as the
 * matrix-vector product (Sec. IV: the product dominates; dots, scalings and the
 * tridiagonal eigenproblem are cheap).  Three device vectors of dtype (four with psi),
 * or the caller's Krylov store with ED_REORTH_FULL; alpha = <v, Hv> and beta = ||w||
 * reduced in double per block then summed on the host in a fixed order (with fp32
 * vectors the product y is kept to about 48 bits -- fp32 value plus its rounding
 * remainder -- until the three-term update has used it, so that only the stored vectors
 * are rounded to fp32); the reorthogonalisation chosen by opts->reorth (default: a second sweep against the last
 * two vectors), with alpha_j corrected by the sweeps' <v_j, w>; lowest eigenvalue of the
 * tridiagonal matrix by Sturm-sequence bisection in double.  With psi and without a
 * Krylov store the ground state comes from a second pass of the same recurrence
 * (vectors recomputed, not stored).  Allocates a small sweep scratch (and the three
 * vectors when work is NULL).  Synchronous.
 * Errors: ED_ERR_EMPTY (dim 0), ED_ERR_INVALID, ED_ERR_OOM, ED_ERR_CUDA.
 */
int ed_lanczos(ed_basis *basis, const double *J, const double *Jz, const ed_lanczos_opts *opts,
               ed_lanczos_result *result);

/*
 * ed_dot -- sum_i conj(x_i) y_i over dim DEVICE elements of dtype, in double, written to
 * the HOST array out[2] = (re, im).  Synchronous.  Scratch lives in the basis.
 */
int ed_dot(ed_basis *basis, const void *x, const void *y, int32_t dtype, double *out, void *stream);

/*
 * ed_count_terms -- how many exchange terms one product generates: *n_flip counts every
 * (row, antiparallel bond) pair (Eq. 16 applied to every basis state), *n_offdiag those
 * whose exchanged configuration has a surviving representative, i.e. the off-diagonal
 * contributions that apply_H gathers.  HOST outputs; synchronous.
 */
int ed_count_terms(const ed_basis *basis, int64_t *n_flip, int64_t *n_offdiag, void *stream);

/*
 * ed_expect_classes -- out[c] = Re <x | H_c | x> for every coupling class c, where H_c is
 * the class-c part of Eq. 21 with unit exchange (J_c = 1) and anisotropy Jz[c], so that
 * H = sum_c J_c H_c.  For a normalised ground state psi this is dE0/dJ_c (Hellmann-Feynman
 * theorem), the derivative the product's adjoint needs.  One pass of the product kernel
 * with per-class partial sums.
 *   Jz: HOST [n_classes].  x: DEVICE vector of dim elements of dtype (the sector's real
 *   or complex types; with fp32 vectors the terms are products of fp32 inputs, the class
 *   sums are carried in double).
 *   out: HOST [n_classes].  Synchronous.  Errors: ED_ERR_INVALID, ED_ERR_CUDA.
 */
int ed_expect_classes(ed_basis *basis, const double *Jz, const void *x, int32_t dtype,
                      double *out, void *stream);

/*
 * Batched product over many sectors (the uneven-sector workload): sectors of one lattice
 * (same sites, bonds, classes) that differ in group, irrep and n_up, each applied to k
 * vectors at once, all in one persistent launch.  Work items (sector, block of rows) are
 * taken warp by warp from a device counter (atomicAdd; no warp waits on another), so
 * sectors of any size mix in one launch.  Each exchange term is searched (Alg. 2) and looked up (Sec. IV) once
 * and applied to the k vectors, stored row-major: x[s][i*k + v].  Vectors are fp32 for real
 * sectors and complex fp32 (interleaved) for sectors with complex characters.
 */
typedef struct ed_batch ed_batch;

/* ed_batch_create -- a batch of n bases (kept by reference: they must outlive the batch),
 * couplings J, Jz (HOST [n_classes]) and block width k in {1, 2, 4, 8}. */
int ed_batch_create(ed_basis *const *bases, int32_t n, const double *J, const double *Jz,
                    int32_t k, ed_batch **out);

/* ed_batch_set_vectors -- DEVICE input / output vectors per sector (HOST arrays of n device
 * pointers; x[s], y[s] hold dim_s * k elements of fp32 or complex fp32).  For k >= 2 every
 * non-empty sector's x[s] and y[s] must be 16-byte aligned, and x[s] 32-byte aligned when
 * a row holds 32 bytes or more (k = 8 real, k >= 4 complex): the kernel moves a row's k
 * entries with 16- and 32-byte accesses.  ED_ERR_INVALID otherwise.  Synchronous: when an
 * earlier ed_batch_apply may still run, the call first waits for it (the launch reads the
 * sector table that this call rewrites). */
int ed_batch_set_vectors(ed_batch *batch, void *const *x, void *const *y);

/* ed_batch_apply -- y[s] = H_s x[s] for every sector, in one launch on stream.  The first call
 * times a few work-item sizes (rows per item) and keeps the fastest, then captures the
 * counter reset and the launch in a CUDA graph that later calls replay.  Asynchronous
 * after the first call. */
int ed_batch_apply(ed_batch *batch, void *stream);

/* ed_batch_info -- rows per work item chosen by the first ed_batch_apply, and item count. */
int ed_batch_info(const ed_batch *batch, int32_t *rows_per_item, int64_t *n_items);

/* ed_batch_free -- release the batch (not its bases). */
void ed_batch_free(ed_batch *batch);

/*
 * ed_dot_noalloc -- sum_i conj(x_i) y_i over n DEVICE elements of dtype, in double, like
 * ed_dot, but without allocating anything and without a basis.  The paper has no
 * counterpart: this exists for callers that cannot allocate device memory when they need
 * the reduction -- a host loop that must not stall the device (cudaMalloc / cudaFree may
 * synchronise it), or a framework that owns all device memory through its own pool.
 *   x, y: DEVICE arrays of n elements (caller-owned).  out: DEVICE array of 2 doubles
 *   (re, im), written by the device; asynchronous on stream.
 *   n: 0 .. 2^30 (1073741824); larger n is refused with ED_ERR_INVALID.
 * The block partials live in a fixed 1 MiB array compiled into the library, present on
 * every device that loads it until the process exits.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  All calls share the array: calls whose work
 * overlaps on the device race on it and must be ordered by the caller (same stream, or
 * events).  Errors: ED_ERR_INVALID, ED_ERR_CUDA.
 */
int ed_dot_noalloc(const void *x, const void *y, int64_t n, int32_t dtype, double *out,
                   void *stream);

/*
 * Vector operations on a slice of a Lanczos vector (Sec. IV: the product dominates the
 * Lanczos iteration; scalings, updates and dot products are streaming passes).  They let a
 * driver that holds only part of every vector -- e.g. one rank of a row-sharded Lanczos --
 * run its rank-local arithmetic in the library; ed_lanczos needs none of them.  fp32
 * vectors are updated and summed in double-float arithmetic (pairs of fp32 words, exact
 * fp32 products), fp64 vectors in fp64; every reduction has a fixed order.  All pointers
 * are DEVICE pointers on the current device, caller-owned; asynchronous on stream.
 */

/* ed_axpy_norm -- w <- w - a v - b vprev over n elements of dtype (vprev may be NULL; a and
 * b real, as in the Hermitian tridiagonal recurrence), then norm2[0] = ||w||^2 in double.
 * scratch: DEVICE array of scratch_len >= 1 doubles for block partials (more blocks are used
 * when it is longer, up to 4 per SM).  Errors: ED_ERR_INVALID (negative n, null pointers,
 * unknown dtype), ED_ERR_CUDA. */
int ed_axpy_norm(void *w, const void *v, const void *vprev, double a, double b, int64_t n,
                 int32_t dtype, double *scratch, int64_t scratch_len, double *norm2, void *stream);

/* ed_scale -- x <- s x over n elements of dtype.  Errors: ED_ERR_INVALID, ED_ERR_CUDA. */
int ed_scale(void *x, double s, int64_t n, int32_t dtype, void *stream);

/* ed_last_error -- message of the last failing call on this thread ("" if none). */
const char *ed_last_error(void);

/* ed_version -- library version string. */
const char *ed_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SCED_H */
