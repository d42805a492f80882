/*
 * h2.h -- C ABI of the GB300 library for the accuracy-controlled, structure-
 * preserving H^2 matrix-matrix product with change of cluster bases (Ma & Jiao,
 * "Accuracy Controlled Structure-Preserving H^2-Matrix-Matrix Product in Linear
 * Complexity with Change of Cluster Bases").
 *
 * Conventions shared by every entry point
 *   - Plain C types only.  Host pointers are marked "host", device pointers
 *     "device" (memory of the current CUDA device, e.g. from cudaMalloc or a torch
 *     CUDA tensor's data_ptr).
 *   - Every call returns an h2_status; no exception or abort crosses the ABI.
 *     On failure h2_last_error() returns a thread-local, human-readable message
 *     and no output handle is created.
 *   - Handles own their device memory; h2_destroy frees it.  Handles are not
 *     thread-safe: do not use one handle from two threads at once.
 *   - Work is enqueued on opts->stream (a cudaStream_t, NULL = the legacy default
 *     stream).  Calls that return host data synchronise that stream.
 *   - Point and vector data are in the caller's ("user") order; the library
 *     permutes to its cluster-tree order internally.
 *   - Complex matrices (the Helmholtz kernel, or h2_import_complex): every complex
 *     number is two doubles (real part, then imaginary part) in host and device
 *     arrays; element counts count complex numbers.  Complex products run in float64
 *     or mixed float32 (h2_precision).
 *   - Arithmetic: see h2_precision.
 */
#ifndef H2_GB300_H
#define H2_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2_matrix* h2_handle;

typedef enum {
  H2_OK = 0,
  H2_EINVAL = 1,       /* bad argument (null pointer, size, parameter range)        */
  H2_ENOMEM = 2,       /* device or host allocation failed                           */
  H2_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed                */
  H2_ESTRUCT = 4,      /* A and B do not share one cluster tree and block partition */
  H2_ETIMEOUT = 5,     /* a bounded device-side wait gave up                        */
  H2_EINTERNAL = 6,    /* internal consistency check failed                          */
  H2_EUNSUPPORTED = 7  /* valid request this library does not implement             */
} h2_status;

/* Kernel functions K(x, y), r = |x - y|; the diagonal (x == y) takes diag_re. */
typedef enum {
  H2_K_LAPLACE = 0,    /* 1 / (4 pi r)                                   */
  H2_K_INV_R2 = 1,     /* 1 / r^2                                        */
  H2_K_HELMHOLTZ = 2   /* exp(-j k r) / (4 pi r), complex (Sec. VI-B)    */
} h2_kernel_kind;

typedef struct {
  int32_t kind;        /* h2_kernel_kind */
  double wavenumber;   /* k of the Helmholtz kernel, ignored otherwise */
  double diag_re;      /* value on the diagonal (real part) */
  double diag_im;      /* imaginary part of the diagonal (Helmholtz only) */
} h2_kernel;

/* Arithmetic of the product.  In every mode the rank decisions (float64 Rayleigh
 * quotients of the normalised Gram sum where float32 could change them) and the
 * re-orthonormalisation of the new bases are float64, and C is stored in float64.  The
 * mixed modes compute the small matrix products (dense targets, Gram matrices,
 * projections, collects, couplings, split) in float32 from float32 copies of A and B, so
 * their Gram matrices carry float32 rounding.  Complex matrices take H2_FP64 and
 * H2_MIXED_FP32 (complex float32 products, float64 Hermitian eigen-decomposition):  */
typedef enum {
  H2_FP64 = 0,          /* every product, Gram matrix and eigen-decomposition in float64 */
  H2_MIXED_FP32 = 1,    /* products in float32 with float32 accumulation (CUDA cores);
                           eigen-decomposition by float32 Jacobi, ranks decided by
                           float64 Rayleigh quotients, kept vectors re-orthonormalised
                           in float64 (Newton-Schulz) */
  H2_MIXED_TF32X3 = 2,  /* as H2_MIXED_FP32, with the products on the tensor cores
                           (tcgen05): each float32 operand split into two TF32 parts,
                           three TF32 products per pair, float32 accumulation */
  H2_MIXED_BF16X3 = 3   /* as H2_MIXED_FP32, with the main coupling pass of every level
                           (Eq. leafcoup_simple / nonleafcoup_simple) and the dense leaf
                           products F F of the dense targets (Sec. III-A) on the tensor
                           cores (tcgen05 kind::f16): each float32 operand split into two
                           BF16 parts, x = hi + lo, three BF16 products per pair (hi hi,
                           hi lo, lo hi), float32 accumulation; about 2^-16 relative error
                           per product.  Levels whose tiles exceed 64 rows, columns or k
                           take the float32 path.  Each operand keeps BF16 tiles of its
                           dense blocks beside its float copy.  Real matrices only. */
} h2_precision;

/* Norm that scales each Gram matrix before the sum (Sec. III-C, "normalized"). */
typedef enum {
  H2_NORM_FROBENIUS = 0, /* ||G_m||_F (default)                                    */
  H2_NORM_SPECTRAL = 1   /* ||G_m||_2, the largest eigenvalue (each component is
                            decomposed once more; float64 eigen kernel)            */
} h2_norm;

/* Truncation rule of the new cluster bases (Sec. III-C, IV-C): the summed,
 * normalised Gram matrix G is decomposed, G = U diag(lambda) U^H, and column m of U
 * is kept when lambda_m / lambda_1 > threshold. */
typedef enum {
  H2_TRUNC_PAPER = 0,  /* threshold = eps: the normalised singular values of G (the
                          paper's statement; error ~ sqrt(eps) in practice)      */
  H2_TRUNC_SV = 1,     /* threshold = eps^2: singular values of the stacked
                          contributions (error ~ eps)                            */
  H2_TRUNC_FULL = 2,   /* keep every vector (no truncation; for testing)         */
  H2_TRUNC_FORMATTED = 3 /* no change of bases: C takes A's row bases and B's column
                          bases and every product is projected onto them (the
                          earlier formatted product the paper compares with,
                          Sec. VI, Table relErr_cube "Existing"); eps is unused   */
} h2_trunc;

typedef struct {
  int32_t precision;   /* h2_precision, default H2_FP64                          */
  int32_t trunc;       /* h2_trunc, default H2_TRUNC_PAPER                       */
  int32_t rank_cap;    /* largest rank of a non-leaf cluster of C, 1..128; 0 =
                          default 48; ranks above it are cut to the cap and
                          counted in h2_stats.cap_hits                            */
  int32_t norm;        /* h2_norm, default H2_NORM_FROBENIUS                     */
  void* stream;        /* cudaStream_t, NULL = legacy default stream            */
  int32_t autotune;    /* 0: fixed kernel choices (default); 1: the first product
                          of a program times the candidate kernels of every launch
                          group and keeps the fastest for later products (results
                          do not depend on the choice in float64; see h2_precision) */
  int32_t reserved;    /* must be 0 */
} h2_opts;             /* a NULL h2_opts* means all defaults */

typedef struct {
  int64_t n;                 /* number of points / matrix order                  */
  int32_t levels;            /* L + 1 (root level 0 .. leaf level L)             */
  int32_t leaf_size;         /* largest leaf cluster                             */
  int32_t l_min;             /* coarsest level holding an admissible block       */
  int32_t csp;               /* sparsity constant: most blocks of one cluster on
                                one level                                         */
  int64_t n_admissible;      /* R blocks, all levels                             */
  int64_t n_dense;           /* F blocks (leaf level)                            */
  int32_t max_rank_row[32];  /* largest row rank per level                       */
  int32_t max_rank_col[32];
  int64_t bytes_stored;      /* algorithmic size of the representation: F entries
                                + coupling entries + leaf basis entries + transfer
                                entries at the actual ranks, times 8 bytes        */
  int64_t device_bytes;      /* device memory held by the handle                 */
  int64_t cap_hits;          /* clusters whose rank was cut at rank_cap (product) */
  double mmp_ms;             /* device time of the product that made this handle
                                (0 for built handles)                             */
  int32_t is_complex;        /* 1: complex elements (bytes above count 16 per element) */
  int32_t reserved;
} h2_stats;

/* Build an H^2 approximation of the kernel matrix K(points_a, points_b) on the
 * device.
 *   points  host, n x 3 row-major (x, y, z per point), user order; copied.
 *   kernel  host; see h2_kernel.
 *   leaf_size  largest number of points of a leaf cluster (>= 1, <= 64).
 *   eta     admissibility parameter of Eq. admCond (> 0).
 *   eps     construction accuracy: a basis keeps the singular vectors of its
 *           (sampled) far field with sigma / sigma_1 > eps.
 * Structure (Sec. II): cardinality-balanced bisection cluster tree with all leaves
 * on level L, block partition by Eq. admCond with bounding boxes.  The numeric
 * construction is not specified by the paper (it cites another method); this library
 * uses nested far-field sampling with interpolative skeletons (sampled far field
 * per cluster, skeleton rows chosen by pivoted Gram-Schmidt).  The real kernels are built
 * on the GPU, level by level, straight into the device arena (the sampled Gram matrices
 * from float32 kernel values with float64 sums, float64 eigen-decompositions, skeletons,
 * couplings and dense blocks); the Helmholtz kernel is built on the host and gives a
 * complex matrix (complex-symmetric: column bases equal row bases).  Errors: H2_EINVAL for
 * bad sizes, non-finite points or an unknown kernel; H2_ENOMEM. */
h2_status h2_build(const double* points, int64_t n, const h2_kernel* kernel,
                   int32_t leaf_size, double eta, double eps, const h2_opts* opts,
                   h2_handle* out);

/* The construction of h2_build on the host only (no GPU, no device memory): the packed
 * arrays of h2_import (complex kernels: two doubles per element) for the points.  For the
 * real kernels h2_build runs the same steps on the GPU with float32 kernel values in the
 * sampled Gram matrices, so a rank may differ by one or two where an eigenvalue lies
 * within float32 noise of eps^2 lambda_1; the accuracy is the same.  Pass
 * NULL arrays to get the element counts in sizes[0..7] (as h2_export: ranks per array,
 * vr, vc, er, ec, s, f, 0); each call runs the construction.  Errors as h2_build.  The
 * paper has no counterpart: its inputs come from a cited construction method. */
h2_status h2_build_packed(const double* points, int64_t n, const h2_kernel* kernel, int32_t leaf_size,
                          double eta, double eps, int64_t* sizes, int32_t* kr, int32_t* kc, double* vr,
                          double* vc, double* er, double* ec, double* s, double* f);

/* Failure injection for tests: after n more device allocations (n >= 0) every further
 * one fails, and the call that needed it returns H2_ENOMEM with no partial result;
 * n < 0 lifts the limit (the default).  Process-wide; never fails.  The paper has no
 * counterpart. */
h2_status h2_set_alloc_limit(int64_t n);

/* Host-only size of the product program of C = A A (no GPU needed): tree, partition
 * and H^2 ranks of the Laplace kernel as h2_build_packed makes them (at eps), storage caps as
 * an import sets them, rank cap 48, truncation rule `trunc`.  *flops gets the
 * multiply-add flops counted over all GEMM items at the padded caps (2 m n k), and
 * *segments / *items the numbers of output matrices and of products.  At constant rank
 * all three grow linearly in N (Sec. V, time complexity at constant rank).  Errors:
 * H2_EINVAL for bad arguments. */
h2_status h2_plan_stats(const double* points, int64_t n, int32_t leaf_size, double eta, double eps, int32_t trunc,
                        double* flops, int64_t* segments, int64_t* items);

/* Host-only self-check of the product program (no device memory, no GPU needed):
 * builds the tree, partition and H^2 ranks of the Laplace kernel (as h2_build_packed, at
 * ε = eps) for the points, then the program of C = A A for every truncation mode
 * (paper, sv, full, formatted), the precisions H2_FP64, H2_MIXED_FP32 and
 * H2_MIXED_BF16X3 and rank caps 24 and 48, and the matvec programs for 1 and 3
 * right-hand sides.  Each is validated: every operand and output of every segment,
 * tensor-core step and eigen task lies inside one live allocation of its region
 * (replayed in program order) or inside its matrix.  *checked gets the number of
 * programs checked (26).  H2_EINTERNAL names the first program and access that fails.
 * The paper has no counterpart: this checks the library's own memory layout. */
h2_status h2_plan_selfcheck(const double* points, int64_t n, int32_t leaf_size, double eta, double eps,
                            int32_t* checked);

/* Host-only digest of the product program (no device memory, no GPU needed): the
 * program of C = A A for the points, built as h2_plan_stats builds it (Laplace ranks
 * at ε = eps, rank cap 48) for `precision` (h2_precision) and `trunc` (h2_trunc),
 * hashed (64-bit FNV-1a) over every field of every segment, item, tensor-core group
 * and step, eigen task, launch and allocation of the work regions.  Equal digests mean
 * equal programs.  The program is built with every host thread; its content does not
 * depend on their number.  Errors: H2_EINVAL for bad arguments.  The paper has no
 * counterpart. */
h2_status h2_plan_digest(const double* points, int64_t n, int32_t leaf_size, double eta, double eps,
                         int32_t precision, int32_t trunc, uint64_t* digest);

/* Create a handle from host arrays that describe an H^2 matrix on the same tree
 * and partition that h2_build(points, n, kernel, leaf_size, eta, ...) makes.  Used
 * to feed matrices built elsewhere (e.g. by a reference implementation) to the
 * product.  All arrays are host, float64, tree order, concatenated in this order:
 *   kr, kc      int32 ranks per cluster, clusters ordered by level then index
 *               (2^(L+1) - 1 entries each)
 *   vr, vc      per leaf t (index order): |t| x kr_t (resp. kc_t), row-major
 *   er, ec      per non-leaf (l, t), levels 0..L-1: (k_t1 + k_t2) x k_t, row-major
 *   s           per admissible block, ordered by level then (t, s): kr_t x kc_s
 *   f           per dense leaf block, ordered by (t, s): |t| x |s|
 * Errors: H2_EINVAL if a rank is negative or larger than the cluster allows. */
h2_status h2_import(const double* points, int64_t n, int32_t leaf_size, double eta,
                    const int32_t* kr, const int32_t* kc, const double* vr,
                    const double* vc, const double* er, const double* ec,
                    const double* s, const double* f, const h2_opts* opts,
                    h2_handle* out);

/* h2_import for a complex matrix: the same arguments and layout, every array element a
 * complex number stored as two doubles (real, imaginary); kr, kc as for h2_import.  The
 * handle multiplies with complex handles only (H2_FP64, H2_MIXED_FP32).  Errors as
 * h2_import. */
h2_status h2_import_complex(const double* points, int64_t n, int32_t leaf_size, double eta,
                            const int32_t* kr, const int32_t* kc, const double* vr,
                            const double* vc, const double* er, const double* ec,
                            const double* s, const double* f, const h2_opts* opts,
                            h2_handle* out);

/* The inverse of h2_import: copy the representation to host arrays in the same
 * packed layout (a complex handle: two doubles per element, h2_stats.is_complex).  Pass NULL for the arrays to query sizes only: the element counts
 * are written to sizes[0..5] = {ranks (each of kr, kc), vr, vc, er, ec, s, f}
 * (sizes has 8 entries: nranks, nvr, nvc, ner, nec, ns, nf, 0). */
h2_status h2_export(h2_handle h, int64_t* sizes, int32_t* kr, int32_t* kc, double* vr,
                    double* vc, double* er, double* ec, double* s, double* f);

/* C = A x B with change of cluster bases (Sec. III leaf level, Sec. IV non-leaf
 * levels, top-down split of the couplings held by non-leaf blocks).  C keeps A's
 * partition and gets new orthonormal nested bases truncated at eps (see h2_trunc).
 * A and B must come from the same points, leaf size and eta (else H2_ESTRUCT).
 * The product is enqueued on opts->stream; the call returns after it has been
 * launched and synchronises only to finish its setup.  *C owns its memory.
 * In place: when *C holds, on entry, a handle made by an earlier product with the same
 * structure, storage caps, truncation, rank cap and precision, the product is written
 * into it (its old contents are replaced); any other handle in *C is left untouched and
 * replaced by a new one (the caller still owns and destroys the old).  *C must not be A
 * or B (H2_EINVAL).  A product's output may be an operand of later products in any
 * precision. */
h2_status h2_mmp(h2_handle A, h2_handle B, double eps, const h2_opts* opts,
                 h2_handle* C);

/* C[i] = A[i] x B[i] for i < count: independent products (for instance problems of
 * different sizes) enqueued in order on opts->stream with the same eps and options.
 * Instances with equal points, leaf size and eta share one cached program and its
 * work regions, which is safe because the products run in stream order.  C[i] follow
 * the in-place rule of h2_mmp.  On an error the products of instances before the
 * failing one have been enqueued and their C[i] are valid; the error names the
 * instance. */
h2_status h2_mmp_batched(const h2_handle* A, const h2_handle* B, int32_t count, double eps,
                         const h2_opts* opts, h2_handle* C);

/* y = H x in exact H^2 arithmetic (Sec. II representation; the products A(B x) of
 * Eq. error in Sec. VI-A are formed with it): forward transform with the column bases,
 * coupling matrices, backward transform with the row bases, plus the dense near field.
 * x, y: device float64 (complex handles: two doubles per entry), column-major n x nrhs,
 * user order; y is overwritten (x and y must not overlap).  nrhs 1..16384.  Enqueued on the stream of the handle's
 * last call.  Errors: H2_EINVAL for null pointers or nrhs out of range. */
h2_status h2_matvec(h2_handle h, const double* x, double* y, int64_t nrhs);

/* y = H x like h2_matvec (real handles; H2_EUNSUPPORTED for complex ones), but the call
 * allocates no memory at all: its work space
 * (the tree-ordered copies of x and y, the coefficient vectors of every level and
 * the block lists) lives in one fixed 32 MiB array compiled into the library.  The
 * paper has no counterpart; it exists for callers that may not allocate device
 * memory during the call, such as code running under a device-memory budget fixed
 * in advance, or hosts that gave all free device memory to another allocator.
 *   x, y   device float64, column-major n x nrhs, user order; y is overwritten.
 *   nrhs   1..64.
 * Returns H2_EINVAL when the matrix and nrhs need more than the 32 MiB (roughly
 * n * nrhs * 16 bytes plus the coefficient vectors and block lists).  Every device
 * that loads the library holds the array until the process exits.  All calls share
 * it: calls that overlap on the GPU (different streams or threads) race and return
 * wrong results.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress).  Every call copies the block lists from pageable host
 * memory into the array (cudaMemcpyAsync), which stream capture does not support:
 * do not capture the call into a CUDA graph.
 * Enqueued on the stream of the handle's last call. */
h2_status h2_matvec_noalloc(h2_handle h, const double* x, double* y, int64_t nrhs);

/* Dense n x n matrix of the H^2 matrix (Sec. II: R blocks V_t S_ts V_s^T through the
 * nested bases, F blocks as stored), device float64 (complex: two doubles per entry),
 * column-major, user order; for testing, n <= 16384 (H2_EINVAL above).  Synchronises the
 * handle's stream. */
h2_status h2_to_dense(h2_handle h, double* out);

/* Statistics; synchronises. */
h2_status h2_info(h2_handle h, h2_stats* stats);

/* Tree order of the points: perm[p] = user index of tree position p (host, n
 * entries); and the blocks of one level, sorted by (t, s): kind 0 = admissible R,
 * 1 = dense F, 2 = non-leaf NL.  Pass NULL arrays to query *count. */
h2_status h2_tree_perm(h2_handle h, int64_t* perm);
h2_status h2_level_blocks(h2_handle h, int32_t level, int32_t* t, int32_t* s,
                          int8_t* kind, int64_t* count);

/* Kernel timing of the next products made from A (device events around every
 * launch group of h2_mmp; off by default because it adds event records).  After a
 * product, h2_trace_read returns, for up to `cap` launch groups in program order,
 * the kernel kind (0 GEMM, 1 eigen, 2 memset), the level, the device time in ms and
 * a work count: for a GEMM group the multiply-add flops at the plan's padded dims
 * (2 m n k per product), for an eigen group the number of cluster bases it decomposes;
 * *count gets the number of groups.  Synchronises. */
h2_status h2_trace_enable(h2_handle A, int32_t on);
h2_status h2_trace_read(h2_handle C, int32_t cap, int32_t* kind, int32_t* level, double* ms,
                        double* flops, int32_t* count);
/* Number of CUDA kernels this library has launched in this process so far (GEMM,
 * eigen, conversion and permutation kernels; not the no-allocation matvec's, and
 * not the memsets and copies made through the CUDA runtime).  The difference of two readings counts the
 * kernels of the calls in between; pure host function, never fails for a non-NULL
 * argument. */
h2_status h2_kernel_launches(uint64_t* count);
/* Multiply-add flops (2 per multiply-add) the GEMM kernel executed at the actual
 * ranks during the traced product that made C (counted on the device). */
h2_status h2_trace_flops(h2_handle C, double* executed);
/* Name of the phase of launch group i of the traced product (static string; NULL
 * if out of range): bprod, rprod, leaf_blockprod, leaf_dense_gram, leaf_dense,
 * collect, nl_gram, eig, proj, rimage, coup, split, zero. */
const char* h2_trace_phase(h2_handle C, int32_t i);

void h2_destroy(h2_handle h);
const char* h2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
