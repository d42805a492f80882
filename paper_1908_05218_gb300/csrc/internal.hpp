// Internal declarations of the H^2 library (host side).
#pragma once
#include <array>
#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/h2.h"

namespace h2 {

// Error carried to the C ABI boundary.
struct Error : std::runtime_error {
  h2_status code;
  Error(h2_status c, const std::string& m) : std::runtime_error(m), code(c) {}
};

enum BlockKind : int8_t { KR = 0, KF = 1, KNL = 2 };

struct Block {
  int32_t t, s;
  int8_t kind;
  int64_t idx;  // index among R blocks of its level, or among F blocks
};

// Cluster tree and block partition (Sec. II): complete binary tree, root level 0,
// leaves at level L, cluster t of level l has children 2t, 2t+1.
struct Structure {
  int64_t n = 0;
  int leaf_size = 0;
  double eta = 0;
  int L = 0;
  int LS = 0;  // largest leaf cluster (padded row count of leaf blocks)
  std::vector<double> pts;  // tree order, n x 3
  std::vector<int64_t> perm;  // tree position -> user index
  std::vector<std::vector<int64_t>> start, size;  // per level, per cluster
  std::vector<std::vector<std::array<double, 3>>> lo, hi;
  std::vector<std::vector<Block>> blocks;  // per level, sorted by (t, s)
  std::vector<std::vector<int32_t>> row_ptr;  // CSR over blocks[l] by row cluster
  std::vector<std::vector<int32_t>> col_ptr, col_list;  // CSC: positions by column
  std::vector<int64_t> nR;  // admissible blocks per level
  int64_t nF = 0;
  int lmin = 0;
  int csp = 0;

  // position of block (t, s) in blocks[l], -1 if absent: a binary search over row t's
  // blocks, which are sorted by s
  int32_t find(int l, int64_t t, int64_t s) const {
    const std::vector<int32_t>& rp = row_ptr[l];
    if (t < 0 || t + 1 >= (int64_t)rp.size()) return -1;
    const std::vector<Block>& bl = blocks[l];
    int32_t lo = rp[t], hi = rp[t + 1];
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo) / 2;
      if (bl[mid].s < s) lo = mid + 1;
      else hi = mid;
    }
    return (lo < rp[t + 1] && bl[lo].s == s) ? lo : -1;
  }
  static int node(int l, int64_t t) { return (int)((1LL << l) - 1 + t); }
  int nnodes() const { return (int)((1LL << (L + 1)) - 1); }
};

std::shared_ptr<Structure> build_structure(const double* user_pts, int64_t n, int leaf_size,
                                           double eta);
bool same_structure(const Structure& a, const Structure& b);

// Numeric H^2 matrix on the device.  All matrices row-major, padded: a leaf basis
// is LS x K[L]; the stacked transfer of a level-l cluster is 2K[l+1] x K[l] (child 1
// in rows [0, K[l+1]), child 2 in rows [K[l+1], 2K[l+1])); couplings K_r[l] x K_c[l];
// dense blocks LS x LS.  Every padded entry is exactly zero.
struct Mat {
  std::shared_ptr<Structure> st;
  std::vector<int> Kr, Kc;  // caps (padded dims) per level
  double* arena = nullptr;  // device
  int64_t arena_elems = 0;
  int64_t off_Vr = 0, off_Vc = 0, off_F = 0;
  std::vector<int64_t> off_Er, off_Ec, off_S;
  int32_t* d_kr = nullptr;  // device ranks, indexed by Structure::node
  int32_t* d_kc = nullptr;
  float* arena32 = nullptr;  // float copy of the arena (mixed precision), made on first use
  int64_t arena32_cap = 0;     // floats allocated for arena32 (the copy, then the F tiles)
  bool arena32_stale = false;  // the arena was rewritten (by a product) since arena32 was made
  bool ftiles = false;         // arena32 also holds the operand tiles of the dense blocks
  float* bases32 = nullptr;  // float copy of the bases written by a mixed product into this matrix
  std::vector<int32_t> h_kr, h_kc;  // host copies
  bool ranks_on_host = false;
  unsigned long long* d_cap = nullptr;  // device counter of ranks cut at the cap
  void* stream = nullptr;
  std::vector<void*> extra_allocs;  // device buffers owned by the handle
  bool cplx = false;                // complex float64 (double2) elements: complex kernel functions
  size_t esize() const { return cplx ? 16 : 8; }

  int64_t Vr(int64_t t) const { return off_Vr + t * st->LS * Kr[st->L]; }
  int64_t Vc(int64_t t) const { return off_Vc + t * st->LS * Kc[st->L]; }
  int64_t Er(int l, int64_t t) const { return off_Er[l] + t * 2LL * Kr[l + 1] * Kr[l]; }
  int64_t Ec(int l, int64_t t) const { return off_Ec[l] + t * 2LL * Kc[l + 1] * Kc[l]; }
  int64_t S(int l, int64_t r) const { return off_S[l] + r * (int64_t)Kr[l] * Kc[l]; }
  int64_t F(int64_t f) const { return off_F + f * (int64_t)st->LS * st->LS; }
};

int64_t mat_elems(Mat& m);  // computes the offsets from the caps; returns the arena size
void alloc_mat(Mat& m);  // computes offsets from caps, allocates + zeroes arena and ranks
void free_mat(Mat& m);
void sync_ranks_to_host(Mat& m);

// ---------------------------------------------------------------- device program
// Offsets into one of eight arenas: the tag in bits 60-62 selects it, so a tagged
// offset is never negative and -1 can mark "absent".  A, B, C are the matrices; P
// holds data that lives for the whole product (couplings of non-leaf targets of C
// until the top-down split), G0/G1 hold what level l hands to level l-1 (ping-pong
// by level parity), S holds the temporaries of one level.
enum Arena : int64_t { AR_A = 0, AR_B = 1, AR_C = 2, AR_P = 3, AR_G0 = 4, AR_G1 = 5, AR_S = 6, AR_X = 7 };
constexpr int kArenas = 8;
constexpr int kTagShift = 60;
// storage caps are multiples of four (16-byte rows and offsets for float32 copies)
inline int cap_round(int k) { return (k + 3) & ~3; }
constexpr int64_t kOffMask = (int64_t(1) << kTagShift) - 1;
inline int64_t tag(Arena a, int64_t off) { return (a << kTagShift) | off; }
inline int arena_of(int64_t t) { return (int)((t >> kTagShift) & 7); }
inline int64_t offset_of(int64_t t) { return t & kOffMask; }

// Segmented batched GEMM: out[m x n] (=|+=) sum_items op(A) op(B), one CTA per segment.
// m, n, k are the padded dims; a dim reference (rank array << kRefShift | cluster node,
// -1 = none) bounds the loop by the actual rank read on the device, so padded zeros
// are skipped.  Rank arrays: 0 A.kr, 1 A.kc, 2 B.kr, 3 B.kc, 4 C.kr, 5 C.kc.
// SF_CA / SF_CB: conjugate A / B (complex operands; real kernels ignore them).
// SF_TILE: the output (a sum segment: its inputs) is a tensor-core operand tile (BF16
// split, device.cuh) of trows rows and ldc (sum: lda) columns; with SF_TILE_T the matrix
// element (r, c) sits at tile position (c, r).  Only in products of H2_MIXED_BF16X3.
enum SegFlags : uint8_t { SF_TA = 1, SF_TB = 2, SF_ACC = 4, SF_SUM = 8, SF_CA = 16, SF_CB = 32, SF_TILE = 64,
                          SF_TILE_T = 128 };
// Seg::flags2, SF2_SYM: the output block lies on the diagonal of a symmetric matrix (m ==
// n, mref == nref): the float32 kernel computes its lower tiles and 4 x 4 blocks and writes
// each off-diagonal one to both positions (mixed real products only)
enum SegFlags2 : uint8_t { SF2_SYM = 1 };
enum RankSrc : int32_t { RK_AR = 0, RK_AC = 1, RK_BR = 2, RK_BC = 3, RK_CR = 4, RK_CC = 5 };
constexpr int kRefShift = 26;
inline int32_t rref(RankSrc s, int node) { return (int32_t)((s << kRefShift) | node); }
struct Seg {
  int64_t out;
  int32_t first, count;
  int16_t m, n, k, lda, ldb, ldc;
  int32_t mref, nref;
  uint8_t flags;
  uint8_t flags2;  // SegFlags2
  int16_t inst;  // product instance: index into the launch's arena tables (0 for one product)
  int32_t trows;  // SF_TILE: rows of the tile (a multiple of 8)
};
struct Item {
  int64_t a = 0, b = 0;
  int32_t kref = -1;         // bound of this item's k (see Seg), -1 = none
  int16_t lda = 0, ldb = 0;  // this item's leading dimensions, 0 = the segment's
  int16_t kpad = 0;          // this item's padded k, 0 = the segment's
  int16_t pad0 = 0;
  int32_t pad1 = 0;
  Item() = default;
  Item(int64_t a_, int64_t b_, int32_t k_ = -1, int16_t lda_ = 0, int16_t ldb_ = 0, int16_t kpad_ = 0)
      : a(a_), b(b_), kref(k_), lda(lda_), ldb(ldb_), kpad(kpad_) {}
};

// The tensor-core coupling pass (H2_MIXED_BF16X3) sums targets in pairs: the targets
// (i, k) and (i', k) of sibling row clusters i, i' share the B operand of every common
// term, so one step multiplies the two stacked A tiles (slot 0: the even cluster, slot 1:
// the odd one) by that B tile.  A group is one such pair (or a single target); its steps
// are the union of the two targets' terms, ordered by B tile.
struct TcGroup {
  int64_t out[2];        // tagged outputs of the slots (-1: no target in the slot)
  int32_t mref[2];       // row rank references of the slots
  int32_t nref;          // column rank reference (the shared k)
  int32_t first, count;  // steps
  int16_t m, n, ldc;     // output caps (rows, columns) and leading dim
  uint8_t acc;           // bit s: slot s adds to its output (else stores it)
  uint8_t pad0;
  int16_t inst;          // product instance
  int16_t pad1;
};
struct TcStep {
  int64_t a[2];          // A tiles of the slots (rp x kpad; -1: no term for the slot)
  int64_t b;             // the B tile (np x kpad)
  int32_t kref;          // rank reference bounding k (-1: kpad)
  int16_t kpad;          // tile k, a multiple of 16
  int16_t pad0;
};

// Normalised Gram sum + eigen-decomposition + truncation for one cluster.
struct EigTask {
  int64_t g[3];      // tagged offsets of the three Gram matrices (-1: absent)
  int64_t out;       // tagged offset of the new basis / stacked transfer (n_pad x kcap)
  int32_t rank_out;  // node id whose rank is written
  int32_t child1, child2;  // node ids of the children (ranks in the same rank array), -1: leaf
  int32_t nleaf;     // leaf: cluster size; active rows [0, nleaf)
  int16_t n_pad, half, kcap, col;  // Gram dim, child offset, output row stride, 1 = column basis
  int16_t klim;                     // largest rank kept (the rank cap; <= kcap)
  int16_t inst;                     // product instance (index into the arena tables)
  int16_t pad2[2];
};

struct Launch {
  enum Kind { GEMM, EIG, MEMSET, COPY_RANKS } kind;
  int64_t first = 0, count = 0;  // range in segs / eigs
  int64_t off = 0, elems = 0;    // MEMSET: tagged offset and size
  int level = -1;
  bool tc = false;               // coupling pass on the tensor cores: first / count index the
                                 // plan's TcGroups
  bool sums = false;             // GEMM whose segments are all plain sums (SF_SUM)
  int aux = 0;                   // GEMM: largest n; EIG: largest Gram dim; tc: B tile rows
  int aux2 = 0;                  // GEMM: largest max(m, n); EIG: largest rank limit; tc: A tile rows
  int aux3 = 0;                  // tc: largest tile k
  const char* phase = "";
  double flops = 0;              // GEMM: counted 2 m n k over the group
};

// Allocator of the program's large arrays: resize() leaves new elements of trivially
// copyable types unconstructed instead of value-initialising them, so that growing an
// array by hundreds of millions of entries costs no serial fill; the loops that follow
// every such resize write each new element (in parallel, touching the pages first).
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept(std::is_nothrow_default_constructible<U>::value) {
    if constexpr (!std::is_trivially_copyable<U>::value) ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... Args>
  void construct(U* p, Args&&... args) {
    ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...);
  }
};
template <class T>
using PlanArray = std::vector<T, UninitAlloc<T>>;

struct Plan {
  PlanArray<Seg> segs;
  PlanArray<Item> items;
  std::vector<EigTask> eigs;
  PlanArray<TcGroup> tgroups;
  PlanArray<TcStep> tsteps;
  std::vector<Launch> launches;
  int64_t region[kArenas] = {0, 0, 0, 0, 0, 0, 0, 0};  // sizes of P, G0, G1, S (others 0)
  // device copies
  Seg* d_segs = nullptr;
  Item* d_items = nullptr;
  EigTask* d_eigs = nullptr;
  TcGroup* d_tgroups = nullptr;
  TcStep* d_tsteps = nullptr;
  // work regions owned by the plan (matvec plans); product plans take theirs from the
  // per-stream work space at run time (see region_bytes)
  double* d_region[kArenas] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int region_esize = 8;  // bytes per element of the work regions (4 for a mixed product, 16 complex)
  bool cplx = false;     // complex operands: complex GEMM and Hermitian eigen kernels
  int64_t scratch_elems = 0;    // float64 eigen work space for Gram matrices above 112 (taken
                                // with the work regions, so that concurrent products never share it)
  int64_t flops = 0;     // counted 2mnk over GEMM segments (padded dims)
  // elements after A's and B's float copies that the program reads: the operand tiles of
  // their dense blocks (H2_MIXED_BF16X3, ftile_elems), 0 if none
  int64_t fext = 0;
  std::vector<int> ckr, ckc;  // caps of the product
  // allocations and resets of the work regions in program order (launch = index of
  // the first launch group emitted after the event); validate_plan replays them to
  // check that every access stays inside one live allocation
  struct AllocEv {
    int32_t launch;
    int8_t arena, reset;
    int64_t start, size;
  };
  std::vector<AllocEv> aev;
};

struct MmpParams {
  double eps;
  int trunc;
  int rank_cap;
  int precision;
  int norm = H2_NORM_FROBENIUS;
  int autotune = 0;
};
// float32 operands and work regions (every precision but H2_FP64)
inline bool is_mixed(int precision) { return precision != H2_FP64; }
// Operand tiles of the dense leaf blocks for the tensor-core dense products
// (H2_MIXED_BF16X3): after a matrix's float copy (arena_elems floats), the tile of dense
// block f as an A operand (rows x k) at arena_elems + f T, and as a B operand (transposed)
// at arena_elems + (nF + f) T; T = pad8(LS) x pad16(LS) floats (BF16 hi and lo parts)
inline int64_t ftile_elems(int LS) { return (int64_t)((LS + 7) & ~7) * ((LS + 15) & ~15); }
void launch_f_tiles(const double* arena, int64_t off_F, int64_t nF, int LS, float* dst, void* stream);
// the eigen launches of the mixed product that take the kept-columns kernel (launch_eig_mixed)
inline bool eig_kept_path(const MmpParams& p, const Launch& L) {
  return is_mixed(p.precision) && L.aux <= 96 && p.norm == H2_NORM_FROBENIUS;
}

// Builds the plan of C = A B; sets C's caps (C must share A's structure).
void build_mmp_plan(const Mat& A, const Mat& B, Mat& C, const MmpParams& p, Plan& plan);
void build_matvec_plan(const Mat& H, int64_t nrhs, Plan& plan, int64_t& off_x, int64_t& off_y);
void validate_plan(const Plan& plan, const int64_t sizes[kArenas]);
// uploads the program; own_regions: allocate the work regions with the plan (matvec
// plans), else they come from the per-stream work space when the plan runs
void upload_plan(Plan& plan, size_t region_esize, bool own_regions);
void free_plan(Plan& plan);

// Runs a plan: arenas[kArenas] device base pointers.
struct Trace {
  std::vector<void*> ev;  // cudaEvent_t, 2 per launch
  bool recorded = false;
};
// Arena base pointers, which of them hold float (bit per arena), and the six rank
// arrays that dim references read.
struct ArenaSet {
  void* p[kArenas] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  uint32_t f32 = 0;
  const int32_t* rk[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  unsigned long long* flops = nullptr;  // executed-flop counter (tracing only)
  int32_t* kr = nullptr;                // the output's rank arrays (written by the eigen step)
  int32_t* kc = nullptr;
  unsigned long long* cap_hits = nullptr;
  double* eig_scratch = nullptr;        // this product's eigen work space (Plan::scratch_elems)
  unsigned int* err = nullptr;          // device word: nonzero when a bounded device wait gave up
  uint32_t c16 = 0;                     // arenas of complex elements (bit per arena; with f32: float2)
  size_t esize(int a) const {  // complex: 16 (float64) or 8 (float32); real: 8 or 4
    return ((c16 >> a) & 1) ? (((f32 >> a) & 1) ? 8 : 16) : (((f32 >> a) & 1) ? 4 : 8);
  }
};
// The same table as the kernels read it, in device memory: one per product instance of
// a launch (segments and eigen tasks carry the instance index).
struct Arenas {
  char* p[kArenas];
  uint32_t f32;
  const int32_t* rk[6];
  unsigned long long* flops;
  int32_t* kr;
  int32_t* kc;
  unsigned long long* cap_hits;
};
Arenas to_arenas(const ArenaSet& a);
// writes `a` to device memory `dst` in stream order (a one-thread kernel taking it by value)
void upload_arenas(Arenas* dst, const Arenas& a, void* stream);
// choice: per launch the launch configuration to use (null: defaults); tune_ev: two
// events per launch recorded around the GEMM launches (autotuner exploration), or null
void run_plan(const Plan& plan, const ArenaSet& ar, const Arenas* d_ars, const MmpParams& p, void* stream,
              bool skip_memset, Trace* trace = nullptr, const int8_t* choice = nullptr, void* const* tune_ev = nullptr);

// device helpers (kernels.cu)
// variant: launch configuration (0 default; see kGemmVariants), results identical for all
void launch_gemm(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                 int maxn, int maxdim, bool fp32, void* stream, int variant = 0);
// a launch group of plain sums only (real operands; fp32: float, else double)
void launch_sum(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars, bool fp32,
                void* stream);
// launch configurations the autotuner tries per GEMM launch group: CUDA-core kernels
// {column slices per CTA, whole segment per CTA}, 3xTF32 tensor-core kernel {4, 2, 1} CTAs
// per SM, BF16 coupling kernel four (stages, accumulators) pairs (tc.cu)
constexpr int kGemmVariants = 2, kMmaVariants = 3, kEigVariants = 4, kTcVariants = 4, kTuneCandidates = 4;
// the same segments on the tensor cores, 3xTF32 split products (mma.cu); maxm / maxn bound
// the segments' padded dims; err receives 1 if a bounded wait gave up; variant: launch
// configuration (k per stage, CTAs per SM; results identical for all)
void launch_gemm_mma(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                     int maxm, int maxn, unsigned int* err, int variant, void* stream);
// coupling sums from operand tiles on the tensor cores (tc.cu): groups of up to two
// targets with their steps (A tiles rp x kpad, B tile np x kpad), rp, np the launch's tile
// rows, kpmax its largest k
void init_coup_tc_attributes();  // once per process, before launches or captures (kernel attributes)
void launch_coup_tc(const TcGroup* d_groups, const TcStep* d_steps, int64_t first, int64_t count,
                    const Arenas* d_ars, int rp, int np, int kpmax, unsigned int* err, int variant, void* stream);
void launch_eig(const EigTask* d_eigs, int64_t first, int64_t count, const Arenas* d_ars, double eps, int trunc,
                int norm, int max_npad, double* scratch, void* stream);
// formatted product: C's ranks are A's row ranks and B's column ranks (instance inst)
void launch_copy_ranks(const Arenas* d_ars, int inst, int64_t n, void* stream);
unsigned long long kernel_launches();  // kernels launched by this library so far
void add_kernel_launches(long long d);
void init_kernel_attributes();  // once per process, before launches or captures   // graph replays add their kernels; captures take theirs back
void launch_to_f32(const double* src, float* dst, int64_t n, void* stream);
// the auxiliary streams on which launch_eig_mixed runs its size tiers concurrently, one
// set per calling stream: made before a stream capture that will use them, and handed
// back before the calling stream is destroyed
void prepare_eig_streams(void* stream);
void release_eig_streams(void* stream);
// variant: the threads per size tier (64, 128 or 256; results identical for all)
void launch_eig_mixed(const EigTask* d_eigs, int64_t first, int64_t count, const Arenas* d_ars, double eps,
                      int trunc, int max_npad, int variant, void* stream);
void launch_permute(const double* src, double* dst, const int64_t* user, int64_t rows, int64_t n,
                    int64_t nrhs, bool to_tree, void* stream);
void launch_identity(double* out, int64_t n, void* stream);
h2_status matvec_noalloc(const Mat& m, const int64_t* d_user, const double* x, double* y, int64_t nrhs,
                         std::string& err);
void cuda_check(int err, const char* what);

// complex float64 kernels (zkernels.cu)
void launch_zgemm(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars, int maxn,
                  void* stream);
// the same in complex float32 (mixed product: float2 operands, float2 or double2 output)
void launch_zgemm32(const Seg* d_segs, const Item* d_items, int64_t first, int64_t count, const Arenas* d_ars,
                    int maxn, void* stream);
int64_t zeig_scratch_elems(int max_npad, int64_t count);  // float64 words of eigen work space
void launch_zeig(const EigTask* d_eigs, int64_t first, int64_t count, const Arenas* d_ars, double eps, int trunc,
                 int norm, int max_npad, double* scratch, void* stream);
void launch_zpermute(const double* src, double* dst, const int64_t* user, int64_t rows, int64_t n, int64_t nrhs,
                     bool to_tree, void* stream);
void launch_zidentity(double* out, int64_t n, void* stream);

// construction (builder.cpp): fills host arrays of the packed import layout (complex
// kernels: two doubles, real and imaginary part, per element)
struct Packed {
  std::vector<int32_t> kr, kc;
  std::vector<double> vr, vc, er, ec, s, f;
};
void build_h2_host(const Structure& st, const h2_kernel& k, double eps, Packed& out);
// the construction's parameters (builder.cpp, gbuild.cu): sampled far-field points per
// partner block (real kernels), clusters whose rows are all skeleton rows, extra
// skeleton rows above the rank, largest rank
constexpr int kBuildSamples = 24, kBuildAllRows = 64, kBuildOver = 8, kBuildMaxRank = 64;
// the same construction on the GPU for the real kernels, into m's arena (m.st set; caps,
// arena and ranks made here); H2_EUNSUPPORTED for the complex kernel
void build_h2_device(const Structure& st, const h2_kernel& k, double eps, Mat& m);
// device allocation with the library's failure injection (h2_set_alloc_limit)
void* dev_alloc(size_t bytes);
// One block moved between the packed layout and the padded arena: rows x cols, dense
// (row-major) at packed_off of the concatenated packed arrays, row stride ld at
// arena_off of the arena (transfer.cu).
struct CopyTask {
  int64_t arena_off, packed_off;
  int32_t rows, cols, ld, pad;
};
void launch_copy_tasks(const CopyTask* d_tasks, int64_t ntasks, double* packed, double* arena, bool to_arena,
                       void* stream);
// The packed arrays of a matrix as caller pointers (h2_import / h2_export): ranks, then
// vr, vc, er, ec, s, f and their lengths.
struct PackedView {
  const int32_t* kr = nullptr;
  const int32_t* kc = nullptr;
  const double* arr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t len[6] = {0, 0, 0, 0, 0, 0};
};
// lengths of the six packed arrays from the ranks (a structure's sizes and blocks)
void packed_lengths(const Structure& st, const int32_t* kr, const int32_t* kc, int64_t len[6]);
// the blocks of the packed layout in order and their places in m's arena (m's offsets set)
std::vector<CopyTask> copy_tasks(const Mat& m, const int32_t* kr, const int32_t* kc, int64_t len[6]);
void unpack_view_to_device(const PackedView& v, Mat& m);
// writes the packed arrays of m into the non-null caller pointers (host memory)
void pack_to_host(Mat& m, double* const out[6]);

}  // namespace h2
