// Device program of the product C = A B (Sec. III-IV) and of the H^2 matvec.
//
// The host walks the block structure once and emits launch groups; each group is a
// batch of independent segments (one output matrix each, a sum of small products
// over its items), an eigen batch (new bases), or a memset.  Segments of one group
// never share an output, so every sum has a fixed order: reruns are bitwise equal.
// All dims are the padded caps of the level; padded entries are exactly zero.
// The host threads emit a group's segments over contiguous ranges of its loop into
// their own buffers, joined in loop order (PlanBuilder::par, tc_par): the program does
// not depend on their number.
//
// The product's phases (names as in the paper):
//   bprod   B_j = (V^A_{j,c})^T V^B_{j,r} and its nested form (Sec. III-D, Eq.
//           nonleafproduct)
//   dense   F targets: exact products, admissible factors expanded (Sec. III-A)
//   gram    leaf row / column Grams Eq. Gr1L, Gr2L, Gr3L, case1-ch, case2-ch,
//           case3-ch.  The case-1 Gram is regrouped exactly:
//              sum_{j,k} (F_ij F_jk)(F_ij F_jk)^T = sum_j F_ij (sum_k F_jk F_jk^T) F_ij^T
//           (and its column counterpart), with k over the targets of class R/SUB.
//   eig     normalised sum, eigen-decomposition, truncation -> new bases
//   proj    Eq. leafproj / nonleafproj; collects Eq. Fcollect, nonleafA/B, NLcollect
//   coup    Eq. leafcoup_simple / nonleafcoup_simple, summed per target; the case-1
//           coupling at the leaf level is regrouped as sum_j (V^C_i^T F_ij)(F_jk V^C_k)
//   merge   2 x 2 assembly of children couplings (Eq. nonleafA, first form)
//   split   top-down split of couplings held by NL targets (Sec. IV-E)
#include <omp.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <exception>
#include <map>

#include "internal.hpp"

namespace h2 {

namespace {

enum TClass : int8_t { TC_R = 0, TC_F = 1, TC_NL = 2, TC_SUB = 3 };

// Segments and items emitted by one thread of a parallel loop (PlanBuilder::par); item
// indices in its segments are local until the buffer is appended to the program.
struct SegBuf {
  PlanArray<Seg> segs;
  PlanArray<Item> items;
  int64_t flops = 0;
};

// Emission of one segment into a sink (the program itself, or a SegBuf): out[m x n]
// (=|+=) sum over the items of op(A) op(B), or a plain sum of matrices.
template <class S>
void emit_gemm(S& d, int64_t out, int m, int n, int k, int lda, int ldb, int ldc, uint8_t fl, const Item* it,
               size_t nit, int32_t mref, int32_t nref) {
  if (m <= 0 || n <= 0 || nit == 0) return;
  if (k <= 0) return;  // zero contribution; outputs start at zero
  Seg s{};
  s.out = out;
  s.first = (int32_t)d.items.size();
  s.count = (int32_t)nit;
  s.m = (int16_t)m;
  s.n = (int16_t)n;
  s.k = (int16_t)k;
  s.lda = (int16_t)lda;
  s.ldb = (int16_t)ldb;
  s.ldc = (int16_t)ldc;
  s.mref = mref;
  s.nref = nref;
  s.flags = fl;
  if ((int64_t)d.items.size() + (int64_t)nit > INT32_MAX) throw Error(H2_ENOMEM, "plan too large");
  d.items.insert(d.items.end(), it, it + nit);
  d.segs.push_back(s);
  for (size_t q = 0; q < nit; ++q) d.flops += 2LL * m * n * (it[q].kpad ? it[q].kpad : k);
}
template <class S>
void emit_sum(S& d, int64_t out, int m, int n, int lda, int ldc, bool acc, const int64_t* mats, size_t nm) {
  if (m <= 0 || n <= 0 || nm == 0) return;
  Seg s{};
  s.out = out;
  s.first = (int32_t)d.items.size();
  s.count = (int32_t)nm;
  s.m = (int16_t)m;
  s.n = (int16_t)n;
  s.k = 0;
  s.lda = (int16_t)lda;
  s.ldb = 0;
  s.ldc = (int16_t)ldc;
  s.mref = -1;
  s.nref = -1;
  s.flags = SF_SUM | (acc ? SF_ACC : 0);
  for (size_t q = 0; q < nm; ++q) d.items.push_back(Item{mats[q], 0});
  d.segs.push_back(s);
}

// The emission calls (gemm, gemm1, sum) on a sink: PlanBuilder has them for the program
// itself, PlanBuilder::par hands each thread a set over its own buffer
template <class S>
struct Emit {
  S& d;
  void gemm(int64_t out, int m, int n, int k, int lda, int ldb, int ldc, uint8_t fl, const std::vector<Item>& it,
            int32_t mref = -1, int32_t nref = -1) {
    emit_gemm(d, out, m, n, k, lda, ldb, ldc, fl, it.data(), it.size(), mref, nref);
  }
  void gemm(int64_t out, int m, int n, int k, int lda, int ldb, int ldc, uint8_t fl, const Item* it, size_t nit,
            int32_t mref = -1, int32_t nref = -1) {
    emit_gemm(d, out, m, n, k, lda, ldb, ldc, fl, it, nit, mref, nref);
  }
  void gemm1(int64_t out, int m, int n, int k, int lda, int ldb, int ldc, uint8_t fl, int64_t a, int64_t b,
             int32_t mref = -1, int32_t nref = -1, int32_t kref = -1) {
    const Item x{a, b, kref};
    emit_gemm(d, out, m, n, k, lda, ldb, ldc, fl, &x, 1, mref, nref);
  }
  void sum(int64_t out, int m, int n, int lda, int ldc, bool acc, const std::vector<int64_t>& mats) {
    emit_sum(d, out, m, n, lda, ldc, acc, mats.data(), mats.size());
  }
  void sum(int64_t out, int m, int n, int lda, int ldc, bool acc, const int64_t* mats, size_t nm) {
    emit_sum(d, out, m, n, lda, ldc, acc, mats, nm);
  }
};

// The loop `for x in [0, n): body(x, out)` (body appends to out) in parallel: each
// thread collects a contiguous range of x in its own vector, and the vectors are joined
// in order, so the result is the serial loop's.
template <class T, class F>
std::vector<T> ordered_collect(int64_t n, F&& body) {
  std::vector<std::vector<T>> part;
  int used = 1;
#pragma omp parallel if (n >= 256)
  {
#pragma omp single
    {
      used = omp_get_num_threads();
      part.resize((size_t)used);
    }
    const int id = omp_get_thread_num();
    for (int64_t x = n * id / used; x < n * (id + 1) / used; ++x) body(x, part[(size_t)id]);
  }
  std::vector<T> out;
  size_t tot = 0;
  for (auto& v : part) tot += v.size();
  out.reserve(tot);
  for (auto& v : part) out.insert(out.end(), v.begin(), v.end());
  return out;
}

struct PlanBuilder : Emit<Plan> {
  Plan& P;
  int64_t top[kArenas] = {0, 0, 0, 0, 0, 0, 0, 0};
  size_t g0 = 0;
  explicit PlanBuilder(Plan& p) : Emit<Plan>{p}, P(p) {}

  // bump allocation in one region, 256-byte aligned
  int64_t alloc(Arena a, int64_t elems) {
    int64_t o = top[a];
    top[a] += (elems + 31) & ~int64_t(31);
    P.region[a] = std::max(P.region[a], top[a]);
    P.aev.push_back({(int32_t)P.launches.size(), (int8_t)a, 0, o, elems});
    return tag(a, o);
  }
  void reset(Arena a) {
    top[a] = 0;
    P.aev.push_back({(int32_t)P.launches.size(), (int8_t)a, 1, 0, 0});
  }
  // zero [0, top) of a region at this point of the program; the size is patched by
  // close_memset once the level has been planned
  size_t open_memset(Arena a) {
    Launch z;
    z.kind = Launch::MEMSET;
    z.off = tag(a, 0);
    z.phase = "zero";
    P.launches.push_back(z);
    return P.launches.size() - 1;
  }
  void close_memset(size_t idx, Arena a) { P.launches[idx].elems = top[a]; }
  void begin() { g0 = P.segs.size(); }
  // Rank buckets: the segments of a launch group are independent, so they are ordered by
  // cost class (floor(log2(m n sum k)) at the padded dims), largest first, keeping the
  // program order inside a class; the kernels then start the long sums first.
  void bucket() {
    const size_t n = P.segs.size() - g0;
    if (n < 2) return;
    std::vector<int> cls(n);
    int cmin = INT32_MAX, cmax = INT32_MIN;
#pragma omp parallel for schedule(static, 4096) reduction(min : cmin) reduction(max : cmax) if (n > 65536)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
      const Seg& sg = P.segs[g0 + i];
      double k = 0;
      for (int32_t q = sg.first; q < sg.first + sg.count; ++q) k += P.items[q].kpad ? P.items[q].kpad : sg.k;
      const double c = (double)sg.m * sg.n * std::max(1.0, k);
      cls[i] = -(int)std::floor(std::log2(c));
      cmin = std::min(cmin, cls[i]);
      cmax = std::max(cmax, cls[i]);
    }
    if (cmin == cmax) return;
    // stable counting sort on the class (largest cost first): the segments in nch
    // contiguous chunks, each chunk's share of every class placed after the shares of
    // the classes before it and of the earlier chunks of its class
    const size_t ncls = (size_t)(cmax - cmin) + 1;
    const int64_t nch = n > 65536 ? 64 : 1;
    std::vector<size_t> cnt((size_t)nch * ncls, 0);
#pragma omp parallel for schedule(static, 1) if (nch > 1)
    for (int64_t h = 0; h < nch; ++h)
      for (size_t i = n * h / nch; i < n * (h + 1) / nch; ++i) ++cnt[(size_t)h * ncls + (size_t)(cls[i] - cmin)];
    size_t run = 0;
    for (size_t c = 0; c < ncls; ++c)
      for (int64_t h = 0; h < nch; ++h) {
        const size_t x = cnt[(size_t)h * ncls + c];
        cnt[(size_t)h * ncls + c] = run;
        run += x;
      }
    PlanArray<Seg> sorted(n);
#pragma omp parallel for schedule(static, 1) if (nch > 1)
    for (int64_t h = 0; h < nch; ++h) {
      size_t* at = cnt.data() + (size_t)h * ncls;
      for (size_t i = n * h / nch; i < n * (h + 1) / nch; ++i) sorted[at[(size_t)(cls[i] - cmin)]++] = P.segs[g0 + i];
    }
#pragma omp parallel for schedule(static) if (nch > 1)
    for (int64_t i = 0; i < (int64_t)n; ++i) P.segs[g0 + i] = sorted[i];
  }
  void end(const char* phase, int level) {
    if (P.segs.size() > g0) {
      bucket();
      Launch L;
      L.kind = Launch::GEMM;
      L.first = (int64_t)g0;
      L.count = (int64_t)(P.segs.size() - g0);
      L.level = level;
      L.phase = phase;
      P.launches.push_back(L);
    }
  }
  void eigs(size_t e0, const char* phase, int level) {
    if (P.eigs.size() > e0) {
      Launch L;
      L.kind = Launch::EIG;
      L.first = (int64_t)e0;
      L.count = (int64_t)(P.eigs.size() - e0);
      L.level = level;
      L.phase = phase;
      P.launches.push_back(L);
    }
  }
  // The loop `for x in [0, n): body(x, e)` with the segments emitted through e (an
  // Emit<SegBuf>) in parallel: each thread takes a contiguous range of x into its own
  // buffer, and the buffers are appended in thread order with their item indices
  // rebased, so the program is the one the serial loop writes.  The body must not
  // allocate (alloc / reset) or touch the program directly.
  template <class F>
  void par(int64_t n, F&& body) {
    if (n <= 0) return;
    std::vector<SegBuf> buf;
    std::vector<std::exception_ptr> err;
    int used = 1;
    if (n < 4096) {
      buf.resize(1);
      Emit<SegBuf> e{buf[0]};
      for (int64_t x = 0; x < n; ++x) body(x, e);
    } else {
#pragma omp parallel
      {
#pragma omp single
        {
          used = omp_get_num_threads();
          buf.resize((size_t)used);
          err.resize((size_t)used);
        }
        const int id = omp_get_thread_num();
        const int64_t lo = n * id / used, hi = n * (id + 1) / used;
        try {
          Emit<SegBuf> e{buf[(size_t)id]};
          for (int64_t x = lo; x < hi; ++x) body(x, e);
        } catch (...) {
          err[(size_t)id] = std::current_exception();
        }
      }
      for (auto& e : err)
        if (e) std::rethrow_exception(e);
    }
    std::vector<size_t> so((size_t)used + 1, 0), io((size_t)used + 1, 0);
    for (int t = 0; t < used; ++t) {
      so[t + 1] = so[t] + buf[t].segs.size();
      io[t + 1] = io[t] + buf[t].items.size();
      P.flops += buf[t].flops;
    }
    const size_t s0 = P.segs.size(), i0 = P.items.size();
    if ((int64_t)(i0 + io[used]) > INT32_MAX) throw Error(H2_ENOMEM, "plan too large");
    P.segs.resize(s0 + so[used]);
    P.items.resize(i0 + io[used]);
#pragma omp parallel for schedule(static, 1) if (used > 1)
    for (int t = 0; t < used; ++t) {
      const int32_t base = (int32_t)(i0 + io[t]);
      Seg* ds = P.segs.data() + s0 + so[t];
      for (size_t q = 0; q < buf[t].segs.size(); ++q) {
        ds[q] = buf[t].segs[q];
        ds[q].first += base;
      }
      std::copy(buf[t].items.begin(), buf[t].items.end(), P.items.begin() + (i0 + io[t]));
    }
  }
  // Tensor-core groups written in parallel: body(g, steps, flops) appends the steps of
  // group g (0 <= g < ng) to `steps` (its thread's buffer), adds their flops and returns
  // the group with `first` = the position of its first step in that buffer; each thread
  // takes a contiguous range of g, and the buffers are appended to the program in group
  // order with `first` rebased.  Returns the flops of all groups.
  template <class F>
  int64_t tc_par(int64_t ng, F&& body) {
    if (ng <= 0) return 0;
    struct Buf {
      PlanArray<TcStep> steps;
      PlanArray<TcGroup> groups;
      int64_t fl = 0;
    };
    std::vector<Buf> buf;
    std::vector<std::exception_ptr> err;
    int used = 1;
#pragma omp parallel if (ng >= 4096)
    {
#pragma omp single
      {
        used = omp_get_num_threads();
        buf.resize((size_t)used);
        err.resize((size_t)used);
      }
      const int id = omp_get_thread_num();
      const int64_t lo = ng * id / used, hi = ng * (id + 1) / used;
      try {
        Buf& b = buf[(size_t)id];
        for (int64_t g = lo; g < hi; ++g) b.groups.push_back(body(g, b.steps, b.fl));
      } catch (...) {
        err[(size_t)id] = std::current_exception();
      }
    }
    for (auto& e : err)
      if (e) std::rethrow_exception(e);
    std::vector<size_t> so((size_t)used + 1, 0), go((size_t)used + 1, 0);
    int64_t fl = 0;
    for (int t = 0; t < used; ++t) {
      so[t + 1] = so[t] + buf[t].steps.size();
      go[t + 1] = go[t] + buf[t].groups.size();
      fl += buf[t].fl;
    }
    const size_t st0 = P.tsteps.size(), gr0 = P.tgroups.size();
    if ((int64_t)(st0 + so[used]) > INT32_MAX) throw Error(H2_ENOMEM, "plan too large");
    P.tsteps.resize(st0 + so[used]);
    P.tgroups.resize(gr0 + go[used]);
#pragma omp parallel for schedule(static, 1) if (used > 1)
    for (int t = 0; t < used; ++t) {
      std::copy(buf[t].steps.begin(), buf[t].steps.end(), P.tsteps.begin() + (st0 + so[t]));
      TcGroup* dg = P.tgroups.data() + gr0 + go[t];
      for (size_t q = 0; q < buf[t].groups.size(); ++q) {
        dg[q] = buf[t].groups[q];
        dg[q].first += (int32_t)(st0 + so[t]);
      }
    }
    return fl;
  }
};

struct Triple {
  int32_t pa, pb;  // block positions of (i, j) in A and (j, k) in B
  int32_t tgt;     // target id of (i, k)
};

struct Target {
  int32_t i, k;
  int8_t cls;
  int64_t ssum = -1;   // tagged offset of the summed coupling (R: C's S; SUB/NL: W)
  int32_t cpos = -1;   // position of the block in C's level list (R, F, NL targets)
  bool has_nlnl = false;
};

// lists of values by key in one array (CSR), filled in two passes over the same
// sequence of (key, value): count, then put; each list keeps the order of its puts
template <typename V>
struct Lists {
  std::vector<int64_t> off, cur;
  PlanArray<V> val;  // every entry written by put after finish_count
  explicit Lists(size_t nkeys = 0) : off(nkeys + 1, 0) {}
  void count(size_t key) { ++off[key + 1]; }
  void finish_count() {
    for (size_t k = 1; k < off.size(); ++k) off[k] += off[k - 1];
    val.resize((size_t)off.back());
    cur.assign(off.begin(), off.end() - 1);
  }
  void put(size_t key, const V& v) { val[(size_t)cur[key]++] = v; }
  const V* ptr(size_t key) const { return val.data() + off[key]; }
  size_t size(size_t key) const { return (size_t)(off[key + 1] - off[key]); }
  bool empty(size_t key) const { return off[key + 1] == off[key]; }
};

struct LevelTargets {
  std::vector<Target> tg;       // by row cluster i, then in order of first appearance
  std::vector<int64_t> first;   // targets of row cluster i: [first[i], first[i + 1])
  std::vector<int64_t> tfirst;  // triples of row cluster i: [tfirst[i], tfirst[i + 1])
  std::vector<int32_t> byk;     // the same ranges, ids sorted by column cluster k
  std::vector<Triple> trip;
  Lists<Item> g1;               // leaf case-1 items by target (V^C_i^T F_ij, F_jk V^C_k)
  int32_t find(int64_t i, int64_t k) const {
    int64_t lo = first[i], hi = first[i + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (tg[byk[mid]].k < k) lo = mid + 1;
      else hi = mid;
    }
    return (lo < first[i + 1] && tg[byk[lo]].k == k) ? byk[lo] : -1;
  }
};

int8_t classify(const Structure& st, int l, int64_t i, int64_t k, int32_t& pos) {
  pos = st.find(l, i, k);
  if (pos >= 0) return st.blocks[l][pos].kind;  // R, F or NL
  for (int lv = l - 1; lv >= 0; --lv) {
    int32_t q = st.find(lv, i >> (l - lv), k >> (l - lv));
    if (q >= 0) {
      if (st.blocks[lv][q].kind == KR) return TC_SUB;
      break;
    }
  }
  throw Error(H2_EINTERNAL, "target pair neither a block nor inside an admissible block");
}

void enumerate(const Structure& st, int l, LevelTargets& lt) {
  const auto& bl = st.blocks[l];
  const auto& rp = st.row_ptr[l];
  const int64_t nc = (int64_t)1 << l;
  // each row cluster i independently (its blocks are one run, sorted by column): the
  // targets (i, k) in order of first appearance and the triples in block order; counted
  // in a first pass, written at their offsets in a second
  std::vector<int64_t> ntg(nc + 1, 0), ntr(nc + 1, 0);
  for (int pass = 0; pass < 2; ++pass) {
#pragma omp parallel
    {
      std::vector<int32_t> mark((size_t)nc, -1);  // local target number by column cluster k
      std::vector<int64_t> touched;
#pragma omp for schedule(dynamic, 64)
      for (int64_t i = 0; i < nc; ++i) {
        int32_t nt = 0;
        int64_t ntrip = 0;
        for (int32_t pa = rp[i]; pa < rp[i + 1]; ++pa) {
          const int64_t j = bl[pa].s;
          for (int32_t pb = rp[j]; pb < rp[j + 1]; ++pb) {
            const int64_t k = bl[pb].s;
            int32_t id = mark[k];
            if (id < 0) {
              id = nt++;
              mark[k] = id;
              touched.push_back(k);
              if (pass == 1) {
                Target t;
                t.i = (int32_t)i;
                t.k = (int32_t)k;
                t.cls = classify(st, l, i, k, t.cpos);
                lt.tg[ntg[i] + id] = t;
              }
            }
            if (pass == 1) {
              const int32_t gid = (int32_t)(ntg[i] + id);
              lt.trip[ntr[i] + ntrip] = {pa, pb, gid};
              if (bl[pa].kind == KNL && bl[pb].kind == KNL) lt.tg[gid].has_nlnl = true;
            }
            ++ntrip;
          }
        }
        for (int64_t k : touched) mark[k] = -1;
        touched.clear();
        if (pass == 1) {
          int32_t* b = lt.byk.data() + ntg[i];
          for (int32_t q = 0; q < nt; ++q) b[q] = (int32_t)(ntg[i] + q);
          std::sort(b, b + nt, [&](int32_t x, int32_t y) { return lt.tg[x].k < lt.tg[y].k; });
        }
        if (pass == 0) {
          ntg[i + 1] = nt;
          ntr[i + 1] = ntrip;
        }
      }
    }
    if (pass == 0) {
      for (int64_t i = 0; i < nc; ++i) {
        ntg[i + 1] += ntg[i];
        ntr[i + 1] += ntr[i];
      }
      lt.tg.assign((size_t)ntg[nc], Target());
      lt.trip.resize((size_t)ntr[nc]);
      lt.byk.resize((size_t)ntg[nc]);
      lt.first = ntg;
      lt.tfirst = ntr;
    }
  }
}

}  // namespace

void build_mmp_plan(const Mat& A, const Mat& B, Mat& C, const MmpParams& prm, Plan& P) {
  const Structure& st = *A.st;
  const int L = st.L, LS = st.LS, lmin = st.lmin;
  PlanBuilder pb(P);
  // complex operands (complex kernel functions): the program is the same, with the
  // conjugations of the paper's formulas on the operands (flags SF_CA / SF_CB, ignored
  // for real operands), and P^B of the nested projection formed without conjugation
  const bool cplx = A.cplx;
  P.cplx = cplx;
  C.cplx = cplx;
  {
    // room for the program up front (the arrays reach GBs at N = 1M: growing them by
    // reallocation copies them several times): about 1.5 items per triple (i, j, k) and
    // 18 segments per block on the cube-array workloads; the estimate only sizes the
    // reservation
    int64_t trip = 0, nblk = 0;
    for (int l = 0; l <= L; ++l) {
      const auto& rp = st.row_ptr[l];
      const auto& cp = st.col_ptr[l];
      for (int64_t j = 0; j < ((int64_t)1 << l); ++j) trip += (int64_t)(cp[j + 1] - cp[j]) * (rp[j + 1] - rp[j]);
      nblk += (int64_t)st.blocks[l].size();
    }
    P.items.reserve(P.items.size() + (size_t)(trip + trip / 2 + 16 * nblk));
    P.segs.reserve(P.segs.size() + (size_t)(20 * nblk));
    P.aev.reserve(P.aev.size() + (size_t)(20 * nblk));  // about 15 allocations per block
    // the tensor-core passes' steps: at most one per coupling term and dense product
    if (prm.precision == H2_MIXED_BF16X3 && !A.cplx) P.tsteps.reserve(P.tsteps.size() + (size_t)(trip + trip / 2));
  }
  // caps of C: leaf LS, non-leaf min(2 K[l+1], cap) (no cap in full mode), 0 above l_min;
  // each rounded up to a multiple of four for storage
  const bool formatted = prm.trunc == H2_TRUNC_FORMATTED;
  C.Kr.assign(L + 1, 0);
  C.Kc.assign(L + 1, 0);
  if (formatted) {  // C keeps A's row bases and B's column bases
    C.Kr = A.Kr;
    C.Kc = B.Kc;
  } else {
    // (storage caps rounded up to multiples of four; the rank limit is kept apart)
    C.Kr[L] = C.Kc[L] = cap_round(LS);
    for (int l = L - 1; l >= lmin; --l) {
      int cap = prm.trunc == H2_TRUNC_FULL ? 1 << 20 : prm.rank_cap;
      C.Kr[l] = cap_round(std::min(2 * C.Kr[l + 1], cap));
      C.Kc[l] = cap_round(std::min(2 * C.Kc[l + 1], cap));
    }
  }
  mat_elems(C);  // offsets of C's arrays
  // H2_MIXED_BF16X3: the main coupling pass of a level runs on the tensor cores from BF16
  // split operand tiles (tc.cu) where the tiles fit (rows, columns and k from 1 to 64):
  // the producers of its operands (projections, R images) write them as tiles of RP (A
  // operands: rows of C's row cluster) or NP (B operands, transposed: columns of C's
  // column cluster) rows and KP columns, and the next level's collects read them as tiles
  const bool tcmode = prm.precision == H2_MIXED_BF16X3 && !cplx;
  auto pad8 = [](int x) { return (x + 7) & ~7; };
  auto pad16 = [](int x) { return (x + 15) & ~15; };
  std::vector<char> tcl(L + 1, 0);
  for (int l = lmin; l <= L && tcmode; ++l)
    tcl[l] = C.Kr[l] > 0 && C.Kc[l] > 0 && pad8(C.Kr[l]) <= 64 && pad8(C.Kc[l]) <= 64 && B.Kr[l] > 0 &&
             A.Kc[l] > 0 && pad16(B.Kr[l]) <= 64 && pad16(A.Kc[l]) <= 64 && (l < L || pad16(LS) <= 64);
  // the segment just emitted, if any, writes an operand tile of tr rows and kp columns
  // (transposed: matrix element (r, c) at tile position (c, r))
  // (d: the sink the segment went to, the program or a thread's buffer)
  auto tile_out = [](auto& d, size_t nseg, int tr, int kp, bool transposed) {
    if (d.segs.size() == nseg) return;
    Seg& sg = d.segs.back();
    sg.flags |= SF_TILE | (transposed ? SF_TILE_T : 0);
    sg.ldc = (int16_t)kp;
    sg.trows = tr;
  };
  // the segment just emitted for output `out`, if any, is a diagonal block of a symmetric
  // Gram matrix: the float32 kernel computes its lower half (SF2_SYM)
  const bool symok = !cplx && (prm.precision == H2_MIXED_FP32 || prm.precision == H2_MIXED_BF16X3);
  auto sym_at = [symok](auto& d, int64_t out) {
    if (symok && !d.segs.empty() && d.segs.back().out == out) d.segs.back().flags2 |= SF2_SYM;
  };
  // the sum segment just emitted, if any, reads operand tiles
  auto tile_in = [](auto& d, size_t nseg, int tr, int kp, bool transposed) {
    if (d.segs.size() == nseg) return;
    Seg& sg = d.segs.back();
    sg.flags |= SF_TILE | (transposed ? SF_TILE_T : 0);
    sg.lda = (int16_t)kp;
    sg.trows = tr;
  };
  auto rA = [&](int l) { return A.Kr[l]; };
  auto cA = [&](int l) { return A.Kc[l]; };
  auto rB = [&](int l) { return B.Kr[l]; };
  auto cB = [&](int l) { return B.Kc[l]; };
  auto rC = [&](int l) { return C.Kr[l]; };
  auto cC = [&](int l) { return C.Kc[l]; };
  auto tA = [&](int64_t o) { return tag(AR_A, o); };
  auto tB = [&](int64_t o) { return tag(AR_B, o); };
  auto tC = [&](int64_t o) { return tag(AR_C, o); };
  // reads of C's new bases: in the mixed product the eigen step also writes a float
  // copy of them (arena X), so that every GEMM operand has the product's type
  const Arena basis_src = is_mixed(prm.precision) ? AR_X : AR_C;
  auto tCb = [&](int64_t o) { return tag(basis_src, o); };
  auto G = [](int l) { return (l & 1) ? AR_G1 : AR_G0; };
  // rank references of cluster t of level l (loop bounds read on the device)
  auto AR = [](int l, int64_t t) { return rref(RK_AR, Structure::node(l, t)); };
  auto AC = [](int l, int64_t t) { return rref(RK_AC, Structure::node(l, t)); };
  auto BR = [](int l, int64_t t) { return rref(RK_BR, Structure::node(l, t)); };
  auto BC = [](int l, int64_t t) { return rref(RK_BC, Structure::node(l, t)); };
  auto CR = [](int l, int64_t t) { return rref(RK_CR, Structure::node(l, t)); };
  auto CC = [](int l, int64_t t) { return rref(RK_CC, Structure::node(l, t)); };
  const int64_t LS2 = (int64_t)LS * LS;

  const size_t zP = pb.open_memset(AR_P);  // couplings held by NL targets accumulate
  if (formatted) {
    Launch cr;
    cr.kind = Launch::COPY_RANKS;
    cr.elems = st.nnodes();
    cr.phase = "copy_ranks";
    P.launches.push_back(cr);
  }
  // per-level data handed to the next level up (in G[level parity])
  std::vector<std::vector<int64_t>> Bj(L + 1), PA(L + 1), PB(L + 1), Ahat(L + 1), Bhat(L + 1);
  std::vector<LevelTargets> LT(L + 1);

  for (int l = L; l >= lmin; --l) {
    const bool leaf = l == L;
    const int c = l + 1;
    const Arena g = G(l);
    pb.reset(g);
    pb.reset(AR_S);
    const size_t zG = pb.open_memset(g), zS = pb.open_memset(AR_S);
    LevelTargets& lt = LT[l];
    enumerate(st, l, lt);
    const auto& bl = st.blocks[l];
    const int64_t nb = (int64_t)bl.size(), nc = 1LL << l;

    // ---- B_j (Sec. III-D, Eq. nonleafproduct)
    Bj[l].resize(nc);
    for (int64_t j = 0; j < nc; ++j) Bj[l][j] = pb.alloc(g, (int64_t)cA(l) * rB(l));
    if (leaf) {
      pb.begin();
      for (int64_t j = 0; j < nc; ++j)
        pb.gemm1(Bj[l][j], cA(l), rB(l), LS, cA(l), rB(l), rB(l), SF_TA, tA(A.Vc(j)), tB(B.Vr(j)), AC(l, j), BR(l, j));
      pb.end("bprod", l);
    } else {
      std::vector<int64_t> tmp(2 * nc);
      for (auto& x : tmp) x = pb.alloc(AR_S, (int64_t)cA(c) * rB(l));
      pb.begin();
      for (int64_t j = 0; j < nc; ++j)
        for (int a = 0; a < 2; ++a)
          pb.gemm1(tmp[2 * j + a], cA(c), rB(l), rB(c), rB(c), rB(l), rB(l), 0, Bj[c][2 * j + a],
                   tB(B.Er(l, j) + (int64_t)a * rB(c) * rB(l)), AC(c, 2 * j + a), BR(l, j), BR(c, 2 * j + a));
      pb.end("bprod", l);
      pb.begin();
      for (int64_t j = 0; j < nc; ++j) {
        std::vector<Item> it;
        for (int a = 0; a < 2; ++a)
          it.push_back({tA(A.Ec(l, j) + (int64_t)a * cA(c) * cA(l)), tmp[2 * j + a], AC(c, 2 * j + a)});
        pb.gemm(Bj[l][j], cA(l), rB(l), cA(c), cA(l), rB(l), rB(l), SF_TA, it, AC(l, j), BR(l, j));
      }
      pb.end("bprod", l);
    }

    // ---- targets: where each summed coupling lives
    for (auto& T : lt.tg) {
      if (T.cls == TC_F) continue;
      if (T.cls == TC_R) T.ssum = tC(C.S(l, bl[T.cpos].idx));
      else if (T.cls == TC_NL) T.ssum = pb.alloc(AR_P, (int64_t)rC(l) * cC(l));
      else T.ssum = pb.alloc(g, (int64_t)rC(l) * cC(l));
    }
    // R-block products of this level: T1 = S^A B_j, T2 = B_j S^B
    std::vector<int64_t> T1(nb, -1), T2(nb, -1), PAS(nb, -1), SBP(nb, -1);
    Ahat[l].assign(nb, -1);
    Bhat[l].assign(nb, -1);
    // operand tiles of the tensor-core coupling pass (tcl[l]): rows and k
    const int RP = pad8(rC(l)), NP = pad8(cC(l)), KP1 = pad16(LS), KP2 = pad16(rB(l)), KP3 = pad16(cA(l));
    for (int64_t p = 0; p < nb; ++p) {
      Ahat[l][p] = pb.alloc(g, tcl[l] ? (int64_t)RP * KP2 : (int64_t)rC(l) * rB(l));
      Bhat[l][p] = pb.alloc(g, tcl[l] ? (int64_t)NP * KP3 : (int64_t)cA(l) * cC(l));
      if (bl[p].kind == KR) {
        T1[p] = pb.alloc(AR_S, (int64_t)rA(l) * rB(l));
        T2[p] = pb.alloc(AR_S, (int64_t)cA(l) * cB(l));
        PAS[p] = pb.alloc(AR_S, tcl[l] ? (int64_t)RP * KP3 : (int64_t)rC(l) * cA(l));
        SBP[p] = pb.alloc(AR_S, tcl[l] ? (int64_t)NP * KP2 : (int64_t)rB(l) * cC(l));
      }
    }
    pb.begin();
    pb.par(nb, [&](int64_t p, auto& e) {
      const Block& b = bl[p];
      if (b.kind != KR) return;
      e.gemm1(T1[p], rA(l), rB(l), cA(l), cA(l), rB(l), rB(l), 0, tA(A.S(l, b.idx)), Bj[l][b.s], AR(l, b.t),
              BR(l, b.s), AC(l, b.s));
      e.gemm1(T2[p], cA(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, Bj[l][b.t], tB(B.S(l, b.idx)), AC(l, b.t),
              BC(l, b.s), BR(l, b.t));
    });
    pb.end("rprod", l);

    // Gram matrices of the new bases (row: gr x gr, column: gc x gc)
    const int gr = leaf ? LS : 2 * rC(c), gc = leaf ? LS : 2 * cC(c);
    std::vector<int64_t> G1r(nc, -1), G2r(nc, -1), G3r(nc, -1), G1c(nc, -1), G2c(nc, -1), G3c(nc, -1);
    // per-block factors reused after the eigen step
    std::vector<int64_t> Y(nb, -1), Yb(nb, -1), Ach(nb, -1), Bch(nb, -1), Wr(nc, -1), Wc(nc, -1), Wcp(nc, -1);
    std::vector<int64_t> Mt(lt.tg.size(), -1);

    if (leaf) {
      // ===================================================== leaf level (Sec. III)
      std::vector<int64_t> Q(nb, -1), Rr(nb, -1), Wsum(nb, -1), Wsc(nb, -1);
      for (int64_t p = 0; p < nb; ++p)
        if (bl[p].kind == KF) {
          Y[p] = pb.alloc(AR_S, (int64_t)LS * rB(l));
          Yb[p] = pb.alloc(AR_S, (int64_t)cA(l) * LS);
          // (C's leaf caps are LS rounded up to a multiple of four: V^C^T F has rC rows
          // of LS, F V^C has LS rows of stride cC)
          Q[p] = pb.alloc(AR_S, (int64_t)std::max(LS, rC(l)) * LS);   // F F^T, later F W, later V^C^T F
          Rr[p] = pb.alloc(AR_S, (int64_t)LS * std::max(LS, cC(l)));  // F^T F, later W F, later F V^C
        }
      Lists<int64_t> Ksets(nb), Isets(nb);
      const size_t ntg = lt.tg.size();
      Lists<Item> gF(ntg), gZ(ntg), gZp(ntg), gZpp(ntg), g1(ntg);
      // The lists keyed by target or by the block (i, j) hold entries of one row cluster
      // i only, so the rows are processed in parallel, each in triple order.  The lists
      // keyed by the block (j, k) (Isets) collect over the rows i of column j: they are
      // built per block from column j's blocks (i, j), which come in the order of i, the
      // order of the triples.
      auto iset_terms = [&](int64_t q, auto&& f) {
        const Block& bb = bl[q];
        if (bb.kind != KF) return;
        for (int32_t x = st.col_ptr[l][bb.t]; x < st.col_ptr[l][bb.t + 1]; ++x) {
          const int32_t pa = st.col_list[l][x];
          if (bl[pa].kind != KF) continue;
          const int32_t id = lt.find(bl[pa].t, bb.s);
          if (id < 0) throw Error(H2_EINTERNAL, "missing target");
          if (lt.tg[id].cls != TC_F) f(pa);
        }
      };
      for (int pass = 0; pass < 2; ++pass) {
        int missing = 0;
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t i = 0; i < nc; ++i)
          for (int64_t x = lt.tfirst[i]; x < lt.tfirst[i + 1]; ++x) {
            const Triple& tr = lt.trip[x];
            const Block &ba = bl[tr.pa], &bb = bl[tr.pb];
            const Target& T = lt.tg[tr.tgt];
            if (T.cls == TC_F) {
              if (ba.kind == KF && bb.kind == KF) {
                if (pass) gF.put(tr.tgt, {tA(A.F(ba.idx)), tB(B.F(bb.idx))});
                else gF.count(tr.tgt);
              } else if (ba.kind == KF) {
                if (pass) gZ.put(tr.tgt, {Y[tr.pa], tB(B.S(l, bb.idx)), BR(l, ba.s)});
                else gZ.count(tr.tgt);
              } else if (bb.kind == KF) {
                if (pass) gZp.put(tr.tgt, {tA(A.S(l, ba.idx)), Yb[tr.pb], AC(l, ba.s)});
                else gZp.count(tr.tgt);
              } else {
                if (pass) gZpp.put(tr.tgt, {T1[tr.pa], tB(B.S(l, bb.idx)), BR(l, ba.s)});
                else gZpp.count(tr.tgt);
              }
            } else if (ba.kind == KF && bb.kind == KF) {
              if (pass) {
                Ksets.put(tr.pa, Q[tr.pb]);
                g1.put(tr.tgt, {tr.pa, tr.pb});  // (V^C_i^T F_ij)(F_jk V^C_k) after the eig (blocks)
              } else {
                Ksets.count(tr.pa);
                g1.count(tr.tgt);
              }
            }
          }
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : missing)
        for (int64_t q = 0; q < nb; ++q) {
          try {
            if (pass) iset_terms(q, [&](int32_t pa) { Isets.put(q, Rr[pa]); });
            else iset_terms(q, [&](int32_t) { Isets.count(q); });
          } catch (const Error&) {
            ++missing;
          }
        }
        if (missing) throw Error(H2_EINTERNAL, "missing target");
        if (pass == 0) {
          gF.finish_count();
          gZ.finish_count();
          gZp.finish_count();
          gZpp.finish_count();
          g1.finish_count();
          Ksets.finish_count();
          Isets.finish_count();
        }
      }
      std::vector<int64_t> Z(lt.tg.size(), -1), Zp(lt.tg.size(), -1), Zpp(lt.tg.size(), -1);
      for (size_t q = 0; q < lt.tg.size(); ++q) {
        if (lt.tg[q].cls != TC_F) continue;
        if (!gZ.empty(q) || !gZpp.empty(q)) Z[q] = pb.alloc(AR_S, (int64_t)LS * cB(l));
        if (!gZp.empty(q)) Zp[q] = pb.alloc(AR_S, (int64_t)rA(l) * LS);
        if (!gZpp.empty(q)) Zpp[q] = pb.alloc(AR_S, (int64_t)rA(l) * cB(l));
      }
      for (int64_t p = 0; p < nb; ++p) {
        if (!Ksets.empty(p)) Wsum[p] = pb.alloc(AR_S, LS2);
        if (!Isets.empty(p)) Wsc[p] = pb.alloc(AR_S, LS2);
      }
      for (int64_t t = 0; t < nc; ++t) {
        G3r[t] = pb.alloc(AR_S, LS2);
        G3c[t] = pb.alloc(AR_S, LS2);
      }
      // L1: per-block products
      pb.begin();
      pb.par(nb, [&](int64_t p, auto& e) {
        const Block& b = bl[p];
        if (b.kind != KF) return;
        e.gemm1(Y[p], LS, rB(l), LS, LS, rB(l), rB(l), 0, tA(A.F(b.idx)), tB(B.Vr(b.s)), -1, BR(l, b.s));
        e.gemm1(Yb[p], cA(l), LS, LS, cA(l), LS, LS, SF_TA, tA(A.Vc(b.t)), tB(B.F(b.idx)), AC(l, b.t));
        if (formatted) return;
        e.gemm1(Q[p], LS, LS, LS, LS, LS, LS, SF_TB | SF_CB, tB(B.F(b.idx)), tB(B.F(b.idx)));
        e.gemm1(Rr[p], LS, LS, LS, LS, LS, LS, SF_TA | SF_CB, tA(A.F(b.idx)), tA(A.F(b.idx)));
      });
      if (!formatted)
        pb.par(nc, [&](int64_t t, auto& e) {
          e.gemm1(G3r[t], LS, LS, rA(l), rA(l), rA(l), LS, SF_TB | SF_CB, tA(A.Vr(t)), tA(A.Vr(t)), -1, -1, AR(l, t));
          sym_at(e.d, G3r[t]);
          e.gemm1(G3c[t], LS, LS, cB(l), cB(l), cB(l), LS, SF_TB | SF_CB, tB(B.Vc(t)), tB(B.Vc(t)), -1, -1, BC(l, t));
          sym_at(e.d, G3c[t]);
        });
      pb.end("leaf_blockprod", l);
      // L2: dense targets (Sec. III-A) and Gram pieces (the dense products F F of the
      // dense targets on the tensor cores instead, tcF below)
      const bool tcF = tcmode && ((LS + 7) & ~7) <= 64;
      pb.begin();
      pb.par((int64_t)lt.tg.size(), [&](int64_t q, auto& e) {
        const Target& T = lt.tg[q];
        if (T.cls != TC_F) return;
        if (!tcF) e.gemm(tC(C.F(bl[T.cpos].idx)), LS, LS, LS, LS, LS, LS, SF_ACC, gF.ptr(q), gF.size(q));
        e.gemm(Z[q], LS, cB(l), rB(l), rB(l), cB(l), cB(l), 0, gZ.ptr(q), gZ.size(q), -1, BC(l, T.k));
        e.gemm(Zp[q], rA(l), LS, cA(l), cA(l), LS, LS, 0, gZp.ptr(q), gZp.size(q), AR(l, T.i));
        e.gemm(Zpp[q], rA(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, gZpp.ptr(q), gZpp.size(q), AR(l, T.i),
               BC(l, T.k));
      });
      if (!formatted) {
        pb.par(nb, [&](int64_t p, auto& e) {
          e.sum(Wsum[p], LS, LS, LS, LS, false, Ksets.ptr(p), Ksets.size(p));
          e.sum(Wsc[p], LS, LS, LS, LS, false, Isets.ptr(p), Isets.size(p));
        });
        // Eq. Gr2L / case2-ch over the dense blocks of row t / column t: the Gram
        // matrices allocated first (in cluster order), then the products emitted
        for (int64_t t = 0; t < nc; ++t) {
          bool rf = false, cf = false;
          for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1] && !rf; ++p) rf = bl[p].kind == KF;
          for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1] && !cf; ++q) cf = bl[st.col_list[l][q]].kind == KF;
          if (rf) G2r[t] = pb.alloc(AR_S, LS2);
          if (cf) G2c[t] = pb.alloc(AR_S, LS2);
        }
        pb.par(nc, [&](int64_t t, auto& e) {
          std::vector<Item> r2, c2;
          for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p)
            if (bl[p].kind == KF) r2.push_back({Y[p], Y[p], BR(l, bl[p].s)});
          for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1]; ++q) {
            int32_t p = st.col_list[l][q];
            if (bl[p].kind == KF) c2.push_back({Yb[p], Yb[p], AC(l, bl[p].t)});
          }
          if (!r2.empty()) {
            e.gemm(G2r[t], LS, LS, rB(l), rB(l), rB(l), LS, SF_TB | SF_CB, r2);  // Eq. Gr2L
            sym_at(e.d, G2r[t]);
          }
          if (!c2.empty()) {
            e.gemm(G2c[t], LS, LS, cA(l), LS, LS, LS, SF_TA | SF_CB, c2);  // Eq. case2-ch
            sym_at(e.d, G2c[t]);
          }
        });
      }
      pb.end("leaf_dense_gram", l);
      if (tcF) {
        // ---- the dense products F^A_ij F^B_jk of the dense targets (i, k) on the tensor
        // cores (tc.cu): the operand tiles of A's and B's dense blocks follow their float
        // copies; targets in sibling pairs (i, i') sharing the B tile of each common j,
        // the terms of a pair merged by B tile.  Each target's F^C block is stored here
        // (its first contribution); the later passes add to it.
        const int TP = (LS + 7) & ~7, KPF = (LS + 15) & ~15;
        const int64_t Tn = ftile_elems(LS), nF = st.nF;
        P.fext = 2 * nF * Tn;
        auto fterms = [&](int64_t q, std::vector<Item>& out) {
          out.clear();
          if (q < 0) return;
          for (size_t x = 0; x < gF.size(q); ++x) {
            const Item& it = gF.ptr(q)[x];
            const int64_t fa = (offset_of(it.a) - A.off_F) / LS2, fb = (offset_of(it.b) - B.off_F) / LS2;
            out.push_back(Item(tA(A.arena_elems + fa * Tn), tB(B.arena_elems + (nF + fb) * Tn), -1, 0, 0, KPF));
          }
          std::sort(out.begin(), out.end(), [](const Item& x, const Item& y) { return x.b < y.b; });
        };
        auto fhas = [&](int64_t q) { return lt.tg[q].cls == TC_F && gF.size(q) > 0; };
        // (the targets of row cluster i are [first[i], first[i + 1]), in target order)
        const std::vector<std::array<int32_t, 2>> grp = ordered_collect<std::array<int32_t, 2>>(
            (int64_t)lt.first.size() - 1, [&](int64_t i, std::vector<std::array<int32_t, 2>>& out) {
              for (int64_t q = lt.first[i]; q < lt.first[i + 1]; ++q) {
                if (!fhas(q)) continue;
                const Target& T = lt.tg[q];
                const int32_t sib = lt.find(T.i ^ 1, T.k);
                const bool paired = sib >= 0 && fhas(sib);
                if (!(T.i & 1)) out.push_back({(int32_t)q, paired ? sib : -1});
                else if (!paired) out.push_back({-1, (int32_t)q});
              }
            });
        const int64_t ng = (int64_t)grp.size();
        auto merge = [&](const std::vector<Item>& t0, const std::vector<Item>& t1, PlanArray<TcStep>& out) {
          size_t i0 = 0, i1 = 0;
          int64_t n = 0;
          while (i0 < t0.size() || i1 < t1.size()) {
            const bool take0 = i0 < t0.size() && (i1 >= t1.size() || t0[i0].b <= t1[i1].b);
            const bool take1 = i1 < t1.size() && (i0 >= t0.size() || t1[i1].b <= t0[i0].b);
            const Item& x = take0 ? t0[i0] : t1[i1];
            TcStep sp;
            sp.a[0] = take0 ? t0[i0].a : -1;
            sp.a[1] = take1 ? t1[i1].a : -1;
            sp.b = x.b;
            sp.kref = -1;
            sp.kpad = (int16_t)KPF;
            sp.pad0 = 0;
            out.push_back(sp);
            ++n;
            if (take0) ++i0;
            if (take1) ++i1;
          }
          return n;
        };
        const size_t gr0 = P.tgroups.size();
        const int64_t fl = pb.tc_par(ng, [&](int64_t gq, PlanArray<TcStep>& steps, int64_t& flg) {
          thread_local std::vector<Item> t0, t1;
          fterms(grp[gq][0], t0);
          fterms(grp[gq][1], t1);
          const size_t f0 = steps.size();
          const int64_t n = merge(t0, t1, steps);
          TcGroup G{};
          for (int sl = 0; sl < 2; ++sl) {
            const int32_t q = grp[gq][sl];
            G.out[sl] = q >= 0 ? tC(C.F(bl[lt.tg[q].cpos].idx)) : -1;
            G.mref[sl] = -1;
          }
          G.nref = -1;
          G.first = (int32_t)f0;
          G.count = (int32_t)n;
          G.m = (int16_t)LS;
          G.n = (int16_t)LS;
          G.ldc = (int16_t)LS;
          for (size_t x = f0; x < steps.size(); ++x)
            flg += 2LL * LS * LS * KPF * ((steps[x].a[0] >= 0) + (steps[x].a[1] >= 0));
          return G;
        });
        P.flops += fl;
        if (ng > 0) {
          Launch Lc;
          Lc.kind = Launch::GEMM;
          Lc.tc = true;
          Lc.first = (int64_t)gr0;
          Lc.count = ng;
          Lc.level = l;
          Lc.phase = "leaf_dense";
          Lc.aux = TP;   // B tile rows
          Lc.aux2 = TP;  // A tile rows
          Lc.aux3 = KPF;
          Lc.flops = (double)fl;
          P.launches.push_back(Lc);
        }
      }

      // L3: Z += V^A_i Z''; F W and W F (into the storage of F F^T, F^T F)
      pb.begin();
      for (size_t q = 0; q < lt.tg.size(); ++q) {
        const Target& T = lt.tg[q];
        if (T.cls == TC_F && Zpp[q] >= 0)
          pb.gemm1(Z[q], LS, cB(l), rA(l), rA(l), cB(l), cB(l), SF_ACC, tA(A.Vr(T.i)), Zpp[q], -1, BC(l, T.k),
                   AR(l, T.i));
      }
      for (int64_t p = 0; p < nb && !formatted; ++p) {
        if (Wsum[p] >= 0) pb.gemm1(Q[p], LS, LS, LS, LS, LS, LS, 0, tA(A.F(bl[p].idx)), Wsum[p]);
        if (Wsc[p] >= 0) pb.gemm1(Rr[p], LS, LS, LS, LS, LS, LS, SF_CB, Wsc[p], tB(B.F(bl[p].idx)));
      }
      pb.end("leaf_dense_gram", l);
      // L4: Eq. Gr1L / case1-ch regrouped; dense targets, F += Z V^B_k^T
      pb.begin();
      for (size_t q = 0; q < lt.tg.size(); ++q) {
        const Target& T = lt.tg[q];
        if (T.cls == TC_F && Z[q] >= 0)
          pb.gemm1(tC(C.F(bl[T.cpos].idx)), LS, LS, cB(l), cB(l), cB(l), LS, SF_TB | SF_ACC, Z[q], tB(B.Vc(T.k)), -1,
                   -1, BC(l, T.k));
      }
      for (int64_t t = 0; t < nc && !formatted; ++t) {
        std::vector<Item> r1, c1;
        for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p)
          if (Wsum[p] >= 0) r1.push_back({Q[p], tA(A.F(bl[p].idx))});
        for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1]; ++q) {
          int32_t p = st.col_list[l][q];
          if (Wsc[p] >= 0) c1.push_back({tB(B.F(bl[p].idx)), Rr[p]});
        }
        if (!r1.empty()) {
          G1r[t] = pb.alloc(AR_S, LS2);
          pb.gemm(G1r[t], LS, LS, LS, LS, LS, LS, SF_TB | SF_CB, r1);
          sym_at(P, G1r[t]);
        }
        if (!c1.empty()) {
          G1c[t] = pb.alloc(AR_S, LS2);
          pb.gemm(G1c[t], LS, LS, LS, LS, LS, LS, SF_TA, c1);
          sym_at(P, G1c[t]);
        }
      }
      pb.end("leaf_dense_gram", l);
      pb.begin();
      for (size_t q = 0; q < lt.tg.size(); ++q) {
        const Target& T = lt.tg[q];
        if (T.cls == TC_F && Zp[q] >= 0)
          pb.gemm1(tC(C.F(bl[T.cpos].idx)), LS, LS, rA(l), rA(l), LS, LS, SF_ACC, tA(A.Vr(T.i)), Zp[q], -1, -1,
                   AR(l, T.i));
      }
      pb.end("leaf_dense", l);
      // case-1 couplings after the eig reuse Q (as V^C_i^T F_ij) and Rr (as F_jk V^C_k)
      for (int64_t p = 0; p < nb; ++p) {
        // (the tensor-core pass reads them as tiles: storage of their own, zero past the
        // written entries, instead of Q / Rr's)
        Ach[p] = tcl[l] ? (Q[p] >= 0 ? pb.alloc(AR_S, (int64_t)RP * KP1) : -1) : Q[p];
        Bch[p] = tcl[l] ? (Rr[p] >= 0 ? pb.alloc(AR_S, (int64_t)NP * KP1) : -1) : Rr[p];
      }
      lt.g1 = std::move(g1);
    } else {
      // ================================================ non-leaf level (Sec. IV)
      std::vector<int64_t> Ac(nb, -1), Bc(nb, -1);
      for (int64_t p = 0; p < nb; ++p)
        if (bl[p].kind == KNL) {
          Ac[p] = pb.alloc(AR_S, (int64_t)gr * 2 * rB(c));
          Bc[p] = pb.alloc(AR_S, (int64_t)2 * cA(c) * gc);
          Y[p] = pb.alloc(AR_S, (int64_t)gr * rB(l));
          Yb[p] = pb.alloc(AR_S, (int64_t)cA(l) * gc);
        }
      // steps 1-2: collected NL blocks of A and B (Eq. nonleafA / nonleafB)
      pb.begin();
      const int hr = rC(c), hc = cC(c);
      pb.par(nb, [&](int64_t p, auto& e) {
        const Block& b = bl[p];
        if (b.kind != KNL) return;
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) {
            int32_t cp = st.find(c, 2 * b.t + a, 2 * b.s + bb);
            if (cp < 0) throw Error(H2_EINTERNAL, "missing child block");
            size_t ns = e.d.segs.size();
            e.sum(Ac[p] + (int64_t)a * hr * 2 * rB(c) + (int64_t)bb * rB(c), hr, rB(c), rB(c), 2 * rB(c), false,
                  &Ahat[c][cp], 1);
            if (tcl[c]) tile_in(e.d, ns, pad8(rC(c)), pad16(rB(c)), false);  // the children's tiles
            ns = e.d.segs.size();
            e.sum(Bc[p] + (int64_t)a * cA(c) * gc + (int64_t)bb * hc, cA(c), hc, hc, gc, false, &Bhat[c][cp], 1);
            if (tcl[c]) tile_in(e.d, ns, pad8(cC(c)), pad16(cA(c)), true);
          }
      });
      pb.end("collect", l);
      // Gram factors: Y = (NL^A)_coll E^B_j, Yb = (E^A_j)^T (NL^B)_coll, W = P_ch E
      for (int64_t t = 0; t < nc; ++t) {
        Wr[t] = pb.alloc(AR_S, (int64_t)gr * rA(l));
        Wc[t] = pb.alloc(AR_S, (int64_t)gc * cB(l));
        if (cplx) Wcp[t] = pb.alloc(AR_S, (int64_t)gc * cB(l));
        G3r[t] = pb.alloc(AR_S, (int64_t)gr * gr);
        G3c[t] = pb.alloc(AR_S, (int64_t)gc * gc);
      }
      // (every stacked operand is taken per child half, each bounded by the child's rank:
      // the rows / columns and k past a child's rank are zero padding)
      pb.begin();
      pb.par(nb, [&](int64_t p, auto& e) {
        const Block& b = bl[p];
        if (b.kind != KNL) return;
        for (int a = 0; a < 2; ++a) {  // rows of C's row child a; k over B's row children
          std::vector<Item> it;
          for (int bb = 0; bb < 2; ++bb)
            it.push_back(Item(Ac[p] + (int64_t)a * hr * 2 * rB(c) + (int64_t)bb * rB(c),
                              tB(B.Er(l, b.s) + (int64_t)bb * rB(c) * rB(l)), BR(c, 2 * b.s + bb)));
          e.gemm(Y[p] + (int64_t)a * hr * rB(l), hr, rB(l), rB(c), 2 * rB(c), rB(l), rB(l), 0, it,
                 CR(c, 2 * b.t + a), BR(l, b.s));
        }
        for (int bc = 0; bc < 2; ++bc) {  // columns of C's column child bc; k over A's column children
          std::vector<Item> it;
          for (int aa = 0; aa < 2; ++aa)
            it.push_back(Item(tA(A.Ec(l, b.t) + (int64_t)aa * cA(c) * cA(l)),
                              Bc[p] + (int64_t)aa * cA(c) * gc + (int64_t)bc * hc, AC(c, 2 * b.t + aa)));
          e.gemm(Yb[p] + (int64_t)bc * hc, cA(l), hc, cA(c), cA(l), gc, gc, SF_TA, it, AC(l, b.t),
                 CC(c, 2 * b.s + bc));
        }
      });
      pb.par(nc, [&](int64_t t, auto& e) {
        for (int a = 0; a < 2; ++a) {
          e.gemm1(Wr[t] + (int64_t)a * hr * rA(l), hr, rA(l), rA(c), rA(c), rA(l), rA(l), 0, PA[c][2 * t + a],
                  tA(A.Er(l, t) + (int64_t)a * rA(c) * rA(l)), CR(c, 2 * t + a), AR(l, t), AR(c, 2 * t + a));
          e.gemm1(Wc[t] + (int64_t)a * hc * cB(l), hc, cB(l), cB(c), hc, cB(l), cB(l), SF_TA | SF_CB, PB[c][2 * t + a],
                  tB(B.Ec(l, t) + (int64_t)a * cB(c) * cB(l)), CC(c, 2 * t + a), BC(l, t), BC(c, 2 * t + a));
          if (cplx)  // P^B_ch^T E^B without conjugation, for the nested projection (Eq. nonleafproj)
            e.gemm1(Wcp[t] + (int64_t)a * hc * cB(l), hc, cB(l), cB(c), hc, cB(l), cB(l), SF_TA, PB[c][2 * t + a],
                    tB(B.Ec(l, t) + (int64_t)a * cB(c) * cB(l)), CC(c, 2 * t + a), BC(l, t), BC(c, 2 * t + a));
        }
      });
      // Eq. case1-ch-nl from the children's summed couplings, without assembling M:
      // block (a, a') of G1r_i = sum over targets (i, k), b of S_{ia,kb} S_{ia',kb}^T
      std::vector<std::vector<std::pair<int32_t, int32_t>>> trow(nc), tcol(nc);  // (target, -) per i / per k
      for (size_t q = 0; q < lt.tg.size(); ++q) {
        const Target& T = lt.tg[q];
        if (!T.has_nlnl || T.cls == TC_NL) continue;
        trow[T.i].push_back({(int32_t)q, 0});
        tcol[T.k].push_back({(int32_t)q, 0});
      }
      // the children's summed couplings S_{ia,kb} of each such target, looked up once
      std::vector<int64_t> css(lt.tg.size() * 4, -1);
      int missing = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : missing)
      for (int64_t q = 0; q < (int64_t)lt.tg.size(); ++q) {
        const Target& T = lt.tg[q];
        if (!T.has_nlnl || T.cls == TC_NL) continue;
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            const int32_t id = LT[c].find(2 * T.i + a, 2 * T.k + b);
            if (id < 0) ++missing;
            else css[q * 4 + a * 2 + b] = LT[c].tg[id].ssum;
          }
      }
      if (missing) throw Error(H2_EINTERNAL, "missing child target");
      auto child_ssum = [&](int32_t q, int a, int b) { return css[(size_t)q * 4 + a * 2 + b]; };
      // the Gram matrices are symmetric (real) or Hermitian: of their 2 x 2 child blocks
      // the block (1, 0) of a real one is the transpose of (0, 1), copied after the Gram
      // launches instead of computed (the same products in the same order give exactly
      // the transposed values)
      std::vector<std::array<int64_t, 3>> mirror;  // (Gram matrix, half, leading dim)
      auto skip_10 = [&](int a, int a2) { return !cplx && a == 1 && a2 == 0; };
      if (!formatted) {
        // the Gram matrices allocated first (in cluster order), then the products emitted
        for (int64_t t = 0; t < nc; ++t) {
          if (!trow[t].empty()) {
            G1r[t] = pb.alloc(AR_S, (int64_t)gr * gr);
            if (!cplx) mirror.push_back({G1r[t], hr, gr});
          }
          if (!tcol[t].empty()) {
            G1c[t] = pb.alloc(AR_S, (int64_t)gc * gc);
            if (!cplx) mirror.push_back({G1c[t], hc, gc});
          }
        }
        pb.par(nc, [&](int64_t t, auto& e) {
          if (!trow[t].empty())
            for (int a = 0; a < 2; ++a)
              for (int a2 = 0; a2 < 2; ++a2) {
                if (skip_10(a, a2)) continue;
                std::vector<Item> it;
                for (auto& tq : trow[t])
                  for (int b = 0; b < 2; ++b)
                    it.push_back({child_ssum(tq.first, a, b), child_ssum(tq.first, a2, b),
                                  CC(c, 2 * lt.tg[tq.first].k + b)});
                e.gemm(G1r[t] + (int64_t)a * hr * gr + (int64_t)a2 * hr, hr, hr, hc, hc, hc, gr, SF_TB | SF_CB, it,
                       CR(c, 2 * t + a), CR(c, 2 * t + a2));
                if (a == a2) sym_at(e.d, G1r[t] + (int64_t)a * hr * gr + (int64_t)a2 * hr);
              }
          if (!tcol[t].empty())
            for (int b = 0; b < 2; ++b)
              for (int b2 = 0; b2 < 2; ++b2) {
                if (skip_10(b, b2)) continue;
                std::vector<Item> it;
                for (auto& tq : tcol[t])
                  for (int a = 0; a < 2; ++a)
                    it.push_back({child_ssum(tq.first, a, b), child_ssum(tq.first, a, b2),
                                  CR(c, 2 * lt.tg[tq.first].i + a)});
                e.gemm(G1c[t] + (int64_t)b * hc * gc + (int64_t)b2 * hc, hc, hc, hr, hc, hc, gc, SF_TA | SF_CB, it,
                       CC(c, 2 * t + b), CC(c, 2 * t + b2));
                if (b == b2) sym_at(e.d, G1c[t] + (int64_t)b * hc * gc + (int64_t)b2 * hc);
              }
        });
      }
      pb.end("nl_gram", l);
      pb.begin();
      if (!formatted) {
        for (int64_t t = 0; t < nc; ++t) {
          bool rn = false, cn = false;
          for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1] && !rn; ++p) rn = bl[p].kind == KNL;
          for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1] && !cn; ++q) cn = bl[st.col_list[l][q]].kind == KNL;
          if (rn) {
            G2r[t] = pb.alloc(AR_S, (int64_t)gr * gr);
            if (!cplx) mirror.push_back({G2r[t], hr, gr});
          }
          if (cn) {
            G2c[t] = pb.alloc(AR_S, (int64_t)gc * gc);
            if (!cplx) mirror.push_back({G2c[t], hc, gc});
          }
          if (!cplx) {
            mirror.push_back({G3r[t], hr, gr});
            mirror.push_back({G3c[t], hc, gc});
          }
        }
        pb.par(nc, [&](int64_t t, auto& e) {
          std::vector<Item> r2, c2;
          for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p)
            if (bl[p].kind == KNL) r2.push_back({Y[p], Y[p], BR(l, bl[p].s)});
          for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1]; ++q) {
            int32_t p = st.col_list[l][q];
            if (bl[p].kind == KNL) c2.push_back({Yb[p], Yb[p], AC(l, bl[p].t)});
          }
          // (each Gram matrix in its 2 x 2 blocks of children, bounded by the children's ranks)
          if (!r2.empty())  // Eq. case2-ch-nl
            for (int a = 0; a < 2; ++a)
              for (int a2 = 0; a2 < 2; ++a2) {
                if (skip_10(a, a2)) continue;
                std::vector<Item> it;
                for (const Item& y : r2)
                  it.push_back(Item(y.a + (int64_t)a * hr * rB(l), y.b + (int64_t)a2 * hr * rB(l), y.kref));
                e.gemm(G2r[t] + (int64_t)a * hr * gr + (int64_t)a2 * hr, hr, hr, rB(l), rB(l), rB(l), gr,
                       SF_TB | SF_CB, it, CR(c, 2 * t + a), CR(c, 2 * t + a2));
                if (a == a2) sym_at(e.d, G2r[t] + (int64_t)a * hr * gr + (int64_t)a2 * hr);
              }
          if (!c2.empty())
            for (int b = 0; b < 2; ++b)
              for (int b2 = 0; b2 < 2; ++b2) {
                if (skip_10(b, b2)) continue;
                std::vector<Item> it;
                for (const Item& y : c2) it.push_back(Item(y.a + (int64_t)b * hc, y.b + (int64_t)b2 * hc, y.kref));
                e.gemm(G2c[t] + (int64_t)b * hc * gc + (int64_t)b2 * hc, hc, hc, cA(l), gc, gc, gc, SF_TA | SF_CB, it,
                       CC(c, 2 * t + b), CC(c, 2 * t + b2));
                if (b == b2) sym_at(e.d, G2c[t] + (int64_t)b * hc * gc + (int64_t)b2 * hc);
              }
          for (int a = 0; a < 2; ++a)  // Eq. case3-ch-nl
            for (int a2 = 0; a2 < 2; ++a2) {
              if (skip_10(a, a2)) continue;
              e.gemm1(G3r[t] + (int64_t)a * hr * gr + (int64_t)a2 * hr, hr, hr, rA(l), rA(l), rA(l), gr, SF_TB | SF_CB,
                      Wr[t] + (int64_t)a * hr * rA(l), Wr[t] + (int64_t)a2 * hr * rA(l), CR(c, 2 * t + a),
                      CR(c, 2 * t + a2), AR(l, t));
              if (a == a2) sym_at(e.d, G3r[t] + (int64_t)a * hr * gr + (int64_t)a2 * hr);
              e.gemm1(G3c[t] + (int64_t)a * hc * gc + (int64_t)a2 * hc, hc, hc, cB(l), cB(l), cB(l), gc, SF_TB | SF_CB,
                      Wc[t] + (int64_t)a * hc * cB(l), Wc[t] + (int64_t)a2 * hc * cB(l), CC(c, 2 * t + a),
                      CC(c, 2 * t + a2), BC(l, t));
              if (a == a2) sym_at(e.d, G3c[t] + (int64_t)a * hc * gc + (int64_t)a2 * hc);
            }
        });
      }
      pb.end("nl_gram", l);
      pb.begin();  // the (1, 0) blocks: transposes of the (0, 1) blocks (plain sums)
      pb.par((int64_t)mirror.size(), [&](int64_t x, auto& e) {
        const auto& mm = mirror[x];
        if (mm[1] <= 0) return;
        const int64_t src = mm[0] + mm[1];
        e.sum(mm[0] + mm[1] * mm[2], (int)mm[1], (int)mm[1], (int)mm[2], (int)mm[2], false, &src, 1);
        e.d.segs.back().flags |= SF_TA;
      });
      pb.end("nl_gram", l);
      for (size_t q = 0; q < lt.tg.size(); ++q)
        if (lt.tg[q].has_nlnl && lt.tg[q].cls != TC_NL) Mt[q] = pb.alloc(AR_S, (int64_t)gr * cC(l));
    }

    // ---- eig: new leaf bases / stacked transfer matrices of C (formatted product:
    // copies of A's row and B's column bases, also into the float shadow if any)
    if (formatted) {
      pb.begin();
      for (int64_t t = 0; t < nc; ++t)
        for (Arena dst : {AR_C, basis_src}) {
          if (dst == AR_X || dst == AR_C) {
            if (leaf) {
              pb.sum(tag(dst, C.Vr(t)), LS, rC(l), rC(l), rC(l), false, {tA(A.Vr(t))});
              pb.sum(tag(dst, C.Vc(t)), LS, cC(l), cC(l), cC(l), false, {tB(B.Vc(t))});
            } else {
              pb.sum(tag(dst, C.Er(l, t)), 2 * rC(c), rC(l), rC(l), rC(l), false, {tA(A.Er(l, t))});
              pb.sum(tag(dst, C.Ec(l, t)), 2 * cC(c), cC(l), cC(l), cC(l), false, {tB(B.Ec(l, t))});
            }
          }
          if (basis_src == AR_C) break;
        }
      pb.end("copy_bases", l);
    }
    size_t e0 = P.eigs.size();
    for (int64_t t = 0; t < nc && !formatted; ++t)
      for (int col = 0; col < 2; ++col) {
        EigTask e{};
        e.g[0] = col ? G1c[t] : G1r[t];
        e.g[1] = col ? G2c[t] : G2r[t];
        e.g[2] = col ? G3c[t] : G3r[t];
        e.out = tC(leaf ? (col ? C.Vc(t) : C.Vr(t)) : (col ? C.Ec(l, t) : C.Er(l, t)));
        e.rank_out = Structure::node(l, t);
        e.child1 = leaf ? -1 : Structure::node(c, 2 * t);
        e.child2 = leaf ? -1 : Structure::node(c, 2 * t + 1);
        e.nleaf = leaf ? (int32_t)st.size[l][t] : 0;
        e.n_pad = (int16_t)(col ? gc : gr);
        e.half = leaf ? 0 : (int16_t)(col ? cC(c) : rC(c));
        e.kcap = (int16_t)(col ? cC(l) : rC(l));
        e.klim = leaf ? (int16_t)LS
                      : (int16_t)std::min<int>(e.kcap, prm.trunc == H2_TRUNC_FULL ? 1 << 14 : prm.rank_cap);
        e.col = (int16_t)col;
        P.eigs.push_back(e);
      }
    pb.eigs(e0, "eig", l);

    // ---- projections (Eq. leafproj / nonleafproj) and collects (Eq. Fcollect, NLcollect)
    PA[l].resize(nc);
    PB[l].resize(nc);
    for (int64_t t = 0; t < nc; ++t) {
      PA[l][t] = pb.alloc(g, (int64_t)rC(l) * rA(l));
      PB[l][t] = pb.alloc(g, (int64_t)cB(l) * cC(l));
    }
    pb.begin();
    pb.par(nc, [&](int64_t t, auto& e) {
      if (leaf) {
        e.gemm1(PA[l][t], rC(l), rA(l), LS, rC(l), rA(l), rA(l), SF_TA | SF_CA, tCb(C.Vr(t)), tA(A.Vr(t)), CR(l, t),
                AR(l, t));
        e.gemm1(PB[l][t], cB(l), cC(l), LS, cB(l), cC(l), cC(l), SF_TA | SF_CB, tB(B.Vc(t)), tCb(C.Vc(t)), BC(l, t),
                CC(l, t));
      } else {  // (k over the children, each bounded by its rank)
        const int hr = rC(c), hc = cC(c);
        std::vector<Item> ia, ib;
        for (int a = 0; a < 2; ++a) {
          ia.push_back(Item(tCb(C.Er(l, t) + (int64_t)a * hr * rC(l)), Wr[t] + (int64_t)a * hr * rA(l), CR(c, 2 * t + a)));
          ib.push_back(Item((cplx ? Wcp[t] : Wc[t]) + (int64_t)a * hc * cB(l), tCb(C.Ec(l, t) + (int64_t)a * hc * cC(l)),
                            CC(c, 2 * t + a)));
        }
        e.gemm(PA[l][t], rC(l), rA(l), hr, rC(l), rA(l), rA(l), SF_TA | SF_CA, ia, CR(l, t), AR(l, t));
        e.gemm(PB[l][t], cB(l), cC(l), hc, cB(l), cC(l), cC(l), SF_TA | SF_CB, ib, BC(l, t), CC(l, t));
      }
    });
    // (with the tensor-core coupling pass the coupling operands go out as tiles: A
    // operands rows x k, B operands transposed)
    const bool tl = tcl[l];
    pb.par(nb, [&](int64_t p, auto& e) {
      const Block& b = bl[p];
      size_t ns = e.d.segs.size();
      if (leaf && b.kind == KF) {
        e.gemm1(Ahat[l][p], rC(l), rB(l), LS, rC(l), rB(l), rB(l), SF_TA | SF_CA, tCb(C.Vr(b.t)), Y[p], CR(l, b.t),
                BR(l, b.s));
        if (tl) tile_out(e.d, ns, RP, KP2, false);
        ns = e.d.segs.size();
        e.gemm1(Bhat[l][p], cA(l), cC(l), LS, LS, cC(l), cC(l), SF_CB, Yb[p], tCb(C.Vc(b.s)), AC(l, b.t), CC(l, b.s));
        if (tl) tile_out(e.d, ns, NP, KP3, true);
        ns = e.d.segs.size();
        e.gemm1(Ach[p], rC(l), LS, LS, rC(l), LS, LS, SF_TA | SF_CA, tCb(C.Vr(b.t)), tA(A.F(b.idx)), CR(l, b.t));
        if (tl) tile_out(e.d, ns, RP, KP1, false);
        ns = e.d.segs.size();
        e.gemm1(Bch[p], LS, cC(l), LS, LS, cC(l), cC(l), SF_CB, tB(B.F(b.idx)), tCb(C.Vc(b.s)), -1, CC(l, b.s));
        if (tl) tile_out(e.d, ns, NP, KP1, true);
      } else if (!leaf && b.kind == KNL) {  // (k over the children, each bounded by its rank)
        const int hr = rC(c), hc = cC(c);
        std::vector<Item> ia, ib;
        for (int a = 0; a < 2; ++a) {
          ia.push_back(Item(tCb(C.Er(l, b.t) + (int64_t)a * hr * rC(l)), Y[p] + (int64_t)a * hr * rB(l),
                            CR(c, 2 * b.t + a)));
          ib.push_back(Item(Yb[p] + (int64_t)a * hc, tCb(C.Ec(l, b.s) + (int64_t)a * hc * cC(l)), CC(c, 2 * b.s + a)));
        }
        e.gemm(Ahat[l][p], rC(l), rB(l), hr, rC(l), rB(l), rB(l), SF_TA | SF_CA, ia, CR(l, b.t), BR(l, b.s));
        if (tl) tile_out(e.d, ns, RP, KP2, false);
        ns = e.d.segs.size();
        e.gemm(Bhat[l][p], cA(l), cC(l), hc, gc, cC(l), cC(l), SF_CB, ib, AC(l, b.t), CC(l, b.s));
        if (tl) tile_out(e.d, ns, NP, KP3, true);
      }
    });
    if (!leaf) {
      // M E^C_k from the children's sums: half a = sum_b S_{ia,kb} T^C_{kb}
      const int hr = rC(c), hc = cC(c);
      pb.par((int64_t)lt.tg.size(), [&](int64_t q, auto& e) {
        if (Mt[q] < 0) return;
        const Target& T = lt.tg[q];
        for (int a = 0; a < 2; ++a) {
          std::vector<Item> it;
          for (int b = 0; b < 2; ++b) {
            const int32_t f = LT[c].find(2 * T.i + a, 2 * T.k + b);
            if (f < 0) throw Error(H2_EINTERNAL, "missing child target");
            it.push_back({LT[c].tg[f].ssum, tCb(C.Ec(l, T.k) + (int64_t)b * hc * cC(l)), CC(c, 2 * T.k + b)});
          }
          e.gemm(Mt[q] + (int64_t)a * hr * cC(l), hr, cC(l), hc, hc, cC(l), cC(l), SF_CB, it, CR(c, 2 * T.i + a),
                 CC(l, T.k));
        }
      });
    }
    pb.end("proj", l);
    // R images (Eq. nonleafA / nonleafB) and the case-2/3/4 factors
    pb.begin();
    pb.par(nb, [&](int64_t p, auto& e) {
      const Block& b = bl[p];
      if (b.kind != KR) return;
      size_t ns = e.d.segs.size();
      e.gemm1(Ahat[l][p], rC(l), rB(l), rA(l), rA(l), rB(l), rB(l), 0, PA[l][b.t], T1[p], CR(l, b.t), BR(l, b.s),
              AR(l, b.t));
      if (tcl[l]) tile_out(e.d, ns, RP, KP2, false);
      ns = e.d.segs.size();
      e.gemm1(Bhat[l][p], cA(l), cC(l), cB(l), cB(l), cC(l), cC(l), 0, T2[p], PB[l][b.s], AC(l, b.t), CC(l, b.s),
              BC(l, b.s));
      if (tcl[l]) tile_out(e.d, ns, NP, KP3, true);
      ns = e.d.segs.size();
      e.gemm1(PAS[p], rC(l), cA(l), rA(l), rA(l), cA(l), cA(l), 0, PA[l][b.t], tA(A.S(l, b.idx)), CR(l, b.t),
              AC(l, b.s), AR(l, b.t));
      if (tcl[l]) tile_out(e.d, ns, RP, KP3, false);
      ns = e.d.segs.size();
      e.gemm1(SBP[p], rB(l), cC(l), cB(l), cB(l), cC(l), cC(l), 0, tB(B.S(l, b.idx)), PB[l][b.s], BR(l, b.t),
              CC(l, b.s), BC(l, b.s));
      if (tcl[l]) tile_out(e.d, ns, NP, KP2, true);
    });
    pb.end("rimage", l);

    // ---- couplings (Eq. leafcoup_simple / nonleafcoup_simple), summed per target in
    // one segment: case-1 (leaf: (V^C^T F)(F V^C)), case-2/4 (Ahat SBP), case-3 (PAS Bhat);
    // above the leaf level case-1 (E^C^T (M E^C)) is a separate first pass
    // the items of each target: case-1 first, then its triples in order.  The triples
    // are grouped by target (a stable counting sort); the targets' segments and items are
    // then written in parallel, in the order one gemm call per target would give
    const size_t ntg = lt.tg.size();
    auto counted = [&](const Triple& tr) {
      const Block &ba = bl[tr.pa], &bb = bl[tr.pb];
      if (lt.tg[tr.tgt].cls == TC_F) return false;
      if (ba.kind == KNL && bb.kind == KNL) return false;
      if (ba.kind == KF && bb.kind == KF) return false;  // case-1 (leaf), above
      return true;
    };
    // (per row cluster in parallel: the triples of row i only name targets of row i)
    const int64_t nrow = (int64_t)lt.first.size() - 1;
    std::vector<int64_t> toff(ntg + 1, 0);  // counted triples per target
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < nrow; ++i)
      for (int64_t x = lt.tfirst[i]; x < lt.tfirst[i + 1]; ++x)
        if (counted(lt.trip[x])) ++toff[lt.trip[x].tgt + 1];
    for (size_t q = 0; q < ntg; ++q) toff[q + 1] += toff[q];
    std::vector<int32_t> tord((size_t)toff[ntg]);
    {
      std::vector<int64_t> cur(toff.begin(), toff.end() - 1);
#pragma omp parallel for schedule(dynamic, 256)
      for (int64_t i = 0; i < nrow; ++i)
        for (int64_t x = lt.tfirst[i]; x < lt.tfirst[i + 1]; ++x)
          if (counted(lt.trip[x])) tord[cur[lt.trip[x].tgt]++] = (int32_t)x;
    }
    const int kmax = std::max(std::max(leaf ? LS : 0, rB(l)), cA(l));
    if (!leaf) {
      pb.begin();
      pb.par((int64_t)lt.tg.size(), [&](int64_t q, auto& e) {
        const Target& T = lt.tg[q];
        if (Mt[q] >= 0) {  // (k over the children of i, each bounded by its rank)
          const int hr = rC(c);
          std::vector<Item> it;
          for (int a = 0; a < 2; ++a)
            it.push_back(Item(tCb(C.Er(l, T.i) + (int64_t)a * hr * rC(l)), Mt[q] + (int64_t)a * hr * cC(l),
                              CR(c, 2 * T.i + a)));
          e.gemm(T.ssum, rC(l), cC(l), hr, rC(l), cC(l), cC(l), SF_TA | SF_CA | SF_ACC, it, CR(l, T.i), CC(l, T.k));
        }
      });
      pb.end("coup", l);
    }
    if (tcl[l]) {
      // ---- the tensor-core pass (tc.cu): the targets in sibling pairs, each pair's terms
      // merged by B tile into steps (TcGroup / TcStep)
      const int cm = rC(l), cn = cC(l);
      auto has_terms = [&](int64_t q) {
        return lt.tg[q].cls != TC_F && ((leaf ? (int64_t)lt.g1.size(q) : 0) + (toff[q + 1] - toff[q])) > 0;
      };
      // a target's terms (case 1, cases 2/4, case 3) as operand tiles, ordered by B tile
      auto terms = [&](int64_t q, std::vector<Item>& out) {
        out.clear();
        if (q < 0) return;
        if (leaf)
          for (size_t x = 0; x < lt.g1.size(q); ++x) {
            const Item& g1 = lt.g1.ptr(q)[x];
            out.push_back(Item(Ach[g1.a], Bch[g1.b], -1, 0, 0, KP1));
          }
        for (int64_t y = toff[q]; y < toff[q + 1]; ++y) {
          const Triple& tr = lt.trip[tord[y]];
          const Block &ba = bl[tr.pa], &bb = bl[tr.pb];
          if (bb.kind == KR) out.push_back(Item(Ahat[l][tr.pa], SBP[tr.pb], BR(l, ba.s), 0, 0, KP2));
          else out.push_back(Item(PAS[tr.pa], Bhat[l][tr.pb], AC(l, ba.s), 0, 0, KP3));
        }
        std::sort(out.begin(), out.end(), [](const Item& x, const Item& y) { return x.b < y.b; });
      };
      // groups: a target of an even row cluster with the target of the next cluster and
      // the same column cluster, if that one has terms; an odd-row target alone otherwise
      // (the targets of row cluster i are [first[i], first[i + 1]), in target order)
      const std::vector<std::array<int32_t, 2>> grp = ordered_collect<std::array<int32_t, 2>>(
          nrow, [&](int64_t i, std::vector<std::array<int32_t, 2>>& out) {
            for (int64_t q = lt.first[i]; q < lt.first[i + 1]; ++q) {
              if (!has_terms(q)) continue;
              const Target& T = lt.tg[q];
              const int32_t sib = lt.find(T.i ^ 1, T.k);
              const bool paired = sib >= 0 && has_terms(sib);
              if (!(T.i & 1)) out.push_back({(int32_t)q, paired ? sib : -1});
              else if (!paired) out.push_back({-1, (int32_t)q});
            }
          });
      const int64_t ng = (int64_t)grp.size();
      // the union of the two targets' B tiles, in order, one step per B tile
      auto merge = [&](const std::vector<Item>& t0, const std::vector<Item>& t1, PlanArray<TcStep>& out) {
        size_t i0 = 0, i1 = 0;
        int64_t n = 0;
        while (i0 < t0.size() || i1 < t1.size()) {
          const bool take0 = i0 < t0.size() && (i1 >= t1.size() || t0[i0].b <= t1[i1].b);
          const bool take1 = i1 < t1.size() && (i0 >= t0.size() || t1[i1].b <= t0[i0].b);
          const Item& x = take0 ? t0[i0] : t1[i1];
          TcStep st;
          st.a[0] = take0 ? t0[i0].a : -1;
          st.a[1] = take1 ? t1[i1].a : -1;
          st.b = x.b;
          st.kref = x.kref;
          st.kpad = x.kpad;
          st.pad0 = 0;
          out.push_back(st);
          ++n;
          if (take0) ++i0;
          if (take1) ++i1;
        }
        return n;
      };
      const size_t gr0 = P.tgroups.size();
      const int64_t fl = pb.tc_par(ng, [&](int64_t gq, PlanArray<TcStep>& steps, int64_t& flg) {
        thread_local std::vector<Item> t0, t1;
        terms(grp[gq][0], t0);
        terms(grp[gq][1], t1);
        const size_t f0 = steps.size();
        const int64_t n = merge(t0, t1, steps);
        TcGroup G{};
        for (int sl = 0; sl < 2; ++sl) {
          const int32_t q = grp[gq][sl];
          G.out[sl] = q >= 0 ? lt.tg[q].ssum : -1;
          G.mref[sl] = q >= 0 ? CR(l, lt.tg[q].i) : -1;
          // the first contribution is stored, unless the case-1 pass above has written
          if (q >= 0 && Mt[q] >= 0) G.acc |= (uint8_t)(1u << sl);
        }
        G.nref = CC(l, lt.tg[grp[gq][0] >= 0 ? grp[gq][0] : grp[gq][1]].k);
        G.first = (int32_t)f0;
        G.count = (int32_t)n;
        G.m = (int16_t)cm;
        G.n = (int16_t)cn;
        G.ldc = (int16_t)cn;
        for (size_t x = f0; x < steps.size(); ++x)
          flg += 2LL * cm * cn * steps[x].kpad * ((steps[x].a[0] >= 0) + (steps[x].a[1] >= 0));
        return G;
      });
      P.flops += fl;
      if (ng > 0) {
        Launch Lc;
        Lc.kind = Launch::GEMM;
        Lc.tc = true;
        Lc.first = (int64_t)gr0;
        Lc.count = ng;
        Lc.level = l;
        Lc.phase = "coup";
        Lc.aux = NP;   // B tile rows (the MMA's N)
        Lc.aux2 = RP;  // A tile rows
        Lc.aux3 = std::max(std::max(leaf ? KP1 : 0, KP2), KP3);
        Lc.flops = (double)fl;
        P.launches.push_back(Lc);
      }
    } else {
      pb.begin();
      const int cm = rC(l), cn = cC(l);
      // a segment per target with items (gemm's rules: no segment for empty sums)
      std::vector<int64_t> sidx(ntg + 1, 0), ioff(ntg + 1, 0);
      for (size_t q = 0; q < ntg; ++q) {
        const int64_t cnt = lt.tg[q].cls == TC_F ? 0 : (leaf ? (int64_t)lt.g1.size(q) : 0) + (toff[q + 1] - toff[q]);
        const bool emit = cnt > 0 && cm > 0 && cn > 0 && kmax > 0;
        sidx[q + 1] = sidx[q] + (emit ? 1 : 0);
        ioff[q + 1] = ioff[q] + (emit ? cnt : 0);
      }
      const size_t s0 = P.segs.size(), i0 = P.items.size();
      if ((int64_t)i0 + ioff[ntg] > INT32_MAX) throw Error(H2_ENOMEM, "plan too large");
      P.segs.resize(s0 + (size_t)sidx[ntg]);
      P.items.resize(i0 + (size_t)ioff[ntg]);
      int64_t fl = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : fl)
      for (int64_t q = 0; q < (int64_t)ntg; ++q) {
        if (sidx[q + 1] == sidx[q]) continue;
        const Target& T = lt.tg[q];
        Item* it = P.items.data() + i0 + ioff[q];
        int64_t n = 0;
        if (leaf)
          for (size_t x = 0; x < lt.g1.size(q); ++x) {
            const Item& g = lt.g1.ptr(q)[x];
            it[n++] = Item(Ach[g.a], Bch[g.b], -1, LS, cn, LS);
          }
        for (int64_t y = toff[q]; y < toff[q + 1]; ++y) {
          const Triple& tr = lt.trip[tord[y]];
          const Block &ba = bl[tr.pa], &bb = bl[tr.pb];
          if (bb.kind == KR)  // case-2, case-4
            it[n++] = Item(Ahat[l][tr.pa], SBP[tr.pb], BR(l, ba.s), rB(l), cn, rB(l));
          else  // case-3
            it[n++] = Item(PAS[tr.pa], Bhat[l][tr.pb], AC(l, ba.s), cA(l), cn, cA(l));
        }
        Seg sg{};
        sg.out = T.ssum;
        sg.first = (int32_t)(i0 + ioff[q]);
        sg.count = (int32_t)n;
        sg.m = (int16_t)cm;
        sg.n = (int16_t)cn;
        sg.k = (int16_t)kmax;
        sg.lda = (int16_t)kmax;
        sg.ldb = (int16_t)cn;
        sg.ldc = (int16_t)cn;
        sg.mref = CR(l, T.i);
        sg.nref = CC(l, T.k);
        // the first contribution to the target's coupling is stored, not added, unless the
        // case-1 pass above the leaf level has written it already
        sg.flags = Mt[q] >= 0 ? SF_ACC : 0;
        P.segs[s0 + sidx[q]] = sg;
        for (int64_t x = 0; x < n; ++x) fl += 2LL * cm * cn * (it[x].kpad ? it[x].kpad : kmax);
      }
      P.flops += fl;
      pb.end("coup", l);
    }
    pb.close_memset(zG, g);
    pb.close_memset(zS, AR_S);
    // the children's data of this level are consumed: free the lists
    if (c <= L) {
      Ahat[c].clear();
      Bhat[c].clear();
      PA[c].clear();
      PB[c].clear();
      Bj[c].clear();
    }
  }

  // ============================================ top-down split of NL-held couplings
  std::vector<std::vector<int64_t>> H(L + 1);
  for (int l = lmin; l < L; ++l) {
    H[l].assign(st.blocks[l].size(), -1);
    for (auto& T : LT[l].tg)
      if (T.cls == TC_NL) H[l][T.cpos] = T.ssum;
  }
  for (int l = lmin; l < L; ++l) {
    const int c = l + 1;
    const auto& bl = st.blocks[l];
    const int hr = rC(c), hc = cC(c);
    pb.reset(AR_S);
    const size_t zS = pb.open_memset(AR_S);
    std::vector<int64_t> Xt(bl.size(), -1), X(bl.size(), -1);
    for (size_t p = 0; p < bl.size(); ++p)
      if (bl[p].kind == KNL && H[l][p] >= 0) {
        Xt[p] = pb.alloc(AR_S, (int64_t)rC(l) * 2 * hc);
        X[p] = pb.alloc(AR_S, (int64_t)2 * hr * 2 * hc);
      }
    if (c < L)
      for (size_t p = 0; p < st.blocks[c].size(); ++p)
        if (st.blocks[c][p].kind == KNL && H[c][p] < 0) {
          int32_t pp = st.find(l, st.blocks[c][p].t >> 1, st.blocks[c][p].s >> 1);
          if (pp >= 0 && X[pp] >= 0) H[c][p] = pb.alloc(AR_P, (int64_t)rC(c) * cC(c));
        }
    // (the children's halves of Xt and X, each bounded by the children's ranks)
    const int64_t nbl = (int64_t)bl.size();
    pb.begin();
    pb.par(nbl, [&](int64_t p, auto& e) {
      if (Xt[p] >= 0)
        for (int b = 0; b < 2; ++b)
          e.gemm1(Xt[p] + (int64_t)b * hc, rC(l), hc, cC(l), cC(l), cC(l), 2 * hc, SF_TB, H[l][p],
                  tCb(C.Ec(l, bl[p].s) + (int64_t)b * hc * cC(l)), CR(l, bl[p].t), CC(c, 2 * bl[p].s + b),
                  CC(l, bl[p].s));
    });
    pb.end("split", l);
    pb.begin();
    pb.par(nbl, [&](int64_t p, auto& e) {
      if (X[p] >= 0)
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b)
            e.gemm1(X[p] + (int64_t)a * hr * 2 * hc + (int64_t)b * hc, hr, hc, rC(l), rC(l), 2 * hc, 2 * hc, 0,
                    tCb(C.Er(l, bl[p].t) + (int64_t)a * hr * rC(l)), Xt[p] + (int64_t)b * hc, CR(c, 2 * bl[p].t + a),
                    CC(c, 2 * bl[p].s + b), CR(l, bl[p].t));
    });
    pb.end("split", l);
    std::vector<std::pair<int64_t, int64_t>> Fupd;
    std::vector<int32_t> Frow;
    // the children's parts of X: added to R children's couplings and to NL children's
    // held ones (plain sums, one launch); F children's parts go through X E^C (a second
    // launch) into F += V^C (X E^C) (a third)
    std::vector<std::pair<int64_t, int32_t>> fpart;  // (part of X, child block)
    pb.begin();
    {
      // (the F children's parts collected per block, then listed in block order)
      std::vector<std::array<std::pair<int64_t, int32_t>, 4>> fp((size_t)nbl);
      std::vector<int8_t> nfp((size_t)nbl, 0);
      pb.par(nbl, [&](int64_t p, auto& e) {
        if (X[p] < 0) return;
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) {
            int32_t cp = st.find(c, 2 * bl[p].t + a, 2 * bl[p].s + bb);
            const Block& cb = st.blocks[c][cp];
            int64_t xab = X[p] + (int64_t)a * hr * 2 * hc + (int64_t)bb * hc;
            if (cb.kind == KR) e.sum(tC(C.S(c, cb.idx)), hr, hc, 2 * hc, cC(c), true, {xab});
            else if (cb.kind == KNL) e.sum(H[c][cp], hr, hc, 2 * hc, cC(c), true, {xab});
            else fp[p][nfp[p]++] = {xab, cp};
          }
      });
      for (int64_t p = 0; p < nbl; ++p)
        for (int x = 0; x < nfp[p]; ++x) fpart.push_back(fp[p][x]);
    }
    pb.end("split", l);
    pb.begin();
    for (const auto& f : fpart) {
      const Block& cb = st.blocks[c][f.second];
      int64_t tmp = pb.alloc(AR_S, (int64_t)rC(c) * LS);
      pb.gemm1(tmp, rC(c), LS, cC(c), 2 * hc, cC(c), LS, SF_TB, f.first, tCb(C.Vc(cb.s)), CR(c, cb.t), -1,
               CC(c, cb.s));
      Fupd.push_back({tmp, tC(C.F(cb.idx))});
      Frow.push_back(cb.t);
    }
    pb.end("split", l);
    pb.begin();
    pb.par((int64_t)Fupd.size(), [&](int64_t q, auto& e) {
      e.gemm1(Fupd[q].second, LS, LS, rC(c), rC(c), LS, LS, SF_ACC, tCb(C.Vr(Frow[q])), Fupd[q].first, -1, -1,
              CR(c, Frow[q]));
    });
    pb.end("split", c);
    pb.close_memset(zS, AR_S);
  }
  pb.close_memset(zP, AR_P);
}

void build_matvec_plan(const Mat& H, int64_t nrhs, Plan& P, int64_t& off_x, int64_t& off_y) {
  const Structure& st = *H.st;
  const int L = st.L, LS = st.LS;
  PlanBuilder pb(P);
  P.cplx = H.cplx;
  const int64_t nl = 1LL << L;
  const int nr = (int)nrhs;
  const Arena W = AR_P;
  off_x = pb.alloc(W, nl * LS * nrhs);
  off_y = pb.alloc(W, nl * LS * nrhs);
  std::vector<int64_t> xh(L + 1), yh(L + 1);
  for (int l = 0; l <= L; ++l) {
    xh[l] = pb.alloc(W, (1LL << l) * H.Kc[l] * nrhs);
    yh[l] = pb.alloc(W, (1LL << l) * H.Kr[l] * nrhs);
  }
  auto tH = [&](int64_t o) { return tag(AR_A, o); };
  // forward transform
  pb.begin();
  for (int64_t t = 0; t < nl; ++t)
    pb.gemm1(xh[L] + t * H.Kc[L] * nrhs, H.Kc[L], nr, LS, H.Kc[L], nr, nr, SF_TA, tH(H.Vc(t)), off_x + t * LS * nrhs);
  pb.end("mv_forward", L);
  for (int l = L - 1; l >= 0; --l) {
    pb.begin();
    for (int64_t t = 0; t < (1LL << l); ++t)
      pb.gemm1(xh[l] + t * H.Kc[l] * nrhs, H.Kc[l], nr, 2 * H.Kc[l + 1], H.Kc[l], nr, nr, SF_TA, tH(H.Ec(l, t)),
               xh[l + 1] + 2 * t * H.Kc[l + 1] * nrhs);
    pb.end("mv_forward", l);
  }
  // coupling and near field
  pb.begin();
  for (int l = 0; l <= L; ++l) {
    const auto& bl = st.blocks[l];
    for (int64_t t = 0; t < (1LL << l); ++t) {
      std::vector<Item> cr, fr;
      for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p) {
        const Block& b = bl[p];
        if (b.kind == KR) cr.push_back({tH(H.S(l, b.idx)), xh[l] + b.s * H.Kc[l] * nrhs});
        if (b.kind == KF) fr.push_back({tH(H.F(b.idx)), off_x + b.s * LS * nrhs});
      }
      pb.gemm(yh[l] + t * H.Kr[l] * nrhs, H.Kr[l], nr, H.Kc[l], H.Kc[l], nr, nr, 0, cr);
      pb.gemm(off_y + t * LS * nrhs, LS, nr, LS, LS, nr, nr, 0, fr);
    }
  }
  pb.end("mv_coupling", -1);
  // backward transform
  for (int l = 0; l < L; ++l) {
    pb.begin();
    for (int64_t t = 0; t < (1LL << l); ++t)
      pb.gemm1(yh[l + 1] + 2 * t * H.Kr[l + 1] * nrhs, 2 * H.Kr[l + 1], nr, H.Kr[l], H.Kr[l], nr, nr, SF_ACC,
               tH(H.Er(l, t)), yh[l] + t * H.Kr[l] * nrhs);
    pb.end("mv_backward", l);
  }
  pb.begin();
  for (int64_t t = 0; t < nl; ++t)
    pb.gemm1(off_y + t * LS * nrhs, LS, nr, H.Kr[L], H.Kr[L], nr, nr, SF_ACC, tH(H.Vr(t)), yh[L] + t * H.Kr[L] * nrhs);
  pb.end("mv_backward", L);
}

}  // namespace h2
