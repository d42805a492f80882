// C ABI of the H^2 library: handle lifetime, device memory, plan execution.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "internal.hpp"

// Product plans are cached process-wide by (structure, caps of A and B, options):
// handles on equal points share one structure and, with equal caps, one plan and
// its work regions.  Products that share a plan must run in stream order.
struct PlanKey {
  const h2::Structure* st;
  std::vector<int> akr, akc, bkr, bkc;
  int trunc, cap, precision;
  bool cplx;
  bool operator==(const PlanKey& o) const {
    return st == o.st && akr == o.akr && akc == o.akc && bkr == o.bkr && bkc == o.bkc && trunc == o.trunc &&
           cap == o.cap && precision == o.precision && cplx == o.cplx;
  }
};
// Autotuning state of a program (h2_opts.autotune): for every GEMM launch group the
// launch configuration in use (-1: still exploring) and the device time measured for
// each candidate.  Product p of the exploration runs candidate p mod ncand on every
// undecided group with events around each GEMM launch; the next tuned product reads
// the times (they are complete by then: it synchronises on the last event) and a group
// whose candidates are all measured keeps its fastest.  The candidates leave every
// result bit-identical, so tuning changes only the time.
struct TuneState {
  std::mutex mu;
  int ncand = 0;
  int explored = 0;
  bool pending = false;
  std::vector<int8_t> choice;
  std::vector<std::vector<float>> ms;
  std::vector<void*> ev;
  ~TuneState() {
    for (void* e : ev) cudaEventDestroy((cudaEvent_t)e);
  }
};
struct PlanEntry {
  h2::Plan plan;
  TuneState tune;
  ~PlanEntry() { h2::free_plan(plan); }
};

struct h2_matrix {
  h2::Mat m;
  std::vector<std::shared_ptr<PlanEntry>> plans_held;  // plans of products made from this handle
  std::map<int64_t, std::unique_ptr<h2::Plan>> mv_plans;  // by nrhs
  std::map<int64_t, std::pair<int64_t, int64_t>> mv_offs;
  int64_t* d_user = nullptr;  // padded tree row -> user index (-1: padding)
  // device arena tables the kernels read: slot 0 for the product written into this
  // handle, slot 1 for its matvec (stream-ordered uploads; concurrent use of one handle
  // on two streams is not supported)
  h2::Arenas* d_ars = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  int origin_trunc = -1, origin_cap = -1, origin_prec = -1;
  bool trace_on = false;     // on A: trace the products made from it
  h2::Trace trace;           // on C: events of the product that made it
  const h2::Plan* trace_plan = nullptr;
  std::shared_ptr<PlanEntry> made_by;  // on C: the plan of the product that made it
  const h2_matrix* origin_A = nullptr;
  const h2_matrix* origin_B = nullptr;
  // frees everything the handle owns (also for a handle whose making failed halfway)
  ~h2_matrix() {
    for (void* e : trace.ev) cudaEventDestroy((cudaEvent_t)e);
    for (auto& kv : mv_plans) h2::free_plan(*kv.second);
    if (d_user) cudaFree(d_user);
    if (d_ars) cudaFree(d_ars);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    h2::free_mat(m);
  }
};

namespace {
thread_local std::string g_err;
std::mutex g_cache_mu;
std::vector<std::pair<PlanKey, std::weak_ptr<PlanEntry>>> g_plans;
struct StructKey {
  uint64_t hash;
  int64_t n;
  int leaf;
  double eta;
};
std::vector<std::pair<StructKey, std::weak_ptr<h2::Structure>>> g_structs;

uint64_t fnv1a(const void* p, size_t bytes) {
  const unsigned char* b = (const unsigned char*)p;
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < bytes; ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

// the structure of (points, leaf, eta), shared with live handles on equal points
std::shared_ptr<h2::Structure> structure_for(const double* pts, int64_t n, int leaf, double eta) {
  if (!pts || n < 1) return h2::build_structure(pts, n, leaf, eta);
  StructKey key{fnv1a(pts, (size_t)n * 3 * sizeof(double)), n, leaf, eta};
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto it = g_structs.begin(); it != g_structs.end();) {
    auto sp = it->second.lock();
    if (!sp) {
      it = g_structs.erase(it);
      continue;
    }
    const StructKey& k = it->first;
    if (k.hash == key.hash && k.n == n && k.leaf == leaf && k.eta == eta) {
      bool same = true;
      for (int64_t p = 0; p < n && same; ++p)
        for (int d = 0; d < 3; ++d)
          if (sp->pts[3 * p + d] != pts[3 * sp->perm[p] + d]) {
            same = false;
            break;
          }
      if (same) return sp;
    }
    ++it;
  }
  auto st = h2::build_structure(pts, n, leaf, eta);
  g_structs.push_back({key, st});
  return st;
}

h2_status fail(h2_status c, const std::string& m) {
  g_err = m;
  return c;
}

template <class F>
h2_status guarded(F&& f) {
  try {
    f();
    return H2_OK;
  } catch (const h2::Error& e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc&) {
    return fail(H2_ENOMEM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(H2_EINTERNAL, e.what());
  }
}

// failure injection for tests: >= 0 = device allocations still allowed, -1 = no limit
static std::atomic<int64_t> g_alloc_left{-1};

void* dmalloc(size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 256;
  int64_t left = g_alloc_left.load();
  while (left > 0 && !g_alloc_left.compare_exchange_weak(left, left - 1)) {
  }
  if (left == 0)
    throw h2::Error(H2_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes refused (allocation limit)");
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw h2::Error(H2_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  return p;
}

h2_opts defaults(const h2_opts* o) {
  h2_opts d{};
  d.precision = H2_FP64;
  d.trunc = H2_TRUNC_PAPER;
  d.rank_cap = 48;
  d.stream = nullptr;
  if (o) {
    d = *o;
    if (d.rank_cap <= 0) d.rank_cap = 48;
  }
  if (d.precision < H2_FP64 || d.precision > H2_MIXED_BF16X3) throw h2::Error(H2_EINVAL, "bad precision");
  if (d.norm != H2_NORM_FROBENIUS && d.norm != H2_NORM_SPECTRAL) throw h2::Error(H2_EINVAL, "bad norm");
  if (d.autotune != 0 && d.autotune != 1) throw h2::Error(H2_EINVAL, "autotune must be 0 or 1");
  if (d.reserved != 0) throw h2::Error(H2_EINVAL, "h2_opts.reserved must be 0");
  if (d.trunc < 0 || d.trunc > 3) throw h2::Error(H2_EINVAL, "bad truncation mode");
  if (d.rank_cap > 128) throw h2::Error(H2_EINVAL, "rank_cap above 128");
  return d;
}

int64_t round32(int64_t x) { return (x + 31) & ~int64_t(31); }

void make_user_map(h2_matrix* h) {
  const h2::Structure& st = *h->m.st;
  int64_t nl = 1LL << st.L, rows = nl * st.LS;
  std::vector<int64_t> user(rows, -1);
  for (int64_t t = 0; t < nl; ++t)
    for (int64_t r = 0; r < st.size[st.L][t]; ++r) user[t * st.LS + r] = st.perm[st.start[st.L][t] + r];
  h->d_user = (int64_t*)dmalloc(rows * sizeof(int64_t));
  h2::cuda_check(cudaMemcpy(h->d_user, user.data(), rows * sizeof(int64_t), cudaMemcpyHostToDevice), "upload user map");
}

}  // namespace

namespace h2 {

void* dev_alloc(size_t bytes) { return dmalloc(bytes); }

void cuda_check(int err, const char* what) {
  if (err != cudaSuccess) {
    cudaGetLastError();
    throw Error(H2_ECUDA, std::string(what) + ": " + cudaGetErrorString((cudaError_t)err));
  }
}

int64_t mat_elems(Mat& m) {
  const Structure& st = *m.st;
  const int L = st.L;
  const int64_t nl = 1LL << L, LS = st.LS;
  int64_t o = 0;
  m.off_Vr = o;
  o += round32(nl * LS * m.Kr[L]);
  m.off_Vc = o;
  o += round32(nl * LS * m.Kc[L]);
  m.off_Er.assign(L, 0);
  m.off_Ec.assign(L, 0);
  for (int l = 0; l < L; ++l) {
    m.off_Er[l] = o;
    o += round32((1LL << l) * 2LL * m.Kr[l + 1] * m.Kr[l]);
    m.off_Ec[l] = o;
    o += round32((1LL << l) * 2LL * m.Kc[l + 1] * m.Kc[l]);
  }
  m.off_S.assign(L + 1, 0);
  for (int l = 0; l <= L; ++l) {
    m.off_S[l] = o;
    o += round32(st.nR[l] * (int64_t)m.Kr[l] * m.Kc[l]);
  }
  m.off_F = o;
  o += round32(st.nF * LS * LS);
  m.arena_elems = o;
  return o;
}

void alloc_mat(Mat& m) {
  const Structure& st = *m.st;
  int64_t o = mat_elems(m);
  m.arena = (double*)dmalloc(o * m.esize());
  cuda_check(cudaMemset(m.arena, 0, o * m.esize()), "zero arena");
  const int nn = st.nnodes();
  m.d_kr = (int32_t*)dmalloc(2 * nn * sizeof(int32_t) + 64);
  m.d_kc = m.d_kr + nn;
  cuda_check(cudaMemset(m.d_kr, 0, 2 * nn * sizeof(int32_t) + 64), "zero ranks");
  m.d_cap = (unsigned long long*)((char*)m.d_kr + ((2 * nn * sizeof(int32_t) + 15) & ~size_t(15)));
}

void free_mat(Mat& m) {
  if (m.arena) cudaFree(m.arena);
  if (m.arena32) cudaFree(m.arena32);
  if (m.bases32) cudaFree(m.bases32);
  m.arena32 = m.bases32 = nullptr;
  if (m.d_kr) cudaFree(m.d_kr);
  for (void* p : m.extra_allocs) cudaFree(p);
  m.arena = nullptr;
  m.d_kr = m.d_kc = nullptr;
  m.extra_allocs.clear();
}

void sync_ranks_to_host(Mat& m) {
  if (m.ranks_on_host) return;
  const int nn = m.st->nnodes();
  m.h_kr.resize(nn);
  m.h_kc.resize(nn);
  cuda_check(cudaStreamSynchronize((cudaStream_t)m.stream), "synchronise");
  cuda_check(cudaMemcpy(m.h_kr.data(), m.d_kr, nn * sizeof(int32_t), cudaMemcpyDeviceToHost), "ranks");
  cuda_check(cudaMemcpy(m.h_kc.data(), m.d_kc, nn * sizeof(int32_t), cudaMemcpyDeviceToHost), "ranks");
  m.ranks_on_host = true;
}

// Large copies between caller memory (pageable, e.g. numpy arrays) and the device:
// the range is page-locked for the copy so that it goes by DMA, then released; if it
// cannot be registered (already registered, or refused) the plain copy is used.
static void copy_host(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind, const char* what) {
  void* host = (void*)(kind == cudaMemcpyHostToDevice ? src : dst);
  bool reg = false;
  if (bytes >= ((size_t)64 << 20)) {
    reg = cudaHostRegister(host, bytes, cudaHostRegisterDefault) == cudaSuccess;
    if (!reg) cudaGetLastError();
  }
  cudaError_t e = cudaMemcpy(dst, src, bytes, kind);
  if (reg) cudaHostUnregister(host);
  cuda_check(e, what);
}

// Blocks of the packed layout (vr, vc, er, ec, s, f back to back, each block dense at
// the actual ranks) and where they sit in the padded arena; len gets the six lengths.
std::vector<CopyTask> copy_tasks(const Mat& m, const int32_t* kr, const int32_t* kc, int64_t len[6]) {
  const Structure& st = *m.st;
  const int L = st.L;
  const int64_t LS = st.LS;
  std::vector<CopyTask> tk;
  int64_t off = 0;
  auto add = [&](int64_t arena_off, int64_t rows, int64_t cols, int64_t ld) {
    if (rows > 0 && cols > 0) tk.push_back({arena_off, off, (int32_t)rows, (int32_t)cols, (int32_t)ld, 0});
    off += rows * cols;
  };
  int64_t mark = 0;
  for (int col = 0; col < 2; ++col) {  // leaf bases
    const int32_t* rk = col ? kc : kr;
    const int K = col ? m.Kc[L] : m.Kr[L];
    for (int64_t t = 0; t < (1LL << L); ++t) add(col ? m.Vc(t) : m.Vr(t), st.size[L][t], rk[Structure::node(L, t)], K);
    len[col] = off - mark;
    mark = off;
  }
  for (int col = 0; col < 2; ++col) {  // stacked transfers: child 1 rows, then child 2 rows
    const int32_t* rk = col ? kc : kr;
    const auto& K = col ? m.Kc : m.Kr;
    for (int l = 0; l < L; ++l)
      for (int64_t t = 0; t < (1LL << l); ++t) {
        const int k = rk[Structure::node(l, t)], k1 = rk[Structure::node(l + 1, 2 * t)],
                  k2 = rk[Structure::node(l + 1, 2 * t + 1)];
        const int64_t base = col ? m.Ec(l, t) : m.Er(l, t);
        add(base, k1, k, K[l]);
        add(base + (int64_t)K[l + 1] * K[l], k2, k, K[l]);
      }
    len[2 + col] = off - mark;
    mark = off;
  }
  for (int l = 0; l <= L; ++l)  // couplings
    for (auto& b : st.blocks[l])
      if (b.kind == KR) add(m.S(l, b.idx), kr[Structure::node(l, b.t)], kc[Structure::node(l, b.s)], m.Kc[l]);
  len[4] = off - mark;
  mark = off;
  for (auto& b : st.blocks[L])  // dense leaf blocks
    if (b.kind == KF) add(m.F(b.idx), st.size[L][b.t], st.size[L][b.s], LS);
  len[5] = off - mark;
  return tk;
}

void packed_lengths(const Structure& st, const int32_t* kr, const int32_t* kc, int64_t len[6]) {
  const int L = st.L;
  for (int i = 0; i < 6; ++i) len[i] = 0;
  for (int64_t t = 0; t < (1LL << L); ++t) {
    len[0] += st.size[L][t] * kr[Structure::node(L, t)];
    len[1] += st.size[L][t] * kc[Structure::node(L, t)];
  }
  for (int l = 0; l < L; ++l)
    for (int64_t t = 0; t < (1LL << l); ++t) {
      len[2] += (int64_t)(kr[Structure::node(l + 1, 2 * t)] + kr[Structure::node(l + 1, 2 * t + 1)]) * kr[Structure::node(l, t)];
      len[3] += (int64_t)(kc[Structure::node(l + 1, 2 * t)] + kc[Structure::node(l + 1, 2 * t + 1)]) * kc[Structure::node(l, t)];
    }
  for (int l = 0; l <= L; ++l)
    for (auto& b : st.blocks[l]) {
      if (b.kind == KR) len[4] += (int64_t)kr[Structure::node(l, b.t)] * kc[Structure::node(l, b.s)];
      if (b.kind == KF) len[5] += st.size[L][b.t] * st.size[L][b.s];
    }
}

// the copy tasks of a complex matrix as tasks over doubles (two per element)
static void scale_tasks(std::vector<CopyTask>& tk) {
  for (CopyTask& c : tk) {
    c.arena_off *= 2;
    c.packed_off *= 2;
    c.cols *= 2;
    c.ld *= 2;
  }
}

// packed host arrays -> padded device arena (caps = largest rank per level, rounded up
// to a multiple of four): the arrays are copied as they are into a device staging
// buffer and scattered into the zeroed arena by transfer.cu's kernel
void unpack_view_to_device(const PackedView& v, Mat& m) {
  const Structure& st = *m.st;
  const int L = st.L, nn = st.nnodes();
  m.Kr.assign(L + 1, 0);
  m.Kc.assign(L + 1, 0);
  for (int l = 0; l <= L; ++l)
    for (int64_t t = 0; t < (1LL << l); ++t) {
      int kr = v.kr[Structure::node(l, t)], kc = v.kc[Structure::node(l, t)];
      if (kr < 0 || kc < 0 || kr > st.size[l][t] || kc > st.size[l][t] || kr > 128 || kc > 128)
        throw Error(H2_EINVAL, "rank out of range");
      if (l < L) {
        int64_t lr = (int64_t)v.kr[Structure::node(l + 1, 2 * t)] + v.kr[Structure::node(l + 1, 2 * t + 1)];
        int64_t lc = (int64_t)v.kc[Structure::node(l + 1, 2 * t)] + v.kc[Structure::node(l + 1, 2 * t + 1)];
        if (kr > lr || kc > lc) throw Error(H2_EINVAL, "rank above the sum of the children's ranks");
      }
      m.Kr[l] = std::max(m.Kr[l], kr);
      m.Kc[l] = std::max(m.Kc[l], kc);
    }
  for (int l = 0; l <= L; ++l) {  // storage caps: multiples of four
    m.Kr[l] = cap_round(m.Kr[l]);
    m.Kc[l] = cap_round(m.Kc[l]);
  }
  mat_elems(m);  // the arena layout (offsets) the copy tasks point into
  int64_t len[6];
  std::vector<CopyTask> tk = copy_tasks(m, v.kr, v.kc, len);
  for (int i = 0; i < 6; ++i) {
    if (v.len[i] != len[i]) throw Error(H2_EINVAL, "packed array has the wrong length");
    if (len[i] && !v.arr[i]) throw Error(H2_EINVAL, "null array");
  }
  alloc_mat(m);  // zeroed: padded entries stay exactly zero
  // complex elements are two doubles: the same blocks, twice as wide in doubles
  const int w = m.cplx ? 2 : 1;
  if (w == 2) scale_tasks(tk);
  int64_t total = 0;
  for (int i = 0; i < 6; ++i) total += len[i] * w;
  double* stage = (double*)dmalloc(std::max<int64_t>(1, total) * sizeof(double));
  CopyTask* d_tk = (CopyTask*)dmalloc(std::max<size_t>(1, tk.size()) * sizeof(CopyTask));
  try {
    int64_t off = 0;
    for (int i = 0; i < 6; ++i) {
      if (len[i])
        copy_host(stage + off, v.arr[i], len[i] * w * sizeof(double), cudaMemcpyHostToDevice, "upload arrays");
      off += len[i] * w;
    }
    if (!tk.empty())
      cuda_check(cudaMemcpy(d_tk, tk.data(), tk.size() * sizeof(CopyTask), cudaMemcpyHostToDevice), "upload tasks");
    launch_copy_tasks(d_tk, (int64_t)tk.size(), stage, m.arena, true, nullptr);
    cuda_check(cudaGetLastError(), "scatter");
    cuda_check(cudaDeviceSynchronize(), "scatter");
  } catch (...) {
    cudaFree(stage);
    cudaFree(d_tk);
    throw;
  }
  cudaFree(stage);
  cudaFree(d_tk);
  cuda_check(cudaMemcpy(m.d_kr, v.kr, nn * sizeof(int32_t), cudaMemcpyHostToDevice), "upload ranks");
  cuda_check(cudaMemcpy(m.d_kc, v.kc, nn * sizeof(int32_t), cudaMemcpyHostToDevice), "upload ranks");
  m.h_kr.assign(v.kr, v.kr + nn);
  m.h_kc.assign(v.kc, v.kc + nn);
  m.ranks_on_host = true;
}

// padded device arena -> the packed arrays (gathered on the device into a staging
// buffer, then one copy per requested array into the caller's memory)
void pack_to_host(Mat& m, double* const out[6]) {
  sync_ranks_to_host(m);
  int64_t len[6];
  std::vector<CopyTask> tk = copy_tasks(m, m.h_kr.data(), m.h_kc.data(), len);
  const int w = m.cplx ? 2 : 1;
  if (w == 2) scale_tasks(tk);
  int64_t total = 0;
  for (int i = 0; i < 6; ++i) total += len[i] * w;
  double* stage = (double*)dmalloc(std::max<int64_t>(1, total) * sizeof(double));
  CopyTask* d_tk = (CopyTask*)dmalloc(std::max<size_t>(1, tk.size()) * sizeof(CopyTask));
  try {
    if (!tk.empty())
      cuda_check(cudaMemcpy(d_tk, tk.data(), tk.size() * sizeof(CopyTask), cudaMemcpyHostToDevice), "upload tasks");
    launch_copy_tasks(d_tk, (int64_t)tk.size(), stage, m.arena, false, nullptr);
    cuda_check(cudaGetLastError(), "gather");
    cuda_check(cudaDeviceSynchronize(), "gather");
    int64_t off = 0;
    for (int i = 0; i < 6; ++i) {
      if (len[i] && out[i])
        copy_host(out[i], stage + off, len[i] * w * sizeof(double), cudaMemcpyDeviceToHost, "download arrays");
      off += len[i] * w;
    }
  } catch (...) {
    cudaFree(stage);
    cudaFree(d_tk);
    throw;
  }
  cudaFree(stage);
  cudaFree(d_tk);
}

// Host-side check that every access of a plan stays inside its arena: run before a
// plan's first upload so that an indexing error is reported instead of executed.
void validate_plan(const Plan& P, const int64_t sizes[kArenas]) {
  // live allocations of the work regions, replayed in program order; a region is
  // bump-allocated between resets, so its live list stays sorted by start
  std::vector<std::pair<int64_t, int64_t>> live[kArenas];
  // lookup table of each region: entry b = the last live allocation starting at or
  // before offset b * kBucket (-1: none), extended as allocations are appended (their
  // starts increase) and cleared with the region
  constexpr int64_t kBucket = 512;
  std::vector<int32_t> bucket[kArenas];
  size_t done[kArenas] = {};
  size_t ev = 0;
  auto is_work = [](int64_t a) { return a == AR_P || a == AR_G0 || a == AR_G1 || a == AR_S; };
  auto check = [&](int64_t tagged, int64_t extent, const char* what) {
    if (extent <= 0) return;
    int64_t a = arena_of(tagged), off = offset_of(tagged);
    if (tagged < 0 || off + extent > sizes[a])
      throw Error(H2_EINTERNAL, std::string("plan access out of bounds: ") + what);
    if (!is_work(a)) return;
    // the last allocation starting at or before off: from the table's entry for off's
    // bucket, forward over the allocations that start inside the bucket
    const auto& v = live[a];
    const auto& bt = bucket[a];
    const size_t b = (size_t)(off / kBucket);
    int64_t h = bt.empty() ? -1 : bt[std::min(b, bt.size() - 1)];
    while (h + 1 < (int64_t)v.size() && v[(size_t)h + 1].first <= off) ++h;
    if (h < 0 || v[(size_t)h].first + v[(size_t)h].second < off + extent)
      throw Error(H2_EINTERNAL, std::string("plan access outside its allocation: ") + what);
  };
  // an operand tile of tr rows and kp columns holding an m x n matrix (transposed: n x m)
  auto check_tile = [&](int64_t tagged, int tr, int kp, int m, int n, bool tt, const char* what) {
    if (tr <= 0 || tr % 8 || kp <= 0 || kp % 16) throw Error(H2_EINTERNAL, std::string("bad tile shape: ") + what);
    if ((tt ? n : m) > tr || (tt ? m : n) > kp)
      throw Error(H2_EINTERNAL, std::string("matrix larger than its tile: ") + what);
    check(tagged, (int64_t)tr * kp, what);
  };
  auto check_seg = [&](const Seg& s) {
    bool ta = s.flags & SF_TA, tb = s.flags & SF_TB;
    const bool tile = s.flags & SF_TILE, tt = s.flags & SF_TILE_T;
    if ((s.flags2 & SF2_SYM) && (s.m != s.n || s.mref != s.nref || (s.flags & (SF_SUM | SF_TILE))))
      throw Error(H2_EINTERNAL, "symmetric block that is not square");
    if (tile && !(s.flags & SF_SUM)) {
      if (s.flags & SF_ACC) throw Error(H2_EINTERNAL, "tile outputs are written, not accumulated");
      check_tile(s.out, s.trows, s.ldc, s.m, s.n, tt, "tile output");
    } else {
      check(s.out, (int64_t)(s.m - 1) * s.ldc + s.n, "segment output");
      if (s.ldc < s.n) throw Error(H2_EINTERNAL, "segment ldc < n");
    }
    for (int32_t q = s.first; q < s.first + s.count; ++q) {
      const Item& it = P.items[q];
      if (s.flags & SF_SUM) {
        if (tile) {
          check_tile(it.a, s.trows, s.lda, s.m, s.n, tt, "tile sum input");
          continue;
        }
        if (ta) {  // a transposed input (n x m)
          if (s.lda < s.m) throw Error(H2_EINTERNAL, "sum lda < m");
          check(it.a, (int64_t)(s.n - 1) * s.lda + s.m, "sum input");
          continue;
        }
        if (s.lda < s.n) throw Error(H2_EINTERNAL, "sum lda < n");
        check(it.a, (int64_t)(s.m - 1) * s.lda + s.n, "sum input");
        continue;
      }
      const int lda = it.lda ? it.lda : s.lda, ldb = it.ldb ? it.ldb : s.ldb;
      const int kp = it.kpad ? it.kpad : s.k;
      if (kp > s.k) throw Error(H2_EINTERNAL, "item k above the segment's");
      if ((!ta && lda < kp) || (ta && lda < s.m) || (!tb && ldb < s.n) || (tb && ldb < kp))
        throw Error(H2_EINTERNAL, "segment leading dimension too small");
      check(it.a, ta ? (int64_t)(kp - 1) * lda + s.m : (int64_t)(s.m - 1) * lda + kp, "segment A");
      check(it.b, tb ? (int64_t)(s.n - 1) * ldb + kp : (int64_t)(kp - 1) * ldb + s.n, "segment B");
    }
  };
  // a group of the tensor-core coupling pass: up to two outputs, steps of A tiles
  // (rp x kpad) and a B tile (np x kpad), rp / np the launch's, kpad from 16 to the
  // launch's largest
  auto check_tc_group = [&](const TcGroup& g, const Launch& L) {
    if (g.m <= 0 || g.n <= 0 || g.ldc < g.n || g.count <= 0 || (g.out[0] < 0 && g.out[1] < 0))
      throw Error(H2_EINTERNAL, "bad tensor-core coupling group");
    if (((g.m + 7) & ~7) != L.aux2 || ((g.n + 7) & ~7) != L.aux || L.aux2 > 64 || L.aux > 64 || L.aux3 > 64)
      throw Error(H2_EINTERNAL, "tensor-core coupling tile rows differ from the launch's");
    if (g.first < 0 || (size_t)g.first + (size_t)g.count > P.tsteps.size())
      throw Error(H2_EINTERNAL, "tensor-core coupling steps out of range");
    for (int sl = 0; sl < 2; ++sl)
      if (g.out[sl] >= 0) check(g.out[sl], (int64_t)(g.m - 1) * g.ldc + g.n, "coupling output");
    for (int32_t q = g.first; q < g.first + g.count; ++q) {
      const TcStep& st = P.tsteps[q];
      if (st.kpad < 16 || st.kpad % 16 || st.kpad > L.aux3) throw Error(H2_EINTERNAL, "bad tensor-core tile k");
      for (int sl = 0; sl < 2; ++sl) {
        if (st.a[sl] >= 0 && g.out[sl] < 0) throw Error(H2_EINTERNAL, "coupling term of an empty slot");
        if (st.a[sl] >= 0) check(st.a[sl], (int64_t)L.aux2 * st.kpad, "coupling A tile");
      }
      if (st.a[0] < 0 && st.a[1] < 0) throw Error(H2_EINTERNAL, "coupling step without a term");
      check(st.b, (int64_t)L.aux * st.kpad, "coupling B tile");
    }
  };
  auto check_eig = [&](const EigTask& e) {
    for (int m = 0; m < 3; ++m)
      if (e.g[m] >= 0) check(e.g[m], (int64_t)e.n_pad * e.n_pad, "eig Gram");
    check(e.out, (int64_t)e.n_pad * e.kcap, "eig output");
    if (e.klim < 0 || e.klim > e.kcap) throw Error(H2_EINTERNAL, "eig rank limit above its stride");
    if (e.child1 < 0 && e.nleaf > e.n_pad) throw Error(H2_EINTERNAL, "eig leaf size above n_pad");
    if (e.child1 >= 0 && 2 * e.half > e.n_pad) throw Error(H2_EINTERNAL, "eig half above n_pad");
  };
  size_t nseg = 0, neig = 0, ngrp = 0;
  for (size_t li = 0; li < P.launches.size(); ++li) {
    for (; ev < P.aev.size() && P.aev[ev].launch <= (int32_t)li; ++ev) {
      const Plan::AllocEv& x = P.aev[ev];
      if (x.reset) {
        live[x.arena].clear();
        bucket[x.arena].clear();
        done[x.arena] = 0;
      } else if (x.size > 0) {  // (an empty allocation shares the next one's start)
        if (!live[x.arena].empty() && live[x.arena].back().first + live[x.arena].back().second > x.start)
          throw Error(H2_EINTERNAL, "plan allocations overlap");
        live[x.arena].push_back({x.start, x.size});
      }
    }
    // extend each table over the allocations appended since: bucket b gets the last
    // allocation with start <= b * kBucket, up to the bucket of the last one's start
    for (int a = 0; a < kArenas; ++a) {
      const auto& v = live[a];
      auto& bt = bucket[a];
      for (size_t q = done[a]; q < v.size(); ++q) {
        const size_t upto = (size_t)(v[q].first / kBucket) + 1;  // buckets whose start is < next bucket
        while (bt.size() < upto) {
          // bucket bt.size() starts at bt.size() * kBucket; allocation q starts at or
          // before it only if bt.size() * kBucket >= v[q].first
          const int64_t bs = (int64_t)bt.size() * kBucket;
          bt.push_back(bs >= v[q].first ? (int32_t)q : (int32_t)q - 1);
        }
      }
      done[a] = v.size();
    }
    const Launch& L = P.launches[li];
    if (L.kind == Launch::GEMM) {
      // segments of one launch are checked in parallel (the live lists are read only)
      std::string err;
#pragma omp parallel for schedule(dynamic, 4096)
      for (int64_t i = L.first; i < L.first + L.count; ++i) {
        try {
          if (L.tc) check_tc_group(P.tgroups[i], L);
          else check_seg(P.segs[i]);
        } catch (std::exception& e) {
#pragma omp critical
          if (err.empty()) err = e.what();
        }
      }
      if (!err.empty()) throw Error(H2_EINTERNAL, err);
      if (L.tc) ngrp += L.count;
      else nseg += L.count;
    } else if (L.kind == Launch::EIG) {
      for (int64_t i = L.first; i < L.first + L.count; ++i) check_eig(P.eigs[i]);
      neig += L.count;
    } else if (L.kind == Launch::MEMSET) {
      const int64_t a = arena_of(L.off);
      if (L.off < 0 || offset_of(L.off) + L.elems > sizes[a]) throw Error(H2_EINTERNAL, "plan memset out of bounds");
    }
  }
  if (nseg != P.segs.size() || neig != P.eigs.size() || ngrp != P.tgroups.size())
    throw Error(H2_EINTERNAL, "plan work outside its launches");
}

void upload_plan(Plan& P, size_t region_esize, bool own_regions) {
  P.d_segs = (Seg*)dmalloc(std::max<size_t>(1, P.segs.size()) * sizeof(Seg));
  P.d_items = (Item*)dmalloc(std::max<size_t>(1, P.items.size()) * sizeof(Item));
  P.d_eigs = (EigTask*)dmalloc(std::max<size_t>(1, P.eigs.size()) * sizeof(EigTask));
  if (!P.segs.empty()) cuda_check(cudaMemcpy(P.d_segs, P.segs.data(), P.segs.size() * sizeof(Seg), cudaMemcpyHostToDevice), "upload segs");
  if (!P.items.empty()) cuda_check(cudaMemcpy(P.d_items, P.items.data(), P.items.size() * sizeof(Item), cudaMemcpyHostToDevice), "upload items");
  if (!P.eigs.empty()) cuda_check(cudaMemcpy(P.d_eigs, P.eigs.data(), P.eigs.size() * sizeof(EigTask), cudaMemcpyHostToDevice), "upload eigs");
  if (!P.tgroups.empty()) {
    P.d_tgroups = (TcGroup*)dmalloc(P.tgroups.size() * sizeof(TcGroup));
    P.d_tsteps = (TcStep*)dmalloc(std::max<size_t>(1, P.tsteps.size()) * sizeof(TcStep));
    cuda_check(cudaMemcpy(P.d_tgroups, P.tgroups.data(), P.tgroups.size() * sizeof(TcGroup), cudaMemcpyHostToDevice),
               "upload coupling groups");
    if (!P.tsteps.empty())
      cuda_check(cudaMemcpy(P.d_tsteps, P.tsteps.data(), P.tsteps.size() * sizeof(TcStep), cudaMemcpyHostToDevice),
                 "upload coupling steps");
  }
  int64_t scratch = 0;
  for (auto& L : P.launches) {
    if (L.kind == Launch::GEMM && !L.tc) {  // (a tensor-core launch has its tile sizes and flops from the plan)
      int mx = 1, md = 1;
      double fl = 0;
      for (int64_t q = L.first; q < L.first + L.count; ++q) {
        const Seg& s = P.segs[q];
        mx = std::max<int>(mx, s.n);
        md = std::max<int>(md, std::max<int>(s.m, s.n));
        if (!(s.flags & SF_SUM))
          for (int32_t q = s.first; q < s.first + s.count; ++q)
            fl += 2.0 * s.m * s.n * (P.items[q].kpad ? P.items[q].kpad : s.k);
      }
      L.aux = mx;
      L.aux2 = md;
      bool sums = L.count > 0;
      for (int64_t q = L.first; q < L.first + L.count && sums; ++q) sums = P.segs[q].flags & SF_SUM;
      L.sums = sums;
      L.flops = fl;
    } else if (L.kind == Launch::EIG) {
      int mx = 1, kl = 1;
      for (int64_t q = L.first; q < L.first + L.count; ++q) {
        mx = std::max<int>(mx, P.eigs[q].n_pad);
        kl = std::max<int>(kl, P.eigs[q].klim);
      }
      L.aux2 = kl;
      if (mx > 256) throw Error(H2_EUNSUPPORTED, "Gram matrix larger than 256 (raise no caps in full mode)");
      L.aux = mx;
      int nn = mx + (mx & 1);
      if (P.cplx)
        scratch = std::max<int64_t>(scratch, zeig_scratch_elems(mx, L.count));
      else if (nn > 112)
        scratch = std::max<int64_t>(scratch, L.count * 2LL * nn * (nn + 1));
    }
  }
  P.scratch_elems = scratch;
  P.region_esize = (int)region_esize;
  if (own_regions)
    for (int a = AR_P; a <= AR_S; ++a) P.d_region[a] = (double*)dmalloc(std::max<int64_t>(1, P.region[a]) * region_esize);
}

void free_plan(Plan& P) {
  for (void* q : {(void*)P.d_segs, (void*)P.d_items, (void*)P.d_eigs, (void*)P.d_tgroups, (void*)P.d_tsteps})
    if (q) cudaFree(q);
  for (int a = 0; a < kArenas; ++a) {
    if (P.d_region[a]) cudaFree(P.d_region[a]);
    P.d_region[a] = nullptr;
  }
  P.d_segs = nullptr;
  P.d_items = nullptr;
  P.d_eigs = nullptr;
  P.d_tgroups = nullptr;
  P.d_tsteps = nullptr;
}

void run_plan(const Plan& P, const ArenaSet& ar, const Arenas* d_ars, const MmpParams& prm, void* stream,
              bool skip_memset, Trace* tr, const int8_t* choice, void* const* tune_ev) {
  if (tr) {
    while (tr->ev.size() < 2 * P.launches.size()) {
      cudaEvent_t e;
      cuda_check(cudaEventCreate(&e), "event");
      tr->ev.push_back((void*)e);
    }
    tr->recorded = true;
  }
  for (size_t li = 0; li < P.launches.size(); ++li) {
    const Launch& L = P.launches[li];
    if (tr) cuda_check(cudaEventRecord((cudaEvent_t)tr->ev[2 * li], (cudaStream_t)stream), "event");
    if (L.kind == Launch::MEMSET) {
      if (skip_memset || L.elems == 0) continue;
      int a = arena_of(L.off);
      char* p = (char*)ar.p[a] + offset_of(L.off) * ar.esize(a);
      cuda_check(cudaMemsetAsync(p, 0, L.elems * ar.esize(a), (cudaStream_t)stream), "memset");
    } else if (L.kind == Launch::COPY_RANKS) {
      // formatted product: C's ranks are A's row ranks and B's column ranks
      launch_copy_ranks(d_ars, 0, L.elems, stream);
    } else if (L.kind == Launch::GEMM) {
      const int v = choice ? choice[li] : 0;
      if (tune_ev) cuda_check(cudaEventRecord((cudaEvent_t)tune_ev[2 * li], (cudaStream_t)stream), "event");
      if (L.sums && !P.cplx)  // plain sums: one warp per segment
        launch_sum(P.d_segs, P.d_items, L.first, L.count, d_ars, is_mixed(prm.precision), stream);
      else if (L.tc)  // coupling sums on the tensor cores from operand tiles
        launch_coup_tc(P.d_tgroups, P.d_tsteps, L.first, L.count, d_ars, L.aux2, L.aux, L.aux3, ar.err,
                       v % kTcVariants, stream);
      else if (P.cplx && is_mixed(prm.precision))
        launch_zgemm32(P.d_segs, P.d_items, L.first, L.count, d_ars, L.aux, stream);
      else if (P.cplx)
        launch_zgemm(P.d_segs, P.d_items, L.first, L.count, d_ars, L.aux, stream);
      else if (prm.precision == H2_MIXED_TF32X3)
        launch_gemm_mma(P.d_segs, P.d_items, L.first, L.count, d_ars, L.aux2, L.aux, ar.err, v % kMmaVariants,
                        stream);
      else
        launch_gemm(P.d_segs, P.d_items, L.first, L.count, d_ars, L.aux, L.aux2, is_mixed(prm.precision),
                    stream, v % kGemmVariants);
      if (tune_ev) cuda_check(cudaEventRecord((cudaEvent_t)tune_ev[2 * li + 1], (cudaStream_t)stream), "event");
    } else {
      const int v = choice ? choice[li] : 0;
      if (P.cplx) {
        launch_zeig(P.d_eigs, L.first, L.count, d_ars, prm.eps, prm.trunc, prm.norm, L.aux, ar.eig_scratch, stream);
      } else if (eig_kept_path(prm, L)) {
        if (tune_ev) cuda_check(cudaEventRecord((cudaEvent_t)tune_ev[2 * li], (cudaStream_t)stream), "event");
        launch_eig_mixed(P.d_eigs, L.first, L.count, d_ars, prm.eps, prm.trunc, L.aux, v % kEigVariants, stream);
        if (tune_ev) cuda_check(cudaEventRecord((cudaEvent_t)tune_ev[2 * li + 1], (cudaStream_t)stream), "event");
      } else {
        launch_eig(P.d_eigs, L.first, L.count, d_ars, prm.eps, prm.trunc, prm.norm, L.aux, ar.eig_scratch, stream);
      }
    }
    cuda_check(cudaGetLastError(), L.phase);
    if (tr) cuda_check(cudaEventRecord((cudaEvent_t)tr->ev[2 * li + 1], (cudaStream_t)stream), "event");
  }
}

}  // namespace h2

namespace {

// The matrix that the host-only program checks (h2_plan_stats, h2_plan_digest,
// h2_plan_selfcheck) multiply: the structure of the points and the storage caps that an
// import of their Laplace H^2 matrix (host construction at eps) would set, with the
// arena offsets computed; no device memory.  Returns the arena size.
int64_t laplace_host_mat(const double* points, int64_t n, int32_t leaf_size, double eta, double eps, h2::Mat& m) {
  using namespace h2;
  auto st = build_structure(points, n, leaf_size, eta);
  const double h = std::cbrt(1.0 / (double)n);
  h2_kernel k{H2_K_LAPLACE, 0.0, 1.0 / (2.0 * M_PI * h), 0.0};
  Packed p;
  build_h2_host(*st, k, eps, p);
  m.st = st;
  m.Kr.assign(st->L + 1, 0);
  m.Kc.assign(st->L + 1, 0);
  for (int l = 0; l <= st->L; ++l)
    for (int64_t t = 0; t < (1LL << l); ++t) {
      m.Kr[l] = std::max(m.Kr[l], p.kr[Structure::node(l, t)]);
      m.Kc[l] = std::max(m.Kc[l], p.kc[Structure::node(l, t)]);
    }
  for (int l = 0; l <= st->L; ++l) {
    m.Kr[l] = cap_round(m.Kr[l]);
    m.Kc[l] = cap_round(m.Kc[l]);
  }
  return mat_elems(m);
}

}  // namespace

using namespace h2;

extern "C" {

const char* h2_last_error(void) { return g_err.c_str(); }

static Arenas* arena_slot(h2_matrix* h, int slot) {
  if (!h->d_ars) h->d_ars = (Arenas*)dmalloc(2 * sizeof(Arenas));
  return h->d_ars + slot;
}

static void finish_handle(h2_matrix* h, const h2_opts& o) {
  h->m.stream = o.stream;
  make_user_map(h);
}

h2_status h2_build(const double* points, int64_t n, const h2_kernel* kernel, int32_t leaf_size, double eta,
                   double eps, const h2_opts* opts, h2_handle* out) {
  if (!points || !kernel || !out) return fail(H2_EINVAL, "null argument");
  *out = nullptr;
  return guarded([&] {
    h2_opts o = defaults(opts);
    if (!(eps > 0) || !(eps < 1)) throw Error(H2_EINVAL, "eps must lie in (0, 1)");
    if (kernel->kind != H2_K_LAPLACE && kernel->kind != H2_K_INV_R2 && kernel->kind != H2_K_HELMHOLTZ)
      throw Error(H2_EINVAL, "unknown kernel kind");
    if (kernel->kind == H2_K_HELMHOLTZ && !(kernel->wavenumber >= 0 && std::isfinite(kernel->wavenumber)))
      throw Error(H2_EINVAL, "the Helmholtz kernel needs a finite wavenumber >= 0");
    auto h = std::make_unique<h2_matrix>();
    h->m.st = structure_for(points, n, leaf_size, eta);
    h->m.cplx = kernel->kind == H2_K_HELMHOLTZ;
    if (!h->m.cplx) {  // real kernels: built on the GPU, straight into the arena
      build_h2_device(*h->m.st, *kernel, eps, h->m);
      finish_handle(h.get(), o);
      *out = h.release();
      return;
    }
    Packed p;
    build_h2_host(*h->m.st, *kernel, eps, p);
    PackedView v;
    v.kr = p.kr.data();
    v.kc = p.kc.data();
    const std::vector<double>* a[6] = {&p.vr, &p.vc, &p.er, &p.ec, &p.s, &p.f};
    for (int i = 0; i < 6; ++i) {  // lengths in elements (a complex element is two doubles)
      v.arr[i] = a[i]->data();
      v.len[i] = (int64_t)a[i]->size() / (h->m.cplx ? 2 : 1);
    }
    unpack_view_to_device(v, h->m);
    finish_handle(h.get(), o);
    *out = h.release();
  });
}

h2_status h2_build_packed(const double* points, int64_t n, const h2_kernel* kernel, int32_t leaf_size, double eta,
                          double eps, int64_t* sizes, int32_t* kr, int32_t* kc, double* vr, double* vc, double* er,
                          double* ec, double* s, double* f) {
  if (!points || !kernel || !sizes) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    if (!(eps > 0) || !(eps < 1)) throw Error(H2_EINVAL, "eps must lie in (0, 1)");
    if (kernel->kind != H2_K_LAPLACE && kernel->kind != H2_K_INV_R2 && kernel->kind != H2_K_HELMHOLTZ)
      throw Error(H2_EINVAL, "unknown kernel kind");
    auto st = build_structure(points, n, leaf_size, eta);
    Packed p;
    build_h2_host(*st, *kernel, eps, p);
    const int w = kernel->kind == H2_K_HELMHOLTZ ? 2 : 1;
    const std::vector<double>* a[6] = {&p.vr, &p.vc, &p.er, &p.ec, &p.s, &p.f};
    sizes[0] = (int64_t)p.kr.size();
    for (int i = 0; i < 6; ++i) sizes[1 + i] = (int64_t)a[i]->size() / w;
    sizes[7] = 0;
    if (kr) std::copy(p.kr.begin(), p.kr.end(), kr);
    if (kc) std::copy(p.kc.begin(), p.kc.end(), kc);
    double* out[6] = {vr, vc, er, ec, s, f};
    for (int i = 0; i < 6; ++i)
      if (out[i]) std::copy(a[i]->begin(), a[i]->end(), out[i]);
  });
}

h2_status h2_set_alloc_limit(int64_t n) {
  g_alloc_left.store(n < 0 ? -1 : n);
  return H2_OK;
}

h2_status h2_plan_stats(const double* points, int64_t n, int32_t leaf_size, double eta, double eps, int32_t trunc,
                        double* flops, int64_t* segments, int64_t* items) {
  if (!points || !flops || !segments || !items) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    if (!(eps > 0) || !(eps < 1)) throw Error(H2_EINVAL, "eps must lie in (0, 1)");
    if (trunc < H2_TRUNC_PAPER || trunc > H2_TRUNC_FORMATTED) throw Error(H2_EINVAL, "unknown truncation rule");
    Mat m;
    laplace_host_mat(points, n, leaf_size, eta, eps, m);
    const std::shared_ptr<Structure>& st = m.st;
    Plan P;
    Mat C;
    C.st = st;
    MmpParams prm{1e-4, trunc, 48, H2_FP64};
    build_mmp_plan(m, m, C, prm, P);
    *flops = (double)P.flops;
    *segments = (int64_t)P.segs.size();
    *items = (int64_t)P.items.size();
  });
}

h2_status h2_plan_digest(const double* points, int64_t n, int32_t leaf_size, double eta, double eps,
                         int32_t precision, int32_t trunc, uint64_t* digest) {
  if (!points || !digest) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    if (!(eps > 0) || !(eps < 1)) throw Error(H2_EINVAL, "eps must lie in (0, 1)");
    if (trunc < H2_TRUNC_PAPER || trunc > H2_TRUNC_FORMATTED) throw Error(H2_EINVAL, "unknown truncation rule");
    if (precision < H2_FP64 || precision > H2_MIXED_BF16X3) throw Error(H2_EINVAL, "unknown precision");
    Mat m;
    laplace_host_mat(points, n, leaf_size, eta, eps, m);
    const std::shared_ptr<Structure>& st = m.st;
    Plan P;
    Mat C;
    C.st = st;
    MmpParams prm{1e-4, trunc, 48, precision};
    build_mmp_plan(m, m, C, prm, P);
    // FNV-1a over the fields (not the raw structs: their padding bytes are unset)
    uint64_t hsh = 1469598103934665603ull;
    auto mix = [&](auto v) {
      const unsigned char* c = reinterpret_cast<const unsigned char*>(&v);
      for (size_t i = 0; i < sizeof(v); ++i) {
        hsh ^= c[i];
        hsh *= 1099511628211ull;
      }
    };
    for (const Seg& x : P.segs) {
      mix(x.out), mix(x.first), mix(x.count), mix(x.m), mix(x.n), mix(x.k), mix(x.lda), mix(x.ldb), mix(x.ldc);
      mix(x.mref), mix(x.nref), mix(x.flags), mix(x.flags2), mix(x.inst), mix(x.trows);
    }
    for (const Item& x : P.items) mix(x.a), mix(x.b), mix(x.kref), mix(x.lda), mix(x.ldb), mix(x.kpad);
    for (const TcGroup& x : P.tgroups) {
      mix(x.out[0]), mix(x.out[1]), mix(x.mref[0]), mix(x.mref[1]), mix(x.nref), mix(x.first), mix(x.count);
      mix(x.m), mix(x.n), mix(x.ldc), mix(x.acc), mix(x.inst);
    }
    for (const TcStep& x : P.tsteps) mix(x.a[0]), mix(x.a[1]), mix(x.b), mix(x.kref), mix(x.kpad);
    for (const EigTask& x : P.eigs) {
      mix(x.g[0]), mix(x.g[1]), mix(x.g[2]), mix(x.out), mix(x.rank_out), mix(x.child1), mix(x.child2);
      mix(x.nleaf), mix(x.n_pad), mix(x.half), mix(x.kcap), mix(x.col), mix(x.klim), mix(x.inst);
    }
    for (const Launch& x : P.launches) {
      mix((int)x.kind), mix(x.first), mix(x.count), mix(x.off), mix(x.elems), mix(x.level), mix(x.tc);
      mix(x.sums), mix(x.aux), mix(x.aux2), mix(x.aux3), mix(x.flops);
      for (const char* c = x.phase; *c; ++c) mix(*c);
    }
    for (const auto& x : P.aev) mix(x.launch), mix(x.arena), mix(x.reset), mix(x.start), mix(x.size);
    for (int a = 0; a < kArenas; ++a) mix(P.region[a]);
    mix(P.fext), mix(P.flops), mix(P.scratch_elems), mix(P.region_esize);
    *digest = hsh;
  });
}

h2_status h2_plan_selfcheck(const double* points, int64_t n, int32_t leaf_size, double eta, double eps,
                            int32_t* checked) {
  if (!points || !checked) return fail(H2_EINVAL, "null argument");
  *checked = 0;
  return guarded([&] {
    if (!(eps > 0) || !(eps < 1)) throw Error(H2_EINVAL, "eps must lie in (0, 1)");
    // host only: structure, H^2 ranks of the Laplace kernel, storage caps as an import
    // would set them, then every program built and validated (no device memory)
    Mat m;
    const int64_t asz = laplace_host_mat(points, n, leaf_size, eta, eps, m);
    const std::shared_ptr<Structure>& st = m.st;
    for (int trunc : {H2_TRUNC_PAPER, H2_TRUNC_SV, H2_TRUNC_FULL, H2_TRUNC_FORMATTED})
      for (int prec : {H2_FP64, H2_MIXED_FP32, H2_MIXED_BF16X3})
        for (int cap : {24, 48}) {
          Plan P;
          Mat C;
          C.st = st;
          MmpParams prm{1e-4, trunc, cap, prec};
          try {
            build_mmp_plan(m, m, C, prm, P);
            const int64_t csz = mat_elems(C);
            int64_t sizes[kArenas] = {asz + P.fext, asz + P.fext, csz, P.region[AR_P], P.region[AR_G0],
                                      P.region[AR_G1], P.region[AR_S], is_mixed(prec) ? C.off_S[0] : 0};
            validate_plan(P, sizes);
          } catch (Error& e) {
            throw Error(e.code, "product plan (trunc " + std::to_string(trunc) + ", precision " +
                                    std::to_string(prec) + ", cap " + std::to_string(cap) + "): " + e.what());
          }
          ++*checked;
        }
    for (int64_t nrhs : {1, 3}) {
      Plan P;
      int64_t ox, oy;
      build_matvec_plan(m, nrhs, P, ox, oy);
      int64_t sizes[kArenas] = {asz, 0, 0, P.region[AR_P], 0, 0, 0, 0};
      validate_plan(P, sizes);
      ++*checked;
    }
  });
}

h2_status h2_import(const double* points, int64_t n, int32_t leaf_size, double eta, const int32_t* kr,
                    const int32_t* kc, const double* vr, const double* vc, const double* er, const double* ec,
                    const double* s, const double* f, const h2_opts* opts, h2_handle* out) {
  if (!points || !kr || !kc || !out) return fail(H2_EINVAL, "null argument");
  *out = nullptr;
  return guarded([&] {
    h2_opts o = defaults(opts);
    auto h = std::make_unique<h2_matrix>();
    h->m.st = structure_for(points, n, leaf_size, eta);
    PackedView v;
    v.kr = kr;
    v.kc = kc;
    packed_lengths(*h->m.st, kr, kc, v.len);
    const double* a[6] = {vr, vc, er, ec, s, f};
    for (int i = 0; i < 6; ++i) v.arr[i] = a[i];
    unpack_view_to_device(v, h->m);
    finish_handle(h.get(), o);
    *out = h.release();
  });
}

h2_status h2_import_complex(const double* points, int64_t n, int32_t leaf_size, double eta, const int32_t* kr,
                            const int32_t* kc, const double* vr, const double* vc, const double* er, const double* ec,
                            const double* s, const double* f, const h2_opts* opts, h2_handle* out) {
  if (!points || !kr || !kc || !out) return fail(H2_EINVAL, "null argument");
  *out = nullptr;
  return guarded([&] {
    h2_opts o = defaults(opts);
    auto h = std::make_unique<h2_matrix>();
    h->m.st = structure_for(points, n, leaf_size, eta);
    h->m.cplx = true;
    PackedView v;
    v.kr = kr;
    v.kc = kc;
    packed_lengths(*h->m.st, kr, kc, v.len);
    const double* a[6] = {vr, vc, er, ec, s, f};
    for (int i = 0; i < 6; ++i) v.arr[i] = a[i];
    unpack_view_to_device(v, h->m);
    finish_handle(h.get(), o);
    *out = h.release();
  });
}

h2_status h2_export(h2_handle h, int64_t* sizes, int32_t* kr, int32_t* kc, double* vr, double* vc, double* er,
                    double* ec, double* s, double* f) {
  if (!h || !sizes) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    // sizes from the ranks alone; the arrays only when asked for
    sync_ranks_to_host(h->m);
    if (h->m.d_cap) {
      unsigned long long e = 0;
      cuda_check(cudaMemcpy(&e, h->m.d_cap + 2, sizeof(e), cudaMemcpyDeviceToHost), "error word");
      if (e) throw Error(H2_ETIMEOUT, "a bounded wait of the tensor-core kernel gave up: the product is invalid");
    }
    int64_t len[6];
    packed_lengths(*h->m.st, h->m.h_kr.data(), h->m.h_kc.data(), len);
    sizes[0] = (int64_t)h->m.h_kr.size();
    for (int i = 0; i < 6; ++i) sizes[1 + i] = len[i];
    sizes[7] = 0;
    if (kr) std::copy(h->m.h_kr.begin(), h->m.h_kr.end(), kr);
    if (kc) std::copy(h->m.h_kc.begin(), h->m.h_kc.end(), kc);
    double* const out[6] = {vr, vc, er, ec, s, f};
    bool any = false;
    for (int i = 0; i < 6; ++i) any = any || out[i];
    if (any) pack_to_host(h->m, out);
  });
}

}  // extern "C"

namespace {

// ------------------------------------------------------------ work space
// The work regions of a product (P, G0, G1, S) hold nothing between products, so they
// come from one device buffer per stream, grown on demand and reused by every product
// on that stream (a batch takes one slice per product of a merged group).  `gen`
// changes when the buffer moves, which retires programs captured with the old one.
struct Workspace {
  char* base = nullptr;
  size_t bytes = 0;
  uint64_t gen = 0;
};
std::mutex g_ws_mu;
std::map<void*, Workspace> g_ws;

size_t region_bytes(const Plan& P) {
  size_t b = 0;
  for (int a = AR_P; a <= AR_S; ++a) b += ((size_t)std::max<int64_t>(1, P.region[a]) * P.region_esize + 255) & ~size_t(255);
  return b + (((size_t)P.scratch_elems * sizeof(double) + 255) & ~size_t(255));
}

Workspace workspace(void* stream, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_ws_mu);
  Workspace& w = g_ws[stream];
  if (w.bytes < bytes) {
    if (w.base) {
      cuda_check(cudaDeviceSynchronize(), "synchronise");
      cudaFree(w.base);
      w.base = nullptr;
      w.bytes = 0;
    }
    w.base = (char*)dmalloc(bytes);
    w.bytes = bytes;
    ++w.gen;
  }
  return w;
}

// points the work regions of `ar` at `base` (region_bytes(P) bytes)
void place_regions(const Plan& P, ArenaSet& ar, char* base) {
  size_t off = 0;
  for (int a = AR_P; a <= AR_S; ++a) {
    ar.p[a] = base + off;
    off += ((size_t)std::max<int64_t>(1, P.region[a]) * P.region_esize + 255) & ~size_t(255);
  }
  ar.eig_scratch = P.scratch_elems ? (double*)(base + off) : nullptr;
}

// One product made ready to run: its plan (built or from the cache), its output
// handle (reused or new, zeroed in stream order), float copies of A and B if mixed, and
// its arena table.
struct Prepared {
  std::shared_ptr<PlanEntry> ent;
  h2_matrix* out = nullptr;
  std::unique_ptr<h2_matrix> fresh;
  ArenaSet ar;
  MmpParams prm{};
  bool trace = false;
};

Prepared prepare_product(h2_handle A, h2_handle B, double eps, const h2_opts& o, h2_handle existing) {
  Prepared pr;
  if (o.trunc != H2_TRUNC_FULL && o.trunc != H2_TRUNC_FORMATTED && !(eps > 0 && eps < 1))
    throw Error(H2_EINVAL, "eps must lie in (0, 1)");
  if (existing && (existing == A || existing == B))
    throw Error(H2_EINVAL, "the output handle must not be an operand of the product");
  if (!same_structure(*A->m.st, *B->m.st)) throw Error(H2_ESTRUCT, "A and B have different trees or partitions");
  if (A->m.cplx != B->m.cplx) throw Error(H2_EINVAL, "A and B must both be real or both complex");
  if (A->m.cplx && o.precision != H2_FP64 && o.precision != H2_MIXED_FP32)
    throw Error(H2_EUNSUPPORTED, "complex products run in float64 or mixed float32 (H2_FP64, H2_MIXED_FP32)");
  MmpParams prm{eps, o.trunc, o.rank_cap, o.precision, o.norm, o.autotune};
  // plan cache, process-wide
  PlanKey key{A->m.st.get(), A->m.Kr, A->m.Kc, B->m.Kr, B->m.Kc, o.trunc, o.rank_cap, o.precision, A->m.cplx};
  std::shared_ptr<PlanEntry> ent;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (auto it = g_plans.begin(); it != g_plans.end();) {
      auto sp = it->second.lock();
      if (!sp) {
        it = g_plans.erase(it);
        continue;
      }
      if (it->first == key) ent = sp;
      ++it;
    }
  }
  if (!ent) {
    ent = std::make_shared<PlanEntry>();
    Mat Ccaps;
    Ccaps.st = A->m.st;
    build_mmp_plan(A->m, B->m, Ccaps, prm, ent->plan);
    ent->plan.ckr = Ccaps.Kr;
    ent->plan.ckc = Ccaps.Kc;
    {
      Mat probe;
      probe.st = A->m.st;
      probe.Kr = Ccaps.Kr;
      probe.Kc = Ccaps.Kc;
      int64_t csize = mat_elems(probe);
      int64_t sizes[kArenas] = {A->m.arena_elems + ent->plan.fext, B->m.arena_elems + ent->plan.fext, csize,
                                ent->plan.region[AR_P],
                                ent->plan.region[AR_G0], ent->plan.region[AR_G1], ent->plan.region[AR_S],
                                is_mixed(o.precision) ? probe.off_S[0] : 0};
      validate_plan(ent->plan, sizes);
    }
    upload_plan(ent->plan, (A->m.cplx ? 2 : 1) * (is_mixed(o.precision) ? sizeof(float) : sizeof(double)),
                false);
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_plans.push_back({key, ent});
  }
  bool held = false;
  for (auto& p : A->plans_held) held = held || p == ent;
  if (!held) A->plans_held.push_back(ent);
  h2_matrix* out = existing;
  bool reuse = out && out->m.st == A->m.st && out->origin_trunc == o.trunc && out->origin_cap == o.rank_cap &&
               out->origin_prec == o.precision && out->m.Kr == ent->plan.ckr && out->m.Kc == ent->plan.ckc &&
               out->m.cplx == A->m.cplx;
  std::unique_ptr<h2_matrix> fresh;
  if (!reuse) {
    fresh = std::make_unique<h2_matrix>();
    fresh->m.st = A->m.st;
    fresh->m.Kr = ent->plan.ckr;
    fresh->m.Kc = ent->plan.ckc;
    fresh->m.cplx = A->m.cplx;
    alloc_mat(fresh->m);
    fresh->m.stream = o.stream;
    make_user_map(fresh.get());
    cudaEventCreate(&fresh->ev0);
    cudaEventCreate(&fresh->ev1);
    fresh->origin_A = A;
    fresh->origin_B = B;
    fresh->origin_trunc = o.trunc;
    fresh->origin_cap = o.rank_cap;
    fresh->origin_prec = o.precision;
    out = fresh.get();
  }
  out->m.stream = o.stream;
  out->m.ranks_on_host = false;
  out->m.arena32_stale = true;  // this product rewrites C's arena
  cudaStream_t s = (cudaStream_t)o.stream;
  cuda_check(cudaEventRecord(out->ev0, s), "event");
  cuda_check(cudaMemsetAsync(out->m.arena, 0, out->m.arena_elems * out->m.esize(), s), "zero C");
  cuda_check(cudaMemsetAsync(out->m.d_kr, 0, 2 * A->m.st->nnodes() * sizeof(int32_t) + 64, s), "zero ranks");
  ArenaSet ar;
  const bool mixed = is_mixed(o.precision);
  if (mixed) {
    const int w = A->m.cplx ? 2 : 1;  // floats per element
    const int64_t fext = ent->plan.fext;  // the dense blocks' operand tiles after the copy
    for (h2_matrix* h : {A, B}) {
      // the float copy of the whole arena: made on first use, made again when a product
      // has rewritten the arena since (a product's output used as an input); with the
      // operand tiles of its dense blocks after it where the program reads them
      const int64_t need = h->m.arena_elems * w + fext;
      if (h->m.arena32 && h->m.arena32_cap < need) {
        cuda_check(cudaStreamSynchronize((cudaStream_t)o.stream), "synchronise");
        cudaFree(h->m.arena32);
        h->m.arena32 = nullptr;
      }
      if (!h->m.arena32) {
        h->m.arena32 = (float*)dmalloc(need * sizeof(float));
        h->m.arena32_cap = need;
        h->m.arena32_stale = true;
      }
      if (h->m.arena32_stale) {
        launch_to_f32(h->m.arena, h->m.arena32, h->m.arena_elems * w, o.stream);
        cuda_check(cudaGetLastError(), "convert to float");
        h->m.arena32_stale = false;
        h->m.ftiles = false;
      }
      if (fext && !h->m.ftiles) {
        launch_f_tiles(h->m.arena, h->m.off_F, h->m.st->nF, h->m.st->LS, h->m.arena32 + h->m.arena_elems, o.stream);
        cuda_check(cudaGetLastError(), "dense block tiles");
        h->m.ftiles = true;
      }
    }
    ar.p[AR_A] = A->m.arena32;
    ar.p[AR_B] = B->m.arena32;
    if (!out->m.bases32)
      out->m.bases32 = (float*)dmalloc(std::max<int64_t>(1, out->m.off_S[0]) * w * sizeof(float));
    ar.p[AR_X] = out->m.bases32;  // float copy of C's bases, written by the eigen step
    ar.f32 = (1u << AR_A) | (1u << AR_B) | (1u << AR_P) | (1u << AR_G0) | (1u << AR_G1) | (1u << AR_S) |
             (1u << AR_X);
    if (A->m.cplx)  // complex: float2 in the float arenas, double2 in C
      ar.c16 = (1u << AR_A) | (1u << AR_B) | (1u << AR_C) | (1u << AR_P) | (1u << AR_G0) | (1u << AR_G1) |
               (1u << AR_S) | (1u << AR_X);
  } else {
    ar.p[AR_A] = A->m.arena;
    ar.p[AR_B] = B->m.arena;
    if (A->m.cplx)
      ar.c16 = (1u << AR_A) | (1u << AR_B) | (1u << AR_C) | (1u << AR_P) | (1u << AR_G0) | (1u << AR_G1) | (1u << AR_S);
  }
  ar.p[AR_C] = out->m.arena;
  ar.rk[RK_AR] = A->m.d_kr;
  ar.rk[RK_AC] = A->m.d_kc;
  ar.rk[RK_BR] = B->m.d_kr;
  ar.rk[RK_BC] = B->m.d_kc;
  ar.rk[RK_CR] = out->m.d_kr;
  ar.rk[RK_CC] = out->m.d_kc;
  out->made_by = ent;
  out->trace_plan = A->trace_on ? &ent->plan : nullptr;
  if (A->trace_on) {
    ar.flops = out->m.d_cap + 1;  // second counter of the handle's counter block
    cuda_check(cudaMemsetAsync(ar.flops, 0, sizeof(unsigned long long), s), "zero flop counter");
  }
  ar.kr = out->m.d_kr;
  ar.kc = out->m.d_kc;
  ar.cap_hits = out->m.d_cap;
  ar.err = (unsigned int*)(out->m.d_cap + 2);  // third word of the handle's counter block
  pr.ent = ent;
  pr.out = out;
  pr.fresh = std::move(fresh);
  pr.ar = ar;
  pr.prm = prm;
  pr.trace = A->trace_on;
  return pr;
}

}  // namespace

extern "C" {

h2_status h2_mmp(h2_handle A, h2_handle B, double eps, const h2_opts* opts, h2_handle* C) {
  if (!A || !B || !C) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    h2_opts o = defaults(opts);
    Prepared pr = prepare_product(A, B, eps, o, *C);
    h2_matrix* out = pr.out;
    place_regions(pr.ent->plan, pr.ar, workspace(o.stream, region_bytes(pr.ent->plan)).base);
    Arenas* d_ars = arena_slot(out, 0);
    upload_arenas(d_ars, to_arenas(pr.ar), o.stream);
    if (o.autotune) {
      TuneState& ts = pr.ent->tune;
      std::lock_guard<std::mutex> lk(ts.mu);
      const Plan& P = pr.ent->plan;
      const size_t nl = P.launches.size();
      if (ts.choice.empty()) {
        // candidates: every launch kind's variants, taken modulo its own count
        ts.ncand = kTuneCandidates;
        ts.choice.assign(nl, 0);
        ts.ms.assign(nl, std::vector<float>(ts.ncand, -1.f));
        for (size_t li = 0; li < nl; ++li) {
          const Launch& L = P.launches[li];
          if ((L.kind == Launch::GEMM && !P.cplx) ||
              (L.kind == Launch::EIG && !P.cplx && eig_kept_path(pr.prm, L)))
            ts.choice[li] = -1;
        }
        for (size_t i = 0; i < 2 * nl + 1; ++i) {  // two per launch and an end marker
          cudaEvent_t e;
          cuda_check(cudaEventCreate(&e), "event");
          ts.ev.push_back((void*)e);
        }
      }
      if (ts.pending) {  // the times of the last exploration product
        cuda_check(cudaEventSynchronize((cudaEvent_t)ts.ev.back()), "event");
        const int cand = (ts.explored - 1) % ts.ncand;
        for (size_t li = 0; li < nl; ++li) {
          if (ts.choice[li] >= 0) continue;
          float t = 0;
          cuda_check(cudaEventElapsedTime(&t, (cudaEvent_t)ts.ev[2 * li], (cudaEvent_t)ts.ev[2 * li + 1]), "event");
          ts.ms[li][cand] = t;
          int best = 0;
          bool all = true;
          for (int c = 0; c < ts.ncand; ++c) {
            all = all && ts.ms[li][c] >= 0.f;
            if (ts.ms[li][c] >= 0.f && ts.ms[li][c] < ts.ms[li][best]) best = c;
          }
          if (all) ts.choice[li] = (int8_t)best;
        }
        ts.pending = false;
      }
      bool exploring = false;
      std::vector<int8_t> run(nl, 0);
      const int cand = ts.explored % ts.ncand;
      for (size_t li = 0; li < nl; ++li) {
        run[li] = ts.choice[li] >= 0 ? ts.choice[li] : (int8_t)cand;
        exploring = exploring || ts.choice[li] < 0;
      }
      run_plan(pr.ent->plan, pr.ar, d_ars, pr.prm, o.stream, false, pr.trace ? &out->trace : nullptr, run.data(),
               exploring ? ts.ev.data() : nullptr);
      if (exploring) {
        cuda_check(cudaEventRecord((cudaEvent_t)ts.ev.back(), (cudaStream_t)o.stream), "event");
        ts.explored += 1;
        ts.pending = true;
      }
    } else {
      run_plan(pr.ent->plan, pr.ar, d_ars, pr.prm, o.stream, false, pr.trace ? &out->trace : nullptr);
    }
    cuda_check(cudaEventRecord(out->ev1, (cudaStream_t)o.stream), "event");
    out->timed = true;
    if (pr.fresh) *C = pr.fresh.release();
  });
}

}  // extern "C"

namespace {

// ------------------------------------------------------------ batched products
// The products of a batch are independent, so they run as one CUDA graph with one
// branch per product: each branch is that product's own program (the same launches as
// h2_mmp, on its plan's arrays), captured on its own stream forked from a common
// start, and the branches join at the end.  The GPU runs the branches concurrently
// (one product's eigen step beside another's GEMMs).  Each product of a group takes its
// own slice of the work space.  The graph is captured once per (plans, work space, eps,
// truncation, precision) and replayed; only the arena tables change between calls and
// they are written just before the graph in stream order.  A product's launches and
// each segment's order of items are those of h2_mmp, so the results are bit for bit
// those of single products.
struct BatchEntry {
  std::vector<std::shared_ptr<PlanEntry>> plans;
  char* ws_base = nullptr;  // the work space the graph was captured with
  uint64_t ws_gen = 0;
  double eps = 0;
  int trunc = 0, precision = 0, norm = 0;
  Arenas* d_ars = nullptr;  // one table per product
  long long kernels = 0;    // kernels of one run of the graph
  cudaGraphExec_t graph = nullptr;
  ~BatchEntry() {
    if (graph) cudaGraphExecDestroy(graph);
    if (d_ars) cudaFree(d_ars);
  }
};

std::mutex g_batch_mu;
std::vector<std::shared_ptr<BatchEntry>> g_batches;  // most recent last, at most 4 kept

std::shared_ptr<BatchEntry> capture_batch(const std::vector<Prepared*>& grp) {
  auto be = std::make_shared<BatchEntry>();
  be->eps = grp[0]->prm.eps;
  be->trunc = grp[0]->prm.trunc;
  be->precision = grp[0]->prm.precision;
  be->norm = grp[0]->prm.norm;
  for (Prepared* p : grp) be->plans.push_back(p->ent);
  be->d_ars = (Arenas*)dmalloc(grp.size() * sizeof(Arenas));
  init_kernel_attributes();
  std::vector<cudaStream_t> st(grp.size() + 1, nullptr);
  std::vector<cudaEvent_t> ev(grp.size() + 1, nullptr);
  auto release = [&] {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    for (auto x : st)
      if (x) {
        release_eig_streams(x);
        cudaStreamDestroy(x);
      }
  };
  cudaGraph_t g = nullptr;
  try {
    for (auto& x : st) {
      cuda_check(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "capture stream");
      prepare_eig_streams(x);  // (no stream or event is made inside the capture)
    }
    for (auto& e : ev) cuda_check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "capture event");
    const unsigned long long k0 = kernel_launches();
    cuda_check(cudaStreamBeginCapture(st[0], cudaStreamCaptureModeThreadLocal), "begin capture");
    cuda_check(cudaEventRecord(ev[0], st[0]), "fork");
    for (size_t i = 0; i < grp.size(); ++i) {
      cudaStream_t si = st[i + 1];
      cuda_check(cudaStreamWaitEvent(si, ev[0], 0), "fork");
      run_plan(grp[i]->ent->plan, grp[i]->ar, be->d_ars + i, grp[i]->prm, si, false, nullptr);
      cuda_check(cudaEventRecord(ev[i + 1], si), "join");
      cuda_check(cudaStreamWaitEvent(st[0], ev[i + 1], 0), "join");
    }
    cuda_check(cudaStreamEndCapture(st[0], &g), "end capture");
    be->kernels = (long long)(kernel_launches() - k0);
    add_kernel_launches(-be->kernels);  // captured, not launched
    cuda_check(cudaGraphInstantiate(&be->graph, g, 0), "instantiate graph");
    cudaGraphDestroy(g);
  } catch (...) {
    cudaGraph_t gg = nullptr;
    if (st[0]) cudaStreamEndCapture(st[0], &gg);
    if (gg) cudaGraphDestroy(gg);
    if (g) cudaGraphDestroy(g);
    release();
    cudaGetLastError();
    throw;
  }
  release();
  return be;
}

void run_group(std::vector<Prepared*>& grp, const Workspace& ws, void* stream) {
  // each product of the group takes its own slice of the work space
  size_t off = 0;
  for (Prepared* p : grp) {
    place_regions(p->ent->plan, p->ar, ws.base + off);
    off += region_bytes(p->ent->plan);
  }
  std::shared_ptr<BatchEntry> be;
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (auto& e : g_batches) {
      if (e->plans.size() != grp.size() || e->eps != grp[0]->prm.eps || e->trunc != grp[0]->prm.trunc ||
          e->precision != grp[0]->prm.precision || e->norm != grp[0]->prm.norm || e->ws_base != ws.base || e->ws_gen != ws.gen)
        continue;
      bool same = true;
      for (size_t i = 0; i < grp.size() && same; ++i) same = e->plans[i] == grp[i]->ent;
      if (same) be = e;
    }
  }
  if (!be) {
    be = capture_batch(grp);
    be->ws_base = ws.base;
    be->ws_gen = ws.gen;
    std::lock_guard<std::mutex> lk(g_batch_mu);
    g_batches.push_back(be);
    if (g_batches.size() > 4) g_batches.erase(g_batches.begin());
  }
  for (size_t i = 0; i < grp.size(); ++i) upload_arenas(be->d_ars + i, to_arenas(grp[i]->ar), stream);
  cuda_check(cudaGetLastError(), "arena tables");
  cuda_check(cudaGraphLaunch(be->graph, (cudaStream_t)stream), "graph launch");
  add_kernel_launches(be->kernels);
}

}  // namespace

extern "C" {

h2_status h2_mmp_batched(const h2_handle* A, const h2_handle* B, int32_t count, double eps, const h2_opts* opts,
                         h2_handle* C) {
  if (!A || !B || !C || count < 0) return fail(H2_EINVAL, "null argument or negative count");
  for (int32_t i = 0; i < count; ++i)
    if (!A[i] || !B[i]) return fail(H2_EINVAL, "null handle at instance " + std::to_string(i));
  bool traced = false;
  for (int32_t i = 0; i < count; ++i) traced = traced || A[i]->trace_on;
  if (traced || count > 32767) {  // traced products keep their per-launch events: one at a time
    for (int32_t i = 0; i < count; ++i) {
      h2_status st = h2_mmp(A[i], B[i], eps, opts, &C[i]);
      if (st != H2_OK) return fail(st, "instance " + std::to_string(i) + ": " + g_err);
    }
    return H2_OK;
  }
  return guarded([&] {
    h2_opts o = defaults(opts);
    std::vector<Prepared> pr(count);
    for (int32_t i = 0; i < count; ++i) {
      try {
        pr[i] = prepare_product(A[i], B[i], eps, o, C[i]);
      } catch (Error& e) {
        throw Error(e.code, "instance " + std::to_string(i) + ": " + e.what());
      }
    }
    // groups of products whose work spaces fit together in 70 % of the free device
    // memory (the first product of a group always joins)
    size_t free_b = 0, total_b = 0;
    cuda_check(cudaMemGetInfo(&free_b, &total_b), "memory info");
    size_t have = 0;
    {
      std::lock_guard<std::mutex> lk(g_ws_mu);
      auto it = g_ws.find(o.stream);
      if (it != g_ws.end()) have = it->second.bytes;
    }
    const size_t budget = (size_t)(0.7 * (double)(free_b + have));
    std::vector<std::vector<Prepared*>> groups;
    std::vector<size_t> need, wneed;
    for (int32_t i = 0; i < count; ++i) {
      const size_t w = region_bytes(pr[i].ent->plan);
      const size_t b = w;
      if (groups.empty() || need.back() + b > budget) {
        groups.emplace_back();
        need.push_back(0);
        wneed.push_back(0);
      }
      groups.back().push_back(&pr[i]);
      need.back() += b;
      wneed.back() += w;
    }
    const Workspace ws = workspace(o.stream, *std::max_element(wneed.begin(), wneed.end()));
    for (auto& grp : groups) run_group(grp, ws, o.stream);
    for (int32_t i = 0; i < count; ++i) {
      cuda_check(cudaEventRecord(pr[i].out->ev1, (cudaStream_t)o.stream), "event");
      pr[i].out->timed = true;
      if (pr[i].fresh) C[i] = pr[i].fresh.release();
    }
  });
}

h2_status h2_matvec(h2_handle h, const double* x, double* y, int64_t nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "null argument");
  if (nrhs < 1 || nrhs > 16384) return fail(H2_EINVAL, "nrhs must lie in [1, 16384]");
  return guarded([&] {
    auto it = h->mv_plans.find(nrhs);
    if (it == h->mv_plans.end()) {
      auto p = std::make_unique<Plan>();
      int64_t ox, oy;
      build_matvec_plan(h->m, nrhs, *p, ox, oy);
      int64_t sizes[kArenas] = {h->m.arena_elems, 0, 0, p->region[AR_P], 0, 0, 0, 0};
      validate_plan(*p, sizes);
      upload_plan(*p, h->m.esize(), true);
      h->mv_offs[nrhs] = {ox, oy};
      it = h->mv_plans.emplace(nrhs, std::move(p)).first;
    }
    Plan& P = *it->second;
    auto offs = h->mv_offs[nrhs];
    const Structure& st = *h->m.st;
    int64_t rows = (1LL << st.L) * st.LS;
    cudaStream_t s = (cudaStream_t)h->m.stream;
    double* W = P.d_region[AR_P];
    const int w = h->m.cplx ? 2 : 1;  // doubles per element
    cuda_check(cudaMemsetAsync(W, 0, P.region[AR_P] * h->m.esize(), s), "zero workspace");
    double* xt = W + offset_of(offs.first) * w;
    double* yt = W + offset_of(offs.second) * w;
    if (h->m.cplx)
      launch_zpermute(x, xt, h->d_user, rows, st.n, nrhs, true, s);
    else
      launch_permute(x, xt, h->d_user, rows, st.n, nrhs, true, s);
    ArenaSet ar;
    ar.p[AR_A] = h->m.arena;
    ar.p[AR_P] = W;
    if (h->m.cplx) ar.c16 = (1u << AR_A) | (1u << AR_P);
    MmpParams prm{0, 0, 0, 0};
    Arenas* d_ars = arena_slot(h, 1);
    upload_arenas(d_ars, to_arenas(ar), s);
    run_plan(P, ar, d_ars, prm, s, true);
    if (h->m.cplx)
      launch_zpermute(yt, y, h->d_user, rows, st.n, nrhs, false, s);
    else
      launch_permute(yt, y, h->d_user, rows, st.n, nrhs, false, s);
    cuda_check(cudaGetLastError(), "matvec");
  });
}

h2_status h2_matvec_noalloc(h2_handle h, const double* x, double* y, int64_t nrhs) {
  if (!h || !x || !y) return fail(H2_EINVAL, "null argument");
  if (h->m.cplx) return fail(H2_EUNSUPPORTED, "the no-allocation matvec is real only");
  std::string err;
  h2_status st = h2::matvec_noalloc(h->m, h->d_user, x, y, nrhs, err);
  if (st != H2_OK) return fail(st, err);
  return H2_OK;
}

h2_status h2_to_dense(h2_handle h, double* out) {
  if (!h || !out) return fail(H2_EINVAL, "null argument");
  int64_t n = h->m.st->n;
  if (n > 16384) return fail(H2_EINVAL, "to_dense is for n <= 16384");
  return guarded([&] {
    double* eye = (double*)dmalloc(n * n * h->m.esize());
    cudaStream_t s = (cudaStream_t)h->m.stream;
    if (h->m.cplx)
      launch_zidentity(eye, n, s);
    else
      launch_identity(eye, n, s);
    cuda_check(cudaGetLastError(), "identity");
    h2_status st = h2_matvec(h, eye, out, n);
    cudaStreamSynchronize(s);
    cudaFree(eye);
    if (st != H2_OK) throw Error(st, g_err);
  });
}

h2_status h2_info(h2_handle h, h2_stats* s) {
  if (!h || !s) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    Mat& m = h->m;
    sync_ranks_to_host(m);
    const Structure& st = *m.st;
    std::memset(s, 0, sizeof(*s));
    s->n = st.n;
    s->levels = st.L + 1;
    s->leaf_size = st.LS;
    s->l_min = st.lmin;
    s->csp = st.csp;
    for (int l = 0; l <= st.L; ++l) s->n_admissible += st.nR[l];
    s->n_dense = st.nF;
    int64_t bytes = 0;
    for (int l = 0; l <= st.L && l < 32; ++l) {
      int mr = 0, mc = 0;
      for (int64_t t = 0; t < (1LL << l); ++t) {
        mr = std::max(mr, m.h_kr[Structure::node(l, t)]);
        mc = std::max(mc, m.h_kc[Structure::node(l, t)]);
      }
      s->max_rank_row[l] = mr;
      s->max_rank_col[l] = mc;
    }
    for (int l = 0; l <= st.L; ++l)
      for (auto& b : st.blocks[l]) {
        if (b.kind == KR) bytes += (int64_t)m.h_kr[Structure::node(l, b.t)] * m.h_kc[Structure::node(l, b.s)];
        if (b.kind == KF) bytes += st.size[st.L][b.t] * st.size[st.L][b.s];
      }
    for (int64_t t = 0; t < (1LL << st.L); ++t)
      bytes += st.size[st.L][t] * (int64_t)(m.h_kr[Structure::node(st.L, t)] + m.h_kc[Structure::node(st.L, t)]);
    for (int l = 0; l < st.L; ++l)
      for (int64_t t = 0; t < (1LL << l); ++t) {
        bytes += (int64_t)(m.h_kr[Structure::node(l + 1, 2 * t)] + m.h_kr[Structure::node(l + 1, 2 * t + 1)]) *
                 m.h_kr[Structure::node(l, t)];
        bytes += (int64_t)(m.h_kc[Structure::node(l + 1, 2 * t)] + m.h_kc[Structure::node(l + 1, 2 * t + 1)]) *
                 m.h_kc[Structure::node(l, t)];
      }
    s->bytes_stored = bytes * (int64_t)m.esize();
    s->device_bytes = m.arena_elems * (int64_t)m.esize();
    s->is_complex = m.cplx ? 1 : 0;
    if (m.d_cap) {
      unsigned long long c[3] = {0, 0, 0};
      cuda_check(cudaMemcpy(c, m.d_cap, sizeof(c), cudaMemcpyDeviceToHost), "counter");
      s->cap_hits = (int64_t)c[0];
      if (c[2]) throw Error(H2_ETIMEOUT, "a bounded wait of the tensor-core kernel gave up: the product is invalid");
    }
    if (h->timed) {
      float ms = 0;
      cuda_check(cudaEventSynchronize(h->ev1), "event");
      cuda_check(cudaEventElapsedTime(&ms, h->ev0, h->ev1), "event");
      s->mmp_ms = ms;
    }
  });
}

h2_status h2_tree_perm(h2_handle h, int64_t* perm) {
  if (!h || !perm) return fail(H2_EINVAL, "null argument");
  std::copy(h->m.st->perm.begin(), h->m.st->perm.end(), perm);
  return H2_OK;
}

h2_status h2_level_blocks(h2_handle h, int32_t level, int32_t* t, int32_t* s, int8_t* kind, int64_t* count) {
  if (!h || !count) return fail(H2_EINVAL, "null argument");
  const Structure& st = *h->m.st;
  if (level < 0 || level > st.L) return fail(H2_EINVAL, "level out of range");
  const auto& bl = st.blocks[level];
  *count = (int64_t)bl.size();
  if (t && s && kind)
    for (size_t p = 0; p < bl.size(); ++p) {
      t[p] = bl[p].t;
      s[p] = bl[p].s;
      kind[p] = bl[p].kind;
    }
  return H2_OK;
}

h2_status h2_trace_enable(h2_handle A, int32_t on) {
  if (!A) return fail(H2_EINVAL, "null argument");
  A->trace_on = on != 0;
  return H2_OK;
}

h2_status h2_trace_read(h2_handle C, int32_t cap, int32_t* kind, int32_t* level, double* ms, double* flops,
                        int32_t* count) {
  if (!C || !count) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    if (!C->trace_plan || !C->trace.recorded) throw Error(H2_EINVAL, "no traced product on this handle");
    const Plan& P = *C->trace_plan;
    cuda_check(cudaStreamSynchronize((cudaStream_t)C->m.stream), "synchronise");
    int32_t n = (int32_t)P.launches.size();
    *count = n;
    for (int32_t i = 0; i < n && i < cap; ++i) {
      const Launch& L = P.launches[i];
      float t = 0;
      cuda_check(cudaEventElapsedTime(&t, (cudaEvent_t)C->trace.ev[2 * i], (cudaEvent_t)C->trace.ev[2 * i + 1]), "event");
      if (kind) kind[i] = L.kind == Launch::GEMM ? (L.tc ? 3 : 0) : (L.kind == Launch::EIG ? 1 : 2);
      if (level) level[i] = L.level;
      if (ms) ms[i] = t;
      if (flops) flops[i] = L.kind == Launch::EIG ? (double)L.count : L.flops;
    }
  });
}

h2_status h2_kernel_launches(uint64_t* count) {
  if (!count) return fail(H2_EINVAL, "null argument");
  *count = (uint64_t)kernel_launches();
  return H2_OK;
}

h2_status h2_trace_flops(h2_handle C, double* executed) {
  if (!C || !executed) return fail(H2_EINVAL, "null argument");
  return guarded([&] {
    unsigned long long v = 0;
    cuda_check(cudaStreamSynchronize((cudaStream_t)C->m.stream), "synchronise");
    cuda_check(cudaMemcpy(&v, C->m.d_cap + 1, sizeof(v), cudaMemcpyDeviceToHost), "flop counter");
    *executed = (double)v;
  });
}

const char* h2_trace_phase(h2_handle C, int32_t i) {
  if (!C || !C->trace_plan || i < 0 || i >= (int32_t)C->trace_plan->launches.size()) return nullptr;
  return C->trace_plan->launches[i].phase;
}

void h2_destroy(h2_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  delete h;  // the handle's destructor frees what it owns; held plans go with it
}

}  // extern "C"
