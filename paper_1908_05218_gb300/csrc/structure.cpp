// Cluster tree and block partition (Sec. II, Eq. admCond), host side.
//
// The tree is a complete binary tree built by cardinality-balanced bisection: a
// cluster's points are sorted along the longest side of its bounding box (ties of
// the coordinate broken by the user index) and the first (n+1)/2 points form the
// first child.  L is the smallest level with at most leaf_size points per cluster.
// A block (t, s) is admissible when max(diam_t, diam_s) <= eta * dist(t, s) with
// box diagonals and box distance, compared squared, and dist > 0.  Non-admissible
// blocks are dense (F) on the leaf level and subdivided (NL) above it.
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <parallel/algorithm>

#include "internal.hpp"

namespace h2 {

static double diam2(const std::array<double, 3>& lo, const std::array<double, 3>& hi) {
  double d0 = hi[0] - lo[0], d1 = hi[1] - lo[1], d2 = hi[2] - lo[2];
  return d0 * d0 + d1 * d1 + d2 * d2;
}

static double dist2(const std::array<double, 3>& lt, const std::array<double, 3>& ht,
                    const std::array<double, 3>& ls, const std::array<double, 3>& hs) {
  double acc = 0.0;
  for (int d = 0; d < 3; ++d) {
    double g = std::max(0.0, std::max(ls[d] - ht[d], lt[d] - hs[d]));
    acc = acc + g * g;
  }
  return acc;
}

std::shared_ptr<Structure> build_structure(const double* up, int64_t n, int leaf_size,
                                           double eta) {
  if (n < 1 || leaf_size < 1 || leaf_size > 64 || !(eta > 0)) throw Error(H2_EINVAL, "bad n, leaf_size or eta");
  for (int64_t i = 0; i < 3 * n; ++i)
    if (!std::isfinite(up[i])) throw Error(H2_EINVAL, "non-finite point coordinate");
  auto st = std::make_shared<Structure>();
  st->n = n;
  st->leaf_size = leaf_size;
  st->eta = eta;
  int L = 0;
  while ((n + (1LL << L) - 1) / (1LL << L) > leaf_size) ++L;
  if (L > 30) throw Error(H2_EINVAL, "tree too deep");
  st->L = L;
  std::vector<int64_t>& perm = st->perm;
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  st->start.assign(L + 1, {});
  st->size.assign(L + 1, {});
  st->start[0] = {0};
  st->size[0] = {n};
  // The clusters of a level are split in parallel; on the top levels, which have fewer
  // clusters than threads, each sort runs on all threads instead.  The order (coordinate,
  // then user index) is total, so every sort has one result whatever the threads.
  const int nthr = omp_get_max_threads();
  for (int l = 0; l < L; ++l) {
    auto& ns = st->start[l + 1];
    auto& nz = st->size[l + 1];
    ns.resize(2LL << l);
    nz.resize(2LL << l);
    const bool wide = (1LL << l) < nthr;
#pragma omp parallel for schedule(dynamic, 1) if (!wide)
    for (int64_t t = 0; t < (1LL << l); ++t) {
      int64_t s0 = st->start[l][t], m = st->size[l][t];
      std::array<double, 3> lo{INFINITY, INFINITY, INFINITY}, hi{-INFINITY, -INFINITY, -INFINITY};
      for (int64_t p = s0; p < s0 + m; ++p)
        for (int d = 0; d < 3; ++d) {
          double v = up[3 * perm[p] + d];
          lo[d] = std::min(lo[d], v);
          hi[d] = std::max(hi[d], v);
        }
      int axis = 0;
      for (int d = 1; d < 3; ++d)
        if (hi[d] - lo[d] > hi[axis] - lo[axis]) axis = d;
      auto before = [&](int64_t a, int64_t b) {
        double va = up[3 * a + axis], vb = up[3 * b + axis];
        if (va != vb) return va < vb;
        return a < b;
      };
      if (wide && m >= (1 << 16))
        __gnu_parallel::sort(perm.begin() + s0, perm.begin() + s0 + m, before);
      else
        std::sort(perm.begin() + s0, perm.begin() + s0 + m, before);
      int64_t m1 = (m + 1) / 2;
      ns[2 * t] = s0;
      nz[2 * t] = m1;
      ns[2 * t + 1] = s0 + m1;
      nz[2 * t + 1] = m - m1;
    }
  }
  st->pts.resize(3 * n);
  for (int64_t p = 0; p < n; ++p)
    for (int d = 0; d < 3; ++d) st->pts[3 * p + d] = up[3 * perm[p] + d];
  st->lo.assign(L + 1, {});
  st->hi.assign(L + 1, {});
  for (int l = L; l >= 0; --l) {
    int64_t nc = 1LL << l;
    st->lo[l].resize(nc);
    st->hi[l].resize(nc);
    for (int64_t t = 0; t < nc; ++t) {
      std::array<double, 3> lo{INFINITY, INFINITY, INFINITY}, hi{-INFINITY, -INFINITY, -INFINITY};
      if (l == L) {
        for (int64_t p = st->start[l][t]; p < st->start[l][t] + st->size[l][t]; ++p)
          for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], st->pts[3 * p + d]);
            hi[d] = std::max(hi[d], st->pts[3 * p + d]);
          }
      } else {
        for (int c = 0; c < 2; ++c)
          for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], st->lo[l + 1][2 * t + c][d]);
            hi[d] = std::max(hi[d], st->hi[l + 1][2 * t + c][d]);
          }
      }
      st->lo[l][t] = lo;
      st->hi[l][t] = hi;
    }
  }
  int64_t LS = 0;
  for (auto z : st->size[L]) LS = std::max(LS, z);
  st->LS = (int)LS;

  // block partition, level by level, candidates sorted by (t, s)
  st->blocks.assign(L + 1, {});
  st->nR.assign(L + 1, 0);
  std::vector<std::pair<int64_t, int64_t>> cand{{0, 0}};
  const double eta2 = eta * eta;
  for (int l = 0; l <= L; ++l) {
    std::sort(cand.begin(), cand.end());
    std::vector<std::pair<int64_t, int64_t>> next;
    auto& bl = st->blocks[l];
    bl.reserve(cand.size());
    for (auto& c : cand) {
      int64_t t = c.first, s = c.second;
      double dd = dist2(st->lo[l][t], st->hi[l][t], st->lo[l][s], st->hi[l][s]);
      bool adm = false;
      if (dd > 0.0) {
        double dt = diam2(st->lo[l][t], st->hi[l][t]), ds = diam2(st->lo[l][s], st->hi[l][s]);
        adm = std::max(dt, ds) <= eta2 * dd;
      }
      Block b{(int32_t)t, (int32_t)s, KNL, -1};
      if (adm) {
        b.kind = KR;
        b.idx = st->nR[l]++;
      } else if (l == L) {
        b.kind = KF;
        b.idx = st->nF++;
      } else {
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) next.push_back({2 * t + a, 2 * s + bb});
      }
      bl.push_back(b);
    }
    cand.swap(next);
  }
  st->row_ptr.assign(L + 1, {});
  st->col_ptr.assign(L + 1, {});
  st->col_list.assign(L + 1, {});
  st->lmin = L;
  st->csp = 0;
  for (int l = L; l >= 0; --l) {
    auto& bl = st->blocks[l];
    int64_t nc = 1LL << l;
    auto& rp = st->row_ptr[l];
    rp.assign(nc + 1, 0);
    std::vector<int32_t> ccount(nc + 1, 0);
    for (size_t p = 0; p < bl.size(); ++p) {
      rp[bl[p].t + 1]++;
      ccount[bl[p].s + 1]++;
      if (bl[p].kind == KR) st->lmin = std::min(st->lmin, l);
    }
    for (int64_t t = 0; t < nc; ++t) {
      st->csp = std::max(st->csp, std::max(rp[t + 1], ccount[t + 1]));
      rp[t + 1] += rp[t];
      ccount[t + 1] += ccount[t];
    }
    st->col_ptr[l] = ccount;
    st->col_list[l].resize(bl.size());
    std::vector<int32_t> fill(ccount.begin(), ccount.end() - 1);
    for (size_t p = 0; p < bl.size(); ++p) st->col_list[l][fill[bl[p].s]++] = (int32_t)p;
  }
  return st;
}

bool same_structure(const Structure& a, const Structure& b) {
  if (&a == &b) return true;
  if (a.n != b.n || a.L != b.L || a.perm != b.perm) return false;
  for (int l = 0; l <= a.L; ++l) {
    if (a.blocks[l].size() != b.blocks[l].size()) return false;
    for (size_t p = 0; p < a.blocks[l].size(); ++p) {
      const Block &x = a.blocks[l][p], &y = b.blocks[l][p];
      if (x.t != y.t || x.s != y.s || x.kind != y.kind) return false;
    }
  }
  return true;
}

}  // namespace h2
