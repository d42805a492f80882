// H^2 construction on the host (the step before the product).
//
// The paper builds its inputs with a method it cites but does not describe; this
// library reads it as nested far-field compression with sampling, so that an
// N = 1M build stays linear:
//   * far(t): for t and each ancestor, every admissible partner s, sampled with at
//     most `kSamples` points spread evenly over s in tree order;
//   * leaf t: V_t = dominant left singular vectors of K(t, far(t)) (eigenvectors
//     of the Gram matrix with lambda / lambda_1 > eps^2, i.e. sigma/sigma_1 > eps);
//   * non-leaf t: the stacked transfer E_t = dominant left singular vectors of
//     [Q_t1 K(I_t1, far(t)); Q_t2 K(I_t2, far(t))], where I_c are skeleton rows of
//     child c and Q_c = pinv(V_c[I_c, :]) maps samples on I_c to coefficients in
//     V_c (exact, Q_c = V_c^T, while a cluster has at most kAllRows points);
//   * skeleton rows of t: all rows while |t| <= kAllRows, else k_t + kOver rows
//     chosen from I_t1 u I_t2 by greedy pivoted Gram-Schmidt on V_t's rows;
//   * couplings S_ts = Q_t K(I_t, I_s) Q_s^T; dense blocks K(t, s);
//   * the real kernels are symmetric and so is the partition: the column bases
//     equal the row bases.
// Output is the packed layout of h2_import.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.hpp"

namespace h2 {

namespace {

constexpr int kSamples = 24;
constexpr int kAllRows = 64;
constexpr int kOver = 8;
constexpr int kMaxRank = 64;

struct KernelEval {
  h2_kernel k;
  const double* p;
  double operator()(int64_t a, int64_t b) const {
    if (a == b) return k.diag_re;
    double dx = p[3 * a] - p[3 * b], dy = p[3 * a + 1] - p[3 * b + 1], dz = p[3 * a + 2] - p[3 * b + 2];
    double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    if (r == 0.0) return k.diag_re;
    if (k.kind == H2_K_LAPLACE) return 1.0 / (4.0 * M_PI * r);
    return 1.0 / (r * r);
  }
};

// cyclic Jacobi for a symmetric n x n (row-major), eigenvalues descending
void jacobi_eig(std::vector<double> a, int n, std::vector<double>& lam, std::vector<double>& v) {
  v.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double x = a[(size_t)i * n + j] * a[(size_t)i * n + j];
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot || tot == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        double app = a[(size_t)p * n + p], aqq = a[(size_t)q * n + q];
        double tau = (aqq - app) / (2.0 * apq);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int j = 0; j < n; ++j) {
          double x = a[(size_t)p * n + j], y = a[(size_t)q * n + j];
          a[(size_t)p * n + j] = c * x - s * y;
          a[(size_t)q * n + j] = s * x + c * y;
        }
        for (int i = 0; i < n; ++i) {
          double x = a[(size_t)i * n + p], y = a[(size_t)i * n + q];
          a[(size_t)i * n + p] = c * x - s * y;
          a[(size_t)i * n + q] = s * x + c * y;
          double vx = v[(size_t)i * n + p], vy = v[(size_t)i * n + q];
          v[(size_t)i * n + p] = c * vx - s * vy;
          v[(size_t)i * n + q] = s * vx + c * vy;
        }
      }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return a[(size_t)x * n + x] > a[(size_t)y * n + y]; });
  lam.resize(n);
  std::vector<double> vs((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    lam[c] = a[(size_t)idx[c] * n + idx[c]];
    for (int r = 0; r < n; ++r) vs[(size_t)r * n + c] = v[(size_t)r * n + idx[c]];
  }
  v.swap(vs);
}

// dominant left singular vectors of W (m x ncol, row-major): returns m x k basis
std::vector<double> dominant_basis(const std::vector<double>& w, int m, int64_t ncol, double eps, int& k) {
  std::vector<double> g((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      const double* a = &w[(size_t)i * ncol];
      const double* b = &w[(size_t)j * ncol];
      double acc = 0;
      for (int64_t c = 0; c < ncol; ++c) acc += a[c] * b[c];
      g[(size_t)i * m + j] = g[(size_t)j * m + i] = acc;
    }
  std::vector<double> lam, v;
  jacobi_eig(g, m, lam, v);
  k = 0;
  if (m > 0 && lam[0] > 0)
    while (k < m && k < kMaxRank && lam[k] > eps * eps * lam[0]) ++k;
  std::vector<double> out((size_t)m * k);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < k; ++c) out[(size_t)r * k + c] = v[(size_t)r * m + c];
  return out;
}

// pinv of R (p x k, p >= k) via the eigen-decomposition of R^T R
std::vector<double> pinv(const std::vector<double>& R, int p, int k) {
  std::vector<double> g((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double acc = 0;
      for (int r = 0; r < p; ++r) acc += R[(size_t)r * k + i] * R[(size_t)r * k + j];
      g[(size_t)i * k + j] = acc;
    }
  std::vector<double> lam, u;
  jacobi_eig(g, k, lam, u);
  std::vector<double> out((size_t)k * p, 0.0);  // U diag(1/lam) U^T R^T
  std::vector<double> tmp((size_t)k * k, 0.0);
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      double acc = 0;
      for (int c = 0; c < k; ++c)
        if (lam[c] > 1e-14 * lam[0]) acc += u[(size_t)i * k + c] * u[(size_t)j * k + c] / lam[c];
      tmp[(size_t)i * k + j] = acc;
    }
  for (int i = 0; i < k; ++i)
    for (int r = 0; r < p; ++r) {
      double acc = 0;
      for (int j = 0; j < k; ++j) acc += tmp[(size_t)i * k + j] * R[(size_t)r * k + j];
      out[(size_t)i * p + r] = acc;
    }
  return out;
}

// greedy pivoted Gram-Schmidt on the rows of R (m x k): returns chosen row positions
std::vector<int> pick_rows(std::vector<double> R, int m, int k, int want) {
  std::vector<int> chosen;
  std::vector<char> used(m, 0);
  std::vector<double> nrm(m);
  for (int i = 0; i < m; ++i) {
    double acc = 0;
    for (int c = 0; c < k; ++c) acc += R[(size_t)i * k + c] * R[(size_t)i * k + c];
    nrm[i] = acc;
  }
  want = std::min(want, m);
  for (int step = 0; step < want; ++step) {
    int best = -1;
    for (int i = 0; i < m; ++i)
      if (!used[i] && (best < 0 || nrm[i] > nrm[best])) best = i;
    used[best] = 1;
    chosen.push_back(best);
    double nb = std::sqrt(nrm[best]);
    if (nb > 0) {
      std::vector<double> q(k);
      for (int c = 0; c < k; ++c) q[c] = R[(size_t)best * k + c] / nb;
      for (int i = 0; i < m; ++i) {
        if (used[i]) continue;
        double d = 0;
        for (int c = 0; c < k; ++c) d += R[(size_t)i * k + c] * q[c];
        double acc = 0;
        for (int c = 0; c < k; ++c) {
          R[(size_t)i * k + c] -= d * q[c];
          acc += R[(size_t)i * k + c] * R[(size_t)i * k + c];
        }
        nrm[i] = acc;
      }
    }
  }
  std::sort(chosen.begin(), chosen.end());
  return chosen;
}

struct ClusterData {
  std::vector<double> basis;  // leaf: |t| x k ; non-leaf: (k1 + k2) x k
  int k = 0;
  std::vector<int64_t> skel;  // skeleton rows (tree positions)
  std::vector<double> rows;   // V_t[skel, :]  (|skel| x k)
  std::vector<double> Q;      // pinv(rows)    (k x |skel|)
};

}  // namespace

void build_h2_host(const Structure& st, const h2_kernel& kern, double eps, Packed& out) {
  if (kern.kind != H2_K_LAPLACE && kern.kind != H2_K_INV_R2)
    throw Error(H2_EUNSUPPORTED, "complex kernels are not supported on the GPU path");
  const int L = st.L;
  KernelEval K{kern, st.pts.data()};
  std::vector<std::vector<ClusterData>> cd(L + 1);
  // admissible partners per level, by row cluster
  std::vector<std::vector<std::vector<int32_t>>> partners(L + 1);
  for (int l = 0; l <= L; ++l) {
    partners[l].assign(1LL << l, {});
    for (auto& b : st.blocks[l])
      if (b.kind == KR) partners[l][b.t].push_back(b.s);
  }
  auto sample = [&](int lv, int32_t s, std::vector<int64_t>& cols) {
    int64_t s0 = st.start[lv][s], m = st.size[lv][s];
    if (m <= kSamples) {
      for (int64_t q = 0; q < m; ++q) cols.push_back(s0 + q);
    } else {
      for (int q = 0; q < kSamples; ++q) cols.push_back(s0 + (int64_t)((q + 0.5) * (double)m / kSamples));
    }
  };
  for (int l = L; l >= 0; --l) {
    int64_t nc = 1LL << l;
    cd[l].resize(nc);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nc; ++t) {
      std::vector<int64_t> far;
      for (int lv = l; lv >= 0; --lv)
        for (int32_t s : partners[lv][t >> (l - lv)]) sample(lv, s, far);
      ClusterData& c = cd[l][t];
      int64_t ncol = (int64_t)far.size();
      if (l == L) {
        int m = (int)st.size[L][t];
        int64_t s0 = st.start[L][t];
        std::vector<double> w((size_t)m * ncol);
        for (int r = 0; r < m; ++r)
          for (int64_t q = 0; q < ncol; ++q) w[(size_t)r * ncol + q] = K(s0 + r, far[q]);
        c.basis = ncol ? dominant_basis(w, m, ncol, eps, c.k) : std::vector<double>();
        if (!ncol) c.k = 0;
        c.skel.resize(m);
        for (int r = 0; r < m; ++r) c.skel[r] = s0 + r;
        c.rows = c.basis;
        c.Q.assign((size_t)c.k * m, 0.0);
        for (int i = 0; i < c.k; ++i)
          for (int r = 0; r < m; ++r) c.Q[(size_t)i * m + r] = c.basis[(size_t)r * c.k + i];
      } else {
        const ClusterData& c1 = cd[l + 1][2 * t];
        const ClusterData& c2 = cd[l + 1][2 * t + 1];
        int k1 = c1.k, k2 = c2.k, m = k1 + k2;
        std::vector<double> w((size_t)m * ncol, 0.0);
        for (int part = 0; part < 2; ++part) {
          const ClusterData& ch = part ? c2 : c1;
          int kc = ch.k, ns = (int)ch.skel.size(), roff = part ? k1 : 0;
          std::vector<double> ks((size_t)ns * ncol);
          for (int r = 0; r < ns; ++r)
            for (int64_t q = 0; q < ncol; ++q) ks[(size_t)r * ncol + q] = K(ch.skel[r], far[q]);
          for (int i = 0; i < kc; ++i)
            for (int r = 0; r < ns; ++r) {
              double qv = ch.Q[(size_t)i * ns + r];
              if (qv == 0.0) continue;
              double* dst = &w[(size_t)(roff + i) * ncol];
              const double* src = &ks[(size_t)r * ncol];
              for (int64_t q = 0; q < ncol; ++q) dst[q] += qv * src[q];
            }
        }
        c.basis = (ncol && m) ? dominant_basis(w, m, ncol, eps, c.k) : std::vector<double>();
        if (!ncol || !m) c.k = 0;
        // rows of V_t at the candidate rows I_t1 u I_t2
        int n1 = (int)c1.skel.size(), n2 = (int)c2.skel.size(), nc2 = n1 + n2;
        std::vector<double> vc((size_t)nc2 * c.k, 0.0);
        for (int r = 0; r < n1; ++r)
          for (int j = 0; j < c.k; ++j) {
            double acc = 0;
            for (int i = 0; i < k1; ++i) acc += c1.rows[(size_t)r * k1 + i] * c.basis[(size_t)i * c.k + j];
            vc[(size_t)r * c.k + j] = acc;
          }
        for (int r = 0; r < n2; ++r)
          for (int j = 0; j < c.k; ++j) {
            double acc = 0;
            for (int i = 0; i < k2; ++i) acc += c2.rows[(size_t)r * k2 + i] * c.basis[(size_t)(k1 + i) * c.k + j];
            vc[(size_t)(n1 + r) * c.k + j] = acc;
          }
        std::vector<int64_t> cand(c1.skel);
        cand.insert(cand.end(), c2.skel.begin(), c2.skel.end());
        std::vector<int> pick;
        if (st.size[l][t] <= kAllRows || nc2 <= c.k + kOver) {
          pick.resize(nc2);
          std::iota(pick.begin(), pick.end(), 0);
        } else {
          pick = pick_rows(vc, nc2, c.k, c.k + kOver);
        }
        int p = (int)pick.size();
        c.skel.resize(p);
        c.rows.assign((size_t)p * c.k, 0.0);
        for (int r = 0; r < p; ++r) {
          c.skel[r] = cand[pick[r]];
          for (int j = 0; j < c.k; ++j) c.rows[(size_t)r * c.k + j] = vc[(size_t)pick[r] * c.k + j];
        }
        c.Q = c.k ? pinv(c.rows, p, c.k) : std::vector<double>();
      }
    }
  }
  // packed output
  const int nn = st.nnodes();
  out.kr.assign(nn, 0);
  for (int l = 0; l <= L; ++l)
    for (int64_t t = 0; t < (1LL << l); ++t) out.kr[Structure::node(l, t)] = cd[l][t].k;
  out.kc = out.kr;
  out.vr.clear();
  for (int64_t t = 0; t < (1LL << L); ++t) out.vr.insert(out.vr.end(), cd[L][t].basis.begin(), cd[L][t].basis.end());
  out.vc = out.vr;
  out.er.clear();
  for (int l = 0; l < L; ++l)
    for (int64_t t = 0; t < (1LL << l); ++t) out.er.insert(out.er.end(), cd[l][t].basis.begin(), cd[l][t].basis.end());
  out.ec = out.er;
  // couplings, ordered by level then (t, s)
  std::vector<int64_t> soff(L + 2, 0);
  std::vector<std::vector<int64_t>> boff(L + 1);
  int64_t total = 0;
  for (int l = 0; l <= L; ++l) {
    for (auto& b : st.blocks[l])
      if (b.kind == KR) {
        boff[l].push_back(total);
        total += (int64_t)cd[l][b.t].k * cd[l][b.s].k;
      }
  }
  out.s.assign(total, 0.0);
  for (int l = 0; l <= L; ++l) {
    std::vector<const Block*> rb;
    for (auto& b : st.blocks[l])
      if (b.kind == KR) rb.push_back(&b);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < (int64_t)rb.size(); ++q) {
      const Block& b = *rb[q];
      const ClusterData &ct = cd[l][b.t], &cs = cd[l][b.s];
      int kt = ct.k, ks = cs.k, nt = (int)ct.skel.size(), ns = (int)cs.skel.size();
      if (!kt || !ks) continue;
      std::vector<double> kts((size_t)nt * ns);
      for (int i = 0; i < nt; ++i)
        for (int j = 0; j < ns; ++j) kts[(size_t)i * ns + j] = K(ct.skel[i], cs.skel[j]);
      std::vector<double> tmp((size_t)kt * ns, 0.0);  // Q_t K
      for (int a = 0; a < kt; ++a)
        for (int i = 0; i < nt; ++i) {
          double qv = ct.Q[(size_t)a * nt + i];
          for (int j = 0; j < ns; ++j) tmp[(size_t)a * ns + j] += qv * kts[(size_t)i * ns + j];
        }
      double* dst = &out.s[boff[l][b.idx]];
      for (int a = 0; a < kt; ++a)
        for (int c = 0; c < ks; ++c) {
          double acc = 0;
          for (int j = 0; j < ns; ++j) acc += tmp[(size_t)a * ns + j] * cs.Q[(size_t)c * ns + j];
          dst[(size_t)a * ks + c] = acc;
        }
    }
  }
  // dense leaf blocks, ordered by (t, s)
  std::vector<const Block*> fb;
  for (auto& b : st.blocks[L])
    if (b.kind == KF) fb.push_back(&b);
  std::vector<int64_t> foff(fb.size() + 1, 0);
  for (size_t q = 0; q < fb.size(); ++q) foff[q + 1] = foff[q] + st.size[L][fb[q]->t] * st.size[L][fb[q]->s];
  out.f.assign(foff.back(), 0.0);
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < (int64_t)fb.size(); ++q) {
    const Block& b = *fb[q];
    int64_t t0 = st.start[L][b.t], s0 = st.start[L][b.s], mt = st.size[L][b.t], ms = st.size[L][b.s];
    double* dst = &out.f[foff[q]];
    for (int64_t i = 0; i < mt; ++i)
      for (int64_t j = 0; j < ms; ++j) dst[i * ms + j] = K(t0 + i, s0 + j);
  }
}

}  // namespace h2
