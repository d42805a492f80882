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
//   * the kernels are symmetric (K(x, y) = K(y, x), also the complex Helmholtz kernel)
//     and so is the partition: the column bases equal the row bases (R = V S V^T).
// Complex kernels use the same steps with Hermitian Gram matrices (W W^H), a Hermitian
// Jacobi, conjugated inner products in the row selection and pinv(R) = (R^H R)^-1 R^H.
// Output is the packed layout of h2_import (complex: real and imaginary part per element).
#include <algorithm>
#include <cmath>
#include <complex>
#include <numeric>
#include <type_traits>

#include "internal.hpp"

namespace h2 {

namespace {

// far-field points read per partner block: 24 suffice for the smooth real kernels; the
// oscillatory Helmholtz kernel needs more (its far-field ranks grow with the electrical
// size of the blocks)
constexpr int kSamplesReal = kBuildSamples, kSamplesComplex = 128;
constexpr int kAllRows = kBuildAllRows;
constexpr int kOver = kBuildOver;
constexpr int kMaxRank = kBuildMaxRank;

using cd = std::complex<double>;
inline double cj(double x) { return x; }
inline cd cj(cd x) { return std::conj(x); }
inline double re(double x) { return x; }
inline double re(cd x) { return x.real(); }
inline double abs2(double x) { return x * x; }
inline double abs2(cd x) { return x.real() * x.real() + x.imag() * x.imag(); }

template <typename T>
struct KernelEval {
  h2_kernel k;
  const double* p;
  T diag() const;
  T far(double r) const;
  T operator()(int64_t a, int64_t b) const {
    if (a == b) return diag();
    double dx = p[3 * a] - p[3 * b], dy = p[3 * a + 1] - p[3 * b + 1], dz = p[3 * a + 2] - p[3 * b + 2];
    double r = std::sqrt(dx * dx + dy * dy + dz * dz);
    if (r == 0.0) return diag();
    return far(r);
  }
};
template <>
double KernelEval<double>::diag() const { return k.diag_re; }
template <>
double KernelEval<double>::far(double r) const {
  if (k.kind == H2_K_LAPLACE) return 1.0 / (4.0 * M_PI * r);
  return 1.0 / (r * r);
}
template <>
cd KernelEval<cd>::diag() const { return cd(k.diag_re, k.diag_im); }
template <>
cd KernelEval<cd>::far(double r) const {  // exp(-j k r) / (4 pi r)
  const double ph = -k.wavenumber * r, sc = 1.0 / (4.0 * M_PI * r);
  return cd(std::cos(ph) * sc, std::sin(ph) * sc);
}

// cyclic Jacobi for a Hermitian n x n (row-major), eigenvalues descending.  A complex
// pair (p, q) with a_pq = |a_pq| e^{i phi} is rotated by U = diag(1, e^{-i phi}) R, R the
// real rotation of |a_pq| (for real matrices U = R, the symmetric Schur rotation).
template <typename T>
void jacobi_eig(std::vector<T> a, int n, std::vector<double>& lam, std::vector<T>& v) {
  v.assign((size_t)n * n, T(0));
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = T(1);
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0, tot = 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double x = abs2(a[(size_t)i * n + j]);
        tot += x;
        if (i != j) off += x;
      }
    if (off <= 1e-30 * tot || tot == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const T apq = a[(size_t)p * n + q];
        if (apq == T(0)) continue;
        const double mag = std::sqrt(abs2(apq));
        const T e = apq / mag;  // e^{i phi} (real: the sign of a_pq)
        double app = re(a[(size_t)p * n + p]), aqq = re(a[(size_t)q * n + q]);
        double tau = (aqq - app) / (2.0 * mag);
        double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int j = 0; j < n; ++j) {
          T x = a[(size_t)p * n + j], y = e * a[(size_t)q * n + j];
          a[(size_t)p * n + j] = c * x - s * y;
          a[(size_t)q * n + j] = s * x + c * y;
        }
        const T ec = cj(e);
        for (int i = 0; i < n; ++i) {
          T x = a[(size_t)i * n + p], y = ec * a[(size_t)i * n + q];
          a[(size_t)i * n + p] = c * x - s * y;
          a[(size_t)i * n + q] = s * x + c * y;
          T vx = v[(size_t)i * n + p], vy = ec * v[(size_t)i * n + q];
          v[(size_t)i * n + p] = c * vx - s * vy;
          v[(size_t)i * n + q] = s * vx + c * vy;
        }
      }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int x, int y) { return re(a[(size_t)x * n + x]) > re(a[(size_t)y * n + y]); });
  lam.resize(n);
  std::vector<T> vs((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    lam[c] = re(a[(size_t)idx[c] * n + idx[c]]);
    for (int r = 0; r < n; ++r) vs[(size_t)r * n + c] = v[(size_t)r * n + idx[c]];
  }
  v.swap(vs);
}

// dominant left singular vectors of W (m x ncol, row-major): returns m x k basis
template <typename T>
std::vector<T> dominant_basis(const std::vector<T>& w, int m, int64_t ncol, double eps, int& k) {
  std::vector<T> g((size_t)m * m, T(0));
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      const T* a = &w[(size_t)i * ncol];
      const T* b = &w[(size_t)j * ncol];
      T acc = 0;
      for (int64_t c = 0; c < ncol; ++c) acc += a[c] * cj(b[c]);
      g[(size_t)i * m + j] = acc;
      g[(size_t)j * m + i] = cj(acc);
    }
  std::vector<double> lam;
  std::vector<T> v;
  jacobi_eig(g, m, lam, v);
  k = 0;
  if (m > 0 && lam[0] > 0)
    while (k < m && k < kMaxRank && lam[k] > eps * eps * lam[0]) ++k;
  std::vector<T> out((size_t)m * k);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < k; ++c) out[(size_t)r * k + c] = v[(size_t)r * m + c];
  return out;
}

// pinv of R (p x k, p >= k) via the eigen-decomposition of R^H R
template <typename T>
std::vector<T> pinv(const std::vector<T>& R, int p, int k) {
  std::vector<T> g((size_t)k * k, T(0));
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      T acc = 0;
      for (int r = 0; r < p; ++r) acc += cj(R[(size_t)r * k + i]) * R[(size_t)r * k + j];
      g[(size_t)i * k + j] = acc;
    }
  std::vector<double> lam;
  std::vector<T> u;
  jacobi_eig(g, k, lam, u);
  std::vector<T> out((size_t)k * p, T(0));  // U diag(1/lam) U^H R^H
  std::vector<T> tmp((size_t)k * k, T(0));
  for (int i = 0; i < k; ++i)
    for (int j = 0; j < k; ++j) {
      T acc = 0;
      for (int c = 0; c < k; ++c)
        if (lam[c] > 1e-14 * lam[0]) acc += u[(size_t)i * k + c] * cj(u[(size_t)j * k + c]) / lam[c];
      tmp[(size_t)i * k + j] = acc;
    }
  for (int i = 0; i < k; ++i)
    for (int r = 0; r < p; ++r) {
      T acc = 0;
      for (int j = 0; j < k; ++j) acc += tmp[(size_t)i * k + j] * cj(R[(size_t)r * k + j]);
      out[(size_t)i * p + r] = acc;
    }
  return out;
}

// greedy pivoted Gram-Schmidt on the rows of R (m x k): returns chosen row positions
template <typename T>
std::vector<int> pick_rows(std::vector<T> R, int m, int k, int want) {
  std::vector<int> chosen;
  std::vector<char> used(m, 0);
  std::vector<double> nrm(m);
  for (int i = 0; i < m; ++i) {
    double acc = 0;
    for (int c = 0; c < k; ++c) acc += abs2(R[(size_t)i * k + c]);
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
      std::vector<T> q(k);
      for (int c = 0; c < k; ++c) q[c] = R[(size_t)best * k + c] / nb;
      for (int i = 0; i < m; ++i) {
        if (used[i]) continue;
        T d = 0;
        for (int c = 0; c < k; ++c) d += R[(size_t)i * k + c] * cj(q[c]);
        double acc = 0;
        for (int c = 0; c < k; ++c) {
          R[(size_t)i * k + c] -= d * q[c];
          acc += abs2(R[(size_t)i * k + c]);
        }
        nrm[i] = acc;
      }
    }
  }
  std::sort(chosen.begin(), chosen.end());
  return chosen;
}

template <typename T>
struct ClusterData {
  std::vector<T> basis;       // leaf: |t| x k ; non-leaf: (k1 + k2) x k
  int k = 0;
  std::vector<int64_t> skel;  // skeleton rows (tree positions)
  std::vector<T> rows;        // V_t[skel, :]  (|skel| x k)
  std::vector<T> Q;           // pinv(rows)    (k x |skel|)
};

// appends the values of a real or complex array to a packed double array
void put(std::vector<double>& dst, const std::vector<double>& src) { dst.insert(dst.end(), src.begin(), src.end()); }
void put(std::vector<double>& dst, const std::vector<cd>& src) {
  for (const cd& z : src) {
    dst.push_back(z.real());
    dst.push_back(z.imag());
  }
}

template <typename T>
void build_typed(const Structure& st, const h2_kernel& kern, double eps, Packed& out) {
  const int L = st.L;
  KernelEval<T> K{kern, st.pts.data()};
  std::vector<std::vector<ClusterData<T>>> cd(L + 1);
  // admissible partners per level, by row cluster
  std::vector<std::vector<std::vector<int32_t>>> partners(L + 1);
  for (int l = 0; l <= L; ++l) {
    partners[l].assign(1LL << l, {});
    for (auto& b : st.blocks[l])
      if (b.kind == KR) partners[l][b.t].push_back(b.s);
  }
  const int kSamples = std::is_same<T, double>::value ? kSamplesReal : kSamplesComplex;
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
      ClusterData<T>& c = cd[l][t];
      int64_t ncol = (int64_t)far.size();
      if (l == L) {
        int m = (int)st.size[L][t];
        int64_t s0 = st.start[L][t];
        std::vector<T> w((size_t)m * ncol);
        for (int r = 0; r < m; ++r)
          for (int64_t q = 0; q < ncol; ++q) w[(size_t)r * ncol + q] = K(s0 + r, far[q]);
        c.basis = ncol ? dominant_basis(w, m, ncol, eps, c.k) : std::vector<T>();
        if (!ncol) c.k = 0;
        c.skel.resize(m);
        for (int r = 0; r < m; ++r) c.skel[r] = s0 + r;
        c.rows = c.basis;
        c.Q.assign((size_t)c.k * m, T(0));  // V^H (orthonormal V)
        for (int i = 0; i < c.k; ++i)
          for (int r = 0; r < m; ++r) c.Q[(size_t)i * m + r] = cj(c.basis[(size_t)r * c.k + i]);
      } else {
        const ClusterData<T>& c1 = cd[l + 1][2 * t];
        const ClusterData<T>& c2 = cd[l + 1][2 * t + 1];
        int k1 = c1.k, k2 = c2.k, m = k1 + k2;
        std::vector<T> w((size_t)m * ncol, T(0));
        for (int part = 0; part < 2; ++part) {
          const ClusterData<T>& ch = part ? c2 : c1;
          int kc = ch.k, ns = (int)ch.skel.size(), roff = part ? k1 : 0;
          std::vector<T> ks((size_t)ns * ncol);
          for (int r = 0; r < ns; ++r)
            for (int64_t q = 0; q < ncol; ++q) ks[(size_t)r * ncol + q] = K(ch.skel[r], far[q]);
          for (int i = 0; i < kc; ++i)
            for (int r = 0; r < ns; ++r) {
              const T qv = ch.Q[(size_t)i * ns + r];
              if (qv == T(0)) continue;
              T* dst = &w[(size_t)(roff + i) * ncol];
              const T* src = &ks[(size_t)r * ncol];
              for (int64_t q = 0; q < ncol; ++q) dst[q] += qv * src[q];
            }
        }
        c.basis = (ncol && m) ? dominant_basis(w, m, ncol, eps, c.k) : std::vector<T>();
        if (!ncol || !m) c.k = 0;
        // rows of V_t at the candidate rows I_t1 u I_t2
        int n1 = (int)c1.skel.size(), n2 = (int)c2.skel.size(), nc2 = n1 + n2;
        std::vector<T> vc((size_t)nc2 * c.k, T(0));
        for (int r = 0; r < n1; ++r)
          for (int j = 0; j < c.k; ++j) {
            T acc = 0;
            for (int i = 0; i < k1; ++i) acc += c1.rows[(size_t)r * k1 + i] * c.basis[(size_t)i * c.k + j];
            vc[(size_t)r * c.k + j] = acc;
          }
        for (int r = 0; r < n2; ++r)
          for (int j = 0; j < c.k; ++j) {
            T acc = 0;
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
        c.rows.assign((size_t)p * c.k, T(0));
        for (int r = 0; r < p; ++r) {
          c.skel[r] = cand[pick[r]];
          for (int j = 0; j < c.k; ++j) c.rows[(size_t)r * c.k + j] = vc[(size_t)pick[r] * c.k + j];
        }
        c.Q = c.k ? pinv(c.rows, p, c.k) : std::vector<T>();
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
  for (int64_t t = 0; t < (1LL << L); ++t) put(out.vr, cd[L][t].basis);
  out.vc = out.vr;
  out.er.clear();
  for (int l = 0; l < L; ++l)
    for (int64_t t = 0; t < (1LL << l); ++t) put(out.er, cd[l][t].basis);
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
  std::vector<T> sv(total, T(0));
  for (int l = 0; l <= L; ++l) {
    std::vector<const Block*> rb;
    for (auto& b : st.blocks[l])
      if (b.kind == KR) rb.push_back(&b);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < (int64_t)rb.size(); ++q) {
      const Block& b = *rb[q];
      const ClusterData<T> &ct = cd[l][b.t], &cs = cd[l][b.s];
      int kt = ct.k, ks = cs.k, nt = (int)ct.skel.size(), ns = (int)cs.skel.size();
      if (!kt || !ks) continue;
      std::vector<T> kts((size_t)nt * ns);
      for (int i = 0; i < nt; ++i)
        for (int j = 0; j < ns; ++j) kts[(size_t)i * ns + j] = K(ct.skel[i], cs.skel[j]);
      std::vector<T> tmp((size_t)kt * ns, T(0));  // Q_t K
      for (int a = 0; a < kt; ++a)
        for (int i = 0; i < nt; ++i) {
          const T qv = ct.Q[(size_t)a * nt + i];
          for (int j = 0; j < ns; ++j) tmp[(size_t)a * ns + j] += qv * kts[(size_t)i * ns + j];
        }
      T* dst = &sv[boff[l][b.idx]];
      for (int a = 0; a < kt; ++a)
        for (int c = 0; c < ks; ++c) {
          T acc = 0;
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
  out.s.clear();
  put(out.s, sv);
  std::vector<T> fv(foff.back(), T(0));
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < (int64_t)fb.size(); ++q) {
    const Block& b = *fb[q];
    int64_t t0 = st.start[L][b.t], s0 = st.start[L][b.s], mt = st.size[L][b.t], ms = st.size[L][b.s];
    T* dst = &fv[foff[q]];
    for (int64_t i = 0; i < mt; ++i)
      for (int64_t j = 0; j < ms; ++j) dst[i * ms + j] = K(t0 + i, s0 + j);
  }
  out.f.clear();
  put(out.f, fv);
}

}  // namespace

void build_h2_host(const Structure& st, const h2_kernel& kern, double eps, Packed& out) {
  if (kern.kind == H2_K_HELMHOLTZ)
    build_typed<cd>(st, kern, eps, out);
  else if (kern.kind == H2_K_LAPLACE || kern.kind == H2_K_INV_R2)
    build_typed<double>(st, kern, eps, out);
  else
    throw Error(H2_EINVAL, "unknown kernel kind");
}

}  // namespace h2
