// Device program of the product C = A B (Sec. III-IV) and of the H^2 matvec.
//
// The host walks the block structure once and emits launch groups; each group is a
// batch of independent segments (one output matrix each, a sum of small products
// over its items), an eigen batch (new bases), or a memset.  Segments of one group
// never share an output, so every sum has a fixed order: reruns are bitwise equal.
// All dims are the padded caps of the level; padded entries are exactly zero.
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
#include <algorithm>
#include <cstring>
#include <map>

#include "internal.hpp"

namespace h2 {

namespace {

enum TClass : int8_t { TC_R = 0, TC_F = 1, TC_NL = 2, TC_SUB = 3 };

struct PlanBuilder {
  Plan& P;
  int64_t wtop = 0;
  size_t g0 = 0;
  explicit PlanBuilder(Plan& p) : P(p) {}

  int64_t W(int64_t elems) {
    int64_t o = wtop;
    wtop += (elems + 31) & ~int64_t(31);
    return tag(AR_W, o);
  }
  void begin() { g0 = P.segs.size(); }
  void end(const char* phase, int level) {
    if (P.segs.size() > g0) {
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
  void gemm(int64_t out, int m, int n, int k, int lda, int ldb, int ldc, uint8_t fl,
            const std::vector<Item>& it) {
    if (m <= 0 || n <= 0 || it.empty()) return;
    if (k <= 0) return;  // zero contribution; outputs start at zero
    Seg s{};
    s.out = out;
    s.first = (int32_t)P.items.size();
    s.count = (int32_t)it.size();
    s.m = (int16_t)m;
    s.n = (int16_t)n;
    s.k = (int16_t)k;
    s.lda = (int16_t)lda;
    s.ldb = (int16_t)ldb;
    s.ldc = (int16_t)ldc;
    s.flags = fl;
    if ((int64_t)P.items.size() + (int64_t)it.size() > INT32_MAX) throw Error(H2_ENOMEM, "plan too large");
    P.items.insert(P.items.end(), it.begin(), it.end());
    P.segs.push_back(s);
    P.flops += 2LL * m * n * k * (int64_t)it.size();
  }
  void gemm1(int64_t out, int m, int n, int k, int lda, int ldb, int ldc, uint8_t fl, int64_t a, int64_t b) {
    gemm(out, m, n, k, lda, ldb, ldc, fl, {Item{a, b}});
  }
  void sum(int64_t out, int m, int n, int lda, int ldc, bool acc, const std::vector<int64_t>& mats) {
    if (m <= 0 || n <= 0 || mats.empty()) return;
    std::vector<Item> it;
    for (auto a : mats) it.push_back(Item{a, 0});
    Seg s{};
    s.out = out;
    s.first = (int32_t)P.items.size();
    s.count = (int32_t)it.size();
    s.m = (int16_t)m;
    s.n = (int16_t)n;
    s.k = 0;
    s.lda = (int16_t)lda;
    s.ldb = 0;
    s.ldc = (int16_t)ldc;
    s.flags = SF_SUM | (acc ? SF_ACC : 0);
    P.items.insert(P.items.end(), it.begin(), it.end());
    P.segs.push_back(s);
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
  int64_t s24 = -1, s3 = -1, M = -1, Mt = -1;
  int32_t cpos = -1;   // position of the block in C's level list (R, F, NL targets)
  bool has_nlnl = false;
  std::vector<int32_t> child;  // SUB/R targets with NL x NL triples: 4 child target ids
};

struct LevelTargets {
  std::vector<Target> tg;
  std::unordered_map<int64_t, int32_t> id;
  std::vector<Triple> trip;
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
  for (int32_t pa = 0; pa < (int32_t)bl.size(); ++pa) {
    int64_t i = bl[pa].t, j = bl[pa].s;
    for (int32_t pb = rp[j]; pb < rp[j + 1]; ++pb) {
      int64_t k = bl[pb].s;
      int64_t key = Structure::key(i, k);
      auto it = lt.id.find(key);
      int32_t id;
      if (it == lt.id.end()) {
        id = (int32_t)lt.tg.size();
        lt.id[key] = id;
        Target t;
        t.i = (int32_t)i;
        t.k = (int32_t)k;
        t.cls = classify(st, l, i, k, t.cpos);
        lt.tg.push_back(t);
      } else {
        id = it->second;
      }
      lt.trip.push_back({pa, pb, id});
      if (bl[pa].kind == KNL && bl[pb].kind == KNL) lt.tg[id].has_nlnl = true;
    }
  }
}

}  // namespace

void build_mmp_plan(const Mat& A, const Mat& B, Mat& C, const MmpParams& prm, Plan& P) {
  const Structure& st = *A.st;
  const int L = st.L, LS = st.LS, lmin = st.lmin;
  PlanBuilder pb(P);
  // caps of C: leaf LS, non-leaf min(2 K[l+1], cap) (no cap in full mode), 0 above l_min
  C.Kr.assign(L + 1, 0);
  C.Kc.assign(L + 1, 0);
  C.Kr[L] = C.Kc[L] = LS;
  for (int l = L - 1; l >= 0; --l) {
    if (l < lmin) {
      C.Kr[l] = C.Kc[l] = 0;
      continue;
    }
    int cap = prm.trunc == H2_TRUNC_FULL ? 1 << 20 : prm.rank_cap;
    C.Kr[l] = std::min(2 * C.Kr[l + 1], cap);
    C.Kc[l] = std::min(2 * C.Kc[l + 1], cap);
  }
  mat_elems(C);  // offsets of C's arrays
  // zero the workspace first (outputs accumulate)
  {
    Launch z;
    z.kind = Launch::MEMSET;
    z.phase = "zero";
    P.launches.push_back(z);  // size filled at the end
  }
  auto rA = [&](int l) { return A.Kr[l]; };
  auto cA = [&](int l) { return A.Kc[l]; };
  auto rB = [&](int l) { return B.Kr[l]; };
  auto cB = [&](int l) { return B.Kc[l]; };
  auto rC = [&](int l) { return C.Kr[l]; };
  auto cC = [&](int l) { return C.Kc[l]; };
  auto tA = [&](int64_t o) { return tag(AR_A, o); };
  auto tB = [&](int64_t o) { return tag(AR_B, o); };
  auto tC = [&](int64_t o) { return tag(AR_C, o); };

  // ---- B_j on levels l_min..L
  std::vector<std::vector<int64_t>> Bj(L + 1);
  for (int l = L; l >= lmin; --l) {
    int64_t nc = 1LL << l;
    Bj[l].resize(nc);
    for (int64_t j = 0; j < nc; ++j) Bj[l][j] = pb.W((int64_t)cA(l) * rB(l));
  }
  pb.begin();
  for (int64_t j = 0; j < (1LL << L); ++j)
    pb.gemm1(Bj[L][j], cA(L), rB(L), LS, cA(L), rB(L), rB(L), SF_TA, tA(A.Vc(j)), tB(B.Vr(j)));
  pb.end("bprod", L);
  for (int l = L - 1; l >= lmin; --l) {
    int64_t nc = 1LL << l;
    std::vector<int64_t> tmp(2 * nc);
    for (auto& x : tmp) x = pb.W((int64_t)cA(l + 1) * rB(l));
    pb.begin();
    for (int64_t j = 0; j < nc; ++j)
      for (int a = 0; a < 2; ++a)
        pb.gemm1(tmp[2 * j + a], cA(l + 1), rB(l), rB(l + 1), rB(l + 1), rB(l), rB(l), 0, Bj[l + 1][2 * j + a],
                 tB(B.Er(l, j) + (int64_t)a * rB(l + 1) * rB(l)));
    pb.end("bprod", l);
    pb.begin();
    for (int64_t j = 0; j < nc; ++j) {
      std::vector<Item> it;
      for (int a = 0; a < 2; ++a) it.push_back({tA(A.Ec(l, j) + (int64_t)a * cA(l + 1) * cA(l)), tmp[2 * j + a]});
      pb.gemm(Bj[l][j], cA(l), rB(l), cA(l + 1), cA(l), rB(l), rB(l), SF_TA, it);
    }
    pb.end("bprod", l);
  }

  // per-level data that the next level up reads
  std::vector<std::vector<int64_t>> PA(L + 1), PB(L + 1), Ahat(L + 1), Bhat(L + 1);
  std::vector<LevelTargets> LT(L + 1);
  const int64_t LS2 = (int64_t)LS * LS;

  // =========================================================== leaf level (Sec. III)
  {
    const int l = L;
    LevelTargets& lt = LT[l];
    enumerate(st, l, lt);
    const auto& bl = st.blocks[l];
    const int64_t nb = (int64_t)bl.size(), nc = 1LL << l;
    // allocations
    std::vector<int64_t> Y(nb, -1), Yb(nb, -1), T1(nb, -1), T2(nb, -1), Q(nb, -1), Rr(nb, -1), Wsum(nb, -1),
        YW(nb, -1), Wsc(nb, -1), YWc(nb, -1), Ach(nb, -1), Bch(nb, -1);
    Ahat[l].assign(nb, -1);
    Bhat[l].assign(nb, -1);
    for (int64_t p = 0; p < nb; ++p) {
      Ahat[l][p] = pb.W((int64_t)rC(l) * rB(l));
      Bhat[l][p] = pb.W((int64_t)cA(l) * cC(l));
      if (bl[p].kind == KF) {
        Y[p] = pb.W((int64_t)LS * rB(l));
        Yb[p] = pb.W((int64_t)cA(l) * LS);
        Q[p] = pb.W(LS2);
        Rr[p] = pb.W(LS2);
        Ach[p] = pb.W((int64_t)rC(l) * LS);
        Bch[p] = pb.W((int64_t)LS * cC(l));
      } else {
        T1[p] = pb.W((int64_t)rA(l) * rB(l));
        T2[p] = pb.W((int64_t)cA(l) * cB(l));
      }
    }
    std::vector<int64_t> G1r(nc, -1), G2r(nc, -1), G3r(nc), G1c(nc, -1), G2c(nc, -1), G3c(nc);
    for (int64_t t = 0; t < nc; ++t) {
      G3r[t] = pb.W(LS2);
      G3c[t] = pb.W(LS2);
    }
    // which F blocks have a case-1 partner with an R/SUB target (for the Gram sums)
    std::vector<std::vector<int64_t>> Ksets(nb), Isets(nb);  // Q of (j,k) per A-block; Rr of (i,j) per B-block
    std::vector<std::vector<Item>> gF(lt.tg.size()), gZ(lt.tg.size()), gZp(lt.tg.size()), gZpp(lt.tg.size()),
        g1(lt.tg.size()), g24(lt.tg.size()), g3(lt.tg.size());
    std::vector<int64_t> Z(lt.tg.size(), -1), Zp(lt.tg.size(), -1), Zpp(lt.tg.size(), -1);
    for (auto& tr : lt.trip) {
      const Block &ba = bl[tr.pa], &bb = bl[tr.pb];
      Target& T = lt.tg[tr.tgt];
      if (T.cls == TC_F) {
        if (ba.kind == KF && bb.kind == KF) gF[tr.tgt].push_back({tA(A.F(ba.idx)), tB(B.F(bb.idx))});
        else if (ba.kind == KF) gZ[tr.tgt].push_back({Y[tr.pa], tB(B.S(l, bb.idx))});
        else if (bb.kind == KF) gZp[tr.tgt].push_back({tA(A.S(l, ba.idx)), Yb[tr.pb]});
        else gZpp[tr.tgt].push_back({T1[tr.pa], tB(B.S(l, bb.idx))});
      } else {
        if (ba.kind == KF && bb.kind == KF) {
          Ksets[tr.pa].push_back(Q[tr.pb]);
          Isets[tr.pb].push_back(Rr[tr.pa]);
          g1[tr.tgt].push_back({Ach[tr.pa], Bch[tr.pb]});
        } else if (bb.kind == KR) {
          g24[tr.tgt].push_back({Ahat[l][tr.pa], tB(B.S(l, bb.idx))});
        } else {
          g3[tr.tgt].push_back({tA(A.S(l, ba.idx)), Bhat[l][tr.pb]});
        }
      }
    }
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      Target& T = lt.tg[q];
      if (T.cls == TC_F) {
        if (!gZ[q].empty()) Z[q] = pb.W((int64_t)LS * cB(l));
        if (!gZp[q].empty()) Zp[q] = pb.W((int64_t)rA(l) * LS);
        if (!gZpp[q].empty()) Zpp[q] = pb.W((int64_t)rA(l) * cB(l));
        if (Zpp[q] >= 0 && Z[q] < 0) Z[q] = pb.W((int64_t)LS * cB(l));
      } else {
        T.ssum = T.cls == TC_R ? tC(C.S(l, bl[T.cpos].idx)) : pb.W((int64_t)rC(l) * cC(l));
        if (!g24[q].empty()) T.s24 = pb.W((int64_t)rC(l) * cB(l));
        if (!g3[q].empty()) T.s3 = pb.W((int64_t)rA(l) * cC(l));
      }
    }
    for (int64_t p = 0; p < nb; ++p) {
      if (!Ksets[p].empty()) {
        Wsum[p] = pb.W(LS2);
        YW[p] = pb.W(LS2);
      }
      if (!Isets[p].empty()) {
        Wsc[p] = pb.W(LS2);
        YWc[p] = pb.W(LS2);
      }
    }
    // L1: per-block products
    pb.begin();
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind == KF) {
        pb.gemm1(Y[p], LS, rB(l), LS, LS, rB(l), rB(l), 0, tA(A.F(b.idx)), tB(B.Vr(b.s)));
        pb.gemm1(Yb[p], cA(l), LS, LS, cA(l), LS, LS, SF_TA, tA(A.Vc(b.t)), tB(B.F(b.idx)));
        pb.gemm1(Q[p], LS, LS, LS, LS, LS, LS, SF_TB, tB(B.F(b.idx)), tB(B.F(b.idx)));
        pb.gemm1(Rr[p], LS, LS, LS, LS, LS, LS, SF_TA, tA(A.F(b.idx)), tA(A.F(b.idx)));
      } else {
        pb.gemm1(T1[p], rA(l), rB(l), cA(l), cA(l), rB(l), rB(l), 0, tA(A.S(l, b.idx)), Bj[l][b.s]);
        pb.gemm1(T2[p], cA(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, Bj[l][b.t], tB(B.S(l, b.idx)));
      }
    }
    for (int64_t t = 0; t < nc; ++t) {
      pb.gemm1(G3r[t], LS, LS, rA(l), rA(l), rA(l), LS, SF_TB, tA(A.Vr(t)), tA(A.Vr(t)));
      pb.gemm1(G3c[t], LS, LS, cB(l), cB(l), cB(l), LS, SF_TB, tB(B.Vc(t)), tB(B.Vc(t)));
    }
    pb.end("leaf_blockprod", l);
    // L2: dense targets, Gram pieces
    pb.begin();
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      if (T.cls != TC_F) continue;
      int64_t fc = tC(C.F(bl[T.cpos].idx));
      pb.gemm(fc, LS, LS, LS, LS, LS, LS, SF_ACC, gF[q]);
      pb.gemm(Z[q], LS, cB(l), rB(l), rB(l), cB(l), cB(l), 0, gZ[q]);
      pb.gemm(Zp[q], rA(l), LS, cA(l), cA(l), LS, LS, 0, gZp[q]);
      pb.gemm(Zpp[q], rA(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, gZpp[q]);
    }
    for (int64_t p = 0; p < nb; ++p) {
      pb.sum(Wsum[p], LS, LS, LS, LS, false, Ksets[p]);
      pb.sum(Wsc[p], LS, LS, LS, LS, false, Isets[p]);
    }
    for (int64_t t = 0; t < nc; ++t) {
      std::vector<Item> r2, c2;
      for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p)
        if (bl[p].kind == KF) r2.push_back({Y[p], Y[p]});
      for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1]; ++q) {
        int32_t p = st.col_list[l][q];
        if (bl[p].kind == KF) c2.push_back({Yb[p], Yb[p]});
      }
      if (!r2.empty()) {
        G2r[t] = pb.W(LS2);
        pb.gemm(G2r[t], LS, LS, rB(l), rB(l), rB(l), LS, SF_TB, r2);
      }
      if (!c2.empty()) {
        G2c[t] = pb.W(LS2);
        pb.gemm(G2c[t], LS, LS, cA(l), LS, LS, LS, SF_TA, c2);
      }
    }
    pb.end("leaf_dense_gram", l);
    // L3
    pb.begin();
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      if (T.cls != TC_F || Zpp[q] < 0) continue;
      pb.gemm1(Z[q], LS, cB(l), rA(l), rA(l), cB(l), cB(l), SF_ACC, tA(A.Vr(T.i)), Zpp[q]);
    }
    for (int64_t p = 0; p < nb; ++p) {
      if (YW[p] >= 0) pb.gemm1(YW[p], LS, LS, LS, LS, LS, LS, 0, tA(A.F(bl[p].idx)), Wsum[p]);
      if (YWc[p] >= 0) pb.gemm1(YWc[p], LS, LS, LS, LS, LS, LS, 0, Wsc[p], tB(B.F(bl[p].idx)));
    }
    pb.end("leaf_dense_gram", l);
    // L4
    pb.begin();
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      if (T.cls != TC_F || Z[q] < 0) continue;
      pb.gemm1(tC(C.F(bl[T.cpos].idx)), LS, LS, cB(l), cB(l), cB(l), LS, SF_TB | SF_ACC, Z[q], tB(B.Vc(T.k)));
    }
    for (int64_t t = 0; t < nc; ++t) {
      std::vector<Item> r1, c1;
      for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p)
        if (YW[p] >= 0) r1.push_back({YW[p], tA(A.F(bl[p].idx))});
      for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1]; ++q) {
        int32_t p = st.col_list[l][q];
        if (YWc[p] >= 0) c1.push_back({tB(B.F(bl[p].idx)), YWc[p]});
      }
      if (!r1.empty()) {
        G1r[t] = pb.W(LS2);
        pb.gemm(G1r[t], LS, LS, LS, LS, LS, LS, SF_TB, r1);
      }
      if (!c1.empty()) {
        G1c[t] = pb.W(LS2);
        pb.gemm(G1c[t], LS, LS, LS, LS, LS, LS, SF_TA, c1);
      }
    }
    pb.end("leaf_dense_gram", l);
    pb.begin();
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      if (T.cls != TC_F || Zp[q] < 0) continue;
      pb.gemm1(tC(C.F(bl[T.cpos].idx)), LS, LS, rA(l), rA(l), LS, LS, SF_ACC, tA(A.Vr(T.i)), Zp[q]);
    }
    pb.end("leaf_dense", l);
    // eig: new leaf bases
    size_t e0 = P.eigs.size();
    for (int64_t t = 0; t < nc; ++t) {
      for (int col = 0; col < 2; ++col) {
        EigTask e{};
        e.g[0] = col ? G1c[t] : G1r[t];
        e.g[1] = col ? G2c[t] : G2r[t];
        e.g[2] = col ? G3c[t] : G3r[t];
        e.out = tC(col ? C.Vc(t) : C.Vr(t));
        e.rank_out = Structure::node(l, t);
        e.child1 = e.child2 = -1;
        e.nleaf = (int32_t)st.size[l][t];
        e.n_pad = (int16_t)LS;
        e.half = 0;
        e.kcap = (int16_t)(col ? cC(l) : rC(l));
        e.col = (int16_t)col;
        P.eigs.push_back(e);
      }
    }
    pb.eigs(e0, "eig", l);
    // projections and collects
    PA[l].resize(nc);
    PB[l].resize(nc);
    pb.begin();
    for (int64_t t = 0; t < nc; ++t) {
      PA[l][t] = pb.W((int64_t)rC(l) * rA(l));
      PB[l][t] = pb.W((int64_t)cB(l) * cC(l));
      pb.gemm1(PA[l][t], rC(l), rA(l), LS, rC(l), rA(l), rA(l), SF_TA, tC(C.Vr(t)), tA(A.Vr(t)));
      pb.gemm1(PB[l][t], cB(l), cC(l), LS, cB(l), cC(l), cC(l), SF_TA, tB(B.Vc(t)), tC(C.Vc(t)));
    }
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind != KF) continue;
      pb.gemm1(Ahat[l][p], rC(l), rB(l), LS, rC(l), rB(l), rB(l), SF_TA, tC(C.Vr(b.t)), Y[p]);
      pb.gemm1(Bhat[l][p], cA(l), cC(l), LS, LS, cC(l), cC(l), 0, Yb[p], tC(C.Vc(b.s)));
      pb.gemm1(Ach[p], rC(l), LS, LS, rC(l), LS, LS, SF_TA, tC(C.Vr(b.t)), tA(A.F(b.idx)));
      pb.gemm1(Bch[p], LS, cC(l), LS, LS, cC(l), cC(l), 0, tB(B.F(b.idx)), tC(C.Vc(b.s)));
    }
    pb.end("leaf_proj", l);
    pb.begin();
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind != KR) continue;
      pb.gemm1(Ahat[l][p], rC(l), rB(l), rA(l), rA(l), rB(l), rB(l), 0, PA[l][b.t], T1[p]);
      pb.gemm1(Bhat[l][p], cA(l), cC(l), cB(l), cB(l), cC(l), cC(l), 0, T2[p], PB[l][b.s]);
    }
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      if (T.cls == TC_F) continue;
      pb.gemm(T.ssum, rC(l), cC(l), LS, LS, cC(l), cC(l), SF_ACC, g1[q]);
    }
    pb.end("leaf_coup", l);
    pb.begin();
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      if (T.cls == TC_F) continue;
      pb.gemm(T.s24, rC(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, g24[q]);
      pb.gemm(T.s3, rA(l), cC(l), cA(l), cA(l), cC(l), cC(l), 0, g3[q]);
    }
    pb.end("leaf_coup", l);
    pb.begin();
    for (auto& T : lt.tg)
      if (T.cls != TC_F && T.s24 >= 0)
        pb.gemm1(T.ssum, rC(l), cC(l), cB(l), cB(l), cC(l), cC(l), SF_ACC, T.s24, PB[l][T.k]);
    pb.end("leaf_coup", l);
    pb.begin();
    for (auto& T : lt.tg)
      if (T.cls != TC_F && T.s3 >= 0)
        pb.gemm1(T.ssum, rC(l), cC(l), rA(l), rA(l), cC(l), cC(l), SF_ACC, PA[l][T.i], T.s3);
    pb.end("leaf_coup", l);
  }

  // ================================================== non-leaf levels (Sec. IV)
  for (int l = L - 1; l >= lmin; --l) {
    const int c = l + 1;
    LevelTargets& lt = LT[l];
    enumerate(st, l, lt);
    const auto& bl = st.blocks[l];
    const int64_t nb = (int64_t)bl.size(), nc = 1LL << l;
    const int hr = rC(c), hc = cC(c);  // child caps of C
    std::vector<int64_t> Ac(nb, -1), Bc(nb, -1), Yn(nb, -1), Ybn(nb, -1), T1(nb, -1), T2(nb, -1);
    Ahat[l].assign(nb, -1);
    Bhat[l].assign(nb, -1);
    for (int64_t p = 0; p < nb; ++p) {
      Ahat[l][p] = pb.W((int64_t)rC(l) * rB(l));
      Bhat[l][p] = pb.W((int64_t)cA(l) * cC(l));
      if (bl[p].kind == KNL) {
        Ac[p] = pb.W((int64_t)2 * hr * 2 * rB(c));
        Bc[p] = pb.W((int64_t)2 * cA(c) * 2 * hc);
        Yn[p] = pb.W((int64_t)2 * hr * rB(l));
        Ybn[p] = pb.W((int64_t)cA(l) * 2 * hc);
      } else if (bl[p].kind == KR) {
        T1[p] = pb.W((int64_t)rA(l) * rB(l));
        T2[p] = pb.W((int64_t)cA(l) * cB(l));
      }
    }
    // targets
    std::vector<std::vector<Item>> g24(lt.tg.size()), g3(lt.tg.size());
    for (auto& tr : lt.trip) {
      const Block &ba = bl[tr.pa], &bb = bl[tr.pb];
      if (ba.kind == KNL && bb.kind == KNL) continue;
      if (bb.kind == KR) g24[tr.tgt].push_back({Ahat[l][tr.pa], tB(B.S(l, bb.idx))});
      else g3[tr.tgt].push_back({tA(A.S(l, ba.idx)), Bhat[l][tr.pb]});
    }
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      Target& T = lt.tg[q];
      if (T.cls == TC_F) throw Error(H2_EINTERNAL, "dense target above the leaf level");
      T.ssum = T.cls == TC_R ? tC(C.S(l, bl[T.cpos].idx)) : pb.W((int64_t)rC(l) * cC(l));
      if (!g24[q].empty()) T.s24 = pb.W((int64_t)rC(l) * cB(l));
      if (!g3[q].empty()) T.s3 = pb.W((int64_t)rA(l) * cC(l));
      if (T.has_nlnl && T.cls != TC_NL) {
        T.M = pb.W((int64_t)2 * hr * 2 * hc);
        T.Mt = pb.W((int64_t)2 * hr * cC(l));
      }
    }
    // N1: assemble collected NL blocks and merged couplings; R-block products
    pb.begin();
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind == KNL) {
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) {
            int32_t cp = st.find(c, 2 * b.t + a, 2 * b.s + bb);
            if (cp < 0) throw Error(H2_EINTERNAL, "missing child block");
            pb.sum(Ac[p] + (int64_t)a * hr * 2 * rB(c) + (int64_t)bb * rB(c), hr, rB(c), rB(c), 2 * rB(c), false,
                   {Ahat[c][cp]});
            pb.sum(Bc[p] + (int64_t)a * cA(c) * 2 * hc + (int64_t)bb * hc, cA(c), hc, hc, 2 * hc, false, {Bhat[c][cp]});
          }
      } else if (b.kind == KR) {
        pb.gemm1(T1[p], rA(l), rB(l), cA(l), cA(l), rB(l), rB(l), 0, tA(A.S(l, b.idx)), Bj[l][b.s]);
        pb.gemm1(T2[p], cA(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, Bj[l][b.t], tB(B.S(l, b.idx)));
      }
    }
    for (auto& T : lt.tg) {
      if (T.M < 0) continue;
      for (int a = 0; a < 2; ++a)
        for (int bb = 0; bb < 2; ++bb) {
          auto it = LT[c].id.find(Structure::key(2 * T.i + a, 2 * T.k + bb));
          if (it == LT[c].id.end()) throw Error(H2_EINTERNAL, "missing child target");
          pb.sum(T.M + (int64_t)a * hr * 2 * hc + (int64_t)bb * hc, hr, hc, hc, 2 * hc, false,
                 {LT[c].tg[it->second].ssum});
        }
    }
    pb.end("merge", l);
    // N2: Gram factors
    std::vector<int64_t> Wr(nc), Wc(nc);
    pb.begin();
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind != KNL) continue;
      pb.gemm1(Yn[p], 2 * hr, rB(l), 2 * rB(c), 2 * rB(c), rB(l), rB(l), 0, Ac[p], tB(B.Er(l, b.s)));
      pb.gemm1(Ybn[p], cA(l), 2 * hc, 2 * cA(c), cA(l), 2 * hc, 2 * hc, SF_TA, tA(A.Ec(l, b.t)), Bc[p]);
    }
    for (int64_t t = 0; t < nc; ++t) {
      Wr[t] = pb.W((int64_t)2 * hr * rA(l));
      Wc[t] = pb.W((int64_t)2 * hc * cB(l));
      for (int a = 0; a < 2; ++a) {
        pb.gemm1(Wr[t] + (int64_t)a * hr * rA(l), hr, rA(l), rA(c), rA(c), rA(l), rA(l), 0, PA[c][2 * t + a],
                 tA(A.Er(l, t) + (int64_t)a * rA(c) * rA(l)));
        pb.gemm1(Wc[t] + (int64_t)a * hc * cB(l), hc, cB(l), cB(c), hc, cB(l), cB(l), SF_TA, PB[c][2 * t + a],
                 tB(B.Ec(l, t) + (int64_t)a * cB(c) * cB(l)));
      }
    }
    pb.end("nl_gram", l);
    // N3: Grams
    const int gr = 2 * hr, gc = 2 * hc;
    std::vector<int64_t> G1r(nc, -1), G2r(nc, -1), G3r(nc), G1c(nc, -1), G2c(nc, -1), G3c(nc);
    std::vector<std::vector<Item>> r1(nc), c1(nc);
    for (auto& T : lt.tg)
      if (T.M >= 0) {
        r1[T.i].push_back({T.M, T.M});
        c1[T.k].push_back({T.M, T.M});
      }
    pb.begin();
    for (int64_t t = 0; t < nc; ++t) {
      std::vector<Item> r2, c2;
      for (int32_t p = st.row_ptr[l][t]; p < st.row_ptr[l][t + 1]; ++p)
        if (bl[p].kind == KNL) r2.push_back({Yn[p], Yn[p]});
      for (int32_t q = st.col_ptr[l][t]; q < st.col_ptr[l][t + 1]; ++q) {
        int32_t p = st.col_list[l][q];
        if (bl[p].kind == KNL) c2.push_back({Ybn[p], Ybn[p]});
      }
      if (!r1[t].empty()) {
        G1r[t] = pb.W((int64_t)gr * gr);
        pb.gemm(G1r[t], gr, gr, gc, gc, gc, gr, SF_TB, r1[t]);
      }
      if (!c1[t].empty()) {
        G1c[t] = pb.W((int64_t)gc * gc);
        pb.gemm(G1c[t], gc, gc, gr, gc, gc, gc, SF_TA, c1[t]);
      }
      if (!r2.empty()) {
        G2r[t] = pb.W((int64_t)gr * gr);
        pb.gemm(G2r[t], gr, gr, rB(l), rB(l), rB(l), gr, SF_TB, r2);
      }
      if (!c2.empty()) {
        G2c[t] = pb.W((int64_t)gc * gc);
        pb.gemm(G2c[t], gc, gc, cA(l), gc, gc, gc, SF_TA, c2);
      }
      G3r[t] = pb.W((int64_t)gr * gr);
      G3c[t] = pb.W((int64_t)gc * gc);
      pb.gemm1(G3r[t], gr, gr, rA(l), rA(l), rA(l), gr, SF_TB, Wr[t], Wr[t]);
      pb.gemm1(G3c[t], gc, gc, cB(l), cB(l), cB(l), gc, SF_TB, Wc[t], Wc[t]);
    }
    pb.end("nl_gram", l);
    size_t e0 = P.eigs.size();
    for (int64_t t = 0; t < nc; ++t)
      for (int col = 0; col < 2; ++col) {
        EigTask e{};
        e.g[0] = col ? G1c[t] : G1r[t];
        e.g[1] = col ? G2c[t] : G2r[t];
        e.g[2] = col ? G3c[t] : G3r[t];
        e.out = tC(col ? C.Ec(l, t) : C.Er(l, t));
        e.rank_out = Structure::node(l, t);
        e.child1 = Structure::node(c, 2 * t);
        e.child2 = Structure::node(c, 2 * t + 1);
        e.nleaf = 0;
        e.n_pad = (int16_t)(col ? gc : gr);
        e.half = (int16_t)(col ? hc : hr);
        e.kcap = (int16_t)(col ? cC(l) : rC(l));
        e.col = (int16_t)col;
        P.eigs.push_back(e);
      }
    pb.eigs(e0, "eig", l);
    // N4: projections, NL collects, case-1 half products
    PA[l].resize(nc);
    PB[l].resize(nc);
    pb.begin();
    for (int64_t t = 0; t < nc; ++t) {
      PA[l][t] = pb.W((int64_t)rC(l) * rA(l));
      PB[l][t] = pb.W((int64_t)cB(l) * cC(l));
      pb.gemm1(PA[l][t], rC(l), rA(l), gr, rC(l), rA(l), rA(l), SF_TA, tC(C.Er(l, t)), Wr[t]);
      pb.gemm1(PB[l][t], cB(l), cC(l), gc, cB(l), cC(l), cC(l), SF_TA, Wc[t], tC(C.Ec(l, t)));
    }
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind != KNL) continue;
      pb.gemm1(Ahat[l][p], rC(l), rB(l), gr, rC(l), rB(l), rB(l), SF_TA, tC(C.Er(l, b.t)), Yn[p]);
      pb.gemm1(Bhat[l][p], cA(l), cC(l), gc, gc, cC(l), cC(l), 0, Ybn[p], tC(C.Ec(l, b.s)));
    }
    for (auto& T : lt.tg)
      if (T.M >= 0) pb.gemm1(T.Mt, gr, cC(l), gc, gc, cC(l), cC(l), 0, T.M, tC(C.Ec(l, T.k)));
    pb.end("nl_proj", l);
    // N5
    pb.begin();
    for (int64_t p = 0; p < nb; ++p) {
      const Block& b = bl[p];
      if (b.kind != KR) continue;
      pb.gemm1(Ahat[l][p], rC(l), rB(l), rA(l), rA(l), rB(l), rB(l), 0, PA[l][b.t], T1[p]);
      pb.gemm1(Bhat[l][p], cA(l), cC(l), cB(l), cB(l), cC(l), cC(l), 0, T2[p], PB[l][b.s]);
    }
    for (auto& T : lt.tg)
      if (T.M >= 0) pb.gemm1(T.ssum, rC(l), cC(l), gr, rC(l), cC(l), cC(l), SF_TA | SF_ACC, tC(C.Er(l, T.i)), T.Mt);
    pb.end("nl_coup", l);
    pb.begin();
    for (size_t q = 0; q < lt.tg.size(); ++q) {
      const Target& T = lt.tg[q];
      pb.gemm(T.s24, rC(l), cB(l), rB(l), rB(l), cB(l), cB(l), 0, g24[q]);
      pb.gemm(T.s3, rA(l), cC(l), cA(l), cA(l), cC(l), cC(l), 0, g3[q]);
    }
    pb.end("nl_coup", l);
    pb.begin();
    for (auto& T : lt.tg)
      if (T.s24 >= 0) pb.gemm1(T.ssum, rC(l), cC(l), cB(l), cB(l), cC(l), cC(l), SF_ACC, T.s24, PB[l][T.k]);
    pb.end("nl_coup", l);
    pb.begin();
    for (auto& T : lt.tg)
      if (T.s3 >= 0) pb.gemm1(T.ssum, rC(l), cC(l), rA(l), rA(l), cC(l), cC(l), SF_ACC, PA[l][T.i], T.s3);
    pb.end("nl_coup", l);
  }

  // ============================================ top-down split of NL-held couplings
  {
    // H slot per NL block: its target sum if it is a target, else a fresh slot when
    // its parent passes something down
    std::vector<std::vector<int64_t>> H(L + 1);
    for (int l = lmin; l < L; ++l) {
      const auto& bl = st.blocks[l];
      H[l].assign(bl.size(), -1);
      for (auto& T : LT[l].tg)
        if (T.cls == TC_NL) H[l][T.cpos] = T.ssum;
    }
    for (int l = lmin; l < L; ++l) {
      const int c = l + 1;
      const auto& bl = st.blocks[l];
      const int hr = rC(c), hc = cC(c);
      std::vector<int64_t> Xt(bl.size(), -1), X(bl.size(), -1);
      for (size_t p = 0; p < bl.size(); ++p)
        if (bl[p].kind == KNL && H[l][p] >= 0) {
          Xt[p] = pb.W((int64_t)rC(l) * 2 * hc);
          X[p] = pb.W((int64_t)2 * hr * 2 * hc);
        }
      pb.begin();
      for (size_t p = 0; p < bl.size(); ++p)
        if (Xt[p] >= 0)
          pb.gemm1(Xt[p], rC(l), 2 * hc, cC(l), cC(l), cC(l), 2 * hc, SF_TB, H[l][p], tC(C.Ec(l, bl[p].s)));
      pb.end("split", l);
      pb.begin();
      for (size_t p = 0; p < bl.size(); ++p)
        if (X[p] >= 0)
          pb.gemm1(X[p], 2 * hr, 2 * hc, rC(l), rC(l), 2 * hc, 2 * hc, 0, tC(C.Er(l, bl[p].t)), Xt[p]);
      pb.end("split", l);
      if (c < L) {
        // children R: S += X_ab ; children NL: H += X_ab
        for (size_t p = 0; p < st.blocks[c].size(); ++p)
          if (st.blocks[c][p].kind == KNL && H[c][p] < 0) {
            int32_t pp = st.find(l, st.blocks[c][p].t >> 1, st.blocks[c][p].s >> 1);
            if (pp >= 0 && X[pp] >= 0) H[c][p] = pb.W((int64_t)rC(c) * cC(c));
          }
      }
      pb.begin();
      std::vector<int64_t> Ft;
      std::vector<std::pair<int64_t, int64_t>> Fupd;  // (tmp, target F offset) with child row cluster
      std::vector<int32_t> Frow;
      for (size_t p = 0; p < bl.size(); ++p) {
        if (X[p] < 0) continue;
        for (int a = 0; a < 2; ++a)
          for (int bb = 0; bb < 2; ++bb) {
            int32_t cp = st.find(c, 2 * bl[p].t + a, 2 * bl[p].s + bb);
            const Block& cb = st.blocks[c][cp];
            int64_t xab = X[p] + (int64_t)a * hr * 2 * hc + (int64_t)bb * hc;
            if (cb.kind == KR) {
              pb.sum(tC(C.S(c, cb.idx)), hr, hc, 2 * hc, cC(c), true, {xab});
            } else if (cb.kind == KNL) {
              pb.sum(H[c][cp], hr, hc, 2 * hc, cC(c), true, {xab});
            } else {
              int64_t tmp = pb.W((int64_t)rC(c) * LS);
              pb.gemm1(tmp, rC(c), LS, cC(c), 2 * hc, cC(c), LS, SF_TB, xab, tC(C.Vc(cb.s)));
              Fupd.push_back({tmp, tC(C.F(cb.idx))});
              Frow.push_back(cb.t);
            }
          }
      }
      pb.end("split", l);
      pb.begin();
      for (size_t q = 0; q < Fupd.size(); ++q)
        pb.gemm1(Fupd[q].second, LS, LS, rC(c), rC(c), LS, LS, SF_ACC, tC(C.Vr(Frow[q])), Fupd[q].first);
      pb.end("split", c);
    }
  }
  P.w_elems = pb.wtop;
  P.launches[0].off = tag(AR_W, 0);
  P.launches[0].elems = pb.wtop;
}

void build_matvec_plan(const Mat& H, int64_t nrhs, Plan& P, int64_t& off_x, int64_t& off_y) {
  const Structure& st = *H.st;
  const int L = st.L, LS = st.LS;
  PlanBuilder pb(P);
  const int64_t nl = 1LL << L;
  const int nr = (int)nrhs;
  off_x = pb.W(nl * LS * nrhs);
  off_y = pb.W(nl * LS * nrhs);
  std::vector<int64_t> xh(L + 1), yh(L + 1);
  for (int l = 0; l <= L; ++l) {
    xh[l] = pb.W((1LL << l) * H.Kc[l] * nrhs);
    yh[l] = pb.W((1LL << l) * H.Kr[l] * nrhs);
  }
  Launch z;
  z.kind = Launch::MEMSET;
  z.off = tag(AR_W, 0);
  z.elems = pb.wtop;
  z.phase = "zero";
  P.launches.push_back(z);
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
  P.w_elems = pb.wtop;
}

}  // namespace h2
