// plan.hpp — product plans for the biquaternion matrix product (host side).
//
// A plan lists the real matrix products a kernel forms and how their results
// recombine into the eight output components.  It is built from the paper's
// bilinear scheme (Sec. III B, Eq. bilinearH: eight complex products P1..P8
// whose left/right factors are single complex coefficients or their Hadamard
// (+-1) sums, recombined as Q1 = 2P1 - (P5+P6+P7+P8)/4, Q2 = -2P2 + ..., and
// Gauss's three-product complex multiplication, Eq. cmplx-3-real-mult).
// When subalgebra flags mark components absent, the terms they feed are
// omitted (Sec. III B, last paragraph): a complex factor whose real or
// imaginary part is structurally zero needs one or two real products instead
// of three.  For mixed subalgebras a second strategy — the component-wise
// terms a_f b_g expanded from the same bilinear equations, each with the
// reduced Gauss rule — is sometimes cheaper (e.g. real x biquaternion: 8
// products instead of 10); the plan with fewer products is kept.
//
// Everything is exact integer bookkeeping: left/right factors are +-1 sums of
// op(A)/op(B) components, recombination weights are stored times 4 (the
// paper's weights are 2 and 1/4).
#pragma once
#include <array>
#include <cstdint>
#include <cstring>
#include <vector>

namespace hmat {

constexpr int kMaxProducts = 64;   // plan capacity (the component-wise algorithm needs 64)
constexpr int kMaxFactors = 24;    // factor slots per side (8 groups x Re, Im, Re+Im)

// Real-valued linear combination of the 8 components of op(X): sign per component.
struct Comb8 {
  int8_t s[8];
  bool operator==(const Comb8& o) const { return std::memcmp(s, o.s, 8) == 0; }
  bool zero() const {
    for (int c = 0; c < 8; ++c)
      if (s[c]) return false;
    return true;
  }
};

// Kernel-facing plan, independent of op (op signs are applied when loading).
//
// Each side (left = op(A), right = op(B)) has up to 8 groups.  A group is a
// +-1 combination x of the complex coefficients a_1..a_4 restricted to the
// present components: re[e] weights component e (Re a_{e+1}), im[e] weights
// component e+4 (Im a_{e+1}).  A group yields up to three real factors, each
// written to a factor slot: Re = sum_e re[e] X_e, Im = sum_e im[e] X_{e+4},
// and Re+Im (the Gauss factor).  Product p multiplies left slot pl[p] by right
// slot pr[p]; its result enters output component e with weight w4[e][p] / 4.
// In the four-multiplication form (four_m = 1, split mode only) every product
// has a second term: product p is pl[p] pr[p] + s pl2[p] pr2[p], s = -1 when
// bit p of neg2 is set, else +1 (one real GEMM over twice the inner
// dimension).
struct KPlan {
  int32_t np = 0;            // real products (<= kMaxProducts)
  int32_t strategy = 0;      // 0 bilinear (Eq. bilinearH + Gauss), 1 component-wise + Gauss, 2 standard
  int32_t nlg = 0, nrg = 0;  // groups per side (<= 8)
  int32_t nlf = 0, nrf = 0;  // factor slots per side (<= kMaxFactors)
  int8_t lre[8][4], lim[8][4], lslot[8][3];  // slot of Re, Im, Re+Im (-1: not needed)
  int8_t rre[8][4], rim[8][4], rslot[8][3];
  int8_t pl[kMaxProducts], pr[kMaxProducts];
  int8_t w4[8][kMaxProducts];
  // 1 when that side's groups are exactly the eight complex factors of
  // Eq. bilinearH on all eight components (left: a1, a4, a2, a3, then the
  // Hadamard rows; right: b1, b3, b4, b2, then the Hadamard rows), in that order
  int32_t bilinear_left = 0, bilinear_right = 0;
  // 1 when the products are the 24 of Eq. bilinearH with Gauss, in the order
  // (P1: T1, T2, T3), (P2: ...), ..., (P8: ...), with the paper's weights
  int32_t bilinear_full = 0;
  // the four-multiplication form of the full plan (four_m_plan): 16 products
  // Re P_r = Re X Re Y - Im X Im Y, Im P_r = Re X Im Y + Im X Re Y
  int32_t four_m = 0;
  int8_t pl2[kMaxProducts], pr2[kMaxProducts];
  uint64_t neg2 = 0;
};

namespace detail {

enum { CLS_ZERO = 0, CLS_RE = 1, CLS_IM = 2, CLS_CX = 3 };
enum { PART_RE = 0, PART_IM = 1, PART_SUM = 2 };

// A complex combination x over the complex coefficients a_1..a_4 (+-1 each).
struct CComb { int8_t x[4]; };

inline int cls_of(const CComb& x, unsigned flags) {
  int c = 0;
  for (int e = 0; e < 4; ++e) {
    if (!x.x[e]) continue;
    if ((flags >> e) & 1u) c |= CLS_RE;
    if ((flags >> (e + 4)) & 1u) c |= CLS_IM;
  }
  return c;
}

// A real factor: part (Re, Im or Re+Im) of a complex combination restricted to
// the present components.
struct Factor {
  int8_t re[4], im[4];
  int part;
  bool same_group(const Factor& o) const {
    return std::memcmp(re, o.re, 4) == 0 && std::memcmp(im, o.im, 4) == 0;
  }
  bool operator==(const Factor& o) const { return same_group(o) && part == o.part; }
};

inline Factor make_factor(const CComb& x, unsigned flags, int part) {
  Factor f;
  for (int e = 0; e < 4; ++e) {
    f.re[e] = ((flags >> e) & 1u) ? x.x[e] : 0;
    f.im[e] = ((flags >> (e + 4)) & 1u) ? x.x[e] : 0;
  }
  f.part = part;
  return f;
}

// Coefficients of the 8 components in a factor.
inline Comb8 factor_comb(const Factor& f) {
  Comb8 c{};
  for (int e = 0; e < 4; ++e) {
    if (f.part != PART_IM) c.s[e] = f.re[e];
    if (f.part != PART_RE) c.s[e + 4] = f.im[e];
  }
  return c;
}

struct Product {
  Factor l, r;
  int w4[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

// Add the real products of the complex product X*Y, contributing w4[e] * P to
// complex output Q_e (real part -> component e, imaginary -> e+4).
inline void add_complex_product(std::vector<Product>& out, const CComb& X, const CComb& Y,
                                const int w4[4], unsigned fa, unsigned fb) {
  const int cx = cls_of(X, fa), cy = cls_of(Y, fb);
  if (cx == CLS_ZERO || cy == CLS_ZERO) return;
  auto L = [&](int part) { return make_factor(X, fa, part); };
  auto R = [&](int part) { return make_factor(Y, fb, part); };
  // (left factor, right factor, coefficient in Re P, coefficient in Im P)
  struct T { Factor l, r; int cre, cim; };
  std::vector<T> terms;
  if (cx == CLS_CX && cy == CLS_CX) {
    // Gauss: P = (T1 - T2) + i (T3 - T1 - T2)
    terms.push_back({L(PART_RE), R(PART_RE), +1, -1});
    terms.push_back({L(PART_IM), R(PART_IM), -1, -1});
    terms.push_back({L(PART_SUM), R(PART_SUM), 0, +1});
  } else if (cx == CLS_RE) {
    if (cy & CLS_RE) terms.push_back({L(PART_RE), R(PART_RE), +1, 0});
    if (cy & CLS_IM) terms.push_back({L(PART_RE), R(PART_IM), 0, +1});
  } else if (cx == CLS_IM) {
    if (cy & CLS_IM) terms.push_back({L(PART_IM), R(PART_IM), -1, 0});
    if (cy & CLS_RE) terms.push_back({L(PART_IM), R(PART_RE), 0, +1});
  } else if (cy == CLS_RE) {  // X complex, Y real
    terms.push_back({L(PART_RE), R(PART_RE), +1, 0});
    terms.push_back({L(PART_IM), R(PART_RE), 0, +1});
  } else {                    // X complex, Y imaginary
    terms.push_back({L(PART_IM), R(PART_IM), -1, 0});
    terms.push_back({L(PART_RE), R(PART_IM), 0, +1});
  }
  for (const T& t : terms) {
    Product p;
    p.l = t.l;
    p.r = t.r;
    for (int e = 0; e < 4; ++e) {
      p.w4[e] = w4[e] * t.cre;
      p.w4[e + 4] = w4[e] * t.cim;
    }
    out.push_back(p);
  }
}

// The paper's bilinear scheme, Eq. bilinearH: left/right complex factors of
// P1..P8 and the weights (times 4) of P_r in Q_1..Q_4.
inline void bilinear_tables(CComb X[8], CComb Y[8], int w4[8][4]) {
  static const int8_t xs[8][4] = {
      {1, 0, 0, 0},    // P1: M1
      {0, 0, 0, 1},    // P2: M4
      {0, 1, 0, 0},    // P3: M2
      {0, 0, 1, 0},    // P4: M3
      {1, 1, 1, 1},    // P5: M1+M2+M3+M4
      {1, 1, -1, -1},  // P6: M1+M2-M3-M4
      {1, -1, 1, -1},  // P7: M1-M2+M3-M4
      {1, -1, -1, 1}}; // P8: M1-M2-M3+M4
  static const int8_t ys[8][4] = {
      {1, 0, 0, 0},    // P1: N1
      {0, 0, 1, 0},    // P2: N3
      {0, 0, 0, 1},    // P3: N4
      {0, 1, 0, 0},    // P4: N2
      {1, 1, 1, 1}, {1, 1, -1, -1}, {1, -1, 1, -1}, {1, -1, -1, 1}};
  // Q1 = 2P1 - (P5+P6+P7+P8)/4; Q2 = -2P2 + (P5+P6-P7-P8)/4;
  // Q3 = -2P3 + (P5-P6+P7-P8)/4; Q4 = -2P4 + (P5-P6-P7+P8)/4  (times 4 below)
  static const int wt[8][4] = {
      {8, 0, 0, 0}, {0, -8, 0, 0}, {0, 0, -8, 0}, {0, 0, 0, -8},
      {-1, 1, 1, 1}, {-1, 1, -1, -1}, {-1, -1, 1, -1}, {-1, -1, -1, 1}};
  for (int r = 0; r < 8; ++r) {
    for (int e = 0; e < 4; ++e) {
      X[r].x[e] = xs[r][e];
      Y[r].x[e] = ys[r][e];
      w4[r][e] = wt[r][e];
    }
  }
}

// Merge products with identical factors (their weights add) and drop products
// whose weights all vanish.
inline std::vector<Product> merge(const std::vector<Product>& in) {
  std::vector<Product> out;
  for (const Product& p : in) {
    bool merged = false;
    for (Product& q : out) {
      if (q.l == p.l && q.r == p.r) {
        for (int e = 0; e < 8; ++e) q.w4[e] += p.w4[e];
        merged = true;
        break;
      }
    }
    if (!merged) out.push_back(p);
  }
  std::vector<Product> kept;
  for (const Product& p : out) {
    bool any = false;
    for (int e = 0; e < 8; ++e) any |= (p.w4[e] != 0);
    if (any) kept.push_back(p);
  }
  return kept;
}

inline std::vector<Product> bilinear_products(unsigned fa, unsigned fb) {
  CComb X[8], Y[8];
  int w4[8][4];
  bilinear_tables(X, Y, w4);
  std::vector<Product> ps;
  for (int r = 0; r < 8; ++r) add_complex_product(ps, X[r], Y[r], w4[r], fa, fb);
  return merge(ps);
}

// Component-wise terms h[e][f][g] a_f b_g, expanded from the same bilinear
// equations: 4 h[e][f][g] = sum_r w4[r][e] X_r[f] Y_r[g] (each 0 or +-4).
inline std::vector<Product> direct_products(unsigned fa, unsigned fb) {
  CComb X[8], Y[8];
  int w4[8][4];
  bilinear_tables(X, Y, w4);
  std::vector<Product> ps;
  for (int f = 0; f < 4; ++f)
    for (int g = 0; g < 4; ++g) {
      int w[4] = {0, 0, 0, 0};
      bool any = false;
      for (int e = 0; e < 4; ++e) {
        int h = 0;
        for (int r = 0; r < 8; ++r) h += w4[r][e] * X[r].x[f] * Y[r].x[g];
        w[e] = h;
        any |= (h != 0);
      }
      if (!any) continue;
      CComb uf{}, ug{};
      uf.x[f] = 1;
      ug.x[g] = 1;
      add_complex_product(ps, uf, ug, w, fa, fb);
    }
  return merge(ps);
}

// Assign factor slots and groups for one side.
inline bool layout_side(const std::vector<Factor>& uniq, int8_t re[8][4], int8_t im[8][4],
                        int8_t slot[8][3], int32_t* ngroups) {
  std::vector<Factor> groups;
  for (size_t f = 0; f < uniq.size(); ++f) {
    int g = -1;
    for (size_t i = 0; i < groups.size(); ++i)
      if (groups[i].same_group(uniq[f])) { g = (int)i; break; }
    if (g < 0) {
      if (groups.size() >= 8) return false;
      groups.push_back(uniq[f]);
      g = (int)groups.size() - 1;
      std::memcpy(re[g], uniq[f].re, 4);
      std::memcpy(im[g], uniq[f].im, 4);
      slot[g][0] = slot[g][1] = slot[g][2] = -1;
    }
    slot[g][uniq[f].part] = (int8_t)f;
  }
  *ngroups = (int32_t)groups.size();
  return true;
}

}  // namespace detail

namespace detail {
// The component-wise ("standard") algorithm: one real product per pair of
// present components (A_c, B_d) that meets in some output component — 64 for
// full biquaternions, 16 for real quaternions (Sec. III B).  Signs and target
// components come from the same expansion of Eq. bilinearH.
inline std::vector<Product> standard_products(unsigned fa, unsigned fb) {
  CComb X[8], Y[8];
  int w4[8][4];
  bilinear_tables(X, Y, w4);
  std::vector<Product> ps;
  for (int f = 0; f < 4; ++f)
    for (int g = 0; g < 4; ++g) {
      int h[4];
      bool any = false;
      for (int e = 0; e < 4; ++e) {
        int s = 0;
        for (int r = 0; r < 8; ++r) s += w4[r][e] * X[r].x[f] * Y[r].x[g];
        h[e] = s;                      // 4 * (+-1 or 0)
        any |= (s != 0);
      }
      if (!any) continue;
      CComb uf{}, ug{};
      uf.x[f] = 1;
      ug.x[g] = 1;
      // a_f b_g = (Af Bg - Af' Bg') + i (Af Bg' + Af' Bg)   (' = imaginary part)
      const int parts[4][2] = {{PART_RE, PART_RE}, {PART_IM, PART_IM}, {PART_RE, PART_IM}, {PART_IM, PART_RE}};
      const int cre[4] = {+1, -1, 0, 0}, cim[4] = {0, 0, +1, +1};
      for (int t = 0; t < 4; ++t) {
        const int la = parts[t][0], rb = parts[t][1];
        const bool lp = la == PART_RE ? ((fa >> f) & 1u) : ((fa >> (f + 4)) & 1u);
        const bool rp = rb == PART_RE ? ((fb >> g) & 1u) : ((fb >> (g + 4)) & 1u);
        if (!lp || !rp) continue;
        Product p;
        p.l = make_factor(uf, fa, la);
        p.r = make_factor(ug, fb, rb);
        for (int e = 0; e < 4; ++e) {
          p.w4[e] = h[e] * cre[t];
          p.w4[e + 4] = h[e] * cim[t];
        }
        ps.push_back(p);
      }
    }
  return merge(ps);
}
}  // namespace detail

// Algorithms: 0 = the paper's bilinear scheme (or, when cheaper for mixed
// subalgebras, component-wise terms with Gauss's rule); 1 = the component-wise
// ("standard") algorithm with four real products per complex term; 2 = the
// bilinear scheme with each complex product of the full plan formed by four
// real multiplications summed in pairs (four_m_plan; other flag pairs keep
// algorithm 0's plan).
enum { kAlgoBilinear = 0, kAlgoStandard = 1, kAlgoBilinear4M = 2 };

// The four-multiplication form of the paper's full plan g (bilinear_full):
// the same eight complex products P_r of Eq. bilinearH, each as two real
// products of twice the inner dimension instead of Gauss's three (Eq.
// cmplx-3-real-mult):
//   product 2r:     Re P_r = Re X_r Re Y_r - Im X_r Im Y_r,
//   product 2r + 1: Im P_r = Re X_r Im Y_r + Im X_r Re Y_r,
// with P_r's weights w4[r][e] on output components e (real part) and e + 4
// (imaginary part).  Factor slots: group g's Re in slot 2g, its Im in 2g + 1
// (16 per side); no Re + Im factors.  Fewer factor and product planes (16
// instead of 24) for 4/3 of the multiplications.
inline bool four_m_plan(const KPlan& g, KPlan* out) {
  if (!g.bilinear_full || g.nlg != 8 || g.nrg != 8) return false;
  int w4t[8][4];
  detail::CComb X[8], Y[8];
  detail::bilinear_tables(X, Y, w4t);
  KPlan p = g;
  std::memset(p.pl, 0, sizeof(p.pl));
  std::memset(p.pr, 0, sizeof(p.pr));
  std::memset(p.pl2, 0, sizeof(p.pl2));
  std::memset(p.pr2, 0, sizeof(p.pr2));
  std::memset(p.w4, 0, sizeof(p.w4));
  for (int gi = 0; gi < 8; ++gi) {
    p.lslot[gi][0] = (int8_t)(2 * gi);
    p.lslot[gi][1] = (int8_t)(2 * gi + 1);
    p.lslot[gi][2] = -1;
    p.rslot[gi][0] = (int8_t)(2 * gi);
    p.rslot[gi][1] = (int8_t)(2 * gi + 1);
    p.rslot[gi][2] = -1;
  }
  p.nlf = p.nrf = 16;
  p.np = 16;
  p.neg2 = 0;
  for (int r = 0; r < 8; ++r) {
    const int re = 2 * r, im = 2 * r + 1;
    p.pl[re] = (int8_t)(2 * r);       p.pr[re] = (int8_t)(2 * r);         // Re X Re Y
    p.pl2[re] = (int8_t)(2 * r + 1);  p.pr2[re] = (int8_t)(2 * r + 1);    // - Im X Im Y
    p.neg2 |= 1ull << re;
    p.pl[im] = (int8_t)(2 * r);       p.pr[im] = (int8_t)(2 * r + 1);     // Re X Im Y
    p.pl2[im] = (int8_t)(2 * r + 1);  p.pr2[im] = (int8_t)(2 * r);        // + Im X Re Y
    for (int e = 0; e < 4; ++e) {
      p.w4[e][re] = (int8_t)w4t[r][e];
      p.w4[e + 4][im] = (int8_t)w4t[r][e];
    }
  }
  p.four_m = 1;
  *out = p;
  return true;
}

// Build the kernel plan for component activity flags fa (of A) and fb (of B).
inline bool build_plan(unsigned fa, unsigned fb, KPlan* out, int algo = kAlgoBilinear) {
  using namespace detail;
  fa &= 0xFFu;
  fb &= 0xFFu;
  std::vector<Product> chosen;
  int strategy;
  if (algo == kAlgoBilinear4M) {
    KPlan g;
    if (!build_plan(fa, fb, &g, kAlgoBilinear)) return false;
    if (!g.bilinear_full) {
      *out = g;
      return true;
    }
    return four_m_plan(g, out);
  }
  if (algo == kAlgoStandard) {
    chosen = standard_products(fa, fb);
    strategy = 2;
  } else {
    std::vector<Product> bl = bilinear_products(fa, fb);
    std::vector<Product> dr = direct_products(fa, fb);
    const bool use_direct = dr.size() < bl.size();
    chosen = use_direct ? dr : bl;
    strategy = use_direct ? 1 : 0;
  }
  const std::vector<Product>& ps = chosen;
  if (ps.size() > (size_t)kMaxProducts) return false;
  KPlan p;
  std::memset(&p, 0, sizeof(p));
  p.strategy = strategy;
  p.np = (int32_t)ps.size();
  std::vector<Factor> lu, ru;
  auto index_of = [](std::vector<Factor>& v, const Factor& f) {
    for (size_t i = 0; i < v.size(); ++i)
      if (v[i] == f) return (int)i;
    v.push_back(f);
    return (int)v.size() - 1;
  };
  for (size_t i = 0; i < ps.size(); ++i) {
    p.pl[i] = (int8_t)index_of(lu, ps[i].l);
    p.pr[i] = (int8_t)index_of(ru, ps[i].r);
    for (int e = 0; e < 8; ++e) p.w4[e][i] = (int8_t)ps[i].w4[e];
  }
  p.nlf = (int32_t)lu.size();
  p.nrf = (int32_t)ru.size();
  if (!layout_side(lu, p.lre, p.lim, p.lslot, &p.nlg)) return false;
  if (!layout_side(ru, p.rre, p.rim, p.rslot, &p.nrg)) return false;
  // recognise the full bilinear factor groups (enables a butterfly path in the encoder)
  CComb X[8], Y[8];
  int w4t[8][4];
  bilinear_tables(X, Y, w4t);
  auto matches = [](int ng, int8_t re[8][4], int8_t im[8][4], const CComb* C) {
    if (ng != 8) return 0;
    for (int g = 0; g < 8; ++g)
      for (int e = 0; e < 4; ++e)
        if (re[g][e] != C[g].x[e] || im[g][e] != C[g].x[e]) return 0;
    return 1;
  };
  p.bilinear_left = matches(p.nlg, p.lre, p.lim, X);
  p.bilinear_right = matches(p.nrg, p.rre, p.rim, Y);
  if (p.np == 24 && p.bilinear_left && p.bilinear_right) {
    // expected weights: Gauss (T1 -> Re +1, Im -1; T2 -> Re -1, Im -1; T3 -> Im +1)
    // times the weight of P_r in Q_e (Eq. bilinearH, times 4)
    bool ok = true;
    for (int r = 0; r < 8 && ok; ++r) {
      const int gre[3] = {+1, -1, 0}, gim[3] = {-1, -1, +1};
      for (int t = 0; t < 3 && ok; ++t) {
        const int q = 3 * r + t;
        for (int e = 0; e < 4; ++e) {
          ok = ok && (p.w4[e][q] == w4t[r][e] * gre[t]) && (p.w4[e + 4][q] == w4t[r][e] * gim[t]);
        }
        // factors: group r, parts Re / Im / Re+Im on both sides
        ok = ok && (p.pl[q] == p.lslot[r][t]) && (p.pr[q] == p.rslot[r][t]);
      }
    }
    p.bilinear_full = ok ? 1 : 0;
  }
  *out = p;
  return true;
}

// Sign of stored component c under op (Sec. III op equations; QC = vector part negated).
inline int op_sign(int op, int c) {
  static const int8_t m[5][8] = {
      {+1, +1, +1, +1, +1, +1, +1, +1},   // N
      {+1, +1, -1, +1, +1, +1, -1, +1},   // T
      {+1, -1, +1, -1, -1, +1, -1, +1},   // C (complex conjugate)
      {+1, -1, -1, -1, -1, +1, +1, +1},   // H (dagger)
      {+1, -1, -1, -1, +1, -1, -1, -1}};  // QC (quaternion conjugate)
  return m[op][c];
}
inline bool op_transposes(int op) { return op == 1 || op == 3; }

// Coefficient of stored component c in left (side 0) or right (side 1) factor
// slot f, op signs folded in (for tests and hmat_plan_info).
inline void factor_row(const KPlan& p, int side, int f, int op, int8_t row[8]) {
  const int ng = side ? p.nrg : p.nlg;
  for (int c = 0; c < 8; ++c) row[c] = 0;
  for (int g = 0; g < ng; ++g) {
    const int8_t* slot = side ? p.rslot[g] : p.lslot[g];
    const int8_t* re = side ? p.rre[g] : p.lre[g];
    const int8_t* im = side ? p.rim[g] : p.lim[g];
    for (int part = 0; part < 3; ++part) {
      if (slot[part] != f) continue;
      for (int e = 0; e < 4; ++e) {
        if (part != 1) row[e] = (int8_t)(re[e] * op_sign(op, e));
        if (part != 0) row[e + 4] = (int8_t)(im[e] * op_sign(op, e + 4));
      }
    }
  }
}

}  // namespace hmat
