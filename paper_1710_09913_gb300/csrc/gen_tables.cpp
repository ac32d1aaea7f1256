// Build-time generator of the reference-element tables baked into the kernels.
//
// For every (d, p, form) it evaluates, in exact rational arithmetic,
//   projection (Theorem "element-wise DoGIP for weighted projection"):
//       B[0][j][l] = phi_l(x_j),          W = P_{2p} on the reference simplex
//   elliptic (Theorem "element-wise DoGIP for the elliptic problem"):
//       B[r][j][l] = d phi_l / d xhat_r (x_j),  W = P_{2p-2}
// with phi_l the equispaced P_p Lagrange basis in Silvester's product form
//   phi_beta(lambda) = prod_i prod_{m < beta_i} (p lambda_i - m) / (m + 1),
// and the W-basis integrals w_j = int_That phi^W_j, expanded in barycentric
// monomials and integrated with int_That lambda^k = prod k_i! / (|k| + d)!.
// Each exact value is rounded once to double (correct rounding of n / d).
//
// For the quadrature-point matrix-free comparator it also emits TabQ<d, p, form>:
// the same basis values / reference gradients at the points of the collapsed
// Gauss-Jacobi rule with n points per direction (n = p + 1 for the mass integrand
// of degree 2p, n = p for the stiffness integrand of degree 2p - 2; exact for
// element-constant coefficients), evaluated in double, and the rule's weights.
// Output: a C++ header on stdout.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "quad.h"

namespace {

using I128 = __int128;
using U128 = unsigned __int128;

struct Rat {
  I128 n = 0, d = 1;
};
[[noreturn]] void overflow() {
  std::fprintf(stderr, "gen_tables: rational overflow\n");
  std::exit(2);
}
I128 gabs(I128 a) { return a < 0 ? -a : a; }
I128 ggcd(I128 a, I128 b) {
  a = gabs(a);
  b = gabs(b);
  while (b) {
    I128 t = a % b;
    a = b;
    b = t;
  }
  return a;
}
I128 mul(I128 a, I128 b) {
  I128 r;
  if (__builtin_mul_overflow(a, b, &r)) overflow();
  return r;
}
I128 add(I128 a, I128 b) {
  I128 r;
  if (__builtin_add_overflow(a, b, &r)) overflow();
  return r;
}
Rat mk(I128 n, I128 d) {
  if (d < 0) { n = -n; d = -d; }
  I128 g = ggcd(n, d);
  if (g == 0) g = 1;
  return Rat{n / g, d / g};
}
Rat operator*(Rat a, Rat b) {
  I128 g1 = ggcd(a.n, b.d), g2 = ggcd(b.n, a.d);
  if (g1 == 0) g1 = 1;
  if (g2 == 0) g2 = 1;
  return mk(mul(a.n / g1, b.n / g2), mul(a.d / g2, b.d / g1));
}
Rat operator+(Rat a, Rat b) {
  I128 g = ggcd(a.d, b.d);
  return mk(add(mul(a.n, b.d / g), mul(b.n, a.d / g)), mul(a.d / g, b.d));
}
Rat operator-(Rat a, Rat b) { return a + Rat{-b.n, b.d}; }

// n / d rounded once to the nearest double (ties to even): binary long division to
// 55 significant bits plus a sticky bit.
double dbl(Rat a) {
  if (a.n == 0) return 0.0;
  const bool neg = a.n < 0;
  U128 n = (U128)(neg ? -a.n : a.n), d = (U128)a.d;
  U128 q = n / d, r = n % d;
  auto bitlen = [](U128 x) {
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
  };
  if (bitlen(q) > 55) overflow();  // table values are far below 2^55
  uint64_t m = (uint64_t)q;
  int e = 0;
  while (bitlen(m) < 55) {
    r <<= 1;  // r < d < 2^127
    const uint64_t bit = r >= d ? 1u : 0u;
    if (bit) r -= d;
    m = (m << 1) | bit;
    --e;
  }
  const bool sticky = r != 0;
  uint64_t mant = m >> 2;
  const unsigned rem = (unsigned)(m & 3u);
  if (rem > 2 || (rem == 2 && (sticky || (mant & 1u)))) ++mant;
  const double v = std::ldexp((double)mant, e + 2);
  return neg ? -v : v;
}

int binom(int n, int k) {
  long long r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return (int)r;
}

// Multi-indices |a| <= q, product order with the last coordinate fastest.
std::vector<std::vector<int>> multi(int D, int q) {
  std::vector<std::vector<int>> out;
  std::vector<int> a(D, 0);
  int lim = q + 1, tot = 1;
  for (int i = 0; i < D; ++i) tot *= lim;
  for (int c = 0; c < tot; ++c) {
    int t = c, s = 0;
    for (int i = D - 1; i >= 0; --i) { a[i] = t % lim; t /= lim; s += a[i]; }
    if (s <= q) out.push_back(a);
  }
  return out;
}

// P_b(t) = prod_{m<b} (p t - m)/(m+1) and its derivative, at rational t.
Rat fac(int p, int b, Rat t) {
  Rat v{1, 1};
  for (int m = 0; m < b; ++m) v = v * (mk(p, 1) * t - mk(m, 1)) * mk(1, m + 1);
  return v;
}
Rat dfac(int p, int b, Rat t) {
  Rat s{0, 1};
  for (int m = 0; m < b; ++m) {
    Rat term = mk(p, m + 1);
    for (int j = 0; j < b; ++j)
      if (j != m) term = term * (mk(p, 1) * t - mk(j, 1)) * mk(1, j + 1);
    s = s + term;
  }
  return s;
}

std::vector<Rat> bary_of_node(int D, int q, const std::vector<int>& a) {
  std::vector<Rat> lam(D + 1);
  if (q == 0) {
    for (int i = 0; i <= D; ++i) lam[i] = mk(1, D + 1);  // centroid
    return lam;
  }
  int s = 0;
  for (int i = 0; i < D; ++i) { lam[i + 1] = mk(a[i], q); s += a[i]; }
  lam[0] = mk(q - s, q);
  return lam;
}

std::vector<int> beta_of(int D, int p, const std::vector<int>& a) {
  std::vector<int> b(D + 1);
  int s = 0;
  for (int i = 0; i < D; ++i) { b[i + 1] = a[i]; s += a[i]; }
  b[0] = p - s;
  return b;
}

// Coefficients (ascending) of P_b(t) as a polynomial in t.
std::vector<Rat> poly(int q, int b) {
  std::vector<Rat> c{Rat{1, 1}};
  for (int m = 0; m < b; ++m) {
    std::vector<Rat> nc(c.size() + 1, Rat{0, 1});
    for (size_t k = 0; k < c.size(); ++k) {
      nc[k + 1] = nc[k + 1] + c[k] * mk(q, m + 1);
      nc[k] = nc[k] - c[k] * mk(m, m + 1);
    }
    c = nc;
  }
  return c;
}

I128 fact(int n) {
  I128 r = 1;
  for (int i = 2; i <= n; ++i) r *= i;
  return r;
}

// int_That phi^W (degree q) for every W node.
std::vector<Rat> w_integrals(int D, int q) {
  std::vector<Rat> out;
  if (q == 0) { out.push_back(mk(1, fact(D))); return out; }
  for (auto& a : multi(D, q)) {
    auto be = beta_of(D, q, a);
    std::vector<std::vector<Rat>> P;
    for (int i = 0; i <= D; ++i) P.push_back(poly(q, be[i]));
    Rat s{0, 1};
    std::vector<int> k(D + 1, 0);
    while (true) {
      Rat c{1, 1};
      int tot = 0;
      I128 num = 1;
      for (int i = 0; i <= D; ++i) { c = c * P[i][k[i]]; tot += k[i]; num *= fact(k[i]); }
      if (c.n != 0) s = s + c * mk(num, fact(tot + D));
      int i = D;
      while (i >= 0 && ++k[i] == (int)P[i].size()) { k[i] = 0; --i; }
      if (i < 0) break;
    }
    out.push_back(s);
  }
  return out;
}

struct Tables {
  int VT = 0, WT = 0, NB = 0, q = 0;
  long long nnz = 0, nnz1 = 0;
  std::vector<double> B, w, iv;
};

Tables compute(int D, int p, int form) {
  Tables t;
  t.q = form == 0 ? 2 * p : 2 * p - 2;
  t.NB = form == 0 ? 1 : D;
  auto V = multi(D, p), W = multi(D, t.q);
  if (t.q == 0) W = {std::vector<int>(D, 0)};
  t.VT = (int)V.size();
  t.WT = (int)W.size();
  t.B.assign((size_t)t.NB * t.WT * t.VT, 0.0);
  for (int j = 0; j < t.WT; ++j) {
    auto lam = bary_of_node(D, t.q, W[j]);
    for (int l = 0; l < t.VT; ++l) {
      auto be = beta_of(D, p, V[l]);
      std::vector<Rat> vals(t.NB);
      if (form == 0) {
        Rat v{1, 1};
        for (int i = 0; i <= D; ++i) v = v * fac(p, be[i], lam[i]);
        vals[0] = v;
      } else {
        std::vector<Rat> dl(D + 1);
        for (int i = 0; i <= D; ++i) {
          Rat v = dfac(p, be[i], lam[i]);
          for (int k = 0; k <= D; ++k)
            if (k != i) v = v * fac(p, be[k], lam[k]);
          dl[i] = v;
        }
        for (int r = 0; r < D; ++r) vals[r] = dl[r + 1] - dl[0];
      }
      for (int r = 0; r < t.NB; ++r) {
        t.B[((size_t)r * t.WT + j) * t.VT + l] = dbl(vals[r]);
        if (vals[r].n != 0) ++t.nnz;
        if (gabs(vals[r].n) == 1 && vals[r].d == 1) ++t.nnz1;
      }
    }
  }
  for (auto& x : w_integrals(D, t.q)) t.w.push_back(dbl(x));
  for (auto& x : w_integrals(D, p)) t.iv.push_back(dbl(x));
  return t;
}

void print_array(const char* name, const std::vector<double>& v) {
  std::printf("static const double %s[%zu] = {", name, v.size());
  for (size_t i = 0; i < v.size(); ++i) std::printf("%s%.17g", i ? "," : "", v[i]);
  std::printf("};\n");
}

void emit(int D, int p, int form) {
  const Tables t = compute(D, p, form);
  std::printf("template <> struct Tab<%d, %d, %d> {\n", D, p, form);
  std::printf("  static constexpr int D = %d, P = %d, FORM = %d, Q = %d;\n", D, p, form, t.q);
  std::printf("  static constexpr int V = %d, W = %d, NB = %d;\n", t.VT, t.WT, t.NB);
  std::printf("  static constexpr long long NNZ = %lld, NNZ1 = %lld;\n", t.nnz, t.nnz1);
  std::printf("  static constexpr double B[%d][%d][%d] = {", t.NB, t.WT, t.VT);
  for (size_t i = 0; i < t.B.size(); ++i) std::printf("%s%.17g", i ? "," : "", t.B[i]);
  std::printf("};\n  static constexpr double w[%d] = {", t.WT);
  for (int j = 0; j < t.WT; ++j) std::printf("%s%.17g", j ? "," : "", t.w[j]);
  std::printf("};\n  static constexpr double iv[%d] = {", t.VT);
  for (int l = 0; l < t.VT; ++l) std::printf("%s%.17g", l ? "," : "", t.iv[l]);
  std::printf("};\n};\n");
}

// Runtime tables of the higher orders served by the generic kernels (plain arrays).
void emit_hi(int pmin2, int pmax2, int pmin3, int pmax3) {
  std::printf("// Generated by gen_tables.cpp at build time.  Do not edit.\n");
  std::printf("#pragma once\nnamespace dogip_hi {\n");
  std::printf("struct HiTab {\n  int d, p, form, V, W, NB;\n  long long nnz, nnz1;\n"
              "  const double* B;\n  const double* w;\n  const double* iv;\n};\n");
  std::vector<std::string> rows;
  for (int D = 2; D <= 3; ++D)
    for (int p = (D == 2 ? pmin2 : pmin3); p <= (D == 2 ? pmax2 : pmax3); ++p)
      for (int form = 0; form < 2; ++form) {
        const Tables t = compute(D, p, form);
        char nb[64], nw[64], ni[64], row[512];
        std::snprintf(nb, sizeof nb, "B_%d_%d_%d", D, p, form);
        std::snprintf(nw, sizeof nw, "w_%d_%d_%d", D, p, form);
        std::snprintf(ni, sizeof ni, "iv_%d_%d_%d", D, p, form);
        print_array(nb, t.B);
        print_array(nw, t.w);
        print_array(ni, t.iv);
        std::snprintf(row, sizeof row, "  {%d, %d, %d, %d, %d, %d, %lld, %lld, %s, %s, %s},", D, p,
                      form, t.VT, t.WT, t.NB, t.nnz, t.nnz1, nb, nw, ni);
        rows.push_back(row);
      }
  std::printf("static const HiTab kHiTabs[] = {\n");
  for (auto& r : rows) std::printf("%s\n", r.c_str());
  std::printf("};\nconstexpr int kNumHi = %zu;\n}  // namespace dogip_hi\n", rows.size());
}

// Double-precision versions of fac / dfac for irrational points.
double facd(int p, int b, double t) {
  double v = 1.0;
  for (int m = 0; m < b; ++m) v *= (p * t - m) / (m + 1);
  return v;
}
double dfacd(int p, int b, double t) {
  double s = 0.0;
  for (int m = 0; m < b; ++m) {
    double term = (double)p / (m + 1);
    for (int j = 0; j < b; ++j)
      if (j != m) term *= (p * t - j) / (j + 1);
    s += term;
  }
  return s;
}

void emit_qp(int D, int p, int form) {
  const int n = form == 0 ? p + 1 : p;
  const int NB = form == 0 ? 1 : D;
  std::vector<double> pts, wts;
  dogip::simplex_rule(D, n, pts, wts);
  const int QT = (int)wts.size();
  auto V = multi(D, p);
  const int VT = (int)V.size();
  std::vector<double> B((size_t)NB * QT * VT);
  for (int j = 0; j < QT; ++j) {
    double lam[4];
    lam[0] = 1.0;
    for (int i = 0; i < D; ++i) {
      lam[i + 1] = pts[(size_t)j * D + i];
      lam[0] -= lam[i + 1];
    }
    for (int l = 0; l < VT; ++l) {
      auto be = beta_of(D, p, V[l]);
      double vals[3];
      if (form == 0) {
        double v = 1.0;
        for (int i = 0; i <= D; ++i) v *= facd(p, be[i], lam[i]);
        vals[0] = v;
      } else {
        double dl[4];
        for (int i = 0; i <= D; ++i) {
          double v = dfacd(p, be[i], lam[i]);
          for (int k = 0; k <= D; ++k)
            if (k != i) v *= facd(p, be[k], lam[k]);
          dl[i] = v;
        }
        for (int r = 0; r < D; ++r) vals[r] = dl[r + 1] - dl[0];
      }
      for (int r = 0; r < NB; ++r) B[((size_t)r * QT + j) * VT + l] = vals[r];
    }
  }
  std::printf("template <> struct TabQ<%d, %d, %d> {\n", D, p, form);
  std::printf("  static constexpr int D = %d, P = %d, FORM = %d, N1 = %d;\n", D, p, form, n);
  std::printf("  static constexpr int V = %d, W = %d, NB = %d;\n", VT, QT, NB);
  std::printf("  static constexpr double B[%d][%d][%d] = {", NB, QT, VT);
  for (size_t i = 0; i < B.size(); ++i) std::printf("%s%.17g", i ? "," : "", B[i]);
  std::printf("};\n  static constexpr double w[%d] = {", QT);
  for (int j = 0; j < QT; ++j) std::printf("%s%.17g", j ? "," : "", wts[j]);
  std::printf("};\n};\n");
}

}  // namespace

int main(int argc, char** argv) {
  if (argc > 1 && std::string(argv[1]) == "--hi") {
    // --hi pmin2 pmax2 pmin3 pmax3
    emit_hi(std::atoi(argv[2]), std::atoi(argv[3]), std::atoi(argv[4]), std::atoi(argv[5]));
    return 0;
  }
  int pmax2 = argc > 1 ? std::atoi(argv[1]) : 4;
  int pmax3 = argc > 2 ? std::atoi(argv[2]) : 4;
  std::printf("// Generated by gen_tables.cpp at build time.  Do not edit.\n");
  std::printf("#pragma once\nnamespace dogip_tab {\n");
  std::printf("template <int D, int P, int FORM> struct Tab;\n");
  std::printf("template <int D, int P, int FORM> struct TabQ;\n");
  std::printf("constexpr int PMAX2 = %d, PMAX3 = %d;\n", pmax2, pmax3);
  for (int D = 2; D <= 3; ++D)
    for (int p = 1; p <= (D == 2 ? pmax2 : pmax3); ++p)
      for (int form = 0; form < 2; ++form) {
        emit(D, p, form);
        emit_qp(D, p, form);
      }
  std::printf("}  // namespace dogip_tab\n");
  return 0;
}
