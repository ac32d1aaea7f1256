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
// Output: a C++ header on stdout.
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

namespace {

struct Rat {
  long long n = 0, d = 1;
};
long long gabs(long long a) { return a < 0 ? -a : a; }
long long ggcd(long long a, long long b) {
  a = gabs(a);
  b = gabs(b);
  while (b) {
    long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}
Rat mk(long long n, long long d) {
  if (d < 0) { n = -n; d = -d; }
  long long g = ggcd(n, d);
  if (g == 0) g = 1;
  return Rat{n / g, d / g};
}
Rat operator*(Rat a, Rat b) {
  long long g1 = ggcd(a.n, b.d), g2 = ggcd(b.n, a.d);
  if (g1 == 0) g1 = 1;
  if (g2 == 0) g2 = 1;
  return mk((a.n / g1) * (b.n / g2), (a.d / g2) * (b.d / g1));
}
Rat operator+(Rat a, Rat b) {
  long long g = ggcd(a.d, b.d);
  return mk(a.n * (b.d / g) + b.n * (a.d / g), (a.d / g) * b.d);
}
Rat operator-(Rat a, Rat b) { return a + Rat{-b.n, b.d}; }
double dbl(Rat a) { return (double)a.n / (double)a.d; }

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

long long fact(int n) {
  long long r = 1;
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
      long long num = 1;
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

void emit(int D, int p, int form) {
  const int q = form == 0 ? 2 * p : 2 * p - 2;
  const int NB = form == 0 ? 1 : D;
  auto V = multi(D, p), W = multi(D, q);
  if (q == 0) W = {std::vector<int>(D, 0)};
  const int VT = (int)V.size(), WT = (int)W.size();
  std::vector<double> B((size_t)NB * WT * VT);
  long long nnz = 0, nnz1 = 0;
  for (int j = 0; j < WT; ++j) {
    auto lam = bary_of_node(D, q, W[j]);
    for (int l = 0; l < VT; ++l) {
      auto be = beta_of(D, p, V[l]);
      std::vector<Rat> vals(NB);
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
      for (int r = 0; r < NB; ++r) {
        B[((size_t)r * WT + j) * VT + l] = dbl(vals[r]);
        if (vals[r].n != 0) ++nnz;
        if (gabs(vals[r].n) == 1 && vals[r].d == 1) ++nnz1;
      }
    }
  }
  auto w = w_integrals(D, q);
  auto iv = w_integrals(D, p);
  std::printf("template <> struct Tab<%d, %d, %d> {\n", D, p, form);
  std::printf("  static constexpr int D = %d, P = %d, FORM = %d, Q = %d;\n", D, p, form, q);
  std::printf("  static constexpr int V = %d, W = %d, NB = %d;\n", VT, WT, NB);
  std::printf("  static constexpr long long NNZ = %lld, NNZ1 = %lld;\n", nnz, nnz1);
  std::printf("  static constexpr double B[%d][%d][%d] = {", NB, WT, VT);
  for (size_t i = 0; i < B.size(); ++i) std::printf("%s%.17g", i ? "," : "", B[i]);
  std::printf("};\n  static constexpr double w[%d] = {", WT);
  for (int j = 0; j < WT; ++j) std::printf("%s%.17g", j ? "," : "", dbl(w[j]));
  std::printf("};\n  static constexpr double iv[%d] = {", VT);
  for (int l = 0; l < VT; ++l) std::printf("%s%.17g", l ? "," : "", dbl(iv[l]));
  std::printf("};\n};\n");
}

}  // namespace

int main(int argc, char** argv) {
  int pmax2 = argc > 1 ? std::atoi(argv[1]) : 4;
  int pmax3 = argc > 2 ? std::atoi(argv[2]) : 4;
  std::printf("// Generated by gen_tables.cpp at build time.  Do not edit.\n");
  std::printf("#pragma once\nnamespace dogip_tab {\n");
  std::printf("template <int D, int P, int FORM> struct Tab;\n");
  std::printf("constexpr int PMAX2 = %d, PMAX3 = %d;\n", pmax2, pmax3);
  for (int D = 2; D <= 3; ++D)
    for (int p = 1; p <= (D == 2 ? pmax2 : pmax3); ++p)
      for (int form = 0; form < 2; ++form) emit(D, p, form);
  std::printf("}  // namespace dogip_tab\n");
  return 0;
}
