// Solid harmonics and the FMM translation operators (host, FP64, setup only).
//
// The paper applies "FMM [22], [23]" to the panel potentials (Sec. II-C)
// without fixing an expansion; this library uses complex solid harmonics
// with the Condon-Shortley phase,
//   Y_n^m(r) = r^n P_n^m(cos t) e^{i m phi} / (n+m)!      (regular)
//   T_n^m(r) = (n-m)! P_n^m(cos t) e^{i m phi} / r^{n+1}  (irregular)
// for which 1/|x - y| = sum conj(Y_n^m(y)) T_n^m(x)  (|y| < |x|),
//   Y_n^m(a + b) = sum_{k,l} Y_k^l(a) Y_{n-k}^{m-l}(b), and
//   T_n^m(x - y) = sum_{k,l} conj(Y_k^l(y)) T_{n+k}^{m+l}(x).
// With coefficients scaled by the box size h (M~_n = M_n / h^n,
// L~_n = L_n h^{n+1}) every operator is level independent:
//   M2M  M~_n^m(parent) = sum 2^-k M~_k^l(child) conj(Y_{n-k}^{m-l}(d))
//   L2L  L~_k^l(child)  = 2^-(k+1) sum_{n>=k} L~_n^m(parent) Y_{n-k}^{m-l}(d)
//   M2L  L~_k^l = (-1)^{k+l} sum_{n,m} M~_n^m T_{n+k}^{m-l}(t)
// with d = (child centre - parent centre) / h_parent and t = (target centre -
// source centre) / h (an integer vector).  Sources are real, so
// C_n^{-m} = (-1)^m conj(C_n^m) and only m >= 0 is stored: the real vector
// of length (p+1)^2 holds, per n, [Re C_n^0, Re C_n^1, Im C_n^1, ...,
// Re C_n^n, Im C_n^n].  Each operator is stored as a real matrix built by
// applying the complex formula to the real unit vectors, TRANSPOSED
// (element [in][out]) so that kernels read it coalesced.
#include <cmath>
#include <complex>
#include <vector>
#include <algorithm>

#include "xrl_internal.hpp"

namespace xrl {

using cd = std::complex<double>;

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  // Newton iteration on P_n from Chebyshev-like initial guesses; nodes on [0,1], ascending.
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = std::cos(pi * (i + 0.75) / (n + 0.5));
    double pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p2 = p1;
        p1 = p0;
        p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
      }
      pp = n * (z * p0 - p1) / (z * z - 1.0);
      double dz = p0 / pp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    // recompute derivative at the converged node
    double p0 = 1.0, p1 = 0.0;
    for (int j = 1; j <= n; ++j) {
      double p2 = p1;
      p1 = p0;
      p0 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p2) / j;
    }
    pp = n * (z * p0 - p1) / (z * z - 1.0);
    x[i] = 0.5 * (1.0 + z);
    w[i] = 1.0 / ((1.0 - z * z) * pp * pp);   // (2 / ((1-z^2) P'^2)) / 2 on [0,1]
  }
  // ascending order
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return x[a] < x[b]; });
  std::vector<double> xs(n), ws(n);
  for (int i = 0; i < n; ++i) {
    xs[i] = x[idx[i]];
    ws[i] = w[idx[i]];
  }
  x = xs;
  w = ws;
}

namespace {

struct Harm {
  int P;
  std::vector<cd> v;  // [(P+1)][(2P+1)]
  explicit Harm(int P_) : P(P_), v((P_ + 1) * (2 * P_ + 1)) {}
  cd& at(int n, int m) { return v[n * (2 * P + 1) + P + m]; }
  cd get(int n, int m) const { return v[n * (2 * P + 1) + P + m]; }
};

Harm regular(const double r[3], int P) {
  Harm Y(P);
  cd xy(r[0], r[1]);
  double z = r[2], r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  Y.at(0, 0) = 1.0;
  for (int m = 0; m <= P; ++m) {
    if (m > 0) Y.at(m, m) = -xy / (2.0 * m) * Y.at(m - 1, m - 1);
    for (int n = m + 1; n <= P; ++n) {
      cd prev2 = (n - 2 >= m) ? Y.at(n - 2, m) : cd(0.0);
      Y.at(n, m) = ((2.0 * n - 1.0) * z * Y.at(n - 1, m) - r2 * prev2) / double((n + m) * (n - m));
    }
  }
  for (int n = 0; n <= P; ++n)
    for (int m = 1; m <= n; ++m) Y.at(n, -m) = ((m & 1) ? -1.0 : 1.0) * std::conj(Y.at(n, m));
  return Y;
}

Harm irregular(const double r[3], int P) {
  Harm T(P);
  cd xy(r[0], r[1]);
  double z = r[2], r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
  T.at(0, 0) = 1.0 / std::sqrt(r2);
  for (int m = 0; m <= P; ++m) {
    if (m > 0) T.at(m, m) = -(2.0 * m - 1.0) * xy / r2 * T.at(m - 1, m - 1);
    for (int n = m + 1; n <= P; ++n) {
      cd prev2 = (n - 2 >= m) ? T.at(n - 2, m) : cd(0.0);
      T.at(n, m) = ((2.0 * n - 1.0) * z * T.at(n - 1, m) -
                    double((n + m - 1) * (n - m - 1)) * prev2) / r2;
    }
  }
  for (int n = 0; n <= P; ++n)
    for (int m = 1; m <= n; ++m) T.at(n, -m) = ((m & 1) ? -1.0 : 1.0) * std::conj(T.at(n, m));
  return T;
}

inline int ridx(int n, int m, int part) { return m == 0 ? n * n : n * n + 2 * m - 1 + part; }

struct NZ {
  int n, m;
  cd v;
};

Harm from_real(const double* r, int P) {
  Harm C(P);
  for (int n = 0; n <= P; ++n) {
    C.at(n, 0) = cd(r[ridx(n, 0, 0)], 0.0);
    for (int m = 1; m <= n; ++m) {
      cd v(r[ridx(n, m, 0)], r[ridx(n, m, 1)]);
      C.at(n, m) = v;
      C.at(n, -m) = ((m & 1) ? -1.0 : 1.0) * std::conj(v);
    }
  }
  return C;
}

void to_real(const Harm& C, double* r) {
  int P = C.P;
  for (int n = 0; n <= P; ++n) {
    r[ridx(n, 0, 0)] = C.get(n, 0).real();
    for (int m = 1; m <= n; ++m) {
      r[ridx(n, m, 0)] = C.get(n, m).real();
      r[ridx(n, m, 1)] = C.get(n, m).imag();
    }
  }
}

std::vector<NZ> nonzeros(const Harm& C) {
  std::vector<NZ> out;
  for (int n = 0; n <= C.P; ++n)
    for (int m = -n; m <= n; ++m)
      if (C.get(n, m) != cd(0.0)) out.push_back({n, m, C.get(n, m)});
  return out;
}

}  // namespace

void build_translations(int p, const std::vector<int32_t>& offsets, std::vector<double>& m2m,
                        std::vector<double>& l2l, std::vector<double>& m2l) {
  const int nc = (p + 1) * (p + 1);
  const int noff = (int)offsets.size() / 3;
  m2m.assign(8 * nc * nc, 0.0);
  l2l.assign(8 * nc * nc, 0.0);
  m2l.assign((size_t)noff * nc * nc, 0.0);
  std::vector<double> e(nc), out(nc);
  for (int o = 0; o < 8; ++o) {
    double d[3] = {(o & 1) ? 0.25 : -0.25, (o & 2) ? 0.25 : -0.25, (o & 4) ? 0.25 : -0.25};
    Harm Yd = regular(d, p);
    for (int j = 0; j < nc; ++j) {
      std::fill(e.begin(), e.end(), 0.0);
      e[j] = 1.0;
      Harm Mc = from_real(e.data(), p);
      std::vector<NZ> nz = nonzeros(Mc);
      // M2M
      Harm Mp(p);
      for (int n = 0; n <= p; ++n)
        for (int m = -n; m <= n; ++m) {
          cd s = 0.0;
          for (const NZ& q : nz)
            if (q.n <= n && std::abs(m - q.m) <= n - q.n)
              s += std::ldexp(1.0, -q.n) * q.v * std::conj(Yd.get(n - q.n, m - q.m));
          Mp.at(n, m) = s;
        }
      to_real(Mp, out.data());
      for (int i = 0; i < nc; ++i) m2m[(size_t)o * nc * nc + (size_t)j * nc + i] = out[i];
      // L2L (the unit vector is now a parent local expansion)
      Harm Lc(p);
      for (int k = 0; k <= p; ++k)
        for (int l = -k; l <= k; ++l) {
          cd s = 0.0;
          for (const NZ& q : nz)
            if (q.n >= k && std::abs(q.m - l) <= q.n - k) s += q.v * Yd.get(q.n - k, q.m - l);
          Lc.at(k, l) = std::ldexp(1.0, -(k + 1)) * s;
        }
      to_real(Lc, out.data());
      for (int i = 0; i < nc; ++i) l2l[(size_t)o * nc * nc + (size_t)j * nc + i] = out[i];
    }
  }
  for (int code = 0; code < noff; ++code) {
        double t[3] = {(double)offsets[3 * code], (double)offsets[3 * code + 1], (double)offsets[3 * code + 2]};
        Harm T = irregular(t, 2 * p);
        for (int j = 0; j < nc; ++j) {
          std::fill(e.begin(), e.end(), 0.0);
          e[j] = 1.0;
          std::vector<NZ> nz = nonzeros(from_real(e.data(), p));
          Harm L(p);
          for (int k = 0; k <= p; ++k)
            for (int l = -k; l <= k; ++l) {
              cd s = 0.0;
              for (const NZ& q : nz) s += q.v * T.get(q.n + k, q.m - l);
              L.at(k, l) = (((k + l) & 1) ? -1.0 : 1.0) * s;
            }
          to_real(L, out.data());
          for (int i = 0; i < nc; ++i) m2l[(size_t)code * nc * nc + (size_t)j * nc + i] = out[i];
        }
      }
}

}  // namespace xrl
