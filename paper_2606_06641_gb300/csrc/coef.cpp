// Load-time DFT coefficient tables (host, FP64, rounded once to FP32).
//
// Sec. 2.1.2: a symmetric constraint's expansion is evaluated from products
// of one factor per literal at the k+1 roots of unity, combined with the
// constraint's DFT coefficients. Sec. 3.5: roots are built so that paired
// roots are exact conjugates, combinatorial terms are exact integers with the
// division deferred, and mirrored terms are copied rather than recomputed.
#include "coef.h"

#include <algorithm>
#include <cmath>
#include <stdexcept>

namespace afs {

bool Shape::operator<(const Shape& o) const {
  if (type != o.type) return type < o.type;
  if (k != o.k) return k < o.k;
  if (op != o.op) return op < o.op;
  if (param != o.param) return param < o.param;
  return parity < o.parity;
}
bool Shape::operator==(const Shape& o) const {
  return type == o.type && k == o.k && op == o.op && param == o.param && parity == o.parity;
}

// Table 1 and Appendix A: -1 where the constraint holds with t true literals.
void truth_table(const Shape& s, std::vector<int8_t>& f) {
  f.assign(s.k + 1, 1);
  for (int t = 0; t <= s.k; ++t) {
    bool sat = false;
    switch (s.type) {
      case 0: sat = t >= 1; break;                                       // OR
      case 1: sat = (t & 1) == (s.parity ? 1 : 0); break;                // XOR
      case 2: sat = t > 0 && t < s.k; break;                             // NAE
      case 3: sat = t <= 1; break;                                       // AMO
      case 4: sat = t == 1; break;                                       // EO
      case 5: sat = t == s.param; break;                                 // EK
      case 6: sat = s.op == 0 ? t >= s.param : t < s.param; break;       // CARD
      default: throw std::invalid_argument("constraint type");
    }
    f[t] = sat ? -1 : 1;
  }
}

// cos and sin of 2*pi*r/M. The angle is reduced with integers to a multiple
// of pi/2 plus |phi| <= pi/4, so that r and M-r give exact conjugates (the
// mirrored roots of Sec. 3.5) and no repeated exponentiation is involved.
static void unit_root(long long r, long long M, double& c, double& s) {
  r %= M;
  if (r < 0) r += M;
  const long long num = 8 * r;
  const long long q = num / M;
  const long long rem = num - q * M;
  long long quarter;
  double phi;
  if ((q & 1) == 0) {
    quarter = q / 2;
    phi = (M_PI / 4.0) * (static_cast<double>(rem) / static_cast<double>(M));
  } else {
    quarter = (q + 1) / 2;
    phi = -(M_PI / 4.0) * (static_cast<double>(M - rem) / static_cast<double>(M));
  }
  const double cp = std::cos(phi), sp = std::sin(phi);
  switch (quarter & 3) {
    case 0: c = cp; s = sp; break;
    case 1: c = -sp; s = cp; break;
    case 2: c = -cp; s = -sp; break;
    default: c = sp; s = -cp; break;
  }
}

// ---- exact integer combinatorics for f_hat(|S| = d) ------------------------
// Fixed-width two's-complement integers in 64-bit limbs.
namespace {
struct BigVec {
  int W;
  std::vector<uint64_t> v;  // count * W limbs
  BigVec(int count, int width) : W(width), v(static_cast<size_t>(count) * width, 0) {}
  uint64_t* operator[](int i) { return v.data() + static_cast<size_t>(i) * W; }
};

void big_add(uint64_t* r, const uint64_t* a, const uint64_t* b, int W) {
  unsigned __int128 c = 0;
  for (int i = 0; i < W; ++i) {
    c += static_cast<unsigned __int128>(a[i]) + b[i];
    r[i] = static_cast<uint64_t>(c);
    c >>= 64;
  }
}
void big_sub(uint64_t* r, const uint64_t* a, const uint64_t* b, int W) {
  unsigned __int128 c = 1;
  for (int i = 0; i < W; ++i) {
    c += static_cast<unsigned __int128>(a[i]) + static_cast<uint64_t>(~b[i]);
    r[i] = static_cast<uint64_t>(c);
    c >>= 64;
  }
}
double big_to_double(const uint64_t* a, int W) {
  std::vector<uint64_t> m(a, a + W);
  const bool neg = (m[W - 1] >> 63) != 0;
  if (neg) {  // magnitude = ~a + 1
    unsigned __int128 c = 1;
    for (int i = 0; i < W; ++i) {
      c += static_cast<uint64_t>(~m[i]);
      m[i] = static_cast<uint64_t>(c);
      c >>= 64;
    }
  }
  int h = W - 1;
  while (h > 0 && m[h] == 0) --h;
  double v = std::ldexp(static_cast<double>(m[h]), 64 * h);
  if (h > 0) v += std::ldexp(static_cast<double>(m[h - 1]), 64 * (h - 1));
  return neg ? -v : v;
}
}  // namespace

// c_d = f_hat(S) for |S| = d. Grouping Eq. 1's defining sum by the number t of
// -1 entries gives c_d = 2^-k sum_t f(t) [z^t] (1-z)^d (1+z)^(k-d). The
// polynomials are stepped exactly in integers, Q_{d+1} = Q_d (1-z)/(1+z), and
// the single power-of-two division is applied after the integer sum.
void esp_coefficients(const Shape& s, std::vector<double>& c) {
  const int k = s.k;
  std::vector<int8_t> f;
  truth_table(s, f);
  const int W = k / 64 + 2;
  BigVec Q(k + 1, W), R(k + 1, W);
  Q[0][0] = 1;
  for (int step = 0; step < k; ++step)  // (1+z)^k
    for (int t = step + 1; t >= 1; --t) big_add(Q[t], Q[t], Q[t - 1], W);
  std::vector<uint64_t> acc(W), zero(W, 0);
  c.assign(k + 1, 0.0);
  for (int d = 0; d <= k; ++d) {
    std::fill(acc.begin(), acc.end(), 0);
    for (int t = 0; t <= k; ++t) {
      if (f[t] > 0) big_add(acc.data(), acc.data(), Q[t], W);
      else big_sub(acc.data(), acc.data(), Q[t], W);
    }
    c[d] = std::ldexp(big_to_double(acc.data(), W), -k);
    if (d == k) break;
    // R = Q / (1+z) by synthetic division (exact: (1+z) divides Q for d < k)
    std::copy(Q[0], Q[0] + W, R[0]);
    for (int t = 1; t < k; ++t) big_sub(R[t], Q[t], R[t - 1], W);
    // Q = R (1-z)
    std::copy(R[0], R[0] + W, Q[0]);
    for (int t = 1; t < k; ++t) big_sub(Q[t], R[t], R[t - 1], W);
    big_sub(Q[k], zero.data(), R[k - 1], W);
  }
}

void dft_coefficients(const Shape& s, int basis, std::vector<double>& re, std::vector<double>& im) {
  const int k = s.k, N = k + 1, J = N / 2;
  std::vector<double> src(N);
  if (basis == BASIS_PGF) {
    std::vector<int8_t> f;
    truth_table(s, f);
    for (int t = 0; t <= k; ++t) src[t] = f[t];
  } else {
    esp_coefficients(s, src);
  }
  re.assign(J + 1, 0.0);
  im.assign(J + 1, 0.0);
  for (int j = 0; j <= J; ++j) {
    double sr = 0.0, si = 0.0;
    for (int t = 0; t <= k; ++t) {
      double cr, ci;
      unit_root(static_cast<long long>(j) * t, N, cr, ci);
      sr += src[t] * cr;   // w^{-jt} = cos - i sin
      si -= src[t] * ci;
    }
    re[j] = sr / N;
    im[j] = si / N;
  }
  if (N % 2 == 0) im[J] = 0.0;  // the self-conjugate root w = -1 has a real coefficient
  im[0] = 0.0;
}

static void push4(std::vector<float>& o, double a, double b, double c, double d) {
  o.push_back(static_cast<float>(a));
  o.push_back(static_cast<float>(b));
  o.push_back(static_cast<float>(c));
  o.push_back(static_cast<float>(d));
}

// Long probability-generating table (see coef.h): the roots whose
// coefficient is not zero, complex roots by increasing angle theta_j = pi j/N
// and the real root (odd k, theta = pi/2) last; per root the factor
// a_j + b_j l = s_j g_j(l) with, for the form of its 32-root pass,
//   A: g = l tan(theta) + i,  s = b cot(theta),  g' = tan(theta)
//   B: g = l + i cot(theta),  s = b,              g' = 1
// (b_j = sin(theta) e^{i(theta - pi/2)}, so |s_A| = cos, |s_B| = sin and
// arg s = theta - pi/2 for both). E' = E s^k and D' = E s^k g' are stored
// as a shared power of two 2^eb and mantissas. A pass takes form A when
// every factor of its roots is bounded by LONG_FACTOR_BOUND (1/cos(theta)),
// else form B (bound 1/sin(theta); the real root's factor is l itself).
static void build_long_scaled(int k, const std::vector<double>& cr, const std::vector<double>& ci,
                              std::vector<float>& out) {
  const int N = k + 1;
  constexpr double ZERO_ROOT = 1e-13;
  struct Root {
    int j;          // root index (N/2 for the real root)
    double er, ei;  // E_j (complex pair: 2 ft_j; real root: ft_mid)
  };
  std::vector<Root> roots;
  for (int j = 1; j <= k / 2; ++j)
    if (std::hypot(cr[j], ci[j]) > ZERO_ROOT) roots.push_back({j, 2.0 * cr[j], 2.0 * ci[j]});
  const int n_complex = static_cast<int>(roots.size());
  if ((k & 1) && std::fabs(cr[N / 2]) > ZERO_ROOT) roots.push_back({N / 2, cr[N / 2], 0.0});
  const int n = static_cast<int>(roots.size());
  out.clear();
  push4(out, cr[0], n, n_complex, 0);
  for (int p0 = 0; p0 < n; p0 += 32) {
    const int p1 = std::min(n, p0 + 32);
    bool form_a = true;
    for (int r = p0; r < p1; ++r) {
      double c, sn;
      unit_root(roots[r].j, 2LL * N, c, sn);  // angle pi j / N
      if (2 * roots[r].j == N || 1.0 / c >= LONG_FACTOR_BOUND) form_a = false;
    }
    for (int r = p0; r < p1; ++r) {
      const Root& rt = roots[r];
      double c, sn;
      unit_root(rt.j, 2LL * N, c, sn);
      const bool real_root = 2 * rt.j == N;
      if (!form_a && !real_root && 1.0 / sn >= LONG_FACTOR_BOUND)
        throw std::invalid_argument("long table: no scaled factor form fits a root pass");
      double pf, qf, gp, mag_log2;
      if (form_a) {
        pf = sn / c;   // tan
        qf = 1.0;
        gp = pf;
        mag_log2 = k * std::log2(c);
      } else {
        pf = 1.0;
        qf = real_root ? 0.0 : c / sn;  // cot
        gp = 1.0;
        mag_log2 = real_root ? 0.0 : k * std::log2(sn);
      }
      double pc = 1.0, ps = 0.0;  // e^{i k (theta - pi/2)}
      if (!real_root) unit_root(2LL * rt.j * k - static_cast<long long>(k) * N, 4LL * N, pc, ps);
      const double eb = std::floor(mag_log2);
      const double m = std::exp2(mag_log2 - eb);
      const double sr = m * pc, si = m * ps;
      const double er = rt.er * sr - rt.ei * si, ei = rt.er * si + rt.ei * sr;
      push4(out, pf, qf, eb, form_a ? 1.0 : 0.0);
      push4(out, er * gp, ei * gp, er, ei);
    }
  }
}

void build_table(const Shape& s, int basis, int form, std::vector<float>& out) {
  const int k = s.k, N = k + 1;
  std::vector<double> cr, ci;
  dft_coefficients(s, basis, cr, ci);
  out.clear();
  const bool odd = (k & 1) != 0;
  const int mid = N / 2;
  if (form == FORM_SHORT) {
    if (basis == BASIS_PGF) {
      // head: {c0, number of scaled complex roots stored, 0, 0}. A scaled
      // table keeps only the roots whose coefficient is not zero: a truth
      // table with a sparse spectrum (parity: the single root w = -1) costs
      // only its nonzero roots. The exact zeros of such spectra come out of
      // the FP64 DFT as rounding residue (|ft_j| ~ 1e-16); anything at or
      // below ZERO_ROOT (each root contributes at most 2 |ft_j|) is dropped.
      constexpr double ZERO_ROOT = 1e-13;
      const bool scaled = k <= KSCALED_MAX;
      int kept = 0;
      for (int j = 1; j <= k / 2; ++j)
        if (!scaled || std::hypot(cr[j], ci[j]) > ZERO_ROOT) ++kept;
      push4(out, cr[0], scaled ? kept : 0, 0, 0);
      if (odd) push4(out, 0.0, cr[mid], 0, 0);
      for (int j = 1; j <= k / 2; ++j) {
        if (scaled && std::hypot(cr[j], ci[j]) <= ZERO_ROOT) continue;
        // a_j + b_j l = b_j (l + i*gamma_j), gamma_j = cot(pi j/N); E_j = 2 ft_j b_j^k.
        // For k <= KSCALED_MAX the factor is stored scaled, b_j (l + i gamma)
        // = b_j gamma (w + i) with w = l tan(pi j/N), so that a complex
        // multiply by it is two FMAs: {tan, 0, E'_j} with E'_j = 2 ft_j
        // (b_j gamma_j)^k, |b_j gamma_j| = cos(pi j/N). Products of the
        // scaled factors stay below (1 + cot^2)^(k/2) <= 2^100 and each root's
        // contribution keeps its true size (at most 2 |ft_j|).
        double c2, s2;
        unit_root(j, 2LL * N, c2, s2);             // angle pi j / N
        double pc, ps;
        unit_root(2LL * j * k - static_cast<long long>(k) * N, 4LL * N, pc, ps);  // arg b_j^k
        const double mag = std::pow(scaled ? c2 : s2, k);  // |b_j gamma_j|^k or |b_j|^k
        const double br = mag * pc, bi = mag * ps;
        const double er = 2.0 * (cr[j] * br - ci[j] * bi);
        const double ei = 2.0 * (cr[j] * bi + ci[j] * br);
        if (scaled) push4(out, s2 / c2, 0.0, er, ei);
        else push4(out, 0.0, c2 / s2, er, ei);
      }
    } else {
      push4(out, 0.0, 0, 0, 0);
      push4(out, 1.0, cr[0], 0, 0);                // prod (l + 1)
      if (odd) push4(out, -1.0, -cr[mid], 0, 0);   // prod (1 - l) = -prod (l - 1), k odd
      for (int j = 1; j <= k / 2; ++j) {
        // 1 + w^j l = w^j (l + w^-j); E_j = 2 ch_j w^{jk}
        double wc, ws;
        unit_root(j, N, wc, ws);
        double pc, ps;
        unit_root(static_cast<long long>(j) * k, N, pc, ps);
        const double er = 2.0 * (cr[j] * pc - ci[j] * ps);
        const double ei = 2.0 * (cr[j] * ps + ci[j] * pc);
        push4(out, wc, -ws, er, ei);
      }
    }
  } else {
    // every root, real or complex, is two granules {A, b}, {D, E} with the
    // factor written a + b l = A - b (1 - l), A = a + b. In the
    // probability-generating basis A = 1 exactly, so the FP32 rounding of b
    // perturbs a factor by eps*|b| (small at the dominant low roots) instead of
    // eps; with a and b rounded separately that error would add up coherently
    // over the k factors.
    if (basis == BASIS_PGF && k >= LONG_SCALED_MIN_K) {
      build_long_scaled(k, cr, ci, out);
    } else if (basis == BASIS_PGF) {
      push4(out, cr[0], 0, 0, 0);
      if (odd) {
        push4(out, 1.0, 0.0, 1.0, 0.0);
        push4(out, cr[mid], 0.0, cr[mid], 0.0);
      }
      for (int j = 1; j <= k / 2; ++j) {
        double wc, ws;
        unit_root(j, N, wc, ws);
        const double br = 0.5 * (1.0 - wc), bi = -0.5 * ws;
        const double dr = 2.0 * (cr[j] * br - ci[j] * bi), di = 2.0 * (cr[j] * bi + ci[j] * br);
        push4(out, 1.0, 0.0, br, bi);
        push4(out, dr, di, 2.0 * cr[j], 2.0 * ci[j]);
      }
    } else {
      push4(out, 0.0, 0, 0, 0);
      push4(out, 2.0, 0.0, 1.0, 0.0);     // 1 + l
      push4(out, cr[0], 0.0, cr[0], 0.0);
      if (odd) {
        push4(out, 0.0, 0.0, -1.0, 0.0);  // 1 - l
        push4(out, -cr[mid], 0.0, cr[mid], 0.0);
      }
      for (int j = 1; j <= k / 2; ++j) {
        double wc, ws;
        unit_root(j, N, wc, ws);
        const double dr = 2.0 * (cr[j] * wc - ci[j] * ws), di = 2.0 * (cr[j] * ws + ci[j] * wc);
        push4(out, 1.0 + wc, ws, wc, ws);  // 1 + w^j l
        push4(out, dr, di, 2.0 * cr[j], 2.0 * ci[j]);
      }
    }
  }
}

double work_instr(int k, int complex_roots) {
  // per complex root: prefix (4) and suffix (4) complex products and the
  // gradient combine (2) per literal, plus 2 for the value; per real root:
  // 3 per literal plus 1.
  return static_cast<double>(complex_roots) * (10.0 * k + 2.0) + static_cast<double>(k & 1) * (3.0 * k + 1.0);
}

double work_instr(int k, int complex_roots, int real_roots) {
  return static_cast<double>(complex_roots) * (10.0 * k + 2.0) + static_cast<double>(real_roots) * (3.0 * k + 1.0);
}

double work_instr(int k) { return work_instr(k, k / 2); }

}  // namespace afs
