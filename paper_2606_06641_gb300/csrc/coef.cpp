// Load-time DFT coefficient tables (host, FP64, rounded once to FP32).
//
// Sec. 2.1.2: a symmetric constraint's expansion is evaluated from products
// of one factor per literal at the k+1 roots of unity, combined with the
// constraint's DFT coefficients. Sec. 3.5: roots are built so that paired
// roots are exact conjugates, combinatorial terms are exact integers with the
// division deferred, and mirrored terms are copied rather than recomputed.
#include "coef.h"

#include <algorithm>
#include <array>
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

// Long probability-generating table (see coef.h).
//
// Roots. A complex root pair j, -j (theta_j = pi j / N < pi/2) whose exact
// coefficient is not zero is evaluated in one of two factor forms,
//   A: g(l) = p l + i,  p = tan(theta_j) rounded to FP32,
//   B: g(l) = l + i p,  p = cot(theta_j) rounded to FP32,
// and the node the kernel actually uses is z'_j = e^{2 i theta'_j} with
// tan(theta'_j) = p (A) or cot(theta'_j) = p (B) exactly. Rounding tan(theta)
// to FP32 would otherwise perturb every one of the k factors of a product the
// same way (a relative error up to k eps in each product). Instead the
// coefficients are solved in FP64 for the nodes the kernel uses:
// sum_j c'_j z'_j^t = f(t) for t = 0..k, by iterative refinement started
// from the DFT of f at the exact roots (the nodes differ from the roots of
// unity by an angle of about 1e-7, so a few correction steps reach FP64
// accuracy). The identity
//   sum_j c'_j prod_i (q_i + p_i z'_j) = sum_t P(T = t) sum_j c'_j z'_j^t
// then gives the expansion exactly for any nodes, so only per-operation
// rounding remains. Node 0 (z = 1), the real root z = -1 (odd k) and the
// roots not evaluated (zero exact coefficient) stay exact.
//
// Factor. At node z' the literal factor is a' + b' l with a' = (1 + z')/2,
// b' = (1 - z')/2 and a'/b' = i cot(theta'), so a' + b' l = s g(l) with
// s = b'/p (form A, |s| = cos theta') or s = b' (form B, |s| = sin theta').
// The kernel walks the literals in segments of LONG_SEG = 16 (the last
// segment n_last long) and keeps the running product at its true size at
// segment boundaries: P <- P prod_seg g, then P <- P s^16 after every full
// segment; within a segment |g| <= 1/|s| and |s|^16 >= 2^-100 keep P within
// FP32. The root's value is Re(E' P) and each literal's derivative is
// Re(E' P dg/dl / g(l_i)), the factor divided out of the full product
// (|g| >= 1 in form A, >= p in form B, so never zero).
// Roots take form A (one FP32 instruction fewer per complex multiply) up to
// the first block of 32 kept roots that holds a root with cos(theta) below
// LONG_FORM_B_COS (there s^16 would leave FP32's normal range), form B from
// that block on; kernel passes of 8, 16 or 32 roots never straddle it.
//
// FP32 rounding of s^16. It is stored rounded once but applied once per
// segment, so its rounding would add up over the segments. It is the same
// factor for every point, so it is compensated in E': with the rounded s^16
// applied nseg - 1 times, E' P is exact.
// Per kept root (by increasing angle) two granules {p, s^16, 0}, {E', 0, 0}
// with E = 2 c'_j. Head: {c'_0, kept complex roots, c'_mid (the real root's
// coefficient, odd k), 1 if the real root is present}, {first form-B root (a
// multiple of 32; = kept roots if none), number of expanded roots (a
// multiple of 32, all in form A), expansion terms (0, 16 or 32), 0}. After
// the roots' granules, per expanded root its expansion terms. The real
// root's factor is l itself.
//
// Expanded derivative terms. A root's derivative term (A l + B) / (alpha u
// + beta), u = l^2, has its pole at u = -beta/alpha; for the first form-A
// roots (p <= about 3) that pole is far enough from [0, 1] for 1 / (alpha u
// + beta) = sum_n c_n T_n(2u - 1) to converge to FP32 accuracy in 16 or 32
// terms, so the sum over those roots becomes sum_n T_n(2u - 1) (l X_n +
// Y_n) with X_n = sum_r A_r c_{n,r}, Y_n = sum_r B_r c_{n,r}: per literal
// one Chebyshev sum instead of a term per root.
namespace {
struct Cx {
  double r, i;
};
Cx cmul(Cx a, Cx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
Cx cdiv(Cx a, Cx b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
Cx cpow(Cx z, int e) {
  Cx r{1.0, 0.0};
  while (e > 0) {
    if (e & 1) r = cmul(r, z);
    z = cmul(z, z);
    e >>= 1;
  }
  return r;
}
Cx f32(Cx z) { return {static_cast<double>(static_cast<float>(z.r)), static_cast<double>(static_cast<float>(z.i))}; }

// Chebyshev expansion on u in [0, 1] of 1 / (alpha u + beta) (alpha, beta >
// 0): with t = 2u - 1 it is (2/alpha) / (t + s), s = 1 + 2 beta / alpha > 1,
// whose expansion is (2/q) (1/2 + sum_{n >= 1} (-r)^n T_n(t)), q =
// sqrt(s^2 - 1), r = s - q = 1 / (s + q). Written without cancellation:
// alpha q / 2 = sqrt(beta (alpha + beta)), r = alpha / (alpha + 2 beta + 2
// sqrt(beta (alpha + beta))). So c_0 = 1 / m, c_n = 2 (-r)^n / m, m =
// sqrt(beta (alpha + beta)).
void expansion_terms(double alpha, double beta, int nc, double* c) {
  const double m = std::sqrt(beta * (alpha + beta));
  const double r = alpha / (alpha + 2.0 * beta + 2.0 * m);
  double rn = 1.0;
  for (int n = 0; n < nc; ++n) {
    c[n] = (n == 0 ? 1.0 : 2.0 * rn) / m;
    rn *= -r;
  }
}
// The tail after nc terms, sum_{n >= nc} |c_n| = 2 r^nc / ((1 - r) m),
// relative to the function's smallest value on [0, 1], 1 / (alpha + beta).
double cheb_tail(double alpha, double beta, int nc) {
  const double m = std::sqrt(beta * (alpha + beta));
  const double r = alpha / (alpha + 2.0 * beta + 2.0 * m);
  return 2.0 * std::pow(r, nc) / ((1.0 - r) * m) * (alpha + beta);
}
}  // namespace

static void build_long_pgf(const Shape& s, std::vector<float>& out) {
  const int k = s.k, N = k + 1, J = k / 2;  // complex pairs j = 1..J
  const bool odd = (k & 1) != 0;
  std::vector<int8_t> f;
  truth_table(s, f);
  // exact roots of unity w^m, m = 0..N-1 (for the DFT steps)
  std::vector<double> wr(N), wi(N);
  for (int m = 0; m < N; ++m) unit_root(m, N, wr[m], wi[m]);
  std::vector<double> cr(J + 1, 0.0), ci(J + 1, 0.0);
  double cmid = 0.0;
  auto dft_add = [&](const std::vector<double>& src) {  // c_j += (1/N) sum_t src[t] w^{-jt}
    for (int j = 0; j <= J; ++j) {
      double sr = 0.0, si = 0.0;
      for (int t = 0; t <= k; ++t) {
        const int m = static_cast<int>((static_cast<long long>(j) * t) % N);
        sr += src[t] * wr[m];
        si -= src[t] * wi[m];
      }
      cr[j] += sr / N;
      ci[j] += j == 0 ? 0.0 : si / N;
    }
    if (odd) {
      double sm = 0.0;
      for (int t = 0; t <= k; ++t) sm += (t & 1) ? -src[t] : src[t];
      cmid += sm / N;
    }
  };
  std::vector<double> res(N);
  for (int t = 0; t <= k; ++t) res[t] = f[t];
  dft_add(res);  // exact-root coefficients
  constexpr double ZERO_ROOT = 1e-13;
  const bool has_real = odd && std::fabs(cmid) > ZERO_ROOT;
  // kept roots, their forms and nodes
  std::vector<int> kept;
  int first_b = -1;
  std::vector<double> cosj(J + 1, 1.0), sinj(J + 1, 0.0);
  for (int j = 1; j <= J; ++j) {
    unit_root(j, 2LL * N, cosj[j], sinj[j]);  // angle pi j / N
    if (std::hypot(cr[j], ci[j]) <= ZERO_ROOT) continue;
    if (first_b < 0 && cosj[j] < LONG_FORM_B_COS) first_b = static_cast<int>(kept.size());
    kept.push_back(j);
  }
  const int nk = static_cast<int>(kept.size());
  const int form_b_from = first_b < 0 ? nk : first_b / 32 * 32;
  std::vector<Cx> z(J + 1);
  std::vector<double> pv(J + 1, 0.0);
  std::vector<int> formb(J + 1, 0);
  for (int j = 1; j <= J; ++j) {
    double c, sn;
    unit_root(2LL * j, 2LL * N, c, sn);  // exact node w^j
    z[j] = Cx{c, sn};
  }
  for (int r = 0; r < nk; ++r) {
    const int j = kept[r];
    const bool fb = r >= form_b_from;
    const double p = static_cast<float>(fb ? cosj[j] / sinj[j] : sinj[j] / cosj[j]);
    const double t = fb ? 1.0 / p : p, d = 1.0 + t * t;  // tan(theta') = t
    pv[j] = p;
    formb[j] = fb ? 1 : 0;
    z[j] = Cx{(1.0 - t * t) / d, 2.0 * t / d};
  }
  // refine c'_j (j = 0..J) and c'_mid against the nodes
  for (int it = 0; it < 3; ++it) {
    // residual f(t) - [c0 + 2 Re sum_j c_j z_j^t + cmid (-1)^t]
    for (int t = 0; t <= k; ++t) res[t] = f[t] - cr[0] - (odd ? ((t & 1) ? -cmid : cmid) : 0.0);
    for (int j = 1; j <= J; ++j) {
      Cx pw{1.0, 0.0};  // z_j^t by repeated multiplication
      for (int t = 0; t <= k; ++t) {
        res[t] -= 2.0 * (cr[j] * pw.r - ci[j] * pw.i);
        pw = cmul(pw, z[j]);
      }
    }
    dft_add(res);
  }
  const int nseg = (k + LONG_SEG - 1) / LONG_SEG;
  const int n_last = k - LONG_SEG * (nseg - 1);
  // Chebyshev expansion of the leading form-A roots' derivative terms
  // 1 / (p^2 u + 1), u = l^2 (expansion_terms below): the roots whose tail
  // after nc terms is within LONG_CHEB_TOL (a prefix: the pole -1/p^2 moves
  // toward u = 0 as p grows along the table), rounded down to a multiple of
  // 32; nc chosen for the least kernel work, in FP32 operations per literal
  // and restart: 3 per exact root, 2 nc / k per expanded root (the per-root
  // sums), 3.5 nc for the per-literal Chebyshev sum.
  auto n_expandable = [&](int nc) {
    int n = 0;
    while (n < form_b_from) {
      const double p = pv[kept[n]];
      if (cheb_tail(p * p, 1.0, nc) > LONG_CHEB_TOL) break;
      ++n;
    }
    return n / 32 * 32;
  };
  int ncheb = 0, first_x = 0;
  double best = 3.0 * nk;
  for (const int nc : {LONG_CHEB_SHORT, LONG_CHEB_LONG}) {
    const int fx = n_expandable(nc);
    const double cost = 3.0 * (nk - fx) + 2.0 * nc * fx / k + 3.5 * nc;
    if (fx > 0 && cost < best) {
      best = cost;
      ncheb = nc;
      first_x = fx;
    }
  }
  out.clear();
  push4(out, cr[0], nk, has_real ? cmid : 0.0, has_real ? 1.0 : 0.0);
  push4(out, form_b_from, first_x, ncheb, 0);
  for (int r = 0; r < nk; ++r) {
    const int j = kept[r];
    const double p = pv[j];
    const Cx b{0.5 * (1.0 - z[j].r), -0.5 * z[j].i};  // b' = (1 - z')/2
    const Cx E{2.0 * cr[j], 2.0 * ci[j]};
    const Cx sc = formb[j] ? b : Cx{b.r / p, b.i / p};
    if (1.0 / std::hypot(sc.r, sc.i) >= 32768.0) throw std::invalid_argument("long table: root factor bound exceeded");
    const Cx s16 = f32(cpow(sc, 16));
    const Cx r16 = cdiv(cpow(sc, 16), s16);  // exact / rounded s^16
    // E' = E s^n_last (s^16 / fl(s^16))^(nseg-1): with the rounded s^16 at
    // the segment boundaries, E' prod_i g_i is the root's exact product
    const Cx Ep = cmul(cmul(E, cpow(sc, n_last)), cpow(r16, nseg - 1));
    push4(out, p, s16.r, s16.i, 0.0);
    push4(out, Ep.r, Ep.i, 0.0, 0.0);
  }
  // per expanded root its ncheb coefficients c_0 .. c_{ncheb-1}
  for (int r = 0; r < first_x; ++r) {
    const double p = pv[kept[r]];
    double c[LONG_CHEB_LONG];
    expansion_terms(p * p, 1.0, ncheb, c);
    for (int n = 0; n < ncheb; n += 4) push4(out, c[n], c[n + 1], c[n + 2], c[n + 3]);
  }
}

void build_table(const Shape& s, int basis, int form, std::vector<float>& out) {
  if (form == FORM_LONG && basis == BASIS_PGF) {
    build_long_pgf(s, out);
    return;
  }
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
    // paper basis: every root, real or complex, is two granules {A, b},
    // {D, E} with the factor 1 + w^j l written A - b (1 - l), A = 1 + w^j
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
