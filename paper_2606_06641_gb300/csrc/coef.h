// Load-time coefficient tables for the FE+gradient kernels (host code).
#pragma once
#include <cstdint>
#include <vector>

namespace afs {

enum { BASIS_PGF = 0, BASIS_ESP = 1 };
enum { FORM_SHORT = 0, FORM_LONG = 1 };

// Literals per segment of the long kernel's walks: running products are
// brought back to their true size at segment boundaries (long table below).
constexpr int LONG_SEG = 16;
// A pass of long-table roots uses factor form B when one of its roots has
// cos(theta) below this (s^16 would leave FP32's normal range in form A).
constexpr double LONG_FORM_B_COS = 1.0 / 64.0;
// Chebyshev expansion of the long kernel's derivative terms: a table
// expands the derivative terms of its first roots (a multiple of 32, all in
// form A) in LONG_CHEB_SHORT or LONG_CHEB_LONG Chebyshev terms of l^2, or
// none, whichever costs the kernel least; a root qualifies when the
// truncated tail stays below LONG_CHEB_TOL of the term's smallest value.
constexpr int LONG_CHEB_SHORT = 16;
constexpr int LONG_CHEB_LONG = 32;
constexpr double LONG_CHEB_TOL = 1e-8;

// Constraints with k <= KSHORT use the register (short) kernels and the
// short table layout; longer ones use the shared-memory (long) kernel.
constexpr int KSHORT = 32;
// Short probability-generating tables store every complex root in the
// scaled form gamma (w + i) up to this length (see build_table).
constexpr int KSCALED_MAX = 24;

struct Shape {
  int type, k, op, param, parity;
  bool operator<(const Shape& o) const;
  bool operator==(const Shape& o) const;
};

// Number of real (self-conjugate) and complex-pair roots a table carries.
inline int n_cplx_roots(int k) { return k / 2; }
inline int n_real_roots(int k, int basis) { return (k & 1) + (basis == BASIS_ESP ? 1 : 0); }

// f(t) in {-1,+1} for t = 0..k (Table 1, Appendix A); -1 = satisfied.
void truth_table(const Shape& s, std::vector<int8_t>& f);

// FE coefficients in FP64:
//  PGF basis: ft_j = (1/(k+1)) sum_t f(t) w^{-jt},   FE = sum_j ft_j prod_i (a_j + b_j l_i)
//             with a_j = (1+w^j)/2, b_j = (1-w^j)/2.
//  ESP basis: ch_j = (1/(k+1)) sum_d c_d w^{-jd},     FE = sum_j ch_j prod_i (1 + w^j l_i)
//             with c_d = f_hat(|S| = d).
// Only j = 0..floor((k+1)/2) are returned (the rest are exact conjugates).
void dft_coefficients(const Shape& s, int basis, std::vector<double>& re, std::vector<double>& im);

// c_d = f_hat(|S| = d), d = 0..k, from exact integers with one deferred 2^-k.
void esp_coefficients(const Shape& s, std::vector<double>& c);

// FP32 table in the layout the kernels read (float4 granules):
//  short form: {c0,0,0,0}, per real root {alpha, E, 0, 0},
//              per complex root {alpha, gamma, E.re, E.im}
//     the kernel evaluates  FE   = c0 + sum_r E_r prod_i (l_i + alpha_r)
//                                     + sum_j Re(E_j prod_i (l_i + alpha_j + i gamma_j))
//                          dFE/dl_i = sum_r E_r prod_{i'!=i} (...) + sum_j Re(E_j prod_{i'!=i} (...))
//  long form, paper basis: {0,0,0,0}, per root (real roots first, imaginary
//              parts 0) {A.re, A.im, b.re, b.im}, {D.re, D.im, E.re, E.im}
//     with the factor 1 + w^j l = A - b (1 - l):
//     FE = c0 + sum Re(E prod_i F_i),  dFE/dl_i = sum Re(D prod_{i'!=i} F_i')
//  long form, probability-generating basis (every k > KSHORT):
//     head {c0, n kept complex roots, c_mid, has_real}, {first form-B root, 0, 0, 0};
//     per kept complex root (nonzero coefficient, increasing angle) two
//     granules {p, s16.re, s16.im, 0}, {E'.re, E'.im, 0, 0}.
//     The factor of literal i at the root is s g(l_i), g = p l + i (form A,
//     roots before the first form-B root; p = tan of the root's half angle in
//     FP32) or g = l + i p (form B; p = cot); the coefficients are solved for
//     the nodes that p defines. The first form-B root is a multiple of 32.
//     With n_last = k - 16 floor((k-1)/16): s16 = s^16 rounded to FP32,
//     E' = E s^n_last (s^16 / s16)^(nseg - 1), E = 2 c'_j, so that a walk
//     multiplying the g's and s16 after every full segment of 16 literals
//     ends at the root's true product over E'.
//     The real root (odd k, has_real = 1) has the factor l_i and the
//     coefficient c_mid (value and gradient weight).
//     FE = c0 + sum Re(E s^k prod_i g_i) + c_mid prod_i l_i
void build_table(const Shape& s, int basis, int form, std::vector<float>& out);

// Algorithmic FP32 lane instructions of one FE+gradient evaluation of a
// constraint of length k for one restart (see the kernels' cost model).
double work_instr(int k);
// The same with the number of complex roots a table actually keeps.
double work_instr(int k, int complex_roots);
// The same with the complex and real roots a table actually keeps.
double work_instr(int k, int complex_roots, int real_roots);

}  // namespace afs
