// Load-time coefficient tables for the FE+gradient kernels (host code).
#pragma once
#include <cstdint>
#include <vector>

namespace afs {

enum { BASIS_PGF = 0, BASIS_ESP = 1 };
enum { FORM_SHORT = 0, FORM_LONG = 1 };

// Long probability-generating tables use the scaled factor form from this
// length on (below it the direct form, whose products need no exponent
// tracking, costs less per pass).
constexpr int LONG_SCALED_MIN_K = 129;
// Largest factor modulus a scaled long-table root may reach for |l| <= 1:
// 16 such factors (one checkpoint segment) stay below 2^126.
constexpr double LONG_FACTOR_BOUND = 234.0;

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
//  long form, paper basis and probability-generating basis below
//              LONG_SCALED_MIN_K: {c0,0,0,0}, per root (real roots first,
//              imaginary parts 0) {A.re, A.im, b.re, b.im}, {D.re, D.im, E.re, E.im}
//     with the factor a + b l = A - b (1 - l), A = a + b:
//     FE = c0 + sum Re(E prod_i F_i),  dFE/dl_i = sum Re(D prod_{i'!=i} F_i')
//  long form, probability-generating basis from LONG_SCALED_MIN_K on:
//     {c0, n stored, n complex, 0},
//     per stored root {p, q, eb, form}, {D'.re, D'.im, E'.re, E'.im} with the
//     scaled factor g(l) = p l + i q (form 1: p = tan, q = 1; form 0: p = 1,
//     q = cot, 0 for the real root), the form the same for each run of 32
//     roots:  FE = c0 + sum 2^eb Re(E' prod_i g_i),
//             dFE/dl_i = sum 2^eb Re(D' prod_{i'!=i} g_i')
void build_table(const Shape& s, int basis, int form, std::vector<float>& out);

// Algorithmic FP32 lane instructions of one FE+gradient evaluation of a
// constraint of length k for one restart (see the kernels' cost model).
double work_instr(int k);
// The same with the number of complex roots a table actually keeps.
double work_instr(int k, int complex_roots);
// The same with the complex and real roots a table actually keeps.
double work_instr(int k, int complex_roots, int real_roots);

}  // namespace afs
