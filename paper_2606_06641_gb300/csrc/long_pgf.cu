// FE + analytic gradient of long constraints (k > 32) in the
// probability-generating basis.
//
// Sec. 2.1.2: a symmetric constraint's expansion is a combination, with the
// constraint's DFT coefficients, of products over its literals at the roots
// of unity; the gradient of literal i at a root is the product of the other
// literals' factors. Sec. 3.5: conjugate roots are paired, so only the roots
// of one half-plane are evaluated (each complex one counted twice through
// the real part) plus, for odd k, the real root w = -1.
//
// Layout. One CTA per (constraint, RT restarts): NW warps, each warp holds
// 32 / W restarts ("slots") and each slot's W lanes own W roots of a pass;
// passes walk the table's roots W at a time. The literal list is staged with
// cp.async.bulk on an mbarrier (bounded wait), the literal values l = s x of
// the CTA's restarts in shared memory rows, read four at a time by 16-byte
// loads; each warp has a shared row of 64 16-byte entries (two a lane) for
// the values its lanes exchange within a pass: staged octets, root constants
// or four-root fractions, expansion sums.
//
// Factor form (coefficient table built on the host): at every complex root
// the literal factor is s g(l), g = p l + i (form A) or l + i p (form B). In
// slots of 16 and 32 lanes the forward walk multiplies a running product by
// the factors of eight literals at once: their product is a polynomial in p
// whose coefficients are the eight values' elementary symmetric polynomials,
// formed once per pass and shared by all roots of the slot, so an octet
// costs twelve FP32 operations (paired FMAs where the form allows), 1.5 a
// literal. Slots of 8 lanes, where an octet formed per lane would serve only
// 8 roots, take one factor at a time (three FP32 instructions in form A).
// The walk goes in segments of LONG_SEG literals and multiplies by the
// table's s^16 after each full one, so the running product is at its true
// size (|prod| <= 1) at every segment boundary and stays within FP32 inside
// a segment; no exponent bookkeeping is needed.
//
// Gradient by division. With T = E' prod g the root's exact product, the
// derivative in literal i is Re(T g'(l_i) / g(l_i)): the factor divided out
// of the full product. |g| >= 1 in form A and >= p in form B (p at least
// tan(pi / (2 (k + 1))) there), so the division never meets a zero and keeps
// the product's relative error. Each root's term is a rational function of
// l with a quadratic denominator in l^2, so four adjacent roots' terms sum
// to one fraction (numerator of degree 7 in l, denominator of degree 4 in
// l^2, coefficients formed once per pass): per (literal, four roots) twelve
// FMAs and one approximate reciprocal, three FMAs a root, where a pass walks
// more than 4 W literals; shorter passes take one term a root (three FMAs
// and a reciprocal). Either way no prefix and suffix products are rebuilt.
// The lanes then swap roles: each lane takes literals of its slot (pairs of
// adjacent ones on paired FMAs for the fractions) and walks the slot's roots
// or root groups (their constants broadcast from shared memory), summing in
// registers and adding each literal's sum to the slot's gradient row once
// per pass (fixed order, deterministic).
//
// Expanded roots. For a table's leading form-A roots the derivative term's
// factor 1 / (p^2 l^2 + 1) is stored as a Chebyshev series in 2 l^2 - 1 (16
// or 32 terms, tail below 1e-8): their passes skip the per-literal terms and
// add each root's A and B times its terms to per-restart sums X_n, Y_n, and
// one Clenshaw sum per literal, sum_n T_n (l X_n + Y_n), covers all of them.
//
// The real root's factor is l itself, which can be zero: its leave-one-out
// products take a prefix/suffix scan over the slot's lanes after the passes,
// in registers.
#include <cuda_bf16.h>

#include "afsat.h"
#include "afsat_internal.h"
#include "bulk_copy.cuh"
#include "coef.h"
#include "fe_short.cuh"

namespace afs {

namespace {


// 16-byte entries of a warp's shared row: two per lane (a root group's
// coefficients in duplicated pairs take eight entries)
constexpr int LONG_ROW = 64;

// Shared memory of one CTA.
struct LongPgfLayout {
  int kpad, nseg, rt, ep, gp;
  size_t off_ell, off_gs, off_rc, bytes;
  __host__ __device__ LongPgfLayout(int kmax, int W, int NW) {
    kpad = (kmax + LONG_SEG - 1) / LONG_SEG * LONG_SEG;
    nseg = kpad / LONG_SEG;
    rt = NW * (32 / W);
    const int k32 = (kpad + 31) & ~31;
    ep = k32 + 8;                   // literal-value rows: the slots' 16-byte reads fall in distinct banks
    gp = k32 + (W < 32 ? W : 0);    // gradient rows: the slots' column updates fall in distinct banks
    off_ell = static_cast<size_t>(kpad) * 8;                         // literal list (int2)
    off_gs = off_ell + static_cast<size_t>(rt) * ep * 4;            // literal values
    off_rc = off_gs + static_cast<size_t>(rt) * gp * 4;             // gradient accumulators
    bytes = off_rc + static_cast<size_t>(NW) * LONG_ROW * 16;        // each warp's shared row
  }
};

// Approximate reciprocal (PTX rcp.approx, within one unit in the last place)
// of a normal positive number.
__device__ __forceinline__ float rcp_apx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// x y + z in both halves: one paired FP32 instruction
__device__ __forceinline__ float2 ffma2(float2 x, float2 y, float2 z) { return __ffma2_rn(x, y, z); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }

// P <- P (w + i)
__device__ __forceinline__ void gmul(float w, float& r, float& i) {
  const float nr = fmaf(r, w, -i);
  const float ni = fmaf(i, w, r);
  r = nr;
  i = ni;
}
// P <- P (l + i q)
__device__ __forceinline__ void bmul(float l, float q, float& r, float& i) {
  const float nr = fmaf(r, l, -i * q);
  const float ni = fmaf(i, l, r * q);
  r = nr;
  i = ni;
}
// P <- P g(l): form A g = p l + i (three FP32 instructions), form B g = l + i p (four)
template <bool FB>
__device__ __forceinline__ void fmul(float l, float p, float& r, float& i) {
  if constexpr (FB) bmul(l, p, r, i);
  else gmul(l * p, r, i);
}
// P <- P (br + i bi)
__device__ __forceinline__ void cmul(float& r, float& i, float br, float bi) {
  const float nr = fmaf(r, br, -i * bi);
  const float ni = fmaf(r, bi, i * br);
  r = nr;
  i = ni;
}

// NP pairs of adjacent literals a lane (literals c0 + 2 (q W + rl), + 1)
// against the slot's W / 4 root groups: per (pair, group) twelve paired
// FMAs and two reciprocals, each pair's sums added to the gradient row.
template <int W, int NP>
__device__ __forceinline__ void grad_group_pairs(const float4* rs, const float* el, float* gr, int c0, int rl,
                                                 int k) {
  float2 lv[NP], u[NP], v[NP], g[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int i = c0 + 2 * (q * W + rl);
    lv[q] = i < k ? *reinterpret_cast<const float2*>(el + i) : make_float2(0.0f, 0.0f);
    u[q] = __fmul2_rn(lv[q], lv[q]);
    v[q] = __fmul2_rn(u[q], u[q]);
    g[q] = make_float2(0.0f, 0.0f);
  }
#pragma unroll 2
  for (int jq = 0; jq < W / 4; ++jq) {
    const float4* cg = rs + 8 * jq;
    const float4 a0 = cg[0], a1 = cg[1], b0 = cg[2], b1 = cg[3], d0 = cg[4], d1 = cg[5];
    const float2 z0 = lo2(cg[6]);
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float2 hi = ffma2(ffma2(lo2(a0), lv[q], hi2(a0)), u[q], ffma2(lo2(a1), lv[q], hi2(a1)));
      const float2 lo = ffma2(ffma2(lo2(b0), lv[q], hi2(b0)), u[q], ffma2(lo2(b1), lv[q], hi2(b1)));
      const float2 den = ffma2(ffma2(ffma2(lo2(d0), u[q], hi2(d0)), v[q], ffma2(lo2(d1), u[q], hi2(d1))), u[q], z0);
      g[q] = ffma2(ffma2(hi, v[q], lo), make_float2(rcp_apx(den.x), rcp_apx(den.y)), g[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int i = c0 + 2 * (q * W + rl);
    if (i + 1 < k) {
      float2* gp2 = reinterpret_cast<float2*>(gr + i);  // rows and i are even: 8-byte aligned
      const float2 o = *gp2;
      *gp2 = make_float2(o.x + g[q].x, o.y + g[q].y);
    } else if (i < k) {
      gr[i] += g[q].x;
    }
  }
}

// NQ literals a lane (c0 + q W + rl) against the slot's W roots, one term a
// root: three FMAs and a reciprocal per (literal, root).
template <int W, int NQ>
__device__ __forceinline__ void grad_root_terms(const float4* rs, const float* el, float* gr, int c0, int rl,
                                                int k) {
  float lv[NQ], l2[NQ], g[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = c0 + q * W + rl;
    lv[q] = i < k ? el[i] : 0.0f;
    l2[q] = lv[q] * lv[q];
    g[q] = 0.0f;
  }
#pragma unroll 4
  for (int jj = 0; jj < W; ++jj) {
    const float4 c = rs[jj];
#pragma unroll
    for (int q = 0; q < NQ; ++q) g[q] = fmaf(fmaf(c.x, lv[q], c.y), rcp_apx(fmaf(c.z, l2[q], c.w)), g[q]);
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = c0 + q * W + rl;
    if (i < k) gr[i] += g[q];
  }
}

// Gradient of one pass with four adjacent roots' terms summed to one
// fraction N(l) / D(u), u = l^2: N of degree 7 in l, D of degree 4 in u with
// positive coefficients (the product of the four denominators). Pairs first
// (lane ^ 1), then pairs of pairs (lane ^ 2); each lane forms the sums with
// its own root or pair as the first operand (deterministic; the lanes of a
// group may differ in the last bit). The coefficients are published in
// duplicated pairs and each lane evaluates two adjacent literals at once:
// per (literal pair, group) twelve paired FMAs and two reciprocals. Pays off
// once a pass walks more than one chunk of 4 W literals: the coefficients
// cost about seventy instructions a lane.
template <int W>
__device__ __forceinline__ void long_grad_groups(float ta, float tb, float da, float db, int rl, int lane,
                                                 const float* el, float* gr, float4* rc, int k) {
  // pair: N = n0 + n1 l + n2 l^2 + n3 l^3, D = e0 + e1 u + e2 u^2
  const float oa = __shfl_xor_sync(0xffffffffu, ta, 1), ob = __shfl_xor_sync(0xffffffffu, tb, 1);
  const float oda = __shfl_xor_sync(0xffffffffu, da, 1), odb = __shfl_xor_sync(0xffffffffu, db, 1);
  const float n0 = fmaf(tb, odb, ob * db), n1 = fmaf(ta, odb, oa * db);
  const float n2 = fmaf(tb, oda, ob * da), n3 = fmaf(ta, oda, oa * da);
  const float e0 = db * odb, e1 = fmaf(da, odb, oda * db), e2 = da * oda;
  // (N, D) this lane's pair, (M, F) the other one: N F + M D over D F
  const float M0 = __shfl_xor_sync(0xffffffffu, n0, 2), M1 = __shfl_xor_sync(0xffffffffu, n1, 2);
  const float M2 = __shfl_xor_sync(0xffffffffu, n2, 2), M3 = __shfl_xor_sync(0xffffffffu, n3, 2);
  const float F0 = __shfl_xor_sync(0xffffffffu, e0, 2), F1 = __shfl_xor_sync(0xffffffffu, e1, 2);
  const float F2 = __shfl_xor_sync(0xffffffffu, e2, 2);
  // each lane of the group publishes one quarter, duplicated into pairs for
  // the paired evaluation: (Q7 Q6 Q5 Q4), (Q3 Q2 Q1 Q0), (E4 E3 E2 E1), (E0)
  float4 piece;
  switch (rl & 3) {
    case 0:
      piece = make_float4(fmaf(n3, F2, M3 * e2), fmaf(n2, F2, M2 * e2),
                          fmaf(n3, F1, fmaf(n1, F2, fmaf(M3, e1, M1 * e2))),
                          fmaf(n2, F1, fmaf(n0, F2, fmaf(M2, e1, M0 * e2))));
      break;
    case 1:
      piece = make_float4(fmaf(n3, F0, fmaf(n1, F1, fmaf(M3, e0, M1 * e1))),
                          fmaf(n2, F0, fmaf(n0, F1, fmaf(M2, e0, M0 * e1))), fmaf(n1, F0, M1 * e0),
                          fmaf(n0, F0, M0 * e0));
      break;
    case 2:
      piece = make_float4(e2 * F2, fmaf(e1, F2, e2 * F1), fmaf(e0, F2, fmaf(e1, F1, e2 * F0)), fmaf(e0, F1, e1 * F0));
      break;
    default:
      piece = make_float4(e0 * F0, 0.0f, 0.0f, 0.0f);
      break;
  }
  rc[2 * lane] = make_float4(piece.x, piece.x, piece.y, piece.y);
  rc[2 * lane + 1] = make_float4(piece.z, piece.z, piece.w, piece.w);
  __syncwarp();
  // each lane takes pairs of adjacent literals, two pairs per chunk of 4 W
  // (one in a last chunk that ends within its first 2 W); a group's
  // coefficients occupy eight entries
  const float4* rs = rc + 2 * (lane & ~(W - 1));
  int c0 = 0;
  for (; c0 + 2 * W < k; c0 += 4 * W) grad_group_pairs<W, 2>(rs, el, gr, c0, rl, k);
  if (c0 < k) grad_group_pairs<W, 1>(rs, el, gr, c0, rl, k);
}


// An octet of literal values (two quads v, w) staged for the forward walk:
// its elementary symmetric polynomials e1 .. e8 (from the quads' by
// convolution), in the order the form's multiply takes them. Form A prod
// (p l + i) = (1 - p^2 e2 + p^4 e4 - p^6 e6 + p^8 e8) + i p (-e1 + p^2 e3 -
// p^4 e5 + p^6 e7): Horner in p^2 on the pairs, staged (e8, e7, -e6, -e5),
// (e4, e3, -e2, -e1). Form B prod (l + i p) = (e8 + q e6 + q^2 e4 + q^3 e2
// + q^4) + i p (e7 + q e5 + q^2 e3 + q^3 e1) with q = -p^2: staged (e4, e5,
// e6, e7), (e1, e2, e3, e8).
template <bool FB>
__device__ __forceinline__ void oct_stage(float4 v, float4 w, float4& s0, float4& s1) {
  const float pa = v.x + v.y, pb = v.x * v.y, pc = v.z + v.w, pd = v.z * v.w;
  const float a1 = pa + pc, a2 = fmaf(pa, pc, pb + pd), a3 = fmaf(pb, pc, pd * pa), a4 = pb * pd;
  const float qa = w.x + w.y, qb = w.x * w.y, qc = w.z + w.w, qd = w.z * w.w;
  const float b1 = qa + qc, b2 = fmaf(qa, qc, qb + qd), b3 = fmaf(qb, qc, qd * qa), b4 = qb * qd;
  const float e1 = a1 + b1;
  const float e2 = fmaf(a1, b1, a2 + b2);
  const float e3 = fmaf(a2, b1, fmaf(a1, b2, a3 + b3));
  const float e4 = fmaf(a3, b1, fmaf(a2, b2, fmaf(a1, b3, a4 + b4)));
  const float e5 = fmaf(a4, b1, fmaf(a3, b2, fmaf(a2, b3, a1 * b4)));
  const float e6 = fmaf(a4, b2, fmaf(a3, b3, a2 * b4));
  const float e7 = fmaf(a4, b3, a3 * b4);
  const float e8 = a4 * b4;
  if (FB) {
    s0 = make_float4(e4, e5, e6, e7);
    s1 = make_float4(e1, e2, e3, e8);
  } else {
    s0 = make_float4(e8, e7, -e6, -e5);
    s1 = make_float4(e4, e3, -e2, -e1);
  }
}
// P <- P prod over an octet of g(l): form A four paired FMAs, form B two
// paired FMAs and four FP32 instructions, then a complex multiply (twelve
// FP32 operations for eight literals). The terms' magnitudes sum to at most
// 16 times the product's (each factor's |real| + |imag| is at most sqrt(2)
// times its modulus).
template <bool FB>
__device__ __forceinline__ void omul(float4 s0, float4 s1, float p, float p2, float& r, float& i) {
  float fr, fi;
  if constexpr (FB) {
    const float q = -p2;
    const float2 qq = make_float2(q, q);
    float2 t = make_float2(q + s1.y, fmaf(q, s1.x, s1.z));
    t = ffma2(qq, t, lo2(s0));
    t = ffma2(qq, t, hi2(s0));
    fr = fmaf(q, t.x, s1.w);
    fi = p * t.y;
  } else {
    const float2 pp = make_float2(p2, p2);
    float2 t = ffma2(pp, lo2(s0), hi2(s0));
    t = ffma2(pp, t, lo2(s1));
    t = ffma2(pp, t, hi2(s1));
    const float2 f = ffma2(make_float2(p2, p), t, make_float2(1.0f, 0.0f));
    fr = f.x;
    fi = f.y;
  }
  cmul(r, i, fr, fi);
}
static_assert(LONG_SEG % 8 == 0, "segments hold whole octets");

// One pass: the slot's W lanes take roots j0 .. j0 + W - 1. A forward walk
// gives the full product P (true size at every segment boundary, restored by
// s^16) and T = E' P, whose real part is the root's value; the derivative in
// literal t is then Re(U / g_t), U = T dg/dl (p for form A, 1 for form B):
// (U_r w + U_i) / (w^2 + 1) with w = p l in form A, (U_r l + T_i p) /
// (l^2 + p^2) in form B. For the gradient the lanes swap roles: each lane
// publishes its root's derivative constants (or, for long passes, each group
// of four lanes its roots' summed fraction) to the warp's shared row, then
// the slot's lanes take 4 W literals at a time (4 per lane, in registers)
// and walk the slot's roots or groups (broadcast reads), summing in
// registers and adding to the gradient row once per pass (fixed order).
// Lanes past the table's roots get a zero weight and bounded factors.
// An expansion pass (XP) adds its roots' A and B times their Chebyshev
// terms to the slot's sums X_n, Y_n (lane rl holds n = rl and rl + W)
// instead of a derivative term per literal.
template <int W, bool FB, bool XP>
__device__ __forceinline__ float pgf_pass(const float4* tab, int nroots, int j0, int rl, int lane, const float* el,
                                          float* gr, float4* rc, int k, int nseg, int n_last, const float* cheb,
                                          int ncheb, float (&X)[2], float (&Y)[2]) {
  const int j = j0 + rl;
  float p = FB ? 1.0f : 0.0f, s16r = FB ? 0.00390625f : 1.0f, s16i = 0.f, er = 0.f, ei = 0.f;
  if (j < nroots) {
    const float4* rg = tab + 2 + 2 * j;
    const float4 g0 = __ldg(rg), g1 = __ldg(rg + 1);
    p = g0.x;
    s16r = g0.y;
    s16i = g0.z;
    er = g1.x;
    ei = g1.y;
  }
  const float p2 = p * p;
  float Pr = 1.0f, Pi = 0.0f;
  if constexpr (W >= 16) {
    // chunks of W octets (8 W literals): each lane stages the symmetric
    // polynomials of one octet of its slot in two entries of the warp's
    // shared row (halves 0..31 and 32..63), then the slot's lanes walk the
    // chunk's full segments, s^16 after each. A chunk of wc octets covers its
    // 2 wc quads; octet c0 + rl takes quads rl and wc + rl of them (an
    // octet's literals need not be adjacent: any 16 literals of a segment
    // keep the running product within its bound), so the loads and stores
    // are consecutive 16-byte words.
    const int no = k >> 3;
    const float4* e4 = reinterpret_cast<const float4*>(el);
    const float4* rs = rc + (lane & ~(W - 1));
    for (int c0 = 0; c0 < no; c0 += W) {
      const int wc = min(W, no - c0);
      float4 s0 = make_float4(0.0f, 0.0f, 0.0f, 0.0f), s1 = s0;
      if (rl < wc) oct_stage<FB>(e4[2 * c0 + rl], e4[2 * c0 + wc + rl], s0, s1);
      rc[lane] = s0;
      rc[32 + lane] = s1;
      __syncwarp();
      const int s1g = min((c0 + W) / (LONG_SEG / 8), nseg - 1);
      for (int sg = c0 / (LONG_SEG / 8); sg < s1g; ++sg) {
        const float4* os = rs + (sg * (LONG_SEG / 8) - c0);
#pragma unroll
        for (int u = 0; u < LONG_SEG / 8; ++u) omul<FB>(os[u], os[32 + u], p, p2, Pr, Pi);
        cmul(Pr, Pi, s16r, s16i);
      }
      if (c0 + W < no) __syncwarp();  // the chunk is read before the next one is staged
    }
    // the last segment: its full octets (staged in the last chunk), then the literals past them
    if (no > 0) {
      const int cl = (no - 1) / W * W;
      for (int oo = (nseg - 1) * (LONG_SEG / 8); oo < no; ++oo) omul<FB>(rs[oo - cl], rs[32 + oo - cl], p, p2, Pr, Pi);
    }
    for (int t = 8 * no; t < k; ++t) fmul<FB>(el[t], p, Pr, Pi);
    __syncwarp();  // the octets are read before the root constants replace them
  } else {
    // narrow slots (an octet staged per lane would serve only W roots): one
    // factor at a time, literal values read four at a time
    for (int sg = 0; sg + 1 < nseg; ++sg) {
      const float4* e4 = reinterpret_cast<const float4*>(el + sg * LONG_SEG);
#pragma unroll
      for (int u = 0; u < LONG_SEG / 4; ++u) {
        const float4 v = e4[u];
        fmul<FB>(v.x, p, Pr, Pi);
        fmul<FB>(v.y, p, Pr, Pi);
        fmul<FB>(v.z, p, Pr, Pi);
        fmul<FB>(v.w, p, Pr, Pi);
      }
      cmul(Pr, Pi, s16r, s16i);
    }
    const float* e = el + (nseg - 1) * LONG_SEG;
    for (int t = 0; t < n_last; ++t) fmul<FB>(e[t], p, Pr, Pi);
  }
  const float Tr = fmaf(er, Pr, -ei * Pi), Ti = fmaf(er, Pi, ei * Pr);
  float v = Tr;
#pragma unroll
  for (int o = W / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  // the root's derivative term (A l + B') / (alpha u + beta), u = l^2: form A
  // (U = T p, w = p l) A = T_r p^2, B' = T_i p, alpha = p^2, beta = 1; form B
  // (U = T) A = T_r, B' = T_i p, alpha = 1, beta = p^2
  const float ta = FB ? Tr : Tr * p2, tb = Ti * p, da = FB ? 1.0f : p2, db = FB ? p2 : 1.0f;
  if constexpr (XP) {
    float2* r2 = reinterpret_cast<float2*>(rc);
    r2[lane] = make_float2(ta, tb);
    __syncwarp();
    const float2* s2 = r2 + (lane & ~(W - 1));
    const float* cj = cheb + static_cast<size_t>(j0) * ncheb;  // root-major, ncheb terms a root
#pragma unroll
    for (int m = 0; m < 2; ++m) {
      const int n = rl + m * W;
      if (n < ncheb) {
        float x = X[m], y = Y[m];
#pragma unroll 8
        for (int r = 0; r < W; ++r) {
          const float2 ab = s2[r];
          const float c = __ldg(cj + r * ncheb + n);
          x = fmaf(ab.x, c, x);
          y = fmaf(ab.y, c, y);
        }
        X[m] = x;
        Y[m] = y;
      }
    }
  } else if (W >= 16 && k > 4 * W) {
    long_grad_groups<W>(ta, tb, da, db, rl, lane, el, gr, rc, k);
  } else {
    // one term a root: three FMAs and a reciprocal per (literal, root)
    rc[lane] = make_float4(ta, tb, da, db);
    __syncwarp();
    const float4* rs = rc + (lane & ~(W - 1));  // the slot's W roots
    // chunks of 4 W literals; a last chunk takes only the rows of W it reaches
    int c0 = 0;
    for (; c0 + 3 * W < k; c0 += 4 * W) grad_root_terms<W, 4>(rs, el, gr, c0, rl, k);
    const int rows = (k - c0 + W - 1) / W;
    if (rows == 3) grad_root_terms<W, 3>(rs, el, gr, c0, rl, k);
    else if (rows == 2) grad_root_terms<W, 2>(rs, el, gr, c0, rl, k);
    else if (rows == 1) grad_root_terms<W, 1>(rs, el, gr, c0, rl, k);
  }
  __syncwarp();  // the root row is read before the next pass writes it
  return v;
}

// The expanded roots' derivative terms at every literal of the slot: the
// slot's sums (X_n, Y_n) published to the warp's row in duplicated pairs
// (2 W entries a slot, so at most 2 W terms), then per literal sum_n T_n(t)
// (l X_n + Y_n), t = 2 l^2 - 1, by Clenshaw's recurrence, two literals a
// lane on paired FMAs (three a term).
template <int W>
__device__ __forceinline__ void cheb_grad(const float* el, float* gr, float4* rc, int lane, int rl, int k, int ncheb,
                                          const float (&X)[2], const float (&Y)[2]) {
  float4* cx = rc + (lane / W) * (2 * W);
#pragma unroll
  for (int m = 0; m < 2; ++m) {
    const int n = rl + m * W;
    if (n < ncheb) cx[n] = make_float4(X[m], X[m], Y[m], Y[m]);
  }
  __syncwarp();
  const float2 m1 = make_float2(-1.0f, -1.0f);
  for (int i = rl; i < k; i += 2 * W) {
    const bool two = i + W < k;
    const float2 l = make_float2(el[i], two ? el[i + W] : 0.0f);
    const float2 t = ffma2(make_float2(2.0f * l.x, 2.0f * l.y), l, m1);
    const float2 d = make_float2(2.0f * t.x, 2.0f * t.y);
    float2 b1 = make_float2(0.0f, 0.0f), b2 = b1;
#pragma unroll 4
    for (int n = ncheb - 1; n >= 1; --n) {
      const float4 c = cx[n];
      const float2 nb = ffma2(d, b1, ffma2(m1, b2, ffma2(l, lo2(c), hi2(c))));
      b2 = b1;
      b1 = nb;
    }
    const float4 c = cx[0];
    const float2 g = ffma2(t, b1, ffma2(m1, b2, ffma2(l, lo2(c), hi2(c))));
    gr[i] += g.x;
    if (two) gr[i + W] += g.y;
  }
  __syncwarp();  // the row is read before it is written again
}

// resident warps per SM the kernel is compiled for (register cap)
constexpr int LONG_WARPS_PER_SM = 32;

template <typename XT, int W, int NW>
__global__ void __launch_bounds__(NW * 32, LONG_WARPS_PER_SM / NW) fe_grad_long_pgf_kernel(FeGroupArgs a) {
  constexpr int SL = 32 / W;   // restarts per warp
  constexpr int RT = NW * SL;  // restarts per CTA
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bar;
  pdl_wait();
  pdl_trigger();
  const LongPgfLayout L(a.k, W, NW);
  const int tiles = (a.nb + RT - 1) / RT;
  const int cl = blockIdx.x / tiles;
  const int tile = blockIdx.x - cl * tiles;
  const int cb = a.c_begin + cl;
  const int k = __ldg(a.cons_k + cb);
  const int litoff = __ldg(a.cons_lit + cb);
  const float4* tab = a.coef + __ldg(a.cons_tab + cb);  // read through L1
  const float4 head = __ldg(tab);
  const int nroots = static_cast<int>(head.y);
  const bool has_real = head.w > 0.5f;

  int2* lits = reinterpret_cast<int2*>(smem);
  float* ell = reinterpret_cast<float*>(smem + L.off_ell);
  float* gs = reinterpret_cast<float*>(smem + L.off_gs);
  float4* rcs = reinterpret_cast<float4*>(smem + L.off_rc);

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned lit_bytes = static_cast<unsigned>((k + 1) & ~1) * 8u;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&bar, lit_bytes + a.extra_tx);
    bulk_g2s(lits, a.litslot + litoff, lit_bytes, &bar);
  }
  for (int i = tid; i < RT * L.gp; i += NW * 32) gs[i] = 0.0f;
  const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
  if (!mbar_wait_bounded(&bar, 0, limit)) {
    if (tid == 0) atomicExch(a.err, DEV_ERR_TIMEOUT);
    mbar_wait_bounded(&bar, 0, limit);  // let copies in flight land before exit
    return;
  }

  // stage l[r][i] = s_i x[v_i][b] (0 past k and for restarts past nb)
  const XT* x = static_cast<const XT*>(a.x);
  const int bt = tile * RT;
  for (int idx = tid; idx < L.kpad * RT; idx += NW * 32) {
    const int i = idx / RT, r = idx - (idx / RT) * RT;
    float lv = 0.0f;
    if (i < k && bt + r < a.nb) {
      const int2 li = lits[i];
      const float xv = load_x<XT>(x + static_cast<long long>(li.x >> 1) * a.x_pitch + a.b0 + bt + r);
      lv = (li.x & 1) ? -xv : xv;
    }
    ell[r * L.ep + i] = lv;
  }
  __syncthreads();

  const int slot = lane / W, rl = lane & (W - 1);
  const int r = w * SL + slot;
  const float* el = ell + r * L.ep;
  float* gr = gs + r * L.gp;
  float4* rcw = rcs + w * LONG_ROW;
  const int nseg = (k + LONG_SEG - 1) / LONG_SEG;
  const int n_last = k - LONG_SEG * (nseg - 1);
  float fe_part = 0.0f;

  // passes of W roots; from the table's first form-B root on (a multiple of
  // 32, so no pass straddles it) the passes use form B
  // The table's first first_x roots (a multiple of 32, all form A) have
  // their derivative terms expanded in ncheb Chebyshev terms; a slot of W
  // lanes holds at most 2 W of the sums, so narrower slots take every root
  // exactly.
  const float4 h1 = __ldg(tab + 1);
  const int first_b = static_cast<int>(h1.x);
  const int ncheb = static_cast<int>(h1.z);
  const int first_x = ncheb <= 2 * W ? static_cast<int>(h1.y) : 0;
  const float* cheb = reinterpret_cast<const float*>(tab + 2 + 2 * nroots);
  float X[2] = {0.0f, 0.0f}, Y[2] = {0.0f, 0.0f};
  for (int j0 = 0; j0 < nroots; j0 += W) {
    if (j0 < first_x)
      fe_part += pgf_pass<W, false, true>(tab, nroots, j0, rl, lane, el, gr, rcw, k, nseg, n_last, cheb, ncheb, X, Y);
    else if (j0 < first_b)
      fe_part += pgf_pass<W, false, false>(tab, nroots, j0, rl, lane, el, gr, rcw, k, nseg, n_last, cheb, ncheb, X, Y);
    else
      fe_part += pgf_pass<W, true, false>(tab, nroots, j0, rl, lane, el, gr, rcw, k, nseg, n_last, cheb, ncheb, X, Y);
  }
  if (first_x > 0) cheb_grad<W>(el, gr, rcw, lane, rl, k, ncheb, X, Y);

  if (has_real) {
    // the real root: value c_mid prod l, gradient c_mid prod over the other
    // literals (l can be zero, so no division). The slot's lanes split the
    // literals into W contiguous chunks (at most AFS_MAX_LEN / W); across
    // lanes a prefix/suffix scan of the chunk products; within its chunk a
    // lane takes sub-blocks of RR_SUB literals from the last one back, with
    // the suffix after the sub-block carried along, the prefix before it
    // re-multiplied from the chunk's start, and the within-block suffixes in
    // registers.
    constexpr int RR_SUB = 8, RR_NSUB = (AFS_MAX_LEN / W + RR_SUB - 1) / RR_SUB;
    const float em = head.z;
    const int chunk = (k + W - 1) / W;
    const int i0 = min(k, rl * chunk), i1 = min(k, i0 + chunk);
    float sl = 1.0f;
    for (int i = i0; i < i1; ++i) sl *= el[i];
    float inc = sl;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
      const float o = __shfl_up_sync(0xffffffffu, inc, d, W);
      if (rl >= d) inc *= o;
    }
    float pre = __shfl_up_sync(0xffffffffu, inc, 1, W);
    if (rl == 0) pre = 1.0f;
    const float tot = __shfl_sync(0xffffffffu, inc, W - 1, W);
    float sinc = sl;
#pragma unroll
    for (int d = 1; d < W; d <<= 1) {
      const float o = __shfl_down_sync(0xffffffffu, sinc, d, W);
      if (rl + d < W) sinc *= o;
    }
    float suf = __shfl_down_sync(0xffffffffu, sinc, 1, W);
    if (rl == W - 1) suf = 1.0f;
    float C = suf;  // the product after the sub-block
#pragma unroll
    for (int sb = RR_NSUB - 1; sb >= 0; --sb) {
      const int b0 = i0 + sb * RR_SUB;
      if (b0 >= i1) continue;
      float A = em * pre;  // c_mid times the product before the sub-block
      for (int i = i0; i < b0; ++i) A *= el[i];
      float lv[RR_SUB], ws[RR_SUB];
#pragma unroll
      for (int t = 0; t < RR_SUB; ++t) lv[t] = b0 + t < i1 ? el[b0 + t] : 1.0f;
      float w = 1.0f;
#pragma unroll
      for (int t = RR_SUB - 1; t >= 0; --t) {
        ws[t] = w;
        w *= lv[t];
      }
      float pl = A * C;
#pragma unroll
      for (int t = 0; t < RR_SUB; ++t) {
        if (b0 + t < i1) gr[b0 + t] += pl * ws[t];
        pl *= lv[t];
      }
      C *= w;
    }
    fe_part += em * tot;
  }

  if (a.fe != nullptr && rl == 0 && bt + r < a.nb)
    a.fe[static_cast<long long>(__ldg(a.cons_orig + cb)) * a.fe_pitch + a.b0 + bt + r] = head.x + fe_part;
  __syncthreads();
  for (int idx = tid; idx < k * RT; idx += NW * 32) {
    const int i = idx / RT, rr = idx - (idx / RT) * RT;
    if (bt + rr < a.nb) {
      const int2 li = lits[i];
      const float gv = gs[rr * L.gp + i];
      a.go[static_cast<long long>(li.y) * a.go_pitch + bt + rr] = (li.x & 1) ? -gv : gv;
    }
  }
}

template <typename XT, int W, int NW>
void launch_pgf_t(const FeGroupArgs& a, cudaStream_t s) {
  constexpr int RT = NW * (32 / W);
  const LongPgfLayout L(a.k, W, NW);
  const long long tiles = (a.nb + RT - 1) / RT;
  launch_pdl(fe_grad_long_pgf_kernel<XT, W, NW>, dim3(static_cast<unsigned>(tiles * a.c_count)), dim3(NW * 32),
             L.bytes, s, a);
}

template <typename K>
bool raise_cap(K kernel, int optin) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return false;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - static_cast<int>(fa.sharedSizeBytes)) == cudaSuccess;
}

template <typename XT>
bool prepare_xt(int optin) {
  bool ok = true;
  ok &= raise_cap(fe_grad_long_pgf_kernel<XT, 32, 4>, optin);
  ok &= raise_cap(fe_grad_long_pgf_kernel<XT, 32, 8>, optin);
  ok &= raise_cap(fe_grad_long_pgf_kernel<XT, 16, 2>, optin);
  ok &= raise_cap(fe_grad_long_pgf_kernel<XT, 16, 4>, optin);
  ok &= raise_cap(fe_grad_long_pgf_kernel<XT, 8, 2>, optin);
  return ok;
}

template <typename XT>
bool launch_xt(const FeGroupArgs& a, int wl, int nw, cudaStream_t s) {
  if (wl == 32 && nw == 4) launch_pgf_t<XT, 32, 4>(a, s);
  else if (wl == 32 && nw == 8) launch_pgf_t<XT, 32, 8>(a, s);
  else if (wl == 16 && nw == 2) launch_pgf_t<XT, 16, 2>(a, s);
  else if (wl == 16 && nw == 4) launch_pgf_t<XT, 16, 4>(a, s);
  else if (wl == 8 && nw == 2) launch_pgf_t<XT, 8, 2>(a, s);
  else return false;
  return true;
}

template <typename XT>
int occupancy_xt(int wl, int nw, size_t smem) {
  int blocks = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (wl == 32 && nw == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fe_grad_long_pgf_kernel<XT, 32, 4>, 128, smem);
  else if (wl == 32 && nw == 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fe_grad_long_pgf_kernel<XT, 32, 8>, 256, smem);
  else if (wl == 16 && nw == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fe_grad_long_pgf_kernel<XT, 16, 2>, 64, smem);
  else if (wl == 16 && nw == 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fe_grad_long_pgf_kernel<XT, 16, 4>, 128, smem);
  else if (wl == 8 && nw == 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fe_grad_long_pgf_kernel<XT, 8, 2>, 64, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks * nw;
}

}  // namespace

const int LONG_PGF_SHAPES[LONG_PGF_NSHAPES][2] = {{32, 4}, {32, 8}, {16, 2}, {16, 4}, {8, 2}};

size_t long_pgf_smem_bytes(int kmax, int wl, int nw) { return LongPgfLayout(kmax, wl, nw).bytes; }

bool prepare_long_pgf(int optin) {
  if (LongPgfLayout(AFS_MAX_LEN, 8, 2).bytes > static_cast<size_t>(optin)) return false;
  return prepare_xt<float>(optin) && prepare_xt<__nv_bfloat16>(optin);
}

int long_pgf_resident_warps(int xt, int kmax, int wl, int nw) {
  const size_t smem = LongPgfLayout(kmax, wl, nw).bytes;
  return xt == XT_F32 ? occupancy_xt<float>(wl, nw, smem) : occupancy_xt<__nv_bfloat16>(wl, nw, smem);
}

bool launch_fe_long_pgf(const FeGroupArgs& a, int xt, int wl, int nw, cudaStream_t s) {
  return xt == XT_F32 ? launch_xt<float>(a, wl, nw, s) : launch_xt<__nv_bfloat16>(a, wl, nw, s);
}

}  // namespace afs
