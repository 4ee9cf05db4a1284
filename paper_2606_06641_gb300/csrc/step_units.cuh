// Per-warp units of the step shared by the standalone kernels and the
// persistent step kernel: state stores, the fused 3-literal derivative sums,
// the CSR gather with the projected update (Algorithm 1's step and
// projection) and the bit-sliced exact check of one constraint range. COH:
// data written earlier in the same kernel (state, derivative rows, sums,
// check words) is read with L2-coherent loads instead of the read-only cache.
#pragma once
#include <cuda_bf16.h>

#include "afsat_internal.h"
#include "fe_short.cuh"

namespace afs {

template <typename XT>
__device__ __forceinline__ void store_x(XT* p, float v);
template <>
__device__ __forceinline__ void store_x<float>(float* p, float v) {
  *p = v;
}
template <>
__device__ __forceinline__ void store_x<__nv_bfloat16>(__nv_bfloat16* p, float v) {
  *p = __float2bfloat16_rn(v);
}
template <typename XT>
__device__ __forceinline__ float load_x_rw(const XT* p);
template <>
__device__ __forceinline__ float load_x_rw<float>(const float* p) {
  return *p;
}
template <>
__device__ __forceinline__ float load_x_rw<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

// The value a state entry holds once stored (BF16 storage rounds).
template <typename XT>
__device__ __forceinline__ float stored_value(float v);
template <>
__device__ __forceinline__ float stored_value<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float stored_value<__nv_bfloat16>(float v) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

// Fused constraints (k = KFUSE = 3, probability-generating tables): the
// derivative of occurrence `self` is s_self * dFE/dl_self, recomputed from the
// two other literals' state: the real root w = -1 contributes E l1 l2, the
// complex pair (scaled form) Re(E' tan (l1 tan + i)(l2 tan + i)) -- the same
// products at the roots as the FE kernel's gradient, without the self factor.
// Each entry carries the root constants with the other literals' signs
// folded in ({E s1 s2, tan s1, tan s2, E'r tan}, {E'i tan, s_self, v1, v2}),
// read with uniform loads (the warp's lanes share them); the gathers of FB
// occurrences are in flight at a time, R consecutive restarts per lane
// starting at column col.
template <typename XT, int R, int FB, bool OFF32 = false, bool COH = false>
__device__ __forceinline__ void fused_sum(const CsrArgs& a, int v, long long col, bool act, float (&acc)[R]) {
  const int f0 = __ldg(a.fus_off + v), f1 = __ldg(a.fus_off + v + 1);
  const XT* xc = static_cast<const XT*>(a.x) + col;
  // lists are padded to pairs: with FB == FUS_PAD every entry of a batch
  // exists, and col (clamped to the launch's first restart on idle lanes) is
  // a valid column, so the loads need no guard
  constexpr bool PAIRS = FB == FUS_PAD;
  float cs = 0.0f;  // sum of the entries' constant terms (the same for every restart)
  for (int f = f0; f < f1; f += FB) {  // uniform per warp
    float4 c[FB];
    float x1[FB][R], x2[FB][R];
#pragma unroll
    for (int u = 0; u < FB; ++u) {
      const bool ok = PAIRS || f + u < f1;
      c[u] = ok ? __ldg(a.fus + 2 * (f + u)) : make_float4(0.f, 0.f, 0.f, 0.f);
      const int2 vv = ok ? __ldg(reinterpret_cast<const int2*>(a.fus + 2 * (f + u) + 1)) : make_int2(0, 0);
      const bool ld = PAIRS || (act && ok);
      // OFF32: the launch checked that every row offset v * x_pitch fits 32 bits
      const XT* p1 = OFF32 ? xc + static_cast<unsigned>(vv.x) * static_cast<unsigned>(a.x_pitch)
                           : xc + static_cast<long long>(vv.x) * a.x_pitch;
      const XT* p2 = OFF32 ? xc + static_cast<unsigned>(vv.y) * static_cast<unsigned>(a.x_pitch)
                           : xc + static_cast<long long>(vv.y) * a.x_pitch;
      if constexpr (R == 4) {
        if (ld) {
          load_xvec<XT, 4, COH>(p1, x1[u]);
          load_xvec<XT, 4, COH>(p2, x2[u]);
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) x1[u][r] = x2[u][r] = 0.0f;
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          x1[u][r] = ld ? load_x<XT, COH>(p1 + r) : 0.0f;
          x2[u][r] = ld ? load_x<XT, COH>(p2 + r) : 0.0f;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < FB; ++u) {
      // the level expansion of the entry's derivative, x1 (A x2 + B1) + B2 x2
      // (+ C, summed once); an absent occurrence has all constants 0
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float t1 = fmaf(c[u].x, x2[u][r], c[u].y);
        acc[r] = fmaf(x1[u][r], t1, acc[r]);
        acc[r] = fmaf(c[u].z, x2[u][r], acc[r]);
      }
      cs += c[u].w;
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] += cs;
}

// fused_sum for few restarts, where a variable's occurrence list is a chain
// of dependent loads: the warp loads up to 32 entries of the list at once
// (one per lane) and takes each from its lane by shuffles, so a batch of FBW
// occurrences costs one round trip for the state instead of two. The same
// operations in the same order as fused_sum (4 restarts per lane), so the
// sums are bit-identical.
template <typename XT, int FBW, bool OFF32 = false, bool COH = false>
__device__ __forceinline__ void fused_sum_pf(const CsrArgs& a, int v, long long col, bool act, int lane,
                                             float (&acc)[4]) {
  const int f0 = __ldg(a.fus_off + v), f1 = __ldg(a.fus_off + v + 1);
  const XT* xc = static_cast<const XT*>(a.x) + col;
  float cs = 0.0f;
  for (int fb = f0; fb < f1; fb += 32) {  // uniform per warp
    const int cnt = min(32, f1 - fb);
    float4 cl = make_float4(0.f, 0.f, 0.f, 0.f);
    int2 vl = make_int2(0, 0);
    if (lane < cnt) {
      cl = __ldg(a.fus + 2 * (fb + lane));
      vl = __ldg(reinterpret_cast<const int2*>(a.fus + 2 * (fb + lane) + 1));
    }
    for (int u0 = 0; u0 < cnt; u0 += FBW) {
      float4 c[FBW];
      float x1[FBW][4], x2[FBW][4];
#pragma unroll
      for (int u = 0; u < FBW; ++u) {
        const int src = (u0 + u) & 31;
        c[u] = make_float4(__shfl_sync(0xffffffffu, cl.x, src), __shfl_sync(0xffffffffu, cl.y, src),
                           __shfl_sync(0xffffffffu, cl.z, src), __shfl_sync(0xffffffffu, cl.w, src));
        const int v1 = __shfl_sync(0xffffffffu, vl.x, src), v2 = __shfl_sync(0xffffffffu, vl.y, src);
        const XT* p1 = OFF32 ? xc + static_cast<unsigned>(v1) * static_cast<unsigned>(a.x_pitch)
                             : xc + static_cast<long long>(v1) * a.x_pitch;
        const XT* p2 = OFF32 ? xc + static_cast<unsigned>(v2) * static_cast<unsigned>(a.x_pitch)
                             : xc + static_cast<long long>(v2) * a.x_pitch;
        if (act && u0 + u < cnt) {
          load_xvec<XT, 4, COH>(p1, x1[u]);
          load_xvec<XT, 4, COH>(p2, x2[u]);
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r) x1[u][r] = x2[u][r] = 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < FBW; ++u) {
        if (u0 + u < cnt) {  // uniform per warp
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float t1 = fmaf(c[u].x, x2[u][r], c[u].y);
            acc[r] = fmaf(x1[u][r], t1, acc[r]);
            acc[r] = fmaf(c[u].z, x2[u][r], acc[r]);
          }
          cs += c[u].w;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) acc[r] += cs;
}
constexpr int FUSED_PF_BATCH = 4;  // occurrences whose state loads are in flight together (fused_sum_pf)

// Invalidate the 128-byte L2 line at p (128-byte aligned) without writing it
// back. `after` is a value loaded from that line: the operand makes the
// discard wait for the load.
__device__ __forceinline__ void l2_discard_line(const void* p, float after) {
  asm volatile("discard.global.L2 [%0], 128;" ::"l"(p), "f"(after));
}

// Bookkeeping of the step's check, done once per (instance, word) by the
// warps of the instance's first variable: record the lowest solved restart
// and clear the word the next step's check will OR into.
__device__ __forceinline__ void csr_first_var_duty(const CsrArgs& a, int inst, int word, long long wi) {
  if (a.vcur != nullptr) {
    const int valid = min(32, a.B - word * 32);
    const unsigned ok = ~__ldcg(a.vcur + wi) & (valid >= 32 ? ~0u : ((1u << valid) - 1u));
    if (ok) atomicMin(a.solved + inst, word * 32 + __ffs(static_cast<int>(ok)) - 1);
  }
  if (a.vnext != nullptr) a.vnext[wi] = 0u;
}

// Store n <= 4 consecutive state values (one vector store when n == 4).
template <typename XT>
__device__ __forceinline__ void store_xvec(XT* p, const float (&v)[4], int n);
template <>
__device__ __forceinline__ void store_xvec<float>(float* p, const float (&v)[4], int n) {
  if (n == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    for (int e = 0; e < n; ++e) p[e] = v[e];
  }
}
template <>
__device__ __forceinline__ void store_xvec<__nv_bfloat16>(__nv_bfloat16* p, const float (&v)[4], int n) {
  if (n == 4) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]), hi = __floats2bfloat162_rn(v[2], v[3]);
    uint2 u;
    u.x = *reinterpret_cast<const unsigned*>(&lo);
    u.y = *reinterpret_cast<const unsigned*>(&hi);
    *reinterpret_cast<uint2*>(p) = u;
  } else {
    for (int e = 0; e < n; ++e) p[e] = __float2bfloat16_rn(v[e]);
  }
}

// Step-path variant: each lane owns 4 consecutive restarts, so a warp reads
// 512 contiguous bytes of every occurrence row (16-byte vector loads), four
// rows in flight, and updates 4 states. The state, the solved word and the
// instance's first variable are read before the gather so their latency
// overlaps it; 8 lanes together write one sign word. 64 registers (four
// 256-thread blocks per SM) measured faster than squeezing to five blocks.
// The grid is persistent (one wave of resident blocks)
// and warps stride over the (variable, 128-restart tile) tasks, so no partial
// last wave idles the machine. Needs the state's row pitch and the chunk
// start to be multiples of 32 and the buffers 16-byte aligned (true for the
// library's own state and occurrence buffers); lanes past nb are masked.
// OFF32: the launch checked that every state and row offset fits 32 bits.
template <typename XT, bool OFF32, bool COH = false>
__device__ __forceinline__ void csr_vec4_task(const CsrArgs& a, int vl, int tile, int lane) {
  const int bl = tile * 128 + lane * 4;
  const bool act = bl < a.nb;
  const int v = a.v_begin + vl;
  const int s0 = __ldg(a.csr_off + v), s1 = __ldg(a.csr_off + v + 1);
  const int inst = __ldg(a.var_inst + v);
  const int first_var = __ldg(a.var_inst + a.n_vars + inst);
  const int word = (a.b0 + bl) >> 5;
  const long long wi = static_cast<long long>(inst) * a.W + word;
  unsigned sw = 0u;  // solved (or fixed) bits of this lane's restarts
  if (act && a.vcur != nullptr) sw = ~(ld_u32<COH>(a.vcur + wi) >> (bl & 31));
  if (act && a.fixv != nullptr) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const long long g = static_cast<long long>(a.b0 + bl + e) * a.n_fix_groups / a.B;
      if (bl + e < a.nb && a.fixv[g * a.n_vars + v] != 0) sw |= 1u << e;
    }
  }
  const long long xi = OFF32 ? static_cast<long long>(static_cast<unsigned>(v) * static_cast<unsigned>(a.x_pitch) +
                                                     static_cast<unsigned>(a.b0 + bl))
                            : static_cast<long long>(v) * a.x_pitch + a.b0 + bl;
  float xo[4] = {0.f, 0.f, 0.f, 0.f};
  if (act) load_xvec<XT, 4, COH>(static_cast<const XT*>(a.x) + xi, xo);
  const float* col = a.go + (act ? bl : 0);
  float4 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  // fused occurrences: summed by the fused pass beside the FE launches (the
  // step path always provides gf when the instance has fused occurrences)
  const float* gfp = a.gf != nullptr && act ? a.gf + static_cast<long long>(v) * a.gf_pitch + bl : nullptr;
  const bool dis = a.discard_go && act && (lane & 7) == 0;
  // (loaded before the rows so that its latency overlaps theirs)
  const float4 gf = gfp != nullptr ? ld_f4<COH>(reinterpret_cast<const float4*>(gfp)) : make_float4(0.f, 0.f, 0.f, 0.f);
  // most variables have few rows: batches of four, the summation order
  // (row j into acc[j mod 4]) fixed by the slot order
  for (int s = s0; s < s1; s += 4) {
    float4 t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float* rp = OFF32 ? col + static_cast<unsigned>(s + u) * static_cast<unsigned>(a.go_pitch)
                              : col + static_cast<long long>(s + u) * a.go_pitch;
      t[u] = s + u < s1 ? ld_f4<COH>(reinterpret_cast<const float4*>(rp)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[u & 3].x += t[u].x;
      acc[u & 3].y += t[u].y;
      acc[u & 3].z += t[u].z;
      acc[u & 3].w += t[u].w;
    }
  }
  const float g[4] = {gf.x + ((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x)),
                      gf.y + ((acc[0].y + acc[1].y) + (acc[2].y + acc[3].y)),
                      gf.z + ((acc[0].z + acc[1].z) + (acc[2].z + acc[3].z)),
                      gf.w + ((acc[0].w + acc[1].w) + (acc[2].w + acc[3].w))};
  // the rows are dead once read (the next FE pass rewrites them): drop their
  // 128-byte L2 lines without a write-back, so that they make room for rows
  // still to be read instead of costing DRAM writes (g depends on every load)
  if (dis)
    for (int s = s0; s < s1; ++s) l2_discard_line(col + static_cast<long long>(s) * a.go_pitch, g[0]);
  unsigned nib = 0u;
  float xn[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    // a solved restart keeps x_t; restarts past nb only fill the vector
    xn[e] = ((sw >> e) & 1u) ? xo[e] : stored_value<XT>(fminf(fmaxf(fmaf(-a.eta, g[e], xo[e]), -1.0f), 1.0f));
    if (act && bl + e < a.nb) nib |= static_cast<unsigned>(xn[e] < 0.0f) << e;
  }
  if (act) store_xvec<XT>(static_cast<XT*>(a.x_out) + xi, xn, min(4, a.nb - bl));
  // 8 lanes x 4 restarts = one word
  unsigned wv = nib << ((lane & 7) * 4);
  wv |= __shfl_xor_sync(0xffffffffu, wv, 1);
  wv |= __shfl_xor_sync(0xffffffffu, wv, 2);
  wv |= __shfl_xor_sync(0xffffffffu, wv, 4);
  if ((lane & 7) == 0 && act) {
    if (a.sgn != nullptr) a.sgn[static_cast<long long>(v) * a.W + word] = wv;
    if (v == first_var) csr_first_var_duty(a, inst, word, wi);
  }
}

constexpr int CHECK_PLANES = 11;  // counts up to 2047 >= the longest constraint
constexpr int CHECK_STAGE = 32;   // literal words a warp stages at a time
constexpr int CHECK_WARPS = 4;

template <int MAXP>
__device__ __forceinline__ void add_words(unsigned (&P)[CHECK_PLANES], const unsigned* sw, int n, int np) {
  for (int i = 0; i < n; ++i) {
    unsigned carry = sw[i * 32];
#pragma unroll
    for (int p = 0; p < MAXP; ++p) {
      if (p < np) {
        const unsigned t = P[p] & carry;
        P[p] ^= carry;
        carry = t;
      }
    }
  }
}

// Violation word of one constraint from its count planes.
__device__ __forceinline__ unsigned violated_word(const unsigned (&P)[CHECK_PLANES], int k, int np,
                                                  unsigned long long em, const unsigned char* vt) {
  if (k <= 62) {
    unsigned long long m = em & ~(1ull << 63);
    unsigned hit = 0u;
    while (m) {
      const int u = __ffsll(static_cast<long long>(m)) - 1;
      m &= m - 1;
      unsigned e = ~0u;
#pragma unroll
      for (int p = 0; p < 6; ++p)
        if (p < np) e &= ((u >> p) & 1) ? P[p] : ~P[p];
      hit |= e;
    }
    return (em >> 63) ? ~hit : hit;
  }
  unsigned bad = 0u;
  for (int j = 0; j < 32; ++j) {
    int t = 0;
#pragma unroll
    for (int p = 0; p < CHECK_PLANES; ++p)
      if (p < np) t |= static_cast<int>((P[p] >> j) & 1u) << p;
    bad |= static_cast<unsigned>(__ldg(vt + t)) << j;
  }
  return bad;
}

// Gather the literal words of literals [base, base + cnt) (cnt <= 32) into
// the warp's stage, all loads in flight at once: lane j of row i holds the
// truth of literal base + i in restarts 32w + (0..31).
template <bool COH = false>
__device__ __forceinline__ void check_stage(const CheckArgs& a, const unsigned* sg, unsigned* st, int base, int cnt,
                                            int lane) {
  const int e = lane < cnt ? __ldg(a.lit_enc + base + lane) : 0;
  unsigned wv[CHECK_STAGE];
#pragma unroll
  for (int j = 0; j < CHECK_STAGE; ++j) {
    const int enc = __shfl_sync(0xffffffffu, e, j);
    wv[j] = j < cnt ? ld_u32<COH>(sg + static_cast<long long>(enc >> 1) * a.W) ^ (0u - static_cast<unsigned>(enc & 1))
                    : 0u;
  }
#pragma unroll
  for (int j = 0; j < CHECK_STAGE; ++j) st[j * 32] = wv[j];
  __syncwarp();
}


// One warp's share of the per-step check without a block-level merge: range
// `rgi` for the words w0 + 32 * chunk + lane (lane = word of 32 restarts); the
// violation words of the range are ORed straight into vword. `st` is the
// warp's CHECK_STAGE x 32 stage in shared memory.
template <bool COH>
__device__ __forceinline__ void check_unit_warp(const CheckArgs& a, int rgi, int chunk, int lane, unsigned* st) {
  const int wl = chunk * 32 + lane;
  const bool act = wl < a.wc;
  const int w = a.w0 + (act ? wl : 0);
  const int4 rg = __ldg(a.ranges + rgi);
  const int nc = rg.y - rg.x;
  const int offv = __ldg(a.lit_off + rg.x + min(lane, nc));
  const unsigned long long emv = lane < nc ? __ldg(a.em + rg.x + lane) : 0ull;
  const int l0 = __shfl_sync(0xffffffffu, offv, 0);
  const int l1 = __shfl_sync(0xffffffffu, offv, nc);
  const unsigned* sg = a.sgn + w;
  unsigned* stl = st + lane;
  unsigned P[CHECK_PLANES];
  unsigned bad = 0u;
  if (l1 - l0 <= CHECK_STAGE) {
    check_stage<COH>(a, sg, stl, l0, l1 - l0, lane);
    for (int c = 0; c < nc; ++c) {
      const int a0 = __shfl_sync(0xffffffffu, offv, c) - l0;
      const int a1 = __shfl_sync(0xffffffffu, offv, c + 1) - l0;
      const unsigned long long em = __shfl_sync(0xffffffffu, emv, c);
      const int k = a1 - a0;
      const int np = 32 - __clz(k);
#pragma unroll
      for (int p = 0; p < CHECK_PLANES; ++p) P[p] = 0u;
      add_words<6>(P, stl + a0 * 32, k, np);
      bad |= violated_word(P, k, np, em, nullptr);
    }
  } else {
    const int k = l1 - l0;
    const int np = 32 - __clz(k);
#pragma unroll
    for (int p = 0; p < CHECK_PLANES; ++p) P[p] = 0u;
    for (int b = 0; b < k; b += CHECK_STAGE) {
      const int cnt = min(CHECK_STAGE, k - b);
      check_stage<COH>(a, sg, stl, l0 + b, cnt, lane);
      add_words<CHECK_PLANES>(P, stl, cnt, np);
      __syncwarp();
    }
    bad = violated_word(P, k, np, __shfl_sync(0xffffffffu, emv, 0), a.viol + __ldg(a.viol_off + rg.x));
  }
  __syncwarp();  // the stage is read before the warp's next unit stages
  if (act && bad) atomicOr(a.vword + static_cast<long long>(rg.z) * a.W + w, bad);
}

// The per-step check of one run of constraints for one restart word, one
// constraint per lane (for few words, where a lane per word would leave most
// of the warp idle): run `rgi` (<= 31 constraints of one instance, each
// k <= 62, <= CHECK_WIDE_STAGE literals) and word `word`. The run's literal
// words are staged in the warp's shared memory with all loads in flight at
// once; each lane adds its constraint's words into count planes and tests the
// counts, and the warp's violation words are OR-reduced into vword (COUNT:
// the violated constraints per restart are added into unsat instead). The
// same integer results as the lane-per-word forms, bit for bit.
template <bool COH, bool COUNT = false>
__device__ __forceinline__ void check_wide_unit(const CheckArgs& a, int rgi, int word, int lane, unsigned* st) {
  const int4 rg = __ldg(a.ranges + rgi);
  const int nc = rg.y - rg.x;
  const int offv = __ldg(a.lit_off + rg.x + min(lane, nc));
  const unsigned long long em = lane < nc ? __ldg(a.em + rg.x + lane) : 0ull;
  const int l0 = __shfl_sync(0xffffffffu, offv, 0);
  const int nl = __shfl_sync(0xffffffffu, offv, nc) - l0;
  const int own_end = __shfl_down_sync(0xffffffffu, offv, 1);
  const unsigned* sg = a.sgn + word;
  constexpr int PER = CHECK_WIDE_STAGE / 32;
  int e[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) e[j] = lane + 32 * j < nl ? __ldg(a.lit_enc + l0 + lane + 32 * j) : 0;
  unsigned wv[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j)
    wv[j] = lane + 32 * j < nl
                ? ld_u32<COH>(sg + static_cast<long long>(e[j] >> 1) * a.W) ^ (0u - static_cast<unsigned>(e[j] & 1))
                : 0u;
#pragma unroll
  for (int j = 0; j < PER; ++j)
    if (lane + 32 * j < nl) st[lane + 32 * j] = wv[j];
  __syncwarp();
  unsigned bad = 0u;
  if (lane < nc) {
    const int a0 = offv - l0, k = own_end - offv;
    const int np = 32 - __clz(k);
    unsigned P[CHECK_PLANES];
#pragma unroll
    for (int p = 0; p < CHECK_PLANES; ++p) P[p] = 0u;
    for (int i = 0; i < k; ++i) {
      unsigned carry = st[a0 + i];
#pragma unroll
      for (int p = 0; p < 6; ++p) {
        if (p < np) {
          const unsigned t = P[p] & carry;
          P[p] ^= carry;
          carry = t;
        }
      }
    }
    bad = violated_word(P, k, np, em, nullptr);
  }
  __syncwarp();  // the stage is read before the warp's next unit stages
  if constexpr (COUNT) {
    // count mode: lane j adds the run's violated constraints of restart 32 word + j
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = __popc(__ballot_sync(0xffffffffu, (bad >> j) & 1u));
      if (lane == j) cnt = c;
    }
    const int b = word * 32 + lane;
    if (cnt && b < a.B) atomicAdd(a.unsat + static_cast<long long>(rg.z) * a.B + b, cnt);
  } else {
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0 && bad) atomicOr(a.vword + static_cast<long long>(rg.z) * a.W + word, bad);
  }
}

}  // namespace afs
