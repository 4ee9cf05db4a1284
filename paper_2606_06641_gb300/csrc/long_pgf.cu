// FE + analytic gradient of long constraints (k > 32) in the
// probability-generating basis.
//
// Sec. 2.1.2: a symmetric constraint's expansion is a combination, with the
// constraint's DFT coefficients, of products over its literals at the roots
// of unity; the gradient of literal i at a root is the product of the other
// literals' factors, taken here as prefix x suffix (no division, so zero
// factors are safe). Sec. 3.5: conjugate roots are paired, so only the roots
// of one half-plane are evaluated (each complex one counted twice through
// the real part) plus, for odd k, the real root w = -1.
//
// Layout. One CTA per (constraint, RT restarts): NW warps, each warp holds
// 32 / W restarts ("slots") and each slot's W lanes own W roots of a pass;
// passes walk the table's roots W at a time. The literal list is staged with
// cp.async.bulk on an mbarrier (bounded wait), the literal values l = s x of
// the CTA's restarts in shared memory rows, read four at a time by 16-byte
// broadcast loads.
//
// Factor form (coefficient table built on the host): at every complex root
// the literal factor is s (p l + i), so a complex multiply of a running
// product by it is three FP32 instructions (w = p l, two FMAs). Walks go in
// segments of LONG_SEG literals; at each segment boundary running products
// are at their true size (|prod| <= 1), which the table's powers of s
// restore: inside a segment the checkpoint carries s^7 and the suffix s^8,
// so that Re(prefix * suffix) is the true contribution and neither running
// product leaves the FP32 range. No exponent bookkeeping is needed.
//
// Per pass and lane: a forward walk stores one prefix checkpoint per segment
// in shared memory; the backward walk, segment by segment from the end,
// rebuilds the segment's prefixes in registers from the checkpoint, walks the
// suffix down from the gradient weight and writes each contribution
// Re(prefix_t * suffix_t) to a per-warp shared-memory tile (column = lane,
// row = literal); the lanes then sum the tile's rows over the slot's roots
// with 16-byte reads and add them to the slot's gradient row. The sum order
// is fixed (deterministic). The real root's factor is l itself: its product
// and leave-one-out products are real and take a prefix/suffix scan over the
// slot's lanes after the passes.
#include <cuda_bf16.h>

#include "afsat.h"
#include "afsat_internal.h"
#include "bulk_copy.cuh"
#include "coef.h"
#include "fe_short.cuh"

namespace afs {

namespace {

constexpr int LTP = 36;  // tile row pitch in floats (16-byte column reads hit distinct banks)

// Shared memory of one CTA.
struct LongPgfLayout {
  int kpad, nseg, rt, ep, gp;
  size_t off_ell, off_gs, off_ck, off_tile, bytes;
  __host__ __device__ LongPgfLayout(int kmax, int W, int NW) {
    kpad = (kmax + LONG_SEG - 1) / LONG_SEG * LONG_SEG;
    nseg = kpad / LONG_SEG;
    rt = NW * (32 / W);
    const int k32 = (kpad + 31) & ~31;
    ep = k32 + 8;                   // literal-value rows: the slots' 16-byte reads fall in distinct banks
    gp = k32 + (W < 32 ? W : 0);    // gradient rows: the slots' column updates fall in distinct banks
    off_ell = static_cast<size_t>(kpad) * 8;                         // literal list (int2)
    off_gs = off_ell + static_cast<size_t>(rt) * ep * 4;            // literal values
    off_ck = off_gs + static_cast<size_t>(rt) * gp * 4;             // gradient accumulators
    off_tile = off_ck + static_cast<size_t>(NW) * nseg * 32 * 8;    // prefix checkpoints
    bytes = off_tile + static_cast<size_t>(NW) * LONG_SEG * LTP * 4;  // contribution tiles
  }
};

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

// Backward walk of one segment of N literals: prefixes rebuilt from the
// scaled checkpoint Q, suffix S (scaled) walked down, contribution of literal
// t written to tcol[t * LTP]. el is 16-byte aligned; the row is padded, so
// the last vector read may pass N. Form A keeps w = p l per literal in
// registers (computed once for both walks), form B the literal values.
template <int N, bool FB>
__device__ __forceinline__ void pgf_segment(const float* el, float p, float Qr, float Qi, float& Sr, float& Si,
                                            float* tcol) {
  float wv[N], pr[N], pi[N];
  const float sc = FB ? 1.0f : p;
#pragma unroll
  for (int t = 0; t < N; t += 4) {
    const float4 v = *reinterpret_cast<const float4*>(el + t);
    wv[t] = v.x * sc;
    if (t + 1 < N) wv[t + 1] = v.y * sc;
    if (t + 2 < N) wv[t + 2] = v.z * sc;
    if (t + 3 < N) wv[t + 3] = v.w * sc;
  }
  pr[0] = Qr;
  pi[0] = Qi;
#pragma unroll
  for (int t = 0; t + 1 < N; ++t) {
    pr[t + 1] = pr[t];
    pi[t + 1] = pi[t];
    if constexpr (FB) bmul(wv[t], p, pr[t + 1], pi[t + 1]);
    else gmul(wv[t], pr[t + 1], pi[t + 1]);
  }
#pragma unroll
  for (int t = N - 1; t >= 0; --t) {
    tcol[t * LTP] = fmaf(pr[t], Sr, -pi[t] * Si);
    if constexpr (FB) bmul(wv[t], p, Sr, Si);
    else gmul(wv[t], Sr, Si);
  }
}

template <bool FB>
__device__ __forceinline__ void pgf_tail_segment(int n, const float* el, float p, float Qr, float Qi, float& Sr,
                                                 float& Si, float* tcol) {
  switch (n) {
#define AFS_TAIL_CASE(N) \
  case N:                \
    pgf_segment<N, FB>(el, p, Qr, Qi, Sr, Si, tcol); \
    break;
    AFS_TAIL_CASE(1) AFS_TAIL_CASE(2) AFS_TAIL_CASE(3) AFS_TAIL_CASE(4) AFS_TAIL_CASE(5) AFS_TAIL_CASE(6)
    AFS_TAIL_CASE(7) AFS_TAIL_CASE(8) AFS_TAIL_CASE(9) AFS_TAIL_CASE(10) AFS_TAIL_CASE(11) AFS_TAIL_CASE(12)
    AFS_TAIL_CASE(13) AFS_TAIL_CASE(14) AFS_TAIL_CASE(15) AFS_TAIL_CASE(16)
#undef AFS_TAIL_CASE
    default:
      break;
  }
}

// Sums of the warp tile's rows (literals of the segment) over each slot's
// roots, added to the slot's gradient row gseg (n literals in the segment).
template <int W>
__device__ __forceinline__ void tile_column_sums(const float* tw, int lane, float* gseg, int n) {
  if constexpr (W == 8) {
    const int h = lane >> 3, c = lane & 7;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int col = c + 8 * cc;
      const float4* q = reinterpret_cast<const float4*>(tw + col * LTP + h * 8);
      const float4 u0 = q[0], u1 = q[1];
      const float s = ((u0.x + u0.y) + (u0.z + u0.w)) + ((u1.x + u1.y) + (u1.z + u1.w));
      if (col < n) gseg[col] += s;
    }
  } else {
    const int h = lane >> 4, c = lane & 15;
    const float4* q = reinterpret_cast<const float4*>(tw + c * LTP + h * 16);
    const float4 u0 = q[0], u1 = q[1], u2 = q[2], u3 = q[3];
    float s = (((u0.x + u0.y) + (u0.z + u0.w)) + ((u1.x + u1.y) + (u1.z + u1.w))) +
              (((u2.x + u2.y) + (u2.z + u2.w)) + ((u3.x + u3.y) + (u3.z + u3.w)));
    if constexpr (W == 32) {
      s += __shfl_xor_sync(0xffffffffu, s, 16);
      if (lane < n) gseg[lane] += s;
    } else {
      if (c < n) gseg[c] += s;
    }
  }
}

// One pass: the slot's W lanes evaluate roots j0 .. j0 + W - 1 of the table
// for their restart (forward checkpoints, value, backward contributions
// added to the gradient row gr); returns the pass's value summed over the
// slot's roots.
template <int W, bool FB>
__device__ __forceinline__ float pgf_pass(const float4* tab, int nroots, int j0, int rl, int lane, const float* el,
                                          float* gr, float2* myck, float* tw, int nseg, int n_last) {
  const int j = j0 + rl;
  float p = 0.f, s7r = 0.f, s7i = 0.f, s16r = 0.f, s16i = 0.f, sar = 0.f, sai = 0.f, scr = 0.f, sci = 0.f;
  float dr = 0.f, di = 0.f, er = 0.f, ei = 0.f;
  if (j < nroots) {
    const float4* rg = tab + 2 + 4 * j;
    const float4 g0 = __ldg(rg), g1 = __ldg(rg + 1), g2 = __ldg(rg + 2), g3 = __ldg(rg + 3);
    p = g0.x; s7r = g0.y; s7i = g0.z;
    s16r = g1.x; s16i = g1.y; sar = g1.z; sai = g1.w;
    scr = g2.x; sci = g2.y; dr = g2.z; di = g2.w;
    er = g3.x; ei = g3.y;
  }
  // forward: one checkpoint (true size) per segment start
  float Pr = 1.0f, Pi = 0.0f;
  for (int sg = 0; sg + 1 < nseg; ++sg) {
    myck[sg * 32 + lane] = make_float2(Pr, Pi);
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
  myck[(nseg - 1) * 32 + lane] = make_float2(Pr, Pi);
  {
    const float* e = el + (nseg - 1) * LONG_SEG;
    for (int t = 0; t < n_last; ++t) fmul<FB>(e[t], p, Pr, Pi);
  }
  // the pass's value, summed over the slot's roots (every lane of the slot)
  float v = fmaf(er, Pr, -ei * Pi);
#pragma unroll
  for (int o = W / 2; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);

  // backward: the last segment first, then the full ones
  float Sr = dr, Si = di;
  {
    float2 Q = myck[(nseg - 1) * 32 + lane];
    cmul(Q.x, Q.y, sar, sai);
    pgf_tail_segment<FB>(n_last, el + (nseg - 1) * LONG_SEG, p, Q.x, Q.y, Sr, Si, tw + lane);
    cmul(Sr, Si, scr, sci);
    __syncwarp();
    tile_column_sums<W>(tw, lane, gr + (nseg - 1) * LONG_SEG, n_last);
    __syncwarp();  // the tile is read before the next segment's rows
  }
  for (int sg = nseg - 2; sg >= 0; --sg) {
    float2 Q = myck[sg * 32 + lane];
    cmul(Q.x, Q.y, s7r, s7i);
    pgf_segment<LONG_SEG, FB>(el + sg * LONG_SEG, p, Q.x, Q.y, Sr, Si, tw + lane);
    cmul(Sr, Si, s16r, s16i);
    __syncwarp();
    tile_column_sums<W>(tw, lane, gr + sg * LONG_SEG, LONG_SEG);
    __syncwarp();
  }
  return v;
}

template <typename XT, int W, int NW>
__global__ void __launch_bounds__(NW * 32, 24 / NW) fe_grad_long_pgf_kernel(FeGroupArgs a) {
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
  float2* ck = reinterpret_cast<float2*>(smem + L.off_ck);
  float* tls = reinterpret_cast<float*>(smem + L.off_tile);

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
  float2* myck = ck + static_cast<size_t>(w) * L.nseg * 32;
  float* tw = tls + w * LONG_SEG * LTP;
  const int nseg = (k + LONG_SEG - 1) / LONG_SEG;
  const int n_last = k - LONG_SEG * (nseg - 1);
  float fe_part = 0.0f;

  // passes of W roots; from the table's first form-B root on (a multiple of
  // 32, so no pass straddles it) the passes use form B
  const int first_b = static_cast<int>(__ldg(tab + 1).x);
  for (int j0 = 0; j0 < nroots; j0 += W) {
    if (j0 < first_b)
      fe_part += pgf_pass<W, false>(tab, nroots, j0, rl, lane, el, gr, myck, tw, nseg, n_last);
    else
      fe_part += pgf_pass<W, true>(tab, nroots, j0, rl, lane, el, gr, myck, tw, nseg, n_last);
  }

  if (has_real) {
    // the real root: value c_mid prod l, gradient c_mid prod_{i' != i} l_i'.
    // The slot's lanes split the literals into W contiguous chunks; the
    // within-chunk suffixes go to this warp's (now free) checkpoint area.
    const float em = head.z;
    const int chunk = (k + W - 1) / W;
    const int i0 = min(k, rl * chunk), i1 = min(k, i0 + chunk);
    float* scr = reinterpret_cast<float*>(myck);
    float sl = 1.0f;
    for (int i = i1 - 1; i >= i0; --i) {
      scr[(i - i0) * 32 + lane] = sl;
      sl *= el[i];
    }
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
    float pl = em * pre * suf;
    for (int i = i0; i < i1; ++i) {
      gr[i] += pl * scr[(i - i0) * 32 + lane];
      pl *= el[i];
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
