// CUDA kernels of the hot path other than the short FE+gradient kernels:
// long-constraint FE+gradient, CSR gather + projected step, exact check,
// counter-based initialisation and small data-movement helpers.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <map>
#include <mutex>

#include "afsat.h"
#include "afsat_internal.h"
#include "bulk_copy.cuh"
#include "fe_short.cuh"
#include "step_units.cuh"

namespace afs {


// ---------------------------------------------------------------------------
// Long constraints (k > 32) in the paper's basis (the probability-generating
// basis has its own kernel, long_pgf.cu): one CTA per (constraint, RT
// restarts). Factors 1 + w^j l_i, written A - b (1 - l_i).
// Warp w owns restart w of the tile and its lanes own 32 roots at a time.
// The forward pass keeps one prefix checkpoint per LONG_SEG-literal segment
// in shared memory; the backward pass rebuilds a segment's prefixes (and its
// factors) in registers, multiplies them by the running suffix (which starts
// at the gradient weight D_j) and stores each lane's (root's) contributions
// as a row of a per-warp shared-memory tile, whose columns the lanes then
// sum, so lane t ends with literal t of the segment summed over the 32 roots.
// The factors reach 2 in modulus, so running products leave the FP32 range:
// they are renormalised at segment boundaries into a mantissa and an integer
// power of two (exponent field of the IEEE encoding) and the contributions
// are rescaled before the root sum. The literal list is staged with
// cp.async.bulk; the coefficient table is read through L1. Exponents are
// 16-bit (at most 1 bit of growth per literal).
// ---------------------------------------------------------------------------
constexpr int LONG_RT = 8;  // restarts (warps) per CTA; 4 for the longest groups (shared memory)

__device__ __forceinline__ void renorm(float& r, float& i, int& e) {
  const float m = fmaxf(fabsf(r), fabsf(i));
  const int ex = (__float_as_int(m) >> 23) & 0xff;
  if (ex == 0 || ex == 255) return;
  int sh = ex - 127;
  sh = sh > 126 ? 126 : (sh < -126 ? -126 : sh);
  const float sc = __int_as_float((127 - sh) << 23);
  r *= sc;
  i *= sc;
  e += sh;
}

constexpr int LONG_TP = 17;    // row pitch of the transpose tile (conflict-free columns)

// el[t] = u_t = 1 - l_t; the factor is A - b u, passed as (ar, ai) = A and
// (br, bi) = -b so that each component is one FMA. The prefixes of the
// segment are rebuilt from the checkpoint Q (with CF the factors are kept in
// registers for the backward walk, else rebuilt there), then walked
// backwards with the running suffix S; the contribution Re(prefix * S) of
// literal t is written to row `lane`, column t of the warp's tile (scaled by
// 2^escale).
template <bool FULL, bool ESP, bool CF>
__device__ __forceinline__ void long_segment(const float* el, int n, float ar, float ai, float br, float bi,
                                             float Qr, float Qi, float& Sr, float& Si, int escale, float* trow) {
  float pr[LONG_SEG], pi[LONG_SEG], fr[CF ? LONG_SEG : 1], fi[CF ? LONG_SEG : 1];
  pr[0] = Qr;
  pi[0] = Qi;
#pragma unroll
  for (int t = 0; t < LONG_SEG; ++t) {
    if (FULL || t < n) {
      const float ll = el[t];
      const float Fr = fmaf(br, ll, ar), Fi = fmaf(bi, ll, ai);
      if constexpr (CF) {
        fr[t] = Fr;
        fi[t] = Fi;
      }
      if (t + 1 < LONG_SEG) {
        pr[t + 1] = fmaf(pr[t], Fr, -pi[t] * Fi);
        pi[t + 1] = fmaf(pr[t], Fi, pi[t] * Fr);
      }
    }
  }
#pragma unroll
  for (int t = LONG_SEG - 1; t >= 0; --t) {
    float v = 0.0f;
    if (FULL || t < n) {
      v = fmaf(pr[t], Sr, -pi[t] * Si);
      float Fr, Fi;
      if constexpr (CF) {
        Fr = fr[t];
        Fi = fi[t];
      } else {
        const float ll = el[t];
        Fr = fmaf(br, ll, ar);
        Fi = fmaf(bi, ll, ai);
      }
      const float nr = fmaf(Sr, Fr, -Si * Fi);
      const float ni = fmaf(Sr, Fi, Si * Fr);
      Sr = nr;
      Si = ni;
    }
    trow[t] = ESP ? ldexpf(v, escale) : v;
  }
}

// 2^e as a float for -126 <= e <= 127.
__device__ __forceinline__ float exp2_int(int e) { return __int_as_float((e + 127) << 23); }

// Column sums of the warp's 32 x LONG_SEG tile: lane L adds rows
// 16*(L>>4) .. +15 of column L & 15, the two halves meet by one shuffle.
__device__ __forceinline__ float long_column_sum(const float* tile, int lane) {
  const int c = lane & (LONG_SEG - 1), h = lane >> 4;
  float s = 0.0f;
#pragma unroll
  for (int r = 0; r < 16; ++r) s += tile[(h * 16 + r) * LONG_TP + c];
  return s + __shfl_xor_sync(0xffffffffu, s, 16);
}

// Shared memory of one CTA (the coefficient table is read through L1: each
// lane loads its root's two granules once per 32-root pass).
struct LongLayout {
  int kpad, nseg_max, rt;
  __host__ __device__ LongLayout(int kmax, int rt_ = LONG_RT) : rt(rt_) {
    kpad = (kmax + 7) & ~7;
    nseg_max = (kmax + LONG_SEG - 1) / LONG_SEG;
  }
  __host__ __device__ size_t bytes(bool esp) const {
    (void)esp;
    size_t b = static_cast<size_t>(kpad) * 8;                 // literal list
    b += 2 * static_cast<size_t>(rt) * kpad * 4;              // literal values, gradient accumulators
    b += static_cast<size_t>(rt) * nseg_max * 32 * 8;         // prefix checkpoints
    b += static_cast<size_t>(rt) * nseg_max * 32 * 2;         // their power-of-two exponents (16 bits)
    b = (b + 15) & ~static_cast<size_t>(15);
    b += static_cast<size_t>(rt) * 32 * LONG_TP * 4;          // transpose tiles
    return b;
  }
};

template <typename XT, int RT>
__global__ void __launch_bounds__(RT * 32) fe_grad_long_kernel(FeGroupArgs a, int kmax) {
  // the groups that run 4 restarts per CTA (the longest) keep a segment's
  // factors in registers: fewer instructions, more registers per thread
  constexpr bool CF = RT == 4;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bar;
  pdl_wait();
  pdl_trigger();
  const LongLayout L(kmax, RT);
  const int tiles = (a.nb + RT - 1) / RT;
  const int cl = blockIdx.x / tiles;
  const int tile = blockIdx.x - cl * tiles;
  const int cb = a.c_begin + cl;
  const int k = __ldg(a.cons_k + cb);
  const int litoff = __ldg(a.cons_lit + cb);
  const int tab_off = __ldg(a.cons_tab + cb);
  const int nroots = k / 2 + (k & 1) + 1;

  const float4* tab = a.coef + tab_off;  // read through L1
  int2* lits = reinterpret_cast<int2*>(smem);
  float* ell = reinterpret_cast<float*>(lits + L.kpad);
  float* gs = ell + RT * L.kpad;
  float2* ck = reinterpret_cast<float2*>(gs + RT * L.kpad);
  short* cke = reinterpret_cast<short*>(ck + RT * L.nseg_max * 32);
  float* tps = reinterpret_cast<float*>(
      smem + ((reinterpret_cast<unsigned char*>(cke + RT * L.nseg_max * 32) - smem + 15) & ~static_cast<size_t>(15)));

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
  for (int i = tid; i < RT * L.kpad; i += blockDim.x) gs[i] = 0.0f;
  const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
  if (!mbar_wait_bounded(&bar, 0, limit)) {
    if (tid == 0) atomicExch(a.err, DEV_ERR_TIMEOUT);
    mbar_wait_bounded(&bar, 0, limit);  // let copies in flight land before exit
    return;
  }

  // stage u[r][i] = 1 - s_i x[v_i][b]: RT consecutive threads read one row segment
  const XT* x = static_cast<const XT*>(a.x);
  const int bt = tile * RT;
  for (int idx = tid; idx < k * RT; idx += blockDim.x) {
    const int i = idx / RT, r = idx % RT;
    const int2 li = lits[i];
    const int bl = bt + r;
    const float xv =
        bl < a.nb ? load_x<XT>(x + static_cast<long long>(li.x >> 1) * a.x_pitch + a.b0 + bl) : 0.0f;
    const float lv = (li.x & 1) ? -xv : xv;
    ell[r * L.kpad + i] = 1.0f - lv;
  }
  __syncthreads();

  const float* el = ell + w * L.kpad;
  float* gr = gs + w * L.kpad;
  float2* myck = ck + static_cast<size_t>(w) * L.nseg_max * 32;
  short* myce = cke + static_cast<size_t>(w) * L.nseg_max * 32;
  float* tpw = tps + static_cast<size_t>(w) * 32 * LONG_TP;  // this warp's transpose tile
  const int nseg = (k + LONG_SEG - 1) / LONG_SEG;
  float fe_part = 0.0f;

  for (int rg = 0; rg < nroots; rg += 32) {
    const int j = rg + lane;
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f, dr = 0.f, di = 0.f, er = 0.f, ei = 0.f;
    if (j < nroots) {  // factor A - b u: keep (A, -b)
      const float4 t0 = __ldg(tab + 1 + 2 * j), t1 = __ldg(tab + 2 + 2 * j);
      ar = t0.x; ai = t0.y; br = -t0.z; bi = -t0.w;
      dr = t1.x; di = t1.y; er = t1.z; ei = t1.w;
    }
    // forward: prefix checkpoints at segment starts
    float Pr = 1.0f, Pi = 0.0f;
    int Pe = 0;
    for (int seg = 0; seg < nseg; ++seg) {
      myck[seg * 32 + lane] = make_float2(Pr, Pi);
      myce[seg * 32 + lane] = static_cast<short>(Pe);
      const int i0 = seg * LONG_SEG;
      const int n = min(LONG_SEG, k - i0);
      // four literals per 16-byte broadcast read (segments start aligned)
      auto fstep = [&](float ll) {
        const float Fr = fmaf(br, ll, ar), Fi = fmaf(bi, ll, ai);
        const float nr = fmaf(Pr, Fr, -Pi * Fi);
        const float ni = fmaf(Pr, Fi, Pi * Fr);
        Pr = nr;
        Pi = ni;
      };
      int t = 0;
      for (; t + 4 <= n; t += 4) {
        const float4 v = *reinterpret_cast<const float4*>(el + i0 + t);
        fstep(v.x);
        fstep(v.y);
        fstep(v.z);
        fstep(v.w);
      }
      for (; t < n; ++t) fstep(el[i0 + t]);
      renorm(Pr, Pi, Pe);
    }
    const float val0 = fmaf(er, Pr, -ei * Pi);
    float val = ldexpf(val0, Pe);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    fe_part += val;

    // backward: suffix from the gradient weight, segment by segment
    float Sr = dr, Si = di;
    int Se = 0;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int i0 = seg * LONG_SEG;
      const int n = min(LONG_SEG, k - i0);
      const float2 Q = myck[seg * 32 + lane];
      const int escale = myce[seg * 32 + lane] + Se;
      float* trow = tpw + lane * LONG_TP;
      if (n == LONG_SEG)
        long_segment<true, true, CF>(el + i0, n, ar, ai, br, bi, Q.x, Q.y, Sr, Si, escale, trow);
      else
        long_segment<false, true, CF>(el + i0, n, ar, ai, br, bi, Q.x, Q.y, Sr, Si, escale, trow);
      renorm(Sr, Si, Se);
      __syncwarp();
      const float s = long_column_sum(tpw, lane);
      if (lane < n) gr[i0 + lane] += s;
      __syncwarp();  // the tile is read before the next segment's rows
    }
  }
  // value: fe_part holds the sum over all roots in every lane
  if (a.fe != nullptr && lane == 0 && bt + w < a.nb)
    a.fe[static_cast<long long>(__ldg(a.cons_orig + cb)) * a.fe_pitch + a.b0 + bt + w] = __ldg(tab).x + fe_part;
  __syncthreads();
  for (int idx = tid; idx < k * RT; idx += blockDim.x) {
    const int i = idx / RT, r = idx % RT;
    if (bt + r < a.nb) {
      const int2 li = lits[i];
      const float gv = gs[r * L.kpad + i];
      a.go[static_cast<long long>(li.y) * a.go_pitch + bt + r] = (li.x & 1) ? -gv : gv;
    }
  }
}

// Paper-basis long groups whose shared memory at 8 restarts per CTA exceeds
// LONG_RT4_BYTES run 4 restarts per CTA, so that more CTAs fit on an SM (and
// the longest constraints fit at all).
constexpr size_t LONG_RT4_BYTES = 64 * 1024;

template <typename XT>
static void launch_long_esp_t(const FeGroupArgs& a, cudaStream_t s) {
  const bool rt4 = LongLayout(a.k, 8).bytes(true) > LONG_RT4_BYTES;
  const int rt = rt4 ? 4 : 8;
  const size_t smem = LongLayout(a.k, rt).bytes(true);
  const int tiles = (a.nb + rt - 1) / rt;
  const long long blocks = static_cast<long long>(tiles) * a.c_count;
  if (rt4)
    launch_pdl(fe_grad_long_kernel<XT, 4>, dim3(static_cast<unsigned>(blocks)), dim3(128), smem, s, a, a.k);
  else
    launch_pdl(fe_grad_long_kernel<XT, 8>, dim3(static_cast<unsigned>(blocks)), dim3(256), smem, s, a, a.k);
}

template <typename K>
static bool raise_smem_cap(K kernel, int optin) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return false;
  const int cap = optin - static_cast<int>(fa.sharedSizeBytes);
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap) == cudaSuccess;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("AFS_PDL");
    return !(e != nullptr && e[0] == '0');
  }();
  return on;
}

// a.k carries the group's longest constraint for the long kernels; (wl, nw)
// is the probability-generating kernel's tile (lanes per restart, warps)
bool launch_fe_long(const FeGroupArgs& a, int xt, int basis, int wl, int nw, cudaStream_t s) {
  if (basis == 0) return launch_fe_long_pgf(a, xt, wl, nw, s);
  if (xt == XT_F32) launch_long_esp_t<float>(a, s);
  else launch_long_esp_t<__nv_bfloat16>(a, s);
  return true;
}

// ---------------------------------------------------------------------------
// CSR gather and projected step (Algorithm 1, step and projection):
// g[v][b] = sum over the slots of v (fixed order) of go[slot][b];
// x <- clamp(x - eta g, -1, 1), or g written out in evaluation mode.
// One lane per restart, one warp per (variable, 32 restarts).
// ---------------------------------------------------------------------------
// One lane per restart. Evaluation mode (grad != nullptr) writes the summed
// gradient; step mode moves the unsolved restarts and, with sgn, writes the
// sign word of the warp's 32 restarts (the chunk start is a multiple of 32).
template <typename XT>
__global__ void __launch_bounds__(256) csr_update_kernel(CsrArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int tiles = (a.nb + 31) >> 5;
  const long long vl = warp / tiles;
  if (vl >= a.v_count) return;  // uniform per warp
  const int tile = static_cast<int>(warp - vl * tiles);
  const int bl = tile * 32 + lane;
  const bool act = bl < a.nb;
  const int v = a.v_begin + static_cast<int>(vl);
  const int s0 = __ldg(a.csr_off + v), s1 = __ldg(a.csr_off + v + 1);
  float accf[1] = {0.0f};
  fused_sum<XT, 1, 4>(a, v, a.b0 + (act ? bl : 0), act, accf);
  // eight independent loads in flight per lane; the summation order is fixed
  // by the slot order, so the result does not depend on timing
  const float* col = a.go + (act ? bl : 0);
  float acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.f;
  int s = s0;
  for (; s + 7 < s1; s += 8) {
    float t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = __ldg(col + static_cast<long long>(s + u) * a.go_pitch);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += t[u];
  }
  {
    float t[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) t[u] = s + u < s1 ? __ldg(col + static_cast<long long>(s + u) * a.go_pitch) : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += t[u];
  }
  const float g = accf[0] + (((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7])));
  if (a.grad != nullptr) {
    if (act) a.grad[static_cast<long long>(v) * a.grad_pitch + a.b0 + bl] = g;
    return;
  }
  const int inst = __ldg(a.var_inst + v);
  const int word = (a.b0 + tile * 32) >> 5;
  const long long wi = static_cast<long long>(inst) * a.W + word;
  const unsigned viol = a.vcur != nullptr ? a.vcur[wi] : ~0u;
  const bool solved = !((viol >> lane) & 1u) ||
                      (a.fixv != nullptr && act &&
                       a.fixv[static_cast<long long>((a.b0 + bl) * static_cast<long long>(a.n_fix_groups) / a.B) *
                                  a.n_vars + v] != 0);
  if (lane == 0 && v == __ldg(a.var_inst + a.n_vars + inst)) csr_first_var_duty(a, inst, word, wi);
  const long long xi = static_cast<long long>(v) * a.x_pitch + a.b0 + bl;
  float xs = 0.0f;
  if (act) {
    xs = load_x<XT>(static_cast<const XT*>(a.x) + xi);
    if (!solved) xs = stored_value<XT>(fminf(fmaxf(fmaf(-a.eta, g, xs), -1.0f), 1.0f));
    store_x<XT>(static_cast<XT*>(a.x_out) + xi, xs);  // a solved restart keeps x_t
  }
  const unsigned bits = __ballot_sync(0xffffffffu, act && xs < 0.0f);
  if (a.sgn != nullptr && lane == 0) a.sgn[static_cast<long long>(v) * a.W + word] = bits;
}

template <typename XT, bool OFF32>
__global__ void __launch_bounds__(256, 4) csr_update_vec4_kernel(CsrArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const unsigned tiles = static_cast<unsigned>((a.nb + 127) >> 7);
  const unsigned ntask = tiles * static_cast<unsigned>(a.v_count);  // < 2^32 (checked at launch)
  const unsigned stride = gridDim.x * (blockDim.x >> 5);
  for (unsigned task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < ntask; task += stride) {
    const unsigned vl = task / tiles;  // uniform per warp
    csr_vec4_task<XT, OFF32>(a, static_cast<int>(vl), static_cast<int>(task - vl * tiles), lane);
  }
}

// The fused pass: warps stride over the (variable, 128-restart tile) tasks and
// store the summed derivatives of each variable's fused occurrences (4
// restarts per lane) into gf. The gathers are plain vector loads, FUSED_FB
// occurrences (2 rows each) in flight per warp. A staged variant (per-warp
// cp.async.bulk copies of the 512-byte row segments into shared memory,
// double-buffered on mbarriers) measured slower than these loads.
// (two occurrences in flight and 128-thread blocks measured best: more
// resident warps beat deeper per-warp batches for these L2 gathers)
template <typename XT>
constexpr int FUSED_FB = 2;
// launches of up to this many (variable, 128-restart) tasks, which leave each
// warp's occurrence list on the critical path, take the prefetching sums
constexpr long long FUSED_PF_MAX_TASKS = 4096;
constexpr int FUSED_THREADS = 128;
// the persistent grid takes 1/FUSED_GRID_DIV of the resident-block slots (0:
// one block per 4 tasks, no persistent grid, which measured best: the FE
// launches beside it then share the SMs block by block)
constexpr int FUSED_GRID_DIV = 0;

template <typename XT, bool OFF32, bool PF>
__global__ void __launch_bounds__(FUSED_THREADS) fused_grad_kernel(CsrArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const unsigned tiles = static_cast<unsigned>((a.nb + 127) >> 7);
  const unsigned ntask = tiles * static_cast<unsigned>(a.v_count);  // < 2^32 (checked at launch)
  const unsigned stride = gridDim.x * (blockDim.x >> 5);
  for (unsigned task = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); task < ntask; task += stride) {
    const unsigned vl = task / tiles;  // uniform per warp
    const int v = a.v_begin + static_cast<int>(vl);
    const int bl = static_cast<int>(task - vl * tiles) * 128 + lane * 4;
    const bool act = bl < a.nb;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    if constexpr (PF)
      fused_sum_pf<XT, FUSED_PF_BATCH, OFF32>(a, v, a.b0 + (act ? bl : 0), act, lane, acc);
    else
      fused_sum<XT, 4, FUSED_FB<XT>, OFF32>(a, v, a.b0 + (act ? bl : 0), act, acc);
    if (act)
      *reinterpret_cast<float4*>(a.gf + static_cast<long long>(v) * a.gf_pitch + bl) =
          make_float4(acc[0], acc[1], acc[2], acc[3]);
  }
}

// Resident blocks of a kernel on the whole device (cached per kernel).
template <typename K>
static long long resident_blocks(K kernel, int threads, size_t smem = 0) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, long long> cached;  // (kernel, threads) -> blocks
  std::lock_guard<std::mutex> lock(mu);
  const auto key = std::make_pair(reinterpret_cast<const void*>(kernel), threads);
  auto it = cached.find(key);
  if (it == cached.end()) {
    int dev = 0, sms = 1, per = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess || per < 1) per = 1;
    it = cached.emplace(key, static_cast<long long>(sms) * per).first;
  }
  return it->second;
}

template <typename XT, bool OFF32, bool PF>
static void launch_fused_t(const CsrArgs& a, long long blocks, cudaStream_t s) {
  auto kern = fused_grad_kernel<XT, OFF32, PF>;
  if (FUSED_GRID_DIV > 0)
    blocks = std::min(blocks, std::max(1LL, resident_blocks(kern, FUSED_THREADS) / FUSED_GRID_DIV));
  launch_pdl(kern, dim3(static_cast<unsigned>(blocks)), dim3(FUSED_THREADS), 0, s, a);
}

void launch_fused_grad(const CsrArgs& a, int xt, cudaStream_t s) {
  const long long tasks = static_cast<long long>((a.nb + 127) / 128) * a.v_count;
  if (tasks == 0) return;
  if (tasks >= (1ll << 32) - 4096LL * 1024) return;  // (never for instances that load)
  constexpr int W = FUSED_THREADS / 32;
  const long long blocks = (tasks + W - 1) / W;
  // row offsets v * x_pitch in 32 bits when the whole state fits
  const bool off32 = static_cast<unsigned long long>(a.n_vars) * static_cast<unsigned long long>(a.x_pitch) <
                     (1ull << 32);
  // few tasks: the latency of each variable's list dominates (prefetched
  // entries); many: the throughput of the plain batches
  const bool pf = tasks <= FUSED_PF_MAX_TASKS;
  if (xt == XT_F32) {
    if (off32)
      pf ? launch_fused_t<float, true, true>(a, blocks, s) : launch_fused_t<float, true, false>(a, blocks, s);
    else
      pf ? launch_fused_t<float, false, true>(a, blocks, s) : launch_fused_t<float, false, false>(a, blocks, s);
  } else {
    if (off32)
      pf ? launch_fused_t<__nv_bfloat16, true, true>(a, blocks, s)
         : launch_fused_t<__nv_bfloat16, true, false>(a, blocks, s);
    else
      pf ? launch_fused_t<__nv_bfloat16, false, true>(a, blocks, s)
         : launch_fused_t<__nv_bfloat16, false, false>(a, blocks, s);
  }
}

void launch_csr_update(const CsrArgs& a, int xt, cudaStream_t s) {
  const bool vec = a.grad == nullptr && (a.go_pitch % 32) == 0 && (a.x_pitch % 32) == 0 && (a.b0 % 32) == 0 &&
                   (reinterpret_cast<uintptr_t>(a.go) % 16) == 0;
  const long long tasks128 = static_cast<long long>((a.nb + 127) / 128) * a.v_count;
  if (vec && tasks128 < (1ll << 32) - 4096LL * 1024) {
    const long long tiles = (a.nb + 127) / 128;
    long long blocks = (tiles * a.v_count + 7) / 8;
    if (blocks == 0) return;
    // state offsets v * x_pitch + b and row offsets slot * go_pitch in 32 bits
    // when both buffers are that small
    const bool off32 =
        static_cast<unsigned long long>(a.n_vars) * static_cast<unsigned long long>(a.x_pitch) < (1ull << 32) &&
        static_cast<unsigned long long>(a.go_rows) * static_cast<unsigned long long>(a.go_pitch) < (1ull << 32);
    auto go = [&](auto kern) {
      blocks = std::min(blocks, resident_blocks(kern, 256));
      launch_pdl(kern, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
    };
    if (xt == XT_F32) {
      if (off32)
        go(csr_update_vec4_kernel<float, true>);
      else
        go(csr_update_vec4_kernel<float, false>);
    } else {
      if (off32)
        go(csr_update_vec4_kernel<__nv_bfloat16, true>);
      else
        go(csr_update_vec4_kernel<__nv_bfloat16, false>);
    }
    return;
  }
  const long long tiles = (a.nb + 31) / 32;
  const long long nwarps = tiles * a.v_count;
  const long long blocks = (nwarps + 7) / 8;
  if (blocks == 0) return;
  if (xt == XT_F32) launch_pdl(csr_update_kernel<float>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
  else launch_pdl(csr_update_kernel<__nv_bfloat16>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
}

// Sign words of a state written outside the step (initialisation, set_x):
// one warp per (variable, word).
template <typename XT>
__global__ void apply_fixed_kernel(XT* x, long long pitch, int n, int B, const signed char* fixv, int groups) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n) * B) return;
  const int v = static_cast<int>(i / B), b = static_cast<int>(i - static_cast<long long>(v) * B);
  const signed char f = fixv[static_cast<long long>(b) * groups / B * n + v];
  if (f != 0) store_x<XT>(x + static_cast<long long>(v) * pitch + b, f > 0 ? -1.0f : 1.0f);
}

void launch_apply_fixed(void* x, int xt, long long x_pitch, int n, int B, const signed char* fixv, int groups,
                        cudaStream_t s) {
  const long long total = static_cast<long long>(n) * B;
  if (total == 0 || fixv == nullptr || groups <= 0) return;
  const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
  if (xt == XT_F32)
    apply_fixed_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float*>(x), x_pitch, n, B, fixv, groups);
  else
    apply_fixed_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(static_cast<__nv_bfloat16*>(x), x_pitch, n, B, fixv,
                                                            groups);
}

template <typename XT>
__global__ void pack_signs_kernel(const XT* x, long long pitch, int n, int B, unsigned* sgn, int W, int wc) {
  const int lane = threadIdx.x & 31;
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (warp >= static_cast<long long>(n) * wc) return;  // uniform per warp
  const int v = static_cast<int>(warp / wc);
  const int w = static_cast<int>(warp - static_cast<long long>(v) * wc);
  const int b = w * 32 + lane;
  const bool neg = b < B && load_x<XT>(x + static_cast<long long>(v) * pitch + b) < 0.0f;
  const unsigned bits = __ballot_sync(0xffffffffu, neg);
  if (lane == 0) sgn[static_cast<long long>(v) * W + w] = bits;
}

// The first wc words of every row of sgn (row pitch W) from the B restarts
// of x (row pitch x_pitch): x and sgn may point into a column range.
void launch_pack_signs_words(const void* x, int xt, long long x_pitch, int n, int B, unsigned* sgn, int W, int wc,
                             cudaStream_t s) {
  const long long warps = static_cast<long long>(n) * wc;
  if (warps == 0) return;
  const unsigned blocks = static_cast<unsigned>((warps + 7) / 8);
  if (xt == XT_F32)
    pack_signs_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(x), x_pitch, n, B, sgn, W, wc);
  else
    pack_signs_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x), x_pitch, n, B, sgn,
                                                            W, wc);
}

void launch_pack_signs(const void* x, int xt, long long x_pitch, int n, int B, unsigned* sgn, int W,
                       cudaStream_t s) {
  launch_pack_signs_words(x, xt, x_pitch, n, B, sgn, W, W, s);
}

// ---------------------------------------------------------------------------
// Bit-sliced exact check (Algorithm 1's is_sat on the sign-rounded state).
// A thread holds 32 restarts in one word per literal: literal i is true in
// the restarts of S_{v_i} xor (negated ? ~0 : 0), where S_v is the sign word
// of its variable. The true count t of each restart is kept as bit planes
// P_0..P_{np-1} (bit j of P_p is bit p of restart j's count); adding a
// literal word is a ripple of AND/XOR through the planes. For k <= 62 the
// violated set {t : f(t) = +1} (or its complement, when that is smaller) is
// enumerated from a 64-bit mask and each value u becomes an equality word
// AND_p (u_p ? P_p : ~P_p); longer constraints unpack t per restart and read
// the violation table.
// ---------------------------------------------------------------------------
// A warp handles one range (<= 32 literals, or one longer constraint) for 32
// words: lane j owns word w0 + 32*blockIdx.y + j. The range's literal words
// are staged in shared memory, then the constraints are counted from there.
// COUNT = false: the violation words of the range are ORed, and the warps of
// a block merge them per instance before the atomic OR into vword. COUNT =
// true (the exact unsat count of the final state): the violation words are
// added into 5 bit planes (a range has < 32 constraints), and the block adds
// the per-restart counts of its warps per instance into unsat.
template <bool COUNT>
__global__ void __launch_bounds__(CHECK_WARPS * 32) check_bits_kernel(CheckArgs a) {
  __shared__ unsigned stage[CHECK_WARPS][CHECK_STAGE][32];
  __shared__ unsigned bad_s[CHECK_WARPS][COUNT ? 5 : 1][32];
  __shared__ int inst_s[CHECK_WARPS];
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int rgi = blockIdx.x * CHECK_WARPS + wp;
  const int wl = blockIdx.y * 32 + lane;
  const bool act = wl < a.wc;
  const int w = a.w0 + (act ? wl : 0);
  unsigned bad = 0u;
  unsigned C[5] = {0u, 0u, 0u, 0u, 0u};  // COUNT: violated constraints per restart, bit planes
  int inst = -1;
  if (rgi < a.n_ranges) {  // uniform per warp
    const int4 rg = __ldg(a.ranges + rgi);
    inst = rg.z;
    const int nc = rg.y - rg.x;
    // constraint offsets and test masks of the range, one per lane (nc < 32)
    const int offv = __ldg(a.lit_off + rg.x + min(lane, nc));
    const unsigned long long emv = lane < nc ? __ldg(a.em + rg.x + lane) : 0ull;
    const int l0 = __shfl_sync(0xffffffffu, offv, 0);
    const int l1 = __shfl_sync(0xffffffffu, offv, nc);
    const unsigned* sg = a.sgn + w;
    unsigned* st = &stage[wp][0][lane];
    unsigned P[CHECK_PLANES];
    if (l1 - l0 <= CHECK_STAGE) {
      check_stage(a, sg, st, l0, l1 - l0, lane);
      for (int c = 0; c < nc; ++c) {
        const int a0 = __shfl_sync(0xffffffffu, offv, c) - l0;
        const int a1 = __shfl_sync(0xffffffffu, offv, c + 1) - l0;
        const unsigned long long em = __shfl_sync(0xffffffffu, emv, c);
        const int k = a1 - a0;
        const int np = 32 - __clz(k);
#pragma unroll
        for (int p = 0; p < CHECK_PLANES; ++p) P[p] = 0u;
        add_words<6>(P, st + a0 * 32, k, np);  // k <= 32 here
        const unsigned vb = violated_word(P, k, np, em, nullptr);
        if constexpr (COUNT) {
          unsigned carry = vb;
#pragma unroll
          for (int p = 0; p < 5; ++p) {
            const unsigned t = C[p] & carry;
            C[p] ^= carry;
            carry = t;
          }
        } else {
          bad |= vb;
        }
      }
    } else {  // one long constraint, staged 32 literals at a time
      const int k = l1 - l0;
      const int np = 32 - __clz(k);
#pragma unroll
      for (int p = 0; p < CHECK_PLANES; ++p) P[p] = 0u;
      for (int b = 0; b < k; b += CHECK_STAGE) {
        const int cnt = min(CHECK_STAGE, k - b);
        check_stage(a, sg, st, l0 + b, cnt, lane);
        add_words<CHECK_PLANES>(P, st, cnt, np);
        __syncwarp();
      }
      bad = violated_word(P, k, np, __shfl_sync(0xffffffffu, emv, 0), a.viol + __ldg(a.viol_off + rg.x));
      C[0] = bad;
    }
  }
  if constexpr (COUNT) {
#pragma unroll
    for (int p = 0; p < 5; ++p) bad_s[wp][p][lane] = act ? C[p] : 0u;
  } else {
    bad_s[wp][0][lane] = act ? bad : 0u;
  }
  if (lane == 0) inst_s[wp] = inst;
  __syncthreads();
  if constexpr (COUNT) {
    // thread t: word lane t & 31, restarts j = t >> 5, + CHECK_WARPS, ...
    const int wl2 = threadIdx.x & 31;
    const int ww = a.w0 + blockIdx.y * 32 + wl2;
    if (blockIdx.y * 32 + wl2 >= a.wc) return;
    for (int j = threadIdx.x >> 5; j < 32; j += CHECK_WARPS) {
      const int b = ww * 32 + j;
      if (b >= a.B) break;
      int cnt = 0, cur = -1;
      for (int q = 0; q < CHECK_WARPS; ++q) {
        const int iq = inst_s[q];
        if (iq < 0) continue;
        if (iq != cur) {
          if (cur >= 0 && cnt) atomicAdd(a.unsat + static_cast<long long>(cur) * a.B + b, cnt);
          cur = iq;
          cnt = 0;
        }
#pragma unroll
        for (int p = 0; p < 5; ++p) cnt += static_cast<int>((bad_s[q][p][wl2] >> j) & 1u) << p;
      }
      if (cur >= 0 && cnt) atomicAdd(a.unsat + static_cast<long long>(cur) * a.B + b, cnt);
    }
    return;
  }
  if (wp == 0 && act) {
    unsigned acc = 0u;
    int cur = -1;
    for (int j = 0; j < CHECK_WARPS; ++j) {
      const int ij = inst_s[j];
      if (ij < 0) continue;
      if (ij != cur) {
        if (cur >= 0 && acc) atomicOr(a.vword + static_cast<long long>(cur) * a.W + w, acc);
        cur = ij;
        acc = 0u;
      }
      acc |= bad_s[j][0][lane];
    }
    if (cur >= 0 && acc) atomicOr(a.vword + static_cast<long long>(cur) * a.W + w, acc);
  }
}

// One warp per (wide run, word): blockIdx.y is the word.
template <bool COUNT>
__global__ void __launch_bounds__(CHECK_WARPS * 32) check_wide_kernel(CheckArgs a) {
  __shared__ unsigned stage[CHECK_WARPS][CHECK_WIDE_STAGE];
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int rgi = blockIdx.x * CHECK_WARPS + wp;
  if (rgi < a.n_ranges)
    check_wide_unit<false, COUNT>(a, rgi, a.w0 + static_cast<int>(blockIdx.y), lane, stage[wp]);
}

void launch_check_wide(const CheckArgs& a, cudaStream_t s) {
  if (a.n_ranges == 0 || a.wc == 0) return;
  const dim3 grid(static_cast<unsigned>((a.n_ranges + CHECK_WARPS - 1) / CHECK_WARPS), static_cast<unsigned>(a.wc));
  if (a.unsat != nullptr) launch_pdl(check_wide_kernel<true>, grid, dim3(CHECK_WARPS * 32), 0, s, a);
  else launch_pdl(check_wide_kernel<false>, grid, dim3(CHECK_WARPS * 32), 0, s, a);
}

void launch_check_bits(const CheckArgs& a, cudaStream_t s) {
  if (a.n_ranges == 0 || a.wc == 0) return;
  const dim3 grid(static_cast<unsigned>((a.n_ranges + CHECK_WARPS - 1) / CHECK_WARPS),
                  static_cast<unsigned>((a.wc + 31) / 32));
  if (a.unsat != nullptr) launch_pdl(check_bits_kernel<true>, grid, dim3(CHECK_WARPS * 32), 0, s, a);
  else launch_pdl(check_bits_kernel<false>, grid, dim3(CHECK_WARPS * 32), 0, s, a);
}


__global__ void solved_words_kernel(const unsigned* vword, int n_inst, int W, int B, unsigned* out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n_inst) * W) return;
  const int w = static_cast<int>(i % W);
  const int valid = min(32, B - w * 32);
  out[i] = ~vword[i] & (valid >= 32 ? ~0u : (valid <= 0 ? 0u : ((1u << valid) - 1u)));
}

void launch_solved_words(const unsigned* vword, int n_inst, int W, int B, unsigned* out, cudaStream_t s) {
  const long long n = static_cast<long long>(n_inst) * W;
  if (n == 0) return;
  solved_words_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(vword, n_inst, W, B, out);
}

// ---------------------------------------------------------------------------
// Line search (Armijo backtracking per restart)
// ---------------------------------------------------------------------------
// Thread per restart column of a chunk of 64 constraint rows; the sum runs
// over the rows of one instance at a time and is added with an atomic.
__global__ void objective_kernel(const float* fe, long long pitch, int m, const int* cinst, int B, float* out) {
  const int b = blockIdx.y * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const int r0 = blockIdx.x * 64, r1 = min(m, r0 + 64);
  float acc = 0.0f;
  int cur = __ldg(cinst + r0);
  for (int r = r0; r < r1; ++r) {
    const int ir = __ldg(cinst + r);
    if (ir != cur) {
      atomicAdd(out + static_cast<long long>(cur) * B + b, acc);
      acc = 0.0f;
      cur = ir;
    }
    acc += fe[static_cast<long long>(r) * pitch + b];
  }
  atomicAdd(out + static_cast<long long>(cur) * B + b, acc);
}

void launch_objective(const float* fe, long long pitch, int m, const int* cinst, int B, float* out, cudaStream_t s) {
  if (m <= 0 || B <= 0) return;
  const dim3 grid(static_cast<unsigned>((m + 63) / 64), static_cast<unsigned>((B + 127) / 128));
  objective_kernel<<<grid, 128, 0, s>>>(fe, pitch, m, cinst, B, out);
}

template <typename XT>
__global__ void ls_candidate_kernel(LsCandArgs a) {
  const int b = blockIdx.y * blockDim.x + threadIdx.x;
  if (b >= a.B) return;
  const int v0 = blockIdx.x * 64, v1 = min(a.n, v0 + 64);
  const XT* x = static_cast<const XT*>(a.x);
  XT* xc = static_cast<XT*>(a.xc);
  int cur = __ldg(a.var_inst + v0);
  float acc = 0.0f;
  for (int v = v0; v < v1; ++v) {
    const int iv = __ldg(a.var_inst + v);
    if (iv != cur) {
      if (!a.done[static_cast<long long>(cur) * a.B + b]) atomicAdd(a.dec + static_cast<long long>(cur) * a.B + b, acc);
      acc = 0.0f;
      cur = iv;
    }
    if (a.done[static_cast<long long>(iv) * a.B + b]) continue;
    const long long i = static_cast<long long>(v) * a.pitch + b;
    const float xv = load_x<XT>(x + i), gv = a.g[i];
    const bool fixed = a.fixv != nullptr &&
                       a.fixv[static_cast<long long>(b) * a.n_fix_groups / a.B * a.n + v] != 0;
    const float xn = fixed ? xv : stored_value<XT>(fminf(fmaxf(fmaf(-a.eta, gv, xv), -1.0f), 1.0f));
    store_x<XT>(xc + i, xn);
    acc = fmaf(gv, xn - xv, acc);
  }
  if (!a.done[static_cast<long long>(cur) * a.B + b]) atomicAdd(a.dec + static_cast<long long>(cur) * a.B + b, acc);
}

void launch_ls_candidate(const LsCandArgs& a, cudaStream_t s) {
  if (a.n <= 0 || a.B <= 0) return;
  const dim3 grid(static_cast<unsigned>((a.n + 63) / 64), static_cast<unsigned>((a.B + 127) / 128));
  if (a.xt == XT_F32) ls_candidate_kernel<float><<<grid, 128, 0, s>>>(a);
  else ls_candidate_kernel<__nv_bfloat16><<<grid, 128, 0, s>>>(a);
}

__global__ void ls_accept_kernel(const float* f_trial, const float* f0, const float* dec, float c, int trial,
                                 int* done, int* chosen, long long count) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= count || done[i]) return;
  if (f_trial[i] <= fmaf(c, dec[i], f0[i])) {
    done[i] = 1;
    chosen[i] = trial;
  }
}

void launch_ls_accept(const float* f_trial, const float* f0, const float* dec, float c, int trial, int* done,
                      int* chosen, long long count, cudaStream_t s) {
  if (count <= 0) return;
  ls_accept_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(f_trial, f0, dec, c, trial, done, chosen,
                                                                            count);
}

__global__ void fill_int_kernel(int* p, int v, long long n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

void launch_fill_int(int* p, int v, long long n, cudaStream_t s) {
  if (n <= 0) return;
  fill_int_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(p, v, n);
}

// A restart with no violated constraint is solved: record the lowest such
// restart per instance.
__global__ void solved_kernel(const int* unsat, int n_inst, int B, int* solved) {
  pdl_wait();
  pdl_trigger();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n_inst) * B) return;
  const int inst = static_cast<int>(i / B), b = static_cast<int>(i - static_cast<long long>(inst) * B);
  if (unsat[i] == 0) atomicMin(solved + inst, b);
}

void launch_solved(const int* unsat, int n_inst, int B, int* solved, cudaStream_t s) {
  const long long n = static_cast<long long>(n_inst) * B;
  if (n == 0) return;
  launch_pdl(solved_kernel, dim3(static_cast<unsigned>((n + 255) / 256)), dim3(256), 0, s, unsat, n_inst, B, solved);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the round constants, the high halves xor-ed into
// the other words with the key, and a Weyl increment of the key per round.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    if (r < 9) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
  }
  return c;
}

__device__ __forceinline__ float philox_to_unit(unsigned w) {
  return fmaf(2.0f, static_cast<float>(w >> 8) * 0x1p-24f, -1.0f);
}

// x[v][b], b in [0, B): counter (b/4, local variable, instance, 0), key = seed
template <typename XT>
__global__ void init_philox_kernel(XT* x, long long pitch, int n, int B, const int* var_inst,
                                   const int* inst_vbegin, unsigned long long seed) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  const int Q = (B + 3) >> 2;
  if (i >= static_cast<long long>(n) * Q) return;
  const int v = static_cast<int>(i / Q);
  const int q = static_cast<int>(i - static_cast<long long>(v) * Q);
  const int inst = var_inst[v];
  const int vl = v - inst_vbegin[inst];
  const uint4 o = philox4x32_10(make_uint4(static_cast<unsigned>(q), static_cast<unsigned>(vl),
                                           static_cast<unsigned>(inst), 0u),
                                make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32)));
  const unsigned w[4] = {o.x, o.y, o.z, o.w};
  XT* row = x + static_cast<long long>(v) * pitch;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int b = 4 * q + t;
    if (b < B) store_x<XT>(row + b, philox_to_unit(w[t]));
  }
}

void launch_init_philox(void* x, int xt, long long x_pitch, int n, int B, const int* var_inst,
                        unsigned long long seed, cudaStream_t s) {
  // var_inst holds n entries followed by the instance first-variable table
  const int* inst_vbegin = var_inst + n;
  const long long total = static_cast<long long>(n) * ((B + 3) / 4);
  if (total == 0) return;
  const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
  if (xt == XT_F32)
    init_philox_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float*>(x), x_pitch, n, B, var_inst,
                                                     inst_vbegin, seed);
  else
    init_philox_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(static_cast<__nv_bfloat16*>(x), x_pitch, n, B,
                                                             var_inst, inst_vbegin, seed);
}

// ---------------------------------------------------------------------------
// Layout / type conversion of a restart-major array and column gathers.
// ---------------------------------------------------------------------------
template <typename S, typename D>
__global__ void convert_kernel(const S* src, long long sp, D* dst, long long dp, int n, int B) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n) * B) return;
  const int v = static_cast<int>(i / B), b = static_cast<int>(i - static_cast<long long>(v) * B);
  store_x<D>(dst + static_cast<long long>(v) * dp + b, load_x_rw<S>(src + static_cast<long long>(v) * sp + b));
}

void launch_convert_in(const void* src, int sxt, long long sp, void* dst, int dxt, long long dp, int n, int B,
                       cudaStream_t s) {
  const long long total = static_cast<long long>(n) * B;
  if (total == 0) return;
  const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
  using bf = __nv_bfloat16;
  if (sxt == XT_F32 && dxt == XT_F32)
    convert_kernel<float, float><<<blocks, 256, 0, s>>>(static_cast<const float*>(src), sp, static_cast<float*>(dst), dp, n, B);
  else if (sxt == XT_F32 && dxt == XT_BF16)
    convert_kernel<float, bf><<<blocks, 256, 0, s>>>(static_cast<const float*>(src), sp, static_cast<bf*>(dst), dp, n, B);
  else if (sxt == XT_BF16 && dxt == XT_F32)
    convert_kernel<bf, float><<<blocks, 256, 0, s>>>(static_cast<const bf*>(src), sp, static_cast<float*>(dst), dp, n, B);
  else
    convert_kernel<bf, bf><<<blocks, 256, 0, s>>>(static_cast<const bf*>(src), sp, static_cast<bf*>(dst), dp, n, B);
}

template <typename XT>
__global__ void gather_column_kernel(const XT* x, long long pitch, const int* var_inst, int n, const int* col_of,
                                     signed char* out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int col = col_of[var_inst[v]];
  const float xv = load_x_rw<XT>(x + static_cast<long long>(v) * pitch + col);
  out[v] = xv < 0.0f ? -1 : 1;
}

void launch_gather_column(const void* x, int xt, long long x_pitch, const int* var_inst, int n, const int* col_of,
                          signed char* out, cudaStream_t s) {
  if (n == 0) return;
  const unsigned blocks = static_cast<unsigned>((n + 255) / 256);
  if (xt == XT_F32)
    gather_column_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(x), x_pitch, var_inst, n, col_of, out);
  else
    gather_column_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(static_cast<const __nv_bfloat16*>(x), x_pitch, var_inst,
                                                               n, col_of, out);
}

bool prepare_kernels() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  if (LongLayout(AFS_MAX_LEN, 4).bytes(true) + 64 > static_cast<size_t>(optin)) return false;
  bool ok = prepare_long_pgf(optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<float, 8>, optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<float, 4>, optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<__nv_bfloat16, 8>, optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<__nv_bfloat16, 4>, optin);
  return ok;
}

}  // namespace afs
