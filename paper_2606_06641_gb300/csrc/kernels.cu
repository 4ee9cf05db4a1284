// CUDA kernels of the hot path other than the short FE+gradient kernels:
// long-constraint FE+gradient, CSR gather + projected step, exact check,
// counter-based initialisation and small data-movement helpers.
#include <cuda_bf16.h>

#include <cstdint>
#include <cstdlib>

#include "afsat_internal.h"
#include "fe_short.cuh"

namespace afs {

// ---------------------------------------------------------------------------
// Asynchronous bulk copies (global -> shared) completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the barrier for at most ~`limit` SM cycles.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) return false;
  }
  return true;
}

constexpr int DEV_ERR_TIMEOUT = 1;
constexpr long long WAIT_LIMIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz

// ---------------------------------------------------------------------------
// Long constraints (k > 32): one CTA per (constraint, 8 restarts).
//
// Same expansion as the short kernel, in the direct factor form
// a_j + b_j l_i (|a_j + b_j l| <= 1 for the probability-generating basis).
// Warp w owns restart w of the tile and its lanes own 32 roots at a time.
// The forward pass keeps one prefix checkpoint per 32-literal segment in
// shared memory; the backward pass rebuilds a segment's prefixes in registers,
// multiplies them by the running suffix (which starts at the gradient weight
// D_j), and a 31-shuffle reduce-scatter sums the 32 roots so lane t ends with
// literal t of the segment. With the paper's basis (ESP) the factors grow up
// to 2 in modulus, so running products are renormalised at segment boundaries
// into a mantissa and an integer power of two (exponent field of the IEEE
// encoding) and the contributions are rescaled before the root sum.
// The coefficient table and literal list are staged with cp.async.bulk.
// ---------------------------------------------------------------------------
constexpr int LONG_RT = 8;

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

__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int t = 0; t < o; ++t) {
      const float send = up ? v[t] : v[t + o];
      const float keep = up ? v[t + o] : v[t];
      v[t] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// el[t] = u_t = 1 - l_t; the factor is A - b u, passed as (ar, ai) = A and
// (br, bi) = -b so that each component is one FMA.
template <bool FULL>
__device__ __forceinline__ void long_segment(const float* el, int n, float ar, float ai, float br, float bi,
                                             float Qr, float Qi, float& Sr, float& Si, float (&v)[32]) {
  float pr[32], pi[32];
  pr[0] = Qr;
  pi[0] = Qi;
#pragma unroll
  for (int t = 0; t < 31; ++t) {
    if (FULL || t + 1 < n) {
      const float ll = el[t];
      const float Fr = fmaf(br, ll, ar), Fi = fmaf(bi, ll, ai);
      pr[t + 1] = fmaf(pr[t], Fr, -pi[t] * Fi);
      pi[t + 1] = fmaf(pr[t], Fi, pi[t] * Fr);
    }
  }
#pragma unroll
  for (int t = 31; t >= 0; --t) {
    if (FULL || t < n) {
      v[t] = fmaf(pr[t], Sr, -pi[t] * Si);
      const float ll = el[t];
      const float Fr = fmaf(br, ll, ar), Fi = fmaf(bi, ll, ai);
      const float nr = fmaf(Sr, Fr, -Si * Fi);
      const float ni = fmaf(Sr, Fi, Si * Fr);
      Sr = nr;
      Si = ni;
    } else {
      v[t] = 0.0f;
    }
  }
}

struct LongLayout {
  int kpad, tab_cap, nseg_max;
  __host__ __device__ LongLayout(int kmax) {
    kpad = (kmax + 3) & ~3;
    tab_cap = 1 + 2 * (kmax / 2 + 2);
    nseg_max = (kmax + 31) / 32;
  }
  __host__ __device__ size_t bytes(bool esp) const {
    size_t b = static_cast<size_t>(tab_cap) * 16;            // coefficient table
    b += static_cast<size_t>(kpad) * 8;                       // literal list
    b += 2 * static_cast<size_t>(LONG_RT) * kpad * 4;         // literal values, gradient accumulators
    b += static_cast<size_t>(LONG_RT) * nseg_max * 32 * 8;    // prefix checkpoints
    if (esp) b += static_cast<size_t>(LONG_RT) * nseg_max * 32 * 4;
    b += static_cast<size_t>(LONG_RT) * kpad;                 // literal truth bytes
    return b;
  }
};

template <typename XT, bool ESP>
__global__ void __launch_bounds__(256) fe_grad_long_kernel(FeGroupArgs a, int kmax) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long bar;
  pdl_wait();
  pdl_trigger();
  const LongLayout L(kmax);
  const int tiles = (a.nb + LONG_RT - 1) / LONG_RT;
  const int cl = blockIdx.x / tiles;
  const int tile = blockIdx.x - cl * tiles;
  const int cb = a.c_begin + cl;
  const int k = __ldg(a.cons_k + cb);
  const int litoff = __ldg(a.cons_lit + cb);
  const int tab_off = __ldg(a.cons_tab + cb);
  const int nroots = k / 2 + (k & 1) + (ESP ? 1 : 0);

  float4* tab = reinterpret_cast<float4*>(smem);
  int2* lits = reinterpret_cast<int2*>(tab + L.tab_cap);
  float* ell = reinterpret_cast<float*>(lits + L.kpad);
  float* gs = ell + LONG_RT * L.kpad;
  float2* ck = reinterpret_cast<float2*>(gs + LONG_RT * L.kpad);
  int* cke = reinterpret_cast<int*>(ck + LONG_RT * L.nseg_max * 32);
  unsigned char* tru = reinterpret_cast<unsigned char*>(cke + (ESP ? LONG_RT * L.nseg_max * 32 : 0));

  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned tab_bytes = static_cast<unsigned>(1 + 2 * nroots) * 16u;
  const unsigned lit_bytes = static_cast<unsigned>((k + 1) & ~1) * 8u;
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(&bar, tab_bytes + lit_bytes + a.extra_tx);
    bulk_g2s(tab, a.coef + tab_off, tab_bytes, &bar);
    bulk_g2s(lits, a.litslot + litoff, lit_bytes, &bar);
  }
  for (int i = tid; i < LONG_RT * L.kpad; i += blockDim.x) gs[i] = 0.0f;
  const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
  if (!mbar_wait_bounded(&bar, 0, limit)) {
    if (tid == 0) atomicExch(a.err, DEV_ERR_TIMEOUT);
    mbar_wait_bounded(&bar, 0, limit);  // let copies in flight land before exit
    return;
  }

  // stage u[r][i] = 1 - s_i x[v_i][b] and the literal's truth at the rounded
  // point: 8 consecutive threads read one 32-byte row
  const XT* x = static_cast<const XT*>(a.x);
  const int bt = tile * LONG_RT;
  for (int idx = tid; idx < k * LONG_RT; idx += blockDim.x) {
    const int i = idx >> 3, r = idx & 7;
    const int2 li = lits[i];
    const int bl = bt + r;
    const float xv =
        bl < a.nb ? load_x<XT>(x + static_cast<long long>(li.x >> 1) * a.x_pitch + a.b0 + bl) : 0.0f;
    const float l = (li.x & 1) ? -xv : xv;
    ell[r * L.kpad + i] = 1.0f - l;
    tru[r * L.kpad + i] = static_cast<unsigned char>(lit_true(l, li.x & 1));
  }
  __syncthreads();

  const float* el = ell + w * L.kpad;
  float* gr = gs + w * L.kpad;
  float2* myck = ck + static_cast<size_t>(w) * L.nseg_max * 32;
  int* myce = cke + static_cast<size_t>(w) * L.nseg_max * 32;
  const int nseg = (k + 31) >> 5;
  float fe_part = 0.0f;

  // exact check of the state read (Algorithm 1's unsat count): warp w, restart bt + w
  if (a.vflag != nullptr) {
    int t = 0;
    const unsigned char* tr = tru + w * L.kpad;
    for (int i = lane; i < k; i += 32) t += tr[i];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0 && bt + w < a.nb && __ldg(a.viol + __ldg(a.cons_voff + cb) + t))
      a.vflag[static_cast<long long>(blockIdx.x % VFLAG_SLOTS) * a.vflag_stride +
              static_cast<long long>(__ldg(a.cons_inst + cb)) * a.B + a.b0 + bt + w] = 1;
  }

  for (int rg = 0; rg < nroots; rg += 32) {
    const int j = rg + lane;
    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f, dr = 0.f, di = 0.f, er = 0.f, ei = 0.f;
    if (j < nroots) {  // factor A - b u: keep (A, -b)
      const float4 t0 = tab[1 + 2 * j], t1 = tab[2 + 2 * j];
      ar = t0.x; ai = t0.y; br = -t0.z; bi = -t0.w;
      dr = t1.x; di = t1.y; er = t1.z; ei = t1.w;
    }
    // forward: prefix checkpoints at segment starts
    float Pr = 1.0f, Pi = 0.0f;
    int Pe = 0;
    for (int seg = 0; seg < nseg; ++seg) {
      myck[seg * 32 + lane] = make_float2(Pr, Pi);
      if (ESP) myce[seg * 32 + lane] = Pe;
      const int i0 = seg * 32;
      const int n = min(32, k - i0);
#pragma unroll 4
      for (int t = 0; t < n; ++t) {
        const float ll = el[i0 + t];
        const float Fr = fmaf(br, ll, ar), Fi = fmaf(bi, ll, ai);
        const float nr = fmaf(Pr, Fr, -Pi * Fi);
        const float ni = fmaf(Pr, Fi, Pi * Fr);
        Pr = nr;
        Pi = ni;
      }
      if (ESP) renorm(Pr, Pi, Pe);
    }
    float val = fmaf(er, Pr, -ei * Pi);
    if (ESP) val = ldexpf(val, Pe);
    fe_part += val;

    // backward: suffix from the gradient weight, segment by segment
    float Sr = dr, Si = di;
    int Se = 0;
    for (int seg = nseg - 1; seg >= 0; --seg) {
      const int i0 = seg * 32;
      const int n = min(32, k - i0);
      const float2 Q = myck[seg * 32 + lane];
      float v[32];
      const int escale = ESP ? myce[seg * 32 + lane] + Se : 0;
      if (n == 32)
        long_segment<true>(el + i0, n, ar, ai, br, bi, Q.x, Q.y, Sr, Si, v);
      else
        long_segment<false>(el + i0, n, ar, ai, br, bi, Q.x, Q.y, Sr, Si, v);
      if (ESP) {
#pragma unroll
        for (int t = 0; t < 32; ++t) v[t] = ldexpf(v[t], escale);
        renorm(Sr, Si, Se);
      }
      const float s = reduce_scatter32(v, lane);
      if (lane < n) gr[i0 + lane] += s;
    }
  }
  // value: sum of the lanes' root terms
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) fe_part += __shfl_xor_sync(0xffffffffu, fe_part, o);
  if (a.fe != nullptr && lane == 0 && bt + w < a.nb)
    a.fe[static_cast<long long>(__ldg(a.cons_orig + cb)) * a.fe_pitch + a.b0 + bt + w] = tab[0].x + fe_part;
  __syncthreads();
  for (int idx = tid; idx < k * LONG_RT; idx += blockDim.x) {
    const int i = idx >> 3, r = idx & 7;
    if (bt + r < a.nb) {
      const int2 li = lits[i];
      const float gv = gs[r * L.kpad + i];
      a.go[static_cast<long long>(li.y) * a.go_pitch + bt + r] = (li.x & 1) ? -gv : gv;
    }
  }
}

size_t long_smem_bytes(int kmax, bool esp) { return LongLayout(kmax).bytes(esp); }

template <typename XT, bool ESP>
static void launch_long_t(const FeGroupArgs& a, cudaStream_t s) {
  const size_t smem = LongLayout(a.k).bytes(ESP);
  const int tiles = (a.nb + LONG_RT - 1) / LONG_RT;
  const long long blocks = static_cast<long long>(tiles) * a.c_count;
  launch_pdl(fe_grad_long_kernel<XT, ESP>, dim3(static_cast<unsigned>(blocks)), dim3(256), smem, s, a, a.k);
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

bool prepare_kernels() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  if (LongLayout(1024).bytes(true) + 64 > static_cast<size_t>(optin)) return false;
  bool ok = true;
  ok &= raise_smem_cap(fe_grad_long_kernel<float, false>, optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<float, true>, optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<__nv_bfloat16, false>, optin);
  ok &= raise_smem_cap(fe_grad_long_kernel<__nv_bfloat16, true>, optin);
  return ok;
}

// a.k carries the group's longest constraint for the long kernel
void launch_fe_long(const FeGroupArgs& a, int xt, int basis, int /*rt*/, cudaStream_t s) {
  if (xt == XT_F32) {
    if (basis == 0) launch_long_t<float, false>(a, s);
    else launch_long_t<float, true>(a, s);
  } else {
    if (basis == 0) launch_long_t<__nv_bfloat16, false>(a, s);
    else launch_long_t<__nv_bfloat16, true>(a, s);
  }
}

// ---------------------------------------------------------------------------
// CSR gather and projected step (Algorithm 1, step and projection):
// g[v][b] = sum over the slots of v (fixed order) of go[slot][b];
// x <- clamp(x - eta g, -1, 1), or g written out in evaluation mode.
// One lane per restart, one warp per (variable, 32 restarts).
// ---------------------------------------------------------------------------
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

template <typename XT>
__global__ void __launch_bounds__(256) csr_update_kernel(CsrArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int tiles = (a.nb + 31) >> 5;
  const long long vl = warp / tiles;
  if (vl >= a.v_count) return;
  const int tile = static_cast<int>(warp - vl * tiles);
  const int bl = tile * 32 + lane;
  if (bl >= a.nb) return;
  const int v = a.v_begin + static_cast<int>(vl);
  const int s0 = __ldg(a.csr_off + v), s1 = __ldg(a.csr_off + v + 1);
  // eight independent loads in flight per lane; the summation order is fixed
  // by the slot order, so the result does not depend on timing
  const float* col = a.go + bl;
  float acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = 0.f;
  int s = s0;
  for (; s + 7 < s1; s += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldg(col + static_cast<long long>(s + u) * a.go_pitch);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += v[u];
  }
  {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = s + u < s1 ? __ldg(col + static_cast<long long>(s + u) * a.go_pitch) : 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) acc[u] += v[u];
  }
  const float g = ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
  if (a.grad != nullptr) {
    a.grad[static_cast<long long>(v) * a.grad_pitch + a.b0 + bl] = g;
    return;
  }
  if (a.sflag != nullptr && a.sflag[static_cast<long long>(__ldg(a.var_inst + v)) * a.B + a.b0 + bl] != 0) return;
  XT* xp = static_cast<XT*>(a.x) + static_cast<long long>(v) * a.x_pitch + a.b0 + bl;
  const float xn = fminf(fmaxf(fmaf(-a.eta, g, load_x_rw<XT>(xp)), -1.0f), 1.0f);
  store_x<XT>(xp, xn);
}

// Step-path variant: each lane owns 4 consecutive restarts, so a warp reads
// 512 contiguous bytes of every occurrence row (16-byte vector loads) and
// updates 4 states. Needs the state's row pitch and the chunk start to be
// multiples of 4 and the buffers 16-byte aligned (true for the library's own
// state and occurrence buffers); lanes past nb are masked per element.
template <typename XT>
__global__ void __launch_bounds__(256) csr_update_vec4_kernel(CsrArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int tiles = (a.nb + 127) >> 7;
  const long long vl = warp / tiles;
  if (vl >= a.v_count) return;
  const int tile = static_cast<int>(warp - vl * tiles);
  const int bl = tile * 128 + lane * 4;
  if (bl >= a.nb) return;
  const int v = a.v_begin + static_cast<int>(vl);
  const int s0 = __ldg(a.csr_off + v), s1 = __ldg(a.csr_off + v + 1);
  const float* col = a.go + bl;
  float4 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_float4(0.f, 0.f, 0.f, 0.f);
  int s = s0;
  for (; s + 3 < s1; s += 4) {
    float4 t[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) t[u] = __ldg(reinterpret_cast<const float4*>(col + static_cast<long long>(s + u) * a.go_pitch));
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      acc[u].x += t[u].x;
      acc[u].y += t[u].y;
      acc[u].z += t[u].z;
      acc[u].w += t[u].w;
    }
  }
  for (; s < s1; ++s) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(col + static_cast<long long>(s) * a.go_pitch));
    acc[0].x += t.x;
    acc[0].y += t.y;
    acc[0].z += t.z;
    acc[0].w += t.w;
  }
  const float g[4] = {(acc[0].x + acc[1].x) + (acc[2].x + acc[3].x), (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y),
                      (acc[0].z + acc[1].z) + (acc[2].z + acc[3].z), (acc[0].w + acc[1].w) + (acc[2].w + acc[3].w)};
  const int inst = __ldg(a.var_inst + v);
  XT* xp = static_cast<XT*>(a.x) + static_cast<long long>(v) * a.x_pitch + a.b0 + bl;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    if (bl + e >= a.nb) break;
    if (a.sflag != nullptr && a.sflag[static_cast<long long>(inst) * a.B + a.b0 + bl + e] != 0) continue;
    const float xn = fminf(fmaxf(fmaf(-a.eta, g[e], load_x_rw<XT>(xp + e)), -1.0f), 1.0f);
    store_x<XT>(xp + e, xn);
  }
}

void launch_csr_update(const CsrArgs& a, int xt, cudaStream_t s) {
  const bool vec = a.grad == nullptr && (a.go_pitch % 4) == 0 && (a.x_pitch % 4) == 0 && (a.b0 % 4) == 0 &&
                   (reinterpret_cast<uintptr_t>(a.go) % 16) == 0;
  if (vec) {
    const long long tiles = (a.nb + 127) / 128;
    const long long blocks = (tiles * a.v_count + 7) / 8;
    if (blocks == 0) return;
    if (xt == XT_F32) launch_pdl(csr_update_vec4_kernel<float>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
    else launch_pdl(csr_update_vec4_kernel<__nv_bfloat16>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
    return;
  }
  const long long tiles = (a.nb + 31) / 32;
  const long long nwarps = tiles * a.v_count;
  const long long blocks = (nwarps + 7) / 8;
  if (blocks == 0) return;
  if (xt == XT_F32) launch_pdl(csr_update_kernel<float>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
  else launch_pdl(csr_update_kernel<__nv_bfloat16>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
}

// ---------------------------------------------------------------------------
// Exact check (Algorithm 1's unsat count at the sign-rounded point):
// literal true iff (x_v < 0) xor negated; constraint violated iff
// viol[t] = 1 for its true count t. One warp per (range of constraints of
// one instance, 32 restarts); one atomic add per lane per range.
// ---------------------------------------------------------------------------
template <typename XT>
__global__ void __launch_bounds__(256) verify_kernel(VerifyArgs a) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31;
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int tiles = (a.B + 31) >> 5;
  const long long rgi = warp / tiles;
  if (rgi >= a.n_ranges) return;
  const int tile = static_cast<int>(warp - rgi * tiles);
  const int b = tile * 32 + lane;
  const bool act = b < a.B;
  const int4 rg = __ldg(a.ranges + rgi);
  const XT* x = static_cast<const XT*>(a.x);
  int count = 0;
  const XT* xb = x + (act ? b : 0);
  for (int c = rg.x; c < rg.y; ++c) {
    const int l0 = __ldg(a.lit_off + c), l1 = __ldg(a.lit_off + c + 1);
    int t = 0;
    int l = l0;
    for (; l + 3 < l1; l += 4) {  // four independent gathers in flight
      const int e0 = __ldg(a.lit_enc + l), e1 = __ldg(a.lit_enc + l + 1);
      const int e2 = __ldg(a.lit_enc + l + 2), e3 = __ldg(a.lit_enc + l + 3);
      const float x0 = load_x<XT>(xb + static_cast<long long>(e0 >> 1) * a.x_pitch);
      const float x1 = load_x<XT>(xb + static_cast<long long>(e1 >> 1) * a.x_pitch);
      const float x2 = load_x<XT>(xb + static_cast<long long>(e2 >> 1) * a.x_pitch);
      const float x3 = load_x<XT>(xb + static_cast<long long>(e3 >> 1) * a.x_pitch);
      t += (static_cast<int>(x0 < 0.0f) ^ (e0 & 1)) + (static_cast<int>(x1 < 0.0f) ^ (e1 & 1)) +
           (static_cast<int>(x2 < 0.0f) ^ (e2 & 1)) + (static_cast<int>(x3 < 0.0f) ^ (e3 & 1));
    }
    for (; l < l1; ++l) {
      const int enc = __ldg(a.lit_enc + l);
      const float xv = load_x<XT>(xb + static_cast<long long>(enc >> 1) * a.x_pitch);
      t += static_cast<int>(xv < 0.0f) ^ (enc & 1);
    }
    count += __ldg(a.viol + __ldg(a.viol_off + c) + t);
  }
  if (act && count > 0) atomicAdd(a.unsat + static_cast<long long>(rg.z) * a.B + b, count);
}

void launch_verify(const VerifyArgs& a, int xt, cudaStream_t s) {
  const long long tiles = (a.B + 31) / 32;
  const long long nwarps = tiles * a.n_ranges;
  const long long blocks = (nwarps + 7) / 8;
  if (blocks == 0) return;
  if (xt == XT_F32) launch_pdl(verify_kernel<float>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
  else launch_pdl(verify_kernel<__nv_bfloat16>, dim3(static_cast<unsigned>(blocks)), dim3(256), 0, s, a);
}

// Fold of the fused check: restart (inst, b) is solved when no warp flagged a
// violation in any row. Records the lowest solved restart per instance and
// clears the rows the next step's check writes.
__global__ void fold_flags_kernel(FlagArgs a) {
  pdl_wait();
  pdl_trigger();
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(a.n_inst) * a.nb) return;
  const int inst = static_cast<int>(i / a.nb);
  const int b = a.b0 + static_cast<int>(i - static_cast<long long>(inst) * a.nb);
  const long long ui = static_cast<long long>(inst) * a.B + b;
  int any = 0;
#pragma unroll 8
  for (int s = 0; s < VFLAG_SLOTS; ++s) {
    any |= a.vflag_cur[s * a.stride + ui];
    a.vflag_next[s * a.stride + ui] = 0;
  }
  a.sflag[ui] = any ? 0 : 1;
  if (!any) atomicMin(a.solved + inst, b);
}

void launch_fold_flags(const FlagArgs& a, cudaStream_t s) {
  const long long n = static_cast<long long>(a.n_inst) * a.nb;
  if (n == 0) return;
  launch_pdl(fold_flags_kernel, dim3(static_cast<unsigned>((n + 255) / 256)), dim3(256), 0, s, a);
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

}  // namespace afs
