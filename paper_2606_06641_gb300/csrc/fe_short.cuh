// FE + analytic gradient for constraints of length k <= 32 (register kernel).
//
// Sec. 2.1.2: the expansion of a symmetric constraint is a combination of
// products over its literals at the k+1 roots of unity. Per root the factor
// of literal i is affine in l_i = s_i x_{v_i}; the host folds the root's
// scale into one complex constant E so that every factor reads
// (l_i + alpha + i*gamma):
//     FE       = c0 + sum_roots Re(E prod_i (l_i + alpha + i gamma))
//     dFE/dl_i =      sum_roots Re(E prod_{i' != i} (l_i' + alpha + i gamma))
// (alpha = 0 for the probability-generating basis, gamma = 0 for real roots).
// The gradient uses prefix and suffix products, so there is no division and
// zero factors are safe. Each lane owns RPL restarts (restart-major x[v][b]:
// every literal is one coalesced row gather), a warp walks `cpw` consecutive
// constraints of its group, the k-literal loop is unrolled so prefixes live in
// registers, and the roots are a runtime loop. Per (literal, complex root) the
// work is a prefix product (4 FP32 instructions), a suffix product (4) and the
// gradient combine (2). A literal's sign s_i is applied with one multiply per
// value (l = s x on the way in, s dFE/dl on the way out), and only the
// negation bits and the slot reads are kept per literal, so a k = 20 tile
// holds its k literal values, k prefixes and k gradients and little else.
#pragma once
#include <cuda_bf16.h>

#include "afsat_internal.h"
#include "coef.h"

namespace afs {

// State loads. COH = false: through the read-only data cache (__ldg), for
// data no thread writes during the kernel. COH = true: L2-coherent loads
// (__ldcg, bypassing L1), for data written by other thread blocks earlier in
// the same (persistent) kernel.
template <bool COH>
__device__ __forceinline__ float ld_f(const float* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ unsigned short ld_u16(const unsigned short* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float2 ld_f2(const float2* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ float4 ld_f4(const float4* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ unsigned ld_u32(const unsigned* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH>
__device__ __forceinline__ uint2 ld_u2(const uint2* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}

template <typename XT, bool COH = false>
__device__ __forceinline__ float load_x(const XT* p);
template <>
__device__ __forceinline__ float load_x<float, false>(const float* p) {
  return ld_f<false>(p);
}
template <>
__device__ __forceinline__ float load_x<float, true>(const float* p) {
  return ld_f<true>(p);
}
template <>
__device__ __forceinline__ float load_x<__nv_bfloat16, false>(const __nv_bfloat16* p) {
  return __uint_as_float(static_cast<unsigned int>(ld_u16<false>(reinterpret_cast<const unsigned short*>(p))) << 16);
}
template <>
__device__ __forceinline__ float load_x<__nv_bfloat16, true>(const __nv_bfloat16* p) {
  return __uint_as_float(static_cast<unsigned int>(ld_u16<true>(reinterpret_cast<const unsigned short*>(p))) << 16);
}

// N consecutive state values with one vector load (N = 2 or 4; 16-byte or
// 8-byte alignment for FP32, 8- or 4-byte for BF16)
template <typename XT, int N, bool COH = false>
__device__ __forceinline__ void load_xvec(const XT* p, float (&v)[N]) {
  if constexpr (sizeof(XT) == 4) {
    if constexpr (N == 2) {
      const float2 t = ld_f2<COH>(reinterpret_cast<const float2*>(p));
      v[0] = t.x;
      v[1] = t.y;
    } else {
      const float4 t = ld_f4<COH>(reinterpret_cast<const float4*>(p));
      v[0] = t.x;
      v[1] = t.y;
      v[2] = t.z;
      v[3] = t.w;
    }
  } else {
    if constexpr (N == 2) {
      const unsigned t = ld_u32<COH>(reinterpret_cast<const unsigned*>(p));
      v[0] = __uint_as_float(t << 16);
      v[1] = __uint_as_float(t & 0xffff0000u);
    } else {
      const uint2 t = ld_u2<COH>(reinterpret_cast<const uint2*>(p));
      v[0] = __uint_as_float(t.x << 16);
      v[1] = __uint_as_float(t.x & 0xffff0000u);
      v[2] = __uint_as_float(t.y << 16);
      v[3] = __uint_as_float(t.y & 0xffff0000u);
    }
  }
}
template <int N>
__device__ __forceinline__ void store_fvec(float* p, const float (&v)[N]);
template <>
__device__ __forceinline__ void store_fvec<2>(float* p, const float (&v)[2]) {
  *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void store_fvec<4>(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// VEC (with RPL > 1): a lane's RPL restarts are consecutive, so a literal's
// gather is one vector load and a derivative store one vector store. It needs
// the state's row pitch, the chunk start and the derivative pitch to be
// multiples of 32 (the library's own state and buffers); a vector that starts
// below nb then stays inside the padded row, and values past nb are ignored.
// Approximate reciprocal (PTX rcp.approx, within one unit in the last place)
// of a number >= 1.
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// Blocks of 4 warps per SM the short kernel is compiled for (register cap)
// with one restart per lane in the probability-generating basis, where the
// division form holds about 2k values per lane (literal values and gradient
// sums).
constexpr int SHORT_MIN_BLOCKS_SCALED = 6;    // k <= KSCALED_MAX
constexpr int SHORT_MIN_BLOCKS_UNSCALED = 5;  // KSCALED_MAX < k <= 32
template <int K, int RPL, bool SHIFT>
constexpr int short_min_blocks() {
  if (SHIFT || RPL != 1) return 1;
  return K <= KSCALED_MAX ? SHORT_MIN_BLOCKS_SCALED : SHORT_MIN_BLOCKS_UNSCALED;
}

// a * b, computed again where the compiler would otherwise keep the first
// product of the same operands live (k registers) across the forward pass
__device__ __forceinline__ float mul_recompute(float a, float b) {
  float r;
  asm volatile("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}

// One warp's unit of a short group: `warp` indexes (constraint chunk of
// a.cpw constraints, tile of 32 * RPL restarts). COH: the state is read with
// L2-coherent loads (it was written earlier in the same persistent kernel).
template <int K, int RPL, typename XT, bool SHIFT, bool VEC, bool COH>
__device__ __forceinline__ void short_unit(const FeGroupArgs& a, long long warp, int lane) {
  constexpr int TW = 32 * RPL;
  const int tiles = (a.nb + TW - 1) / TW;
  const long long cg = warp / tiles;
  const long long c_first = cg * a.cpw;
  if (c_first >= a.c_count) return;
  const int tile = static_cast<int>(warp - cg * tiles);
  const int c_last = static_cast<int>(min(static_cast<long long>(a.c_count), c_first + a.cpw));
  const XT* x = static_cast<const XT*>(a.x);

  constexpr bool V = VEC && RPL > 1;
  int bl[RPL];
  bool act[RPL];
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    bl[r] = V ? tile * TW + lane * RPL + r : tile * TW + r * 32 + lane;
    act[r] = bl[r] < a.nb;
  }

  for (int c = static_cast<int>(c_first); c < c_last; ++c) {
    const int cb = a.c_begin + c;
    const int2* ls = a.litslot + a.lit_base + static_cast<long long>(c) * K;
    unsigned negm = 0u;
    float l[RPL][K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int enc = __ldg(&ls[i].x);
      negm |= static_cast<unsigned>(enc & 1) << i;
      const float sg = (enc & 1) ? -1.0f : 1.0f;
      const long long row = static_cast<long long>(enc >> 1) * a.x_pitch + a.b0;
      if constexpr (V) {
        float xv[RPL];
        if (act[0]) {
          load_xvec<XT, RPL, COH>(x + row + bl[0], xv);
        } else {
#pragma unroll
          for (int r = 0; r < RPL; ++r) xv[r] = 0.0f;
        }
#pragma unroll
        for (int r = 0; r < RPL; ++r) l[r][i] = xv[r] * sg;
      } else {
#pragma unroll
        for (int r = 0; r < RPL; ++r) l[r][i] = (act[r] ? load_x<XT, COH>(x + row + bl[r]) : 0.0f) * sg;
      }
    }

    const float4* tab = a.coef + __ldg(a.cons_tab + cb);
    const float4 head = __ldg(tab);
    float fe[RPL];
    float g[RPL][K];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      fe[r] = head.x;
#pragma unroll
      for (int i = 0; i < K; ++i) g[r][i] = 0.0f;
    }

    // real roots: factor (l + alpha)
    constexpr int NREAL = (K & 1) + (SHIFT ? 1 : 0);
#pragma unroll
    for (int q = 0; q < NREAL; ++q) {
      const float4 rc = __ldg(tab + 1 + q);
      const float alpha = rc.x, E = rc.y;
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        float pre[K];
        float P = E;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          pre[i] = P;
          if (i + 1 < K) P *= SHIFT ? (l[r][i] + alpha) : l[r][i];
        }
        g[r][K - 1] += pre[K - 1];
        float S = SHIFT ? (l[r][K - 1] + alpha) : l[r][K - 1];
#pragma unroll
        for (int i = K - 2; i >= 0; --i) {
          g[r][i] = fmaf(pre[i], S, g[r][i]);
          S *= SHIFT ? (l[r][i] + alpha) : l[r][i];
        }
        fe[r] = fmaf(E, S, fe[r]);
      }
    }

    constexpr int NC = K / 2;
    // complex roots stored scaled (probability-generating basis, k up to
    // KSCALED_MAX): factor gamma (w + i) with w = l / gamma, gamma^k folded
    // into E', so a running product times the factor is two FMAs
    constexpr bool SCALED = !SHIFT && K <= KSCALED_MAX;
    const int ns = SCALED ? static_cast<int>(head.y) : 0;  // roots stored (zero ones dropped)
#pragma unroll 1
    for (int j = 0; j < ns; ++j) {
      const float4 cc = __ldg(tab + 1 + NREAL + j);
      const float ia = cc.x;  // 1 / gamma
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        // the full product T = E' prod (w_i + i), then each literal's
        // gradient term ia Re(T / (w_i + i)) = ia (Tr w_i + Ti) / (w_i^2 + 1):
        // |w_i + i| >= 1, so dividing a factor out cannot amplify the error,
        // and no prefix products are kept; w is recomputed rather than held
        // (K registers fewer)
        float Tr = cc.z, Ti = cc.w;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const float wi = l[r][i] * ia;
          const float nr = fmaf(Tr, wi, -Ti);
          const float ni = fmaf(Ti, wi, Tr);
          Tr = nr;
          Ti = ni;
        }
        fe[r] += Tr;
        const float Ur = Tr * ia, Ui = Ti * ia;
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const float wi = mul_recompute(l[r][i], ia);
          g[r][i] = fmaf(fmaf(Ur, wi, Ui), rcp_approx(fmaf(wi, wi, 1.0f)), g[r][i]);
        }
      }
    }

    if constexpr (!SCALED && !SHIFT) {
      // probability-generating basis above KSCALED_MAX: factor l + i gamma
      // with |l + i gamma| >= gamma >= cot(pi k / (2 (k + 1))), never zero:
      // the full product T = E' prod (l_i + i gamma) and each literal's term
      // Re(T / (l_i + i gamma)) = (Tr l_i + Ti gamma) / (l_i^2 + gamma^2)
#pragma unroll 1
      for (int j = 0; j < NC; ++j) {
        const float4 cc = __ldg(tab + 1 + NREAL + j);
        const float gam = cc.y, g2 = gam * gam;
#pragma unroll
        for (int r = 0; r < RPL; ++r) {
          float Tr = cc.z, Ti = cc.w;
#pragma unroll
          for (int i = 0; i < K; ++i) {
            const float nr = fmaf(Tr, l[r][i], -Ti * gam);
            const float ni = fmaf(Ti, l[r][i], Tr * gam);
            Tr = nr;
            Ti = ni;
          }
          fe[r] += Tr;
          const float tig = Ti * gam;
#pragma unroll
          for (int i = 0; i < K; ++i)
            g[r][i] = fmaf(fmaf(Tr, l[r][i], tig), rcp_approx(fmaf(l[r][i], l[r][i], g2)), g[r][i]);
        }
      }
    }
    // the paper basis: complex roots are factors (l + alpha) + i gamma, taken
    // by prefix and suffix products (these factors can vanish); RPI roots per
    // iteration are independent product chains interleaved for instruction-
    // level parallelism (they share the literal values and the accumulators)
    // (two interleaved roots measured slower at k = 20: the register growth
    // costs more occupancy than the extra chains win back)
    constexpr int RPI = 1;
#pragma unroll 1
    for (int j = ns; j < (SCALED || !SHIFT ? 0 : NC); j += RPI) {
      float4 cc[RPI];
      bool on[RPI];
#pragma unroll
      for (int q = 0; q < RPI; ++q) {
        on[q] = (q == 0) || (j + q < NC);
        cc[q] = on[q] ? __ldg(tab + 1 + NREAL + j + q) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int r = 0; r < RPL; ++r) {
        float pr[RPI][K], pi[RPI][K];
        float Pr[RPI], Pi[RPI];
#pragma unroll
        for (int q = 0; q < RPI; ++q) {
          Pr[q] = cc[q].z;
          Pi[q] = cc[q].w;
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
#pragma unroll
          for (int q = 0; q < RPI; ++q) {
            pr[q][i] = Pr[q];
            pi[q][i] = Pi[q];
            if (i + 1 < K) {
              const float u = SHIFT ? (l[r][i] + cc[q].x) : l[r][i];
              const float nr = fmaf(Pr[q], u, -Pi[q] * cc[q].y);
              const float ni = fmaf(Pi[q], u, Pr[q] * cc[q].y);
              Pr[q] = nr;
              Pi[q] = ni;
            }
          }
        }
        float Sr[RPI], Si[RPI];
#pragma unroll
        for (int q = 0; q < RPI; ++q) {
          g[r][K - 1] += pr[q][K - 1];
          Sr[q] = SHIFT ? (l[r][K - 1] + cc[q].x) : l[r][K - 1];
          Si[q] = cc[q].y;
        }
#pragma unroll
        for (int i = K - 2; i >= 0; --i) {
#pragma unroll
          for (int q = 0; q < RPI; ++q) {
            g[r][i] = fmaf(pr[q][i], Sr[q], g[r][i]);
            g[r][i] = fmaf(-pi[q][i], Si[q], g[r][i]);
            const float u = SHIFT ? (l[r][i] + cc[q].x) : l[r][i];
            const float nr = fmaf(Sr[q], u, -Si[q] * cc[q].y);
            const float ni = fmaf(Si[q], u, Sr[q] * cc[q].y);
            Sr[q] = nr;
            Si[q] = ni;
          }
        }
#pragma unroll
        for (int q = 0; q < RPI; ++q) fe[r] = fmaf(cc[q].z, Sr[q], fmaf(-cc[q].w, Si[q], fe[r]));
      }
    }

#pragma unroll
    for (int i = 0; i < K; ++i) {
      const float sg = ((negm >> i) & 1u) ? -1.0f : 1.0f;
      const int slot = __ldg(&ls[i].y);
      if (K == KFUSE && slot < 0) continue;  // fused constraint: no derivative row
      float* row = a.go + static_cast<long long>(slot) * a.go_pitch;
      if constexpr (V) {
        if (act[0]) {
          float gv[RPL];
#pragma unroll
          for (int r = 0; r < RPL; ++r) gv[r] = g[r][i] * sg;
          store_fvec<RPL>(row + bl[0], gv);
        }
      } else {
#pragma unroll
        for (int r = 0; r < RPL; ++r)
          if (act[r]) row[bl[r]] = g[r][i] * sg;
      }
    }
    if (a.fe != nullptr) {
      const long long orow = static_cast<long long>(__ldg(a.cons_orig + cb)) * a.fe_pitch + a.b0;
#pragma unroll
      for (int r = 0; r < RPL; ++r)
        if (act[r]) a.fe[orow + bl[r]] = fe[r];
    }
  }
}

template <int K, int RPL, typename XT, bool SHIFT, bool VEC>
__global__ void __launch_bounds__(128, short_min_blocks<K, RPL, SHIFT>()) fe_grad_short_kernel(FeGroupArgs a) {
  pdl_wait();
  pdl_trigger();
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  short_unit<K, RPL, XT, SHIFT, VEC, false>(a, warp, static_cast<int>(threadIdx.x & 31));
}

template <int K, int RPL, typename XT, bool SHIFT>
void launch_short_k(const FeGroupArgs& a_in, int warps, cudaStream_t s) {
  FeGroupArgs a = a_in;
  if (a.cpw < 1) a.cpw = 1;
  const int TW = 32 * RPL;
  const long long tiles = (a.nb + TW - 1) / TW;
  const long long nwarps = tiles * ((a.c_count + a.cpw - 1) / a.cpw);
  const long long blocks = (nwarps + warps - 1) / warps;
  if constexpr (RPL > 1) {
    if (a.vec) {
      launch_pdl(fe_grad_short_kernel<K, RPL, XT, SHIFT, true>, dim3(static_cast<unsigned>(blocks)), dim3(warps * 32),
                 0, s, a);
      return;
    }
  }
  launch_pdl(fe_grad_short_kernel<K, RPL, XT, SHIFT, false>, dim3(static_cast<unsigned>(blocks)), dim3(warps * 32), 0,
             s, a);
}

}  // namespace afs
