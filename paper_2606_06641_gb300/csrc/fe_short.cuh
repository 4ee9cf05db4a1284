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
// zero factors are safe. Each lane owns RPL restarts of one constraint
// (restart-major x[v][b]: every literal is one coalesced row gather), the
// k-literal loop is unrolled so prefixes live in registers, and the roots are
// a runtime loop. Per (literal, complex root) the work is a prefix product
// (4 FP32 instructions), a suffix product (4) and the gradient combine (2).
#pragma once
#include <cuda_bf16.h>

#include "afsat_internal.h"

namespace afs {

template <typename XT>
__device__ __forceinline__ float load_x(const XT* p);
template <>
__device__ __forceinline__ float load_x<float>(const float* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ float load_x<__nv_bfloat16>(const __nv_bfloat16* p) {
  const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
  return __uint_as_float(static_cast<unsigned int>(u) << 16);
}

template <int K, int RPL, typename XT, bool SHIFT>
__global__ void __launch_bounds__(128) fe_grad_short_kernel(FeGroupArgs a) {
  const int lane = threadIdx.x & 31;
  const long long warp = static_cast<long long>(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
  constexpr int TW = 32 * RPL;
  const int tiles = (a.nb + TW - 1) / TW;
  const long long c = warp / tiles;
  if (c >= a.c_count) return;
  const int tile = static_cast<int>(warp - c * tiles);
  const int cb = a.c_begin + static_cast<int>(c);
  const int2* ls = a.litslot + a.lit_base + c * K;
  const XT* x = static_cast<const XT*>(a.x);

  int bl[RPL];
  bool act[RPL];
#pragma unroll
  for (int r = 0; r < RPL; ++r) {
    bl[r] = tile * TW + r * 32 + lane;
    act[r] = bl[r] < a.nb;
  }

  int2 lit[K];
#pragma unroll
  for (int i = 0; i < K; ++i) lit[i] = __ldg(ls + i);

  float l[RPL][K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    const long long row = static_cast<long long>(lit[i].x >> 1) * a.x_pitch + a.b0;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      const float xv = act[r] ? load_x<XT>(x + row + bl[r]) : 0.0f;
      l[r][i] = (lit[i].x & 1) ? -xv : xv;
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
  int ti = 1;

  // real roots: factor (l + alpha)
  constexpr int NREAL = (K & 1) + (SHIFT ? 1 : 0);
#pragma unroll
  for (int q = 0; q < NREAL; ++q) {
    const float4 rc = __ldg(tab + ti + q);
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
  ti += NREAL;

  // complex roots: factor (l + alpha) + i gamma
#pragma unroll 1
  for (int j = 0; j < K / 2; ++j) {
    const float4 cc = __ldg(tab + ti + j);
    const float alpha = cc.x, gam = cc.y;
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
      float pr[K], pi[K];
      float Pr = cc.z, Pi = cc.w;
#pragma unroll
      for (int i = 0; i < K; ++i) {
        pr[i] = Pr;
        pi[i] = Pi;
        if (i + 1 < K) {
          const float u = SHIFT ? (l[r][i] + alpha) : l[r][i];
          const float nr = fmaf(Pr, u, -Pi * gam);
          const float ni = fmaf(Pi, u, Pr * gam);
          Pr = nr;
          Pi = ni;
        }
      }
      g[r][K - 1] += pr[K - 1];
      float Sr = SHIFT ? (l[r][K - 1] + alpha) : l[r][K - 1];
      float Si = gam;
#pragma unroll
      for (int i = K - 2; i >= 0; --i) {
        g[r][i] = fmaf(pr[i], Sr, g[r][i]);
        g[r][i] = fmaf(-pi[i], Si, g[r][i]);
        const float u = SHIFT ? (l[r][i] + alpha) : l[r][i];
        const float nr = fmaf(Sr, u, -Si * gam);
        const float ni = fmaf(Si, u, Sr * gam);
        Sr = nr;
        Si = ni;
      }
      fe[r] = fmaf(cc.z, Sr, fmaf(-cc.w, Si, fe[r]));
    }
  }

#pragma unroll
  for (int i = 0; i < K; ++i) {
    float* row = a.go + static_cast<long long>(lit[i].y) * a.go_pitch;
#pragma unroll
    for (int r = 0; r < RPL; ++r)
      if (act[r]) row[bl[r]] = (lit[i].x & 1) ? -g[r][i] : g[r][i];
  }
  if (a.fe != nullptr) {
    const long long orow = static_cast<long long>(__ldg(a.cons_orig + cb)) * a.fe_pitch + a.b0;
#pragma unroll
    for (int r = 0; r < RPL; ++r)
      if (act[r]) a.fe[orow + bl[r]] = fe[r];
  }
}

template <int K, int RPL, typename XT, bool SHIFT>
void launch_short_k(const FeGroupArgs& a, int warps, cudaStream_t s) {
  const int TW = 32 * RPL;
  const long long tiles = (a.nb + TW - 1) / TW;
  const long long nwarps = tiles * a.c_count;
  const long long blocks = (nwarps + warps - 1) / warps;
  fe_grad_short_kernel<K, RPL, XT, SHIFT><<<static_cast<unsigned>(blocks), warps * 32, 0, s>>>(a);
}

}  // namespace afs
