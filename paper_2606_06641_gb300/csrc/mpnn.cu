// Learned initialiser: a bipartite variable-constraint message-passing
// network that proposes starting points mu_v for the descent, trained on
// assignments found by the solver itself (the paper has no learned part; the
// network is the one the benchmark plan specifies).
//
//   h_v = relu(f_v A_v^T + a_v),  h_c = relu(f_c A_c^T + a_c)
//   per layer l:  P = h_v U_l^T,  m_c = mean_{e in c} s_e P[v_e]
//                 h_c = relu([h_c, m_c] Wc_l^T + bc_l)
//                 Q = h_c V_l^T,  q_v = mean_{e at v} s_e Q[c_e]
//                 h_v = relu([h_v, q_v] Wv_l^T + bv_l)
//   z = h_v w + b,  mu = tanh(z),  loss = mean BCE(sigmoid(-2 z), y)
//
// Dense products run on the tensor cores (mma.sync m16n8k16, BF16 operands
// rounded from the FP32 masters and activations, FP32 accumulation); the
// segment means are deterministic gathers over edge lists; the backward pass
// mirrors the forward; Adam keeps FP32 moments. Every reduction across CTAs
// (the weight gradients' K slices, bias and head gradients, the loss and the
// label-mask sum) writes per-CTA partials that one final pass adds in a fixed
// order, so a gradient is bit-identical from run to run.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "../../include/afsat.h"
#include "afsat_internal.h"

namespace afs {
namespace {

constexpr int H = 64;
constexpr int FV = 4;
constexpr int FC = 16;

#define MCK(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return ::afs::set_error(AFS_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
#define MCKL()                                                                                     \
  do {                                                                                             \
    cudaError_t e_ = cudaPeekAtLastError();                                                        \
    if (e_ != cudaSuccess) {                                                                       \
      cudaGetLastError();                                                                          \
      return ::afs::set_error(AFS_E_CUDA, "mpnn kernel launch: %s", cudaGetErrorString(e_));     \
    }                                                                                              \
  } while (0)

// ---------------------------------------------------------------------------
// BF16 tensor-core GEMM: C[i][j] (=, +=, atomic +=) epi(sum_k A[i][k] B[k][j])
// A[i][k] = A[i*sa0 + k*sa1], B[k][j] = B[k*sb0 + j*sb1]; 64x64 CTA tile,
// 4 warps x (16 rows x 64 columns), K step 16; grid.z splits K.
// ---------------------------------------------------------------------------
struct GemmArgs {
  const float* A;
  long long sa0, sa1;
  const float* B;
  long long sb0, sb1;
  float* C;
  long long ldc;
  int M, N, K;
  const float* bias;
  int relu;
  int mode;  // 0: C = r, 1: C += r, 2: slice partial (C + blockIdx.z * M * N, row pitch N)
  int k_split;
};

__device__ __forceinline__ void mma_bf16(float (&c)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
  __shared__ __align__(16) __nv_bfloat16 As[64][24];  // [row][k], padded rows
  __shared__ __align__(16) __nv_bfloat16 Bs[64][24];  // [col][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int row0 = blockIdx.x * 64, col0 = blockIdx.y * 64;
  const int kbeg = blockIdx.z * g.k_split;
  const int kend = min(g.K, kbeg + g.k_split);
  float acc[8][4];
#pragma unroll
  for (int t = 0; t < 8; ++t)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[t][q] = 0.f;
  for (int k0 = kbeg; k0 < kend; k0 += 16) {
    for (int e = tid; e < 1024; e += 128) {
      const int r = e >> 4, kk = e & 15;
      const int gi = row0 + r, gk = k0 + kk;
      const float v = (gi < g.M && gk < kend) ? g.A[gi * g.sa0 + gk * g.sa1] : 0.f;
      As[r][kk] = __float2bfloat16_rn(v);
    }
    for (int e = tid; e < 1024; e += 128) {
      const int c = e >> 4, kk = e & 15;
      const int gj = col0 + c, gk = k0 + kk;
      const float v = (gj < g.N && gk < kend) ? g.B[gk * g.sb0 + gj * g.sb1] : 0.f;
      Bs[c][kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    const int r = warp * 16 + gid;
    const unsigned a0 = *reinterpret_cast<const unsigned*>(&As[r][2 * tig]);
    const unsigned a1 = *reinterpret_cast<const unsigned*>(&As[r + 8][2 * tig]);
    const unsigned a2 = *reinterpret_cast<const unsigned*>(&As[r][2 * tig + 8]);
    const unsigned a3 = *reinterpret_cast<const unsigned*>(&As[r + 8][2 * tig + 8]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + gid;
      const unsigned b0 = *reinterpret_cast<const unsigned*>(&Bs[c][2 * tig]);
      const unsigned b1 = *reinterpret_cast<const unsigned*>(&Bs[c][2 * tig + 8]);
      mma_bf16(acc[nt], a0, a1, a2, a3, b0, b1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int row = row0 + warp * 16 + gid + 8 * hh;
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int col = col0 + nt * 8 + 2 * tig + q;
        if (row < g.M && col < g.N) {
          float v = acc[nt][2 * hh + q];
          if (g.mode == 2) {
            g.C[(static_cast<long long>(blockIdx.z) * g.M + row) * g.N + col] = v;
          } else {
            float* dst = g.C + row * g.ldc + col;
            if (g.bias) v += g.bias[col];
            if (g.relu) v = fmaxf(v, 0.f);
            *dst = g.mode == 1 ? *dst + v : v;
          }
        }
      }
    }
  }
}

// C[i][j] += sum_z part[z][i][j], z in order
__global__ void slice_sum_kernel(const float* part, int slices, long long mn, int N, float* C, long long ldc) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= mn) return;
  float acc = 0.f;
  for (int z = 0; z < slices; ++z) acc += part[z * mn + i];
  const long long r = i / N, c = i - r * N;
  C[r * ldc + c] += acc;
}

constexpr int WGRAD_KSPLIT = 1024;  // inner-dimension slice of a weight-gradient product

// Slices of a weight-gradient product over K (graph nodes) and the scratch they need.
inline int wgrad_slices(int K) { return (K + WGRAD_KSPLIT - 1) / WGRAD_KSPLIT; }

// mode 0: C = A B (+bias, relu); mode 1: C += A B; mode 2 (weight gradients,
// K = graph nodes): C += A B with the inner dimension split into slices of
// WGRAD_KSPLIT over CTAs, each slice's product written to `scratch` and the
// slices added in order (deterministic).
void gemm(const float* A, long long sa0, long long sa1, const float* B, long long sb0, long long sb1, float* C,
          long long ldc, int M, int N, int K, const float* bias, bool relu, int mode, cudaStream_t s,
          float* scratch = nullptr) {
  if (M <= 0 || N <= 0 || K <= 0) return;  // empty product (weight gradients of an empty graph stay zero)
  GemmArgs g{A, sa0, sa1, B, sb0, sb1, C, ldc, M, N, K, bias, relu ? 1 : 0, mode, K};
  int zsplit = 1;
  if (mode == 2) {
    g.k_split = WGRAD_KSPLIT;
    zsplit = wgrad_slices(K);
    g.C = scratch;
  }
  dim3 grid((M + 63) / 64, (N + 63) / 64, zsplit);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
  if (mode == 2) {
    const long long mn = static_cast<long long>(M) * N;
    slice_sum_kernel<<<static_cast<unsigned>((mn + 255) / 256), 256, 0, s>>>(scratch, zsplit, mn, N, C, ldc);
  }
}

// out[r*ldo + j] = rowscale[r] * sum_{e in [off[r], off[r+1])} s_e * srcscale[src] * src[src*lds + j]
// with src = enc[e] >> 1, s_e = -1 if enc[e] & 1; one thread per (row, feature).
__global__ void edge_mean_kernel(const int* off, const int* enc, const float* src, long long lds,
                                 const float* rowscale, const float* srcscale, float* out, long long ldo, int rows) {
  const int r = blockIdx.x * blockDim.y + threadIdx.y;
  const int j = threadIdx.x;
  if (r >= rows) return;
  float acc = 0.f;
  for (int e = off[r]; e < off[r + 1]; ++e) {
    const int en = __ldg(enc + e);
    const int sidx = en >> 1;
    float v = __ldg(src + sidx * lds + j);
    if (srcscale) v *= __ldg(srcscale + sidx);
    acc += (en & 1) ? -v : v;
  }
  out[r * ldo + j] = rowscale ? acc * rowscale[r] : acc;
}

void edge_mean(const int* off, const int* enc, const float* src, long long lds, const float* rowscale,
               const float* srcscale, float* out, long long ldo, int rows, cudaStream_t s) {
  if (rows <= 0) return;
  dim3 block(H, 4);
  edge_mean_kernel<<<(rows + 3) / 4, block, 0, s>>>(off, enc, src, lds, rowscale, srcscale, out, ldo, rows);
}

// dst[r*ldd + j] = src[r*lds + j] (* [ref[r*ldr + j] > 0] when ref is given), j < 64
__global__ void copy_mask_kernel(const float* src, long long lds, const float* ref, long long ldr, float* dst,
                                 long long ldd, int rows) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(rows) * H) return;
  const long long r = i / H;
  const int j = static_cast<int>(i - r * H);
  float v = src[r * lds + j];
  if (ref && !(ref[r * ldr + j] > 0.f)) v = 0.f;
  dst[r * ldd + j] = v;
}

void copy_mask(const float* src, long long lds, const float* ref, long long ldr, float* dst, long long ldd, int rows,
               cudaStream_t s) {
  const long long n = static_cast<long long>(rows) * H;
  if (n <= 0) return;
  copy_mask_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(src, lds, ref, ldr, dst, ldd, rows);
}

// Fixed-order column sums of a rows x 64 block (optionally weighted per row):
// CTA b adds rows [b*chunk, (b+1)*chunk) in increasing order per thread row
// lane and writes part[b][j]; colsum_final adds the CTA partials in order.
constexpr int RED_CTAS = 128;

inline int red_ctas(int rows) { return std::max(1, std::min(RED_CTAS, (rows + 255) / 256)); }

__global__ void colsum_part_kernel(const float* x, long long ld, int rows, const float* rw, float* part) {
  const int j = threadIdx.x, y = threadIdx.y;  // 64 x 4 threads
  const int chunk = (rows + gridDim.x - 1) / gridDim.x;
  const int r0 = blockIdx.x * chunk, r1 = min(rows, r0 + chunk);
  float acc = 0.f;
  for (int r = r0 + y; r < r1; r += 4) acc = rw ? fmaf(rw[r], x[r * ld + j], acc) : acc + x[r * ld + j];
  __shared__ float p[4][H];
  p[y][j] = acc;
  __syncthreads();
  if (y == 0) part[blockIdx.x * H + j] = ((p[0][j] + p[1][j]) + p[2][j]) + p[3][j];
}

__global__ void colsum_final_kernel(const float* part, int ctas, float* out) {
  const int j = threadIdx.x;
  float acc = 0.f;
  for (int b = 0; b < ctas; ++b) acc += part[b * H + j];
  out[j] += acc;
}

// out[j] += sum_r x[r][j] (rw: sum_r rw[r] x[r][j]); `part` holds RED_CTAS x 64 floats
void colsum(const float* x, long long ld, int rows, float* out, float* part, cudaStream_t s,
            const float* rw = nullptr) {
  if (rows <= 0) return;
  const int ctas = red_ctas(rows);
  colsum_part_kernel<<<ctas, dim3(H, 4), 0, s>>>(x, ld, rows, rw, part);
  colsum_final_kernel<<<1, H, 0, s>>>(part, ctas, out);
}

// Fixed-order sum of n values (or of a[i] * b[i]): CTA partials then one pass.
__global__ void sum_part_kernel(const float* a, const float* b, int n, float* part) {
  const int chunk = (n + gridDim.x - 1) / gridDim.x;
  const int i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  float acc = 0.f;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) acc += b ? a[i] * b[i] : a[i];
  for (int o = 16; o >= 1; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float w[8];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) t += w[k];
    part[blockIdx.x] = t;
  }
}

__global__ void sum_final_kernel(const float* part, int ctas, float* out, int accumulate) {
  if (threadIdx.x != 0) return;
  float t = 0.f;
  for (int b = 0; b < ctas; ++b) t += part[b];
  out[0] = accumulate ? out[0] + t : t;
}

// out[0] (=, +=) sum_i a[i] (* b[i]); `part` holds RED_CTAS floats
void vsum(const float* a, const float* b, int n, float* out, bool accumulate, float* part, cudaStream_t s) {
  const int ctas = red_ctas(n);
  if (n > 0) sum_part_kernel<<<ctas, 256, 0, s>>>(a, b, n, part);
  sum_final_kernel<<<1, 32, 0, s>>>(part, n > 0 ? ctas : 0, out, accumulate ? 1 : 0);
}

// z = h w + b, mu = tanh(z)
__global__ void head_kernel(const float* hv, long long ld, const float* w, const float* b, float* z, float* mu,
                            int n) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  float acc = b[0];
  for (int j = 0; j < H; ++j) acc = fmaf(hv[v * ld + j], w[j], acc);
  z[v] = acc;
  if (mu) mu[v] = tanhf(acc);
}

// l[v] = w_v (softplus(t) - y t) / wsum and dz[v] = -2 w_v (sigmoid(t) - y) / wsum
// with t = -2 z and wsum = max(sum_v w_v, 1) read from the device
__global__ void loss_kernel(const float* z, const float* y, const float* wm, const float* wsum, float* dz, float* l,
                            int n) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const float inv = 1.f / fmaxf(wm ? wsum[0] : static_cast<float>(n), 1.f);
  const float t = -2.f * z[v];
  const float wv = wm ? wm[v] : 1.f;
  const float sp = fmaxf(t, 0.f) + log1pf(expf(-fabsf(t)));
  l[v] = wv * (sp - y[v] * t) * inv;
  const float sig = 1.f / (1.f + expf(-t));
  dz[v] = -2.f * wv * (sig - y[v]) * inv;
}

// dh[v][j] = dz[v] w[j]
__global__ void head_dh_kernel(const float* dz, const float* w, float* dh, int n) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n) * H) return;
  const long long v = i / H;
  dh[i] = dz[v] * w[i - v * H];
}

__global__ void adam_kernel(float* th, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  th[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

// Philox4x32-10 (Salmon et al., SC'11) for the sampling noise.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
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

// Restart b of variable v: for b < B_learn, x = clamp(mu_v + sigma_b eps, -1, 1)
// with sigma_b ramped from sigma_min to sigma_max; other restarts uniform on
// [-1, 1). eps is uniform on [-1, 1) from Philox, counter (b, v, 1, 0).
template <typename XT>
__global__ void sample_kernel(const float* mu, XT* x, long long pitch, int n, int B, int B_learn, float smin,
                              float smax, unsigned long long seed) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n) * B) return;
  const int v = static_cast<int>(i / B), b = static_cast<int>(i - static_cast<long long>(v) * B);
  const uint4 o = philox(make_uint4(static_cast<unsigned>(b), static_cast<unsigned>(v), 1u, 0u),
                         make_uint2(static_cast<unsigned>(seed), static_cast<unsigned>(seed >> 32)));
  const float u = fmaf(2.0f, static_cast<float>(o.x >> 8) * 0x1p-24f, -1.0f);
  float val;
  if (b < B_learn) {
    const float sig = B_learn > 1 ? smin + (smax - smin) * static_cast<float>(b) / (B_learn - 1) : smin;
    val = fminf(fmaxf(fmaf(sig, u, mu[v]), -1.f), 1.f);
  } else {
    val = u;
  }
  if constexpr (sizeof(XT) == 4) {
    x[static_cast<long long>(v) * pitch + b] = val;
  } else {
    x[static_cast<long long>(v) * pitch + b] = __float2bfloat16_rn(val);
  }
}

// Restart b of variable v (B restarts per instance, state already set):
// x = clamp(x + alpha_b mu_v, -1, 1), alpha_b ramped from alpha_min (b = 0)
// to alpha_max (b = B - 1).
template <typename XT>
__global__ void nudge_kernel(const float* mu, XT* x, long long pitch, int n, int B, float amin, float amax) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(n) * B) return;
  const int v = static_cast<int>(i / B), b = static_cast<int>(i - static_cast<long long>(v) * B);
  const float a = B > 1 ? amin + (amax - amin) * static_cast<float>(b) / (B - 1) : amin;
  XT* p = x + static_cast<long long>(v) * pitch + b;
  if constexpr (sizeof(XT) == 4) {
    *p = fminf(fmaxf(fmaf(a, mu[v], *p), -1.f), 1.f);
  } else {
    *p = __float2bfloat16_rn(fminf(fmaxf(fmaf(a, mu[v], __bfloat162float(*p)), -1.f), 1.f));
  }
}

// Features from the instance graph: variable v (degree deg, signed balance
// bal): f_v = (deg/8, bal/max(deg,1), 1, 0), deg_inv = 1/deg (0 if isolated);
// constraint c (length k): f_c = (one-hot type, k/8, param/k for EK and CARD,
// parity for XOR, op for CARD, 1, 0...), k_inv = 1/k.
__global__ void features_kernel(int n, int m, const int* v_off, const int* v_enc, const int* c_off, const int4* cinfo,
                                float* fv, float* deg_inv, float* fc, float* k_inv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int e0 = v_off[i], e1 = v_off[i + 1];
    float bal = 0.f;
    for (int e = e0; e < e1; ++e) bal += (v_enc[e] & 1) ? -1.f : 1.f;
    const float deg = static_cast<float>(e1 - e0);
    deg_inv[i] = deg > 0 ? 1.f / deg : 0.f;
    fv[static_cast<long long>(i) * FV + 0] = deg / 8.f;
    fv[static_cast<long long>(i) * FV + 1] = bal / fmaxf(deg, 1.f);
    fv[static_cast<long long>(i) * FV + 2] = 1.f;
    fv[static_cast<long long>(i) * FV + 3] = 0.f;
  }
  if (i < m) {
    const int4 ci = cinfo[i];  // {type, op, param, parity}
    const float k = static_cast<float>(c_off[i + 1] - c_off[i]);
    k_inv[i] = k > 0 ? 1.f / k : 0.f;
    float f[FC];
#pragma unroll
    for (int q = 0; q < FC; ++q) f[q] = 0.f;
    f[ci.x] = 1.f;
    f[7] = k / 8.f;
    f[8] = (ci.x == AFS_EK || ci.x == AFS_CARD) ? static_cast<float>(ci.z) / fmaxf(k, 1.f) : 0.f;
    f[9] = ci.x == AFS_XOR ? static_cast<float>(ci.w) : 0.f;
    f[10] = ci.x == AFS_CARD ? static_cast<float>(ci.y) : 0.f;
    f[11] = 1.f;
    float4* dst = reinterpret_cast<float4*>(fc + static_cast<long long>(i) * FC);
#pragma unroll
    for (int q = 0; q < FC / 4; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
  }
}

// ---------------------------------------------------------------------------
// per-graph buffers (kept in the handle's extension slot)
// ---------------------------------------------------------------------------
template <typename T>
struct Dev {
  T* p = nullptr;
  size_t n = 0;
  ~Dev() {
    if (p) cudaFree(p);
  }
  cudaError_t alloc(size_t count) {
    if (p) cudaFree(p);
    p = nullptr;
    n = count;
    return cudaMalloc(&p, sizeof(T) * (count ? count : 1));
  }
  cudaError_t upload(const std::vector<T>& h, cudaStream_t s) {
    cudaError_t e = alloc(h.size());
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpyAsync(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s);
  }
};

// Device buffers of one graph, carved from a single allocation (one
// cudaMalloc per bound handle instead of one per buffer).
template <typename T>
struct Span {
  T* p = nullptr;
  size_t n = 0;
};

// One handle's graph as the network sees it: the instance's device arrays
// (built at load) and spans of the network's workspace for the features and
// activations (attached per call).
struct Graph {
  int n = 0, m = 0, layers = 0;
  const int *c_off = nullptr, *c_enc = nullptr, *v_off = nullptr, *v_enc = nullptr;
  const int4* cinfo = nullptr;
  Span<float> k_inv, deg_inv, fv, fc;
  std::vector<Span<float>> Xv, Xc;  // layers + 1 each: [n x 128], [m x 128]
  Span<float> P, Q, z, mu, dz, dhv, dhc, dpre_v, dpre_c, dXv, dXc, dP, dQ, loss;
  // fixed-order reductions: weight-gradient slices, CTA partials, per-variable
  // loss terms, the label-mask sum
  Span<float> wslices, part, lterm, wsum;
};

void release_graph(void* p) { delete static_cast<Graph*>(p); }

int bind_graph(afs_handle* h, int layers, cudaStream_t s, Graph** out) {
  (void)s;
  Graph* g = static_cast<Graph*>(handle_ext(h));
  if (g && g->layers == layers) {
    *out = g;
    return AFS_OK;
  }
  GraphView gv{};
  int rc = graph_view(h, &gv);
  if (rc) return rc;
  g = new Graph();
  g->n = gv.n;
  g->m = gv.m;
  g->layers = layers;
  g->c_off = gv.lit_off_dev;
  g->c_enc = gv.lit_enc_dev;
  g->v_off = gv.v_off_dev;
  g->v_enc = gv.v_enc_dev;
  g->cinfo = gv.cinfo_dev;
  set_handle_ext(h, g, release_graph);
  *out = g;
  return AFS_OK;
}

// The activation and reduction buffers of one forward/backward over graph g,
// carved from a workspace of at least the returned bytes.
size_t carve_workspace(Graph* g, char* base) {
  const int n = g->n, m = g->m, layers = g->layers;
  size_t at = 0;
  auto take = [&](Span<float>& sp, size_t count) {
    sp.n = count;
    if (base) sp.p = reinterpret_cast<float*>(base + at);
    at += (sizeof(float) * std::max<size_t>(count, 1) + 255) / 256 * 256;
  };
  take(g->k_inv, m);
  take(g->deg_inv, n);
  take(g->fv, static_cast<size_t>(n) * FV);
  take(g->fc, static_cast<size_t>(m) * FC);
  g->Xv.resize(layers + 1);
  g->Xc.resize(layers + 1);
  for (int l = 0; l <= layers; ++l) {
    take(g->Xv[l], static_cast<size_t>(n) * 2 * H);
    take(g->Xc[l], static_cast<size_t>(m) * 2 * H);
  }
  const size_t nH = static_cast<size_t>(n) * H, mH = static_cast<size_t>(m) * H;
  take(g->P, nH);
  take(g->Q, mH);
  take(g->z, n);
  take(g->mu, n);
  take(g->dz, n);
  take(g->dhv, nH);
  take(g->dhc, mH);
  take(g->dpre_v, nH);
  take(g->dpre_c, mH);
  take(g->dXv, 2 * nH);
  take(g->dXc, 2 * mH);
  take(g->dP, nH);
  take(g->dQ, mH);
  take(g->loss, 1);
  take(g->wslices, static_cast<size_t>(wgrad_slices(std::max(n, m))) * H * 2 * H);
  take(g->part, static_cast<size_t>(RED_CTAS) * H);
  take(g->lterm, n);
  take(g->wsum, 1);
  return at;
}

}  // namespace
}  // namespace afs

// ---------------------------------------------------------------------------
// network object and ABI
// ---------------------------------------------------------------------------
struct afs_mpnn {
  int layers = 3;
  long long n_params = 0;
  afs::Dev<float> theta, grad, m1, m2;
  // activation workspace, grown to the largest graph seen and reused by every
  // call on this network (calls on one network are stream-ordered)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  ~afs_mpnn() {
    if (ws) cudaFree(ws);
  }
  long long t = 0;
  // offsets into theta
  long long oAv, oav, oAc, oac, ow, ob;
  std::vector<long long> oU, oV, oWc, obc, oWv, obv;
};

using afs::H;

// The handle's graph with this network's workspace attached (grown if needed).
static int bind(afs_mpnn* net, afs_handle* h, cudaStream_t s, afs::Graph** out) {
  afs::Graph* g = nullptr;
  int rc = afs::bind_graph(h, net->layers, s, &g);
  if (rc) return rc;
  const size_t need = afs::carve_workspace(g, nullptr);
  if (need > net->ws_bytes) {
    if (net->ws) {
      cudaError_t e = cudaStreamSynchronize(s);  // earlier work on the old workspace completes first
      if (e == cudaSuccess) e = cudaFree(net->ws);
      net->ws = nullptr;
      net->ws_bytes = 0;
      if (e != cudaSuccess) return afs::set_error(AFS_E_CUDA, "mpnn workspace: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaMalloc(&net->ws, need);
    if (e != cudaSuccess) {
      net->ws = nullptr;
      return afs::set_error(AFS_E_CUDA, "mpnn workspace (%zu bytes): %s", need, cudaGetErrorString(e));
    }
    net->ws_bytes = need;
  }
  afs::carve_workspace(g, static_cast<char*>(net->ws));
  *out = g;
  return AFS_OK;
}

static long long layout(afs_mpnn* net) {
  long long at = 0;
  auto take = [&](long long size) {
    const long long o = at;
    at += size;
    return o;
  };
  net->oAv = take(H * afs::FV);
  net->oav = take(H);
  net->oAc = take(H * afs::FC);
  net->oac = take(H);
  net->oU.clear();
  net->oV.clear();
  net->oWc.clear();
  net->obc.clear();
  net->oWv.clear();
  net->obv.clear();
  for (int l = 0; l < net->layers; ++l) {
    net->oU.push_back(take(H * H));
    net->oV.push_back(take(H * H));
    net->oWc.push_back(take(H * 2 * H));
    net->obc.push_back(take(H));
    net->oWv.push_back(take(H * 2 * H));
    net->obv.push_back(take(H));
  }
  net->ow = take(H);
  net->ob = take(1);
  return at;
}

static int mpnn_forward(afs_mpnn* net, afs::Graph* g, cudaStream_t s) {
  using namespace afs;
  const float* th = net->theta.p;
  const int n = g->n, m = g->m;
  if (n > 0 || m > 0) {
    const int items = std::max(n, m);
    features_kernel<<<(items + 255) / 256, 256, 0, s>>>(n, m, g->v_off, g->v_enc, g->c_off, g->cinfo, g->fv.p,
                                                        g->deg_inv.p, g->fc.p, g->k_inv.p);
  }
  // embeddings into the first halves of the layer-0 inputs
  gemm(g->fv.p, FV, 1, th + net->oAv, 1, FV, g->Xv[0].p, 2 * H, n, H, FV, th + net->oav, true, 0, s);
  gemm(g->fc.p, FC, 1, th + net->oAc, 1, FC, g->Xc[0].p, 2 * H, m, H, FC, th + net->oac, true, 0, s);
  for (int l = 0; l < net->layers; ++l) {
    // P = h_v U^T; m_c = mean s P[v]
    gemm(g->Xv[l].p, 2 * H, 1, th + net->oU[l], 1, H, g->P.p, H, n, H, H, nullptr, false, 0, s);
    edge_mean(g->c_off, g->c_enc, g->P.p, H, g->k_inv.p, nullptr, g->Xc[l].p + H, 2 * H, m, s);
    // h_c' = relu([h_c, m_c] Wc^T + bc)
    gemm(g->Xc[l].p, 2 * H, 1, th + net->oWc[l], 1, 2 * H, g->Xc[l + 1].p, 2 * H, m, H, 2 * H, th + net->obc[l], true,
         0, s);
    // Q = h_c' V^T; q_v = mean s Q[c]
    gemm(g->Xc[l + 1].p, 2 * H, 1, th + net->oV[l], 1, H, g->Q.p, H, m, H, H, nullptr, false, 0, s);
    edge_mean(g->v_off, g->v_enc, g->Q.p, H, g->deg_inv.p, nullptr, g->Xv[l].p + H, 2 * H, n, s);
    // h_v' = relu([h_v, q_v] Wv^T + bv)
    gemm(g->Xv[l].p, 2 * H, 1, th + net->oWv[l], 1, 2 * H, g->Xv[l + 1].p, 2 * H, n, H, 2 * H, th + net->obv[l], true,
         0, s);
  }
  if (n > 0)
    head_kernel<<<(n + 255) / 256, 256, 0, s>>>(g->Xv[net->layers].p, 2 * H, th + net->ow, th + net->ob, g->z.p,
                                                g->mu.p, n);
  MCKL();
  return AFS_OK;
}

static int mpnn_backward(afs_mpnn* net, afs::Graph* g, cudaStream_t s) {
  using namespace afs;
  const float* th = net->theta.p;
  float* gr = net->grad.p;
  const int n = g->n, m = g->m, L = net->layers;
  MCK(cudaMemsetAsync(gr, 0, sizeof(float) * net->n_params, s));
  float* ws = g->wslices.p;
  float* pt = g->part.p;
  // head: gw = sum_v dz_v h_v, gb = sum_v dz_v, dh_v = dz_v w
  colsum(g->Xv[L].p, 2 * H, n, gr + net->ow, pt, s, g->dz.p);
  vsum(g->dz.p, nullptr, n, gr + net->ob, true, pt, s);
  if (n > 0)
    head_dh_kernel<<<static_cast<unsigned>((static_cast<long long>(n) * H + 255) / 256), 256, 0, s>>>(
        g->dz.p, th + net->ow, g->dhv.p, n);
  MCK(cudaMemsetAsync(g->dhc.p, 0, sizeof(float) * static_cast<size_t>(m) * H, s));
  for (int l = L - 1; l >= 0; --l) {
    // variable update: h_v' = relu(Xv Wv^T + bv)
    copy_mask(g->dhv.p, H, g->Xv[l + 1].p, 2 * H, g->dpre_v.p, H, n, s);
    gemm(g->dpre_v.p, 1, H, g->Xv[l].p, 2 * H, 1, gr + net->oWv[l], 2 * H, H, 2 * H, n, nullptr, false, 2, s, ws);
    colsum(g->dpre_v.p, H, n, gr + net->obv[l], pt, s);
    gemm(g->dpre_v.p, H, 1, th + net->oWv[l], 2 * H, 1, g->dXv.p, 2 * H, n, 2 * H, H, nullptr, false, 0, s);
    // q_v = mean_{e at v} s Q[c]  ->  dQ[c] = sum_{e in c} s dq[v] / deg_v
    edge_mean(g->c_off, g->c_enc, g->dXv.p + H, 2 * H, nullptr, g->deg_inv.p, g->dQ.p, H, m, s);
    // Q = h_c' V^T
    gemm(g->dQ.p, 1, H, g->Xc[l + 1].p, 2 * H, 1, gr + net->oV[l], H, H, H, m, nullptr, false, 2, s, ws);
    gemm(g->dQ.p, H, 1, th + net->oV[l], H, 1, g->dhc.p, H, m, H, H, nullptr, false, 1, s);
    // constraint update: h_c' = relu(Xc Wc^T + bc)
    copy_mask(g->dhc.p, H, g->Xc[l + 1].p, 2 * H, g->dpre_c.p, H, m, s);
    gemm(g->dpre_c.p, 1, H, g->Xc[l].p, 2 * H, 1, gr + net->oWc[l], 2 * H, H, 2 * H, m, nullptr, false, 2, s, ws);
    colsum(g->dpre_c.p, H, m, gr + net->obc[l], pt, s);
    gemm(g->dpre_c.p, H, 1, th + net->oWc[l], 2 * H, 1, g->dXc.p, 2 * H, m, 2 * H, H, nullptr, false, 0, s);
    copy_mask(g->dXc.p, 2 * H, nullptr, 0, g->dhc.p, H, m, s);
    // m_c = mean_{e in c} s P[v]  ->  dP[v] = sum_{e at v} s dm[c] / k_c
    edge_mean(g->v_off, g->v_enc, g->dXc.p + H, 2 * H, nullptr, g->k_inv.p, g->dP.p, H, n, s);
    // P = h_v U^T
    gemm(g->dP.p, 1, H, g->Xv[l].p, 2 * H, 1, gr + net->oU[l], H, H, H, n, nullptr, false, 2, s, ws);
    copy_mask(g->dXv.p, 2 * H, nullptr, 0, g->dhv.p, H, n, s);
    gemm(g->dP.p, H, 1, th + net->oU[l], H, 1, g->dhv.p, H, n, H, H, nullptr, false, 1, s);
  }
  // embeddings
  copy_mask(g->dhv.p, H, g->Xv[0].p, 2 * H, g->dpre_v.p, H, n, s);
  gemm(g->dpre_v.p, 1, H, g->fv.p, FV, 1, gr + net->oAv, FV, H, FV, n, nullptr, false, 2, s, ws);
  colsum(g->dpre_v.p, H, n, gr + net->oav, pt, s);
  copy_mask(g->dhc.p, H, g->Xc[0].p, 2 * H, g->dpre_c.p, H, m, s);
  gemm(g->dpre_c.p, 1, H, g->fc.p, FC, 1, gr + net->oAc, FC, H, FC, m, nullptr, false, 2, s, ws);
  colsum(g->dpre_c.p, H, m, gr + net->oac, pt, s);
  MCKL();
  return AFS_OK;
}

extern "C" {

int afs_mpnn_create(int32_t hidden, int32_t layers, uint64_t seed, afs_mpnn** out) {
  if (!out) return afs::set_error(AFS_E_ARG, "out is NULL");
  *out = nullptr;
  if (hidden != H) return afs::set_error(AFS_E_ARG, "hidden width must be %d", H);
  if (layers < 1 || layers > 8) return afs::set_error(AFS_E_ARG, "layers must be 1..8");
  afs_mpnn* net = new afs_mpnn();
  net->layers = layers;
  net->n_params = layout(net);
  // He-uniform weights (fan-in), zero biases; host RNG seeded by `seed`
  std::vector<float> th(net->n_params, 0.f);
  std::mt19937_64 rng(seed);
  auto fill = [&](long long off, int rows, int fan_in) {
    const float a = std::sqrt(6.0f / static_cast<float>(fan_in));
    std::uniform_real_distribution<float> d(-a, a);
    for (long long i = 0; i < static_cast<long long>(rows) * fan_in; ++i) th[off + i] = d(rng);
  };
  fill(net->oAv, H, afs::FV);
  fill(net->oAc, H, afs::FC);
  for (int l = 0; l < layers; ++l) {
    fill(net->oU[l], H, H);
    fill(net->oV[l], H, H);
    fill(net->oWc[l], H, 2 * H);
    fill(net->oWv[l], H, 2 * H);
  }
  fill(net->ow, 1, H);
  cudaError_t e = net->theta.upload(th, nullptr);
  if (e == cudaSuccess) e = net->grad.alloc(net->n_params);
  if (e == cudaSuccess) e = net->m1.alloc(net->n_params);
  if (e == cudaSuccess) e = net->m2.alloc(net->n_params);
  if (e == cudaSuccess) e = cudaMemset(net->m1.p, 0, sizeof(float) * net->n_params);
  if (e == cudaSuccess) e = cudaMemset(net->m2.p, 0, sizeof(float) * net->n_params);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    delete net;
    return afs::set_error(AFS_E_CUDA, "mpnn create: %s", cudaGetErrorString(e));
  }
  *out = net;
  return AFS_OK;
}

void afs_mpnn_free(afs_mpnn* net) { delete net; }

int afs_mpnn_num_params(const afs_mpnn* net, int64_t* n) {
  if (!net || !n) return afs::set_error(AFS_E_ARG, "NULL argument");
  *n = net->n_params;
  return AFS_OK;
}

int afs_mpnn_get_params(afs_mpnn* net, float* theta_dev, void* stream) {
  if (!net || !theta_dev) return afs::set_error(AFS_E_ARG, "NULL argument");
  MCK(cudaMemcpyAsync(theta_dev, net->theta.p, sizeof(float) * net->n_params, cudaMemcpyDeviceToDevice,
                      static_cast<cudaStream_t>(stream)));
  return AFS_OK;
}

int afs_mpnn_set_params(afs_mpnn* net, const float* theta_dev, void* stream) {
  if (!net || !theta_dev) return afs::set_error(AFS_E_ARG, "NULL argument");
  MCK(cudaMemcpyAsync(net->theta.p, theta_dev, sizeof(float) * net->n_params, cudaMemcpyDeviceToDevice,
                      static_cast<cudaStream_t>(stream)));
  return AFS_OK;
}

int afs_mpnn_forward(afs_mpnn* net, afs_handle* h, float* mu_dev, void* stream) {
  if (!net || !h) return afs::set_error(AFS_E_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  afs::Graph* g = nullptr;
  int rc = bind(net, h, s, &g);
  if (rc) return rc;
  rc = mpnn_forward(net, g, s);
  if (rc) return rc;
  if (mu_dev && g->n > 0)
    MCK(cudaMemcpyAsync(mu_dev, g->mu.p, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
  return AFS_OK;
}

int afs_mpnn_loss_grad(afs_mpnn* net, afs_handle* h, const float* y_dev, const float* w_dev, float* grad_dev,
                       float* loss_host, void* stream) {
  if (!net || !h || !y_dev) return afs::set_error(AFS_E_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  afs::Graph* g = nullptr;
  int rc = bind(net, h, s, &g);
  if (rc) return rc;
  rc = mpnn_forward(net, g, s);
  if (rc) return rc;
  // the label-mask sum and the loss are fixed-order device reductions
  if (w_dev) afs::vsum(w_dev, nullptr, g->n, g->wsum.p, false, g->part.p, s);
  if (g->n > 0)
    afs::loss_kernel<<<(g->n + 255) / 256, 256, 0, s>>>(g->z.p, y_dev, w_dev, g->wsum.p, g->dz.p, g->lterm.p, g->n);
  afs::vsum(g->lterm.p, nullptr, g->n, g->loss.p, false, g->part.p, s);
  MCKL();
  rc = mpnn_backward(net, g, s);
  if (rc) return rc;
  if (grad_dev)
    MCK(cudaMemcpyAsync(grad_dev, net->grad.p, sizeof(float) * net->n_params, cudaMemcpyDeviceToDevice, s));
  if (loss_host) {
    MCK(cudaMemcpyAsync(loss_host, g->loss.p, sizeof(float), cudaMemcpyDeviceToHost, s));
    MCK(cudaStreamSynchronize(s));
  }
  return AFS_OK;
}

int afs_mpnn_adam_step(afs_mpnn* net, float lr, void* stream) {
  if (!net) return afs::set_error(AFS_E_ARG, "NULL argument");
  net->t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float bc1 = 1.0f - std::pow(b1, static_cast<float>(net->t));
  const float bc2 = 1.0f - std::pow(b2, static_cast<float>(net->t));
  const long long n = net->n_params;
  afs::adam_kernel<<<static_cast<unsigned>((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      net->theta.p, net->grad.p, net->m1.p, net->m2.p, n, lr, b1, b2, 1e-8f, bc1, bc2);
  MCKL();
  return AFS_OK;
}

int afs_mpnn_init_restarts(afs_mpnn* net, afs_handle* h, int32_t B, uint64_t seed, float uniform_frac,
                           float sigma_min, float sigma_max, void* stream) {
  if (!net || !h) return afs::set_error(AFS_E_ARG, "NULL argument");
  if (uniform_frac < 0.f || uniform_frac > 1.f) return afs::set_error(AFS_E_ARG, "uniform_frac must be in [0, 1]");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  afs::GraphView gv{};
  int rc = afs::graph_view(h, &gv);
  if (rc) return rc;
  if (gv.B != B || gv.x == nullptr) return afs::set_error(AFS_E_STATE, "afs_init_restarts(B) must come first");
  afs::Graph* g = nullptr;
  rc = bind(net, h, s, &g);
  if (rc) return rc;
  rc = mpnn_forward(net, g, s);
  if (rc) return rc;
  const int B_learn = static_cast<int>(std::lround((1.0f - uniform_frac) * B));
  const long long total = static_cast<long long>(gv.n) * B;
  if (total > 0) {
    const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
    if (gv.xt == afs::XT_F32)
      afs::sample_kernel<float><<<blocks, 256, 0, s>>>(g->mu.p, static_cast<float*>(gv.x), gv.pitch, gv.n, B, B_learn,
                                                       sigma_min, sigma_max, seed);
    else
      afs::sample_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(g->mu.p, static_cast<__nv_bfloat16*>(gv.x), gv.pitch,
                                                               gv.n, B, B_learn, sigma_min, sigma_max, seed);
  }
  MCKL();
  return afs::state_written(h, s);
}

int afs_mpnn_nudge_restarts(afs_mpnn* net, afs_handle* h, float alpha_min, float alpha_max, void* stream) {
  if (!net || !h) return afs::set_error(AFS_E_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  afs::GraphView gv{};
  int rc = afs::graph_view(h, &gv);
  if (rc) return rc;
  if (gv.B <= 0 || gv.x == nullptr) return afs::set_error(AFS_E_STATE, "afs_init_restarts must come first");
  afs::Graph* g = nullptr;
  rc = bind(net, h, s, &g);
  if (rc) return rc;
  rc = mpnn_forward(net, g, s);
  if (rc) return rc;
  const long long total = static_cast<long long>(gv.n) * gv.B;
  if (total > 0) {
    const unsigned blocks = static_cast<unsigned>((total + 255) / 256);
    if (gv.xt == afs::XT_F32)
      afs::nudge_kernel<float><<<blocks, 256, 0, s>>>(g->mu.p, static_cast<float*>(gv.x), gv.pitch, gv.n, gv.B,
                                                      alpha_min, alpha_max);
    else
      afs::nudge_kernel<__nv_bfloat16><<<blocks, 256, 0, s>>>(g->mu.p, static_cast<__nv_bfloat16*>(gv.x), gv.pitch,
                                                              gv.n, gv.B, alpha_min, alpha_max);
  }
  MCKL();
  return afs::state_written(h, s);
}

}  // extern "C"
