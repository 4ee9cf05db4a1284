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
// mirrors the forward; Adam keeps FP32 moments.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

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
  int mode;  // 0: C = r, 1: C += r, 2: atomicAdd(C, r)
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
          float* dst = g.C + row * g.ldc + col;
          if (g.mode == 2) {
            atomicAdd(dst, v);
          } else {
            if (g.bias) v += g.bias[col];
            if (g.relu) v = fmaxf(v, 0.f);
            *dst = g.mode == 1 ? *dst + v : v;
          }
        }
      }
    }
  }
}

void gemm(const float* A, long long sa0, long long sa1, const float* B, long long sb0, long long sb1, float* C,
          long long ldc, int M, int N, int K, const float* bias, bool relu, int mode, cudaStream_t s) {
  if (M <= 0 || N <= 0 || K <= 0) return;  // empty product (weight gradients of an empty graph stay zero)
  GemmArgs g{A, sa0, sa1, B, sb0, sb1, C, ldc, M, N, K, bias, relu ? 1 : 0, mode, K};
  int zsplit = 1;
  if (mode == 2) {  // weight gradients: split the long inner dimension over CTAs
    g.k_split = 1024;
    zsplit = (K + g.k_split - 1) / g.k_split;
  }
  dim3 grid((M + 63) / 64, (N + 63) / 64, zsplit);
  gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
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

// out[j] += sum_r x[r*ld + j] (column sums of a rows x 64 block)
__global__ void colsum_kernel(const float* x, long long ld, int rows, float* out) {
  const int j = threadIdx.x;  // 64 columns
  float acc = 0.f;
  for (int r = blockIdx.x * blockDim.y + threadIdx.y; r < rows; r += gridDim.x * blockDim.y) acc += x[r * ld + j];
  __shared__ float part[4][H];
  part[threadIdx.y][j] = acc;
  __syncthreads();
  if (threadIdx.y == 0) atomicAdd(out + j, part[0][j] + part[1][j] + part[2][j] + part[3][j]);
}

void colsum(const float* x, long long ld, int rows, float* out, cudaStream_t s) {
  if (rows <= 0) return;
  const int blocks = std::min(256, (rows + 3) / 4);
  colsum_kernel<<<blocks, dim3(H, 4), 0, s>>>(x, ld, rows, out);
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

// loss += sum_v w_v (softplus(t) - y t) / wsum with t = -2 z; dz = -2 w (sigmoid(t) - y) / wsum
__global__ void loss_kernel(const float* z, const float* y, const float* wm, float inv_wsum, float* dz, float* loss,
                            int n) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (v < n) {
    const float t = -2.f * z[v];
    const float wv = wm ? wm[v] : 1.f;
    const float sp = fmaxf(t, 0.f) + log1pf(expf(-fabsf(t)));
    l = wv * (sp - y[v] * t) * inv_wsum;
    const float sig = 1.f / (1.f + expf(-t));
    dz[v] = -2.f * wv * (sig - y[v]) * inv_wsum;
  }
  for (int o = 16; o >= 1; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l);
}

// dh[v][j] = dz[v] w[j]; gw[j] += sum_v dz[v] h[v][j]; gb += sum_v dz[v]
__global__ void head_bwd_kernel(const float* dz, const float* hv, long long ld, const float* w, float* dh, float* gw,
                                float* gb, int n) {
  const int j = threadIdx.x;
  float acc = 0.f, accb = 0.f;
  for (int v = blockIdx.x * blockDim.y + threadIdx.y; v < n; v += gridDim.x * blockDim.y) {
    const float d = dz[v];
    dh[v * H + j] = d * w[j];
    acc = fmaf(d, hv[v * ld + j], acc);
    if (j == 0) accb += d;
  }
  atomicAdd(gw + j, acc);
  if (j == 0) atomicAdd(gb, accb);
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

struct Graph {
  int n = 0, m = 0, layers = 0;
  Dev<int> c_off, c_enc, v_off, v_enc;
  Dev<float> k_inv, deg_inv, fv, fc;
  std::vector<Dev<float>> Xv, Xc;  // layers + 1 each: [n x 128], [m x 128]
  Dev<float> P, Q, z, mu, dz, dhv, dhc, dpre_v, dpre_c, dXv, dXc, dP, dQ, loss;
};

void release_graph(void* p) { delete static_cast<Graph*>(p); }

int bind_graph(afs_handle* h, int layers, cudaStream_t s, Graph** out) {
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
  const int n = gv.n, m = gv.m;
  const long long E = gv.lit_off[m];
  std::vector<int> c_off(gv.lit_off, gv.lit_off + m + 1), c_enc(gv.lit_enc, gv.lit_enc + E);
  std::vector<int> v_off(n + 1, 0), v_enc(E);
  std::vector<float> k_inv(m), deg_inv(n), fv(static_cast<size_t>(n) * FV, 0.f), fc(static_cast<size_t>(m) * FC, 0.f);
  std::vector<float> bal(n, 0.f);
  for (long long e = 0; e < E; ++e) {
    const int v = gv.lit_enc[e] >> 1;
    v_off[v + 1]++;
    bal[v] += (gv.lit_enc[e] & 1) ? -1.f : 1.f;
  }
  for (int v = 0; v < n; ++v) v_off[v + 1] += v_off[v];
  {
    std::vector<int> fill(v_off.begin(), v_off.end() - 1);
    for (int c = 0; c < m; ++c)
      for (int e = gv.lit_off[c]; e < gv.lit_off[c + 1]; ++e) {
        const int v = gv.lit_enc[e] >> 1;
        v_enc[fill[v]++] = (c << 1) | (gv.lit_enc[e] & 1);
      }
  }
  for (int v = 0; v < n; ++v) {
    const float deg = static_cast<float>(v_off[v + 1] - v_off[v]);
    deg_inv[v] = deg > 0 ? 1.f / deg : 0.f;
    fv[static_cast<size_t>(v) * FV + 0] = deg / 8.f;
    fv[static_cast<size_t>(v) * FV + 1] = bal[v] / std::max(deg, 1.f);
    fv[static_cast<size_t>(v) * FV + 2] = 1.f;
  }
  for (int c = 0; c < m; ++c) {
    const float k = static_cast<float>(gv.lit_off[c + 1] - gv.lit_off[c]);
    k_inv[c] = k > 0 ? 1.f / k : 0.f;
    float* f = &fc[static_cast<size_t>(c) * FC];
    f[gv.ctype[c]] = 1.f;
    f[7] = k / 8.f;
    f[8] = (gv.ctype[c] == AFS_EK || gv.ctype[c] == AFS_CARD) ? gv.cparam[c] / std::max(k, 1.f) : 0.f;
    f[9] = gv.ctype[c] == AFS_XOR ? static_cast<float>(gv.cparity[c]) : 0.f;
    f[10] = gv.ctype[c] == AFS_CARD ? static_cast<float>(gv.cop[c]) : 0.f;
    f[11] = 1.f;
  }
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (x != cudaSuccess && e == cudaSuccess) e = x;
  };
  chk(g->c_off.upload(c_off, s));
  chk(g->c_enc.upload(c_enc, s));
  chk(g->v_off.upload(v_off, s));
  chk(g->v_enc.upload(v_enc, s));
  chk(g->k_inv.upload(k_inv, s));
  chk(g->deg_inv.upload(deg_inv, s));
  chk(g->fv.upload(fv, s));
  chk(g->fc.upload(fc, s));
  g->Xv.resize(layers + 1);
  g->Xc.resize(layers + 1);
  for (int l = 0; l <= layers; ++l) {
    chk(g->Xv[l].alloc(static_cast<size_t>(n) * 2 * H));
    chk(g->Xc[l].alloc(static_cast<size_t>(m) * 2 * H));
  }
  const size_t nH = static_cast<size_t>(n) * H, mH = static_cast<size_t>(m) * H;
  chk(g->P.alloc(nH));
  chk(g->Q.alloc(mH));
  chk(g->z.alloc(n));
  chk(g->mu.alloc(n));
  chk(g->dz.alloc(n));
  chk(g->dhv.alloc(nH));
  chk(g->dhc.alloc(mH));
  chk(g->dpre_v.alloc(nH));
  chk(g->dpre_c.alloc(mH));
  chk(g->dXv.alloc(2 * nH));
  chk(g->dXc.alloc(2 * mH));
  chk(g->dP.alloc(nH));
  chk(g->dQ.alloc(mH));
  chk(g->loss.alloc(1));
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    delete g;
    return set_error(AFS_E_CUDA, "mpnn graph buffers: %s", cudaGetErrorString(e));
  }
  set_handle_ext(h, g, release_graph);
  *out = g;
  return AFS_OK;
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
  long long t = 0;
  // offsets into theta
  long long oAv, oav, oAc, oac, ow, ob;
  std::vector<long long> oU, oV, oWc, obc, oWv, obv;
};

using afs::H;

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
  // embeddings into the first halves of the layer-0 inputs
  gemm(g->fv.p, FV, 1, th + net->oAv, 1, FV, g->Xv[0].p, 2 * H, n, H, FV, th + net->oav, true, 0, s);
  gemm(g->fc.p, FC, 1, th + net->oAc, 1, FC, g->Xc[0].p, 2 * H, m, H, FC, th + net->oac, true, 0, s);
  for (int l = 0; l < net->layers; ++l) {
    // P = h_v U^T; m_c = mean s P[v]
    gemm(g->Xv[l].p, 2 * H, 1, th + net->oU[l], 1, H, g->P.p, H, n, H, H, nullptr, false, 0, s);
    edge_mean(g->c_off.p, g->c_enc.p, g->P.p, H, g->k_inv.p, nullptr, g->Xc[l].p + H, 2 * H, m, s);
    // h_c' = relu([h_c, m_c] Wc^T + bc)
    gemm(g->Xc[l].p, 2 * H, 1, th + net->oWc[l], 1, 2 * H, g->Xc[l + 1].p, 2 * H, m, H, 2 * H, th + net->obc[l], true,
         0, s);
    // Q = h_c' V^T; q_v = mean s Q[c]
    gemm(g->Xc[l + 1].p, 2 * H, 1, th + net->oV[l], 1, H, g->Q.p, H, m, H, H, nullptr, false, 0, s);
    edge_mean(g->v_off.p, g->v_enc.p, g->Q.p, H, g->deg_inv.p, nullptr, g->Xv[l].p + H, 2 * H, n, s);
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
  if (n > 0)
    head_bwd_kernel<<<std::min(256, (n + 3) / 4), dim3(H, 4), 0, s>>>(g->dz.p, g->Xv[L].p, 2 * H, th + net->ow,
                                                                       g->dhv.p, gr + net->ow, gr + net->ob, n);
  MCK(cudaMemsetAsync(g->dhc.p, 0, sizeof(float) * static_cast<size_t>(m) * H, s));
  for (int l = L - 1; l >= 0; --l) {
    // variable update: h_v' = relu(Xv Wv^T + bv)
    copy_mask(g->dhv.p, H, g->Xv[l + 1].p, 2 * H, g->dpre_v.p, H, n, s);
    gemm(g->dpre_v.p, 1, H, g->Xv[l].p, 2 * H, 1, gr + net->oWv[l], 2 * H, H, 2 * H, n, nullptr, false, 2, s);
    colsum(g->dpre_v.p, H, n, gr + net->obv[l], s);
    gemm(g->dpre_v.p, H, 1, th + net->oWv[l], 2 * H, 1, g->dXv.p, 2 * H, n, 2 * H, H, nullptr, false, 0, s);
    // q_v = mean_{e at v} s Q[c]  ->  dQ[c] = sum_{e in c} s dq[v] / deg_v
    edge_mean(g->c_off.p, g->c_enc.p, g->dXv.p + H, 2 * H, nullptr, g->deg_inv.p, g->dQ.p, H, m, s);
    // Q = h_c' V^T
    gemm(g->dQ.p, 1, H, g->Xc[l + 1].p, 2 * H, 1, gr + net->oV[l], H, H, H, m, nullptr, false, 2, s);
    gemm(g->dQ.p, H, 1, th + net->oV[l], H, 1, g->dhc.p, H, m, H, H, nullptr, false, 1, s);
    // constraint update: h_c' = relu(Xc Wc^T + bc)
    copy_mask(g->dhc.p, H, g->Xc[l + 1].p, 2 * H, g->dpre_c.p, H, m, s);
    gemm(g->dpre_c.p, 1, H, g->Xc[l].p, 2 * H, 1, gr + net->oWc[l], 2 * H, H, 2 * H, m, nullptr, false, 2, s);
    colsum(g->dpre_c.p, H, m, gr + net->obc[l], s);
    gemm(g->dpre_c.p, H, 1, th + net->oWc[l], 2 * H, 1, g->dXc.p, 2 * H, m, 2 * H, H, nullptr, false, 0, s);
    copy_mask(g->dXc.p, 2 * H, nullptr, 0, g->dhc.p, H, m, s);
    // m_c = mean_{e in c} s P[v]  ->  dP[v] = sum_{e at v} s dm[c] / k_c
    edge_mean(g->v_off.p, g->v_enc.p, g->dXc.p + H, 2 * H, nullptr, g->k_inv.p, g->dP.p, H, n, s);
    // P = h_v U^T
    gemm(g->dP.p, 1, H, g->Xv[l].p, 2 * H, 1, gr + net->oU[l], H, H, H, n, nullptr, false, 2, s);
    copy_mask(g->dXv.p, 2 * H, nullptr, 0, g->dhv.p, H, n, s);
    gemm(g->dP.p, H, 1, th + net->oU[l], H, 1, g->dhv.p, H, n, H, H, nullptr, false, 1, s);
  }
  // embeddings
  copy_mask(g->dhv.p, H, g->Xv[0].p, 2 * H, g->dpre_v.p, H, n, s);
  gemm(g->dpre_v.p, 1, H, g->fv.p, FV, 1, gr + net->oAv, FV, H, FV, n, nullptr, false, 2, s);
  colsum(g->dpre_v.p, H, n, gr + net->oav, s);
  copy_mask(g->dhc.p, H, g->Xc[0].p, 2 * H, g->dpre_c.p, H, m, s);
  gemm(g->dpre_c.p, 1, H, g->fc.p, FC, 1, gr + net->oAc, FC, H, FC, m, nullptr, false, 2, s);
  colsum(g->dpre_c.p, H, m, gr + net->oac, s);
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
  int rc = afs::bind_graph(h, net->layers, s, &g);
  if (rc) return rc;
  rc = mpnn_forward(net, g, s);
  if (rc) return rc;
  if (mu_dev && g->n > 0)
    MCK(cudaMemcpyAsync(mu_dev, g->mu.p, sizeof(float) * g->n, cudaMemcpyDeviceToDevice, s));
  return AFS_OK;
}

int afs_mpnn_loss_grad(afs_mpnn* net, afs_handle* h, const float* y_dev, const float* w_dev, float wsum,
                       float* grad_dev, float* loss_host, void* stream) {
  if (!net || !h || !y_dev) return afs::set_error(AFS_E_ARG, "NULL argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  afs::Graph* g = nullptr;
  int rc = afs::bind_graph(h, net->layers, s, &g);
  if (rc) return rc;
  rc = mpnn_forward(net, g, s);
  if (rc) return rc;
  MCK(cudaMemsetAsync(g->loss.p, 0, sizeof(float), s));
  const float inv = 1.0f / (wsum > 1.0f ? wsum : 1.0f);
  if (g->n > 0)
    afs::loss_kernel<<<(g->n + 255) / 256, 256, 0, s>>>(g->z.p, y_dev, w_dev, inv, g->dz.p, g->loss.p, g->n);
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
  rc = afs::bind_graph(h, net->layers, s, &g);
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

}  // extern "C"
