// Persistent step kernel: one cooperative launch runs S whole steps of
// Algorithm 1 (exact check, FE + gradient, projected step) for every instance
// and restart of a handle whose constraints are all short (k <= 32).
//
// A step is two phases over flat work lists, separated by a grid barrier:
//   A: the per-step check of the state read (one unit per constraint range
//      and 32 words of restarts), the FE + gradient of every short length
//      bucket (one unit per constraint and 32 restarts) and the fused
//      3-literal derivative sums (one unit per variable and 128 restarts);
//   B: the CSR gather and projected update (one unit per variable and 128
//      restarts), which also writes the sign words the next check reads.
// Every warp strides over the units of a phase, so one launch replaces the
// six or more dependent launches of a step and the graph's per-node latency
// that dominates small restart counts. The barrier's waits are bounded: on
// expiry the kernel records AFS_E_TIMEOUT in the handle's error word and
// returns. Data written earlier in the launch is read with L2-coherent loads.
#include <cuda_bf16.h>

#include "afsat.h"
#include "afsat_internal.h"
#include "bulk_copy.cuh"
#include "fe_short.cuh"
#include "step_units.cuh"

namespace afs {

namespace {

constexpr int PWARPS = PERSIST_WARPS;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier over all (co-resident) blocks: bar[0] counts arrivals,
// bar[1] is the generation. The last block to arrive resets the count and
// advances the generation; the others wait for the generation to move, for at
// most `limit` SM cycles. Returns false (error word set) if a wait gave up.
__device__ bool grid_barrier(unsigned* bar, unsigned& gen, long long limit, int* err) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();  // this block's writes before the arrival
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_gpu(bar + 1) == gen) {
        if (clock64() - t0 > limit) {
          atomicExch(err, DEV_ERR_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    gen += 1;
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

template <typename XT, int K>
__device__ __forceinline__ void short_unit_k(const FeGroupArgs& f, long long u, int lane) {
  short_unit<K, 1, XT, false, false, true>(f, u, lane);
}

// FE + gradient unit of a short group of length k (runtime) for state type XT
template <typename XT>
__device__ void short_unit_any(const FeGroupArgs& f, long long u, int lane) {
  switch (f.k) {
#define AFS_K(K)                     \
  case K:                            \
    short_unit_k<XT, K>(f, u, lane); \
    break;
    AFS_K(1) AFS_K(2) AFS_K(3) AFS_K(4) AFS_K(5) AFS_K(6) AFS_K(7) AFS_K(8) AFS_K(9) AFS_K(10) AFS_K(11) AFS_K(12)
    AFS_K(13) AFS_K(14) AFS_K(15) AFS_K(16) AFS_K(17) AFS_K(18) AFS_K(19) AFS_K(20) AFS_K(21) AFS_K(22) AFS_K(23)
    AFS_K(24) AFS_K(25) AFS_K(26) AFS_K(27) AFS_K(28) AFS_K(29) AFS_K(30) AFS_K(31) AFS_K(32)
#undef AFS_K
    default:
      break;
  }
}

template <typename XT>
__global__ void __launch_bounds__(PWARPS * 32, 2) step_persistent_kernel(PersistArgs a) {
  __shared__ unsigned stage[PWARPS][CHECK_STAGE * 32];
  __shared__ PersistGroup grp[PERSIST_MAX_GROUPS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < a.ng; i += blockDim.x) grp[i] = a.groups[i];
  unsigned gen = 0;
  if (threadIdx.x == 0) gen = ld_acquire_gpu(a.bar + 1);  // no barrier can complete before every block arrives
  __syncthreads();
  const long long limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
  const unsigned nwarps = gridDim.x * PWARPS;
  // warps numbered across blocks first: consecutive units (the costliest
  // come first) land on different SMs instead of sharing one SM's schedulers
  const unsigned gw = wib * gridDim.x + blockIdx.x;
  const unsigned tiles128 = static_cast<unsigned>((a.B + 127) >> 7);
  for (int t = 0; t < a.nsteps; ++t) {
    const int p = (a.parity0 + t) & 1;
    const void* x = p ? a.xb1 : a.xb0;
    void* xo = p ? a.xb0 : a.xb1;
    unsigned* vcur = p ? a.vw1 : a.vw0;
    unsigned* vnext = p ? a.vw0 : a.vw1;
    // ---- phase A: check, FE buckets, fused sums (all read x_t) ----
    // units are numbered by decreasing expected cost; warp gw takes units
    // gw, 2N - 1 - gw, 2N + gw, ... (N warps), so the costliest share a warp
    // with the cheapest
    for (unsigned r = 0; r * nwarps < a.a_units; ++r) {
      const unsigned u = (r & 1) ? (r + 1) * nwarps - 1 - gw : r * nwarps + gw;
      if (u >= a.a_units) continue;  // uniform per warp
      if (u - a.fus0 < a.fus_units) {
        const unsigned task = u - a.fus0;
        const unsigned vl = task / tiles128;
        CsrArgs c = a.fus;
        c.x = x;
        const int v = static_cast<int>(vl);
        const int bl = static_cast<int>(task - vl * tiles128) * 128 + lane * 4;
        const bool act = bl < a.B;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        fused_sum_pf<XT, FUSED_PF_BATCH, false, true>(c, v, act ? bl : 0, act, lane, acc);
        if (act) *reinterpret_cast<float4*>(c.gf + static_cast<long long>(v) * c.gf_pitch + bl) =
                     make_float4(acc[0], acc[1], acc[2], acc[3]);
      } else if (u - a.chk0 < a.chk_units) {
        if (a.check) {
          CheckArgs c = a.chk;
          c.vword = vcur;
          const unsigned t = u - a.chk0;
          if (a.chk_wide)
            check_wide_unit<true>(c, static_cast<int>(t / a.chk_chunks), static_cast<int>(t % a.chk_chunks), lane,
                                  stage[wib]);
          else
            check_unit_warp<true>(c, static_cast<int>(t / a.chk_chunks), static_cast<int>(t % a.chk_chunks), lane,
                                  stage[wib]);
        }
      } else {
        int g = 0;
        while (g + 1 < a.ng && u - grp[g].unit0 >= grp[g].units) ++g;
        FeGroupArgs f = a.fe;
        f.x = x;
        f.k = grp[g].k;
        f.c_begin = grp[g].c_begin;
        f.c_count = grp[g].c_count;
        f.lit_base = grp[g].lit_base;
        short_unit_any<XT>(f, static_cast<long long>(u - grp[g].unit0), lane);
      }
    }
    if (!grid_barrier(a.bar, gen, limit, a.err)) return;
    // ---- phase B: CSR gather and projected step into x_{t+1} ----
    {
      CsrArgs c = a.csr;
      c.x = x;
      c.x_out = xo;
      c.vcur = a.check ? vcur : nullptr;
      c.vnext = vnext;
      for (unsigned u = gw; u < a.csr_units; u += nwarps) {
        const unsigned vl = u / tiles128;
        csr_vec4_task<XT, false, true>(c, static_cast<int>(vl), static_cast<int>(u - vl * tiles128), lane);
      }
    }
    if (!grid_barrier(a.bar, gen, limit, a.err)) return;
  }
}

template <typename XT>
int resident(int dev_sms) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, step_persistent_kernel<XT>, PWARPS * 32, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per * dev_sms;
}

}  // namespace

int persistent_grid(int xt) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  return xt == XT_F32 ? resident<float>(sms) : resident<__nv_bfloat16>(sms);
}

cudaError_t launch_persistent(const PersistArgs& a, int xt, int blocks, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(blocks));
  cfg.blockDim = dim3(PWARPS * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every block resident at once (the barrier needs it)
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (xt == XT_F32) return cudaLaunchKernelEx(&cfg, step_persistent_kernel<float>, a);
  return cudaLaunchKernelEx(&cfg, step_persistent_kernel<__nv_bfloat16>, a);
}

}  // namespace afs
