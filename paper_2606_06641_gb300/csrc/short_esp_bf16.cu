// Dispatch of the short FE+gradient kernel: paper's elementary-symmetric basis, BF16 state.
#include "fe_short.cuh"

namespace afs {

template <int K>
static bool dispatch_rpl(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s) {
  if (rpl == 1) {
    launch_short_k<K, 1, __nv_bfloat16, true>(a, warps, s);
    return true;
  }
  if constexpr (K <= 16 && false) {
    if (rpl == 2) {
      launch_short_k<K, 2, __nv_bfloat16, true>(a, warps, s);
      return true;
    }
  }
  if constexpr (K <= 8 && false) {
    if (rpl == 4) {
      launch_short_k<K, 4, __nv_bfloat16, true>(a, warps, s);
      return true;
    }
  }
  return false;
}

bool launch_short_esp_bf16(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s) {
  switch (a.k) {
    case 1: return dispatch_rpl<1>(a, rpl, warps, s);
    case 2: return dispatch_rpl<2>(a, rpl, warps, s);
    case 3: return dispatch_rpl<3>(a, rpl, warps, s);
    case 4: return dispatch_rpl<4>(a, rpl, warps, s);
    case 5: return dispatch_rpl<5>(a, rpl, warps, s);
    case 6: return dispatch_rpl<6>(a, rpl, warps, s);
    case 7: return dispatch_rpl<7>(a, rpl, warps, s);
    case 8: return dispatch_rpl<8>(a, rpl, warps, s);
    case 9: return dispatch_rpl<9>(a, rpl, warps, s);
    case 10: return dispatch_rpl<10>(a, rpl, warps, s);
    case 11: return dispatch_rpl<11>(a, rpl, warps, s);
    case 12: return dispatch_rpl<12>(a, rpl, warps, s);
    case 13: return dispatch_rpl<13>(a, rpl, warps, s);
    case 14: return dispatch_rpl<14>(a, rpl, warps, s);
    case 15: return dispatch_rpl<15>(a, rpl, warps, s);
    case 16: return dispatch_rpl<16>(a, rpl, warps, s);
    case 17: return dispatch_rpl<17>(a, rpl, warps, s);
    case 18: return dispatch_rpl<18>(a, rpl, warps, s);
    case 19: return dispatch_rpl<19>(a, rpl, warps, s);
    case 20: return dispatch_rpl<20>(a, rpl, warps, s);
    case 21: return dispatch_rpl<21>(a, rpl, warps, s);
    case 22: return dispatch_rpl<22>(a, rpl, warps, s);
    case 23: return dispatch_rpl<23>(a, rpl, warps, s);
    case 24: return dispatch_rpl<24>(a, rpl, warps, s);
    case 25: return dispatch_rpl<25>(a, rpl, warps, s);
    case 26: return dispatch_rpl<26>(a, rpl, warps, s);
    case 27: return dispatch_rpl<27>(a, rpl, warps, s);
    case 28: return dispatch_rpl<28>(a, rpl, warps, s);
    case 29: return dispatch_rpl<29>(a, rpl, warps, s);
    case 30: return dispatch_rpl<30>(a, rpl, warps, s);
    case 31: return dispatch_rpl<31>(a, rpl, warps, s);
    case 32: return dispatch_rpl<32>(a, rpl, warps, s);
    default: return false;
  }
}

}  // namespace afs
