// Dispatch of the short FE+gradient kernel (k <= KSHORT) over the length k
// and the restarts per lane, for one state type XT and one basis (ESP: the
// paper's elementary-symmetric basis, one restart per lane). The build
// generates one translation unit per (basis, state type) that defines the
// matching launch_short_<basis>_<type> with launch_short<XT, ESP>, so the
// k x rpl kernel instantiations compile in parallel.
#pragma once
#include <utility>

#include "fe_short.cuh"

namespace afs {

template <typename XT, bool ESP, int K>
bool short_dispatch_rpl(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s) {
  if (rpl == 1) {
    launch_short_k<K, 1, XT, ESP>(a, warps, s);
    return true;
  }
  if constexpr (K <= 16 && !ESP) {
    if (rpl == 2) {
      launch_short_k<K, 2, XT, ESP>(a, warps, s);
      return true;
    }
  }
  if constexpr (K <= 8 && !ESP) {
    if (rpl == 4) {
      launch_short_k<K, 4, XT, ESP>(a, warps, s);
      return true;
    }
  }
  return false;
}

template <typename XT, bool ESP, int... Km1>
bool short_dispatch_k(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s, std::integer_sequence<int, Km1...>) {
  bool ok = false;
  // k = Km1 + 1 for Km1 = 0 .. KSHORT - 1; exactly one term matches
  (void)((a.k == Km1 + 1 ? (ok = short_dispatch_rpl<XT, ESP, Km1 + 1>(a, rpl, warps, s), true) : false) || ...);
  return ok;
}

// false when no kernel exists for (k, rpl)
template <typename XT, bool ESP>
bool launch_short(const FeGroupArgs& a, int rpl, int warps, cudaStream_t s) {
  return short_dispatch_k<XT, ESP>(a, rpl, warps, s, std::make_integer_sequence<int, KSHORT>{});
}

}  // namespace afs
