// keys.cuh -- detection keys shared by the detection kernels.
//
// A key is (float bits of P) << 32 | ~(map index): for P > 0 the larger key is
// the larger power, then the smaller map index (the output order of Eq. (18)'s
// detections); 0 is "no key".
#pragma once
#include <stdint.h>

namespace ofdm {

// Largest key of the warp: the larger power word, then the larger index word.
__device__ __forceinline__ uint64_t warp_max_key(uint64_t v) {
  const unsigned hi = (unsigned)(v >> 32);
  const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
  const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? (unsigned)v : 0u);
  return ((uint64_t)mh << 32) | ml;
}

// Merge of up to 32 key lists, each sorted descending with its first K
// entries valid, list j at src[32 j]: lane r < K receives the r-th largest
// key of all lists (0 when fewer exist).
template <typename P>
__device__ __forceinline__ uint64_t warp_merge_lists(P src, int nlists, int K, int lane) {
  int h = 0;
  uint64_t head = lane < nlists ? src[lane << 5] : 0, out = 0;
  for (int r = 0; r < K; ++r) {
    const uint64_t m = warp_max_key(head);
    if (lane == r) out = m;
    if (m != 0 && head == m) { ++h; head = h < K ? src[(lane << 5) + h] : 0; }
  }
  return out;
}

}  // namespace ofdm
