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

}  // namespace ofdm
