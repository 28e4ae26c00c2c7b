// The e- and e+ generation kernels with the chord propagator of the field compiled in
// (paper Sec. 2.3; chosen when field_max_iterations > 0). A translation unit of their own
// so that they build in parallel with the analytic-helix kernels.
#include <cuda_runtime.h>

#include "layout.h"
#include "transport.cuh"

namespace adept {

template <class R>
static const void* chord_fn(int species, int minb) {
  if (species == 1) return minb >= 3 ? (const void*)k_transport<R, 1, 3, true> : (const void*)k_transport<R, 1, 2, true>;
  return minb >= 3 ? (const void*)k_transport<R, 2, 3, true> : (const void*)k_transport<R, 2, 2, true>;
}

const void* chord_transport_fn(int precision, int species, int minb) {
  return precision ? chord_fn<float>(species, minb) : chord_fn<double>(species, minb);
}

}  // namespace adept
