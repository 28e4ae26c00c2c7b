// The e- and e+ generation kernels with optional parts compiled in, chosen by the options:
// V = 1 the chord propagator of the field (paper Sec. 2.3; field_max_iterations > 0),
// V = 2 multiple scattering and loss fluctuations (physics != 0), V = 3 both, V = 10 the
// optional physics with the analytic helix in a field. A translation
// unit of their own, so that they build in parallel with the default kernels, which carry
// none of this code.
#include <cuda_runtime.h>

#include "layout.h"
#include "transport.cuh"

namespace adept {

template <class R, int S, int V>
static const void* by_minb(int minb) {
  return minb >= 3 ? (const void*)k_transport<R, S, 3, V> : (const void*)k_transport<R, S, 2, V>;
}

template <class R, int S>
static const void* by_variant(int minb, int variant) {
  if (variant & 1) return (variant & 2) ? by_minb<R, S, 3>(minb) : by_minb<R, S, 1>(minb);
  return (variant & 8) ? by_minb<R, S, 10>(minb) : by_minb<R, S, 2>(minb);
}

const void* variant_transport_fn(int precision, int species, int minb, int variant) {
  if (precision) return species == 1 ? by_variant<float, 1>(minb, variant) : by_variant<float, 2>(minb, variant);
  return species == 1 ? by_variant<double, 1>(minb, variant) : by_variant<double, 2>(minb, variant);
}

}  // namespace adept
