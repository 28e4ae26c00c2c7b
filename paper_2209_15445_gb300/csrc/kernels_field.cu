// The default e- and e+ generation kernels with the analytic helix compiled in (V = 8), for
// calorimeters in a uniform field; the field-free ones carry no helix code. A translation unit
// of its own, so that it builds in parallel with the others.
#include <cuda_runtime.h>

#include "layout.h"
#include "transport.cuh"

namespace adept {

template <class R, int S>
static const void* field_by_minb(int minb) {
  switch (minb) {
    case 1: return (const void*)k_transport<R, S, 1, 8>;
    case 2: return (const void*)k_transport<R, S, 2, 8>;
    case 3: return (const void*)k_transport<R, S, 3, 8>;
    default: return (const void*)k_transport<R, S, 4, 8>;
  }
}

const void* field_transport_fn(int precision, int species, int minb) {
  if (precision) return species == 1 ? field_by_minb<float, 1>(minb) : field_by_minb<float, 2>(minb);
  return species == 1 ? field_by_minb<double, 1>(minb) : field_by_minb<double, 2>(minb);
}

}  // namespace adept
