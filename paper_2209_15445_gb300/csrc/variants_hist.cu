// The generation kernels with the validation histogram of step lengths compiled in
// (ADEPT_FLAG_STEP_HISTOGRAM): V = 4 for every species, and V = 6 for e- and e+ with multiple
// scattering and loss fluctuations as well. The default kernels carry none of it. A
// translation unit of its own, so that it builds in parallel with the others.
#include <cuda_runtime.h>

#include "layout.h"
#include "transport.cuh"

namespace adept {

template <class R, int S, int V>
static const void* hist_by_minb(int minb) {
  return minb >= 3 ? (const void*)k_transport<R, S, 3, V> : (const void*)k_transport<R, S, 2, V>;
}

template <class R>
static const void* hist_by_species(int species, int minb, bool physics) {
  if (species == 0) return hist_by_minb<R, 0, 4>(minb);  // photons have no optional physics
  if (species == 1) return physics ? hist_by_minb<R, 1, 6>(minb) : hist_by_minb<R, 1, 4>(minb);
  return physics ? hist_by_minb<R, 2, 6>(minb) : hist_by_minb<R, 2, 4>(minb);
}

const void* hist_transport_fn(int precision, int species, int minb, int variant) {
  const bool physics = (variant & 2) != 0;
  return precision ? hist_by_species<float>(species, minb, physics) : hist_by_species<double>(species, minb, physics);
}

}  // namespace adept
