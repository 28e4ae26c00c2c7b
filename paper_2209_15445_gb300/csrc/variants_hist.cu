// The generation kernels with the validation histogram of step lengths compiled in
// (ADEPT_FLAG_STEP_HISTOGRAM): V = 4 for every species, and for e- and e+ V = 6 with multiple
// scattering and loss fluctuations as well, 12 and 14 with the helix in a field. The default
// kernels carry none of it. A
// translation unit of its own, so that it builds in parallel with the others.
#include <cuda_runtime.h>

#include "layout.h"
#include "transport.cuh"

namespace adept {

template <class R, int S, int V>
static const void* hist_by_minb(int minb) {
  return minb >= 3 ? (const void*)k_transport<R, S, 3, V> : (const void*)k_transport<R, S, 2, V>;
}

template <class R, int S>
static const void* hist_charged(int minb, int variant) {
  switch (variant & 10) {
    case 0: return hist_by_minb<R, S, 4>(minb);
    case 2: return hist_by_minb<R, S, 6>(minb);
    case 8: return hist_by_minb<R, S, 12>(minb);
    default: return hist_by_minb<R, S, 14>(minb);
  }
}

template <class R>
static const void* hist_by_species(int species, int minb, int variant) {
  if (species == 0) return hist_by_minb<R, 0, 4>(minb);  // photons: no optional physics, no helix
  return species == 1 ? hist_charged<R, 1>(minb, variant) : hist_charged<R, 2>(minb, variant);
}

const void* hist_transport_fn(int precision, int species, int minb, int variant) {
  return precision ? hist_by_species<float>(species, minb, variant) : hist_by_species<double>(species, minb, variant);
}

}  // namespace adept
