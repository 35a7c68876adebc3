// Adjoint of a spectral loss (step A9) - placeholder until the Krylov adjoint lands.
#include <cuda_runtime.h>

#include "internal.h"

namespace bse {

size_t backward_ws_bytes(const DevSys& d, long long nsteps) { return spectrum_ws_bytes(d, nsteps); }

int launch_backward(const DevSys&, const void*, const void*, int, const double*, int, double, const double*,
                    const void*, const void*, const void*, double*, void*, void*, void*, void*, void*, int*, void*) {
  return -1;
}

}  // namespace bse
