// Row layouts of the pair-density arrays read by the W.rho products (steps A4 and the coupling block).
//
// side 0: rho_vv' rows of the direct set, per q [nblk][Nv^2] at qvec_off[q];
// side 1: rho_cc' rows of the direct set, per q [nblk][Nc^2] after the vv' rows;
// side 2: rho_cv' rows of the coupling set, per q [nblk][Nc Nv] after the [nblk][Nv Nc] rho_vc' rows,
//         the q block starting at 2 Nv Nc qblk_off[q].
// vbase is the first vector of the array's q range in the same numbering.
#pragma once

#include "internal.h"

namespace bse {

__host__ __device__ __forceinline__ int side_width(const DevSys& d, int side) {
  return side == 2 ? d.nv * d.nc : (side == 1 ? d.nc * d.nc : d.nv * d.nv);
}

__device__ __forceinline__ long long side_rows_offset(const DevSys& d, int q, int side, long long vbase) {
  const long long nblk = d.qblk_off[q + 1] - d.qblk_off[q];
  if (side == 2) {
    const long long w = (long long)d.nv * d.nc;
    return 2 * w * d.qblk_off[q] - vbase + nblk * w;
  }
  return d.qvec_off[q] - vbase + (side == 1 ? nblk * d.nv * d.nv : 0);
}

}  // namespace bse
