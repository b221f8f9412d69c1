// Where a population lives in a lattice updated in place (AA pattern).
//
// The library's state between steps is, by convention, the post-collision
// populations f*_i(x) of the last step, not yet streamed (what the two-lattice
// pull scheme stores: slot i of cell x).  A one-lattice lattice holds the same
// numbers in one of two arrangements, by the parity of the number t of
// completed steps:
//   t even: f*_i(x) in slot opp(i) of cell x (the local step stored it there;
//           also the arrangement written at create and by set_state);
//   t odd:  f*_i(x) in slot i of cell x + c_i (the shifted step streamed it),
//           or, when x + c_i lies outside the lattice (a wall in y, the open
//           ends in x), in slot opp(i) of cell x.
// Both maps are bijections of the 19 nx ny nz slots, so the whole state is
// recoverable and every slot holds a population.
#pragma once

#include <cstddef>

#include "d3q19.cuh"

namespace stg {

// element index (plane * P + cell) of canonical population i of cell (x, y, z)
__host__ __device__ inline size_t aa_slot(int i, int x, int y, int z, long long t, int nx, int ny, int nz, int bc_x,
                                          int bc_y)
{
    const size_t P = (size_t)nx * ny * nz;
    const size_t own = ((size_t)z * ny + y) * nx + x;
    if ((t & 1) == 0) return (size_t)opp_of(i) * P + own;
    int xt = x + cx_of(i), yt = y + cy_of(i), zt = z + cz_of(i);
    zt = zt < 0 ? zt + nz : (zt >= nz ? zt - nz : zt);
    if (bc_x == 1) xt = xt < 0 ? xt + nx : (xt >= nx ? xt - nx : xt);
    if (bc_y == 1) yt = yt < 0 ? yt + ny : (yt >= ny ? yt - ny : yt);
    if (xt < 0 || xt >= nx || yt < 0 || yt >= ny) return (size_t)opp_of(i) * P + own;
    return (size_t)i * P + ((size_t)zt * ny + yt) * nx + xt;
}

}  // namespace stg
