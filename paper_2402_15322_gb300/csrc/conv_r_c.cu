// conv_r_c.cu -- instantiations of the tiled log-domain group convolution (Sec. 4.2) for radii 12..16
// (split across files so that they compile in parallel).
#include "conv_tile.cuh"

namespace se2ot {

bool launch_tile_c(int r, bool maxpass, const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems,
                   cudaStream_t s, cudaError_t *err)
{
    switch (r) {
    case 12: *err = maxpass ? tile::launch_tile<12, true>(a, probs, items, nitems, s) : tile::launch_tile<12, false>(a, probs, items, nitems, s); return true;
    case 13: *err = maxpass ? tile::launch_tile<13, true>(a, probs, items, nitems, s) : tile::launch_tile<13, false>(a, probs, items, nitems, s); return true;
    case 14: *err = maxpass ? tile::launch_tile<14, true>(a, probs, items, nitems, s) : tile::launch_tile<14, false>(a, probs, items, nitems, s); return true;
    case 15: *err = maxpass ? tile::launch_tile<15, true>(a, probs, items, nitems, s) : tile::launch_tile<15, false>(a, probs, items, nitems, s); return true;
    case 16: *err = maxpass ? tile::launch_tile<16, true>(a, probs, items, nitems, s) : tile::launch_tile<16, false>(a, probs, items, nitems, s); return true;
    default: return false;
    }
}

}  // namespace se2ot
