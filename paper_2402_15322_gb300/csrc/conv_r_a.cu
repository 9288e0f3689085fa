// conv_r_a.cu -- instantiations of the tiled log-domain group convolution (Sec. 4.2) for radii 0..5
// (split across files so that they compile in parallel).
#include "conv_tile.cuh"

namespace se2ot {

bool launch_tile_a(int r, bool maxpass, const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems,
                   cudaStream_t s, cudaError_t *err)
{
    switch (r) {
    case 0: *err = maxpass ? tile::launch_tile<0, true>(a, probs, items, nitems, s) : tile::launch_tile<0, false>(a, probs, items, nitems, s); return true;
    case 1: *err = maxpass ? tile::launch_tile<1, true>(a, probs, items, nitems, s) : tile::launch_tile<1, false>(a, probs, items, nitems, s); return true;
    case 2: *err = maxpass ? tile::launch_tile<2, true>(a, probs, items, nitems, s) : tile::launch_tile<2, false>(a, probs, items, nitems, s); return true;
    case 3: *err = maxpass ? tile::launch_tile<3, true>(a, probs, items, nitems, s) : tile::launch_tile<3, false>(a, probs, items, nitems, s); return true;
    case 4: *err = maxpass ? tile::launch_tile<4, true>(a, probs, items, nitems, s) : tile::launch_tile<4, false>(a, probs, items, nitems, s); return true;
    case 5: *err = maxpass ? tile::launch_tile<5, true>(a, probs, items, nitems, s) : tile::launch_tile<5, false>(a, probs, items, nitems, s); return true;
    default: return false;
    }
}

}  // namespace se2ot
