// conv_r_b.cu -- instantiations of the tiled log-domain group convolution (Sec. 4.2) for radii 6..11
// (split across files so that they compile in parallel).
#include "conv_tile.cuh"

namespace se2ot {

bool launch_tile_b(int r, bool maxpass, const ConvArgs &a, const ConvArgs *probs, const int4 *items, int nitems,
                   cudaStream_t s, cudaError_t *err)
{
    switch (r) {
    case 6: *err = maxpass ? tile::launch_tile<6, true>(a, probs, items, nitems, s) : tile::launch_tile<6, false>(a, probs, items, nitems, s); return true;
    case 7: *err = maxpass ? tile::launch_tile<7, true>(a, probs, items, nitems, s) : tile::launch_tile<7, false>(a, probs, items, nitems, s); return true;
    case 8: *err = maxpass ? tile::launch_tile<8, true>(a, probs, items, nitems, s) : tile::launch_tile<8, false>(a, probs, items, nitems, s); return true;
    case 9: *err = maxpass ? tile::launch_tile<9, true>(a, probs, items, nitems, s) : tile::launch_tile<9, false>(a, probs, items, nitems, s); return true;
    case 10: *err = maxpass ? tile::launch_tile<10, true>(a, probs, items, nitems, s) : tile::launch_tile<10, false>(a, probs, items, nitems, s); return true;
    case 11: *err = maxpass ? tile::launch_tile<11, true>(a, probs, items, nitems, s) : tile::launch_tile<11, false>(a, probs, items, nitems, s); return true;
    default: return false;
    }
}

}  // namespace se2ot
