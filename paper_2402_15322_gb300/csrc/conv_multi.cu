// conv_multi.cu -- one launch for a convolution line of a whole uneven batch (Sec. 4.2 group
// convolution, Appendix A iteration): every work item (problem, field x orientation, tile) runs
// the body of conv_tile.cuh specialised for its problem's radius, so a batch that mixes radii needs
// one launch per line instead of one per radius.  Each item runs exactly the code of the
// per-radius kernel, so the results are bit-identical to it.
#include "conv_tile.cuh"

namespace se2ot {

namespace {

// Dynamic shared memory of the multi-radius kernel: the largest any radius needs.
constexpr size_t multi_smem_floats()
{
    size_t m = 0;
    for (int r = 0; r <= MAX_RADIUS; ++r) m = tile::smem_floats(r) > m ? tile::smem_floats(r) : m;
    return m;
}

template <int R>
__device__ __forceinline__ void run_radius(int r, const ConvArgs &a0, const ConvArgs *probs, const int4 *items)
{
    if (r == R) {
        tile::conv_tile_body<R, false, true>(a0, probs, items);
        return;
    }
    if constexpr (R < MAX_RADIUS) run_radius<R + 1>(r, a0, probs, items);
}

__global__ void __launch_bounds__(tile::THREADS, 6) conv_multi_kernel(const ConvArgs a0, const ConvArgs *probs,
                                                                      const int4 *items)
{
    pdl_launch_dependents();
    pdl_wait();   // the launch order may be written by the previous launch of the same line
    const unsigned slot = a0.order ? a0.order[blockIdx.x] : blockIdx.x;
    run_radius<0>(probs[items[slot].x].r, a0, probs, items);
}

}  // namespace

cudaError_t launch_conv_multi(const ConvArgs &shared, const ConvArgs *probs, const int4 *items, int nitems,
                              cudaStream_t s)
{
    const size_t smem = sizeof(float) * multi_smem_floats();
    static PerDeviceOnce attrs;   // shared-memory limit above 48 KB, once per device
    cudaError_t ea = attrs.run([&]() {
        return cudaFuncSetAttribute(conv_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (ea != cudaSuccess || nitems <= 0) return ea;
    PdlLaunch L(dim3(nitems), dim3(tile::THREADS), smem, s);
    return cudaLaunchKernelEx(&L.cfg, conv_multi_kernel, shared, probs, items);
}

}  // namespace se2ot
