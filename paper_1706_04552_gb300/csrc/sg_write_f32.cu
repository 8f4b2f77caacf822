// sg_write_f32.cu -- float32 instantiations of the map-and-write pass.
#include "sg_write.cuh"

namespace sg {
cudaError_t launch_write_f32(int r, int s, int map, int vk, float *grid,
                             uint64_t vs, cudaStream_t st, const LaunchCfg &cfg)
{
    return launch_write_any<float>(r, s, map, vk, grid, vs, st, cfg);
}
}  // namespace sg
