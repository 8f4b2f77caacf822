// sg_write_u8.cu -- uint8 instantiations of the map-and-write pass.
#include "sg_write.cuh"

namespace sg {
cudaError_t launch_write_u8(int r, int s, int map, int vk, uint8_t *grid,
                            uint64_t vs, cudaStream_t st, const LaunchCfg &cfg)
{
    return launch_write_any<uint8_t>(r, s, map, vk, grid, vs, st, cfg);
}
}  // namespace sg
