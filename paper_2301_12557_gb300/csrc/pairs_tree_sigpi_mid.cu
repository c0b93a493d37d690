// Instantiation of the tree variant of the FP32 pair kernel for MODE_SIGPI / LOS_MID.
#include "pairs_impl.cuh"

namespace pc {

cudaError_t launch_f32t_SIGPI_MID(const PairParams &p, int ipt, int grid, size_t smem, cudaStream_t st) {
    return launch_mode_f32_tree<MODE_SIGPI, LOS_MID>(p, ipt, grid, smem, st);
}
int occ_f32t_SIGPI_MID(const PairParams &p, int ipt, size_t smem) {
    return occupancy_mode_f32_tree<MODE_SIGPI, LOS_MID>(p, ipt, smem);
}

}  // namespace pc
