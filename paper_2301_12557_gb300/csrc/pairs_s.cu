// Instantiation of the pair kernels for MODE_S / LOS_Z.
#include "pairs_impl.cuh"

namespace pc {

cudaError_t launch_f32_S(const PairParams &p, int ipt, int grid, size_t smem, cudaStream_t st) {
    return launch_mode_f32<MODE_S, LOS_Z>(p, ipt, grid, smem, st);
}
int occ_f32_S(const PairParams &p, int ipt, size_t smem) {
    return occupancy_mode_f32<MODE_S, LOS_Z>(p, ipt, smem);
}
cudaError_t launch_f64_S(const PairParams &p, int grid, size_t smem, cudaStream_t st) {
    return launch_mode_f64<MODE_S, LOS_Z>(p, grid, smem, st);
}
int occ_f64_S(const PairParams &p, size_t smem) {
    return occupancy_mode_f64<MODE_S, LOS_Z>(p, smem);
}
cudaError_t launch_rescue_S(const PairParams &p, int grid, cudaStream_t st) {
    return launch_mode_rescue<MODE_S, LOS_Z>(p, grid, st);
}

}  // namespace pc
