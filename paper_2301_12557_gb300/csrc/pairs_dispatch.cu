// Dispatch of the pair and rescue kernels on (mode, line of sight).
#include "pairs_impl.cuh"

namespace pc {

#define PC_DECL(tag)                                                                        \
    cudaError_t launch_f32_##tag(const PairParams &, int, int, size_t, cudaStream_t);       \
    int occ_f32_##tag(const PairParams &, int, size_t);                                     \
    cudaError_t launch_f64_##tag(const PairParams &, int, size_t, cudaStream_t);            \
    int occ_f64_##tag(const PairParams &, size_t);                                          \
    cudaError_t launch_rescue_##tag(const PairParams &, int, cudaStream_t);                \
    cudaError_t launch_f32t_##tag(const PairParams &, int, int, size_t, cudaStream_t);     \
    int occ_f32t_##tag(const PairParams &, int, size_t);
PC_DECL(S)
PC_DECL(SMU_Z)
PC_DECL(SMU_MID)
PC_DECL(SIGPI_Z)
PC_DECL(SIGPI_MID)
#undef PC_DECL

static int variant(const PairParams &p) {
    if (p.mode == MODE_S) return 0;
    if (p.mode == MODE_SMU) return p.los == LOS_Z ? 1 : 2;
    return p.los == LOS_Z ? 3 : 4;
}

size_t pairs_f32_smem(const PairParams &p, int) { return smem_layout(p, false).total; }
size_t pairs_f64_smem(const PairParams &p) { return smem_layout(p, true).total; }

cudaError_t launch_pairs_f32(const PairParams &p, int ipt, int grid, size_t smem, cudaStream_t st) {
    if (p.tree) {
        switch (variant(p)) {
            case 0: return launch_f32t_S(p, ipt, grid, smem, st);
            case 1: return launch_f32t_SMU_Z(p, ipt, grid, smem, st);
            case 2: return launch_f32t_SMU_MID(p, ipt, grid, smem, st);
            case 3: return launch_f32t_SIGPI_Z(p, ipt, grid, smem, st);
            default: return launch_f32t_SIGPI_MID(p, ipt, grid, smem, st);
        }
    }
    switch (variant(p)) {
        case 0: return launch_f32_S(p, ipt, grid, smem, st);
        case 1: return launch_f32_SMU_Z(p, ipt, grid, smem, st);
        case 2: return launch_f32_SMU_MID(p, ipt, grid, smem, st);
        case 3: return launch_f32_SIGPI_Z(p, ipt, grid, smem, st);
        default: return launch_f32_SIGPI_MID(p, ipt, grid, smem, st);
    }
}

int pairs_f32_ctas_per_sm(const PairParams &p, int ipt, size_t smem) {
    if (p.tree) {
        switch (variant(p)) {
            case 0: return occ_f32t_S(p, ipt, smem);
            case 1: return occ_f32t_SMU_Z(p, ipt, smem);
            case 2: return occ_f32t_SMU_MID(p, ipt, smem);
            case 3: return occ_f32t_SIGPI_Z(p, ipt, smem);
            default: return occ_f32t_SIGPI_MID(p, ipt, smem);
        }
    }
    switch (variant(p)) {
        case 0: return occ_f32_S(p, ipt, smem);
        case 1: return occ_f32_SMU_Z(p, ipt, smem);
        case 2: return occ_f32_SMU_MID(p, ipt, smem);
        case 3: return occ_f32_SIGPI_Z(p, ipt, smem);
        default: return occ_f32_SIGPI_MID(p, ipt, smem);
    }
}

cudaError_t launch_pairs_f64(const PairParams &p, int grid, size_t smem, cudaStream_t st) {
    switch (variant(p)) {
        case 0: return launch_f64_S(p, grid, smem, st);
        case 1: return launch_f64_SMU_Z(p, grid, smem, st);
        case 2: return launch_f64_SMU_MID(p, grid, smem, st);
        case 3: return launch_f64_SIGPI_Z(p, grid, smem, st);
        default: return launch_f64_SIGPI_MID(p, grid, smem, st);
    }
}

int pairs_f64_ctas_per_sm(const PairParams &p, size_t smem) {
    switch (variant(p)) {
        case 0: return occ_f64_S(p, smem);
        case 1: return occ_f64_SMU_Z(p, smem);
        case 2: return occ_f64_SMU_MID(p, smem);
        case 3: return occ_f64_SIGPI_Z(p, smem);
        default: return occ_f64_SIGPI_MID(p, smem);
    }
}

cudaError_t launch_rescue(const PairParams &p, cudaStream_t st) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = sms * 4;
    switch (variant(p)) {
        case 0: return launch_rescue_S(p, grid, st);
        case 1: return launch_rescue_SMU_Z(p, grid, st);
        case 2: return launch_rescue_SMU_MID(p, grid, st);
        case 3: return launch_rescue_SIGPI_Z(p, grid, st);
        default: return launch_rescue_SIGPI_MID(p, grid, st);
    }
}

}  // namespace pc
