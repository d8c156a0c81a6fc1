// etics_scf_bins_f32.cu -- the per-warp-bin SCF coefficient pass (see
// etics_scf_bins.cuh) at (n_max, l_max) = (14, 8), the expansion the
// surrogate experiment uses for its bar-perturbed Hernquist sphere (the
// coefficients of Sec. 2.4 eq. 18 in the basis of Sec. 2.5).  12 bins of at most 7
// columns: 384 threads, 105 FP32 accumulators per lane, so one block per SM;
// tiles of 192 particles keep the two 81-column basis buffers within shared
// memory.  Its own translation unit so that it compiles in parallel with the
// other SCF kernels.
#include "etics_internal.h"
#include "etics_scf_bins.cuh"

namespace etics {
constexpr int kBins148Tile = 192;
constexpr int kBins148Blocks = 1;

size_t scf_bins148_workspace_f32(int num_sms) {
    return scf_bins_workspace<float, 15, 8, kBins148Blocks>(num_sms);
}
int scf_coeffs_bins148_f32(const void* posm, int64_t N, double* coeffs, void* ws,
                           const LaunchCtx& ctx) {
    return scf_coeffs_bins_launch<float, 15, 8, kBins148Tile, kBins148Blocks>(posm, N, coeffs, ws,
                                                                              ctx);
}
}  // namespace etics
