// etics_scf_pairs_f32.cu -- the particle-pair SCF coefficient pass (see
// etics_scf_pairs.cuh) at (n_max, l_max) = (10, 6), the expansion of the
// paper's timing runs (Sec. 3.4): bins of at most 4 columns of one level, 16
// warps of up to 128 registers (measured on GB300 at N = 2^20: 60.0 us against
// 62.1 us with 3-column bins and 19 warps).  Its own translation unit so that
// it compiles in parallel with the other SCF kernels.
#include "etics_internal.h"
#include "etics_scf_pairs.cuh"

namespace etics {
constexpr int kPairs106Cap = 4;

size_t scf_pairs106_workspace_f32(int num_sms) {
    return scf_pairs_workspace<11, 6, kPairs106Cap>(num_sms);
}
int scf_coeffs_pairs106_f32(const void* posm, int64_t N, double* coeffs, void* ws,
                            const LaunchCtx& ctx) {
    return scf_coeffs_pairs_launch<11, 6, kPairs106Cap>(posm, N, coeffs, ws, ctx);
}
}  // namespace etics
