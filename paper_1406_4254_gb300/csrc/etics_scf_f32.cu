// etics_scf_f32.cu -- mixed-precision SCF instantiation (FP32 basis and field
// sums, FP64 coefficient accumulation).
#include "etics_internal.h"
#include "etics_scf_bins.cuh"

namespace etics {
size_t scf_workspace_f32(int64_t N, int n_max, int l_max, int num_sms) {
    size_t a = scf_workspace<float>(N, n_max, l_max, num_sms);
    size_t b = 0;
    if (n_max == 10 && l_max == 6) b = scf_pairs106_workspace_f32(num_sms);
    if (n_max == 14 && l_max == 8) b = scf_bins148_workspace_f32(num_sms);
    return a > b ? a : b;
}
int scf_coeffs_f32(const void* posm, int64_t N, int n_max, int l_max, double* coeffs, void* ws,
                   const LaunchCtx& ctx) {
    // specialised kernels for the paper's (10, 6) and (14, 8) expansions:
    // particle pairs on paired FP32 instructions, one level per warp (10, 6);
    // per-warp bins (14, 8)
    if (n_max == 10 && l_max == 6)
        return scf_coeffs_pairs106_f32(posm, N, coeffs, ws, ctx);
    if (n_max == 14 && l_max == 8) return scf_coeffs_bins148_f32(posm, N, coeffs, ws, ctx);
    return scf_coeffs_launch<float>(posm, N, n_max, l_max, coeffs, ws, ctx);
}
int scf_field_f32(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                  void* out, int out_mask, const LaunchCtx& ctx) {
    return scf_field_launch<float>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
}
}  // namespace etics
