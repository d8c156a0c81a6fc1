// etics_scf_f32.cu -- mixed-precision SCF instantiation (FP32 basis and field
// sums, FP64 coefficient accumulation).
#include "etics_internal.h"
#include "etics_scf_impl.cuh"

namespace etics {
size_t scf_workspace_f32(int64_t N, int n_max, int l_max, int num_sms) {
    return scf_workspace<float>(N, n_max, l_max, num_sms);
}
int scf_coeffs_f32(const void* posm, int64_t N, int n_max, int l_max, double* coeffs, void* ws,
                   const LaunchCtx& ctx) {
    return scf_coeffs_launch<float>(posm, N, n_max, l_max, coeffs, ws, ctx);
}
int scf_field_f32(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                  void* out, int out_mask, const LaunchCtx& ctx) {
    return scf_field_launch<float>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
}
}  // namespace etics
