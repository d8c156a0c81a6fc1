// etics_scf_cb_f32.cu -- SCF with the Clutton-Brock radial basis (the
// Plummer model as zeroth term; the alternative basis of paper Sec. 2.5):
// the generic coefficient and field kernels instantiated for basis 1 in
// mixed precision (FP32 basis and field sums, FP64 coefficient accumulation).
#include "etics_internal.h"
#include "etics_scf_impl.cuh"

namespace etics {
int scf_coeffs_cb_f32(const void* posm, int64_t N, int n_max, int l_max, double* coeffs,
                       void* ws, const LaunchCtx& ctx) {
    return scf_coeffs_launch<float, 1>(posm, N, n_max, l_max, coeffs, ws, ctx);
}
int scf_field_cb_f32(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                      void* out, int out_mask, const LaunchCtx& ctx) {
    return scf_field_launch_generic<float, 1>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
}
}  // namespace etics
