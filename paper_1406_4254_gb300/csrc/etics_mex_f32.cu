// etics_mex_f32.cu -- mixed-precision MEX instantiation (FP32 moments and
// in-tile scans, FP64 cross-tile carries).
#include "etics_mex_impl.cuh"

namespace etics {
size_t mex_workspace_f32(int64_t N, int l_max) { return mex_workspace_impl<float>(N, l_max); }
int mex_field_f32(const void* posm, int64_t N, int l_max, void* out, int out_mask, void* ws,
                  const LaunchCtx& ctx) {
    return mex_field_impl<float>(posm, N, l_max, out, out_mask, ws, ctx);
}
int radial_order_f32(const void* posm, int64_t N, uint32_t* order, void* ws, const LaunchCtx& ctx) {
    return radial_order_impl<float>(posm, N, order, ws, ctx);
}
}  // namespace etics
