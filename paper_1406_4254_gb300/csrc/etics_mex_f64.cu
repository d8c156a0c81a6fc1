// etics_mex_f64.cu -- FP64 MEX instantiation (all arithmetic in double precision).
#include "etics_mex_impl.cuh"

namespace etics {
size_t mex_workspace_f64(int64_t N, int l_max) { return mex_workspace_impl<double>(N, l_max); }
int mex_field_f64(const void* posm, int64_t N, int l_max, void* out, int out_mask, void* ws,
                  const LaunchCtx& ctx) {
    return mex_field_impl<double>(posm, N, l_max, out, out_mask, ws, ctx);
}
int radial_order_f64(const void* posm, int64_t N, uint32_t* order, void* ws, const LaunchCtx& ctx) {
    return radial_order_impl<double>(posm, N, order, ws, ctx);
}
}  // namespace etics
