// etics_internal.h -- declarations shared between the C ABI (etics_api.cu)
// and the kernel translation units.
#pragma once

#include "etics_common.cuh"

namespace etics {

// ---- SCF (etics_scf_f32.cu / etics_scf_f64.cu) ----------------------------
size_t scf_workspace_f32(int64_t N, int n_max, int l_max, int num_sms);
// particle-pair coefficient pass at (10, 6) (etics_scf_pairs_f32.cu)
size_t scf_pairs106_workspace_f32(int num_sms);
int scf_coeffs_pairs106_f32(const void* posm, int64_t N, double* coeffs, void* ws,
                            const LaunchCtx& ctx);
// per-warp-bin coefficient pass at (14, 8) (etics_scf_bins_f32.cu)
size_t scf_bins148_workspace_f32(int num_sms);
int scf_coeffs_bins148_f32(const void* posm, int64_t N, double* coeffs, void* ws,
                           const LaunchCtx& ctx);
size_t scf_workspace_f64(int64_t N, int n_max, int l_max, int num_sms);
int scf_coeffs_f32(const void* posm, int64_t N, int n_max, int l_max, double* coeffs, void* ws,
                   const LaunchCtx& ctx);
int scf_coeffs_f64(const void* posm, int64_t N, int n_max, int l_max, double* coeffs, void* ws,
                   const LaunchCtx& ctx);
int scf_field_f32(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                  void* out, int out_mask, const LaunchCtx& ctx);
int scf_field_f64(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                  void* out, int out_mask, const LaunchCtx& ctx);

// ---- SCF with the Clutton-Brock radial basis (etics_scf_cb_f32/f64.cu) ------
int scf_coeffs_cb_f32(const void* posm, int64_t N, int n_max, int l_max, double* coeffs, void* ws,
                      const LaunchCtx& ctx);
int scf_coeffs_cb_f64(const void* posm, int64_t N, int n_max, int l_max, double* coeffs, void* ws,
                      const LaunchCtx& ctx);
int scf_field_cb_f32(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                     void* out, int out_mask, const LaunchCtx& ctx);
int scf_field_cb_f64(const void* posm, int64_t N, int n_max, int l_max, const double* coeffs,
                     void* out, int out_mask, const LaunchCtx& ctx);

// ---- radial sort (etics_sort.cu) -------------------------------------------
struct SortBuffers {
    uint32_t *keys_a, *keys_b, *vals_a, *vals_b;
    uint32_t *hist, *status, *counters;
    void* zero_base;
    size_t zero_bytes;
};
// carve the sort buffers from ws (ws may be null to only compute *total)
SortBuffers sort_buffers(void* ws, int64_t N, size_t* total);
int sort_tiles(int64_t N);
// the 32-bit sort keys alone
template <typename R>
int radial_keys_impl(const void* posm, int64_t N, uint32_t* keys, const LaunchCtx& ctx);
// keys + 4 radix passes + tie fix-up; the order ends in vals_a
template <typename R>
int radial_sort_impl(const void* posm, int64_t N, const SortBuffers& b, const LaunchCtx& ctx);

// the bounded waits made to run out (etics_test_wait_timeout): one radix pass
// over kTimeoutProbeN keys whose only block takes tile 1 while tile 0 never
// publishes (etics_sort.cu); an mbarrier nothing arrives on, with tensor
// memory held (etics_mlp.cu)
constexpr int64_t kTimeoutProbeN = 8192;
int lookback_timeout_probe(void* ws, int64_t spins, const LaunchCtx& ctx);
int mbarrier_timeout_probe(int64_t spins, const LaunchCtx& ctx);

// ---- arithmetic-rate microbenchmark (etics_peak.cu) ------------------------
int fma_peak(int kind, int blocks, int64_t iters, float* sink, double* flops,
             const LaunchCtx& ctx);

// ---- MEX (etics_mex_f32.cu / etics_mex_f64.cu) ----------------------------
size_t mex_workspace_f32(int64_t N, int l_max);
size_t mex_workspace_f64(int64_t N, int l_max);
int mex_field_f32(const void* posm, int64_t N, int l_max, void* out, int out_mask, void* ws,
                  const LaunchCtx& ctx);
int mex_field_f64(const void* posm, int64_t N, int l_max, void* out, int out_mask, void* ws,
                  const LaunchCtx& ctx);
int radial_order_f32(const void* posm, int64_t N, uint32_t* order, void* ws, const LaunchCtx& ctx);
int radial_order_f64(const void* posm, int64_t N, uint32_t* order, void* ws, const LaunchCtx& ctx);

// ---- batches (etics_batch.cu) ------------------------------------------------
int batch_plan_build(const etics_batch_item* items, int ninst, const etics_batch_tuning* tuning,
                     int num_sms, int precision, void* plan, size_t plan_bytes, size_t* need,
                     size_t* ws_bytes, int64_t* coef_total);
template <typename R>
int batch_launch(const void* posm, const void* plan_host, const void* plan_dev, double* coeffs,
                 void* out, int out_mask, void* ws, size_t ws_bytes, const LaunchCtx& ctx);

// ---- coefficient-forecasting MLP (etics_mlp.cu) ------------------------------
int64_t mlp_param_count(const etics_mlp_shape* s);
size_t mlp_workspace(const etics_mlp_shape* s, int batch);
int mlp_forward(const etics_mlp_shape* s, const float* params, const uint16_t* params_bf16,
                const uint16_t* x, int batch, float* y, void* ws, size_t ws_bytes,
                const LaunchCtx& ctx);
int mlp_loss_grad(const etics_mlp_shape* s, const float* params, const uint16_t* params_bf16,
                  const uint16_t* x, const float* target, int batch, float* grads, double* loss,
                  void* ws, size_t ws_bytes, const LaunchCtx& ctx);
int mlp_adam(const etics_mlp_shape* s, float* params, const float* grads, float* m, float* v,
             int64_t t, float lr, float beta1, float beta2, float eps, uint16_t* params_bf16,
             const LaunchCtx& ctx);
int mlp_to_bf16(const etics_mlp_shape* s, const float* params, uint16_t* params_bf16,
                const LaunchCtx& ctx);
int coeff_stats(const double* traj, int T, int D, int stride, double* norm, const LaunchCtx& ctx);
int coeff_features(const double* store, const int32_t* rows, const int32_t* next, int batch, int D,
                   int stride, const double* norm, int per_coeff, uint16_t* x, float* target,
                   const LaunchCtx& ctx);
int coeff_advance(double* ring, int32_t* order, int D, int stride, int horizon,
                  const double* coeffs_in, const float* y, int y_stride, const double* norm,
                  double* coeffs_out, int commit, const LaunchCtx& ctx);
int force_error(const void* a, const void* r, int64_t N, int precision, double tol_a,
                double tol_b, uint64_t* out, const LaunchCtx& ctx);

// ---- leapfrog (etics_step.cu) ----------------------------------------------
int kick_drift_f32(void* posm, void* vel, const void* acc, int64_t N, double dt,
                   const LaunchCtx& ctx);
int kick_drift_f64(void* posm, void* vel, const void* acc, int64_t N, double dt,
                   const LaunchCtx& ctx);
int kick_f32(void* vel, const void* acc, int64_t N, double dt, const LaunchCtx& ctx);
int kick_f64(void* vel, const void* acc, int64_t N, double dt, const LaunchCtx& ctx);

}  // namespace etics
