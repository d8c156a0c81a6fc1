// etics_api.cu -- the C ABI of include/etics.h: argument validation,
// workspace sizing, the device error word and dispatch to the kernels.
#include <atomic>
#include <mutex>

#include "etics_internal.h"

namespace {

// The device error word: one per device (a __device__ variable lives on
// every device the library is used on).  Host code only ever uses its device
// address, fetched per device with cudaGetSymbolAddress.
__device__ unsigned int g_error_word;

std::mutex g_mutex;
constexpr int kMaxDevices = 64;
unsigned* g_err_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};
std::atomic<uint64_t> g_launches{0};
void** g_events = nullptr;
int g_n_events = 0;
std::atomic<int64_t> g_wait_limit{0};

int current_device_state(unsigned** err, int* num_sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ETICS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_err_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_error_word) != cudaSuccess) return ETICS_ERR_CUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return ETICS_ERR_CUDA;
        g_err_ptr[dev] = static_cast<unsigned*>(p);
        g_num_sms[dev] = sms;
    }
    *err = g_err_ptr[dev];
    *num_sms = g_num_sms[dev];
    return ETICS_OK;
}

struct CtxHolder {
    etics::LaunchCtx ctx;
    uint64_t launches = 0;
    ~CtxHolder() { g_launches += launches; }
};

int make_ctx(void* stream, CtxHolder& h) {
    unsigned* err = nullptr;
    int sms = 0;
    const int rc = current_device_state(&err, &sms);
    if (rc) return rc;
    h.ctx.stream = static_cast<cudaStream_t>(stream);
    h.ctx.err = err;
    h.ctx.num_sms = sms;
    h.ctx.launches = &h.launches;
    h.ctx.events = g_events;
    h.ctx.n_events = g_n_events;
    h.ctx.wait_limit = g_wait_limit.load();
    return ETICS_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
bool valid_precision(int p) { return p == ETICS_FP64 || p == ETICS_MIXED; }
bool valid_n(int64_t N) { return N >= 0 && N < (int64_t(1) << 30); }

int check_particles(const void* p, int64_t N) {
    if (N > 0 && (!p || !aligned(p, 16))) return ETICS_ERR_ARG;
    return ETICS_OK;
}

}  // namespace

extern "C" {

size_t etics_workspace_bytes(int64_t N, int n_max, int l_max, int method, int precision) {
    if (!valid_n(N) || !valid_precision(precision) || n_max < 0 || l_max < 0) return 0;
    unsigned* err = nullptr;
    int sms = 0;
    if (current_device_state(&err, &sms)) return 0;
    if (method == ETICS_SCF) {
        if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return 0;
        return precision == ETICS_MIXED ? etics::scf_workspace_f32(N, n_max, l_max, sms)
                                        : etics::scf_workspace_f64(N, n_max, l_max, sms);
    }
    if (method == ETICS_MEX) {
        if (l_max > ETICS_MEX_LMAX_LIMIT) return 0;
        return precision == ETICS_MIXED ? etics::mex_workspace_f32(N, l_max)
                                        : etics::mex_workspace_f64(N, l_max);
    }
    return 0;
}

int etics_scf_coeffs(const void* posm, int64_t N, int n_max, int l_max, int precision,
                     double* coeffs, void* ws, size_t ws_bytes, void* stream) {
    if (!valid_n(N) || !valid_precision(precision) || !coeffs || !aligned(coeffs, 8))
        return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0) return ETICS_ERR_ARG;
    if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if (check_particles(posm, N)) return ETICS_ERR_ARG;
    if (!ws || !aligned(ws, 256)) return ETICS_ERR_ARG;
    if (ws_bytes < etics_workspace_bytes(N, n_max, l_max, ETICS_SCF, precision))
        return ETICS_ERR_WORKSPACE;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    etics::stage_event(h.ctx, 0);
    rc = precision == ETICS_MIXED
             ? etics::scf_coeffs_f32(posm, N, n_max, l_max, coeffs, ws, h.ctx)
             : etics::scf_coeffs_f64(posm, N, n_max, l_max, coeffs, ws, h.ctx);
    etics::stage_event(h.ctx, 2);
    return rc;
}

int etics_scf_field(const void* posm, int64_t N, int n_max, int l_max, int precision,
                    const double* coeffs, void* accpot, int out_mask, void* stream) {
    if (!valid_n(N) || !valid_precision(precision) || !coeffs || !aligned(coeffs, 8))
        return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0) return ETICS_ERR_ARG;
    if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if ((out_mask & (ETICS_OUT_ACC | ETICS_OUT_POT)) == 0 || (out_mask & ~3)) return ETICS_ERR_ARG;
    if (check_particles(posm, N) || check_particles(accpot, N)) return ETICS_ERR_ARG;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    etics::stage_event(h.ctx, 0);
    rc = precision == ETICS_MIXED
             ? etics::scf_field_f32(posm, N, n_max, l_max, coeffs, accpot, out_mask, h.ctx)
             : etics::scf_field_f64(posm, N, n_max, l_max, coeffs, accpot, out_mask, h.ctx);
    etics::stage_event(h.ctx, 1);
    return rc;
}

int etics_scf_coeffs_basis(const void* posm, int64_t N, int n_max, int l_max, int basis,
                           int precision, double* coeffs, void* ws, size_t ws_bytes,
                           void* stream) {
    if (basis == ETICS_BASIS_HO)
        return etics_scf_coeffs(posm, N, n_max, l_max, precision, coeffs, ws, ws_bytes, stream);
    if (basis != ETICS_BASIS_CB) return ETICS_ERR_ARG;
    if (!valid_n(N) || !valid_precision(precision) || !coeffs || !aligned(coeffs, 8))
        return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0) return ETICS_ERR_ARG;
    if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if (check_particles(posm, N)) return ETICS_ERR_ARG;
    if (!ws || !aligned(ws, 256)) return ETICS_ERR_ARG;
    if (ws_bytes < etics_workspace_bytes(N, n_max, l_max, ETICS_SCF, precision))
        return ETICS_ERR_WORKSPACE;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    etics::stage_event(h.ctx, 0);
    rc = precision == ETICS_MIXED
             ? etics::scf_coeffs_cb_f32(posm, N, n_max, l_max, coeffs, ws, h.ctx)
             : etics::scf_coeffs_cb_f64(posm, N, n_max, l_max, coeffs, ws, h.ctx);
    etics::stage_event(h.ctx, 2);
    return rc;
}

int etics_scf_field_basis(const void* posm, int64_t N, int n_max, int l_max, int basis,
                          int precision, const double* coeffs, void* accpot, int out_mask,
                          void* stream) {
    if (basis == ETICS_BASIS_HO)
        return etics_scf_field(posm, N, n_max, l_max, precision, coeffs, accpot, out_mask, stream);
    if (basis != ETICS_BASIS_CB) return ETICS_ERR_ARG;
    if (!valid_n(N) || !valid_precision(precision) || !coeffs || !aligned(coeffs, 8))
        return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0) return ETICS_ERR_ARG;
    if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if ((out_mask & (ETICS_OUT_ACC | ETICS_OUT_POT)) == 0 || (out_mask & ~3)) return ETICS_ERR_ARG;
    if (check_particles(posm, N) || check_particles(accpot, N)) return ETICS_ERR_ARG;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    etics::stage_event(h.ctx, 0);
    rc = precision == ETICS_MIXED
             ? etics::scf_field_cb_f32(posm, N, n_max, l_max, coeffs, accpot, out_mask, h.ctx)
             : etics::scf_field_cb_f64(posm, N, n_max, l_max, coeffs, accpot, out_mask, h.ctx);
    etics::stage_event(h.ctx, 1);
    return rc;
}

int etics_mex_field(const void* posm, int64_t N, int l_max, int precision, void* accpot,
                    int out_mask, void* ws, size_t ws_bytes, void* stream) {
    if (!valid_n(N) || !valid_precision(precision) || l_max < 0) return ETICS_ERR_ARG;
    if (l_max > ETICS_MEX_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if ((out_mask & (ETICS_OUT_ACC | ETICS_OUT_POT)) == 0 || (out_mask & ~3)) return ETICS_ERR_ARG;
    if (check_particles(posm, N) || check_particles(accpot, N)) return ETICS_ERR_ARG;
    if (!ws || !aligned(ws, 256)) return ETICS_ERR_ARG;
    if (ws_bytes < etics_workspace_bytes(N, 0, l_max, ETICS_MEX, precision))
        return ETICS_ERR_WORKSPACE;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    return precision == ETICS_MIXED
               ? etics::mex_field_f32(posm, N, l_max, accpot, out_mask, ws, h.ctx)
               : etics::mex_field_f64(posm, N, l_max, accpot, out_mask, ws, h.ctx);
}

int etics_radial_sort(const void* posm, int64_t N, int precision, uint32_t* order, void* ws,
                      size_t ws_bytes, void* stream) {
    if (!valid_n(N) || !valid_precision(precision)) return ETICS_ERR_ARG;
    if (check_particles(posm, N) || (N > 0 && (!order || !aligned(order, 4)))) return ETICS_ERR_ARG;
    if (!ws || !aligned(ws, 256)) return ETICS_ERR_ARG;
    if (ws_bytes < etics_workspace_bytes(N, 0, 0, ETICS_MEX, precision)) return ETICS_ERR_WORKSPACE;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    return precision == ETICS_MIXED ? etics::radial_order_f32(posm, N, order, ws, h.ctx)
                                    : etics::radial_order_f64(posm, N, order, ws, h.ctx);
}

int etics_radial_keys(const void* posm, int64_t N, int precision, uint32_t* keys, void* stream) {
    if (!valid_n(N) || !valid_precision(precision)) return ETICS_ERR_ARG;
    if (check_particles(posm, N) || (N > 0 && (!keys || !aligned(keys, 4)))) return ETICS_ERR_ARG;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    return precision == ETICS_MIXED ? etics::radial_keys_impl<float>(posm, N, keys, h.ctx)
                                    : etics::radial_keys_impl<double>(posm, N, keys, h.ctx);
}

int etics_leapfrog_step(void* posm, void* vel, void* accpot, int64_t N, double dt, int method,
                        int n_max, int l_max, int precision, double* coeffs_out, void* ws,
                        size_t ws_bytes, void* stream) {
    if (!valid_n(N) || !valid_precision(precision) || !(dt == dt)) return ETICS_ERR_ARG;
    if (method != ETICS_SCF && method != ETICS_MEX) return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0) return ETICS_ERR_ARG;
    if (method == ETICS_SCF && (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT))
        return ETICS_ERR_UNSUPPORTED;
    if (method == ETICS_MEX && l_max > ETICS_MEX_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if (check_particles(posm, N) || check_particles(vel, N) || check_particles(accpot, N))
        return ETICS_ERR_ARG;
    if (!ws || !aligned(ws, 256)) return ETICS_ERR_ARG;
    if (coeffs_out && !aligned(coeffs_out, 8)) return ETICS_ERR_ARG;
    const size_t need = etics_workspace_bytes(N, n_max, l_max, method, precision);
    const size_t ncoef = (size_t)(n_max + 1) * (l_max + 1) * (l_max + 1);
    const size_t coef_bytes = method == ETICS_SCF && !coeffs_out ? (ncoef * 8 + 255) / 256 * 256 : 0;
    if (ws_bytes < need + coef_bytes) return ETICS_ERR_WORKSPACE;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    const bool mixed = precision == ETICS_MIXED;
    rc = mixed ? etics::kick_drift_f32(posm, vel, accpot, N, dt, h.ctx)
               : etics::kick_drift_f64(posm, vel, accpot, N, dt, h.ctx);
    if (rc) return rc;
    if (method == ETICS_SCF) {
        // coefficients go to coeffs_out, or to the end of the workspace
        double* c = coeffs_out ? coeffs_out
                               : reinterpret_cast<double*>(static_cast<uint8_t*>(ws) + need);
        rc = mixed ? etics::scf_coeffs_f32(posm, N, n_max, l_max, c, ws, h.ctx)
                   : etics::scf_coeffs_f64(posm, N, n_max, l_max, c, ws, h.ctx);
        if (rc) return rc;
        rc = mixed ? etics::scf_field_f32(posm, N, n_max, l_max, c, accpot, 3, h.ctx)
                   : etics::scf_field_f64(posm, N, n_max, l_max, c, accpot, 3, h.ctx);
    } else {
        rc = mixed ? etics::mex_field_f32(posm, N, l_max, accpot, 3, ws, h.ctx)
                   : etics::mex_field_f64(posm, N, l_max, accpot, 3, ws, h.ctx);
    }
    if (rc) return rc;
    return mixed ? etics::kick_f32(vel, accpot, N, dt, h.ctx)
                 : etics::kick_f64(vel, accpot, N, dt, h.ctx);
}

int etics_leapfrog_step_coeffs(void* posm, void* vel, void* accpot, int64_t N, double dt,
                               int n_max, int l_max, int precision, const double* coeffs,
                               void* stream) {
    if (!valid_n(N) || !valid_precision(precision) || !(dt == dt)) return ETICS_ERR_ARG;
    if (n_max < 0 || l_max < 0 || !coeffs || !aligned(coeffs, 8)) return ETICS_ERR_ARG;
    if (n_max > ETICS_NMAX_LIMIT || l_max > ETICS_LMAX_LIMIT) return ETICS_ERR_UNSUPPORTED;
    if (check_particles(posm, N) || check_particles(vel, N) || check_particles(accpot, N))
        return ETICS_ERR_ARG;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    const bool mixed = precision == ETICS_MIXED;
    rc = mixed ? etics::kick_drift_f32(posm, vel, accpot, N, dt, h.ctx)
               : etics::kick_drift_f64(posm, vel, accpot, N, dt, h.ctx);
    if (rc) return rc;
    rc = mixed ? etics::scf_field_f32(posm, N, n_max, l_max, coeffs, accpot, 3, h.ctx)
               : etics::scf_field_f64(posm, N, n_max, l_max, coeffs, accpot, 3, h.ctx);
    if (rc) return rc;
    return mixed ? etics::kick_f32(vel, accpot, N, dt, h.ctx)
                 : etics::kick_f64(vel, accpot, N, dt, h.ctx);
}

// ---- coefficient-forecasting MLP ---------------------------------------------
namespace {
bool mlp_args(const etics_mlp_shape* s, const float* params, const uint16_t* pb) {
    return etics::mlp_param_count(s) > 0 && params && pb && aligned(params, 4) && aligned(pb, 2);
}
}  // namespace

int64_t etics_mlp_param_count(const etics_mlp_shape* shape) {
    return etics::mlp_param_count(shape);
}

size_t etics_mlp_workspace_bytes(const etics_mlp_shape* shape, int batch) {
    return etics::mlp_workspace(shape, batch);
}

int etics_mlp_forward(const etics_mlp_shape* shape, const float* params,
                      const uint16_t* params_bf16, const uint16_t* x, int batch, float* y,
                      void* ws, size_t ws_bytes, void* stream) {
    if (!mlp_args(shape, params, params_bf16) || batch < 0) return ETICS_ERR_ARG;
    if (batch > 0 && (!x || !y || !ws || !aligned(x, 2) || !aligned(y, 4) || !aligned(ws, 256)))
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::mlp_forward(shape, params, params_bf16, x, batch, y, ws, ws_bytes, h.ctx);
}

int etics_mlp_loss_grad(const etics_mlp_shape* shape, const float* params,
                        const uint16_t* params_bf16, const uint16_t* x, const float* target,
                        int batch, float* grads, double* loss, void* ws, size_t ws_bytes,
                        void* stream) {
    if (!mlp_args(shape, params, params_bf16) || batch < 1) return ETICS_ERR_ARG;
    if (!x || !target || !grads || !loss || !ws || !aligned(x, 2) || !aligned(target, 4) ||
        !aligned(grads, 4) || !aligned(loss, 8) || !aligned(ws, 256))
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::mlp_loss_grad(shape, params, params_bf16, x, target, batch, grads, loss, ws,
                                ws_bytes, h.ctx);
}

int etics_mlp_adam(const etics_mlp_shape* shape, float* params, const float* grads, float* m,
                   float* v, int64_t t, float lr, float beta1, float beta2, float eps,
                   uint16_t* params_bf16, void* stream) {
    if (!mlp_args(shape, params, params_bf16) || !grads || !m || !v || t < 1) return ETICS_ERR_ARG;
    if (!aligned(grads, 4) || !aligned(m, 4) || !aligned(v, 4)) return ETICS_ERR_ARG;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f &&
          lr == lr))
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::mlp_adam(shape, params, grads, m, v, t, lr, beta1, beta2, eps, params_bf16,
                           h.ctx);
}

int etics_mlp_to_bf16(const etics_mlp_shape* shape, const float* params, uint16_t* params_bf16,
                      void* stream) {
    if (!mlp_args(shape, params, params_bf16)) return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::mlp_to_bf16(shape, params, params_bf16, h.ctx);
}

int etics_coeff_stats(const double* traj, int T, int D, int stride, double* norm, void* stream) {
    if (!traj || !norm || T < 5 || D < 1 || stride < 1 || stride > 4 || !aligned(traj, 8) ||
        !aligned(norm, 8))
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::coeff_stats(traj, T, D, stride, norm, h.ctx);
}

int etics_coeff_features(const double* store, const int32_t* rows, const int32_t* next_rows,
                         int batch, int D, int stride, const double* norm, int layout, uint16_t* x,
                         float* target, void* stream) {
    if (!store || !rows || !norm || !x || batch < 0 || D < 1 || (next_rows && !target) ||
        stride < 1 || stride > 4)
        return ETICS_ERR_ARG;
    if (layout != ETICS_FEAT_JOINT && layout != ETICS_FEAT_PER_COEFF) return ETICS_ERR_ARG;
    if (!aligned(store, 8) || !aligned(rows, 4) || !aligned(norm, 8) || !aligned(x, 2) ||
        (next_rows && (!aligned(next_rows, 4) || !aligned(target, 4))))
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::coeff_features(store, rows, next_rows, batch, D, stride, norm,
                                 layout == ETICS_FEAT_PER_COEFF, x, target, h.ctx);
}

int etics_coeff_advance(double* ring, int32_t* order, int D, int stride, int horizon,
                        const double* coeffs_in, const float* y, int y_stride, const double* norm,
                        double* coeffs_out, int commit, void* stream) {
    if (!ring || !order || D < 1 || (!coeffs_in == !y) || (y && !norm)) return ETICS_ERR_ARG;
    if (y && (stride < 1 || stride > 4 || horizon < 1 || horizon > stride || y_stride < 1))
        return ETICS_ERR_ARG;
    if (!commit && !coeffs_out) return ETICS_ERR_ARG;
    if (!aligned(ring, 8) || !aligned(order, 4) || (coeffs_in && !aligned(coeffs_in, 8)) ||
        (y && !aligned(y, 4)) || (coeffs_out && !aligned(coeffs_out, 8)))
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::coeff_advance(ring, order, D, stride, horizon, coeffs_in, y, y_stride, norm,
                                coeffs_out, commit, h.ctx);
}

int etics_force_error(const void* a, const void* r, int64_t N, int precision, double tol_a,
                      double tol_b, uint64_t* out, void* stream) {
    if (!valid_n(N) || !valid_precision(precision) || !out || !aligned(out, 8)) return ETICS_ERR_ARG;
    if (check_particles(a, N) || check_particles(r, N)) return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::force_error(a, r, N, precision, tol_a, tol_b, out, h.ctx);
}

int etics_scf_batch_plan(const etics_batch_item* items, int ninst,
                         const etics_batch_tuning* tuning, int precision, void* plan,
                         size_t plan_bytes, size_t* plan_bytes_needed, size_t* ws_bytes,
                         int64_t* coeff_count) {
    if (!valid_precision(precision) || ninst <= 0 || !items || !plan_bytes_needed)
        return ETICS_ERR_ARG;
    unsigned* err = nullptr;
    int sms = 0;
    const int rc = current_device_state(&err, &sms);
    if (rc) return rc;
    return etics::batch_plan_build(items, ninst, tuning, sms, precision, plan, plan_bytes,
                                   plan_bytes_needed, ws_bytes, coeff_count);
}

int etics_scf_batch(const void* posm, const void* plan_host, const void* plan_dev, int precision,
                    double* coeffs, void* accpot, int out_mask, void* ws, size_t ws_bytes,
                    void* stream) {
    if (!valid_precision(precision) || !plan_host || !plan_dev || !coeffs || !ws) return ETICS_ERR_ARG;
    if (!aligned(posm, 16) || !aligned(coeffs, 8) || !aligned(ws, 256) || !aligned(plan_dev, 16))
        return ETICS_ERR_ARG;
    if (accpot && (!aligned(accpot, 16) || (out_mask & (ETICS_OUT_ACC | ETICS_OUT_POT)) == 0 ||
                   (out_mask & ~3)))
        return ETICS_ERR_ARG;
    CtxHolder h;
    int rc = make_ctx(stream, h);
    if (rc) return rc;
    etics::stage_event(h.ctx, 0);
    return precision == ETICS_MIXED
               ? etics::batch_launch<float>(posm, plan_host, plan_dev, coeffs, accpot, out_mask, ws,
                                            ws_bytes, h.ctx)
               : etics::batch_launch<double>(posm, plan_host, plan_dev, coeffs, accpot, out_mask,
                                             ws, ws_bytes, h.ctx);
}

int etics_get_error(void* stream) {
    unsigned* err = nullptr;
    int sms = 0;
    if (current_device_state(&err, &sms)) return ETICS_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned host = 0;
    if (cudaMemcpyAsync(&host, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return ETICS_ERR_CUDA;
    if (cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return ETICS_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return ETICS_ERR_CUDA;
    return host ? -(int)host : ETICS_OK;
}

const char* etics_strerror(int status) {
    switch (status) {
        case ETICS_OK: return "ok";
        case ETICS_ERR_ARG: return "invalid argument";
        case ETICS_ERR_CUDA: return "CUDA runtime error";
        case ETICS_ERR_WORKSPACE: return "workspace too small";
        case ETICS_ERR_NONFINITE: return "non-finite input or FP32 overflow";
        case ETICS_ERR_TIMEOUT: return "inter-block wait timed out";
        case ETICS_ERR_UNSUPPORTED: return "parameters beyond the compiled limits";
        default: return "unknown status";
    }
}

uint64_t etics_launch_count(void) { return g_launches.load(); }

int etics_set_wait_limit(int64_t spins) {
    if (spins < 0) return ETICS_ERR_ARG;
    g_wait_limit = spins;
    return ETICS_OK;
}

int etics_test_wait_timeout(int which, int64_t spins, void* ws, size_t ws_bytes, void* stream) {
    if (spins < 0) return ETICS_ERR_ARG;
    if (which != ETICS_WAIT_LOOKBACK && which != ETICS_WAIT_MBARRIER) return ETICS_ERR_ARG;
    if (which == ETICS_WAIT_LOOKBACK) {
        if (!ws || !aligned(ws, 256)) return ETICS_ERR_ARG;
        if (ws_bytes < etics_workspace_bytes(etics::kTimeoutProbeN, 0, 0, ETICS_MEX, ETICS_MIXED))
            return ETICS_ERR_WORKSPACE;
    }
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return which == ETICS_WAIT_LOOKBACK ? etics::lookback_timeout_probe(ws, spins, h.ctx)
                                        : etics::mbarrier_timeout_probe(spins, h.ctx);
}

int etics_fma_peak(int kind, int blocks, int64_t iters, float* sink, double* flops_host,
                   void* stream) {
    if (kind != ETICS_PEAK_FFMA && kind != ETICS_PEAK_FFMA2 && kind != ETICS_PEAK_DFMA)
        return ETICS_ERR_ARG;
    if (blocks < 1 || blocks > (1 << 20) || iters < 0 || !sink || !aligned(sink, 4) ||
        !flops_host)
        return ETICS_ERR_ARG;
    CtxHolder h;
    const int rc = make_ctx(stream, h);
    if (rc) return rc;
    return etics::fma_peak(kind, blocks, iters, sink, flops_host, h.ctx);
}

int etics_set_stage_events(void** events, int n_events) {
    if (n_events < 0 || (n_events > 0 && !events)) return ETICS_ERR_ARG;
    g_events = n_events > 0 ? events : nullptr;
    g_n_events = n_events;
    return ETICS_OK;
}

}  // extern "C"
