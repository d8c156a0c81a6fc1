// etics_step.cu -- the kick and drift halves of the kick-drift-kick leapfrog
// step that surrounds the force calculation (paper Secs. 3.4 and 5.4).
#include "etics_internal.h"

namespace etics {

template <typename R>
__global__ void kick_drift_kernel(Vec4<R>* __restrict__ posm, Vec4<R>* __restrict__ vel,
                                  const Vec4<R>* __restrict__ acc, int64_t N, R dt) {
    const R h = R(0.5) * dt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        Vec4<R> v = ld4(vel + i);
        const Vec4<R> a = ld4(acc + i);
        Vec4<R> x = ld4(posm + i);
        v.x = fma(h, a.x, v.x);
        v.y = fma(h, a.y, v.y);
        v.z = fma(h, a.z, v.z);
        x.x = fma(dt, v.x, x.x);
        x.y = fma(dt, v.y, x.y);
        x.z = fma(dt, v.z, x.z);
        st4(vel + i, v);
        st4(posm + i, x);
    }
}

template <typename R>
__global__ void kick_kernel(Vec4<R>* __restrict__ vel, const Vec4<R>* __restrict__ acc, int64_t N,
                            R dt) {
    const R h = R(0.5) * dt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        Vec4<R> v = ld4(vel + i);
        const Vec4<R> a = ld4(acc + i);
        v.x = fma(h, a.x, v.x);
        v.y = fma(h, a.y, v.y);
        v.z = fma(h, a.z, v.z);
        st4(vel + i, v);
    }
}

static int grid_for(int64_t N, const LaunchCtx& ctx) {
    int64_t g = (N + 255) / 256;
    const int64_t cap = (int64_t)ctx.num_sms * 16;
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

template <typename R>
static int kick_drift_impl(void* posm, void* vel, const void* acc, int64_t N, double dt,
                           const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    kick_drift_kernel<R><<<grid_for(N, ctx), 256, 0, ctx.stream>>>(
        reinterpret_cast<Vec4<R>*>(posm), reinterpret_cast<Vec4<R>*>(vel),
        reinterpret_cast<const Vec4<R>*>(acc), N, (R)dt);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

template <typename R>
static int kick_impl(void* vel, const void* acc, int64_t N, double dt, const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    kick_kernel<R><<<grid_for(N, ctx), 256, 0, ctx.stream>>>(
        reinterpret_cast<Vec4<R>*>(vel), reinterpret_cast<const Vec4<R>*>(acc), N, (R)dt);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

int kick_drift_f32(void* p, void* v, const void* a, int64_t N, double dt, const LaunchCtx& c) {
    return kick_drift_impl<float>(p, v, a, N, dt, c);
}
int kick_drift_f64(void* p, void* v, const void* a, int64_t N, double dt, const LaunchCtx& c) {
    return kick_drift_impl<double>(p, v, a, N, dt, c);
}
int kick_f32(void* v, const void* a, int64_t N, double dt, const LaunchCtx& c) {
    return kick_impl<float>(v, a, N, dt, c);
}
int kick_f64(void* v, const void* a, int64_t N, double dt, const LaunchCtx& c) {
    return kick_impl<double>(v, a, N, dt, c);
}

}  // namespace etics
