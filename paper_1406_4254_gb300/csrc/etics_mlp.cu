// etics_mlp.cu -- the coefficient-forecasting MLP: bf16 tensor-core products
// with FP32 accumulation, its training (MSE loss, back-propagation, Adam) and
// the FP64 glue that turns a history of SCF coefficient vectors into network
// inputs and a network output back into the next coefficient vector.
//
// The paper has no learned part; the forecast replaces plain reuse of the
// coefficients over several steps (temporal softening, end of Sec. 4.1), so
// that the coefficient pass (the first of the two SCF passes, Sec. 3.3) can be
// skipped on most steps.
//
// Rounding points (the oracle's quantize=True mirrors them): every matrix
// product takes bf16 operands (weights, the inputs, hidden activations and
// back-propagated errors) and accumulates in FP32; biases, tanh, the loss, its
// gradient and Adam run in FP32; the feature / update glue in FP64.
//
// Products run as C_part[s] = op(A) op(B) over K-slice s (split-K, slices
// written to separate buffers) followed by an epilogue kernel that sums the
// slices in a fixed order, so every result is deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "etics_internal.h"
#include "etics_tc.cuh"

namespace etics {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 32, kPadK = 8;
constexpr int kGemmThreads = 128;
constexpr int kLossBlocks = 256;
constexpr int kTargetBlocks = 304;      // two blocks per SM on a 152-SM part

using bf16 = __nv_bfloat16;

__device__ __forceinline__ void mma_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Stage a (64 x 32) operand tile into smem as T[r][k] (k contiguous).
//  KM: the operand is stored with k contiguous: X[r * ld + k]
//  RM: the operand is stored with r contiguous: X[k * ld + r]
// Out-of-range elements (r >= R, k >= ke) are zero.
template <bool RM>
__device__ __forceinline__ void load_tile(bf16 (*T)[kBK + kPadK], const bf16* __restrict__ X,
                                          int64_t ld, int r0, int R, int k0, int ke, int tid) {
    const bf16 zero = __float2bfloat16_rn(0.0f);
    if (!RM) {
        const int r = tid >> 1, kh = (tid & 1) * 16;
        const int gr = r0 + r, gk = k0 + kh;
        const bf16* src = X + (int64_t)gr * ld + gk;
        if (gr < R && gk + 16 <= ke && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const uint4 v0 = *reinterpret_cast<const uint4*>(src);
            const uint4 v1 = *reinterpret_cast<const uint4*>(src + 8);
            *reinterpret_cast<uint4*>(&T[r][kh]) = v0;
            *reinterpret_cast<uint4*>(&T[r][kh + 8]) = v1;
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
                T[r][kh + e] = (gr < R && gk + e < ke) ? src[e] : zero;
        }
    } else {
        const int k = tid >> 2, rc = (tid & 3) * 16;
        const int gk = k0 + k, gr = r0 + rc;
        const bf16* src = X + (int64_t)gk * ld + gr;
        if (gk < ke && gr + 16 <= R && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            uint4 v[2];
            v[0] = *reinterpret_cast<const uint4*>(src);
            v[1] = *reinterpret_cast<const uint4*>(src + 8);
            const bf16* e16 = reinterpret_cast<const bf16*>(v);
#pragma unroll
            for (int e = 0; e < 16; ++e) T[rc + e][k] = e16[e];
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e)
                T[rc + e][k] = (gk < ke && gr + e < R) ? src[e] : zero;
        }
    }
}

// part[z][M][N] = sum over k in slice z of A(m, k) B(k, n).
//  A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]
//  B(k, n) = TB ? B[k * ldb + n] : B[n * ldb + k]
// 64 x 64 block tile, four warps of 32 x 32, m16n8k16 bf16 MMAs.
template <bool TA, bool TB>
__global__ void __launch_bounds__(kGemmThreads)
mlp_gemm_kernel(const bf16* __restrict__ A, int64_t lda, const bf16* __restrict__ B, int64_t ldb,
                float* __restrict__ part, int M, int N, int K, int kslice) {
    __shared__ __align__(16) bf16 As[kBM][kBK + kPadK];
    __shared__ __align__(16) bf16 Bs[kBN][kBK + kPadK];
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int kb = blockIdx.z * kslice;
    const int ke = min(K, kb + kslice);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.0f;
    for (int k0 = kb; k0 < ke; k0 += kBK) {
        load_tile<TA>(As, A, lda, m0, M, k0, ke, tid);
        load_tile<TB>(Bs, B, ldb, n0, N, k0, ke, tid);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * t + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][kk + 2 * t + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_16816(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
    float* out = part + (size_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + wm + i * 16 + g;
            const int c = n0 + wn + j * 8 + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int rr = r + 8 * h;
                if (rr >= M) continue;
                if (c < N) out[(size_t)rr * N + c] = acc[i][j][2 * h];
                if (c + 1 < N) out[(size_t)rr * N + c + 1] = acc[i][j][2 * h + 1];
            }
        }
}

// sum of the K slices (in slice order) + bias, then tanh or the tanh
// derivative factor (1 - h^2); FP32 and/or bf16 outputs
__global__ void mlp_epilogue_kernel(const float* __restrict__ part, int splits, int M, int N,
                                    const float* __restrict__ bias, int act,
                                    const float* __restrict__ h, float* __restrict__ out,
                                    bf16* __restrict__ out_b) {
    const int64_t MN = (int64_t)M * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN;
         i += (int64_t)gridDim.x * blockDim.x) {
        float s = part[i];
        for (int z = 1; z < splits; ++z) s += part[(size_t)z * MN + i];
        if (bias) s += bias[i % N];
        if (act) s = tanhf(s);
        if (h) {
            const float hv = h[i];
            s *= 1.0f - hv * hv;
        }
        if (out) out[i] = s;
        if (out_b) out_b[i] = __float2bfloat16_rn(s);
    }
}

// dY = 2 (Y - T) / count (FP32 and bf16); per-block FP64 partial sums of
// (Y - T)^2 in a fixed grid, summed by mlp_loss_final_kernel
__global__ void __launch_bounds__(256)
mlp_mse_kernel(const float* __restrict__ y, const float* __restrict__ tg, int64_t count,
               float scale, float* __restrict__ dy, bf16* __restrict__ dyb,
               double* __restrict__ block_sums) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = y[i] - tg[i];
        s += (double)d * (double)d;
        const float gv = scale * d;
        dy[i] = gv;
        dyb[i] = __float2bfloat16_rn(gv);
    }
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; ++w) b += red[w];
        block_sums[blockIdx.x] = b;
    }
}

__global__ void mlp_loss_final_kernel(const double* __restrict__ block_sums, int n,
                                      double inv_count, double* __restrict__ loss) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += block_sums[i];
        *loss = s * inv_count;
    }
}

// db[n] = sum over rows of dz[m][n] in two deterministic stages: FP64 sums
// of row chunk blockIdx.y (rows in order), then the chunk sums in order
constexpr int kColChunks = 128;

__global__ void mlp_colsum_partial_kernel(const float* __restrict__ dz, int M, int N, int rows,
                                          double* __restrict__ part) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const int m0 = blockIdx.y * rows, m1 = min(M, m0 + rows);
    double s = 0.0;
    for (int m = m0; m < m1; ++m) s += dz[(size_t)m * N + n];
    part[(size_t)blockIdx.y * N + n] = s;
}

__global__ void mlp_colsum_final_kernel(const double* __restrict__ part, int chunks, int N,
                                        float* __restrict__ db) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += part[(size_t)c * N + n];
    db[n] = (float)s;
}

__global__ void mlp_adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                                float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                                float b1, float b2, float eps, float bc1, float bc2,
                                bf16* __restrict__ pb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
        p[i] = pi;
        pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void mlp_to_bf16_kernel(const float* __restrict__ p, int64_t n, bf16* __restrict__ pb) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        pb[i] = __float2bfloat16_rn(p[i]);
}

// ---- forecast glue (FP64, single roundings in the written order) -----------
// A forecast works on a history of eight true coefficient vectors c_0..c_7
// (oldest first) spaced `stride` steps apart, and predicts the vector k steps
// after c_7 for each horizon k = 1..stride.  Differences are backward
// differences along the history (d1_i = c_i - c_{i-1}, ...).
constexpr int kHist = 8;
constexpr int kLinFeat = 7;
constexpr int kMaxStride = 4;

__device__ __forceinline__ bf16 to_bf16(double v) { return __float2bfloat16_rn((float)v); }

// normaliser rows: mu, 1/sigma, 1/s1, 1/s2, 1/s3, 1/s4, s4 (scales of the
// stride-spaced differences), then per horizon k (from row 7 + 9 (k-1)):
// the fitted linear predictor beta_k[0..6], the RMS q_k of its residual, 1/q_k
__host__ __device__ constexpr int norm_rows(int stride) { return 7 + 9 * stride; }
__host__ __device__ constexpr int norm_beta(int k) { return 7 + 9 * (k - 1); }

// backward differences of NV values: dk[i] = k-th difference ending at c[i],
// one FP64 subtraction each
template <int NV>
__device__ __forceinline__ void differences(const double (&c)[NV], double (&d1)[NV],
                                            double (&d2)[NV], double (&d3)[NV], double (&d4)[NV]) {
#pragma unroll
    for (int i = 1; i < NV; ++i) d1[i] = __dsub_rn(c[i], c[i - 1]);
#pragma unroll
    for (int i = 2; i < NV; ++i) d2[i] = __dsub_rn(d1[i], d1[i - 1]);
#pragma unroll
    for (int i = 3; i < NV; ++i) d3[i] = __dsub_rn(d2[i], d2[i - 1]);
#pragma unroll
    for (int i = 4; i < NV; ++i) d4[i] = __dsub_rn(d3[i], d3[i - 1]);
}

// regressors of a history (differences ending at c_7 over their RMS): the
// network's feature blocks 1..7 before their bf16 rounding
__device__ __forceinline__ void lin_regressors(const double (&d1)[kHist], const double (&d2)[kHist],
                                               const double (&d3)[kHist], const double (&d4)[kHist],
                                               const double* __restrict__ norm, int D, int j,
                                               double (&u)[kLinFeat]) {
    const double is4 = norm[(size_t)5 * D + j];
    u[0] = __dmul_rn(d1[7], norm[(size_t)2 * D + j]);
    u[1] = __dmul_rn(d2[7], norm[(size_t)3 * D + j]);
    u[2] = __dmul_rn(d3[7], norm[(size_t)4 * D + j]);
#pragma unroll
    for (int k = 0; k < 4; ++k) u[3 + k] = __dmul_rn(d4[7 - k], is4);
}

// beta_k . u, summed left to right
__device__ __forceinline__ double lin_predict(const double (&u)[kLinFeat],
                                              const double* __restrict__ norm, int D, int j, int k) {
    const double* bk = norm + (size_t)norm_beta(k) * D + j;
    double s = __dmul_rn(bk[0], u[0]);
#pragma unroll
    for (int i = 1; i < kLinFeat; ++i) s = __dadd_rn(s, __dmul_rn(bk[(size_t)i * D], u[i]));
    return s;
}

// the cubic through c_4..c_7 evaluated k/stride of a spacing after c_7
// (Newton's backward form): ((c_7 + s d1_7) + s(s+1)/2 d2_7) + s(s+1)(s+2)/6 d3_7
__device__ __forceinline__ double cubic_base(double c7, double d1, double d2, double d3, int k,
                                             int stride) {
    const double s = __ddiv_rn((double)k, (double)stride);
    const double a2 = __dmul_rn(__dmul_rn(s, __dadd_rn(s, 1.0)), 0.5);
    const double a3 = __ddiv_rn(__dmul_rn(a2, __dadd_rn(s, 2.0)), 3.0);
    return __dadd_rn(__dadd_rn(__dadd_rn(c7, __dmul_rn(s, d1)), __dmul_rn(a2, d2)), __dmul_rn(a3, d3));
}

// rows 0-6 of a trajectory traj[T][D] (one thread per coefficient): the mean,
// 1/standard deviation, 1/RMS of the k-th stride-spaced backward differences
// (k = 1..4, over every t where they exist) and s4; a reciprocal of a zero
// scale is 0
__global__ void coeff_stats_kernel(const double* __restrict__ traj, int T, int D, int stride,
                                   double* __restrict__ norm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    double s = 0.0;
    for (int t = 0; t < T; ++t) s += traj[(size_t)t * D + j];
    const double mu = s / T;
    double v = 0.0;
    for (int t = 0; t < T; ++t) {
        const double c = traj[(size_t)t * D + j];
        v += (c - mu) * (c - mu);
    }
    double q[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = stride; t < T; ++t) {
        double c[5], d1[5], d2[5], d3[5], d4[5];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const int ti = t - (4 - i) * stride;
            c[i] = ti >= 0 ? traj[(size_t)ti * D + j] : 0.0;
        }
        differences<5>(c, d1, d2, d3, d4);
        q[1] += d1[4] * d1[4];
        if (t >= 2 * stride) q[2] += d2[4] * d2[4];
        if (t >= 3 * stride) q[3] += d3[4] * d3[4];
        if (t >= 4 * stride) q[4] += d4[4] * d4[4];
    }
    norm[j] = mu;
    const double sigma = sqrt(v / T);
    norm[(size_t)D + j] = sigma > 0.0 ? 1.0 / sigma : 0.0;
    double sk = 0.0;
    for (int k = 1; k <= 4; ++k) {
        const int cnt = T - k * stride;
        sk = cnt > 0 ? sqrt(q[k] / cnt) : 0.0;
        norm[(size_t)(1 + k) * D + j] = sk > 0.0 ? 1.0 / sk : 0.0;
    }
    norm[(size_t)6 * D + j] = sk;
}

// history c_0..c_7 ending at trajectory index t (stride apart), its
// differences and regressors
__device__ __forceinline__ void traj_history(const double* __restrict__ traj, int D, int j, int t,
                                             int stride, const double* __restrict__ norm,
                                             double (&c)[kHist], double (&d1)[kHist],
                                             double (&d2)[kHist], double (&d3)[kHist],
                                             double (&u)[kLinFeat]) {
    double d4[kHist];
#pragma unroll
    for (int i = 0; i < kHist; ++i) c[i] = traj[(size_t)(t - (kHist - 1 - i) * stride) * D + j];
    differences<kHist>(c, d1, d2, d3, d4);
    lin_regressors(d1, d2, d3, d4, norm, D, j, u);
}

// the fitted linear predictors of every coefficient (one thread each): over
// every history of the trajectory with all its horizons inside it (newest
// index t from 7 stride to T-1-stride), the target of horizon k,
// t_k = (c_{t+k} - cubic_k) / s4, is regressed by least squares on the
// regressors u: G beta_k = h_k with G = sum u u^T + lambda tr(G)/7 I
// (lambda = 1e-12; beta = 0 where G vanishes), solved by Cholesky; q_k = RMS
// of t_k - beta_k . u over the same histories (q = 1, beta = 0 without any)
__global__ void coeff_linfit_kernel(const double* __restrict__ traj, int T, int D, int stride,
                                    double* __restrict__ norm) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= D) return;
    constexpr int F = kLinFeat;
    double G[F][F], h[kMaxStride][F];
#pragma unroll
    for (int a = 0; a < F; ++a) {
#pragma unroll
        for (int k = 0; k < kMaxStride; ++k) h[k][a] = 0.0;
#pragma unroll
        for (int b = 0; b < F; ++b) G[a][b] = 0.0;
    }
    const double is4 = norm[(size_t)5 * D + j];
    const int t_lo = (kHist - 1) * stride, t_hi = T - 1 - stride;
    auto target = [&](const double (&c)[kHist], const double (&d1)[kHist], const double (&d2)[kHist],
                      const double (&d3)[kHist], int t, int k) -> double {
        const double base = cubic_base(c[7], d1[7], d2[7], d3[7], k, stride);
        return __dmul_rn(__dsub_rn(traj[(size_t)(t + k) * D + j], base), is4);
    };
    for (int t = t_lo; t <= t_hi; ++t) {
        double c[kHist], d1[kHist], d2[kHist], d3[kHist], u[F];
        traj_history(traj, D, j, t, stride, norm, c, d1, d2, d3, u);
#pragma unroll
        for (int a = 0; a < F; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) G[a][b] += u[a] * u[b];
#pragma unroll
        for (int k = 0; k < kMaxStride; ++k) {
            if (k >= stride) break;
            const double tg = target(c, d1, d2, d3, t, k + 1);
#pragma unroll
            for (int a = 0; a < F; ++a) h[k][a] += u[a] * tg;
        }
    }
    double tr = 0.0;
#pragma unroll
    for (int a = 0; a < F; ++a) tr += G[a][a];
    const bool solve = t_hi >= t_lo && tr > 0.0;
    if (solve) {
        const double ridge = 1e-12 * tr / F;
        // Cholesky G = L L^T (lower triangle of G overwritten by L)
#pragma unroll
        for (int a = 0; a < F; ++a) {
            double dsum = G[a][a] + ridge;
#pragma unroll
            for (int k = 0; k < a; ++k) dsum -= G[a][k] * G[a][k];
            const double lkk = sqrt(dsum > 0.0 ? dsum : 0.0);
            G[a][a] = lkk;
#pragma unroll
            for (int b = a + 1; b < F; ++b) {
                double v = G[b][a];
#pragma unroll
                for (int k = 0; k < a; ++k) v -= G[b][k] * G[a][k];
                G[b][a] = lkk > 0.0 ? v / lkk : 0.0;
            }
        }
    }
    for (int k = 1; k <= stride; ++k) {
        double beta[F];
#pragma unroll
        for (int a = 0; a < F; ++a) beta[a] = 0.0;
        if (solve) {
            double z[F];
#pragma unroll
            for (int a = 0; a < F; ++a) {       // L z = h_k
                double v = h[k - 1][a];
#pragma unroll
                for (int i = 0; i < a; ++i) v -= G[a][i] * z[i];
                z[a] = G[a][a] > 0.0 ? v / G[a][a] : 0.0;
            }
#pragma unroll
            for (int a = F - 1; a >= 0; --a) {  // L^T beta_k = z
                double v = z[a];
#pragma unroll
                for (int i = a + 1; i < F; ++i) v -= G[i][a] * beta[i];
                beta[a] = G[a][a] > 0.0 ? v / G[a][a] : 0.0;
            }
        }
#pragma unroll
        for (int a = 0; a < F; ++a) norm[(size_t)(norm_beta(k) + a) * D + j] = beta[a];
    }
    for (int k = 1; k <= stride; ++k) {
        double q = 1.0;
        if (t_hi >= t_lo) {
            double ss = 0.0;
            for (int t = t_lo; t <= t_hi; ++t) {
                double c[kHist], d1[kHist], d2[kHist], d3[kHist], u[F];
                traj_history(traj, D, j, t, stride, norm, c, d1, d2, d3, u);
                const double r = __dsub_rn(target(c, d1, d2, d3, t, k), lin_predict(u, norm, D, j, k));
                ss += r * r;
            }
            q = sqrt(ss / (t_hi - t_lo + 1));
        }
        norm[(size_t)(norm_beta(k) + 7) * D + j] = q;
        norm[(size_t)(norm_beta(k) + 8) * D + j] = q > 0.0 ? 1.0 / q : 0.0;
    }
}

// features of the history store[rows[b][0..7]] (oldest first), block blk of
// coefficient j at x[b][blk * D + j] (joint layout: one row per history) or at
// x[b * D + j][blk] (per-coefficient layout: one row per coefficient); with
// next, the targets of the horizons k = 1..stride (next vectors
// store[next[b][k-1]]): what the fitted predictor misses, over q_k, at
// target[(b * D + j) * stride + k-1] (per coefficient) or
// target[(b * stride + k-1) * D + j] (joint)
__global__ void coeff_features_kernel(const double* __restrict__ store,
                                      const int32_t* __restrict__ rows,
                                      const int32_t* __restrict__ next, int B, int D, int stride,
                                      const double* __restrict__ norm, int per_coeff,
                                      bf16* __restrict__ x, float* __restrict__ target) {
    const int64_t total = (int64_t)B * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / D), j = (int)(i % D);
        double c[kHist], d1[kHist], d2[kHist], d3[kHist], d4[kHist];
#pragma unroll
        for (int k = 0; k < kHist; ++k) c[k] = store[(size_t)rows[b * kHist + k] * D + j];
        differences<kHist>(c, d1, d2, d3, d4);
        const double is4 = norm[(size_t)5 * D + j];
        // element stride between blocks and the position of block 0
        const size_t bs = per_coeff ? 1 : (size_t)D;
        bf16* xr = per_coeff ? x + (size_t)i * kHist : x + (size_t)b * kHist * D + j;
        xr[0] = to_bf16(__dmul_rn(__dsub_rn(c[7], norm[j]), norm[(size_t)D + j]));
        xr[bs] = to_bf16(__dmul_rn(d1[7], norm[(size_t)2 * D + j]));
        xr[2 * bs] = to_bf16(__dmul_rn(d2[7], norm[(size_t)3 * D + j]));
        xr[3 * bs] = to_bf16(__dmul_rn(d3[7], norm[(size_t)4 * D + j]));
#pragma unroll
        for (int k = 0; k < 4; ++k) xr[(size_t)(4 + k) * bs] = to_bf16(__dmul_rn(d4[7 - k], is4));
        if (next) {
            double u[kLinFeat];
            lin_regressors(d1, d2, d3, d4, norm, D, j, u);
            for (int k = 1; k <= stride; ++k) {
                const double cn = store[(size_t)next[b * stride + k - 1] * D + j];
                const double tk = __dmul_rn(
                    __dsub_rn(cn, cubic_base(c[7], d1[7], d2[7], d3[7], k, stride)), is4);
                const double tau = __dmul_rn(__dsub_rn(tk, lin_predict(u, norm, D, j, k)),
                                             norm[(size_t)(norm_beta(k) + 8) * D + j]);
                const size_t o = per_coeff ? (size_t)i * stride + (k - 1)
                                           : ((size_t)b * stride + (k - 1)) * D + j;
                target[o] = (float)tau;
            }
        }
    }
}

// a forecast or a push.  Forecast (y given): the vector k steps after the
// ring's newest, cubic_k + s4 (beta_k . u + q_k y[j * y_stride]); with
// commit it is also written into the oldest slot.  Push (cin given): cin is
// written into the oldest slot.  A write rotates the slot order.  One block.
constexpr int kAdvanceThreads = 256;
__global__ void __launch_bounds__(kAdvanceThreads)
coeff_advance_kernel(double* __restrict__ ring, int32_t* __restrict__ order, int D,
                                     int stride, int k, const double* cin,
                                     const float* __restrict__ y, int y_stride,
                                     const double* __restrict__ norm, double* cout, int commit) {
    __shared__ int32_t o[kHist];
    if (threadIdx.x < kHist) o[threadIdx.x] = order[threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.x; j < D; j += blockDim.x) {
        double nv;
        if (cin) {
            nv = cin[j];
        } else {
            double c[kHist], d1[kHist], d2[kHist], d3[kHist], d4[kHist], u[kLinFeat];
#pragma unroll
            for (int i = 0; i < kHist; ++i) c[i] = ring[(size_t)o[i] * D + j];
            differences<kHist>(c, d1, d2, d3, d4);
            lin_regressors(d1, d2, d3, d4, norm, D, j, u);
            const double base = cubic_base(c[7], d1[7], d2[7], d3[7], k, stride);
            const double t4 = __dadd_rn(lin_predict(u, norm, D, j, k),
                                        __dmul_rn(norm[(size_t)(norm_beta(k) + 7) * D + j],
                                                  (double)y[(size_t)j * y_stride]));
            nv = __dadd_rn(base, __dmul_rn(norm[(size_t)6 * D + j], t4));
        }
        if (commit) ring[(size_t)o[0] * D + j] = nv;
        if (cout) cout[j] = nv;
    }
    __syncthreads();
    if (commit && threadIdx.x < kHist) order[threadIdx.x] = o[(threadIdx.x + 1) % kHist];
}

// relative acceleration error e_i = |a_i - r_i| / |r_i| (Sec. 4.2): counts of
// e_i > tol_a and e_i > tol_b and the largest e_i (atomics on integers and on
// the order-preserving bits of a non-negative double: deterministic)
template <typename R>
__global__ void force_error_kernel(const Vec4<R>* __restrict__ a, const Vec4<R>* __restrict__ r,
                                   int64_t N, double tol_a, double tol_b,
                                   unsigned long long* __restrict__ out) {
    unsigned long long ca = 0, cb = 0, mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Vec4<R> u = ld4(a + i), v = ld4(r + i);
        const double dx = (double)u.x - (double)v.x, dy = (double)u.y - (double)v.y,
                     dz = (double)u.z - (double)v.z;
        const double nr = sqrt((double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z);
        const double nd = sqrt(dx * dx + dy * dy + dz * dz);
        const double e = nr > 0.0 ? nd / nr : (nd > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0);
        ca += e > tol_a;
        cb += e > tol_b;
        const unsigned long long bits = (unsigned long long)__double_as_longlong(e);
        mx = bits > mx ? bits : mx;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ca += __shfl_xor_sync(0xffffffffu, ca, o);
        cb += __shfl_xor_sync(0xffffffffu, cb, o);
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        if (ca) atomicAdd(out, ca);
        if (cb) atomicAdd(out + 1, cb);
        atomicMax(out + 2, mx);
    }
}

// ---- host planning ---------------------------------------------------------
// A product runs on the tcgen05 kernel (128 x 128 tiles, K step 64) when both
// output dimensions fill a tile at least half, else on the mma.sync kernel
// (64 x 64 tiles, K step 32).  Split-K brings the block count near two per SM
// while keeping >= 4 (mma.sync) or >= 2 (tcgen05) K steps per slice.
struct GemmShape { int M, N, K, splits, kslice; bool tc; };

GemmShape gemm_shape(int M, int N, int K) {
    GemmShape s{M, N, K, 1, 0, M >= 64 && N >= 64};
    const int bm = s.tc ? tc::kM : kBM, bn = s.tc ? tc::kN : kBN, bk = s.tc ? tc::kK : kBK;
    const int tiles = ((M + bm - 1) / bm) * ((N + bn - 1) / bn);
    const int ktiles = (K + bk - 1) / bk;
    int splits = (kTargetBlocks + tiles - 1) / tiles;
    const int min_steps = s.tc ? 2 : 4;
    const int max_splits = ktiles / min_steps > 1 ? ktiles / min_steps : 1;
    if (splits > max_splits) splits = max_splits;
    if (splits > 64) splits = 64;
    if (splits < 1) splits = 1;
    const int per = (ktiles + splits - 1) / splits;
    s.kslice = per * bk;
    s.splits = (ktiles + per - 1) / per;
    return s;
}

struct MlpLayout {
    int L;
    int d[6];
    int64_t woff[5], boff[5];          // parameter offsets
    int64_t nparam;
    int dmax;
    // workspace offsets (bytes)
    size_t h32[5], hb[5], y32, dz32[2], dzb[2], part, loss_blocks, colsum, total;
};

bool valid_shape(const etics_mlp_shape* s) {
    if (!s || s->nlayers < 1 || s->nlayers > ETICS_MLP_MAX_LAYERS) return false;
    for (int i = 0; i <= s->nlayers; ++i)
        if (s->dims[i] < 1 || s->dims[i] > (1 << 20)) return false;
    return true;
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

MlpLayout mlp_layout(const etics_mlp_shape* s, int B) {
    MlpLayout o{};
    o.L = s->nlayers;
    int64_t p = 0;
    o.dmax = 0;
    for (int i = 0; i <= o.L; ++i) {
        o.d[i] = s->dims[i];
        if (o.d[i] > o.dmax) o.dmax = o.d[i];
    }
    for (int i = 0; i < o.L; ++i) {
        o.woff[i] = p;
        p += (int64_t)o.d[i] * o.d[i + 1];
        o.boff[i] = p;
        p += o.d[i + 1];
    }
    o.nparam = p;
    size_t off = 0;
    const size_t Bz = (size_t)(B > 0 ? B : 1);
    for (int i = 0; i + 1 < o.L; ++i) {
        o.h32[i] = off; off += al256(Bz * o.d[i + 1] * 4);
        o.hb[i] = off;  off += al256(Bz * o.d[i + 1] * 2);
    }
    o.y32 = off; off += al256(Bz * o.d[o.L] * 4);
    for (int k = 0; k < 2; ++k) {
        o.dz32[k] = off; off += al256(Bz * o.dmax * 4);
        o.dzb[k] = off;  off += al256(Bz * o.dmax * 2);
    }
    // the largest split-K partial buffer over all products
    size_t pmax = 0;
    for (int i = 0; i < o.L; ++i) {
        const GemmShape f = gemm_shape((int)Bz, o.d[i + 1], o.d[i]);            // forward
        const GemmShape w = gemm_shape(o.d[i], o.d[i + 1], (int)Bz);            // dW
        pmax = std::max(pmax, (size_t)f.splits * f.M * f.N);
        pmax = std::max(pmax, (size_t)w.splits * w.M * w.N);
        if (i > 0) {
            const GemmShape h = gemm_shape((int)Bz, o.d[i], o.d[i + 1]);        // dH
            pmax = std::max(pmax, (size_t)h.splits * h.M * h.N);
        }
    }
    o.part = off; off += al256(pmax * 4);
    o.loss_blocks = off; off += al256(kLossBlocks * 8);
    o.colsum = off; off += al256((size_t)kColChunks * o.dmax * 8);
    o.total = off;
    return o;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<unsigned char*>(ws) + off); }

int grid_1d(int64_t n, const LaunchCtx& ctx) {
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)ctx.num_sms * 8;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

// The driver's tensor-map encoder, fetched once through the runtime (the
// library links only the CUDA runtime); null when the driver has none.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return (EncodeTiledFn) nullptr;
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// Tensor map of one bf16 operand for gemm_tma_kernel: R rows (M or N) by K,
// X[r * ld + k] (k contiguous, MN == false) or X[k * ld + r] (r contiguous);
// 128-byte swizzle, out-of-range elements read as zero.  False when the
// layout does not meet TMA's rules (16-byte aligned base and row stride).
bool operand_map(CUtensorMap* map, const bf16* X, int64_t ld, int R, int K, bool MN) {
    const EncodeTiledFn enc = encode_tiled();
    if (!enc || (reinterpret_cast<uintptr_t>(X) & 15) || ld <= 0 || (ld * 2) % 16 ||
        ld >= (int64_t(1) << 31))
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(MN ? R : K), (cuuint64_t)(MN ? K : R)};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {64u, MN ? 64u : 128u};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(X), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// product + epilogue
template <bool TA, bool TB>
int gemm(const bf16* A, int64_t lda, const bf16* Bm, int64_t ldb, int M, int N, int K, float* part,
         const float* bias, int act, const float* h, float* out, bf16* out_b,
         const LaunchCtx& ctx) {
    const GemmShape s = gemm_shape(M, N, K);
    stage_event(ctx, 0);
    CUtensorMap ma, mb;
    if (s.tc && operand_map(&ma, A, lda, M, K, TA) && operand_map(&mb, Bm, ldb, N, K, TB)) {
        auto k = tc::gemm_tma_kernel<TA, TB>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc::kSmemTmaBytes))
            return ETICS_ERR_CUDA;
        dim3 grid((N + tc::kN - 1) / tc::kN, (M + tc::kM - 1) / tc::kM, s.splits);
        k<<<grid, tc::kThreads, tc::kSmemTmaBytes, ctx.stream>>>(ma, mb, part, M, N, K, s.kslice,
                                                                 ctx.err);
    } else if (s.tc) {
        auto k = tc::gemm_kernel<TA, TB>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tc::kSmemBytes))
            return ETICS_ERR_CUDA;
        dim3 grid((N + tc::kN - 1) / tc::kN, (M + tc::kM - 1) / tc::kM, s.splits);
        k<<<grid, tc::kThreads, tc::kSmemBytes, ctx.stream>>>(A, lda, Bm, ldb, part, M, N, K,
                                                              s.kslice, ctx.err);
    } else {
        dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, s.splits);
        mlp_gemm_kernel<TA, TB><<<grid, kGemmThreads, 0, ctx.stream>>>(A, lda, Bm, ldb, part, M,
                                                                      N, K, s.kslice);
    }
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    stage_event(ctx, 1);
    mlp_epilogue_kernel<<<grid_1d((int64_t)M * N, ctx), 256, 0, ctx.stream>>>(
        part, s.splits, M, N, bias, act, h, out, out_b);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    stage_event(ctx, 2);
    *ctx.launches += 2;
    return ETICS_OK;
}

// forward pass; activations stay in ws for the backward pass
int forward_impl(const MlpLayout& o, const float* params, const bf16* pb, const bf16* x, int B,
                 float* y, void* ws, const LaunchCtx& ctx) {
    const bf16* a = x;
    for (int i = 0; i < o.L; ++i) {
        const bool last = i == o.L - 1;
        int rc = gemm<false, true>(a, o.d[i], pb + o.woff[i], o.d[i + 1], B, o.d[i + 1], o.d[i],
                                   at<float>(ws, o.part), params + o.boff[i], last ? 0 : 1,
                                   nullptr, last ? y : at<float>(ws, o.h32[i]),
                                   last ? nullptr : at<bf16>(ws, o.hb[i]), ctx);
        if (rc) return rc;
        if (!last) a = at<bf16>(ws, o.hb[i]);
    }
    return ETICS_OK;
}

}  // namespace

// ---- entry points used by the C ABI -----------------------------------------
int64_t mlp_param_count(const etics_mlp_shape* s) {
    if (!valid_shape(s)) return -1;
    return mlp_layout(s, 1).nparam;
}

size_t mlp_workspace(const etics_mlp_shape* s, int B) {
    if (!valid_shape(s) || B < 0) return 0;
    return mlp_layout(s, B).total;
}

int mlp_forward(const etics_mlp_shape* s, const float* params, const uint16_t* pb,
                const uint16_t* x, int B, float* y, void* ws, size_t ws_bytes,
                const LaunchCtx& ctx) {
    const MlpLayout o = mlp_layout(s, B);
    if (ws_bytes < o.total) return ETICS_ERR_WORKSPACE;
    if (B == 0) return ETICS_OK;
    return forward_impl(o, params, reinterpret_cast<const bf16*>(pb),
                        reinterpret_cast<const bf16*>(x), B, y, ws, ctx);
}

int mlp_loss_grad(const etics_mlp_shape* s, const float* params, const uint16_t* pbits,
                  const uint16_t* xbits, const float* target, int B, float* grads, double* loss,
                  void* ws, size_t ws_bytes, const LaunchCtx& ctx) {
    const MlpLayout o = mlp_layout(s, B);
    if (ws_bytes < o.total) return ETICS_ERR_WORKSPACE;
    if (B == 0) return ETICS_ERR_ARG;
    const bf16* pb = reinterpret_cast<const bf16*>(pbits);
    const bf16* x = reinterpret_cast<const bf16*>(xbits);
    float* y = at<float>(ws, o.y32);
    int rc = forward_impl(o, params, pb, x, B, y, ws, ctx);
    if (rc) return rc;
    const int L = o.L;
    const int64_t count = (int64_t)B * o.d[L];
    int cur = 0;
    mlp_mse_kernel<<<kLossBlocks, 256, 0, ctx.stream>>>(
        y, target, count, (float)(2.0 / (double)count), at<float>(ws, o.dz32[cur]),
        at<bf16>(ws, o.dzb[cur]), at<double>(ws, o.loss_blocks));
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    mlp_loss_final_kernel<<<1, 32, 0, ctx.stream>>>(at<double>(ws, o.loss_blocks), kLossBlocks,
                                                    1.0 / (double)count, loss);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    *ctx.launches += 2;
    for (int i = L - 1; i >= 0; --i) {
        const int din = o.d[i], dout = o.d[i + 1];
        const bf16* a_in = i == 0 ? x : at<bf16>(ws, o.hb[i - 1]);
        const bf16* dzb = at<bf16>(ws, o.dzb[cur]);
        // dW_i = a_in^T dz
        rc = gemm<true, true>(a_in, din, dzb, dout, din, dout, B, at<float>(ws, o.part), nullptr, 0,
                              nullptr, grads + o.woff[i], nullptr, ctx);
        if (rc) return rc;
        {
            const int rows = (B + kColChunks - 1) / kColChunks;
            const int chunks = (B + rows - 1) / rows;
            const dim3 g1((dout + 127) / 128, chunks);
            mlp_colsum_partial_kernel<<<g1, 128, 0, ctx.stream>>>(
                at<float>(ws, o.dz32[cur]), B, dout, rows, at<double>(ws, o.colsum));
            mlp_colsum_final_kernel<<<(dout + 127) / 128, 128, 0, ctx.stream>>>(
                at<double>(ws, o.colsum), chunks, dout, grads + o.boff[i]);
            if (cudaGetLastError()) return ETICS_ERR_CUDA;
            *ctx.launches += 2;
        }
        if (i > 0) {
            // dz_{i-1} = (dz W_i^T) * (1 - h_{i-1}^2)
            const int nxt = cur ^ 1;
            rc = gemm<false, false>(dzb, dout, pb + o.woff[i], dout, B, din, dout,
                                    at<float>(ws, o.part), nullptr, 0, at<float>(ws, o.h32[i - 1]),
                                    at<float>(ws, o.dz32[nxt]), at<bf16>(ws, o.dzb[nxt]), ctx);
            if (rc) return rc;
            cur = nxt;
        }
    }
    return ETICS_OK;
}

int mlp_adam(const etics_mlp_shape* s, float* params, const float* grads, float* m, float* v,
             int64_t t, float lr, float b1, float b2, float eps, uint16_t* pb,
             const LaunchCtx& ctx) {
    const int64_t n = mlp_layout(s, 1).nparam;
    const double bc1 = 1.0 / (1.0 - pow((double)b1, (double)t));
    const double bc2 = 1.0 / (1.0 - pow((double)b2, (double)t));
    mlp_adam_kernel<<<grid_1d(n, ctx), 256, 0, ctx.stream>>>(
        params, grads, m, v, n, lr, b1, b2, eps, (float)bc1, (float)bc2, reinterpret_cast<bf16*>(pb));
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

int mbarrier_timeout_probe(int64_t spins, const LaunchCtx& ctx) {
    tc::wait_timeout_kernel<<<1, tc::kThreads, 0, ctx.stream>>>((long long)spins, ctx.err);
    if (cudaGetLastError() != cudaSuccess) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

int mlp_to_bf16(const etics_mlp_shape* s, const float* params, uint16_t* pb, const LaunchCtx& ctx) {
    const int64_t n = mlp_layout(s, 1).nparam;
    mlp_to_bf16_kernel<<<grid_1d(n, ctx), 256, 0, ctx.stream>>>(params, n,
                                                               reinterpret_cast<bf16*>(pb));
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

int coeff_stats(const double* traj, int T, int D, int stride, double* norm, const LaunchCtx& ctx) {
    coeff_stats_kernel<<<(D + 127) / 128, 128, 0, ctx.stream>>>(traj, T, D, stride, norm);
    coeff_linfit_kernel<<<(D + 63) / 64, 64, 0, ctx.stream>>>(traj, T, D, stride, norm);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    *ctx.launches += 2;
    return ETICS_OK;
}

int coeff_features(const double* store, const int32_t* rows, const int32_t* next, int B, int D,
                   int stride, const double* norm, int per_coeff, uint16_t* x, float* target,
                   const LaunchCtx& ctx) {
    if (B == 0) return ETICS_OK;
    coeff_features_kernel<<<grid_1d((int64_t)B * D, ctx), 256, 0, ctx.stream>>>(
        store, rows, next, B, D, stride, norm, per_coeff, reinterpret_cast<bf16*>(x), target);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

int coeff_advance(double* ring, int32_t* order, int D, int stride, int horizon, const double* cin,
                  const float* y, int y_stride, const double* norm, double* cout, int commit,
                  const LaunchCtx& ctx) {
    coeff_advance_kernel<<<1, kAdvanceThreads, 0, ctx.stream>>>(ring, order, D, stride, horizon,
                                                                 cin, y, y_stride, norm, cout,
                                                                 commit);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

int force_error(const void* a, const void* r, int64_t N, int precision, double tol_a, double tol_b,
                uint64_t* out, const LaunchCtx& ctx) {
    if (cudaMemsetAsync(out, 0, 3 * sizeof(uint64_t), ctx.stream)) return ETICS_ERR_CUDA;
    if (N == 0) return ETICS_OK;
    auto* o = reinterpret_cast<unsigned long long*>(out);
    if (precision == ETICS_MIXED)
        force_error_kernel<float><<<grid_1d(N, ctx), 256, 0, ctx.stream>>>(
            static_cast<const Vec4<float>*>(a), static_cast<const Vec4<float>*>(r), N, tol_a,
            tol_b, o);
    else
        force_error_kernel<double><<<grid_1d(N, ctx), 256, 0, ctx.stream>>>(
            static_cast<const Vec4<double>*>(a), static_cast<const Vec4<double>*>(r), N, tol_a,
            tol_b, o);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

}  // namespace etics
