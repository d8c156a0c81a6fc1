// etics_common.cuh -- types, compile-time tables and device helpers shared by
// the sm_103a kernels of the SCF / MEX expansion force library.
//
// All basis constants are computed here at compile time (constexpr) from
// their definitions; nothing is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "etics.h"

namespace etics {

constexpr int kNmaxLimit = ETICS_NMAX_LIMIT;   // 16
constexpr int kLmaxLimit = ETICS_LMAX_LIMIT;   // 14
constexpr int kMexLmaxLimit = ETICS_MEX_LMAX_LIMIT;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// particle vectors: float4 for the mixed path, 4 doubles (16-byte aligned,
// loaded as two 16-byte halves) for the FP64 path
// ---------------------------------------------------------------------------
struct __align__(16) dvec4 { double x, y, z, w; };

template <typename R> struct Vec4T;
template <> struct Vec4T<float> { using type = float4; };
template <> struct Vec4T<double> { using type = dvec4; };
template <typename R> using Vec4 = typename Vec4T<R>::type;

__device__ __forceinline__ float4 ld4(const float4* p) { return *p; }
__device__ __forceinline__ dvec4 ld4(const dvec4* p) {
    const double2* q = reinterpret_cast<const double2*>(p);
    double2 a = q[0], b = q[1];
    return dvec4{a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ void st4(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void st4(dvec4* p, dvec4 v) {
    double2* q = reinterpret_cast<double2*>(p);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}
template <typename R> __device__ __forceinline__ Vec4<R> mk4(R a, R b, R c, R d);
template <> __device__ __forceinline__ float4 mk4<float>(float a, float b, float c, float d) {
    return make_float4(a, b, c, d);
}
template <> __device__ __forceinline__ dvec4 mk4<double>(double a, double b, double c, double d) {
    return dvec4{a, b, c, d};
}

// ---------------------------------------------------------------------------
// device error word: the first data error wins (ETICS_ERR_* codes)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void report(unsigned* err, int code) {
    if (err) atomicCAS(err, 0u, (unsigned)(-code));
}

__device__ __forceinline__ bool finite4(float a, float b, float c, float d) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}
__device__ __forceinline__ bool finite4(double a, double b, double c, double d) {
    return isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d);
}

// ---------------------------------------------------------------------------
// compile-time tables
// ---------------------------------------------------------------------------
constexpr double csqrt(double x) {
    if (x <= 0.0) return 0.0;
    double g = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 400; ++i) {
        double ng = 0.5 * (g + x / g);
        if (ng == g) break;
        g = ng;
    }
    return g;
}

struct BasisTables {
    // Gegenbauer recursion C_n = a[l][n] xi C_{n-1} - b[l][n] C_{n-2}, alpha = 2l + 3/2:
    //   a = 2 (n + alpha - 1) / n,  b = (n + 2 alpha - 2) / n   (n >= 1; C_{-1} = 0)
    float ga_f[kLmaxLimit + 1][kNmaxLimit + 1];
    float gb_f[kLmaxLimit + 1][kNmaxLimit + 1];
    double ga_d[kLmaxLimit + 1][kNmaxLimit + 1];
    double gb_d[kLmaxLimit + 1][kNmaxLimit + 1];
    // real orthonormal normalisation of the unnormalised harmonics used on
    // the GPU (Re/Im of r^l P_l^m e^{i m phi}):  K_lm = sqrt((2l+1)/(4 pi)
    // (l-m)!/(l+m)!), times sqrt2 for m > 0.  Indexed [l*(l+1)/2 + m], m >= 0.
    double knorm[(kLmaxLimit + 1) * (kLmaxLimit + 2) / 2];
    // knorm / (l-m)!: the normalisation of the factorial-scaled harmonics
    // (l-m)! Z_l^m that the coefficient passes evaluate (harm_level_exact)
    double knorm_fact[(kLmaxLimit + 1) * (kLmaxLimit + 2) / 2];
    // MEX weights 4pi/(2l+1) K_lm^2 = (l-m)!/(l+m)! (times 2 for m > 0)
    float mexw_f[(kLmaxLimit + 1) * (kLmaxLimit + 2) / 2];
    double mexw_d[(kLmaxLimit + 1) * (kLmaxLimit + 2) / 2];
    // 1/J_nl, J_nl = -K_nl (n+4l+2)!/n! / (2^(8l+6) (n+2l+3/2) pi prod_{k=0}^{2l}(k+1/2)^2),
    // K_nl = n(n+4l+3)/2 + (l+1)(2l+1)
    double inv_j[kNmaxLimit + 1][kLmaxLimit + 1];
    // Clutton-Brock basis (Plummer zeroth term): Gegenbauer alpha = l + 1 and
    // 1/J_nl, J_nl = -K_nl 2^-(4l+6) (n+2l+1)! / (n! (n+l+1) (l!)^2),
    // K_nl = 4n(n+2l+2) + (2l+1)(2l+3)
    float ga_cb_f[kLmaxLimit + 1][kNmaxLimit + 1];
    float gb_cb_f[kLmaxLimit + 1][kNmaxLimit + 1];
    double ga_cb_d[kLmaxLimit + 1][kNmaxLimit + 1];
    double gb_cb_d[kLmaxLimit + 1][kNmaxLimit + 1];
    double inv_j_cb[kNmaxLimit + 1][kLmaxLimit + 1];
    // Rescaled polynomials Ct_n = C_n / gam_n, gam_n = a_1 a_2 ... a_n
    // (gam_0 = 1), obey Ct_n = xi Ct_{n-1} - bs_n Ct_{n-2} with
    // bs_n = b_n / (a_n a_{n-1}) (n >= 2; bs_1 = 0), and their derivatives
    // Dt_n = Ct_{n-1} + xi Dt_{n-1} - bs_n Dt_{n-2}: one instruction fewer
    // per step than the plain recursion.  The kernels recur on Ct and fold
    // gam_n into the coefficients.  [basis][l][n], basis 0 HO, 1 CB.
    float gbs_f[2][kLmaxLimit + 1][kNmaxLimit + 1];
    double gbs_d[2][kLmaxLimit + 1][kNmaxLimit + 1];
    double ggam[2][kLmaxLimit + 1][kNmaxLimit + 1];
};

constexpr BasisTables make_tables() {
    BasisTables t{};
    for (int l = 0; l <= kLmaxLimit; ++l) {
        const double alpha = 2.0 * l + 1.5;
        for (int n = 0; n <= kNmaxLimit; ++n) {
            double a = 0.0, b = 0.0;
            if (n >= 1) {
                a = 2.0 * (n + alpha - 1.0) / n;
                b = (n + 2.0 * alpha - 2.0) / n;
            }
            t.ga_d[l][n] = a;
            t.gb_d[l][n] = b;
            t.ga_f[l][n] = (float)a;
            t.gb_f[l][n] = (float)b;
        }
        for (int m = 0; m <= l; ++m) {
            double ratio = 1.0;   // (l-m)!/(l+m)!
            for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
            const int idx = l * (l + 1) / 2 + m;
            double k2 = (2.0 * l + 1.0) / (4.0 * kPi) * ratio * (m > 0 ? 2.0 : 1.0);
            t.knorm[idx] = csqrt(k2);
            double fact = 1.0;   // (l-m)!
            for (int k = 2; k <= l - m; ++k) fact *= (double)k;
            t.knorm_fact[idx] = t.knorm[idx] / fact;
            const double w = ratio * (m > 0 ? 2.0 : 1.0);
            t.mexw_d[idx] = w;
            t.mexw_f[idx] = (float)w;
        }
    }
    for (int n = 0; n <= kNmaxLimit; ++n) {
        for (int l = 0; l <= kLmaxLimit; ++l) {
            const double K = 0.5 * n * (n + 4.0 * l + 3.0) + (l + 1.0) * (2.0 * l + 1.0);
            double num = 1.0;
            for (int k = n + 1; k <= n + 4 * l + 2; ++k) num *= (double)k;
            double den = (n + 2.0 * l + 1.5) * kPi;
            for (int k = 0; k <= 2 * l; ++k) den *= (k + 0.5) * (k + 0.5);
            for (int k = 0; k < 8 * l + 6; ++k) den *= 2.0;
            const double J = -K * num / den;
            t.inv_j[n][l] = 1.0 / J;
        }
    }
    for (int l = 0; l <= kLmaxLimit; ++l) {
        const double alpha = l + 1.0;
        for (int n = 0; n <= kNmaxLimit; ++n) {
            double a = 0.0, b = 0.0;
            if (n >= 1) {
                a = 2.0 * (n + alpha - 1.0) / n;
                b = (n + 2.0 * alpha - 2.0) / n;
            }
            t.ga_cb_d[l][n] = a;
            t.gb_cb_d[l][n] = b;
            t.ga_cb_f[l][n] = (float)a;
            t.gb_cb_f[l][n] = (float)b;
            const double K = 4.0 * n * (n + 2.0 * l + 2.0) + (2.0 * l + 1.0) * (2.0 * l + 3.0);
            double num = 1.0;                         // (n+2l+1)!/n!
            for (int k = n + 1; k <= n + 2 * l + 1; ++k) num *= (double)k;
            double den = (n + l + 1.0);
            for (int k = 2; k <= l; ++k) den *= (double)k * (double)k;   // (l!)^2
            for (int k = 0; k < 4 * l + 6; ++k) den *= 2.0;
            t.inv_j_cb[n][l] = 1.0 / (-K * num / den);
        }
    }
    for (int basis = 0; basis < 2; ++basis) {
        for (int l = 0; l <= kLmaxLimit; ++l) {
            double gam = 1.0;
            for (int n = 0; n <= kNmaxLimit; ++n) {
                const double a = basis == 0 ? t.ga_d[l][n] : t.ga_cb_d[l][n];
                const double b = basis == 0 ? t.gb_d[l][n] : t.gb_cb_d[l][n];
                const double ap = n >= 2 ? (basis == 0 ? t.ga_d[l][n - 1] : t.ga_cb_d[l][n - 1]) : 0.0;
                if (n >= 1) gam *= a;
                const double bs = n >= 2 ? b / (a * ap) : 0.0;
                t.gbs_d[basis][l][n] = bs;
                t.gbs_f[basis][l][n] = (float)bs;
                t.ggam[basis][l][n] = gam;
            }
        }
    }
    return t;
}

static __constant__ BasisTables c_tab = make_tables();

// The same tables as a compile-time object, for recursion constants that have
// to become instruction immediates: a paired FP32 instruction takes register
// operands only, so a constant-memory value would need a load into registers
// at every use when the registers are too few to keep it.
constexpr BasisTables kTabCE = make_tables();
template <int B, int L, int N>
struct GegBsConst {
    static constexpr float v = kTabCE.gbs_f[B][L][N];
};

// rescaled Gegenbauer recursion constant bs_n and scale gam_n of radial basis
// B (0 Hernquist-Ostriker, 1 Clutton-Brock; see BasisTables)
template <typename R, int B = 0> __device__ __forceinline__ R geg_bs(int l, int n) {
    if constexpr (sizeof(R) == 4) return c_tab.gbs_f[B][l][n];
    else return c_tab.gbs_d[B][l][n];
}
__device__ __forceinline__ double geg_gamma(int basis, int l, int n) { return c_tab.ggam[basis][l][n]; }
__device__ __forceinline__ double inv_j_of(int basis, int n, int l) {
    return basis == 0 ? c_tab.inv_j[n][l] : c_tab.inv_j_cb[n][l];
}

// Radial seeds of basis B at radius r, the form both SCF passes use: the
// radial factor of level l is phi_nl(r) = pre_l C_n(xi) with
// pre_l = pre0 st^l = -r^l g(r)^(2l+1), so that phi_nl Y_lm evaluated with
// the harmonic at the unit vector is pre0 st^l C_n(xi) Z_lm(u):
//   HO: g = 1/(1+r),       st = r/(1+r)^2, xi = (r-1)/(r+1),     dxi/dr = 2/(1+r)^2
//   CB: g = 1/sqrt(1+r^2), st = r/(1+r^2), xi = (r^2-1)/(r^2+1), dxi/dr = 4r/(1+r^2)^2
// with pre0 = -g.  tau enters the radial derivative,
// d pre_l/dr = pre_l (l/r - (2l+1) tau), tau = 1/(1+r) (HO), r/(1+r^2) (CB);
// q = st/r = g^2 scales the solid-harmonic gradient term (pre_l / r).
template <typename R, int B>
struct RadialSeed {
    R pre0, st, xi, dxdr, tau, q;
    __device__ __forceinline__ explicit RadialSeed(R r) {
        if constexpr (B == 0) {
            const R t = R(1) / (R(1) + r);
            pre0 = -t;
            q = t * t;
            st = r * q;
            xi = R(1) - R(2) * t;
            dxdr = R(2) * q;
            tau = t;
        } else {
            q = R(1) / (R(1) + r * r);
            pre0 = -sqrt(q);
            st = r * q;
            xi = R(1) - R(2) * q;
            dxdr = R(4) * r * q * q;
            tau = r * q;
        }
    }
};
template <typename R> __device__ __forceinline__ R mex_w(int idx);
template <> __device__ __forceinline__ float mex_w<float>(int idx) { return c_tab.mexw_f[idx]; }
template <> __device__ __forceinline__ double mex_w<double>(int idx) { return c_tab.mexw_d[idx]; }

// ---------------------------------------------------------------------------
// Unnormalised solid harmonics at a point u (used at the unit vector):
//   Z_l^m(u) = |u|^l P_l^m(cos t) e^{i m phi} (no Condon-Shortley phase),
//   C_l^m = Re Z_l^m, S_l^m = Im Z_l^m, m = 0..l.
// Cartesian l-upward recursion (the stable direction, no cot(theta)):
//   Z_m^m     = (2m-1) (ux + i uy) Z_{m-1}^{m-1}
//   Z_{m+1}^m = (2m+1) uz Z_m^m
//   (l-m) Z_l^m = (2l-1) uz Z_{l-1}^m - (l+m-1) |u|^2 Z_{l-2}^m
// Gradient (homogeneous of degree l-1) from level l-1 by the ladder relations
//   d/dz Z_l^m = (l+m) Z_{l-1}^m,
//   (d/dx - i d/dy) Z_l^m = (l+m)(l+m-1) Z_{l-1}^{m-1},
//   (d/dx + i d/dy) Z_l^m = -Z_{l-1}^{m+1}   (m >= 1),
// and for m = 0: grad C_l^0 = (-C_{l-1}^1, -S_{l-1}^1, l C_{l-1}^0).
// Arrays are indexed by m and must be used with compile-time l (unrolled).
// ---------------------------------------------------------------------------
template <typename R, int L>
__device__ __forceinline__ void harm_level(const R* C1, const R* S1, const R* C2, const R* S2,
                                           R ux, R uy, R uz, R uu, R* C, R* S) {
    if constexpr (L == 0) {
        C[0] = R(1);
        S[0] = R(0);
    } else {
        constexpr R d = R(2 * L - 1);
        C[L] = d * (ux * C1[L - 1] - uy * S1[L - 1]);
        S[L] = d * (ux * S1[L - 1] + uy * C1[L - 1]);
        C[L - 1] = d * uz * C1[L - 1];
        S[L - 1] = (L - 1 == 0) ? R(0) : d * uz * S1[L - 1];
#pragma unroll
        for (int m = 0; m + 2 <= L; ++m) {
            const R a = R(2 * L - 1) / R(L - m);
            const R b = R(L + m - 1) / R(L - m);
            C[m] = a * uz * C1[m] - b * uu * C2[m];
            S[m] = (m == 0) ? R(0) : a * uz * S1[m] - b * uu * S2[m];
        }
    }
}

// The same harmonics scaled by (L-m)!, for the coefficient passes:
//   H_L^m = (L-m)! Z_L^m(u) on the unit sphere (|u| = 1 taken exactly),
//   H_m^m     = (2m-1) (ux + i uy) H_{m-1}^{m-1}
//   H_{m+1}^m = (2m+1) uz H_m^m
//   H_L^m     = (2L-1) uz H_{L-1}^m - (L+m-1)(L-m-1) H_{L-2}^m.
// Every recursion constant is an integer, exact in FP32.  With the ratios
// (2L-1)/(L-m) and (L+m-1)/(L-m) rounded to FP32 (harm_level above) the
// rounding of the constants leaks into lower harmonics and, through
// uz Z_1^0, into a constant: a bias of about -2e-8 in P_l (l >= 3, m = 0)
// with a non-zero mean over the sphere, which every particle adds
// coherently to the coefficients c_{n,l,0}.  Here only the individual
// roundings remain, and they average out.  The factor 1/(L-m)! goes into the
// FP64 normalisation (knorm_fact).
template <typename R, int L>
__device__ __forceinline__ void harm_level_exact(const R* C1, const R* S1, const R* C2,
                                                 const R* S2, R ux, R uy, R uz, R* C, R* S) {
    if constexpr (L == 0) {
        C[0] = R(1);
        S[0] = R(0);
    } else {
        constexpr R d = R(2 * L - 1);
        C[L] = d * (ux * C1[L - 1] - uy * S1[L - 1]);
        S[L] = d * (ux * S1[L - 1] + uy * C1[L - 1]);
        const R duz = d * uz;
        C[L - 1] = duz * C1[L - 1];
        S[L - 1] = (L - 1 == 0) ? R(0) : duz * S1[L - 1];
#pragma unroll
        for (int m = 0; m + 2 <= L; ++m) {
            const R b = R((L + m - 1) * (L - m - 1));
            C[m] = fma(duz, C1[m], -b * C2[m]);
            S[m] = (m == 0) ? R(0) : fma(duz, S1[m], -b * S2[m]);
        }
    }
}

// gradient of C_L^m (gc) and S_L^m (gs) from level L-1 values (C1, S1; m <= L-1)
template <typename R, int L>
__device__ __forceinline__ void harm_grad(const R* C1, const R* S1, int m, R gc[3], R gs[3]) {
    // values of level L-1 outside 0..L-1 are zero
    auto c1 = [&](int k) -> R { return (k >= 0 && k <= L - 1) ? C1[k] : R(0); };
    auto s1 = [&](int k) -> R { return (k >= 1 && k <= L - 1) ? S1[k] : R(0); };
    if (m == 0) {
        gc[0] = -c1(1);
        gc[1] = -s1(1);
        gc[2] = R(L) * c1(0);
        gs[0] = gs[1] = gs[2] = R(0);
    } else {
        const R a = R((L + m) * (L + m - 1));
        gc[0] = R(0.5) * (a * c1(m - 1) - c1(m + 1));
        gc[1] = R(-0.5) * (a * s1(m - 1) + s1(m + 1));
        gc[2] = R(L + m) * c1(m);
        gs[0] = R(0.5) * (a * s1(m - 1) - s1(m + 1));
        gs[1] = R(0.5) * (a * c1(m - 1) + c1(m + 1));
        gs[2] = R(L + m) * s1(m);
    }
}

// v += grad sum_m (ac[m] C_L^m + as[m] S_L^m) (as[0] unused), from the level
// L-1 values.  The ladder relations above, regrouped by the level L-1
// harmonic they multiply: each direction becomes one dot product with lowered
// coefficients, 2L-1 terms instead of 2L+1 gradient triples.
template <typename R, int L>
__device__ __forceinline__ void grad_contract(const R* C1, const R* S1, const R* ac, const R* as,
                                              R& vx, R& vy, R& vz) {
    if constexpr (L >= 1) {
#pragma unroll
        for (int k = 0; k <= L - 1; ++k) {
            // coefficients of C_{L-1}^k
            R xc = R(0), yc = R(0);
            if (k + 1 <= L) {
                const R h = R(0.5 * (L + k + 1) * (L + k));
                xc = h * ac[k + 1];
                yc = (k + 1 >= 1) ? h * as[k + 1] : R(0);
            }
            if (k >= 2) {
                xc = fma(R(-0.5), ac[k - 1], xc);
                yc = fma(R(0.5), as[k - 1], yc);
            }
            if (k == 1) xc -= ac[0];
            vx = fma(xc, C1[k], vx);
            vy = fma(yc, C1[k], vy);
            vz = fma(R(L + k) * ac[k], C1[k], vz);
            if (k >= 1) {
                // coefficients of S_{L-1}^k
                R xs = R(0), ys = R(0);
                if (k + 1 <= L) {
                    const R h = R(0.5 * (L + k + 1) * (L + k));
                    xs = h * as[k + 1];
                    ys = -h * ac[k + 1];
                }
                if (k >= 2) {
                    xs = fma(R(-0.5), as[k - 1], xs);
                    ys = fma(R(-0.5), ac[k - 1], ys);
                }
                if (k == 1) ys -= ac[0];
                vx = fma(xs, S1[k], vx);
                vy = fma(ys, S1[k], vy);
                vz = fma(R(L + k) * as[k], S1[k], vz);
            }
        }
    }
}

// column layout of one harmonic level: col 0 = C_l^0, col 2m-1 = C_l^m,
// col 2m = S_l^m (m >= 1); 2l+1 columns, padded to a multiple of 4.
__host__ __device__ __forceinline__ int ncol_pad(int l) { return ((2 * l + 1 + 3) / 4) * 4; }
__host__ __device__ __forceinline__ int col_offset(int l) {
    int o = 0;
    for (int k = 0; k < l; ++k) o += ncol_pad(k);
    return o;
}
__host__ __device__ __forceinline__ int col_total(int lmax) { return col_offset(lmax + 1); }

// launch context handed from the C ABI to the kernel launchers
// Programmatic dependent launch.  A kernel started by launch_pdl may be
// scheduled while the previous kernel in its stream drains (its launch
// latency overlaps the predecessor's tail); it must execute pdl_wait()
// (griddepcontrol.wait: returns once every prerequisite grid has completed
// and its memory is visible) before it touches global memory that the
// predecessor reads or writes.  No kernel triggers its dependents
// explicitly: the implicit trigger at block exit keeps waiting blocks from
// holding SM slots that a concurrent stream could use.  pdl_wait() is a
// no-op in a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { cudaGridDependencySynchronize(); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    return e != cudaSuccess ? e : cudaGetLastError();
}

struct LaunchCtx {
    cudaStream_t stream;
    unsigned* err;        // device error word
    int num_sms;
    uint64_t* launches;   // host launch counter
    void** events;        // stage events (nullable)
    int n_events;
    int64_t wait_limit;   // bound of the radix sort's lookback waits (0: default)
};

inline void stage_event(const LaunchCtx& ctx, int k) {
    if (ctx.events && k < ctx.n_events && ctx.events[k])
        cudaEventRecord((cudaEvent_t)ctx.events[k], ctx.stream);
}

}  // namespace etics
