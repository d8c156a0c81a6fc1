// etics_scf_impl.cuh -- SCF coefficient and field kernels (templated on the
// arithmetic type; instantiated for float in etics_scf_f32.cu and for double
// in etics_scf_f64.cu).
//
// Method (paper Sec. 2.4 eq. 18, basis of Sec. 2.5, two passes of Sec. 3.3):
//   c_nlm = (1/J_nl) sum_k m_k phi_nl(r_k) Y_lm(x_k)             (coefficients)
//   Phi   = sum c_nlm phi_nl(r) Y_lm,  a = -grad Phi              (field)
//   phi_nl = -r^l (1+r)^-(2l+1) C_n^(2l+3/2)(xi),  xi = (r-1)/(r+1).
//
// GB300 design (not the paper's per-(n,l) kernel loop of Sec. 3.3):
//   * coefficient pass: one persistent kernel.  Per tile of T particles, half
//     the block evaluates the radial basis m_k phi_nl (Gegenbauer recursion)
//     and the other half the angular basis (Cartesian solid harmonics, no
//     trigonometry, no cot(theta)); both land in shared memory.  The
//     contraction c[n][l,col] += sum_k R[l][n][k] Y[l,col][k] is then done
//     with each thread owning an (n_rows x 4 columns) register tile of one l
//     over a strided subset of the tile's particles (4 particles per 16-byte
//     shared load).  FP32 partial sums are flushed into per-block FP64
//     accumulators every few tiles; per-block FP64 partials are summed in a
//     fixed order by a finalize kernel (deterministic).
//   * field pass: one thread per particle; coefficients (pre-multiplied by the
//     harmonic normalisation) broadcast from shared memory; the gradient of
//     phi_nl(r) Y_lm is built from the Cartesian gradient of the solid
//     harmonic, which is regular on the z axis and at the origin.
#pragma once

#include "etics_common.cuh"

namespace etics {

template <typename R> struct ScfCfg;
template <> struct ScfCfg<float> {
    static constexpr int kThreads = 256;   // coefficient kernel block
    static constexpr int kTile = 128;      // particles per tile (2 threads each in phase 1)
};
template <> struct ScfCfg<double> {
    static constexpr int kThreads = 128;
    static constexpr int kTile = 64;
};
constexpr int kFieldThreads = 256;
constexpr int kFlushTiles = 16;

struct ScfCoeffParams {
    const void* posm;
    int64_t N;
    int n_max, l_max;
    int T;            // particles per tile (multiple of 4)
    int W, G;         // register-tile items and particle groups per item
    int ntiles;
    int l_split;      // radial levels [0, l_split) by the first half of the block
    double* partial;  // [gridDim.x][W*NR*4]
    unsigned* err;
};

__host__ __device__ constexpr int ncol_pad_c(int l) { return ((2 * l + 1 + 3) / 4) * 4; }
__host__ __device__ constexpr int col_offset_c(int l) {
    int o = 0;
    for (int k = 0; k < l; ++k) o += ncol_pad_c(k);
    return o;
}
__host__ __device__ inline int scf_items(int l_max) { return col_total(l_max) / 4; }

// shared-memory bytes of the coefficient kernel
template <typename R>
__host__ inline size_t scf_coeff_smem(int NR, int l_max, int T, int W, int G) {
    size_t main = (size_t)(l_max + 1) * NR * T + (size_t)col_total(l_max) * T;
    size_t red = (size_t)W * G * NR * 4;
    size_t elems = main > red ? main : red;
    size_t bytes = ((elems * sizeof(R) + 15) / 16) * 16;
    return bytes + (size_t)W * NR * 4 * sizeof(double);
}

// phase 1, angular half: write the factorial-scaled harmonics (l-m)! Z_l^m
// (harm_level_exact; the finalize applies knorm_fact) of level 0..l_max for
// particle k into Ys[col][k] (compile-time recursion over the level).
// PAD: levels padded to multiples of 4 columns (col_offset_c); otherwise the
// dense layout, level l starting at column l*l.  uu is unused: the
// harmonics are taken on the unit sphere.
template <typename R, int L, int LMU, bool PAD = true>
__device__ __forceinline__ void angular_levels(R (&C)[3][LMU + 1], R (&S)[3][LMU + 1], R ux, R uy,
                                               R uz, R uu, int l_max, R* Ys, int T, int k) {
    if constexpr (L <= LMU) {
        if (L > l_max) return;
        constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
        harm_level_exact<R, L>(C[s1], S[s1], C[s2], S[s2], ux, uy, uz, C[s0], S[s0]);
        constexpr int co = PAD ? col_offset_c(L) : L * L;
        Ys[(size_t)(co + 0) * T + k] = C[s0][0];
#pragma unroll
        for (int m = 1; m <= L; ++m) {
            Ys[(size_t)(co + 2 * m - 1) * T + k] = C[s0][m];
            Ys[(size_t)(co + 2 * m) * T + k] = S[s0][m];
        }
        angular_levels<R, L + 1, LMU, PAD>(C, S, ux, uy, uz, uu, l_max, Ys, T, k);
    }
}

// phase 1, radial part: Rs[l][n][k] = m phi_nl(r_k) / (r^l gam_n) = w_l Ct_n(xi)
// for levels l in [l_begin, l_end] (compile-time recursion over the level, n
// unrolled to NR so the recursion constants are immediates; Ct_n the rescaled
// Gegenbauer polynomial, gam_n restored in the finalize).  Rows n > n_max
// stay zero.  w_l = m pre0 st^l (RadialSeed of basis B).
template <typename R, int NR, int L, int LMU, int B = 0>
__device__ __forceinline__ void radial_levels(R* Rs, int T, int k, int n_max, int l_begin,
                                              int l_end, R w, R st, R xi) {
    if constexpr (L <= LMU) {
        if (L > l_end) return;
        if (L >= l_begin) {
            R* row = Rs + (size_t)L * NR * T + k;
            R cm1 = R(0), c = R(1);
            row[0] = w;
#pragma unroll
            for (int n = 1; n < NR; ++n) {
                if (n <= n_max) {
                    const R cn = fma(xi, c, -geg_bs<R, B>(L, n) * cm1);
                    cm1 = c;
                    c = cn;
                    row[(size_t)n * T] = w * c;
                }
            }
        }
        radial_levels<R, NR, L + 1, LMU, B>(Rs, T, k, n_max, l_begin, l_end, w * st, st, xi);
    }
}

template <typename R, int NR, int LMU, int B = 0>
__global__ void __launch_bounds__(ScfCfg<R>::kThreads, 2)
scf_coeff_kernel(ScfCoeffParams p) {
    constexpr int TH = ScfCfg<R>::kThreads;
    using V4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int T = p.T, TC = T / 4, L1 = p.l_max + 1;
    const int ncols = col_total(p.l_max);
    const size_t main_elems = (size_t)L1 * NR * T + (size_t)ncols * T;
    const size_t red_elems = (size_t)p.W * p.G * NR * 4;
    const size_t union_elems = main_elems > red_elems ? main_elems : red_elems;
    R* Rs = reinterpret_cast<R*>(smem_raw);
    R* Ys = Rs + (size_t)L1 * NR * T;
    double* accd = reinterpret_cast<double*>(smem_raw + ((union_elems * sizeof(R) + 15) / 16) * 16);
    const int nout = p.W * NR * 4;
    const int tid = threadIdx.x;

    for (size_t e = tid; e < union_elems; e += TH) Rs[e] = R(0);
    for (int e = tid; e < nout; e += TH) accd[e] = 0.0;

    // register-tile item of this thread: level l, columns col0..col0+3
    const int item = tid / p.G, g = tid % p.G;
    const bool active = item < p.W;
    int il = 0, col0 = 0;
    if (active) {
        int it = item;
        for (int l = 0; l <= p.l_max; ++l) {
            const int nch = ncol_pad(l) / 4;
            if (it < nch) { il = l; col0 = col_offset(l) + 4 * it; break; }
            it -= nch;
        }
    }
    R acc[NR][4];
#pragma unroll
    for (int n = 0; n < NR; ++n)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[n][j] = R(0);

    const V4* posm = reinterpret_cast<const V4*>(p.posm);
    __syncthreads();

    auto flush = [&]() {
        __syncthreads();
        R* red = Rs;
        if (active) {
#pragma unroll
            for (int n = 0; n < NR; ++n)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    red[(size_t)g * nout + (item * NR + n) * 4 + j] = acc[n][j];
                    acc[n][j] = R(0);
                }
        }
        __syncthreads();
        for (int o = tid; o < nout; o += TH) {
            R s = R(0);
            for (int gg = 0; gg < p.G; ++gg) s += red[(size_t)gg * nout + o];
            accd[o] += (double)s;
        }
        __syncthreads();
        for (size_t e = tid; e < union_elems; e += TH) Rs[e] = R(0);
        __syncthreads();
    };

    // this thread's particle of the current tile (prefetched one tile ahead)
    const int kp = tid < T ? tid : tid - T;
    auto load_particle = [&](int tile) -> V4 {
        const int64_t gi = (int64_t)tile * T + kp;
        if (tid < 2 * T && tile < p.ntiles && gi < p.N) return ld4(posm + gi);
        return mk4<R>(R(0), R(0), R(0), R(0));
    };
    V4 cur = load_particle(blockIdx.x);
    int since_flush = 0;
    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        // ---- phase 1: basis functions of the tile's particles -------------
        if (tid < 2 * T) {
            const int k = kp;
            R x = R(0), y = R(0), z = R(0), m = R(0);
            if (finite4(cur.x, cur.y, cur.z, cur.w)) { x = cur.x; y = cur.y; z = cur.z; m = cur.w; }
            else if (tid < T) report(p.err, ETICS_ERR_NONFINITE);
            const R r = sqrt(x * x + y * y + z * z);
            const RadialSeed<R, B> rs(r);
            if (tid < T) {
                // radial levels [0, l_split)
                radial_levels<R, NR, 0, LMU, B>(Rs, T, k, p.n_max, 0, p.l_split - 1, m * rs.pre0,
                                                rs.st, rs.xi);
            } else {
                // angular basis of every level, then radial levels [l_split, l_max]
                const R inv = r > R(0) ? R(1) / r : R(0);
                const R ux = x * inv, uy = y * inv, uz = z * inv;
                const R uu = ux * ux + uy * uy + uz * uz;
                R C[3][LMU + 1], S[3][LMU + 1];
                angular_levels<R, 0, LMU>(C, S, ux, uy, uz, uu, p.l_max, Ys, T, k);
                radial_levels<R, NR, 0, LMU, B>(Rs, T, k, p.n_max, p.l_split, p.l_max,
                                                m * rs.pre0, rs.st, rs.xi);
            }
        }
        cur = load_particle(tile + gridDim.x);
        __syncthreads();
        // ---- phase 2: register-tiled contraction over the tile -------------
        if (active) {
            const V4* Rv4 = reinterpret_cast<const V4*>(Rs + (size_t)il * NR * T);
            const V4* Yv4 = reinterpret_cast<const V4*>(Ys + (size_t)col0 * T);
            for (int c = g; c < TC; c += p.G) {
                V4 yv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) yv[j] = ld4(Yv4 + (size_t)j * TC + c);
#pragma unroll
                for (int n = 0; n < NR; ++n) {
                    const V4 rv = ld4(Rv4 + (size_t)n * TC + c);
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        R a = acc[n][j];
                        a = fma(rv.x, yv[j].x, a);
                        a = fma(rv.y, yv[j].y, a);
                        a = fma(rv.z, yv[j].z, a);
                        a = fma(rv.w, yv[j].w, a);
                        acc[n][j] = a;
                    }
                }
            }
        }
        __syncthreads();
        if (++since_flush == kFlushTiles) {
            flush();
            since_flush = 0;
        }
    }
    if (since_flush) flush();
    double* out = p.partial + (size_t)blockIdx.x * nout;
    for (int o = tid; o < nout; o += TH) out[o] = accd[o];
}

// Sum the per-block partials in a fixed order and apply K_lm / J_nl.
// One warp per output coefficient c[n][l*l+l+m].
static __global__ void scf_finalize_kernel(const double* __restrict__ partial, int nblocks, int n_max,
                                    int l_max, int NR, int basis, double* __restrict__ coeffs) {
    const int nj = (l_max + 1) * (l_max + 1);
    const int nc = (n_max + 1) * nj;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nc) return;
    const int n = warp / nj, jj = warp % nj;
    int l = 0;
    while ((l + 1) * (l + 1) <= jj) ++l;
    const int m = jj - l * l - l;
    const int col = (m == 0) ? 0 : (m > 0 ? 2 * m - 1 : -2 * m);
    const int item = col_offset(l) / 4 + col / 4;
    const int idx = (item * NR + n) * 4 + (col & 3);
    const int stride = scf_items(l_max) * NR * 4;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(size_t)b * stride + idx];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int am = m < 0 ? -m : m;
        coeffs[warp] = s * c_tab.knorm_fact[l * (l + 1) / 2 + am] * inv_j_of(basis, n, l) *
                       geg_gamma(basis, l, n);
    }
}

// ---------------------------------------------------------------------------
// field pass
// ---------------------------------------------------------------------------
// NM1 > 0: specialised for n_max + 1 == NM1 and l_max == LM (n loop unrolled,
// coefficient row stride and recursion constants known at compile time);
// NM1 == 0: generic, n_max and l_max <= LM at run time.
template <typename R, int LM, bool ACC, int NM1, int BASIS = 0>
struct FieldEval {
    using V4 = Vec4<R>;
    R C[3][LM + 1], S[3][LM + 1];
    // t: the basis's tau (radial derivative factor), see RadialSeed
    R ux, uy, uz, uu, t, xi, dxdr, st, pre, preR;
    R pot, gr, gx, gy, gz;
    const R* cs;
    int ncols, n_max, l_max;

    template <int L>
    __device__ __forceinline__ void level() {
        if constexpr (L <= LM) {
            if (NM1 == 0 && L > l_max) return;
            constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
            harm_level<R, L>(C[s1], S[s1], C[s2], S[s2], ux, uy, uz, uu, C[s0], S[s0]);
            constexpr int NC = 2 * L + 1;
            constexpr int NQ = ncol_pad_c(L) / 4;
            constexpr int CO = col_offset_c(L);
            R A[NC], B[NC];
#pragma unroll
            for (int c = 0; c < NC; ++c) { A[c] = R(0); B[c] = R(0); }
            // FP32: the column sums run as packed pairs (columns 2i, 2i+1:
            // one paired FMA for two columns; the padded table has a zero
            // partner for the last, odd column)
            constexpr int NP = (NC + 1) / 2;
            float2 A2[NP], B2[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) { A2[i] = make_float2(0.f, 0.f); B2[i] = make_float2(0.f, 0.f); }
            R cm1 = R(0), cn = R(1), dm1 = R(0), dn = R(0);
            constexpr int kStride = NM1 > 0 ? col_offset_c(LM + 1) : 0;
            const int stride = NM1 > 0 ? kStride : ncols;
            const int nlim = NM1 > 0 ? NM1 - 1 : n_max;
            const R* row = cs + CO;
#pragma unroll (NM1 > 0 ? NM1 : 4)
            for (int n = 0; n <= nlim; ++n, row += stride) {
                if (n > 0) {
                    // rescaled polynomials (the table holds gam_n c_nlm)
                    const R bs = geg_bs<R, BASIS>(L, n);
                    const R cnew = fma(xi, cn, -bs * cm1);
                    if (ACC) {
                        const R dnew = fma(-bs, dm1, fma(xi, dn, cn));
                        dm1 = dn;
                        dn = dnew;
                    }
                    cm1 = cn;
                    cn = cnew;
                }
                if constexpr (sizeof(R) == 4) {
                    // a pair whose second column is the padding (the last,
                    // odd column) runs as one scalar FMA
                    const float2 cc = make_float2(cn, cn), dd = make_float2(dn, dn);
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const V4 v = ld4(reinterpret_cast<const V4*>(row) + q);
                        if (4 * q + 1 < NC) {
                            A2[2 * q] = __ffma2_rn(make_float2(v.x, v.y), cc, A2[2 * q]);
                            if (ACC) B2[2 * q] = __ffma2_rn(make_float2(v.x, v.y), dd, B2[2 * q]);
                        } else if (4 * q < NC) {
                            A2[2 * q].x = fmaf(v.x, cn, A2[2 * q].x);
                            if (ACC) B2[2 * q].x = fmaf(v.x, dn, B2[2 * q].x);
                        }
                        if (4 * q + 3 < NC) {
                            A2[2 * q + 1] = __ffma2_rn(make_float2(v.z, v.w), cc, A2[2 * q + 1]);
                            if (ACC) B2[2 * q + 1] = __ffma2_rn(make_float2(v.z, v.w), dd, B2[2 * q + 1]);
                        } else if (4 * q + 2 < NC) {
                            A2[2 * q + 1].x = fmaf(v.z, cn, A2[2 * q + 1].x);
                            if (ACC) B2[2 * q + 1].x = fmaf(v.z, dn, B2[2 * q + 1].x);
                        }
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < NQ; ++q) {
                        const V4 v = ld4(reinterpret_cast<const V4*>(row) + q);
                        const R vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int c = 4 * q + e;
                            if (c < NC) {
                                A[c] = fma(vv[e], cn, A[c]);
                                if (ACC) B[c] = fma(vv[e], dn, B[c]);
                            }
                        }
                    }
                }
            }
            if constexpr (sizeof(R) == 4) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    A[c] = (c & 1) ? A2[c / 2].y : A2[c / 2].x;
                    B[c] = (c & 1) ? B2[c / 2].y : B2[c / 2].x;
                }
            }
            // angular sums with the level's harmonics
            R P = A[0] * C[s0][0];
            R Q = ACC ? B[0] * C[s0][0] : R(0);
#pragma unroll
            for (int m = 1; m <= L; ++m) {
                P = fma(A[2 * m - 1], C[s0][m], P);
                P = fma(A[2 * m], S[s0][m], P);
                if (ACC) {
                    Q = fma(B[2 * m - 1], C[s0][m], Q);
                    Q = fma(B[2 * m], S[s0][m], Q);
                }
            }
            pot = fma(pre, P, pot);
            if (ACC) {
                gr = fma(pre, R(-(2 * L + 1)) * t * P + dxdr * Q, gr);
                if constexpr (L >= 1) {
                    R vx = R(0), vy = R(0), vz = R(0);
                    R ac[L + 1], as[L + 1];
#pragma unroll
                    for (int m = 0; m <= L; ++m) {
                        ac[m] = A[m == 0 ? 0 : 2 * m - 1];
                        as[m] = m == 0 ? R(0) : A[2 * m];
                    }
                    grad_contract<R, L>(C[s1], S[s1], ac, as, vx, vy, vz);
                    gx = fma(preR, vx, gx);
                    gy = fma(preR, vy, gy);
                    gz = fma(preR, vz, gz);
                    preR *= st;
                }
            }
            pre *= st;
            level<L + 1>();
        }
    }
};

template <typename R, int LM, bool ACC, int NM1, int B = 0>
__global__ void __launch_bounds__(kFieldThreads, 2)
scf_field_kernel(const Vec4<R>* __restrict__ posm, int64_t N, int n_max, int l_max,
                 const double* __restrict__ coeffs, Vec4<R>* __restrict__ out, int out_mask,
                 unsigned* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* cs = reinterpret_cast<R*>(smem_raw);
    const int ncols = col_total(l_max);
    const int nj = (l_max + 1) * (l_max + 1);
    pdl_wait();   // the coefficients come from the previous kernel
    for (int e = threadIdx.x; e < (n_max + 1) * ncols; e += blockDim.x) {
        const int n = e / ncols;
        int c = e % ncols, l = 0;
        while (c >= ncol_pad(l)) { c -= ncol_pad(l); ++l; }
        R v = R(0);
        if (c < 2 * l + 1) {
            const int m = (c == 0) ? 0 : ((c & 1) ? (c + 1) / 2 : -(c / 2));
            const int am = m < 0 ? -m : m;
            v = (R)(coeffs[(size_t)n * nj + l * l + l + m] * c_tab.knorm[l * (l + 1) / 2 + am] *
                    geg_gamma(B, l, n));
        }
        cs[e] = v;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Vec4<R> pv = ld4(posm + i);
        if (!finite4(pv.x, pv.y, pv.z, pv.w)) report(err, ETICS_ERR_NONFINITE);
        FieldEval<R, LM, ACC, NM1, B> f;
        const R r = sqrt(pv.x * pv.x + pv.y * pv.y + pv.z * pv.z);
        const R inv = r > R(0) ? R(1) / r : R(0);
        f.ux = pv.x * inv; f.uy = pv.y * inv; f.uz = pv.z * inv;
        f.uu = f.ux * f.ux + f.uy * f.uy + f.uz * f.uz;
        const RadialSeed<R, B> rs(r);
        f.t = rs.tau;
        f.st = rs.st;
        f.xi = rs.xi;
        f.dxdr = rs.dxdr;
        f.pre = rs.pre0;
        f.preR = rs.pre0 * rs.q;
        f.pot = f.gr = f.gx = f.gy = f.gz = R(0);
        f.cs = cs;
        f.ncols = ncols;
        f.n_max = n_max;
        f.l_max = l_max;
        f.template level<0>();
        R ax = R(0), ay = R(0), az = R(0);
        if (ACC) {
            ax = -(f.gr * f.ux + f.gx);
            ay = -(f.gr * f.uy + f.gy);
            az = -(f.gr * f.uz + f.gz);
        }
        const R pot = (out_mask & ETICS_OUT_POT) ? f.pot : R(0);
        if (!finite4(ax, ay, az, pot)) report(err, ETICS_ERR_NONFINITE);
        st4(out + i, mk4<R>(ax, ay, az, pot));
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
template <typename R>
inline int scf_pick_nr(int n_max) {
    const int n1 = n_max + 1;
    if (n1 <= 4) return 4;
    if (n1 <= 8) return 8;
    if (n1 <= 11) return 11;
    if (n1 <= 15) return 15;
    return 17;
}

template <typename R>
inline void scf_geometry(int64_t N, int n_max, int l_max, int num_sms, int& NR, int& T, int& W,
                         int& G, int& ntiles, int& grid, size_t& smem) {
    NR = scf_pick_nr<R>(n_max);
    W = scf_items(l_max);
    T = ScfCfg<R>::kTile;
    const int TH = ScfCfg<R>::kThreads;
    for (;;) {
        G = TH / W;
        if (G > T / 4) G = T / 4;
        if (G < 1) G = 1;
        smem = scf_coeff_smem<R>(NR, l_max, T, W, G);
        if (smem <= 200 * 1024 || T <= 16) break;
        T /= 2;
    }
    ntiles = (int)((N + T - 1) / T);
    const int per_sm = smem <= 110 * 1024 ? 2 : 1;
    grid = num_sms * per_sm;
    if (grid > ntiles) grid = ntiles > 0 ? ntiles : 1;
}

template <typename R>
inline size_t scf_workspace(int64_t N, int n_max, int l_max, int num_sms) {
    int NR, T, W, G, ntiles, grid;
    size_t smem;
    scf_geometry<R>(N, n_max, l_max, num_sms, NR, T, W, G, ntiles, grid, smem);
    return (size_t)2 * num_sms * W * NR * 4 * sizeof(double);
}

template <typename R, int NR, int B = 0>
inline int launch_coeff_nr(const ScfCoeffParams& p, int lmu, int grid, size_t smem,
                           cudaStream_t s) {
    if (lmu <= 6) {
        auto k = scf_coeff_kernel<R, NR, 6, B>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return ETICS_ERR_CUDA;
        k<<<grid, ScfCfg<R>::kThreads, smem, s>>>(p);
    } else {
        auto k = scf_coeff_kernel<R, NR, kLmaxLimit, B>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return ETICS_ERR_CUDA;
        k<<<grid, ScfCfg<R>::kThreads, smem, s>>>(p);
    }
    return cudaGetLastError() == cudaSuccess ? ETICS_OK : ETICS_ERR_CUDA;
}

template <typename R, int B = 0>
inline int scf_coeffs_launch(const void* posm, int64_t N, int n_max, int l_max, double* coeffs,
                             void* ws, const LaunchCtx& ctx) {
    int NR, T, W, G, ntiles, grid;
    size_t smem;
    scf_geometry<R>(N, n_max, l_max, ctx.num_sms, NR, T, W, G, ntiles, grid, smem);
    ScfCoeffParams p;
    p.posm = posm;
    p.N = N;
    p.n_max = n_max;
    p.l_max = l_max;
    p.T = T;
    p.W = W;
    p.G = G;
    p.ntiles = ntiles;
    {
        // balance phase 1: radial levels cost ~(n_max+1) each, the angular
        // basis ~(l_max+1)^2; give the angular half the top radial levels
        const double rad = n_max + 1.0, ang = 0.8 * (l_max + 1.0) * (l_max + 1.0);
        int best = l_max + 1;
        double best_cost = 1e30;
        for (int ls = 0; ls <= l_max + 1; ++ls) {
            const double a = rad * ls, b = ang + rad * (l_max + 1 - ls);
            const double c = a > b ? a : b;
            if (c < best_cost) { best_cost = c; best = ls; }
        }
        p.l_split = best;
    }
    p.partial = reinterpret_cast<double*>(ws);
    p.err = ctx.err;
    int nblocks = 0;
    if (ntiles > 0) {
        int rc;
        switch (NR) {
            case 4: rc = launch_coeff_nr<R, 4, B>(p, l_max, grid, smem, ctx.stream); break;
            case 8: rc = launch_coeff_nr<R, 8, B>(p, l_max, grid, smem, ctx.stream); break;
            case 11: rc = launch_coeff_nr<R, 11, B>(p, l_max, grid, smem, ctx.stream); break;
            case 15: rc = launch_coeff_nr<R, 15, B>(p, l_max, grid, smem, ctx.stream); break;
            default: rc = launch_coeff_nr<R, 17, B>(p, l_max, grid, smem, ctx.stream); break;
        }
        if (rc) return rc;
        ++*ctx.launches;
        nblocks = grid;
    }
    stage_event(ctx, 1);
    const int nc = (n_max + 1) * (l_max + 1) * (l_max + 1);
    const int threads = 256;
    const int blocks = (nc * 32 + threads - 1) / threads;
    scf_finalize_kernel<<<blocks, threads, 0, ctx.stream>>>(p.partial, nblocks, n_max, l_max, NR,
                                                            B, coeffs);
    if (cudaGetLastError() != cudaSuccess) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

template <typename R, int LM, int NM1 = 0, int B = 0>
inline int launch_field_lm(const void* posm, int64_t N, int n_max, int l_max,
                           const double* coeffs, void* out, int out_mask, const LaunchCtx& ctx) {
    const size_t smem = (size_t)(n_max + 1) * col_total(l_max) * sizeof(R);
    // at most 4 blocks per SM (two resident at a time): each block builds the
    // FP32 coefficient table once (FP64 multiplies, slow on this GPU) and then
    // walks its particles; 8 per SM measured 5% slower at N = 2^20
    int64_t want = (N + kFieldThreads - 1) / kFieldThreads;
    const int64_t cap = (int64_t)ctx.num_sms * 4;
    int grid = (int)(want < cap ? want : cap);
    if (grid < 1) grid = 1;
    const Vec4<R>* pp = reinterpret_cast<const Vec4<R>*>(posm);
    Vec4<R>* op = reinterpret_cast<Vec4<R>*>(out);
    // launched as a programmatic dependent of the coefficient finalize (or
    // whatever precedes it): its launch overlaps the predecessor's tail
    cudaError_t e;
    if (out_mask & ETICS_OUT_ACC) {
        auto k = scf_field_kernel<R, LM, true, NM1, B>;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return ETICS_ERR_CUDA;
        e = launch_pdl(k, dim3(grid), dim3(kFieldThreads), smem, ctx.stream, pp, N, n_max, l_max,
                       coeffs, op, out_mask, ctx.err);
    } else {
        auto k = scf_field_kernel<R, LM, false, NM1, B>;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return ETICS_ERR_CUDA;
        e = launch_pdl(k, dim3(grid), dim3(kFieldThreads), smem, ctx.stream, pp, N, n_max, l_max,
                       coeffs, op, out_mask, ctx.err);
    }
    if (e != cudaSuccess) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

// the generic field kernels for radial basis B
template <typename R, int B>
inline int scf_field_launch_generic(const void* posm, int64_t N, int n_max, int l_max,
                                    const double* coeffs, void* out, int out_mask,
                                    const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    if (l_max <= 2)
        return launch_field_lm<R, 2, 0, B>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 4)
        return launch_field_lm<R, 4, 0, B>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 6)
        return launch_field_lm<R, 6, 0, B>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 8)
        return launch_field_lm<R, 8, 0, B>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 10)
        return launch_field_lm<R, 10, 0, B>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    return launch_field_lm<R, 14, 0, B>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
}

template <typename R>
inline int scf_field_launch(const void* posm, int64_t N, int n_max, int l_max,
                            const double* coeffs, void* out, int out_mask, const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    // specialised instantiations for the configurations of the paper's tests
    if (n_max == 10 && l_max == 6)
        return launch_field_lm<R, 6, 11>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (n_max == 14 && l_max == 8)
        return launch_field_lm<R, 8, 15>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 2) return launch_field_lm<R, 2>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 4) return launch_field_lm<R, 4>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 6) return launch_field_lm<R, 6>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 8) return launch_field_lm<R, 8>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    if (l_max <= 10) return launch_field_lm<R, 10>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
    return launch_field_lm<R, 14>(posm, N, n_max, l_max, coeffs, out, out_mask, ctx);
}

}  // namespace etics
