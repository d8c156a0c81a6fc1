// etics_mex_impl.cuh -- MEX kernels after the radial sort (templated on the
// arithmetic type; instantiated in etics_mex_f32.cu / etics_mex_f64.cu).
//
// Method (paper Sec. 2.4 eqs. 15-17, the sorted cumulative sums of Sec. 2.2):
//   q_lm(i) = sum_{j before i} m_j r_j^l Y_lm(j),  p_lm(i) = sum_{j after i} m_j r_j^-(l+1) Y_lm(j)
//   Phi_i   = -sum_l 4pi/(2l+1) sum_m [q_lm(i) r_i^-(l+1) + p_lm(i) r_i^l] Y_lm(i)
// and a_i = -grad Phi_i at fixed q, p.
//
// GB300 design (the paper ran one library scan per (l, m) and direction):
//   pass 1  gathers the particles in radial order (sorted copy), and reduces
//           each tile's moments m rho^l Y and m rho^-(l+1) Y (rho = r / s_t,
//           s_t a power of two per tile, so FP32 never overflows) to FP64.
//           It also scans each thread's sums over its kMexP particles inside
//           the tile and stores every thread's exclusive prefix (inner) and
//           suffix (outer).
//   carry   scans the per-tile FP64 sums in a fixed order: exclusive forward
//           for the inner moments, exclusive reverse (a true suffix sum) for
//           the outer ones -- deterministic.
//   pass 2  adds the tile carry to those per-thread prefixes and suffixes,
//           evaluates the field at every particle from the exclusive q and p
//           in a forward and a reverse sweep, and scatters (a, Phi) back to
//           the caller's order.
// All harmonics are the unnormalised Cartesian solid harmonics of
// etics_common.cuh; the MEX weights (l-m)!/(l+m)! (x2 for m > 0) restore the
// orthonormal normalisation and the 4pi/(2l+1) factor at once.
#pragma once

#include "etics_internal.h"

namespace etics {

constexpr int kMexThreads = 128;
// particles per thread (consecutive).  7 rather than 8: at N = 2^20 the 1171
// tiles of 896 particles fill 1.93 waves of the 608 resident blocks instead
// of 1.68 (1024 tiles), measured pass 1 57.3 -> 53.3 us, pass 2 67.5 -> 61.5 us
constexpr int kMexP = 7;
constexpr int kMexTile = kMexThreads * kMexP;     // 896
constexpr int kMexLB = kMexLmaxLimit;             // compiled level bound (10)
constexpr int kMexNC = 49;                        // components of one level group, at most

// Level groups: the per-thread moment arrays hold the components of one group
// of levels, so that l_max up to kMexLB needs no more registers than l_max = 6.
// A group's harmonics are recurred from level 0 (cheap next to the sums).
constexpr int kMexGroups = 3;
__host__ __device__ constexpr int mex_group_l0(int g) { return g == 0 ? 0 : (g == 1 ? 7 : 9); }
__host__ __device__ constexpr int mex_group_l1(int g) { return g == 0 ? 6 : (g == 1 ? 8 : 10); }
__host__ __device__ constexpr int mex_ncomp(int l_max) { return (l_max + 1) * (l_max + 1); }
// components per side in the buffers: the l_max <= 6 kernels always use the
// full 49 (zeros above l_max), so that their strides and loops are constants
__host__ __device__ constexpr int mex_layout_ncomp(int l_max) {
    return l_max <= 6 ? kMexNC : mex_ncomp(l_max);
}
static_assert(mex_group_l1(kMexGroups - 1) == kMexLB, "groups cover the compiled levels");
static_assert(mex_ncomp(6) <= kMexNC && mex_ncomp(8) - mex_ncomp(6) <= kMexNC &&
              mex_ncomp(10) - mex_ncomp(8) <= kMexNC, "group size");
inline int mex_ngroups(int l_max) {
    int g = 1;
    while (g < kMexGroups && mex_group_l0(g) <= l_max) ++g;
    return g;
}

inline int mex_tiles(int64_t N) { return (int)((N + kMexTile - 1) / kMexTile); }

// shared-memory slot of tile particle i (thread i / kMexP owns particles
// i..i+kMexP-1): stored particle-major so that a warp reading its threads'
// k-th particles touches consecutive 16-byte words (no bank conflicts)
__host__ __device__ constexpr int mex_slot(int i) {
    return (i % kMexP) * kMexThreads + i / kMexP;
}

// tile scale exponent: s_t = 2^e with e halfway (in log2) between the first
// and last radius of the tile (first radius 0 -> use the last)
template <typename R>
__device__ __forceinline__ int tile_exponent(R r_first, R r_last) {
    if (!(r_last > R(0))) return 0;
    const int el = ilogb(r_last);
    const int ef = r_first > R(0) ? ilogb(r_first) : el;
    const int s = ef + el;
    return s >= 0 ? s / 2 : -((-s + 1) / 2);
}

template <typename R>
__device__ __forceinline__ R radius(R x, R y, R z) {
    return sqrt(x * x + y * y + z * z);
}

template <typename R>
struct MexParticle {
    R ux, uy, uz, uu, rho, m;
    bool origin;
    __device__ __forceinline__ void init(const Vec4<R>& v, R scale) {
        const R r = radius<R>(v.x, v.y, v.z);
        origin = !(r > R(0));
        const R inv = origin ? R(0) : R(1) / r;
        ux = v.x * inv; uy = v.y * inv; uz = v.z * inv;
        uu = ux * ux + uy * uy + uz * uz;
        rho = r * scale;
        m = v.w;
    }
};

// moment of column c of level L: index L*L + c
template <typename R, int L>
__device__ __forceinline__ R harm_col(const R* C, const R* S, int c) {
    return c == 0 ? C[0] : ((c & 1) ? C[(c + 1) / 2] : S[c / 2]);
}

// ---- moments of one particle added to (ain, aout): levels L0..L1 of the
// group (component L*L + c at index L*L + c - L0*L0), levels below L0 only
// recurred
template <typename R, int L0, int L1, int L>
__device__ __forceinline__ void mex_moments(R (&C)[3][L1 + 1], R (&S)[3][L1 + 1],
                                            const MexParticle<R>& pt, int l_max, R win, R wout,
                                            R irho, R (&ain)[kMexNC], R (&aout)[kMexNC]) {
    if constexpr (L <= L1) {
        if (L > l_max) return;
        constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
        harm_level<R, L>(C[s1], S[s1], C[s2], S[s2], pt.ux, pt.uy, pt.uz, pt.uu, C[s0], S[s0]);
        if constexpr (L >= L0) {
            constexpr int o = L * L - L0 * L0;
#pragma unroll
            for (int c = 0; c <= 2 * L; ++c) {
                const R y = harm_col<R, L>(C[s0], S[s0], c);
                ain[o + c] = fma(win, y, ain[o + c]);
                aout[o + c] = fma(wout, y, aout[o + c]);
            }
        }
        mex_moments<R, L0, L1, L + 1>(C, S, pt, l_max, win * pt.rho, wout * irho, irho, ain,
                                      aout);
    }
}

template <typename R, int L0, int L1>
__device__ __forceinline__ void particle_moments(const MexParticle<R>& pt, int l_max,
                                                 R (&ain)[kMexNC], R (&aout)[kMexNC]) {
    R C[3][L1 + 1], S[3][L1 + 1];
    const R irho = pt.origin ? R(0) : R(1) / pt.rho;
    // a particle at the origin has no outer moment (nothing lies inside it)
    mex_moments<R, L0, L1, 0>(C, S, pt, l_max, pt.m, pt.origin ? R(0) : pt.m * irho, irho, ain,
                              aout);
}

// ---- forward sweep, one particle: inner (q) part of the field, then q += own
// inner moment.  On entry q is the inner sum over the particles before this
// one (exclusive).  In tile units (rho = r / s):
//   Phi_q = -(1/s) sum_l rho^-(l+1) sum_m w_lm q Y
//   a_q   = (1/s^2) sum_l rho^-(l+2) sum_m w_lm q [G - (2l+1) Y u]
// with Y, G the unnormalised harmonic and its gradient at the unit vector u.
template <typename R, int L0, int L1, int L, bool ACC>
__device__ __forceinline__ void mex_fwd(R (&C)[3][L1 + 1], R (&S)[3][L1 + 1],
                                        const MexParticle<R>& pt, int l_max, R win, R rinv,
                                        R irho, R (&q)[kMexNC], R& pot, R& ax, R& ay, R& az) {
    if constexpr (L <= L1) {
        if (L > l_max) return;
        constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
        harm_level<R, L>(C[s1], S[s1], C[s2], S[s2], pt.ux, pt.uy, pt.uz, pt.uu, C[s0], S[s0]);
        if constexpr (L >= L0) {
            constexpr int o = L * L - L0 * L0;
            if (!pt.origin) {
                R P = R(0), vx = R(0), vy = R(0), vz = R(0);
                R qc[L + 1], qs[L + 1];
#pragma unroll
                for (int mm = 0; mm <= L; ++mm) {
                    const R w = mex_w<R>(L * (L + 1) / 2 + mm);
                    const int cc = o + (mm == 0 ? 0 : 2 * mm - 1);
                    qc[mm] = w * q[cc];
                    P = fma(qc[mm], C[s0][mm], P);
                    qs[mm] = R(0);
                    if (mm > 0) {
                        qs[mm] = w * q[cc + 1];
                        P = fma(qs[mm], S[s0][mm], P);
                    }
                }
                if (ACC && L >= 1) grad_contract<R, L>(C[s1], S[s1], qc, qs, vx, vy, vz);
                pot = fma(rinv, P, pot);
                if (ACC) {
                    const R f = rinv * irho;
                    const R k = R(2 * L + 1) * P;
                    ax = fma(f, vx - k * pt.ux, ax);
                    ay = fma(f, vy - k * pt.uy, ay);
                    az = fma(f, vz - k * pt.uz, az);
                }
            }
#pragma unroll
            for (int c = 0; c <= 2 * L; ++c)
                q[o + c] = fma(win, harm_col<R, L>(C[s0], S[s0], c), q[o + c]);
        }
        mex_fwd<R, L0, L1, L + 1, ACC>(C, S, pt, l_max, win * pt.rho, rinv * irho, irho, q, pot,
                                       ax, ay, az);
    }
}

// ---- reverse sweep, one particle: outer (p) part of the field, then p += own
// outer moment.  On entry p is the outer sum over the particles after this one:
//   Phi_p = -(1/s) sum_l rho^l sum_m w_lm p Y,   a_p = (1/s^2) sum_l rho^(l-1) sum_m w_lm p G
template <typename R, int L0, int L1, int L, bool ACC>
__device__ __forceinline__ void mex_rev(R (&C)[3][L1 + 1], R (&S)[3][L1 + 1],
                                        const MexParticle<R>& pt, int l_max, R wout, R rl,
                                        R rlm1, R irho, R (&p)[kMexNC], R& pot, R& ax, R& ay,
                                        R& az) {
    if constexpr (L <= L1) {
        if (L > l_max) return;
        constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
        harm_level<R, L>(C[s1], S[s1], C[s2], S[s2], pt.ux, pt.uy, pt.uz, pt.uu, C[s0], S[s0]);
        if constexpr (L >= L0) {
            constexpr int o = L * L - L0 * L0;
            R P = R(0), vx = R(0), vy = R(0), vz = R(0);
            R pc[L + 1], ps[L + 1];
#pragma unroll
            for (int mm = 0; mm <= L; ++mm) {
                const R w = mex_w<R>(L * (L + 1) / 2 + mm);
                const int cc = o + (mm == 0 ? 0 : 2 * mm - 1);
                pc[mm] = w * p[cc];
                P = fma(pc[mm], C[s0][mm], P);
                ps[mm] = R(0);
                if (mm > 0) {
                    ps[mm] = w * p[cc + 1];
                    P = fma(ps[mm], S[s0][mm], P);
                }
            }
            if (ACC && L >= 1) grad_contract<R, L>(C[s1], S[s1], pc, ps, vx, vy, vz);
            pot = fma(rl, P, pot);
            if (ACC && L >= 1) {
                ax = fma(rlm1, vx, ax);
                ay = fma(rlm1, vy, ay);
                az = fma(rlm1, vz, az);
            }
#pragma unroll
            for (int c = 0; c <= 2 * L; ++c)
                p[o + c] = fma(wout, harm_col<R, L>(C[s0], S[s0], c), p[o + c]);
        }
        mex_rev<R, L0, L1, L + 1, ACC>(C, S, pt, l_max, wout * irho, rl * pt.rho, rl, irho, p,
                                       pot, ax, ay, az);
    }
}

// Exclusive scan over the 32 lanes of a warp of each of the kMexNC components
// in v (forward: prefix in lane order; backward: suffix), in two rounds of at
// most kMexScanHalf components.  buf: the warp's 32 x kMexScanHalf slots (row
// = lane; the odd row length keeps both access patterns free of bank
// conflicts).  total[c] receives the warp's sum of component c.
constexpr int kMexScanHalf = (kMexNC + 1) / 2;
static_assert(kMexScanHalf % 2 == 1, "row length must be odd");
template <typename R, bool kForward, int C0, int NC>
__device__ __forceinline__ void scan_rows_part(R (&v)[kMexNC], R* buf, R* total, int lane) {
#pragma unroll
    for (int j = 0; j < NC; ++j) buf[lane * kMexScanHalf + j] = v[C0 + j];
    __syncwarp();
    if (lane < NC) {
        R run = R(0);
#pragma unroll
        for (int t = 0; t < 32; ++t) {
            const int r = kForward ? t : 31 - t;
            const R x = buf[r * kMexScanHalf + lane];
            buf[r * kMexScanHalf + lane] = run;
            run += x;
        }
        total[C0 + lane] = run;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < NC; ++j) v[C0 + j] = buf[lane * kMexScanHalf + j];
    __syncwarp();
}
template <typename R, bool kForward>
__device__ __forceinline__ void scan_rows(R (&v)[kMexNC], R* buf, R* total, int lane) {
    scan_rows_part<R, kForward, 0, kMexScanHalf>(v, buf, total, lane);
    scan_rows_part<R, kForward, kMexScanHalf, kMexNC - kMexScanHalf>(v, buf, total, lane);
}

// ---------------------------------------------------------------------------
// pass 1: gather into radial order + per-tile FP64 moment sums
// ---------------------------------------------------------------------------
// resident blocks per SM the kernels' registers are sized for: FP32 with one
// level group 4 (16 warps hide the gather latency); the multi-group kernels
// and FP64 need more registers (FP64 pass 2 at 4 blocks spilled ~1 KB)
template <typename R, int NG>
constexpr int mex_pass1_blocks() { return sizeof(R) == 4 ? (NG == 1 ? 4 : 3) : 1; }
template <typename R, int NG>
constexpr int mex_pass2_blocks() { return sizeof(R) == 4 ? (NG == 1 ? 4 : 2) : (NG == 1 ? 2 : 1); }

template <typename R, int NG>
__global__ void __launch_bounds__(kMexThreads, mex_pass1_blocks<R, NG>())
mex_pass1_kernel(const Vec4<R>* __restrict__ posm, const uint32_t* __restrict__ perm, int64_t N,
                 int l_max, Vec4<R>* __restrict__ sorted, double* __restrict__ tile_agg,
                 R* __restrict__ thread_sums, unsigned* err) {
    __shared__ Vec4<R> s_pt[kMexTile];
    __shared__ R s_red[kMexThreads / 32][2 * kMexNC];
    pdl_wait();
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kMexTile;
    const int64_t rem = N - base;
    const int nt = (int)(rem < kMexTile ? rem : kMexTile);
    // gather in radial order: coalesced index loads, independent particle loads
    uint32_t idx[kMexP];
#pragma unroll
    for (int j = 0; j < kMexP; ++j) {
        const int i = tid + j * kMexThreads;
        idx[j] = i < nt ? perm[base + i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kMexP; ++j) {
        const int i = tid + j * kMexThreads;
        Vec4<R> v = mk4<R>(R(0), R(0), R(0), R(0));
        if (i < nt) {
            // an index >= N can only come from a sort whose lookback timed
            // out (already reported): it gathers a massless particle at 0
            if ((int64_t)idx[j] < N) {
                v = ld4(posm + idx[j]);
                if (!finite4(v.x, v.y, v.z, v.w)) {
                    report(err, ETICS_ERR_NONFINITE);
                    v = mk4<R>(R(0), R(0), R(0), R(0));
                }
            }
            st4(sorted + base + i, v);
        }
        st4(&s_pt[mex_slot(i)], v);
    }
    __syncthreads();
    int e;
    {
        const Vec4<R> a = s_pt[mex_slot(0)], b = s_pt[mex_slot(nt - 1)];
        e = tile_exponent<R>(radius<R>(a.x, a.y, a.z), radius<R>(b.x, b.y, b.z));
    }
    const R scale = ldexp(R(1), -e);
    const int lane = tid & 31, warp = tid >> 5;
    // One level group per iteration: this thread's moment sums over its kMexP
    // particles; their exclusive prefix (inner) and suffix (outer) over the
    // tile, by a transposed scan through shared memory (every thread writes
    // its row of sums, each lane scans one component serially down the 32
    // rows in lane order, every thread reads its row back; the rows live
    // where the particles were); every thread's prefix and suffix stored, the
    // tile's FP64 sums (tile scale undone) stored.  l_max <= 6 is the single
    // group with constant sizes.
    const int ncomp = NG == 1 ? kMexNC : mex_layout_ncomp(l_max);
    for (int g = 0; g < NG; ++g) {
        const int L0 = mex_group_l0(g), L1 = mex_group_l1(g);
        if (L0 > l_max) break;
        if (g > 0) {
            // the previous group's scan rows overwrote the particles
            __syncthreads();
            for (int i = tid; i < kMexTile; i += kMexThreads)
                st4(&s_pt[mex_slot(i)],
                    i < nt ? ld4(sorted + base + i) : mk4<R>(R(0), R(0), R(0), R(0)));
            __syncthreads();
        }
        const int c0 = L0 * L0;
        const int gn = NG == 1 ? kMexNC : mex_ncomp(L1 < l_max ? L1 : l_max) - c0;
        R ain[kMexNC], aout[kMexNC];
#pragma unroll
        for (int c = 0; c < kMexNC; ++c) { ain[c] = R(0); aout[c] = R(0); }
#pragma unroll 1
        for (int k = 0; k < kMexP; ++k) {
            MexParticle<R> pt;
            pt.init(s_pt[k * kMexThreads + tid], scale);
            if (NG == 1 || g == 0) particle_moments<R, 0, 6>(pt, l_max, ain, aout);
            else if (g == 1) particle_moments<R, 7, 8>(pt, l_max, ain, aout);
            else particle_moments<R, 9, 10>(pt, l_max, ain, aout);
        }
        static_assert(kMexThreads / 32 * 32 * kMexScanHalf * sizeof(R) <= sizeof(s_pt), "rows");
        __syncthreads();
        R* rows = reinterpret_cast<R*>(s_pt) + warp * 32 * kMexScanHalf;
        scan_rows<R, true>(ain, rows, &s_red[warp][0], lane);
        scan_rows<R, false>(aout, rows, &s_red[warp][kMexNC], lane);
        __syncthreads();
        {
            R* ts = thread_sums + (size_t)blockIdx.x * 2 * ncomp * kMexThreads + tid;
#pragma unroll
            for (int c = 0; c < kMexNC; ++c) {
                if (c < gn) {
                    R q = R(0), pp = R(0);
                    for (int w = 0; w < warp; ++w) q += s_red[w][c];
                    for (int w = kMexThreads / 32 - 1; w > warp; --w) pp += s_red[w][kMexNC + c];
                    ts[(size_t)(c0 + c) * kMexThreads] = q + ain[c];
                    ts[(size_t)(ncomp + c0 + c) * kMexThreads] = pp + aout[c];
                }
            }
        }
        for (int c = tid; c < 2 * gn; c += kMexThreads) {
            const bool inner = c < gn;
            const int lc = inner ? c : c - gn;
            double sum = 0.0;
            for (int w = 0; w < kMexThreads / 32; ++w)
                sum += (double)s_red[w][(inner ? 0 : kMexNC) + lc];
            const int cc = c0 + lc;
            int l = 0;
            while ((l + 1) * (l + 1) <= cc) ++l;
            // undo the tile scale: inner moments scale as s^l, outer as s^-(l+1)
            sum = inner ? ldexp(sum, l * e) : ldexp(sum, -(l + 1) * e);
            if (!isfinite(sum)) report(err, ETICS_ERR_NONFINITE);
            tile_agg[(size_t)blockIdx.x * 2 * ncomp + (inner ? 0 : ncomp) + cc] = sum;
        }
    }
}

// ---------------------------------------------------------------------------
// carry: exclusive scans of the tile sums over tiles, one block per
// component; forward for inner moments, reverse for outer (fixed order).
// FP64 arithmetic is slow on this GPU (about 1/76 of the FP32 rate), so the scan
// keeps the FP64 additions per block near the minimum: thread t owns a
// contiguous run of scan positions, adds them in order, the run totals are
// scanned by one warp-shuffle scan per warp and one over the warp totals,
// then each thread writes its positions' exclusive sums.  Every addition
// order depends only on (ntiles, ncomp): deterministic.
// ---------------------------------------------------------------------------
constexpr int kCarryThreads = 256;
constexpr int kCarryWarps = kCarryThreads / 32;
static __global__ void __launch_bounds__(kCarryThreads)
mex_carry_kernel(const double* __restrict__ tile_agg, int ntiles, int ncomp,
                 double* __restrict__ carry) {
    __shared__ double s_w[kCarryWarps];
    pdl_wait();   // the tile sums come from pass 1
    const int c = blockIdx.x;
    const bool rev = c >= ncomp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int chunk = (ntiles + kCarryThreads - 1) / kCarryThreads;
    const int o0 = tid * chunk;
    const int o1 = o0 + chunk < ntiles ? o0 + chunk : ntiles;
    const size_t stride = (size_t)2 * ncomp;
    auto at = [&](int o) { return (size_t)(rev ? ntiles - 1 - o : o) * stride + c; };
    // this thread's run, in scan order (read coherently after the wait)
    double local = 0.0;
#pragma unroll 4
    for (int o = o0; o < o1; ++o) local += __ldcg(tile_agg + at(o));
    // inclusive scan of the run totals over the warp
    double x = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const double t = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += t;
    }
    double ex = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) ex = 0.0;
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the warp totals, in warp order
        double w = lane < kCarryWarps ? s_w[lane] : 0.0;
#pragma unroll
        for (int d = 1; d < kCarryWarps; d <<= 1) {
            const double t = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += t;
        }
        double we = __shfl_up_sync(0xffffffffu, w, 1);
        if (lane == 0) we = 0.0;
        __syncwarp();
        if (lane < kCarryWarps) s_w[lane] = we;
    }
    __syncthreads();
    double run = warp == 0 ? ex : s_w[warp] + ex;
    for (int o = o0; o < o1; ++o) {
        const size_t i = at(o);
        carry[i] = run;
        run += __ldcg(tile_agg + i);
    }
}

// ---------------------------------------------------------------------------
// pass 2: field from the exclusive sums, per level group
// ---------------------------------------------------------------------------
// Group G: this thread's exclusive inner sum (tile carry + in-tile prefix from
// pass 1), the forward sweep (inner part of the field, added to s_f), its
// exclusive outer sum (a true suffix sum, never total minus prefix), the
// reverse sweep (outer part); the last group present completes each
// particle's field and scatters it back to the caller's order.
template <typename R, int NG, int G, bool ACC>
__device__ __forceinline__ void mex_pass2_group(const Vec4<R>* s_pt, Vec4<R>* s_f, R* s_q0,
                                                R* s_p0, const double* carry,
                                                const R* thread_sums, const uint32_t* perm,
                                                int64_t base, int64_t N, int l_max, int e,
                                                R scale, bool last, Vec4<R>* out, int out_mask,
                                                unsigned* err) {
    constexpr int L0 = mex_group_l0(G), L1 = mex_group_l1(G);
    if (L0 > l_max) return;
    const int tid = threadIdx.x;
    const int ncomp = NG == 1 ? kMexNC : mex_layout_ncomp(l_max);
    const int c0 = L0 * L0;
    const int gn = NG == 1 ? kMexNC : mex_ncomp(L1 < l_max ? L1 : l_max) - c0;
    if (G > 0) __syncthreads();   // the previous group's readers of s_q0 / s_p0 are done
    for (int c = tid; c < 2 * gn; c += kMexThreads) {
        const bool inner = c < gn;
        const int lc = inner ? c : c - gn;
        const int cc = c0 + lc;
        int l = 0;
        while ((l + 1) * (l + 1) <= cc) ++l;
        const double v = carry[(size_t)blockIdx.x * 2 * ncomp + (inner ? 0 : ncomp) + cc];
        if (inner) s_q0[lc] = (R)ldexp(v, -l * e);
        else s_p0[lc] = (R)ldexp(v, (l + 1) * e);
    }
    __syncthreads();
    const R* ts = thread_sums + (size_t)blockIdx.x * 2 * ncomp * kMexThreads + tid;
    R a[kMexNC];
#pragma unroll
    for (int c = 0; c < kMexNC; ++c)
        a[c] = c < gn ? s_q0[c] + ts[(size_t)(c0 + c) * kMexThreads] : R(0);
#pragma unroll 1
    for (int k = 0; k < kMexP; ++k) {
        MexParticle<R> pt;
        pt.init(s_pt[k * kMexThreads + tid], scale);
        const R irho = pt.origin ? R(0) : R(1) / pt.rho;
        R C[3][L1 + 1], S[3][L1 + 1];
        R pot = R(0), ax = R(0), ay = R(0), az = R(0);
        if (G > 0) {
            const Vec4<R> f = s_f[k * kMexThreads + tid];
            ax = f.x; ay = f.y; az = f.z; pot = f.w;
        }
        mex_fwd<R, L0, L1, 0, ACC>(C, S, pt, l_max, pt.m, irho, irho, a, pot, ax, ay, az);
        st4(&s_f[k * kMexThreads + tid], mk4<R>(ax, ay, az, pot));
    }
    R b[kMexNC];
#pragma unroll
    for (int c = 0; c < kMexNC; ++c)
        b[c] = c < gn ? s_p0[c] + ts[(size_t)(ncomp + c0 + c) * kMexThreads] : R(0);
    const R s1 = scale, s2 = scale * scale;
#pragma unroll 1
    for (int k = kMexP - 1; k >= 0; --k) {
        MexParticle<R> pt;
        pt.init(s_pt[k * kMexThreads + tid], scale);
        const R irho = pt.origin ? R(0) : R(1) / pt.rho;
        R C[3][L1 + 1], S[3][L1 + 1];
        const Vec4<R> f = s_f[k * kMexThreads + tid];
        R pot = f.w, ax = f.x, ay = f.y, az = f.z;
        const R wout = pt.origin ? R(0) : pt.m * irho;
        mex_rev<R, L0, L1, 0, ACC>(C, S, pt, l_max, wout, R(1), R(0), irho, b, pot, ax, ay, az);
        if (!last) {
            st4(&s_f[k * kMexThreads + tid], mk4<R>(ax, ay, az, pot));
            continue;
        }
        const int64_t i = base + (int64_t)tid * kMexP + k;
        // perm[i] >= N only after a timed-out sort (reported): no store
        if (i < N && (int64_t)perm[i] < N) {
            const R potv = (out_mask & ETICS_OUT_POT) ? -pot * s1 : R(0);
            const R fx = ACC ? ax * s2 : R(0);
            const R fy = ACC ? ay * s2 : R(0);
            const R fz = ACC ? az * s2 : R(0);
            if (!finite4(fx, fy, fz, potv)) report(err, ETICS_ERR_NONFINITE);
            st4(out + perm[i], mk4<R>(fx, fy, fz, potv));
        }
    }
}

template <typename R, int NG, int G, bool ACC>
__device__ __forceinline__ void mex_pass2_groups(const Vec4<R>* s_pt, Vec4<R>* s_f, R* s_q0,
                                                 R* s_p0, const double* carry,
                                                 const R* thread_sums, const uint32_t* perm,
                                                 int64_t base, int64_t N, int l_max, int e,
                                                 R scale, Vec4<R>* out, int out_mask,
                                                 unsigned* err) {
    if constexpr (G < NG) {
        const bool last = G + 1 == NG || mex_group_l0(G + 1) > l_max;
        mex_pass2_group<R, NG, G, ACC>(s_pt, s_f, s_q0, s_p0, carry, thread_sums, perm, base,
                                       N, l_max, e, scale, last, out, out_mask, err);
        mex_pass2_groups<R, NG, G + 1, ACC>(s_pt, s_f, s_q0, s_p0, carry, thread_sums, perm,
                                            base, N, l_max, e, scale, out, out_mask, err);
    }
}

template <typename R, int NG, bool ACC>
__global__ void __launch_bounds__(kMexThreads, mex_pass2_blocks<R, NG>())
mex_pass2_kernel(const Vec4<R>* __restrict__ sorted, const uint32_t* __restrict__ perm, int64_t N,
                 int l_max, const double* __restrict__ carry, const R* __restrict__ thread_sums,
                 Vec4<R>* __restrict__ out, int out_mask, unsigned* err) {
    __shared__ Vec4<R> s_pt[kMexTile];
    __shared__ Vec4<R> s_f[kMexTile];   // each particle's field so far
    __shared__ R s_q0[kMexNC], s_p0[kMexNC];
    pdl_wait();
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kMexTile;
    const int64_t rem = N - base;
    const int nt = (int)(rem < kMexTile ? rem : kMexTile);
    for (int i = tid; i < kMexTile; i += kMexThreads)
        st4(&s_pt[mex_slot(i)], i < nt ? ld4(sorted + base + i) : mk4<R>(R(0), R(0), R(0), R(0)));
    __syncthreads();
    int e;
    {
        const Vec4<R> a = s_pt[mex_slot(0)], b = s_pt[mex_slot(nt - 1)];
        e = tile_exponent<R>(radius<R>(a.x, a.y, a.z), radius<R>(b.x, b.y, b.z));
    }
    const R scale = ldexp(R(1), -e);
    mex_pass2_groups<R, NG, 0, ACC>(s_pt, s_f, s_q0, s_p0, carry, thread_sums, perm, base, N,
                                    l_max, e, scale, out, out_mask, err);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename R>
struct MexBuffers {
    SortBuffers sort;
    Vec4<R>* sorted;
    double* tile_agg;    // [tile][2 * ncomp]: inner then outer sums (ncomp: mex_layout_ncomp)
    double* carry;       // [tile][2 * ncomp]
    R* thread_sums;      // [tile][2 * ncomp][kMexThreads], in-tile exclusive prefix / suffix
};

// ncomp = mex_layout_ncomp(l_max) components per side
template <typename R>
inline MexBuffers<R> mex_buffers(void* ws, int64_t N, int l_max, size_t* total) {
    MexBuffers<R> b{};
    size_t off = 0;
    b.sort = sort_buffers(ws, N, &off);
    uint8_t* p = reinterpret_cast<uint8_t*>(ws);
    auto take = [&](size_t bytes) {
        uint8_t* q = p ? p + off : nullptr;
        off += (bytes + 255) / 256 * 256;
        return q;
    };
    const size_t n = (size_t)(N > 0 ? N : 1);
    const size_t nt = (size_t)(mex_tiles(N) > 0 ? mex_tiles(N) : 1);
    const size_t nc = (size_t)mex_layout_ncomp(l_max > 0 ? l_max : 0);
    b.sorted = reinterpret_cast<Vec4<R>*>(take(n * sizeof(Vec4<R>)));
    b.tile_agg = reinterpret_cast<double*>(take(nt * 2 * nc * sizeof(double)));
    b.carry = reinterpret_cast<double*>(take(nt * 2 * nc * sizeof(double)));
    b.thread_sums = reinterpret_cast<R*>(take(nt * 2 * nc * kMexThreads * sizeof(R)));
    if (total) *total = off;
    return b;
}

template <typename R>
inline size_t mex_workspace_impl(int64_t N, int l_max) {
    size_t total = 0;
    mex_buffers<R>(nullptr, N, l_max, &total);
    return total;
}

template <typename R, int NG>
inline int mex_passes(const MexBuffers<R>& b, const Vec4<R>* pp, int64_t N, int l_max, void* out,
                      int out_mask, const LaunchCtx& ctx) {
    const int nt = mex_tiles(N);
    const int ncomp = mex_layout_ncomp(l_max);
    if (launch_pdl(mex_pass1_kernel<R, NG>, dim3(nt), dim3(kMexThreads), 0, ctx.stream, pp,
                   (const uint32_t*)b.sort.vals_a, N, l_max, b.sorted, b.tile_agg, b.thread_sums,
                   ctx.err))
        return ETICS_ERR_CUDA;
    ++*ctx.launches;
    stage_event(ctx, 3);
    if (launch_pdl(mex_carry_kernel, dim3(2 * ncomp), dim3(kCarryThreads), 0, ctx.stream,
                   (const double*)b.tile_agg, nt, ncomp, b.carry))
        return ETICS_ERR_CUDA;
    ++*ctx.launches;
    stage_event(ctx, 4);
    Vec4<R>* op = reinterpret_cast<Vec4<R>*>(out);
    const cudaError_t le = (out_mask & ETICS_OUT_ACC)
        ? launch_pdl(mex_pass2_kernel<R, NG, true>, dim3(nt), dim3(kMexThreads), 0, ctx.stream,
                     (const Vec4<R>*)b.sorted, (const uint32_t*)b.sort.vals_a, N, l_max,
                     (const double*)b.carry, (const R*)b.thread_sums, op, out_mask, ctx.err)
        : launch_pdl(mex_pass2_kernel<R, NG, false>, dim3(nt), dim3(kMexThreads), 0, ctx.stream,
                     (const Vec4<R>*)b.sorted, (const uint32_t*)b.sort.vals_a, N, l_max,
                     (const double*)b.carry, (const R*)b.thread_sums, op, out_mask, ctx.err);
    if (le) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    stage_event(ctx, 5);
    return ETICS_OK;
}

template <typename R>
inline int mex_field_impl(const void* posm, int64_t N, int l_max, void* out, int out_mask,
                          void* ws, const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    MexBuffers<R> b = mex_buffers<R>(ws, N, l_max, nullptr);
    stage_event(ctx, 0);
    int rc = radial_sort_impl<R>(posm, N, b.sort, ctx);
    if (rc) return rc;
    stage_event(ctx, 2);
    const Vec4<R>* pp = reinterpret_cast<const Vec4<R>*>(posm);
    // l_max <= 6: one level group (the kernels specialised for it)
    if (mex_ngroups(l_max) == 1) return mex_passes<R, 1>(b, pp, N, l_max, out, out_mask, ctx);
    return mex_passes<R, kMexGroups>(b, pp, N, l_max, out, out_mask, ctx);
}

template <typename R>
inline int radial_order_impl(const void* posm, int64_t N, uint32_t* order, void* ws,
                             const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    MexBuffers<R> b = mex_buffers<R>(ws, N, 0, nullptr);
    int rc = radial_sort_impl<R>(posm, N, b.sort, ctx);
    if (rc) return rc;
    if (cudaMemcpyAsync(order, b.sort.vals_a, (size_t)N * 4, cudaMemcpyDeviceToDevice, ctx.stream))
        return ETICS_ERR_CUDA;
    return ETICS_OK;
}

}  // namespace etics
