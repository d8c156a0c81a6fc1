// etics_scf_bins.cuh -- SCF coefficient pass specialised for a fixed
// (n_max, l_max): each warp owns a "bin" of at most kBinCap harmonic columns
// (a compile-time plan), each lane accumulates the contributions of its own
// particles to the bin's (n, column) coefficients in registers over all the
// tiles it visits, and only the angular basis of a tile goes through shared
// memory.  The radial basis of the bin's levels is evaluated by the lane
// itself (Gegenbauer recursion with immediate constants), so there is no
// per-tile cross-thread reduction and no padding work.  Method as in
// etics_scf_impl.cuh (paper Sec. 2.4 eq. 18, Sec. 2.5 basis).
#pragma once

#include "etics_scf_impl.cuh"

namespace etics {

constexpr int kBinCap = 7;
constexpr int kBinFlushTiles = 16;

struct BinSeg { int l, c0, n; };          // columns c0..c0+n-1 of level l
struct BinDef { int nseg; BinSeg seg[4]; int ncol; };
template <int LM>
struct BinPlan {
    static constexpr int kCols = (LM + 1) * (LM + 1);
    int nbins;
    BinDef bin[kCols];
};

// full bins of one level first (descending l), then the remainders packed
// first-fit decreasing (each remainder stays whole)
template <int LM>
constexpr BinPlan<LM> make_bin_plan() {
    BinPlan<LM> p{};
    p.nbins = 0;
    int rem_l[LM + 1] = {}, rem_c0[LM + 1] = {}, rem_n[LM + 1] = {};
    int nrem = 0;
    for (int l = LM; l >= 0; --l) {
        const int nc = 2 * l + 1;
        int c = 0;
        for (; c + kBinCap <= nc; c += kBinCap) {
            BinDef& b = p.bin[p.nbins++];
            b.nseg = 1;
            b.seg[0] = BinSeg{l, c, kBinCap};
            b.ncol = kBinCap;
        }
        if (c < nc) { rem_l[nrem] = l; rem_c0[nrem] = c; rem_n[nrem] = nc - c; ++nrem; }
    }
    // sort remainders by size (descending), stable
    for (int i = 1; i < nrem; ++i)
        for (int j = i; j > 0 && rem_n[j] > rem_n[j - 1]; --j) {
            int t = rem_n[j]; rem_n[j] = rem_n[j - 1]; rem_n[j - 1] = t;
            t = rem_l[j]; rem_l[j] = rem_l[j - 1]; rem_l[j - 1] = t;
            t = rem_c0[j]; rem_c0[j] = rem_c0[j - 1]; rem_c0[j - 1] = t;
        }
    const int first_rem_bin = p.nbins;
    for (int i = 0; i < nrem; ++i) {
        int target = -1;
        for (int b = first_rem_bin; b < p.nbins; ++b)
            if (p.bin[b].ncol + rem_n[i] <= kBinCap && p.bin[b].nseg < 4) { target = b; break; }
        if (target < 0) { target = p.nbins++; p.bin[target].nseg = 0; p.bin[target].ncol = 0; }
        BinDef& b = p.bin[target];
        b.seg[b.nseg++] = BinSeg{rem_l[i], rem_c0[i], rem_n[i]};
        b.ncol += rem_n[i];
    }
    return p;
}

// column offset of column c of level l inside its bin (for the finalize)
template <int LM>
struct BinIndex {
    int bin[(LM + 1) * (LM + 1)];
    int slot[(LM + 1) * (LM + 1)];
};
template <int LM>
constexpr BinIndex<LM> make_bin_index() {
    BinIndex<LM> ix{};
    constexpr BinPlan<LM> p = make_bin_plan<LM>();
    for (int b = 0; b < p.nbins; ++b) {
        int off = 0;
        for (int s = 0; s < p.bin[b].nseg; ++s) {
            const BinSeg g = p.bin[b].seg[s];
            for (int c = 0; c < g.n; ++c) {
                ix.bin[g.l * g.l + g.c0 + c] = b;
                ix.slot[g.l * g.l + g.c0 + c] = off + c;
            }
            off += g.n;
        }
    }
    return ix;
}

template <int LM>
struct BinConst {
    static constexpr BinPlan<LM> plan = make_bin_plan<LM>();
    static constexpr int nbins = plan.nbins;
};
// device copy of the column -> (bin, slot) map, read with run-time indices
template <int LM>
static __constant__ BinIndex<LM> c_bin_index = make_bin_index<LM>();

struct ScfBinParams {
    const void* posm;
    int64_t N;
    int ntiles;
    double* partial;   // [gridDim.x][nbins][NR][kBinCap]
    unsigned* err;
};

// contributions of one particle to segment S of bin B: the Gegenbauer values
// of the segment's level times the (mass and radial prefactor scaled)
// harmonics of its columns
template <typename R, int NR, int LM, int B, int S>
__device__ __forceinline__ void bin_segment(R (&acc)[NR][kBinCap], const R* Ys, int T, int k,
                                            R xi, R w0, R st) {
    constexpr BinDef bd = BinConst<LM>::plan.bin[B];
    if constexpr (S < bd.nseg) {
        constexpr BinSeg g = bd.seg[S];
        constexpr int off = [] {
            int o = 0;
            for (int s = 0; s < S; ++s) o += BinConst<LM>::plan.bin[B].seg[s].n;
            return o;
        }();
        // w_l = m * (-(1+r)^-1) * (r/(1+r)^2)^l
        R w = w0;
#pragma unroll
        for (int i = 0; i < g.l; ++i) w *= st;
        R y[g.n];
#pragma unroll
        for (int c = 0; c < g.n; ++c) y[c] = w * Ys[(size_t)(g.l * g.l + g.c0 + c) * T + k];
        R cm1 = R(0), cn = R(1);
#pragma unroll
        for (int n = 0; n < NR; ++n) {
            if (n > 0) {
                const R cnew = fma(xi, cn, -geg_bs<R>(g.l, n) * cm1);   // rescaled
                cm1 = cn;
                cn = cnew;
            }
#pragma unroll
            for (int c = 0; c < g.n; ++c) acc[n][off + c] = fma(cn, y[c], acc[n][off + c]);
        }
        bin_segment<R, NR, LM, B, S + 1>(acc, Ys, T, k, xi, w0, st);
    }
}

template <typename R, int NR, int LM, int B>
__device__ __forceinline__ void bin_tile(R (&acc)[NR][kBinCap], const R* Ys, const Vec4<R>* s_rad,
                                         int T, int lane) {
#pragma unroll 1
    for (int k = lane; k < T; k += 32) {
        const Vec4<R> rd = s_rad[k];   // (xi, st, w0, -)
        bin_segment<R, NR, LM, B, 0>(acc, Ys, T, k, rd.x, rd.z, rd.y);
    }
}

template <typename R, int NR, int LM, int B>
__device__ __forceinline__ void bin_dispatch(int warp, R (&acc)[NR][kBinCap], const R* Ys,
                                             const Vec4<R>* s_rad, int T, int lane) {
    if constexpr (B < BinConst<LM>::nbins) {
        if (warp == B) bin_tile<R, NR, LM, B>(acc, Ys, s_rad, T, lane);
        else bin_dispatch<R, NR, LM, B + 1>(warp, acc, Ys, s_rad, T, lane);
    }
}

// TP: particles per tile (at most one per thread in phase 1; the default,
// one per thread, keeps every thread busy there; fewer particles per tile
// keep the two basis buffers of a large l_max within shared memory).
// MINB: resident blocks per SM the registers are sized for.
template <int LM>
constexpr int bins_threads() { return BinConst<LM>::nbins * 32; }
template <typename R, int NR, int LM, int TP = bins_threads<LM>(), int MINB = 2>
__global__ void __launch_bounds__(bins_threads<LM>(), MINB)
scf_coeff_bins_kernel(ScfBinParams p) {
    constexpr int NB = BinConst<LM>::nbins;
    constexpr int TH = NB * 32;         // threads: one warp per bin
    constexpr int T = TP;               // particles per tile
    static_assert(T <= TH && T % 32 == 0, "tile");
    constexpr int NCOL = (LM + 1) * (LM + 1);
    constexpr int NOUT = NB * NR * kBinCap;
    using V4 = Vec4<R>;
    // dynamic shared memory: accd [NOUT] doubles, then two buffers of
    // s_rad [T] and Ys [NCOL][T]: the basis of the next tile is evaluated into
    // one while the warps contract the current tile from the other
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* accd = reinterpret_cast<double*>(smem_raw);
    V4* s_rad0 = reinterpret_cast<V4*>(smem_raw + ((NOUT * sizeof(double) + 15) / 16) * 16);
    R* Ys0 = reinterpret_cast<R*>(s_rad0 + T);
    V4* s_rad1 = reinterpret_cast<V4*>(Ys0 + (size_t)NCOL * T);
    R* Ys1 = reinterpret_cast<R*>(s_rad1 + T);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const V4* posm = reinterpret_cast<const V4*>(p.posm);
    for (int e = tid; e < NOUT; e += TH) accd[e] = 0.0;
    R acc[NR][kBinCap];
#pragma unroll
    for (int n = 0; n < NR; ++n)
#pragma unroll
        for (int c = 0; c < kBinCap; ++c) acc[n][c] = R(0);

    auto flush = [&]() {
        // butterfly sum over the warp's lanes, lane 0 adds to the FP64 block sums
#pragma unroll
        for (int n = 0; n < NR; ++n)
#pragma unroll
            for (int c = 0; c < kBinCap; ++c) {
                R v = acc[n][c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) accd[(warp * NR + n) * kBinCap + c] += (double)v;
                acc[n][c] = R(0);
            }
    };
    auto load = [&](int tile) -> V4 {
        const int64_t gi = (int64_t)tile * T + tid;
        return (tid < T && tile < p.ntiles && gi < p.N) ? ld4(posm + gi)
                                                      : mk4<R>(R(0), R(0), R(0), R(0));
    };
    // phase 1: one particle per thread (threads tid < T) -> angular basis +
    // radial seeds
    auto basis = [&](const V4& cur, V4* s_rad, R* Ys) {
        if (T < TH && tid >= T) return;
        R x = R(0), y = R(0), z = R(0), m = R(0);
        if (finite4(cur.x, cur.y, cur.z, cur.w)) { x = cur.x; y = cur.y; z = cur.z; m = cur.w; }
        else report(p.err, ETICS_ERR_NONFINITE);
        const R r = sqrt(x * x + y * y + z * z);
        const R t = R(1) / (R(1) + r);
        s_rad[tid] = mk4<R>(R(1) - R(2) * t, r * t * t, -m * t, R(0));
        const R inv = r > R(0) ? R(1) / r : R(0);
        const R ux = x * inv, uy = y * inv, uz = z * inv;
        const R uu = ux * ux + uy * uy + uz * uz;
        R C[3][LM + 1], S[3][LM + 1];
        angular_levels<R, 0, LM, false>(C, S, ux, uy, uz, uu, LM, Ys, T, tid);
    };

    V4 cur = load(blockIdx.x);
    if (blockIdx.x < p.ntiles) basis(cur, s_rad0, Ys0);
    cur = load(blockIdx.x + gridDim.x);
    __syncthreads();
    int since = 0, buf = 0;
    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x, buf ^= 1) {
        // basis of the next tile into the other buffer (its last reader, the
        // contraction of the previous tile, finished before the last barrier)
        const int nxt = tile + gridDim.x;
        if (nxt < p.ntiles) {
            basis(cur, buf ? s_rad0 : s_rad1, buf ? Ys0 : Ys1);
            cur = load(nxt + gridDim.x);
        }
        // phase 2: each warp accumulates its bin over this tile's particles
        bin_dispatch<R, NR, LM, 0>(warp, acc, buf ? Ys1 : Ys0, buf ? s_rad1 : s_rad0, T, lane);
        __syncthreads();
        if (++since == kBinFlushTiles) { flush(); since = 0; }
    }
    if (since) flush();
    __syncthreads();
    double* out = p.partial + (size_t)blockIdx.x * NOUT;
    for (int e = tid; e < NOUT; e += TH) out[e] = accd[e];
}

// sum block partials in a fixed order; one warp per output c[n][l*l+l+m]
template <int NR, int LM>
__global__ void scf_finalize_bins_kernel(const double* __restrict__ partial, int nblocks,
                                         double* __restrict__ coeffs) {
    constexpr int NJ = (LM + 1) * (LM + 1);
    constexpr int NOUT = BinConst<LM>::nbins * NR * kBinCap;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= NR * NJ) return;
    const int n = warp / NJ, jj = warp % NJ;
    int l = 0;
    while ((l + 1) * (l + 1) <= jj) ++l;
    const int m = jj - l * l - l;
    const int col = (m == 0) ? 0 : (m > 0 ? 2 * m - 1 : -2 * m);
    const int b = c_bin_index<LM>.bin[l * l + col];
    const int slot = c_bin_index<LM>.slot[l * l + col];
    const int idx = (b * NR + n) * kBinCap + slot;
    double s = 0.0;
    for (int k = lane; k < nblocks; k += 32) s += partial[(size_t)k * NOUT + idx];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int am = m < 0 ? -m : m;
        coeffs[warp] = s * c_tab.knorm_fact[l * (l + 1) / 2 + am] * c_tab.inv_j[n][l] *
                       geg_gamma(0, l, n);
    }
}

template <typename R, int NR, int LM, int MINB = 2>
inline size_t scf_bins_workspace(int num_sms) {
    return (size_t)MINB * num_sms * BinConst<LM>::nbins * NR * kBinCap * sizeof(double);
}

template <typename R, int NR, int LM, int TP = bins_threads<LM>(), int MINB = 2>
inline int scf_coeffs_bins_launch(const void* posm, int64_t N, double* coeffs, void* ws,
                                  const LaunchCtx& ctx) {
    constexpr int NB = BinConst<LM>::nbins;
    constexpr int TH = NB * 32;
    constexpr int T = TP;
    const int ntiles = (int)((N + T - 1) / T);
    int grid = ctx.num_sms * MINB;
    if (grid > ntiles) grid = ntiles > 0 ? ntiles : 1;
    ScfBinParams p{posm, N, ntiles, reinterpret_cast<double*>(ws), ctx.err};
    constexpr int NOUT = NB * NR * kBinCap;
    constexpr size_t smem = ((NOUT * sizeof(double) + 15) / 16) * 16 +
                            2 * (T * sizeof(Vec4<R>) + (size_t)(LM + 1) * (LM + 1) * T * sizeof(R));
    static_assert(smem <= 227 * 1024, "bins kernel shared memory");
    int nblocks = 0;
    if (ntiles > 0) {
        auto k = scf_coeff_bins_kernel<R, NR, LM, TP, MINB>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ||
            cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100))
            return ETICS_ERR_CUDA;
        k<<<grid, TH, smem, ctx.stream>>>(p);
        if (cudaGetLastError() != cudaSuccess) return ETICS_ERR_CUDA;
        ++*ctx.launches;
        nblocks = grid;
    }
    stage_event(ctx, 1);
    const int nc = NR * (LM + 1) * (LM + 1);
    scf_finalize_bins_kernel<NR, LM><<<(nc * 32 + 255) / 256, 256, 0, ctx.stream>>>(
        p.partial, nblocks, coeffs);
    if (cudaGetLastError() != cudaSuccess) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

}  // namespace etics
