// etics_scf_pairs.cuh -- SCF coefficient pass (paper Sec. 2.4 eq. 18, basis
// of Sec. 2.5, first pass of Sec. 3.3) specialised for a fixed (n_max, l_max)
// on the FP32 path, with the particle loop run two particles at a time on
// Blackwell's paired FP32 instructions.
//
//   c_nlm = (1/J_nl) sum_k m_k phi_nl(r_k) Y_lm(x_k)
//   phi_nl Y_lm = w_l(r) Ct_n(xi) H_l^m(u) * (gam_n knorm_lm / (l-m)!)
//   w_l = -m (1+r)^-1 (r/(1+r)^2)^l,  Ct_n the rescaled Gegenbauer polynomial,
//   H_l^m = (l-m)! Z_l^m (harm_level_exact); the bracket is applied in FP64
//   by the finalize.
//
// Work split (one block per SM, persistent over tiles of kPairTile particles):
//   * phase 1: thread k of the block evaluates particle k of the next tile:
//     xi and the harmonics of every column already scaled by w_l, into a
//     shared-memory buffer (two buffers: phase 1 of tile t+1 runs while the
//     contraction of tile t reads the other);
//   * phase 2: warp b owns one "bin" -- at most CAP columns of a single level
//     l -- and accumulates c[n][col] for n = 0..NR-1 over the tile; lane j
//     takes the particle pairs (2p, 2p+1), p = j, j+32, ...: one paired load
//     brings both particles' values of a column, the Gegenbauer recursion runs
//     on the pair (paired multiply + paired FMA per step) and each of the
//     NR x ncol updates is one paired FMA (__ffma2_rn): two particles per
//     instruction.  Accumulators are FP32 register pairs.
//   * every kPairFlushTiles tiles each warp reduces its own accumulators
//     (pair halves, then a butterfly over the lanes) and adds them to its FP64
//     block sums in shared memory; no block-wide synchronisation is needed
//     for that.  The per-block FP64 sums are added in a fixed order by the
//     finalize kernel: deterministic.
//
// Bins are sorted by cost (columns) so that the lightest warps are the ones
// that do no phase-1 work (threads beyond the tile).
#pragma once

#include <atomic>

#include "etics_scf_impl.cuh"

namespace etics {

constexpr int kPairTile = 512;        // particles per tile (one per phase-1 thread)
constexpr int kPairFlushTiles = 16;   // tiles between FP64 flushes

struct PairBin { int l, c0, nc; };

template <int LM, int CAP>
struct PairPlan {
    static constexpr int kCols = (LM + 1) * (LM + 1);
    int nbins;
    PairBin bin[kCols];
    int bin_of[kCols];    // dense column l*l + c -> bin
    int slot_of[kCols];   // -> column inside the bin
};

// each level's 2l+1 columns split as evenly as possible into
// ceil((2l+1)/CAP) bins; bins sorted by column count (descending), then by
// level (descending)
template <int LM, int CAP>
constexpr PairPlan<LM, CAP> make_pair_plan() {
    PairPlan<LM, CAP> p{};
    p.nbins = 0;
    for (int l = LM; l >= 0; --l) {
        const int nc = 2 * l + 1;
        const int nb = (nc + CAP - 1) / CAP;
        int c = 0;
        for (int b = 0; b < nb; ++b) {
            const int w = nc / nb + (b < nc % nb ? 1 : 0);
            p.bin[p.nbins++] = PairBin{l, c, w};
            c += w;
        }
    }
    for (int i = 1; i < p.nbins; ++i)
        for (int j = i; j > 0 && (p.bin[j].nc > p.bin[j - 1].nc ||
                                  (p.bin[j].nc == p.bin[j - 1].nc &&
                                   p.bin[j].l > p.bin[j - 1].l)); --j) {
            const PairBin t = p.bin[j];
            p.bin[j] = p.bin[j - 1];
            p.bin[j - 1] = t;
        }
    for (int b = 0; b < p.nbins; ++b)
        for (int c = 0; c < p.bin[b].nc; ++c) {
            const int col = p.bin[b].l * p.bin[b].l + p.bin[b].c0 + c;
            p.bin_of[col] = b;
            p.slot_of[col] = c;
        }
    return p;
}

template <int LM, int CAP>
struct PairConst {
    static constexpr PairPlan<LM, CAP> plan = make_pair_plan<LM, CAP>();
    static constexpr int nbins = plan.nbins;
    static constexpr int threads = nbins * 32;
};
template <int LM, int CAP>
static __constant__ PairPlan<LM, CAP> c_pair_plan = make_pair_plan<LM, CAP>();

struct ScfPairParams {
    const float4* posm;
    int64_t N;
    int64_t per;       // particles per block (even): block b takes [b*per, (b+1)*per)
    double* partial;   // [gridDim.x][nbins][NR][CAP]
    unsigned* err;
};

// phase 1 for one particle: xi, and w_l H_l^m of every column (dense layout
// l*l + c: c = 0 -> m = 0, 2m-1 -> cos, 2m -> sin), level by level
template <int L, int LM>
__device__ __forceinline__ void pair_angular(float (&C)[3][LM + 1], float (&S)[3][LM + 1],
                                             float ux, float uy, float uz, float w, float st,
                                             float* H, int k) {
    if constexpr (L <= LM) {
        constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
        harm_level_exact<float, L>(C[s1], S[s1], C[s2], S[s2], ux, uy, uz, C[s0], S[s0]);
        H[(L * L) * kPairTile + k] = w * C[s0][0];
#pragma unroll
        for (int m = 1; m <= L; ++m) {
            H[(L * L + 2 * m - 1) * kPairTile + k] = w * C[s0][m];
            H[(L * L + 2 * m) * kPairTile + k] = w * S[s0][m];
        }
        pair_angular<L + 1, LM>(C, S, ux, uy, uz, w * st, st, H, k);
    }
}

// recursion steps n = N..NR-1 of one particle pair: Ct_n = xi Ct_{n-1} -
// bs_n Ct_{n-2}, then acc[n][c] += Ct_n y_c; bs_n an immediate
template <int NR, int CAP, int NC, int L, int N>
__device__ __forceinline__ void pair_steps(float2 (&acc)[NR][CAP], const float2 (&y)[NC],
                                           float2 xi, float2 cm1, float2 cn) {
    if constexpr (N < NR) {
        constexpr float nb = -GegBsConst<0, L, N>::v;
        const float2 cnew = __ffma2_rn(make_float2(nb, nb), cm1, __fmul2_rn(xi, cn));
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[N][c] = __ffma2_rn(cnew, y[c], acc[N][c]);
        pair_steps<NR, CAP, NC, L, N + 1>(acc, y, xi, cn, cnew);
    }
}

// phase 2 for bin B over the first `np` particle pairs of one tile
template <int NR, int LM, int CAP, int B>
__device__ __forceinline__ void pair_bin_tile(float2 (&acc)[NR][CAP], const float* H,
                                              const float* xs, int lane, int np) {
    constexpr PairBin bd = PairConst<LM, CAP>::plan.bin[B];
    constexpr int NC = bd.nc;
    constexpr int col0 = bd.l * bd.l + bd.c0;
    const float2* H2 = reinterpret_cast<const float2*>(H);
    const float2* x2 = reinterpret_cast<const float2*>(xs);
#pragma unroll 1
    for (int p = lane; p < np; p += 32) {
        const float2 xi = x2[p];
        float2 y[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c] = H2[(col0 + c) * (kPairTile / 2) + p];
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[0][c] = __fadd2_rn(acc[0][c], y[c]);
        if constexpr (NR > 1) {
            // Ct_0 = 1, Ct_1 = xi; Ct_n = xi Ct_{n-1} - bs_n Ct_{n-2}
#pragma unroll
            for (int c = 0; c < NC; ++c) acc[1][c] = __ffma2_rn(xi, y[c], acc[1][c]);
            pair_steps<NR, CAP, NC, bd.l, 2>(acc, y, xi, make_float2(1.0f, 1.0f), xi);
        }
    }
}

template <int NR, int LM, int CAP, int B>
__device__ __forceinline__ void pair_dispatch(int warp, float2 (&acc)[NR][CAP], const float* H,
                                              const float* xs, int lane, int np) {
    if constexpr (B < PairConst<LM, CAP>::nbins) {
        if (warp == B) pair_bin_tile<NR, LM, CAP, B>(acc, H, xs, lane, np);
        else pair_dispatch<NR, LM, CAP, B + 1>(warp, acc, H, xs, lane, np);
    }
}

template <int NR, int LM, int CAP>
constexpr size_t pair_smem_bytes() {
    constexpr int NB = PairConst<LM, CAP>::nbins;
    return ((size_t)NB * NR * CAP * sizeof(double) + 15) / 16 * 16 +
           2 * ((size_t)(LM + 1) * (LM + 1) * kPairTile + kPairTile) * sizeof(float);
}

template <int NR, int LM, int CAP>
__global__ void __launch_bounds__(PairConst<LM, CAP>::threads, 1)
scf_coeff_pairs_kernel(ScfPairParams p) {
    constexpr int NB = PairConst<LM, CAP>::nbins;
    constexpr int TH = NB * 32;
    constexpr int NCOL = (LM + 1) * (LM + 1);
    constexpr int NOUT = NB * NR * CAP;
    static_assert(TH >= kPairTile, "one phase-1 thread per tile particle");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double* accd = reinterpret_cast<double*>(smem_raw);
    float* buf0 = reinterpret_cast<float*>(smem_raw + ((size_t)NOUT * sizeof(double) + 15) / 16 * 16);
    // buffer b: NCOL x kPairTile scaled harmonics, then kPairTile values of xi
    constexpr size_t kBuf = (size_t)NCOL * kPairTile + kPairTile;
    auto Hb = [&](int b) { return buf0 + b * kBuf; };
    auto Xb = [&](int b) { return buf0 + b * kBuf + (size_t)NCOL * kPairTile; };
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int e = tid; e < NOUT; e += TH) accd[e] = 0.0;
    pdl_wait();   // the particles may come from the previous kernel (a drift)

    float2 acc[NR][CAP];
#pragma unroll
    for (int n = 0; n < NR; ++n)
#pragma unroll
        for (int c = 0; c < CAP; ++c) acc[n][c] = make_float2(0.0f, 0.0f);

    // Flush: every warp total of the NR x CAP accumulators (pair halves
    // added, then a butterfly over the lanes) is kept by lane (index % 32),
    // so that the FP64 additions into the block sums run as a few warp-wide
    // instructions instead of one instruction per value (FP64 issue is slow
    // on this GPU).  Columns beyond the bin's width hold zeros.
    constexpr int kPerWarp = NR * CAP;
    constexpr int kRounds = (kPerWarp + 31) / 32;
    auto flush = [&]() {
        float mine[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; ++r) mine[r] = 0.0f;
#pragma unroll
        for (int n = 0; n < NR; ++n)
#pragma unroll
            for (int c = 0; c < CAP; ++c) {
                float v = acc[n][c].x + acc[n][c].y;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                const int idx = n * CAP + c;
                if (lane == (idx & 31)) mine[idx >> 5] = v;
                acc[n][c] = make_float2(0.0f, 0.0f);
            }
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int idx = r * 32 + lane;
            if (idx < kPerWarp) accd[warp * kPerWarp + idx] += (double)mine[r];
        }
    };
    // this block's particles: one contiguous range, so that every block has
    // the same work up to one particle pair (the last tile may be partial;
    // its phase 2 runs over the pairs it holds)
    const int64_t lo = (int64_t)blockIdx.x * p.per;
    const int64_t hi = lo + p.per < p.N ? lo + p.per : p.N;
    const int ntb = hi > lo ? (int)((hi - lo + kPairTile - 1) / kPairTile) : 0;
    auto load = [&](int t) -> float4 {
        const int64_t gi = lo + (int64_t)t * kPairTile + tid;
        return (tid < kPairTile && t < ntb && gi < hi) ? p.posm[gi]
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    auto pairs_in = [&](int t) {
        const int64_t left = hi - lo - (int64_t)t * kPairTile;
        return (int)(((left < kPairTile ? left : kPairTile) + 1) / 2);
    };
    auto phase1 = [&](const float4& v, float* Hs, float* Xs) {
        if (tid >= kPairTile) return;
        float x = 0.f, y = 0.f, z = 0.f, m = 0.f;
        if (finite4(v.x, v.y, v.z, v.w)) { x = v.x; y = v.y; z = v.z; m = v.w; }
        else report(p.err, ETICS_ERR_NONFINITE);
        const float r = sqrtf(x * x + y * y + z * z);
        const float t = 1.0f / (1.0f + r);
        Xs[tid] = 1.0f - 2.0f * t;
        const float inv = r > 0.0f ? 1.0f / r : 0.0f;
        float C[3][LM + 1], S[3][LM + 1];
        pair_angular<0, LM>(C, S, x * inv, y * inv, z * inv, -m * t, r * t * t, Hs, tid);
    };

    float4 cur = load(0);
    if (ntb > 0) phase1(cur, Hb(0), Xb(0));
    cur = load(1);
    __syncthreads();
    int since = 0, b = 0;
    for (int t = 0; t < ntb; ++t, b ^= 1) {
        if (t + 1 < ntb) {
            phase1(cur, Hb(b ^ 1), Xb(b ^ 1));
            cur = load(t + 2);
        }
        pair_dispatch<NR, LM, CAP, 0>(warp, acc, Hb(b), Xb(b), lane, pairs_in(t));
        if (++since == kPairFlushTiles) { flush(); since = 0; }
        __syncthreads();
    }
    if (since) flush();
    __syncthreads();
    double* out = p.partial + (size_t)blockIdx.x * NOUT;
    for (int e = tid; e < NOUT; e += TH) out[e] = accd[e];
}

// Block sums added in block order; one warp per output c[n][l*l+l+m], four
// warps per block so that the FP64 additions (slow on this GPU) are spread
// over as many SMs as there are blocks.
constexpr int kFinThreads = 128;
template <int NR, int LM, int CAP>
__global__ void __launch_bounds__(kFinThreads)
scf_finalize_pairs_kernel(const double* __restrict__ partial, int nblocks,
                          double* __restrict__ coeffs) {
    constexpr int NJ = (LM + 1) * (LM + 1);
    constexpr int NOUT = PairConst<LM, CAP>::nbins * NR * CAP;
    pdl_wait();   // the partials come from the coefficient kernel
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= NR * NJ) return;
    const int n = warp / NJ, jj = warp % NJ;
    int l = 0;
    while ((l + 1) * (l + 1) <= jj) ++l;
    const int m = jj - l * l - l;
    const int col = l * l + ((m == 0) ? 0 : (m > 0 ? 2 * m - 1 : -2 * m));
    const int idx = (c_pair_plan<LM, CAP>.bin_of[col] * NR + n) * CAP +
                    c_pair_plan<LM, CAP>.slot_of[col];
    double s = 0.0;
#pragma unroll 4
    for (int k = lane; k < nblocks; k += 32) s += __ldcg(partial + (size_t)k * NOUT + idx);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int am = m < 0 ? -m : m;
        coeffs[warp] = s * c_tab.knorm_fact[l * (l + 1) / 2 + am] * c_tab.inv_j[n][l] *
                       geg_gamma(0, l, n);
    }
}

template <int NR, int LM, int CAP>
inline size_t scf_pairs_workspace(int num_sms) {
    return (size_t)num_sms * PairConst<LM, CAP>::nbins * NR * CAP * sizeof(double);
}

template <int NR, int LM, int CAP>
inline int scf_coeffs_pairs_launch(const void* posm, int64_t N, double* coeffs, void* ws,
                                   const LaunchCtx& ctx) {
    constexpr int TH = PairConst<LM, CAP>::threads;
    constexpr size_t smem = pair_smem_bytes<NR, LM, CAP>();
    static_assert(smem <= 227 * 1024, "pairs kernel shared memory");
    const int ntiles = (int)((N + kPairTile - 1) / kPairTile);
    int grid = ctx.num_sms;
    if (grid > ntiles) grid = ntiles > 0 ? ntiles : 1;
    // contiguous, equal ranges (an even number of particles each): at
    // N = 2^20 each of the 152 blocks takes 6900 particles (13 full tiles and
    // one of 244) instead of 13 or 14 full tiles
    int64_t per = (N + grid - 1) / grid;
    per += per & 1;
    ScfPairParams p{reinterpret_cast<const float4*>(posm), N, per,
                    reinterpret_cast<double*>(ws), ctx.err};
    int nblocks = 0;
    if (ntiles > 0) {
        auto k = scf_coeff_pairs_kernel<NR, LM, CAP>;
        // the function attributes are set once per device (a host call per
        // launch would sit between the caller's events and the kernel)
        static std::atomic<uint64_t> attr_done{0};
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return ETICS_ERR_CUDA;
        const uint64_t bit = uint64_t(1) << (dev & 63);
        if (!(attr_done.load() & bit)) {
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ||
                cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100))
                return ETICS_ERR_CUDA;
            attr_done.fetch_or(bit);
        }
        if (launch_pdl(k, dim3(grid), dim3(TH), smem, ctx.stream, p)) return ETICS_ERR_CUDA;
        ++*ctx.launches;
        nblocks = grid;
    }
    stage_event(ctx, 1);
    const int nc = NR * (LM + 1) * (LM + 1);
    if (launch_pdl(scf_finalize_pairs_kernel<NR, LM, CAP>,
                   dim3((nc * 32 + kFinThreads - 1) / kFinThreads), dim3(kFinThreads), 0,
                   ctx.stream, (const double*)p.partial, nblocks, coeffs))
        return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

}  // namespace etics
