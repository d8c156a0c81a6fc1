// etics_batch.cu -- SCF for a batch of independent systems of uneven size and
// expansion order in one pass (the paper notes the GPU is under-loaded at
// small N, Sec. 3.4; batching many systems fills it).
//
// A host-built plan lists, for every system (instance), its particle range,
// (n_max, l_max), its slice of the packed coefficient output and its tiles.
// Three kernels then cover the whole batch:
//   1. coefficients: persistent blocks walk contiguous ranges of the
//      instance-major tile list; a block flushes its FP64 sums into one
//      "segment" slot each time the instance changes (segments of one
//      instance are contiguous, so the finalize sums them in a fixed order).
//      Mixed precision: particle pairs on paired FP32 instructions, every lane
//      of the block owning one "bin" (one level, up to three columns) of the
//      instance's expansion (batch_pairs_kernel).  FP64: register tiles of
//      four columns over a shared-memory radial basis (batch_coeff_kernel);
//   2. finalize: one warp per output coefficient of any instance;
//   3. field: one block per work item (a chunk of one instance's particles),
//      the instance's coefficients staged in shared memory.
// No grid-wide barrier is needed, so the three launches capture into a CUDA
// graph as three nodes.  Tile size, blocks per SM and field chunking are
// tuning parameters (etics_batch_tuning) chosen by the autotuner.
#include <algorithm>
#include <cstring>
#include <vector>

#include "etics_batch_layout.h"
#include "etics_scf_impl.cuh"

namespace etics {

constexpr int kBatchThreads = 256;

constexpr int kBatchMagic = 0x45544232;   // "ETB2"
constexpr size_t kMaxDynSmem = 227 * 1024;  // opt-in shared memory per block on sm_103a

struct BatchHeader {
    int magic, precision;
    int ninst, nblocks, nseg, nfield;
    int T, blocks_per_sm, field_threads, field_chunk;
    int ntiles;
    int64_t ntot, coef_total;
    int64_t seg_stride;            // doubles per segment slot
    size_t smem_coef;              // dynamic shared memory of the coefficient kernel
    size_t ws_bytes;               // workspace: nseg * seg_stride doubles
    // byte offsets of the tables inside the plan
    int64_t off_inst, off_block, off_seg, off_field, off_tile, off_layout, off_chunk;
    int64_t total_bytes;
    // mixed precision: floats of the basis/staging region, chunks, and the
    // byte offset of the chunk counter in the workspace
    int64_t bp_hfloats;
    int nchunks, pad;
    int64_t counter_off;
};
struct BatchInst {
    int64_t offset, n, coef_offset;
    int n_max, l_max, first_tile, ntiles, first_seg, nseg;
};
struct BatchBlock { int tile_begin, tile_end, first_seg, pad; };
struct BatchField { int64_t begin; int count, inst; };
struct BatchChunk { int inst, tile_begin, tile_end, pad; };

template <typename T>
__host__ __device__ inline const T* plan_table(const void* plan, int64_t off) {
    return reinterpret_cast<const T*>(static_cast<const unsigned char*>(plan) + off);
}

// ---------------------------------------------------------------------------
// 1. coefficients
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kBatchThreads)
batch_coeff_kernel(const Vec4<R>* __restrict__ posm, const void* __restrict__ plan,
                   double* __restrict__ partial, unsigned* err) {
    constexpr int TH = kBatchThreads, NR = kBatchNR, LMU = kBatchLM;
    using V4 = Vec4<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const BatchHeader hd = *plan_table<BatchHeader>(plan, 0);
    const BatchInst* insts = plan_table<BatchInst>(plan, hd.off_inst);
    const BatchBlock* blocks = plan_table<BatchBlock>(plan, hd.off_block);
    const int* tile_inst = plan_table<int>(plan, hd.off_tile);
    const int T = hd.T, TC = T / 4;
    const int tid = threadIdx.x;
    // shared layout sized for the largest expansion (l_max = LMU, NR rows); the
    // reduction scratch (at most TH * NR * 4 values) overlays the basis tiles,
    // the FP64 sums follow both
    const size_t main_max = (size_t)(LMU + 1) * NR * T + (size_t)col_total(LMU) * T;
    const size_t red_max = (size_t)TH * NR * 4;
    const size_t union_max = main_max > red_max ? main_max : red_max;
    R* Rs = reinterpret_cast<R*>(smem_raw);
    double* accd = reinterpret_cast<double*>(smem_raw + ((union_max * sizeof(R) + 15) / 16) * 16);
    R acc[NR][4];

    for (int bi = blockIdx.x; bi < hd.nblocks; bi += gridDim.x) {
        const BatchBlock blk = blocks[bi];
        int seg = blk.first_seg;
        int cur = -1;
        int n_max = 0, l_max = 0, W = 1, G = 1, il = 0, col0 = 0, l_split = 0;
        bool active = false;
        size_t union_elems = 0;
        int nout = 0;
        R* Ys = Rs;
        // add the register tiles of the G particle groups to the FP64 sums; the
        // reduction scratch overlays the basis tiles, which are cleared again
        auto flush_acc = [&]() {
            __syncthreads();
            R* red = Rs;
            const int item = tid / G, g = tid % G;
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
                for (int gg = 0; gg < G; ++gg) s += red[(size_t)gg * nout + o];
                accd[o] += (double)s;
            }
            __syncthreads();
            for (size_t e = tid; e < union_elems; e += TH) Rs[e] = R(0);
            __syncthreads();
        };
        // store the instance's sums into this block's segment slot
        auto emit = [&]() {
            flush_acc();
            double* out = partial + (size_t)seg * hd.seg_stride;
            for (int o = tid; o < nout; o += TH) out[o] = accd[o];
            __syncthreads();
        };
        int since = 0;
        for (int tile = blk.tile_begin; tile < blk.tile_end; ++tile) {
            const int inst = tile_inst[tile];
            if (inst != cur) {
                if (cur >= 0) { emit(); ++seg; }
                cur = inst;
                since = 0;
                const BatchInst in = insts[inst];
                n_max = in.n_max;
                l_max = in.l_max;
                W = scf_items(l_max);
                G = TH / W;
                if (G > TC) G = TC;
                if (G < 1) G = 1;
                nout = W * NR * 4;
                const size_t main_elems = (size_t)(l_max + 1) * NR * T + (size_t)col_total(l_max) * T;
                const size_t red_elems = (size_t)W * G * NR * 4;
                union_elems = main_elems > red_elems ? main_elems : red_elems;
                Ys = Rs + (size_t)(l_max + 1) * NR * T;
                const int item = tid / G;
                active = item < W;
                il = 0;
                col0 = 0;
                if (active) {
                    int it = item;
                    for (int l = 0; l <= l_max; ++l) {
                        const int nch = ncol_pad(l) / 4;
                        if (it < nch) { il = l; col0 = col_offset(l) + 4 * it; break; }
                        it -= nch;
                    }
                }
                {   // balance the two halves of phase 1 (same rule as the single-system kernel)
                    const double rad = n_max + 1.0, ang = 0.8 * (l_max + 1.0) * (l_max + 1.0);
                    double best_cost = 1e30;
                    l_split = l_max + 1;
                    for (int ls = 0; ls <= l_max + 1; ++ls) {
                        const double a = rad * ls, b = ang + rad * (l_max + 1 - ls);
                        const double c = a > b ? a : b;
                        if (c < best_cost) { best_cost = c; l_split = ls; }
                    }
                }
#pragma unroll
                for (int n = 0; n < NR; ++n)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[n][j] = R(0);
                __syncthreads();
                for (size_t e = tid; e < union_elems; e += TH) Rs[e] = R(0);
                for (int e = tid; e < nout; e += TH) accd[e] = 0.0;
                __syncthreads();
            }
            const BatchInst in = insts[inst];
            const int lt = tile - in.first_tile;
            // ---- phase 1 -------------------------------------------------
            if (tid < 2 * T) {
                const int k = tid < T ? tid : tid - T;
                const int64_t li = (int64_t)lt * T + k;
                R x = R(0), y = R(0), z = R(0), m = R(0);
                if (li < in.n) {
                    const V4 v = ld4(posm + in.offset + li);
                    if (finite4(v.x, v.y, v.z, v.w)) { x = v.x; y = v.y; z = v.z; m = v.w; }
                    else if (tid < T) report(err, ETICS_ERR_NONFINITE);
                }
                const R r = sqrt(x * x + y * y + z * z);
                const R t = R(1) / (R(1) + r);
                const R st = r * t * t;
                const R xi = R(1) - R(2) * t;
                if (tid < T) {
                    radial_levels<R, NR, 0, LMU>(Rs, T, k, n_max, 0, l_split - 1, -m * t, st, xi);
                } else {
                    const R inv = r > R(0) ? R(1) / r : R(0);
                    const R ux = x * inv, uy = y * inv, uz = z * inv;
                    const R uu = ux * ux + uy * uy + uz * uz;
                    R C[3][LMU + 1], S[3][LMU + 1];
                    angular_levels<R, 0, LMU>(C, S, ux, uy, uz, uu, l_max, Ys, T, k);
                    radial_levels<R, NR, 0, LMU>(Rs, T, k, n_max, l_split, l_max, -m * t, st, xi);
                }
            }
            __syncthreads();
            // ---- phase 2 -------------------------------------------------
            if (active) {
                const int g = tid % G;
                const V4* Rv4 = reinterpret_cast<const V4*>(Rs + (size_t)il * NR * T);
                const V4* Yv4 = reinterpret_cast<const V4*>(Ys + (size_t)col0 * T);
                for (int c = g; c < TC; c += G) {
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
            if (++since == kFlushTiles) { flush_acc(); since = 0; }
        }
        if (cur >= 0) emit();
    }
}

// ---------------------------------------------------------------------------
// 1b. coefficients, mixed precision: particle pairs, one bin per lane
// ---------------------------------------------------------------------------
// phase 1 for one particle: w_l H_l^m of every column of levels 0..l_max
// (dense column l*l + c) into H[col * T + k]; w_l = -m (1+r)^-1 (r/(1+r)^2)^l
template <int L>
__device__ __forceinline__ void bp_angular(float (&C)[3][kBatchLM + 1], float (&S)[3][kBatchLM + 1],
                                           float ux, float uy, float uz, float w, float st,
                                           float* H, int T, int k, int l_max) {
    if constexpr (L <= kBatchLM) {
        if (L > l_max) return;
        constexpr int s0 = L % 3, s1 = (L + 2) % 3, s2 = (L + 1) % 3;
        harm_level_exact<float, L>(C[s1], S[s1], C[s2], S[s2], ux, uy, uz, C[s0], S[s0]);
        H[(size_t)(L * L) * T + k] = w * C[s0][0];
#pragma unroll
        for (int m = 1; m <= L; ++m) {
            H[(size_t)(L * L + 2 * m - 1) * T + k] = w * C[s0][m];
            H[(size_t)(L * L + 2 * m) * T + k] = w * S[s0][m];
        }
        bp_angular<L + 1>(C, S, ux, uy, uz, w * st, st, H, T, k, l_max);
    }
}

// phase 2 for one lane: its bin's kBpCap columns (float2 offsets o0..o2 into
// H2) over the particle pairs p = p0, p0 + step, ... < np; the rescaled
// Gegenbauer recursion Ct_n = xi Ct_{n-1} - bs_n Ct_{n-2} (Ct_0 = 1,
// Ct_1 = xi) runs on the pair for the NRR = n_max + 1 rows; nbl[n] = -bs_n of
// the bin's level, held in registers for the tile
template <int NRR>
__device__ __forceinline__ void bp_rows(float2 (&acc)[kBatchNR][kBpCap], const float2* H2,
                                        const float2* X2, const float* nbl, int o0, int o1, int o2,
                                        int p0, int np, int step) {
    float nb[NRR];
#pragma unroll
    for (int n = 2; n < NRR; ++n) nb[n] = nbl[n];
#pragma unroll 1
    for (int p = p0; p < np; p += step) {
        const float2 xi = X2[p];
        const float2 y[kBpCap] = {H2[o0 + p], H2[o1 + p], H2[o2 + p]};
#pragma unroll
        for (int c = 0; c < kBpCap; ++c) acc[0][c] = __fadd2_rn(acc[0][c], y[c]);
        if constexpr (NRR > 1) {
#pragma unroll
            for (int c = 0; c < kBpCap; ++c) acc[1][c] = __ffma2_rn(xi, y[c], acc[1][c]);
        }
        float2 cm1 = make_float2(1.0f, 1.0f), cn = xi;
#pragma unroll
        for (int n = 2; n < NRR; ++n) {
            const float2 cnew = __ffma2_rn(make_float2(nb[n], nb[n]), cm1, __fmul2_rn(xi, cn));
#pragma unroll
            for (int c = 0; c < kBpCap; ++c) acc[n][c] = __ffma2_rn(cnew, y[c], acc[n][c]);
            cm1 = cn;
            cn = cnew;
        }
    }
}

// bp_rows for the instance's row count (a uniform chain of compares)
template <int NRR>
__device__ __forceinline__ void bp_rows_n(int nrr, float2 (&acc)[kBatchNR][kBpCap], const float2* H2,
                                          const float2* X2, const float* nbl, int o0, int o1, int o2,
                                          int p0, int np, int step) {
    if constexpr (NRR <= kBatchNR) {
        if (nrr == NRR) bp_rows<NRR>(acc, H2, X2, nbl, o0, o1, o2, p0, np, step);
        else bp_rows_n<NRR + 1>(nrr, acc, H2, X2, nbl, o0, o1, o2, p0, np, step);
    }
}

// 16-byte asynchronous global -> shared copies (the next tile's particles)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Blocks claim chunks (at most kBpChunkTiles tiles of one instance, heaviest
// instances first) from a counter in the workspace; chunk c writes its FP64
// sums c[n][l*l + col] into segment slot c, so the result does not depend on
// which block ran which chunk.  The counter is zeroed before every launch.
__global__ void __launch_bounds__(kBpThreads, 1)
batch_pairs_kernel(const float4* __restrict__ posm, const void* __restrict__ plan,
                   double* __restrict__ partial, unsigned* counter, unsigned* err) {
    constexpr int NR = kBatchNR, CAP = kBpCap;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_claim[2];
    const BatchHeader hd = *plan_table<BatchHeader>(plan, 0);
    const BatchInst* insts = plan_table<BatchInst>(plan, hd.off_inst);
    const BatchChunk* chunks = plan_table<BatchChunk>(plan, hd.off_chunk);
    const BatchLayout* layouts = plan_table<BatchLayout>(plan, hd.off_layout);
    const int T = hd.T, TP = T / 2;
    // recursion constants, the basis region (w_l H of the tile; the emit
    // stages the lanes' sums there), xi, and the prefetched particles
    float* snb = reinterpret_cast<float*>(smem_raw);
    float* H = reinterpret_cast<float*>(smem_raw + kBpNbBytes);
    float* X = H + hd.bp_hfloats;
    float4* P = reinterpret_cast<float4*>(X + T);   // the next tile's particles, one per thread
    const float2* H2 = reinterpret_cast<const float2*>(H);
    const float2* X2 = reinterpret_cast<const float2*>(X);
    const int tid = threadIdx.x;
    for (int e = tid; e < (kBatchLM + 1) * kBpNbStride; e += kBpThreads) {
        const int l = e / kBpNbStride, n = e % kBpNbStride;
        snb[e] = n < NR ? -c_tab.gbs_f[0][l][n] : 0.0f;
    }
    float2 acc[NR][CAP];
#pragma unroll
    for (int n = 0; n < NR; ++n)
#pragma unroll
        for (int c = 0; c < CAP; ++c) acc[n][c] = make_float2(0.0f, 0.0f);

    auto prefetch = [&](int tl, const BatchInst& inr) {
        const int64_t li = (int64_t)(tl - inr.first_tile) * T + tid;
        if (li < inr.n) cp_async16(P + tid, posm + inr.offset + li);
        cp_async_commit();
    };
    if (tid == 0) s_claim[0] = (int)atomicAdd(counter, 1u);
    __syncthreads();
    int cur = s_claim[0], slot = 0;
    bool first = true;
    while (cur < hd.nchunks) {
        // claim the next chunk now, so that the last tile of this one can
        // prefetch its first particles
        if (tid == 0) s_claim[slot ^ 1] = (int)atomicAdd(counter, 1u);
        __syncthreads();
        const int nxt = s_claim[slot ^ 1];
        const BatchChunk ch = chunks[cur];
        const BatchInst in = insts[ch.inst];
        const int n_max = in.n_max;
        const BatchLayout* lay = layouts + in.l_max;
        int o0, o1, o2, rank, nlanes;
        const float* nbl;
        {
            const BatchLane ln = lay->lane[tid];
            o0 = ln.col[0] * TP;
            o1 = ln.col[1] * TP;
            o2 = ln.col[2] * TP;
            rank = ln.rank;
            nlanes = ln.nlanes;
            nbl = snb + ln.level * kBpNbStride;
        }
        for (int tile = ch.tile_begin; tile < ch.tile_end; ++tile) {
            // ---- phase 1: one particle per thread --------------------------
            // each thread's particle arrives by an asynchronous copy into its
            // own slot of P, issued during the previous tile
            if (tid < T) {
                if (first) { prefetch(tile, in); first = false; }
                cp_async_wait_all();
                const int64_t li = (int64_t)(tile - in.first_tile) * T + tid;
                float x = 0.f, y = 0.f, z = 0.f, m = 0.f;
                if (li < in.n) {
                    const float4 v = P[tid];
                    if (finite4(v.x, v.y, v.z, v.w)) { x = v.x; y = v.y; z = v.z; m = v.w; }
                    else report(err, ETICS_ERR_NONFINITE);
                }
                const float r = sqrtf(x * x + y * y + z * z);
                // the slot is free once r has consumed its value
                if (tile + 1 < ch.tile_end) prefetch(tile + 1, in);
                else if (nxt < hd.nchunks) {
                    const BatchChunk cn = chunks[nxt];
                    prefetch(cn.tile_begin, insts[cn.inst]);
                }
                const float t = 1.0f / (1.0f + r);
                X[tid] = 1.0f - 2.0f * t;
                const float inv = r > 0.0f ? 1.0f / r : 0.0f;
                float C[3][kBatchLM + 1], S[3][kBatchLM + 1];
                bp_angular<0>(C, S, x * inv, y * inv, z * inv, -m * t, r * t * t, H, T, tid,
                              in.l_max);
            }
            __syncthreads();
            // ---- phase 2: this lane's bin over its particle pairs ----------
            bp_rows_n<1>(n_max + 1, acc, H2, X2, nbl, o0, o1, o2, rank, TP, nlanes);
            __syncthreads();
        }
        // ---- emit: the lanes' FP32 sums (pair halves added) are staged in the
        // basis region, then each output adds its bin's lanes in lane order
        {
            float* red = H;
#pragma unroll
            for (int n = 0; n < NR; ++n)
#pragma unroll
                for (int c = 0; c < CAP; ++c) {
                    red[(n * CAP + c) * kBpThreads + tid] = acc[n][c].x + acc[n][c].y;
                    acc[n][c] = make_float2(0.0f, 0.0f);
                }
            __syncthreads();
            double* out = partial + (size_t)cur * hd.seg_stride;
            const int nb = lay->nbins;
            for (int o = tid; o < nb * NR * CAP; o += kBpThreads) {
                const int b = o % nb, q = o / nb, n = q / CAP, c = q % CAP;
                const BatchBin bn = lay->bin[b];
                if (c < bn.nc && n <= n_max) {
                    const float* src = red + (n * CAP + c) * kBpThreads + bn.lane0;
                    float s0 = 0.0f, s1 = 0.0f;
                    int k = 0;
                    for (; k + 1 < bn.nlanes; k += 2) { s0 += src[k]; s1 += src[k + 1]; }
                    if (k < bn.nlanes) s0 += src[k];
                    out[n * kBpCols + bn.col0 + c] = (double)s0 + (double)s1;
                }
            }
            __syncthreads();
        }
        cur = nxt;
        slot ^= 1;
    }
}

// ---------------------------------------------------------------------------
// 2. finalize: ordered sum of an instance's segments, times K_lm / J_nl
// ---------------------------------------------------------------------------
__global__ void batch_finalize_kernel(const void* __restrict__ plan,
                                      const double* __restrict__ partial,
                                      double* __restrict__ coeffs) {
    const BatchHeader hd = *plan_table<BatchHeader>(plan, 0);
    const BatchInst* insts = plan_table<BatchInst>(plan, hd.off_inst);
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= hd.coef_total) return;
    int lo = 0, hi = hd.ninst - 1;          // instance holding output `warp`
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (insts[mid].coef_offset <= warp) lo = mid; else hi = mid - 1;
    }
    const BatchInst in = insts[lo];
    const int nj = (in.l_max + 1) * (in.l_max + 1);
    const int local = (int)(warp - in.coef_offset);
    const int n = local / nj, jj = local % nj;
    int l = 0;
    while ((l + 1) * (l + 1) <= jj) ++l;
    const int m = jj - l * l - l;
    const int col = (m == 0) ? 0 : (m > 0 ? 2 * m - 1 : -2 * m);
    // mixed plans keep dense sums c[n][l*l + col]; FP64 plans four-column items
    const int idx = hd.precision == ETICS_MIXED
                        ? n * kBpCols + l * l + col
                        : ((col_offset(l) / 4 + col / 4) * kBatchNR + n) * 4 + (col & 3);
    double s = 0.0;
    for (int k = lane; k < in.nseg; k += 32) s += partial[(size_t)(in.first_seg + k) * hd.seg_stride + idx];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int am = m < 0 ? -m : m;
        coeffs[warp] = s * c_tab.knorm_fact[l * (l + 1) / 2 + am] * c_tab.inv_j[n][l] *
                       geg_gamma(0, l, n);
    }
}

// ---------------------------------------------------------------------------
// 3. field: one work item (a chunk of one instance) per block iteration
// ---------------------------------------------------------------------------
template <typename R, bool ACC>
__global__ void __launch_bounds__(256)
batch_field_kernel(const Vec4<R>* __restrict__ posm, const void* __restrict__ plan,
                   const double* __restrict__ coeffs, Vec4<R>* __restrict__ out, int out_mask,
                 unsigned* err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* cs = reinterpret_cast<R*>(smem_raw);
    const BatchHeader hd = *plan_table<BatchHeader>(plan, 0);
    const BatchInst* insts = plan_table<BatchInst>(plan, hd.off_inst);
    const BatchField* items = plan_table<BatchField>(plan, hd.off_field);
    for (int w = blockIdx.x; w < hd.nfield; w += gridDim.x) {
        const BatchField it = items[w];
        const BatchInst in = insts[it.inst];
        const int ncols = col_total(in.l_max);
        const int nj = (in.l_max + 1) * (in.l_max + 1);
        __syncthreads();
        for (int e = threadIdx.x; e < (in.n_max + 1) * ncols; e += blockDim.x) {
            const int n = e / ncols;
            int c = e % ncols, l = 0;
            while (c >= ncol_pad(l)) { c -= ncol_pad(l); ++l; }
            R v = R(0);
            if (c < 2 * l + 1) {
                const int m = (c == 0) ? 0 : ((c & 1) ? (c + 1) / 2 : -(c / 2));
                const int am = m < 0 ? -m : m;
                v = (R)(coeffs[in.coef_offset + (int64_t)n * nj + l * l + l + m] *
                        c_tab.knorm[l * (l + 1) / 2 + am] * geg_gamma(0, l, n));
            }
            cs[e] = v;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < it.count; k += blockDim.x) {
            const int64_t i = in.offset + it.begin + k;
            const Vec4<R> pv = ld4(posm + i);
            if (!finite4(pv.x, pv.y, pv.z, pv.w)) report(err, ETICS_ERR_NONFINITE);
            FieldEval<R, kBatchLM, ACC, 0> f;
            const R r = sqrt(pv.x * pv.x + pv.y * pv.y + pv.z * pv.z);
            const R inv = r > R(0) ? R(1) / r : R(0);
            f.ux = pv.x * inv; f.uy = pv.y * inv; f.uz = pv.z * inv;
            f.uu = f.ux * f.ux + f.uy * f.uy + f.uz * f.uz;
            f.t = R(1) / (R(1) + r);
            f.st = r * f.t * f.t;
            f.xi = R(1) - R(2) * f.t;
            f.dxdr = R(2) * f.t * f.t;
            f.pre = -f.t;
            f.preR = -f.t * f.t * f.t;
            f.pot = f.gr = f.gx = f.gy = f.gz = R(0);
            f.cs = cs;
            f.ncols = ncols;
            f.n_max = in.n_max;
            f.l_max = in.l_max;
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
}

// ---------------------------------------------------------------------------
// host: plan construction and launch
// ---------------------------------------------------------------------------
static size_t align16(size_t x) { return (x + 15) / 16 * 16; }

int batch_plan_build(const etics_batch_item* items, int ninst, const etics_batch_tuning* tuning,
                     int num_sms, int precision, void* plan, size_t plan_bytes, size_t* need,
                     size_t* ws_bytes, int64_t* coef_total) {
    if (ninst <= 0 || !items) return ETICS_ERR_ARG;
    etics_batch_tuning tn{};
    tn.tile = precision == ETICS_FP64 ? 32 : 64;
    tn.blocks_per_sm = 2;
    tn.field_threads = 256;
    tn.field_chunk = 2048;
    if (tuning) {
        if (tuning->tile > 0) tn.tile = tuning->tile;
        if (tuning->blocks_per_sm > 0) tn.blocks_per_sm = tuning->blocks_per_sm;
        if (tuning->field_threads > 0) tn.field_threads = tuning->field_threads;
        if (tuning->field_chunk > 0) tn.field_chunk = tuning->field_chunk;
    }
    if (precision == ETICS_MIXED) {
        // particle pairs: tiles of a multiple of 64 particles, at most one per
        // thread (the tile size is rounded up)
        if (!(tuning && tuning->tile > 0)) tn.tile = kBpMaxTile;
        if (tn.tile < 8 || tn.tile > kBpMaxTile) return ETICS_ERR_ARG;
        tn.tile = (tn.tile + 63) / 64 * 64;
    } else if (tn.tile % 4 || tn.tile < 8 || tn.tile > kBatchThreads / 2) {
        return ETICS_ERR_ARG;
    }
    if (tn.field_threads % 32 || tn.field_threads < 32 || tn.field_threads > 256) return ETICS_ERR_ARG;
    if (tn.blocks_per_sm < 1 || tn.blocks_per_sm > 8 || tn.field_chunk < 1) return ETICS_ERR_ARG;
    int64_t ntot = 0, ctot = 0, ntiles = 0, nfield = 0, nchunks = 0;
    int lmax_all = 0;
    for (int i = 0; i < ninst; ++i) {
        const etics_batch_item& it = items[i];
        if (it.n < 0 || it.n_max < 0 || it.l_max < 0) return ETICS_ERR_ARG;
        if (it.n_max > kBatchNR - 1 || it.l_max > kBatchLM) return ETICS_ERR_UNSUPPORTED;
        if (it.l_max > lmax_all) lmax_all = it.l_max;
        ntot += it.n;
        ctot += (int64_t)(it.n_max + 1) * (it.l_max + 1) * (it.l_max + 1);
        const int64_t nt = (it.n + tn.tile - 1) / tn.tile;
        ntiles += nt;
        nchunks += (nt + kBpChunkTiles - 1) / kBpChunkTiles;
        nfield += (it.n + tn.field_chunk - 1) / tn.field_chunk;
    }
    if (ntot >= (int64_t(1) << 30) || ntiles >= (int64_t(1) << 30)) return ETICS_ERR_ARG;
    const bool mixed = precision == ETICS_MIXED;
    // FP64: persistent blocks over static tile ranges, one segment per
    // (block, instance).  Mixed: blocks claim chunks, one segment per chunk
    int nblocks = (int)(num_sms * tn.blocks_per_sm);
    const int64_t units = mixed ? nchunks : ntiles;
    if (nblocks > units) nblocks = (int)(units > 0 ? units : 1);
    const int64_t nseg_max = mixed ? (nchunks > 0 ? nchunks : 1) : nblocks + ninst;
    BatchHeader hd{};
    hd.magic = kBatchMagic;
    hd.precision = precision;
    hd.ninst = ninst;
    hd.nblocks = nblocks;
    hd.nfield = (int)nfield;
    hd.T = tn.tile;
    hd.blocks_per_sm = tn.blocks_per_sm;
    hd.field_threads = tn.field_threads;
    hd.field_chunk = tn.field_chunk;
    hd.ntiles = (int)ntiles;
    hd.ntot = ntot;
    hd.coef_total = ctot;
    hd.seg_stride = (int64_t)scf_items(kBatchLM) * kBatchNR * 4;   // FP64 layout
    if (hd.seg_stride < (int64_t)kBatchNR * kBpCols) hd.seg_stride = (int64_t)kBatchNR * kBpCols;
    hd.ws_bytes = (size_t)nseg_max * (size_t)hd.seg_stride * sizeof(double);
    if (mixed) {
        hd.nchunks = (int)nchunks;
        hd.counter_off = (int64_t)((hd.ws_bytes + 255) / 256 * 256);
        hd.ws_bytes = (size_t)hd.counter_off + 256;
        const int64_t hcols = (int64_t)(lmax_all + 1) * (lmax_all + 1) * tn.tile;
        hd.bp_hfloats = hcols > kBpRedFloats ? hcols : kBpRedFloats;
        hd.smem_coef = kBpNbBytes + (size_t)(hd.bp_hfloats + tn.tile) * sizeof(float) +
                       (size_t)tn.tile * 4 * sizeof(float);
        if (hd.smem_coef > kMaxDynSmem) return ETICS_ERR_UNSUPPORTED;
    } else {
        const size_t main_max =
            (size_t)(kBatchLM + 1) * kBatchNR * tn.tile + (size_t)col_total(kBatchLM) * tn.tile;
        const size_t red_max = (size_t)kBatchThreads * kBatchNR * 4;
        const size_t el = main_max > red_max ? main_max : red_max;
        const size_t rsz = precision == ETICS_FP64 ? 8 : 4;
        hd.smem_coef = ((el * rsz + 15) / 16) * 16 + (size_t)hd.seg_stride * sizeof(double);
        // the largest FP64 tiles do not fit one block's shared memory
        if (hd.smem_coef > kMaxDynSmem) return ETICS_ERR_UNSUPPORTED;
    }
    size_t off = align16(sizeof(BatchHeader));
    hd.off_inst = (int64_t)off; off += align16(sizeof(BatchInst) * ninst);
    hd.off_block = (int64_t)off; off += align16(sizeof(BatchBlock) * nblocks);
    hd.off_seg = (int64_t)off; off += align16(sizeof(int) * nseg_max);
    hd.off_field = (int64_t)off; off += align16(sizeof(BatchField) * (nfield > 0 ? nfield : 1));
    hd.off_tile = (int64_t)off; off += align16(sizeof(int) * (ntiles > 0 ? ntiles : 1));
    hd.off_layout = (int64_t)off;
    if (mixed) off += align16(sizeof(BatchLayout) * (kBatchLM + 1));
    hd.off_chunk = (int64_t)off;
    if (mixed) off += align16(sizeof(BatchChunk) * (nchunks > 0 ? nchunks : 1));
    hd.total_bytes = (int64_t)off;
    *need = off;
    if (!plan) {
        if (ws_bytes) *ws_bytes = hd.ws_bytes;
        if (coef_total) *coef_total = ctot;
        return ETICS_OK;
    }
    if (plan_bytes < off) return ETICS_ERR_WORKSPACE;
    unsigned char* pb = static_cast<unsigned char*>(plan);
    std::memset(pb, 0, off);
    BatchInst* insts = reinterpret_cast<BatchInst*>(pb + hd.off_inst);
    BatchBlock* blocks = reinterpret_cast<BatchBlock*>(pb + hd.off_block);
    int* segs = reinterpret_cast<int*>(pb + hd.off_seg);
    BatchField* fields = reinterpret_cast<BatchField*>(pb + hd.off_field);
    int* tile_inst = reinterpret_cast<int*>(pb + hd.off_tile);
    int64_t o = 0, co = 0;
    int t = 0, f = 0;
    for (int i = 0; i < ninst; ++i) {
        BatchInst& in = insts[i];
        in.offset = o;
        in.n = items[i].n;
        in.n_max = items[i].n_max;
        in.l_max = items[i].l_max;
        in.coef_offset = co;
        in.first_tile = t;
        in.ntiles = (int)((in.n + tn.tile - 1) / tn.tile);
        for (int k = 0; k < in.ntiles; ++k) tile_inst[t + k] = i;
        for (int64_t b = 0; b < in.n; b += tn.field_chunk) {
            fields[f].begin = b;
            fields[f].count = (int)((in.n - b) < tn.field_chunk ? (in.n - b) : tn.field_chunk);
            fields[f].inst = i;
            ++f;
        }
        t += in.ntiles;
        o += in.n;
        co += (int64_t)(in.n_max + 1) * (in.l_max + 1) * (in.l_max + 1);
    }
    if (mixed) {
        BatchLayout* lays = reinterpret_cast<BatchLayout*>(pb + hd.off_layout);
        for (int l = 0; l <= kBatchLM; ++l) batch_layout(l, lays[l]);
        // chunks of the heaviest instances first (cost per tile: the busiest
        // lane's pairs times the per-pair work of n_max+1 rows, plus the
        // harmonics of phase 1), so that the light ones fill the tail; an
        // instance's chunks are consecutive, its segments in tile order
        auto cost = [&](const BatchInst& in) -> double {
            int nb = 0;
            for (int l = 0; l <= in.l_max; ++l) nb += (2 * l + 1 + kBpCap - 1) / kBpCap;
            const int lanes = kBpThreads / nb;
            const int pairs = (tn.tile / 2 + lanes - 1) / lanes;
            return pairs * (5.0 * (in.n_max + 1) + 6.0) + 5.0 * (in.l_max + 1) * (in.l_max + 1);
        };
        std::vector<int> order(ninst);
        for (int i = 0; i < ninst; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return cost(insts[a]) > cost(insts[b]); });
        BatchChunk* chunks = reinterpret_cast<BatchChunk*>(pb + hd.off_chunk);
        int c = 0;
        for (int i : order) {
            BatchInst& in = insts[i];
            in.first_seg = c;
            in.nseg = 0;
            for (int k0 = 0; k0 < in.ntiles; k0 += kBpChunkTiles) {
                const int k1 = k0 + kBpChunkTiles < in.ntiles ? k0 + kBpChunkTiles : in.ntiles;
                chunks[c++] = BatchChunk{i, in.first_tile + k0, in.first_tile + k1, 0};
                ++in.nseg;
            }
        }
        hd.nseg = c;
        std::memcpy(pb, &hd, sizeof(hd));
        if (ws_bytes) *ws_bytes = hd.ws_bytes;
        if (coef_total) *coef_total = ctot;
        return ETICS_OK;
    }
    // contiguous tile ranges per block, balanced by estimated cost per tile
    // (proportional to (n_max+1)(l_max+1)^2 plus fixed work)
    auto tile_cost = [&](const BatchInst& in) -> double {
        return (in.n_max + 1.0) * (in.l_max + 1.0) * (in.l_max + 1.0) + 40.0;
    };
    double total_cost = 0.0;
    for (int k = 0; k < ntiles; ++k) total_cost += tile_cost(insts[tile_inst[k]]);
    int nseg = 0, k = 0;
    double acc_cost = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        blocks[b].tile_begin = k;
        blocks[b].first_seg = nseg;
        const double target = total_cost * (b + 1) / nblocks;
        int last_inst = -1;
        while (k < ntiles && (acc_cost < target || b == nblocks - 1)) {
            const BatchInst& in = insts[tile_inst[k]];
            if (tile_inst[k] != last_inst) { segs[nseg++] = tile_inst[k]; last_inst = tile_inst[k]; }
            acc_cost += tile_cost(in);
            ++k;
        }
        blocks[b].tile_end = k;
    }
    hd.nseg = nseg;
    // segments of each instance are contiguous in block order
    for (int i = 0; i < ninst; ++i) { insts[i].first_seg = -1; insts[i].nseg = 0; }
    for (int s = 0; s < nseg; ++s) {
        BatchInst& in = insts[segs[s]];
        if (in.first_seg < 0) in.first_seg = s;
        ++in.nseg;
    }
    for (int i = 0; i < ninst; ++i)
        if (insts[i].first_seg < 0) insts[i].first_seg = 0;
    std::memcpy(pb, &hd, sizeof(hd));
    if (ws_bytes) *ws_bytes = hd.ws_bytes;
    if (coef_total) *coef_total = ctot;
    return ETICS_OK;
}

template <typename R>
int batch_launch(const void* posm, const void* plan_host, const void* plan_dev, double* coeffs,
                 void* out, int out_mask, void* ws, size_t ws_bytes, const LaunchCtx& ctx) {
    const BatchHeader& hd = *static_cast<const BatchHeader*>(plan_host);
    if (hd.magic != kBatchMagic || (hd.precision == ETICS_MIXED) != (sizeof(R) == 4))
        return ETICS_ERR_ARG;   // not a plan, or built for the other precision
    if (ws_bytes < hd.ws_bytes) return ETICS_ERR_WORKSPACE;
    if (hd.ntiles > 0) {
        if constexpr (sizeof(R) == 4) {
            auto k = batch_pairs_kernel;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hd.smem_coef))
                return ETICS_ERR_CUDA;
            unsigned* counter =
                reinterpret_cast<unsigned*>(static_cast<unsigned char*>(ws) + hd.counter_off);
            if (cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx.stream)) return ETICS_ERR_CUDA;
            k<<<hd.nblocks, kBpThreads, hd.smem_coef, ctx.stream>>>(
                reinterpret_cast<const float4*>(posm), plan_dev, static_cast<double*>(ws), counter,
                ctx.err);
        } else {
            auto k = batch_coeff_kernel<R>;
            if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)hd.smem_coef))
                return ETICS_ERR_CUDA;
            k<<<hd.nblocks, kBatchThreads, hd.smem_coef, ctx.stream>>>(
                reinterpret_cast<const Vec4<R>*>(posm), plan_dev, static_cast<double*>(ws), ctx.err);
        }
        if (cudaGetLastError()) return ETICS_ERR_CUDA;
        ++*ctx.launches;
    }
    stage_event(ctx, 1);
    if (hd.coef_total > 0) {
        const int64_t threads = hd.coef_total * 32;
        batch_finalize_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, ctx.stream>>>(
            plan_dev, static_cast<const double*>(ws), coeffs);
        if (cudaGetLastError()) return ETICS_ERR_CUDA;
        ++*ctx.launches;
    }
    stage_event(ctx, 2);
    if (out && hd.nfield > 0) {
        const size_t smem = (size_t)(kBatchNR) * col_total(kBatchLM) * sizeof(R);
        int grid = hd.nfield < ctx.num_sms * 8 ? hd.nfield : ctx.num_sms * 8;
        if (out_mask & ETICS_OUT_ACC) {
            auto k = batch_field_kernel<R, true>;
            if (smem > 48 * 1024 &&
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
                return ETICS_ERR_CUDA;
            k<<<grid, hd.field_threads, smem, ctx.stream>>>(
                reinterpret_cast<const Vec4<R>*>(posm), plan_dev, coeffs,
                reinterpret_cast<Vec4<R>*>(out), out_mask, ctx.err);
        } else {
            auto k = batch_field_kernel<R, false>;
            if (smem > 48 * 1024 &&
                cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
                return ETICS_ERR_CUDA;
            k<<<grid, hd.field_threads, smem, ctx.stream>>>(
                reinterpret_cast<const Vec4<R>*>(posm), plan_dev, coeffs,
                reinterpret_cast<Vec4<R>*>(out), out_mask, ctx.err);
        }
        if (cudaGetLastError()) return ETICS_ERR_CUDA;
        ++*ctx.launches;
    }
    stage_event(ctx, 3);
    return ETICS_OK;
}

template int batch_launch<float>(const void*, const void*, const void*, double*, void*, int, void*,
                                 size_t, const LaunchCtx&);
template int batch_launch<double>(const void*, const void*, const void*, double*, void*, int,
                                  void*, size_t, const LaunchCtx&);

}  // namespace etics
