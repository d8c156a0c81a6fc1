// etics_tc.cuh -- a bf16 GEMM slice on the 5th-generation tensor cores
// (tcgen05): operands staged in shared memory in the canonical K-major layout,
// the FP32 accumulator in tensor memory (TMEM), completion tracked by an
// mbarrier that tcgen05.commit arrives on, the result read back with
// tcgen05.ld.  Used by the MLP products of etics_mlp.cu whose tiles are large
// enough (M >= 64, N >= 64); every wait is bounded.
//
// part[z][M][N] = sum over k in slice z of A(m, k) B(k, n), with
//   A(m, k) = TA ? A[k * lda + m] : A[m * lda + k]
//   B(k, n) = TB ? B[k * ldb + n] : B[n * ldb + k]
// Block tile 128 x 128, K step 64 (four m128 n128 k16 MMAs).  Two kernels:
// gemm_tma_kernel, whose operand tiles arrive by TMA (cp.async.bulk.tensor)
// with the 128-byte swizzle into a ring of stages, for operands whose
// addresses and row strides are multiples of 16 bytes; and gemm_kernel, which
// stages any layout with plain loads into the unswizzled canonical layout.
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; the encoder is fetched at run time)
#include <cuda_bf16.h>

#include "etics_common.cuh"

namespace etics {
namespace tc {

using bf16 = __nv_bfloat16;

constexpr int kM = 128, kN = 128, kK = 64;
constexpr int kThreads = 128;
constexpr int kStages = 2;
constexpr int kTileElems = kM * kK;          // one operand tile (A or B: kN == kM)
constexpr int kTmemCols = kN;                // FP32 accumulator: 128 lanes x 128 columns
constexpr long long kSpinLimit = 1ll << 22;
// second, longer bound of the final drain before tensor memory is freed
constexpr long long kDrainLimit = 1ll << 26;

// shared memory of one block (dynamic, 1024-byte aligned base)
struct Smem {
    bf16 a[kStages][kTileElems];
    bf16 b[kStages][kTileElems];
    unsigned long long mbar[kStages];
    uint32_t tmem;
};
constexpr size_t kSmemBytes = sizeof(Smem) + 1024;

// Canonical K-major layout without swizzle: 8 x 8 "core matrices" (8 rows of
// 16 bytes, 128 contiguous bytes each); core (i, j) covers rows 8i..8i+7 and
// k = 8j..8j+7 and sits at element offset (i * 8 + j) * 64.  So the next core
// along K is 128 bytes away (leading byte offset) and the next along M/N
// 1024 bytes (stride byte offset).
__device__ __forceinline__ int tile_offset(int r, int k) {
    return (((r >> 3) * 8 + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128 >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((1024 >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                            ((uint32_t)(kN >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// bounded wait for the completion of the phase with this parity
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity,
                                          long long limit = kSpinLimit) {
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (i > 32) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void mma_id(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t adesc, uint64_t bdesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Stage the (128 x 64) tile of operand X (rows r0.., k = k0..) into T in the
// canonical layout; out-of-range elements are zero.
//  RM == false: X[r * ld + k] (k contiguous);  RM == true: X[k * ld + r]
template <bool RM>
__device__ __forceinline__ void stage(bf16* T, const bf16* __restrict__ X, int64_t ld, int r0,
                                      int R, int k0, int ke, int tid) {
    const bf16 zero = __float2bfloat16_rn(0.0f);
#pragma unroll
    for (int it = 0; it < (kM * kK / 8) / kThreads; ++it) {
        const int chunk = it * kThreads + tid;       // 1024 chunks of 8 elements
        if (!RM) {
            const int r = chunk >> 3, kc = (chunk & 7) * 8;
            const int gr = r0 + r, gk = k0 + kc;
            const bf16* src = X + (int64_t)gr * ld + gk;
            bf16* dst = T + tile_offset(r, kc);
            if (gr < R && gk + 8 <= ke && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) dst[e] = (gr < R && gk + e < ke) ? src[e] : zero;
            }
        } else {
            // r contiguous in memory: each thread gathers 8 consecutive k of one
            // row (8 two-byte loads, each coalesced across the warp's
            // consecutive rows) and writes them as one 16-byte core-matrix row
            const int r = chunk & (kM - 1), kc = (chunk >> 7) * 8;
            const int gr = r0 + r, gk = k0 + kc;
            const bf16* src = X + (int64_t)gk * ld + gr;
            alignas(16) bf16 v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                v[e] = (gr < R && gk + e < ke) ? src[(int64_t)e * ld] : zero;
            *reinterpret_cast<uint4*>(T + tile_offset(r, kc)) = *reinterpret_cast<const uint4*>(v);
        }
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads)
gemm_kernel(const bf16* __restrict__ A, int64_t lda, const bf16* __restrict__ B, int64_t ldb,
            float* __restrict__ part, int M, int N, int K, int kslice, unsigned* err) {
    extern __shared__ unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                        ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kM, n0 = blockIdx.x * kN;
    const int kb = blockIdx.z * kslice;
    const int ke = min(K, kb + kslice);
    const int nk = (ke - kb + kK - 1) / kK;

    if (warp == 0) tmem_alloc(smem_u32(&sm.tmem), kTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&sm.mbar[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    // every decision that guards a barrier or a warp-collective instruction
    // is made uniform over the block with __syncthreads_and
    bool ok = true;
    int issued = 0;                   // tiles whose MMAs were issued (uniform)
    if (nk > 0) {
        stage<TA>(sm.a[0], A, lda, m0, M, kb, ke, tid);
        stage<TB>(sm.b[0], B, ldb, n0, N, kb, ke, tid);
    }
    for (int kt = 0; kt < nk; ++kt) {
        const int s = kt & 1;
        fence_async_smem();           // this tile's shared-memory writes -> async proxy
        if (!__syncthreads_and(ok)) { ok = false; break; }
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sm.a[s]), b0 = smem_u32(sm.b[s]);
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk)   // k16 step = two cores = 256 bytes
                mma(tmem, make_desc(a0 + kk * 256), make_desc(b0 + kk * 256),
                    (kt > 0 || kk > 0) ? 1u : 0u);
            commit(smem_u32(&sm.mbar[s]));
        }
        issued = kt + 1;
        if (kt + 1 < nk) {
            const int s2 = (kt + 1) & 1;
            // the MMAs of tile kt-1 read stage s2: wait for them before refilling it
            if (kt >= 1 && !mbar_wait(smem_u32(&sm.mbar[s2]), (uint32_t)(((kt - 1) >> 1) & 1)))
                ok = false;
            if (ok) {
                const int k0 = kb + (kt + 1) * kK;
                stage<TA>(sm.a[s2], A, lda, m0, M, k0, ke, tid);
                stage<TB>(sm.b[s2], B, ldb, n0, N, k0, ke, tid);
            }
        }
    }
    ok = __syncthreads_and(ok);
    // the last commit covers every MMA issued before it; on failure this is
    // still the (bounded) wait for the MMAs in flight before TMEM is freed,
    // tried once more with a much longer bound.  Should that run out as well,
    // TMEM is freed with MMAs possibly still writing it: the error word says
    // ETICS_ERR_TIMEOUT, and the host must treat that as fatal for the
    // context (later tensor-memory users on the SM could see those writes).
    const uint32_t last_bar = smem_u32(&sm.mbar[(issued - 1) & 1]);
    const uint32_t last_par = (uint32_t)(((issued - 1) >> 1) & 1);
    bool drained = issued == 0 || mbar_wait(last_bar, last_par);
    if (!drained) drained = mbar_wait(last_bar, last_par, kDrainLimit);
    ok = __syncthreads_and(ok && drained && issued == nk);
    if (!ok && tid == 0) report(err, ETICS_ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
        // warp w reads TMEM lanes 32w..32w+31 = tile rows 32w.., 32 columns at a time
        const int row = m0 + warp * 32 + lane;
        float* out = part + (size_t)blockIdx.z * M * N;
#pragma unroll 1
        for (int c0 = 0; c0 < kN; c0 += 32) {
            float v[32];
            if (nk > 0) {
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0f;
            }
            if (row < M) {
                float* dst = out + (size_t)row * N + n0 + c0;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (n0 + c0 + i < N) dst[i] = v[i];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// TMA-fed variant.  One lane of warp 0 copies the operand tiles of each K
// step into a ring of kTmaStages stages (cp.async.bulk.tensor, 128-byte
// swizzle), one lane of warp 1 issues the MMAs, the four warps read the
// accumulator back.  Per stage s: full[s] completes when both tiles have
// landed (one arrive with the expected byte count, then the copies' bytes),
// empty[s] when the MMAs that read the stage have completed (tcgen05.commit).
// Shared-memory layouts (bf16; each tile 1024-byte aligned):
//   K-major operand (row r, k contiguous in memory): one box of 64 k x 128
//     rows; row r at r * 128 bytes, its 16-byte chunks XOR-swizzled by r % 8;
//     8-row groups 1024 bytes apart (the descriptor's stride byte offset);
//     the next k16 step starts 32 bytes further.
//   MN-major operand (k rows, r contiguous in memory): two boxes of 64 r x
//     64 k, the second (r + 64) 8192 bytes after the first (leading byte
//     offset); k-row at k * 128 bytes inside a box, 8-k groups 1024 bytes
//     apart (stride byte offset); the next k16 step starts 2048 bytes further.
// Every copy starts at an x coordinate that is a multiple of 64 elements
// (128 bytes); boxes reaching past the tensor are zero-filled by the copy.
// ---------------------------------------------------------------------------
// three stages (96 KB) leave room for two blocks per SM, so that one block's
// TMEM read-back and stores overlap the other's MMAs (16384 x 4096 x 4096:
// 676 TFLOP/s with four stages and one block per SM, 866 with this)
constexpr int kTmaStages = 3;
constexpr uint32_t kTileBytes = (uint32_t)kTileElems * 2;   // 16 KB
struct SmemTma {
    bf16 a[kTmaStages][kTileElems];
    bf16 b[kTmaStages][kTileElems];
    unsigned long long full[kTmaStages];
    unsigned long long empty[kTmaStages];
    unsigned long long done;
    uint32_t tmem;
    int loaded;     // K steps whose copies were issued
    int consumed;   // K steps whose MMAs were issued
};
constexpr size_t kSmemTmaBytes = sizeof(SmemTma) + 1024;
static_assert(kTileBytes % 1024 == 0, "tiles keep the 1024-byte alignment of the swizzle");

// shared-memory descriptor with the 128-byte swizzle (mode 2 in bits 61-63)
__device__ __forceinline__ uint64_t make_desc_sw128(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// the (128 rows x 64 k) tile of one operand at (r0, k0) into dst
template <bool MN>
__device__ __forceinline__ void tma_tile(uint32_t dst, const CUtensorMap* map, int r0, int k0,
                                         uint32_t bar) {
    if (MN) {
        tma_load_2d(dst, map, r0, k0, bar);
        tma_load_2d(dst + 8192, map, r0 + 64, k0, bar);
    } else {
        tma_load_2d(dst, map, k0, r0, bar);
    }
}

// descriptor of the k16 step kk of a tile at addr
template <bool MN>
__device__ __forceinline__ uint64_t tile_desc(uint32_t addr, int kk) {
    return MN ? make_desc_sw128(addr + (uint32_t)kk * 2048u, 8192u, 1024u)
              : make_desc_sw128(addr + (uint32_t)kk * 32u, 16u, 1024u);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(kThreads, 2)
gemm_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                float* __restrict__ part, int M, int N, int K, int kslice, unsigned* err) {
    extern __shared__ unsigned char smem_raw[];
    SmemTma& sm = *reinterpret_cast<SmemTma*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                              ~uintptr_t(1023));
    constexpr uint32_t idesc = kIdesc | (TA ? 1u << 15 : 0u) | (TB ? 1u << 16 : 0u);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kM, n0 = blockIdx.x * kN;
    const int kb = blockIdx.z * kslice;
    const int ke = min(K, kb + kslice);
    const int nk = ke > kb ? (ke - kb + kK - 1) / kK : 0;

    if (warp == 0) tmem_alloc(smem_u32(&sm.tmem), kTmemCols);
    if (tid == 0) {
        for (int s = 0; s < kTmaStages; ++s) {
            mbar_init(smem_u32(&sm.full[s]), 1);
            mbar_init(smem_u32(&sm.empty[s]), 1);
        }
        mbar_init(smem_u32(&sm.done), 1);
        sm.loaded = 0;
        sm.consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sm.tmem;

    bool ok = true;
    if (warp == 0 && lane == 0) {
        // copies: stage s is refilled once the MMAs of its previous use are done
        int kt = 0;
        for (; kt < nk; ++kt) {
            const int s = kt % kTmaStages;
            if (kt >= kTmaStages &&
                !mbar_wait(smem_u32(&sm.empty[s]), (uint32_t)((kt / kTmaStages - 1) & 1))) {
                ok = false;
                break;
            }
            const uint32_t full = smem_u32(&sm.full[s]);
            mbar_expect_tx(full, 2 * kTileBytes);
            const int k0 = kb + kt * kK;
            tma_tile<TA>(smem_u32(sm.a[s]), &tmA, m0, k0, full);
            tma_tile<TB>(smem_u32(sm.b[s]), &tmB, n0, k0, full);
        }
        sm.loaded = kt;
    } else if (warp == 1 && lane == 0) {
        // MMAs: four k16 steps per stage, then the stage is released
        int kt = 0;
        for (; kt < nk; ++kt) {
            const int s = kt % kTmaStages;
            if (!mbar_wait(smem_u32(&sm.full[s]), (uint32_t)((kt / kTmaStages) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sm.a[s]), b0 = smem_u32(sm.b[s]);
#pragma unroll
            for (int kk = 0; kk < kK / 16; ++kk)
                mma_id(tmem, tile_desc<TA>(a0, kk), tile_desc<TB>(b0, kk), idesc,
                       (kt > 0 || kk > 0) ? 1u : 0u);
            commit(smem_u32(&sm.empty[s]));
        }
        sm.consumed = kt;
        // arrives once every MMA issued above has completed
        commit(smem_u32(&sm.done));
    }
    __syncwarp();
    ok = __syncthreads_and(ok);
    // Every MMA issued has completed when `done` completes; on a timed-out
    // wait this is also the (bounded) wait before TMEM is freed, tried once
    // more with a much longer bound, and copies still in flight are waited
    // for (bounded) so that none lands after the block has exited.
    bool drained = mbar_wait(smem_u32(&sm.done), 0u);
    if (!drained) drained = mbar_wait(smem_u32(&sm.done), 0u, kDrainLimit);
    if (!ok && tid == 0) {
        for (int kt = sm.consumed; kt < sm.loaded; ++kt)
            if (!mbar_wait(smem_u32(&sm.full[kt % kTmaStages]),
                           (uint32_t)((kt / kTmaStages) & 1)))
                drained = false;
    }
    ok = __syncthreads_and(ok && drained && sm.consumed == nk);
    if (!ok && tid == 0) report(err, ETICS_ERR_TIMEOUT);
    tc_fence_after();
    if (ok) {
        // warp w reads TMEM lanes 32w..32w+31 = tile rows 32w.., 32 columns at a time
        const int row = m0 + warp * 32 + lane;
        float* out = part + (size_t)blockIdx.z * M * N;
#pragma unroll 1
        for (int c0 = 0; c0 < kN; c0 += 32) {
            float v[32];
            if (nk > 0) {
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) v[i] = 0.0f;
            }
            if (row < M) {
                float* dst = out + (size_t)row * N + n0 + c0;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (n0 + c0 + i < N) dst[i] = v[i];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// A wait that runs out on purpose: tensor memory held, an mbarrier that
// nothing arrives on, a bound of `limit` tries.  Nothing is issued to the
// tensor cores, so freeing the columns afterwards is safe; the error word
// receives ETICS_ERR_TIMEOUT (what the product kernel does when a wait gives
// up).
__global__ void __launch_bounds__(kThreads) wait_timeout_kernel(long long limit, unsigned* err) {
    __shared__ unsigned long long bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), 32);
    if (tid == 0) {
        mbar_init(smem_u32(&bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const bool ok = __syncthreads_and(mbar_wait(smem_u32(&bar), 0u, limit));
    if (!ok && tid == 0) report(err, ETICS_ERR_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 32);
}

}  // namespace tc
}  // namespace etics
