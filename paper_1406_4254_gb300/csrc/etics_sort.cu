// etics_sort.cu -- the radial sort of MEX (paper Sec. 2.2: the cumulative
// sums need the particles ordered by radius; Sec. 3.2 used a library merge
// sort).
//
// GB300 design: a hand-written stable LSD radix sort (4 passes of 8 bits) of
// the high 32 bits of the FP64 r^2 bit pattern, one kernel per pass
// ("one-sweep": per-tile digit ranking with warp ballots, the tile's keys
// placed in digit order in shared memory, a decoupled lookback over tiles for
// the digit offsets, coalesced writes of digit runs).  Runs of equal high
// words are then ordered by the low 32 bits and the particle index, which
// reproduces the exact FP64 order (r^2 = (x*x + y*y) + z*z rounded as a CPU
// does, ties by index).  The passes and the tie fix-up are launched with
// programmatic dependent launch, so each launch overlaps its predecessor's
// tail.
#include "etics_internal.h"

namespace etics {

constexpr int kSortThreads = 256;
constexpr int kSortKpt = 16;
constexpr int kSortTile = kSortThreads * kSortKpt;   // 4096 keys per tile
constexpr int kLookbackWindow = 32;
constexpr int kStatusPad = kLookbackWindow;   // zeroed tiles before tile 0
constexpr int kMatchDigits = 8;               // rank with match_any up to this many digits
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr int64_t kSpinLimit = int64_t(1) << 22;   // default bound of a lookback wait

int sort_tiles(int64_t N) { return (int)((N + kSortTile - 1) / kSortTile); }

// r^2 exactly as a CPU evaluates (x*x + y*y) + z*z in FP64, no contraction
__device__ __forceinline__ double r2_fp64(double x, double y, double z) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}

// High 32 bits of the FP64 bit pattern of r^2 (the sort key; positive doubles
// order like their bit patterns).
//
// FP32 particles: every square is exact in FP64, so fl64(fl64(x*x+y*y)+z*z)
// differs from the exact sum S by at most 2 FP64 ulps.  S is evaluated as an
// FP32 pair (hi, lo) with error ~2^-45 |S| (exact products by FMA, TwoSum),
// and the key is read off the pair: the top 20 mantissa bits of hi, minus one
// when lo < 0 borrows across a bucket boundary (the low 3 mantissa bits of hi
// are zero).  Only when S lies within 2^-40 |S| of a bucket boundary is the
// key recomputed in FP64, so the result always equals the FP64 evaluation.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ uint32_t key_from_fp64(double r2) {
    return (uint32_t)((uint64_t)__double_as_longlong(r2) >> 32);
}

__device__ __forceinline__ uint32_t r2_key(float x, float y, float z) {
    const float hx = x * x, lx = fmaf(x, x, -hx);
    const float hy = y * y, ly = fmaf(y, y, -hy);
    const float hz = z * z, lz = fmaf(z, z, -hz);
    float s1, e1, s2, e2;
    two_sum(hx, hy, s1, e1);
    two_sum(s1, hz, s2, e2);
    const float low = ((lx + ly) + lz) + (e1 + e2);
    const float hi = s2 + low;                  // fast two-sum: |s2| >= |low|
    const float lo = low - (hi - s2);
    const uint32_t hb = __float_as_uint(hi);
    const uint32_t exp8 = hb >> 23, frac = hb & 0x7fffffu;
    // tiny (r^2 < 2^-63), non-finite or overflowing sums take the FP64 route
    bool exact_needed = exp8 < 64u || exp8 == 255u;
    uint32_t key = 0;
    if (!exact_needed) {
        key = ((exp8 + 896u) << 20) | (frac >> 3);   // FP64 exponent field = exp8 - 127 + 1023
        if ((frac & 7u) == 0u) {
            if (fabsf(lo) <= hi * 0x1p-40f) exact_needed = true;   // too close to call
            else if (lo < 0.0f) key -= 1u;                        // borrow below the boundary
        }
    }
    if (exact_needed) {
        const double dx = x, dy = y, dz = z;
        key = key_from_fp64(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                      __dmul_rn(dz, dz)));
    }
    return key;
}
__device__ __forceinline__ uint32_t r2_key(double x, double y, double z) {
    return key_from_fp64(r2_fp64(x, y, z));
}

constexpr int kKeygenIlp = 4;

template <typename R>
__global__ void __launch_bounds__(256)
keygen_kernel(const Vec4<R>* __restrict__ posm, int64_t N, uint32_t* __restrict__ key,
              uint32_t* __restrict__ hist, unsigned* err) {
    // one private copy of the 4 digit histograms per warp (less atomic contention)
    __shared__ uint32_t sh[8][4 * 256];
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < 8 * 4 * 256; i += blockDim.x) (&sh[0][0])[i] = 0;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < N;
         i0 += stride * kKeygenIlp) {
        Vec4<R> v[kKeygenIlp];
#pragma unroll
        for (int u = 0; u < kKeygenIlp; ++u) {
            const int64_t i = i0 + u * stride;
            if (i < N) v[u] = ld4(posm + i);
        }
#pragma unroll
        for (int u = 0; u < kKeygenIlp; ++u) {
            const int64_t i = i0 + u * stride;
            if (i >= N) break;
            uint32_t hi;
            if (finite4(v[u].x, v[u].y, v[u].z, v[u].w)) {
                hi = r2_key(v[u].x, v[u].y, v[u].z);
            } else {
                report(err, ETICS_ERR_NONFINITE);
                hi = 0xffffffffu;
            }
            key[i] = hi;
            // the histograms of digits 1 and 2 are counted by the radix
            // passes 0 and 1 (their keys are in registers there anyway)
            atomicAdd(&sh[warp][hi & 255], 1u);
            // the top byte (sign + high exponent bits) takes very few values:
            // aggregate equal digits within the warp before the atomic
            const uint32_t d3 = hi >> 24;
            const unsigned same = __match_any_sync(__activemask(), d3);
            if ((same & ((1u << (threadIdx.x & 31)) - 1u)) == 0u)
                atomicAdd(&sh[warp][768 + d3], (uint32_t)__popc(same));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) {
        if (i >= 256 && i < 768) continue;   // digits 1, 2: counted by the passes
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += sh[w][i];
        if (t) atomicAdd(&hist[i], t);
    }
}

template <typename R>
__global__ void radial_keys_kernel(const Vec4<R>* __restrict__ posm, int64_t N,
                                   uint32_t* __restrict__ keys, unsigned* err) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const Vec4<R> v = ld4(posm + i);
        if (finite4(v.x, v.y, v.z, v.w)) {
            keys[i] = r2_key(v.x, v.y, v.z);
        } else {
            report(err, ETICS_ERR_NONFINITE);
            keys[i] = 0xffffffffu;
        }
    }
}

template <typename R>
int radial_keys_impl(const void* posm, int64_t N, uint32_t* keys, const LaunchCtx& ctx) {
    if (N == 0) return ETICS_OK;
    int g = (int)((N + 255) / 256);
    if (g > ctx.num_sms * 8) g = ctx.num_sms * 8;
    radial_keys_kernel<R><<<g, 256, 0, ctx.stream>>>(reinterpret_cast<const Vec4<R>*>(posm), N,
                                                      keys, ctx.err);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}
template int radial_keys_impl<float>(const void*, int64_t, uint32_t*, const LaunchCtx&);
template int radial_keys_impl<double>(const void*, int64_t, uint32_t*, const LaunchCtx&);

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) {
    *reinterpret_cast<volatile uint32_t*>(p) = v;
}

// Stable rank of every key among the equal digits of its warp, keys taken in
// tile order (slot s, then lane).  The lanes that share a digit are found
// either with __match_any_sync (fast when a warp holds few distinct digits)
// or with one ballot per digit bit plus one for validity (a cost independent
// of how many distinct digits there are).
template <bool kMatch>
__device__ __forceinline__ void rank_in_warp(const uint32_t (&d)[kSortKpt], uint32_t (&rank)[kSortKpt],
                                             uint32_t* whist, int lane) {
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int s = 0; s < kSortKpt; ++s) {
        unsigned mask;
        if (kMatch) {
            mask = __match_any_sync(0xffffffffu, d[s]);
        } else {
            const unsigned vb = __ballot_sync(0xffffffffu, d[s] < 256u);
            mask = d[s] < 256u ? vb : ~vb;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const bool bit = (d[s] >> b) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, bit);
                mask &= bit ? bal : ~bal;
            }
        }
        const unsigned lower = mask & below;
        uint32_t before = 0;
        if (d[s] < 256u) before = whist[d[s]];
        rank[s] = before + (uint32_t)__popc(lower);
        __syncwarp();
        if (d[s] < 256u && lower == 0u) whist[d[s]] = before + (uint32_t)__popc(mask);
        __syncwarp();
    }
}

// One pass of the stable LSD radix sort (8-bit digit at `shift`) over tiles
// of kSortTile keys.  Order of work in a tile: load and rank; publish the
// tile's digit counts (status word: flag | count); scan the global histogram
// and the tile counts together; place the keys in digit order in shared
// memory; then find the exclusive prefix of each digit over earlier tiles by
// a decoupled lookback; finally write the keys out in digit runs.  `status`
// holds kStatusPad zeroed (never published) tiles before tile 0, so a
// lookback window may reach below tile 0 without a bounds test: tile 0
// always publishes an inclusive prefix, which ends every walk first.
// Launched with programmatic stream serialisation: nothing global is touched
// before griddepcontrol.wait.
__global__ void __launch_bounds__(kSortThreads, 2)
onesweep_kernel(const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
                uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out,
                const uint32_t* hist, uint32_t* status, uint32_t* counter, int shift,
                int64_t N, int64_t spin_limit, uint32_t* __restrict__ next_hist, unsigned* err) {
    __shared__ uint32_t s_keys[kSortTile];
    __shared__ uint32_t s_vals[kSortTile];
    __shared__ uint32_t s_whist[kSortThreads / 32][256];
    __shared__ uint32_t s_dexcl[256];
    __shared__ uint32_t s_gbase[256];
    __shared__ uint32_t s_scan[2][kSortThreads / 32];
    __shared__ uint32_t s_tile;
    __shared__ uint32_t s_next[256];   // this tile's histogram of the next digit
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < (kSortThreads / 32) * 256; i += kSortThreads) (&s_whist[0][0])[i] = 0;
    s_next[tid] = 0;
    pdl_wait();
    if (tid == 0) s_tile = atomicAdd(counter, 1u);
    const int dig = tid;
    // the histogram may have been completed by the kernel just before this
    // one (a programmatic dependent launch): a coherent load after the wait,
    // never the non-coherent read-only path
    const uint32_t gcount = __ldcg(hist + dig);
    // digits present in this pass over all keys: few -> rank with match_any
    const int ndig = __syncthreads_count(gcount != 0u);
    const uint32_t tile = s_tile;
    const int64_t start = (int64_t)tile * kSortTile;

    uint32_t k[kSortKpt], v[kSortKpt], d[kSortKpt], rank[kSortKpt];
#pragma unroll
    for (int s = 0; s < kSortKpt; ++s) {
        const int64_t idx = start + (int64_t)warp * kSortKpt * 32 + s * 32 + lane;
        if (idx < N) {
            k[s] = keys_in[idx];
            v[s] = vals_in ? vals_in[idx] : (uint32_t)idx;   // first pass: identity
            d[s] = (k[s] >> shift) & 255u;
        } else {
            k[s] = 0xffffffffu;
            v[s] = 0;
            d[s] = 256u;   // not a digit: out of range
        }
    }
    if (ndig <= kMatchDigits) rank_in_warp<true>(d, rank, s_whist[warp], lane);
    else rank_in_warp<false>(d, rank, s_whist[warp], lane);
    if (next_hist) {
        // the next pass's digit of this tile's keys (the order of the keys
        // does not matter for a histogram): added to the global histogram,
        // which the next pass reads after this one has completed
#pragma unroll
        for (int s = 0; s < kSortKpt; ++s)
            if (d[s] < 256u) atomicAdd(&s_next[(k[s] >> (shift + 8)) & 255u], 1u);
    }
    __syncthreads();
    if (next_hist && s_next[tid]) atomicAdd(&next_hist[tid], s_next[tid]);
    // per digit (one thread each): offsets over warps and the tile count
    uint32_t count = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t t = s_whist[w][dig];
        s_whist[w][dig] = count;
        count += t;
    }
    // publish at once: tile 0 (and any digit no key has) as inclusive
    uint32_t* st = status + (size_t)(tile + kStatusPad) * 256 + dig;
    const bool lookback = tile != 0 && gcount != 0u;
    st_volatile(st, (lookback ? kFlagAgg : kFlagInc) | count);
    // exclusive scans of the global histogram (start of each digit) and of
    // the tile counts (start of each digit in the tile), together
    uint32_t xa = gcount, xb = count;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t ta = __shfl_up_sync(0xffffffffu, xa, o);
        const uint32_t tb = __shfl_up_sync(0xffffffffu, xb, o);
        if (lane >= o) { xa += ta; xb += tb; }
    }
    if (lane == 31) { s_scan[0][warp] = xa; s_scan[1][warp] = xb; }
    __syncthreads();
    uint32_t ba = 0, bb = 0;
    for (int w = 0; w < warp; ++w) { ba += s_scan[0][w]; bb += s_scan[1][w]; }
    const uint32_t hexcl = ba + xa - gcount;
    s_dexcl[dig] = bb + xb - count;
    __syncthreads();
#pragma unroll
    for (int s = 0; s < kSortKpt; ++s) {
        if (d[s] < 256u) {
            const uint32_t pos = s_dexcl[d[s]] + s_whist[warp][d[s]] + rank[s];
            s_keys[pos] = k[s];
            s_vals[pos] = v[s];
        }
    }
    // decoupled lookback over earlier tiles for this digit: a window of
    // predecessors is read at once; flags become bit masks; counts are summed
    // up to the first inclusive prefix, or up to the first predecessor that
    // has not published (then that one word is polled before the next window).
    // The poll gives up after spin_limit tries: the error word records
    // ETICS_ERR_TIMEOUT and the tile goes on with the partial prefix (at most
    // the true one), so its output positions stay below N; keys that no
    // longer match the histogram (a later pass of a timed-out sort) can
    // compute a position >= N, and such a store is skipped below.
    uint32_t excl = 0;
    if (lookback) {
        const uint32_t* p = st - 256;   // tile - 1
        int64_t spins = 0;
        for (;;) {
            uint32_t w[kLookbackWindow];
#pragma unroll
            for (int j = 0; j < kLookbackWindow; ++j) w[j] = ld_volatile(p - j * 256);
            uint32_t pub = 0, inc = 0;
#pragma unroll
            for (int j = 0; j < kLookbackWindow; ++j) {
                const uint32_t f = w[j] >> 30;
                pub |= (f != 0u ? 1u : 0u) << j;
                inc |= (f == (kFlagInc >> 30) ? 1u : 0u) << j;
            }
            const int first_wait = ~pub ? __ffs(~pub) - 1 : kLookbackWindow;
            const int first_inc = inc ? __ffs(inc) - 1 : kLookbackWindow;
            const bool done = first_inc < first_wait;
            const int used = done ? first_inc + 1 : first_wait;
            const uint32_t take = used >= 32 ? 0xffffffffu : ((1u << used) - 1u);
#pragma unroll
            for (int j = 0; j < kLookbackWindow; ++j)
                if ((take >> j) & 1u) excl += w[j] & kCountMask;
            if (done) break;
            p -= (size_t)used * 256;
            if (used < kLookbackWindow) {
                bool timed_out = false;
                while ((ld_volatile(p) >> 30) == 0u) {
                    if (++spins > spin_limit) { timed_out = true; break; }
                    __nanosleep(32);
                }
                if (timed_out) { report(err, ETICS_ERR_TIMEOUT); break; }
            }
        }
        st_volatile(st, kFlagInc | (excl + count));
    }
    s_gbase[dig] = hexcl + excl;
    __syncthreads();
    const int64_t rem = N - start;
    const int nvalid = (int)(rem < kSortTile ? rem : kSortTile);
    if (nvalid == kSortTile) {
#pragma unroll
        for (int s = 0; s < kSortKpt; ++s) {
            const int i = tid + s * kSortThreads;
            const uint32_t kk = s_keys[i];
            const uint32_t dd = (kk >> shift) & 255u;
            const uint32_t pos = s_gbase[dd] + (uint32_t)i - s_dexcl[dd];
            if (pos < N) {
                keys_out[pos] = kk;
                vals_out[pos] = s_vals[i];
            } else {
                report(err, ETICS_ERR_TIMEOUT);
            }
        }
    } else {
        for (int i = tid; i < nvalid; i += kSortThreads) {
            const uint32_t kk = s_keys[i];
            const uint32_t dd = (kk >> shift) & 255u;
            const uint32_t pos = s_gbase[dd] + (uint32_t)i - s_dexcl[dd];
            if (pos < N) {
                keys_out[pos] = kk;
                vals_out[pos] = s_vals[i];
            } else {
                report(err, ETICS_ERR_TIMEOUT);
            }
        }
    }
}

// Runs of equal high words: order by (low word of the FP64 r^2, index).  The
// run's first element owns it; the low words are evaluated here, in FP64, for
// the run members only.  The radix passes are stable and began from index
// order, so a run's members arrive in index order: a stable sort by the low
// word alone gives the (low word, index) order.
// An index >= N (only after a timed-out sort) reads nothing and sorts last.
template <typename R>
__device__ __forceinline__ uint32_t r2_low(const Vec4<R>* posm, uint32_t i, int64_t N) {
    if ((int64_t)i >= N) return 0xffffffffu;
    const Vec4<R> v = ld4(posm + i);
    if (!finite4(v.x, v.y, v.z, v.w)) return 0xffffffffu;
    return (uint32_t)(uint64_t)__double_as_longlong(r2_fp64((double)v.x, (double)v.y, (double)v.z));
}

constexpr int kFixThreads = 256;   // one thread per digit in the block sort below
constexpr int kFixTile = 2048;
constexpr int kFixLocal = 16;      // runs up to this length: one thread, in registers
constexpr int kFixLongMax = kFixTile / (kFixLocal + 1) + 1;   // long runs starting in a tile

// a run of at most kFixLocal members, by one thread (insertion sort)
template <typename R>
__device__ __forceinline__ void sort_run_local(const Vec4<R>* posm, int64_t N, uint32_t* val,
                                               int64_t s, int len) {
    uint32_t lows[kFixLocal], ids[kFixLocal];
    for (int a = 0; a < len; ++a) ids[a] = val[s + a];
    for (int a = 0; a < len; ++a) lows[a] = r2_low<R>(posm, ids[a], N);
    for (int a = 1; a < len; ++a) {
        const uint32_t va = ids[a], la = lows[a];
        int b = a - 1;
        while (b >= 0 && (lows[b] > la || (lows[b] == la && ids[b] > va))) {
            ids[b + 1] = ids[b];
            lows[b + 1] = lows[b];
            --b;
        }
        ids[b + 1] = va;
        lows[b + 1] = la;
    }
    for (int a = 0; a < len; ++a) val[s + a] = ids[a];
}

// A long run (any length), by the whole block: a stable LSD radix sort of
// the members by their low word, 4 passes of 8 bits, ping-ponging between
// val (the sorted order) and tmp (the sort's spare value buffer, over the
// same positions); the low word is re-evaluated from the particle whenever it
// is needed, so nothing is written outside val/tmp[s, s + len).  Each pass:
// digit histogram, exclusive scan, then chunks of kFixThreads members in
// order, each member ranked among equal digits of its warp (ballots) and of
// the earlier warps of the chunk.
template <typename R>
__device__ void sort_run_block(const Vec4<R>* posm, int64_t N, uint32_t* val, uint32_t* tmp,
                               int64_t s, int64_t len, uint32_t (*s_cnt)[256], uint32_t* s_off,
                               uint32_t* s_wsum) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kFixThreads / 32;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        const uint32_t* src = (pass & 1) ? tmp : val;
        uint32_t* dst = (pass & 1) ? val : tmp;
        for (int w = 0; w < NW; ++w) s_cnt[w][tid] = 0u;
        __syncthreads();
        for (int64_t i = tid; i < len; i += kFixThreads)
            atomicAdd(&s_cnt[0][(r2_low<R>(posm, src[s + i], N) >> shift) & 255u], 1u);
        __syncthreads();
        {
            // exclusive scan over the 256 digits (thread = digit)
            const uint32_t c = s_cnt[0][tid];
            uint32_t x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += t;
            }
            if (lane == 31) s_wsum[warp] = x;
            __syncthreads();
            uint32_t b = 0;
            for (int w = 0; w < warp; ++w) b += s_wsum[w];
            s_off[tid] = b + x - c;
            s_cnt[0][tid] = 0u;
        }
        __syncthreads();
        for (int64_t c0 = 0; c0 < len; c0 += kFixThreads) {
            const int64_t i = c0 + tid;
            const bool valid = i < len;
            const uint32_t v = valid ? src[s + i] : 0u;
            const uint32_t d = valid ? (r2_low<R>(posm, v, N) >> shift) & 255u : 256u;
            const unsigned vb = __ballot_sync(0xffffffffu, valid);
            unsigned mask = valid ? vb : ~vb;
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool on = (d >> bit) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, on);
                mask &= on ? bal : ~bal;
            }
            const unsigned lower = mask & ((1u << lane) - 1u);
            if (valid && lower == 0u) s_cnt[warp][d] = (uint32_t)__popc(mask);
            __syncthreads();
            uint32_t total = 0;   // thread = digit: exclusive prefix over the warps
            for (int w = 0; w < NW; ++w) {
                const uint32_t t = s_cnt[w][tid];
                s_cnt[w][tid] = total;
                total += t;
            }
            __syncthreads();
            if (valid) dst[s + s_off[d] + s_cnt[warp][d] + (uint32_t)__popc(lower)] = v;
            __syncthreads();
            s_off[tid] += total;
            for (int w = 0; w < NW; ++w) s_cnt[w][tid] = 0u;
            __syncthreads();
        }
    }
    // 4 passes: the result is back in val
}

// One block per tile of kFixTile sorted positions; the keys of the tile and
// one position on either side are staged in shared memory.  A run belongs to
// the tile where it starts.  The block lists the runs that start in its tile;
// each thread finds the end of its runs by a search over the sorted keys and
// sorts those of at most kFixLocal members itself (so the dependent loads of
// all short runs are in flight together); then the block sorts the longer
// runs one after the other.  A long run may extend over later tiles: no
// other run starts inside it, so no other block touches its positions.
template <typename R>
__global__ void __launch_bounds__(kFixThreads)
tie_fixup_kernel(const uint32_t* __restrict__ key, const Vec4<R>* __restrict__ posm,
                 uint32_t* __restrict__ val, uint32_t* __restrict__ tmp, int64_t N,
                 unsigned* err) {
    __shared__ uint32_t s_key[kFixTile + 2];
    __shared__ int s_runs[kFixTile / 2];
    __shared__ int s_nruns, s_nlong;
    __shared__ int64_t s_long_s[kFixLongMax], s_long_n[kFixLongMax];
    // the long-run sort's counters reuse the staged keys and the run list
    // (both dead by then)
    static_assert(sizeof(uint32_t) * (kFixThreads / 32) * 256 <= sizeof(s_key), "counters");
    static_assert(sizeof(uint32_t) * (256 + kFixThreads / 32) <= sizeof(s_runs), "offsets");
    auto s_cnt = reinterpret_cast<uint32_t (*)[256]>(s_key);
    uint32_t* s_off = reinterpret_cast<uint32_t*>(s_runs);
    uint32_t* s_wsum = s_off + 256;
    const int64_t base = (int64_t)blockIdx.x * kFixTile;
    const int64_t rem = N - base;
    const int nt = (int)(rem < kFixTile ? rem : kFixTile);
    if (threadIdx.x == 0) { s_nruns = 0; s_nlong = 0; }
    pdl_wait();
    // s_key[i + 1] = key[base + i] for i in [-1, nt]; sentinels outside [0, N)
    for (int i = threadIdx.x - 1; i <= nt; i += kFixThreads) {
        const int64_t g = base + i;
        uint32_t v;
        if (g < 0) v = key[0] ^ 1u;             // differs from key[0]
        else if (g >= N) v = key[N - 1] ^ 1u;   // differs from key[N-1]
        else v = key[g];
        s_key[i + 1] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt; i += kFixThreads) {
        const uint32_t k = s_key[i + 1];
        if (s_key[i] != k && s_key[i + 2] == k) s_runs[atomicAdd(&s_nruns, 1)] = i;
    }
    __syncthreads();
    const int nruns = s_nruns;   // at most kFixTile / 2 (each run has >= 2 members)
    for (int r = threadIdx.x; r < nruns; r += kFixThreads) {
        const int64_t s = base + s_runs[r];
        const uint32_t k = s_key[s_runs[r] + 1];
        // last member: the keys are sorted, so it is the last position
        // holding k.  A run that ends inside the tile is found by bisection
        // over the staged keys (s_key[j + 1] is the key of local index j);
        // only a run that reaches the tile's end continues with doubling
        // steps and bisection over the keys in global memory.
        int64_t lo;
        if (s_key[nt] != k) {
            int a = s_runs[r] + 1, b = nt - 1;   // key(a) == k, key(b) != k
            while (b - a > 1) {
                const int mid = a + (b - a) / 2;
                if (s_key[mid + 1] == k) a = mid;
                else b = mid;
            }
            lo = base + a;
        } else if (s_key[nt + 1] != k) {
            lo = base + nt - 1;
        } else {
            lo = base + nt;                       // key[lo] == k
            int64_t hi = N, step = 1;
            for (;;) {
                const int64_t probe = lo + step;
                if (probe >= N || key[probe] != k) { hi = probe < N ? probe : N; break; }
                lo = probe;
                step <<= 1;
            }
            while (hi - lo > 1) {
                const int64_t mid = lo + (hi - lo) / 2;
                if (key[mid] == k) lo = mid;
                else hi = mid;
            }
        }
        const int64_t len = lo - s + 1;
        if (len <= kFixLocal) {
            sort_run_local<R>(posm, N, val, s, (int)len);
        } else {
            // sorted keys: long runs starting here do not overlap, so there
            // are fewer than kFixLongMax; unsorted keys (only after a
            // timed-out radix pass) can claim more, and those runs stay as
            // they are
            const int slot = atomicAdd(&s_nlong, 1);
            if (slot < kFixLongMax) {
                s_long_s[slot] = s;
                s_long_n[slot] = len;
            } else {
                report(err, ETICS_ERR_TIMEOUT);
            }
        }
    }
    __syncthreads();   // s_key and s_runs are dead from here
    const int nlong = s_nlong < kFixLongMax ? s_nlong : kFixLongMax;
    for (int r = 0; r < nlong; ++r)
        sort_run_block<R>(posm, N, val, tmp, s_long_s[r], s_long_n[r], s_cnt, s_off, s_wsum);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
SortBuffers sort_buffers(void* ws, int64_t N, size_t* total) {
    SortBuffers b{};
    uint8_t* p = reinterpret_cast<uint8_t*>(ws);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        uint8_t* q = p ? p + off : nullptr;
        off += (bytes + 255) / 256 * 256;
        return q;
    };
    const size_t n4 = (size_t)(N > 0 ? N : 1) * 4;
    b.keys_a = reinterpret_cast<uint32_t*>(take(n4));
    b.keys_b = reinterpret_cast<uint32_t*>(take(n4));
    b.vals_a = reinterpret_cast<uint32_t*>(take(n4));
    b.vals_b = reinterpret_cast<uint32_t*>(take(n4));
    const size_t nst = (size_t)sort_tiles(N);
    b.zero_bytes = (4 * 256 + 4 * (nst + kStatusPad) * 256 + 64) * 4;
    b.zero_bytes = (b.zero_bytes + 255) / 256 * 256;
    uint8_t* z = take(b.zero_bytes);
    b.hist = reinterpret_cast<uint32_t*>(z);
    b.status = b.hist ? b.hist + 4 * 256 : nullptr;
    b.counters = b.status ? b.status + 4 * (nst + kStatusPad) * 256 : nullptr;
    b.zero_base = z;
    if (total) *total = off;
    return b;
}

template <typename R>
int radial_sort_impl(const void* posm, int64_t N, const SortBuffers& b, const LaunchCtx& ctx) {
    if (cudaMemsetAsync(b.zero_base, 0, b.zero_bytes, ctx.stream)) return ETICS_ERR_CUDA;
    // few, long-lived blocks: each zeroes and merges 8 private histograms
    int kg = (int)((N + 256 * kKeygenIlp - 1) / (256 * kKeygenIlp));
    if (kg > ctx.num_sms * 2) kg = ctx.num_sms * 2;
    keygen_kernel<R><<<kg, 256, 0, ctx.stream>>>(reinterpret_cast<const Vec4<R>*>(posm), N,
                                                  b.keys_a, b.hist, ctx.err);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    stage_event(ctx, 1);
    const int nst = sort_tiles(N);
    uint32_t *kin = b.keys_a, *vin = b.vals_a, *kout = b.keys_b, *vout = b.vals_b;
    for (int pass = 0; pass < 4; ++pass) {
        const uint32_t* vals_in = pass == 0 ? nullptr : vin;
        // passes 0 and 1 count the histograms of digits 1 and 2
        uint32_t* next_hist = pass < 2 ? b.hist + (pass + 1) * 256 : nullptr;
        if (launch_pdl(onesweep_kernel, dim3(nst), dim3(kSortThreads), 0, ctx.stream, (const uint32_t*)kin,
                       vals_in, kout, vout, (const uint32_t*)(b.hist + pass * 256),
                       b.status + (size_t)pass * (nst + kStatusPad) * 256, b.counters + pass, 8 * pass,
                       N, ctx.wait_limit > 0 ? ctx.wait_limit : kSpinLimit, next_hist, ctx.err))
            return ETICS_ERR_CUDA;
        ++*ctx.launches;
        uint32_t* t = kin; kin = kout; kout = t;
        t = vin; vin = vout; vout = t;
    }
    // after 4 passes the sorted keys/values are back in keys_a / vals_a
    const int fg = (int)((N + kFixTile - 1) / kFixTile);
    if (launch_pdl(tie_fixup_kernel<R>, dim3(fg), dim3(kFixThreads), 0, ctx.stream,
                   (const uint32_t*)b.keys_a, reinterpret_cast<const Vec4<R>*>(posm), b.vals_a,
                   b.vals_b, N, ctx.err))
        return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

// One radix pass made to time out: kTimeoutProbeN keys, all 0, so the pass
// histogram has one digit; the tile counter starts at 1, so the single block
// takes tile 1 and looks back at tile 0, which never runs and never
// publishes.  The lookback gives up after `spins` polls, records
// ETICS_ERR_TIMEOUT and writes its tile at positions [0, kSortTile), inside
// the output buffers.
static __global__ void timeout_probe_setup_kernel(uint32_t* hist, uint32_t* counters, uint32_t n) {
    if (threadIdx.x == 0) {
        hist[0] = n;
        counters[0] = 1u;
    }
}

int lookback_timeout_probe(void* ws, int64_t spins, const LaunchCtx& ctx) {
    static_assert(kTimeoutProbeN == 2 * kSortTile, "the probe sorts two tiles");
    const SortBuffers b = sort_buffers(ws, kTimeoutProbeN, nullptr);
    if (cudaMemsetAsync(b.zero_base, 0, b.zero_bytes, ctx.stream) ||
        cudaMemsetAsync(b.keys_a, 0, kTimeoutProbeN * sizeof(uint32_t), ctx.stream))
        return ETICS_ERR_CUDA;
    timeout_probe_setup_kernel<<<1, 32, 0, ctx.stream>>>(b.hist, b.counters,
                                                         (uint32_t)kTimeoutProbeN);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    onesweep_kernel<<<1, kSortThreads, 0, ctx.stream>>>(b.keys_a, nullptr, b.keys_b, b.vals_b,
                                                         b.hist, b.status, b.counters, 0,
                                                         kTimeoutProbeN, spins, nullptr, ctx.err);
    if (cudaGetLastError()) return ETICS_ERR_CUDA;
    ++*ctx.launches;
    return ETICS_OK;
}

template int radial_sort_impl<float>(const void*, int64_t, const SortBuffers&, const LaunchCtx&);
template int radial_sort_impl<double>(const void*, int64_t, const SortBuffers&, const LaunchCtx&);

}  // namespace etics
