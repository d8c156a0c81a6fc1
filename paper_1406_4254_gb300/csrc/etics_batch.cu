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
//      instance are contiguous, so the finalize sums them in a fixed order);
//   2. finalize: one warp per output coefficient of any instance;
//   3. field: one block per work item (a chunk of one instance's particles),
//      the instance's coefficients staged in shared memory.
// No grid-wide barrier is needed, so the three launches capture into a CUDA
// graph as three nodes.  Tile size, blocks per SM and field chunking are
// tuning parameters (etics_batch_tuning) chosen by the autotuner.
#include <cstring>

#include "etics_scf_impl.cuh"

namespace etics {

constexpr int kBatchNR = 15;    // n_max <= 14
constexpr int kBatchLM = 8;     // l_max <= 8
constexpr int kBatchThreads = 256;

constexpr int kBatchMagic = 0x45544231;   // "ETB1"
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
    int64_t off_inst, off_block, off_seg, off_field, off_tile;
    int64_t total_bytes;
};
struct BatchInst {
    int64_t offset, n, coef_offset;
    int n_max, l_max, first_tile, ntiles, first_seg, nseg;
};
struct BatchBlock { int tile_begin, tile_end, first_seg, pad; };
struct BatchField { int64_t begin; int count, inst; };

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
    const int item = col_offset(l) / 4 + col / 4;
    const int idx = (item * kBatchNR + n) * 4 + (col & 3);
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
    if (tn.tile % 4 || tn.tile < 8 || tn.tile > kBatchThreads / 2) return ETICS_ERR_ARG;
    if (tn.field_threads % 32 || tn.field_threads < 32 || tn.field_threads > 256) return ETICS_ERR_ARG;
    if (tn.blocks_per_sm < 1 || tn.blocks_per_sm > 8 || tn.field_chunk < 1) return ETICS_ERR_ARG;
    int64_t ntot = 0, ctot = 0, ntiles = 0, nfield = 0;
    for (int i = 0; i < ninst; ++i) {
        const etics_batch_item& it = items[i];
        if (it.n < 0 || it.n_max < 0 || it.l_max < 0) return ETICS_ERR_ARG;
        if (it.n_max > kBatchNR - 1 || it.l_max > kBatchLM) return ETICS_ERR_UNSUPPORTED;
        ntot += it.n;
        ctot += (int64_t)(it.n_max + 1) * (it.l_max + 1) * (it.l_max + 1);
        ntiles += (it.n + tn.tile - 1) / tn.tile;
        nfield += (it.n + tn.field_chunk - 1) / tn.field_chunk;
    }
    if (ntot >= (int64_t(1) << 30) || ntiles >= (int64_t(1) << 30)) return ETICS_ERR_ARG;
    int nblocks = (int)(num_sms * tn.blocks_per_sm);
    if (nblocks > ntiles) nblocks = (int)(ntiles > 0 ? ntiles : 1);
    const int64_t nseg_max = nblocks + ninst;
    BatchHeader hd{};
    hd.magic = kBatchMagic;
    hd.precision = precision;
    hd.ws_bytes = (size_t)nseg_max * (size_t)scf_items(kBatchLM) * kBatchNR * 4 * sizeof(double);
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
    hd.seg_stride = (int64_t)scf_items(kBatchLM) * kBatchNR * 4;
    {
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
    // contiguous tile ranges per block, balanced by estimated cost per tile
    // (proportional to (n_max+1)(l_max+1)^2 + fixed work)
    double total_cost = 0.0;
    for (int k = 0; k < ntiles; ++k) {
        const BatchInst& in = insts[tile_inst[k]];
        total_cost += (in.n_max + 1.0) * (in.l_max + 1.0) * (in.l_max + 1.0) + 40.0;
    }
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
            acc_cost += (in.n_max + 1.0) * (in.l_max + 1.0) * (in.l_max + 1.0) + 40.0;
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
        auto k = batch_coeff_kernel<R>;
        if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hd.smem_coef))
            return ETICS_ERR_CUDA;
        int grid = hd.nblocks;
        k<<<grid, kBatchThreads, hd.smem_coef, ctx.stream>>>(
            reinterpret_cast<const Vec4<R>*>(posm), plan_dev, static_cast<double*>(ws), ctx.err);
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
