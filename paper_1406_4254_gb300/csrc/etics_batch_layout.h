// etics_batch_layout.h -- lane layout of the mixed-precision batched SCF
// coefficient pass (plain C++, shared by the plan builder and its host test).
#pragma once

#include <cstddef>
#include <cstdint>

namespace etics {

constexpr int kBatchNR = 15;    // n_max <= 14
constexpr int kBatchLM = 8;     // l_max <= 8

// Mixed-precision coefficient pass (batch_pairs_kernel).  A block of
// kBpThreads lanes handles one tile of up to kBpMaxTile particles of one
// instance at a time.  The instance's expansion is cut into bins -- each
// level's 2l+1 columns split evenly into ceil((2l+1)/kBpCap) bins -- and the
// lanes are shared out evenly among the bins: lane j owns bin b(j) and takes
// the particle pairs p = rank, rank + nlanes, ... of the tile.  The layout
// depends only on l_max and is built on the host (batch_layout).  Blocks take
// chunks of at most kBpChunkTiles tiles of one instance at a time.
constexpr int kBpThreads = 512;
constexpr int kBpMaxTile = 512;
constexpr int kBpCap = 3;
constexpr int kBpCols = (kBatchLM + 1) * (kBatchLM + 1);
constexpr int kBpMaxBins = 30;        // sum over l <= 8 of ceil((2l+1)/3)
constexpr int kBpChunkTiles = 16;     // tiles per claimed chunk (one FP32 accumulation window)
constexpr int kBpNbStride = 17;       // shared recursion constants per level (bank padding)
constexpr size_t kBpNbBytes = ((size_t)(kBatchLM + 1) * kBpNbStride * sizeof(float) + 15) / 16 * 16;
constexpr int64_t kBpRedFloats = (int64_t)kBatchNR * kBpCap * kBpThreads;

struct BatchLane { int16_t col[kBpCap]; int16_t level, rank, nlanes; };
struct BatchBin { int16_t level, col0, nc, lane0, nlanes, pad; };
struct BatchLayout {
    int nbins, pad;
    BatchBin bin[kBpMaxBins];
    BatchLane lane[kBpThreads];
};

// bins of levels 0..l_max (dense columns l*l + c: c = 0 -> m = 0, 2m-1 -> cos,
// 2m -> sin) and an equal share of the lanes for each: every bin costs the
// same per particle pair (kBpCap paired FMAs and two recursion instructions
// per row), so the shares differ by at most one lane.  Slots beyond a bin's
// width repeat its first column; their sums are never read.
inline void batch_layout(int l_max, BatchLayout& lay) {
    int nb = 0;
    for (int l = 0; l <= l_max; ++l) {
        const int nc = 2 * l + 1, k = (nc + kBpCap - 1) / kBpCap;
        int c = 0;
        for (int b = 0; b < k; ++b) {
            const int w = nc / k + (b < nc % k ? 1 : 0);
            lay.bin[nb].level = (int16_t)l;
            lay.bin[nb].col0 = (int16_t)(l * l + c);
            lay.bin[nb].nc = (int16_t)w;
            lay.bin[nb].pad = 0;
            ++nb;
            c += w;
        }
    }
    lay.nbins = nb;
    lay.pad = 0;
    int lane0 = 0;
    for (int b = 0; b < nb; ++b) {
        const int n = kBpThreads / nb + (b < kBpThreads % nb ? 1 : 0);
        lay.bin[b].lane0 = (int16_t)lane0;
        lay.bin[b].nlanes = (int16_t)n;
        for (int r = 0; r < n; ++r) {
            BatchLane& ln = lay.lane[lane0 + r];
            for (int c = 0; c < kBpCap; ++c)
                ln.col[c] = (int16_t)(lay.bin[b].col0 + (c < lay.bin[b].nc ? c : 0));
            ln.level = lay.bin[b].level;
            ln.rank = (int16_t)r;
            ln.nlanes = (int16_t)n;
        }
        lane0 += n;
    }
}

}  // namespace etics
