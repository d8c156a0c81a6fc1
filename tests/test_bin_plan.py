"""Host-side check of the per-warp-bin plans of the SCF coefficient pass: for
every level bound the plan assigns each harmonic column (l, c), c < 2l+1,
to exactly one bin slot, no bin holds more than its column capacity or four
level segments, and the finalize's column -> (bin, slot) map inverts the
plan.  The plans are compile-time C++; a small host program prints them."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1406_4254_gb300", "csrc")

PROGRAM = r"""
#include "etics_scf_bins.cuh"
#include <cstdio>
template <int LM> void show() {
    constexpr auto p = etics::BinConst<LM>::plan;
    constexpr auto ix = etics::make_bin_index<LM>();
    printf("LM %d %d %d\n", LM, p.nbins, etics::kBinCap);
    for (int b = 0; b < p.nbins; ++b) {
        printf("B %d %d", b, p.bin[b].nseg);
        for (int s = 0; s < p.bin[b].nseg; ++s)
            printf(" %d %d %d", p.bin[b].seg[s].l, p.bin[b].seg[s].c0, p.bin[b].seg[s].n);
        printf("\n");
    }
    for (int j = 0; j < (LM + 1) * (LM + 1); ++j) printf("I %d %d %d\n", j, ix.bin[j], ix.slot[j]);
}
int main() { show<2>(); show<4>(); show<6>(); show<8>(); return 0; }
"""


def _plans(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "plan.cu"
    exe = tmp_path / "plan"
    src.write_text(PROGRAM)
    r = subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                        "-o", str(exe), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    plans, cur = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "LM":
            cur = {"lm": int(f[1]), "nbins": int(f[2]), "cap": int(f[3]), "bins": [], "index": {}}
            plans[cur["lm"]] = cur
        elif f[0] == "B":
            v = list(map(int, f[3:]))
            cur["bins"].append([tuple(v[i:i + 3]) for i in range(0, len(v), 3)])
        else:
            cur["index"][int(f[1])] = (int(f[2]), int(f[3]))
    return plans


def test_bin_plans_cover_every_column_once(tmp_path):
    for lm, p in _plans(tmp_path).items():
        assert len(p["bins"]) == p["nbins"]
        seen = {}
        for b, segs in enumerate(p["bins"]):
            assert 1 <= len(segs) <= 4, (lm, b)
            assert sum(n for _, _, n in segs) <= p["cap"], (lm, b)
            off = 0
            for l, c0, n in segs:
                assert 0 <= l <= lm and n >= 1 and 0 <= c0 and c0 + n <= 2 * l + 1, (lm, b)
                for c in range(c0, c0 + n):
                    j = l * l + c
                    assert j not in seen, (lm, j)
                    seen[j] = (b, off + c - c0)
                off += n
        assert sorted(seen) == list(range((lm + 1) ** 2)), lm
        # the finalize's map is the inverse of the plan
        assert seen == p["index"], lm


PAIR_PROGRAM = r"""
#include "etics_scf_pairs.cuh"
#include <cstdio>
template <int LM, int CAP> void show() {
    constexpr auto p = etics::make_pair_plan<LM, CAP>();
    printf("LM %d %d %d\n", LM, CAP, p.nbins);
    for (int b = 0; b < p.nbins; ++b) printf("B %d %d %d %d\n", b, p.bin[b].l, p.bin[b].c0, p.bin[b].nc);
    for (int j = 0; j < (LM + 1) * (LM + 1); ++j) printf("I %d %d %d\n", j, p.bin_of[j], p.slot_of[j]);
}
int main() { show<6, 3>(); show<6, 4>(); show<8, 3>(); return 0; }
"""


def test_pair_plans_split_each_level_evenly_and_invert(tmp_path):
    """The particle-pair coefficient pass: every bin is one level's run of at
    most CAP consecutive columns, each level is split into ceil((2l+1)/CAP)
    bins whose widths differ by at most one, bins are ordered by width
    (widest first, so the threads beyond the tile sit in the lightest warps),
    and the finalize's column -> (bin, slot) map inverts the plan."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src, exe = tmp_path / "pairs.cu", tmp_path / "pairs"
    src.write_text(PAIR_PROGRAM)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, "-I",
                        os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    plans, cur = [], None
    for line in out.splitlines():
        f = list(map(int, line.split()[1:]))
        if line.startswith("LM"):
            cur = {"lm": f[0], "cap": f[1], "nbins": f[2], "bins": [], "index": {}}
            plans.append(cur)
        elif line.startswith("B"):
            cur["bins"].append(tuple(f[1:]))
        else:
            cur["index"][f[0]] = (f[1], f[2])
    assert len(plans) == 3
    for p in plans:
        lm, cap = p["lm"], p["cap"]
        assert len(p["bins"]) == p["nbins"] == sum(-(-(2 * l + 1) // cap) for l in range(lm + 1))
        seen = {}
        widths = {}
        for b, (l, c0, nc) in enumerate(p["bins"]):
            assert 0 <= l <= lm and 1 <= nc <= cap and 0 <= c0 and c0 + nc <= 2 * l + 1
            widths.setdefault(l, []).append(nc)
            for c in range(c0, c0 + nc):
                j = l * l + c
                assert j not in seen
                seen[j] = (b, c - c0)
        assert sorted(seen) == list(range((lm + 1) ** 2))
        assert seen == p["index"]
        for l, w in widths.items():
            assert max(w) - min(w) <= 1 and sum(w) == 2 * l + 1, (lm, cap, l, w)
        nc_order = [nc for _, _, nc in p["bins"]]
        assert nc_order == sorted(nc_order, reverse=True)


LAYOUT_PROGRAM = r"""
#include "etics_batch_layout.h"
#include <cstdio>
int main() {
    static etics::BatchLayout lay;
    printf("K %d %d %d\n", etics::kBpThreads, etics::kBpCap, etics::kBpMaxBins);
    for (int lm = 0; lm <= etics::kBatchLM; ++lm) {
        etics::batch_layout(lm, lay);
        printf("LM %d %d\n", lm, lay.nbins);
        for (int b = 0; b < lay.nbins; ++b)
            printf("B %d %d %d %d %d\n", lay.bin[b].level, lay.bin[b].col0, lay.bin[b].nc,
                   lay.bin[b].lane0, lay.bin[b].nlanes);
        for (int j = 0; j < etics::kBpThreads; ++j)
            printf("L %d %d %d %d %d %d\n", lay.lane[j].col[0], lay.lane[j].col[1],
                   lay.lane[j].col[2], lay.lane[j].level, lay.lane[j].rank, lay.lane[j].nlanes);
    }
    return 0;
}
"""


def test_batch_lane_layouts(tmp_path):
    """The mixed-precision batch pass: for every l_max the bins cover each
    dense column l*l + c exactly once, one level per bin, at most three
    columns, each level split evenly; every lane belongs to one bin (ranks
    0..nlanes-1 on consecutive lanes), the shares differ by at most one lane,
    and the bin's lanes take each particle pair of a tile exactly once."""
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("g++ not available")
    src, exe = tmp_path / "layout.cpp", tmp_path / "layout"
    src.write_text(LAYOUT_PROGRAM)
    r = subprocess.run([gxx, "-std=c++17", "-I", CSRC, "-o", str(exe), str(src)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    lays, cur, consts = {}, None, None
    for line in out.splitlines():
        f = list(map(int, line.split()[1:]))
        if line.startswith("K"):
            consts = f
        elif line.startswith("LM"):
            cur = {"nbins": f[1], "bins": [], "lanes": []}
            lays[f[0]] = cur
        elif line.startswith("B"):
            cur["bins"].append(tuple(f))
        else:
            cur["lanes"].append(tuple(f))
    threads, cap, maxbins = consts
    assert sorted(lays) == list(range(9))
    for lm, lay in lays.items():
        bins = lay["bins"]
        assert len(bins) == lay["nbins"] == sum(-(-(2 * l + 1) // cap) for l in range(lm + 1))
        assert len(bins) <= maxbins
        seen, widths = set(), {}
        for l, col0, nc, lane0, nl in bins:
            assert 1 <= nc <= cap and l * l <= col0 and col0 + nc <= (l + 1) * (l + 1)
            widths.setdefault(l, []).append(nc)
            for j in range(col0, col0 + nc):
                assert j not in seen
                seen.add(j)
        assert seen == set(range((lm + 1) ** 2))
        for l, w in widths.items():
            assert max(w) - min(w) <= 1 and sum(w) == 2 * l + 1
        shares = [nl for *_, nl in bins]
        assert sum(shares) == threads and max(shares) - min(shares) <= 1
        lanes = lay["lanes"]
        assert len(lanes) == threads
        nxt = 0
        for l, col0, nc, lane0, nl in bins:
            assert lane0 == nxt
            nxt += nl
            for r in range(nl):
                c0, c1, c2, lev, rank, nls = lanes[lane0 + r]
                assert (lev, rank, nls) == (l, r, nl)
                assert [c0, c1, c2] == [col0 + (c if c < nc else 0) for c in range(cap)]
            for tp in (32, 96, 256):
                pairs = sorted(p for r in range(nl) for p in range(r, tp, nl))
                assert pairs == list(range(tp))
