// Host-side check of the wide pass kernel's index maps
// (paper_2606_18981_gb300/csrc/qft_wide.cuh): the same constexpr functions
// the kernel runs, evaluated exhaustively on the CPU.
//
//   * the stage-0 and stage-1 thread maps are bijections onto their tile bits,
//     and the exchange round (tile bit 3) is warp bit 0 in both maps;
//   * every shared-memory address the kernel forms as base + compile-time
//     offset equals the layout function of the tile index it stands for
//     (128-byte TMA swizzle for the tile buffer, padded exchange buffer);
//   * the exchange buffer's layout is injective, fits its allocation, and in
//     each round the writers cover exactly the indices the readers read;
//   * every warp-wide shared-memory access is bank-conflict free: within each
//     half warp (16 lanes x 8 bytes) the 8-byte slots mod 16 are distinct;
//   * stores: lanes 0..7 (middle/last passes) or 0..15 (first pass) write
//     consecutive output addresses when the planner's store maps hold.
// Prints one line per check and "ALL OK" when every check holds.  With the
// argument --dump it prints the thread maps instead (one line per thread:
// tid, wide_x0, wide_x1 middle/last, wide_x1 first pass), which the numpy
// replay of the kernel's data flow (tests/wide_emulator.py) reads.
#include <cstdint>
#include <cstdio>
#include <set>
#include <string>
#include <vector>

#include "qft_wide.cuh"

using namespace qft;

static int g_fail = 0;
static void check(bool ok, const char* what) {
    std::printf("%-72s %s\n", what, ok ? "ok" : "FAIL");
    if (!ok) ++g_fail;
}

static bool half_warps_conflict_free(const std::vector<uint32_t>& addr_of_tid, int warp) {
    for (int h = 0; h < 2; ++h) {
        std::set<uint32_t> slots;
        for (int l = 0; l < 16; ++l) slots.insert(addr_of_tid[warp * 32 + h * 16 + l] % 16u);
        if (slots.size() != 16) return false;
    }
    return true;
}

int main(int argc, char** argv) {
    const int NT = kWideThreads;
    if (argc > 1 && std::string(argv[1]) == "--dump") {
        for (int t = 0; t < NT; ++t) std::printf("%d %u %u %u\n", t, wide_x0(t), wide_x1(t, false), wide_x1(t, true));
        return 0;
    }
    // 1. thread maps
    {
        std::set<uint32_t> s0, s1t, s1f;
        bool bits0 = true, bits1 = true, round = true;
        for (int t = 0; t < NT; ++t) {
            const uint32_t a = wide_x0(t), bt = wide_x1(t, true), bf = wide_x1(t, false);
            s0.insert(a);
            s1t.insert(bt);
            s1f.insert(bf);
            bits0 = bits0 && (a < 512u);
            bits1 = bits1 && ((bt & 0x1F0u) == 0) && ((bf & 0x1F0u) == 0) && bt < (1u << 14) && bf < (1u << 14);
            const uint32_t r = (t >> 5) & 1u;
            round = round && ((a >> 3) & 1u) == r && ((bt >> 3) & 1u) == r && ((bf >> 3) & 1u) == r;
        }
        check(s0.size() == 512 && bits0, "stage-0 map: bijection onto tile bits 0..8");
        check(s1t.size() == 512 && s1f.size() == 512 && bits1, "stage-1 maps: bijections onto tile bits {0..3, 9..13}");
        check(round, "exchange round bit (tile bit 3) = warp bit 0 in every map");
    }
    // 2. base + offset addressing equals the layout functions
    {
        bool okT = true, okW = true, okR = true;
        for (int t = 0; t < NT; ++t)
            for (uint32_t j = 0; j < 32; ++j) {
                const uint32_t xs0 = wide_x0(t) | (j << 9);
                okT = okT && wide_swz128(xs0) == wide_swz128(wide_x0(t)) + (j << 9);
                okW = okW && wide_zpad(wide_compress(xs0)) == wide_a0(t) + wide_k0(j);
                for (int top = 0; top < 2; ++top) {
                    const uint32_t xs1 = wide_x1(t, top) | (j << 4);
                    okR = okR && wide_zpad(wide_compress(xs1)) == wide_a1(t, top) + wide_k1(j);
                }
            }
        check(okT, "tile buffer: swz128(x0 | j<<9) = swz128(x0) + j<<9");
        check(okW, "exchange writes: zpad(compress(x0 | j<<9)) = a0 + k0(j)");
        check(okR, "exchange reads: zpad(compress(x1 | j<<4)) = a1 + k1(j), both maps");
    }
    // 3. layouts: injective, in bounds; each round's writers and readers cover the same half tile
    {
        std::set<uint32_t> z;
        bool inb = true;
        for (uint32_t i = 0; i < 8192; ++i) {
            z.insert(wide_zpad(i));
            inb = inb && wide_zpad(i) < kWideZElems;
        }
        check(z.size() == 8192 && inb, "exchange layout: injective on 8192 indices and < kWideZElems");
        std::set<uint32_t> sw;
        for (uint32_t x = 0; x < (1u << 14); ++x) sw.insert(wide_swz128(x));
        check(sw.size() == (1u << 14) && *sw.rbegin() < (1u << 14), "128-byte swizzle: a permutation of the tile");
        bool cover = true;
        for (int r = 0; r < 2; ++r)
            for (int top = 0; top < 2; ++top) {
                std::set<uint32_t> wr, rd;
                for (int t = 0; t < NT; ++t) {
                    if (((t >> 5) & 1) != r) continue;
                    for (uint32_t j = 0; j < 32; ++j) {
                        wr.insert(wide_a0(t) + wide_k0(j));
                        rd.insert(wide_a1(t, top) + wide_k1(j));
                    }
                }
                cover = cover && wr.size() == 8192 && wr == rd;
            }
        check(cover, "each round: 8192 distinct slots written, exactly those read");
        check(kWideSmemBytes + 10 * 1024 <= 227 * 1024, "shared memory (dynamic + static) within 227 KiB");
    }
    // 4. bank conflicts, per warp instruction (fixed j)
    {
        bool okT = true, okW = true, okR0 = true, okR1 = true;
        std::vector<uint32_t> aT(NT), aW(NT), aR0(NT), aR1(NT);
        for (uint32_t j = 0; j < 32; ++j) {
            for (int t = 0; t < NT; ++t) {
                aT[t] = wide_swz128(wide_x0(t)) + (j << 9);
                aW[t] = wide_a0(t) + wide_k0(j);
                aR0[t] = wide_a1(t, false) + wide_k1(j);
                aR1[t] = wide_a1(t, true) + wide_k1(j);
            }
            for (int w = 0; w < NT / 32; ++w) {
                okT = okT && half_warps_conflict_free(aT, w);
                okW = okW && half_warps_conflict_free(aW, w);
                okR0 = okR0 && half_warps_conflict_free(aR0, w);
                okR1 = okR1 && half_warps_conflict_free(aR1, w);
            }
        }
        check(okT, "stage-0 tile-buffer reads: conflict free");
        check(okW, "exchange writes: conflict free");
        check(okR0, "exchange reads, middle/last-pass map: conflict free");
        check(okR1, "exchange reads, first-pass map: conflict free");
    }
    // 5. store runs: with p_out[b] = b for b < 3 (middle/last) or p_out[13 - i] = i (first pass)
    {
        bool mid = true, top = true;
        for (int w = 0; w < NT / 32; ++w)
            for (int l = 0; l < 32; ++l) {
                const uint32_t bf = wide_x1(w * 32 + l, false), bt = wide_x1(w * 32 + l, true);
                mid = mid && (bf & 7u) == uint32_t(l & 7);
                uint32_t o = 0;
                for (int i = 0; i < 4; ++i) o |= ((bt >> (13 - i)) & 1u) << i;
                top = top && o == uint32_t(l & 15);
            }
        check(mid, "middle/last-pass stores: lanes 8k..8k+7 write output addresses +0..+7");
        check(top, "first-pass stores: lanes 16k..16k+15 write output addresses +0..+15");
    }
    std::printf(g_fail ? "FAILED %d\n" : "ALL OK\n", g_fail);
    return g_fail ? 1 : 0;
}
