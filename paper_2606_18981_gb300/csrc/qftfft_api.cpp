// qftfft_api.cpp -- host planner and C ABI of libqftfft (see include/qftfft.h).
//
// The planner turns the n-wire (A)QFT circuit (Sec. 3 step 2, Fig. 1) into a
// few HBM passes (Sec. 3.1: the planner fuses gates into blocks and emits a
// device-agnostic schedule; here each pass is one launch of the pass kernel):
//
//   * n <= tile bits: one pass, the whole state is one CTA tile;
//   * otherwise the wires are split top-down into groups G_1 .. G_P, one per
//     pass, each pass's tile being G_j plus "batch" wires that sit at the
//     lowest addresses so every HBM run is >= 2^coalesce amplitudes long.
//
// Output order NATURAL (the swaps applied) is produced by layout adapters:
// pass 1 writes the top wires to the lowest addresses and the lowest wires to
// the top (out of place into the workspace), the middle passes work in place
// there, and the last pass writes the bit-reversed layout back into the
// caller's state.  BITREV order keeps the identity layout and runs in place.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/qftfft.h"
#include <nvtx3/nvToolsExt.h>
#include "plan_host.hpp"


using namespace qft;

namespace qft {

thread_local int g_last_cuda = 0;

int set_cuda_error(cudaError_t e) {
    g_last_cuda = static_cast<int>(e);
    return QFT_ERR_CUDA;
}

void set_cuda_error_code(int e) { g_last_cuda = e; }

bool plan_device_ready(const qft_plan_s* pl) {
    return !pl->precision || pl->passes.empty() || pl->passes[0].tc_a_hi != nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

}  // namespace qft

namespace {
int cuda_fail(cudaError_t e) { return qft::set_cuda_error(e); }
}  // namespace

namespace {

// Host copy of the kernel's buffer-B swizzle: the low SW bits of a tile index
// XORed with the XOR-fold of its higher SW-bit groups (SW = 4 for 8-byte,
// 3 for 16-byte amplitudes).
uint32_t swizzle(uint32_t x, size_t esize) {
    const int SW = esize == 8 ? 4 : 3;
    uint32_t y = x >> SW, f = 0;
    for (int i = 0; i < 16 / SW + 1; ++i) { f ^= y; y >>= SW; }
    return x ^ (f & ((1u << SW) - 1));
}

int effective_k(int n, int k) { return (k < 0 || k > n - 1) ? std::max(n - 1, 0) : k; }

// Build one pass from its wire group [glo, glo + a), batch wires, and the
// input/output wire -> address maps.
//
// Logical wires 0 .. m-1 are the transform's wires (m = pl->n); a subset plan
// has further logical wires m .. n-1 (n = pl->n_addr address bits) that carry
// no gate: the kernel's phases only see bits below m (P.n = m), so these
// wires act as a batch index.
bool build_pass(qft_plan_s* pl, PassHost& ph, int glo, int a, const std::vector<int>& batch_in,
                const std::vector<int>& Lin, const std::vector<int>& Lout, bool first, bool last) {
    const int n = pl->n_addr;
    const int m = pl->n;
    PassParams& P = ph.prm;
    std::memset(&P, 0, sizeof(P));
    P.n = m;
    P.kk = pl->kk;
    P.first = first;
    P.last = last;
    P.inv_root_n = std::ldexp(1.0, -m / 2) * ((m & 1) ? std::sqrt(0.5) : 1.0);
    ph.wires = a;

    std::vector<char> in_tile(n, 0);
    for (int w = glo; w < glo + a; ++w) in_tile[w] = 1;
    std::vector<int> batch = batch_in;
    for (int w : batch) in_tile[w] = 1;
    std::vector<int> wire_at(n);
    for (int w = 0; w < n; ++w) wire_at[Lin[w]] = w;
    // Fill the tile to the full tile width with the lowest-address non-tile
    // wires: more batch wires only lengthen the HBM runs and keep every
    // thread of the CTA busy in every stage.
    {
        int have = a + static_cast<int>(batch.size());
        for (int adr = 0; adr < n && have < std::min(pl->TB, n); ++adr) {
            const int w = wire_at[adr];
            if (!in_tile[w]) {
                in_tile[w] = 1;
                batch.push_back(w);
                ++have;
            }
        }
    }
    std::vector<int> tw, nt;  // tile wires / non-tile wires, sorted by input address
    for (int adr = 0; adr < n; ++adr) (in_tile[wire_at[adr]] ? tw : nt).push_back(wire_at[adr]);
    const int tb = static_cast<int>(tw.size());
    if (tb > kMaxTileBits || tb < 1) return false;
    P.tb = tb;
    P.num_tiles = int64_t(1) << (n - tb);
    std::vector<int> pos(n, -1);
    for (int i = 0; i < tb; ++i) {
        P.p_wire[i] = tw[i];
        P.p_out[i] = Lout[tw[i]];
        pos[tw[i]] = i;
    }
    P.paired = 0;
    const int pb0 = 0;
    const int rmax = pl->rmax;
    // tile coordinate segments (bit m of the tile coordinate <-> wire nt[m])
    P.nseg = 0;
    for (int m = 0; m < static_cast<int>(nt.size());) {
        int len = 1;
        int dir = 0;
        while (m + len < static_cast<int>(nt.size()) && nt[m + len] == nt[m + len - 1] + 1) {
            const int d = Lout[nt[m + len]] - Lout[nt[m + len - 1]];
            if (d != 1 && d != -1) break;
            if (dir == 0) dir = d;
            else if (d != dir) break;
            ++len;
        }
        if (P.nseg >= kMaxSegs) return false;
        TileSeg& S = P.seg[P.nseg++];
        S.src = m;
        S.len = len;
        S.wire = nt[m];
        S.out = Lout[nt[m]];
        S.out_rev = dir < 0 ? 1 : 0;
        m += len;
    }
    // TMA dims: runs of tile / non-tile input address bits, tile runs cut to <= 8 bits
    const int inner_mult = static_cast<int>(pl->esize / 8);  // UINT64 elements per amplitude
    int nd = 0;
    int adr = 0;
    int m_of_adr = 0;  // tile-coordinate bit index of the next non-tile address
    if (!in_tile[wire_at[0]]) return false;  // the lowest address must be a tile bit (contiguous runs)
    while (adr < n) {
        const bool t = in_tile[wire_at[adr]];
        int len = 1;
        while (adr + len < n && static_cast<bool>(in_tile[wire_at[adr + len]]) == t) ++len;
        if (t) {
            int left = len, start = adr;
            while (left > 0) {
                const int maxbits = (nd == 0) ? (inner_mult == 2 ? 7 : 8) : 8;
                const int cut = std::min(left, maxbits);
                if (nd >= kMaxDims) return false;
                ph.gdim[nd] = (cuuint64_t(1) << cut) * (nd == 0 ? inner_mult : 1);
                ph.box[nd] = (cuuint32_t(1) << cut) * (nd == 0 ? inner_mult : 1);
                if (nd > 0) ph.gstride[nd - 1] = (cuuint64_t(1) << start) * pl->esize;
                P.dim_src[nd] = 0;
                P.dim_len[nd] = 0;
                ++nd;
                start += cut;
                left -= cut;
            }
        } else {
            if (nd >= kMaxDims) return false;
            ph.gdim[nd] = cuuint64_t(1) << len;
            ph.box[nd] = 1;
            ph.gstride[nd - 1] = (cuuint64_t(1) << adr) * pl->esize;
            P.dim_src[nd] = m_of_adr;
            P.dim_len[nd] = len;
            m_of_adr += len;
            ++nd;
        }
        adr += len;
    }
    P.ndims = nd;
    ph.run_bits = 0;
    while (ph.run_bits < n && in_tile[wire_at[ph.run_bits]]) ++ph.run_bits;
    for (int d = nd; d < kMaxDims; ++d) {  // pad to rank 5 with extent-1 dims
        ph.gdim[d] = 1;
        ph.box[d] = 1;
        ph.gstride[d - 1] = (cuuint64_t(1) << n) * pl->esize;
        P.dim_src[d] = 0;
        P.dim_len[d] = 0;
    }
    for (int d = 0; d < kMaxDims; ++d) P.dim_scale[d] = 1;

    // Stages: the group's wires top-down, split into blocks that are
    // consecutive both as wires and as tile bits; within each such run the
    // first block takes the remainder so later blocks have rmax wires.
    std::vector<std::pair<int, int>> runs;  // (top wire, length)
    for (int w = glo + a - 1; w >= glo;) {
        int len = 1;
        while (w - len >= glo && pos[w - len] == pos[w - len + 1] - 1) ++len;
        runs.push_back({w, len});
        w -= len;
    }
    P.nstages = 0;
    for (auto& rr : runs) {
        // as few stages as rmax allows, sizes as equal as possible (larger first)
        const int len = rr.second;
        const int nst = (len + rmax - 1) / rmax;
        int top = rr.first;
        for (int i = 0; i < nst; ++i) {
            const int r = len / nst + (i < len % nst ? 1 : 0);
            if (P.nstages >= kMaxStages) return false;
            StageDesc& S = P.st[P.nstages++];
            S.r = r;
            S.wlo = top - r + 1;
            S.q = pos[S.wlo];
            S.cross = (top < m - 1) ? 1 : 0;
            S.ngbits = tb - r - pb0;
            S.tile_above = 0;
            for (int w : nt)
                if (w > top && w < m) S.tile_above = 1;
            for (int e = 0; e < kMaxR; ++e)
                S.img[e] = e >= r ? 0 : static_cast<int32_t>(swizzle(1u << (S.q + e), pl->esize));
            top -= r;
        }
    }
    // Lane order of each stage's group index.
    const bool unit16 = pl->esize == 16;  // buffer-B access width: 16 bytes (complex128)
    const int SW = unit16 ? 3 : 4;                    // swizzle slot bits
    const int wave_lanes = unit16 ? 3 : 4;            // log2 lanes per SMEM wavefront
    for (int s = 0; s < P.nstages; ++s) {
        StageDesc& S = P.st[s];
        std::vector<int> others;
        for (int p = pb0; p < tb; ++p)
            if (p < S.q || p >= S.q + S.r) others.push_back(p);
        std::vector<int> order;
        if (s == P.nstages - 1) {
            // last stage stores to HBM: lanes follow the output address bits
            order = others;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P.p_out[x] < P.p_out[y]; });
        } else {
            // lanes of one wavefront on distinct residues mod SW (bank-conflict free)
            std::vector<char> used_res(SW, 0), taken(tb, 0);
            for (int p : others) {
                if (static_cast<int>(order.size()) >= wave_lanes) break;
                const int res = (p - pb0) % SW;  // residue of the buffer-B unit bit
                if (!used_res[res]) {
                    used_res[res] = 1;
                    taken[p] = 1;
                    order.push_back(p);
                }
            }
            for (int p : others)
                if (!taken[p]) order.push_back(p);
        }
        for (int i = 0; i < S.ngbits; ++i) S.gpos[i] = order[i];
        const int hi_w = S.wlo + S.r - 1;
        S.lo_tw = S.hi_tw = 0;
        for (int i = 0; i < S.ngbits; ++i)
            if (P.p_wire[S.gpos[i]] > hi_w && P.p_wire[S.gpos[i]] < m) (i < 5 ? S.lo_tw : S.hi_tw) = 1;
        if (!S.lo_tw && !S.hi_tw) S.hi_tw = 1;  // keep one (all-ones) factor so tau is defined
    }
    int ntab = 0, nU = 0;
    for (int s = 0; s < P.nstages; ++s) {
        P.st[s].uoff = nU;
        nU += P.st[s].r;
        P.tab_off[s] = ntab;
        const int ng = 1 << P.st[s].ngbits;
        ntab += 32 + (ng > 32 ? ng >> 5 : 1);
    }
    P.ntab = ntab;
    P.nU = nU;
    int maxr = 0;
    for (int s = 0; s < P.nstages; ++s) maxr = std::max(maxr, static_cast<int>(P.st[s].r));
    P.ntw = maxr;
    ph.smem = pass_smem_bytes(P, pl->esize);
    if (ph.smem > 227 * 1024 - 4096) return false;
    // Two CTAs per SM (16 warps) when the pass's buffers fit twice into the
    // SM's 228 KB of shared memory (with the static part and the 1 KB the
    // system reserves per CTA) and its stages are small enough for 128
    // registers per thread.
    ph.minb = 1;
    if (pl->dtype == QFT_C64 && pl->threads == 256 && maxr <= 4 &&
        2 * (ph.smem + 3 * 1024) <= 228 * 1024)
        ph.minb = 2;
    // double-float: the same with blocks of <= 3 wires (tiles of <= 2^11 pairs;
    // 4.1 KB of static shared memory plus the 1 KB reserve)
    if (pl->df && pl->threads == 256 && maxr <= 3 && 2 * (ph.smem + 5 * 1024) <= 228 * 1024) ph.minb = 2;
    const int64_t tiles = P.num_tiles;
    ph.grid = static_cast<int>(std::min<int64_t>(tiles, int64_t(pl->num_sms) * ph.minb));
    return true;
}

// Wide pass (complex64, qft_wide.cuh): a tile of 2^14 amplitudes in the bit
// order x0..x3 = the 4 lowest input addresses (batch), x4..x8 = E1 extra batch
// wires then the r1 wires of the pass's low block, x9..x13 = E0 extra batch
// wires then the r0 wires of its top block (E = 5 - r).  The TMA box
// dimensions follow that order (tile bits of consecutive input addresses share
// one dimension), so the tile lands in shared memory in x order; the
// tile-coordinate dimensions (box extent 1) follow.  extra_mode picks the extra
// batch wires: 0 = the lowest free input addresses (stage 1's first), 1 = the
// same with stage 0's first, 2 = the free addresses just below the low block
// (so they extend its TMA dimension).  Returns false when the shape does not
// fit (more than 5 TMA dimensions, or store maps that would not coalesce).
bool build_pass_wide(qft_plan_s* pl, PassHost& ph, int glo, int a, int r0, const std::vector<int>& Lin,
                     const std::vector<int>& Lout, bool first, bool last, bool top, int extra_mode) {
    const int n = pl->n;       // transform wires: phases, normalisation
    const int na = pl->n_addr; // address bits (> n: a subset plan's upper wires, a batch index)
    const int r1 = a - r0;
    if (r0 < 4 || r0 > 5 || r1 < 3 || r1 > 5) return false;
    const int E0 = 5 - r0, E1 = 5 - r1;
    std::vector<int> wire_at(na);
    for (int w = 0; w < na; ++w) wire_at[Lin[w]] = w;
    std::vector<char> used(na, 0);
    for (int w = glo; w < glo + a; ++w) used[w] = 1;
    int xw[14];
    for (int b = 0; b < 4; ++b) {
        const int w = wire_at[b];
        if (used[w]) return false;
        xw[b] = w;
        used[w] = 1;
    }
    std::vector<int> ex0, ex1;
    if (extra_mode == 2) {
        std::vector<int> below;  // free wires at decreasing addresses under the low block
        for (int adr = Lin[glo] - 1; adr >= 0 && static_cast<int>(below.size()) < E0 + E1; --adr)
            if (!used[wire_at[adr]]) below.push_back(wire_at[adr]);
        if (static_cast<int>(below.size()) < E0 + E1) return false;
        for (int i = E1 - 1; i >= 0; --i) ex1.push_back(below[i]);
        for (int i = E0 + E1 - 1; i >= E1; --i) ex0.push_back(below[i]);
    } else {
        std::vector<int> cand;
        for (int adr = 0; adr < na; ++adr)
            if (!used[wire_at[adr]]) cand.push_back(wire_at[adr]);
        if (static_cast<int>(cand.size()) < E0 + E1) return false;
        const int nfirst = extra_mode == 0 ? E1 : E0;
        for (int i = 0; i < E0 + E1; ++i) ((i < nfirst) == (extra_mode == 0) ? ex1 : ex0).push_back(cand[i]);
    }
    int x = 4;
    for (int w : ex1) xw[x++] = w;
    for (int w = glo; w < glo + r1; ++w) xw[x++] = w;
    for (int w : ex0) xw[x++] = w;
    for (int w = glo + r1; w < glo + a; ++w) xw[x++] = w;
    std::vector<char> in_tile(na, 0);
    for (int b = 0; b < 14; ++b) in_tile[xw[b]] = 1;

    PassParams& P = ph.prm;
    std::memset(&P, 0, sizeof(P));
    P.n = n;
    P.kk = pl->kk;
    P.first = first;
    P.last = last;
    P.tb = 14;
    P.num_tiles = int64_t(1) << (na - 14);
    P.inv_root_n = std::ldexp(1.0, -n / 2) * ((n & 1) ? std::sqrt(0.5) : 1.0);
    ph.wires = a;
    for (int b = 0; b < 14; ++b) {
        P.p_wire[b] = xw[b];
        P.p_out[b] = Lout[xw[b]];
    }
    // coalesced stores: the first pass stores along x13..x10 (output 0..3), the others along x0..x2
    if (top) {
        for (int i = 0; i < 4; ++i)
            if (P.p_out[13 - i] != i) return false;
    } else {
        for (int i = 0; i < 3; ++i)
            if (P.p_out[i] != i) return false;
    }
    // tile-coordinate wires in input address order -> segments
    std::vector<int> nt;
    for (int adr = 0; adr < na; ++adr)
        if (!in_tile[wire_at[adr]]) nt.push_back(wire_at[adr]);
    P.nseg = 0;
    for (int m = 0; m < static_cast<int>(nt.size());) {
        int len = 1, dir = 0;
        while (m + len < static_cast<int>(nt.size()) && nt[m + len] == nt[m + len - 1] + 1) {
            const int d = Lout[nt[m + len]] - Lout[nt[m + len - 1]];
            if (d != 1 && d != -1) break;
            if (dir == 0) dir = d;
            else if (d != dir) break;
            ++len;
        }
        if (P.nseg >= kMaxSegs) return false;
        TileSeg& S = P.seg[P.nseg++];
        S.src = m;
        S.len = len;
        S.wire = nt[m];
        S.out = Lout[nt[m]];
        S.out_rev = dir < 0 ? 1 : 0;
        m += len;
    }
    // TMA dimensions: x0..x3, then runs of x bits at consecutive addresses (<= 8 bits), then
    // the tile-coordinate address runs
    int nd = 0;
    auto add_dim = [&](int len, int adr, int src, bool tile_dim) -> bool {
        if (nd >= kMaxDims) return false;
        ph.gdim[nd] = cuuint64_t(1) << len;
        ph.box[nd] = tile_dim ? (cuuint32_t(1) << len) : 1;
        if (nd > 0) ph.gstride[nd - 1] = (cuuint64_t(1) << adr) * 8;
        P.dim_src[nd] = tile_dim ? 0 : src;
        P.dim_len[nd] = tile_dim ? 0 : len;
        P.dim_scale[nd] = 1;
        ++nd;
        return true;
    };
    if (!add_dim(4, 0, 0, true)) return false;
    for (int b = 4; b < 14;) {
        int len = 1;
        while (b + len < 14 && len < 8 && Lin[xw[b + len]] == Lin[xw[b + len - 1]] + 1) ++len;
        if (!add_dim(len, Lin[xw[b]], 0, true)) return false;
        b += len;
    }
    for (int m = 0; m < static_cast<int>(nt.size());) {
        int len = 1;
        while (m + len < static_cast<int>(nt.size()) && Lin[nt[m + len]] == Lin[nt[m + len - 1]] + 1) ++len;
        if (!add_dim(len, Lin[nt[m]], m, false)) return false;
        m += len;
    }
    P.ndims = nd;
    for (int d = nd; d < kMaxDims; ++d) {
        ph.gdim[d] = 1;
        ph.box[d] = 1;
        ph.gstride[d - 1] = (cuuint64_t(1) << na) * 8;
        P.dim_src[d] = 0;
        P.dim_len[d] = 0;
        P.dim_scale[d] = 1;
    }
    P.load_mode = 0;
    ph.run_bits = 0;
    while (ph.run_bits < na && in_tile[wire_at[ph.run_bits]]) ++ph.run_bits;
    // the two register stages (also read by describe_pass and the CPU plan checks)
    const int rr[2] = {r0, r1}, qq[2] = {9 + E0, 4 + E1}, wl[2] = {glo + r1, glo};
    P.nstages = 2;
    int ntab = 0;
    for (int s = 0; s < 2; ++s) {
        StageDesc& S = P.st[s];
        S.r = rr[s];
        S.wlo = wl[s];
        S.q = qq[s];
        const int hi = S.wlo + S.r - 1;
        S.cross = hi < n - 1 ? 1 : 0;
        S.ngbits = 14 - S.r;
        S.tile_above = 0;
        for (int w : nt)
            if (w > hi && w < n) S.tile_above = 1;  // wires >= n: batch index, no phase
        S.uoff = s ? r0 : 0;
        int i = 0;
        for (int b = 0; b < 14; ++b)
            if (b < S.q || b >= S.q + S.r) S.gpos[i++] = b;
        S.lo_tw = S.hi_tw = 0;
        for (int g = 0; g < S.ngbits; ++g)
            if (P.p_wire[S.gpos[g]] > hi && P.p_wire[S.gpos[g]] < n) (g < 5 ? S.lo_tw : S.hi_tw) = 1;
        if (!S.lo_tw && !S.hi_tw) S.hi_tw = 1;
        P.tab_off[s] = ntab;
        ntab += 32 + (1 << (S.ngbits - 5));
    }
    P.ntab = ntab;
    P.nU = r0 + r1;
    P.ntw = std::max(r0, r1);
    ph.smem = kWideSmem;
    ph.minb = 1;
    ph.grid = static_cast<int>(std::min<int64_t>(P.num_tiles, pl->num_sms));
    ph.wide = 1;
    ph.wide_r0 = r0;
    ph.wide_r1 = r1;
    ph.wide_top = top ? 1 : 0;
    WideParams& W = ph.wp;
    std::memset(&W, 0, sizeof(W));
    W.n = n;
    W.kk = pl->kk;
    W.first = first;
    W.last = last;
    W.wlo0 = glo + r1;
    W.wlo1 = glo;
    W.l2_prefetch = pl->l2_prefetch;
    W.num_tiles = P.num_tiles;
    for (int b = 0; b < 14; ++b) {
        W.p_wire[b] = P.p_wire[b];
        W.p_out[b] = P.p_out[b];
    }
    W.nseg = P.nseg;
    for (int g = 0; g < kMaxSegs; ++g) W.seg[g] = P.seg[g];
    for (int d = 0; d < kMaxDims; ++d) {
        W.dim_src[d] = P.dim_src[d];
        W.dim_len[d] = P.dim_len[d];
    }
    for (int j = 0; j < 32; ++j) {
        int64_t o = 0;
        for (int e = 0; e < 5; ++e)
            if ((j >> e) & 1) o += int64_t(1) << P.p_out[4 + e];
        W.oj[j] = o;
    }
    W.inv_root_n = P.inv_root_n;
    return true;
}

int plan_passes_wide_split(qft_plan_s* pl, const std::vector<int>& a);

// Natural-order complex64 plans on wide passes: P = ceil(n / 10) passes of
// 7..10 wires each; the first pass moves the 4 top wires to the lowest
// addresses (layout L1 below), the middle passes run in place on L1, the
// last pass writes the bit-reversed order.  Also subset plans on the low n
// of n_addr address bits (w0 = 0): the upper wires keep their addresses in
// every layout and act as a batch index (the kernel's phases read the
// transform's n wires only).
int plan_passes_wide(qft_plan_s* pl) {
    const int n = pl->n;
    if (pl->dtype != QFT_C64 || pl->order != QFT_ORDER_NATURAL || pl->w0 != 0 || pl->precision) return QFT_ERR_UNSUPPORTED;
    const int P = std::max(2, (n + 9) / 10);
    if (P > kMaxPasses) return QFT_ERR_UNSUPPORTED;
    // Pass widths: as even as possible.  The wider passes go first; if a pass
    // of that split has no wide shape, the wider passes are tried at the end
    // instead, then in the middle.
    std::vector<std::vector<int>> splits;
    {
        std::vector<int> a(P, n / P);
        const int extra = n % P;
        for (int j = 0; j < extra; ++j) a[j] += 1;
        splits.push_back(a);
        std::vector<int> b(P, n / P);
        for (int j = 0; j < extra; ++j) b[P - 1 - j] += 1;
        splits.push_back(b);
        std::vector<int> c(P, n / P);
        for (int j = 0; j < extra; ++j) c[1 + j % (P > 2 ? P - 2 : 1)] += 1;
        splits.push_back(c);
    }
    for (const auto& a : splits) {
        const int rc = plan_passes_wide_split(pl, a);
        if (rc == QFT_OK) return rc;
        pl->passes.clear();
    }
    return QFT_ERR_UNSUPPORTED;
}

int plan_passes_wide_split(qft_plan_s* pl, const std::vector<int>& a) {
    const int n = pl->n;
    const int P = static_cast<int>(a.size());
    for (int j = 0; j < P; ++j)
        if (a[j] < 7 || a[j] > 10) return QFT_ERR_UNSUPPORTED;
    if (n - a[0] < 4) return QFT_ERR_UNSUPPORTED;
    std::vector<int> glo(P);
    {
        int t = n;
        for (int j = 0; j < P; ++j) { t -= a[j]; glo[j] = t; }
    }
    const int na = pl->n_addr;
    std::vector<int> ident(na), brev(na), L1(na);
    for (int w = 0; w < na; ++w) {
        ident[w] = w;
        brev[w] = w < n ? n - 1 - w : w;
        L1[w] = w;
    }
    // Layout between the passes: the 4 top wires reversed at addresses 0..3
    // (the batch bits of the later passes, already where the bit reversal
    // puts them), every other wire shifted up by 4.  The first pass then
    // writes 256-byte runs (its batch wires 0..3 and top wires land on
    // addresses 0..7), and each later pass's wires sit on consecutive
    // addresses -- the last pass's tile is one contiguous 128 KiB block.
    for (int w = 0; w < n - 4; ++w) L1[w] = w + 4;
    for (int e = 0; e < 4; ++e) L1[n - 1 - e] = e;
    for (int j = 0; j < P; ++j) {
        const bool first = j == 0, last = j == P - 1;
        const std::vector<int>& Lin = first ? ident : L1;
        const std::vector<int>& Lout = last ? brev : L1;
        PassHost ph;
        bool ok = false;
        for (int r0 = 5; r0 >= 4 && !ok; --r0)
            for (int mode = 0; mode < 3 && !ok; ++mode)
                ok = build_pass_wide(pl, ph, glo[j], a[j], r0, Lin, Lout, first, last, first, mode);
        if (!ok) return QFT_ERR_UNSUPPORTED;
        ph.in_buf = first ? 0 : 1;
        ph.out_buf = last ? 0 : 1;
        pl->passes.push_back(ph);
    }
    const int g1 = pl->passes[0].grid;
    if (g1 > kMaxPartials) return QFT_ERR_UNSUPPORTED;
    pl->passes.back().prm.npartials = g1;
    pl->passes.back().wp.npartials = g1;
    return QFT_OK;
}

int plan_passes_subset(qft_plan_s* pl);

// The split of n wires into P passes of <= cap wires (the last >= cmin) with
// the fewest register stages of <= rmax wires in all, the wider passes first
// among equals; a holds a valid split on entry and the best one on return.
// Returns its stage count.
int df_stage_split(int n, int P, int cap, int cmin, int rmax, std::vector<int>& a) {
    auto stages = [&](const std::vector<int>& v) {
        int t = 0;
        for (int x : v) t += (x + rmax - 1) / rmax;
        return t;
    };
    std::vector<int> cur(P), best = a;
    int best_st = stages(a);
    std::function<void(int, int)> rec = [&](int j, int left) {
        if (j == P - 1) {
            if (left < std::min(cmin, n) || left > cap) return;
            cur[j] = left;
            const int st = stages(cur);
            if (st < best_st || (st == best_st && cur > best)) {
                best_st = st;
                best = cur;
            }
            return;
        }
        for (int x = std::min(cap, left - 1); x >= 1; --x) {
            cur[j] = x;
            rec(j + 1, left - x);
        }
    };
    rec(0, n);
    a = best;
    return best_st;
}

// The whole register, or (subset plans with w0 = 0) its low n bits with the
// bits above as a batch index: logical wires n .. n_addr-1 stay at their own
// addresses in every map.
int plan_passes(qft_plan_s* pl) {
    if (pl->w0 != 0) return plan_passes_subset(pl);
    if (pl->wide_tiles) {
        const int rc = plan_passes_wide(pl);
        if (rc == QFT_OK || pl->wide_tiles == 1) return rc;  // 1: asked for (tile_bits = 14); 2: the default
        pl->passes.clear();
    }
    const int n = pl->n, na = pl->n_addr;
    std::vector<int> ident(na);
    for (int w = 0; w < na; ++w) ident[w] = w;
    std::vector<int> brev = ident;
    for (int w = 0; w < n; ++w) brev[w] = n - 1 - w;
    const bool natural = pl->order == QFT_ORDER_NATURAL;

    if (n <= (pl->precision ? std::min(pl->rmax, 6) : pl->TB)) {  // a single pass: 2J <= 128 rows
        PassHost ph;
        if (!build_pass(pl, ph, 0, n, {}, ident, natural ? brev : ident, true, true)) return QFT_ERR_UNSUPPORTED;
        ph.prm.load_mode = 1;
        ph.in_buf = ph.out_buf = 0;
        pl->passes.push_back(ph);
        return QFT_OK;
    }
    if (natural && pl->df && pl->rmax <= 3 && !pl->shape_given && pl->cmin >= 3) {
        // double-float plans pay per register stage and per pass: one
        // coalescing bit less (64-byte HBM runs; the kernel is bound by its
        // arithmetic, not HBM) where that saves a pass without adding a stage
        // (n = 28: 3 passes of 10 / 9 / 9 wires in 10 stages instead of 4)
        auto even = [&](int P) {
            std::vector<int> v(P, n / P);
            for (int j = 0; j < n % P; ++j) v[j] += 1;
            return v;
        };
        const int cap1 = pl->TB - pl->cmin, cap2 = cap1 + 1;
        const int P1 = (n + cap1 - 1) / cap1, P2 = (n + cap2 - 1) / cap2;
        if (P2 >= 2 && P2 < P1) {
            std::vector<int> v1 = even(P1), v2 = even(P2);
            const int s1 = df_stage_split(n, P1, cap1, pl->cmin, pl->rmax, v1);
            const int s2 = df_stage_split(n, P2, cap2, pl->cmin - 1, pl->rmax, v2);
            if (s2 <= s1) pl->cmin -= 1;
        }
    }
    const int TB = pl->TB, cmin = pl->cmin;
    const int cap = TB - cmin;
    int P;
    std::vector<int> a;
    if (natural) {
        P = (n + cap - 1) / cap;
        if (pl->precision && P < 2) P = 2;  // n = 7 with 7-wire blocks: no single 7-wire pass
        a.assign(P, n / P);
        if (pl->pass_split == 1 && P >= 3) {
            // extra wires to the middle passes first: the first and last
            // passes then keep more batch wires (longer HBM runs, fewer pages
            // touched per tile on the strided side of the bit reversal)
            int extra = n % P;
            for (int j = 1; j < P - 1 && extra > 0; ++j, --extra) a[j] += 1;
            for (int j = 0; j < P && extra > 0; j += P - 1, --extra) a[j] += 1;
        } else {
            for (int j = 0; j < n % P; ++j) a[j] += 1;
        }
        if (pl->df && pl->rmax <= 3 && P >= 2) {
            // double-float plans with blocks of <= 3 wires (512 threads, or
            // 256 threads two CTAs per SM) are
            // bound by the arithmetic per register stage (cross twiddles,
            // shared-memory round trips, barriers):
            // the pass widths with the fewest stages in all (multiples of the
            // stage size where possible; every pass >= cmin wires so the last
            // pass keeps full HBM runs), the wider passes first
            df_stage_split(n, P, cap, cmin, pl->rmax, a);
        }
    } else if (pl->precision) {
        // tensor tier: every pass is one block of <= cap wires
        P = (n + cap - 1) / cap;
        if (P < 2) P = 2;
        a.assign(P, n / P);
        for (int j = 0; j < n % P; ++j) a[j] += 1;
    } else {
        P = 1 + (n - TB + cap - 1) / cap;
        if (P < 2) P = 2;
        a.assign(P, n / P);
        for (int j = 0; j < n % P; ++j) a[j] += 1;
        // the last pass (contiguous, no batch wires) may hold up to TB wires
        for (int j = 0; j < P - 1; ++j) {
            while (a[j] > cap) { a[j]--; a[P - 1]++; }
        }
        if (a[P - 1] > TB) return QFT_ERR_UNSUPPORTED;
    }
    if (P > kMaxPasses) return QFT_ERR_UNSUPPORTED;
    for (int j = 0; j < P; ++j)
        if (a[j] > cap + (natural || j < P - 1 ? 0 : cmin) || a[j] < 1) return QFT_ERR_UNSUPPORTED;

    std::vector<int> glo(P);
    {
        int top = n;
        for (int j = 0; j < P; ++j) { top -= a[j]; glo[j] = top; }
    }
    const int c1 = std::min(TB - a[0], glo[0]);
    int ctop = 0, shift = 0;
    std::vector<int> L1 = ident;
    if (natural) {
        ctop = std::min({c1, a[0], TB - a[P - 1], a[P - 1]});
        // pass_split: the first pass keeps its extra batch wires on the input
        // side, and the top wires moved low stay at the coalescing minimum so
        // the last pass's wires keep forming as few blocks as possible
        if (pl->pass_split == 1) ctop = std::min(ctop, pl->cmin);
        if (ctop < 1) return QFT_ERR_UNSUPPORTED;
        if ((pl->precision || (pl->df && pl->rmax <= 3)) && ctop < a[P - 1]) {
            // the last pass's wires on consecutive addresses, so that they
            // form as few blocks as possible (the tensor-core tier runs one
            // block per pass; double-float plans pay per register stage): the
            // top wires go (reversed) to the lowest addresses and every other
            // wire moves up by ctop
            shift = ctop;
            for (int w = 0; w < n - ctop; ++w) L1[w] = w + ctop;
            for (int e = 0; e < ctop; ++e) L1[n - 1 - e] = e;
        } else {
            for (int e = 0; e < ctop; ++e) {
                L1[n - 1 - e] = e;           // top wires to the lowest addresses (their final place)
                L1[e] = n - ctop + e;        // lowest wires to the top
            }
        }
    }
    for (int j = 0; j < P; ++j) {
        PassHost ph;
        const bool first = j == 0, last = j == P - 1;
        std::vector<int> batch;
        const std::vector<int>& Lin = first ? ident : L1;
        std::vector<int> Lout;
        if (first) {
            for (int w = 0; w < c1; ++w) batch.push_back(w);
            Lout = natural ? L1 : ident;
        } else if (!last) {
            const int cj = std::min(TB - a[j], glo[j] + shift);
            std::vector<int> wat(na);
            for (int w = 0; w < na; ++w) wat[Lin[w]] = w;
            for (int adr = 0; adr < cj; ++adr) batch.push_back(wat[adr]);
            Lout = Lin;
        } else {
            if (natural)
                for (int e = 0; e < ctop; ++e) batch.push_back(n - 1 - e);
            Lout = natural ? brev : ident;
        }
        if (!build_pass(pl, ph, glo[j], a[j], batch, Lin, Lout, first, last)) return QFT_ERR_UNSUPPORTED;
        ph.prm.load_mode = 0;
        if (natural) {
            ph.in_buf = first ? 0 : 1;
            ph.out_buf = last ? 0 : 1;
        } else {
            ph.in_buf = ph.out_buf = 0;
        }
        pl->passes.push_back(ph);
    }
    const int g1 = pl->passes[0].grid;
    if (g1 > kMaxPartials) return QFT_ERR_UNSUPPORTED;
    pl->passes.back().prm.npartials = g1;
    return QFT_OK;
}

// Subset plans (a QFT on index bits [w0, w0 + m) of 2^n_addr amplitudes, for
// every value of the other bits).  Logical wire w < m sits at address
// w0 + w; the other logical wires m, m+1, ... take the remaining addresses in
// increasing order.  NATURAL order reverses the transform's bits only:
// logical w < m leaves through address w0 + m - 1 - w.
//   * One pass when the m wires plus the low batch bits that make the HBM
//     runs fit a tile: each tile holds whole transforms and is rewritten in
//     place.
//   * Several passes when the lowest cmin address bits are batch bits
//     (w0 >= cmin): every pass's tile takes them for its runs, the passes
//     cover the transform's wires top-down, and the layout stays the
//     identity until the last pass (NATURAL: through the workspace buffer,
//     whose last pass writes the reversed addresses; BITREV: in place).
int plan_passes_subset(qft_plan_s* pl) {
    const int n = pl->n_addr, m = pl->n, w0 = pl->w0;
    const bool natural = pl->order == QFT_ORDER_NATURAL;
    std::vector<int> Lin(n), Lout(n);
    {
        int b = m;
        for (int adr = 0; adr < n; ++adr)
            if (adr < w0 || adr >= w0 + m) Lin[b++] = adr;
        for (int w = 0; w < m; ++w) Lin[w] = w0 + w;
        Lout = Lin;
        if (natural)
            for (int w = 0; w < m; ++w) Lout[w] = w0 + m - 1 - w;
    }
    const int TB = pl->TB, cmin = pl->cmin;
    const int low = std::min(w0, cmin);  // low batch bits a single-pass tile needs for its runs
    if (m + low <= TB) {
        PassHost ph;
        if (!build_pass(pl, ph, 0, m, {}, Lin, Lout, true, true)) return QFT_ERR_UNSUPPORTED;
        ph.prm.load_mode = ph.run_bits >= ph.prm.tb ? 1 : 0;  // tiles that are address bits 0 .. tb-1: 1D copies
        ph.in_buf = ph.out_buf = 0;
        pl->passes.push_back(ph);
        return QFT_OK;
    }
    if (w0 < cmin) return QFT_ERR_UNSUPPORTED;
    const int cap = TB - cmin;
    const int P = (m + cap - 1) / cap;
    if (P > kMaxPasses) return QFT_ERR_UNSUPPORTED;
    std::vector<int> a(P, m / P);
    for (int j = 0; j < m % P; ++j) a[j] += 1;
    std::vector<int> batch;
    for (int adr = 0; adr < cmin; ++adr) batch.push_back(m + adr);  // logical wires at addresses 0 .. cmin-1
    int top = m;
    for (int j = 0; j < P; ++j) {
        top -= a[j];
        PassHost ph;
        const bool first = j == 0, last = j == P - 1;
        if (!build_pass(pl, ph, top, a[j], batch, Lin, last ? Lout : Lin, first, last)) return QFT_ERR_UNSUPPORTED;
        ph.prm.load_mode = 0;
        if (natural) {
            ph.in_buf = first ? 0 : 1;
            ph.out_buf = last ? 0 : 1;
        } else {
            ph.in_buf = ph.out_buf = 0;
        }
        pl->passes.push_back(ph);
    }
    const int g1 = pl->passes[0].grid;
    if (g1 > kMaxPartials) return QFT_ERR_UNSUPPORTED;
    pl->passes.back().prm.npartials = g1;
    return QFT_OK;
}

// Tensor-core tier: for each pass (one block of r wires) build the block's
// 2^r x 2^r unitary in FP64 by running its gates (unnormalised H on each wire
// from the top, then the controlled phases of distance <= kk, Sec. 2 / Fig. 1)
// on the basis vectors, embed it as the real matrix [[Re, -Im], [Im, Re]],
// pad it to 128 x kpad, and round it on the device to the operand format (hi
// and lo parts).  The matrices are plan-owned device memory.
// Host-only check at plan creation: every pass is one block whose GEMM fits.
int check_tensor_passes(qft_plan_s* pl) {
    for (auto& ph : pl->passes) {
        const PassParams& P = ph.prm;
        if (P.nstages != 1) return QFT_ERR_UNSUPPORTED;
        const int J = 1 << P.st[0].r;
        const int kstep = pl->precision == QFT_PREC_TF32 ? 8 : 16;
        ph.tc_kpad = std::max(kstep, (2 * J + kstep - 1) / kstep * kstep);
        const int ng = 1 << P.st[0].ngbits;
        ph.tc_ncols = std::max(16, (ng + 15) / 16 * 16);
        // 7-wire blocks (2J = 256 > 128 rows) only on the fast kernel, whose
        // B operand carries the real embedding
        if (ph.tc_ncols > 256 || (2 * J > 128 && !tc_fast_pass(P))) return QFT_ERR_UNSUPPORTED;
        ph.smem = tc_smem_bytes(P, pl->precision, ph.tc_kpad, ph.tc_ncols);
        if (ph.smem > 227 * 1024 - 4096) return QFT_ERR_UNSUPPORTED;
        // the tensor-core kernels run one CTA per SM (each holds all 512 TMEM columns)
        ph.minb = 1;
        ph.grid = static_cast<int>(std::min<int64_t>(P.num_tiles, pl->num_sms));
    }
    // the last pass sums one norm partial per CTA of the first pass
    pl->passes.back().prm.npartials = pl->passes[0].grid;
    return QFT_OK;
}

// Device side, once per plan (at its first execute): build and upload the matrices.
int prepare_tensor_passes(qft_plan_s* pl) {
    const double two_pi = 6.283185307179586476925286766559;
    for (auto& ph : pl->passes) {
        if (ph.tc_a_hi) continue;
        const PassParams& P = ph.prm;
        const int r = P.st[0].r;
        const int J = 1 << r;
        const int kpad = ph.tc_kpad;
        std::vector<double> Fre(size_t(J) * J), Fim(size_t(J) * J);
        std::vector<double> vr(J), vi(J);
        for (int ji = 0; ji < J; ++ji) {
            std::fill(vr.begin(), vr.end(), 0.0);
            std::fill(vi.begin(), vi.end(), 0.0);
            vr[ji] = 1.0;
            for (int t = r - 1; t >= 0; --t) {
                const int bit = 1 << t;
                for (int j = 0; j < J; ++j)
                    if (!(j & bit)) {
                        const double ar = vr[j], ai = vi[j], br = vr[j | bit], bi = vi[j | bit];
                        vr[j] = ar + br; vi[j] = ai + bi;
                        vr[j | bit] = ar - br; vi[j | bit] = ai - bi;
                    }
                const int lo = std::max(0, t - pl->kk);
                const int mask = (bit - 1) & ~((1 << lo) - 1);
                for (int j = 0; j < J; ++j)
                    if (j & bit) {
                        const double th = pl->dir * two_pi * static_cast<double>(j & mask) / static_cast<double>(2 * bit);
                        const double c = std::cos(th), s = std::sin(th);
                        const double xr = vr[j] * c - vi[j] * s;
                        vi[j] = vr[j] * s + vi[j] * c;
                        vr[j] = xr;
                    }
            }
            for (int jo = 0; jo < J; ++jo) {
                Fre[size_t(jo) * J + ji] = vr[jo];
                Fim[size_t(jo) * J + ji] = vi[jo];
            }
        }
        std::vector<double> A(size_t(128) * kpad, 0.0);
        for (int jo = 0; jo < J; ++jo)
            for (int ji = 0; ji < J; ++ji) {
                const double fr = Fre[size_t(jo) * J + ji], fi = Fim[size_t(jo) * J + ji];
                if (2 * J > 128) {  // [Re F | Im F]; the kernel's B operand holds [Re x; -Im x] and [Im x; Re x]
                    A[size_t(jo) * kpad + ji] = fr;
                    A[size_t(jo) * kpad + J + ji] = fi;
                    continue;
                }
                A[size_t(jo) * kpad + ji] = fr;
                A[size_t(jo) * kpad + J + ji] = -fi;
                A[size_t(J + jo) * kpad + ji] = fi;
                A[size_t(J + jo) * kpad + J + ji] = fr;
            }
        const size_t eb = pl->precision == QFT_PREC_TF32 ? 4 : 2;
        const size_t abytes = size_t(128) * kpad * eb;
        double* d_src = nullptr;
        cudaError_t e = cudaMalloc(&d_src, A.size() * sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&ph.tc_a_hi, abytes);
        if (e == cudaSuccess) e = cudaMalloc(&ph.tc_a_lo, abytes);
        if (e == cudaSuccess) e = cudaMemcpy(d_src, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = tc_prepare_a(pl->precision, d_src, ph.tc_a_hi, ph.tc_a_lo, kpad, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(d_src);
        if (e != cudaSuccess) {
            cudaFree(ph.tc_a_hi);
            cudaFree(ph.tc_a_lo);
            ph.tc_a_hi = ph.tc_a_lo = nullptr;
            return set_cuda_error(e);
        }
    }
    return QFT_OK;
}

// Tensor maps of every pass for the buffers of one execute: the first pass
// reads `in` (the caller's input; the state itself for in-place execution),
// later passes read the state or the workspace buffer.
int encode_maps(qft_plan_s* pl, const void* in, const void* state, const void* work) {
    if (pl->map_in == in && pl->map_state == state && pl->map_work == work && !pl->maps.empty()) return QFT_OK;
    auto fn = get_encode_fn();
    pl->maps.assign(pl->passes.size(), CUtensorMap{});
    for (size_t i = 0; i < pl->passes.size(); ++i) {
        PassHost& ph = pl->passes[i];
        if (ph.prm.load_mode == 1) continue;
        if (!fn) return cuda_fail(cudaErrorNotSupported);
        const void* base = ph.in_buf == 0 ? (i == 0 ? in : state) : work;
        const cuuint32_t estride[5] = {1, 1, 1, 1, 1};
        CUresult r = fn(&pl->maps[i], CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, const_cast<void*>(base), ph.gdim,
                        ph.gstride, ph.box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        ph.wide ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            qft::set_cuda_error_code(static_cast<int>(r));
            pl->maps.clear();
            return QFT_ERR_CUDA;
        }
    }
    pl->map_in = in;
    pl->map_state = state;
    pl->map_work = work;
    return QFT_OK;
}

}  // namespace

extern "C" {

int qft_version(void) { return 200; }  // 0.2.0: double-float complex128, real, subset and phase-estimation calls, qft_opts.pass_split

int qft_last_cuda_error(void) { return qft::g_last_cuda; }

const char* qft_strerror(int code) {
    switch (code) {
        case QFT_OK: return "ok";
        case QFT_ERR_BAD_ARG: return "invalid argument";
        case QFT_ERR_SIZE: return "length is zero or not a power of two";
        case QFT_ERR_BUDGET: return "request exceeds the HBM admission budget";
        case QFT_ERR_CUDA: return "CUDA call failed";
        case QFT_ERR_TIMEOUT: return "bounded wait expired";
        case QFT_ERR_NOMEM: return "out of memory";
        case QFT_ERR_UNSUPPORTED: return "unsupported configuration";
        case QFT_ERR_STATE: return "call out of order";
        case QFT_ERR_CANCELED: return "request canceled";
        default: return "unknown error";
    }
}

}  // extern "C"

namespace {

// Plan of an n-wire QFT on index bits [w0, w0 + n) of 2^n_addr amplitudes.
int create_plan(qft_plan_t* out, int n_addr, int w0, int n, int k, int direction, int dtype, const qft_opts* opts) {
    if (!out) return QFT_ERR_BAD_ARG;
    *out = nullptr;
    if (dtype != QFT_C64 && dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    if (direction != QFT_FORWARD && direction != QFT_INVERSE) return QFT_ERR_BAD_ARG;
    const int nmax = dtype == QFT_C64 ? 34 : 33;
    if (n < 1 || w0 < 0 || n_addr > nmax || w0 + n > n_addr) return QFT_ERR_BAD_ARG;
    const bool subset = n_addr != n;
    if (subset && opts && opts->precision != QFT_PREC_NATIVE && opts->precision != QFT_PREC_FP64)
        return QFT_ERR_UNSUPPORTED;
    qft_plan_s* pl = new (std::nothrow) qft_plan_s();
    if (!pl) return QFT_ERR_NOMEM;
    pl->n = n;
    pl->n_addr = n_addr;
    pl->w0 = w0;
    pl->k = k;
    pl->kk = effective_k(n, k);
    pl->dir = direction;
    pl->dtype = dtype;
    pl->esize = dtype == QFT_C64 ? 8 : 16;
    pl->TB = dtype == QFT_C64 ? 13 : 12;
    pl->cmin = dtype == QFT_C64 ? 4 : 3;  // HBM runs of >= 128 bytes
    pl->rmax = kMaxStageR;
    pl->threads = 256;
    bool rmax_given = false;
    bool fp64 = false;
    if (opts) {
        if (opts->order != QFT_ORDER_NATURAL && opts->order != QFT_ORDER_BITREV) { delete pl; return QFT_ERR_BAD_ARG; }
        pl->order = opts->order;
        if (opts->tile_bits == 14 && dtype == QFT_C64) {
            // the wide pass kernel: natural order, complex64, the CUDA-core path, the whole
            // register or its low n wires (w0 = 0)
            if (opts->order != QFT_ORDER_NATURAL || w0 != 0 || (opts->precision != QFT_PREC_NATIVE) ||
                opts->threads || opts->max_stage_bits || opts->coalesce_bits) {
                delete pl;
                return QFT_ERR_UNSUPPORTED;
            }
            pl->wide_tiles = n >= 14 ? 1 : 0;
        } else if (opts->tile_bits) {
            if (opts->tile_bits < 4 || opts->tile_bits > (dtype == QFT_C64 ? 13 : 12)) { delete pl; return QFT_ERR_BAD_ARG; }
            pl->TB = opts->tile_bits;
        }
        // small tiles keep at least 3 transform wires per pass unless told otherwise
        if (opts->tile_bits && opts->tile_bits <= 13 && !opts->coalesce_bits) pl->cmin = std::min(pl->cmin, std::max(1, pl->TB - 3));
        if (opts->coalesce_bits) {
            if (opts->coalesce_bits < 1 || opts->coalesce_bits > 6) { delete pl; return QFT_ERR_BAD_ARG; }
            pl->cmin = opts->coalesce_bits;
        }
        if (opts->precision < QFT_PREC_NATIVE || opts->precision > QFT_PREC_FP64) { delete pl; return QFT_ERR_BAD_ARG; }
        if (opts->precision == QFT_PREC_FP64) {
            if (dtype != QFT_C128) { delete pl; return QFT_ERR_UNSUPPORTED; }
            fp64 = true;
        } else if (opts->precision != QFT_PREC_NATIVE) {
            if (dtype != QFT_C64) { delete pl; return QFT_ERR_UNSUPPORTED; }
            pl->precision = opts->precision;
            // one fused block of <= f wires per pass, f = max_stage_bits (4..7;
            // 0 = 6): 2^12-amplitude tiles for f = 5, 6 (2^(12-r) GEMM columns
            // per r-wire block); 2^11 for f = 7, whose operands need the shared
            // memory of the other half, and for f = 4, whose 3-wire blocks
            // would otherwise exceed the 256 columns of one MMA
            const int f = opts->max_stage_bits ? opts->max_stage_bits : 6;
            if (f < 4 || f > 7) { delete pl; return QFT_ERR_BAD_ARG; }
            pl->TB = (f == 7 || f == 4) ? 11 : 12;
            pl->cmin = pl->TB - f;
            pl->rmax = f;
        }
        if (opts->wait_limit_ms < 0) { delete pl; return QFT_ERR_BAD_ARG; }
        if (opts->wait_limit_ms) pl->wait_limit_ns = uint64_t(opts->wait_limit_ms) * 1000000ull;
        pl->test_skip_first_load = opts->test_skip_first_load ? 1 : 0;
        if (opts->threads) {
            if (opts->threads != 256 && opts->threads != 512) { delete pl; return QFT_ERR_BAD_ARG; }
            pl->threads = opts->threads;
            if (pl->threads == 512) pl->rmax = 4;
        }
        // packed FP32x2 paired stages measured slower than one group per thread
        // on GB300 in every shape and were removed; the field stays for the ABI
        if (opts->paired) { delete pl; return QFT_ERR_UNSUPPORTED; }
        if (opts->pass_split < 0 || opts->pass_split > 2) { delete pl; return QFT_ERR_BAD_ARG; }
        pl->pass_split = opts->pass_split == 1 ? 1 : 0;
        if (opts->max_stage_bits && !pl->precision) {
            rmax_given = true;
            if (opts->max_stage_bits < 1 || opts->max_stage_bits > (pl->threads == 512 ? 4 : kMaxStageR)) {
                delete pl;
                return QFT_ERR_BAD_ARG;
            }
            pl->rmax = opts->max_stage_bits;
        }
    }
    // Shapes measured fastest on GB300 (the autotuner's choices), used when the
    // caller leaves the knobs at 0: complex64 with n >= 27 takes 2^12-amplitude
    // tiles (two CTAs per SM) with the left-over wires on the middle passes;
    // double-float complex128 with n >= 21 takes 512 threads.
    // (For subset plans the array size decides: their passes sweep all of it.)
    const bool shape_given = opts && (opts->tile_bits || opts->coalesce_bits || opts->threads || rmax_given);
    pl->shape_given = shape_given;
    if (!shape_given && dtype == QFT_C64 && !pl->precision && n_addr >= 27) {
        pl->TB = 12;
        pl->cmin = 4;
        if (!(opts && opts->pass_split)) pl->pass_split = 1;
    }
    if (!shape_given && dtype == QFT_C128 && !fp64 && n_addr >= 21) pl->threads = 512;
    // complex64, natural order, arrays of >= 2^23 amplitudes (the whole register,
    // or a transform of >= 14 wires on its low bits): the wide pass kernel where
    // the planner finds wide shapes (2^14-amplitude tiles, so ceil(n / 10)
    // passes), else the shapes above.
    if (!shape_given && dtype == QFT_C64 && !pl->precision && w0 == 0 && pl->order == QFT_ORDER_NATURAL &&
        n >= 14 && n_addr >= 23)
        pl->wide_tiles = 2;
    // complex64 tiles of <= 2^12 amplitudes fit two CTAs per SM; blocks of <= 4
    // wires keep the kernel within the 128 registers that needs.
    if (dtype == QFT_C64 && !pl->precision && pl->threads == 256 && pl->TB <= 12 && !rmax_given)
        pl->rmax = std::min(pl->rmax, 4);
    // complex128 runs in double-float unless FP64 was asked for: 256 threads
    // with blocks of <= 4 wires (16 pair-of-pairs amplitudes per thread in
    // registers), or 512 threads with blocks of <= 3 wires (twice the warps).
    if (dtype == QFT_C128 && !fp64) {
        pl->df = true;
        pl->rmax = std::min(pl->rmax, pl->threads == 512 ? 3 : 4);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            pl->num_sms = sms;
    } else {
        cudaGetLastError();
    }
    // gate counters before fusion (Table 2)
    pl->n_h = n;
    pl->n_cp = 0;
    for (int t = n - 1; t >= 0; --t) pl->n_cp += std::min(pl->kk, t);
    pl->n_swap = n / 2;
    int rc = plan_passes(pl);
    if (rc == QFT_OK && pl->precision) rc = check_tensor_passes(pl);
    if (rc != QFT_OK) {
        delete pl;
        return rc;
    }
    const size_t N = size_t(1) << n_addr;
    const bool need_work = pl->order == QFT_ORDER_NATURAL && pl->passes.size() > 1;
    pl->ws_bytes = kMetaBytes + (need_work ? N * pl->esize : 0);
    *out = pl;
    return QFT_OK;
}

}  // namespace

extern "C" {

int qft_plan_create(qft_plan_t* out, int n, int k, int direction, int dtype, const qft_opts* opts) {
    return create_plan(out, n, 0, n, k, direction, dtype, opts);
}

int qft_plan_create_subset(qft_plan_t* out, int n_addr, int w0, int n, int k, int direction, int dtype,
                           const qft_opts* opts) {
    return create_plan(out, n_addr, w0, n, k, direction, dtype, opts);
}

int qft_plan_destroy(qft_plan_t plan) {
    delete plan;
    return QFT_OK;
}

int qft_plan_get_info(qft_plan_t pl, qft_plan_info* info) {
    if (!pl || !info) return QFT_ERR_BAD_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n = pl->n;
    info->k_eff = pl->kk;
    info->direction = pl->dir;
    info->dtype = pl->dtype;
    info->order = pl->order;
    info->n_h = pl->n_h;
    info->n_cp = pl->n_cp;
    info->n_swap = pl->n_swap;
    info->passes = static_cast<int>(pl->passes.size());
    for (size_t i = 0; i < pl->passes.size() && i < 8; ++i) {
        const PassHost& ph = pl->passes[i];
        info->wires_per_pass[i] = ph.wires;
        info->stages_per_pass[i] = ph.prm.nstages;
        info->tile_bits[i] = ph.prm.tb;
        info->coalesce_bits[i] = ph.run_bits;
    }
    info->workspace_bytes = pl->ws_bytes;
    info->bytes_per_execute = static_cast<long long>(pl->passes.size()) * 2LL * (1LL << pl->n_addr) * static_cast<long long>(pl->esize);
    info->n_addr = pl->n_addr;
    info->w0 = pl->w0;
    for (const PassHost& ph : pl->passes)
        for (int s = 0; s < ph.prm.nstages; ++s) {
            info->fused_blocks += 1;
            info->max_fused_size = std::max(info->max_fused_size, static_cast<int>(ph.prm.st[s].r));
        }
    return QFT_OK;
}

size_t qft_workspace_size(qft_plan_t pl) { return pl ? pl->ws_bytes : 0; }

int qft_load(qft_plan_t pl, void* d_state, const void* src, size_t len, int src_on_device, qft_stream_t stream) {
    if (!pl || !d_state || !src) return QFT_ERR_BAD_ARG;
    if (len != (size_t(1) << pl->n_addr)) return QFT_ERR_SIZE;
    if (src == d_state) return QFT_OK;
    cudaError_t e = cudaMemcpyAsync(d_state, src, len * pl->esize,
                                    src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QFT_OK : cuda_fail(e);
}

int qft_load_padded(qft_plan_t pl, void* d_state, const void* src, size_t len, int src_on_device,
                    qft_stream_t stream) {
    if (!pl || !d_state || (!src && len)) return QFT_ERR_BAD_ARG;
    const size_t N = size_t(1) << pl->n_addr;
    if (len > N) return QFT_ERR_SIZE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* dst = static_cast<char*>(d_state);
    cudaError_t e = cudaSuccess;
    if (len && src != d_state)
        e = cudaMemcpyAsync(dst, src, len * pl->esize, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                            st);
    if (e == cudaSuccess && len < N) e = cudaMemsetAsync(dst + len * pl->esize, 0, (N - len) * pl->esize, st);
    return e == cudaSuccess ? QFT_OK : cuda_fail(e);
}

int qft_read(qft_plan_t pl, const void* d_state, void* dst, int dst_on_device, qft_stream_t stream) {
    if (!pl || !d_state || !dst) return QFT_ERR_BAD_ARG;
    if (dst == d_state) return QFT_OK;
    cudaError_t e = cudaMemcpyAsync(dst, d_state, (size_t(1) << pl->n_addr) * pl->esize,
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    reinterpret_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? QFT_OK : cuda_fail(e);
}

namespace {
// Passes [i0, i1) of one execute.  The first pass reads d_in (d_state for an
// in-place transform); the result lands in d_state.
int execute_range(qft_plan_t pl, const void* d_in, void* d_state, void* d_workspace, double* d_scale_in,
                  int scale_mode, qft_stream_t stream, size_t i0, size_t i1) {
    if (!pl || !d_in || !d_state || !d_workspace) return QFT_ERR_BAD_ARG;
    if (scale_mode < QFT_SCALE_STATE || scale_mode > QFT_SCALE_INV_N) return QFT_ERR_BAD_ARG;
    // a subset plan runs many transforms at once: there is no one state to normalise
    if (pl->n_addr != pl->n && scale_mode == QFT_SCALE_STATE) return QFT_ERR_BAD_ARG;
    if ((reinterpret_cast<uintptr_t>(d_state) & 255) || (reinterpret_cast<uintptr_t>(d_workspace) & 255) ||
        (reinterpret_cast<uintptr_t>(d_in) & 255))
        return QFT_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    char* ws = static_cast<char*>(d_workspace);
    void* work = ws + kMetaBytes;
    std::lock_guard<std::mutex> lock(pl->mu);
    if (pl->precision && !pl->passes[0].tc_a_hi) {
        const int prc = prepare_tensor_passes(pl);
        if (prc != QFT_OK) return prc;
    }
    int rc = encode_maps(pl, d_in, d_state, work);
    if (rc != QFT_OK) return rc;
    cudaError_t e = cudaSuccess;
    if (i0 == 0) {
        // status word and (double-float plans) the maximum exponent of the input
        e = cudaMemsetAsync(ws + kStatusOff, 0, kMaxExpOff + sizeof(int32_t) - kStatusOff, st);
        if (e != cudaSuccess) return cuda_fail(e);
        if (pl->df) {
            e = launch_df_maxexp(d_in, size_t(1) << pl->n_addr, reinterpret_cast<int*>(ws + kMaxExpOff), pl->num_sms,
                                 st);
            if (e != cudaSuccess) return cuda_fail(e);
        }
    }
    // One NVTX range per execute and one per pass (host-side markers a profiler
    // lines up with the pass kernels; no cost without a tool attached).
    static const char* const kPassNames[kMaxPasses] = {"qft pass 1", "qft pass 2", "qft pass 3", "qft pass 4",
                                                       "qft pass 5", "qft pass 6", "qft pass 7", "qft pass 8"};
    nvtxRangePushA(pl->df ? "qft execute (complex128, double-float)" : "qft execute");
    struct RangePop {
        ~RangePop() { nvtxRangePop(); }
    } pop_execute;
    for (size_t i = i0; i < i1; ++i) {
        PassHost& ph = pl->passes[i];
        PassParams P = ph.prm;
        nvtxRangePushA(kPassNames[i < kMaxPasses ? i : kMaxPasses - 1]);
        RangePop pop_pass;
        P.scale_mode = scale_mode;
        P.in = ph.in_buf == 0 ? (i == 0 ? d_in : static_cast<const void*>(d_state)) : work;
        P.out = ph.out_buf == 0 ? d_state : work;
        P.partials = reinterpret_cast<double*>(ws + kPartialOff);
        P.meta = reinterpret_cast<double*>(ws);
        P.user_scale = d_scale_in;
        P.status = reinterpret_cast<int32_t*>(ws + kStatusOff);
        P.wait_limit_ns = pl->wait_limit_ns;
        P.test_skip_first_load = pl->test_skip_first_load;
        if (ph.wide) {
            WideParams W = ph.wp;
            W.scale_mode = scale_mode;
            W.out = P.out;
            W.partials = P.partials;
            W.npartials = P.npartials;
            W.meta = P.meta;
            W.user_scale = P.user_scale;
            W.status = P.status;
            W.wait_limit_ns = P.wait_limit_ns;
            W.test_skip_first_load = P.test_skip_first_load;
            e = launch_pass_wide(pl->dir, ph.wide_r0, ph.wide_r1, ph.wide_top, pl->maps[i], W, ph.grid, st);
        } else if (pl->precision)
            e = launch_tc_pass(pl->dir, pl->precision, pl->maps[i], P, ph.tc_a_hi, ph.tc_a_lo, ph.tc_kpad,
                               ph.tc_ncols, ph.grid, ph.smem, st);
        else if (pl->df)
            e = launch_pass_df(pl->dir, pl->threads, ph.minb, pl->maps[i], P, ph.grid, ph.smem, st);
        else
            e = launch_pass(pl->dtype, pl->dir, pl->threads, ph.minb, pl->maps[i], P, ph.grid, ph.smem, st);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return QFT_OK;
}
}  // namespace

int qft_execute(qft_plan_t pl, void* d_state, void* d_workspace, double* d_scale_in, int scale_mode,
                qft_stream_t stream) {
    if (!pl) return QFT_ERR_BAD_ARG;
    return execute_range(pl, d_state, d_state, d_workspace, d_scale_in, scale_mode, stream, 0, pl->passes.size());
}

int qft_execute_oop(qft_plan_t pl, const void* d_in, void* d_out, void* d_workspace, double* d_scale_in,
                    int scale_mode, qft_stream_t stream) {
    if (!pl) return QFT_ERR_BAD_ARG;
    return execute_range(pl, d_in, d_out, d_workspace, d_scale_in, scale_mode, stream, 0, pl->passes.size());
}

int qft_execute_pass(qft_plan_t pl, int pass, void* d_state, void* d_workspace, double* d_scale_in,
                     int scale_mode, qft_stream_t stream) {
    if (!pl || pass < 0 || pass >= static_cast<int>(pl->passes.size())) return QFT_ERR_BAD_ARG;
    return execute_range(pl, d_state, d_state, d_workspace, d_scale_in, scale_mode, stream, size_t(pass),
                         size_t(pass) + 1);
}

int qft_plan_describe_pass(qft_plan_t pl, int i, long long* out, int cap) {
    if (!pl || !out || i < 0 || i >= static_cast<int>(pl->passes.size())) return QFT_ERR_BAD_ARG;
    const PassHost& ph = pl->passes[i];
    const PassParams& P = ph.prm;
    std::vector<long long> v;
    v.insert(v.end(), {P.n, P.kk, P.tb, P.nstages, P.first, P.last, P.load_mode, (long long)P.num_tiles});
    for (int s = 0; s < kMaxStages; ++s) {
        const StageDesc& S = P.st[s];
        v.insert(v.end(), {S.wlo, S.r, S.q, S.cross, S.ngbits, S.tile_above, S.uoff});
        for (int e = 0; e < kMaxR; ++e) v.push_back(S.img[e]);
        v.push_back(S.lo_tw);
        v.push_back(S.hi_tw);
        for (int b = 0; b < kMaxTileBits; ++b) v.push_back(S.gpos[b]);
    }
    for (int b = 0; b < kMaxTileBits; ++b) v.push_back(P.p_wire[b]);
    for (int b = 0; b < kMaxTileBits; ++b) v.push_back(P.p_out[b]);
    v.push_back(P.nseg);
    for (int g = 0; g < kMaxSegs; ++g) v.insert(v.end(), {P.seg[g].src, P.seg[g].len, P.seg[g].wire, P.seg[g].out, P.seg[g].out_rev});
    v.push_back(P.ndims);
    for (int d = 0; d < kMaxDims; ++d) v.push_back(P.dim_src[d]);
    for (int d = 0; d < kMaxDims; ++d) v.push_back(P.dim_len[d]);
    for (int d = 0; d < kMaxDims; ++d) v.push_back((long long)ph.gdim[d]);
    for (int d = 0; d < 4; ++d) v.push_back((long long)ph.gstride[d]);
    for (int d = 0; d < kMaxDims; ++d) v.push_back((long long)ph.box[d]);
    v.insert(v.end(), {ph.grid, (long long)ph.smem, ph.in_buf, ph.out_buf, P.npartials, ph.run_bits, P.paired, ph.minb,
                       pl->n_addr, ph.wide});
    for (size_t j = 0; j < v.size() && static_cast<int>(j) < cap; ++j) out[j] = v[j];
    return static_cast<int>(v.size());
}

int qft_get_scale_in(qft_plan_t pl, const void* d_workspace, double* out, qft_stream_t stream) {
    if (!pl || !d_workspace || !out) return QFT_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaMemcpy(out, d_workspace, sizeof(double), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? QFT_OK : cuda_fail(e);
}

int qft_check_status(qft_plan_t pl, const void* d_workspace, qft_stream_t stream) {
    if (!pl || !d_workspace) return QFT_ERR_BAD_ARG;
    cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e);
    int32_t s = 0;
    e = cudaMemcpy(&s, static_cast<const char*>(d_workspace) + kStatusOff, sizeof(s), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    return s;
}

}  // extern "C"
