// plan.hpp -- pass descriptors shared by the host planner (planner.cpp) and the
// pass kernels (qft_pass.cu).  Internal to libqftfft; not part of the C ABI.
//
// Model (Sec. 2-3 of the QFT->FFT paper).  The circuit on n wires processes
// wires t = n-1 .. 0: H(t), then the controlled phases CP(c, t) with
// c = t-d, d = 1..min(k, t), phase e^{s 2 pi i / 2^{d+1}} on |1_c 1_t>.  A
// controlled phase is diagonal and commutes with every H except H(c) and
// H(t), so the circuit regroups exactly into blocks B = [lo, hi] of
// consecutive wires, processed top-down, each being
//   (a) a diagonal "cross" twiddle exp(s 2 pi i phi(I) / 2^n) with
//       phi(I) = sum_{c in B} sum_{t > hi, t-c <= k} I_c I_t 2^{n-1-(t-c)},
//       i.e. the controlled phases whose target was processed earlier and
//       whose control lies in B (Eq. 5 read as a product of two-level
//       updates), followed by
//   (b) the sub-circuit on B: H(t) then CP(c, t) for c in B, t = hi .. lo.
// A block is one register stage: each thread holds the 2^r amplitudes that
// differ only in B's r wires.  A pass is one HBM sweep: a CTA tile holds the
// 2^tb amplitudes that differ in the pass's wire group G (its blocks) plus a
// few "batch" wires that make the HBM runs contiguous.  The qubit-reversal
// swaps are realised as a change of the wire -> address map between the
// input and output of passes (a layout adapter, Sec. 3.1), never as a sweep
// of their own.
#pragma once
#include <cstdint>

namespace qft {

constexpr int kMaxStages = 8;
constexpr int kMaxTileBits = 14;
constexpr int kMaxSegs = 8;
constexpr int kMaxPasses = 8;
constexpr int kMaxDims = 5;
constexpr int kMaxR = 7;       // wires per block (6 and 7 only in the tensor-core tier; table planes)
constexpr int kMaxStageR = 5;  // wires per register stage of the CUDA-core pass kernel
// The pass kernel runs with 256 threads per CTA (register stages of up to 5
// wires) or 512 threads (stages of up to 4 wires).

// One register stage (one fused block of wires).
struct StageDesc {
    int32_t wlo;    // lowest logical wire of the block
    int32_t r;      // wires in the block (1..kMaxR); the block is wires [wlo, wlo + r)
    int32_t q;      // tile index bit that holds wire wlo; the block occupies tile bits [q, q + r)
    int32_t cross;  // 1 if some wire above the block exists (cross twiddle (a) is not identity)
    int32_t ngbits; // tb - r: bits of the group index
    int32_t tile_above;  // 1 if a tile-coordinate wire lies above the block (per-tile twiddle U needed)
    int32_t uoff;        // offset of this stage's r per-tile twiddles in the U table
    int32_t img[kMaxR];  // swizzled buffer-B offset of each register bit (1 << (q + e) mapped)
    int32_t lo_tw;       // 1 if a lane-part tile bit lies above the block (its twiddle table is not all 1)
    int32_t hi_tw;       // 1 if a high-part tile bit lies above the block
    int32_t gpos[kMaxTileBits];  // group-index bit i -> tile index bit (lanes use the low group bits)
};

// A run of tile-coordinate bits [src, src+len) that carry the consecutive
// logical wires [wire, wire+len) and land on output address bits starting at
// out (out_rev = 0: wire+i -> out+i) or ending at out (out_rev = 1:
// wire+i -> out-i).
struct TileSeg {
    int32_t src, len, wire, out, out_rev;
};

struct PassParams {
    int32_t n;          // qubits
    int32_t kk;         // effective AQFT cutoff (n-1 = exact)
    int32_t tb;         // tile bits: amplitudes per tile = 2^tb
    int32_t nstages;
    int32_t first;      // 1: accumulate ||x||^2 of the raw input (stage 0 reads it)
    int32_t last;       // 1: apply the output scale (and publish scale_in)
    int32_t load_mode;  // 0: TMA tensor map; 1: contiguous 1D bulk copy of 2^tb amplitudes per tile
    int32_t scale_mode; // QFT_SCALE_*
    int64_t num_tiles;  // 2^(n - tb)
    StageDesc st[kMaxStages];
    int32_t tab_off[kMaxStages];   // group-table entry offset of each stage (32 lane + high entries)
    int32_t ntab;                  // total group-table entries
    int32_t nU;                    // per-tile twiddles of all stages (sum of r)
    int32_t p_wire[kMaxTileBits];  // tile index bit -> logical wire
    int32_t p_out[kMaxTileBits];   // tile index bit -> output address bit
    int32_t nseg;
    TileSeg seg[kMaxSegs];         // tile coordinate -> logical wires / output address bits
    int32_t ndims;                 // TMA tensor rank (always 5 in the map; unused dims have extent 1)
    int32_t dim_src[kMaxDims];     // TMA box coordinate of dim d = (tile >> dim_src) & (2^dim_len - 1)
    int32_t dim_len[kMaxDims];     //   (dim_len = 0: coordinate 0, a dim inside the tile)
    int32_t dim_scale[kMaxDims];   //   coordinate multiplier (2 for the inner dim of complex128)
    double inv_root_n;             // 2^{-n/2}: the folded 1/sqrt(2) of the n Hadamards
    const void* in;                // bulk mode: state base address (tile t at in + t * 2^tb)
    void* out;                     // output state base
    double* partials;              // first pass writes one partial ||x||^2 per CTA; last pass reads them
    int32_t npartials;             // number of partials the last pass sums
    double* meta;                  // workspace: meta[0] = scale_in
    double* user_scale;            // optional extra copy of scale_in
    int32_t* status;               // workspace status word (bounded waits report here)
    uint64_t wait_limit_ns;        // bound of each tile wait
    int32_t test_skip_first_load;  // test hook: never issue the first load (the wait must expire)
    int32_t paired;                // always 0 (kept so the pass record keeps its layout)
    int32_t ntw;                   // twiddle planes in the group tables (the widest block of the pass)
};

// One tile of one pass of one transform in a batched launch.
// Shared-memory layout of a batched launch: the largest tile (2^max_tb
// amplitudes) sizes buffer B and the nbuf (1 or 2) load buffers; the group
// tables hold max_ntab entries of tw_stride twiddle bytes (the widest block's
// planes) plus offsets.
struct BatchLayout {
    int32_t max_tb;
    int32_t max_ntab;
    int32_t nbuf;
    int32_t tw_stride;
    int32_t threads;  // CTA size of the batch kernel (256 or 512)
};

// Partial-norm slots per first-pass tile in a batch (one per warp, up to 16 warps).
constexpr int kBatchNormSlots = 16;

struct BatchItem {
    int32_t desc;         // index of the transform's PassParams for this pass
    int32_t shape;        // passes with equal shape ids share group tables
    int64_t tile;         // tile index within the pass
    int32_t wait_ctr;     // counter to wait on before loading (-1: none)
    int32_t wait_target;  // value that counter must reach
    int32_t signal_ctr;   // counter to increment when this tile is stored (-1: none)
    int32_t map;          // index of the tensor map (-1: 1D bulk load)
};

// Launch parameters of one pass of the wide kernel (qft_wide.cuh: complex64,
// 2^14-amplitude tiles, two register stages); built by the planner, buffers
// filled per execute.
// Group mode of the wide pass kernel: the last pass keeps the decode scales of
// at most this many tiles per CTA, so a launch has at most this many tiles per SM.
constexpr int kWideGroupTilesPerCta = 512;
// ... and its transforms take at most this many distinct cutoffs k.
constexpr int kWideGroupMaxK = 4;

struct WideParams {
    int32_t n, kk;
    int32_t first, last, scale_mode;
    int32_t wlo0, wlo1;   // lowest wire of the stage-0 (top) and stage-1 blocks
    int32_t l2_prefetch;  // 1: also prefetch the tile after next into L2
    int32_t test_skip_first_load;
    int64_t num_tiles;
    int32_t p_wire[14];  // tile bit x -> logical wire
    int32_t p_out[14];   // tile bit x -> output address bit
    int32_t nseg;
    TileSeg seg[kMaxSegs];          // tile coordinate -> wires / output address bits
    int32_t dim_src[kMaxDims], dim_len[kMaxDims];  // TMA coordinate of dim d from the tile index
    int64_t oj[32];                 // output offset of stage-1 register j (x bits 4..8)
    double inv_root_n;
    void* out;
    double* partials;
    int32_t npartials;
    double* meta;
    double* user_scale;
    int32_t* status;
    uint64_t wait_limit_ns;
    // Group mode (the kernel's GROUP instantiations): one launch runs this pass
    // for G transforms of the same plan; tile s is local tile s & (2^lt_bits - 1)
    // of transform s >> lt_bits (num_tiles = G << lt_bits, lt_bits <= 6).
    int32_t lt_bits;
    const void* maps;         // per transform: the pass's input CUtensorMap (device, 64-byte aligned)
    void* const* outs;        // per transform: the pass's output base (device)
    double* tpart;            // per tile: the first pass's squared-norm sum, read by the last pass
    double* const* gscale;    // per transform: where the last pass stores scale_in (entries may be null)
    // the transforms' cutoffs: transforms [gk_end[i-1], gk_end[i]) have k_eff = gk_val[i] (i < gk_n)
    int32_t gk_n;
    int32_t gk_end[kWideGroupMaxK];
    int32_t gk_val[kWideGroupMaxK];
};

}  // namespace qft
