// qft_tc.cuh -- the precision tier: a pass whose fused block of r <= 7 wires is
// applied as a dense complex GEMM on the 5th-generation tensor cores.
//
// Within one block the circuit is a fixed 2^r x 2^r unitary F (the block's
// Hadamards and controlled phases, Sec. 2 / Fig. 1) applied to every column of
// 2^r amplitudes after that column's cross twiddle (the controlled phases from
// wires above the block, Eq. 5).  The planner builds F in FP64 on the host,
// embeds it as the real matrix [[Re F, -Im F], [Im F, Re F]] (2^{r+1} square,
// padded to M = 128 rows) and rounds it to the tier's operand format, split
// into hi + lo parts for the x3 tiers.  Per tile the kernel
//   1. loads the tile by TMA (as the CUDA-core pass kernel does),
//   2. applies the cross twiddles in FP32 on the CUDA cores, scales each column
//      by a power of two (its largest component near 2^14, so FP16 neither
//      overflows nor loses the low part to subnormals), and writes the column as
//      [Re; Im] into the B operand in shared memory (hi and lo parts),
//   3. issues tcgen05.mma (one elected thread; D = 128 x N FP32 in tensor
//      memory; hi*hi + lo*hi + hi*lo for the split tiers),
//   4. reads D back with tcgen05.ld, undoes the column scale, applies the output
//      scale and stores through the pass's output address map.
// Operand layout: K-major, no swizzle, 8-row x 16-byte core matrices, the K
// neighbour of a core matrix 128 bytes further (leading byte offset) and the
// next group of 8 rows K/kc * 128 bytes further (stride byte offset).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "plan.hpp"
#include "qft_device.cuh"

namespace qft {

// precision tiers (qft_opts.precision)
enum TcPrec { TC_TF32 = 1, TC_BF16 = 2, TC_BF16X3 = 3, TC_FP16 = 4, TC_FP16X3 = 5 };

template <int PREC> struct TcOp;
template <> struct TcOp<TC_TF32> { static constexpr int bytes = 4, kind = 2, fmt = 2, split = 0; };
template <> struct TcOp<TC_BF16> { static constexpr int bytes = 2, kind = 1, fmt = 1, split = 0; };
template <> struct TcOp<TC_BF16X3> { static constexpr int bytes = 2, kind = 1, fmt = 1, split = 1; };
template <> struct TcOp<TC_FP16> { static constexpr int bytes = 2, kind = 1, fmt = 0, split = 0; };
template <> struct TcOp<TC_FP16X3> { static constexpr int bytes = 2, kind = 1, fmt = 0, split = 1; };

// Round x to the operand format; hi = rounded value (stored), returns it as float.
template <int PREC>
__device__ __forceinline__ float store_op(void* dst, float x) {
    if constexpr (PREC == TC_TF32) {
        uint32_t t;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(x));
        *static_cast<uint32_t*>(dst) = t;
        return __uint_as_float(t);
    } else if constexpr (PREC == TC_BF16 || PREC == TC_BF16X3) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        *static_cast<__nv_bfloat16*>(dst) = h;
        return __bfloat162float(h);
    } else {
        const __half h = __float2half_rn(x);
        *static_cast<__half*>(dst) = h;
        return __half2float(h);
    }
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFF) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFF) << 32;
    d |= static_cast<uint64_t>(1) << 46;  // descriptor version; base offset 0; no swizzle
    return d;
}

template <int KIND>
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
    if constexpr (KIND == 2)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
                     "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
    else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
                     "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Byte offset of element (row, k) in a K-major no-swizzle operand with kpad columns.
template <int EB>
__device__ __forceinline__ uint32_t op_offset(int row, int k, int kpad) {
    constexpr int kc = 16 / EB;
    return static_cast<uint32_t>((row >> 3) * (kpad / kc) * 128 + (k / kc) * 128 + (row & 7) * 16 + (k % kc) * EB);
}

struct TcParams {
    const void* a_hi;  // 128 x kpad operand (already in the shared-memory layout), hi part
    const void* a_lo;  // lo part (x3 tiers)
    int32_t kpad;      // K of the GEMM (2^{r+1} rounded up to the MMA K step)
    int32_t ncols;     // N of the GEMM: columns per tile rounded up to a multiple of 16
};

constexpr int kTcThreads = 128;

template <int DIR, int PREC>
__global__ void __launch_bounds__(kTcThreads, 1)
    qft_tc_pass_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ PassParams P,
                       const __grid_constant__ TcParams Q) {
    using V = float2;
    using Op = TcOp<PREC>;
    constexpr int EB = Op::bytes;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar_load, mbar_mma;
    __shared__ uint32_t s_taddr;
    __shared__ double red[kTcThreads / 32];
    __shared__ __align__(16) V Ubuf[kMaxR * kMaxStages];

    const int tid = threadIdx.x;
    const StageDesc& S = P.st[0];
    const int r = S.r;
    const int J = 1 << r;
    const int ng = 1 << S.ngbits;  // columns (groups) of the tile
    const int kpad = Q.kpad, ncols = Q.ncols;
    const uint32_t tile_elems = 1u << P.tb;
    const uint32_t tile_bytes = tile_elems * 8u;
    const size_t a_bytes = static_cast<size_t>(128) * kpad * EB;
    const size_t b_bytes = static_cast<size_t>(ncols) * kpad * EB;
    const uint32_t d_bytes = static_cast<uint32_t>(2 * J) * static_cast<uint32_t>(ncols) * 4u;
    unsigned char* Tb = smem_raw;  // tile, later the D staging area (rows < 2^{r+1})
    unsigned char* A_hi = Tb + (tile_bytes > d_bytes ? tile_bytes : d_bytes);
    unsigned char* A_lo = A_hi + a_bytes;
    unsigned char* B_hi = A_lo + (Op::split ? a_bytes : 0);
    unsigned char* B_lo = B_hi + b_bytes;
    unsigned char* tab_raw = B_lo + (Op::split ? b_bytes : 0);
    int* col_exp = reinterpret_cast<int*>(tab_raw);
    tab_raw += 4 * 256;
    GroupTab<V> tab;
    tab.ntab = P.ntab;
    tab.tw = reinterpret_cast<V*>(tab_raw);
    tab.ob = reinterpret_cast<int64_t*>(tab_raw + kMaxR * sizeof(V) * static_cast<size_t>(P.ntab));
    tab.pb = reinterpret_cast<uint32_t*>(tab_raw + (kMaxR * sizeof(V) + 8) * static_cast<size_t>(P.ntab));
    tab.sb = tab.pb + P.ntab;
    V* T = reinterpret_cast<V*>(Tb);
    float* D = reinterpret_cast<float*>(Tb);

    build_group_tables<float, DIR, kTcThreads>(P, tab);
    // the fixed block matrix (hi, lo) into shared memory
    {
        const uint4* src = static_cast<const uint4*>(Q.a_hi);
        uint4* dst = reinterpret_cast<uint4*>(A_hi);
        for (size_t i = tid; i < a_bytes / 16; i += kTcThreads) dst[i] = src[i];
        if (Op::split) {
            src = static_cast<const uint4*>(Q.a_lo);
            dst = reinterpret_cast<uint4*>(A_lo);
            for (size_t i = tid; i < a_bytes / 16; i += kTcThreads) dst[i] = src[i];
        }
        // zero B once: padding columns (>= ng) stay zero, the others are rewritten per tile
        for (size_t i = tid; i < b_bytes / 16; i += kTcThreads) {
            reinterpret_cast<uint4*>(B_hi)[i] = make_uint4(0, 0, 0, 0);
            if (Op::split) reinterpret_cast<uint4*>(B_lo)[i] = make_uint4(0, 0, 0, 0);
        }
    }
    // One accumulator per K step where tensor memory allows (<= 512 columns):
    // each accumulator then sums only 16 (8 for TF32) products before the
    // accumulators are added pairwise in FP32 on the CUDA cores, which keeps
    // the FP32 accumulation error of the long dot products down.
    uint32_t cols_pow2 = 16;
    while (cols_pow2 < static_cast<uint32_t>(ncols)) cols_pow2 <<= 1;
    const int kstep_n = kpad / (32 / EB);
    int nacc = 1;
    while (nacc * 2 <= kstep_n && cols_pow2 * static_cast<uint32_t>(nacc * 2) <= 512u) nacc *= 2;
    uint32_t tcols = 32;
    while (tcols < cols_pow2 * static_cast<uint32_t>(nacc)) tcols <<= 1;
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&mbar_load, 1);
        mbar_init(&mbar_mma, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;

    float scale = 1.f;
    if (P.last && !P.first) {
        double s = 0.0;
        for (int i = tid; i < P.npartials; i += kTcThreads) s += P.partials[i];
        const double scale_in = sqrt(block_sum<kTcThreads>(s, red));
        scale = static_cast<float>(output_factor(P, scale_in));
        if (blockIdx.x == 0 && tid == 0) {
            P.meta[0] = scale_in;
            if (P.user_scale) *P.user_scale = scale_in;
        }
    }
    const uint32_t idesc = (1u << 4) | (static_cast<uint32_t>(Op::fmt) << 7) | (static_cast<uint32_t>(Op::fmt) << 10) |
                           (static_cast<uint32_t>(ncols >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
    const uint32_t lbo = 128u, sbo = static_cast<uint32_t>(kpad / (16 / EB)) * 128u;
    const int kstep = 32 / EB;
    const uint32_t koff_step = static_cast<uint32_t>(kstep / (16 / EB)) * 128u;

    double norm_acc = 0.0;
    uint32_t ph_load = 0, ph_mma = 0;
    bool aborted = false;
    for (int64_t tile = blockIdx.x; tile < P.num_tiles; tile += gridDim.x) {
        if (tid == 0) {
            fence_proxy_async_smem();
            issue_tile_load(P, &tmap, tile, Tb, &mbar_load, tile_bytes);
        }
        compute_tile_twiddles<float, DIR>(P, tile, Ubuf);
        uint64_t I_tile;
        int64_t out_tile;
        tile_coords(P, tile, I_tile, out_tile);
        const bool ok = mbar_wait_bounded(&mbar_load, ph_load, P.wait_limit_ns);
        ph_load ^= 1u;
        if (__syncthreads_or(!ok)) { aborted = true; break; }
        if (P.first && P.last) {
            double s = 0.0;
            for (uint32_t i = tid; i < tile_elems; i += kTcThreads) {
                const V a = T[i];
                s += static_cast<double>(a.x) * a.x + static_cast<double>(a.y) * a.y;
            }
            const double scale_in = sqrt(block_sum<kTcThreads>(s, red));
            scale = static_cast<float>(output_factor(P, scale_in));
            if (tid == 0) {
                P.meta[0] = scale_in;
                if (P.user_scale) *P.user_scale = scale_in;
            }
        }
        // 2. columns: cross twiddle, column scale, [Re; Im] into B (hi / lo)
        for (int g = tid; g < ng; g += kTcThreads) {
            const int lo5 = P.tab_off[0] + (g & 31), hi5 = P.tab_off[0] + 32 + (g >> 5);
            const uint32_t pb = tab.pb[lo5] | tab.pb[hi5];
            V tau[6];
            for (int e = 0; e < r; ++e) {
                if (S.cross) {
                    V t = cmul(tab.tw[e * tab.ntab + lo5], tab.tw[e * tab.ntab + hi5]);
                    if (S.tile_above) t = cmul(t, Ubuf[S.uoff + e]);
                    tau[e] = t;
                } else {
                    tau[e] = make_float2(1.f, 0.f);
                }
            }
            float amax = 0.f;
            for (int j = 0; j < J; ++j) {
                V x = T[pb + (static_cast<uint32_t>(j) << S.q)];
                if (P.first && !P.last) norm_acc += static_cast<double>(x.x) * x.x + static_cast<double>(x.y) * x.y;
                for (int e = 0; e < r; ++e)
                    if (j & (1 << e)) x = cmul(x, tau[e]);
                T[pb + (static_cast<uint32_t>(j) << S.q)] = x;
                amax = fmaxf(amax, fmaxf(fabsf(x.x), fabsf(x.y)));
            }
            const int ex = amax > 0.f ? 14 - ilogbf(amax) : 0;
            col_exp[g] = ex;
            for (int j = 0; j < J; ++j) {
                const V x = T[pb + (static_cast<uint32_t>(j) << S.q)];
                const float re = ldexpf(x.x, ex), im = ldexpf(x.y, ex);
                const float hre = store_op<PREC>(B_hi + op_offset<EB>(g, j, kpad), re);
                const float him = store_op<PREC>(B_hi + op_offset<EB>(g, J + j, kpad), im);
                if (Op::split) {
                    store_op<PREC>(B_lo + op_offset<EB>(g, j, kpad), re - hre);
                    store_op<PREC>(B_lo + op_offset<EB>(g, J + j, kpad), im - him);
                }
            }
            for (int k = 2 * J; k < kpad; ++k) {  // K padding
                store_op<PREC>(B_hi + op_offset<EB>(g, k, kpad), 0.f);
                if (Op::split) store_op<PREC>(B_lo + op_offset<EB>(g, k, kpad), 0.f);
            }
        }
        fence_proxy_async_smem();  // B written by threads, read by the tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // 3. the GEMM
        if (tid == 0) {
            const uint32_t a0 = smem_u32(A_hi), a1 = smem_u32(A_lo), b0 = smem_u32(B_hi), b1 = smem_u32(B_lo);
            for (int kb = 0; kb < kpad / kstep; ++kb) {
                const uint32_t ko = static_cast<uint32_t>(kb) * koff_step;
                const uint32_t dst = taddr + static_cast<uint32_t>(kb % nacc) * cols_pow2;
                const uint32_t acc = kb >= nacc ? 1u : 0u;
                umma<Op::kind>(dst, umma_desc(a0 + ko, lbo, sbo), umma_desc(b0 + ko, lbo, sbo), idesc, acc);
                if (Op::split) {
                    umma<Op::kind>(dst, umma_desc(a1 + ko, lbo, sbo), umma_desc(b0 + ko, lbo, sbo), idesc, 1);
                    umma<Op::kind>(dst, umma_desc(a0 + ko, lbo, sbo), umma_desc(b1 + ko, lbo, sbo), idesc, 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar_mma)));
        }
        const bool okm = mbar_wait_bounded(&mbar_mma, ph_mma, P.wait_limit_ns);
        ph_mma ^= 1u;
        if (__syncthreads_or(!okm)) { aborted = true; break; }
        tc_fence_after();
        // 4. D (128 rows x ncols) from tensor memory to shared memory, row m = lane
        {
            const int w = tid >> 5, l = tid & 31;
            const int m = w * 32 + l;
            for (int c = 0; c < ncols; c += 16) {
                float sum[16];
                // pairwise sum over the accumulators: level by level, 16 columns at a time
                float part[8][16];
                const int np = nacc < 8 ? nacc : 8;
                for (int a0 = 0; a0 < nacc; a0 += np) {
                    for (int i = 0; i < np; ++i) {
                        uint32_t v[16];
                        const uint32_t a = taddr + (static_cast<uint32_t>(w * 32) << 16) +
                                           static_cast<uint32_t>(a0 + i) * cols_pow2 + static_cast<uint32_t>(c);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                              "=r"(v[14]), "=r"(v[15])
                            : "r"(a));
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int j = 0; j < 16; ++j) part[i][j] = __uint_as_float(v[j]);
                    }
                    for (int width = 1; width < np; width *= 2)
                        for (int i = 0; i + width < np; i += 2 * width)
#pragma unroll
                            for (int j = 0; j < 16; ++j) part[i][j] += part[i + width][j];
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[j] = a0 == 0 ? part[0][j] : sum[j] + part[0][j];
                }
                if (m < 2 * J)
                    for (int j = 0; j < 16; ++j) D[m * ncols + c + j] = sum[j];
            }
        }
        tc_fence_before();
        __syncthreads();
        // 5. store: output j of column g is (D[j][g], D[J + j][g]) / 2^ex * scale
        {
            V* __restrict__ out = static_cast<V*>(P.out);
            for (int idx = tid; idx < ng * J; idx += kTcThreads) {
                const int g = idx % ng, j = idx / ng;
                const int lo5 = P.tab_off[0] + (g & 31), hi5 = P.tab_off[0] + 32 + (g >> 5);
                int64_t o = out_tile + tab.ob[lo5] + tab.ob[hi5];
                for (int e = 0; e < r; ++e)
                    if (j & (1 << e)) o += int64_t(1) << P.p_out[S.q + e];
                const float f = ldexpf(scale, -col_exp[g]);
                out[o] = make_float2(D[j * ncols + g] * f, D[(J + j) * ncols + g] * f);
            }
        }
        __syncthreads();
    }
    if (aborted && tid == 0) atomicExch(P.status, -5);
    if (!aborted && P.first && !P.last) {
        const double tot = block_sum<kTcThreads>(norm_acc, red);
        if (tid == 0) P.partials[blockIdx.x] = tot;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(tcols));
}

// ---------------------------------------------------------------- fast path
//
// Tiles of 2^TB amplitudes with one block of R wires: TB = 12 with R = 4..6
// (plans of fused blocks of 5 or 6 wires, n >= 13), TB = 11 with R = 4..7
// (blocks of 4 or 7 wires, n >= 11).  NT = 2^{TB-4} threads (256 or 128);
// thread t owns column c = t % NG of
// the tile (NG = 2^{TB-R} columns) and the 16 consecutive block indices j of
// chunk t / NG, so lanes run along consecutive columns.  Per tile: TMA load
// (double-buffered, the tile after next streams in during the GEMM), cross
// twiddles and column scaling in registers, operands written as 16-byte
// core-matrix rows, the MMAs from one thread, all TMEM loads of a 16-column
// chunk in flight before one wait, and the outputs stored from the result
// staging area with lanes along columns.
//
// The real embedding of the complex product Y = F X:
//   R <= 6: A = [[Re F, -Im F], [Im F, Re F]] (2^{R+1} <= 128 rows), B's row c
//           = [Re x_c; Im x_c]; D = A B holds [Re y_c; Im y_c] in rows 0..2J-1
//           of GEMM column c (N = NG);
//   R = 7:  2J = 256 rows do not fit one M = 128 MMA, and [[Re, -Im], [Im, Re]]
//           in two halves would need 2 x 128 KiB of FP16 hi + lo operands.  So
//           A = [Re F | Im F] (128 x 256) and B carries the embedding: row c =
//           [Re x_c; -Im x_c] and row NG + c = [Im x_c; Re x_c], so D column c
//           is Re y_c and column NG + c is Im y_c (N = 2 NG).  The split tiers'
//           low parts of -x are the negated low parts of x (rounding to
//           nearest is symmetric), so both rows come from one rounding.

// Round 16 consecutive K entries of one operand row (k0 a multiple of 16) to
// the operand format and write them as 16-byte core-matrix rows at p0, p0 +
// 128, ...; the rounded values come back in r.
template <int PREC>
__device__ __forceinline__ void write_op16(unsigned char* p0, const float (&v)[16], float (&r)[16]) {
    if constexpr (TcOp<PREC>::bytes == 2) {
#pragma unroll
        for (int m = 0; m < 2; ++m) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float a = v[m * 8 + 2 * h], b = v[m * 8 + 2 * h + 1];
                if constexpr (PREC == TC_BF16 || PREC == TC_BF16X3) {
                    const __nv_bfloat162 t = __floats2bfloat162_rn(a, b);
                    const float2 f = __bfloat1622float2(t);
                    r[m * 8 + 2 * h] = f.x;
                    r[m * 8 + 2 * h + 1] = f.y;
                    w[h] = *reinterpret_cast<const uint32_t*>(&t);
                } else {
                    const __half2 t = __floats2half2_rn(a, b);
                    const float2 f = __half22float2(t);
                    r[m * 8 + 2 * h] = f.x;
                    r[m * 8 + 2 * h + 1] = f.y;
                    w[h] = *reinterpret_cast<const uint32_t*>(&t);
                }
            }
            *reinterpret_cast<uint4*>(p0 + m * 128) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            uint32_t w[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(w[h]) : "f"(v[m * 4 + h]));
                r[m * 4 + h] = __uint_as_float(w[h]);
            }
            *reinterpret_cast<uint4*>(p0 + m * 128) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

template <int PREC, int R, int TBITS>
struct TcFast {
    static constexpr int EB = TcOp<PREC>::bytes;
    static constexpr int TB = TBITS;             // tile bits
    static constexpr int NT = 1 << (TB - 4);     // threads: 16 amplitudes each
    static constexpr int J = 1 << R;
    static constexpr int NG = 1 << (TB - R);     // tile columns
    static constexpr bool BEMB = R == 7;         // the embedding in B (see above)
    static constexpr int N = BEMB ? 2 * NG : NG; // GEMM N
    static constexpr int KPAD = 2 * J;
    static constexpr int KSTEP = 32 / EB;  // K per MMA
    static constexpr int KSTEPS = KPAD / KSTEP;
    // accumulators (TMEM: NACC x N <= 512 columns; at most 8, so one readback
    // chunk keeps its 8 x 16 values in registers)
    static constexpr int NACC0 = (KSTEPS < 512 / N) ? KSTEPS : 512 / N;
    static constexpr int NACC = NACC0 < 8 ? NACC0 : 8;
    static constexpr uint32_t TILE_BYTES = (1u << TB) * 8u;
    static constexpr size_t D_BYTES = size_t(2 * J) * NG * 4;
    static constexpr size_t A_BYTES = size_t(128) * KPAD * EB;
    static constexpr size_t B_BYTES = size_t(N) * KPAD * EB;
    static constexpr int SPLIT = TcOp<PREC>::split;
    static size_t smem(int ntab, int ntw) {
        return 2 * size_t(TILE_BYTES) + D_BYTES + A_BYTES * (SPLIT ? 2 : 1) + B_BYTES * (SPLIT ? 2 : 1) +
               size_t(ntab) * (size_t(ntw) * 8 + 8 + 4 + 4);
    }
};

template <int DIR, int PREC, int R, int TB>
__global__ void __launch_bounds__(TcFast<PREC, R, TB>::NT, 1)
    qft_tc_fast_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ PassParams P,
                       const __grid_constant__ TcParams Q) {
    using V = float2;
    using F = TcFast<PREC, R, TB>;
    using Op = TcOp<PREC>;
    constexpr int NT = F::NT;
    constexpr int J = F::J, NG = F::NG, N = F::N, KPAD = F::KPAD, EB = F::EB;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar_load[2];
    __shared__ __align__(8) uint64_t mbar_mma;
    __shared__ uint32_t s_taddr;
    __shared__ double red[NT / 32];
    __shared__ float s_amax[NT];
    __shared__ int s_exp[NG];
    __shared__ int64_t s_obc[NG];
    __shared__ __align__(16) V Ubuf[kMaxR * kMaxStages];

    const int tid = threadIdx.x;
    const StageDesc& S = P.st[0];
    unsigned char* const T0 = smem_raw;  // two tile buffers
    // results, column-major: column c holds its 2J rows (Re then Im), 16-byte
    // chunks XOR-swizzled by (c & 7) so that both the row-wise writes from
    // tensor memory and the column-wise reads are conflict-free
    float* const D = reinterpret_cast<float*>(smem_raw + 2 * F::TILE_BYTES);
    unsigned char* const A_hi = smem_raw + 2 * F::TILE_BYTES + F::D_BYTES;
    unsigned char* const A_lo = A_hi + F::A_BYTES;
    unsigned char* const B_hi = A_lo + (F::SPLIT ? F::A_BYTES : 0);
    unsigned char* const B_lo = B_hi + F::B_BYTES;
    unsigned char* const tab_raw = B_lo + (F::SPLIT ? F::B_BYTES : 0);
    GroupTab<V> tab;
    tab.ntab = P.ntab;
    tab.tw = reinterpret_cast<V*>(tab_raw);
    tab.ob = reinterpret_cast<int64_t*>(tab_raw + size_t(P.ntw) * sizeof(V) * P.ntab);
    tab.pb = reinterpret_cast<uint32_t*>(tab_raw + (size_t(P.ntw) * sizeof(V) + 8) * P.ntab);
    tab.sb = tab.pb + P.ntab;

    build_group_tables<float, DIR, NT>(P, tab);
    {
        const uint4* src = static_cast<const uint4*>(Q.a_hi);
        for (size_t i = tid; i < F::A_BYTES / 16; i += NT) reinterpret_cast<uint4*>(A_hi)[i] = src[i];
        if (F::SPLIT) {
            src = static_cast<const uint4*>(Q.a_lo);
            for (size_t i = tid; i < F::A_BYTES / 16; i += NT) reinterpret_cast<uint4*>(A_lo)[i] = src[i];
        }
    }
    constexpr uint32_t kTcols = static_cast<uint32_t>(N * F::NACC) < 32u ? 32u : static_cast<uint32_t>(N * F::NACC);
    if (tid < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_taddr)),
                     "r"(kTcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&mbar_load[0], 1);
        mbar_init(&mbar_load[1], 1);
        mbar_init(&mbar_mma, 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;

    float scale = 1.f;
    if (P.last) {  // never also the first pass here: scale_in from the first pass's partials
        double s = 0.0;
        for (int i = tid; i < P.npartials; i += NT) s += P.partials[i];
        const double scale_in = sqrt(block_sum<NT>(s, red));
        scale = static_cast<float>(output_factor(P, scale_in));
        if (blockIdx.x == 0 && tid == 0) {
            P.meta[0] = scale_in;
            if (P.user_scale) *P.user_scale = scale_in;
        }
    }
    constexpr uint32_t idesc = (1u << 4) | (static_cast<uint32_t>(Op::fmt) << 7) |
                               (static_cast<uint32_t>(Op::fmt) << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
                               (static_cast<uint32_t>(128 >> 4) << 24);
    constexpr int KC = 16 / EB;
    constexpr uint32_t lbo = 128u, sbo = static_cast<uint32_t>(KPAD / KC) * 128u;
    constexpr uint32_t koff_step = static_cast<uint32_t>(F::KSTEP / KC) * 128u;

    const int c = tid % NG, jq = tid / NG;  // column, chunk of 16 block indices
    const int lo5 = P.tab_off[0] + (c & 31), hi5 = P.tab_off[0] + 32 + (c >> 5);
    const uint32_t q = static_cast<uint32_t>(S.q);
    bool jmajor = false;  // a block wire holds output address bit 0
#pragma unroll
    for (int e = 0; e < R; ++e) jmajor = jmajor || P.p_out[S.q + e] == 0;
    if (jq == 0) s_obc[c] = tab.ob[lo5] + tab.ob[hi5];  // output offset of each column (tile-invariant)

    double norm_acc = 0.0;
    uint32_t ph_load = 0u, ph_mma = 0u;
    bool aborted = false;
    int64_t tile = blockIdx.x;
    if (tid == 0 && !P.test_skip_first_load) {
        if (tile < P.num_tiles) issue_tile_load(P, &tmap, tile, T0, &mbar_load[0], F::TILE_BYTES);
        if (tile + gridDim.x < P.num_tiles)
            issue_tile_load(P, &tmap, tile + gridDim.x, T0 + F::TILE_BYTES, &mbar_load[1], F::TILE_BYTES);
    }
    for (int k = 0; tile < P.num_tiles; tile += gridDim.x, ++k) {
        const int buf = k & 1;
        const V* const T = reinterpret_cast<const V*>(T0 + buf * F::TILE_BYTES);
        compute_tile_twiddles<float, DIR>(P, tile, Ubuf);
        uint64_t I_tile;
        int64_t out_tile;
        tile_coords(P, tile, I_tile, out_tile);
        const bool ok = mbar_wait_bounded(&mbar_load[buf], (ph_load >> buf) & 1u, P.wait_limit_ns);
        ph_load ^= 1u << buf;
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        // 1. this thread's 16 amplitudes: cross twiddle, column scale, operands
        V x[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = T[tab.pb[lo5] | tab.pb[hi5] | (static_cast<uint32_t>(jq * 16 + i) << q)];
        if (P.first) {
            float a = 0.f;
#pragma unroll
            for (int i = 0; i < 16; ++i) a += x[i].x * x[i].x + x[i].y * x[i].y;
            norm_acc += static_cast<double>(a);
        }
        if (S.cross) {
            V tau[R];
#pragma unroll
            for (int e = 0; e < R; ++e) {
                if (S.lo_tw && S.hi_tw) tau[e] = cmul(tab.tw[e * tab.ntab + lo5], tab.tw[e * tab.ntab + hi5]);
                else if (S.lo_tw) tau[e] = tab.tw[e * tab.ntab + lo5];
                else tau[e] = tab.tw[e * tab.ntab + hi5];
                if (S.tile_above) tau[e] = cmul(tau[e], Ubuf[S.uoff + e]);
            }
            // block index j = jq * 16 + i: the chunk bits (>= 4) give one factor
            V bq = make_float2(1.f, 0.f);
#pragma unroll
            for (int e = 4; e < R; ++e)
                if ((jq >> (e - 4)) & 1) bq = cmul(bq, tau[e]);
            V tl[4], th[4];
            tl[1] = tau[0];
            tl[2] = tau[1];
            tl[3] = cmul(tau[0], tau[1]);
            th[0] = bq;
            th[1] = cmul(bq, tau[2]);
            th[2] = cmul(bq, tau[3]);
            th[3] = cmul(th[1], tau[3]);
#pragma unroll
            for (int i = 1; i < 16; ++i)
                if (i & 3) x[i] = cmul(x[i], tl[i & 3]);
            if (jq) {
#pragma unroll
                for (int i = 0; i < 16; ++i) x[i] = cmul(x[i], th[i >> 2]);
            } else {
#pragma unroll
                for (int i = 4; i < 16; ++i) x[i] = cmul(x[i], th[i >> 2]);
            }
        }
        float amax = 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i) amax = fmaxf(amax, fmaxf(fabsf(x[i].x), fabsf(x[i].y)));
        s_amax[tid] = amax;
        __syncthreads();
        float cm = 0.f;
#pragma unroll
        for (int h = 0; h < J / 16; ++h) cm = fmaxf(cm, s_amax[h * NG + c]);
        // exponent so that the column's largest component is near 2^14
        int ex = 0;
        if (cm > 0.f) {
            const int e8 = static_cast<int>((__float_as_uint(cm) >> 23) & 255u);
            ex = 14 - (e8 - 127);
            ex = ex < -100 ? -100 : (ex > 100 ? 100 : ex);
        }
        if (jq == 0) s_exp[c] = ex;
        {
            const float sc = __uint_as_float(static_cast<uint32_t>(ex + 127) << 23);
            float re[16], im[16], rr[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                re[i] = x[i].x * sc;
                im[i] = x[i].y * sc;
            }
            const uint32_t ore = op_offset<EB>(c, jq * 16, KPAD), oim = op_offset<EB>(c, J + jq * 16, KPAD);
            // R = 7: row NG + c = [Im; Re], and row c's second half is -Im
            const uint32_t ore2 = op_offset<EB>(NG + c, J + jq * 16, KPAD), oim2 = op_offset<EB>(NG + c, jq * 16, KPAD);
            float ng[16];
            write_op16<PREC>(B_hi + ore, re, rr);
            if (F::BEMB) write_op16<PREC>(B_hi + ore2, re, rr);
            if (F::SPLIT) {
#pragma unroll
                for (int i = 0; i < 16; ++i) re[i] -= rr[i];
                write_op16<PREC>(B_lo + ore, re, rr);
                if (F::BEMB) write_op16<PREC>(B_lo + ore2, re, rr);
            }
            write_op16<PREC>(B_hi + (F::BEMB ? oim2 : oim), im, rr);
            if (F::BEMB) {
#pragma unroll
                for (int i = 0; i < 16; ++i) ng[i] = -rr[i];
                write_op16<PREC>(B_hi + oim, ng, rr);  // -hi(Im): exact
            }
            if (F::SPLIT) {
#pragma unroll
                for (int i = 0; i < 16; ++i) im[i] += F::BEMB ? rr[i] : -rr[i];  // Im - hi(Im)
                write_op16<PREC>(B_lo + (F::BEMB ? oim2 : oim), im, rr);
                if (F::BEMB) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) ng[i] = -rr[i];
                    write_op16<PREC>(B_lo + oim, ng, rr);
                }
            }
        }
        fence_proxy_async_smem();  // B written by threads, read by the tensor cores
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // 2. prefetch the tile after next into the consumed buffer; the GEMM
        if (tid == 0) {
            const int64_t nt = tile + 2 * static_cast<int64_t>(gridDim.x);
            if (nt < P.num_tiles) issue_tile_load(P, &tmap, nt, T0 + buf * F::TILE_BYTES, &mbar_load[buf], F::TILE_BYTES);
            const uint32_t a0 = smem_u32(A_hi), a1 = smem_u32(A_lo), b0 = smem_u32(B_hi), b1 = smem_u32(B_lo);
#pragma unroll
            for (int kb = 0; kb < F::KSTEPS; ++kb) {
                const uint32_t ko = static_cast<uint32_t>(kb) * koff_step;
                const uint32_t dst = taddr + static_cast<uint32_t>(kb % F::NACC) * N;
                const uint32_t acc = kb >= F::NACC ? 1u : 0u;
                umma<Op::kind>(dst, umma_desc(a0 + ko, lbo, sbo), umma_desc(b0 + ko, lbo, sbo), idesc, acc);
                if (F::SPLIT) {
                    umma<Op::kind>(dst, umma_desc(a1 + ko, lbo, sbo), umma_desc(b0 + ko, lbo, sbo), idesc, 1);
                    umma<Op::kind>(dst, umma_desc(a0 + ko, lbo, sbo), umma_desc(b1 + ko, lbo, sbo), idesc, 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar_mma)));
        }
        const bool okm = mbar_wait_bounded(&mbar_mma, ph_mma, P.wait_limit_ns);
        ph_mma ^= 1u;
        if (__syncthreads_or(!okm)) {
            aborted = true;
            break;
        }
        tc_fence_after();
        // 3. accumulators -> D: warp w reads TMEM lanes 32 (w & 3).. (rows m) for
        //    its share (w >> 2) of the GEMM columns, 16 columns per step, the
        //    accumulators summed pairwise.  R = 7: GEMM column cc >= NG is the
        //    imaginary part of tile column cc - NG (staging row m + J).
        {
            constexpr int CG = NT / 128;  // column groups (warp quads)
            const int w = tid >> 5, l = tid & 31, qd = w & 3, chalf = w >> 2;
            const int m = qd * 32 + l;
            if (F::BEMB || qd * 32 < 2 * J) {
#pragma unroll 1
                for (int cc = chalf * (N / CG); cc < (chalf + 1) * (N / CG); cc += 16) {
                    uint32_t v[F::NACC][16];
#pragma unroll
                    for (int a = 0; a < F::NACC; ++a) {
                        const uint32_t addr = taddr + (static_cast<uint32_t>(qd * 32) << 16) +
                                              static_cast<uint32_t>(a * N + cc);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                            : "=r"(v[a][0]), "=r"(v[a][1]), "=r"(v[a][2]), "=r"(v[a][3]), "=r"(v[a][4]), "=r"(v[a][5]),
                              "=r"(v[a][6]), "=r"(v[a][7]), "=r"(v[a][8]), "=r"(v[a][9]), "=r"(v[a][10]),
                              "=r"(v[a][11]), "=r"(v[a][12]), "=r"(v[a][13]), "=r"(v[a][14]), "=r"(v[a][15])
                            : "r"(addr));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        float s[F::NACC];
#pragma unroll
                        for (int a = 0; a < F::NACC; ++a) s[a] = __uint_as_float(v[a][j]);
#pragma unroll
                        for (int width = 1; width < F::NACC; width *= 2)
#pragma unroll
                            for (int a = 0; a + width < F::NACC; a += 2 * width) s[a] += s[a + width];
                        const int col = F::BEMB ? (cc + j) % NG : cc + j;
                        const int row = F::BEMB && cc + j >= NG ? m + J : m;
                        D[col * (2 * J) + ((((row >> 2) ^ (col & 7)) << 2) | (row & 3))] = s[0];
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
        // 4. outputs: amplitude j of column c is (D[j][c], D[J + j][c]) * 2^-ex * scale.
        //    Lanes run along the columns, unless a block wire holds output address
        //    bit 0 (the first pass of a natural-order plan): then along j, so that
        //    every warp store covers a contiguous output run.
        if (jmajor) {
            const int j = tid % J;
            const int64_t jofs = out_tile + [&] {
                int64_t o = 0;
#pragma unroll
                for (int e = 0; e < R; ++e)
                    if ((j >> e) & 1) o += int64_t(1) << P.p_out[S.q + e];
                return o;
            }();
            const int sre = ((j >> 2) << 2) | (j & 3), sim = (((J + j) >> 2) << 2) | (j & 3);
            V* __restrict__ out = static_cast<V*>(P.out) + jofs;
#pragma unroll 4
            for (int kk = 0; kk < 16; ++kk) {
                const int cc = tid / J + kk * (NT / J);
                const int sw = (cc & 7) << 2;
                const float f = scale * __uint_as_float(static_cast<uint32_t>(127 - s_exp[cc]) << 23);
                const float* Dc = D + cc * (2 * J);
                out[s_obc[cc]] = make_float2(Dc[sre ^ sw] * f, Dc[sim ^ sw] * f);
            }
        } else {
            const float f = scale * __uint_as_float(static_cast<uint32_t>(127 - s_exp[c]) << 23);
            int64_t base = out_tile + tab.ob[lo5] + tab.ob[hi5];
#pragma unroll
            for (int e = 4; e < R; ++e)
                if ((jq >> (e - 4)) & 1) base += int64_t(1) << P.p_out[S.q + e];
            int64_t oo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) oo[e] = int64_t(1) << P.p_out[S.q + e];
            V* __restrict__ out = static_cast<V*>(P.out) + base;
            const float4* Dc = reinterpret_cast<const float4*>(D + c * (2 * J));
            float re[16], im[16];
#pragma unroll
            for (int h = 0; h < 4; ++h) {  // rows jq*16 + 4h .. +3 (Re) and J + the same (Im)
                const float4 a = Dc[((jq * 16) / 4 + h) ^ (c & 7)];
                const float4 bb = Dc[((J + jq * 16) / 4 + h) ^ (c & 7)];
                re[4 * h] = a.x; re[4 * h + 1] = a.y; re[4 * h + 2] = a.z; re[4 * h + 3] = a.w;
                im[4 * h] = bb.x; im[4 * h + 1] = bb.y; im[4 * h + 2] = bb.z; im[4 * h + 3] = bb.w;
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                int64_t o = 0;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (i & (1 << e)) o += oo[e];
                out[o] = make_float2(re[i] * f, im[i] * f);
            }
        }

    }
    if (aborted && tid == 0) {
        atomicExch(P.status, -5);  // QFT_ERR_TIMEOUT
        for (int b = 0; b < 2; ++b) mbar_wait_bounded(&mbar_load[b], (ph_load >> b) & 1u, P.wait_limit_ns);
    }
    if (!aborted && P.first) {
        const double tot = block_sum<NT>(norm_acc, red);
        if (tid == 0) P.partials[blockIdx.x] = tot;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcols));
}

// The fast path serves passes of a plan of more than one pass with one block
// of 4..6 wires in 2^12-amplitude tiles or of 4..7 wires in 2^11-amplitude tiles.
static inline bool tc_fast_ok(const PassParams& P) {
    if (P.nstages != 1 || (P.first && P.last)) return false;
    const int r = P.st[0].r;
    return (P.tb == 12 && r >= 4 && r <= 6) || (P.tb == 11 && r >= 4 && r <= 7);
}

template <int PREC>
static inline size_t tc_fast_smem(const PassParams& P) {
    if (P.tb == 11) {
        switch (P.st[0].r) {
            case 4: return TcFast<PREC, 4, 11>::smem(P.ntab, P.ntw);
            case 5: return TcFast<PREC, 5, 11>::smem(P.ntab, P.ntw);
            case 6: return TcFast<PREC, 6, 11>::smem(P.ntab, P.ntw);
            default: return TcFast<PREC, 7, 11>::smem(P.ntab, P.ntw);
        }
    }
    switch (P.st[0].r) {
        case 4: return TcFast<PREC, 4, 12>::smem(P.ntab, P.ntw);
        case 5: return TcFast<PREC, 5, 12>::smem(P.ntab, P.ntw);
        default: return TcFast<PREC, 6, 12>::smem(P.ntab, P.ntw);
    }
}

template <int DIR, int PREC, int R, int TB>
static cudaError_t launch_tc_fast_t(const CUtensorMap& map, const PassParams& P, const TcParams& Q, int grid,
                                    size_t smem, cudaStream_t st) {
    auto kern = qft_tc_fast_kernel<DIR, PREC, R, TB>;
    {
        const cudaError_t e = ensure_dynamic_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, TcFast<PREC, R, TB>::NT, smem, st>>>(map, P, Q);
    return cudaGetLastError();
}

template <int DIR, int PREC>
static cudaError_t launch_tc_t(const CUtensorMap& map, const PassParams& P, const TcParams& Q, int grid, size_t smem,
                               cudaStream_t st) {
    if (tc_fast_ok(P)) {
        if (P.tb == 11) {
            switch (P.st[0].r) {
                case 4: return launch_tc_fast_t<DIR, PREC, 4, 11>(map, P, Q, grid, smem, st);
                case 5: return launch_tc_fast_t<DIR, PREC, 5, 11>(map, P, Q, grid, smem, st);
                case 6: return launch_tc_fast_t<DIR, PREC, 6, 11>(map, P, Q, grid, smem, st);
                default: return launch_tc_fast_t<DIR, PREC, 7, 11>(map, P, Q, grid, smem, st);
            }
        }
        switch (P.st[0].r) {
            case 4: return launch_tc_fast_t<DIR, PREC, 4, 12>(map, P, Q, grid, smem, st);
            case 5: return launch_tc_fast_t<DIR, PREC, 5, 12>(map, P, Q, grid, smem, st);
            default: return launch_tc_fast_t<DIR, PREC, 6, 12>(map, P, Q, grid, smem, st);
        }
    }
    auto kern = qft_tc_pass_kernel<DIR, PREC>;
    {
        const cudaError_t e = ensure_dynamic_smem(kern, smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<grid, kTcThreads, smem, st>>>(map, P, Q);
    return cudaGetLastError();
}

template <int DIR>
cudaError_t launch_tc_dir(int prec, const CUtensorMap& map, const PassParams& P, const TcParams& Q, int grid,
                          size_t smem, cudaStream_t st) {
    switch (prec) {
        case TC_TF32: return launch_tc_t<DIR, TC_TF32>(map, P, Q, grid, smem, st);
        case TC_BF16: return launch_tc_t<DIR, TC_BF16>(map, P, Q, grid, smem, st);
        case TC_BF16X3: return launch_tc_t<DIR, TC_BF16X3>(map, P, Q, grid, smem, st);
        case TC_FP16: return launch_tc_t<DIR, TC_FP16>(map, P, Q, grid, smem, st);
        default: return launch_tc_t<DIR, TC_FP16X3>(map, P, Q, grid, smem, st);
    }
}

// The kernels of each direction are instantiated in their own translation
// unit (qft_tc_fwd.cu, qft_tc_inv.cu), so the two compile in parallel.
extern template cudaError_t launch_tc_dir<-1>(int, const CUtensorMap&, const PassParams&, const TcParams&, int, size_t,
                                              cudaStream_t);
extern template cudaError_t launch_tc_dir<+1>(int, const CUtensorMap&, const PassParams&, const TcParams&, int, size_t,
                                              cudaStream_t);

}  // namespace qft
