// qft_device.cuh -- device helpers shared by the pass, batch and tensor-core
// kernels: mbarrier / TMA wrappers, complex arithmetic, exact-phase twiddles,
// the buffer-B swizzle, the block sub-circuit, group tables and tile
// coordinates.  Internal to libqftfft.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <mutex>
#include <type_traits>

#include "plan.hpp"
#include "qft_df.cuh"

namespace qft {

// ------------------------------------------------------------------ helpers

// Raise a kernel's dynamic shared-memory limit to at least `smem` on the
// current device.  The attribute belongs to the function in the device's
// context, so it is shared by every host thread: the limit only ever grows
// (a thread that needs less never lowers it under another thread's launch),
// tracked per kernel (keyed by its address) and device in one process-wide
// table.
inline cudaError_t ensure_dynamic_smem_raw(const void* kern, size_t smem) {
    struct Entry {
        const void* kern;
        int dev;
        size_t smem;
    };
    static std::mutex mu;
    static Entry table[256];
    static int used = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int i = 0;
    while (i < used && !(table[i].kern == kern && table[i].dev == dev)) ++i;
    if (i < used && smem <= table[i].smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    if (i < used) {
        table[i].smem = smem;
    } else if (used < 256) {
        table[used++] = Entry{kern, dev, smem};
    }
    return cudaSuccess;
}

template <typename K>
inline cudaError_t ensure_dynamic_smem(K kern, size_t smem) {
    return ensure_dynamic_smem_raw(reinterpret_cast<const void*>(kern), smem);
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<dfloat> { using type = dcomplex; };

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: gives up after limit_ns (the caller reports QFT_ERR_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_5d(void* dst, const CUtensorMap* map, const int32_t c[5],
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]),
        "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void bulk_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Index of the lowest set bit of j (j > 0).  Written as plain arithmetic so
// that, with j a constant of an unrolled loop, it folds to a constant and the
// register arrays it indexes stay in registers (an opaque intrinsic there
// would force those arrays into local memory).
__host__ __device__ constexpr int low_bit(int j) {
    return (j & 1) ? 0 : (j & 2) ? 1 : (j & 4) ? 2 : (j & 8) ? 3 : (j & 16) ? 4 : (j & 32) ? 5 : 6;
}

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    V r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// complex64: the real and imaginary parts of an amplitude sit in one 64-bit
// register pair, so a complex add or subtract is one packed FP32x2
// instruction (add/sub.rn.f32x2, sm_100 and later; per-lane IEEE
// round-to-nearest, the same results as two scalar adds) -- half the
// instructions of the butterfly network.
__device__ __forceinline__ uint64_t f2pack(float x, float y) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 f2unpack(uint64_t r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a.x, a.y)), "l"(f2pack(b.x, b.y)));
    return f2unpack(d);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a.x, a.y)), "l"(f2pack(b.x, b.y)));
    return f2unpack(d);
}
// lane-wise a * b and a * b + c on FP32 pairs (packed FP32x2)
__device__ __forceinline__ float2 cmul2(float2 a, float2 b) {
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2pack(a.x, a.y)), "l"(f2pack(b.x, b.y)));
    return f2unpack(d);
}
__device__ __forceinline__ float2 cfma2(float2 a, float2 b, float2 c) {
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2pack(a.x, a.y)), "l"(f2pack(b.x, b.y)), "l"(f2pack(c.x, c.y)));
    return f2unpack(d);
}
// double-float complex128 amplitudes (qft_df.cuh)
__device__ __forceinline__ dcomplex cadd(dcomplex a, dcomplex b) { return dc_add(a, b); }
__device__ __forceinline__ dcomplex csub(dcomplex a, dcomplex b) { return dc_sub(a, b); }
__device__ __forceinline__ dcomplex cmul(dcomplex a, dcomplex b) { return dc_mul(a, b); }

// exp(2 pi i m / 32) for m = 0..15 (cos, sin): the rotations of controlled
// phases between wires at distance <= 4 inside one register block
// (R_2 .. R_5 and their products).
#define QFT_W32_COS 1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708, 0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785, 0.0, -0.19509032201612826785, -0.38268343236508977173, -0.55557023301960222474, -0.70710678118654752440, -0.83146961230254523708, -0.92387953251128675613, -0.98078528040323044913
#define QFT_W32_SIN 0.0, 0.19509032201612826785, 0.38268343236508977173, 0.55557023301960222474, 0.70710678118654752440, 0.83146961230254523708, 0.92387953251128675613, 0.98078528040323044913, 1.0, 0.98078528040323044913, 0.92387953251128675613, 0.83146961230254523708, 0.70710678118654752440, 0.55557023301960222474, 0.38268343236508977173, 0.19509032201612826785
__device__ constexpr double kW32c[16] = {QFT_W32_COS};
__device__ constexpr double kW32s[16] = {QFT_W32_SIN};
// Compile-time copies for constant initialisers evaluated by the host compiler
// (a local array here must never reach device code at run time).
constexpr double w32c_ct(int i) {
    const double t[16] = {QFT_W32_COS};
    return t[i];
}
constexpr double w32s_ct(int i) {
    const double t[16] = {QFT_W32_SIN};
    return t[i];
}

// z *= exp(DIR * 2 pi i m / 32).  With m a compile-time constant after loop
// unrolling the trivial rotations (1, +-i, -1) reduce to moves and negations.
template <int DIR, typename V>
__device__ __forceinline__ void rot32(V& z, int m) {
    using T = decltype(z.x);
    m &= 31;
    if (m == 0) return;
    const bool neg = m >= 16;
    const int mm = m & 15;
    if (mm == 8) {  // multiply by DIR * i
        const T t = z.x;
        if (DIR > 0) { z.x = -z.y; z.y = t; } else { z.x = z.y; z.y = -t; }
    } else if (mm != 0) {
        const T c = static_cast<T>(kW32c[mm]);
        const T s = static_cast<T>(DIR > 0 ? kW32s[mm] : -kW32s[mm]);
        const T re = z.x * c - z.y * s;
        z.y = z.x * s + z.y * c;
        z.x = re;
    }
    if (neg) { z.x = -z.x; z.y = -z.y; }
}

// The same rotations for double-float amplitudes: the constants are split
// into FP32 pairs at compile time, the products formed by df_dot2.
struct W32Pair {
    float ch[16], cl[16], sh[16], sl[16];
    constexpr W32Pair() : ch(), cl(), sh(), sl() {
        for (int i = 0; i < 16; ++i) {
            ch[i] = static_cast<float>(w32c_ct(i));
            cl[i] = static_cast<float>(w32c_ct(i) - static_cast<double>(ch[i]));
            sh[i] = static_cast<float>(w32s_ct(i));
            sl[i] = static_cast<float>(w32s_ct(i) - static_cast<double>(sh[i]));
        }
    }
};
__device__ constexpr W32Pair kW32df{};

template <int DIR>
__device__ __forceinline__ void rot32(dcomplex& z, int m) {
    m &= 31;
    if (m == 0) return;
    const bool neg = m >= 16;
    const int mm = m & 15;
    dfloat x = z.re(), y = z.im();
    if (mm == 8) {
        const dfloat t = x;
        if (DIR > 0) { x = df_neg(y); y = t; } else { x = y; y = df_neg(t); }
    } else if (mm != 0) {
        const dfloat c(kW32df.ch[mm], kW32df.cl[mm]);
        const dfloat s = DIR > 0 ? dfloat(kW32df.sh[mm], kW32df.sl[mm]) : dfloat(-kW32df.sh[mm], -kW32df.sl[mm]);
        // (x + i y)(c + i s) = (x c - y s) + i (x s + y c)
        const dfloat re = df_dot2(x, c, y, s);
        y = df_dot2(x, s, df_neg(y), c);
        x = re;
    }
    if (neg) { x = df_neg(x); y = df_neg(y); }
    z = dc_make(x, y);
}

// The complex number 1 of each amplitude type.
template <typename V> __device__ __forceinline__ V cunit() { V r; r.x = 1; r.y = 0; return r; }
template <> __device__ __forceinline__ dcomplex cunit<dcomplex>() { return dc_make(dfloat(1), dfloat(0)); }

__device__ __forceinline__ void sincospi_t(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sincospi_t(double x, double* s, double* c) { sincospi(x, s, c); }

// exp(DIR * 2 pi i beta / 2^n) for an exact integer phase beta (any 64-bit
// value; only beta mod 2^n matters), n <= 40.  The phase is reduced exactly
// in fixed point (2^40 = one turn) to the nearest quarter turn, so the
// floating-point sine/cosine only sees |x| <= 1/4 (in units of pi).
template <typename T, int DIR>
__device__ __forceinline__ typename Vec2<T>::type phase_turns(uint64_t beta, int n) {
    if constexpr (std::is_same<T, dfloat>::value) {
        // double-float twiddles: the FP64 value split into a pair
        const double2 w = phase_turns<double, DIR>(beta, n);
        return dc_make(dfloat(w.x), dfloat(w.y));
    } else {
        const uint64_t b = (beta << (64 - n)) >> 24;            // beta mod 2^n, scaled to 2^40 per turn
        const uint64_t q4 = (b + (1ull << 37)) >> 38;            // nearest quarter turn, 0..4
        const int64_t rem = static_cast<int64_t>(b) - static_cast<int64_t>(q4 << 38);  // |rem| <= 2^37
        const T x = static_cast<T>(rem) * static_cast<T>(1.0 / 549755813888.0);      // rem / 2^39
        T s, c;
        sincospi_t(x, &s, &c);
        typename Vec2<T>::type r;
        switch (q4 & 3) {
            case 0: r.x = c; r.y = s; break;
            case 1: r.x = -s; r.y = c; break;
            case 2: r.x = -c; r.y = -s; break;
            default: r.x = s; r.y = -c; break;
        }
        if (DIR < 0) r.y = -r.y;
        return r;
    }
}

// XOR swizzle of buffer B: the low SW bits of a tile index are XORed with the
// XOR-fold of its higher SW-bit groups.  A bank-conflict-free access needs the
// lanes of one SMEM wavefront (16 lanes x 8 bytes, or 8 lanes x 16 bytes) to
// hit distinct SW-bit slots; with this map that holds whenever those lanes'
// tile bits have distinct residues mod SW, which the planner arranges.
template <int SW>
__device__ __forceinline__ uint32_t swz(uint32_t x) {
    uint32_t y = x >> SW;
    uint32_t f = 0;
#pragma unroll
    for (int i = 0; i < 16 / SW + 1; ++i) { f ^= y; y >>= SW; }
    return x ^ (f & ((1u << SW) - 1));
}

// The r-wire sub-circuit of one block, in registers (Sec. 2, Fig. 1): for the
// block's wires from the top down, the (unnormalised) butterfly H then the
// controlled phases from the lower wires of the block within distance kk.
// v[j]: bit e of j is wire wlo + e.  The 1/sqrt(2) of every H is folded into
// the pass's final scale.
template <int DIR, int R, typename V>
__device__ __forceinline__ void block_circuit(V (&v)[1 << R], int kk) {
    constexpr int NJ = 1 << R;
#pragma unroll
    for (int t = R - 1; t >= 0; --t) {
        const int bit = 1 << t;
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
            if (!(j & bit)) {
                const V a = v[j], b = v[j | bit];
                v[j] = cadd(a, b);
                v[j | bit] = csub(a, b);
            }
        }
        if (kk >= R - 1) {
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j & bit) rot32<DIR>(v[j], (j & (bit - 1)) << (4 - t));
        } else {
            int lo = t - kk;
            if (lo < 0) lo = 0;
            const int mask = (bit - 1) & ~((1 << lo) - 1);
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j & bit) rot32<DIR>(v[j], (j & mask) << (4 - t));
        }
    }
}

// Per-stage group tables.  A group g (the 2^r amplitudes one thread holds in a
// stage) splits as g = (g & 31) | (g >> 5) << 5 into a lane part and a high
// part whose tile bits are disjoint, so every per-group quantity that is
// additive over disjoint bits is the combination of one lane entry (index
// g & 31) and one high entry (index 32 + (g >> 5)):
//   pb  tile index bits (OR),  sb  their swizzled buffer-B offset (XOR),
//   ob  output address offset (sum),
//   V   the cross-twiddle factors exp(s 2 pi i beta_e / 2^n) of the group's
//       tile wires above the block, one per block wire e (product).
// The tile coordinate's share of the cross twiddle, U_e, is computed once per
// tile.  beta_e is additive over disjoint wire sets, so the full cross twiddle
// of block wire e is U_e * V_e(lane entry) * V_e(high entry).
template <typename V>
struct GroupTab {
    uint32_t* pb;
    uint32_t* sb;  // swz(pb): the swizzle is XOR-linear, so a group's buffer-B base is sb[lane] ^ sb[high]
    int64_t* ob;
    V* tw;  // [e][entry], e < ntw: plane e holds factor e of every entry (lane reads are consecutive)
    int ntab;
};

// Integer phase beta_e of block wire c = wlo + e for the logical bits I (only
// wires above hi = wlo + r - 1 matter): the controlled phases CP(c, t) with
// t > hi, t - c <= kk, in units of 2^-n turns (Eq. 5 / Sec. 2).
__device__ __forceinline__ uint64_t cross_phase(uint64_t I, int n, int hi, int c, int kk) {
    const uint64_t rh = (__brevll(I) >> (64 - n)) & ((1ull << (n - 1 - hi)) - 1ull);
    uint64_t m = rh;
    const int lowcut = n - 1 - c - kk;  // keep targets t <= c + kk
    if (lowcut > 0) m &= ~((1ull << lowcut) - 1ull);
    return m << c;
}

// Deterministic CTA-wide sum (fixed shuffle tree, then warps in order).
template <int NT>
__device__ __forceinline__ double block_sum(double x, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) red[w] = x;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < NT / 32; ++i) t += red[i];
    __syncthreads();
    return t;
}

// Output factor of the decode step (Sec. 3 step 4) times the folded 2^{-n/2}.
__device__ __forceinline__ double output_factor(const PassParams& P, double scale_in) {
    switch (P.scale_mode) {
        case 0: return scale_in > 0.0 ? P.inv_root_n / scale_in : 0.0;  // state
        case 1: return P.inv_root_n;                                     // unitary
        case 2: return 1.0;                                              // unnormalised
        default: return P.inv_root_n * P.inv_root_n;                     // 1/N
    }
}

// Amplitude input/output of the pass kernels.  float2 / double2 states are
// read and written as they are.  The double-float complex128 kernel keeps
// amplitudes as dcomplex pairs between passes (the workspace holds 16-byte df
// pairs, like double2) and converts only where the caller's FP64 data enters
// (the first pass) and leaves (the last pass), with the exponent shift of its
// range normalisation (qft_df.cuh).
struct AmpIO {
    int raw_in;     // the tile holds the caller's FP64 input (first pass of a df transform)
    int raw_out;    // the output is the caller's FP64 state (last pass of a df transform)
    int shift_in;   // input scaled by 2^-shift_in
    int shift_out;  // output scaled by 2^shift_out
};

template <typename T>
struct AmpTraits {
    using V = typename Vec2<T>::type;
    static constexpr bool kDF = false;
    __device__ static __forceinline__ V load(const V* A, uint32_t i, const AmpIO&) { return A[i]; }
    // |v|^2 summed over a group: norm_add per amplitude, norm_done once
    using NormAcc = V;  // per-component sums (x: real parts, y: imaginary parts)
    __device__ static __forceinline__ void norm_add(NormAcc& a, const V& v) {
        if constexpr (sizeof(T) == 4) {
            a = cfma2(v, v, a);  // one packed FP32x2 fma per amplitude
        } else {
            a.x += v.x * v.x;
            a.y += v.y * v.y;
        }
    }
    __device__ static __forceinline__ double norm_done(NormAcc a) { return static_cast<double>(a.x + a.y); }
    __device__ static __forceinline__ double norm2_at(const V* A, uint32_t i, const AmpIO&) {
        const V a = A[i];
        return static_cast<double>(a.x) * a.x + static_cast<double>(a.y) * a.y;
    }
    __device__ static __forceinline__ void settle(V&) {}
    __device__ static __forceinline__ void store(V* out, int64_t o, V w, T scale, const AmpIO&) {
        if constexpr (sizeof(T) == 4) {
            out[o] = cmul2(w, make_float2(scale, scale));  // one packed FP32x2 multiply
        } else {
            w.x *= scale;
            w.y *= scale;
            out[o] = w;
        }
    }
    // output factor f (decode scale) as the kernel's scale; the shift is unused
    __device__ static __forceinline__ void out_scale(double f, T& scale, int& shift_out, int) {
        scale = static_cast<T>(f);
        shift_out = 0;
    }
};

template <>
struct AmpTraits<dfloat> {
    using V = dcomplex;
    static constexpr bool kDF = true;
    __device__ static __forceinline__ V load(const V* A, uint32_t i, const AmpIO& io) {
        if (io.raw_in) {
            const double2 d = reinterpret_cast<const double2*>(A)[i];
            return dc_make(df_from_double_shift(d.x, io.shift_in), df_from_double_shift(d.y, io.shift_in));
        }
        return A[i];
    }
    // sum of |v|^2: exact squares of the high parts (two_prod) plus 2 hi lo,
    // accumulated with two_sum, returned as FP64
    using NormAcc = dfloat;
    __device__ static __forceinline__ void norm_add1(NormAcc& a, dfloat z) {
        const float p = z.hi * z.hi;
        float e = __fmaf_rn(z.hi, z.hi, -p);
        e = __fmaf_rn(2.f * z.hi, z.lo, e);
        const dfloat s = two_sum(a.hi, p);
        a.hi = s.hi;
        a.lo += s.lo + e;
    }
    __device__ static __forceinline__ void norm_add(NormAcc& a, const V& v) {
        norm_add1(a, v.re());
        norm_add1(a, v.im());
    }
    __device__ static __forceinline__ double norm_done(NormAcc a) {
        return static_cast<double>(a.hi) + static_cast<double>(a.lo);
    }
    __device__ static __forceinline__ double norm2_at(const V* A, uint32_t i, const AmpIO& io) {
        NormAcc a(0.f, 0.f);
        norm_add(a, load(A, i, io));
        return norm_done(a);
    }
    __device__ static __forceinline__ void settle(V& v) { v = dc_norm(v); }
    // Only the last pass has an output scale (the others run with scale 1).
    __device__ static __forceinline__ void store(V* out, int64_t o, V w, dfloat scale, const AmpIO& io) {
        if (io.raw_out) {
            const dfloat re = df_mul(w.re(), scale), im = df_mul(w.im(), scale);
            double2 d;
            d.x = df_to_double_shift(re, io.shift_out);
            d.y = df_to_double_shift(im, io.shift_out);
            reinterpret_cast<double2*>(out)[o] = d;
        } else {
            out[o] = dc_norm(w);
        }
    }
    // f * 2^k = m * 2^(e + k) with m in [1/2, 1): the pair carries m, the FP64
    // conversion of the output adds e + k to the exponent
    __device__ static __forceinline__ void out_scale(double f, dfloat& scale, int& shift_out, int k) {
        int e = 0;
        const double m = frexp(f, &e);
        scale = dfloat(m);
        shift_out = (m == 0.0) ? 0 : e + k;
    }
};

// Exponent shift of the double-float range normalisation: the largest biased
// FP64 exponent of the input (written by the maximum-exponent pre-pass into
// the workspace's metadata) less the bias, so that the largest scaled
// component lies in [1, 2).  0 for an all-zero input.
__device__ __forceinline__ int df_shift_from_meta(const double* meta) {
    const int mx = reinterpret_cast<const int*>(meta)[4];
    return mx > 0 ? mx - 1023 : 0;
}

__device__ __forceinline__ void issue_tile_load(const PassParams& P, const CUtensorMap* map, int64_t tile,
                                                void* dstA, uint64_t* bar, uint32_t bytes) {
    mbar_arrive_expect_tx(bar, bytes);
    if (P.load_mode == 1) {
        const char* src = static_cast<const char*>(P.in) + static_cast<int64_t>(bytes) * tile;
        bulk_load_1d(dstA, src, bytes, bar);
    } else {
        int32_t c[5];
#pragma unroll
        for (int d = 0; d < 5; ++d) {
            const int len = P.dim_len[d];
            c[d] = len ? static_cast<int32_t>((tile >> P.dim_src[d]) & ((int64_t(1) << len) - 1)) : 0;
        }
        tma_load_5d(dstA, map, c, bar);
    }
}

// Logical bits of the tile coordinate and its output address offset.
__device__ __forceinline__ void tile_coords(const PassParams& P, int64_t tile, uint64_t& I_tile, int64_t& out_tile) {
    I_tile = 0;
    out_tile = 0;
    for (int sg = 0; sg < P.nseg; ++sg) {
        const TileSeg& G = P.seg[sg];
        const uint64_t v = (static_cast<uint64_t>(tile) >> G.src) & ((1ull << G.len) - 1ull);
        I_tile |= v << G.wire;
        if (G.out_rev)
            out_tile += static_cast<int64_t>((__brevll(v) >> (64 - G.len)) << (G.out - G.len + 1));
        else
            out_tile += static_cast<int64_t>(v << G.out);
    }
}

// U_e for every stage of one tile: thread i < nU computes entry i.
template <typename T, int DIR>
__device__ __forceinline__ void compute_tile_twiddles(const PassParams& P, int64_t tile,
                                                      typename Vec2<T>::type* Ubuf) {
    const int i = threadIdx.x;
    if (i >= P.nU || tile >= P.num_tiles) return;
    int s = 0;
    while (s + 1 < P.nstages && P.st[s + 1].uoff <= i) ++s;
    const StageDesc& S = P.st[s];
    const int e = i - S.uoff;
    uint64_t I_tile;
    int64_t dummy;
    tile_coords(P, tile, I_tile, dummy);
    const uint64_t beta = cross_phase(I_tile, P.n, S.wlo + S.r - 1, S.wlo + e, P.kk);
    Ubuf[i] = phase_turns<T, DIR>(beta, P.n);
}

// exp(DIR * 2 pi i beta / 2^n) as a double-float pair with FP32 operations
// only: the same exact reduction to the nearest quarter turn as phase_turns,
// then df_turns40 on the rest (tab: its 129-entry table).
template <int DIR>
__device__ __forceinline__ dcomplex phase_turns_df(uint64_t beta, int n, const dcomplex* tab) {
    const uint64_t b = (beta << (64 - n)) >> 24;  // beta mod 2^n, scaled to 2^40 per turn
    const uint64_t q4 = (b + (1ull << 37)) >> 38;
    const int64_t rem = static_cast<int64_t>(b) - static_cast<int64_t>(q4 << 38);
    const dcomplex z = df_turns40(rem, tab);
    const dfloat c = z.re(), s = z.im();
    dfloat x, y;
    switch (q4 & 3) {
        case 0: x = c; y = s; break;
        case 1: x = df_neg(s); y = c; break;
        case 2: x = df_neg(c); y = df_neg(s); break;
        default: x = s; y = df_neg(c); break;
    }
    if (DIR < 0) y = df_neg(y);
    return dc_make(x, y);
}

// The table of df_turns40 ((cos, sin) of 2 pi k / 2^10, k = 0..128), by the
// NT threads of a CTA (FP64 once per launch).
template <int NT>
__device__ __forceinline__ void build_turns40_table(dcomplex* tab) {
    for (int k = threadIdx.x; k <= 128; k += NT) {
        double s, c;
        sincospi(k * (1.0 / 512.0), &s, &c);
        tab[k] = dc_make(dfloat(c), dfloat(s));
    }
}

// compute_tile_twiddles for double-float amplitudes: the per-tile factors come
// from phase_turns_df, so that the FP64 pipe (1/64 of the FP32 rate) is off
// the path every tile takes.
template <int DIR>
__device__ __forceinline__ void compute_tile_twiddles_df(const PassParams& P, int64_t tile, dcomplex* Ubuf,
                                                         const dcomplex* tab) {
    const int i = threadIdx.x;
    if (i >= P.nU || tile >= P.num_tiles) return;
    int s = 0;
    while (s + 1 < P.nstages && P.st[s + 1].uoff <= i) ++s;
    const StageDesc& S = P.st[s];
    const int e = i - S.uoff;
    uint64_t I_tile;
    int64_t dummy;
    tile_coords(P, tile, I_tile, dummy);
    const uint64_t beta = cross_phase(I_tile, P.n, S.wlo + S.r - 1, S.wlo + e, P.kk);
    Ubuf[i] = phase_turns_df<DIR>(beta, P.n, tab);
}

// Build the group tables (pb, ob, cross-twiddle factors of the group's tile
// wires) of every stage of pass P into shared memory.
template <typename T, int DIR, int NT>
__device__ __forceinline__ void build_group_tables(const PassParams& P, GroupTab<typename Vec2<T>::type>& tab) {
    using V = typename Vec2<T>::type;
    const int tid = threadIdx.x;
    const int ntab = tab.ntab;
    for (int s = 0; s < P.nstages; ++s) {
        const StageDesc& S = P.st[s];
        const int ng = 1 << S.ngbits;
        const int nhi = ng > 32 ? ng >> 5 : 1;
        for (int i = tid; i < 32 + nhi; i += NT) {
            const int g = i < 32 ? (i < ng ? i : 0) : ((i - 32) << 5);
            uint32_t pb = 0;
            uint64_t iw = 0;
            int64_t ob = 0;
            for (int b = 0; b < S.ngbits; ++b) {
                if ((g >> b) & 1) {
                    const int p = S.gpos[b];
                    pb |= 1u << p;
                    iw |= 1ull << P.p_wire[p];
                    ob += int64_t(1) << P.p_out[p];
                }
            }
            const int idx = P.tab_off[s] + i;
            tab.pb[idx] = pb;
            tab.sb[idx] = swz<sizeof(V) == 8 ? 4 : 3>(pb);
            tab.ob[idx] = ob;
            for (int e = 0; e < P.ntw; ++e) {
                V w = cunit<V>();
                if (S.cross && e < S.r) w = phase_turns<T, DIR>(cross_phase(iw, P.n, S.wlo + S.r - 1, S.wlo + e, P.kk), P.n);
                tab.tw[e * ntab + idx] = w;
            }
        }
    }
}

// The same tables with one thread per (stage, entry, twiddle plane): the work
// of all stages is spread over the CTA, so a build costs about one bit loop
// and one phase evaluation per thread (the batched launch rebuilds them
// whenever a CTA's next item has another pass shape).
template <typename T, int DIR, int NT>
__device__ __forceinline__ void build_group_tables_wide(const PassParams& P, GroupTab<typename Vec2<T>::type>& tab) {
    using V = typename Vec2<T>::type;
    const int ntab = tab.ntab;
    const int ntw = P.ntw;
    int total = 0;
    for (int s = 0; s < P.nstages; ++s) {
        const int ng = 1 << P.st[s].ngbits;
        total += (32 + (ng > 32 ? ng >> 5 : 1)) * ntw;
    }
    for (int w = threadIdx.x; w < total; w += NT) {
        int s = 0, rem = w, nent = 0;
        for (; s < P.nstages; ++s) {
            const int ng = 1 << P.st[s].ngbits;
            nent = 32 + (ng > 32 ? ng >> 5 : 1);
            if (rem < nent * ntw) break;
            rem -= nent * ntw;
        }
        const StageDesc& S = P.st[s];
        const int e = rem / nent, i = rem - e * nent;  // consecutive threads: consecutive entries of one plane
        const int ng = 1 << S.ngbits;
        const int g = i < 32 ? (i < ng ? i : 0) : ((i - 32) << 5);
        uint32_t pb = 0;
        uint64_t iw = 0;
        int64_t ob = 0;
        for (int b = 0; b < S.ngbits; ++b) {
            if ((g >> b) & 1) {
                const int p = S.gpos[b];
                pb |= 1u << p;
                iw |= 1ull << P.p_wire[p];
                ob += int64_t(1) << P.p_out[p];
            }
        }
        const int idx = P.tab_off[s] + i;
        if (e == 0) {
            tab.pb[idx] = pb;
            tab.sb[idx] = swz<sizeof(V) == 8 ? 4 : 3>(pb);
            tab.ob[idx] = ob;
        }
        V tw = cunit<V>();
        if (S.cross && e < S.r) tw = phase_turns<T, DIR>(cross_phase(iw, P.n, S.wlo + S.r - 1, S.wlo + e, P.kk), P.n);
        tab.tw[e * ntab + idx] = tw;
    }
}

}  // namespace qft
