// qft_mc.cu -- the Monte Carlo backend of Sec. 6: estimates of single output
// bins of the (A)QFT "in the sum-over-histories style".
//
// The amplitude <y|U_k|x> is a sum over input indices j of x_j times the
// phase that the kept controlled rotations give the path j -> y (the
// closed-form matrix element exp(s 2 pi i phase(j, y) / N) / sqrt(N), with
// phase(j, y) = sum of j_a y_b 2^(a+b) over n-1-k <= a+b <= n-1, mod 2^n;
// j y mod 2^n for the exact transform).  Drawing input indices with
// importance weights gives unbiased estimates of single bins and of the power
// spectrum, at a cost set by the number of samples instead of 2^n.
//
//   qft_mc_prepare  the proposal, exact in integers: per index an integer
//                   weight q_j = floor(m_j 2^S / 2^(E+1)) + 1 (0 for x_j = 0),
//                   m_j = max(|Re x_j|, |Im x_j|), 2^E <= max m < 2^(E+1),
//                   S = min(62 - n, 52), formed by shifting the significand of
//                   m_j (q_j >= 1 for every nonzero x_j, so the estimator is
//                   unbiased); prefix sums of q in blocks of 4096 indices and
//                   the blocks' exclusive offsets, T = sum q.
//   qft_mc_sample   for each given uniform u: t = floor(u 2^53 T / 2^53), the
//                   index j with C_{j-1} <= t < C_j (two binary searches), and
//                   the weight w = x_j T / q_j.
//   qft_mc_bins     per bin y: the mean of z = w exp(s 2 pi i phase(j, y)/N)
//                   / sqrt(N), the unbiased power estimate
//                   (|sum z|^2 - sum |z|^2) / (M (M - 1)) and the standard
//                   error of the mean.
//
// The proposal and the draws are integer operations and the weights one
// correctly rounded FP64 division and product, so they are the same bits on
// any IEEE machine; the bins
// evaluate the phase exactly in integers and the sine and cosine in FP32,
// and sum in FP32 over runs of 32 samples and in FP64 beyond.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/qftfft.h"
#include "plan_host.hpp"
#include "qft_device.cuh"
#include "qft_phase64.cuh"

namespace qft {
namespace {

constexpr int kMcChunk = 4096;          // indices per prefix-sum block
constexpr int kMcScanThreads = 256;     // 16 indices per thread
constexpr int kMcSampleBlocks = 1024;   // blocks of the sampling kernel (partial sums of |w|^2)
constexpr int kMcBinsPerBlock = 8;      // bins evaluated together per sample load
constexpr int kMcMaxSplit = 32;         // sample chunks per bin group
constexpr int kMcMaxBins = 1 << 16;

struct McLayout {
    size_t meta, bsum, wpart, part, cdf, total;
};

__host__ __device__ inline size_t mc_align(size_t b) { return (b + 255) / 256 * 256; }

// Workspace of a proposal over K entries: the sections the bins read first,
// at offsets that do not depend on K (so qft_mc_bins takes any workspace),
// then the K-sized ones.
__host__ __device__ inline McLayout mc_layout(int64_t K) {
    const int64_t nb = (K + kMcChunk - 1) / kMcChunk;
    McLayout L;
    L.meta = 0;                                                         // T, max magnitude bits
    L.wpart = 256;                                                      // sum |w|^2 per sampling block
    L.part = L.wpart + mc_align(size_t(kMcSampleBlocks) * 8);           // bin partial sums
    L.bsum = L.part + mc_align(size_t(kMcMaxSplit) * kMcMaxBins * 16);  // nb block offsets
    L.cdf = L.bsum + mc_align(size_t(nb) * 8);                          // local inclusive prefix sums
    L.total = L.cdf + mc_align(size_t(K) * 8);
    return L;
}

// ceil(log2 K), K >= 1: the proposal's S = min(62 - lg, 52) keeps T below 2^63.
inline int mc_lg(int64_t K) {
    int lg = 0;
    while ((int64_t(1) << lg) < K) ++lg;
    return lg;
}

// The bits of |f| as an FP64 number, by integer operations (the FP32 -> FP64
// conversion is exact; doing it in integers keeps it off the FP64 pipe).
__device__ __forceinline__ uint64_t abs_f32_as_f64_bits(float f) {
    const uint32_t fb = __float_as_uint(f) & 0x7FFFFFFFu;
    if (fb == 0u) return 0ull;
    const uint32_t e = fb >> 23, m = fb & 0x7FFFFFu;
    if (e == 255u) return (0x7FFull << 52) | (static_cast<uint64_t>(m) << 29);
    if (e == 0u) {  // subnormal: m 2^-149, normalised
        const int p = 31 - __clz(m);  // highest set bit, 0..22
        return (static_cast<uint64_t>(p + 874) << 52) | ((static_cast<uint64_t>(m) << (52 - p)) & 0xFFFFFFFFFFFFFull);
    }
    return (static_cast<uint64_t>(e + 896u) << 52) | (static_cast<uint64_t>(m) << 29);
}

// The magnitude used by the proposal, max(|Re|, |Im|) as FP64 bits: for
// non-negative doubles the integer order of the bits is the value order.
__device__ __forceinline__ uint64_t mag_bits(float2 v) {
    const uint64_t a = abs_f32_as_f64_bits(v.x), b = abs_f32_as_f64_bits(v.y);
    return a > b ? a : b;
}
__device__ __forceinline__ uint64_t mag_bits(double2 v) {
    const uint64_t a = static_cast<uint64_t>(__double_as_longlong(v.x)) & 0x7FFFFFFFFFFFFFFFull;
    const uint64_t b = static_cast<uint64_t>(__double_as_longlong(v.y)) & 0x7FFFFFFFFFFFFFFFull;
    return a > b ? a : b;
}
// q_j from the bits of m_j: the significand shifted to the common scale, plus one.
__device__ __forceinline__ uint64_t mc_weight(uint64_t bits, int emax, int S) {
    if (bits == 0) return 0;
    const int eb = static_cast<int>(bits >> 52);
    const int e = eb > 0 ? eb : 1;
    const uint64_t sig = (bits & 0xFFFFFFFFFFFFFull) | (eb > 0 ? (1ull << 52) : 0ull);
    const int sh = emax - e + 53 - S;
    return (sh < 64 ? sig >> sh : 0ull) + 1ull;
}
__device__ __forceinline__ double2 as_d2(float2 v) { return make_double2(v.x, v.y); }
__device__ __forceinline__ double2 as_d2(double2 v) { return v; }

__device__ __forceinline__ uint64_t shfl_xor_u64(uint64_t v, int o) {
    const uint32_t lo = __shfl_xor_sync(0xffffffffu, static_cast<uint32_t>(v), o);
    const uint32_t hi = __shfl_xor_sync(0xffffffffu, static_cast<uint32_t>(v >> 32), o);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl_up_u64(uint64_t v, int o) {
    const uint32_t lo = __shfl_up_sync(0xffffffffu, static_cast<uint32_t>(v), o);
    const uint32_t hi = __shfl_up_sync(0xffffffffu, static_cast<uint32_t>(v >> 32), o);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

// max_j m_j (as bits) into *maxbits (zeroed by the caller).
template <typename V>
__global__ void mc_max_kernel(const V* __restrict__ x, int64_t N, unsigned long long* maxbits) {
    uint64_t m = 0;
    for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < N; j += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t b = mag_bits(x[j]);
        m = b > m ? b : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t b = shfl_xor_u64(m, o);
        m = b > m ? b : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(maxbits, static_cast<unsigned long long>(m));
}

// Exclusive scan of one value per thread across a block of NT threads
// (warp shuffles, then the warp totals); returns the thread's exclusive
// prefix and the block total in *total.
template <int NT>
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* warp_tot, uint64_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = shfl_up_u64(incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint64_t t = lane < NT / 32 ? warp_tot[lane] : 0;
        uint64_t ti = t;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = shfl_up_u64(ti, o);
            if (lane >= o) ti += y;
        }
        if (lane < NT / 32) warp_tot[lane] = ti - t;  // exclusive prefix of the warp totals
        if (lane == NT / 32 - 1) warp_tot[NT / 32] = ti;
    }
    __syncthreads();
    const uint64_t r = warp_tot[w] + incl - v;
    *total = warp_tot[NT / 32];
    __syncthreads();
    return r;
}

// q_j and its inclusive prefix within each block of kMcChunk indices
// (cdf[j]); the block's total into bsum[b].  Loads and stores are coalesced
// (index i * 256 + t of the block for thread t); the scan runs on 16
// consecutive indices per thread through shared memory, padded by one word
// per 16 so that those reads and writes are free of bank conflicts.
template <typename V>
__global__ void __launch_bounds__(kMcScanThreads)
    mc_quant_scan_kernel(const V* __restrict__ x, int64_t N, int lg, const unsigned long long* maxbits,
                         uint64_t* __restrict__ cdf, uint64_t* __restrict__ bsum) {
    constexpr int IT = kMcChunk / kMcScanThreads;
    constexpr int NT = kMcScanThreads;
    __shared__ uint64_t warp_tot[NT / 32 + 1];
    __shared__ uint64_t qs[kMcChunk + kMcChunk / 16];
    const uint64_t mb = *maxbits;
    const int emax = static_cast<int>(mb >> 52) > 0 ? static_cast<int>(mb >> 52) : 1;
    const int S = 62 - lg < 52 ? 62 - lg : 52;
    const int64_t base = blockIdx.x * int64_t(kMcChunk);
    const int t = threadIdx.x;
    auto pad = [](int e) { return e + (e >> 4); };
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = i * NT + t;
        qs[pad(e)] = base + e < N ? mc_weight(mag_bits(x[base + e]), emax, S) : 0ull;
    }
    __syncthreads();
    uint64_t q[IT];
    uint64_t run = 0;
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        run += qs[pad(t * IT + i)];
        q[i] = run;  // thread-local inclusive prefix
    }
    uint64_t total;
    const uint64_t off = block_exclusive_scan<NT>(run, warp_tot, &total);
#pragma unroll
    for (int i = 0; i < IT; ++i) qs[pad(t * IT + i)] = off + q[i];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int e = i * NT + t;
        if (base + e < N) cdf[base + e] = qs[pad(e)];
    }
    if (t == 0) bsum[blockIdx.x] = total;
}

// In place: bsum[b] <- sum of bsum[0 .. b-1]; the grand total T into meta[0].
__global__ void __launch_bounds__(1024) mc_scan_offsets_kernel(uint64_t* bsum, int64_t nb, uint64_t* meta) {
    constexpr int IT = 8;
    __shared__ uint64_t warp_tot[1024 / 32 + 1];
    uint64_t carry = 0;
    for (int64_t c0 = 0; c0 < nb; c0 += 1024 * IT) {
        const int64_t j0 = c0 + int64_t(threadIdx.x) * IT;
        uint64_t v[IT];
        uint64_t run = 0;
#pragma unroll
        for (int i = 0; i < IT; ++i) {
            v[i] = j0 + i < nb ? bsum[j0 + i] : 0;
            const uint64_t t = v[i];
            v[i] = run;  // exclusive within the thread
            run += t;
        }
        uint64_t total;
        const uint64_t base = block_exclusive_scan<1024>(run, warp_tot, &total);
#pragma unroll
        for (int i = 0; i < IT; ++i)
            if (j0 + i < nb) bsum[j0 + i] = carry + base + v[i];
        carry += total;
    }
    if (threadIdx.x == 0) meta[0] = carry;
}

// One draw per uniform: the entry's input index (pos[s] for a sparse list,
// else s) and its weight; per block the sum of |w|^2.
template <typename V>
__global__ void __launch_bounds__(256)
    mc_sample_kernel(const V* __restrict__ x, int64_t N, const int64_t* __restrict__ pos,
                     const uint64_t* __restrict__ cdf, const uint64_t* __restrict__ boff, int64_t nb,
                     const uint64_t* __restrict__ meta, const double* __restrict__ u, int64_t m,
                     int64_t* __restrict__ idx, double2* __restrict__ w, double* __restrict__ wpart) {
    __shared__ double red[8];
    const uint64_t T = meta[0];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        if (T == 0) {
            idx[i] = 0;
            w[i] = make_double2(0.0, 0.0);
            continue;
        }
        const uint64_t u53 = __double2ull_rz(__dmul_rn(u[i], 9007199254740992.0));  // u 2^53, exact
        const uint64_t hi = __umul64hi(u53, T), lo = u53 * T;
        const uint64_t t = (hi << 11) | (lo >> 53);  // floor(u53 T / 2^53) < T
        // the block: the last b with boff[b] <= t
        int64_t a = 0, b = nb - 1;
        while (a < b) {
            const int64_t mid = a + (b - a + 1) / 2;
            if (boff[mid] <= t) a = mid; else b = mid - 1;
        }
        const uint64_t r = t - boff[a];
        const int64_t base = a * kMcChunk;
        int64_t c = base + kMcChunk - 1 < N - 1 ? base + kMcChunk - 1 : N - 1;
        int64_t s = base;  // the first index with cdf > r
        while (s < c) {
            const int64_t mid = s + (c - s) / 2;
            if (cdf[mid] > r) c = mid; else s = mid + 1;
        }
        const uint64_t q = cdf[s] - (s > base ? cdf[s - 1] : 0);
        const double f = __ddiv_rn(__ull2double_rn(T), __ull2double_rn(q));
        const double2 v = as_d2(x[s]);
        const double2 wv = make_double2(__dmul_rn(v.x, f), __dmul_rn(v.y, f));
        idx[i] = pos ? pos[s] : s;
        w[i] = wv;
        acc = __dadd_rn(acc, __dadd_rn(__dmul_rn(wv.x, wv.x), __dmul_rn(wv.y, wv.y)));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k];
        wpart[blockIdx.x] = s;
    }
}

// exp(DIR 2 pi i F / 2^64) from the top 32 bits fh of a 64-bit fixed-point
// phase F (one turn = 2^64; the low word is below 2^-32 of a turn): the
// nearest quarter turn exactly in 32-bit integers, the remainder rounded to
// 22 bits (|x| <= 1/4 half-turn) and converted to FP32 by the 2^23-offset
// trick (an integer add and an exact FP32 subtraction: no conversion
// instruction, which for 64-bit integers runs on the FP64 pipe), then the
// Taylor sine and cosine of qft_phase64.cuh (no range reduction needed).
template <int DIR>
__device__ __forceinline__ float2 mc_phase_hi(uint32_t fh) {
    const uint32_t q4 = (fh + (1u << 29)) >> 30;                       // nearest quarter turn (mod 4)
    const int32_t rem = static_cast<int32_t>(fh - (q4 << 30));          // |rem| <= 2^29
    const int32_t r = (rem + 128) >> 8;                                 // rounded, |r| <= 2^21
    const float xr = __int_as_float(0x4B400000 + r) - 12582912.0f;      // = r exactly
    float sn, cs;
    sincospi_quarter(xr * (1.0f / 8388608.0f), sn, cs);                 // r / 2^23 half-turns
    // q4 quarter turns more, without branches: (c, s) = (cs, sn), (-sn, cs),
    // (-cs, -sn), (sn, -cs) for q4 mod 4 = 0, 1, 2, 3 (signs by the sign bit)
    const uint32_t q = q4 & 3u;
    const float tc = (q & 1u) ? sn : cs, ts = (q & 1u) ? cs : sn;
    const float c = __int_as_float(__float_as_int(tc) ^ static_cast<int>(((q + 1u) & 2u) << 30));
    const uint32_t sneg = (q & 2u) ^ (DIR < 0 ? 2u : 0u);
    const float s = __int_as_float(__float_as_int(ts) ^ static_cast<int>(sneg << 30));
    return make_float2(c, s);
}

// Bins: block (g, c) takes the kMcBinsPerBlock bins of group g and the
// samples of chunk c; per sample it forms the integer phase of each bin
// (exact: j y; range k: the windows of the set bits of y), the FP32
// sine/cosine and the product with the FP32 weight, summed in FP32 over
// runs of 32 samples and in FP64 beyond; the block's sums go to part[c][bin].
template <int DIR, bool EXACT>
__global__ void __launch_bounds__(256)
    mc_bins_kernel(int n, int kk, const int64_t* __restrict__ idx, const double2* __restrict__ w, int64_t m,
                   const int64_t* __restrict__ ys, int nbins, double2* __restrict__ part) {
    constexpr int B = kMcBinsPerBlock;
    __shared__ uint64_t win[64];
    __shared__ double2 red[256 / 32][B];
    if (!EXACT && threadIdx.x < n) {
        const int b = threadIdx.x;  // output bit b: input bits [max(0, n-1-kk-b), n-1-b]
        int lo = n - 1 - kk - b;
        if (lo < 0) lo = 0;
        const int hi = n - 1 - b;
        win[b] = ((hi - lo + 1) >= 64 ? ~0ull : ((1ull << (hi - lo + 1)) - 1ull)) << lo;
    }
    __syncthreads();
    const int g0 = blockIdx.x * B;
    // the bins as 64-bit fixed-point factors: the exact phase j y / 2^n turns
    // is j (y << (64 - n)) mod 2^64
    uint64_t y[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        y[b] = g0 + b < nbins ? static_cast<uint64_t>(ys[g0 + b]) : 0ull;
        if (EXACT) y[b] <<= (64 - n);
    }
    const int64_t per = (m + gridDim.y - 1) / gridDim.y;
    const int64_t s0 = blockIdx.y * per, s1 = s0 + per < m ? s0 + per : m;
    double2 dacc[B];
    float2 facc[B];
#pragma unroll
    for (int b = 0; b < B; ++b) {
        dacc[b] = make_double2(0.0, 0.0);
        facc[b] = make_float2(0.f, 0.f);
    }
    int cnt = 0;
    // one sample ahead: its index and weight load while this one is evaluated
    int64_t i = s0 + threadIdx.x;
    uint64_t jn = 0;
    double2 wn = make_double2(0.0, 0.0);
    if (i < s1) {
        jn = static_cast<uint64_t>(idx[i]);
        wn = w[i];
    }
    for (; i < s1; i += blockDim.x) {
        const uint64_t j = jn;
        const float2 wf = make_float2(static_cast<float>(wn.x), static_cast<float>(wn.y));
        if (i + blockDim.x < s1) {
            jn = static_cast<uint64_t>(idx[i + blockDim.x]);
            wn = w[i + blockDim.x];
        }
#pragma unroll
        for (int b = 0; b < B; ++b) {
            uint32_t fh;
            if constexpr (EXACT) {
                // the high word of the low 64 bits of j * y'
                const uint32_t jl = static_cast<uint32_t>(j), jh = static_cast<uint32_t>(j >> 32);
                const uint32_t yl = static_cast<uint32_t>(y[b]), yh = static_cast<uint32_t>(y[b] >> 32);
                fh = __umulhi(jl, yl) + jl * yh + jh * yl;
            } else {
                uint64_t p = 0;
#pragma unroll 1
                for (int bit = 0; bit < n; ++bit)
                    if ((y[b] >> bit) & 1ull) p += (j & win[bit]) << bit;
                fh = static_cast<uint32_t>((p << (64 - n)) >> 32);
            }
            const float2 e = mc_phase_hi<DIR>(fh);
            facc[b].x += wf.x * e.x - wf.y * e.y;
            facc[b].y += wf.x * e.y + wf.y * e.x;
        }
        if (++cnt == 32) {
#pragma unroll
            for (int b = 0; b < B; ++b) {
                dacc[b].x += facc[b].x;
                dacc[b].y += facc[b].y;
                facc[b] = make_float2(0.f, 0.f);
            }
            cnt = 0;
        }
    }
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
#pragma unroll
    for (int b = 0; b < B; ++b) {
        double sx = dacc[b].x + facc[b].x, sy = dacc[b].y + facc[b].y;
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_xor_sync(0xffffffffu, sx, o);
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
        }
        if (lane == 0) red[wq][b] = make_double2(sx, sy);
    }
    __syncthreads();
    if (threadIdx.x < B && g0 + threadIdx.x < nbins) {
        double sx = 0.0, sy = 0.0;
        for (int k = 0; k < 256 / 32; ++k) {
            sx += red[k][threadIdx.x].x;
            sy += red[k][threadIdx.x].y;
        }
        part[size_t(blockIdx.y) * nbins + g0 + threadIdx.x] = make_double2(sx, sy);
    }
}

// Per bin: the chunks' sums in order, then mean, power estimate, standard error.
__global__ void mc_finalize_kernel(int n, int64_t m, int nbins, int split, const double2* __restrict__ part,
                                   const double* __restrict__ wpart, int nwpart, double* __restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    double sx = 0.0, sy = 0.0;
    for (int c = 0; c < split; ++c) {
        sx += part[size_t(c) * nbins + b].x;
        sy += part[size_t(c) * nbins + b].y;
    }
    double q = 0.0;
    for (int k = 0; k < nwpart; ++k) q += wpart[k];
    const double inv_n = ldexp(1.0, -n);  // |z|^2 = |w|^2 / N
    const double inv_root = sqrt(inv_n);
    sx *= inv_root;
    sy *= inv_root;
    q *= inv_n;
    const double M = static_cast<double>(m);
    const double mr = sx / M, mi = sy / M;
    out[4 * b] = mr;
    out[4 * b + 1] = mi;
    out[4 * b + 2] = m > 1 ? (sx * sx + sy * sy - q) / (M * (M - 1.0)) : 0.0;
    const double v = m > 1 ? (q / M - (mr * mr + mi * mi)) / (M - 1.0) : 0.0;
    out[4 * b + 3] = v > 0.0 ? sqrt(v) : 0.0;
}

int mc_launch_error() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QFT_OK : set_cuda_error(e);
}

}  // namespace
}  // namespace qft

using namespace qft;

namespace qft {
namespace {

// The proposal over the K entries of x (dense: K = 2^n, lg = n).
int mc_prepare_list(int64_t K, int lg, int dtype, const void* d_x, void* d_workspace, cudaStream_t st) {
    const McLayout L = mc_layout(K);
    char* ws = static_cast<char*>(d_workspace);
    uint64_t* meta = reinterpret_cast<uint64_t*>(ws + L.meta);
    uint64_t* bsum = reinterpret_cast<uint64_t*>(ws + L.bsum);
    uint64_t* cdf = reinterpret_cast<uint64_t*>(ws + L.cdf);
    const int64_t nb = (K + kMcChunk - 1) / kMcChunk;
    cudaError_t e = cudaMemsetAsync(meta, 0, 256, st);
    if (e != cudaSuccess) return set_cuda_error(e);
    auto* mx = reinterpret_cast<unsigned long long*>(meta + 1);
    const int gmax = static_cast<int>(K / 256 < 152 * 16 ? (K + 255) / 256 : 152 * 16);
    if (dtype == QFT_C64) {
        mc_max_kernel<<<gmax, 256, 0, st>>>(static_cast<const float2*>(d_x), K, mx);
        mc_quant_scan_kernel<<<static_cast<unsigned>(nb), kMcScanThreads, 0, st>>>(static_cast<const float2*>(d_x), K,
                                                                                   lg, mx, cdf, bsum);
    } else {
        mc_max_kernel<<<gmax, 256, 0, st>>>(static_cast<const double2*>(d_x), K, mx);
        mc_quant_scan_kernel<<<static_cast<unsigned>(nb), kMcScanThreads, 0, st>>>(static_cast<const double2*>(d_x), K,
                                                                                   lg, mx, cdf, bsum);
    }
    mc_scan_offsets_kernel<<<1, 1024, 0, st>>>(bsum, nb, meta);
    return mc_launch_error();
}

int mc_sample_list(int64_t K, int dtype, const int64_t* d_pos, const void* d_x, const void* d_workspace,
                   const double* d_u, int64_t m, int64_t* d_index, double* d_weight, cudaStream_t st) {
    const McLayout L = mc_layout(K);
    const char* ws = static_cast<const char*>(d_workspace);
    const uint64_t* meta = reinterpret_cast<const uint64_t*>(ws + L.meta);
    const uint64_t* boff = reinterpret_cast<const uint64_t*>(ws + L.bsum);
    const uint64_t* cdf = reinterpret_cast<const uint64_t*>(ws + L.cdf);
    double* wpart = reinterpret_cast<double*>(const_cast<char*>(ws) + L.wpart);
    const int64_t nb = (K + kMcChunk - 1) / kMcChunk;
    auto* w2 = reinterpret_cast<double2*>(d_weight);
    if (dtype == QFT_C64)
        mc_sample_kernel<<<kMcSampleBlocks, 256, 0, st>>>(static_cast<const float2*>(d_x), K, d_pos, cdf, boff, nb,
                                                          meta, d_u, m, d_index, w2, wpart);
    else
        mc_sample_kernel<<<kMcSampleBlocks, 256, 0, st>>>(static_cast<const double2*>(d_x), K, d_pos, cdf, boff, nb,
                                                          meta, d_u, m, d_index, w2, wpart);
    return mc_launch_error();
}

bool misaligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; }

}  // namespace
}  // namespace qft

extern "C" {

size_t qft_mc_workspace_size(int n) {
    if (n < 1 || n > 34) return 0;
    return mc_layout(int64_t(1) << n).total;
}

size_t qft_mc_sparse_workspace_size(int64_t K) {
    if (K < 1 || K > (int64_t(1) << 34)) return 0;
    return mc_layout(K).total;
}

int qft_mc_prepare(int n, int dtype, const void* d_x, void* d_workspace, qft_stream_t stream) {
    if (!d_x || !d_workspace || (dtype != QFT_C64 && dtype != QFT_C128)) return QFT_ERR_BAD_ARG;
    if (n < 1 || n > (dtype == QFT_C64 ? 34 : 33)) return QFT_ERR_BAD_ARG;
    if (misaligned(d_x, 16) || misaligned(d_workspace, 256)) return QFT_ERR_BAD_ARG;
    return mc_prepare_list(int64_t(1) << n, n, dtype, d_x, d_workspace, reinterpret_cast<cudaStream_t>(stream));
}

int qft_mc_prepare_sparse(int64_t K, int dtype, const void* d_vals, void* d_workspace, qft_stream_t stream) {
    if (!d_vals || !d_workspace || (dtype != QFT_C64 && dtype != QFT_C128)) return QFT_ERR_BAD_ARG;
    if (K < 1 || K > (int64_t(1) << 34)) return QFT_ERR_BAD_ARG;
    if (misaligned(d_vals, 16) || misaligned(d_workspace, 256)) return QFT_ERR_BAD_ARG;
    return mc_prepare_list(K, mc_lg(K), dtype, d_vals, d_workspace, reinterpret_cast<cudaStream_t>(stream));
}

int qft_mc_sample(int n, int dtype, const void* d_x, const void* d_workspace, const double* d_uniforms, int64_t m,
                  int64_t* d_index, double* d_weight, qft_stream_t stream) {
    if (!d_x || !d_workspace || !d_uniforms || !d_index || !d_weight || m < 1) return QFT_ERR_BAD_ARG;
    if (dtype != QFT_C64 && dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    if (n < 1 || n > (dtype == QFT_C64 ? 34 : 33)) return QFT_ERR_BAD_ARG;
    if (misaligned(d_x, 16) || misaligned(d_workspace, 256) || misaligned(d_uniforms, 8) ||
        misaligned(d_index, 8) || misaligned(d_weight, 16))
        return QFT_ERR_BAD_ARG;
    return mc_sample_list(int64_t(1) << n, dtype, nullptr, d_x, d_workspace, d_uniforms, m, d_index, d_weight,
                          reinterpret_cast<cudaStream_t>(stream));
}

int qft_mc_sample_sparse(int64_t K, int dtype, const int64_t* d_pos, const void* d_vals, const void* d_workspace,
                         const double* d_uniforms, int64_t m, int64_t* d_index, double* d_weight,
                         qft_stream_t stream) {
    if (!d_pos || !d_vals || !d_workspace || !d_uniforms || !d_index || !d_weight || m < 1) return QFT_ERR_BAD_ARG;
    if (dtype != QFT_C64 && dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    if (K < 1 || K > (int64_t(1) << 34)) return QFT_ERR_BAD_ARG;
    if (misaligned(d_pos, 8) || misaligned(d_vals, 16) || misaligned(d_workspace, 256) ||
        misaligned(d_uniforms, 8) || misaligned(d_index, 8) || misaligned(d_weight, 16))
        return QFT_ERR_BAD_ARG;
    return mc_sample_list(K, dtype, d_pos, d_vals, d_workspace, d_uniforms, m, d_index, d_weight,
                          reinterpret_cast<cudaStream_t>(stream));
}

int qft_mc_bins(int n, int k, int direction, const int64_t* d_index, const double* d_weight, int64_t m,
                const int64_t* d_bins, int nbins, const void* d_workspace, double* d_out, qft_stream_t stream) {
    if (!d_index || !d_weight || !d_workspace || !d_out || m < 1 || nbins < 0 || nbins > kMcMaxBins)
        return QFT_ERR_BAD_ARG;
    if (nbins > 0 && !d_bins) return QFT_ERR_BAD_ARG;
    if (n < 1 || n > 62 || (direction != QFT_FORWARD && direction != QFT_INVERSE)) return QFT_ERR_BAD_ARG;
    if (misaligned(d_index, 8) || misaligned(d_weight, 16) || misaligned(d_bins, 8) || misaligned(d_out, 8) ||
        misaligned(d_workspace, 256))
        return QFT_ERR_BAD_ARG;
    if (nbins == 0) return QFT_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const McLayout L = mc_layout(1);  // the sections the bins use sit at fixed offsets
    char* ws = static_cast<char*>(const_cast<void*>(d_workspace));
    auto* part = reinterpret_cast<double2*>(ws + L.part);
    const double* wpart = reinterpret_cast<const double*>(ws + L.wpart);
    const int kk = (k < 0 || k > n - 1) ? n - 1 : k;
    const bool exact = kk >= n - 1;
    const int groups = (nbins + kMcBinsPerBlock - 1) / kMcBinsPerBlock;
    // about eight waves of two 256-thread blocks per SM, for balance
    int split = (16 * 152 + groups - 1) / groups;
    if (split > kMcMaxSplit) split = kMcMaxSplit;
    if (int64_t(split) > (m + 255) / 256) split = static_cast<int>((m + 255) / 256);
    if (split < 1) split = 1;
    const dim3 grid(groups, split);
    const auto* w2 = reinterpret_cast<const double2*>(d_weight);
    if (direction < 0) {
        if (exact) mc_bins_kernel<-1, true><<<grid, 256, 0, st>>>(n, kk, d_index, w2, m, d_bins, nbins, part);
        else mc_bins_kernel<-1, false><<<grid, 256, 0, st>>>(n, kk, d_index, w2, m, d_bins, nbins, part);
    } else {
        if (exact) mc_bins_kernel<+1, true><<<grid, 256, 0, st>>>(n, kk, d_index, w2, m, d_bins, nbins, part);
        else mc_bins_kernel<+1, false><<<grid, 256, 0, st>>>(n, kk, d_index, w2, m, d_bins, nbins, part);
    }
    mc_finalize_kernel<<<(nbins + 127) / 128, 128, 0, st>>>(n, m, nbins, split, part, wpart, kMcSampleBlocks, d_out);
    return mc_launch_error();
}

}  // extern "C"
