// qft_qpe.cu -- quantum phase estimation on the QFT engine (the eigenvalue
// estimation the paper names as the next use of a QFT state-vector
// simulator: a state with overlap on the eigenvectors of an operator, a
// sequence of controlled evolutions, and a Fourier readout, Sec. 6).
//
// The operator is given in its eigenbasis: d = 2^d_bits eigenvectors with
// eigenphases theta_j (in turns, U u_j = e^{2 pi i theta_j} u_j) and the input
// state's overlaps c_j.  The joint register is m counting qubits (the low index
// bits) times the d system states (the high bits).  Starting from
// H^{(x)m}|0> (x) sum_j c_j |u_j>, the controlled evolutions C-U^{2^k} (control
// counting qubit k) multiply the amplitude of |y>|u_j> by e^{2 pi i theta_j 2^k}
// for every set bit k of y, so after all m of them
//
//     psi[j 2^m + y] = c_j e^{2 pi i phi_j(y)} / sqrt(2^m),
//     phi_j(y) = sum_k y_k frac(theta_j 2^k) = frac(theta_j y)  (mod 1),
//
// which qft_qpe_prepare writes in one sweep.  The phase is kept in 64-bit
// fixed point (2^64 = one turn): Theta_j = frac(theta_j) 2^64, and the sum of
// the controlled evolutions' phases is the integer product Theta_j y mod 2^64,
// exact for every y; only the final sine/cosine rounds.  The
// Fourier readout is the transform of the counting qubits with
// omega = e^{-2 pi i / 2^m} (the paper's QFT convention, which is the
// textbook inverse QFT of phase estimation): a subset plan
// (qft_plan_create_subset with w0 = 0, n = m, n_addr = m + d_bits, FORWARD,
// scale QFT_SCALE_UNITARY).  qft_qpe_probabilities then sums |psi|^2 over the
// system states: P(x) = sum_j |psi[j 2^m + x]|^2, the distribution of the
// counting register, which peaks at x ~ theta_j 2^m.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/qftfft.h"
#include "plan_host.hpp"
#include "qft_phase64.cuh"

namespace qft {
namespace {

// Per eigenvector j, once: Theta_j = frac(theta_j) 2^64 (64-bit fixed point,
// one turn = 2^64) and the amplitude c_j / sqrt(2^m) rounded to the element
// type, so that the per-amplitude sweep does no FP64 arithmetic (GB300's FP64
// pipe runs at a small fraction of its FP32 rate).
template <typename V, typename T>
__global__ void qpe_setup_kernel(const double* __restrict__ theta, const double2* __restrict__ coef, int d,
                                 double inv_sqrt_M, uint64_t* __restrict__ th64, V* __restrict__ cs) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    const double f = theta[j] - floor(theta[j]);  // exact
    const double t = ldexp(f, 64);                // exact scaling; < 2^64
    th64[j] = t >= 18446744073709551615.0 ? 0ull : __double2ull_rn(t);
    const double2 c = coef[j];
    V v;
    v.x = static_cast<T>(c.x * inv_sqrt_M);
    v.y = static_cast<T>(c.y * inv_sqrt_M);
    cs[j] = v;
}

// exp(2 pi i phase / 2^64): reduced exactly in integers to the nearest quarter
// turn, the rest (|x| <= 1/8 turn) in the element type (qft_phase64.cuh).
template <typename T>
__device__ __forceinline__ void phase64(uint64_t phase, T& c, T& s) {
    if constexpr (sizeof(T) == 4) {
        phase64_f32(phase, c, s);
    } else {
        int64_t rem;
        const uint64_t q4 = phase64_quarter(phase, rem);
        T sn, cs;
        sincospi(static_cast<double>(rem) * (1.0 / 9223372036854775808.0), &sn, &cs);
        rotate_quarters(q4, cs, sn, c, s);
    }
}

template <typename V, typename T>
__global__ void __launch_bounds__(256) qpe_prepare_kernel(V* __restrict__ psi, int m, int d,
                                                          const uint64_t* __restrict__ th64,
                                                          const V* __restrict__ cs) {
    const uint64_t M = uint64_t(1) << m, total = M * uint64_t(d);
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < total; i += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t y = i & (M - 1);
        const int j = static_cast<int>(i >> m);
        T c, s;
        phase64<T>(th64[j] * y, c, s);  // frac(theta_j y), exact mod 2^64
        const V a = cs[j];
        V r;
        r.x = a.x * c - a.y * s;
        r.y = a.x * s + a.y * c;
        psi[i] = r;
    }
}

// P(x) = sum_j |psi[j 2^m + x]|^2.  Each thread takes kXU counting values
// (one grid stride apart) and kJU system states per step, so kXU * kJU reads
// are in flight per thread.  complex64 sums each step's kJU squares in FP32
// (a relative error of at most ~2 kJU 2^-24, below the state's own rounding)
// and carries the total in FP64; complex128 sums in FP64 throughout.
constexpr int kXU = 4, kJU = 4;

template <typename V, typename T>
__global__ void __launch_bounds__(256) qpe_prob_kernel(const V* __restrict__ psi, int m, int d, double* __restrict__ prob) {
    const uint64_t M = uint64_t(1) << m;
    const uint64_t S = uint64_t(gridDim.x) * blockDim.x;
    for (uint64_t x0 = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; x0 < M; x0 += kXU * S) {
        double p[kXU];
#pragma unroll
        for (int u = 0; u < kXU; ++u) p[u] = 0.0;
        int j = 0;
        for (; j + kJU <= d; j += kJU) {
            V a[kXU][kJU];
#pragma unroll
            for (int u = 0; u < kXU; ++u) {
                const uint64_t x = x0 + u * S;
#pragma unroll
                for (int v = 0; v < kJU; ++v) {
                    if (x < M) a[u][v] = psi[uint64_t(j + v) * M + x];
                    else a[u][v].x = a[u][v].y = T(0);
                }
            }
#pragma unroll
            for (int u = 0; u < kXU; ++u) {
                T t = T(0);
#pragma unroll
                for (int v = 0; v < kJU; ++v) {
                    t = fma(a[u][v].x, a[u][v].x, t);
                    t = fma(a[u][v].y, a[u][v].y, t);
                }
                p[u] += static_cast<double>(t);
            }
        }
        for (; j < d; ++j) {  // d < kJU
#pragma unroll
            for (int u = 0; u < kXU; ++u) {
                const uint64_t x = x0 + u * S;
                if (x < M) {
                    const V a = psi[uint64_t(j) * M + x];
                    p[u] += static_cast<double>(fma(a.x, a.x, a.y * a.y));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kXU; ++u) {
            const uint64_t x = x0 + u * S;
            if (x < M) prob[x] = p[u];
        }
    }
}

int grid_for(uint64_t work) {
    uint64_t b = (work + 255) / 256;
    if (b > 152 * 8) b = 152 * 8;
    return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace
}  // namespace qft

extern "C" {

size_t qft_qpe_workspace_size(int m, int d_bits) {
    if (m < 1 || d_bits < 0 || m > 40 || d_bits > 20) return 0;
    return (size_t(1) << d_bits) * (sizeof(uint64_t) + sizeof(double2));
}

int qft_qpe_prepare(void* d_state, int m, int d_bits, const double* d_theta, const void* d_coef, int dtype,
                    void* d_workspace, qft_stream_t stream) {
    if (!d_state || !d_theta || !d_coef || !d_workspace) return QFT_ERR_BAD_ARG;
    if (reinterpret_cast<uintptr_t>(d_workspace) % 16 != 0) return QFT_ERR_BAD_ARG;
    if (dtype != QFT_C64 && dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    const int nmax = dtype == QFT_C64 ? 34 : 33;
    if (m < 1 || d_bits < 0 || d_bits > 20 || m + d_bits > nmax) return QFT_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int d = 1 << d_bits;
    // workspace: d scaled coefficients (16 bytes each, complex128-sized for
    // both dtypes) followed by the d fixed-point phases
    void* cs = d_workspace;
    uint64_t* th64 = reinterpret_cast<uint64_t*>(static_cast<char*>(d_workspace) + size_t(d) * sizeof(double2));
    const double inv = 1.0 / std::sqrt(static_cast<double>(uint64_t(1) << m));
    const int sblocks = (d + 255) / 256;
    const auto* coef = static_cast<const double2*>(d_coef);
    const int grid = qft::grid_for((uint64_t(1) << m) * d);
    if (dtype == QFT_C64) {
        qft::qpe_setup_kernel<float2, float><<<sblocks, 256, 0, st>>>(d_theta, coef, d, inv, th64, static_cast<float2*>(cs));
        qft::qpe_prepare_kernel<float2, float><<<grid, 256, 0, st>>>(static_cast<float2*>(d_state), m, d, th64,
                                                                     static_cast<const float2*>(cs));
    } else {
        qft::qpe_setup_kernel<double2, double><<<sblocks, 256, 0, st>>>(d_theta, coef, d, inv, th64,
                                                                        static_cast<double2*>(cs));
        qft::qpe_prepare_kernel<double2, double><<<grid, 256, 0, st>>>(static_cast<double2*>(d_state), m, d, th64,
                                                                       static_cast<const double2*>(cs));
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QFT_OK : qft::set_cuda_error(e);
}

int qft_qpe_probabilities(const void* d_state, int m, int d_bits, int dtype, double* d_prob, qft_stream_t stream) {
    if (!d_state || !d_prob) return QFT_ERR_BAD_ARG;
    if (dtype != QFT_C64 && dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    if (m < 1 || d_bits < 0 || d_bits > 20 || m + d_bits > 34) return QFT_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int grid = qft::grid_for(((uint64_t(1) << m) + qft::kXU - 1) / qft::kXU);
    if (dtype == QFT_C64)
        qft::qpe_prob_kernel<float2, float><<<grid, 256, 0, st>>>(static_cast<const float2*>(d_state), m, 1 << d_bits,
                                                                  d_prob);
    else
        qft::qpe_prob_kernel<double2, double><<<grid, 256, 0, st>>>(static_cast<const double2*>(d_state), m,
                                                                    1 << d_bits, d_prob);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? QFT_OK : qft::set_cuda_error(e);
}

}  // extern "C"
