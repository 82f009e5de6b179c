// qft_real.cu -- real-input transforms of N = 2^n samples on the (n-1)-qubit
// complex QFT (the real-to-complex packing named as future work beside the
// paper's encode step, Sec. 3 step 1 / Sec. 6).
//
// Forward (R2C, numpy.fft.rfft): the N reals x are read as M = N/2 complex
// numbers z_m = x_{2m} + i x_{2m+1} (the same bytes), Z = DFT_M z is computed
// out of place into the output buffer by the complex plan, and one sweep
// separates the spectra of the even and odd samples and joins them:
//
//   E_k = (Z_k + conj Z_{M-k}) / 2,   O_k = (Z_k - conj Z_{M-k}) / (2i),
//   X_k = E_k + W^k O_k,   X_{M-k} = conj(E_k - W^k O_k),   W = e^{-2 pi i / N},
//
// for k = 0 .. M/2 (Z_M = Z_0), one thread per pair (k, M-k), in place.
//
// Inverse (C2R, numpy.fft.irfft): from X_0 .. X_M (a Hermitian half
// spectrum; only the real parts of X_0 and X_M are used) one sweep forms
//
//   A_k = X_k + conj X_{M-k},   B_k = (X_k - conj X_{M-k}) e^{+2 pi i k / N},
//   Z_k = A_k + i B_k,          Z_{M-k} = conj A_k + i conj B_k,
//
// into the output buffer, and the inverse complex QFT of M points in place
// leaves x_{2m} + i x_{2m+1} there: the N reals, in order.
//
// complex64 computes in FP32 with twiddles from the exact-phase sine/cosine;
// complex128 in FP64 with twiddles from two plan-owned tables (W^k =
// T1[k >> L0] T0[k mod 2^L0], built in FP64 on the host), so no FP64
// sine/cosine runs per element.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <new>
#include <vector>

#include "../../include/qftfft.h"
#include "plan_host.hpp"
#include "qft_device.cuh"

namespace qft {
namespace {

template <typename V> __device__ __forceinline__ V conj_(V a) { a.y = -a.y; return a; }
template <typename V, typename S> __device__ __forceinline__ V scal(V a, S f) { a.x *= f; a.y *= f; return a; }
// -i a
template <typename V> __device__ __forceinline__ V mul_mi(V a) { V r; r.x = a.y; r.y = -a.x; return r; }
// +i a
template <typename V> __device__ __forceinline__ V mul_pi(V a) { V r; r.x = -a.y; r.y = a.x; return r; }

// W^k = exp(DIR 2 pi i k / 2^n) for the element type.
template <typename T, int DIR>
__device__ __forceinline__ typename Vec2<T>::type twiddle(uint64_t k, int n, const double2* t0, const double2* t1,
                                                         int L0) {
    if constexpr (sizeof(T) == 4) {
        return phase_turns<float, DIR>(k, n);
    } else {
        const double2 a = t0[k & ((uint64_t(1) << L0) - 1)];
        const double2 b = t1[k >> L0];
        return cmul(a, b);
    }
}

// R2C separation sweep, in place on Z (M + 1 entries; Z[M] is written).
template <typename T>
__global__ void __launch_bounds__(256) qft_r2c_post_kernel(typename Vec2<T>::type* __restrict__ Z, uint64_t M,
                                                           int n, T f, const double2* t0, const double2* t1,
                                                           int L0) {
    using V = typename Vec2<T>::type;
    const uint64_t half = M >> 1;
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k <= half;
         k += uint64_t(gridDim.x) * blockDim.x) {
        const uint64_t km = (M - k) & (M - 1);
        const V zk = Z[k], zm = Z[km];
        const V E = scal(cadd(zk, conj_(zm)), T(0.5));
        const V O = scal(mul_mi(csub(zk, conj_(zm))), T(0.5));
        const V WO = cmul(twiddle<T, -1>(k, n, t0, t1, L0), O);
        const V a = scal(cadd(E, WO), f);
        const V b = scal(conj_(csub(E, WO)), f);
        if (k == 0) {
            Z[0] = a;
            Z[M] = b;
        } else {
            Z[k] = a;
            if (k != half) Z[km] = b;
        }
    }
}

// C2R merge sweep: X (M + 1 entries) -> Z (M entries), out of place.
template <typename T>
__global__ void __launch_bounds__(256) qft_c2r_pre_kernel(const typename Vec2<T>::type* __restrict__ X,
                                                          typename Vec2<T>::type* __restrict__ Z, uint64_t M, int n,
                                                          T f, const double2* t0, const double2* t1, int L0) {
    using V = typename Vec2<T>::type;
    const uint64_t half = M >> 1;
    for (uint64_t k = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; k <= half;
         k += uint64_t(gridDim.x) * blockDim.x) {
        V xk = X[k], xm = X[M - k];
        if (k == 0) {  // only the real parts of X_0 and X_M enter
            xk.y = T(0);
            xm.y = T(0);
        }
        const V A = cadd(xk, conj_(xm));
        const V B = cmul(csub(xk, conj_(xm)), twiddle<T, +1>(k, n, t0, t1, L0));
        Z[k] = scal(cadd(A, mul_pi(B)), f);
        if (k != 0 && k != half) Z[M - k] = scal(cadd(conj_(A), mul_pi(conj_(B))), f);
    }
}

int launch_grid(uint64_t work, int num_sms) {
    uint64_t b = (work + 255) / 256;
    const uint64_t cap = uint64_t(num_sms) * 8;
    if (b > cap) b = cap;
    return static_cast<int>(b < 1 ? 1 : b);
}

double scale_factor(int mode, int n) {
    switch (mode) {
        case QFT_SCALE_UNNORM: return 1.0;
        case QFT_SCALE_UNITARY: return std::ldexp(1.0, -n / 2) * ((n & 1) ? std::sqrt(0.5) : 1.0);
        case QFT_SCALE_INV_N: return std::ldexp(1.0, -n);
        default: return -1.0;
    }
}

}  // namespace
}  // namespace qft

struct qft_rplan_s {
    qft_plan_t sub = nullptr;  // n - 1 qubits, exact, natural order
    int n = 0, dir = -1, dtype = 0, num_sms = 148;
    double2* t0 = nullptr;     // complex128: exp(dir 2 pi i j / N), j < 2^L0
    double2* t1 = nullptr;     //             exp(dir 2 pi i j 2^L0 / N), j <= 2^(n-2-L0)
    int L0 = 0;
    ~qft_rplan_s() {
        if (sub) qft_plan_destroy(sub);
        if (t0) cudaFree(t0);
        if (t1) cudaFree(t1);
    }
};

extern "C" {

int qft_rplan_create(qft_rplan_t* out, int n, int direction, int dtype, const qft_opts* opts) {
    if (!out) return QFT_ERR_BAD_ARG;
    *out = nullptr;
    if (dtype != QFT_C64 && dtype != QFT_C128) return QFT_ERR_BAD_ARG;
    if (direction != QFT_FORWARD && direction != QFT_INVERSE) return QFT_ERR_BAD_ARG;
    if (n < 2 || n > (dtype == QFT_C64 ? 34 : 33)) return QFT_ERR_BAD_ARG;
    qft_opts o{};
    if (opts) o = *opts;
    if (o.order != QFT_ORDER_NATURAL) return QFT_ERR_UNSUPPORTED;  // the sweeps need natural order
    if (o.precision >= QFT_PREC_TF32 && o.precision <= QFT_PREC_FP16X3) return QFT_ERR_UNSUPPORTED;
    qft_rplan_s* rp = new (std::nothrow) qft_rplan_s();
    if (!rp) return QFT_ERR_NOMEM;
    rp->n = n;
    rp->dir = direction;
    rp->dtype = dtype;
    int rc = qft_plan_create(&rp->sub, n - 1, -1, direction, dtype, &o);
    if (rc != QFT_OK) {
        delete rp;
        return rc;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            rp->num_sms = sms;
    } else {
        cudaGetLastError();
    }
    if (dtype == QFT_C128) {
        // k runs over 0 .. M/2 = 2^(n-2): low table 2^L0 entries, high table up to 2^(n-2-L0) + 1
        const int kb = n - 2;
        rp->L0 = (kb + 1) / 2;
        const size_t n0 = size_t(1) << rp->L0, n1 = (size_t(1) << (kb - rp->L0)) + 1;
        std::vector<double2> h0(n0), h1(n1);
        const double sgn = direction;
        // angle 2 pi j / 2^n for j < 2^n: the ratio is exact, one rounding in the product
        auto w = [&](uint64_t j) {
            const double a = 2.0 * M_PI * std::ldexp(static_cast<double>(j), -n);
            double2 r;
            r.x = std::cos(a);
            r.y = sgn * std::sin(a);
            return r;
        };
        for (size_t j = 0; j < n0; ++j) h0[j] = w(j);
        for (size_t j = 0; j < n1; ++j) h1[j] = w(uint64_t(j) << rp->L0);
        if (cudaMalloc(&rp->t0, n0 * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&rp->t1, n1 * sizeof(double2)) != cudaSuccess ||
            cudaMemcpy(rp->t0, h0.data(), n0 * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(rp->t1, h1.data(), n1 * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            delete rp;
            return QFT_ERR_NOMEM;
        }
    }
    *out = rp;
    return QFT_OK;
}

int qft_rplan_destroy(qft_rplan_t rp) {
    delete rp;
    return QFT_OK;
}

size_t qft_rplan_workspace_size(qft_rplan_t rp) { return rp ? qft_workspace_size(rp->sub) : 0; }

int qft_rplan_execute(qft_rplan_t rp, const void* d_in, void* d_out, void* d_workspace, int scale_mode,
                      qft_stream_t stream) {
    if (!rp || !d_in || !d_out || !d_workspace) return QFT_ERR_BAD_ARG;
    if (d_in == static_cast<const void*>(d_out)) return QFT_ERR_BAD_ARG;
    const double f = qft::scale_factor(scale_mode, rp->n);
    if (f < 0) return QFT_ERR_BAD_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const uint64_t M = uint64_t(1) << (rp->n - 1);
    const int grid = qft::launch_grid(M / 2 + 1, rp->num_sms);
    cudaError_t e;
    if (rp->dir == QFT_FORWARD) {
        int rc = qft_execute_oop(rp->sub, d_in, d_out, d_workspace, nullptr, QFT_SCALE_UNNORM, stream);
        if (rc != QFT_OK) return rc;
        if (rp->dtype == QFT_C64)
            qft::qft_r2c_post_kernel<float><<<grid, 256, 0, st>>>(static_cast<float2*>(d_out), M, rp->n,
                                                                  static_cast<float>(f), nullptr, nullptr, 0);
        else
            qft::qft_r2c_post_kernel<double><<<grid, 256, 0, st>>>(static_cast<double2*>(d_out), M, rp->n, f,
                                                                   rp->t0, rp->t1, rp->L0);
        e = cudaGetLastError();
        return e == cudaSuccess ? QFT_OK : qft::set_cuda_error(e);
    }
    if (rp->dtype == QFT_C64)
        qft::qft_c2r_pre_kernel<float><<<grid, 256, 0, st>>>(static_cast<const float2*>(d_in),
                                                             static_cast<float2*>(d_out), M, rp->n,
                                                             static_cast<float>(f), nullptr, nullptr, 0);
    else
        qft::qft_c2r_pre_kernel<double><<<grid, 256, 0, st>>>(static_cast<const double2*>(d_in),
                                                              static_cast<double2*>(d_out), M, rp->n, f, rp->t0,
                                                              rp->t1, rp->L0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return qft::set_cuda_error(e);
    return qft_execute(rp->sub, d_out, d_workspace, nullptr, QFT_SCALE_UNNORM, stream);
}

}  // extern "C"
