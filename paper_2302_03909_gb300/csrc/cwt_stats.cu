// Statistics of a computed W: the environment-dependent wavelet power
// spectrum (Wang & He, arXiv:2302.03909, Sec. 5, Eqs. 41 and 43) and the
// inverse CWT (Sec. 2, Eqs. 5 and 6).  Host entry points are declared in
// include/cwt.h; plan internals come from cwt_plan_impl.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "../../include/cwt.h"
#include "cwt_kernels.cuh"
#include "cwt_plan_impl.h"

using namespace cwtk;

namespace {

constexpr int kEnvThreads = 256;
constexpr int64_t kEnvChunk = 32768;

// grid (chunks, S): |W|^2 summed over the chunk's positions with delta > 0 and
// delta < 0; CTAs of row 0 also count the positions of each environment.
template <typename D>
__global__ void __launch_bounds__(kEnvThreads) k_env_rows(const void* __restrict__ W, const void* __restrict__ delta,
                                                          int64_t N, int is_complex, double* __restrict__ part,
                                                          int64_t* __restrict__ counts) {
    __shared__ double red[2 * (kEnvThreads / 32)];
    __shared__ int cnt[2];
    const int s = blockIdx.y, c = blockIdx.x;
    const int64_t n0 = (int64_t)c * kEnvChunk, n1 = n0 + kEnvChunk < N ? n0 + kEnvChunk : N;
    if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
    __syncthreads();
    float ap = 0.f, an = 0.f;
    int cp = 0, cn = 0;
    for (int64_t n = n0 + threadIdx.x; n < n1; n += kEnvThreads) {
        float v2;
        if (is_complex) {
            const float2 v = __ldg(&((const float2*)W)[(int64_t)s * N + n]);
            v2 = fmaf(v.x, v.x, v.y * v.y);
        } else {
            const float v = __ldg(&((const float*)W)[(int64_t)s * N + n]);
            v2 = v * v;
        }
        const D dl = __ldg(&((const D*)delta)[n]);   // sign tested in the field's own precision
        if (dl > D(0)) { ap += v2; cp++; }
        else if (dl < D(0)) { an += v2; cn++; }
    }
    double sp, sn;
    block_sum2<kEnvThreads>(ap, an, &sp, &sn, red);
    if (s == 0) {
        atomicAdd(&cnt[0], cp);   // integer counts: order-independent
        atomicAdd(&cnt[1], cn);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[((int64_t)s * gridDim.x + c) * 2 + 0] = sp;
        part[((int64_t)s * gridDim.x + c) * 2 + 1] = sn;
        if (s == 0) {
            counts[2 * c + 0] = cnt[0];
            counts[2 * c + 1] = cnt[1];
        }
    }
}

__global__ void k_env_finalize(const double* __restrict__ part, const int64_t* __restrict__ counts, int chunks,
                               int S, int64_t N, double* __restrict__ p_pos, double* __restrict__ p_neg,
                               double* __restrict__ frac) {
    const int s = blockIdx.x;
    double ap = 0.0, an = 0.0;
    int64_t cp = 0, cn = 0;
    for (int i = threadIdx.x; i < chunks; i += 32) {
        ap += part[((int64_t)s * chunks + i) * 2 + 0];
        an += part[((int64_t)s * chunks + i) * 2 + 1];
        cp += counts[2 * i + 0];
        cn += counts[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ap += __shfl_xor_sync(0xffffffffu, ap, o);
        an += __shfl_xor_sync(0xffffffffu, an, o);
        cp += __shfl_xor_sync(0xffffffffu, cp, o);
        cn += __shfl_xor_sync(0xffffffffu, cn, o);
    }
    if (threadIdx.x == 0) {
        p_pos[s] = cp ? ap / (double)cp : 0.0;
        p_neg[s] = cn ? an / (double)cn : 0.0;
        if (s == 0) {
            frac[0] = (double)cp / (double)N;
            frac[1] = (double)cn / (double)N;
        }
    }
}

// f(n) = sum_s coef[s] * W(s, n)  (real part; coef folds 1/K, sqrt(w), the
// trapezoid weight and the Morlet's factor 2)
__global__ void k_icwt(const void* __restrict__ W, int64_t N, int S, int is_complex,
                       const double* __restrict__ coef, float* __restrict__ out) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    double acc = 0.0;
    if (is_complex) {
        const float2* Wc = (const float2*)W;
        for (int s = 0; s < S; s++) acc += coef[s] * (double)__ldg(&Wc[(int64_t)s * N + n]).x;
    } else {
        const float* Wr = (const float*)W;
        for (int s = 0; s < S; s++) acc += coef[s] * (double)__ldg(&Wr[(int64_t)s * N + n]);
    }
    out[n] = (float)acc;
}

constexpr double kPi = 3.14159265358979323846264338327950288;

// K_psi = int_0^inf psi_hat(k) / k dk (Table 2; Morlet by quadrature in ln k)
double admissibility(int wavelet, double omega0) {
    switch (wavelet) {
    case CWT_WAVELET_GDW: return 2.0 * std::pow(8.0 * kPi / 9.0, 0.25);
    case CWT_WAVELET_CBSW: return 0.5 * std::sqrt(15.0 / 62.0) * (27.0 * std::log(3.0) - 32.0 * std::log(2.0));
    case CWT_WAVELET_CWGDW: return 4.0 * std::pow(kPi, 0.25) / std::sqrt(1.0 + 5.0 * std::exp(1.0));
    }
    // psi_hat(k) / k dk = psi_hat(e^t) dt; trapezoid in t (exponentially decaying ends)
    const double w2 = omega0 * omega0;
    const double cn = std::pow(kPi, -0.25) / std::sqrt(1.0 - 2.0 * std::exp(-0.75 * w2) + std::exp(-w2));
    const double t0 = std::log(1e-12), t1 = std::log(omega0 + 40.0);
    const int n = 400000;
    const double h = (t1 - t0) / n;
    double acc = 0.0;
    for (int i = 0; i <= n; i++) {
        const double k = std::exp(t0 + i * h);
        const double v = std::exp(-0.5 * (k - omega0) * (k - omega0)) - std::exp(-0.5 * (k * k + w2));
        acc += (i == 0 || i == n) ? 0.5 * v : v;
    }
    return std::sqrt(2.0 * kPi) * cn * acc * h;
}

}  // namespace

extern "C" cwt_status cwt_env_power(cwt_plan* plan, const void* W_dev, const void* delta_dev, double* p_pos_dev,
                                    double* p_neg_dev, double* frac_dev, void* stream) {
    if (!plan || !W_dev || !delta_dev || !p_pos_dev || !p_neg_dev || !frac_dev) return CWT_ERR_INVALID_ARG;
    cwt_status st = plan_check_device(plan);
    if (st != CWT_OK) return st;
    const int64_t chunks = (plan->N + kEnvChunk - 1) / kEnvChunk;
    if (chunks > 65535 || plan->S > 65535) return plan_fail(plan, CWT_ERR_UNSUPPORTED, "signal too long");
    if (!plan->d_env_part) {
        if (cudaMalloc((void**)&plan->d_env_part, (size_t)chunks * plan->S * 2 * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void**)&plan->d_env_cnt, (size_t)chunks * 2 * sizeof(int64_t)) != cudaSuccess)
            return plan_fail(plan, CWT_ERR_OOM, "cudaMalloc of the environment partial sums");
    }
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((unsigned)chunks, (unsigned)plan->S);
    const int cplx = plan->wavelet == CWT_WAVELET_MORLET;
    if (plan->opts.input_dtype == CWT_INPUT_F64)
        k_env_rows<double><<<grid, kEnvThreads, 0, s>>>(W_dev, delta_dev, plan->N, cplx, plan->d_env_part, plan->d_env_cnt);
    else
        k_env_rows<float><<<grid, kEnvThreads, 0, s>>>(W_dev, delta_dev, plan->N, cplx, plan->d_env_part, plan->d_env_cnt);
    if (cudaGetLastError() != cudaSuccess) return plan_fail(plan, CWT_ERR_CUDA, "k_env_rows launch");
    k_env_finalize<<<plan->S, 32, 0, s>>>(plan->d_env_part, plan->d_env_cnt, (int)chunks, plan->S, plan->N, p_pos_dev,
                                         p_neg_dev, frac_dev);
    if (cudaGetLastError() != cudaSuccess) return plan_fail(plan, CWT_ERR_CUDA, "k_env_finalize launch");
    return CWT_OK;
}

extern "C" cwt_status cwt_icwt(cwt_plan* plan, const void* W_dev, float* f_out_dev, void* stream) {
    if (!plan || !W_dev || !f_out_dev) return CWT_ERR_INVALID_ARG;
    if (plan->S < 2) return plan_fail(plan, CWT_ERR_INVALID_ARG, "the inverse needs at least two scales");
    cwt_status st = plan_check_device(plan);
    if (st != CWT_OK) return st;
    if (!plan->d_icwt_coef) {
        // trapezoid weights in x = ln w over the scales sorted by w = w~ / dx
        const int S = plan->S;
        std::vector<int> idx(S);
        std::iota(idx.begin(), idx.end(), 0);
        std::sort(idx.begin(), idx.end(), [&](int a, int b) { return plan->w_tilde[a] < plan->w_tilde[b]; });
        std::vector<double> coef(S, 0.0);
        const double K = admissibility(plan->wavelet, plan->opts.omega0);
        const double factor = (plan->wavelet == CWT_WAVELET_MORLET ? 2.0 : 1.0) / K;
        for (int i = 0; i < S; i++) {
            const double w = plan->w_tilde[idx[i]] / plan->opts.dx;
            const double xl = std::log(plan->w_tilde[idx[i > 0 ? i - 1 : i]] / plan->opts.dx);
            const double xr = std::log(plan->w_tilde[idx[i < S - 1 ? i + 1 : i]] / plan->opts.dx);
            coef[idx[i]] = factor * std::sqrt(w) * 0.5 * (xr - xl);   // int W / sqrt(w) dw = int W sqrt(w) dln w
        }
        if (cudaMalloc((void**)&plan->d_icwt_coef, S * sizeof(double)) != cudaSuccess)
            return plan_fail(plan, CWT_ERR_OOM, "cudaMalloc of the inverse weights");
        if (cudaMemcpy(plan->d_icwt_coef, coef.data(), S * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
            return plan_fail(plan, CWT_ERR_CUDA, "upload of the inverse weights");
    }
    const int threads = 256;
    const int64_t blocks = (plan->N + threads - 1) / threads;
    k_icwt<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(W_dev, plan->N, plan->S,
                                                                  plan->wavelet == CWT_WAVELET_MORLET,
                                                                  plan->d_icwt_coef, f_out_dev);
    if (cudaGetLastError() != cudaSuccess) return plan_fail(plan, CWT_ERR_CUDA, "k_icwt launch");
    return CWT_OK;
}
