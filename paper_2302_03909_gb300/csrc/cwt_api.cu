// Host side of the GB300 FFTCWT: planner, workspace, launches, plan-time
// tuning, batches of grouped launches and the C ABI declared in
// include/cwt.h.  Transform definition: Wang & He (RASTI 2023,
// arXiv:2302.03909), Sec. 3.1, Eqs. 8-10; power spectrum Eq. 42.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <set>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "../../include/cwt.h"
#include "cwt_kernels.cuh"
#include "cwt_tables.cuh"
#include "cwt_bluestein.cuh"
#include "cwt_tc.cuh"
#include "cwt_plan_impl.h"

using namespace cwtk;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kMaxLogM = 25;           // M <= 2^25 (zero boundary of N = 2^24)
constexpr int kBandMaxLog = 10;        // band kernels up to L = 1024 when M > kLmax
constexpr int kWideLog = 10;           // pass-2 DFT length of wide scales (M <= 2^23)
constexpr size_t kWideBatchBytes = size_t(32) << 20;   // intermediate per wide launch; one per stream
// the tile pipeline of pass 2 pays a fill and drain per launch: larger launches
// (more tiles per CTA) by default
constexpr size_t kWideBatchBytesTc = size_t(128) << 20;

// ----------------------------------------------------------- launch shapes

// tiles of T columns per CTA of the W-writing kernels: as many as keep the
// grid at >= kMinCtas CTAs (two per SM: the band value table and the job set-up
// are paid once per CTA), at most kMaxD
constexpr int kMaxD = 8;
constexpr int kPackMinLog = 4;             // real-input forward by the M/2-point packed form from M = 16
constexpr int kMinCtas = 152 * 2;
int pick_D(int64_t tiles_total, int min_ctas) {
    int64_t d = tiles_total / min_ctas;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kMaxD, d));
}

const Tables& tables() {
    static const Tables t = [] {
        Tables x;
        std::memset((void*)&x, 0, sizeof(x));
        fill_band_tables(x);
        fill_p1_tables(x);
        fill_wide_tables(x);
        fill_fwd_tables(x);
        fill_tc_tables(x);
        return x;
    }();
    return t;
}

int ilog2(int64_t v) { int l = 0; while ((int64_t(1) << l) < v) l++; return l; }
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// FP64 wavelet spectra of Table 2 for planning, up to the constant factor
double psi_hat_shape(int wavelet, double omega0, double u) {
    if (wavelet == CWT_WAVELET_GDW) return u * u * std::exp(-u * u);
    if (wavelet == CWT_WAVELET_CBSW) {
        if (u == 0.0) return 0.0;
        double sn = std::sin(0.5 * u), s2 = sn * sn;
        return s2 * s2 * s2 / (u * u * u * u);
    }
    if (wavelet == CWT_WAVELET_CWGDW)
        return u * 0.5 * ((u - 1.0) * std::exp(u - 0.5 * u * u) + (u + 1.0) * std::exp(-u - 0.5 * u * u));
    return std::exp(-0.5 * (u - omega0) * (u - omega0)) - std::exp(-0.5 * (u * u + omega0 * omega0));
}

double wavelet_cn(int wavelet, double omega0) {
    if (wavelet == CWT_WAVELET_GDW) return std::pow(18.0 * kPi, -0.25);
    if (wavelet == CWT_WAVELET_CBSW) return std::sqrt(30.0 / 31.0);
    if (wavelet == CWT_WAVELET_CWGDW) return std::sqrt(8.0 / (1.0 + 5.0 * std::exp(1.0))) / std::pow(kPi, 0.25);
    double w2 = omega0 * omega0;
    return std::pow(kPi, -0.25) / std::sqrt(1.0 - 2.0 * std::exp(-0.75 * w2) + std::exp(-w2));
}

// psi_hat(u) = C * shape(u): C = 8 sqrt(pi) C_N (GDW), sqrt(2 pi) C_N (Morlet)
double wavelet_spectrum_const(int wavelet, double omega0) {
    double cn = wavelet_cn(wavelet, omega0);
    if (wavelet == CWT_WAVELET_GDW) return 8.0 * std::sqrt(kPi) * cn;
    if (wavelet == CWT_WAVELET_CBSW) return 64.0 * cn;
    return std::sqrt(2.0 * kPi) * cn;   // Morlet, CW-GDW
}

// [u_lo, u_hi] outside which |psi_hat| < eps * max |psi_hat|
void wavelet_band_scan(int wavelet, double omega0, double eps, double* u_lo, double* u_hi) {
    // the CBSW spectrum only decays as u^-4: scan further, more coarsely
    const bool slow = wavelet == CWT_WAVELET_CBSW;
    const double step = slow ? 1.0 / 64.0 : 1.0 / 1024.0, U = slow ? 8192.0 : 80.0;
    double mx = 0.0;
    for (double u = -U; u <= U; u += step) mx = std::max(mx, std::fabs(psi_hat_shape(wavelet, omega0, u)));
    double lo = U, hi = -U;
    for (double u = -U; u <= U; u += step) {
        if (std::fabs(psi_hat_shape(wavelet, omega0, u)) >= eps * mx) {
            lo = std::min(lo, u);
            hi = std::max(hi, u);
        }
    }
    if (lo > hi) { lo = hi = 0.0; }
    *u_lo = lo - 2 * step;
    *u_hi = hi + 2 * step;
}

// the scan depends only on (wavelet, omega0, eps): plans of one shape family reuse it
void wavelet_band(int wavelet, double omega0, double eps, double* u_lo, double* u_hi) {
    static std::mutex mu;
    static std::map<std::tuple<int, double, double>, std::pair<double, double>> memo;
    const auto key = std::make_tuple(wavelet, omega0, eps);
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = memo.find(key);
        if (it != memo.end()) {
            *u_lo = it->second.first;
            *u_hi = it->second.second;
            return;
        }
    }
    wavelet_band_scan(wavelet, omega0, eps, u_lo, u_hi);
    std::lock_guard<std::mutex> lock(mu);
    memo[key] = {*u_lo, *u_hi};
}

}  // namespace

// The spectrum over all M unsigned bins k = b + L a (F(k) for k <= M/2, conj
// F(M - k) above: real signal), transposed to Ft[b A + a] so that the wide
// scales' pass 1 reads each column b contiguously.  32 x 32 tiles through
// shared memory; grid (ceil(L / 32), ceil(A / 32)), block (32, 8).
struct TransposeArgs {
    const float2* Fp;
    float2* Ft;
    int32_t M, L, A, pad_;
};
__device__ __forceinline__ void spec_transpose_body(const TransposeArgs& ta, const Cta c) {
    const float2* __restrict__ Fp = ta.Fp;
    float2* __restrict__ Ft = ta.Ft;
    const int M = ta.M, L = ta.L, A = ta.A;
    __shared__ float2 tile[32][33];
    const int b0 = c.x * 32, a0 = c.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int i = ty; i < 32; i += 8) {
        const int a = a0 + i, b = b0 + tx;
        if (a < A && b < L) {
            const int k = b + L * a;
            float2 f;
            if (k <= (M >> 1)) {
                f = __ldg(&Fp[k]);
            } else {
                f = __ldg(&Fp[M - k]);
                f.y = -f.y;
            }
            tile[i][tx] = f;
        }
    }
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
        const int b = b0 + i, a = a0 + tx;
        if (a < A && b < L) Ft[(int64_t)b * A + a] = tile[tx][i];
    }
}
static __global__ void k_spec_transpose(TransposeArgs a) { spec_transpose_body(a, cta_plain()); }
static __global__ void k_spec_transpose_g(GroupMap g) {
    Cta c;
    const TransposeArgs& a = group_args<TransposeArgs>(g, c);
    spec_transpose_body(a, c);
}

// ------------------------------------------------ zero boundary, short wavelets
//
// For a scale whose dilated wavelet is negligible beyond E samples (E <= N/4,
// E <= M - N), the zero-padded transform (length M) restricted to n < N is the
// linear convolution of f with h(j) = sqrt(w~ dx) psi(w~ j) (Eq. 7), and the
// periodic N-point transform differs from it only by the wrapped terms:
//   W_zero(n) = W_N(n) - sum_{j=n+1}^{E} h(j) f(N + n - j),          n < E,
//   W_zero(n) = W_N(n) - sum_{j=-E}^{n-N} h(j) f(n - N - j),          n >= N - E.
// Such rows are computed by a periodic child plan and corrected here.

struct EdgeRow { int32_t E; int32_t h_off; };
constexpr int kEdgeThreads = 256;
constexpr int64_t kEdgeMax = 4096;           // largest E handled this way

// grid (2 * chunks, rows): block b corrects outputs i in [64 c, 64 c + 64) of
// one edge (b even: left, n = i; b odd: right, n = N - E + i), i < E.  With
// k the term index, the two sums are sliding dot products:
//   left:  corr(i) = sum_{k=0}^{E-1-i} f(N-1-k) h(i+1+k),
//   right: corr(i) = sum_{k=0}^{i}     h(-E+k)  f(i-k),
// taken over tiles of kEdgeKT terms staged in shared memory; the 4 threads of
// an output take a quarter of each tile and their sums are added in a fixed
// order.  With power, each block records its change of sum |W|^2.
constexpr int kEdgeOut = 64;                 // outputs per block
constexpr int kEdgeSplit = kEdgeThreads / kEdgeOut;
constexpr int kEdgeKT = 512;

__device__ __forceinline__ float load_f(const void* signal, int f64, int64_t m) {
    return f64 ? (float)__ldg(&((const double*)signal)[m]) : __ldg(&((const float*)signal)[m]);
}

struct EdgeFixArgs {
    const void* signal;
    void* W;
    const float2* h;
    const EdgeRow* rows;
    double* delta;
    int64_t N;
    int32_t sig_f64, do_power;
};
template <bool CPLX>
__device__ __forceinline__ void edge_fix_body(const EdgeFixArgs& ea, const Cta c) {
    const void* __restrict__ signal = ea.signal;
    const int sig_f64 = ea.sig_f64;
    const int64_t N = ea.N;
    void* W = ea.W;
    const float2* __restrict__ h = ea.h;
    const EdgeRow* __restrict__ rows = ea.rows;
    double* __restrict__ delta = ea.delta;
    __shared__ float fs[kEdgeKT + kEdgeOut];
    __shared__ float2 hs[kEdgeKT + kEdgeOut];
    __shared__ float2 part[kEdgeSplit][kEdgeOut];
    __shared__ double red[2 * (kEdgeThreads / 32)];
    const int r = c.y;
    const EdgeRow er = rows[r];
    const int E = er.E;
    const bool left = (c.x & 1) == 0;
    const int i0 = (c.x >> 1) * kEdgeOut;
    const int o = threadIdx.x % kEdgeOut, q = threadIdx.x / kEdgeOut;
    const int i = i0 + o;
    const float2* hr = h + er.h_off + E;              // hr[j], j in [-E, E]
    float dpow = 0.f;
    if (i0 < E) {                                     // block-uniform
        // terms of this block: left k in [0, E - 1 - i0], right k in [0, i0 + 63]
        const int kmax = left ? E - 1 - i0 : min(i0 + kEdgeOut - 1, E - 1);
        const int klast = left ? E - 1 - i : i;       // this output's last term
        float cr = 0.f, ci = 0.f;
        for (int k0 = 0; k0 <= kmax; k0 += kEdgeKT) {
            __syncthreads();
            if (left) {
                // fs[kk] = f(N-1-k0-kk), hs[u] = h(i0+1+k0+u), u < KT + 63
                for (int u = threadIdx.x; u < kEdgeKT; u += kEdgeThreads) {
                    const int k = k0 + u;
                    fs[u] = k <= kmax ? load_f(signal, sig_f64, N - 1 - k) : 0.f;
                }
                for (int u = threadIdx.x; u < kEdgeKT + kEdgeOut; u += kEdgeThreads) {
                    const int j = i0 + 1 + k0 + u;
                    hs[u] = j <= E ? __ldg(&hr[j]) : make_float2(0.f, 0.f);
                }
            } else {
                // hs[kk] = h(-E+k0+kk), fs[u] = f(i0 - k0 - KT + 1 + u), u < KT + 63
                for (int u = threadIdx.x; u < kEdgeKT; u += kEdgeThreads) {
                    const int k = k0 + u;
                    hs[u] = k <= kmax ? __ldg(&hr[-E + k]) : make_float2(0.f, 0.f);
                }
                for (int u = threadIdx.x; u < kEdgeKT + kEdgeOut; u += kEdgeThreads) {
                    const int m = i0 - k0 - kEdgeKT + 1 + u;
                    fs[u] = (m >= 0 && m < E) ? load_f(signal, sig_f64, m) : 0.f;
                }
            }
            __syncthreads();
            if (i < E) {
                // this thread's quarter of the tile, clipped to the output's terms
                const int kb = q * (kEdgeKT / kEdgeSplit);
                const int ke = min(kb + kEdgeKT / kEdgeSplit, klast - k0 + 1);
#pragma unroll 8
                for (int kk = kb; kk < ke; kk++) {
                    float fv;
                    float2 hv;
                    if (left) {
                        fv = fs[kk];
                        hv = hs[o + kk];
                    } else {
                        hv = hs[kk];
                        fv = fs[o - kk + kEdgeKT - 1];
                    }
                    cr = fmaf(hv.x, fv, cr);
                    ci = fmaf(hv.y, fv, ci);
                }
            }
        }
        part[q][o] = make_float2(cr, ci);
        __syncthreads();
        if (q == 0 && i < E) {
            float2 c = part[0][o];
#pragma unroll
            for (int u = 1; u < kEdgeSplit; u++) c = make_float2(c.x + part[u][o].x, c.y + part[u][o].y);
            const int64_t n = left ? (int64_t)i : N - E + i;
            if constexpr (CPLX) {
                float2* w_ = (float2*)W + (int64_t)r * N + n;
                const float2 ov = *w_;
                const float2 w = make_float2(ov.x - c.x, ov.y - c.y);
                *w_ = w;
                dpow = (w.x * w.x + w.y * w.y) - (ov.x * ov.x + ov.y * ov.y);
            } else {
                float* w_ = (float*)W + (int64_t)r * N + n;
                const float ov = *w_, w = ov - c.x;
                *w_ = w;
                dpow = w * w - ov * ov;
            }
        }
    }
    if (ea.do_power) {
        double s0, s1;
        block_sum2<kEdgeThreads>(dpow, 0.f, &s0, &s1, red);
        if (threadIdx.x == 0) delta[(int64_t)r * c.nx + c.x] = s0;
    }
}
template <bool CPLX>
static __global__ void __launch_bounds__(kEdgeThreads) k_edge_fix(EdgeFixArgs a) {
    edge_fix_body<CPLX>(a, cta_plain());
}
template <bool CPLX>
static __global__ void __launch_bounds__(kEdgeThreads) k_edge_fix_g(GroupMap g) {
    Cta c;
    const EdgeFixArgs& a = group_args<EdgeFixArgs>(g, c);
    edge_fix_body<CPLX>(a, c);
}

// spectrum[r] += (sum of the row's block changes, fixed order) / N
struct EdgePowerArgs {
    const double* delta;
    double* spectrum;
    int64_t N;
    int32_t bpr, pad_;
};
__device__ __forceinline__ void edge_power_body(const EdgePowerArgs& a, const Cta c) {
    if (threadIdx.x != 0) return;
    double acc = 0.0;
    for (int b = 0; b < a.bpr; b++) acc += a.delta[(int64_t)c.x * a.bpr + b];
    a.spectrum[c.x] += acc / (double)a.N;
}
static __global__ void k_edge_power(EdgePowerArgs a) { edge_power_body(a, cta_plain()); }
static __global__ void k_edge_power_g(GroupMap g) {
    Cta c;
    const EdgePowerArgs& a = group_args<EdgePowerArgs>(g, c);
    edge_power_body(a, c);
}

namespace {

// half width (in units of x) beyond which |psi(x)| < 1e-9 of its peak: the GDW's
// (x^2 - 2) e^{-x^2/4} / 2 is 6.8e-10 at x = 10, the Morlet's envelope e^{-x^2/2}
// 6.7e-10 at x = 6.5.  Terms beyond it change W by ~1e-10 relative, far below
// the FP32 path's own rounding.
double psi_support(int wavelet) { return wavelet == CWT_WAVELET_GDW ? 10.0 : 6.5; }

int64_t edge_width(int wavelet, double wt) { return (int64_t)std::ceil(psi_support(wavelet) / wt) + 1; }

// The scale's spectrum is negligible (1e-7 of its peak) at the Nyquist frequency.
// Only then is the sampled wavelet the short one of support edge_width: a
// spectrum cut off at the Nyquist frequency rings, and the transform then
// depends on the padded length itself.
bool nyquist_clear(int wavelet, double omega0, double wt) {
    double u_lo, u_hi;
    wavelet_band(wavelet, omega0, 1e-7, &u_lo, &u_hi);
    const double nyq = kPi / wt;
    return u_hi < nyq && u_lo > -nyq;
}

// psi(x) of Table 2 (GDW, Morlet), FP64
void psi_x(int wavelet, double omega0, double x, double* re, double* im) {
    if (wavelet == CWT_WAVELET_GDW) {
        *re = std::pow(18.0 * kPi, -0.25) * (2.0 - x * x) * std::exp(-0.25 * x * x);
        *im = 0.0;
        return;
    }
    const double cn = wavelet_cn(wavelet, omega0), env = std::exp(-0.5 * x * x);
    *re = cn * (std::cos(omega0 * x) - std::exp(-0.5 * omega0 * omega0)) * env;
    *im = -cn * std::sin(omega0 * x) * env;
}

}  // namespace

// Periodic boundary with N not a power of two: ext[m] = f((m - E) mod N),
// m < N + 2E, the signal extended periodically by E samples on each side.
struct ExtendArgs {
    const void* f;
    void* ext;
    int64_t N, E;
    int32_t f64, pad_;
};
// One modulo per thread: the source index then advances by the grid stride
// reduced mod N, wrapping with one subtraction.
__device__ __forceinline__ void periodic_extend_body(const ExtendArgs& a, const Cta c) {
    const int64_t N = a.N, E = a.E, total = N + 2 * E;
    const int64_t stride = (int64_t)c.nx * blockDim.x, step = stride % N;
    int64_t m = c.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= total) return;
    int64_t src = ((m - E) % N + N) % N;
    for (; m < total; m += stride) {
        if (a.f64) ((double*)a.ext)[m] = __ldg(&((const double*)a.f)[src]);
        else ((float*)a.ext)[m] = __ldg(&((const float*)a.f)[src]);
        src += step;
        if (src >= N) src -= N;
    }
}
static __global__ void k_periodic_extend(ExtendArgs a) { periodic_extend_body(a, cta_plain()); }
static __global__ void k_periodic_extend_g(GroupMap g) {
    Cta c;
    const ExtendArgs& a = group_args<ExtendArgs>(g, c);
    periodic_extend_body(a, c);
}

// Forward transform of a real signal (Params::fpack): the forward passes leave
// Z, the M/2-point e^{-} DFT of z(q) = f(2q) + i f(2q + 1), in F[0 .. M/2).
// The DFTs of the even and odd samples are E(k) = (Z(k) + conj Z(-k)) / 2 and
// O(k) = (Z(k) - conj Z(-k)) / (2i) (indices mod M/2), the e^{-} DFT of f is
// X(k) = E(k) + e^{-2 pi i k / M} O(k), and F(k) = conj X(k) for k <= M/2 (the
// paper's e^{+} sign, Eq. 8).  One thread takes the pair (k, M/2 - k): both
// outputs read the same two values, so the pass runs in place.
struct UntangleArgs {
    float2* F;
    const float2* tw_lo;
    const float2* tw_hi;
    int64_t M;
    int32_t h, pad_;
};
// conj(E + w O) from za = Z(a), zb = Z(-a), w = e^{-2 pi i a / M}
__device__ __forceinline__ float2 untangle_one(float2 za, float2 zb, float2 w) {
    const float2 e = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y - zb.y));
    const float2 o = make_float2(0.5f * (za.y + zb.y), -0.5f * (za.x - zb.x));
    return make_float2(e.x + (w.x * o.x - w.y * o.y), -(e.y + (w.x * o.y + w.y * o.x)));
}
__device__ __forceinline__ float2 untangle_tw(const UntangleArgs& a, int64_t j) {
    const float2 hi = __ldg(&a.tw_hi[j >> a.h]), lo = __ldg(&a.tw_lo[j & ((int64_t(1) << a.h) - 1)]);
    return make_float2(hi.x * lo.x - hi.y * lo.y, hi.x * lo.y + hi.y * lo.x);
}
__device__ __forceinline__ void untangle_body(const UntangleArgs& a, const Cta c) {
    const int64_t half = a.M >> 1;
    for (int64_t k = c.x * (int64_t)blockDim.x + threadIdx.x; k <= (half >> 1); k += (int64_t)c.nx * blockDim.x) {
        const int64_t kp = half - k;
        const float2 zk = a.F[k], zkp = a.F[kp == half ? 0 : kp];
        a.F[k] = untangle_one(zk, zkp, untangle_tw(a, k));
        a.F[kp] = untangle_one(zkp, zk, untangle_tw(a, kp));
    }
}
static __global__ void k_fwd_untangle(UntangleArgs a) { untangle_body(a, cta_plain()); }
static __global__ void k_fwd_untangle_g(GroupMap g) {
    Cta c;
    const UntangleArgs& a = group_args<UntangleArgs>(g, c);
    untangle_body(a, c);
}

// ====================================================================== plan


namespace {

cwt_status fail(cwt_plan* p, cwt_status st, const std::string& msg) {
    if (p) p->err = msg;
    return st;
}

cwt_status cuda_fail(cwt_plan* p, cudaError_t e, const char* what) {
    return fail(p, e == cudaErrorMemoryAllocation ? CWT_ERR_OOM : CWT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CWT_CUDA(p, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cuda_fail((p), e_, #call);       \
    } while (0)

template <typename T>
cwt_status dev_alloc(cwt_plan* p, T** ptr, size_t count) {
    if (count == 0) { *ptr = nullptr; return CWT_OK; }
    cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
    if (e != cudaSuccess) { *ptr = nullptr; return cuda_fail(p, e, "cudaMalloc"); }
    p->ws_bytes += count * sizeof(T);
    return CWT_OK;
}

// A per-call buffer: allocated with the plan, or (CWT_SCRATCH_CALLER) an
// offset into the caller's scratch, bound by bind_scratch for each call.
constexpr size_t kScratchAlign = 256;
template <typename T>
cwt_status scratch_alloc(cwt_plan* p, T** ptr, size_t count) {
    if (p->opts.scratch != CWT_SCRATCH_CALLER) return dev_alloc(p, ptr, count);
    *ptr = nullptr;
    if (count == 0) return CWT_OK;
    p->scratch_slots.push_back({reinterpret_cast<void**>(ptr), p->scratch_own});
    p->scratch_own += (count * sizeof(T) + kScratchAlign - 1) / kScratchAlign * kScratchAlign;
    return CWT_OK;
}

// bytes of scratch of a plan with its child and sub-plans
size_t scratch_tree(const cwt_plan* p) {
    size_t subs = 0;
    for (const cwt_plan* q : p->subs) subs = std::max(subs, scratch_tree(q));
    return p->scratch_own + (p->child ? scratch_tree(p->child) : 0) + subs;
}

// points every per-call buffer of the tree into base (nullptr: unbinds)
void set_scratch(cwt_plan* p, char* base) {
    for (const auto& sl : p->scratch_slots) {
        void* a = base ? (void*)(base + sl.off) : nullptr;
        std::memcpy(sl.ptr, &a, sizeof a);
    }
    size_t off = p->scratch_own;
    if (p->child) {
        set_scratch(p->child, base ? base + off : nullptr);
        off += scratch_tree(p->child);
    }
    for (cwt_plan* q : p->subs) set_scratch(q, base ? base + off : nullptr);
    p->scratch_base = base;
}

template <typename T>
cwt_status upload(cwt_plan* p, T** ptr, const std::vector<T>& host) {
    cwt_status st = dev_alloc(p, ptr, host.size());
    if (st != CWT_OK || host.empty()) return st;
    CWT_CUDA(p, cudaMemcpy(*ptr, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice));
    return CWT_OK;
}

void release_events(cwt_plan* p) {
    for (auto& r : p->pending) {
        p->ev_pool.push_back(r.a);
        p->ev_pool.push_back(r.b);
    }
    p->pending.clear();
}

void free_plan(cwt_plan* p) {
    release_events(p);
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    p->ev_pool.clear();
    for (int i = 0; i < cwt_plan::kSide; i++) {
        if (p->side[i]) cudaStreamDestroy(p->side[i]);
        if (p->ev_join[i]) cudaEventDestroy(p->ev_join[i]);
    }
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_pre) cudaEventDestroy(p->ev_pre);
    if (p->ev_pfwd) cudaEventDestroy(p->ev_pfwd);
    for (cudaEvent_t e : p->hc_ev) cudaEventDestroy(e);
    if (p->hc_stream) cudaStreamDestroy(p->hc_stream);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->opts.scratch == CWT_SCRATCH_CALLER) set_scratch(p, nullptr);   // not the plan's to free
    void* ptrs[] = {p->d_jobs, p->d_tile_job, p->d_part_off, p->d_part_cnt, p->d_Fp, p->d_Ft, p->d_Y,
                    p->d_partials, p->d_tw_lo, p->d_tw_hi, p->d_tw_tab, p->h_sig, p->h_W,
                    p->h_spec, p->d_pw_partials, p->d_env_part, p->d_env_cnt, p->d_icwt_coef};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    void* bsb[] = {p->d_bs_chirp, p->d_bs_G, p->d_bs_work};
    for (void* q : bsb)
        if (q) cudaFree(q);
    void* edge[] = {p->d_edge_rows, p->d_edge_h, p->d_edge_delta};
    for (void* q : edge)
        if (q) cudaFree(q);
    if (p->child) free_plan(p->child);
    for (cwt_plan* q : p->subs) free_plan(q);
    if (p->d_ext) cudaFree(p->d_ext);
    if (p->h_err) cudaFreeHost(p->h_err);
    delete p;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return (EncodeTiledFn)f;
    }();
    return fn;
}
bool enc_ok() { return encode_tiled() != nullptr; }

// The tile pipeline's TMA map of Y as float rows: [slab][1024 rows][2 A floats];
// boxes of 256 rows x 8 complex columns land in shared memory with the 64-byte
// swizzle the kernels read
cwt_status encode_ymap(cwt_plan* p) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return fail(p, CWT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const int64_t M = p->M, A = M >> p->wide_logl;
    const cuuint64_t dims[3] = {(cuuint64_t)(2 * A), 1024, (cuuint64_t)(p->y_count / (size_t)M)};
    const cuuint64_t strides[2] = {(cuuint64_t)(A * 8), (cuuint64_t)(M * 8)};
    const cuuint32_t box[3] = {16, 256, 1}, estr[3] = {1, 1, 1};
    if (enc(&p->ymap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, p->d_Y, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return fail(p, CWT_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return CWT_OK;
}

// binds a call's scratch to the plan tree (and encodes the TMA maps of Y at
// their new addresses)
cwt_status bind_scratch(cwt_plan* p, char* base) {
    set_scratch(p, base);
    cwt_status st = CWT_OK;
    std::vector<cwt_plan*> todo{p};
    while (!todo.empty() && st == CWT_OK) {
        cwt_plan* q = todo.back();
        todo.pop_back();
        if (q->ymap_on) st = encode_ymap(q);
        if (q->child) todo.push_back(q->child);
        for (cwt_plan* r : q->subs) todo.push_back(r);
    }
    return st;
}

double out_row_bytes(const cwt_plan* p) {
    return (double)p->N * (p->wavelet == CWT_WAVELET_MORLET ? 8.0 : 4.0);
}

double job_rows(const Job& J) { return (J.g[0].row >= 0) + (J.g[1].row >= 0); }

// the scale's psi_hat generator on the grid of Mg points (0: the plan's M)
ScaleGen make_gen(const cwt_plan* p, double wt, int row, int64_t Mg = 0) {
    ScaleGen g{};
    const double Mgrid = (double)(Mg ? Mg : p->M);
    double alpha = 2.0 * kPi / (Mgrid * wt);
    g.a_hi = (float)alpha;
    g.a_lo = (float)(alpha - (double)g.a_hi);
    g.amp = (float)(std::sqrt(p->opts.dx / wt) / Mgrid *
                    wavelet_spectrum_const(p->wavelet, p->opts.omega0));
    double k0 = p->opts.omega0 / alpha;
    double k0i = std::floor(k0);
    if (k0i > 2147483647.0) k0i = 2147483647.0;
    g.k0_int = (int32_t)k0i;
    g.k0_frac = (float)(k0 - k0i);
    g.row = row;
    g.part_off = 0;
    return g;
}

void scale_band(const cwt_plan* p, double wt, double u_lo, double u_hi, int64_t* klo, int64_t* khi) {
    const int64_t lo_lim = -(p->M / 2) + 1, hi_lim = p->M / 2;
    double alpha = 2.0 * kPi / ((double)p->M * wt);
    double a = std::ceil(u_lo / alpha), b = std::floor(u_hi / alpha);
    int64_t lo = a < (double)lo_lim ? lo_lim : (a > (double)hi_lim ? hi_lim : (int64_t)a);
    int64_t hi = b > (double)hi_lim ? hi_lim : (b < (double)lo_lim ? lo_lim : (int64_t)b);
    if (hi < lo) { lo = hi = 0; }
    *klo = lo;
    *khi = hi;
}

size_t stage_smem(int logl, int T) { return (size_t)(1 << logl) * (size_t)row_stride(T) * sizeof(float2); }

// Pass 2 of the wide scales: with L = 1024 the tile pipeline (tensor-core
// stages of cwt_tc.cuh with a reduced precision; in FP32 the register stages
// of cwt_f32tile.cuh unless opts.wide2_kernel, resolved per plan, is 2), else
// the CTA Stockham kernel
bool wide2_on_tc(const cwt_plan* p) {
    return p->wide_logl == 10 && (p->opts.precision != CWT_PRECISION_FP32 || p->opts.wide2_kernel != 2);
}
const Entry& wide2_entry(const cwt_plan* p) { return tables().wide2[p->wide_logl][p->crop]; }

cwt_status opt_in_smem(cwt_plan* p, const void* fn);

// CTAs of kernel fn (nt threads, smem bytes of shared memory) the device holds
// at once; 0 when unknown
int64_t resident_ctas(cwt_plan* p, const void* fn, int nt, size_t smem, int* sms_out) {
    int sms = 0, n = 0;
    *sms_out = 0;
    if (!fn || opt_in_smem(p, fn) != CWT_OK) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, nt, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    *sms_out = sms;
    return (int64_t)n * sms;
}

// Tiles per CTA of a W-writing launch of njobs jobs of tiles_job tiles each
// (ceil(tiles_job / D) CTAs per job), given the CTAs the device holds at once
// (slots): the D in 1..kMaxD with the shortest makespan in tile times,
// ceil(CTAs / slots) x (D + kCtaSetup), among those keeping at least min_ctas
// CTAs (or all of the launch's tiles); ties go to the larger D.  A launch whose
// CTAs fill a whole number of waves then ends together instead of leaving a
// part-empty last wave.  Plans asking for fewer CTAs than SMs (made for
// batches, whose grouped launches merge many plans) keep pick_D's largest D.
constexpr double kCtaSetup = 0.5;          // a CTA's set-up (band values, job), in tile times
int pick_D_waves(int64_t tiles_job, int64_t njobs, int min_ctas, int64_t slots, int sms) {
    if (slots <= 0 || min_ctas < sms) return pick_D(tiles_job * njobs, min_ctas);
    const int64_t floor_ctas = std::min<int64_t>(min_ctas, tiles_job * njobs);
    int best = 1;
    double best_t = 1e300;
    for (int d = 1; d <= kMaxD; d++) {
        const int64_t ctas = njobs * ((tiles_job + d - 1) / d);
        if (ctas < floor_ctas) break;      // a larger D has no more CTAs
        const double t = (double)((ctas + slots - 1) / slots) * ((double)d + kCtaSetup);
        if (t <= best_t) {
            best_t = t;
            best = d;
        }
    }
    return best;
}

// twiddle tables of length p->M (FP64 generated, FP32 stored): the two-level
// e^{-2 pi i j / M} and the stage tables e^{-2 pi i i / L}, L <= kLmax
cwt_status upload_twiddles(cwt_plan* p) {
    const int64_t M = p->M;
    p->h = (p->logM + 1) / 2;
    std::vector<float2> lo(size_t(1) << p->h), hi(size_t(1) << (p->logM - p->h)), tt(2 * kLmax);
    for (size_t j = 0; j < lo.size(); j++) {
        double a = -2.0 * kPi * (double)j / (double)M;
        lo[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (size_t j = 0; j < hi.size(); j++) {
        double a = -2.0 * kPi * (double)(j << p->h) / (double)M;
        hi[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    tt[0] = tt[1] = make_float2(1.f, 0.f);
    for (int L = 2; L <= kLmax; L *= 2)
        for (int i = 0; i < L; i++) {
            double a = -2.0 * kPi * (double)i / (double)L;
            tt[L + i] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
    cwt_status st;
    if ((st = upload(p, &p->d_tw_lo, lo)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_tw_hi, hi)) != CWT_OK) return st;
    return upload(p, &p->d_tw_tab, tt);
}

cwt_status build_plan(cwt_plan* p) {
    const Tables& tb = tables();
    const int64_t M = p->M;
    double u_lo = -1e300, u_hi = 1e300;
    bool full = p->opts.eps_trunc <= 0.0;
    if (!full) wavelet_band(p->wavelet, p->opts.omega0, p->opts.eps_trunc, &u_lo, &u_hi);

    // jobs: real wavelets pair consecutive rows, the Morlet takes one row each;
    // rows that a child plan computes are left out
    const int per = wav_real(p->wavelet) ? 2 : 1;
    std::vector<int> own_rows;
    for (int r = 0; r < p->S; r++)
        if (r < p->child_r0 || r >= p->child_r0 + p->child_n) own_rows.push_back(r);
    std::vector<Job> all;
    for (size_t i0 = 0; i0 < own_rows.size(); i0 += per) {
        Job J{};
        int64_t klo = 0, khi = -1;
        for (int q = 0; q < 2; q++) {
            const size_t i = i0 + q;
            const int s = i < own_rows.size() ? own_rows[i] : -1;
            if (q < per && s >= 0) {
                J.g[q] = make_gen(p, p->w_tilde[s], s);
                int64_t a, b;
                if (full) { a = -(M / 2) + 1; b = M / 2; }
                else scale_band(p, p->w_tilde[s], u_lo, u_hi, &a, &b);
                if (khi < klo) { klo = a; khi = b; }
                else { klo = std::min(klo, a); khi = std::max(khi, b); }
            } else {
                J.g[q] = ScaleGen{};
                J.g[q].row = -1;
            }
        }
        J.k_lo = (int32_t)klo;
        J.K = (int32_t)(khi - klo + 1);
        all.push_back(J);
    }

    // shapes: band kernels take K <= L (L <= 1024, or <= M when M <= kLmax); wider bands
    // take the two-pass path with pass-2 length 2^wide_logl
    const bool small = M <= kLmax;
    p->wide_logl = std::max(kWideLog, p->logM - kLmaxLog);
    p->wide_loga = p->logM - p->wide_logl;
    // band groups by (log2 L, direct depth): slots kLmaxLog + 1 .. + 4 hold the
    // L = 1024 groups of depth 2, 4, 8 and 16 (bands up to 2048 .. 16384 bins)
    std::vector<std::vector<Job>> by_logl(kLmaxLog + 1 + kBandRdMax);
    std::vector<Job> wide;
    for (const Job& J : all) {
        int lk = std::max(1, ilog2(J.K));
        if (small) by_logl[std::min(lk, p->logM)].push_back(J);
        else if (lk <= kBandMaxLog) by_logl[lk].push_back(J);
        else if (p->opts.band_depth >= 2 && J.K <= (2 << kBandDepthLog)) by_logl[kLmaxLog + 1].push_back(J);
        else if (p->opts.band_depth >= 4 && J.K <= (4 << kBandDepthLog)) by_logl[kLmaxLog + 2].push_back(J);
        else if (p->opts.band_depth >= 8 && J.K <= (8 << kBandDepthLog)) by_logl[kLmaxLog + 3].push_back(J);
        else if (p->opts.band_depth >= 16 && J.K <= (16 << kBandDepthLog)) by_logl[kLmaxLog + 4].push_back(J);
        else wide.push_back(J);
    }

    // band groups (jobs reordered: band groups first, then wide batches)
    std::vector<int32_t> tile_job;
    p->part_off.assign(p->S, 0);
    p->part_cnt.assign(p->S, 0);
    int64_t nparts = 0;
    auto assign_parts = [&](Job& J, int ntiles) {
        for (int q = 0; q < 2; q++) {
            if (J.g[q].row < 0) continue;
            J.g[q].part_off = (int32_t)nparts;
            p->part_off[J.g[q].row] = (int32_t)nparts;
            p->part_cnt[J.g[q].row] = ntiles;
            nparts += ntiles;
        }
    };
    for (int slot = 1; slot <= kLmaxLog + kBandRdMax; slot++) {
        if (by_logl[slot].empty()) continue;
        const int ll = slot <= kLmaxLog ? slot : kBandDepthLog;
        cwt_plan::BandGroup g;
        g.logl = ll;
        g.rdi = slot <= kLmaxLog ? 0 : slot - kLmaxLog;
        const int64_t A = M >> ll;
        const int T = tb.band[ll][0].T;
        const int64_t tiles_job = (A + T - 1) / T;
        const int crop = p->N < M ? 1 : 0;
        const Entry& be = g.rdi ? tb.band_rd[g.rdi][crop] : tb.band[ll][crop];
        int sms = 0;
        const int64_t slots = resident_ctas(p, (const void*)be.fn, be.NT,
                                            (size_t)((1 << g.rdi) << ll) * sizeof(float2) + stage_smem(ll, be.T), &sms);
        const int D = pick_D_waves(tiles_job, (int64_t)by_logl[slot].size(), p->opts.min_ctas, slots, sms);
        const int per_job = (int)((tiles_job + D - 1) / D);
        g.D = D;
        g.ntiles = 0;
        g.tj_off = tile_job.size();
        g.bytes = 0;
        g.job0 = (int)p->jobs.size();
        g.njobs = (int)by_logl[slot].size();
        for (Job J : by_logl[slot]) {
            J.tile0 = g.ntiles;
            int idx = (int)p->jobs.size();
            for (int t = 0; t < per_job; t++) tile_job.push_back(idx);
            g.ntiles += per_job;
            assign_parts(J, per_job);
            g.bytes += job_rows(J) * out_row_bytes(p) + 8.0 * J.K;
            p->jobs.push_back(J);
        }
        p->groups.push_back(g);
    }
    p->n_band_jobs = (int64_t)p->jobs.size();
    if (!wide.empty()) {
        const int64_t A = M >> p->wide_logl;
        const int T2 = tb.wide2[p->wide_logl][0].T;
        p->wide_G = (int)std::max<int64_t>(1, p->opts.wide_batch_bytes / (int64_t)((size_t)M * sizeof(float2)));
        const int64_t tiles_job = (A + T2 - 1) / T2;
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
        const int L = 1 << p->wide_logl;
        // batches: up to wide_G consecutive jobs with the same pass-1 shape
        const size_t job_base = p->jobs.size();
        std::vector<int> batch_of(wide.size());
        for (size_t i = 0; i < wide.size(); i++) {
            const Job& J = wide[i];
            // pass 1 of column b has at most ceil(K / L) band bins: a pruned band tile of
            // L1 = 2^ceil(log2) points over A1 = A / L1 columns d1, with the widest
            // column-count variant that fits A1; the whole A-point DFT when L1 = A, and
            // for A <= 128, where the pruned tiles would be CTAs of a few threads
            int l1 = std::max(1, ilog2(((int64_t)J.K + L - 1) / L));
            int var = -1;
            if (p->wide_loga >= 8 && l1 <= kLmaxLog - 2 && l1 < p->wide_loga) {
                const int64_t A1 = int64_t(1) << (p->wide_loga - l1);
                for (int q = 0; q < kP1Var && var < 0; q++)
                    if (tb.wide1p[l1][q].T <= A1) var = q;
            }
            if (var < 0) l1 = -1;
            if (p->wide.empty() || p->wide.back().count >= p->wide_G || p->wide.back().logl1 != l1 ||
                p->wide.back().var != var)
                p->wide.push_back({(int)(job_base + i), 0, l1, var, 0.0, 0.0, 1});
            auto& wb = p->wide.back();
            wb.count++;
            wb.band_bytes += 8.0 * J.K;
            wb.out_bytes += job_rows(J) * out_row_bytes(p);
            batch_of[i] = (int)p->wide.size() - 1;
        }
        // pass-2 tiles per CTA, from each batch's own job count (batches split by
        // pass-1 shape are often smaller than wide_G).  The tile pipeline is
        // resident as one CTA per SM: about one CTA per SM per launch, each
        // looping over its tiles (set-up, fill and drain paid once per CTA).
        for (auto& wb : p->wide) {
            if (wide2_on_tc(p)) {
                const int64_t per = std::max<int64_t>(1, sms / wb.count);
                wb.D = (int)((tiles_job + per - 1) / per);
            } else {
                const Entry& e2 = tb.wide2[p->wide_logl][p->N < M ? 1 : 0];
                int sms2 = 0;
                const int64_t slots = resident_ctas(p, (const void*)e2.fn, e2.NT, stage_smem(p->wide_logl, e2.T), &sms2);
                wb.D = pick_D_waves(tiles_job, wb.count, p->opts.min_ctas, slots, sms2);
            }
        }
        for (size_t i = 0; i < wide.size(); i++) {
            Job J = wide[i];
            J.tile0 = 0;
            const int D = p->wide[batch_of[i]].D;
            assign_parts(J, (int)((tiles_job + D - 1) / D));
            p->jobs.push_back(J);
        }
    }
    p->n_partials = nparts;
    p->fwd_small = small;
    p->crop = p->N < M;
    p->fwd_in_bytes = (double)p->N * (p->opts.input_dtype == CWT_INPUT_F64 ? 8.0 : 4.0);
    p->fwd_out_bytes = 8.0 * (double)(M / 2 + 1);

    cwt_status st;
    if ((st = upload(p, &p->d_jobs, p->jobs)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_tile_job, tile_job)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_part_off, p->part_off)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_part_cnt, p->part_cnt)) != CWT_OK) return st;
    if ((st = upload_twiddles(p)) != CWT_OK) return st;
    if ((st = scratch_alloc(p, &p->d_Fp, (size_t)(M / 2 + 1))) != CWT_OK) return st;
    if (!p->wide.empty() && (st = scratch_alloc(p, &p->d_Ft, (size_t)M)) != CWT_OK) return st;
    size_t ycount = 0;
    if (!small) ycount = (size_t)M;
    p->y_stride = (size_t)M * (size_t)std::max(1, std::min<int>(p->wide_G, (int)wide.size()));
    if (!p->wide.empty())
        ycount = std::max(ycount, p->y_stride * (size_t)std::min<size_t>(p->wide.size(), cwt_plan::kSide + 1));
    if ((st = scratch_alloc(p, &p->d_Y, ycount)) != CWT_OK) return st;
    p->y_count = ycount;
    if (!p->wide.empty() && wide2_on_tc(p)) {
        p->ymap_on = true;
        if (!enc_ok()) return fail(p, CWT_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        // with caller scratch the map is encoded when a call binds its scratch
        if (p->opts.scratch != CWT_SCRATCH_CALLER && (st = encode_ymap(p)) != CWT_OK) return st;
        CWT_CUDA(p, cudaHostAlloc((void**)&p->h_err, sizeof(int32_t), cudaHostAllocMapped));
        *p->h_err = 0;
        CWT_CUDA(p, cudaHostGetDevicePointer((void**)&p->d_err, p->h_err, 0));
    }
    if ((st = scratch_alloc(p, &p->d_partials, (size_t)std::max<int64_t>(1, nparts))) != CWT_OK) return st;
    if (p->child) {
        std::vector<EdgeRow> er(p->child_n);
        std::vector<float2> h;
        int64_t emax = 0;
        for (int i = 0; i < p->child_n; i++) {
            const double wt = p->w_tilde[p->child_r0 + i];
            const int64_t E = edge_width(p->wavelet, wt);
            er[i] = {(int32_t)E, (int32_t)h.size()};
            const double nrm = std::sqrt(wt * p->opts.dx);
            for (int64_t j = -E; j <= E; j++) {
                double re, im;
                psi_x(p->wavelet, p->opts.omega0, wt * (double)j, &re, &im);
                h.push_back(make_float2((float)(nrm * re), (float)(nrm * im)));
            }
            emax = std::max(emax, E);
        }
        p->edge_bpr = (int32_t)(2 * ((emax + kEdgeOut - 1) / kEdgeOut));
        EdgeRow* d_er = nullptr;
        if ((st = upload(p, &d_er, er)) != CWT_OK) return st;
        p->d_edge_rows = d_er;
        if ((st = upload(p, &p->d_edge_h, h)) != CWT_OK) return st;
        if ((st = scratch_alloc(p, &p->d_edge_delta, (size_t)p->child_n * p->edge_bpr)) != CWT_OK) return st;
    }

    // side streams and events, and the shared-memory opt-in of every kernel the
    // plan launches, are set up here so that no call made while capturing needs them
    CWT_CUDA(p, cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
    if (p->child) {
        CWT_CUDA(p, cudaEventCreateWithFlags(&p->ev_pre, cudaEventDisableTiming));
        CWT_CUDA(p, cudaEventCreateWithFlags(&p->ev_pfwd, cudaEventDisableTiming));
    }

    for (int i = 0; i < cwt_plan::kSide; i++) {
        CWT_CUDA(p, cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking));
        CWT_CUDA(p, cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming));
    }
    std::vector<const void*> fns;
    if (small) fns.push_back((const void*)tb.fwd_small[p->logM].fn);
    else {
        fns.push_back((const void*)tb.fwd1[p->wide_loga].fn);
        fns.push_back((const void*)tb.fwd2[p->wide_logl].fn);
    }
    for (const auto& g : p->groups)
        fns.push_back((const void*)(g.rdi ? tb.band_rd[g.rdi][p->crop].fn : tb.band[g.logl][p->crop].fn));
    for (const auto& wb : p->wide) {
        fns.push_back(wb.logl1 < 0 ? (const void*)tb.wide1[p->wide_loga].fn
                                   : (const void*)tb.wide1p[wb.logl1][wb.var].fn);
        if (wide2_on_tc(p)) {
            fns.push_back((const void*)tb.wide2_tc[p->opts.precision][p->crop].fn);
            fns.push_back((const void*)tb.wide2_tc[p->opts.precision][p->crop].gfn);
        } else {
            fns.push_back((const void*)wide2_entry(p).fn);
        }
    }
    for (const void* f : fns) {
        if (!f) return fail(p, CWT_ERR_INTERNAL, "missing kernel instantiation");
        if ((st = opt_in_smem(p, f)) != CWT_OK) return st;
    }
    return CWT_OK;
}

Params base_params(const cwt_plan* p) {
    Params P{};
    P.Fp = p->d_Fp;
    P.Fp_out = p->d_Fp;
    P.Ft = p->d_Ft;
    P.Y = p->d_Y;
    P.partials = p->d_partials;
    P.tw_lo = p->d_tw_lo;
    P.tw_hi = p->d_tw_hi;
    P.tw_tab = p->d_tw_tab;
    P.jobs = p->d_jobs;
    P.tile_job = p->d_tile_job;
    P.N = p->N;
    P.out_off = p->out_off;
    P.out_len = p->out_len;
    P.M = (int32_t)p->M;
    P.h = p->h;
    P.wavelet = p->wavelet;
    P.sig_f64 = p->opts.input_dtype == CWT_INPUT_F64;
    P.half_w0sq = (float)(0.5 * p->opts.omega0 * p->opts.omega0);
    // the Morlet's correction term is below eps_trunc (relative to the spectrum's
    // peak, ~1) where (v^2 + omega0^2) / 2 > -ln(eps); never skipped without truncation
    const double cv2 = p->opts.eps_trunc > 0.0 ? -2.0 * std::log(p->opts.eps_trunc) - p->opts.omega0 * p->opts.omega0
                                               : 1e30;
    P.corr_v2 = (float)std::min(1e30, std::max(0.0, cv2));
    return P;
}

cudaEvent_t take_event(cwt_plan* p) {
    if (!p->ev_pool.empty()) {
        cudaEvent_t e = p->ev_pool.back();
        p->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Event pair around one launch when the timing hook is on.
struct LaunchTimer {
    cwt_plan* p;
    int cls;
    double bytes;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    LaunchTimer(cwt_plan* p_, int cls_, double bytes_, cudaStream_t s_) : p(p_), cls(cls_), bytes(bytes_), s(s_) {
        if (p->timing) {
            a = take_event(p);
            b = take_event(p);
            if (a) cudaEventRecord(a, s);
        }
    }
    void done() {
        if (!a || !b) return;
        cudaEventRecord(b, s);
        p->pending.push_back({cls, a, b, bytes});
    }
};

// Lets a kernel use all the shared memory the device allows beyond its static
// part (once per kernel and device; dynamic requests above 48 KB need it).
cwt_status opt_in_smem(cwt_plan* p, const void* fn) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    std::lock_guard<std::mutex> lock(mu);
    if (done.count({p->device, fn})) return CWT_OK;
    cudaFuncAttributes fa{};
    CWT_CUDA(p, cudaFuncGetAttributes(&fa, fn));
    int optin = 0;
    CWT_CUDA(p, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device));
    CWT_CUDA(p, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes));
    done.insert({p->device, fn});
    return CWT_OK;
}

// Stream-order operations of a launch sequence: made, or recorded by a batch.
cwt_status ev_record(cwt_plan* p, cudaEvent_t e, cudaStream_t s) {
    if (p->rec) p->rec->record(e, s);
    else CWT_CUDA(p, cudaEventRecord(e, s));
    return CWT_OK;
}
cwt_status ev_wait(cwt_plan* p, cudaStream_t s, cudaEvent_t e) {
    if (p->rec) p->rec->wait(s, e);
    else CWT_CUDA(p, cudaStreamWaitEvent(s, e, 0));
    return CWT_OK;
}
template <class A>
void rec_launch(cwt_plan* p, const void* gfn, dim3 grid, dim3 block, size_t smem, cudaStream_t s, const A& a) {
    p->rec->add(s, gfn, grid, block, smem, &a, sizeof(A));
}

cwt_status launch(cwt_plan* p, const Entry& e, dim3 grid, size_t smem, const Params& P, cudaStream_t s, int cls,
                  double bytes) {
    if (!e.fn || !e.gfn) return fail(p, CWT_ERR_INTERNAL, "missing kernel instantiation");
    if (p->rec) {
        rec_launch(p, (const void*)e.gfn, grid, dim3(e.NT), smem, s, P);
        return CWT_OK;
    }
    cwt_status st = opt_in_smem(p, (const void*)e.fn);
    if (st != CWT_OK) return st;
    LaunchTimer lt(p, cls, bytes, s);
    e.fn<<<grid, e.NT, smem, s>>>(P);
    CWT_CUDA(p, cudaGetLastError());
    lt.done();
    return CWT_OK;
}

cwt_status check_device(cwt_plan* p) {
    int d = -1;
    CWT_CUDA(p, cudaGetDevice(&d));
    if (d != p->device) return fail(p, CWT_ERR_INVALID_ARG, "current device differs from the plan's device");
    return CWT_OK;
}

// The forward kernels over M = p->M points: one CTA when M <= kLmax, else the
// A-point column DFTs (pass 1, through p->d_Y) and the L-point DFTs (pass 2).
// P selects the input (the real signal, or P.cin) and the output (P.Fp_out, by
// P.cmode).
cwt_status launch_forward(cwt_plan* p, const Params& P, cudaStream_t fs, double in_bytes, double out_bytes) {
    const Tables& tb = tables();
    cwt_status st;
    // a real signal: the M/2-point DFT of its samples packed in pairs, then the
    // untangle pass (k_fwd_untangle); complex inputs (P.cin) take the M-point form
    if (!P.cin && P.cmode == 0 && p->logM >= kPackMinLog) {
        Params Q = P;
        Q.fpack = 1;
        Q.cmode = 3;                                  // the passes write Z whole
        const int lmt = p->logM - 1;
        if (lmt <= kLmaxLog) {
            Q.A = 1;
            st = launch(p, tb.fwd_small[lmt], dim3(1), stage_smem(lmt, 1), Q, fs, CWT_KCLASS_FORWARD, in_bytes);
        } else {
            const Entry& e1 = tb.fwd1[p->wide_loga - 1];
            const int L = 1 << p->wide_logl;
            st = launch(p, e1, dim3((L + e1.T - 1) / e1.T), stage_smem(p->wide_loga - 1, e1.T), Q, fs,
                        CWT_KCLASS_FORWARD, in_bytes);
            if (st == CWT_OK) {
                const Entry& e2 = tb.fwd2[p->wide_logl];
                Q.A = (int32_t)((p->M >> 1) >> p->wide_logl);
                st = launch(p, e2, dim3((Q.A + e2.T - 1) / e2.T), stage_smem(p->wide_logl, e2.T), Q, fs,
                            CWT_KCLASS_FORWARD, 0.0);
            }
        }
        if (st != CWT_OK) return st;
        const int64_t pairs = (p->M >> 2) + 1;
        const unsigned blocks = (unsigned)std::min<int64_t>(4096, (pairs + 255) / 256);
        const UntangleArgs a{P.Fp_out, p->d_tw_lo, p->d_tw_hi, p->M, p->h, 0};
        if (p->rec) {
            rec_launch(p, (const void*)k_fwd_untangle_g, dim3(blocks), dim3(256), 0, fs, a);
            return CWT_OK;
        }
        LaunchTimer lt(p, CWT_KCLASS_FORWARD, out_bytes, fs);
        k_fwd_untangle<<<blocks, 256, 0, fs>>>(a);
        CWT_CUDA(p, cudaGetLastError());
        lt.done();
        return CWT_OK;
    }
    if (p->fwd_small) {
        const Entry& e = tb.fwd_small[p->logM];
        Params Q = P;
        Q.A = 1;
        return launch(p, e, dim3(1), stage_smem(p->logM, 1), Q, fs, CWT_KCLASS_FORWARD, in_bytes + out_bytes);
    }
    const Entry& e1 = tb.fwd1[p->wide_loga];
    const int L = 1 << p->wide_logl;
    if ((st = launch(p, e1, dim3((L + e1.T - 1) / e1.T), stage_smem(p->wide_loga, e1.T), P, fs, CWT_KCLASS_FORWARD,
                     in_bytes)) != CWT_OK)
        return st;
    const Entry& e2 = tb.fwd2[p->wide_logl];
    Params Q = P;
    Q.A = (int32_t)(p->M >> p->wide_logl);
    return launch(p, e2, dim3((Q.A + e2.T - 1) / e2.T), stage_smem(p->wide_logl, e2.T), Q, fs, CWT_KCLASS_FORWARD,
                  out_bytes);
}

// W rows of jobs j0 .. j0 + n - 1
std::vector<int> rows_of_jobs(const cwt_plan* p, int j0, int n) {
    std::vector<int> r;
    for (int j = j0; j < j0 + n; j++)
        for (int q = 0; q < 2; q++)
            if (p->jobs[j].g[q].row >= 0) r.push_back(p->jobs[j].g[q].row);
    return r;
}

// cwt_exec_host: the W rows `rows` are final once the work queued on `s` so
// far is done.  The copy stream waits for that point and copies them to the
// host (runs of consecutive rows as one copy) while later launches run.
cwt_status host_copy_rows(cwt_plan* p, cudaStream_t s, std::vector<int> rows) {
    auto& h = p->hc;
    if (!h.on || rows.empty()) return CWT_OK;
    if (h.nev == p->hc_ev.size()) {
        cudaEvent_t e = nullptr;
        CWT_CUDA(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        p->hc_ev.push_back(e);
    }
    cudaEvent_t e = p->hc_ev[h.nev++];
    CWT_CUDA(p, cudaEventRecord(e, s));
    CWT_CUDA(p, cudaStreamWaitEvent(p->hc_stream, e, 0));
    std::sort(rows.begin(), rows.end());
    for (size_t i = 0; i < rows.size();) {
        size_t j = i + 1;
        while (j < rows.size() && rows[j] == rows[j - 1] + 1) j++;
        const size_t off = (size_t)rows[i] * h.row_bytes, n = (j - i) * h.row_bytes;
        CWT_CUDA(p, cudaMemcpyAsync(h.dst + off, h.src + off, n, cudaMemcpyDeviceToHost, p->hc_stream));
        for (size_t k = i; k < j; k++) h.done[rows[k]] = 1;
        i = j;
    }
    return CWT_OK;
}

// Periodic boundary for any N (a plan made by create_bluestein): the chirp
// transform of cwt_bluestein.cuh on the call's stream.  Signal stage:
// X = f c, X2 = conj(D(X) D(conj c)), Cv = conj(D(X2)) = P conv1.  Per job:
// X = psi-product Cv / P, X2 = conj(D(X) D(c)), X = conj(D(X2)), W = conj(c) X / P.
cwt_status run_bluestein(cwt_plan* p, const void* signal, void* W, double* spectrum, cudaStream_t s) {
    using BsFn = void (*)(BsArgs);
    const int64_t P = p->M;
    float2* Cv = p->d_bs_work;                   // then X, X2 of each stream
    float2* X = Cv + P;
    float2* X2 = X + P;
    const Params B = base_params(p);
    BsArgs a{};
    a.signal = signal;
    a.chirp = p->d_bs_chirp;
    a.W = W;
    a.partials = p->d_partials;
    a.N = p->N;
    a.P = (int32_t)P;
    a.sig_f64 = B.sig_f64;
    a.wavelet = p->wavelet;
    a.do_power = spectrum != nullptr;
    a.half_w0sq = B.half_w0sq;
    a.corr_v2 = B.corr_v2;
    a.inv_p = (float)(1.0 / (double)P);
    const unsigned gp = (unsigned)std::min<int64_t>((P + kBsThreads - 1) / kBsThreads, 4096);
    const unsigned go = (unsigned)((p->N + kBsOutBlock - 1) / kBsOutBlock);
    auto elem = [&](BsFn fn, const void* gfn, unsigned grid, cudaStream_t es, int cls, double bytes) -> cwt_status {
        if (p->rec) {
            rec_launch(p, gfn, dim3(grid), dim3(kBsThreads), 0, es, a);
            return CWT_OK;
        }
        LaunchTimer lt(p, cls, bytes, es);
        fn<<<grid, kBsThreads, 0, es>>>(a);
        CWT_CUDA(p, cudaGetLastError());
        lt.done();
        return CWT_OK;
    };
    auto fft = [&](const float2* in, float2* out, const float2* G, int mode, float2* Y, cudaStream_t es) -> cwt_status {
        Params Q = B;
        Q.cin = in;
        Q.Fp_out = out;
        Q.cG = G;
        Q.cmode = mode;
        Q.Y = Y;
        return launch_forward(p, Q, es, 8.0 * (double)P, 8.0 * (double)P);
    };
    cwt_status st;
    a.dst = X;
    if ((st = elem(k_bs_sig, (const void*)k_bs_sig_g, gp, s, CWT_KCLASS_FORWARD, 4.0 * (double)p->N)) != CWT_OK)
        return st;
    if ((st = fft(X, X2, p->d_bs_G, 1, p->d_Y, s)) != CWT_OK) return st;
    if ((st = fft(X2, Cv, nullptr, 2, p->d_Y, s)) != CWT_OK) return st;
    // the jobs are independent: round robin over the call's stream and the side
    // streams, each with its own X, X2 and forward intermediate
    const int nst = p->timing == 2 ? 1 : std::min<int>((int)p->jobs.size(), p->bs_streams);
    cudaStream_t streams[cwt_plan::kSide + 1] = {s};
    if (nst > 1) {
        if ((st = ev_record(p, p->ev_fork, s)) != CWT_OK) return st;
        for (int i = 1; i < nst; i++) {
            streams[i] = p->side[i - 1];
            if ((st = ev_wait(p, streams[i], p->ev_fork)) != CWT_OK) return st;
        }
    }
    for (size_t j = 0; j < p->jobs.size(); j++) {
        const int si = (int)(j % nst);
        cudaStream_t es = streams[si];
        float2* Xs = X + 2 * P * si;
        float2* X2s = Xs + P;
        float2* Ys = p->d_Y ? p->d_Y + P * si : nullptr;
        a.J = p->jobs[j];
        a.src = Cv;
        a.dst = Xs;
        if ((st = elem(k_bs_scale, (const void*)k_bs_scale_g, gp, es, CWT_KCLASS_WIDE1, 0.0)) != CWT_OK) return st;
        if ((st = fft(Xs, X2s, p->d_bs_G + P, 1, Ys, es)) != CWT_OK) return st;
        if ((st = fft(X2s, Xs, nullptr, 2, Ys, es)) != CWT_OK) return st;
        a.src = Xs;
        if ((st = elem(k_bs_out, (const void*)k_bs_out_g, go, es, CWT_KCLASS_WIDE2,
                       job_rows(a.J) * out_row_bytes(p))) != CWT_OK)
            return st;
    }
    for (int i = 1; i < nst; i++) {
        if ((st = ev_record(p, p->ev_join[i - 1], streams[i])) != CWT_OK) return st;
        if ((st = ev_wait(p, s, p->ev_join[i - 1])) != CWT_OK) return st;
    }
    if (spectrum) {
        LaunchTimer lt(p, CWT_KCLASS_POWER, 8.0 * (double)(p->n_partials + p->S), s);
        if (p->rec) {
            const PowerArgs pa{p->d_partials, p->d_part_off, p->d_part_cnt, spectrum, p->out_len, p->S, 0};
            rec_launch(p, (const void*)k_power_finalize_g, dim3(p->S), dim3(32), 0, s, pa);
        } else {
            k_power_finalize<<<p->S, 32, 0, s>>>(p->d_partials, p->d_part_off, p->d_part_cnt, p->S, p->out_len,
                                                 spectrum);
            CWT_CUDA(p, cudaGetLastError());
            lt.done();
        }
    }
    return CWT_OK;
}

cwt_status run_launches(cwt_plan* p, const void* signal, void* W, double* spectrum, cudaStream_t s) {
    const Tables& tb = tables();
    if (p->bs) return run_bluestein(p, signal, W, spectrum, s);
    cwt_status st;
    if (!p->subs.empty()) {                      // N not a power of two: sub-plans by padded length
        const int f64 = p->opts.input_dtype == CWT_INPUT_F64;
        const size_t se = f64 ? sizeof(double) : sizeof(float);
        const size_t we = p->wavelet == CWT_WAVELET_MORLET ? sizeof(float2) : sizeof(float);
        const bool ext = p->boundary == CWT_BOUNDARY_PERIODIC;   // zero boundary: the signal itself
        if (ext) {
            LaunchTimer lt(p, CWT_KCLASS_FORWARD, 0.0, s);
            const int64_t total = p->N + 2 * p->ext_E;
            // about 8 samples per thread: the per-thread modulo is then amortised
            const unsigned blocks = (unsigned)std::min<int64_t>(4096, (total + 2047) / 2048);
            const ExtendArgs a{signal, p->d_ext, p->N, p->ext_E, f64, 0};
            if (p->rec) {
                rec_launch(p, (const void*)k_periodic_extend_g, dim3(blocks), dim3(256), 0, s, a);
            } else {
                k_periodic_extend<<<blocks, 256, 0, s>>>(a);
                CWT_CUDA(p, cudaGetLastError());
                lt.done();
            }
        }
        // recording a batch: the sub-plans (disjoint rows) each on a stream of
        // their own, forked after the extension, joined by the call's stream
        const int sub_fork = p->rec ? p->rec->level_of((const void*)s) : 0;
        int sub_level = sub_fork;
        for (size_t i = 0; i < p->subs.size(); i++) {
            const void* sig = ext ? (const void*)((const char*)p->d_ext + (size_t)(p->ext_E - p->sub_E[i]) * se)
                                  : signal;
            void* Wi = (char*)W + (size_t)p->sub_r0[i] * (size_t)p->N * we;
            double* spi = spectrum ? spectrum + p->sub_r0[i] : nullptr;
            cudaStream_t ss = s;
            if (p->rec) {
                const void* key = &p->subs[i];
                p->rec->stream_level[key] = sub_fork;
                ss = (cudaStream_t)key;
            }
            if ((st = run_launches(p->subs[i], sig, Wi, spi, ss)) != CWT_OK) return st;
            if (p->rec) sub_level = std::max(sub_level, p->rec->level_of((const void*)ss));
        }
        if (p->rec) p->rec->stream_level[(const void*)s] = std::max(p->rec->level_of((const void*)s), sub_level);
        return CWT_OK;
    }
    Params P = base_params(p);
    P.signal = signal;
    P.W = W;
    P.do_power = spectrum != nullptr;

    // rows with short wavelet support: a periodic N-point child plan (with its
    // own side streams) on the call's stream, then the edge correction of those
    // rows.  This plan's forward transform runs beside the child on a side
    // stream, and the edge correction beside this plan's own work.
    const size_t esz = p->wavelet == CWT_WAVELET_MORLET ? sizeof(float2) : sizeof(float);
    void* Wc = p->child ? (char*)W + (size_t)p->child_r0 * (size_t)p->N * esz : nullptr;
    double* sc = (p->child && spectrum) ? spectrum + p->child_r0 : nullptr;
    auto edge_fix = [&](cudaStream_t es) -> cwt_status {
        {
            LaunchTimer lt(p, CWT_KCLASS_BAND, 0.0, es);
            const dim3 grid((unsigned)p->edge_bpr, (unsigned)p->child_n);
            const EdgeRow* rows = (const EdgeRow*)p->d_edge_rows;
            const int f64 = p->opts.input_dtype == CWT_INPUT_F64;
            const EdgeFixArgs a{signal, Wc, p->d_edge_h, rows, p->d_edge_delta, p->N, f64, sc != nullptr};
            const bool cplx = p->wavelet == CWT_WAVELET_MORLET;
            if (p->rec) {
                rec_launch(p, cplx ? (const void*)k_edge_fix_g<true> : (const void*)k_edge_fix_g<false>, grid,
                           dim3(kEdgeThreads), 0, es, a);
            } else {
                if (cplx) k_edge_fix<true><<<grid, kEdgeThreads, 0, es>>>(a);
                else k_edge_fix<false><<<grid, kEdgeThreads, 0, es>>>(a);
                CWT_CUDA(p, cudaGetLastError());
                lt.done();
            }
        }
        if (sc) {
            LaunchTimer lt(p, CWT_KCLASS_POWER, 0.0, es);
            const EdgePowerArgs a{p->d_edge_delta, sc, p->N, p->edge_bpr, 0};
            if (p->rec) {
                rec_launch(p, (const void*)k_edge_power_g, dim3(p->child_n), dim3(32), 0, es, a);
            } else {
                k_edge_power<<<p->child_n, 32, 0, es>>>(a);
                CWT_CUDA(p, cudaGetLastError());
                lt.done();
            }
        }
        return CWT_OK;
    };
    if (p->jobs.empty()) {                       // every row comes from the child
        if ((st = run_launches(p->child, signal, Wc, sc, s)) != CWT_OK) return st;
        return edge_fix(s);
    }
    // timing mode 2 serialises every launch on the call's stream, so that each
    // launch's event pair measures that kernel alone
    const bool serial = p->timing == 2;
    cudaStream_t fs = s;                         // stream of this plan's forward transform
    if (p->child && !serial) {
        if ((st = ev_record(p, p->ev_pre, s)) != CWT_OK) return st;
        if ((st = ev_wait(p, p->side[0], p->ev_pre)) != CWT_OK) return st;
        fs = p->side[0];
    }

    // 1. forward transform F(m) = sum_n f(n) e^{+2 pi i m n / M}, m <= M/2
    if ((st = launch_forward(p, P, fs, p->fwd_in_bytes, p->fwd_out_bytes)) != CWT_OK) return st;

    // the wide scales' pass 1 reads the spectrum column by column: transpose it once
    if (!p->wide.empty()) {
        const int L = 1 << p->wide_logl;
        const int A = (int)(p->M >> p->wide_logl);
        LaunchTimer lt(p, CWT_KCLASS_FORWARD, 0.0, fs);
        const TransposeArgs a{p->d_Fp, p->d_Ft, (int32_t)p->M, L, A, 0};
        const dim3 grid((L + 31) / 32, (A + 31) / 32);
        if (p->rec) {
            rec_launch(p, (const void*)k_spec_transpose_g, grid, dim3(32, 8), 0, fs, a);
        } else {
            k_spec_transpose<<<grid, dim3(32, 8), 0, fs>>>(a);
            CWT_CUDA(p, cudaGetLastError());
            lt.done();
        }
    }

    if (p->child) {
        if ((st = ev_record(p, p->ev_pfwd, fs)) != CWT_OK) return st;
        if ((st = run_launches(p->child, signal, Wc, sc, s)) != CWT_OK) return st;
        if ((st = ev_wait(p, s, p->ev_pfwd)) != CWT_OK) return st;
    }

    // 2-3. band scales (one launch per DFT length) and wide-scale batches
    //      (pass 1 then pass 2 through an L2-sized intermediate) are independent
    //      once F exists: they are spread over the call's stream and side
    //      streams forked after the forward transform; each stream has its own
    //      intermediate Y.
    const int nwork = (int)(p->groups.size() + p->wide.size());
    const int nstreams = serial ? 1 : std::min(nwork, cwt_plan::kSide + 1);
    cudaStream_t streams[cwt_plan::kSide + 1] = {s};
    if (nstreams > 1) {
        if ((st = ev_record(p, p->ev_fork, s)) != CWT_OK) return st;
        for (int i = 1; i < nstreams; i++) {
            streams[i] = p->side[i - 1];
            if ((st = ev_wait(p, streams[i], p->ev_fork)) != CWT_OK) return st;
        }
    }
    if (p->child) {
        if ((st = edge_fix(streams[nstreams - 1])) != CWT_OK) return st;
        std::vector<int> cr(p->child_n);
        for (int i = 0; i < p->child_n; i++) cr[i] = p->child_r0 + i;
        if ((st = host_copy_rows(p, streams[nstreams - 1], cr)) != CWT_OK) return st;
    }
    int next = 0;
    // wide batches first (longest chains), round robin; band groups fill in
    for (size_t wi = 0; wi < p->wide.size(); wi++) {
        const auto& wb = p->wide[wi];
        const int si = next++ % nstreams;
        cudaStream_t ws = streams[si];
        const Entry& e2 = wide2_entry(p);
        const int L = 1 << p->wide_logl;
        Params Q = P;
        Q.job0 = wb.job0;
        Q.A = (int32_t)(p->M >> p->wide_logl);
        Q.Y = p->d_Y + (size_t)si * p->y_stride;
        const bool tc = wide2_on_tc(p);
        Q.yperm = tc && p->opts.precision != CWT_PRECISION_FP32;   // Y rows in the tensor-core stages' order
        if (wb.logl1 < 0) {
            const Entry& e1 = tb.wide1[p->wide_loga];
            if ((st = launch(p, e1, dim3((L + e1.T - 1) / e1.T, wb.count), stage_smem(p->wide_loga, e1.T), Q, ws,
                             CWT_KCLASS_WIDE1, wb.band_bytes)) != CWT_OK)
                return st;
        } else {
            const EntryP& e1 = tb.wide1p[wb.logl1][wb.var];
            const int A1 = Q.A >> wb.logl1;
            const int tpb = (A1 + e1.T - 1) / e1.T;
            size_t smem = (size_t)(1 << wb.logl1) * sizeof(float2) + stage_smem(wb.logl1, e1.T);
            if (!e1.fn || !e1.gfn) return fail(p, CWT_ERR_INTERNAL, "missing pass-1 instantiation");
            const Wide1pArgs a{Q, L, tpb, {0, 0}};
            const dim3 grid(L * tpb, wb.count);
            if (p->rec) {
                rec_launch(p, (const void*)e1.gfn, grid, dim3(e1.NT), smem, ws, a);
            } else {
                if ((st = opt_in_smem(p, (const void*)e1.fn)) != CWT_OK) return st;
                LaunchTimer lt(p, CWT_KCLASS_WIDE1, wb.band_bytes, ws);
                e1.fn<<<grid, e1.NT, smem, ws>>>(a);
                CWT_CUDA(p, cudaGetLastError());
                lt.done();
            }
        }
        Q.D = wb.D;
        const int tiles2 = (Q.A + e2.T - 1) / e2.T;
        const dim3 grid2((tiles2 + Q.D - 1) / Q.D, wb.count);
        if (tc) {
            const TcEntry& te = tb.wide2_tc[p->opts.precision][p->crop];
            Q.yz0 = (int32_t)((size_t)si * p->y_stride / (size_t)p->M);
            Q.err = p->d_err;
            if (!te.fn || !te.gfn) return fail(p, CWT_ERR_INTERNAL, "missing tensor-core pass-2 instantiation");
            if (p->rec) {
                rec_launch(p, (const void*)te.gfn, grid2, dim3(kTcThreads), te.gsmem, ws, Q);
            } else {
                if ((st = opt_in_smem(p, (const void*)te.fn)) != CWT_OK) return st;
                LaunchTimer lt(p, CWT_KCLASS_WIDE2, wb.out_bytes, ws);
                te.fn<<<grid2, te.NT, te.smem, ws>>>(Q, p->ymap);
                CWT_CUDA(p, cudaGetLastError());
                lt.done();
            }
        } else if ((st = launch(p, e2, grid2, stage_smem(p->wide_logl, e2.T), Q, ws, CWT_KCLASS_WIDE2,
                                wb.out_bytes)) != CWT_OK) {
            return st;
        }
        if ((st = host_copy_rows(p, ws, rows_of_jobs(p, wb.job0, wb.count))) != CWT_OK) return st;
    }
    // recording a batch: every band group on a stream of its own (a key only the
    // recorder sees), forked where the band work may start, so that independent
    // groups share one dependency level; the call's stream joins them all
    const int fork_level = p->rec ? p->rec->level_of((const void*)s) : 0;
    int band_level = fork_level;
    for (size_t gi = 0; gi < p->groups.size(); gi++) {
        const auto& g = p->groups[gi];
        const Entry& e = g.rdi ? tb.band_rd[g.rdi][p->crop] : tb.band[g.logl][p->crop];
        Params Q = P;
        Q.A = (int32_t)(p->M >> g.logl);
        Q.tile_job = p->d_tile_job + g.tj_off;
        Q.D = g.D;
        size_t smem = (size_t)((1 << g.rdi) << g.logl) * sizeof(float2) + stage_smem(g.logl, e.T);
        cudaStream_t gs = streams[next++ % nstreams];
        if (p->rec) {
            const void* key = &p->groups[gi];
            p->rec->stream_level[key] = fork_level;
            gs = (cudaStream_t)key;
        }
        if ((st = launch(p, e, dim3(g.ntiles), smem, Q, gs, CWT_KCLASS_BAND, g.bytes)) != CWT_OK) return st;
        if (p->rec) band_level = std::max(band_level, p->rec->level_of((const void*)gs));
        if ((st = host_copy_rows(p, gs, rows_of_jobs(p, g.job0, g.njobs))) != CWT_OK) return st;
    }
    if (p->rec) p->rec->stream_level[(const void*)s] = std::max(p->rec->level_of((const void*)s), band_level);
    for (int i = 1; i < nstreams; i++) {
        if ((st = ev_record(p, p->ev_join[i - 1], streams[i])) != CWT_OK) return st;
        if ((st = ev_wait(p, s, p->ev_join[i - 1])) != CWT_OK) return st;
    }

    // 4. power spectrum: fixed-order reduction of the per-tile partials
    if (spectrum) {
        LaunchTimer lt(p, CWT_KCLASS_POWER, 8.0 * (double)(p->n_partials + p->S), s);
        if (p->rec) {
            const PowerArgs a{p->d_partials, p->d_part_off, p->d_part_cnt, spectrum, p->out_len, p->S, 0};
            rec_launch(p, (const void*)k_power_finalize_g, dim3(p->S), dim3(32), 0, s, a);
        } else {
            k_power_finalize<<<p->S, 32, 0, s>>>(p->d_partials, p->d_part_off, p->d_part_cnt, p->S, p->out_len,
                                                 spectrum);
            CWT_CUDA(p, cudaGetLastError());
            lt.done();
        }
    }
    return CWT_OK;
}

// Runs the launch sequence as a CUDA graph captured on the call's stream and
// replayed while (signal, W, spectrum) repeat.  Direct launches when timing is
// on, on the legacy default stream, inside a caller's own capture, or if
// capture is unavailable.
// A tensor-core pass 2 of an earlier call (this plan or one of its sub-plans)
// whose bounded wait for a TMA copy gave up: reported once, as CWT_ERR_TIMEOUT.
bool take_timeout(cwt_plan* p) {
    bool t = false;
    if (p->h_err && *(volatile int32_t*)p->h_err) {
        *(volatile int32_t*)p->h_err = 0;
        t = true;
    }
    if (p->child) t |= take_timeout(p->child);
    for (cwt_plan* q : p->subs) t |= take_timeout(q);
    return t;
}

cwt_status run(cwt_plan* p, const void* signal, void* W, double* spectrum, cudaStream_t s) {
    if (take_timeout(p)) return fail(p, CWT_ERR_TIMEOUT, "a tensor-core pass 2 of an earlier call gave up waiting");
    if (p->opts.scratch == CWT_SCRATCH_CALLER) {
        // the scratch changes from call to call: no graph replay
        if (!p->scratch_base) return fail(p, CWT_ERR_INVALID_ARG, "the plan runs with caller scratch (cwt_exec_scratch)");
        return run_launches(p, signal, W, spectrum, s);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (p->timing || p->hc.on || !p->graphs_ok || s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread ||
        cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return run_launches(p, signal, W, spectrum, s);
    if (p->gexec && p->gkey[0] == signal && p->gkey[1] == W && p->gkey[2] == spectrum) {
        CWT_CUDA(p, cudaGraphLaunch(p->gexec, s));
        return CWT_OK;
    }
    // capture only when a call repeats the previous call's pointers: a caller
    // with fresh buffers every call (a request server) launches directly
    if (p->skey[0] != signal || p->skey[1] != W || p->skey[2] != spectrum) {
        p->skey[0] = signal;
        p->skey[1] = W;
        p->skey[2] = spectrum;
        return run_launches(p, signal, W, spectrum, s);
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        p->graphs_ok = false;
        return run_launches(p, signal, W, spectrum, s);
    }
    cwt_status st = run_launches(p, signal, W, spectrum, s);
    cudaError_t e = cudaStreamEndCapture(s, &g);
    cudaGraphExec_t x = nullptr;
    if (st == CWT_OK && e == cudaSuccess) e = cudaGraphInstantiate(&x, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != CWT_OK || e != cudaSuccess) {
        cudaGetLastError();
        p->graphs_ok = false;
        return run_launches(p, signal, W, spectrum, s);
    }
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->gexec = x;
    p->gkey[0] = signal;
    p->gkey[1] = W;
    p->gkey[2] = spectrum;
    CWT_CUDA(p, cudaGraphLaunch(x, s));
    return CWT_OK;
}

bool aligned(const void* q, size_t a) { return ((uintptr_t)q % a) == 0; }

}  // namespace

cwt_status plan_fail(cwt_plan* p, cwt_status st, const char* msg) { return fail(p, st, msg); }
cwt_status plan_check_device(cwt_plan* p) { return check_device(p); }

// Periodic boundary with N not a power of two (GDW, Morlet).  A scale whose
// wavelet is negligible beyond E samples gives the same W on [0, N) as the
// zero-boundary transform of the signal extended periodically by E samples on
// each side, kept on [E, E + N), when the padded length M is at least
// N + 2E + 1: an output n in the window reads the extended samples n - E ..
// n + E directly, and its wrapped neighbours n + t - M (|t| <= E) fall below
// index 0 while n + t + M lies beyond the extension's N + 2E samples.  (Every
// output of the extended signal would need N + 3E + 1; only the window is
// kept.)  Consecutive rows sharing the power-of-two length M >= N + 2E + 1 form
// one zero-boundary sub-plan of fft_len M; a row of the group with a shorter
// support E' <= E needs less.  Scales
// whose spectrum is not negligible (1e-7 of its peak) at the Nyquist frequency
// are refused: their band-limited wavelet rings instead of decaying.
// Periodic boundary for any N, every wavelet and every scale: the N-point
// transforms of Eqs. 8-9 by Bluestein's chirp transform (cwt_bluestein.cuh)
// over power-of-two FFTs of length P >= 2N - 1.  wt: the rows' w~.  No band
// truncation: every bin of the N-point grid enters.
cwt_status create_bluestein(cwt_plan** plan, int64_t N, const double* wt, int32_t n_scales, int32_t wavelet,
                            const cwt_plan_opts& o) {
    int64_t P = 4;
    while (P < 2 * N - 1) P <<= 1;
    if (P > (int64_t(1) << kMaxLogM)) return CWT_ERR_UNSUPPORTED;
    cwt_plan* p = new (std::nothrow) cwt_plan();
    if (!p) return CWT_ERR_OOM;
    p->N = N;
    p->out_len = N;
    p->M = P;
    p->logM = ilog2(P);
    p->S = n_scales;
    p->wavelet = wavelet;
    p->boundary = CWT_BOUNDARY_PERIODIC;
    p->opts = o;
    p->opts.scale_unit = CWT_SCALE_W_TILDE;
    p->w_tilde.assign(wt, wt + n_scales);
    p->bs = true;
    p->fwd_small = P <= kLmax;
    p->wide_logl = std::max(kWideLog, p->logM - kLmaxLog);
    p->wide_loga = p->logM - p->wide_logl;
    auto bail = [&](cwt_status st) {
        free_plan(p);
        return st;
    };
    if (cudaGetDevice(&p->device) != cudaSuccess) return bail(CWT_ERR_CUDA);
    // jobs: a Morlet row each, or two real-wavelet rows; one power partial per
    // output block of each row
    const int per = wav_real(wavelet) ? 2 : 1;
    const int64_t nb = (N + kBsOutBlock - 1) / kBsOutBlock;
    p->part_off.assign(n_scales, 0);
    p->part_cnt.assign(n_scales, 0);
    int64_t nparts = 0;
    for (int32_t i0 = 0; i0 < n_scales; i0 += per) {
        Job J{};
        for (int q = 0; q < 2; q++) {
            const int32_t s = i0 + q;
            if (q < per && s < n_scales) {
                J.g[q] = make_gen(p, wt[s], s, N);
                J.g[q].part_off = (int32_t)nparts;
                p->part_off[s] = (int32_t)nparts;
                p->part_cnt[s] = (int32_t)nb;
                nparts += nb;
            } else {
                J.g[q] = ScaleGen{};
                J.g[q].row = -1;
            }
        }
        J.k_lo = 0;
        J.K = (int32_t)N;
        p->jobs.push_back(J);
    }
    p->n_partials = nparts;
    // c_j = e^{i pi j^2 / N}, the phase reduced exactly: j^2 mod 2N
    std::vector<float2> chirp((size_t)N);
    for (int64_t j = 0; j < N; j++) {
        const int64_t r = (int64_t)(((unsigned __int128)j * (unsigned __int128)j) % (unsigned __int128)(2 * N));
        const double ang = kPi * (double)r / (double)N;
        chirp[(size_t)j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
    cwt_status st;
    if ((st = upload(p, &p->d_jobs, p->jobs)) != CWT_OK) return bail(st);
    if ((st = upload(p, &p->d_part_off, p->part_off)) != CWT_OK) return bail(st);
    if ((st = upload(p, &p->d_part_cnt, p->part_cnt)) != CWT_OK) return bail(st);
    if ((st = upload_twiddles(p)) != CWT_OK) return bail(st);
    if ((st = upload(p, &p->d_bs_chirp, chirp)) != CWT_OK) return bail(st);
    if ((st = scratch_alloc(p, &p->d_partials, (size_t)std::max<int64_t>(1, nparts))) != CWT_OK) return bail(st);
    if ((st = dev_alloc(p, &p->d_bs_G, (size_t)(2 * P))) != CWT_OK) return bail(st);
    p->bs_streams = std::min<int>((int)p->jobs.size(), cwt_plan::kSide + 1);
    if ((st = scratch_alloc(p, &p->d_bs_work, (size_t)(P + 2 * P * p->bs_streams))) != CWT_OK) return bail(st);
    if (!p->fwd_small && (st = scratch_alloc(p, &p->d_Y, (size_t)(P * p->bs_streams))) != CWT_OK) return bail(st);
    if (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess) return bail(CWT_ERR_CUDA);
    for (int i = 0; i < cwt_plan::kSide; i++)
        if (cudaStreamCreateWithFlags(&p->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&p->ev_join[i], cudaEventDisableTiming) != cudaSuccess)
            return bail(CWT_ERR_CUDA);
    // D of the chirp sequences: [0] conj(c) (signal stage), [1] c (scales); a
    // plan with caller scratch computes them in a temporary one
    char* tmp = nullptr;
    if (p->opts.scratch == CWT_SCRATCH_CALLER) {
        const cudaError_t e = cudaMalloc((void**)&tmp, p->scratch_own);
        if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? CWT_ERR_OOM : CWT_ERR_CUDA);
        set_scratch(p, tmp);
    }
    struct TmpScratch {   // freed on every return (after the plan, on the error paths)
        char* t;
        ~TmpScratch() {
            if (t) cudaFree(t);
        }
    } tmp_guard{tmp};
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(CWT_ERR_CUDA);
    const Params B = base_params(p);
    const unsigned gp = (unsigned)std::min<int64_t>((P + kBsThreads - 1) / kBsThreads, 4096);
    for (int q = 0; q < 2 && st == CWT_OK; q++) {
        BsArgs a{};
        a.chirp = p->d_bs_chirp;
        a.dst = p->d_bs_work + P;
        a.N = N;
        a.P = (int32_t)P;
        a.conj_c = q == 0;
        k_bs_seq<<<gp, kBsThreads, 0, s>>>(a);
        if (cudaGetLastError() != cudaSuccess) st = CWT_ERR_CUDA;
        Params Q = B;
        Q.cin = p->d_bs_work + P;
        Q.Fp_out = p->d_bs_G + q * P;
        Q.cmode = 3;
        Q.Y = p->d_Y;
        if (st == CWT_OK) st = launch_forward(p, Q, s, 0.0, 0.0);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && st == CWT_OK) st = CWT_ERR_CUDA;
    cudaStreamDestroy(s);
    if (st != CWT_OK) return bail(st);
    if (tmp) set_scratch(p, nullptr);
    *plan = p;
    return CWT_OK;
}

cwt_status create_periodic_extended(cwt_plan** plan, int64_t N, const double* scales, int32_t n_scales,
                                    int32_t wavelet, const cwt_plan_opts& o) {
    std::vector<double> wt(n_scales);
    for (int32_t i = 0; i < n_scales; i++) wt[i] = o.scale_unit == CWT_SCALE_DILATION ? 1.0 / scales[i] : scales[i];
    // rows the extended-signal form cannot take (Mr = 0): other wavelets, scales
    // whose spectrum is not negligible at the Nyquist frequency, and padded
    // lengths beyond 2^kMaxLogM go to the Bluestein form (create_bluestein)
    const bool ext_ok = wavelet == CWT_WAVELET_GDW || wavelet == CWT_WAVELET_MORLET;
    double u_lo = 0.0, u_hi = 0.0;
    if (ext_ok) wavelet_band(wavelet, o.omega0, 1e-7, &u_lo, &u_hi);
    std::vector<int64_t> E(n_scales, 0), Mr(n_scales, 0);
    for (int32_t i = 0; i < n_scales; i++) {
        if (!ext_ok) continue;
        const double nyq = kPi / wt[i];                  // u at the Nyquist frequency
        if (u_hi >= nyq || u_lo <= -nyq) continue;
        const int64_t e = edge_width(wavelet, wt[i]);
        const int64_t m = int64_t(1) << ilog2(N + 2 * e + 1);
        if (m > (int64_t(1) << kMaxLogM)) continue;
        E[i] = e;
        Mr[i] = m;
    }
    int64_t P = 4;                               // the Bluestein form's FFT length
    while (P < 2 * N - 1) P <<= 1;
    for (int32_t i = 0; i < n_scales; i++)
        if (Mr[i] == 0 && P > (int64_t(1) << kMaxLogM)) return CWT_ERR_UNSUPPORTED;
    cwt_plan* p = new (std::nothrow) cwt_plan();
    if (!p) return CWT_ERR_OOM;
    p->N = N;
    p->out_len = N;
    p->S = n_scales;
    p->wavelet = wavelet;
    p->boundary = CWT_BOUNDARY_PERIODIC;
    p->opts = o;
    p->w_tilde = wt;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        free_plan(p);
        return CWT_ERR_CUDA;
    }
    for (int32_t r0 = 0; r0 < n_scales;) {
        int32_t r1 = r0 + 1;
        while (r1 < n_scales && Mr[r1] == Mr[r0]) r1++;
        int64_t Eg = 0;
        for (int32_t i = r0; i < r1; i++) Eg = std::max(Eg, E[i]);
        cwt_plan* sub = nullptr;
        cwt_status st;
        if (Mr[r0] == 0) {
            // Bluestein rows read the signal itself (the extension's middle, E = 0)
            st = create_bluestein(&sub, N, wt.data() + r0, r1 - r0, wavelet, o);
        } else {
            cwt_plan_opts so = o;
            so.scale_unit = CWT_SCALE_W_TILDE;
            so.fft_len = Mr[r0];
            st = cwt_plan_create_ex(&sub, N + 2 * Eg, wt.data() + r0, r1 - r0, wavelet, CWT_BOUNDARY_ZERO, &so);
            if (st == CWT_OK) {
                sub->out_off = Eg;
                sub->out_len = N;
            }
        }
        if (st != CWT_OK) {
            free_plan(p);
            return st;
        }
        p->subs.push_back(sub);
        p->sub_r0.push_back(r0);
        p->sub_E.push_back(Eg);
        p->ext_E = std::max(p->ext_E, Eg);
        p->ws_bytes += sub->ws_bytes;
        p->M = std::max(p->M, sub->M);
        r0 = r1;
    }
    p->logM = ilog2(p->M);
    const size_t se = o.input_dtype == CWT_INPUT_F64 ? sizeof(double) : sizeof(float);
    cwt_status st = scratch_alloc(p, reinterpret_cast<char**>(&p->d_ext), (size_t)(N + 2 * p->ext_E) * se);
    if (st != CWT_OK) {
        free_plan(p);
        return st;
    }
    *plan = p;
    return CWT_OK;
}

// ==================================================================== batches

// A batch runs the launch sequences of several plans, each bound to its own
// signal, W and spectrum, as grouped launches.  Every plan's launches are
// recorded with their dependency levels (Recorder); the launches of one kernel
// instantiation at one level, from all plans, become one grid whose CTAs find
// their own launch's argument and block coordinates through a per-CTA index
// (GroupMap).  The levels run one after another on the call's stream; the
// groups of a level are spread over n_streams streams.
constexpr int kBatchMaxStreams = 8;

struct cwt_batch {
    int device = -1;
    struct Group {
        const void* gfn;
        dim3 block;
        size_t smem;
        int level;
        int64_t ctas;
        int32_t stride;
        size_t args_off, geom_off, sub_off;     // byte offsets into d_buf
    };
    std::vector<Group> groups;                  // in level order
    std::vector<int> level_first;               // groups of level l: [level_first[l], level_first[l + 1])
    unsigned char* d_buf = nullptr;
    int n_streams = 1;
    cudaStream_t side[kBatchMaxStreams] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kBatchMaxStreams] = {};
    int64_t recorded = 0, ctas = 0;
};

namespace {

void set_rec(cwt_plan* p, Recorder* r) {
    p->rec = r;
    if (p->child) set_rec(p->child, r);
    for (cwt_plan* q : p->subs) set_rec(q, r);
}

void free_batch(cwt_batch* b) {
    if (!b) return;
    if (b->d_buf) cudaFree(b->d_buf);
    for (int i = 0; i < kBatchMaxStreams; i++) {
        if (b->side[i]) cudaStreamDestroy(b->side[i]);
        if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    delete b;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

// Zero boundary with N not a power of two (GDW, Morlet).  The zero-padded
// transform restricted to n < N is the linear convolution of f with the
// dilated wavelet; with M' >= N + E + 1 points (E: the support of the dilated
// wavelet, beyond which it is negligible) no output n < N sees a wrapped term,
// so a scale gives the same W with any such M' as with the default M (the
// power of two >= 2N).  Consecutive rows sharing the power-of-two length
// M' = min(M, pow2 >= N + E + 1) form zero-boundary sub-plans of fft_len M'.
// *plan stays NULL (and CWT_OK is returned) when every row needs the default M.
cwt_status create_zero_split(cwt_plan** plan, int64_t N, const double* scales, int32_t n_scales, int32_t wavelet,
                             const cwt_plan_opts& o) {
    *plan = nullptr;
    const int64_t Mdef = int64_t(1) << ilog2(2 * N);
    std::vector<double> wt(n_scales);
    std::vector<int64_t> Mr(n_scales);
    bool shorter = false;
    for (int32_t i = 0; i < n_scales; i++) {
        wt[i] = o.scale_unit == CWT_SCALE_DILATION ? 1.0 / scales[i] : scales[i];
        const int64_t E = edge_width(wavelet, wt[i]);
        Mr[i] = nyquist_clear(wavelet, o.omega0, wt[i]) ? std::min(Mdef, int64_t(1) << ilog2(N + E + 1)) : Mdef;
        shorter |= Mr[i] < Mdef;
    }
    if (!shorter || Mdef > (int64_t(1) << kMaxLogM)) return CWT_OK;
    cwt_plan* p = new (std::nothrow) cwt_plan();
    if (!p) return CWT_ERR_OOM;
    p->N = N;
    p->out_len = N;
    p->S = n_scales;
    p->wavelet = wavelet;
    p->boundary = CWT_BOUNDARY_ZERO;
    p->opts = o;
    p->w_tilde = wt;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        free_plan(p);
        return CWT_ERR_CUDA;
    }
    for (int32_t r0 = 0; r0 < n_scales;) {
        int32_t r1 = r0 + 1;
        while (r1 < n_scales && Mr[r1] == Mr[r0]) r1++;
        cwt_plan_opts so = o;
        so.scale_unit = CWT_SCALE_W_TILDE;
        so.fft_len = Mr[r0];
        cwt_plan* sub = nullptr;
        cwt_status st = cwt_plan_create_ex(&sub, N, wt.data() + r0, r1 - r0, wavelet, CWT_BOUNDARY_ZERO, &so);
        if (st != CWT_OK) {
            free_plan(p);
            return st;
        }
        p->subs.push_back(sub);
        p->sub_r0.push_back(r0);
        p->sub_E.push_back(0);
        p->ws_bytes += sub->ws_bytes;
        p->M = std::max(p->M, Mr[r0]);
        r0 = r1;
    }
    p->logM = ilog2(p->M);
    *plan = p;
    return CWT_OK;
}

// Plan-time tuning (opts.tune = 1).  Plans with candidate plan options are
// created and timed on this device, running the transform with power on a zero
// signal into temporary buffers of the output's size (the kernels' work does
// not depend on the values); the fastest plan is kept and the others
// destroyed.  Two stages, each keeping any value the caller fixed:
//   1. launch shape: the CTA target of the W-writing launches (152, 304, 608)
//      and the intermediate of a wide-scale launch (64, 128, 256 MiB for the
//      tile pipeline of pass 2; 16, 32 MiB for the CTA Stockham kernel);
//   2. stage fusion: the band kernels' direct depth (4, 2, 1), i.e. whether a
//      band of up to 4096 / 2048 bins is evaluated in one pass with the first
//      DFT stage fed by a Horner sum, or goes through the two-pass path.
// With the environment variable CWT_TUNE_CACHE naming a file, the choice is
// looked up there first (keyed by the device and every input of the plan) and
// appended after tuning, so a later process skips the timing.
namespace {

constexpr uint64_t kTuneVersion = 4;   // 4: wave-aware tiles per CTA; 3: pass-2 kernel per plan, per-batch pass-2 grids

uint64_t fnv1a(uint64_t h, const void* data, size_t n) {
    const unsigned char* b = (const unsigned char*)data;
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

std::string tune_key(int64_t N, const double* scales, int32_t n_scales, int32_t wavelet, int32_t boundary,
                     const cwt_plan_opts& o, std::string* device_name) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, dev);
    uint64_t h = 14695981039346656037ull;
    h = fnv1a(h, &kTuneVersion, sizeof(kTuneVersion));
    h = fnv1a(h, prop.name, std::strlen(prop.name));
    h = fnv1a(h, &prop.multiProcessorCount, sizeof(int));
    h = fnv1a(h, &N, sizeof(N));
    h = fnv1a(h, &n_scales, sizeof(n_scales));
    h = fnv1a(h, scales, sizeof(double) * (size_t)n_scales);
    h = fnv1a(h, &wavelet, sizeof(wavelet));
    h = fnv1a(h, &boundary, sizeof(boundary));
    const double d[3] = {o.omega0, o.dx, o.eps_trunc};
    const int64_t q[8] = {o.scale_unit, o.input_dtype, o.fft_len, o.precision, o.min_ctas, o.wide_batch_bytes,
                          o.band_depth, o.wide2_kernel};
    h = fnv1a(h, d, sizeof(d));
    h = fnv1a(h, q, sizeof(q));
    char buf[32];
    std::snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)h);
    if (device_name) {
        *device_name = prop.name;
        for (char& ch : *device_name)
            if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
    }
    return buf;
}

std::mutex g_tune_mu;

bool tune_cache_lookup(const std::string& key, cwt_plan_opts* o) {
    const char* path = std::getenv("CWT_TUNE_CACHE");
    if (!path || !*path) return false;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        char k[64];
        int ctas = 0, depth = 0;
        long long wb = 0;
        if (std::sscanf(line, "%63s %d %lld %d", k, &ctas, &wb, &depth) == 4 && key == k && ctas > 0 && wb > 0 &&
            (depth == 1 || depth == 2 || depth == 4)) {
            o->min_ctas = ctas;
            o->wide_batch_bytes = wb;
            o->band_depth = depth;
            found = true;          // the last entry for a key wins
        }
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(const std::string& key, const cwt_plan_opts& o, float ms, const std::string& dev) {
    const char* path = std::getenv("CWT_TUNE_CACHE");
    if (!path || !*path) return;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %lld %d %.4f %s\n", key.c_str(), o.min_ctas, (long long)o.wide_batch_bytes, o.band_depth,
                 ms, dev.c_str());
    std::fclose(f);
}

}  // namespace

cwt_status create_tuned(cwt_plan** plan, int64_t N, const double* scales, int32_t n_scales, int32_t wavelet,
                        int32_t boundary, const cwt_plan_opts& o) {
    std::string dev_name;
    const std::string key = tune_key(N, scales, n_scales, wavelet, boundary, o, &dev_name);
    {
        cwt_plan_opts oc = o;
        if (tune_cache_lookup(key, &oc)) {
            oc.tune = 0;
            cwt_status st = cwt_plan_create_ex(plan, N, scales, n_scales, wavelet, boundary, &oc);
            if (st == CWT_OK) (*plan)->opts.tune = 1;
            return st;
        }
    }
    struct Cand { int32_t ctas; int64_t wb; int32_t depth; };
    std::vector<Cand> cands;
    const std::vector<int64_t> wb_cands =
        o.precision == CWT_PRECISION_FP32 && o.wide2_kernel == 2
            ? std::vector<int64_t>{int64_t(32) << 20, int64_t(16) << 20}
        : o.precision == CWT_PRECISION_FP32 && o.wide2_kernel == 0
            ? std::vector<int64_t>{int64_t(128) << 20, int64_t(32) << 20, int64_t(256) << 20}
                                          : std::vector<int64_t>{int64_t(128) << 20, int64_t(64) << 20, int64_t(256) << 20};
    const int32_t depth0 = o.band_depth ? o.band_depth : 4;
    for (int32_t c : {152 * 2, 152, 152 * 4})
        for (int64_t wb : wb_cands) {
            const Cand k{o.min_ctas ? o.min_ctas : c, o.wide_batch_bytes ? o.wide_batch_bytes : wb, depth0};
            bool dup = false;
            for (const Cand& q : cands) dup |= q.ctas == k.ctas && q.wb == k.wb;
            if (!dup) cands.push_back(k);
        }
    cwt_plan* best = nullptr;
    Cand best_c{};
    float best_ms = 0.f;
    void* sig = nullptr;
    void* W = nullptr;
    double* sp = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cwt_status rc = CWT_OK;
    auto cuda_ok = [&](cudaError_t e) {
        if (e == cudaSuccess) return true;
        cudaGetLastError();
        rc = e == cudaErrorMemoryAllocation ? CWT_ERR_OOM : CWT_ERR_CUDA;
        return false;
    };
    // creates and times one candidate; keeps it if it is the fastest so far
    auto try_cand = [&](const Cand& c) -> bool {
        cwt_plan_opts oc = o;
        oc.tune = 0;
        oc.min_ctas = c.ctas;
        oc.wide_batch_bytes = c.wb;
        oc.band_depth = c.depth;
        cwt_plan* q = nullptr;
        if ((rc = cwt_plan_create_ex(&q, N, scales, n_scales, wavelet, boundary, &oc)) != CWT_OK) return false;
        if (!sig) {
            const size_t se = o.input_dtype == CWT_INPUT_F64 ? sizeof(double) : sizeof(float);
            const size_t we = wavelet == CWT_WAVELET_MORLET ? sizeof(float2) : sizeof(float);
            if (!cuda_ok(cudaMalloc(&sig, (size_t)N * se)) || !cuda_ok(cudaMemset(sig, 0, (size_t)N * se)) ||
                !cuda_ok(cudaMalloc(&W, (size_t)n_scales * (size_t)N * we)) ||
                !cuda_ok(cudaMalloc(&sp, (size_t)n_scales * sizeof(double))) ||
                !cuda_ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) || !cuda_ok(cudaEventCreate(&e0)) ||
                !cuda_ok(cudaEventCreate(&e1))) {
                free_plan(q);
                return false;
            }
        }
        float ms = 0.f;
        for (int i = 0; i < 3 && rc == CWT_OK; i++) rc = cwt_exec_with_power(q, sig, W, sp, st);
        if (rc == CWT_OK && cuda_ok(cudaEventRecord(e0, st))) {
            for (int i = 0; i < 5 && rc == CWT_OK; i++) rc = cwt_exec_with_power(q, sig, W, sp, st);
            if (rc == CWT_OK && cuda_ok(cudaEventRecord(e1, st)) && cuda_ok(cudaEventSynchronize(e1)))
                cuda_ok(cudaEventElapsedTime(&ms, e0, e1));
        }
        if (rc != CWT_OK) {
            free_plan(q);
            return false;
        }
        if (!best || ms < best_ms) {
            if (best) free_plan(best);
            best = q;
            best_c = c;
            best_ms = ms;
        } else {
            free_plan(q);
        }
        return true;
    };
    bool ok = true;
    for (const Cand& c : cands)
        if (!(ok = try_cand(c))) break;
    if (ok && o.band_depth == 0)
        for (int32_t d : {8, 16, 2, 1}) {
            const Cand c{best_c.ctas, best_c.wb, d};
            if (!(ok = try_cand(c))) break;
        }
    if (st) cudaStreamSynchronize(st);
    if (sig) cudaFree(sig);
    if (W) cudaFree(W);
    if (sp) cudaFree(sp);
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != CWT_OK) {
        if (best) free_plan(best);
        return rc;
    }
    best->opts.tune = 1;
    tune_cache_store(key, best->opts, best_ms / 5.f, dev_name);
    *plan = best;
    return CWT_OK;
}

// ====================================================================== ABI

extern "C" {

void cwt_plan_opts_default(cwt_plan_opts* o) {
    if (!o) return;
    o->omega0 = 6.0;
    o->dx = 1.0;
    o->scale_unit = CWT_SCALE_DILATION;
    o->input_dtype = CWT_INPUT_F32;
    o->fft_len = 0;
    o->eps_trunc = 1e-10;
    o->min_ctas = 0;
    o->tune = 0;
    o->wide_batch_bytes = 0;
    o->precision = CWT_PRECISION_FP32;
    o->band_depth = 0;
    o->wide2_kernel = 0;
    o->scratch = CWT_SCRATCH_PLAN;
}

cwt_status cwt_plan_create(cwt_plan** plan, int64_t N, const double* scales, int32_t n_scales, int32_t wavelet,
                           int32_t boundary) {
    cwt_plan_opts o;
    cwt_plan_opts_default(&o);
    return cwt_plan_create_ex(plan, N, scales, n_scales, wavelet, boundary, &o);
}

cwt_status cwt_plan_create_ex(cwt_plan** plan, int64_t N, const double* scales, int32_t n_scales,
                              int32_t wavelet, int32_t boundary, const cwt_plan_opts* opts) {
    if (!plan) return CWT_ERR_INVALID_ARG;
    *plan = nullptr;
    cwt_plan_opts o;
    cwt_plan_opts_default(&o);
    if (opts) o = *opts;
    if (N < 2 || n_scales < 1 || !scales) return CWT_ERR_INVALID_ARG;
    if (wavelet < CWT_WAVELET_GDW || wavelet > CWT_WAVELET_CWGDW) return CWT_ERR_INVALID_ARG;
    if (boundary != CWT_BOUNDARY_PERIODIC && boundary != CWT_BOUNDARY_ZERO) return CWT_ERR_INVALID_ARG;
    if (o.scale_unit != CWT_SCALE_DILATION && o.scale_unit != CWT_SCALE_W_TILDE) return CWT_ERR_INVALID_ARG;
    if (o.input_dtype != CWT_INPUT_F32 && o.input_dtype != CWT_INPUT_F64) return CWT_ERR_INVALID_ARG;
    if (!(o.dx > 0.0) || !std::isfinite(o.dx) || !std::isfinite(o.omega0) || !(o.eps_trunc >= 0.0) ||
        o.eps_trunc >= 1.0)
        return CWT_ERR_INVALID_ARG;
    if (wavelet == CWT_WAVELET_MORLET && !(o.omega0 > 0.0)) return CWT_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n_scales; i++)
        if (!std::isfinite(scales[i]) || !(scales[i] > 0.0)) return CWT_ERR_INVALID_ARG;
    if (o.min_ctas < 0 || o.min_ctas > (1 << 20) || o.wide_batch_bytes < 0 ||
        o.wide_batch_bytes > (int64_t(1) << 36) || (o.tune != 0 && o.tune != 1) ||
        o.precision < CWT_PRECISION_FP32 || o.precision > CWT_PRECISION_BF16X3 ||
        (o.band_depth != 0 && o.band_depth != 1 && o.band_depth != 2 && o.band_depth != 4 && o.band_depth != 8 &&
         o.band_depth != 16) ||
        o.wide2_kernel < 0 || o.wide2_kernel > 2 || (o.scratch != CWT_SCRATCH_PLAN && o.scratch != CWT_SCRATCH_CALLER) ||
        (o.scratch == CWT_SCRATCH_CALLER && o.tune != 0))
        return CWT_ERR_INVALID_ARG;
    if (o.tune) return create_tuned(plan, N, scales, n_scales, wavelet, boundary, o);
    if (o.min_ctas == 0) o.min_ctas = kMinCtas;
    if (o.band_depth == 0) o.band_depth = 4;
    const int32_t req_wide2_kernel = o.wide2_kernel;      // as given (0: chosen per plan)
    const int64_t req_wide_batch_bytes = o.wide_batch_bytes;

    int64_t M;
    if (boundary == CWT_BOUNDARY_PERIODIC) {
        if (o.fft_len != 0 && o.fft_len != N) return CWT_ERR_INVALID_ARG;
        if (!is_pow2(N)) return create_periodic_extended(plan, N, scales, n_scales, wavelet, o);
        M = N;
    } else {
        if (o.fft_len != 0) {
            if (o.fft_len < N) return CWT_ERR_INVALID_ARG;
            if (!is_pow2(o.fft_len)) return CWT_ERR_UNSUPPORTED;
            M = o.fft_len;
        } else {
            M = int64_t(1) << ilog2(2 * N);
            if (!is_pow2(N) && (wavelet == CWT_WAVELET_GDW || wavelet == CWT_WAVELET_MORLET)) {
                cwt_status st = create_zero_split(plan, N, scales, n_scales, wavelet, o);
                if (st != CWT_OK || *plan) return st;
            }
        }
    }
    if (M < 2 || M > (int64_t(1) << kMaxLogM)) return CWT_ERR_UNSUPPORTED;
    // the wide scales' FP32 pass 2: the tile pipeline from M = 2^21, where it
    // measured faster, the CTA Stockham kernel below; the default wide batch
    // follows the kernel
    if (o.wide2_kernel == 0) o.wide2_kernel = M >= (int64_t(1) << 21) ? 1 : 2;
    if (o.wide_batch_bytes == 0)
        o.wide_batch_bytes =
            (int64_t)(o.precision == CWT_PRECISION_FP32 && o.wide2_kernel == 2 ? kWideBatchBytes : kWideBatchBytesTc);

    cwt_plan* p = new (std::nothrow) cwt_plan();
    if (!p) return CWT_ERR_OOM;
    p->N = N;
    p->out_len = N;
    p->M = M;
    p->logM = ilog2(M);
    p->S = n_scales;
    p->wavelet = wavelet;
    p->boundary = boundary;
    p->opts = o;
    p->w_tilde.resize(n_scales);
    for (int32_t i = 0; i < n_scales; i++)
        p->w_tilde[i] = o.scale_unit == CWT_SCALE_DILATION ? 1.0 / scales[i] : scales[i];
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        free_plan(p);
        return CWT_ERR_CUDA;
    }
    // zero boundary with the default padding (M = 2N): a contiguous run of rows
    // with short wavelet support goes to a periodic N-point child plan
    if (boundary == CWT_BOUNDARY_ZERO && o.fft_len == 0 && is_pow2(N) && N >= 1024 &&
        (wavelet == CWT_WAVELET_GDW || wavelet == CWT_WAVELET_MORLET)) {
        // the correction costs ~E^2 per row against the saving of half an M-point
        // transform: E <= max(N / 512, 256) (N / 512 measured best at N = 2^20, 2^22)
        const int64_t emax = std::min<int64_t>({kEdgeMax, std::max<int64_t>(N / 512, 256), N / 4, M - N});
        int r0 = -1, r1 = -1;
        bool contiguous = true;
        for (int32_t i = 0; i < n_scales; i++) {
            if (edge_width(wavelet, p->w_tilde[i]) > emax || !nyquist_clear(wavelet, o.omega0, p->w_tilde[i]))
                continue;
            if (r0 < 0) r0 = i;
            else if (r1 != i) contiguous = false;
            r1 = i + 1;
        }
        if (r0 >= 0 && contiguous) {
            cwt_plan_opts co = o;
            co.scale_unit = CWT_SCALE_W_TILDE;
            co.fft_len = 0;
            co.wide2_kernel = req_wide2_kernel;          // the child chooses by its own length
            co.wide_batch_bytes = req_wide_batch_bytes;
            cwt_status cs = cwt_plan_create_ex(&p->child, N, p->w_tilde.data() + r0, r1 - r0, wavelet,
                                               CWT_BOUNDARY_PERIODIC, &co);
            if (cs != CWT_OK) {
                free_plan(p);
                return cs;
            }
            p->child_r0 = r0;
            p->child_n = r1 - r0;
            p->ws_bytes += p->child->ws_bytes;
        }
    }
    cwt_status st = build_plan(p);
    if (st != CWT_OK) {
        free_plan(p);
        return st;
    }
    *plan = p;
    return CWT_OK;
}

cwt_status cwt_plan_destroy(cwt_plan* plan) {
    if (!plan) return CWT_OK;
    cudaDeviceSynchronize();
    free_plan(plan);
    return CWT_OK;
}

cwt_status cwt_plan_info(const cwt_plan* plan, int64_t* fft_len, size_t* workspace_bytes, int32_t* out_is_complex) {
    if (!plan) return CWT_ERR_INVALID_ARG;
    if (fft_len) *fft_len = plan->M;
    if (workspace_bytes) *workspace_bytes = plan->ws_bytes;
    if (out_is_complex) *out_is_complex = plan->wavelet == CWT_WAVELET_MORLET;
    return CWT_OK;
}

static cwt_status check_exec_args(cwt_plan* plan, const void* signal, const void* W) {
    if (!plan) return CWT_ERR_INVALID_ARG;
    if (!signal || !W) return fail(plan, CWT_ERR_INVALID_ARG, "null signal or W pointer");
    size_t se = plan->opts.input_dtype == CWT_INPUT_F64 ? 8 : 4;
    size_t we = plan->wavelet == CWT_WAVELET_MORLET ? 8 : 4;
    if (!aligned(signal, se) || !aligned(W, we)) return fail(plan, CWT_ERR_INVALID_ARG, "misaligned pointer");
    return check_device(plan);
}

cwt_status cwt_exec(cwt_plan* plan, const void* signal_dev, void* W_dev, void* stream) {
    cwt_status st = check_exec_args(plan, signal_dev, W_dev);
    if (st != CWT_OK) return st;
    return run(plan, signal_dev, W_dev, nullptr, (cudaStream_t)stream);
}

cwt_status cwt_exec_with_power(cwt_plan* plan, const void* signal_dev, void* W_dev, double* spectrum_dev,
                               void* stream) {
    cwt_status st = check_exec_args(plan, signal_dev, W_dev);
    if (st != CWT_OK) return st;
    if (!spectrum_dev || !aligned(spectrum_dev, 8)) return fail(plan, CWT_ERR_INVALID_ARG, "bad spectrum pointer");
    return run(plan, signal_dev, W_dev, spectrum_dev, (cudaStream_t)stream);
}

cwt_status cwt_plan_scratch_bytes(const cwt_plan* plan, size_t* bytes) {
    if (!plan || !bytes) return CWT_ERR_INVALID_ARG;
    *bytes = plan->opts.scratch == CWT_SCRATCH_CALLER ? scratch_tree(plan) : 0;
    return CWT_OK;
}

cwt_status cwt_exec_scratch(cwt_plan* plan, const void* signal_dev, void* W_dev, double* spectrum_dev,
                            void* scratch_dev, size_t scratch_bytes, void* stream) {
    cwt_status st = check_exec_args(plan, signal_dev, W_dev);
    if (st != CWT_OK) return st;
    if (plan->opts.scratch != CWT_SCRATCH_CALLER)
        return fail(plan, CWT_ERR_INVALID_ARG, "the plan has its own scratch (cwt_exec_with_power)");
    if (spectrum_dev && !aligned(spectrum_dev, 8)) return fail(plan, CWT_ERR_INVALID_ARG, "bad spectrum pointer");
    if (!scratch_dev || !aligned(scratch_dev, kScratchAlign) || scratch_bytes < scratch_tree(plan))
        return fail(plan, CWT_ERR_INVALID_ARG, "scratch missing, misaligned or too small");
    if ((st = bind_scratch(plan, (char*)scratch_dev)) == CWT_OK)
        st = run(plan, signal_dev, W_dev, spectrum_dev, (cudaStream_t)stream);
    set_scratch(plan, nullptr);
    return st;
}

cwt_status cwt_wavelet_power(cwt_plan* plan, const void* W_dev, double* spectrum_dev, void* stream) {
    if (!plan) return CWT_ERR_INVALID_ARG;
    size_t we = plan->wavelet == CWT_WAVELET_MORLET ? 8 : 4;
    if (!W_dev || !aligned(W_dev, we) || !spectrum_dev || !aligned(spectrum_dev, 8))
        return fail(plan, CWT_ERR_INVALID_ARG, "bad W or spectrum pointer");
    cwt_status st = check_device(plan);
    if (st != CWT_OK) return st;
    const int64_t chunk = 32768;
    int64_t chunks = (plan->N + chunk - 1) / chunk;
    if (chunks > 65535) return fail(plan, CWT_ERR_UNSUPPORTED, "row too long");
    if (!plan->d_pw_partials || plan->pw_chunks != chunks) {
        if (plan->d_pw_partials) cudaFree(plan->d_pw_partials);
        plan->d_pw_partials = nullptr;
        CWT_CUDA(plan, cudaMalloc((void**)&plan->d_pw_partials, (size_t)chunks * plan->S * sizeof(double)));
        plan->pw_chunks = chunks;
    }
    cudaStream_t s = (cudaStream_t)stream;
    dim3 grid((unsigned)chunks, (unsigned)plan->S);
    LaunchTimer lt(plan, CWT_KCLASS_POWER, out_row_bytes(plan) * plan->S, s);
    k_power_rows<256><<<grid, 256, 0, s>>>(W_dev, plan->N, plan->wavelet == CWT_WAVELET_MORLET, chunk,
                                           plan->d_pw_partials);
    CWT_CUDA(plan, cudaGetLastError());
    lt.done();
    k_power_finalize_uniform<<<plan->S, 32, 0, s>>>(plan->d_pw_partials, (int32_t)chunks, plan->S, plan->N,
                                                    spectrum_dev);
    CWT_CUDA(plan, cudaGetLastError());
    return CWT_OK;
}

cwt_status cwt_exec_host(cwt_plan* plan, const void* signal_host, void* W_host, double* spectrum_host,
                         void* stream) {
    if (!plan) return CWT_ERR_INVALID_ARG;
    if (!signal_host || !W_host) return fail(plan, CWT_ERR_INVALID_ARG, "null host pointer");
    if (plan->opts.scratch == CWT_SCRATCH_CALLER)
        return fail(plan, CWT_ERR_INVALID_ARG, "the plan runs with caller scratch (cwt_exec_scratch)");
    cwt_status st = check_device(plan);
    if (st != CWT_OK) return st;
    size_t se = plan->opts.input_dtype == CWT_INPUT_F64 ? 8 : 4;
    size_t we = plan->wavelet == CWT_WAVELET_MORLET ? 8 : 4;
    size_t sig_bytes = (size_t)plan->N * se, w_bytes = (size_t)plan->N * (size_t)plan->S * we;
    if (!plan->h_sig) CWT_CUDA(plan, cudaMalloc(&plan->h_sig, sig_bytes));
    if (!plan->h_W) CWT_CUDA(plan, cudaMalloc(&plan->h_W, w_bytes));
    if (!plan->h_spec) CWT_CUDA(plan, cudaMalloc((void**)&plan->h_spec, (size_t)plan->S * sizeof(double)));
    cudaStream_t s = (cudaStream_t)stream;
    if (!plan->hc_stream) CWT_CUDA(plan, cudaStreamCreateWithFlags(&plan->hc_stream, cudaStreamNonBlocking));
    if (plan->hc_ev.empty()) {                   // [0]: joins the copy stream back into s
        cudaEvent_t e = nullptr;
        CWT_CUDA(plan, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        plan->hc_ev.push_back(e);
    }
    CWT_CUDA(plan, cudaMemcpyAsync(plan->h_sig, signal_host, sig_bytes, cudaMemcpyHostToDevice, s));
    // rows of W are copied out as the launches that finish them complete
    // (host_copy_rows), overlapping the copy with the rest of the transform
    auto& h = plan->hc;
    h.on = true;
    h.dst = (char*)W_host;
    h.src = (const char*)plan->h_W;
    h.row_bytes = (size_t)plan->N * we;
    h.done.assign((size_t)plan->S, 0);
    h.nev = 1;
    st = run(plan, plan->h_sig, plan->h_W, spectrum_host ? plan->h_spec : nullptr, s);
    h.on = false;
    if (h.nev > 1) {
        CWT_CUDA(plan, cudaEventRecord(plan->hc_ev[0], plan->hc_stream));
        CWT_CUDA(plan, cudaStreamWaitEvent(s, plan->hc_ev[0], 0));
    }
    if (st != CWT_OK) {
        cudaStreamSynchronize(s);
        return st;
    }
    // rows no launch reported (sub-plans, a plan whose rows all come from its
    // child): copied after the whole transform, runs of rows at a time
    for (int32_t r = 0; r < plan->S;) {
        if (h.done[r]) {
            r++;
            continue;
        }
        int32_t e = r + 1;
        while (e < plan->S && !h.done[e]) e++;
        CWT_CUDA(plan, cudaMemcpyAsync((char*)W_host + (size_t)r * h.row_bytes, (const char*)plan->h_W +
                                       (size_t)r * h.row_bytes, (size_t)(e - r) * h.row_bytes,
                                       cudaMemcpyDeviceToHost, s));
        r = e;
    }
    if (spectrum_host)
        CWT_CUDA(plan, cudaMemcpyAsync(spectrum_host, plan->h_spec, (size_t)plan->S * sizeof(double),
                                       cudaMemcpyDeviceToHost, s));
    CWT_CUDA(plan, cudaStreamSynchronize(s));
    return CWT_OK;
}

cwt_status cwt_scales_paper_grid(int64_t N, int32_t wavelet, double omega0, int32_t n_subs, double* w_tilde_out,
                                 int32_t* n_out) {
    if (N < 2 || n_subs < 1 || !n_out) return CWT_ERR_INVALID_ARG;
    double cw;
    if (wavelet == CWT_WAVELET_GDW) cw = 2.0 / std::sqrt(5.0);
    else if (wavelet == CWT_WAVELET_CBSW) cw = 0.466094761079290;     // Table 2, footnote b
    else if (wavelet == CWT_WAVELET_CWGDW) cw = 0.428218886729052;    // Table 2, footnote c
    else if (wavelet == CWT_WAVELET_MORLET) {
        if (!(omega0 > 0.0)) return CWT_ERR_INVALID_ARG;
        cw = 2.0 / (omega0 + std::sqrt(omega0 * omega0 + 2.0));
    } else return CWT_ERR_INVALID_ARG;
    int n_levs = (int)std::lround(std::log2((double)N));
    *n_out = n_levs * n_subs;
    if (w_tilde_out) {
        double wmin = cw * kPi / (double)N;
        for (int i = 0; i < n_levs; i++)
            for (int j = 0; j < n_subs; j++)
                w_tilde_out[i * n_subs + j] = wmin * std::pow(2.0, i + (double)j / n_subs);
    }
    return CWT_OK;
}

cwt_status cwt_plan_set_timing(cwt_plan* plan, int32_t enable) {
    if (!plan) return CWT_ERR_INVALID_ARG;
    if (!plan->pending.empty()) cudaDeviceSynchronize();
    release_events(plan);
    if (enable < 0 || enable > 2) return CWT_ERR_INVALID_ARG;
    plan->timing = enable;
    if (plan->child) cwt_plan_set_timing(plan->child, enable);
    for (cwt_plan* q : plan->subs) cwt_plan_set_timing(q, enable);
    for (int c = 0; c < CWT_KCLASS_COUNT; c++) {
        plan->t_ms[c] = 0.0;
        plan->t_launches[c] = 0;
        plan->t_bytes[c] = 0.0;
    }
    return CWT_OK;
}

cwt_status cwt_plan_get_timing(cwt_plan* plan, int32_t cls, double* total_ms, int64_t* launches,
                               double* algorithmic_bytes) {
    if (!plan || cls < 0 || cls >= CWT_KCLASS_COUNT) return CWT_ERR_INVALID_ARG;
    for (auto& r : plan->pending) {
        CWT_CUDA(plan, cudaEventSynchronize(r.b));
        float ms = 0.f;
        CWT_CUDA(plan, cudaEventElapsedTime(&ms, r.a, r.b));
        plan->t_ms[r.cls] += ms;
        plan->t_launches[r.cls] += 1;
        plan->t_bytes[r.cls] += r.bytes;
    }
    release_events(plan);
    double cm = 0.0, cb = 0.0;
    int64_t cn = 0;
    std::vector<cwt_plan*> kids(plan->subs);
    if (plan->child) kids.push_back(plan->child);
    for (cwt_plan* q : kids) {
        double m = 0.0, b = 0.0;
        int64_t n = 0;
        cwt_status st = cwt_plan_get_timing(q, cls, &m, &n, &b);
        if (st != CWT_OK) return st;
        cm += m;
        cn += n;
        cb += b;
    }
    if (total_ms) *total_ms = plan->t_ms[cls] + cm;
    if (launches) *launches = plan->t_launches[cls] + cn;
    if (algorithmic_bytes) *algorithmic_bytes = plan->t_bytes[cls] + cb;
    return CWT_OK;
}

cwt_status cwt_batch_create(cwt_batch** batch, cwt_plan* const* plans, const void* const* signals_dev,
                            void* const* W_dev, double* const* spectra_dev, int32_t n, int32_t n_streams) {
    if (!batch) return CWT_ERR_INVALID_ARG;
    *batch = nullptr;
    if (!plans || !signals_dev || !W_dev || n < 1 || n_streams < 1 || n_streams > kBatchMaxStreams)
        return CWT_ERR_INVALID_ARG;
    std::set<const cwt_plan*> seen;
    for (int32_t i = 0; i < n; i++) {
        cwt_plan* p = plans[i];
        if (!p || !seen.insert(p).second) return CWT_ERR_INVALID_ARG;      // each plan once: its workspace is its own
        cwt_status st = check_exec_args(p, signals_dev[i], W_dev[i]);
        if (st != CWT_OK) return st;
        double* sp = spectra_dev ? spectra_dev[i] : nullptr;
        if (sp && !aligned(sp, 8)) return fail(p, CWT_ERR_INVALID_ARG, "bad spectrum pointer");
        if (p->timing) return fail(p, CWT_ERR_INVALID_ARG, "timing is on: a batch records the plan's launches");
        if (p->opts.scratch == CWT_SCRATCH_CALLER)
            return fail(p, CWT_ERR_INVALID_ARG, "a plan with caller scratch cannot join a batch");
    }
    // 1. record every plan's launch sequence with its dependency levels; the
    //    plan's own pointer stands for the call's stream (never passed to CUDA)
    Recorder rec;
    for (int32_t i = 0; i < n; i++) {
        cwt_plan* p = plans[i];
        rec.stream_level.clear();
        rec.event_level.clear();
        set_rec(p, &rec);
        cwt_status st = run_launches(p, signals_dev[i], W_dev[i], spectra_dev ? spectra_dev[i] : nullptr,
                                     (cudaStream_t)(void*)p);
        set_rec(p, nullptr);
        if (st != CWT_OK) return st;
    }
    // 2. group by (level, grouped kernel)
    std::map<std::pair<int, const void*>, std::vector<int>> by;
    for (int i = 0; i < (int)rec.launches.size(); i++) {
        const RecLaunch& r = rec.launches[i];
        if ((int64_t)r.grid.x * r.grid.y * r.grid.z == 0) continue;
        by[{r.level, r.gfn}].push_back(i);
    }
    cwt_batch* b = new (std::nothrow) cwt_batch();
    if (!b) return CWT_ERR_OOM;
    b->device = plans[0]->device;
    b->n_streams = n_streams;
    b->recorded = (int64_t)rec.launches.size();
    std::vector<unsigned char> host;
    auto take = [&](size_t bytes) {
        const size_t off = align16(host.size());
        host.resize(off + bytes, 0);
        return off;
    };
    for (const auto& kv : by) {
        const std::vector<int>& idx = kv.second;
        const RecLaunch& r0 = rec.launches[idx[0]];
        cwt_batch::Group g{};
        g.gfn = r0.gfn;
        g.block = r0.block;
        g.level = r0.level;
        g.stride = (int32_t)align16(r0.arg.size() * 4);
        g.smem = 0;
        for (int i : idx) {
            const RecLaunch& r = rec.launches[i];
            if (r.arg.size() != r0.arg.size() || r.block.x != r0.block.x || r.block.y != r0.block.y ||
                r.block.z != r0.block.z || r.grid.z != 1) {
                free_batch(b);
                return fail(plans[0], CWT_ERR_INTERNAL, "inconsistent launches of one kernel");
            }
            g.smem = std::max(g.smem, r.smem);
            g.ctas += (int64_t)r.grid.x * r.grid.y;
        }
        if (g.ctas > INT32_MAX) {
            free_batch(b);
            return fail(plans[0], CWT_ERR_UNSUPPORTED, "batch too large for one grouped launch");
        }
        g.args_off = take((size_t)g.stride * idx.size());
        g.geom_off = take(sizeof(int2) * idx.size());
        g.sub_off = take(sizeof(int32_t) * (size_t)g.ctas);
        int32_t first = 0;
        for (size_t k = 0; k < idx.size(); k++) {
            const RecLaunch& r = rec.launches[idx[k]];
            std::memcpy(host.data() + g.args_off + k * g.stride, r.arg.data(), r.arg.size() * 4);
            const int2 geo = make_int2(first, (int)r.grid.x);
            std::memcpy(host.data() + g.geom_off + k * sizeof(int2), &geo, sizeof(int2));
            int32_t* sub = (int32_t*)(host.data() + g.sub_off);
            const int32_t cnt = (int32_t)(r.grid.x * r.grid.y);
            for (int32_t c = 0; c < cnt; c++) sub[first + c] = (int32_t)k;
            first += cnt;
        }
        b->ctas += g.ctas;
        b->groups.push_back(g);
    }
    // level index (std::map orders the groups by level)
    const int nlev = b->groups.empty() ? 0 : b->groups.back().level + 1;
    b->level_first.assign(nlev + 1, (int)b->groups.size());
    for (int gi = (int)b->groups.size() - 1; gi >= 0; gi--) b->level_first[b->groups[gi].level] = gi;
    for (int l = nlev - 1; l >= 0; l--) b->level_first[l] = std::min(b->level_first[l], b->level_first[l + 1]);
    // 3. device tables, streams, shared-memory opt-in of the grouped kernels
    cudaError_t e = cudaMalloc(&b->d_buf, std::max<size_t>(host.size(), 16));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_buf, host.data(), host.size(), cudaMemcpyHostToDevice);
    for (int i = 1; i < n_streams && e == cudaSuccess; i++) {
        e = cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess && n_streams > 1) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        free_batch(b);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CWT_ERR_OOM : fail(plans[0], CWT_ERR_CUDA, cudaGetErrorString(e));
    }
    for (const auto& g : b->groups) {
        cwt_status st = opt_in_smem(plans[0], g.gfn);
        if (st != CWT_OK) {
            free_batch(b);
            return st;
        }
    }
    *batch = b;
    return CWT_OK;
}

cwt_status cwt_batch_exec(cwt_batch* b, void* stream) {
    if (!b) return CWT_ERR_INVALID_ARG;
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d != b->device) return CWT_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int nlev = (int)b->level_first.size() - 1;
    for (int l = 0; l < nlev; l++) {
        const int g0 = b->level_first[l], g1 = b->level_first[l + 1];
        const int k = std::min(b->n_streams, g1 - g0);
        if (k > 1) {
            if (cudaEventRecord(b->ev_fork, s) != cudaSuccess) return CWT_ERR_CUDA;
            for (int j = 1; j < k; j++)
                if (cudaStreamWaitEvent(b->side[j], b->ev_fork, 0) != cudaSuccess) return CWT_ERR_CUDA;
        }
        for (int gi = g0; gi < g1; gi++) {
            const cwt_batch::Group& g = b->groups[gi];
            GroupMap gm{b->d_buf + g.args_off, (const int32_t*)(b->d_buf + g.sub_off),
                        (const int2*)(b->d_buf + g.geom_off), g.stride};
            void* args[] = {&gm};
            const int j = (gi - g0) % k;
            if (cudaLaunchKernel(g.gfn, dim3((unsigned)g.ctas), g.block, args, g.smem, j ? b->side[j] : s) !=
                cudaSuccess)
                return CWT_ERR_CUDA;
        }
        for (int j = 1; j < k; j++) {
            if (cudaEventRecord(b->ev_join[j], b->side[j]) != cudaSuccess) return CWT_ERR_CUDA;
            if (cudaStreamWaitEvent(s, b->ev_join[j], 0) != cudaSuccess) return CWT_ERR_CUDA;
        }
    }
    return CWT_OK;
}

cwt_status cwt_batch_info(const cwt_batch* b, int32_t* n_levels, int32_t* n_launches, int64_t* n_ctas,
                          int64_t* n_recorded) {
    if (!b) return CWT_ERR_INVALID_ARG;
    if (n_levels) *n_levels = (int32_t)b->level_first.size() - 1;
    if (n_launches) *n_launches = (int32_t)b->groups.size();
    if (n_ctas) *n_ctas = b->ctas;
    if (n_recorded) *n_recorded = b->recorded;
    return CWT_OK;
}

cwt_status cwt_batch_destroy(cwt_batch* b) {
    if (b) cudaDeviceSynchronize();
    free_batch(b);
    return CWT_OK;
}

cwt_status cwt_plan_get_opts(const cwt_plan* plan, cwt_plan_opts* opts) {
    if (!plan || !opts) return CWT_ERR_INVALID_ARG;
    *opts = plan->opts;
    return CWT_OK;
}

const char* cwt_status_string(cwt_status s) {
    switch (s) {
    case CWT_OK: return "ok";
    case CWT_ERR_INVALID_ARG: return "invalid argument";
    case CWT_ERR_UNSUPPORTED: return "unsupported configuration";
    case CWT_ERR_OOM: return "out of memory";
    case CWT_ERR_CUDA: return "CUDA error";
    case CWT_ERR_TIMEOUT: return "device wait timed out";
    case CWT_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char* cwt_plan_last_error(const cwt_plan* plan) {
    return plan ? plan->err.c_str() : "null plan";
}

}  // extern "C"
