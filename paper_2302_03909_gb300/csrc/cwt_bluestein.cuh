// Periodic boundary for any length N: the N-point DFTs of Eqs. 8-9 by
// Bluestein's chirp transform on power-of-two FFTs of length P >= 2N - 1.
//
// With c_j = e^{i pi j^2 / N} and m n = (m^2 + n^2 - (m - n)^2) / 2,
//   sum_n x_n e^{+2 pi i m n / N} = c_m  sum_n (x_n c_n) conj(c_{m-n}),
//   sum_m z_m e^{-2 pi i m n / N} = conj(c_n) sum_m (z_m conj(c_m)) c_{n-m},
// linear convolutions with a chirp that a cyclic convolution of length P
// computes exactly for output indices < N.  A cyclic convolution is
//   a (*) g = (1/P) conj(D(conj(D(a) D(g))))
// with D the e^{-} DFT of length P (the library's forward kernels).
//
// Per call:
//   conv1 = (f c) (*) conj(c)              F_hat(m) = c_m conv1(m) (times dx)
// and per job (a Morlet scale, or two real-wavelet scales as Z_a + i Z_b):
//   a2(m) = Z(m) conj(c_m) = psi-product(m) conv1(m)   (the chirps cancel)
//   W(n)  = conj(c_n) (a2 (*) c)(n)
// where the psi-product carries amp psi_hat(alpha m~) with alpha = 2 pi / (N w~),
// m~ the signed frequency of bin m (the N-point grid of Eq. 10) and the 1/N of
// the inverse transform.  D(g) of both chirp sequences is computed once, at
// plan creation.
#pragma once
#include "cwt_kernels.cuh"

namespace cwtk {

constexpr int kBsThreads = 256;
constexpr int kBsOutPer = 8;                        // outputs per thread of the output kernel
constexpr int kBsOutBlock = kBsThreads * kBsOutPer; // outputs per block (one power partial per row)

struct BsArgs {
    const void* signal;      // signal stage: N samples (f32 or f64)
    const float2* chirp;     // c_j, j < N
    const float2* src;       // P values: conv stage output (conj of D, not yet divided by P)
    float2* dst;             // P values
    void* W;                 // output rows [S][N]
    double* partials;        // power partials of the output rows
    Job J;                   // scale stage / output: the job
    int64_t N;
    int32_t P, sig_f64, wavelet, do_power;
    float half_w0sq, corr_v2, inv_p;
    int32_t conj_c;          // chirp sequence: conj(c) instead of c
};

// signed frequency of bin m of the N-point grid (m <= N/2: m, else m - N)
__device__ __forceinline__ int bs_signed(int64_t m, int64_t N) { return (int)(2 * m <= N ? m : m - N); }

// dst(j) = g_P(j): c_{|j|} (or its conjugate) for j < N and for P - j < N, 0 between
__device__ __forceinline__ void bs_seq_body(const BsArgs& a, const Cta c) {
    for (int64_t j = (int64_t)c.x * kBsThreads + threadIdx.x; j < a.P; j += (int64_t)c.nx * kBsThreads) {
        const int64_t k = j < a.N ? j : (a.P - j < a.N ? a.P - j : -1);
        float2 v = make_float2(0.f, 0.f);
        if (k >= 0) {
            v = __ldg(&a.chirp[k]);
            if (a.conj_c) v.y = -v.y;
        }
        a.dst[j] = v;
    }
}

// dst(n) = f(n) c_n for n < N, 0 up to P
__device__ __forceinline__ void bs_sig_body(const BsArgs& a, const Cta c) {
    for (int64_t n = (int64_t)c.x * kBsThreads + threadIdx.x; n < a.P; n += (int64_t)c.nx * kBsThreads) {
        float2 v = make_float2(0.f, 0.f);
        if (n < a.N) {
            const float f = a.sig_f64 ? (float)__ldg(&((const double*)a.signal)[n]) : __ldg(&((const float*)a.signal)[n]);
            const float2 ch = __ldg(&a.chirp[n]);
            v = make_float2(f * ch.x, f * ch.y);
        }
        a.dst[n] = v;
    }
}

// dst(m) = conv1(m) (amp_a psi_a + i amp_b psi_b)(m~) for m < N, 0 up to P;
// conv1 = src / P
__device__ __forceinline__ void bs_scale_body(const BsArgs& a, const Cta c) {
    const bool real = wav_real(a.wavelet);
    for (int64_t m = (int64_t)c.x * kBsThreads + threadIdx.x; m < a.P; m += (int64_t)c.nx * kBsThreads) {
        float2 v = make_float2(0.f, 0.f);
        if (m < a.N) {
            const int k = bs_signed(m, a.N);
            float2 f = __ldg(&a.src[m]);
            f = make_float2(f.x * a.inv_p, f.y * a.inv_p);
            const float g0 = psi_gen(a.J.g[0], a.wavelet, a.half_w0sq, a.corr_v2, k);
            if (real) {
                const float g1 = a.J.g[1].row >= 0 ? psi_gen(a.J.g[1], a.wavelet, a.half_w0sq, a.corr_v2, k) : 0.f;
                v = make_float2(fmaf(f.x, g0, -f.y * g1), fmaf(f.x, g1, f.y * g0));
            } else {
                v = make_float2(f.x * g0, f.y * g0);
            }
        }
        a.dst[m] = v;
    }
}

// W rows of the job: val(n) = conj(c_n) src(n) / P for n < N (Morlet: the
// complex row; real wavelets: re -> row a, im -> row b), and one power partial
// per block and row: block b covers n in [b kBsOutBlock, (b + 1) kBsOutBlock)
__device__ __forceinline__ void bs_out_body(const BsArgs& a, const Cta c) {
    __shared__ double red[2 * (kBsThreads / 32)];
    const bool real = wav_real(a.wavelet);
    const int ra = a.J.g[0].row, rb = a.J.g[1].row;
    float pw0 = 0.f, pw1 = 0.f;
#pragma unroll
    for (int i = 0; i < kBsOutPer; i++) {
        const int64_t n = (int64_t)c.x * kBsOutBlock + i * kBsThreads + threadIdx.x;
        if (n < a.N) {
            const float2 s = __ldg(&a.src[n]);
            const float2 ch = __ldg(&a.chirp[n]);
            const float2 v = make_float2((ch.x * s.x + ch.y * s.y) * a.inv_p, (ch.x * s.y - ch.y * s.x) * a.inv_p);
            if (real) {
                __stcs((float*)a.W + (int64_t)ra * a.N + n, v.x);
                pw0 = fmaf(v.x, v.x, pw0);
                if (rb >= 0) {
                    __stcs((float*)a.W + (int64_t)rb * a.N + n, v.y);
                    pw1 = fmaf(v.y, v.y, pw1);
                }
            } else {
                __stcs((float2*)a.W + (int64_t)ra * a.N + n, v);
                pw0 = fmaf(v.x, v.x, fmaf(v.y, v.y, pw0));
            }
        }
    }
    if (!a.do_power) return;
    double s0, s1;
    block_sum2<kBsThreads>(pw0, pw1, &s0, &s1, red);
    if (threadIdx.x == 0) {
        a.partials[a.J.g[0].part_off + c.x] = s0;
        if (real && rb >= 0) a.partials[a.J.g[1].part_off + c.x] = s1;
    }
}

#define CWT_BS_KERNELS(name)                                                                            \
    static __global__ void __launch_bounds__(kBsThreads) k_bs_##name(BsArgs a) { bs_##name##_body(a, cta_plain()); } \
    static __global__ void __launch_bounds__(kBsThreads) k_bs_##name##_g(GroupMap g) {                 \
        Cta c;                                                                                          \
        const BsArgs& a = group_args<BsArgs>(g, c);                                                     \
        bs_##name##_body(a, c);                                                                         \
    }
CWT_BS_KERNELS(seq)
CWT_BS_KERNELS(sig)
CWT_BS_KERNELS(scale)
CWT_BS_KERNELS(out)
#undef CWT_BS_KERNELS

}  // namespace cwtk
