// Device code of the GB300 FFTCWT (Wang & He, arXiv:2302.03909, Sec. 3.1).
//
// The transform of one scale is an inverse DFT of length M of the product
// Z(k) = F(k) psi_hat(alpha k) amp over the signed frequency k (Eqs. 9-10).
// psi_hat is negligible outside a band [k_lo, k_lo + K) of the scale, so each
// inverse DFT is evaluated as a band-pruned Cooley-Tukey factorisation
// M = A * B with output index n = d + A c (d < A, c < B):
//
//   X(d + A c) = sum_{b<B} e^{-2 pi i b c / B} Y(b, d),
//   Y(b, d)    = sum_{k in band, k = b mod B} Z(k) e^{-2 pi i k d / M}.
//
// When K <= r B the inner sum has at most r terms and is evaluated directly
// while the shared-memory tile is filled (single-pass kernel).  Wider bands
// use a second factorisation (pass 1: A-point DFTs over the columns b, with
// the e^{-2 pi i b d / M} twiddle; pass 2: B-point DFTs over b).  All DFTs
// run in shared memory as Stockham radix-2/4/8 stages.
//
// Real wavelets (GDW): two scales share one complex transform,
// Z = Z_a + i Z_b with Z_a, Z_b Hermitian, so Re X = W_a and Im X = W_b.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cwtk {

constexpr int kLmaxLog = 13;              // largest DFT held by one CTA
constexpr int kLmax = 1 << kLmaxLog;
constexpr int kTileElems = 8192;          // complex elements per CTA tile

enum { WAV_GDW = 0, WAV_MORLET = 1 };
enum { SRC_BAND = 0, SRC_Y = 1, SRC_SIGNAL = 2 };
enum { SINK_W = 0, SINK_FWD = 1 };
enum { P1_BAND = 0, P1_SIGNAL = 1 };

// Per-scale generator of amp * psi_hat(alpha k) in FP32 from FP64-derived constants.
struct ScaleGen {
    float a_hi, a_lo;   // alpha = 2 pi / (M w~), split so a_hi + a_lo is exact to ~2^-48
    float amp;          // sqrt(dx / w~) / M * (8 sqrt(pi) C_N  |  sqrt(2 pi) C_N)
    float k0_frac;      // Morlet: omega0 / alpha = k0_int + k0_frac
    int32_t k0_int;
    int32_t row;        // output row of W, -1 if this half of the job is unused
    int32_t part_off;   // offset of this row's power partial sums
    int32_t pad_;
};

// One complex inverse transform: a Morlet scale, or a pair of GDW scales.
struct Job {
    ScaleGen g[2];
    int32_t k_lo;       // signed lowest bin of the band
    int32_t K;          // band width in bins (1..M)
    int32_t r;          // direct depth of the single-pass kernel
    int32_t tile0;      // first tile of this job within its launch
};

struct Params {
    const float2* Fp;        // F(m) = sum_n f(n) e^{+2 pi i m n / M}, m in [0, M/2]
    float2* Fp_out;          // forward pass sink
    float2* Y;               // pass-1 -> pass-2 intermediate [B][A]
    const void* signal;      // N samples, f32 or f64
    void* W;                 // [S][N] f32 (GDW) or complex64 (Morlet)
    double* partials;        // power partial sums
    const float2* tw_lo;     // e^{-2 pi i j / M}, low  h bits
    const float2* tw_hi;     // e^{-2 pi i j / M}, high bits
    const float2* tw_L;      // e^{-2 pi i j / kLmax}
    int64_t N;
    int32_t M, logM, h;      // M = 2^logM, two-level table split h
    int32_t A;               // number of columns d (= M / B)
    int32_t T_eff;           // columns per tile (<= template T)
    int32_t job;             // job index for single-job launches
    int32_t wavelet;
    int32_t sig_f64;
    int32_t do_power;
    float half_w0sq;         // omega0^2 / 2
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by -i
__device__ __forceinline__ float2 cmi(float2 a) { return make_float2(a.y, -a.x); }

// e^{-2 pi i j / M}, j in [0, M)
__device__ __forceinline__ float2 tw_m(const Params& p, uint32_t j) {
    float2 hi = __ldg(&p.tw_hi[j >> p.h]);
    float2 lo = __ldg(&p.tw_lo[j & ((1u << p.h) - 1u)]);
    return cmul(hi, lo);
}

// amp * psi_hat(alpha k) for the signed bin k (Table 2 spectra)
__device__ __forceinline__ float psi_gen(const ScaleGen& g, int wavelet, float half_w0sq, int k) {
    float kf = (float)k;
    float v = fmaf(g.a_hi, kf, g.a_lo * kf);
    if (wavelet == WAV_GDW) {
        float v2 = v * v;
        return g.amp * v2 * expf(-v2);
    }
    float d = (float)(k - g.k0_int) - g.k0_frac;           // k - omega0/alpha, exact integer part
    float t = fmaf(g.a_hi, d, g.a_lo * d);                 // alpha k - omega0
    return g.amp * (expf(-0.5f * t * t) - expf(fmaf(-0.5f * v, v, -half_w0sq)));
}

// F at the signed bin k: F(-k) = conj F(k) for a real signal
__device__ __forceinline__ float2 spec_at(const float2* __restrict__ Fp, int k) {
    if (k >= 0) return __ldg(&Fp[k]);
    float2 f = __ldg(&Fp[-k]);
    return make_float2(f.x, -f.y);
}

// Z(k) of a job (the pointwise product of Eq. 10, scaled)
__device__ __forceinline__ float2 band_value(const Params& p, const Job& J, int k) {
    float2 f = spec_at(p.Fp, k);
    float g0 = psi_gen(J.g[0], p.wavelet, p.half_w0sq, k);
    if (p.wavelet == WAV_GDW) {
        float g1 = J.g[1].row >= 0 ? psi_gen(J.g[1], p.wavelet, p.half_w0sq, k) : 0.f;
        return make_float2(fmaf(f.x, g0, -f.y * g1), fmaf(f.x, g1, f.y * g0));
    }
    return make_float2(f.x * g0, f.y * g0);
}

__device__ __forceinline__ float load_signal(const Params& p, int64_t n) {
    if (n >= p.N) return 0.f;
    return p.sig_f64 ? (float)__ldg(&((const double*)p.signal)[n]) : __ldg(&((const float*)p.signal)[n]);
}

// ------------------------------------------------------- radix-R DFTs (sign -)

template <int R> __device__ __forceinline__ void dft(float2* v);

template <> __device__ __forceinline__ void dft<2>(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}

template <> __device__ __forceinline__ void dft<4>(float2* v) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d13 = cmi(csub(v[1], v[3]));
    v[0] = cadd(s02, s13); v[2] = csub(s02, s13);
    v[1] = cadd(d02, d13); v[3] = csub(d02, d13);
}

template <> __device__ __forceinline__ void dft<8>(float2* v) {
    const float r = 0.70710678118654752440f;
    float2 e[4] = {v[0], v[2], v[4], v[6]};
    float2 o[4] = {v[1], v[3], v[5], v[7]};
    dft<4>(e);
    dft<4>(o);
    // o[q] *= e^{-2 pi i q / 8}
    o[1] = make_float2(r * (o[1].x + o[1].y), r * (o[1].y - o[1].x));
    o[2] = cmi(o[2]);
    o[3] = make_float2(r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y));
#pragma unroll
    for (int q = 0; q < 4; q++) {
        v[q] = cadd(e[q], o[q]);
        v[q + 4] = csub(e[q], o[q]);
    }
}

// ------------------------------------------------------- shared-memory FFT

// T columns of an L-point DFT in shared memory.  TFAST: element (l, t) at
// l * (T + PAD) + t and threads walk t fastest; otherwise at t * (L + PAD) + l
// and threads walk l fastest.  Columns t >= T_eff are left untouched.
template <int LOGL, int T, int NT, bool TFAST, int PAD>
struct SmemFFT {
    static constexpr int L = 1 << LOGL;

    __device__ static __forceinline__ int addr(int l, int t) {
        return TFAST ? l * (T + PAD) + t : t * (L + PAD) + l;
    }

    template <int LOGR, int LOGNS>
    __device__ static __forceinline__ void stage(float2* buf, int T_eff, const float2* __restrict__ twL) {
        constexpr int R = 1 << LOGR;
        constexpr int NB = (L / R) * T;                   // butterflies per stage
        constexpr int BPT = (NB + NT - 1) / NT;           // per thread
        constexpr int NS = 1 << LOGNS;
        float2 v[BPT][R];
        int jj[BPT], tt[BPT];
#pragma unroll
        for (int q = 0; q < BPT; q++) {
            int idx = threadIdx.x + q * NT;
            int j, t;
            if (TFAST) { t = idx % T; j = idx / T; }
            else { j = idx % (L / R); t = idx / (L / R); }
            jj[q] = j; tt[q] = t;
            if (idx < NB && t < T_eff) {
#pragma unroll
                for (int r = 0; r < R; r++) v[q][r] = buf[addr(j + r * (L / R), t)];
                if (LOGNS > 0) {
                    int k = j & (NS - 1);
#pragma unroll
                    for (int r = 1; r < R; r++) {
                        int ti = (r * k) << (kLmaxLog - LOGNS - LOGR);
                        v[q][r] = cmul(v[q][r], __ldg(&twL[ti]));
                    }
                }
                dft<R>(v[q]);
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < BPT; q++) {
            int idx = threadIdx.x + q * NT;
            int j = jj[q], t = tt[q];
            if (idx < NB && t < T_eff) {
                int k = j & (NS - 1);
                int base = (j - k) * R + k;
#pragma unroll
                for (int r = 0; r < R; r++) buf[addr(base + r * NS, t)] = v[q][r];
            }
        }
        __syncthreads();
    }

    template <int LOGNS>
    __device__ static __forceinline__ void stages(float2* buf, int T_eff, const float2* __restrict__ twL) {
        if constexpr (LOGNS < LOGL) {
            constexpr int LOGR = (LOGNS == 0 && (LOGL % 3) != 0) ? (LOGL % 3) : 3;
            stage<LOGR, LOGNS>(buf, T_eff, twL);
            stages<LOGNS + LOGR>(buf, T_eff, twL);
        }
    }

    // in: natural order; out: natural order (Stockham autosort). Caller syncs before.
    __device__ static __forceinline__ void run(float2* buf, int T_eff, const float2* __restrict__ twL) {
        stages<0>(buf, T_eff, twL);
    }
};

// ------------------------------------------------------------ block reduce

template <int NT>
__device__ __forceinline__ void block_sum2(float a, float b, double* out_a, double* out_b, double* red) {
    double da = a, db = b;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        da += __shfl_xor_sync(0xffffffffu, da, o);
        db += __shfl_xor_sync(0xffffffffu, db, o);
    }
    constexpr int NW = (NT + 31) / 32;
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[w] = da; red[NW + w] = db; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int i = 0; i < NW; i++) { sa += red[i]; sb += red[NW + i]; }
        *out_a = sa; *out_b = sb;
    }
}

// ------------------------------------------------------------ final pass

// Tile = T_eff consecutive columns d of one job; computes the B-point DFTs
// over b and writes X(d + A c) for c < B.
template <int LOGB, int T, int NT, int SRC, int SINK>
__global__ void __launch_bounds__(NT) k_final(Params p, const Job* __restrict__ jobs,
                                              const int32_t* __restrict__ tile_job) {
    constexpr int B = 1 << LOGB;
    constexpr int PAD = (T < 16 && T > 1) ? 1 : 0;
    using FFT = SmemFFT<LOGB, T, NT, true, PAD>;
    extern __shared__ float2 smem[];
    float2* X = smem;
    float2* Zs = smem + B * (T + PAD);
    __shared__ double red[2 * ((NT + 31) / 32)];

    const int tile = blockIdx.x;
    const int T_eff = p.T_eff;
    Job J;
    int d0 = 0;
    if (SRC == SRC_BAND || SINK == SINK_W) {
        int ji = tile_job ? __ldg(&tile_job[tile]) : p.job;
        J = jobs[ji];
        d0 = (tile - J.tile0) * T_eff;
    } else {
        d0 = tile * T_eff;
    }

    if (SRC == SRC_BAND) {
        for (int i = threadIdx.x; i < J.K; i += NT) Zs[i] = band_value(p, J, J.k_lo + i);
        __syncthreads();
        const int kend = J.k_lo + J.K;
        for (int e = threadIdx.x; e < B * T; e += NT) {
            int t = e % T, b = e / T;
            if (t >= T_eff) continue;
            uint32_t d = (uint32_t)(d0 + t);
            int first = J.k_lo + (((b - J.k_lo) % B) + B) % B;
            float2 acc = make_float2(0.f, 0.f);
            for (int k = first; k < kend; k += B) {
                uint32_t j = ((uint32_t)k * d) & (uint32_t)(p.M - 1);
                float2 z = Zs[k - J.k_lo];
                float2 w = tw_m(p, j);
                acc = cadd(acc, cmul(z, w));
            }
            X[FFT::addr(b, t)] = acc;
        }
    } else if (SRC == SRC_Y) {
        for (int e = threadIdx.x; e < B * T; e += NT) {
            int t = e % T, b = e / T;
            if (t >= T_eff) continue;
            X[FFT::addr(b, t)] = p.Y[(int64_t)b * p.A + d0 + t];
        }
    } else {  // SRC_SIGNAL: whole transform in one tile (A = 1, T_eff = 1)
        for (int b = threadIdx.x; b < B; b += NT) X[FFT::addr(b, 0)] = make_float2(load_signal(p, b), 0.f);
    }
    __syncthreads();
    FFT::run(X, T_eff, p.tw_L);

    if (SINK == SINK_FWD) {
        const int half = p.M >> 1;
        for (int e = threadIdx.x; e < B * T; e += NT) {
            int t = e % T, c = e / T;
            if (t >= T_eff) continue;
            int n = d0 + t + p.A * c;
            if (n <= half) {
                float2 v = X[FFT::addr(c, t)];
                p.Fp_out[n] = make_float2(v.x, -v.y);
            }
        }
        return;
    }

    // SINK_W: crop to n < N, store, accumulate |W|^2
    float pw0 = 0.f, pw1 = 0.f;
    const bool two = (p.wavelet == WAV_GDW) && (J.g[1].row >= 0);
    float* Wr0 = (float*)p.W + (int64_t)J.g[0].row * p.N;
    float* Wr1 = two ? (float*)p.W + (int64_t)J.g[1].row * p.N : nullptr;
    float2* Wc = (float2*)p.W + (int64_t)J.g[0].row * p.N;
    for (int e = threadIdx.x; e < B * T; e += NT) {
        int t = e % T, c = e / T;
        if (t >= T_eff) continue;
        int64_t n = (int64_t)d0 + t + (int64_t)p.A * c;
        if (n >= p.N) continue;
        float2 v = X[FFT::addr(c, t)];
        if (p.wavelet == WAV_GDW) {
            Wr0[n] = v.x;
            pw0 = fmaf(v.x, v.x, pw0);
            if (two) { Wr1[n] = v.y; pw1 = fmaf(v.y, v.y, pw1); }
        } else {
            Wc[n] = v;
            pw0 = fmaf(v.x, v.x, fmaf(v.y, v.y, pw0));
        }
    }
    if (p.do_power) {
        double s0, s1;
        block_sum2<NT>(pw0, pw1, &s0, &s1, red);
        if (threadIdx.x == 0) {
            int slot = tile - J.tile0;
            p.partials[J.g[0].part_off + slot] = s0;
            if (two) p.partials[J.g[1].part_off + slot] = s1;
        }
    }
}

// ------------------------------------------------------------ pass 1

// Tile = T1 consecutive columns b; A-point DFT over a of x(b + B a), then the
// twiddle e^{-2 pi i b d / M}; writes Y[b][d].
template <int LOGA, int T1, int NT, int MODE>
__global__ void __launch_bounds__(NT) k_pass1(Params p, const Job* __restrict__ jobs) {
    constexpr int A = 1 << LOGA;
    constexpr int PAD = 1;
    using FFT = SmemFFT<LOGA, T1, NT, false, PAD>;
    extern __shared__ float2 smem[];
    float2* X = smem;
    const int B = p.M >> LOGA;
    const int b0 = blockIdx.x * T1;
    const int half = p.M >> 1;
    Job J;
    if (MODE == P1_BAND) J = jobs[p.job];

    for (int e = threadIdx.x; e < A * T1; e += NT) {
        int t = e % T1, a = e / T1;
        int k = b0 + t + B * a;                 // unsigned bin in [0, M)
        float2 v = make_float2(0.f, 0.f);
        if (MODE == P1_BAND) {
            int ks = k <= half ? k : k - p.M;
            if (ks >= J.k_lo && ks < J.k_lo + J.K) v = band_value(p, J, ks);
        } else {
            v.x = load_signal(p, k);
        }
        X[FFT::addr(a, t)] = v;
    }
    __syncthreads();
    FFT::run(X, T1, p.tw_L);
    for (int e = threadIdx.x; e < A * T1; e += NT) {
        int d = e % A, t = e / A;
        uint32_t b = (uint32_t)(b0 + t);
        float2 v = cmul(X[FFT::addr(d, t)], tw_m(p, (b * (uint32_t)d) & (uint32_t)(p.M - 1)));
        p.Y[(int64_t)b * A + d] = v;
    }
}

// ------------------------------------------------------------ power

// spectrum[s] = (sum of the row's partials in fixed order) / N
static __global__ void k_power_finalize(const double* __restrict__ partials, const int32_t* __restrict__ off,
                                        const int32_t* __restrict__ cnt, int32_t S, int64_t N,
                                        double* __restrict__ spectrum) {
    int s = blockIdx.x;
    if (s >= S) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < cnt[s]; i += 32) acc += partials[off[s] + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) spectrum[s] = acc / (double)N;
}

// spectrum[s] = (sum_c partials[s * chunks + c] in fixed order) / N
static __global__ void k_power_finalize_uniform(const double* __restrict__ partials, int32_t chunks, int32_t S,
                                                int64_t N, double* __restrict__ spectrum) {
    int s = blockIdx.x;
    if (s >= S) return;
    double acc = 0.0;
    for (int i = threadIdx.x; i < chunks; i += 32) acc += partials[(int64_t)s * chunks + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) spectrum[s] = acc / (double)N;
}

// Partial sums of |W|^2 over chunks of each row: grid (chunks, S)
template <int NT>
__global__ void __launch_bounds__(NT) k_power_rows(const void* __restrict__ W, int64_t N, int is_complex,
                                                   int64_t chunk, double* __restrict__ partials) {
    __shared__ double red[2 * ((NT + 31) / 32)];
    int s = blockIdx.y, c = blockIdx.x;
    int64_t n0 = (int64_t)c * chunk, n1 = n0 + chunk < N ? n0 + chunk : N;
    float acc = 0.f;
    if (is_complex) {
        const float2* row = (const float2*)W + (int64_t)s * N;
        for (int64_t n = n0 + threadIdx.x; n < n1; n += NT) {
            float2 v = __ldg(&row[n]);
            acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
        }
    } else {
        const float* row = (const float*)W + (int64_t)s * N;
        for (int64_t n = n0 + threadIdx.x; n < n1; n += NT) {
            float v = __ldg(&row[n]);
            acc = fmaf(v, v, acc);
        }
    }
    double tot, unused;
    block_sum2<NT>(acc, 0.f, &tot, &unused, red);
    if (threadIdx.x == 0) partials[(int64_t)s * gridDim.x + c] = tot;
}

}  // namespace cwtk
