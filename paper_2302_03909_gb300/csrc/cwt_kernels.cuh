// Device code of the GB300 FFTCWT (Wang & He, arXiv:2302.03909, Sec. 3.1).
//
// The transform of one scale is an inverse DFT of length M of the product
// Z(k) = F(k) psi_hat(alpha k) amp over the signed frequency k (Eqs. 9-10).
// psi_hat is negligible outside a band [k_lo, k_lo + K) of the scale, so each
// inverse DFT is evaluated as a band-pruned Cooley-Tukey factorisation
// M = A * L with output index n = d + A c (d < A, c < L):
//
//   X(d + A c) = sum_{b<L} e^{-2 pi i b c / L} Y(b, d),
//   Y(b, d)    = sum_{k in band, k = b mod L} Z(k) e^{-2 pi i k d / M}.
//
// Band kernel (K <= L): one CTA tile = T consecutive columns d; Y(b, d) has a
// single term and is formed in registers while the first DFT stage is
// loaded.  Wide kernels (K > L): pass 1 runs the A-point DFTs over the
// columns b (x(b + L a) = Z(b + L a)) with the twiddle e^{-2 pi i b d / M}
// into an intermediate Y[b][d]; pass 2 runs the L-point DFTs over b.
//
// Every CTA-level DFT is a Stockham FFT of at most three stages, each stage a
// radix-2..32 DFT held in registers (constant twiddles folded by the
// compiler), with stage twiddles from FP64-generated tables and one shared-
// memory exchange between stages.  The first stage is filled straight from
// the source and the last stage writes straight to global memory.
//
// Real wavelets (GDW): two scales share one complex transform,
// Z = Z_a + i Z_b with Z_a, Z_b Hermitian, so Re X = W_a and Im X = W_b.
//
// Every kernel is a body taking its argument and its block coordinates (Cta),
// with two entry points: the plain kernel (one launch of one plan) and the
// grouped kernel "_g" (the launches of one kernel made by many plans, merged
// into one grid; see GroupMap).  Both run the same body, so they compute the
// same values bit for bit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cwtk {

constexpr int kLmaxLog = 13;              // largest DFT held by one CTA
constexpr int kLmax = 1 << kLmaxLog;

enum { WAV_GDW = 0, WAV_MORLET = 1, WAV_CBSW = 2, WAV_CWGDW = 3 };   // Table 2

// real, even wavelets give real rows; two scales share one complex transform
__host__ __device__ constexpr bool wav_real(int w) { return w != WAV_MORLET; }

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
    int32_t tile0;      // first tile of this job within its launch
    int32_t pad_;
};

struct Params {
    const float2* Fp;        // F(m) = sum_n f(n) e^{+2 pi i m n / M}, m in [0, M/2]
    const float2* Ft;        // wide pass 1: Ft[b A + a] = F(k), k = b + L a over all M unsigned bins
    float2* Fp_out;          // forward pass sink
    float2* Y;               // pass-1 -> pass-2 intermediate, [job][b][d]
    const void* signal;      // N samples, f32 or f64
    void* W;                 // [S][N] f32 (GDW) or complex64 (Morlet)
    double* partials;        // power partial sums
    const float2* tw_lo;     // e^{-2 pi i j / M}, low  h bits of j
    const float2* tw_hi;     // e^{-2 pi i j / M}, high bits of j
    const float2* tw_tab;    // tw_tab[L + i] = e^{-2 pi i i / L}, L = 2, 4, .., kLmax
    const Job* jobs;
    const int32_t* tile_job; // band launches: tile -> job
    int64_t N;
    int64_t out_off, out_len; // W rows keep outputs n in [out_off, out_off + out_len), row stride out_len
    int32_t M, h;            // M = 2^logM, two-level table split h
    int32_t A;               // number of columns d (= M / L)
    int32_t job0;            // wide launches: job = job0 + blockIdx.y
    int32_t D;               // tiles per CTA of the W-writing kernels
    int32_t wavelet;
    int32_t sig_f64;
    int32_t do_power;
    float half_w0sq;         // omega0^2 / 2
    float corr_v2;           // Morlet: the correction e^{-(v^2 + omega0^2)/2} is below the band
                             // truncation threshold for v^2 >= corr_v2
    int32_t yperm;           // wide pass 1: Y rows in the order of the tensor-core pass 2 (tc_rho)
    int32_t yz0;             // tensor-core pass 2: index of this launch's first Y slab in the plan's Y
    int32_t* err;            // tensor-core pass 2: set to 1 when a bounded wait gives up
    // complex transforms of the forward kernels (the Bluestein path): with cin set,
    // the forward reads M complex values from cin instead of the real signal and
    // writes all M outputs, by cmode: 1 conj(X G), 2 conj(X), 3 X (X the e^{-} DFT)
    const float2* cin;
    const float2* cG;
    int32_t cmode;
    int32_t fpack;           // forward: 1 = real input packed as f(2q) + i f(2q + 1), an M/2-point DFT
};

// Rows of the wide-scale intermediate in the order the tensor-core pass 2
// reads them (L = 1024): bits 1-2 and 6-7 of the row index swapped (an involution).
__host__ __device__ constexpr int tc_rho(int b) { return (b & ~0xC6) | ((b & 0x06) << 5) | ((b & 0xC0) >> 5); }

// Block coordinates of a CTA within its launch.  A plain launch takes them from
// blockIdx and gridDim.  A grouped launch merges the launches of one kernel
// made by several plans into one grid: each CTA then takes the coordinates it
// has within the launch it came from (see group_args).
struct Cta {
    int x, y;   // blockIdx.x, blockIdx.y of the original launch
    int nx;     // its gridDim.x
};
__device__ __forceinline__ Cta cta_plain() { return {(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x}; }

// Grouped launch descriptor.  CTA b of the merged grid runs CTA (x, y) of
// sub-launch i = cta_sub[b], where geom[i] = (first merged CTA of i, grid.x of
// i) and x + nx y = b - first; the kernel argument of sub-launch i is the
// struct at args + i * stride.  The sub-launches of one grouped launch are
// independent of each other (no order among them is kept).
struct GroupMap {
    const unsigned char* args;
    const int32_t* cta_sub;
    const int2* geom;
    int32_t stride;
};

// Copies this CTA's kernel argument into shared memory and returns it; sets c.
// Every thread of the block must call it (it ends with a barrier).
template <class A>
__device__ __forceinline__ const A& group_args(const GroupMap& g, Cta& c) {
    static_assert(sizeof(A) % 4 == 0, "argument structs are copied as 32-bit words");
    __shared__ __align__(16) uint32_t sa[sizeof(A) / 4];
    const int i = __ldg(&g.cta_sub[blockIdx.x]);
    const int2 geo = __ldg(&g.geom[i]);
    const int local = (int)blockIdx.x - geo.x;
    c.x = local % geo.y;
    c.y = local / geo.y;
    c.nx = geo.y;
    const uint32_t* src = (const uint32_t*)(g.args + (size_t)i * (size_t)g.stride);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
    for (int w = tid; w < (int)(sizeof(A) / 4); w += nthr) sa[w] = __ldg(&src[w]);
    __syncthreads();
    return *reinterpret_cast<const A*>(sa);
}

// Pruned pass-1 launch argument (the pass-2 length L and the tiles per column)
struct Wide1pArgs {
    Params p;
    int32_t L, tpb;
    int32_t pad_[2];
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// e^{-2 pi i j / M}, j in [0, M)
__device__ __forceinline__ float2 tw_m(const Params& p, uint32_t j) {
    float2 hi = __ldg(&p.tw_hi[j >> p.h]);
    float2 lo = __ldg(&p.tw_lo[j & ((1u << p.h) - 1u)]);
    return cmul(hi, lo);
}

// e^x = 2^(x log2 e) with the hardware base-2 exponential (relative error
// about 2^-22 for the arguments that matter here, |x| < 40; flushes to 0 below)
__device__ __forceinline__ float exp_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x * 1.44269504088896341f));
    return y;
}

// amp * psi_hat(alpha k) for the signed bin k (Table 2 spectra)
__device__ __forceinline__ float psi_gen(const ScaleGen& g, int wavelet, float half_w0sq, float corr_v2, int k) {
    float kf = (float)k;
    float v = fmaf(g.a_hi, kf, g.a_lo * kf);
    if (wavelet == WAV_GDW) {
        float v2 = v * v;
        return g.amp * v2 * exp_fast(-v2);
    }
    if (wavelet == WAV_CBSW) {                              // 64 C_N sin^6(u/2) / u^4
        if (v == 0.f) return 0.f;
        const float sn = sinf(0.5f * v), s2 = sn * sn, v2 = v * v;
        return g.amp * (s2 * s2 * s2) / (v2 * v2);
    }
    if (wavelet == WAV_CWGDW) {                             // sqrt(2 pi) C_N u (u cosh u - sinh u) e^{-u^2/2}
        const float h = -0.5f * v * v;
        return g.amp * v * 0.5f * ((v - 1.f) * exp_fast(v + h) + (v + 1.f) * exp_fast(h - v));
    }
    float d = (float)(k - g.k0_int) - g.k0_frac;           // k - omega0/alpha, exact integer part
    float t = fmaf(g.a_hi, d, g.a_lo * d);                 // alpha k - omega0
    const float v2 = v * v;
    const float corr = v2 < corr_v2 ? exp_fast(fmaf(-0.5f, v2, -half_w0sq)) : 0.f;
    return g.amp * (exp_fast(-0.5f * t * t) - corr);
}

// F is re-read by every scale: keep it in L2 (evict-last)
__device__ __forceinline__ float2 ld_keep(const float2* q) {
    uint64_t pol;
    float2 v;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(q), "l"(pol));
    return v;
}

// F at the signed bin k: F(-k) = conj F(k) for a real signal
__device__ __forceinline__ float2 spec_at(const float2* __restrict__ Fp, int k) {
    float2 f = ld_keep(&Fp[k >= 0 ? k : -k]);
    return make_float2(f.x, k >= 0 ? f.y : -f.y);
}

// Z(k) of a job (the pointwise product of Eq. 10, scaled) given f = F(k)
__device__ __forceinline__ float2 band_value_f(const Params& p, const Job& J, int k, float2 f) {
    float g0 = psi_gen(J.g[0], p.wavelet, p.half_w0sq, p.corr_v2, k);
    if (wav_real(p.wavelet)) {
        float g1 = J.g[1].row >= 0 ? psi_gen(J.g[1], p.wavelet, p.half_w0sq, p.corr_v2, k) : 0.f;
        return make_float2(fmaf(f.x, g0, -f.y * g1), fmaf(f.x, g1, f.y * g0));
    }
    return make_float2(f.x * g0, f.y * g0);
}

__device__ __forceinline__ float2 band_value(const Params& p, const Job& J, int k) {
    return band_value_f(p, J, k, spec_at(p.Fp, k));
}

__device__ __forceinline__ float load_signal(const Params& p, int n) {
    if (n >= p.N) return 0.f;
    return p.sig_f64 ? (float)__ldg(&((const double*)p.signal)[n]) : __ldg(&((const float*)p.signal)[n]);
}

// ------------------------------------------------- register DFTs (sign -)

// cos and -sin of 2 pi q / 32
__host__ __device__ constexpr float kc32(int q) {
    return q == 1 ? 9.807852804e-01f : q == 2 ? 9.238795325e-01f : q == 3 ? 8.314696123e-01f
         : q == 5 ? 5.555702330e-01f : q == 6 ? 3.826834324e-01f : q == 7 ? 1.950903220e-01f
         : q == 9 ? -1.950903220e-01f : q == 10 ? -3.826834324e-01f : q == 11 ? -5.555702330e-01f
         : q == 13 ? -8.314696123e-01f : q == 14 ? -9.238795325e-01f : q == 15 ? -9.807852804e-01f : 0.f;
}
__host__ __device__ constexpr float ks32(int q) {
    return q == 1 ? -1.950903220e-01f : q == 2 ? -3.826834324e-01f : q == 3 ? -5.555702330e-01f
         : q == 5 ? -8.314696123e-01f : q == 6 ? -9.238795325e-01f : q == 7 ? -9.807852804e-01f
         : q == 9 ? -9.807852804e-01f : q == 10 ? -9.238795325e-01f : q == 11 ? -8.314696123e-01f
         : q == 13 ? -5.555702330e-01f : q == 14 ? -3.826834324e-01f : q == 15 ? -1.950903220e-01f : 0.f;
}

// x * e^{-2 pi i Q / 32}, 0 <= Q < 16
template <int Q>
__device__ __forceinline__ float2 mul_w32(float2 x) {
    constexpr float r = 0.70710678118654752440f;
    if constexpr (Q == 0) return x;
    else if constexpr (Q == 8) return make_float2(x.y, -x.x);
    else if constexpr (Q == 4) return make_float2(r * (x.x + x.y), r * (x.y - x.x));
    else if constexpr (Q == 12) return make_float2(r * (x.y - x.x), -r * (x.x + x.y));
    else {
        constexpr float c = kc32(Q), s = ks32(Q);
        return make_float2(fmaf(x.x, c, -x.y * s), fmaf(x.x, s, x.y * c));
    }
}

template <int R, int Q>
__device__ __forceinline__ void dft_combine(float2* v, const float2* e, const float2* o) {
    if constexpr (Q < R / 2) {
        float2 t = mul_w32<Q * (32 / R)>(o[Q]);
        v[Q] = cadd(e[Q], t);
        v[Q + R / 2] = csub(e[Q], t);
        dft_combine<R, Q + 1>(v, e, o);
    }
}

// In-place R-point DFT X(q) = sum_r v(r) e^{-2 pi i r q / R}, natural order.
template <int R>
__device__ __forceinline__ void dft(float2* v) {
    if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        d13 = make_float2(d13.y, -d13.x);
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, d13);
        v[3] = csub(d02, d13);
    } else if constexpr (R > 4) {
        float2 e[R / 2], o[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; i++) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft<R / 2>(e);
        dft<R / 2>(o);
        dft_combine<R, 0>(v, e, o);
    }
}

// ------------------------------------------------------- CTA-level FFT plan

// L = 2^LOGL splits into ceil(LOGL / MAXLR) Stockham stages of at most
// 2^MAXLR points each (larger radices first).  MAXLR = 5 keeps 32 complex
// values per thread; MAXLR = 4 halves the registers per thread for higher
// occupancy at the cost of more shared-memory exchanges.
__host__ __device__ constexpr int n_stages(int logl, int maxlr = 5) { return (logl + maxlr - 1) / maxlr; }
__host__ __device__ constexpr int stage_logr(int logl, int s, int maxlr = 5) {
    return logl / n_stages(logl, maxlr) + (s < logl % n_stages(logl, maxlr) ? 1 : 0);
}
__host__ __device__ constexpr int stage_logns(int logl, int s, int maxlr = 5) {
    return s == 0 ? 0 : stage_logns(logl, s - 1, maxlr) + stage_logr(logl, s - 1, maxlr);
}
// butterflies of the last (smallest-radix) stage
__host__ __device__ constexpr int max_bfly(int logl, int maxlr = 5) {
    return 1 << (logl - stage_logr(logl, n_stages(logl, maxlr) - 1, maxlr));
}
// threads per column = butterflies of the first (largest-radix) stage; a
// thread takes NB / col_threads butterflies of a later stage, so that every
// thread holds the same number of values in every stage
__host__ __device__ constexpr int col_threads(int logl, int maxlr = 5) {
    return 1 << (logl - stage_logr(logl, 0, maxlr));
}
// odd smem row stride for T columns (bank spread for both thread mappings)
__host__ __device__ constexpr int row_stride(int T) { return T == 1 ? 1 : ((T & 1) ? T : T + 1); }

// CTAs per SM requested from the register allocator (caps registers at
// 65536 / (NT * min_blocks), i.e. 128 per thread for NT <= 512)
__host__ __device__ constexpr int min_blocks(int nt) { return nt >= 512 ? 1 : 512 / nt; }

template <int LOGL, int S, int MAXLR = 5>
struct Stage {
    static constexpr int LR = stage_logr(LOGL, S, MAXLR), R = 1 << LR;
    static constexpr int LNS = stage_logns(LOGL, S, MAXLR), NS = 1 << LNS;
    static constexpr int NB = (1 << LOGL) >> LR;   // butterflies per column
};

// Stage S >= 1 input: v[r] = buf[(j + r NB) * TT + t] times the stage twiddle
// e^{-2 pi i r (j mod NS) / (NS R)}
template <int LOGL, int S, int TT, int MAXLR>
__device__ __forceinline__ void stage_load(float2* v, const float2* buf, int j, int t,
                                           const float2* __restrict__ tw_tab) {
    using St = Stage<LOGL, S, MAXLR>;
#pragma unroll
    for (int r = 0; r < St::R; r++) v[r] = buf[(j + r * St::NB) * TT + t];
    if constexpr (S > 0) {
        const int k = j & (St::NS - 1);
        const float2* tw = tw_tab + (St::NS * St::R);
#pragma unroll
        for (int r = 1; r < St::R; r++) v[r] = cmul(v[r], __ldg(&tw[r * k]));
    }
}

// Non-final stage output: buf[((j - k) R + k + r NS) * TT + t]
template <int LOGL, int S, int TT, int MAXLR>
__device__ __forceinline__ void stage_store(const float2* v, float2* buf, int j, int t) {
    using St = Stage<LOGL, S, MAXLR>;
    const int k = j & (St::NS - 1);
    const int base = (j - k) * St::R + k;
#pragma unroll
    for (int r = 0; r < St::R; r++) buf[(base + r * St::NS) * TT + t] = v[r];
}

// Middle stage S (0 < S < NST - 1): load, twiddle, DFT, exchange.  Each
// thread holds its NB / P butterflies across the barrier.
template <int LOGL, int S, int T, int TT, int MAXLR>
__device__ __forceinline__ void cta_mid_stage(float2* buf, const float2* __restrict__ tw_tab, int tlim) {
    using St = Stage<LOGL, S, MAXLR>;
    constexpr int P = col_threads(LOGL, MAXLR), NBT = St::NB / P;
    __syncthreads();
    const int t = threadIdx.x % T, j = threadIdx.x / T;
    float2 v[NBT][St::R];
    const bool act = t < tlim;
    if (act) {
#pragma unroll
        for (int q = 0; q < NBT; q++) {
            stage_load<LOGL, S, TT, MAXLR>(v[q], buf, j + q * P, t, tw_tab);
            dft<St::R>(v[q]);
        }
    }
    __syncthreads();
    if (act) {
#pragma unroll
        for (int q = 0; q < NBT; q++) stage_store<LOGL, S, TT, MAXLR>(v[q], buf, j + q * P, t);
    }
}

template <int LOGL, int S, int NST, int T, int TT, int MAXLR>
__device__ __forceinline__ void cta_mid_stages(float2* buf, const float2* __restrict__ tw_tab, int tlim) {
    if constexpr (S < NST - 1) {
        cta_mid_stage<LOGL, S, T, TT, MAXLR>(buf, tw_tab, tlim);
        cta_mid_stages<LOGL, S + 1, NST, T, TT, MAXLR>(buf, tw_tab, tlim);
    }
}

// Runs the CTA FFT of T columns of length L.  fill(v, j, t, stride) produces
// the first stage's R inputs x(j + r stride); out(v, j, t, stride) consumes
// the last stage's R outputs X(j + r stride).  The last stage maps threads
// j-fastest when LAST_JFAST (coalesced writes along the DFT index),
// t-fastest otherwise.  Only columns t < tlim (<= T) are computed.
template <int LOGL, int T, int NT, bool LAST_JFAST, int MAXLR, class Fill, class Out, bool FILL_IN_BUF = false>
__device__ __forceinline__ void cta_fft(float2* buf, const float2* __restrict__ tw_tab, Fill& fill, Out& out,
                                        int tlim) {
    constexpr int NST = n_stages(LOGL, MAXLR);
    constexpr int TT = row_stride(T);
    const int tid = threadIdx.x;
    {
        using S0 = Stage<LOGL, 0, MAXLR>;
        constexpr bool last = (NST == 1);
        const int t = (last && LAST_JFAST) ? tid / S0::NB : tid % T;
        const int j = (last && LAST_JFAST) ? tid % S0::NB : tid / T;
        float2 v[S0::R];
        const bool act = j < S0::NB && t < tlim;
        if (act) {
            fill(v, j, t, S0::NB);
            dft<S0::R>(v);
        }
        if constexpr (FILL_IN_BUF && !last) __syncthreads();   // the fill read buf in place
        if (act) {
            if constexpr (last) out(v, j, t, S0::NB);
            else stage_store<LOGL, 0, TT, MAXLR>(v, buf, j, t);
        }
    }
    if constexpr (NST >= 2) {
        cta_mid_stages<LOGL, 1, NST, T, TT, MAXLR>(buf, tw_tab, tlim);
        __syncthreads();
        using SL = Stage<LOGL, NST - 1, MAXLR>;
        constexpr int P = col_threads(LOGL, MAXLR);
        const int t = LAST_JFAST ? tid / P : tid % T;
        const int j = LAST_JFAST ? tid % P : tid / T;
        if (t < tlim) {
#pragma unroll
            for (int jj = j; jj < SL::NB; jj += P) {
                float2 v[SL::R];
                stage_load<LOGL, NST - 1, TT, MAXLR>(v, buf, jj, t, tw_tab);
                dft<SL::R>(v);
                out(v, jj, t, SL::NB);
            }
        }
    }
}

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

// ------------------------------------------------------- output to W rows

// Cache policy of the two large streams.  W is written once and never read
// back here: its stores are cache-streaming (evict-first).  The wide-scale
// intermediate Y is stored with an L2 evict-last policy by pass 1, so that it
// is still on chip when pass 2 reads it, exactly once (evict-first).
__device__ __forceinline__ void st_stream(float2* q, float2 v) { __stcs(q, v); }
__device__ __forceinline__ void st_stream(float* q, float v) { __stcs(q, v); }
__device__ __forceinline__ uint64_t l2_policy_keep() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ void st_keep(float2* q, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(q), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ float2 ld_once(const float2* q) { return __ldcs(q); }

// Stores X(d + A c) for the last stage's outputs c = j + r * cstride
// (d = d0 + t) at W[row][n - out_off]; with CROP, only outputs n in
// [out_off, out_off + out_len) are kept (the zero-boundary crop, or the
// window of a periodically extended signal).  Accumulates |W|^2 per row.
template <bool CROP>
struct WOut {
    const Params* p;
    float* r0;           // GDW rows (re -> r0, im -> r1)
    float* r1;
    float2* rc;          // Morlet row
    int d0;
    float pw0, pw1;
    template <int R>
    __device__ __forceinline__ void operator()(const float2 (&v)[R], int j, int t, int cstride) {
        const int n0 = d0 + t + p->A * j;
        const int step = p->A * cstride;
        const int off = CROP ? (int)p->out_off : 0;    // without the crop (M = N) the window is [0, N)
        const unsigned len = (unsigned)p->out_len;
        if (rc) {
            float2* q = rc + (n0 - off);
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!CROP || (unsigned)(n0 + r * step - off) < len) {
                    st_stream(q + r * step, v[r]);
                    pw0 = fmaf(v[r].x, v[r].x, fmaf(v[r].y, v[r].y, pw0));
                }
            }
        } else {
            float* q0 = r0 + (n0 - off);
            float* q1 = r1 ? r1 + (n0 - off) : q0;
            const bool two = r1 != nullptr;
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (!CROP || (unsigned)(n0 + r * step - off) < len) {
                    st_stream(q0 + r * step, v[r].x);
                    pw0 = fmaf(v[r].x, v[r].x, pw0);
                    if (two) {
                        st_stream(q1 + r * step, v[r].y);
                        pw1 = fmaf(v[r].y, v[r].y, pw1);
                    }
                }
            }
        }
    }
};

template <bool CROP>
__device__ __forceinline__ WOut<CROP> make_wout(const Params& p, const Job& J, int d0) {
    WOut<CROP> o;
    o.p = &p;
    o.d0 = d0;
    o.pw0 = o.pw1 = 0.f;
    if (wav_real(p.wavelet)) {
        o.rc = nullptr;
        o.r0 = (float*)p.W + (int64_t)J.g[0].row * p.out_len;
        o.r1 = J.g[1].row >= 0 ? (float*)p.W + (int64_t)J.g[1].row * p.out_len : nullptr;
    } else {
        o.rc = (float2*)p.W + (int64_t)J.g[0].row * p.out_len;
        o.r0 = o.r1 = nullptr;
    }
    return o;
}

template <int NT, class O>
__device__ __forceinline__ void write_partials(const Params& p, const Job& J, const O& o, int slot, double* red) {
    if (!p.do_power) return;
    double s0, s1;
    block_sum2<NT>(o.pw0, o.pw1, &s0, &s1, red);
    if (threadIdx.x == 0) {
        p.partials[J.g[0].part_off + slot] = s0;
        if (J.g[1].row >= 0 && wav_real(p.wavelet)) p.partials[J.g[1].part_off + slot] = s1;
    }
}

// ------------------------------------------------------------ band kernel

// First-stage fill of a band tile.  The sub-problem has length Mp = M / mult
// and its band is [kb, kb + L); Zs[i] holds z(kb + i) (zero past the band).
// Slot rho of the first stage takes k_rho = kb + ((rho - kb) mod L) and
// x(rho) = Zs[k_rho - kb] e^{-2 pi i k_rho d / Mp}.  For the slots
// rho = j + r NB0 of one thread, k_rho grows by NB0 per slot except once,
// where it wraps by -L, so the twiddle is carried by a recurrence (at most
// 32 steps) from one exact anchor.
//
// With direct depth RD > 1 the band may be up to RD L bins wide: residue rho
// then collects the RD bins k_rho + i L (i < RD), and since
// e^{-2 pi i (k + i L) d / Mp} = e^{-2 pi i k d / Mp} h^i with h =
// e^{-2 pi i L d / Mp} a per-thread constant, the slot value is
// w_rho * sum_i Zs[e + i L] h^i (Horner), Zs zero past the band.
template <int LOGL, int RD = 1>
struct BandFill {
    const Params* p;
    const float2* Zs;
    int kb;          // first bin of the band (sub-problem index space)
    uint32_t mult;   // e^{-2 pi i x / Mp} = e^{-2 pi i (x mult) / M}
    int d0;
    template <int R>
    __device__ __forceinline__ void operator()(float2 (&v)[R], int j, int t, int nb) {
        constexpr int L = 1 << LOGL;
        const uint32_t d = (uint32_t)(d0 + t);
        const uint32_t mask = (uint32_t)(p->M - 1);
        const int e0 = (j - kb) & (L - 1);
        const int r_w = (L - e0 + nb - 1) / nb;          // slot index of the wrap (>= R: none)
        const uint32_t k0 = (uint32_t)(kb + e0);
        // e^{-2 pi i k_r d / Mp} over the slots as CH interleaved recurrences
        // (chain depth R / CH): w_{r + CH} = w_r g^CH, times h^{-1} =
        // e^{-2 pi i (-L) d / Mp} once when the chain crosses the wrap slot r_w
        constexpr int CH = R >= 8 ? 4 : 1;
        const float2 g = tw_m(*p, ((uint32_t)nb * d * mult) & mask);
        const float2 h = tw_m(*p, ((uint32_t)(-L) * d * mult) & mask);
        float2 w[CH];
        w[0] = tw_m(*p, (k0 * d * mult) & mask);
#pragma unroll
        for (int c = 1; c < CH; c++) w[c] = cmul(w[c - 1], c == r_w ? cmul(g, h) : g);
        float2 gc = g;
#pragma unroll
        for (int c = 1; c < CH; c++) gc = cmul(gc, g);
        const float2 gch = cmul(gc, h);
        float2 hd = make_float2(1.f, 0.f);
        if constexpr (RD > 1) hd = tw_m(*p, ((uint32_t)L * d * mult) & mask);   // e^{-2 pi i L d / Mp}
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int e = (e0 + r * nb) & (L - 1);
            float2 z = Zs[e + (RD - 1) * L];
#pragma unroll
            for (int i = RD - 2; i >= 0; i--) z = cadd(cmul(z, hd), Zs[e + i * L]);
            v[r] = cmul(z, w[r % CH]);
            if (r + CH < R) w[r % CH] = cmul(w[r % CH], (r < r_w && r + CH >= r_w) ? gch : gc);
        }
    }
};

// One CTA handles D consecutive tiles of T columns of one job (D = p.D at
// run time): the band values, the job descriptor and the power reduction are
// paid once per CTA.
template <int LOGL, int T, bool CROP, int RD, int MAXLR>
__device__ __forceinline__ void band_body(const Params& p, const Cta c) {
    constexpr int L = 1 << LOGL;
    constexpr int NT = T * col_threads(LOGL, MAXLR);
    extern __shared__ float2 smem[];
    float2* Zs = smem;
    float2* buf = smem + RD * L;
    __shared__ double red[2 * ((NT + 31) / 32)];
    __shared__ Job sJ;

    const int tile = c.x;
    if (threadIdx.x == 0) sJ = p.jobs[__ldg(&p.tile_job[tile])];
    __syncthreads();
    const Job& J = sJ;
    const int dbase = (tile - J.tile0) * T * p.D;
    // the job's band values Z(k) = F(k) amp psi_hat(alpha k), generated here from the
    // spectrum (Eq. 10) into shared memory: no per-scale product goes to global memory
    for (int i = threadIdx.x; i < RD * L; i += NT)
        Zs[i] = i < J.K ? band_value(p, J, J.k_lo + i) : make_float2(0.f, 0.f);
    WOut<CROP> out = make_wout<CROP>(p, J, dbase);
#pragma unroll 1
    for (int q = 0; q < p.D; q++) {
        const int d0 = dbase + q * T;
        if (d0 >= p.A) break;
        __syncthreads();
        BandFill<LOGL, RD> fill{&p, Zs, J.k_lo, 1u, d0};
        out.d0 = d0;
        cta_fft<LOGL, T, NT, false, MAXLR>(buf, p.tw_tab, fill, out, min(T, p.A - d0));
    }
    write_partials<NT>(p, J, out, tile - J.tile0, red);
}

template <int LOGL, int T, bool CROP, int RD = 1, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL, MAXLR), min_blocks(T * col_threads(LOGL, MAXLR)))
    k_band(Params p) {
    band_body<LOGL, T, CROP, RD, MAXLR>(p, cta_plain());
}
template <int LOGL, int T, bool CROP, int RD = 1, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL, MAXLR), min_blocks(T * col_threads(LOGL, MAXLR)))
    k_band_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    band_body<LOGL, T, CROP, RD, MAXLR>(p, c);
}

// ------------------------------------------------------------ wide pass 1

// x(a) = Z(b + L a) for column b (zero outside the band) ...
struct Wide1Fill {
    const Params* p;
    const Job* J;
    int b0, L, A;
    template <int R>
    __device__ __forceinline__ void operator()(float2 (&v)[R], int j, int t, int stride) {
        const int half = p->M >> 1;
        const int kend = J->k_lo + J->K;
        const float2* col = p->Ft + (int64_t)(b0 + t) * A;   // column b of the spectrum, contiguous in a
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int a = j + r * stride;
            const int k = b0 + t + L * a;                      // unsigned bin in [0, M)
            const int ks = k <= half ? k : k - p->M;
            v[r] = (ks >= J->k_lo && ks < kend) ? band_value_f(*p, *J, ks, __ldg(&col[a])) : make_float2(0.f, 0.f);
        }
    }
};

// ... and Y[b][d] = e^{-2 pi i b d / M} * (A-point DFT)(d).  Column layout:
// full pass 1 (COLS_B): the tile's columns are b0 + t and d = c; pruned pass
// 1: one column b, the tile's columns are d1 = d0 + t and d = d1 + A1 c.
// The twiddle over the R outputs of a thread is a recurrence from one anchor.
template <bool COLS_B>
struct YOut {
    const Params* p;
    float2* Y;
    int b0, d0, A, A1;
    template <int R>
    __device__ __forceinline__ void operator()(const float2 (&v)[R], int j, int t, int stride) {
        const uint32_t b = (uint32_t)(COLS_B ? b0 + t : b0);
        const uint32_t d1 = (uint32_t)(COLS_B ? 0 : d0 + t);
        const uint32_t mask = (uint32_t)(p->M - 1);
        float2* row = Y + (int64_t)(p->yperm ? (uint32_t)tc_rho((int)b) : b) * A;
        const uint64_t pol = l2_policy_keep();
        const uint32_t dj = d1 + (uint32_t)A1 * (uint32_t)j;
        constexpr int CH = R >= 8 ? 4 : 1;                 // interleaved recurrences
        // e^{-2 pi i b d / Mt} for the transform length Mt = M >> fpack, from the M table
        const uint32_t sh = (uint32_t)p->fpack;
        const float2 g = tw_m(*p, ((b * (uint32_t)A1 * (uint32_t)stride) << sh) & mask);
        float2 w[CH];
        w[0] = tw_m(*p, ((b * dj) << sh) & mask);
#pragma unroll
        for (int c = 1; c < CH; c++) w[c] = cmul(w[c - 1], g);
        float2 gc = g;
#pragma unroll
        for (int c = 1; c < CH; c++) gc = cmul(gc, g);
#pragma unroll
        for (int r = 0; r < R; r++) {
            st_keep(row + (dj + (uint32_t)A1 * (uint32_t)(r * stride)), cmul(v[r], w[r % CH]), pol);
            if (r + CH < R) w[r % CH] = cmul(w[r % CH], gc);
        }
    }
};

// grid (L / T, jobs in batch): T columns b of the A-point DFTs of one job
template <int LOGA, int T, int MAXLR>
__device__ __forceinline__ void wide1_body(const Params& p, const Cta c) {
    constexpr int NT = T * col_threads(LOGA, MAXLR);
    extern __shared__ float2 smem[];
    const int L = p.M >> LOGA;
    __shared__ Job sJ;
    if (threadIdx.x == 0) sJ = p.jobs[p.job0 + c.y];
    __syncthreads();
    const int b0 = c.x * T;
    Wide1Fill fill{&p, &sJ, b0, L, 1 << LOGA};
    YOut<true> out{&p, p.Y + (int64_t)c.y * p.M, b0, 0, 1 << LOGA, 1};
    cta_fft<LOGA, T, NT, true, MAXLR>(smem, p.tw_tab, fill, out, min(T, L - b0));
}

template <int LOGA, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGA, MAXLR), min_blocks(T * col_threads(LOGA, MAXLR))) k_wide1(Params p) {
    wide1_body<LOGA, T, MAXLR>(p, cta_plain());
}
template <int LOGA, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGA, MAXLR), min_blocks(T * col_threads(LOGA, MAXLR))) k_wide1_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    wide1_body<LOGA, T, MAXLR>(p, c);
}

// Pruned pass 1: column b only holds the band bins k = b mod L, i.e. the
// sub-band a in [a0, a0 + P_b) of the A-point problem (k = b + L a), so its
// A-point DFT is itself a band tile of L1 >= P_b points over A1 = A / L1
// columns d1 (d = d1 + A1 c1).  grid (L * tiles_per_b, jobs in batch).
template <int LOGL1, int T, int MAXLR>
__device__ __forceinline__ void wide1p_body(const Params& p, const int L, const int tiles_per_b, const Cta c) {
    constexpr int L1 = 1 << LOGL1;
    constexpr int NT = T * col_threads(LOGL1, MAXLR);
    extern __shared__ float2 smem[];
    float2* Zs = smem;
    float2* buf = smem + L1;
    __shared__ Job sJ;
    if (threadIdx.x == 0) sJ = p.jobs[p.job0 + c.y];
    __syncthreads();
    const Job& J = sJ;
    const int b = c.x / tiles_per_b;
    const int d0 = (c.x - b * tiles_per_b) * T;
    const int A = p.M / L;
    const int A1 = A >> LOGL1;
    const int kb0 = J.k_lo + ((b - J.k_lo) & (L - 1));      // first band bin = b mod L
    const int khi = J.k_lo + J.K - 1;
    const int a0 = (kb0 - b) / L;                             // exact: kb0 = b (mod L)
    const float2* col = p.Ft + (int64_t)b * A;                // unsigned bin b + L a at col[a mod A]
    for (int i = threadIdx.x; i < L1; i += NT) {
        const int k = kb0 + L * i;
        Zs[i] = k <= khi ? band_value_f(p, J, k, __ldg(&col[(a0 + i) & (A - 1)])) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    BandFill<LOGL1> fill{&p, Zs, a0, (uint32_t)L, d0};
    YOut<false> out{&p, p.Y + (int64_t)c.y * p.M, b, d0, A, A1};
    cta_fft<LOGL1, T, NT, false, MAXLR>(buf, p.tw_tab, fill, out, min(T, A1 - d0));
}

template <int LOGL1, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL1, MAXLR), min_blocks(T * col_threads(LOGL1, MAXLR)))
    k_wide1p(Wide1pArgs a) {
    wide1p_body<LOGL1, T, MAXLR>(a.p, a.L, a.tpb, cta_plain());
}
template <int LOGL1, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL1, MAXLR), min_blocks(T * col_threads(LOGL1, MAXLR)))
    k_wide1p_g(GroupMap g) {
    Cta c;
    const Wide1pArgs& a = group_args<Wide1pArgs>(g, c);
    wide1p_body<LOGL1, T, MAXLR>(a.p, a.L, a.tpb, c);
}

// ------------------------------------------------------------ wide pass 2

// x(b) = Y[b][d0 + t]
struct YFill {
    const float2* Y;
    int A, d0;
    template <int R>
    __device__ __forceinline__ void operator()(float2 (&v)[R], int j, int t, int stride) {
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = ld_once(&Y[(int64_t)(j + r * stride) * A + d0 + t]);
    }
};

// grid (A / (T D), jobs in batch): D = p.D tiles of T columns d of the
// L-point DFTs over b
template <int LOGL, int T, bool CROP, int MAXLR>
__device__ __forceinline__ void wide2_body(const Params& p, const Cta c) {
    constexpr int NT = T * col_threads(LOGL, MAXLR);
    extern __shared__ float2 smem[];
    __shared__ double red[2 * ((NT + 31) / 32)];
    __shared__ Job sJ;
    if (threadIdx.x == 0) sJ = p.jobs[p.job0 + c.y];
    __syncthreads();
    const Job& J = sJ;
    const int dbase = c.x * T * p.D;
    WOut<CROP> out = make_wout<CROP>(p, J, dbase);
#pragma unroll 1
    for (int q = 0; q < p.D; q++) {
        const int d0 = dbase + q * T;
        if (d0 >= p.A) break;
        if (q > 0) __syncthreads();
        YFill fill{p.Y + (int64_t)c.y * p.M, p.A, d0};
        out.d0 = d0;
        cta_fft<LOGL, T, NT, false, MAXLR>(smem, p.tw_tab, fill, out, min(T, p.A - d0));
    }
    write_partials<NT>(p, J, out, c.x, red);
}

template <int LOGL, int T, bool CROP, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL, MAXLR), min_blocks(T * col_threads(LOGL, MAXLR)))
    k_wide2(Params p) {
    wide2_body<LOGL, T, CROP, MAXLR>(p, cta_plain());
}
template <int LOGL, int T, bool CROP, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL, MAXLR), min_blocks(T * col_threads(LOGL, MAXLR)))
    k_wide2_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    wide2_body<LOGL, T, CROP, MAXLR>(p, c);
}

// ------------------------------------------------------------ forward

// x(a) = f(b + L a) (zero past N)
struct SigFill {
    const Params* p;
    int b0, L;
    template <int R>
    __device__ __forceinline__ void operator()(float2 (&v)[R], int j, int t, int stride) {
        if (p->cin) {
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = __ldg(&p->cin[b0 + t + L * (j + r * stride)]);
        } else if (p->fpack) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int q = b0 + t + L * (j + r * stride);
                v[r] = make_float2(load_signal(*p, 2 * q), load_signal(*p, 2 * q + 1));
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = make_float2(load_signal(*p, b0 + t + L * (j + r * stride)), 0.f);
        }
    }
};

// F(n) = conj X(n) for n = d0 + t + A c <= M/2 (the forward uses the paper's
// e^{+} sign: sum_n f(n) e^{+2 pi i m n / M} = conj of the e^{-} DFT of real f).
// Complex transforms (mode > 0) write every n < M: conj(X(n) G(n)), conj X(n)
// or X(n).
struct FOut {
    float2* F;
    int A, d0, half;
    const float2* G;
    int mode;
    template <int R>
    __device__ __forceinline__ void operator()(const float2 (&v)[R], int j, int t, int stride) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int n = d0 + t + A * (j + r * stride);
            if (mode == 0) {
                if (n <= half) F[n] = make_float2(v[r].x, -v[r].y);
            } else if (mode == 1) {
                const float2 x = cmul(v[r], __ldg(&G[n]));
                F[n] = make_float2(x.x, -x.y);
            } else {
                F[n] = mode == 2 ? make_float2(v[r].x, -v[r].y) : v[r];
            }
        }
    }
};

// pass 1 of the forward: grid L / T, A-point DFTs of the columns b
template <int LOGA, int T, int MAXLR>
__device__ __forceinline__ void fwd1_body(const Params& p, const Cta c) {
    constexpr int NT = T * col_threads(LOGA, MAXLR);
    extern __shared__ float2 smem[];
    const int L = (p.M >> p.fpack) >> LOGA;
    const int b0 = c.x * T;
    SigFill fill{&p, b0, L};
    YOut<true> out{&p, p.Y, b0, 0, 1 << LOGA, 1};
    cta_fft<LOGA, T, NT, true, MAXLR>(smem, p.tw_tab, fill, out, min(T, L - b0));
}
template <int LOGA, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGA, MAXLR), min_blocks(T * col_threads(LOGA, MAXLR))) k_fwd1(Params p) {
    fwd1_body<LOGA, T, MAXLR>(p, cta_plain());
}
template <int LOGA, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGA, MAXLR), min_blocks(T * col_threads(LOGA, MAXLR))) k_fwd1_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    fwd1_body<LOGA, T, MAXLR>(p, c);
}

// pass 2 of the forward (or the whole forward when A = 1): grid A / T
template <int LOGL, int T, int MAXLR>
__device__ __forceinline__ void fwd2_body(const Params& p, const Cta c) {
    constexpr int NT = T * col_threads(LOGL, MAXLR);
    extern __shared__ float2 smem[];
    const int d0 = c.x * T;
    FOut out{p.Fp_out, p.A, d0, p.M >> 1, p.cG, p.cmode};
    if (p.A == 1) {
        SigFill fill{&p, 0, 1};
        cta_fft<LOGL, T, NT, false, MAXLR>(smem, p.tw_tab, fill, out, 1);
    } else {
        YFill fill{p.Y, p.A, d0};
        cta_fft<LOGL, T, NT, false, MAXLR>(smem, p.tw_tab, fill, out, min(T, p.A - d0));
    }
}
template <int LOGL, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL, MAXLR), min_blocks(T * col_threads(LOGL, MAXLR))) k_fwd2(Params p) {
    fwd2_body<LOGL, T, MAXLR>(p, cta_plain());
}
template <int LOGL, int T, int MAXLR = 5>
__global__ void __launch_bounds__(T * col_threads(LOGL, MAXLR), min_blocks(T * col_threads(LOGL, MAXLR))) k_fwd2_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    fwd2_body<LOGL, T, MAXLR>(p, c);
}

// ------------------------------------------------------------ power

// spectrum[s] = (sum of the row's partials in fixed order) / N
__device__ __forceinline__ void power_finalize_body(const double* __restrict__ partials, const int32_t* __restrict__ off,
                                                    const int32_t* __restrict__ cnt, int32_t S, int64_t N,
                                                    double* __restrict__ spectrum, int s) {
    if (s >= S || cnt[s] == 0) return;          // rows without partials belong to a child plan
    double acc = 0.0;
    for (int i = threadIdx.x; i < cnt[s]; i += 32) acc += partials[off[s] + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) spectrum[s] = acc / (double)N;
}
static __global__ void k_power_finalize(const double* __restrict__ partials, const int32_t* __restrict__ off,
                                        const int32_t* __restrict__ cnt, int32_t S, int64_t N,
                                        double* __restrict__ spectrum) {
    power_finalize_body(partials, off, cnt, S, N, spectrum, blockIdx.x);
}
struct PowerArgs {
    const double* partials;
    const int32_t* off;
    const int32_t* cnt;
    double* spectrum;
    int64_t N;
    int32_t S, pad_;
};
static __global__ void k_power_finalize_g(GroupMap g) {
    Cta c;
    const PowerArgs& a = group_args<PowerArgs>(g, c);
    power_finalize_body(a.partials, a.off, a.cnt, a.S, a.N, a.spectrum, c.x);
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
