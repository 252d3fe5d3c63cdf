// Tensor-core form of the wide scales' second pass (L = 1024-point DFTs).
//
// The inverse DFT of Eq. 9 restricted to one pass-2 column d is
//   X(c) = sum_{b<1024} x(b) w^{b c},  w = e^{-2 pi i / 1024},  x(b) = Y[b][d].
// With b = b0 + 32 b1 and c = c1 + 32 c2 it factors into two 32-point DFT
// stages written as dense matrix products with F[u][v] = e^{-2 pi i u v / 32}:
//   U[c1][b0] = sum_{b1} F[c1][b1] x(b0 + 32 b1)            (stage A)
//   V[c1][b0] = U[c1][b0] w^{b0 c1}                          (twiddle, FP32)
//   X(c1 + 32 c2) = sum_{b0} V[c1][b0] F[b0][c2]              (stage B)
// Complex products are real products with the real and imaginary parts
// stacked along the contraction (K = 64):
//   Re = [Fr | -Fi] [xr; xi],  Im = [Fi | Fr] [xr; xi]   (stage A, F on the left)
//   Re = [Vr | Vi] [Fr; -Fi],  Im = [Vr | Vi] [Fi; Fr]   (stage B, F on the right).
// One warp computes one column with warp-level MMAs (m16n8k16, FP32
// accumulation).  Stage A's accumulator tile (rows c1, columns b0) has the
// register layout of stage B's left operand, so the twiddled accumulators
// feed stage B without any exchange, and because F is symmetric the
// fragments of stage A's left operand are also stage B's right operand.
//
// Operand precision (cwt_precision): FP16 (the column scaled by a power of
// two so that it fits FP16's range), BF16, or hi + lo pairs of either with
// three products per block (hi hi + lo hi + hi lo), which keep about 22 (FP16)
// or 16 (BF16) bits.
// Twiddles, accumulators, the power sums and the output stay FP32.
//
// A CTA takes tiles of 8 consecutive columns, Y[0..1023][d0..d0+7]; each of
// 8 compute warps reads its column from shared memory in the MMA operand
// pattern and writes its 1024 outputs to a staging tile, from which W rows
// are stored with 16-byte vector stores.  Pass 1 writes the rows of Y in the
// order tc_rho (bits 1-2 and 6-7 of the row swapped) and a tile lands in
// shared memory with the 16-byte pairs of each 64-byte row swizzled as the
// TMA 64-byte swizzle places them: the operand reads of a warp and its output
// writes then touch at most two lanes per bank pair.
//   k_wide2_tma: the tile is loaded by TMA (one thread, mbarrier completion,
//     two buffers); 8 compute warps and 4 (2 for the hi + lo forms) store
//     warps work on consecutive tiles at once, handing the staging tile over
//     through named barriers.
//   k_wide2_tc_g: the grouped-launch form (batches), copies with cp.async and
//     stores from the compute warps, same arithmetic and results.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cwt_kernels.cuh"

namespace cwtk {

enum { TC_FP16 = 1, TC_BF16 = 2, TC_FP16X3 = 3, TC_BF16X3 = 4 };   // cwt_precision values of the tensor-core forms
__host__ __device__ constexpr bool tc_x3(int form) { return form == TC_FP16X3 || form == TC_BF16X3; }
__host__ __device__ constexpr bool tc_bf(int form) { return form == TC_BF16 || form == TC_BF16X3; }

constexpr int kTcCols = 8;                             // columns (one per warp) per CTA tile
constexpr int kTcThreads = 32 * kTcCols;
constexpr int kTcTile = 1024 * kTcCols;               // float2 per tile buffer


// float2 index of (row i, column w < 8) in a 1024-byte-aligned tile buffer of
// 64-byte rows, the 16-byte pairs of columns swizzled as the TMA 64-byte
// swizzle stores them (chunk ^= bits 1-2 of the row)
__host__ __device__ __forceinline__ int tc_slot(int i, int w) {
    return 8 * i + 2 * ((w >> 1) ^ ((i >> 1) & 3)) + (w & 1);
}

__device__ __forceinline__ uint32_t u32_of(__half2 h) { return *reinterpret_cast<uint32_t*>(&h); }
__device__ __forceinline__ uint32_t u32_of(__nv_bfloat162 h) { return *reinterpret_cast<uint32_t*>(&h); }

// two values packed as an MMA operand register (a in the low half)
template <int FORM>
__device__ __forceinline__ uint32_t tc_pack(float a, float b) {
    if constexpr (tc_bf(FORM)) return u32_of(__floats2bfloat162_rn(a, b));
    else return u32_of(__floats2half2_rn(a, b));
}
// hi + lo split of two values, a = hi + lo: to about 2^-22 relative in FP16
// pairs, 2^-16 in BF16 pairs
template <int FORM>
__device__ __forceinline__ void tc_split(float a, float b, uint32_t& hi, uint32_t& lo) {
    if constexpr (tc_bf(FORM)) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 f = __bfloat1622float2(h);
        hi = u32_of(h);
        lo = u32_of(__floats2bfloat162_rn(a - f.x, b - f.y));
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 f = __half22float2(h);
        hi = u32_of(h);
        lo = u32_of(__floats2half2_rn(a - f.x, b - f.y));
    }
}

template <int FORM>
__device__ __forceinline__ void tc_mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (tc_bf(FORM))
        asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    else
        asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Operand fragment table of F in shared memory, one uint4 per lane:
// FA[v][mt][ks][lane], stage A's left operand Ar = [Fr | -Fi], 32 x 64,
// registers q = 0..3 of the m16k16 fragment (mt, ks): rows 16 mt + g + 8 (q & 1),
// columns 16 ks + 2 t + 8 (q >> 1) + {0, 1}.  Ai = [Fi | Fr] is Ar with its
// halves exchanged and one negated.
// Stage B's right operands [Fr; -Fi], [Fi; Fr] are their transposes (F is
// symmetric): the k16n8 fragment (ks, nt) is registers (nt & 1) and (nt & 1) + 2
// of FA's fragment (nt >> 1, ks).  v = 0: operand values; v = 1 (hi + lo
// forms): their remainders.
constexpr int kTcFA = 2 * 4 * 32;              // uint4 per v: [mt][ks][lane] of Ar
__host__ __device__ constexpr int tc_nv(int form) { return tc_x3(form) ? 2 : 1; }

template <int FORM>
__device__ __forceinline__ void tc_build_frags(const float2* tw32, uint4* FA, int nthreads) {
    for (int i = threadIdx.x; i < kTcFA; i += nthreads) {
        const int lane = i & 31, ks = (i >> 5) & 3, mt = (i >> 7) & 1, ri = 0;
        const int g = lane >> 2, t = lane & 3;
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int row = 16 * mt + g + 8 * (q & 1);
            float a[2];
#pragma unroll
            for (int e = 0; e < 2; e++) {
                const int col = 16 * ks + 2 * t + 8 * (q >> 1) + e;
                const float2 w = tw32[(row * (col & 31)) & 31];   // (cos, -sin)(2 pi j / 32)
                a[e] = ri == 0 ? (col < 32 ? w.x : -w.y) : (col < 32 ? w.y : w.x);
            }
            if constexpr (tc_x3(FORM)) tc_split<FORM>(a[0], a[1], hi[q], lo[q]);
            else hi[q] = tc_pack<FORM>(a[0], a[1]);
        }
        FA[i] = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        if constexpr (tc_x3(FORM)) FA[kTcFA + i] = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// Twiddle seeds of the lanes, lane-major: tws[((2 mt + hr) * 3 + k) * 32 + lane]
// for the rows c1 = 16 mt + g + 8 hr: k = 0, 1: w^{c1 (2 t + k)} (b0 = 2 t + k),
// k = 2: w^{8 c1}; the twiddle of b0 = 8 nt + 2 t + j is w^{c1 (2 t + j)} (w^{8 c1})^nt.
constexpr int kTcTws = 12 * 32;                // float2
__device__ __forceinline__ void tc_build_twiddles(const float2* __restrict__ tw1024, float2* tws, int nthreads) {
    for (int i = threadIdx.x; i < kTcTws; i += nthreads) {
        const int ln = i & 31, r = i >> 5, k = r % 3, mh = r / 3;
        const int c1 = 16 * (mh >> 1) + (ln >> 2) + 8 * (mh & 1);
        const int b0 = k == 2 ? 8 : 2 * (ln & 3) + k;
        tws[i] = __ldg(&tw1024[(c1 * b0) & 1023]);
    }
}

// 2^e as a float, e in [-120, 120]
__device__ __forceinline__ float tc_pow2(int e) { return __int_as_float((e + 127) << 23); }

__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_arrive(int id, int n) {
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// One warp: the 1024-point DFT of one column.  Input x(b) at in[base + 8 off(b)],
// output X(c) (in the input's units) at out[base + 8 off(c)], where base is the
// lane's slot of row tc_rho(g + 64 t) and off(.) the lane-independent part of
// tc_rho: the inputs b = (g + 64 t) + 8 nt + 512 s + 256 h + 32 j, the outputs
// c = (g + 64 t) + 16 mt + 8 (e >> 1) + 32 (e & 1) + 256 nt keep bits 1-2 and 6-7
// lane-fixed.  twl, FA: offset by the lane.  Only stage-B n-tiles nt0 <= nt < nt1
// (outputs c in [256 nt, 256 nt + 256)) are computed.  before_out() runs once
// before the first output is written.
// Left-operand fragments of Ar = [Fr | -Fi] for this lane, [mt][ks][q] (the
// FA layout above); those of Ai = [Fi | Fr] follow from them: (mt, ks) of Ai is
// -(mt, ks + 2) of Ar for ks < 2 and (mt, ks - 2) of Ar for ks >= 2.
struct TcFrags {
    uint32_t r[2][4][4];
    __device__ __forceinline__ void ai(int mt, int ks, uint32_t (&o)[4]) const {
#pragma unroll
        for (int q = 0; q < 4; q++) o[q] = ks < 2 ? r[mt][ks + 2][q] ^ 0x80008000u : r[mt][ks - 2][q];
    }
};
__device__ __forceinline__ void tc_load_frags(const uint4* __restrict__ FA, TcFrags& f) {
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            const uint4 v = FA[(mt * 4 + ks) * 32];
            f.r[mt][ks][0] = v.x;
            f.r[mt][ks][1] = v.y;
            f.r[mt][ks][2] = v.z;
            f.r[mt][ks][3] = v.w;
        }
}

template <int FORM, class BeforeOut>
__device__ __forceinline__ void tc_column(const float2* in, float2* out, int base, const float2* __restrict__ tws,
                                          const uint4* __restrict__ FA, const TcFrags& fr, int nt0, int nt1,
                                          BeforeOut before_out) {
    constexpr bool X3 = tc_x3(FORM);
    constexpr bool SCALE = !tc_bf(FORM);
    // stage A right operand [xr; xi] (K = (part, b1), N = b0): for k-step ks and
    // n-tile nt, register h holds b1 = 16 (ks & 1) + 2 t + 8 h + {0, 1}, b0 = 8 nt + g,
    // real parts for ks < 2, imaginary parts for ks >= 2
    uint32_t xb[4][4][2], xb_lo[X3 ? 4 : 1][4][2];
    float sc = 1.f, inv = 1.f;
    if constexpr (SCALE) {
        // a power of two that brings the column's largest part below 2^10, so
        // that stage A's outputs stay below 32 sqrt(2) 2^10 < 65504 (FP16)
        float m[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int h = 0; h < 2; h++)
#pragma unroll
                    for (int j = 0; j < 2; j++) {
                        const float2 x = in[base + 8 * (8 * nt + 512 * s + 256 * h + 32 * j)];
                        m[nt] = fmaxf(m[nt], fmaxf(fabsf(x.x), fabsf(x.y)));
                    }
        float mm = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
        int e = 0;
        if (mm > 0.f) e = min(120, max(-120, 9 - (((__float_as_int(mm) >> 23) & 0xff) - 127)));
        sc = tc_pow2(e);
        inv = tc_pow2(-e);
    }
#pragma unroll
    for (int nt = 0; nt < 4; nt++)
#pragma unroll
        for (int s = 0; s < 2; s++)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                float2 a = in[base + 8 * (8 * nt + 512 * s + 256 * h)];
                float2 b = in[base + 8 * (8 * nt + 512 * s + 256 * h + 32)];
                if constexpr (SCALE) {
                    a.x *= sc; a.y *= sc; b.x *= sc; b.y *= sc;
                }
                if constexpr (X3) {
                    tc_split<FORM>(a.x, b.x, xb[s][nt][h], xb_lo[s][nt][h]);
                    tc_split<FORM>(a.y, b.y, xb[s + 2][nt][h], xb_lo[s + 2][nt][h]);
                } else {
                    xb[s][nt][h] = tc_pack<FORM>(a.x, b.x);
                    xb[s + 2][nt][h] = tc_pack<FORM>(a.y, b.y);
                }
            }
    __syncwarp();   // every lane has read its inputs (in may be the output buffer)

    // per 16-row block mt of c1: stage A, the twiddle, then stage B for those rows
    // (stage B's left operand [Vr | Vi] holds rows c1 = 16 mt + g + 8 (q & 1),
    // b0 = 16 (ks & 1) + 8 (q >> 1) + 2 t + {0, 1} in register q of k-step ks)
#pragma unroll
    for (int mt = 0; mt < 2; mt++) {
        float dr[4][4], di[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) dr[nt][e] = di[nt][e] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
            uint32_t ai[4];
            fr.ai(mt, ks, ai);
            const uint32_t(&ar)[4] = fr.r[mt][ks];
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                tc_mma<FORM>(dr[nt], ar, xb[ks][nt][0], xb[ks][nt][1]);
                tc_mma<FORM>(di[nt], ai, xb[ks][nt][0], xb[ks][nt][1]);
            }
            if constexpr (X3) {
                // the remainders' fragments, from shared memory (Ai's from Ar's as above)
                const uint4 rl = FA[kTcFA + (mt * 4 + ks) * 32];
                const uint4 rl2 = FA[kTcFA + (mt * 4 + (ks ^ 2)) * 32];
                const uint32_t arl[4] = {rl.x, rl.y, rl.z, rl.w};
                const uint32_t neg = ks < 2 ? 0x80008000u : 0u;
                const uint32_t ail[4] = {rl2.x ^ neg, rl2.y ^ neg, rl2.z ^ neg, rl2.w ^ neg};
#pragma unroll
                for (int nt = 0; nt < 4; nt++) {
                    tc_mma<FORM>(dr[nt], ar, xb_lo[ks][nt][0], xb_lo[ks][nt][1]);
                    tc_mma<FORM>(dr[nt], arl, xb[ks][nt][0], xb[ks][nt][1]);
                    tc_mma<FORM>(di[nt], ai, xb_lo[ks][nt][0], xb_lo[ks][nt][1]);
                    tc_mma<FORM>(di[nt], ail, xb[ks][nt][0], xb[ks][nt][1]);
                }
            }
        }
        // V = U w^{b0 c1}; accumulator e of tile (mt, nt): c1 = 16 mt + g + 8 (e >> 1), b0 = 8 nt + 2 t + (e & 1);
        // the twiddles of n-tile nt: seeds times (w^{8 c1})^nt
        float2 T[4], S[2];
#pragma unroll
        for (int e = 0; e < 4; e++) T[e] = tws[((2 * mt + (e >> 1)) * 3 + (e & 1)) * 32];
#pragma unroll
        for (int hr = 0; hr < 2; hr++) S[hr] = tws[((2 * mt + hr) * 3 + 2) * 32];
        uint32_t va[4][4], va_lo[X3 ? 4 : 1][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            float vr[4], vi[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (nt > 0) {
                    const float2 st = S[e >> 1];
                    T[e] = make_float2(fmaf(T[e].x, st.x, -T[e].y * st.y), fmaf(T[e].x, st.y, T[e].y * st.x));
                }
                vr[e] = fmaf(dr[nt][e], T[e].x, -di[nt][e] * T[e].y);
                vi[e] = fmaf(dr[nt][e], T[e].y, di[nt][e] * T[e].x);
            }
            // n-tile nt feeds k-steps nt >> 1 (real) and 2 + (nt >> 1) (imaginary),
            // registers 2 (nt & 1) + {0, 1} (rows g, g + 8)
            const int ks = nt >> 1, q = 2 * (nt & 1);
#pragma unroll
            for (int r = 0; r < 2; r++) {
                if constexpr (X3) {
                    tc_split<FORM>(vr[2 * r], vr[2 * r + 1], va[ks][q + r], va_lo[ks][q + r]);
                    tc_split<FORM>(vi[2 * r], vi[2 * r + 1], va[ks + 2][q + r], va_lo[ks + 2][q + r]);
                } else {
                    va[ks][q + r] = tc_pack<FORM>(vr[2 * r], vr[2 * r + 1]);
                    va[ks + 2][q + r] = tc_pack<FORM>(vi[2 * r], vi[2 * r + 1]);
                }
            }
        }
        if (mt == 0) before_out();
        // stage B for these rows, the n-tiles side by side (independent accumulators)
        float xr[4][4], xi[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++)
#pragma unroll
            for (int e = 0; e < 4; e++) xr[nt][e] = xi[nt][e] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ks++) {
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                if (nt < nt0 || nt >= nt1) continue;
                const int m2 = nt >> 1, q0 = nt & 1;
                uint32_t ai[4];
                fr.ai(m2, ks, ai);
                const uint32_t r0 = fr.r[m2][ks][q0], r1 = fr.r[m2][ks][q0 + 2];
                const uint32_t i0 = ai[q0], i1 = ai[q0 + 2];
                tc_mma<FORM>(xr[nt], va[ks], r0, r1);
                tc_mma<FORM>(xi[nt], va[ks], i0, i1);
                if constexpr (X3) {
                    const uint4 rl = FA[kTcFA + (m2 * 4 + ks) * 32];
                    const uint4 rl2 = FA[kTcFA + (m2 * 4 + (ks ^ 2)) * 32];
                    const uint32_t neg = ks < 2 ? 0x80008000u : 0u;
                    tc_mma<FORM>(xr[nt], va_lo[ks], r0, r1);
                    tc_mma<FORM>(xr[nt], va[ks], q0 ? rl.y : rl.x, q0 ? rl.w : rl.z);
                    tc_mma<FORM>(xi[nt], va_lo[ks], i0, i1);
                    tc_mma<FORM>(xi[nt], va[ks], (q0 ? rl2.y : rl2.x) ^ neg, (q0 ? rl2.w : rl2.z) ^ neg);
                }
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            if (nt < nt0 || nt >= nt1) continue;
#pragma unroll
            for (int e = 0; e < 4; e++)
                out[base + 8 * (16 * mt + 8 * (e >> 1) + 32 * (e & 1) + 256 * nt)] =
                    make_float2(xr[nt][e] * inv, xi[nt][e] * inv);
        }
    }
}

// n-tiles of stage B that hold outputs kept in W for the columns d0 .. d0 + 7
__device__ __forceinline__ void tc_nt_range(const Params& p, bool crop, int d0, int& nt0, int& nt1) {
    nt0 = 0;
    nt1 = 4;
    if (!crop) return;
    const long long A = p.A, off = p.out_off, len = p.out_len;
    const long long clo = (off - (d0 + kTcCols - 1) + A - 1) / A;   // may be <= 0
    const long long chi = (off + len - 1 - d0) / A;
    nt0 = (int)(clo > 0 ? (clo / 256 < 4 ? clo / 256 : 4) : 0);
    nt1 = (int)(chi < 0 ? 0 : (chi / 256 + 1 < 4 ? chi / 256 + 1 : 4));
}

// W rows from a staging tile (rows i = tc_rho(c) for outputs c; i = c with
// RHO = false, the FP32 tile pipeline's natural order): thread k of
// NTHR (a multiple of 128) stores columns 2 (k & 3), + 1 of the rows
// i = r0 + R m, r0 = k >> 2, R = NTHR / 4, m < 4096 / NTHR.  tc_rho permutes
// bits, so c = tc_rho(r0) + tc_rho(R m) and the slot of row i is the slot of
// r0 plus 8 R m: every address is a per-thread base plus a constant.
// Accumulates |W|^2 into pw0 (Morlet, GDW row a) and pw1 (GDW row b).
template <int NTHR, bool CROP, bool RHO = true>
__device__ __forceinline__ void tc_store_tile(const float2* buf, const Params& p, const Job& J, int d0, int k,
                                              float& pw0, float& pw1) {
    constexpr int R = NTHR / 4, NM = 1024 / R, B = 8;   // rows per thread, loads in flight
    const int A = p.A;
    const int off = CROP ? (int)p.out_off : 0;
    const unsigned len = (unsigned)p.out_len;
    const int wc = k & 3, r0 = k >> 2;
    const float2* src = buf + tc_slot(r0, 2 * wc);
    const int c0 = RHO ? tc_rho(r0) : r0;
    const int n0 = d0 + 2 * wc + A * c0;          // output index of row r0's first column
    if (!wav_real(p.wavelet)) {
        float2* row = (float2*)p.W + (int64_t)J.g[0].row * p.out_len + (n0 - off);
        const bool al = !((uintptr_t)row & 15);
#pragma unroll
        for (int m0 = 0; m0 < NM; m0 += B) {
            float4 v[B];
#pragma unroll
            for (int b = 0; b < B; b++) v[b] = *reinterpret_cast<const float4*>(src + 8 * R * (m0 + b));
#pragma unroll
            for (int b = 0; b < B; b++) {
                const int dc = RHO ? tc_rho(R * (m0 + b)) : R * (m0 + b);
                float2* q2 = row + (int64_t)A * dc;
                bool k0 = true, k1 = true;
                if (CROP) {
                    const int n = n0 + A * dc;
                    k0 = (unsigned)(n - off) < len;
                    k1 = (unsigned)(n + 1 - off) < len;
                }
                if (k0 && k1 && al) {
                    __stcs(reinterpret_cast<float4*>(q2), v[b]);
                } else {
                    if (k0) __stcs(q2, make_float2(v[b].x, v[b].y));
                    if (k1) __stcs(q2 + 1, make_float2(v[b].z, v[b].w));
                }
                if (k0) pw0 = fmaf(v[b].x, v[b].x, fmaf(v[b].y, v[b].y, pw0));
                if (k1) pw0 = fmaf(v[b].z, v[b].z, fmaf(v[b].w, v[b].w, pw0));
            }
        }
    } else {
        float* ra = (float*)p.W + (int64_t)J.g[0].row * p.out_len + (n0 - off);
        float* rb = J.g[1].row >= 0 ? (float*)p.W + (int64_t)J.g[1].row * p.out_len + (n0 - off) : nullptr;
        const bool ala = !((uintptr_t)ra & 7), alb = rb && !((uintptr_t)rb & 7);
#pragma unroll
        for (int m0 = 0; m0 < NM; m0 += B) {
            float4 v[B];
#pragma unroll
            for (int b = 0; b < B; b++) v[b] = *reinterpret_cast<const float4*>(src + 8 * R * (m0 + b));
#pragma unroll
            for (int b = 0; b < B; b++) {
                const int dc = RHO ? tc_rho(R * (m0 + b)) : R * (m0 + b);
                bool k0 = true, k1 = true;
                if (CROP) {
                    const int n = n0 + A * dc;
                    k0 = (unsigned)(n - off) < len;
                    k1 = (unsigned)(n + 1 - off) < len;
                }
                float* qa = ra + (int64_t)A * dc;
                if (k0 && k1 && ala) __stcs(reinterpret_cast<float2*>(qa), make_float2(v[b].x, v[b].z));
                else {
                    if (k0) __stcs(qa, v[b].x);
                    if (k1) __stcs(qa + 1, v[b].z);
                }
                if (k0) pw0 = fmaf(v[b].x, v[b].x, pw0);
                if (k1) pw0 = fmaf(v[b].z, v[b].z, pw0);
                if (rb) {
                    float* qb = rb + (int64_t)A * dc;
                    if (k0 && k1 && alb) __stcs(reinterpret_cast<float2*>(qb), make_float2(v[b].y, v[b].w));
                    else {
                        if (k0) __stcs(qb, v[b].y);
                        if (k1) __stcs(qb + 1, v[b].w);
                    }
                    if (k0) pw1 = fmaf(v[b].y, v[b].y, pw1);
                    if (k1) pw1 = fmaf(v[b].w, v[b].w, pw1);
                }
            }
        }
    }
}

// the lane's slot of row tc_rho(g + 64 t) = (g & 1) + 2 t + 64 (g >> 1) in column w
__device__ __forceinline__ int tc_col_base(int lane, int w) {
    const int g = lane >> 2, t = lane & 3;
    return tc_slot((g & 1) + 2 * t + 64 * (g >> 1), w);
}

// dynamic shared memory of the two kernels: tile buffers (1024-byte aligned;
// 1 KiB of slack for the alignment), the twiddles and the F fragments
__host__ __device__ constexpr size_t tc_frag_bytes(int form) { return (size_t)tc_nv(form) * kTcFA * 16; }
__host__ __device__ constexpr size_t tc_smem_bytes(int form) {     // k_wide2_tc_g: one buffer
    return 1024 + (size_t)kTcTile * sizeof(float2) + kTcTws * sizeof(float2) + tc_frag_bytes(form);
}
// store warps of k_wide2_tma: 4 beside the 8 compute warps for the single-product
// forms; none for the hi + lo forms, whose compute warps need more registers than
// 12 warps leave (they store each tile themselves, in place)
__host__ __device__ constexpr int tma_store_warps(int form) { return tc_x3(form) ? 0 : 4; }
__host__ __device__ constexpr size_t tma_smem_bytes(int form) {    // k_wide2_tma: 3 (2 without store warps) buffers
    return 1024 + (size_t)(tma_store_warps(form) ? 3 : 2) * kTcTile * sizeof(float2) + kTcTws * sizeof(float2) +
           tc_frag_bytes(form);
}
__host__ __device__ constexpr int tma_threads(int form) { return 32 * (kTcCols + tma_store_warps(form)); }

__device__ __forceinline__ float2* tc_align1024(void* p) {
    return reinterpret_cast<float2*>(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// ---------------------------------------------------------------- grouped form

// grid (A / (8 D), jobs in batch), 256 threads: D = p.D tiles of 8 columns;
// the compute warps also copy (cp.async) and store
template <int FORM, bool CROP>
__device__ __forceinline__ void wide2_tc_body(const Params& p, const Cta c) {
    extern __shared__ unsigned char smem_raw[];
    float2* buf = tc_align1024(smem_raw);
    float2* twl = buf + kTcTile;
    uint4* FA = reinterpret_cast<uint4*>(twl + kTcTws);
    __shared__ double red[2 * (kTcThreads / 32)];
    __shared__ Job sJ;
    __shared__ float2 tw32[32];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (tid == 0) sJ = p.jobs[p.job0 + c.y];
    if (tid < 32) tw32[tid] = __ldg(&p.tw_tab[32 + tid]);
    tc_build_twiddles(p.tw_tab + 1024, twl, kTcThreads);
    __syncthreads();
    tc_build_frags<FORM>(tw32, FA, kTcThreads);
    __syncthreads();
    TcFrags fr;
    tc_load_frags(FA + lane, fr);
    const Job& J = sJ;
    const int A = p.A;
    const float2* Yj = p.Y + (int64_t)c.y * p.M;
    const int tile0 = c.x * p.D;
    const int ntile = min(p.D, A / kTcCols - tile0);
    const int col_base = tc_col_base(lane, w);
    const int wc = tid & 3, rr = tid >> 2;
    const int lslot = tc_slot(rr, 2 * wc);       // rows 64 it + rr: + 512 it
    constexpr int kStore = tma_store_warps(FORM) ? 32 * tma_store_warps(FORM) : kTcThreads;
    float pw0 = 0.f, pw1 = 0.f;
#pragma unroll 1
    for (int q = 0; q < ntile; q++) {
        const int d0 = (tile0 + q) * kTcCols;
        if (q > 0) __syncthreads();              // every thread is done with the previous tile
        const float2* src = Yj + (int64_t)rr * A + d0 + 2 * wc;
#pragma unroll
        for (int it = 0; it < 1024 / 64; it++) cp_async16(buf + lslot + 512 * it, src + (int64_t)(64 * it) * A);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        int nt0, nt1;
        tc_nt_range(p, CROP, d0, nt0, nt1);
        tc_column<FORM>(buf, buf, col_base, twl + lane, FA + lane, fr, nt0, nt1, [] {});
        __syncthreads();
        // as many storing threads as k_wide2_tma has (the same rows per thread, so
        // the power sums are added in the same order and equal bit for bit)
        if (tid < kStore) tc_store_tile<kStore, CROP>(buf, p, J, d0, tid, pw0, pw1);
    }
    struct { float pw0, pw1; } o{pw0, pw1};
    write_partials<kTcThreads>(p, J, o, c.x, red);
}

template <int FORM, bool CROP>
__global__ void __launch_bounds__(kTcThreads, 1) k_wide2_tc_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    wide2_tc_body<FORM, CROP>(p, c);
}

// ---------------------------------------------------------------- TMA form

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 4 TMA loads of 256 rows x 8 columns: the tile Y[slab z][0..1023][d0 .. d0 + 7]
__device__ __forceinline__ void tma_load_tile(const CUtensorMap* map, float2* dst, uint64_t* bar, int d0, int z) {
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kTcTile * 8) : "memory");
#pragma unroll
    for (int k = 0; k < 4; k++)
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
            "[%5];" ::"r"(smem_u32(dst + 2048 * k)),
            "l"(map), "r"(2 * d0), "r"(256 * k), "r"(z), "r"(b)
            : "memory");
}

// waits for phase `parity` of the mbarrier; gives up (returns false) after
// 2^31 SM clock cycles, about a second
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t b = smem_u32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred P; mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2; selp.u32 %0, 1, 0, P; }"
            : "=r"(done)
            : "r"(b), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1ll << 31)) return false;
    }
}

// grid (A / (8 D), jobs in launch), tma_threads(FORM) threads: warps 0..7 compute.
// The tile of step q is loaded by TMA into buffer q % NB one step ahead; each
// compute warp writes its outputs in place and arrives on named barrier
// 1 + q % 3.  With store warps (NS > 0, NB = 3 buffers) those sync on that
// barrier, store the tile and arrive on the mbarrier empty[q % 3]; the TMA of
// step q + 1 (into the buffer of step q - 2) waits for it.  The compute warps
// never wait for each other or for the stores of the current step, so they
// drift apart and overlap their phases.  Without store warps (NS = 0, the hi + lo
// forms, NB = 2) the compute warps store each tile themselves after a CTA barrier.
template <int FORM, bool CROP>
__device__ __forceinline__ void wide2_tma_body(const Params& p, const CUtensorMap* ymap, const Cta c) {
    constexpr int NT = tma_threads(FORM), NC = 32 * kTcCols, NS = NT - NC;
    constexpr int NB = NS ? 3 : 2;
    extern __shared__ unsigned char smem_raw[];
    float2* ibuf = tc_align1024(smem_raw);
    float2* twl = ibuf + NB * kTcTile;
    uint4* FA = reinterpret_cast<uint4*>(twl + kTcTws);
    __shared__ double red[2 * (NT / 32)];
    __shared__ Job sJ;
    __shared__ float2 tw32[32];
    __shared__ __align__(8) uint64_t full[3], empty[3];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        sJ = p.jobs[p.job0 + c.y];
        for (int b = 0; b < 3; b++) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[b])), "r"(NS / 32 > 0 ? NS / 32 : 1)
                         : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 32) tw32[tid] = __ldg(&p.tw_tab[32 + tid]);
    tc_build_twiddles(p.tw_tab + 1024, twl, NT);
    __syncthreads();
    tc_build_frags<FORM>(tw32, FA, NT);
    const int A = p.A;
    const int z = p.yz0 + c.y;
    const int tile0 = c.x * p.D;
    const int ntile = min(p.D, A / kTcCols - tile0);
    if (tid == 0 && ntile > 0) tma_load_tile(ymap, ibuf, &full[0], tile0 * kTcCols, z);
    __syncthreads();
    const Job& J = sJ;
    float pw0 = 0.f, pw1 = 0.f;
    bool ok = true;
    if (w < kTcCols) {
        const int col_base = tc_col_base(lane, w);
        TcFrags fr;
        tc_load_frags(FA + lane, fr);
#pragma unroll 1
        for (int q = 0; q < ntile; q++) {
            const int d0 = (tile0 + q) * kTcCols;
            float2* buf = ibuf + (q % NB) * kTcTile;
            if (!mbar_wait(&full[q % NB], (q / NB) & 1)) ok = false;
            if constexpr (NS == 0) {
                // every thread is past step q - 1 and its stores (its in-place writes ordered
                // before the next copy into that buffer)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncthreads();
            }
            if (tid == 0 && q + 1 < ntile) {
                // step q + 1 goes into the buffer of step q + 1 - NB, once that tile is stored
                if (NS && q + 1 >= NB && !mbar_wait(&empty[(q + 1) % NB], ((q + 1 - NB) / NB) & 1)) ok = false;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                tma_load_tile(ymap, ibuf + ((q + 1) % NB) * kTcTile, &full[(q + 1) % NB], d0 + kTcCols, z);
            }
            int nt0, nt1;
            tc_nt_range(p, CROP, d0, nt0, nt1);
            tc_column<FORM>(buf, buf, col_base, twl + lane, FA + lane, fr, nt0, nt1, [] {});
            if constexpr (NS == 0) {
                __syncthreads();
                tc_store_tile<NT, CROP>(buf, p, J, d0, tid, pw0, pw1);
            } else {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // in-place writes before later copies
                named_arrive(1 + q % 3, NT);     // step q's outputs are in its buffer
            }
        }
    } else {
#pragma unroll 1
        for (int q = 0; q < ntile; q++) {
            named_sync(1 + q % 3, NT);
            tc_store_tile<(NS > 0 ? NS : 128), CROP>(ibuf + (q % NB) * kTcTile, p, J, (tile0 + q) * kTcCols, tid - NC,
                                                     pw0, pw1);
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[q % NB])) : "memory");
        }
    }
    if (!ok) {
        // a copy may still be in flight: wait for it (bounded) before the CTA exits
        if (ntile > 0) mbar_wait(&full[(ntile - 1) % NB], ((ntile - 1) / NB) & 1);
        if (p.err) *(volatile int32_t*)p.err = 1;
    }
    struct { float pw0, pw1; } o{pw0, pw1};
    write_partials<NT>(p, J, o, c.x, red);
}

template <int FORM, bool CROP>
__global__ void __launch_bounds__(tma_threads(FORM), 1)
    k_wide2_tma(Params p, const __grid_constant__ CUtensorMap ymap) {
    wide2_tma_body<FORM, CROP>(p, &ymap, cta_plain());
}

}  // namespace cwtk
