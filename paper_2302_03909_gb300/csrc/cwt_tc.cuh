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
// A CTA of 8 warps takes 8 consecutive columns: the tile Y[0..1023][d0..d0+7]
// is copied into shared memory with cp.async (the next tile's copy overlaps
// the current tile's work), each warp reads its column in the MMA operand
// pattern, writes its outputs back in place, and the CTA stores W rows with
// 16-byte vector stores.
#pragma once

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


// float2 index of element (row r, column w < 8) in a tile buffer.  The 16-byte
// pairs of columns of a row are permuted by bits 1 and 6 of r, so that the
// operand reads of a warp (rows g + 64 t + const over its lanes) and its
// in-place output writes hit at most two lanes per bank pair.  Every access
// pattern below keeps bits 1 and 6 of r fixed per thread, so its index is a
// per-thread base plus a compile-time offset of 8 (r - r_thread).
__device__ __forceinline__ int tc_slot(int r, int w) {
    const int sig = ((r >> 1) & 1) | (((r >> 6) & 1) << 1);
    return (r << 3) + ((((w >> 1) ^ sig)) << 1) + (w & 1);
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

// Copies the tile Y[0..1023][d0 .. d0 + 7] into buf: thread tid moves rows
// r = 64 it + (tid >> 2), columns 2 wc, 2 wc + 1 (wc = tid & 3), 16 bytes per
// step; slot0 / slot1 are its slots of even / odd steps in row 64 it.
__device__ __forceinline__ void tc_load_tile(float2* buf, const float2* __restrict__ src, int64_t A, int slot0,
                                             int slot1) {
#pragma unroll
    for (int it = 0; it < 1024 / 64; it++)
        cp_async16(buf + (it & 1 ? slot1 : slot0) + 512 * it, src + (int64_t)(64 * it) * A);
    cp_async_commit();
}

// Operand fragment tables of F, in shared memory, one entry per lane:
//   FA[v][ri][mt][ks][lane] (uint4): stage A's left operand Ar = [Fr | -Fi]
//     (ri = 0) or Ai = [Fi | Fr] (ri = 1), 32 x 64, registers q = 0..3 of the
//     m16k16 fragment (mt, ks): rows 16 mt + g + 8 (q & 1), columns
//     16 ks + 2 t + 8 (q >> 1) + {0, 1};
//   FB[v][ri][m2][ks][q0][lane] (uint2): stage B's right operand, the
//     transpose [Fr; -Fi] / [Fi; Fr] (F is symmetric), k16n8 fragment (ks,
//     nt = 2 m2 + q0): the registers q0 and q0 + 2 of FA's fragment (m2, ks).
// v = 0: the operand values, v = 1 (hi + lo forms): their remainders.
constexpr int kTcFA = 2 * 2 * 4 * 32;          // uint4 per v
constexpr int kTcFB = 2 * 2 * 4 * 2 * 32;      // uint2 per v
template <int FORM>
__host__ __device__ constexpr int tc_nbuf() { return tc_x3(FORM) ? 2 : 1; }
// dynamic shared memory of the tensor-core pass 2
__host__ __device__ constexpr size_t tc_smem_bytes(int form) {
    return (size_t)(tc_x3(form) ? 2 : 1) * kTcTile * sizeof(float2) + 1024 * sizeof(float2) +
           (size_t)(tc_x3(form) ? 2 : 1) * (kTcFA * 16 + kTcFB * 8);
}

template <int FORM>
__device__ __forceinline__ void tc_build_frags(const float2* tw32, uint4* FA, uint2* FB) {
    constexpr int NV = tc_x3(FORM) ? 2 : 1;
    for (int i = threadIdx.x; i < kTcFA; i += kTcThreads) {
        const int lane = i & 31, ks = (i >> 5) & 3, mt = (i >> 7) & 1, ri = i >> 8;
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
#pragma unroll
        for (int v = 0; v < NV; v++) {
            const uint32_t* r = v ? lo : hi;
            FA[v * kTcFA + i] = make_uint4(r[0], r[1], r[2], r[3]);
            // FA fragment (m2 = mt, ks) serves FB (ks, nt = 2 mt + q0), q0 = 0, 1
#pragma unroll
            for (int q0 = 0; q0 < 2; q0++)
                FB[v * kTcFB + ((((ri * 2 + mt) * 4 + ks) * 2 + q0) * 32 + lane)] = make_uint2(r[q0], r[q0 + 2]);
        }
    }
}

// 2^e as a float, e in [-120, 120]
__device__ __forceinline__ float tc_pow2(int e) { return __int_as_float((e + 127) << 23); }

// One warp: the 1024-point DFT of column w of the tile in buf, outputs X(c)
// written back into the column's slots (in the input's units).  base: this
// lane's slot of row g + 64 t of column w; twl: the lane's 32 twiddles,
// [(16 mt + 4 nt + e) * 32] apart; FA, FB offset by the lane.
template <int FORM>
__device__ __forceinline__ void tc_column(float2* buf, int base, const float2* __restrict__ twl,
                                          const uint4* __restrict__ FA, const uint2* __restrict__ FB, int nt0,
                                          int nt1) {
    constexpr bool X3 = tc_x3(FORM);
    constexpr bool SCALE = !tc_bf(FORM);
    // stage A right operand [xr; xi] (K = (part, b1), N = b0): for k-step ks
    // and n-tile nt, register h holds b1 = 16 (ks & 1) + 2 t + 8 h + {0, 1},
    // b0 = 8 nt + g, real parts for ks < 2, imaginary parts for ks >= 2:
    // x(b) with b = (g + 64 t) + 8 nt + 512 s + 256 h + 32 j
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
                        const float2 x = buf[base + 8 * (8 * nt + 512 * s + 256 * h + 32 * j)];
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
                float2 a = buf[base + 8 * (8 * nt + 512 * s + 256 * h)];
                float2 b = buf[base + 8 * (8 * nt + 512 * s + 256 * h + 32)];
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
    __syncwarp();   // every lane has read its inputs: the column's slots may be overwritten

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
            const uint4 r4 = FA[((0 * 2 + mt) * 4 + ks) * 32], i4 = FA[((1 * 2 + mt) * 4 + ks) * 32];
            const uint32_t ar[4] = {r4.x, r4.y, r4.z, r4.w}, ai[4] = {i4.x, i4.y, i4.z, i4.w};
#pragma unroll
            for (int nt = 0; nt < 4; nt++) {
                tc_mma<FORM>(dr[nt], ar, xb[ks][nt][0], xb[ks][nt][1]);
                tc_mma<FORM>(di[nt], ai, xb[ks][nt][0], xb[ks][nt][1]);
            }
            if constexpr (X3) {
                const uint4 rl = FA[kTcFA + ((0 * 2 + mt) * 4 + ks) * 32], il = FA[kTcFA + ((1 * 2 + mt) * 4 + ks) * 32];
                const uint32_t arl[4] = {rl.x, rl.y, rl.z, rl.w}, ail[4] = {il.x, il.y, il.z, il.w};
#pragma unroll
                for (int nt = 0; nt < 4; nt++) {
                    tc_mma<FORM>(dr[nt], ar, xb_lo[ks][nt][0], xb_lo[ks][nt][1]);
                    tc_mma<FORM>(dr[nt], arl, xb[ks][nt][0], xb[ks][nt][1]);
                    tc_mma<FORM>(di[nt], ai, xb_lo[ks][nt][0], xb_lo[ks][nt][1]);
                    tc_mma<FORM>(di[nt], ail, xb[ks][nt][0], xb[ks][nt][1]);
                }
            }
        }
        // V = U w^{b0 c1}; accumulator e of tile (mt, nt): c1 = 16 mt + g + 8 (e >> 1), b0 = 8 nt + 2 t + (e & 1)
        uint32_t va[4][4], va_lo[X3 ? 4 : 1][4];
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            float vr[4], vi[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float2 T = twl[(16 * mt + 4 * nt + e) * 32];
                vr[e] = fmaf(dr[nt][e], T.x, -di[nt][e] * T.y);
                vi[e] = fmaf(dr[nt][e], T.y, di[nt][e] * T.x);
            }
            // n-tile nt feeds k-steps nt >> 1 (real) and 2 + (nt >> 1) (imaginary), registers
            // 2 (nt & 1) + {0, 1} (rows g, g + 8)
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
        // stage B for these rows; only n-tiles nt0 <= nt < nt1 hold kept outputs
#pragma unroll
        for (int nt = 0; nt < 4; nt++) {
            if (nt < nt0 || nt >= nt1) continue;
            float xr[4] = {0.f, 0.f, 0.f, 0.f}, xi[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int ks = 0; ks < 4; ks++) {
                const uint2 br = FB[((((0 * 2 + (nt >> 1)) * 4 + ks) * 2 + (nt & 1)) * 32)];
                const uint2 bi = FB[((((1 * 2 + (nt >> 1)) * 4 + ks) * 2 + (nt & 1)) * 32)];
                tc_mma<FORM>(xr, va[ks], br.x, br.y);
                tc_mma<FORM>(xi, va[ks], bi.x, bi.y);
                if constexpr (X3) {
                    const uint2 brl = FB[kTcFB + ((((0 * 2 + (nt >> 1)) * 4 + ks) * 2 + (nt & 1)) * 32)];
                    const uint2 bil = FB[kTcFB + ((((1 * 2 + (nt >> 1)) * 4 + ks) * 2 + (nt & 1)) * 32)];
                    tc_mma<FORM>(xr, va_lo[ks], br.x, br.y);
                    tc_mma<FORM>(xr, va[ks], brl.x, brl.y);
                    tc_mma<FORM>(xi, va_lo[ks], bi.x, bi.y);
                    tc_mma<FORM>(xi, va[ks], bil.x, bil.y);
                }
            }
            // accumulator e: c = 16 mt + g + 8 (e >> 1) + 32 (8 nt + 2 t + (e & 1))
            //              = (g + 64 t) + 16 mt + 8 (e >> 1) + 256 nt + 32 (e & 1)
#pragma unroll
            for (int e = 0; e < 4; e++)
                buf[base + 8 * (16 * mt + 8 * (e >> 1) + 256 * nt + 32 * (e & 1))] =
                    make_float2(xr[e] * inv, xi[e] * inv);
        }
    }
}

// grid (A / (8 D), jobs in batch): D = p.D tiles of 8 columns d.  The
// single-product forms keep two CTAs per SM (one tile buffer each); the hi +
// lo forms, with twice the operand registers, one CTA per SM with two tile
// buffers (the next tile's copy overlapping the current tile's work).
template <int FORM, bool CROP>
__device__ __forceinline__ void wide2_tc_body(const Params& p, const Cta c) {
    constexpr int NBUF = tc_nbuf<FORM>();
    extern __shared__ __align__(16) float2 smem[];
    float2* twl = smem + NBUF * kTcTile;
    uint4* FA = reinterpret_cast<uint4*>(twl + 1024);
    uint2* FB = reinterpret_cast<uint2*>(FA + (tc_x3(FORM) ? 2 : 1) * kTcFA);
    __shared__ double red[2 * (kTcThreads / 32)];
    __shared__ Job sJ;
    __shared__ float2 tw32[32];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    if (tid == 0) sJ = p.jobs[p.job0 + c.y];
    if (tid < 32) tw32[tid] = __ldg(&p.tw_tab[32 + tid]);
    // the lanes' twiddles w^{b0 c1} in the order they are used, lane-major
    for (int i = tid; i < 1024; i += kTcThreads) {
        const int ln = i & 31, r = i >> 5;
        const int c1 = 16 * (r >> 4) + (ln >> 2) + 8 * ((r & 3) >> 1);
        const int b0 = 8 * ((r >> 2) & 3) + 2 * (ln & 3) + (r & 1);
        twl[i] = __ldg(&p.tw_tab[1024 + ((c1 * b0) & 1023)]);
    }
    __syncthreads();
    tc_build_frags<FORM>(tw32, FA, FB);
    __syncthreads();
    const Job& J = sJ;
    const int A = p.A;
    const float2* Yj = p.Y + (int64_t)c.y * p.M;
    const int tile0 = c.x * p.D;
    const int ntile = min(p.D, A / kTcCols - tile0);
    const int off = CROP ? (int)p.out_off : 0;
    const unsigned len = (unsigned)p.out_len;
    const bool real = wav_real(p.wavelet);
    float* r0 = real ? (float*)p.W + (int64_t)J.g[0].row * p.out_len : nullptr;
    float* r1 = (real && J.g[1].row >= 0) ? (float*)p.W + (int64_t)J.g[1].row * p.out_len : nullptr;
    float2* rc = real ? nullptr : (float2*)p.W + (int64_t)J.g[0].row * p.out_len;
    // this warp's slot of row g + 64 t in its column w (operand reads, in-place outputs)
    const int col_base = tc_slot(lane >> 2 | (lane & 3) << 6, w);
    // this thread's slots for the copies and the row stores: rows 64 it + (tid >> 2),
    // columns 2 wc, 2 wc + 1; even / odd it
    const int wc = tid & 3, rr = tid >> 2;
    const int slot0 = tc_slot(rr, 2 * wc), slot1 = tc_slot(rr + 64, 2 * wc) - 512;
    float pw0 = 0.f, pw1 = 0.f;
    if (NBUF == 2 && ntile > 0) tc_load_tile(smem, Yj + (int64_t)rr * A + tile0 * kTcCols + 2 * wc, A, slot0, slot1);
#pragma unroll 1
    for (int q = 0; q < ntile; q++) {
        float2* buf = smem + (NBUF == 2 ? (q & 1) * kTcTile : 0);
        const int d0 = (tile0 + q) * kTcCols;
        if (NBUF == 1) {
            if (q > 0) __syncthreads();          // every thread is done with the previous tile
            tc_load_tile(buf, Yj + (int64_t)rr * A + d0 + 2 * wc, A, slot0, slot1);
        }
        cp_async_wait_all();
        __syncthreads();                         // the tile is in (two buffers: the other one is free)
        if (NBUF == 2 && q + 1 < ntile)
            tc_load_tile(smem + ((q + 1) & 1) * kTcTile, Yj + (int64_t)rr * A + d0 + kTcCols + 2 * wc, A, slot0,
                         slot1);
        // n-tiles of stage B that hold kept outputs (c in [256 nt, 256 nt + 256))
        int nt0 = 0, nt1 = 4;
        if (CROP) {
            const long long clo = ((long long)off - (d0 + kTcCols - 1) + A - 1) / A;   // may be <= 0
            const long long chi = ((long long)off + (long long)len - 1 - d0) / A;
            nt0 = (int)(clo > 0 ? (clo / 256 < 4 ? clo / 256 : 4) : 0);
            nt1 = (int)(chi < 0 ? 0 : (chi / 256 + 1 < 4 ? chi / 256 + 1 : 4));
        }
        tc_column<FORM>(buf, col_base, twl + lane, FA + lane, FB + lane, nt0, nt1);
        __syncthreads();
        // W rows: X(c) of columns d0 + 2 wc, + 1 at n = d + A c, c = 64 it + rr
        const int n0 = d0 + 2 * wc + A * rr;
        const int64_t step = (int64_t)64 * A;
        if (rc) {
            float2* dst = rc + (n0 - off);
            const bool al = !((uintptr_t)dst & 15);
#pragma unroll 4
            for (int it = 0; it < 16; it++) {
                const float4 v = *reinterpret_cast<const float4*>(buf + (it & 1 ? slot1 : slot0) + 512 * it);
                float2* q2 = dst + step * it;
                bool k0 = true, k1 = true;
                if (CROP) {
                    const int n = n0 + 64 * A * it;
                    k0 = (unsigned)(n - off) < len;
                    k1 = (unsigned)(n + 1 - off) < len;
                }
                if (k0 && k1 && al) {
                    __stcs(reinterpret_cast<float4*>(q2), v);
                } else {
                    if (k0) __stcs(q2, make_float2(v.x, v.y));
                    if (k1) __stcs(q2 + 1, make_float2(v.z, v.w));
                }
                if (k0) pw0 = fmaf(v.x, v.x, fmaf(v.y, v.y, pw0));
                if (k1) pw0 = fmaf(v.z, v.z, fmaf(v.w, v.w, pw0));
            }
        } else {
            float* da = r0 + (n0 - off);
            float* db = r1 ? r1 + (n0 - off) : nullptr;
            const bool ala = !((uintptr_t)da & 7), alb = db && !((uintptr_t)db & 7);
#pragma unroll 4
            for (int it = 0; it < 16; it++) {
                const float4 v = *reinterpret_cast<const float4*>(buf + (it & 1 ? slot1 : slot0) + 512 * it);
                bool k0 = true, k1 = true;
                if (CROP) {
                    const int n = n0 + 64 * A * it;
                    k0 = (unsigned)(n - off) < len;
                    k1 = (unsigned)(n + 1 - off) < len;
                }
                float* qa = da + step * it;
                if (k0 && k1 && ala) __stcs(reinterpret_cast<float2*>(qa), make_float2(v.x, v.z));
                else {
                    if (k0) __stcs(qa, v.x);
                    if (k1) __stcs(qa + 1, v.z);
                }
                if (k0) pw0 = fmaf(v.x, v.x, pw0);
                if (k1) pw0 = fmaf(v.z, v.z, pw0);
                if (db) {
                    float* qb = db + step * it;
                    if (k0 && k1 && alb) __stcs(reinterpret_cast<float2*>(qb), make_float2(v.y, v.w));
                    else {
                        if (k0) __stcs(qb, v.y);
                        if (k1) __stcs(qb + 1, v.w);
                    }
                    if (k0) pw1 = fmaf(v.y, v.y, pw1);
                    if (k1) pw1 = fmaf(v.w, v.w, pw1);
                }
            }
        }
    }
    struct { float pw0, pw1; } o{pw0, pw1};
    write_partials<kTcThreads>(p, J, o, c.x, red);
}

template <int FORM, bool CROP>
__global__ void __launch_bounds__(kTcThreads, 3 - tc_nbuf<FORM>()) k_wide2_tc(Params p) {
    wide2_tc_body<FORM, CROP>(p, cta_plain());
}
template <int FORM, bool CROP>
__global__ void __launch_bounds__(kTcThreads, 3 - tc_nbuf<FORM>()) k_wide2_tc_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    wide2_tc_body<FORM, CROP>(p, c);
}

}  // namespace cwtk
