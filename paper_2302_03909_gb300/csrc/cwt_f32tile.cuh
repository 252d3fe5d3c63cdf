// FP32 form of the wide scales' second pass (L = 1024-point DFTs) on the tile
// pipeline of the tensor-core forms.
//
// Pass 2 takes, for each column d of Y, X(c) = sum_{b<1024} x(b) w^{b c} with
// w = e^{-2 pi i / 1024} and x(b) = Y[b][d] (the inverse DFT of Eq. 9 split
// into two passes).  With b = l + 32 b1 and c = c1 + 32 c2 it factors into
//   U_l(c1)       = sum_{b1} x(l + 32 b1) e^{-2 pi i b1 c1 / 32}   (radix-32 DFT)
//   V_l(c1)       = U_l(c1) w^{l c1}                               (twiddle)
//   X(c1 + 32 c2) = sum_{l} V_l(c1) e^{-2 pi i l c2 / 32}          (radix-32 DFT)
// the same two stages, on the same twiddle table, as the CTA Stockham kernel
// (k_wide2 with L = 1024), so both give the same W bit for bit.
//
// A CTA takes tiles of 8 consecutive columns, Y[0..1023][d0..d0+7], loaded
// by TMA with the 64-byte swizzle (tc_slot: 8 complex values per row, the
// 16-byte pairs of row r XOR-ed by bits 1-2 of r); rows are in natural order.
// 32 threads compute one column: thread l of column c holds x(l + 32 b1) for
// b1 < 32 in registers, runs the first DFT and the twiddle, writes V_l(c1)
// back into the column at row 32 c1 + (l ^ c1), and after a barrier reads
// V_b0(l) for b0 < 32 from rows 32 l + (b0 ^ l) (thread l now holds stage 2's
// c1 = l), runs the second DFT and writes X(l + 32 c2) to row l + 32 c2.
// The 32 threads of a column are spread over 4 warps: the compute warps form
// two groups of 4 (columns 0-3 and 4-7), and lane l of warp u of a group takes
// the group's column (u + l / 8) mod 4.  Under the swizzle, one column's rows
// touch only 8 of the 16 bank pairs, so a warp on a single column would put
// 4 lanes on a bank pair; with 4 columns per warp every access of the kernel
// puts 2 lanes on each bank pair, the minimum for 32 8-byte accesses.
//
// k_wide2_f32: 8 compute warps and 4 store warps, 3 tile buffers.  A store
//   thread issues the TMA loads (mbarrier completion); the compute warps
//   wait only for their tile's bytes, synchronise within their group (named
//   barriers 5 and 6) around the in-place exchange, and hand the outputs to the
//   store warps through named barriers 1 + q % 3; the store warps store W rows
//   with 16-byte stores and reload the buffer with the tile three steps ahead.
// k_wide2_f32_g: the grouped-launch form (batches): one buffer copied with
//   cp.async, the same arithmetic and the same 128 storing threads, so the
//   same results.
#pragma once
#include "cwt_tc.cuh"

namespace cwtk {

constexpr int kF32Bufs = 3;
constexpr int kF32Compute = 32 * kTcCols;            // 32 threads per column
constexpr int kF32Store = 128;                       // store threads
constexpr int kF32Threads = kF32Compute + kF32Store;

// dynamic shared memory: 1 KB of alignment slack, the tile buffers and the
// twiddle table w^{l c1}
__host__ __device__ constexpr size_t f32_smem_bytes(bool pipelined) {
    return 1024 + ((size_t)(pipelined ? kF32Bufs : 1) * kTcTile + 1024) * sizeof(float2);
}

// twf[c1 * 32 + l] = w^{l c1}, from the FP64-generated 1024-point table
__device__ __forceinline__ void f32_build_twiddles(const float2* __restrict__ tw1024, float2* twf, int nthreads) {
    for (int i = threadIdx.x; i < 1024; i += nthreads) {
        const int l = i & 31, c1 = i >> 5;
        twf[i] = __ldg(&tw1024[(l * c1) & 1023]);
    }
}

// The 1024-point DFTs of 4 of the tile's columns, in place, by the 128
// compute threads of group g (threads 128 g .. 128 g + 127, columns
// 4 g .. 4 g + 3; named barrier bar + g of 128 threads).  Lane l of the
// group's warp u takes column 4 g + ((u + l / 8) mod 4).  With
// B = tc_slot(l, c), row 32 u + (l ^ v) of column c lies at slot
// 256 u + (B ^ K(v)), K(v) = 8 v + 2 ((v >> 1) & 3), and row l + 32 u at
// slot 256 u + B.  The two groups synchronise independently, and group 1
// enters its first tile only when group 0 has written its exchange (named
// barrier 7, once), so that one group's shared-memory phases overlap the
// other's arithmetic.
__device__ __forceinline__ void f32_tile_dft(float2* buf, const float2* __restrict__ twf, int bar, bool lead) {
    const int t = threadIdx.x, l = t & 31, g = t >> 7;
    const int c = 4 * g + ((((t >> 5) & 3) + (l >> 3)) & 3);
    const int B = tc_slot(l, c);
    bar += g;
    float2 v[32];
#pragma unroll
    for (int b1 = 0; b1 < 32; b1++) v[b1] = buf[256 * b1 + B];
    dft<32>(v);
#pragma unroll
    for (int c1 = 0; c1 < 32; c1++) v[c1] = cmul(v[c1], twf[c1 * 32 + l]);
    named_sync(bar, 128);                        // every thread of the column has read its inputs
#pragma unroll
    for (int c1 = 0; c1 < 32; c1++) buf[256 * c1 + (B ^ (8 * c1 + 2 * ((c1 >> 1) & 3)))] = v[c1];
    named_sync(bar, 128);
    if (lead && g == 0) named_arrive(7, 256);    // releases group 1 into its first tile
#pragma unroll
    for (int b0 = 0; b0 < 32; b0++) v[b0] = buf[256 * l + (B ^ (8 * b0 + 2 * ((b0 >> 1) & 3)))];
    named_sync(bar, 128);                        // the exchange is read before the outputs overwrite it
    dft<32>(v);
#pragma unroll
    for (int c2 = 0; c2 < 32; c2++) buf[256 * c2 + B] = v[c2];
}

// grid (A / (8 D), jobs in launch), kF32Threads threads: warps 0..7 compute,
// warps 8..11 store.  Tile q of the CTA lives in buffer q % 3.  Store thread 0
// loads tiles 0..2, and tile q + 3 into buffer q % 3 once the store warps have
// stored tile q and passed their own barrier (id 4).  The compute warps wait
// for full[q % 3], compute, and arrive on named barrier 1 + q % 3, on which
// the store warps wait.  The compute warps are at most three tiles ahead of
// the stores, so the three barrier ids never hold two generations at once.
template <bool CROP>
__device__ __forceinline__ void wide2_f32_body(const Params& p, const CUtensorMap* ymap, const Cta c) {
    constexpr int NT = kF32Threads, NB = kF32Bufs;
    extern __shared__ unsigned char smem_raw[];
    float2* bufs = tc_align1024(smem_raw);
    float2* twf = bufs + NB * kTcTile;
    __shared__ double red[2 * (NT / 32)];
    __shared__ Job sJ;
    __shared__ __align__(8) uint64_t full[NB];
    const int tid = threadIdx.x;
    if (tid == 0) {
        sJ = p.jobs[p.job0 + c.y];
        for (int b = 0; b < NB; b++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    f32_build_twiddles(p.tw_tab + 1024, twf, NT);
    const int A = p.A;
    const int z = p.yz0 + c.y;
    const int tile0 = c.x * p.D;
    const int ntile = min(p.D, A / kTcCols - tile0);
    __syncthreads();
    const Job& J = sJ;
    float pw0 = 0.f, pw1 = 0.f;
    if (tid < kF32Compute) {
        bool ok = true;
#pragma unroll 1
        for (int q = 0; q < ntile; q++) {
            if (!mbar_wait(&full[q % NB], (q / NB) & 1)) ok = false;
            if (q == 0 && tid >= 128) named_sync(7, 256);   // group 1 starts half a tile behind group 0
            f32_tile_dft(bufs + (q % NB) * kTcTile, twf, 5, q == 0);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // in-place writes before later copies
            named_arrive(1 + q % 3, NT);         // tile q's outputs are in its buffer
        }
        if (!ok) {
            // copies still in flight: wait (bounded) for the last ones, then report
            for (int q = max(0, ntile - NB); q < ntile; q++) mbar_wait(&full[q % NB], (q / NB) & 1);
            if (p.err) *(volatile int32_t*)p.err = 1;
        }
    } else {
        const int k = tid - kF32Compute;
        if (k == 0)
            for (int q = 0; q < min(NB, ntile); q++)
                tma_load_tile(ymap, bufs + q * kTcTile, &full[q], (tile0 + q) * kTcCols, z);
#pragma unroll 1
        for (int q = 0; q < ntile; q++) {
            float2* buf = bufs + (q % NB) * kTcTile;
            named_sync(1 + q % 3, NT);
            tc_store_tile<kF32Store, CROP, false>(buf, p, J, (tile0 + q) * kTcCols, k, pw0, pw1);
            if (q + NB < ntile) {
                named_sync(4, kF32Store);        // every store thread has read the buffer
                if (k == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    tma_load_tile(ymap, buf, &full[q % NB], (tile0 + q + NB) * kTcCols, z);
                }
            }
        }
    }
    struct { float pw0, pw1; } o{pw0, pw1};
    write_partials<NT>(p, J, o, c.x, red);
}

template <bool CROP>
__global__ void __launch_bounds__(kF32Threads, 1) k_wide2_f32(Params p, const __grid_constant__ CUtensorMap ymap) {
    wide2_f32_body<CROP>(p, &ymap, cta_plain());
}

// grouped form: kTcThreads threads, one buffer in the same layout, copied
// with cp.async; stores by threads 0..127 with the store warps' mapping
template <bool CROP>
__device__ __forceinline__ void wide2_f32_g_body(const Params& p, const Cta c) {
    constexpr int NT = kTcThreads;
    static_assert(NT == kF32Compute, "the compute threads of the pipelined form");
    extern __shared__ unsigned char smem_raw[];
    float2* buf = tc_align1024(smem_raw);
    float2* twf = buf + kTcTile;
    __shared__ double red[2 * (NT / 32)];
    __shared__ Job sJ;
    const int tid = threadIdx.x;
    if (tid == 0) sJ = p.jobs[p.job0 + c.y];
    f32_build_twiddles(p.tw_tab + 1024, twf, NT);
    __syncthreads();
    const Job& J = sJ;
    const int A = p.A;
    const float2* Yj = p.Y + (int64_t)c.y * p.M;
    const int tile0 = c.x * p.D;
    const int ntile = min(p.D, A / kTcCols - tile0);
    const int wc = tid & 3, rr = tid >> 2;
    const int lslot = tc_slot(rr, 2 * wc);      // rows rr + 64 it at lslot + 512 it
    float pw0 = 0.f, pw1 = 0.f;
#pragma unroll 1
    for (int q = 0; q < ntile; q++) {
        const int d0 = (tile0 + q) * kTcCols;
        if (q > 0) __syncthreads();              // the previous tile is stored
        const float2* src = Yj + (int64_t)rr * A + d0 + 2 * wc;
#pragma unroll
        for (int it = 0; it < 1024 / 64; it++) cp_async16(buf + lslot + 512 * it, src + (int64_t)(64 * it) * A);
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        if (q == 0 && tid >= 128) named_sync(7, 256);
        f32_tile_dft(buf, twf, 5, q == 0);
        __syncthreads();
        if (tid < kF32Store) tc_store_tile<kF32Store, CROP, false>(buf, p, J, d0, tid, pw0, pw1);
    }
    struct { float pw0, pw1; } o{pw0, pw1};
    write_partials<NT>(p, J, o, c.x, red);
}

template <bool CROP>
__global__ void __launch_bounds__(kTcThreads, 1) k_wide2_f32_g(GroupMap g) {
    Cta c;
    const Params& p = group_args<Params>(g, c);
    wide2_f32_g_body<CROP>(p, c);
}

}  // namespace cwtk
