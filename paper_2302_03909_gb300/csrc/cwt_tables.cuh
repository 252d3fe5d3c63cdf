// Kernel dispatch tables of the GB300 FFTCWT: launch shapes of every
// kernel instantiation and the Tables the planner indexes.  The tables are
// filled by several translation units (cwt_tab_*.cu) so that nvcc compiles
// the template instantiations in parallel.
#pragma once

#include <cuda.h>

#include <utility>

#include "cwt_kernels.cuh"

namespace cwtk {

// T columns per CTA: T * max_bfly(LOGL) ~ 256 (128 for one-stage DFTs); the CTA
// runs T * col_threads(LOGL) threads
constexpr int kThreadsTarget = 256;
// (three-stage DFTs keep 2 columns, 1 at L = 8192, so 128 registers fit)
constexpr int band_T(int logl) {
    return n_stages(logl) == 1 ? 128
         : n_stages(logl) == 3 ? (logl >= 13 ? 1 : 2)
         : (kThreadsTarget / max_bfly(logl) < 1 ? 1 : kThreadsTarget / max_bfly(logl));
}
constexpr int wide1_T(int loga) { return band_T(loga); }
// pruned pass 1: the band-kernel column count; smaller variants for small A1 = A / L1
constexpr int wide1p_T(int logl) { return band_T(logl); }
// pruned pass-1 variants: column count T = min(wide1p_T(L1), 128 >> q), q < kP1Var
constexpr int kP1Var = 7;
constexpr int p1var_T(int logl, int q) { return wide1p_T(logl) < (128 >> q) ? wide1p_T(logl) : (128 >> q); }
// direct depths of the L = 1024 band kernel (bands up to RD * 1024 bins,
// RD = 2^i for i <= kBandRdMax)
constexpr int kBandDepthLog = 10;
constexpr int kBandRdMax = 4;

// fn: the kernel; gfn: its grouped form (one launch over several plans' launches)
using KernFn = void (*)(Params);
using KernFnG = void (*)(GroupMap);
struct Entry { KernFn fn; KernFnG gfn; int T, NT, logl; };
using KernFnP = void (*)(Wide1pArgs);
struct EntryP { KernFnP fn; KernFnG gfn; int T, NT, logl; };
// tensor-core pass 2: fn takes the TMA map of the plan's Y and runs NT threads
// (plain launches); gfn is the grouped form (kTcThreads threads, cp.async)
using KernFnTma = void (*)(Params, CUtensorMap);
struct TcEntry { KernFnTma fn; KernFnG gfn; int NT; size_t smem, gsmem; };   // gfn: kTcThreads threads

template <int LOGL, int T, bool CROP, int RD = 1>
Entry band_entry() { return {k_band<LOGL, T, CROP, RD>, k_band_g<LOGL, T, CROP, RD>, T, T * col_threads(LOGL), LOGL}; }
template <int LOGL, int T>
Entry wide1_entry() { return {k_wide1<LOGL, T>, k_wide1_g<LOGL, T>, T, T * col_threads(LOGL), LOGL}; }
template <int LOGL, int T, bool CROP>
Entry wide2_entry() { return {k_wide2<LOGL, T, CROP>, k_wide2_g<LOGL, T, CROP>, T, T * col_threads(LOGL), LOGL}; }
template <int LOGL, int T>
Entry fwd1_entry() { return {k_fwd1<LOGL, T>, k_fwd1_g<LOGL, T>, T, T * col_threads(LOGL), LOGL}; }
template <int LOGL, int T>
Entry fwd2_entry() { return {k_fwd2<LOGL, T>, k_fwd2_g<LOGL, T>, T, T * col_threads(LOGL), LOGL}; }
template <int LOGL, int T>
EntryP wide1p_entry() { return {k_wide1p<LOGL, T>, k_wide1p_g<LOGL, T>, T, T * col_threads(LOGL), LOGL}; }

struct Tables {
    Entry band[kLmaxLog + 1][2];            // [log2 L][crop]
    Entry band_rd[kBandRdMax + 1][2];       // L = 1024 with direct depth 2^(i): [i][crop], i = 1 .. kBandRdMax
    Entry wide1[kLmaxLog + 1];
    Entry fwd1[kLmaxLog + 1];
    Entry fwd_small[kLmaxLog + 1];
    Entry wide2[kLmaxLog + 1][2];           // [log2 L][crop]
    Entry fwd2[kLmaxLog + 1];
    EntryP wide1p[kLmaxLog + 1][kP1Var];    // [log2 L1][column-count variant]
    TcEntry wide2_tc[5][2];                 // pass 2 with L = 1024, tile pipeline: [precision][crop]
};

void fill_band_tables(Tables& t);   // cwt_tab_band.cu
void fill_p1_tables(Tables& t);     // cwt_tab_p1.cu
void fill_wide_tables(Tables& t);   // cwt_tab_wide.cu
void fill_fwd_tables(Tables& t);    // cwt_tab_fwd.cu
void fill_tc_tables(Tables& t);     // cwt_tab_tc.cu

}  // namespace cwtk
