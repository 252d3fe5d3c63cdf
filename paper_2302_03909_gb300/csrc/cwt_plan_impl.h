// Internal: the plan object shared by the translation units of the library
// (planner and launches in cwt_api.cu, statistics of W in cwt_stats.cu).
// Not part of the C ABI.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/cwt.h"
#include "cwt_kernels.cuh"

// Launch recording for batches (cwt_batch_create).  A plan whose rec is set
// records each launch (the grouped form of its kernel, the launch shape and
// the argument struct) instead of making it.  The level of a launch is its
// depth in the plan's stream and event order: every launch a launch depends on
// has a lower level, so running the levels one after another, each level's
// launches in any order or at once, keeps every dependency.
struct RecLaunch {
    const void* gfn;
    dim3 grid, block;
    size_t smem;
    int level;
    std::vector<uint32_t> arg;
};
struct Recorder {
    std::vector<RecLaunch> launches;
    std::unordered_map<const void*, int> stream_level, event_level;
    int level_of(const void* s) const {
        auto it = stream_level.find(s);
        return it == stream_level.end() ? 0 : it->second;
    }
    void add(cudaStream_t s, const void* gfn, dim3 grid, dim3 block, size_t smem, const void* arg, size_t bytes) {
        const int l = level_of((const void*)s);
        RecLaunch r{gfn, grid, block, smem, l, std::vector<uint32_t>((bytes + 3) / 4, 0u)};
        std::memcpy(r.arg.data(), arg, bytes);
        launches.push_back(std::move(r));
        stream_level[(const void*)s] = l + 1;
    }
    void record(cudaEvent_t e, cudaStream_t s) { event_level[(const void*)e] = level_of((const void*)s); }
    void wait(cudaStream_t s, cudaEvent_t e) {
        auto it = event_level.find((const void*)e);
        const int el = it == event_level.end() ? 0 : it->second;
        stream_level[(const void*)s] = std::max(level_of((const void*)s), el);
    }
};

struct cwt_plan {
    int64_t N = 0, M = 0;
    int64_t out_off = 0, out_len = 0;     // kept output window (out_len = N unless a sub-plan)
    int logM = 0, h = 0;
    int32_t S = 0;
    int wavelet = 0, boundary = 0;
    cwt_plan_opts opts{};
    int device = -1;
    std::vector<double> w_tilde;

    std::vector<cwtk::Job> jobs;
    struct BandGroup { int logl; int rdi; int ntiles; int D; size_t tj_off; double bytes; int job0, njobs; };  // depth 2^rdi
    std::vector<BandGroup> groups;        // single-pass jobs by DFT length
    struct WideBatch { int job0; int count; int logl1, var; double band_bytes, out_bytes; int D; };  // logl1 < 0: full pass 1; D: pass-2 tiles per CTA
    std::vector<WideBatch> wide;          // wide jobs, in L2-sized batches
    int wide_logl = 0, wide_loga = 0, wide_G = 0;
    size_t y_stride = 0;                  // elements of Y per stream
    size_t y_count = 0;                   // elements of Y (all streams)
    int fwd_small = 0;
    int crop = 0;                         // N < M: drop the padded outputs
    int64_t n_partials = 0;
    std::vector<int32_t> part_off, part_cnt;
    int64_t n_band_jobs = 0;

    // device memory
    cwtk::Job* d_jobs = nullptr;
    int32_t* d_tile_job = nullptr;
    int32_t* d_part_off = nullptr;
    int32_t* d_part_cnt = nullptr;
    float2* d_Fp = nullptr;
    float2* d_Ft = nullptr;
    float2* d_Y = nullptr;
    double* d_partials = nullptr;
    float2* d_tw_lo = nullptr;
    float2* d_tw_hi = nullptr;
    float2* d_tw_tab = nullptr;
    size_t ws_bytes = 0;
    // periodic boundary for any N (Bluestein chirp transform; M = P >= 2N - 1
    // the power-of-two FFT length): chirp c_j (N), D of the two chirp
    // sequences ([0]: conj(c) for the signal, [1]: c for the scales; P each),
    // work buffers (conv1, then X and X2 of each stream; P each)
    bool bs = false;
    int bs_streams = 1;                   // streams the jobs are spread over (per-stream X, X2 and Y)
    float2* d_bs_chirp = nullptr;
    float2* d_bs_G = nullptr;
    float2* d_bs_work = nullptr;
    // cwt_exec_host buffers
    void* h_sig = nullptr;
    void* h_W = nullptr;
    double* h_spec = nullptr;
    // cwt_exec_host: rows of W go to the host as soon as the launch that
    // finishes them is done, on a copy stream that waits for that launch
    // (set only during that call; rows it does not reach are copied at the end)
    struct HostCopy {
        bool on = false;
        char* dst = nullptr;              // host W
        const char* src = nullptr;        // device W of this call
        size_t row_bytes = 0;
        std::vector<char> done;           // per row: copy issued
        size_t nev = 0;                   // events used in this call
    } hc;
    cudaStream_t hc_stream = nullptr;
    std::vector<cudaEvent_t> hc_ev;
    // cwt_wavelet_power scratch
    double* d_pw_partials = nullptr;
    int64_t pw_chunks = 0;
    // cwt_env_power and cwt_icwt scratch (allocated on first use)
    double* d_env_part = nullptr;
    int64_t* d_env_cnt = nullptr;
    double* d_icwt_coef = nullptr;

    // band groups run on side streams forked from the call's stream
    static constexpr int kSide = 2;
    cudaStream_t side[kSide] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kSide] = {};

    // captured launch sequence, replayed while the call's pointers repeat
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[3] = {};
    const void* skey[3] = {};             // pointers of the last direct call
    bool graphs_ok = true;

    // timing hook (cwt_plan_set_timing)
    struct TimedLaunch { int cls; cudaEvent_t a, b; double bytes; };
    int timing = 0;                       // 1: events per launch; 2: also every launch on the call's stream
    std::vector<cudaEvent_t> ev_pool;
    std::vector<TimedLaunch> pending;
    double t_ms[CWT_KCLASS_COUNT] = {};
    int64_t t_launches[CWT_KCLASS_COUNT] = {};
    double t_bytes[CWT_KCLASS_COUNT] = {};
    double fwd_in_bytes = 0, fwd_out_bytes = 0;

    // zero boundary: the rows child_r0 .. child_r0 + child_n - 1, whose wavelet
    // support E (samples) is short, come from a periodic N-point child plan
    // followed by an edge correction of their 2E outermost outputs
    cwt_plan* child = nullptr;
    int32_t child_r0 = 0, child_n = 0;
    cudaEvent_t ev_pre = nullptr, ev_pfwd = nullptr;   // this plan's forward beside the child
    int32_t edge_bpr = 0;                 // correction blocks per row
    void* d_edge_rows = nullptr;          // per row: E and the offset of its h table
    float2* d_edge_h = nullptr;           // h(j) = sqrt(w~ dx) psi(w~ j), j in [-E, E]
    double* d_edge_delta = nullptr;       // per block: change of the row's sum of |W|^2

    // periodic boundary, N not a power of two: the rows come from zero-boundary
    // sub-plans of the periodically extended signal (rows sub_r0[i] ..), each
    // keeping the window [E_i, E_i + N) of its outputs
    std::vector<cwt_plan*> subs;
    std::vector<int32_t> sub_r0;
    std::vector<int64_t> sub_E;
    int64_t ext_E = 0;                    // extension on each side of the shared buffer
    void* d_ext = nullptr;                // N + 2 ext_E samples, the input's dtype

    Recorder* rec = nullptr;              // set while a batch records this plan's launches

    // caller-supplied scratch (opts.scratch = CWT_SCRATCH_CALLER): each per-call
    // buffer is an offset into the call's scratch.  This plan's own buffers lie
    // in [0, scratch_own); the child plan's tree follows; the sub-plans' trees
    // follow that, all at one offset (they run one after another).
    struct ScratchSlot { void** ptr; size_t off; };
    std::vector<ScratchSlot> scratch_slots;
    size_t scratch_own = 0;
    char* scratch_base = nullptr;         // bound for the duration of one call
    bool ymap_on = false;                 // the tile pipeline's TMA map of Y is in use

    // tensor-core pass 2 (opts.precision != FP32, L = 1024): TMA map of Y, and a
    // flag in mapped host memory that its kernel sets when a bounded wait gives up
    CUtensorMap ymap{};
    int32_t* h_err = nullptr;             // host view (cudaHostAlloc, mapped)
    int32_t* d_err = nullptr;             // device view

    std::string err;
};

// records msg as the plan's last error and returns st
cwt_status plan_fail(cwt_plan* p, cwt_status st, const char* msg);
// CWT_ERR_INVALID_ARG unless the current device is the plan's
cwt_status plan_check_device(cwt_plan* p);
