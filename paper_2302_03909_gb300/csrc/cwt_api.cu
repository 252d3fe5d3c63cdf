// Host side of the GB300 FFTCWT: planner, workspace, launches and the C ABI
// declared in include/cwt.h.  Transform definition: Wang & He (RASTI 2023,
// arXiv:2302.03909), Sec. 3.1, Eqs. 8-10; power spectrum Eq. 42.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cwt.h"
#include "cwt_kernels.cuh"

using namespace cwtk;

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr int kMaxLogM = 25;          // M <= 2^25 (zero boundary of N = 2^24)
constexpr int kSingleMaxLogB = 10;    // single-pass DFT length when M > kLmax
constexpr int kMaxDepth = 4;          // direct depth of the single-pass kernel

// ----------------------------------------------------------- launch shapes

constexpr int final_T(int logb) {
    int t = kTileElems >> logb;
    return t < 1 ? 1 : (t > 64 ? 64 : t);
}
constexpr int final_NT(int logb) {
    int e = (1 << logb) * final_T(logb) / 8;
    return e < 32 ? 32 : (e > 256 ? 256 : e);
}
constexpr int final_pad(int logb) {
    return (final_T(logb) < 16 && final_T(logb) > 1) ? 1 : 0;
}
constexpr int p1_T(int loga) {
    int t = kTileElems >> loga;
    return t < 1 ? 1 : (t > 16 ? 16 : t);
}
constexpr int p1_NT(int loga) {
    int e = (1 << loga) * p1_T(loga) / 8;
    return e < 32 ? 32 : (e > 256 ? 256 : e);
}

using FinalFn = void (*)(Params, const Job*, const int32_t*);
using Pass1Fn = void (*)(Params, const Job*);

struct FinalEntry { FinalFn fn; int T, NT; };
struct Pass1Entry { Pass1Fn fn; int T1, NT; };

template <int LOGB, int SRC, int SINK>
FinalEntry final_entry() {
    return {k_final<LOGB, final_T(LOGB), final_NT(LOGB), SRC, SINK>, final_T(LOGB), final_NT(LOGB)};
}
template <int LOGA, int MODE>
Pass1Entry pass1_entry() {
    return {k_pass1<LOGA, p1_T(LOGA), p1_NT(LOGA), MODE>, p1_T(LOGA), p1_NT(LOGA)};
}

template <int SRC, int SINK, int... L>
void fill_final(FinalEntry* tab, std::integer_sequence<int, L...>) {
    ((tab[L + 1] = final_entry<L + 1, SRC, SINK>()), ...);
}
template <int MODE, int... L>
void fill_pass1(Pass1Entry* tab, std::integer_sequence<int, L...>) {
    ((tab[L + 1] = pass1_entry<L + 1, MODE>()), ...);
}

struct Tables {
    FinalEntry band_w[kLmaxLog + 1];     // single pass, band source, W sink
    FinalEntry y_w[kLmaxLog + 1];        // pass 2 of the inverse
    FinalEntry y_fwd[kLmaxLog + 1];      // pass 2 of the forward
    FinalEntry sig_fwd[kLmaxLog + 1];    // one-tile forward
    Pass1Entry p1_band[kLmaxLog + 1];
    Pass1Entry p1_sig[kLmaxLog + 1];
    Tables() {
        std::memset((void*)this, 0, sizeof(*this));
        auto seq = std::make_integer_sequence<int, kLmaxLog>{};
        fill_final<SRC_BAND, SINK_W>(band_w, seq);
        fill_final<SRC_Y, SINK_W>(y_w, seq);
        fill_final<SRC_Y, SINK_FWD>(y_fwd, seq);
        fill_final<SRC_SIGNAL, SINK_FWD>(sig_fwd, seq);
        fill_pass1<P1_BAND>(p1_band, seq);
        fill_pass1<P1_SIGNAL>(p1_sig, seq);
    }
};

const Tables& tables() {
    static Tables t;
    return t;
}

int ilog2(int64_t v) { int l = 0; while ((int64_t(1) << l) < v) l++; return l; }
bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// FP64 wavelet spectra of Table 2 for planning, up to the constant factor
double psi_hat_shape(int wavelet, double omega0, double u) {
    if (wavelet == CWT_WAVELET_GDW) return u * u * std::exp(-u * u);
    return std::exp(-0.5 * (u - omega0) * (u - omega0)) - std::exp(-0.5 * (u * u + omega0 * omega0));
}

double wavelet_cn(int wavelet, double omega0) {
    if (wavelet == CWT_WAVELET_GDW) return std::pow(18.0 * kPi, -0.25);
    double w2 = omega0 * omega0;
    return std::pow(kPi, -0.25) / std::sqrt(1.0 - 2.0 * std::exp(-0.75 * w2) + std::exp(-w2));
}

// psi_hat(u) = C * shape(u): C = 8 sqrt(pi) C_N (GDW), sqrt(2 pi) C_N (Morlet)
double wavelet_spectrum_const(int wavelet, double omega0) {
    double cn = wavelet_cn(wavelet, omega0);
    return wavelet == CWT_WAVELET_GDW ? 8.0 * std::sqrt(kPi) * cn : std::sqrt(2.0 * kPi) * cn;
}

// [u_lo, u_hi] outside which |psi_hat| < eps * max |psi_hat|
void wavelet_band(int wavelet, double omega0, double eps, double* u_lo, double* u_hi) {
    const double step = 1.0 / 1024.0, U = 80.0;
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

}  // namespace

// ====================================================================== plan

struct cwt_plan {
    int64_t N = 0, M = 0;
    int logM = 0, h = 0;
    int32_t S = 0;
    int wavelet = 0, boundary = 0;
    cwt_plan_opts opts{};
    int device = -1;
    std::vector<double> w_tilde;

    std::vector<Job> jobs;
    struct Group { int logb; int T_eff; int ntiles; int kmax; size_t tj_off; std::vector<int> job_ids; };
    std::vector<Group> groups;            // single-pass jobs by DFT length
    std::vector<int> two_pass;            // jobs using pass 1 + pass 2
    int tp_loga = 0, tp_logb = 0, tp_T_eff = 0, tp_ntiles2 = 0;
    int fwd_small = 0, fwd_loga = 0, fwd_logb = 0, fwd_T_eff = 0;
    int64_t n_partials = 0;
    std::vector<int32_t> part_off, part_cnt;

    // device memory
    Job* d_jobs = nullptr;
    int32_t* d_tile_job = nullptr;
    int32_t* d_part_off = nullptr;
    int32_t* d_part_cnt = nullptr;
    float2* d_Fp = nullptr;
    float2* d_Y = nullptr;
    double* d_partials = nullptr;
    float2* d_tw_lo = nullptr;
    float2* d_tw_hi = nullptr;
    float2* d_tw_L = nullptr;
    size_t ws_bytes = 0;
    // cwt_exec_host buffers
    void* h_sig = nullptr;
    void* h_W = nullptr;
    double* h_spec = nullptr;
    // cwt_wavelet_power scratch
    double* d_pw_partials = nullptr;
    int64_t pw_chunks = 0;

    // timing hook (cwt_plan_set_timing)
    struct TimedLaunch { int cls; cudaEvent_t a, b; double bytes; };
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<TimedLaunch> pending;
    double t_ms[CWT_KCLASS_COUNT] = {};
    int64_t t_launches[CWT_KCLASS_COUNT] = {};
    double t_bytes[CWT_KCLASS_COUNT] = {};
    // algorithmic bytes of each launch group
    std::vector<double> group_bytes;
    double fwd_in_bytes = 0, fwd_out_bytes = 0;

    std::string err;
};

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
    void* ptrs[] = {p->d_jobs, p->d_tile_job, p->d_part_off, p->d_part_cnt, p->d_Fp, p->d_Y,
                    p->d_partials, p->d_tw_lo, p->d_tw_hi, p->d_tw_L, p->h_sig, p->h_W,
                    p->h_spec, p->d_pw_partials};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

double out_row_bytes(const cwt_plan* p);
double job_rows(const Job& J);

ScaleGen make_gen(const cwt_plan* p, double wt, int row) {
    ScaleGen g{};
    double alpha = 2.0 * kPi / ((double)p->M * wt);
    g.a_hi = (float)alpha;
    g.a_lo = (float)(alpha - (double)g.a_hi);
    g.amp = (float)(std::sqrt(p->opts.dx / wt) / (double)p->M *
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

cwt_status build_plan(cwt_plan* p) {
    const Tables& tb = tables();
    const int64_t M = p->M;
    double u_lo = -1e300, u_hi = 1e300;
    bool full = p->opts.eps_trunc <= 0.0;
    if (!full) wavelet_band(p->wavelet, p->opts.omega0, p->opts.eps_trunc, &u_lo, &u_hi);

    // jobs: GDW pairs (2i, 2i+1); Morlet one scale each
    const int per = (p->wavelet == CWT_WAVELET_GDW) ? 2 : 1;
    for (int s0 = 0; s0 < p->S; s0 += per) {
        Job J{};
        int64_t klo = 0, khi = -1;
        for (int q = 0; q < 2; q++) {
            int s = s0 + q;
            if (q < per && s < p->S) {
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
        p->jobs.push_back(J);
    }

    // transform shapes
    const bool small = M <= kLmax;
    p->tp_logb = std::max(kSingleMaxLogB, p->logM - kLmaxLog);
    p->tp_loga = p->logM - p->tp_logb;
    std::vector<std::vector<int>> by_logb(kLmaxLog + 1);
    for (int j = 0; j < (int)p->jobs.size(); j++) {
        Job& J = p->jobs[j];
        int lk = std::max(1, ilog2(J.K));
        if (small) {
            int lb = std::min(lk, p->logM);
            J.r = (int32_t)((J.K + (1 << lb) - 1) >> lb);
            by_logb[lb].push_back(j);
        } else if (lk <= kSingleMaxLogB) {
            J.r = 1;
            by_logb[lk].push_back(j);
        } else if (J.K <= kMaxDepth << kSingleMaxLogB) {
            J.r = (int32_t)((J.K + (1 << kSingleMaxLogB) - 1) >> kSingleMaxLogB);
            by_logb[kSingleMaxLogB].push_back(j);
        } else {
            J.r = 0;
            J.tile0 = 0;
            p->two_pass.push_back(j);
        }
    }

    // single-pass groups and their tile -> job maps; power partial layout
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
    for (int lb = 1; lb <= kLmaxLog; lb++) {
        if (by_logb[lb].empty()) continue;
        cwt_plan::Group g;
        g.logb = lb;
        int64_t A = M >> lb;
        g.T_eff = (int)std::min<int64_t>(tb.band_w[lb].T, A);
        int per_job = (int)(A / g.T_eff);
        g.ntiles = 0;
        g.kmax = 0;
        g.tj_off = tile_job.size();
        for (int j : by_logb[lb]) {
            Job& J = p->jobs[j];
            J.tile0 = g.ntiles;
            for (int t = 0; t < per_job; t++) tile_job.push_back(j);
            g.ntiles += per_job;
            g.kmax = std::max(g.kmax, (int)J.K);
            assign_parts(J, per_job);
            g.job_ids.push_back(j);
        }
        p->groups.push_back(g);
    }
    if (!p->two_pass.empty()) {
        int64_t A = M >> p->tp_logb;
        p->tp_T_eff = (int)std::min<int64_t>(tb.y_w[p->tp_logb].T, A);
        p->tp_ntiles2 = (int)(A / p->tp_T_eff);
        for (int j : p->two_pass) assign_parts(p->jobs[j], p->tp_ntiles2);
    }
    p->n_partials = nparts;
    for (const auto& g : p->groups) {
        double b = 0;
        for (int j : g.job_ids) b += job_rows(p->jobs[j]) * out_row_bytes(p) + 8.0 * p->jobs[j].K;
        p->group_bytes.push_back(b);
    }
    p->fwd_in_bytes = (double)p->N * (p->opts.input_dtype == CWT_INPUT_F64 ? 8.0 : 4.0);
    p->fwd_out_bytes = 8.0 * (double)(M / 2 + 1);

    // forward transform shape
    if (small) {
        p->fwd_small = 1;
        p->fwd_logb = p->logM;
        p->fwd_T_eff = 1;
    } else {
        p->fwd_small = 0;
        p->fwd_logb = p->tp_logb;
        p->fwd_loga = p->tp_loga;
        p->fwd_T_eff = (int)std::min<int64_t>(tb.y_fwd[p->fwd_logb].T, M >> p->fwd_logb);
    }

    // twiddle tables (FP64 generated, FP32 stored)
    p->h = (p->logM + 1) / 2;
    std::vector<float2> lo(size_t(1) << p->h), hi(size_t(1) << (p->logM - p->h)), tl(kLmax);
    for (size_t j = 0; j < lo.size(); j++) {
        double a = -2.0 * kPi * (double)j / (double)M;
        lo[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (size_t j = 0; j < hi.size(); j++) {
        double a = -2.0 * kPi * (double)(j << p->h) / (double)M;
        hi[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    for (size_t j = 0; j < tl.size(); j++) {
        double a = -2.0 * kPi * (double)j / (double)kLmax;
        tl[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }

    cwt_status st;
    if ((st = upload(p, &p->d_jobs, p->jobs)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_tile_job, tile_job)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_part_off, p->part_off)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_part_cnt, p->part_cnt)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_tw_lo, lo)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_tw_hi, hi)) != CWT_OK) return st;
    if ((st = upload(p, &p->d_tw_L, tl)) != CWT_OK) return st;
    if ((st = dev_alloc(p, &p->d_Fp, (size_t)(M / 2 + 1))) != CWT_OK) return st;
    if (!p->fwd_small || !p->two_pass.empty())
        if ((st = dev_alloc(p, &p->d_Y, (size_t)M)) != CWT_OK) return st;
    if ((st = dev_alloc(p, &p->d_partials, (size_t)std::max<int64_t>(1, nparts))) != CWT_OK) return st;
    return CWT_OK;
}

Params base_params(const cwt_plan* p) {
    Params P{};
    P.Fp = p->d_Fp;
    P.Fp_out = p->d_Fp;
    P.Y = p->d_Y;
    P.partials = p->d_partials;
    P.tw_lo = p->d_tw_lo;
    P.tw_hi = p->d_tw_hi;
    P.tw_L = p->d_tw_L;
    P.N = p->N;
    P.M = (int32_t)p->M;
    P.logM = p->logM;
    P.h = p->h;
    P.wavelet = p->wavelet;
    P.sig_f64 = p->opts.input_dtype == CWT_INPUT_F64;
    P.half_w0sq = (float)(0.5 * p->opts.omega0 * p->opts.omega0);
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

cwt_status launch_final(cwt_plan* p, const FinalEntry& fe, int ntiles, size_t smem, const Params& P,
                        const int32_t* tile_job, cudaStream_t s, int cls, double bytes) {
    if (smem > 48 * 1024) {
        CWT_CUDA(p, cudaFuncSetAttribute((const void*)fe.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    }
    LaunchTimer lt(p, cls, bytes, s);
    fe.fn<<<ntiles, fe.NT, smem, s>>>(P, p->d_jobs, tile_job);
    CWT_CUDA(p, cudaGetLastError());
    lt.done();
    return CWT_OK;
}

cwt_status launch_pass1(cwt_plan* p, const Pass1Entry& pe, int loga, const Params& P, cudaStream_t s, int cls,
                        double bytes) {
    size_t smem = (size_t)pe.T1 * (size_t)((1 << loga) + 1) * sizeof(float2);
    if (smem > 48 * 1024) {
        CWT_CUDA(p, cudaFuncSetAttribute((const void*)pe.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    }
    int B = (int)(p->M >> loga);
    LaunchTimer lt(p, cls, bytes, s);
    pe.fn<<<B / pe.T1, pe.NT, smem, s>>>(P, p->d_jobs);
    CWT_CUDA(p, cudaGetLastError());
    lt.done();
    return CWT_OK;
}

double out_row_bytes(const cwt_plan* p) {
    return (double)p->N * (p->wavelet == CWT_WAVELET_MORLET ? 8.0 : 4.0);
}

double job_rows(const Job& J) { return (J.g[0].row >= 0) + (J.g[1].row >= 0); }

size_t final_smem(int logb, int kmax) {
    return ((size_t)(1 << logb) * (size_t)(final_T(logb) + final_pad(logb)) + (size_t)kmax) * sizeof(float2);
}

cwt_status check_device(cwt_plan* p) {
    int d = -1;
    CWT_CUDA(p, cudaGetDevice(&d));
    if (d != p->device) return fail(p, CWT_ERR_INVALID_ARG, "current device differs from the plan's device");
    return CWT_OK;
}

cwt_status run(cwt_plan* p, const void* signal, void* W, double* spectrum, cudaStream_t s) {
    const Tables& tb = tables();
    cwt_status st;
    Params P = base_params(p);
    P.signal = signal;
    P.W = W;
    P.do_power = spectrum != nullptr;

    // 1. forward transform F(m) = sum_n f(n) e^{+2 pi i m n / M}, m <= M/2
    if (p->fwd_small) {
        const FinalEntry& fe = tb.sig_fwd[p->fwd_logb];
        Params Q = P;
        Q.A = 1;
        Q.T_eff = 1;
        if ((st = launch_final(p, fe, 1, final_smem(p->fwd_logb, 0), Q, nullptr, s, CWT_KCLASS_FORWARD,
                               p->fwd_in_bytes + p->fwd_out_bytes)) != CWT_OK)
            return st;
    } else {
        Params Q = P;
        if ((st = launch_pass1(p, tb.p1_sig[p->fwd_loga], p->fwd_loga, Q, s, CWT_KCLASS_FORWARD,
                               p->fwd_in_bytes)) != CWT_OK)
            return st;
        const FinalEntry& fe = tb.y_fwd[p->fwd_logb];
        Q.A = (int32_t)(p->M >> p->fwd_logb);
        Q.T_eff = p->fwd_T_eff;
        if ((st = launch_final(p, fe, Q.A / Q.T_eff, final_smem(p->fwd_logb, 0), Q, nullptr, s, CWT_KCLASS_FORWARD,
                               p->fwd_out_bytes)) != CWT_OK)
            return st;
    }

    // 2. single-pass scales, one launch per DFT length
    for (size_t gi = 0; gi < p->groups.size(); gi++) {
        const auto& g = p->groups[gi];
        const FinalEntry& fe = tb.band_w[g.logb];
        Params Q = P;
        Q.A = (int32_t)(p->M >> g.logb);
        Q.T_eff = g.T_eff;
        if ((st = launch_final(p, fe, g.ntiles, final_smem(g.logb, g.kmax), Q, p->d_tile_job + g.tj_off, s,
                               CWT_KCLASS_BAND, p->group_bytes[gi])) != CWT_OK)
            return st;
    }

    // 3. wide-band scales: pass 1 (A-point DFTs + twiddle) then pass 2
    for (int j : p->two_pass) {
        Params Q = P;
        Q.job = j;
        const Job& J = p->jobs[j];
        if ((st = launch_pass1(p, tb.p1_band[p->tp_loga], p->tp_loga, Q, s, CWT_KCLASS_WIDE1, 8.0 * J.K)) !=
            CWT_OK)
            return st;
        const FinalEntry& fe = tb.y_w[p->tp_logb];
        Q.A = (int32_t)(p->M >> p->tp_logb);
        Q.T_eff = p->tp_T_eff;
        if ((st = launch_final(p, fe, p->tp_ntiles2, final_smem(p->tp_logb, 0), Q, nullptr, s, CWT_KCLASS_WIDE2,
                               job_rows(J) * out_row_bytes(p))) != CWT_OK)
            return st;
    }

    // 4. power spectrum: fixed-order reduction of the per-tile partials
    if (spectrum) {
        LaunchTimer lt(p, CWT_KCLASS_POWER, 8.0 * (double)(p->n_partials + p->S), s);
        k_power_finalize<<<p->S, 32, 0, s>>>(p->d_partials, p->d_part_off, p->d_part_cnt, p->S, p->N, spectrum);
        CWT_CUDA(p, cudaGetLastError());
        lt.done();
    }
    return CWT_OK;
}

bool aligned(const void* q, size_t a) { return ((uintptr_t)q % a) == 0; }

}  // namespace

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
    if (wavelet != CWT_WAVELET_GDW && wavelet != CWT_WAVELET_MORLET) return CWT_ERR_INVALID_ARG;
    if (boundary != CWT_BOUNDARY_PERIODIC && boundary != CWT_BOUNDARY_ZERO) return CWT_ERR_INVALID_ARG;
    if (o.scale_unit != CWT_SCALE_DILATION && o.scale_unit != CWT_SCALE_W_TILDE) return CWT_ERR_INVALID_ARG;
    if (o.input_dtype != CWT_INPUT_F32 && o.input_dtype != CWT_INPUT_F64) return CWT_ERR_INVALID_ARG;
    if (!(o.dx > 0.0) || !std::isfinite(o.dx) || !std::isfinite(o.omega0) || !(o.eps_trunc >= 0.0) ||
        o.eps_trunc >= 1.0)
        return CWT_ERR_INVALID_ARG;
    if (wavelet == CWT_WAVELET_MORLET && !(o.omega0 > 0.0)) return CWT_ERR_INVALID_ARG;
    for (int32_t i = 0; i < n_scales; i++)
        if (!std::isfinite(scales[i]) || !(scales[i] > 0.0)) return CWT_ERR_INVALID_ARG;

    int64_t M;
    if (boundary == CWT_BOUNDARY_PERIODIC) {
        if (o.fft_len != 0 && o.fft_len != N) return CWT_ERR_INVALID_ARG;
        if (!is_pow2(N)) return CWT_ERR_UNSUPPORTED;
        M = N;
    } else {
        if (o.fft_len != 0) {
            if (o.fft_len < N) return CWT_ERR_INVALID_ARG;
            if (!is_pow2(o.fft_len)) return CWT_ERR_UNSUPPORTED;
            M = o.fft_len;
        } else {
            M = int64_t(1) << ilog2(2 * N);
        }
    }
    if (M < 2 || M > (int64_t(1) << kMaxLogM)) return CWT_ERR_UNSUPPORTED;

    cwt_plan* p = new (std::nothrow) cwt_plan();
    if (!p) return CWT_ERR_OOM;
    p->N = N;
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
    cwt_status st = check_device(plan);
    if (st != CWT_OK) return st;
    size_t se = plan->opts.input_dtype == CWT_INPUT_F64 ? 8 : 4;
    size_t we = plan->wavelet == CWT_WAVELET_MORLET ? 8 : 4;
    size_t sig_bytes = (size_t)plan->N * se, w_bytes = (size_t)plan->N * (size_t)plan->S * we;
    if (!plan->h_sig) CWT_CUDA(plan, cudaMalloc(&plan->h_sig, sig_bytes));
    if (!plan->h_W) CWT_CUDA(plan, cudaMalloc(&plan->h_W, w_bytes));
    if (!plan->h_spec) CWT_CUDA(plan, cudaMalloc((void**)&plan->h_spec, (size_t)plan->S * sizeof(double)));
    cudaStream_t s = (cudaStream_t)stream;
    CWT_CUDA(plan, cudaMemcpyAsync(plan->h_sig, signal_host, sig_bytes, cudaMemcpyHostToDevice, s));
    st = run(plan, plan->h_sig, plan->h_W, spectrum_host ? plan->h_spec : nullptr, s);
    if (st != CWT_OK) return st;
    CWT_CUDA(plan, cudaMemcpyAsync(W_host, plan->h_W, w_bytes, cudaMemcpyDeviceToHost, s));
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
    plan->timing = enable != 0;
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
    if (total_ms) *total_ms = plan->t_ms[cls];
    if (launches) *launches = plan->t_launches[cls];
    if (algorithmic_bytes) *algorithmic_bytes = plan->t_bytes[cls];
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
