// Per-kernel launch counting and CUDA-event timing (include/helm_trace.h).
#include <string.h>
#include <mutex>
#include <vector>

#include "helm_trace.h"
#include "trace.h"

namespace helm {

static const char *kNames[K_COUNT] = {
    "assemble", "sources", "restriction_taps", "restrict", "line_factor_fp64", "line_factor_fp32",
    "line_sweep_fp64", "line_sweep_fp32", "residual_fp64", "misfit", "scatter_adjoint_rhs", "grad_accumulate",
    "g_u_p_rhs", "z_rhs_base", "hess_accumulate", "hyper_terms", "dot_partial", "sum_partials", "axpby",
    "fill", "sub", "regR", "dct_matrix", "p2_scale", "dgemm_dct", "line_gb_prepass", "split_diag", "refine_start", "refine_update",
    "refine_finish", "refine_accumulate", "field_grad", "g_coefficients", "hess_finish",
    "zgemm_tf32x3", "zinv_block", "ztranspose", "bcr_form_blocks", "bcr_level0_update", "bcr_solve_level0",
    "zgemm_split_reduce",
};

namespace {
struct Rec {
    int id;
    cudaEvent_t a, b;
    cudaStream_t st;
    double flops;
};
std::mutex g_mu;
bool g_on = false;
int g_only = -1;   // kernel index timed alone (-1: all)
int64_t g_launch[K_COUNT] = {};
int64_t g_timed[K_COUNT] = {};
double g_ms[K_COUNT] = {};
double g_flops[K_COUNT] = {};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}
}  // namespace

TraceScope::TraceScope(int id, cudaStream_t st, double flops) : id_(id), st_(st), a_(nullptr), flops_(flops) {
    std::lock_guard<std::mutex> lk(g_mu);
    ++g_launch[id];
    if (g_on && (g_only < 0 || g_only == id)) {
        a_ = get_event();
        if (a_) cudaEventRecord(a_, st_);
    }
}

TraceScope::~TraceScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t b = get_event();
    if (!b) return;
    cudaEventRecord(b, st_);
    g_recs.push_back(Rec{id_, a_, b, st_, flops_});
}

}  // namespace helm

using namespace helm;

extern "C" void helm_trace_enable(int on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    // events are created here, not at launch time: creating one while other host threads
    // launch kernels can delay those launches
    constexpr size_t kPool = 16384;
    while (g_on && g_pool.size() + 2 * g_recs.size() < kPool) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); break; }
        g_pool.push_back(e);
    }
}

extern "C" int32_t helm_trace_select(const char *kernel_name) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!kernel_name || !kernel_name[0]) { g_only = -1; return 0; }
    for (int i = 0; i < K_COUNT; ++i)
        if (strcmp(kNames[i], kernel_name) == 0) { g_only = i; return 0; }
    return -1;
}

extern "C" void helm_trace_reset(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : g_recs) {
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    memset(g_launch, 0, sizeof g_launch);
    memset(g_timed, 0, sizeof g_timed);
    memset(g_ms, 0, sizeof g_ms);
    memset(g_flops, 0, sizeof g_flops);
}

extern "C" int32_t helm_trace_read(helm_trace_entry *out, int32_t max) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    for (auto &r : g_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_ms[r.id] += ms;
            g_flops[r.id] += r.flops;
            ++g_timed[r.id];
        }
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    int n = 0;
    for (int i = 0; i < K_COUNT && n < max; ++i) {
        if (g_launch[i] == 0) continue;
        helm_trace_entry &e = out[n++];
        memset(&e, 0, sizeof e);
        strncpy(e.name, kNames[i], sizeof(e.name) - 1);
        e.launches = g_launch[i];
        e.total_ms = g_ms[i];
        e.timed = g_timed[i];
        e.flops = g_flops[i];
    }
    return n;
}

extern "C" int32_t helm_trace_timeline(helm_trace_event *out, int32_t max) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaDeviceSynchronize() != cudaSuccess) return -1;
    std::vector<cudaStream_t> streams;
    int n = 0;
    for (size_t i = 0; i < g_recs.size() && n < max; ++i) {
        const Rec &r = g_recs[i];
        float t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&t0, g_recs[0].a, r.a) != cudaSuccess ||
            cudaEventElapsedTime(&t1, g_recs[0].a, r.b) != cudaSuccess)
            return -1;
        int sid = 0;
        while (sid < (int)streams.size() && streams[sid] != r.st) ++sid;
        if (sid == (int)streams.size()) streams.push_back(r.st);
        out[n++] = helm_trace_event{r.id, sid, (double)t0, (double)t1};
    }
    return n;
}

extern "C" const char *helm_trace_kernel_name(int32_t id) { return (id >= 0 && id < K_COUNT) ? kNames[id] : nullptr; }

extern "C" int64_t helm_launch_count(void) {
    std::lock_guard<std::mutex> lk(g_mu);
    int64_t t = 0;
    for (int i = 0; i < K_COUNT; ++i) t += g_launch[i];
    return t;
}
