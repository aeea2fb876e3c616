// Launch accounting (see prof.h) and its C-ABI entry points.
#include "prof.h"

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"

namespace qsim {

namespace {
struct Rec {
    cudaEvent_t a, b;
    int c;
};
std::atomic<bool> g_on{false};
std::mutex g_mu;
std::vector<Rec> g_recs;         // launches recorded since the last collect
std::vector<cudaEvent_t> g_pool; // reusable events
std::vector<cudaEvent_t> g_open; // started, not yet ended (per launch nesting)
std::vector<int> g_open_cls;
long long g_untimed[KC_COUNT];   // launches counted when events could not be made
double g_bytes[KC_COUNT];
double g_flops[KC_COUNT];

const char *kNames[KC_COUNT] = {"init", "dense", "phase", "diag", "swap", "param",
                                "tiled", "fused_tc", "reduce", "trotter_diag", "adjoint", "hpsi", "evolve", "host_copy"};

cudaEvent_t take() {
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

thread_local bool t_suspended = false;
bool prof_enabled() { return g_on.load(std::memory_order_relaxed) && !t_suspended; }
void prof_suspend(bool on) { t_suspended = on; }

void prof_add_work(int c, double bytes, double flops) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_bytes[c] += bytes;
    g_flops[c] += flops;
}

void prof_begin(cudaStream_t st, int c) {
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEvent_t e = take();
    if (e) cudaEventRecord(e, st);
    g_open.push_back(e);
    g_open_cls.push_back(c);
}

void prof_end(cudaStream_t st, int c) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_open.empty()) return;
    cudaEvent_t a = g_open.back();
    g_open.pop_back();
    g_open_cls.pop_back();
    cudaEvent_t b = take();
    if (a && b) {
        cudaEventRecord(b, st);
        g_recs.push_back({a, b, c});
    } else {
        g_untimed[c]++;
        if (a) g_pool.push_back(a);
        if (b) g_pool.push_back(b);
    }
}

}  // namespace qsim

using namespace qsim;

extern "C" {

qs_status qs_profile_enable(int on) {
    g_on.store(on != 0);
    return QS_OK;
}

qs_status qs_profile_collect(double *total_ms, long long *launches, double *bytes, double *flops,
                             int n_classes) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (n_classes < 0 || (n_classes > 0 && (!total_ms || !launches || !bytes || !flops))) {
        set_error("bad output arrays");
        return QS_ERR_ARG;
    }
    std::vector<double> ms(KC_COUNT, 0.0);
    std::vector<long long> cnt(KC_COUNT, 0);
    qs_status st = QS_OK;
    for (const Rec &r : g_recs) {
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
        if (e != cudaSuccess && st == QS_OK) st = cuda_status(e, "profile events");
        ms[r.c] += t;
        cnt[r.c] += 1;
        g_pool.push_back(r.a);
        g_pool.push_back(r.b);
    }
    g_recs.clear();
    for (int c = 0; c < KC_COUNT; ++c) {
        cnt[c] += g_untimed[c];
        g_untimed[c] = 0;
    }
    for (int c = 0; c < n_classes && c < KC_COUNT; ++c) {
        total_ms[c] = ms[c];
        launches[c] = cnt[c];
        bytes[c] = g_bytes[c];
        flops[c] = g_flops[c];
    }
    for (int c = KC_COUNT; c < n_classes; ++c) {
        total_ms[c] = 0.0;
        launches[c] = 0;
        bytes[c] = flops[c] = 0.0;
    }
    for (int c = 0; c < KC_COUNT; ++c) g_bytes[c] = g_flops[c] = 0.0;
    return st;
}

const char *qs_profile_class_name(int c) { return (c >= 0 && c < KC_COUNT) ? kNames[c] : ""; }

int qs_profile_class_count(void) { return KC_COUNT; }

}  // extern "C"
