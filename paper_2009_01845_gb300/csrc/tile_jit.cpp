// Pass kernels specialised for one pass structure, compiled at run time.
//
// The generic tiled kernel decodes every op of a pass from its parameters at
// run time (a switch per op, loops over active bits and diagonal factors,
// constant loads), which costs about as many instructions as the gates'
// arithmetic. A specialised kernel is the same device pieces (tile_device.cuh)
// called in a straight line, with the descriptor's structure (ops, bits,
// stage maps, swizzles) as a `__device__ constexpr` object: each op's decode
// and its loop bounds fold away at compile time, and the compiler can
// schedule across op boundaries. The pass's values (matrix entries, diagonal
// factors) are a kernel parameter block, so passes that differ only in their
// angles (the steps of a Trotter evolution, the parameter sets of a
// variational circuit) share one kernel.
//
// The source is generated here, compiled with NVRTC for the device's
// architecture, loaded as a CUDA library and cached by structure (the bytes
// of the descriptor with its run-time pointers and values cleared; two passes
// share a kernel only if those bytes are equal). When a kernel is compiled is a
// process-wide policy (qs_jit_set_policy): never; in the background once a
// pass is launched a second time (the default: one-off circuits never pay for
// a compile, repeated ones switch to the specialised kernel when it is ready);
// in the background at the first launch; or before the first launch. Until a
// pass's kernel is ready the generic kernel runs it. Compiles run on worker
// threads (NVRTC only, no CUDA calls); libraries are loaded by the launching
// thread, never while its stream is being captured into a graph.
#include <nvrtc.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "prof.h"
#include "tiled.h"

namespace qsim {

// Texts of the headers the generated source includes (written by the build
// from include/qsim.h and this directory's device.cuh, tiled.h,
// tile_device.cuh).
#include "jit_headers.inc"

namespace jit_detail {

// stand-ins for the system headers the device headers include; the fixed-width
// types have the host's widths (LP64)
const char *kStdintStub =
    "#pragma once\n"
    "typedef signed char int8_t; typedef unsigned char uint8_t;\n"
    "typedef short int16_t; typedef unsigned short uint16_t;\n"
    "typedef int int32_t; typedef unsigned int uint32_t;\n"
    "typedef long long int64_t; typedef unsigned long long uint64_t;\n"
    "typedef decltype(sizeof(0)) size_t;\n";

enum JitState { JS_NEW = 0, JS_QUEUED, JS_COMPILING, JS_READY, JS_FAILED };

// key flags: the arithmetic in bits 0 and 2 (complex64, complex128 in FP64 or
// in double-float), the values compiled in (bit 1)
template <typename R> constexpr unsigned char kTypeCode = 0;
template <> constexpr unsigned char kTypeCode<double> = 1;
template <> constexpr unsigned char kTypeCode<dd> = 4;
constexpr unsigned char kKeyFolded = 2;

constexpr int kMaxEntries = 1024;  // distinct passes tracked per process

struct JitEntry {
    std::vector<unsigned char> key;  // flags byte + normalised descriptor bytes
    int type = 0;                    // arithmetic: kTypeCode<R>
    int state = JS_NEW;
    long long hits = 0;
    std::vector<char> cubin;
    std::string log;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kern = nullptr;
    int blocks = 0;  // resident CTAs on the device (grid size)
    size_t smem = 0;
    bool load_failed = false;
};

struct JitGlobal {
    std::mutex mu;
    std::condition_variable cv, idle;
    std::unordered_map<uint64_t, std::vector<std::shared_ptr<JitEntry>>> table;
    std::deque<std::shared_ptr<JitEntry>> queue;
    std::vector<std::thread> workers;
    int busy = 0;
    int entries = 0;
    std::unordered_map<uint64_t, int> full_seen;  // launches per exact pass (by hash)
    bool stop = false;
    std::atomic<int> policy{-1};
    std::atomic<long long> jit_launches{0}, generic_launches{0}, compiled{0}, failed{0};
    std::atomic<long long> compile_us{0};
    std::string arch;  // e.g. "sm_103a"
    bool exit_hook_after_compile = false;
};

// Never destroyed: worker threads may still use it while the process exits.
JitGlobal &G() {
    static JitGlobal *g = new JitGlobal();
    return *g;
}

// At exit: no new compile starts, the ones in flight finish, the workers end.
// (A compile still inside NVRTC while NVRTC's own exit-time destructors run
// would crash the exit.) Registered when the workers start and again after the
// first compile completes, so that it runs before whatever NVRTC registered
// on first use (exit handlers run in reverse order of registration).
void jit_at_exit() {
    JitGlobal &g = G();
    std::vector<std::thread> ws;
    {
        std::lock_guard<std::mutex> lk(g.mu);
        if (g.stop) return;
        g.stop = true;
        g.queue.clear();
        ws.swap(g.workers);
    }
    g.cv.notify_all();
    for (auto &t : ws)
        if (t.joinable()) t.join();
}

thread_local int t_policy_override = -1;

int policy_now() {
    if (t_policy_override >= 0) return t_policy_override;
    JitGlobal &g = G();
    int p = g.policy.load();
    if (p < 0) {
        p = QS_JIT_TIERED;
        if (const char *e = std::getenv("QSIM_JIT")) {
            if (!std::strncmp(e, "off", 3)) p = QS_JIT_OFF;
            else if (!std::strncmp(e, "eager", 5)) p = QS_JIT_EAGER;
            else if (!std::strncmp(e, "sync", 4)) p = QS_JIT_SYNC;
            if (std::strstr(e, "+fold")) p |= QS_JIT_FOLD;
        }
        int expect = -1;
        g.policy.compare_exchange_strong(expect, p);
        p = g.policy.load();
    }
    return p;
}

uint64_t fnv(const unsigned char *b, size_t n) {
    uint64_t h = 1469598103934665603ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
    return h;
}

// ------------------------------------------------------------------ source generation
struct Src {
    std::string s;
    void f(const char *fmt, ...) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        const int n = std::vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        if (n > 0) s.append(buf, (size_t)std::min(n, (int)sizeof(buf) - 1));
    }
};

void real_lit(Src &o, float v) { o.f("%af", (double)v); }
void real_lit(Src &o, double v) { o.f("%a", v); }
template <typename R> void cplx_lit(Src &o, const V<R> &v) {
    if constexpr (is_dd<R>) {
        // the paired layout: {{re.h, im.h}, {re.l, im.l}}
        o.f("{{%af,%af},{%af,%af}}", (double)v.h.x, (double)v.h.y, (double)v.l.x, (double)v.l.y);
    } else {
        o.s += "{";
        real_lit(o, v.x);
        o.s += ",";
        real_lit(o, v.y);
        o.s += "}";
    }
}
template <typename T> void int_list(Src &o, const T *a, int n) {
    o.s += "{";
    for (int i = 0; i < n; ++i) o.f(i ? ",%lld" : "%lld", (long long)a[i]);
    o.s += "}";
}

// index one past the last element of a[] that is not all zero bytes
template <typename T> int used(const T *a, int n) {
    static const T z{};
    while (n > 0 && std::memcmp(&a[n - 1], &z, sizeof(T)) == 0) --n;
    return n;
}

// folded: the pass's values are compiled in too (kP holds them); otherwise
// they come from the value block v at run time
template <typename R> std::string generate(const TileParams<R> &P, bool folded) {
    constexpr int RB = TileCfg<R>::RB;
    constexpr int WB = TileCfg<R>::WB;
    const char *RT = is_dd<R> ? "dd" : sizeof(R) == 4 ? "float" : "double";
    Src o;
    o.s.reserve(1 << 17);
    o.s += "#include \"tile_device.cuh\"\nusing namespace qsim;\n";
    o.f("__device__ constexpr TileParams<%s> kP = {\n", RT);
    o.f(".n = %d, .k = %d, .n_stages = %d, .n_free = %d, .total_tiles = %lluull,\n", P.n, P.k, P.n_stages, P.n_free,
        (unsigned long long)P.total_tiles);
    o.s += ".tins = {";
    int_list(o, P.tins.pos, (int)(sizeof(P.tins.pos) / sizeof(P.tins.pos[0])));
    o.f(", %d},\n.gbit = ", (int)P.tins.count);
    int_list(o, P.gbit, 16);
    o.f(",\n.pmat = nullptr, .pm_stride = %uu, .n_grad = %d, .gpart = nullptr,\n.gslot = ", P.pm_stride, P.n_grad);
    int_list(o, P.gslot, kTileMaxGrad);
    o.f(",\n.ising = nullptr, .ising_stride = %uu, .nq = %d, .ising_thr = nullptr, .ising_thr_stride = %uu,\n",
        P.ising_stride, P.nq, P.ising_thr_stride);
    o.f(".tile_mask = %lluull,\n.dfac = {\n", (unsigned long long)P.tile_mask);
    const int ndf = used(P.dfac, kTileMaxDFac);
    for (int i = 0; i < ndf; ++i) {
        const TileDFac<R> &d = P.dfac[i];
        o.f("{%u,%u,%u,%u,%uu,%lluull,%lluull,", d.type, d.tkind, d.a, d.mr, d.mt, (unsigned long long)d.mo,
            (unsigned long long)d.tmask);
        cplx_lit<R>(o, d.v0);
        o.s += ",";
        cplx_lit<R>(o, d.v1);
        o.s += ",";
        cplx_lit<R>(o, d.v2);
        o.s += "},\n";
    }
    o.s += "},\n.st = {\n";
    for (int i = 0; i < P.n_stages; ++i) {
        const TileStage &st = P.st[i];
        o.s += "{";
        int_list(o, st.rloc, 6);
        o.s += ",";
        int_list(o, st.wloc, 3);
        o.s += ",";
        int_list(o, st.lloc, 5);
        o.s += ",";
        int_list(o, st.fcol, 9);
        o.f(",%u,%u,", st.need_lt, st.rflip);
        int_list(o, st.rw, 6);
        o.s += ",";
        int_list(o, st.rr, 6);
        o.f(",%u,%u},\n", st.op_begin, st.op_end);
    }
    o.s += "},\n.op = {\n";
    const int nops = used(P.op, kTileMaxOps);
    for (int i = 0; i < nops; ++i) {
        const TileOp &op = P.op[i];
        o.f("{%u,%u,%u,%u,%u,%u,%u,%u,%uu,%uu,%lluull,%lluull},\n", op.type, op.a, op.b, op.tkind, op.mr, op.pm,
            op.gl, op.fx, op.mt, op.m, (unsigned long long)op.mo, (unsigned long long)op.tmask);
    }
    o.s += "},\n.mat = {\n";
    const int nmat = used(P.mat, kTileMaxMat);
    for (int i = 0; i < nmat; ++i) {
        cplx_lit<R>(o, P.mat[i]);
        o.s += (i % 4 == 3) ? ",\n" : ",";
    }
    o.s += "}};\n\n";
    // the kernel: the generic kernel's loop over stages and ops, unrolled here
    const int NT = 32 << WB;
    o.f("extern \"C\" __global__ void __launch_bounds__(%d, %d) qs_tile_pass(V<%s> *__restrict__ psi,\n"
        "    const __grid_constant__ TilePtrs<%s> q, const __grid_constant__ TileVals<%s> v) {\n",
        NT, TileCfg<R>::kMinBlocks, RT, RT, RT);
    o.f("  using R = %s;\n  constexpr int RB = %d, NW = %d;\n", RT, RB, 1 << WB);
    o.s +=
        "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
        "  uint32_t *tab = reinterpret_cast<uint32_t *>(smem_raw + (sizeof(V<R>) << kP.k));\n"
        "  uint16_t *ltab = reinterpret_cast<uint16_t *>(tab + kP.n_stages * (NW * 32));\n"
        "  __shared__ GradT<R> gsm[kTileMaxGrad][NW];\n"
        "  __shared__ V<R> s_e[16];\n"
        "  __shared__ V<R> s_qp[1 << RB];\n"
        "  const TileScratch<R> sc{gsm, s_e, s_qp};\n"
        "  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;\n"
        "  V<R> a[1 << RB];\n"
        "  tile_tables<R, RB>(kP, tab, ltab, lane, warp);\n"
        "  for (uint64_t t = blockIdx.x; t < kP.total_tiles; t += gridDim.x) {\n"
        "    const uint64_t tbase = tile_base<R>(kP, t);\n"
        "    tile_load<R, RB>(a, psi, kP, tbase, lane, warp);\n";
    for (int s = 0; s < P.n_stages; ++s) {
        const TileStage &st = P.st[s];
        if (s > 0) o.f("    tile_transpose<R, RB>(a, smem_raw, tab, kP, %d);\n", s);
        o.s += "    {\n";
        if (st.need_lt) o.f("      const uint32_t lt = ltab[%d * (NW * 32) + threadIdx.x];\n", s);
        else o.s += "      const uint32_t lt = 0u;\n";
        for (int op = st.op_begin; op < st.op_end; ++op)
            o.f("      tile_op<R, RB, 2>(a, kP, %s, q, %d, kP.st[%d], t, tbase, lt, lane, warp, sc);\n",
                folded ? "kP.mat, kP.dfac" : "v.mat, v.dfac", op, s);
        o.s += "    }\n";
    }
    o.s += "    tile_store<R, RB>(psi, a, kP, tbase, lane, warp);\n";
    if (P.n_grad > 0) o.s += "    tile_grad_flush<R>(kP, q, t, sc);\n";
    o.s += "  }\n}\n";
    return o.s;
}

// ------------------------------------------------------------------ compile
bool nvrtc_compile(const std::string &src, const std::string &arch, std::vector<char> *cubin, std::string *log) {
    const char *hdr_src[] = {kJitSrc_qsim_h, kJitSrc_device_cuh, kJitSrc_tiled_h, kJitSrc_tile_device_cuh,
                             kStdintStub,    kStdintStub,        "",             ""};
    const char *hdr_name[] = {"qsim.h",   "device.cuh", "tiled.h",        "tile_device.cuh",
                              "stdint.h", "cstdint",    "cuda_runtime.h", "stddef.h"};
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "qs_tile_pass.cu", 8, hdr_src, hdr_name) != NVRTC_SUCCESS) {
        *log = "nvrtcCreateProgram failed";
        return false;
    }
    const std::string a = "--gpu-architecture=" + arch;
    // -default-device: the headers' unannotated declarations (the C-ABI, host
    // helpers) are taken as device functions; none is called
    static const bool verbose = std::getenv("QSIM_JIT_VERBOSE") != nullptr;
    const char *opts[] = {a.c_str(), "-std=c++20", "-default-device", "-DQSIM_PASS_KERNEL=1", "--ptxas-options=-v"};
    const nvrtcResult r = nvrtcCompileProgram(prog, verbose ? 5 : 4, opts);
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    if (ls > 1) {
        log->resize(ls);
        nvrtcGetProgramLog(prog, &(*log)[0]);
    }
    bool ok = r == NVRTC_SUCCESS;
    if (ok) {
        size_t n = 0;
        ok = nvrtcGetCUBINSize(prog, &n) == NVRTC_SUCCESS && n > 0;
        if (ok) {
            cubin->resize(n);
            ok = nvrtcGetCUBIN(prog, cubin->data()) == NVRTC_SUCCESS;
        }
    } else if (log->empty()) {
        *log = nvrtcGetErrorString(r);
    }
    nvrtcDestroyProgram(&prog);
    return ok;
}

template <typename R> std::string generate_from_key(const std::vector<unsigned char> &key) {
    TileParams<R> P;
    std::memcpy(&P, key.data() + 1, sizeof(P));
    return generate<R>(P, (key[0] & kKeyFolded) != 0);
}

void compile_entry(const std::shared_ptr<JitEntry> &e, const std::string &arch) {
    const auto t0 = std::chrono::steady_clock::now();
    const std::string src = e->type == kTypeCode<dd>       ? generate_from_key<dd>(e->key)
                            : e->type == kTypeCode<double> ? generate_from_key<double>(e->key)
                                                           : generate_from_key<float>(e->key);
    std::vector<char> cubin;
    std::string log;
    const bool ok = nvrtc_compile(src, arch, &cubin, &log);
    const long long us =
        std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
    JitGlobal &g = G();
    g.compile_us += us;
    std::lock_guard<std::mutex> lk(g.mu);
    if (ok) {
        e->cubin.swap(cubin);
        e->state = JS_READY;
        ++g.compiled;
    } else {
        e->log = log;
        e->state = JS_FAILED;
        ++g.failed;
    }
    if (std::getenv("QSIM_JIT_VERBOSE"))
        std::fprintf(stderr, "[qsim jit] %s in %.2f s (%zu source bytes)\n%s\n", ok ? "compiled" : "FAILED", us * 1e-6,
                     src.size(), log.c_str());
}

void worker_loop() {
    JitGlobal &g = G();
    while (true) {
        std::shared_ptr<JitEntry> e;
        std::string arch;
        {
            std::unique_lock<std::mutex> lk(g.mu);
            g.cv.wait(lk, [&] { return g.stop || !g.queue.empty(); });
            if (g.stop) return;
            e = g.queue.front();
            g.queue.pop_front();
            e->state = JS_COMPILING;
            ++g.busy;
            arch = g.arch;
        }
        compile_entry(e, arch);
        bool hook = false;
        {
            std::lock_guard<std::mutex> lk(g.mu);
            --g.busy;
            if (!g.exit_hook_after_compile) hook = g.exit_hook_after_compile = true;
        }
        if (hook) std::atexit(jit_at_exit);
        g.idle.notify_all();
    }
}

// callers hold g.mu
void start_workers(JitGlobal &g) {
    if (!g.workers.empty() || g.stop) return;
    std::atexit(jit_at_exit);
    unsigned hw = std::thread::hardware_concurrency();
    const int n = (int)std::max(1u, std::min(8u, hw > 2 ? hw / 2 : 1u));
    for (int i = 0; i < n; ++i) g.workers.emplace_back(worker_loop);
}

qs_status set_arch(JitGlobal &g, int device) {
    if (!g.arch.empty()) return QS_OK;
    int major = 0, minor = 0;
    QS_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
    QS_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
    // the library is built for sm_103a only; specialised kernels match it
    g.arch = (major == 10 && minor == 3) ? "sm_103a" : "";
    return QS_OK;
}

// load a ready entry's library (launching thread, stream not capturing)
template <typename R> qs_status load_entry(JitEntry &e, int device) {
    QS_CUDA_TRY(cudaLibraryLoadData(&e.lib, e.cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0));
    QS_CUDA_TRY(cudaLibraryGetKernel(&e.kern, e.lib, "qs_tile_pass"));
    TileParams<R> P;
    std::memcpy(&P, e.key.data() + 1, sizeof(P));
    e.smem = tile_smem_bytes<R>(P.k, P.n_stages);
    QS_CUDA_TRY(cudaKernelSetAttributeForDevice(e.kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)e.smem,
                                                device));
    int bps = 0, sms = 0;
    QS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void *)e.kern, 32 << TileCfg<R>::WB,
                                                              e.smem));
    QS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    e.blocks = std::max(1, bps) * sms;
    std::vector<char>().swap(e.cubin);
    return QS_OK;
}

// per-thread host buffer for a launch's value block (too large for the stack
// of every caller)
template <typename R> unsigned char *vals_buf() {
    thread_local std::vector<unsigned char> buf(sizeof(TileVals<R>));
    return buf.data();
}

}  // namespace jit_detail

using namespace jit_detail;

// Launch the pass on its specialised kernel if one is (or, by the policy, can
// now be made) ready; *launched = false leaves the launch to the generic
// kernel. Counts the launch either way.
template <typename R>
qs_status tile_jit_launch_t(qs_state *s, const TileParams<R> &p, bool *launched) {
    *launched = false;
    JitGlobal &g = G();
    const int policy_raw = policy_now();
    const int policy = policy_raw & ~QS_JIT_FOLD;
    const bool fold = (policy_raw & QS_JIT_FOLD) != 0;
    if (policy == QS_JIT_OFF) {
        ++g.generic_launches;
        return QS_OK;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    QS_CUDA_TRY(cudaStreamIsCapturing(s->stream, &cs));
    const bool capturing = cs != cudaStreamCaptureStatusNone;
    // keys: flags (kTypeCode, kKeyFolded: values compiled in), then the
    // descriptor with its run-time pointers and the Ising op's tau (which only
    // the table kernel reads) cleared; the structure key also clears the
    // values (matrix entries, diagonal factors)
    std::vector<unsigned char> full(1 + sizeof(TileParams<R>));
    full[0] = kTypeCode<R> | kKeyFolded;
    {
        TileParams<R> &k = *reinterpret_cast<TileParams<R> *>(full.data() + 1);
        std::memcpy(&k, &p, sizeof(p));
        k.pmat = nullptr;
        k.gpart = nullptr;
        k.ising = nullptr;
        k.ising_thr = nullptr;
        for (int o = 0; o < kTileMaxOps; ++o)
            if (k.op[o].type == TOP_ISING) k.op[o].tmask = 0;
    }
    std::vector<unsigned char> key(full);
    key[0] = kTypeCode<R>;
    {
        TileParams<R> &k = *reinterpret_cast<TileParams<R> *>(key.data() + 1);
        std::memset(k.mat, 0, sizeof(k.mat));
        for (int f = 0; f < kTileMaxDFac; ++f) {
            std::memset(&k.dfac[f].v0, 0, sizeof(k.dfac[f].v0));
            std::memset(&k.dfac[f].v1, 0, sizeof(k.dfac[f].v1));
            std::memset(&k.dfac[f].v2, 0, sizeof(k.dfac[f].v2));
        }
    }
    const uint64_t h = fnv(key.data(), key.size());
    const uint64_t hf = fnv(full.data(), full.size());
    std::shared_ptr<JitEntry> e;
    bool compile_here = false;
    {
        std::lock_guard<std::mutex> lk(g.mu);
        if (!capturing) QS_TRY(set_arch(g, s->device));
        if (g.arch.empty()) {
            ++g.generic_launches;
            return QS_OK;
        }
        // second tier: a pass repeated with the same values gets a kernel with
        // its values compiled in as well (a few percent faster); it is queued
        // once the exact pass has been launched twice (counted by hash; the
        // entry itself compares whole keys)
        std::shared_ptr<JitEntry> ef;
        if (policy != QS_JIT_OFF) {
            // existing folded kernels are used whatever the flag; new ones are
            // made only under QS_JIT_FOLD
            auto fb = g.table.find(hf);
            if (fb != g.table.end())
                for (auto &c : fb->second)
                    if (c->key == full) {
                        ef = c;
                        break;
                    }
            if (!ef && fold && !capturing && !g.stop && ++g.full_seen[hf] >= 2 && g.entries < kMaxEntries) {
                ++g.entries;
                ef = std::make_shared<JitEntry>();
                ef->key = full;
                ef->type = kTypeCode<R>;
                ef->state = JS_QUEUED;
                g.table[hf].push_back(ef);
                start_workers(g);
                g.queue.push_back(ef);
                g.cv.notify_one();
                if (g.full_seen.size() > (1u << 20)) g.full_seen.clear();
            }
            if (ef && ef->state == JS_READY && !ef->kern && !ef->load_failed && !capturing) {
                if (load_entry<R>(*ef, s->device) != QS_OK) {
                    ef->load_failed = true;
                    clear_error();
                    ++g.failed;
                }
            }
            if (ef && ef->kern) e = ef;
        }
        auto &bucket = g.table[h];
        for (auto &c : bucket)
            if (!e && c->key == key) {
                e = c;
                break;
            }
        if (!e) {
            // a bounded cache: past kMaxEntries distinct passes (e.g. a long
            // Trotter evolution, whose every step has its own angles) new
            // passes stay on the generic kernel
            if (g.entries >= kMaxEntries) {
                ++g.generic_launches;
                return QS_OK;
            }
            ++g.entries;
            e = std::make_shared<JitEntry>();
            e->key = std::move(key);
            e->type = kTypeCode<R>;
            bucket.push_back(e);
        }
        ++e->hits;
        if (e->state == JS_NEW && !capturing && !g.stop) {
            if (policy == QS_JIT_SYNC) {
                e->state = JS_COMPILING;
                compile_here = true;
            } else if (policy == QS_JIT_EAGER || e->hits >= 2) {
                e->state = JS_QUEUED;
                start_workers(g);
                g.queue.push_back(e);
                g.cv.notify_one();
            }
        }
    }
    if (compile_here) {
        compile_entry(e, g.arch);
        g.idle.notify_all();
    }
    if (policy == QS_JIT_SYNC && !capturing) {
        // a pass queued earlier under another policy: wait for it
        std::unique_lock<std::mutex> lk(g.mu);
        g.idle.wait(lk, [&] { return g.stop || (e->state != JS_QUEUED && e->state != JS_COMPILING); });
    }
    {
        std::lock_guard<std::mutex> lk(g.mu);
        if (e->state == JS_READY && !e->kern && !e->load_failed && !capturing) {
            const qs_status st = load_entry<R>(*e, s->device);
            if (st != QS_OK) {
                e->load_failed = true;
                clear_error();
                ++g.failed;
            }
        }
        if (!e->kern) {
            ++g.generic_launches;
            return QS_OK;
        }
    }
    const uint64_t grid = std::min<uint64_t>(p.total_tiles, (uint64_t)e->blocks);
    if (grid == 0) {
        *launched = true;
        return QS_OK;
    }
    V<R> *psi = (V<R> *)s->data;
    TilePtrs<R> q{p.pmat, p.gpart, p.ising_thr};
    TileVals<R> &vals = *reinterpret_cast<TileVals<R> *>(vals_buf<R>());
    std::memcpy(vals.mat, p.mat, sizeof(vals.mat));
    std::memcpy(vals.dfac, p.dfac, sizeof(vals.dfac));
    void *args[] = {&psi, &q, &vals};
    QS_CUDA_TRY(cudaLaunchKernel((const void *)e->kern, dim3((unsigned)grid), dim3(32 << TileCfg<R>::WB), args,
                                 e->smem, s->stream));
    ++g.jit_launches;
    *launched = true;
    return QS_OK;
}

template qs_status tile_jit_launch_t<float>(qs_state *, const TileParams<float> &, bool *);
template qs_status tile_jit_launch_t<double>(qs_state *, const TileParams<double> &, bool *);
template qs_status tile_jit_launch_t<dd>(qs_state *, const TileParams<dd> &, bool *);

int jit_policy() { return policy_now(); }

// Run f with this thread's policy set to `policy` (a plan's autotuning runs
// specialise its passes before the plan captures them).
qs_status with_jit_policy(int policy, const std::function<qs_status()> &f) {
    const int old = t_policy_override;
    t_policy_override = policy;
    const qs_status st = f();
    t_policy_override = old;
    return st;
}

}  // namespace qsim

using namespace qsim;

extern "C" qs_status qs_jit_set_policy(int policy) {
    clear_error();
    const int base = policy & ~QS_JIT_FOLD;
    if (base < QS_JIT_OFF || base > QS_JIT_SYNC || (policy & ~(QS_JIT_FOLD | 3))) {
        set_error("unknown specialisation policy %d", policy);
        return QS_ERR_ARG;
    }
    G().policy.store(policy);
    return QS_OK;
}

extern "C" qs_status qs_jit_wait(void) {
    clear_error();
    JitGlobal &g = G();
    std::unique_lock<std::mutex> lk(g.mu);
    g.idle.wait(lk, [&] { return (g.queue.empty() || g.workers.empty()) && g.busy == 0; });
    return QS_OK;
}

extern "C" qs_status qs_jit_cancel(void) {
    clear_error();
    JitGlobal &g = G();
    std::unique_lock<std::mutex> lk(g.mu);
    for (auto &e : g.queue) e->state = JS_NEW;  // may be queued again by a later launch
    g.queue.clear();
    g.idle.wait(lk, [&] { return g.busy == 0; });
    return QS_OK;
}

extern "C" qs_status qs_jit_stats(long long *specialised_launches, long long *generic_launches, long long *compiled,
                                  long long *failed, double *compile_seconds) {
    clear_error();
    JitGlobal &g = G();
    if (specialised_launches) *specialised_launches = g.jit_launches.load();
    if (generic_launches) *generic_launches = g.generic_launches.load();
    if (compiled) *compiled = g.compiled.load();
    if (failed) *failed = g.failed.load();
    if (compile_seconds) *compile_seconds = g.compile_us.load() * 1e-6;
    return QS_OK;
}
