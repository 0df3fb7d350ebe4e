// extern "C" entry points of lsw.h: argument checks, then the internal calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <utility>
#include <vector>
#include <atomic>
#include <mutex>
#include <new>

#include "lsw_internal.cuh"

namespace lsw {

static thread_local char g_last_error[512];
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launch_counter() { return g_launches.load(std::memory_order_relaxed); }

namespace {
std::atomic<unsigned long long> g_replays{0};
}
void count_graph_replay() { g_replays.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::atomic<int> g_graphs{1};
}
bool graphs_enabled() { return g_graphs.load() != 0; }

void set_last_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

namespace {
struct TimerState {
    std::mutex mu;
    char family[64] = {0};
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<TimedSpan> captured;     // recorded into a graph being captured
    double ms = 0, bytes = 0, flops = 0;
    unsigned long long launches = 0;
} g_timer;

void drain_timer() {
    for (auto& pe : g_timer.pending) {
        float t = 0;
        cudaEventSynchronize(pe.second);
        if (cudaEventElapsedTime(&t, pe.first, pe.second) == cudaSuccess) g_timer.ms += t;
        cudaEventDestroy(pe.first);
        cudaEventDestroy(pe.second);
    }
    g_timer.pending.clear();
}
}  // namespace

KTimer::KTimer(const char* family, cudaStream_t st, double bytes, double flops) {
    std::lock_guard<std::mutex> lk(g_timer.mu);
    if (!g_timer.on || strncmp(family, g_timer.family, sizeof g_timer.family) != 0) return;
    // work being captured into a graph runs at each replay: its events
    // become nodes of the graph (see timer_take_captured)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return;
    captured_ = cs != cudaStreamCaptureStatusNone;
    st_ = st;
    bytes_ = bytes;
    flops_ = flops;
    cudaEventCreate(&e0_);
    cudaEventCreate(&e1_);
    // inside a capture, an external record node: the event is recorded at
    // every replay (a plain record would only order the capture's streams)
    cudaEventRecordWithFlags(e0_, st_, captured_ ? cudaEventRecordExternal : cudaEventRecordDefault);
}

KTimer::~KTimer() {
    if (!e0_) return;
    cudaEventRecordWithFlags(e1_, st_, captured_ ? cudaEventRecordExternal : cudaEventRecordDefault);
    std::lock_guard<std::mutex> lk(g_timer.mu);
    if (captured_) {
        g_timer.captured.push_back(TimedSpan{e0_, e1_, bytes_, flops_});
        return;
    }
    g_timer.pending.emplace_back(e0_, e1_);
    g_timer.bytes += bytes_;
    g_timer.flops += flops_;
    g_timer.launches += 1;
}

std::vector<TimedSpan> timer_take_captured() {
    std::lock_guard<std::mutex> lk(g_timer.mu);
    std::vector<TimedSpan> v;
    v.swap(g_timer.captured);
    return v;
}

// After a replay of the graph that holds the spans has finished: add each
// span's elapsed time (while the timer is still on).
void timer_harvest(const std::vector<TimedSpan>& spans) {
    if (spans.empty()) return;
    std::lock_guard<std::mutex> lk(g_timer.mu);
    if (!g_timer.on) return;
    for (const auto& sp : spans) {
        float t = 0;
        cudaEventSynchronize(sp.e1);
        if (cudaEventElapsedTime(&t, sp.e0, sp.e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        g_timer.ms += t;
        g_timer.bytes += sp.bytes;
        g_timer.flops += sp.flops;
        g_timer.launches += 1;
    }
}

void timer_release(std::vector<TimedSpan>& spans) {
    for (auto& sp : spans) {
        cudaEventDestroy(sp.e0);
        cudaEventDestroy(sp.e1);
    }
    spans.clear();
}

namespace {
constexpr int kPool = 8, kSlots = 8;
std::mutex g_pool_mu;
cudaStream_t g_pool[64][kSlots][kPool] = {};
thread_local int g_slot = 0;     // which pool this host thread forks onto
}  // namespace

void set_worker_slot(int slot) { g_slot = slot >= 0 && slot < kSlots ? slot : 0; }

Fork::Fork(cudaStream_t parent) : parent_(parent) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        for (int i = 0; i < kPool; ++i) {
            cudaStream_t* slot = (dev >= 0 && dev < 64) ? &g_pool[dev][g_slot][i] : nullptr;
            if (slot && !*slot) cudaStreamCreateWithFlags(slot, cudaStreamNonBlocking);
            streams_[i] = slot ? *slot : parent;
        }
    }
    cudaEventCreateWithFlags(&start_, cudaEventDisableTiming);
    cudaEventRecord(start_, parent_);
}

Fork::~Fork() {
    if (used_) join();
    if (start_) cudaEventDestroy(start_);
}

cudaStream_t Fork::child(int i) {
    const int k = i % kPool;
    if (!(used_ & (1u << k))) {
        cudaStreamWaitEvent(streams_[k], start_, 0);
        used_ |= 1u << k;
    }
    return streams_[k];
}

lsw_status Fork::join() {
    for (int k = 0; k < kPool; ++k) {
        if (!(used_ & (1u << k))) continue;
        cudaEvent_t e;
        LSW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        LSW_CUDA(cudaEventRecord(e, streams_[k]));
        LSW_CUDA(cudaStreamWaitEvent(parent_, e, 0));
        cudaEventDestroy(e);
    }
    used_ = 0;
    return LSW_OK;
}

lsw_status green_init(lsw_green* g, cudaStream_t st);
lsw_status noalloc_setup();
lsw_status contrast(const lsw_green* g, const double* vel, double* chi, cudaStream_t st);
lsw_status point_sources(const lsw_green* g, const int32_t* pos_host, int nsrc, int prec, void* u0,
                         cudaStream_t st);

}  // namespace lsw

namespace lsw {
namespace {
// Arithmetic-peak probe: eight independent fused multiply-add chains per
// thread, enough warps per SM to hide the pipeline latency.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(T* out, int iters, T a, T b) {
    T x0 = (T)threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
            x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
        }
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}

template <typename T>
lsw_status fma_peak(int iters, double* tflops, cudaStream_t st) {
    int dev = 0, sms = 0;
    LSW_CUDA(cudaGetDevice(&dev));
    LSW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;
    DevBuf out;
    LSW_TRY(out.alloc(sizeof(T) * (size_t)blocks * threads, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    LSW_CUDA(cudaEventCreate(&e0));
    LSW_CUDA(cudaEventCreate(&e1));
    k_fma_probe<T><<<blocks, threads, 0, st>>>(out.as<T>(), iters / 8 + 1, (T)0.999, (T)0.001);   // warm-up
    LSW_LAUNCH_CHECK();
    cudaEventRecord(e0, st);
    k_fma_probe<T><<<blocks, threads, 0, st>>>(out.as<T>(), iters, (T)0.999, (T)0.001);
    LSW_LAUNCH_CHECK();
    cudaEventRecord(e1, st);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    LSW_CUDA(err);
    const double flops = 2.0 * 64.0 * (double)iters * blocks * threads;
    *tflops = ms > 0.f ? flops / (ms * 1e-3) / 1e12 : 0.0;
    return LSW_OK;
}
}  // namespace
}  // namespace lsw

using namespace lsw;

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

static bool grid_ok(int n) { return n >= 1 && n <= 2048 && is_pow2(n); }

extern "C" {

uint64_t lsw_graph_replay_count(void) { return lsw::g_replays.load(); }

lsw_status lsw_set_graphs(int enable) {
    lsw::g_graphs.store(enable != 0 ? 1 : 0);
    return LSW_OK;
}


const char* lsw_status_string(lsw_status s) {
    switch (s) {
        case LSW_OK: return "ok";
        case LSW_ERR_INVALID_ARG: return "invalid argument";
        case LSW_ERR_UNSUPPORTED_SIZE: return "unsupported size (grid sides must be powers of two <= 2048)";
        case LSW_ERR_OOM: return "device allocation failed";
        case LSW_ERR_CUDA: return "CUDA runtime error";
        case LSW_ERR_NOT_CONVERGED: return "not converged within max_iter";
        case LSW_ERR_DIVERGED: return "diverged";
        case LSW_ERR_NUMERIC: return "NaN or Inf";
        case LSW_ERR_TIMEOUT: return "timeout";
        default: return "unknown status";
    }
}

// Last CUDA error text of the calling thread (not part of lsw.h's contract
// beyond diagnostics).
const char* lsw_last_error(void) { return g_last_error; }

uint64_t lsw_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

lsw_status lsw_kernel_timer_start(const char* family) {
    if (!family) return LSW_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_timer.mu);
    drain_timer();
    strncpy(g_timer.family, family, sizeof g_timer.family - 1);
    g_timer.on = true;
    g_timer.ms = g_timer.bytes = g_timer.flops = 0;
    g_timer.launches = 0;
    return LSW_OK;
}

lsw_status lsw_kernel_timer_read(double* ms, double* bytes, double* flops, uint64_t* launches) {
    std::lock_guard<std::mutex> lk(g_timer.mu);
    drain_timer();
    if (ms) *ms = g_timer.ms;
    if (bytes) *bytes = g_timer.bytes;
    if (flops) *flops = g_timer.flops;
    if (launches) *launches = g_timer.launches;
    return LSW_OK;
}

lsw_status lsw_kernel_timer_stop(void) {
    std::lock_guard<std::mutex> lk(g_timer.mu);
    drain_timer();
    g_timer.on = false;
    return LSW_OK;
}

lsw_status lsw_measure_peak(int kind, double* tflops, void* stream) {
    if (!tflops || (kind != 0 && kind != 1)) return LSW_ERR_INVALID_ARG;
    *tflops = 0.0;
    // about 20 ms of work at GB300 rates (78 TFLOP/s FP32, 1.25 FP64)
    return kind == 0 ? fma_peak<float>(8192, tflops, S(stream)) : fma_peak<double>(256, tflops, S(stream));
}

lsw_status lsw_mempool_usage(uint64_t* used_current, uint64_t* used_high, int reset_high) {
    int dev = 0;
    LSW_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    LSW_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    if (reset_high) {
        uint64_t zero = 0;
        LSW_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    uint64_t cur = 0, high = 0;
    LSW_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur));
    LSW_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high));
    if (used_current) *used_current = cur;
    if (used_high) *used_high = high;
    return LSW_OK;
}

lsw_status lsw_build_green(const lsw_grid* grid, void* stream, lsw_green** out) {
    if (!grid || !out) return LSW_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid_ok(grid->nz) || !grid_ok(grid->nx)) return LSW_ERR_UNSUPPORTED_SIZE;
    if (!(grid->h > 0) || !(grid->c0 > 0) || !(grid->freq_hz > 0) || !std::isfinite(grid->h) ||
        !std::isfinite(grid->c0) || !std::isfinite(grid->freq_hz))
        return LSW_ERR_INVALID_ARG;
    lsw_green* g = new (std::nothrow) lsw_green();
    if (!g) return LSW_ERR_OOM;
    cudaGetDevice(&g->device);
    {
        // Scratch comes from the device's default stream-ordered pool; keep
        // freed blocks cached there instead of unmapping them at every
        // synchronisation, so repeated calls do not pay for new mappings.
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, g->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    g->nz = grid->nz;
    g->nx = grid->nx;
    g->h = grid->h;
    g->c0 = grid->c0;
    g->freq = grid->freq_hz;
    g->k = 2.0 * M_PI * grid->freq_hz / grid->c0;
    lsw_status st = green_init(g, S(stream));
    if (st == LSW_OK) st = noalloc_setup();
    if (st != LSW_OK) {
        lsw_destroy_green(g);
        return st;
    }
    *out = g;
    return LSW_OK;
}

lsw_status lsw_destroy_green(lsw_green* g) {
    if (!g) return LSW_ERR_INVALID_ARG;
    if (g->table) cudaFree(g->table);
    if (g->tw64) cudaFree(g->tw64);
    if (g->tw32) cudaFree(g->tw32);
    free_spectrum(&g->full);
    delete g;
    return LSW_OK;
}

lsw_status lsw_green_table(const lsw_green* g, void* table, void* stream) {
    if (!g || !table) return LSW_ERR_INVALID_ARG;
    const size_t n = (size_t)(g->nz + 1) * (g->nx + 1);
    LSW_CUDA(cudaMemcpyAsync(table, g->table, n * sizeof(double2), cudaMemcpyDeviceToDevice, S(stream)));
    return LSW_OK;
}

lsw_status lsw_green_spectrum(const lsw_green* g, void* spec, void* stream) {
    if (!g || !spec) return LSW_ERR_INVALID_ARG;
    const size_t n = (size_t)(g->nz + 1) * (g->nx + 1);
    LSW_CUDA(cudaMemcpyAsync(spec, g->full.q64, n * sizeof(double2), cudaMemcpyDeviceToDevice, S(stream)));
    return LSW_OK;
}

lsw_status lsw_contrast(const lsw_green* g, const double* velocity, double* chi, void* stream) {
    if (!g || !velocity || !chi) return LSW_ERR_INVALID_ARG;
    return contrast(g, velocity, chi, S(stream));
}

lsw_status lsw_point_sources(const lsw_green* g, const int32_t* positions, int nsrc, int prec, void* u0,
                             void* stream) {
    if (!g || !positions || !u0 || nsrc <= 0) return LSW_ERR_INVALID_ARG;
    if (prec != LSW_C128 && prec != LSW_C64) return LSW_ERR_INVALID_ARG;
    return point_sources(g, positions, nsrc, prec, u0, S(stream));
}

lsw_status lsw_apply_operator(const lsw_green* g, int prec, const double* chi, const void* u, const void* u0,
                              void* y, int nbatch, int mode, void* stream) {
    if (!g || !chi || nbatch < 0) return LSW_ERR_INVALID_ARG;
    if (mode < LSW_OP_FORWARD || mode > LSW_OP_ADJOINT) return LSW_ERR_INVALID_ARG;
    if (prec != LSW_C128 && prec != LSW_C64) return LSW_ERR_INVALID_ARG;
    if (nbatch == 0) return LSW_OK;
    if (!u || !y || y == u || (u0 && y == u0)) return LSW_ERR_INVALID_ARG;
    if (mode != LSW_OP_FORWARD && mode != LSW_OP_RESIDUAL) u0 = nullptr;
    cudaStream_t st = S(stream);
    const long long n = (long long)g->nz * g->nx;
    OpGeom geo{g->nz, g->nx, chi, g->nz, nullptr, 1};
    DevBuf work;
    if (prec == LSW_C128) {
        LSW_TRY(work.alloc(sizeof(double2) * 2 * n * nbatch, st));
        return op_apply<double>(g, g->full, geo, mode, (const double2*)u, (const double2*)u0, (double2*)y, nbatch,
                                work.as<double2>(), st);
    }
    LSW_TRY(work.alloc(sizeof(float2) * 2 * n * nbatch, st));
    return op_apply<float>(g, g->full, geo, mode, (const float2*)u, (const float2*)u0, (float2*)y, nbatch,
                           work.as<float2>(), st);
}

}  // extern "C"
