// Event-based timing of tracked kernel classes (nk_prof_* in include/nk.h).

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/nk.h"
#include "nk_internal.h"

namespace {

struct Slot {
    cudaEvent_t start, stop;
    int cls;
    double work, exec;
    bool closed;
};

std::mutex g_mu;
bool g_on = false;
std::vector<Slot> g_slots;
size_t g_used = 0;
std::atomic<long long> g_launches{0};

}  // namespace

namespace nk {

void note_launch(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

cudaError_t allow_max_dynamic_smem(const void *func) {
    static std::mutex mu;
    static std::vector<std::pair<const void *, int>> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    for (auto &d : done)
        if (d.first == func && d.second == dev) return cudaSuccess;
    int optin = 0;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
    done.emplace_back(func, dev);
    return cudaSuccess;
}

int prof_begin(int cls, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return -1;
    if (g_used == g_slots.size()) {
        Slot s{};
        if (cudaEventCreate(&s.start) != cudaSuccess || cudaEventCreate(&s.stop) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
        g_slots.push_back(s);
    }
    Slot &s = g_slots[g_used];
    s.cls = cls;
    s.work = 0.0;
    s.exec = 0.0;
    s.closed = false;
    if (cudaEventRecord(s.start, st) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (int)g_used++;
}

void prof_end(int slot, cudaStream_t st, double work, double executed) {
    if (slot < 0) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if ((size_t)slot >= g_used) return;
    Slot &s = g_slots[slot];
    if (cudaEventRecord(s.stop, st) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    s.work = work;
    s.exec = executed < 0.0 ? work : executed;
    s.closed = true;
}

}  // namespace nk

extern "C" {

int64_t nk_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

nk_status nk_prof_enable(int32_t on) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    g_used = 0;
    return NK_OK;
}

nk_status nk_prof_read(int32_t cls, double *ms, int64_t *launches, double *work) {
    if (cls < 0 || cls >= NK_PROF_N || !ms || !launches || !work) return NK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    double t = 0.0, w = 0.0;
    int64_t n = 0;
    for (size_t i = 0; i < g_used; ++i) {
        Slot &s = g_slots[i];
        if (s.cls != cls || !s.closed) continue;
        if (cudaEventSynchronize(s.stop) != cudaSuccess) return NK_ERR_CUDA;
        float e = 0.f;
        if (cudaEventElapsedTime(&e, s.start, s.stop) != cudaSuccess) return NK_ERR_CUDA;
        t += e;
        w += s.work;
        ++n;
    }
    *ms = t;
    *launches = n;
    *work = w;
    return NK_OK;
}

nk_status nk_prof_read_executed(int32_t cls, double *executed) {
    if (cls < 0 || cls >= NK_PROF_N || !executed) return NK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    double x = 0.0;
    for (size_t i = 0; i < g_used; ++i)
        if (g_slots[i].cls == cls && g_slots[i].closed) x += g_slots[i].exec;
    *executed = x;
    return NK_OK;
}

nk_status nk_prof_trace(int32_t max, int32_t *cls, double *t0_ms, double *t1_ms, int32_t *n_out) {
    if (!n_out || max < 0 || (max > 0 && (!cls || !t0_ms || !t1_ms))) return NK_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mu);
    int32_t n = 0;
    cudaEvent_t first = nullptr;
    for (size_t i = 0; i < g_used; ++i) {
        Slot &s = g_slots[i];
        if (!s.closed) continue;
        if (cudaEventSynchronize(s.stop) != cudaSuccess) return NK_ERR_CUDA;
        if (!first) first = s.start;
        if (n < max) {
            float a = 0.f, b = 0.f;
            if (cudaEventElapsedTime(&a, first, s.start) != cudaSuccess ||
                cudaEventElapsedTime(&b, first, s.stop) != cudaSuccess)
                return NK_ERR_CUDA;
            cls[n] = s.cls;
            t0_ms[n] = a;
            t1_ms[n] = b;
        }
        ++n;
    }
    *n_out = n;
    return NK_OK;
}

}  // extern "C"
