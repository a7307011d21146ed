// Diagnostic timing of the library's tensor-core GEMM launches (no
// counterpart in the paper; it exists so a caller can see how long the
// dominant kernel of a call takes on the device, apart from the pre-passes
// around it).  While timing is on, every GEMM launcher records a CUDA event
// before and after its launch on the launch stream; reading synchronises on
// those events and sums their elapsed times.
#include <mutex>
#include <vector>

#include "internal.h"

namespace moa {
namespace {

struct EventPair {
    cudaEvent_t a = nullptr, b = nullptr;
};

std::mutex g_mu;
bool g_on = false;
std::vector<EventPair> g_done;  // pairs recorded since the last start
std::vector<EventPair> g_free;  // recycled pairs (created on the device that was current then)
int g_dev = -1;                 // device the pairs belong to

void release_all_locked() {
    for (auto &p : g_done) g_free.push_back(p);
    g_done.clear();
}

void destroy_all_locked() {
    release_all_locked();
    for (auto &p : g_free) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    g_free.clear();
}

}  // namespace

GemmTimer::GemmTimer(cudaStream_t s) : stream_(s) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_on) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g_dev) return;  // timing covers the device it started on
    EventPair p;
    if (!g_free.empty()) {
        p = g_free.back();
        g_free.pop_back();
    } else if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    if (cudaEventRecord(p.a, s) != cudaSuccess) {
        g_free.push_back(p);
        return;
    }
    a_ = p.a;
    b_ = p.b;
}

void GemmTimer::done() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cudaEventRecord(b_, stream_) == cudaSuccess && g_on) {
        g_done.push_back(EventPair{a_, b_});
    } else {
        g_free.push_back(EventPair{a_, b_});
    }
    a_ = b_ = nullptr;
}

GemmTimer::~GemmTimer() { done(); }

}  // namespace moa

using namespace moa;

extern "C" moa_status moa_kernel_timing(int enable) {
    std::lock_guard<std::mutex> lk(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MOA_ERR_CUDA;
    if (enable) {
        if (g_dev != dev) {  // pairs of another device are not reused
            if (g_dev >= 0) {
                int cur = dev;
                cudaSetDevice(g_dev);
                cudaDeviceSynchronize();
                destroy_all_locked();
                cudaSetDevice(cur);
            }
            g_dev = dev;
        }
        release_all_locked();
        g_on = true;
    } else {
        g_on = false;
    }
    return MOA_OK;
}

extern "C" moa_status moa_kernel_timing_read(int64_t *launches, double *total_ms) {
    if (!launches || !total_ms) return MOA_ERR_NULL;
    std::lock_guard<std::mutex> lk(g_mu);
    double sum = 0.0;
    for (auto &p : g_done) {
        float ms = 0.0f;
        if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess)
            return MOA_ERR_CUDA;
        sum += ms;
    }
    *launches = (int64_t)g_done.size();
    *total_ms = sum;
    return MOA_OK;
}
