// gq_alloc.cu -- caching device allocator behind every dbuf of the library.
#include <mutex>
#include <vector>

#include "gq_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kClasses = 48;   // 2^8 .. 2^55 bytes

struct Pool {
    std::mutex mu;
    std::vector<void *> free_list[kMaxDevices][kClasses];
    size_t cached = 0;
};

Pool &pool() {
    static Pool *P = new Pool;   // never destroyed: the driver may already be gone at exit
    return *P;
}

int size_class(size_t bytes, size_t *cap) {
    int c = 0;
    size_t s = 256;
    while (s < bytes && c < kClasses - 1) {
        s <<= 1;
        ++c;
    }
    *cap = s;
    return c;
}

// Frees the cached blocks of one device.  Devices without cached blocks are
// not touched: selecting a device that does not exist would leave an error
// for the next launch check to find, and selecting one that does would start
// a context on it.
void release_device_locked(Pool &P, int dev) {
    bool any = false;
    for (int c = 0; c < kClasses && !any; ++c) any = !P.free_list[dev][c].empty();
    if (!any) return;
    int cur = 0;
    if (cudaGetDevice(&cur) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) {
        (void)cudaGetLastError();   // clear it: the blocks stay cached
        return;
    }
    for (int c = 0; c < kClasses; ++c) {
        for (void *p : P.free_list[dev][c]) {
            cudaFree(p);
            P.cached -= (size_t)256 << c;
        }
        P.free_list[dev][c].clear();
    }
    cudaSetDevice(cur);
}

}  // namespace

void *gq_dev_alloc(size_t bytes, size_t *cap, int *device) {
    int dev = 0;
    GQ_CUDA(cudaGetDevice(&dev));
    GQ_REQUIRE(dev < kMaxDevices, GQ_ERR_UNSUPPORTED, "device index >= 64");
    int c = size_class(bytes, cap);
    Pool &P = pool();
    {
        std::lock_guard<std::mutex> lk(P.mu);
        auto &fl = P.free_list[dev][c];
        if (!fl.empty()) {
            void *p = fl.back();
            fl.pop_back();
            P.cached -= *cap;
            *device = dev;
            return p;
        }
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, *cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        std::lock_guard<std::mutex> lk(P.mu);
        release_device_locked(P, dev);
        e = cudaMalloc(&p, *cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw gq_error{GQ_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
        }
    }
    *device = dev;
    return p;
}

void gq_dev_free(void *p, size_t cap, int device) {
    if (!p) return;
    int c = 0;
    size_t s = 256;
    while (s < cap && c < kClasses - 1) {
        s <<= 1;
        ++c;
    }
    Pool &P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    P.free_list[device][c].push_back(p);
    P.cached += cap;
}

size_t gq_dev_cached_bytes() {
    Pool &P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    return P.cached;
}

void gq_dev_release_cache() {
    Pool &P = pool();
    std::lock_guard<std::mutex> lk(P.mu);
    for (int d = 0; d < kMaxDevices; ++d) release_device_locked(P, d);
}
