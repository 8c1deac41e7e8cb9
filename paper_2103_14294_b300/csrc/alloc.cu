// Device memory of the library: through the caller's allocator hook when one is set
// (huge_set_allocator), else cudaMalloc / cudaFree. Each block remembers the allocator that
// made it, so changing the hook later never frees a block with the wrong allocator.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "internal.h"

namespace huge {
namespace {

struct Hook {
    huge_alloc_fn alloc = nullptr;
    huge_free_fn free = nullptr;
    void *ctx = nullptr;
};

std::mutex g_mu;
Hook g_hook;
struct Owner {
    Hook hook;
    int device;
};
std::unordered_map<void *, Owner> g_owner;  // blocks made by a hook -> that hook and device

}  // namespace

cudaError_t dev_malloc_raw(void **p, size_t n) {
    *p = nullptr;
    Hook h;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        h = g_hook;
    }
    if (!h.alloc) return cudaMalloc(p, n);
    int dev = 0;
    cudaGetDevice(&dev);
    void *q = h.alloc(h.ctx, n, dev);
    if (!q) return cudaErrorMemoryAllocation;
    std::lock_guard<std::mutex> lk(g_mu);
    g_owner[q] = Owner{h, dev};
    *p = q;
    return cudaSuccess;
}

void dev_free(void *p) {
    if (!p) return;
    Owner o;
    bool hooked = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_owner.find(p);
        if (it != g_owner.end()) {
            o = it->second;
            hooked = true;
            g_owner.erase(it);
        }
    }
    if (!hooked) {
        cudaFree(p);
        return;
    }
    o.hook.free(o.hook.ctx, p, o.device);  // the device the block was made on
}

}  // namespace huge

extern "C" int huge_set_allocator(huge_alloc_fn alloc, huge_free_fn free_fn, void *ctx) {
    using namespace huge;
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(HUGE_EINVAL, "set both the allocation and the release function, or neither");
    std::lock_guard<std::mutex> lk(g_mu);
    g_hook.alloc = alloc;
    g_hook.free = free_fn;
    g_hook.ctx = ctx;
    return HUGE_OK;
}
