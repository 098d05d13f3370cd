// Device-memory pool of the serving loop: first-fit bookkeeping of offsets
// in one region the caller reserved once (include/ctm.h, ctm_pool_*).  Host
// code only: the handles carved from the blocks (ctm_create_in) never call
// cudaMalloc or cudaFree, so admission and retirement neither allocate nor
// wait for other streams' work.
#include <cstddef>
#include <iterator>
#include <map>
#include <mutex>
#include <new>

#include "internal.h"

struct ctm_pool_s {
    size_t size = 0, grain = 1, used = 0;
    std::map<size_t, size_t> free_blocks;  // offset -> length, no two adjacent
    std::map<size_t, size_t> taken;        // offset -> length of every allocated block
    std::mutex mu;
};

namespace {
size_t round_up(size_t n, size_t g) { return (n + g - 1) / g * g; }
}  // namespace

extern "C" {

ctm_status ctm_pool_create(size_t bytes, size_t grain, ctm_pool* out) {
    if (!out) return CTM_ERR_ARG;
    *out = nullptr;
    if (bytes == 0 || grain == 0 || (grain & (grain - 1)) != 0) return CTM_ERR_ARG;
    ctm_pool_s* p = new (std::nothrow) ctm_pool_s();
    if (!p) return CTM_ERR_OOM;
    p->size = bytes / grain * grain;  // whole granules only
    p->grain = grain;
    if (p->size) p->free_blocks[0] = p->size;
    *out = p;
    return CTM_OK;
}

ctm_status ctm_pool_alloc(ctm_pool p, size_t bytes, size_t* offset) {
    if (!p || !offset || bytes == 0) return CTM_ERR_ARG;
    std::lock_guard<std::mutex> lock(p->mu);
    const size_t n = round_up(bytes, p->grain);
    for (auto it = p->free_blocks.begin(); it != p->free_blocks.end(); ++it) {
        if (it->second < n) continue;
        const size_t at = it->first, len = it->second;
        p->free_blocks.erase(it);
        if (len > n) p->free_blocks[at + n] = len - n;
        p->taken[at] = n;
        p->used += n;
        *offset = at;
        return CTM_OK;
    }
    return CTM_ERR_OOM;
}

ctm_status ctm_pool_free(ctm_pool p, size_t offset, size_t bytes) {
    if (!p) return CTM_ERR_ARG;
    std::lock_guard<std::mutex> lock(p->mu);
    auto t = p->taken.find(offset);
    if (t == p->taken.end() || t->second != round_up(bytes, p->grain)) return CTM_ERR_ARG;
    size_t at = offset, len = t->second;
    p->taken.erase(t);
    p->used -= len;
    // merge with the free neighbours on either side
    auto next = p->free_blocks.lower_bound(at);
    if (next != p->free_blocks.end() && next->first == at + len) {
        len += next->second;
        next = p->free_blocks.erase(next);
    }
    if (next != p->free_blocks.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == at) {
            at = prev->first;
            len += prev->second;
            p->free_blocks.erase(prev);
        }
    }
    p->free_blocks[at] = len;
    return CTM_OK;
}

ctm_status ctm_pool_stats(ctm_pool p, size_t* used, size_t* largest_free, size_t* free_blocks) {
    if (!p) return CTM_ERR_ARG;
    std::lock_guard<std::mutex> lock(p->mu);
    size_t big = 0;
    for (const auto& f : p->free_blocks) big = f.second > big ? f.second : big;
    if (used) *used = p->used;
    if (largest_free) *largest_free = big;
    if (free_blocks) *free_blocks = p->free_blocks.size();
    return CTM_OK;
}

ctm_status ctm_pool_destroy(ctm_pool p) {
    delete p;
    return CTM_OK;
}

}  // extern "C"
