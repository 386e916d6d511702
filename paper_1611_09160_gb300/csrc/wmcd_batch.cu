// Batches of independent simulations advanced together, and the device-memory pool that
// holds their state (wmcd_batch_* in include/wmcd.h).
//
// Every kernel of a sweep takes the array of the resident simulations' views and selects one
// with blockIdx.y, so one launch per phase serves the whole batch. The launch sequence of a
// batched sweep depends only on the batch's bounds (largest N, most layers, ...), not on the
// random draws, so it is recorded once as a CUDA graph and replayed every sweep; the device
// keeps each simulation's sweep counter and slot counts. Membership changes mark the graph
// stale; it is recorded again before the next step.
#include <algorithm>
#include <cstring>
#include <map>
#include <new>
#include <vector>
#include "wmcd_host.h"

namespace wmcd {

// First-fit allocator over one device allocation. Free blocks are kept by offset and merged
// with their neighbours on release; every block is a multiple of 256 bytes.
class Pool {
public:
    void init(char* base, size_t size) {
        base_ = base;
        size_ = size & ~(size_t)255;
        free_.clear();
        if (size_) free_[0] = size_;
    }
    bool alloc(size_t n, size_t* off) {
        n = round(n);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < n) continue;
            *off = it->first;
            const size_t rest = it->second - n, next = it->first + n;
            free_.erase(it);
            if (rest) free_[next] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t n) {
        n = round(n);
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const {
        size_t t = 0;
        for (auto& f : free_) t += f.second;
        return t;
    }
    size_t largest() const {
        size_t t = 0;
        for (auto& f : free_) t = std::max(t, f.second);
        return t;
    }
    char* base() const { return base_; }
    static size_t round(size_t n) { return (n + 255) & ~(size_t)255; }

private:
    char* base_ = nullptr;
    size_t size_ = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
};

struct Member {
    wmcd_handle* H = nullptr;
    size_t off = 0, bytes = 0;
    int slot = -1;
};

struct Batch {
    int capacity = 0;
    int dev = 0;
    void* pool_mem = nullptr;
    Pool pool;
    std::vector<int> slot_pos;       // slot -> index in members (= blockIdx.y), -1 if free
    std::vector<Member> members;     // dense
    SimView* dviews = nullptr;       // capacity views, in member order
    GroupDims g;
    int block_warps = kStageWarps;
    int serial_threads = kSerialThreads;
    bool stale = true;
    cudaStream_t admit_stream = nullptr, capture_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_sweep = 0;
    Handle prof;                     // event pool and per-class times while profiling
    ForkJoin fj;                     // side streams for launches that run side by side
};

void batch_view_changed(void* batch) { static_cast<Batch*>(batch)->stale = true; }

// bounds over the resident simulations
static GroupDims group_bounds(const std::vector<Member>& ms, int block_warps, int serial_threads) {
    GroupDims g;
    g.S = (int)ms.size();
    g.maxN = 1;
    g.maxCells = 1;
    g.maxL = 0;
    g.maxK3 = 1;
    g.maxMF = 0;
    g.stage_cap = 1;
    g.pw_blocks = 1;
    g.pw = false;
    g.prec_mask = 0;
    g.block_warps = block_warps;
    g.serial_threads = serial_threads;
    g.smem_maxN = 0;
    g.any_global_serial = false;
    for (const Member& m : ms) {
        const GroupDims& o = m.H->h.g;
        g.smem_maxN = std::max(g.smem_maxN, o.smem_maxN);
        for (int c = 0; c < 3; c++) g.smem_cls[c] = std::max(g.smem_cls[c], o.smem_cls[c]);
        g.any_global_serial = g.any_global_serial || o.any_global_serial;
        g.maxN = std::max(g.maxN, o.maxN);
        g.maxCells = std::max(g.maxCells, o.maxCells);
        g.maxL = std::max(g.maxL, o.maxL);
        g.maxK3 = std::max(g.maxK3, o.maxK3);
        g.maxMF = std::max(g.maxMF, o.maxMF);
        g.stage_cap = std::max(g.stage_cap, o.stage_cap);
        g.ncap = std::max(g.ncap, o.ncap);
        g.pw_blocks = std::max(g.pw_blocks, o.pw_blocks);
        g.pw = g.pw || o.pw;
        g.prec_mask |= o.prec_mask;
        for (int l = 0; l < o.maxL; l++) {
            g.bigM[l] = std::max(g.bigM[l], o.bigM[l]);
            for (int ls = l; ls < 2 * kMaxLayers; ls += kLevel2) {   // the layer and its second colouring
                g.Mmax[ls] = std::max(g.Mmax[ls], o.Mmax[ls]);
                g.keys[ls] = std::max(g.keys[ls], o.keys[ls]);
                g.nq[ls] = std::max(g.nq[ls], o.nq[ls]);
                g.coloured[ls] = g.coloured[ls] || o.coloured[ls];
                g.cap_l[ls] = std::max(g.cap_l[ls], o.cap_l[ls]);
            }
        }
    }
    for (int l = 0; l < g.maxL; l++) {
        for (int ls = l; ls < 2 * kMaxLayers; ls += kLevel2) {
            g.keys[ls] = std::max(g.keys[ls], 1);
            g.nq[ls] = std::max(g.nq[ls], 1);
        }
    }
    return g;
}

// refresh the device views and record the batched sweep as a graph
static int rebuild(Batch* b, cudaStream_t s) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    b->launches_per_sweep = 0;
    if (b->members.empty()) { b->stale = false; return WMCD_OK; }
    // largest simulations first: their blocks are scheduled first and the long ones do not
    // start in a late wave (blockIdx.y follows this order)
    std::stable_sort(b->members.begin(), b->members.end(),
                     [](const Member& x, const Member& y) { return x.H->h.N > y.H->h.N; });
    for (size_t i = 0; i < b->members.size(); i++) b->slot_pos[b->members[i].slot] = (int)i;
    std::vector<SimView> views(b->members.size());
    for (size_t i = 0; i < b->members.size(); i++) views[i] = b->members[i].H->h.v;
    // pageable source: the copy is staged before the call returns, ordered after earlier steps
    if (cudaMemcpyAsync(b->dviews, views.data(), views.size() * sizeof(SimView), cudaMemcpyHostToDevice, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return WMCD_ECUDA;
    }
    b->g = group_bounds(b->members, b->block_warps, b->serial_threads);
    prepare_staged(b->g);
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return WMCD_ECUDA;
    }
    const int64_t n = enqueue_sweep(b->dviews, b->g, nullptr, nullptr, b->capture_stream, &b->fj);
    if (cudaStreamEndCapture(b->capture_stream, &graph) != cudaSuccess || !graph) {
        cudaGetLastError();
        return WMCD_ECUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { cudaGetLastError(); b->exec = nullptr; return WMCD_ECUDA; }
    b->launches_per_sweep = n;
    b->stale = false;
    return WMCD_OK;
}

static void release_member(Batch* b, size_t idx) {
    Member m = b->members[idx];
    Handle* h = &m.H->h;
    h->batch = nullptr;
    for (auto& u : h->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFree(p);
    delete m.H;
    b->pool.release(m.off, m.bytes);
    b->slot_pos[m.slot] = -1;
    if (idx + 1 != b->members.size()) {
        b->members[idx] = b->members.back();
        b->slot_pos[b->members[idx].slot] = (int)idx;
    }
    b->members.pop_back();
    b->stale = true;
}

}  // namespace wmcd

using namespace wmcd;

struct wmcd_batch { Batch b; };

extern "C" int wmcd_batch_create(int capacity, int64_t pool_bytes, wmcd_batch** out) {
    if (!out || capacity < 1 || capacity > 65535 || pool_bytes < 256) return WMCD_EINVAL;
    *out = nullptr;
    wmcd_batch* B = new (std::nothrow) wmcd_batch();
    if (!B) return WMCD_ENOMEM;
    Batch* b = &B->b;
    b->capacity = capacity;
    cudaGetDevice(&b->dev);
    b->slot_pos.assign(capacity, -1);
    bool ok = cudaMalloc(&b->pool_mem, (size_t)pool_bytes) == cudaSuccess &&
              cudaMalloc((void**)&b->dviews, sizeof(SimView) * (size_t)capacity) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->admit_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->fj.side[0], cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&b->fj.side[1], cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fj.fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fj.join[0], cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fj.join[1], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        wmcd_batch_destroy(B);
        return WMCD_ENOMEM;
    }
    b->pool.init((char*)b->pool_mem, (size_t)pool_bytes);
    *out = B;
    return WMCD_OK;
}

extern "C" int wmcd_batch_need(const wmcd_params* params, int64_t* bytes) {
    if (!params || !bytes) return WMCD_EINVAL;
    wmcd_handle* H = new (std::nothrow) wmcd_handle();
    if (!H) return WMCD_ENOMEM;
    Arena count;
    count.count_only = true;
    const int rc = create_handle(H, params, nullptr, nullptr, 0, nullptr, &count);
    delete H;   // a counting pass allocates and launches nothing
    if (rc) return rc;
    *bytes = (int64_t)Pool::round(count.used);
    return WMCD_OK;
}

extern "C" int wmcd_batch_admit(wmcd_batch* B, const wmcd_params* params, const double* pos, const int32_t* chain_len,
                                int64_t n_chains, int* slot) {
    if (!B || !params || !pos || !chain_len || !slot || n_chains < 1) return WMCD_EINVAL;
    Batch* b = &B->b;
    int64_t need = 0;
    int rc = wmcd_batch_need(params, &need);
    if (rc) return rc;
    int free_slot = -1;
    for (int k = 0; k < b->capacity; k++) if (b->slot_pos[k] < 0) { free_slot = k; break; }
    size_t off = 0;
    if (free_slot < 0 || !b->pool.alloc((size_t)need, &off)) return WMCD_EFULL;
    wmcd_handle* H = new (std::nothrow) wmcd_handle();
    if (!H) { b->pool.release(off, (size_t)need); return WMCD_ENOMEM; }
    Arena a;
    a.base = b->pool.base() + off;
    a.size = (size_t)need;
    rc = create_handle(H, params, pos, chain_len, n_chains, b->admit_stream, &a);
    if (rc) {
        destroy_handle(H);
        b->pool.release(off, (size_t)need);
        return rc;
    }
    H->h.batch = b;
    Member m;
    m.H = H;
    m.off = off;
    m.bytes = (size_t)need;
    m.slot = free_slot;
    b->slot_pos[free_slot] = (int)b->members.size();
    b->members.push_back(m);
    b->stale = true;
    *slot = free_slot;
    return WMCD_OK;
}

extern "C" int wmcd_batch_step(wmcd_batch* B, int64_t n_sweeps, void* stream) {
    if (!B || n_sweeps < 0) return WMCD_EINVAL;
    Batch* b = &B->b;
    cudaStream_t s = (cudaStream_t)stream;
    if (b->stale) {
        const int rc = rebuild(b, s);
        if (rc) return rc;
    }
    if (!b->exec || n_sweeps == 0) return last_cuda_status();
    if (b->prof.prof) {
        // timed launch by launch, outside the graph (same kernels, same order)
        for (int64_t k = 0; k < n_sweeps; k++) enqueue_sweep(b->dviews, b->g, nullptr, &b->prof, s, nullptr);
    } else {
        for (int64_t k = 0; k < n_sweeps; k++)
            if (cudaGraphLaunch(b->exec, s) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    }
    // host-side counters of each member follow its device sweep counter
    for (Member& m : b->members) {
        Handle* h = &m.H->h;
        h->sweep += (uint64_t)n_sweeps;
        h->tr_pw_count = h->g.pw ? slot_count(h, K_PWCOUNT, 0, h->sweep - 1, h->v.expect_F) : 0;
    }
    return last_cuda_status();
}

extern "C" int wmcd_batch_handle(wmcd_batch* B, int slot, wmcd_handle** h) {
    if (!B || !h || slot < 0 || slot >= B->b.capacity || B->b.slot_pos[slot] < 0) return WMCD_EINVAL;
    *h = B->b.members[B->b.slot_pos[slot]].H;
    return WMCD_OK;
}

extern "C" int wmcd_batch_retire(wmcd_batch* B, int slot, void* stream) {
    if (!B || slot < 0 || slot >= B->b.capacity || B->b.slot_pos[slot] < 0) return WMCD_EINVAL;
    Batch* b = &B->b;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) { cudaGetLastError(); return WMCD_ECUDA; }
    release_member(b, (size_t)b->slot_pos[slot]);
    return WMCD_OK;
}

extern "C" int wmcd_batch_set_block(wmcd_batch* B, int stage_warps, int serial_threads) {
    if (!B || stage_warps < 1 || stage_warps > kMaxStageWarps) return WMCD_EINVAL;
    if (serial_threads != 32 && serial_threads != 128 && serial_threads != 512) return WMCD_EINVAL;
    Batch* b = &B->b;
    if (b->block_warps != stage_warps || b->serial_threads != serial_threads) {
        b->block_warps = stage_warps;
        b->serial_threads = serial_threads;
        b->stale = true;
    }
    return WMCD_OK;
}

extern "C" int wmcd_batch_info(wmcd_batch* B, int64_t* resident, int64_t* pool_free, int64_t* largest_free,
                               int64_t* launches_per_sweep) {
    if (!B) return WMCD_EINVAL;
    if (resident) *resident = (int64_t)B->b.members.size();
    if (pool_free) *pool_free = (int64_t)B->b.pool.free_bytes();
    if (largest_free) *largest_free = (int64_t)B->b.pool.largest();
    if (launches_per_sweep) *launches_per_sweep = B->b.stale ? 0 : B->b.launches_per_sweep;
    return WMCD_OK;
}

extern "C" int wmcd_batch_profile(wmcd_batch* B, int enable) {
    if (!B) return WMCD_EINVAL;
    B->b.prof.prof = enable != 0;
    return WMCD_OK;
}

extern "C" int wmcd_batch_kernel_times(wmcd_batch* B, int64_t* launches, double* ms, int n_classes, void* stream) {
    if (!B || n_classes < 0) return WMCD_EINVAL;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return WMCD_ECUDA;
    return take_kernel_times(&B->b.prof, launches, ms, n_classes);
}

extern "C" int wmcd_batch_destroy(wmcd_batch* B) {
    if (!B) return WMCD_EINVAL;
    Batch* b = &B->b;
    cudaDeviceSynchronize();
    for (auto& u : b->prof.ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
    for (auto e : b->prof.ev_pool) cudaEventDestroy(e);
    while (!b->members.empty()) release_member(b, b->members.size() - 1);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->admit_stream) cudaStreamDestroy(b->admit_stream);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    for (int c = 0; c < 2; c++) {
        if (b->fj.side[c]) cudaStreamDestroy(b->fj.side[c]);
        if (b->fj.join[c]) cudaEventDestroy(b->fj.join[c]);
    }
    if (b->fj.fork) cudaEventDestroy(b->fj.fork);
    if (b->dviews) cudaFree(b->dviews);
    if (b->pool_mem) cudaFree(b->pool_mem);
    cudaGetLastError();
    delete B;
    return WMCD_OK;
}
