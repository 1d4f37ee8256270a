// psf_batch.cu -- one persistent fused insert + update + query kernel per iteration
// across many tables (render sessions of different sizes and depths).
//
// Work is cut into warp units: 32 vertices of one table (insert), 32 dirty-bitmap
// words = 1024 slots of one table (update), 32 paths of one table (query).  Per phase,
// each warp walks the global unit range with a stride of the whole grid and finds its
// table by binary search over the per-table prefix sums (kept in shared memory).  The
// phases are separated by a grid barrier; the kernel is launched cooperatively so every
// block is resident, and each wait is bounded by a timeout.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>

#include "psf.h"
#include "psf_device.cuh"
#include "psf_table.h"

namespace {

using psf::kThreads;
using psf::TableView;

struct BatchItemDev {
    TableView t;
    const float4* v;
    float* out;
    unsigned* slots;  // the item's slot cache (D*P), or nullptr
    unsigned P;
    unsigned D;
    unsigned long long nverts;
};

struct BatchCtl {  // barrier words and sticky status (not overwritten by psf_batch_set)
    unsigned barrier_count;
    unsigned barrier_gen;
    unsigned status;
    unsigned pad[61];
};
static_assert(sizeof(BatchCtl) == 256, "control block is 256 bytes");

struct BatchHdr {  // written by psf_batch_set
    unsigned n;
    unsigned phantom;
    unsigned long long timeout_ns;
    unsigned long long units[3];  // warp units per phase
    unsigned active_blocks[3];    // blocks that work in each phase (the first ones: a few per SM)
    unsigned pad2;
    unsigned long long pad[25];
};
static_assert(sizeof(BatchHdr) == 256, "batch header is 256 bytes");

constexpr unsigned kMaxItems = PSF_MAX_BATCH;
constexpr size_t kBeginBytes = 3 * (kMaxItems + 1) * sizeof(unsigned long long);

size_t batch_bytes(uint32_t max_items) {
    return sizeof(BatchCtl) + sizeof(BatchHdr) + kBeginBytes + static_cast<size_t>(max_items) * sizeof(BatchItemDev);
}

// Grid-wide barrier for a co-resident grid.  The wait is bounded: on timeout the block
// records PSF_STATUS_TIMEOUT (batch and every table) and the kernel leaves.
__device__ bool grid_barrier(BatchCtl* ctl, const BatchHdr* h, const BatchItemDev* __restrict__ items) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* gen_p = &ctl->barrier_gen;
        const unsigned gen = *gen_p;
        __threadfence();
        const unsigned expected = gridDim.x + h->phantom;
        const unsigned arrived = atomicAdd(&ctl->barrier_count, 1u) + 1u;
        if (arrived == expected) {
            atomicExch(&ctl->barrier_count, 0u);
            __threadfence();
            atomicAdd(&ctl->barrier_gen, 1u);
        } else {
            const unsigned long long t0 = psf::global_timer_ns();
            while (*gen_p == gen) {
                if (psf::global_timer_ns() - t0 > h->timeout_ns) {
                    ok = 0;
                    atomicOr(&ctl->status, psf::kStatusTimeout);
                    for (unsigned i = 0; i < h->n; ++i) atomicOr(&items[i].t.hdr->status, psf::kStatusTimeout);
                    break;
                }
                __nanosleep(256);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void load_begin(unsigned long long* s_begin, const unsigned long long* begin, unsigned n) {
    __syncthreads();
    for (unsigned i = threadIdx.x; i <= n; i += blockDim.x) s_begin[i] = begin[i];
    __syncthreads();
}

// Blocks that work in each phase: cap blocks per SM (of the per_sm resident ones) times the SMs,
// or 0 (all of them) when there is no cap below per_sm.
void phase_blocks(const psf_batch_config& c, int sms, int per_sm, unsigned out[3]) {
    for (int ph = 0; ph < 3; ++ph) {
        const unsigned cap = c.phase_blocks_per_sm[ph];
        out[ph] = cap && static_cast<int>(cap) < per_sm ? cap * static_cast<unsigned>(sms) : 0u;
    }
}

// Table owning warp unit u: the last i with begin[i] <= u (tables without units are skipped).
__device__ __forceinline__ unsigned find_item(const unsigned long long* s_begin, unsigned n, unsigned long long u) {
    unsigned lo = 0, hi = n;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        if (s_begin[mid] <= u)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

template <int kMode>
__global__ void __launch_bounds__(kThreads)
    k_batch(BatchCtl* ctl, const BatchHdr* __restrict__ h, const unsigned long long* __restrict__ begin,
            const BatchItemDev* __restrict__ items) {
    __shared__ unsigned long long s_begin[kMaxItems + 1];
    __shared__ psf::LaneSums s_stage[kThreads];
    psf::LaneSums* stage = s_stage + (threadIdx.x & ~31u);
    const unsigned n = h->n;
    if (n == 0) return;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long warp = (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    // a phase runs on its first active_blocks[p] blocks (all when 0); the others go straight to
    // the barrier that ends it
    auto phase_warps = [h](int p) {
        const unsigned a = h->active_blocks[p] && h->active_blocks[p] < gridDim.x ? h->active_blocks[p] : gridDim.x;
        return (static_cast<unsigned long long>(a) * blockDim.x) >> 5;
    };
    unsigned long long nwarps = phase_warps(0);

    // phase 1: scatter every table's vertices
    load_begin(s_begin, begin, n);
    for (unsigned long long u = warp; warp < nwarps && u < h->units[0]; u += nwarps) {
        const unsigned it = find_item(s_begin, n, u);
        const BatchItemDev& b = items[it];
        const unsigned long long i = (u - s_begin[it]) * 32ull + lane;
        const bool valid = i < b.nverts;
        float4 v0 = make_float4(0, 0, 0, 0), v1 = v0, v2 = v0, v3 = v0;
        if (valid) {
            const float4* r = b.v + 4 * i;
            v0 = __ldcs(r);
            v1 = __ldcs(r + 1);
            v2 = __ldcs(r + 2);
            v3 = __ldcs(r + 3);
        }
        unsigned len = 0, leaders = 0;
        if (b.slots) {  // warp-uniform, like the level test: a warp's 32 vertices belong to one item
            psf::SlotNote note{b.t.levels > 1 ? psf::read_level(b.t, static_cast<unsigned>(i / b.P)) : 0u, psf::kNoSlot};
            if (b.t.levels > 1)
                psf::insert_warp<kMode, true, true>(b.t, valid, v0, v1, v2, v3, &len, stage, &leaders, &note);
            else
                psf::insert_warp<kMode, false, true>(b.t, valid, v0, v1, v2, v3, &len, stage, &leaders, &note);
            if (valid) b.slots[i] = note.slot;
        } else if (b.t.levels > 1) {
            psf::insert_warp<kMode, true>(b.t, valid, v0, v1, v2, v3, &len, stage, &leaders);
        } else {
            psf::insert_warp<kMode, false>(b.t, valid, v0, v1, v2, v3, &len, stage, &leaders);
        }
        if (len > 16u) atomicMax(&b.t.hdr->max_probe, len);  // only long probes are recorded here
    }
    psf::bulk_wait_done();  // this thread's bulk sums have landed before the barrier publishes them
    if (!grid_barrier(ctl, h, items)) return;

    // phase 2: blend every table's touched cells
    load_begin(s_begin, begin + (kMaxItems + 1), n);
    nwarps = phase_warps(1);
    for (unsigned long long u = warp; warp < nwarps && u < h->units[1]; u += nwarps) {
        const unsigned it = find_item(s_begin, n, u);
        const BatchItemDev& b = items[it];
        const unsigned long long w0 = (u - s_begin[it]) * 32ull;
        const unsigned long long nwords = ((1ull << b.t.log2cap) + 31ull) >> 5;
        if (w0 == 0 && lane == 0) {
            if (b.t.h_status) *reinterpret_cast<volatile unsigned*>(b.t.h_status) = b.t.hdr->status;
            b.t.hdr->iterations += 1;
        }
        const unsigned total = psf::update_words(b.t, w0, nwords);
        if (lane == 0 && total) atomicAdd(&b.t.hdr->touched, static_cast<unsigned long long>(total));
    }
    if (!grid_barrier(ctl, h, items)) return;

    // phase 3: every table's control-variate query
    load_begin(s_begin, begin + 2 * (kMaxItems + 1), n);
    nwarps = phase_warps(2);
    for (unsigned long long u = warp; warp < nwarps && u < h->units[2]; u += nwarps) {
        const unsigned it = find_item(s_begin, n, u);
        const BatchItemDev& b = items[it];
        const unsigned long long p = (u - s_begin[it]) * 32ull + lane;
        if (p < b.P) {
            if (b.slots)
                psf::query_path<true>(b.t, psf::cv_estimator(b.t), b.v, b.P, b.D, p, b.out, b.slots);
            else
                psf::query_path(b.t, psf::cv_estimator(b.t), b.v, b.P, b.D, p, b.out);
        }
    }
}

}  // namespace

struct psf_batch {
    uint32_t max_items;
    psf_batch_config cfg;
    char* d_buf;
    char* h_stage;
    cudaEvent_t staged;
    bool pending;
    int device;
    int sms;
    int per_sm[2];
    unsigned phase_active[3];  // blocks that work in each phase (0: all)
};

extern "C" {

int psf_batch_create(uint32_t max_items, const psf_batch_config* cfg, psf_batch** out) {
    if (!out || max_items == 0 || max_items > kMaxItems) return PSF_ERR_INVALID_ARG;
    *out = nullptr;
    psf_batch* b = new (std::nothrow) psf_batch();
    if (!b) return PSF_ERR_NO_MEM;
    b->max_items = max_items;
    b->cfg = cfg ? *cfg : psf_batch_config{};
    if (b->cfg.insert_mode > 1) {
        delete b;
        return PSF_ERR_INVALID_ARG;
    }
    const size_t bytes = batch_bytes(max_items);
    bool ok = psf_cuda_ok(cudaGetDevice(&b->device), "cudaGetDevice") &&
              psf_cuda_ok(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device), "attribute") &&
              psf_cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->per_sm[0], k_batch<psf::kAggWarp>, kThreads, 0),
                          "occupancy") &&
              psf_cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->per_sm[1], k_batch<psf::kAggNone>, kThreads, 0),
                          "occupancy");
    if (ok) ok = psf_cuda_ok(cudaMalloc(reinterpret_cast<void**>(&b->d_buf), bytes), "cudaMalloc");
    if (ok) {
        ok = psf_cuda_ok(cudaHostAlloc(reinterpret_cast<void**>(&b->h_stage), bytes, cudaHostAllocDefault), "cudaHostAlloc");
        if (!ok) cudaFree(b->d_buf);
    }
    if (ok) {
        ok = psf_cuda_ok(cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming), "cudaEventCreate");
        if (!ok) {
            cudaFree(b->d_buf);
            cudaFreeHost(b->h_stage);
        }
    }
    if (ok) {
        std::memset(b->h_stage, 0, bytes);
        ok = psf_cuda_ok(cudaMemset(b->d_buf, 0, bytes), "cudaMemset");
        if (!ok) {
            cudaFree(b->d_buf);
            cudaFreeHost(b->h_stage);
            cudaEventDestroy(b->staged);
        }
    }
    if (!ok) {
        delete b;
        return PSF_ERR_CUDA;
    }
    int per_sm = b->per_sm[b->cfg.insert_mode == 1 ? 1 : 0];
    if (b->cfg.blocks_per_sm && static_cast<int>(b->cfg.blocks_per_sm) < per_sm) per_sm = static_cast<int>(b->cfg.blocks_per_sm);
    phase_blocks(b->cfg, b->sms, per_sm, b->phase_active);
    *out = b;
    return PSF_OK;
}

int psf_batch_set(psf_batch* b, const psf_batch_item* items, uint32_t n, void* stream) {
    if (!b || n > b->max_items || (n && !items)) return PSF_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        const psf_batch_item& it = items[i];
        if (!it.table || it.table->view.payload != psf::kPayloadRGB) return PSF_ERR_INVALID_ARG;
        const unsigned long long nv = static_cast<unsigned long long>(it.P) * it.D;
        if (nv && (!it.d_vertices || !it.d_out_rgb || (reinterpret_cast<uintptr_t>(it.d_vertices) & 15u) ||
                   (reinterpret_cast<uintptr_t>(it.d_out_rgb) & 3u) || (reinterpret_cast<uintptr_t>(it.d_slots) & 3u)))
            return PSF_ERR_INVALID_ARG;
    }
    // the staging buffer may still feed the previous copy
    if (b->pending && !psf_cuda_ok(cudaEventSynchronize(b->staged), "cudaEventSynchronize")) return PSF_ERR_CUDA;
    BatchHdr* h = reinterpret_cast<BatchHdr*>(b->h_stage + sizeof(BatchCtl));
    unsigned long long* begin = reinterpret_cast<unsigned long long*>(b->h_stage + sizeof(BatchCtl) + sizeof(BatchHdr));
    BatchItemDev* dev = reinterpret_cast<BatchItemDev*>(b->h_stage + sizeof(BatchCtl) + sizeof(BatchHdr) + kBeginBytes);
    h->n = n;
    h->phantom = b->cfg.test_phantom_blocks;
    for (int ph = 0; ph < 3; ++ph) h->active_blocks[ph] = b->phase_active[ph];
    h->timeout_ns = 1000ull * (b->cfg.barrier_timeout_us ? b->cfg.barrier_timeout_us : 2000000u);
    unsigned long long acc[3] = {0, 0, 0};
    for (uint32_t i = 0; i < n; ++i) {
        const psf_batch_item& it = items[i];
        BatchItemDev& d = dev[i];
        d.t = it.table->view;
        // each launch inserts the item's vertices and blends them: one iteration of P*D vertices
        it.table->iter_vertices = 0;
        psf_count_iteration_vertices(it.table, static_cast<unsigned long long>(it.P) * it.D);
        d.v = reinterpret_cast<const float4*>(it.d_vertices);
        d.out = it.d_out_rgb;
        d.slots = it.d_slots;
        d.P = it.P;
        d.D = it.D;
        d.nverts = static_cast<unsigned long long>(it.P) * it.D;
        const unsigned long long nwords = ((1ull << it.table->cfg.log2_capacity) + 31ull) >> 5;
        const unsigned long long units[3] = {(d.nverts + 31) / 32, (nwords + 31) / 32,
                                             (static_cast<unsigned long long>(it.P) + 31) / 32};
        for (int ph = 0; ph < 3; ++ph) {
            begin[ph * (kMaxItems + 1) + i] = acc[ph];
            acc[ph] += units[ph];
        }
    }
    for (int ph = 0; ph < 3; ++ph) {
        begin[ph * (kMaxItems + 1) + n] = acc[ph];
        h->units[ph] = acc[ph];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t off = sizeof(BatchCtl);
    const size_t len = sizeof(BatchHdr) + kBeginBytes + static_cast<size_t>(n) * sizeof(BatchItemDev);
    if (!psf_cuda_ok(cudaMemcpyAsync(b->d_buf + off, b->h_stage + off, len, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync") ||
        !psf_cuda_ok(cudaEventRecord(b->staged, st), "cudaEventRecord"))
        return PSF_ERR_CUDA;
    b->pending = true;
    return PSF_OK;
}

int psf_batch_launch(psf_batch* b, void* stream) {
    if (!b) return PSF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int mode = b->cfg.insert_mode == 1 ? 1 : 0;
    int per_sm = b->per_sm[mode];
    if (b->cfg.blocks_per_sm && static_cast<int>(b->cfg.blocks_per_sm) < per_sm) per_sm = static_cast<int>(b->cfg.blocks_per_sm);
    if (per_sm < 1) return PSF_ERR_INVALID_ARG;
    // a fresh barrier for every launch (a timed-out launch leaves its count behind)
    if (!psf_cuda_ok(cudaMemsetAsync(b->d_buf, 0, 2 * sizeof(unsigned), st), "cudaMemsetAsync")) return PSF_ERR_CUDA;
    BatchCtl* ctl = reinterpret_cast<BatchCtl*>(b->d_buf);
    const BatchHdr* h = reinterpret_cast<const BatchHdr*>(b->d_buf + sizeof(BatchCtl));
    const unsigned long long* begin = reinterpret_cast<const unsigned long long*>(b->d_buf + sizeof(BatchCtl) + sizeof(BatchHdr));
    const BatchItemDev* items =
        reinterpret_cast<const BatchItemDev*>(b->d_buf + sizeof(BatchCtl) + sizeof(BatchHdr) + kBeginBytes);
    void* args[] = {&ctl, &h, &begin, &items};
    const dim3 grid(static_cast<unsigned>(b->sms * per_sm)), block(kThreads);
    const void* fn = mode == 1 ? reinterpret_cast<const void*>(k_batch<psf::kAggNone>)
                               : reinterpret_cast<const void*>(k_batch<psf::kAggWarp>);
    return psf_cuda_ok(cudaLaunchCooperativeKernel(fn, grid, block, args, 0, st), "k_batch") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_batch_step(psf_batch* b, const psf_batch_item* items, uint32_t n, void* stream) {
    const int rc = psf_batch_set(b, items, n, stream);
    return rc != PSF_OK ? rc : psf_batch_launch(b, stream);
}

int psf_batch_status(psf_batch* b, uint32_t* status, void* stream) {
    if (!b || !status) return PSF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned s = 0;
    if (!psf_cuda_ok(cudaMemcpyAsync(&s, b->d_buf + offsetof(BatchCtl, status), sizeof(s), cudaMemcpyDeviceToHost, st),
                     "cudaMemcpyAsync") ||
        !psf_cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize"))
        return PSF_ERR_CUDA;
    *status = s;
    return PSF_OK;
}

int psf_batch_destroy(psf_batch* b) {
    if (!b) return PSF_OK;
    cudaEventDestroy(b->staged);
    cudaFreeHost(b->h_stage);
    cudaFree(b->d_buf);
    delete b;
    return PSF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free batched step.  Some callers cannot allocate device memory on the
// path that drives the filter: an application that reserved all device memory in its
// own pool up front (a cudaMalloc there fails or fragments the pool), or a renderer
// whose per-frame loop must not call cudaMalloc/cudaFree because they can synchronize
// the whole device and stall its other streams.  This entry point runs the same fused
// kernel with its descriptors and barrier words in a fixed array that is part of the
// library image on every GPU that loads it.
// ---------------------------------------------------------------------------
namespace {

constexpr unsigned kNoAllocMaxItems = PSF_NOALLOC_MAX_ITEMS;
constexpr size_t kNoAllocBytes =
    sizeof(BatchCtl) + sizeof(BatchHdr) + kBeginBytes + static_cast<size_t>(kNoAllocMaxItems) * sizeof(BatchItemDev);
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call on a device and kept between calls.  Host code may not use the
// name as an address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
char* g_noalloc_base[kNoAllocMaxDevices];  // device address of g_noalloc_scratch, per device
int g_noalloc_sms[kNoAllocMaxDevices];
int g_noalloc_per_sm[kNoAllocMaxDevices][2];

// Once per device, with that device current: resolve the array's device address.
bool noalloc_setup(int dev) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_base[dev]) return true;
    void* p = nullptr;
    int sms = 0, m0 = 0, m1 = 0;
    if (!psf_cuda_ok(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress") ||
        !psf_cuda_ok(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "attribute") ||
        !psf_cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m0, k_batch<psf::kAggWarp>, kThreads, 0), "occupancy") ||
        !psf_cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m1, k_batch<psf::kAggNone>, kThreads, 0), "occupancy"))
        return false;
    g_noalloc_sms[dev] = sms;
    g_noalloc_per_sm[dev][0] = m0;
    g_noalloc_per_sm[dev][1] = m1;
    g_noalloc_base[dev] = static_cast<char*>(p);
    return true;
}

}  // namespace

extern "C" int psf_batch_step_noalloc(const psf_batch_item* items, uint32_t n, const psf_batch_config* cfg,
                                      void* stream) {
    if (n > kNoAllocMaxItems) {
        psf_cuda_ok(cudaErrorInvalidValue, "psf_batch_step_noalloc: more items than PSF_NOALLOC_MAX_ITEMS");
        return PSF_ERR_TOO_MANY;
    }
    if (n && !items) return PSF_ERR_INVALID_ARG;
    const psf_batch_config c = cfg ? *cfg : psf_batch_config{};
    if (c.insert_mode > 1) return PSF_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < n; ++i) {
        const psf_batch_item& it = items[i];
        if (!it.table || it.table->view.payload != psf::kPayloadRGB) return PSF_ERR_INVALID_ARG;
        const unsigned long long nv = static_cast<unsigned long long>(it.P) * it.D;
        if (nv && (!it.d_vertices || !it.d_out_rgb || (reinterpret_cast<uintptr_t>(it.d_vertices) & 15u) ||
                   (reinterpret_cast<uintptr_t>(it.d_out_rgb) & 3u) || (reinterpret_cast<uintptr_t>(it.d_slots) & 3u)))
            return PSF_ERR_INVALID_ARG;
    }
    int dev = 0;
    if (!psf_cuda_ok(cudaGetDevice(&dev), "cudaGetDevice")) return PSF_ERR_CUDA;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return PSF_ERR_INVALID_ARG;
    if (!noalloc_setup(dev)) return PSF_ERR_CUDA;
    if (n == 0) return PSF_OK;

    // descriptors are built in this thread's static staging area (no heap), then copied
    alignas(64) thread_local unsigned char stage[kNoAllocBytes];
    BatchHdr* h = reinterpret_cast<BatchHdr*>(stage + sizeof(BatchCtl));
    unsigned long long* begin = reinterpret_cast<unsigned long long*>(stage + sizeof(BatchCtl) + sizeof(BatchHdr));
    BatchItemDev* dev_items = reinterpret_cast<BatchItemDev*>(stage + sizeof(BatchCtl) + sizeof(BatchHdr) + kBeginBytes);
    std::memset(h, 0, sizeof(BatchHdr));
    h->n = n;
    h->phantom = c.test_phantom_blocks;
    {
        int per_sm = g_noalloc_per_sm[dev][c.insert_mode == 1 ? 1 : 0];
        if (c.blocks_per_sm && static_cast<int>(c.blocks_per_sm) < per_sm) per_sm = static_cast<int>(c.blocks_per_sm);
        phase_blocks(c, g_noalloc_sms[dev], per_sm, h->active_blocks);
    }
    h->timeout_ns = 1000ull * (c.barrier_timeout_us ? c.barrier_timeout_us : 2000000u);
    unsigned long long acc[3] = {0, 0, 0};
    for (uint32_t i = 0; i < n; ++i) {
        const psf_batch_item& it = items[i];
        BatchItemDev& d = dev_items[i];
        d.t = it.table->view;
        // each launch inserts the item's vertices and blends them: one iteration of P*D vertices
        it.table->iter_vertices = 0;
        psf_count_iteration_vertices(it.table, static_cast<unsigned long long>(it.P) * it.D);
        d.v = reinterpret_cast<const float4*>(it.d_vertices);
        d.out = it.d_out_rgb;
        d.slots = it.d_slots;
        d.P = it.P;
        d.D = it.D;
        d.nverts = static_cast<unsigned long long>(it.P) * it.D;
        const unsigned long long nwords = ((1ull << it.table->cfg.log2_capacity) + 31ull) >> 5;
        const unsigned long long units[3] = {(d.nverts + 31) / 32, (nwords + 31) / 32,
                                             (static_cast<unsigned long long>(it.P) + 31) / 32};
        for (int ph = 0; ph < 3; ++ph) {
            begin[ph * (kMaxItems + 1) + i] = acc[ph];
            acc[ph] += units[ph];
        }
    }
    for (int ph = 0; ph < 3; ++ph) {
        begin[ph * (kMaxItems + 1) + n] = acc[ph];
        h->units[ph] = acc[ph];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char* base = g_noalloc_base[dev];
    const size_t len = sizeof(BatchHdr) + kBeginBytes + static_cast<size_t>(n) * sizeof(BatchItemDev);
    // the barrier words and the status start at zero on every call
    if (!psf_cuda_ok(cudaMemsetAsync(base, 0, sizeof(BatchCtl), st), "cudaMemsetAsync") ||
        !psf_cuda_ok(cudaMemcpyAsync(base + sizeof(BatchCtl), stage + sizeof(BatchCtl), len, cudaMemcpyHostToDevice, st),
                     "cudaMemcpyAsync"))
        return PSF_ERR_CUDA;
    const int mode = c.insert_mode == 1 ? 1 : 0;
    int per_sm = g_noalloc_per_sm[dev][mode];
    if (c.blocks_per_sm && static_cast<int>(c.blocks_per_sm) < per_sm) per_sm = static_cast<int>(c.blocks_per_sm);
    if (per_sm < 1) return PSF_ERR_INVALID_ARG;
    BatchCtl* ctl = reinterpret_cast<BatchCtl*>(base);
    const BatchHdr* dh = reinterpret_cast<const BatchHdr*>(base + sizeof(BatchCtl));
    const unsigned long long* dbegin = reinterpret_cast<const unsigned long long*>(base + sizeof(BatchCtl) + sizeof(BatchHdr));
    const BatchItemDev* ditems = reinterpret_cast<const BatchItemDev*>(base + sizeof(BatchCtl) + sizeof(BatchHdr) + kBeginBytes);
    void* args[] = {&ctl, &dh, &dbegin, &ditems};
    const dim3 grid(static_cast<unsigned>(g_noalloc_sms[dev] * per_sm)), block(kThreads);
    const void* fn = mode == 1 ? reinterpret_cast<const void*>(k_batch<psf::kAggNone>)
                               : reinterpret_cast<const void*>(k_batch<psf::kAggWarp>);
    return psf_cuda_ok(cudaLaunchCooperativeKernel(fn, grid, block, args, 0, st), "k_batch") ? PSF_OK : PSF_ERR_CUDA;
}
