// psf.cu -- kernels and C ABI of the progressive spatio-temporal filtering hot path.
//
// Per iteration (one table = one render session):
//   k_insert  one thread per vertex, lanes of a warp on one key merged (adjacent runs,
//             or match_any with hierarchy levels), one head per group probes the
//             open-addressing table and adds the group's 64-bit fixed-point sums with one
//             bulk (TMA) reduction (eq. 5-6, Alg. 1)
//   k_update  one warp per 1024 slots of the dirty bitmap, set bits compacted across
//             the warp, one lane per touched cell applies eq. (10)-(11)
//   k_query   one thread per path, walking its vertices from the last to the first,
//             one probe per vertex, or none with the slot cache (Section "Control
//             variates", CVEstimator); k_query_tiled splits it by depth (a launch knob)
// Also here: the progressive and staged inserts, the YCoCg two-band SH payload's insert
// (k_insert_sh; its blend and query are k_update<true> and k_query<., true>), the sharded
// session's record merge and approximant copy, export, reset and statistics.
// Grids are persistent (grid-stride) and sized as a multiple of the SM count.

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "psf.h"
#include "psf_device.cuh"
#include "psf_table.h"

using psf::DevHeader;
using psf::Slot;
using psf::TableView;

thread_local std::string psf_g_last_error;

using psf::kThreads;

// Every accepted vertex adds codes of magnitude at most 2^(15+F) to a cell (|fl32(w L_c)| and
// w are at most 2^15; the SH payload's (w n_j) n_k at most 2^15 (1 + 2^-10)^2 after rounding),
// so n vertices cannot overflow a 64-bit sum while n < 2^(48-F) (SH: 2^(47-F)).
void psf_count_iteration_vertices(psf_table* t, unsigned long long n) {
    const unsigned shift = 48u - t->cfg.frac_bits - (t->cfg.payload == psf::kPayloadSH ? 1u : 0u);
    t->iter_vertices += n;
    if (t->iter_vertices >= (1ull << shift)) t->host_status |= PSF_STATUS_SUM_RANGE;
}

bool psf_cuda_ok(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return true;
    psf_g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

namespace {

bool cuda_ok(cudaError_t e, const char* what) { return psf_cuda_ok(e, what); }

// Mapped pinned status words, one per table, handed out from slabs that live until the
// process exits: creating and destroying a table (as a server does for every session) then
// makes no pinned allocation or free, either of which can synchronize the device.
struct StatusWord {
    unsigned* host;
    unsigned* dev;
};

std::mutex g_status_mu;
std::vector<StatusWord> g_status_free;

bool status_take(StatusWord* w) {
    std::lock_guard<std::mutex> lock(g_status_mu);
    if (g_status_free.empty()) {
        constexpr unsigned kSlab = 4096;
        unsigned* host = nullptr;
        unsigned* dev = nullptr;
        if (!cuda_ok(cudaHostAlloc(reinterpret_cast<void**>(&host), kSlab * sizeof(unsigned),
                                   cudaHostAllocMapped | cudaHostAllocPortable),
                     "cudaHostAlloc"))
            return false;
        if (!cuda_ok(cudaHostGetDevicePointer(reinterpret_cast<void**>(&dev), host, 0), "cudaHostGetDevicePointer")) {
            cudaFreeHost(host);
            return false;
        }
        g_status_free.reserve(g_status_free.size() + kSlab);
        for (unsigned i = kSlab; i-- > 0;) g_status_free.push_back(StatusWord{host + i, dev + i});
    }
    *w = g_status_free.back();
    g_status_free.pop_back();
    return true;
}

void status_give(const StatusWord& w) {
    std::lock_guard<std::mutex> lock(g_status_mu);
    g_status_free.push_back(w);
}

struct Layout {
    size_t hdr, keys, slots, mirror, dirty, total;
};

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// Where the keys live (no result depends on it), measured on the B300.  Keys inside the slot
// records put a probe's key in the same 64-byte half of the record as the sums that its bulk
// reduction adds to, so the insert touches one DRAM atom per group instead of two; a dense
// key array packs four keys per sector, which keeps a probing query's key reads in L2 longer.
// With the slot-cache calls (no key read in the query) the keys in the records win on every
// workload measured: 1920x1080 with the FP16 copy 12.56 vs 12.41 G vertices/s, with FP32
// 12.08 vs 11.51; 1280x720 FP16 17.34 vs 16.76; 64 batched sessions 13.92 vs 13.70.  With the
// probing query (psf_query_cv, psf_step) the dense array wins at 2^24 slots (1920x1080 FP16:
// 10.38 vs 9.65) and the records win for FP32 tables up to 2^22 slots (1280x720: 13.4 vs
// 12.8).  The default (key_layout 0) follows the probing path, which needs no caller buffer;
// callers of the slot-cache calls set 2, as the autotuner chooses for them.
bool keys_inline(const psf_config* c) {
    if (c->payload == psf::kPayloadSH) return false;  // SH records have no key field
    return c->key_layout == 2 || (c->key_layout == 0 && c->log2_capacity <= 22 && !c->cache_fp16);
}

bool config_valid(const psf_config* c) {
    if (!c) return false;
    if (c->key_layout > 2 || c->levels > 4) return false;
    if (c->log2_capacity < 4 || c->log2_capacity > 30) return false;
    if (c->pos_bits_q > 20 || c->dir_bits_d > 5) return false;
    if (c->frac_bits < 8 || c->frac_bits > 32) return false;
    if (!(c->alpha_min >= 0.0f && c->alpha_min <= 1.0f)) return false;
    if (!(c->beta == c->beta) || c->blend_mode > 1 || c->use_normal > 1 || c->cache_fp16 > 1) return false;
    if (c->payload > psf::kPayloadSH) return false;
    if (c->payload == psf::kPayloadSH &&
        (c->cache_fp16 || c->levels > 1 || c->key_layout == 2 || !(c->sh_ridge >= 0.0f && c->sh_ridge <= 3.0e38f)))
        return false;
    return true;
}

Layout layout_of(const psf_config* c) {
    const size_t cap = size_t{1} << c->log2_capacity;
    Layout L{};
    size_t off = 0;
    L.hdr = off;
    off = align256(off + sizeof(DevHeader));
    L.keys = off;
    if (!keys_inline(c)) off = align256(off + cap * sizeof(unsigned long long));
    L.slots = off;
    off = align256(off + cap * (c->payload == psf::kPayloadSH ? sizeof(psf::SlotSH) : sizeof(Slot)));
    L.mirror = off;
    if (c->cache_fp16) off = align256(off + cap * sizeof(uint2));
    L.dirty = off;
    off = align256(off + ((cap + 31) / 32) * sizeof(unsigned));
    L.total = off;
    return L;
}

int grid_for(const psf_table* t, int per_sm, unsigned long long work_items, uint32_t limit = 0) {
    if (limit && static_cast<int>(limit) < per_sm) per_sm = static_cast<int>(limit);
    const unsigned long long need = (work_items + kThreads - 1) / kThreads;
    const unsigned long long full = static_cast<unsigned long long>(t->sms) * static_cast<unsigned long long>(per_sm);
    return static_cast<int>(std::max<unsigned long long>(1, std::min(need, full)));
}

}  // namespace

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// With kSlots the kernel also notes each vertex's slot for the query (slots[i]; vertices
// are depth-major records of P paths, so vertex i has depth i / P).
template <int kMode, bool kHier, bool kSlots = false>
__global__ void __launch_bounds__(kThreads, kHier ? 4 : 0) k_insert(TableView t, const float4* __restrict__ v, unsigned long long n,
                                                     unsigned P = 0, unsigned* __restrict__ slots = nullptr) {
    __shared__ unsigned s_max_probe;
    __shared__ unsigned long long s_leaders;
    __shared__ psf::LaneSums s_stage[kThreads];
    if (threadIdx.x == 0) {
        s_max_probe = 0;
        s_leaders = 0;
    }
    __syncthreads();
    psf::LaneSums* stage = s_stage + (threadIdx.x & ~31u);
    unsigned max_len = 0;
    unsigned leaders = 0;  // counted by lane 0 of each warp
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    // the next tile's records are loaded while the current tile probes and adds
    unsigned long long base = static_cast<unsigned long long>(blockIdx.x) * blockDim.x;
    float4 v0 = make_float4(0, 0, 0, 0), v1 = v0, v2 = v0, v3 = v0;
    if (base + threadIdx.x < n) {
        const float4* r = v + 4 * (base + threadIdx.x);  // streamed once: evict-first
        v0 = __ldcs(r);
        v1 = __ldcs(r + 1);
        v2 = __ldcs(r + 2);
        v3 = __ldcs(r + 3);
    }
    for (; base < n; base += stride) {
        const unsigned long long nx = base + stride + threadIdx.x;
        float4 n0 = make_float4(0, 0, 0, 0), n1 = n0, n2 = n0, n3 = n0;
        if (nx < n) {
            const float4* r = v + 4 * nx;
            n0 = __ldcs(r);
            n1 = __ldcs(r + 1);
            n2 = __ldcs(r + 2);
            n3 = __ldcs(r + 3);
        }
        if constexpr (kSlots) {
            const unsigned long long i = base + threadIdx.x;
            psf::SlotNote note{kHier ? psf::read_level(t, static_cast<unsigned>(i / P)) : 0u, psf::kNoSlot};
            psf::insert_warp<kMode, kHier, true>(t, i < n, v0, v1, v2, v3, &max_len, stage, &leaders, &note);
            if (i < n) slots[i] = note.slot;
        } else {
            psf::insert_warp<kMode, kHier>(t, base + threadIdx.x < n, v0, v1, v2, v3, &max_len, stage, &leaders);
        }
        v0 = n0;
        v1 = n1;
        v2 = n2;
        v3 = n3;
    }
    psf::bulk_wait_done();  // this thread's sums have landed before the kernel ends
    if (max_len) atomicMax(&s_max_probe, max_len);
    if ((threadIdx.x & 31u) == 0 && leaders) atomicAdd(&s_leaders, static_cast<unsigned long long>(leaders));
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_max_probe) atomicMax(&t.hdr->max_probe, s_max_probe);
        if (s_leaders) atomicAdd(&t.hdr->leaders, s_leaders);
    }
}

// k_insert for a table with the SH payload (flat tables; the next grid-stride tile's records
// are loaded while the current one probes and adds).  With kSlots it also notes each vertex's
// slot for the query (slots[i]).
template <int kMode, bool kSlots = false>
__global__ void __launch_bounds__(kThreads) k_insert_sh(TableView t, const float4* __restrict__ v, unsigned long long n,
                                                       unsigned* __restrict__ slots = nullptr) {
    __shared__ unsigned s_max_probe;
    __shared__ unsigned long long s_leaders;
    __shared__ psf::ShSums s_stage[kThreads];
    if (threadIdx.x == 0) {
        s_max_probe = 0;
        s_leaders = 0;
    }
    __syncthreads();
    psf::ShSums* stage = s_stage + (threadIdx.x & ~31u);
    unsigned max_len = 0, leaders = 0;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    unsigned long long base = static_cast<unsigned long long>(blockIdx.x) * blockDim.x;
    float4 v0 = make_float4(0, 0, 0, 0), v1 = v0, v2 = v0, v3 = v0;
    if (base + threadIdx.x < n) {
        const float4* r = v + 4 * (base + threadIdx.x);
        v0 = __ldcs(r);
        v1 = __ldcs(r + 1);
        v2 = __ldcs(r + 2);
        v3 = __ldcs(r + 3);
    }
    for (; base < n; base += stride) {
        const unsigned long long nx = base + stride + threadIdx.x;
        float4 n0 = make_float4(0, 0, 0, 0), n1 = n0, n2 = n0, n3 = n0;
        if (nx < n) {
            const float4* r = v + 4 * nx;
            n0 = __ldcs(r);
            n1 = __ldcs(r + 1);
            n2 = __ldcs(r + 2);
            n3 = __ldcs(r + 3);
        }
        const unsigned noted = psf::insert_warp_sh<kMode>(t, base + threadIdx.x < n, v0, v1, v2, v3, &max_len, stage,
                                                           &leaders);
        if constexpr (kSlots)
            if (base + threadIdx.x < n) slots[base + threadIdx.x] = noted;
        v0 = n0;
        v1 = n1;
        v2 = n2;
        v3 = n3;
    }
    psf::bulk_wait_done();
    if (max_len) atomicMax(&s_max_probe, max_len);
    if ((threadIdx.x & 31u) == 0 && leaders) atomicAdd(&s_leaders, static_cast<unsigned long long>(leaders));
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_max_probe) atomicMax(&t.hdr->max_probe, s_max_probe);
        if (s_leaders) atomicAdd(&t.hdr->leaders, s_leaders);
    }
}

// Progressive update values (Section "Progressive solver", eq. (9); Alg. 1 and Alg. 2):
// one thread per path walks its vertices last to first; the FP32 approximant of each
// vertex's cell (read before this iteration's blend, so it is L~old) feeds the value of
// the vertex before it, which is then scattered like a plain insert.  Warps hold 32 paths
// at the same depth, so the warp-level merge of equal keys applies unchanged.
template <int kMode, bool kHier>
__global__ void __launch_bounds__(kThreads) k_insert_progressive(TableView t, const float4* __restrict__ v, unsigned P,
                                                                 unsigned D, unsigned field) {
    __shared__ unsigned s_max_probe;
    __shared__ unsigned long long s_leaders;
    __shared__ psf::LaneSums s_stage[kThreads];
    if (threadIdx.x == 0) {
        s_max_probe = 0;
        s_leaders = 0;
    }
    __syncthreads();
    psf::LaneSums* stage = s_stage + (threadIdx.x & ~31u);
    unsigned max_len = 0, leaders = 0;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long base = static_cast<unsigned long long>(blockIdx.x) * blockDim.x; base < P; base += stride) {
        const unsigned long long p = base + threadIdx.x;
        const bool valid = p < P;
        float3 c_next = make_float3(0.0f, 0.0f, 0.0f), le_next = c_next;
        for (int j = static_cast<int>(D) - 1; j >= 0; --j) {
            float4 v0 = make_float4(0, 0, 0, 0), v1 = v0, v2 = v0, v3 = v0;
            float3 c = make_float3(0.0f, 0.0f, 0.0f);
            if (valid) {
                const float4* r = v + 4 * (static_cast<unsigned long long>(j) * P + p);
                v0 = __ldcs(r);
                v1 = __ldcs(r + 1);
                v2 = __ldcs(r + 2);
                v3 = __ldcs(r + 3);
                c = psf::cell_value(t, v0, v1, v2, /*fp32_master=*/true, psf::read_level(t, static_cast<unsigned>(j)));
            }
            const float3 le = make_float3(v3.x, v3.y, v3.z);
            float4 val = v3;  // (value_r, value_g, value_b, t_b)
            if (field == 0) {  // L~_o: L_e,j + t_j L~old(x_{j+1})
                val.x = __fadd_rn(le.x, __fmul_rn(v1.w, c_next.x));
                val.y = __fadd_rn(le.y, __fmul_rn(v2.w, c_next.y));
                val.z = __fadd_rn(le.z, __fmul_rn(v3.w, c_next.z));
            } else {  // L~_{o\e}: t_j (L_e,j+1 + L~old(x_{j+1}))
                val.x = __fmul_rn(v1.w, __fadd_rn(le_next.x, c_next.x));
                val.y = __fmul_rn(v2.w, __fadd_rn(le_next.y, c_next.y));
                val.z = __fmul_rn(v3.w, __fadd_rn(le_next.z, c_next.z));
            }
            // the range rule applies to the vertex's own record (its L_e as the value, a finite
            // throughput); a record that fails it is dropped through a NaN value, and the
            // computed value of one that passes saturates at |w value| = 2^15
            const bool own_ok = fabsf(__fmul_rn(v0.w, v3.x)) <= 32768.0f && fabsf(__fmul_rn(v0.w, v3.y)) <= 32768.0f &&
                                fabsf(__fmul_rn(v0.w, v3.z)) <= 32768.0f && isfinite(v1.w) && isfinite(v2.w) &&
                                isfinite(v3.w);
            if (!own_ok) val.x = __int_as_float(0x7fffffff);
            psf::insert_warp<kMode, kHier, false, true>(t, valid, v0, v1, v2, val, &max_len, stage, &leaders);
            c_next = c;
            le_next = le;
        }
    }
    psf::bulk_wait_done();  // this thread's sums have landed before the kernel ends
    if (max_len) atomicMax(&s_max_probe, max_len);
    if ((threadIdx.x & 31u) == 0 && leaders) atomicAdd(&s_leaders, static_cast<unsigned long long>(leaders));
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_max_probe) atomicMax(&t.hdr->max_probe, s_max_probe);
        if (s_leaders) atomicAdd(&t.hdr->leaders, s_leaders);
    }
}

// k_insert with the vertex records staged through shared memory.  Every warp owns a
// double buffer of 2 KB tiles (32 records) and its own mbarriers: lane 0 starts the bulk
// copy of the warp's next tile, then waits for the current one; the warps of a block
// never wait for each other.
constexpr unsigned kWarpsPerBlock = kThreads / 32;

template <int kMode, bool kHier>
__global__ void __launch_bounds__(kThreads, 5) k_insert_staged(TableView t, const float4* __restrict__ v, unsigned long long n) {
    __shared__ alignas(128) float4 s_tile[kWarpsPerBlock][2][32 * 4];
    __shared__ alignas(8) unsigned long long s_bar[kWarpsPerBlock][2];
    __shared__ unsigned s_max_probe;
    __shared__ unsigned long long s_leaders;
    __shared__ psf::LaneSums s_stage[kThreads];
    const unsigned lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    if (lane == 0) {
        psf::mbar_init(&s_bar[wib][0]);
        psf::mbar_init(&s_bar[wib][1]);
        psf::mbar_init_fence();
    }
    if (threadIdx.x == 0) {
        s_max_probe = 0;
        s_leaders = 0;
    }
    __syncthreads();
    const unsigned long long ntiles = (n + 31) / 32;
    const unsigned long long nwarps = static_cast<unsigned long long>(gridDim.x) * kWarpsPerBlock;
    auto issue = [&](unsigned long long tile, unsigned buf) {
        const unsigned long long first = tile * 32;
        const unsigned long long cnt = n - first < 32 ? n - first : 32;
        psf::bulk_load(s_tile[wib][buf], v + 4 * first, static_cast<unsigned>(cnt * 64), &s_bar[wib][buf]);
    };
    psf::LaneSums* stage = s_stage + (threadIdx.x & ~31u);
    unsigned max_len = 0, leaders = 0;
    unsigned long long tile = static_cast<unsigned long long>(blockIdx.x) * kWarpsPerBlock + wib;
    if (lane == 0 && tile < ntiles) issue(tile, 0);
    bool ok = true, pending_other = false;
    unsigned k = 0;
    for (; tile < ntiles; tile += nwarps, ++k) {
        const unsigned buf = k & 1u;
        int got = 1;
        if (lane == 0) {
            const unsigned long long next = tile + nwarps;
            pending_other = next < ntiles;
            if (pending_other) issue(next, buf ^ 1u);
            got = psf::mbar_wait(&s_bar[wib][buf], (k >> 1) & 1u);
        }
        ok = __shfl_sync(psf::kFull, got, 0) != 0;
        __syncwarp();  // lane 0 saw the tile land; order the other lanes' reads after it
        if (!ok) break;
        const unsigned long long i = tile * 32 + lane;
        const bool valid = i < n;
        float4 v0 = make_float4(0, 0, 0, 0), v1 = v0, v2 = v0, v3 = v0;
        if (valid) psf::read_staged(s_tile[wib][buf], lane, v0, v1, v2, v3);
        psf::insert_warp<kMode, kHier>(t, valid, v0, v1, v2, v3, &max_len, stage, &leaders);
        __syncwarp();  // the tile is consumed before its buffer is refilled
    }
    if (!ok && lane == 0) {
        atomicOr(&t.hdr->status, psf::kStatusTimeout);
        // let a copy still in flight land before the warp leaves (bounded)
        if (pending_other) psf::mbar_wait(&s_bar[wib][(k & 1u) ^ 1u], ((k + 1) >> 1) & 1u);
    }
    psf::bulk_wait_done();  // this thread's sums have landed before the kernel ends
    if (max_len) atomicMax(&s_max_probe, max_len);
    if (lane == 0 && leaders) atomicAdd(&s_leaders, static_cast<unsigned long long>(leaders));
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_max_probe) atomicMax(&t.hdr->max_probe, s_max_probe);
        if (s_leaders) atomicAdd(&t.hdr->leaders, s_leaders);
    }
}

// k_query with the vertex records staged through shared memory, per warp: a warp owns 32
// consecutive paths and walks their depths from last to first; each depth of those paths
// is one contiguous 2 KB tile, copied while the previous one is probed.
__global__ void __launch_bounds__(kThreads, 5) k_query_staged(TableView t, psf::Estimator e, const float4* __restrict__ v,
                                                           unsigned P, unsigned D, float* __restrict__ out) {
    __shared__ alignas(128) float4 s_tile[kWarpsPerBlock][2][32 * 4];
    __shared__ alignas(8) unsigned long long s_bar[kWarpsPerBlock][2];
    const unsigned lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    if (lane == 0) {
        psf::mbar_init(&s_bar[wib][0]);
        psf::mbar_init(&s_bar[wib][1]);
        psf::mbar_init_fence();
    }
    __syncwarp();
    const unsigned long long nunits = (static_cast<unsigned long long>(P) + 31) / 32;
    const unsigned long long nwarps = static_cast<unsigned long long>(gridDim.x) * kWarpsPerBlock;
    auto issue = [&](unsigned long long u, unsigned j, unsigned buf) {
        const unsigned long long first = u * 32;
        const unsigned long long cnt = P - first < 32 ? P - first : 32;
        psf::bulk_load(s_tile[wib][buf], v + 4 * (static_cast<unsigned long long>(j) * P + first), static_cast<unsigned>(cnt * 64),
                       &s_bar[wib][buf]);
    };
    unsigned long long u = static_cast<unsigned long long>(blockIdx.x) * kWarpsPerBlock + wib;
    unsigned j = D - 1;
    if (lane == 0 && u < nunits) issue(u, j, 0);
    bool ok = true, pending_other = false;
    unsigned k = 0;
    float3 c_next = make_float3(0.0f, 0.0f, 0.0f);
    while (u < nunits) {
        const unsigned buf = k & 1u;
        const unsigned long long nu = j > 0 ? u : u + nwarps;
        const unsigned nj = j > 0 ? j - 1 : D - 1;
        int got = 1;
        if (lane == 0) {
            pending_other = nu < nunits;
            if (pending_other) issue(nu, nj, buf ^ 1u);
            got = psf::mbar_wait(&s_bar[wib][buf], (k >> 1) & 1u);
        }
        ok = __shfl_sync(psf::kFull, got, 0) != 0;
        __syncwarp();
        if (!ok) break;
        if (j == D - 1) c_next = make_float3(0.0f, 0.0f, 0.0f);
        const unsigned long long p = u * 32 + lane;
        if (p < P) {
            float4 v0, v1, v2, v3;
            psf::read_staged(s_tile[wib][buf], lane, v0, v1, v2, v3);
            const float3 c = psf::cell_value(t, v0, v1, v2, false, psf::read_level(t, j));
            float o0 = v3.x, o1 = v3.y, o2 = v3.z;
            if (j + 1 < D && j >= e.j_begin && j < e.j_end) {
                o0 = psf::combine(e, v3.x, v1.w, c_next.x, c.x);
                o1 = psf::combine(e, v3.y, v2.w, c_next.y, c.y);
                o2 = psf::combine(e, v3.z, v3.w, c_next.z, c.z);
            }
            float* o = out + 3 * (static_cast<unsigned long long>(j) * P + p);
            o[0] = o0;
            o[1] = o1;
            o[2] = o2;
            c_next = c;
        }
        __syncwarp();  // the tile is consumed before its buffer is refilled
        u = nu;
        j = nj;
        ++k;
    }
    if (!ok && lane == 0) {
        atomicOr(&t.hdr->status, psf::kStatusTimeout);
        if (pending_other) psf::mbar_wait(&s_bar[wib][(k & 1u) ^ 1u], ((k + 1) >> 1) & 1u);
    }
}

template <bool kSH = false>
__global__ void __launch_bounds__(kThreads, kSH ? 3 : 4) k_update(TableView t) {
    __shared__ unsigned long long s_touched;
    if (threadIdx.x == 0) s_touched = 0;
    __syncthreads();
    const unsigned long long nwords = ((1ull << t.log2cap) + 31ull) >> 5;
    const unsigned long long warp = (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (static_cast<unsigned long long>(gridDim.x) * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        // every earlier kernel on this stream has finished: publish the sticky status
        if (t.h_status) *reinterpret_cast<volatile unsigned*>(t.h_status) = t.hdr->status;
        t.hdr->iterations += 1;
    }
    unsigned long long touched = 0;
    for (unsigned long long w0 = warp * 32ull; w0 < nwords; w0 += nwarps * 32ull) touched += psf::update_words<kSH>(t, w0, nwords);
    if ((threadIdx.x & 31u) == 0 && touched) atomicAdd(&s_touched, touched);
    __syncthreads();
    if (threadIdx.x == 0 && s_touched) atomicAdd(&t.hdr->touched, s_touched);
}

template <bool kSlots = false, bool kSH = false>
__global__ void __launch_bounds__(kThreads) k_query(TableView t, psf::Estimator e, const float4* __restrict__ v,
                                                    unsigned P, unsigned D, float* __restrict__ out,
                                                    const unsigned* __restrict__ slots = nullptr) {
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long p = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; p < P;
         p += stride)
        psf::query_path<kSlots, kSH>(t, e, v, P, D, p, out, slots);
}

// The query split by depth (psf::query_tile): one warp per tile of 32 / D paths, grid-stride
// over the tiles.  Requires D <= 32.
template <bool kSlots, bool kSH>
__global__ void __launch_bounds__(kThreads) k_query_tiled(TableView t, psf::Estimator e, const float4* __restrict__ v,
                                                          unsigned P, unsigned D, float* __restrict__ out,
                                                          const unsigned* __restrict__ slots) {
    const unsigned long long ntiles = psf::query_tiles(P, D);
    const unsigned long long warp = (static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = (static_cast<unsigned long long>(gridDim.x) * blockDim.x) >> 5;
    for (unsigned long long tile = warp; tile < ntiles; tile += nwarps)
        psf::query_tile<kSlots, kSH>(t, e, v, P, D, tile, out, slots);
}

__global__ void __launch_bounds__(kThreads) k_export(TableView t, unsigned long long s0, unsigned long long s1,
                                                     psf_cell_record* out, unsigned* count) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long base = s0 + static_cast<unsigned long long>(blockIdx.x) * blockDim.x; base < s1;
         base += stride) {
        const unsigned long long s = base + threadIdx.x;
        const unsigned long long key = s < s1 ? *psf::key_ptr(t, s) : psf::kEmpty;
        const bool live = key != psf::kEmpty;
        const unsigned m = __ballot_sync(psf::kFull, live);
        if (!m) continue;
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(count, __popc(m));
        first = __shfl_sync(psf::kFull, first, 0);
        if (!live) continue;
        psf_cell_record r;
        r.key = key;
        const Slot& a = t.slots[s];
        r.sum[0] = a.s[0];
        r.sum[1] = a.s[1];
        r.sum[2] = a.s[2];
        r.c_new = a.c;
        r.c_old = a.c_old;
        const float4 L = a.L;
        r.L[0] = L.x;
        r.L[1] = L.y;
        r.L[2] = L.z;
        if (t.mirror) {
            const uint2 h = t.mirror[s];
            r.L_fp16[0] = static_cast<uint16_t>(h.x & 0xffffu);
            r.L_fp16[1] = static_cast<uint16_t>(h.x >> 16);
            r.L_fp16[2] = static_cast<uint16_t>(h.y & 0xffffu);
        } else {
            r.L_fp16[0] = r.L_fp16[1] = r.L_fp16[2] = 0;
        }
        r.pad = 0;
        out[first + __popc(m & ((1u << lane) - 1u))] = r;
    }
}

__global__ void __launch_bounds__(kThreads) k_export_sh(TableView t, unsigned long long s0, unsigned long long s1,
                                                        psf_sh_cell_record* out, unsigned* count) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long base = s0 + static_cast<unsigned long long>(blockIdx.x) * blockDim.x; base < s1;
         base += stride) {
        const unsigned long long s = base + threadIdx.x;
        const unsigned long long key = s < s1 ? *psf::key_ptr(t, s) : psf::kEmpty;
        const bool live = key != psf::kEmpty;
        const unsigned m = __ballot_sync(psf::kFull, live);
        if (!m) continue;
        unsigned first = 0;
        if (lane == 0) first = atomicAdd(count, __popc(m));
        first = __shfl_sync(psf::kFull, first, 0);
        if (!live) continue;
        psf_sh_cell_record r;
        r.key = key;
        const psf::SlotSH& a = t.sh[s];
        for (int c = 0; c < psf::kShSums; ++c) r.sum[c] = a.s[c];
        r.c_old = a.c_old;
        r.coef[0] = a.coef_a.x;
        r.coef[1] = a.coef_a.y;
        r.coef[2] = a.coef_a.z;
        r.coef[3] = a.coef_a.w;
        r.coef[4] = a.coef_c.x;
        r.coef[5] = a.coef_c.y;
        out[first + __popc(m & ((1u << lane) - 1u))] = r;
    }
}

// Pre-aggregated records of other tables (a sharded session's exchange) added to this
// table: one record per thread, the warp probing together; each record's three sums and
// counter are added with 64-bit atomics and the cell is marked touched.  A record whose key
// has bit 63 set is not a cell key: it is dropped with PSF_STATUS_RANGE.
__global__ void __launch_bounds__(kThreads) k_insert_records(TableView t, const psf_record* __restrict__ r,
                                                             unsigned long long n) {
    __shared__ unsigned s_max_probe;
    if (threadIdx.x == 0) s_max_probe = 0;
    __syncthreads();
    unsigned max_len = 0;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long base = static_cast<unsigned long long>(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        psf_record rec{};
        bool need = false;
        if (i < n) {
            rec = r[i];
            need = (rec.key >> 63) == 0;
            if (!need) {
                atomicOr(&t.hdr->status, psf::kStatusRange);
                atomicAdd(&t.hdr->dropped, 1ull);
            }
        }
        long long slot;
        unsigned len;
        psf::probe_warp(t, need, rec.key, &slot, &len);
        if (need) {
            max_len = len > max_len ? len : max_len;
            if (slot < 0) {
                atomicOr(&t.hdr->status, psf::kStatusTableFull);
                atomicAdd(&t.hdr->dropped, 1ull);
            } else {
                Slot* a = t.slots + slot;
                atomicAdd(reinterpret_cast<unsigned long long*>(&a->s[0]), static_cast<unsigned long long>(rec.sum[0]));
                atomicAdd(reinterpret_cast<unsigned long long*>(&a->s[1]), static_cast<unsigned long long>(rec.sum[1]));
                atomicAdd(reinterpret_cast<unsigned long long*>(&a->s[2]), static_cast<unsigned long long>(rec.sum[2]));
                atomicAdd(reinterpret_cast<unsigned long long*>(&a->c), static_cast<unsigned long long>(rec.c_new));
                atomicOr(t.dirty + (slot >> 5), 1u << (slot & 31));
            }
        }
    }
    if (max_len) atomicMax(&s_max_probe, max_len);
    __syncthreads();
    if (threadIdx.x == 0 && s_max_probe) atomicMax(&t.hdr->max_probe, s_max_probe);
}

// The approximant of the given cells written into this table (a sharded session's replica of
// cells other ranks own): each key is found or claimed and its FP32 approximant (and FP16
// copy) set; the cell's counters are left as they are.
__global__ void __launch_bounds__(kThreads) k_set_approximant(TableView t, const unsigned long long* __restrict__ keys,
                                                              const float* __restrict__ L, unsigned long long n) {
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long base = static_cast<unsigned long long>(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const unsigned long long key = i < n ? keys[i] : 0ull;
        const bool need = i < n && (key >> 63) == 0;
        if (i < n && !need) {
            atomicOr(&t.hdr->status, psf::kStatusRange);
            atomicAdd(&t.hdr->dropped, 1ull);
        }
        long long slot;
        unsigned len;
        psf::probe_warp(t, need, key, &slot, &len);
        if (need) {
            if (slot < 0) {
                atomicOr(&t.hdr->status, psf::kStatusTableFull);
                atomicAdd(&t.hdr->dropped, 1ull);
            } else {
                const float x = L[3 * i], y = L[3 * i + 1], z = L[3 * i + 2];
                float4 cur = t.slots[slot].L;
                cur.x = x;
                cur.y = y;
                cur.z = z;
                t.slots[slot].L = cur;
                if (t.mirror) t.mirror[slot] = psf::pack_half4(x, y, z);
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_count_live(TableView t, unsigned long long* count) {
    __shared__ unsigned long long s_count;
    if (threadIdx.x == 0) s_count = 0;
    __syncthreads();
    const unsigned long long cap = 1ull << t.log2cap;
    unsigned long long mine = 0;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long s = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; s < cap; s += stride)
        mine += *psf::key_ptr(t, s) != psf::kEmpty;
    if (mine) atomicAdd(&s_count, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_count) atomicAdd(count, s_count);
}

// Empty key fields of a table whose keys live inside the slot records.
__global__ void __launch_bounds__(kThreads) k_init_keys(TableView t) {
    const unsigned long long cap = 1ull << t.log2cap;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long s = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; s < cap; s += stride)
        *psf::key_ptr(t, s) = psf::kEmpty;
}

// Global counter reset: c_old := 0 in every slot (the approximant is kept).
__global__ void __launch_bounds__(kThreads) k_reset(TableView t) {
    const unsigned long long cap = 1ull << t.log2cap;
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    for (unsigned long long s = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; s < cap; s += stride) {
        if (t.payload == psf::kPayloadSH)
            t.sh[s].c_old = 0;
        else
            t.slots[s].c_old = 0;
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace {

// Resident 256-thread blocks per SM of kernel `fn` on this table's device (queried once per
// kernel and cached in the table; 1 if the query fails).
int resident_blocks(const psf_table* t, const void* fn) {
    for (int i = 0; i < t->occ_n; ++i)
        if (t->occ_fn[i] == fn) return t->occ_blocks[i];
    int blocks = 0;
    if (!cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kThreads, 0), "occupancy") || blocks < 1)
        blocks = 1;
    if (t->occ_n < 16) {
        t->occ_fn[t->occ_n] = fn;
        t->occ_blocks[t->occ_n] = blocks;
        ++t->occ_n;
    }
    return blocks;
}

template <typename Kernel, typename... Args>
void launch_sized(const psf_table* t, Kernel kernel, unsigned long long work, cudaStream_t st, Args... args) {
    const int grid = grid_for(t, resident_blocks(t, reinterpret_cast<const void*>(kernel)), work,
                              t->launch.insert_blocks_per_sm);
    kernel<<<grid, kThreads, 0, st>>>(args...);
}

// The insert kernels for a flat table (kHier = false) or for one with hierarchy levels.
template <bool kHier>
void launch_insert(const psf_table* t, const float4* v, unsigned long long n, cudaStream_t st) {
    const bool none = t->launch.insert_mode == 1;
    if (t->launch.vertex_staging & 1u) {
        if (none)
            launch_sized(t, k_insert_staged<psf::kAggNone, kHier>, n, st, t->view, v, n);
        else
            launch_sized(t, k_insert_staged<psf::kAggWarp, kHier>, n, st, t->view, v, n);
    } else if (none) {
        launch_sized(t, k_insert<psf::kAggNone, kHier>, n, st, t->view, v, n, 0u, static_cast<unsigned*>(nullptr));
    } else {
        launch_sized(t, k_insert<psf::kAggWarp, kHier>, n, st, t->view, v, n, 0u, static_cast<unsigned*>(nullptr));
    }
}

template <bool kHier>
void launch_insert_slots(const psf_table* t, const float4* v, uint32_t P, uint32_t D, unsigned* slots, cudaStream_t st) {
    const unsigned long long n = static_cast<unsigned long long>(P) * D;
    if (t->launch.insert_mode == 1)
        launch_sized(t, k_insert<psf::kAggNone, kHier, true>, n, st, t->view, v, n, P, slots);
    else
        launch_sized(t, k_insert<psf::kAggWarp, kHier, true>, n, st, t->view, v, n, P, slots);
}

// The depth-split query: one warp per tile of 32 / D paths, grid-stride over the tiles, sized
// by the kernel's own resident-block count.
template <bool kSlots, bool kSH>
void launch_tiled_query(const psf_table* t, const psf::Estimator& e, const float4* v, uint32_t P, uint32_t D, float* out,
                        const unsigned* slots, cudaStream_t st) {
    const unsigned T = 32u / D;
    const unsigned long long tiles = (static_cast<unsigned long long>(P) + T - 1) / T;
    const int grid = grid_for(t, resident_blocks(t, reinterpret_cast<const void*>(k_query_tiled<kSlots, kSH>)),
                              tiles * 32ull, t->launch.query_blocks_per_sm);
    k_query_tiled<kSlots, kSH><<<grid, kThreads, 0, st>>>(t->view, e, v, P, D, out, slots);
}

template <bool kHier>
void launch_insert_progressive(const psf_table* t, const float4* v, uint32_t P, uint32_t D, uint32_t field,
                               cudaStream_t st) {
    if (t->launch.insert_mode == 1)
        launch_sized(t, k_insert_progressive<psf::kAggNone, kHier>, P, st, t->view, v, P, D, field);
    else
        launch_sized(t, k_insert_progressive<psf::kAggWarp, kHier>, P, st, t->view, v, P, D, field);
}

}  // namespace

namespace {

// Every occupied cell as a record of type Rec (written by `kernel` over chunks of slots),
// sorted by key on the host.
template <typename Rec>
int export_cells(psf_table* t, void (*kernel)(TableView, unsigned long long, unsigned long long, Rec*, unsigned*),
                 Rec* h_out, size_t cap_out, size_t* n_out, void* stream) {
    if (!n_out || (cap_out && !h_out)) return PSF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned long long cap = 1ull << t->cfg.log2_capacity;
    const unsigned long long chunk = std::min<unsigned long long>(cap, 1ull << 20);
    void* scratch = nullptr;
    const size_t scratch_bytes = chunk * sizeof(Rec) + 256;
    if (!cuda_ok(cudaMallocAsync(&scratch, scratch_bytes, st), "cudaMallocAsync")) return PSF_ERR_CUDA;
    Rec* d_rec = reinterpret_cast<Rec*>(static_cast<char*>(scratch) + 256);
    unsigned* d_count = static_cast<unsigned*>(scratch);
    std::vector<Rec> all;
    int rc = PSF_OK;
    for (unsigned long long s0 = 0; s0 < cap && rc == PSF_OK; s0 += chunk) {
        unsigned n = 0;
        const int grid = grid_for(t, 4, chunk);
        if (!cuda_ok(cudaMemsetAsync(d_count, 0, sizeof(unsigned), st), "cudaMemsetAsync")) {
            rc = PSF_ERR_CUDA;
            break;
        }
        kernel<<<grid, kThreads, 0, st>>>(t->view, s0, s0 + chunk, d_rec, d_count);
        if (!cuda_ok(cudaGetLastError(), "k_export") ||
            !cuda_ok(cudaMemcpyAsync(&n, d_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") ||
            !cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize")) {
            rc = PSF_ERR_CUDA;
            break;
        }
        const size_t old = all.size();
        all.resize(old + n);
        if (n && !cuda_ok(cudaMemcpyAsync(all.data() + old, d_rec, n * sizeof(Rec), cudaMemcpyDeviceToHost, st),
                          "cudaMemcpyAsync"))
            rc = PSF_ERR_CUDA;
        if (rc == PSF_OK && !cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize")) rc = PSF_ERR_CUDA;
    }
    cudaFreeAsync(scratch, st);
    if (!cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize") && rc == PSF_OK) rc = PSF_ERR_CUDA;
    if (rc != PSF_OK) return rc;
    std::sort(all.begin(), all.end(), [](const Rec& a, const Rec& b) { return a.key < b.key; });
    *n_out = all.size();
    if (all.size() > cap_out) return PSF_ERR_NO_MEM;
    if (!all.empty()) std::memcpy(h_out, all.data(), all.size() * sizeof(Rec));
    return PSF_OK;
}

}  // namespace

extern "C" {

int psf_abi_version(void) { return PSF_ABI_VERSION; }

const char* psf_last_cuda_error(void) { return psf_g_last_error.c_str(); }

size_t psf_table_bytes(const psf_config* cfg) {
    if (!config_valid(cfg)) return 0;
    return layout_of(cfg).total;
}

int psf_create(const psf_config* cfg, void* d_mem, size_t bytes, void* stream, psf_table** out) {
    if (!out || !config_valid(cfg) || !d_mem) return PSF_ERR_INVALID_ARG;
    *out = nullptr;
    if (reinterpret_cast<uintptr_t>(d_mem) & 255u) return PSF_ERR_INVALID_ARG;
    const Layout L = layout_of(cfg);
    if (bytes < L.total) return PSF_ERR_NO_MEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    psf_table* t = new (std::nothrow) psf_table();
    if (!t) return PSF_ERR_NO_MEM;
    t->cfg = *cfg;
    t->mem = d_mem;
    t->bytes = bytes;
    if (!cuda_ok(cudaGetDevice(&t->device), "cudaGetDevice") ||
        !cuda_ok(cudaDeviceGetAttribute(&t->sms, cudaDevAttrMultiProcessorCount, t->device), "cudaDeviceGetAttribute") ||
        !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->update_blocks_per_sm,
                                                               cfg->payload == psf::kPayloadSH ? k_update<true> : k_update<false>,
                                                               kThreads, 0),
                 "occupancy") ||
        !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->query_blocks_per_sm, k_query<false>, kThreads, 0), "occupancy") ||
        !cuda_ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&t->staged_query_blocks_per_sm, k_query_staged, kThreads, 0),
                 "occupancy")) {
        delete t;
        return PSF_ERR_CUDA;
    }
    StatusWord word;
    if (!status_take(&word)) {
        delete t;
        return PSF_ERR_CUDA;
    }
    t->h_status = word.host;
    *t->h_status = 0;
    // direct vertex loads (measured: with bulk sums the TMA-staged tiles are slower, 133 vs
    // 120 us on 1280x720x4, as both go through the TMA unit), bulk sums
    t->launch = psf_launch_config{0u, 0u, 0u, 0u, 0u, 0u, 0u};
    t->view.sum_path = psf::kSumsBulk;
    char* base = static_cast<char*>(d_mem);
    TableView& v = t->view;
    v.hdr = reinterpret_cast<DevHeader*>(base + L.hdr);
    v.slots = reinterpret_cast<Slot*>(base + L.slots);
    if (keys_inline(cfg)) {
        v.keys = &v.slots[0].key;
        v.key_stride = sizeof(Slot) / sizeof(unsigned long long);
    } else {
        v.keys = reinterpret_cast<unsigned long long*>(base + L.keys);
        v.key_stride = 1;
    }
    v.slots = reinterpret_cast<Slot*>(base + L.slots);
    v.mirror = cfg->cache_fp16 ? reinterpret_cast<uint2*>(base + L.mirror) : nullptr;
    v.dirty = reinterpret_cast<unsigned*>(base + L.dirty);
    v.h_status = word.dev;
    t->d_status = word.dev;
    v.log2cap = cfg->log2_capacity;
    v.max_probe = std::min<uint32_t>(PSF_MAX_PROBE, 1u << std::min<uint32_t>(cfg->log2_capacity, 31u));
    v.q = cfg->pos_bits_q;
    v.d = cfg->dir_bits_d;
    v.use_normal = cfg->use_normal;
    v.frac_bits = cfg->frac_bits;
    v.cv_max_depth = cfg->cv_max_depth;
    v.blend_mode = cfg->blend_mode;
    v.alpha_min = cfg->alpha_min;
    v.beta = cfg->beta;
    v.levels = cfg->levels == 0 ? 1u : cfg->levels;
    v.payload = cfg->payload;
    v.ridge = cfg->sh_ridge;
    v.sh = cfg->payload == psf::kPayloadSH ? reinterpret_cast<psf::SlotSH*>(base + L.slots) : nullptr;

    const size_t cap = size_t{1} << cfg->log2_capacity;
    bool ok = cuda_ok(cudaMemsetAsync(base, 0, L.total, st), "cudaMemsetAsync");
    if (ok && !keys_inline(cfg)) {
        ok = cuda_ok(cudaMemsetAsync(base + L.keys, 0xff, cap * sizeof(unsigned long long), st), "cudaMemsetAsync");
    } else if (ok) {
        k_init_keys<<<grid_for(t, 4, cap), kThreads, 0, st>>>(v);
        ok = cuda_ok(cudaGetLastError(), "k_init_keys");
    }
    if (!ok) {
        status_give(word);
        delete t;
        return PSF_ERR_CUDA;
    }
    *out = t;
    return PSF_OK;
}

int psf_insert(psf_table* t, const float* d_vertices, uint64_t n, void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    if (n == 0) return PSF_OK;
    if (!d_vertices || (reinterpret_cast<uintptr_t>(d_vertices) & 15u)) return PSF_ERR_INVALID_ARG;
    const float4* v = reinterpret_cast<const float4*>(d_vertices);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    psf_count_iteration_vertices(t, n);
    if (t->view.payload == psf::kPayloadSH) {
        if (t->launch.insert_mode == 1)
            launch_sized(t, k_insert_sh<psf::kAggNone>, n, st, t->view, v, n, static_cast<unsigned*>(nullptr));
        else
            launch_sized(t, k_insert_sh<psf::kAggWarp>, n, st, t->view, v, n, static_cast<unsigned*>(nullptr));
    } else if (t->view.levels > 1) {
        launch_insert<true>(t, v, n, st);
    } else {
        launch_insert<false>(t, v, n, st);
    }
    return cuda_ok(cudaGetLastError(), "k_insert") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_insert_progressive(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, uint32_t field, void* stream) {
    if (!t || field > 1 || t->view.payload != psf::kPayloadRGB) return PSF_ERR_INVALID_ARG;
    if (P == 0 || D == 0) return PSF_OK;
    if (!d_vertices || (reinterpret_cast<uintptr_t>(d_vertices) & 15u)) return PSF_ERR_INVALID_ARG;
    const float4* v = reinterpret_cast<const float4*>(d_vertices);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    psf_count_iteration_vertices(t, static_cast<unsigned long long>(P) * D);
    if (t->view.levels > 1)
        launch_insert_progressive<true>(t, v, P, D, field, st);
    else
        launch_insert_progressive<false>(t, v, P, D, field, st);
    return cuda_ok(cudaGetLastError(), "k_insert_progressive") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_update(psf_table* t, void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    const unsigned long long nwords = ((1ull << t->cfg.log2_capacity) + 31ull) >> 5;
    const int grid = grid_for(t, t->update_blocks_per_sm, nwords, t->launch.update_blocks_per_sm);  // a warp per 32 words
    if (t->view.payload == psf::kPayloadSH)
        k_update<true><<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(t->view);
    else
        k_update<false><<<grid, kThreads, 0, static_cast<cudaStream_t>(stream)>>>(t->view);
    if (!cuda_ok(cudaGetLastError(), "k_update")) return PSF_ERR_CUDA;
    t->iter_vertices = 0;
    return static_cast<int>((*reinterpret_cast<volatile unsigned*>(t->h_status) | t->host_status) & 0x7fffffffu);
}

namespace {

int launch_query(psf_table* t, const psf::Estimator& e, const float* d_vertices, uint32_t P, uint32_t D, float* d_out_rgb,
                 void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    if (P == 0 || D == 0) return PSF_OK;
    if (!d_vertices || !d_out_rgb || (reinterpret_cast<uintptr_t>(d_vertices) & 15u) ||
        (reinterpret_cast<uintptr_t>(d_out_rgb) & 3u))
        return PSF_ERR_INVALID_ARG;
    const float4* v = reinterpret_cast<const float4*>(d_vertices);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (t->launch.query_layout == 1 && D <= 32u) {
        if (t->view.payload == psf::kPayloadSH)
            launch_tiled_query<false, true>(t, e, v, P, D, d_out_rgb, nullptr, st);
        else
            launch_tiled_query<false, false>(t, e, v, P, D, d_out_rgb, nullptr, st);
    } else if (t->view.payload == psf::kPayloadSH) {
        const int grid = grid_for(t, resident_blocks(t, reinterpret_cast<const void*>(k_query<false, true>)), P,
                                  t->launch.query_blocks_per_sm);
        k_query<false, true><<<grid, kThreads, 0, st>>>(t->view, e, v, P, D, d_out_rgb);
    } else if (t->launch.vertex_staging & 2u) {
        const int grid = grid_for(t, t->staged_query_blocks_per_sm, P, t->launch.query_blocks_per_sm);
        k_query_staged<<<grid, kThreads, 0, st>>>(t->view, e, v, P, D, d_out_rgb);
    } else {
        const int grid = grid_for(t, t->query_blocks_per_sm, P, t->launch.query_blocks_per_sm);
        k_query<false><<<grid, kThreads, 0, st>>>(t->view, e, v, P, D, d_out_rgb);
    }
    return cuda_ok(cudaGetLastError(), "k_query") ? PSF_OK : PSF_ERR_CUDA;
}

}  // namespace

int psf_query_cv(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, float* d_out_rgb, void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    return launch_query(t, psf::cv_estimator(t->view), d_vertices, P, D, d_out_rgb, stream);
}

int psf_query_biased(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, float gamma, uint32_t j_begin,
                     uint32_t j_end, float* d_out_rgb, void* stream) {
    if (!t || !(gamma == gamma)) return PSF_ERR_INVALID_ARG;
    return launch_query(t, psf::Estimator{gamma, gamma, 1.0f, j_begin, j_end}, d_vertices, P, D, d_out_rgb, stream);
}

int psf_insert_slots(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, uint32_t* d_slots, void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    const unsigned long long n = static_cast<unsigned long long>(P) * D;
    if (n == 0) return PSF_OK;
    if (!d_vertices || !d_slots || (reinterpret_cast<uintptr_t>(d_vertices) & 15u) ||
        (reinterpret_cast<uintptr_t>(d_slots) & 3u))
        return PSF_ERR_INVALID_ARG;
    const float4* v = reinterpret_cast<const float4*>(d_vertices);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    psf_count_iteration_vertices(t, n);
    if (t->view.payload == psf::kPayloadSH) {
        if (t->launch.insert_mode == 1)
            launch_sized(t, k_insert_sh<psf::kAggNone, true>, n, st, t->view, v, n, d_slots);
        else
            launch_sized(t, k_insert_sh<psf::kAggWarp, true>, n, st, t->view, v, n, d_slots);
    } else if (t->view.levels > 1)
        launch_insert_slots<true>(t, v, P, D, d_slots, st);
    else
        launch_insert_slots<false>(t, v, P, D, d_slots, st);
    return cuda_ok(cudaGetLastError(), "k_insert") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_query_cv_slots(psf_table* t, const float* d_vertices, const uint32_t* d_slots, uint32_t P, uint32_t D,
                       float* d_out_rgb, void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    if (P == 0 || D == 0) return PSF_OK;
    if (!d_vertices || !d_slots || !d_out_rgb || (reinterpret_cast<uintptr_t>(d_vertices) & 15u) ||
        (reinterpret_cast<uintptr_t>(d_slots) & 3u) || (reinterpret_cast<uintptr_t>(d_out_rgb) & 3u))
        return PSF_ERR_INVALID_ARG;
    const float4* v = reinterpret_cast<const float4*>(d_vertices);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (t->view.payload == psf::kPayloadSH) {
        const int grid = grid_for(t, resident_blocks(t, reinterpret_cast<const void*>(k_query<true, true>)), P,
                                  t->launch.query_blocks_per_sm);
        k_query<true, true><<<grid, kThreads, 0, st>>>(t->view, psf::cv_estimator(t->view), v, P, D, d_out_rgb, d_slots);
    } else if (t->launch.query_layout == 1 && D <= 32u) {
        launch_tiled_query<true, false>(t, psf::cv_estimator(t->view), v, P, D, d_out_rgb, d_slots, st);
    } else {
        const int grid = grid_for(t, resident_blocks(t, reinterpret_cast<const void*>(k_query<true>)), P,
                                  t->launch.query_blocks_per_sm);
        k_query<true><<<grid, kThreads, 0, st>>>(t->view, psf::cv_estimator(t->view), v, P, D, d_out_rgb, d_slots);
    }
    return cuda_ok(cudaGetLastError(), "k_query") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_step(psf_table* t, const float* d_vertices, uint32_t P, uint32_t D, float* d_out_rgb, void* stream) {
    int rc = psf_insert(t, d_vertices, static_cast<uint64_t>(P) * D, stream);
    if (rc != PSF_OK) return rc;
    rc = psf_update(t, stream);
    if (rc < 0) return rc;
    return psf_query_cv(t, d_vertices, P, D, d_out_rgb, stream);
}

int psf_insert_records(psf_table* t, const psf_record* d_records, uint64_t n, void* stream) {
    if (!t || t->view.payload != psf::kPayloadRGB) return PSF_ERR_INVALID_ARG;
    if (n == 0) return PSF_OK;
    if (!d_records || (reinterpret_cast<uintptr_t>(d_records) & 7u)) return PSF_ERR_INVALID_ARG;
    launch_sized(t, k_insert_records, n, static_cast<cudaStream_t>(stream), t->view, d_records,
                 static_cast<unsigned long long>(n));
    return cuda_ok(cudaGetLastError(), "k_insert_records") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_set_approximant(psf_table* t, const uint64_t* d_keys, const float* d_L, uint64_t n, void* stream) {
    if (!t || t->view.payload != psf::kPayloadRGB) return PSF_ERR_INVALID_ARG;
    if (n == 0) return PSF_OK;
    if (!d_keys || !d_L || (reinterpret_cast<uintptr_t>(d_keys) & 7u) || (reinterpret_cast<uintptr_t>(d_L) & 3u))
        return PSF_ERR_INVALID_ARG;
    launch_sized(t, k_set_approximant, n, static_cast<cudaStream_t>(stream), t->view,
                 reinterpret_cast<const unsigned long long*>(d_keys), d_L, static_cast<unsigned long long>(n));
    return cuda_ok(cudaGetLastError(), "k_set_approximant") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_reset(psf_table* t, void* stream) {
    if (!t) return PSF_ERR_INVALID_ARG;
    const unsigned long long cap = 1ull << t->cfg.log2_capacity;
    k_reset<<<grid_for(t, 4, cap), kThreads, 0, static_cast<cudaStream_t>(stream)>>>(t->view);
    return cuda_ok(cudaGetLastError(), "k_reset") ? PSF_OK : PSF_ERR_CUDA;
}

int psf_set_launch_config(psf_table* t, const psf_launch_config* c) {
    if (!t || !c || c->insert_mode > 1 || c->vertex_staging > 3 || c->sum_reduction > 1 || c->query_layout > 1)
        return PSF_ERR_INVALID_ARG;
    t->launch = *c;
    t->view.sum_path = c->sum_reduction;
    return PSF_OK;
}

int psf_get_launch_config(const psf_table* t, psf_launch_config* out) {
    if (!t || !out) return PSF_ERR_INVALID_ARG;
    *out = t->launch;
    return PSF_OK;
}

int psf_export(psf_table* t, psf_cell_record* h_out, size_t cap_out, size_t* n_out, void* stream) {
    if (!t || t->view.payload != psf::kPayloadRGB) return PSF_ERR_INVALID_ARG;
    return export_cells(t, k_export, h_out, cap_out, n_out, stream);
}

int psf_export_sh(psf_table* t, psf_sh_cell_record* h_out, size_t cap_out, size_t* n_out, void* stream) {
    if (!t || t->view.payload != psf::kPayloadSH) return PSF_ERR_INVALID_ARG;
    return export_cells(t, k_export_sh, h_out, cap_out, n_out, stream);
}

int psf_get_stats(psf_table* t, psf_stats* out, void* stream) {
    if (!t || !out) return PSF_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* scratch = nullptr;
    if (!cuda_ok(cudaMallocAsync(&scratch, 256 + sizeof(DevHeader), st), "cudaMallocAsync")) return PSF_ERR_CUDA;
    unsigned long long* d_count = static_cast<unsigned long long*>(scratch);
    DevHeader h{};
    unsigned long long live = 0;
    bool ok = cuda_ok(cudaMemsetAsync(d_count, 0, sizeof(unsigned long long), st), "cudaMemsetAsync");
    if (ok) {
        k_count_live<<<grid_for(t, 4, 1ull << t->cfg.log2_capacity), kThreads, 0, st>>>(t->view, d_count);
        ok = cuda_ok(cudaGetLastError(), "k_count_live") &&
             cuda_ok(cudaMemcpyAsync(&live, d_count, sizeof(live), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync") &&
             cuda_ok(cudaMemcpyAsync(&h, t->view.hdr, sizeof(h), cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync");
    }
    cudaFreeAsync(scratch, st);
    ok = cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize") && ok;
    if (!ok) return PSF_ERR_CUDA;
    out->capacity = 1ull << t->cfg.log2_capacity;
    out->live_cells = live;
    out->dropped_vertices = h.dropped;
    out->zero_weight_vertices = h.zero_weight;
    out->iterations = h.iterations;
    out->status = h.status | t->host_status;
    out->max_probe = h.max_probe;
    out->table_bytes = layout_of(&t->cfg).total;
    out->touched_cells = h.touched;
    out->leader_groups = h.leaders;
    return PSF_OK;
}

int psf_destroy(psf_table* t) {
    if (!t) return PSF_OK;
    status_give(StatusWord{t->h_status, t->d_status});  // no CUDA call: nothing here waits on the device
    delete t;
    return PSF_OK;
}

}  // extern "C"
