// psf_device.cuh -- device-side building blocks of the filtering hot path (sm_103a).
//
// Table memory (one contiguous caller-owned allocation, every array 256-byte aligned):
//   DevHeader                       status word and counters
//   keys   u64[cap]                 packed cell key or kEmpty (open addressing, linear probe);
//                                   absent when the keys live inside the slot records
//   slots  Slot[cap]  (64 B)        sums + c_new (bytes 0-31), key (32-39, when inside),
//                                   c_old (40-47), approximant L~ (48-63): one aligned
//                                   64-byte block per cell
//   mirror uint2[cap] (8 B)         FP16 copy of L~ read by queries (cache_fp16 = 1)
//   dirty  u32[cap/32]              one bit per slot: touched this iteration
// Tables with the YCoCg two-band SH payload keep dense keys and 192-byte SlotSH records
// (sixteen 64-bit sums, c_old, six coefficients) instead of Slot and the FP16 copy.
// Inserts touch keys + the first 32-byte sector of a slot (atomics); the blend reads and
// writes exactly one 64-byte block per touched cell, the DRAM access granularity, so
// scattered cells cost no partial bursts; queries read keys + the second sector of the
// slot (FP32) or the compact 8-byte FP16 copy.

#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

namespace psf {

constexpr unsigned long long kEmpty = ~0ull;  // bit 63 set: never a valid key
constexpr int kThreads = 256;                 // threads per block of every kernel
constexpr unsigned kFull = 0xffffffffu;

constexpr unsigned kStatusTableFull = 1u;
constexpr unsigned kStatusRange = 2u;
constexpr unsigned kStatusTimeout = 4u;

struct DevHeader {
    unsigned int status;
    unsigned int max_probe;
    unsigned long long dropped;
    unsigned long long zero_weight;
    unsigned long long iterations;
    unsigned long long touched;  // cells blended by all updates so far
    unsigned long long leaders;  // (warp, key) groups scattered by all inserts so far
    unsigned int barrier_count;  // grid barrier of the batched kernel
    unsigned int barrier_gen;
    unsigned int pad[50];
};
static_assert(sizeof(DevHeader) == 256, "header is one 256-byte block");

struct alignas(64) Slot {
    long long s[3];          // this iteration's sum of round(w L_c 2^F)
    long long c;             // this iteration's counter c_new = sum of round(w 2^F)
    unsigned long long key;  // the cell key when keys live in the slots (unused otherwise)
    long long c_old;         // cumulative counter of blended iterations
    float4 L;                // the approximant (r, g, b, unused)
};
static_assert(sizeof(Slot) == 64, "one slot is one 64-byte block");

// Insert aggregation modes (a launch-time choice, results are identical)
constexpr int kAggWarp = 0;  // lanes of a warp on one key merged, one probe per group
constexpr int kAggNone = 1;  // every vertex probes and adds on its own

struct SlotSH;  // the SH payload's slot record (below)

struct TableView {
    DevHeader* hdr;
    unsigned long long* keys;  // key of slot s at keys[s * key_stride]
    unsigned key_stride;       // 1: dense key array; 8: the key field of the 64-byte slot records
    Slot* slots;
    uint2* mirror;  // FP16 query copy (cache_fp16), else nullptr
    unsigned* dirty;
    unsigned* h_status;  // host-mapped copy of the status word (may be nullptr)
    uint32_t log2cap;
    uint32_t max_probe;
    uint32_t q;
    uint32_t d;
    uint32_t use_normal;
    uint32_t frac_bits;
    uint32_t cv_max_depth;
    uint32_t blend_mode;
    float alpha_min;
    float beta;
    uint32_t levels;    // hierarchy levels, 1..4 (1: a flat table)
    uint32_t sum_path;  // how a group's sums reach its slot: kSumsBulk or kSumsRed
    uint32_t payload;   // kPayloadRGB or kPayloadSH (the cell holds a YCoCg two-band SH fit)
    float ridge;        // SH payload: ridge weight on band 1, relative to the cell's weight
    SlotSH* sh;         // SH payload: the 192-byte slot records (slots is unused then)
};

constexpr uint32_t kPayloadRGB = 0;
constexpr uint32_t kPayloadSH = 1;

constexpr uint32_t kSumsBulk = 0;  // one 32-byte bulk reduction from shared memory (TMA)
constexpr uint32_t kSumsRed = 1;   // four 64-bit reductions

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------
// Bulk staging of vertex tiles into shared memory: one thread arms an mbarrier with the
// tile's byte count and starts a cp.async.bulk copy (the TMA unit moves the bytes, not the
// load/store units); the block waits on the barrier's phase.  Waits are bounded.
// ---------------------------------------------------------------------------
constexpr unsigned kTileVerts = kThreads;  // one vertex per thread
constexpr unsigned long long kStageTimeoutNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// L2 eviction-priority policies for per-access cache hints (createpolicy, sm_80+).
__device__ __forceinline__ unsigned long long policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long policy_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// A hash key read at L2 (bypassing L1) that asks L2 to keep the line: the key array is the
// part of the table every probe touches.
__device__ __forceinline__ unsigned long long load_key(const unsigned long long* p, unsigned long long policy) {
    unsigned long long v;
    asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(policy));
    return v;
}

// The FP16 copy is written by the blend and read by the query that follows it: the blend's
// stores carry an L2 evict-last hint, so the lines it writes stay in L2 for the query
// (measured on 1920x1080, depth 5: blend 168 -> 154 us, query 231 -> 215 us).
__device__ __forceinline__ void store_mirror(uint2* p, uint2 v) {
    const unsigned long long keep = policy_evict_last();
    asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(keep) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Arm `bar` for `bytes` and copy them from global to shared memory (called by one thread).
// Both addresses are 16-byte aligned and bytes is a multiple of 16.
// The vertex records are read once: the copy carries an evict-first L2 policy so the stream
// does not push the table out of L2.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    const unsigned long long policy = policy_evict_first();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait (at most about a second) for the phase of `bar` with this parity to complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    while (!mbar_test(bar, parity))
        if (global_timer_ns() - t0 > kStageTimeoutNs) return false;
    return true;
}

// Vertex t of a staged tile.  Lanes read the four 16-byte vectors of their 64-byte records
// in an order rotated by (t >> 1) & 3, so the eight lanes of each quarter-warp touch eight
// different groups of banks; selects put the vectors back in order.
__device__ __forceinline__ void read_staged(const float4* tile, unsigned t, float4& v0, float4& v1, float4& v2,
                                            float4& v3) {
    const unsigned rot = (t >> 1) & 3u;
    const float4* rec = tile + 4 * t;
    const float4 r0 = rec[rot], r1 = rec[(1u + rot) & 3u], r2 = rec[(2u + rot) & 3u], r3 = rec[(3u + rot) & 3u];
    // vector m was read at step (m - rot) & 3
    v0 = rot == 0 ? r0 : rot == 1 ? r3 : rot == 2 ? r2 : r1;
    v1 = rot == 0 ? r1 : rot == 1 ? r0 : rot == 2 ? r3 : r2;
    v2 = rot == 0 ? r2 : rot == 1 ? r1 : rot == 2 ? r0 : r3;
    v3 = rot == 0 ? r3 : rot == 1 ? r2 : rot == 2 ? r1 : r0;
}

__device__ __forceinline__ unsigned long long* key_ptr(const TableView& t, unsigned long long s) {
    return t.keys + s * t.key_stride;
}

// ---------------------------------------------------------------------------
// Cell key: Section "Basis functions and data structures: spatio-directional
// hashing".  Every decision that yields an integer is taken in FP32 with explicitly
// rounded operations (no contraction), in a fixed order.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// floor(p * 2^q) biased by 2^15; false outside [-2^15, 2^15) or for NaN.
__device__ __forceinline__ bool quantise_axis(float p, float scale, unsigned* out) {
    const float f = floorf(__fmul_rn(p, scale));  // exact: power-of-two scale
    if (!(f >= -32768.0f && f <= 32767.0f)) return false;
    *out = static_cast<unsigned>(static_cast<int>(f) + 32768);
    return true;
}

__device__ __forceinline__ unsigned dominant_axis_bin(float nx, float ny, float nz) {
    const float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
    if (ax >= ay && ax >= az) return nx >= 0.0f ? 0u : 1u;
    if (ay >= az) return ny >= 0.0f ? 2u : 3u;
    return nz >= 0.0f ? 4u : 5u;
}

__device__ __forceinline__ unsigned octa_bin(float g, float half, int top) {
    int b = static_cast<int>(floorf(__fmul_rn(g, half)));
    b = b < 0 ? 0 : b;
    return static_cast<unsigned>(b > top ? top : b);
}

// Packed key of the vertex (v0 = position, v1 = normal, v2 = incoming direction).
__device__ __forceinline__ bool cell_key(const TableView& t, const float4& v0, const float4& v1,
                                         const float4& v2, unsigned long long* key) {
    if (!(isfinite(v1.x) && isfinite(v1.y) && isfinite(v1.z) && isfinite(v2.x) && isfinite(v2.y) &&
          isfinite(v2.z)))
        return false;
    const float scale = pow2f(static_cast<int>(t.q));
    unsigned bx, by, bz;
    // quantise_axis rejects NaN and +-inf positions through its range test
    if (!quantise_axis(v0.x, scale, &bx) || !quantise_axis(v0.y, scale, &by) ||
        !quantise_axis(v0.z, scale, &bz))
        return false;
    const unsigned nb = t.use_normal ? dominant_axis_bin(v1.x, v1.y, v1.z) : 0u;
    // omega_o = -d; octahedral map onto [-1, 1]^2
    const float wx = -v2.x, wy = -v2.y, wz = -v2.z;
    const float s = __fadd_rn(__fadd_rn(fabsf(wx), fabsf(wy)), fabsf(wz));
    if (!(s > 0.0f) || isinf(s)) return false;
    float u = __fdiv_rn(wx, s);
    float v = __fdiv_rn(wy, s);
    if (wz < 0.0f) {  // lower hemisphere: fold the triangles outwards, sgn(0) = +1
        const float su = u >= 0.0f ? 1.0f : -1.0f;
        const float sv = v >= 0.0f ? 1.0f : -1.0f;
        const float fu = __fsub_rn(1.0f, fabsf(v));
        const float fv = __fsub_rn(1.0f, fabsf(u));
        u = __fmul_rn(fu, su);
        v = __fmul_rn(fv, sv);
    }
    const float half = pow2f(static_cast<int>(t.d) - 1);
    const int top = (1 << t.d) - 1;
    const unsigned bu = octa_bin(__fadd_rn(u, 1.0f), half, top);
    const unsigned bv = octa_bin(__fadd_rn(v, 1.0f), half, top);
    const unsigned long long dbin = (static_cast<unsigned long long>(bu) << t.d) | bv;
    *key = (static_cast<unsigned long long>(nb) << 58) | (dbin << 48) |
           (static_cast<unsigned long long>(bx) << 32) | (static_cast<unsigned long long>(by) << 16) | bz;
    return true;
}

// The key of the same vertex at hierarchy level l (Section "Progressive hierarchical
// solver"): cells 2^l times wider, so each signed position index is floor-divided by 2^l
// (an arithmetic shift) and the level goes into bits 61-62; the normal and direction bins
// (bits 48-60) are kept.  floor(floor(p 2^q) / 2^l) = floor(p 2^(q-l)).
__device__ __forceinline__ unsigned long long level_key(unsigned long long k0, unsigned l) {
    if (l == 0) return k0;
    auto axis = [l](unsigned long long k, int shift) {
        const int i = static_cast<int>((k >> shift) & 0xFFFFull) - 32768;
        return static_cast<unsigned long long>((i >> l) + 32768) << shift;
    };
    return (static_cast<unsigned long long>(l) << 61) | (k0 & 0x1FFF000000000000ull) | axis(k0, 32) | axis(k0, 16) |
           axis(k0, 0);
}

// The level a vertex at path depth j reads: min(j, levels - 1).  The paper picks the level
// by a path-footprint heuristic it does not spell out; a path's footprint widens with every
// bounce, and this rule takes the depth as that footprint's measure.
__device__ __forceinline__ unsigned read_level(const TableView& t, unsigned j) {
    return j < t.levels - 1u ? j : t.levels - 1u;
}

// Fixed-point contributions of an accepted vertex (eq. 5-6): round(fl32(w L_c) 2^F), round(w 2^F).
// Returns 1 = accepted, 2 = range rule, 3 = zero fixed-point weight.  With kSaturate (the
// progressive values, whose record has passed the range rule already) a product beyond
// +-2^15 is saturated there instead of rejected; a NaN product is still rejected.
template <bool kSaturate = false>
__device__ __forceinline__ int vertex_values(const TableView& t, const float4& v0, const float4& v3,
                                             long long* s, long long* cw) {
    const float w = v0.w;
    if (!(w >= 0.0f && w <= 32768.0f)) return 2;
    float p0 = __fmul_rn(w, v3.x), p1 = __fmul_rn(w, v3.y), p2 = __fmul_rn(w, v3.z);
    if constexpr (kSaturate) {
        if (isnan(p0) || isnan(p1) || isnan(p2)) return 2;
        p0 = fminf(fmaxf(p0, -32768.0f), 32768.0f);
        p1 = fminf(fmaxf(p1, -32768.0f), 32768.0f);
        p2 = fminf(fmaxf(p2, -32768.0f), 32768.0f);
    } else if (!(fabsf(p0) <= 32768.0f && fabsf(p1) <= 32768.0f && fabsf(p2) <= 32768.0f)) {
        return 2;
    }
    const float sc = pow2f(static_cast<int>(t.frac_bits));
    *cw = __float2ll_rn(__fmul_rn(w, sc));
    if (*cw == 0) return 3;
    s[0] = __float2ll_rn(__fmul_rn(p0, sc));
    s[1] = __float2ll_rn(__fmul_rn(p1, sc));
    s[2] = __float2ll_rn(__fmul_rn(p2, sc));
    return 1;
}

// MurmurHash3's 64-bit finaliser (Appleby, public domain): a bijective avalanche mix.
__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__device__ __forceinline__ unsigned long long home_slot(const TableView& t, unsigned long long key) {
    return fmix64(key) >> (64 - t.log2cap);
}

// Find or claim the slot of `key` for every lane with `need` set (linear probing from
// fmix64(key), claim by CAS on kEmpty), the whole warp stepping together: one warp-uniform
// loop whose trip count is the longest probe among the lanes, with no divergent exits to
// reconverge.  Slot indices are 32-bit (capacity <= 2^30).  *slot receives the slot, or -1
// when max_probe slots were visited without success; *len the slots visited.
__device__ __forceinline__ void probe_warp(const TableView& t, bool need, unsigned long long key, long long* slot,
                                           unsigned* len) {
    const unsigned mask = (1u << t.log2cap) - 1u;
    const unsigned long long keep = policy_evict_last();
    unsigned s = static_cast<unsigned>(home_slot(t, key));
    unsigned n = 0;
    long long found = -1;
    while (__any_sync(kFull, need)) {
        if (need) {
            ++n;
            unsigned long long* kp = t.keys + static_cast<unsigned long long>(s) * t.key_stride;
            const unsigned long long k = load_key(kp, keep);
            bool hit = k == key;
            if (!hit && k == kEmpty) {
                const unsigned long long old = atomicCAS(kp, kEmpty, key);
                hit = old == kEmpty || old == key;
            }
            if (hit) {
                found = s;
                need = false;
            } else if (n >= t.max_probe) {
                need = false;
            } else {
                s = (s + 1) & mask;
            }
        }
    }
    *slot = found;
    *len = n;
}

// Per-warp staging of the lanes' sums (32 B per lane): donors' sums for the merge, and each
// leader's merged sums as the source of its bulk reduction.
struct alignas(16) LaneSums {
    long long v[4];
};

// Before a lane rewrites its LaneSums slot: its earlier bulk reductions have read it.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Before the sums are read by other threads (kernel end, grid barrier): this thread's bulk
// reductions have been performed, and they are ordered before its later generic accesses.
__device__ __forceinline__ void bulk_wait_done() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Add the four 64-bit sums at `src` (shared memory) into the first sector of slot `dst` with
// one bulk reduction (cp.reduce.async.bulk .add.u64): each element is added atomically, and
// the L2 takes one 32-byte operation instead of four.  Measured on the B300 (random sectors,
// plus the dirty-bit reduction): 29 vs 21 G groups/s on 256 MB, 24 vs 11 on 1 GB.
__device__ __forceinline__ void bulk_add_sums(Slot* dst, const LaneSums* src) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // src's generic writes first
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(32u)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// A group's head adds the group's sums to its cell's slot (from probe_warp; -1: the
// table is full and the group's vertices are dropped).  Every update is a reduction whose
// result is not read (fire and forget); the touched bit is set unconditionally, so no warp
// waits on an atomic round trip.  `src` is this lane's LaneSums slot (the bulk reduction's
// source).
__device__ __forceinline__ void add_group(const TableView& t, long long slot, unsigned members, const long long sums[4],
                                          LaneSums* src) {
    if (slot < 0) {
        atomicOr(&t.hdr->status, kStatusTableFull);
        atomicAdd(&t.hdr->dropped, static_cast<unsigned long long>(__popc(members)));
        return;
    }
    Slot* a = t.slots + slot;
    if (t.sum_path == kSumsBulk) {
        bulk_wait_read();
        *src = LaneSums{{sums[0], sums[1], sums[2], sums[3]}};
        bulk_add_sums(a, src);
    } else {
        atomicAdd(reinterpret_cast<unsigned long long*>(&a->s[0]), static_cast<unsigned long long>(sums[0]));
        atomicAdd(reinterpret_cast<unsigned long long*>(&a->s[1]), static_cast<unsigned long long>(sums[1]));
        atomicAdd(reinterpret_cast<unsigned long long*>(&a->s[2]), static_cast<unsigned long long>(sums[2]));
        atomicAdd(reinterpret_cast<unsigned long long*>(&a->c), static_cast<unsigned long long>(sums[3]));
    }
    atomicOr(t.dirty + (slot >> 5), 1u << (slot & 31));
}

// Probe for every lane with `head` set (the whole warp calls this), then each head adds
// its group's sums.  Returns the head's slot (-1 for other lanes or a full table).
__device__ __forceinline__ long long scatter_heads(const TableView& t, bool head, unsigned long long key,
                                                   unsigned members, const long long sums[4], unsigned* max_len,
                                                   LaneSums* src) {
    long long slot;
    unsigned len;
    probe_warp(t, head, key, &slot, &len);
    if (head) {
        *max_len = len > *max_len ? len : *max_len;
        add_group(t, slot, members, sums, src);
    }
    return head ? slot : -1;
}

// The slot cache: an insert can note, for each vertex, the slot of the cell its query will
// read (the level min(j, levels - 1) for path depth j), so that the query reads the
// approximant there without hashing or probing.  kNoSlot: the vertex was not added (range
// rule, zero weight, full table); its query probes as usual.
constexpr unsigned kNoSlot = 0xffffffffu;
struct SlotNote {
    unsigned level;  // in: the hierarchy level whose slot to note
    unsigned slot;   // out: that slot, or kNoSlot
};

// The lanes after `lane` that continue its run (the consecutive set bits of `joined` from
// lane + 1 on), which a run's head reports as its members.
__device__ __forceinline__ unsigned heads_after(unsigned joined, unsigned lane) {
    const unsigned rest = lane < 31 ? ~(joined >> (lane + 1)) : 0u;  // first 0 bit = next head
    const unsigned len = lane < 31 ? static_cast<unsigned>(__ffs(rest)) - 1u : 0u;  // rest != 0 (bit 31-lane is 0)
    return len ? (((1u << len) - 1u) << (lane + 1)) : 0u;
}

// One warp's worth of vertices (one per lane, `valid` lanes only): classify, then add each
// accepted vertex to its cell.  With kAggWarp, lanes holding the same key are merged
// (runs of adjacent lanes in a flat table, any lanes with kHier) and one lane per group
// probes once and adds the group's sums; a warp without repeats (the common case after the
// first bounce) skips the merge.  Integer sums are exact, so every mode gives bit-identical
// tables.  With kHier the vertex is added to its cell at every hierarchy level (t.levels of
// them).  A lane's LaneSums slot holds its own sums while a kHier group merges and the sums
// its bulk reduction reads; every write to the slot waits for the lane's earlier bulk
// reductions to have read it.
template <int kMode, bool kHier = false, bool kSlots = false, bool kSaturate = false>
__device__ __forceinline__ void insert_warp(const TableView& t, bool valid, const float4& v0, const float4& v1,
                                            const float4& v2, const float4& v3, unsigned* max_len,
                                            LaneSums* stage, unsigned* leaders, SlotNote* note = nullptr) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long key0 = 0;
    long long own[4] = {0, 0, 0, 0};
    int cls = 0;
    if (valid) {
        if (!cell_key(t, v0, v1, v2, &key0))
            cls = 2;
        else
            cls = vertex_values<kSaturate>(t, v0, v3, own, &own[3]);
    }
    const unsigned accepted = __ballot_sync(kFull, cls == 1);
    const unsigned ranged = __ballot_sync(kFull, cls == 2);
    const unsigned zero_w = __ballot_sync(kFull, cls == 3);
    if (lane == 0 && (ranged | zero_w)) {
        if (ranged) {
            atomicOr(&t.hdr->status, kStatusRange);
            atomicAdd(&t.hdr->dropped, static_cast<unsigned long long>(__popc(ranged)));
        }
        if (zero_w) atomicAdd(&t.hdr->zero_weight, static_cast<unsigned long long>(__popc(zero_w)));
    }
    const unsigned nlevels = kHier ? t.levels : 1u;
    if constexpr (kSlots) note->slot = kNoSlot;
    if (kMode == kAggNone) {
        for (unsigned l = 0; l < nlevels; ++l) {
            const long long hs =
                scatter_heads(t, cls == 1, kHier ? level_key(key0, l) : key0, 1u << lane, own, max_len, stage + lane);
            if constexpr (kSlots)
                if (l == note->level && hs >= 0) note->slot = static_cast<unsigned>(hs);
        }
        *leaders += nlevels * __popc(accepted);
        return;
    }
    for (unsigned l = 0; l < nlevels; ++l) {
        const unsigned long long key = kHier ? level_key(key0, l) : key0;
        long long sums[4] = {own[0], own[1], own[2], own[3]};
        if constexpr (!kHier) {
            // Runs of adjacent lanes on one key (neighbouring pixels in one cell) are merged:
            // a run's first lane (its head) adds the run's sums with a segmented warp
            // reduction (five shuffle steps).  A key that repeats without being adjacent is
            // added once per run, which the integer sums absorb exactly.  (Measured on the
            // B300: 112 vs 120 us for match_any on 1280x720x4.)
            const unsigned long long prev = __shfl_up_sync(kFull, key, 1);
            const bool joins = cls == 1 && lane > 0 && ((accepted >> (lane - 1)) & 1u) && prev == key;
            const unsigned joined = __ballot_sync(kFull, joins);
            if (joined) {
                const unsigned heads = ~joined;  // every lane that does not continue a run starts one
#pragma unroll
                for (unsigned off = 1; off < 32; off <<= 1) {
                    // lane + off is in this lane's run if no run starts in (lane, lane + off]
                    const bool in_run = lane + off < 32 && ((heads >> (lane + 1)) & ((1u << off) - 1u)) == 0;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const long long o = __shfl_down_sync(kFull, sums[c], off);
                        if (in_run) sums[c] += o;
                    }
                }
            }
            const bool head = cls == 1 && !joins;
            const long long hs =
                scatter_heads(t, head, key, (1u << lane) | heads_after(joined, lane), sums, max_len, stage + lane);
            *leaders += __popc(__ballot_sync(kFull, head));
            if constexpr (kSlots) {
                // a lane's head: the last lane at or before it that does not continue a run
                const unsigned upto = lane == 31 ? kFull : ((2u << lane) - 1u);
                const long long s = __shfl_sync(kFull, hs, 31 - __clz(~joined & upto));
                if (cls == 1 && l == note->level && s >= 0) note->slot = static_cast<unsigned>(s);
            }
        } else {
            // Every level: lanes on one key anywhere in the warp are found with match_any (the
            // coarser levels repeat keys across the warp); a group's lowest lane adds the other
            // members' sums, staged in shared memory, then probes once and adds.  (Measured on
            // the B300 with 2 and 3 levels: 205 / 284 us vs 254 / 346 us for adjacent runs.)
            unsigned group = 0;
            if (cls == 1) group = __match_any_sync(accepted, key);
            const bool donor = cls == 1 && (group & ((1u << lane) - 1u)) != 0u;
            if (__any_sync(kFull, donor)) {
                if (donor) {
                    bulk_wait_read();
                    stage[lane] = LaneSums{{own[0], own[1], own[2], own[3]}};
                }
                __syncwarp();
                if (cls == 1 && !donor) {
                    unsigned rest = group & ~(1u << lane);
                    while (rest) {
                        const LaneSums m = stage[__ffs(rest) - 1];
                        rest &= rest - 1u;
                        sums[0] += m.v[0];
                        sums[1] += m.v[1];
                        sums[2] += m.v[2];
                        sums[3] += m.v[3];
                    }
                }
                __syncwarp();
            }
            const long long hs = scatter_heads(t, cls == 1 && !donor, key, group, sums, max_len, stage + lane);
            *leaders += __popc(__ballot_sync(kFull, cls == 1 && !donor));
            if constexpr (kSlots) {
                const long long s = __shfl_sync(kFull, hs, cls == 1 ? __ffs(group) - 1 : static_cast<int>(lane));
                if (cls == 1 && l == note->level && s >= 0) note->slot = static_cast<unsigned>(s);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// YCoCg two-band spherical-harmonics payload (Section "Basis functions and data
// structures: spatio-directional hashing", last paragraph: luminance in two SH bands over
// the normal, chroma per cell).  Per cell and iteration the luminance is fitted over the
// normal by weighted least squares on the two bands (their span is {1, n_x, n_y, n_z}:
// Y(n) ~ a + g . n) with a ridge of `ridge` times the cell's weight on band 1; chroma is
// the weighted mean.  The integer moments make the fit order-free: the centred moments
// W sum(w n n^T) - sum(w n) sum(w n)^T and W sum(w Y n) - sum(w Y) sum(w n) are formed
// exactly in 128-bit integers and rounded once to FP32.  eq. (10)-(11) blend the six
// coefficients.  YCoCg: Y = R/4 + G/2 + B/4, Co = R/2 - B/2, Cg = G/2 - R/4 - B/4.
// ---------------------------------------------------------------------------
constexpr int kShSums = 16;  // Y, Co, Cg, c_new, n(3), Y n(3), n n(xx, xy, xz, yy, yz, zz)

struct alignas(64) SlotSH {
    long long s[kShSums];  // this iteration's fixed-point sums (bytes 0-127: one bulk reduction)
    long long c_old;       // cumulative counter of blended iterations
    long long unused;
    float4 coef_a;         // a, g_x, g_y, g_z: luminance a + g . n
    float2 coef_c;         // Co, Cg
    float pad[6];
};
static_assert(sizeof(SlotSH) == 192, "an SH slot is three 64-byte blocks");

struct alignas(16) ShSums {
    long long v[kShSums];
};

// Fixed-point codes of an accepted vertex for the SH payload, each rounded to nearest even at
// 2^F from an FP32 value taken with one rounding per step in this order: p_c = w L_c,
// wY = (p_r/4 + p_g/2) + p_b/4, wCo = p_r/2 - p_b/2, wCg = (p_g/2 - p_r/4) - p_b/4,
// m_k = w n_k, Yn_k = wY n_k, nn_jk = m_j n_k.  Returns 1 = accepted, 2 = range rule (that of
// the RGB payload, plus |n_k| <= 1 + 2^-10: unit normals), 3 = zero fixed-point weight.
__device__ __forceinline__ int sh_values(const TableView& t, const float4& v0, const float4& v1, const float4& v3,
                                         long long c[kShSums]) {
    const float w = v0.w;
    if (!(w >= 0.0f && w <= 32768.0f)) return 2;
    constexpr float kNormalBound = 1.0009765625f;  // 1 + 2^-10
    if (!(fabsf(v1.x) <= kNormalBound && fabsf(v1.y) <= kNormalBound && fabsf(v1.z) <= kNormalBound)) return 2;
    const float p0 = __fmul_rn(w, v3.x), p1 = __fmul_rn(w, v3.y), p2 = __fmul_rn(w, v3.z);
    if (!(fabsf(p0) <= 32768.0f && fabsf(p1) <= 32768.0f && fabsf(p2) <= 32768.0f)) return 2;
    const float sc = pow2f(static_cast<int>(t.frac_bits));
    const long long cw = __float2ll_rn(__fmul_rn(w, sc));
    if (cw == 0) return 3;
    const float wY = __fadd_rn(__fadd_rn(__fmul_rn(0.25f, p0), __fmul_rn(0.5f, p1)), __fmul_rn(0.25f, p2));
    const float wCo = __fsub_rn(__fmul_rn(0.5f, p0), __fmul_rn(0.5f, p2));
    const float wCg = __fsub_rn(__fsub_rn(__fmul_rn(0.5f, p1), __fmul_rn(0.25f, p0)), __fmul_rn(0.25f, p2));
    const float mx = __fmul_rn(w, v1.x), my = __fmul_rn(w, v1.y), mz = __fmul_rn(w, v1.z);
    auto fx = [sc](float x) { return __float2ll_rn(__fmul_rn(x, sc)); };
    c[0] = fx(wY);
    c[1] = fx(wCo);
    c[2] = fx(wCg);
    c[3] = cw;
    c[4] = fx(mx);
    c[5] = fx(my);
    c[6] = fx(mz);
    c[7] = fx(__fmul_rn(wY, v1.x));
    c[8] = fx(__fmul_rn(wY, v1.y));
    c[9] = fx(__fmul_rn(wY, v1.z));
    c[10] = fx(__fmul_rn(mx, v1.x));
    c[11] = fx(__fmul_rn(mx, v1.y));
    c[12] = fx(__fmul_rn(mx, v1.z));
    c[13] = fx(__fmul_rn(my, v1.y));
    c[14] = fx(__fmul_rn(my, v1.z));
    c[15] = fx(__fmul_rn(mz, v1.z));
    return 1;
}

// One warp's worth of vertices into an SH table (flat tables only): classify, merge runs of
// adjacent lanes on one key (kAggWarp, the segmented shuffle reduction of insert_warp over
// the sixteen sums), then one head per group probes and adds the group's sums to the
// slot's first 128 bytes with one bulk reduction.  Returns the slot of this lane's cell for
// the slot cache (kNoSlot where the vertex was not added).
template <int kMode>
__device__ __forceinline__ unsigned insert_warp_sh(const TableView& t, bool valid, const float4& v0, const float4& v1,
                                                   const float4& v2, const float4& v3, unsigned* max_len, ShSums* stage,
                                                   unsigned* leaders) {
    const unsigned lane = threadIdx.x & 31u;
    unsigned long long key = 0;
    long long own[kShSums];
#pragma unroll
    for (int c = 0; c < kShSums; ++c) own[c] = 0;
    int cls = 0;
    if (valid) {
        if (!cell_key(t, v0, v1, v2, &key))
            cls = 2;
        else
            cls = sh_values(t, v0, v1, v3, own);
    }
    const unsigned accepted = __ballot_sync(kFull, cls == 1);
    const unsigned ranged = __ballot_sync(kFull, cls == 2);
    const unsigned zero_w = __ballot_sync(kFull, cls == 3);
    if (lane == 0 && (ranged | zero_w)) {
        if (ranged) {
            atomicOr(&t.hdr->status, kStatusRange);
            atomicAdd(&t.hdr->dropped, static_cast<unsigned long long>(__popc(ranged)));
        }
        if (zero_w) atomicAdd(&t.hdr->zero_weight, static_cast<unsigned long long>(__popc(zero_w)));
    }
    bool head = cls == 1;
    unsigned members = 1u << lane;
    unsigned joined = 0;
    if (kMode == kAggWarp) {
        const unsigned long long prev = __shfl_up_sync(kFull, key, 1);
        const bool joins = cls == 1 && lane > 0 && ((accepted >> (lane - 1)) & 1u) && prev == key;
        joined = __ballot_sync(kFull, joins);
        if (joined) {
            const unsigned heads = ~joined;
#pragma unroll
            for (unsigned off = 1; off < 32; off <<= 1) {
                const bool in_run = lane + off < 32 && ((heads >> (lane + 1)) & ((1u << off) - 1u)) == 0;
#pragma unroll
                for (int c = 0; c < kShSums; ++c) {
                    const long long o = __shfl_down_sync(kFull, own[c], off);
                    if (in_run) own[c] += o;
                }
            }
        }
        head = cls == 1 && !joins;
        members |= heads_after(joined, lane);
    }
    long long slot;
    unsigned len;
    probe_warp(t, head, key, &slot, &len);
    if (head) {
        *max_len = len > *max_len ? len : *max_len;
        if (slot < 0) {
            atomicOr(&t.hdr->status, kStatusTableFull);
            atomicAdd(&t.hdr->dropped, static_cast<unsigned long long>(__popc(members)));
        } else {
            bulk_wait_read();
            ShSums* src = stage + lane;
#pragma unroll
            for (int c = 0; c < kShSums; c += 2)
                *reinterpret_cast<longlong2*>(&src->v[c]) = make_longlong2(own[c], own[c + 1]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(t.sh + slot),
                         "r"(smem_u32(src)), "r"(128u)
                         : "memory");
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            atomicOr(t.dirty + (slot >> 5), 1u << (slot & 31));
        }
    }
    *leaders += __popc(__ballot_sync(kFull, head));
    // a lane's head: the last lane at or before it that does not continue a run
    const unsigned upto = lane == 31 ? kFull : ((2u << lane) - 1u);
    const long long hs = __shfl_sync(kFull, head ? slot : -1ll, 31 - __clz(~joined & upto));
    return cls == 1 && hs >= 0 ? static_cast<unsigned>(hs) : kNoSlot;
}

// A signed 128-bit integer rounded to the nearest float: the bits below the top 64 are
// folded into a sticky bit, which keeps the single rounding of the 64-bit conversion
// correct, then the exponent is restored exactly.
__device__ __forceinline__ float i128_to_float(__int128 x) {
    const bool neg = x < 0;
    const unsigned __int128 m = neg ? static_cast<unsigned __int128>(0) - static_cast<unsigned __int128>(x)
                                    : static_cast<unsigned __int128>(x);
    const unsigned long long hi = static_cast<unsigned long long>(m >> 64);
    float f;
    if (hi == 0) {
        f = __ull2float_rn(static_cast<unsigned long long>(m));
    } else {
        const int sh = 64 - __clzll(static_cast<long long>(hi));  // 1..64
        const unsigned long long kept = static_cast<unsigned long long>(m >> sh);
        const unsigned long long low = static_cast<unsigned long long>(m);
        const unsigned long long lost = sh == 64 ? low : (low & ((1ull << sh) - 1ull));
        f = ldexpf(__ull2float_rn(kept | (lost != 0ull ? 1ull : 0ull)), sh);
    }
    return neg ? -f : f;
}

// This iteration's SH fit of one touched cell in FP32: out = a, g_x, g_y, g_z, Co, Cg.  The
// regularised normal equations (S + ridge I) g = s, with S and s the centred moments over
// W^2, are solved by a Cholesky factorisation; a pivot that is not positive (the
// regularised matrix is not positive definite) leaves band 1 at 0 for this iteration.
__device__ __forceinline__ void sh_fit(float ridge, const long long S[kShSums], float out[6]) {
    const long long W = S[3];
    const float fW = __ll2float_rn(W);
    const float inv = __fdiv_rn(1.0f, fW);
    auto centred = [W, inv](long long wxy, long long x, long long y) {
        const __int128 m = static_cast<__int128>(W) * wxy - static_cast<__int128>(x) * y;
        return __fmul_rn(__fmul_rn(i128_to_float(m), inv), inv);
    };
    const float a00 = __fadd_rn(centred(S[10], S[4], S[4]), ridge);
    const float a01 = centred(S[11], S[4], S[5]);
    const float a02 = centred(S[12], S[4], S[6]);
    const float a11 = __fadd_rn(centred(S[13], S[5], S[5]), ridge);
    const float a12 = centred(S[14], S[5], S[6]);
    const float a22 = __fadd_rn(centred(S[15], S[6], S[6]), ridge);
    const float r0 = centred(S[7], S[0], S[4]);
    const float r1 = centred(S[8], S[0], S[5]);
    const float r2 = centred(S[9], S[0], S[6]);
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    if (a00 > 0.0f) {
        const float l00 = sqrtf(a00);
        const float l10 = __fdiv_rn(a01, l00), l20 = __fdiv_rn(a02, l00);
        const float d11 = __fsub_rn(a11, __fmul_rn(l10, l10));
        if (d11 > 0.0f) {
            const float l11 = sqrtf(d11);
            const float l21 = __fdiv_rn(__fsub_rn(a12, __fmul_rn(l20, l10)), l11);
            const float d22 = __fsub_rn(__fsub_rn(a22, __fmul_rn(l20, l20)), __fmul_rn(l21, l21));
            if (d22 > 0.0f) {
                const float l22 = sqrtf(d22);
                const float y0 = __fdiv_rn(r0, l00);
                const float y1 = __fdiv_rn(__fsub_rn(r1, __fmul_rn(l10, y0)), l11);
                const float y2 = __fdiv_rn(__fsub_rn(__fsub_rn(r2, __fmul_rn(l20, y0)), __fmul_rn(l21, y1)), l22);
                g2 = __fdiv_rn(y2, l22);
                g1 = __fdiv_rn(__fsub_rn(y1, __fmul_rn(l21, g2)), l11);
                g0 = __fdiv_rn(__fsub_rn(__fsub_rn(y0, __fmul_rn(l10, g1)), __fmul_rn(l20, g2)), l00);
            }
        }
    }
    const float Ym = __fdiv_rn(__ll2float_rn(S[0]), fW);
    const float nx = __fdiv_rn(__ll2float_rn(S[4]), fW), ny = __fdiv_rn(__ll2float_rn(S[5]), fW),
                nz = __fdiv_rn(__ll2float_rn(S[6]), fW);
    out[0] = __fsub_rn(Ym, __fadd_rn(__fadd_rn(__fmul_rn(g0, nx), __fmul_rn(g1, ny)), __fmul_rn(g2, nz)));
    out[1] = g0;
    out[2] = g1;
    out[3] = g2;
    out[4] = __fdiv_rn(__ll2float_rn(S[1]), fW);
    out[5] = __fdiv_rn(__ll2float_rn(S[2]), fW);
}

// eq. (10)-(11) on the six coefficients of one touched SH slot, then its sums are cleared.
__device__ __forceinline__ void blend_sh(const TableView& t, unsigned long long s) {
    SlotSH* p = t.sh + s;
    const longlong2* q = reinterpret_cast<const longlong2*>(p->s);
    long long S[kShSums];
#pragma unroll
    for (int c = 0; c < kShSums; c += 2) {
        const longlong2 x = __ldcg(q + c / 2);
        S[c] = x.x;
        S[c + 1] = x.y;
    }
    const long long co = __ldcg(&p->c_old);
    float4 ca = __ldcg(&p->coef_a);
    float2 cc = __ldcg(&p->coef_c);
    const long long cn = S[3];
    if (cn > 0) {
        const long long ctot = co > (0x7fffffffffffffffll - cn) ? 0x7fffffffffffffffll : co + cn;
        float alpha = t.alpha_min;
        if (t.blend_mode == 0)
            alpha = fmaxf(sqrtf(__fdiv_rn(__ll2float_rn(cn), __ll2float_rn(ctot))), t.alpha_min);
        const float keep = 1.0f - alpha;
        float fit[6];
        sh_fit(t.ridge, S, fit);
        ca.x = fmaf(alpha, fit[0], keep * ca.x);
        ca.y = fmaf(alpha, fit[1], keep * ca.y);
        ca.z = fmaf(alpha, fit[2], keep * ca.z);
        ca.w = fmaf(alpha, fit[3], keep * ca.w);
        cc.x = fmaf(alpha, fit[4], keep * cc.x);
        cc.y = fmaf(alpha, fit[5], keep * cc.y);
        __stcg(&p->c_old, ctot);
        __stcg(&p->coef_a, ca);
        __stcg(&p->coef_c, cc);
    }
    longlong2* w = reinterpret_cast<longlong2*>(p->s);
#pragma unroll
    for (int c = 0; c < kShSums / 2; ++c) __stcg(w + c, make_longlong2(0, 0));
}

// The RGB of SH slot s at normal n: Y = a + g . n, then the YCoCg inverse
// R = Y + Co - Cg, G = Y + Cg, B = Y - Co - Cg.
__device__ __forceinline__ float3 sh_eval(const TableView& t, unsigned long long s, const float4& n) {
    const float4 a = __ldcg(&t.sh[s].coef_a);
    const float2 c = __ldcg(&t.sh[s].coef_c);
    const float Y = __fadd_rn(__fadd_rn(__fadd_rn(a.x, __fmul_rn(a.y, n.x)), __fmul_rn(a.z, n.y)), __fmul_rn(a.w, n.z));
    return make_float3(__fsub_rn(__fadd_rn(Y, c.x), c.y), __fadd_rn(Y, c.y), __fsub_rn(__fsub_rn(Y, c.x), c.y));
}

// ---------------------------------------------------------------------------
// Temporal blend of one touched cell: eq. (10)-(11).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint2 pack_half4(float a, float b, float c) {
    const float lim = 65504.0f;  // largest finite binary16: saturate instead of overflowing to inf
    const __half ha = __float2half_rn(fminf(fmaxf(a, -lim), lim));
    const __half hb = __float2half_rn(fminf(fmaxf(b, -lim), lim));
    const __half hc = __float2half_rn(fminf(fmaxf(c, -lim), lim));
    uint2 r;
    r.x = static_cast<unsigned>(__half_as_ushort(ha)) | (static_cast<unsigned>(__half_as_ushort(hb)) << 16);
    r.y = static_cast<unsigned>(__half_as_ushort(hc));
    return r;
}

struct SlotData {
    longlong2 a01;  // sum_r, sum_g
    longlong2 a23;  // sum_b, c_new
    longlong2 kc;   // key field, c_old
    float4 L;
};

__device__ __forceinline__ SlotData load_slot(const TableView& t, unsigned long long s) {
    const longlong2* p = reinterpret_cast<const longlong2*>(t.slots + s);
    SlotData d;
    d.a01 = __ldcg(p);
    d.a23 = __ldcg(p + 1);
    d.kc = __ldcg(p + 2);
    d.L = __ldcg(reinterpret_cast<const float4*>(p + 3));
    return d;
}

// The blend of one loaded slot, then its stores: every store follows the loads it
// overwrites, so no store waits on an outstanding load of the same bytes.
__device__ __forceinline__ void blend_store(const TableView& t, unsigned long long s, SlotData d) {
    longlong2* p = reinterpret_cast<longlong2*>(t.slots + s);
    const longlong2 z = make_longlong2(0, 0);
    const long long cn = d.a23.y;
    if (cn > 0) {  // always true for a touched slot (accepted vertices add weight >= 1)
        const long long co = d.kc.y;
        const long long ctot = co > (0x7fffffffffffffffll - cn) ? 0x7fffffffffffffffll : co + cn;
        const float fcn = __ll2float_rn(cn);
        float alpha = t.alpha_min;
        if (t.blend_mode == 0) alpha = fmaxf(sqrtf(__fdiv_rn(fcn, __ll2float_rn(ctot))), t.alpha_min);
        const float keep = 1.0f - alpha;
        d.L.x = fmaf(alpha, __fdiv_rn(__ll2float_rn(d.a01.x), fcn), keep * d.L.x);
        d.L.y = fmaf(alpha, __fdiv_rn(__ll2float_rn(d.a01.y), fcn), keep * d.L.y);
        d.L.z = fmaf(alpha, __fdiv_rn(__ll2float_rn(d.a23.x), fcn), keep * d.L.z);
        __stcg(p + 2, make_longlong2(d.kc.x, ctot));  // the key field is written back unchanged
        __stcg(reinterpret_cast<float4*>(p + 3), d.L);
        if (t.mirror) store_mirror(t.mirror + s, pack_half4(d.L.x, d.L.y, d.L.z));
    }
    __stcg(p, z);
    __stcg(p + 1, z);
}

// Position of the n-th (0-based) set bit of w (n < popc(w)).
__device__ __forceinline__ unsigned select_bit(unsigned w, unsigned n) {
    unsigned pos = 0;
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
        const unsigned low = __popc(w & ((1u << sh) - 1u));
        if (n >= low) {
            n -= low;
            w >>= sh;
            pos += sh;
        }
    }
    return pos;
}

// One warp blends every touched slot of dirty words [w0, w0 + 32): the set bits are
// compacted across the warp (prefix sum of popcounts) so all 32 lanes stay busy.
// Returns the number of cells blended (the same value in every lane).
template <bool kSH = false>
__device__ __forceinline__ unsigned update_words(const TableView& t, unsigned long long w0, unsigned long long nwords) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long wi = w0 + lane;
    unsigned word = wi < nwords ? __ldcg(t.dirty + wi) : 0u;
    if (word) t.dirty[wi] = 0u;
    const unsigned cnt = __popc(word);
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned x = __shfl_up_sync(kFull, incl, o);
        if (lane >= static_cast<unsigned>(o)) incl += x;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    const unsigned excl = incl - cnt;
    // one slot per lane per round (measured: with the register count this allows, four
    // blocks per SM beat three blocks holding two slots per lane, 33 vs 36 us)
    for (unsigned r = 0; r < total; r += 32) {
        const unsigned idx = r + lane;
        unsigned owner = 0;  // number of lanes whose inclusive count is <= idx
#pragma unroll
        for (unsigned step = 16; step > 0; step >>= 1) {
            const unsigned v = __shfl_sync(kFull, incl, owner + step - 1);
            if (v <= idx) owner += step;
        }
        owner &= 31u;
        const unsigned ow = __shfl_sync(kFull, word, owner);
        const unsigned oe = __shfl_sync(kFull, excl, owner);
        if (idx < total) {
            const unsigned long long slot = (w0 + owner) * 32ull + select_bit(ow, idx - oe);
            if constexpr (kSH)
                blend_sh(t, slot);
            else
                blend_store(t, slot, load_slot(t, slot));
        }
    }
    return total;
}

// ---------------------------------------------------------------------------
// Control-variate query: Section "Control variates", equation CVEstimator.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 value_at(const TableView& t, unsigned long long s, bool fp32_master = false) {
    if (t.mirror && !fp32_master) {
        const uint2 h = __ldcg(t.mirror + s);
        return make_float3(__half2float(__ushort_as_half(static_cast<unsigned short>(h.x & 0xffffu))),
                           __half2float(__ushort_as_half(static_cast<unsigned short>(h.x >> 16))),
                           __half2float(__ushort_as_half(static_cast<unsigned short>(h.y & 0xffffu))));
    }
    const float4 L = __ldcg(&t.slots[s].L);
    return make_float3(L.x, L.y, L.z);
}

// The approximant of the vertex's cell at hierarchy level `level`, 0 if the cell is
// absent.  The value at the home
// slot is loaded together with its key, so the common case (key found at its home slot)
// costs one round trip instead of two.
__device__ __forceinline__ float3 cell_value(const TableView& t, const float4& v0, const float4& v1,
                                             const float4& v2, bool fp32_master = false, unsigned level = 0) {
    const float3 zero = make_float3(0.0f, 0.0f, 0.0f);
    unsigned long long key;
    if (!cell_key(t, v0, v1, v2, &key)) return zero;
    key = level_key(key, level);
    const unsigned long long mask = (1ull << t.log2cap) - 1ull;
    const unsigned long long keep = policy_evict_last();
    unsigned long long s = home_slot(t, key);
    const unsigned long long k0 = load_key(key_ptr(t, s), keep);
    const float3 c0 = value_at(t, s, fp32_master);
    if (k0 == key) return c0;
    if (k0 == kEmpty) return zero;
    for (unsigned i = 1; i < t.max_probe; ++i) {
        s = (s + 1) & mask;
        const unsigned long long k = load_key(key_ptr(t, s), keep);
        if (k == key) return value_at(t, s, fp32_master);
        if (k == kEmpty) return zero;
    }
    return zero;
}

// The SH payload's approximant of the vertex's cell evaluated at the vertex's own normal (0 if
// the cell is absent); the home slot's coefficients are loaded together with its key.
__device__ __forceinline__ float3 cell_value_sh(const TableView& t, const float4& v0, const float4& v1,
                                                const float4& v2) {
    const float3 zero = make_float3(0.0f, 0.0f, 0.0f);
    unsigned long long key;
    if (!cell_key(t, v0, v1, v2, &key)) return zero;
    const unsigned long long mask = (1ull << t.log2cap) - 1ull;
    const unsigned long long keep = policy_evict_last();
    unsigned long long s = home_slot(t, key);
    const unsigned long long k0 = load_key(key_ptr(t, s), keep);
    const float3 c0 = sh_eval(t, s, v1);
    if (k0 == key) return c0;
    if (k0 == kEmpty) return zero;
    for (unsigned i = 1; i < t.max_probe; ++i) {
        s = (s + 1) & mask;
        const unsigned long long k = load_key(key_ptr(t, s), keep);
        if (k == key) return sh_eval(t, s, v1);
        if (k == kEmpty) return zero;
    }
    return zero;
}

// The estimators that use the approximant are affine in (L_j, t_j C_{j+1}, C_j):
//   control variate (Section "Control variates", CVEstimator):  a = 1, b = c = beta
//   biased predictor-corrector (Section "Biased estimation"):    a = b = gamma, c = 1
// applied to vertices j_begin <= j < j_end that have a successor; other vertices keep L_j.
struct Estimator {
    float a, b, c;
    unsigned j_begin, j_end;
};

__host__ __device__ __forceinline__ Estimator cv_estimator(const TableView& t) {
    return Estimator{1.0f, t.beta, t.beta, 0u, t.cv_max_depth};
}

// out_j = a L_j - b (t_j C_{j+1}) + c C_j
__device__ __forceinline__ float combine(const Estimator& e, float L, float tj, float c_next, float c_self) {
    const float h = __fmul_rn(tj, c_next);
    return __fadd_rn(__fsub_rn(__fmul_rn(e.a, L), __fmul_rn(e.b, h)), __fmul_rn(e.c, c_self));
}

// All vertices of path p (depth-major records j*P + p), last to first so that each vertex
// is probed once: its cell value serves as C_j here and as C_{j+1} for vertex j - 1.  With
// kSlots a vertex whose slot the insert noted reads the approximant there directly.
template <bool kSlots = false, bool kSH = false>
__device__ __forceinline__ void query_path(const TableView& t, const Estimator& e, const float4* __restrict__ v,
                                           unsigned P, unsigned D, unsigned long long p, float* __restrict__ out,
                                           const unsigned* __restrict__ slots = nullptr) {
    float3 c_next = make_float3(0.0f, 0.0f, 0.0f);
    for (int j = static_cast<int>(D) - 1; j >= 0; --j) {
        const unsigned long long i = static_cast<unsigned long long>(j) * P + p;
        const float4* r = v + 4 * i;  // streamed once: evict-first
        const float4 v0 = __ldcs(r), v1 = __ldcs(r + 1), v2 = __ldcs(r + 2), v3 = __ldcs(r + 3);
        float3 c;
        if constexpr (kSH) {
            if constexpr (kSlots) {
                const unsigned sl = __ldcs(slots + i);
                c = sl != kNoSlot ? sh_eval(t, sl, v1) : cell_value_sh(t, v0, v1, v2);
            } else {
                c = cell_value_sh(t, v0, v1, v2);
            }
        } else if constexpr (kSlots) {
            const unsigned sl = __ldcs(slots + i);
            c = sl != kNoSlot ? value_at(t, sl) : cell_value(t, v0, v1, v2, false, read_level(t, static_cast<unsigned>(j)));
        } else {
            c = cell_value(t, v0, v1, v2, false, read_level(t, static_cast<unsigned>(j)));
        }
        float o0 = v3.x, o1 = v3.y, o2 = v3.z;
        if (j + 1 < static_cast<int>(D) && static_cast<unsigned>(j) >= e.j_begin && static_cast<unsigned>(j) < e.j_end) {
            o0 = combine(e, v3.x, v1.w, c_next.x, c.x);
            o1 = combine(e, v3.y, v2.w, c_next.y, c.y);
            o2 = combine(e, v3.z, v3.w, c_next.z, c.z);
        }
        float* o = out + 3 * i;
        o[0] = o0;
        o[1] = o1;
        o[2] = o2;
        c_next = c;
    }
}

// The query split by depth: a warp takes tile `tile` of T = 32 / D paths at all D depths, one
// lane per vertex (lane k: depth k / T, path tile * T + k % T), so every vertex's record, slot
// and approximant loads are in flight at once instead of one dependent chain per path.  Lane
// k receives C_{j+1} of its path from lane k + T with one shuffle.  The whole warp calls it;
// requires 1 <= D <= 32.  With kSlots a vertex whose slot the insert noted reads the
// approximant there; kSH reads the SH payload's fit at the vertex's normal.
__host__ __device__ __forceinline__ unsigned long long query_tiles(unsigned P, unsigned D) {
    const unsigned T = 32u / D;
    return (static_cast<unsigned long long>(P) + T - 1) / T;
}

template <bool kSlots, bool kSH = false>
__device__ __forceinline__ void query_tile(const TableView& t, const Estimator& e, const float4* __restrict__ v,
                                           unsigned P, unsigned D, unsigned long long tile, float* __restrict__ out,
                                           const unsigned* __restrict__ slots) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned T = 32u / D;
    const unsigned j = lane / T, q = lane - j * T;
    const unsigned long long p = tile * T + q;
    const bool act = j < D && p < P;
    float3 c = make_float3(0.0f, 0.0f, 0.0f);
    float4 v1 = make_float4(0, 0, 0, 0), v2 = v1, v3 = v1;
    unsigned long long i = 0;
    if (act) {
        i = static_cast<unsigned long long>(j) * P + p;
        const float4* r = v + 4 * i;  // streamed once: evict-first
        if constexpr (kSlots) {
            const unsigned sl = __ldcs(slots + i);
            v1 = __ldcs(r + 1);
            v2 = __ldcs(r + 2);
            v3 = __ldcs(r + 3);
            c = sl != kNoSlot ? value_at(t, sl) : cell_value(t, __ldcs(r), v1, v2, false, read_level(t, j));
        } else {
            const float4 v0 = __ldcs(r);
            v1 = __ldcs(r + 1);
            v2 = __ldcs(r + 2);
            v3 = __ldcs(r + 3);
            if constexpr (kSH)
                c = cell_value_sh(t, v0, v1, v2);
            else
                c = cell_value(t, v0, v1, v2, false, read_level(t, j));
        }
    }
    // vertex j + 1 of the same path is lane + T (a lane past the warp reads its own value, which
    // no active lane uses)
    const unsigned src = lane + T < 32u ? lane + T : lane;
    const float n0 = __shfl_sync(kFull, c.x, src);
    const float n1 = __shfl_sync(kFull, c.y, src);
    const float n2 = __shfl_sync(kFull, c.z, src);
    if (act) {
        float o0 = v3.x, o1 = v3.y, o2 = v3.z;
        if (j + 1 < D && j >= e.j_begin && j < e.j_end) {
            o0 = combine(e, v3.x, v1.w, n0, c.x);
            o1 = combine(e, v3.y, v2.w, n1, c.y);
            o2 = combine(e, v3.z, v3.w, n2, c.z);
        }
        float* o = out + 3 * i;
        o[0] = o0;
        o[1] = o1;
        o[2] = o2;
    }
}

}  // namespace psf
