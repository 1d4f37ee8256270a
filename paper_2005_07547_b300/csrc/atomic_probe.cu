// atomic_probe.cu -- L2 64-bit atomic throughput microbenchmark.
//
// Measurement only, not part of the filtering path: it gives the rate the insert
// kernel's atomics are compared against (its "atomic roofline").  Each group of work
// picks a pseudo-random target (SplitMix64 finaliser of the group index, Steele et
// al., OOPSLA 2014) and issues:
//   mode 0: one 64-bit reduction (red.add, result unused) to a random word
//   mode 1: one 64-bit atomic add whose result is used (atom.add)
//   mode 2: four 64-bit reductions into one random 32-byte sector plus one 32-bit
//           reduction (red.or) into a bitmap word -- the insert's per-key pattern
//   mode 3: one 64-bit reduction per lane with all 32 lanes of a warp on one word
//   mode 4: mode 2's pattern with the four 64-bit additions issued as ONE bulk
//           reduction of 32 bytes from shared memory (cp.reduce.async.bulk .add.u64,
//           the TMA path), each thread cycling two 32-byte source slots
//   mode 5: mode 4 without the bitmap reduction
// With n_distinct > 0 the targets of modes 2, 4 and 5 are drawn from a fixed set of
// n_distinct pseudo-random sectors (the footprint of an insert that touches n_distinct
// cells of a larger table); 0 spreads them over every sector of the buffer.
// The caller times the launch; ops = groups (modes 0, 1, 3) or 5 x groups (modes 2, 4, 5).

#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void bulk_reduce_add_u64(unsigned long long* dst, const void* src, unsigned bytes) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(src));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], %2;" ::"l"(dst), "r"(s),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

template <int kMode>
__global__ void __launch_bounds__(256) k_probe(unsigned long long* words, unsigned long long n_words,
                                               unsigned long long n_groups, unsigned long long n_distinct,
                                               unsigned long long* sink) {
    __shared__ alignas(128) unsigned long long s_src[kMode >= 4 ? 256 * 2 * 4 : 1];
    const unsigned long long stride = static_cast<unsigned long long>(gridDim.x) * blockDim.x;
    unsigned long long acc = 0;
    unsigned k = 0;
    for (unsigned long long g = static_cast<unsigned long long>(blockIdx.x) * blockDim.x + threadIdx.x; g < n_groups;
         g += stride) {
        const unsigned long long h = mix(g);
        if (kMode == 0) {
            atomicAdd(words + h % n_words, 1ull);
        } else if (kMode == 1) {
            acc += atomicAdd(words + h % n_words, 1ull);
        } else if (kMode == 2) {
            const unsigned long long sector = n_distinct ? mix(h % n_distinct + 0x5bd1e995ull) % (n_words / 4) : h % (n_words / 4);
            unsigned long long* w = words + 4 * sector;
            atomicAdd(w, 1ull);
            atomicAdd(w + 1, 2ull);
            atomicAdd(w + 2, 3ull);
            atomicAdd(w + 3, 4ull);
            unsigned* bitmap = reinterpret_cast<unsigned*>(words + n_words) ;
            atomicOr(bitmap + (sector >> 5), 1u << (sector & 31));
        } else if (kMode == 4 || kMode == 5) {
            const unsigned long long sector = n_distinct ? mix(h % n_distinct + 0x5bd1e995ull) % (n_words / 4) : h % (n_words / 4);
            unsigned long long* src = s_src + (threadIdx.x * 2 + (k & 1u)) * 4;
            // the slot written now was last read by the bulk copy issued two groups ago
            asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            src[0] = 1ull;
            src[1] = 2ull;
            src[2] = 3ull;
            src[3] = 4ull;
            bulk_reduce_add_u64(words + 4 * sector, src, 32u);
            if (kMode == 4) {
                unsigned* bitmap = reinterpret_cast<unsigned*>(words + n_words);
                atomicOr(bitmap + (sector >> 5), 1u << (sector & 31));
            }
            ++k;
        } else {
            atomicAdd(words + mix(g >> 5) % n_words, 1ull);
        }
    }
    if (kMode >= 4) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (kMode == 1 && acc == 0xffffffffffffffffull) *sink = acc;  // keep the results live
}

}  // namespace

extern "C" {

// words: n_words 64-bit words (a multiple of 4), followed (modes 2, 4) by n_words / 128
// 32-bit bitmap words.  Returns 0, or -1 for bad arguments, -3 for a CUDA error.
int atomic_probe(unsigned long long* words, unsigned long long n_words, unsigned long long n_groups,
                 unsigned long long n_distinct, int mode, int blocks, void* stream) {
    if (!words || n_words < 128 || (n_words & 3u) || mode < 0 || mode > 5 || blocks < 1 ||
        (reinterpret_cast<uintptr_t>(words) & 31u))
        return -1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long* sink = words;
    switch (mode) {
        case 0: k_probe<0><<<blocks, 256, 0, st>>>(words, n_words, n_groups, n_distinct, sink); break;
        case 1: k_probe<1><<<blocks, 256, 0, st>>>(words, n_words, n_groups, n_distinct, sink); break;
        case 2: k_probe<2><<<blocks, 256, 0, st>>>(words, n_words, n_groups, n_distinct, sink); break;
        case 4: k_probe<4><<<blocks, 256, 0, st>>>(words, n_words, n_groups, n_distinct, sink); break;
        case 5: k_probe<5><<<blocks, 256, 0, st>>>(words, n_words, n_groups, n_distinct, sink); break;
        default: k_probe<3><<<blocks, 256, 0, st>>>(words, n_words, n_groups, n_distinct, sink); break;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
