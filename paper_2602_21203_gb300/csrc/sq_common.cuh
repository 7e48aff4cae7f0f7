// Shared device helpers of the Squint CUDA library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <utility>

// Programmatic dependent launch: every kernel first waits until the grids it depends on
// have finished and their writes are visible, then lets its own dependent grid be
// scheduled, so a dependent kernel's launch overlaps this one's execution.
#define SQ_KERNEL_ENTRY()                                              \
    do {                                                               \
        asm volatile("griddepcontrol.wait;" ::: "memory");             \
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); \
    } while (0)

namespace sq {

// The scheduling priority of a launch: its stream's (kept by graph kernel nodes, so a
// graph instantiated to use node priorities schedules each branch's blocks as its
// stream would).
inline int stream_priority(cudaStream_t s) {
    int p = 0;
    if (cudaStreamGetPriority(s, &p) != cudaSuccess) p = 0;
    return p;
}

// Launch with programmatic stream serialization allowed (inside graphs: a programmatic edge).
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributePriority;
    at[1].val.priority = stream_priority(s);
    cfg.attrs = at;
    cfg.numAttrs = 2;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// The same with a 1-D thread-block cluster of cluster.x CTAs (cluster.x == 1: no cluster attribute).
template <typename... KArgs, typename... Args>
inline void launch_kc(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, dim3 cluster,
                      Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[3];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributePriority;
    at[1].val.priority = stream_priority(s);
    at[2].id = cudaLaunchAttributeClusterDimension;
    at[2].val.clusterDim.x = cluster.x;
    at[2].val.clusterDim.y = 1;
    at[2].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = cluster.x > 1 ? 3 : 2;
    cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Philox4x32-10 (Salmon et al., SC'11, Sec. 3.2): ten rounds of two 32x32->64
// multiplies; the high halves are xored with the other counter words and the
// round key; the key is bumped by the Weyl constants between rounds.
__host__ __device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        c[1] = (uint32_t)p1;
        c[3] = (uint32_t)p0;
        c[0] = n0;
        c[2] = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Draw addressing shared by every random quantity of the learner:
// counter (element, stream | sub << 16, word_lo, word_hi), key (seed_lo, seed_hi).
__host__ __device__ __forceinline__ void draw_block(uint32_t out[4], uint64_t seed, uint32_t element,
                                                    uint32_t stream, uint32_t sub, uint64_t word) {
    out[0] = element;
    out[1] = (stream & 0xFFFFu) | (sub << 16);
    out[2] = (uint32_t)word;
    out[3] = (uint32_t)(word >> 32);
    philox4x32_10(out, (uint32_t)seed, (uint32_t)(seed >> 32));
}

enum Stream : uint32_t {
    kStreamIndex = 1,
    kStreamShiftT = 2,
    kStreamShiftT1 = 3,
    kStreamEpsTarget = 4,
    kStreamEpsActor = 5,
    kStreamInit = 16,
    kStreamAct = 32,
};

// floor(w * n / 2^32): integer in [0, n).
__host__ __device__ __forceinline__ uint32_t range_draw(uint32_t w, uint32_t n) {
    return (uint32_t)(((uint64_t)w * n) >> 32);
}

// Uniform in (0, 1) from the top 23 bits: exact in FP32.
__device__ __forceinline__ float uniform01f(uint32_t w) {
    return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-07f;  // 2^-23
}

// Standard normal pair by Box-Muller from two words.
__device__ __forceinline__ void box_muller(uint32_t w0, uint32_t w1, float& z0, float& z1) {
    const float u1 = uniform01f(w0);
    const float u2 = uniform01f(w1);
    const float rad = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    z0 = rad * c;
    z1 = rad * s;
}

// Normal noise eps[k] (k < dim) of row `element` of a stream addressed by `word`.
__device__ __forceinline__ float normal_draw(uint64_t seed, uint32_t element, uint32_t stream, uint64_t word, int k) {
    uint32_t w[4];
    draw_block(w, seed, element, stream, (uint32_t)(k >> 1), word);
    float z0, z1;
    box_muller(w[0], w[1], z0, z1);
    return (k & 1) ? z1 : z0;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One-shot bulk copy global -> shared through the TMA engine, completing on an mbarrier
// (addresses 16-byte aligned, size a multiple of 16 and below 1 MiB).
__device__ __forceinline__ void bulk_load_init(uint64_t* bar) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// The same copy with an evict-first L2 policy: for data read once (replay-ring frames),
// so that it does not displace the weights and activations the update keeps reusing.
__device__ __forceinline__ void bulk_load_stream(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    uint64_t policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            d),
        "l"(src), "r"(bytes), "r"(b), "l"(policy)
        : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}
// Wait for phase `parity` of the barrier, giving up after ~1 s of clock (returns false).
__device__ __forceinline__ bool bulk_load_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(b), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 2000000000ll) return false;
        __nanosleep(64);   // leave the issue slots to resident warps with work
    }
}

template <typename T> __device__ __forceinline__ T ld(const T* p) { return *p; }

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ double to_f(double x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

}  // namespace sq
