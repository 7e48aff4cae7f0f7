// Fused LayerNorm-MLP forward on tcgen05 (sm_103a).
//
// The critic and actor heads (Sec. IV "Normalization": Linear -> LayerNorm -> ReLU for
// every hidden layer, a plain Linear output layer) run as one launch per chain instead
// of one GEMM and one LayerNorm launch per layer.  A block of 128 rows stays on chip
// from the head input to the output:
//
//   cluster of CL CTAs per row block; CTA q computes columns [q NS, (q + 1) NS) of every
//   hidden layer (NS = H / CL), so each SM streams 1 / CL of the weights
//   warp 4 / lane 0   TMA producer: the block's input rows into the activation region
//                     (128-byte swizzled 64-wide K slabs), then every layer's weight
//                     slabs through a shared-memory ring (mbarrier complete_tx)
//   warp 0 / lane 0   MMA issuer: tcgen05.mma M = 128, N = NS (K = 16 per step) from
//                     the activation region and the ring into tensor memory
//   warps 0-3         epilogue, one thread per row: bias, LayerNorm statistics over the
//                     whole row (each CTA's mean and centred sum of squares of its slice,
//                     sent to every CTA of the cluster with st.async and combined in rank
//                     order), ReLU; the BF16 result is written into this CTA's activation
//                     region as the next layer's A operand and copied to the other CTAs of
//                     the cluster with one shared-to-shared bulk copy each; saved FP32
//                     activations leave through a per-warp transpose as coalesced rows,
//                     the BF16 copy by a TMA store of the CTA's own slabs
//   output layer      K split over the cluster (each CTA multiplies its own column slice
//                     of the last hidden layer); the partial tile is staged in the idle
//                     weight ring, each band of rows bulk-copied to the CTA that finishes
//                     it, and the partials added in rank order
//
// Data that crosses CTAs travels by st.async and bulk copies that complete transaction
// bytes on the receiver's mbarrier, so no cluster-scope fence or cluster-wide barrier is
// needed between the layers, and the producer streams ahead undisturbed.
// Every wait is bounded; past the limit the waiting thread records a code in *err and
// gives up, the CTA waits (bounded) for its copies in flight, frees its tensor memory and
// returns.
#include "sq_mlp_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace sq {

namespace {

constexpr int BM = 128;
constexpr int SLAB = 64;                  // K elements per slab (128 bytes of BF16)
constexpr int SLAB_BYTES = BM * 128;      // one activation slab: 128 rows x 128 B
constexpr int kThreads = 160;
constexpr int STG_LD = 36;                // staging row stride (floats)
constexpr int STG_BYTES = 4 * 32 * STG_LD * 4;
constexpr int SMEM_LIMIT = 232448;
constexpr long long kWaitDefault = 4000000000ll;   // ~2 s at 2 GHz

struct MlpProbDev {
    CUtensorMap tx;                           // X [M, kin], box 64 x 128
    CUtensorMap tw[kMlpMaxHidden + 1];        // hidden W_l, box 64 x NS; output W, box 64 x nop
    CUtensorMap tph[kMlpMaxHidden];           // BF16 saved output of hidden layer l, box 64 x 128 (store)
    const float* bias[kMlpMaxHidden + 1];
    const float* g[kMlpMaxHidden];
    const float* beta[kMlpMaxHidden];
    float* pre[kMlpMaxHidden];
    float* post[kMlpMaxHidden];
    float* mean[kMlpMaxHidden];
    float* rstd[kMlpMaxHidden];
    int has_ph[kMlpMaxHidden];
    float* out; int64_t ldo;
    int M, nk0, cta0;
};
struct MlpArgs {
    MlpProbDev p[kMlpMaxProbs];
    int n_probs, nh, H, CL, NS, nout, nop;
    int stages, stage_bytes, a_bytes, par_floats;
    int ldr;          // row stride (floats) of the output tile staging: nop, padded when it fits
    uint32_t tmem_cols;
    float eps;
    int* err;
    long long wait_limit;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive_local(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    if (CLUSTER)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    return ok != 0;
}
// Bounded wait: false (and *err = code) if the phase did not complete within `limit` cycles.
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, long long limit) {
    if (mbar_try_wait<CLUSTER>(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait<CLUSTER>(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"((uint64_t)map),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// The shared::cluster address of `addr` (this CTA's shared memory) in CTA `rank`.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// Two floats into shared memory of a cluster CTA, completing 8 bytes of transaction count
// on the barrier `bar` (a shared::cluster address in that CTA).
__device__ __forceinline__ void st_async_v2(uint32_t addr, float x, float y, uint32_t bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "f"(x), "f"(y), "r"(bar)
                 : "memory");
}
// Bulk copy of `bytes` (a multiple of 16) from this CTA's shared memory to a cluster CTA's,
// completing that many bytes of transaction count on its barrier.
__device__ __forceinline__ void bulk_s2s(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst),
                 "r"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16_kk(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}
// 32 consecutive floats of shared memory (16-byte aligned, the same for every thread).
__device__ __forceinline__ void ld_par32(const float* p, float (&v)[32]) {
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(p + j);
        v[j] = x.x; v[j + 1] = x.y; v[j + 2] = x.z; v[j + 3] = x.w;
    }
}
// The first n (<= 4, or none if n <= 0) of four consecutive outputs.
__device__ __forceinline__ void store_out4(float* dst, float4 v, int n) {
    if (n > 0) dst[0] = v.x;
    if (n > 1) dst[1] = v.y;
    if (n > 2) dst[2] = v.z;
    if (n > 3) dst[3] = v.w;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// 32 values of row `lr` (this warp's rows 0..31) at columns [col, col + 32) of dst:
// transposed through the warp's staging tile so that each store instruction writes four
// whole 128-byte row segments.
__device__ __forceinline__ void store_rows_coalesced(float* stg, const float (&v)[32], float* dst, int64_t ld,
                                                     int row0, int M, int col, int lane) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(stg + lane * STG_LD + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int rr = 4 * i + lane / 8;
        const float4 x = *reinterpret_cast<const float4*>(stg + rr * STG_LD + 4 * (lane % 8));
        if (row0 + rr < M) *reinterpret_cast<float4*>(dst + (int64_t)(row0 + rr) * ld + col + 4 * (lane % 8)) = x;
    }
}

__global__ void __launch_bounds__(kThreads, 1) mlp_tc_kernel(const __grid_constant__ MlpArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    const int CL = a.CL, NS = a.NS, H = a.H, nh = a.nh;
    const uint32_t a_base = smem_u32(smem);
    const uint32_t ring = a_base + a.a_bytes;
    float* ring_f = reinterpret_cast<float*>(smem + a.a_bytes);
    float* stg = reinterpret_cast<float*>(smem + a.a_bytes + S * a.stage_bytes);
    float* xbuf = stg + 4 * 32 * STG_LD;                                 // [2][CL][BM][2]: (mean, M2) of each CTA
    float* par = xbuf + 2 * CL * BM * 2;                                 // bias, g, beta slices; output bias
    uint64_t* bars = reinterpret_cast<uint64_t*>(par + a.par_floats);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);     // tmem address, issued, consumed
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8 * s; };
    auto empty = [&](int s) { return bar0 + 8 * (S + s); };
    const uint32_t x_full = bar0 + 8 * (2 * S), acc_full = x_full + 8, a_ready = x_full + 16;
    const uint32_t xbar0 = x_full + 24, out_bar = x_full + 40;

    int pi = 0;
    while (pi + 1 < a.n_probs && (int)blockIdx.x >= a.p[pi + 1].cta0) ++pi;
    const MlpProbDev& P = a.p[pi];
    const int rank = CL > 1 ? (int)cluster_rank() : 0;
    const int m0 = ((int)blockIdx.x - P.cta0) / CL * BM;
    const int M = P.M;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long wlim = a.wait_limit;
    int* err = a.err;
    const int hslabs = (H + SLAB - 1) / SLAB;
    const int nop = a.nop, ldr = a.ldr;             // row stride of the output staging (floats)
    const int band = BM / CL;                       // rows of the output each CTA finishes
    auto nk = [&](int l) { return l == 0 ? P.nk0 : (l < nh ? hslabs : (CL > 1 ? NS / SLAB : hslabs)); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(x_full, 1);
        mbar_init(acc_full, 1);
        mbar_init(a_ready, 1);
        mbar_init(xbar0, 1);
        mbar_init(xbar0 + 8, 1);
        mbar_init(out_bar, 1);
        slot[1] = 0;
        slot[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (CL > 1) {
            // the bytes the cluster's CTAs send this one: row statistics (each exchange) and
            // the output partials of its band of rows
            mbar_expect_tx(xbar0, (uint32_t)(CL * BM * 8));
            mbar_expect_tx(xbar0 + 8, (uint32_t)(CL * BM * 8));
            mbar_expect_tx(out_bar, (uint32_t)(CL * band * ldr * 4));
        }
    }
    if (threadIdx.x == 128) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.tx)) : "memory");
        for (int l = 0; l <= nh; ++l)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.tw[l])) : "memory");
    }
    __syncthreads();
    // every CTA of the cluster has started and initialised its barriers before any remote access
    if (CL > 1) cluster_sync_all();
    // inputs are read, and tensor memory taken, only once the previous kernel has finished
    SQ_KERNEL_ENTRY();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = slot[0];

    if (warp == 4) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            mbar_expect_tx(x_full, (uint32_t)(P.nk0 * SLAB_BYTES));
            for (int kb = 0; kb < P.nk0; ++kb) tma_load_2d(a_base + kb * SLAB_BYTES, &P.tx, kb * SLAB, m0, x_full);
            int it = 0;
            bool ok = true;
            for (int l = 0; l <= nh && ok; ++l) {
                const bool last = l == nh;
                const uint32_t bytes = (uint32_t)((last ? nop : NS) * 128);
                const int row0 = last ? 0 : rank * NS;
                const int kcol0 = (last && CL > 1) ? rank * NS : 0;
                for (int kb = 0; kb < nk(l); ++kb, ++it) {
                    const int s = it % S;
                    if (it >= S && !mbar_wait(empty(s), ((it / S) - 1) & 1, err, 30, wlim)) { ok = false; break; }
                    mbar_expect_tx(full(s), bytes);
                    tma_load_2d(ring + s * a.stage_bytes, &P.tw[l], kcol0 + kb * SLAB, row0, full(s));
                }
            }
            slot[1] = it;
        }
    } else {
        const int r = warp * 32 + lane;                 // row of the block = tensor-memory lane
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        // this CTA's slices of the bias, LayerNorm gain and shift of every hidden layer, and
        // the output bias, staged by warps 1-3 while the first layer's operands arrive (the
        // first epilogue's barrier orders them before any use)
        if (warp > 0) {
            for (int i = threadIdx.x - 32; i < nh * 3 * NS; i += 96) {
                const int l = i / (3 * NS), k = (i % (3 * NS)) / NS, j = i % NS;
                const float* src = k == 0 ? P.bias[l] : (k == 1 ? P.g[l] : P.beta[l]);
                par[i] = src[rank * NS + j];
            }
            for (int j = threadIdx.x - 32; j < nop; j += 96) par[nh * 3 * NS + j] = j < a.nout ? P.bias[nh][j] : 0.f;
        }
        // the problem's output pointers, read once: P is reached through a generic pointer
        // into the parameter block, which the compiler would re-read after every store
        float* const p_out = P.out;
        const int64_t p_ldo = P.ldo;
        float* stg_w = stg + warp * 32 * STG_LD;
        int it = 0;                                      // weight slab sequence (issuer)
        bool dead = false;                               // the issuer gave up on a wait
        for (int l = 0; l <= nh; ++l) {
            const bool last = l == nh;
            // ---------------------------------------------------------------- MMA issue
            if (threadIdx.x == 0) {
                if (!dead) {
                    if (l == 0) dead = !mbar_wait(x_full, 0, err, 31, wlim);
                    else dead = !mbar_wait<true>(a_ready, (l - 1) & 1, err, 32, wlim);
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = idesc_bf16_kk(BM, last ? nop : NS);
                const int nkl = nk(l);
                for (int kb = 0; kb < nkl && !dead; ++kb) {
                    const int s = it % S;
                    if (!mbar_wait(full(s), (it / S) & 1, err, 33, wlim)) { dead = true; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t as = a_base + kb * SLAB_BYTES, bs = ring + s * a.stage_bytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(tmem, sw128_desc(as + kk * 32), sw128_desc(bs + kk * 32), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(empty(s));
                    ++it;
                }
                slot[2] = it;
                mma_commit(acc_full);
            }
            __syncwarp();
            mbar_wait(acc_full, l & 1, err, 34, wlim);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (l == 0) epi_bar();   // the staged parameter slices
            if (!last) {
                // ------------------------------------------------------------ hidden layer epilogue
                const int c0 = rank * NS;                 // this CTA's first column
                const float* pb = par + l * 3 * NS;       // bias, gain, shift of the slice
                const float* pg = pb + NS;
                const float* pbeta = pb + 2 * NS;
                float* const s_pre = P.pre[l];
                float* const s_post = P.post[l];
                float* const s_mean = P.mean[l];
                float* const s_rstd = P.rstd[l];
                const bool s_ph = P.has_ph[l] != 0;
                // statistics of this CTA's NS columns of the row: mean, then centred squares
                float s1 = 0.f;
                for (int c = 0; c < NS; c += 32) {
                    float v[32], b[32];
                    tmem_ld32(trow + c, v);
                    ld_par32(pb + c, b);
#pragma unroll
                    for (int j = 0; j < 32; ++j) s1 += v[j] + b[j];
                }
                const float mq = s1 / (float)NS;
                float m2 = 0.f;
                for (int c = 0; c < NS; c += 32) {
                    float v[32], b[32];
                    tmem_ld32(trow + c, v);
                    ld_par32(pb + c, b);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float d = v[j] + b[j] - mq;
                        m2 += d * d;
                    }
                }
                // the whole row's statistics: every CTA sends (mean, M2) of its slice to every
                // CTA of the cluster; they are combined in rank order (Chan et al.'s pairwise
                // update for equal counts: M2 = sum M2_q + NS sum (mean_q - mean)^2)
                float mean = mq, var = m2 / (float)H;
                if (CL > 1) {
                    const int b = l & 1;
                    float* buf = xbuf + b * CL * BM * 2;
                    const uint32_t mine = smem_u32(buf + (rank * BM + r) * 2), xb = xbar0 + 8 * b;
                    for (int q = 0; q < CL; ++q) st_async_v2(mapa(mine, q), mq, m2, mapa(xb, q));
                    mbar_wait<true>(xb, (l >> 1) & 1, err, 35, wlim);
                    // armed again for its next use (every CTA's sends of that use follow this
                    // CTA's sends of the next exchange, which follow all of its reads here)
                    if (threadIdx.x == 0) mbar_expect_tx(xb, (uint32_t)(CL * BM * 8));
                    float ms = 0.f;
                    for (int q = 0; q < CL; ++q) ms += buf[(q * BM + r) * 2];
                    mean = ms / (float)CL;
                    float M2 = 0.f;
                    for (int q = 0; q < CL; ++q) {
                        const float d = buf[(q * BM + r) * 2] - mean;
                        M2 += buf[(q * BM + r) * 2 + 1] + (float)NS * d * d;
                    }
                    var = M2 / (float)H;
                }
                const float rstd = 1.0f / sqrtf(var + a.eps);
                // the previous layer's TMA store has read this CTA's slabs before they are rewritten
                if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                epi_bar();
                // the last hidden layer feeds only this CTA's K slice of the output layer:
                // kept locally, at the start of the activation region
                const bool bcast = CL > 1 && l + 1 < nh;
                const int kpos0 = (CL > 1 && l + 1 == nh) ? 0 : c0;
                for (int c = 0; c < NS; c += 32) {
                    float v[32], y[32];
                    tmem_ld32(trow + c, v);
                    ld_par32(pb + c, y);
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] += y[j];
                    ld_par32(pg + c, y);
                    {   // g xhat + beta rounded once: the backward rebuilds the ReLU mask the same way
                        float bt[32];
                        ld_par32(pbeta + c, bt);
#pragma unroll
                        for (int j = 0; j < 32; ++j) y[j] = fmaxf(__fmaf_rn(y[j], (v[j] - mean) * rstd, bt[j]), 0.f);
                    }
                    if (s_pre) store_rows_coalesced(stg_w, v, s_pre, H, m0 + warp * 32, M, c0 + c, lane);
                    if (s_post) store_rows_coalesced(stg_w, y, s_post, H, m0 + warp * 32, M, c0 + c, lane);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = kpos0 + c + 8 * u;
                        uint4 w;
                        w.x = pack_bf16(y[8 * u], y[8 * u + 1]);
                        w.y = pack_bf16(y[8 * u + 2], y[8 * u + 3]);
                        w.z = pack_bf16(y[8 * u + 4], y[8 * u + 5]);
                        w.w = pack_bf16(y[8 * u + 6], y[8 * u + 7]);
                        *reinterpret_cast<uint4*>(smem + (k / SLAB) * SLAB_BYTES + r * 128 +
                                                  ((((k % SLAB) / 8) ^ (r & 7)) * 16)) = w;
                    }
                }
                if (H % SLAB)   // the K padding of the last slab reads as zero in the next layer
                    for (int k = H; k < hslabs * SLAB; k += 8)
                        *reinterpret_cast<uint4*>(smem + (k / SLAB) * SLAB_BYTES + r * 128 +
                                                  ((((k % SLAB) / 8) ^ (r & 7)) * 16)) = make_uint4(0u, 0u, 0u, 0u);
                if (rank == 0 && m0 + r < M) {
                    if (s_mean) s_mean[m0 + r] = mean;
                    if (s_rstd) s_rstd[m0 + r] = rstd;
                }
                // the activation writes before the async proxy (MMA, TMA store, bulk copies)
                // reads them; tensor-memory reads before the next layer's MMAs
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                epi_bar();
                if (threadIdx.x == 0) {
                    if (s_ph) {
                        for (int j = 0; j < (NS + SLAB - 1) / SLAB; ++j)
                            tma_store_2d(&P.tph[l], a_base + (kpos0 / SLAB + j) * SLAB_BYTES, c0 + j * SLAB, m0);
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                    if (bcast) {
                        // this CTA's slice (whole slabs) into the same place of every other
                        // CTA's activation region; each copy completes on the receiver's barrier
                        const uint32_t src = a_base + (c0 / SLAB) * SLAB_BYTES, bytes = (uint32_t)NS * 256;
                        for (int q = 0; q < CL; ++q)
                            if (q != rank) bulk_s2s(mapa(src, q), src, bytes, mapa(a_ready, q));
                        mbar_expect_tx(a_ready, (uint32_t)(CL - 1) * bytes);
                    } else {
                        mbar_arrive_local(a_ready);
                    }
                }
            } else {
                // ------------------------------------------------------------ output layer epilogue
                const int nout = a.nout;
                const float* pob = par + nh * 3 * NS;
                // this row's output (or partial output) into the idle weight ring, then coalesced
                for (int c = 0; c < nop; c += 16) {
                    float v[16];
                    tmem_ld16(trow + c, v);
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(ring_f + r * ldr + c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                epi_bar();
                // four consecutive columns a thread: element e of the band is (row, 4 c4)
                const int nq = (nout + 3) / 4;
                if (CL == 1) {
                    for (int e = threadIdx.x; e < BM * nq; e += BM) {
                        const int row = e / nq, col = 4 * (e % nq);
                        const float4 x = *reinterpret_cast<const float4*>(ring_f + row * ldr + col);
                        const float4 bo = *reinterpret_cast<const float4*>(pob + col);
                        store_out4(p_out + (int64_t)(m0 + row) * p_ldo + col, make_float4(x.x + bo.x, x.y + bo.y,
                                   x.z + bo.z, x.w + bo.w), m0 + row < M ? nout - col : 0);
                    }
                } else {
                    // band q of the partial tile to CTA q (slot `rank` of its receive area,
                    // after its own K slice); the K split's partials are added in rank order
                    const uint32_t recv = a_base + (uint32_t)NS * 256, bb = (uint32_t)(band * ldr * 4);
                    if (threadIdx.x == 0)
                        for (int q = 0; q < CL; ++q)
                            bulk_s2s(mapa(recv + rank * bb, q), ring + q * bb, bb, mapa(out_bar, q));
                    mbar_wait<true>(out_bar, 0, err, 36, wlim);
                    const float* rv = reinterpret_cast<const float*>(smem + (size_t)NS * 256);
                    for (int e = threadIdx.x; e < band * nq; e += BM) {
                        const int row = e / nq, col = 4 * (e % nq);
                        float4 v = *reinterpret_cast<const float4*>(pob + col);
                        for (int q = 0; q < CL; ++q) {
                            const float4 x = *reinterpret_cast<const float4*>(rv + (q * band + row) * ldr + col);
                            v.x += x.x; v.y += x.y; v.z += x.z; v.w += x.w;
                        }
                        const int grow = m0 + rank * band + row;
                        store_out4(p_out + (int64_t)grow * p_ldo + col, v, grow < M ? nout - col : 0);
                    }
                }
            }
        }
        if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        (void)dead;
    }
    __syncthreads();
    // after a wait gave up: weight copies issued but never consumed still land in this
    // CTA's shared memory; wait for them (bounded) before the CTA can leave
    if (threadIdx.x == 0)
        for (int i = (int)slot[2]; i < (int)slot[1]; ++i) mbar_wait(full(i % S), (i / S) & 1, err, 37, wlim);
    // no CTA of the cluster leaves while a peer may still write into its shared memory
    if (CL > 1) cluster_sync_all();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    }
}

// ============================================================================ backward
// The input-gradient chain of a LayerNorm MLP head (Alg. 1's critic and actor steps):
//   step 0          dpost_{nh-1} = dout W_nh
//   hidden lh       dpre_lh = LayerNorm(+ReLU) backward of dpost_lh (Ba et al.):
//                   dn = dpost (x) [post > 0], dxh = dn (x) g,
//                   dpre = rstd (dxh - mean(dxh) - xhat mean(dxh (x) xhat)),
//                   then dpost_{lh-1} = dpre_lh W_lh (lh > 0)
//   final           dX[:, c0 : c0 + ncols] = dpre_0 W_0[:, c0 : c0 + ncols]
// in one launch, with the same cluster split as the forward: CTA q computes columns
// [q NS, (q + 1) NS) of every hidden gradient (tcgen05 M = 128, N = NS, the weights as
// MN-major operands streamed by TMA), xhat and dxh kept in tensor memory between the
// two LayerNorm passes, the row sums of dxh and dxh xhat exchanged with st.async, the
// BF16 dpre slice copied to the other CTAs by bulk copies.  Per hidden layer the kernel
// also leaves what the weight gradients need: dpre in BF16 (TMA store) and, per 128-row
// block, the column sums of dn xhat, dn and dpre (the LayerNorm gain, shift and bias
// gradients once the row blocks are added).  The final step is split over the output
// columns (each CTA ncols / CL of them) or, for a few columns, over K (each CTA its own
// dpre_0 slice; the partial tiles added in rank order by the CTA owning each band of rows).
struct MlpBwdProbDev {
    CUtensorMap tdo;                          // dout [M, nout], box 64 x 128 (K-major A of step 0)
    CUtensorMap tw[kMlpMaxHidden + 1];        // W_l [out_l, in_l] as MN-major B: dims {in_l, out_l}, box 64 x 64
    CUtensorMap tdp[kMlpMaxHidden];           // dpre of hidden layer l, BF16 [M, H], box 64 x 128 (store)
    const float* g[kMlpMaxHidden];
    const float* beta[kMlpMaxHidden];         // set: the ReLU mask is rebuilt from pre
    const float* pre[kMlpMaxHidden];
    const float* post[kMlpMaxHidden];
    const float* mean[kMlpMaxHidden];
    const float* rstd[kMlpMaxHidden];
    float* colpart[kMlpMaxHidden];            // [row blocks][3][H] or null
    int has_dp[kMlpMaxHidden];
    float* dx; int64_t lddx;
    int M, cta0;
};
struct MlpBwdArgs {
    MlpBwdProbDev p[kMlpMaxProbs];
    int n_probs, nh, H, CL, NS, nko;
    int c0, ncols, nfin, fin_ksplit;   // ncols = 0: no final step (the chain stops at dpre_0)
    int stages, stage_bytes, a_bytes, ldr;
    uint32_t tmem_cols;
    int* err;
    long long wait_limit;
};

// MN-major operand tile: 64-wide blocks of 64 K rows (128-byte swizzled), the blocks 8 KB
// apart along MN; the descriptor of K step kk of a slab.
__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(8192 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
__host__ __device__ constexpr uint32_t idesc_bf16_kn(int M, int N) {   // A K-major, B MN-major
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]), "f"(v[8]), "f"(v[9]),
        "f"(v[10]), "f"(v[11]), "f"(v[12]), "f"(v[13]), "f"(v[14]), "f"(v[15]), "f"(v[16]), "f"(v[17]), "f"(v[18]),
        "f"(v[19]), "f"(v[20]), "f"(v[21]), "f"(v[22]), "f"(v[23]), "f"(v[24]), "f"(v[25]), "f"(v[26]), "f"(v[27]),
        "f"(v[28]), "f"(v[29]), "f"(v[30]), "f"(v[31])
        : "memory");
}
// Row `lane` of this warp's rows [row0, row0 + 32), columns [col, col + 32) of src, read as
// coalesced 128-byte row segments through the warp's staging tile (rows >= M read as 0).
__device__ __forceinline__ void load_rows_coalesced(float* stg, const float* src, int64_t ld, int row0, int M, int col,
                                                    int lane, float (&v)[32]) {
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int rr = 4 * i + lane / 8;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row0 + rr < M) x = *reinterpret_cast<const float4*>(src + (int64_t)(row0 + rr) * ld + col + 4 * (lane % 8));
        *reinterpret_cast<float4*>(stg + rr * STG_LD + 4 * (lane % 8)) = x;
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(stg + lane * STG_LD + j);
        v[j] = x.x; v[j + 1] = x.y; v[j + 2] = x.z; v[j + 3] = x.w;
    }
}
// The two halves of load_rows_coalesced, for software pipelining: issue the eight 16-byte
// reads of a 32 x 32 tile (kept in flight in registers), then pass them through the
// staging tile into row `lane`.
__device__ __forceinline__ void issue_rows(float4 (&pf)[8], const float* src, int64_t ld, int row0, int M, int col,
                                           int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int rr = 4 * i + lane / 8;
        pf[i] = row0 + rr < M ? __ldg(reinterpret_cast<const float4*>(src + (int64_t)(row0 + rr) * ld + col + 4 * (lane % 8)))
                              : make_float4(0.f, 0.f, 0.f, 0.f);
    }
}
__device__ __forceinline__ void stage_rows(float* stg, const float4 (&pf)[8], int lane, float (&v)[32]) {
    __syncwarp();
#pragma unroll
    for (int i = 0; i < 8; ++i) *reinterpret_cast<float4*>(stg + (4 * i + lane / 8) * STG_LD + 4 * (lane % 8)) = pf[i];
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; j += 4) {
        const float4 x = *reinterpret_cast<const float4*>(stg + lane * STG_LD + j);
        v[j] = x.x; v[j + 1] = x.y; v[j + 2] = x.z; v[j + 3] = x.w;
    }
}
// Column sums (as warp_col_sum) of the elementwise product a (x) b.
__device__ __forceinline__ float warp_col_sum_prod(float* stg, const float (&a)[32], const float (&b)[32], int lane) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(stg + lane * STG_LD + j) =
            make_float4(a[j] * b[j], a[j + 1] * b[j + 1], a[j + 2] * b[j + 2], a[j + 3] * b[j + 3]);
    __syncwarp();
    float t = 0.f;
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) t += stg[rr * STG_LD + lane];
    return t;
}
// Sum over this warp's 32 rows of each of 32 columns (lane j returns column j's sum, rows
// added in order) through the warp's staging tile.
__device__ __forceinline__ float warp_col_sum(float* stg, const float (&v)[32], int lane) {
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; j += 4)
        *reinterpret_cast<float4*>(stg + lane * STG_LD + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    __syncwarp();
    float t = 0.f;
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) t += stg[rr * STG_LD + lane];
    return t;
}

__global__ void __launch_bounds__(kThreads, 1) mlp_bwd_tc_kernel(const __grid_constant__ MlpBwdArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int S = a.stages;
    const int CL = a.CL, NS = a.NS, H = a.H, nh = a.nh, nfin = a.nfin;
    const bool ksplit = a.fin_ksplit != 0;
    const int nsteps = nh + (a.ncols > 0 ? 1 : 0);
    const uint32_t a_base = smem_u32(smem);
    const uint32_t ring = a_base + a.a_bytes;
    float* ring_f = reinterpret_cast<float*>(smem + a.a_bytes);
    float* stg = reinterpret_cast<float*>(smem + a.a_bytes + S * a.stage_bytes);
    float* xbuf = stg + 4 * 32 * STG_LD;                                 // [2][CL][BM][2]: row sums of each CTA
    float* colacc = xbuf + 2 * CL * BM * 2;                              // [4 warps][3][NS] column sums
    float* par = colacc + 4 * 3 * NS;                                    // g (then beta) slices of the hidden layers
    uint64_t* bars = reinterpret_cast<uint64_t*>(par + ((2 * nh * NS + 3) / 4) * 4);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);     // tmem address, issued, consumed
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8 * s; };
    auto empty = [&](int s) { return bar0 + 8 * (S + s); };
    const uint32_t a0_full = bar0 + 8 * (2 * S), acc_full = a0_full + 8, a_ready = a0_full + 16;
    const uint32_t xbar0 = a0_full + 24, out_bar = a0_full + 40;

    int pi = 0;
    while (pi + 1 < a.n_probs && (int)blockIdx.x >= a.p[pi + 1].cta0) ++pi;
    const MlpBwdProbDev& P = a.p[pi];
    const int rank = CL > 1 ? (int)cluster_rank() : 0;
    const int m0 = ((int)blockIdx.x - P.cta0) / CL * BM;
    const int rb = m0 / BM;
    const int M = P.M;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long wlim = a.wait_limit;
    int* err = a.err;
    const int hslabs = (H + SLAB - 1) / SLAB;
    const int ldr = a.ldr, band = BM / CL;
    // K slabs of step s: dout's, H's, or (final, split over K) this CTA's slice
    auto nk = [&](int st) { return st == 0 ? a.nko : (st < nh ? hslabs : ((ksplit && CL > 1) ? NS / SLAB : hslabs)); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(a0_full, 1);
        mbar_init(acc_full, 1);
        mbar_init(a_ready, 1);
        mbar_init(xbar0, 1);
        mbar_init(xbar0 + 8, 1);
        mbar_init(out_bar, 1);
        slot[1] = 0;
        slot[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        if (CL > 1) {
            mbar_expect_tx(xbar0, (uint32_t)(CL * BM * 8));
            mbar_expect_tx(xbar0 + 8, (uint32_t)(CL * BM * 8));
            if (ksplit) mbar_expect_tx(out_bar, (uint32_t)(CL * band * ldr * 4));
        }
    }
    if (threadIdx.x == 128) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.tdo)) : "memory");
        for (int l = a.ncols > 0 ? 0 : 1; l <= nh; ++l)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.tw[l])) : "memory");
    }
    __syncthreads();
    if (CL > 1) cluster_sync_all();
    SQ_KERNEL_ENTRY();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(a.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = slot[0];

    if (warp == 4) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            mbar_expect_tx(a0_full, (uint32_t)(a.nko * SLAB_BYTES));
            for (int kb = 0; kb < a.nko; ++kb) tma_load_2d(a_base + kb * SLAB_BYTES, &P.tdo, kb * SLAB, m0, a0_full);
            int it = 0;
            bool ok = true;
            for (int st = 0; st < nsteps && ok; ++st) {
                const bool fin = st == nh;
                const int wl = nh - st;                        // the weight this step multiplies by
                const int N = fin ? nfin : NS;
                const int n0 = fin ? (ksplit ? a.c0 : a.c0 + rank * nfin) : rank * NS;
                const int k0 = (fin && ksplit) ? rank * NS : 0;
                for (int kb = 0; kb < nk(st); ++kb, ++it) {
                    const int s = it % S;
                    if (it >= S && !mbar_wait(empty(s), ((it / S) - 1) & 1, err, 40, wlim)) { ok = false; break; }
                    mbar_expect_tx(full(s), (uint32_t)(N * 128));
                    for (int j = 0; j < N / 64; ++j)
                        tma_load_2d(ring + s * a.stage_bytes + j * 8192, &P.tw[wl], n0 + 64 * j, k0 + kb * SLAB, full(s));
                }
            }
            slot[1] = it;
        }
    } else {
        const int r = warp * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        float* stg_w = stg + warp * 32 * STG_LD;
        const bool rebuild = P.beta[0] != nullptr;   // the ReLU mask from pre, g and beta
        if (warp > 0)
            for (int i = threadIdx.x - 32; i < (rebuild ? 2 : 1) * nh * NS; i += 96) {
                const int l = (i / NS) % nh;
                par[i] = (i < nh * NS ? P.g[l] : P.beta[l])[rank * NS + i % NS];
            }
        float* const p_dx = P.dx;
        const int64_t p_lddx = P.lddx;
        int it = 0;
        bool dead = false;
        for (int st = 0; st < nsteps; ++st) {
            const bool fin = st == nh;
            // this step's first tile of pre and the row statistics, read while its MMAs run
            const int lh = nh - 1 - st;
            const bool valid = m0 + r < M;
            float4 pf[8];
            float mean = 0.f, rstd = 0.f;
            if (!fin) {
                if (rebuild) issue_rows(pf, P.pre[lh], H, m0 + warp * 32, M, rank * NS, lane);
                if (valid) {
                    mean = __ldg(P.mean[lh] + m0 + r);
                    rstd = __ldg(P.rstd[lh] + m0 + r);
                }
            }
            // ---------------------------------------------------------------- MMA issue
            if (threadIdx.x == 0) {
                if (!dead) {
                    if (st == 0) dead = !mbar_wait(a0_full, 0, err, 41, wlim);
                    else dead = !mbar_wait<true>(a_ready, (st - 1) & 1, err, 42, wlim);
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = idesc_bf16_kn(BM, fin ? nfin : NS);
                for (int kb = 0; kb < nk(st) && !dead; ++kb) {
                    const int s = it % S;
                    if (!mbar_wait(full(s), (it / S) & 1, err, 43, wlim)) { dead = true; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t as = a_base + kb * SLAB_BYTES, bs = ring + s * a.stage_bytes;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_bf16(tmem, sw128_desc(as + kk * 32), sw128_desc_mn(bs + kk * 2048), idesc,
                                 (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(empty(s));
                    ++it;
                }
                slot[2] = it;
                mma_commit(acc_full);
            }
            __syncwarp();
            mbar_wait(acc_full, st & 1, err, 44, wlim);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (st == 0) epi_bar();   // the staged g slices
            if (!fin) {
                // ------------------------------------------------------------ LayerNorm (+ReLU) backward
                const int c0 = rank * NS;
                const float* gsl = par + lh * NS;
                const float* bsl = par + (nh + lh) * NS;
                const float* const s_pre = P.pre[lh];
                const float* const s_post = P.post[lh];
                float* const s_col = P.colpart[lh];
                const bool s_dp = P.has_dp[lh] != 0;
                float s1 = 0.f, s2 = 0.f;
                for (int c = 0; c < NS; c += 32) {
                    float dp[32], xh[32], t[32];
                    if (rebuild) {
                        stage_rows(stg_w, pf, lane, xh);
                        if (c + 32 < NS) issue_rows(pf, s_pre, H, m0 + warp * 32, M, c0 + c + 32, lane);
                    } else {
                        load_rows_coalesced(stg_w, s_pre, H, m0 + warp * 32, M, c0 + c, lane, xh);
                    }
                    tmem_ld32(trow + c, dp);
#pragma unroll
                    for (int j = 0; j < 32; ++j) xh[j] = (xh[j] - mean) * rstd;
                    ld_par32(gsl + c, t);
                    if (rebuild) {
                        float bt[32];
                        ld_par32(bsl + c, bt);
#pragma unroll
                        for (int j = 0; j < 32; ++j) dp[j] = (valid && __fmaf_rn(t[j], xh[j], bt[j]) > 0.f) ? dp[j] : 0.f;
                    } else {
                        float po[32];
                        load_rows_coalesced(stg_w, s_post, H, m0 + warp * 32, M, c0 + c, lane, po);
#pragma unroll
                        for (int j = 0; j < 32; ++j) dp[j] = (valid && po[j] > 0.f) ? dp[j] : 0.f;   // dn
                    }
                    if (s_col) {
                        colacc[(warp * 3 + 0) * NS + c + lane] = warp_col_sum_prod(stg_w, dp, xh, lane);
                        colacc[(warp * 3 + 1) * NS + c + lane] = warp_col_sum(stg_w, dp, lane);
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        t[j] *= dp[j];                          // dxh
                        s1 += t[j];
                        s2 += t[j] * xh[j];
                    }
                    tmem_st32(trow + NS + c, xh);
                    tmem_st32(trow + 2 * NS + c, t);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                if (CL > 1) {
                    const int b = st & 1;
                    float* buf = xbuf + b * CL * BM * 2;
                    const uint32_t mine = smem_u32(buf + (rank * BM + r) * 2), xb = xbar0 + 8 * b;
                    for (int q = 0; q < CL; ++q) st_async_v2(mapa(mine, q), s1, s2, mapa(xb, q));
                    mbar_wait<true>(xb, (st >> 1) & 1, err, 45, wlim);
                    if (threadIdx.x == 0) mbar_expect_tx(xb, (uint32_t)(CL * BM * 8));
                    s1 = 0.f;
                    s2 = 0.f;
                    for (int q = 0; q < CL; ++q) {
                        s1 += buf[(q * BM + r) * 2];
                        s2 += buf[(q * BM + r) * 2 + 1];
                    }
                }
                const float m1 = s1 / (float)H, m2 = s2 / (float)H;
                // the previous layer's TMA store has read this CTA's slabs before they are rewritten
                if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                epi_bar();
                const bool last_hidden = lh == 0;
                // dpre_0 feeds the final step: every CTA needs all of it when that step splits
                // the output columns, only its own slice (kept at the start) when it splits K
                const bool bcast = CL > 1 && !(last_hidden && (ksplit || nsteps == nh));
                const int kpos0 = (CL > 1 && last_hidden && ksplit && nsteps > nh) ? 0 : c0;
                for (int c = 0; c < NS; c += 32) {
                    float xh[32], v[32];
                    {
                        float dxh[32];
                        tmem_ld32(trow + NS + c, xh);
                        tmem_ld32(trow + 2 * NS + c, dxh);
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = rstd * (dxh[j] - m1 - xh[j] * m2);   // dpre
                    }
                    if (s_col) colacc[(warp * 3 + 2) * NS + c + lane] = warp_col_sum(stg_w, v, lane);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = kpos0 + c + 8 * u;
                        uint4 w;
                        w.x = pack_bf16(v[8 * u], v[8 * u + 1]);
                        w.y = pack_bf16(v[8 * u + 2], v[8 * u + 3]);
                        w.z = pack_bf16(v[8 * u + 4], v[8 * u + 5]);
                        w.w = pack_bf16(v[8 * u + 6], v[8 * u + 7]);
                        *reinterpret_cast<uint4*>(smem + (k / SLAB) * SLAB_BYTES + r * 128 +
                                                  ((((k % SLAB) / 8) ^ (r & 7)) * 16)) = w;
                    }
                }
                if (H % SLAB)
                    for (int k = H; k < hslabs * SLAB; k += 8)
                        *reinterpret_cast<uint4*>(smem + (k / SLAB) * SLAB_BYTES + r * 128 +
                                                  ((((k % SLAB) / 8) ^ (r & 7)) * 16)) = make_uint4(0u, 0u, 0u, 0u);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                epi_bar();
                if (s_col) {   // this row block's column sums of the slice, warps added in order
                    for (int i = threadIdx.x; i < 3 * NS; i += BM) {
                        const int k = i / NS, j = i % NS;
                        const float t = ((colacc[(0 * 3 + k) * NS + j] + colacc[(1 * 3 + k) * NS + j]) +
                                         colacc[(2 * 3 + k) * NS + j]) + colacc[(3 * 3 + k) * NS + j];
                        s_col[((int64_t)rb * 3 + k) * H + c0 + j] = t;
                    }
                    epi_bar();   // read before the next layer's column sums overwrite them
                }
                if (threadIdx.x == 0) {
                    if (s_dp) {
                        for (int j = 0; j < (NS + SLAB - 1) / SLAB; ++j)
                            tma_store_2d(&P.tdp[lh], a_base + (kpos0 / SLAB + j) * SLAB_BYTES, c0 + j * SLAB, m0);
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                    if (bcast) {
                        const uint32_t src = a_base + (c0 / SLAB) * SLAB_BYTES, bytes = (uint32_t)NS * 256;
                        for (int q = 0; q < CL; ++q)
                            if (q != rank) bulk_s2s(mapa(src, q), src, bytes, mapa(a_ready, q));
                        mbar_expect_tx(a_ready, (uint32_t)(CL - 1) * bytes);
                    } else {
                        mbar_arrive_local(a_ready);
                    }
                }
            } else if (!ksplit) {
                // ------------------------------------------------------------ final step, split over columns
                for (int c = 0; c < nfin; c += 32) {
                    float v[32];
                    tmem_ld32(trow + c, v);
                    store_rows_coalesced(stg_w, v, p_dx, p_lddx, m0 + warp * 32, M, rank * nfin + c, lane);
                }
            } else {
                // ------------------------------------------------------------ final step, split over K
                for (int c = 0; c < nfin; c += 16) {
                    float v[16];
                    tmem_ld16(trow + c, v);
#pragma unroll
                    for (int j = 0; j < 16; j += 4)
                        *reinterpret_cast<float4*>(ring_f + r * ldr + c + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                epi_bar();
                const int ncols = a.ncols;
                if (CL == 1) {
                    for (int e = threadIdx.x; e < BM * ncols; e += BM) {
                        const int row = e / ncols, col = e % ncols;
                        if (m0 + row < M) p_dx[(int64_t)(m0 + row) * p_lddx + col] = ring_f[row * ldr + col];
                    }
                } else {
                    const uint32_t recv = a_base + (uint32_t)NS * 256, bb = (uint32_t)(band * ldr * 4);
                    if (threadIdx.x == 0)
                        for (int q = 0; q < CL; ++q) bulk_s2s(mapa(recv + rank * bb, q), ring + q * bb, bb, mapa(out_bar, q));
                    mbar_wait<true>(out_bar, 0, err, 46, wlim);
                    const float* rv = reinterpret_cast<const float*>(smem + (size_t)NS * 256);
                    for (int e = threadIdx.x; e < band * ncols; e += BM) {
                        const int row = e / ncols, col = e % ncols;
                        float v = 0.f;
                        for (int q = 0; q < CL; ++q) v += rv[(q * band + row) * ldr + col];
                        const int grow = m0 + rank * band + row;
                        if (grow < M) p_dx[(int64_t)grow * p_lddx + col] = v;
                    }
                }
            }
        }
        if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
        (void)dead;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = (int)slot[2]; i < (int)slot[1]; ++i) mbar_wait(full(i % S), (i / S) & 1, err, 47, wlim);
    if (CL > 1) cluster_sync_all();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D BF16 tensor map over `outer` rows of `inner` elements (row stride ld), 128-byte
// swizzle, box box_inner x box_outer, zero fill outside the matrix.
bool make_map(CUtensorMap* m, const void* ptr, int64_t inner, int64_t outer, int64_t ld, int box_inner, int box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * 2) & 15) || inner < 1 || outer < 1 || box_outer > 256)
        return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    std::memset(m, 0, sizeof(*m));
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int round16(int n) { return (n + 15) / 16 * 16; }

// Shared-memory plan of one launch; false if it does not fit: the activation region (the
// input's or a hidden layer's K slabs, whichever is wider), the weight ring (which also
// stages the output tile), the FP32 store staging, the statistics exchange buffers, the
// parameter slices and the barriers.
bool plan(int H, int CL, int nh, int nop, int kin, int* a_bytes, int* stage_bytes, int* stages, int* par_floats,
          int* smem) {
    const int NS = H / CL;
    const int k0 = (kin + SLAB - 1) / SLAB, hs = (H + SLAB - 1) / SLAB;
    *a_bytes = std::max(k0, hs) * SLAB_BYTES;
    *stage_bytes = std::max(NS, nop) * 128;
    *par_floats = (nh * 3 * NS + nop + 3) / 4 * 4;
    const int fixed = 1024 + STG_BYTES + 2 * CL * BM * 2 * 4 + *par_floats * 4 + 256;
    const int n = (SMEM_LIMIT - fixed - *a_bytes) / *stage_bytes;
    *stages = std::min(n, 8);
    *smem = fixed + *a_bytes + *stages * *stage_bytes;
    return *stages >= 2 && *stages * *stage_bytes >= BM * nop * 4;
}

// Row stride of the output staging: padded by 4 floats (fewer bank conflicts) when the
// receive area after the CTA's own K slice has room for it.
int out_ldr(int H, int CL, int nop, int ring_bytes) {
    const int NS = H / CL;
    const bool recv_room = CL == 1 || (nop + 4) * 2 <= H - NS;
    return (recv_room && BM * (nop + 4) * 4 <= ring_bytes) ? nop + 4 : nop;
}

}  // namespace

namespace {

// Shared-memory plan of a backward launch (the same regions as the forward's, plus the
// column-sum staging; no output receive area unless the final step splits K).
bool plan_bwd(int H, int CL, int nh, int nko, int nfin, bool ksplit, int* a_bytes, int* stage_bytes, int* stages,
              int* ldr, int* smem) {
    const int NS = H / CL;
    const int hs = (H + SLAB - 1) / SLAB;
    *ldr = nfin + 4;
    // the activation region also holds the final step's receive area after the own slice
    *a_bytes = std::max(nko, hs) * SLAB_BYTES;
    if (ksplit && CL > 1) *a_bytes = std::max(*a_bytes, (NS * 256 + BM * *ldr * 4 + 1023) / 1024 * 1024);
    *stage_bytes = std::max(NS, nfin) * 128;
    const int fixed = 1024 + STG_BYTES + 2 * CL * BM * 2 * 4 + 4 * 3 * NS * 4 + ((2 * nh * NS + 3) / 4) * 16 + 256;
    const int n = (SMEM_LIMIT - fixed - *a_bytes) / *stage_bytes;
    *stages = std::min(n, 8);
    *smem = fixed + *a_bytes + *stages * *stage_bytes;
    if (*stages < 2) return false;
    if (ksplit && *stages * *stage_bytes < BM * *ldr * 4) return false;   // the partial tile staged in the ring
    return true;
}

// Cluster size of a backward launch: slices of whole 64-column blocks (the MN-major
// weight tiles are 64 columns wide) whose gradient, xhat and dxh fit in tensor memory
// (3 NS <= 512 columns).
int mlp_bwd_cluster(int H, int nout, int force) {
    auto ok = [&](int CL) {
        const int NS = H / CL;
        return H % CL == 0 && NS % SLAB == 0 && 3 * NS <= 512;
    };
    (void)nout;
    if ((force == 1 || force == 2 || force == 4 || force == 8) && ok(force)) return force;
    for (int CL : {4, 2, 1})
        if (ok(CL)) return CL;
    return 0;
}

// Final step: split over the output columns when each CTA gets a multiple of 64 of them,
// else over K with one 64-column tile.
void fin_split(int ncols, int CL, int* nfin, bool* ksplit) {
    if (CL == 1 && ncols % 64 == 0 && ncols <= 256) { *nfin = ncols; *ksplit = false; return; }
    if (CL > 1 && ncols % (64 * CL) == 0 && ncols / CL <= 256) { *nfin = ncols / CL; *ksplit = false; return; }
    *nfin = 64;
    *ksplit = true;
}

}  // namespace

bool mlp_bwd_tc_supported(int nh, int H, int nout, int kin, int c0, int ncols, int force_cluster) {
    if (nh < 1 || nh > kMlpMaxHidden || H < 32 || H > 1024 || H % 32 || nout < 1 || nout > 256 || kin < 1 ||
        c0 < 0 || c0 % 8 || ncols < 0 || c0 + ncols > kin)
        return false;
    const int CL = mlp_bwd_cluster(H, nout, force_cluster);
    if (!CL) return false;
    int nfin = 0;
    bool ks = false;
    if (ncols > 0) fin_split(ncols, CL, &nfin, &ks);
    if (ks && ncols > 64) return false;
    int ab, sb, st, ldr, sm;
    return plan_bwd(H, CL, nh, (nout + SLAB - 1) / SLAB, nfin, ks, &ab, &sb, &st, &ldr, &sm);
}

void mlp_bwd_tc_prepare() {
    cudaFuncSetAttribute(mlp_bwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
}

int launch_mlp_bwd_tc(const MlpTcBwdProblem* p, int n, int nh, int H, int nout, int kin, int c0, int ncols, int* err,
                      const TcWait* wait, cudaStream_t s, int force_cluster) {
    if (n < 1 || n > kMlpMaxProbs || !mlp_bwd_tc_supported(nh, H, nout, kin, c0, ncols, force_cluster)) return -1;
    const int CL = mlp_bwd_cluster(H, nout, force_cluster);
    MlpBwdArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n_probs = n; a.nh = nh; a.H = H; a.CL = CL; a.NS = H / CL; a.nko = (nout + SLAB - 1) / SLAB;
    a.c0 = c0; a.ncols = ncols;
    bool ks = false;
    if (ncols > 0) fin_split(ncols, CL, &a.nfin, &ks);
    a.fin_ksplit = ks ? 1 : 0;
    a.err = err;
    a.wait_limit = wait && wait->cycles > 0 ? wait->cycles : kWaitDefault;
    int smem = 0;
    if (!plan_bwd(H, CL, nh, a.nko, a.nfin, ks, &a.a_bytes, &a.stage_bytes, &a.stages, &a.ldr, &smem)) return -1;
    const int need_cols = std::max(3 * a.NS, a.nfin);
    a.tmem_cols = 32;
    while ((int)a.tmem_cols < need_cols) a.tmem_cols *= 2;
    int ctas = 0;
    for (int i = 0; i < n; ++i) {
        const MlpTcBwdProblem& q = p[i];
        MlpBwdProbDev& d = a.p[i];
        if (q.M < 1 || !q.dout || (ncols > 0 && !q.dx) || (ncols == 0 && !q.dpre_bf[0])) return -1;
        if (!make_map(&d.tdo, q.dout, nout, q.M, q.ld_dout, SLAB, BM)) return -2;
        for (int l = 0; l <= nh; ++l) {
            const int in = l == 0 ? kin : H, out = l == nh ? nout : H;
            if (!q.w[l] && (l > 0 || ncols > 0)) return -1;
            if (q.w[l] && !make_map(&d.tw[l], q.w[l], in, out, q.ldw[l], SLAB, SLAB)) return -2;
            if (l == nh) break;
            // the shifts of every hidden layer or of none; post only when they are absent
            if (!q.g[l] || !q.pre[l] || !q.mean[l] || !q.rstd[l] || (!q.beta[l]) != (!q.beta[0]) ||
                (!q.beta[l] && !q.post[l]))
                return -1;
            d.g[l] = q.g[l]; d.beta[l] = q.beta[l]; d.pre[l] = q.pre[l]; d.post[l] = q.post[l];
            d.mean[l] = q.mean[l]; d.rstd[l] = q.rstd[l];
            d.colpart[l] = q.colpart[l];
            d.has_dp[l] = q.dpre_bf[l] != nullptr;
            if (d.has_dp[l] && !make_map(&d.tdp[l], q.dpre_bf[l], H, q.M, H, SLAB, BM)) return -2;
        }
        d.dx = q.dx; d.lddx = q.lddx;
        d.M = q.M;
        d.cta0 = ctas;
        ctas += (q.M + BM - 1) / BM * CL;
    }
    launch_kc(mlp_bwd_tc_kernel, dim3(ctas), dim3(kThreads), (size_t)smem, s, dim3(CL), a);
    return 0;
}

bool mlp_tc_supported(int nh, int H, int nout, int kin) {
    return nh >= 1 && nh <= kMlpMaxHidden && H >= 32 && H <= 1024 && H % 32 == 0 && nout >= 1 && nout <= 256 &&
           kin >= 1 && kin <= 1024 && mlp_tc_cluster(H, nout) > 0;
}

int mlp_tc_cluster(int H, int nout, int force) {
    const int nop = round16(nout);
    auto ok = [&](int CL) {
        const int NS = H / CL;
        if (H % CL || NS > 256 || NS % 32) return false;
        if (force && force != 1 && force != 2 && force != 4 && force != 8) return false;
        // slices in whole slabs; the output receive area after the CTA's own K slice
        if (CL > 1 && (NS % SLAB || nop * 2 > H - NS)) return false;
        int ab, sb, st, pf, sm;
        return plan(H, CL, kMlpMaxHidden, nop, std::min(H, 1024), &ab, &sb, &st, &pf, &sm);
    };
    if (force) return ok(force) ? force : 0;
    for (int CL : {4, 8, 2, 1})
        if (ok(CL)) return CL;
    return 0;
}

void mlp_tc_prepare() {
    cudaFuncSetAttribute(mlp_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_LIMIT);
    encode_fn();
}

int launch_mlp_tc(const MlpTcProblem* p, int n, int nh, int H, int nout, float eps, int* err, const TcWait* wait,
                  cudaStream_t s, int force_cluster) {
    if (n < 1 || n > kMlpMaxProbs || nh < 1 || nh > kMlpMaxHidden) return -1;
    const int CL = mlp_tc_cluster(H, nout, force_cluster);
    if (!CL) return -1;
    MlpArgs a;
    std::memset(&a, 0, sizeof(a));
    a.n_probs = n; a.nh = nh; a.H = H; a.CL = CL; a.NS = H / CL; a.nout = nout; a.nop = round16(nout);
    a.eps = eps; a.err = err;

    a.wait_limit = wait && wait->cycles > 0 ? wait->cycles : kWaitDefault;
    int kin_max = 0;
    for (int i = 0; i < n; ++i) kin_max = std::max(kin_max, p[i].kin);
    if (kin_max > 1024) return -1;
    int smem = 0;
    if (!plan(H, CL, nh, a.nop, kin_max, &a.a_bytes, &a.stage_bytes, &a.stages, &a.par_floats, &smem)) return -1;
    a.ldr = out_ldr(H, CL, a.nop, a.stages * a.stage_bytes);
    const int need_cols = std::max(std::max(a.NS, a.nop), 32);
    a.tmem_cols = 32;
    while ((int)a.tmem_cols < need_cols) a.tmem_cols *= 2;
    int ctas = 0;
    for (int i = 0; i < n; ++i) {
        const MlpTcProblem& q = p[i];
        MlpProbDev& d = a.p[i];
        if (q.M < 1 || !q.x || !q.out || q.kin < 1) return -1;
        if (!make_map(&d.tx, q.x, q.kin, q.M, q.ldx, SLAB, BM)) return -2;
        for (int l = 0; l <= nh; ++l) {
            const bool last = l == nh;
            const int in = l == 0 ? q.kin : H;
            if (!q.w[l] || !q.bias[l]) return -1;
            if (!make_map(&d.tw[l], q.w[l], in, last ? nout : H, q.ldw[l], SLAB, last ? a.nop : a.NS)) return -2;
            d.bias[l] = q.bias[l];
            if (!last) {
                if (!q.g[l] || !q.beta[l]) return -1;
                d.g[l] = q.g[l]; d.beta[l] = q.beta[l];
                d.pre[l] = q.save[l].pre; d.post[l] = q.save[l].post;
                d.mean[l] = q.save[l].mean; d.rstd[l] = q.save[l].rstd;
                d.has_ph[l] = q.save[l].posth != nullptr;
                if (d.has_ph[l] && !make_map(&d.tph[l], q.save[l].posth, H, q.M, H, SLAB, BM)) return -2;
            }
        }
        d.out = q.out; d.ldo = q.ldo;
        d.M = q.M; d.nk0 = (q.kin + SLAB - 1) / SLAB;
        d.cta0 = ctas;
        ctas += (q.M + BM - 1) / BM * CL;
    }
    launch_kc(mlp_tc_kernel, dim3(ctas), dim3(kThreads), (size_t)smem, s, dim3(CL), a);
    return 0;
}

}  // namespace sq
