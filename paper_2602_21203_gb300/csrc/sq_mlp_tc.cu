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
//                     whole row (partial sums of the CL CTAs exchanged through
//                     distributed shared memory, added in rank order), ReLU; the BF16
//                     result is written straight into the activation region of every
//                     CTA of the cluster as the next layer's A operand; saved FP32
//                     activations leave through a per-warp transpose as coalesced rows,
//                     the BF16 copy by a TMA store of the CTA's own slabs
//   output layer      K split over the cluster (each CTA multiplies its own column slice
//                     of the last hidden layer); the partial tiles are pushed to the CTA
//                     owning each band of rows and added in rank order
//
// Cross-CTA ordering uses mbarriers with remote arrivals (release / acquire at cluster
// scope), so the producer never joins a cluster-wide barrier while it streams ahead.
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
constexpr int XBUF_BYTES = 2 * 4 * BM * 4;
constexpr int SMEM_LIMIT = 232448;
constexpr long long kWaitDefault = 4000000000ll;   // ~2 s at 2 GHz
constexpr int kMaxCluster = 4;

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
    int stages, stage_bytes, a_bytes;
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
// Arrive on the barrier at a shared::cluster address (this CTA's or a peer's), releasing
// this thread's earlier writes at cluster scope.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar) : "memory");
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
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}
__device__ __forceinline__ void st_cluster_f32(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v4f(uint32_t addr, float a, float b, float c, float d) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
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
    const uint32_t a_base = smem_u32(smem);
    const uint32_t ring = a_base + a.a_bytes;
    float* stg = reinterpret_cast<float*>(smem + a.a_bytes + S * a.stage_bytes);
    float* xbuf = stg + 4 * 32 * STG_LD;                                 // [2][kMaxCluster][BM]
    uint64_t* bars = reinterpret_cast<uint64_t*>(xbuf + 2 * kMaxCluster * BM);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2 * S + 6);     // tmem address, issued, consumed
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8 * s; };
    auto empty = [&](int s) { return bar0 + 8 * (S + s); };
    const uint32_t x_full = bar0 + 8 * (2 * S), acc_full = x_full + 8, a_ready = x_full + 16;
    const uint32_t xbar0 = x_full + 24, out_bar = x_full + 40;

    int pi = 0;
    while (pi + 1 < a.n_probs && (int)blockIdx.x >= a.p[pi + 1].cta0) ++pi;
    const MlpProbDev& P = a.p[pi];
    const int CL = a.CL, NS = a.NS, H = a.H, nh = a.nh;
    const int rank = CL > 1 ? (int)cluster_rank() : 0;
    const int m0 = ((int)blockIdx.x - P.cta0) / CL * BM;
    const int M = P.M;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const long long wlim = a.wait_limit;
    int* err = a.err;
    const int hslabs = (H + SLAB - 1) / SLAB;
    auto nk = [&](int l) { return l == 0 ? P.nk0 : (l < nh ? hslabs : (CL > 1 ? NS / SLAB : hslabs)); };

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(x_full, 1);
        mbar_init(acc_full, 1);
        mbar_init(a_ready, CL);
        mbar_init(xbar0, CL);
        mbar_init(xbar0 + 8, CL);
        mbar_init(out_bar, CL);
        slot[1] = 0;
        slot[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
                const uint32_t bytes = (uint32_t)((last ? a.nop : NS) * 128);
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
        float* stg_w = stg + warp * 32 * STG_LD;
        int it = 0;                                      // weight slab sequence (issuer)
        bool dead = false;                               // the issuer gave up on a wait
        int xph = 0;                                     // exchange phase
        // Sum of v over the CTAs of the cluster, in rank order (every thread: its own row).
        auto exchange = [&](float v) -> float {
            if (CL == 1) return v;
            const int b = xph & 1;
            float* buf = xbuf + b * kMaxCluster * BM;
            const uint32_t mine = smem_u32(buf + rank * BM + r);
            for (int q = 0; q < CL; ++q) st_cluster_f32(mapa(mine, q), v);
            asm volatile("fence.acq_rel.cluster;" ::: "memory");
            epi_bar();
            if (threadIdx.x == 0)
                for (int q = 0; q < CL; ++q) mbar_arrive_cluster(mapa(xbar0 + 8 * b, q));
            mbar_wait<true>(xbar0 + 8 * b, (xph >> 1) & 1, err, 35, wlim);
            ++xph;
            float t = 0.f;
            for (int q = 0; q < CL; ++q) t += buf[q * BM + r];
            return t;
        };
        for (int l = 0; l <= nh; ++l) {
            const bool last = l == nh;
            // ---------------------------------------------------------------- MMA issue
            if (threadIdx.x == 0) {
                if (!dead) {
                    if (l == 0) dead = !mbar_wait(x_full, 0, err, 31, wlim);
                    else dead = !mbar_wait<true>(a_ready, (l - 1) & 1, err, 32, wlim);
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = idesc_bf16_kk(BM, last ? a.nop : NS);
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
            if (!last) {
                // ------------------------------------------------------------ hidden layer epilogue
                const int c0 = rank * NS;                 // this CTA's first column
                const float* bias = P.bias[l] + c0;
                const float* gg = P.g[l] + c0;
                const float* bb = P.beta[l] + c0;
                float s1 = 0.f;
                for (int c = 0; c < NS; c += 32) {
                    float v[32];
                    tmem_ld32(trow + c, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) s1 += v[j] + __ldg(bias + c + j);
                }
                const float mean = exchange(s1) / (float)H;
                float s2 = 0.f;
                for (int c = 0; c < NS; c += 32) {
                    float v[32];
                    tmem_ld32(trow + c, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float d = v[j] + __ldg(bias + c + j) - mean;
                        s2 += d * d;
                    }
                }
                // the previous layer's TMA store has read this CTA's slabs before they are rewritten
                if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                const float rstd = 1.0f / sqrtf(exchange(s2) / (float)H + a.eps);
                // the last hidden layer feeds only this CTA's K slice of the output layer:
                // kept locally, at the start of the activation region
                const bool bcast = CL > 1 && l + 1 < nh;
                const int kpos0 = (CL > 1 && l + 1 == nh) ? 0 : c0;
                for (int c = 0; c < NS; c += 32) {
                    float v[32], y[32];
                    tmem_ld32(trow + c, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        v[j] += __ldg(bias + c + j);
                        y[j] = fmaxf((v[j] - mean) * rstd * __ldg(gg + c + j) + __ldg(bb + c + j), 0.f);
                    }
                    if (P.pre[l]) store_rows_coalesced(stg_w, v, P.pre[l], H, m0 + warp * 32, M, c0 + c, lane);
                    if (P.post[l]) store_rows_coalesced(stg_w, y, P.post[l], H, m0 + warp * 32, M, c0 + c, lane);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = kpos0 + c + 8 * u;
                        const uint32_t addr = a_base + (k / SLAB) * SLAB_BYTES + r * 128 + ((((k % SLAB) / 8) ^ (r & 7)) * 16);
                        const uint32_t w0 = pack_bf16(y[8 * u], y[8 * u + 1]), w1 = pack_bf16(y[8 * u + 2], y[8 * u + 3]);
                        const uint32_t w2 = pack_bf16(y[8 * u + 4], y[8 * u + 5]), w3 = pack_bf16(y[8 * u + 6], y[8 * u + 7]);
                        if (bcast)
                            for (int q = 0; q < CL; ++q) st_cluster_v4(mapa(addr, q), w0, w1, w2, w3);
                        else
                            st_cluster_v4(addr, w0, w1, w2, w3);
                    }
                }
                if (H % SLAB)   // the K padding of the last slab reads as zero in the next layer
                    for (int k = H; k < hslabs * SLAB; k += 8) {
                        const uint32_t addr = a_base + (k / SLAB) * SLAB_BYTES + r * 128 + ((((k % SLAB) / 8) ^ (r & 7)) * 16);
                        st_cluster_v4(addr, 0u, 0u, 0u, 0u);
                    }
                if (rank == 0 && m0 + r < M) {
                    if (P.mean[l]) P.mean[l][m0 + r] = mean;
                    if (P.rstd[l]) P.rstd[l][m0 + r] = rstd;
                }
                // generic-proxy writes of the activation region before the async proxy (MMA,
                // TMA store) reads it; tensor-memory reads before the next layer's MMAs
                asm volatile("fence.proxy.async;" ::: "memory");
                asm volatile("fence.acq_rel.cluster;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                epi_bar();
                if (threadIdx.x == 0) {
                    if (P.has_ph[l]) {
                        for (int j = 0; j < (NS + SLAB - 1) / SLAB; ++j)
                            tma_store_2d(&P.tph[l], a_base + (kpos0 / SLAB + j) * SLAB_BYTES, c0 + j * SLAB, m0);
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                    if (CL > 1)
                        for (int q = 0; q < CL; ++q) mbar_arrive_cluster(mapa(a_ready, q));
                    else
                        mbar_arrive_local(a_ready);
                }
            } else {
                // ------------------------------------------------------------ output layer epilogue
                const int nop = a.nop, nout = a.nout;
                const float* bias = P.bias[nh];
                if (CL == 1) {
                    for (int c = 0; c < nop; c += 16) {
                        float v[16];
                        tmem_ld16(trow + c, v);
                        if (m0 + r < M)
#pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (c + j < nout) P.out[(int64_t)(m0 + r) * P.ldo + c + j] = v[j] + __ldg(bias + c + j);
                    }
                } else {
                    // push this row's partial to the CTA that owns its band of rows: slot
                    // [rank][row in band] of that CTA's receive area (after its own K slice)
                    const int band = BM / CL;
                    const uint32_t recv = a_base + (uint32_t)NS * 256;
                    const uint32_t dst = mapa(recv + (uint32_t)((rank * band + r % band) * nop) * 4, r / band);
                    for (int c = 0; c < nop; c += 16) {
                        float v[16];
                        tmem_ld16(trow + c, v);
#pragma unroll
                        for (int j = 0; j < 16; j += 4) st_cluster_v4f(dst + (c + j) * 4, v[j], v[j + 1], v[j + 2], v[j + 3]);
                    }
                    asm volatile("fence.acq_rel.cluster;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    epi_bar();
                    if (threadIdx.x == 0)
                        for (int q = 0; q < CL; ++q) mbar_arrive_cluster(mapa(out_bar, q));
                    mbar_wait<true>(out_bar, 0, err, 36, wlim);
                    const float* rv = reinterpret_cast<const float*>(smem + (size_t)NS * 256);
                    for (int e = threadIdx.x; e < band * nout; e += BM) {
                        const int row = e / nout, col = e % nout;
                        float v = __ldg(bias + col);
                        for (int q = 0; q < CL; ++q) v += rv[(q * band + row) * nop + col];
                        const int grow = m0 + rank * band + row;
                        if (grow < M) P.out[(int64_t)grow * P.ldo + col] = v;
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

// Shared-memory plan of one launch; false if it does not fit.
bool plan(int H, int CL, int nop, int kin, int* a_bytes, int* stage_bytes, int* stages) {
    const int NS = H / CL;
    const int k0 = (kin + SLAB - 1) / SLAB, hs = (H + SLAB - 1) / SLAB;
    *a_bytes = std::max(k0, hs) * SLAB_BYTES;
    *stage_bytes = std::max(NS, nop) * 128;
    const int fixed = 1024 + STG_BYTES + XBUF_BYTES + 256;
    const int n = (SMEM_LIMIT - fixed - *a_bytes) / *stage_bytes;
    *stages = std::min(n, 8);
    return *stages >= 2;
}

}  // namespace

bool mlp_tc_supported(int nh, int H, int nout, int kin) {
    return nh >= 1 && nh <= kMlpMaxHidden && H >= 32 && H <= 1024 && H % 32 == 0 && nout >= 1 && nout <= 256 &&
           kin >= 1 && kin <= 1024 && mlp_tc_cluster(H, nout) > 0;
}

int mlp_tc_cluster(int H, int nout, int force) {
    const int nop = round16(nout);
    auto ok = [&](int CL) {
        const int NS = H / CL;
        if (H % CL || NS > 256 || NS % 32) return false;
        if (CL > 1 && (NS % SLAB || nop > (H - NS) / 2)) return false;   // slices in whole slabs; output receive area
        int ab, sb, st;
        return plan(H, CL, nop, std::min(H, 1024), &ab, &sb, &st);
    };
    if (force) return ok(force) ? force : 0;
    for (int CL : {4, 2, 1})
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
    if (!plan(H, CL, a.nop, kin_max, &a.a_bytes, &a.stage_bytes, &a.stages)) return -1;
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
    launch_kc(mlp_tc_kernel, dim3(ctas), dim3(kThreads), SMEM_LIMIT, s, dim3(CL), a);
    return 0;
}

}  // namespace sq
