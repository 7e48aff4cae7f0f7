// BF16 tensor-core GEMM for sm_103a: D[M,N] (+)= sum_pairs A[M,K] B[N,K]^T, FP32
// accumulation in tensor memory.
//
// Per CTA one 128 x 128 output tile, or one K range of it when the launch splits K over
// a thread-block cluster (few output tiles, long K):
//   warp 1 / lane 0   TMA producer: initialises the barriers (before the programmatic
//                     wait), then streams 128B-swizzled 64-wide K slabs of A and B into a
//                     6-stage shared-memory ring (mbarrier complete_tx)
//   warp 0 / lane 0   MMA issuer: 4 x tcgen05.mma (K = 16 each) per slab, commit frees
//                     the slab, a final commit signals the accumulator
//   warps 0-3         epilogue: each thread moves its accumulator row from tensor memory
//                     to shared memory (the idle operand ring); after a cluster barrier
//                     each CTA of the cluster adds the partial tiles of its band of rows
//                     in rank order through distributed shared memory, then applies
//                     bias and the optional ReLU mask and stores FP32 and/or BF16 rows
//                     with coalesced vector stores
// Operands are K-major (K contiguous) or MN-major (M or N contiguous), so the
// forward X W^T, the data gradient dY W and the weight gradient dY^T X all run
// from the row-major buffers without transposed copies.
// Every wait is bounded: past the launch's wait limit (kWaitCycles unless the host
// sets another) the waiting thread records an error code in *err and gives up; the
// tile is abandoned, the CTA waits (bounded again) for the operand copies it still
// has in flight, and TMEM is still freed.
#include "sq_tc.cuh"

#include <cuda.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

namespace sq {

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 6;
constexpr int TILE_BYTES = BM * BK * 2;                // 16 KB per operand per stage
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256 + BN * 4 + (2 * BN + 4 * BM) * 4;
// MX-FP8: each stage also holds the A and B block-scale atoms (512 B each), after the
// barriers and epilogue vectors (which take < 4 KB past the operand stages)
constexpr int SF_ATOM = 512;
constexpr int SF_OFF = STAGES * STAGE_BYTES + 4096;
constexpr int SMEM_BYTES_MX = SF_OFF + STAGES * 2 * SF_ATOM + 1024;
static_assert((2 * STAGES + 1) * 8 + 16 + (3 * BN + 4 * BM) * 4 <= 4096, "epilogue vectors overlap the scale atoms");
static_assert(SMEM_BYTES_MX <= 232448, "shared memory above the per-CTA limit");
constexpr int RED_LD = BN + 4;   // FP32 row stride of the accumulator tile in shared memory
static_assert(BM * RED_LD * 4 <= STAGES * STAGE_BYTES, "accumulator tile must fit in the operand stages");
constexpr long long kWaitCycles = 4000000000ll;        // ~2 s at 2 GHz
constexpr int kMaxProbs = 4;

struct TcProb {
    CUtensorMap ta[2];
    CUtensorMap tb[2];
    int M, N, K, n_pairs;
    int tiles_n, tile_start;   // tile_start: first CTA of this problem
    const float* bias;
    float* c; int64_t ldc;
    __nv_bfloat16* cbf; int64_t ldcbf;
    const float* mask; int64_t ldmask;
    int accumulate;
    const float* scale_a; const float* scale_b;
    const uint8_t* sf_a; const uint8_t* sf_b;   // MX block-scale atoms
    int64_t sfa_tile, sfb_tile;                 // bytes per 128-row (column) tile of sf_a (sf_b)
    const float* ln_g; const float* ln_beta;
    float* ln_post; __nv_bfloat16* ln_posth;
    float* ln_mean; float* ln_rstd;
    float ln_eps; int ln_relu;
};
struct TcBatch {
    TcProb p[kMaxProbs];
    int n;
    int splits;       // CTAs per output tile = cluster size (K split)
    int ln;           // LayerNorm epilogue: the cluster is the row block's column tiles (splits == 1)
    int* err;
    long long wait_limit;   // clock cycles a wait may take before it gives up
    int stall;        // failure test: the producer issues no operand loads, so the first
                      // operand wait runs out (nothing else is in flight when it does)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false (and *err = code) if the phase did not complete within `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, long long limit) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
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
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Arrive at and wait on the cluster barrier (every thread of every CTA of the cluster);
// release/acquire order this CTA's shared-memory writes before the other CTAs' reads.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Generic address of the same shared-memory location in CTA `rank` of the cluster
// (distributed shared memory; ordinary loads through it are scheduled like any other).
__device__ __forceinline__ const float* map_rank(const float* p, int rank) {
    uint64_t r;
    asm("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
    return reinterpret_cast<const float*>(r);
}
// Shared-memory matrix descriptor, 128-byte swizzle (sm_100 family descriptor version 1).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, majorness, N, M.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// Instruction descriptor of kind::f8f6f4 with e4m3 A and B (format code 0), FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N, bool a_mn, bool b_mn) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
// Instruction descriptor of kind::mxf8f6f4 (block-scaled): e4m3 A and B, FP32 accumulator,
// UE8M0 scales (bit 23), and the byte of each 32-bit scale column this MMA uses
// (b_sf_id at bits 4-5, a_sf_id at bits 29-30): the 32-element K block within the slab.
__host__ __device__ constexpr uint32_t idesc_mx(int M, int N, uint32_t sf_id) {
    return (sf_id << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | (1u << 23) |
           ((uint32_t)(M >> 4) << 24) | (sf_id << 29);
}
// D (+)= (A . 2^sfA) (B . 2^sfB)^T over K = 32, scales per row / column from tensor memory.
__device__ __forceinline__ void mma_mx(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t sfa_tmem, uint32_t sfb_tmem, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf8f6f4.block_scale.scale_vec::1X [%0], %1, %2, %3, [%4], [%5], p;\n}" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa_tmem), "r"(sfb_tmem), "r"(acc)
        : "memory");
}
// Shared-memory descriptor of a 32-row x 16-byte block-scale atom without swizzle
// (8-row core matrices of 128 contiguous bytes, 128 B apart).
__device__ __forceinline__ uint64_t sf_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(128 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Copy a 32 x 128-bit scale atom from shared memory into tensor memory, repeated in each
// of the four 32-lane quarters (lane r0 + 32 w, 4 columns: the scales of rows r0 + 32 c).
__device__ __forceinline__ void sf_copy(uint32_t taddr, uint64_t sdesc) {
    asm volatile("tcgen05.cp.cta_group::1.32x128b.warpx4 [%0], %1;" ::"r"(taddr), "l"(sdesc) : "memory");
}
__device__ __forceinline__ void bulk_copy_s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
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
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Operand tile in shared memory: K-major is 128 rows x 128 B (8-row groups 1024 B apart);
// MN-major is two 64-wide column blocks of 64 K rows (K groups of 8 rows 1024 B apart,
// the second MN block 8 KB further).  Descriptor of the 16-wide K step kk.
template <bool MN>
__device__ __forceinline__ uint64_t operand_desc(uint32_t tile, int kk) {
    if (MN) return sw128_desc(tile + kk * 2048, 8192, 1024);
    return sw128_desc(tile + kk * 32, 16, 1024);
}

template <bool MN>
__device__ __forceinline__ void load_operand(uint32_t dst, const CUtensorMap* map, int mn0, int k0, uint32_t bar) {
    if (MN) {
        tma_load_2d(dst, map, mn0, k0, bar);
        tma_load_2d(dst + 8192, map, mn0 + 64, k0, bar);
    } else {
        tma_load_2d(dst, map, k0, mn0, bar);
    }
}

// F8 = 1: e4m3 operands, 128-element (128-byte) K slabs, kind::f8f6f4 MMAs with K = 32,
// and the per-tensor scales applied in the epilogue.  The K step of a slab is 32 bytes in
// both types, so the shared-memory descriptors are the same.  F8 = 2 (MX-FP8): the same
// slabs with one UE8M0 scale per 32 elements of K per row of A and per column of B; each
// stage brings the slab's scale atoms along, copies them into tensor memory (columns of
// their own per stage) and the block-scaled MMAs apply them.
template <bool A_MN, bool B_MN, int F8 = 0>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ TcBatch gb) {
    constexpr bool MX = F8 == 2;
    constexpr int BKE = F8 ? 128 : BK;   // K elements per slab
    constexpr uint32_t TMEM_COLS = MX ? 256 : BN;   // MX: accumulator + 6 stages x (4 + 4) scale columns
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    // tmem_slot[1]: operand stages the producer issued; tmem_slot[2]: stages the MMA
    // issuer consumed (the copies of the ones in between are still in flight after a
    // wait gave up)
    float* bias_s = reinterpret_cast<float*>(tmem_slot + 4);          // [BN]
    float* g_s = bias_s + BN;                                          // [BN] LayerNorm gain
    float* beta_s = g_s + BN;                                          // [BN] LayerNorm shift
    float* ln_s1 = beta_s + BN;                                        // [BM] row sums of this tile
    float* ln_s2 = ln_s1 + BM;                                         // [BM] centred squares
    float* ln_mean_s = ln_s2 + BM;                                     // [BM]
    float* ln_rstd_s = ln_mean_s + BM;                                 // [BM]
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done_bar = smem_u32(bars + 2 * STAGES);

    int pi = 0;
    while (pi + 1 < gb.n && (int)blockIdx.x >= gb.p[pi + 1].tile_start) ++pi;
    const TcProb& P = gb.p[pi];
    // the problem's scalars, read once: P lives in the parameter block and is reached
    // through a generic pointer, which the compiler would otherwise re-read after every store
    const int pM = P.M, pN = P.N, pK = P.K, n_pairs = P.n_pairs, tiles_n = P.tiles_n;
    const float* const p_bias = P.bias;
    float* const p_c = P.c;
    const int64_t p_ldc = P.ldc;
    __nv_bfloat16* const p_cbf = P.cbf;
    const int64_t p_ldcbf = P.ldcbf;
    const float* const p_mask = P.mask;
    const int64_t p_ldmask = P.ldmask;
    const bool p_acc = P.accumulate != 0;
    const float* const p_sa = P.scale_a;
    const float* const p_sb = P.scale_b;
    const int cta = blockIdx.x - P.tile_start;
    const int crank = (int)cluster_rank();
    const int t = cta / gb.splits, split = gb.ln ? 0 : crank;   // K split rank (0 in LayerNorm mode)
    const int m0 = (t / tiles_n) * BM, n0 = (t % tiles_n) * BN;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const uint32_t base = smem_u32(smem);
    const int nkb = (pK + BKE - 1) / BKE;
    // this CTA's share of the (pair, K slab) iterations
    const int it0 = (int)((int64_t)nkb * n_pairs * split / gb.splits);
    const int total = (int)((int64_t)nkb * n_pairs * (split + 1) / gb.splits) - it0;
    const bool producer = warp == 1 && lane == 0, issuer = warp == 0 && lane == 0;
    const long long wlim = gb.wait_limit;
    auto load_stage = [&](int i) {
        const int s = i % STAGES;
        const int pr = (it0 + i) / nkb, kb = (it0 + i) % nkb;
        const uint32_t st = base + s * STAGE_BYTES;
        mbar_expect_tx(full0 + 8 * s, STAGE_BYTES + (MX ? 2 * SF_ATOM : 0));
        load_operand<A_MN>(st, &P.ta[pr], m0, kb * BKE, full0 + 8 * s);
        load_operand<B_MN>(st + TILE_BYTES, &P.tb[pr], n0, kb * BKE, full0 + 8 * s);
        if constexpr (MX) {
            const uint32_t sf = base + SF_OFF + s * 2 * SF_ATOM;
            bulk_copy_s(sf, P.sf_a + (m0 / BM) * P.sfa_tile + (int64_t)kb * SF_ATOM, SF_ATOM, full0 + 8 * s);
            bulk_copy_s(sf + SF_ATOM, P.sf_b + (n0 / BN) * P.sfb_tile + (int64_t)kb * SF_ATOM, SF_ATOM, full0 + 8 * s);
        }
    };

    // CTA-local setup overlaps the tail of the previous kernel (programmatic launch)
    if (producer) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done_bar, 1);
        tmem_slot[1] = 0;
        tmem_slot[2] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int q = 0; q < n_pairs; ++q) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.ta[q])) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&P.tb[q])) : "memory");
        }
    }
    // inputs are read, and tensor memory taken, only once the previous kernel has finished:
    // a kernel that holds tensor memory never waits on a later one
    SQ_KERNEL_ENTRY();
    const int pre = gb.stall ? 0 : (total < STAGES ? total : STAGES);
    if (producer)
        for (int i = 0; i < pre; ++i) load_stage(i);   // first stages: no slot to wait for
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    // the bias is first read in the epilogue, after the cluster barrier
    if (warp >= 2) {
        for (int j = threadIdx.x - 64; j < BN; j += 64) bias_s[j] = (p_bias && n0 + j < pN) ? p_bias[n0 + j] : 0.f;
        if (gb.ln)
            for (int j = threadIdx.x - 64; j < BN; j += 64) {
                g_s[j] = n0 + j < pN ? P.ln_g[n0 + j] : 0.f;
                beta_s[j] = n0 + j < pN ? P.ln_beta[n0 + j] : 0.f;
            }
    }

    if (producer) {
        int issued = pre;
        for (int i = pre; i < total && !gb.stall; ++i) {
            const int s = i % STAGES;
            if (!mbar_wait(empty0 + 8 * s, ((i / STAGES) - 1) & 1, gb.err, 1, wlim)) break;
            load_stage(i);
            issued = i + 1;
        }
        tmem_slot[1] = issued;
    } else if (issuer) {
        // MMA issuer
        constexpr uint32_t idesc = F8 ? idesc_e4m3(BM, BN, A_MN, B_MN) : idesc_bf16(BM, BN, A_MN, B_MN);
        if constexpr (MX) {
            int i = 0;
            for (; i < total; ++i) {
                const int s = i % STAGES;
                if (!mbar_wait(full0 + 8 * s, (i / STAGES) & 1, gb.err, 2, wlim)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = base + s * STAGE_BYTES;
                const uint32_t sf = base + SF_OFF + s * 2 * SF_ATOM;
                const uint32_t sfa_t = tmem + BN + 8 * s, sfb_t = sfa_t + 4;
                // scale copies and MMAs issued by one thread run in order
                sf_copy(sfa_t, sf_desc(sf));
                sf_copy(sfb_t, sf_desc(sf + SF_ATOM));
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    mma_mx(tmem, operand_desc<false>(st, kk), operand_desc<false>(st + TILE_BYTES, kk),
                           idesc_mx(BM, BN, (uint32_t)kk), sfa_t, sfb_t, (i > 0 || kk > 0) ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
            tmem_slot[2] = i;
            mma_commit(done_bar);
        } else {
            int i = 0;
            for (; i < total; ++i) {
                const int s = i % STAGES;
                if (!mbar_wait(full0 + 8 * s, (i / STAGES) & 1, gb.err, 2, wlim)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t st = base + s * STAGE_BYTES;
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    if constexpr (F8)
                        mma_e4m3(tmem, operand_desc<A_MN>(st, kk), operand_desc<B_MN>(st + TILE_BYTES, kk), idesc,
                                 (i > 0 || kk > 0) ? 1u : 0u);
                    else
                        mma_bf16(tmem, operand_desc<A_MN>(st, kk), operand_desc<B_MN>(st + TILE_BYTES, kk), idesc,
                                 (i > 0 || kk > 0) ? 1u : 0u);
                mma_commit(empty0 + 8 * s);
            }
            tmem_slot[2] = i;
            mma_commit(done_bar);
        }
    }
    __syncwarp();

    // epilogue, part 1: every thread moves its accumulator row from tensor memory into
    // shared memory (the operand stages are idle once the final commit has arrived)
    const bool have = mbar_wait(done_bar, 0, gb.err, 3, wlim);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* red = reinterpret_cast<float*>(smem);   // [BM][RED_LD]
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    {
        float* mine = red + (warp * 32 + lane) * RED_LD;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(trow + c0, r);
#pragma unroll
            for (int j = 0; j < 32; j += 4)
                *reinterpret_cast<float4*>(mine + c0 + j) =
                    make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                __uint_as_float(r[j + 3]));
        }
    }
    (void)have;   // a wait that gave up has set *err; the tile's values are then meaningless
    if (gb.ln) {
        // LayerNorm statistics of each output row over the cluster's column tiles: each CTA
        // sums its 128 columns of the row, the cluster exchanges the sums (rank order), then
        // the centred squares the same way
        __syncthreads();   // accumulator rows, bias, gain and shift staged
        // warp w takes rows w, w + 4, ... (8 at a time); lane l sums columns 4l .. 4l + 3 and a
        // butterfly adds the lanes, so a row's sum has the same order wherever the row sits
        // in the tile; the cluster exchange is then one row per thread
        const int cq = lane * 4;
        const int nvl = n0 + cq < pN ? min(4, pN - n0 - cq) : 0;
        // per-tensor FP8: the accumulator is scaled back before the bias, as in part 2
        const float sc = F8 == 1 ? __ldg(p_sa) * __ldg(p_sb) : 1.f;
        auto row_pass = [&](float* dst, bool centred) {
#pragma unroll 1
            for (int g = 0; g < BM / 4; g += 8) {
                float p[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int lr = warp + 4 * (g + i);
                    const float4 x = *reinterpret_cast<const float4*>(red + lr * RED_LD + cq);
                    const float mu = centred ? ln_mean_s[lr] : 0.f;
                    const float v0 = fmaf(x.x, sc, bias_s[cq]) - mu, v1 = fmaf(x.y, sc, bias_s[cq + 1]) - mu;
                    const float v2 = fmaf(x.z, sc, bias_s[cq + 2]) - mu, v3 = fmaf(x.w, sc, bias_s[cq + 3]) - mu;
                    const float w0 = centred ? v0 * v0 : v0, w1 = centred ? v1 * v1 : v1;
                    const float w2 = centred ? v2 * v2 : v2, w3 = centred ? v3 * v3 : v3;
                    p[i] = ((nvl > 0 ? w0 : 0.f) + (nvl > 1 ? w1 : 0.f)) + ((nvl > 2 ? w2 : 0.f) + (nvl > 3 ? w3 : 0.f));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int i = 0; i < 8; ++i) p[i] += __shfl_xor_sync(0xffffffffu, p[i], o);
                if (lane == 0)
#pragma unroll
                    for (int i = 0; i < 8; ++i) dst[warp + 4 * (g + i)] = p[i];
            }
        };
        const int lrow = warp * 32 + lane;
        row_pass(ln_s1, false);
        cluster_sync();
        {
            float tot = 0.f;
            for (int q = 0; q < tiles_n; ++q) tot += *map_rank(ln_s1 + lrow, q);
            ln_mean_s[lrow] = tot / (float)pN;
        }
        __syncthreads();
        row_pass(ln_s2, true);
        cluster_sync();
        {
            float var = 0.f;
            for (int q = 0; q < tiles_n; ++q) var += *map_rank(ln_s2 + lrow, q);
            const float rstd = 1.0f / sqrtf(var / (float)pN + P.ln_eps);
            ln_rstd_s[lrow] = rstd;
            if (crank == 0 && m0 + lrow < pM) {
                P.ln_mean[m0 + lrow] = ln_mean_s[lrow];
                P.ln_rstd[m0 + lrow] = rstd;
            }
        }
    }
    cluster_sync();
    // part 2: CTA `split` of the cluster finishes rows [split BM / S, (split + 1) BM / S),
    // adding the S partial tiles in rank order.  Warp w takes rows rb0 + w, rb0 + w + 4, ...,
    // 4 columns a lane, 8 rows at a time so that their loads are in flight together; each
    // output (mask, FP32 store or accumulate, BF16 store) then runs as its own loop.
    {
        const int S = gb.splits;
        const int rb0 = split * BM / S, rb1 = (split + 1) * BM / S;
        const int cq = lane * 4;
        const int col = n0 + cq;
        const int nv = col < pN ? min(4, pN - col) : 0;   // valid columns of this lane
        const int nrows = rb1 - rb0 > warp ? (rb1 - rb0 - warp + 3) / 4 : 0;
        const bool cvec = nv == 4 && (p_ldc & 3) == 0 && ((reinterpret_cast<uintptr_t>(p_c) & 15) == 0);
        const bool hvec = nv == 4 && (p_ldcbf & 3) == 0 && ((reinterpret_cast<uintptr_t>(p_cbf) & 7) == 0);
        const bool mvec = nv == 4 && (p_ldmask & 3) == 0 && ((reinterpret_cast<uintptr_t>(p_mask) & 15) == 0);
        float bias4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) bias4[j] = bias_s[cq + j];
        const float fp8_scale = F8 == 1 ? __ldg(p_sa) * __ldg(p_sb) : 1.f;
        const float* mine = red + (rb0 + warp) * RED_LD + cq;   // row g of this warp at mine + 4 g RED_LD
#pragma unroll 1
        for (int g0 = 0; g0 < nrows; g0 += 8) {
            const int cnt = min(8, nrows - g0);
            float4 acc[8];
            // BF16: rank order acc = bias + p_0 + p_1 + ...; FP8: acc = (p_0 + p_1 + ...) * scale + bias
            // (two ranks' loads in flight at a time)
#pragma unroll
            for (int i = 0; i < 8; ++i)
                acc[i] = F8 ? make_float4(0.f, 0.f, 0.f, 0.f) : make_float4(bias4[0], bias4[1], bias4[2], bias4[3]);
            int q = 0;
            for (; q + 1 < S; q += 2) {
                const float* s0 = map_rank(mine, q) + (size_t)g0 * 4 * RED_LD;
                const float* s1 = map_rank(mine, q + 1) + (size_t)g0 * 4 * RED_LD;
                float4 x0[8], x1[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    x0[i] = i < cnt ? *reinterpret_cast<const float4*>(s0 + (size_t)i * 4 * RED_LD) : make_float4(0.f, 0.f, 0.f, 0.f);
                    x1[i] = i < cnt ? *reinterpret_cast<const float4*>(s1 + (size_t)i * 4 * RED_LD) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc[i].x += x0[i].x; acc[i].y += x0[i].y; acc[i].z += x0[i].z; acc[i].w += x0[i].w;
                    acc[i].x += x1[i].x; acc[i].y += x1[i].y; acc[i].z += x1[i].z; acc[i].w += x1[i].w;
                }
            }
            if (q < S) {
                // (LayerNorm mode: one partial, this CTA's own, at its rank in the row cluster)
                const float* s0 = map_rank(mine, gb.ln ? crank : q) + (size_t)g0 * 4 * RED_LD;
                float4 x0[8];
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    x0[i] = i < cnt ? *reinterpret_cast<const float4*>(s0 + (size_t)i * 4 * RED_LD) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc[i].x += x0[i].x; acc[i].y += x0[i].y; acc[i].z += x0[i].z; acc[i].w += x0[i].w;
                }
            }
            if constexpr (F8) {
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    acc[i].x = fmaf(acc[i].x, fp8_scale, bias4[0]);
                    acc[i].y = fmaf(acc[i].y, fp8_scale, bias4[1]);
                    acc[i].z = fmaf(acc[i].z, fp8_scale, bias4[2]);
                    acc[i].w = fmaf(acc[i].w, fp8_scale, bias4[3]);
                }
            }
            const int row0 = m0 + rb0 + warp + 4 * g0;   // row of entry i: row0 + 4 i
            const int rows_ok = nv > 0 ? max(0, min(cnt, (pM - row0 + 3) / 4)) : 0;
            if (p_mask) {
                if (mvec) {
                    float4 mk[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) mk[i] = *reinterpret_cast<const float4*>(p_mask + (int64_t)(row0 + 4 * i) * p_ldmask + col);
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) {
                            if (!(mk[i].x > 0.f)) acc[i].x = 0.f;
                            if (!(mk[i].y > 0.f)) acc[i].y = 0.f;
                            if (!(mk[i].z > 0.f)) acc[i].z = 0.f;
                            if (!(mk[i].w > 0.f)) acc[i].w = 0.f;
                        }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) {
                            const float* mk = p_mask + (int64_t)(row0 + 4 * i) * p_ldmask + col;
                            if (!(mk[0] > 0.f)) acc[i].x = 0.f;
                            if (nv > 1 && !(mk[1] > 0.f)) acc[i].y = 0.f;
                            if (nv > 2 && !(mk[2] > 0.f)) acc[i].z = 0.f;
                            if (nv > 3 && !(mk[3] > 0.f)) acc[i].w = 0.f;
                        }
                }
            }
            if (p_c) {
                if (cvec) {
                    if (p_acc) {
                        float4 old[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (i < rows_ok) old[i] = *reinterpret_cast<const float4*>(p_c + (int64_t)(row0 + 4 * i) * p_ldc + col);
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (i < rows_ok) {
                                acc[i].x += old[i].x; acc[i].y += old[i].y; acc[i].z += old[i].z; acc[i].w += old[i].w;
                            }
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) *reinterpret_cast<float4*>(p_c + (int64_t)(row0 + 4 * i) * p_ldc + col) = acc[i];
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) {
                            float* dst = p_c + (int64_t)(row0 + 4 * i) * p_ldc + col;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float v = j == 0 ? acc[i].x : j == 1 ? acc[i].y : j == 2 ? acc[i].z : acc[i].w;
                                if (j < nv) dst[j] = p_acc ? dst[j] + v : v;
                            }
                        }
                }
            }
            if (p_cbf) {
                if (hvec) {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) {
                            __nv_bfloat162 lo = __floats2bfloat162_rn(acc[i].x, acc[i].y);
                            __nv_bfloat162 hi = __floats2bfloat162_rn(acc[i].z, acc[i].w);
                            uint2 u;
                            u.x = *reinterpret_cast<uint32_t*>(&lo);
                            u.y = *reinterpret_cast<uint32_t*>(&hi);
                            *reinterpret_cast<uint2*>(p_cbf + (int64_t)(row0 + 4 * i) * p_ldcbf + col) = u;
                        }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (i < rows_ok) {
                            __nv_bfloat16* dst = p_cbf + (int64_t)(row0 + 4 * i) * p_ldcbf + col;
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float v = j == 0 ? acc[i].x : j == 1 ? acc[i].y : j == 2 ? acc[i].z : acc[i].w;
                                if (j < nv) dst[j] = __float2bfloat16_rn(v);
                            }
                        }
                }
            }
            if (gb.ln) {
                // y = (x - mean) rstd g + beta, ReLU: FP32 and BF16 rows of the LayerNorm output
                float g4[4], b4[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) { g4[j] = g_s[cq + j]; b4[j] = beta_s[cq + j]; }
                const bool pvec = nv == 4 && (pN % 4) == 0;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (i < rows_ok) {
                        const int lr = rb0 + warp + 4 * (g0 + i);
                        const float mean = ln_mean_s[lr], rstd = ln_rstd_s[lr];
                        float y[4] = {acc[i].x, acc[i].y, acc[i].z, acc[i].w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            y[j] = (y[j] - mean) * rstd * g4[j] + b4[j];
                            if (P.ln_relu) y[j] = fmaxf(y[j], 0.f);
                        }
                        const int64_t off = (int64_t)(row0 + 4 * i) * pN + col;
                        if (pvec) {
                            *reinterpret_cast<float4*>(P.ln_post + off) = make_float4(y[0], y[1], y[2], y[3]);
                            if (P.ln_posth) {
                                __nv_bfloat162 lo = __floats2bfloat162_rn(y[0], y[1]);
                                __nv_bfloat162 hi = __floats2bfloat162_rn(y[2], y[3]);
                                uint2 u;
                                u.x = *reinterpret_cast<uint32_t*>(&lo);
                                u.y = *reinterpret_cast<uint32_t*>(&hi);
                                *reinterpret_cast<uint2*>(P.ln_posth + off) = u;
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (j < nv) {
                                    P.ln_post[off + j] = y[j];
                                    if (P.ln_posth) P.ln_posth[off + j] = __float2bfloat16_rn(y[j]);
                                }
                        }
                    }
            }
        }
    }
    // no CTA of the cluster leaves while another may still read its shared memory
    cluster_sync();
    // after a wait gave up: operand copies issued but never consumed still land in this
    // CTA's shared memory; wait for them (bounded) before the CTA can leave
    if (threadIdx.x == 0)
        for (int i = (int)tmem_slot[2]; i < (int)tmem_slot[1]; ++i)
            mbar_wait(full0 + 8 * (i % STAGES), (i / STAGES) & 1, gb.err, 4, wlim);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
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

// 2-D BF16 tensor map over a row-major matrix with `outer` rows of `inner` elements
// (row stride ld elements), 128-byte swizzle, zero fill outside the matrix.
bool make_map(CUtensorMap* m, const void* ptr, int64_t inner, int64_t outer, int64_t ld, int box_inner, int box_outer,
              bool fp8 = false) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int64_t es = fp8 ? 1 : 2;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * es) & 15) || inner < 1 || outer < 1) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * es)};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    std::memset(m, 0, sizeof(*m));
    return fn(m, fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims,
              strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool operand_map(CUtensorMap* m, const TcOperand& o, int mn_extent, int k_extent, bool fp8 = false) {
    if (fp8)          // K-major only: 128 elements (128 bytes) of K by 128 rows
        return !o.mn_major && make_map(m, o.ptr, k_extent, mn_extent, o.ld, 128, 128, true);
    if (o.mn_major)   // element (mn, k) at ptr[k * ld + mn]
        return make_map(m, o.ptr, mn_extent, k_extent, o.ld, 64, 64);
    return make_map(m, o.ptr, k_extent, mn_extent, o.ld, 64, 128);   // element (mn, k) at ptr[mn * ld + k]
}

template <bool A_MN, bool B_MN>
void set_smem_attr() {
    cudaFuncSetAttribute(tc_gemm_kernel<A_MN, B_MN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (!A_MN && !B_MN) {
        cudaFuncSetAttribute(tc_gemm_kernel<false, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
        cudaFuncSetAttribute(tc_gemm_kernel<false, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_BYTES_MX);
    }
}

}  // namespace

// K split of a launch (the cluster size): enough CTAs to cover the SMs when the launch
// has few output tiles, every problem keeping at least kMinSplitIters K slabs per split.
constexpr int kSplitTarget = 148, kMinSplitIters = 6, kMaxSplits = 8;

namespace {
int g_max_splits = 1;   // largest cluster the device can co-schedule for the GEMM kernel
}

int tc_max_cluster() { return g_max_splits; }

void tc_prepare() {
    set_smem_attr<false, false>();
    set_smem_attr<false, true>();
    set_smem_attr<true, true>();
    set_smem_attr<true, false>();
    encode_fn();
    static bool done = false;
    if (done) return;
    done = true;
    for (int S = 2; S <= kMaxSplits; S *= 2) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(S);
        cfg.blockDim = dim3(128);
        cfg.dynamicSmemBytes = SMEM_BYTES;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = S;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, tc_gemm_kernel<false, false>, &cfg) != cudaSuccess || n < 1) {
            cudaGetLastError();
            break;
        }
        g_max_splits = S;
    }
}

int launch_tc_gemm(const TcGemm* probs, int n_probs, int* err, cudaStream_t s, bool allow_split,
                   const TcWait* wait) {
    for (int base = 0; base < n_probs; base += kMaxProbs) {
        TcBatch gb;
        std::memset(&gb, 0, sizeof(gb));
        gb.n = std::min(kMaxProbs, n_probs - base);
        gb.err = err;
        gb.wait_limit = wait && wait->cycles > 0 ? wait->cycles : kWaitCycles;
        gb.stall = wait ? wait->stall : 0;
        int tiles = 0, min_iters = 1 << 30;
        bool a_mn = probs[base].a[0].mn_major, b_mn = probs[base].b[0].mn_major;
        const int f8k = probs[base].fp8;
        const bool f8 = f8k != 0;
        const bool ln = probs[base].ln_g != nullptr;
        for (int i = 0; i < gb.n; ++i) {
            const TcGemm& g = probs[base + i];
            TcProb& p = gb.p[i];
            if (g.a[0].mn_major != a_mn || g.b[0].mn_major != b_mn || g.n_pairs < 1 || g.n_pairs > 2) return -1;
            if (g.fp8 != f8k || f8k < 0 || f8k > 2 || (f8 && (g.n_pairs != 1 || a_mn || b_mn)) ||
                (f8k == 1 && (!g.scale_a || !g.scale_b)) || (f8k == 2 && (!g.sf_a || !g.sf_b)))
                return -1;
            if ((g.ln_g != nullptr) != ln ||
                (ln && (!g.ln_beta || !g.ln_post || !g.ln_mean || !g.ln_rstd || g.cbf || g.mask || g.accumulate ||
                        (g.N + BN - 1) / BN > g_max_splits || (g.N + BN - 1) / BN != (probs[base].N + BN - 1) / BN)))
                return -3;
            for (int q = 0; q < g.n_pairs; ++q) {
                if (!operand_map(&p.ta[q], g.a[q], g.M, g.K, f8)) return -2;
                if (!operand_map(&p.tb[q], g.b[q], g.N, g.K, f8)) return -2;
            }
            p.M = g.M; p.N = g.N; p.K = g.K; p.n_pairs = g.n_pairs;
            p.bias = g.bias; p.c = g.c; p.ldc = g.ldc; p.cbf = g.cbf; p.ldcbf = g.ldcbf;
            p.mask = g.mask; p.ldmask = g.ldmask; p.accumulate = g.accumulate;
            p.scale_a = g.scale_a; p.scale_b = g.scale_b;
            p.sf_a = g.sf_a; p.sf_b = g.sf_b;
            p.sfa_tile = (int64_t)((g.K + 127) / 128) * SF_ATOM;
            p.sfb_tile = p.sfa_tile;
            p.ln_g = g.ln_g; p.ln_beta = g.ln_beta; p.ln_post = g.ln_post; p.ln_posth = g.ln_posth;
            p.ln_mean = g.ln_mean; p.ln_rstd = g.ln_rstd; p.ln_eps = g.ln_eps; p.ln_relu = g.ln_relu;
            p.tiles_n = (g.N + BN - 1) / BN;
            p.tile_start = tiles;   // in tiles for now, scaled by the split below
            tiles += ((g.M + BM - 1) / BM) * p.tiles_n;
            const int bke = f8 ? 128 : BK;
            min_iters = std::min(min_iters, ((g.K + bke - 1) / bke) * g.n_pairs);
        }
        if (!tiles) continue;
        int S = std::min(std::min(g_max_splits, std::max(1, kSplitTarget / tiles)), min_iters / kMinSplitIters);
        S = allow_split && !ln ? std::max(S, 1) : 1;
        gb.splits = S;
        gb.ln = ln ? 1 : 0;
        for (int i = 0; i < gb.n; ++i) gb.p[i].tile_start *= S;
        // LayerNorm mode: one cluster per row block, its CTAs the block's column tiles
        const dim3 grid(tiles * S), cluster(ln ? gb.p[0].tiles_n : S);
        if (f8k == 2) launch_kc(tc_gemm_kernel<false, false, 2>, grid, dim3(128), SMEM_BYTES_MX, s, cluster, gb);
        else if (f8) launch_kc(tc_gemm_kernel<false, false, 1>, grid, dim3(128), SMEM_BYTES, s, cluster, gb);
        else if (!a_mn && !b_mn) launch_kc(tc_gemm_kernel<false, false>, grid, dim3(128), SMEM_BYTES, s, cluster, gb);
        else if (!a_mn && b_mn) launch_kc(tc_gemm_kernel<false, true>, grid, dim3(128), SMEM_BYTES, s, cluster, gb);
        else if (a_mn && b_mn) launch_kc(tc_gemm_kernel<true, true>, grid, dim3(128), SMEM_BYTES, s, cluster, gb);
        else launch_kc(tc_gemm_kernel<true, false>, grid, dim3(128), SMEM_BYTES, s, cluster, gb);
    }
    return 0;
}

// ---------------------------------------------------------------- FP8 quantisation
namespace {
struct QuantBatch { QuantItem it[kQuantMaxItems]; int n; float* part; };

// Whether row r of an item can be read 8 elements (16 bytes) at a time.
__device__ __forceinline__ bool quant_vec(const QuantItem& q) {
    return (q.cols % 8) == 0 && (q.src_ld % 8) == 0 && (reinterpret_cast<uintptr_t>(q.src) & 15) == 0 &&
           (q.dst_ld % 8) == 0 && (reinterpret_cast<uintptr_t>(q.dst) & 7) == 0;
}

// Pass 1: block b of item i takes rows b, b + kQuantBlocks, ... and writes max |x| to
// part[i * kQuantBlocks + b].
__global__ void __launch_bounds__(256) amax_kernel(QuantBatch qb) {
    SQ_KERNEL_ENTRY();
    const QuantItem& q = qb.it[blockIdx.y];
    const bool vec = quant_vec(q);
    float m = 0.f;
    for (int r = blockIdx.x; r < q.rows; r += kQuantBlocks) {
        const __nv_bfloat16* src = q.src + (int64_t)r * q.src_ld;
        if (vec) {
            for (int j = threadIdx.x * 8; j < q.cols; j += blockDim.x * 8) {
                const uint4 u = *reinterpret_cast<const uint4*>(src + j);
                const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = __bfloat1622float2(h[k]);
                    m = fmaxf(m, fmaxf(fabsf(f.x), fabsf(f.y)));
                }
            }
        } else {
            for (int j = threadIdx.x; j < q.cols; j += blockDim.x) m = fmaxf(m, fabsf(__bfloat162float(src[j])));
        }
    }
    m = warp_max(m);
    __shared__ float wm[8];
    if (threadIdx.x % 32 == 0) wm[threadIdx.x / 32] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = wm[0];
        for (int w = 1; w < (int)(blockDim.x / 32); ++w) t = fmaxf(t, wm[w]);
        qb.part[blockIdx.y * kQuantBlocks + blockIdx.x] = t;
    }
}

__device__ __forceinline__ uint8_t to_e4m3(float x) {
    return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// Pass 2: every block reduces the item's partial maxima, scale = amax / 448 (the largest
// finite e4m3 value), and writes e4m3(x / scale) for its rows; block 0 stores the scale.
__global__ void __launch_bounds__(256) quantize_kernel(QuantBatch qb) {
    SQ_KERNEL_ENTRY();
    const QuantItem& q = qb.it[blockIdx.y];
    __shared__ float sc;
    if (threadIdx.x < 32) {
        float m = 0.f;
        for (int b = threadIdx.x; b < kQuantBlocks; b += 32) m = fmaxf(m, qb.part[blockIdx.y * kQuantBlocks + b]);
        m = warp_max(m);
        if (threadIdx.x == 0) {
            const float s = m > 0.f ? m / 448.f : 1.f;
            sc = s;
            if (blockIdx.x == 0) *q.scale = s;
        }
    }
    __syncthreads();
    const float s = sc;
    const bool vec = quant_vec(q);
    for (int r = blockIdx.x; r < q.rows; r += kQuantBlocks) {
        const __nv_bfloat16* src = q.src + (int64_t)r * q.src_ld;
        uint8_t* dst = q.dst + (int64_t)r * q.dst_ld;
        if (vec) {
            for (int j = threadIdx.x * 8; j < q.dst_ld; j += blockDim.x * 8) {
                uint32_t w[2] = {0u, 0u};
                if (j < q.cols) {
                    const uint4 u = *reinterpret_cast<const uint4*>(src + j);
                    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 f = __bfloat1622float2(h[k]);
                        w[k / 2] |= ((uint32_t)to_e4m3(f.x / s) | ((uint32_t)to_e4m3(f.y / s) << 8)) << (16 * (k % 2));
                    }
                }
                *reinterpret_cast<uint2*>(dst + j) = make_uint2(w[0], w[1]);
            }
        } else {
            for (int j = threadIdx.x; j < q.dst_ld; j += blockDim.x)
                dst[j] = j < q.cols ? to_e4m3(__bfloat162float(src[j]) / s) : to_e4m3(0.f);
        }
    }
}
}  // namespace

int64_t quant_workspace() { return (int64_t)kQuantMaxItems * kQuantBlocks; }

void launch_quantize_e4m3(const QuantItem* items, int n, float* part, cudaStream_t s) {
    for (int base = 0; base < n; base += kQuantMaxItems) {
        QuantBatch qb;
        std::memset(&qb, 0, sizeof(qb));
        qb.n = std::min(kQuantMaxItems, n - base);
        qb.part = part;
        for (int i = 0; i < qb.n; ++i) qb.it[i] = items[base + i];
        launch_k(amax_kernel, dim3(kQuantBlocks, qb.n), dim3(256), 0, s, qb);
        launch_k(quantize_kernel, dim3(kQuantBlocks, qb.n), dim3(256), 0, s, qb);
    }
}

// ---------------------------------------------------------------- MX-FP8 quantisation
namespace {
// One warp per (row, 128-column slab) of an item: lane l takes columns 4l .. 4l + 3 of the
// slab, so a 32-element block is 8 lanes.  Block scale 2^e with e the smallest integer for
// which max|x| <= 448 2^e (448: the largest finite e4m3 value), stored as the UE8M0 byte
// e + 127 (e >= -127); codes e4m3(x 2^-e) rounded to nearest even.  Rows from the item's
// end to its last 128-row tile only get zero scale bytes.
__global__ void __launch_bounds__(256) quantize_mx_kernel(QuantBatch qb) {
    SQ_KERNEL_ENTRY();
    const QuantItem& q = qb.it[blockIdx.y];
    const int slabs = (q.cols + 127) / 128;
    const int tiles_r = (q.rows + 127) / 128;
    const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (w >= tiles_r * 128 * slabs) return;
    const int lane = threadIdx.x % 32;
    const int r = w / slabs, slab = w - r * slabs;
    const int j0 = slab * 128 + lane * 4;
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < q.rows) {
        const __nv_bfloat16* src = q.src + (int64_t)r * q.src_ld;
        if ((q.src_ld & 3) == 0 && (reinterpret_cast<uintptr_t>(q.src) & 7) == 0 && j0 + 3 < q.cols) {
            const uint2 u = *reinterpret_cast<const uint2*>(src + j0);
            const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
            const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
            v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
        } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
                if (j0 + t < q.cols) v[t] = __bfloat162float(src[j0 + t]);
        }
    }
    float m = fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3])));
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    // m = 1.f 2^(eb - 127): 448 = 1.75 2^8, so e = eb - 135 if the fraction is <= 0.75, else eb - 134
    const uint32_t bits = __float_as_uint(m);
    const int eb = (int)(bits >> 23);
    int e = eb == 0 ? -127 : ((bits & 0x7FFFFFu) <= 0x600000u ? eb - 135 : eb - 134);
    e = max(e, -127);
    if ((lane & 7) == 0) {
        const int rr = r & 127;
        q.sf[((int64_t)(r >> 7) * slabs + slab) * 512 + (rr & 31) * 16 + (rr >> 5) * 4 + (lane >> 3)] =
            r < q.rows ? (uint8_t)(e + 127) : (uint8_t)0;
    }
    if (r >= q.rows || j0 >= q.dst_ld) return;
    const float inv = __uint_as_float((uint32_t)(127 - e) << 23);   // 2^-e, exact
    const uint32_t c = (uint32_t)to_e4m3(v[0] * inv) | ((uint32_t)to_e4m3(v[1] * inv) << 8) |
                       ((uint32_t)to_e4m3(v[2] * inv) << 16) | ((uint32_t)to_e4m3(v[3] * inv) << 24);
    *reinterpret_cast<uint32_t*>(q.dst + (int64_t)r * q.dst_ld + j0) = c;
}
}  // namespace

int64_t mx_scale_bytes(int rows, int cols) { return (int64_t)((rows + 127) / 128) * ((cols + 127) / 128) * 512; }

void launch_quantize_mx(const QuantItem* items, int n, cudaStream_t s) {
    for (int base = 0; base < n; base += kQuantMaxItems) {
        QuantBatch qb;
        std::memset(&qb, 0, sizeof(qb));
        qb.n = std::min(kQuantMaxItems, n - base);
        int64_t warps = 0;
        for (int i = 0; i < qb.n; ++i) {
            qb.it[i] = items[base + i];
            warps = std::max<int64_t>(warps, (int64_t)((qb.it[i].rows + 127) / 128) * 128 * ((qb.it[i].cols + 127) / 128));
        }
        if (warps) launch_k(quantize_mx_kernel, dim3((unsigned)((warps + 7) / 8), qb.n), dim3(256), 0, s, qb);
    }
}

// ---------------------------------------------------------------- casts
namespace {
constexpr int kMaxCast = 48;
struct CastBatch { CastItem it[kMaxCast]; int row_start[kMaxCast + 1]; int n; };

// One CTA per (matrix, row): FP32 row -> BF16 row of a padded matrix (pad columns zero).
__global__ void cast_rows_kernel(CastBatch cb) {
    SQ_KERNEL_ENTRY();
    int i = 0;
    while (i + 1 < cb.n && (int)blockIdx.x >= cb.row_start[i + 1]) ++i;
    const CastItem& c = cb.it[i];
    const int r = blockIdx.x - cb.row_start[i];
    const float* src = c.src + (int64_t)r * c.src_ld;
    __nv_bfloat16* dst = c.dst + (int64_t)r * c.dst_ld;
    for (int j = threadIdx.x; j < c.dst_ld; j += blockDim.x)
        dst[j] = __float2bfloat16_rn(j < c.cols ? src[j] : 0.f);
}
}  // namespace

void launch_cast_rows(const CastItem* items, int n, cudaStream_t s) {
    for (int base = 0; base < n; base += kMaxCast) {
        CastBatch cb;
        cb.n = std::min(kMaxCast, n - base);
        int rows = 0;
        for (int i = 0; i < cb.n; ++i) {
            cb.it[i] = items[base + i];
            cb.row_start[i] = rows;
            rows += items[base + i].rows;
        }
        cb.row_start[cb.n] = rows;
        if (rows) launch_k(cast_rows_kernel, dim3(rows), dim3(128), 0, s, cb);
    }
}

}  // namespace sq
