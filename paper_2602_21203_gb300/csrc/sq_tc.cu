// BF16 tensor-core GEMM for sm_103a: D[M,N] (+)= sum_pairs A[M,K] B[N,K]^T, FP32
// accumulation in tensor memory.
//
// Per CTA one 128 x 128 output tile:
//   warp 0 / lane 0   TMA producer: 128B-swizzled 64-wide K slabs of A and B into a
//                     4-stage shared-memory ring (mbarrier complete_tx)
//   warp 1 / lane 0   MMA issuer: 4 x tcgen05.mma (K = 16 each) per slab, commit frees
//                     the slab, a final commit signals the accumulator
//   warps 0-3         epilogue: tcgen05.ld 32 lanes x 16 columns at a time, bias,
//                     optional ReLU mask, FP32 and/or BF16 stores
// Operands are K-major (K contiguous) or MN-major (M or N contiguous), so the
// forward X W^T, the data gradient dY W and the weight gradient dY^T X all run
// from the row-major buffers without transposed copies.
// Every wait is bounded: past kWaitCycles the waiting thread records an error
// code in *err and gives up; the tile is abandoned and TMEM is still freed.
#include "sq_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

namespace sq {

namespace {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 4;
constexpr int TILE_BYTES = BM * BK * 2;                // 16 KB per operand per stage
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256 + BN * 4;
constexpr long long kWaitCycles = 4000000000ll;        // ~2 s at 2 GHz
constexpr int kMaxProbs = 4;

struct TcProb {
    CUtensorMap ta[2];
    CUtensorMap tb[2];
    int M, N, K, n_pairs;
    int tiles_n, tile_start;
    const float* bias;
    float* c; int64_t ldc;
    __nv_bfloat16* cbf; int64_t ldcbf;
    const float* mask; int64_t ldmask;
    int accumulate;
};
struct TcBatch {
    TcProb p[kMaxProbs];
    int n;
    int* err;
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
// Bounded wait: false (and *err = code) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
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

template <bool A_MN, bool B_MN>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const __grid_constant__ TcBatch gb) {
    SQ_KERNEL_ENTRY();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 1);
    float* bias_s = reinterpret_cast<float*>(tmem_slot + 4);          // [BN]
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES), done_bar = smem_u32(bars + 2 * STAGES);

    int pi = 0;
    while (pi + 1 < gb.n && (int)blockIdx.x >= gb.p[pi + 1].tile_start) ++pi;
    const TcProb& P = gb.p[pi];
    const int t = blockIdx.x - P.tile_start;
    const int m0 = (t / P.tiles_n) * BM, n0 = (t % P.tiles_n) * BN;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int j = threadIdx.x; j < BN; j += blockDim.x) bias_s[j] = (P.bias && n0 + j < P.N) ? P.bias[n0 + j] : 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t base = smem_u32(smem);
    const int nkb = (P.K + BK - 1) / BK;
    const int total = nkb * P.n_pairs;

    if (warp == 0 && lane == 0) {
        // producer
        for (int i = 0; i < total; ++i) {
            const int s = i % STAGES;
            if (i >= STAGES && !mbar_wait(empty0 + 8 * s, ((i / STAGES) - 1) & 1, gb.err, 1)) break;
            const int pr = i / nkb, kb = i % nkb;
            const uint32_t st = base + s * STAGE_BYTES;
            mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
            load_operand<A_MN>(st, &P.ta[pr], m0, kb * BK, full0 + 8 * s);
            load_operand<B_MN>(st + TILE_BYTES, &P.tb[pr], n0, kb * BK, full0 + 8 * s);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16(BM, BN, A_MN, B_MN);
        bool ok = true;
        for (int i = 0; i < total; ++i) {
            const int s = i % STAGES;
            if (!mbar_wait(full0 + 8 * s, (i / STAGES) & 1, gb.err, 2)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = base + s * STAGE_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, operand_desc<A_MN>(st, kk), operand_desc<B_MN>(st + TILE_BYTES, kk), idesc,
                         (i > 0 || kk > 0) ? 1u : 0u);
            mma_commit(empty0 + 8 * s);
        }
        mma_commit(done_bar);
        (void)ok;
    }
    __syncwarp();

    // epilogue
    const bool have = mbar_wait(done_bar, 0, gb.err, 3);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const bool row_ok = have && row < P.M;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        tmem_ld32(trow + c0, r);
        if (!row_ok || n0 + c0 >= P.N) continue;
        float v[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + bias_s[c0 + j];
        if (P.mask) {
            const float* mk = P.mask + (int64_t)row * P.ldmask + n0 + c0;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (n0 + c0 + j < P.N && !(mk[j] > 0.f)) v[j] = 0.f;
        }
        const bool full = n0 + c0 + 32 <= P.N;
        if (P.c) {
            float* dst = P.c + (int64_t)row * P.ldc + n0 + c0;
            if (full && !P.accumulate && ((reinterpret_cast<uintptr_t>(dst) & 15) == 0)) {
#pragma unroll
                for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
            } else {
                for (int j = 0; j < 32; ++j)
                    if (n0 + c0 + j < P.N) dst[j] = P.accumulate ? dst[j] + v[j] : v[j];
            }
        }
        if (P.cbf) {
            __nv_bfloat16* dst = P.cbf + (int64_t)row * P.ldcbf + n0 + c0;
            for (int j = 0; j < 32; ++j)
                if (n0 + c0 + j < P.N) dst[j] = __float2bfloat16_rn(v[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
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
bool make_map(CUtensorMap* m, const void* ptr, int64_t inner, int64_t outer, int64_t ld, int box_inner, int box_outer) {
    auto fn = encode_fn();
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(ptr) & 15) || ((ld * 2) & 15) || inner < 1 || outer < 1) return false;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estr[2] = {1, 1};
    std::memset(m, 0, sizeof(*m));
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool operand_map(CUtensorMap* m, const TcOperand& o, int mn_extent, int k_extent) {
    if (o.mn_major)   // element (mn, k) at ptr[k * ld + mn]
        return make_map(m, o.ptr, mn_extent, k_extent, o.ld, 64, 64);
    return make_map(m, o.ptr, k_extent, mn_extent, o.ld, 64, 128);   // element (mn, k) at ptr[mn * ld + k]
}

template <bool A_MN, bool B_MN>
void set_smem_attr() {
    cudaFuncSetAttribute(tc_gemm_kernel<A_MN, B_MN>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

}  // namespace

void tc_prepare() {
    set_smem_attr<false, false>();
    set_smem_attr<false, true>();
    set_smem_attr<true, true>();
    set_smem_attr<true, false>();
    encode_fn();
}

int launch_tc_gemm(const TcGemm* probs, int n_probs, int* err, cudaStream_t s) {
    for (int base = 0; base < n_probs; base += kMaxProbs) {
        TcBatch gb;
        std::memset(&gb, 0, sizeof(gb));
        gb.n = std::min(kMaxProbs, n_probs - base);
        gb.err = err;
        int tiles = 0;
        bool a_mn = probs[base].a[0].mn_major, b_mn = probs[base].b[0].mn_major;
        for (int i = 0; i < gb.n; ++i) {
            const TcGemm& g = probs[base + i];
            TcProb& p = gb.p[i];
            if (g.a[0].mn_major != a_mn || g.b[0].mn_major != b_mn || g.n_pairs < 1 || g.n_pairs > 2) return -1;
            for (int q = 0; q < g.n_pairs; ++q) {
                if (!operand_map(&p.ta[q], g.a[q], g.M, g.K)) return -2;
                if (!operand_map(&p.tb[q], g.b[q], g.N, g.K)) return -2;
            }
            p.M = g.M; p.N = g.N; p.K = g.K; p.n_pairs = g.n_pairs;
            p.bias = g.bias; p.c = g.c; p.ldc = g.ldc; p.cbf = g.cbf; p.ldcbf = g.ldcbf;
            p.mask = g.mask; p.ldmask = g.ldmask; p.accumulate = g.accumulate;
            p.tiles_n = (g.N + BN - 1) / BN;
            p.tile_start = tiles;
            tiles += ((g.M + BM - 1) / BM) * p.tiles_n;
        }
        if (!tiles) continue;
        if (!a_mn && !b_mn) launch_k(tc_gemm_kernel<false, false>, dim3(tiles), dim3(128), SMEM_BYTES, s, gb);
        else if (!a_mn && b_mn) launch_k(tc_gemm_kernel<false, true>, dim3(tiles), dim3(128), SMEM_BYTES, s, gb);
        else if (a_mn && b_mn) launch_k(tc_gemm_kernel<true, true>, dim3(tiles), dim3(128), SMEM_BYTES, s, gb);
        else launch_k(tc_gemm_kernel<true, false>, dim3(tiles), dim3(128), SMEM_BYTES, s, gb);
    }
    return 0;
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
