// Tensor-core (tcgen05) 3x3 convolutions for 32 -> 32 channels, stride 1: the
// forward, the data gradient and the weight gradient of the encoder's inner layers.
//
// Activation format between these layers: "padded HWC" BF16 - per image (H+4) x (W+4)
// rows of 32 channels (64 B), the valid pixels at rows (y+2)(W+4) + x+2, zeros
// elsewhere.  On a virtual output grid that keeps the input's row width Wp, output
// pixel q = oy Wp + ox reads input row q + origin(ky, kx), so each of the nine
// taps is the same shared-memory image seen from a shifted start row: the A
// operand of tap (ky, kx) is a descriptor whose start address moves by
// origin(ky, kx) rows, with no im2col copy.  Columns ox >= out_w of the virtual
// grid are computed and discarded.
//
// Shared-memory operand layout: the canonical no-swizzle K-major layout with
// channels split into 4 planes of 8 (16 B per pixel row per plane): element
// (row r, channel c) at (c / 8) * PLANE + r * 16 + (c % 8) * 2.  Any start row is a
// valid descriptor start.  TMA loads each plane of an image box by box.
#include "sq_kernels.cuh"
#include "sq_tc.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

namespace sq {

namespace {

constexpr long long kWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
constexpr int kCh = 32;                            // channels in and out
constexpr int kWBytes = 9 * kCh * kCh * 2;         // 18432 B: one layer's filter in BF16

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
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"((uint64_t)src), "r"(bytes), "r"(bar)
                 : "memory");
}
// No-swizzle shared-memory descriptor (core matrices of 8 rows x 16 B).  K-major operand:
// lbo = stride between core matrices along K, sbo = along M/N.  MN-major operand:
// lbo = stride along K, sbo = along M/N (checked against the oracle's convolution).
__device__ __forceinline__ uint64_t plain_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
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
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t cols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols));
}

// ---------------------------------------------------------------- forward / data gradient
struct ConvArgs {
    CUtensorMap tin;                 // input planes: dims {8, 4, nimg * in_rows}
    const __nv_bfloat16* w;          // filter, layout [tap][plane][out ch][8]
    int nimg, in_rows, Wp, out_h, out_w, off0, n_tiles, load_rows, tmem_cols;
    const float* bias;               // forward: bias[out ch]
    int relu;
    const __nv_bfloat16* mask;       // data gradient: padded-HWC activation of the layer below (mask > 0)
    __nv_bfloat16* out_phwc;         // padded-HWC output (grid width out_w + 4), interior written
    float* out_chw;                  // optional CHW FP32 output [nimg, 32, out_h, out_w]
    __nv_bfloat16* out_chw_bf;       // optional CHW BF16 copy
    int* err;
};

// Persistent and warp-specialised: CTA c takes images c, c + gridDim.x, ...  Warp 0 (one
// lane) loads the filter once and each image by TMA into one of two shared-memory
// buffers; warp 1 (one lane) owns the tensor memory and issues each image's MMAs into
// one of two accumulators; warps 2..5 (TMEM lane quarters 2, 3, 0, 1) drain an
// accumulator (bias, ReLU, mask, stores) while the next image is loaded and multiplied.
// Barriers: full/empty per image buffer, tfull/tempty per accumulator; every wait is
// bounded and a wait that gives up records its code in *err and stops that role.
constexpr int kConvThreads = 192;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__global__ void __launch_bounds__(kConvThreads) conv32_tc_kernel(const __grid_constant__ ConvArgs a) {
    SQ_KERNEL_ENTRY();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t plane = (uint32_t)a.load_rows * 16;
    const uint32_t ibytes = 4 * plane;
    uint8_t* w_s = smem + 2 * ibytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(w_s + kWBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 10);
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + 2), tfull0 = smem_u32(bars + 4),
                   tempty0 = smem_u32(bars + 6), done_bar = smem_u32(bars + 8);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int n_local = (int)blockIdx.x < a.nimg ? (a.nimg - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t cols = 2 * (uint32_t)a.tmem_cols;

    if (warp == 1) tmem_alloc(smem_u32(tmem_slot), cols);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(full0 + 8 * b, 1);
            mbar_init(empty0 + 8 * b, 1);
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, 4);   // one arrival per epilogue warp
        }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t w_u = smem_u32(w_s);

    if (warp == 0) {
        if (lane == 0) {
            // producer: the filter with the first image, then image i into buffer i % 2 once
            // the MMAs of image i - 2 have read it
            int issued = 0;
            for (int i = 0; i < n_local; ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(empty0 + 8 * b, ((i - 2) >> 1) & 1, a.err, 13)) break;
                const int img = (int)blockIdx.x + i * (int)gridDim.x;
                const uint32_t dst = smem_u32(smem) + b * ibytes;
                mbar_expect_tx(full0 + 8 * b, ibytes + (i == 0 ? (uint32_t)kWBytes : 0u));
                for (int c = 0; c < 4; ++c)
                    for (int bb = 0; bb < a.load_rows / 128; ++bb)
                        tma_load_3d(dst + c * plane + bb * 2048, &a.tin, 0, c, img * a.in_rows + bb * 128, full0 + 8 * b);
                if (i == 0) bulk_load(w_u, a.w, kWBytes, full0);
                issued = i + 1;
            }
            // the last loads have landed before the CTA can finish (immediate unless a consumer gave up)
            for (int i = issued - 2 < 0 ? 0 : issued - 2; i < issued; ++i)
                mbar_wait(full0 + 8 * (i & 1), (i >> 1) & 1, a.err, 14);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(128, kCh, false, false);
            for (int i = 0; i < n_local; ++i) {
                const int b = i & 1;
                if (!mbar_wait(full0 + 8 * b, (i >> 1) & 1, a.err, 11)) break;
                if (i >= 2 && !mbar_wait(tempty0 + 8 * b, ((i - 2) >> 1) & 1, a.err, 15)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t img_u = smem_u32(smem) + b * ibytes;
                const uint32_t acc = tmem + b * (uint32_t)a.tmem_cols;
                for (int t = 0; t < a.n_tiles; ++t)
                    for (int tap = 0; tap < 9; ++tap) {
                        const int row0 = t * 128 + a.off0 + (tap / 3) * a.Wp + (tap % 3);
                        for (int kc = 0; kc < 2; ++kc) {
                            const uint64_t ad = plain_desc(img_u + 2 * kc * plane + row0 * 16, plane, 128);
                            const uint64_t bd = plain_desc(w_u + tap * 2048 + 2 * kc * 512, 512, 128);
                            mma_bf16(acc + t * kCh, ad, bd, idesc, (tap | kc) ? 1u : 0u);
                        }
                    }
                mma_commit(empty0 + 8 * b);
                mma_commit(tfull0 + 8 * b);
            }
            // every MMA this CTA issued has completed before the tensor memory is freed
            mma_commit(done_bar);
            mbar_wait(done_bar, 0, a.err, 16);
        }
        __syncwarp();
    } else {
        const int quarter = warp % 4;
        const int wpo = a.out_w + 4;
        const int64_t out_img = (int64_t)(a.out_h + 4) * wpo * kCh;
        // a thread's output pixel in each tile, and the bias, are the same for every image
        int oy_t[4], ox_t[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int q = t * 128 + quarter * 32 + lane;
            oy_t[t] = q / a.Wp;
            ox_t[t] = q - oy_t[t] * a.Wp;
        }
        float bias_r[kCh];
#pragma unroll
        for (int j = 0; j < kCh; ++j) bias_r[j] = a.bias ? a.bias[j] : 0.f;
        for (int i = 0; i < n_local; ++i) {
            const int b = i & 1;
            const bool have = mbar_wait(tfull0 + 8 * b, (i >> 1) & 1, a.err, 12);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int img = (int)blockIdx.x + i * (int)gridDim.x;
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                if (t >= a.n_tiles || !have) break;
                uint32_t r0[16], r1[16];
                const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + b * (uint32_t)a.tmem_cols + t * kCh;
                tmem_ld16(taddr, r0);
                tmem_ld16(taddr + 16, r1);
                const int oy = oy_t[t], ox = ox_t[t];
                if (oy >= a.out_h || ox >= a.out_w) continue;
                float v[kCh];
#pragma unroll
                for (int j = 0; j < 16; ++j) { v[j] = __uint_as_float(r0[j]); v[16 + j] = __uint_as_float(r1[j]); }
                const int64_t prow = ((int64_t)(oy + 2) * wpo + ox + 2) * kCh;
                if (a.bias) {
#pragma unroll
                    for (int j = 0; j < kCh; ++j) v[j] += bias_r[j];
                }
                if (a.relu) {
#pragma unroll
                    for (int j = 0; j < kCh; ++j) v[j] = fmaxf(v[j], 0.f);
                }
                if (a.mask) {
                    const uint4* mk = reinterpret_cast<const uint4*>(a.mask + (int64_t)img * out_img + prow);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const uint4 m4 = mk[c];
                        const __nv_bfloat16* mb = reinterpret_cast<const __nv_bfloat16*>(&m4);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (!(__bfloat162float(mb[j]) > 0.f)) v[c * 8 + j] = 0.f;
                    }
                }
                if (a.out_phwc) {
                    uint4* dst = reinterpret_cast<uint4*>(a.out_phwc + (int64_t)img * out_img + prow);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) hb[j] = __float2bfloat16_rn(v[c * 8 + j]);
                        dst[c] = *reinterpret_cast<const uint4*>(hb);
                    }
                }
                if (a.out_chw || a.out_chw_bf) {
                    const int64_t plane_px = (int64_t)a.out_h * a.out_w;
                    const int64_t base = (int64_t)img * kCh * plane_px + (int64_t)oy * a.out_w + ox;
#pragma unroll
                    for (int j = 0; j < kCh; ++j) {
                        if (a.out_chw) a.out_chw[base + j * plane_px] = v[j];
                        if (a.out_chw_bf) a.out_chw_bf[base + j * plane_px] = __float2bfloat16_rn(v[j]);
                    }
                }
            }
            // this warp's lanes of the accumulator are read: it may take the image after next
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty0 + 8 * b);
            if (!have) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_dealloc(tmem, cols);
    }
}

// ---------------------------------------------------------------- weight gradient
// D_tap[co, ci] += sum_q dy[q, co] x[q + origin(tap), ci] over the virtual grid of
// the input's padded row width (dy = 0 outside the valid outputs), origin(ky, kx) =
// (2 + ky) Wp + 2 + kx.  A = dy^T, MN-major: the threads copy dy's 16-byte pixel chunks
// unchanged into four channel planes of kq pixel rows (no transpose); rows 32..127 of the
// 128-row MMA read whatever follows in shared memory (inside the allocation: the dy
// buffers come first) and land in accumulator rows that are never read.  B stacks the
// three horizontal taps: shared memory holds
// twelve slots (kx, channel plane), slot (kx, p) = rows origin(0, kx) + [0, slot_rows)
// of plane p, SLOT apart, so one MN-major operand of N = 96 (kx, ci) starting ky Wp
// rows into every slot covers taps (ky, 0..2); its accumulator columns ky 96 + kx 32 +
// ci are tap 32 + ci.  Three MMAs per 16 pixels instead of nine.
struct WgradArgs {
    CUtensorMap tin;                 // layer input planes, dims {8, 4, nimg * in_rows}, box {8, 1, box_rows}
    const __nv_bfloat16* dy;         // padded-HWC gradient at the layer's pre-activation (grid out_w + 4)
    int nimg, in_rows, Wp, out_h, out_w, kq, slot_rows, box_rows, per_cta;
    float* work;                     // [ctas, 32, 289]: partial dW (co, ci*9 + tap) and db (col 288)
    int* err;
};

constexpr int kDyBytesMax = 32768;
constexpr uint32_t kWgTileBytes = kCh * (kCh * 9 + 1) * 4;   // the partial tile, staged at the end
// bytes from the (1024-aligned) start of shared memory to the barriers: the operand buffers,
// at least as many as the partial tile that reuses them
__host__ __device__ inline uint32_t wgrad_operand_bytes(uint32_t xbytes, uint32_t dybytes) {
    const uint32_t ops = 2 * xbytes + 2 * dybytes;
    return ops > kWgTileBytes ? ops : kWgTileBytes;
}

__global__ void __launch_bounds__(128) wgrad32_tc_kernel(const __grid_constant__ WgradArgs a) {
    SQ_KERNEL_ENTRY();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t slot = (uint32_t)a.slot_rows * 16;
    const uint32_t xbytes = 12 * slot;
    const uint32_t dplane = (uint32_t)a.kq * 16;                 // one 8-channel plane of dy
    const uint32_t dybytes = 4 * dplane;
    uint8_t* ds[2] = {smem, smem + dybytes};
    uint8_t* xs[2] = {smem + 2 * dybytes, smem + 2 * dybytes + xbytes};
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + wgrad_operand_bytes(xbytes, dybytes));
    float* red = reinterpret_cast<float*>(bars + 8);             // [128][8] bias partials
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(red + 128 * 8);
    const uint32_t tma_bar[2] = {smem_u32(bars), smem_u32(bars + 1)};
    const uint32_t mma_bar[2] = {smem_u32(bars + 2), smem_u32(bars + 3)};
    const uint32_t done_bar = smem_u32(bars + 4);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int i0 = blockIdx.x * a.per_cta, i1 = min(a.nimg, i0 + a.per_cta);

    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), 512);
    if (threadIdx.x == 32) {
        for (int b = 0; b < 2; ++b) { mbar_init(tma_bar[b], 1); mbar_init(mma_bar[b], 1); }
        mbar_init(done_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int wpo = a.out_w + 4;
    const int64_t dy_img = (int64_t)(a.out_h + 4) * wpo * kCh;
    float bsum[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int cc = threadIdx.x % 4;         // the 8-channel chunk this thread stages
    bool ok = true;
    constexpr uint32_t idesc = idesc_bf16(128, 3 * kCh, true, true);

    // Every thread runs every iteration (the barriers inside must match); a wait that
    // gives up only records the error and stops further MMA issue.
    for (int i = i0; i < i1; ++i) {
        const int li = i - i0, b = li & 1;
        if (li >= 2 && !mbar_wait(mma_bar[b], ((li - 2) >> 1) & 1, a.err, 21)) ok = false;
        if (threadIdx.x == 0 && ok) {
            const int boxes = a.slot_rows / a.box_rows;
            const int row0 = i * a.in_rows + 2 * a.Wp + 2;
            mbar_expect_tx(tma_bar[b], xbytes);
            for (int kx = 0; kx < 3; ++kx)
                for (int c = 0; c < 4; ++c)
                    for (int bb = 0; bb < boxes; ++bb)
                        tma_load_3d(smem_u32(xs[b]) + (kx * 4 + c) * slot + bb * a.box_rows * 16, &a.tin, 0, c,
                                    row0 + kx + bb * a.box_rows, tma_bar[b]);
        }
        // stage dy: the 16-byte chunk of channels 8 cc .. 8 cc + 7 of pixel q at cc PLANE + 16 q
        // (zero outside the valid outputs); a thread's loads for eight pixels are issued
        // before any of them is stored
        uint8_t* d = ds[b];
        for (int j0 = threadIdx.x; j0 < a.kq * 4; j0 += 8 * blockDim.x) {
            uint4 v4[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                const int q = j >> 2;
                const int oy = q / a.Wp, ox = q - (q / a.Wp) * a.Wp;
                v4[u] = make_uint4(0, 0, 0, 0);
                if (j < a.kq * 4 && oy < a.out_h && ox < a.out_w)
                    v4[u] = *reinterpret_cast<const uint4*>(a.dy + (int64_t)i * dy_img +
                                                            ((int64_t)(oy + 2) * wpo + ox + 2) * kCh + cc * 8);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u * blockDim.x;
                if (j >= a.kq * 4) break;
                const int q = j >> 2;
                const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&v4[u]);
                *reinterpret_cast<uint4*>(d + cc * dplane + q * 16) = v4[u];
#pragma unroll
                for (int k = 0; k < 8; ++k) bsum[k] += __bfloat162float(hv[k]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 32) {
            if (!ok || !mbar_wait(tma_bar[b], (li >> 1) & 1, a.err, 22)) {
                ok = false;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // descriptors built once; each MMA adds its start offset in 16-byte units
                // (shared-memory addresses stay below 2^18: the 14-bit field never carries)
                const uint64_t a0 = plain_desc(smem_u32(ds[b]), 128, dplane);
                const uint64_t b0 = plain_desc(smem_u32(xs[b]), 128, slot);
                for (int k = 0; k < a.kq / 16; ++k)
#pragma unroll
                    for (int ky = 0; ky < 3; ++ky)
                        mma_bf16(tmem + ky * 3 * kCh, a0 + (uint64_t)(k * 16), b0 + (uint64_t)(k * 16 + ky * a.Wp),
                                 idesc, (i > i0 || k > 0) ? 1u : 0u);
            }
            mma_commit(mma_bar[b]);
        }
        __syncwarp();
    }
    if (threadIdx.x == 32) mma_commit(done_bar);
    __syncwarp();
    const bool have = mbar_wait(done_bar, 0, a.err, 23) && ok && i1 > i0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // bias partials: reduce the 32 threads of each chunk in a fixed order.  The partial
    // tile [co][ci * 9 + tap | bias] is assembled in shared memory (the operand buffers are
    // idle once the last MMA has completed) and stored by all threads, coalesced.
#pragma unroll
    for (int k = 0; k < 8; ++k) red[threadIdx.x * 8 + k] = bsum[k];
    __syncthreads();
    constexpr int NW = kCh * 9 + 1;
    float* tile = reinterpret_cast<float*>(smem);   // [kCh][NW]
    if (threadIdx.x < kCh) {
        const int co = threadIdx.x;
        float s = 0.f;
        for (int t = co / 8; t < 128; t += 4) s += red[t * 8 + (co % 8)];
        tile[co * NW + kCh * 9] = s;
    }
    if (warp == 0) {
        const int co = lane;
        for (int tap = 0; tap < 9; ++tap) {
            uint32_t r0[16], r1[16];
            tmem_ld16(tmem + tap * kCh, r0);
            tmem_ld16(tmem + tap * kCh + 16, r1);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                tile[co * NW + j * 9 + tap] = have ? __uint_as_float(r0[j]) : 0.f;
                tile[co * NW + (16 + j) * 9 + tap] = have ? __uint_as_float(r1[j]) : 0.f;
            }
        }
    }
    __syncthreads();
    float* out = a.work + (int64_t)blockIdx.x * kCh * NW;
    for (int e = threadIdx.x; e < kCh * NW; e += blockDim.x) out[e] = tile[e];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_dealloc(tmem, 512);
    }
}

// 32 elements per block and 8 groups of CTAs: group g adds CTA partials g, g + 8, ... in
// increasing order, then the group sums are added in group order (a fixed order, so
// partials reduced once per whole batch or after chunks give the same bits).
constexpr int kRed32Groups = 8;
__global__ void __launch_bounds__(32 * kRed32Groups) wgrad32_reduce_kernel(const float* __restrict__ work, int splits,
                                                                            float* __restrict__ dw,
                                                                            float* __restrict__ db) {
    SQ_KERNEL_ENTRY();
    constexpr int N = kCh * 9 + 1;
    constexpr int tot = kCh * N;
    __shared__ float part[kRed32Groups][33];
    const int tx = threadIdx.x % 32, g = threadIdx.x / 32;
    const int e = blockIdx.x * 32 + tx;
    float s = 0.f;
    if (e < tot) {
        int z = g;
        for (; z + 3 * kRed32Groups < splits; z += 4 * kRed32Groups) {   // four partials' loads in flight
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = work[(int64_t)(z + u * kRed32Groups) * tot + e];
#pragma unroll
            for (int u = 0; u < 4; ++u) s += v[u];
        }
        for (; z < splits; z += kRed32Groups) s += work[(int64_t)z * tot + e];
    }
    part[g][tx] = s;
    __syncthreads();
    if (g != 0 || e >= tot) return;
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < kRed32Groups; ++k) a += part[k][tx];
    const int co = e / N, col = e - co * N;
    if (col == N - 1) db[co] = a;
    else dw[co * (N - 1) + col] = a;
}

// ---------------------------------------------------------------- first layer straight to padded HWC
// The encoder's first convolution (few input channels, any stride, 32 outputs) for the
// tensor-core path: one thread per output pixel holds its 32 channels, the filter and bias
// are broadcast from shared memory, and the ReLU output goes straight to the padded-HWC
// BF16 image the next (tensor-core) layer reads.  Each output is accumulated over
// k = (ci, ky, kx) in order with fused multiply-adds, then the bias is added: the same
// arithmetic as the CUDA-core implicit GEMM followed by the layout conversion.
__global__ void __launch_bounds__(256) conv0_phwc_kernel(ConvShape sh, const float* __restrict__ x,
                                                         const float* __restrict__ w, const float* __restrict__ bias,
                                                         __nv_bfloat16* __restrict__ out) {
    SQ_KERNEL_ENTRY();
    extern __shared__ float w_s[];   // [K][32] then bias [32]
    const int K = sh.Cin * 9;
    for (int e = threadIdx.x; e < K * kCh; e += blockDim.x) {
        const int k = e / kCh, co = e % kCh;
        w_s[e] = w[(int64_t)co * K + k];
    }
    if (threadIdx.x < kCh) w_s[K * kCh + threadIdx.x] = bias[threadIdx.x];
    __syncthreads();
    // two output pixels per thread (blockDim apart, so each half stays coalesced): every
    // weight read from shared memory feeds both
    const int64_t npix = (int64_t)sh.nimg * sh.OH * sh.OW;
    const int64_t p0 = (int64_t)blockIdx.x * 2 * blockDim.x + threadIdx.x;
    if (p0 >= npix) return;
    const int64_t pp[2] = {p0, p0 + blockDim.x};
    const bool has1 = pp[1] < npix;
    const float* xb[2];
    __nv_bfloat16* dst[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int64_t p = has1 || h == 0 ? pp[h] : pp[0];
        const int img = (int)(p / (sh.OH * sh.OW));
        const int rem = (int)(p - (int64_t)img * sh.OH * sh.OW);
        const int oy = rem / sh.OW, ox = rem - (rem / sh.OW) * sh.OW;
        xb[h] = x + (int64_t)img * sh.x_img_stride + (int64_t)(oy * sh.stride) * sh.W + ox * sh.stride;
        dst[h] = out + ((int64_t)img * (sh.OH + 4) * (sh.OW + 4) + (int64_t)(oy + 2) * (sh.OW + 4) + ox + 2) * kCh;
    }
    float acc0[kCh], acc1[kCh];
#pragma unroll
    for (int co = 0; co < kCh; ++co) { acc0[co] = 0.f; acc1[co] = 0.f; }
    for (int ci = 0; ci < sh.Cin; ++ci)
#pragma unroll
        for (int t = 0; t < 9; ++t) {
            const int64_t off = (int64_t)ci * sh.H * sh.W + (t / 3) * sh.W + (t % 3);
            const float xv0 = __ldg(xb[0] + off), xv1 = __ldg(xb[1] + off);
            const float* wk = w_s + (ci * 9 + t) * kCh;
#pragma unroll
            for (int co = 0; co < kCh; ++co) {
                const float wv = wk[co];
                acc0[co] = fmaf(xv0, wv, acc0[co]);
                acc1[co] = fmaf(xv1, wv, acc1[co]);
            }
        }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (h == 1 && !has1) break;
        __align__(16) __nv_bfloat16 hb[kCh];
#pragma unroll
        for (int co = 0; co < kCh; ++co) {
            float v = (h == 0 ? acc0[co] : acc1[co]) + w_s[K * kCh + co];
            if (!(v > 0.f)) v = 0.f;
            hb[co] = __float2bfloat16_rn(v);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) reinterpret_cast<uint4*>(dst[h])[c] = reinterpret_cast<const uint4*>(hb)[c];
    }
}


// ---------------------------------------------------------------- first layer on tensor cores
// The first encoder layer (few input channels, any stride, 32 outputs) as an implicit GEMM
// on tcgen05: D[pixel, co] = sum_k A[pixel, k] W[co, k] with k = (ci, ky, kx) in the
// filter's own order, K = 9 Cin zero-padded to 8 PL.  A 128-pixel tile of A is gathered
// by the threads (thread r: pixel r, its K inputs rounded to BF16) into the canonical
// no-swizzle K-major layout, PL planes of 8 k-values (2048 B each); the filter is held as
// the N = 32 operand in the same layout.  One thread issues the PL / 2 MMAs (K = 16) of a
// tile into one of two accumulators; while they run the threads drain the previous tile
// (bias, ReLU, BF16, padded-HWC store) and then gather the next one.  Persistent CTAs.
struct Conv0Args {
    ConvShape sh;
    const float* x;       // NCHW FP32, image stride sh.x_img_stride
    const float* w;       // [32][K] FP32
    const float* bias;    // [32]
    __nv_bfloat16* out;   // padded HWC BF16, grid (OH + 4) x (OW + 4) per image
    int64_t npix;
    int K, n_tiles;
    int* err;
};

// two floats rounded to BF16 (nearest even), the first in the low half
__device__ __forceinline__ uint32_t pack2_bf16(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

template <int PL>
__global__ void __launch_bounds__(128, PL == 4 ? 5 : 2) conv0_tc_kernel(const __grid_constant__ Conv0Args a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    constexpr uint32_t kTile = PL * 2048;            // one A tile: PL planes of 128 rows x 16 B
    uint8_t* b_s = smem + 2 * kTile;                  // the filter: PL planes of 32 rows x 16 B
    float* bias_s = reinterpret_cast<float*>(b_s + PL * 512);
    uint64_t* bars = reinterpret_cast<uint64_t*>(bias_s + kCh);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);
    const uint32_t a_u = smem_u32(smem), b_u = smem_u32(b_s), bar0 = smem_u32(bars);
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const ConvShape& sh = a.sh;
    const int opix = sh.OH * sh.OW;

    // inputs are read, and tensor memory taken, only once the previous kernel has finished,
    // as in every tcgen05 kernel of the library: a kernel lets its dependents launch before
    // it allocates, so one that allocated before its wait could hold columns its primary needs
    SQ_KERNEL_ENTRY();
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), 64);
    if (threadIdx.x == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int e = threadIdx.x; e < 32 * PL; e += 128) {   // filter row co, 8 k-values of plane c
        const int co = e / PL, c = e % PL;
        __align__(16) __nv_bfloat16 hb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int k = 8 * c + j;
            hb[j] = __float2bfloat16_rn(k < a.K ? a.w[(int64_t)co * a.K + k] : 0.f);
        }
        *reinterpret_cast<uint4*>(b_s + c * 512 + co * 16) = *reinterpret_cast<const uint4*>(hb);
    }
    if (threadIdx.x < kCh) bias_s[threadIdx.x] = a.bias[threadIdx.x];
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int n_local = (int)blockIdx.x < a.n_tiles ? (a.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int hw = sh.H * sh.W;
    bool ok = true;

    // this thread's pixel of tile t: its K inputs (loads issued, not yet waited for) ...
    auto load = [&](int t, float (&v)[8 * PL]) {
        const int64_t p = (int64_t)t * 128 + threadIdx.x;
        const bool valid = p < a.npix;
        const float* src = a.x;
        if (valid) {
            const int img = (int)(p / opix);
            const int rem = (int)(p - (int64_t)img * opix);
            const int oy = rem / sh.OW, ox = rem - oy * sh.OW;
            src += (int64_t)img * sh.x_img_stride + (int64_t)(oy * sh.stride) * sh.W + ox * sh.stride;
        }
#pragma unroll
        for (int k = 0; k < 8 * PL; ++k) {
            const int ci = k / 9, tap = k % 9;
            v[k] = (valid && k < a.K) ? __ldg(src + ci * hw + (tap / 3) * sh.W + tap % 3) : 0.f;
        }
    };
    // ... and written as BF16 into its row of A tile buffer b
    auto put = [&](int b, const float (&v)[8 * PL]) {
        uint8_t* dst = smem + b * kTile + threadIdx.x * 16;
#pragma unroll
        for (int c = 0; c < PL; ++c) {
            uint4 w4;
            w4.x = pack2_bf16(v[8 * c], v[8 * c + 1]);
            w4.y = pack2_bf16(v[8 * c + 2], v[8 * c + 3]);
            w4.z = pack2_bf16(v[8 * c + 4], v[8 * c + 5]);
            w4.w = pack2_bf16(v[8 * c + 6], v[8 * c + 7]);
            *reinterpret_cast<uint4*>(dst + c * 2048) = w4;
        }
    };
    // epilogue: this thread's accumulator row of tile t (buffer b) to its output pixel
    auto drain = [&](int t, int b) {
        uint32_t r0[16], r1[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)b * kCh;
        tmem_ld16(taddr, r0);
        tmem_ld16(taddr + 16, r1);
        const int64_t p = (int64_t)t * 128 + threadIdx.x;
        if (p >= a.npix) return;
        const int img = (int)(p / opix);
        const int rem = (int)(p - (int64_t)img * opix);
        const int oy = rem / sh.OW, ox = rem - oy * sh.OW;
        uint4* dst = reinterpret_cast<uint4*>(
            a.out + (((int64_t)img * (sh.OH + 4) + oy + 2) * (sh.OW + 4) + ox + 2) * kCh);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float f[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int co = 8 * c + j;
                const float v = __uint_as_float(co < 16 ? r0[co] : r1[co - 16]) + bias_s[co];
                f[j] = v > 0.f ? v : 0.f;
            }
            uint4 w4;
            w4.x = pack2_bf16(f[0], f[1]);
            w4.y = pack2_bf16(f[2], f[3]);
            w4.z = pack2_bf16(f[4], f[5]);
            w4.w = pack2_bf16(f[6], f[7]);
            dst[c] = w4;
        }
    };

    constexpr uint32_t idesc = idesc_bf16(128, kCh, false, false);
    for (int i = 0; i < n_local; ++i) {
        const int t = (int)blockIdx.x + i * (int)gridDim.x, b = i & 1;
        float v[8 * PL];
        load(t, v);   // in flight while the previous tile drains
        if (i > 0 && ok) {
            // the MMAs of tile i - 1 (and so of tile i - 2, which read buffer b) are complete
            const int pb = b ^ 1;
            ok = mbar_wait(bar0 + 8 * pb, ((i - 1) >> 1) & 1, a.err, 17);
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (ok) drain(t - (int)gridDim.x, pb);
        }
        put(b, v);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kc = 0; kc < PL / 2; ++kc)
                mma_bf16(tmem + (uint32_t)b * kCh, plain_desc(a_u + b * kTile + kc * 4096, 2048, 128),
                         plain_desc(b_u + kc * 1024, 512, 128), idesc, kc > 0 ? 1u : 0u);
            mma_commit(bar0 + 8 * b);
        }
        __syncwarp();
    }
    if (n_local > 0) {
        const int i = n_local - 1, b = i & 1;
        if (mbar_wait(bar0 + 8 * b, (i >> 1) & 1, a.err, 18) && ok) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            drain((int)blockIdx.x + i * (int)gridDim.x, b);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem_dealloc(tmem, 64);
    }
}

// ---------------------------------------------------------------- layout conversions
// CHW FP32 (per image stride img_stride) -> padded HWC BF16 interior.
__global__ void to_phwc_kernel(const float* __restrict__ src, int64_t img_stride, int nimg, int H, int W,
                               __nv_bfloat16* __restrict__ dst) {
    SQ_KERNEL_ENTRY();
    const int64_t n = (int64_t)nimg * H * W;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int img = (int)(p / (H * W));
    const int rem = (int)(p - (int64_t)img * H * W);
    const int y = rem / W, x = rem - (rem / W) * W;
    const float* s = src + img * img_stride + rem;
    __nv_bfloat16* d = dst + ((int64_t)img * (H + 4) * (W + 4) + (int64_t)(y + 2) * (W + 4) + x + 2) * kCh;
    __align__(16) __nv_bfloat16 hb[kCh];
#pragma unroll
    for (int c = 0; c < kCh; ++c) hb[c] = __float2bfloat16_rn(s[(int64_t)c * H * W]);
#pragma unroll
    for (int c = 0; c < 4; ++c) reinterpret_cast<uint4*>(d)[c] = reinterpret_cast<const uint4*>(hb)[c];
}

// Padded HWC BF16 interior -> NCHW FP32.
__global__ void from_phwc_kernel(const __nv_bfloat16* __restrict__ src, int nimg, int H, int W, float* __restrict__ dst) {
    SQ_KERNEL_ENTRY();
    const int64_t n = (int64_t)nimg * kCh * H * W;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int img = (int)(e / ((int64_t)kCh * H * W));
    const int rem = (int)(e - (int64_t)img * kCh * H * W);
    const int c = rem / (H * W), p = rem - (rem / (H * W)) * (H * W);
    const int y = p / W, x = p - (p / W) * W;
    dst[e] = __bfloat162float(src[((int64_t)img * (H + 4) * (W + 4) + (int64_t)(y + 2) * (W + 4) + x + 2) * kCh + c]);
}

// FP32 filter w[co][ci][ky][kx] -> forward layout [tap][ci/8][co][ci%8] and data-gradient
// layout (tap' = 8 - tap, channels swapped) [tap'][co/8][ci][co%8].
__global__ void conv_weight_cast_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ fwd,
                                        __nv_bfloat16* __restrict__ bwd) {
    SQ_KERNEL_ENTRY();
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= kCh * kCh * 9) return;
    const int co = e / (kCh * 9), rem = e - co * kCh * 9, ci = rem / 9, tap = rem - (rem / 9) * 9;
    const __nv_bfloat16 v = __float2bfloat16_rn(w[e]);
    fwd[tap * kCh * kCh + (ci / 8) * kCh * 8 + co * 8 + (ci % 8)] = v;
    bwd[(8 - tap) * kCh * kCh + (co / 8) * kCh * 8 + ci * 8 + (co % 8)] = v;
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

// Planes of a padded-HWC tensor: dims {8 channels, 4 planes, rows}, box {8, 1, 128}.
bool plane_map(CUtensorMap* m, const __nv_bfloat16* base, int64_t rows, int box_rows = 128) {
    auto fn = encode_fn();
    if (!fn || (reinterpret_cast<uintptr_t>(base) & 15) || box_rows < 8 || box_rows > 256) return false;
    cuuint64_t dims[3] = {8, 4, (cuuint64_t)rows};
    cuuint64_t strides[2] = {16, 64};
    cuuint32_t box[3] = {8, 1, (cuuint32_t)box_rows};
    cuuint32_t estr[3] = {1, 1, 1};
    std::memset(m, 0, sizeof(*m));
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }

size_t conv_smem(int load_rows) { return 1024 + 2 * 4 * (size_t)load_rows * 16 + kWBytes + 10 * 8 + 16; }
constexpr int kConvCtasPerSm = 2;   // resident CTAs per SM of the persistent convolution
int g_num_sms = 152;                 // set by conv_tc_prepare
size_t wgrad_smem(int slot_rows, int kq) {
    return 1024 + wgrad_operand_bytes(12 * (uint32_t)slot_rows * 16, 4 * (uint32_t)kq * 16) + 64 + 128 * 8 * 4 + 16;
}

}  // namespace

// Geometry of one call: the conv reads input rows up to (n_tiles * 128 - 1) + off0 + 2 Wp + 2.
int launch_conv32_tc(const ConvTc& c, int* err, cudaStream_t s) {
    if (c.nimg <= 0) return 0;
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    const int mv = c.out_h * c.Wp;
    a.n_tiles = (mv + 127) / 128;
    if (a.n_tiles > 4) return -1;
    a.tmem_cols = a.n_tiles <= 1 ? 32 : (a.n_tiles <= 2 ? 64 : 128);
    const int max_row = a.n_tiles * 128 - 1 + c.off0 + 2 * c.Wp + 2;
    a.load_rows = round_up(max_row + 1, 128);
    if (conv_smem(a.load_rows) > 200 * 1024) return -1;
    if (!plane_map(&a.tin, c.in, (int64_t)c.nimg * c.in_rows)) return -2;
    a.w = c.w; a.nimg = c.nimg; a.in_rows = c.in_rows; a.Wp = c.Wp; a.out_h = c.out_h; a.out_w = c.out_w;
    a.off0 = c.off0; a.bias = c.bias; a.relu = c.relu; a.mask = c.mask; a.out_phwc = c.out_phwc;
    a.out_chw = c.out_chw; a.out_chw_bf = c.out_chw_bf; a.err = err;
    const size_t smem = conv_smem(a.load_rows);
    const int ctas = std::min(c.nimg, g_num_sms * kConvCtasPerSm);
    launch_k(conv32_tc_kernel, dim3(ctas), dim3(kConvThreads), smem, s, a);
    return 0;
}

int64_t wgrad32_tc_workspace(int nimg) { return (int64_t)std::min(nimg, 148) * kCh * (kCh * 9 + 1); }

int wgrad32_per_cta(int nimg) {
    const int ctas = std::max(1, std::min(nimg, 148));
    return (nimg + ctas - 1) / ctas;
}

int launch_wgrad32_tc_partials(const WgradTc& c, int per_cta, float* work, int* err, cudaStream_t s) {
    if (c.nimg <= 0) return 0;
    if (per_cta < 1) return -1;
    WgradArgs a;
    std::memset(&a, 0, sizeof(a));
    a.kq = round_up(c.out_h * c.Wp, 16);
    // a slot covers the rows every K step of every vertical tap reads: kq + 2 Wp, loaded in
    // equal boxes of at most 256 rows, a multiple of 8 rows (128 B) each
    const int need = a.kq + 2 * c.Wp;
    const int nb = (need + 255) / 256;
    a.box_rows = round_up((need + nb - 1) / nb, 8);
    a.slot_rows = nb * a.box_rows;
    if (wgrad_smem(a.slot_rows, a.kq) > 220 * 1024 || (a.kq / 8) * 512 + 2048 > kDyBytesMax + 2048) return -1;
    if (!plane_map(&a.tin, c.x, (int64_t)c.nimg * c.in_rows, a.box_rows)) return -2;
    a.per_cta = per_cta;
    const int grid = (c.nimg + per_cta - 1) / per_cta;
    a.dy = c.dy; a.nimg = c.nimg; a.in_rows = c.in_rows; a.Wp = c.Wp; a.out_h = c.out_h; a.out_w = c.out_w;
    a.work = work; a.err = err;
    launch_k(wgrad32_tc_kernel, dim3(grid), dim3(128), wgrad_smem(a.slot_rows, a.kq), s, a);
    return 0;
}

void launch_wgrad32_reduce(const float* work, int ctas, float* dw, float* db, cudaStream_t s) {
    launch_k(wgrad32_reduce_kernel, dim3((kCh * (kCh * 9 + 1) + 31) / 32), dim3(32 * kRed32Groups), 0, s, work, ctas,
             dw, db);
}

int launch_wgrad32_tc(const WgradTc& c, float* work, float* dw, float* db, int* err, cudaStream_t s) {
    if (c.nimg <= 0) return 0;
    const int pc = wgrad32_per_cta(c.nimg);
    const int rc = launch_wgrad32_tc_partials(c, pc, work, err, s);
    if (rc != 0) return rc;
    launch_wgrad32_reduce(work, (c.nimg + pc - 1) / pc, dw, db, s);
    return 0;
}

void conv_tc_prepare() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        sms > 0)
        g_num_sms = sms;
    cudaFuncSetAttribute(conv32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(wgrad32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(conv0_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(conv0_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(conv0_tc_kernel<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    encode_fn();
}

void launch_conv0_phwc(const ConvShape& sh, const float* x, const float* w, const float* b, __nv_bfloat16* out,
                       cudaStream_t s) {
    const int64_t npix = (int64_t)sh.nimg * sh.OH * sh.OW;
    if (npix <= 0) return;
    const size_t smem = ((size_t)sh.Cin * 9 * kCh + kCh) * sizeof(float);
    launch_k(conv0_phwc_kernel, dim3((unsigned)((npix + 511) / 512)), dim3(256), smem, s, sh, x, w, b, out);
}

namespace {
template <int PL>
size_t conv0_tc_smem() { return 128 + 2 * PL * 2048 + PL * 512 + kCh * 4 + 32; }
// CTAs per SM in the grid (each holds 64 tensor-memory columns, 512 per SM); the
// SQUINT_CONV0_CTAS environment variable (1..8) overrides it
int conv0_ctas_per_sm() {
    static int n = [] {
        const char* e = std::getenv("SQUINT_CONV0_CTAS");
        const int v = e ? std::atoi(e) : 4;
        return v >= 1 && v <= 8 ? v : 4;
    }();
    return n;
}
template <int PL>
void conv0_tc_go(const Conv0Args& a, cudaStream_t s) {
    // at least 28 KB of shared memory per CTA keeps at most 8 of them (8 x 64 columns) on an SM
    const size_t smem = std::max(conv0_tc_smem<PL>(), (size_t)28 * 1024 + 1);
    const int ctas = std::min(a.n_tiles, g_num_sms * conv0_ctas_per_sm());
    launch_k(conv0_tc_kernel<PL>, dim3(ctas), dim3(128), smem, s, a);
}
}  // namespace

int launch_conv0_tc(const ConvShape& sh, const float* x, const float* w, const float* b, __nv_bfloat16* out,
                    int* err, cudaStream_t s) {
    const int K = sh.Cin * 9;
    if (sh.Cout != kCh || K > 144 || sh.nimg < 0 || sh.stride < 1) return -1;
    const int64_t npix = (int64_t)sh.nimg * sh.OH * sh.OW;
    if (npix <= 0) return 0;
    Conv0Args a;
    std::memset(&a, 0, sizeof(a));
    a.sh = sh; a.x = x; a.w = w; a.bias = b; a.out = out; a.npix = npix; a.K = K; a.err = err;
    a.n_tiles = (int)((npix + 127) / 128);
    if (K <= 32) conv0_tc_go<4>(a, s);
    else if (K <= 64) conv0_tc_go<8>(a, s);
    else conv0_tc_go<18>(a, s);
    return 0;
}

void launch_to_phwc(const float* src, int64_t img_stride, int nimg, int H, int W, __nv_bfloat16* dst, cudaStream_t s) {
    const int64_t n = (int64_t)nimg * H * W;
    if (n) launch_k(to_phwc_kernel, dim3((unsigned)((n + 127) / 128)), dim3(128), 0, s, src, img_stride, nimg, H, W, dst);
}
void launch_from_phwc(const __nv_bfloat16* src, int nimg, int H, int W, float* dst, cudaStream_t s) {
    const int64_t n = (int64_t)nimg * kCh * H * W;
    if (n) launch_k(from_phwc_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, src, nimg, H, W, dst);
}
void launch_conv_weight_cast(const float* w, __nv_bfloat16* fwd, __nv_bfloat16* bwd, cudaStream_t s) {
    launch_k(conv_weight_cast_kernel, dim3((kCh * kCh * 9 + 255) / 256), dim3(256), 0, s, w, fwd, bwd);
}

}  // namespace sq
