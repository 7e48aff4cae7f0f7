// Front end of the update (steps a1-a4) and of inference.
//
// One CTA per (sample, frame): it draws the slot and the crop offset, stages
// the uint8 frame in shared memory with 128-bit loads, and forms the squinted
// image from integer f x f box sums over the replicate-padded, shifted frame
// (Sec. IV "Resolution Squinting": area downsampling; the shift is the
// DrQ-style random-shift augmentation).
#include <algorithm>
#include <mutex>

#include "sq_kernels.cuh"

namespace sq {

__global__ void __launch_bounds__(256) frontend_kernel(FrontendArgs a) {
    SQ_KERNEL_ENTRY();
    extern __shared__ __align__(16) uint8_t frame[];
    const int b = blockIdx.x;
    const int which = blockIdx.y;                 // 0: o_t, 1: o_{t+1}
    const uint64_t u = (uint64_t)*a.update_idx + (uint64_t)a.idx_offset;

    uint32_t w[4];
    draw_block(w, a.seed, (uint32_t)b, kStreamIndex, 0, u);
    const int64_t idx = (int64_t)range_draw(w[0], (uint32_t)a.n_slots);
    const int64_t nxt = (idx + 1) % a.n_slots;
    const int64_t slot = which ? nxt : idx;
    draw_block(w, a.seed, (uint32_t)b, which ? kStreamShiftT1 : kStreamShiftT, 0, u);
    const int span = 2 * a.pad + 1;
    const int dx = (int)range_draw(w[0], (uint32_t)span);
    const int dy = (int)range_draw(w[1], (uint32_t)span);

    const int64_t fbytes = (int64_t)a.C * a.H * a.W;
    const uint8_t* src = a.obs + slot * fbytes;
    {
    __shared__ uint64_t bar;
    // the whole frame in one TMA bulk copy when aligned (most bytes in flight per SM)
    const bool bulk = fbytes > 0 && (fbytes & 15) == 0 && fbytes < (1 << 20) && (((uintptr_t)src) & 15) == 0;
    if (bulk) {
        if (threadIdx.x == 0) {
            bulk_load_init(&bar);
            bulk_load_stream(frame, src, (uint32_t)fbytes, &bar);
        }
        // one thread waits (the others at the block barrier issue nothing meanwhile)
        if (threadIdx.x == 0 && !bulk_load_wait(&bar, 0) && a.err) atomicCAS(a.err, 0, 31);
        __syncthreads();
    } else {
        for (int64_t i = threadIdx.x; i < fbytes; i += blockDim.x) frame[i] = src[i];
        __syncthreads();
    }

    const int hs = a.H / a.f, ws = a.W / a.f;
    const int plane = hs * ws;
    const int n_out = a.C * plane;
    const float denom = 255.0f * (float)(a.f * a.f);
    const int64_t row = (int64_t)which * a.B + b;
    float* xo = a.x + row * n_out;
    // f = 4 with 4-byte-aligned frame rows: a lane per output column j, a warp per output
    // row.  Each of the 4 source rows gives the lane's 4 bytes as one byte permute of two
    // aligned 32-bit words and one dp4a (exact integer sums); the permute selector, fixed
    // per lane, also replicates the edge byte where the shifted window leaves the frame
    // (replicate padding), so every lane runs the same instructions.
    if (a.f == 4 && (a.W & 3) == 0 && ws == 32 && (blockDim.x % 32) == 0) {
        const int j = threadIdx.x % 32;
        const int x0 = j * 4 + dx - a.pad;
        const int wpr = a.W / 4;                        // words per frame row
        int wlo;
        uint32_t sel = 0;
        if (x0 >= 0 && x0 + 3 <= a.W - 1) {             // interior: bytes k .. k+3 of (lo, hi)
            wlo = x0 >> 2;
            const int k = x0 & 3;
            sel = (uint32_t)k | ((uint32_t)(k + 1) << 4) | ((uint32_t)(k + 2) << 8) | ((uint32_t)(k + 3) << 12);
        } else if (x0 < 0) {                            // left edge: bytes max(x0 + v, 0) of the first word
            wlo = 0;
#pragma unroll
            for (int v = 0; v < 4; ++v) sel |= (uint32_t)max(x0 + v, 0) << (4 * v);
        } else {                                        // right edge: bytes of the last word (as hi)
            wlo = wpr - 2;
#pragma unroll
            for (int v = 0; v < 4; ++v) sel |= (uint32_t)(4 + min(x0 + v, a.W - 1) - (a.W - 4)) << (4 * v);
        }
        const int whi = min(wlo + 1, wpr - 1);
        const uint32_t* f32 = reinterpret_cast<const uint32_t*>(frame);
        const int warps = blockDim.x / 32;
        for (int c = 0; c < a.C; ++c) {
            const uint32_t* plane32 = f32 + (int64_t)c * a.H * wpr;
            for (int i = threadIdx.x / 32; i < hs; i += warps) {
                uint32_t sum = 0;
#pragma unroll
                for (int uu = 0; uu < 4; ++uu) {
                    const int y = min(max(i * 4 + uu + dy - a.pad, 0), a.H - 1);
                    const uint32_t* rp = plane32 + y * wpr;
                    sum = __dp4a(__byte_perm(rp[wlo], rp[whi], sel), 0x01010101u, sum);
                }
                const int o = (c * hs + i) * 32 + j;
                const float val = (float)sum / denom - 0.5f;
                xo[o] = val;
                if (a.x_bf) a.x_bf[row * n_out + o] = __float2bfloat16_rn(val);
                if (a.sums) a.sums[row * n_out + o] = (uint16_t)sum;
            }
        }
    } else
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        const int c = o / plane;
        const int i = (o - c * plane) / ws;
        const int j = o - c * plane - i * ws;
        uint32_t sum = 0;
        for (int uu = 0; uu < a.f; ++uu) {
            const int y = min(max(i * a.f + uu + dy - a.pad, 0), a.H - 1);
            const uint8_t* rp = frame + ((int64_t)c * a.H + y) * a.W;
            for (int vv = 0; vv < a.f; ++vv) {
                const int xx = min(max(j * a.f + vv + dx - a.pad, 0), a.W - 1);
                sum += rp[xx];
            }
        }
        const float val = (float)sum / denom - 0.5f;
        xo[o] = val;
        if (a.x_bf) a.x_bf[row * n_out + o] = __float2bfloat16_rn(val);
        if (a.sums) a.sums[row * n_out + o] = (uint16_t)sum;
    }

    }

    const int64_t row = (int64_t)which * a.B + b;
    if (threadIdx.x == 0) {
        a.idx_out[row] = (int32_t)slot;
        a.shift_out[2 * row] = dx;
        a.shift_out[2 * row + 1] = dy;
        if (which == 0) {
            a.r_out[b] = a.reward[idx];
            a.d_out[b] = (float)a.done[idx];
        }
    }
    for (int t = 0; t < a.n_dst; ++t) {
        const CopyDst& d = a.dst[t];
        const bool mine = (d.which == 1) == (which == 1);
        if (!mine) continue;
        const int width = d.which == 2 ? a.A : a.P;
        const float* s = d.which == 2 ? a.action + idx * a.A : a.proprio + slot * a.P;
        for (int k = threadIdx.x; k < width; k += blockDim.x) {
            d.ptr[(int64_t)b * d.ld + d.col + k] = s[k];
            if (d.ptr_h) d.ptr_h[(int64_t)b * d.ld_h + d.col + k] = __float2bfloat16_rn(s[k]);
        }
    }
}

void launch_frontend(const FrontendArgs& a, cudaStream_t s) {
    const size_t smem = (size_t)a.C * a.H * a.W;
    launch_k(frontend_kernel, dim3(dim3(a.B, 2)), dim3(256), smem, s, a);
}

// Inference: one CTA per row; no shift (crop at the centre offset p = pad means
// the identity, so it is left out entirely).
__global__ void __launch_bounds__(256) act_frontend_kernel(ActFrontArgs a) {
    SQ_KERNEL_ENTRY();
    extern __shared__ __align__(16) uint8_t frame[];
    const int r = blockIdx.x;
    const int q = a.row_req[r];
    const int64_t fbytes = (int64_t)a.C * a.H * a.W;
    const uint8_t* src = a.obs[q] + (int64_t)a.row_in_req[r] * fbytes;
    if ((fbytes & 15) == 0 && (((uintptr_t)src) & 15) == 0) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(frame);
        for (int64_t i = threadIdx.x; i < fbytes / 16; i += blockDim.x) d4[i] = __ldg(s4 + i);
    } else {
        for (int64_t i = threadIdx.x; i < fbytes; i += blockDim.x) frame[i] = src[i];
    }
    __syncthreads();
    const int hs = a.H / a.f, ws = a.W / a.f, plane = hs * ws, n_out = a.C * plane;
    const float denom = 255.0f * (float)(a.f * a.f);
    if (a.f == 4 && (a.W & 3) == 0) {   // aligned 4-byte row segments summed by dp4a
        for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
            const int c = o / plane, i = (o - c * plane) / ws, j = o - c * plane - i * ws;
            uint32_t sum = 0;
#pragma unroll
            for (int uu = 0; uu < 4; ++uu) {
                const uint32_t w = *reinterpret_cast<const uint32_t*>(frame + ((int64_t)c * a.H + i * 4 + uu) * a.W + j * 4);
                sum = __dp4a(w, 0x01010101u, sum);
            }
            a.x[(int64_t)r * n_out + o] = (float)sum / denom - 0.5f;
        }
    } else
    for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
        const int c = o / plane, i = (o - c * plane) / ws, j = o - c * plane - i * ws;
        uint32_t sum = 0;
        for (int uu = 0; uu < a.f; ++uu) {
            const uint8_t* rp = frame + ((int64_t)c * a.H + i * a.f + uu) * a.W + j * a.f;
            for (int vv = 0; vv < a.f; ++vv) sum += rp[vv];
        }
        a.x[(int64_t)r * n_out + o] = (float)sum / denom - 0.5f;
    }
    const float* p = a.prop[q] + (int64_t)a.row_in_req[r] * a.P;
    for (int k = threadIdx.x; k < a.P; k += blockDim.x) a.xin[(int64_t)r * a.ld_xin + a.col + k] = p[k];
}

void launch_act_frontend(const ActFrontArgs& a, cudaStream_t s) {
    if (a.rows <= 0) return;
    const size_t smem = (size_t)a.C * a.H * a.W;
    launch_k(act_frontend_kernel, dim3(a.rows), dim3(256), smem, s, a);
}

// Squint at insert: one thread per output value, the f x f box sum of a uint8 frame
// rounded half up to its mean, written into ring slot (slot0 + frame) mod n_slots.
__global__ void __launch_bounds__(256) squint_store_kernel(const uint8_t* __restrict__ src, int n, int C, int H,
                                                          int W, int f, uint8_t* __restrict__ ring, int64_t slot0,
                                                          int64_t n_slots) {
    SQ_KERNEL_ENTRY();
    const int hs = H / f, ws = W / f;
    const int64_t per = (int64_t)C * hs * ws;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * per) return;
    const int img = (int)(e / per);
    const int r = (int)(e - (int64_t)img * per);
    const int c = r / (hs * ws), i = (r / ws) % hs, j = r % ws;
    const uint8_t* p = src + (((int64_t)img * C + c) * H + (int64_t)i * f) * W + (int64_t)j * f;
    uint32_t sum = 0;
    for (int u = 0; u < f; ++u)
        for (int v = 0; v < f; ++v) sum += p[(int64_t)u * W + v];
    const uint32_t ff = (uint32_t)(f * f);
    const int64_t slot = (slot0 + img) % n_slots;
    ring[slot * per + r] = (uint8_t)((sum + ff / 2) / ff);
}

void launch_squint_store(const uint8_t* src, int n, int C, int H, int W, int f, uint8_t* ring, int64_t slot0,
                         int64_t n_slots, cudaStream_t s) {
    const int64_t total = (int64_t)n * C * (H / f) * (W / f);
    if (total <= 0) return;
    launch_k(squint_store_kernel, dim3((unsigned)((total + 255) / 256)), dim3(256), 0, s, src, n, C, H, W, f, ring,
             slot0, n_slots);
}

// Opt the kernels in to a whole frame of dynamic shared memory (with the kernel's own
// static shared memory a 48 KiB frame is already above the default limit).  The limit is a
// per-function attribute shared by every handle of the process, so it only ever grows.
void frontend_prepare(size_t frame_bytes) {
    static std::mutex mu;
    static size_t granted = 0;
    std::lock_guard<std::mutex> lk(mu);
    granted = std::max(granted, frame_bytes);
    cudaFuncSetAttribute(frontend_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)granted);
    cudaFuncSetAttribute(act_frontend_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)granted);
    // all of the unified L1 / shared memory as shared: as many whole frames in flight per SM as fit
    cudaFuncSetAttribute(frontend_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(act_frontend_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

}  // namespace sq
