// Front end of the update (steps a1-a4) and of inference.
//
// One CTA per (sample, frame): it draws the slot and the crop offset and forms
// the squinted image from integer f x f box sums over the replicate-padded,
// shifted frame (Sec. IV "Resolution Squinting": area downsampling; the shift
// is the DrQ-style random-shift augmentation).  For f = 4 on power-of-two
// widths up to 128 the rows are read straight from global memory with 16-byte
// loads; other sizes stage the frame in shared memory first.
#include <algorithm>
#include <mutex>

#include "sq_kernels.cuh"

namespace sq {

// f = 4 read straight from global memory: frame base 16-byte aligned, W a power of two in
// [16, 128], |dx - pad| <= 12, the H / 4 output rows of a channel a whole number of warp
// iterations (512 / W rows each) and the outputs aligned for vector stores.
__host__ __device__ inline bool squint4_direct(const FrontendArgs& a) {
    return a.f == 4 && a.C > 0 && a.H >= 4 && a.W >= 16 && a.W <= 128 && (a.W & (a.W - 1)) == 0 && a.pad <= 12 &&
           (a.H / 4) % (512 / a.W) == 0 && ((int64_t)a.C * a.H * a.W) % 16 == 0 &&
           (reinterpret_cast<uintptr_t>(a.obs) & 15) == 0 && (reinterpret_cast<uintptr_t>(a.x) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(a.x_bf) & 7) == 0 && (reinterpret_cast<uintptr_t>(a.sums) & 7) == 0;
}

// The f = 4 squint of one frame without staging it.  A lane owns 4 output columns (16
// source bytes) of one output row: lanes g Lr .. g Lr + Lr - 1 (Lr = W / 16) share output
// row g of the warp iteration, which covers 32 / Lr output rows.  For each of the 4 box
// rows the lane loads its 16 bytes and forms its window shifted by s = dx - pad from 12
// words (the previous lane's chunk, its own, the next lane's; past either end of the row
// the edge byte replicated, which is the replicate padding), then adds one byte permute
// and one dp4a per output.  FS = floor(s / 4) is fixed per frame, so every window index is
// a constant; the byte offset s mod 4 is the permute selector `sel`.  xo, xo_bf, so point
// at the frame's first output (xo_bf, so may be null).
template <int FS>
__device__ __forceinline__ void squint4_direct_rows(const FrontendArgs& a, const uint4* __restrict__ frame4, int dy,
                                                    uint32_t sel, float* __restrict__ xo, __nv_bfloat16* xo_bf,
                                                    uint16_t* so, float denom) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int lg = __ffs(a.W) - 5;             // log2(W / 16)
    const int Lr = 1 << lg;
    const int q = lane & (Lr - 1), g = lane >> lg;
    const int RW = 32 >> lg;                   // output rows per warp iteration
    const int hs = a.H >> 2, ws = a.W >> 2;
    const int itc = hs / RW;                   // warp iterations per channel
    const bool first = q == 0, last = q == Lr - 1;
    for (int c = 0; c < a.C; ++c) {
        const uint4* plane = frame4 + c * a.H * Lr + q;
        for (int it = warp; it < itc; it += nwarps) {
            const int i = it * RW + g;         // output row of this lane in channel c
            const int yb = 4 * i + dy - a.pad;
            uint4 v[4];
#pragma unroll
            for (int uu = 0; uu < 4; ++uu) v[uu] = __ldcs(plane + min(max(yb + uu, 0), a.H - 1) * Lr);
            uint32_t acc[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int uu = 0; uu < 4; ++uu) {
                const uint32_t w[4] = {v[uu].x, v[uu].y, v[uu].z, v[uu].w};
                uint32_t win[12];
#pragma unroll
                for (int m = 0; m < 4; ++m) win[4 + m] = w[m];
                if constexpr (FS < 0) {        // window words 4 + FS .. 3 from the previous chunk
                    const uint32_t edge = __byte_perm(w[0], 0u, 0x0000u);
#pragma unroll
                    for (int m = 4 + FS; m < 4; ++m) {
                        const uint32_t p = __shfl_up_sync(0xffffffffu, w[m], 1);
                        win[m] = first ? edge : p;
                    }
                } else {                       // window words 8 .. 8 + FS from the next chunk
                    const uint32_t edge = __byte_perm(w[3], 0u, 0x3333u);
#pragma unroll
                    for (int m = 0; m <= FS; ++m) {
                        const uint32_t p = __shfl_down_sync(0xffffffffu, w[m], 1);
                        win[8 + m] = last ? edge : p;
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    acc[k] = __dp4a(__byte_perm(win[4 + k + FS], win[5 + k + FS], sel), 0x01010101u, acc[k]);
            }
            const int o = (c * hs + i) * ws + 4 * q;
            float val[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) val[k] = (float)acc[k] / denom - 0.5f;
            *reinterpret_cast<float4*>(xo + o) = make_float4(val[0], val[1], val[2], val[3]);
            if (xo_bf) {
                __nv_bfloat162 lo = __floats2bfloat162_rn(val[0], val[1]);
                __nv_bfloat162 hi = __floats2bfloat162_rn(val[2], val[3]);
                uint2 u;
                u.x = *reinterpret_cast<uint32_t*>(&lo);
                u.y = *reinterpret_cast<uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(xo_bf + o) = u;
            }
            if (so) *reinterpret_cast<uint2*>(so + o) = make_uint2(acc[0] | (acc[1] << 16), acc[2] | (acc[3] << 16));
        }
    }
}

__global__ void __launch_bounds__(256, 4) frontend_kernel(FrontendArgs a) {
    SQ_KERNEL_ENTRY();
    extern __shared__ __align__(16) uint8_t frame[];
    const int b = blockIdx.x;
    const int which = blockIdx.y;                 // 0: o_t, 1: o_{t+1}
    const uint64_t u = (uint64_t)*a.update_idx + (uint64_t)a.idx_offset;

    // the slot and shift draws, once per frame: lane 0 of warp 0 the index, the other
    // lanes the shift (the same draw), shared through shared memory
    __shared__ int64_t s_idx;
    __shared__ int s_shift[2];
    const int span = 2 * a.pad + 1;
    if (threadIdx.x < 32) {
        uint32_t w[4];
        draw_block(w, a.seed, (uint32_t)b, threadIdx.x == 0 ? kStreamIndex : (which ? kStreamShiftT1 : kStreamShiftT),
                   0, u);
        if (threadIdx.x == 0) s_idx = (int64_t)range_draw(w[0], (uint32_t)a.n_slots);
        if (threadIdx.x == 1) {
            s_shift[0] = (int)range_draw(w[0], (uint32_t)span);
            s_shift[1] = (int)range_draw(w[1], (uint32_t)span);
        }
    }
    __syncthreads();
    const int64_t idx = s_idx;
    const int64_t nxt = (idx + 1) % a.n_slots;
    const int64_t slot = which ? nxt : idx;
    const int dx = s_shift[0], dy = s_shift[1];

    const int64_t fbytes = (int64_t)a.C * a.H * a.W;
    const uint8_t* src = a.obs + slot * fbytes;
    const int hs = a.H / a.f, ws = a.W / a.f;
    const int plane = hs * ws;
    const int n_out = a.C * plane;
    const float denom = 255.0f * (float)(a.f * a.f);
    if (squint4_direct(a) && (blockDim.x % 32) == 0) {
        const int s = dx - a.pad;
        const uint32_t o = (uint32_t)(s & 3);
        const uint32_t sel = o | ((o + 1) << 4) | ((o + 2) << 8) | ((o + 3) << 12);
        const int64_t base = ((int64_t)which * a.B + b) * n_out;
        const uint4* f4 = reinterpret_cast<const uint4*>(src);
        float* xo = a.x + base;
        __nv_bfloat16* xb = a.x_bf ? a.x_bf + base : nullptr;
        uint16_t* so = a.sums ? a.sums + base : nullptr;
        switch (s >> 2) {                         // floor(s / 4), in [-3, 3]
            case -3: squint4_direct_rows<-3>(a, f4, dy, sel, xo, xb, so, denom); break;
            case -2: squint4_direct_rows<-2>(a, f4, dy, sel, xo, xb, so, denom); break;
            case -1: squint4_direct_rows<-1>(a, f4, dy, sel, xo, xb, so, denom); break;
            case 0: squint4_direct_rows<0>(a, f4, dy, sel, xo, xb, so, denom); break;
            case 1: squint4_direct_rows<1>(a, f4, dy, sel, xo, xb, so, denom); break;
            case 2: squint4_direct_rows<2>(a, f4, dy, sel, xo, xb, so, denom); break;
            default: squint4_direct_rows<3>(a, f4, dy, sel, xo, xb, so, denom); break;
        }
    } else {
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

    const int64_t row = (int64_t)which * a.B + b;
    float* xo = a.x + row * n_out;
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
    for (int t = 0; t < a.n_dst && threadIdx.x < 32; ++t) {   // one warp: rows of at most a few dozen
        const CopyDst& d = a.dst[t];
        const bool mine = (d.which == 1) == (which == 1);
        if (!mine) continue;
        const int width = d.which == 2 ? a.A : a.P;
        const float* s = d.which == 2 ? a.action + idx * a.A : a.proprio + slot * a.P;
        for (int k = threadIdx.x; k < width; k += 32) {
            d.ptr[(int64_t)b * d.ld + d.col + k] = s[k];
            if (d.ptr_h) d.ptr_h[(int64_t)b * d.ld_h + d.col + k] = __float2bfloat16_rn(s[k]);
        }
    }
}

void launch_frontend(const FrontendArgs& a, cudaStream_t s) {
    const size_t smem = squint4_direct(a) ? 0 : (size_t)a.C * a.H * a.W;   // the direct squint stages nothing
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
