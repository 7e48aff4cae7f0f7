// Dense contractions on CUDA cores: grouped GEMM and valid 3x3 convolutions as
// implicit GEMMs.  These are the plain FP32 path of the update (and, in FP64,
// the reference-precision kernels the layer-level gradient checks use).
//
// Tile: 64 x 64 outputs x 16 reduction steps per stage, 256 threads, 4 x 4
// outputs per thread, operands staged in shared memory k-major.
#include <type_traits>

#include "sq_kernels.cuh"

#include <algorithm>
#include <vector>

namespace sq {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
constexpr int kMaxProbs = 8;

struct GemmBatch {
    GemmProblem p[kMaxProbs];
    int tile_start[kMaxProbs + 1];
    int tiles_n[kMaxProbs];
    int n;
};

template <typename T, int LAYOUT>
__global__ void __launch_bounds__(NT) gemm_kernel(GemmBatch gb) {
    SQ_KERNEL_ENTRY();
    __shared__ T As[BK][BM + 4];
    __shared__ T Bs[BK][BN + 4];
    int pi = 0;
    while (pi + 1 < gb.n && (int)blockIdx.x >= gb.tile_start[pi + 1]) ++pi;
    const GemmProblem& P = gb.p[pi];
    const int t = blockIdx.x - gb.tile_start[pi];
    const int m0 = (t / gb.tiles_n[pi]) * BM;
    const int n0 = (t % gb.tiles_n[pi]) * BN;
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;

    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    constexpr bool A_K = (LAYOUT == kKK || LAYOUT == kKN);
    constexpr bool B_K = (LAYOUT == kKK);
    for (int s = 0; s < P.n_sum; ++s) {
        const T* A = static_cast<const T*>(P.A) + (int64_t)s * P.a_sum;
        const T* Bm = static_cast<const T*>(P.B) + (int64_t)s * P.b_sum;
        for (int k0 = 0; k0 < P.K; k0 += BK) {
            // stage A: 64 x 16, 4 elements per thread
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int ml, kl;
                if (A_K) { ml = tid / 4; kl = (tid % 4) * 4 + e; }
                else     { kl = tid / 16; ml = (tid % 16) * 4 + e; }
                const int m = m0 + ml, k = k0 + kl;
                As[kl][ml] = (m < P.M && k < P.K) ? A[(int64_t)m * P.sa_m + (int64_t)k * P.sa_k] : T(0);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int nl, kl;
                if (B_K) { nl = tid / 4; kl = (tid % 4) * 4 + e; }
                else     { kl = tid / 16; nl = (tid % 16) * 4 + e; }
                const int n = n0 + nl, k = k0 + kl;
                Bs[kl][nl] = (n < P.N && k < P.K) ? Bm[(int64_t)n * P.sb_n + (int64_t)k * P.sb_k] : T(0);
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                T a[4], bb[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * bb[j];
            }
            __syncthreads();
        }
    }
    T* C = static_cast<T*>(P.C);
    const T* bias = static_cast<const T*>(P.bias);
    const T* mask = static_cast<const T*>(P.mask);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= P.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= P.N) continue;
            T v = acc[i][j];
            if (bias) v += bias[n];
            if (mask && !(mask[(int64_t)m * P.sm_m + (int64_t)n * P.sm_n] > T(0))) v = T(0);
            T* dst = C + (int64_t)m * P.sc_m + (int64_t)n * P.sc_n;
            *dst = P.accumulate ? *dst + v : v;
        }
    }
}

}  // namespace

template <typename T>
void launch_gemm(const GemmProblem* probs, int n_probs, GemmLayout layout, cudaStream_t s) {
    for (int base = 0; base < n_probs; base += kMaxProbs) {
        GemmBatch gb{};
        gb.n = std::min(kMaxProbs, n_probs - base);
        int tiles = 0;
        for (int i = 0; i < gb.n; ++i) {
            gb.p[i] = probs[base + i];
            if (gb.p[i].n_sum < 1) gb.p[i].n_sum = 1;
            gb.tile_start[i] = tiles;
            gb.tiles_n[i] = (gb.p[i].N + BN - 1) / BN;
            tiles += ((gb.p[i].M + BM - 1) / BM) * gb.tiles_n[i];
        }
        gb.tile_start[gb.n] = tiles;
        if (tiles == 0) continue;
        switch (layout) {
            case kKK: launch_k(gemm_kernel<T, kKK>, dim3(tiles), dim3(NT), 0, s, gb); break;
            case kKN: launch_k(gemm_kernel<T, kKN>, dim3(tiles), dim3(NT), 0, s, gb); break;
            case kMN: launch_k(gemm_kernel<T, kMN>, dim3(tiles), dim3(NT), 0, s, gb); break;
        }
    }
}
template void launch_gemm<float>(const GemmProblem*, int, GemmLayout, cudaStream_t);
template void launch_gemm<double>(const GemmProblem*, int, GemmLayout, cudaStream_t);

// ---------------------------------------------------------------- convolutions
// Implicit GEMM, tile 128 pixels x 32 channels x 16 reduction steps.
namespace {
constexpr int CBM = 128, CBN = 32, CBK = 16;

// Forward: M = nimg*OH*OW pixels, N = Cout, K = Cin*9.
template <typename T>
__global__ void __launch_bounds__(NT) conv_fwd_kernel(ConvShape sh, const T* __restrict__ x, const T* __restrict__ w,
                                                      const T* __restrict__ bias, T* __restrict__ y, int relu) {
    SQ_KERNEL_ENTRY();
    __shared__ T As[CBK][CBM + 4];
    __shared__ T Bs[CBK][CBN + 4];
    const int tid = threadIdx.x;
    const int M = sh.nimg * sh.OH * sh.OW, N = sh.Cout, K = sh.Cin * 9;
    const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * CBN;
    // each thread stages pixel ml = tid % 128 at reduction rows tid/128 + 2e
    const int ml = tid % CBM;
    const int m = m0 + ml;
    int64_t xbase = -1;
    if (m < M) {
        const int img = m / (sh.OH * sh.OW);
        const int rem = m - img * sh.OH * sh.OW;
        const int oy = rem / sh.OW, ox = rem - (rem / sh.OW) * sh.OW;
        xbase = (int64_t)img * sh.x_img_stride + (int64_t)(oy * sh.stride) * sh.W + ox * sh.stride;
    }
    const int ty = tid % 32, tx = tid / 32;   // lanes walk pixels (coalesced stores), warps walk channels
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int64_t plane = (int64_t)sh.H * sh.W;
    for (int k0 = 0; k0 < K; k0 += CBK) {
#pragma unroll
        for (int e = 0; e < CBK / 2; ++e) {
            const int kl = tid / CBM + 2 * e;
            const int k = k0 + kl;
            T v = T(0);
            if (xbase >= 0 && k < K) {
                const int ci = k / 9, r = k - ci * 9, ky = r / 3, kx = r - ky * 3;
                v = x[xbase + ci * plane + ky * sh.W + kx];
            }
            As[kl][ml] = v;
        }
        for (int e = tid; e < CBK * CBN; e += NT) {
            const int nl = e / CBK, kl = e % CBK;
            const int n = n0 + nl, k = k0 + kl;
            Bs[kl][nl] = (n < N && k < K) ? w[(int64_t)n * K + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CBK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 32 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 8 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mm = m0 + ty + 32 * i;
        if (mm >= M) continue;
        const int img = mm / (sh.OH * sh.OW);
        const int rem = mm - img * sh.OH * sh.OW;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 8 * j;
            if (n >= N) continue;
            T v = acc[i][j] + bias[n];
            if (relu && !(v > T(0))) v = T(0);
            y[(int64_t)img * sh.y_img_stride + (int64_t)n * sh.OH * sh.OW + rem] = v;
        }
    }
}

// Data gradient: M = nimg*H*W input pixels, N = Cin, K = Cout*9.
template <typename T>
__global__ void __launch_bounds__(NT) conv_dgrad_kernel(ConvShape sh, const T* __restrict__ dy, const T* __restrict__ w,
                                                        T* __restrict__ dx, const T* __restrict__ mask) {
    SQ_KERNEL_ENTRY();
    __shared__ T As[CBK][CBM + 4];
    __shared__ T Bs[CBK][CBN + 4];
    const int tid = threadIdx.x;
    const int M = sh.nimg * sh.H * sh.W, N = sh.Cin, K = sh.Cout * 9;
    const int m0 = blockIdx.x * CBM, n0 = blockIdx.y * CBN;
    const int ml = tid % CBM;
    const int m = m0 + ml;
    int img = 0, iy = 0, ix = 0;
    if (m < M) {
        img = m / (sh.H * sh.W);
        const int rem = m - img * sh.H * sh.W;
        iy = rem / sh.W;
        ix = rem - iy * sh.W;
    }
    const int ty = tid % 32, tx = tid / 32;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int64_t oplane = (int64_t)sh.OH * sh.OW;
    const T* dyi = dy + (int64_t)img * sh.y_img_stride;
    for (int k0 = 0; k0 < K; k0 += CBK) {
#pragma unroll
        for (int e = 0; e < CBK / 2; ++e) {
            const int kl = tid / CBM + 2 * e;
            const int k = k0 + kl;
            T v = T(0);
            if (m < M && k < K) {
                const int co = k / 9, r = k - co * 9, ky = r / 3, kx = r - ky * 3;
                const int ty_ = iy - ky, tx_ = ix - kx;
                if (ty_ >= 0 && tx_ >= 0 && ty_ % sh.stride == 0 && tx_ % sh.stride == 0) {
                    const int oy = ty_ / sh.stride, ox = tx_ / sh.stride;
                    if (oy < sh.OH && ox < sh.OW) v = dyi[co * oplane + oy * sh.OW + ox];
                }
            }
            As[kl][ml] = v;
        }
        for (int e = tid; e < CBK * CBN; e += NT) {
            const int nl = e % CBN, kl = e / CBN;
            const int n = n0 + nl, k = k0 + kl;
            T v = T(0);
            if (n < N && k < K) {
                const int co = k / 9, r = k - co * 9;
                v = w[((int64_t)co * sh.Cin + n) * 9 + r];
            }
            Bs[kl][nl] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CBK; ++kk) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 32 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 8 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int mm = m0 + ty + 32 * i;
        if (mm >= M) continue;
        const int im = mm / (sh.H * sh.W);
        const int rem = mm - im * sh.H * sh.W;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx + 8 * j;
            if (n >= N) continue;
            const int64_t off = (int64_t)im * sh.x_img_stride + (int64_t)n * sh.H * sh.W + rem;
            T v = acc[i][j];
            if (mask && !(mask[off] > T(0))) v = T(0);
            dx[off] = v;
        }
    }
}

// Weight gradient, split over the pixel reduction: rows = Cout, cols = Cin*9 + 1
// (the last column is the bias gradient), partial sums per split in `work`.
constexpr int WBM = 32, WBN = 64, WBK = 32;
template <typename T>
__global__ void __launch_bounds__(NT) conv_wgrad_kernel(ConvShape sh, const T* __restrict__ dy, const T* __restrict__ x,
                                                        T* __restrict__ work, int chunk) {
    SQ_KERNEL_ENTRY();
    __shared__ T As[WBK][WBM + 4];
    __shared__ T Bs[WBK][WBN + 4];
    const int tid = threadIdx.x;
    const int M = sh.Cout, N = sh.Cin * 9 + 1;
    const int P = sh.nimg * sh.OH * sh.OW;
    const int n0 = blockIdx.x * WBN, m0 = blockIdx.y * WBM;
    const int p_begin = blockIdx.z * chunk, p_end = min(P, p_begin + chunk);
    const int tx = tid % 16, ty = tid / 16;   // 16 x 4 cols, 16 x 2 rows
    T acc[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
    const int64_t oplane = (int64_t)sh.OH * sh.OW, iplane = (int64_t)sh.H * sh.W;
    for (int k0 = p_begin; k0 < p_end; k0 += WBK) {
        // A: dy[co, pixel]; pixel fastest across threads
        for (int e = tid; e < WBK * WBM; e += NT) {
            const int kl = e % WBK, ml = e / WBK;
            const int p = k0 + kl, co = m0 + ml;
            T v = T(0);
            if (p < p_end && co < M) {
                const int img = p / (int)oplane;
                const int rem = p - img * (int)oplane;
                v = dy[(int64_t)img * sh.y_img_stride + co * oplane + rem];
            }
            As[kl][ml] = v;
        }
        // B: x[ci, oy*s+ky, ox*s+kx] for col j = (ci, ky, kx); pixel fastest
        for (int e = tid; e < WBK * WBN; e += NT) {
            const int kl = e % WBK, nl = e / WBK;
            const int p = k0 + kl, j = n0 + nl;
            T v = T(0);
            if (p < p_end && j < N) {
                if (j == N - 1) {
                    v = T(1);
                } else {
                    const int img = p / (int)oplane;
                    const int rem = p - img * (int)oplane;
                    const int oy = rem / sh.OW, ox = rem - oy * sh.OW;
                    const int ci = j / 9, r = j - ci * 9, ky = r / 3, kx = r - ky * 3;
                    v = x[(int64_t)img * sh.x_img_stride + ci * iplane + (int64_t)(oy * sh.stride + ky) * sh.W +
                          ox * sh.stride + kx];
                }
            }
            Bs[kl][nl] = v;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < WBK; ++kk) {
            T a[2], b[4];
#pragma unroll
            for (int i = 0; i < 2; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
        }
        __syncthreads();
    }
    T* out = work + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int co = m0 + ty + 16 * i;
        if (co >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int col = n0 + tx + 16 * j;
            if (col < N) out[(int64_t)co * N + col] = acc[i][j];
        }
    }
}

// Weight gradient of a layer with 32 outputs and at most 31 input taps (Cin * 9 + 1 <= 32
// columns with the bias), i.e. the encoder's first convolution: 128 threads, thread t
// owns output rows 2 (t / 8), 2 (t / 8) + 1 and columns 4 (t % 8) .. + 3.  Per tile of 64
// pixels every thread issues all of its gathers (16 of dy, 16 of x) before storing them,
// transposed into padded shared memory (pixel fastest), then accumulates over the tile's
// pixels in order.  Partial sums per split in `work`, as for conv_wgrad_kernel.  PHWC: dy
// is read as the padded-HWC BF16 gradient (grid (OH + 4) x (OW + 4), 32 channels), one
// 16-byte chunk of 8 channels per load, instead of FP32 planes (the same values: BF16
// widens exactly).
constexpr int kW0Tile = 64;
template <bool PHWC>
__global__ void __launch_bounds__(128) conv_wgrad_c32_kernel(ConvShape sh, const void* __restrict__ dy_v,
                                                             const float* __restrict__ x, float* __restrict__ work,
                                                             int chunk) {
    SQ_KERNEL_ENTRY();
    __shared__ float dys[32][kW0Tile + 1];   // [co][pixel]
    __shared__ float xs[32][kW0Tile + 1];    // [column][pixel]; column N - 1 is the bias (1)
    const int t = threadIdx.x;
    const int N = sh.Cin * 9 + 1;
    const int P = sh.nimg * sh.OH * sh.OW;
    const int oplane = sh.OH * sh.OW;
    const int64_t iplane = (int64_t)sh.H * sh.W;
    const int p_begin = blockIdx.x * chunk, p_end = min(P, p_begin + chunk);
    const int cg = t / 8, jg = t % 8;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    const float* dy = static_cast<const float*>(dy_v);
    const __nv_bfloat16* dyp = static_cast<const __nv_bfloat16*>(dy_v);
    const int wpo = sh.OW + 4;
    const int64_t pimg = (int64_t)(sh.OH + 4) * wpo * 32;
    // every gather of this thread is for pixel pl = t % 64 of the tile; its x gathers are for
    // columns jb + 2u, whose input offsets do not depend on the tile
    const int pl_t = t % kW0Tile, jb = t / kW0Tile;
    int xoff[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int j = jb + 2 * u;
        const int ci = j / 9, r = j - ci * 9, ky = r / 3, kx = r - ky * 3;
        xoff[u] = j < N - 1 ? (int)(ci * iplane) + ky * sh.W + kx : 0;
    }
    float vd[16], vx[16];
    uint4 vq[2];
    // the next tile's loads are issued before the current tile is computed
    auto gather = [&](int k0) {
        const int p = k0 + pl_t;
        const bool in = p < p_end;
        const int img = in ? p / oplane : 0, rem = in ? p - img * oplane : 0;
        const int oy = rem / sh.OW, ox = rem - oy * sh.OW;
        if (PHWC) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int cc = jb + 2 * u;   // (t + 128 u) / 64
                vq[u] = in ? *reinterpret_cast<const uint4*>(dyp + (int64_t)img * pimg +
                                                              ((int64_t)(oy + 2) * wpo + ox + 2) * 32 + cc * 8)
                           : make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int co = jb + 2 * u;
                vd[u] = in ? dy[(int64_t)img * sh.y_img_stride + (int64_t)co * oplane + rem] : 0.f;
            }
        }
        const float* xb = x + (int64_t)img * sh.x_img_stride + (int64_t)(oy * sh.stride) * sh.W + ox * sh.stride;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int j = jb + 2 * u;
            vx[u] = (in && j < N - 1) ? xb[xoff[u]] : ((in && j == N - 1) ? 1.f : 0.f);
        }
    };
    if (p_begin < p_end) gather(p_begin);
    for (int k0 = p_begin; k0 < p_end; k0 += kW0Tile) {
        __syncthreads();   // the previous tile has been consumed
        if (PHWC) {
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int e = t + u * 128;
                const uint32_t w4[4] = {vq[u].x, vq[u].y, vq[u].z, vq[u].w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {   // a BF16 value is the upper half of its FP32 value
                    const uint32_t wv = w4[k / 2];
                    dys[(e / kW0Tile) * 8 + k][e % kW0Tile] = __uint_as_float((k & 1) ? (wv & 0xFFFF0000u) : (wv << 16));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int e = t + u * 128;
            if (!PHWC) dys[e / kW0Tile][e % kW0Tile] = vd[u];
            xs[e / kW0Tile][e % kW0Tile] = vx[u];
        }
        __syncthreads();
        if (k0 + kW0Tile < p_end) gather(k0 + kW0Tile);
        const int np = min(kW0Tile, p_end - k0);
#pragma unroll 4
        for (int pl = 0; pl < np; ++pl) {
            const float d0 = dys[2 * cg][pl], d1 = dys[2 * cg + 1][pl];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float xv = xs[4 * jg + k][pl];
                acc[0][k] = fmaf(d0, xv, acc[0][k]);
                acc[1][k] = fmaf(d1, xv, acc[1][k]);
            }
        }
    }
    float* out = work + (int64_t)blockIdx.x * 32 * N;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int col = 4 * jg + k;
            if (col < N) out[(2 * cg + i) * N + col] = acc[i][k];
        }
}

// 32 elements per block and 16 split groups: group g adds splits g, g + 16, ... in
// increasing order, then the group sums are added in group order (a fixed order).
constexpr int kRedGroups = 16;
template <typename T>
__global__ void __launch_bounds__(32 * kRedGroups) wgrad_reduce_kernel(const T* __restrict__ work, int splits,
                                                                          int M, int N, T* __restrict__ dw,
                                                                          T* __restrict__ db) {
    SQ_KERNEL_ENTRY();
    __shared__ T part[kRedGroups][33];
    const int tx = threadIdx.x % 32, g = threadIdx.x / 32;
    const int64_t tot = (int64_t)M * N;
    const int e = blockIdx.x * 32 + tx;
    T s = T(0);
    if (e < tot) {
        int z = g;
        for (; z + 3 * kRedGroups < splits; z += 4 * kRedGroups) {   // four splits' loads in flight
            T v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = work[(int64_t)(z + u * kRedGroups) * tot + e];
#pragma unroll
            for (int u = 0; u < 4; ++u) s += v[u];
        }
        for (; z < splits; z += kRedGroups) s += work[(int64_t)z * tot + e];
    }
    part[g][tx] = s;
    __syncthreads();
    if (g != 0 || e >= tot) return;
    T a = T(0);
#pragma unroll
    for (int k = 0; k < kRedGroups; ++k) a += part[k][tx];
    const int co = e / N, col = e - co * N;
    if (col == N - 1) db[co] = a;
    else dw[(int64_t)co * (N - 1) + col] = a;
}

int wgrad_splits(const ConvShape& sh) {
    const int P = sh.nimg * sh.OH * sh.OW;
    const int tiles = ((sh.Cin * 9 + 1 + WBN - 1) / WBN) * ((sh.Cout + WBM - 1) / WBM);
    int splits = std::max(1, (2 * 152 + tiles - 1) / tiles);
    splits = std::min(splits, std::max(1, P / (4 * WBK)));
    return splits;
}
}  // namespace

template <typename T>
void launch_conv_fwd(const ConvShape& sh, const T* x, const T* w, const T* b, T* y, bool relu, cudaStream_t s) {
    const int M = sh.nimg * sh.OH * sh.OW;
    if (M == 0) return;
    dim3 grid((M + CBM - 1) / CBM, (sh.Cout + CBN - 1) / CBN);
    launch_k(conv_fwd_kernel<T>, dim3(grid), dim3(NT), 0, s, sh, x, w, b, y, relu ? 1 : 0);
}
template <typename T>
void launch_conv_dgrad(const ConvShape& sh, const T* dy, const T* w, T* dx, const T* mask, cudaStream_t s) {
    const int M = sh.nimg * sh.H * sh.W;
    if (M == 0) return;
    dim3 grid((M + CBM - 1) / CBM, (sh.Cin + CBN - 1) / CBN);
    launch_k(conv_dgrad_kernel<T>, dim3(grid), dim3(NT), 0, s, sh, dy, w, dx, mask);
}
int64_t conv_wgrad_workspace(const ConvShape& sh) {
    return (int64_t)wgrad_splits(sh) * sh.Cout * (sh.Cin * 9 + 1);
}
template <typename T>
void launch_conv_wgrad(const ConvShape& sh, const T* dy, const T* x, T* dw, T* db, T* work, cudaStream_t s) {
    const int P = sh.nimg * sh.OH * sh.OW;
    const int splits = wgrad_splits(sh);
    const int chunk = (P + splits - 1) / splits;
    const int N = sh.Cin * 9 + 1;
    if (std::is_same<T, float>::value && sh.Cout == 32 && N <= 32)
        launch_k(conv_wgrad_c32_kernel<false>, dim3(splits), dim3(128), 0, s, sh, (const void*)dy, (const float*)x,
                 (float*)work, chunk);
    else
        launch_k(conv_wgrad_kernel<T>, dim3((N + WBN - 1) / WBN, (sh.Cout + WBM - 1) / WBM, splits), dim3(NT), 0, s,
                 sh, dy, x, work, chunk);
    const int tot = sh.Cout * N;
    launch_k(wgrad_reduce_kernel<T>, dim3((tot + 31) / 32), dim3(32 * kRedGroups), 0, s, work, splits, sh.Cout, N, dw,
             db);
}

int launch_conv_wgrad_phwc(const ConvShape& sh, const __nv_bfloat16* dy_phwc, const float* x, float* dw, float* db,
                           float* work, cudaStream_t s) {
    const int P = sh.nimg * sh.OH * sh.OW;
    const int N = sh.Cin * 9 + 1;
    if (sh.Cout != 32 || N > 32) return -1;
    const int splits = wgrad_splits(sh);
    const int chunk = (P + splits - 1) / splits;
    launch_k(conv_wgrad_c32_kernel<true>, dim3(splits), dim3(128), 0, s, sh, (const void*)dy_phwc, x, work, chunk);
    launch_k(wgrad_reduce_kernel<float>, dim3((sh.Cout * N + 31) / 32), dim3(32 * kRedGroups), 0, s, work, splits,
             sh.Cout, N, dw, db);
    return 0;
}

template void launch_conv_fwd<float>(const ConvShape&, const float*, const float*, const float*, float*, bool, cudaStream_t);
template void launch_conv_fwd<double>(const ConvShape&, const double*, const double*, const double*, double*, bool, cudaStream_t);
template void launch_conv_dgrad<float>(const ConvShape&, const float*, const float*, float*, const float*, cudaStream_t);
template void launch_conv_dgrad<double>(const ConvShape&, const double*, const double*, double*, const double*, cudaStream_t);
template void launch_conv_wgrad<float>(const ConvShape&, const float*, const float*, float*, float*, float*, cudaStream_t);
template void launch_conv_wgrad<double>(const ConvShape&, const double*, const double*, double*, double*, double*, cudaStream_t);

}  // namespace sq
