// LayerNorm, categorical (C51) target and loss, tanh-Gaussian head, temperature
// step, Adam and polyak.  All FP32; every reduction runs in a fixed order so a
// replayed graph reproduces an eager run bit for bit.
#include "sq_kernels.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace sq {

namespace {
constexpr int kMaxLn = 8;
template <typename P> struct Batch { P p[kMaxLn]; int n; };

// ---------------------------------------------------------------- LayerNorm
// One warp per row: mean, variance (two passes over the row), affine, optional ReLU.
// Rows up to 32 * kVpt wide are held in registers (all loads issued before any use).
constexpr int kVpt = 16;

__global__ void ln_fwd_kernel(Batch<LnProblem> b, int relu, float eps) {
    SQ_KERNEL_ENTRY();
    const int warps = blockDim.x / 32;
    const int lane = threadIdx.x % 32;
    int gw = blockIdx.x * warps + threadIdx.x / 32;
    int pi = 0;
    while (pi < b.n && gw >= b.p[pi].rows) { gw -= b.p[pi].rows; ++pi; }
    if (pi >= b.n) return;
    const LnProblem& P = b.p[pi];
    const float* x = P.pre + (int64_t)gw * P.ld_pre;
    float* y = P.out + (int64_t)gw * P.ld_out;
    if (P.n <= 32 * kVpt) {
        // the row and its affine parameters are loaded together, before any use
        float xv[kVpt], gv[kVpt], bv[kVpt];
#pragma unroll
        for (int k = 0; k < kVpt; ++k) {
            const int j = lane + 32 * k;
            xv[k] = j < P.n ? x[j] : 0.f;
            gv[k] = j < P.n ? P.g[j] : 0.f;
            bv[k] = j < P.n ? P.beta[j] : 0.f;
        }
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < kVpt; ++k) s += xv[k];
        const float mean = warp_sum(s) / (float)P.n;
        float q = 0.f;
#pragma unroll
        for (int k = 0; k < kVpt; ++k) {
            const int j = lane + 32 * k;
            const float d = j < P.n ? xv[k] - mean : 0.f;
            q += d * d;
        }
        const float var = warp_sum(q) / (float)P.n;
        const float rstd = 1.0f / sqrtf(var + eps);
#pragma unroll
        for (int k = 0; k < kVpt; ++k) {
            const int j = lane + 32 * k;
            if (j >= P.n) break;
            float v = (xv[k] - mean) * rstd * gv[k] + bv[k];
            if (relu) v = fmaxf(v, 0.f);
            y[j] = v;
            if (P.out_bf) P.out_bf[(int64_t)gw * P.ld_out_bf + j] = __float2bfloat16_rn(v);
        }
        if (lane == 0) { P.mean[gw] = mean; P.rstd[gw] = rstd; }
        return;
    }
    float s = 0.f;
    for (int j = lane; j < P.n; j += 32) s += x[j];
    const float mean = warp_sum(s) / (float)P.n;
    float q = 0.f;
    for (int j = lane; j < P.n; j += 32) { const float d = x[j] - mean; q += d * d; }
    const float var = warp_sum(q) / (float)P.n;
    const float rstd = 1.0f / sqrtf(var + eps);
    for (int j = lane; j < P.n; j += 32) {
        float v = (x[j] - mean) * rstd * P.g[j] + P.beta[j];
        if (relu) v = fmaxf(v, 0.f);
        y[j] = v;
        if (P.out_bf) P.out_bf[(int64_t)gw * P.ld_out_bf + j] = __float2bfloat16_rn(v);
    }
    if (lane == 0) { P.mean[gw] = mean; P.rstd[gw] = rstd; }
}

// LayerNorm backward: dpre = rstd (dxh - mean(dxh) - xh mean(dxh xh)), dxh = dn g.
// One warp per row, 8 rows per block, all rows of a block from one problem.  When column
// sums are wanted, each warp also stores its row's dn xh, dn and dpre in shared memory and
// the block adds its 8 rows in warp order into a partial row of `part`; the block that
// finishes last for a problem (ticket counter) then adds the partial rows in block order,
// so the sums do not depend on which block finished when.
struct LnBwdBatch {
    LnBwdProblem p[kMaxLn];
    int block_start[kMaxLn + 1];
    int64_t part_off[kMaxLn];
    int n;
    float* part;
    unsigned* tickets;   // one per problem, zero between launches
};
constexpr int kLnRows = 8;

__global__ void __launch_bounds__(256) ln_bwd_row_kernel(LnBwdBatch b, int want_cols) {
    SQ_KERNEL_ENTRY();
    extern __shared__ float acc[];   // [8 warps][3][n] when want_cols
    int pi = 0;
    while (pi + 1 < b.n && (int)blockIdx.x >= b.block_start[pi + 1]) ++pi;
    const LnBwdProblem& P = b.p[pi];
    const int lb = blockIdx.x - b.block_start[pi];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int row = lb * kLnRows + warp;
    const bool cols = want_cols && (P.dg || P.dbeta || P.dbias) && !P.terms;
    float* tx = P.terms ? P.terms + (int64_t)row * P.n : nullptr;                  // dn xh of this row
    float* tn = P.terms ? P.terms + ((int64_t)P.rows + row) * P.n : nullptr;       // dn of this row
    float* my = acc + (size_t)warp * 3 * P.n;
    if (row < P.rows && P.n <= 32 * kVpt) {
        const float* dout = P.dout + (int64_t)row * P.ld_dout;
        const float* out = P.out ? P.out + (int64_t)row * P.ld_out : nullptr;
        const float* pre = P.pre + (int64_t)row * P.ld_pre;
        const float mean = P.mean[row], rstd = P.rstd[row];
        float dn[kVpt], xh[kVpt], gg[kVpt];
#pragma unroll
        for (int k = 0; k < kVpt; ++k) {
            const int j = lane + 32 * k;
            const bool in = j < P.n;
            const float d = in ? dout[j] : 0.f;
            const float o = (in && out) ? out[j] : 1.f;
            dn[k] = (out && !(o > 0.f)) ? 0.f : d;
            xh[k] = in ? (pre[j] - mean) * rstd : 0.f;
            gg[k] = in ? P.g[j] : 0.f;
        }
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int k = 0; k < kVpt; ++k) {
            const float dxh = dn[k] * gg[k];
            s1 += dxh;
            s2 += dxh * xh[k];
        }
        const float m1 = warp_sum(s1) / (float)P.n;
        const float m2 = warp_sum(s2) / (float)P.n;
        float* dpre = P.dpre + (int64_t)row * P.ld_dpre;
#pragma unroll
        for (int k = 0; k < kVpt; ++k) {
            const int j = lane + 32 * k;
            if (j >= P.n) break;
            const float v = rstd * (dn[k] * gg[k] - m1 - xh[k] * m2);
            dpre[j] = v;
            if (P.dpre_bf) P.dpre_bf[(int64_t)row * P.ld_dpre_bf + j] = __float2bfloat16_rn(v);
            if (cols) {
                my[j] = dn[k] * xh[k];
                my[P.n + j] = dn[k];
                my[2 * P.n + j] = v;
            }
            if (tx) { tx[j] = dn[k] * xh[k]; tn[j] = dn[k]; }
        }
    } else if (row < P.rows) {
        const float* dout = P.dout + (int64_t)row * P.ld_dout;
        const float* out = P.out ? P.out + (int64_t)row * P.ld_out : nullptr;
        const float* pre = P.pre + (int64_t)row * P.ld_pre;
        const float mean = P.mean[row], rstd = P.rstd[row];
        float s1 = 0.f, s2 = 0.f;
        for (int j = lane; j < P.n; j += 32) {
            const float dn = (out && !(out[j] > 0.f)) ? 0.f : dout[j];
            const float dxh = dn * P.g[j];
            const float xh = (pre[j] - mean) * rstd;
            s1 += dxh;
            s2 += dxh * xh;
        }
        const float m1 = warp_sum(s1) / (float)P.n;
        const float m2 = warp_sum(s2) / (float)P.n;
        float* dpre = P.dpre + (int64_t)row * P.ld_dpre;
        for (int j = lane; j < P.n; j += 32) {
            const float dn = (out && !(out[j] > 0.f)) ? 0.f : dout[j];
            const float xh = (pre[j] - mean) * rstd;
            const float v = rstd * (dn * P.g[j] - m1 - xh * m2);
            dpre[j] = v;
            if (P.dpre_bf) P.dpre_bf[(int64_t)row * P.ld_dpre_bf + j] = __float2bfloat16_rn(v);
            if (cols) {
                my[j] = dn * xh;
                my[P.n + j] = dn;
                my[2 * P.n + j] = v;
            }
            if (tx) { tx[j] = dn * xh; tn[j] = dn; }
        }
    } else if (cols) {
        for (int j = lane; j < P.n; j += 32) { my[j] = 0.f; my[P.n + j] = 0.f; my[2 * P.n + j] = 0.f; }
    }
    if (!cols) return;
    __syncthreads();
    float* part = b.part + b.part_off[pi];
    for (int j = threadIdx.x; j < 3 * P.n; j += blockDim.x) {
        float t = 0.f;
        for (int w = 0; w < kLnRows; ++w) t += acc[(size_t)w * 3 * P.n + j];
        part[(int64_t)lb * 3 * P.n + j] = t;
    }
    // publish this block's partial row, then take a ticket
    __shared__ int last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int blocks = b.block_start[pi + 1] - b.block_start[pi];
        last = atomicAdd(&b.tickets[pi], 1u) == (unsigned)(blocks - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int blocks = b.block_start[pi + 1] - b.block_start[pi];
    for (int j = threadIdx.x; j < P.n; j += blockDim.x) {
        float sg = 0.f, sb = 0.f, sd = 0.f;
        int k = 0;
        for (; k + 8 <= blocks; k += 8) {   // eight partial rows' loads in flight, added in order
            float g8[8], b8[8], d8[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float* pk = part + (int64_t)(k + u) * 3 * P.n;
                g8[u] = __ldcg(pk + j);
                b8[u] = __ldcg(pk + P.n + j);
                d8[u] = __ldcg(pk + 2 * P.n + j);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) { sg += g8[u]; sb += b8[u]; sd += d8[u]; }
        }
        for (; k < blocks; ++k) {
            const float* pk = part + (int64_t)k * 3 * P.n;
            sg += __ldcg(pk + j);
            sb += __ldcg(pk + P.n + j);
            sd += __ldcg(pk + 2 * P.n + j);
        }
        if (P.dg) P.dg[j] = sg;
        if (P.dbeta) P.dbeta[j] = sb;
        if (P.dbias) P.dbias[j] = sd;
    }
    if (threadIdx.x == 0) b.tickets[pi] = 0u;
}

constexpr int kColX = 32, kColY = 16, kMaxCol = 16;
struct ColBatch { ColSumProblem p[kMaxCol]; int n; };
__global__ void __launch_bounds__(kColX * kColY) colsum_kernel(ColBatch b) {
    SQ_KERNEL_ENTRY();
    __shared__ float part[kColY][kColX + 1];
    const ColSumProblem& P = b.p[blockIdx.y];
    const int tx = threadIdx.x % kColX, ty = threadIdx.x / kColX;
    const int j = blockIdx.x * kColX + tx;
    float s = 0.f;
    if (j < P.n) {
        int r = ty;
        for (; r + 7 * kColY < P.rows; r += 8 * kColY) {   // eight rows' loads in flight, added in order
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = P.in[(int64_t)(r + u * kColY) * P.ld + j];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; r < P.rows; r += kColY) s += P.in[(int64_t)r * P.ld + j];
    }
    part[ty][tx] = s;
    __syncthreads();
    if (ty == 0 && j < P.n) {
        float a = 0.f;
        for (int y = 0; y < kColY; ++y) a += part[y][tx];
        P.out[j] = a;
    }
}

// Block-wide reductions for one row per block (blockDim = 128).
__device__ float block_sum(float v, float* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    float t = 0.f;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += sh[i];
    return t;
}

// ---------------------------------------------------------------- C51 target
// One warp per sample (kHeadRows samples a block, V atoms a lane: atom j = lane + 32 k):
// average of the target critics' categorical distributions, projected onto the fixed
// support as m_j = sum_i P_i max(0, 1 - |b_i - j|)   (linear interpolation between the
// two neighbouring atoms of b_i = (clip(r + gamma (1-d)(z_i - alpha log pi')) - v_min)/dz),
// the sum over i in order.  Clipped double Q: per sample the distribution of the target
// critic with the smaller mean (ties to critic 0).  MSE critics (K = 1): y = r + gamma
// (1-d)(Q_bar - alpha log pi') with Q_bar the average (or, with clipped double Q, the
// minimum) of the target outputs.  Softmax statistics by warp shuffles, no block barrier.
constexpr int kHeadRows = 8;

template <int V>
__global__ void __launch_bounds__(32 * kHeadRows) c51_target_kernel(C51TargetArgs a) {
    SQ_KERNEL_ENTRY();
    __shared__ float sp[kHeadRows][32 * V], sb[kHeadRows][32 * V];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int row = blockIdx.x * kHeadRows + warp;
    if (a.steps && blockIdx.x == 0 && threadIdx.x == 0) {
        const int act = (((uint64_t)*a.update_idx + 1) % (uint64_t)a.policy_freq) == 0;
        a.steps[0] += 1;
        a.steps[2] += 1;
        a.steps[1] += act;
        *a.do_actor = act;
    }
    if (row >= a.B) return;
    const float alpha = a.log_alpha ? expf(*a.log_alpha) : a.alpha_value;
    const float r = a.r[row], nd = 1.0f - a.d[row], lp = a.logp_next[row];
    if (a.mse) {
        if (lane == 0) {
            float qb = a.cdq ? INFINITY : 0.f;
            for (int e = 0; e < a.E; ++e) {
                const float q = a.logits_bar[(int64_t)e * a.B + row];
                qb = a.cdq ? fminf(qb, q) : qb + q;
            }
            if (!a.cdq) qb /= (float)a.E;
            a.m[row] = r + a.gamma * nd * (qb - alpha * lp);
        }
        return;
    }
    const int K = a.K;
    const float dz = (a.v_max - a.v_min) / (float)(K - 1);
    int pick = -1;   // clipped double Q: the critic whose distribution is used
    if (a.cdq) {
        float best = INFINITY;
        for (int e = 0; e < a.E; ++e) {
            const float* lg = a.logits_bar + ((int64_t)e * a.B + row) * K;
            float l[V], mx = -INFINITY;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int j = lane + 32 * k;
                l[k] = j < K ? lg[j] : -INFINITY;
                mx = fmaxf(mx, l[k]);
            }
            mx = warp_max(mx);
            float s = 0.f, q = 0.f;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int j = lane + 32 * k;
                if (j < K) {
                    const float p = expf(l[k] - mx);
                    s += p;
                    q += p * (a.v_min + (float)j * dz);
                }
            }
            s = warp_sum(s);
            q = warp_sum(q) / s;
            if (q < best) { best = q; pick = e; }
        }
    }
    float pb[V];
#pragma unroll
    for (int k = 0; k < V; ++k) pb[k] = 0.f;
    for (int e = 0; e < a.E; ++e) {
        if (pick >= 0 && e != pick) continue;
        const float* lg = a.logits_bar + ((int64_t)e * a.B + row) * K;
        float l[V], mx = -INFINITY;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int j = lane + 32 * k;
            l[k] = j < K ? lg[j] : -INFINITY;
            mx = fmaxf(mx, l[k]);
        }
        mx = warp_max(mx);
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (lane + 32 * k < K) s += expf(l[k] - mx);
        s = warp_sum(s);
#pragma unroll
        for (int k = 0; k < V; ++k)
            if (lane + 32 * k < K) pb[k] += expf(l[k] - mx) / s;
    }
    const float n_used = pick >= 0 ? 1.f : (float)a.E;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int j = lane + 32 * k;
        if (j >= K) break;
        const float zj = a.v_min + (float)j * dz;
        float tz = r + a.gamma * nd * (zj - alpha * lp);
        tz = fminf(fmaxf(tz, a.v_min), a.v_max);
        sp[warp][j] = pb[k] / n_used;
        sb[warp][j] = fminf(fmaxf((tz - a.v_min) / dz, 0.f), (float)(K - 1));
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int j = lane + 32 * k;
        if (j >= K) break;
        float acc = 0.f;
        for (int i = 0; i < K; ++i) acc += sp[warp][i] * fmaxf(0.f, 1.0f - fabsf(sb[warp][i] - (float)j));
        a.m[(int64_t)row * K + j] = acc;
    }
}

// ---------------------------------------------------------------- cross entropy
// One warp per (critic, sample): -sum m log softmax(l), d/dl = (softmax - m)/B, Q = sum softmax z.
// MSE critics (K = 1): loss (Q - y)^2 with y = m[row], dQ = 2 (Q - y) / B, Q = the output.
template <int V>
__global__ void __launch_bounds__(32 * kHeadRows) ce_kernel(CeArgs a) {
    SQ_KERNEL_ENTRY();
    const int lane = threadIdx.x % 32;
    const int er = blockIdx.x * kHeadRows + threadIdx.x / 32;   // e * B + row
    if (er >= a.E * a.B) return;
    const int row = er % a.B;
    const int K = a.K;
    const float* lg = a.logits + (int64_t)er * K;
    const float* m = a.m + (int64_t)row * K;
    if (a.mse) {
        if (lane == 0) {
            const float q = lg[0], err = q - m[0];
            const float g = 2.0f * err * a.scale;
            a.dlogits[er] = g;
            if (a.dlogits_bf) a.dlogits_bf[(int64_t)er * a.ld_bf] = __float2bfloat16_rn(g);
            a.row_loss[er] = err * err;
            a.row_q[er] = q;
        }
        return;
    }
    const float dz = (a.v_max - a.v_min) / (float)(K - 1);
    float l[V], mv[V], mx = -INFINITY;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int j = lane + 32 * k;
        l[k] = j < K ? lg[j] : -INFINITY;
        mv[k] = j < K ? m[j] : 0.f;
        mx = fmaxf(mx, l[k]);
    }
    mx = warp_max(mx);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < V; ++k)
        if (lane + 32 * k < K) s += expf(l[k] - mx);
    s = warp_sum(s);
    const float lse = mx + logf(s);
    float loss = 0.f, q = 0.f;
#pragma unroll
    for (int k = 0; k < V; ++k) {
        const int j = lane + 32 * k;
        if (j >= K) break;
        const float ls = l[k] - lse;
        const float p = expf(ls);
        loss -= mv[k] * ls;
        q += p * (a.v_min + (float)j * dz);
        const float g = (p - mv[k]) * a.scale;
        a.dlogits[(int64_t)er * K + j] = g;
        if (a.dlogits_bf) a.dlogits_bf[(int64_t)er * a.ld_bf + j] = __float2bfloat16_rn(g);
    }
    loss = warp_sum(loss);
    q = warp_sum(q);
    if (lane == 0) { a.row_loss[er] = loss; a.row_q[er] = q; }
}

// Actor objective through the critics, one warp per sample over all critics:
// Q_i = sum p z (or the scalar output), combined as the average (d/dQ_i = -1/(E B)) or,
// with clipped double Q, the minimum (d/dQ_i = -1/B for the smaller critic, ties to 0);
// categorical critics pass it on as dQ/dl_j = p_j (z_j - Q).
constexpr int kMaxE = 8;
template <int V>
__global__ void __launch_bounds__(32 * kHeadRows) actor_q_kernel(ActorQArgs a) {
    SQ_KERNEL_ENTRY();
    if (!*a.do_actor) return;
    const int lane = threadIdx.x % 32;
    const int row = blockIdx.x * kHeadRows + threadIdx.x / 32;
    if (row >= a.B) return;
    const int K = a.K;
    const float dz = a.mse ? 0.f : (a.v_max - a.v_min) / (float)(K - 1);
    float qv[kMaxE], mxv[kMaxE], sv[kMaxE];
#pragma unroll
    for (int e = 0; e < kMaxE; ++e) {
        if (e >= a.E) break;
        const float* lg = a.logits + ((int64_t)e * a.B + row) * K;
        if (a.mse) {
            qv[e] = lg[0];
        } else {
            float l[V], mx = -INFINITY;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int j = lane + 32 * k;
                l[k] = j < K ? lg[j] : -INFINITY;
                mx = fmaxf(mx, l[k]);
            }
            mx = warp_max(mx);
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < V; ++k)
                if (lane + 32 * k < K) s += expf(l[k] - mx);
            s = warp_sum(s);
            float q = 0.f;
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const int j = lane + 32 * k;
                if (j < K) q += expf(l[k] - mx) / s * (a.v_min + (float)j * dz);
            }
            qv[e] = warp_sum(q);
            mxv[e] = mx;
            sv[e] = s;
        }
        if (lane == 0) a.row_q[(int64_t)e * a.B + row] = qv[e];
    }
    int pick = -1;
    if (a.cdq) {
        pick = 0;
#pragma unroll
        for (int e = 1; e < kMaxE; ++e)
            if (e < a.E && qv[e] < qv[pick]) pick = e;
    }
#pragma unroll
    for (int e = 0; e < kMaxE; ++e) {
        if (e >= a.E) break;
        const float dq = pick < 0 ? -1.0f / (float)(a.E * a.B) : (e == pick ? -1.0f / (float)a.B : 0.f);
        const int64_t er = (int64_t)e * a.B + row;
        if (a.mse) {
            if (lane == 0) {
                a.dlogits[er] = dq;
                if (a.dlogits_bf) a.dlogits_bf[er * a.ld_bf] = __float2bfloat16_rn(dq);
            }
            continue;
        }
        const float* lg = a.logits + er * K;
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const int j = lane + 32 * k;
            if (j >= K) break;
            const float p = expf(lg[j] - mxv[e]) / sv[e];
            const float g = dq * p * (a.v_min + (float)j * dz - qv[e]);
            a.dlogits[er * K + j] = g;
            if (a.dlogits_bf) a.dlogits_bf[er * a.ld_bf + j] = __float2bfloat16_rn(g);
        }
    }
}

// ---------------------------------------------------------------- tanh-Gaussian head
__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// log_std = lo + (hi-lo)/2 (tanh(raw)+1); u = mu + std eps; a = tanh(u);
// log pi = sum_k [-eps^2/2 - log_std - log(2 pi)/2 - 2 (log 2 - u - softplus(-2u))].
__global__ void actor_head_kernel(ActorHeadArgs a) {
    SQ_KERNEL_ENTRY();
    const int row = a.row0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.rows) return;
    const bool tgt = row < a.B;
    const int el = tgt ? row : row - a.B;
    const uint64_t u = a.update_idx ? (uint64_t)*a.update_idx : 0;
    const float* o = a.out + (int64_t)row * a.ld_out;
    float lp = 0.f;
    for (int k = 0; k < a.A; ++k) {
        const float eps = a.eps_in ? a.eps_in[(int64_t)row * a.A + k]
                                   : normal_draw(a.seed, (uint32_t)el, tgt ? kStreamEpsTarget : kStreamEpsActor, u, k);
        const float mu = o[k], raw = o[a.A + k];
        const float ls = a.lo + 0.5f * (a.hi - a.lo) * (tanhf(raw) + 1.0f);
        const float sd = expf(ls);
        const float uu = mu + sd * eps;
        const float act = tanhf(uu);
        lp += -0.5f * eps * eps - ls - 0.91893853320467274f - 2.0f * (0.69314718055994531f - uu - softplusf(-2.0f * uu));
        if (a.eps) a.eps[(int64_t)row * a.A + k] = eps;
        if (tgt) {
            a.a_dst0[(int64_t)row * a.ld0 + k] = act;
            if (a.a_dst0_h) a.a_dst0_h[(int64_t)row * a.ld0_h + k] = __float2bfloat16_rn(act);
        } else {
            a.a_dst1[(int64_t)el * a.ld1 + k] = act;
            if (a.a_dst1_h) a.a_dst1_h[(int64_t)el * a.ld1_h + k] = __float2bfloat16_rn(act);
        }
    }
    a.logp[row] = lp;
}

// Reparameterised backward: du = da (1 - a^2) + dlogp 2a; dlog_std = du std eps - dlogp;
// draw = dlog_std (hi-lo)/2 (1 - tanh(raw)^2).
__global__ void actor_head_bwd_kernel(ActorHeadBwdArgs a) {
    SQ_KERNEL_ENTRY();
    if (a.do_actor && !*a.do_actor) return;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.B) return;
    const float dlogp = a.dlogp_rows ? a.dlogp_rows[row] : expf(*a.log_alpha) / (float)a.B;
    const float* o = a.out + (int64_t)row * a.ld_out;
    for (int k = 0; k < a.A; ++k) {
        const float eps = a.eps[(int64_t)row * a.A + k];
        const float mu = o[k], raw = o[a.A + k];
        const float th = tanhf(raw);
        const float sd = expf(a.lo + 0.5f * (a.hi - a.lo) * (th + 1.0f));
        const float act = tanhf(mu + sd * eps);
        const int64_t ldd = a.ld_da ? a.ld_da : a.A;
        float dq = a.da[(int64_t)row * ldd + k];
        if (a.da2) dq += a.da2[(int64_t)row * ldd + k];
        const float du = dq * (1.0f - act * act) + dlogp * 2.0f * act;
        const float dls = du * sd * eps - dlogp;
        const float draw = dls * 0.5f * (a.hi - a.lo) * (1.0f - th * th);
        a.dout[(int64_t)row * 2 * a.A + k] = du;
        a.dout[(int64_t)row * 2 * a.A + a.A + k] = draw;
        if (a.dout_bf) {
            a.dout_bf[(int64_t)row * a.ld_dout_bf + k] = __float2bfloat16_rn(du);
            a.dout_bf[(int64_t)row * a.ld_dout_bf + a.A + k] = __float2bfloat16_rn(draw);
        }
    }
}

// Inference head: tanh(mu) or tanh(mu + std eps) with eps from the request key.
__global__ void act_head_kernel(ActHeadArgs a) {
    SQ_KERNEL_ENTRY();
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= a.rows) return;
    const int q = a.row_req[row];
    const int rr = a.row_in_req[row];
    const float* o = a.out + (int64_t)row * a.ld_out;
    float* dst = a.req_actions[q] + (int64_t)rr * a.A;
    const bool mean_mode = a.req_mode[q] != 0;
    const uint64_t key = a.req_key[q];
    for (int k = 0; k < a.A; ++k) {
        float uu = o[k];
        if (!mean_mode) {
            const float eps = normal_draw(a.seed, (uint32_t)rr, kStreamAct, key, k);
            const float ls = a.lo + 0.5f * (a.hi - a.lo) * (tanhf(o[a.A + k]) + 1.0f);
            uu += expf(ls) * eps;
        }
        dst[k] = tanhf(uu);
    }
}

// ---------------------------------------------------------------- temperature + statistics
// stats layout: 0 critic loss, 1 actor loss, 2 alpha loss, 3 alpha, 4 q mean, 5 entropy, 6 update idx (as float bits: low), 7 unused
// Adam's bias correction 1 - beta^t, in FP32 as 1 - 2^(t log2 beta): a handful of
// instructions where the double-precision pow is a long chain on the FP64 units
// (relative error of beta^t ~ t |log2 beta| 2^-24, below 1e-4 while beta^t matters).
__device__ __forceinline__ float bias_correction(double beta, int t) {
    return 1.0f - exp2f((float)t * log2f((float)beta));
}

__global__ void alpha_kernel(AlphaArgs a) {
    SQ_KERNEL_ENTRY();
    __shared__ float red[32];
    float s = 0.f;
    for (int i = threadIdx.x; i < a.B; i += blockDim.x) s += a.logp_t[i];
    s = block_sum(s, red);
    if (threadIdx.x != 0) return;
    const float mean_logp = s / (float)a.B;
    const float alpha = expf(*a.log_alpha);
    const float loss = -alpha * (mean_logp + a.target_entropy);
    const float g = loss;                       // d/d log_alpha of -exp(la) c
    const int t = a.steps[2];
    const float mm = (float)a.b1 * *a.m + (float)(1.0 - a.b1) * g;
    const float vv = (float)a.b2 * *a.v + (float)(1.0 - a.b2) * g * g;
    *a.m = mm;
    *a.v = vv;
    const float bc1 = bias_correction(a.b1, t);
    const float bc2 = bias_correction(a.b2, t);
    const float la = *a.log_alpha - (float)a.lr * (mm / bc1) / (sqrtf(vv / bc2) + (float)a.eps);
    *a.log_alpha = la;
    a.stats[2] = loss;
    a.stats[3] = expf(la);
    a.stats[5] = -mean_logp;
}

__global__ void stats_kernel(StatsArgs a) {
    SQ_KERNEL_ENTRY();
    __shared__ float red[32];
    const int n = a.E * a.B;
    float l = 0.f, q = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) { l += a.row_loss[i]; q += a.row_q[i]; }
    l = block_sum(l, red);
    q = block_sum(q, red);
    float al = 0.f;
    const bool act = *a.do_actor != 0;
    if (act) {
        const float alpha = expf(*a.log_alpha);
        for (int i = threadIdx.x; i < a.B; i += blockDim.x) {
            float qm = a.cdq ? INFINITY : 0.f;
            for (int e = 0; e < a.E; ++e) {
                const float q = a.row_q_actor[e * a.B + i];
                qm = a.cdq ? fminf(qm, q) : qm + q;
            }
            al += alpha * a.logp_t[i] - (a.cdq ? qm : qm / (float)a.E);
        }
    }
    al = block_sum(al, red);
    if (threadIdx.x == 0) {
        a.stats[0] = l / (float)a.B;
        a.stats[1] = act ? al / (float)a.B : NAN;
        a.stats[4] = q / (float)n;
        const int64_t u = *a.update_idx;
        a.stats[6] = __int_as_float((int)(u & 0xffffffff));
        a.stats[7] = __int_as_float((int)(u >> 32));
        *a.update_idx = u + 1;
    }
}

// ---------------------------------------------------------------- Adam and polyak
// One Adam step; ibc1, ibc2 the reciprocals of the bias corrections 1 - beta^t (one
// division and one square root an element).  Every operation's rounding is spelled out,
// so an element gets the same bits whichever code path (four a thread or one) takes it.
__device__ __forceinline__ float adam_one(float p, float g, float& m, float& v, float b1, float b2, float c1, float c2,
                                          float lr, float ep, float ibc1, float ibc2) {
    m = __fmaf_rn(b1, m, __fmul_rn(c1, g));
    v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(c2, g), g));
    const float step = __fdiv_rn(__fmul_rn(lr, __fmul_rn(m, ibc1)), __fadd_rn(__fsqrt_rn(__fmul_rn(v, ibc2)), ep));
    return __fsub_rn(p, step);
}

// Row tasks of an elementwise pass over [0, n) of a parameter range: each weight matrix
// with a BF16 copy is walked by its rows (a row's element c lands at dst[r ld + c]), the
// elements between and after the matrices in rows of kPlainCols.  A block takes one row:
// no per-element search for the copy an element belongs to.
constexpr int kPlainCols = 1024, kMaxRowRanges = 2 * kMaxBfSeg + 1;
// threads of a row task: rows of the heads are 101 to 2,592 elements long
constexpr int kRowThreads = 128;
struct RowRange {
    int64_t off, len;             // elements [off, off + len) of the range
    int cols;                     // row length (the last row may be shorter: len)
    int row0;                     // first row task of this range
    int64_t ld, ldt;              // row strides of the copies
    __nv_bfloat16* dst;           // BF16 copy of the updated value (or null)
    __nv_bfloat16* tdst;          // BF16 copy of the updated target (or null)
};
struct RowPlan { RowRange r[kMaxRowRanges]; int n, rows; };

__device__ __forceinline__ float polyak_one(float t, float s, float keep, float tau) {
    return __fmaf_rn(keep, t, tau * s);
}

// Adam over one row task (with the polyak of the target copy when a.target is set).
// Rows whose FP32 arrays share one 16-byte alignment go by float4: the first elements up
// to the boundary and the last ones past the final whole vector one a thread, the rest
// four a thread (the BF16 copies as pairs where their row offset is even); rows whose
// arrays are aligned differently go one element a thread.  Every element takes the same
// arithmetic either way.
__global__ void __launch_bounds__(kRowThreads) adam_rows_kernel(const __grid_constant__ AdamArgs a,
                                                        const __grid_constant__ RowPlan plan) {
    SQ_KERNEL_ENTRY();
    if (a.enable && !*a.enable) return;
    const int t = *a.step;
    const float ibc1 = 1.0f / bias_correction(a.b1, t), ibc2 = 1.0f / bias_correction(a.b2, t);
    const float b1 = (float)a.b1, b2 = (float)a.b2, lr = (float)a.lr, ep = (float)a.eps;
    const float c1 = (float)(1.0 - a.b1), c2 = (float)(1.0 - a.b2);
    const float tau = a.tau, keep = 1.0f - a.tau;
    int k = 0;
    while (k + 1 < plan.n && (int)blockIdx.x >= plan.r[k + 1].row0) ++k;
    const RowRange& R = plan.r[k];
    const int r = (int)blockIdx.x - R.row0;
    const int64_t base = R.off + (int64_t)r * R.cols;
    const int lim = (int)min((int64_t)R.cols, R.len - (int64_t)r * R.cols);
    float* __restrict__ p = a.p + base;
    const float* __restrict__ g = a.g + base;
    float* __restrict__ m = a.m + base;
    float* __restrict__ v = a.v + base;
    float* __restrict__ tg = a.target ? a.target + base : nullptr;
    __nv_bfloat16* dst = R.dst ? R.dst + (int64_t)r * R.ld : nullptr;
    __nv_bfloat16* tdst = R.tdst ? R.tdst + (int64_t)r * R.ldt : nullptr;
    __nv_bfloat16* pbf = a.p_bf ? a.p_bf + base : nullptr;
    auto one = [&](int c) {
        const float np = adam_one(p[c], g[c], m[c], v[c], b1, b2, c1, c2, lr, ep, ibc1, ibc2);
        p[c] = np;
        if (dst) dst[c] = __float2bfloat16_rn(np);
        if (pbf) pbf[c] = __float2bfloat16_rn(np);
        if (tg) {
            const float nt = polyak_one(tg[c], np, keep, tau);
            tg[c] = nt;
            if (tdst) tdst[c] = __float2bfloat16_rn(nt);
        }
    };
    const uintptr_t ap = reinterpret_cast<uintptr_t>(p);
    const bool same = ((ap ^ reinterpret_cast<uintptr_t>(g)) & 15) == 0 &&
                      ((ap ^ reinterpret_cast<uintptr_t>(m)) & 15) == 0 &&
                      ((ap ^ reinterpret_cast<uintptr_t>(v)) & 15) == 0 &&
                      (!tg || ((ap ^ reinterpret_cast<uintptr_t>(tg)) & 15) == 0) && (ap & 3) == 0;
    if (!same) {
        for (int c = threadIdx.x; c < lim; c += blockDim.x) one(c);
        return;
    }
    const int head = min(lim, (int)(((16 - (ap & 15)) & 15) / 4));
    const int nvec = (lim - head) / 4;
    const int tail0 = head + 4 * nvec;
    // the scalar elements: [0, head) and [tail0, lim), at most three of each, taken by the
    // first threads after their vectors (their loads issued first, so that both are in flight)
    const int ns = head + (lim - tail0);
    const int cs = (int)threadIdx.x < head ? (int)threadIdx.x : tail0 + (int)threadIdx.x - head;
    float sp = 0.f, sg = 0.f, sm = 0.f, sv = 0.f, st = 0.f;
    if ((int)threadIdx.x < ns) {
        sp = p[cs]; sg = g[cs]; sm = m[cs]; sv = v[cs];
        if (tg) st = tg[cs];
    }
    // a BF16 copy takes pairs where its first vector element is 4-byte aligned (then every
    // one is: vectors are 8 bytes of BF16 apart)
    auto even = [&](const __nv_bfloat16* d) { return d && (reinterpret_cast<uintptr_t>(d + head) & 3) == 0; };
    const bool pr_dst = even(dst), pr_pbf = even(pbf), pr_tdst = even(tdst);
    auto put4 = [&](__nv_bfloat16* d, bool pairs, int c, const float (&x)[4]) {
        if (pairs) {
            *reinterpret_cast<__nv_bfloat162*>(d + c) = __floats2bfloat162_rn(x[0], x[1]);
            *reinterpret_cast<__nv_bfloat162*>(d + c + 2) = __floats2bfloat162_rn(x[2], x[3]);
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) d[c + u] = __float2bfloat16_rn(x[u]);
        }
    };
    for (int q = threadIdx.x; q < nvec; q += blockDim.x) {
        const int c = head + 4 * q;
        const float4 p4 = *reinterpret_cast<const float4*>(p + c);
        const float4 g4 = *reinterpret_cast<const float4*>(g + c);
        float4 m4 = *reinterpret_cast<const float4*>(m + c);
        float4 v4 = *reinterpret_cast<const float4*>(v + c);
        const float4 t4 = tg ? *reinterpret_cast<const float4*>(tg + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        float np[4], nt[4];
        np[0] = adam_one(p4.x, g4.x, m4.x, v4.x, b1, b2, c1, c2, lr, ep, ibc1, ibc2);
        np[1] = adam_one(p4.y, g4.y, m4.y, v4.y, b1, b2, c1, c2, lr, ep, ibc1, ibc2);
        np[2] = adam_one(p4.z, g4.z, m4.z, v4.z, b1, b2, c1, c2, lr, ep, ibc1, ibc2);
        np[3] = adam_one(p4.w, g4.w, m4.w, v4.w, b1, b2, c1, c2, lr, ep, ibc1, ibc2);
        *reinterpret_cast<float4*>(p + c) = make_float4(np[0], np[1], np[2], np[3]);
        *reinterpret_cast<float4*>(m + c) = m4;
        *reinterpret_cast<float4*>(v + c) = v4;
        if (dst) put4(dst, pr_dst, c, np);
        if (pbf) put4(pbf, pr_pbf, c, np);
        if (tg) {
            nt[0] = polyak_one(t4.x, np[0], keep, tau);
            nt[1] = polyak_one(t4.y, np[1], keep, tau);
            nt[2] = polyak_one(t4.z, np[2], keep, tau);
            nt[3] = polyak_one(t4.w, np[3], keep, tau);
            *reinterpret_cast<float4*>(tg + c) = make_float4(nt[0], nt[1], nt[2], nt[3]);
            if (tdst) put4(tdst, pr_tdst, c, nt);
        }
    }
    if ((int)threadIdx.x < ns) {
        const float np = adam_one(sp, sg, sm, sv, b1, b2, c1, c2, lr, ep, ibc1, ibc2);
        p[cs] = np; m[cs] = sm; v[cs] = sv;
        if (dst) dst[cs] = __float2bfloat16_rn(np);
        if (pbf) pbf[cs] = __float2bfloat16_rn(np);
        if (tg) {
            const float nt = polyak_one(st, np, keep, tau);
            tg[cs] = nt;
            if (tdst) tdst[cs] = __float2bfloat16_rn(nt);
        }
    }
}

// Polyak alone (target <- (1 - tau) target + tau src) over the same row tasks.
__global__ void __launch_bounds__(kRowThreads) polyak_rows_kernel(const __grid_constant__ PolyakArgs a,
                                                          const __grid_constant__ RowPlan plan) {
    SQ_KERNEL_ENTRY();
    const float tau = a.tau, keep = 1.0f - a.tau;
    int k = 0;
    while (k + 1 < plan.n && (int)blockIdx.x >= plan.r[k + 1].row0) ++k;
    const RowRange& R = plan.r[k];
    const int r = (int)blockIdx.x - R.row0;
    const int64_t base = R.off + (int64_t)r * R.cols;
    const int lim = (int)min((int64_t)R.cols, R.len - (int64_t)r * R.cols);
    float* __restrict__ tg = a.target + base;
    const float* __restrict__ sv = a.src + base;
    __nv_bfloat16* tdst = R.tdst ? R.tdst + (int64_t)r * R.ldt : nullptr;
    constexpr int U = 4;
    for (int c0 = threadIdx.x; c0 < lim; c0 += U * blockDim.x) {
        float tv[U], xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * blockDim.x;
            if (c < lim) { tv[u] = tg[c]; xv[u] = sv[c]; }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * blockDim.x;
            if (c >= lim) break;
            const float nt = polyak_one(tv[u], xv[u], keep, tau);
            tg[c] = nt;
            if (tdst) tdst[c] = __float2bfloat16_rn(nt);
        }
    }
    if (a.update_idx && blockIdx.x == 0 && threadIdx.x == 0) *a.update_idx += 1;
}

// The row tasks of [0, n) with the matrices seg (copies dst) and, matching them one for
// one, tseg (copies tdst; may be empty).  False if the segments overlap or leave [0, n).
bool row_plan(int64_t n, const BfSeg* seg, int n_seg, const BfSeg* tseg, int n_tseg, RowPlan* plan) {
    std::memset(plan, 0, sizeof(*plan));
    int order[kMaxBfSeg];
    for (int i = 0; i < n_seg; ++i) order[i] = i;
    std::sort(order, order + n_seg, [&](int x, int y) { return seg[x].off < seg[y].off; });
    int64_t cur = 0;
    int rows = 0;
    auto add = [&](int64_t off, int64_t len, int cols, int64_t ld, __nv_bfloat16* dst, int64_t ldt,
                   __nv_bfloat16* tdst) {
        if (len <= 0) return true;
        if (plan->n >= kMaxRowRanges) return false;
        RowRange& R = plan->r[plan->n++];
        R.off = off; R.len = len; R.cols = cols; R.row0 = rows; R.ld = ld; R.ldt = ldt; R.dst = dst; R.tdst = tdst;
        rows += (int)((len + cols - 1) / cols);
        return true;
    };
    for (int q = 0; q < n_seg; ++q) {
        const int i = order[q];
        const BfSeg& S = seg[i];
        const int64_t len = (int64_t)S.rows * S.cols;
        if (S.off < cur || S.off + len > n || S.cols < 1) return false;
        if (!add(cur, S.off - cur, kPlainCols, 0, nullptr, 0, nullptr)) return false;
        const bool t = i < n_tseg;
        if (t && (tseg[i].off != S.off || tseg[i].rows != S.rows || tseg[i].cols != S.cols)) return false;
        if (!add(S.off, len, S.cols, S.ld, S.dst, t ? tseg[i].ld : 0, t ? tseg[i].dst : nullptr)) return false;
        cur = S.off + len;
    }
    if (!add(cur, n - cur, kPlainCols, 0, nullptr, 0, nullptr)) return false;
    plan->rows = rows;
    return true;
}

// dx = dy where y > 0, else 0 (the ReLU's backward given its output y).
template <typename T>
__global__ void relu_bwd_kernel(int64_t n, const T* __restrict__ dy, const T* __restrict__ y, T* __restrict__ dx) {
    SQ_KERNEL_ENTRY();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dx[i] = y[i] > T(0) ? dy[i] : T(0);
}

template <typename P> Batch<P> make_batch(const P* p, int n) {
    Batch<P> b{};
    b.n = n;
    for (int i = 0; i < n; ++i) b.p[i] = p[i];
    return b;
}
}  // namespace

void launch_ln_fwd(const LnProblem* p, int n, bool relu, float eps, cudaStream_t s) {
    for (int base = 0; base < n; base += kMaxLn) {
        const int cnt = std::min(kMaxLn, n - base);
        auto b = make_batch(p + base, cnt);
        int rows = 0;
        for (int i = 0; i < cnt; ++i) rows += b.p[i].rows;
        if (rows) launch_k(ln_fwd_kernel, dim3((rows + 7) / 8), dim3(256), 0, s, b, relu ? 1 : 0, eps);
    }
}
void ln_prepare() {
    cudaFuncSetAttribute(ln_bwd_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kLnRows * 3 * 2048 * 4);
}

int64_t ln_bwd_workspace(const LnBwdProblem* p, int n) {
    int64_t w = 0;
    for (int i = 0; i < n; ++i) w += (int64_t)((p[i].rows + kLnRows - 1) / kLnRows) * 3 * p[i].n;
    return w + kLnTickets;
}

void launch_ln_bwd(const LnBwdProblem* p, int n, float* work, cudaStream_t s) {
    for (int base = 0; base < n; base += kMaxLn) {
        const int cnt = std::min(kMaxLn, n - base);
        LnBwdBatch b{};
        b.n = cnt;
        int blocks = 0, cols = 0;
        int64_t off = 0;
        bool any_col = false;
        for (int i = 0; i < cnt; ++i) {
            b.p[i] = p[base + i];
            b.block_start[i] = blocks;
            b.part_off[i] = off;
            const int nb = (b.p[i].rows + kLnRows - 1) / kLnRows;
            blocks += nb;
            off += (int64_t)nb * 3 * b.p[i].n;
            cols = std::max(cols, b.p[i].n);
            any_col |= (b.p[i].dg || b.p[i].dbeta || b.p[i].dbias) && !b.p[i].terms;
        }
        b.block_start[cnt] = blocks;
        if (!blocks) continue;
        const bool want = any_col && work && cols <= 2048;
        const size_t smem = want ? (size_t)kLnRows * 3 * cols * sizeof(float) : 0;
        // the tickets sit in the first kLnTickets words of the workspace, the partials after them
        b.tickets = reinterpret_cast<unsigned*>(work);
        b.part = work ? work + kLnTickets : nullptr;
        launch_k(ln_bwd_row_kernel, dim3(blocks), dim3(32 * kLnRows), smem, s, b, want ? 1 : 0);
    }
}
void launch_ln_bwd_cols(const LnBwdProblem* p, int n, cudaStream_t s) {
    std::vector<ColSumProblem> cs;
    for (int i = 0; i < n; ++i) {
        const LnBwdProblem& q = p[i];
        if (!q.terms || q.rows <= 0) continue;
        if (q.dg) cs.push_back(ColSumProblem{q.rows, q.n, q.terms, q.n, q.dg});
        if (q.dbeta) cs.push_back(ColSumProblem{q.rows, q.n, q.terms + (int64_t)q.rows * q.n, q.n, q.dbeta});
        if (q.dbias) cs.push_back(ColSumProblem{q.rows, q.n, q.dpre, q.ld_dpre, q.dbias});
    }
    if (!cs.empty()) launch_colsum(cs.data(), (int)cs.size(), s);
}

void launch_colsum(const ColSumProblem* p, int n, cudaStream_t s) {
    for (int base = 0; base < n; base += kMaxCol) {
        const int cnt = std::min(kMaxCol, n - base);
        ColBatch b{};
        b.n = cnt;
        for (int i = 0; i < cnt; ++i) b.p[i] = p[base + i];
        int cols = 0;
        for (int i = 0; i < cnt; ++i) cols = std::max(cols, b.p[i].n);
        if (cols) launch_k(colsum_kernel, dim3(dim3((cols + kColX - 1) / kColX, cnt)), dim3(kColX * kColY), 0, s, b);
    }
}
void launch_actor_head(const ActorHeadArgs& a, cudaStream_t s) {
    if (a.rows > a.row0) launch_k(actor_head_kernel, dim3((a.rows - a.row0 + 127) / 128), dim3(128), 0, s, a);
}
void launch_actor_head_bwd(const ActorHeadBwdArgs& a, cudaStream_t s) {
    launch_k(actor_head_bwd_kernel, dim3((a.B + 127) / 128), dim3(128), 0, s, a);
}
// atoms per lane: 4 up to 128 atoms, 8 up to 256 (the most a configuration takes)
void launch_c51_target(const C51TargetArgs& a, cudaStream_t s) {
    const dim3 g((a.B + kHeadRows - 1) / kHeadRows), t(32 * kHeadRows);
    if (a.K <= 128) launch_k(c51_target_kernel<4>, g, t, 0, s, a);
    else launch_k(c51_target_kernel<8>, g, t, 0, s, a);
}
void launch_ce(const CeArgs& a, cudaStream_t s) {
    const dim3 g((a.E * a.B + kHeadRows - 1) / kHeadRows), t(32 * kHeadRows);
    if (a.K <= 128) launch_k(ce_kernel<4>, g, t, 0, s, a);
    else launch_k(ce_kernel<8>, g, t, 0, s, a);
}
void launch_actor_q(const ActorQArgs& a, cudaStream_t s) {
    const dim3 g((a.B + kHeadRows - 1) / kHeadRows), t(32 * kHeadRows);
    if (a.K <= 128) launch_k(actor_q_kernel<4>, g, t, 0, s, a);
    else launch_k(actor_q_kernel<8>, g, t, 0, s, a);
}
void launch_alpha_step(const AlphaArgs& a, cudaStream_t s) { launch_k(alpha_kernel, dim3(1), dim3(256), 0, s, a); }
void launch_stats(const StatsArgs& a, cudaStream_t s) { launch_k(stats_kernel, dim3(1), dim3(256), 0, s, a); }
int launch_adam(const AdamArgs& a, cudaStream_t s) {
    if (a.n <= 0) return 0;
    RowPlan plan;
    if (!row_plan(a.n, a.seg, a.n_seg, a.tseg, a.target ? a.n_tseg : 0, &plan) || plan.rows < 1) return -1;
    launch_k(adam_rows_kernel, dim3(plan.rows), dim3(kRowThreads), 0, s, a, plan);
    return 0;
}
template <typename T>
void launch_relu_bwd(int64_t n, const T* dy, const T* y, T* dx, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    launch_k(relu_bwd_kernel<T>, dim3(blocks), dim3(256), 0, s, n, dy, y, dx);
}
template void launch_relu_bwd<float>(int64_t, const float*, const float*, float*, cudaStream_t);
template void launch_relu_bwd<double>(int64_t, const double*, const double*, double*, cudaStream_t);

int launch_polyak(const PolyakArgs& a, cudaStream_t s) {
    if (a.n <= 0) return 0;
    // the copies are described by the target segments alone: pass them as both lists
    RowPlan plan;
    if (!row_plan(a.n, a.seg, a.n_seg, a.seg, a.n_seg, &plan) || plan.rows < 1) return -1;
    launch_k(polyak_rows_kernel, dim3(plan.rows), dim3(kRowThreads), 0, s, a, plan);
    return 0;
}
void launch_act_head(const ActHeadArgs& a, cudaStream_t s) {
    if (a.rows > 0) launch_k(act_head_kernel, dim3((a.rows + 127) / 128), dim3(128), 0, s, a);
}

}  // namespace sq
