// LayerNorm, categorical (C51) target and loss, tanh-Gaussian head, temperature
// step, Adam and polyak.  All FP32; every reduction runs in a fixed order so a
// replayed graph reproduces an eager run bit for bit.
#include "sq_kernels.cuh"

#include <algorithm>

namespace sq {

namespace {
constexpr int kMaxLn = 8;
template <typename P> struct Batch { P p[kMaxLn]; int n; };

// ---------------------------------------------------------------- LayerNorm
// One warp per row: mean, variance (two passes over the row), affine, optional ReLU.
__global__ void ln_fwd_kernel(Batch<LnProblem> b, int relu, float eps) {
    const int warps = blockDim.x / 32;
    const int lane = threadIdx.x % 32;
    int gw = blockIdx.x * warps + threadIdx.x / 32;
    int pi = 0;
    while (pi < b.n && gw >= b.p[pi].rows) { gw -= b.p[pi].rows; ++pi; }
    if (pi >= b.n) return;
    const LnProblem& P = b.p[pi];
    const float* x = P.pre + (int64_t)gw * P.ld_pre;
    float s = 0.f;
    for (int j = lane; j < P.n; j += 32) s += x[j];
    const float mean = warp_sum(s) / (float)P.n;
    float q = 0.f;
    for (int j = lane; j < P.n; j += 32) { const float d = x[j] - mean; q += d * d; }
    const float var = warp_sum(q) / (float)P.n;
    const float rstd = 1.0f / sqrtf(var + eps);
    float* y = P.out + (int64_t)gw * P.ld_out;
    for (int j = lane; j < P.n; j += 32) {
        float v = (x[j] - mean) * rstd * P.g[j] + P.beta[j];
        if (relu) v = fmaxf(v, 0.f);
        y[j] = v;
        if (P.out_bf) P.out_bf[(int64_t)gw * P.ld_out_bf + j] = __float2bfloat16_rn(v);
    }
    if (lane == 0) { P.mean[gw] = mean; P.rstd[gw] = rstd; }
}

// Row part of the LayerNorm backward: dpre = rstd (dxh - mean(dxh) - xh mean(dxh xh)), dxh = dn g.
__global__ void ln_bwd_row_kernel(Batch<LnBwdProblem> b) {
    const int warps = blockDim.x / 32;
    const int lane = threadIdx.x % 32;
    int gw = blockIdx.x * warps + threadIdx.x / 32;
    int pi = 0;
    while (pi < b.n && gw >= b.p[pi].rows) { gw -= b.p[pi].rows; ++pi; }
    if (pi >= b.n) return;
    const LnBwdProblem& P = b.p[pi];
    const float* dout = P.dout + (int64_t)gw * P.ld_dout;
    const float* out = P.out ? P.out + (int64_t)gw * P.ld_out : nullptr;
    const float* pre = P.pre + (int64_t)gw * P.ld_pre;
    const float mean = P.mean[gw], rstd = P.rstd[gw];
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
    float* dpre = P.dpre + (int64_t)gw * P.ld_dpre;
    for (int j = lane; j < P.n; j += 32) {
        const float dn = (out && !(out[j] > 0.f)) ? 0.f : dout[j];
        const float xh = (pre[j] - mean) * rstd;
        const float v = rstd * (dn * P.g[j] - m1 - xh * m2);
        dpre[j] = v;
        if (P.dpre_bf) P.dpre_bf[(int64_t)gw * P.ld_dpre_bf + j] = __float2bfloat16_rn(v);
    }
}

// Column part: dg = sum dn xh, dbeta = sum dn, dbias = sum dpre.  Block (32 columns x
// 16 row slices): thread (x, y) sums rows y, y+16, ... in order, then the 16 slice
// sums are added in slice order, so the result does not depend on scheduling.
constexpr int kColX = 32, kColY = 16;
__global__ void __launch_bounds__(kColX * kColY) ln_bwd_col_kernel(Batch<LnBwdProblem> b) {
    __shared__ float part[3][kColY][kColX + 1];
    const LnBwdProblem& P = b.p[blockIdx.y];
    const int tx = threadIdx.x % kColX, ty = threadIdx.x / kColX;
    const int j = blockIdx.x * kColX + tx;
    float sg = 0.f, sb = 0.f, sd = 0.f;
    if (j < P.n) {
        for (int r = ty; r < P.rows; r += kColY) {
            const float o = P.out ? P.out[(int64_t)r * P.ld_out + j] : 1.f;
            const float dn = (P.out && !(o > 0.f)) ? 0.f : P.dout[(int64_t)r * P.ld_dout + j];
            const float xh = (P.pre[(int64_t)r * P.ld_pre + j] - P.mean[r]) * P.rstd[r];
            sg += dn * xh;
            sb += dn;
            if (P.dbias) sd += P.dpre[(int64_t)r * P.ld_dpre + j];
        }
    }
    part[0][ty][tx] = sg;
    part[1][ty][tx] = sb;
    part[2][ty][tx] = sd;
    __syncthreads();
    if (ty == 0 && j < P.n) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int y = 0; y < kColY; ++y) { a0 += part[0][y][tx]; a1 += part[1][y][tx]; a2 += part[2][y][tx]; }
        if (P.dg) P.dg[j] = a0;
        if (P.dbeta) P.dbeta[j] = a1;
        if (P.dbias) P.dbias[j] = a2;
    }
}

__global__ void __launch_bounds__(kColX * kColY) colsum_kernel(Batch<ColSumProblem> b) {
    __shared__ float part[kColY][kColX + 1];
    const ColSumProblem& P = b.p[blockIdx.y];
    const int tx = threadIdx.x % kColX, ty = threadIdx.x / kColX;
    const int j = blockIdx.x * kColX + tx;
    float s = 0.f;
    if (j < P.n)
        for (int r = ty; r < P.rows; r += kColY) s += P.in[(int64_t)r * P.ld + j];
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
__device__ float block_max(float v, float* sh) {
    v = warp_max(v);
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    float t = -INFINITY;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) t = fmaxf(t, sh[i]);
    return t;
}

constexpr int kMaxAtoms = 256;

// ---------------------------------------------------------------- C51 target
// One block per sample: average of the target critics' categorical
// distributions, projected onto the fixed support as
// m_j = sum_i P_i max(0, 1 - |b_i - j|)   (linear interpolation between the two
// neighbouring atoms of b_i = (clip(r + gamma (1-d)(z_i - alpha log pi')) - v_min)/dz).
__global__ void c51_target_kernel(C51TargetArgs a) {
    __shared__ float pbar[kMaxAtoms];
    __shared__ float bpos[kMaxAtoms];
    __shared__ float red[32];
    const int row = blockIdx.x;
    const float alpha = a.log_alpha ? expf(*a.log_alpha) : a.alpha_value;
    const float dz = (a.v_max - a.v_min) / (float)(a.K - 1);
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) pbar[j] = 0.f;
    for (int e = 0; e < a.E; ++e) {
        const float* lg = a.logits_bar + ((int64_t)e * a.B + row) * a.K;
        float mx = -INFINITY;
        for (int j = threadIdx.x; j < a.K; j += blockDim.x) mx = fmaxf(mx, lg[j]);
        mx = block_max(mx, red);
        float s = 0.f;
        for (int j = threadIdx.x; j < a.K; j += blockDim.x) s += expf(lg[j] - mx);
        s = block_sum(s, red);
        for (int j = threadIdx.x; j < a.K; j += blockDim.x) pbar[j] += expf(lg[j] - mx) / s;
    }
    const float r = a.r[row], nd = 1.0f - a.d[row], lp = a.logp_next[row];
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) {
        pbar[j] /= (float)a.E;
        const float zj = a.v_min + (float)j * dz;
        float tz = r + a.gamma * nd * (zj - alpha * lp);
        tz = fminf(fmaxf(tz, a.v_min), a.v_max);
        bpos[j] = fminf(fmaxf((tz - a.v_min) / dz, 0.f), (float)(a.K - 1));
    }
    __syncthreads();
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) {
        float acc = 0.f;
        for (int i = 0; i < a.K; ++i) acc += pbar[i] * fmaxf(0.f, 1.0f - fabsf(bpos[i] - (float)j));
        a.m[(int64_t)row * a.K + j] = acc;
    }
}

// ---------------------------------------------------------------- cross entropy
// One block per (critic, sample): -sum m log softmax(l), d/dl = (softmax - m)/B, Q = sum softmax z.
__global__ void ce_kernel(CeArgs a) {
    __shared__ float red[32];
    const int er = blockIdx.x;          // e * B + row
    const int row = er % a.B;
    const float* lg = a.logits + (int64_t)er * a.K;
    const float* m = a.m + (int64_t)row * a.K;
    const float dz = (a.v_max - a.v_min) / (float)(a.K - 1);
    float mx = -INFINITY;
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) mx = fmaxf(mx, lg[j]);
    mx = block_max(mx, red);
    float s = 0.f;
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) s += expf(lg[j] - mx);
    s = block_sum(s, red);
    const float lse = mx + logf(s);
    float loss = 0.f, q = 0.f;
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) {
        const float ls = lg[j] - lse;
        const float p = expf(ls);
        loss -= m[j] * ls;
        q += p * (a.v_min + (float)j * dz);
        const float g = (p - m[j]) * a.scale;
        a.dlogits[(int64_t)er * a.K + j] = g;
        if (a.dlogits_bf) a.dlogits_bf[(int64_t)er * a.ld_bf + j] = __float2bfloat16_rn(g);
    }
    loss = block_sum(loss, red);
    q = block_sum(q, red);
    if (threadIdx.x == 0) { a.row_loss[er] = loss; a.row_q[er] = q; }
}

// Actor objective through the critics: Q = sum p z, dQ/dl_j = p_j (z_j - Q),
// d(-mean_i Q_i / B)/dl = -(1/(E B)) p (z - Q).
__global__ void actor_q_kernel(ActorQArgs a) {
    if (!*a.do_actor) return;
    __shared__ float red[32];
    __shared__ float qs;
    const int er = blockIdx.x;
    const float* lg = a.logits + (int64_t)er * a.K;
    const float dz = (a.v_max - a.v_min) / (float)(a.K - 1);
    float mx = -INFINITY;
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) mx = fmaxf(mx, lg[j]);
    mx = block_max(mx, red);
    float s = 0.f;
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) s += expf(lg[j] - mx);
    s = block_sum(s, red);
    float q = 0.f;
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) q += expf(lg[j] - mx) / s * (a.v_min + (float)j * dz);
    q = block_sum(q, red);
    if (threadIdx.x == 0) { qs = q; a.row_q[er] = q; }
    __syncthreads();
    const float scale = -1.0f / (float)(a.E * a.B);
    for (int j = threadIdx.x; j < a.K; j += blockDim.x) {
        const float p = expf(lg[j] - mx) / s;
        const float g = scale * p * (a.v_min + (float)j * dz - qs);
        a.dlogits[(int64_t)er * a.K + j] = g;
        if (a.dlogits_bf) a.dlogits_bf[(int64_t)er * a.ld_bf + j] = __float2bfloat16_rn(g);
    }
}

// ---------------------------------------------------------------- tanh-Gaussian head
__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.f) + log1pf(expf(-fabsf(x))); }

// log_std = lo + (hi-lo)/2 (tanh(raw)+1); u = mu + std eps; a = tanh(u);
// log pi = sum_k [-eps^2/2 - log_std - log(2 pi)/2 - 2 (log 2 - u - softplus(-2u))].
__global__ void actor_head_kernel(ActorHeadArgs a) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
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
        if (tgt) a.a_dst0[(int64_t)row * a.ld0 + k] = act;
        else a.a_dst1[(int64_t)el * a.ld1 + k] = act;
    }
    a.logp[row] = lp;
}

// Reparameterised backward: du = da (1 - a^2) + dlogp 2a; dlog_std = du std eps - dlogp;
// draw = dlog_std (hi-lo)/2 (1 - tanh(raw)^2).
__global__ void actor_head_bwd_kernel(ActorHeadBwdArgs a) {
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
        const float du = a.da[(int64_t)row * ldd + k] * (1.0f - act * act) + dlogp * 2.0f * act;
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
__global__ void alpha_kernel(AlphaArgs a) {
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
    const float bc1 = (float)(1.0 - pow(a.b1, (double)t));
    const float bc2 = (float)(1.0 - pow(a.b2, (double)t));
    const float la = *a.log_alpha - (float)a.lr * (mm / bc1) / (sqrtf(vv / bc2) + (float)a.eps);
    *a.log_alpha = la;
    a.stats[2] = loss;
    a.stats[3] = expf(la);
    a.stats[5] = -mean_logp;
}

__global__ void stats_kernel(StatsArgs a) {
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
            float qm = 0.f;
            for (int e = 0; e < a.E; ++e) qm += a.row_q_actor[e * a.B + i];
            al += alpha * a.logp_t[i] - qm / (float)a.E;
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
__global__ void adam_kernel(AdamArgs a) {
    if (a.enable && !*a.enable) return;
    __shared__ float bc[2];
    if (threadIdx.x == 0) {
        const double t = (double)*a.step;
        bc[0] = (float)(1.0 - pow(a.b1, t));
        bc[1] = (float)(1.0 - pow(a.b2, t));
    }
    __syncthreads();
    const float b1 = (float)a.b1, b2 = (float)a.b2, lr = (float)a.lr, ep = (float)a.eps;
    const float c1 = (float)(1.0 - a.b1), c2 = (float)(1.0 - a.b2);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const float g = a.g[i];
        const float m = b1 * a.m[i] + c1 * g;
        const float v = b2 * a.v[i] + c2 * g * g;
        a.m[i] = m;
        a.v[i] = v;
        const float p = a.p[i] - lr * (m / bc[0]) / (sqrtf(v / bc[1]) + ep);
        a.p[i] = p;
        if (a.p_bf) a.p_bf[i] = __float2bfloat16_rn(p);
    }
}

__global__ void polyak_kernel(PolyakArgs a) {
    const float keep = 1.0f - a.tau;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
        a.target[i] = keep * a.target[i] + a.tau * a.src[i];
    if (a.update_idx && blockIdx.x == 0 && threadIdx.x == 0) *a.update_idx += 1;
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
        if (rows) ln_fwd_kernel<<<(rows + 7) / 8, 256, 0, s>>>(b, relu ? 1 : 0, eps);
    }
}
void launch_ln_bwd(const LnBwdProblem* p, int n, cudaStream_t s) {
    for (int base = 0; base < n; base += kMaxLn) {
        const int cnt = std::min(kMaxLn, n - base);
        auto b = make_batch(p + base, cnt);
        int rows = 0, cols = 0;
        bool any_col = false;
        for (int i = 0; i < cnt; ++i) {
            rows += b.p[i].rows;
            cols = std::max(cols, b.p[i].n);
            any_col |= b.p[i].dg || b.p[i].dbeta || b.p[i].dbias;
        }
        if (!rows) continue;
        ln_bwd_row_kernel<<<(rows + 7) / 8, 256, 0, s>>>(b);
        if (any_col) ln_bwd_col_kernel<<<dim3((cols + kColX - 1) / kColX, cnt), kColX * kColY, 0, s>>>(b);
    }
}
void launch_colsum(const ColSumProblem* p, int n, cudaStream_t s) {
    for (int base = 0; base < n; base += kMaxLn) {
        const int cnt = std::min(kMaxLn, n - base);
        auto b = make_batch(p + base, cnt);
        int cols = 0;
        for (int i = 0; i < cnt; ++i) cols = std::max(cols, b.p[i].n);
        if (cols) colsum_kernel<<<dim3((cols + kColX - 1) / kColX, cnt), kColX * kColY, 0, s>>>(b);
    }
}
void launch_actor_head(const ActorHeadArgs& a, cudaStream_t s) {
    actor_head_kernel<<<(a.rows + 127) / 128, 128, 0, s>>>(a);
}
void launch_actor_head_bwd(const ActorHeadBwdArgs& a, cudaStream_t s) {
    actor_head_bwd_kernel<<<(a.B + 127) / 128, 128, 0, s>>>(a);
}
void launch_c51_target(const C51TargetArgs& a, cudaStream_t s) { c51_target_kernel<<<a.B, 128, 0, s>>>(a); }
void launch_ce(const CeArgs& a, cudaStream_t s) { ce_kernel<<<a.E * a.B, 128, 0, s>>>(a); }
void launch_actor_q(const ActorQArgs& a, cudaStream_t s) { actor_q_kernel<<<a.E * a.B, 128, 0, s>>>(a); }
void launch_alpha_step(const AlphaArgs& a, cudaStream_t s) { alpha_kernel<<<1, 256, 0, s>>>(a); }
void launch_stats(const StatsArgs& a, cudaStream_t s) { stats_kernel<<<1, 256, 0, s>>>(a); }
void launch_adam(const AdamArgs& a, cudaStream_t s) {
    const int blocks = (int)std::min<int64_t>((a.n + 255) / 256, 152 * 8);
    if (a.n > 0) adam_kernel<<<blocks, 256, 0, s>>>(a);
}
void launch_polyak(const PolyakArgs& a, cudaStream_t s) {
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((a.n + 255) / 256, 152 * 8));
    polyak_kernel<<<blocks, 256, 0, s>>>(a);
}
void launch_act_head(const ActHeadArgs& a, cudaStream_t s) {
    if (a.rows > 0) act_head_kernel<<<(a.rows + 127) / 128, 128, 0, s>>>(a);
}

}  // namespace sq
