// The launch schedule of one Squint SAC update and its CUDA-graph capture.
//
// One update (Algorithm 1, inner loop) as issued here:
//   front end (a1-a4)      slots, shifts, squint of o_t and o_{t+1} (one launch)
//   encoder (a5)           conv stack on 2B frames (o_t with activations kept)
//   projections (a6)       four heads in one grouped GEMM + LayerNorm
//   target (a7-a9)         actor on z', tanh-Gaussian sample, target critics, C51 projection
//   critic step (a10-a12)  critics on (z, s, a), cross entropy, backward into critics,
//                          critic projection and encoder, Adam over the critic group
//   temperature (a13)      Adam on log alpha from log pi at s_t
//   actor step (a14-a15)   critics with updated weights on (z_sg, s, a~), backward to the
//                          action, tanh-Gaussian and actor MLP backward, Adam (actor group)
//   polyak (a16)           target critics <- (1-tau) target + tau critics
// Every launch reads its scalars (update index, step counts, alpha, actor flag)
// from device memory, so k updates are captured once as a graph and replayed.
#include "sq_internal.h"

#include <cmath>
#include <cstring>

using namespace sq;

namespace {

GemmProblem lin_fwd(const float* X, int64_t ldx, int rows, const float* W, const float* b, int in, int out, float* Y,
                    int64_t ldy) {
    GemmProblem p{};
    p.M = rows; p.N = out; p.K = in;
    p.A = X; p.sa_m = ldx; p.sa_k = 1;
    p.B = W; p.sb_n = in; p.sb_k = 1;
    p.C = Y; p.sc_m = ldy; p.sc_n = 1;
    p.bias = b;
    p.n_sum = 1;
    return p;
}
// dX[m, j] = sum_n dY[m, n] W[n, col0 + j], j < ncols
GemmProblem lin_dx(const float* dY, int64_t ldd, int rows, const float* W, int in, int out, int col0, int ncols,
                   float* dX, int64_t ldx) {
    GemmProblem p{};
    p.M = rows; p.N = ncols; p.K = out;
    p.A = dY; p.sa_m = ldd; p.sa_k = 1;
    p.B = W + col0; p.sb_n = 1; p.sb_k = in;
    p.C = dX; p.sc_m = ldx; p.sc_n = 1;
    p.n_sum = 1;
    return p;
}
// dW[n, j] = sum_m dY[m, n] X[m, j]
GemmProblem lin_dw(const float* dY, int64_t ldd, int rows, const float* X, int64_t ldx, int in, int out, float* dW) {
    GemmProblem p{};
    p.M = out; p.N = in; p.K = rows;
    p.A = dY; p.sa_m = 1; p.sa_k = ldd;
    p.B = X; p.sb_n = 1; p.sb_k = ldx;
    p.C = dW; p.sc_m = in; p.sc_n = 1;
    p.n_sum = 1;
    return p;
}

// Parameter pointer of set e: online params, or the target copy of the critic range.
struct PSet {
    const float* base;   // params or target
    int64_t shift;       // subtracted from canonical offsets
    const float* at(int64_t off) const { return base + (off - shift); }
};

void mlp_forward(MlpBufs& mb, const std::vector<Lin>* layers[], const PSet sets[], int E, const float* X, int64_t ldx,
                 int rows, float ln_eps, cudaStream_t s) {
    const int nh = (int)layers[0]->size() - 1;
    GemmProblem g[2];
    LnProblem lp[2];
    for (int l = 0; l <= nh; ++l) {
        for (int e = 0; e < E; ++e) {
            const Lin& ly = (*layers[e])[l];
            const float* in = l == 0 ? X : mb.post[l - 1] + (int64_t)e * rows * ly.in;
            const int64_t ldi = l == 0 ? ldx : ly.in;
            float* y = l < nh ? mb.pre[l] + (int64_t)e * rows * ly.out : mb.out + (int64_t)e * rows * ly.out;
            g[e] = lin_fwd(in, ldi, rows, sets[e].at(ly.w), sets[e].at(ly.b), ly.in, ly.out, y, ly.out);
        }
        launch_gemm<float>(g, E, kKK, s);
        if (l == nh) break;
        for (int e = 0; e < E; ++e) {
            const Lin& ly = (*layers[e])[l];
            LnProblem p{};
            p.rows = rows; p.n = ly.out;
            p.pre = mb.pre[l] + (int64_t)e * rows * ly.out; p.ld_pre = ly.out;
            p.g = sets[e].at(ly.g); p.beta = sets[e].at(ly.beta);
            p.out = mb.post[l] + (int64_t)e * rows * ly.out; p.ld_out = ly.out;
            p.mean = mb.mean[l] + (int64_t)e * rows; p.rstd = mb.rstd[l] + (int64_t)e * rows;
            lp[e] = p;
        }
        launch_ln_fwd(lp, E, true, ln_eps, s);
    }
}

// Backward through an MLP evaluated by E parameter sets (all in `params`).
// dout: [E, rows, n_out] (contiguous per set), rows offset `r0` into the stored activations.
// grads: null for input-gradient only.  dX (optional) = sum over sets of the input
// gradient restricted to columns [col0, col0 + ncols), masked by mask > 0 if given.
void mlp_backward(const MlpBufs& mb, int r0, const std::vector<Lin>* layers[], const float* params, float* grads,
                  int E, const float* X, int64_t ldx, int rows, const float* dout, std::vector<float*>& dpost,
                  std::vector<float*>& dpre, int col0, int ncols, float* dX, int64_t lddx, const float* mask,
                  int64_t ldmask, cudaStream_t s) {
    const int nh = (int)layers[0]->size() - 1;
    const int R = mb.rows;   // rows of the stored activations per set
    GemmProblem g[4];
    // output layer
    {
        int n = 0;
        for (int e = 0; e < E; ++e) {
            const Lin& ly = (*layers[e])[nh];
            const float* de = dout + (int64_t)e * rows * ly.out;
            const float* h = mb.post[nh - 1] + ((int64_t)e * R + r0) * ly.in;
            if (grads) g[n++] = lin_dw(de, ly.out, rows, h, ly.in, ly.in, ly.out, grads + ly.w);
        }
        if (n) launch_gemm<float>(g, n, kMN, s);
        if (grads) {
            ColSumProblem cs[2];
            for (int e = 0; e < E; ++e) {
                const Lin& ly = (*layers[e])[nh];
                cs[e] = ColSumProblem{rows, ly.out, dout + (int64_t)e * rows * ly.out, ly.out, grads + ly.b};
            }
            launch_colsum(cs, E, s);
        }
        for (int e = 0; e < E; ++e) {
            const Lin& ly = (*layers[e])[nh];
            g[e] = lin_dx(dout + (int64_t)e * rows * ly.out, ly.out, rows, params + ly.w, ly.in, ly.out, 0, ly.in,
                          dpost[nh - 1] + (int64_t)e * rows * ly.in, ly.in);
        }
        launch_gemm<float>(g, E, kKN, s);
    }
    for (int l = nh - 1; l >= 0; --l) {
        LnBwdProblem lb[2];
        for (int e = 0; e < E; ++e) {
            const Lin& ly = (*layers[e])[l];
            LnBwdProblem p{};
            p.rows = rows; p.n = ly.out;
            p.dout = dpost[l] + (int64_t)e * rows * ly.out; p.ld_dout = ly.out;
            p.out = mb.post[l] + ((int64_t)e * R + r0) * ly.out; p.ld_out = ly.out;
            p.pre = mb.pre[l] + ((int64_t)e * R + r0) * ly.out; p.ld_pre = ly.out;
            p.mean = mb.mean[l] + (int64_t)e * R + r0; p.rstd = mb.rstd[l] + (int64_t)e * R + r0;
            p.g = params + ly.g;
            p.dpre = dpre[l] + (int64_t)e * rows * ly.out; p.ld_dpre = ly.out;
            if (grads) { p.dg = grads + ly.g; p.dbeta = grads + ly.beta; p.dbias = grads + ly.b; }
            lb[e] = p;
        }
        launch_ln_bwd(lb, E, s);
        if (grads) {
            for (int e = 0; e < E; ++e) {
                const Lin& ly = (*layers[e])[l];
                const float* xin = l == 0 ? X : mb.post[l - 1] + ((int64_t)e * R + r0) * ly.in;
                const int64_t ldi = l == 0 ? ldx : ly.in;
                g[e] = lin_dw(dpre[l] + (int64_t)e * rows * ly.out, ly.out, rows, xin, ldi, ly.in, ly.out, grads + ly.w);
            }
            launch_gemm<float>(g, E, kMN, s);
        }
        if (l > 0) {
            for (int e = 0; e < E; ++e) {
                const Lin& ly = (*layers[e])[l];
                g[e] = lin_dx(dpre[l] + (int64_t)e * rows * ly.out, ly.out, rows, params + ly.w, ly.in, ly.out, 0, ly.in,
                              dpost[l - 1] + (int64_t)e * rows * ly.in, ly.in);
            }
            launch_gemm<float>(g, E, kKN, s);
        }
    }
    if (dX) {
        const Lin& l0 = (*layers[0])[0];
        GemmProblem p = lin_dx(dpre[0], l0.out, rows, params + l0.w, l0.in, l0.out, col0, ncols, dX, lddx);
        p.n_sum = E;
        p.a_sum = (int64_t)rows * l0.out;
        p.b_sum = E > 1 ? (*layers[1])[0].w - l0.w : 0;
        if (mask) { p.mask = mask; p.sm_m = ldmask; p.sm_n = 1; }
        launch_gemm<float>(&p, 1, kKN, s);
    }
}

void alloc_mlp(squint_handle* h, MlpBufs& mb, const std::vector<Lin>& layers, int E, int rows) {
    const int nh = (int)layers.size() - 1;
    mb.E = E;
    mb.rows = rows;
    mb.pre.resize(nh); mb.post.resize(nh); mb.mean.resize(nh); mb.rstd.resize(nh);
    for (int l = 0; l < nh; ++l) {
        mb.pre[l] = h->dalloc<float>((int64_t)E * rows * layers[l].out);
        mb.post[l] = h->dalloc<float>((int64_t)E * rows * layers[l].out);
        mb.mean[l] = h->dalloc<float>((int64_t)E * rows);
        mb.rstd[l] = h->dalloc<float>((int64_t)E * rows);
    }
    mb.out = h->dalloc<float>((int64_t)E * rows * layers[nh].out);
}

constexpr uint32_t kStateMagic = 0x54535153u;  // "SQST"

}  // namespace

int squint_handle::allocate() {
    const int B = c.batch, A = c.action_dim, K = c.atoms, E = 2;
    SQ_CK(this, cudaGetDevice(&device));
    const int64_t n = L.total;
    params = dalloc<float>(n); grads = dalloc<float>(n);
    adam_m = dalloc<float>(n); adam_v = dalloc<float>(n);
    target = dalloc<float>(L.target_n);
    policy_buf[0] = dalloc<float>(n);
    policy_buf[1] = dalloc<float>(n);
    d_update_idx = dalloc<int64_t>(1);
    d_steps = dalloc<int32_t>(4);
    d_do_actor = dalloc<int32_t>(1);
    d_stats = dalloc<float>((int64_t)c.max_k * 8);
    const int64_t img = (int64_t)c.obs_c * L.hs * L.ws;
    x2 = dalloc<float>(2 * B * img);
    sums = dalloc<uint16_t>(2 * B * img);
    idx2 = dalloc<int32_t>(2 * B);
    shift2 = dalloc<int32_t>(4 * B);
    for (const auto& cv : L.conv) conv_out.push_back(dalloc<float>((int64_t)2 * B * cv.cout * cv.oh * cv.ow));
    if (L.D > 0) {
        proj_pre = dalloc<float>((int64_t)5 * B * L.D);
        proj_mean = dalloc<float>(5 * B);
        proj_rstd = dalloc<float>(5 * B);
    }
    xa = dalloc<float>((int64_t)2 * B * L.da);
    xcbar = dalloc<float>((int64_t)B * L.dc);
    xc = dalloc<float>((int64_t)B * L.dc);
    xq = dalloc<float>((int64_t)B * L.dc);
    alloc_mlp(this, actor_mlp, L.actor, 1, 2 * B);
    alloc_mlp(this, tcrit_mlp, L.critic[0], E, B);
    alloc_mlp(this, crit_mlp, L.critic[0], E, B);
    alloc_mlp(this, qcrit_mlp, L.critic[0], E, B);
    logp = dalloc<float>(2 * B);
    eps = dalloc<float>(2 * B * A);
    m = dalloc<float>((int64_t)B * K);
    r = dalloc<float>(B);
    d = dalloc<float>(B);
    dlogits = dalloc<float>((int64_t)E * B * K);
    dlogits_q = dalloc<float>((int64_t)E * B * K);
    row_loss = dalloc<float>(E * B);
    row_q = dalloc<float>(E * B);
    row_q_actor = dalloc<float>(E * B);
    for (int l = 0; l < c.n_hidden; ++l) {
        const int w = std::max(c.hidden[l], 1);
        dpost.push_back(dalloc<float>((int64_t)E * B * w));
        dpre.push_back(dalloc<float>((int64_t)E * B * w));
    }
    dh = dalloc<float>((int64_t)B * L.zdim);
    if (L.D > 0) dproj = dalloc<float>((int64_t)B * L.D);
    dz = dalloc<float>((int64_t)B * L.feat);
    int64_t maxc = 0, maxw = 0;
    for (const auto& cv : L.conv) {
        maxc = std::max<int64_t>(maxc, (int64_t)B * cv.cout * cv.oh * cv.ow);
        maxc = std::max<int64_t>(maxc, (int64_t)B * cv.cin * cv.h * cv.w);
        ConvShape sh{B, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                     (int64_t)cv.cout * cv.oh * cv.ow};
        maxw = std::max(maxw, conv_wgrad_workspace(sh));
    }
    dconv_a = dalloc<float>(maxc);
    dconv_b = dalloc<float>(maxc);
    wgrad_work = dalloc<float>(maxw);
    da = dalloc<float>((int64_t)B * A);
    dout_a = dalloc<float>((int64_t)B * 2 * A);
    for (void* p : allocations)
        if (!p) { g_last_error = "device allocation failed"; return SQUINT_ENOMEM; }
    if (allocations.size() && !allocations.back()) return SQUINT_ENOMEM;
    if (cudaMallocHost(&h_stats, sizeof(float) * 8 * c.max_k) != cudaSuccess) return SQUINT_ENOMEM;
    SQ_CK(this, cudaStreamCreateWithFlags(&capture_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
        SQ_CK(this, cudaEventCreateWithFlags(&policy_ready[i], cudaEventDisableTiming));
        SQ_CK(this, cudaEventCreateWithFlags(&policy_released[i], cudaEventDisableTiming));
    }
    SQ_CK(this, cudaEventCreateWithFlags(&req_event, cudaEventDisableTiming));
    frontend_prepare((size_t)c.obs_c * c.obs_h * c.obs_w);

    std::vector<float> p;
    init_params_host(c, L, p);
    SQ_CK(this, cudaMemcpy(params, p.data(), n * sizeof(float), cudaMemcpyHostToDevice));
    SQ_CK(this, cudaMemset(grads, 0, n * sizeof(float)));
    SQ_CK(this, cudaMemset(adam_m, 0, n * sizeof(float)));
    SQ_CK(this, cudaMemset(adam_v, 0, n * sizeof(float)));
    SQ_CK(this, cudaMemcpy(target, params + L.critic_begin, L.target_n * sizeof(float), cudaMemcpyDeviceToDevice));
    SQ_CK(this, cudaMemset(d_update_idx, 0, sizeof(int64_t)));
    SQ_CK(this, cudaMemset(d_steps, 0, 4 * sizeof(int32_t)));
    SQ_CK(this, cudaMemset(d_do_actor, 0, sizeof(int32_t)));
    return after_param_change();
}

void squint_handle::release() {
    cudaDeviceSynchronize();
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    for (void* p : allocations) if (p) cudaFree(p);
    allocations.clear();
    if (h_stats) cudaFreeHost(h_stats);
    h_stats = nullptr;
    if (h_req) cudaFreeHost(h_req);
    h_req = nullptr;
    if (capture_stream) cudaStreamDestroy(capture_stream);
    capture_stream = nullptr;
    for (int i = 0; i < 2; ++i) {
        if (policy_ready[i]) cudaEventDestroy(policy_ready[i]);
        if (policy_released[i]) cudaEventDestroy(policy_released[i]);
        policy_ready[i] = policy_released[i] = nullptr;
    }
    if (req_event) cudaEventDestroy(req_event);
    req_event = nullptr;
    for (void* p : act_allocs) if (p) cudaFree(p);
    act_allocs.clear();
}

int squint_handle::after_param_change() {
    SQ_CK(this, cudaDeviceSynchronize());
    for (int i = 0; i < 2; ++i)
        SQ_CK(this, cudaMemcpy(policy_buf[i], params, L.total * sizeof(float), cudaMemcpyDeviceToDevice));
    ++policy_version;
    return SQUINT_OK;
}

void squint_handle::record_update(int j, cudaStream_t s, bool debug) {
    const int B = c.batch, A = c.action_dim, P = c.proprio_dim, K = c.atoms, E = 2;
    const int F = L.feat, Z = L.zdim, Dd = L.D, Dc = L.dc, Da = L.da;
    const float ln_eps = (float)c.ln_eps;
    float* W = params;
    float* G = grads;
    float* stats = d_stats + 8 * j;

    mark(s);
    // ---- a1-a4: minibatch, gathers, shift, squint
    FrontendArgs fa{};
    fa.obs = ring.obs; fa.proprio = ring.proprio; fa.action = ring.action; fa.reward = ring.reward; fa.done = ring.done;
    fa.n_slots = ring.n;
    fa.C = c.obs_c; fa.H = c.obs_h; fa.W = c.obs_w; fa.f = c.squint_f; fa.pad = c.shift_pad;
    fa.P = P; fa.A = A; fa.B = B;
    fa.seed = c.seed; fa.update_idx = d_update_idx;
    fa.x = x2; fa.x_bf = nullptr; fa.sums = debug ? sums : nullptr;
    fa.idx_out = idx2; fa.shift_out = shift2; fa.r_out = r; fa.d_out = d;
    fa.dst[0] = CopyDst{xc, Dc, Z, 0};
    fa.dst[1] = CopyDst{xc, Dc, Z + P, 2};
    fa.dst[2] = CopyDst{xq, Dc, Z, 0};
    fa.dst[3] = CopyDst{xa + (int64_t)B * Da, Da, Z, 0};
    fa.dst[4] = CopyDst{xa, Da, Z, 1};
    fa.dst[5] = CopyDst{xcbar, Dc, Z, 1};
    fa.n_dst = 6;
    fa.steps = d_steps; fa.do_actor = d_do_actor; fa.policy_freq = c.policy_freq;
    launch_frontend(fa, s);

    mark(s);
    // ---- a5: encoder on o_t (rows < B) and o_{t+1} (rows >= B)
    const float* in = x2;
    for (size_t l = 0; l < L.conv.size(); ++l) {
        const ConvL& cv = L.conv[l];
        ConvShape sh{2 * B, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                     (int64_t)cv.cout * cv.oh * cv.ow};
        launch_conv_fwd<float>(sh, in, W + cv.wo, W + cv.bo, conv_out[l], true, s);
        in = conv_out[l];
    }
    const float* z = conv_out.back();          // [2B, F]
    const float* z1 = z + (int64_t)B * F;

    mark(s);
    // ---- a6: per-head projections (or the flattened features straight into the heads)
    const PSet online{W, 0};
    const PSet tgt{target, L.critic_begin};
    if (Dd > 0) {
        GemmProblem g[4] = {
            lin_fwd(z1, F, B, W + L.aproj.w, W + L.aproj.b, F, Dd, proj_pre + 0 * (int64_t)B * Dd, Dd),
            lin_fwd(z1, F, B, tgt.at(L.cproj.w), tgt.at(L.cproj.b), F, Dd, proj_pre + 1 * (int64_t)B * Dd, Dd),
            lin_fwd(z, F, B, W + L.cproj.w, W + L.cproj.b, F, Dd, proj_pre + 2 * (int64_t)B * Dd, Dd),
            lin_fwd(z, F, B, W + L.aproj.w, W + L.aproj.b, F, Dd, proj_pre + 3 * (int64_t)B * Dd, Dd),
        };
        launch_gemm<float>(g, 4, kKK, s);
        LnProblem lp[4];
        const float* gs[4] = {W + L.aproj.g, tgt.at(L.cproj.g), W + L.cproj.g, W + L.aproj.g};
        const float* bs[4] = {W + L.aproj.beta, tgt.at(L.cproj.beta), W + L.cproj.beta, W + L.aproj.beta};
        float* outs[4] = {xa, xcbar, xc, xa + (int64_t)B * Da};
        const int64_t lds[4] = {Da, Dc, Dc, Da};
        for (int i = 0; i < 4; ++i) {
            LnProblem p{};
            p.rows = B; p.n = Dd;
            p.pre = proj_pre + i * (int64_t)B * Dd; p.ld_pre = Dd;
            p.g = gs[i]; p.beta = bs[i];
            p.out = outs[i]; p.ld_out = lds[i];
            p.mean = proj_mean + i * B; p.rstd = proj_rstd + i * B;
            lp[i] = p;
        }
        launch_ln_fwd(lp, 4, false, ln_eps, s);
    } else {
        const size_t fb = (size_t)F * sizeof(float);
        cudaMemcpy2DAsync(xa, Da * sizeof(float), z1, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xa + (int64_t)B * Da, Da * sizeof(float), z, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xcbar, Dc * sizeof(float), z1, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xc, Dc * sizeof(float), z, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xq, Dc * sizeof(float), z, fb, fb, B, cudaMemcpyDeviceToDevice, s);
    }

    mark(s);
    // ---- a7: actor (pre-update) on both halves; tanh-Gaussian sample
    const std::vector<Lin>* act_layers[1] = {&L.actor};
    const std::vector<Lin>* crit_layers[2] = {&L.critic[0], &L.critic[1]};
    {
        PSet ps[1] = {online};
        mlp_forward(actor_mlp, act_layers, ps, 1, xa, Da, 2 * B, ln_eps, s);
        ActorHeadArgs ah{};
        ah.rows = 2 * B; ah.B = B; ah.A = A;
        ah.out = actor_mlp.out; ah.ld_out = 2 * A;
        ah.lo = (float)c.log_std_min; ah.hi = (float)c.log_std_max;
        ah.seed = c.seed; ah.update_idx = d_update_idx;
        ah.a_dst0 = xcbar + Z + P; ah.ld0 = Dc;
        ah.a_dst1 = xq + Z + P; ah.ld1 = Dc;
        ah.logp = logp; ah.eps = eps;
        launch_actor_head(ah, s);
    }
    mark(s);
    // ---- a8-a9: target critics and the projected categorical target
    {
        PSet ps[2] = {tgt, tgt};
        mlp_forward(tcrit_mlp, crit_layers, ps, E, xcbar, Dc, B, ln_eps, s);
        C51TargetArgs ct{};
        ct.B = B; ct.K = K; ct.E = E;
        ct.logits_bar = tcrit_mlp.out; ct.r = r; ct.d = d; ct.logp_next = logp;
        ct.log_alpha = W + L.log_alpha;
        ct.gamma = (float)c.gamma; ct.v_min = (float)c.v_min; ct.v_max = (float)c.v_max;
        ct.m = m;
        launch_c51_target(ct, s);
    }
    mark(s);
    // ---- a10: online critics and the cross entropy
    {
        PSet ps[2] = {online, online};
        mlp_forward(crit_mlp, crit_layers, ps, E, xc, Dc, B, ln_eps, s);
        CeArgs ce{};
        ce.B = B; ce.K = K; ce.E = E; ce.logits = crit_mlp.out; ce.m = m;
        ce.v_min = (float)c.v_min; ce.v_max = (float)c.v_max;
        ce.scale = 1.0f / (float)B;
        ce.dlogits = dlogits; ce.row_loss = row_loss; ce.row_q = row_q;
        launch_ce(ce, s);
    }
    mark(s);
    // ---- a11: backward through critics, critic projection, encoder
    {
        const float* mask = Dd > 0 ? nullptr : z;      // flatten path: mask by the last conv's ReLU
        mlp_backward(crit_mlp, 0, crit_layers, W, G, E, xc, Dc, B, dlogits, dpost, dpre, 0, Z, Dd > 0 ? dh : dz,
                     Dd > 0 ? Z : F, mask, F, s);
        if (Dd > 0) {
            LnBwdProblem p{};
            p.rows = B; p.n = Dd;
            p.dout = dh; p.ld_dout = Dd;
            p.pre = proj_pre + 2 * (int64_t)B * Dd; p.ld_pre = Dd;
            p.mean = proj_mean + 2 * B; p.rstd = proj_rstd + 2 * B;
            p.g = W + L.cproj.g;
            p.dpre = dproj; p.ld_dpre = Dd;
            p.dg = G + L.cproj.g; p.dbeta = G + L.cproj.beta; p.dbias = G + L.cproj.b;
            launch_ln_bwd(&p, 1, s);
            GemmProblem gw = lin_dw(dproj, Dd, B, z, F, F, Dd, G + L.cproj.w);
            launch_gemm<float>(&gw, 1, kMN, s);
            GemmProblem gx = lin_dx(dproj, Dd, B, W + L.cproj.w, F, Dd, 0, F, dz, F);
            gx.mask = z; gx.sm_m = F; gx.sm_n = 1;
            launch_gemm<float>(&gx, 1, kKN, s);
        }
        mark(s);
        const float* cur = dz;
        for (int l = (int)L.conv.size() - 1; l >= 0; --l) {
            const ConvL& cv = L.conv[l];
            ConvShape sh{B, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                         (int64_t)cv.cout * cv.oh * cv.ow};
            const float* xin = l == 0 ? x2 : conv_out[l - 1];
            launch_conv_wgrad<float>(sh, cur, xin, G + cv.wo, G + cv.bo, wgrad_work, s);
            if (l > 0) {
                float* nxt = (cur == dconv_a) ? dconv_b : dconv_a;
                launch_conv_dgrad<float>(sh, cur, W + cv.wo, nxt, conv_out[l - 1], s);
                cur = nxt;
            }
        }
    }
    mark(s);
    // ---- a12: Adam over encoder + critic projection + critics
    {
        AdamArgs ad{};
        ad.p = W; ad.g = G; ad.m = adam_m; ad.v = adam_v; ad.n = L.critic_end;
        ad.step = d_steps + 0;
        ad.lr = c.lr; ad.b1 = c.adam_b1; ad.b2 = c.adam_b2; ad.eps = c.adam_eps;
        launch_adam(ad, s);
    }
    mark(s);
    // ---- a13: temperature
    {
        AlphaArgs al{};
        al.B = B; al.logp_t = logp + B;
        al.log_alpha = W + L.log_alpha; al.m = adam_m + L.log_alpha; al.v = adam_v + L.log_alpha;
        al.steps = d_steps;
        al.lr = c.lr; al.b1 = c.adam_b1; al.b2 = c.adam_b2; al.eps = c.adam_eps;
        al.target_entropy = std::isnan(c.target_entropy) ? -(float)A : (float)c.target_entropy;
        al.stats = stats;
        launch_alpha_step(al, s);
    }
    mark(s);
    // ---- a14: actor step on stop-gradient features with the updated critics
    {
        if (Dd > 0) {
            GemmProblem g = lin_fwd(z, F, B, W + L.cproj.w, W + L.cproj.b, F, Dd, proj_pre + 4 * (int64_t)B * Dd, Dd);
            launch_gemm<float>(&g, 1, kKK, s);
            LnProblem p{};
            p.rows = B; p.n = Dd;
            p.pre = proj_pre + 4 * (int64_t)B * Dd; p.ld_pre = Dd;
            p.g = W + L.cproj.g; p.beta = W + L.cproj.beta;
            p.out = xq; p.ld_out = Dc;
            p.mean = proj_mean + 4 * B; p.rstd = proj_rstd + 4 * B;
            launch_ln_fwd(&p, 1, false, ln_eps, s);
        }
        PSet ps[2] = {online, online};
        mlp_forward(qcrit_mlp, crit_layers, ps, E, xq, Dc, B, ln_eps, s);
        ActorQArgs aq{};
        aq.B = B; aq.K = K; aq.E = E; aq.logits = qcrit_mlp.out;
        aq.v_min = (float)c.v_min; aq.v_max = (float)c.v_max;
        aq.dlogits = dlogits_q; aq.row_q = row_q_actor; aq.do_actor = d_do_actor;
        launch_actor_q(aq, s);
        mlp_backward(qcrit_mlp, 0, crit_layers, W, nullptr, E, xq, Dc, B, dlogits_q, dpost, dpre, Z + P, A, da, A,
                     nullptr, 0, s);
        ActorHeadBwdArgs hb{};
        hb.B = B; hb.A = A;
        hb.out = actor_mlp.out + (int64_t)B * 2 * A; hb.ld_out = 2 * A;
        hb.eps = eps + (int64_t)B * A; hb.da = da; hb.log_alpha = W + L.log_alpha;
        hb.lo = (float)c.log_std_min; hb.hi = (float)c.log_std_max;
        hb.dout = dout_a; hb.do_actor = d_do_actor;
        launch_actor_head_bwd(hb, s);
        mlp_backward(actor_mlp, B, act_layers, W, G, 1, xa + (int64_t)B * Da, Da, B, dout_a, dpost, dpre, 0, Z,
                     Dd > 0 ? dh : nullptr, Z, nullptr, 0, s);
        if (Dd > 0) {
            LnBwdProblem p{};
            p.rows = B; p.n = Dd;
            p.dout = dh; p.ld_dout = Dd;
            p.pre = proj_pre + 3 * (int64_t)B * Dd; p.ld_pre = Dd;
            p.mean = proj_mean + 3 * B; p.rstd = proj_rstd + 3 * B;
            p.g = W + L.aproj.g;
            p.dpre = dproj; p.ld_dpre = Dd;
            p.dg = G + L.aproj.g; p.dbeta = G + L.aproj.beta; p.dbias = G + L.aproj.b;
            launch_ln_bwd(&p, 1, s);
            GemmProblem gw = lin_dw(dproj, Dd, B, z, F, F, Dd, G + L.aproj.w);
            launch_gemm<float>(&gw, 1, kMN, s);
        }
        AdamArgs ad{};
        ad.p = W + L.actor_begin; ad.g = G + L.actor_begin; ad.m = adam_m + L.actor_begin; ad.v = adam_v + L.actor_begin;
        ad.n = L.actor_end - L.actor_begin;
        ad.step = d_steps + 1; ad.enable = d_do_actor;
        ad.lr = c.lr; ad.b1 = c.adam_b1; ad.b2 = c.adam_b2; ad.eps = c.adam_eps;
        launch_adam(ad, s);
    }
    mark(s);
    // ---- statistics, then a16: polyak (also advances the update index)
    {
        StatsArgs st{};
        st.B = B; st.E = E; st.row_loss = row_loss; st.row_q = row_q; st.row_q_actor = row_q_actor;
        st.logp_t = logp + B; st.log_alpha = W + L.log_alpha; st.do_actor = d_do_actor;
        st.update_idx = d_update_idx; st.stats = stats;
        launch_stats(st, s);
        PolyakArgs pa{target, W + L.critic_begin, L.target_n, (float)c.tau, d_update_idx};
        launch_polyak(pa, s);
    }
    mark(s);
}

int squint_handle::run_updates(int k, squint_update_stats* stats, cudaStream_t s, bool use_graph) {
    if (use_graph) {
        auto it = graphs.find(k);
        if (it == graphs.end()) {
            // make the capture stream start after the caller's pending work
            cudaEvent_t ev;
            SQ_CK(this, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            SQ_CK(this, cudaEventRecord(ev, s));
            SQ_CK(this, cudaStreamWaitEvent(capture_stream, ev, 0));
            SQ_CK(this, cudaStreamSynchronize(capture_stream));
            cudaEventDestroy(ev);
            cudaGraph_t graph;
            SQ_CK(this, cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
            for (int j = 0; j < k; ++j) record_update(j, capture_stream, false);
            SQ_CK(this, cudaStreamEndCapture(capture_stream, &graph));
            size_t n_nodes = 0;
            SQ_CK(this, cudaGraphGetNodes(graph, nullptr, &n_nodes));
            std::vector<cudaGraphNode_t> nodes(n_nodes);
            SQ_CK(this, cudaGraphGetNodes(graph, nodes.data(), &n_nodes));
            int64_t kernels = 0;
            for (auto nd : nodes) {
                cudaGraphNodeType t;
                SQ_CK(this, cudaGraphNodeGetType(nd, &t));
                kernels += t == cudaGraphNodeTypeKernel;
            }
            graph_kernels[k] = kernels;
            cudaGraphExec_t exec;
            SQ_CK(this, cudaGraphInstantiate(&exec, graph, 0));
            cudaGraphDestroy(graph);
            it = graphs.emplace(k, exec).first;
        }
        SQ_CK(this, cudaGraphLaunch(it->second, s));
    } else {
        for (int j = 0; j < k; ++j) record_update(j, s, true);
        SQ_CK(this, cudaGetLastError());
    }
    if (stats) {
        SQ_CK(this, cudaMemcpyAsync(h_stats, d_stats, sizeof(float) * 8 * k, cudaMemcpyDeviceToHost, s));
        SQ_CK(this, cudaStreamSynchronize(s));
        for (int j = 0; j < k; ++j) {
            const float* q = h_stats + 8 * j;
            squint_update_stats& o = stats[j];
            o.critic_loss = q[0]; o.actor_loss = q[1]; o.alpha_loss = q[2]; o.alpha = q[3];
            o.q_mean = q[4]; o.entropy = q[5];
            uint32_t lo, hi;
            std::memcpy(&lo, q + 6, 4);
            std::memcpy(&hi, q + 7, 4);
            o.update_idx = (int64_t)(((uint64_t)hi << 32) | lo);
        }
    }
    return SQUINT_OK;
}

size_t squint_handle::state_bytes() const {
    return 48 + sizeof(float) * (size_t)(3 * L.total + L.target_n);
}

int squint_handle::save_state(uint8_t* out) {
    SQ_CK(this, cudaDeviceSynchronize());
    uint32_t hdr32[2] = {kStateMagic, 1};
    int64_t hdr64[2] = {L.total, L.target_n};
    int32_t steps[4];
    int64_t u;
    SQ_CK(this, cudaMemcpy(steps, d_steps, sizeof(steps), cudaMemcpyDeviceToHost));
    SQ_CK(this, cudaMemcpy(&u, d_update_idx, sizeof(u), cudaMemcpyDeviceToHost));
    std::memcpy(out, hdr32, 8);
    std::memcpy(out + 8, hdr64, 16);
    std::memcpy(out + 24, steps, 16);
    std::memcpy(out + 40, &u, 8);
    uint8_t* p = out + 48;
    const size_t nb = sizeof(float) * L.total;
    SQ_CK(this, cudaMemcpy(p, params, nb, cudaMemcpyDeviceToHost)); p += nb;
    SQ_CK(this, cudaMemcpy(p, adam_m, nb, cudaMemcpyDeviceToHost)); p += nb;
    SQ_CK(this, cudaMemcpy(p, adam_v, nb, cudaMemcpyDeviceToHost)); p += nb;
    SQ_CK(this, cudaMemcpy(p, target, sizeof(float) * L.target_n, cudaMemcpyDeviceToHost));
    return SQUINT_OK;
}

int squint_handle::load_state(const uint8_t* in) {
    uint32_t hdr32[2];
    int64_t hdr64[2];
    std::memcpy(hdr32, in, 8);
    std::memcpy(hdr64, in + 8, 16);
    if (hdr32[0] != kStateMagic || hdr32[1] != 1 || hdr64[0] != L.total || hdr64[1] != L.target_n) {
        g_last_error = "state does not match this configuration";
        return SQUINT_EINVAL;
    }
    SQ_CK(this, cudaDeviceSynchronize());
    SQ_CK(this, cudaMemcpy(d_steps, in + 24, 16, cudaMemcpyHostToDevice));
    SQ_CK(this, cudaMemcpy(d_update_idx, in + 40, 8, cudaMemcpyHostToDevice));
    const uint8_t* p = in + 48;
    const size_t nb = sizeof(float) * L.total;
    SQ_CK(this, cudaMemcpy(params, p, nb, cudaMemcpyHostToDevice)); p += nb;
    SQ_CK(this, cudaMemcpy(adam_m, p, nb, cudaMemcpyHostToDevice)); p += nb;
    SQ_CK(this, cudaMemcpy(adam_v, p, nb, cudaMemcpyHostToDevice)); p += nb;
    SQ_CK(this, cudaMemcpy(target, p, sizeof(float) * L.target_n, cudaMemcpyHostToDevice));
    return after_param_change();
}

int squint_handle::debug_tensor(const char* name, void* host, size_t* bytes) {
    const int B = c.batch, A = c.action_dim, K = c.atoms;
    const int64_t img = (int64_t)c.obs_c * L.hs * L.ws;
    const std::string n(name);
    const void* src = nullptr;
    size_t sz = 0;
    if (n == "idx") { src = idx2; sz = 4 * B; }
    else if (n == "nxt") { src = idx2 + B; sz = 4 * B; }
    else if (n == "shift_t") { src = shift2; sz = 8 * B; }
    else if (n == "shift_t1") { src = shift2 + 2 * B; sz = 8 * B; }
    else if (n == "sums_t") { src = sums; sz = 2 * B * img; }
    else if (n == "sums_t1") { src = sums + B * img; sz = 2 * B * img; }
    else if (n == "x_t") { src = x2; sz = 4 * B * img; }
    else if (n == "x_t1") { src = x2 + B * img; sz = 4 * B * img; }
    else if (n == "m") { src = m; sz = 4 * (size_t)B * K; }
    else if (n == "logits") { src = crit_mlp.out; sz = 4 * (size_t)2 * B * K; }
    else if (n == "logits_target") { src = tcrit_mlp.out; sz = 4 * (size_t)2 * B * K; }
    else if (n == "logp_next") { src = logp; sz = 4 * B; }
    else if (n == "logp_t") { src = logp + B; sz = 4 * B; }
    else if (n == "a_next") { src = nullptr; sz = 4 * (size_t)B * A; }
    else if (n == "a_pi") { src = nullptr; sz = 4 * (size_t)B * A; }
    else if (n == "grads") { src = grads; sz = 4 * (size_t)L.total; }
    else if (n == "z_t") { src = conv_out.back(); sz = 4 * (size_t)B * L.feat; }
    else if (n == "target") { src = target; sz = 4 * (size_t)L.target_n; }
    else { g_last_error = "unknown debug tensor"; return SQUINT_EINVAL; }
    if (!host) { *bytes = sz; return SQUINT_OK; }
    if (*bytes < sz) { *bytes = sz; return SQUINT_EINVAL; }
    *bytes = sz;
    SQ_CK(this, cudaDeviceSynchronize());
    if (n == "a_next" || n == "a_pi") {
        const float* base = n == "a_next" ? xcbar : xq;
        SQ_CK(this, cudaMemcpy2D(host, A * sizeof(float), base + L.zdim + c.proprio_dim, L.dc * sizeof(float),
                                 A * sizeof(float), B, cudaMemcpyDeviceToHost));
        return SQUINT_OK;
    }
    SQ_CK(this, cudaMemcpy(host, src, sz, cudaMemcpyDeviceToHost));
    return SQUINT_OK;
}

int squint_handle::refresh_policy(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(act_mu);
    // write the snapshot inference is not using, after inference that last read it
    const int i = 1 - policy_active;
    SQ_CK(this, cudaStreamWaitEvent(s, policy_released[i], 0));
    SQ_CK(this, cudaMemcpyAsync(policy_buf[i], params, L.total * sizeof(float), cudaMemcpyDeviceToDevice, s));
    SQ_CK(this, cudaEventRecord(policy_ready[i], s));
    policy_active = i;
    ++policy_version;
    return SQUINT_OK;
}

// ---------------------------------------------------------------- inference
size_t squint_handle::act_row_bytes() const {
    size_t f = (size_t)c.obs_c * L.hs * L.ws;
    for (const auto& cv : L.conv) f += (size_t)cv.cout * cv.oh * cv.ow;
    f += (size_t)L.D + 2 + L.da;
    for (int l = 0; l < c.n_hidden; ++l) f += 2 * (size_t)c.hidden[l] + 2;
    f += 2 * (size_t)c.action_dim;
    return f * sizeof(float) + 8;
}

int squint_handle::ensure_act_capacity(int rows, int n_reqs) {
    if (rows <= act_cap && n_reqs <= req_cap) return SQUINT_OK;
    SQ_CK(this, cudaDeviceSynchronize());
    for (void* p : act_allocs) if (p) cudaFree(p);
    act_allocs.clear();
    if (h_req) { cudaFreeHost(h_req); h_req = nullptr; }
    const int cap = std::max(((std::max(rows, act_cap) + 255) / 256) * 256, 256);
    const int rcap = std::max(std::max(n_reqs, req_cap), 64);
    auto al = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return nullptr;
        act_allocs.push_back(p);
        return p;
    };
    const int64_t img = (int64_t)c.obs_c * L.hs * L.ws;
    ax = (float*)al(sizeof(float) * cap * img);
    aconv.clear();
    for (const auto& cv : L.conv) aconv.push_back((float*)al(sizeof(float) * (size_t)cap * cv.cout * cv.oh * cv.ow));
    if (L.D > 0) {
        apre = (float*)al(sizeof(float) * (size_t)cap * L.D);
        amean = (float*)al(sizeof(float) * cap);
        arstd = (float*)al(sizeof(float) * cap);
    }
    axin = (float*)al(sizeof(float) * (size_t)cap * L.da);
    const int nh = c.n_hidden;
    act_mlp = MlpBufs{};
    act_mlp.E = 1; act_mlp.rows = cap;
    act_mlp.pre.resize(nh); act_mlp.post.resize(nh); act_mlp.mean.resize(nh); act_mlp.rstd.resize(nh);
    for (int l = 0; l < nh; ++l) {
        act_mlp.pre[l] = (float*)al(sizeof(float) * (size_t)cap * c.hidden[l]);
        act_mlp.post[l] = (float*)al(sizeof(float) * (size_t)cap * c.hidden[l]);
        act_mlp.mean[l] = (float*)al(sizeof(float) * cap);
        act_mlp.rstd[l] = (float*)al(sizeof(float) * cap);
    }
    act_mlp.out = (float*)al(sizeof(float) * (size_t)cap * 2 * c.action_dim);
    req_bytes = (size_t)cap * 8 + (size_t)rcap * (8 * 4 + 4) + 64;
    d_req = al(req_bytes);
    for (void* p : act_allocs) if (!p) { g_last_error = "inference allocation failed"; act_cap = 0; return SQUINT_ENOMEM; }
    if (cudaMallocHost(&h_req, req_bytes) != cudaSuccess) { act_cap = 0; return SQUINT_ENOMEM; }
    act_cap = cap;
    req_cap = rcap;
    req_event_live = false;
    return SQUINT_OK;
}

int squint_handle::act(const squint_act_request* reqs, int n_reqs, cudaStream_t s, int64_t* version_used) {
    std::lock_guard<std::mutex> lk(act_mu);
    int rows = 0;
    for (int q = 0; q < n_reqs; ++q) {
        const squint_act_request& rq = reqs[q];
        if (rq.n < 1 || !rq.obs || !rq.proprio || !rq.actions || (rq.mode != 0 && rq.mode != 1)) {
            g_last_error = "invalid inference request";
            return SQUINT_EINVAL;
        }
        rows += rq.n;
    }
    if (rows == 0) return SQUINT_OK;
    int rc = ensure_act_capacity(rows, n_reqs);
    if (rc != SQUINT_OK) return rc;
    if (req_event_live) SQ_CK(this, cudaEventSynchronize(req_event));
    // pack: row_req[cap] row_in[cap] | obs[rcap] prop[rcap] act[rcap] key[rcap] (8 B each) | mode[rcap]
    uint8_t* hb = static_cast<uint8_t*>(h_req);
    int32_t* row_req = reinterpret_cast<int32_t*>(hb);
    int32_t* row_in = row_req + act_cap;
    uint64_t* p64 = reinterpret_cast<uint64_t*>(hb + (size_t)act_cap * 8);
    int32_t* modes = reinterpret_cast<int32_t*>(p64 + 4 * (size_t)req_cap);
    int r = 0;
    for (int q = 0; q < n_reqs; ++q) {
        for (int i = 0; i < reqs[q].n; ++i, ++r) { row_req[r] = q; row_in[r] = i; }
        p64[q] = (uint64_t)(uintptr_t)reqs[q].obs;
        p64[req_cap + q] = (uint64_t)(uintptr_t)reqs[q].proprio;
        p64[2 * req_cap + q] = (uint64_t)(uintptr_t)reqs[q].actions;
        p64[3 * req_cap + q] = reqs[q].rng_key;
        modes[q] = reqs[q].mode;
    }
    SQ_CK(this, cudaMemcpyAsync(d_req, h_req, req_bytes, cudaMemcpyHostToDevice, s));
    SQ_CK(this, cudaEventRecord(req_event, s));
    req_event_live = true;
    uint8_t* db = static_cast<uint8_t*>(d_req);
    const int32_t* d_row_req = reinterpret_cast<const int32_t*>(db);
    const int32_t* d_row_in = d_row_req + act_cap;
    const uint64_t* d64 = reinterpret_cast<const uint64_t*>(db + (size_t)act_cap * 8);
    const int32_t* d_modes = reinterpret_cast<const int32_t*>(d64 + 4 * (size_t)req_cap);

    const int pi = policy_active;
    const float* Wp = policy_buf[pi];
    SQ_CK(this, cudaStreamWaitEvent(s, policy_ready[pi], 0));
    if (version_used) *version_used = policy_version;

    const int F = L.feat, Da = L.da, Dd = L.D, A = c.action_dim;
    ActFrontArgs af{};
    af.obs = reinterpret_cast<const uint8_t* const*>(d64);
    af.prop = reinterpret_cast<const float* const*>(d64 + req_cap);
    af.row_req = d_row_req; af.row_in_req = d_row_in;
    af.rows = rows; af.C = c.obs_c; af.H = c.obs_h; af.W = c.obs_w; af.f = c.squint_f; af.P = c.proprio_dim;
    af.x = ax; af.xin = axin; af.ld_xin = Da; af.col = L.zdim;
    launch_act_frontend(af, s);
    const float* in = ax;
    for (size_t l = 0; l < L.conv.size(); ++l) {
        const ConvL& cv = L.conv[l];
        ConvShape sh{rows, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                     (int64_t)cv.cout * cv.oh * cv.ow};
        launch_conv_fwd<float>(sh, in, Wp + cv.wo, Wp + cv.bo, aconv[l], true, s);
        in = aconv[l];
    }
    if (Dd > 0) {
        GemmProblem g = lin_fwd(in, F, rows, Wp + L.aproj.w, Wp + L.aproj.b, F, Dd, apre, Dd);
        launch_gemm<float>(&g, 1, kKK, s);
        LnProblem p{};
        p.rows = rows; p.n = Dd; p.pre = apre; p.ld_pre = Dd;
        p.g = Wp + L.aproj.g; p.beta = Wp + L.aproj.beta;
        p.out = axin; p.ld_out = Da; p.mean = amean; p.rstd = arstd;
        launch_ln_fwd(&p, 1, false, (float)c.ln_eps, s);
    } else {
        SQ_CK(this, cudaMemcpy2DAsync(axin, Da * sizeof(float), in, F * sizeof(float), F * sizeof(float), rows,
                                      cudaMemcpyDeviceToDevice, s));
    }
    const std::vector<Lin>* layers[1] = {&L.actor};
    PSet ps[1] = {PSet{Wp, 0}};
    mlp_forward(act_mlp, layers, ps, 1, axin, Da, rows, (float)c.ln_eps, s);
    ActHeadArgs ha{};
    ha.rows = rows; ha.A = A; ha.out = act_mlp.out; ha.ld_out = 2 * A;
    ha.row_req = d_row_req; ha.row_in_req = d_row_in;
    ha.req_key = d64 + 3 * req_cap; ha.req_mode = d_modes;
    ha.req_actions = reinterpret_cast<float* const*>(d64 + 2 * req_cap);
    ha.lo = (float)c.log_std_min; ha.hi = (float)c.log_std_max; ha.seed = c.seed;
    launch_act_head(ha, s);
    SQ_CK(this, cudaEventRecord(policy_released[pi], s));
    SQ_CK(this, cudaGetLastError());
    return SQUINT_OK;
}

// Phase names, in the order their boundaries are marked in record_update.
static const char* kPhaseNames[] = {
    "frontend",          // a1-a4
    "encoder_fwd",       // a5
    "projections",       // a6
    "actor_fwd",         // a7
    "target_critics",    // a8-a9
    "critic_fwd_ce",     // a10
    "critic_bwd",        // a11 (MLP + projection)
    "encoder_bwd",       // a11 (conv wgrad/dgrad)
    "adam_critic",       // a12
    "alpha_step",        // a13
    "actor_step",        // a14-a15
    "stats_polyak",      // a16
};

const char* sq::phase_name(int i) {
    return (i >= 0 && i < (int)(sizeof(kPhaseNames) / sizeof(kPhaseNames[0]))) ? kPhaseNames[i] : nullptr;
}

int squint_handle::profile_update(float* ms, int cap, int* n_phases, cudaStream_t s) {
    std::vector<cudaEvent_t> ev;
    phase_events = &ev;
    record_update(0, s, false);
    phase_events = nullptr;
    int rc = SQUINT_OK;
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = SQUINT_ECUDA;
    const int n = (int)ev.size() - 1;
    if (n_phases) *n_phases = n;
    for (int i = 0; rc == SQUINT_OK && i < n && i < cap; ++i) {
        if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) rc = SQUINT_ECUDA;
    }
    for (auto e : ev) cudaEventDestroy(e);
    if (rc != SQUINT_OK) { failed = true; g_last_error = "profiling failed"; }
    return rc;
}
