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
//
// Contractions go through GemmBuilder: CUDA-core FP32 kernels in the plain path,
// tcgen05 BF16 kernels (FP32 accumulation) in the tensor-core path, where every
// GEMM operand has a BF16 shadow written by the kernel that produces it.
#include "sq_sched.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <tuple>

using namespace sq;

namespace sq {

static int64_t pad8(int64_t n) { return (n + 7) / 8 * 8; }
constexpr int kLongK = 1024;   // reductions at least this long may split K over a cluster
// The sets' input gradients are left apart by the fused chain from two row blocks a set
// on: with one, the GEMM that adds them is a single short CTA and the chain's own final
// step costs more (batch 32: 3,404 against 3,876 updates/s), while at batch 512 the GEMM's
// few long CTAs sit on the critical chain beside the encoder backward (2,474 against 2,405)
constexpr int kFinSplitRows = 256;
constexpr int kCh32 = 32;   // channels of the tensor-core convolutions

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

// ---------------------------------------------------------------- GemmBuilder
bool GemmBuilder::fwd(const Mat& X, int rows, const LayerRef& W, float* Y, int64_t ldy, __nv_bfloat16* Yh,
                      int64_t ldyh, const LnProblem* ln, bool relu) {
    flops_ += 2.0 * rows * W.out * W.in;
    kind_ = bf_ ? "tc_gemm_fwd" : "gemm_f32_fwd";
    if (!bf_) {
        fp_.push_back(lin_fwd(X.f, X.ld, rows, W.w, W.b, W.in, W.out, Y, ldy));
        lay_ = kKK;
        return false;
    }
    TcGemm g{};
    g.M = rows; g.N = W.out; g.K = W.in; g.n_pairs = 1;
    g.a[0] = TcOperand{X.h, X.ldh, false};
    g.b[0] = TcOperand{W.wh, W.ldh, false};
    g.bias = W.b;
    g.c = Y; g.ldc = ldy;
    g.cbf = Yh; g.ldcbf = ldyh;
    bool fused = false;
    if (ln && !Yh && W.out <= 128 * tc_max_cluster() && ln->ld_out == W.out && ln->ld_out_bf == W.out) {
        g.ln_g = ln->g; g.ln_beta = ln->beta;
        g.ln_post = ln->out; g.ln_posth = ln->out_bf;
        g.ln_mean = ln->mean; g.ln_rstd = ln->rstd;
        g.ln_eps = (float)h_->c.ln_eps; g.ln_relu = relu ? 1 : 0;
        fused = true;
    }
    if (h_->fp8 && W.w8 && X.h) {
        // FP8: quantise X (per tensor) into this stream's arena at flush, e4m3 weights
        // (MX-FP8: the codes are followed by their block-scale atoms in the arena)
        squint_handle::F8Arena* ar = h_->arena_for(s_);
        const int64_t ld8 = (W.in + 15) / 16 * 16;
        const int64_t codes = ((int64_t)rows * ld8 + 255) / 256 * 256;
        const int64_t sfb = h_->mx ? (mx_scale_bytes(rows, W.in) + 255) / 256 * 256 : 0;
        const int qi = (int)q8_.size();
        if (ar->buf && arena_used_ + codes + sfb <= ar->bytes && qi < kF8Scales && (!h_->mx || W.sf8)) {
            uint8_t* dst = ar->buf + arena_used_;
            uint8_t* sf = h_->mx ? dst + codes : nullptr;
            arena_used_ += codes + sfb;
            q8_.push_back(QuantItem{X.h, X.ldh, rows, W.in, dst, ld8, ar->scales + qi, sf});
            qbytes_ += 3.0 * rows * W.in;
            g.a[0] = TcOperand{dst, ld8, false};
            g.b[0] = TcOperand{W.w8, W.ld8, false};
            if (h_->mx) {
                g.fp8 = 2; g.sf_a = sf; g.sf_b = W.sf8;
            } else {
                g.fp8 = 1; g.scale_a = ar->scales + qi; g.scale_b = W.s8;
            }
            (fused ? tc8ln_ : tc8_).push_back(g);
            return fused;
        }
    }
    (fused ? tcln_ : tc_).push_back(g);
    return fused;
}

void GemmBuilder::dx(const Mat* dY, const LayerRef* W, int n_pairs, int rows, int col0, int ncols, float* dX,
                     int64_t ldx, const float* mask, int64_t ldm) {
    if (ncols <= 0 || rows <= 0) return;           // no input columns wanted (state-based: no features)
    flops_ += 2.0 * rows * ncols * W[0].out * n_pairs;
    kind_ = bf_ ? "tc_gemm_dx" : "gemm_f32_dx";
    if (!bf_) {
        GemmProblem p{};
        p.M = rows; p.N = ncols; p.K = W[0].out;
        p.A = dY[0].f; p.sa_m = dY[0].ld; p.sa_k = 1;
        p.B = W[0].w + col0; p.sb_n = 1; p.sb_k = W[0].in;
        p.C = dX; p.sc_m = ldx; p.sc_n = 1;
        p.n_sum = n_pairs;
        p.a_sum = n_pairs > 1 ? dY[1].f - dY[0].f : 0;
        p.b_sum = n_pairs > 1 ? W[1].w - W[0].w : 0;
        if (mask) { p.mask = mask; p.sm_m = ldm; p.sm_n = 1; }
        fp_.push_back(p);
        lay_ = kKN;
        return;
    }
    TcGemm g{};
    g.M = rows; g.N = ncols; g.K = W[0].out; g.n_pairs = n_pairs;
    for (int q = 0; q < n_pairs; ++q) {
        g.a[q] = TcOperand{dY[q].h, dY[q].ldh, false};
        g.b[q] = TcOperand{W[q].wh + col0, W[q].ldh, true};
    }
    g.c = dX; g.ldc = ldx;
    g.mask = mask; g.ldmask = ldm;
    tc_.push_back(g);
}

void GemmBuilder::dw(const Mat& dY, int rows, const Mat& X, const LayerRef& W, float* dW) {
    flops_ += 2.0 * rows * W.out * W.in;
    kind_ = bf_ ? "tc_gemm_dw" : "gemm_f32_dw";
    if (!bf_) {
        GemmProblem p{};
        p.M = W.out; p.N = W.in; p.K = rows;
        p.A = dY.f; p.sa_m = 1; p.sa_k = dY.ld;
        p.B = X.f; p.sb_n = 1; p.sb_k = X.ld;
        p.C = dW; p.sc_m = W.in; p.sc_n = 1;
        p.n_sum = 1;
        fp_.push_back(p);
        lay_ = kMN;
        return;
    }
    TcGemm g{};
    g.M = W.out; g.N = W.in; g.K = rows; g.n_pairs = 1;
    g.a[0] = TcOperand{dY.h, dY.ldh, true};
    g.b[0] = TcOperand{X.h, X.ldh, true};
    g.c = dW; g.ldc = W.in;
    tc_.push_back(g);
}

void GemmBuilder::flush() {
    if (fp_.empty() && tc_.empty() && tc8_.empty() && tcln_.empty() && tc8ln_.empty()) return;
    if (!q8_.empty()) {
        ProfScope ps(h_, s_, h_->mx ? "quantize_mxfp8" : "quantize_fp8", qbytes_, 1);
        if (h_->mx) launch_quantize_mx(q8_.data(), (int)q8_.size(), s_);
        else launch_quantize_e4m3(q8_.data(), (int)q8_.size(), h_->arena_for(s_)->part, s_);
    }
    {
        ProfScope ps(h_, s_, kind_, flops_, 0);
        if (!fp_.empty()) launch_gemm<float>(fp_.data(), (int)fp_.size(), lay_, s_);
        // the K split over a cluster pays for long reductions over few output tiles (the
        // projections from the flattened features, K = 2592); elsewhere it is opt-in
        for (auto* v : {&tc8_, &tc8ln_, &tc_, &tcln_}) {
            if (v->empty()) continue;
            int kmax = 0;
            for (const TcGemm& g : *v) kmax = std::max(kmax, g.K);
            const bool split = split_ && (h_->gemm_split || kmax >= kLongK);
            if (launch_tc_gemm(v->data(), (int)v->size(), h_->d_err, s_, split, &h_->gemm_wait) != 0)
                h_->launch_failed = true;
        }
    }
    fp_.clear();
    tc_.clear();
    tc8_.clear();
    tcln_.clear();
    tc8ln_.clear();
    q8_.clear();
    arena_used_ = 0;
    qbytes_ = 0;
    flops_ = 0;
}

// ---------------------------------------------------------------- parameter views
LayerRef layer_ref(squint_handle* h, const Lin& ly, bool target, const float* base) {
    auto P = [&](int64_t off) -> const float* {
        if (off < 0) return nullptr;
        if (target) return h->target + (off - h->L.critic_begin);
        return (base ? base : h->params) + off;
    };
    LayerRef r;
    r.w = P(ly.w); r.b = P(ly.b);
    r.in = ly.in; r.out = ly.out;
    if (ly.ln) { r.g = P(ly.g); r.beta = P(ly.beta); }
    auto it = h->lin_bf.find(ly.w);
    if (it != h->lin_bf.end() && !base) {
        r.wh = target ? it->second.tg : it->second.on;
        r.ldh = it->second.ld;
    }
    auto f8 = h->lin_f8.find(ly.w);
    if (f8 != h->lin_f8.end() && !base) {
        r.w8 = target ? f8->second.tg : f8->second.on;
        r.s8 = target ? f8->second.s_tg : f8->second.s_on;
        r.ld8 = f8->second.ld;
        r.sf8 = target ? f8->second.sf_tg : f8->second.sf_on;
        if (!r.w8) r.s8 = nullptr;
    }
    return r;
}

MlpRef mlp_ref(squint_handle* h, const std::vector<Lin>& layers, bool target, const float* base) {
    MlpRef m;
    for (const auto& l : layers) m.push_back(layer_ref(h, l, target, base));
    return m;
}

void mlp_forward(squint_handle* h, MlpBufs& mb, const MlpRef* sets, int E, const Mat& X, int rows, bool bf16,
                 cudaStream_t s, bool split, bool keep, int r0) {
    const int nh = (int)sets[0].size() - 1;
    // the chains that take the fused kernel (bit 0 online critics, 1 actor, 2 target
    // critics, 3 the actor step's critics; other buffers always)
    const int site = &mb == &h->crit_mlp ? 1 : &mb == &h->actor_mlp ? 2 : &mb == &h->tcrit_mlp ? 4
                   : &mb == &h->qcrit_mlp ? 8 : 0;
    if (bf16 && !h->fp8 && h->mlp_fused && (site == 0 || (h->mlp_fused_sites & site)) && X.h && rows > 0 &&
        E <= kMlpMaxProbs) {
        // the whole chain in one launch: hidden activations stay on chip between layers
        const int H = sets[0][0].out, nout = sets[0][nh].out, kin = sets[0][0].in;
        bool ok = mlp_tc_supported(nh, H, nout, kin);
        for (int l = 0; l < nh; ++l) ok = ok && sets[0][l].out == H;
        for (int e = 0; e < E && ok; ++e)
            for (int l = 0; l <= nh; ++l) ok = ok && sets[e][l].wh;
        if (ok) {
            MlpTcProblem pr[kMlpMaxProbs];
            double flops = 0;
            for (int e = 0; e < E; ++e) {
                MlpTcProblem& q = pr[e];
                std::memset(&q, 0, sizeof(q));
                q.M = rows; q.x = X.h; q.ldx = X.ldh; q.kin = kin;
                for (int l = 0; l <= nh; ++l) {
                    const LayerRef& ly = sets[e][l];
                    q.w[l] = ly.wh; q.ldw[l] = ly.ldh; q.bias[l] = ly.b;
                    flops += 2.0 * rows * ly.in * ly.out;
                    if (l == nh) break;
                    q.g[l] = ly.g; q.beta[l] = ly.beta;
                    if (keep) {
                        const int64_t off = ((int64_t)e * rows + r0) * H;
                        q.save[l] = MlpTcSave{mb.pre[l] + off, mb.post[l] + off,
                                              mb.posth.empty() ? nullptr : mb.posth[l] + off,
                                              mb.mean[l] + ((int64_t)e * rows + r0), mb.rstd[l] + ((int64_t)e * rows + r0)};
                    }
                }
                q.out = mb.out + ((int64_t)e * rows + r0) * nout; q.ldo = nout;
            }
            // the chain's cluster size; the per-chain 8 only where each CTA keeps at least 64
            // of the hidden columns (an explicit SQUINT_MLP_CL applies as given)
            int cluster = site ? h->mlp_cluster_site[__builtin_ctz(site)] : h->mlp_cluster;
            if (!h->mlp_cluster && cluster == 8 && H / 8 < 64) cluster = 0;
            ProfScope ps(h, s, "mlp_tc_fwd", flops, 0);
            if (launch_mlp_tc(pr, E, nh, H, nout, (float)h->c.ln_eps, h->d_err, &h->gemm_wait, s, cluster) == 0) {
                if (keep) mb.tc_saved = true;
                return;
            }
        }
    }
    mb.tc_saved = false;
    for (int l = 0; l <= nh; ++l) {
        // the hidden layers' LayerNorm (+ReLU) problems; on the tensor-core path the GEMM
        // computes them in its epilogue
        LnProblem lp[2];
        if (l < nh)
            for (int e = 0; e < E; ++e) {
                const LayerRef& ly = sets[e][l];
                LnProblem p{};
                p.rows = rows; p.n = ly.out;
                p.pre = mb.pre[l] + ((int64_t)e * rows + r0) * ly.out; p.ld_pre = ly.out;
                p.g = ly.g; p.beta = ly.beta;
                p.out = mb.post[l] + ((int64_t)e * rows + r0) * ly.out; p.ld_out = ly.out;
                if (bf16 && !mb.posth.empty()) { p.out_bf = mb.posth[l] + ((int64_t)e * rows + r0) * ly.out; p.ld_out_bf = ly.out; }
                p.mean = mb.mean[l] + ((int64_t)e * rows + r0); p.rstd = mb.rstd[l] + ((int64_t)e * rows + r0);
                lp[e] = p;
            }
        bool fused = l < nh && bf16 && h->fuse_ln && !mb.posth.empty();
        {
            GemmBuilder gb(h, s, bf16, split);
            for (int e = 0; e < E; ++e) {
                const LayerRef& ly = sets[e][l];
                Mat in = X;
                if (l > 0) {
                    in.f = mb.post[l - 1] + ((int64_t)e * rows + r0) * ly.in;
                    in.ld = ly.in;
                    in.h = mb.posth.empty() ? nullptr : mb.posth[l - 1] + ((int64_t)e * rows + r0) * ly.in;
                    in.ldh = ly.in;
                }
                float* y = l < nh ? mb.pre[l] + ((int64_t)e * rows + r0) * ly.out : mb.out + ((int64_t)e * rows + r0) * ly.out;
                const bool f = gb.fwd(in, rows, ly, y, ly.out, nullptr, 0, fused ? &lp[e] : nullptr, true);
                fused = fused && f;
            }
        }
        if (l == nh || fused) continue;
        ProfScope ps(h, s, "layernorm_fwd", 4.0 * E * rows * sets[0][l].out * (bf16 ? 3.5 : 3.0), 1);
        launch_ln_fwd(lp, E, true, (float)h->c.ln_eps, s);
    }
}

}  // namespace sq

namespace {

// The BF16 backward through a head MLP with the fused chain kernel: one launch for the
// input-gradient chain and every hidden LayerNorm backward (the input gradient itself in
// the same launch for one parameter set, or for two sets given a second destination dX2,
// which then holds set 1's product and dX set 0's; else one GEMM that adds the sets'
// products); the weight gradients (GEMMs) and the gain, shift and bias gradients (column
// sums of the kernel's per-row-block sums) on `side`.  False (nothing launched) if the
// shapes are outside the kernel's range; *split = whether dX and dX2 hold the sets'
// products apart.
bool fused_backward(squint_handle* h, const MlpBufs& mb, int r0, const MlpRef* sets, float* grads, int E, const Mat& X,
                    int rows, const Mat& dout, int ncols, float* dX, int64_t lddx, const float* mask, int64_t ldmask,
                    cudaStream_t s, cudaStream_t side, int col0, bool join, float* dX2, bool* split) {
    const int nh = (int)sets[0].size() - 1;
    const int R = mb.rows;
    const int H = sets[0][0].out, nout = sets[0][nh].out, kin = sets[0][0].in;
    if (mb.posth.empty() || (grads && (int)h->mlp_colpart.size() < nh)) return false;
    for (int l = 0; l < nh; ++l)
        if (sets[0][l].out != H) return false;
    for (int e = 0; e < E; ++e)
        for (int l = 0; l <= nh; ++l)
            if (!sets[e][l].wh) return false;
    const int fcl = h->mlp_bwd_cluster;
    if (!mlp_bwd_tc_supported(nh, H, nout, kin, 0, 0, fcl)) return false;
    const bool fin = dX && ncols > 0 && (E == 1 || dX2) && !mask &&
                     mlp_bwd_tc_supported(nh, H, nout, kin, col0, ncols, fcl);
    *split = fin && E > 1;
    const int nrb = (rows + 127) / 128;
    auto G = [&](const float* p) { return grads + (p - h->params); };
    auto post = [&](int l, int e) {
        Mat m;
        m.f = mb.post[l] + ((int64_t)e * R + r0) * H; m.ld = H;
        m.h = mb.posth[l] + ((int64_t)e * R + r0) * H; m.ldh = H;
        return m;
    };
    auto dpre = [&](int l, int e) {
        Mat m;
        m.f = h->dpre[l] + (int64_t)e * rows * H; m.ld = H;
        m.h = h->dpre_h[l] + (int64_t)e * rows * H; m.ldh = H;
        return m;
    };
    auto dout_e = [&](int e) {
        Mat m = dout;
        m.f += (int64_t)e * rows * dout.ld;
        m.h += (int64_t)e * rows * dout.ldh;
        return m;
    };
    if (grads) {   // the output layer's weight and bias gradients need only dout
        h->fork(s, side);
        {
            GemmBuilder gb(h, side, true);
            for (int e = 0; e < E; ++e) gb.dw(dout_e(e), rows, post(nh - 1, e), sets[e][nh], G(sets[e][nh].w));
        }
        ColSumProblem cs[2];
        for (int e = 0; e < E; ++e) cs[e] = ColSumProblem{rows, nout, dout_e(e).f, dout.ld, G(sets[e][nh].b)};
        ProfScope ps(h, side, "colsum", 4.0 * E * rows * nout, 1);
        launch_colsum(cs, E, side);
    }
    MlpTcBwdProblem pr[kMlpMaxProbs];
    double flops = 0;
    for (int e = 0; e < E; ++e) {
        MlpTcBwdProblem& q = pr[e];
        std::memset(&q, 0, sizeof(q));
        q.M = rows; q.dout = dout_e(e).h; q.ld_dout = dout.ldh;
        for (int l = 0; l <= nh; ++l) {
            q.w[l] = sets[e][l].wh; q.ldw[l] = sets[e][l].ldh;
            if (l == nh) break;
            const int64_t off = ((int64_t)e * R + r0) * H;
            q.g[l] = sets[e][l].g;
            // the fused forward's saves: the ReLU mask is rebuilt from pre, g and beta
            if (mb.tc_saved) q.beta[l] = sets[e][l].beta;
            q.pre[l] = mb.pre[l] + off; q.post[l] = mb.post[l] + off;
            q.mean[l] = mb.mean[l] + (int64_t)e * R + r0; q.rstd[l] = mb.rstd[l] + (int64_t)e * R + r0;
            if (grads || (l == 0 && !fin)) q.dpre_bf[l] = dpre(l, e).h;
            if (grads) q.colpart[l] = h->mlp_colpart[l] + (int64_t)e * nrb * 3 * H;
        }
        if (fin) { q.dx = e == 0 ? dX : dX2; q.lddx = lddx; }
        flops += 2.0 * rows * ((double)nout * H + (double)(nh - 1) * H * H + (fin ? (double)H * ncols : 0.0));
    }
    {
        ProfScope ps(h, s, "mlp_tc_bwd", flops, 0);
        if (launch_mlp_bwd_tc(pr, E, nh, H, nout, kin, fin ? col0 : 0, fin ? ncols : 0, h->d_err, &h->gemm_wait, s, fcl) != 0)
            h->launch_failed = true;
    }
    if (!fin && dX && ncols > 0) {   // the input gradient summed over the parameter sets
        GemmBuilder gb(h, s, true);
        Mat d[2] = {dpre(0, 0), E > 1 ? dpre(0, 1) : dpre(0, 0)};
        LayerRef w[2] = {sets[0][0], E > 1 ? sets[1][0] : sets[0][0]};
        gb.dx(d, w, E, rows, col0, ncols, dX, lddx, mask, ldmask);
    }
    if (grads) {
        h->fork(s, side);
        {
            GemmBuilder gb(h, side, true);
            for (int l = nh - 1; l >= 0; --l)
                for (int e = 0; e < E; ++e) gb.dw(dpre(l, e), rows, l == 0 ? X : post(l - 1, e), sets[e][l], G(sets[e][l].w));
        }
        std::vector<ColSumProblem> cs;
        for (int l = 0; l < nh; ++l)
            for (int e = 0; e < E; ++e) {
                const float* part = h->mlp_colpart[l] + (int64_t)e * nrb * 3 * H;
                cs.push_back(ColSumProblem{nrb, H, part, 3 * H, G(sets[e][l].g)});
                cs.push_back(ColSumProblem{nrb, H, part + H, 3 * H, G(sets[e][l].beta)});
                cs.push_back(ColSumProblem{nrb, H, part + 2 * H, 3 * H, G(sets[e][l].b)});
            }
        ProfScope ps(h, side, "colsum", 4.0 * cs.size() * nrb * H, 1);
        launch_colsum(cs.data(), (int)cs.size(), side);
        if (join) h->fork(side, s);
    }
    return true;
}

// Backward through an MLP evaluated by E online parameter sets.  dout [E, rows, n_out]
// (FP32 + BF16 shadow); activations stored with R rows per set, read from row r0.
// Parameter gradients land at the canonical offsets of `grads` (null: input gradient
// only).  dX (optional) = sum over sets of the input gradient, input columns
// [col0, col0 + ncols) into dX[:, 0 .. ncols).  With dX2 (same layout) the fused chain
// may leave the two sets' input gradients apart, set 0's in dX and set 1's in dX2, for
// the reader to add: the return value says whether it did (false: dX holds the sum).
bool mlp_backward(squint_handle* h, const MlpBufs& mb, int r0, const MlpRef* sets, float* grads, int E, const Mat& X,
                  int rows, const Mat& dout, int ncols, float* dX, int64_t lddx, const float* mask, int64_t ldmask,
                  cudaStream_t s, cudaStream_t side, int col0 = 0, bool join = true, float* dX2 = nullptr) {
    // weight and bias gradients go to `side` as soon as their inputs exist; the main
    // stream carries only the chain of input gradients; `side` is joined at the end
    // (join = false: the caller joins it later)
    const bool bf = h->bf16;
    const int nh = (int)sets[0].size() - 1;
    const int R = mb.rows;
    // which chains take the fused kernel: all (1), those without weight gradients (2), those
    // of one parameter set (3)
    // (2 and 3 only after the fused forward, whose saves the chain reads without post)
    const bool want_fused = h->mlp_bwd_fused == 1 ||
                            (mb.tc_saved && ((h->mlp_bwd_fused == 2 && !grads) || (h->mlp_bwd_fused == 3 && E == 1)));
    bool split = false;
    if (bf && h->mlp_fused && want_fused && dout.h && rows > 0 && E <= kMlpMaxProbs &&
        fused_backward(h, mb, r0, sets, grads, E, X, rows, dout, ncols, dX, lddx, mask, ldmask, s, side, col0, join,
                       h->mlp_fin_split && rows >= kFinSplitRows ? dX2 : nullptr, &split))
        return split;
    auto G = [&](const float* p) { return grads + (p - h->params); };
    auto post = [&](int l, int e) {
        const int n = sets[e][l].out;
        Mat m;
        m.f = mb.post[l] + ((int64_t)e * R + r0) * n; m.ld = n;
        if (bf) { m.h = mb.posth[l] + ((int64_t)e * R + r0) * n; m.ldh = n; }
        return m;
    };
    auto dpre = [&](int l, int e) {
        const int n = sets[e][l].out;
        Mat m;
        m.f = h->dpre[l] + (int64_t)e * rows * n; m.ld = n;
        if (bf) { m.h = h->dpre_h[l] + (int64_t)e * rows * n; m.ldh = n; }
        return m;
    };
    auto dout_e = [&](int e) {
        Mat m = dout;
        m.f += (int64_t)e * rows * dout.ld;
        if (m.h) m.h += (int64_t)e * rows * dout.ldh;
        return m;
    };
    // output layer; the column sums of the whole chain (biases, LayerNorm gains and shifts)
    // are collected and added up in one launch after the last weight gradient
    std::vector<ColSumProblem> cols;
    double col_bytes = 0;
    if (grads) {
        h->fork(s, side);
        {
            GemmBuilder gb(h, side, bf);
            for (int e = 0; e < E; ++e) gb.dw(dout_e(e), rows, post(nh - 1, e), sets[e][nh], G(sets[e][nh].w));
        }
        for (int e = 0; e < E; ++e)
            cols.push_back(ColSumProblem{rows, sets[e][nh].out, dout_e(e).f, dout.ld, G(sets[e][nh].b)});
        col_bytes += 4.0 * E * rows * sets[0][nh].out;
    }
    {
        GemmBuilder gb(h, s, bf);
        for (int e = 0; e < E; ++e) {
            const Mat d = dout_e(e);
            gb.dx(&d, &sets[e][nh], 1, rows, 0, sets[e][nh].in, h->dpost[nh - 1] + (int64_t)e * rows * sets[e][nh].in,
                  sets[e][nh].in);
        }
    }
    for (int l = nh - 1; l >= 0; --l) {
        LnBwdProblem lb[2];
        for (int e = 0; e < E; ++e) {
            const LayerRef& ly = sets[e][l];
            LnBwdProblem p{};
            p.rows = rows; p.n = ly.out;
            p.dout = h->dpost[l] + (int64_t)e * rows * ly.out; p.ld_dout = ly.out;
            p.out = post(l, e).f; p.ld_out = ly.out;
            p.pre = mb.pre[l] + ((int64_t)e * R + r0) * ly.out; p.ld_pre = ly.out;
            p.mean = mb.mean[l] + (int64_t)e * R + r0; p.rstd = mb.rstd[l] + (int64_t)e * R + r0;
            p.g = ly.g;
            p.dpre = dpre(l, e).f; p.ld_dpre = ly.out;
            if (bf) { p.dpre_bf = dpre(l, e).h; p.ld_dpre_bf = ly.out; }
            if (grads) { p.dg = G(ly.g); p.dbeta = G(ly.beta); p.dbias = G(ly.b); }
            if (grads && !mb.lnterms.empty()) p.terms = mb.lnterms[l] + (int64_t)e * 2 * rows * ly.out;
            lb[e] = p;
        }
        {
            ProfScope ps(h, s, "layernorm_bwd", 4.0 * E * rows * sets[0][l].out * (grads ? 9.0 : 5.0), 1);
            launch_ln_bwd(lb, E, h->ln_work, s);
        }
        if (grads) {
            // the LayerNorm's column sums and the weight gradients beside the input-gradient chain
            h->fork(s, side);
            for (int e = 0; e < E; ++e) {
                const LnBwdProblem& q = lb[e];
                if (q.terms) {
                    if (q.dg) cols.push_back(ColSumProblem{q.rows, q.n, q.terms, q.n, q.dg});
                    if (q.dbeta) cols.push_back(ColSumProblem{q.rows, q.n, q.terms + (int64_t)q.rows * q.n, q.n, q.dbeta});
                    if (q.dbias) cols.push_back(ColSumProblem{q.rows, q.n, q.dpre, q.ld_dpre, q.dbias});
                }
            }
            col_bytes += 4.0 * E * rows * sets[0][l].out * 3.0;
            GemmBuilder gb(h, side, bf);
            for (int e = 0; e < E; ++e) gb.dw(dpre(l, e), rows, l == 0 ? X : post(l - 1, e), sets[e][l], G(sets[e][l].w));
        }
        if (l > 0) {
            GemmBuilder gb(h, s, bf);
            for (int e = 0; e < E; ++e) {
                const Mat d = dpre(l, e);
                gb.dx(&d, &sets[e][l], 1, rows, 0, sets[e][l].in, h->dpost[l - 1] + (int64_t)e * rows * sets[e][l].in,
                      sets[e][l].in);
            }
        }
    }
    if (!cols.empty()) {
        ProfScope ps(h, side, "colsum", col_bytes, 1);
        launch_colsum(cols.data(), (int)cols.size(), side);
    }
    if (dX) {
        GemmBuilder gb(h, s, bf);
        Mat d[2] = {dpre(0, 0), E > 1 ? dpre(0, 1) : dpre(0, 0)};
        LayerRef w[2] = {sets[0][0], E > 1 ? sets[1][0] : sets[0][0]};
        gb.dx(d, w, E, rows, col0, ncols, dX, lddx, mask, ldmask);
    }
    if (grads && join) h->fork(side, s);
    return false;
}

void alloc_mlp(squint_handle* h, MlpBufs& mb, const std::vector<Lin>& layers, int E, int rows, bool terms = false) {
    const int nh = (int)layers.size() - 1;
    mb.E = E;
    mb.rows = rows;
    mb.pre.resize(nh); mb.post.resize(nh); mb.mean.resize(nh); mb.rstd.resize(nh);
    for (int l = 0; l < nh; ++l) {
        if (terms) mb.lnterms.push_back(h->dalloc<float>((int64_t)E * 2 * rows * layers[l].out));
        mb.pre[l] = h->dalloc<float>((int64_t)E * rows * layers[l].out);
        mb.post[l] = h->dalloc<float>((int64_t)E * rows * layers[l].out);
        mb.mean[l] = h->dalloc<float>((int64_t)E * rows);
        mb.rstd[l] = h->dalloc<float>((int64_t)E * rows);
        if (h->bf16) mb.posth.push_back(h->dalloc<__nv_bfloat16>((int64_t)E * rows * layers[l].out));
    }
    mb.out = h->dalloc<float>((int64_t)E * rows * layers[nh].out);
}

}  // namespace

int squint_handle::allocate() {
    const int B = c.batch, A = c.action_dim, K = c.critic_kind == 1 ? 1 : c.atoms, E = 2;
    fp8 = c.precision == SQUINT_PREC_FP8 || c.precision == SQUINT_PREC_MXFP8;
    mx = c.precision == SQUINT_PREC_MXFP8;
    if (const char* e = std::getenv("SQUINT_FUSED_LN")) fuse_ln = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_GEMM_SPLIT")) gemm_split = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_DRAW_AHEAD")) draw_ahead = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_MLP_FUSED")) mlp_fused = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_MLP_CL")) {
        // one value for every chain, or one per chain: "online,actor,target,actor-step"
        mlp_cluster = std::atoi(e);
        for (int i = 0; i < 4; ++i) mlp_cluster_site[i] = mlp_cluster;   // (also replaces the defaults)
        const char* p = e;
        for (int i = 0; i < 4 && p; ++i) {
            mlp_cluster_site[i] = std::atoi(p);
            p = std::strchr(p, ',');
            if (p) ++p;
        }
    }
    if (const char* e = std::getenv("SQUINT_MLP_SITES")) mlp_fused_sites = std::atoi(e);
    if (const char* e = std::getenv("SQUINT_MLP_BWD")) mlp_bwd_fused = std::atoi(e);
    if (const char* e = std::getenv("SQUINT_PRIO")) prio_branches = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_FUSE_POLYAK")) fuse_polyak = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_MLP_BWD_CL")) mlp_bwd_cluster = std::atoi(e);
    if (const char* e = std::getenv("SQUINT_MLP_FIN_SPLIT")) mlp_fin_split = std::atoi(e) != 0;
    if (const char* e = std::getenv("SQUINT_SPLIT_ACTOR_FWD")) split_actor_fwd = std::atoi(e) != 0;
    bf16 = c.precision == SQUINT_PREC_BF16 || fp8;
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
    d_err = dalloc<int32_t>(1);
    d_stats = dalloc<float>((int64_t)c.max_k * 8);
    const int64_t img = (int64_t)L.img_c * L.hs * L.ws;
    x2 = dalloc<float>(2 * B * img);
    sums = dalloc<uint16_t>(2 * B * img);
    idx2 = dalloc<int32_t>(2 * B);
    shift2 = dalloc<int32_t>(4 * B);
    // tensor-core convolutions for the 32 -> 32 stride-1 layers of a BF16 learner
    if (bf16) {
        tc_conv = L.conv.size() >= 2 && L.conv[0].cout == 32;
        for (size_t l = 1; l < L.conv.size(); ++l) {
            const ConvL& cv = L.conv[l];
            if (cv.cin != 32 || cv.cout != 32 || cv.s != 1) tc_conv = false;
        }
    }
    // encoder recompute: chunk size rounded up to the weight gradient's images per CTA, so
    // the chunked weight gradient has the same partition (and bits) as the whole-batch one
    if (c.recompute_chunk < 0 || (c.recompute_chunk > 0 && !tc_conv)) {
        g_last_error = "recompute_chunk needs a BF16 learner with 32-channel stride-1 inner convolutions";
        return SQUINT_EINVAL;
    }
    if (c.recompute_chunk > 0) {
        const int pc = wgrad32_per_cta(B);
        rc_chunk = std::min((c.recompute_chunk + pc - 1) / pc * pc, 2 * B);
    }
    const int enc_imgs = rc_chunk ? rc_chunk : 2 * B;   // images held by the encoder's buffers
    for (size_t l = 0; l < L.conv.size(); ++l) {
        const ConvL& cv = L.conv[l];
        const int64_t per = (int64_t)cv.cout * cv.oh * cv.ow;
        if (l + 1 == L.conv.size()) conv_out.push_back(dalloc<float>(2 * B * per));     // features z
        else if (l == 0) conv_out.push_back(tc_conv ? nullptr : dalloc<float>(2 * B * per));
        else conv_out.push_back(tc_conv ? nullptr : dalloc<float>(2 * B * per));
    }
    if (L.D > 0) {
        proj_pre = dalloc<float>((int64_t)5 * B * L.D);
        proj_mean = dalloc<float>(5 * B);
        proj_rstd = dalloc<float>(5 * B);
        proj_terms = dalloc<float>((int64_t)2 * B * L.D);
    }
    xa = dalloc<float>((int64_t)2 * B * L.da);
    xcbar = dalloc<float>((int64_t)B * L.dc);
    xc = dalloc<float>((int64_t)B * L.dc);
    xq = dalloc<float>((int64_t)B * L.dc);
    alloc_mlp(this, actor_mlp, L.actor, 1, 2 * B, true);
    alloc_mlp(this, tcrit_mlp, L.critic[0], E, B);
    alloc_mlp(this, crit_mlp, L.critic[0], E, B, true);
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
        if (bf16) dpre_h.push_back(dalloc<__nv_bfloat16>((int64_t)E * B * w));
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
    if (!tc_conv) dconv_b = dalloc<float>(maxc);
    wgrad_work = dalloc<float>(maxw);
    dxq = dalloc<float>((int64_t)B * L.dc);
    dxq2 = dalloc<float>((int64_t)B * L.dc);
    {
        int wmax = std::max(L.D, 1);
        for (int l = 0; l < c.n_hidden; ++l) wmax = std::max(wmax, c.hidden[l]);
        ln_work = dalloc<float>(kLnTickets + (int64_t)2 * ((B + 7) / 8) * 3 * wmax);
        if (ln_work) cudaMemset(ln_work, 0, kLnTickets * sizeof(float));
    }
    ln_prepare();
    if (bf16)
        for (int l = 0; l < c.n_hidden; ++l)
            mlp_colpart.push_back(dalloc<float>((int64_t)2 * ((B + 127) / 128) * 3 * std::max(c.hidden[l], 1)));
    dout_a = dalloc<float>((int64_t)B * 2 * A);
    if (bf16) {
        // padded BF16 weight copies: online for every linear layer, target for the critic range
        auto add = [&](const Lin& ly, bool with_target) {
            LinBf lb;
            lb.ld = pad8(ly.in);
            lb.on = dalloc<__nv_bfloat16>((int64_t)ly.out * lb.ld);
            if (with_target) lb.tg = dalloc<__nv_bfloat16>((int64_t)ly.out * lb.ld);
            lin_bf[ly.w] = lb;
            if (fp8) {
                // e4m3 copies (row stride a multiple of 16 bytes), one scale per copy
                LinF8 f;
                f.ld = (ly.in + 15) / 16 * 16;
                float* sc = dalloc<float>(2);
                f.on = dalloc<uint8_t>((int64_t)ly.out * f.ld);
                f.s_on = sc;
                if (with_target) { f.tg = dalloc<uint8_t>((int64_t)ly.out * f.ld); f.s_tg = sc + 1; }
                if (mx) {
                    f.sf_on = dalloc<uint8_t>(mx_scale_bytes(ly.out, ly.in));
                    if (with_target) f.sf_tg = dalloc<uint8_t>(mx_scale_bytes(ly.out, ly.in));
                }
                lin_f8[ly.w] = f;
            }
        };
        if (L.D > 0) { add(L.cproj, true); add(L.aproj, false); }
        for (int e = 0; e < 2; ++e) for (const auto& ly : L.critic[e]) add(ly, true);
        for (const auto& ly : L.actor) add(ly, false);
        if (fp8) {
            for (auto& a : f8_arena) {
                a.bytes = int64_t(24) << 20;
                a.buf = dalloc<uint8_t>(a.bytes);
                a.part = dalloc<float>(quant_workspace());
                a.scales = dalloc<float>(kF8Scales);
            }
        }
        z_h = dalloc<__nv_bfloat16>((int64_t)2 * B * L.feat);
        xa_h = dalloc<__nv_bfloat16>((int64_t)2 * B * pad8(L.da));
        xcbar_h = dalloc<__nv_bfloat16>((int64_t)B * pad8(L.dc));
        xc_h = dalloc<__nv_bfloat16>((int64_t)B * pad8(L.dc));
        xq_h = dalloc<__nv_bfloat16>((int64_t)B * pad8(L.dc));
        dlogits_h = dalloc<__nv_bfloat16>((int64_t)E * B * pad8(K));
        dlogits_qh = dalloc<__nv_bfloat16>((int64_t)E * B * pad8(K));
        if (L.D > 0) dproj_h = dalloc<__nv_bfloat16>((int64_t)B * L.D);
        dout_ah = dalloc<__nv_bfloat16>((int64_t)B * pad8(2 * A));
    }
    // the front end's outputs twice over: update j of a call reads set j % 2 while the
    // front end of update j + 1 writes the other
    fe_set[0] = FeSet{x2, r, d, xa, xcbar, xc, xq, xa_h, xcbar_h, xc_h, xq_h};
    fe_set[1] = fe_set[0];
    if (c.max_k > 1) {
        FeSet& f = fe_set[1];
        f.x2 = dalloc<float>(2 * B * img);
        f.r = dalloc<float>(B);
        f.d = dalloc<float>(B);
        f.xa = dalloc<float>((int64_t)2 * B * L.da);
        f.xcbar = dalloc<float>((int64_t)B * L.dc);
        f.xc = dalloc<float>((int64_t)B * L.dc);
        f.xq = dalloc<float>((int64_t)B * L.dc);
        if (bf16) {
            f.xa_h = dalloc<__nv_bfloat16>((int64_t)2 * B * pad8(L.da));
            f.xcbar_h = dalloc<__nv_bfloat16>((int64_t)B * pad8(L.dc));
            f.xc_h = dalloc<__nv_bfloat16>((int64_t)B * pad8(L.dc));
            f.xq_h = dalloc<__nv_bfloat16>((int64_t)B * pad8(L.dc));
        }
    }
    // padded-HWC BF16 activations (forward: enc_imgs images; backward: one chunk of o_t)
    const int bwd_imgs = rc_chunk ? rc_chunk : B;
    if (tc_conv) {
        const int nl = (int)L.conv.size();
        for (int l = 0; l < nl - 1; ++l) {
            const ConvL& cv = L.conv[l];
            const int64_t img = (int64_t)(cv.oh + 4) * (cv.ow + 4) * 32;
            act_p.push_back(dalloc<__nv_bfloat16>(enc_imgs * img));
            dact_p.push_back(dalloc<__nv_bfloat16>(bwd_imgs * img));
        }
        const ConvL& last = L.conv.back();
        dz_p = dalloc<__nv_bfloat16>((int64_t)bwd_imgs * (last.oh + 4) * (last.ow + 4) * 32);
        wconv_fwd.assign(nl, nullptr);
        wconv_bwd.assign(nl, nullptr);
        for (int l = 1; l < nl; ++l) {
            wconv_fwd[l] = dalloc<__nv_bfloat16>(9 * 32 * 32);
            wconv_bwd[l] = dalloc<__nv_bfloat16>(9 * 32 * 32);
        }
        // with recompute every inner layer keeps its partials until all chunks are done
        wgrad_tc_work = dalloc<float>((rc_chunk ? nl - 1 : 1) * wgrad32_tc_workspace(B));
    }
    for (void* p : allocations)
        if (!p) { g_last_error = "device allocation failed"; return SQUINT_ENOMEM; }
    if (bf16)   // the BF16 head inputs' pad columns stay zero
        for (const FeSet& f : fe_set) {
            SQ_CK(this, cudaMemset(f.xa_h, 0, (size_t)2 * B * pad8(L.da) * 2));
            SQ_CK(this, cudaMemset(f.xcbar_h, 0, (size_t)B * pad8(L.dc) * 2));
            SQ_CK(this, cudaMemset(f.xc_h, 0, (size_t)B * pad8(L.dc) * 2));
            SQ_CK(this, cudaMemset(f.xq_h, 0, (size_t)B * pad8(L.dc) * 2));
        }
    if (tc_conv) {
        // padded buffers keep zero borders: only interiors are ever written
        for (size_t l = 0; l < act_p.size(); ++l) {
            const ConvL& cv = L.conv[l];
            const int64_t img = (int64_t)(cv.oh + 4) * (cv.ow + 4) * 32;
            SQ_CK(this, cudaMemset(act_p[l], 0, (size_t)enc_imgs * img * 2));
            SQ_CK(this, cudaMemset(dact_p[l], 0, (size_t)bwd_imgs * img * 2));
        }
        const ConvL& last = L.conv.back();
        SQ_CK(this, cudaMemset(dz_p, 0, (size_t)bwd_imgs * (last.oh + 4) * (last.ow + 4) * 32 * 2));
        conv_tc_prepare();
    }
    if (bf16) {
        if (L.feat % 8) { g_last_error = "BF16 path needs a feature width divisible by 8"; return SQUINT_EINVAL; }
        auto item = [&](const Lin& ly, bool tgt) {
            const LinBf& lb = lin_bf[ly.w];
            const float* src = tgt ? target + (ly.w - L.critic_begin) : params + ly.w;
            return CastItem{src, ly.in, ly.out, ly.in, tgt ? lb.tg : lb.on, lb.ld};
        };
        if (L.D > 0) { cast_critic.push_back(item(L.cproj, false)); cast_target.push_back(item(L.cproj, true)); }
        for (int e = 0; e < 2; ++e)
            for (const auto& ly : L.critic[e]) { cast_critic.push_back(item(ly, false)); cast_target.push_back(item(ly, true)); }
        if (L.D > 0) cast_actor.push_back(item(L.aproj, false));
        for (const auto& ly : L.actor) cast_actor.push_back(item(ly, false));
        auto seg = [&](const Lin& ly, int64_t begin, bool tgt) {
            const LinBf& lb = lin_bf[ly.w];
            return BfSeg{ly.w - begin, ly.out, ly.in, lb.ld, tgt ? lb.tg : lb.on};
        };
        if (L.D > 0) {
            seg_critic.push_back(seg(L.cproj, L.critic_begin, false));
            seg_target.push_back(seg(L.cproj, L.critic_begin, true));
            seg_actor.push_back(seg(L.aproj, L.actor_begin, false));
        }
        for (int e = 0; e < 2; ++e)
            for (const auto& ly : L.critic[e]) {
                seg_critic.push_back(seg(ly, L.critic_begin, false));
                seg_target.push_back(seg(ly, L.critic_begin, true));
            }
        for (const auto& ly : L.actor) seg_actor.push_back(seg(ly, L.actor_begin, false));
        if ((int)seg_critic.size() > kMaxBfSeg || (int)seg_actor.size() > kMaxBfSeg) {
            g_last_error = "too many weight matrices for the fused BF16 copies";
            return SQUINT_EINVAL;
        }
        if (fp8) {
            auto q = [&](const Lin& ly, bool tgt) {
                const LinBf& lb = lin_bf[ly.w];
                const LinF8& f = lin_f8[ly.w];
                return QuantItem{tgt ? lb.tg : lb.on, lb.ld, ly.out, ly.in, tgt ? f.tg : f.on, f.ld,
                                 tgt ? f.s_tg : f.s_on, tgt ? f.sf_tg : f.sf_on};
            };
            if (L.D > 0) { quant_critic.push_back(q(L.cproj, false)); quant_target.push_back(q(L.cproj, true)); }
            for (int e = 0; e < 2; ++e)
                for (const auto& ly : L.critic[e]) { quant_critic.push_back(q(ly, false)); quant_target.push_back(q(ly, true)); }
            if (L.D > 0) quant_actor.push_back(q(L.aproj, false));
            for (const auto& ly : L.actor) quant_actor.push_back(q(ly, false));
        }
        // inference snapshots: BF16 actor-path matrices and conv filter layouts per snapshot
        std::vector<const Lin*> pol;
        if (L.D > 0) pol.push_back(&L.aproj);
        for (const auto& ly : L.actor) pol.push_back(&ly);
        int64_t tot = 0;
        for (const Lin* ly : pol) {
            policy_bf_off[ly->w] = {tot, pad8(ly->in)};
            tot += (int64_t)ly->out * pad8(ly->in);
        }
        for (int i = 0; i < 2; ++i) {
            policy_bf[i] = dalloc<__nv_bfloat16>(tot);
            for (const Lin* ly : pol) {
                const auto& o = policy_bf_off[ly->w];
                cast_policy[i].push_back(CastItem{policy_buf[i] + ly->w, ly->in, ly->out, ly->in, policy_bf[i] + o.first,
                                                  o.second});
            }
            if (tc_conv) policy_wconv[i] = dalloc<__nv_bfloat16>((int64_t)(L.conv.size() - 1) * 9 * 32 * 32);
        }
        if (tc_conv) policy_wconv_scratch = dalloc<__nv_bfloat16>(9 * 32 * 32);
        tc_prepare();
        mlp_tc_prepare();
        mlp_bwd_tc_prepare();
    }
    if (cudaMallocHost(&h_stats, sizeof(float) * 8 * c.max_k) != cudaSuccess) return SQUINT_ENOMEM;
    {
        // the update's critical chain (main stream; weight gradients, critic forward and
        // polyak branches, which it joins) one level below the serving streams; the
        // encoder backward (which has slack until the update ends) and the next update's
        // front end at the lowest priority
        int least = 0, greatest = 0;
        SQ_CK(this, cudaDeviceGetStreamPriorityRange(&least, &greatest));
        const int crit = greatest < least ? greatest + 1 : greatest;
        SQ_CK(this, cudaStreamCreateWithPriority(&capture_stream, cudaStreamNonBlocking, prio_branches ? crit : 0));
        for (int i = 0; i < 5; ++i) {
            const bool low = i == 0 || i == 3 || i == 4;
            SQ_CK(this, cudaStreamCreateWithPriority(&side[i], cudaStreamNonBlocking,
                                                     prio_branches ? (low ? least : crit) : 0));
        }
    }
    for (auto& e : fork_ev) SQ_CK(this, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) SQ_CK(this, cudaEventCreateWithFlags(&policy_ready[i], cudaEventDisableTiming));
    arenas.push_back(&arena);
    frontend_prepare(L.conv.empty() ? 0 : (size_t)c.obs_c * c.obs_h * c.obs_w);

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
    SQ_CK(this, cudaMemset(d_err, 0, sizeof(int32_t)));
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
    free_arena(arena);
    arenas.clear();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    capture_stream = nullptr;
    for (auto& st : side) { if (st) cudaStreamDestroy(st); st = nullptr; }
    for (auto& e : fork_ev) { if (e) cudaEventDestroy(e); e = nullptr; }
    for (int i = 0; i < 2; ++i) {
        if (policy_ready[i]) cudaEventDestroy(policy_ready[i]);
        policy_ready[i] = nullptr;
    }
}

void squint_handle::quantize_weights(const std::vector<QuantItem>& q, cudaStream_t s) {
    if (!fp8 || q.empty()) return;
    double bytes = 0;
    for (const auto& it : q) bytes += 3.0 * it.rows * it.cols;
    if (mx) {
        ProfScope ps(this, s, "quantize_mxfp8", bytes, 1);
        launch_quantize_mx(q.data(), (int)q.size(), s);
        return;
    }
    ProfScope ps(this, s, "quantize_fp8", bytes, 1);
    launch_quantize_e4m3(q.data(), (int)q.size(), arena_for(s)->part, s);
}

void squint_handle::snapshot_bf16(int i, cudaStream_t s) {
    if (!bf16) return;
    launch_cast_rows(cast_policy[i].data(), (int)cast_policy[i].size(), s);
    if (tc_conv)
        for (size_t l = 1; l < L.conv.size(); ++l)
            launch_conv_weight_cast(policy_buf[i] + L.conv[l].wo, policy_wconv[i] + (l - 1) * 9 * 32 * 32,
                                    policy_wconv_scratch, s);
}

int squint_handle::after_param_change() {
    SQ_CK(this, cudaDeviceSynchronize());
    for (int i = 0; i < 2; ++i) {
        SQ_CK(this, cudaMemcpy(policy_buf[i], params, L.total * sizeof(float), cudaMemcpyDeviceToDevice));
        snapshot_bf16(i, 0);
    }
    if (bf16) {
        launch_cast_rows(cast_critic.data(), (int)cast_critic.size(), 0);
        launch_cast_rows(cast_actor.data(), (int)cast_actor.size(), 0);
        launch_cast_rows(cast_target.data(), (int)cast_target.size(), 0);
        quantize_weights(quant_critic, 0);
        quantize_weights(quant_actor, 0);
        quantize_weights(quant_target, 0);
        cast_conv_weights(0);
        SQ_CK(this, cudaDeviceSynchronize());
    }
    ++policy_version;
    return SQUINT_OK;
}

void squint_handle::record_update(int j, int k, cudaStream_t s, bool debug) {
    const int B = c.batch, A = c.action_dim, P = c.proprio_dim, K = c.critic_kind == 1 ? 1 : c.atoms, E = 2;
    const int F = L.feat, Z = L.zdim, Dd = L.D, Dc = L.dc, Da = L.da;
    const int64_t Dc8 = pad8(Dc), Da8 = pad8(Da), K8 = pad8(K);
    const float ln_eps = (float)c.ln_eps;
    float* W = params;
    float* G = grads;
    float* stats = d_stats + 8 * j;
    // branches: s1 encoder backward, s2 weight gradients of the MLPs, s3 critic forward / polyak,
    // s4 the encoder's inner weight gradients beside its data-gradient chain
    cudaStream_t s1 = branch(s, 0), s2 = branch(s, 1), s3 = branch(s, 2), s4 = branch(s, 3);
    // the next update's front end, drawn beside this update into the other buffer set
    cudaStream_t sp = branch(s, 4);
    const bool draw_next = draw_ahead && j + 1 < k;
    use_set(j & 1);
    auto cast_rows = [&](const float* src, int64_t ld, int rows, int cols, __nv_bfloat16* dst, int64_t ldh,
                         cudaStream_t st) {
        if (!bf16) return;
        CastItem it{src, ld, rows, cols, dst, ldh};
        ProfScope ps(this, st, "cast_bf16", 6.0 * rows * cols, 1);
        launch_cast_rows(&it, 1, st);
    };
    auto ln_fwd = [&](const LnProblem* p, int n, bool relu, cudaStream_t st) {
        double bytes = 0;
        for (int i = 0; i < n; ++i) bytes += 12.0 * p[i].rows * p[i].n;
        ProfScope ps(this, st, "layernorm_fwd", bytes, 1);
        launch_ln_fwd(p, n, relu, ln_eps, st);
    };
    auto ln_bwd = [&](const LnBwdProblem* p, int n, cudaStream_t st) {
        double bytes = 0;
        for (int i = 0; i < n; ++i) bytes += 36.0 * p[i].rows * p[i].n;
        ProfScope ps(this, st, "layernorm_bwd", bytes, 1);
        launch_ln_bwd(p, n, ln_work, st);
    };
    auto adam = [&](int64_t begin, int64_t end, const int32_t* step, const int32_t* enable, cudaStream_t st,
                    const std::vector<BfSeg>* segs = nullptr, bool with_polyak = false) {
        if (end <= begin) return;                  // empty range (state-based: no encoder)
        AdamArgs ad{};
        if (segs) {
            for (size_t k = 0; k < segs->size(); ++k) ad.seg[k] = (*segs)[k];
            ad.n_seg = (int)segs->size();
        }
        if (with_polyak) {   // the target copy of this (critic) range in the same pass
            ad.target = target;
            ad.tau = (float)c.tau;
            if (bf16) {
                for (size_t k = 0; k < seg_target.size(); ++k) ad.tseg[k] = seg_target[k];
                ad.n_tseg = (int)seg_target.size();
            }
        }
        ad.p = W + begin; ad.g = G + begin; ad.m = adam_m + begin; ad.v = adam_v + begin;
        ad.n = end - begin;
        ad.step = step; ad.enable = enable;
        ad.lr = c.lr; ad.b1 = c.adam_b1; ad.b2 = c.adam_b2; ad.eps = c.adam_eps;
        double bf_bytes = 0;   // the BF16 copies written alongside
        for (int k = 0; k < ad.n_seg; ++k) bf_bytes += 2.0 * ad.seg[k].rows * ad.seg[k].cols;
        for (int k = 0; k < ad.n_tseg; ++k) bf_bytes += 2.0 * ad.tseg[k].rows * ad.tseg[k].cols;
        ProfScope ps(this, st, "adam", (with_polyak ? 36.0 : 28.0) * (double)ad.n + bf_bytes, 1);
        if (launch_adam(ad, st) != 0) launch_failed = true;
    };
    auto conv_flops = [&](const ConvL& cv, int nimg) { return 2.0 * nimg * cv.oh * cv.ow * cv.cout * cv.cin * 9; };

    mark(s);
    // ---- a1-a4: minibatch, gathers, shift, squint of update j + ahead into set `set`
    // (the update index the draws use is read before this update advances it)
    auto frontend = [&](int set, int ahead, cudaStream_t st) {
        const FeSet& fs = fe_set[set];
        FrontendArgs fa{};
        fa.obs = ring.obs; fa.proprio = ring.proprio; fa.action = ring.action; fa.reward = ring.reward; fa.done = ring.done;
        fa.n_slots = ring.n;
        fa.C = c.obs_c; fa.H = c.obs_h; fa.W = c.obs_w; fa.f = c.squint_f; fa.pad = c.shift_pad;
        if (L.conv.empty()) { fa.C = 0; fa.H = fa.W = fa.f = 1; fa.pad = 0; }   // state-based: no image
        fa.P = P; fa.A = A; fa.B = B;
        fa.seed = c.seed; fa.update_idx = d_update_idx; fa.idx_offset = ahead;
        fa.x = fs.x2; fa.x_bf = nullptr; fa.sums = debug ? sums : nullptr;
        fa.idx_out = idx2; fa.shift_out = shift2; fa.r_out = fs.r; fa.d_out = fs.d;
        // the transition fields land in the head inputs, with their BF16 shadows in BF16 mode
        fa.dst[0] = CopyDst{fs.xc, Dc, Z, 0, fs.xc_h, Dc8};
        fa.dst[1] = CopyDst{fs.xc, Dc, Z + P, 2, fs.xc_h, Dc8};
        fa.dst[2] = CopyDst{fs.xq, Dc, Z, 0, fs.xq_h, Dc8};
        fa.dst[3] = CopyDst{fs.xa + (int64_t)B * Da, Da, Z, 0, fs.xa_h ? fs.xa_h + (int64_t)B * Da8 : nullptr, Da8};
        fa.dst[4] = CopyDst{fs.xa, Da, Z, 1, fs.xa_h, Da8};
        fa.dst[5] = CopyDst{fs.xcbar, Dc, Z, 1, fs.xcbar_h, Dc8};
        fa.n_dst = 6;
        fa.err = d_err;
        // frames read and squinted images written, plus the transition rows gathered
        // (s_t, s_{t+1}, a_t, r, d) and written into the head inputs (with BF16 shadows)
        const int64_t img = (int64_t)L.img_c * L.hs * L.ws;
        const double trans = B * (4.0 * (2 * P + A + 1) + 1 + (5.0 * P + A) * (bf16 ? 6.0 : 4.0) + 8.0);
        ProfScope ps(this, st, "frontend", 2.0 * B * fa.C * fa.H * fa.W + 2.0 * B * img * 4 + trans, 1);
        launch_frontend(fa, st);
    };
    if (j == 0 || !draw_ahead) frontend(j & 1, 0, s);   // else drawn by the previous update

    mark(s);
    // ---- a5: encoder on o_t (rows < B) and o_{t+1} (rows >= B)
    const int nconv = (int)L.conv.size();
    // tensor-core encoder over images [i0, i0 + n) of x2; layers 0 .. upto, where layer
    // nconv - 1 writes the features of those rows (FP32 and BF16)
    auto enc_tc = [&](int i0, int n, int upto, cudaStream_t st) {
        const ConvL& c0 = L.conv[0];
        const int64_t img0 = (int64_t)c.obs_c * c0.h * c0.w;
        ConvShape sh{n, c0.cin, c0.h, c0.w, c0.cout, c0.s, c0.oh, c0.ow, img0, (int64_t)c0.cout * c0.oh * c0.ow};
        {
            // first layer on tensor cores (CUDA cores outside that kernel's range), written
            // straight into the padded-HWC input of layer 1
            ProfScope ps(this, st, "conv_tc_fwd", conv_flops(c0, n), 0);
            if (launch_conv0_tc(sh, x2 + (int64_t)i0 * img0, W + c0.wo, W + c0.bo, act_p[0], d_err, st) < 0)
                launch_conv0_phwc(sh, x2 + (int64_t)i0 * img0, W + c0.wo, W + c0.bo, act_p[0], st);
        }
        for (int l = 1; l <= upto; ++l) {
            const ConvL& cv = L.conv[l];
            ConvTc ct{};
            ct.in = act_p[l - 1];
            ct.nimg = n;
            ct.Wp = cv.w + 4;
            ct.in_rows = (cv.h + 4) * ct.Wp;
            ct.out_h = cv.oh; ct.out_w = cv.ow;
            ct.off0 = 2 * ct.Wp + 2;
            ct.w = wconv_fwd[l];
            ct.bias = W + cv.bo;
            ct.relu = 1;
            if (l < nconv - 1) ct.out_phwc = act_p[l];
            else { ct.out_chw = conv_out[l] + (int64_t)i0 * F; ct.out_chw_bf = z_h + (int64_t)i0 * F; }
            ProfScope ps(this, st, "conv_tc_fwd", conv_flops(cv, n), 0);
            if (launch_conv32_tc(ct, d_err, st) != 0) launch_failed = true;
        }
    };
    if (tc_conv) {
        const int chunk = rc_chunk ? rc_chunk : 2 * B;
        for (int i0 = 0; i0 < 2 * B; i0 += chunk) enc_tc(i0, std::min(chunk, 2 * B - i0), nconv - 1, s);
    } else {
        const float* in = x2;
        for (int l = 0; l < nconv; ++l) {
            const ConvL& cv = L.conv[l];
            ConvShape sh{2 * B, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                         (int64_t)cv.cout * cv.oh * cv.ow};
            ProfScope ps(this, s, "conv_f32_fwd", conv_flops(cv, 2 * B), 0);
            launch_conv_fwd<float>(sh, in, W + cv.wo, W + cv.bo, conv_out[l], true, s);
            in = conv_out[l];
        }
    }
    float* z = nconv ? conv_out.back() : nullptr;   // [2B, F] (state-based: F = 0, no features)
    if (!tc_conv && F > 0) cast_rows(z, F, 2 * B, F, z_h, F, s);
    const Mat zt{z, F, z_h, F};
    const Mat zt1 = zt.rows(B);

    if (draw_next) {
        // the next update's minibatch while this one runs its latency-bound heads; it
        // writes the set update j - 1 used (finished: its branches joined before this
        // update began) and is joined before this update advances the update index
        fork(s, sp);
        frontend((j + 1) & 1, 1, sp);
    }
    mark(s);
    // ---- a6: per-head projections (or the flattened features straight into the heads)
    if (Dd > 0) {
        const LayerRef ap = layer_ref(this, L.aproj, false), cp = layer_ref(this, L.cproj, false);
        const LayerRef cpt = layer_ref(this, L.cproj, true);
        {
            GemmBuilder gb(this, s, bf16);
            gb.fwd(zt1, B, ap, proj_pre + 0 * (int64_t)B * Dd, Dd);
            gb.fwd(zt1, B, cpt, proj_pre + 1 * (int64_t)B * Dd, Dd);
            gb.fwd(zt, B, cp, proj_pre + 2 * (int64_t)B * Dd, Dd);
            gb.fwd(zt, B, ap, proj_pre + 3 * (int64_t)B * Dd, Dd);
        }
        LnProblem lp[4];
        const LayerRef* refs[4] = {&ap, &cpt, &cp, &ap};
        float* outs[4] = {xa, xcbar, xc, xa + (int64_t)B * Da};
        __nv_bfloat16* outs_h[4] = {xa_h, xcbar_h, xc_h, xa_h ? xa_h + (int64_t)B * Da8 : nullptr};
        const int64_t lds[4] = {Da, Dc, Dc, Da};
        const int64_t lds_h[4] = {Da8, Dc8, Dc8, Da8};
        for (int i = 0; i < 4; ++i) {
            LnProblem p{};
            p.rows = B; p.n = Dd;
            p.pre = proj_pre + i * (int64_t)B * Dd; p.ld_pre = Dd;
            p.g = refs[i]->g; p.beta = refs[i]->beta;
            p.out = outs[i]; p.ld_out = lds[i];
            if (bf16) { p.out_bf = outs_h[i]; p.ld_out_bf = lds_h[i]; }
            p.mean = proj_mean + i * B; p.rstd = proj_rstd + i * B;
            lp[i] = p;
        }
        ln_fwd(lp, 4, false, s);
    } else if (F > 0) {
        const size_t fb = (size_t)F * sizeof(float);
        cudaMemcpy2DAsync(xa, Da * sizeof(float), zt1.f, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xa + (int64_t)B * Da, Da * sizeof(float), z, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xcbar, Dc * sizeof(float), zt1.f, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xc, Dc * sizeof(float), z, fb, fb, B, cudaMemcpyDeviceToDevice, s);
        cudaMemcpy2DAsync(xq, Dc * sizeof(float), z, fb, fb, B, cudaMemcpyDeviceToDevice, s);
    }
    if (Dd == 0) {     // flatten path: the features were copied in FP32 only
        cast_rows(xa, Da, 2 * B, Da, xa_h, Da8, s);
        cast_rows(xc, Dc, B, Dc, xc_h, Dc8, s);
    }

    const MlpRef actor_on = mlp_ref(this, L.actor, false);
    const MlpRef crit_on[2] = {mlp_ref(this, L.critic[0], false), mlp_ref(this, L.critic[1], false)};
    const MlpRef crit_tg[2] = {mlp_ref(this, L.critic[0], true), mlp_ref(this, L.critic[1], true)};

    // ---- a10 (forward part) on branch s3: online critics on (z, s, a), independent of the target
    fork(s, s3);
    mlp_forward(this, crit_mlp, crit_on, E, Mat{xc, Dc, xc_h, Dc8}, B, bf16, s3);

    mark(s);
    // ---- a7: actor (pre-update) on both halves; tanh-Gaussian sample.  Split: the o_{t+1}
    // half, which only the target reads, on the critical chain without saved activations,
    // and the o_t half (read by the temperature and actor steps, differentiated in the
    // actor step) with its saves and its sample on s2, joined before the critic Adam
    // (rows are independent in the fused forward and the sample, so the results are those
    // of one launch over both halves)
    const bool split_actor = split_actor_fwd && bf16 && !fp8 && mlp_fused && (mlp_fused_sites & 2);
    if (split_actor) {
        fork(s, s2);
        mlp_forward(this, actor_mlp, &actor_on, 1, Mat{xa + (int64_t)B * Da, Da, xa_h + (int64_t)B * Da8, Da8}, B, bf16,
                    s2, true, true, B);
    }
    {
        if (split_actor) mlp_forward(this, actor_mlp, &actor_on, 1, Mat{xa, Da, xa_h, Da8}, B, bf16, s, true, false);
        else mlp_forward(this, actor_mlp, &actor_on, 1, Mat{xa, Da, xa_h, Da8}, 2 * B, bf16, s);
        ActorHeadArgs ah{};
        ah.rows = 2 * B; ah.B = B; ah.A = A;
        ah.out = actor_mlp.out; ah.ld_out = 2 * A;
        ah.lo = (float)c.log_std_min; ah.hi = (float)c.log_std_max;
        ah.seed = c.seed; ah.update_idx = d_update_idx;
        ah.a_dst0 = xcbar + Z + P; ah.ld0 = Dc;
        ah.a_dst1 = xq + Z + P; ah.ld1 = Dc;
        if (bf16) {
            ah.a_dst0_h = xcbar_h + Z + P; ah.ld0_h = Dc8;
            ah.a_dst1_h = xq_h + Z + P; ah.ld1_h = Dc8;
        }
        ah.logp = logp; ah.eps = eps;
        if (split_actor) {
            ActorHeadArgs at = ah;   // the o_t half's sample on s2, after its forward
            at.row0 = B;
            ProfScope ps(this, s2, "heads_losses", 0, 1);
            launch_actor_head(at, s2);
        }
        {
            if (split_actor) ah.rows = B;   // the target half
            ProfScope ps(this, s, "heads_losses", 0, 1);
            launch_actor_head(ah, s);
        }
        if (Dd == 0) cast_rows(xcbar, Dc, B, Dc, xcbar_h, Dc8, s);
    }
    mark(s);
    // ---- a8-a9: target critics and the projected categorical target
    {
        mlp_forward(this, tcrit_mlp, crit_tg, E, Mat{xcbar, Dc, xcbar_h, Dc8}, B, bf16, s, true, false);
        C51TargetArgs ct{};
        ct.B = B; ct.K = K; ct.E = E;
        ct.logits_bar = tcrit_mlp.out; ct.r = r; ct.d = d; ct.logp_next = logp;
        ct.log_alpha = W + L.log_alpha;
        ct.gamma = (float)c.gamma; ct.v_min = (float)c.v_min; ct.v_max = (float)c.v_max;
        ct.m = m;
        ct.cdq = c.cdq; ct.mse = c.critic_kind == 1;
        // the step counters advance here, before their first reader (the critic Adam)
        ct.steps = d_steps; ct.do_actor = d_do_actor; ct.update_idx = d_update_idx; ct.policy_freq = c.policy_freq;
        ProfScope ps(this, s, "heads_losses", 0, 1);
        launch_c51_target(ct, s);
    }
    mark(s);
    // ---- a10: cross entropy against the projected target (joins the critic forward)
    fork(s3, s);
    {
        CeArgs ce{};
        ce.B = B; ce.K = K; ce.E = E; ce.logits = crit_mlp.out; ce.m = m;
        ce.v_min = (float)c.v_min; ce.v_max = (float)c.v_max;
        ce.scale = 1.0f / (float)B;
        ce.dlogits = dlogits; ce.row_loss = row_loss; ce.row_q = row_q;
        ce.mse = c.critic_kind == 1;
        if (bf16) { ce.dlogits_bf = dlogits_h; ce.ld_bf = K8; }
        ProfScope ps(this, s, "heads_losses", 0, 1);
        launch_ce(ce, s);
    }
    mark(s);
    // ---- a11: backward through critics and the critic projection (weight gradients on s2)
    {
        const Mat dl{dlogits, K, dlogits_h, K8};
        const float* mask = Dd > 0 ? nullptr : z;      // flatten path: mask by the last conv's ReLU
        // (with a projection its backward below joins s2 before the critic Adam)
        mlp_backward(this, crit_mlp, 0, crit_on, G, E, Mat{xc, Dc, xc_h, Dc8}, B, dl, Z, Dd > 0 ? dh : dz,
                     Dd > 0 ? Z : F, mask, F, s, s2, 0, Dd == 0);
        if (Dd > 0) {
            const LayerRef cp = layer_ref(this, L.cproj, false);
            LnBwdProblem p{};
            p.rows = B; p.n = Dd;
            p.dout = dh; p.ld_dout = Dd;
            p.pre = proj_pre + 2 * (int64_t)B * Dd; p.ld_pre = Dd;
            p.mean = proj_mean + 2 * B; p.rstd = proj_rstd + 2 * B;
            p.g = cp.g;
            p.dpre = dproj; p.ld_dpre = Dd;
            if (bf16) { p.dpre_bf = dproj_h; p.ld_dpre_bf = Dd; }
            p.dg = G + L.cproj.g; p.dbeta = G + L.cproj.beta; p.dbias = G + L.cproj.b;
            p.terms = proj_terms;
            ln_bwd(&p, 1, s);
            const Mat dp{dproj, Dd, dproj_h, Dd};
            fork(s, s2);
            {
                ProfScope ps(this, s2, "colsum", 12.0 * B * Dd, 1);
                launch_ln_bwd_cols(&p, 1, s2);
            }
            {
                GemmBuilder gb(this, s2, bf16);
                gb.dw(dp, B, zt, cp, G + L.cproj.w);
            }
            {
                GemmBuilder gb(this, s, bf16);
                gb.dx(&dp, &cp, 1, B, 0, F, dz, F, z, F);
            }
            fork(s2, s);
        }
    }
    mark(s);
    // ---- a12 (critic range): Adam over critic projection + critics, BF16 copies
    // (Adam writes the BF16 copies of the critic weights as it updates them)
    adam(L.critic_begin, L.critic_end, d_steps + 0, nullptr, s, bf16 ? &seg_critic : nullptr, fuse_polyak);
    quantize_weights(quant_critic, s);

    // ---- a11 (encoder part) + a12 (encoder range) on branch s1, beside the actor step
    fork(s, s1);
    {
        const float* cur = dz;
        if (tc_conv) {
            // o_t images in chunks (one chunk = the whole batch without recompute); with
            // recompute, each chunk's activations are recomputed first, and the inner
            // layers' weight-gradient partials stay at their whole-batch CTA slots until
            // one reduce per layer after the last chunk
            const ConvL& last = L.conv.back();
            const ConvL& c0 = L.conv[0];
            const int pc = wgrad32_per_cta(B);
            const int64_t wslot = (int64_t)kCh32 * (kCh32 * 9 + 1);
            const int chunk = rc_chunk ? rc_chunk : B;
            // without recompute, layer l's weight gradient runs on s4 as soon as its output
            // gradient exists, beside the data gradients of the layers below (chunks of the
            // recompute path reuse the activation buffers, so they stay in one order)
            cudaStream_t sw = rc_chunk ? s1 : s4;
            for (int i0 = 0; i0 < B; i0 += chunk) {
                const int n = std::min(chunk, B - i0);
                if (rc_chunk) enc_tc(i0, n, nconv - 2, s1);
                {
                    ProfScope ps(this, s1, "layout_phwc", 6.0 * n * F, 1);
                    launch_to_phwc(dz + (int64_t)i0 * F, F, n, last.oh, last.ow, dz_p, s1);
                }
                const __nv_bfloat16* cur_p = dz_p;
                for (int l = nconv - 1; l >= 1; --l) {
                    const ConvL& cv = L.conv[l];
                    WgradTc wt{};
                    wt.x = act_p[l - 1];
                    wt.dy = cur_p;
                    wt.nimg = n;
                    wt.Wp = cv.w + 4;
                    wt.in_rows = (cv.h + 4) * wt.Wp;
                    wt.out_h = cv.oh; wt.out_w = cv.ow;
                    {
                        fork(s1, sw);
                        ProfScope ps(this, sw, "conv_tc_wgrad", conv_flops(cv, n), 0);
                        int rc;
                        if (rc_chunk) {
                            float* work = wgrad_tc_work + (int64_t)(l - 1) * wgrad32_tc_workspace(B) +
                                          (int64_t)(i0 / pc) * wslot;
                            rc = launch_wgrad32_tc_partials(wt, pc, work, d_err, sw);
                        } else {
                            rc = launch_wgrad32_tc(wt, wgrad_tc_work, G + cv.wo, G + cv.bo, d_err, sw);
                        }
                        if (rc != 0) launch_failed = true;
                    }
                    ConvTc ct{};
                    ct.in = cur_p;
                    ct.nimg = n;
                    ct.Wp = cv.ow + 4;
                    ct.in_rows = (cv.oh + 4) * ct.Wp;
                    ct.out_h = cv.h; ct.out_w = cv.w;
                    ct.off0 = 0;
                    ct.w = wconv_bwd[l];
                    ct.mask = act_p[l - 1];
                    ct.out_phwc = dact_p[l - 1];
                    {
                        ProfScope ps(this, s1, "conv_tc_dgrad", conv_flops(cv, n), 0);
                        if (launch_conv32_tc(ct, d_err, s1) != 0) launch_failed = true;
                    }
                    cur_p = dact_p[l - 1];
                }
                // with recompute, each chunk's first-layer gradient is kept in FP32 planes (the
                // padded-HWC buffer holds one chunk); otherwise the first layer's weight
                // gradient reads the padded-HWC gradient directly
                if (rc_chunk) {
                    ProfScope ps(this, s1, "layout_phwc", 6.0 * n * c0.cout * c0.oh * c0.ow, 1);
                    launch_from_phwc(dact_p[0], n, c0.oh, c0.ow, dconv_a + (int64_t)i0 * c0.cout * c0.oh * c0.ow, s1);
                }
            }
            if (rc_chunk)
                for (int l = nconv - 1; l >= 1; --l) {
                    const ConvL& cv = L.conv[l];
                    ProfScope ps(this, s1, "conv_tc_wgrad", 0.0, 0);
                    launch_wgrad32_reduce(wgrad_tc_work + (int64_t)(l - 1) * wgrad32_tc_workspace(B),
                                          (B + pc - 1) / pc, G + cv.wo, G + cv.bo, s1);
                }
            ConvShape sh{B, c0.cin, c0.h, c0.w, c0.cout, c0.s, c0.oh, c0.ow, (int64_t)c0.cin * c0.h * c0.w,
                         (int64_t)c0.cout * c0.oh * c0.ow};
            {
                ProfScope ps(this, s1, "conv_f32_wgrad", conv_flops(c0, B), 0);
                if (rc_chunk) dconv0 = dconv_a;
                if (rc_chunk)
                    launch_conv_wgrad<float>(sh, dconv_a, x2, G + c0.wo, G + c0.bo, wgrad_work, s1);
                else if (launch_conv_wgrad_phwc(sh, dact_p[0], x2, G + c0.wo, G + c0.bo, wgrad_work, s1) != 0)
                    launch_failed = true;
            }
            fork(sw, s1);   // the inner layers' weight gradients before the encoder's Adam
        }
        for (int l = tc_conv ? -1 : nconv - 1; l >= 0; --l) {
            const ConvL& cv = L.conv[l];
            ConvShape sh{B, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                         (int64_t)cv.cout * cv.oh * cv.ow};
            const float* xin = l == 0 ? x2 : conv_out[l - 1];
            if (l == 0) dconv0 = cur;
            {
                ProfScope ps(this, s1, "conv_f32_wgrad", conv_flops(cv, B), 0);
                launch_conv_wgrad<float>(sh, cur, xin, G + cv.wo, G + cv.bo, wgrad_work, s1);
            }
            if (l > 0) {
                float* nxt = (cur == dconv_a) ? dconv_b : dconv_a;
                ProfScope ps(this, s1, "conv_f32_dgrad", conv_flops(cv, B), 0);
                launch_conv_dgrad<float>(sh, cur, W + cv.wo, nxt, conv_out[l - 1], s1);
                cur = nxt;
            }
        }
        adam(0, L.critic_begin, d_steps + 0, nullptr, s1);
        if (tc_conv) {
            ProfScope ps(this, s1, "cast_bf16", 6.0 * 9 * 32 * 32 * (nconv - 1), 1);
            cast_conv_weights(s1);
        }
    }
    // ---- a16 on branch s3: polyak of the updated critics, BF16 target copies (or in the
    // critic Adam's pass)
    fork(s, s3);
    if (!fuse_polyak) {
        PolyakArgs pa{};
        pa.target = target; pa.src = W + L.critic_begin; pa.n = L.target_n; pa.tau = (float)c.tau;
        if (bf16) {   // polyak writes the BF16 copies of the target weights as it updates them
            for (size_t k = 0; k < seg_target.size(); ++k) pa.seg[k] = seg_target[k];
            pa.n_seg = (int)seg_target.size();
        }
        {
            double bf_bytes = 0;
            for (int k = 0; k < pa.n_seg; ++k) bf_bytes += 2.0 * pa.seg[k].rows * pa.seg[k].cols;
            ProfScope ps(this, s3, "polyak", 12.0 * (double)L.target_n + bf_bytes, 1);
            if (launch_polyak(pa, s3) != 0) launch_failed = true;
        }
    }
    quantize_weights(quant_target, s3);
    mark(s);
    // ---- a13 on branch s3: temperature, from log pi of the pre-update actor at s_t; the
    // actor step first reads the new alpha in its head backward (joined there)
    {
        AlphaArgs al{};
        al.B = B; al.logp_t = logp + B;
        al.log_alpha = W + L.log_alpha; al.m = adam_m + L.log_alpha; al.v = adam_v + L.log_alpha;
        al.steps = d_steps;
        al.lr = c.lr; al.b1 = c.adam_b1; al.b2 = c.adam_b2; al.eps = c.adam_eps;
        al.target_entropy = std::isnan(c.target_entropy) ? -(float)A : (float)c.target_entropy;
        al.stats = stats;
        ProfScope ps(this, s3, "heads_losses", 0, 1);
        launch_alpha_step(al, s3);
    }
    mark(s);
    // ---- a14: actor step on stop-gradient features with the updated critics
    {
        if (Dd > 0) {
            const LayerRef cp = layer_ref(this, L.cproj, false);
            {
                GemmBuilder gb(this, s, bf16);
                gb.fwd(zt, B, cp, proj_pre + 4 * (int64_t)B * Dd, Dd);
            }
            LnProblem p{};
            p.rows = B; p.n = Dd;
            p.pre = proj_pre + 4 * (int64_t)B * Dd; p.ld_pre = Dd;
            p.g = cp.g; p.beta = cp.beta;
            p.out = xq; p.ld_out = Dc;
            if (bf16) { p.out_bf = xq_h; p.ld_out_bf = Dc8; }
            p.mean = proj_mean + 4 * B; p.rstd = proj_rstd + 4 * B;
            ln_fwd(&p, 1, false, s);
        } else {
            cast_rows(xq, Dc, B, Dc, xq_h, Dc8, s);
        }
        mlp_forward(this, qcrit_mlp, crit_on, E, Mat{xq, Dc, xq_h, Dc8}, B, bf16, s);
        ActorQArgs aq{};
        aq.B = B; aq.K = K; aq.E = E; aq.logits = qcrit_mlp.out;
        aq.v_min = (float)c.v_min; aq.v_max = (float)c.v_max;
        aq.dlogits = dlogits_q; aq.row_q = row_q_actor; aq.do_actor = d_do_actor;
        aq.cdq = c.cdq; aq.mse = c.critic_kind == 1;
        if (bf16) { aq.dlogits_bf = dlogits_qh; aq.ld_bf = K8; }
        {
            ProfScope ps(this, s, "heads_losses", 0, 1);
            launch_actor_q(aq, s);
        }
        // ---- statistics on branch s3 once the actor objective is known (nothing later in
        // the update reads the update index it advances)
        fork(s, s3);
        if (draw_next) fork(sp, s3);   // the next front end read the index this advances
        {
            StatsArgs st{};
            st.B = B; st.E = E; st.row_loss = row_loss; st.row_q = row_q; st.row_q_actor = row_q_actor;
            st.logp_t = logp + B; st.log_alpha = W + L.log_alpha; st.do_actor = d_do_actor;
            st.update_idx = d_update_idx; st.stats = stats; st.cdq = c.cdq;
            ProfScope ps(this, s3, "heads_losses", 0, 1);
            launch_stats(st, s3);
        }
        // only the action columns of the critics' input gradient are used (the head
        // backward): from column Z + P rounded down to 8 (16-byte aligned BF16 operand)
        const int a0 = (Z + P) / 8 * 8;
        const bool dxq_split = mlp_backward(this, qcrit_mlp, 0, crit_on, nullptr, E, Mat{xq, Dc, xq_h, Dc8}, B,
                                            Mat{dlogits_q, K, dlogits_qh, K8}, Dc - a0, dxq + a0, Dc, nullptr, 0, s, s2,
                                            a0, true, dxq2 + a0);
        fork(s3, s);   // the new alpha (and the statistics) before the head backward
        ActorHeadBwdArgs hb{};
        hb.B = B; hb.A = A;
        hb.out = actor_mlp.out + (int64_t)B * 2 * A; hb.ld_out = 2 * A;
        hb.eps = eps + (int64_t)B * A; hb.da = dxq + Z + P; hb.ld_da = Dc; hb.log_alpha = W + L.log_alpha;
        if (dxq_split) hb.da2 = dxq2 + Z + P;   // the second critic's part, added in the head
        hb.lo = (float)c.log_std_min; hb.hi = (float)c.log_std_max;
        hb.dout = dout_a; hb.do_actor = d_do_actor;
        if (bf16) { hb.dout_bf = dout_ah; hb.ld_dout_bf = pad8(2 * A); }
        {
            ProfScope ps(this, s, "heads_losses", 0, 1);
            launch_actor_head_bwd(hb, s);
        }
        // the actor MLP's weight gradients stay on s2 beside the projection's backward and
        // are joined before the actor Adam
        mlp_backward(this, actor_mlp, B, &actor_on, G, 1, Mat{xa, Da, xa_h, Da8}.rows(B), B,
                     Mat{dout_a, 2 * A, dout_ah, pad8(2 * A)}, Z, Dd > 0 ? dh : nullptr, Z, nullptr, 0, s, s2, 0,
                     false);
        if (Dd > 0) {
            const LayerRef ap = layer_ref(this, L.aproj, false);
            LnBwdProblem p{};
            p.rows = B; p.n = Dd;
            p.dout = dh; p.ld_dout = Dd;
            p.pre = proj_pre + 3 * (int64_t)B * Dd; p.ld_pre = Dd;
            p.mean = proj_mean + 3 * B; p.rstd = proj_rstd + 3 * B;
            p.g = ap.g;
            p.dpre = dproj; p.ld_dpre = Dd;
            if (bf16) { p.dpre_bf = dproj_h; p.ld_dpre_bf = Dd; }
            p.dg = G + L.aproj.g; p.dbeta = G + L.aproj.beta; p.dbias = G + L.aproj.b;
            p.terms = proj_terms;
            ln_bwd(&p, 1, s);
            // the projection's gain, shift and bias gradients beside its weight gradient
            fork(s, s2);
            {
                ProfScope ps(this, s2, "colsum", 12.0 * B * Dd, 1);
                launch_ln_bwd_cols(&p, 1, s2);
            }
            GemmBuilder gb(this, s, bf16);
            gb.dw(Mat{dproj, Dd, dproj_h, Dd}, B, zt, ap, G + L.aproj.w);
        }
        fork(s2, s);
        adam(L.actor_begin, L.actor_end, d_steps + 1, d_do_actor, s, bf16 ? &seg_actor : nullptr);
        quantize_weights(quant_actor, s);
    }
    // join the encoder branch (the polyak / temperature / statistics branch joined above)
    fork(s1, s);
    fork(s3, s);
    mark(s);
    mark(s);
}

void squint_handle::drop_graphs() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    graphs.clear();
    graph_kernels.clear();
}

void squint_handle::cast_conv_weights(cudaStream_t s) {
    if (!tc_conv) return;
    for (size_t l = 1; l < L.conv.size(); ++l)
        launch_conv_weight_cast(params + L.conv[l].wo, wconv_fwd[l], wconv_bwd[l], s);
}

int squint_handle::run_updates(int k, squint_update_stats* stats, cudaStream_t s, bool use_graph) {
    launch_failed = false;
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
            for (int j = 0; j < k; ++j) record_update(j, k, capture_stream, false);
            SQ_CK(this, cudaStreamEndCapture(capture_stream, &graph));
            if (launch_failed) {
                cudaGraphDestroy(graph);
                g_last_error = "a tensor-core operand could not be described by a tensor map";
                return SQUINT_EINVAL;
            }
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
            SQ_CK(this, cudaGraphInstantiateWithFlags(&exec, graph,
                                                      prio_branches ? cudaGraphInstantiateFlagUseNodePriority : 0));
            cudaGraphDestroy(graph);
            it = graphs.emplace(k, exec).first;
        }
        SQ_CK(this, cudaGraphLaunch(it->second, s));
        use_set((k - 1) & 1);   // the debug views show the last update's buffers
    } else {
        for (int j = 0; j < k; ++j) record_update(j, k, s, true);
        SQ_CK(this, cudaGetLastError());
        if (launch_failed) {
            g_last_error = "a tensor-core operand could not be described by a tensor map";
            return SQUINT_EINVAL;
        }
    }
    if (stats) {
        int32_t err = 0;
        SQ_CK(this, cudaMemcpyAsync(h_stats, d_stats, sizeof(float) * 8 * k, cudaMemcpyDeviceToHost, s));
        SQ_CK(this, cudaMemcpyAsync(&err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SQ_CK(this, cudaStreamSynchronize(s));
        if (err) {
            failed = true;
            g_last_error = "a bounded device wait ran out";
            return SQUINT_ETIMEOUT;
        }
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

// Phase names, in the order their boundaries are marked in record_update.
static const char* kPhaseNames[] = {
    "frontend",          // a1-a4
    "encoder_fwd",       // a5
    "projections",       // a6 (then the online critic forward starts on a side branch)
    "actor_fwd",         // a7
    "target_critics",    // a8-a9
    "critic_ce",         // a10 (waits for the critic forward)
    "critic_bwd",        // a11 critics and projection (weight gradients on a side branch)
    "adam_polyak_fork",  // a12 critic range; encoder backward and polyak start on side branches
    "alpha_step",        // a13
    "actor_step",        // a14-a15, then waits for the encoder backward and polyak
    "stats",             // statistics, update index
};

const char* sq::phase_name(int i) {
    return (i >= 0 && i < (int)(sizeof(kPhaseNames) / sizeof(kPhaseNames[0]))) ? kPhaseNames[i] : nullptr;
}

int squint_handle::profile_update(float* ms, int cap, int* n_phases, cudaStream_t s) {
    // captured (with its phase events) and replayed, like the timed graph
    std::vector<cudaEvent_t> ev;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SQ_CK(this, cudaStreamSynchronize(s));
    SQ_CK(this, cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
    phase_events = &ev;
    record_update(0, 1, capture_stream, false);
    phase_events = nullptr;
    SQ_CK(this, cudaStreamEndCapture(capture_stream, &graph));
    int rc = launch_failed ? SQUINT_EINVAL : SQUINT_OK;
    if (rc == SQUINT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = SQUINT_ECUDA;
    if (rc == SQUINT_OK && cudaGraphLaunch(exec, s) != cudaSuccess) rc = SQUINT_ECUDA;
    if (rc == SQUINT_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = SQUINT_ECUDA;
    const int n = (int)ev.size() - 1;
    if (n_phases) *n_phases = n;
    for (int i = 0; rc == SQUINT_OK && i < n && i < cap; ++i) {
        if (cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]) != cudaSuccess) rc = SQUINT_ECUDA;
    }
    for (auto e : ev) cudaEventDestroy(e);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (rc != SQUINT_OK) { failed = true; g_last_error = "profiling failed"; }
    return rc;
}

// One update with every launch in order on one stream, each bracketed by its own
// events, captured as a graph and replayed (so the host's launch cost does not show up
// as device time); launches are grouped by kernel class.  The replay is one real update.
int squint_handle::replay_profiled(std::vector<ProfEntry>& recs, bool in_order, cudaEvent_t base, cudaStream_t s) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    SQ_CK(this, cudaStreamSynchronize(s));
    SQ_CK(this, cudaStreamBeginCapture(capture_stream, cudaStreamCaptureModeThreadLocal));
    if (base) record_timing(base, capture_stream);
    prof = &recs;
    serial = in_order;
    record_update(0, 1, capture_stream, false);
    serial = false;
    prof = nullptr;
    SQ_CK(this, cudaStreamEndCapture(capture_stream, &graph));
    int rc = launch_failed ? SQUINT_EINVAL : SQUINT_OK;
    if (rc == SQUINT_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = SQUINT_ECUDA;
    if (rc == SQUINT_OK && cudaGraphLaunch(exec, s) != cudaSuccess) rc = SQUINT_ECUDA;
    if (rc == SQUINT_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = SQUINT_ECUDA;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    return rc;
}

// One update as the timed graph runs it (concurrent branches), with an event pair around
// every launch: each launch's start and end relative to the update's start, and its branch.
int squint_handle::trace_update(int cap, char* names, int* lanes, float* t0, float* t1, int* n, cudaStream_t s) {
    std::vector<ProfEntry> recs;
    cudaEvent_t base = nullptr;
    SQ_CK(this, cudaEventCreate(&base));
    int rc = replay_profiled(recs, false, base, s);
    for (size_t i = 0; i < recs.size(); ++i) {
        const ProfEntry& e = recs[i];
        float a = 0.f, b = 0.f;
        if (rc == SQUINT_OK && (cudaEventElapsedTime(&a, base, e.a) != cudaSuccess ||
                                cudaEventElapsedTime(&b, base, e.b) != cudaSuccess))
            rc = SQUINT_ECUDA;
        if (rc == SQUINT_OK && (int)i < cap) {
            std::snprintf(names + 32 * i, 32, "%s", e.name);
            lanes[i] = e.lane;
            t0[i] = a;
            t1[i] = b;
        }
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    cudaEventDestroy(base);
    if (rc != SQUINT_OK) { failed = true; g_last_error = "update trace failed"; return rc; }
    *n = (int)recs.size();
    return SQUINT_OK;
}

int squint_handle::profile_kernels(int cap, char* names, int* launches, float* ms, double* work, int* unit, int* n,
                                   cudaStream_t s) {
    std::vector<ProfEntry> recs;
    int rc = replay_profiled(recs, true, nullptr, s);
    std::vector<std::string> order;
    std::map<std::string, std::tuple<int, double, double, int>> agg;
    for (auto& e : recs) {
        float t = 0.f;
        if (rc == SQUINT_OK && cudaEventElapsedTime(&t, e.a, e.b) != cudaSuccess) rc = SQUINT_ECUDA;
        auto it = agg.find(e.name);
        if (it == agg.end()) {
            order.push_back(e.name);
            agg[e.name] = std::make_tuple(1, (double)t, e.work, e.unit);
        } else {
            std::get<0>(it->second) += 1;
            std::get<1>(it->second) += t;
            std::get<2>(it->second) += e.work;
        }
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    if (rc != SQUINT_OK) { failed = true; g_last_error = "kernel profiling failed"; return rc; }
    *n = (int)order.size();
    for (int i = 0; i < (int)order.size() && i < cap; ++i) {
        const auto& v = agg[order[i]];
        std::snprintf(names + 32 * i, 32, "%s", order[i].c_str());
        launches[i] = std::get<0>(v);
        ms[i] = (float)std::get<1>(v);
        work[i] = std::get<2>(v);
        unit[i] = std::get<3>(v);
    }
    return SQUINT_OK;
}
