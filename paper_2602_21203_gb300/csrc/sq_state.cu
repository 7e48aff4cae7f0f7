// Learner state transfer, debug views, policy snapshots and batched inference.
#include "sq_sched.h"

#include <cstring>

using namespace sq;

namespace {
constexpr uint32_t kStateMagic = 0x54535153u;  // "SQST"
}  // namespace

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
    const int B = c.batch, A = c.action_dim, K = c.critic_kind == 1 ? 1 : c.atoms;
    const int64_t img = (int64_t)L.img_c * L.hs * L.ws;
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
    else if (n == "dxq") { src = dxq; sz = 4 * (size_t)B * L.dc; }
    else if (n == "a_pi") { src = nullptr; sz = 4 * (size_t)B * A; }
    else if (n == "grads") { src = grads; sz = 4 * (size_t)L.total; }
    else if (n == "z_t") { src = conv_out.empty() ? nullptr : conv_out.back(); sz = 4 * (size_t)B * L.feat; }
    else if (n == "target") { src = target; sz = 4 * (size_t)L.target_n; }
    else if (n == "dconv0" && !L.conv.empty()) {
        // gradient at the first conv's pre-activation (after the ReLU mask), FP32 planes
        src = dconv0; sz = 4 * (size_t)B * L.conv[0].cout * L.conv[0].oh * L.conv[0].ow;
        if (!src) { g_last_error = "dconv0: this learner keeps that gradient in padded HWC (dconv0_phwc)"; return SQUINT_EINVAL; }
    } else if (n == "dconv0_phwc" && tc_conv && !rc_chunk) {
        // the same as BF16 padded HWC: per image (oh + 4) x (ow + 4) pixels of 32 channels,
        // pixel (y, x) at row (y + 2) (ow + 4) + x + 2
        src = dact_p[0]; sz = 2 * (size_t)B * (L.conv[0].oh + 4) * (L.conv[0].ow + 4) * 32;
    } else if (n.size() == 5 && n.compare(0, 4, "conv") == 0 && n[4] >= '0' && n[4] < '0' + (int)L.conv.size() &&
               conv_out[n[4] - '0']) {
        // conv layer l's output (after ReLU) for the o_t images, FP32 planes
        const ConvL& cv = L.conv[n[4] - '0'];
        src = conv_out[n[4] - '0']; sz = 4 * (size_t)B * cv.cout * cv.oh * cv.ow;
    }
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
    if (sz) SQ_CK(this, cudaMemcpy(host, src, sz, cudaMemcpyDeviceToHost));
    return SQUINT_OK;
}

int squint_handle::refresh_policy(cudaStream_t s) {
    std::lock_guard<std::mutex> lk(act_mu);
    // write the snapshot inference is not using, after inference that last read it
    const int i = 1 - policy_active;
    for (sq::ActArena* a : arenas)
        if (a->released[i]) SQ_CK(this, cudaStreamWaitEvent(s, a->released[i], 0));
    SQ_CK(this, cudaMemcpyAsync(policy_buf[i], params, L.total * sizeof(float), cudaMemcpyDeviceToDevice, s));
    snapshot_bf16(i, s);
    SQ_CK(this, cudaEventRecord(policy_ready[i], s));
    policy_active = i;
    ++policy_version;
    return SQUINT_OK;
}

// ---------------------------------------------------------------- inference
size_t squint_handle::act_row_bytes() const {
    size_t f = (size_t)L.img_c * L.hs * L.ws;
    for (const auto& cv : L.conv) f += (size_t)cv.cout * cv.oh * cv.ow;
    f += (size_t)L.D + 2 + L.da;
    for (int l = 0; l < c.n_hidden; ++l) f += 2 * (size_t)c.hidden[l] + 2;
    f += 2 * (size_t)c.action_dim;
    return f * sizeof(float) + 8;
}

void squint_handle::free_arena(sq::ActArena& a) {
    if (a.req_event_live) cudaEventSynchronize(a.req_event);
    for (int i = 0; i < 2; ++i)
        if (a.released[i]) cudaEventSynchronize(a.released[i]);
    for (void* p : a.allocs) if (p) cudaFree(p);
    a.allocs.clear();
    if (a.h_req) cudaFreeHost(a.h_req);
    a.h_req = nullptr;
    if (a.req_event) cudaEventDestroy(a.req_event);
    a.req_event = nullptr;
    for (int i = 0; i < 2; ++i) {
        if (a.released[i]) cudaEventDestroy(a.released[i]);
        a.released[i] = nullptr;
    }
    a.cap = a.rcap = 0;
    a.bytes = 0;
    a.req_event_live = false;
}

int squint_handle::alloc_arena(sq::ActArena& a, int rows, int n_reqs) {
    if (rows <= a.cap && n_reqs <= a.rcap) return SQUINT_OK;
    const int cap = std::max(((std::max(rows, a.cap) + 255) / 256) * 256, 256);
    const int rcap = std::max(std::max(n_reqs, a.rcap), 64);
    free_arena(a);
    auto al = [&](size_t bytes) -> void* {
        void* p = nullptr;
        bytes = std::max<size_t>(bytes, 16);
        if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        a.allocs.push_back(p);
        a.bytes += bytes;
        return p;
    };
    const int64_t img = (int64_t)L.img_c * L.hs * L.ws;
    a.ax = (float*)al(sizeof(float) * cap * img);
    a.aconv.clear();
    for (const auto& cv : L.conv) a.aconv.push_back((float*)al(sizeof(float) * (size_t)cap * cv.cout * cv.oh * cv.ow));
    if (L.D > 0) {
        a.apre = (float*)al(sizeof(float) * (size_t)cap * L.D);
        a.amean = (float*)al(sizeof(float) * cap);
        a.arstd = (float*)al(sizeof(float) * cap);
    }
    a.axin = (float*)al(sizeof(float) * (size_t)cap * L.da);
    const int nh = c.n_hidden;
    a.mlp = MlpBufs{};
    a.mlp.E = 1; a.mlp.rows = cap;
    a.mlp.pre.resize(nh); a.mlp.post.resize(nh); a.mlp.mean.resize(nh); a.mlp.rstd.resize(nh);
    for (int l = 0; l < nh; ++l) {
        a.mlp.pre[l] = (float*)al(sizeof(float) * (size_t)cap * c.hidden[l]);
        a.mlp.post[l] = (float*)al(sizeof(float) * (size_t)cap * c.hidden[l]);
        a.mlp.mean[l] = (float*)al(sizeof(float) * cap);
        a.mlp.rstd[l] = (float*)al(sizeof(float) * cap);
    }
    a.mlp.out = (float*)al(sizeof(float) * (size_t)cap * 2 * c.action_dim);
    a.aphwc.clear();
    a.mlp.posth.clear();
    a.az_h = a.axin_h = nullptr;
    if (bf16) {
        // BF16 inference buffers; padded borders and pad columns stay zero
        if (tc_conv)
            for (size_t l = 0; l + 1 < L.conv.size(); ++l) {
                const size_t bytes = 2 * (size_t)cap * (L.conv[l].oh + 4) * (L.conv[l].ow + 4) * 32;
                a.aphwc.push_back((__nv_bfloat16*)al(bytes));
                if (a.aphwc.back()) SQ_CK(this, cudaMemset(a.aphwc.back(), 0, bytes));
            }
        a.az_h = (__nv_bfloat16*)al(2 * (size_t)cap * L.feat);
        const size_t xb = 2 * (size_t)cap * ((L.da + 7) / 8 * 8);
        a.axin_h = (__nv_bfloat16*)al(xb);
        if (a.axin_h) SQ_CK(this, cudaMemset(a.axin_h, 0, xb));
        for (int l = 0; l < nh; ++l) a.mlp.posth.push_back((__nv_bfloat16*)al(2 * (size_t)cap * c.hidden[l]));
    }
    a.req_bytes = (size_t)cap * 8 + (size_t)rcap * (8 * 4 + 4) + 64;
    a.d_req = al(a.req_bytes);
    for (void* p : a.allocs)
        if (!p) { g_last_error = "inference allocation failed"; free_arena(a); return SQUINT_ENOMEM; }
    if (cudaMallocHost(&a.h_req, a.req_bytes) != cudaSuccess) { free_arena(a); return SQUINT_ENOMEM; }
    SQ_CK(this, cudaEventCreateWithFlags(&a.req_event, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) SQ_CK(this, cudaEventCreateWithFlags(&a.released[i], cudaEventDisableTiming));
    SQ_CK(this, cudaDeviceSynchronize());   // the zeroed borders before any batch
    a.cap = cap;
    a.rcap = rcap;
    return SQUINT_OK;
}

int squint_handle::act(sq::ActArena& a, const squint_act_request* reqs, int n_reqs, cudaStream_t s,
                       int64_t* version_used) {
    std::lock_guard<std::mutex> lk(act_mu);
    int rows = 0;
    for (int q = 0; q < n_reqs; ++q) {
        const squint_act_request& rq = reqs[q];
        if (rq.n < 1 || (!rq.obs && !L.conv.empty()) || !rq.proprio || !rq.actions || (rq.mode != 0 && rq.mode != 1)) {
            g_last_error = "invalid inference request";
            return SQUINT_EINVAL;
        }
        rows += rq.n;
    }
    if (rows == 0) return SQUINT_OK;
    int rc = alloc_arena(a, rows, n_reqs);
    if (rc != SQUINT_OK) return rc;
    if (a.req_event_live) SQ_CK(this, cudaEventSynchronize(a.req_event));
    const int act_cap = a.cap, req_cap = a.rcap;
    float* ax = a.ax; float* apre = a.apre; float* amean = a.amean; float* arstd = a.arstd; float* axin = a.axin;
    const std::vector<float*>& aconv = a.aconv;
    const std::vector<__nv_bfloat16*>& aphwc = a.aphwc;
    __nv_bfloat16* az_h = a.az_h; __nv_bfloat16* axin_h = a.axin_h;
    // pack: row_req[cap] row_in[cap] | obs[rcap] prop[rcap] act[rcap] key[rcap] (8 B each) | mode[rcap]
    uint8_t* hb = static_cast<uint8_t*>(a.h_req);
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
    SQ_CK(this, cudaMemcpyAsync(a.d_req, a.h_req, a.req_bytes, cudaMemcpyHostToDevice, s));
    SQ_CK(this, cudaEventRecord(a.req_event, s));
    a.req_event_live = true;
    uint8_t* db = static_cast<uint8_t*>(a.d_req);
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
    if (L.conv.empty()) { af.C = 0; af.H = af.W = af.f = 1; }   // state-based: no image
    af.x = ax; af.xin = axin; af.ld_xin = Da; af.col = L.zdim;
    launch_act_frontend(af, s);
    // BF16 policy: layer-0 conv on CUDA cores, the 32-channel convs and every linear
    // layer on tcgen05 with the snapshot's BF16 copies, no K split (each row's result
    // is independent of the other rows of the batch)
    const bool tc = bf16 && tc_conv;
    const float* in = ax;
    for (size_t l = 0; l < L.conv.size(); ++l) {
        const ConvL& cv = L.conv[l];
        if (tc && l > 0) {
            ConvTc ct{};
            ct.in = aphwc[l - 1];
            ct.nimg = rows;
            ct.Wp = cv.w + 4;
            ct.in_rows = (cv.h + 4) * ct.Wp;
            ct.out_h = cv.oh; ct.out_w = cv.ow;
            ct.off0 = 2 * ct.Wp + 2;
            ct.w = policy_wconv[pi] + (l - 1) * 9 * 32 * 32;
            ct.bias = Wp + cv.bo;
            ct.relu = 1;
            if (l + 1 < L.conv.size()) ct.out_phwc = aphwc[l];
            else { ct.out_chw = aconv[l]; ct.out_chw_bf = az_h; }
            if (launch_conv32_tc(ct, d_err, s) != 0) { g_last_error = "tensor-core conv launch"; return SQUINT_ECUDA; }
            in = aconv[l];
            continue;
        }
        ConvShape sh{rows, cv.cin, cv.h, cv.w, cv.cout, cv.s, cv.oh, cv.ow, (int64_t)cv.cin * cv.h * cv.w,
                     (int64_t)cv.cout * cv.oh * cv.ow};
        if (tc && l == 0) {   // first layer straight into the padded-HWC input of the tensor-core layers
            if (launch_conv0_tc(sh, in, Wp + cv.wo, Wp + cv.bo, aphwc[0], d_err, s) < 0)
                launch_conv0_phwc(sh, in, Wp + cv.wo, Wp + cv.bo, aphwc[0], s);
            continue;
        }
        launch_conv_fwd<float>(sh, in, Wp + cv.wo, Wp + cv.bo, aconv[l], true, s);
        in = aconv[l];
    }
    if (bf16 && !tc && F > 0) {
        CastItem ci{in, F, rows, F, az_h, F};
        launch_cast_rows(&ci, 1, s);
    }
    auto bf_ref = [&](const Lin& ly) {
        LayerRef r = layer_ref(this, ly, false, Wp);
        if (bf16) {
            const auto& o = policy_bf_off.at(ly.w);
            r.wh = policy_bf[pi] + o.first;
            r.ldh = o.second;
        }
        return r;
    };
    if (Dd > 0) {
        if (bf16) {
            GemmBuilder gb(this, s, true, false);
            gb.fwd(Mat{const_cast<float*>(in), F, az_h, F}, rows, bf_ref(L.aproj), apre, Dd);
        } else {
            GemmProblem g = lin_fwd(in, F, rows, Wp + L.aproj.w, Wp + L.aproj.b, F, Dd, apre, Dd);
            launch_gemm<float>(&g, 1, kKK, s);
        }
        LnProblem p{};
        p.rows = rows; p.n = Dd; p.pre = apre; p.ld_pre = Dd;
        p.g = Wp + L.aproj.g; p.beta = Wp + L.aproj.beta;
        p.out = axin; p.ld_out = Da; p.mean = amean; p.rstd = arstd;
        launch_ln_fwd(&p, 1, false, (float)c.ln_eps, s);
    } else if (F > 0) {
        SQ_CK(this, cudaMemcpy2DAsync(axin, Da * sizeof(float), in, F * sizeof(float), F * sizeof(float), rows,
                                      cudaMemcpyDeviceToDevice, s));
    }
    const int64_t Da8 = (Da + 7) / 8 * 8;
    if (bf16) {
        CastItem ci{axin, Da, rows, Da, axin_h, Da8};   // projected features and proprio, BF16
        launch_cast_rows(&ci, 1, s);
    }
    MlpRef actor_ref;
    for (const auto& ly : L.actor) actor_ref.push_back(bf_ref(ly));
    mlp_forward(this, a.mlp, &actor_ref, 1, Mat{axin, Da, axin_h, Da8}, rows, bf16, s, false, false);
    ActHeadArgs ha{};
    ha.rows = rows; ha.A = A; ha.out = a.mlp.out; ha.ld_out = 2 * A;
    ha.row_req = d_row_req; ha.row_in_req = d_row_in;
    ha.req_key = d64 + 3 * req_cap; ha.req_mode = d_modes;
    ha.req_actions = reinterpret_cast<float* const*>(d64 + 2 * req_cap);
    ha.lo = (float)c.log_std_min; ha.hi = (float)c.log_std_max; ha.seed = c.seed;
    launch_act_head(ha, s);
    SQ_CK(this, cudaEventRecord(a.released[pi], s));
    SQ_CK(this, cudaGetLastError());
    return SQUINT_OK;
}

