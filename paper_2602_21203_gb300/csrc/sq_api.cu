// C ABI of the Squint learner: handle, parameter layout, the launch schedule of
// one SAC update (Algorithm 1, inner loop), CUDA-graph capture of k updates,
// state transfer and batched actor inference.
#include "squint.h"
#include "sq_internal.h"

#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <string>

namespace sq {

thread_local std::string g_last_error;

void set_error(const char* fmt, const char* a, const char* b, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), fmt, a, b, line);
    g_last_error = buf;
}

// ---------------------------------------------------------------- layout
static int64_t add_lin(Layout& L, int64_t off, Lin& l, int in, int out, bool ln) {
    l.in = in;
    l.out = out;
    l.ln = ln;
    l.w = off; off += (int64_t)in * out;
    l.b = off; off += out;
    if (ln) { l.g = off; off += out; l.beta = off; off += out; }
    else { l.g = l.beta = -1; }
    (void)L;
    return off;
}

bool build_layout(const squint_config& c, Layout& L) {
    // conv_layers == 0: state-based SAC (Sec. VII, Fig. 6 left), no image and no encoder;
    // the heads read the state vector (proprio_dim wide) and the observation fields are unused
    const bool state_based = c.conv_layers == 0;
    if (state_based) {
        if (c.proj_dim != 0 || c.proprio_dim < 1) return false;
    } else {
        if (c.obs_c < 1 || c.obs_h < 1 || c.obs_w < 1 || c.squint_f < 1) return false;
        if (c.obs_h % c.squint_f || c.obs_w % c.squint_f) return false;
        if (c.conv_layers < 1 || c.conv_layers > SQUINT_MAX_CONV || c.conv_ch < 1) return false;
    }
    if (c.n_hidden < 1 || c.n_hidden > SQUINT_MAX_HIDDEN || c.n_critics != 2) return false;
    if (c.atoms < 2 || c.atoms > 256 || c.action_dim < 1 || c.proprio_dim < 0 || c.proj_dim < 0) return false;
    if (c.critic_kind < 0 || c.critic_kind > 1 || c.cdq < 0 || c.cdq > 1) return false;
    if (c.batch < 1 || c.policy_freq < 1 || c.shift_pad < 0) return false;
    if (!(c.v_max > c.v_min)) return false;
    L = Layout{};
    int cin = state_based ? 0 : c.obs_c, h = state_based ? 0 : c.obs_h / c.squint_f,
        w = state_based ? 0 : c.obs_w / c.squint_f;
    L.hs = h;
    L.ws = w;
    L.img_c = cin;
    int64_t off = 0;
    for (int l = 0; l < c.conv_layers; ++l) {
        ConvL cv;
        cv.cin = cin; cv.cout = c.conv_ch; cv.h = h; cv.w = w;
        cv.s = c.conv_stride[l] > 0 ? c.conv_stride[l] : (l == 0 ? 2 : 1);
        cv.oh = (h - 3) / cv.s + 1;
        cv.ow = (w - 3) / cv.s + 1;
        if (h < 3 || w < 3 || cv.oh < 1 || cv.ow < 1) return false;
        cv.wo = off; off += (int64_t)cv.cout * cin * 9;
        cv.bo = off; off += cv.cout;
        L.conv.push_back(cv);
        cin = cv.cout; h = cv.oh; w = cv.ow;
    }
    L.feat = cin * h * w;
    L.D = c.proj_dim;
    L.zdim = L.D > 0 ? L.D : L.feat;
    L.dc = L.zdim + c.proprio_dim + c.action_dim;
    L.da = L.zdim + c.proprio_dim;
    L.critic_begin = off;                 // critic projection starts the target range
    if (L.D > 0) off = add_lin(L, off, L.cproj, L.feat, L.D, true);
    for (int e = 0; e < 2; ++e) {
        int in = L.dc;
        L.critic[e].resize(c.n_hidden + 1);
        for (int l = 0; l < c.n_hidden; ++l) { off = add_lin(L, off, L.critic[e][l], in, c.hidden[l], true); in = c.hidden[l]; }
        off = add_lin(L, off, L.critic[e][c.n_hidden], in, c.critic_kind == 1 ? 1 : c.atoms, false);
    }
    L.critic_end = off;
    L.actor_begin = off;
    if (L.D > 0) off = add_lin(L, off, L.aproj, L.feat, L.D, true);
    {
        int in = L.da;
        L.actor.resize(c.n_hidden + 1);
        for (int l = 0; l < c.n_hidden; ++l) { off = add_lin(L, off, L.actor[l], in, c.hidden[l], true); in = c.hidden[l]; }
        off = add_lin(L, off, L.actor[c.n_hidden], in, 2 * c.action_dim, false);
    }
    L.actor_end = off;
    L.log_alpha = off; off += 1;
    L.total = off;
    L.target_n = L.critic_end - L.critic_begin;
    return true;
}

// Uniform(+-1/sqrt(fan_in)) for weights and biases, 1 / 0 for LayerNorm, log(alpha0);
// element e of the t-th tensor (canonical order) draws block (e, init stream, t).
void init_params_host(const squint_config& c, const Layout& L, std::vector<float>& p) {
    p.assign(L.total, 0.f);
    int t = 0;
    auto uni = [&](int64_t off, int64_t n, int fan) {
        const double bound = 1.0 / std::sqrt((double)fan);
        for (int64_t e = 0; e < n; ++e) {
            uint32_t w[4];
            draw_block(w, c.seed, (uint32_t)e, kStreamInit, 0, (uint64_t)t);
            const double u = ((double)(w[0] >> 9) + 0.5) * (1.0 / 8388608.0);
            p[off + e] = (float)((2.0 * u - 1.0) * bound);
        }
        ++t;
    };
    auto fill = [&](int64_t off, int64_t n, float v) { for (int64_t e = 0; e < n; ++e) p[off + e] = v; ++t; };
    auto lin = [&](const Lin& l) {
        uni(l.w, (int64_t)l.in * l.out, l.in);
        uni(l.b, l.out, l.in);
        if (l.ln) { fill(l.g, l.out, 1.f); fill(l.beta, l.out, 0.f); }
    };
    for (const auto& cv : L.conv) { uni(cv.wo, (int64_t)cv.cout * cv.cin * 9, cv.cin * 9); uni(cv.bo, cv.cout, cv.cin * 9); }
    if (L.D > 0) lin(L.cproj);
    for (int e = 0; e < 2; ++e) for (const auto& l : L.critic[e]) lin(l);
    if (L.D > 0) lin(L.aproj);
    for (const auto& l : L.actor) lin(l);
    p[L.log_alpha] = (float)std::log(c.init_alpha);
}

}  // namespace sq

using namespace sq;

// ================================================================ C ABI
extern "C" {

const char* squint_strerror(int code) {
    switch (code) {
        case SQUINT_OK: return "ok";
        case SQUINT_EINVAL: return "invalid argument";
        case SQUINT_ENOMEM: return "out of device memory or over budget";
        case SQUINT_ECUDA: return "CUDA error";
        case SQUINT_ETIMEOUT: return "timed out";
        case SQUINT_EAGAIN: return "not ready";
        case SQUINT_ESTATE: return "invalid state";
        default: return "unknown error";
    }
}

const char* squint_last_error(void) { return g_last_error.c_str(); }

size_t squint_struct_size(const char* name) {
    if (!name) return 0;
    const std::string n(name);
    if (n == "squint_config") return sizeof(squint_config);
    if (n == "squint_replay") return sizeof(squint_replay);
    if (n == "squint_update_stats") return sizeof(squint_update_stats);
    if (n == "squint_act_request") return sizeof(squint_act_request);
    if (n == "squint_serve_result") return sizeof(squint_serve_result);
    return 0;
}

int squint_config_preset(const char* name, squint_config* c) {
    if (!name || !c) return SQUINT_EINVAL;
    std::memset(c, 0, sizeof(*c));
    c->obs_c = 3; c->proprio_dim = 12; c->action_dim = 6; c->n_critics = 2;
    c->n_hidden = 2; c->policy_freq = 1; c->precision = SQUINT_PREC_FP32; c->max_k = 8;
    c->gamma = 0.99; c->lr = 3e-4; c->tau = 0.005; c->init_alpha = 0.1; c->target_entropy = NAN;
    c->ln_eps = 1e-5; c->log_std_min = -5.0; c->log_std_max = 2.0;
    c->adam_b1 = 0.9; c->adam_b2 = 0.999; c->adam_eps = 1e-8; c->seed = 0;
    const std::string n(name);
    if (n == "small_b32") {
        c->obs_h = c->obs_w = 64; c->squint_f = 4; c->shift_pad = 4; c->batch = 32;
        c->conv_layers = 2; c->conv_ch = 16; c->proj_dim = 0; c->hidden[0] = c->hidden[1] = 256;
        c->atoms = 51; c->v_min = -10; c->v_max = 10;
    } else if (n == "train_b512") {
        c->obs_h = c->obs_w = 128; c->squint_f = 4; c->shift_pad = 8; c->batch = 512;
        c->conv_layers = 4; c->conv_ch = 32; c->proj_dim = 256; c->hidden[0] = c->hidden[1] = 512;
        c->atoms = 101; c->v_min = -20; c->v_max = 20;
    } else if (n == "tiny_b8") {
        c->obs_h = c->obs_w = 64; c->squint_f = 4; c->shift_pad = 4; c->batch = 8;
        c->conv_layers = 2; c->conv_ch = 8; c->proj_dim = 0; c->hidden[0] = c->hidden[1] = 32;
        c->atoms = 11; c->v_min = -10; c->v_max = 10;
    } else {
        g_last_error = "unknown preset";
        return SQUINT_EINVAL;
    }
    c->conv_stride[0] = 2;
    for (int l = 1; l < SQUINT_MAX_CONV; ++l) c->conv_stride[l] = 1;
    return SQUINT_OK;
}

int64_t squint_param_count(const squint_config* c) {
    Layout L;
    if (!c || !build_layout(*c, L)) return -1;
    return L.total;
}

int squint_create(const squint_config* cfg, const squint_replay* ring, squint_handle** out) {
    if (!cfg || !out) return SQUINT_EINVAL;
    *out = nullptr;
    auto* h = new (std::nothrow) squint_handle();
    if (!h) return SQUINT_ENOMEM;
    h->c = *cfg;
    if (!build_layout(h->c, h->L)) {
        g_last_error = "invalid configuration";
        delete h;
        return SQUINT_EINVAL;
    }
    if (h->c.max_k < 1) h->c.max_k = 8;
    if (h->c.precision != SQUINT_PREC_FP32 && h->c.precision != SQUINT_PREC_BF16 &&
        h->c.precision != SQUINT_PREC_FP8 && h->c.precision != SQUINT_PREC_MXFP8) {
        delete h;
        return SQUINT_EINVAL;
    }
    int rc = h->allocate();
    if (rc == SQUINT_OK && ring) rc = squint_set_replay(h, ring);
    if (rc != SQUINT_OK) {
        h->release();
        delete h;
        return rc;
    }
    *out = h;
    return SQUINT_OK;
}

int squint_set_replay(squint_handle* h, const squint_replay* ring) {
    if (!h || !ring) return SQUINT_EINVAL;
    if (ring->n < 2 || ring->n > 0xFFFFFFFFll || (!ring->obs && !h->L.conv.empty()) || !ring->proprio ||
        !ring->action || !ring->reward || !ring->done)
        return SQUINT_EINVAL;
    const squint_replay& o = h->ring;
    const bool same = h->has_ring && o.obs == ring->obs && o.proprio == ring->proprio && o.action == ring->action &&
                      o.reward == ring->reward && o.done == ring->done && o.n == ring->n;
    if (!same && !h->graphs.empty()) {
        // captured updates hold the old ring's addresses and size: the next update of
        // each k captures again
        SQ_CK(h, cudaDeviceSynchronize());
        h->drop_graphs();
    }
    h->ring = *ring;
    h->has_ring = true;
    return SQUINT_OK;
}

int squint_set_debug(squint_handle* h, const char* name, int64_t value) {
    if (!h || !name) return SQUINT_EINVAL;
    const std::string n(name);
    sq::TcWait w = h->gemm_wait;
    if (n == "wait_cycles" && value >= 0) w.cycles = value;
    else if (n == "stall_gemm_loads" && (value == 0 || value == 1)) w.stall = (int)value;
    else { sq::g_last_error = "unknown debug setting or value"; return SQUINT_EINVAL; }
    if (w.cycles != h->gemm_wait.cycles || w.stall != h->gemm_wait.stall) {
        SQ_CK(h, cudaDeviceSynchronize());
        h->drop_graphs();   // captured updates hold the old settings
    }
    h->gemm_wait = w;
    return SQUINT_OK;
}

int squint_destroy(squint_handle* h) {
    if (!h) return SQUINT_OK;
    squint_serve_stop(h);
    h->release();
    delete h;
    return SQUINT_OK;
}

int squint_update(squint_handle* h, int k, squint_update_stats* stats, void* stream) {
    if (!h) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (!h->has_ring) return SQUINT_ESTATE;
    if (k < 1 || k > h->c.max_k) return SQUINT_EINVAL;
    return h->run_updates(k, stats, (cudaStream_t)stream, true);
}

int squint_update_eager(squint_handle* h, int k, squint_update_stats* stats, void* stream) {
    if (!h) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (!h->has_ring) return SQUINT_ESTATE;
    if (k < 1 || k > h->c.max_k) return SQUINT_EINVAL;
    return h->run_updates(k, stats, (cudaStream_t)stream, false);
}

// The device statistics (8 words an update: six floats, the update index as two 32-bit
// halves, low first) are the bytes of squint_update_stats on a little-endian host.
static_assert(sizeof(squint_update_stats) == 32 && offsetof(squint_update_stats, update_idx) == 24,
              "squint_update_stats must match the device statistics layout");

int squint_update_async(squint_handle* h, int k, squint_update_stats* stats, void* stream) {
    if (!h) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (!h->has_ring) return SQUINT_ESTATE;
    if (k < 1 || k > h->c.max_k) return SQUINT_EINVAL;
    if (stats) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, stats) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();
            g_last_error = "squint_update_async: stats must be page-locked host memory";
            return SQUINT_EINVAL;
        }
    }
    const cudaStream_t s = (cudaStream_t)stream;
    const int rc = h->run_updates(k, nullptr, s, true);
    if (rc != SQUINT_OK || !stats) return rc;
    SQ_CK(h, cudaMemcpyAsync(stats, h->d_stats, sizeof(squint_update_stats) * k, cudaMemcpyDeviceToHost, s));
    return SQUINT_OK;
}

int squint_update_check(squint_handle* h, void* stream) {
    if (!h) return SQUINT_EINVAL;
    int32_t err = 0;
    SQ_CK(h, cudaMemcpyAsync(&err, h->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    SQ_CK(h, cudaStreamSynchronize((cudaStream_t)stream));
    if (err) {
        h->failed = true;
        g_last_error = "a bounded device wait ran out";
        return SQUINT_ETIMEOUT;
    }
    return h->failed ? SQUINT_ESTATE : SQUINT_OK;
}

int squint_get_params(squint_handle* h, float* host, int64_t n) {
    if (!h || !host || n != h->L.total) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    SQ_CK(h, cudaDeviceSynchronize());
    SQ_CK(h, cudaMemcpy(host, h->params, n * sizeof(float), cudaMemcpyDeviceToHost));
    return SQUINT_OK;
}

int squint_set_params(squint_handle* h, const float* host, int64_t n) {
    if (!h || !host || n != h->L.total) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    SQ_CK(h, cudaDeviceSynchronize());
    SQ_CK(h, cudaMemcpy(h->params, host, n * sizeof(float), cudaMemcpyHostToDevice));
    // targets copy the critics again, moments restart
    SQ_CK(h, cudaMemcpy(h->target, h->params + h->L.critic_begin, h->L.target_n * sizeof(float),
                        cudaMemcpyDeviceToDevice));
    SQ_CK(h, cudaMemset(h->adam_m, 0, n * sizeof(float)));
    SQ_CK(h, cudaMemset(h->adam_v, 0, n * sizeof(float)));
    return h->after_param_change();
}

int squint_get_state(squint_handle* h, void* host, size_t* bytes) {
    if (!h || !bytes) return SQUINT_EINVAL;
    const size_t need = h->state_bytes();
    if (!host) { *bytes = need; return SQUINT_OK; }
    if (*bytes < need) { *bytes = need; return SQUINT_EINVAL; }
    if (h->failed) return SQUINT_ESTATE;
    *bytes = need;
    return h->save_state(static_cast<uint8_t*>(host));
}

int squint_set_state(squint_handle* h, const void* host, size_t bytes) {
    if (!h || !host || bytes != h->state_bytes()) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    return h->load_state(static_cast<const uint8_t*>(host));
}

int squint_debug_tensor(squint_handle* h, const char* name, void* host, size_t* bytes) {
    if (!h || !name || !bytes) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    return h->debug_tensor(name, host, bytes);
}

int64_t squint_device_bytes(squint_handle* h) { return h ? h->device_bytes : 0; }

int64_t squint_graph_kernel_count(squint_handle* h, int k) {
    if (!h) return 0;
    auto it = h->graph_kernels.find(k);
    return it == h->graph_kernels.end() ? 0 : it->second;
}

int squint_profile_update(squint_handle* h, float* ms, int cap, int* n_phases, void* stream) {
    if (!h || !ms || cap < 0) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (!h->has_ring) return SQUINT_ESTATE;
    return h->profile_update(ms, cap, n_phases, (cudaStream_t)stream);
}

const char* squint_phase_name(int i) { return sq::phase_name(i); }

int squint_trace_update(squint_handle* h, int cap, char* names, int* lanes, float* t0, float* t1, int* n, void* stream) {
    if (!h || cap < 0 || !names || !lanes || !t0 || !t1 || !n) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (!h->has_ring) return SQUINT_ESTATE;
    return h->trace_update(cap, names, lanes, t0, t1, n, (cudaStream_t)stream);
}

int squint_profile_kernels(squint_handle* h, int cap, char* names, int* launches, float* ms, double* work, int* unit,
                           int* n, void* stream) {
    if (!h || cap < 0 || !names || !launches || !ms || !work || !unit || !n) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    if (!h->has_ring) return SQUINT_ESTATE;
    return h->profile_kernels(cap, names, launches, ms, work, unit, n, (cudaStream_t)stream);
}

int squint_refresh_policy(squint_handle* h, void* stream) {
    if (!h) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    return h->refresh_policy((cudaStream_t)stream);
}

int squint_act(squint_handle* h, const squint_act_request* reqs, int n_reqs, void* stream) {
    if (!h || (!reqs && n_reqs > 0) || n_reqs < 0) return SQUINT_EINVAL;
    if (h->failed) return SQUINT_ESTATE;
    return h->act(h->arena, reqs, n_reqs, (cudaStream_t)stream);
}

}  // extern "C"
