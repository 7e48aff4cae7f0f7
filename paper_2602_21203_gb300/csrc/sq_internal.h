// Internal definition of the learner handle.
#pragma once

#include "squint.h"
#include "sq_kernels.cuh"
#include "sq_tc.cuh"
#include "sq_mlp_tc.cuh"

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace sq {

extern thread_local std::string g_last_error;
void set_error(const char* fmt, const char* a, const char* b, int line);

#define SQ_CK(h, call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            ::sq::set_error("%s: %s (line %d)", #call, cudaGetErrorString(e_), __LINE__);      \
            (h)->failed = true;                                                                 \
            return SQUINT_ECUDA;                                                                \
        }                                                                                       \
    } while (0)

struct Lin { int64_t w = -1, b = -1, g = -1, beta = -1; int in = 0, out = 0; bool ln = false; };
struct ConvL { int cin, cout, h, w, oh, ow, s; int64_t wo, bo; };

// Canonical flat parameter layout (offsets in floats).
struct Layout {
    int hs = 0, ws = 0;
    int img_c = 0;                        // channels of the training image (0: state-based, no image)
    std::vector<ConvL> conv;
    int feat = 0, D = 0, zdim = 0, dc = 0, da = 0;
    Lin cproj, aproj;
    std::vector<Lin> critic[2];
    std::vector<Lin> actor;
    int64_t critic_begin = 0, critic_end = 0, actor_begin = 0, actor_end = 0, log_alpha = 0, total = 0, target_n = 0;
};

bool build_layout(const squint_config& c, Layout& L);
const char* phase_name(int i);
void init_params_host(const squint_config& c, const Layout& L, std::vector<float>& p);

// Activations of one MLP evaluated on `rows` rows by E parameter sets.
struct MlpBufs {
    int E = 0, rows = 0;
    std::vector<float*> pre, post, mean, rstd;   // per hidden layer: [E, rows, n]
    std::vector<__nv_bfloat16*> posth;           // BF16 shadows of post (tensor-core path)
    float* out = nullptr;                        // [E, rows, n_out]
    std::vector<float*> lnterms;                 // per hidden layer: [E][2][rows, n] deferred
                                                 // LayerNorm column-sum terms (backward with weights)
    bool tc_saved = false;                       // the saves were written by the fused forward kernel
};

// BF16 padded copy of one linear layer's weight (online and, for the critic range, target).
struct LinBf { __nv_bfloat16* on = nullptr; __nv_bfloat16* tg = nullptr; int64_t ld = 0; };

// Activation buffers of one inference batch: the one squint_act uses, or a serving
// slot's (several batches in flight each need their own).
struct ActArena {
    int cap = 0, rcap = 0;                 // rows and requests the buffers hold
    float* ax = nullptr;
    std::vector<float*> aconv;
    float* apre = nullptr; float* amean = nullptr; float* arstd = nullptr;
    float* axin = nullptr;
    MlpBufs mlp;
    std::vector<__nv_bfloat16*> aphwc;     // BF16 inference: padded-HWC conv outputs (l < L-1)
    __nv_bfloat16* az_h = nullptr;         // BF16 inference: encoder features [cap, F]
    __nv_bfloat16* axin_h = nullptr;       // BF16 inference: actor input [cap, pad8(Da)]
    void* d_req = nullptr;                 // packed per-request arrays
    void* h_req = nullptr;                 // pinned staging
    size_t req_bytes = 0;
    cudaEvent_t req_event = nullptr;       // the staging's upload finished
    bool req_event_live = false;
    cudaEvent_t released[2] = {nullptr, nullptr};   // this arena's last batch finished reading policy buffer i
    std::vector<void*> allocs;
    size_t bytes = 0;                      // device bytes held
};

struct ServeState;

}  // namespace sq

struct squint_handle {
    squint_config c{};
    sq::Layout L;
    squint_replay ring{};
    bool has_ring = false;
    bool failed = false;
    bool bf16 = false;                // tensor-core contractions (SQUINT_PREC_BF16 or FP8)
    bool fp8 = false;                 // forward linear layers in e4m3 (SQUINT_PREC_FP8 or MXFP8)
    bool mx = false;                  // ... with MX block scales (SQUINT_PREC_MXFP8)
    // hidden-layer LayerNorm in the GEMM epilogue (tensor-core path), chosen by
    // SQUINT_FUSED_LN=1 in the environment at creation; off by default: at batch 512 the
    // separate LayerNorm kernel gives more updates/s (1,310 vs 1,264 on the same GPU)
    bool fuse_ln = false;
    // K split over clusters in the update's GEMMs, chosen by SQUINT_GEMM_SPLIT=1; off by
    // default: inside the concurrent update graph it gave 1,307 updates/s against 1,321
    // without (clusters wait for co-scheduled SMs while the side streams hold some)
    bool gemm_split = false;
    // in a call of k updates, each update's minibatch drawn (front end) while the previous
    // update runs; SQUINT_DRAW_AHEAD=0 at creation draws every one in line instead
    bool draw_ahead = true;
    // head MLP chains of the BF16 learner as one fused tensor-core launch each
    // (SQUINT_MLP_FUSED=0 at creation: a GEMM and a LayerNorm launch per layer instead);
    // SQUINT_MLP_CL=1/2/4/8 forces the cluster size of the fused launches.  Backward chains
    // without weight gradients (the actor step's, through the critics) run as one fused
    // launch; those with weight gradients as GEMMs beside LayerNorm-backward launches, which
    // measure faster inside the update's concurrent graph (the clusters of a fused launch
    // wait for free SMs beside the encoder backward).  SQUINT_MLP_BWD at creation: 0 no
    // fused chain, 1 every chain, 2 the default, 3 chains of one parameter set;
    // SQUINT_MLP_BWD_CL: the fused chain's cluster size
    bool mlp_fused = true;
    int mlp_cluster = 0;
    int mlp_fused_sites = 15;   // SQUINT_MLP_SITES: which forward chains are fused (bit mask)
    // cluster size per chain (bit order of the mask; 0: the launcher's choice, 4 for 512-wide
    // heads): the actor's and the target critics' chains on the main stream take 8 (more
    // SMs for their latency-bound layers; the online critics beside them and the actor
    // step's critics beside the encoder backward keep 4, which co-schedule more easily)
    int mlp_cluster_site[4] = {0, 8, 8, 0};
    int mlp_bwd_fused = 2;
    int mlp_bwd_cluster = 0;
    // the actor step's chain through the two critics ends with each critic's input
    // gradient in the same fused launch (two buffers, added by the head backward) instead
    // of a GEMM over both, from a batch of two row blocks on (SQUINT_MLP_FIN_SPLIT=0 at
    // creation: the GEMM at every batch)
    bool mlp_fin_split = true;
    // the actor's forward as two launches (the target's half on the critical chain without
    // saves, the o_t half with its saves on a side branch) on the fused BF16 path
    // (SQUINT_SPLIT_ACTOR_FWD=0 at creation: one launch over both halves)
    bool split_actor_fwd = true;
    // branch priorities (SQUINT_PRIO=0 at creation: every stream at the default priority)
    bool prio_branches = true;
    // the polyak of the target critics inside the critic Adam's pass (SQUINT_FUSE_POLYAK=0
    // at creation: its own launch beside the actor step)
    bool fuse_polyak = true;
    bool launch_failed = false;       // a tensor map could not describe an operand
    // bounded waits of the update's tensor-core GEMMs (cycles 0: the default limit) and
    // the failure-test switch that makes them run out (squint_set_debug)
    sq::TcWait gemm_wait{0, 0};
    void drop_graphs();
    int device = 0;
    int* d_err = nullptr;             // device error word of bounded waits

    // parameters and optimiser state
    float* params = nullptr;
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* target = nullptr;
    float* policy_buf[2] = {nullptr, nullptr};   // inference snapshots (same layout as params)
    // BF16 inference: per snapshot, padded BF16 copies of the actor-path matrices (actor
    // projection and actor MLP; weight offset -> element offset in policy_bf, row stride)
    // and the tensor-core filter layouts of conv layers 1.. (9 x 32 x 32 each)
    __nv_bfloat16* policy_bf[2] = {nullptr, nullptr};
    __nv_bfloat16* policy_wconv[2] = {nullptr, nullptr};
    __nv_bfloat16* policy_wconv_scratch = nullptr;    // unused data-gradient layout output
    std::map<int64_t, std::pair<int64_t, int64_t>> policy_bf_off;
    std::vector<sq::CastItem> cast_policy[2];
    void snapshot_bf16(int i, cudaStream_t s);
    int policy_active = 0;
    int64_t policy_version = 0;
    cudaEvent_t policy_ready[2] = {nullptr, nullptr};     // copy into buffer i finished
    int64_t* d_update_idx = nullptr;
    int32_t* d_steps = nullptr;       // critic, actor, alpha
    int32_t* d_do_actor = nullptr;
    float* d_stats = nullptr;         // [max_k, 8]
    float* h_stats = nullptr;         // pinned

    // update activations
    float* x2 = nullptr;              // [2B, C, Hs, Ws]
    uint16_t* sums = nullptr;         // [2B, C, Hs, Ws]
    int32_t* idx2 = nullptr;          // [2B]
    int32_t* shift2 = nullptr;        // [2B, 2]
    std::vector<float*> conv_out;     // [2B, ch, oh, ow]
    float* proj_pre = nullptr;        // [5, B, D]: ap(z'), cbar(z'), cp(z), ap(z), cp_new(z)
    float* proj_mean = nullptr;       // [5, B]
    float* proj_rstd = nullptr;
    float* xa = nullptr;              // [2B, Da]
    float* xcbar = nullptr;           // [B, Dc]
    float* xc = nullptr;              // [B, Dc]
    float* xq = nullptr;              // [B, Dc]
    // The front end's outputs of one update (squinted images, r, d and the head inputs
    // it writes the transition fields into).  Update j of a call uses set j % 2, so the
    // front end of update j + 1 can run while update j still reads its own set; use_set
    // points the members above and below at a set.
    struct FeSet {
        float* x2 = nullptr; float* r = nullptr; float* d = nullptr;
        float* xa = nullptr; float* xcbar = nullptr; float* xc = nullptr; float* xq = nullptr;
        __nv_bfloat16* xa_h = nullptr; __nv_bfloat16* xcbar_h = nullptr;
        __nv_bfloat16* xc_h = nullptr; __nv_bfloat16* xq_h = nullptr;
    };
    FeSet fe_set[2];
    void use_set(int i) {
        const FeSet& f = fe_set[i];
        x2 = f.x2; r = f.r; d = f.d; xa = f.xa; xcbar = f.xcbar; xc = f.xc; xq = f.xq;
        xa_h = f.xa_h; xcbar_h = f.xcbar_h; xc_h = f.xc_h; xq_h = f.xq_h;
    }
    sq::MlpBufs actor_mlp, tcrit_mlp, crit_mlp, qcrit_mlp;
    float* logp = nullptr;            // [2B]
    float* eps = nullptr;             // [2B, A]
    float* m = nullptr;               // [B, K]
    float* r = nullptr;
    float* d = nullptr;
    float* dlogits = nullptr;         // [E, B, K]
    float* dlogits_q = nullptr;       // [E, B, K]
    float* row_loss = nullptr;        // [E B]
    float* row_q = nullptr;           // [E B]
    float* row_q_actor = nullptr;     // [E B]
    std::vector<float*> dpost, dpre;  // per hidden layer [E, B, n] (critic bwd; reused by actor bwd)
    float* dh = nullptr;              // [B, zdim]
    float* dproj = nullptr;           // [B, D]
    float* dz = nullptr;              // [B, F] (masked: gradient at the last conv's pre-activation)
    float* dconv_a = nullptr;         // ping-pong conv gradients
    float* dconv_b = nullptr;
    float* wgrad_work = nullptr;
    // FP32 gradient at the first conv's pre-activation [B, ch, oh, ow] as the last update
    // left it (the buffer the first layer's weight gradient read; FP32-plane paths only)
    const float* dconv0 = nullptr;
    float* dxq = nullptr;             // [B, Dc] input gradient of the critics in the actor step
    float* dxq2 = nullptr;            // [B, Dc] the second critic's part of it, when kept apart
    float* ln_work = nullptr;         // LayerNorm backward column partials
    // fused head backward: per hidden layer [2][row blocks][3][H] column sums of each 128-row
    // block (LayerNorm gain, shift and bias gradients once the row blocks are added)
    std::vector<float*> mlp_colpart;
    float* dout_a = nullptr;          // [B, 2A]

    // BF16 shadows (tensor-core path)
    std::map<int64_t, sq::LinBf> lin_bf;       // keyed by the canonical weight offset
    // FP8 mode: e4m3 copies of the linear weights (quantised from the BF16 copies after
    // every cast) and, per stream, an arena for the forward GEMMs' quantised activations
    struct LinF8 { uint8_t* on = nullptr; uint8_t* tg = nullptr; int64_t ld = 0; float* s_on = nullptr;
                   float* s_tg = nullptr; uint8_t* sf_on = nullptr; uint8_t* sf_tg = nullptr; };
    std::map<int64_t, LinF8> lin_f8;
    std::vector<sq::QuantItem> quant_critic, quant_actor, quant_target;
    float* f8_part = nullptr;             // amax partials of the weight quantisation
    struct F8Arena { uint8_t* buf = nullptr; int64_t bytes = 0; float* part = nullptr; float* scales = nullptr; };
    F8Arena f8_arena[4];                  // main stream, side streams 0..2
    F8Arena* arena_for(cudaStream_t s) {
        for (int k = 0; k < 3; ++k)
            if (s == side[k]) return &f8_arena[k + 1];
        return &f8_arena[0];
    }
    void quantize_weights(const std::vector<sq::QuantItem>& q, cudaStream_t s);
    std::vector<sq::CastItem> cast_critic, cast_actor, cast_target;
    // the same BF16 copies as segments of the critic / actor / target ranges, written by
    // Adam and polyak in the update (the casts above serve full refreshes)
    std::vector<sq::BfSeg> seg_critic, seg_actor, seg_target;
    float* proj_terms = nullptr;               // [2][B, D] deferred LayerNorm column-sum terms
    __nv_bfloat16* z_h = nullptr;              // [2B, F]
    __nv_bfloat16* xa_h = nullptr;             // [2B, Da8]
    __nv_bfloat16* xcbar_h = nullptr;          // [B, Dc8]
    __nv_bfloat16* xc_h = nullptr;
    __nv_bfloat16* xq_h = nullptr;
    __nv_bfloat16* dlogits_h = nullptr;        // [E, B, K8]
    __nv_bfloat16* dlogits_qh = nullptr;
    std::vector<__nv_bfloat16*> dpre_h;        // per hidden layer [E, B, n]
    __nv_bfloat16* dproj_h = nullptr;          // [B, D]
    __nv_bfloat16* dout_ah = nullptr;          // [B, 16]
    // tensor-core convolutions (BF16 mode, inner layers 32 -> 32, stride 1)
    bool tc_conv = false;
    std::vector<__nv_bfloat16*> act_p;         // [l]: padded-HWC output of conv l (2B images), l < L-1
    std::vector<__nv_bfloat16*> dact_p;        // [l]: padded-HWC gradient at conv l's pre-activation (B images)
    __nv_bfloat16* dz_p = nullptr;             // padded-HWC gradient at the last conv's pre-activation
    std::vector<__nv_bfloat16*> wconv_fwd, wconv_bwd;   // [l]: BF16 filter layouts (l >= 1)
    float* wgrad_tc_work = nullptr;

    // inference: the arena squint_act uses, and every arena that may read a policy buffer
    // (this one and the serving slots'), guarded by act_mu
    sq::ActArena arena;
    std::vector<sq::ActArena*> arenas;
    cudaStream_t capture_stream = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
    std::map<int, int64_t> graph_kernels;
    // concurrent branches of one update: library-owned streams joined back before it ends
    // (side[4]: the next update's front end, drawn while this update runs)
    cudaStream_t side[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t fork_ev[32] = {};
    int fork_next = 0;
    bool serial = false;                  // profiling: every launch in order on the main stream
    struct ProfEntry { const char* name; cudaEvent_t a, b; double work; int unit; int lane; };
    std::vector<ProfEntry>* prof = nullptr;   // per-launch records while profiling kernels
    // stream of branch i (the main stream itself when serial)
    cudaStream_t branch(cudaStream_t main, int i) const { return serial ? main : side[i]; }
    // make `to` wait for the work issued so far on `from`
    void fork(cudaStream_t from, cudaStream_t to) {
        if (from == to) return;
        cudaEvent_t e = fork_ev[fork_next++ % 32];
        cudaEventRecord(e, from);
        cudaStreamWaitEvent(to, e, 0);
    }
    int profile_kernels(int cap, char* names, int* launches, float* ms, double* work, int* unit, int* n,
                        cudaStream_t s);
    int trace_update(int cap, char* names, int* lanes, float* t0, float* t1, int* n, cudaStream_t s);
    // one update captured with an event pair around every launch and replayed
    int replay_profiled(std::vector<ProfEntry>& recs, bool in_order, cudaEvent_t base, cudaStream_t s);
    // the branch a stream is: 0 the main stream, i + 1 side[i]
    int lane_of(cudaStream_t st) const {
        for (int i = 0; i < 5; ++i)
            if (side[i] && st == side[i]) return i + 1;
        return 0;
    }
    std::vector<cudaEvent_t>* phase_events = nullptr;   // set while profiling an eager update
    // timing event on `s`; under stream capture it becomes an event-record node of the graph
    static void record_timing(cudaEvent_t e, cudaStream_t s) {
        cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(s, &st);
        if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
        else cudaEventRecord(e, s);
    }
    void mark(cudaStream_t s) {
        if (phase_events) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            record_timing(e, s);
            phase_events->push_back(e);
        }
    }
    int profile_update(float* ms, int cap, int* n_phases, cudaStream_t s);

    std::vector<void*> allocations;
    int64_t device_bytes = 0;             // sum of the dalloc sizes
    int rc_chunk = 0;                     // encoder recompute chunk (images), 0 = off
    std::shared_ptr<sq::ServeState> serve;   // guarded by serve_mu
    std::mutex serve_mu;
    std::mutex act_mu;

    int allocate();
    void release();
    int after_param_change();
    int run_updates(int k, squint_update_stats* stats, cudaStream_t s, bool use_graph);
    // update j of k recorded on s (its front end drawn by update j - 1 when j > 0; it
    // draws update j + 1's when j + 1 < k)
    void record_update(int j, int k, cudaStream_t s, bool debug);
    void cast_conv_weights(cudaStream_t s);
    size_t state_bytes() const;
    int save_state(uint8_t* out);
    int load_state(const uint8_t* in);
    int debug_tensor(const char* name, void* host, size_t* bytes);
    int refresh_policy(cudaStream_t s);
    // (re)allocate an arena for `rows` rows and `n_reqs` requests (caller holds act_mu)
    int alloc_arena(sq::ActArena& a, int rows, int n_reqs);
    void free_arena(sq::ActArena& a);
    size_t act_row_bytes() const;
    // one ragged inference batch with arena a on stream s
    int act(sq::ActArena& a, const squint_act_request* reqs, int n_reqs, cudaStream_t s,
            int64_t* version_used = nullptr);

    // Device allocation; a failure is recorded as a null entry that allocate() reports.
    template <typename T> T* dalloc(int64_t n) {
        void* p = nullptr;
        if (n <= 0) n = 1;
        if (cudaMalloc(&p, (size_t)n * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        allocations.push_back(p);
        if (p) device_bytes += (int64_t)((size_t)n * sizeof(T));
        return static_cast<T*>(p);
    }
};
