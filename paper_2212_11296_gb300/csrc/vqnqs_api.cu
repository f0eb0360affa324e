// C ABI of libvqnqs: context, workspace plan and the per-chunk pipeline of the
// local-energy path (Sec. 2 Eq. local-energy evaluated with the VQ-NQS of
// Sec. 3.1, reusing per-location work by (row, code) keys as in Sec. 3.2).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vqnqs_internal.cuh"

using namespace vq;

struct vqnqs_ctx {
    int L = 0, N = 0, periodic = 0, layers = 0, d = 0, heads = 0, K = 0, nb = 0;
    double J = 1.0;
    int device = 0, num_sms = 0;
    size_t nparams = 0;
    float* blob = nullptr;  // device copy of the weight blob
    const float *tok_emb = nullptr, *pos_emb = nullptr, *lnf_g = nullptr, *lnf_b = nullptr, *w_head = nullptr,
                *b_head = nullptr;
    std::vector<LayerW> lw;
    int* bonds = nullptr;          // [nb][2]
    int* status = nullptr;         // device status word
    long long* stats = nullptr;    // ST_* slots
    std::vector<void*> owned;      // device allocations freed by destroy
    std::string err;
    // stage timing (vqnqs_profile_*) and launch counting
    bool prof = false;
    std::vector<cudaEvent_t> ev_free;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    long long st_calls[VQNQS_MAX_STAGES] = {}, st_launches[VQNQS_MAX_STAGES] = {};
    double st_ms[VQNQS_MAX_STAGES] = {};
    long long launches = 0;
};

namespace {

int fail(vqnqs_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define VQ_CK(call)                                                                                       \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess)                                                                            \
            return fail(ctx, VQNQS_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

enum Stage { S_CONFIG, S_EMBED, S_LN1, S_QKV, S_ATTN, S_VQ, S_DEDUPE, S_POSTLN, S_MLP1, S_MLP2, S_HEAD, S_ELOC,
             S_MEANVAR, S_COUNT };
const char* kStageNames[S_COUNT] = {"config", "embed", "ln1", "qkv_gemm", "attention", "vq_argmin", "dedupe",
                                    "post_ln", "mlp_up", "mlp_down", "head", "eloc", "mean_var"};

cudaEvent_t take_event(vqnqs_ctx* c) {
    if (c->ev_free.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
}

// Brackets one stage: counts its launches and, when profiling, records events.
struct StageScope {
    vqnqs_ctx* c;
    int stage, nl;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    StageScope(vqnqs_ctx* c_, int stage_, int nl_, cudaStream_t st_) : c(c_), stage(stage_), nl(nl_), st(st_) {
        if (c->prof && (a = take_event(c))) cudaEventRecord(a, st);
    }
    ~StageScope() {
        c->launches += nl;
        c->st_calls[stage] += 1;
        c->st_launches[stage] += nl;
        if (a) {
            cudaEvent_t b = take_event(c);
            if (b) {
                cudaEventRecord(b, st);
                c->pending.push_back({stage, a, b});
            } else {
                c->ev_free.push_back(a);
            }
        }
    }
};

#define VQ_STAGE(id, nl, call)                  \
    do {                                        \
        StageScope scope_(ctx, (id), (nl), st); \
        VQ_CK(call);                            \
    } while (0)

std::vector<int> make_bonds(int L, int periodic) {
    std::vector<int> b;
    for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x) {
            int p = y * L + x;
            if (x + 1 < L || periodic) { b.push_back(p); b.push_back(y * L + (x + 1) % L); }
            if (y + 1 < L || periodic) { b.push_back(p); b.push_back(((y + 1) % L) * L + x); }
        }
    return b;
}

struct Plan {
    int S = 0;
    long long Cmax = 0, Rmax = 0, Umax = 0;
    int hash_bits = 0;
    size_t counters, cnt, cfg_off, diag, cfg_sample, cfg_i, cfg_j, uid_a, uid_b, code, X_a, X_b, A, Y, scratch,
        keys, vals, rep_uid, rep_code, logp, ratio, total;
};

Plan make_plan(const vqnqs_ctx* c, int S, bool with_bonds) {
    Plan p;
    p.S = S;
    p.Cmax = (long long)S * (with_bonds ? (1 + c->nb) : 1);
    p.Rmax = p.Cmax * c->N;
    p.Umax = p.Rmax > 3LL * c->N ? p.Rmax : 3LL * c->N;
    int hb = 1;
    while ((1LL << hb) < 2 * p.Rmax) ++hb;
    p.hash_bits = hb;
    const size_t d = c->d;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    p.counters = take(CNT_SLOTS * sizeof(int));
    p.cnt = take((size_t)S * sizeof(int));
    p.cfg_off = take((size_t)(S + 1) * sizeof(int));
    p.diag = take((size_t)S * sizeof(float));
    p.cfg_sample = take((size_t)p.Cmax * sizeof(int));
    p.cfg_i = take((size_t)p.Cmax * sizeof(int));
    p.cfg_j = take((size_t)p.Cmax * sizeof(int));
    p.uid_a = take((size_t)p.Rmax * sizeof(int));
    p.uid_b = take((size_t)p.Rmax * sizeof(int));
    p.code = take((size_t)p.Rmax * sizeof(int));
    p.X_a = take((size_t)p.Umax * d * sizeof(float));
    p.X_b = take((size_t)p.Umax * d * sizeof(float));
    p.A = take((size_t)p.Umax * d * sizeof(float));
    p.Y = take((size_t)p.Umax * d * sizeof(float));
    size_t attn = (size_t)p.Umax * 3 * d * sizeof(float) + align256((size_t)p.Rmax * d * sizeof(float));
    size_t mlp = (size_t)p.Umax * 4 * d * sizeof(float);
    p.scratch = take(attn > mlp ? attn : mlp);
    p.keys = take(((size_t)1 << hb) * sizeof(unsigned long long));
    p.vals = take(((size_t)1 << hb) * sizeof(int));
    p.rep_uid = take((size_t)p.Umax * sizeof(int));
    p.rep_code = take((size_t)p.Umax * sizeof(int));
    p.logp = take((size_t)p.Umax * 2 * sizeof(float));
    p.ratio = take((size_t)p.Cmax * sizeof(float));
    p.total = o;
    return p;
}

int default_chunk(const vqnqs_ctx* c, bool with_bonds) {
    // aim for about 2M token rows per chunk in the worst case
    long long per = (long long)(with_bonds ? (1 + c->nb) : 1) * c->N;
    long long s = (2LL << 20) / per;
    if (s < 1) s = 1;
    if (s > 65536) s = 65536;
    return (int)s;
}

// Largest chunk whose plan fits in ws_bytes (0 if even one sample does not).
int fit_chunk(const vqnqs_ctx* c, int B, size_t ws_bytes, bool with_bonds) {
    int hi = B < 65536 ? B : 65536;
    if (make_plan(c, 1, with_bonds).total > ws_bytes) return 0;
    int lo = 1;
    while (lo < hi) {
        int mid = lo + (hi - lo + 1) / 2;
        if (make_plan(c, mid, with_bonds).total <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

int grid_for(const vqnqs_ctx* c, long long items, int per_block, int per_sm) {
    long long g = (items + per_block - 1) / per_block;
    long long cap = (long long)c->num_sms * per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

template <typename T>
T* at(void* ws, size_t off) { return reinterpret_cast<T*>(static_cast<char*>(ws) + off); }

int build_tables(vqnqs_ctx* ctx, cudaStream_t st) {
    const int d = ctx->d, K = ctx->K;
    for (int l = 0; l < ctx->layers; ++l) {
        LayerW& w = ctx->lw[l];
        VQ_CK(launch_table_T(w.codebook, w.w_o, w.b_o, K, d, w.T, w.cnorm, st));
        VQ_CK(launch_transpose_bf16(w.w_qkv, d, 3 * d, w.wqkv_t, st));
        VQ_CK(launch_transpose_bf16(w.w_1, d, 4 * d, w.w1_t, st));
        VQ_CK(launch_transpose_bf16(w.w_2, 4 * d, d, w.w2_t, st));
    }
    return VQNQS_OK;
}

void bind_weights(vqnqs_ctx* c) {
    const size_t d = c->d, K = c->K;
    const float* p = c->blob;
    auto take = [&](size_t n) { const float* r = p; p += n; return r; };
    c->tok_emb = take(3 * d);
    c->pos_emb = take((size_t)c->N * d);
    for (int l = 0; l < c->layers; ++l) {
        LayerW& w = c->lw[l];
        w.ln1_g = take(d); w.ln1_b = take(d);
        w.w_qkv = take(d * 3 * d); w.b_qkv = take(3 * d);
        w.codebook = take(K * d);
        w.w_o = take(d * d); w.b_o = take(d);
        w.ln2_g = take(d); w.ln2_b = take(d);
        w.w_1 = take(d * 4 * d); w.b_1 = take(4 * d);
        w.w_2 = take(4 * d * d); w.b_2 = take(d);
    }
    c->lnf_g = take(d); c->lnf_b = take(d);
    c->w_head = take(2 * d); c->b_head = take(2);
}

// One chunk of samples through the whole path.
int run_chunk(vqnqs_ctx* ctx, const Plan& P, void* ws, const uint8_t* spins, int S, bool with_bonds, int flags,
              float* e_loc_out, float* log_psi_out, cudaStream_t st) {
    const int N = ctx->N, d = ctx->d, K = ctx->K;
    const bool reuse = (flags & VQNQS_REUSE) != 0;
    int* counters = at<int>(ws, P.counters);
    Chunk ch;
    ch.spins = spins; ch.S = S; ch.N = N; ch.L = ctx->L; ch.d = d; ch.heads = ctx->heads; ch.K = K;
    ch.cfg_sample = at<int>(ws, P.cfg_sample);
    ch.cfg_i = at<int>(ws, P.cfg_i);
    ch.cfg_j = at<int>(ws, P.cfg_j);
    ch.cfg_off = at<int>(ws, P.cfg_off);
    ch.counters = counters;
    float* diag = at<float>(ws, P.diag);
    const int g_s = grid_for(ctx, S, 1, 8);
    {
        StageScope scope_(ctx, S_CONFIG, 3, st);
        VQ_CK(launch_count_configs(spins, S, N, ctx->bonds, ctx->nb, (float)ctx->J, with_bonds, at<int>(ws, P.cnt),
                                   diag, ctx->status, st, g_s));
        VQ_CK(launch_scan_configs(at<int>(ws, P.cnt), S, at<int>(ws, P.cfg_off), counters, N, st));
        VQ_CK(launch_fill_configs(spins, S, N, ctx->bonds, ctx->nb, with_bonds, ch.cfg_off, at<int>(ws, P.cfg_sample),
                                  at<int>(ws, P.cfg_i), at<int>(ws, P.cfg_j), st, g_s));
    }

    int* uid_cur = at<int>(ws, P.uid_a);
    int* uid_next = at<int>(ws, P.uid_b);
    float* X_cur = at<float>(ws, P.X_a);
    float* X_next = at<float>(ws, P.X_b);
    float* A = at<float>(ws, P.A);
    float* Y = at<float>(ws, P.Y);
    float* qkv = at<float>(ws, P.scratch);
    float* O = at<float>(ws, P.scratch + align256((size_t)P.Umax * 3 * d * sizeof(float)));
    float* Hid = at<float>(ws, P.scratch);
    int* code = at<int>(ws, P.code);
    int* rep_uid = at<int>(ws, P.rep_uid);
    int* rep_code = at<int>(ws, P.rep_code);
    const int Umax = (int)P.Umax, Rmax = (int)P.Rmax;
    const int g_rows = grid_for(ctx, P.Rmax, 8, 16);
    const int g_urows = grid_for(ctx, P.Umax, 8, 16);

    VQ_STAGE(S_EMBED, reuse ? 2 : 1, launch_embed(ch, ctx->tok_emb, ctx->pos_emb, reuse, X_cur, uid_cur, st, g_rows));
    for (int l = 0; l < ctx->layers; ++l) {
        const LayerW& w = ctx->lw[l];
        const int us = CNT_U0 + l, un = CNT_U0 + l + 1;
        VQ_STAGE(S_LN1, 1, launch_layernorm(X_cur, counters, us, w.ln1_g, w.ln1_b, d, A, nullptr, st, g_urows));
        VQ_STAGE(S_QKV, 1, launch_sgemm(A, w.w_qkv, w.b_qkv, nullptr, qkv, counters, us, Umax, 3 * d, d, EPI_BIAS, st,
                                        ctx->num_sms));
        VQ_STAGE(S_ATTN, 1, launch_attention_f32(ch, uid_cur, qkv, O, st, grid_for(ctx, P.Cmax * ctx->heads, 1, 8)));
        VQ_STAGE(S_VQ, 1, launch_vq_argmin(O, counters, w.codebook, w.cnorm, K, d, code, ctx->stats + ST_NEAR_TIES,
                                           Rmax, st, ctx->num_sms));
        VQ_STAGE(S_DEDUPE, reuse ? 3 : 1,
                 launch_dedupe(uid_cur, code, counters, un, Rmax, at<unsigned long long>(ws, P.keys),
                               at<int>(ws, P.vals), P.hash_bits, uid_next, rep_uid, rep_code, reuse, ctx->status, st,
                               ctx->num_sms));
        VQ_STAGE(S_POSTLN, 1, launch_residual_vq_ln(X_cur, rep_uid, rep_code, w.T, counters, un, w.ln2_g, w.ln2_b, d,
                                                    Y, A, nullptr, st, g_urows));
        VQ_STAGE(S_MLP1, 1, launch_sgemm(A, w.w_1, w.b_1, nullptr, Hid, counters, un, Umax, 4 * d, d, EPI_BIAS_GELU,
                                         st, ctx->num_sms));
        VQ_STAGE(S_MLP2, 1, launch_sgemm(Hid, w.w_2, w.b_2, Y, X_next, counters, un, Umax, d, 4 * d, EPI_BIAS_RESID,
                                         st, ctx->num_sms));
        std::swap(uid_cur, uid_next);
        std::swap(X_cur, X_next);
    }
    float* logp = at<float>(ws, P.logp);
    VQ_STAGE(S_HEAD, 1, launch_head(X_cur, counters, CNT_U0 + ctx->layers, ctx->lnf_g, ctx->lnf_b, ctx->w_head,
                                    ctx->b_head, d, logp, st, g_urows));
    float* ratio = at<float>(ws, P.ratio);
    {
        StageScope scope_(ctx, S_ELOC, e_loc_out ? 2 : 1, st);
        VQ_CK(launch_eloc(ch, uid_cur, logp, ratio, log_psi_out, st, grid_for(ctx, P.Cmax, 8, 16)));
        if (e_loc_out)
            VQ_CK(launch_eloc_reduce(ch, diag, ratio, (float)ctx->J, e_loc_out, st, grid_for(ctx, S, 8, 16)));
    }
    ctx->launches += 1;
    VQ_CK(launch_accumulate_stats(counters, ctx->layers, S, ctx->stats, st));
    return VQNQS_OK;
}

int run(vqnqs_ctx* ctx, int B, const uint8_t* spins, float* e_loc, double* mean_var, float* log_psi, int flags,
        void* ws, size_t ws_bytes, void* stream, bool with_bonds) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (B < 0) return fail(ctx, VQNQS_ERR_ARG, "B must be >= 0");
    if (flags & ~(VQNQS_REUSE | VQNQS_BF16)) return fail(ctx, VQNQS_ERR_ARG, "unknown flag bits");
    if (flags & VQNQS_BF16) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_BF16 is not available in this build");
    if (B == 0) return VQNQS_OK;
    if (!spins) return fail(ctx, VQNQS_ERR_ARG, "spins is NULL");
    if (with_bonds && !e_loc) return fail(ctx, VQNQS_ERR_ARG, "e_loc is NULL");
    if (!with_bonds && !log_psi) return fail(ctx, VQNQS_ERR_ARG, "log_psi is NULL");
    if (!ws) return fail(ctx, VQNQS_ERR_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(ctx, VQNQS_ERR_ARG, "workspace must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int cur = -1;
    VQ_CK(cudaGetDevice(&cur));
    if (cur != ctx->device) return fail(ctx, VQNQS_ERR_ARG, "current device differs from the context's device");
    int S = fit_chunk(ctx, B, ws_bytes, with_bonds);
    if (S == 0) return fail(ctx, VQNQS_ERR_WORKSPACE, "workspace smaller than the one-sample minimum");
    const Plan P = make_plan(ctx, S, with_bonds);
    for (int s0 = 0; s0 < B; s0 += S) {
        const int Sc = (B - s0) < S ? (B - s0) : S;
        int rc = run_chunk(ctx, P, ws, spins + (size_t)s0 * ctx->N, Sc, with_bonds, flags,
                           e_loc ? e_loc + s0 : nullptr, log_psi ? log_psi + s0 : nullptr, st);
        if (rc != VQNQS_OK) return rc;
    }
    if (mean_var) VQ_STAGE(S_MEANVAR, 1, launch_mean_var(e_loc, B, mean_var, st));
    return VQNQS_OK;
}

}  // namespace

extern "C" {

size_t vqnqs_num_params(int n_max, int layers, int d_model, int K) {
    if (n_max <= 0 || layers <= 0 || d_model <= 0 || K <= 0) return 0;
    const size_t d = d_model;
    size_t per = 2 * d + d * 3 * d + 3 * d + (size_t)K * d + d * d + d + 2 * d + d * 4 * d + 4 * d + 4 * d * d + d;
    return 3 * d + (size_t)n_max * d + (size_t)layers * per + 2 * d + 2 * d + 2;
}

int vqnqs_create(int L, int periodic, double J, int layers, int d_model, int heads, int K, const float* weights,
                 vqnqs_ctx** out) {
    if (!out) return VQNQS_ERR_ARG;
    *out = nullptr;
    if (L < 2 || L * L > 512 || layers < 1 || layers > VQNQS_MAX_LAYERS || d_model < 32 || d_model % 32 ||
        d_model > 1024 || heads < 1 || d_model % heads || K < 1 || K > 65535 || !weights)
        return VQNQS_ERR_ARG;
    const int dh = d_model / heads;
    if (!(dh == 8 || dh == 16 || dh == 32)) return VQNQS_ERR_ARG;
    vqnqs_ctx* ctx = new vqnqs_ctx();
    ctx->L = L; ctx->N = L * L; ctx->periodic = periodic ? 1 : 0; ctx->J = J;
    ctx->layers = layers; ctx->d = d_model; ctx->heads = heads; ctx->K = K;
    auto bail = [&](int code) { vqnqs_destroy(ctx); return code; };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(VQNQS_ERR_CUDA);
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return bail(VQNQS_ERR_CUDA);
    ctx->nparams = vqnqs_num_params(ctx->N, layers, d_model, K);
    auto dalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        ctx->owned.push_back(p);
        return p;
    };
    ctx->blob = static_cast<float*>(dalloc(ctx->nparams * sizeof(float)));
    std::vector<int> bonds = make_bonds(L, ctx->periodic);
    ctx->nb = (int)bonds.size() / 2;
    ctx->bonds = static_cast<int*>(dalloc(bonds.size() * sizeof(int)));
    ctx->status = static_cast<int*>(dalloc(sizeof(int)));
    ctx->stats = static_cast<long long*>(dalloc(ST_SLOTS * sizeof(long long)));
    ctx->lw.resize(layers);
    const size_t d = d_model;
    for (int l = 0; l < layers; ++l) {
        LayerW& w = ctx->lw[l];
        w.T = static_cast<float*>(dalloc((size_t)K * d * sizeof(float)));
        w.cnorm = static_cast<float*>(dalloc((size_t)K * sizeof(float)));
        w.wqkv_t = static_cast<__nv_bfloat16*>(dalloc(3 * d * d * sizeof(__nv_bfloat16)));
        w.w1_t = static_cast<__nv_bfloat16*>(dalloc(4 * d * d * sizeof(__nv_bfloat16)));
        w.w2_t = static_cast<__nv_bfloat16*>(dalloc(4 * d * d * sizeof(__nv_bfloat16)));
        if (!w.T || !w.cnorm || !w.wqkv_t || !w.w1_t || !w.w2_t) return bail(VQNQS_ERR_OOM);
    }
    if (!ctx->blob || !ctx->bonds || !ctx->status || !ctx->stats) return bail(VQNQS_ERR_OOM);
    if (cudaMemcpy(ctx->bonds, bonds.data(), bonds.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->stats, 0, ST_SLOTS * sizeof(long long)) != cudaSuccess)
        return bail(VQNQS_ERR_CUDA);
    bind_weights(ctx);
    int rc = vqnqs_set_weights(ctx, weights, 0, nullptr);
    if (rc != VQNQS_OK) return bail(rc);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(VQNQS_ERR_CUDA);
    *out = ctx;
    return VQNQS_OK;
}

int vqnqs_set_weights(vqnqs_ctx* ctx, const float* weights, int is_device, void* stream) {
    if (!ctx || !weights) return VQNQS_ERR_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    VQ_CK(cudaMemcpyAsync(ctx->blob, weights, ctx->nparams * sizeof(float),
                          is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (!is_device) VQ_CK(cudaStreamSynchronize(st));
    return build_tables(ctx, st);
}

size_t vqnqs_workspace_bytes(const vqnqs_ctx* ctx, int chunk_samples, int flags) {
    (void)flags;
    if (!ctx) return 0;
    int S = chunk_samples > 0 ? chunk_samples : default_chunk(ctx, true);
    return make_plan(ctx, S, true).total;
}

int vqnqs_log_psi(vqnqs_ctx* ctx, int B, const uint8_t* spins, float* log_psi, int flags, void* ws, size_t ws_bytes,
                  void* stream) {
    return run(ctx, B, spins, nullptr, nullptr, log_psi, flags, ws, ws_bytes, stream, false);
}

int vqnqs_local_energy(vqnqs_ctx* ctx, int B, const uint8_t* spins, float* e_loc, double* mean_var, float* log_psi,
                       int flags, void* ws, size_t ws_bytes, void* stream) {
    return run(ctx, B, spins, e_loc, mean_var, log_psi, flags, ws, ws_bytes, stream, true);
}

int vqnqs_get_stats(vqnqs_ctx* ctx, vqnqs_stats* out) {
    if (!ctx || !out) return VQNQS_ERR_ARG;
    VQ_CK(cudaDeviceSynchronize());
    long long st[ST_SLOTS];
    int status = 0;
    VQ_CK(cudaMemcpy(st, ctx->stats, sizeof(st), cudaMemcpyDeviceToHost));
    VQ_CK(cudaMemcpy(&status, ctx->status, sizeof(int), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->samples = st[ST_SAMPLES];
    out->configs = st[ST_CONFIGS];
    out->rows = st[ST_ROWS];
    out->near_ties = st[ST_NEAR_TIES];
    for (int l = 0; l <= ctx->layers; ++l) out->unique_rows[l] = st[ST_U0 + l];
    out->device_status = status;
    // analytic FLOPs, 2 per multiply-add
    const double d = ctx->d, K = ctx->K, N = ctx->N, Ly = ctx->layers;
    const double rows = (double)out->rows, cfgs = (double)out->configs;
    const double attn = cfgs * Ly * 2.0 * d * N * (N + 1);
    const double vq = rows * Ly * 2.0 * K * d;
    out->flops_full = rows * Ly * 24.0 * d * d + attn + vq + rows * 4.0 * d;
    double done = attn + vq;
    for (int l = 0; l < ctx->layers; ++l)
        done += (double)out->unique_rows[l] * 6.0 * d * d + (double)out->unique_rows[l + 1] * 16.0 * d * d;
    done += (double)out->unique_rows[ctx->layers] * 4.0 * d;
    out->flops_done = done;
    return VQNQS_OK;
}

int vqnqs_reset_stats(vqnqs_ctx* ctx) {
    if (!ctx) return VQNQS_ERR_ARG;
    VQ_CK(cudaDeviceSynchronize());
    VQ_CK(cudaMemset(ctx->stats, 0, ST_SLOTS * sizeof(long long)));
    VQ_CK(cudaMemset(ctx->status, 0, sizeof(int)));
    VQ_CK(cudaDeviceSynchronize());
    return VQNQS_OK;
}

int vqnqs_profile_enable(vqnqs_ctx* ctx, int enable) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->prof = enable != 0;
    return VQNQS_OK;
}

int vqnqs_profile_read(vqnqs_ctx* ctx, vqnqs_stage_time* out, int max_stages, int* n_out) {
    if (!ctx || !out || !n_out || max_stages < 0) return VQNQS_ERR_ARG;
    VQ_CK(cudaDeviceSynchronize());
    for (auto& p : ctx->pending) {
        float ms = 0.f;
        VQ_CK(cudaEventElapsedTime(&ms, p.a, p.b));
        ctx->st_ms[p.stage] += ms;
        ctx->ev_free.push_back(p.a);
        ctx->ev_free.push_back(p.b);
    }
    ctx->pending.clear();
    int n = S_COUNT < max_stages ? S_COUNT : max_stages;
    for (int i = 0; i < n; ++i) {
        std::memset(&out[i], 0, sizeof(out[i]));
        std::snprintf(out[i].name, sizeof(out[i].name), "%s", kStageNames[i]);
        out[i].calls = ctx->st_calls[i];
        out[i].launches = ctx->st_launches[i];
        out[i].ms = ctx->st_ms[i];
        ctx->st_calls[i] = ctx->st_launches[i] = 0;
        ctx->st_ms[i] = 0.0;
    }
    *n_out = n;
    return VQNQS_OK;
}

int64_t vqnqs_launch_count(const vqnqs_ctx* ctx) { return ctx ? ctx->launches : 0; }

const char* vqnqs_last_error(const vqnqs_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void vqnqs_destroy(vqnqs_ctx* ctx) {
    if (!ctx) return;
    cudaDeviceSynchronize();
    for (auto& p : ctx->pending) { cudaEventDestroy(p.a); cudaEventDestroy(p.b); }
    for (auto e : ctx->ev_free) cudaEventDestroy(e);
    for (void* p : ctx->owned) cudaFree(p);
    delete ctx;
}

}  // extern "C"
