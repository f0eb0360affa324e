// C ABI of libvqnqs: context, workspace plan and the per-chunk pipeline of the
// local-energy path (Sec. 2 Eq. local-energy evaluated with the VQ-NQS of
// Sec. 3.1, reusing per-location work by (row, code) keys as in Sec. 3.2).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vqnqs_internal.cuh"

using namespace vq;

struct vqnqs_ctx {
    int L = 0, N = 0, periodic = 0, layers = 0, d = 0, heads = 0, K = 0, nb = 0;
    int vq_heads = 1, vq_bits = 0;  // quantizer heads; bits of one head's field in a packed code
    int vq_words = 1;               // 32-bit words of a code (2 when the heads need more than 32 bits)
    int half_block = 0;             // final attention-only half-block (its weights in hw)
    int G = 1, P = 0;               // spins per token; positions (rows) per sample = N / G
    int model = MODEL_HEISENBERG;
    int max_conn = 0;  // connected configurations per sample at most (bonds, or sites for the Ising chain)
    double J = 1.0, Gamma = 0.0;
    int device = 0, num_sms = 0;
    size_t nparams = 0;
    float* blob = nullptr;  // device copy of the weight blob
    const float *tok_emb = nullptr, *pos_emb = nullptr, *lnf_g = nullptr, *lnf_b = nullptr, *w_head = nullptr,
                *b_head = nullptr;
    std::vector<LayerW> lw;
    LayerW hw{};  // the final half-block: ln1, w_qkv, w_o and their biases, transposes and maps
    int* bonds = nullptr;          // [nb][2] bonds of the context's lattice (side L)
    int* bonds_all = nullptr;      // bond tables of every side 2 .. L, concatenated
    std::vector<int> side_bond_off, side_nb;  // per side: first bond in bonds_all, count
    int* status = nullptr;         // device status word
    int* gemm_m = nullptr;         // row count slot of vqnqs_gemm_bf16
    int* assign_counters = nullptr;  // counter slots of vqnqs_vq_assign
    int* assign_rows = nullptr;      // identity row list of vqnqs_vq_assign
    int assign_rows_cap = 1 << 22;
    float* lp_scratch = nullptr;     // log psi target of vqnqs_codes when the caller passes none
    int bn[3] = {0, 0, 0};           // output tile width of the QKV, MLP up, MLP down GEMMs
    int patch_items = 4;             // tensor-core patch: work items per CTA (sample, tile, slice)
    int rows_slices = 2;             // changed-row kernel: (sample, head, slice) items per SM
    int lp_scratch_cap = 65536;
    long long* stats = nullptr;    // ST_* slots
    bool bwd_tc = false;           // the backward's contractions can run on the tensor cores (split operands)
    int* dims = nullptr;           // device ints {d, 3d, 4d, K}: row counts of the backward's weight-gradient GEMMs
    float* zeros = nullptr;        // device zeros [max(4d, K)]: bias of those GEMMs
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

enum Stage { S_CONFIG, S_ACTIVE, S_EMBED, S_LN1, S_QKV, S_ATTN, S_VQ, S_DEDUPE, S_POSTLN, S_MLP1, S_MLP2, S_HEAD, S_ELOC,
             S_MEANVAR, S_BACKWARD, S_CERT, S_CLASSIFY, S_PATCH, S_RECOMP, S_RECOMP_WHOLE, S_HALF, S_EXACT,
             S_BWD_RECOMP, S_BWD_GEMM, S_BWD_ATTN, S_BWD_ROWS, S_COUNT };
const char* kStageNames[S_COUNT] = {"config", "active_rows", "embed", "ln1", "qkv_gemm", "attention", "vq_argmin", "dedupe",
                                    "post_ln", "mlp_up", "mlp_down", "head", "eloc", "mean_var", "backward",
                                    "inc_certificate", "inc_classify", "inc_patch", "inc_recompute",
                                    "inc_recompute_whole", "half_block", "inc_exact_delta", "bwd_recompute",
                                    "bwd_gemm", "bwd_attention", "bwd_rowwise"};
static_assert(S_COUNT <= VQNQS_MAX_STAGES, "stage table larger than the ABI's VQNQS_MAX_STAGES");

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
    int S = 0;                       // samples per chunk
    long long Cmax = 0, Rmax = 0, Umax = 0;
    int hash_bits = 0;
    size_t counters, cnt, cfg_off, diag, cfg_sample, cfg_i, cfg_j, cfg_row, row_cfg, act_cnt, act_off, act_rows,
        uid_a, uid_b, code, X_a, X_b, A, Y, scratch, keys, vals, rep_uid, rep_code, logp, ratio, bstat, cert,
        vq_rows, rc_rows, rc_cnt, list_tc, list_simt, dpos, dcnt, ex_rows, code_hi, tab_lo, tab_hi, blist, bdist, bosq,
        total;
};

// Workspace layout for chunks of at most S samples, C configurations and R rows.
Plan make_plan_budget(const vqnqs_ctx* c, int S, long long C, long long R) {
    Plan p;
    p.S = S;
    p.Cmax = C;
    p.Rmax = R;
    const long long emb_rows = (long long)((1 << c->G) + 1) * c->P;  // the reuse path's embedding table
    p.Umax = p.Rmax > emb_rows ? p.Rmax : emb_rows;
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
    p.cfg_row = take((size_t)(p.Cmax + 1) * sizeof(int));
    p.row_cfg = take((size_t)p.Rmax * sizeof(int));
    p.act_cnt = take((size_t)p.Cmax * sizeof(int));
    p.act_off = take((size_t)(p.Cmax + 1) * sizeof(int));
    p.act_rows = take((size_t)p.Rmax * sizeof(int));
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
    p.logp = take((size_t)p.Umax * (1 << c->G) * sizeof(float));
    p.ratio = take((size_t)p.Cmax * sizeof(float));
    // incremental path: samples' softmax statistics and certificates, search and recompute lists
    p.bstat = take((size_t)S * c->N * c->heads * sizeof(float2));
    p.cert = take((size_t)S * c->N * sizeof(CertRow));
    p.vq_rows = take((size_t)p.Rmax * sizeof(int));
    p.rc_rows = take((size_t)p.Rmax * sizeof(int2));
    p.rc_cnt = take((size_t)2 * S * sizeof(int));  // per sample: head and tail counts of the recompute list
    p.list_tc = take((size_t)p.Cmax * sizeof(int));
    p.list_simt = take((size_t)p.Cmax * sizeof(int));
    p.dpos = take((size_t)p.Cmax * INC_MAX_KEYS * sizeof(short));
    p.dcnt = take((size_t)p.Cmax * sizeof(int));
    p.ex_rows = take((size_t)p.Rmax * sizeof(int2));  // split operands: rows for the exact correction
    // two-word codes: the high words, and the words of each code id
    const size_t wbytes = c->vq_words > 1 ? (size_t)p.Rmax * sizeof(int) : 0;
    p.code_hi = take(wbytes);
    p.tab_lo = take(wbytes);
    p.tab_hi = take(wbytes);
    // the samples' rows for the certificate from the tensor-core distances: list, distances, ||o||^2
    const bool tc_cert = c->vq_heads == 1 && vq_tc_supported(c->K, c->d);
    const size_t srows = (size_t)S * c->N;
    p.blist = take(tc_cert ? (srows + 1) * sizeof(int) : 0);
    p.bdist = take(tc_cert ? srows * c->K * sizeof(float) : 0);
    p.bosq = take(tc_cert ? srows * sizeof(float) : 0);
    p.total = o;
    return p;
}

// Uniform chunks of S samples of the context's lattice (worst case: every bond anti-aligned).
Plan make_plan(const vqnqs_ctx* c, int S, bool with_bonds) {
    const long long C = (long long)S * (with_bonds ? (1 + c->max_conn) : 1);
    return make_plan_budget(c, S, C, C * c->P);
}

int default_chunk(const vqnqs_ctx* c, bool with_bonds) {
    // aim for about 2M token rows per chunk in the worst case
    long long per = (long long)(with_bonds ? (1 + c->max_conn) : 1) * c->P;
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
        VQ_CK(launch_table_T(w.codebook, w.w_o, w.b_o, K, d, ctx->vq_heads, w.T, w.cnorm, st));
        VQ_CK(launch_transpose_bf16(w.w_qkv, d, 3 * d, w.wqkv_t, st, true));
        VQ_CK(launch_transpose_bf16(w.w_1, d, 4 * d, w.w1_t, st, true));
        VQ_CK(launch_transpose_bf16(w.w_2, 4 * d, d, w.w2_t, st, true));
        if (ctx->vq_heads == 1) {  // the tensor-core search and the incremental certificate: one head
            VQ_CK(launch_split_tf32(w.codebook, (size_t)K * d, w.cb_hi, w.cb_lo, st));
            VQ_CK(launch_codeword_dist(w.codebook, K, d, w.wd, st));
        } else if (ctx->vq_words == 1 && K <= 1024) {  // the incremental certificate per quantizer head
            const int dq = d / ctx->vq_heads;
            for (int h = 0; h < ctx->vq_heads; ++h)
                VQ_CK(launch_codeword_dist(w.codebook + (size_t)h * K * dq, K, dq, w.wd + (size_t)h * K * K, st));
        }
        if (ctx->bwd_tc) {  // the backward's split weight planes
            const int cap = ctx->num_sms * 16;
            VQ_CK(launch_split_planes(w.w_qkv, d, 3 * d, w.wqkv_s, d, st, cap));
            VQ_CK(launch_split_planes(w.w_1, d, 4 * d, w.w1_s, d, st, cap));
            VQ_CK(launch_split_planes(w.w_2, 4 * d, d, w.w2_s, 4 * d, st, cap));
            VQ_CK(launch_split_planes(w.w_o, d, d, w.wo_s, d, st, cap));
            VQ_CK(launch_split_planes(w.codebook, K, d, w.cb_s, K, st, cap));
            VQ_CK(launch_transpose_bf16(w.codebook, K, d, w.cbT_s, st, true));
        }
    }
    if (ctx->half_block) {
        VQ_CK(launch_transpose_bf16(ctx->hw.w_qkv, d, 3 * d, ctx->hw.wqkv_t, st));
        VQ_CK(launch_transpose_bf16(ctx->hw.w_o, d, d, ctx->hw.wo_t, st));
    }
    return VQNQS_OK;
}

int build_weight_tmaps(vqnqs_ctx* ctx) {
    const long long d = ctx->d;
    for (int l = 0; l < ctx->layers; ++l) {
        LayerW& w = ctx->lw[l];
        // the maps cover the hi rows and the split lo rows after them
        VQ_CK(make_tmap_bf16(&w.tm_wqkv, w.wqkv_t, 2 * 3 * d, (int)d, ctx->bn[0]));
        VQ_CK(make_tmap_bf16(&w.tm_w1, w.w1_t, 2 * 4 * d, (int)d, ctx->bn[1]));
        VQ_CK(make_tmap_bf16(&w.tm_w2, w.w2_t, 2 * d, 4 * (int)d, ctx->bn[2]));
    }
    if (ctx->bwd_tc) {  // B operands of the backward's dX = dY W^T: box rows = the output tile width
        const int K = ctx->K;
        for (int l = 0; l < ctx->layers; ++l) {
            LayerW& w = ctx->lw[l];
            VQ_CK(make_tmap_bf16(&w.tm_wqkv_s, w.wqkv_s, 2 * d, 3 * (int)d, tc_pick_bn((int)d)));
            VQ_CK(make_tmap_bf16(&w.tm_w1_s, w.w1_s, 2 * d, 4 * (int)d, tc_pick_bn((int)d)));
            VQ_CK(make_tmap_bf16(&w.tm_w2_s, w.w2_s, 8 * d, (int)d, tc_pick_bn(4 * (int)d)));
            VQ_CK(make_tmap_bf16(&w.tm_wo_s, w.wo_s, 2 * d, (int)d, tc_pick_bn((int)d)));
            VQ_CK(make_tmap_bf16(&w.tm_cb_s, w.cb_s, 2LL * K, (int)d, tc_pick_bn(K)));
            VQ_CK(make_tmap_bf16(&w.tm_cbT_s, w.cbT_s, 2 * d, K, tc_pick_bn((int)d)));
        }
    }
    if (ctx->half_block) {
        VQ_CK(make_tmap_bf16(&ctx->hw.tm_wqkv, ctx->hw.wqkv_t, 3 * d, (int)d, ctx->bn[0]));
        VQ_CK(make_tmap_bf16(&ctx->hw.tm_wo, ctx->hw.wo_t, d, (int)d, ctx->bn[2]));
    }
    return VQNQS_OK;
}

void bind_weights(vqnqs_ctx* c) {
    const size_t d = c->d, K = c->K;
    const float* p = c->blob;
    auto take = [&](size_t n) { const float* r = p; p += n; return r; };
    c->tok_emb = take((size_t)((1 << c->G) + 1) * d);
    c->pos_emb = take((size_t)c->P * d);
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
    if (c->half_block) {
        LayerW& w = c->hw;
        w.ln1_g = take(d); w.ln1_b = take(d);
        w.w_qkv = take(d * 3 * d); w.b_qkv = take(3 * d);
        w.w_o = take(d * d); w.b_o = take(d);
    }
    c->lnf_g = take(d); c->lnf_b = take(d);
    c->w_head = take((size_t)(1 << c->G) * d); c->b_head = take((size_t)1 << c->G);
}

// Lattice groups of a single-lattice batch.
Groups uniform_groups(const vqnqs_ctx* c, int B) {
    Groups g;
    std::memset(&g, 0, sizeof(g));
    g.n = 1;
    g.first[0] = 0;
    g.first[1] = B;
    g.N[0] = c->N;
    g.nb[0] = c->side_nb[c->L];
    g.bond_off[0] = c->side_bond_off[c->L];
    g.spin_off[0] = 0;
    return g;
}

Chunk make_chunk(const vqnqs_ctx* ctx, const Plan& P, void* ws, const uint8_t* spins, const Groups& g, int s0, int S) {
    Chunk ch;
    ch.spins = spins; ch.bonds = ctx->bonds_all; ch.g = g; ch.s0 = s0; ch.S = S;
    ch.N = ctx->P; ch.G = ctx->G; ch.d = ctx->d; ch.heads = ctx->heads; ch.K = ctx->K; ch.model = ctx->model;
    ch.cfg_sample = at<int>(ws, P.cfg_sample);
    ch.cfg_i = at<int>(ws, P.cfg_i);
    ch.cfg_j = at<int>(ws, P.cfg_j);
    ch.cfg_off = at<int>(ws, P.cfg_off);
    ch.cfg_row = at<int>(ws, P.cfg_row);
    ch.row_cfg = at<int>(ws, P.row_cfg);
    ch.counters = at<int>(ws, P.counters);
    return ch;
}

// One chunk of samples (global s0 .. s0+S-1 of the batch described by g) through the whole path.
int run_chunk(vqnqs_ctx* ctx, const Plan& P, void* ws, const uint8_t* spins, const Groups& grp, int s0, int S,
              bool with_bonds, int flags, float* e_loc_out, float* log_psi_out, cudaStream_t st,
              int* codes_out = nullptr, int* cfg_codes_out = nullptr) {
    const int N = ctx->P, d = ctx->d, K = ctx->K;  // N: positions (rows) per sample
    const bool reuse = (flags & VQNQS_REUSE) != 0;
    int* counters = at<int>(ws, P.counters);
    Chunk ch = make_chunk(ctx, P, ws, spins, grp, s0, S);
    float* diag = at<float>(ws, P.diag);
    const int g_s = grid_for(ctx, S, 1, 8);
    const float diag_coef = ctx->model == MODEL_TFIM_CHAIN ? (float)-ctx->J : (float)(0.25 * ctx->J);
    const float offdiag = ctx->model == MODEL_TFIM_CHAIN ? (float)-ctx->Gamma : (float)(-0.5 * ctx->J);
    VQ_STAGE(S_CONFIG, 5, launch_configs(ch, diag_coef, with_bonds, at<int>(ws, P.cnt), diag,
                                         at<int>(ws, P.cfg_off), at<int>(ws, P.cfg_sample), at<int>(ws, P.cfg_i),
                                         at<int>(ws, P.cfg_j), at<int>(ws, P.cfg_row), at<int>(ws, P.row_cfg),
                                         ctx->status, st, g_s));

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

    const bool bf16 = (flags & VQNQS_BF16) != 0;
    const bool inc = with_bonds && (flags & VQNQS_INCREMENTAL) != 0;
    // split operands: BF16 lo planes after the hi ones (elements) of the LN outputs, Q/K/V and MLP hidden rows
    const bool split = bf16 && (flags & VQNQS_BF16_SPLIT) != 0;
    // two-word codes: the words of each code id (the residual step decodes the heads' fields)
    const int* tab_lo = ctx->vq_words > 1 ? at<int>(ws, P.tab_lo) : nullptr;
    const int* tab_hi = ctx->vq_words > 1 ? at<int>(ws, P.tab_hi) : nullptr;
    const size_t a_lo = split ? (size_t)P.Umax * d : 0;
    const size_t qkv_lo = split ? (size_t)P.Umax * 3 * d : 0;
    int* act_rows = at<int>(ws, P.act_rows);
    const int* cfg_off = at<int>(ws, P.cfg_off);
    float2* bstat = at<float2>(ws, P.bstat);
    CertRow* cert = at<CertRow>(ws, P.cert);
    int* vq_rows = at<int>(ws, P.vq_rows);
    int2* rc_rows = at<int2>(ws, P.rc_rows);
    int* rc_cnt = at<int>(ws, P.rc_cnt);
    const int* act_off = at<int>(ws, P.act_off);
    int* list_tc = at<int>(ws, P.list_tc);
    int* list_simt = at<int>(ws, P.list_simt);
    short* dpos = at<short>(ws, P.dpos);
    int* dcnt = at<int>(ws, P.dcnt);
    VQ_STAGE(S_ACTIVE, 3, launch_active_rows(ch, reuse ? 1 : 0, at<int>(ws, P.act_cnt), at<int>(ws, P.act_off),
                                             act_rows, ctx->stats, st, grid_for(ctx, P.Cmax, 8, 16)));
    __nv_bfloat16* A16 = reinterpret_cast<__nv_bfloat16*>(A);
    __nv_bfloat16* qkv16 = reinterpret_cast<__nv_bfloat16*>(qkv);
    __nv_bfloat16* Hid16 = reinterpret_cast<__nv_bfloat16*>(Hid);
    VQ_STAGE(S_EMBED, reuse ? 2 : 1, launch_embed(ch, ctx->tok_emb, ctx->pos_emb, reuse, X_cur, uid_cur, st, g_rows));
    for (int l = 0; l < ctx->layers; ++l) {
        const LayerW& w = ctx->lw[l];
        const int us = CNT_U0 + l, un = CNT_U0 + l + 1;
        if (bf16) {
            VQ_STAGE(S_LN1, 1, launch_layernorm(X_cur, counters, us, w.ln1_g, w.ln1_b, d, nullptr, A16, st, g_urows,
                                                a_lo));
            VQ_STAGE(S_QKV, 1, launch_gemm_tc(A16, Umax, w.tm_wqkv, w.b_qkv, nullptr, qkv16, counters, us, 3 * d, d, 0,
                                              ctx->status, st, ctx->num_sms, ctx->bn[0], split));
            if (inc) {  // the samples' own configurations only, with their softmax statistics
                if (attention_tc_supported(N, d / ctx->heads, split))
                    VQ_STAGE(S_ATTN, 1, launch_attention_tc(ch, uid_cur, qkv16, O, 1, ctx->status, st,
                                                            grid_for(ctx, (long long)S * ctx->heads, 1, 4), cfg_off, S,
                                                            bstat, nullptr, qkv_lo));
                else
                    VQ_STAGE(S_ATTN, 1, launch_attention_bf16in(ch, uid_cur, qkv16, O, 1, st,
                                                                grid_for(ctx, (long long)S * ctx->heads, 1, 8), cfg_off,
                                                                S, bstat));
            } else if (attention_tc_supported(N, d / ctx->heads, split))
                VQ_STAGE(S_ATTN, 1, launch_attention_tc(ch, uid_cur, qkv16, O, reuse ? 1 : 0, ctx->status, st,
                                                        grid_for(ctx, P.Cmax * ctx->heads, 1, 4), nullptr, 0,
                                                        nullptr, nullptr, qkv_lo));
            else
                VQ_STAGE(S_ATTN, 1, launch_attention_bf16in(ch, uid_cur, qkv16, O, reuse ? 1 : 0, st,
                                                            grid_for(ctx, P.Cmax * ctx->heads, 1, 8)));
        } else {
            VQ_STAGE(S_LN1, 1, launch_layernorm(X_cur, counters, us, w.ln1_g, w.ln1_b, d, A, nullptr, st, g_urows));
            VQ_STAGE(S_QKV, 1, launch_sgemm(A, w.w_qkv, w.b_qkv, nullptr, qkv, counters, us, Umax, 3 * d, d, EPI_BIAS,
                                            st, ctx->num_sms));
            if (inc)
                VQ_STAGE(S_ATTN, 1, launch_attention_f32(ch, uid_cur, qkv, O, 1, st,
                                                         grid_for(ctx, (long long)S * ctx->heads, 1, 8), cfg_off, S,
                                                         bstat));
            else
                VQ_STAGE(S_ATTN, 1, launch_attention_f32(ch, uid_cur, qkv, O, reuse ? 1 : 0, st,
                                                         grid_for(ctx, P.Cmax * ctx->heads, 1, 8)));
        }
        if (inc) {
            // the samples' rows: codeword and certificate; then the connected configurations
            if (ctx->vq_heads > 1)
                VQ_STAGE(S_CERT, 1, launch_base_cert_heads(ch, O, w.codebook, w.cnorm, w.wd, K, d, ctx->vq_heads,
                                                           ctx->vq_bits, code, cert, ctx->stats, counters, rc_cnt,
                                                           st, ctx->num_sms));
            else if (bf16 && vq_tc_supported(K, d))  // the samples' codes from the search the connected rows get
                VQ_STAGE(S_CERT, 3, launch_base_cert_tc(ch, O, w.tm_cb_hi, w.tm_cb_lo, w.cnorm, w.wd, K, d, code,
                                                        cert, ctx->stats, counters, rc_cnt, at<int>(ws, P.blist),
                                                        at<float>(ws, P.bdist), at<float>(ws, P.bosq), ctx->status,
                                                        st, ctx->num_sms));
            else
                VQ_STAGE(S_CERT, 1, launch_base_cert(ch, O, w.codebook, w.cnorm, w.wd, K, d, code, cert, ctx->stats,
                                                     counters, rc_cnt, st));
            const int g_cfg = grid_for(ctx, P.Cmax, 1, 3);
            const bool tc_inc = bf16 && patch_tc_supported(d, ctx->heads) &&
                                attention_tc_supported(N, d / ctx->heads, split) &&
                                attention_rows_tc_supported(N, d, ctx->heads);
            VQ_STAGE(S_CLASSIFY, 1, launch_inc_classify(ch, uid_cur, tc_inc ? 1 : 0, list_tc, list_simt, dpos, dcnt,
                                                        vq_rows, ctx->stats, st, grid_for(ctx, P.Cmax, 8, 8)));
            if (tc_inc) {
                // tensor cores: rows patched, their changed rows recomputed against the sample's keys,
                // configurations with many changes recomputed whole
                int2* ex_rows = at<int2>(ws, P.ex_rows);
                VQ_STAGE(S_PATCH, 1, launch_inc_patch(ch, uid_cur, qkv16, O, bstat, cert, w.codebook, w.wd, code,
                                                      vq_rows, act_off, rc_rows, rc_cnt, list_tc, list_simt, dpos,
                                                      dcnt, 1, split ? 1 : 0, ex_rows, ctx->status, ctx->stats, st,
                                                      g_cfg, ctx->patch_items));
                if (split)
                    VQ_STAGE(S_EXACT, 1, launch_inc_exact_delta(ch, uid_cur, qkv16, qkv_lo, O, bstat, dpos, dcnt,
                                                                ex_rows, counters + CNT_EX, st,
                                                                grid_for(ctx, P.Rmax, 8, 8)));
                VQ_STAGE(S_RECOMP, 1, launch_attention_rows_tc(ch, uid_cur, qkv16, O, rc_rows, act_off, rc_cnt, dpos,
                                                               dcnt, ctx->status, ctx->stats, st, ctx->num_sms,
                                                               qkv_lo, ctx->rows_slices));
                VQ_STAGE(S_RECOMP_WHOLE, 1,
                         launch_attention_tc(ch, uid_cur, qkv16, O, 1, ctx->status, st,
                                             grid_for(ctx, P.Cmax * ctx->heads, 1, 2), list_simt, 0, nullptr,
                                             counters + CNT_SCL, qkv_lo, counters + CNT_SCW));
            } else if (bf16) {
                VQ_STAGE(S_PATCH, 1, launch_inc_patch(ch, uid_cur, qkv16, O, bstat, cert, w.codebook, w.wd, code,
                                                      vq_rows, act_off, rc_rows, rc_cnt, list_tc, list_simt, dpos,
                                                      dcnt, 0, 0, nullptr, ctx->status, ctx->stats, st, g_cfg));
                VQ_STAGE(S_RECOMP, 1, launch_inc_attention(ch, uid_cur, qkv16, O, act_off, rc_rows, rc_cnt, 0,
                                                           ctx->stats, st, ctx->num_sms));
            } else {
                VQ_STAGE(S_PATCH, 1, launch_inc_patch(ch, uid_cur, qkv, O, bstat, cert, w.codebook, w.wd, code,
                                                      vq_rows, act_off, rc_rows, rc_cnt, list_tc, list_simt, dpos,
                                                      dcnt, 0, ctx->status, ctx->stats, st, g_cfg));
                VQ_STAGE(S_RECOMP, 1, launch_inc_attention(ch, uid_cur, qkv, O, act_off, rc_rows, rc_cnt, 0, ctx->stats,
                                                           st, ctx->num_sms));
            }
        }
        const int* vq_list = inc ? vq_rows : act_rows;
        const int vq_slot = inc ? CNT_V : CNT_A;
        if (ctx->vq_heads > 1) {  // one search per quantizer head, FP32 on the CUDA cores
            int* code_hi = ctx->vq_words > 1 ? at<int>(ws, P.code_hi) : nullptr;
            VQ_STAGE(S_VQ, ctx->vq_heads,
                     launch_vq_argmin_heads(O, counters, vq_list, w.codebook, w.cnorm, K, d, ctx->vq_heads,
                                            ctx->vq_bits, code, ctx->stats + ST_NEAR_TIES, Rmax, st, ctx->num_sms,
                                            vq_slot, code_hi));
            if (code_hi)  // two-word codes: a dense id per distinct code, the dedupe keys on the id
                VQ_STAGE(S_DEDUPE, 3,
                         launch_code_words(counters, vq_slot, CNT_CW, vq_list, Rmax, code, code_hi,
                                           at<unsigned long long>(ws, P.keys), at<int>(ws, P.vals), P.hash_bits,
                                           at<int>(ws, P.tab_hi), at<int>(ws, P.tab_lo), ctx->status, st,
                                           ctx->num_sms));
        }
        else if (bf16 && vq_tc_supported(K, d))
            VQ_STAGE(S_VQ, 1, launch_vq_tc(w.tm_cb_hi, w.tm_cb_lo, O, counters, vq_list, w.cnorm, K, d, code,
                                           ctx->stats + ST_NEAR_TIES, ctx->status, st, ctx->num_sms, Rmax, vq_slot));
        else
            VQ_STAGE(S_VQ, 1, launch_vq_argmin(O, counters, vq_list, w.codebook, w.cnorm, K, d, code,
                                               ctx->stats + ST_NEAR_TIES, Rmax, st, ctx->num_sms, vq_slot));
        if (codes_out) {  // codes of every row: [sample][layer][position] (no connected configurations here)
            ctx->launches += 1;
            VQ_CK(launch_copy_codes(ch, code, l, ctx->layers, codes_out, st, g_rows));
        }
        if (cfg_codes_out) {  // codes of every configuration: [sample][configuration][layer][position]
            ctx->launches += 1;
            VQ_CK(launch_copy_cfg_codes(ch, code, l, ctx->layers, 1 + ctx->max_conn, cfg_codes_out, st, g_rows));
        }
        VQ_STAGE(S_DEDUPE, reuse ? 3 : 1,
                 launch_dedupe(ch, uid_cur, code, un, Rmax, at<unsigned long long>(ws, P.keys),
                               at<int>(ws, P.vals), P.hash_bits, uid_next, rep_uid, rep_code, reuse, ctx->status, st,
                               ctx->num_sms));
        if (bf16) {
            VQ_STAGE(S_POSTLN, 1, launch_residual_vq_ln(X_cur, rep_uid, rep_code, w.T, counters, un, w.ln2_g, w.ln2_b,
                                                        d, Y, nullptr, A16, st, g_urows, ctx->vq_heads, K,
                                                        ctx->vq_bits, a_lo, tab_lo, tab_hi));
            // split: the hidden rows' lo plane follows the hi one (Umax rows of 4d, over the dead attention output)
            VQ_STAGE(S_MLP1, 1, launch_gemm_tc(A16, Umax, w.tm_w1, w.b_1, nullptr, Hid16, counters, un, 4 * d, d, 1,
                                               ctx->status, st, ctx->num_sms, ctx->bn[1], split));
            VQ_STAGE(S_MLP2, 1, launch_gemm_tc(Hid16, Umax, w.tm_w2, w.b_2, Y, X_next, counters, un, d, 4 * d, 2,
                                               ctx->status, st, ctx->num_sms, ctx->bn[2], split));
        } else {
            VQ_STAGE(S_POSTLN, 1, launch_residual_vq_ln(X_cur, rep_uid, rep_code, w.T, counters, un, w.ln2_g, w.ln2_b,
                                                        d, Y, A, nullptr, st, g_urows, ctx->vq_heads, K,
                                                        ctx->vq_bits, 0, tab_lo, tab_hi));
            VQ_STAGE(S_MLP1, 1, launch_sgemm(A, w.w_1, w.b_1, nullptr, Hid, counters, un, Umax, 4 * d, d,
                                             EPI_BIAS_GELU, st, ctx->num_sms));
            VQ_STAGE(S_MLP2, 1, launch_sgemm(Hid, w.w_2, w.b_2, Y, X_next, counters, un, Umax, d, 4 * d,
                                             EPI_BIAS_RESID, st, ctx->num_sms));
        }
        std::swap(uid_cur, uid_next);
        std::swap(X_cur, X_next);
    }
    const int* uid_final = uid_cur;
    const float* X_head = X_cur;
    int head_slot = CNT_U0 + ctx->layers;
    if (ctx->half_block) {
        // Table 1's final half-block: LN and QKV on the unique rows, attention over the active
        // rows, then W_o and the residual per active row.  Without a quantizer the rows stay
        // distinct from here on: each active row is its own row for the head and the ratios.
        const LayerW& w = ctx->hw;
        const int us = CNT_U0 + ctx->layers;
        if (bf16) {
            VQ_STAGE(S_LN1, 1, launch_layernorm(X_cur, counters, us, w.ln1_g, w.ln1_b, d, nullptr, A16, st, g_urows));
            VQ_STAGE(S_QKV, 1, launch_gemm_tc(A16, Umax, w.tm_wqkv, w.b_qkv, nullptr, qkv16, counters, us, 3 * d, d, 0,
                                              ctx->status, st, ctx->num_sms, ctx->bn[0]));
            if (attention_tc_supported(N, d / ctx->heads))
                VQ_STAGE(S_ATTN, 1, launch_attention_tc(ch, uid_cur, qkv16, O, reuse ? 1 : 0, ctx->status, st,
                                                        grid_for(ctx, P.Cmax * ctx->heads, 1, 4)));
            else
                VQ_STAGE(S_ATTN, 1, launch_attention_bf16in(ch, uid_cur, qkv16, O, reuse ? 1 : 0, st,
                                                            grid_for(ctx, P.Cmax * ctx->heads, 1, 8)));
        } else {
            VQ_STAGE(S_LN1, 1, launch_layernorm(X_cur, counters, us, w.ln1_g, w.ln1_b, d, A, nullptr, st, g_urows));
            VQ_STAGE(S_QKV, 1, launch_sgemm(A, w.w_qkv, w.b_qkv, nullptr, qkv, counters, us, Umax, 3 * d, d, EPI_BIAS,
                                            st, ctx->num_sms));
            VQ_STAGE(S_ATTN, 1, launch_attention_f32(ch, uid_cur, qkv, O, reuse ? 1 : 0, st,
                                                     grid_for(ctx, P.Cmax * ctx->heads, 1, 8)));
        }
        StageScope scope_(ctx, S_HALF, 3, st);
        VQ_CK(launch_half_gather(counters, act_rows, uid_cur, O, X_cur, d, bf16 ? nullptr : A, bf16 ? A16 : nullptr, Y,
                                 st, g_rows));
        if (bf16)
            VQ_CK(launch_gemm_tc(A16, Umax, w.tm_wo, w.b_o, Y, X_next, counters, CNT_A, d, d, 2, ctx->status, st,
                                 ctx->num_sms, ctx->bn[2]));
        else
            VQ_CK(launch_sgemm(A, w.w_o, w.b_o, Y, X_next, counters, CNT_A, Umax, d, d, EPI_BIAS_RESID, st,
                               ctx->num_sms));
        VQ_CK(launch_half_ids(ch, reuse ? 1 : 0, act_off, uid_next, st, grid_for(ctx, P.Cmax, 8, 16)));
        uid_final = uid_next;
        X_head = X_next;
        head_slot = CNT_A;
    }
    float* logp = at<float>(ws, P.logp);
    VQ_STAGE(S_HEAD, 1, launch_head(X_head, counters, head_slot, ctx->lnf_g, ctx->lnf_b, ctx->w_head, ctx->b_head, d,
                                    logp, st, g_urows, ctx->G));
    float* ratio = at<float>(ws, P.ratio);
    {
        StageScope scope_(ctx, S_ELOC, e_loc_out ? 2 : 1, st);
        VQ_CK(launch_eloc(ch, uid_final, logp, ratio, log_psi_out, st, grid_for(ctx, P.Cmax, 8, 16)));
        if (e_loc_out)
            VQ_CK(launch_eloc_reduce(ch, diag, ratio, offdiag, e_loc_out, st, grid_for(ctx, S, 8, 16)));
    }
    ctx->launches += 1;
    VQ_CK(launch_accumulate_stats(counters, ctx->layers, S, ctx->stats, st));
    return VQNQS_OK;
}

// Flags of the local-energy, log psi and codes paths for this context's model.
int check_flags(vqnqs_ctx* ctx, int flags) {
    if (flags & ~(VQNQS_REUSE | VQNQS_BF16 | VQNQS_INCREMENTAL | VQNQS_BF16_SPLIT))
        return fail(ctx, VQNQS_ERR_ARG, "unknown flag bits");
    if (flags & VQNQS_INCREMENTAL) {
        if (!(flags & VQNQS_REUSE)) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL needs VQNQS_REUSE");
        if (ctx->vq_heads > 1 && (ctx->vq_words > 1 || ctx->K > 1024))
            return fail(ctx, VQNQS_ERR_ARG,
                        "VQNQS_INCREMENTAL with several quantizer heads needs a one-word code and K <= 1024");
        if (ctx->half_block) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL: no final half-block");
        if (ctx->G > 1) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL: one spin per token");
        if (!incremental_supported(ctx->d, ctx->heads))
            return fail(ctx, VQNQS_ERR_ARG,
                        "VQNQS_INCREMENTAL needs d_model in {32, 64, 128, 256, 512} and d_model/heads in {16, 32}, "
                        "a multiple of d_model/32");
    }
    if ((flags & VQNQS_BF16) && ctx->d % 64) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_BF16 needs d_model % 64 == 0");
    if (flags & VQNQS_BF16_SPLIT) {
        if (!(flags & VQNQS_BF16)) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_BF16_SPLIT needs VQNQS_BF16");
        if (ctx->half_block) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_BF16_SPLIT: no final half-block");
        if (!attention_tc_supported(ctx->P, ctx->d / ctx->heads, true))
            return fail(ctx, VQNQS_ERR_ARG, "VQNQS_BF16_SPLIT needs d_model/heads in {16, 32} and at most 256 positions");
        if ((flags & VQNQS_INCREMENTAL) &&
            !(patch_tc_supported(ctx->d, ctx->heads) && attention_rows_tc_supported(ctx->P, ctx->d, ctx->heads)))
            return fail(ctx, VQNQS_ERR_ARG,
                        "VQNQS_BF16_SPLIT with VQNQS_INCREMENTAL needs d_model/heads = 32 and d_model in {128, 256}");
    }
    return VQNQS_OK;
}

int run(vqnqs_ctx* ctx, int B, const uint8_t* spins, float* e_loc, double* mean_var, float* log_psi, int flags,
        void* ws, size_t ws_bytes, void* stream, bool with_bonds, int* codes = nullptr, int* cfg_codes = nullptr) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (B < 0) return fail(ctx, VQNQS_ERR_ARG, "B must be >= 0");
    if (int rc = check_flags(ctx, flags)) return rc;
    if ((codes || cfg_codes) && ctx->vq_words > 1)
        return fail(ctx, VQNQS_ERR_ARG, "codes: the quantizer's codes are wider than 32 bits");
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
    const Groups g = uniform_groups(ctx, B);
    for (int s0 = 0; s0 < B; s0 += S) {
        const int Sc = (B - s0) < S ? (B - s0) : S;
        int rc = run_chunk(ctx, P, ws, spins, g, s0, Sc, with_bonds, flags, e_loc ? e_loc + s0 : nullptr,
                           log_psi ? log_psi + s0 : nullptr, st,
                           codes ? codes + (size_t)s0 * ctx->layers * ctx->P : nullptr,
                           cfg_codes ? cfg_codes + (size_t)s0 * (1 + ctx->max_conn) * ctx->layers * ctx->P : nullptr);
        if (rc != VQNQS_OK) return rc;
    }
    if (mean_var) VQ_STAGE(S_MEANVAR, 1, launch_mean_var(e_loc, B, mean_var, st));
    return VQNQS_OK;
}

// ---- gradient of log psi ---------------------------------------------------------
struct ParamOff {
    size_t tok, pos, lnf_g, lnf_b, wh, bh;
    struct L { size_t ln1_g, ln1_b, wqkv, bqkv, cb, wo, bo, ln2_g, ln2_b, w1, b1, w2, b2; };
    std::vector<L> l;
};

ParamOff param_offsets(const vqnqs_ctx* c) {
    ParamOff o;
    const size_t d = c->d, K = c->K;
    size_t p = 0;
    auto take = [&](size_t n) { size_t r = p; p += n; return r; };
    o.tok = take(3 * d);
    o.pos = take((size_t)c->N * d);
    o.l.resize(c->layers);
    for (int l = 0; l < c->layers; ++l) {
        auto& w = o.l[l];
        w.ln1_g = take(d); w.ln1_b = take(d); w.wqkv = take(3 * d * d); w.bqkv = take(3 * d);
        w.cb = take(K * d); w.wo = take(d * d); w.bo = take(d); w.ln2_g = take(d); w.ln2_b = take(d);
        w.w1 = take(4 * d * d); w.b1 = take(4 * d); w.w2 = take(4 * d * d); w.b2 = take(d);
    }
    o.lnf_g = take(d); o.lnf_b = take(d); o.wh = take(2 * d); o.bh = take(2);
    return o;
}

struct GradPlan {
    int S = 0, B = 0;
    long long R = 0;
    size_t seeds, counters, cnt, cfg_off, diag, cfg_sample, cfg_i, cfg_j, act_cnt, act_off, act_rows, uid_a, uid_b,
        rep_uid, rep_code, code, X, dX, dY, A1, Oatt, Y, V, A2, dA, dV, dO, dgam, dbet, Af, QKV, dQKV, H1, G4, dG4, OW,
        DG, alpha, onehot, arow, dlog, csumK, stat, cfg_row, row_cfg, s16, tw, colpart, kpart, total;
};

constexpr int kColParts = 1 << 20;  // floats of partial column sums (slabs x columns)
constexpr int kSplitK = 16;              // K splits of a weight-gradient GEMM, at most
constexpr size_t kSplitKElems = 1 << 20;  // floats of one split's partial result, at most (in x out <= 1 M)

GradPlan make_grad_plan(const vqnqs_ctx* c, int S, int B) {
    GradPlan p;
    p.S = S;
    p.B = B;
    p.R = (long long)S * c->N;
    const size_t R = p.R, d = c->d, K = c->K, L = c->layers;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    const size_t f = sizeof(float);
    p.seeds = take((size_t)(B > 0 ? B : 1) * f);
    p.counters = take(CNT_SLOTS * sizeof(int));
    p.cnt = take(S * sizeof(int)); p.cfg_off = take((S + 1) * sizeof(int)); p.diag = take(S * f);
    p.cfg_sample = take(S * sizeof(int)); p.cfg_i = take(S * sizeof(int)); p.cfg_j = take(S * sizeof(int));
    p.act_cnt = take(S * sizeof(int)); p.act_off = take(S * sizeof(int)); p.act_rows = take(R * sizeof(int));
    p.uid_a = take(R * sizeof(int)); p.uid_b = take(R * sizeof(int));
    p.rep_uid = take(R * sizeof(int)); p.rep_code = take(R * sizeof(int));
    p.code = take(L * R * sizeof(int));
    p.X = take((L + 1) * R * d * f);
    p.dX = take(R * d * f); p.dY = take(R * d * f); p.A1 = take(R * d * f); p.Oatt = take(R * d * f);
    p.Y = take(R * d * f); p.V = take(R * d * f); p.A2 = take(R * d * f); p.dA = take(R * d * f);
    p.dV = take(R * d * f); p.dO = take(R * d * f); p.dgam = take(R * d * f); p.dbet = take(R * d * f);
    p.Af = take(R * d * f);
    p.QKV = take(R * 3 * d * f); p.dQKV = take(R * 3 * d * f);
    p.H1 = take(R * 4 * d * f); p.G4 = take(R * 4 * d * f); p.dG4 = take(R * 4 * d * f);
    p.OW = take(R * K * f); p.DG = take(R * K * f); p.alpha = take(R * K * f); p.onehot = take(R * K * f);
    p.arow = take(R * f); p.dlog = take(2 * R * f); p.csumK = take((size_t)S * K * f);
    p.stat = take(R * c->heads * 3 * f);
    p.cfg_row = take((S + 1) * sizeof(int));
    p.row_cfg = take(R * sizeof(int));
    // tensor-core backward: one activation as split planes [2R][max(4d, K)], and the two transposed
    // split operands of a weight-gradient GEMM, [2 in][R] and [2 out][R] with in + out <= max(5d, K + d)
    p.s16 = take(c->bwd_tc ? R * std::max(4 * d, K) * 4 : 0);
    p.tw = take(c->bwd_tc ? R * std::max(5 * d, K + d) * 4 : 0);
    p.colpart = take((size_t)kColParts * f);  // row-slab partial column sums
    p.kpart = take(c->bwd_tc ? (size_t)kSplitK * kSplitKElems * f : 0);  // split-K partial weight gradients
    p.total = o;
    return p;
}

int grad_default_chunk(const vqnqs_ctx* c) {
    long long s = (256LL << 10) / c->N;
    return (int)(s < 1 ? 1 : (s > 65536 ? 65536 : s));
}

// One chunk: forward with saved residual streams, then the backward.  OUT is the
// gradient base of this chunk (grad, or O + first sample * P), groups of G rows.
int grad_chunk(vqnqs_ctx* ctx, const GradPlan& P, void* ws, const uint8_t* spins, int S, const float* seeds,
               float* OUT, int G, long long ostride, cudaStream_t st, int flags) {
    const int N = ctx->N, d = ctx->d, K = ctx->K, Ly = ctx->layers, H = ctx->heads;
    const int R = S * N, ng = R / G;
    const int cap = ctx->num_sms * 16, sms = ctx->num_sms;
    // the summed gradient's contractions on the tensor cores (split operands) with VQNQS_BF16
    const bool tcb = ctx->bwd_tc && (flags & VQNQS_BF16) && G == R && R % 8 == 0;
    int* counters = at<int>(ws, P.counters);
    Chunk ch;
    ch.spins = spins; ch.bonds = ctx->bonds_all; ch.g = uniform_groups(ctx, S); ch.s0 = 0; ch.S = S;
    ch.model = ctx->model;
    ch.N = N; ch.d = d; ch.heads = H; ch.K = K;
    ch.cfg_sample = at<int>(ws, P.cfg_sample); ch.cfg_i = at<int>(ws, P.cfg_i); ch.cfg_j = at<int>(ws, P.cfg_j);
    ch.cfg_off = at<int>(ws, P.cfg_off); ch.cfg_row = at<int>(ws, P.cfg_row); ch.row_cfg = at<int>(ws, P.row_cfg);
    ch.counters = counters;
    const ParamOff po = param_offsets(ctx);
    auto X = [&](int l) { return at<float>(ws, P.X + (size_t)l * R * d * sizeof(float)); };
    auto code = [&](int l) { return at<int>(ws, P.code + (size_t)l * R * sizeof(int)); };
    float *dX = at<float>(ws, P.dX), *dY = at<float>(ws, P.dY), *A1 = at<float>(ws, P.A1), *Oatt = at<float>(ws, P.Oatt);
    float *Y = at<float>(ws, P.Y), *V = at<float>(ws, P.V), *A2 = at<float>(ws, P.A2), *dA = at<float>(ws, P.dA);
    float *dV = at<float>(ws, P.dV), *dO = at<float>(ws, P.dO), *dgam = at<float>(ws, P.dgam);
    float *dbet = at<float>(ws, P.dbet), *Af = at<float>(ws, P.Af), *QKV = at<float>(ws, P.QKV);
    float *dQKV = at<float>(ws, P.dQKV), *H1 = at<float>(ws, P.H1), *G4 = at<float>(ws, P.G4);
    float *dG4 = at<float>(ws, P.dG4), *OW = at<float>(ws, P.OW), *DG = at<float>(ws, P.DG);
    float *alpha = at<float>(ws, P.alpha), *onehot = at<float>(ws, P.onehot), *arow = at<float>(ws, P.arow);
    float *dlog = at<float>(ws, P.dlog), *csumK = at<float>(ws, P.csumK);
    int *uid = at<int>(ws, P.uid_a), *uid_b = at<int>(ws, P.uid_b), *act = at<int>(ws, P.act_rows);
    int *rep_uid = at<int>(ws, P.rep_uid), *rep_code = at<int>(ws, P.rep_code);
    const int g_rows = grid_for(ctx, R, 8, 16);

    // forward, keeping x_l and the codes
    VQ_STAGE(S_CONFIG, 5, launch_configs(ch, 0.f, 0, at<int>(ws, P.cnt), at<float>(ws, P.diag),
                                         at<int>(ws, P.cfg_off), at<int>(ws, P.cfg_sample), at<int>(ws, P.cfg_i),
                                         at<int>(ws, P.cfg_j), at<int>(ws, P.cfg_row), at<int>(ws, P.row_cfg),
                                         ctx->status, st, grid_for(ctx, S, 1, 8)));
    VQ_STAGE(S_ACTIVE, 3, launch_active_rows(ch, 0, at<int>(ws, P.act_cnt), at<int>(ws, P.act_off), act, ctx->stats,
                                             st, grid_for(ctx, S, 8, 16)));
    VQ_STAGE(S_EMBED, 1, launch_embed(ch, ctx->tok_emb, ctx->pos_emb, 0, X(0), uid, st, g_rows));
    __nv_bfloat16* S16 = tcb ? at<__nv_bfloat16>(ws, P.s16) : nullptr;  // split planes of one activation
    __nv_bfloat16* TW = tcb ? at<__nv_bfloat16>(ws, P.tw) : nullptr;    // transposed split planes
    const long long Kp = ((long long)R + 63) / 64 * 64;                  // row count rounded to the K step
    for (int l = 0; l < Ly; ++l) {
        const LayerW& w = ctx->lw[l];
        if (tcb) {
            VQ_STAGE(S_LN1, 1, launch_layernorm(X(l), counters, CNT_R, w.ln1_g, w.ln1_b, d, A1, S16, st, g_rows,
                                                (size_t)R * d));
            VQ_STAGE(S_QKV, 1, launch_gemm_tc(S16, R, w.tm_wqkv, w.b_qkv, nullptr, QKV, counters, CNT_R, 3 * d, d, 3,
                                              ctx->status, st, sms, ctx->bn[0], true));
        } else {
            VQ_STAGE(S_LN1, 1, launch_layernorm(X(l), counters, CNT_R, w.ln1_g, w.ln1_b, d, A1, nullptr, st, g_rows));
            VQ_STAGE(S_QKV, 1, launch_sgemm(A1, w.w_qkv, w.b_qkv, nullptr, QKV, counters, CNT_R, R, 3 * d, d, EPI_BIAS,
                                            st, sms));
        }
        VQ_STAGE(S_ATTN, 1, launch_attention_f32(ch, uid, QKV, Oatt, 0, st, grid_for(ctx, (long long)S * H, 1, 8)));
        VQ_STAGE(S_VQ, 1, launch_vq_argmin(Oatt, counters, act, w.codebook, w.cnorm, K, d, code(l),
                                           ctx->stats + ST_NEAR_TIES, R, st, sms));
        VQ_STAGE(S_DEDUPE, 1, launch_dedupe(ch, uid, code(l), CNT_U0 + l + 1, R, nullptr, nullptr, 0, uid_b, rep_uid,
                                            rep_code, 0, ctx->status, st, sms));
        if (tcb) {  // MLP hidden rows as split planes [2R][4d] in the H1 buffer
            __nv_bfloat16* H16 = reinterpret_cast<__nv_bfloat16*>(H1);
            VQ_STAGE(S_POSTLN, 1, launch_residual_vq_ln(X(l), rep_uid, rep_code, w.T, counters, CNT_R, w.ln2_g, w.ln2_b,
                                                        d, Y, nullptr, S16, st, g_rows, 1, K, 0, (size_t)R * d));
            VQ_STAGE(S_MLP1, 1, launch_gemm_tc(S16, R, w.tm_w1, w.b_1, nullptr, H16, counters, CNT_R, 4 * d, d, 1,
                                               ctx->status, st, sms, ctx->bn[1], true));
            VQ_STAGE(S_MLP2, 1, launch_gemm_tc(H16, R, w.tm_w2, w.b_2, Y, X(l + 1), counters, CNT_R, d, 4 * d, 2,
                                               ctx->status, st, sms, ctx->bn[2], true));
        } else {
            VQ_STAGE(S_POSTLN, 1, launch_residual_vq_ln(X(l), rep_uid, rep_code, w.T, counters, CNT_R, w.ln2_g, w.ln2_b,
                                                        d, Y, A2, nullptr, st, g_rows));
            VQ_STAGE(S_MLP1, 1, launch_sgemm(A2, w.w_1, w.b_1, nullptr, G4, counters, CNT_R, R, 4 * d, d,
                                             EPI_BIAS_GELU, st, sms));
            VQ_STAGE(S_MLP2, 1, launch_sgemm(G4, w.w_2, w.b_2, Y, X(l + 1), counters, CNT_R, R, d, 4 * d,
                                             EPI_BIAS_RESID, st, sms));
        }
    }

    StageScope s_bwd(ctx, S_BACKWARD, 0, st);
    auto gg = [&](bool ta, bool tb, const float* A, const float* B, float* C, int M, int Nn, int Kk, int lda, int ldb,
                  int ldc, long long sA, long long sB, long long sC, int batch, int acc) {
        StageScope sc(ctx, S_BWD_GEMM, 1, st);
        return launch_gemm_gen(ta, tb, A, B, C, M, Nn, Kk, lda, ldb, ldc, sA, sB, sC, batch, acc, st, sms);
    };
    float* colpart = at<float>(ws, P.colpart);
    float* kpart = tcb ? at<float>(ws, P.kpart) : nullptr;
    auto colsum = [&](const float* Xm, int ncol, size_t off) {
        StageScope sc(ctx, S_BWD_ROWS, 1, st);
        return launch_colsum(Xm, R, G, ncol, OUT + off, ostride, 1, st, cap, colpart, kColParts);
    };
    // split-operand tensor-core contractions (tcb): C[R][Nn] = A[R][kdim] W^T with W's split planes
    // as the B operand (map tmW, Nn rows) ...
    auto gx = [&](const float* A, int kdim, const CUtensorMap& tmW, int Nn, float* C) -> cudaError_t {
        StageScope sc(ctx, S_BWD_GEMM, 2, st);
        cudaError_t e = launch_split_planes(A, R, kdim, S16, R, st, cap);
        if (e != cudaSuccess) return e;
        return launch_gemm_tc(S16, R, tmW, ctx->zeros, nullptr, C, counters, CNT_R, Nn, kdim, 3, ctx->status, st, sms,
                              tc_pick_bn(Nn), true);
    };
    // ... and C[in][out] += X^T dY summed over the R rows (the weight gradient): both operands
    // transposed into K-major split planes, the row count padded to the K step with zeros
    auto gw = [&](const float* Xs, int in, int dim_slot, const float* dYs, int out, float* C) -> cudaError_t {
        // few output tiles over a long K (the rows): split K so that every SM takes a share,
        // then add the partials into C in a fixed order
        const long long tiles = (long long)((in + 127) / 128) * (out / tc_pick_bn(out));
        const long long mpad = (in + 127) / 128 * 128;
        int ks = (int)(sms / (tiles > 0 ? tiles : 1));
        if (ks > kSplitK) ks = kSplitK;
        if (ks > 1 && (size_t)ks * mpad * out > (size_t)kSplitK * kSplitKElems) ks = 1;
        StageScope sc(ctx, S_BWD_GEMM, ks > 1 ? 4 : 3, st);
        __nv_bfloat16* XT = TW;                            // [2 in][R]
        __nv_bfloat16* YT = TW + (size_t)2 * in * R;       // [2 out][R]
        cudaError_t e = launch_transpose_bf16(Xs, R, in, XT, st, true);
        if (e == cudaSuccess) e = launch_transpose_bf16(dYs, R, out, YT, st, true);
        CUtensorMap tmY;
        if (e == cudaSuccess) e = make_tmap_bf16_strided(&tmY, YT, 2LL * out, R, R, tc_pick_bn(out));
        if (e != cudaSuccess) return e;
        if (ks > 1) {
            e = launch_gemm_tc(XT, in, tmY, ctx->zeros, nullptr, kpart, ctx->dims, dim_slot, out, (int)Kp, 3,
                               ctx->status, st, sms, tc_pick_bn(out), true, R, ks);
            if (e != cudaSuccess) return e;
            const int KB = (int)(Kp / 64), KBs = (KB + ks - 1) / ks;  // the splits the kernel used
            return launch_splitk_add(kpart, (KB + KBs - 1) / KBs, mpad, in, out, C, st, sms);
        }
        return launch_gemm_tc(XT, in, tmY, ctx->zeros, C, C, ctx->dims, dim_slot, out, (int)Kp, 2, ctx->status, st, sms,
                              tc_pick_bn(out), true, R);
    };
    // head
    ctx->launches += 1;
    VQ_CK(launch_head_bwd(X(Ly), spins, seeds, R, N, d, ctx->lnf_g, ctx->lnf_b, ctx->w_head, ctx->b_head, dX, Af, dlog,
                          dgam, dbet, st, cap));
    VQ_CK(gg(true, false, Af, dlog, OUT + po.wh, d, 2, G, d, 2, 2, (long long)G * d, (long long)G * 2, ostride, ng, 1));
    VQ_CK(colsum(dlog, 2, po.bh));
    VQ_CK(colsum(dgam, d, po.lnf_g));
    VQ_CK(colsum(dbet, d, po.lnf_b));
    for (int l = Ly - 1; l >= 0; --l) {
        const LayerW& w = ctx->lw[l];
        const auto& o = po.l[l];
        // recompute the block internals from x_l
        {
            StageScope sc(ctx, S_BWD_RECOMP, 7, st);
            if (tcb) {
                VQ_CK(launch_layernorm(X(l), counters, CNT_R, w.ln1_g, w.ln1_b, d, A1, S16, st, g_rows, (size_t)R * d));
                VQ_CK(launch_gemm_tc(S16, R, w.tm_wqkv, w.b_qkv, nullptr, QKV, counters, CNT_R, 3 * d, d, 3,
                                     ctx->status, st, sms, ctx->bn[0], true));
            } else {
                VQ_CK(launch_layernorm(X(l), counters, CNT_R, w.ln1_g, w.ln1_b, d, A1, nullptr, st, g_rows));
                VQ_CK(launch_sgemm(A1, w.w_qkv, w.b_qkv, nullptr, QKV, counters, CNT_R, R, 3 * d, d, EPI_BIAS, st, sms));
            }
            // the softmax statistics of every row and head go to the attention backward
            VQ_CK(launch_attention_f32(ch, uid, QKV, Oatt, 0, st, grid_for(ctx, (long long)S * H, 1, 8), nullptr, 0,
                                       at<float2>(ws, P.stat)));
            VQ_CK(launch_quant_residual(X(l), code(l), w.T, w.codebook, R, d, Y, V, st, cap));
            if (tcb) {
                VQ_CK(launch_layernorm(Y, counters, CNT_R, w.ln2_g, w.ln2_b, d, A2, S16, st, g_rows, (size_t)R * d));
                VQ_CK(launch_gemm_tc(S16, R, w.tm_w1, w.b_1, nullptr, H1, counters, CNT_R, 4 * d, d, 3, ctx->status, st,
                                     sms, ctx->bn[1], true));
            } else {
                VQ_CK(launch_layernorm(Y, counters, CNT_R, w.ln2_g, w.ln2_b, d, A2, nullptr, st, g_rows));
                VQ_CK(launch_sgemm(A2, w.w_1, w.b_1, nullptr, H1, counters, CNT_R, R, 4 * d, d, EPI_BIAS, st, sms));
            }
            VQ_CK(launch_gelu_fwd(H1, G4, (size_t)R * 4 * d, st, cap));
        }
        // MLP: x' = y + GELU(LN2(y) W1 + b1) W2 + b2, dX holds d/dx'
        if (tcb) VQ_CK(gw(G4, 4 * d, 2, dX, d, OUT + o.w2));
        else VQ_CK(gg(true, false, G4, dX, OUT + o.w2, 4 * d, d, G, 4 * d, d, d, (long long)G * 4 * d, (long long)G * d,
                      ostride, ng, 1));
        VQ_CK(colsum(dX, d, o.b2));
        if (tcb) VQ_CK(gx(dX, d, w.tm_w2_s, 4 * d, dG4));
        else VQ_CK(gg(false, true, dX, w.w_2, dG4, R, 4 * d, d, d, d, 4 * d, 0, 0, 0, 1, 0));
        ctx->launches += 1;
        VQ_CK(launch_gelu_bwd(H1, dG4, (size_t)R * 4 * d, st, cap));
        if (tcb) VQ_CK(gw(A2, d, 0, dG4, 4 * d, OUT + o.w1));
        else VQ_CK(gg(true, false, A2, dG4, OUT + o.w1, d, 4 * d, G, d, 4 * d, 4 * d, (long long)G * d,
                      (long long)G * 4 * d, ostride, ng, 1));
        VQ_CK(colsum(dG4, 4 * d, o.b1));
        if (tcb) VQ_CK(gx(dG4, 4 * d, w.tm_w1_s, d, dA));
        else VQ_CK(gg(false, true, dG4, w.w_1, dA, R, d, 4 * d, 4 * d, 4 * d, d, 0, 0, 0, 1, 0));
        VQ_CK(cudaMemcpyAsync(dY, dX, (size_t)R * d * sizeof(float), cudaMemcpyDeviceToDevice, st));
        ctx->launches += 1;
        VQ_CK(launch_ln_bwd(Y, dA, w.ln2_g, R, d, dY, 1, dgam, dbet, st, cap));
        VQ_CK(colsum(dgam, d, o.ln2_g));
        VQ_CK(colsum(dbet, d, o.ln2_b));
        // y = x + V W_o + b_o
        if (tcb) {
            VQ_CK(gx(dY, d, w.tm_wo_s, d, dV));
            VQ_CK(gw(V, d, 0, dY, d, OUT + o.wo));
        } else {
            VQ_CK(gg(false, true, dY, w.w_o, dV, R, d, d, d, d, d, 0, 0, 0, 1, 0));
            VQ_CK(gg(true, false, V, dY, OUT + o.wo, d, d, G, d, d, d, (long long)G * d, (long long)G * d, ostride, ng,
                     1));
        }
        VQ_CK(colsum(dY, d, o.bo));
        // straight-through quantizer (Eq. st)
        if (tcb) {
            VQ_CK(gx(Oatt, d, w.tm_cb_s, K, OW));
            VQ_CK(gx(dV, d, w.tm_cb_s, K, DG));
        } else {
            VQ_CK(gg(false, true, Oatt, w.codebook, OW, R, K, d, d, d, K, 0, 0, 0, 1, 0));
            VQ_CK(gg(false, true, dV, w.codebook, DG, R, K, d, d, d, K, 0, 0, 0, 1, 0));
        }
        ctx->launches += 1;
        VQ_CK(launch_st_rows(OW, DG, Oatt, w.cnorm, R, K, d, alpha, arow, st, cap));
        if (tcb) VQ_CK(gx(alpha, K, w.tm_cbT_s, d, dO));
        else VQ_CK(gg(false, false, alpha, w.codebook, dO, R, d, K, K, d, d, 0, 0, 0, 1, 0));
        ctx->launches += 1;
        VQ_CK(launch_st_do(Oatt, arow, R, d, dO, st, cap));
        if (tcb) VQ_CK(gw(alpha, K, 3, Oatt, d, OUT + o.cb));
        else VQ_CK(gg(true, false, alpha, Oatt, OUT + o.cb, K, d, G, K, d, d, (long long)G * K, (long long)G * d,
                      ostride, ng, 1));
        ctx->launches += 3;
        VQ_CK(launch_colsum(alpha, R, G, K, csumK, K, 0, st, cap, colpart, kColParts));
        VQ_CK(launch_sub_scaled_rows(OUT + o.cb, csumK, w.codebook, K, d, ng, ostride, st, cap));
        VQ_CK(launch_onehot(code(l), R, K, onehot, st, cap));
        if (tcb) VQ_CK(gw(onehot, K, 3, dV, d, OUT + o.cb));
        else VQ_CK(gg(true, false, onehot, dV, OUT + o.cb, K, d, G, K, d, d, (long long)G * K, (long long)G * d,
                      ostride, ng, 1));
        // attention
        {
            StageScope sc(ctx, S_BWD_ATTN, 2, st);
            VQ_CK(launch_attention_bwd(QKV, Oatt, dO, at<float2>(ws, P.stat), S, N, d, H, dQKV,
                                       at<float>(ws, P.stat) + 2 * (size_t)R * H, st, cap));
        }
        // qkv = LN1(x) W_qkv + b_qkv
        if (tcb) VQ_CK(gw(A1, d, 0, dQKV, 3 * d, OUT + o.wqkv));
        else VQ_CK(gg(true, false, A1, dQKV, OUT + o.wqkv, d, 3 * d, G, d, 3 * d, 3 * d, (long long)G * d,
                      (long long)G * 3 * d, ostride, ng, 1));
        VQ_CK(colsum(dQKV, 3 * d, o.bqkv));
        if (tcb) VQ_CK(gx(dQKV, 3 * d, w.tm_wqkv_s, d, dA));
        else VQ_CK(gg(false, true, dQKV, w.w_qkv, dA, R, d, 3 * d, 3 * d, 3 * d, d, 0, 0, 0, 1, 0));
        VQ_CK(cudaMemcpyAsync(dX, dY, (size_t)R * d * sizeof(float), cudaMemcpyDeviceToDevice, st));
        ctx->launches += 1;
        VQ_CK(launch_ln_bwd(X(l), dA, w.ln1_g, R, d, dX, 1, dgam, dbet, st, cap));
        VQ_CK(colsum(dgam, d, o.ln1_g));
        VQ_CK(colsum(dbet, d, o.ln1_b));
    }
    ctx->launches += 1;
    VQ_CK(launch_embed_bwd(dX, spins, S, N, d, G / N, OUT + po.tok, OUT + po.pos, ostride, 1, st, cap));
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

size_t vqnqs_num_params_arch(int n_max, int layers, int d_model, int K, int half_block, int token_group) {
    if (!(token_group == 1 || token_group == 2 || token_group == 4) || n_max % token_group) return 0;
    const size_t base = vqnqs_num_params(n_max, layers, d_model, K);
    if (!base) return 0;
    const size_t d = d_model, V = (size_t)1 << token_group;
    // token embeddings V + 1 rows (3 for single spins), n_max / G positions, a V-way head
    size_t n = base - 3 * d - (size_t)n_max * d - 2 * d - 2 + (V + 1) * d + (size_t)(n_max / token_group) * d + V * d + V;
    return half_block ? n + 2 * d + 3 * d * d + 3 * d + d * d + d : n;
}

namespace {
// Shared by vqnqs_create (L x L Heisenberg lattice) and vqnqs_create_tfim (N-site chain).
int create_ctx(int model, int L, int N, int periodic, double J, double Gamma, int layers, int d_model, int heads,
               int K, const float* weights, vqnqs_ctx** out, int vq_heads = 1, int half_block = 0,
               int token_group = 1) {
    if (!out) return VQNQS_ERR_ARG;
    *out = nullptr;
    if (N < 2 || N > 512 || layers < 1 || layers > VQNQS_MAX_LAYERS || d_model < 32 || d_model % 32 ||
        d_model > 1024 || heads < 1 || d_model % heads || K < 1 || K > 65535 || !weights)
        return VQNQS_ERR_ARG;
    int vq_bits = 1;
    while ((1 << vq_bits) < K) ++vq_bits;
    // heads of vq_bits each: 32 / vq_bits per code word, at most two words
    if (vq_heads < 1 || vq_heads > 8 || d_model % vq_heads || (d_model / vq_heads) % 8 ||
        (vq_heads > 1 && vq_heads > 2 * (32 / vq_bits)))
        return VQNQS_ERR_ARG;
    if (!(token_group == 1 || token_group == 2 || token_group == 4) || N % token_group) return VQNQS_ERR_ARG;
    const int dh = d_model / heads;
    if (!(dh == 8 || dh == 16 || dh == 32)) return VQNQS_ERR_ARG;
    vqnqs_ctx* ctx = new vqnqs_ctx();
    ctx->model = model;
    ctx->L = L; ctx->N = N; ctx->periodic = periodic ? 1 : 0; ctx->J = J; ctx->Gamma = Gamma;
    ctx->layers = layers; ctx->d = d_model; ctx->heads = heads; ctx->K = K;
    ctx->vq_heads = vq_heads; ctx->vq_bits = vq_heads > 1 ? vq_bits : 0;
    ctx->vq_words = vq_heads > 1 && vq_heads > 32 / vq_bits ? 2 : 1;
    ctx->half_block = half_block ? 1 : 0;
    ctx->G = token_group;
    ctx->P = N / token_group;
    auto bail = [&](int code) { vqnqs_destroy(ctx); return code; };
    if (cudaGetDevice(&ctx->device) != cudaSuccess) return bail(VQNQS_ERR_CUDA);
    if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess)
        return bail(VQNQS_ERR_CUDA);
    ctx->nparams = vqnqs_num_params_arch(ctx->N, layers, d_model, K, ctx->half_block, ctx->G);
    auto dalloc = [&](size_t bytes) -> void* {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        ctx->owned.push_back(p);
        return p;
    };
    ctx->blob = static_cast<float*>(dalloc(ctx->nparams * sizeof(float)));
    std::vector<int> bonds, all;
    if (model == MODEL_TFIM_CHAIN) {  // (p, p+1), and (N-1, 0) when periodic; one bond table (index 0)
        for (int q = 0; q + 1 < N; ++q) { bonds.push_back(q); bonds.push_back(q + 1); }
        if (ctx->periodic && N > 2) { bonds.push_back(N - 1); bonds.push_back(0); }
        all = bonds;
        ctx->side_bond_off.assign(1, 0);
        ctx->side_nb.assign(1, (int)bonds.size() / 2);
    } else {  // the lattice's bonds, and those of every side 2 .. L for ragged batches
        bonds = make_bonds(L, ctx->periodic);
        ctx->side_bond_off.assign(L + 1, 0);
        ctx->side_nb.assign(L + 1, 0);
        for (int s = 2; s <= L; ++s) {
            std::vector<int> b = make_bonds(s, ctx->periodic);
            ctx->side_bond_off[s] = (int)all.size() / 2;
            ctx->side_nb[s] = (int)b.size() / 2;
            all.insert(all.end(), b.begin(), b.end());
        }
    }
    ctx->nb = (int)bonds.size() / 2;
    ctx->max_conn = model == MODEL_TFIM_CHAIN ? N : ctx->nb;
    ctx->bonds = static_cast<int*>(dalloc(bonds.size() * sizeof(int)));
    ctx->bonds_all = static_cast<int*>(dalloc(all.size() * sizeof(int)));
    ctx->status = static_cast<int*>(dalloc(sizeof(int)));
    ctx->stats = static_cast<long long*>(dalloc(ST_SLOTS * sizeof(long long)));
    ctx->lw.resize(layers);
    const size_t d = d_model;
    // the backward's contractions on the tensor cores: shapes the split GEMM takes, one quantizer
    // head, no half-block, single-spin tokens
    ctx->bwd_tc = d_model % 64 == 0 && K % 64 == 0 && vq_heads == 1 && !half_block && token_group == 1;
    if (ctx->bwd_tc) {
        const int dims[4] = {d_model, 3 * d_model, 4 * d_model, K};
        ctx->dims = static_cast<int*>(dalloc(sizeof(dims)));
        const size_t nz = (size_t)std::max(4 * d_model, K);
        ctx->zeros = static_cast<float*>(dalloc(nz * sizeof(float)));
        if (!ctx->dims || !ctx->zeros) return bail(VQNQS_ERR_OOM);
        if (cudaMemcpy(ctx->dims, dims, sizeof(dims), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(ctx->zeros, 0, nz * sizeof(float)) != cudaSuccess)
            return bail(VQNQS_ERR_CUDA);
    }
    for (int l = 0; l < layers; ++l) {
        LayerW& w = ctx->lw[l];
        w.T = static_cast<float*>(dalloc((size_t)vq_heads * K * d * sizeof(float)));
        w.cnorm = static_cast<float*>(dalloc((size_t)vq_heads * K * sizeof(float)));
        // BF16 transposes with their split lo planes: [2 out][in]
        w.wqkv_t = static_cast<__nv_bfloat16*>(dalloc(2 * 3 * d * d * sizeof(__nv_bfloat16)));
        w.w1_t = static_cast<__nv_bfloat16*>(dalloc(2 * 4 * d * d * sizeof(__nv_bfloat16)));
        w.w2_t = static_cast<__nv_bfloat16*>(dalloc(2 * 4 * d * d * sizeof(__nv_bfloat16)));
        w.cb_hi = static_cast<float*>(dalloc((size_t)K * d * sizeof(float)));
        w.cb_lo = static_cast<float*>(dalloc((size_t)K * d * sizeof(float)));
        w.wd = static_cast<float*>(dalloc((size_t)vq_heads * K * K * sizeof(float)));  // one table per head
        if (!w.T || !w.cnorm || !w.wqkv_t || !w.w1_t || !w.w2_t || !w.cb_hi || !w.cb_lo || !w.wd)
            return bail(VQNQS_ERR_OOM);
        if (ctx->bwd_tc) {
            const size_t b2 = 2 * sizeof(__nv_bfloat16);
            w.wqkv_s = static_cast<__nv_bfloat16*>(dalloc(3 * d * d * b2));
            w.w1_s = static_cast<__nv_bfloat16*>(dalloc(4 * d * d * b2));
            w.w2_s = static_cast<__nv_bfloat16*>(dalloc(4 * d * d * b2));
            w.wo_s = static_cast<__nv_bfloat16*>(dalloc(d * d * b2));
            w.cb_s = static_cast<__nv_bfloat16*>(dalloc((size_t)K * d * b2));
            w.cbT_s = static_cast<__nv_bfloat16*>(dalloc((size_t)K * d * b2));
            if (!w.wqkv_s || !w.w1_s || !w.w2_s || !w.wo_s || !w.cb_s || !w.cbT_s) return bail(VQNQS_ERR_OOM);
        }
    }
    if (ctx->half_block) {
        ctx->hw.wqkv_t = static_cast<__nv_bfloat16*>(dalloc(3 * d * d * sizeof(__nv_bfloat16)));
        ctx->hw.wo_t = static_cast<__nv_bfloat16*>(dalloc(d * d * sizeof(__nv_bfloat16)));
        if (!ctx->hw.wqkv_t || !ctx->hw.wo_t) return bail(VQNQS_ERR_OOM);
    }
    if (!ctx->blob || !ctx->bonds || !ctx->status || !ctx->stats) return bail(VQNQS_ERR_OOM);
    if (!ctx->bonds_all ||
        cudaMemcpy(ctx->bonds_all, all.data(), all.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ctx->bonds, bonds.data(), bonds.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ctx->status, 0, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->stats, 0, ST_SLOTS * sizeof(long long)) != cudaSuccess)
        return bail(VQNQS_ERR_CUDA);
    ctx->gemm_m = static_cast<int*>(dalloc(sizeof(int)));
    ctx->assign_counters = static_cast<int*>(dalloc(CNT_SLOTS * sizeof(int)));
    ctx->assign_rows = static_cast<int*>(dalloc((size_t)ctx->assign_rows_cap * sizeof(int)));
    ctx->lp_scratch = static_cast<float*>(dalloc((size_t)ctx->lp_scratch_cap * sizeof(float)));
    if (!ctx->gemm_m || !ctx->assign_counters || !ctx->assign_rows || !ctx->lp_scratch) return bail(VQNQS_ERR_OOM);
    bind_weights(ctx);
    int rc = vqnqs_set_weights(ctx, weights, 0, nullptr);
    if (rc != VQNQS_OK) return bail(rc);
    if (vq_heads == 1 && vq_tc_supported(K, d_model)) {
        for (int l = 0; l < layers; ++l) {
            LayerW& w = ctx->lw[l];
            if (make_tmap_codebook(&w.tm_cb_hi, w.cb_hi, K, d_model) != cudaSuccess ||
                make_tmap_codebook(&w.tm_cb_lo, w.cb_lo, K, d_model) != cudaSuccess)
                return bail(VQNQS_ERR_CUDA);
        }
    }
    if (d_model % 64 == 0) {
        ctx->bn[0] = tc_pick_bn(3 * d_model);
        ctx->bn[1] = tc_pick_bn(4 * d_model);
        ctx->bn[2] = tc_pick_bn(d_model);
        if (build_weight_tmaps(ctx) != VQNQS_OK) return bail(VQNQS_ERR_CUDA);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(VQNQS_ERR_CUDA);
    *out = ctx;
    return VQNQS_OK;
}
}  // namespace

int vqnqs_create(int L, int periodic, double J, int layers, int d_model, int heads, int K, const float* weights,
                 vqnqs_ctx** out) {
    if (L < 2 || L * L > 512) {
        if (out) *out = nullptr;
        return VQNQS_ERR_ARG;
    }
    return create_ctx(MODEL_HEISENBERG, L, L * L, periodic, J, 0.0, layers, d_model, heads, K, weights, out);
}

int vqnqs_create_tfim(int N, int periodic, double J, double Gamma, int layers, int d_model, int heads, int K,
                      const float* weights, vqnqs_ctx** out) {
    return create_ctx(MODEL_TFIM_CHAIN, 0, N, periodic, J, Gamma, layers, d_model, heads, K, weights, out);
}

int vqnqs_create_arch(int L, int periodic, double J, int layers, int d_model, int heads, int K, int vq_heads,
                      int half_block, int token_group, const float* weights, vqnqs_ctx** out) {
    if (L < 2 || L * L > 512) {
        if (out) *out = nullptr;
        return VQNQS_ERR_ARG;
    }
    return create_ctx(MODEL_HEISENBERG, L, L * L, periodic, J, 0.0, layers, d_model, heads, K, weights, out,
                      vq_heads, half_block, token_group);
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

int vqnqs_local_energy_ragged(vqnqs_ctx* ctx, int n_groups, const int* L_g, const int* B_g, const uint8_t* spins,
                              float* e_loc, double* mean_var, int flags, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (ctx->model != MODEL_HEISENBERG) return fail(ctx, VQNQS_ERR_ARG, "ragged: square-lattice contexts only");
    if (ctx->G > 1) return fail(ctx, VQNQS_ERR_ARG, "ragged: one spin per token");
    if (n_groups < 1 || n_groups > MAX_GROUPS || !L_g || !B_g)
        return fail(ctx, VQNQS_ERR_ARG, "ragged: need 1..8 groups and host arrays L_g, B_g");
    if (int rc = check_flags(ctx, flags)) return rc;
    Groups g;
    std::memset(&g, 0, sizeof(g));
    g.n = n_groups;
    long long spin_off = 0;
    int total = 0;
    for (int i = 0; i < n_groups; ++i) {
        if (L_g[i] < 2 || L_g[i] > ctx->L || B_g[i] < 0)
            return fail(ctx, VQNQS_ERR_ARG, "ragged: lattice sides must be 2 .. L of the context, B_g >= 0");
        g.first[i] = total;
        g.N[i] = L_g[i] * L_g[i];
        g.nb[i] = ctx->side_nb[L_g[i]];
        g.bond_off[i] = ctx->side_bond_off[L_g[i]];
        g.spin_off[i] = spin_off;
        spin_off += (long long)B_g[i] * g.N[i];
        total += B_g[i];
    }
    g.first[n_groups] = total;
    if (total == 0) return VQNQS_OK;
    if (!spins || !e_loc || !ws) return fail(ctx, VQNQS_ERR_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(ctx, VQNQS_ERR_ARG, "workspace must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // budgets: the largest uniform chunk of the context's lattice that fits, with
    // per-sample arrays sized for as many samples as configurations
    int S = fit_chunk(ctx, 65536, ws_bytes, true);
    Plan P;
    for (; S > 0; --S) {
        const Plan u = make_plan(ctx, S, true);
        P = make_plan_budget(ctx, (int)u.Cmax, u.Cmax, u.Rmax);
        if (P.total <= ws_bytes) break;
    }
    if (S == 0) return fail(ctx, VQNQS_ERR_WORKSPACE, "workspace smaller than the one-sample minimum");
    // partition the samples, in order, into chunks that respect the budgets
    int s0 = 0, grp = 0;
    while (s0 < total) {
        long long C = 0, R = 0;
        int s1 = s0;
        while (s1 < total) {
            while (s1 >= g.first[grp + 1]) ++grp;
            const long long cs = 1 + g.nb[grp], rs = cs * g.N[grp];
            long long k = g.first[grp + 1] - s1;
            k = std::min(k, (P.Cmax - C) / cs);
            k = std::min(k, (P.Rmax - R) / rs);
            k = std::min(k, (long long)P.S - (s1 - s0));
            if (k <= 0) break;
            s1 += (int)k;
            C += k * cs;
            R += k * rs;
        }
        if (s1 == s0) return fail(ctx, VQNQS_ERR_INTERNAL, "ragged: empty chunk");
        const int rc = run_chunk(ctx, P, ws, spins, g, s0, s1 - s0, true, flags, e_loc + s0, nullptr, st);
        if (rc != VQNQS_OK) return rc;
        s0 = s1;
        grp = 0;
    }
    if (mean_var) VQ_STAGE(S_MEANVAR, 1, launch_mean_var(e_loc, total, mean_var, st));
    return VQNQS_OK;
}

int vqnqs_codes(vqnqs_ctx* ctx, int B, const uint8_t* spins, int* codes, float* log_psi, int flags, void* ws,
                size_t ws_bytes, void* stream) {
    if (ctx && B > 0 && !codes) return fail(ctx, VQNQS_ERR_ARG, "codes is NULL");
    if (!log_psi && ctx && B > 0) {
        // log psi goes to the workspace-free scratch of the context when not wanted
        if (ctx->lp_scratch_cap < B) return fail(ctx, VQNQS_ERR_ARG, "codes: pass log_psi for B > 65536");
        log_psi = ctx->lp_scratch;
    }
    return run(ctx, B, spins, nullptr, nullptr, log_psi, flags, ws, ws_bytes, stream, false, codes);
}

int vqnqs_local_energy(vqnqs_ctx* ctx, int B, const uint8_t* spins, float* e_loc, double* mean_var, float* log_psi,
                       int flags, void* ws, size_t ws_bytes, void* stream) {
    return run(ctx, B, spins, e_loc, mean_var, log_psi, flags, ws, ws_bytes, stream, true);
}

int vqnqs_local_energy_codes(vqnqs_ctx* ctx, int B, const uint8_t* spins, float* e_loc, int* codes, int flags,
                             void* ws, size_t ws_bytes, void* stream) {
    if (ctx && B > 0 && !codes) return fail(ctx, VQNQS_ERR_ARG, "codes is NULL");
    return run(ctx, B, spins, e_loc, nullptr, nullptr, flags, ws, ws_bytes, stream, true, nullptr, codes);
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
    out->active_rows = st[ST_ACTIVE];
    out->attn_pairs = st[ST_PAIRS];
    out->inc_base_rows = st[ST_INC_BASE];
    out->inc_patched_rows = st[ST_INC_PATCHED];
    out->inc_certified_rows = st[ST_INC_CERT];
    out->inc_full_rows = st[ST_INC_FULL];
    out->inc_searched_rows = st[ST_INC_VQ];
    out->inc_patch_pairs = st[ST_INC_PPAIRS];
    out->inc_full_pairs = st[ST_INC_FPAIRS];
    out->inc_whole_pairs = st[ST_INC_WPAIRS];
    // analytic FLOPs, 2 per multiply-add
    const double d = ctx->d, K = ctx->K, N = ctx->P, Ly = ctx->layers;
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

namespace {
// The tensor-core GEMM on its own; split: A [2M][K], Bt [2N][K] and a BF16 C [2M][N] hold lo planes.
int gemm_entry(vqnqs_ctx* ctx, int M, int N, int K, const void* A, const void* Bt, const float* bias, const float* R,
               void* C, int epilogue, void* stream, bool split) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (M < 0 || N <= 0 || K <= 0 || K % 64 || !tc_pick_bn(N) || epilogue < 0 || epilogue > 4)
        return fail(ctx, VQNQS_ERR_ARG, "gemm: need M >= 0, K % 64 == 0, N % 64 == 0, epilogue 0..4");
    if (!A || !Bt || !bias || !C || (epilogue == 2 && !R)) return fail(ctx, VQNQS_ERR_ARG, "gemm: null pointer");
    auto misaligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; };
    if (misaligned(A) || misaligned(Bt) || misaligned(C) || (R && misaligned(R)))
        return fail(ctx, VQNQS_ERR_ARG, "gemm: pointers must be 16-byte aligned");
    if (M == 0) return VQNQS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (split && M > (1 << 29)) return fail(ctx, VQNQS_ERR_ARG, "gemm: M too large for split planes");
    CUtensorMap tb;
    VQ_CK(make_tmap_bf16(&tb, Bt, split ? 2LL * N : N, K, tc_pick_bn(N)));
    VQ_CK(launch_set_int(ctx->gemm_m, M, st));
    ctx->launches += 2;
    VQ_CK(launch_gemm_tc(static_cast<const __nv_bfloat16*>(A), M, tb, bias, R, C, ctx->gemm_m, 0, N, K, epilogue,
                         ctx->status, st, ctx->num_sms, 0, split));
    return VQNQS_OK;
}
}  // namespace

int vqnqs_gemm_bf16(vqnqs_ctx* ctx, int M, int N, int K, const void* A, const void* Bt, const float* bias,
                    const float* R, void* C, int epilogue, void* stream) {
    return gemm_entry(ctx, M, N, K, A, Bt, bias, R, C, epilogue, stream, false);
}

int vqnqs_gemm_bf16_split(vqnqs_ctx* ctx, int M, int N, int K, const void* A2, const void* Bt2, const float* bias,
                          const float* R, void* C, int epilogue, void* stream) {
    return gemm_entry(ctx, M, N, K, A2, Bt2, bias, R, C, epilogue, stream, true);
}

size_t vqnqs_grad_workspace_bytes(const vqnqs_ctx* ctx, int B, int chunk_samples) {
    if (!ctx || B < 0) return 0;
    int S = chunk_samples > 0 ? chunk_samples : grad_default_chunk(ctx);
    if (B > 0 && S > B) S = B;
    return make_grad_plan(ctx, S, B).total;
}

int vqnqs_grad_log_psi(vqnqs_ctx* ctx, int B, const uint8_t* spins, const float* seeds, const float* e_loc, float* O,
                       float* grad, int flags, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (ctx->vq_heads > 1) return fail(ctx, VQNQS_ERR_ARG, "grad_log_psi: one quantizer head only");
    if (ctx->half_block) return fail(ctx, VQNQS_ERR_ARG, "grad_log_psi: no final half-block");
    if (ctx->G > 1) return fail(ctx, VQNQS_ERR_ARG, "grad_log_psi: one spin per token");
    if (B < 0) return fail(ctx, VQNQS_ERR_ARG, "B must be >= 0");
    if (flags & ~(VQNQS_REUSE | VQNQS_BF16 | VQNQS_INCREMENTAL | VQNQS_BF16_SPLIT))
        return fail(ctx, VQNQS_ERR_ARG, "unknown flag bits");
    if (flags & VQNQS_INCREMENTAL) {
        if (!(flags & VQNQS_REUSE)) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL needs VQNQS_REUSE");
        if (ctx->vq_heads > 1) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL needs one quantizer head");
        if (ctx->half_block) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL: no final half-block");
        if (ctx->G > 1) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_INCREMENTAL: one spin per token");
        if (!incremental_supported(ctx->d, ctx->heads))
            return fail(ctx, VQNQS_ERR_ARG,
                        "VQNQS_INCREMENTAL needs d_model in {32, 64, 128, 256, 512} and d_model/heads in {16, 32}, "
                        "a multiple of d_model/32");
    }
    if (seeds && e_loc) return fail(ctx, VQNQS_ERR_ARG, "give seeds or e_loc, not both");
    if (!O && !grad) return fail(ctx, VQNQS_ERR_ARG, "nothing to compute: O and grad are NULL");
    if (B == 0) return VQNQS_OK;
    if (!spins || !ws) return fail(ctx, VQNQS_ERR_ARG, "null pointer");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(ctx, VQNQS_ERR_ARG, "workspace must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // largest chunk that fits
    int lo = 0, hi = B < 65536 ? B : 65536;
    while (lo < hi) {
        int mid = lo + (hi - lo + 1) / 2;
        if (make_grad_plan(ctx, mid, B).total <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    if (lo == 0) return fail(ctx, VQNQS_ERR_WORKSPACE, "workspace smaller than the one-sample minimum");
    const GradPlan P = make_grad_plan(ctx, lo, B);
    const long long Pn = (long long)ctx->nparams;
    float* sd = at<float>(ws, P.seeds);
    if (e_loc) {
        ctx->launches += 1;
        VQ_CK(launch_seeds_from_eloc(e_loc, B, sd, st));
    } else if (seeds && !O) {
        VQ_CK(cudaMemcpyAsync(sd, seeds, (size_t)B * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    const bool weighted = (e_loc || seeds) && !O;
    if (O) VQ_CK(cudaMemsetAsync(O, 0, (size_t)B * Pn * sizeof(float), st));
    if (grad) VQ_CK(cudaMemsetAsync(grad, 0, (size_t)Pn * sizeof(float), st));
    for (int s0 = 0; s0 < B; s0 += lo) {
        const int S = (B - s0) < lo ? (B - s0) : lo;
        const uint8_t* sp = spins + (size_t)s0 * ctx->N;
        int rc;
        if (O) rc = grad_chunk(ctx, P, ws, sp, S, nullptr, O + (size_t)s0 * Pn, ctx->N, Pn, st, flags);
        else rc = grad_chunk(ctx, P, ws, sp, S, weighted ? sd + s0 : nullptr, grad, S * ctx->N, 0, st, flags);
        if (rc != VQNQS_OK) return rc;
    }
    if (O && grad) {  // grad = sum_b w_b O_b
        if (e_loc || seeds) {
            const float* w = e_loc ? sd : seeds;
            ctx->launches += 1;
            VQ_CK(launch_gemm_gen(false, false, w, O, grad, 1, (int)Pn, B, B, (int)Pn, (int)Pn, 0, 0, 0, 1, 0, st,
                                  ctx->num_sms));
        } else {
            ctx->launches += 1;
            VQ_CK(launch_colsum(O, B, B, (int)Pn, grad, 0, 0, st, ctx->num_sms * 16));
        }
    }
    return VQNQS_OK;
}

size_t vqnqs_energy_grad_partials_workspace_bytes(const vqnqs_ctx* ctx, int B, int chunk_samples) {
    if (!ctx || B < 0) return 0;
    return align256(2 * ctx->nparams * sizeof(float)) + vqnqs_grad_workspace_bytes(ctx, B, chunk_samples);
}

int vqnqs_energy_grad_partials(vqnqs_ctx* ctx, int B, const uint8_t* spins, const float* e_loc, double* partials,
                               int flags, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (B < 0 || !partials) return fail(ctx, VQNQS_ERR_ARG, "energy_grad_partials: need B >= 0 and partials");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long Pn = (long long)ctx->nparams;
    if (B == 0) {  // a rank without samples contributes zeros
        VQ_CK(cudaMemsetAsync(partials, 0, (size_t)(2 * Pn + 3) * sizeof(double), st));
        return VQNQS_OK;
    }
    if (!spins || !e_loc || !ws) return fail(ctx, VQNQS_ERR_ARG, "energy_grad_partials: null pointer");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(ctx, VQNQS_ERR_ARG, "workspace must be 256-byte aligned");
    const size_t head = align256(2 * ctx->nparams * sizeof(float));
    if (ws_bytes <= head) return fail(ctx, VQNQS_ERR_WORKSPACE, "energy_grad_partials: workspace too small");
    float* s_eo = static_cast<float*>(ws);
    float* s_o = s_eo + Pn;
    void* gws = static_cast<char*>(ws) + head;
    // sum_b E_b O_b (seeds E) and sum_b O_b (unit seeds): two backward passes
    int rc = vqnqs_grad_log_psi(ctx, B, spins, e_loc, nullptr, nullptr, s_eo, flags, gws, ws_bytes - head, stream);
    if (rc != VQNQS_OK) return rc;
    rc = vqnqs_grad_log_psi(ctx, B, spins, nullptr, nullptr, nullptr, s_o, flags, gws, ws_bytes - head, stream);
    if (rc != VQNQS_OK) return rc;
    ctx->launches += 2;
    VQ_CK(launch_grad_partials(s_eo, s_o, Pn, e_loc, B, partials, st, ctx->num_sms * 8));
    return VQNQS_OK;
}

int vqnqs_energy_grad_combine(vqnqs_ctx* ctx, const double* partials, float* grad, double* mean_var, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (!partials || !grad) return fail(ctx, VQNQS_ERR_ARG, "energy_grad_combine: null pointer");
    ctx->launches += 1;
    VQ_CK(launch_energy_grad_combine(partials, (long long)ctx->nparams, grad, mean_var,
                                     static_cast<cudaStream_t>(stream), ctx->num_sms * 8));
    return VQNQS_OK;
}

int vqnqs_vq_assign(vqnqs_ctx* ctx, int layer, int R, const float* O, int* code, int use_tensor_cores,
                    void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (ctx->vq_heads > 1) return fail(ctx, VQNQS_ERR_ARG, "vq_assign: one quantizer head only");
    if (layer < 0 || layer >= ctx->layers || R < 0) return fail(ctx, VQNQS_ERR_ARG, "vq_assign: bad layer or R");
    if (R > 0 && (!O || !code)) return fail(ctx, VQNQS_ERR_ARG, "vq_assign: null pointer");
    if ((reinterpret_cast<uintptr_t>(O) & 15)) return fail(ctx, VQNQS_ERR_ARG, "vq_assign: O must be 16-byte aligned");
    if (use_tensor_cores && !vq_tc_supported(ctx->K, ctx->d))
        return fail(ctx, VQNQS_ERR_ARG, "vq_assign: tensor-core path needs K % 16 == 0, K <= 512, d % 32 == 0");
    if (R == 0) return VQNQS_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const LayerW& w = ctx->lw[layer];
    // counters: CNT_A / CNT_R = R, rows listed 0 .. R-1 (identity) in the context's scratch
    if (ctx->assign_rows_cap < R) return fail(ctx, VQNQS_ERR_ARG, "vq_assign: R above the context's row capacity");
    ctx->launches += 2;
    VQ_CK(launch_assign_setup(ctx->assign_counters, ctx->assign_rows, R, st));
    if (use_tensor_cores)
        VQ_CK(launch_vq_tc(w.tm_cb_hi, w.tm_cb_lo, O, ctx->assign_counters, ctx->assign_rows, w.cnorm, ctx->K,
                           ctx->d, code, ctx->stats + ST_NEAR_TIES, ctx->status, st, ctx->num_sms, R));
    else
        VQ_CK(launch_vq_argmin(O, ctx->assign_counters, ctx->assign_rows, w.codebook, w.cnorm, ctx->K, ctx->d, code,
                               ctx->stats + ST_NEAR_TIES, R, st, ctx->num_sms));
    return VQNQS_OK;
}

size_t vqnqs_compress_workspace_bytes(int R) {
    if (R < 0) return 0;
    const size_t H = (size_t)1 << compress_hash_bits(R);
    return align256(H * sizeof(unsigned long long)) + align256(H * sizeof(int));
}

int vqnqs_compress_rows(vqnqs_ctx* ctx, int R, const int* uid, const int* code, int* new_id, int* rep_uid,
                        int* rep_code, int* count, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (R < 0) return fail(ctx, VQNQS_ERR_ARG, "compress: R must be >= 0");
    if (!count || (R > 0 && (!uid || !code || !new_id || !rep_uid || !rep_code)))
        return fail(ctx, VQNQS_ERR_ARG, "compress: null pointer");
    const size_t need = vqnqs_compress_workspace_bytes(R);
    if (!ws || ws_bytes < need) return fail(ctx, VQNQS_ERR_WORKSPACE, "compress: workspace too small");
    if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(ctx, VQNQS_ERR_ARG, "workspace must be 256-byte aligned");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int hb = compress_hash_bits(R);
    const size_t H = (size_t)1 << hb;
    ctx->launches += 3;
    VQ_CK(launch_compress_pairs(R, uid, code, new_id, rep_uid, rep_code, count, static_cast<unsigned long long*>(ws),
                                at<int>(ws, align256(H * sizeof(unsigned long long))), hb, ctx->status, st,
                                ctx->num_sms));
    return VQNQS_OK;
}

int vqnqs_autotune(vqnqs_ctx* ctx, int M, void* ws, size_t ws_bytes, vqnqs_tuning* out, void* stream) {
    if (!ctx || !out || M < 128) return ctx ? fail(ctx, VQNQS_ERR_ARG, "autotune: need out and M >= 128") : VQNQS_ERR_ARG;
    ctx->err.clear();
    if (ctx->d % 64) return fail(ctx, VQNQS_ERR_ARG, "autotune: the tensor-core GEMMs need d_model % 64 == 0");
    const size_t d = ctx->d;
    const size_t need = align256((size_t)M * 4 * d * 2) + align256((size_t)M * 4 * d * 4) * 2;
    if (!ws || ws_bytes < need) return fail(ctx, VQNQS_ERR_WORKSPACE, "autotune: workspace too small");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    __nv_bfloat16* A = static_cast<__nv_bfloat16*>(ws);
    float* C = at<float>(ws, align256((size_t)M * 4 * d * 2));
    float* Rm = at<float>(ws, align256((size_t)M * 4 * d * 2) + align256((size_t)M * 4 * d * 4));
    VQ_CK(cudaMemsetAsync(ws, 0, need, st));
    VQ_CK(launch_set_int(ctx->gemm_m, M, st));
    const LayerW& w = ctx->lw[0];
    struct Shape { const __nv_bfloat16* Bt; int N, K, epi; const float* bias; } shapes[3] = {
        {w.wqkv_t, 3 * (int)d, (int)d, 0, w.b_qkv}, {w.w1_t, 4 * (int)d, (int)d, 1, w.b_1}, {w.w2_t, (int)d, 4 * (int)d, 2, w.b_2}};
    const int cand[4] = {64, 128, 192, 256};
    std::memset(out, 0, sizeof(*out));
    cudaEvent_t e0, e1;
    VQ_CK(cudaEventCreate(&e0));
    VQ_CK(cudaEventCreate(&e1));
    for (int s = 0; s < 3; ++s) {
        float best = 1e30f;
        for (int ci = 0; ci < 4; ++ci) {
            const int BN = cand[ci];
            out->ms[s][ci] = -1.f;
            if (shapes[s].N % BN) continue;
            CUtensorMap tb;
            VQ_CK(make_tmap_bf16(&tb, shapes[s].Bt, shapes[s].N, shapes[s].K, BN));
            for (int rep = 0; rep < 2; ++rep)
                VQ_CK(launch_gemm_tc(A, M, tb, shapes[s].bias, Rm, C, ctx->gemm_m, 0, shapes[s].N, shapes[s].K,
                                     shapes[s].epi, ctx->status, st, ctx->num_sms, BN));
            VQ_CK(cudaEventRecord(e0, st));
            for (int rep = 0; rep < 5; ++rep)
                VQ_CK(launch_gemm_tc(A, M, tb, shapes[s].bias, Rm, C, ctx->gemm_m, 0, shapes[s].N, shapes[s].K,
                                     shapes[s].epi, ctx->status, st, ctx->num_sms, BN));
            VQ_CK(cudaEventRecord(e1, st));
            VQ_CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            VQ_CK(cudaEventElapsedTime(&ms, e0, e1));
            out->ms[s][ci] = ms / 5.f;
            ctx->launches += 7;
            if (ms < best) { best = ms; ctx->bn[s] = BN; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out->qkv_bn = ctx->bn[0];
    out->mlp_up_bn = ctx->bn[1];
    out->mlp_down_bn = ctx->bn[2];
    return build_weight_tmaps(ctx);
}

int vqnqs_autotune_chunk(vqnqs_ctx* ctx, int B, const uint8_t* spins, int flags, const int* cand, int n_cand, void* ws,
                         size_t ws_bytes, int* best, float* ms, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (B <= 0 || !spins || !cand || n_cand <= 0 || !best || !ms || !ws)
        return fail(ctx, VQNQS_ERR_ARG, "autotune_chunk: need samples, candidates, workspace and outputs");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* e_loc = ctx->lp_scratch;  // local energies go to the context's scratch (B <= its capacity)
    if (B > ctx->lp_scratch_cap) return fail(ctx, VQNQS_ERR_ARG, "autotune_chunk: at most 65536 samples");
    cudaEvent_t e0, e1;
    VQ_CK(cudaEventCreate(&e0));
    VQ_CK(cudaEventCreate(&e1));
    *best = 0;
    float best_ms = 1e30f;
    int rc = VQNQS_OK;
    for (int i = 0; i < n_cand && rc == VQNQS_OK; ++i) {
        ms[i] = -1.f;
        if (cand[i] <= 0) continue;
        const size_t need = make_plan(ctx, cand[i], true).total;
        if (need > ws_bytes) continue;  // does not fit the given workspace
        // a workspace of exactly this plan makes run() use chunks of cand[i] samples
        rc = run(ctx, B, spins, e_loc, nullptr, nullptr, flags, ws, need, stream, true);
        if (rc != VQNQS_OK) break;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = fail(ctx, VQNQS_ERR_CUDA, "event"); break; }
        for (int rep = 0; rep < 2 && rc == VQNQS_OK; ++rep)
            rc = run(ctx, B, spins, e_loc, nullptr, nullptr, flags, ws, need, stream, true);
        if (rc != VQNQS_OK) break;
        float t = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = fail(ctx, VQNQS_ERR_CUDA, "autotune_chunk: event timing");
            break;
        }
        ms[i] = t / 2.f;
        if (ms[i] < best_ms) { best_ms = ms[i]; *best = cand[i]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == VQNQS_OK && *best == 0) return fail(ctx, VQNQS_ERR_WORKSPACE, "autotune_chunk: no candidate fits");
    return rc;
}

int vqnqs_autotune_incremental(vqnqs_ctx* ctx, int B, const uint8_t* spins, int flags, void* ws, size_t ws_bytes,
                               vqnqs_inc_tuning* out, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (B <= 0 || !spins || !out || !ws) return fail(ctx, VQNQS_ERR_ARG, "autotune_incremental: need samples and output");
    if (!(flags & VQNQS_INCREMENTAL) || !(flags & VQNQS_BF16))
        return fail(ctx, VQNQS_ERR_ARG, "autotune_incremental: needs VQNQS_BF16 | VQNQS_INCREMENTAL");
    if (B > ctx->lp_scratch_cap) return fail(ctx, VQNQS_ERR_ARG, "autotune_incremental: at most 65536 samples");
    const int rc0 = check_flags(ctx, flags);
    if (rc0 != VQNQS_OK) return rc0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float* e_loc = ctx->lp_scratch;
    static const int kPatch[3] = {2, 4, 8}, kRows[5] = {1, 2, 4, 8, 16};
    cudaEvent_t e0, e1;
    VQ_CK(cudaEventCreate(&e0));
    VQ_CK(cudaEventCreate(&e1));
    int rc = VQNQS_OK;
    // one local-energy evaluation untimed, then two timed, per setting
    auto time_it = [&](float* ms) {
        rc = run(ctx, B, spins, e_loc, nullptr, nullptr, flags, ws, ws_bytes, stream, true);
        if (rc != VQNQS_OK) return;
        if (cudaEventRecord(e0, st) != cudaSuccess) { rc = fail(ctx, VQNQS_ERR_CUDA, "event"); return; }
        for (int rep = 0; rep < 2 && rc == VQNQS_OK; ++rep)
            rc = run(ctx, B, spins, e_loc, nullptr, nullptr, flags, ws, ws_bytes, stream, true);
        if (rc != VQNQS_OK) return;
        float t = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            rc = fail(ctx, VQNQS_ERR_CUDA, "autotune_incremental: event timing");
            return;
        }
        *ms = t / 2.f;
    };
    const int keep_p = ctx->patch_items, keep_r = ctx->rows_slices;
    // the patch's items per CTA first (with the current changed-row setting), then the changed rows'
    float best = 1e30f;
    int bp = keep_p;
    for (int i = 0; i < 3 && rc == VQNQS_OK; ++i) {
        ctx->patch_items = kPatch[i];
        out->patch_ms[i] = -1.f;
        time_it(&out->patch_ms[i]);
        if (rc == VQNQS_OK && out->patch_ms[i] < best) { best = out->patch_ms[i]; bp = kPatch[i]; }
    }
    ctx->patch_items = bp;
    best = 1e30f;
    int br = keep_r;
    for (int i = 0; i < 5 && rc == VQNQS_OK; ++i) {
        ctx->rows_slices = kRows[i];
        out->rows_ms[i] = -1.f;
        time_it(&out->rows_ms[i]);
        if (rc == VQNQS_OK && out->rows_ms[i] < best) { best = out->rows_ms[i]; br = kRows[i]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != VQNQS_OK) {
        ctx->patch_items = keep_p;
        ctx->rows_slices = keep_r;
        return rc;
    }
    ctx->rows_slices = br;
    out->patch_items = bp;
    out->rows_slices = br;
    return VQNQS_OK;
}

// ---- autoregressive sampling -----------------------------------------------------
namespace {
struct SamplePlan {
    int S = 0;
    size_t counters, rows, X, Xn, Y, A, qkv, O, H1, code, logp, cache, total;
};

// Workspace of a chunk of S samples: per-row buffers of one position and the
// keys and values of every layer and position ([layer][S][N][2d], FP32 or BF16).
SamplePlan make_sample_plan(const vqnqs_ctx* c, int S, bool bf16) {
    SamplePlan p;
    p.S = S;
    const size_t d = c->d, f = sizeof(float), e = bf16 ? 2 : 4;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align256(o + bytes); return r; };
    p.counters = take(CNT_SLOTS * sizeof(int));
    p.rows = take((size_t)S * sizeof(int));
    p.X = take((size_t)S * d * f);
    p.Xn = take((size_t)S * d * f);
    p.Y = take((size_t)S * d * f);
    p.A = take((size_t)S * d * f);
    p.qkv = take((size_t)S * 3 * d * f);
    p.O = take((size_t)S * d * f);
    p.H1 = take((size_t)S * 4 * d * f);
    p.code = take((size_t)S * sizeof(int));
    p.logp = take((size_t)S * 2 * f);
    p.cache = take((size_t)c->layers * S * c->N * 2 * d * e);
    p.total = o;
    return p;
}
}  // namespace

size_t vqnqs_sample_workspace_bytes(const vqnqs_ctx* ctx, int chunk_samples, int flags) {
    if (!ctx) return 0;
    const int S = chunk_samples > 0 ? chunk_samples : 1024;
    return make_sample_plan(ctx, S, (flags & VQNQS_BF16) != 0).total;
}

int vqnqs_sample(vqnqs_ctx* ctx, int B, const float* uniforms, uint8_t* spins, float* log_psi, int flags, void* ws,
                 size_t ws_bytes, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (ctx->vq_heads > 1) return fail(ctx, VQNQS_ERR_ARG, "sample: one quantizer head only");
    if (ctx->half_block) return fail(ctx, VQNQS_ERR_ARG, "sample: no final half-block");
    if (ctx->G > 1) return fail(ctx, VQNQS_ERR_ARG, "sample: one spin per token");
    if (B < 0) return fail(ctx, VQNQS_ERR_ARG, "B must be >= 0");
    if (flags & ~(VQNQS_REUSE | VQNQS_BF16 | VQNQS_INCREMENTAL)) return fail(ctx, VQNQS_ERR_ARG, "unknown flag bits");
    const bool bf16 = (flags & VQNQS_BF16) != 0;
    if (bf16 && ctx->d % 64) return fail(ctx, VQNQS_ERR_ARG, "VQNQS_BF16 needs d_model % 64 == 0");
    if (B == 0) return VQNQS_OK;
    if (!uniforms || !spins || !log_psi) return fail(ctx, VQNQS_ERR_ARG, "uniforms, spins and log_psi are required");
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return fail(ctx, VQNQS_ERR_ARG, "workspace must be 256-byte aligned");
    // largest chunk whose workspace fits
    int lo = 0, hi = B;
    while (lo < hi) {
        const int mid = lo + (hi - lo + 1) / 2;
        if (make_sample_plan(ctx, mid, bf16).total <= ws_bytes) lo = mid;
        else hi = mid - 1;
    }
    if (lo == 0) return fail(ctx, VQNQS_ERR_WORKSPACE, "workspace smaller than the one-sample minimum");
    const SamplePlan P = make_sample_plan(ctx, lo, bf16);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int N = ctx->N, d = ctx->d, K = ctx->K, H = ctx->heads;
    int* counters = at<int>(ws, P.counters);
    int* rows = at<int>(ws, P.rows);
    float* X = at<float>(ws, P.X);
    float* Xn = at<float>(ws, P.Xn);
    float* Y = at<float>(ws, P.Y);
    float* A = at<float>(ws, P.A);
    float* qkv = at<float>(ws, P.qkv);
    float* O = at<float>(ws, P.O);
    float* H1 = at<float>(ws, P.H1);
    int* code = at<int>(ws, P.code);
    float* logp = at<float>(ws, P.logp);
    __nv_bfloat16* A16 = reinterpret_cast<__nv_bfloat16*>(A);
    __nv_bfloat16* qkv16 = reinterpret_cast<__nv_bfloat16*>(qkv);
    __nv_bfloat16* H16 = reinterpret_cast<__nv_bfloat16*>(H1);
    const size_t cache_layer = (size_t)P.S * N * 2 * d;
    for (int s0 = 0; s0 < B; s0 += P.S) {
        const int S = std::min(P.S, B - s0);
        const float* u = uniforms + (size_t)s0 * N;
        uint8_t* sp = spins + (size_t)s0 * N;
        float* lp = log_psi + s0;
        const int g_rows = grid_for(ctx, S, 8, 16);
        ctx->launches += 1;
        VQ_CK(launch_assign_setup(counters, rows, S, st));  // S rows, listed 0 .. S-1
        for (int p = 0; p < N; ++p) {
            ctx->launches += 1;
            VQ_CK(launch_sample_embed(S, p, N, d, sp, ctx->tok_emb, ctx->pos_emb, X, st));
            for (int l = 0; l < ctx->layers; ++l) {
                const LayerW& w = ctx->lw[l];
                ctx->launches += 7;
                if (bf16) {
                    __nv_bfloat16* cache = reinterpret_cast<__nv_bfloat16*>(at<uint8_t>(ws, P.cache)) + l * cache_layer;
                    VQ_CK(launch_layernorm(X, counters, CNT_A, w.ln1_g, w.ln1_b, d, nullptr, A16, st, g_rows));
                    VQ_CK(launch_gemm_tc(A16, P.S, w.tm_wqkv, w.b_qkv, nullptr, qkv16, counters, CNT_A, 3 * d, d, 0,
                                         ctx->status, st, ctx->num_sms, ctx->bn[0]));
                    VQ_CK(launch_decode_attention(S, p, N, d, H, qkv16, cache, O, st));
                } else {
                    float* cache = at<float>(ws, P.cache) + l * cache_layer;
                    VQ_CK(launch_layernorm(X, counters, CNT_A, w.ln1_g, w.ln1_b, d, A, nullptr, st, g_rows));
                    VQ_CK(launch_sgemm(A, w.w_qkv, w.b_qkv, nullptr, qkv, counters, CNT_A, P.S, 3 * d, d, EPI_BIAS, st,
                                       ctx->num_sms));
                    VQ_CK(launch_decode_attention(S, p, N, d, H, qkv, cache, O, st));
                }
                if (bf16 && vq_tc_supported(K, d))
                    VQ_CK(launch_vq_tc(w.tm_cb_hi, w.tm_cb_lo, O, counters, rows, w.cnorm, K, d, code,
                                       ctx->stats + ST_NEAR_TIES, ctx->status, st, ctx->num_sms, P.S));
                else
                    VQ_CK(launch_vq_argmin(O, counters, rows, w.codebook, w.cnorm, K, d, code, ctx->stats + ST_NEAR_TIES,
                                           P.S, st, ctx->num_sms));
                if (bf16) {
                    VQ_CK(launch_residual_vq_ln(X, rows, code, w.T, counters, CNT_A, w.ln2_g, w.ln2_b, d, Y, nullptr,
                                                A16, st, g_rows));
                    VQ_CK(launch_gemm_tc(A16, P.S, w.tm_w1, w.b_1, nullptr, H16, counters, CNT_A, 4 * d, d, 1,
                                         ctx->status, st, ctx->num_sms, ctx->bn[1]));
                    VQ_CK(launch_gemm_tc(H16, P.S, w.tm_w2, w.b_2, Y, Xn, counters, CNT_A, d, 4 * d, 2, ctx->status, st,
                                         ctx->num_sms, ctx->bn[2]));
                } else {
                    VQ_CK(launch_residual_vq_ln(X, rows, code, w.T, counters, CNT_A, w.ln2_g, w.ln2_b, d, Y, A, nullptr,
                                                st, g_rows));
                    VQ_CK(launch_sgemm(A, w.w_1, w.b_1, nullptr, H1, counters, CNT_A, P.S, 4 * d, d, EPI_BIAS_GELU, st,
                                       ctx->num_sms));
                    VQ_CK(launch_sgemm(H1, w.w_2, w.b_2, Y, Xn, counters, CNT_A, P.S, d, 4 * d, EPI_BIAS_RESID, st,
                                       ctx->num_sms));
                }
                std::swap(X, Xn);
            }
            ctx->launches += 2;
            VQ_CK(launch_head(X, counters, CNT_A, ctx->lnf_g, ctx->lnf_b, ctx->w_head, ctx->b_head, d, logp, st,
                              g_rows));
            VQ_CK(launch_sample_draw(S, p, N, logp, u, sp, lp, st));
        }
    }
    return VQNQS_OK;
}

// ---- variational Monte Carlo step --------------------------------------------------
namespace {
__global__ void k_sgd(float* __restrict__ w, const float* __restrict__ g, size_t n, float lr) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        w[i] = __fsub_rn(w[i], __fmul_rn(lr, g[i]));  // product and difference rounded apart (no FMA)
}
}  // namespace

size_t vqnqs_vmc_workspace_bytes(const vqnqs_ctx* ctx, int B, int flags) {
    if (!ctx || B <= 0) return 0;
    const size_t a = vqnqs_sample_workspace_bytes(ctx, std::min(B, 1024), flags);
    const size_t b = vqnqs_workspace_bytes(ctx, 0, flags);
    const size_t c = vqnqs_grad_workspace_bytes(ctx, B, 0);
    return std::max(a, std::max(b, c));
}

int vqnqs_vmc_step(vqnqs_ctx* ctx, int B, const float* uniforms, float lr, uint8_t* spins, float* e_loc, float* grad,
                   double* mean_var, int flags, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (ctx->vq_heads > 1) return fail(ctx, VQNQS_ERR_ARG, "vmc_step: one quantizer head only");
    if (ctx->half_block) return fail(ctx, VQNQS_ERR_ARG, "vmc_step: no final half-block");
    if (ctx->G > 1) return fail(ctx, VQNQS_ERR_ARG, "vmc_step: one spin per token");
    if (B <= 0 || !uniforms || !spins || !e_loc || !grad || !mean_var)
        return fail(ctx, VQNQS_ERR_ARG, "vmc step: B > 0 and every buffer are required");
    // e_loc holds the drawn configurations' log psi until the local energies overwrite it
    int rc = vqnqs_sample(ctx, B, uniforms, spins, e_loc, flags, ws, ws_bytes, stream);
    if (rc != VQNQS_OK) return rc;
    rc = vqnqs_local_energy(ctx, B, spins, e_loc, mean_var, nullptr, flags, ws, ws_bytes, stream);
    if (rc != VQNQS_OK) return rc;
    rc = vqnqs_grad_log_psi(ctx, B, spins, nullptr, e_loc, nullptr, grad, flags, ws, ws_bytes, stream);
    if (rc != VQNQS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ctx->launches += 1;
    k_sgd<<<grid_for(ctx, (long long)ctx->nparams, 256, 8), 256, 0, st>>>(ctx->blob, grad, ctx->nparams, lr);
    VQ_CK(cudaGetLastError());
    return build_tables(ctx, st);  // the weights changed: rebuild their derived tables
}

int vqnqs_get_weights(vqnqs_ctx* ctx, float* weights, void* stream) {
    if (!ctx || !weights) return VQNQS_ERR_ARG;
    VQ_CK(cudaMemcpyAsync(weights, ctx->blob, ctx->nparams * sizeof(float), cudaMemcpyDeviceToDevice,
                          static_cast<cudaStream_t>(stream)));
    return VQNQS_OK;
}

int vqnqs_check_timeout_path(vqnqs_ctx* ctx, long long limit_cycles, void* stream) {
    if (!ctx) return VQNQS_ERR_ARG;
    ctx->err.clear();
    if (limit_cycles < 1 || limit_cycles > 4000000000LL)
        return fail(ctx, VQNQS_ERR_ARG, "limit_cycles must be 1 .. 4e9");
    ctx->launches += 1;
    VQ_CK(launch_timeout_probe(ctx->status, limit_cycles, static_cast<cudaStream_t>(stream)));
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
