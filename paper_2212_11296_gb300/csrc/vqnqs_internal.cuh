// Internal declarations shared by the kernel translation units of libvqnqs.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/vqnqs.h"

namespace vq {

constexpr int BOS = 2;          // begin-of-sequence token id
constexpr float LN_EPS = 1e-5f; // LayerNorm epsilon (biased variance)
constexpr float NEAR_TIE_REL = 1e-6f;

// Slots of the per-chunk device counter array (int32).
enum {
    CNT_C = 0,      // configurations in the chunk
    CNT_R = 1,      // rows = C * N
    CNT_A = 2,      // active rows: rows whose attention and codeword are computed
    CNT_V = 3,      // incremental path: rows of the current layer listed for the codeword search
    CNT_TCL = 4,    //   connected configurations patched on the tensor cores (list length)
    CNT_SCL = 5,    //   connected configurations patched on the CUDA cores (list length)
    CNT_TCW = 6,    //   work counters of the two patch kernels (next list entry); on the
    CNT_SCW = 7,    //   tensor-core path CNT_SCW feeds the attention of the whole recomputes
    CNT_U0 = 8,     // CNT_U0 + l: unique rows feeding layer l (l = 0..layers)
    CNT_EX = 8 + VQNQS_MAX_LAYERS + 2,  // split operands: patched rows listed for the exact correction
    CNT_CW = CNT_EX + 1,                // two-word codes: distinct (hi, lo) code pairs of the layer
    CNT_SLOTS = CNT_CW + 1
};

// Slots of the context's persistent device statistics (int64).
enum {
    ST_SAMPLES = 0,
    ST_CONFIGS = 1,
    ST_ROWS = 2,
    ST_NEAR_TIES = 3,
    ST_U0 = 4,      // ST_U0 + l
    ST_ACTIVE = 4 + VQNQS_MAX_LAYERS + 2,  // rows whose attention and code are computed (per layer)
    ST_PAIRS = ST_ACTIVE + 1,              // causal query-key pairs of those rows (per layer)
    ST_INC_BASE = ST_PAIRS + 1,            // incremental path, summed over layers: samples' own rows
    ST_INC_PATCHED,                        //   rows corrected for the changed keys only
    ST_INC_CERT,                           //   patched rows whose code was proved to be the sample's
    ST_INC_FULL,                           //   rows recomputed over all keys
    ST_INC_VQ,                             //   rows given to the codeword search
    ST_INC_PPAIRS,                         //   (patched row, changed key) pairs, per head
    ST_INC_FPAIRS,                         //   query-key pairs of the recomputed rows, per head
    ST_INC_WPAIRS,                         //   causal query-key pairs of configurations recomputed whole
    ST_SLOTS
};

// Incremental path (k_incremental.cu): the certificate of one of a sample's rows.
// Codeword j (!= code) cannot become the nearest while ||delta|| < rho of j; the
// CERT_T smallest radii are listed ascending, `next` is the one after them.
constexpr int CERT_T = 8;
constexpr int INC_MAX_KEYS = 64;  // changed positions patched per configuration (more: recompute)
struct CertRow {
    float next, eta;
    int n, code;
    int j[CERT_T];
    float rho[CERT_T], gap[CERT_T];
};

struct LayerW {
    const float *ln1_g, *ln1_b, *w_qkv, *b_qkv, *codebook, *w_o, *b_o;
    const float *ln2_g, *ln2_b, *w_1, *b_1, *w_2, *b_2;
    float* T;       // [K][d] codebook @ w_o + b_o: the quantized vector after the output projection
    float* cnorm;   // [K] ||W_j||^2
    __nv_bfloat16 *wqkv_t, *w1_t, *w2_t;  // BF16 transposes [out][in] for the tensor-core GEMMs
    CUtensorMap tm_wqkv, tm_w1, tm_w2;    // TMA maps of the transposes (valid when d % 64 == 0)
    float* wd;                            // [K][K] ||W_a - W_c|| (incremental path's certificates)
    float *cb_hi, *cb_lo;                 // codebook split into TF32 hi / lo parts
    CUtensorMap tm_cb_hi, tm_cb_lo;       // their TMA maps (valid when vq_tc_supported)
    __nv_bfloat16* wo_t = nullptr;        // final half-block only: BF16 transpose of W_o
    CUtensorMap tm_wo;                    //   and its TMA map
    // tensor-core backward (split operands): the weights as stored, each as a BF16 hi plane and a lo
    // plane after it ([2 rows][cols]), as the B operand of dX = dY W^T; the codebook also transposed
    __nv_bfloat16 *wqkv_s = nullptr, *w1_s = nullptr, *w2_s = nullptr, *wo_s = nullptr, *cb_s = nullptr,
                  *cbT_s = nullptr;
    CUtensorMap tm_wqkv_s, tm_w1_s, tm_w2_s, tm_wo_s, tm_cb_s, tm_cbT_s;
};

// Lattice groups of a batch (one group for a single lattice, up to MAX_GROUPS
// for a ragged batch of several lattice sizes): global samples
// first[g] .. first[g+1]-1 are L[g] x L[g] lattices with N[g] sites, whose spins
// start at byte spin_off[g] of the batch's spin array (N[g] bytes per sample)
// and whose bonds are bonds[bond_off[g] .. bond_off[g] + nb[g]).
constexpr int MAX_GROUPS = 8;
struct Groups {
    int n;
    int first[MAX_GROUPS + 1];
    int N[MAX_GROUPS], nb[MAX_GROUPS], bond_off[MAX_GROUPS];
    long long spin_off[MAX_GROUPS];
};

// Hamiltonians: the square-lattice Heisenberg model (connected configurations:
// one nearest-neighbour exchange) and the transverse-field Ising chain
// (connected configurations: one spin flip; cfg_j = CFG_FLIP).
enum { MODEL_HEISENBERG = 0, MODEL_TFIM_CHAIN = 1 };
constexpr int CFG_FLIP = 0x3fffffff;

// Per-chunk view of the problem handed to the kernels.  Rows of a chunk are
// (configuration, position) pairs stored configuration after configuration;
// configuration c owns rows cfg_row[c] .. cfg_row[c+1]-1.
struct Chunk {
    const uint8_t* spins;   // spins of the whole batch
    const int* bonds;       // bond table of all groups, [.][2]
    Groups g;
    int s0, S;              // this chunk holds global samples s0 .. s0+S-1 (local index b)
    int N, d, heads, K;     // N: largest number of positions (position-embedding rows)
    int G = 1;              // spins per token: a sample of n sites has n / G positions
    int model;              // MODEL_*
    const int* cfg_sample;  // [C] local sample of each configuration
    const int* cfg_i;       // [C] exchanged site pair (-1 for the sample itself)
    const int* cfg_j;
    const int* cfg_off;     // [S + 1] first configuration of each sample
    const int* cfg_row;     // [C + 1] first row of each configuration
    const int* row_cfg;     // [R] configuration of each row
    int* counters;          // CNT_* slots
};

__device__ __forceinline__ int sample_group(const Chunk& ch, int b) {
    const int gb = ch.s0 + b;
    int g = 0;
    while (g + 1 < ch.g.n && gb >= ch.g.first[g + 1]) ++g;
    return g;
}
// positions (rows) of sample b: its sites over the token group size
__device__ __forceinline__ int sample_N(const Chunk& ch, int b) { return ch.g.N[sample_group(ch, b)] / ch.G; }
__device__ __forceinline__ const uint8_t* sample_spins(const Chunk& ch, int b) {
    const int g = sample_group(ch, b);
    return ch.spins + ch.g.spin_off[g] + (long long)(ch.s0 + b - ch.g.first[g]) * ch.g.N[g];
}
__device__ __forceinline__ int cfg_N(const Chunk& ch, int c) { return sample_N(ch, ch.cfg_sample[c]); }

// First position whose rows differ from the sample's own rows.  Exchanging
// sites i and j changes the inputs (tokens s_{p-1}) only at p = i+1 and
// p = j+1, and a causal network's rows at p <= min(i, j) see none of them
// (Sec. 2: conditionals before the changed site are unchanged).
__device__ __forceinline__ int cfg_first_changed(int ci, int cj) { return ci < 0 ? 0 : min(ci, cj) + 1; }
// The same for tokens of G spins: the group of the first changed site is the first
// changed token input one position later.
__device__ __forceinline__ int cfg_p0(const Chunk& ch, int c) {
    const int ci = ch.cfg_i[c], cj = ch.cfg_j[c];
    return ci < 0 ? 0 : min(ci, cj) / ch.G + 1;
}

// Spin at site q of the configuration whose sample spins are s and whose exchanged
// pair is (ci, cj), or whose site ci is flipped when cj == CFG_FLIP.
__device__ __forceinline__ int cfg_spin(const uint8_t* s, int ci, int cj, int q) {
    if (q == ci) return cj == CFG_FLIP ? 1 - (s[q] & 1) : s[cj] & 1;
    if (q == cj) return s[ci] & 1;
    return s[q] & 1;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- launchers (each returns cudaGetLastError of its launch) -------------------

// configuration enumeration (k_config.cu): configurations, then row offsets; the
// diagonal element is diag_coef * sum over bonds of sigma_i sigma_j
cudaError_t launch_configs(const Chunk& ch, float diag_coef, int with_bonds, int* cnt, float* diag, int* cfg_off,
                           int* cfg_sample, int* cfg_i, int* cfg_j, int* cfg_row, int* row_cfg, int* status,
                           cudaStream_t st, int grid);
cudaError_t launch_embed(const Chunk& ch, const float* tok_emb, const float* pos_emb, int reuse, float* X0,
                         int* uid0, cudaStream_t st, int grid);
// V = 2^G outputs (log-softmax over the values of a token's spin group)
cudaError_t launch_head(const float* X, const int* counters, int u_slot, const float* g, const float* b,
                        const float* w_head, const float* b_head, int d, float* logp, cudaStream_t st, int grid,
                        int G = 1);
// final half-block (no quantizer): active row a (counters[CNT_A] of them, row act_rows[a])
// gets G_o[a] = O[row] (FP32 or BF16) and G_x[a] = X[uid[row]]; then every chunk row
// gets the index of its active row (of the sample's row before the first changed site)
cudaError_t launch_half_gather(const int* counters, const int* act_rows, const int* uid, const float* O,
                               const float* X, int d, float* G_o, __nv_bfloat16* G_o16, float* G_x, cudaStream_t st,
                               int grid);
cudaError_t launch_half_ids(const Chunk& ch, int prefix_reuse, const int* act_off, int* uid_out, cudaStream_t st,
                            int grid);
cudaError_t launch_eloc(const Chunk& ch, const int* uid, const float* logp, float* ratio, float* log_psi_out,
                        cudaStream_t st, int grid);
// e_loc = diag + offdiag * sum over connected configurations of psi(s') / psi(s)
cudaError_t launch_eloc_reduce(const Chunk& ch, const float* diag, const float* ratio, float offdiag,
                               float* e_loc_out, cudaStream_t st, int grid);
cudaError_t launch_copy_codes(const Chunk& ch, const int* code, int l, int layers, int* out, cudaStream_t st,
                              int grid);
// codes of every configuration's rows: out [S][per_sample][layers][N] of the chunk's samples
cudaError_t launch_copy_cfg_codes(const Chunk& ch, const int* code, int l, int layers, int per_sample, int* out,
                                  cudaStream_t st, int grid);
cudaError_t launch_mean_var(const float* e_loc, int B, double* mean_var, cudaStream_t st);
cudaError_t launch_accumulate_stats(const int* counters, int layers, int S, long long* stats, cudaStream_t st);

// LayerNorm and per-location helpers (k_rowops.cu)
// lo_off > 0: out_bf16 also gets the split lo plane lo_off elements after the hi one
cudaError_t launch_layernorm(const float* X, const int* counters, int u_slot, const float* g, const float* b, int d,
                             float* out_f32, __nv_bfloat16* out_bf16, cudaStream_t st, int grid, size_t lo_off = 0);
// residual with the quantized vector's projection, then LN2; with vq_heads > 1 the
// code packs one bits-wide field per head and T holds vq_heads tables of K rows
cudaError_t launch_residual_vq_ln(const float* X, const int* rep_uid, const int* rep_code, const float* T,
                                  const int* counters, int u_slot, const float* g, const float* b, int d, float* Y,
                                  float* A_f32, __nv_bfloat16* A_bf16, cudaStream_t st, int grid, int vq_heads = 1,
                                  int K = 0, int bits = 0, size_t lo_off = 0, const int* tab_lo = nullptr,
                                  const int* tab_hi = nullptr);
// T and cnorm of a layer's codebook ([vq_heads][K][d / vq_heads])
cudaError_t launch_table_T(const float* codebook, const float* w_o, const float* b_o, int K, int d, int vq_heads,
                           float* T, float* cnorm, cudaStream_t st);
// WT [cols][rows] = bf16(W^T); with lo, WT holds [2 cols][rows]: the split lo plane follows
cudaError_t launch_transpose_bf16(const float* W, int rows, int cols, __nv_bfloat16* WT, cudaStream_t st,
                                  bool lo = false);

// FP32 SIMT GEMM (k_gemm_f32.cu): C[M,N] = A[M,K] @ B[K,N] + bias (+GELU) (+R); M = counters[u_slot]
enum { EPI_BIAS = 0, EPI_BIAS_GELU = 1, EPI_BIAS_RESID = 2 };
cudaError_t launch_sgemm(const float* A, const float* B, const float* bias, const float* R, float* C,
                         const int* counters, int u_slot, int Mmax, int N, int K, int epi, cudaStream_t st,
                         int num_sms);

// active rows (k_config.cu): with prefix reuse, the rows p >= first changed position of every
// configuration, listed in act_rows[0 .. counters[CNT_A]); without it every row.
cudaError_t launch_active_rows(const Chunk& ch, int prefix_reuse, int* act_cnt, int* act_off, int* act_rows,
                               long long* stats, cudaStream_t st, int grid);

// attention (k_attn.cu): O[r] for the active rows (all rows when prefix_reuse == 0) of the
// configurations cfg_list[0 .. n_list) (all of the chunk's when cfg_list is NULL); with
// stats, also (max scaled score, sum of exp(score - max)) per (sample * N + p, head)
cudaError_t launch_attention_f32(const Chunk& ch, const int* uid, const float* qkv, float* O, int prefix_reuse,
                                 cudaStream_t st, int grid, const int* cfg_list = nullptr, int n_list = 0,
                                 float2* stats = nullptr);
cudaError_t launch_attention_bf16in(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                                   int prefix_reuse, cudaStream_t st, int grid, const int* cfg_list = nullptr,
                                   int n_list = 0, float2* stats = nullptr);
// tensor-core attention (k_attn_tc.cu): dh in {16, 32}, N <= 448 (<= 256 with split operands, whose
// shared-memory tiles are twice as large); cfg_list and stats as above.  lo_off != 0: split operands,
// the BF16 lo plane of Q/K/V lo_off elements after the hi plane qkv.
bool attention_tc_supported(int N, int dh, bool split = false);
cudaError_t launch_attention_tc(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O, int prefix_reuse,
                                int* status, cudaStream_t st, int grid, const int* cfg_list = nullptr,
                                int n_list = 0, float2* stats = nullptr, const int* n_list_dev = nullptr,
                                size_t lo_off = 0, int* work = nullptr);

// BF16 tensor-core GEMM (k_gemm_tc.cu): C[M,N] = A[M,K] @ Bt[N,K]^T + bias, M = counters[u_slot]
// epi: 0 BF16 out, 1 BF16 out of GELU, 2 FP32 out + R, 3 FP32 out
int tc_pick_bn(int N);
cudaError_t make_tmap_bf16(CUtensorMap* map, const void* base, long long rows, int cols, int box_rows);
// the same for rows of ld elements of which the first cols are read (cols <= ld; ld * 2 % 16 == 0)
cudaError_t make_tmap_bf16_strided(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld,
                                   int box_rows);
// BN = output tile width (64, 128, 192 or 256 dividing N; 0 picks the widest); tmB's box must be [BN x 64].
// split: A is [2 Arows][K] (hi plane, then lo plane), tmB covers [2N][K] (hi rows, then lo rows), three
// passes per K block; BF16 outputs (epi 0, 1) are [2 Arows][N] (hi, then lo plane).
// a_inner > 0: A's rows hold a_inner elements (K may exceed it; those K blocks read zeros)
cudaError_t launch_gemm_tc(const __nv_bfloat16* A, long long Arows, const CUtensorMap& tmB, const float* bias,
                           const float* R, void* Cout, const int* counters, int u_slot, int N, int K, int epi,
                           int* status, cudaStream_t st, int num_sms, int BN = 0, bool split = false,
                           long long a_inner = 0, int ksplit = 1);
// ksplit > 1 (epi 3 only): the K blocks are divided into ksplit ranges, each written as an FP32
// partial result at rows [s Mpad, s Mpad + Arows) of Cout (Mpad = Arows rounded up to 128), for
// launch_splitk_add: C[m][n] += sum over s, in order, of those partials (m < M)
cudaError_t launch_splitk_add(const float* part, int ksplit, long long Mpad, int M, int N, float* C, cudaStream_t st,
                              int num_sms);
// dst [2 plane_rows][cols] BF16: row r of src (FP32 [rows][cols]) split into hi (row r) and lo (row plane_rows + r)
cudaError_t launch_split_planes(const float* src, long long rows, int cols, __nv_bfloat16* dst, long long plane_rows,
                                cudaStream_t st, int cap);
cudaError_t launch_set_int(int* p, int v, cudaStream_t st);
cudaError_t launch_timeout_probe(int* status, long long limit_cycles, cudaStream_t st);

// nearest codeword (k_vq.cu): rows act_rows[0 .. counters[CNT_A]) (or 0 .. counters[CNT_R] when act_rows is NULL)
cudaError_t launch_vq_argmin(const float* O, const int* counters, const int* act_rows, const float* codebook,
                             const float* cnorm, int K, int d, int* code, long long* near_ties, int Rmax,
                             cudaStream_t st, int num_sms, int a_slot = CNT_A);
// the same per quantizer head: segment h of every row against codebook h, packed codes (heads beyond
// 32 / bits per word go to the second word code_hi)
cudaError_t launch_vq_argmin_heads(const float* O, const int* counters, const int* act_rows, const float* codebook,
                                   const float* cnorm, int K, int d, int vq_heads, int bits, int* code,
                                   long long* near_ties, int Rmax, cudaStream_t st, int num_sms, int a_slot = CNT_A,
                                   int* code_hi = nullptr);
// two-word codes: the listed rows' (hi, lo) code words -> a dense code id in lo (k_dedupe.cu)
cudaError_t launch_code_words(int* counters, int a_slot, int cnt_slot, const int* rows, int Rmax, int* lo,
                              const int* hi, unsigned long long* keys, int* vals, int hash_bits, int* tab_hi,
                              int* tab_lo, int* status, cudaStream_t st, int num_sms);

cudaError_t launch_assign_setup(int* counters, int* rows, int R, cudaStream_t st);

// autoregressive sampling steps (k_sample.cu)
cudaError_t launch_sample_embed(int S, int p, int N, int d, const uint8_t* spins, const float* tok_emb,
                                const float* pos_emb, float* X, cudaStream_t st);
cudaError_t launch_decode_attention(int S, int p, int N, int d, int H, const float* qkv, float* cache, float* O,
                                    cudaStream_t st);
cudaError_t launch_decode_attention(int S, int p, int N, int d, int H, const __nv_bfloat16* qkv,
                                    __nv_bfloat16* cache, float* O, cudaStream_t st);
cudaError_t launch_sample_draw(int S, int p, int N, const float* logp, const float* u, uint8_t* spins,
                               float* log_psi, cudaStream_t st);

// nearest codeword on the tensor cores, split-TF32 (k_vq_tc.cu)
bool vq_tc_supported(int K, int d);
cudaError_t make_tmap_codebook(CUtensorMap* map, const float* base, int K, int d);
cudaError_t launch_split_tf32(const float* W, size_t n, float* hi, float* lo, cudaStream_t st);
cudaError_t launch_vq_tc(const CUtensorMap& tm_hi, const CUtensorMap& tm_lo, const float* O, const int* counters,
                         const int* act_rows, const float* cnorm, int K, int d, int* code, long long* near_ties,
                         int* status, cudaStream_t st, int num_sms, int Rmax, int a_slot = CNT_A,
                         float* dist_out = nullptr, float* osq_out = nullptr);

// incremental evaluation of the connected configurations (k_incremental.cu)
bool incremental_supported(int d, int heads);
bool patch_tc_supported(int d, int heads);  // BF16 path: rows patched on the tensor cores
// attention of listed rows sharing a sample's keys except at changed positions (k_attn_rows_tc.cu)
bool attention_rows_tc_supported(int N, int d, int heads);
cudaError_t launch_attention_rows_tc(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                                     const int2* list, const int* act_off, const int* count, const short* dpos,
                                     const int* dcnt, int* status, long long* stats, cudaStream_t st, int num_sms,
                                     size_t lo_off = 0, int slices_per_sm = 2);
// per connected configuration: changed positions (first INC_MAX_KEYS), their count, and the work list it joins
// (BF16 path: tensor-core patch, or recomputed whole with its rows searched; FP32 path: CUDA-core patch)
cudaError_t launch_inc_classify(const Chunk& ch, const int* uid, int tc_ok, int* list_tc, int* list_simt, short* dpos,
                                int* dcnt, int* vq_rows, long long* stats, cudaStream_t st, int grid);
cudaError_t launch_codeword_dist(const float* W, int K, int d, float* wd, cudaStream_t st);
cudaError_t launch_base_cert(const Chunk& ch, const float* O, const float* codebook, const float* cnorm,
                             const float* wd, int K, int d, int* code, CertRow* cert, long long* stats,
                             int* counters, int* rc_cnt, cudaStream_t st);
// the same from the split-TF32 tensor-core distances (k_vq_tc in distance mode) of the chunk's sample rows:
// list holds S N + 1 ints, dist S N K floats and osq S N floats of workspace (K a multiple of 16)
cudaError_t launch_base_cert_tc(const Chunk& ch, const float* O, const CUtensorMap& tm_hi, const CUtensorMap& tm_lo,
                                const float* cnorm, const float* wd, int K, int d, int* code, CertRow* cert,
                                long long* stats, int* counters, int* rc_cnt, int* list, float* dist, float* osq,
                                int* status, cudaStream_t st, int num_sms);
// the same with H > 1 quantizer heads (packed codes of `bits` per head, one word): the row's radius is the
// smallest over its segments, no candidate list; wd holds H tables [K][K]
cudaError_t launch_base_cert_heads(const Chunk& ch, const float* O, const float* codebook, const float* cnorm,
                                   const float* wd, int K, int d, int H, int bits, int* code, CertRow* cert,
                                   long long* stats, int* counters, int* rc_cnt, cudaStream_t st, int num_sms);
// wd: the layer's ||W_a - W_c|| table; split (BF16 qkv only): the Q/K/V in qkv are the hi plane of split
// operands, and rows the certificate does not settle are listed in ex_rows (count in CNT_EX) for
// launch_inc_exact_delta instead of being written with the BF16 correction
cudaError_t launch_inc_patch(const Chunk& ch, const int* uid, const float* qkv, float* O, const float2* bstat,
                             const CertRow* cert, const float* codebook, const float* wd, int* code, int* vq_rows,
                             const int* act_off, int2* rc_rows, int* rc_cnt, const int* list_tc,
                             const int* list_simt, const short* dpos, const int* dcnt, int use_tc, int* status,
                             long long* stats, cudaStream_t st, int grid);
cudaError_t launch_inc_patch(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                             const float2* bstat, const CertRow* cert, const float* codebook, const float* wd,
                             int* code, int* vq_rows, const int* act_off, int2* rc_rows, int* rc_cnt,
                             const int* list_tc, const int* list_simt, const short* dpos, const int* dcnt, int use_tc,
                             int split, int2* ex_rows, int* status, long long* stats, cudaStream_t st, int grid,
                             int items_per_cta = 4);
// split operands: o + delta of the listed rows (row, position) from the hi + lo planes of Q/K/V in FP32
// (one warp per row; d_model in {128, 256}, d_model / heads = 32); n_list_dev[0] rows
cudaError_t launch_inc_exact_delta(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, size_t lo_off, float* O,
                                   const float2* bstat, const short* dpos, const int* dcnt, const int2* list,
                                   const int* n_list_dev, cudaStream_t st, int grid);
cudaError_t launch_inc_attention(const Chunk& ch, const int* uid, const float* qkv, float* O, const int* act_off,
                                 const int2* rc_rows, const int* rc_cnt, int tail_only, long long* stats, cudaStream_t st,
                                 int num_sms);
cudaError_t launch_inc_attention(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                                 const int* act_off, const int2* rc_rows, const int* rc_cnt, int tail_only, long long* stats,
                                 cudaStream_t st, int num_sms);

// dedupe (k_dedupe.cu); with prefix reuse a row before its configuration's first changed
// position takes the code of the same position of the sample's own configuration.
cudaError_t launch_dedupe(const Chunk& ch, const int* uid_cur, const int* code, int u_slot_next, int Rmax,
                          unsigned long long* keys, int* vals, int hash_bits, int* uid_next, int* rep_uid,
                          int* rep_code, int reuse, int* status, cudaStream_t st, int num_sms);

// standalone (I, V) compression of R (row id, code) pairs (k_dedupe.cu)
int compress_hash_bits(int R);
cudaError_t launch_compress_pairs(int R, const int* uid, const int* code, int* new_id, int* rep_uid, int* rep_code,
                                  int* count, unsigned long long* keys, int* vals, int hash_bits, int* status,
                                  cudaStream_t st, int num_sms);

// ---- backward (k_gemm_f32_gen.cu, k_backward.cu, vqnqs_grad.cu) ----
cudaError_t launch_gemm_gen(bool ta, bool tb, const float* A, const float* B, float* C, int M, int N, int K, int lda,
                            int ldb, int ldc, long long sA, long long sB, long long sC, int batch, int accumulate,
                            cudaStream_t st, int num_sms);
cudaError_t launch_head_bwd(const float* X, const uint8_t* spins, const float* seed, int R, int N, int d,
                            const float* g, const float* b, const float* w, const float* bh, float* dX, float* Af,
                            float* dlog, float* dgam, float* dbet, cudaStream_t st, int cap);
cudaError_t launch_ln_bwd(const float* X, const float* dA, const float* g, int R, int d, float* dX, int accumulate,
                          float* dgam, float* dbet, cudaStream_t st, int cap);
cudaError_t launch_gelu_bwd(const float* H, float* dG, size_t n, cudaStream_t st, int cap);
cudaError_t launch_gelu_fwd(const float* H, float* G, size_t n, cudaStream_t st, int cap);
cudaError_t launch_st_rows(const float* OW, const float* DG, const float* O, const float* cnorm, int R, int K, int d,
                           float* alpha, float* arow, cudaStream_t st, int cap);
cudaError_t launch_st_do(const float* O, const float* arow, int R, int d, float* dO, cudaStream_t st, int cap);
cudaError_t launch_onehot(const int* code, int R, int K, float* Hm, cudaStream_t st, int cap);
cudaError_t launch_quant_residual(const float* X, const int* code, const float* T, const float* cb, int R, int d,
                                  float* Y, float* V, cudaStream_t st, int cap);
// out[z][n] (+)= sum of rows z G .. z G + G - 1 of column n; a single group of many rows is summed
// in row slabs through part (part_cap floats) when given, in a fixed order
cudaError_t launch_colsum(const float* X, int rows, int G, int ncol, float* out, long long out_stride, int accumulate,
                          cudaStream_t st, int cap, float* part = nullptr, int part_cap = 0);
cudaError_t launch_embed_bwd(const float* dX0, const uint8_t* spins, int S, int N, int d, int G, float* dtok,
                             float* dpos, long long out_stride, int accumulate, cudaStream_t st, int cap);
// stats [R][H]: the forward's (maximum scaled score, sum of exp(score - maximum)) per row and head; O the
// forward's attention output; Dst [R][H] receives dO . O per row and head
cudaError_t launch_attention_bwd(const float* QKV, const float* O, const float* dO, const float2* stats, int S, int N,
                                 int d, int H, float* dQKV, float* Dst, cudaStream_t st, int cap);
cudaError_t launch_seeds_from_eloc(const float* e_loc, int B, float* seeds, cudaStream_t st);
// sharded energy gradient: partials [2P + 3] = (sum E O, sum O, sum E, sum E^2, n), and their combination
cudaError_t launch_grad_partials(const float* s_eo, const float* s_o, long long P, const float* e_loc, int B,
                                 double* out, cudaStream_t st, int cap);
cudaError_t launch_energy_grad_combine(const double* part, long long P, float* grad, double* mean_var, cudaStream_t st,
                                       int cap);
cudaError_t launch_sub_scaled_rows(float* out, const float* csum, const float* W, int K, int d, int groups,
                                   long long stride, cudaStream_t st, int cap);

}  // namespace vq
