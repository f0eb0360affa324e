// Internal declarations shared by the kernel translation units of libvqnqs.
#pragma once

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
    CNT_U0 = 2,     // CNT_U0 + l: unique rows feeding layer l (l = 0..layers)
    CNT_SLOTS = 2 + VQNQS_MAX_LAYERS + 2
};

// Slots of the context's persistent device statistics (int64).
enum {
    ST_SAMPLES = 0,
    ST_CONFIGS = 1,
    ST_ROWS = 2,
    ST_NEAR_TIES = 3,
    ST_U0 = 4,      // ST_U0 + l
    ST_SLOTS = 4 + VQNQS_MAX_LAYERS + 2
};

struct LayerW {
    const float *ln1_g, *ln1_b, *w_qkv, *b_qkv, *codebook, *w_o, *b_o;
    const float *ln2_g, *ln2_b, *w_1, *b_1, *w_2, *b_2;
    float* T;       // [K][d] codebook @ w_o + b_o: the quantized vector after the output projection
    float* cnorm;   // [K] ||W_j||^2
    __nv_bfloat16 *wqkv_t, *w1_t, *w2_t;  // BF16 transposes [out][in] for the tensor-core GEMMs
};

// Per-chunk view of the problem handed to the kernels.
struct Chunk {
    const uint8_t* spins;   // [S][N] spins of this chunk's samples
    int S;                  // samples in the chunk
    int N, L, d, heads, K;
    const int* cfg_sample;  // [C] sample of each configuration
    const int* cfg_i;       // [C] exchanged site pair (-1 for the sample itself)
    const int* cfg_j;
    const int* cfg_off;     // [S + 1] first configuration of each sample
    int* counters;          // CNT_* slots
};

__device__ __forceinline__ int cfg_spin(const uint8_t* spins, int N, int b, int ci, int cj, int q) {
    int src = q;
    if (q == ci) src = cj;
    else if (q == cj) src = ci;
    return spins[(size_t)b * N + src];
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

// configuration enumeration (k_config.cu)
cudaError_t launch_count_configs(const uint8_t* spins, int S, int N, const int* bonds, int nb, float J,
                                 int with_bonds, int* cnt, float* diag, int* status, cudaStream_t st, int grid);
cudaError_t launch_scan_configs(const int* cnt, int S, int* cfg_off, int* counters, int N, cudaStream_t st);
cudaError_t launch_fill_configs(const uint8_t* spins, int S, int N, const int* bonds, int nb, int with_bonds,
                                const int* cfg_off, int* cfg_sample, int* cfg_i, int* cfg_j, cudaStream_t st,
                                int grid);
cudaError_t launch_embed(const Chunk& ch, const float* tok_emb, const float* pos_emb, int reuse, float* X0,
                         int* uid0, cudaStream_t st, int grid);
cudaError_t launch_head(const float* X, const int* counters, int u_slot, const float* g, const float* b,
                        const float* w_head, const float* b_head, int d, float* logp, cudaStream_t st, int grid);
cudaError_t launch_eloc(const Chunk& ch, const int* uid, const float* logp, float* ratio, float* log_psi_out,
                        cudaStream_t st, int grid);
cudaError_t launch_eloc_reduce(const Chunk& ch, const float* diag, const float* ratio, float J, float* e_loc_out,
                               cudaStream_t st, int grid);
cudaError_t launch_mean_var(const float* e_loc, int B, double* mean_var, cudaStream_t st);
cudaError_t launch_accumulate_stats(const int* counters, int layers, int S, long long* stats, cudaStream_t st);

// LayerNorm and per-location helpers (k_rowops.cu)
cudaError_t launch_layernorm(const float* X, const int* counters, int u_slot, const float* g, const float* b, int d,
                             float* out_f32, __nv_bfloat16* out_bf16, cudaStream_t st, int grid);
cudaError_t launch_residual_vq_ln(const float* X, const int* rep_uid, const int* rep_code, const float* T,
                                  const int* counters, int u_slot, const float* g, const float* b, int d, float* Y,
                                  float* A_f32, __nv_bfloat16* A_bf16, cudaStream_t st, int grid);
cudaError_t launch_table_T(const float* codebook, const float* w_o, const float* b_o, int K, int d, float* T,
                           float* cnorm, cudaStream_t st);
cudaError_t launch_transpose_bf16(const float* W, int rows, int cols, __nv_bfloat16* WT, cudaStream_t st);

// FP32 SIMT GEMM (k_gemm_f32.cu): C[M,N] = A[M,K] @ B[K,N] + bias (+GELU) (+R); M = counters[u_slot]
enum { EPI_BIAS = 0, EPI_BIAS_GELU = 1, EPI_BIAS_RESID = 2 };
cudaError_t launch_sgemm(const float* A, const float* B, const float* bias, const float* R, float* C,
                         const int* counters, int u_slot, int Mmax, int N, int K, int epi, cudaStream_t st,
                         int num_sms);

// attention (k_attn.cu): O[r] for rows r < counters[CNT_R]
cudaError_t launch_attention_f32(const Chunk& ch, const int* uid, const float* qkv, float* O, cudaStream_t st,
                                 int grid);

// nearest codeword (k_vq.cu)
cudaError_t launch_vq_argmin(const float* O, const int* counters, const float* codebook, const float* cnorm, int K,
                             int d, int* code, long long* near_ties, int Rmax, cudaStream_t st, int num_sms);

// dedupe (k_dedupe.cu)
cudaError_t launch_dedupe(const int* uid_cur, const int* code, int* counters, int u_slot_next, int Rmax,
                          unsigned long long* keys, int* vals, int hash_bits, int* uid_next, int* rep_uid,
                          int* rep_code, int reuse, int* status, cudaStream_t st, int num_sms);

}  // namespace vq
