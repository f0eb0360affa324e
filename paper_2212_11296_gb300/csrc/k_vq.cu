// Nearest-codeword assignment, FP32 on CUDA cores (Sec. 3.1, Eq. vq).
//
//   code(o) = argmin_j ||o - W_j||^2 = argmin_j (||W_j||^2 - 2 o . W_j),  lowest j on ties.
//
// With H quantizer heads each segment o_h (d / H values, row stride d) is
// assigned against its own codebook by one launch, and the packed code holds
// c_h in bits [h * bits, (h + 1) * bits).  Codes wider than one word (Table 1's
// 8 heads of 64 codes: 48 bits) take two: head h goes to word h / hpw at bit
// (h % hpw) * bits, hpw = 32 / bits heads per word.
//
// The o . W_j products are a [rows x d] x [d x K] contraction tiled like the
// FP32 GEMM (128 rows x 128 codewords per pass, 8x8 per thread); the epilogue
// keeps (best, index, second best) per row in registers and merges across the
// 16 threads that share a row with butterfly shuffles (an order-independent
// merge, so every lane ends with the same answer).  Rows whose relative gap
// (l2 - l1) / l1 between the best two squared distances is below 1e-6 are
// counted as near ties.
#include "vqnqs_internal.cuh"

namespace vq {

constexpr int VQ_BM = 128, VQ_BN = 128, VQ_BK = 8, VQ_THREADS = 256;

struct Best {
    float v1;
    int i1;
    float v2;
};

__device__ __forceinline__ void best_merge(Best& a, float c1, int j1, float c2) {
    if (c1 < a.v1 || (c1 == a.v1 && j1 < a.i1)) {
        a.v2 = fminf(a.v1, c2);
        a.v1 = c1;
        a.i1 = j1;
    } else {
        a.v2 = fminf(a.v2, c1);
    }
}

__global__ void __launch_bounds__(VQ_THREADS, 2)
k_vq_argmin(const float* __restrict__ O, int ldo, const int* __restrict__ counters, const int* __restrict__ act_rows,
            const float* __restrict__ W, const float* __restrict__ cnorm, int K, int d, int* __restrict__ code,
            int shift, int accumulate, long long* __restrict__ near_ties, int a_slot) {
    __shared__ __align__(16) float As[2][VQ_BK][VQ_BM];
    __shared__ __align__(16) float Bs[2][VQ_BK][VQ_BN];  // Bs[k][j] = W[j][k]
    __shared__ int s_ties;
    const int R = act_rows ? counters[a_slot] : counters[CNT_R];  // rows to assign
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int a_row = tid >> 1, a_k = (tid & 1) * 4;
    const int b_j = tid >> 1, b_k = (tid & 1) * 4;  // codeword rows are loaded like A rows
    if (tid == 0) s_ties = 0;

    for (int m0 = blockIdx.x * VQ_BM; m0 < R; m0 += gridDim.x * VQ_BM) {
        Best best[8];
        float osq[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) { best[i].v1 = INFINITY; best[i].i1 = 0x7fffffff; best[i].v2 = INFINITY; osq[i] = 0.f; }
        const bool a_ok = (m0 + a_row) < R;
        const int a_src = a_ok ? (act_rows ? act_rows[m0 + a_row] : m0 + a_row) : 0;
        const float* a_ptr = O + (size_t)a_src * ldo + a_k;

        for (int n0 = 0; n0 < K; n0 += VQ_BN) {
            float acc[8][8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
            const bool b_ok = (n0 + b_j) < K;
            const float* b_ptr = W + (size_t)(n0 + b_j) * d + b_k;
            float4 ra = a_ok ? *reinterpret_cast<const float4*>(a_ptr) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 rb = b_ok ? *reinterpret_cast<const float4*>(b_ptr) : make_float4(0.f, 0.f, 0.f, 0.f);
            As[0][a_k][a_row] = ra.x; As[0][a_k + 1][a_row] = ra.y; As[0][a_k + 2][a_row] = ra.z; As[0][a_k + 3][a_row] = ra.w;
            Bs[0][b_k][b_j] = rb.x; Bs[0][b_k + 1][b_j] = rb.y; Bs[0][b_k + 2][b_j] = rb.z; Bs[0][b_k + 3][b_j] = rb.w;
            __syncthreads();
            int buf = 0;
            for (int k0 = 0; k0 < d; k0 += VQ_BK) {
                const bool more = (k0 + VQ_BK) < d;
                if (more) {
                    ra = a_ok ? *reinterpret_cast<const float4*>(a_ptr + k0 + VQ_BK) : make_float4(0.f, 0.f, 0.f, 0.f);
                    rb = b_ok ? *reinterpret_cast<const float4*>(b_ptr + k0 + VQ_BK) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int kk = 0; kk < VQ_BK; ++kk) {
                    float a[8], b[8];
                    float4 t;
                    t = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
                    a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
                    t = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
                    a[4] = t.x; a[5] = t.y; a[6] = t.z; a[7] = t.w;
                    t = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
                    b[0] = t.x; b[1] = t.y; b[2] = t.z; b[3] = t.w;
                    t = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
                    b[4] = t.x; b[5] = t.y; b[6] = t.z; b[7] = t.w;
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                    if (n0 == 0) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) osq[i] = fmaf(a[i], a[i], osq[i]);
                    }
                }
                if (more) {
                    const int nb = buf ^ 1;
                    As[nb][a_k][a_row] = ra.x; As[nb][a_k + 1][a_row] = ra.y; As[nb][a_k + 2][a_row] = ra.z; As[nb][a_k + 3][a_row] = ra.w;
                    Bs[nb][b_k][b_j] = rb.x; Bs[nb][b_k + 1][b_j] = rb.y; Bs[nb][b_k + 2][b_j] = rb.z; Bs[nb][b_k + 3][b_j] = rb.w;
                    __syncthreads();
                    buf = nb;
                }
            }
            // per-thread scan of its 8 codewords, in increasing index
#pragma unroll
            for (int i = 0; i < 8; ++i) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                    if (n < K) {
                        const float sc = fmaf(-2.f, acc[i][j], cnorm[n]);
                        best_merge(best[i], sc, n, INFINITY);
                    }
                }
            }
            __syncthreads();
        }
        // merge across the 16 lanes sharing these rows (lanes 0-15 or 16-31 of the warp)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int off = 8; off > 0; off >>= 1) {
                float c1 = __shfl_xor_sync(0xffffffffu, best[i].v1, off);
                int j1 = __shfl_xor_sync(0xffffffffu, best[i].i1, off);
                float c2 = __shfl_xor_sync(0xffffffffu, best[i].v2, off);
                best_merge(best[i], c1, j1, c2);
            }
        }
        if (tx == 0) {
            int ties = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
                if (m < R) {
                    const int r = act_rows ? act_rows[m] : m;
                    const int c = best[i].i1 < K ? best[i].i1 : 0;  // no finite distance: codeword 0
                    code[r] = (accumulate ? code[r] : 0) | (c << shift);
                    const float l1 = best[i].v1 + osq[i], l2 = best[i].v2 + osq[i];
                    if (K > 1 && (l2 - l1) < NEAR_TIE_REL * fmaxf(l1, 1e-30f)) ++ties;
                }
            }
            if (ties) atomicAdd(&s_ties, ties);
        }
    }
    __syncthreads();
    if (tid == 0 && s_ties) atomicAdd(reinterpret_cast<unsigned long long*>(near_ties), (unsigned long long)s_ties);
}

__global__ void k_assign_setup(int* __restrict__ counters, int* __restrict__ rows, int R) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R; i += gridDim.x * blockDim.x) rows[i] = i;
    if (blockIdx.x == 0 && threadIdx.x == 0) { counters[CNT_A] = R; counters[CNT_R] = R; }
}

cudaError_t launch_assign_setup(int* counters, int* rows, int R, cudaStream_t st) {
    int grid = (R + 255) / 256;
    k_assign_setup<<<grid < 1024 ? (grid < 1 ? 1 : grid) : 1024, 256, 0, st>>>(counters, rows, R);
    return cudaGetLastError();
}

cudaError_t launch_vq_argmin(const float* O, const int* counters, const int* act_rows, const float* codebook,
                             const float* cnorm, int K, int d, int* code, long long* near_ties, int Rmax,
                             cudaStream_t st, int num_sms, int a_slot) {
    if (d % VQ_BK) return cudaErrorInvalidValue;
    int tiles = (Rmax + VQ_BM - 1) / VQ_BM;
    int grid = tiles < 2 * num_sms ? tiles : 2 * num_sms;
    if (grid < 1) grid = 1;
    k_vq_argmin<<<grid, VQ_THREADS, 0, st>>>(O, d, counters, act_rows, codebook, cnorm, K, d, code, 0, 0, near_ties,
                                             a_slot);
    return cudaGetLastError();
}

cudaError_t launch_vq_argmin_heads(const float* O, const int* counters, const int* act_rows, const float* codebook,
                                   const float* cnorm, int K, int d, int vq_heads, int bits, int* code,
                                   long long* near_ties, int Rmax, cudaStream_t st, int num_sms, int a_slot,
                                   int* code_hi) {
    const int dq = d / vq_heads;
    if (d % vq_heads || dq % VQ_BK || bits < 1) return cudaErrorInvalidValue;
    const int hpw = 32 / bits;  // heads per code word
    if (vq_heads > hpw && !code_hi) return cudaErrorInvalidValue;
    int tiles = (Rmax + VQ_BM - 1) / VQ_BM;
    int grid = tiles < 2 * num_sms ? tiles : 2 * num_sms;
    if (grid < 1) grid = 1;
    for (int h = 0; h < vq_heads; ++h) {  // segment h: its own codebook, its bits of its code word
        const int w = h / hpw, f = h - w * hpw;
        k_vq_argmin<<<grid, VQ_THREADS, 0, st>>>(O + (size_t)h * dq, d, counters, act_rows,
                                                 codebook + (size_t)h * K * dq, cnorm + (size_t)h * K, K, dq,
                                                 w ? code_hi : code, f * bits, f > 0 ? 1 : 0, near_ties, a_slot);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace vq
