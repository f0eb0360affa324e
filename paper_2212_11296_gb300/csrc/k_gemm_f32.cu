// FP32 CUDA-core GEMM for the per-location operations (Sec. 3.2): QKV projection,
// MLP up (+GELU) and MLP down (+residual).  C[M,N] = A[M,K] @ B[K,N] + bias.
//
// 128x128 output tile per CTA, K step 8, 256 threads with an 8x8 register
// block each, double-buffered shared memory, persistent over tiles with the
// row count M read from device memory (so the launch needs no host sync).
// Every output element accumulates k = 0..K-1 in the same order regardless of
// which other rows share its tile: a row's result depends only on that row.
#include "vqnqs_internal.cuh"

namespace vq {

constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8, SG_THREADS = 256;

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

template <int EPI>
__global__ void __launch_bounds__(SG_THREADS, 2)
k_sgemm(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ bias,
        const float* __restrict__ R, float* __restrict__ C, const int* __restrict__ counters, int u_slot, int N,
        int K) {
    __shared__ __align__(16) float As[2][SG_BK][SG_BM];
    __shared__ __align__(16) float Bs[2][SG_BK][SG_BN];
    const int M = counters[u_slot];
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int n_tiles = (N + SG_BN - 1) / SG_BN;
    const int m_tiles = (M + SG_BM - 1) / SG_BM;
    const int a_row = tid >> 1, a_k = (tid & 1) * 4;
    const int b_k = tid >> 5, b_col = (tid & 31) * 4;

    for (int tile = blockIdx.x; tile < m_tiles * n_tiles; tile += gridDim.x) {
        const int m0 = (tile / n_tiles) * SG_BM, n0 = (tile % n_tiles) * SG_BN;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

        const bool a_ok = (m0 + a_row) < M;
        const bool b_ok = (n0 + b_col) < N;
        const float* a_ptr = A + (size_t)(m0 + a_row) * K + a_k;
        const float* b_ptr = B + (size_t)b_k * N + n0 + b_col;
        float4 ra = a_ok ? *reinterpret_cast<const float4*>(a_ptr) : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 rb = b_ok ? *reinterpret_cast<const float4*>(b_ptr) : make_float4(0.f, 0.f, 0.f, 0.f);
        As[0][a_k + 0][a_row] = ra.x; As[0][a_k + 1][a_row] = ra.y;
        As[0][a_k + 2][a_row] = ra.z; As[0][a_k + 3][a_row] = ra.w;
        *reinterpret_cast<float4*>(&Bs[0][b_k][b_col]) = rb;
        __syncthreads();

        int buf = 0;
        for (int k0 = 0; k0 < K; k0 += SG_BK) {
            const bool more = (k0 + SG_BK) < K;
            if (more) {
                ra = a_ok ? *reinterpret_cast<const float4*>(a_ptr + k0 + SG_BK) : make_float4(0.f, 0.f, 0.f, 0.f);
                rb = b_ok ? *reinterpret_cast<const float4*>(b_ptr + (size_t)(k0 + SG_BK) * N)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int kk = 0; kk < SG_BK; ++kk) {
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
            }
            if (more) {
                const int nb = buf ^ 1;
                As[nb][a_k + 0][a_row] = ra.x; As[nb][a_k + 1][a_row] = ra.y;
                As[nb][a_k + 2][a_row] = ra.z; As[nb][a_k + 3][a_row] = ra.w;
                *reinterpret_cast<float4*>(&Bs[nb][b_k][b_col]) = rb;
                __syncthreads();
                buf = nb;
            }
        }

        // epilogue
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (m >= M) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n = n0 + h * 64 + tx * 4;
                if (n >= N) continue;
                float v[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float x = acc[i][h * 4 + j] + bias[n + j];
                    if (EPI == EPI_BIAS_GELU) x = gelu_erf(x);
                    v[j] = x;
                }
                if (EPI == EPI_BIAS_RESID) {
                    float4 r = *reinterpret_cast<const float4*>(R + (size_t)m * N + n);
                    v[0] += r.x; v[1] += r.y; v[2] += r.z; v[3] += r.w;
                }
                *reinterpret_cast<float4*>(C + (size_t)m * N + n) = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_sgemm(const float* A, const float* B, const float* bias, const float* R, float* C,
                         const int* counters, int u_slot, int Mmax, int N, int K, int epi, cudaStream_t st,
                         int num_sms) {
    if ((N % 4) || (K % SG_BK)) return cudaErrorInvalidValue;
    long long tiles = (long long)((Mmax + SG_BM - 1) / SG_BM) * ((N + SG_BN - 1) / SG_BN);
    int grid = (int)(tiles < 2LL * num_sms ? tiles : 2LL * num_sms);
    if (grid < 1) grid = 1;
    switch (epi) {
        case EPI_BIAS: k_sgemm<EPI_BIAS><<<grid, SG_THREADS, 0, st>>>(A, B, bias, R, C, counters, u_slot, N, K); break;
        case EPI_BIAS_GELU:
            k_sgemm<EPI_BIAS_GELU><<<grid, SG_THREADS, 0, st>>>(A, B, bias, R, C, counters, u_slot, N, K);
            break;
        case EPI_BIAS_RESID:
            k_sgemm<EPI_BIAS_RESID><<<grid, SG_THREADS, 0, st>>>(A, B, bias, R, C, counters, u_slot, N, K);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vq
