// General FP32 CUDA-core GEMM used by the hand-written backward pass:
//
//   C_z[M, N] (+)= op(A_z)[M, K] @ op(B_z)[K, N]      for z = 0 .. batch-1
//
// op(A) = A ([M][lda]) or A^T (A stored [K][lda]); op(B) = B ([K][ldb]) or B^T
// (B stored [N][ldb]); every batch z offsets A, B, C by its own stride.  The
// backward uses it for dX = dY W^T, for dW = X^T dY summed over all rows (the
// weighted energy gradient) and, batched over samples, for per-sample dW (O_k).
// Same 128x128x8 tiling and 8x8 register blocks as the forward GEMM; loads are
// element-guarded so any M, N, K work.
#include "vqnqs_internal.cuh"

namespace vq {

constexpr int GG_BM = 128, GG_BN = 128, GG_BK = 8, GG_THREADS = 256;

template <bool TA, bool TB>
__device__ __forceinline__ void gg_load(const float* __restrict__ A, const float* __restrict__ B, int lda, int ldb,
                                        int M, int N, int K, int m0, int n0, int k0, int tid, float (&ra)[4],
                                        float (&rb)[4]) {
    if (!TA) {  // A[m][k]: thread loads 4 consecutive k of row m
        const int m = m0 + (tid >> 1), k = k0 + (tid & 1) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) ra[i] = (m < M && k + i < K) ? A[(size_t)m * lda + k + i] : 0.f;
    } else {    // A stored [k][m]: thread loads 4 consecutive m of row k
        const int k = k0 + (tid >> 5), m = m0 + (tid & 31) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) ra[i] = (k < K && m + i < M) ? A[(size_t)k * lda + m + i] : 0.f;
    }
    if (!TB) {  // B[k][n]: 4 consecutive n of row k
        const int k = k0 + (tid >> 5), n = n0 + (tid & 31) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) rb[i] = (k < K && n + i < N) ? B[(size_t)k * ldb + n + i] : 0.f;
    } else {    // B stored [n][k]: 4 consecutive k of row n
        const int n = n0 + (tid >> 1), k = k0 + (tid & 1) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) rb[i] = (n < N && k + i < K) ? B[(size_t)n * ldb + k + i] : 0.f;
    }
}

template <bool TA, bool TB>
__device__ __forceinline__ void gg_store(float (*As)[GG_BM], float (*Bs)[GG_BN], int tid, const float (&ra)[4],
                                         const float (&rb)[4]) {
    if (!TA) {
        const int m = tid >> 1, k = (tid & 1) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) As[k + i][m] = ra[i];
    } else {
        const int k = tid >> 5, m = (tid & 31) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) As[k][m + i] = ra[i];
    }
    if (!TB) {
        const int k = tid >> 5, n = (tid & 31) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) Bs[k][n + i] = rb[i];
    } else {
        const int n = tid >> 1, k = (tid & 1) * 4;
#pragma unroll
        for (int i = 0; i < 4; ++i) Bs[k + i][n] = rb[i];
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(GG_THREADS, 2)
k_gemm_gen(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ C, int M, int N, int K,
           int lda, int ldb, int ldc, long long sA, long long sB, long long sC, int batch, int accumulate) {
    __shared__ __align__(16) float As[2][GG_BK][GG_BM];
    __shared__ __align__(16) float Bs[2][GG_BK][GG_BN];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int n_tiles = (N + GG_BN - 1) / GG_BN, m_tiles = (M + GG_BM - 1) / GG_BM;
    const long long per = (long long)m_tiles * n_tiles;
    for (long long t = blockIdx.x; t < per * batch; t += gridDim.x) {
        const int z = (int)(t / per);
        const int tt = (int)(t - (long long)z * per);
        const int m0 = (tt / n_tiles) * GG_BM, n0 = (tt % n_tiles) * GG_BN;
        const float* Az = A + z * sA;
        const float* Bz = B + z * sB;
        float* Cz = C + z * sC;
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
        float ra[4], rb[4];
        gg_load<TA, TB>(Az, Bz, lda, ldb, M, N, K, m0, n0, 0, tid, ra, rb);
        gg_store<TA, TB>(As[0], Bs[0], tid, ra, rb);
        __syncthreads();
        int buf = 0;
        for (int k0 = 0; k0 < K; k0 += GG_BK) {
            const bool more = (k0 + GG_BK) < K;
            if (more) gg_load<TA, TB>(Az, Bz, lda, ldb, M, N, K, m0, n0, k0 + GG_BK, tid, ra, rb);
#pragma unroll
            for (int kk = 0; kk < GG_BK; ++kk) {
                float a[8], b[8];
                float4 q = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
                a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
                q = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
                a[4] = q.x; a[5] = q.y; a[6] = q.z; a[7] = q.w;
                q = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
                b[0] = q.x; b[1] = q.y; b[2] = q.z; b[3] = q.w;
                q = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
                b[4] = q.x; b[5] = q.y; b[6] = q.z; b[7] = q.w;
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            if (more) {
                gg_store<TA, TB>(As[buf ^ 1], Bs[buf ^ 1], tid, ra, rb);
                __syncthreads();
                buf ^= 1;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
                if (n >= N) continue;
                float* c = Cz + (size_t)m * ldc + n;
                *c = accumulate ? *c + acc[i][j] : acc[i][j];
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_gemm_gen(bool ta, bool tb, const float* A, const float* B, float* C, int M, int N, int K, int lda,
                            int ldb, int ldc, long long sA, long long sB, long long sC, int batch, int accumulate,
                            cudaStream_t st, int num_sms) {
    if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
    long long tiles = (long long)((M + GG_BM - 1) / GG_BM) * ((N + GG_BN - 1) / GG_BN) * batch;
    int grid = (int)(tiles < 4LL * num_sms ? tiles : 4LL * num_sms);
    if (ta && tb) k_gemm_gen<true, true><<<grid, GG_THREADS, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, accumulate);
    else if (ta) k_gemm_gen<true, false><<<grid, GG_THREADS, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, accumulate);
    else if (tb) k_gemm_gen<false, true><<<grid, GG_THREADS, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, accumulate);
    else k_gemm_gen<false, false><<<grid, GG_THREADS, 0, st>>>(A, B, C, M, N, K, lda, ldb, ldc, sA, sB, sC, batch, accumulate);
    return cudaGetLastError();
}

}  // namespace vq
