// Autoregressive direct sampling (Sec. 2: psi = sqrt(P), P(s) = prod_p P(s_p | s_<p),
// so configurations are drawn exactly from |psi|^2 one site at a time).
//
// A batch of S samples advances one position p at a time: the token at p (the
// spin drawn at p - 1, begin-of-sequence at p = 0) goes through every block,
// whose attention reads the keys and values of positions 0..p kept in a
// per-layer cache, and the head's conditional P(up | s_<p) decides the spin at
// p against the given uniform number: up when u < P(up).  The per-location
// steps (LayerNorm, GEMMs, nearest codeword, residual) run as the local-energy
// path's kernels on the S rows; this file holds the steps specific to
// sampling.
#include <algorithm>

#include "vqnqs_internal.cuh"

namespace vq {

namespace {

template <typename T>
__device__ __forceinline__ float tof(T x);
template <>
__device__ __forceinline__ float tof<float>(float x) { return x; }
template <>
__device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

}  // namespace

// X[b] = tok_emb[token] + pos_emb[p]; the token is the spin drawn at p - 1.
__global__ void k_sample_embed(int S, int p, int N, int d, const uint8_t* __restrict__ spins,
                               const float* __restrict__ tok_emb, const float* __restrict__ pos_emb,
                               float* __restrict__ X) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)S * d; e += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / d), k = (int)(e - (size_t)b * d);
        const int tok = p == 0 ? BOS : (spins[(size_t)b * N + p - 1] & 1);
        X[e] = tok_emb[(size_t)tok * d + k] + pos_emb[(size_t)p * d + k];
    }
}

// One warp per (sample, head): the new row's key and value go to cache[b][p]
// (layout [S][N][2d]: keys, then values), then softmax(q k^T / sqrt(dh)) v over
// positions 0..p.  The weights of a warp sit in shared memory (N floats).
template <typename T, int DH>
__global__ void __launch_bounds__(256)
k_decode_attention(int S, int p, int N, int d, int H, const T* __restrict__ qkv, T* __restrict__ cache,
                   float* __restrict__ O) {
    extern __shared__ float s_w[];  // [8 warps][N]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float* P = s_w + warp * N;
    const float scale = rsqrtf((float)DH);
    for (int item = blockIdx.x * 8 + warp; item < S * H; item += gridDim.x * 8) {
        const int b = item / H, h = item - b * H;
        const T* row = qkv + (size_t)b * 3 * d;
        T* cb = cache + (size_t)b * N * 2 * d;
        if (lane < DH) {
            cb[(size_t)p * 2 * d + h * DH + lane] = row[d + h * DH + lane];
            cb[(size_t)p * 2 * d + d + h * DH + lane] = row[2 * d + h * DH + lane];
        }
        __syncwarp();
        float q[DH];
#pragma unroll
        for (int t = 0; t < DH; ++t) q[t] = tof(row[h * DH + t]);
        float mx = -INFINITY;
        for (int j = lane; j <= p; j += 32) {
            const T* k = cb + (size_t)j * 2 * d + h * DH;
            float s = 0.f;
#pragma unroll
            for (int t = 0; t < DH; ++t) s = fmaf(q[t], tof(k[t]), s);
            s *= scale;
            P[j] = s;
            mx = fmaxf(mx, s);
        }
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        float l = 0.f;
        for (int j = lane; j <= p; j += 32) {
            const float e = expf(P[j] - mx);
            P[j] = e;
            l += e;
        }
        l = warp_sum(l);
        __syncwarp();
        if (lane < DH) {
            float a = 0.f;
            for (int j = 0; j <= p; ++j) a = fmaf(P[j], tof(cb[(size_t)j * 2 * d + d + h * DH + lane]), a);
            O[(size_t)b * d + h * DH + lane] = a / l;
        }
        __syncwarp();
    }
}

// s_p = up when u[b][p] < P(up | s_<p); log psi accumulates half the chosen log conditional.
__global__ void k_sample_draw(int S, int p, int N, const float* __restrict__ logp, const float* __restrict__ u,
                              uint8_t* __restrict__ spins, float* __restrict__ log_psi) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < S; b += gridDim.x * blockDim.x) {
        const float lup = logp[2 * (size_t)b + 1];
        const int s = u[(size_t)b * N + p] < expf(lup) ? 1 : 0;
        spins[(size_t)b * N + p] = (uint8_t)s;
        const float lc = s ? lup : logp[2 * (size_t)b];
        log_psi[b] = (p == 0 ? 0.f : log_psi[b]) + 0.5f * lc;
    }
}

cudaError_t launch_sample_embed(int S, int p, int N, int d, const uint8_t* spins, const float* tok_emb,
                                const float* pos_emb, float* X, cudaStream_t st) {
    const size_t n = (size_t)S * d;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    k_sample_embed<<<grid, 256, 0, st>>>(S, p, N, d, spins, tok_emb, pos_emb, X);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_decode_attention_t(int S, int p, int N, int d, int H, const T* qkv, T* cache, float* O,
                                      cudaStream_t st) {
    const int dh = d / H;
    const size_t smem = (size_t)8 * N * sizeof(float);
    const int grid = (S * H + 7) / 8;
    switch (dh) {
        case 8: k_decode_attention<T, 8><<<grid, 256, smem, st>>>(S, p, N, d, H, qkv, cache, O); break;
        case 16: k_decode_attention<T, 16><<<grid, 256, smem, st>>>(S, p, N, d, H, qkv, cache, O); break;
        case 32: k_decode_attention<T, 32><<<grid, 256, smem, st>>>(S, p, N, d, H, qkv, cache, O); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
cudaError_t launch_decode_attention(int S, int p, int N, int d, int H, const float* qkv, float* cache, float* O,
                                    cudaStream_t st) {
    return launch_decode_attention_t<float>(S, p, N, d, H, qkv, cache, O, st);
}
cudaError_t launch_decode_attention(int S, int p, int N, int d, int H, const __nv_bfloat16* qkv,
                                    __nv_bfloat16* cache, float* O, cudaStream_t st) {
    return launch_decode_attention_t<__nv_bfloat16>(S, p, N, d, H, qkv, cache, O, st);
}

cudaError_t launch_sample_draw(int S, int p, int N, const float* logp, const float* u, uint8_t* spins,
                               float* log_psi, cudaStream_t st) {
    const int grid = (S + 255) / 256;
    k_sample_draw<<<grid, 256, 0, st>>>(S, p, N, logp, u, spins, log_psi);
    return cudaGetLastError();
}

}  // namespace vq
