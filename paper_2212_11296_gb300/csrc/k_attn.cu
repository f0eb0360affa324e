// Causal multi-head self-attention, FP32 on CUDA cores (Sec. 3.1 location mixer).
//
// One CTA per (configuration, head): the configuration's K and V rows for that
// head are gathered by row id into shared memory, then each thread owns one
// query position p and runs an online softmax over keys 0..p in chunks of 4.
// The chunk loop is warp-uniform; chunks past a thread's own p are exact
// no-ops (scale 1, weight 0), so a row's output never depends on which other
// rows share its warp.  The attention output (before W_o) goes to O[row].
// The Q/K/V input is FP32 (plain path) or BF16 (BF16 path: the QKV GEMM's
// rounded output); products and sums are FP32 either way.
#include "vqnqs_internal.cuh"

namespace vq {

__device__ __forceinline__ float4 load4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 load4(const __nv_bfloat16* p) {
    uint2 u = *reinterpret_cast<const uint2*>(p);
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x), b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    return make_float4(fa.x, fa.y, fb.x, fb.y);
}

// cfg_list (optional): the configurations to process, n_list of them (all
// configurations of the chunk when NULL).  stats (optional): the softmax
// maximum of the scaled scores and the sum of exp(score - maximum) of every
// computed (row, head), at [(sample * N + p) * heads + head].
template <int DH, typename T>
__global__ void k_attention_f32(Chunk ch, const int* __restrict__ uid, const T* __restrict__ qkv,
                                float* __restrict__ O, int prefix_reuse, const int* __restrict__ cfg_list,
                                int n_list, float2* __restrict__ stats) {
    extern __shared__ __align__(16) float s_kv[];  // [N][DH] keys then [N][DH] values
    const int d = ch.d, H = ch.heads;
    const int C = cfg_list ? n_list : ch.counters[CNT_C];
    const float scale = rsqrtf((float)DH);
    float* sK = s_kv;
    float* sV = s_kv + (size_t)ch.N * DH;
    const int ld = 3 * d;
    for (int item = blockIdx.x; item < C * H; item += gridDim.x) {
        const int ci = item / H, h = item - ci * H;
        const int c = cfg_list ? cfg_list[ci] : ci;
        const int N = cfg_N(ch, c);
        const int* urow = uid + ch.cfg_row[c];
        for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
            int j = e / (DH / 4), t4 = (e - j * (DH / 4)) * 4;
            const T* src = qkv + (size_t)urow[j] * ld + h * DH + t4;
            *reinterpret_cast<float4*>(&sK[j * DH + t4]) = load4(src + d);
            *reinterpret_cast<float4*>(&sV[j * DH + t4]) = load4(src + 2 * d);
        }
        __syncthreads();
        const int p = threadIdx.x;
        const int p0 = prefix_reuse ? cfg_p0(ch, c) : 0;
        const bool active = p < N && p >= p0;
        float q[DH], acc[DH];
        if (active) {
            const T* src = qkv + (size_t)urow[p] * ld + h * DH;
#pragma unroll
            for (int t = 0; t < DH; t += 4) {
                float4 v = load4(src + t);
                q[t] = v.x; q[t + 1] = v.y; q[t + 2] = v.z; q[t + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int t = 0; t < DH; ++t) q[t] = 0.f;
        }
#pragma unroll
        for (int t = 0; t < DH; ++t) acc[t] = 0.f;
        float m = -INFINITY, l = 0.f;
        // warp-uniform bound: the largest p in this warp (no keys at all when the
        // whole warp lies before the first changed position)
        int pw = min(N - 1, (int)(threadIdx.x | 31));
        if (pw < p0) pw = -1;
        for (int j0 = 0; j0 <= pw; j0 += 4) {
            float s[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int j = j0 + i;
                float dot = 0.f;
                if (j < N) {
#pragma unroll
                    for (int t = 0; t < DH; t += 4) {
                        float4 k4 = *reinterpret_cast<const float4*>(&sK[j * DH + t]);
                        dot = fmaf(q[t], k4.x, dot);
                        dot = fmaf(q[t + 1], k4.y, dot);
                        dot = fmaf(q[t + 2], k4.z, dot);
                        dot = fmaf(q[t + 3], k4.w, dot);
                    }
                }
                s[i] = (active && j <= p) ? dot * scale : -INFINITY;
            }
            const float mx = fmaxf(fmaxf(s[0], s[1]), fmaxf(s[2], s[3]));
            const float mn = fmaxf(m, mx);
            const float corr = (mn == -INFINITY) ? 1.f : expf(m - mn);
            float e[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) e[i] = (s[i] == -INFINITY) ? 0.f : expf(s[i] - mn);
            l = l * corr + ((e[0] + e[1]) + (e[2] + e[3]));
#pragma unroll
            for (int t = 0; t < DH; t += 4) {
                float a0 = acc[t] * corr, a1 = acc[t + 1] * corr, a2 = acc[t + 2] * corr, a3 = acc[t + 3] * corr;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int j = min(j0 + i, N - 1);
                    float4 v4 = *reinterpret_cast<const float4*>(&sV[j * DH + t]);
                    a0 = fmaf(e[i], v4.x, a0);
                    a1 = fmaf(e[i], v4.y, a1);
                    a2 = fmaf(e[i], v4.z, a2);
                    a3 = fmaf(e[i], v4.w, a3);
                }
                acc[t] = a0; acc[t + 1] = a1; acc[t + 2] = a2; acc[t + 3] = a3;
            }
            m = mn;
        }
        if (active) {
            if (stats) stats[((size_t)ch.cfg_sample[c] * ch.N + p) * H + h] = make_float2(m, l);
            const float inv = 1.f / l;
            float* dst = O + ((size_t)ch.cfg_row[c] + p) * d + h * DH;
#pragma unroll
            for (int t = 0; t < DH; t += 4)
                *reinterpret_cast<float4*>(dst + t) =
                    make_float4(acc[t] * inv, acc[t + 1] * inv, acc[t + 2] * inv, acc[t + 3] * inv);
        }
        __syncthreads();
    }
}

// Largest dynamic shared memory already granted to an instantiation (the
// attribute is set outside any stream capture, on the first call that needs it).
template <int X, typename T>
size_t set_attr_once(size_t v) {
    static size_t granted = 0;
    if (v > granted) granted = v;
    return granted;
}

template <typename T>
cudaError_t launch_attention_t(const Chunk& ch, const int* uid, const T* qkv, float* O, int prefix_reuse,
                               cudaStream_t st, int grid, const int* cfg_list, int n_list, float2* stats) {
    const int DH = ch.d / ch.heads;
    const int threads = ((ch.N + 31) / 32) * 32;
    const size_t smem = (size_t)2 * ch.N * DH * sizeof(float);
    if (threads > 1024) return cudaErrorInvalidValue;
    switch (DH) {
#define VQ_ATT_CASE(X)                                                                                        \
    case X:                                                                                                   \
        if (smem > 48 * 1024 && smem > set_attr_once<X, T>(0)) {                                              \
            cudaFuncSetAttribute(k_attention_f32<X, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            set_attr_once<X, T>(smem);                                                                        \
        }                                                                                                     \
        k_attention_f32<X, T><<<grid, threads, smem, st>>>(ch, uid, qkv, O, prefix_reuse, cfg_list, n_list, stats); \
        break;
        VQ_ATT_CASE(8)
        VQ_ATT_CASE(16)
        VQ_ATT_CASE(32)
#undef VQ_ATT_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_attention_f32(const Chunk& ch, const int* uid, const float* qkv, float* O, int prefix_reuse,
                                 cudaStream_t st, int grid, const int* cfg_list, int n_list, float2* stats) {
    return launch_attention_t<float>(ch, uid, qkv, O, prefix_reuse, st, grid, cfg_list, n_list, stats);
}

cudaError_t launch_attention_bf16in(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                                   int prefix_reuse, cudaStream_t st, int grid, const int* cfg_list, int n_list,
                                   float2* stats) {
    return launch_attention_t<__nv_bfloat16>(ch, uid, qkv, O, prefix_reuse, st, grid, cfg_list, n_list, stats);
}

}  // namespace vq
