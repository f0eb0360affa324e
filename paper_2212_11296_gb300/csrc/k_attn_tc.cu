// Causal multi-head self-attention on the tensor cores (BF16 path, Sec. 3.1
// location mixer): BF16 Q/K/V, FP32 scores and accumulation in TMEM.
//
// One work item = (configuration, head).  A CTA of 4 warps:
//   1. gathers the configuration's K rows and V rows of this head by row id
//      into shared memory (K as a [keys x dh] K-major operand, V transposed
//      to a [dh x keys] K-major operand), in the no-swizzle canonical layout
//      (8-row x 16-byte core matrices);
//   2. per 128-query tile: gathers Q, thread 0 issues S = Q K^T with
//      tcgen05.mma (M = 128, N = keys, K = dh) into TMEM;
//   3. every thread owns one query row: two passes over its TMEM row (causal
//      max, then exp2 / sum), writing P as BF16 into shared memory;
//   4. thread 0 issues O = P V (M = 128, N = dh, K = keys) into TMEM columns
//      already read; each thread scales its row by 1/sum and stores FP32 O.
// With prefix reuse, query tiles wholly before the configuration's first
// changed position are skipped and rows before it are not stored.
// Waits on the MMA barrier are bounded (VQNQS_DEV_TIMEOUT on expiry).
#include "tc_common.cuh"

namespace vq {

constexpr int AT_THREADS = 128;
constexpr int AT_MAX_N = 448;  // keys per configuration handled in one TMEM tile

__device__ __forceinline__ uint64_t desc_kmajor_none(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // version; layout type 0 = no swizzle
    return d;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// byte offset of element (r, k) in a K-major no-swizzle tile with kd columns
__device__ __forceinline__ uint32_t core_off(int r, int k, int kd) {
    return (uint32_t)((r >> 3) * (kd >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

template <int DH>
__global__ void __launch_bounds__(AT_THREADS)
k_attention_tc(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv, float* __restrict__ O,
               int prefix_reuse, int Npad, uint32_t tmem_cols, int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int N = ch.N, d = ch.d, H = ch.heads;
    uint8_t* sK = smem;                            // [Npad x DH]
    uint8_t* sVt = sK + (size_t)Npad * DH * 2;     // [DH x Npad]
    uint8_t* sQ = sVt + (size_t)Npad * DH * 2;     // [128 x DH]
    uint8_t* sP = sQ + 128 * DH * 2;               // [128 x Npad]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sP + (size_t)128 * Npad * 2);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_holder, tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    const float sl2 = 1.4426950408889634f * rsqrtf((float)DH);  // log2(e) / sqrt(dh)
    const int C = ch.counters[CNT_C];
    const int ld = 3 * d;

    for (int item = blockIdx.x; item < C * H && ok; item += gridDim.x) {
        const int c = item / H, h = item - c * H;
        const int* urow = uid + (size_t)c * N;
        const int p0 = prefix_reuse ? cfg_first_changed(ch.cfg_i[c], ch.cfg_j[c]) : 0;
        // keys and transposed values, rows >= N zero
        for (int u = tid; u < Npad * (DH / 8); u += AT_THREADS) {
            const int j = u / (DH / 8), kb = u - j * (DH / 8);
            uint4 kv = make_uint4(0, 0, 0, 0), vv = make_uint4(0, 0, 0, 0);
            if (j < N) {
                const __nv_bfloat16* src = qkv + (size_t)urow[j] * ld + h * DH + kb * 8;
                kv = *reinterpret_cast<const uint4*>(src + d);
                vv = *reinterpret_cast<const uint4*>(src + 2 * d);
            }
            *reinterpret_cast<uint4*>(sK + core_off(j, kb * 8, DH)) = kv;
            const __nv_bfloat16* ve = reinterpret_cast<const __nv_bfloat16*>(&vv);
#pragma unroll
            for (int e = 0; e < 8; ++e)
                *reinterpret_cast<__nv_bfloat16*>(sVt + core_off(kb * 8 + e, j, Npad)) = ve[e];
        }
        for (int q0 = (p0 / 128) * 128; q0 < N && ok; q0 += 128) {
            const int nk = min(N, q0 + 128);             // keys this tile can see
            const int nk16 = (nk + 15) & ~15;            // MMA N (multiple of 16)
            const int nk32 = (nk + 31) & ~31;            // columns read back
            for (int u = tid; u < 128 * (DH / 8); u += AT_THREADS) {
                const int r = u / (DH / 8), kb = u - r * (DH / 8);
                uint4 qv = make_uint4(0, 0, 0, 0);
                if (q0 + r < N) qv = *reinterpret_cast<const uint4*>(qkv + (size_t)urow[q0 + r] * ld + h * DH + kb * 8);
                *reinterpret_cast<uint4*>(sQ + core_off(r, kb * 8, DH)) = qv;
            }
            fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                const uint64_t dq = desc_kmajor_none(tc::smem_u32(sQ), 128, (DH / 8) * 128);
                const uint64_t dk = desc_kmajor_none(tc::smem_u32(sK), 128, (DH / 8) * 128);
                for (int n0 = 0; n0 < nk16; n0 += 256) {
                    const int nn = min(256, nk16 - n0);
                    const uint32_t idesc = tc::idesc_bf16_f32(128, nn);
                    // rows n0.. of K start (n0 / 8) core-row groups further
                    const uint64_t dkn = dk + (uint64_t)(((n0 / 8) * (DH / 8) * 128) >> 4);
#pragma unroll
                    for (int ks = 0; ks < DH / 16; ++ks)
                        tc::mma_bf16(tmem + n0, dq + (uint64_t)(ks * 16), dkn + (uint64_t)(ks * 16), idesc,
                                     ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            ok = __syncthreads_and(tc::mbar_wait(bar, phase, status)) != 0;
            phase ^= 1;
            tc::tc_fence_after();
            if (!ok) break;
            // softmax of this thread's row (query position p = q0 + tid)
            const int p = q0 + tid;
            const int plim = min(p, N - 1);  // keys 0..plim are visible
            float mx = -INFINITY;
            for (int c0 = 0; c0 < nk32; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + lane_base + c0, r);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (c0 + j <= plim) mx = fmaxf(mx, __uint_as_float(r[j]));
            }
            const float mb = mx * sl2;
            float sum = 0.f;
            for (int c0 = 0; c0 < nk32; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + lane_base + c0, r);
                if (c0 < nk16) {
#pragma unroll
                    for (int j8 = 0; j8 < 32; j8 += 8) {
                        if (c0 + j8 >= nk16) break;
                        uint32_t pk[4];
#pragma unroll
                        for (int e = 0; e < 8; e += 2) {
                            const int j = c0 + j8 + e;
                            float e0 = (j <= plim) ? exp2f(fmaf(__uint_as_float(r[j8 + e]), sl2, -mb)) : 0.f;
                            float e1 = (j + 1 <= plim) ? exp2f(fmaf(__uint_as_float(r[j8 + e + 1]), sl2, -mb)) : 0.f;
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(e0, e1);
                            float2 back = __bfloat1622float2(b2);
                            sum += back.x + back.y;
                            pk[e / 2] = *reinterpret_cast<uint32_t*>(&b2);
                        }
                        *reinterpret_cast<uint4*>(sP + core_off(tid, c0 + j8, Npad)) =
                            make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    }
                }
            }
            tc::tc_fence_before();
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc::tc_fence_after();
                const uint32_t idesc = tc::idesc_bf16_f32(128, DH);
                const uint64_t dp = desc_kmajor_none(tc::smem_u32(sP), 128, (Npad / 8) * 128);
                const uint64_t dv = desc_kmajor_none(tc::smem_u32(sVt), 128, (Npad / 8) * 128);
                for (int ks = 0; ks < nk16 / 16; ++ks)
                    tc::mma_bf16(tmem, dp + (uint64_t)(ks * 16), dv + (uint64_t)(ks * 16), idesc, ks > 0 ? 1u : 0u);
                tc::mma_commit(bar);
            }
            ok = __syncthreads_and(tc::mbar_wait(bar, phase, status)) != 0;
            phase ^= 1;
            tc::tc_fence_after();
            if (!ok) break;
            {
                uint32_t r[32];
                tc::tmem_ld32(tmem + lane_base, r);
                if (p < N && p >= p0) {
                    const float inv = 1.f / sum;
                    float* dst = O + ((size_t)c * N + p) * d + h * DH;
#pragma unroll
                    for (int t = 0; t < DH; t += 4)
                        *reinterpret_cast<float4*>(dst + t) =
                            make_float4(__uint_as_float(r[t]) * inv, __uint_as_float(r[t + 1]) * inv,
                                        __uint_as_float(r[t + 2]) * inv, __uint_as_float(r[t + 3]) * inv);
                }
            }
            tc::tc_fence_before();
            __syncthreads();
        }
        __syncthreads();
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
}

bool attention_tc_supported(int N, int dh) { return (dh == 16 || dh == 32) && N <= AT_MAX_N; }

cudaError_t launch_attention_tc(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O, int prefix_reuse,
                                int* status, cudaStream_t st, int grid) {
    const int DH = ch.d / ch.heads;
    if (!attention_tc_supported(ch.N, DH)) return cudaErrorInvalidValue;
    const int Npad = (ch.N + 31) & ~31;
    uint32_t cols = 32;
    while ((int)cols < Npad) cols <<= 1;
    const size_t smem = 1024 + (size_t)Npad * DH * 2 * 2 + 128 * DH * 2 + (size_t)128 * Npad * 2 + 64;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    // the TMEM columns of all CTAs resident on one SM must fit in its 512: cap the
    // residency through the shared-memory request
    const size_t smem_sm = 228 * 1024;
    const size_t max_ctas = 512 / cols;
    size_t smem_req = smem;
    if (smem_sm / smem_req > max_ctas) smem_req = smem_sm / (max_ctas + 1) + 1024;
    switch (DH) {
        case 16:
            cudaFuncSetAttribute(k_attention_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
            k_attention_tc<16><<<grid, AT_THREADS, smem_req, st>>>(ch, uid, qkv, O, prefix_reuse, Npad, cols, status);
            break;
        case 32:
            cudaFuncSetAttribute(k_attention_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
            k_attention_tc<32><<<grid, AT_THREADS, smem_req, st>>>(ch, uid, qkv, O, prefix_reuse, Npad, cols, status);
            break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vq
