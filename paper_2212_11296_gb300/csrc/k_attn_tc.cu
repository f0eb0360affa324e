// Causal multi-head self-attention on the tensor cores (BF16 path, Sec. 3.1
// location mixer): BF16 Q/K/V, FP32 scores and accumulation in TMEM.
//
// One work item = (configuration, head).  A CTA of 8 warps:
//   1. gathers the configuration's K rows and V rows of this head by row id
//      into shared memory (K as a [keys x dh] K-major operand; V staged row by
//      row, then transposed to a [dh x keys] K-major operand with ldmatrix.trans
//      / stmatrix), in the no-swizzle canonical layout (8-row x 16-byte core
//      matrices), every store phase writing 128 contiguous bytes;
//   2. per 128-query tile: gathers Q, thread 0 issues S = Q K^T with
//      tcgen05.mma (M = 128, N = keys, K = dh) into TMEM;
//   3. two threads own each query row (alternate 32-column chunks of its TMEM
//      lane): two passes (causal max, then exp2 / sum) combined through shared
//      memory, writing P as BF16 into shared memory; chunks wholly left of the
//      diagonal take a compare-free path, chunks right of it are skipped;
//   4. thread 0 issues O = P V (M = 128, N = dh, K = keys) into TMEM columns
//      already read; each thread scales half of its row by 1/sum and stores it.
// With prefix reuse, query tiles start at the configuration's first changed
// position: rows before it are neither computed nor stored.
// Waits on the MMA barrier are bounded (VQNQS_DEV_TIMEOUT on expiry).
#include <algorithm>

#include "tc_common.cuh"

namespace vq {

constexpr int AT_THREADS = 256;
constexpr int AT_MAX_N = 448;  // keys per configuration handled in one TMEM tile

using tc::core_off;
using tc::desc_kmajor_none;
using tc::fence_proxy_async_smem;

using tc::ldsm_x4_trans;
using tc::stsm_x4;

// 2^x with the SFU's approximate exponential (flushes denormals); the softmax
// weights it feeds are rounded to BF16 right after.
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 16 consecutive 32-bit TMEM columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int DH>
__global__ void __launch_bounds__(AT_THREADS)
k_attention_tc(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv, float* __restrict__ O,
               int prefix_reuse, int Npad, uint32_t tmem_cols, int* __restrict__ status,
               const int* __restrict__ cfg_list, int n_list, const int* __restrict__ n_list_dev,
               float2* __restrict__ stats) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int d = ch.d, H = ch.heads;
    constexpr int VS = 2 * DH + 16;                // row stride of the V staging rows (bank-conflict free)
    uint8_t* sK = smem;                            // [Npad x DH] K-major core layout
    uint8_t* sVt = sK + (size_t)Npad * DH * 2;     // [DH x Npad]
    uint8_t* sQ = sVt + (size_t)Npad * DH * 2;     // [128 x DH]
    uint8_t* sP = sQ + 128 * DH * 2;               // [128 x Npad]; V staging rows alias it
    uint64_t* bar = reinterpret_cast<uint64_t*>(sP + (size_t)128 * Npad * 2);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 1);
    __shared__ float s_red[2][128];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & 127, half = tid >> 7;  // two threads per query row
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(tmem_holder, tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    const float sl2 = 1.4426950408889634f * rsqrtf((float)DH);  // log2(e) / sqrt(dh)
    const int C = cfg_list ? (n_list_dev ? *n_list_dev : n_list) : ch.counters[CNT_C];
    const int ld = 3 * d;

    for (int item = blockIdx.x; item < C * H && ok; item += gridDim.x) {
        const int ci = item / H, h = item - ci * H;
        const int c = cfg_list ? cfg_list[ci] : ci;
        const int N = cfg_N(ch, c);
        const int* urow = uid + ch.cfg_row[c];
        const int p0 = prefix_reuse ? cfg_p0(ch, c) : 0;
        // keys: position-fastest mapping, so each 8-thread phase writes 128 contiguous bytes
        for (int u = tid; u < Npad * (DH / 8); u += AT_THREADS) {
            const int j = u % Npad, kb = u / Npad;
            uint4 kv = make_uint4(0, 0, 0, 0);
            if (j < N) kv = *reinterpret_cast<const uint4*>(qkv + (size_t)urow[j] * ld + d + h * DH + kb * 8);
            *reinterpret_cast<uint4*>(sK + core_off(j, kb * 8, DH)) = kv;
        }
        // values: row-major staging, then 8x8 transposes into the [DH x Npad] operand
        for (int u = tid; u < Npad * (DH / 8); u += AT_THREADS) {
            const int j = u / (DH / 8), kb = u - j * (DH / 8);
            uint4 vv = make_uint4(0, 0, 0, 0);
            if (j < N) vv = *reinterpret_cast<const uint4*>(qkv + (size_t)urow[j] * ld + 2 * d + h * DH + kb * 8);
            *reinterpret_cast<uint4*>(sP + j * VS + kb * 16) = vv;
        }
        __syncthreads();
        for (int blk = warp; blk < (Npad / 8) * (DH / 32); blk += AT_THREADS / 32) {
            // four 8x8 matrices: key block jb, dh blocks kq*4 .. kq*4+3
            const int jb = blk / (DH / 32), kq = blk - jb * (DH / 32);
            const int m = lane >> 3, r = lane & 7;
            uint32_t f[4];
            ldsm_x4_trans(tc::smem_u32(sP + (jb * 8 + r) * VS + (kq * 4 + m) * 16), f);
            stsm_x4(tc::smem_u32(sVt + core_off((kq * 4 + m) * 8 + r, jb * 8, Npad)), f);
        }
        if (DH == 16) {  // the two dh blocks of a key block in one x4 with two key blocks
            for (int blk = warp; blk < Npad / 16; blk += AT_THREADS / 32) {
                const int m = lane >> 3, r = lane & 7;
                const int jb = blk * 2 + (m >> 1), kb = m & 1;
                uint32_t f[4];
                ldsm_x4_trans(tc::smem_u32(sP + (jb * 8 + r) * VS + kb * 16), f);
                stsm_x4(tc::smem_u32(sVt + core_off(kb * 8 + r, jb * 8, Npad)), f);
            }
        }
        __syncthreads();
        // query tiles start at the first changed position: no row before it is computed
        for (int q0 = p0; q0 < N && ok; q0 += 128) {
            const int nk = min(N, q0 + 128);             // keys this tile can see
            const int nk16 = (nk + 15) & ~15;            // MMA N (multiple of 16)
            const int nk32 = (nk + 31) & ~31;            // columns read back
            for (int u = tid; u < 128 * (DH / 8); u += AT_THREADS) {
                const int r = u & 127, kb = u >> 7;
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
            // softmax of query position p = q0 + row; this thread takes every other
            // 32-column chunk, starting with chunk `half`
            const int p = q0 + row;
            const int plim = min(p, N - 1);  // keys 0..plim are visible
            // tcgen05.ld is warp-collective: which chunks are read is decided by the
            // warp's last row (q0 need not be 32-aligned), the masks per row
            const int plim_w = min(q0 + (warp & 3) * 32 + 31, N - 1);
            float mx = -INFINITY;
            for (int c0 = half * 32; c0 < nk32; c0 += 64) {
                if (c0 > plim_w) break;  // chunks wholly past the warp's diagonal are invisible
                uint32_t r[32];
                tc::tmem_ld32(tmem + lane_base + c0, r);
                if (c0 + 31 <= plim) {
                    float m0 = __uint_as_float(r[0]), m1 = __uint_as_float(r[1]);
#pragma unroll
                    for (int j = 2; j < 32; j += 2) {
                        m0 = fmaxf(m0, __uint_as_float(r[j]));
                        m1 = fmaxf(m1, __uint_as_float(r[j + 1]));
                    }
                    mx = fmaxf(mx, fmaxf(m0, m1));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j <= plim) mx = fmaxf(mx, __uint_as_float(r[j]));
                }
            }
            s_red[half][row] = mx;
            __syncthreads();
            mx = fmaxf(s_red[0][row], s_red[1][row]);
            const float mb = mx * sl2;
            float sum = 0.f;
            for (int c0 = half * 32; c0 < nk32 && c0 < nk16; c0 += 64) {
                uint32_t pk[16];
                if (c0 > plim_w) {  // invisible chunk: P = 0 (still read by the PV MMA up to nk16)
#pragma unroll
                    for (int j = 0; j < 16; ++j) pk[j] = 0u;
                } else {
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + lane_base + c0, r);
                    const bool full = c0 + 31 <= plim;
#pragma unroll
                    for (int j = 0; j < 32; j += 2) {
                        float e0 = ex2_approx(fmaf(__uint_as_float(r[j]), sl2, -mb));
                        float e1 = ex2_approx(fmaf(__uint_as_float(r[j + 1]), sl2, -mb));
                        if (!full) {
                            e0 = (c0 + j <= plim) ? e0 : 0.f;
                            e1 = (c0 + j + 1 <= plim) ? e1 : 0.f;
                        }
                        sum += e0 + e1;
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(e0, e1);
                        pk[j / 2] = *reinterpret_cast<uint32_t*>(&b2);
                    }
                }
#pragma unroll
                for (int j8 = 0; j8 < 4; ++j8)
                    if (c0 + j8 * 8 < nk16)
                        *reinterpret_cast<uint4*>(sP + core_off(row, c0 + j8 * 8, Npad)) =
                            make_uint4(pk[4 * j8], pk[4 * j8 + 1], pk[4 * j8 + 2], pk[4 * j8 + 3]);
            }
            __syncthreads();  // both halves read s_red (max) before it is reused for sums
            s_red[half][row] = sum;
            tc::tc_fence_before();
            fence_proxy_async_smem();
            __syncthreads();
            sum = s_red[0][row] + s_red[1][row];
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
                // each of the row's two threads stores half of the DH output columns
                uint32_t r[16];
                tmem_ld16(tmem + lane_base + half * (DH / 2), r);
                if (p < N && p >= p0) {
                    if (stats && half == 0)  // natural-log units: exp(s / sqrt(dh) - m)
                        stats[((size_t)ch.cfg_sample[c] * ch.N + p) * H + h] = make_float2(mx * rsqrtf((float)DH), sum);
                    const float inv = 1.f / sum;
                    float* dst = O + ((size_t)ch.cfg_row[c] + p) * d + h * DH + half * (DH / 2);
#pragma unroll
                    for (int t = 0; t < DH / 2; t += 4)
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
                                int* status, cudaStream_t st, int grid, const int* cfg_list, int n_list,
                                float2* stats, const int* n_list_dev) {
    const int DH = ch.d / ch.heads;
    if (!attention_tc_supported(ch.N, DH)) return cudaErrorInvalidValue;
    const int Npad = (ch.N + 31) & ~31;
    uint32_t cols = 32;
    while ((int)cols < Npad) cols <<= 1;
    const size_t smem = 1024 + (size_t)Npad * DH * 2 * 2 + 128 * DH * 2 +
                        std::max((size_t)128 * Npad * 2, (size_t)Npad * (2 * DH + 16)) + 64;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    // the TMEM columns of all CTAs resident on one SM must fit in its 512: cap the
    // residency through the shared-memory request
    const size_t smem_sm = 228 * 1024;
    const size_t max_ctas = 512 / cols;
    size_t smem_req = smem;
    if (smem_sm / smem_req > max_ctas) smem_req = smem_sm / (max_ctas + 1) + 1024;
    static size_t granted[2] = {};  // attribute set once per instantiation and size, outside captures
#define VQ_ATC(D, SLOT)                                                                                        \
    {                                                                                                          \
        if (smem_req > granted[SLOT]) {                                                                        \
            cudaFuncSetAttribute(k_attention_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req); \
            granted[SLOT] = smem_req;                                                                          \
        }                                                                                                      \
        k_attention_tc<D><<<grid, AT_THREADS, smem_req, st>>>(ch, uid, qkv, O, prefix_reuse, Npad, cols, status,   \
                                                              cfg_list, n_list, n_list_dev, stats);          \
    }
    if (DH == 16) {
        VQ_ATC(16, 0)
    } else if (DH == 32) {
        VQ_ATC(32, 1)
    } else {
        return cudaErrorInvalidValue;
    }
#undef VQ_ATC
    return cudaGetLastError();
}

}  // namespace vq
