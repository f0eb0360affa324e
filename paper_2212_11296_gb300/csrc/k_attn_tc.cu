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
//   4. P V in 32-key chunks through two P tiles in shared memory: while thread 0's
//      MMAs of chunk j (O += P_j V_j, M = 128, N = dh) run, the threads write
//      chunk j + 1 into the other tile; O accumulates in TMEM columns whose scores
//      were consumed by chunk 0; each thread scales half of its row by 1/sum and
//      stores it.  The chunked P keeps the shared memory of a CTA near 113 KB
//      even with split operands, so two CTAs share an SM.
// With prefix reuse, query tiles start at the configuration's first changed
// position: rows before it are neither computed nor stored.
// Items go to CTAs round-robin, or, given a work counter (zero at launch), each CTA
// takes the next item from it when it finishes one: items of very different sizes
// (configurations with different first changed positions) then leave no long tail.
// Waits on the MMA barrier are bounded (VQNQS_DEV_TIMEOUT on expiry).
//
// Split operands (SPLIT): Q, K and V arrive as two BF16 planes, x = hi + lo
// (hi = bf16(x), lo = bf16(x - hi), the lo plane lo_off elements after the hi
// one), and P is written the same way; each product is hi.hi + hi.lo + lo.hi,
// three MMAs into the same FP32 accumulator.  An operand pair represents x to
// 2^-17 relative (one BF16 value: 2^-9), the dropped lo.lo term is below
// 2^-18 of the product, so scores and outputs carry FP32-grade error.
#include <algorithm>

#include "tc_common.cuh"

namespace vq {

constexpr int AT_THREADS = 256;
constexpr int AT_MAX_N = 448;  // keys per configuration handled in one TMEM tile

using tc::core_off;
using tc::cp_async16;
using tc::cp_async_wait_all;
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

using tc::tmem_ld16;

// BF16 hi and lo parts of two floats, packed as bf16x2 words
__device__ __forceinline__ void split_pack2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Shared-memory plan of one CTA: K and V^T tiles, then a region holding the Q tile and
// two P chunk tiles (each with NP planes), which the V staging rows alias; barriers last.
constexpr int PCH = 32;                      // keys per P chunk
constexpr size_t PCB = (size_t)128 * PCH * 2;  // one plane of one P chunk tile
__host__ __device__ constexpr size_t attn_tile_bytes(int Npad, int DH) { return (size_t)Npad * DH * 2; }
// Q and the two P tiles, or (while an item is staged) the V staging rows and the item's row ids
__host__ __device__ constexpr size_t attn_region_bytes(int Npad, int DH, int NP) {
    return (size_t)NP * 128 * DH * 2 + 2 * NP * PCB > (size_t)NP * Npad * (2 * DH + 16) + (size_t)Npad * 4
               ? (size_t)NP * 128 * DH * 2 + 2 * NP * PCB
               : (size_t)NP * Npad * (2 * DH + 16) + (size_t)Npad * 4;
}
// (+ 1 KB beside the barriers for more than 256 keys: the row exchange then may not alias Q, which
// the second key block's scores read again)
__host__ __device__ constexpr size_t attn_smem_bytes(int Npad, int DH, bool split) {
    return 128 + (split ? 2 : 1) * 2 * attn_tile_bytes(Npad, DH) + attn_region_bytes(Npad, DH, split ? 2 : 1) + 64 +
           (Npad > 256 ? 1024 : 0);
}

// TWO: the item may hold more than 256 keys (two key blocks; Npad > 256)
template <int DH, bool SPLIT, bool TWO>
__global__ void __launch_bounds__(AT_THREADS, 2)
k_attention_tc(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv, size_t lo_off,
               float* __restrict__ O, int prefix_reuse, int Npad, uint32_t tmem_cols, int* __restrict__ status,
               const int* __restrict__ cfg_list, int n_list, const int* __restrict__ n_list_dev,
               float2* __restrict__ stats, int* __restrict__ work) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const int d = ch.d, H = ch.heads;
    constexpr int VS = 2 * DH + 16;                // row stride of the V staging rows (bank-conflict free)
    constexpr int NP = SPLIT ? 2 : 1;              // operand planes: hi (and lo)
    const size_t tb = attn_tile_bytes(Npad, DH);
    uint8_t* sK = smem;                            // [NP][Npad x DH] K-major core layout
    uint8_t* sVt = sK + NP * tb;                   // [NP][DH x Npad]
    uint8_t* sQ = sVt + NP * tb;                   // [NP][128 x DH]; V staging rows alias Q and P
    uint8_t* sP = sQ + NP * 128 * DH * 2;          // [2 tiles][NP][128 x PCH]
    uint8_t* sStage = sQ;                          // [NP][Npad x VS]
    const size_t pb = (size_t)Npad * VS;           // one staging plane
    int* s_uid = reinterpret_cast<int*>(sStage + NP * pb);  // [Npad] the item's row ids, while staging
    uint64_t* bar = reinterpret_cast<uint64_t*>(sQ + attn_region_bytes(Npad, DH, NP));  // S MMAs
    uint64_t* pbar = bar + 1;                      // [2]: MMAs reading P tile 0 / 1
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(pbar + 2);
    // [2][128] row exchange: over Q once Q has been read (at most 256 keys), else beside the barriers
    float (*s_red)[128] = reinterpret_cast<float (*)[128]>(TWO ? reinterpret_cast<uint8_t*>(bar) + 64 : sQ);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & 127, half = tid >> 7;  // two threads per query row
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(&pbar[0], 1);
        tc::mbar_init(&pbar[1], 1);
        tc::fence_barrier_init();
    }
    uint32_t pph[2] = {0u, 0u};  // phases of pbar
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
    __shared__ int s_next;
    // the next item: from the work counter (every thread has read the previous one: each
    // item ends with a barrier) or round-robin
    auto next_item = [&](int prev) {
        if (!work) return prev < 0 ? (int)blockIdx.x : prev + (int)gridDim.x;
        if (tid == 0) s_next = atomicAdd(work, 1);
        __syncthreads();
        return s_next;
    };

    for (int item = next_item(-1); item < C * H && ok; item = next_item(item)) {
        const int ci = item / H, h = item - ci * H;
        const int c = cfg_list ? cfg_list[ci] : ci;
        const int N = cfg_N(ch, c);
        const int* urow = uid + ch.cfg_row[c];
        const int p0 = prefix_reuse ? cfg_p0(ch, c) : 0;
        // the row ids first, then every key and value row with cp.async (all copies in flight
        // at once); keys: position-fastest mapping, so each 8-thread phase writes 128
        // contiguous bytes; values: row-major staging rows, transposed below
        for (int j = tid; j < N; j += AT_THREADS) s_uid[j] = urow[j];
        __syncthreads();
        for (int pl = 0; pl < NP; ++pl) {
            const __nv_bfloat16* src = qkv + pl * lo_off;
            for (int u = tid; u < Npad * (DH / 8); u += AT_THREADS) {
                const int j = u % Npad, kb = u / Npad;
                cp_async16(tc::smem_u32(sK + pl * tb + core_off(j, kb * 8, DH)),
                           j < N ? src + (size_t)s_uid[j] * ld + d + h * DH + kb * 8 : qkv, j < N ? 16 : 0);
            }
            for (int u = tid; u < Npad * (DH / 8); u += AT_THREADS) {
                const int j = u / (DH / 8), kb = u - j * (DH / 8);
                cp_async16(tc::smem_u32(sStage + pl * pb + j * VS + kb * 16),
                           j < N ? src + (size_t)s_uid[j] * ld + 2 * d + h * DH + kb * 8 : qkv, j < N ? 16 : 0);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int pl = 0; pl < NP; ++pl) {
            uint8_t* stg = sStage + pl * pb;
            uint8_t* vt = sVt + pl * tb;
            for (int blk = warp; blk < (Npad / 8) * (DH / 32); blk += AT_THREADS / 32) {
                // four 8x8 matrices: key block jb, dh blocks kq*4 .. kq*4+3
                const int jb = blk / (DH / 32), kq = blk - jb * (DH / 32);
                const int m = lane >> 3, r = lane & 7;
                uint32_t f[4];
                ldsm_x4_trans(tc::smem_u32(stg + (jb * 8 + r) * VS + (kq * 4 + m) * 16), f);
                stsm_x4(tc::smem_u32(vt + core_off((kq * 4 + m) * 8 + r, jb * 8, Npad)), f);
            }
            if (DH == 16) {  // the two dh blocks of a key block in one x4 with two key blocks
                for (int blk = warp; blk < Npad / 16; blk += AT_THREADS / 32) {
                    const int m = lane >> 3, r = lane & 7;
                    const int jb = blk * 2 + (m >> 1), kb = m & 1;
                    uint32_t f[4];
                    ldsm_x4_trans(tc::smem_u32(stg + (jb * 8 + r) * VS + kb * 16), f);
                    stsm_x4(tc::smem_u32(vt + core_off(kb * 8 + r, jb * 8, Npad)), f);
                }
            }
        }
        __syncthreads();
        // query tiles aligned to the last position: a partial tile, if any, holds the first rows
        // (fewest keys) rather than the last ones; warps whose rows all lie before p0 skip the
        // softmax, and no row before p0 is stored
        const int qs = max(0, N - 128 * ((N - p0 + 127) / 128));
        for (int q0 = qs; q0 < N && ok; q0 += 128) {
            const int nk = min(N, q0 + 128);             // keys this tile can see
            const int nk16 = (nk + 15) & ~15;            // MMA N (multiple of 16)
            const int nk32 = (nk + 31) & ~31;            // columns read back
            {  // this thread's query row is tile row `row` (the u loop steps by a multiple of 128)
                const bool qin = q0 + row < N;
                const size_t qoff = qin ? (size_t)urow[q0 + row] * ld + h * DH : 0;
                for (int pl = 0; pl < NP; ++pl)
                    for (int u = tid; u < 128 * (DH / 8); u += AT_THREADS) {
                        const int kb = u >> 7;
                        cp_async16(tc::smem_u32(sQ + pl * 128 * DH * 2 + core_off(row, kb * 8, DH)),
                                   qkv + pl * lo_off + qoff + kb * 8, qin ? 16 : 0);
                    }
                cp_async_wait_all();
            }
            fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            // S = Q K^T for keys [kb, kb + n16) into TMEM columns [cb, cb + n16), issued by thread 0;
            // every thread waits for it
            auto scores = [&](int kb, int n16, int cb) {
                if (tid == 0) {
                    tc::tc_fence_after();
                    // (Q plane, K plane) pairs: hi.hi, then hi.lo and lo.hi with split operands
                    constexpr int NPROD = SPLIT ? 3 : 1;
                    for (int n0 = 0; n0 < n16; n0 += 256) {
                        const int nn = min(256, n16 - n0);
                        const uint32_t idesc = tc::idesc_bf16_f32(128, nn);
#pragma unroll
                        for (int pr = 0; pr < NPROD; ++pr) {
                            const int qp = pr == 2 ? 1 : 0, kp = pr == 1 ? 1 : 0;
                            const uint64_t dq =
                                desc_kmajor_none(tc::smem_u32(sQ + qp * 128 * DH * 2), 128, (DH / 8) * 128);
                            const uint64_t dk = desc_kmajor_none(tc::smem_u32(sK + kp * tb), 128, (DH / 8) * 128);
                            const uint64_t dkn = dk + (uint64_t)((((kb + n0) / 8) * (DH / 8) * 128) >> 4);
#pragma unroll
                            for (int ks = 0; ks < DH / 16; ++ks)
                                tc::mma_bf16(tmem + cb + n0, dq + (uint64_t)(ks * 16), dkn + (uint64_t)(ks * 16),
                                             idesc, (pr | ks) > 0 ? 1u : 0u);
                        }
                    }
                    tc::mma_commit(bar);
                }
                ok = (__syncthreads_and(tc::mbar_wait(bar, phase, status)) != 0) && ok;
                phase ^= 1;
                tc::tc_fence_after();
            };
            // softmax of query position p = q0 + row; this thread takes every other
            // 32-column chunk, starting with chunk `half`
            const int p = q0 + row;
            const int plim = min(p, N - 1);  // keys 0..plim are visible
            // tcgen05.ld is warp-collective: which chunks are read is decided by the
            // warp's last row (q0 need not be 32-aligned), the masks per row
            const int plim_w = min(q0 + (warp & 3) * 32 + 31, N - 1);
            // a warp whose rows all lie past the configuration's last position has nothing to
            // compute: its P rows are zero and its outputs are not stored
            const bool wpad = q0 + (warp & 3) * 32 >= N || q0 + (warp & 3) * 32 + 31 < p0;
            // the row's largest visible score among keys [kb, kend) held at TMEM column cb + k - kb
            auto max_pass = [&](int cb, int kb, int kend) {
                float mx = -INFINITY;
                const int n32 = (kend - kb + 31) & ~31;
                for (int c0 = half * 32; c0 < n32 && !wpad; c0 += 64) {
                    const int k0 = kb + c0;
                    if (k0 > plim_w) break;  // chunks wholly past the warp's diagonal are invisible
                    uint32_t r[32];
                    tc::tmem_ld32(tmem + lane_base + cb + c0, r);
                    if (k0 + 31 <= plim) {
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
                            if (k0 + j <= plim) mx = fmaxf(mx, __uint_as_float(r[j]));
                    }
                }
                return mx;
            };
            // more than 256 keys: two key blocks, [0, 256) and [256, nk), each taking at most
            // 256 TMEM columns; the maxima of both are found first (block 1's scores, then
            // block 0's over them), so P needs no rescaling
            const bool two = TWO && nk16 > 256;
            float mx;
            if (!two) {
                scores(0, nk16, 0);
                if (!ok) break;
                mx = max_pass(0, 0, nk);
            } else {
                scores(256, nk16 - 256, 0);
                if (!ok) break;
                const float m1 = max_pass(0, 256, nk);
                tc::tc_fence_before();
                __syncthreads();  // block 1's scores are read before block 0's overwrite them
                scores(0, 256, 0);
                if (!ok) break;
                mx = fmaxf(max_pass(0, 0, 256), m1);
            }
            s_red[half][row] = mx;
            __syncthreads();
            mx = fmaxf(s_red[0][row], s_red[1][row]);
            const float mb = mx * sl2;
            float sum = 0.f;
            int pend[2] = {0, 0};
            // P V over keys [kb, kb + n16) whose scores sit at TMEM column cb + k - kb, in chunks of
            // PCH keys through double-buffered P tiles (pend: MMAs still reading a tile); the
            // output accumulates in TMEM columns [0, DH) (first: the first chunk overwrites them)
            auto pv = [&](int cb, int kb, int n16, bool first) {
                const int nch = (n16 + PCH - 1) / PCH;
                for (int jc = 0; jc < nch && ok; ++jc) {
                    const int u = jc & 1;
                    uint8_t* pt = sP + (size_t)u * NP * PCB;
                    if (pend[u]) {  // the MMAs of the chunk two before read this tile
                        ok = __syncthreads_and(tc::mbar_wait(&pbar[u], pph[u], status)) != 0;
                        pph[u] ^= 1;
                        pend[u] = 0;
                        tc::tc_fence_after();
                        if (!ok) break;
                    }
                    const int c0 = jc * PCH + half * 16;  // this thread's 16 keys of the chunk
                    const int k0 = kb + c0;
                    uint32_t pk[8], pl[8];
                    if (wpad || k0 > plim_w || c0 >= n16) {  // no rows, invisible, or past the MMA's keys
#pragma unroll
                        for (int j = 0; j < 8; ++j) pk[j] = pl[j] = 0u;
                    } else {
                        uint32_t r[16];
                        tmem_ld16(tmem + lane_base + cb + c0, r);
                        const bool full = k0 + 15 <= plim;
#pragma unroll
                        for (int j = 0; j < 16; j += 2) {
                            float e0 = ex2_approx(fmaf(__uint_as_float(r[j]), sl2, -mb));
                            float e1 = ex2_approx(fmaf(__uint_as_float(r[j + 1]), sl2, -mb));
                            if (!full) {
                                e0 = (k0 + j <= plim) ? e0 : 0.f;
                                e1 = (k0 + j + 1 <= plim) ? e1 : 0.f;
                            }
                            sum += e0 + e1;
                            if (SPLIT) {
                                split_pack2(e0, e1, pk[j / 2], pl[j / 2]);
                            } else {
                                __nv_bfloat162 b2 = __floats2bfloat162_rn(e0, e1);
                                pk[j / 2] = *reinterpret_cast<uint32_t*>(&b2);
                            }
                        }
                    }
#pragma unroll
                    for (int j8 = 0; j8 < 2; ++j8) {
                        const uint32_t off = core_off(row, half * 16 + j8 * 8, PCH);
                        *reinterpret_cast<uint4*>(pt + off) =
                            make_uint4(pk[4 * j8], pk[4 * j8 + 1], pk[4 * j8 + 2], pk[4 * j8 + 3]);
                        if (SPLIT)
                            *reinterpret_cast<uint4*>(pt + PCB + off) =
                                make_uint4(pl[4 * j8], pl[4 * j8 + 1], pl[4 * j8 + 2], pl[4 * j8 + 3]);
                    }
                    tc::fence_proxy_async_smem();
                    tc::tc_fence_before();
                    __syncthreads();
                    if (tid == 0) {
                        tc::tc_fence_after();
                        const uint32_t idesc = tc::idesc_bf16_f32(128, DH);
                        const int kk = min(PCH, n16 - jc * PCH);  // keys of this chunk the MMA covers
                        constexpr int NPROD = SPLIT ? 3 : 1;     // (P plane, V plane): hi.hi, hi.lo, lo.hi
#pragma unroll
                        for (int pr = 0; pr < NPROD; ++pr) {
                            const int pp = pr == 2 ? 1 : 0, vp = pr == 1 ? 1 : 0;
                            const uint64_t dp = desc_kmajor_none(tc::smem_u32(pt + pp * PCB), 128, (PCH / 8) * 128);
                            const uint64_t dv =
                                desc_kmajor_none(tc::smem_u32(sVt + vp * tb), 128, (Npad / 8) * 128) +
                                (uint64_t)((((kb + jc * PCH) / 8) * 128) >> 4);
                            for (int ks = 0; ks < kk / 16; ++ks)
                                tc::mma_bf16(tmem, dp + (uint64_t)(ks * 16), dv + (uint64_t)(ks * 16), idesc,
                                             (!first || (jc | pr | ks) > 0) ? 1u : 0u);
                        }
                        tc::mma_commit(&pbar[u]);
                    }
                    pend[u] = 1;
                }
            };
            pv(0, 0, two ? 256 : nk16, true);
            if (two && ok) {
                tc::tc_fence_before();
                __syncthreads();  // every read of block 0's scores is done
                scores(256, nk16 - 256, 32);  // block 1 again, beside the output columns
                if (ok) pv(32, 256, nk16 - 256, false);
            }
            // the last chunk's MMAs (and every earlier one) have completed
            for (int u = 0; u < 2; ++u)
                if (pend[u]) {
                    ok = (__syncthreads_and(tc::mbar_wait(&pbar[u], pph[u], status)) != 0) && ok;
                    pph[u] ^= 1;
                }
            tc::tc_fence_after();
            if (!ok) break;
            s_red[half][row] = sum;
            __syncthreads();
            sum = s_red[0][row] + s_red[1][row];
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

bool attention_tc_supported(int N, int dh, bool split) {
    if (!(dh == 16 || dh == 32) || N > AT_MAX_N) return false;
    return attn_smem_bytes((N + 31) & ~31, dh, split) <= 227 * 1024;
}

cudaError_t launch_attention_tc(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O, int prefix_reuse,
                                int* status, cudaStream_t st, int grid, const int* cfg_list, int n_list,
                                float2* stats, const int* n_list_dev, size_t lo_off, int* work) {
    const int DH = ch.d / ch.heads;
    const bool split = lo_off != 0;
    if (!attention_tc_supported(ch.N, DH, split)) return cudaErrorInvalidValue;
    const int Npad = (ch.N + 31) & ~31;
    uint32_t cols = 32;
    while ((int)cols < Npad) cols <<= 1;
    if (cols > 256) cols = 256;  // more than 256 keys: two key blocks of at most 256 columns
    const size_t smem = attn_smem_bytes(Npad, DH, split);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    // the TMEM columns of all CTAs resident on one SM must fit in its 512: cap the
    // residency through the shared-memory request
    const size_t smem_sm = 228 * 1024;
    const size_t max_ctas = 512 / cols;
    size_t smem_req = smem;
    if (smem_sm / smem_req > max_ctas) smem_req = smem_sm / (max_ctas + 1) + 1024;
    static size_t granted[6] = {};  // attribute set once per instantiation and size, outside captures
#define VQ_ATC(D, SP, TW, SLOT)                                                                                 \
    {                                                                                                           \
        if (smem_req > granted[SLOT]) {                                                                         \
            cudaFuncSetAttribute(k_attention_tc<D, SP, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                 (int)smem_req);                                                                \
            granted[SLOT] = smem_req;                                                                           \
        }                                                                                                       \
        k_attention_tc<D, SP, TW><<<grid, AT_THREADS, smem_req, st>>>(ch, uid, qkv, lo_off, O, prefix_reuse,    \
                                                                      Npad, cols, status, cfg_list, n_list,     \
                                                                      n_list_dev, stats, work);                \
    }
    const bool two = Npad > 256;  // split operands take at most 256 positions (attention_tc_supported)
    if (DH == 16) {
        if (split) VQ_ATC(16, true, false, 2) else if (two) VQ_ATC(16, false, true, 4) else VQ_ATC(16, false, false, 0)
    } else if (DH == 32) {
        if (split) VQ_ATC(32, true, false, 3) else if (two) VQ_ATC(32, false, true, 5) else VQ_ATC(32, false, false, 1)
    } else {
        return cudaErrorInvalidValue;
    }
#undef VQ_ATC
    return cudaGetLastError();
}

}  // namespace vq
