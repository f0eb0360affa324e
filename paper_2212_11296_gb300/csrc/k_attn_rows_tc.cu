// Causal attention of listed rows of many connected configurations that share
// one sample's keys and values except at a few changed positions (BF16 path,
// dh = 32; tensor cores for the sample's keys, CUDA cores for the changes).
//
// A configuration one exchange away from sample s has the same row ids as s
// except at its changed positions D (Sec. 3.2 keys rows on their quantized
// history, so equal ids mean equal keys and values).  For a listed row
// (configuration c, position p) with query q:
//   softmax over s's keys 0..p   ->  maximum m, sum l, numerator A = sum_j P_j v_j
// computed for 128 rows at once (S = Q K_s^T and A = P V_s on the tensor cores,
// P rounded to BF16), then each row swaps its configuration's keys in at the
// changed positions k <= p, exactly as the softmax identity allows:
//   m' = max(m, q.k_c / sqrt(dh)),  r = exp(m - m'),
//   A' = r (A - sum_k bf16(e_s,k) v_s,k) + sum_k e'_c,k v_c,k,
//   l' = r (l - sum_k e_s,k) + sum_k e'_c,k,     o = A' / l'
// (e_s,k = exp(q.k_s / sqrt(dh) - m) removed the way it was added; e'_c,k
// against m').  One work item = (sample, head, slice): s's K and V of the head
// are staged once for all the item's tiles.
//
// Split operands (SPLIT, as in k_attn_tc.cu): Q, K and V arrive as BF16 hi and
// lo planes (lo_off elements apart) and P is split the same way, three MMAs per
// product; the changed keys' corrections read hi + lo in FP32, and the removed
// weight is the one the split P carried (hi + lo of e).
//
// Rows come from a per-sample list of (row, position) pairs laid out like the
// active rows (sample b's entries start at act_off[first configuration of b];
// count[b] of them, or the whole region when count is NULL).  Each
// configuration's changed positions are dpos[c][0 .. dcnt[c]) (at most
// INC_MAX_KEYS).  Waits on the MMA barrier are bounded.
#include <algorithm>

#include "tc_common.cuh"

namespace vq {

namespace {

constexpr int AR_THREADS = 256;
constexpr int DH = 32;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

using tc::tmem_ld16;
using tc::cp_async16;
using tc::cp_async_wait_all;

// 8 consecutive BF16 values (16-byte aligned) as floats; with SPLIT the value is hi + lo,
// the lo plane lo_off elements further on
template <bool SPLIT>
__device__ __forceinline__ void ld8(const __nv_bfloat16* p, size_t lo_off, float (&out)[8]) {
    const uint4 u = *reinterpret_cast<const uint4*>(p);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f = __bfloat1622float2(h[k]);
        out[2 * k] = f.x;
        out[2 * k + 1] = f.y;
    }
    if (SPLIT) {
        const uint4 ul = *reinterpret_cast<const uint4*>(p + lo_off);
        const __nv_bfloat162* l = reinterpret_cast<const __nv_bfloat162*>(&ul);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __bfloat1622float2(l[k]);
            out[2 * k] += f.x;
            out[2 * k + 1] += f.y;
        }
    }
}
// q . x over DH values read eight at a time
template <bool SPLIT>
__device__ __forceinline__ float dot_dh(const float (&q)[DH], const __nv_bfloat16* p, size_t lo_off) {
    float s = 0.f;
#pragma unroll
    for (int t8 = 0; t8 < DH; t8 += 8) {
        float x[8];
        ld8<SPLIT>(p + t8, lo_off, x);
#pragma unroll
        for (int t = 0; t < 8; ++t) s = fmaf(q[t8 + t], x[t], s);
    }
    return s;
}
// a += w x over 16 values
template <bool SPLIT>
__device__ __forceinline__ void axpy16(float w, const __nv_bfloat16* p, size_t lo_off, float (&a)[16]) {
#pragma unroll
    for (int t8 = 0; t8 < 16; t8 += 8) {
        float x[8];
        ld8<SPLIT>(p + t8, lo_off, x);
#pragma unroll
        for (int t = 0; t < 8; ++t) a[t8 + t] = fmaf(w, x[t], a[t8 + t]);
    }
}

__device__ __forceinline__ void split_pack2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// the value a BF16 operand (pair, with SPLIT) carries for x
template <bool SPLIT>
__device__ __forceinline__ float operand_value(float x) {
    const float h = __bfloat162float(__float2bfloat16_rn(x));
    return SPLIT ? h + __bfloat162float(__float2bfloat16_rn(x - h)) : h;
}

// Shared-memory plan (as in k_attn_tc.cu): K and V^T tiles, then a region holding the Q
// tile and two P chunk tiles of PCH keys (each with NP planes), aliased by the V staging rows.
constexpr int PCH = 32;
constexpr size_t PCB = (size_t)128 * PCH * 2;
__host__ __device__ constexpr size_t rows_tile_bytes(int Npad) { return (size_t)Npad * DH * 2; }
// Q and the two P tiles, or (while an item is staged) the V staging rows and the sample's row ids
__host__ __device__ constexpr size_t rows_region_bytes(int Npad, int NP) {
    return (size_t)NP * 128 * DH * 2 + 2 * NP * PCB > (size_t)NP * Npad * (2 * DH + 16) + (size_t)Npad * 4
               ? (size_t)NP * 128 * DH * 2 + 2 * NP * PCB
               : (size_t)NP * Npad * (2 * DH + 16) + (size_t)Npad * 4;
}
__host__ __device__ constexpr size_t rows_smem_bytes(int Npad, bool split) {
    return 128 + (split ? 2 : 1) * 2 * rows_tile_bytes(Npad) + rows_region_bytes(Npad, split ? 2 : 1) + 64;
}

}  // namespace

template <bool SPLIT>
__global__ void __launch_bounds__(AR_THREADS, 2)
k_attention_rows_tc(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv, size_t lo_off,
                    float* __restrict__ O, const int2* __restrict__ list, const int* __restrict__ act_off,
                    const int* __restrict__ count, const short* __restrict__ dpos, const int* __restrict__ dcnt,
                    int slices, int Npad, uint32_t tmem_cols, int* __restrict__ status, long long* __restrict__ stats) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    constexpr int VS = 2 * DH + 16;               // row stride of the V staging rows (bank-conflict free)
    constexpr int NP = SPLIT ? 2 : 1;             // operand planes: hi (and lo)
    const int d = ch.d, H = ch.heads;
    const size_t tb = rows_tile_bytes(Npad);
    const size_t pb = (size_t)Npad * VS;          // one V staging plane
    uint8_t* sK = smem;                           // [NP][Npad x DH] K-major
    uint8_t* sVt = sK + NP * tb;                  // [NP][DH x Npad]
    uint8_t* sQ = sVt + NP * tb;                  // [NP][128 x DH]; V staging rows alias Q and P
    uint8_t* sP = sQ + NP * 128 * DH * 2;         // [2 tiles][NP][128 x PCH]
    uint8_t* sStage = sQ;
    uint64_t* bar = reinterpret_cast<uint64_t*>(sQ + rows_region_bytes(Npad, NP));  // S MMAs
    uint64_t* pbar = bar + 1;                     // [2]: MMAs reading P tile 0 / 1
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(pbar + 2);
    float (*s_red)[128] = reinterpret_cast<float (*)[128]>(sQ);  // [2][128], used once Q has been read
    __shared__ int s_pw[4];
    __shared__ unsigned long long s_pairs;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int row = tid & 127, half = tid >> 7;  // two threads per query row
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(&pbar[0], 1);
        tc::mbar_init(&pbar[1], 1);
        tc::fence_barrier_init();
        s_pairs = 0;
    }
    uint32_t pph[2] = {0u, 0u};  // phases of pbar
    unsigned long long pairs = 0;  // query-key pairs of this thread's rows (head 0, first half)
    if (blockIdx.x == 0 && tid == 0 && stats)  // the layer's search list is complete: count it
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_VQ]), (unsigned long long)ch.counters[CNT_V]);
    if (warp == 0) tc::tmem_alloc(tmem_holder, tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t phase = 0;
    bool ok = true;
    const float sl2 = 1.4426950408889634f * rsqrtf((float)DH);  // log2(e) / sqrt(dh)
    const int ld = 3 * d;
    const int items = ch.S * H * slices;

    for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
        const int z = item % slices, bh = item / slices;
        const int b = bh / H, h = bh - b * H;
        const int c0b = ch.cfg_off[b];
        const int start = act_off[c0b];
        int n;
        if (count) {
            n = count[b];
        } else {  // the sample's whole region of active rows
            const int c1b = ch.cfg_off[b + 1];
            n = (c1b < ch.counters[CNT_C] ? act_off[c1b] : ch.counters[CNT_A]) - start;
        }
        if (z * 128 >= n) continue;  // block-uniform: no tile for this slice
        const int2* lst = list + start;
        const int rb = ch.cfg_row[ch.cfg_off[b]];
        const int N = sample_N(ch, b);
        const int* ub = uid + rb;
        __syncthreads();  // the previous item's readers of the shared tiles are done
        // s's row ids, then its keys (position-fastest mapping: each 8-thread phase writes 128
        // contiguous bytes) and values (row-major staging rows, transposed below) with cp.async
        int* s_uid = reinterpret_cast<int*>(sStage + NP * pb);
        for (int j = tid; j < N; j += AR_THREADS) s_uid[j] = ub[j];
        __syncthreads();
        for (int pl = 0; pl < NP; ++pl) {
            const __nv_bfloat16* src = qkv + pl * lo_off;
            for (int u = tid; u < Npad * (DH / 8); u += AR_THREADS) {
                const int j = u % Npad, kb = u / Npad;
                cp_async16(tc::smem_u32(sK + pl * tb + tc::core_off(j, kb * 8, DH)),
                           j < N ? src + (size_t)s_uid[j] * ld + d + h * DH + kb * 8 : qkv, j < N ? 16 : 0);
            }
            for (int u = tid; u < Npad * (DH / 8); u += AR_THREADS) {
                const int j = u / (DH / 8), kb = u - j * (DH / 8);
                cp_async16(tc::smem_u32(sStage + pl * pb + j * VS + kb * 16),
                           j < N ? src + (size_t)s_uid[j] * ld + 2 * d + h * DH + kb * 8 : qkv, j < N ? 16 : 0);
            }
        }
        cp_async_wait_all();
        __syncthreads();
        for (int pl = 0; pl < NP; ++pl)
            for (int blk = warp; blk < (Npad / 8) * (DH / 32); blk += AR_THREADS / 32) {
                const int jb = blk / (DH / 32), kq = blk - jb * (DH / 32);
                const int m = lane >> 3, r = lane & 7;
                uint32_t f[4];
                tc::ldsm_x4_trans(tc::smem_u32(sStage + pl * pb + (jb * 8 + r) * VS + (kq * 4 + m) * 16), f);
                tc::stsm_x4(tc::smem_u32(sVt + pl * tb + tc::core_off((kq * 4 + m) * 8 + r, jb * 8, Npad)), f);
            }
        __syncthreads();
        for (int t0 = z * 128; t0 < n && ok; t0 += slices * 128) {
            // this thread's row: (row index, position), or none
            int rrow = -1, p = -1;
            if (t0 + row < n) {
                const int2 e = lst[t0 + row];
                rrow = e.x;
                p = e.y;
            }
            {  // this thread's query row is tile row `row` (the u loop steps by a multiple of 128)
                const size_t qoff = rrow >= 0 ? (size_t)uid[rrow] * ld + h * DH : 0;
                for (int pl = 0; pl < NP; ++pl)
                    for (int u = tid; u < 128 * (DH / 8); u += AR_THREADS) {
                        const int kb = u >> 7;
                        cp_async16(tc::smem_u32(sQ + pl * 128 * DH * 2 + tc::core_off(row, kb * 8, DH)),
                                   qkv + pl * lo_off + qoff + kb * 8, rrow >= 0 ? 16 : 0);
                    }
                cp_async_wait_all();
            }
            // the tile's key range: up to its largest position (warp maxima for uniform TMEM reads)
            const int pw = __reduce_max_sync(0xffffffffu, p);
            if (lane == 0 && half == 0) s_pw[warp] = pw;
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            const int plim_w = s_pw[warp & 3];  // the warp's rows: keys 0..plim_w cover them all
            const int ptile = max(max(s_pw[0], s_pw[1]), max(s_pw[2], s_pw[3]));
            const int nk16 = ((ptile + 1) + 15) & ~15;  // MMA N
            const int nk32 = ((ptile + 1) + 31) & ~31;  // columns read back
            if (ptile < 0) {  // only skipped rows in this tile
                tc::tc_fence_after();
                __syncthreads();
                continue;
            }
            if (tid == 0) {
                tc::tc_fence_after();
                constexpr int NPROD = SPLIT ? 3 : 1;  // (Q plane, K plane): hi.hi, hi.lo, lo.hi
                for (int n0 = 0; n0 < nk16; n0 += 256) {
                    const int nn = min(256, nk16 - n0);
#pragma unroll
                    for (int pr = 0; pr < NPROD; ++pr) {
                        const int qp = pr == 2 ? 1 : 0, kp = pr == 1 ? 1 : 0;
                        const uint64_t dq =
                            tc::desc_kmajor_none(tc::smem_u32(sQ + qp * 128 * DH * 2), 128, (DH / 8) * 128);
                        const uint64_t dk = tc::desc_kmajor_none(tc::smem_u32(sK + kp * tb), 128, (DH / 8) * 128);
                        const uint64_t dkn = dk + (uint64_t)(((n0 / 8) * (DH / 8) * 128) >> 4);
#pragma unroll
                        for (int ks = 0; ks < DH / 16; ++ks)
                            tc::mma_bf16(tmem + n0, dq + (uint64_t)(ks * 16), dkn + (uint64_t)(ks * 16),
                                         tc::idesc_bf16_f32(128, nn), (pr | ks) > 0 ? 1u : 0u);
                    }
                }
                tc::mma_commit(bar);
            }
            ok = __syncthreads_and(tc::mbar_wait(bar, phase, status)) != 0;
            phase ^= 1;
            tc::tc_fence_after();
            if (!ok) break;
            // softmax over s's keys 0..p; this thread takes every other 32-column chunk
            const int plim = p;  // -1: no keys
            float mx = -INFINITY;
            for (int c0 = half * 32; c0 < nk32; c0 += 64) {
                if (c0 > plim_w) break;  // warp-uniform
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
            const float mb = (p >= 0) ? mx * sl2 : 0.f;
            float sum = 0.f;
            // P V in chunks of PCH keys, double-buffered P tiles (pend: MMAs of this tile still reading them)
            const int nch = (nk16 + PCH - 1) / PCH;
            int pend[2] = {0, 0};
            for (int jc = 0; jc < nch && ok; ++jc) {
                const int u = jc & 1;
                uint8_t* pt = sP + (size_t)u * NP * PCB;
                if (pend[u]) {  // chunk jc - 2's MMAs read this tile
                    ok = __syncthreads_and(tc::mbar_wait(&pbar[u], pph[u], status)) != 0;
                    pph[u] ^= 1;
                    pend[u] = 0;
                    tc::tc_fence_after();
                    if (!ok) break;
                }
                const int c0 = jc * PCH + half * 16;  // this thread's 16 keys of the chunk
                uint32_t pk[8], plo[8];
                if (c0 > plim_w || c0 >= nk16) {  // invisible to the warp's rows, or past the MMA's keys: P = 0
#pragma unroll
                    for (int j = 0; j < 8; ++j) pk[j] = plo[j] = 0u;
                } else {
                    uint32_t r[16];
                    tmem_ld16(tmem + lane_base + c0, r);
                    const bool full = c0 + 15 <= plim;
#pragma unroll
                    for (int j = 0; j < 16; j += 2) {
                        float e0 = ex2_approx(fmaf(__uint_as_float(r[j]), sl2, -mb));
                        float e1 = ex2_approx(fmaf(__uint_as_float(r[j + 1]), sl2, -mb));
                        if (!full) {
                            e0 = (c0 + j <= plim) ? e0 : 0.f;
                            e1 = (c0 + j + 1 <= plim) ? e1 : 0.f;
                        }
                        sum += e0 + e1;
                        if (SPLIT) {
                            split_pack2(e0, e1, pk[j / 2], plo[j / 2]);
                        } else {
                            __nv_bfloat162 b2 = __floats2bfloat162_rn(e0, e1);
                            pk[j / 2] = *reinterpret_cast<uint32_t*>(&b2);
                        }
                    }
                }
#pragma unroll
                for (int j8 = 0; j8 < 2; ++j8) {
                    const uint32_t off = tc::core_off(row, half * 16 + j8 * 8, PCH);
                    *reinterpret_cast<uint4*>(pt + off) = make_uint4(pk[4 * j8], pk[4 * j8 + 1], pk[4 * j8 + 2], pk[4 * j8 + 3]);
                    if (SPLIT)
                        *reinterpret_cast<uint4*>(pt + PCB + off) =
                            make_uint4(plo[4 * j8], plo[4 * j8 + 1], plo[4 * j8 + 2], plo[4 * j8 + 3]);
                }
                tc::fence_proxy_async_smem();
                tc::tc_fence_before();
                __syncthreads();
                if (tid == 0) {
                    tc::tc_fence_after();
                    const uint32_t idesc = tc::idesc_bf16_f32(128, DH);
                    const int kk = min(PCH, nk16 - jc * PCH);  // keys of this chunk the MMA covers
                    constexpr int NPROD = SPLIT ? 3 : 1;     // (P plane, V plane): hi.hi, hi.lo, lo.hi
#pragma unroll
                    for (int pr = 0; pr < NPROD; ++pr) {
                        const int pp = pr == 2 ? 1 : 0, vp = pr == 1 ? 1 : 0;
                        const uint64_t dp = tc::desc_kmajor_none(tc::smem_u32(pt + pp * PCB), 128, (PCH / 8) * 128);
                        const uint64_t dv = tc::desc_kmajor_none(tc::smem_u32(sVt + vp * tb), 128, (Npad / 8) * 128) +
                                            (uint64_t)(((jc * PCH / 8) * 128) >> 4);
                        for (int ks = 0; ks < kk / 16; ++ks)
                            tc::mma_bf16(tmem, dp + (uint64_t)(ks * 16), dv + (uint64_t)(ks * 16), idesc,
                                         (jc | pr | ks) > 0 ? 1u : 0u);
                    }
                    tc::mma_commit(&pbar[u]);
                }
                pend[u] = 1;
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
                uint32_t r[16];
                tmem_ld16(tmem + lane_base + half * (DH / 2), r);  // this thread's half of the dims
                if (p >= 0) {
                    float a[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) a[t] = __uint_as_float(r[t]);
                    // swap the configuration's keys in at its changed positions k <= p
                    const int c = ch.row_cfg[rrow];
                    const int nd = dcnt[c];
                    const int* uc = uid + (rrow - p);
                    const short* dp = dpos + (size_t)c * INC_MAX_KEYS;
                    float q[DH];
#pragma unroll
                    for (int t8 = 0; t8 < DH; t8 += 8) {
                        float x[8];
                        ld8<SPLIT>(qkv + (size_t)uid[rrow] * ld + h * DH + t8, lo_off, x);
#pragma unroll
                        for (int t = 0; t < 8; ++t) q[t8 + t] = x[t];
                    }
                    // one pass over the changed keys before the row (ascending) with a running
                    // maximum m2 for the configuration's weights (add and ladd are rescaled when
                    // it grows); the next key's position and row ids load while this one is used
                    float m2 = mb, lsub = 0.f, ladd = 0.f;  // log2-unit maximum; removed and added weight
                    float add[16];
#pragma unroll
                    for (int t = 0; t < 16; ++t) add[t] = 0.f;
                    int kn = nd > 0 ? dp[0] : 0x7fffffff;
                    int ubn = 0, ucn = 0;
                    if (kn <= p) { ubn = ub[kn]; ucn = uc[kn]; }
                    for (int i = 0; i < nd && kn <= p; ++i) {
                        const int ukb = ubn, ukc = ucn;
                        kn = i + 1 < nd ? dp[i + 1] : 0x7fffffff;
                        if (kn <= p) { ubn = ub[kn]; ucn = uc[kn]; }
                        const float sb = dot_dh<SPLIT>(q, qkv + (size_t)ukb * ld + d + h * DH, lo_off);
                        const float sc = dot_dh<SPLIT>(q, qkv + (size_t)ukc * ld + d + h * DH, lo_off);
                        const float eb = ex2_approx(fmaf(sb, sl2, -mb));  // as s's softmax added it
                        const float ebq = operand_value<SPLIT>(eb);
                        axpy16<SPLIT>(-ebq, qkv + (size_t)ukb * ld + 2 * d + h * DH + half * 16, lo_off, a);
                        const float xc = sc * sl2;
                        if (xc > m2) {  // a new maximum: rescale what was added so far
                            const float f = ex2_approx(m2 - xc);
#pragma unroll
                            for (int t = 0; t < 16; ++t) add[t] *= f;
                            ladd *= f;
                            m2 = xc;
                        }
                        const float ec = ex2_approx(xc - m2);
                        axpy16<SPLIT>(ec, qkv + (size_t)ukc * ld + 2 * d + h * DH + half * 16, lo_off, add);
                        lsub += eb;
                        ladd += ec;
                    }
                    const float rs = ex2_approx(mb - m2);  // rescale of s's part (1 if no new maximum)
                    if (h == 0 && half == 0) pairs += p + 1;
                    const float inv = 1.f / (rs * (sum - lsub) + ladd);
                    float* dst = O + (size_t)rrow * d + h * DH + half * 16;
#pragma unroll
                    for (int t = 0; t < 16; t += 4)
                        *reinterpret_cast<float4*>(dst + t) =
                            make_float4((rs * a[t] + add[t]) * inv, (rs * a[t + 1] + add[t + 1]) * inv,
                                        (rs * a[t + 2] + add[t + 2]) * inv, (rs * a[t + 3] + add[t + 3]) * inv);
                }
            }
            tc::tc_fence_before();
            __syncthreads();
        }
    }
    if (pairs) atomicAdd(&s_pairs, pairs);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
    if (tid == 0 && s_pairs && stats) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_FPAIRS]), s_pairs);
}

bool attention_rows_tc_supported(int N, int d, int heads) {
    return d / heads == DH && N <= 256 && rows_smem_bytes((N + 31) & ~31, true) <= 227 * 1024;
}
// (two CTAs per SM need rows_smem_bytes(256, true) plus the static words within half of the SM's 228 KB)

cudaError_t launch_attention_rows_tc(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                                     const int2* list, const int* act_off, const int* count, const short* dpos,
                                     const int* dcnt, int* status, long long* stats, cudaStream_t st, int num_sms,
                                     size_t lo_off, int slices_per_sm) {
    if (!attention_rows_tc_supported(ch.N, ch.d, ch.heads)) return cudaErrorInvalidValue;
    const bool split = lo_off != 0;
    const int Npad = (ch.N + 31) & ~31;
    uint32_t cols = 32;
    while ((int)cols < Npad) cols <<= 1;
    const size_t smem = rows_smem_bytes(Npad, split);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const size_t max_ctas = 512 / cols;  // TMEM columns of the CTAs resident on one SM
    size_t smem_req = smem;
    if ((228 * 1024) / smem_req > max_ctas) smem_req = (228 * 1024) / (max_ctas + 1) + 1024;
    const int sh = ch.S * ch.heads;
    int slices = ((slices_per_sm < 1 ? 1 : slices_per_sm) * num_sms + sh - 1) / sh;
    if (slices < 1) slices = 1;
    if (slices > 64) slices = 64;
#define VQ_ROWS(SP, SLOT)                                                                                         \
    {                                                                                                             \
        static size_t granted = 0;                                                                                \
        if (smem_req > granted) {                                                                                 \
            cudaFuncSetAttribute(k_attention_rows_tc<SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,            \
                                 (int)smem_req);                                                                  \
            granted = smem_req;                                                                                   \
        }                                                                                                         \
        k_attention_rows_tc<SP><<<sh * slices, AR_THREADS, smem_req, st>>>(ch, uid, qkv, lo_off, O, list, act_off, \
                                                                           count, dpos, dcnt, slices, Npad, cols, \
                                                                           status, stats);                        \
    }
    if (split) VQ_ROWS(true, 1) else VQ_ROWS(false, 0)
#undef VQ_ROWS
    return cudaGetLastError();
}

}  // namespace vq
