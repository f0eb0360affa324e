// Incremental evaluation of the connected configurations (exact up to rounding).
//
// Sec. 3.2 removes the redundancy of the per-location operations by keying rows
// on their quantized history; it leaves the self-attention and the quantizer
// dense over every row of every configuration, and names attention "not yet
// optimized" (Sec. 3.2, Sec. 5.1).  This file removes most of that dense work
// without changing what is computed.
//
// Take a connected configuration c of sample s and a layer.  Let D be the
// positions whose row id differs from s's row id at the same position (they
// start at the first exchanged site; the ids of every other position are equal,
// so are their inputs).  For a row p outside D:
//
//  * the query is s's query and the keys/values differ from s's only at D, so
//    with s's softmax maximum m and normaliser l (scaled scores),
//      l'  = l - sum_{k in D, k<p} e_s(k) + sum_{k in D, k<p} e_c(k),
//      o'  = o + delta,  delta = ( sum_k e_c(k) (v_c(k) - o) - e_s(k) (v_s(k) - o) ) / l'
//    with e_x(k) = exp(q . k_x(k) / sqrt(dh) - m): |D| keys instead of p + 1.
//    A row whose removed weight exceeds half of l (cancellation) or whose new
//    scores overflow the old maximum is recomputed over all keys instead.
//
//  * its code is s's code c unless some codeword j gets closer: since
//      ||o+delta - W_j||^2 - ||o+delta - W_c||^2 = g_j - 2 delta . (W_j - W_c)
//    with g_j = ||o - W_j||^2 - ||o - W_c||^2 (Eq. vq's distances of s's row),
//    j cannot win while ||delta|| < rho_j = (g_j - eta) / (2 ||W_j - W_c||).
//    Each of s's rows keeps its CERT_T smallest rho_j (with j and g_j) and the
//    next one; a patched row with ||delta|| below every rho keeps c, one below
//    the next rho checks the listed candidates exactly, and any other row (or a
//    failed check) goes to the ordinary nearest-codeword search with o'.
//    eta is a rounding allowance on the distances (relative 2^-16).
//
// Rows in D (their query changed) are recomputed over all keys by
// k_inc_attention, which keeps s's keys and values for one head in shared
// memory and patches only the positions in D for each configuration.
//
// Row outcomes (per layer): the code is taken from s; or the row is searched
// with the corrected output; or its attention is recomputed, then searched.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "tc_common.cuh"

namespace vq {

namespace {

constexpr float CERT_ETA_REL = 1.52587890625e-05f;  // 2^-16

// 2^x with the SFU's approximate exponential (relative error ~2^-22; flushes denormals)
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Ascending list of the positions p in [lo, hi) with pred(p), written to out
// (at most cap entries); returns the full count to every thread.  Every thread
// of the block calls it; blockDim.x is a multiple of 32 and at most 1024.
template <typename Pred>
__device__ int block_compact(int lo, int hi, Pred pred, int* out, int cap, int* s_warp) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    int total = 0;
    for (int q = lo; q < hi; q += blockDim.x) {
        const int p = q + tid;
        const bool f = p < hi && pred(p);
        const unsigned m = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_warp[warp] = __popc(m);
        __syncthreads();
        int off = total;
        for (int w = 0; w < warp; ++w) off += s_warp[w];
        int add = 0;
        for (int w = 0; w < nw; ++w) add += s_warp[w];
        const int i = off + __popc(m & ((1u << lane) - 1));
        if (f && i < cap) out[i] = p;
        total += add;
        __syncthreads();
    }
    return total;
}

}  // namespace

// One warp, one sample row: the nearest codeword (lowest index on ties; codeword 0 when no
// distance is finite) from the row's distances dist[0..K) to every codeword, the row's
// near-tie count (added to `ties` by lane 0), and its certificate: the CERT_T smallest radii
// rho_j = (g_j - eta) / (2 ||W_j - W_c||), g_j = dist[j] - dist[c], ascending (lowest index
// first on equal radii) with j and g_j, then the next radius.  rho: K floats of the warp's
// shared scratch.  Every lane returns the codeword.
__device__ int cert_from_dist(const float* dist, float* rho, float eta, int K, const float* __restrict__ wd,
                              CertRow* __restrict__ cr, int& ties) {
    const int lane = threadIdx.x & 31;
    float v1 = INFINITY, v2 = INFINITY;
    int i1 = 0x7fffffff;
    for (int j = lane; j < K; j += 32) {
        const float v = dist[j];
        if (v < v1 || (v == v1 && j < i1)) { v2 = v1; v1 = v; i1 = j; }
        else if (v < v2) v2 = v;
    }
    for (int o = 16; o; o >>= 1) {
        const float ov1 = __shfl_xor_sync(0xffffffffu, v1, o), ov2 = __shfl_xor_sync(0xffffffffu, v2, o);
        const int oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
        if (ov1 < v1 || (ov1 == v1 && oi1 < i1)) { v2 = fminf(v1, ov2); v1 = ov1; i1 = oi1; }
        else v2 = fminf(v2, ov1);
    }
    const int c = i1 < K ? i1 : 0;  // no finite distance: codeword 0
    if (lane == 0 && K > 1 && (v2 - v1) < NEAR_TIE_REL * fmaxf(v1, 1e-30f)) ++ties;
    for (int j = lane; j < K; j += 32) {
        const float w = wd[(size_t)c * K + j];
        rho[j] = (j == c || w <= 0.f) ? INFINITY : (dist[j] - v1 - eta) / (2.f * w);
    }
    __syncwarp();
    // the CERT_T + 1 smallest radii, ascending (lowest index first on equal radii)
    int n = 0;
    for (int t = 0; t <= CERT_T; ++t) {
        float bv = INFINITY;
        int bj = 0x7fffffff;
        for (int j = lane; j < K; j += 32) {
            const float v = rho[j];
            if (v < bv || (v == bv && j < bj)) { bv = v; bj = j; }
        }
        for (int o = 16; o; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ov < bv || (ov == bv && oj < bj)) { bv = ov; bj = oj; }
        }
        if (t == CERT_T || bv == INFINITY) {
            if (lane == 0) cr->next = bv;
            break;
        }
        if (lane == 0) {
            cr->j[t] = bj;
            cr->rho[t] = bv;
            cr->gap[t] = dist[bj] - v1;
        }
        if (lane == (bj & 31)) rho[bj] = INFINITY;
        ++n;
        __syncwarp();
    }
    if (lane == 0) {
        cr->n = n;
        cr->eta = eta;
        cr->code = c;
    }
    __syncwarp();
    return c;
}

// ---- s's rows: nearest codeword and its certificate ---------------------------------
// One CTA of 256 threads per RB rows of the chunk's samples (row r = b * N + p),
// thread j computing codeword j's distances to the RB rows.
// Distances are expanded as ||o||^2 - 2 o.W_j + ||W_j||^2 in FP32 (as the
// ordinary search does); the certificate radii use the table wd[c][j] = ||W_c - W_j||.
template <int RB>
__global__ void __launch_bounds__(256)
k_base_cert(Chunk ch, const float* __restrict__ O, const float* __restrict__ codebook, const float* __restrict__ cnorm,
            const float* __restrict__ wd, int K, int d, int* __restrict__ code, CertRow* __restrict__ cert,
            long long* __restrict__ near_ties, int* __restrict__ counters, int* __restrict__ rc_cnt,
            long long* __restrict__ stats) {
    extern __shared__ __align__(16) float smem_f[];
    float* sO = smem_f;                    // [RB][d]
    float* sW = sO + RB * d;               // [32 dims][256 codewords]
    float* sDist = sW + 32 * 256;          // [RB][K]
    float* sRho = sDist + RB * K;          // [8 warps][K]
    __shared__ float sOsq[RB];
    __shared__ int sRow[RB];
    __shared__ float sCnMax;
    __shared__ int sTies;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int N = ch.N;
    const int r0 = blockIdx.x * RB;
    if (blockIdx.x == 0 && tid == 0) {  // the lists the classify and patch kernels fill next
        counters[CNT_V] = 0;
        counters[CNT_TCL] = counters[CNT_SCL] = counters[CNT_TCW] = counters[CNT_SCW] = 0;
        counters[CNT_EX] = 0;
    }
    if (blockIdx.x == 0)
        for (int b = tid; b < 2 * ch.S; b += blockDim.x) rc_cnt[b] = 0;  // head and tail counts per sample
    if (tid == 0) { sTies = 0; sCnMax = 0.f; }
    if (tid < RB) {
        const int r = r0 + tid, b = r / N, p = r - b * N;
        sRow[tid] = (b < ch.S && p < sample_N(ch, b)) ? ch.cfg_row[ch.cfg_off[b]] + p : -1;
    }
    __syncthreads();
    {
        float mx = 0.f;
        for (int j = tid; j < K; j += blockDim.x) mx = fmaxf(mx, cnorm[j]);
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(reinterpret_cast<int*>(&sCnMax), __float_as_int(mx));  // non-negative floats
    }
    for (int e = tid; e < RB * (d / 4); e += blockDim.x) {
        const int r = e / (d / 4), t4 = (e - r * (d / 4)) * 4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sRow[r] >= 0) v = *reinterpret_cast<const float4*>(O + (size_t)sRow[r] * d + t4);
        *reinterpret_cast<float4*>(sO + r * d + t4) = v;
    }
    __syncthreads();
    for (int r = warp; r < RB; r += 8) {
        float s = 0.f;
        for (int t = lane; t < d; t += 32) s = fmaf(sO[r * d + t], sO[r * d + t], s);
        s = warp_sum(s);
        if (lane == 0) sOsq[r] = s;
    }
    for (int jg = 0; jg < K; jg += 256) {
        const int j = jg + tid;
        float acc[RB];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r] = 0.f;
        // codeword j's next 32 dims travel in registers while the current ones are used
        float4 wn[8];
        auto load_w = [&](int d0) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                wn[q] = j < K ? *reinterpret_cast<const float4*>(codebook + (size_t)j * d + d0 + 4 * q)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        load_w(0);
        for (int d0 = 0; d0 < d; d0 += 32) {
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                sW[(4 * q) * 256 + tid] = wn[q].x;
                sW[(4 * q + 1) * 256 + tid] = wn[q].y;
                sW[(4 * q + 2) * 256 + tid] = wn[q].z;
                sW[(4 * q + 3) * 256 + tid] = wn[q].w;
            }
            __syncthreads();
            if (d0 + 32 < d) load_w(d0 + 32);
#pragma unroll 2
            for (int dd = 0; dd < 32; dd += 4) {
                const float w0 = sW[dd * 256 + tid], w1 = sW[(dd + 1) * 256 + tid];
                const float w2 = sW[(dd + 2) * 256 + tid], w3 = sW[(dd + 3) * 256 + tid];
#pragma unroll
                for (int r = 0; r < RB; ++r) {
                    const float4 o = *reinterpret_cast<const float4*>(sO + r * d + d0 + dd);
                    acc[r] = fmaf(o.x, w0, fmaf(o.y, w1, fmaf(o.z, w2, fmaf(o.w, w3, acc[r]))));
                }
            }
        }
        if (j < K) {
            const float cn = cnorm[j];
#pragma unroll
            for (int r = 0; r < RB; ++r) sDist[r * K + j] = fmaf(-2.f, acc[r], sOsq[r]) + cn;
        }
    }
    __syncthreads();
    int ties = 0;
    for (int r = warp; r < RB; r += 8) {
        const int row = sRow[r];
        if (row < 0) continue;  // warp-uniform
        const int c = cert_from_dist(sDist + r * K, sRho + warp * K, CERT_ETA_REL * (sOsq[r] + sCnMax), K, wd,
                                     cert + (r0 + r), ties);
        if (lane == 0) code[row] = c;
        __syncwarp();
    }
    if (ties) atomicAdd(&sTies, ties);
    __syncthreads();
    if (tid == 0 && sTies) atomicAdd(reinterpret_cast<unsigned long long*>(near_ties), (unsigned long long)sTies);
    if (tid == 0) {
        int n = 0;
        for (int r = 0; r < RB; ++r) n += sRow[r] >= 0;
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_BASE]), (unsigned long long)n);
    }
}

// ---- s's rows from the tensor-core distances (BF16 path) ------------------------------
// The distances come from the split-TF32 search of k_vq_tc (distance mode) over the
// list below, so the samples' codes are the ones that search gives; the certificate is
// taken from them as above.  Their error (about 2^-21 of ||o|| ||W||) is far inside eta.

// The chunk's sample rows, in the order of the certificate rows: entry b N + p is the
// row of position p of sample b (positions past the sample's length take its first row,
// whose distances are computed and ignored); list[0] holds the count S N.
__global__ void k_base_rows(Chunk ch, int* __restrict__ list) {
    const int total = ch.S * ch.N;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int b = i / ch.N, p = i - b * ch.N;
        list[1 + i] = ch.cfg_row[ch.cfg_off[b]] + (p < sample_N(ch, b) ? p : 0);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) list[0] = total;
}

// One warp per sample row r = b N + p: its distances dist[r][0..K) and ||o||^2 = osq[r]
// staged in shared memory, then code, near ties and certificate by cert_from_dist.
__global__ void __launch_bounds__(256)
k_base_cert_dist(Chunk ch, const float* __restrict__ dist, const float* __restrict__ osq,
                 const float* __restrict__ cnorm, const float* __restrict__ wd, int K, int* __restrict__ code,
                 CertRow* __restrict__ cert, long long* __restrict__ near_ties, int* __restrict__ counters,
                 int* __restrict__ rc_cnt, long long* __restrict__ stats) {
    extern __shared__ __align__(16) float smem_c[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* sD = smem_c + (size_t)warp * 2 * K;  // this warp's row: distances, then radii
    float* sRho = sD + K;
    __shared__ float sCnMax;
    __shared__ int sTies, sRows;
    if (blockIdx.x == 0 && tid == 0) {  // the lists the classify and patch kernels fill next
        counters[CNT_V] = 0;
        counters[CNT_TCL] = counters[CNT_SCL] = counters[CNT_TCW] = counters[CNT_SCW] = 0;
        counters[CNT_EX] = 0;
    }
    if (blockIdx.x == 0)
        for (int b = tid; b < 2 * ch.S; b += blockDim.x) rc_cnt[b] = 0;  // head and tail counts per sample
    if (tid == 0) { sTies = 0; sRows = 0; sCnMax = 0.f; }
    __syncthreads();
    {
        float mx = 0.f;
        for (int j = tid; j < K; j += blockDim.x) mx = fmaxf(mx, cnorm[j]);
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomicMax(reinterpret_cast<int*>(&sCnMax), __float_as_int(mx));  // non-negative floats
    }
    __syncthreads();
    const int N = ch.N, total = ch.S * N;
    int ties = 0, rows = 0;
    for (int r = blockIdx.x * 8 + warp; r < total; r += gridDim.x * 8) {
        const int b = r / N, p = r - b * N;
        if (p >= sample_N(ch, b)) continue;  // warp-uniform
        const float* dg = dist + (size_t)r * K;
        for (int j = 4 * lane; j < K; j += 128)  // K is a multiple of 16
            *reinterpret_cast<float4*>(sD + j) = *reinterpret_cast<const float4*>(dg + j);
        __syncwarp();
        const int c = cert_from_dist(sD, sRho, CERT_ETA_REL * (osq[r] + sCnMax), K, wd, cert + r, ties);
        if (lane == 0) code[ch.cfg_row[ch.cfg_off[b]] + p] = c;
        ++rows;
        __syncwarp();
    }
    if (lane == 0 && ties) atomicAdd(&sTies, ties);
    if (lane == 0 && rows) atomicAdd(&sRows, rows);
    __syncthreads();
    if (tid == 0 && sTies) atomicAdd(reinterpret_cast<unsigned long long*>(near_ties), (unsigned long long)sTies);
    if (tid == 0 && sRows)
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_BASE]), (unsigned long long)sRows);
}

// ---- s's rows with H > 1 quantizer heads (Eq. vq per segment) ---------------------------
// One warp per sample row.  Segment h of the row (dq = d / H values) is assigned against
// codebook h (distances ||o_h||^2 - 2 o_h . W_hj + ||W_hj||^2 in FP32, lowest index on
// ties) and its code goes to bits [h bits, (h + 1) bits) of the packed code.  The row's
// certificate keeps no candidate list: its radius is the smallest over the segments of
//   min_{j != c_h} (g_hj - eta_h) / (2 ||W_hj - W_hc||),  g_hj = ||o_h - W_hj||^2 - ||o_h - W_hc||^2,
// and since ||delta_h|| <= ||delta||, a connected row with ||delta|| below it keeps every
// segment's code; any other goes to the per-head search.  wd holds H tables [K][K].
__global__ void __launch_bounds__(256)
k_base_cert_heads(Chunk ch, const float* __restrict__ O, const float* __restrict__ codebook,
                  const float* __restrict__ cnorm, const float* __restrict__ wd, int K, int d, int H, int bits,
                  int* __restrict__ code, CertRow* __restrict__ cert, long long* __restrict__ near_ties,
                  int* __restrict__ counters, int* __restrict__ rc_cnt, long long* __restrict__ stats) {
    extern __shared__ __align__(16) float smem_h[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* sO = smem_h + warp * (d + K);  // this warp's row
    float* sDist = sO + d;                // its distances to one codebook
    const int N = ch.N, dq = d / H;
    if (blockIdx.x == 0 && tid == 0) {  // the lists the classify and patch kernels fill next
        counters[CNT_V] = 0;
        counters[CNT_TCL] = counters[CNT_SCL] = counters[CNT_TCW] = counters[CNT_SCW] = 0;
        counters[CNT_EX] = 0;
    }
    if (blockIdx.x == 0)
        for (int b = tid; b < 2 * ch.S; b += blockDim.x) rc_cnt[b] = 0;
    long long ties = 0, rows = 0;
    for (int r = blockIdx.x * 8 + warp; r < ch.S * N; r += gridDim.x * 8) {
        const int b = r / N, p = r - b * N;
        if (p >= sample_N(ch, b)) continue;  // warp-uniform
        const int row = ch.cfg_row[ch.cfg_off[b]] + p;
        for (int t = lane; t < d; t += 32) sO[t] = O[(size_t)row * d + t];
        __syncwarp();
        float radius = INFINITY;
        unsigned packed = 0;
        for (int h = 0; h < H; ++h) {
            const float* oh = sO + h * dq;
            float osq = 0.f;
            for (int t = lane; t < dq; t += 32) osq = fmaf(oh[t], oh[t], osq);
            osq = warp_sum(osq);
            const float* Wh = codebook + (size_t)h * K * dq;
            const float* cn = cnorm + (size_t)h * K;
            float v1 = INFINITY, v2 = INFINITY, cmax = 0.f;
            int i1 = 0x7fffffff;
            for (int j = lane; j < K; j += 32) {
                float dot = 0.f;
                for (int t = 0; t < dq; ++t) dot = fmaf(oh[t], Wh[(size_t)j * dq + t], dot);
                const float v = fmaf(-2.f, dot, osq) + cn[j];
                sDist[j] = v;
                cmax = fmaxf(cmax, cn[j]);
                if (v < v1 || (v == v1 && j < i1)) { v2 = v1; v1 = v; i1 = j; }
                else if (v < v2) v2 = v;
            }
            for (int o = 16; o; o >>= 1) {
                const float ov1 = __shfl_xor_sync(0xffffffffu, v1, o), ov2 = __shfl_xor_sync(0xffffffffu, v2, o);
                const int oi1 = __shfl_xor_sync(0xffffffffu, i1, o);
                cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
                if (ov1 < v1 || (ov1 == v1 && oi1 < i1)) { v2 = fminf(v1, ov2); v1 = ov1; i1 = oi1; }
                else v2 = fminf(v2, ov1);
            }
            __syncwarp();
            const int c = i1 < K ? i1 : 0;  // no finite distance: codeword 0
            const float eta = CERT_ETA_REL * (osq + cmax);
            const float* wdh = wd + (size_t)h * K * K + (size_t)c * K;
            float rmin = INFINITY;
            for (int j = lane; j < K; j += 32) {
                const float w = wdh[j];
                if (j != c && w > 0.f) rmin = fminf(rmin, (sDist[j] - v1 - eta) / (2.f * w));
            }
            for (int o = 16; o; o >>= 1) rmin = fminf(rmin, __shfl_xor_sync(0xffffffffu, rmin, o));
            radius = fminf(radius, rmin);
            packed |= (unsigned)c << (h * bits);
            if (lane == 0 && K > 1 && (v2 - v1) < NEAR_TIE_REL * fmaxf(v1, 1e-30f)) ++ties;
            __syncwarp();
        }
        if (lane == 0) {
            code[row] = (int)packed;
            CertRow* cr = cert + r;
            cr->next = radius;
            cr->eta = 0.f;
            cr->n = 0;
            cr->code = (int)packed;
            ++rows;
        }
        __syncwarp();
    }
    if (lane == 0 && ties) atomicAdd(reinterpret_cast<unsigned long long*>(near_ties), (unsigned long long)ties);
    if (lane == 0 && rows) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_BASE]), (unsigned long long)rows);
}

// ---- connected configurations: changed positions and the work lists ------------------
// One warp per connected configuration: the positions whose row id differs from
// the sample's (ascending, the first INC_MAX_KEYS kept) and their count.  With
// tc_ok (BF16 path) a configuration with at most PATCH_TC_KEYS of them joins the
// tensor-core patch list, any other is recomputed whole: it joins list_full and
// all its rows from the first changed site join the search list.  Without tc_ok
// every configuration joins the CUDA-core patch list (list_simt).
constexpr int PATCH_TC_KEYS = 16;

bool patch_tc_supported(int d, int heads) { return d / heads == 32 && (d == 128 || d == 256); }

__global__ void k_inc_classify(Chunk ch, const int* __restrict__ uid, int tc_ok, int* __restrict__ list_tc,
                               int* __restrict__ list_simt, short* __restrict__ dpos, int* __restrict__ dcnt,
                               int* __restrict__ vq_rows, long long* __restrict__ stats) {
    const int C = ch.counters[CNT_C];
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    long long full_rows = 0, whole_pairs = 0;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < C; c += nw) {
        const int ci = ch.cfg_i[c];
        if (ci < 0) continue;  // the sample itself (warp-uniform)
        const int b = ch.cfg_sample[c];
        const int rc = ch.cfg_row[c], rb = ch.cfg_row[ch.cfg_off[b]];
        const int N = cfg_N(ch, c);
        const int p0 = cfg_first_changed(ci, ch.cfg_j[c]);
        int nd = 0;
        for (int q = p0; q < N; q += 32) {
            const int p = q + lane;
            const bool f = p < N && uid[rc + p] != uid[rb + p];
            const unsigned m = __ballot_sync(0xffffffffu, f);
            const int i = nd + __popc(m & ((1u << lane) - 1));
            if (f && i < INC_MAX_KEYS) dpos[(size_t)c * INC_MAX_KEYS + i] = (short)p;
            nd += __popc(m);
        }
        if (!tc_ok) {
            if (lane == 0) {
                dcnt[c] = nd;
                list_simt[atomicAdd(&ch.counters[CNT_SCL], 1)] = c;
            }
        } else if (nd <= PATCH_TC_KEYS) {
            if (lane == 0) {
                dcnt[c] = nd;
                list_tc[atomicAdd(&ch.counters[CNT_TCL], 1)] = c;
            }
        } else {  // recomputed whole: every row from p0 is searched
            int base = 0;
            if (lane == 0) {
                dcnt[c] = nd;
                list_simt[atomicAdd(&ch.counters[CNT_SCL], 1)] = c;
                base = atomicAdd(&ch.counters[CNT_V], N - p0);
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            for (int p = p0 + lane; p < N; p += 32) vq_rows[base + p - p0] = rc + p;
            full_rows += lane == 0 ? N - p0 : 0;
            // rows p0 .. N - 1, row p attending to keys 0 .. p
            whole_pairs += lane == 0 ? (long long)(N - p0) * (N + p0 + 1) / 2 : 0;
        }
    }
    if (full_rows) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_FULL]), (unsigned long long)full_rows);
    if (whole_pairs)
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_WPAIRS]), (unsigned long long)whole_pairs);
}

// Next entry of a work list for the whole CTA (-1 when the list is done).
__device__ __forceinline__ int next_item(int* counters, int work_slot, int list_slot, int* s_item) {
    if (threadIdx.x == 0) *s_item = atomicAdd(&counters[work_slot], 1);
    __syncthreads();
    const int i = *s_item;
    __syncthreads();
    return i < counters[list_slot] ? i : -1;
}

// ---- connected configurations on the tensor cores (BF16 path, dh = 32) ----------------
// One work item = (sample b, tile of 128 positions, slice z of b's connected
// configurations).  The item stages what belongs to the sample once: the tile's
// queries (BF16, K-major) in shared memory, the sample's outputs o of the tile's rows in
// TMEM columns [d, 2d), ||o_h||, ||q~_h|| and the softmax statistics in registers, and
// the rows' certificates in shared memory.  It then walks the slice (every `slices`-th
// configuration of b with at most PATCH_TC_KEYS changed positions and its first changed
// position inside the tile).  Tile row r is TMEM lane r and belongs to threads r and
// r + 128, each of which takes half of the heads.  Per configuration c:
//   1. the changed positions' keys are staged beside each other (the sample's in slots
//      0..15, c's in 16..31, zero-filled) and their values transposed;
//   2. per head h: S_h = Q_h [K_s; K_c]_h^T (M = 128, N = 32) into TMEM columns 32h..;
//   3. a tile row is patched when its position is at or after c's first changed position
//      and not itself changed; per such row and head, the BF16 weights
//      e = exp(s / sqrt(dh) - m) of the changed keys before the row (the sample's
//      negated) form the A operand;
//   4. per head: E_h [V_s; V_c]_h (N = 32) into the columns the scores came from:
//      sum_k e_c v_c - e_s v_s;
//   5. per row: delta = (acc - (sum e_c - sum e_s) o) / l' with o read from TMEM; delta
//      goes back to TMEM, the two threads' partial norms are added, and the certificate
//      is checked as in k_inc_patch with ||delta|| replaced by ||delta|| + B, B a bound
//      on the error of the BF16 computation (below), and each listed candidate's
//      projection by |delta . (W_j - W_c)| + B ||W_j - W_c||;
//   6. only a row that is searched (certificate not met) has o + delta written to O; a
//      certified row keeps the sample's codeword and writes nothing else.  With split
//      operands (the path whose Q/K/V carry a BF16 lo plane) a row that the certificate
//      does not settle is listed instead, and k_inc_exact_delta forms its correction from
//      the split operands in FP32, so every output that reaches the search carries
//      FP32-grade error.  c's changed positions inside the tile are listed for the
//      recompute and the search.
//
// The bound B.  The kernel reads only the hi planes: q~ = bf16(q), k~, v~ (each
// within 2^-9 relative of the exact value, or equal to it on the plain BF16
// path), e~ = exp2(s~ sl2 - m) with s~ = q~ . k~ accumulated in FP32, and the
// MMA takes e^ = bf16(e~).  Per head, |s~ - s| <= 2^-8 (1 + 2^-7) ||q~|| ||k~||
// (two relative 2^-9 perturbations plus the 32-term FP32 sum), so
// |e~ / e - 1| <= tau = 2^dx - 1 + 2^-20 with dx = 2^-8 1.01 sl2 ||q~|| kmax, kmax
// the largest ||k~|| among the head's changed keys (the sample's and the
// configuration's; the 2^-20 covers ex2.approx and the rounding of its argument;
// 2^dx - 1 is bounded by y + y^2, y = dx ln 2, which holds for y <= 1), and
// e^ v~ - e v = (e^ - e) v~ + e (v~ - v) has norm <= e (tau + 2^-8) ||v~||.
// With A = (tau + 2^-8) sum_k e~ ||v~|| and T = tau sum_k e~ over the row's
// changed keys, the numerator and the weight sum w differ from exact by at most
// 1.1 (A + T ||o||) and the normaliser by at most 1.1 T (e <= 1.1 e~ while
// tau <= 0.1), so
//   ||delta~_h - delta_h|| <= B_h = 1.1 (A + T (||o_h|| + ||delta~_h||)) / (l~' - 1.1 T)
// per head and B = sqrt(sum_h B_h^2).  A row with tau > 0.1, or
// l~' - 1.1 T <= l~' / 2, is recomputed over all keys.
using tc::cp_async16;
using tc::cp_async_wait_all;

// The BF16 weights of one head for a row with nk changed keys before it (nk <= NKB):
// e_s = exp(s_s / sqrt(dh) - m) negated in slots 0..15, e_c in 16..31, zeros beyond
// nk; seb, sec their sums; guard set when a new score overflows the sample's max.
// sv += sum_k e ||v~|| over the row's changed keys (vn2[k] = (||v~_s||, ||v~_c||) of
// slot pair k), the value-norm sum of the bound B above.
template <int NKB>
__device__ __forceinline__ void patch_weights(uint32_t (&s)[32], int nk, float sl2, float m2, bool& guard, float& seb,
                                              float& sec, uint32_t (&e16)[16], const float2* __restrict__ vn2,
                                              float& sv) {
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        float eb = 0.f, ec = 0.f;
        if (kk < NKB && kk < nk) {
            const float xc = __uint_as_float(s[16 + kk]) * sl2 - m2;
            if (xc > 115.f) guard = true;
            eb = ex2_approx(__uint_as_float(s[kk]) * sl2 - m2);
            ec = ex2_approx(fminf(xc, 115.f));
            const float2 v = vn2[kk];
            sv = fmaf(eb, v.x, fmaf(ec, v.y, sv));
        }
        seb += eb;
        sec += ec;
        s[kk] = __float_as_uint(-eb);
        s[16 + kk] = __float_as_uint(ec);
    }
#pragma unroll
    for (int j2 = 0; j2 < 16; ++j2) {
        const __nv_bfloat162 v2 = __floats2bfloat162_rn(__uint_as_float(s[2 * j2]), __uint_as_float(s[2 * j2 + 1]));
        e16[j2] = *reinterpret_cast<const uint32_t*>(&v2);
    }
}

constexpr int RES_THREADS = 512;  // four threads per tile row, a quarter of the heads each
constexpr int RES_LCAP = 1024;    // list entries gathered before one flush to the global lists
constexpr int RES_MAX_CFG = 544;  // a sample's connected configurations one item may walk (N <= 256: <= 513)

struct ResLayout {
    size_t q, e, k, v, cert, n2, pr, kx, vn, dp, vq, full, bar, total;
};
__host__ __device__ inline ResLayout res_layout(int d, int H) {
    ResLayout L;
    size_t o = 0;
    auto a128 = [](size_t x) { return (x + 127) & ~(size_t)127; };
    L.q = o;    o += a128((size_t)128 * d * 2);
    L.e = o;    o += a128((size_t)128 * d * 2);
    L.k = o;    o += (size_t)H * 2048;
    L.v = o;    o += (size_t)H * 2048;
    L.cert = o; o += a128(128 * sizeof(CertRow));
    L.n2 = o;   o += 4 * 128 * sizeof(float2);
    L.pr = o;   o += 4 * 128 * CERT_T * sizeof(float);
    L.kx = o;   o += (size_t)H * sizeof(float);
    L.vn = o;   o += (size_t)H * 32 * sizeof(float);
    L.dp = o;   o += 2 * 64 * sizeof(int);
    L.vq = o;   o += RES_LCAP * sizeof(int);
    L.full = o; o += RES_LCAP * sizeof(int2);
    L.bar = o;  o += 64;
    L.total = o + 128;  // + alignment of the dynamic base
    return L;
}

__global__ void __launch_bounds__(RES_THREADS, 1)
k_inc_patch_res(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv,
                float* __restrict__ O, const float2* __restrict__ bstat, const CertRow* __restrict__ cert,
                const float* __restrict__ codebook, const float* __restrict__ wd, int* __restrict__ code,
                int* __restrict__ vq_rows, const int* __restrict__ act_off, int2* __restrict__ rc_rows,
                int* __restrict__ rc_cnt, const short* __restrict__ dpos, const int* __restrict__ dcnt, int split,
                int2* __restrict__ ex_rows, int slices, uint32_t tmem_cols, int* __restrict__ status,
                long long* __restrict__ stats) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    constexpr int DH = 32;
    constexpr int HQ = 2;                         // most heads per thread (H <= 8)
    const int d = ch.d, H = ch.heads, NM = ch.N;  // d == 32 H, H in {4, 8}
    const int hq = H / 4;                         // heads per thread
    const ResLayout L = res_layout(d, H);
    uint8_t* sQ = smem + L.q;    // [128 x d] the tile's queries
    uint8_t* sE = smem + L.e;    // [128 x d] the weights, head h in columns 32h .. 32h + 31
    uint8_t* sK = smem + L.k;    // per head [32 key slots x 32 dims]
    uint8_t* sV = smem + L.v;    // per head [32 key slots x 32 dims], read as the MN-major B operand
    const CertRow* sCert = reinterpret_cast<const CertRow*>(smem + L.cert);  // [128]
    float2* sN2 = reinterpret_cast<float2*>(smem + L.n2);  // [4 quarters][128]: ||delta~||^2, B^2 (-1: guard)
    float* sP = reinterpret_cast<float*>(smem + L.pr);     // [4 quarters][128][CERT_T]: projections
    float* sKx = reinterpret_cast<float*>(smem + L.kx);    // [H] largest ||k~|| of the key slots
    float2* sVn = reinterpret_cast<float2*>(smem + L.vn);  // [H][16] ||v~|| of slot pairs (sample's, c's)
    // [2 configurations: this, next][64]: changed positions in 0..15, their row ids in 32..63
    // (the sample's in 32..47, the configuration's in 48..63)
    int* sD = reinterpret_cast<int*>(smem + L.dp);
    int* sVq = reinterpret_cast<int*>(smem + L.vq);        // rows to search
    int2* sFull = reinterpret_cast<int2*>(smem + L.full);  // rows to recompute (row, position)
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 1);
    __shared__ int sNvq, sNfull, sBase[2], s_item;
    __shared__ int sCL[RES_MAX_CFG];  // the item's configurations, as indices into its slice
    __shared__ int s_warp[32];
    __shared__ long long sCnt[4];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int qq = tid >> 7, r = tid & 127;
    const int h0 = qq * hq;
    const int ld = 3 * d;
    const int nkv = H * 32 * (DH / 8);  // 16-byte chunks of one configuration's keys (or values)
    const float sl2 = 1.4426950408889634f * rsqrtf((float)DH);
    const float cdx = 3.90625e-3f * 1.01f * sl2;  // 2^-8 (1 + 2^-7), log2 units
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
        sNvq = 0;
        sNfull = 0;
    }
    if (tid < 4) sCnt[tid] = 0;
    if (warp == 0) tc::tmem_alloc(tmem_holder, tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;  // warps w, w + 4, w + 8, w + 12 share lanes
    const uint32_t t_acc = tmem + lane_base, t_o = tmem + lane_base + (uint32_t)d;
    uint32_t phase = 0;
    bool ok = true;
    unsigned n_patched = 0, n_cert = 0, n_full = 0, n_pairs = 0;  // this thread's counts
    const int ntile = (NM + 127) / 128;
    const int items = ch.S * ntile * slices;

    // keys (part 1) or values (part 2) of configuration c's changed positions, the sample's
    // in slots 0..15 and c's in 16..31, zero-filled, into dst with cp.async; dl: c's changed
    // positions and their row ids in shared memory (layout of sD).  Both tiles take the
    // K-major core layout of [32 slots x 32 dims] per head; the value MMA reads theirs as an
    // MN-major B operand.
    auto stage_kv = [&](uint8_t* dst, int part, const int* dl, int nd) {
        for (int u = tid; u < nkv; u += RES_THREADS) {
            const int h = u / (32 * (DH / 8)), rem = u - h * 32 * (DH / 8);
            const int n = rem & 31, t8 = (rem >> 5) * 8;
            const bool in = (n & 15) < nd;
            cp_async16(tc::smem_u32(dst + h * 2048 + tc::core_off(n, t8, DH)),
                       in ? qkv + (size_t)dl[32 + n] * ld + part * d + h * DH + t8 : qkv, in ? 16 : 0);
        }
    };
    // c's changed positions and their row ids into dl (lanes 0 .. nd - 1 of warp w0)
    auto load_changed = [&](int* dl, int c, int nd, const int* ub, const int* uc, int w0) {
        const int k = tid - 32 * w0;
        if (k >= 0 && k < nd) {
            const int q = dpos[(size_t)c * INC_MAX_KEYS + k];
            dl[k] = q;
            dl[32 + k] = ub[q];
            dl[48 + k] = uc[q];
        }
    };

    // the 128 threads of the four warps that hold tile rows 32 (warp % 4) .. + 31
    auto quad_sync = [&]() { asm volatile("bar.sync %0, 128;" ::"r"(1 + (warp & 3)) : "memory"); };

    for (;;) {
        if (tid == 0) s_item = atomicAdd(&ch.counters[CNT_TCW], 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= items || !ok) break;
        const int tq = item / (ch.S * slices);  // the last tiles (most patched rows) first
        const int rest = item - tq * ch.S * slices;
        const int b = rest / slices, z = rest - b * slices;
        const int t0 = (ntile - 1 - tq) * 128;
        const int N = sample_N(ch, b);
        if (t0 >= N) continue;
        const int tend = min(N, t0 + 128);
        const int cb0 = ch.cfg_off[b], cb1 = ch.cfg_off[b + 1];
        // the slice's configurations patched here (at most PATCH_TC_KEYS changed positions, the
        // first inside the tile or before it), in order; the walk below reads them from smem
        const int cs0 = cb0 + 1 + z;
        const int ncand = cs0 < cb1 ? (cb1 - cs0 + slices - 1) / slices : 0;
        const int nC = block_compact(
            0, min(ncand, RES_MAX_CFG),
            [&](int i) {
                const int cc = cs0 + i * slices;
                return dcnt[cc] <= PATCH_TC_KEYS && cfg_first_changed(ch.cfg_i[cc], ch.cfg_j[cc]) < tend;
            },
            sCL, RES_MAX_CFG, s_warp);
        if (nC == 0) continue;
        int ci = 0;
        int c = cs0 + sCL[0] * slices;
        const int rb = ch.cfg_row[cb0];
        const int* ub = uid + rb;
        const int p = t0 + r;
        const bool valid = p < N;
        // ---- the sample's tile: queries and certificate rows (cp.async), outputs into TMEM
        for (int u = tid; u < 128 * (d / 8); u += RES_THREADS) {
            const int rr = u / (d / 8), k8 = (u - rr * (d / 8)) * 8;
            const bool in = t0 + rr < N;
            const __nv_bfloat16* src = in ? qkv + (size_t)ub[t0 + rr] * ld + k8 : qkv;
            cp_async16(tc::smem_u32(sQ + tc::core_off(rr, k8, d)), src, in ? 16 : 0);
        }
        {
            constexpr int CW = (int)(sizeof(CertRow) / 16);  // 16-byte words of a certificate row
            const uint8_t* cg = reinterpret_cast<const uint8_t*>(cert + (size_t)b * NM + t0);
            for (int u = tid; u < 128 * CW; u += RES_THREADS) {
                const bool in = t0 + u / CW < N;
                cp_async16(tc::smem_u32(smem + L.cert + (size_t)u * 16),
                           in ? cg + (size_t)u * 16 : reinterpret_cast<const uint8_t*>(cert), in ? 16 : 0);
            }
        }
        float on[HQ], qn[HQ];
        float2 mls[HQ];
        {
            const float* orow = O + (size_t)(rb + (valid ? p : 0)) * d;
#pragma unroll
            for (int hh = 0; hh < HQ; ++hh) {
                on[hh] = 0.f;
                mls[hh] = make_float2(0.f, 1.f);
                if (hh >= hq) continue;
                const int h = h0 + hh;
                uint32_t a[32];
                float s2 = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float4 o4 = valid ? *reinterpret_cast<const float4*>(orow + h * 32 + 4 * t)
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
                    a[4 * t] = __float_as_uint(o4.x);
                    a[4 * t + 1] = __float_as_uint(o4.y);
                    a[4 * t + 2] = __float_as_uint(o4.z);
                    a[4 * t + 3] = __float_as_uint(o4.w);
                    s2 = fmaf(o4.x, o4.x, fmaf(o4.y, o4.y, fmaf(o4.z, o4.z, fmaf(o4.w, o4.w, s2))));
                }
                on[hh] = sqrtf(s2);
                tc::tmem_st32(t_o + h * 32, a);
                if (valid) mls[hh] = bstat[((size_t)b * NM + p) * H + h];
            }
        }
        // the first configuration's changed positions, keys and values
        int buf = 0;
        int nd = dcnt[c], rc = ch.cfg_row[c], p0 = cfg_first_changed(ch.cfg_i[c], ch.cfg_j[c]);
        load_changed(sD, c, nd, ub, uid + rc, 0);
        __syncthreads();
        stage_kv(sK, 1, sD, nd);
        stage_kv(sV, 2, sD, nd);
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int hh = 0; hh < HQ; ++hh) {  // ||q~_h|| in the bound's units
            qn[hh] = 0.f;
            if (hh >= hq) continue;
            float s2 = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < 4; ++c8) {
                const uint4 u = *reinterpret_cast<const uint4*>(sQ + tc::core_off(r, (h0 + hh) * 32 + c8 * 8, d));
                const __nv_bfloat162* b2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = __bfloat1622float2(b2[k]);
                    s2 = fmaf(f.x, f.x, fmaf(f.y, f.y, s2));
                }
            }
            qn[hh] = cdx * sqrtf(s2);
        }
        const CertRow& cr = sCert[r];
        // ---- the slice's configurations; the next one's keys and values load during this one
        while (ok) {
            const int* dl = sD + buf * 64;
            // staged keys and values of c: slot norms (one slot of one tile per thread; a warp
            // covers the 32 slots of one head): the values' per slot, the keys' largest per head
            for (int u = tid; u < 2 * H * 32; u += RES_THREADS) {
                const int kv = u / (H * 32), hn = u - kv * (H * 32);
                const int h = hn >> 5, n = hn & 31;
                const uint8_t* tile = (kv ? sV : sK) + h * 2048;
                float s2 = 0.f;
#pragma unroll
                for (int c8 = 0; c8 < 4; ++c8) {
                    const uint4 x = *reinterpret_cast<const uint4*>(tile + tc::core_off(n, c8 * 8, DH));
                    const __nv_bfloat162* b2 = reinterpret_cast<const __nv_bfloat162*>(&x);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 f = __bfloat1622float2(b2[k]);
                        s2 = fmaf(f.x, f.x, fmaf(f.y, f.y, s2));
                    }
                }
                const float nrm = sqrtf(s2);
                if (kv) {
                    reinterpret_cast<float*>(sVn)[h * 32 + (n & 15) * 2 + (n >> 4)] = nrm;
                } else {
                    // non-negative floats order as their bit patterns
                    const unsigned mx = __reduce_max_sync(0xffffffffu, __float_as_uint(nrm));
                    if (n == 0) sKx[h] = __uint_as_float(mx);
                }
            }
            // this row's role: patched (at or after p0, not changed), with nk changed keys before it
            int nk = 0;
            bool changed = false;
            for (int k = 0; k < nd; ++k) {
                const int q = dl[k];
                nk += q < p;
                changed |= q == p;
            }
            const bool prow = valid && p >= p0 && !changed;
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {  // S_h = Q_h [K_s; K_c]_h^T
                tc::tc_fence_after();
                const uint64_t dq = tc::desc_kmajor_none(tc::smem_u32(sQ), 128, (d / 8) * 128);
                for (int h = 0; h < H; ++h) {
                    const uint64_t dk = tc::desc_kmajor_none(tc::smem_u32(sK + h * 2048), 128, (DH / 8) * 128);
#pragma unroll
                    for (int ks = 0; ks < DH / 16; ++ks)
                        tc::mma_bf16(tmem + h * 32, dq + (uint64_t)(h * DH + ks * 16), dk + (uint64_t)(ks * 16),
                                     tc::idesc_bf16_f32(128, 32), ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            // the next configuration of the slice, while the scores form (its changed positions by
            // the last warp: warp 0 issues the MMAs)
            const int cn = ci + 1 < nC ? cs0 + sCL[ci + 1] * slices : -1;
            int nd_n = 0, rc_n = 0, p0_n = 0;
            int* dl_n = sD + (buf ^ 1) * 64;
            if (cn >= 0) {
                nd_n = dcnt[cn];
                rc_n = ch.cfg_row[cn];
                p0_n = cfg_first_changed(ch.cfg_i[cn], ch.cfg_j[cn]);
                load_changed(dl_n, cn, nd_n, ub, uid + rc_n, RES_THREADS / 32 - 1);
            }
            // every thread waits for the scores itself (a timeout is settled at the end barrier)
            ok = tc::mbar_wait(bar, phase, status) && ok;
            phase ^= 1;
            tc::tc_fence_after();
            float w[HQ], inv[HQ], ea[HQ], et[HQ];
            bool guard = false;
            // warps sharing TMEM lanes hold the same rows: they skip rows without work together
            const bool wact = __any_sync(0xffffffffu, prow);
            const int nkw = __reduce_max_sync(0xffffffffu, prow ? nk : 0);
            const int nkr = prow ? nk : 0;
            if (wact) {
#pragma unroll
                for (int hh = 0; hh < HQ; ++hh) {
                    if (hh >= hq) break;
                    const int h = h0 + hh;
                    uint32_t s[32];
                    tc::tmem_ld32(t_acc + h * 32, s);
                    const float2 ml = mls[hh];
                    const float m2 = ml.x * 1.4426950408889634f;
                    float seb = 0.f, sec = 0.f, sv = 0.f;
                    uint32_t e16[16];
                    const float2* vn2 = sVn + h * 16;
                    if (nkw <= 4)
                        patch_weights<4>(s, nkr, sl2, m2, guard, seb, sec, e16, vn2, sv);
                    else if (nkw <= 8)
                        patch_weights<8>(s, nkr, sl2, m2, guard, seb, sec, e16, vn2, sv);
                    else
                        patch_weights<16>(s, nkr, sl2, m2, guard, seb, sec, e16, vn2, sv);
                    // the bound's A and T from tau of the head's largest changed key norm
                    const float y = qn[hh] * sKx[h] * (0.69314718f * 1.0001f);
                    if (y > 0.09f) guard = true;
                    const float tau = fmaf(y, y, y) + 9.5367431640625e-07f;  // + 2^-20
                    const float aa = (tau + 3.90625e-3f) * sv, at = tau * (seb + sec);
#pragma unroll
                    for (int c8 = 0; c8 < 4; ++c8)
                        *reinterpret_cast<uint4*>(sE + tc::core_off(r, h * 32 + c8 * 8, d)) =
                            make_uint4(e16[4 * c8], e16[4 * c8 + 1], e16[4 * c8 + 2], e16[4 * c8 + 3]);
                    if (!(seb <= 0.5f * ml.y)) guard = true;  // cancellation
                    w[hh] = sec - seb;
                    const float lp = ml.y - seb + sec;
                    if (!(lp - 1.1f * at > 0.5f * lp)) guard = true;
                    inv[hh] = 1.f / lp;
                    const float f = 1.1f / (lp - 1.1f * at);
                    ea[hh] = aa * f;
                    et[hh] = at * f;
                }
            }
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            if (tid == 0) {  // E_h [V_s; V_c]_h into the columns the scores came from
                tc::tc_fence_after();
                const uint64_t de = tc::desc_kmajor_none(tc::smem_u32(sE), 128, (d / 8) * 128);
                for (int h = 0; h < H; ++h) {
                    // MN-major B: 8-slot groups (K) 512 bytes apart, 8-dim groups (N) 128 bytes apart
                    const uint64_t dv = tc::desc_kmajor_none(tc::smem_u32(sV + h * 2048), 512, 128);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
                        tc::mma_bf16(tmem + h * 32, de + (uint64_t)(h * 32 + ks * 16), dv + (uint64_t)(ks * 64),
                                     tc::idesc_bf16_f32_bmn(128, DH), ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            // the score MMAs are done with sK (every thread waited), and dl_n is visible
            if (cn >= 0) stage_kv(sK, 1, dl_n, nd_n);
            ok = tc::mbar_wait(bar, phase, status) && ok;
            phase ^= 1;
            tc::tc_fence_after();
            if (cn >= 0) stage_kv(sV, 2, dl_n, nd_n);  // the value MMAs are done with sV
            // pass A: delta = (acc - w o) / l' for the own heads, back into TMEM; partial norm and B^2
            float n2 = 0.f, b2 = 0.f;
#pragma unroll
            for (int hh = 0; hh < HQ; ++hh) {
                if (hh >= hq || !wact) break;
                const int h = h0 + hh;
                float hn2 = 0.f;
#pragma unroll
                for (int c16 = 0; c16 < 32; c16 += 16) {  // two 16-column halves of the head
                    uint32_t a[16], o[16];
                    tc::tmem_ld16(t_acc + h * 32 + c16, a);
                    tc::tmem_ld16(t_o + h * 32 + c16, o);
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const float dv = (__uint_as_float(a[t]) - w[hh] * __uint_as_float(o[t])) * inv[hh];
                        hn2 = fmaf(dv, dv, hn2);
                        a[t] = __float_as_uint(dv);
                    }
                    tc::tmem_st16(t_acc + h * 32 + c16, a);
                }
                n2 += hn2;
                // B_h = 1.1 (A + T (||o_h|| + ||delta~_h||)) / (l~' - 1.1 T)
                const float bh = ea[hh] + et[hh] * (on[hh] + sqrtf(hn2));
                b2 = fmaf(bh, bh, b2);
            }
            sN2[tid] = make_float2(n2, guard ? -1.f : b2);
            quad_sync();
            float bnd;
            {  // the same sums, in the same order, for the row's four threads
                const float2 a0 = sN2[r], a1 = sN2[128 + r], a2 = sN2[256 + r], a3 = sN2[384 + r];
                n2 = ((a0.x + a1.x) + a2.x) + a3.x;
                guard = a0.y < 0.f || a1.y < 0.f || a2.y < 0.f || a3.y < 0.f;
                bnd = guard ? 0.f : sqrtf(((a0.y + a1.y) + a2.y) + a3.y);
            }
            int md = -1, nc = 0;
            if (prow) {
                if (guard) {
                    md = 2;
                } else {
                    // ||delta|| <= ||delta~|| + B for the exact correction of these inputs
                    const float dn = sqrtf(n2) + bnd;
                    if (!(dn < cr.next)) {
                        md = 1;
                    } else {
                        while (nc < cr.n && cr.rho[nc] <= dn) ++nc;
                        md = nc ? 3 : 0;
                    }
                }
            }
            // pass B: exact check of the listed candidates, each thread over its heads
            // (md agrees between the warps of a row, so their TMEM loads stay warp-uniform)
            // md agrees between the four warps of a quad (the same rows), so they enter together
            if (__any_sync(0xffffffffu, md == 3)) {
                {
                    float proj[CERT_T];
#pragma unroll
                    for (int i = 0; i < CERT_T; ++i) proj[i] = 0.f;
                    const float* wc = codebook + (size_t)(md == 3 ? cr.code : 0) * d;
                    for (int hc = 0; hc < 2 * hq; ++hc) {  // 16-column halves of the own heads
                        const int col = (h0 + (hc >> 1)) * 32 + (hc & 1) * 16;
                        uint32_t a[16];
                        tc::tmem_ld16(t_acc + col, a);
                        if (md == 3) {
#pragma unroll
                            for (int i = 0; i < CERT_T; ++i) {
                                if (i >= nc) break;
                                const float* wj = codebook + (size_t)cr.j[i] * d + col;
                                float sacc = 0.f;
#pragma unroll
                                for (int t = 0; t < 16; t += 4) {
                                    const float4 a4 = *reinterpret_cast<const float4*>(wj + t);
                                    const float4 c4 = *reinterpret_cast<const float4*>(wc + col + t);
                                    sacc = fmaf(__uint_as_float(a[t]), a4.x - c4.x, sacc);
                                    sacc = fmaf(__uint_as_float(a[t + 1]), a4.y - c4.y, sacc);
                                    sacc = fmaf(__uint_as_float(a[t + 2]), a4.z - c4.z, sacc);
                                    sacc = fmaf(__uint_as_float(a[t + 3]), a4.w - c4.w, sacc);
                                }
                                proj[i] += sacc;
                            }
                        }
                    }
                    if (md == 3) {
#pragma unroll
                        for (int i = 0; i < CERT_T; ++i) sP[tid * CERT_T + i] = proj[i];
                    }
                }
                quad_sync();
                if (md == 3) {
                    md = 0;
                    for (int i = 0; i < nc; ++i) {
                        const float wj = wd[(size_t)cr.code * ch.K + cr.j[i]];  // ||W_j - W_c||
                        const float pj = ((sP[r * CERT_T + i] + sP[(128 + r) * CERT_T + i]) +
                                          sP[(256 + r) * CERT_T + i]) + sP[(384 + r) * CERT_T + i];
                        if (!(cr.gap[i] - 2.f * (pj + bnd * wj) > cr.eta)) md = 1;
                    }
                }
            }
            // split operands: a row the certificate does not settle gets its exact correction
            // from them (k_inc_exact_delta) before the search
            if (split && md == 1 && qq == 0) ex_rows[atomicAdd(&ch.counters[CNT_EX], 1)] = make_int2(rc + p, p);
            // a searched row: o + delta goes to O for the vector quantizer
            if (!split && __any_sync(0xffffffffu, md == 1)) {
                float* xo = O + (size_t)(rc + (p < N ? p : 0)) * d;
                for (int hc = 0; hc < 2 * hq; ++hc) {  // 16-column halves of the own heads
                    const int col = (h0 + (hc >> 1)) * 32 + (hc & 1) * 16;
                    uint32_t a[16], o[16];
                    tc::tmem_ld16(t_acc + col, a);
                    tc::tmem_ld16(t_o + col, o);
                    if (md == 1) {
#pragma unroll
                        for (int t = 0; t < 16; t += 4)
                            *reinterpret_cast<float4*>(xo + col + t) = make_float4(
                                __uint_as_float(o[t]) + __uint_as_float(a[t]),
                                __uint_as_float(o[t + 1]) + __uint_as_float(a[t + 1]),
                                __uint_as_float(o[t + 2]) + __uint_as_float(a[t + 2]),
                                __uint_as_float(o[t + 3]) + __uint_as_float(a[t + 3]));
                    }
                }
            }
            if (qq == 0) {
                if (md == 0) code[rc + p] = cr.code;
                if (md >= 1) sVq[atomicAdd(&sNvq, 1)] = rc + p;
                if (md == 2) sFull[atomicAdd(&sNfull, 1)] = make_int2(rc + p, p);
                n_patched += (md == 0 || md == 1);
                n_cert += md == 0;
                n_full += md == 2;
                n_pairs += prow ? nk : 0;
            }
            // c's changed positions inside the tile: recomputed, then searched
            if (tid < nd && dl[tid] >= t0 && dl[tid] < tend) {
                sVq[atomicAdd(&sNvq, 1)] = rc + dl[tid];
                sFull[atomicAdd(&sNfull, 1)] = make_int2(rc + dl[tid], dl[tid]);
                ++n_full;
            }
            cp_async_wait_all();
            tc::tc_fence_before();
            ok = __syncthreads_and(ok) != 0;
            if (!ok) break;
            // the gathered lists go out when another configuration might not fit, and at the end
            const bool last = cn < 0;
            if (last || sNvq > RES_LCAP - 144 || sNfull > RES_LCAP - 144) {
                if (tid == 0) {
                    sBase[0] = sNvq ? atomicAdd(&ch.counters[CNT_V], sNvq) : 0;
                    sBase[1] = sNfull ? act_off[cb0] + atomicAdd(&rc_cnt[b], sNfull) : 0;
                }
                __syncthreads();
                for (int i = tid; i < sNvq; i += RES_THREADS) vq_rows[sBase[0] + i] = sVq[i];
                for (int i = tid; i < sNfull; i += RES_THREADS) rc_rows[sBase[1] + i] = sFull[i];
                __syncthreads();
                if (tid == 0) { sNvq = 0; sNfull = 0; }
                __syncthreads();
            }
            if (last) break;
            ++ci;
            c = cn;
            nd = nd_n;
            rc = rc_n;
            p0 = p0_n;
            buf ^= 1;
        }
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[0]), (unsigned long long)n_patched);
    atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[1]), (unsigned long long)n_cert);
    atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[2]), (unsigned long long)n_full);
    atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[3]), (unsigned long long)n_pairs);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
    if (tid == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_PATCHED]), (unsigned long long)sCnt[0]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_CERT]), (unsigned long long)sCnt[1]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_FULL]), (unsigned long long)sCnt[2]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_PPAIRS]), (unsigned long long)sCnt[3]);
    }
}

// ---- split operands: exact correction of the rows the certificate did not settle -------
// One warp per listed row (row r of configuration c, position p, the sample's query):
// lane l holds dims [l PER, (l + 1) PER) of every vector, a head (32 dims) spans 32 / PER
// lanes.  For each changed position k < p of c (ascending in dpos), with q, k and v read
// as hi + lo from the two planes and the sample's softmax maximum m and sum l,
//   e_s = exp(q . k_s / sqrt(32) - m),  e_c = exp(q . k_c / sqrt(32) - m),
//   o' = o + (sum e_c (v_c - o) - e_s (v_s - o)) / (l - sum e_s + sum e_c)
// in FP32; o' goes to O[r] for the nearest-codeword search.  The patch kernel lists only
// rows without cancellation or overflow of the new scores (its guard), and at most
// PATCH_TC_KEYS changed positions.
template <int PER>
__device__ __forceinline__ void ld_split(const __nv_bfloat16* __restrict__ p, size_t lo_off, float (&x)[PER]) {
#pragma unroll
    for (int i = 0; i < PER; i += 4) {
        const uint2 h = *reinterpret_cast<const uint2*>(p + i);
        const uint2 l = *reinterpret_cast<const uint2*>(p + lo_off + i);
        const float2 h0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.x));
        const float2 h1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.y));
        const float2 l0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l.x));
        const float2 l1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&l.y));
        x[i] = h0.x + l0.x;
        x[i + 1] = h0.y + l0.y;
        x[i + 2] = h1.x + l1.x;
        x[i + 3] = h1.y + l1.y;
    }
}

template <int PER>
__global__ void __launch_bounds__(256)
k_inc_exact_delta(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv, size_t lo_off,
                  float* __restrict__ O, const float2* __restrict__ bstat, const short* __restrict__ dpos,
                  const int* __restrict__ dcnt, const int2* __restrict__ list, const int* __restrict__ n_list) {
    constexpr int LPH = 32 / PER;  // lanes per head (32 dims)
    const int n = *n_list;
    const int d = ch.d, H = ch.heads, ld = 3 * d;
    const int lane = threadIdx.x & 31, h = lane / LPH;
    const float rs = 0.17677669529663688f;  // 1 / sqrt(32)
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += (gridDim.x * blockDim.x) >> 5) {
        const int2 e = list[i];
        const int r = e.x, p = e.y;
        const int c = ch.row_cfg[r], b = ch.cfg_sample[c];
        const int rb = ch.cfg_row[ch.cfg_off[b]], rc = ch.cfg_row[c];
        const int* ub = uid + rb;
        const int* uc = uid + rc;
        float q[PER], o[PER], acc[PER];
        ld_split<PER>(qkv + (size_t)ub[p] * ld + lane * PER, lo_off, q);
#pragma unroll
        for (int t = 0; t < PER; t += 4) {
            const float4 x = *reinterpret_cast<const float4*>(O + (size_t)(rb + p) * d + lane * PER + t);
            o[t] = x.x; o[t + 1] = x.y; o[t + 2] = x.z; o[t + 3] = x.w;
            acc[t] = acc[t + 1] = acc[t + 2] = acc[t + 3] = 0.f;
        }
        const float2 ml = bstat[((size_t)b * ch.N + p) * H + h];  // (maximum scaled score, sum)
        float sum_s = 0.f, sum_c = 0.f;
        const int nd = min(dcnt[c], INC_MAX_KEYS);
        const short* dp = dpos + (size_t)c * INC_MAX_KEYS;
        // 32 changed positions at a time: lane k holds the k-th one and its two row ids, so
        // the key loop below issues its key and value loads without dependent index loads
        for (int k0 = 0; k0 < nd; k0 += 32) {
            int kp_l = 0x7fffffff, ub_l = 0, uc_l = 0;
            if (k0 + lane < nd) {
                kp_l = dp[k0 + lane];
                ub_l = ub[kp_l];
                uc_l = uc[kp_l];
            }
            const int nk = __popc(__ballot_sync(0xffffffffu, kp_l < p));  // ascending: these lie before the row
            for (int k = 0; k < nk; ++k) {
                const int ukb = __shfl_sync(0xffffffffu, ub_l, k), ukc = __shfl_sync(0xffffffffu, uc_l, k);
                float ks[PER], kc[PER], vs[PER], vc[PER];
                ld_split<PER>(qkv + (size_t)ukb * ld + d + lane * PER, lo_off, ks);
                ld_split<PER>(qkv + (size_t)ukc * ld + d + lane * PER, lo_off, kc);
                ld_split<PER>(qkv + (size_t)ukb * ld + 2 * d + lane * PER, lo_off, vs);
                ld_split<PER>(qkv + (size_t)ukc * ld + 2 * d + lane * PER, lo_off, vc);
                float ss = 0.f, scv = 0.f;
#pragma unroll
                for (int t = 0; t < PER; ++t) {
                    ss = fmaf(q[t], ks[t], ss);
                    scv = fmaf(q[t], kc[t], scv);
                }
#pragma unroll
                for (int w = LPH / 2; w > 0; w >>= 1) {
                    ss += __shfl_xor_sync(0xffffffffu, ss, w);
                    scv += __shfl_xor_sync(0xffffffffu, scv, w);
                }
                const float es = __expf(ss * rs - ml.x), ec = __expf(scv * rs - ml.x);
#pragma unroll
                for (int t = 0; t < PER; ++t) acc[t] = fmaf(ec, vc[t] - o[t], fmaf(-es, vs[t] - o[t], acc[t]));
                sum_s += es;
                sum_c += ec;
            }
            if (nk < 32) break;  // the next block lies after the row
        }
        const float inv = 1.f / (ml.y - sum_s + sum_c);
#pragma unroll
        for (int t = 0; t < PER; t += 4)
            *reinterpret_cast<float4*>(O + (size_t)r * d + lane * PER + t) =
                make_float4(fmaf(acc[t], inv, o[t]), fmaf(acc[t + 1], inv, o[t + 1]), fmaf(acc[t + 2], inv, o[t + 2]),
                            fmaf(acc[t + 3], inv, o[t + 3]));
    }
}

cudaError_t launch_inc_exact_delta(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, size_t lo_off, float* O,
                                   const float2* bstat, const short* dpos, const int* dcnt, const int2* list,
                                   const int* n_list_dev, cudaStream_t st, int grid) {
    if (ch.d / ch.heads != 32) return cudaErrorInvalidValue;
    if (ch.d == 256)
        k_inc_exact_delta<8><<<grid, 256, 0, st>>>(ch, uid, qkv, lo_off, O, bstat, dpos, dcnt, list, n_list_dev);
    else if (ch.d == 128)
        k_inc_exact_delta<4><<<grid, 256, 0, st>>>(ch, uid, qkv, lo_off, O, bstat, dpos, dcnt, list, n_list_dev);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---- connected configurations: correction of the unchanged-query rows ----------------
// One CTA per connected configuration (grid-stride), one warp per row over all
// heads: lane l holds dims [l*PER, (l+1)*PER) (PER = d / 32), so a head spans
// LPH = dh / PER consecutive lanes and its scores are reduced over them.
// The changed positions' keys and values (s's and the configuration's) are
// staged in shared memory in blocks of KB keys; a configuration with more
// changed positions than one block processes one row per warp per round.
template <typename T, int PER>
struct PatchRow {
    float q[PER], ob[PER], acc[PER];
    float m, l, seb, sec;
    bool over;
    int pairs;
};

// NV consecutive elements as floats; p is aligned to NV elements (NV a power of two)
template <int NV>
__device__ __forceinline__ void ld_vec(const float* p, float (&out)[NV]) {
    if constexpr (NV % 4 == 0) {
#pragma unroll
        for (int i = 0; i < NV; i += 4) {
            const float4 v = *reinterpret_cast<const float4*>(p + i);
            out[i] = v.x; out[i + 1] = v.y; out[i + 2] = v.z; out[i + 3] = v.w;
        }
    } else if constexpr (NV == 2) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        out[0] = v.x; out[1] = v.y;
    } else {
        out[0] = *p;
    }
}
template <int NV>
__device__ __forceinline__ void ld_vec(const __nv_bfloat16* p, float (&out)[NV]) {
    if constexpr (NV % 8 == 0) {
#pragma unroll
        for (int i = 0; i < NV; i += 8) {
            const uint4 u = *reinterpret_cast<const uint4*>(p + i);
            const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = __bfloat1622float2(h[k]);
                out[i + 2 * k] = f.x;
                out[i + 2 * k + 1] = f.y;
            }
        }
    } else if constexpr (NV == 4) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
        const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
        out[0] = a.x; out[1] = a.y; out[2] = b.x; out[3] = b.y;
    } else if constexpr (NV == 2) {
        const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
        out[0] = a.x; out[1] = a.y;
    } else {
        out[0] = __bfloat162float(*p);
    }
}
template <int NV>
__device__ __forceinline__ void st_vec(float* p, const float (&v)[NV]) {
    if constexpr (NV % 4 == 0) {
#pragma unroll
        for (int i = 0; i < NV; i += 4)
            *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else if constexpr (NV == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
        *p = v[0];
    }
}

// Staged key rows hold lane l's PER dims [l*PER, (l+1)*PER) lane-interleaved in
// float4 groups (group c of lane l at float4 index c*32 + l), so each 16-byte
// shared load of a warp is one contiguous 512-byte block (no bank conflicts).
template <int PER>
__device__ __forceinline__ int perm_pos(int t) {
    if constexpr (PER >= 4) return ((((t % PER) >> 2) * 32 + t / PER) << 2) + (t & 3);
    else return t;
}
template <int PER>
__device__ __forceinline__ void ld_perm(const float* row, int lane, float (&out)[PER]) {
    if constexpr (PER >= 4) {
#pragma unroll
        for (int c = 0; c < PER / 4; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(row + ((c * 32 + lane) << 2));
            out[4 * c] = v.x; out[4 * c + 1] = v.y; out[4 * c + 2] = v.z; out[4 * c + 3] = v.w;
        }
    } else {
        ld_vec<PER>(row + lane * PER, out);
    }
}

// segmented sum over the LPH lanes of a head (aligned groups of consecutive lanes)
__device__ __forceinline__ float head_sum(float v, int lph) {
    for (int o = lph >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T, int PER>
__global__ void __launch_bounds__(256, PER >= 16 ? 1 : 3)
k_inc_patch(Chunk ch, const int* __restrict__ uid, const T* __restrict__ qkv, float* __restrict__ O,
            const float2* __restrict__ bstat, const CertRow* __restrict__ cert, const float* __restrict__ codebook,
            int* __restrict__ code, int* __restrict__ vq_rows, const int* __restrict__ act_off,
            int2* __restrict__ rc_rows, int* __restrict__ rc_cnt, const int* __restrict__ list_simt,
            const short* __restrict__ dpos, const int* __restrict__ dcnt, int kb_keys, long long* __restrict__ stats) {
    extern __shared__ __align__(16) uint8_t smem_u8[];
    const int d = ch.d, H = ch.heads, NM = ch.N;
    const int dh = d / H, lph = dh / PER;
    float* sKb = reinterpret_cast<float*>(smem_u8);  // [kb_keys][d]: s's keys at the changed positions
    float* sKc = sKb + (size_t)kb_keys * d;          // the configuration's keys there
    float* sVb = sKc + (size_t)kb_keys * d;
    float* sVc = sVb + (size_t)kb_keys * d;
    int* sD = reinterpret_cast<int*>(sVc + (size_t)kb_keys * d);  // [NM] changed positions
    int* sRows = sD + NM;                                         // [NM] positions to patch
    int* sVq = sRows + NM;                                        // [NM] rows for the search
    int* sFull = sVq + NM;                                        // [NM] rows to recompute
    uint8_t* sFlag = reinterpret_cast<uint8_t*>(sFull + NM);      // [NM]
    __shared__ int s_warp[32];
    __shared__ int sNvq, sNfull, sBase[2], s_item;
    __shared__ long long sCnt[4];  // patched rows, certified rows, recomputed rows, patched pairs
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int ld = 3 * d;
    const float sl2 = 1.4426950408889634f * rsqrtf((float)dh);  // log2(e) / sqrt(dh)
    const int head = (lane * PER) / dh;
    if (tid < 4) sCnt[tid] = 0;
    for (int item; (item = next_item(ch.counters, CNT_SCW, CNT_SCL, &s_item)) >= 0;) {
        const int c = list_simt[item];
        const int b = ch.cfg_sample[c];
        const int rc = ch.cfg_row[c], rb = ch.cfg_row[ch.cfg_off[b]];
        const int N = cfg_N(ch, c);
        const int p0 = cfg_first_changed(ch.cfg_i[c], ch.cfg_j[c]);
        const int* uc = uid + rc;
        const int* ub = uid + rb;
        const int nd = dcnt[c];
        for (int p = tid; p < N; p += blockDim.x) sFlag[p] = 0;
        __syncthreads();
        if (nd <= INC_MAX_KEYS)
            for (int i = tid; i < nd; i += blockDim.x) {
                sD[i] = dpos[(size_t)c * INC_MAX_KEYS + i];
                sFlag[sD[i]] = 1;
            }
        __syncthreads();
        const bool over_all = nd > INC_MAX_KEYS;  // too many changed positions: recompute every row
        const int np = over_all ? 0 : block_compact(p0, N, [&](int p) { return sFlag[p] == 0; }, sRows, NM, s_warp);
        // rows to recompute: the changed positions (all rows when over_all)
        for (int i = tid; i < (over_all ? N - p0 : nd); i += blockDim.x) {
            const int p = over_all ? p0 + i : sD[i];
            sVq[i] = rc + p;
            sFull[i] = rc + p;
        }
        if (tid == 0) {
            sNvq = over_all ? N - p0 : nd;
            sNfull = sNvq;
            sCnt[2] += sNvq;
        }
        __syncthreads();
        auto stage = [&](int k0, int nk) {  // converted to FP32 once per configuration
            for (int e = tid; e < nk * (d / 4); e += blockDim.x) {
                const int kk = e / (d / 4), t = (e - kk * (d / 4)) * 4;
                const int k = sD[k0 + kk];
                const T* xb = qkv + (size_t)ub[k] * ld;
                const T* xc = qkv + (size_t)uc[k] * ld;
                const int pos = (int)((size_t)kk * d) + perm_pos<PER>(t);  // 4 dims t..t+3 stay together
                float f[4];
                ld_vec<4>(xb + d + t, f);
                *reinterpret_cast<float4*>(sKb + pos) = make_float4(f[0], f[1], f[2], f[3]);
                ld_vec<4>(xc + d + t, f);
                *reinterpret_cast<float4*>(sKc + pos) = make_float4(f[0], f[1], f[2], f[3]);
                ld_vec<4>(xb + 2 * d + t, f);
                *reinterpret_cast<float4*>(sVb + pos) = make_float4(f[0], f[1], f[2], f[3]);
                ld_vec<4>(xc + 2 * d + t, f);
                *reinterpret_cast<float4*>(sVc + pos) = make_float4(f[0], f[1], f[2], f[3]);
            }
        };
        auto row_init = [&](PatchRow<T, PER>& R, int p) {
            ld_vec<PER>(qkv + (size_t)uc[p] * ld + lane * PER, R.q);
            ld_vec<PER>(O + (size_t)(rb + p) * d + lane * PER, R.ob);
            const float2 ml = bstat[((size_t)b * NM + p) * H + head];
            R.m = ml.x * 1.4426950408889634f;  // log2 units
            R.l = ml.y;
#pragma unroll
            for (int i = 0; i < PER; ++i) R.acc[i] = 0.f;
            R.seb = R.sec = 0.f;
            R.over = false;
            R.pairs = 0;
        };
        // keys k0 .. k0+nk-1 of the staged block, all before position p (the caller counts them)
        auto row_keys = [&](PatchRow<T, PER>& R, int nk) {
            for (int kk = 0; kk < nk; ++kk) {
                float kb[PER], kc[PER];
                ld_perm<PER>(sKb + (size_t)kk * d, lane, kb);
                ld_perm<PER>(sKc + (size_t)kk * d, lane, kc);
                float db0 = 0.f, db1 = 0.f, dc0 = 0.f, dc1 = 0.f;  // two partial sums each: shorter chains
#pragma unroll
                for (int i = 0; i < PER; i += 2) {
                    db0 = fmaf(R.q[i], kb[i], db0);
                    dc0 = fmaf(R.q[i], kc[i], dc0);
                    if (i + 1 < PER) {
                        db1 = fmaf(R.q[i + 1], kb[i + 1], db1);
                        dc1 = fmaf(R.q[i + 1], kc[i + 1], dc1);
                    }
                }
                const float db = head_sum(db0 + db1, lph);
                const float dc = head_sum(dc0 + dc1, lph);
                const float xb = db * sl2 - R.m, xc = dc * sl2 - R.m;  // log2 units
                if (xc > 115.f) R.over = true;                         // e^80
                const float eb = ex2_approx(xb), ec = ex2_approx(fminf(xc, 115.f));
                R.seb += eb;
                R.sec += ec;
                float vb[PER], vc[PER];
                ld_perm<PER>(sVb + (size_t)kk * d, lane, vb);
                ld_perm<PER>(sVc + (size_t)kk * d, lane, vc);
#pragma unroll
                for (int i = 0; i < PER; ++i) R.acc[i] = fmaf(ec, vc[i], fmaf(-eb, vb[i], R.acc[i]));
            }
            R.pairs += nk;
        };
        auto row_finish = [&](PatchRow<T, PER>& R, int p) {
            const bool guard = R.over || !(R.seb <= 0.5f * R.l);
            int md;
            if (__any_sync(0xffffffffu, guard)) {
                md = 2;
            } else {
                const float inv = 1.f / (R.l - R.seb + R.sec), w = R.sec - R.seb;
                float n2 = 0.f;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    R.acc[i] = (R.acc[i] - w * R.ob[i]) * inv;  // delta
                    n2 = fmaf(R.acc[i], R.acc[i], n2);
                }
                const float dn = sqrtf(warp_sum(n2)) * (1.f + 1e-5f);
                const CertRow* cr = cert + ((size_t)b * NM + p);
                md = 0;
                if (!(dn < cr->next)) {
                    md = 1;
                } else {
                    const int n = cr->n;
                    if (n > 0 && cr->rho[0] <= dn) {  // exact check of the listed candidates
                        float wc[PER];
                        ld_vec<PER>(codebook + (size_t)cr->code * d + lane * PER, wc);
                        float dwc = 0.f;  // delta . W_c
#pragma unroll
                        for (int t = 0; t < PER; ++t) dwc = fmaf(R.acc[t], wc[t], dwc);
                        for (int i = 0; i < n && cr->rho[i] <= dn; ++i) {
                            float wj[PER];
                            ld_vec<PER>(codebook + (size_t)cr->j[i] * d + lane * PER, wj);
                            float s = -dwc;
#pragma unroll
                            for (int t = 0; t < PER; ++t) s = fmaf(R.acc[t], wj[t], s);
                            s = warp_sum(s);
                            if (!(cr->gap[i] - 2.f * s > cr->eta)) { md = 1; break; }
                        }
                    }
                }
                if (md == 0 && lane == 0) code[rc + p] = cr->code;
                if (md == 1) {  // searched with the corrected output o + delta
                    float o2[PER];
#pragma unroll
                    for (int t = 0; t < PER; ++t) o2[t] = R.ob[t] + R.acc[t];
                    st_vec<PER>(O + (size_t)(rc + p) * d + lane * PER, o2);
                }
            }
            if (lane == 0) {
                if (md >= 1) sVq[atomicAdd(&sNvq, 1)] = rc + p;
                if (md == 2) sFull[atomicAdd(&sNfull, 1)] = rc + p;
                if (md == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[1]), 1ull);
                if (md <= 1) atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[0]), 1ull);
                if (md == 2) atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[2]), 1ull);
                atomicAdd(reinterpret_cast<unsigned long long*>(&sCnt[3]), (unsigned long long)R.pairs);
            }
        };
        if (nd <= kb_keys) {
            stage(0, nd);
            __syncthreads();
            int kc = 0;  // changed keys before the warp's current row (rows ascend)
            for (int i = warp; i < np; i += nw) {
                const int p = sRows[i];
                while (kc < nd && sD[kc] < p) ++kc;
                PatchRow<T, PER> R;
                row_init(R, p);
                row_keys(R, kc);
                row_finish(R, p);
            }
        } else {
            for (int i0 = 0; i0 < np; i0 += nw) {
                const int i = i0 + warp;
                const int p = i < np ? sRows[i] : N;  // a warp without a row only stages
                PatchRow<T, PER> R;
                if (i < np) row_init(R, p);
                for (int k0 = 0; k0 < nd; k0 += kb_keys) {
                    const int nk = min(kb_keys, nd - k0);
                    __syncthreads();
                    stage(k0, nk);
                    __syncthreads();
                    int kc = 0;
                    while (kc < nk && sD[k0 + kc] < p) ++kc;
                    if (i < np) row_keys(R, kc);
                }
                if (i < np) row_finish(R, p);
            }
        }
        __syncthreads();
        if (tid == 0) {  // one atomic per list
            sBase[0] = sNvq ? atomicAdd(&ch.counters[CNT_V], sNvq) : 0;
            // rows of a configuration with more changed positions than its list holds go
            // to the tail of the sample's region: the CUDA-core recompute takes those
            // (it finds the changes by comparing row ids), the tensor-core one the head
            if (!sNfull) {
                sBase[1] = 0;
            } else if (over_all) {
                const int c1 = ch.cfg_off[b + 1];
                const int end = c1 < ch.counters[CNT_C] ? act_off[c1] : ch.counters[CNT_A];
                sBase[1] = end - atomicAdd(&rc_cnt[ch.S + b], sNfull) - sNfull;
            } else {
                sBase[1] = act_off[ch.cfg_off[b]] + atomicAdd(&rc_cnt[b], sNfull);
            }
        }
        __syncthreads();
        for (int i = tid; i < sNvq; i += blockDim.x) vq_rows[sBase[0] + i] = sVq[i];
        for (int i = tid; i < sNfull; i += blockDim.x) rc_rows[sBase[1] + i] = make_int2(sFull[i], sFull[i] - rc);
        __syncthreads();
    }
    if (tid == 0) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_PATCHED]), (unsigned long long)sCnt[0]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_CERT]), (unsigned long long)sCnt[1]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_FULL]), (unsigned long long)sCnt[2]);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_PPAIRS]), (unsigned long long)sCnt[3]);
    }
}

// ---- connected configurations: rows recomputed over all keys ------------------------
// A sample's recompute list holds (row, position) pairs at the head of its
// region of active rows (rc_cnt[b] of them) and, at the tail (rc_cnt[S + b]),
// the rows of configurations with more changed positions than their lists
// hold; tail_only leaves the head to k_attention_rows_tc.
// One CTA per (sample, head, slice).  s's keys and values for the head (and s's
// row ids) stay in shared memory; each warp takes one listed (configuration,
// row) at a time.  Scores: one key per lane; a key whose row id differs from
// s's is read from the configuration's row in global memory.  Weighted sum:
// lane = (key group, 4 dims) over s's values, plus a correction for the
// changed keys (their value minus s's, weighted).
template <typename T, int DH>
__global__ void __launch_bounds__(256)
k_inc_attention(Chunk ch, const int* __restrict__ uid, const T* __restrict__ qkv, float* __restrict__ O,
                const int* __restrict__ act_off, const int2* __restrict__ rc_rows, const int* __restrict__ rc_cnt,
                int slices, int tail_only, long long* __restrict__ stats) {
    extern __shared__ __align__(16) float smem_f[];
    constexpr int KS = DH + 4;    // key row stride: 16-byte rows, 8 consecutive keys on distinct banks
    constexpr int G = 32 / (DH / 4);  // key groups in the weighted sum (lanes per group: DH / 4)
    const int d = ch.d, H = ch.heads, NM = ch.N;
    float* sK = smem_f;                              // [NM][KS]
    float* sV = sK + (size_t)NM * KS;                // [NM][DH]
    int* sUb = reinterpret_cast<int*>(sV + (size_t)NM * DH);  // [NM] s's row ids
    float* sP = reinterpret_cast<float*>(sUb + NM);  // [8 warps][NM] scores, then weights
    int* sL = reinterpret_cast<int*>(sP + 8 * NM);   // [8 warps][NM] changed keys of the row
    __shared__ long long sPairs;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ld = 3 * d;
    const float sl2 = 1.4426950408889634f * rsqrtf((float)DH);  // log2(e) / sqrt(dh)
    if (tid == 0) sPairs = 0;
    if (blockIdx.x == 0 && tid == 0)
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_VQ]), (unsigned long long)ch.counters[CNT_V]);
    const int items = ch.S * H * slices;
    const int g = lane / (DH / 4), c4 = (lane % (DH / 4)) * 4;  // key group, first of 4 dims
    long long pairs = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int z = item % slices, bh = item / slices;
        const int b = bh / H, h = bh - b * H;
        const int nh = tail_only ? 0 : rc_cnt[b], nt = rc_cnt[ch.S + b];
        const int n = nh + nt;
        if (z * 8 >= n) continue;  // block-uniform: nothing for this slice
        const int rb = ch.cfg_row[ch.cfg_off[b]];
        const int N = sample_N(ch, b);
        const int2* head = rc_rows + act_off[ch.cfg_off[b]];  // (row, position) pairs
        const int c1 = ch.cfg_off[b + 1];
        const int2* tail = rc_rows + (c1 < ch.counters[CNT_C] ? act_off[c1] : ch.counters[CNT_A]) - nt;
        auto entry = [&](int i) { return i < nh ? head[i] : tail[i - nh]; };
        __syncthreads();  // the previous item's readers are done
        for (int e = tid; e < N * (DH / 4); e += blockDim.x) {
            const int j = e / (DH / 4), t = (e - j * (DH / 4)) * 4;
            const T* x = qkv + (size_t)uid[rb + j] * ld + h * DH + t;
            float kx[4], vx[4];
            ld_vec<4>(x + d, kx);
            ld_vec<4>(x + 2 * d, vx);
            *reinterpret_cast<float4*>(sK + j * KS + t) = make_float4(kx[0], kx[1], kx[2], kx[3]);
            *reinterpret_cast<float4*>(sV + j * DH + t) = make_float4(vx[0], vx[1], vx[2], vx[3]);
        }
        for (int j = tid; j < N; j += blockDim.x) sUb[j] = uid[rb + j];
        __syncthreads();
        float* P = sP + warp * NM;
        int* Lw = sL + warp * NM;
        const int stride = slices * 8;
        int i = z * 8 + warp;
        int2 it = i < n ? entry(i) : make_int2(0, 0);
        int uq = i < n ? uid[it.x] : 0;
        for (; i < n; i += stride) {
            const int row = it.x, p = it.y;
            const int* uc = uid + (row - p);
            float q[DH];
            ld_vec<DH>(qkv + (size_t)uq * ld + h * DH, q);
            if (i + stride < n) {  // the next item's descriptor and query row, in flight meanwhile
                it = entry(i + stride);
                uq = uid[it.x];
            }
            int* Uw = reinterpret_cast<int*>(P);  // the configuration's row ids 0..p (all loads in flight at once)
            for (int j = lane; j <= p; j += 32) Uw[j] = uc[j];
            __syncwarp();
            float mx = -INFINITY;
            int nl = 0;  // changed keys listed so far (warp-uniform)
            for (int j0 = 0; j0 <= p; j0 += 32) {
                const int j = j0 + lane;
                float s = -INFINITY;
                bool changed = false;
                if (j <= p) {
                    const int u = Uw[j];
                    changed = u != sUb[j];
                    float kx[DH];
                    if (changed) ld_vec<DH>(qkv + (size_t)u * ld + d + h * DH, kx);
                    else ld_vec<DH>(sK + j * KS, kx);
                    float a = 0.f;
#pragma unroll
                    for (int t = 0; t < DH; ++t) a = fmaf(q[t], kx[t], a);
                    s = a * sl2;  // log2 units
                    P[j] = s;
                }
                const unsigned m = __ballot_sync(0xffffffffu, changed);
                if (changed) Lw[nl + __popc(m & ((1u << lane) - 1))] = j;
                nl += __popc(m);
                mx = fmaxf(mx, s);
            }
            for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            float l = 0.f;
            for (int j = lane; j <= p; j += 32) {
                const float e = ex2_approx(P[j] - mx);
                P[j] = e;
                l += e;
            }
            l = warp_sum(l);
            __syncwarp();
            // weighted sum over s's values (lane: key group g, dims c4..c4+3)
            float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
            for (int j = g; j <= p; j += G) {
                const float w = P[j];
                const float4 v = *reinterpret_cast<const float4*>(sV + j * DH + c4);
                a0 = fmaf(w, v.x, a0); a1 = fmaf(w, v.y, a1); a2 = fmaf(w, v.z, a2); a3 = fmaf(w, v.w, a3);
            }
            // the changed keys: their value minus s's
            for (int t = g; t < nl; t += G) {
                const int j = Lw[t];
                const float w = P[j];
                float vx[4];
                ld_vec<4>(qkv + (size_t)uc[j] * ld + 2 * d + h * DH + c4, vx);
                const float4 v = *reinterpret_cast<const float4*>(sV + j * DH + c4);
                a0 = fmaf(w, vx[0] - v.x, a0); a1 = fmaf(w, vx[1] - v.y, a1);
                a2 = fmaf(w, vx[2] - v.z, a2); a3 = fmaf(w, vx[3] - v.w, a3);
            }
            for (int o = DH / 4; o < 32; o <<= 1) {  // sum the key groups
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
                a3 += __shfl_xor_sync(0xffffffffu, a3, o);
            }
            if (g == 0) {
                const float inv = 1.f / l;
                *reinterpret_cast<float4*>(O + (size_t)row * d + h * DH + c4) =
                    make_float4(a0 * inv, a1 * inv, a2 * inv, a3 * inv);
            }
            if (h == 0) pairs += p + 1;  // counted once per row (the FLOP count covers all heads)
            __syncwarp();
        }
    }
    if (lane == 0 && pairs) atomicAdd(reinterpret_cast<unsigned long long*>(&sPairs), (unsigned long long)pairs);
    __syncthreads();
    if (tid == 0 && sPairs) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_FPAIRS]), (unsigned long long)sPairs);
}

// ---- ||W_c - W_j|| table -------------------------------------------------------------
__global__ void k_codeword_dist(const float* __restrict__ W, int K, int d, float* __restrict__ wd) {
    const int lane = threadIdx.x & 31;
    for (int pr = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); pr < K * K; pr += gridDim.x * (blockDim.x >> 5)) {
        const int a = pr / K, c = pr - a * K;
        float s = 0.f;
        for (int t = lane; t < d; t += 32) {
            const float x = W[(size_t)a * d + t] - W[(size_t)c * d + t];
            s = fmaf(x, x, s);
        }
        s = warp_sum(s);
        if (lane == 0) wd[pr] = sqrtf(s);
    }
}

// ---- launchers ------------------------------------------------------------------------

bool incremental_supported(int d, int heads) {
    const int dh = d / heads, per = d / 32;
    return (dh == 16 || dh == 32) && d % 32 == 0 && (per == 1 || per == 2 || per == 4 || per == 8 || per == 16) &&
           dh % per == 0;
}

constexpr int CERT_RB = 16;  // sample rows per CTA (240 CTAs for 15 samples of 256 sites)
size_t base_cert_smem(int d, int K) {
    return ((size_t)CERT_RB * d + 32 * 256 + CERT_RB * (size_t)K + 8 * (size_t)K) * 4;
}

cudaError_t launch_base_cert(const Chunk& ch, const float* O, const float* codebook, const float* cnorm,
                             const float* wd, int K, int d, int* code, CertRow* cert, long long* stats,
                             int* counters, int* rc_cnt, cudaStream_t st) {
    const size_t smem = base_cert_smem(d, K);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    static size_t granted = 0;
    if (smem > granted) {
        cudaFuncSetAttribute(k_base_cert<CERT_RB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        granted = smem;
    }
    const int blocks = (ch.S * ch.N + CERT_RB - 1) / CERT_RB;
    k_base_cert<CERT_RB><<<blocks, 256, smem, st>>>(ch, O, codebook, cnorm, wd, K, d, code, cert, stats + ST_NEAR_TIES,
                                           counters, rc_cnt, stats);
    return cudaGetLastError();
}

cudaError_t launch_base_cert_tc(const Chunk& ch, const float* O, const CUtensorMap& tm_hi, const CUtensorMap& tm_lo,
                                const float* cnorm, const float* wd, int K, int d, int* code, CertRow* cert,
                                long long* stats, int* counters, int* rc_cnt, int* list, float* dist, float* osq,
                                int* status, cudaStream_t st, int num_sms) {
    const int total = ch.S * ch.N;
    const size_t smem = (size_t)8 * 2 * K * sizeof(float);
    if (K % 16 || smem > 227 * 1024) return cudaErrorInvalidValue;
    static size_t granted = 0;
    if (smem > granted && smem > 48 * 1024) {
        cudaFuncSetAttribute(k_base_cert_dist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        granted = smem;
    }
    int g = (total + 255) / 256;
    if (g > 4 * num_sms) g = 4 * num_sms;
    k_base_rows<<<g < 1 ? 1 : g, 256, 0, st>>>(ch, list);
    cudaError_t e = launch_vq_tc(tm_hi, tm_lo, O, list, list + 1, cnorm, K, d, code, nullptr, status, st, num_sms,
                                 total, 0, dist, osq);
    if (e != cudaSuccess) return e;
    int blocks = (total + 7) / 8;
    if (blocks > 8 * num_sms) blocks = 8 * num_sms;
    k_base_cert_dist<<<blocks < 1 ? 1 : blocks, 256, smem, st>>>(ch, dist, osq, cnorm, wd, K, code, cert,
                                                                 stats + ST_NEAR_TIES, counters, rc_cnt, stats);
    return cudaGetLastError();
}

cudaError_t launch_base_cert_heads(const Chunk& ch, const float* O, const float* codebook, const float* cnorm,
                                   const float* wd, int K, int d, int H, int bits, int* code, CertRow* cert,
                                   long long* stats, int* counters, int* rc_cnt, cudaStream_t st, int num_sms) {
    const size_t smem = (size_t)8 * (d + K) * sizeof(float);
    if (H < 2 || d % H || H * bits > 32 || smem > 227 * 1024) return cudaErrorInvalidValue;
    static size_t granted = 0;
    if (smem > granted) {
        cudaFuncSetAttribute(k_base_cert_heads, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        granted = smem;
    }
    const int rows = ch.S * ch.N;
    int blocks = (rows + 7) / 8;
    if (blocks > 4 * num_sms) blocks = 4 * num_sms;
    k_base_cert_heads<<<blocks, 256, smem, st>>>(ch, O, codebook, cnorm, wd, K, d, H, bits, code, cert,
                                                 stats + ST_NEAR_TIES, counters, rc_cnt, stats);
    return cudaGetLastError();
}

// changed keys staged per block: about 64 KB of FP32 keys and values (three CTAs per SM)
int inc_patch_keys(int d) {
    int kb = 4096 / d;
    return kb < 1 ? 1 : (kb > INC_MAX_KEYS ? INC_MAX_KEYS : kb);
}
size_t inc_patch_smem(int d, int N) {
    return (size_t)4 * inc_patch_keys(d) * d * 4 + (size_t)4 * N * 4 + (size_t)((N + 15) & ~15);
}

template <typename T>
cudaError_t launch_inc_patch_t(const Chunk& ch, const int* uid, const T* qkv, float* O, const float2* bstat,
                               const CertRow* cert, const float* codebook, const float* wd, int* code, int* vq_rows,
                               const int* act_off, int2* rc_rows, int* rc_cnt, const int* list_tc,
                               const int* list_simt, const short* dpos, const int* dcnt, int use_tc, int split,
                               int2* ex_rows, int* status, long long* stats, cudaStream_t st, int grid,
                               int items_per_cta) {
    if (!incremental_supported(ch.d, ch.heads)) return cudaErrorInvalidValue;
    const int kb = inc_patch_keys(ch.d);
    const size_t smem = inc_patch_smem(ch.d, ch.N);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
#define VQ_PATCH(P)                                                                                          \
    {                                                                                                        \
        static size_t granted = 0;                                                                           \
        if (smem > granted) {                                                                                \
            cudaFuncSetAttribute(k_inc_patch<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            granted = smem;                                                                                  \
        }                                                                                                    \
        k_inc_patch<T, P><<<grid, 256, smem, st>>>(ch, uid, qkv, O, bstat, cert, codebook, code, vq_rows,      \
                                                   act_off, rc_rows, rc_cnt, list_simt, dpos, dcnt, kb, stats);            \
    }
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        if (use_tc) {  // the classify kernel left no configuration to the CUDA cores
            const int d = ch.d;
            // a sample has at most 2N + 1 configurations: one item's walk list holds them all
            if (2 * ch.N + 1 > RES_MAX_CFG) return cudaErrorInvalidValue;
            const uint32_t cols = 2 * d <= 256 ? 256 : 512;  // scores/sums and the sample's outputs
            if (2 * d > 512) return cudaErrorInvalidValue;
            const size_t smem = res_layout(d, ch.heads).total;
            if (smem > 227 * 1024) return cudaErrorInvalidValue;
            // the TMEM columns of the CTAs resident on one SM must fit in its 512
            const int per_sm = (int)(512 / cols);
            size_t smem_req = smem;
            if ((size_t)(228 * 1024) / smem_req > (size_t)per_sm) smem_req = (228 * 1024) / (per_sm + 1) + 1024;
            static size_t granted_res = 0;
            if (smem_req > granted_res) {
                cudaFuncSetAttribute(k_inc_patch_res, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_req);
                granted_res = smem_req;
            }
            int dev = 0, sms = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return cudaErrorInvalidDevice;
            const int g = (sms > 0 ? sms : 1) * per_sm;
            // items (sample, tile, slice): about items_per_cta per CTA
            const int ntile = (ch.N + 127) / 128;
            const int sb = ch.S * ntile;
            const int ipc = items_per_cta < 1 ? 1 : items_per_cta;
            int slices = (ipc * g + sb - 1) / sb;
            slices = slices < 1 ? 1 : (slices > 64 ? 64 : slices);
            k_inc_patch_res<<<g, RES_THREADS, smem_req, st>>>(ch, uid, qkv, O, bstat, cert, codebook, wd, code, vq_rows,
                                                      act_off, rc_rows, rc_cnt, dpos, dcnt, split, ex_rows, slices,
                                                      cols, status, stats);
            return cudaGetLastError();
        }
    }
    switch (ch.d / 32) {
        case 1: VQ_PATCH(1) break;
        case 2: VQ_PATCH(2) break;
        case 4: VQ_PATCH(4) break;
        case 8: VQ_PATCH(8) break;
        case 16: VQ_PATCH(16) break;
        default: return cudaErrorInvalidValue;
    }
#undef VQ_PATCH
    return cudaGetLastError();
}

size_t inc_attention_smem(int N, int dh) {
    return ((size_t)N * (dh + 4) + (size_t)N * dh + (size_t)N + 8 * (size_t)N + 8 * (size_t)N) * 4;
}

template <typename T>
cudaError_t launch_inc_attention_t(const Chunk& ch, const int* uid, const T* qkv, float* O, const int* act_off,
                                   const int2* rc_rows, const int* rc_cnt, int tail_only, long long* stats,
                                   cudaStream_t st, int num_sms) {
    const int dh = ch.d / ch.heads;
    const size_t smem = inc_attention_smem(ch.N, dh);
    if (smem > 227 * 1024 || !incremental_supported(ch.d, ch.heads)) return cudaErrorInvalidValue;
    // enough (sample, head, slice) items for about two CTAs per SM
    const int sh = ch.S * ch.heads;
    int slices = (2 * num_sms + sh - 1) / sh;
    if (slices < 1) slices = 1;
    if (slices > 64) slices = 64;
    const int grid = sh * slices;
#define VQ_IATT(D)                                                                                               \
    {                                                                                                            \
        static size_t granted = 0;                                                                               \
        if (smem > granted) {                                                                                    \
            cudaFuncSetAttribute(k_inc_attention<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            granted = smem;                                                                                      \
        }                                                                                                        \
        k_inc_attention<T, D><<<grid, 256, smem, st>>>(ch, uid, qkv, O, act_off, rc_rows, rc_cnt, slices,       \
                                                       tail_only, stats);                                     \
    }
    if (dh == 32) VQ_IATT(32) else VQ_IATT(16)
#undef VQ_IATT
    return cudaGetLastError();
}

cudaError_t launch_inc_patch(const Chunk& ch, const int* uid, const float* qkv, float* O, const float2* bstat,
                             const CertRow* cert, const float* codebook, const float* wd, int* code, int* vq_rows,
                             const int* act_off, int2* rc_rows, int* rc_cnt, const int* list_tc,
                             const int* list_simt, const short* dpos, const int* dcnt, int use_tc, int* status,
                             long long* stats, cudaStream_t st, int grid) {
    return launch_inc_patch_t<float>(ch, uid, qkv, O, bstat, cert, codebook, wd, code, vq_rows, act_off, rc_rows,
                                     rc_cnt, list_tc, list_simt, dpos, dcnt, use_tc, 0, nullptr, status, stats, st,
                                     grid, 4);
}
cudaError_t launch_inc_patch(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                             const float2* bstat, const CertRow* cert, const float* codebook, const float* wd,
                             int* code, int* vq_rows, const int* act_off, int2* rc_rows, int* rc_cnt,
                             const int* list_tc, const int* list_simt, const short* dpos, const int* dcnt, int use_tc,
                             int split, int2* ex_rows, int* status, long long* stats, cudaStream_t st, int grid,
                             int items_per_cta) {
    return launch_inc_patch_t<__nv_bfloat16>(ch, uid, qkv, O, bstat, cert, codebook, wd, code, vq_rows, act_off,
                                             rc_rows, rc_cnt, list_tc, list_simt, dpos, dcnt, use_tc, split, ex_rows,
                                             status, stats, st, grid, items_per_cta);
}
cudaError_t launch_inc_attention(const Chunk& ch, const int* uid, const float* qkv, float* O, const int* act_off,
                                 const int2* rc_rows, const int* rc_cnt, int tail_only, long long* stats, cudaStream_t st,
                                 int num_sms) {
    return launch_inc_attention_t<float>(ch, uid, qkv, O, act_off, rc_rows, rc_cnt, tail_only, stats, st, num_sms);
}
cudaError_t launch_inc_attention(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                                 const int* act_off, const int2* rc_rows, const int* rc_cnt, int tail_only, long long* stats,
                                 cudaStream_t st, int num_sms) {
    return launch_inc_attention_t<__nv_bfloat16>(ch, uid, qkv, O, act_off, rc_rows, rc_cnt, tail_only, stats, st, num_sms);
}

cudaError_t launch_inc_classify(const Chunk& ch, const int* uid, int tc_ok, int* list_tc, int* list_simt, short* dpos,
                                int* dcnt, int* vq_rows, long long* stats, cudaStream_t st, int grid) {
    k_inc_classify<<<grid, 256, 0, st>>>(ch, uid, tc_ok, list_tc, list_simt, dpos, dcnt, vq_rows, stats);
    return cudaGetLastError();
}

cudaError_t launch_codeword_dist(const float* W, int K, int d, float* wd, cudaStream_t st) {
    k_codeword_dist<<<256, 256, 0, st>>>(W, K, d, wd);
    return cudaGetLastError();
}

}  // namespace vq
