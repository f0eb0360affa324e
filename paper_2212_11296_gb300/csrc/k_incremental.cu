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
    float* rho = sRho + warp * K;
    int ties = 0;
    for (int r = warp; r < RB; r += 8) {
        const int row = sRow[r];
        if (row < 0) continue;  // warp-uniform
        const float* dist = sDist + r * K;
        // nearest (lowest index on ties) and second nearest distance
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
        const int c = i1;
        const float eta = CERT_ETA_REL * (sOsq[r] + sCnMax);
        if (lane == 0) {
            code[row] = c;
            if (K > 1 && (v2 - v1) < NEAR_TIE_REL * fmaxf(v1, 1e-30f)) ++ties;
        }
        for (int j = lane; j < K; j += 32) {
            const float w = wd[(size_t)c * K + j];
            rho[j] = (j == c || w <= 0.f) ? INFINITY : (dist[j] - v1 - eta) / (2.f * w);
        }
        __syncwarp();
        // the CERT_T + 1 smallest radii, ascending (lowest index first on equal radii)
        CertRow* cr = cert + (r0 + r);
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
    long long full_rows = 0;
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
        }
    }
    if (full_rows) atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_INC_FULL]), (unsigned long long)full_rows);
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
// One CTA of 256 threads takes configurations from the tensor-core list.  Per
// tile of up to 128 patched rows, tile row r is TMEM lane r and belongs to two
// threads, r and r + 128, each of which takes half of the heads:
//   1. the rows' queries (the sample's: a patched row's input is unchanged) are
//      copied into shared memory with cp.async (K-major, d columns), the
//      changed positions' keys beside them and their values transposed;
//   2. per head h: S_h = Q_h [K_s; K_c]_h^T (M = 128, N = 32): the sample's keys
//      at the changed positions in columns 0..15, the configuration's in 16..31;
//   3. per row and head: the BF16 weights e = exp(s / sqrt(dh) - m) of the
//      changed keys before the row (the sample's negated) as the A operand;
//   4. per head: E_h [V_s; V_c]_h (N = 32) into the TMEM columns the scores came
//      from: sum_k e_c v_c - e_s v_s;
//   5. per row: delta = (acc - (sum e_c - sum e_s) o) / l' with the sample's
//      outputs o read by the row's own threads; delta goes back to TMEM, the two
//      threads' partial norms are added, and the certificate is checked as in
//      k_inc_patch with ||delta|| replaced by ||delta|| + B, B a bound on the
//      error of the BF16 computation (below), and each listed candidate's
//      projection by |delta . (W_j - W_c)| + B ||W_j - W_c||;
//   6. only a row that is searched (certificate not met) has o + delta written
//      to O; a certified row keeps the sample's codeword and writes nothing else.
//      With split operands (the path whose Q/K/V carry a BF16 lo plane) a row
//      that the certificate does not settle is listed instead, and
//      k_inc_exact_delta forms its correction from the split operands in FP32,
//      so every output that reaches the search carries FP32-grade error.
//
// The bound B.  The kernel reads only the hi planes: q~ = bf16(q), k~, v~ (each
// within 2^-9 relative of the exact value, or equal to it on the plain BF16
// path), e~ = exp2(s~ sl2 - m) with s~ = q~ . k~ accumulated in FP32, and the
// MMA takes e^ = bf16(e~).  Per head, |s~ - s| <= 2^-8 (1 + 2^-7) ||q~|| ||k~||
// (two relative 2^-9 perturbations plus the 32-term FP32 sum), so
// |e~ / e - 1| <= tau = 2^dx - 1 + 2^-20 with dx = 2^-8 1.01 sl2 ||q~|| ||k~||
// (the 2^-20 covers ex2.approx and the rounding of its argument; 2^dx - 1 is
// bounded by y + y^2, y = dx ln 2, which holds for y <= 1), and
// e^ v~ - e v = (e^ - e) v~ + e (v~ - v) has norm <= e (tau + 2^-8) ||v~||.
// With A = sum_k e~ (tau + 2^-8) ||v~|| and T = sum_k e~ tau over the row's
// changed keys (the sample's and the configuration's), the numerator and the
// weight sum w differ from exact by at most 1.1 (A + T ||o||) and the
// normaliser by at most 1.1 T (e <= 1.1 e~ while tau <= 0.1), so
//   ||delta~_h - delta_h|| <= B_h = 1.1 (A + T (||o_h|| + ||delta~_h||)) / (l~' - 1.1 T)
// per head and B = sqrt(sum_h B_h^2).  A row with tau > 0.1 for some key, or
// l~' - 1.1 T <= l~' / 2, is recomputed over all keys.
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

size_t patch_tc_smem(int d, int heads, int N) {
    return 128 + (size_t)128 * d * 2 + (size_t)heads * 4096 + (size_t)2 * 128 * (2 + CERT_T) * 4 + 64 +
           (size_t)4 * N * 4 + (size_t)((N + 15) & ~15) + (size_t)2 * heads * 32 * 4;
}

// e~ (tau + 2^-8) ||v~|| and e~ tau of one changed key (see the bound B above), with
// 2^dx - 1 = e^y - 1 <= y + y^2 for y = dx ln 2 <= 1; sets guard when tau would exceed 0.1
__device__ __forceinline__ void patch_err_terms(float e, float dx, float vn, float& acc_a, float& acc_t, bool& guard) {
    const float y = dx * 0.69314718f * 1.0001f;
    const float tau = fmaf(y, y, y) + 9.5367431640625e-07f;  // + 2^-20
    if (y > 0.09f) guard = true;
    acc_a = fmaf(e * (tau + 3.90625e-3f), vn, acc_a);
    acc_t = fmaf(e, tau, acc_t);
}

// The BF16 weights of one head for a row with nk changed keys before it (nk <= NKB):
// e_s = exp(s_s / sqrt(dh) - m) negated in slots 0..15, e_c in 16..31, zeros beyond
// nk; seb, sec their sums; guard set when a new score overflows the sample's max.
// Also the error bound's sums over the row's changed keys: aa += e (tau + 2^-8) ||v~||,
// at += e tau (patch_err_terms), with dx = qn ||k~|| per key (qn = 2^-8 1.01 sl2 ||q~||).
template <int NKB>
__device__ __forceinline__ void patch_weights(uint32_t (&s)[32], int nk, float sl2, float m2, bool& guard, float& seb,
                                              float& sec, uint32_t (&e16)[16], float qn, const float* __restrict__ kn,
                                              const float* __restrict__ vn, float& aa, float& at) {
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
        float eb = 0.f, ec = 0.f;
        if (kk < NKB && kk < nk) {
            const float xc = __uint_as_float(s[16 + kk]) * sl2 - m2;
            if (xc > 115.f) guard = true;
            eb = ex2_approx(__uint_as_float(s[kk]) * sl2 - m2);
            ec = ex2_approx(fminf(xc, 115.f));
            patch_err_terms(eb, qn * kn[kk], vn[kk], aa, at, guard);
            patch_err_terms(ec, qn * kn[16 + kk], vn[16 + kk], aa, at, guard);
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

__global__ void __launch_bounds__(256, 2)
k_inc_patch_tc(Chunk ch, const int* __restrict__ uid, const __nv_bfloat16* __restrict__ qkv,
               float* __restrict__ O, const float2* __restrict__ bstat, const CertRow* __restrict__ cert,
               const float* __restrict__ codebook, const float* __restrict__ wd, int* __restrict__ code,
               int* __restrict__ vq_rows, const int* __restrict__ act_off, int2* __restrict__ rc_rows,
               int* __restrict__ rc_cnt, const int* __restrict__ list_tc, const short* __restrict__ dpos,
               const int* __restrict__ dcnt, int split, int2* __restrict__ ex_rows, uint32_t tmem_cols,
               int* __restrict__ status, long long* __restrict__ stats) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    constexpr int DH = 32;
    const int d = ch.d, H = ch.heads, NM = ch.N;  // d == 32 H
    const int HH = H / 2;                         // heads per thread
    uint8_t* sQE = smem;                          // [128 x d] queries, then [128 x d] weights
    uint8_t* sK = sQE + 128 * d * 2;              // per head [32 keys x 32 dims]
    uint8_t* sVt = sK + H * 2048;                 // per head [32 dims x 32 keys]
    // [2 halves][128]: partial ||delta~||^2 and B^2 (B^2 = -1: the thread's heads need a recompute)
    float2* sN2 = reinterpret_cast<float2*>(sVt + H * 2048);
    float* sP = reinterpret_cast<float*>(sN2 + 256);        // [2 halves][128][CERT_T]: partial projections
    uint64_t* bar = reinterpret_cast<uint64_t*>(sP + 256 * CERT_T);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + 1);
    int* sD = reinterpret_cast<int*>(tmem_holder + 4);  // [PATCH_TC_KEYS]
    int* sRows = sD + PATCH_TC_KEYS;                    // [NM]
    int* sVq = sRows + NM;                              // [NM]
    int* sFull = sVq + NM;                              // [NM]
    uint8_t* sFlag = reinterpret_cast<uint8_t*>(sFull + NM);  // [NM]
    float* sKn = reinterpret_cast<float*>(sFlag + ((NM + 15) & ~15));  // [H][32]: ||k~|| of the key slots
    float* sVn = sKn + H * 32;                                         // [H][32]: ||v~||
    __shared__ int s_warp[32];
    __shared__ int sNvq, sNfull, sBase[2], s_item;
    __shared__ long long sCnt[4];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int half = tid >> 7, r = tid & 127;
    const int h0 = half * HH;
    const int ld = 3 * d;
    const float sl2 = 1.4426950408889634f * rsqrtf((float)DH);
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_barrier_init();
    }
    if (tid < 4) sCnt[tid] = 0;
    if (warp == 0) tc::tmem_alloc(tmem_holder, tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;  // warps w and w + 4 share TMEM lanes
    uint32_t phase = 0;
    bool ok = true;
    long long n_patched = 0, n_cert = 0, n_full = 0, n_pairs = 0;
    for (int item; ok && (item = next_item(ch.counters, CNT_TCW, CNT_TCL, &s_item)) >= 0;) {
        const int c = list_tc[item];
        const int b = ch.cfg_sample[c];
        const int rc = ch.cfg_row[c], rb = ch.cfg_row[ch.cfg_off[b]];
        const int N = cfg_N(ch, c);
        const int p0 = cfg_first_changed(ch.cfg_i[c], ch.cfg_j[c]);
        const int* uc = uid + rc;
        const int* ub = uid + rb;
        const int nd = dcnt[c];  // <= PATCH_TC_KEYS
        for (int p = tid; p < N; p += blockDim.x) sFlag[p] = 0;
        __syncthreads();
        if (tid < nd) {
            sD[tid] = dpos[(size_t)c * INC_MAX_KEYS + tid];
            sFlag[sD[tid]] = 1;
        }
        __syncthreads();
        const int np = block_compact(p0, N, [&](int p) { return sFlag[p] == 0; }, sRows, NM, s_warp);
        if (tid < nd) {  // changed positions: recompute, then search
            sVq[tid] = rc + sD[tid];
            sFull[tid] = rc + sD[tid];
        }
        if (tid == 0) { sNvq = nd; sNfull = nd; }
        n_full += tid == 0 ? nd : 0;
        for (int t0 = 0; t0 < np && ok; t0 += 128) {
            const int nrow = min(128, np - t0);
            const int p = r < nrow ? sRows[t0 + r] : -1;
            // keys of the changed positions, zero-filled to 16 + 16 per head
            for (int u = tid; u < H * 32 * (DH / 8); u += blockDim.x) {
                const int h = u / (32 * (DH / 8)), rem = u - h * 32 * (DH / 8);
                const int n = rem & 31, t8 = (rem >> 5) * 8;  // key slot, first of 8 dims
                const int kk = n & 15;
                const __nv_bfloat16* x = qkv;
                if (kk < nd) x = qkv + (size_t)(n < 16 ? ub[sD[kk]] : uc[sD[kk]]) * ld + d + h * DH + t8;
                cp_async16(tc::smem_u32(sK + h * 2048 + tc::core_off(n, t8, DH)), x, kk < nd ? 16 : 0);
            }
            // the row's query: thread (r, half) copies chunks half, half + 2, ...
            {
                const __nv_bfloat16* qrow = p >= 0 ? qkv + (size_t)ub[p] * ld : qkv;
                const int nb = p >= 0 ? 16 : 0;
                for (int k8 = half * 8; k8 < d; k8 += 16)
                    cp_async16(tc::smem_u32(sQE + tc::core_off(r, k8, d)), qrow + k8, nb);
            }
            // values, transposed: dims are the rows of the [dims x keys] operand
            for (int u0 = tid; u0 < H * 32 * (DH / 8); u0 += 4 * blockDim.x) {
                uint4 vv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = u0 + i * blockDim.x;
                    const int h = u / (32 * (DH / 8)), rem = u - h * 32 * (DH / 8);
                    const int n = rem & 31, t8 = (rem >> 5) * 8, kk = n & 15;
                    vv[i] = make_uint4(0, 0, 0, 0);
                    if (u < H * 32 * (DH / 8) && kk < nd)
                        vv[i] = *reinterpret_cast<const uint4*>(
                            qkv + (size_t)(n < 16 ? ub[sD[kk]] : uc[sD[kk]]) * ld + 2 * d + h * DH + t8);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int u = u0 + i * blockDim.x;
                    if (u >= H * 32 * (DH / 8)) break;
                    const int h = u / (32 * (DH / 8)), rem = u - h * 32 * (DH / 8);
                    const int n = rem & 31, t8 = (rem >> 5) * 8;
                    const __nv_bfloat16* ve = reinterpret_cast<const __nv_bfloat16*>(&vv[i]);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        *reinterpret_cast<__nv_bfloat16*>(sVt + h * 2048 + tc::core_off(t8 + e, n, 32)) = ve[e];
                }
            }
            cp_async_wait_all();
            tc::fence_proxy_async_smem();
            tc::tc_fence_before();
            __syncthreads();
            // norms of the staged key and value slots (zero-filled slots give 0); read after the
            // next block-wide barrier
            for (int u = tid; u < H * 32; u += blockDim.x) {
                const int h = u >> 5, n = u & 31;
                float kk2 = 0.f, vv2 = 0.f;
#pragma unroll
                for (int t = 0; t < DH; ++t) {
                    const float kx = __bfloat162float(
                        *reinterpret_cast<const __nv_bfloat16*>(sK + h * 2048 + tc::core_off(n, t, DH)));
                    const float vx = __bfloat162float(
                        *reinterpret_cast<const __nv_bfloat16*>(sVt + h * 2048 + tc::core_off(t, n, 32)));
                    kk2 = fmaf(kx, kx, kk2);
                    vv2 = fmaf(vx, vx, vv2);
                }
                sKn[u] = sqrtf(kk2);
                sVn[u] = sqrtf(vv2);
            }
            if (tid == 0) {
                tc::tc_fence_after();
                const uint64_t dq = tc::desc_kmajor_none(tc::smem_u32(sQE), 128, (d / 8) * 128);
                for (int h = 0; h < H; ++h) {
                    const uint64_t dk = tc::desc_kmajor_none(tc::smem_u32(sK + h * 2048), 128, (DH / 8) * 128);
#pragma unroll
                    for (int ks = 0; ks < DH / 16; ++ks)
                        tc::mma_bf16(tmem + h * 32, dq + (uint64_t)(h * DH + ks * 16), dk + (uint64_t)(ks * 16),
                                     tc::idesc_bf16_f32(128, 32), ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            ok = __syncthreads_and(tc::mbar_wait(bar, phase, status)) != 0;
            phase ^= 1;
            tc::tc_fence_after();
            if (!ok) break;
            float w[4], inv[4];  // per own head: sum e_c - sum e_s, 1 / l'
            float ea[4], et[4];  // per own head: the bound's sums A and T, times 1.1 / (l~' - 1.1 T)
            bool guard = false;
            int nk = 0;  // changed keys before this row
            while (p >= 0 && nk < nd && sD[nk] < p) ++nk;
            // warps w and w + 4 hold the same rows: both skip a tile's padding rows together
            const bool wact = __any_sync(0xffffffffu, p >= 0);
            const int nkw = __reduce_max_sync(0xffffffffu, nk);
            if (wact) {
                float2 mls[4];
                const float2* bs = bstat + ((size_t)b * NM + (p >= 0 ? p : 0)) * H + h0;
#pragma unroll
                for (int hh = 0; hh < 4; ++hh) mls[hh] = (hh < HH && p >= 0) ? bs[hh] : make_float2(0.f, 1.f);
                const float cdx = 3.90625e-3f * 1.01f * sl2;  // 2^-8 (1 + 2^-7), log2 units
#pragma unroll
                for (int hh = 0; hh < 4; ++hh) {
                    if (hh >= HH) break;
                    const int h = h0 + hh;
                    // ||q~|| of this head, from the staged query before its columns take the weights
                    float qn = 0.f;
#pragma unroll
                    for (int c8 = 0; c8 < 4; ++c8) {
                        const uint4 u = *reinterpret_cast<const uint4*>(sQE + tc::core_off(r, h * 32 + c8 * 8, d));
                        const __nv_bfloat162* b2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float2 f = __bfloat1622float2(b2[k]);
                            qn = fmaf(f.x, f.x, fmaf(f.y, f.y, qn));
                        }
                    }
                    qn = cdx * sqrtf(qn);
                    uint32_t s[32];
                    tc::tmem_ld32(tmem + lane_base + h * 32, s);
                    const float2 ml = mls[hh];
                    const float m2 = ml.x * 1.4426950408889634f;
                    float seb = 0.f, sec = 0.f;
                    uint32_t e16[16];  // the 32 weights as packed BF16 pairs
                    float aa = 0.f, at = 0.f;  // the error bound's sums A and T
                    const float* kn = sKn + h * 32;
                    const float* vn = sVn + h * 32;
                    if (nkw <= 4)
                        patch_weights<4>(s, nk, sl2, m2, guard, seb, sec, e16, qn, kn, vn, aa, at);
                    else if (nkw <= 8)
                        patch_weights<8>(s, nk, sl2, m2, guard, seb, sec, e16, qn, kn, vn, aa, at);
                    else
                        patch_weights<16>(s, nk, sl2, m2, guard, seb, sec, e16, qn, kn, vn, aa, at);
#pragma unroll
                    for (int c8 = 0; c8 < 4; ++c8)
                        *reinterpret_cast<uint4*>(sQE + tc::core_off(r, h * 32 + c8 * 8, d)) =
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
            if (tid == 0) {
                tc::tc_fence_after();
                const uint64_t de = tc::desc_kmajor_none(tc::smem_u32(sQE), 128, (d / 8) * 128);
                for (int h = 0; h < H; ++h) {
                    const uint64_t dv = tc::desc_kmajor_none(tc::smem_u32(sVt + h * 2048), 128, (32 / 8) * 128);
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks)
                        tc::mma_bf16(tmem + h * 32, de + (uint64_t)(h * 32 + ks * 16), dv + (uint64_t)(ks * 16),
                                     tc::idesc_bf16_f32(128, DH), ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            ok = __syncthreads_and(tc::mbar_wait(bar, phase, status)) != 0;
            phase ^= 1;
            tc::tc_fence_after();
            if (!ok) break;
            // pass A: delta = (acc - w o) / l' for the own heads, back into TMEM; partial norm
            const float* orow = O + (size_t)(rb + (p >= 0 ? p : 0)) * d;
            float n2 = 0.f, b2 = 0.f;
#pragma unroll
            for (int hh = 0; hh < 4; ++hh) {
                if (hh >= HH || !wact) break;
                const int h = h0 + hh;
                float4 o4[8];
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    o4[t] = p >= 0 ? *reinterpret_cast<const float4*>(orow + h * 32 + 4 * t) : make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t a[32];
                tc::tmem_ld32(tmem + lane_base + h * 32, a);
                float hn2 = 0.f, on2 = 0.f;
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float d0 = (__uint_as_float(a[4 * t]) - w[hh] * o4[t].x) * inv[hh];
                    const float d1 = (__uint_as_float(a[4 * t + 1]) - w[hh] * o4[t].y) * inv[hh];
                    const float d2 = (__uint_as_float(a[4 * t + 2]) - w[hh] * o4[t].z) * inv[hh];
                    const float d3 = (__uint_as_float(a[4 * t + 3]) - w[hh] * o4[t].w) * inv[hh];
                    hn2 = fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, fmaf(d3, d3, hn2))));
                    on2 = fmaf(o4[t].x, o4[t].x, fmaf(o4[t].y, o4[t].y, fmaf(o4[t].z, o4[t].z, fmaf(o4[t].w, o4[t].w, on2))));
                    a[4 * t] = __float_as_uint(d0);
                    a[4 * t + 1] = __float_as_uint(d1);
                    a[4 * t + 2] = __float_as_uint(d2);
                    a[4 * t + 3] = __float_as_uint(d3);
                }
                n2 += hn2;
                // B_h = 1.1 (A + T (||o_h|| + ||delta~_h||)) / (l~' - 1.1 T)
                const float bh = ea[hh] + et[hh] * (sqrtf(on2) + sqrtf(hn2));
                b2 = fmaf(bh, bh, b2);
                tc::tmem_st32(tmem + lane_base + h * 32, a);
            }
            sN2[tid] = make_float2(n2, guard ? -1.f : b2);
            __syncthreads();
            {  // the same sums, in the same order, for both threads of the row
                const float2 a0 = sN2[r], a1 = sN2[128 + r];
                n2 = a0.x + a1.x;
                guard = a0.y < 0.f || a1.y < 0.f;
            }
            const float bnd = guard ? 0.f : sqrtf(sN2[r].y + sN2[128 + r].y);
            const CertRow* cr = cert + ((size_t)b * NM + (p >= 0 ? p : 0));
            int md = -1, nc = 0;
            if (p >= 0) {
                if (guard) {
                    md = 2;
                } else {
                    // ||delta|| <= ||delta~|| + B for the exact correction of these inputs
                    const float dn = sqrtf(n2) + bnd;
                    if (!(dn < cr->next)) {
                        md = 1;
                    } else {
                        while (nc < cr->n && cr->rho[nc] <= dn) ++nc;
                        md = nc ? 3 : 0;
                    }
                }
            }
            // pass B: exact check of the listed candidates, each thread over its heads
            // (md agrees between warps w and w + 4, so their TMEM loads stay warp-uniform)
            if (__any_sync(0xffffffffu, md == 3)) {
                float proj[CERT_T];
#pragma unroll
                for (int i = 0; i < CERT_T; ++i) proj[i] = 0.f;
                const float* wc = codebook + (size_t)(md == 3 ? cr->code : 0) * d;
                for (int hh = 0; hh < HH; ++hh) {
                    const int h = h0 + hh;
                    uint32_t a[32];
                    tc::tmem_ld32(tmem + lane_base + h * 32, a);
                    if (md == 3) {
                        for (int i = 0; i < nc; ++i) {
                            const float* wj = codebook + (size_t)cr->j[i] * d + h * 32;
                            float sacc = 0.f;
#pragma unroll
                            for (int t = 0; t < 32; t += 4) {
                                const float4 a4 = *reinterpret_cast<const float4*>(wj + t);
                                const float4 c4 = *reinterpret_cast<const float4*>(wc + h * 32 + t);
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
            __syncthreads();
            if (md == 3) {
                md = 0;
                for (int i = 0; i < nc; ++i) {
                    const float wj = wd[(size_t)cr->code * ch.K + cr->j[i]];  // ||W_j - W_c||
                    if (!(cr->gap[i] - 2.f * (sP[r * CERT_T + i] + sP[(128 + r) * CERT_T + i] + bnd * wj) > cr->eta))
                        md = 1;
                }
            }
            // split operands: a row the certificate does not settle gets its exact correction
            // from them (k_inc_exact_delta) before the search
            if (split && md == 1 && half == 0) ex_rows[atomicAdd(&ch.counters[CNT_EX], 1)] = make_int2(rc + p, p);
            // a searched row: o + delta goes to O for the vector quantizer
            if (!split && __any_sync(0xffffffffu, md == 1)) {
                float* xo = O + (size_t)(rc + (p >= 0 ? p : 0)) * d;
                for (int hh = 0; hh < HH; ++hh) {
                    const int h = h0 + hh;
                    uint32_t a[32];
                    tc::tmem_ld32(tmem + lane_base + h * 32, a);
                    if (md == 1) {
#pragma unroll
                        for (int t = 0; t < 32; t += 4) {
                            const float4 o4 = *reinterpret_cast<const float4*>(orow + h * 32 + t);
                            *reinterpret_cast<float4*>(xo + h * 32 + t) =
                                make_float4(o4.x + __uint_as_float(a[t]), o4.y + __uint_as_float(a[t + 1]),
                                            o4.z + __uint_as_float(a[t + 2]), o4.w + __uint_as_float(a[t + 3]));
                        }
                    }
                }
            }
            if (half == 0) {
                if (md == 0) code[rc + p] = cr->code;
                if (md >= 1) sVq[atomicAdd(&sNvq, 1)] = rc + p;
                if (md == 2) sFull[atomicAdd(&sNfull, 1)] = rc + p;
                n_patched += (md == 0 || md == 1);
                n_cert += md == 0;
                n_full += md == 2;
                n_pairs += p >= 0 ? nk : 0;
            }
            tc::tc_fence_before();
            __syncthreads();  // TMEM and the staging space are free for the next tile
        }
        __syncthreads();
        if (tid == 0) {  // one atomic per list
            sBase[0] = sNvq ? atomicAdd(&ch.counters[CNT_V], sNvq) : 0;
            sBase[1] = sNfull ? act_off[ch.cfg_off[b]] + atomicAdd(&rc_cnt[b], sNfull) : 0;
        }
        __syncthreads();
        for (int i = tid; i < sNvq; i += blockDim.x) vq_rows[sBase[0] + i] = sVq[i];
        for (int i = tid; i < sNfull; i += blockDim.x) rc_rows[sBase[1] + i] = make_int2(sFull[i], sFull[i] - rc);
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
        for (int k = 0; k < nd; ++k) {
            const int kp = dp[k];
            if (kp >= p) break;  // ascending: the rest lie after the row
            float ks[PER], kc[PER];
            ld_split<PER>(qkv + (size_t)ub[kp] * ld + d + lane * PER, lo_off, ks);
            ld_split<PER>(qkv + (size_t)uc[kp] * ld + d + lane * PER, lo_off, kc);
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
            float vs[PER], vc[PER];
            ld_split<PER>(qkv + (size_t)ub[kp] * ld + 2 * d + lane * PER, lo_off, vs);
            ld_split<PER>(qkv + (size_t)uc[kp] * ld + 2 * d + lane * PER, lo_off, vc);
#pragma unroll
            for (int t = 0; t < PER; ++t) acc[t] = fmaf(ec, vc[t] - o[t], fmaf(-es, vs[t] - o[t], acc[t]));
            sum_s += es;
            sum_c += ec;
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
                               int2* ex_rows, int* status, long long* stats, cudaStream_t st, int grid) {
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
            const uint32_t cols = ch.heads * 32 <= 128 ? 128 : 256;
            size_t smem_tc = patch_tc_smem(ch.d, ch.heads, ch.N);
            if (smem_tc > 227 * 1024) return cudaErrorInvalidValue;
            // the TMEM columns of the CTAs resident on one SM must fit in its 512
            const size_t max_ctas = 512 / cols;
            if ((228 * 1024) / smem_tc > max_ctas) smem_tc = (228 * 1024) / (max_ctas + 1) + 1024;
            static size_t granted_tc = 0;
            if (smem_tc > granted_tc) {
                cudaFuncSetAttribute(k_inc_patch_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tc);
                granted_tc = smem_tc;
            }
            k_inc_patch_tc<<<grid, 256, smem_tc, st>>>(ch, uid, qkv, O, bstat, cert, codebook, wd, code, vq_rows,
                                                      act_off, rc_rows, rc_cnt, list_tc, dpos, dcnt, split, ex_rows,
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
                                     grid);
}
cudaError_t launch_inc_patch(const Chunk& ch, const int* uid, const __nv_bfloat16* qkv, float* O,
                             const float2* bstat, const CertRow* cert, const float* codebook, const float* wd,
                             int* code, int* vq_rows, const int* act_off, int2* rc_rows, int* rc_cnt,
                             const int* list_tc, const int* list_simt, const short* dpos, const int* dcnt, int use_tc,
                             int split, int2* ex_rows, int* status, long long* stats, cudaStream_t st, int grid) {
    return launch_inc_patch_t<__nv_bfloat16>(ch, uid, qkv, O, bstat, cert, codebook, wd, code, vq_rows, act_off,
                                             rc_rows, rc_cnt, list_tc, list_simt, dpos, dcnt, use_tc, split, ex_rows,
                                             status, stats, st, grid);
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
