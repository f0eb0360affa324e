// Nearest-codeword assignment on the tensor cores with FP32-grade distances
// (Sec. 3.1, Eq. vq): code(o) = argmin_j ||W_j||^2 - 2 o . W_j, lowest j on ties.
//
// o . W_j is a [rows x d] x [d x K] contraction.  Each FP32 operand x is split
// into x_hi = tf32(x) and x_lo = tf32(x - x_hi); the product is accumulated as
// o_hi W_hi + o_hi W_lo + o_lo W_hi (the lo x lo term is below 2^-22 relative),
// which keeps the dot products at FP32 accuracy on the TF32 tensor pipe.
//
// Persistent CTA of 10 warps per SM, 128-row tiles of active rows:
//   warps 0-3  loaders: gather the tile's O rows, split them, write the hi/lo A
//              chunks (32 columns, 128-byte swizzle) into the shared-memory ring;
//              the next two chunks' global loads are in flight while a loader
//              waits for a free slot;
//   warps 4-7  epilogue: read the accumulator columns from TMEM and reduce
//              (best, index, second best) per row; the accumulator is double
//              buffered when it fits, so this overlaps the next tile's MMAs;
//   warp 8     one thread issues the tcgen05.mma (kind::tf32, M = 128,
//              N <= 256, K = 8) and releases slots by tcgen05.commit;
//   warp 9     one thread: TMA of the codebook hi/lo chunks (precomputed per
//              layer), running a ring slot ahead of the MMAs.
// All waits are bounded (VQNQS_DEV_TIMEOUT).
// Distance mode (dist_out given): instead of the assignment, the epilogue writes
// every listed row's distances ||o||^2 - 2 o . W_j + ||W_j||^2 to dist_out[m][j]
// and ||o||^2 to osq_out[m] (m: the row's index in the list); codes and the
// near-tie count are left alone.
#include "tc_common.cuh"

namespace vq {

constexpr int VT_BM = 128, VT_BK = 32, VT_THREADS = 320;

__host__ __device__ constexpr uint32_t idesc_tf32_f32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// byte offset of element (r, k) (4-byte elements, 32 per row) in a 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + (k & 3) * 4);
}

struct VqBest {
    float v1;
    int i1;
    float v2;
};

__device__ __forceinline__ void vq_merge(VqBest& a, float c, int j) {
    if (c < a.v1 || (c == a.v1 && j < a.i1)) {
        a.v2 = a.v1;
        a.v1 = c;
        a.i1 = j;
    } else {
        a.v2 = fminf(a.v2, c);
    }
}

template <int KC>  // codewords per pass (N of the MMA), K <= 2 * KC
__global__ void __launch_bounds__(VT_THREADS, 1)
k_vq_tc(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
        const float* __restrict__ O, const int* __restrict__ counters, const int* __restrict__ act_rows,
        const float* __restrict__ cnorm, int K, int d, int* __restrict__ code, long long* __restrict__ near_ties,
        int* __restrict__ status, int VT_STAGES, uint32_t tmem_cols, int ACC, int a_slot,
        float* __restrict__ dist_out, float* __restrict__ osq_out) {
    constexpr int A_BYTES = VT_BM * VT_BK * 4;   // 16 KB per part
    constexpr int B_BYTES = KC * VT_BK * 4;      // per part and pass
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int passes = (K + KC - 1) / KC;
    const int SLOT = 2 * A_BYTES + passes * 2 * B_BYTES;  // A_hi, A_lo, then per pass B_hi, B_lo
    uint64_t* fullA = reinterpret_cast<uint64_t*>(smem + VT_STAGES * SLOT);
    uint64_t* fullB = fullA + VT_STAGES;
    uint64_t* empty = fullB + VT_STAGES;
    uint64_t* accf = empty + VT_STAGES;  // [2]
    uint64_t* acce = accf + 2;           // [2]
    uint64_t* osqf = acce + 2;           // [2] loaders -> epilogue: row norms written
    uint64_t* done = osqf + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    float* osq_s = reinterpret_cast<float*>(tmem_holder + 4);  // [2][128]
    float* cn_s = osq_s + 2 * VT_BM;                            // [K] codeword norms
    __shared__ int s_ties;

    const int R = counters[a_slot];  // rows listed in act_rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
    const int tiles = (R + VT_BM - 1) / VT_BM, KB = d / VT_BK;
    if (tid == 0) {
        for (int s = 0; s < VT_STAGES; ++s) {
            tc::mbar_init(&fullA[s], 128);
            tc::mbar_init(&fullB[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(&accf[a], 1);
            tc::mbar_init(&acce[a], 128);
            tc::mbar_init(&osqf[a], 128);
        }
        tc::mbar_init(done, 1);
        tc::fence_barrier_init();
        s_ties = 0;
    }
    for (int j = tid; j < K; j += blockDim.x) cn_s[j] = cnorm[j];
    if (warp == 8) tc::tmem_alloc(tmem_holder, tmem_cols);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;
    const int accw = passes * KC;  // TMEM columns of one accumulator

    if (warp == 9) {
        // ---- TMA producer: codebook hi/lo chunks, one ring slot ahead of the MMAs ----
        if (lane == 0) {
            tc::prefetch_tmap(&tm_hi);
            tc::prefetch_tmap(&tm_lo);
            bool ok = true;
            int it = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % VT_STAGES;
                    const uint32_t ph = (it / VT_STAGES) & 1;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, status)) { ok = false; break; }
                    uint8_t* slot = smem + s * SLOT;
                    tc::mbar_arrive_expect_tx(&fullB[s], passes * 2 * B_BYTES);
                    for (int ps = 0; ps < passes; ++ps) {
                        uint8_t* bh = slot + 2 * A_BYTES + ps * 2 * B_BYTES;
                        tc::tma_load_2d(bh, &tm_hi, kb * VT_BK, ps * KC, &fullB[s]);
                        tc::tma_load_2d(bh + B_BYTES, &tm_lo, kb * VT_BK, ps * KC, &fullB[s]);
                    }
                }
            }
            if (!ok) {  // drain this thread's own copies still in flight
                for (int j = it - VT_STAGES; j < it; ++j)
                    if (j >= 0) tc::mbar_wait(&fullB[j % VT_STAGES], (j / VT_STAGES) & 1, status, 100000000LL);
            }
        }
    } else if (warp == 8) {
        // ---- MMA issue ------------------------------------------------------------------
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_tf32_f32(VT_BM, KC);
            bool ok = true;
            int it = 0, i = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
                const int a = i % ACC;
                if (!tc::mbar_wait(&acce[a], ((i / ACC) & 1) ^ 1, status)) { ok = false; break; }
                tc::tc_fence_after();
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % VT_STAGES;
                    const uint32_t ph = (it / VT_STAGES) & 1;
                    uint8_t* slot = smem + s * SLOT;
                    if (!tc::mbar_wait(&fullB[s], ph, status) || !tc::mbar_wait(&fullA[s], ph, status)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint64_t dah = tc::desc_kmajor_sw128(tc::smem_u32(slot));
                    const uint64_t dal = tc::desc_kmajor_sw128(tc::smem_u32(slot + A_BYTES));
                    for (int ps = 0; ps < passes; ++ps) {
                        uint8_t* bh = slot + 2 * A_BYTES + ps * 2 * B_BYTES;
                        const uint64_t dbh = tc::desc_kmajor_sw128(tc::smem_u32(bh));
                        const uint64_t dbl = tc::desc_kmajor_sw128(tc::smem_u32(bh + B_BYTES));
                        const uint32_t dt = tmem + a * accw + ps * KC;
#pragma unroll
                        for (int k = 0; k < VT_BK / 8; ++k) {
                            const uint32_t acc0 = (kb | k) != 0 ? 1u : 0u;
                            mma_tf32(dt, dah + 2 * k, dbh + 2 * k, idesc, acc0);
                            mma_tf32(dt, dah + 2 * k, dbl + 2 * k, idesc, 1u);
                            mma_tf32(dt, dal + 2 * k, dbh + 2 * k, idesc, 1u);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[a]);
            }
            tc::mma_commit(done);
            tc::mbar_wait(done, 0, status, 100000000LL);
        }
    } else if (warp < 4) {
        // ---- loaders: thread tid owns tile row tid; loads of the next two chunks
        // are in flight while this thread waits for a free slot -----------------
        int it = 0, i = 0;
        int t = blockIdx.x, kb = 0;
        float4 cur[VT_BK / 4];
        auto issue = [&](int tt, int kk, float4 (&dst)[VT_BK / 4]) {
            const int m = tt * VT_BM + tid;
            const bool valid = tt < tiles && m < R;
            const float* src = O + (size_t)(valid ? act_rows[m] : 0) * d + kk * VT_BK;
#pragma unroll
            for (int q = 0; q < VT_BK / 4; ++q)
                dst[q] = valid ? *reinterpret_cast<const float4*>(src + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        // register ring: the chunks at distance 1 and 2 are in flight while this one is stored
        float4 n1[VT_BK / 4];
        auto advance = [&](int& tt, int& kk) {
            if (++kk == KB) { kk = 0; tt += gridDim.x; }
        };
        int t1 = t, k1 = 0, t2, k2;
        advance(t1, k1);
        t2 = t1; k2 = k1;
        advance(t2, k2);
        if (t < tiles) issue(t, 0, cur);
        if (t1 < tiles) issue(t1, k1, n1);
        float osq = 0.f;
        bool ok = true;
        while (t < tiles && ok) {
            float4 n3[VT_BK / 4];
            if (t2 < tiles) issue(t2, k2, n3);
            const int s = it % VT_STAGES;
            const uint32_t ph = (it / VT_STAGES) & 1;
            if (!tc::mbar_wait(&empty[s], ph ^ 1, status)) { ok = false; break; }
            uint8_t* slot = smem + s * SLOT;
#pragma unroll
            for (int q = 0; q < VT_BK / 4; ++q) {
                const float4 v = cur[q];
                osq = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, osq))));
                const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
                const float4 lo = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
                const uint32_t off = sw128_off(tid, 4 * q);
                *reinterpret_cast<float4*>(slot + off) = h;
                *reinterpret_cast<float4*>(slot + A_BYTES + off) = lo;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tc::mbar_arrive(&fullA[s]);
            ++it;
            if (kb == KB - 1) {  // row norm of this tile for the epilogue
                const int a = i % ACC;
                // the epilogue reads slot a's previous norms before it releases accumulator a
                if (!tc::mbar_wait(&acce[a], ((i / ACC) & 1) ^ 1, status)) { ok = false; break; }
                osq_s[a * VT_BM + tid] = osq;
                tc::mbar_arrive(&osqf[a]);
                osq = 0.f;
                ++i;
            }
#pragma unroll
            for (int q = 0; q < VT_BK / 4; ++q) { cur[q] = n1[q]; n1[q] = n3[q]; }
            t = t1; kb = k1;
            t1 = t2; k1 = k2;
            advance(t2, k2);
        }
    } else {
        // ---- epilogue: warps 4-7 own TMEM lanes 32 (w - 4) .. + 31 -----------------
        const int row = tid - 128;
        const uint32_t lb = (uint32_t)((warp - 4) * 32) << 16;
        int ties = 0, i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const int a = i % ACC;
            const uint32_t ph = (i / ACC) & 1;
            if (!tc::mbar_wait(&accf[a], ph, status) || !tc::mbar_wait(&osqf[a], ph, status)) break;
            tc::tc_fence_after();
            VqBest best;
            best.v1 = INFINITY; best.i1 = 0x7fffffff; best.v2 = INFINITY;
            const float osq = osq_s[a * VT_BM + row];
            const int m = t * VT_BM + row;
            for (int c0 = 0; c0 < accw; c0 += 32) {
                uint32_t r[32];
                tc::tmem_ld32(tmem + lb + a * accw + c0, r);
                if (dist_out) {  // K is a multiple of 16: a group of four columns is all in or all out
                    if (m < R) {
                        float* dr = dist_out + (size_t)m * K + c0;
#pragma unroll
                        for (int j = 0; j < 32; j += 4)
                            if (c0 + j < K)
                                *reinterpret_cast<float4*>(dr + j) =
                                    make_float4(fmaf(-2.f, __uint_as_float(r[j]), osq) + cn_s[c0 + j],
                                                fmaf(-2.f, __uint_as_float(r[j + 1]), osq) + cn_s[c0 + j + 1],
                                                fmaf(-2.f, __uint_as_float(r[j + 2]), osq) + cn_s[c0 + j + 2],
                                                fmaf(-2.f, __uint_as_float(r[j + 3]), osq) + cn_s[c0 + j + 3]);
                    }
                    __syncwarp();  // the next tcgen05.ld is warp-collective
                    continue;
                }
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int n = c0 + j;
                    if (n < K) vq_merge(best, fmaf(-2.f, __uint_as_float(r[j]), cn_s[n]), n);
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acce[a]);
            if (dist_out) {
                if (m < R) osq_out[m] = osq;
            } else if (m < R) {
                if (best.i1 >= K) {  // no finite distance: codeword 0, and the status says so
                    best.i1 = 0;
                    atomicOr(status, VQNQS_DEV_NONFINITE);
                }
                code[act_rows[m]] = best.i1;
                const float l1 = best.v1 + osq, l2 = best.v2 + osq;
                if (K > 1 && (l2 - l1) < NEAR_TIE_REL * fmaxf(l1, 1e-30f)) ++ties;
            }
        }
        if (ties) atomicAdd(&s_ties, ties);
    }
    __syncwarp();
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0 && s_ties) atomicAdd(reinterpret_cast<unsigned long long*>(near_ties), (unsigned long long)s_ties);
    if (warp == 8) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, tmem_cols);
    }
}

// codebook split for the tensor-core argmin: hi = tf32(W), lo = tf32(W - hi)
__global__ void k_split_tf32(const float* __restrict__ W, size_t n, float* __restrict__ hi, float* __restrict__ lo) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float h = tf32_round(W[i]);
        hi[i] = h;
        lo[i] = tf32_round(W[i] - h);
    }
}

cudaError_t launch_split_tf32(const float* W, size_t n, float* hi, float* lo, cudaStream_t st) {
    k_split_tf32<<<256, 256, 0, st>>>(W, n, hi, lo);
    return cudaGetLastError();
}

bool vq_tc_supported(int K, int d) {
    const int KC = K > 256 ? 256 : K;
    const bool inst = KC == 16 || KC == 32 || KC == 48 || KC == 64 || KC == 96 || KC == 128 || KC == 192 || KC == 256;
    return inst && K <= 512 && K % KC == 0 && d % VT_BK == 0;
}

// Tensor map of a [K][d] FP32 codebook part: boxes of 32 columns x KC rows, 128-byte swizzle.
cudaError_t make_tmap_codebook(CUtensorMap* map, const float* base, int K, int d) {
    typedef CUresult (*Fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                           const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                           CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static Fn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return cudaErrorNotSupported;
        fn = reinterpret_cast<Fn>(p);
    }
    const int KC = K > 256 ? 256 : K;
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)K};
    cuuint64_t strides[1] = {(cuuint64_t)d * 4};
    cuuint32_t box[2] = {(cuuint32_t)VT_BK, (cuuint32_t)KC};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_vq_tc(const CUtensorMap& tm_hi, const CUtensorMap& tm_lo, const float* O, const int* counters,
                         const int* act_rows, const float* cnorm, int K, int d, int* code, long long* near_ties,
                         int* status, cudaStream_t st, int num_sms, int Rmax, int a_slot, float* dist_out,
                         float* osq_out) {
    if (!vq_tc_supported(K, d)) return cudaErrorInvalidValue;
    const int KC = K > 256 ? 256 : K;
    const int passes = (K + KC - 1) / KC;
    const size_t slot = 2 * (size_t)VT_BM * VT_BK * 4 + (size_t)passes * 2 * KC * VT_BK * 4;
    const size_t limit = 227 * 1024;
    const size_t extra = 256 + 2 * VT_BM * 4 + (size_t)K * 4;  // barriers, TMEM address, row and codeword norms
    int stages = (1024 + 2 * slot + extra <= limit) ? 2 : 1;
    size_t smem = 1024 + stages * slot + extra;
    if (smem > limit) return cudaErrorInvalidValue;
    const int acc = (2 * passes * KC <= 512) ? 2 : 1;  // double-buffered accumulator when it fits
    uint32_t cols = 32;
    while ((int)cols < acc * passes * KC) cols <<= 1;
    // every CTA resident on an SM holds `cols` TMEM columns: cap the residency
    const size_t max_ctas = 512 / cols;
    if ((228 * 1024) / smem > max_ctas) smem = (228 * 1024) / (max_ctas + 1) + 1024;
    int tiles = (Rmax + VT_BM - 1) / VT_BM;
    int grid = tiles < num_sms ? tiles : num_sms;
    if (grid < 1) grid = 1;
    static size_t granted[9] = {};  // per instantiation; set once per size, outside captures
#define VQ_TC_CASE(X)                                                                                      \
    if (KC == X) {                                                                                         \
        size_t& gr = granted[(X == 16) ? 0 : (X == 32) ? 1 : (X == 48) ? 2 : (X == 64) ? 3 : (X == 96) ? 4 \
                             : (X == 128) ? 5 : (X == 192) ? 6 : 7];                                       \
        if (smem > gr) {                                                                                   \
            cudaFuncSetAttribute(k_vq_tc<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);      \
            gr = smem;                                                                                     \
        }                                                                                                  \
        k_vq_tc<X><<<grid, VT_THREADS, smem, st>>>(tm_hi, tm_lo, O, counters, act_rows, cnorm, K, d, code,  \
                                                   near_ties, status, stages, cols, acc, a_slot, dist_out, \
                                                   osq_out);                                               \
        return cudaGetLastError();                                                                         \
    }
    VQ_TC_CASE(16) VQ_TC_CASE(32) VQ_TC_CASE(48) VQ_TC_CASE(64) VQ_TC_CASE(96) VQ_TC_CASE(128) VQ_TC_CASE(192)
    VQ_TC_CASE(256)
#undef VQ_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace vq
