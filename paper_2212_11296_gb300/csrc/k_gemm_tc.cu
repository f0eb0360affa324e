// BF16 tensor-core GEMM for the per-location operations (Sec. 3.2: QKV
// projection, MLP up + GELU, MLP down + residual), FP32 accumulation in TMEM.
//
//   C[M, N] = A[M, K] @ Bt[N, K]^T + bias (+ epilogue),  A and Bt K-major BF16.
//
// Persistent kernel, one CTA per SM, 18 warps:
//   warp 0      one thread issues TMA tile loads (128-byte swizzle) into a ring
//               of STAGES shared-memory slots, completion tracked by mbarriers;
//   warp 1      one thread issues tcgen05.mma (M = 128, N = BN, K = 16) into a
//               double-buffered TMEM accumulator and commits slot releases;
//               the warp also owns the TMEM allocation;
//   warps 2-17  epilogue (four warps per 32-lane TMEM quarter, every fourth
//               32-column chunk): tcgen05.ld, bias / activation / residual in
//               FP32, TMA stores of 32 x 32 chunks, then release the
//               accumulator buffer so the next tile's MMAs overlap.
// The row count M is read from device memory (unique rows are only known on
// the device).  Every wait is bounded; on timeout the kernel sets
// VQNQS_DEV_TIMEOUT, drains its own in-flight copies and frees its TMEM.
// A row's result depends only on that row: the K loop order is fixed.
//
// Split operands (a_lo_row > 0): A and Bt each hold a BF16 lo plane after the
// hi one (A's at row a_lo_row, Bt's at row N), x = hi + lo with hi = bf16(x),
// lo = bf16(x - hi), and the K loop runs three passes into one accumulator:
// A_hi Bt_hi, A_hi Bt_lo, A_lo Bt_hi (the lo.lo term, below 2^-18 of a
// product, is dropped): FP32-grade products from BF16 MMAs.  BF16 outputs
// (epilogues 0 and 1) are then written the same way, the lo plane at row
// c_lo_row.
#include <cstdio>

#include "tc_common.cuh"

namespace vq {

constexpr int TC_BM = 128, TC_BK = 64;

// 16 epilogue warps, four per TMEM lane quarter; per epilogue warp one 32 x 32 output chunk slot
constexpr int EPI_WARPS = 16, SLOT_BYTES = 4096, TC_THREADS = 64 + 32 * EPI_WARPS;

template <int BN>
struct TcCfg {
    // as many ring stages (up to 6) as fit beside the output slots
    static constexpr int STAGES_FIT = (227 * 1024 - 1024 - 512 - EPI_WARPS * SLOT_BYTES) / (TC_BM * TC_BK * 2 + BN * TC_BK * 2);
    static constexpr int STAGES = STAGES_FIT < 6 ? STAGES_FIT : 6;
    static constexpr int A_BYTES = TC_BM * TC_BK * 2;
    static constexpr int B_BYTES = BN * TC_BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int TMEM_COLS = 2 * BN <= 128 ? 128 : (2 * BN <= 256 ? 256 : 512);
    // barriers (2 STAGES + 5 + EPI_WARPS words) and the TMEM address after the slots
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + (size_t)EPI_WARPS * SLOT_BYTES + 512;
    static_assert((2 * STAGES + 5 + EPI_WARPS) * 8 + 4 <= 512, "barrier block");
    static_assert(SMEM <= 227 * 1024, "shared memory per CTA");
};

// erf by Abramowitz & Stegun 7.1.26 (|error| <= 1.5e-7 for all real x):
// erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2), t = 1 / (1 + p |z|),
// odd in z.  Evaluated with the SFU's reciprocal and exponential; the BF16 outputs
// it feeds resolve 4e-3 relative.
__device__ __forceinline__ float erf_as(float z) {
    const float s = fabsf(z);
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, s, 1.0f)));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    float e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-s * s * 1.4426950408889634f));
    return copysignf(fmaf(-poly, e, 1.0f), z);
}
__device__ __forceinline__ float gelu_tc(float x) {
    const float h = 0.5f * x;
    return fmaf(h, erf_as(x * 0.70710678118654752f), h);
}

// 2D TMA store of a shared-memory box (bulk group of this thread) and the waits on it.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(tc::smem_u32(src))
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

template <int BN, int EPI>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_gemm_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const __grid_constant__ CUtensorMap tmC, const __grid_constant__ CUtensorMap tmR,
          const float* __restrict__ bias, const float* __restrict__ R, void* __restrict__ Cout,
          const int* __restrict__ counters, int u_slot, int N, int K, int a_lo_row, int c_lo_row,
          int* __restrict__ status, int ksplit) {
    using C = TcCfg<BN>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + C::STAGES * C::A_BYTES;
    uint8_t* sOut = sB + C::STAGES * C::B_BYTES;  // [EPI_WARPS][SLOT_BYTES], 1024-byte aligned
    uint64_t* full = reinterpret_cast<uint64_t*>(sOut + EPI_WARPS * SLOT_BYTES);
    uint64_t* empty = full + C::STAGES;
    uint64_t* accf = empty + C::STAGES;
    uint64_t* acce = accf + 2;
    uint64_t* done = acce + 2;
    uint64_t* rbar = done + 1;  // [EPI_WARPS]: residual chunk loads
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(rbar + EPI_WARPS);

    const int M = counters[u_slot];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_tiles = N / BN, m_tiles = (M + TC_BM - 1) / TC_BM, tiles_mn = m_tiles * n_tiles;
    // split K: work item t = (split sk, output tile); split sk takes K blocks [sk KBs, (sk + 1) KBs)
    // and writes its partial tile at row sk * Mpad of the output
    const int total = tiles_mn * ksplit;
    const int KB = K / TC_BK;
    const int KBs = (KB + ksplit - 1) / ksplit;
    const int NPASS = a_lo_row > 0 ? 3 : 1;  // split operands: three passes
    const int Mpad = m_tiles * TC_BM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
        for (int a = 0; a < 2; ++a) { tc::mbar_init(&accf[a], 1); tc::mbar_init(&acce[a], 32 * EPI_WARPS); }
        tc::mbar_init(done, 1);
        for (int w = 0; w < EPI_WARPS; ++w) tc::mbar_init(&rbar[w], 1);
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc(tmem_holder, C::TMEM_COLS);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            tc::prefetch_tmap(&tmA);
            tc::prefetch_tmap(&tmB);
            bool ok = true;
            int it = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x) {
                const int sk = t / tiles_mn, tt = t - sk * tiles_mn;
                const int m0 = (tt / n_tiles) * TC_BM, n0 = (tt % n_tiles) * BN;
                const int kb0 = sk * KBs, nkb = min(KB, kb0 + KBs) - kb0;
                for (int kbt = 0; kbt < NPASS * nkb; ++kbt, ++it) {
                    const int s = it % C::STAGES;
                    const uint32_t ph = (it / C::STAGES) & 1;
                    // pass 0: A_hi Bt_hi, pass 1: A_hi Bt_lo, pass 2: A_lo Bt_hi
                    const int pass = kbt / nkb, kb = kb0 + kbt - pass * nkb;
                    if (!tc::mbar_wait(&empty[s], ph ^ 1, status)) { ok = false; break; }
                    tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
                    tc::tma_load_2d(sA + s * C::A_BYTES, &tmA, kb * TC_BK, m0 + (pass == 2 ? a_lo_row : 0), &full[s]);
                    tc::tma_load_2d(sB + s * C::B_BYTES, &tmB, kb * TC_BK, n0 + (pass == 1 ? N : 0), &full[s]);
                }
            }
            if (!ok) {  // wait (bounded) for the copies this thread still has in flight
                for (int j = it - C::STAGES; j < it; ++j)
                    if (j >= 0) tc::mbar_wait(&full[j % C::STAGES], (j / C::STAGES) & 1, status, 100000000LL);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = tc::idesc_bf16_f32(TC_BM, BN);
            bool ok = true;
            int it = 0, i = 0;
            for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
                const int a = i & 1;
                const uint32_t aph = (i >> 1) & 1;
                if (!tc::mbar_wait(&acce[a], aph ^ 1, status)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t d_tmem = tmem + a * BN;
                const int sk = t / tiles_mn;
                const int nkb = min(KB, sk * KBs + KBs) - sk * KBs;
                for (int kbt = 0; kbt < NPASS * nkb; ++kbt, ++it) {
                    const int s = it % C::STAGES;
                    const uint32_t ph = (it / C::STAGES) & 1;
                    if (!tc::mbar_wait(&full[s], ph, status)) { ok = false; break; }
                    tc::tc_fence_after();
                    const uint64_t da = tc::desc_kmajor_sw128(tc::smem_u32(sA + s * C::A_BYTES));
                    const uint64_t db = tc::desc_kmajor_sw128(tc::smem_u32(sB + s * C::B_BYTES));
#pragma unroll
                    for (int k = 0; k < TC_BK / 16; ++k)
                        tc::mma_bf16(d_tmem, da + 2 * k, db + 2 * k, idesc, (kbt | k) != 0 ? 1u : 0u);
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&accf[a]);
            }
            // every MMA this thread issued has completed before TMEM is freed
            tc::mma_commit(done);
            tc::mbar_wait(done, 0, status, 100000000LL);
        }
    } else {
        // warps 2..17: four warps per TMEM lane quarter, each taking every fourth 32-column chunk.
        // A chunk of 32 rows x 32 columns whose rows all exist goes out through the warp's
        // shared-memory slot and a TMA store (rows 128 bytes apart for FP32 with the 128-byte
        // swizzle, 64 bytes apart for BF16 with the 64-byte swizzle: conflict-free writes);
        // a chunk reaching past the M rows is stored row by row.  The residual chunk
        // (epilogue 2) arrives in the same slot by TMA before the accumulator is read.
        const int q = warp & 3;  // TMEM lanes 32q .. 32q+31 are reachable from this warp
        const int part = (warp - 2) >> 2;
        const int ew = warp - 2;
        uint8_t* slot = sOut + ew * SLOT_BYTES;
        constexpr bool F32OUT = EPI >= 2;
        uint32_t rph = 0;  // residual barrier phase
        int i = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < total && ok; t += gridDim.x, ++i) {
            const int a = i & 1;
            const uint32_t aph = (i >> 1) & 1;
            if (!tc::mbar_wait(&accf[a], aph, status)) { ok = false; break; }
            tc::tc_fence_after();
            const int sk = t / tiles_mn, tt = t - sk * tiles_mn;
            const int m0 = (tt / n_tiles) * TC_BM, n0 = (tt % n_tiles) * BN;
            const int rb = m0 + q * 32;  // the chunk's first row
            const int row = rb + lane;
            const int orow = sk * Mpad;  // this split's partial output rows
            const bool boxed = rb + 32 <= M;  // warp-uniform
#pragma unroll 1
            for (int c = part * 32; c < BN && ok; c += 128) {
                const int n = n0 + c;
                if (boxed) {  // the slot is free once the previous store has read it
                    if (lane == 0) {
                        bulk_wait_read0();
                        if (EPI == 2) {
                            tc::mbar_arrive_expect_tx(&rbar[ew], SLOT_BYTES);
                            tc::tma_load_2d(slot, &tmR, n, rb, &rbar[ew]);
                        }
                    }
                    __syncwarp();
                }
                uint32_t r[32];
                tc::tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + a * BN + c, r);
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]) + bias[n + j];
                if (EPI == 1 || EPI == 4) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = gelu_tc(v[j]);
                }
                if (boxed) {
                    if (F32OUT) {  // row `lane` at lane * 128 bytes, 16-byte chunk k at k ^ (lane & 7)
                        float4* srow = reinterpret_cast<float4*>(slot + lane * 128);
                        if (EPI == 2) {
                            if (!tc::mbar_wait(&rbar[ew], rph, status)) {
                                ok = false;  // drain the load into the slot (bounded) before leaving
                                tc::mbar_wait(&rbar[ew], rph, status, 100000000LL);
                            }
                            rph ^= 1;
#pragma unroll
                            for (int k = 0; k < 8; ++k) {
                                const float4 x = srow[k ^ (lane & 7)];
                                v[4 * k] += x.x; v[4 * k + 1] += x.y; v[4 * k + 2] += x.z; v[4 * k + 3] += x.w;
                            }
                        }
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            srow[k ^ (lane & 7)] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
                    } else {  // row `lane` at lane * 64 bytes, 16-byte chunk k at k ^ ((lane >> 1) & 3)
                        // (split outputs: the lo box in the slot's second half, same pattern)
                        uint4* srow = reinterpret_cast<uint4*>(slot + lane * 64);
                        uint4* srow_lo = reinterpret_cast<uint4*>(slot + 2048 + lane * 64);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            uint32_t p[4], pl[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float a = v[8 * k + 2 * j], b = v[8 * k + 2 * j + 1];
                                __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                                p[j] = *reinterpret_cast<uint32_t*>(&h);
                                const float2 hf = __bfloat1622float2(h);
                                __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
                                pl[j] = *reinterpret_cast<uint32_t*>(&l);
                            }
                            srow[k ^ ((lane >> 1) & 3)] = make_uint4(p[0], p[1], p[2], p[3]);
                            if (c_lo_row > 0) srow_lo[k ^ ((lane >> 1) & 3)] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
                        }
                    }
                    tc::fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0 && ok) {
                        if (!F32OUT && c_lo_row > 0) {  // both boxes in one bulk group
                            asm volatile(
                                "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                                    reinterpret_cast<uint64_t>(&tmC)),
                                "r"(n), "r"(rb), "r"(tc::smem_u32(slot))
                                : "memory");
                            tma_store_2d(&tmC, slot + 2048, n, rb + c_lo_row);
                        } else {
                            tma_store_2d(&tmC, slot, n, rb + orow);
                        }
                    }
                } else if (row < M) {
                    if (EPI == 2) {  // FP32 out + residual
                        const float4* rr = reinterpret_cast<const float4*>(R + (size_t)row * N + n);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 x = rr[j];
                            v[4 * j] += x.x; v[4 * j + 1] += x.y; v[4 * j + 2] += x.z; v[4 * j + 3] += x.w;
                        }
                    }
                    if (F32OUT) {
                        float4* out = reinterpret_cast<float4*>(static_cast<float*>(Cout) + ((size_t)row + orow) * N + n);
#pragma unroll
                        for (int j = 0; j < 8; ++j) out[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    } else {
                        uint32_t p[16], pl[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                            p[j] = *reinterpret_cast<uint32_t*>(&h);
                            const float2 hf = __bfloat1622float2(h);
                            __nv_bfloat162 l = __floats2bfloat162_rn(v[2 * j] - hf.x, v[2 * j + 1] - hf.y);
                            pl[j] = *reinterpret_cast<uint32_t*>(&l);
                        }
                        uint4* out = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(Cout) + (size_t)row * N + n);
#pragma unroll
                        for (int j = 0; j < 4; ++j) out[j] = make_uint4(p[4 * j], p[4 * j + 1], p[4 * j + 2], p[4 * j + 3]);
                        if (c_lo_row > 0) {
                            uint4* lo = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(Cout) +
                                                                 ((size_t)row + c_lo_row) * N + n);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                lo[j] = make_uint4(pl[4 * j], pl[4 * j + 1], pl[4 * j + 2], pl[4 * j + 3]);
                        }
                    }
                }
            }
            tc::tc_fence_before();
            tc::mbar_arrive(&acce[a]);
        }
        if (lane == 0) bulk_wait0();  // this warp's stores have landed before the kernel ends
    }
    __syncwarp();
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

__global__ void k_set_int(int* p, int v) { *p = v; }

// C[m][n] += sum over s (in order) of part[s * Mpad + m][n], m < M
__global__ void k_splitk_add(const float* __restrict__ part, int ksplit, long long Mpad, int M, int N,
                             float* __restrict__ C) {
    const long long total = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const long long m = i / N, n = i - m * N;
        float s = C[i];
        for (int k = 0; k < ksplit; ++k) s += part[((long long)k * Mpad + m) * N + n];
        C[i] = s;
    }
}

// A bounded wait on an mbarrier that no thread arrives on: it must give up
// after about limit_cycles and record VQNQS_DEV_TIMEOUT (exercises the
// failure path every tensor-core kernel relies on, without a fault).
__global__ void k_timeout_probe(int* status, long long limit_cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) tc::mbar_wait(&bar, 0, status, limit_cycles);
}

cudaError_t launch_timeout_probe(int* status, long long limit_cycles, cudaStream_t st) {
    k_timeout_probe<<<1, 32, 0, st>>>(status, limit_cycles);
    return cudaGetLastError();
}

// ---- host side -----------------------------------------------------------------
namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

template <int BN, int EPI>
cudaError_t launch_bn(const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tcm, const CUtensorMap& trm,
                      const float* bias, const float* R, void* Cout,
                      const int* counters, int u_slot, int Mmax, int N, int K, int a_lo_row, int c_lo_row,
                      int* status, cudaStream_t st, int num_sms, int ksplit) {
    using C = TcCfg<BN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    long long tiles = (long long)((Mmax + TC_BM - 1) / TC_BM) * (N / BN) * ksplit;
    int grid = (int)(tiles < num_sms ? tiles : num_sms);
    if (grid < 1) grid = 1;
    k_gemm_tc<BN, EPI><<<grid, TC_THREADS, C::SMEM, st>>>(ta, tb, tcm, trm, bias, R, Cout, counters, u_slot, N, K,
                                                          a_lo_row, c_lo_row, status, ksplit);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_epi(int BN, const CUtensorMap& ta, const CUtensorMap& tb, const CUtensorMap& tcm,
                       const CUtensorMap& trm, const float* bias, const float* R, void* Cout, const int* counters,
                       int u_slot, int Mmax, int N, int K, int a_lo_row, int c_lo_row, int* status, cudaStream_t st,
                       int num_sms, int ksplit) {
#define VQ_BN(B)                                                                                                   \
    launch_bn<B, EPI>(ta, tb, tcm, trm, bias, R, Cout, counters, u_slot, Mmax, N, K, a_lo_row, c_lo_row, status, st, \
                      num_sms, ksplit)
    switch (BN) {
        case 64: return VQ_BN(64);
        case 128: return VQ_BN(128);
        case 192: return VQ_BN(192);
        case 256: return VQ_BN(256);
        default: return cudaErrorInvalidValue;
    }
#undef VQ_BN
}

// Output (and residual) maps: [rows][cols] row-major, boxes of 32 x 32 elements, the
// 64-byte swizzle for BF16 rows of a box (64 bytes), the 128-byte one for FP32 (128 bytes).
cudaError_t make_tmap_out(CUtensorMap* map, const void* base, long long rows, int cols, bool f32) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const int es = f32 ? 4 : 2;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (cols * es) % 16 || rows < 1) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * es};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    f32 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_splitk_add(const float* part, int ksplit, long long Mpad, int M, int N, float* C, cudaStream_t st,
                              int num_sms) {
    const long long total = (long long)M * N;
    long long g = (total + 255) / 256;
    if (g > 8LL * num_sms) g = 8LL * num_sms;
    k_splitk_add<<<(int)(g > 0 ? g : 1), 256, 0, st>>>(part, ksplit, Mpad, M, N, C);
    return cudaGetLastError();
}

cudaError_t launch_set_int(int* p, int v, cudaStream_t st) {
    k_set_int<<<1, 1, 0, st>>>(p, v);
    return cudaGetLastError();
}

int tc_pick_bn(int N) {
    if (N % 256 == 0) return 256;
    if (N % 192 == 0) return 192;
    if (N % 128 == 0) return 128;
    if (N % 64 == 0) return 64;
    return 0;
}

cudaError_t make_tmap_bf16(CUtensorMap* map, const void* base, long long rows, int cols, int box_rows) {
    return make_tmap_bf16_strided(map, base, rows, cols, cols, box_rows);
}

cudaError_t make_tmap_bf16_strided(CUtensorMap* map, const void* base, long long rows, long long cols, long long ld,
                                   int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16 || cols > ld) return cudaErrorInvalidValue;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_gemm_tc(const __nv_bfloat16* A, long long Arows, const CUtensorMap& tmB, const float* bias,
                           const float* R, void* Cout, const int* counters, int u_slot, int N, int K, int epi,
                           int* status, cudaStream_t st, int num_sms, int BN, bool split, long long a_inner,
                           int ksplit) {
    if (BN <= 0) BN = tc_pick_bn(N);
    if (!BN || N % BN || K % TC_BK || K <= 0 || epi < 0 || epi > 4 || (epi == 2 && !R)) return cudaErrorInvalidValue;
    if (ksplit < 1 || (ksplit > 1 && epi != 3)) return cudaErrorInvalidValue;  // split K: FP32 partial tiles
    {  // every split takes at least one K block
        const int KB = K / TC_BK;
        if (ksplit > KB) ksplit = KB;
        const int KBs = (KB + ksplit - 1) / ksplit;
        ksplit = (KB + KBs - 1) / KBs;
    }
    if (Arows < 1) return cudaSuccess;  // no rows to compute
    if (split && Arows > (1LL << 30)) return cudaErrorInvalidValue;
    // split: A (and a BF16 C) hold their lo plane Arows rows after the hi one
    const int a_lo_row = split ? (int)Arows : 0;
    const int c_lo_row = split && epi < 2 ? (int)Arows : 0;
    CUtensorMap ta, tcm, trm;
    // a_inner: A's stored row length when it is shorter than K (K blocks past it read zeros)
    cudaError_t e = a_inner > 0 ? make_tmap_bf16_strided(&ta, A, split ? 2 * Arows : Arows, a_inner, a_inner, TC_BM)
                                : make_tmap_bf16(&ta, A, split ? 2 * Arows : Arows, K, TC_BM);
    if (e != cudaSuccess) return e;
    const long long Mpad = (Arows + TC_BM - 1) / TC_BM * TC_BM;
    e = make_tmap_out(&tcm, Cout, ksplit > 1 ? ksplit * Mpad : (c_lo_row ? 2 * Arows : Arows), N, epi >= 2);
    if (e != cudaSuccess) return e;
    if (epi == 2) {
        e = make_tmap_out(&trm, R, Arows, N, true);
        if (e != cudaSuccess) return e;
    } else {
        trm = tcm;  // not read
    }
    const int Mmax = (int)Arows;
#define VQ_EPI(E) \
    launch_epi<E>(BN, ta, tmB, tcm, trm, bias, R, Cout, counters, u_slot, Mmax, N, K, a_lo_row, c_lo_row, status, st, \
                  num_sms, ksplit)
    switch (epi) {
        case 0: return VQ_EPI(0);
        case 1: return VQ_EPI(1);
        case 2: return VQ_EPI(2);
        case 3: return VQ_EPI(3);
        case 4: return VQ_EPI(4);
        default: return cudaErrorInvalidValue;
    }
#undef VQ_EPI
}

}  // namespace vq
