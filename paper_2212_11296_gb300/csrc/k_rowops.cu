// Row-wise per-location operations: LayerNorm, the quantized residual update and
// the weight-derived tables (Sec. 3.1 block, Sec. 3.2 per-location ops).
#include "vqnqs_internal.cuh"

namespace vq {

// One warp per row; d % 32 == 0 and d <= 1024 so each lane keeps d / 32 values.
template <int PER>
__device__ __forceinline__ void ln_row(const float (&x)[PER], int lane, int d, const float* __restrict__ g,
                                       const float* __restrict__ b, float (&y)[PER]) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) s += x[i];
    float mu = warp_sum(s) / d;
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < PER; ++i) { float t = x[i] - mu; v += t * t; }
    float rstd = rsqrtf(warp_sum(v) / d + LN_EPS);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        int k = lane + 32 * i;
        y[i] = (x[i] - mu) * rstd * g[k] + b[k];
    }
}

// BF16 value of y at out[o] and, when lo_off > 0, the BF16 rounding of its
// remainder y - bf16(y) at out[lo_off + o] (the split-operand lo plane).
__device__ __forceinline__ void store_bf16_split(__nv_bfloat16* __restrict__ out, size_t o, size_t lo_off, float y) {
    const __nv_bfloat16 h = __float2bfloat16_rn(y);
    out[o] = h;
    if (lo_off) out[lo_off + o] = __float2bfloat16_rn(y - __bfloat162float(h));
}

template <int PER>
__global__ void k_layernorm(const float* __restrict__ X, const int* __restrict__ counters, int u_slot,
                            const float* __restrict__ g, const float* __restrict__ b, int d,
                            float* __restrict__ out_f32, __nv_bfloat16* __restrict__ out_bf16, size_t lo_off) {
    const int U = counters[u_slot];
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < U; u += gridDim.x * wpb) {
        float x[PER], y[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) x[i] = X[(size_t)u * d + lane + 32 * i];
        ln_row<PER>(x, lane, d, g, b, y);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            size_t o = (size_t)u * d + lane + 32 * i;
            if (out_f32) out_f32[o] = y[i];
            if (out_bf16) store_bf16_split(out_bf16, o, lo_off, y[i]);
        }
    }
}

// y = x[rep_uid] + T[rep_code]  (T = codebook @ W_o + b_o), then A = LN2(y).
// With H quantizer heads the code packs c_h in bits [h * bits, (h + 1) * bits)
// and T holds one table per head (b_o in head 0's): y = x + sum_h T_h[c_h].
// Two-word codes (tab_lo given): rep_code is a code id whose words are
// tab_lo[id] (heads 0 .. hpw-1) and tab_hi[id] (the rest), hpw = 32 / bits.
template <int PER>
__global__ void k_residual_vq_ln(const float* __restrict__ X, const int* __restrict__ rep_uid,
                                 const int* __restrict__ rep_code, const float* __restrict__ T,
                                 const int* __restrict__ counters, int u_slot, const float* __restrict__ g,
                                 const float* __restrict__ b, int d, float* __restrict__ Y,
                                 float* __restrict__ A_f32, __nv_bfloat16* __restrict__ A_bf16, int vq_heads, int K,
                                 int bits, size_t lo_off, const int* __restrict__ tab_lo,
                                 const int* __restrict__ tab_hi) {
    const int U = counters[u_slot];
    const int mask = vq_heads == 1 ? -1 : (1 << bits) - 1;
    const int hpw = bits > 0 ? 32 / bits : 1;
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < U; u += gridDim.x * wpb) {
        const float* x = X + (size_t)rep_uid[u] * d;
        const int code = tab_lo ? tab_lo[rep_code[u]] : rep_code[u];
        const int code_hi = tab_lo ? tab_hi[rep_code[u]] : 0;
        const float* t = T + (size_t)(code & mask) * d;
        float y[PER], a[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) y[i] = t[lane + 32 * i];
        for (int h = 1; h < vq_heads; ++h) {
            const int wd = h / hpw, f = h - wd * hpw;
            const float* th = T + ((size_t)h * K + (((wd ? code_hi : code) >> (f * bits)) & mask)) * d;
#pragma unroll
            for (int i = 0; i < PER; ++i) y[i] += th[lane + 32 * i];
        }
#pragma unroll
        for (int i = 0; i < PER; ++i) y[i] = x[lane + 32 * i] + y[i];
        ln_row<PER>(y, lane, d, g, b, a);
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            size_t o = (size_t)u * d + lane + 32 * i;
            Y[o] = y[i];
            if (A_f32) A_f32[o] = a[i];
            if (A_bf16) store_bf16_split(A_bf16, o, lo_off, a[i]);
        }
    }
}

// Per quantizer head h and codeword j (codebook [H][K][d / H]):
// T_h[j] = W_h,j @ w_o[rows h * d / H ..] (+ b_o for h = 0) and cnorm_h[j] = ||W_h,j||^2,
// one block per (h, j).  With one head: T[j] = W_j @ w_o + b_o.
__global__ void k_table_T(const float* __restrict__ cb, const float* __restrict__ wo, const float* __restrict__ bo,
                          int K, int d, int vq_heads, float* __restrict__ T, float* __restrict__ cnorm) {
    extern __shared__ float s_w[];
    const int dq = d / vq_heads;
    for (int hj = blockIdx.x; hj < vq_heads * K; hj += gridDim.x) {
        const int h = hj / K;
        for (int k = threadIdx.x; k < dq; k += blockDim.x) s_w[k] = cb[(size_t)hj * dq + k];
        __syncthreads();
        for (int n = threadIdx.x; n < d; n += blockDim.x) {
            float acc = 0.f;
            for (int k = 0; k < dq; ++k) acc = fmaf(s_w[k], wo[((size_t)h * dq + k) * d + n], acc);
            T[(size_t)hj * d + n] = h == 0 ? acc + bo[n] : acc;
        }
        if (threadIdx.x == 0) {
            float s = 0.f;
            for (int k = 0; k < dq; ++k) s = fmaf(s_w[k], s_w[k], s);
            cnorm[hj] = s;
        }
        __syncthreads();
    }
}

// WT[c][r] = bf16(W[r][c]); with lo, also the split lo plane WT[cols + c][r] = bf16(W[r][c] - WT[c][r])
__global__ void k_transpose_bf16(const float* __restrict__ W, int rows, int cols, __nv_bfloat16* __restrict__ WT,
                                 int lo) {
    __shared__ float tile[32][33];
    for (int by = blockIdx.y; by * 32 < rows; by += gridDim.y)
        for (int bx = blockIdx.x; bx * 32 < cols; bx += gridDim.x) {
            int r = by * 32 + threadIdx.y, c = bx * 32 + threadIdx.x;
            tile[threadIdx.y][threadIdx.x] = (r < rows && c < cols) ? W[(size_t)r * cols + c] : 0.f;
            __syncthreads();
            int r2 = by * 32 + threadIdx.x, c2 = bx * 32 + threadIdx.y;
            if (r2 < rows && c2 < cols) {
                const float x = tile[threadIdx.x][threadIdx.y];
                const __nv_bfloat16 h = __float2bfloat16_rn(x);
                WT[(size_t)c2 * rows + r2] = h;
                if (lo) WT[((size_t)cols + c2) * rows + r2] = __float2bfloat16_rn(x - __bfloat162float(h));
            }
            __syncthreads();
        }
}

// dst[r][c] = bf16(src[r][c]) (hi plane), dst[plane_rows + r][c] = bf16(src[r][c] - hi) (lo plane)
__global__ void k_split_planes(const float* __restrict__ src, long long n, int cols, __nv_bfloat16* __restrict__ dst,
                               long long lo_off) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float x = src[i];
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        dst[i] = h;
        dst[lo_off + i] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// every d_model the context accepts: 32 .. 1024 in steps of 32
#define VQ_DISPATCH_PER(d, KERNEL, ...)                                 \
    switch ((d) / 32) {                                                 \
        case 1: KERNEL<1><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 2: KERNEL<2><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 3: KERNEL<3><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 4: KERNEL<4><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 5: KERNEL<5><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 6: KERNEL<6><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 7: KERNEL<7><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 8: KERNEL<8><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 9: KERNEL<9><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 10: KERNEL<10><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 11: KERNEL<11><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 12: KERNEL<12><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 13: KERNEL<13><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 14: KERNEL<14><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 15: KERNEL<15><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 16: KERNEL<16><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 17: KERNEL<17><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 18: KERNEL<18><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 19: KERNEL<19><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 20: KERNEL<20><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 21: KERNEL<21><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 22: KERNEL<22><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 23: KERNEL<23><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 24: KERNEL<24><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 25: KERNEL<25><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 26: KERNEL<26><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 27: KERNEL<27><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 28: KERNEL<28><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 29: KERNEL<29><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 30: KERNEL<30><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 31: KERNEL<31><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        case 32: KERNEL<32><<<grid, 256, 0, st>>>(__VA_ARGS__); break; \
        default: return cudaErrorInvalidValue;                          \
    }

cudaError_t launch_layernorm(const float* X, const int* counters, int u_slot, const float* g, const float* b, int d,
                             float* out_f32, __nv_bfloat16* out_bf16, cudaStream_t st, int grid, size_t lo_off) {
    VQ_DISPATCH_PER(d, k_layernorm, X, counters, u_slot, g, b, d, out_f32, out_bf16, lo_off);
    return cudaGetLastError();
}

cudaError_t launch_residual_vq_ln(const float* X, const int* rep_uid, const int* rep_code, const float* T,
                                  const int* counters, int u_slot, const float* g, const float* b, int d, float* Y,
                                  float* A_f32, __nv_bfloat16* A_bf16, cudaStream_t st, int grid, int vq_heads, int K,
                                  int bits, size_t lo_off, const int* tab_lo, const int* tab_hi) {
    VQ_DISPATCH_PER(d, k_residual_vq_ln, X, rep_uid, rep_code, T, counters, u_slot, g, b, d, Y, A_f32, A_bf16,
                    vq_heads, K, bits, lo_off, tab_lo, tab_hi);
    return cudaGetLastError();
}

cudaError_t launch_table_T(const float* codebook, const float* w_o, const float* b_o, int K, int d, int vq_heads,
                           float* T, float* cnorm, cudaStream_t st) {
    if (vq_heads < 1 || d % vq_heads) return cudaErrorInvalidValue;
    int grid = vq_heads * K < 1024 ? vq_heads * K : 1024;
    k_table_T<<<grid, 256, d * sizeof(float), st>>>(codebook, w_o, b_o, K, d, vq_heads, T, cnorm);
    return cudaGetLastError();
}

cudaError_t launch_split_planes(const float* src, long long rows, int cols, __nv_bfloat16* dst, long long plane_rows,
                                cudaStream_t st, int cap) {
    const long long n = rows * cols;
    long long g = (n + 255) / 256;
    if (g > cap) g = cap;
    k_split_planes<<<(int)(g < 1 ? 1 : g), 256, 0, st>>>(src, n, cols, dst, plane_rows * cols);
    return cudaGetLastError();
}

cudaError_t launch_transpose_bf16(const float* W, int rows, int cols, __nv_bfloat16* WT, cudaStream_t st, bool lo) {
    dim3 grid((cols + 31) / 32 < 1024 ? (cols + 31) / 32 : 1024, (rows + 31) / 32 < 1024 ? (rows + 31) / 32 : 1024);
    k_transpose_bf16<<<grid, dim3(32, 32), 0, st>>>(W, rows, cols, WT, lo ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace vq
