// Hand-written backward of log psi (Sec. 2 gradient estimator; Sec. 3.1,
// Eq. st straight-through quantizer), FP32 on CUDA cores.  Row-wise pieces;
// the contractions (dX = dY W^T, dW = X^T dY) run in k_gemm_f32_gen.cu.
#include "vqnqs_internal.cuh"

namespace vq {

// ---- head: d/dx of 1/2 log_softmax(LN_f(x) W_h + b_h)[s_p], scaled by the sample's seed ----
// Writes dX (grad wrt x_L), A_f = LN_f(x) and dlogits for dW_h / db_h, and
// da_f * xhat (for d lnf_g) and da_f (for d lnf_b).
__global__ void k_head_bwd(const float* __restrict__ X, const uint8_t* __restrict__ spins, const float* __restrict__ seed,
                           int R, int N, int d, const float* __restrict__ g, const float* __restrict__ bta,
                           const float* __restrict__ w, const float* __restrict__ bh, float* __restrict__ dX,
                           float* __restrict__ Af, float* __restrict__ dlog, float* __restrict__ dgam,
                           float* __restrict__ dbet) {
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < R; r += gridDim.x * wpb) {
        const float* x = X + (size_t)r * d;
        float s = 0.f;
        for (int k = lane; k < d; k += 32) s += x[k];
        const float mu = warp_sum(s) / d;
        float v = 0.f;
        for (int k = lane; k < d; k += 32) { float t = x[k] - mu; v += t * t; }
        const float rstd = rsqrtf(warp_sum(v) / d + LN_EPS);
        float z0 = 0.f, z1 = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float a = (x[k] - mu) * rstd * g[k] + bta[k];
            Af[(size_t)r * d + k] = a;
            z0 += a * w[2 * k];
            z1 += a * w[2 * k + 1];
        }
        z0 = warp_sum(z0) + bh[0];
        z1 = warp_sum(z1) + bh[1];
        const float m = fmaxf(z0, z1);
        const float e0 = expf(z0 - m), e1 = expf(z1 - m);
        const float p0 = e0 / (e0 + e1), p1 = e1 / (e0 + e1);
        const int b = r / N;
        const int sp = spins[r] & 1;  // spins are [samples][N], row r = b * N + p
        const float sc = 0.5f * (seed ? seed[b] : 1.f);
        const float d0 = sc * ((sp == 0 ? 1.f : 0.f) - p0), d1 = sc * ((sp == 1 ? 1.f : 0.f) - p1);
        if (lane == 0) { dlog[2 * (size_t)r] = d0; dlog[2 * (size_t)r + 1] = d1; }
        // LN_f backward
        float sdx = 0.f, sdxx = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float xh = (x[k] - mu) * rstd;
            const float da = d0 * w[2 * k] + d1 * w[2 * k + 1];
            const float dxh = da * g[k];
            sdx += dxh;
            sdxx += dxh * xh;
            dgam[(size_t)r * d + k] = da * xh;
            dbet[(size_t)r * d + k] = da;
        }
        sdx = warp_sum(sdx) / d;
        sdxx = warp_sum(sdxx) / d;
        for (int k = lane; k < d; k += 32) {
            const float xh = (x[k] - mu) * rstd;
            const float dxh = (d0 * w[2 * k] + d1 * w[2 * k + 1]) * g[k];
            dX[(size_t)r * d + k] = rstd * (dxh - sdx - xh * sdxx);
        }
    }
}

// ---- LayerNorm backward: dx (+)= d LN(x)/dx applied to da; da*xhat -> dgam, da -> dbet ----
__global__ void k_ln_bwd(const float* __restrict__ X, const float* __restrict__ dA, const float* __restrict__ g, int R,
                         int d, float* __restrict__ dX, int accumulate, float* __restrict__ dgam,
                         float* __restrict__ dbet) {
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < R; r += gridDim.x * wpb) {
        const float* x = X + (size_t)r * d;
        const float* da = dA + (size_t)r * d;
        float s = 0.f;
        for (int k = lane; k < d; k += 32) s += x[k];
        const float mu = warp_sum(s) / d;
        float v = 0.f;
        for (int k = lane; k < d; k += 32) { float t = x[k] - mu; v += t * t; }
        const float rstd = rsqrtf(warp_sum(v) / d + LN_EPS);
        float sdx = 0.f, sdxx = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float xh = (x[k] - mu) * rstd;
            const float dxh = da[k] * g[k];
            sdx += dxh;
            sdxx += dxh * xh;
            dgam[(size_t)r * d + k] = da[k] * xh;
            dbet[(size_t)r * d + k] = da[k];
        }
        sdx = warp_sum(sdx) / d;
        sdxx = warp_sum(sdxx) / d;
        for (int k = lane; k < d; k += 32) {
            const float xh = (x[k] - mu) * rstd;
            const float val = rstd * (da[k] * g[k] - sdx - xh * sdxx);
            dX[(size_t)r * d + k] = accumulate ? dX[(size_t)r * d + k] + val : val;
        }
    }
}

// dH = dG * GELU'(H) (erf form), in place on dG
__global__ void k_gelu_bwd(const float* __restrict__ H, float* __restrict__ dG, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float h = H[i];
        const float cdf = 0.5f * (1.f + erff(h * 0.70710678118654752f));
        const float pdf = 0.3989422804014327f * expf(-0.5f * h * h);
        dG[i] *= cdf + h * pdf;
    }
}

// GELU forward for the recomputation: G = GELU(H)
__global__ void k_gelu_fwd(const float* __restrict__ H, float* __restrict__ G, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float h = H[i];
        G[i] = 0.5f * h * (1.f + erff(h * 0.70710678118654752f));
    }
}

// ---- straight-through quantizer (Eq. st), per row --------------------------------
// Inputs: OW[r][j] = o . W_j, DG[r][j] = W_j . dV (dV = grad wrt the quantized vector),
// osq[r] = ||o||^2, cnorm[j] = ||W_j||^2.  With n_j = ||o - W_j||, D = -n,
// s = softmax(D), dD_j = s_j (DG_j - sum_k s_k DG_k); the gradient wrt o is
// sum_j dD_j (-(o - W_j) / n_j) = -(sum_j a_j) o + sum_j a_j W_j with a_j = dD_j / n_j,
// and wrt W_j it is a_j (o - W_j).  Writes alpha[r][j] = a_j and arow[r] = sum_j a_j.
// One warp per row; D values staged in shared memory (K <= 4096).
__global__ void k_st_rows(const float* __restrict__ OW, const float* __restrict__ DG, const float* __restrict__ O,
                          const float* __restrict__ cnorm, int R, int K, int d, float* __restrict__ alpha,
                          float* __restrict__ arow) {
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < R; r += gridDim.x * wpb) {
        const float* o = O + (size_t)r * d;
        float q = 0.f;
        for (int k = lane; k < d; k += 32) q += o[k] * o[k];
        const float osq = warp_sum(q);
        const float* ow = OW + (size_t)r * K;
        const float* dg = DG + (size_t)r * K;
        float mx = -INFINITY;
        for (int j = lane; j < K; j += 32) {
            const float n = sqrtf(fmaxf(osq - 2.f * ow[j] + cnorm[j], 0.f));
            mx = fmaxf(mx, -n);
        }
#pragma unroll
        for (int o2 = 16; o2 > 0; o2 >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o2));
        float se = 0.f, sdg = 0.f;
        for (int j = lane; j < K; j += 32) {
            const float n = sqrtf(fmaxf(osq - 2.f * ow[j] + cnorm[j], 0.f));
            const float e = expf(-n - mx);
            se += e;
            sdg += e * dg[j];
        }
        se = warp_sum(se);
        sdg = warp_sum(sdg) / se;  // sum_k s_k DG_k
        float asum = 0.f;
        for (int j = lane; j < K; j += 32) {
            const float n = sqrtf(fmaxf(osq - 2.f * ow[j] + cnorm[j], 0.f));
            const float s = expf(-n - mx) / se;
            const float dD = s * (dg[j] - sdg);
            const float a = n > 1e-30f ? dD / n : 0.f;
            alpha[(size_t)r * K + j] = a;
            asum += a;
        }
        asum = warp_sum(asum);
        if (lane == 0) arow[r] = asum;
    }
}

// dO[r] = -arow[r] * O[r] + AW[r]  (AW = alpha @ W, computed by a GEMM into dO beforehand)
__global__ void k_st_do(const float* __restrict__ O, const float* __restrict__ arow, int R, int d,
                        float* __restrict__ dO) {
    const size_t n = (size_t)R * d;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dO[i] = dO[i] - arow[i / d] * O[i];
}

// One-hot rows of the chosen codes (for d codebook[c] += dV by a GEMM)
__global__ void k_onehot(const int* __restrict__ code, int R, int K, float* __restrict__ H) {
    const size_t n = (size_t)R * K;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        H[i] = (code[i / K] == (int)(i % K)) ? 1.f : 0.f;
}

// Y = X + T[code] and V = codebook[code] (recomputation of the quantized residual)
__global__ void k_quant_residual(const float* __restrict__ X, const int* __restrict__ code, const float* __restrict__ T,
                                 const float* __restrict__ cb, int R, int d, float* __restrict__ Y,
                                 float* __restrict__ V) {
    const size_t n = (size_t)R * d;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const size_t r = i / d, k = i - r * d;
        const int c = code[r];
        Y[i] = X[i] + T[(size_t)c * d + k];
        V[i] = cb[(size_t)c * d + k];
    }
}

// Column sums over row groups: out[z][n] (+)= sum_{rows r of group z} X[r][n]; groups of G rows.
__global__ void k_colsum(const float* __restrict__ X, int rows, int G, int ncol, float* __restrict__ out,
                         long long out_stride, int accumulate) {
    const int groups = (rows + G - 1) / G;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)groups * ncol;
         t += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(t / ncol), n = (int)(t - (long long)z * ncol);
        const int r1 = min(rows, (z + 1) * G);
        float s = 0.f;
        for (int r = z * G; r < r1; ++r) s += X[(size_t)r * ncol + n];
        float* o = out + z * out_stride + n;
        *o = accumulate ? *o + s : s;
    }
}

// The same for one group of many rows, in two fixed-order stages: block (x, y) sums its 32
// columns over row slab y (8 row lanes, coalesced 128-byte row segments) into part[y][n];
// then out[n] (+)= sum over the slabs in slab order.
__global__ void k_colsum_slabs(const float* __restrict__ X, int rows, int ncol, int slab, float* __restrict__ part) {
    __shared__ float red[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    const int r0 = blockIdx.y * slab, r1 = min(rows, r0 + slab);
    float s = 0.f;
    if (n < ncol)
        for (int r = r0 + threadIdx.y; r < r1; r += 8) s += X[(size_t)r * ncol + n];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < ncol) {
        float t = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        part[(size_t)blockIdx.y * ncol + n] = t;
    }
}
__global__ void k_colsum_finish(const float* __restrict__ part, int slabs, int ncol, float* __restrict__ out,
                                int accumulate) {
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < ncol; n += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int y = 0; y < slabs; ++y) s += part[(size_t)y * ncol + n];
        out[n] = accumulate ? out[n] + s : s;
    }
}

// Embedding backward: dtok[t] (+)= sum of dX0 rows with token t; dpos[p] (+)= sum over the
// group's samples of dX0[b][p].  Groups of G samples (G = all samples for the summed
// gradient, G = 1 for per-sample gradients).
__global__ void k_embed_bwd(const float* __restrict__ dX0, const uint8_t* __restrict__ spins, int S, int N, int d,
                            int G, float* __restrict__ dtok, float* __restrict__ dpos, long long out_stride,
                            int accumulate) {
    const int groups = (S + G - 1) / G;
    const long long items = (long long)groups * (3 + N) * d;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < items; t += (long long)gridDim.x * blockDim.x) {
        const int z = (int)(t / ((3 + N) * d));
        const int rem = (int)(t - (long long)z * (3 + N) * d);
        const int row = rem / d, k = rem - row * d;
        const int b0 = z * G, b1 = min(S, b0 + G);
        float s = 0.f;
        float* o;
        if (row < 3) {  // token row: 0 down, 1 up, 2 begin-of-sequence
            for (int b = b0; b < b1; ++b)
                for (int p = 0; p < N; ++p) {
                    const int tok = p == 0 ? BOS : (spins[(size_t)b * N + p - 1] & 1);
                    if (tok == row) s += dX0[((size_t)b * N + p) * d + k];
                }
            o = dtok + z * out_stride + (size_t)row * d + k;
        } else {
            const int p = row - 3;
            for (int b = b0; b < b1; ++b) s += dX0[((size_t)b * N + p) * d + k];
            o = dpos + z * out_stride + (size_t)p * d + k;
        }
        *o = accumulate ? *o + s : s;
    }
}

// ---- causal attention backward, one CTA per (sample, head), FP32 ----------------
// Inputs per row: QKV [R][3d], the attention output O [R][d], dO [R][d] and the forward's
// softmax statistics stats [R][H] = (m_p, l_p) (maximum scaled score, sum of exp(s - m_p)).
// With P_pj = exp(s_pj - m_p) / l_p, s_pj = q_p . k_j / sqrt(dh), D_p = dO_p . O_p and
// dS_pj = P_pj (dO_p . v_j - D_p):
//   dQ_p = scale sum_{j<=p} dS_pj k_j            (query-side kernel, which also stores D_p)
//   dK_j = scale sum_{p>=j} dS_pj q_p,  dV_j = sum_{p>=j} P_pj dO_p   (key-side kernel).
// Two threads per row (or key), each holding half of the head's dims; a dot product is
// the pair's two halves added with one shuffle.  Every lane of a warp reads the same key
// (query-side) or the same query row (key-side) from shared memory in each step, so the
// reads are broadcasts; on the key side a warp walks the query rows from its first key
// with the rows before a lane's key masked.
constexpr int ABWD_THREADS = 512;  // 256 rows (or keys) per pass, two threads each

template <int DH>
__global__ void __launch_bounds__(ABWD_THREADS) k_attention_bwd_q(const float* __restrict__ QKV, const float* __restrict__ O,
                                                          const float* __restrict__ dO, const float2* __restrict__ stats,
                                                          int S, int N, int d, int H, float* __restrict__ dQKV,
                                                          float* __restrict__ Dst) {
    constexpr int HD = DH / 2;  // dims per thread
    extern __shared__ __align__(16) float sm[];
    float *sK = sm, *sV = sK + (size_t)N * DH;
    const float scale = rsqrtf((float)DH);
    const int ld = 3 * d;
    const int hf = threadIdx.x & 1;
    for (int item = blockIdx.x; item < S * H; item += gridDim.x) {
        const int b = item / H, h = item - b * H;
        const size_t r0 = (size_t)b * N;
        for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
            const int j = e / (DH / 4), t = (e - j * (DH / 4)) * 4;
            const float* src = QKV + (r0 + j) * ld + h * DH + t;
            *reinterpret_cast<float4*>(sK + j * DH + t) = *reinterpret_cast<const float4*>(src + d);
            *reinterpret_cast<float4*>(sV + j * DH + t) = *reinterpret_cast<const float4*>(src + 2 * d);
        }
        __syncthreads();
        for (int pb = 0; pb < N; pb += ABWD_THREADS / 2) {
        const int p = pb + (threadIdx.x >> 1);
        const bool act = p < N;
        const size_t row = r0 + (act ? p : 0);
        float q[HD], g[HD], dq[HD];
        float Dp = 0.f;
#pragma unroll
        for (int t = 0; t < HD; t += 4) {
            const float4 q4 = *reinterpret_cast<const float4*>(QKV + row * ld + h * DH + hf * HD + t);
            const float4 g4 = *reinterpret_cast<const float4*>(dO + row * d + h * DH + hf * HD + t);
            const float4 o4 = *reinterpret_cast<const float4*>(O + row * d + h * DH + hf * HD + t);
            q[t] = q4.x; q[t + 1] = q4.y; q[t + 2] = q4.z; q[t + 3] = q4.w;
            g[t] = g4.x; g[t + 1] = g4.y; g[t + 2] = g4.z; g[t + 3] = g4.w;
            Dp = fmaf(g4.x, o4.x, fmaf(g4.y, o4.y, fmaf(g4.z, o4.z, fmaf(g4.w, o4.w, Dp))));
            dq[t] = dq[t + 1] = dq[t + 2] = dq[t + 3] = 0.f;
        }
        Dp += __shfl_xor_sync(0xffffffffu, Dp, 1);
        const float2 ml = stats[row * H + h];
        const float il = 1.f / ml.y;
        // warp-uniform walk over the keys of the warp's last row; keys after a lane's row are masked
        const int pw = min(N - 1, pb + (int)((threadIdx.x | 31) >> 1));
        for (int j = 0; j <= pw; ++j) {
            const float* kj = sK + j * DH + hf * HD;
            const float* vj = sV + j * DH + hf * HD;
            float s = 0.f, dp = 0.f;
#pragma unroll
            for (int t = 0; t < HD; t += 4) {
                const float4 k4 = *reinterpret_cast<const float4*>(kj + t);
                const float4 v4 = *reinterpret_cast<const float4*>(vj + t);
                s = fmaf(q[t], k4.x, fmaf(q[t + 1], k4.y, fmaf(q[t + 2], k4.z, fmaf(q[t + 3], k4.w, s))));
                dp = fmaf(g[t], v4.x, fmaf(g[t + 1], v4.y, fmaf(g[t + 2], v4.z, fmaf(g[t + 3], v4.w, dp))));
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            dp += __shfl_xor_sync(0xffffffffu, dp, 1);
            const float P = (act && j <= p) ? __expf(s * scale - ml.x) * il : 0.f;
            const float dS = P * (dp - Dp);
#pragma unroll
            for (int t = 0; t < HD; t += 4) {
                const float4 k4 = *reinterpret_cast<const float4*>(kj + t);
                dq[t] = fmaf(dS, k4.x, dq[t]);
                dq[t + 1] = fmaf(dS, k4.y, dq[t + 1]);
                dq[t + 2] = fmaf(dS, k4.z, dq[t + 2]);
                dq[t + 3] = fmaf(dS, k4.w, dq[t + 3]);
            }
        }
        if (act) {
            float* dst = dQKV + row * (size_t)ld + h * DH + hf * HD;
#pragma unroll
            for (int t = 0; t < HD; t += 4)
                *reinterpret_cast<float4*>(dst + t) =
                    make_float4(dq[t] * scale, dq[t + 1] * scale, dq[t + 2] * scale, dq[t + 3] * scale);
            if (hf == 0) Dst[row * H + h] = Dp;
        }
        }
        __syncthreads();
    }
}

template <int DH>
__global__ void __launch_bounds__(ABWD_THREADS) k_attention_bwd_kv(const float* __restrict__ QKV, const float* __restrict__ dO,
                                                           const float2* __restrict__ stats,
                                                           const float* __restrict__ Dst, int S, int N, int d, int H,
                                                           float* __restrict__ dQKV) {
    constexpr int HD = DH / 2;
    extern __shared__ __align__(16) float sm[];
    float *sQ = sm, *sG = sQ + (size_t)N * DH;
    float *sM = sG + (size_t)N * DH, *sIL = sM + N, *sD = sIL + N;
    const float scale = rsqrtf((float)DH);
    const int ld = 3 * d;
    const int hf = threadIdx.x & 1;
    for (int item = blockIdx.x; item < S * H; item += gridDim.x) {
        const int b = item / H, h = item - b * H;
        const size_t r0 = (size_t)b * N;
        for (int e = threadIdx.x; e < N * (DH / 4); e += blockDim.x) {
            const int q = e / (DH / 4), t = (e - q * (DH / 4)) * 4;
            *reinterpret_cast<float4*>(sQ + q * DH + t) =
                *reinterpret_cast<const float4*>(QKV + (r0 + q) * ld + h * DH + t);
            *reinterpret_cast<float4*>(sG + q * DH + t) = *reinterpret_cast<const float4*>(dO + (r0 + q) * d + h * DH + t);
        }
        for (int q = threadIdx.x; q < N; q += blockDim.x) {
            const float2 ml = stats[(r0 + q) * H + h];
            sM[q] = ml.x;
            sIL[q] = 1.f / ml.y;
            sD[q] = Dst[(r0 + q) * H + h];
        }
        __syncthreads();
        for (int jb = 0; jb < N; jb += ABWD_THREADS / 2) {
        const int j = jb + (threadIdx.x >> 1);
        const int jw = jb + ((threadIdx.x & ~31) >> 1);  // the warp's first key
        const bool act = j < N;
        const size_t row = r0 + (act ? j : 0);
        float k[HD], v[HD], dk[HD], dv[HD];
#pragma unroll
        for (int t = 0; t < HD; t += 4) {
            const float4 k4 = *reinterpret_cast<const float4*>(QKV + row * ld + d + h * DH + hf * HD + t);
            const float4 v4 = *reinterpret_cast<const float4*>(QKV + row * ld + 2 * d + h * DH + hf * HD + t);
            k[t] = k4.x; k[t + 1] = k4.y; k[t + 2] = k4.z; k[t + 3] = k4.w;
            v[t] = v4.x; v[t + 1] = v4.y; v[t + 2] = v4.z; v[t + 3] = v4.w;
            dk[t] = dk[t + 1] = dk[t + 2] = dk[t + 3] = 0.f;
            dv[t] = dv[t + 1] = dv[t + 2] = dv[t + 3] = 0.f;
        }
        for (int q = jw; q < N; ++q) {  // warp-uniform walk; rows before this lane's key are masked
            const float* qq = sQ + q * DH + hf * HD;
            const float* gq = sG + q * DH + hf * HD;
            float s = 0.f, dp = 0.f;
#pragma unroll
            for (int t = 0; t < HD; t += 4) {
                const float4 q4 = *reinterpret_cast<const float4*>(qq + t);
                const float4 g4 = *reinterpret_cast<const float4*>(gq + t);
                s = fmaf(k[t], q4.x, fmaf(k[t + 1], q4.y, fmaf(k[t + 2], q4.z, fmaf(k[t + 3], q4.w, s))));
                dp = fmaf(v[t], g4.x, fmaf(v[t + 1], g4.y, fmaf(v[t + 2], g4.z, fmaf(v[t + 3], g4.w, dp))));
            }
            s += __shfl_xor_sync(0xffffffffu, s, 1);
            dp += __shfl_xor_sync(0xffffffffu, dp, 1);
            const bool vis = act && q >= j;
            const float P = vis ? __expf(s * scale - sM[q]) * sIL[q] : 0.f;
            const float dS = P * (dp - sD[q]);
#pragma unroll
            for (int t = 0; t < HD; t += 4) {
                const float4 q4 = *reinterpret_cast<const float4*>(qq + t);
                const float4 g4 = *reinterpret_cast<const float4*>(gq + t);
                dk[t] = fmaf(dS, q4.x, dk[t]);
                dk[t + 1] = fmaf(dS, q4.y, dk[t + 1]);
                dk[t + 2] = fmaf(dS, q4.z, dk[t + 2]);
                dk[t + 3] = fmaf(dS, q4.w, dk[t + 3]);
                dv[t] = fmaf(P, g4.x, dv[t]);
                dv[t + 1] = fmaf(P, g4.y, dv[t + 1]);
                dv[t + 2] = fmaf(P, g4.z, dv[t + 2]);
                dv[t + 3] = fmaf(P, g4.w, dv[t + 3]);
            }
        }
        if (act) {
            float* dst = dQKV + row * (size_t)ld + h * DH + hf * HD;
#pragma unroll
            for (int t = 0; t < HD; t += 4) {
                *reinterpret_cast<float4*>(dst + d + t) =
                    make_float4(dk[t] * scale, dk[t + 1] * scale, dk[t + 2] * scale, dk[t + 3] * scale);
                *reinterpret_cast<float4*>(dst + 2 * d + t) = make_float4(dv[t], dv[t + 1], dv[t + 2], dv[t + 3]);
            }
        }
        }
        __syncthreads();
    }
}

// ---- launchers -------------------------------------------------------------------
static int g_grid(long long items, int per_block, int cap) {
    long long g = (items + per_block - 1) / per_block;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

cudaError_t launch_head_bwd(const float* X, const uint8_t* spins, const float* seed, int R, int N, int d,
                            const float* g, const float* b, const float* w, const float* bh, float* dX, float* Af,
                            float* dlog, float* dgam, float* dbet, cudaStream_t st, int cap) {
    k_head_bwd<<<g_grid(R, 8, cap), 256, 0, st>>>(X, spins, seed, R, N, d, g, b, w, bh, dX, Af, dlog, dgam, dbet);
    return cudaGetLastError();
}
cudaError_t launch_ln_bwd(const float* X, const float* dA, const float* g, int R, int d, float* dX, int accumulate,
                          float* dgam, float* dbet, cudaStream_t st, int cap) {
    k_ln_bwd<<<g_grid(R, 8, cap), 256, 0, st>>>(X, dA, g, R, d, dX, accumulate, dgam, dbet);
    return cudaGetLastError();
}
cudaError_t launch_gelu_bwd(const float* H, float* dG, size_t n, cudaStream_t st, int cap) {
    k_gelu_bwd<<<g_grid((long long)n, 256, cap), 256, 0, st>>>(H, dG, n);
    return cudaGetLastError();
}
cudaError_t launch_gelu_fwd(const float* H, float* G, size_t n, cudaStream_t st, int cap) {
    k_gelu_fwd<<<g_grid((long long)n, 256, cap), 256, 0, st>>>(H, G, n);
    return cudaGetLastError();
}
cudaError_t launch_st_rows(const float* OW, const float* DG, const float* O, const float* cnorm, int R, int K, int d,
                           float* alpha, float* arow, cudaStream_t st, int cap) {
    k_st_rows<<<g_grid(R, 8, cap), 256, 0, st>>>(OW, DG, O, cnorm, R, K, d, alpha, arow);
    return cudaGetLastError();
}
cudaError_t launch_st_do(const float* O, const float* arow, int R, int d, float* dO, cudaStream_t st, int cap) {
    k_st_do<<<g_grid((long long)R * d, 256, cap), 256, 0, st>>>(O, arow, R, d, dO);
    return cudaGetLastError();
}
cudaError_t launch_onehot(const int* code, int R, int K, float* Hm, cudaStream_t st, int cap) {
    k_onehot<<<g_grid((long long)R * K, 256, cap), 256, 0, st>>>(code, R, K, Hm);
    return cudaGetLastError();
}
cudaError_t launch_quant_residual(const float* X, const int* code, const float* T, const float* cb, int R, int d,
                                  float* Y, float* V, cudaStream_t st, int cap) {
    k_quant_residual<<<g_grid((long long)R * d, 256, cap), 256, 0, st>>>(X, code, T, cb, R, d, Y, V);
    return cudaGetLastError();
}
cudaError_t launch_colsum(const float* X, int rows, int G, int ncol, float* out, long long out_stride, int accumulate,
                          cudaStream_t st, int cap, float* part, int part_cap) {
    const long long groups = (rows + G - 1) / G;
    if (groups == 1 && part && rows > 4096) {  // one long group: row slabs in parallel, then a fixed-order sum
        int slabs = (rows + 1023) / 1024;
        if ((long long)slabs * ncol > part_cap) slabs = part_cap / ncol;
        if (slabs > 1) {
            const int slab = (rows + slabs - 1) / slabs;
            slabs = (rows + slab - 1) / slab;
            k_colsum_slabs<<<dim3((ncol + 31) / 32, slabs), dim3(32, 8), 0, st>>>(X, rows, ncol, slab, part);
            k_colsum_finish<<<(ncol + 255) / 256, 256, 0, st>>>(part, slabs, ncol, out, accumulate);
            return cudaGetLastError();
        }
    }
    k_colsum<<<g_grid(groups * ncol, 256, cap), 256, 0, st>>>(X, rows, G, ncol, out, out_stride, accumulate);
    return cudaGetLastError();
}
cudaError_t launch_embed_bwd(const float* dX0, const uint8_t* spins, int S, int N, int d, int G, float* dtok,
                             float* dpos, long long out_stride, int accumulate, cudaStream_t st, int cap) {
    const long long groups = (S + G - 1) / G;
    k_embed_bwd<<<g_grid(groups * (3 + N) * d, 256, cap), 256, 0, st>>>(dX0, spins, S, N, d, G, dtok, dpos,
                                                                        out_stride, accumulate);
    return cudaGetLastError();
}
cudaError_t launch_attention_bwd(const float* QKV, const float* O, const float* dO, const float2* stats, int S, int N,
                                 int d, int H, float* dQKV, float* Dst, cudaStream_t st, int cap) {
    const int DH = d / H;
    const int threads = ABWD_THREADS;
    const size_t smem = ((size_t)2 * N * DH + 3 * N) * sizeof(float);
    if (smem > 227 * 1024 || DH % 8) return cudaErrorInvalidValue;
    const int grid = g_grid((long long)S * H, 1, cap);
    static size_t granted[3] = {};
    switch (DH) {
#define VQ_ABWD(X)                                                                                            \
    case X:                                                                                                   \
        if (smem > granted[X / 16]) {                                                                         \
            cudaFuncSetAttribute(k_attention_bwd_q<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
            cudaFuncSetAttribute(k_attention_bwd_kv<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            granted[X / 16] = smem;                                                                           \
        }                                                                                                     \
        k_attention_bwd_q<X><<<grid, threads, smem, st>>>(QKV, O, dO, stats, S, N, d, H, dQKV, Dst);          \
        k_attention_bwd_kv<X><<<grid, threads, smem, st>>>(QKV, dO, stats, Dst, S, N, d, H, dQKV);            \
        break;
        VQ_ABWD(8)
        VQ_ABWD(16)
        VQ_ABWD(32)
#undef VQ_ABWD
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vq
