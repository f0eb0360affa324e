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
// Inputs per row: QKV [R][3d] and dO [R][d].  The query-side kernel recomputes
// each row's softmax statistics (m_p, l_p) and D_p = dO_p . O_p, stores them in
// stat [R][H][3] and accumulates dQ_p = scale sum_{j<=p} dS_pj K_j; the key-side
// kernel then accumulates dK_j = scale sum_{p>=j} dS_pj Q_p and
// dV_j = sum_{p>=j} P_pj dO_p, with dS_pj = P_pj (dO_p . V_j - D_p).
__device__ __forceinline__ void attn_bwd_stage(const float* __restrict__ QKV, const float* __restrict__ dO,
                                               size_t r0, int N, int d, int h, int DH, float* sQ, float* sK,
                                               float* sV, float* sdO) {
    const int ld = 3 * d;
    for (int e = threadIdx.x; e < N * DH; e += blockDim.x) {
        const int j = e / DH, t = e - j * DH;
        const float* src = QKV + (r0 + j) * ld + h * DH + t;
        sQ[e] = src[0];
        sK[e] = src[d];
        sV[e] = src[2 * d];
        sdO[e] = dO[(r0 + j) * d + h * DH + t];
    }
}

template <int DH>
__global__ void __launch_bounds__(512) k_attention_bwd_q(const float* __restrict__ QKV, const float* __restrict__ dO,
                                                         int S, int N, int d, int H, float* __restrict__ dQKV,
                                                         float* __restrict__ stat) {
    extern __shared__ __align__(16) float sm[];
    float *sQ = sm, *sK = sQ + (size_t)N * DH, *sV = sK + (size_t)N * DH, *sdO = sV + (size_t)N * DH;
    const float scale = rsqrtf((float)DH);
    for (int item = blockIdx.x; item < S * H; item += gridDim.x) {
        const int b = item / H, h = item - b * H;
        const size_t r0 = (size_t)b * N;
        attn_bwd_stage(QKV, dO, r0, N, d, h, DH, sQ, sK, sV, sdO);
        __syncthreads();
        const int p = threadIdx.x;
        if (p < N) {
            float m = -INFINITY, l = 0.f, acc[DH];
#pragma unroll
            for (int t = 0; t < DH; ++t) acc[t] = 0.f;
            for (int j = 0; j <= p; ++j) {
                float s = 0.f;
#pragma unroll
                for (int t = 0; t < DH; ++t) s = fmaf(sQ[p * DH + t], sK[j * DH + t], s);
                s *= scale;
                const float mn = fmaxf(m, s);
                const float corr = expf(m - mn), e = expf(s - mn);
                l = l * corr + e;
#pragma unroll
                for (int t = 0; t < DH; ++t) acc[t] = fmaf(e, sV[j * DH + t], acc[t] * corr);
                m = mn;
            }
            float Dp = 0.f;
#pragma unroll
            for (int t = 0; t < DH; ++t) Dp = fmaf(sdO[p * DH + t], acc[t] / l, Dp);
            float* so = stat + ((r0 + p) * H + h) * 3;
            so[0] = m; so[1] = l; so[2] = Dp;
            float dq[DH];
#pragma unroll
            for (int t = 0; t < DH; ++t) dq[t] = 0.f;
            for (int j = 0; j <= p; ++j) {
                float s = 0.f, dp = 0.f;
#pragma unroll
                for (int t = 0; t < DH; ++t) {
                    s = fmaf(sQ[p * DH + t], sK[j * DH + t], s);
                    dp = fmaf(sdO[p * DH + t], sV[j * DH + t], dp);
                }
                const float P = expf(s * scale - m) / l;
                const float dS = P * (dp - Dp);
#pragma unroll
                for (int t = 0; t < DH; ++t) dq[t] = fmaf(dS, sK[j * DH + t], dq[t]);
            }
            float* dst = dQKV + (r0 + p) * (size_t)(3 * d) + h * DH;
#pragma unroll
            for (int t = 0; t < DH; ++t) dst[t] = dq[t] * scale;
        }
        __syncthreads();
    }
}

template <int DH>
__global__ void __launch_bounds__(512) k_attention_bwd_kv(const float* __restrict__ QKV, const float* __restrict__ dO,
                                                          int S, int N, int d, int H, float* __restrict__ dQKV,
                                                          const float* __restrict__ stat) {
    extern __shared__ __align__(16) float sm[];
    float *sQ = sm, *sK = sQ + (size_t)N * DH, *sV = sK + (size_t)N * DH, *sdO = sV + (size_t)N * DH;
    float *sM = sdO + (size_t)N * DH, *sL = sM + N, *sD = sL + N;
    const float scale = rsqrtf((float)DH);
    for (int item = blockIdx.x; item < S * H; item += gridDim.x) {
        const int b = item / H, h = item - b * H;
        const size_t r0 = (size_t)b * N;
        attn_bwd_stage(QKV, dO, r0, N, d, h, DH, sQ, sK, sV, sdO);
        for (int p = threadIdx.x; p < N; p += blockDim.x) {
            const float* si = stat + ((r0 + p) * H + h) * 3;
            sM[p] = si[0]; sL[p] = si[1]; sD[p] = si[2];
        }
        __syncthreads();
        const int j = threadIdx.x;
        if (j < N) {
            float dk[DH], dv[DH];
#pragma unroll
            for (int t = 0; t < DH; ++t) { dk[t] = 0.f; dv[t] = 0.f; }
            for (int q = j; q < N; ++q) {
                float s = 0.f, dp = 0.f;
#pragma unroll
                for (int t = 0; t < DH; ++t) {
                    s = fmaf(sQ[q * DH + t], sK[j * DH + t], s);
                    dp = fmaf(sdO[q * DH + t], sV[j * DH + t], dp);
                }
                const float P = expf(s * scale - sM[q]) / sL[q];
                const float dS = P * (dp - sD[q]);
#pragma unroll
                for (int t = 0; t < DH; ++t) {
                    dk[t] = fmaf(dS, sQ[q * DH + t], dk[t]);
                    dv[t] = fmaf(P, sdO[q * DH + t], dv[t]);
                }
            }
            float* dst = dQKV + (r0 + j) * (size_t)(3 * d) + h * DH;
#pragma unroll
            for (int t = 0; t < DH; ++t) {
                dst[d + t] = dk[t] * scale;
                dst[2 * d + t] = dv[t];
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
cudaError_t launch_attention_bwd(const float* QKV, const float* dO, int S, int N, int d, int H, float* dQKV,
                                 float* stat, cudaStream_t st, int cap) {
    const int DH = d / H;
    const int threads = ((N + 31) / 32) * 32;
    const size_t smem = ((size_t)4 * N * DH + 3 * N) * sizeof(float);
    if (threads > 512 || smem > 227 * 1024) return cudaErrorInvalidValue;
    const int grid = g_grid((long long)S * H, 1, cap);
    static size_t granted[3] = {};
    switch (DH) {
#define VQ_ABWD(X)                                                                                           \
    case X:                                                                                                  \
        if (smem > granted[X / 16]) {                                                                        \
            cudaFuncSetAttribute(k_attention_bwd_q<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            cudaFuncSetAttribute(k_attention_bwd_kv<X>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);\
            granted[X / 16] = smem;                                                                          \
        }                                                                                                    \
        k_attention_bwd_q<X><<<grid, threads, smem, st>>>(QKV, dO, S, N, d, H, dQKV, stat);                  \
        k_attention_bwd_kv<X><<<grid, threads, smem, st>>>(QKV, dO, S, N, d, H, dQKV, stat);                 \
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
