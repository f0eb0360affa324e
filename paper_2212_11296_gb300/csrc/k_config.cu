// Connected-configuration enumeration, embedding, head and the local-energy
// assembly (Sec. 2 Eq. local-energy; Sec. 4 Heisenberg model, Marshall sign).
#include "vqnqs_internal.cuh"

namespace vq {

// ---- bonds: diagonal energy and anti-aligned count per sample ------------------
// Sec. 4: H = J sum_<ij> S_i.S_j.  In the Marshall-rotated S^z basis a bond gives
// (J/4) sigma_i sigma_j on the diagonal and -J/2 to the configuration with the
// two spins exchanged when they differ (Sec. 2: a k-local term touches only its
// own sites).
__global__ void k_count_configs(const uint8_t* __restrict__ spins, int S, int N, const int* __restrict__ bonds,
                                int nb, float J, int with_bonds, int* __restrict__ cnt, float* __restrict__ diag,
                                int* __restrict__ status) {
    __shared__ int s_red[2][32];
    for (int b = blockIdx.x; b < S; b += gridDim.x) {
        const uint8_t* s = spins + (size_t)b * N;
        int bad = 0;
        for (int p = threadIdx.x; p < N; p += blockDim.x) bad |= (s[p] > 1);
        int anti = 0, zz = 0;
        if (with_bonds) {
            for (int t = threadIdx.x; t < nb; t += blockDim.x) {
                int si = s[bonds[2 * t]] & 1, sj = s[bonds[2 * t + 1]] & 1;
                anti += (si != sj);
                zz += (si == sj) ? 1 : -1;
            }
        }
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, VQNQS_DEV_BAD_SPIN);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            anti += __shfl_xor_sync(0xffffffffu, anti, o);
            zz += __shfl_xor_sync(0xffffffffu, zz, o);
        }
        int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        if ((threadIdx.x & 31) == 0) { s_red[0][w] = anti; s_red[1][w] = zz; }
        __syncthreads();
        if (threadIdx.x == 0) {
            int a = 0, z = 0;
            for (int i = 0; i < nw; ++i) { a += s_red[0][i]; z += s_red[1][i]; }
            cnt[b] = a;
            diag[b] = 0.25f * J * (float)z;
        }
        __syncthreads();
    }
}

// Exclusive scan of (1 + anti-aligned count) over the chunk's samples; one block.
__global__ void k_scan_configs(const int* __restrict__ cnt, int S, int* __restrict__ cfg_off,
                               int* __restrict__ counters, int N) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < S; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = (i < S) ? 1 + cnt[i] : 0;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            int nw = blockDim.x >> 5;
            int t = (lane < nw) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) s_warp[lane] = t;
        }
        __syncthreads();
        int incl = x + (w > 0 ? s_warp[w - 1] : 0) + s_carry;
        if (i < S) cfg_off[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        cfg_off[S] = s_carry;
        counters[CNT_C] = s_carry;
        counters[CNT_R] = s_carry * N;
    }
}

// Writes the sample itself, then its anti-aligned bonds in bond order.
__global__ void k_fill_configs(const uint8_t* __restrict__ spins, int S, int N, const int* __restrict__ bonds,
                               int nb, int with_bonds, const int* __restrict__ cfg_off, int* __restrict__ cfg_sample,
                               int* __restrict__ cfg_i, int* __restrict__ cfg_j) {
    __shared__ int s_warp[32];
    for (int b = blockIdx.x; b < S; b += gridDim.x) {
        const uint8_t* s = spins + (size_t)b * N;
        int off = cfg_off[b];
        if (threadIdx.x == 0) { cfg_sample[off] = b; cfg_i[off] = -1; cfg_j[off] = -1; }
        if (!with_bonds) continue;
        int run = off + 1;
        for (int base = 0; base < nb; base += blockDim.x) {
            int t = base + threadIdx.x;
            int bi = 0, bj = 0, f = 0;
            if (t < nb) {
                bi = bonds[2 * t]; bj = bonds[2 * t + 1];
                f = ((s[bi] & 1) != (s[bj] & 1));
            }
            unsigned m = __ballot_sync(0xffffffffu, f);
            int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
            if (lane == 0) s_warp[w] = __popc(m);
            __syncthreads();
            int before = 0, total = 0;
            for (int i = 0; i < nw; ++i) { if (i < w) before += s_warp[i]; total += s_warp[i]; }
            if (f) {
                int c = run + before + __popc(m & ((1u << lane) - 1u));
                cfg_sample[c] = b; cfg_i[c] = bi; cfg_j[c] = bj;
            }
            run += total;
            __syncthreads();
        }
    }
}

// ---- active rows -------------------------------------------------------------------
__global__ void k_active_count(Chunk ch, int prefix_reuse, int* __restrict__ act_cnt) {
    const int C = ch.counters[CNT_C];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x)
        act_cnt[c] = ch.N - (prefix_reuse ? cfg_first_changed(ch.cfg_i[c], ch.cfg_j[c]) : 0);
}

// Exclusive scan of act_cnt over the chunk's configurations (one block); total -> CNT_A.
__global__ void k_active_scan(Chunk ch, const int* __restrict__ act_cnt, int* __restrict__ act_off) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    const int C = ch.counters[CNT_C];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < C; base += blockDim.x) {
        int i = base + threadIdx.x;
        int v = (i < C) ? act_cnt[i] : 0;
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            int nw = blockDim.x >> 5;
            int t = (lane < nw) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) s_warp[lane] = t;
        }
        __syncthreads();
        int incl = x + (w > 0 ? s_warp[w - 1] : 0) + s_carry;
        if (i < C) act_off[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) ch.counters[CNT_A] = s_carry;
}

// One warp per configuration writes its active rows (ascending).
__global__ void k_active_fill(Chunk ch, int prefix_reuse, const int* __restrict__ act_off,
                              int* __restrict__ act_rows) {
    const int C = ch.counters[CNT_C], N = ch.N;
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < C; c += gridDim.x * wpb) {
        const int p0 = prefix_reuse ? cfg_first_changed(ch.cfg_i[c], ch.cfg_j[c]) : 0;
        const int off = act_off[c];
        for (int p = p0 + lane; p < N; p += 32) act_rows[off + p - p0] = c * N + p;
    }
}

// ---- embedding: x0 = tok_emb[token] + pos_emb[p], token = s_{p-1} (BOS at p = 0) --------
// reuse: rows are keyed by (p, token) -> uid p * 3 + token, table of 3N rows.
// full:  every (config, position) row gets its own copy.
__global__ void k_embed_table(const float* __restrict__ tok_emb, const float* __restrict__ pos_emb, int N, int d,
                              float* __restrict__ X0) {
    size_t total = (size_t)3 * N * d;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(e % d);
        int u = (int)(e / d);
        int p = u / 3, t = u % 3;
        X0[e] = tok_emb[(size_t)t * d + k] + pos_emb[(size_t)p * d + k];
    }
}

__global__ void k_embed_rows(Chunk ch, const float* __restrict__ tok_emb, const float* __restrict__ pos_emb,
                             int reuse, float* __restrict__ X0, int* __restrict__ uid0) {
    const int N = ch.N, d = ch.d;
    const int R = ch.counters[CNT_R];
    // one warp per row
    int lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < R; r += gridDim.x * wpb) {
        int c = r / N, p = r - c * N;
        int t = BOS;
        if (p > 0) t = cfg_spin(ch.spins, N, ch.cfg_sample[c], ch.cfg_i[c], ch.cfg_j[c], p - 1) & 1;
        if (reuse) {
            if (lane == 0) uid0[r] = p * 3 + t;
        } else {
            if (lane == 0) uid0[r] = r;
            for (int k = lane; k < d; k += 32)
                X0[(size_t)r * d + k] = tok_emb[(size_t)t * d + k] + pos_emb[(size_t)p * d + k];
        }
    }
    if (reuse && blockIdx.x == 0 && threadIdx.x == 0) ch.counters[CNT_U0] = 3 * N;
    if (!reuse && blockIdx.x == 0 && threadIdx.x == 0) ch.counters[CNT_U0] = R;
}

// ---- head: log P(. | s_<p) = log_softmax(LN_f(x) W_head + b_head) ----------------
__global__ void k_head(const float* __restrict__ X, const int* __restrict__ counters, int u_slot,
                       const float* __restrict__ g, const float* __restrict__ bta, const float* __restrict__ w,
                       const float* __restrict__ bh, int d, float* __restrict__ logp) {
    const int U = counters[u_slot];
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int u = blockIdx.x * wpb + (threadIdx.x >> 5); u < U; u += gridDim.x * wpb) {
        const float* x = X + (size_t)u * d;
        float s = 0.f;
        for (int k = lane; k < d; k += 32) s += x[k];
        float mu = warp_sum(s) / d;
        float v = 0.f;
        for (int k = lane; k < d; k += 32) { float t = x[k] - mu; v += t * t; }
        float rstd = rsqrtf(warp_sum(v) / d + LN_EPS);
        float z0 = 0.f, z1 = 0.f;
        for (int k = lane; k < d; k += 32) {
            float a = (x[k] - mu) * rstd * g[k] + bta[k];
            z0 += a * w[2 * k];
            z1 += a * w[2 * k + 1];
        }
        z0 = warp_sum(z0) + bh[0];
        z1 = warp_sum(z1) + bh[1];
        if (lane == 0) {
            float m = fmaxf(z0, z1);
            float lse = m + logf(expf(z0 - m) + expf(z1 - m));
            logp[2 * (size_t)u] = z0 - lse;
            logp[2 * (size_t)u + 1] = z1 - lse;
        }
    }
}

// ---- log-ratio per configuration ------------------------------------------------
// Delta_c = 1/2 sum_p [log P(s'_p | row of c at p) - log P(s_p | row of the sample at p)],
// summed term by term so that positions whose rows agree contribute exact zeros.
__global__ void k_eloc_ratio(Chunk ch, const int* __restrict__ uid, const float* __restrict__ logp,
                             float* __restrict__ ratio, float* __restrict__ log_psi_out) {
    const int N = ch.N;
    const int C = ch.counters[CNT_C];
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < C; c += gridDim.x * wpb) {
        int b = ch.cfg_sample[c], ci = ch.cfg_i[c], cj = ch.cfg_j[c];
        int base = ch.cfg_off[b];
        const uint8_t* s = ch.spins + (size_t)b * N;
        float acc = 0.f;
        if (ci < 0) {
            for (int p = lane; p < N; p += 32) acc += logp[2 * (size_t)uid[(size_t)c * N + p] + (s[p] & 1)];
            acc = warp_sum(acc);
            if (lane == 0) {
                ratio[c] = 0.f;
                if (log_psi_out) log_psi_out[b] = 0.5f * acc;
            }
        } else {
            for (int p = lane; p < N; p += 32) {
                int sp = s[p] & 1;
                int spc = (p == ci) ? (s[cj] & 1) : (p == cj) ? (s[ci] & 1) : sp;
                acc += logp[2 * (size_t)uid[(size_t)c * N + p] + spc] - logp[2 * (size_t)uid[(size_t)base * N + p] + sp];
            }
            acc = warp_sum(acc);
            if (lane == 0) ratio[c] = expf(0.5f * acc);
        }
    }
}

// E_loc(s) = (J/4) sum_b sigma_i sigma_j - (J/2) sum_c psi(s^c)/psi(s); one warp per sample.
__global__ void k_eloc_reduce(Chunk ch, const float* __restrict__ diag, const float* __restrict__ ratio, float J,
                              float* __restrict__ e_loc) {
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < ch.S; b += gridDim.x * wpb) {
        int c0 = ch.cfg_off[b] + 1, c1 = ch.cfg_off[b + 1];
        float acc = 0.f;
        for (int c = c0 + lane; c < c1; c += 32) acc += ratio[c];
        acc = warp_sum(acc);
        if (lane == 0) e_loc[b] = diag[b] - 0.5f * J * acc;
    }
}

// FP64 mean and variance (1/B) of the local energies; one block, fixed order.
__global__ void k_mean_var(const float* __restrict__ e, int B, double* __restrict__ mv) {
    __shared__ double s_w[32];
    __shared__ double s_mean;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    double a = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) a += (double)e[i];
    a = warp_sum_d(a);
    if (lane == 0) s_w[w] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += s_w[i];
        s_mean = B > 0 ? t / B : 0.0;
    }
    __syncthreads();
    double m = s_mean;
    double v = 0.0;
    for (int i = threadIdx.x; i < B; i += blockDim.x) { double t = (double)e[i] - m; v += t * t; }
    v = warp_sum_d(v);
    __syncthreads();
    if (lane == 0) s_w[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < nw; ++i) t += s_w[i];
        mv[0] = m;
        mv[1] = B > 0 ? t / B : 0.0;
    }
}

__global__ void k_accumulate_stats(const int* __restrict__ counters, int layers, int S, long long* __restrict__ st) {
    if (threadIdx.x == 0) {
        st[ST_SAMPLES] += S;
        st[ST_CONFIGS] += counters[CNT_C];
        st[ST_ROWS] += (long long)counters[CNT_R];
    }
    for (int l = threadIdx.x; l <= layers; l += blockDim.x) st[ST_U0 + l] += counters[CNT_U0 + l];
}

// ---- launchers -----------------------------------------------------------------
cudaError_t launch_count_configs(const uint8_t* spins, int S, int N, const int* bonds, int nb, float J,
                                 int with_bonds, int* cnt, float* diag, int* status, cudaStream_t st, int grid) {
    k_count_configs<<<grid, 256, 0, st>>>(spins, S, N, bonds, nb, J, with_bonds, cnt, diag, status);
    return cudaGetLastError();
}
cudaError_t launch_scan_configs(const int* cnt, int S, int* cfg_off, int* counters, int N, cudaStream_t st) {
    k_scan_configs<<<1, 1024, 0, st>>>(cnt, S, cfg_off, counters, N);
    return cudaGetLastError();
}
cudaError_t launch_fill_configs(const uint8_t* spins, int S, int N, const int* bonds, int nb, int with_bonds,
                                const int* cfg_off, int* cfg_sample, int* cfg_i, int* cfg_j, cudaStream_t st,
                                int grid) {
    k_fill_configs<<<grid, 256, 0, st>>>(spins, S, N, bonds, nb, with_bonds, cfg_off, cfg_sample, cfg_i, cfg_j);
    return cudaGetLastError();
}
cudaError_t launch_embed(const Chunk& ch, const float* tok_emb, const float* pos_emb, int reuse, float* X0,
                         int* uid0, cudaStream_t st, int grid) {
    if (reuse) {
        k_embed_table<<<grid, 256, 0, st>>>(tok_emb, pos_emb, ch.N, ch.d, X0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_embed_rows<<<grid, 256, 0, st>>>(ch, tok_emb, pos_emb, reuse, X0, uid0);
    return cudaGetLastError();
}
cudaError_t launch_active_rows(const Chunk& ch, int prefix_reuse, int* act_cnt, int* act_off, int* act_rows,
                               cudaStream_t st, int grid) {
    k_active_count<<<grid, 256, 0, st>>>(ch, prefix_reuse, act_cnt);
    k_active_scan<<<1, 1024, 0, st>>>(ch, act_cnt, act_off);
    k_active_fill<<<grid, 256, 0, st>>>(ch, prefix_reuse, act_off, act_rows);
    return cudaGetLastError();
}
cudaError_t launch_head(const float* X, const int* counters, int u_slot, const float* g, const float* b,
                        const float* w_head, const float* b_head, int d, float* logp, cudaStream_t st, int grid) {
    k_head<<<grid, 256, 0, st>>>(X, counters, u_slot, g, b, w_head, b_head, d, logp);
    return cudaGetLastError();
}
cudaError_t launch_eloc(const Chunk& ch, const int* uid, const float* logp, float* ratio, float* log_psi_out,
                        cudaStream_t st, int grid) {
    k_eloc_ratio<<<grid, 256, 0, st>>>(ch, uid, logp, ratio, log_psi_out);
    return cudaGetLastError();
}
cudaError_t launch_eloc_reduce(const Chunk& ch, const float* diag, const float* ratio, float J, float* e_loc_out,
                               cudaStream_t st, int grid) {
    k_eloc_reduce<<<grid, 256, 0, st>>>(ch, diag, ratio, J, e_loc_out);
    return cudaGetLastError();
}
cudaError_t launch_mean_var(const float* e_loc, int B, double* mean_var, cudaStream_t st) {
    k_mean_var<<<1, 1024, 0, st>>>(e_loc, B, mean_var);
    return cudaGetLastError();
}
cudaError_t launch_accumulate_stats(const int* counters, int layers, int S, long long* stats, cudaStream_t st) {
    k_accumulate_stats<<<1, 128, 0, st>>>(counters, layers, S, stats);
    return cudaGetLastError();
}

}  // namespace vq
