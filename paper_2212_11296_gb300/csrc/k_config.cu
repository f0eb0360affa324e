// Connected-configuration enumeration, embedding, head and the local-energy
// assembly (Sec. 2 Eq. local-energy; Sec. 4 Heisenberg model, Marshall sign).
#include "vqnqs_internal.cuh"

namespace vq {

// ---- bonds: diagonal energy and connected-configuration count per sample -----------
// Sec. 4 Heisenberg model, H = J sum_<ij> S_i.S_j: in the Marshall-rotated S^z
// basis a bond gives (J/4) sigma_i sigma_j on the diagonal and -J/2 to the
// configuration with the two spins exchanged when they differ (Sec. 2: a
// k-local term touches only its own sites).  Sec. 4 transverse-field Ising
// chain, H = -J sum sigma^z sigma^z - Gamma sum sigma^x: -J sigma_i sigma_j per
// bond on the diagonal, -Gamma to each of the N single flips (Sec. 2).
__global__ void k_count_configs(Chunk ch, float diag_coef, int with_bonds, int* __restrict__ cnt,
                                float* __restrict__ diag, int* __restrict__ status) {
    __shared__ int s_red[2][32];
    for (int b = blockIdx.x; b < ch.S; b += gridDim.x) {
        const int g = sample_group(ch, b);
        const int N = ch.g.N[g], nb = ch.g.nb[g];
        const int* bonds = ch.bonds + 2 * ch.g.bond_off[g];
        const uint8_t* s = sample_spins(ch, b);
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
            cnt[b] = (ch.model == MODEL_TFIM_CHAIN && with_bonds) ? N : a;
            diag[b] = diag_coef * (float)z;
        }
        __syncthreads();
    }
}

// One-block exclusive scan of v(i) for i < n; writes off[0..n] and returns the total in *total.
template <typename F>
__device__ void block_exclusive_scan(int n, F v_of, int* __restrict__ off, int* __restrict__ total) {
    __shared__ int s_warp[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const int v = (i < n) ? v_of(i) : 0;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            const int nw = blockDim.x >> 5;
            int t = (lane < nw) ? s_warp[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            if (lane < nw) s_warp[lane] = t;
        }
        __syncthreads();
        const int incl = x + (w > 0 ? s_warp[w - 1] : 0) + s_carry;
        if (i < n) off[i] = incl - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = incl;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[n] = s_carry;
        *total = s_carry;
    }
}

// First configuration of each sample: exclusive scan of (1 + anti-aligned count).
__global__ void k_scan_configs(Chunk ch, const int* __restrict__ cnt, int* __restrict__ cfg_off) {
    block_exclusive_scan(ch.S, [&](int i) { return 1 + cnt[i]; }, cfg_off, &ch.counters[CNT_C]);
}

// Writes the sample itself, then its anti-aligned bonds in bond order.
__global__ void k_fill_configs(Chunk ch, int with_bonds, int* __restrict__ cfg_sample, int* __restrict__ cfg_i,
                               int* __restrict__ cfg_j) {
    __shared__ int s_warp[32];
    for (int b = blockIdx.x; b < ch.S; b += gridDim.x) {
        const int g = sample_group(ch, b);
        const int nb = ch.g.nb[g];
        const int* bonds = ch.bonds + 2 * ch.g.bond_off[g];
        const uint8_t* s = sample_spins(ch, b);
        const int off = ch.cfg_off[b];
        if (threadIdx.x == 0) { cfg_sample[off] = b; cfg_i[off] = -1; cfg_j[off] = -1; }
        if (!with_bonds) continue;
        if (ch.model == MODEL_TFIM_CHAIN) {  // every single flip, in site order
            for (int q = threadIdx.x; q < ch.g.N[g]; q += blockDim.x) {
                cfg_sample[off + 1 + q] = b;
                cfg_i[off + 1 + q] = q;
                cfg_j[off + 1 + q] = CFG_FLIP;
            }
            continue;
        }
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

// First row of each configuration (exclusive scan of its number of sites); total -> CNT_R.
__global__ void k_scan_rows(Chunk ch, int* __restrict__ cfg_row) {
    block_exclusive_scan(ch.counters[CNT_C], [&](int c) { return cfg_N(ch, c); }, cfg_row, &ch.counters[CNT_R]);
}

__global__ void k_fill_row_cfg(Chunk ch, int* __restrict__ row_cfg) {
    const int C = ch.counters[CNT_C];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < C; c += gridDim.x * wpb) {
        const int r0 = ch.cfg_row[c], r1 = ch.cfg_row[c + 1];
        for (int r = r0 + lane; r < r1; r += 32) row_cfg[r] = c;
    }
}

// ---- active rows -------------------------------------------------------------------
__global__ void k_active_count(Chunk ch, int prefix_reuse, int* __restrict__ act_cnt, long long* __restrict__ stats) {
    const int C = ch.counters[CNT_C];
    long long rows = 0, pairs = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < C; c += gridDim.x * blockDim.x) {
        const int N = cfg_N(ch, c);
        const long long p0 = prefix_reuse ? cfg_p0(ch, c) : 0;
        act_cnt[c] = N - (int)p0;
        rows += N - p0;
        pairs += ((long long)N * (N + 1) - p0 * (p0 + 1)) / 2;  // sum over active rows p of (p + 1) keys
    }
    for (int o = 16; o > 0; o >>= 1) {
        rows += __shfl_xor_sync(0xffffffffu, rows, o);
        pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    }
    if ((threadIdx.x & 31) == 0 && (rows || pairs)) {
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_ACTIVE]), (unsigned long long)rows);
        atomicAdd(reinterpret_cast<unsigned long long*>(&stats[ST_PAIRS]), (unsigned long long)pairs);
    }
}

// Exclusive scan of act_cnt over the chunk's configurations (one block); total -> CNT_A.
__global__ void k_active_scan(Chunk ch, const int* __restrict__ act_cnt, int* __restrict__ act_off) {
    block_exclusive_scan(ch.counters[CNT_C], [&](int i) { return act_cnt[i]; }, act_off, &ch.counters[CNT_A]);
}

// One warp per configuration writes its active rows (ascending).
__global__ void k_active_fill(Chunk ch, int prefix_reuse, const int* __restrict__ act_off,
                              int* __restrict__ act_rows) {
    const int C = ch.counters[CNT_C];
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < C; c += gridDim.x * wpb) {
        const int p0 = prefix_reuse ? cfg_p0(ch, c) : 0;
        const int off = act_off[c], r0 = ch.cfg_row[c], N = cfg_N(ch, c);
        for (int p = p0 + lane; p < N; p += 32) act_rows[off + p - p0] = r0 + p;
    }
}

// ---- embedding: x0 = tok_emb[token] + pos_emb[p], token = s_{p-1} (BOS at p = 0) --------
// With tokens of G spins the token at position p is the value of group p - 1,
// sum_k s[(p-1) G + k] 2^k, and BOS = 2^G: V = 2^G + 1 token values (3 for G = 1).
// reuse: rows are keyed by (p, token) -> uid p * V + token, table of V N rows.
// full:  every (config, position) row gets its own copy.
__global__ void k_embed_table(const float* __restrict__ tok_emb, const float* __restrict__ pos_emb, int N, int d,
                              int V, float* __restrict__ X0) {
    size_t total = (size_t)V * N * d;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        int k = (int)(e % d);
        int u = (int)(e / d);
        int p = u / V, t = u % V;
        X0[e] = tok_emb[(size_t)t * d + k] + pos_emb[(size_t)p * d + k];
    }
}

// value of the spin group at position p of configuration c (G spins, bit k = spin k)
__device__ __forceinline__ int cfg_group(const Chunk& ch, const uint8_t* s, int c, int p) {
    int v = 0;
    for (int k = 0; k < ch.G; ++k) v |= cfg_spin(s, ch.cfg_i[c], ch.cfg_j[c], p * ch.G + k) << k;
    return v;
}

__global__ void k_embed_rows(Chunk ch, const float* __restrict__ tok_emb, const float* __restrict__ pos_emb,
                             int reuse, float* __restrict__ X0, int* __restrict__ uid0) {
    const int N = ch.N, d = ch.d, V = (1 << ch.G) + 1;
    const int R = ch.counters[CNT_R];
    if (reuse) {  // row ids only: one thread per row
        for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
            const int c = ch.row_cfg[r], p = r - ch.cfg_row[c];
            int t = ch.G == 1 ? BOS : (1 << ch.G);
            if (p > 0) t = cfg_group(ch, sample_spins(ch, ch.cfg_sample[c]), c, p - 1);
            uid0[r] = p * V + t;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) ch.counters[CNT_U0] = V * N;
        return;
    }
    // one warp per row
    int lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    for (int r = blockIdx.x * wpb + (threadIdx.x >> 5); r < R; r += gridDim.x * wpb) {
        const int c = ch.row_cfg[r], p = r - ch.cfg_row[c];
        int t = ch.G == 1 ? BOS : (1 << ch.G);
        if (p > 0) t = cfg_group(ch, sample_spins(ch, ch.cfg_sample[c]), c, p - 1);
        if (reuse) {
            if (lane == 0) uid0[r] = p * V + t;
        } else {
            if (lane == 0) uid0[r] = r;
            for (int k = lane; k < d; k += 32)
                X0[(size_t)r * d + k] = tok_emb[(size_t)t * d + k] + pos_emb[(size_t)p * d + k];
        }
    }
    if (reuse && blockIdx.x == 0 && threadIdx.x == 0) ch.counters[CNT_U0] = V * N;
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

// The head of tokens of G spins: V = 2^G logits (W_head [d][V]), log-softmax.
template <int V>
__global__ void k_head_groups(const float* __restrict__ X, const int* __restrict__ counters, int u_slot,
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
        float z[V];
#pragma unroll
        for (int j = 0; j < V; ++j) z[j] = 0.f;
        for (int k = lane; k < d; k += 32) {
            const float a = (x[k] - mu) * rstd * g[k] + bta[k];
#pragma unroll
            for (int j = 0; j < V; ++j) z[j] += a * w[(size_t)V * k + j];
        }
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            z[j] = warp_sum(z[j]) + bh[j];
            m = fmaxf(m, z[j]);
        }
        float se = 0.f;
#pragma unroll
        for (int j = 0; j < V; ++j) se += expf(z[j] - m);
        const float lse = m + logf(se);
        if (lane < V) {
            float zl = 0.f;
#pragma unroll
            for (int j = 0; j < V; ++j) zl = j == lane ? z[j] : zl;
            logp[(size_t)V * u + lane] = zl - lse;
        }
    }
}

// ---- log-ratio per configuration ------------------------------------------------
// Delta_c = 1/2 sum_p [log P(s'_p | row of c at p) - log P(s_p | row of the sample at p)],
// summed term by term so that positions whose rows agree contribute exact zeros.
__global__ void k_eloc_ratio(Chunk ch, const int* __restrict__ uid, const float* __restrict__ logp,
                             float* __restrict__ ratio, float* __restrict__ log_psi_out) {
    const int C = ch.counters[CNT_C];
    const int V = 1 << ch.G;  // values of a token's spin group (2 for single spins)
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < C; c += gridDim.x * wpb) {
        const int b = ch.cfg_sample[c], ci = ch.cfg_i[c];
        const int N = sample_N(ch, b);
        const int* urow = uid + ch.cfg_row[c];
        const int* ubase = uid + ch.cfg_row[ch.cfg_off[b]];
        const uint8_t* s = sample_spins(ch, b);
        float acc = 0.f;
        if (ci < 0) {
            for (int p = lane; p < N; p += 32) acc += logp[(size_t)V * urow[p] + cfg_group(ch, s, c, p)];
            acc = warp_sum(acc);
            if (lane == 0) {
                ratio[c] = 0.f;
                if (log_psi_out) log_psi_out[b] = 0.5f * acc;
            }
        } else {
            const int cs = ch.cfg_off[b];  // the sample's own configuration
            for (int p = lane; p < N; p += 32) {
                const int vc = cfg_group(ch, s, c, p), vs = cfg_group(ch, s, cs, p);
                acc += logp[(size_t)V * urow[p] + vc] - logp[(size_t)V * ubase[p] + vs];
            }
            acc = warp_sum(acc);
            if (lane == 0) ratio[c] = expf(0.5f * acc);
        }
    }
}

// E_loc(s) = (J/4) sum_b sigma_i sigma_j - (J/2) sum_c psi(s^c)/psi(s); one warp per sample.
__global__ void k_eloc_reduce(Chunk ch, const float* __restrict__ diag, const float* __restrict__ ratio, float offdiag,
                              float* __restrict__ e_loc) {
    int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int b = blockIdx.x * wpb + (threadIdx.x >> 5); b < ch.S; b += gridDim.x * wpb) {
        int c0 = ch.cfg_off[b] + 1, c1 = ch.cfg_off[b + 1];
        float acc = 0.f;
        for (int c = c0 + lane; c < c1; c += 32) acc += ratio[c];
        acc = warp_sum(acc);
        if (lane == 0) e_loc[b] = diag[b] + offdiag * acc;
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
cudaError_t launch_configs(const Chunk& ch, float diag_coef, int with_bonds, int* cnt, float* diag, int* cfg_off,
                           int* cfg_sample, int* cfg_i, int* cfg_j, int* cfg_row, int* row_cfg, int* status,
                           cudaStream_t st, int grid) {
    k_count_configs<<<grid, 256, 0, st>>>(ch, diag_coef, with_bonds, cnt, diag, status);
    k_scan_configs<<<1, 1024, 0, st>>>(ch, cnt, cfg_off);
    k_fill_configs<<<grid, 256, 0, st>>>(ch, with_bonds, cfg_sample, cfg_i, cfg_j);
    k_scan_rows<<<1, 1024, 0, st>>>(ch, cfg_row);
    k_fill_row_cfg<<<grid * 4, 256, 0, st>>>(ch, row_cfg);
    return cudaGetLastError();
}
cudaError_t launch_embed(const Chunk& ch, const float* tok_emb, const float* pos_emb, int reuse, float* X0,
                         int* uid0, cudaStream_t st, int grid) {
    if (reuse) {
        k_embed_table<<<grid, 256, 0, st>>>(tok_emb, pos_emb, ch.N, ch.d, (1 << ch.G) + 1, X0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_embed_rows<<<grid, 256, 0, st>>>(ch, tok_emb, pos_emb, reuse, X0, uid0);
    return cudaGetLastError();
}
// out[(b * layers + l) * N + p] = code of row (configuration b, position p); here every
// configuration is a sample and every row is computed.
__global__ void k_copy_codes(Chunk ch, const int* __restrict__ code, int l, int layers, int* __restrict__ out) {
    const int R = ch.counters[CNT_R], N = ch.N;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const int b = ch.row_cfg[r], p = r - ch.cfg_row[b];
        out[((size_t)b * layers + l) * N + p] = code[r];
    }
}

cudaError_t launch_copy_codes(const Chunk& ch, const int* code, int l, int layers, int* out, cudaStream_t st,
                              int grid) {
    k_copy_codes<<<grid, 256, 0, st>>>(ch, code, l, layers, out);
    return cudaGetLastError();
}

// out[((b * per_sample + k) * layers + l) * N + p] = code of position p of configuration k of
// chunk sample b (k = 0: the sample, k >= 1: its connected configurations in enumeration
// order); a row before its configuration's first changed position takes the sample's code
// at that position (the same computation on the same inputs, not recomputed).
__global__ void k_copy_cfg_codes(Chunk ch, const int* __restrict__ code, int l, int layers, int per_sample,
                                 int* __restrict__ out) {
    const int R = ch.counters[CNT_R], N = ch.N;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        const int c = ch.row_cfg[r], p = r - ch.cfg_row[c];
        const int b = ch.cfg_sample[c], k = c - ch.cfg_off[b];
        const int v = p < cfg_p0(ch, c) ? code[ch.cfg_row[ch.cfg_off[b]] + p] : code[r];
        out[(((size_t)b * per_sample + k) * layers + l) * N + p] = v;
    }
}

cudaError_t launch_copy_cfg_codes(const Chunk& ch, const int* code, int l, int layers, int per_sample, int* out,
                                  cudaStream_t st, int grid) {
    k_copy_cfg_codes<<<grid, 256, 0, st>>>(ch, code, l, layers, per_sample, out);
    return cudaGetLastError();
}

cudaError_t launch_active_rows(const Chunk& ch, int prefix_reuse, int* act_cnt, int* act_off, int* act_rows,
                               long long* stats, cudaStream_t st, int grid) {
    k_active_count<<<grid, 256, 0, st>>>(ch, prefix_reuse, act_cnt, stats);
    k_active_scan<<<1, 1024, 0, st>>>(ch, act_cnt, act_off);
    k_active_fill<<<grid, 256, 0, st>>>(ch, prefix_reuse, act_off, act_rows);
    return cudaGetLastError();
}
cudaError_t launch_head(const float* X, const int* counters, int u_slot, const float* g, const float* b,
                        const float* w_head, const float* b_head, int d, float* logp, cudaStream_t st, int grid,
                        int G) {
    switch (G) {
        case 1: k_head<<<grid, 256, 0, st>>>(X, counters, u_slot, g, b, w_head, b_head, d, logp); break;
        case 2: k_head_groups<4><<<grid, 256, 0, st>>>(X, counters, u_slot, g, b, w_head, b_head, d, logp); break;
        case 4: k_head_groups<16><<<grid, 256, 0, st>>>(X, counters, u_slot, g, b, w_head, b_head, d, logp); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
// ---- final half-block (Table 1's networks): attention and W_o, no quantizer ------------
// Its outputs are not quantized, so every active row is its own row from here on.
__global__ void k_half_gather(const int* __restrict__ counters, const int* __restrict__ act_rows,
                              const int* __restrict__ uid, const float* __restrict__ O, const float* __restrict__ X,
                              int d, float* __restrict__ G_o, __nv_bfloat16* __restrict__ G_o16,
                              float* __restrict__ G_x) {
    const int A = counters[CNT_A];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int a = blockIdx.x * wpb + (threadIdx.x >> 5); a < A; a += gridDim.x * wpb) {
        const int row = act_rows[a];
        const float* o = O + (size_t)row * d;
        const float* x = X + (size_t)uid[row] * d;
        for (int k = lane * 4; k < d; k += 128) {
            const float4 ov = *reinterpret_cast<const float4*>(o + k);
            *reinterpret_cast<float4*>(G_x + (size_t)a * d + k) = *reinterpret_cast<const float4*>(x + k);
            if (G_o) *reinterpret_cast<float4*>(G_o + (size_t)a * d + k) = ov;
            if (G_o16) {
                const __nv_bfloat162 h0 = __floats2bfloat162_rn(ov.x, ov.y), h1 = __floats2bfloat162_rn(ov.z, ov.w);
                uint2 u;
                u.x = *reinterpret_cast<const uint32_t*>(&h0);
                u.y = *reinterpret_cast<const uint32_t*>(&h1);
                *reinterpret_cast<uint2*>(G_o16 + (size_t)a * d + k) = u;
            }
        }
    }
}

// Row ids after the half-block: position p of configuration c is its active row
// act_off[c] + p - p0, or the sample's active row act_off[cfg_off[b]] + p before p0.
__global__ void k_half_ids(Chunk ch, int prefix_reuse, const int* __restrict__ act_off, int* __restrict__ uid_out) {
    const int C = ch.counters[CNT_C];
    const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    for (int c = blockIdx.x * wpb + (threadIdx.x >> 5); c < C; c += gridDim.x * wpb) {
        const int b = ch.cfg_sample[c];
        const int p0 = prefix_reuse ? cfg_p0(ch, c) : 0;
        const int N = cfg_N(ch, c), r0 = ch.cfg_row[c];
        const int own = act_off[c], base = act_off[ch.cfg_off[b]];
        for (int p = lane; p < N; p += 32) uid_out[r0 + p] = p >= p0 ? own + p - p0 : base + p;
    }
}

cudaError_t launch_half_gather(const int* counters, const int* act_rows, const int* uid, const float* O,
                               const float* X, int d, float* G_o, __nv_bfloat16* G_o16, float* G_x, cudaStream_t st,
                               int grid) {
    if (d % 4) return cudaErrorInvalidValue;
    k_half_gather<<<grid, 256, 0, st>>>(counters, act_rows, uid, O, X, d, G_o, G_o16, G_x);
    return cudaGetLastError();
}
cudaError_t launch_half_ids(const Chunk& ch, int prefix_reuse, const int* act_off, int* uid_out, cudaStream_t st,
                            int grid) {
    k_half_ids<<<grid, 256, 0, st>>>(ch, prefix_reuse, act_off, uid_out);
    return cudaGetLastError();
}

cudaError_t launch_eloc(const Chunk& ch, const int* uid, const float* logp, float* ratio, float* log_psi_out,
                        cudaStream_t st, int grid) {
    k_eloc_ratio<<<grid, 256, 0, st>>>(ch, uid, logp, ratio, log_psi_out);
    return cudaGetLastError();
}
cudaError_t launch_eloc_reduce(const Chunk& ch, const float* diag, const float* ratio, float offdiag,
                               float* e_loc_out, cudaStream_t st, int grid) {
    k_eloc_reduce<<<grid, 256, 0, st>>>(ch, diag, ratio, offdiag, e_loc_out);
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
