// Compressed (I, V) representation of the hidden states (Sec. 3.2).
//
// After the quantizer of layer l, the input of every per-location operation of
// that layer is fixed by the pair (row id at layer l, codeword index): the
// residual stream x_l is a function of the row id and the quantized vector of
// the codeword.  Rows with equal pairs therefore share one new row id, and the
// per-location work runs once per id.  The table is an open-addressing hash
// (linear probing, load <= 1/2) over 64-bit keys; the thread whose CAS claims
// a slot takes a fresh id with atomicAdd and records the representative pair.
// A second pass looks every row's key up.  Probes are bounded by the table
// size; running past the bound sets VQNQS_DEV_HASH_OVERFLOW and leaves the row
// on id 0 instead of spinning.
//
// With reuse off, every row keeps its own id (the plain full recompute).
#include "vqnqs_internal.cuh"

namespace vq {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}

__device__ __forceinline__ unsigned long long make_key(int uid, int code) {
    // row id in the high word, the (packed) code in the low one; 0 = empty slot
    return ((((unsigned long long)(unsigned)uid) << 32) | (unsigned)code) + 1ULL;
}

__global__ void k_hash_clear(unsigned long long* __restrict__ keys, size_t H, int* __restrict__ counters,
                             int u_slot_next) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < H; i += (size_t)gridDim.x * blockDim.x)
        keys[i] = 0ULL;
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[u_slot_next] = 0;
}

// Code of row r: its own, or (before its configuration's first changed position)
// the code of the same position in the sample's own configuration, which is
// the same computation on the same inputs.
__device__ __forceinline__ int row_code(const Chunk& ch, const int* __restrict__ code, int r) {
    const int c = ch.row_cfg[r], p = r - ch.cfg_row[c];
    if (p < cfg_p0(ch, c)) return code[ch.cfg_row[ch.cfg_off[ch.cfg_sample[c]]] + p];
    return code[r];
}

// Inserts key; the thread that claims the slot takes the next id from *counter
// and records the representative pair.  Returns false when the probe bound ran out.
__device__ __forceinline__ bool hash_insert(unsigned long long* __restrict__ keys, int* __restrict__ vals,
                                            unsigned long long mask, int u, int c, int* __restrict__ counter,
                                            int* __restrict__ rep_uid, int* __restrict__ rep_code) {
    const unsigned long long key = make_key(u, c);
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long prev = atomicCAS(&keys[h], 0ULL, key);
        if (prev == 0ULL) {
            const int id = atomicAdd(counter, 1);
            vals[h] = id;
            rep_uid[id] = u;
            rep_code[id] = c;
            return true;
        }
        if (prev == key) return true;
        h = (h + 1) & mask;
    }
    return false;
}

// Id of an inserted key, or -1 when the probe bound ran out.
__device__ __forceinline__ int hash_lookup(const unsigned long long* __restrict__ keys, const int* __restrict__ vals,
                                           unsigned long long mask, int u, int c) {
    const unsigned long long key = make_key(u, c);
    unsigned long long h = mix64(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        const unsigned long long k = keys[h];
        if (k == key) return vals[h];
        if (k == 0ULL) return -1;
        h = (h + 1) & mask;
    }
    return -1;
}

__global__ void k_dedupe_insert(Chunk ch, const int* __restrict__ uid_cur, const int* __restrict__ code,
                                int u_slot_next, unsigned long long* __restrict__ keys,
                                int* __restrict__ vals, unsigned long long mask, int* __restrict__ rep_uid,
                                int* __restrict__ rep_code, int* __restrict__ status) {
    int* counters = ch.counters;
    const int R = counters[CNT_R];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
        if (!hash_insert(keys, vals, mask, uid_cur[r], row_code(ch, code, r), &counters[u_slot_next], rep_uid,
                         rep_code))
            atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
}

__global__ void k_dedupe_lookup(Chunk ch, const int* __restrict__ uid_cur, const int* __restrict__ code,
                                const unsigned long long* __restrict__ keys,
                                const int* __restrict__ vals, unsigned long long mask, int* __restrict__ uid_next,
                                int* __restrict__ status) {
    const int R = ch.counters[CNT_R];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        int id = hash_lookup(keys, vals, mask, uid_cur[r], row_code(ch, code, r));
        if (id < 0) {
            atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
            id = 0;
        }
        uid_next[r] = id;
    }
}

// ---- standalone (I, V) compression of R (row id, code) pairs --------------------
__global__ void k_pairs_insert(int R, const int* __restrict__ uid, const int* __restrict__ code,
                               unsigned long long* __restrict__ keys, int* __restrict__ vals, unsigned long long mask,
                               int* __restrict__ count, int* __restrict__ rep_uid, int* __restrict__ rep_code,
                               int* __restrict__ status) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
        if (!hash_insert(keys, vals, mask, uid[r], code[r], count, rep_uid, rep_code))
            atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
}

__global__ void k_pairs_lookup(int R, const int* __restrict__ uid, const int* __restrict__ code,
                               const unsigned long long* __restrict__ keys, const int* __restrict__ vals,
                               unsigned long long mask, int* __restrict__ new_id, int* __restrict__ status) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        int id = hash_lookup(keys, vals, mask, uid[r], code[r]);
        if (id < 0) {
            atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
            id = 0;
        }
        new_id[r] = id;
    }
}

// ---- two-word codes: a dense code id per distinct (hi, lo) pair ------------------
// Over the listed rows (act_rows[0 .. counters[a_slot])): insert every pair, then
// replace the row's lo word by the pair's id; tab_hi / tab_lo [id] give the words back.
__global__ void k_words_insert(const int* __restrict__ counters, int a_slot, const int* __restrict__ rows,
                               const int* __restrict__ lo, const int* __restrict__ hi,
                               unsigned long long* __restrict__ keys, int* __restrict__ vals, unsigned long long mask,
                               int* __restrict__ count, int* __restrict__ tab_hi, int* __restrict__ tab_lo,
                               int* __restrict__ status) {
    const int n = counters[a_slot];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = rows[i];
        if (!hash_insert(keys, vals, mask, hi[r], lo[r], count, tab_hi, tab_lo)) atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
    }
}
__global__ void k_words_lookup(const int* __restrict__ counters, int a_slot, const int* __restrict__ rows,
                               int* __restrict__ lo, const int* __restrict__ hi,
                               const unsigned long long* __restrict__ keys, const int* __restrict__ vals,
                               unsigned long long mask, int* __restrict__ status) {
    const int n = counters[a_slot];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int r = rows[i];
        int id = hash_lookup(keys, vals, mask, hi[r], lo[r]);
        if (id < 0) {
            atomicOr(status, VQNQS_DEV_HASH_OVERFLOW);
            id = 0;
        }
        lo[r] = id;
    }
}

cudaError_t launch_code_words(int* counters, int a_slot, int cnt_slot, const int* rows, int Rmax, int* lo,
                              const int* hi, unsigned long long* keys, int* vals, int hash_bits, int* tab_hi,
                              int* tab_lo, int* status, cudaStream_t st, int num_sms) {
    const size_t H = (size_t)1 << hash_bits;
    const unsigned long long mask = (unsigned long long)H - 1ULL;
    int grid = (Rmax + 255) / 256;
    if (grid > 8 * num_sms) grid = 8 * num_sms;
    if (grid < 1) grid = 1;
    k_hash_clear<<<8 * num_sms, 256, 0, st>>>(keys, H, counters, cnt_slot);
    k_words_insert<<<grid, 256, 0, st>>>(counters, a_slot, rows, lo, hi, keys, vals, mask, &counters[cnt_slot], tab_hi,
                                         tab_lo, status);
    k_words_lookup<<<grid, 256, 0, st>>>(counters, a_slot, rows, lo, hi, keys, vals, mask, status);
    return cudaGetLastError();
}

__global__ void k_identity_keys(const int* __restrict__ uid_cur, const int* __restrict__ code,
                                int* __restrict__ counters, int u_slot_next, int* __restrict__ uid_next,
                                int* __restrict__ rep_uid, int* __restrict__ rep_code) {
    const int R = counters[CNT_R];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
        uid_next[r] = r;
        rep_uid[r] = uid_cur[r];
        rep_code[r] = code[r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[u_slot_next] = R;
}

int compress_hash_bits(int R) {
    int hb = 4;
    while ((1LL << hb) < 2LL * R) ++hb;
    return hb;
}

cudaError_t launch_compress_pairs(int R, const int* uid, const int* code, int* new_id, int* rep_uid, int* rep_code,
                                  int* count, unsigned long long* keys, int* vals, int hash_bits, int* status,
                                  cudaStream_t st, int num_sms) {
    const size_t H = (size_t)1 << hash_bits;
    const unsigned long long mask = (unsigned long long)H - 1ULL;
    int grid = (R + 255) / 256;
    if (grid > 8 * num_sms) grid = 8 * num_sms;
    if (grid < 1) grid = 1;
    k_hash_clear<<<8 * num_sms, 256, 0, st>>>(keys, H, count, 0);
    k_pairs_insert<<<grid, 256, 0, st>>>(R, uid, code, keys, vals, mask, count, rep_uid, rep_code, status);
    k_pairs_lookup<<<grid, 256, 0, st>>>(R, uid, code, keys, vals, mask, new_id, status);
    return cudaGetLastError();
}

cudaError_t launch_dedupe(const Chunk& ch, const int* uid_cur, const int* code, int u_slot_next, int Rmax,
                          unsigned long long* keys, int* vals, int hash_bits, int* uid_next, int* rep_uid,
                          int* rep_code, int reuse, int* status, cudaStream_t st, int num_sms) {
    int* counters = ch.counters;
    int grid = (Rmax + 255) / 256;
    if (grid > 8 * num_sms) grid = 8 * num_sms;
    if (grid < 1) grid = 1;
    if (!reuse) {
        k_identity_keys<<<grid, 256, 0, st>>>(uid_cur, code, counters, u_slot_next, uid_next, rep_uid, rep_code);
        return cudaGetLastError();
    }
    const size_t H = (size_t)1 << hash_bits;
    const unsigned long long mask = (unsigned long long)H - 1ULL;
    k_hash_clear<<<8 * num_sms, 256, 0, st>>>(keys, H, counters, u_slot_next);
    k_dedupe_insert<<<grid, 256, 0, st>>>(ch, uid_cur, code, u_slot_next, keys, vals, mask, rep_uid, rep_code, status);
    k_dedupe_lookup<<<grid, 256, 0, st>>>(ch, uid_cur, code, keys, vals, mask, uid_next, status);
    return cudaGetLastError();
}

}  // namespace vq
